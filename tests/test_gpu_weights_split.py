"""Modified weights of the mixed-precision form, whose products are formed in
split precision (FP32 hi/lo pairs with exact FMA products, TwoSum over runs
of up to 256 particles, FP64 accumulation across runs), against the oracle's FP64
Eq. modified_weights.

Tolerance: each product carries about 2^-48 ~ 3.6e-15 relative error and each
chunk's run sum about the same relative to the sum of its terms, so the
max-norm relative error of a cluster's weights stays near 1e-14 for weights
of similar magnitude; the bound is 1e-12, as for the FP64 path.
"""
import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_02250_gb300 import build, kitc
    build.build()
    torch.cuda.set_device(0)
    return kitc


def dev(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, np.float64)).cuda()


def _maxrel(a, b):
    return float(np.abs(a - b).max() / max(np.abs(b).max(), 1e-300))


@pytest.mark.parametrize("n", [1, 4, 8, 12, 16])
@pytest.mark.parametrize("mode", [0, 1])
def test_mixed_weights_match_oracle(K, orc, n, mode):
    x, f = wl.plummer_with_background(9000, 150 + n)
    p = K.Params(theta=0.7, degree=n, leaf_size=300, eps=0.01, precision=K.MIXED, weights=mode)
    t = K.kitc_build_tree(dev(x), p)
    K.kitc_modified_weights(t, dev(f))
    got = t.weights()
    t.free()
    ref = orc.Tree(x, 300).modified_weights(f, n)
    errs = [_maxrel(got[c], ref[c]) for c in range(len(ref))]
    assert max(errs) <= TOL, max(errs)


def test_mixed_weights_degree_map(K, orc):
    x, f = wl.uniform_cube(12000, 160)
    p = K.Params(theta=0.7, degree=6, leaf_size=300, eps=0.01, precision=K.MIXED)
    t = K.kitc_build_tree(dev(x), p)
    deg = np.random.default_rng(161).integers(0, 13, t.stats()["n_clusters"]).astype(np.int32)
    K.kitc_set_degrees(t, deg)
    K.kitc_modified_weights(t, dev(f))
    got = t.weights()
    t.free()
    ref, foff = orc.Tree(x, 300).modified_weights_var(f, deg)
    for c in np.nonzero(deg)[0]:
        k = (int(deg[c]) + 1) ** 3 * 3
        assert _maxrel(got[foff[c]:foff[c] + k], ref[foff[c]:foff[c] + k]) <= TOL, c


def test_weights_of_large_and_small_magnitude(K, orc):
    """Weights spanning 1e-20..1e20 keep their relative accuracy (the FP32 pairs
    carry the exponent range of FP32)."""
    x, f = wl.uniform_cube(4000, 162)
    f = f * np.array([1e20, 1.0, 1e-20])
    p = K.Params(theta=0.7, degree=5, leaf_size=250, eps=0.01, precision=K.MIXED)
    t = K.kitc_build_tree(dev(x), p)
    K.kitc_modified_weights(t, dev(f))
    got = t.weights()
    t.free()
    ref = orc.Tree(x, 250).modified_weights(f, 5)
    for q in range(3):
        assert _maxrel(got[..., q], ref[..., q]) <= TOL, q


@pytest.mark.parametrize("n", [4, 5])
def test_basis_at_and_near_grid_points(K, orc, n):
    """One leaf whose box is exactly [0, 1]^3 (corner particles): particles on
    grid points (0, 1/2 for even n, 1; Eq. Barycentric-1D's coincident case),
    within 1e-25 and 1e-30 of the grid point 0 (taken as coinciding by the
    FP32-pair basis, |q| <= 2^-60; by the oracle evaluated, L = 1 within 1e-25),
    and a slab of particles on one plane of a flat second leaf's box."""
    g = wl.rng(163)
    x = g.uniform(0.0, 1.0, size=(1500, 3))
    special = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [0.0, 0.5, 1.0], [1e-25, 0.5, 1e-30],
                        [0.5, 1e-22, 0.5], [1.0, 1e-25, 0.0]])
    x = np.vstack([special, x])
    f = g.uniform(-1.0, 1.0, size=(len(x), 3))
    p = K.Params(theta=0.7, degree=n, leaf_size=len(x), eps=0.01, precision=K.MIXED)
    t = K.kitc_build_tree(dev(x), p)
    assert t.stats()["n_clusters"] == 1
    K.kitc_modified_weights(t, dev(f))
    got = t.weights()
    t.free()
    ref = orc.Tree(x, len(x)).modified_weights(f, n)
    assert _maxrel(got[0], ref[0]) <= TOL
    # a flat axis: every z equal, so every grid point of that axis coincides
    # (the last one is taken, reading R9)
    xs = x.copy()
    xs[:, 2] = 0.3
    t = K.kitc_build_tree(dev(xs), p)
    K.kitc_modified_weights(t, dev(f))
    got = t.weights()
    t.free()
    ref = orc.Tree(xs, len(xs)).modified_weights(f, n)
    assert _maxrel(got[0], ref[0]) <= TOL
