"""GPU parity of every step of the hot path against the FP64 CPU oracle,
through the C ABI.

Tolerances: integer work (tree order, boxes, list entries, interaction
counts) must be bit-exact; FP64 results must agree to a relative L2 error of
1e-12; the mixed form (FP32 kernel values, FP64 sums) is held to
MIXED_TOL, derived from FP32 rounding: a pair's value
carries a few units of 2^-24 ~ 6e-8 of relative error, and sums over runs of
<= 8 terms, three levels deep, add about sqrt(3 * 4) units more, so the
relative L2 error of u sits near 3e-7; the bound keeps a factor ~3 margin.
"""
import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

from mixed_parity import check_mixed

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-6
ST, RO, SR, POLY = 0, 1, 2, 99


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


def gpu_treecode(K, x, f, tgt=None, **kw):
    p = K.Params(**kw)
    out, st = K.treecode(dev(x), dev(f), p, None if tgt is None else dev(tgt))
    return out.cpu().numpy(), st


# --------------------------------------------------------------------- tree
TREE_CASES = {
    "uniform": lambda: (wl.uniform_cube(20000, 31)[0], 150),
    "slab": lambda: (np.column_stack([np.random.default_rng(1).uniform(0, 16, 30000),
                                      np.random.default_rng(2).uniform(0, 16, 30000),
                                      np.random.default_rng(3).uniform(0, 9, 30000)]), 400),
    "sphere": lambda: (wl.sphere_surface(20000, 32)[0], 100),
    "plummer": lambda: (wl.plummer_with_background(20000, 33)[0], 64),
    "one": lambda: (np.array([[0.25, -0.5, 1.0]]), 4),
    "root_leaf": lambda: (wl.uniform_cube(500, 34)[0], 500),
    "duplicates": lambda: (np.vstack([np.full((300, 3), 0.125), wl.uniform_cube(700, 35)[0]]), 50),
    # ten groups of 200 coincident points, N0 = 100: ten chains down to the
    # depth limit, more clusters than the first room the build reserves (the
    # build is repeated with more room) and several rounds of levels
    "chains": lambda: (np.repeat(wl.uniform_cube(10, 36)[0], 200, axis=0), 100),
}


@pytest.mark.parametrize("case", sorted(TREE_CASES))
def test_tree_is_identical(K, orc, case):
    x, N0 = TREE_CASES[case]()
    t = K.kitc_build_tree(dev(x), K.Params(leaf_size=N0))
    g = t.download()
    o = orc.Tree(x, N0)
    assert g["perm"].tolist() == o.perm.tolist()
    for k in ("lo", "hi"):
        assert np.array_equal(g[k], getattr(o, k)), k
    for k in ("begin", "end", "first_child", "n_child", "level", "parent"):
        assert np.array_equal(g[k], getattr(o, k)), k
    st = t.stats()
    assert st["n_clusters"] == o.nclusters and st["n_leaves"] == int((o.n_child == 0).sum())
    t.free()


# ------------------------------------------------------------------ weights
@pytest.mark.parametrize("mode", [0, 1])
@pytest.mark.parametrize("n,kernel", [(1, ST), (4, SR), (8, ST), (12, RO), (16, ST)])
def test_modified_weights_match(K, orc, n, kernel, mode):
    # mode 1: Algorithm 1 on every cluster; mode 0: leaves by Algorithm 1,
    # parents from their children (exact by Sec. 2, so equal up to rounding)
    win = 6 if kernel == SR else 3
    x, f = wl.uniform_cube(12000, 36, win=win)
    t = K.kitc_build_tree(dev(x), K.Params(leaf_size=300, degree=n, kernel=kernel, weights=mode))
    K.kitc_modified_weights(t, dev(f))
    g = t.weights()
    o = orc.Tree(x, 300).modified_weights(f, n)
    scale = np.abs(o).max()
    err = np.abs(g - o).max() / scale
    print("weights n=%d mode=%d max rel err %.2e" % (n, mode, err))
    assert err <= 1e-13
    t.free()


def test_weights_with_particle_on_grid_point(K, orc):
    n = 4
    s = orc.cheb_points(n, 0.0, 1.0)
    x = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [s[1], s[3], s[2]]])
    f = np.array([[0.0, 0, 0], [0.0, 0, 0], [1.0, 2.0, 3.0]])
    t = K.kitc_build_tree(dev(x), K.Params(leaf_size=10, degree=n))
    K.kitc_modified_weights(t, dev(f))
    g = t.weights()[0]
    assert np.array_equal(g[1, 3, 2], f[2])
    t.free()


# -------------------------------------------------------------------- lists
@pytest.mark.parametrize("B", [64, 17])
def test_batch_lists_are_identical(K, orc, B):
    x, f = wl.uniform_cube(15000, 37)
    p = K.Params(theta=0.6, degree=3, leaf_size=200, eps=0.01, mac=K.MAC_BATCH, target_batch=B)
    t = K.kitc_build_tree(dev(x), p)
    K.kitc_modified_weights(t, dev(f))
    K.kitc_evaluate(t, dev(x))
    g = t.lists()
    o = orc.Tree(x, 200)
    r = o.treecode_batch(f, o.modified_weights(f, 3), 3, ST, 0.01, 0.6, x, B, B, lists=True,
                         evaluate=False)
    assert g["tperm"].tolist() == r["tperm"].tolist()
    assert np.array_equal(g["nfar"], r["nfar"]) and np.array_equal(g["nnear"], r["nnear"])
    assert np.array_equal(g["far"], r["far_list"]) and np.array_equal(g["near"], r["near_list"])
    st = t.stats()
    assert st["near_pairs"] == r["counts"][0] and st["far_points"] == r["counts"][1]
    t.free()


@pytest.mark.parametrize("theta", [0.5, 0.8])
def test_particle_mac_counts_are_algorithm2(K, orc, theta):
    x, f = wl.uniform_cube(15000, 38)
    p = K.Params(theta=theta, degree=4, leaf_size=150, eps=0.01, mac=K.MAC_PARTICLE)
    t = K.kitc_build_tree(dev(x), p)
    K.kitc_modified_weights(t, dev(f))
    K.kitc_evaluate(t, dev(x))
    st = t.stats()
    o = orc.Tree(x, 150)
    _, cnt = o.treecode(f, o.modified_weights(f, 4), 4, ST, 0.01, theta, x)
    assert st["near_pairs"] == cnt[0] and st["far_points"] == cnt[1]
    t.free()


# --------------------------------------------------------------- evaluation
def _oracle(orc, x, f, kernel, eps, theta, n, N0, mac, B, tgt=None):
    o = orc.Tree(x, N0)
    fh = o.modified_weights(f, n)
    tg = x if tgt is None else tgt
    if mac == 0:
        return o.treecode(f, fh, n, kernel, eps, theta, tg)[0]
    return o.treecode_batch(f, fh, n, kernel, eps, theta, tg, B, B)["out"]


@pytest.mark.parametrize("kernel", [ST, RO, SR, POLY])
@pytest.mark.parametrize("mac", [0, 1])
def test_fp64_treecode_matches_oracle(K, orc, kernel, mac):
    win = 6 if kernel == SR else 3
    x, f = wl.uniform_cube(7919, 39, win=win)   # ragged: 7919 = 123 * 64 + 47
    kw = dict(kernel=kernel, eps=0.02, theta=0.6, degree=5, leaf_size=200, mac=mac, target_batch=64)
    got, st = gpu_treecode(K, x, f, **kw)
    ref = _oracle(orc, x, f, kernel, 0.02, 0.6, 5, 200, mac, 64)
    assert st["far_points"] > 0 and st["near_pairs"] > 0
    assert orc.rel_l2(ref, got) <= FP64_TOL


@pytest.mark.parametrize("kernel", [ST, RO, SR])
@pytest.mark.parametrize("mac", [0, 1])
def test_mixed_treecode_matches_oracle(K, orc, kernel, mac):
    win = 6 if kernel == SR else 3
    x, f = wl.uniform_cube(20000, 40, win=win)
    kw = dict(kernel=kernel, eps=0.005, theta=0.6, degree=6, leaf_size=400, mac=mac,
              precision=K.MIXED)
    got, _ = gpu_treecode(K, x, f, **kw)
    ref = _oracle(orc, x, f, kernel, 0.005, 0.6, 6, 400, mac, 64)
    check_mixed(ref, got, "kernel=%d mac=%d" % (kernel, mac))


@pytest.mark.parametrize("B", [32, 17])
@pytest.mark.parametrize("mac", [0, 1, 2])
def test_mixed_one_target_per_lane(K, orc, B, mac):
    """Batches of <= 32 targets run the mixed Stokeslet with one target per lane."""
    x, f = wl.uniform_cube(20011, 46)
    kw = dict(eps=0.005, theta=0.6, degree=6, leaf_size=400, mac=mac, target_batch=B,
              precision=K.MIXED)
    got, st = gpu_treecode(K, x, f, **kw)
    o = orc.Tree(x, 400)
    fh = o.modified_weights(f, 6)
    if mac == 0:
        ref = o.treecode(f, fh, 6, ST, 0.005, 0.6, x)[0]
    else:
        ref = o.treecode_batch(f, fh, 6, ST, 0.005, 0.6, x, B, B, all_targets=(mac == 2))["out"]
    assert st["far_points"] > 0
    check_mixed(ref, got, "one target per lane B=%d mac=%d" % (B, mac))
    y, _ = wl.uniform_cube(1001, 47)
    d = K.kitc_direct(dev(y), dev(x), dev(f), K.Params(eps=0.005, precision=K.MIXED,
                                                       target_batch=B)).cpu().numpy()
    check_mixed(orc.direct(ST, 0.005, y, x, f), d, "direct B=%d" % B)


def test_separate_targets_ragged(K, orc):
    x, f = wl.uniform_cube(9000, 41)
    y, _ = wl.uniform_cube(1234, 42, -1.6, 1.4)
    got, _ = gpu_treecode(K, x, f, tgt=y, eps=0.01, theta=0.7, degree=4, leaf_size=250,
                          target_batch=40)
    ref = _oracle(orc, x, f, ST, 0.01, 0.7, 4, 250, 0, 40, tgt=y)
    assert orc.rel_l2(ref, got) <= FP64_TOL


def test_polynomial_kernel_exact_on_gpu(K, orc):
    # far field of a degree-3 kernel is exact for n >= 3 (Sec. 2): GPU treecode = direct sum
    x, f = wl.uniform_cube(6000, 43)
    got, st = gpu_treecode(K, x, f, kernel=POLY, eps=0.0, theta=0.9, degree=3, leaf_size=60)
    assert st["far_points"] > 0
    ud = orc.direct(POLY, 0.0, x, x, f)
    assert orc.rel_l2(ud, got) < 1e-12


@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
@pytest.mark.parametrize("kernel", [ST, RO, SR])
def test_direct_matches_oracle(K, orc, precision, tol, kernel):
    win = 6 if kernel == SR else 3
    x, f = wl.uniform_cube(5000, 44, win=win)
    y, _ = wl.uniform_cube(3001, 45)
    p = K.Params(kernel=kernel, eps=0.003, precision=precision)
    got = K.kitc_direct(dev(y), dev(x), dev(f), p).cpu().numpy()
    ref = orc.direct(kernel, 0.003, y, x, f)
    e = orc.rel_l2(ref, got)
    print("direct kernel=%d precision=%d rel_l2=%.3e" % (kernel, precision, e))
    assert e <= tol
    if precision == 1:
        check_mixed(ref, got, "direct kernel=%d" % kernel)


# --------------------------------------------------------------- edge cases
def test_single_particle(K, orc):
    x = np.array([[0.1, 0.2, 0.3]])
    f = np.array([[1.0, -2.0, 0.5]])
    got, st = gpu_treecode(K, x, f, eps=0.05, degree=3, leaf_size=1)
    np.testing.assert_allclose(got, orc.direct(ST, 0.05, x, x, f), rtol=1e-14)


@pytest.mark.parametrize("theta", [0.0])
def test_theta_zero_is_direct(K, orc, theta):
    x, f = wl.uniform_cube(3000, 46)
    got, st = gpu_treecode(K, x, f, eps=0.01, theta=theta, degree=4, leaf_size=100)
    assert st["far_points"] == 0
    assert orc.rel_l2(orc.direct(ST, 0.01, x, x, f), got) <= FP64_TOL


def test_root_leaf_is_direct(K, orc):
    x, f = wl.uniform_cube(700, 47)
    got, st = gpu_treecode(K, x, f, eps=0.01, theta=0.7, degree=4, leaf_size=700)
    assert st["n_clusters"] == 1
    assert orc.rel_l2(orc.direct(ST, 0.01, x, x, f), got) <= FP64_TOL


def test_eps_zero_skips_coincident_pair(K, orc):
    x, f = wl.uniform_cube(2000, 48)
    got, _ = gpu_treecode(K, x, f, eps=0.0, theta=0.6, degree=5, leaf_size=100)
    ref = _oracle(orc, x, f, ST, 0.0, 0.6, 5, 100, 0, 64)
    assert np.all(np.isfinite(got))
    assert orc.rel_l2(ref, got) <= FP64_TOL


def test_deterministic_and_host_api_identical(K):
    x, f = wl.uniform_cube(30000, 49)
    kw = dict(eps=0.005, theta=0.7, degree=6, leaf_size=500, precision=K.MIXED)
    a, _ = gpu_treecode(K, x, f, **kw)
    b, _ = gpu_treecode(K, x, f, **kw)
    h = K.kitc_solve_host(x, f, K.Params(**kw))
    assert np.array_equal(a, b) and np.array_equal(a, h)


def test_invalid_arguments_and_state(K):
    import ctypes
    import torch
    x = dev(wl.uniform_cube(100, 50)[0])
    L = K.lib()
    p = K.Params().c()
    h = ctypes.c_void_p()
    host = np.zeros((100, 3))
    # a host pointer where device memory is required is refused before any launch
    assert L.kitc_build_tree(K._np(host), 100, ctypes.byref(p), None, ctypes.byref(h)) == 1
    assert L.kitc_build_tree(None, 100, ctypes.byref(p), None, ctypes.byref(h)) == 1
    for field, bad in (("degree", 0), ("degree", 17), ("leaf_size", 0), ("theta", -1.0),
                       ("eps", -0.1), ("kernel", 5), ("target_batch", 65), ("precision", 3),
                       ("precision", -1)):
        q = K.Params().c()
        setattr(q, field, bad)
        assert L.kitc_build_tree(ctypes.c_void_p(x.data_ptr()), 100, ctypes.byref(q), None,
                                 ctypes.byref(h)) == 1, field
    assert L.kitc_build_tree(ctypes.c_void_p(x.data_ptr()), 0, ctypes.byref(p), None,
                             ctypes.byref(h)) == 1
    for prec in (K.MIXED, K.MIXED_LEAF):  # the test kernel is FP64 only
        q = K.Params(kernel=K.TEST_POLY, precision=prec).c()
        assert L.kitc_build_tree(ctypes.c_void_p(x.data_ptr()), 100, ctypes.byref(q), None,
                                 ctypes.byref(h)) == 1, prec
    t = K.kitc_build_tree(x, K.Params())
    out = torch.empty((100, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KitcError) as e:
        K.kitc_evaluate(t, x, out)
    assert e.value.status == 5
    t.free()


def test_watchdog_times_out_and_context_survives(K, orc):
    assert K.kitc_watchdog_selftest(50) == 4
    x, f = wl.uniform_cube(2000, 51)
    got, _ = gpu_treecode(K, x, f, eps=0.01, theta=0.7, degree=3, leaf_size=100)
    ref = _oracle(orc, x, f, ST, 0.01, 0.7, 3, 100, 0, 64)
    assert orc.rel_l2(ref, got) <= FP64_TOL


# ------------------------------------------------------------------ forests
def _systems(num, seed, nmin, nmax):
    return wl.batched_systems(num, seed, nmin=nmin, nmax=nmax)


@pytest.mark.parametrize("mac", [0, 1])
@pytest.mark.parametrize("precision,tol", [(0, FP64_TOL), (1, MIXED_TOL)])
def test_forest_matches_oracle_per_system(K, orc, mac, precision, tol):
    systems = _systems(7, 52, 300, 6000)
    counts = [len(x) for x, _ in systems]
    x = np.vstack([s[0] for s in systems])
    f = np.vstack([s[1] for s in systems])
    p = K.Params(theta=0.7, degree=5, leaf_size=250, eps=0.01, mac=mac, precision=precision)
    t = K.kitc_build_forest(dev(x), counts, p)
    K.kitc_modified_weights(t, dev(f))
    got = K.kitc_evaluate_forest(t, dev(x), counts).cpu().numpy()
    st = t.stats()
    t.free()
    off = np.concatenate([[0], np.cumsum(counts)])
    near = far = 0
    for k in range(len(counts)):
        xs, fs = x[off[k]:off[k + 1]], f[off[k]:off[k + 1]]
        o = orc.Tree(xs, 250)
        fh = o.modified_weights(fs, 5)
        if mac == 0:
            ref, cnt = o.treecode(fs, fh, 5, ST, 0.01, 0.7, xs)
        else:
            r = o.treecode_batch(fs, fh, 5, ST, 0.01, 0.7, xs, 64, 64)
            ref, cnt = r["out"], r["counts"]
        near += cnt[0]
        far += cnt[1]
        assert orc.rel_l2(ref, got[off[k]:off[k + 1]]) <= tol, k
        if precision == 1:
            check_mixed(ref, got[off[k]:off[k + 1]], "forest system %d" % k)
    assert st["near_pairs"] == near and st["far_points"] == far


def test_forest_of_one_equals_tree(K):
    x, f = wl.uniform_cube(5000, 53)
    p = K.Params(theta=0.7, degree=4, leaf_size=200, eps=0.01)
    a, _ = gpu_treecode(K, x, f, theta=0.7, degree=4, leaf_size=200, eps=0.01)
    t = K.kitc_build_forest(dev(x), [len(x)], p)
    K.kitc_modified_weights(t, dev(f))
    b = K.kitc_evaluate_forest(t, dev(x), [len(x)]).cpu().numpy()
    t.free()
    assert np.array_equal(a, b)


# ------------------------------------------------------------ kitc_apply
@pytest.mark.parametrize("precision", [0, 1, 2])
def test_apply_replays_with_new_weights(K, precision):
    import torch
    x, f1 = wl.uniform_cube(20000, 54)
    _, f2 = wl.uniform_cube(20000, 55)
    p = K.Params(theta=0.7, degree=6, leaf_size=500, eps=0.005, precision=precision,
                 mac=K.MAC_BATCH)
    xd = dev(x)
    t = K.kitc_build_tree(xd, p)
    K.kitc_modified_weights(t, dev(f1))
    K.kitc_evaluate(t, xd)
    w = dev(f2)
    out = torch.empty((len(x), 3), dtype=torch.float64, device="cuda")
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        K.kitc_apply(t, w, out)           # eager run + capture + replay
        a = out.cpu().numpy()
        w.copy_(dev(f1))                 # same buffer, new contents: pure replay
        K.kitc_apply(t, w, out)
        b = out.cpu().numpy()
    t.free()
    ref2, _ = gpu_treecode(K, x, f2, theta=0.7, degree=6, leaf_size=500, eps=0.005,
                           precision=precision, mac=K.MAC_BATCH)
    ref1, _ = gpu_treecode(K, x, f1, theta=0.7, degree=6, leaf_size=500, eps=0.005,
                           precision=precision, mac=K.MAC_BATCH)
    assert np.array_equal(a, ref2) and np.array_equal(b, ref1)


def test_apply_on_forest_and_before_evaluate(K):
    import torch
    systems = _systems(5, 56, 500, 5000)
    counts = [len(s[0]) for s in systems]
    x = np.vstack([s[0] for s in systems])
    f = np.vstack([s[1] for s in systems])
    p = K.Params(theta=0.7, degree=5, leaf_size=300, eps=0.01, precision=K.MIXED)
    t = K.kitc_build_forest(dev(x), counts, p)
    out = torch.empty((len(x), 3), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KitcError) as e:
        K.kitc_apply(t, dev(f), out)
    assert e.value.status == 5
    K.kitc_modified_weights(t, dev(np.zeros_like(f)))
    K.kitc_evaluate_forest(t, dev(x), counts)
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        K.kitc_apply(t, dev(f), out)
        got = out.cpu().numpy()
    t2 = K.kitc_build_forest(dev(x), counts, p)
    K.kitc_modified_weights(t2, dev(f))
    ref = K.kitc_evaluate_forest(t2, dev(x), counts).cpu().numpy()
    t.free()
    t2.free()
    assert np.array_equal(got, ref)
