"""The FP32x2 rotlet evaluator (paired records, one row per far-field run,
cross-product sums split into positive and negative parts) against the FP64
CPU oracle: every pair count of a grid row (odd n + 1 adds a zero-weight point
far away), both MAC modes, ragged batches and leaves, separate targets, and
eps = 0 with coincident pairs (Sec. 1: the pair is left out).  Tolerance as in
test_gpu_parity (MIXED_TOL, from FP32 rounding)."""
import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

from mixed_parity import check_mixed

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6
RO = 1


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


def _run(K, x, f, tgt=None, **kw):
    out, st = K.treecode(dev(x), dev(f), K.Params(kernel=RO, precision=K.MIXED, **kw),
                         None if tgt is None else dev(tgt))
    return out.cpu().numpy(), st


def _oracle(orc, x, f, eps, theta, n, N0, mac, B, tgt=None):
    o = orc.Tree(x, N0)
    fh = o.modified_weights(f, n)
    tg = x if tgt is None else tgt
    if mac == 0:
        return o.treecode(f, fh, n, RO, eps, theta, tg)[0]
    return o.treecode_batch(f, fh, n, RO, eps, theta, tg, B, B)["out"]


@pytest.mark.parametrize("mac", [0, 1])
@pytest.mark.parametrize("n", [1, 2, 4, 7, 10])
def test_sphere_rows_of_every_pair_count(K, orc, n, mac):
    x, f = wl.sphere_surface(12001, 61)           # ragged: 12001 = 187 * 64 + 33
    got, st = _run(K, x, f, eps=0.005, theta=0.6, degree=n, leaf_size=301, mac=mac)
    ref = _oracle(orc, x, f, 0.005, 0.6, n, 301, mac, 64)
    assert st["far_points"] > 0 and st["near_pairs"] > 0
    check_mixed(ref, got, "rotlet n=%d mac=%d" % (n, mac))


@pytest.mark.parametrize("mac", [0, 1, 2])
@pytest.mark.parametrize("B", [32, 17])
def test_small_batches(K, orc, B, mac):
    """Batches of <= 32 targets (the second target slot of a lane stays idle)."""
    x, f = wl.sphere_surface(9001, 67)
    got, _ = _run(K, x, f, eps=0.005, theta=0.6, degree=5, leaf_size=301, mac=mac, target_batch=B)
    o = orc.Tree(x, 301)
    fh = o.modified_weights(f, 5)
    if mac == 0:
        ref = o.treecode(f, fh, 5, RO, 0.005, 0.6, x)[0]
    else:
        ref = o.treecode_batch(f, fh, 5, RO, 0.005, 0.6, x, B, B, all_targets=(mac == 2))["out"]
    check_mixed(ref, got, "rotlet small batches B=%d mac=%d" % (B, mac))


def test_eps_zero_leaves_out_coincident_pairs(K, orc):
    x, f = wl.uniform_cube(3000, 62)
    x = np.vstack([x, x[:7]])                     # seven sources twice: coincident pairs
    f = np.vstack([f, f[:7]])
    got, _ = _run(K, x, f, eps=0.0, theta=0.6, degree=5, leaf_size=100)
    ref = _oracle(orc, x, f, 0.0, 0.6, 5, 100, 0, 64)
    check_mixed(ref, got, "rotlet eps=0")


def test_separate_targets_ragged_batches(K, orc):
    x, f = wl.sphere_surface(9000, 63)
    y, _ = wl.uniform_cube(1234, 64, -1.3, 1.3)
    got, _ = _run(K, x, f, tgt=y, eps=0.01, theta=0.7, degree=6, leaf_size=250, target_batch=40)
    ref = _oracle(orc, x, f, 0.01, 0.7, 6, 250, 0, 40, tgt=y)
    check_mixed(ref, got, "rotlet separate targets")


def test_direct_sum_of_paired_records(K, orc):
    x, f = wl.uniform_cube(3001, 65)              # odd: the last record is padded
    y, _ = wl.uniform_cube(777, 66)
    got = K.kitc_direct(dev(y), dev(x), dev(f), K.Params(kernel=RO, precision=K.MIXED, eps=0.003))
    ref = orc.direct(RO, 0.003, y, x, f)
    check_mixed(ref, got.cpu().numpy(), "rotlet direct")
