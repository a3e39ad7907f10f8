"""The benchmark configurations as parity cases at their own sizes.

* N = 10,000 uniform in [-1,1]^3 (seed 1), f ~ U[-1,1]^3, Stokeslet, eps = 0.01,
  theta = 0.7, n = 4, N0 = 500: the GPU treecode (FP64 and mixed) against the
  oracle's Algorithm 2, and both against the full FP64 direct sum (10^8 pairs).
* N = 1,000,000 uniform (seed 2), eps = 1e-3, the bench point (all-targets
  MAC, theta = 0.68, n = 9, N0 = 4000) in the launch configuration the bench
  times, in both mixed forms (leaf-offset and hi/lo near-field differences):
  sampled targets against the oracle's treecode with the same MAC rule
  computed one by one, and the relative L2 error against the FP64 direct sum
  within 1e-6.
* N = 1,000,000 on the unit sphere (seed 3), torques N(0,1), rotlet, eps = 0.005:
  the sphere sweep's fastest point with E <= 1e-6 (all-targets MAC, theta = 0.7,
  n = 6, N0 = 2000) and the per-target MAC at theta = 0.5, n = 4, each on the
  FP32x2 rotlet path: sampled targets against the oracle one by one, exact
  interaction counts, and E against the FP64 direct sum within 1e-6.
* The plain FP64 treecode at the point the bench times it (N = 10^6 uniform,
  batch MAC, theta = 0.65, n = 8, N0 = 4000): sampled targets against the
  oracle at 1e-12, exact interaction counts.
* The paper's own workloads (Sec. 8.1, 8.2) at full size, FP64 and mixed:
  Example 1 (organisms, N = 640,000, eps = 0.02, theta = 0.7, n = 7, N0 = 2000,
  per-target MAC) and Example 2 (helical rods, N = 966,400, Stokeslet +
  rotlet, eps = 0.3, theta = 0.7, n = 7, N0 = 1000), sampled targets against the
  oracle's Algorithm 2; and Example 1 at N = 5.12M in FP64.
Every mixed comparison also bounds the error of every single target
(mixed_parity.check_mixed).
"""
import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

from mixed_parity import FP64_TOL, check_mixed

pytestmark = pytest.mark.gpu


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


def test_config_n10k(K, orc):
    x, f = wl.uniform_cube(10_000, 1)
    ref_tc, _ = orc.treecode(x, f, orc.STOKESLET, 0.01, 0.7, 4, 500)
    direct = orc.direct(orc.STOKESLET, 0.01, x, x, f)
    e_oracle = orc.rel_l2(direct, ref_tc)
    for prec, tol in ((K.FP64, 1e-12), (K.MIXED, 1e-6)):
        p = K.Params(theta=0.7, degree=4, leaf_size=500, eps=0.01, precision=prec)
        out, st = K.treecode(dev(x), dev(f), p)
        got = out.cpu().numpy()
        assert orc.rel_l2(ref_tc, got) <= tol
        if prec == K.MIXED:
            check_mixed(ref_tc, got, "N=10^4")
        e = orc.rel_l2(direct, got)
        print("N=10^4 precision=%d E_vs_direct=%.3e (oracle %.3e)" % (prec, e, e_oracle))
        assert abs(e - e_oracle) <= (1e-12 if prec == K.FP64 else 1e-6)
    gd = K.kitc_direct(dev(x), dev(x), dev(f), K.Params(eps=0.01, precision=K.FP64)).cpu().numpy()
    assert orc.rel_l2(direct, gd) <= 1e-12


@pytest.mark.parametrize("prec", ["MIXED_LEAF", "MIXED"])
def test_config_bench_point_1m(K, orc, prec):
    """The mixed treecode where the bench times it (the headline's leaf-offset
    form, and the hi/lo form timed beside it), against the oracle's treecode
    with the same MAC rule on sampled targets (exact counts)."""
    import torch
    import bench
    x, f = wl.uniform_cube(bench.N, bench.SEED)
    xd, fd = dev(x), dev(f)
    mac = bench.MAC_IDS[bench.MAC]
    p = K.Params(theta=bench.THETA, degree=bench.DEGREE, leaf_size=bench.LEAF, eps=bench.EPS,
                 precision=getattr(K, prec), mac=mac, target_batch=bench.BATCH)
    out, st = K.treecode(xd, fd, p)
    got = out.cpu().numpy()
    sel = wl.sample_indices(len(x), 300, 2024)
    o = orc.Tree(x, bench.LEAF)
    ref = o.treecode_batch(f, o.modified_weights(f, bench.DEGREE), bench.DEGREE, orc.STOKESLET,
                           bench.EPS, bench.THETA, x, bench.BATCH, bench.BATCH, select=sel,
                           all_targets=(mac == K.MAC_ALL))
    check_mixed(ref["out"][sel], got[sel], "bench point N=10^6 %s" % prec)
    assert st["far_points"] == ref["counts"][1] and st["near_pairs"] == ref["counts"][0]
    idx = torch.from_numpy(wl.sample_indices(len(x), 2000, 102)).cuda()
    d = K.kitc_direct(xd[idx].contiguous(), xd, fd, K.Params(eps=bench.EPS, precision=K.FP64)).cpu().numpy()
    e = orc.rel_l2(d, got[idx.cpu().numpy()])
    print("bench point E vs direct on 2000 samples: %.3e" % e)
    assert e <= 1e-6


def test_config_fp64_point_1m(K, orc):
    """The metric's comparison point: the plain FP64 treecode where the bench
    times it, against the oracle's batch-MAC treecode on sampled targets."""
    import bench
    theta, n, leaf, mac = bench.FP64_POINT
    assert mac == "batch"
    x, f = wl.uniform_cube(bench.N, bench.SEED)
    p = K.Params(theta=theta, degree=n, leaf_size=leaf, eps=bench.EPS, precision=K.FP64,
                 mac=K.MAC_BATCH, target_batch=bench.BATCH)
    out, st = K.treecode(dev(x), dev(f), p)
    got = out.cpu().numpy()
    sel = wl.sample_indices(len(x), 300, 2026)
    o = orc.Tree(x, leaf)
    ref = o.treecode_batch(f, o.modified_weights(f, n), n, orc.STOKESLET, bench.EPS, theta, x,
                           bench.BATCH, bench.BATCH, select=sel)
    e = orc.rel_l2(ref["out"][sel], got[sel])
    print("FP64 point N=10^6 rel_l2 vs oracle on 300 samples: %.3e" % e)
    assert e <= FP64_TOL
    assert st["far_points"] == ref["counts"][1] and st["near_pairs"] == ref["counts"][0]


def _paper_case(K, orc, x, f, kernel, eps, leaf, what):
    """theta = 0.7, n = 7, per-target MAC (Algorithm 2), both precisions, 300
    sampled targets against the oracle evaluated target by target."""
    xd, fd = dev(x), dev(f)
    sel = wl.sample_indices(len(x), 300, 2027)
    o = orc.Tree(x, leaf)
    fh = o.modified_weights(f, 7)
    ref, _ = o.treecode(f, fh, 7, kernel, eps, 0.7, x[sel])
    for prec in (K.FP64, K.MIXED):
        p = K.Params(theta=0.7, degree=7, leaf_size=leaf, eps=eps, kernel=kernel, precision=prec,
                     mac=K.MAC_PARTICLE, target_batch=64)
        out, st = K.treecode(xd, fd, p)
        got = out.cpu().numpy()[sel]
        if prec == K.FP64:
            e = orc.rel_l2(ref, got)
            print("%s FP64 rel_l2 vs oracle: %.3e" % (what, e))
            assert e <= FP64_TOL
        else:
            check_mixed(ref, got, what)


def test_config_paper_example1_640k(K, orc):
    x, f = wl.organisms(320_000, 31)
    _paper_case(K, orc, x, f, orc.STOKESLET, 0.02, 2000, "Example 1 N=640K")


def test_config_paper_example1_5m_fp64(K, orc):
    """Example 1 at N = 5.12M (the size where our error departs most from the
    paper's table): the FP64 treecode against the oracle's Algorithm 2 on
    sampled targets."""
    x, f = wl.organisms(2_560_000, 31)
    xd, fd = dev(x), dev(f)
    sel = wl.sample_indices(len(x), 200, 2028)
    o = orc.Tree(x, 2000)
    ref, _ = o.treecode(f, o.modified_weights(f, 7), 7, orc.STOKESLET, 0.02, 0.7, x[sel])
    p = K.Params(theta=0.7, degree=7, leaf_size=2000, eps=0.02, precision=K.FP64,
                 mac=K.MAC_PARTICLE, target_batch=64)
    out, st = K.treecode(xd, fd, p)
    e = orc.rel_l2(ref, out.cpu().numpy()[sel])
    print("Example 1 N=5.12M FP64 rel_l2 vs oracle on 200 samples: %.3e" % e)
    assert e <= FP64_TOL


def test_config_paper_example2_rods(K, orc):
    x, f = wl.helical_rods(80, 33, spacing=16.0 / 79)
    assert len(x) == 966_400
    _paper_case(K, orc, x, f, orc.STOKESLET_ROTLET, 0.3, 1000, "Example 2 N=966,400")


@pytest.mark.parametrize("theta,n,mac", [(0.7, 6, 2), (0.5, 4, 0)])
def test_config_sphere_rotlet_1m(K, orc, theta, n, mac):
    import torch
    x, f = wl.sphere_surface(1_000_000, 3)
    xd, fd = dev(x), dev(f)
    p = K.Params(theta=theta, degree=n, leaf_size=2000, eps=0.005, kernel=K.ROTLET,
                 precision=K.MIXED, mac=mac, target_batch=64)
    out, st = K.treecode(xd, fd, p)
    got = out.cpu().numpy()
    sel = wl.sample_indices(len(x), 300, 2025)
    o = orc.Tree(x, 2000)
    fh = o.modified_weights(f, n)
    if mac == 0:
        ref, cnt = o.treecode(f, fh, n, orc.ROTLET, 0.005, theta, x[sel])
        check_mixed(ref, got[sel], "sphere rotlet theta=%.1f n=%d" % (theta, n))
    else:
        r = o.treecode_batch(f, fh, n, orc.ROTLET, 0.005, theta, x, 64, 64, select=sel, all_targets=True)
        check_mixed(r["out"][sel], got[sel], "sphere rotlet theta=%.1f n=%d" % (theta, n))
        assert st["far_points"] == r["counts"][1] and st["near_pairs"] == r["counts"][0]
    idx = torch.from_numpy(wl.sample_indices(len(x), 2000, 102)).cuda()
    d = K.kitc_direct(xd[idx].contiguous(), xd, fd,
                      K.Params(eps=0.005, kernel=K.ROTLET, precision=K.FP64)).cpu().numpy()
    e = orc.rel_l2(d, got[idx.cpu().numpy()])
    print("sphere rotlet theta=%.1f n=%d mac=%d E vs direct on 2000 samples: %.3e" % (theta, n, mac, e))
    assert e <= 1e-6
