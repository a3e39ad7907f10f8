"""The benchmark configurations as parity cases at their own sizes.

* N = 10,000 uniform in [-1,1]^3 (seed 1), f ~ U[-1,1]^3, Stokeslet, eps = 0.01,
  theta = 0.7, n = 4, N0 = 500: the GPU treecode (FP64 and mixed) against the
  oracle's Algorithm 2, and both against the full FP64 direct sum (10^8 pairs).
* N = 1,000,000 uniform (seed 2), eps = 1e-3, the bench point (batch MAC,
  theta = 0.7, n = 9, N0 = 4000) in the launch configuration the bench times:
  sampled targets against the oracle's batch-MAC treecode computed one by one,
  and the relative L2 error against the FP64 direct sum within 1e-6.
* N = 1,000,000 on the unit sphere (seed 3), torques N(0,1), rotlet, eps = 0.005:
  the sphere sweep's fastest point with E <= 1e-6 (all-targets MAC, theta = 0.7,
  n = 6, N0 = 2000) and the per-target MAC at theta = 0.5, n = 4, each on the
  FP32x2 rotlet path: sampled targets against the oracle one by one, exact
  interaction counts, and E against the FP64 direct sum within 1e-6.
"""
import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

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
        e = orc.rel_l2(direct, got)
        print("N=10^4 precision=%d E_vs_direct=%.3e (oracle %.3e)" % (prec, e, e_oracle))
        assert abs(e - e_oracle) <= (1e-12 if prec == K.FP64 else 1e-6)
    gd = K.kitc_direct(dev(x), dev(x), dev(f), K.Params(eps=0.01, precision=K.FP64)).cpu().numpy()
    assert orc.rel_l2(direct, gd) <= 1e-12


def test_config_bench_point_1m(K, orc):
    import torch
    x, f = wl.uniform_cube(1_000_000, 2)
    xd, fd = dev(x), dev(f)
    p = K.Params(theta=0.7, degree=9, leaf_size=4000, eps=1e-3, precision=K.MIXED,
                 mac=K.MAC_BATCH, target_batch=64)
    out, st = K.treecode(xd, fd, p)
    got = out.cpu().numpy()
    sel = wl.sample_indices(len(x), 300, 2024)
    o = orc.Tree(x, 4000)
    ref = o.treecode_batch(f, o.modified_weights(f, 9), 9, orc.STOKESLET, 1e-3, 0.7, x, 64, 64,
                           select=sel)
    assert orc.rel_l2(ref["out"][sel], got[sel]) <= 1e-6
    assert st["far_points"] == ref["counts"][1] and st["near_pairs"] == ref["counts"][0]
    idx = torch.from_numpy(wl.sample_indices(len(x), 2000, 102)).cuda()
    d = K.kitc_direct(xd[idx].contiguous(), xd, fd, K.Params(eps=1e-3, precision=K.FP64)).cpu().numpy()
    e = orc.rel_l2(d, got[idx.cpu().numpy()])
    print("bench point E vs direct on 2000 samples: %.3e" % e)
    assert e <= 1e-6


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
        assert orc.rel_l2(ref, got[sel]) <= 1e-6
    else:
        r = o.treecode_batch(f, fh, n, orc.ROTLET, 0.005, theta, x, 64, 64, select=sel, all_targets=True)
        assert orc.rel_l2(r["out"][sel], got[sel]) <= 1e-6
        assert st["far_points"] == r["counts"][1] and st["near_pairs"] == r["counts"][0]
    idx = torch.from_numpy(wl.sample_indices(len(x), 2000, 102)).cuda()
    d = K.kitc_direct(xd[idx].contiguous(), xd, fd,
                      K.Params(eps=0.005, kernel=K.ROTLET, precision=K.FP64)).cpu().numpy()
    e = orc.rel_l2(d, got[idx.cpu().numpy()])
    print("sphere rotlet theta=%.1f n=%d mac=%d E vs direct on 2000 samples: %.3e" % (theta, n, mac, e))
    assert e <= 1e-6
