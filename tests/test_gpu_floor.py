"""Precision floor of the mixed forms, required before any mixed number is
quoted: the mixed direct sum against the FP64 direct sum on sampled targets of
the N = 10^6 uniform Stokeslet system (eps = 1e-3) stays within 2e-7 relative
L2.  The mixed treecode cannot be more accurate than this floor."""
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


def test_mixed_direct_floor(K):
    import torch
    x, f = wl.uniform_cube(1_000_000, 2)
    xd, fd = torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda()
    idx = torch.from_numpy(wl.sample_indices(len(x), 2000, 102)).cuda()
    yd = xd[idx].contiguous()
    ref = K.kitc_direct(yd, xd, fd, K.Params(eps=1e-3, precision=K.FP64)).cpu().numpy()
    got = K.kitc_direct(yd, xd, fd, K.Params(eps=1e-3, precision=K.MIXED)).cpu().numpy()
    e = float(np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum()))
    print("mixed direct-sum floor: %.3e" % e)
    assert e <= 2e-7


def test_leaf_offset_near_field_floor(K):
    """The same bound for the near field of KITC_MIXED_LEAF (differences from
    leaf-local FP32 offsets): theta = 0 makes every pair a near pair, so the
    treecode is the direct sum in that form."""
    import torch
    x, f = wl.uniform_cube(1_000_000, 2)
    xd, fd = torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda()
    idx = torch.from_numpy(wl.sample_indices(len(x), 2000, 102)).cuda()
    yd = xd[idx].contiguous()
    ref = K.kitc_direct(yd, xd, fd, K.Params(eps=1e-3, precision=K.FP64)).cpu().numpy()
    p = K.Params(theta=0.0, degree=1, leaf_size=4000, eps=1e-3, precision=K.MIXED_LEAF,
                 mac=K.MAC_ALL)
    out, st = K.treecode(xd, fd, p, yd)
    assert st["far_points"] == 0 and st["near_pairs"] == 2000 * len(x)
    got = out.cpu().numpy()
    e = float(np.sqrt(((got - ref) ** 2).sum() / (ref ** 2).sum()))
    print("leaf-offset near-field floor: %.3e" % e)
    assert e <= 2e-7
