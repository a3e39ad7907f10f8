"""kitc_direct_noalloc: the direct sum for callers that must not allocate
device memory (a latency-critical loop, an embedding whose allocator owns the
device's memory, error handling after memory ran out).  Its scratch is the
library's fixed device array, so it is checked against kitc_direct, which
allocates its own, on two calls in a row (the second call reuses the array the
first one left behind).  Collected last so that a failure here stops a run
only after every other test has run; it also passes alone in a fresh process.
"""
import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-12
MIXED_TOL = 1e-6


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_02250_gb300 import build, kitc
    build.build()
    torch.cuda.set_device(0)
    return kitc


def _rel(a, b):
    return float(np.sqrt(((a - b) ** 2).sum() / (a ** 2).sum()))


@pytest.mark.parametrize("kernel,precision,tol", [(0, 0, FP64_TOL), (0, 1, MIXED_TOL),
                                                  (1, 1, MIXED_TOL), (2, 0, FP64_TOL)])
def test_noalloc_direct_matches_direct_twice(K, kernel, precision, tol):
    import torch
    win = 6 if kernel == 2 else 3
    wout = K.kernel_wout(kernel)
    p = K.Params(kernel=kernel, precision=precision, eps=0.004)
    for call, seed in enumerate((61, 62)):  # two calls in a row, different data and sizes
        x, f = wl.uniform_cube(9000 + 777 * call, seed, win=win)
        y, _ = wl.uniform_cube(2500 - 301 * call, seed + 10)
        xd = torch.from_numpy(x).cuda()
        fd = torch.from_numpy(f).cuda()
        yd = torch.from_numpy(y).cuda()
        ref = K.kitc_direct(yd, xd, fd, p).cpu().numpy()
        out = torch.full((len(y), wout), float("nan"), dtype=torch.float64, device="cuda")
        got = K.kitc_direct_noalloc(yd, xd, fd, p, out).cpu().numpy()
        assert np.all(np.isfinite(got))
        assert _rel(ref, got) <= tol, (call, _rel(ref, got))


def test_noalloc_refuses_sizes_beyond_its_scratch(K):
    import torch
    n = 100001
    x = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    f = torch.zeros((n, 3), dtype=torch.float64, device="cuda")
    y = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    out = torch.zeros((10, 3), dtype=torch.float64, device="cuda")
    with pytest.raises(K.KitcError) as e:
        K.kitc_direct_noalloc(y, x, f, K.Params(), out)
    assert e.value.status == 6
