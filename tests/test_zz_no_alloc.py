"""kitc_direct_noalloc: the direct sum for callers that must not allocate
device memory (a latency-critical loop, an embedding whose allocator owns the
device's memory, error handling after memory ran out).  Its scratch is the
library's fixed device array, so it is checked against kitc_direct, which
allocates its own, on two calls in a row (the second call reuses the array the
first one left behind).  After the first call on the device (its set-up), a
call allocates nothing: neither the device's default memory pool, nor torch's
allocator, nor the device's free memory change across it.  Collected last so
that a failure here stops a run only after every other test has run; it also
passes alone in a fresh process.
"""
import gc

import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

from devpool import USED_MEM_HIGH, Pool

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


def test_noalloc_allocates_nothing_after_setup(K):
    """The first call on the device is the set-up (the scratch array and the
    kernels are loaded).  Every later call -- any kernel, either precision --
    leaves the pool's reserved and used bytes, its high-water mark, torch's
    allocator and the device's free memory as they were."""
    import torch
    x, f = wl.uniform_cube(20000, 71, win=6)
    y, _ = wl.uniform_cube(3000, 72)
    xd = torch.from_numpy(x).cuda()
    f6 = torch.from_numpy(f).cuda()
    f3 = f6[:, :3].contiguous()
    yd = torch.from_numpy(y).cuda()
    outs = {k: torch.zeros((len(y), K.kernel_wout(k)), dtype=torch.float64, device="cuda")
            for k in (0, 1, 2)}
    calls = [(0, 1, f3), (1, 1, f3), (2, 1, f6), (0, 0, f3), (1, 0, f3), (2, 0, f6)]
    K.kitc_direct_noalloc(yd, xd, f3, K.Params(kernel=0, precision=1, eps=0.004), outs[0])
    pool = Pool(torch.cuda.current_device())
    gc.collect()  # no collection inside the window: it frees test temporaries
    gc.disable()
    try:
        torch.cuda.synchronize()
        before = pool.snapshot()
        pool.reset_high()
        for kernel, prec, w in calls:
            K.kitc_direct_noalloc(yd, xd, w, K.Params(kernel=kernel, precision=prec, eps=0.004),
                                  outs[kernel])
        torch.cuda.synchronize()
        after = pool.snapshot()
    finally:
        gc.enable()
    assert after == before, (before, after)
    assert pool.get(USED_MEM_HIGH) == before[1]
    # and the last call's result is the direct sum
    ref = K.kitc_direct(yd, xd, f6, K.Params(kernel=2, precision=0, eps=0.004)).cpu().numpy()
    assert _rel(ref, outs[2].cpu().numpy()) <= FP64_TOL
