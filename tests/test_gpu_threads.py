"""Several host threads driving the library at once, each on its own CUDA
stream with its own handles: the results equal those of one thread (the
library's shared state is limited to per-thread read-back buffers and kernel
attributes that are set once to fixed values)."""
import threading

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


def test_concurrent_threads_match_sequential(K):
    import torch
    inputs = [wl.uniform_cube(30000 + 1000 * i, 200 + i) for i in range(4)]
    params = [K.Params(theta=0.7, degree=6, leaf_size=400, eps=0.001, precision=K.MIXED,
                       mac=K.MAC_BATCH),
              K.Params(theta=0.6, degree=5, leaf_size=300, eps=0.002, precision=K.FP64),
              K.Params(theta=0.7, degree=8, leaf_size=500, eps=0.001, precision=K.MIXED),
              K.Params(theta=0.5, degree=4, leaf_size=200, eps=0.01, precision=K.FP64,
                       mac=K.MAC_BATCH)]

    def run(i):
        x, f = inputs[i]
        xd = torch.from_numpy(x).cuda()
        fd = torch.from_numpy(f).cuda()
        out, _ = K.treecode(xd, fd, params[i])
        return out.cpu().numpy()

    seq = [run(i) for i in range(4)]
    res = [None] * 4
    errors = []

    def worker(i):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                for _ in range(3):
                    r = run(i)
                s.synchronize()
            res[i] = r
        except Exception as e:  # reported after join
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(i,)) for i in range(4)]
    for t in threads:
        t.start()
    for t in threads:
        t.join()
    assert not errors, errors
    for a, b in zip(seq, res):
        assert np.array_equal(a, b)
