"""The autotuner on small systems: the theta walk stops at the first theta
within the error budget, the choice is the fastest feasible record, and the
forest tuner returns the fastest of its (N0, batch, MAC) candidates."""
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


def test_tune_walks_theta_down_to_the_budget(K):
    import torch
    from paper_1902_02250_gb300 import tune
    x, f = wl.uniform_cube(30000, 71)
    xd, fd = torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda()
    idx = wl.sample_indices(30000, 2000, 72)
    ref = K.kitc_direct(xd[torch.from_numpy(idx).cuda()].contiguous(), xd, fd,
                        K.Params(eps=0.01, precision=K.FP64)).cpu().numpy()
    budget = 2e-5
    base = K.Params(eps=0.01, precision=K.MIXED)
    best, recs = tune.tune(xd, fd, base, budget, idx, ref, thetas=(0.9, 0.8, 0.7, 0.6),
                           degrees=(4, 6), leaves=(500,), macs=(K.MAC_PARTICLE, K.MAC_ALL))
    assert best is not None
    p, rec = best
    assert rec["E"] <= budget and p.theta == rec["theta"] and p.degree == rec["degree"]
    for mac in (K.MAC_PARTICLE, K.MAC_ALL):
        for n in (4, 6):
            walk = [r for r in recs if r["mac"] == mac and r["degree"] == n]
            # thetas in descending order, only the last one within the budget
            assert [r["theta"] for r in walk] == [0.9, 0.8, 0.7, 0.6][:len(walk)]
            assert all(r["E"] > budget for r in walk[:-1])
            if walk[-1]["E"] <= budget:
                assert rec["ms"] <= walk[-1]["ms"]
    feasible = [r for r in recs if r["E"] <= budget]
    assert rec["ms"] == min(r["ms"] for r in feasible)


def test_tune_forest_returns_the_fastest_candidate(K):
    import torch
    from paper_1902_02250_gb300 import tune
    systems = [wl.uniform_cube(n, 80 + k) for k, n in enumerate((3000, 700, 12000, 5000))]
    counts = np.array([len(s[0]) for s in systems], np.int64)
    xd = torch.from_numpy(np.vstack([s[0] for s in systems])).cuda()
    fd = torch.from_numpy(np.vstack([s[1] for s in systems])).cuda()
    log = []
    base = K.Params(theta=0.7, degree=5, eps=0.01, precision=K.MIXED)
    p, ms = tune.tune_forest(xd, fd, counts, base, leaves=(200, 800), batches=(32, 64),
                             macs=(K.MAC_PARTICLE, K.MAC_BATCH, K.MAC_ALL), log=log.append)
    assert len(log) == 12
    fastest = min(log, key=lambda r: r["ms"])
    assert ms == fastest["ms"]
    assert (p.leaf_size, p.target_batch, p.mac) == (fastest["leaf_size"], fastest["target_batch"],
                                                    fastest["mac"])
    assert (p.theta, p.degree, p.eps, p.precision) == (0.7, 5, 0.01, K.MIXED)
