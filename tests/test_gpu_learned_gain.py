"""What the trained degree selector gains over the fixed-degree treecode.

A selector is trained on the GPU (the library's own gradient and Adam
kernels) from per-cluster far-field errors that the treecode measures on one
Plummer system; it then picks the degrees of a second system drawn with
another seed.  At an error no larger than the learned run's (both measured
against the FP64 direct sum on sampled targets), the best fixed degree needs
more far-field grid points, so the learned run does less evaluation work.
"""
import math

import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

pytestmark = pytest.mark.gpu

N = 300_000
LEAF = 500


@pytest.fixture(scope="module")
def K():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1902_02250_gb300 import build, kitc
    build.build()
    torch.cuda.set_device(0)
    return kitc


def _params(K, **kw):
    b = dict(theta=0.7, degree=8, leaf_size=LEAF, eps=1e-3, precision=K.MIXED, mac=K.MAC_BATCH,
             target_batch=64)
    b.update(kw)
    return K.Params(**b)


def _rel(a, b):
    return math.sqrt(float(((a - b) ** 2).sum()) / float((a ** 2).sum()))


def test_learned_degrees_beat_the_fixed_degree_at_matched_error(K):
    import torch
    from paper_1902_02250_gb300 import learned as LD
    xt, ft = wl.plummer_with_background(N, 41)
    meas = LD.measure(torch.from_numpy(xt).cuda(), torch.from_numpy(ft).cuda(), _params(K))
    lab, valid, tau = LD.labels(meas, 0.5e-6)
    rows = torch.from_numpy(np.nonzero(valid)[0]).cuda()
    params, rep = LD.train(meas["features"][rows].contiguous(), lab[valid], steps=2000)
    majority = np.bincount(lab[valid]).max() / valid.sum()
    assert rep["accuracy"] > majority + 0.05        # the network learned more than the prior

    x, f = wl.plummer_with_background(N, 42)
    xd, fd = torch.from_numpy(x).cuda(), torch.from_numpy(f).cuda()
    idx = wl.sample_indices(N, 3000, 43)
    ref = K.kitc_direct(xd[torch.from_numpy(idx).cuda()].contiguous(), xd, fd,
                        K.Params(eps=1e-3, precision=K.FP64)).cpu().numpy()
    out = torch.empty((N, 3), dtype=torch.float64, device="cuda")
    st = LD.learned_step(xd, fd, _params(K), params, out)
    e_learned = _rel(ref, out.cpu().numpy()[idx])
    far_learned = st["far_points"]
    fixed = []
    for n in range(4, 15):
        t = K.kitc_build_tree(xd, _params(K, degree=n))
        K.kitc_modified_weights(t, fd)
        K.kitc_evaluate(t, xd, out)
        e = _rel(ref, out.cpu().numpy()[idx])
        fixed.append((n, e, t.stats()["far_points"]))
        t.free()
        if e <= e_learned:
            break
    n, e_fixed, far_fixed = fixed[-1]
    print("learned E=%.3e far=%d; fixed n=%d E=%.3e far=%d; search %s"
          % (e_learned, far_learned, n, e_fixed, far_fixed, fixed))
    assert e_learned <= 2e-6
    assert e_fixed <= e_learned            # the fixed degree that matches the learned error
    assert far_learned < 0.9 * far_fixed   # ... needs at least 10% more far-field work
