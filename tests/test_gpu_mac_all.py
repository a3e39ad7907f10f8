"""The all-targets batch rule (KITC_MAC_ALL: a cluster is accepted for a target
batch iff every target of the batch accepts it by Eq. MAC) against the oracle's
same rule: identical lists and counts, FP64 results to 1e-12, mixed to 1e-6."""
import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

from mixed_parity import check_mixed

pytestmark = pytest.mark.gpu

ST, RO, SR = 0, 1, 2


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


@pytest.mark.parametrize("B", [64, 17])
def test_lists_are_identical(K, orc, B):
    x, f = wl.plummer_with_background(15000, 170)
    p = K.Params(theta=0.6, degree=3, leaf_size=200, eps=0.01, mac=K.MAC_ALL, target_batch=B)
    t = K.kitc_build_tree(dev(x), p)
    K.kitc_modified_weights(t, dev(f))
    K.kitc_evaluate(t, dev(x))
    g = t.lists()
    o = orc.Tree(x, 200)
    r = o.treecode_batch(f, o.modified_weights(f, 3), 3, ST, 0.01, 0.6, x, B, B, lists=True,
                         evaluate=False, all_targets=True)
    assert g["tperm"].tolist() == r["tperm"].tolist()
    assert np.array_equal(g["nfar"], r["nfar"]) and np.array_equal(g["nnear"], r["nnear"])
    assert np.array_equal(g["far"], r["far_list"]) and np.array_equal(g["near"], r["near_list"])
    st = t.stats()
    assert st["near_pairs"] == r["counts"][0] and st["far_points"] == r["counts"][1]
    t.free()


@pytest.mark.parametrize("kernel", [ST, RO, SR])
@pytest.mark.parametrize("prec", [0, 1])
def test_treecode_matches_oracle(K, orc, kernel, prec):
    win = 6 if kernel == SR else 3
    x, f = wl.uniform_cube(12001, 171, win=win)
    p = K.Params(theta=0.7, degree=6, leaf_size=250, eps=0.01, kernel=kernel, precision=prec,
                 mac=K.MAC_ALL)
    out, st = K.treecode(dev(x), dev(f), p)
    got = out.cpu().numpy()
    o = orc.Tree(x, 250)
    sel = wl.sample_indices(len(x), 3000, 172)
    r = o.treecode_batch(f, o.modified_weights(f, 6), 6, kernel, 0.01, 0.7, x, 64, 64,
                         select=sel, all_targets=True)
    assert st["far_points"] == r["counts"][1] and st["near_pairs"] == r["counts"][0]
    if prec == 0:
        e = orc.rel_l2(r["out"][sel], got[sel])
        assert e <= 1e-12, e
    else:
        check_mixed(r["out"][sel], got[sel], "all-targets MAC kernel=%d" % kernel)
