"""Pins of the oracle's treecode (Algorithm 2 and the batch variant):
theta -> 0 gives the direct sum, a kernel of degree <= n in y is reproduced
exactly at any theta, every source is counted once per target, the error
falls with n, and Example 1's error has the paper's order of magnitude."""
import os

import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

ST, RO, SR, POLY = 0, 1, 2, 99
GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.mark.parametrize("kernel", [ST, RO, SR])
def test_theta_zero_is_direct_sum(orc, kernel):
    x, f = wl.uniform_cube(1200, 21, win=orc.kernel_win(kernel))
    ud = orc.direct(kernel, 0.05, x, x, f)
    ut, cnt = orc.treecode(x, f, kernel, 0.05, 0.0, 3, 100)
    assert cnt[2] == 0 and cnt[0] == len(x) ** 2
    assert orc.rel_l2(ud, ut) < 1e-14


@pytest.mark.parametrize("n,exact", [(3, True), (5, True), (2, False)])
def test_polynomial_kernel_reproduced_exactly(orc, n, exact):
    # the test kernel has degree 3 in each y_l: the far field of Eq.
    # pc_approximation_3D is exact for n >= 3 at any theta (Sec. 2), so the
    # treecode equals the direct sum to roundoff; n = 2 is not exact.
    x, f = wl.uniform_cube(3000, 22)
    ud = orc.direct(POLY, 0.0, x, x, f)
    ut, cnt = orc.treecode(x, f, POLY, 0.0, 0.9, n, 50)
    assert cnt[2] > 0
    e = orc.rel_l2(ud, ut)
    assert (e < 1e-12) if exact else (e > 1e-6)


@pytest.mark.parametrize("theta", [0.3, 0.7, 0.95])
def test_each_source_counted_once(orc, theta):
    x, f = wl.uniform_cube(2500, 23)
    t = orc.Tree(x, 60)
    fh = t.modified_weights(f, 2)
    _, cnt = t.treecode(f, fh, 2, ST, 0.01, theta, x)
    assert cnt[0] + cnt[4] == len(x) ** 2
    assert cnt[1] == 27 * cnt[2]


def test_single_leaf_is_direct(orc):
    x, f = wl.uniform_cube(400, 24)
    ud = orc.direct(ST, 0.01, x, x, f)
    ut, cnt = orc.treecode(x, f, ST, 0.01, 0.7, 4, 400)
    assert cnt[2] == 0
    assert orc.rel_l2(ud, ut) < 1e-14


def test_error_falls_with_degree(orc):
    x, f = wl.uniform_cube(4000, 25)
    ud = orc.direct(ST, 0.01, x, x, f)
    errs = [orc.rel_l2(ud, orc.treecode(x, f, ST, 0.01, 0.7, n, 100)[0]) for n in (1, 3, 5, 7)]
    assert all(a > b for a, b in zip(errs[:-1], errs[1:])), errs
    assert errs[-1] < 3e-5


def test_separate_targets(orc):
    # targets need not be sources (Sec. 8)
    x, f = wl.uniform_cube(2000, 26)
    y, _ = wl.uniform_cube(300, 27, -1.5, 1.5)
    ud = orc.direct(SR, 0.1, y, x, np.hstack([f, f[::-1]]))
    ut, _ = orc.treecode(x, np.hstack([f, f[::-1]]), SR, 0.1, 0.6, 6, 100, tgt=y)
    assert orc.rel_l2(ud, ut) < 1e-4


def test_example1_error_order_of_magnitude(orc):
    # Table CaseI_new: N = 10K, theta = 0.7, n = 7, N0 = 2000, eps = 0.02 -> E = 2.25e-6.
    rows = np.loadtxt(os.path.join(GOLDEN, "table_caseI_new.txt"))
    E_paper = dict(zip(rows[:, 0].astype(int), rows[:, 1]))[10000]
    x, f = wl.organisms(5000, 28)
    ud = orc.direct(ST, 0.02, x, x, f)
    ut, _ = orc.treecode(x, f, ST, 0.02, 0.7, 7, 2000)
    E = orc.rel_l2(ud, ut)
    assert E_paper / 10 < E < E_paper * 10, (E, E_paper)


def test_batch_of_one_is_per_target(orc):
    # with one target per batch the batch box is a point and the batch MAC is Eq. MAC
    x, f = wl.uniform_cube(1500, 29)
    t = orc.Tree(x, 80)
    fh = t.modified_weights(f, 4)
    u1, c1 = t.treecode(f, fh, 4, ST, 0.01, 0.7, x)
    r = t.treecode_batch(f, fh, 4, ST, 0.01, 0.7, x, 1, 1)
    assert np.array_equal(c1, r["counts"])
    assert orc.rel_l2(u1, r["out"]) < 1e-14


@pytest.mark.parametrize("batch", [16, 64])
def test_batch_lists_are_valid(orc, batch):
    x, f = wl.uniform_cube(3000, 30)
    t = orc.Tree(x, 100)
    fh = t.modified_weights(f, 3)
    r = t.treecode_batch(f, fh, 3, ST, 0.01, 0.7, x, batch, batch, lists=True)
    assert r["counts"][0] + r["counts"][4] == len(x) ** 2
    ctr = 0.5 * (t.lo + t.hi)
    rad = 0.5 * np.linalg.norm(t.hi - t.lo, axis=1)
    of = on = 0
    for b in range(len(r["nfar"])):
        tg = x[r["tperm"][b * batch:(b + 1) * batch]]
        far = r["far_list"][of:of + r["nfar"][b]]
        near = r["near_list"][on:on + r["nnear"][b]]
        of += r["nfar"][b]
        on += r["nnear"][b]
        assert np.all(t.n_child[near] == 0)
        for c in far:  # a batch-accepted cluster passes Eq. MAC for every target
            R = np.linalg.norm(tg - ctr[c], axis=1)
            assert np.all(rad[c] <= 0.7 * R)
        # the far and near clusters cover every source exactly once
        cover = np.zeros(len(x), int)
        for c in np.concatenate([far, near]):
            cover[t.begin[c]:t.end[c]] += 1
        assert np.all(cover == 1)
    ud = orc.direct(ST, 0.01, x, x, f)
    # the batch traversal only refines where the per-target one accepts, so it
    # is at least about as accurate
    up, _ = t.treecode(f, fh, 3, ST, 0.01, 0.7, x)
    assert orc.rel_l2(ud, r["out"]) < 1.05 * orc.rel_l2(ud, up)


def test_variable_degree_uniform_equals_fixed(orc):
    x, f = wl.uniform_cube(3000, 31)
    t = orc.Tree(x, 100)
    n = 4
    fh = t.modified_weights(f, n)
    deg = np.full(t.nclusters, n, np.int32)
    fv, foff = t.modified_weights_var(f, deg)
    assert np.array_equal(fv, fh.ravel())
    u1, c1 = t.treecode(f, fh, n, ST, 0.01, 0.7, x)
    u2, c2, bad = t.treecode_var(f, fv, deg, foff, ST, 0.01, 0.7, x)
    assert bad == 0 and np.array_equal(u1, u2) and np.array_equal(c1, c2)


def test_variable_degree_polynomial_kernel_exact(orc):
    # every accepted cluster with n_c >= 3 reproduces the degree-3 test kernel
    x, f = wl.uniform_cube(3000, 32)
    t = orc.Tree(x, 60)
    g = np.random.default_rng(3)
    deg = g.integers(3, 7, t.nclusters).astype(np.int32)
    fv, foff = t.modified_weights_var(f, deg)
    u, cnt, bad = t.treecode_var(f, fv, deg, foff, POLY, 0.0, 0.9, x)
    assert bad == 0 and cnt[2] > 0
    # far grid points counted with each cluster's own degree
    assert cnt[1] != 64 * cnt[2]
    assert orc.rel_l2(orc.direct(POLY, 0.0, x, x, f), u) < 1e-12
    deg2 = deg.copy()
    deg2[deg2 == 3] = 2   # one degree too low somewhere: no longer exact
    fv2, foff2 = t.modified_weights_var(f, deg2)
    u2, _, _ = t.treecode_var(f, fv2, deg2, foff2, POLY, 0.0, 0.9, x)
    assert orc.rel_l2(orc.direct(POLY, 0.0, x, x, f), u2) > 1e-8


def test_variable_degree_batch_matches_per_target_form(orc):
    x, f = wl.uniform_cube(2000, 33)
    t = orc.Tree(x, 80)
    deg = np.random.default_rng(4).integers(2, 9, t.nclusters).astype(np.int32)
    fv, foff = t.modified_weights_var(f, deg)
    u1, c1, _ = t.treecode_var(f, fv, deg, foff, ST, 0.01, 0.7, x)
    u2, c2 = t.treecode_batch_var(f, fv, deg, foff, ST, 0.01, 0.7, x, 1, 1)
    assert np.array_equal(c1, c2) and orc.rel_l2(u1, u2) < 1e-14


def test_all_targets_rule_batch_of_one_is_per_target(orc):
    # with one target per batch the all-targets rule is Eq. MAC itself
    x, f = wl.uniform_cube(1500, 34)
    t = orc.Tree(x, 80)
    fh = t.modified_weights(f, 4)
    u1, c1 = t.treecode(f, fh, 4, ST, 0.01, 0.7, x)
    r = t.treecode_batch(f, fh, 4, ST, 0.01, 0.7, x, 1, 1, all_targets=True)
    assert np.array_equal(c1, r["counts"])
    assert orc.rel_l2(u1, r["out"]) < 1e-14


@pytest.mark.parametrize("batch", [16, 64])
def test_all_targets_rule_lists(orc, batch):
    """Every accepted cluster passes Eq. MAC for each target of its batch; a
    cluster that fails it for some target is never accepted for the batch; the
    lists cover every source once per target; the work lies between the
    per-target MAC's and the box rule's."""
    x, f = wl.uniform_cube(3000, 35)
    t = orc.Tree(x, 100)
    fh = t.modified_weights(f, 3)
    r = t.treecode_batch(f, fh, 3, ST, 0.01, 0.7, x, batch, batch, lists=True, all_targets=True)
    rb = t.treecode_batch(f, fh, 3, ST, 0.01, 0.7, x, batch, batch, all_targets=False)
    _, cp = t.treecode(f, fh, 3, ST, 0.01, 0.7, x)
    assert r["counts"][0] + r["counts"][4] == len(x) ** 2
    work = lambda c: c[0] + c[1]  # noqa: E731
    assert work(cp) <= work(r["counts"]) <= work(rb["counts"])
    ctr = 0.5 * (t.lo + t.hi)
    rad = 0.5 * np.linalg.norm(t.hi - t.lo, axis=1)
    of = on = 0
    for b in range(len(r["nfar"])):
        tg = x[r["tperm"][b * batch:(b + 1) * batch]]
        far = r["far_list"][of:of + r["nfar"][b]]
        near = r["near_list"][on:on + r["nnear"][b]]
        of += r["nfar"][b]
        on += r["nnear"][b]
        for c in far:
            assert np.all(rad[c] <= 0.7 * np.linalg.norm(tg - ctr[c], axis=1))
        for c in near:  # a leaf kept near fails Eq. MAC for some target
            assert np.any(rad[c] > 0.7 * np.linalg.norm(tg - ctr[c], axis=1))
        cover = np.zeros(len(x), int)
        for c in np.concatenate([far, near]):
            cover[t.begin[c]:t.end[c]] += 1
        assert np.all(cover == 1)
