"""Pins of the oracle's degree-selector inputs (oracle/learn.py): features of a
hand-computed cluster, the far-field error's exactness where interpolation is
exact (Sec. 3: a degree-n interpolant reproduces polynomials of degree <= n),
its decay with n, and the sampling rule."""
import math

import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl

ST, POLY = 0, 99


@pytest.fixture(scope="module")
def L(orc):
    from oracle import learn
    return learn


def test_splitmix_unit_properties(L):
    u = L.splitmix_unit(7, np.zeros(100000, np.int64), np.arange(100000))
    assert u.min() >= 0.0 and u.max() < 1.0
    assert abs(u.mean() - 0.5) < 0.005 and abs(u.var() - 1.0 / 12) < 0.002
    assert np.array_equal(u, L.splitmix_unit(7, np.zeros(100000, np.int64), np.arange(100000)))
    v = L.splitmix_unit(8, np.zeros(100000, np.int64), np.arange(100000))
    w = L.splitmix_unit(7, np.ones(100000, np.int64), np.arange(100000))
    assert abs(np.corrcoef(u, v)[0, 1]) < 0.02 and abs(np.corrcoef(u, w)[0, 1]) < 0.02


def test_features_hand_case(orc, L):
    # eight sources at the corners of the unit cube: one leaf, the root
    x = np.array([[i, j, k] for i in (0, 1) for j in (0, 1) for k in (0, 1)], np.float64)
    f = np.tile([1.0, 0.0, 0.0], (8, 1))
    f[0] = [0.0, 2.0, 0.0]
    tg = np.array([[10.0, 0.5, 0.5], [12.0, 0.5, 0.5]])
    t = orc.Tree(x, 8)
    assert t.nclusters == 1
    lists = t.treecode_batch(f, t.modified_weights(f, 2), 2, ST, 0.01, 0.7, tg, 64, 64,
                             lists=True, evaluate=False)
    assert list(lists["far_list"]) == [0]     # r = sqrt(3)/2 <= 0.7 * 9.5
    F = L.features(t, f, tg, lists, 64, 0.01)[0]
    r = math.sqrt(3) / 2
    q = [r / 9.5, r / 11.5]
    want = [math.log(9), math.log(r), min(q), sum(q) / 2, max(q), 0.01 / r,
            math.log(1e-30 + math.sqrt(7 ** 2 + 2 ** 2)), math.log(1e-30 + 9.0),
            math.log(1e-30 + 2.0), 1.0, 1.0, 0.0]
    assert np.allclose(F, want, rtol=1e-14, atol=1e-15)


def _far_errors(orc, L, x, f, kernel, n, tg, S, seed, leaf=200, B=64):
    t = orc.Tree(x, leaf)
    lists = t.treecode_batch(f, t.modified_weights(f, 1), 1, kernel, 0.01, 0.7, tg, B, B,
                             lists=True, evaluate=False)
    fh = t.modified_weights(f, n)
    return L.far_errors(t, f, lambda c: fh[c].reshape(-1, 3), lambda c: n, kernel, 0.01, tg, lists,
                        B, S, seed), t, lists


def test_far_error_vanishes_for_polynomial_kernel(orc, L):
    x, f = wl.uniform_cube(3000, 81)
    tg = wl.uniform_cube(1500, 82)[0]
    (e3, n3), t, lists = _far_errors(orc, L, x, f, POLY, 3, tg, 8, 5)
    (e1, n1), _, _ = _far_errors(orc, L, x, f, POLY, 1, tg, 8, 5)
    assert n3.sum() > 0 and np.array_equal(n1, n3)
    assert e3.sum() <= 1e-24 * max(e1.sum(), 1.0) + 1e-26   # exact at n = 3
    assert e1.sum() > 1e-10                                  # the cubic is not linear


def test_far_error_decays_with_degree_and_sample_rule(orc, L):
    x, f = wl.uniform_cube(3000, 83)
    tg = wl.uniform_cube(1500, 84)[0]
    errs = []
    for n in (2, 5, 8):
        (e, ns), t, lists = _far_errors(orc, L, x, f, ST, n, tg, 8, 9)
        errs.append(e.sum())
    assert errs[0] > 20 * errs[1] > 0 and errs[1] > 20 * errs[2] > 0
    acc = L.accepting_targets(t, lists, len(tg), 64)
    sizes = np.array([len(a) for a in acc])
    assert np.all(ns <= sizes) and np.all(ns[sizes <= 8] == sizes[sizes <= 8])
    # with S above every count, every accepting target is taken
    (_, ns_all), _, _ = _far_errors(orc, L, x, f, ST, 2, tg, 10 ** 9, 9)
    assert np.array_equal(ns_all, sizes)
