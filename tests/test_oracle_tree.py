"""Pins of the oracle's tree (Sec. 6) and modified weights (Sec. 4-5,
Eq. modified_weights): structural invariants, the leaf counts the paper
states, polynomial exactness (partition of unity and moments)."""
import math

import numpy as np
import pytest

from paper_1902_02250_gb300 import workloads as wl


def _check_tree_invariants(orc, t, x, N0):
    m = t.nclusters
    assert t.begin[0] == 0 and t.end[0] == len(x)
    # root box: smallest box enclosing the particles
    np.testing.assert_array_equal(t.lo[0], x.min(axis=0))
    np.testing.assert_array_equal(t.hi[0], x.max(axis=0))
    assert sorted(t.perm.tolist()) == list(range(len(x)))
    for c in range(m):
        idx = t.perm[t.begin[c]:t.end[c]]
        pts = x[idx]
        assert np.all(pts >= t.lo[c]) and np.all(pts <= t.hi[c])
        cnt = t.end[c] - t.begin[c]
        assert cnt > 0
        if t.n_child[c] == 0:
            assert cnt <= N0 or t.level[c] >= 40
            # every split is a stable partition and the root starts in user
            # order, so each leaf lists its particles in increasing user index
            assert np.all(np.diff(idx) > 0)
            continue
        assert cnt > N0
        ch = range(t.first_child[c], t.first_child[c] + t.n_child[c])
        # children tile the parent range in order, each one level deeper
        assert t.begin[ch[0]] == t.begin[c] and t.end[ch[-1]] == t.end[c]
        for a, b in zip(ch[:-1], ch[1:]):
            assert t.end[a] == t.begin[b]
        for k in ch:
            assert t.parent[k] == c and t.level[k] == t.level[c] + 1
        # Sec. 6 bisection: sides > l_max/sqrt(2) are halved, others kept
        side = t.hi[c] - t.lo[c]
        split = side > side.max() / math.sqrt(2.0)
        assert t.n_child[c] <= 2 ** split.sum()
        for k in ch:
            ks = t.hi[k] - t.lo[k]
            for l in range(3):
                if split[l]:
                    mid = 0.5 * (t.lo[c, l] + t.hi[c, l])
                    assert t.lo[k, l] in (t.lo[c, l], mid) and t.hi[k, l] in (mid, t.hi[c, l])
                    assert abs(ks[l] - 0.5 * side[l]) <= 1e-15 * side[l]
                else:
                    assert t.lo[k, l] == t.lo[c, l] and t.hi[k, l] == t.hi[c, l]


def test_small_tree_invariants(orc):
    x, _ = wl.uniform_cube(3000, 1)
    t = orc.Tree(x, 100)
    _check_tree_invariants(orc, t, x, 100)


def test_root_level_partition_is_stable(orc):
    x, _ = wl.uniform_cube(500, 2)
    t = orc.Tree(x, 100)
    for k in range(t.first_child[0], t.first_child[0] + t.n_child[0]):
        assert np.all(np.diff(t.perm[t.begin[k]:t.end[k]]) > 0)


def test_single_leaf_when_n_le_N0(orc):
    x, _ = wl.uniform_cube(500, 3)
    t = orc.Tree(x, 500)
    assert t.nclusters == 1 and t.n_child[0] == 0
    np.testing.assert_array_equal(t.perm, np.arange(500))


def test_paper_leaf_count_uniform_cube(orc):
    # Sec. 8.1: N0 = 2000 in a cube gives 8 children per cluster and leaves of
    # about N / 8^d = 1250 particles; N = 640K -> depth 3, 512 leaves.
    x, _ = wl.uniform_cube(640_000, 4, 0.0, 10.0)
    t = orc.Tree(x, 2000)
    leaves = np.flatnonzero(t.n_child == 0)
    assert len(leaves) == 512
    assert np.all(t.level[leaves] == 3)
    assert np.all(t.n_child[t.n_child > 0] == 8)
    sizes = t.end[leaves] - t.begin[leaves]
    assert abs(sizes.mean() - 1250) < 1e-9 and sizes.max() <= 2000


def test_slab_gives_four_children(orc):
    # Sec. 6 / Example 2: a slab is bisected in its long directions only.
    g = np.random.default_rng(9)
    x = np.column_stack([g.uniform(0, 16, 20000), g.uniform(0, 16, 20000), g.uniform(0, 9, 20000)])
    t = orc.Tree(x, 1000)
    assert t.n_child[0] == 4
    assert np.all(t.hi[1:5, 2] - t.lo[1:5, 2] == t.hi[0, 2] - t.lo[0, 2])
    _check_tree_invariants(orc, t, x, 1000)


def test_degenerate_identical_points(orc):
    x = np.ones((50, 3))
    t = orc.Tree(x, 10)
    assert t.nclusters == 1 and t.n_child[0] == 0


def test_midpoint_tie_goes_up(orc):
    x = np.array([[0.0, 0, 0], [2.0, 2, 2], [1.0, 1, 1]])  # the last one sits on the midpoint
    t = orc.Tree(x, 1)
    # children by octant code: code 0 holds particle 0; code 7 holds 2 then 1 is split again
    first = t.first_child[0]
    assert t.perm[t.begin[first]] == 0
    assert set(t.perm[t.begin[first + 1]:t.end[first + 1]].tolist()) == {1, 2}


@pytest.mark.parametrize("n", [1, 3, 6])
def test_modified_weights_moments(orc, n):
    # Eq. modified_weights reproduces all moments y^alpha with alpha_l <= n:
    # sum_k s_k^alpha fhat_k = sum_j y_j^alpha f_j (polynomial exactness, Sec. 2).
    x, f = wl.uniform_cube(1500, 5)
    t = orc.Tree(x, 200)
    fh = t.modified_weights(f, n)
    g = np.random.default_rng(n)
    for c in [0] + list(g.choice(t.nclusters, 4, replace=False)):
        s = t.cluster_points(c, n)
        y = x[t.perm[t.begin[c]:t.end[c]]]
        fj = f[t.perm[t.begin[c]:t.end[c]]]
        ctr = 0.5 * (t.lo[c] + t.hi[c])
        for alpha in [(0, 0, 0), (n, 0, 0), (1, min(1, n), 0), (n, n, n), (0, n, min(2, n))]:
            ys = np.prod((y - ctr) ** np.array(alpha), axis=1)
            lhs = np.einsum("abcq,a,b,c->q", fh[c], (s[0] - ctr[0]) ** alpha[0],
                            (s[1] - ctr[1]) ** alpha[1], (s[2] - ctr[2]) ** alpha[2])
            rhs = ys @ fj
            scale = np.abs(ys)[:, None].T @ np.abs(fj)
            np.testing.assert_allclose(lhs, rhs, rtol=0, atol=1e-12 * scale.max() + 1e-300)
        # not exact one degree higher (sensitivity of the pin)
        a = (n + 1, 0, 0)
        ys = np.prod((y - ctr) ** np.array(a), axis=1)
        lhs = np.einsum("abcq,a->q", fh[c].sum(axis=(1, 2))[:, None, None, :],
                        (s[0] - ctr[0]) ** a[0])
        assert np.abs(lhs - ys @ fj).max() > 1e-10 * (np.abs(ys) @ np.abs(fj)).max()


def test_modified_weights_partition_of_unity(orc):
    x, f = wl.uniform_cube(2000, 6)
    t = orc.Tree(x, 300)
    fh = t.modified_weights(f, 5)
    for c in range(t.nclusters):
        fj = f[t.perm[t.begin[c]:t.end[c]]]
        np.testing.assert_allclose(fh[c].sum(axis=(0, 1, 2)), fj.sum(axis=0), rtol=0,
                                   atol=1e-12 * np.abs(fj).sum())


def test_particle_on_grid_point_puts_weight_there(orc):
    # coincident-point branch inside Eq. modified_weights
    n = 4
    s = orc.cheb_points(n, 0.0, 1.0)
    x = np.array([[0.0, 0.0, 0.0], [1.0, 1.0, 1.0], [s[1], s[3], s[2]]])
    f = np.array([[0.0, 0, 0], [0.0, 0, 0], [1.0, 2.0, 3.0]])
    t = orc.Tree(x, 10)
    fh = t.modified_weights(f, n)[0]
    # grid point (k1, k2, k3) = (1, 3, 2) holds the whole weight
    assert np.array_equal(fh[1, 3, 2], f[2])
    fh[1, 3, 2] = 0
    assert np.all(fh == 0)
