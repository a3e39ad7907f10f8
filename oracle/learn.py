"""Plain numpy reference of the degree selector's inputs (FP64).

Test infrastructure, like the rest of ``oracle/``: only tests and the
benchmark's CPU leg use it.  For a source tree and the batch-MAC interaction
lists of ``Tree.treecode_batch(..., lists=True)`` it computes

* the 12 features of every cluster (the definitions, one cluster at a time):
  log(1 + N_c), log r_c, min / mean / max of r_c / |x - y_c| over the targets
  x that accept c, min(eps / r_c, 10), log |sum f|, log sum |f|, log max |f|,
  middle / longest and shortest / longest box side, and the level;
* the far-field error of every cluster on sampled accepting targets: the
  cluster's far field (Eq. pc_approximation_3D: a direct sum over its tensor
  grid of Chebyshev points with the modified weights as charges) minus the
  direct sum over its own sources (Eq. pc_interaction_3D).

The sample of targets is drawn with SplitMix64 (Steele, Lea and Flood, 2014),
written here from its definition: z = key + 0x9e3779b97f4a7c15, then
z = (z ^ z >> 30) * 0xbf58476d1ce4e5b9, z = (z ^ z >> 27) * 0x94d049bb133111eb,
z ^= z >> 31; the unit number is (z >> 11) * 2^-53.  The key of (seed, cluster
c, target slot s) is seed ^ (c << 32) ^ s, and a target is taken when the unit
number is below min(1, S / number of accepting targets).
"""
import numpy as np

from . import oracle as _o

_M64 = (1 << 64) - 1


def splitmix_unit(seed, c, slot):
    """Unit numbers in [0, 1) of the keys seed ^ (c << 32) ^ slot (arrays)."""
    c = np.asarray(c, np.uint64)
    slot = np.asarray(slot, np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(int(seed) & _M64) ^ (c << np.uint64(32)) ^ slot
        z = z + np.uint64(0x9e3779b97f4a7c15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xbf58476d1ce4e5b9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94d049bb133111eb)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def accepting_targets(tree, lists, nt, batch):
    """For each cluster: the target slots (target-tree order) that accept it
    under the batch MAC, from the per-batch far lists."""
    acc = [[] for _ in range(tree.nclusters)]
    off = 0
    for b, k in enumerate(lists["nfar"]):
        s0, s1 = b * batch, min(nt, (b + 1) * batch)
        for c in lists["far_list"][off:off + k]:
            acc[int(c)].extend(range(s0, s1))
        off += k
    return [np.asarray(a, np.int64) for a in acc]


def cluster_centre_radius(tree, c):
    """Centre of the box and its half diagonal (the cluster radius of Sec. 6)."""
    lo, hi = tree.lo[c], tree.hi[c]
    ctr = 0.5 * (lo + hi)
    return ctr, 0.5 * float(np.sqrt(((hi - lo) ** 2).sum()))


def features(tree, w, tgt, lists, batch, eps):
    """n_clusters x 12 features in FP64 (rounded to FP32 by the caller if needed)."""
    w = np.asarray(w, np.float64)
    tgt = np.asarray(tgt, np.float64)
    nt = len(tgt)
    tx = tgt[lists["tperm"]]                       # target slot order
    acc = accepting_targets(tree, lists, nt, batch)
    F = np.zeros((tree.nclusters, 12))
    for c in range(tree.nclusters):
        ctr, r = cluster_centre_radius(tree, c)
        idx = tree.perm[tree.begin[c]:tree.end[c]]
        f = w[idx]
        fn = np.sqrt((f ** 2).sum(axis=1))
        F[c, 0] = np.log1p(len(idx))
        F[c, 1] = np.log(max(r, 1e-12))
        if len(acc[c]):
            R = np.sqrt(((tx[acc[c]] - ctr) ** 2).sum(axis=1))
            q = np.where(R > 0, r / np.where(R > 0, R, 1.0), 0.0)
            F[c, 2], F[c, 3], F[c, 4] = q.min(), q.mean(), q.max()
        F[c, 5] = min(eps / max(r, 1e-300), 10.0)
        F[c, 6] = np.log(1e-30 + np.sqrt((f.sum(axis=0) ** 2).sum()))
        F[c, 7] = np.log(1e-30 + fn.sum())
        F[c, 8] = np.log(1e-30 + fn.max())
        side = np.sort(tree.hi[c] - tree.lo[c])[::-1]
        F[c, 9] = side[1] / side[0] if side[0] > 0 else 1.0
        F[c, 10] = side[2] / side[0] if side[0] > 0 else 1.0
        F[c, 11] = tree.level[c]
    return F


def grid_points(tree, c, n):
    """The (n+1)^3 tensor grid of cluster c, k1 slowest (the weights' order)."""
    s = tree.cluster_points(c, n)
    g = np.stack(np.meshgrid(s[0], s[1], s[2], indexing="ij"), axis=-1)
    return g.reshape(-1, 3)


def far_errors(tree, w, fhat_of, degree_of, kernel, eps, tgt, lists, batch, S, seed):
    """(err2, n_samples) per cluster.  fhat_of(c) gives cluster c's modified
    weights ((n_c+1)^3 x w_in, k1 slowest); degree_of(c) its degree."""
    w = np.asarray(w, np.float64)
    tgt = np.asarray(tgt, np.float64)
    nt = len(tgt)
    tx = tgt[lists["tperm"]]
    acc = accepting_targets(tree, lists, nt, batch)
    m = tree.nclusters
    err2 = np.zeros(m)
    ns = np.zeros(m, np.int64)
    for c in range(m):
        a = acc[c]
        if len(a) == 0:
            continue
        pc = min(1.0, float(S) / float(max(len(a), 1)))
        take = a[splitmix_unit(seed, c, a) < pc]
        if len(take) == 0:
            continue
        n = degree_of(c)
        far = _o.direct(kernel, eps, tx[take], grid_points(tree, c, n), fhat_of(c))
        idx = tree.perm[tree.begin[c]:tree.end[c]]
        near = _o.direct(kernel, eps, tx[take], tree.x[idx], w[idx])
        err2[c] = ((far - near) ** 2).sum()
        ns[c] = len(take)
    return err2, ns
