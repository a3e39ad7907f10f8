"""ctypes binding of ``kitc_oracle.c`` -- the plain FP64 CPU oracle.

Test infrastructure: only ``tests/``, ``__graft_entry__.smoke`` and the
CPU-baseline leg of ``bench.py`` may call it.  It shares no code with the
CUDA library.  Each wrapper names the passage of the paper that its C
function follows (see the C source for the full statement).
"""
import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "kitc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle_kitc.so")

STOKESLET, ROTLET, STOKESLET_ROTLET, TEST_POLY = 0, 1, 2, 99

_lib = None


def build(force=False):
    """Compile the oracle with gcc: FP64, no FMA contraction, OpenMP."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp", "-fPIC",
           "-shared", "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = ctypes.CDLL(_LIB_PATH)
        P, I64, I, D = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int, ctypes.c_double
        L.or_kernel_win.argtypes = [I]
        L.or_kernel_wout.argtypes = [I]
        L.or_num_threads.restype = I
        L.or_set_num_threads.argtypes = [I]
        L.or_cheb_points.argtypes = [I, D, D, P]
        L.or_bary_weights.argtypes = [I, P]
        L.or_bary_basis.argtypes = [I, P, P, D, P]
        L.or_mrs_functions.argtypes = [D, D, P]
        L.or_kernel_apply.argtypes = [I, D, P, P, P, P]
        L.or_direct.argtypes = [I, D, P, I64, P, P, I64, P]
        L.or_rel_l2.argtypes = [P, P, I64, I]
        L.or_rel_l2.restype = D
        L.or_tree_build.argtypes = [P, I64, I]
        L.or_tree_build.restype = P
        L.or_tree_free.argtypes = [P]
        L.or_tree_nclusters.argtypes = [P]
        L.or_tree_nclusters.restype = I64
        L.or_tree_get.argtypes = [P] * 10
        L.or_cluster_points.argtypes = [P, I64, I, P]
        L.or_modified_weights.argtypes = [P, P, P, I, I, P]
        L.or_treecode.argtypes = [P, P, P, P, I, I, D, D, P, I64, P, P]
        L.or_modified_weights_var.argtypes = [P, P, P, I, P, P, P]
        L.or_treecode_var.argtypes = [P, P, P, P, P, P, I, D, D, P, I64, P, P]
        L.or_treecode_var.restype = I64
        L.or_treecode_batch_var.argtypes = [P, P, P, P, P, P, I, D, D, P, I64, I, I, P, P, P]
        L.or_num_batches.argtypes = [I64, I]
        L.or_num_batches.restype = I64
        L.or_treecode_batch.argtypes = [P, P, P, P, I, I, D, D, P, I64, I, I, I, P, P, P, P,
                                        P, P, P, I64, P, I64]
        L.or_treecode_batch_all.argtypes = L.or_treecode_batch.argtypes
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def num_threads():
    return lib().or_num_threads()


def set_num_threads(n):
    lib().or_set_num_threads(int(n))


def kernel_win(kernel):
    return lib().or_kernel_win(kernel)


def kernel_wout(kernel):
    return lib().or_kernel_wout(kernel)


def cheb_points(n, a=-1.0, b=1.0):
    """Eq. Chebyshev_points mapped to [a, b] (Sec. 3 interval map)."""
    s = np.empty(n + 1)
    lib().or_cheb_points(n, a, b, _p(s))
    return s


def bary_weights(n):
    """Eq. barycentric_weights (simple weights)."""
    w = np.empty(n + 1)
    lib().or_bary_weights(n, _p(w))
    return w


def bary_basis(s, w, t):
    """Eq. Barycentric-1D with the DBL_MIN coincident-point rule (Sec. 3, 5)."""
    s, w = _f64(s), _f64(w)
    L = np.empty(len(s))
    lib().or_bary_basis(len(s) - 1, _p(s), _p(w), float(t), _p(L))
    return L


def mrs_functions(r2, eps):
    """Eq. MRS_kernels: (H1, H2, Q, D1, D2) at r^2."""
    H = np.empty(5)
    lib().or_mrs_functions(float(r2), float(eps), _p(H))
    return H


def kernel_apply(kernel, eps, x, y, f):
    """One summand k(x, y) f of Eq. N-body (Eqs. Velocity_1, MRS_2)."""
    x, y, f = _f64(x), _f64(y), _f64(f)
    u = np.zeros(kernel_wout(kernel))
    lib().or_kernel_apply(kernel, float(eps), _p(x), _p(y), _p(f), _p(u))
    return u


def direct(kernel, eps, tgt, src, w):
    """Eq. N-body by direct summation (self term kept; MRS kernels are regular)."""
    tgt, src = _f64(tgt, (-1, 3)), _f64(src, (-1, 3))
    w = _f64(w, (len(src), kernel_win(kernel)))
    out = np.empty((len(tgt), kernel_wout(kernel)))
    lib().or_direct(kernel, float(eps), _p(tgt), len(tgt), _p(src), _p(w), len(src), _p(out))
    return out


def rel_l2(ud, ut):
    """Eq. error: relative L2 error of ut against ud (rows concatenated)."""
    ud, ut = _f64(ud), _f64(ut)
    assert ud.shape == ut.shape
    m = ud.shape[1] if ud.ndim == 2 else 1
    return lib().or_rel_l2(_p(ud), _p(ut), ud.shape[0], m)


class Tree:
    """Sec. 6 tree: BFS-numbered clusters, children contiguous and ordered by
    octant code; particles permuted into contiguous cluster ranges."""

    def __init__(self, x, leaf_size):
        self.x = _f64(x, (-1, 3))
        self.n = len(self.x)
        self.leaf_size = int(leaf_size)
        self._h = lib().or_tree_build(_p(self.x), self.n, self.leaf_size)
        m = lib().or_tree_nclusters(self._h)
        self.nclusters = m
        self.perm = np.empty(self.n, np.int64)
        self.lo = np.empty((m, 3))
        self.hi = np.empty((m, 3))
        self.begin = np.empty(m, np.int64)
        self.end = np.empty(m, np.int64)
        self.first_child = np.empty(m, np.int32)
        self.n_child = np.empty(m, np.int32)
        self.level = np.empty(m, np.int32)
        self.parent = np.empty(m, np.int32)
        lib().or_tree_get(self._h, _p(self.perm), _p(self.lo), _p(self.hi), _p(self.begin),
                          _p(self.end), _p(self.first_child), _p(self.n_child),
                          _p(self.level), _p(self.parent))

    def __del__(self):
        h = getattr(self, "_h", None)
        if h and _lib is not None:
            _lib.or_tree_free(h)
            self._h = None

    @property
    def is_leaf(self):
        return self.n_child == 0

    def cluster_points(self, c, n):
        """The (n+1) mapped Chebyshev points of each axis of cluster c."""
        s = np.empty((3, n + 1))
        lib().or_cluster_points(self._h, int(c), n, _p(s))
        return s

    def modified_weights(self, w, n):
        """Eq. modified_weights for every cluster: [cluster][k1][k2][k3][comp]."""
        w = _f64(w, (self.n, -1))
        win = w.shape[1]
        np1 = n + 1
        fhat = np.empty((self.nclusters, np1, np1, np1, win))
        lib().or_modified_weights(self._h, _p(self.x), _p(w), win, n, _p(fhat))
        return fhat

    def weight_offsets(self, deg, win):
        """Offsets (in doubles) of each cluster's weights for per-cluster degrees."""
        deg = np.asarray(deg, np.int64)
        sizes = np.where(deg > 0, (deg + 1) ** 3 * win, 0)
        return np.concatenate([[0], np.cumsum(sizes)[:-1]]).astype(np.int64), int(sizes.sum())

    def modified_weights_var(self, w, deg):
        """Eq. modified_weights with degree deg[c] per cluster (0: none).
        Returns (flat fhat, offsets)."""
        w = _f64(w, (self.n, -1))
        win = w.shape[1]
        deg = np.ascontiguousarray(deg, np.int32)
        foff, tot = self.weight_offsets(deg, win)
        fhat = np.zeros(max(tot, 1))
        lib().or_modified_weights_var(self._h, _p(self.x), _p(w), win, _p(deg), _p(foff), _p(fhat))
        return fhat, foff

    def treecode_var(self, w, fhat, deg, foff, kernel, eps, theta, tgt):
        """Algorithm 2 with a degree per cluster; returns (out, counts, bad) where
        bad counts far interactions with clusters of degree 0 (must be 0)."""
        w = _f64(w, (self.n, kernel_win(kernel)))
        deg = np.ascontiguousarray(deg, np.int32)
        foff = np.ascontiguousarray(foff, np.int64)
        tgt = _f64(tgt, (-1, 3))
        out = np.empty((len(tgt), kernel_wout(kernel)))
        cnt = np.zeros(5, np.int64)
        bad = lib().or_treecode_var(self._h, _p(self.x), _p(w), _p(_f64(fhat)), _p(deg), _p(foff),
                                    kernel, float(eps), float(theta), _p(tgt), len(tgt), _p(out),
                                    _p(cnt))
        return out, cnt, bad

    def treecode_batch_var(self, w, fhat, deg, foff, kernel, eps, theta, tgt, batch, tgt_leaf,
                           select=None):
        """Batch-MAC variant with a degree per cluster; returns (out, counts)."""
        w = _f64(w, (self.n, kernel_win(kernel)))
        deg = np.ascontiguousarray(deg, np.int32)
        foff = np.ascontiguousarray(foff, np.int64)
        tgt = _f64(tgt, (-1, 3))
        nt = len(tgt)
        out = np.empty((nt, kernel_wout(kernel)))
        cnt = np.zeros(5, np.int64)
        sel = None
        if select is not None:
            sel = np.zeros(nt, np.uint8)
            sel[np.asarray(select)] = 1
        lib().or_treecode_batch_var(self._h, _p(self.x), _p(w), _p(_f64(fhat)), _p(deg), _p(foff),
                                    kernel, float(eps), float(theta), _p(tgt), nt, batch, tgt_leaf,
                                    _p(sel), _p(out), _p(cnt))
        return out, cnt

    def treecode(self, w, fhat, n, kernel, eps, theta, tgt):
        """Algorithm 2 (per-target MAC).  Returns (out, counts) with counts =
        [near pairs, far grid points, accepted clusters, direct leaves,
        sources inside accepted clusters], each summed over targets."""
        w = _f64(w, (self.n, kernel_win(kernel)))
        fhat = _f64(fhat)
        tgt = _f64(tgt, (-1, 3))
        out = np.empty((len(tgt), kernel_wout(kernel)))
        cnt = np.zeros(5, np.int64)
        lib().or_treecode(self._h, _p(self.x), _p(w), _p(fhat), n, kernel, float(eps),
                          float(theta), _p(tgt), len(tgt), _p(out), _p(cnt))
        return out, cnt

    def treecode_batch(self, w, fhat, n, kernel, eps, theta, tgt, batch, tgt_leaf,
                       lists=False, evaluate=True, select=None, all_targets=False):
        """Batch-MAC variant (targets grouped by the tree on the targets).
        Returns a dict with out, counts, tperm, nfar, nnear and, when lists,
        far_list / near_list (concatenated per batch, traversal order).
        select: optional target indices; only those rows of out are summed.
        all_targets: a cluster is accepted for a batch iff every target of the
        batch accepts it by Eq. MAC (instead of the box-distance rule)."""
        w = _f64(w, (self.n, kernel_win(kernel)))
        fhat = _f64(fhat)
        tgt = _f64(tgt, (-1, 3))
        nt = len(tgt)
        nb = lib().or_num_batches(nt, batch)
        out = np.empty((nt, kernel_wout(kernel))) if evaluate else None
        cnt = np.zeros(5, np.int64)
        tperm = np.empty(nt, np.int64)
        nfar = np.empty(nb, np.int64)
        nnear = np.empty(nb, np.int64)
        L = lib()
        sel = None
        if select is not None:
            sel = np.zeros(nt, np.uint8)
            sel[np.asarray(select)] = 1
        fn = L.or_treecode_batch_all if all_targets else L.or_treecode_batch
        fn(self._h, _p(self.x), _p(w), _p(fhat), n, kernel, float(eps),
                            float(theta), _p(tgt), nt, batch, tgt_leaf, 0 if evaluate else 1,
                            _p(sel), _p(out), _p(cnt), _p(tperm), _p(nfar), _p(nnear), None, 0,
                            None, 0)
        res = dict(out=out, counts=cnt, tperm=tperm, nfar=nfar, nnear=nnear)
        if lists:
            fl = np.empty(max(1, int(nfar.sum())), np.int64)
            nl = np.empty(max(1, int(nnear.sum())), np.int64)
            fn(self._h, _p(self.x), _p(w), _p(fhat), n, kernel, float(eps),
                                float(theta), _p(tgt), nt, batch, tgt_leaf, 1, None, None, None,
                                None, None, None, _p(fl), len(fl), _p(nl), len(nl))
            res["far_list"] = fl[:int(nfar.sum())]
            res["near_list"] = nl[:int(nnear.sum())]
        return res


def treecode(x, w, kernel, eps, theta, n, leaf_size, tgt=None):
    """Algorithm 2 end to end: build tree, modified weights, traversal."""
    t = Tree(x, leaf_size)
    fhat = t.modified_weights(w, n)
    out, cnt = t.treecode(w, fhat, n, kernel, eps, theta, t.x if tgt is None else tgt)
    return out, cnt
