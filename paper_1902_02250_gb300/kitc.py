"""Python binding of libkitc (include/kitc.h): argument marshalling only.

Every step of the treecode runs in the CUDA library; this module passes
pointers, sizes and the current torch stream, and turns status codes into
exceptions.  There is no fallback: without the built library or a CUDA
device the calls raise.
"""
import ctypes
import dataclasses
import os

import numpy as np

from . import build as _build

STOKESLET, ROTLET, STOKESLET_ROTLET, TEST_POLY = 0, 1, 2, 99
FP64, MIXED, MIXED_LEAF = 0, 1, 2
MAC_PARTICLE, MAC_BATCH, MAC_ALL = 0, 1, 2
WEIGHTS_UPWARD, WEIGHTS_ALGORITHM1 = 0, 1

_STATUS = {0: "ok", 1: "invalid argument", 2: "CUDA error", 3: "out of device memory",
           4: "device-side wait timed out", 5: "call out of order",
           6: "size exceeds the room reserved by the call"}


class KitcError(RuntimeError):
    def __init__(self, status, where):
        super().__init__("%s: %s (status %d)" % (where, _STATUS.get(status, "?"), status))
        self.status = status


class _Params(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("degree", ctypes.c_int), ("leaf_size", ctypes.c_int),
                ("eps", ctypes.c_double), ("kernel", ctypes.c_int), ("precision", ctypes.c_int),
                ("mac", ctypes.c_int), ("target_batch", ctypes.c_int), ("weights", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("n_sources", ctypes.c_int64), ("n_clusters", ctypes.c_int64),
                ("n_leaves", ctypes.c_int64), ("depth", ctypes.c_int32),
                ("degree", ctypes.c_int32), ("n_targets", ctypes.c_int64),
                ("n_batches", ctypes.c_int64), ("far_entries", ctypes.c_int64),
                ("near_entries", ctypes.c_int64), ("near_pairs", ctypes.c_int64),
                ("far_points", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("ms_tree", ctypes.c_float), ("ms_weights", ctypes.c_float),
                ("ms_lists", ctypes.c_float), ("ms_evaluate", ctypes.c_float),
                ("near_exec", ctypes.c_int64), ("far_exec", ctypes.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


@dataclasses.dataclass
class Params:
    """kitc_params: MAC theta (Eq. MAC), degree n, leaf size N0, MRS eps,
    kernel, precision, MAC mode, targets per batch (<= 64) and how the
    modified weights are formed (upward pass or Algorithm 1 everywhere)."""
    theta: float = 0.7
    degree: int = 8
    leaf_size: int = 2000
    eps: float = 0.001
    kernel: int = STOKESLET
    precision: int = FP64
    mac: int = MAC_PARTICLE
    target_batch: int = 64
    weights: int = WEIGHTS_UPWARD

    def c(self):
        return _Params(float(self.theta), int(self.degree), int(self.leaf_size), float(self.eps),
                       int(self.kernel), int(self.precision), int(self.mac),
                       int(self.target_batch), int(self.weights))


_lib = None
SYMBOLS = ["kitc_build_tree", "kitc_build_forest", "kitc_modified_weights", "kitc_evaluate",
           "kitc_evaluate_forest", "kitc_apply", "kitc_direct", "kitc_direct_noalloc",
           "kitc_solve_host", "kitc_get_stats", "kitc_tree_download", "kitc_weights_download",
           "kitc_lists_download", "kitc_free_tree", "kitc_status_string", "kitc_kernel_win",
           "kitc_kernel_wout", "kitc_set_wait_limit_ms", "kitc_watchdog_selftest",
           "kitc_launch_count", "kitc_set_degrees", "kitc_plan_targets",
           "kitc_evaluate_planned", "kitc_plan_targets_forest", "kitc_cluster_features",
           "kitc_cluster_far_errors",
           "kitc_mlp_workspace_bytes",
           "kitc_mlp_forward", "kitc_mlp_loss_grad", "kitc_mlp_adam_step",
           "kitc_peak_launch", "kitc_peak_ops_per_launch",
           "kitc_pipeline_create", "kitc_pipeline_run", "kitc_pipeline_replay",
           "kitc_pipeline_status", "kitc_pipeline_graph_launches", "kitc_pipeline_free"]


def library_path():
    return _build.LIB


def lib():
    """Loads the in-tree libkitc.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        path = library_path()
        if not os.path.exists(path):
            raise RuntimeError("libkitc.so is not built (%s); run __graft_entry__.build()" % path)
        L = ctypes.CDLL(path)
        P, I64, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        PP = ctypes.POINTER(_Params)
        L.kitc_build_tree.argtypes = [P, I64, PP, P, ctypes.POINTER(P)]
        L.kitc_build_forest.argtypes = [P, P, I, PP, P, ctypes.POINTER(P)]
        L.kitc_evaluate_forest.argtypes = [P, P, P, P, P]
        L.kitc_apply.argtypes = [P, P, P, P]
        L.kitc_modified_weights.argtypes = [P, P, P]
        L.kitc_evaluate.argtypes = [P, P, I64, P, P]
        L.kitc_direct.argtypes = [P, I64, P, P, I64, PP, P, P]
        L.kitc_direct_noalloc.argtypes = [P, I64, P, P, I64, PP, P, P]
        L.kitc_solve_host.argtypes = [P, P, I64, P, I64, PP, P, P]
        L.kitc_get_stats.argtypes = [P, ctypes.POINTER(Stats)]
        L.kitc_tree_download.argtypes = [P] * 11
        L.kitc_weights_download.argtypes = [P, P, P]
        L.kitc_lists_download.argtypes = [P] * 9
        L.kitc_free_tree.argtypes = [P]
        L.kitc_free_tree.restype = None
        L.kitc_status_string.argtypes = [I]
        L.kitc_status_string.restype = ctypes.c_char_p
        L.kitc_kernel_win.argtypes = [I]
        L.kitc_kernel_wout.argtypes = [I]
        L.kitc_set_wait_limit_ms.argtypes = [I]
        L.kitc_watchdog_selftest.argtypes = [I, P]
        L.kitc_launch_count.argtypes = []
        L.kitc_launch_count.restype = I64
        L.kitc_set_degrees.argtypes = [P, P, P]
        L.kitc_plan_targets.argtypes = [P, P, I64, P]
        L.kitc_evaluate_planned.argtypes = [P, P, P]
        L.kitc_plan_targets_forest.argtypes = [P, P, P, P]
        L.kitc_cluster_features.argtypes = [P, P, P, P]
        L.kitc_cluster_far_errors.argtypes = [P, P, I, ctypes.c_uint64, P, P, P]
        L.kitc_mlp_workspace_bytes.argtypes = [I64]
        L.kitc_mlp_workspace_bytes.restype = ctypes.c_size_t
        L.kitc_mlp_forward.argtypes = [P, P, I64, P, P, I, P, P]
        L.kitc_mlp_loss_grad.argtypes = [P, P, P, I64, P, P, P, P]
        F = ctypes.c_float
        L.kitc_mlp_adam_step.argtypes = [P, P, P, P, I, F, F, F, F, P]
        L.kitc_peak_launch.argtypes = [I, I, I, I, P, P]
        L.kitc_peak_ops_per_launch.argtypes = [I, I, I, I]
        L.kitc_peak_ops_per_launch.restype = ctypes.c_double
        L.kitc_pipeline_create.argtypes = [P, P, P, P, I, PP, ctypes.c_double, P, ctypes.POINTER(P)]
        L.kitc_pipeline_run.argtypes = [P, P, P, P, P, P]
        L.kitc_pipeline_replay.argtypes = [P, P, P, P, P, P]
        L.kitc_pipeline_status.argtypes = [P, ctypes.POINTER(Stats), P]
        L.kitc_pipeline_graph_launches.argtypes = [P]
        L.kitc_pipeline_graph_launches.restype = I64
        L.kitc_pipeline_free.argtypes = [P]
        for name in ("kitc_build_tree", "kitc_build_forest", "kitc_evaluate_forest", "kitc_apply",
                     "kitc_modified_weights", "kitc_evaluate", "kitc_direct",
                     "kitc_direct_noalloc",
                     "kitc_solve_host", "kitc_get_stats", "kitc_tree_download",
                     "kitc_weights_download", "kitc_lists_download", "kitc_watchdog_selftest",
                     "kitc_set_degrees", "kitc_plan_targets", "kitc_evaluate_planned",
                     "kitc_plan_targets_forest",
                     "kitc_cluster_features",
                     "kitc_cluster_far_errors", "kitc_mlp_forward", "kitc_mlp_loss_grad",
                     "kitc_mlp_adam_step", "kitc_peak_launch", "kitc_pipeline_create",
                     "kitc_pipeline_run", "kitc_pipeline_replay", "kitc_pipeline_status",
                     "kitc_pipeline_free"):
            getattr(L, name).restype = I
        _lib = L
    return _lib


def _check(status, where):
    if status != 0:
        raise KitcError(status, where)


def _stream(stream=None):
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def _dptr(t, cols, name):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64
            and t.is_contiguous() and t.dim() == 2 and t.shape[1] == cols):
        raise ValueError("%s must be a contiguous CUDA float64 tensor of shape (n, %d)" % (name, cols))
    return ctypes.c_void_p(t.data_ptr())


def _np(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def kernel_win(kernel):
    return lib().kitc_kernel_win(kernel)


def kernel_wout(kernel):
    return lib().kitc_kernel_wout(kernel)


def set_wait_limit_ms(ms):
    return lib().kitc_set_wait_limit_ms(int(ms))


def kitc_launch_count():
    """Kernels launched by libkitc in this process so far."""
    return lib().kitc_launch_count()


def kitc_watchdog_selftest(limit_ms=50, stream=None):
    """Status of a bounded device wait on a barrier nothing completes (4 = timed out)."""
    return lib().kitc_watchdog_selftest(int(limit_ms), _stream(stream))


PEAK_FFMA, PEAK_FFMA2, PEAK_DFMA, PEAK_RSQRT = 0, 1, 2, 3


def kitc_peak_launch(kind, blocks, threads, iters, sink, stream=None):
    """One arithmetic-issue micro-benchmark launch (include/kitc_peak.h);
    sink: CUDA float32 tensor of >= blocks * threads elements."""
    import torch
    if not (isinstance(sink, torch.Tensor) and sink.is_cuda and sink.dtype == torch.float32
            and sink.numel() >= blocks * threads):
        raise ValueError("sink must be a CUDA float32 tensor of >= blocks * threads elements")
    _check(lib().kitc_peak_launch(int(kind), int(blocks), int(threads), int(iters),
                                  ctypes.c_void_p(sink.data_ptr()), _stream(stream)),
           "kitc_peak_launch")


def kitc_peak_ops_per_launch(kind, blocks, threads, iters):
    """Flops (FMA kinds) or reciprocal square roots of one kitc_peak_launch."""
    return lib().kitc_peak_ops_per_launch(int(kind), int(blocks), int(threads), int(iters))


def measure_peak(kind, target_ms=40.0, repeats=3, device=None):
    """Measured issue rate of one pipe (ops/s): the micro-benchmark sized to run
    about target_ms, on every SM (8 CTAs of 256 threads each), best of
    `repeats` timed launches with CUDA events on the launching stream."""
    import torch
    dev = torch.device("cuda") if device is None else device
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    blocks, threads = sms * 8, 256
    sink = torch.empty(blocks * threads, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def run(iters):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        kitc_peak_launch(kind, blocks, threads, iters, sink, stream)
        e1.record(stream)
        e1.synchronize()
        return e0.elapsed_time(e1)

    iters = 64
    run(iters)
    ms = run(iters)
    while ms < target_ms / 4 and iters < (1 << 24):
        iters *= 4
        ms = run(iters)
    iters = max(1, int(iters * target_ms / max(ms, 1e-3)))
    run(iters)
    best = min(run(iters) for _ in range(repeats))
    ops = kitc_peak_ops_per_launch(kind, blocks, threads, iters)
    return {"ops_per_s": ops / (best / 1e3), "ms": best, "iters": iters, "blocks": blocks,
            "threads": threads}


class Tree:
    """A kitc_tree handle (owned by the library, freed with free())."""

    def __init__(self, handle, params, n):
        self._h = handle
        self.params = params
        self.n = n
        self.degrees = None  # host copy of a per-cluster degree map (kitc_set_degrees)

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("tree already freed")
        return self._h

    def free(self):
        if self._h:
            lib().kitc_free_tree(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def stats(self):
        s = Stats()
        _check(lib().kitc_get_stats(self.handle, ctypes.byref(s)), "kitc_get_stats")
        return s.as_dict()

    def download(self, stream=None):
        st = self.stats()
        m, n = st["n_clusters"], st["n_sources"]
        out = dict(perm=np.empty(n, np.int64), lo=np.empty((m, 3)), hi=np.empty((m, 3)),
                   begin=np.empty(m, np.int64), end=np.empty(m, np.int64),
                   first_child=np.empty(m, np.int32), n_child=np.empty(m, np.int32),
                   level=np.empty(m, np.int32), parent=np.empty(m, np.int32))
        _check(lib().kitc_tree_download(self.handle, *[_np(out[k]) for k in (
            "perm", "lo", "hi", "begin", "end", "first_child", "n_child", "level", "parent")],
            _stream(stream)), "kitc_tree_download")
        return out

    def weights(self, stream=None):
        """FP64 modified weights: [clusters, n+1, n+1, n+1, w_in], or with a
        per-cluster degree map the flat concatenation over clusters with n_c > 0."""
        st = self.stats()
        if self.degrees is not None:
            g = self.degrees.astype(np.int64) + 1
            tot = int((g ** 3 * (self.degrees > 0)).sum()) * kernel_win(self.params.kernel)
            f = np.empty(max(tot, 1))
            _check(lib().kitc_weights_download(self.handle, _np(f), _stream(stream)),
                   "kitc_weights_download")
            return f[:tot]
        np1 = st["degree"] + 1
        f = np.empty((st["n_clusters"], np1, np1, np1, kernel_win(self.params.kernel)))
        _check(lib().kitc_weights_download(self.handle, _np(f), _stream(stream)),
               "kitc_weights_download")
        return f

    def lists(self, stream=None):
        st = self.stats()
        nb, nt = st["n_batches"], st["n_targets"]
        r = dict(tperm=np.empty(nt, np.int64), nfar=np.empty(nb, np.int64),
                 nnear=np.empty(nb, np.int64), far=np.empty(max(1, st["far_entries"]), np.int32),
                 far_mask=np.empty(max(1, st["far_entries"]), np.uint64),
                 near=np.empty(max(1, st["near_entries"]), np.int32),
                 near_mask=np.empty(max(1, st["near_entries"]), np.uint64))
        _check(lib().kitc_lists_download(self.handle, *[_np(r[k]) for k in (
            "tperm", "nfar", "nnear", "far", "far_mask", "near", "near_mask")], _stream(stream)),
            "kitc_lists_download")
        r["far"] = r["far"][:st["far_entries"]]
        r["far_mask"] = r["far_mask"][:st["far_entries"]]
        r["near"] = r["near"][:st["near_entries"]]
        r["near_mask"] = r["near_mask"][:st["near_entries"]]
        return r


def kitc_build_tree(src_xyz, params, stream=None):
    """Sec. 6 tree of the sources (CUDA float64 tensor, n x 3)."""
    h = ctypes.c_void_p()
    p = params.c()
    _check(lib().kitc_build_tree(_dptr(src_xyz, 3, "src_xyz"), src_xyz.shape[0], ctypes.byref(p),
                                 _stream(stream), ctypes.byref(h)), "kitc_build_tree")
    return Tree(h.value, params, src_xyz.shape[0])


def kitc_build_forest(src_xyz, counts, params, stream=None):
    """One Sec. 6 tree per system; counts[k] rows of src_xyz belong to system k."""
    counts = np.ascontiguousarray(counts, np.int64)
    h = ctypes.c_void_p()
    p = params.c()
    _check(lib().kitc_build_forest(_dptr(src_xyz, 3, "src_xyz"), _np(counts), len(counts),
                                   ctypes.byref(p), _stream(stream), ctypes.byref(h)),
           "kitc_build_forest")
    return Tree(h.value, params, src_xyz.shape[0])


def kitc_evaluate_forest(tree, tgt_xyz, tgt_counts, out=None, stream=None):
    """Algorithm 2 per system of a forest; returns out (sum(tgt_counts) x w_out)."""
    import torch
    wout = kernel_wout(tree.params.kernel)
    tgt_counts = np.ascontiguousarray(tgt_counts, np.int64)
    if out is None:
        out = torch.empty((tgt_xyz.shape[0], wout), dtype=torch.float64, device=tgt_xyz.device)
    _check(lib().kitc_evaluate_forest(tree.handle, _dptr(tgt_xyz, 3, "tgt_xyz"), _np(tgt_counts),
                                      _dptr(out, wout, "out"), _stream(stream)),
           "kitc_evaluate_forest")
    return out


def kitc_modified_weights(tree, w, stream=None):
    """Eq. modified_weights for every cluster; w is n x w_in (CUDA float64)."""
    _check(lib().kitc_modified_weights(tree.handle, _dptr(w, kernel_win(tree.params.kernel), "w"),
                                       _stream(stream)), "kitc_modified_weights")


def kitc_evaluate(tree, tgt_xyz, out=None, stream=None):
    """Algorithm 2 at the targets; returns out (n_tgt x w_out, CUDA float64)."""
    import torch
    wout = kernel_wout(tree.params.kernel)
    if out is None:
        out = torch.empty((tgt_xyz.shape[0], wout), dtype=torch.float64, device=tgt_xyz.device)
    _check(lib().kitc_evaluate(tree.handle, _dptr(tgt_xyz, 3, "tgt_xyz"), tgt_xyz.shape[0],
                               _dptr(out, wout, "out"), _stream(stream)), "kitc_evaluate")
    return out


def kitc_set_degrees(tree, degrees, stream=None):
    """Degree n_c per cluster (int32, one per cluster: numpy or CUDA tensor), or
    None for the uniform degree.  Weights and lists must be computed again."""
    if degrees is None:
        _check(lib().kitc_set_degrees(tree.handle, None, _stream(stream)), "kitc_set_degrees")
        tree.degrees = None
        return
    if isinstance(degrees, np.ndarray):
        h = np.ascontiguousarray(degrees, np.int32)
        ptr = _np(h)
    else:
        import torch
        if degrees.dtype != torch.int32 or not degrees.is_contiguous():
            raise ValueError("degrees must be a contiguous int32 tensor")
        h = degrees.cpu().numpy()
        ptr = degrees.data_ptr()
    if h.shape != (tree.stats()["n_clusters"],):
        raise ValueError("degrees must hold one value per cluster")
    _check(lib().kitc_set_degrees(tree.handle, ptr, _stream(stream)), "kitc_set_degrees")
    tree.degrees = h.copy()


def kitc_apply(tree, w, out, stream=None):
    """New weights, same sources and targets as the last evaluate (CUDA-graph replay)."""
    _check(lib().kitc_apply(tree.handle, _dptr(w, kernel_win(tree.params.kernel), "w"),
                            _dptr(out, kernel_wout(tree.params.kernel), "out"), _stream(stream)),
           "kitc_apply")
    return out


def kitc_direct(tgt_xyz, src_xyz, w, params, out=None, stream=None):
    """Eq. N-body by direct summation on the GPU."""
    import torch
    wout = kernel_wout(params.kernel)
    if out is None:
        out = torch.empty((tgt_xyz.shape[0], wout), dtype=torch.float64, device=tgt_xyz.device)
    p = params.c()
    _check(lib().kitc_direct(_dptr(tgt_xyz, 3, "tgt_xyz"), tgt_xyz.shape[0],
                             _dptr(src_xyz, 3, "src_xyz"), _dptr(w, kernel_win(params.kernel), "w"),
                             src_xyz.shape[0], ctypes.byref(p), _dptr(out, wout, "out"),
                             _stream(stream)), "kitc_direct")
    return out


def kitc_direct_noalloc(tgt_xyz, src_xyz, w, params, out, stream=None):
    """kitc_direct for callers that must not allocate device memory: the
    library's fixed 8 MiB device scratch array is used instead (at most 100000
    sources; overlapping calls race on it).  out must be given."""
    wout = kernel_wout(params.kernel)
    p = params.c()
    _check(lib().kitc_direct_noalloc(_dptr(tgt_xyz, 3, "tgt_xyz"), tgt_xyz.shape[0],
                                     _dptr(src_xyz, 3, "src_xyz"),
                                     _dptr(w, kernel_win(params.kernel), "w"), src_xyz.shape[0],
                                     ctypes.byref(p), _dptr(out, wout, "out"), _stream(stream)),
           "kitc_direct_noalloc")
    return out


def kitc_solve_host(src_xyz, w, params, tgt_xyz=None, out=None, stream=None):
    """End to end from host (numpy float64) arrays: copies in, treecode, copies out."""
    src_xyz = np.ascontiguousarray(src_xyz, np.float64)
    w = np.ascontiguousarray(w, np.float64)
    n = src_xyz.shape[0]
    nt = n if tgt_xyz is None else tgt_xyz.shape[0]
    wout = kernel_wout(params.kernel)
    if out is None:
        out = np.empty((nt, wout))
    tp = None
    if tgt_xyz is not None:
        tgt_xyz = np.ascontiguousarray(tgt_xyz, np.float64)
        tp = _np(tgt_xyz)
    p = params.c()
    _check(lib().kitc_solve_host(_np(src_xyz), _np(w), n, tp, nt, ctypes.byref(p), _np(out),
                                 _stream(stream)), "kitc_solve_host")
    return out


def treecode(src_xyz, w, params, tgt_xyz=None, stream=None):
    """build tree -> modified weights -> evaluate (device tensors)."""
    t = kitc_build_tree(src_xyz, params, stream)
    try:
        kitc_modified_weights(t, w, stream)
        out = kitc_evaluate(t, src_xyz if tgt_xyz is None else tgt_xyz, stream=stream)
        return out, t.stats()
    finally:
        t.free()


class Pipeline:
    """A kitc_pipeline handle (include/kitc_pipeline.h): the whole treecode
    queued without host synchronization or allocation, sized once from
    example inputs; run() queues it, replay() goes through the handle's CUDA
    graph, status() waits and reports the last run."""

    def __init__(self, src_xyz, params, src_counts=None, tgt_xyz=None, tgt_counts=None,
                 slack=1.25, stream=None):
        ns = src_xyz.shape[0]
        sc = np.ascontiguousarray([ns] if src_counts is None else src_counts, np.int64)
        self.self_targets = tgt_xyz is None
        nt = ns if tgt_xyz is None else tgt_xyz.shape[0]
        tc = None
        if tgt_xyz is not None:
            tc = np.ascontiguousarray([nt] if tgt_counts is None else tgt_counts, np.int64)
            if len(tc) != len(sc):
                raise ValueError("tgt_counts must have one entry per system")
        self.params = params
        self.n_src, self.n_tgt = ns, nt
        self.num_systems = len(sc)
        h = ctypes.c_void_p()
        p = params.c()
        _check(lib().kitc_pipeline_create(
            _dptr(src_xyz, 3, "src_xyz"), _np(sc),
            None if tgt_xyz is None else _dptr(tgt_xyz, 3, "tgt_xyz"),
            None if tc is None else _np(tc), len(sc), ctypes.byref(p), float(slack),
            _stream(stream), ctypes.byref(h)), "kitc_pipeline_create")
        self._h = h.value

    @property
    def handle(self):
        if not self._h:
            raise RuntimeError("pipeline already freed")
        return self._h

    def _args(self, src_xyz, w, tgt_xyz, out):
        import torch
        wout = kernel_wout(self.params.kernel)
        if out is None:
            out = torch.empty((self.n_tgt, wout), dtype=torch.float64, device=src_xyz.device)
        if src_xyz.shape[0] != self.n_src or (tgt_xyz is not None and tgt_xyz.shape[0] != self.n_tgt):
            raise ValueError("sizes differ from the ones the pipeline was created for")
        t = None if tgt_xyz is None else _dptr(tgt_xyz, 3, "tgt_xyz")
        return (_dptr(src_xyz, 3, "src_xyz"), _dptr(w, kernel_win(self.params.kernel), "w"), t,
                _dptr(out, wout, "out")), out

    def run(self, src_xyz, w, tgt_xyz=None, out=None, stream=None):
        a, out = self._args(src_xyz, w, tgt_xyz, out)
        _check(lib().kitc_pipeline_run(self.handle, *a, _stream(stream)), "kitc_pipeline_run")
        return out

    def replay(self, src_xyz, w, tgt_xyz=None, out=None, stream=None):
        a, out = self._args(src_xyz, w, tgt_xyz, out)
        _check(lib().kitc_pipeline_replay(self.handle, *a, _stream(stream)), "kitc_pipeline_replay")
        return out

    def status(self, stream=None):
        """(status code, stats dict) of the last run; waits for the stream."""
        s = Stats()
        code = lib().kitc_pipeline_status(self.handle, ctypes.byref(s), _stream(stream))
        return code, s.as_dict()

    def check(self, stream=None):
        code, st = self.status(stream)
        _check(code, "kitc_pipeline_status")
        return st

    def graph_launches(self):
        return lib().kitc_pipeline_graph_launches(self.handle)

    def free(self):
        if self._h:
            lib().kitc_pipeline_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass


# ------------------------------------------------------- degree selection
NFEAT, MLP_HIDDEN, MLP_CLASSES = 12, 64, 6
MLP_NPARAM = 2 * 12 + 64 * 12 + 64 + 64 * 64 + 64 + 6 * 64 + 6


def _dev(t, dtype, shape, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda or t.dtype != dtype or not t.is_contiguous():
        raise ValueError("%s must be a contiguous CUDA %s tensor" % (name, dtype))
    if shape is not None and tuple(t.shape) != tuple(shape):
        raise ValueError("%s must have shape %s" % (name, shape))
    return ctypes.c_void_p(t.data_ptr())


def kitc_plan_targets(tree, tgt_xyz, stream=None):
    """Target tree and interaction lists for tgt_xyz, without evaluating."""
    _check(lib().kitc_plan_targets(tree.handle, _dptr(tgt_xyz, 3, "tgt_xyz"), tgt_xyz.shape[0],
                                   _stream(stream)), "kitc_plan_targets")


def kitc_plan_targets_forest(tree, tgt_xyz, tgt_counts, stream=None):
    """Target trees and lists of every system of a forest, without evaluating."""
    tgt_counts = np.ascontiguousarray(tgt_counts, np.int64)
    _check(lib().kitc_plan_targets_forest(tree.handle, _dptr(tgt_xyz, 3, "tgt_xyz"),
                                          _np(tgt_counts), _stream(stream)),
           "kitc_plan_targets_forest")


def kitc_evaluate_planned(tree, out=None, stream=None):
    """Algorithm 2 at the targets of the last kitc_plan_targets (no list build)."""
    import torch
    wout = kernel_wout(tree.params.kernel)
    nt = tree.stats()["n_targets"]
    if out is None:
        out = torch.empty((nt, wout), dtype=torch.float64, device="cuda")
    _check(lib().kitc_evaluate_planned(tree.handle, _dptr(out, wout, "out"), _stream(stream)),
           "kitc_evaluate_planned")
    return out


def kitc_cluster_features(tree, w, out=None, stream=None):
    """FP32 features (n_clusters x 12) of every source cluster."""
    import torch
    m = tree.stats()["n_clusters"]
    if out is None:
        out = torch.empty((m, NFEAT), dtype=torch.float32, device=w.device)
    _check(lib().kitc_cluster_features(tree.handle, _dptr(w, kernel_win(tree.params.kernel), "w"),
                                       _dev(out, torch.float32, (m, NFEAT), "out"),
                                       _stream(stream)), "kitc_cluster_features")
    return out


def kitc_cluster_far_errors(tree, w, max_samples=32, seed=1, stream=None):
    """(err2, n_samples) per cluster: summed squared far-field error of sampled
    accepting targets against the direct sum over the cluster's sources."""
    import torch
    m = tree.stats()["n_clusters"]
    err2 = torch.empty(m, dtype=torch.float64, device=w.device)
    ns = torch.empty(m, dtype=torch.int32, device=w.device)
    _check(lib().kitc_cluster_far_errors(tree.handle, _dptr(w, kernel_win(tree.params.kernel), "w"),
                                         int(max_samples), int(seed) & (2 ** 64 - 1),
                                         ctypes.c_void_p(err2.data_ptr()),
                                         ctypes.c_void_p(ns.data_ptr()), _stream(stream)),
           "kitc_cluster_far_errors")
    return err2, ns


def kitc_mlp_forward(params, features, class_degree=None, logits=True, zero_unused=False,
                     stream=None):
    """(logits or None, degrees or None) of the selector for the feature rows;
    zero_unused gives degree 0 to clusters that no target accepts."""
    import torch
    m = features.shape[0]
    lg = torch.empty((m, MLP_CLASSES), dtype=torch.float32, device=features.device) if logits else None
    deg = None
    cls = None
    if class_degree is not None:
        cls = np.ascontiguousarray(class_degree, np.int32)
        if cls.shape != (MLP_CLASSES,):
            raise ValueError("class_degree must hold %d degrees" % MLP_CLASSES)
        deg = torch.empty(m, dtype=torch.int32, device=features.device)
    _check(lib().kitc_mlp_forward(_dev(params, torch.float32, (MLP_NPARAM,), "params"),
                                  _dev(features, torch.float32, (m, NFEAT), "features"), m,
                                  None if lg is None else ctypes.c_void_p(lg.data_ptr()),
                                  None if cls is None else _np(cls), int(bool(zero_unused)),
                                  None if deg is None else ctypes.c_void_p(deg.data_ptr()),
                                  _stream(stream)), "kitc_mlp_forward")
    return lg, deg


class MLPTrainer:
    """Device buffers of one training run (gradient, Adam moments, workspace)."""

    def __init__(self, params, m):
        import torch
        self.params = params
        self.m = int(m)
        dev_ = params.device
        self.grad = torch.zeros(MLP_NPARAM, dtype=torch.float32, device=dev_)
        self.m1 = torch.zeros_like(self.grad)
        self.m2 = torch.zeros_like(self.grad)
        self.loss = torch.zeros(2, dtype=torch.float32, device=dev_)
        nb = lib().kitc_mlp_workspace_bytes(self.m)
        self.work = torch.empty((nb + 15) // 16 * 4, dtype=torch.float32, device=dev_)
        self.step_count = 0

    def loss_grad(self, features, labels, stream=None):
        import torch
        _check(lib().kitc_mlp_loss_grad(_dev(self.params, torch.float32, (MLP_NPARAM,), "params"),
                                        _dev(features, torch.float32, (self.m, NFEAT), "features"),
                                        _dev(labels, torch.int32, (self.m,), "labels"), self.m,
                                        ctypes.c_void_p(self.loss.data_ptr()),
                                        ctypes.c_void_p(self.grad.data_ptr()),
                                        ctypes.c_void_p(self.work.data_ptr()), _stream(stream)),
               "kitc_mlp_loss_grad")
        return self.loss, self.grad

    def adam(self, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
        self.step_count += 1
        _check(lib().kitc_mlp_adam_step(ctypes.c_void_p(self.params.data_ptr()),
                                        ctypes.c_void_p(self.grad.data_ptr()),
                                        ctypes.c_void_p(self.m1.data_ptr()),
                                        ctypes.c_void_p(self.m2.data_ptr()), self.step_count,
                                        lr, beta1, beta2, eps, _stream(stream)),
               "kitc_mlp_adam_step")

    def step(self, features, labels, lr, stream=None):
        self.loss_grad(features, labels, stream)
        self.adam(lr, stream=stream)
