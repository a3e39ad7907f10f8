// C ABI of libkitc: argument checks, handle life cycle, stage timing.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "common.cuh"

#include <atomic>

int g_wait_limit_ms = 2000;
// Split-precision weight products for the mixed form (KITC_WEIGHTS_SPLIT=0 at
// build time turns them off).
#ifndef KITC_WEIGHTS_SPLIT
#define KITC_WEIGHTS_SPLIT 1
#endif
static const bool g_weights_split = KITC_WEIGHTS_SPLIT != 0;

static std::atomic<int64_t> g_launches{0};

void kitc_count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

struct kitc_tree_s {
    kitc_params p{};
    int win = 3, wout = 3, device = 0;
    TreeDev src, tgt;
    WeightsDev wts;
    ListsDev lists;
    DevBuf flags;            // int [4]: work counter, error flag
    bool has_weights = false, evaluated = false, pairs_planned = false;
    EvalArgs last{};          // evaluator arguments of the last evaluate (reused by kitc_apply)
    // CUDA graph of weights + packing + evaluator (kitc_apply)
    cudaGraphExec_t graph = nullptr;
    const void *graph_w = nullptr, *graph_out = nullptr;
    cudaStream_t graph_stream = nullptr;
    int64_t graph_launches = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev[8] = {};
    bool ev_ok = false;
    bool stage_done[4] = {false, false, false, false};
    // degree per cluster (kitc_set_degrees)
    bool var = false;
    std::vector<int32_t> hdeg;
    DevBuf cdeg, roff, chebt;  // int32 [nclus], int64 [nclus] record offsets, double [17][17]
    int64_t proxy_bytes = 0;
    bool lists_ready = false;  // target tree + lists of the last plan or evaluation
    DevBuf learn;              // scratch of the feature and error kernels
};

// ---------------------------------------------------------------------------
// shared helpers
// ---------------------------------------------------------------------------
kitc_status kitc_from_cuda(cudaError_t e)
{
    if (e == cudaSuccess) return KITC_OK;
    cudaGetLastError();  // clear a non-sticky error so later calls start clean
    return e == cudaErrorMemoryAllocation ? KITC_ERR_OOM : KITC_ERR_CUDA;
}

// 64 bytes of pinned host memory per calling thread for the small read-backs
// (error flags, totals).  Every call that uses it synchronizes its stream
// before reading, so calls of one thread never overlap on it, and threads
// never share it.
kitc_status host_readback_buffer(void **p)
{
    static thread_local void *buf = nullptr;
    if (!buf) KITC_CUDA(cudaHostAlloc(&buf, 64, cudaHostAllocPortable));
    *p = buf;
    return KITC_OK;
}

kitc_status dev_alloc(void **p, size_t bytes, cudaStream_t s)
{
    static std::atomic<bool> pool_set[64] = {};
    int dev = 0;
    KITC_CUDA(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && !pool_set[dev].load()) {
        // keep freed blocks in this process's pool between calls
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
            uint64_t thr = UINT64_MAX;
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
        }
        pool_set[dev] = true;
    }
    *p = nullptr;
    if (bytes == 0) bytes = 16;
    KITC_CUDA(cudaMallocAsync(p, bytes, s));
    return KITC_OK;
}

void dev_free(void *p, cudaStream_t s)
{
    if (p) cudaFreeAsync(p, s);
}

kitc_status DevBuf::reserve(size_t b, cudaStream_t s, bool keep)
{
    if (b <= bytes && ptr) return KITC_OK;
    void *np_ = nullptr;
    KITC_TRY(dev_alloc(&np_, b, s));
    if (keep && ptr && bytes) {
        cudaError_t e = cudaMemcpyAsync(np_, ptr, bytes, cudaMemcpyDeviceToDevice, s);
        if (e != cudaSuccess) {
            dev_free(np_, s);
            return kitc_from_cuda(e);
        }
    }
    dev_free(ptr, s);
    ptr = np_;
    bytes = b;
    return KITC_OK;
}

void DevBuf::release(cudaStream_t s)
{
    dev_free(ptr, s);
    ptr = nullptr;
    bytes = 0;
}

void cheb_cos_table(int n, double *t)
{
    const double pi = 3.14159265358979323846;
    for (int k = 0; k <= KITC_MAX_DEGREE; ++k) t[k] = k <= n ? cos((double)k * pi / (double)n) : 0.0;
}

bool valid_count(int64_t n) { return n >= 1 && n <= (int64_t)INT32_MAX - 1024; }

bool device_accessible(const void *ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged ||
           at.type == cudaMemoryTypeHost;
}

bool valid_direct_params(const kitc_params *p)
{
    return p && kitc_kernel_win(p->kernel) >= 0 && p->eps >= 0.0 && isfinite(p->eps) &&
           (p->precision == KITC_FP64 || is_mixed(p->precision)) && p->target_batch >= 0 &&
           p->target_batch <= KITC_MAX_BATCH &&
           !(p->kernel == KITC_TEST_POLY && is_mixed(p->precision));
}

bool valid_params(const kitc_params *p)
{
    if (!p) return false;
    if (!(p->theta >= 0.0) || !isfinite(p->theta)) return false;
    if (p->degree < 1 || p->degree > KITC_MAX_DEGREE) return false;
    if (p->leaf_size < 1) return false;
    if (!(p->eps >= 0.0) || !isfinite(p->eps)) return false;
    if (kitc_kernel_win(p->kernel) < 0) return false;
    if (p->precision != KITC_FP64 && !is_mixed(p->precision)) return false;
    if (p->mac != KITC_MAC_PARTICLE && p->mac != KITC_MAC_BATCH && p->mac != KITC_MAC_ALL)
        return false;
    if (p->target_batch < 0 || p->target_batch > KITC_MAX_BATCH) return false;
    if (p->kernel == KITC_TEST_POLY && is_mixed(p->precision)) return false;
    if (p->weights != KITC_WEIGHTS_UPWARD && p->weights != KITC_WEIGHTS_ALGORITHM1) return false;
    return true;
}

int batch_of(const kitc_params &p) { return p.target_batch == 0 ? KITC_MAX_BATCH : p.target_batch; }

void fill_eval_common(EvalArgs &a, const kitc_params &p, int *flags)
{
    a.degree = p.degree;
    cheb_cos_table(p.degree, a.cheb);
    a.eps = p.eps;
    a.queue = flags;
    a.err = flags + 1;
    a.wait_ns = (unsigned long long)g_wait_limit_ms * 1000000ull;
    a.leaf = uses_leaf_offsets(p);
}

bool weights_split_enabled() { return g_weights_split; }

kitc_status read_error_flag(int *d_err, cudaStream_t s)
{
    int *h = nullptr;
    KITC_TRY(host_readback_buffer(reinterpret_cast<void **>(&h)));
    KITC_CUDA(cudaMemcpyAsync(h, d_err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    return h[0] ? KITC_ERR_TIMEOUT : KITC_OK;
}

namespace {

void record(kitc_tree t, int i, cudaStream_t s)
{
    if (t->ev_ok) cudaEventRecord(t->ev[i], s);
}


void free_handle(kitc_tree t)
{
    cudaStream_t s = t->stream;
    if (t->graph) cudaGraphExecDestroy(t->graph);
    t->src.release(s);
    t->tgt.release(s);
    t->wts.release(s);
    t->lists.release(s);
    t->flags.release(s);
    for (DevBuf *b : {&t->cdeg, &t->roff, &t->chebt, &t->learn}) b->release(s);
    if (t->ev_ok)
        for (auto &e : t->ev) cudaEventDestroy(e);
    delete t;
}

}  // namespace

// ---------------------------------------------------------------------------
// ABI
// ---------------------------------------------------------------------------
extern "C" {

int kitc_kernel_win(int kernel)
{
    switch (kernel) {
    case KITC_STOKESLET: case KITC_ROTLET: case KITC_TEST_POLY: return 3;
    case KITC_STOKESLET_ROTLET: return 6;
    default: return -1;
    }
}

int kitc_kernel_wout(int kernel)
{
    switch (kernel) {
    case KITC_STOKESLET: case KITC_TEST_POLY: return 3;
    case KITC_ROTLET: case KITC_STOKESLET_ROTLET: return 6;
    default: return -1;
    }
}

const char *kitc_status_string(kitc_status s)
{
    switch (s) {
    case KITC_OK: return "ok";
    case KITC_ERR_INVALID_ARG: return "invalid argument";
    case KITC_ERR_CUDA: return "CUDA error";
    case KITC_ERR_OOM: return "out of device memory";
    case KITC_ERR_TIMEOUT: return "device-side wait timed out";
    case KITC_ERR_STATE: return "call out of order";
    case KITC_ERR_TOO_LARGE: return "size exceeds the room reserved by the call";
    default: return "unknown status";
    }
}

int kitc_set_wait_limit_ms(int ms)
{
    int old = g_wait_limit_ms;
    if (ms > 0) g_wait_limit_ms = ms;
    return old;
}

static kitc_status build_impl(const double *src_xyz, int64_t n_src, const int64_t *counts,
                              int nsys, const kitc_params *p, void *stream, kitc_tree *out)
{
    if (!out) return KITC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_params(p) || !valid_count(n_src) || !device_accessible(src_xyz))
        return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    kitc_tree t = new kitc_tree_s();
    t->p = *p;
    t->p.target_batch = batch_of(*p);
    t->win = kitc_kernel_win(p->kernel);
    t->wout = kitc_kernel_wout(p->kernel);
    t->stream = s;
    cudaGetDevice(&t->device);
    t->ev_ok = true;
    for (auto &e : t->ev)
        if (cudaEventCreate(&e) != cudaSuccess) t->ev_ok = false;
    record(t, 0, s);
    kitc_status st = tree_build(src_xyz, n_src, p->leaf_size, s, t->src, counts, nsys);
    if (st == KITC_OK) st = t->flags.reserve(4 * sizeof(int), s);
    record(t, 1, s);
    if (st != KITC_OK) {
        free_handle(t);
        return st;
    }
    t->stage_done[0] = true;
    *out = t;
    return KITC_OK;
}

kitc_status kitc_build_tree(const double *src_xyz, int64_t n_src, const kitc_params *p,
                            void *stream, kitc_tree *out)
{
    return build_impl(src_xyz, n_src, nullptr, 1, p, stream, out);
}

kitc_status kitc_build_forest(const double *src_xyz, const int64_t *counts, int num_systems,
                              const kitc_params *p, void *stream, kitc_tree *out)
{
    if (out) *out = nullptr;
    if (!counts || num_systems < 1) return KITC_ERR_INVALID_ARG;
    int64_t tot = 0;
    for (int k = 0; k < num_systems; ++k) {
        if (counts[k] < 1) return KITC_ERR_INVALID_ARG;
        tot += counts[k];
    }
    return build_impl(src_xyz, tot, counts, num_systems, p, stream, out);
}

// Kernel launches of the weights pass and the evaluator records; the host-side
// plans must exist (prepare_weights).
static kitc_status launch_weights(kitc_tree t, const double *w, cudaStream_t s)
{
    const bool mixed = is_mixed(t->p.precision);
    const bool pairs = uses_pair_records(t->p.kernel, mixed);
    t->wts.rowpairs = pairs && uses_row_pairs(t->p.kernel);
    const bool leaf = uses_leaf_offsets(t->p);
    if (t->var) {
        KITC_TRY(weights_launch_var(t->src, w, t->wts, s));
        KITC_TRY(pack_proxies_var(t->src, t->wts, t->cdeg.as<int32_t>(), t->roff.as<int64_t>(),
                                  mixed, pairs, s));
        if (pairs)
            KITC_TRY(pack_pairs_launch(&t->src, w, t->src.n, t->wts.pair_ranges, leaf, s,
                                       t->wts.src, t->wts.pbegin));
        else
            KITC_TRY(pack_sources(&t->src, nullptr, w, t->src.n, t->win, mixed, s, t->wts.src));
        return KITC_OK;
    }
    KITC_TRY(weights_launch(t->src, w, t->wts, s));
    if (pairs) {  // FP32x2 evaluator records
        KITC_TRY(pack_proxy_pairs(t->src, t->wts, s));
        KITC_TRY(pack_pairs_launch(&t->src, w, t->src.n, t->wts.pair_ranges, leaf, s,
                                   t->wts.src, t->wts.pbegin));
    } else {
        KITC_TRY(pack_proxies(t->src, t->wts, mixed, s));
        KITC_TRY(pack_sources(&t->src, nullptr, w, t->src.n, t->win, mixed, s, t->wts.src));
    }
    return KITC_OK;
}

static kitc_status prepare_weights(kitc_tree t, cudaStream_t s)
{
    t->wts.split = is_mixed(t->p.precision) && g_weights_split;
    if (t->var) {
        if (!t->wts.planned || !t->wts.var) {
            KITC_TRY(weights_plan_var(t->src, t->win, t->hdeg, s, t->wts));
            KITC_TRY(t->wts.proxy.reserve((size_t)std::max<int64_t>(t->proxy_bytes, 16), s));
        }
    } else {
        KITC_TRY(weights_plan(t->src, t->win, t->p.degree, t->p.weights, s, t->wts));
    }
    if (uses_pair_records(t->p.kernel, is_mixed(t->p.precision)) && !t->pairs_planned) {
        KITC_TRY(pack_pairs_plan(&t->src, t->src.n, uses_leaf_offsets(t->p), s,
                                 t->wts.src, t->wts.pbegin,
                                 &t->wts.pair_ranges));
        t->pairs_planned = true;
    }
    return KITC_OK;
}

kitc_status kitc_modified_weights(kitc_tree t, const double *w, void *stream)
{
    if (!t || !device_accessible(w)) return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    t->stream = s;
    t->has_weights = false;
    record(t, 2, s);
    KITC_TRY(prepare_weights(t, s));
    KITC_TRY(launch_weights(t, w, s));
    record(t, 3, s);
    t->has_weights = true;
    t->stage_done[1] = true;
    return KITC_OK;
}

// Target tree (leaf size = target batch) and the interaction lists.
static kitc_status plan_impl(kitc_tree t, const double *tgt_xyz, int64_t n_tgt,
                             const int64_t *counts, int nsys, cudaStream_t s)
{
    const kitc_params &p = t->p;
    int B = p.target_batch;
    t->lists_ready = false;
    KITC_TRY(tree_build(tgt_xyz, n_tgt, B, s, t->tgt, counts, nsys));
    KITC_TRY(lists_build(t->src, t->tgt, B, p.theta, p.degree, t->var ? t->cdeg.as<int32_t>() : nullptr,
                         p.mac, s, t->lists));
    t->lists_ready = true;
    return KITC_OK;
}

// tgt_xyz == NULL: the targets and lists of the last plan (kitc_evaluate_planned).
static kitc_status evaluate_impl(kitc_tree t, const double *tgt_xyz, int64_t n_tgt,
                                 const int64_t *counts, int nsys, double *out, void *stream)
{
    if (!t || !device_accessible(out)) return KITC_ERR_INVALID_ARG;
    if (tgt_xyz && (!valid_count(n_tgt) || !device_accessible(tgt_xyz))) return KITC_ERR_INVALID_ARG;
    if (!t->has_weights || (!tgt_xyz && !t->lists_ready)) return KITC_ERR_STATE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    t->stream = s;
    const kitc_params &p = t->p;
    int B = p.target_batch;
    t->evaluated = false;
    record(t, 4, s);
    if (tgt_xyz) {
        KITC_TRY(plan_impl(t, tgt_xyz, n_tgt, counts, nsys, s));
    } else {
        n_tgt = t->lists.nt;
        if (t->var) KITC_TRY(lists_recount(t->cdeg.as<int32_t>(), s, t->lists));
    }
    record(t, 5, s);
    EvalArgs a{};
    a.tx = t->tgt.xs.as<double>();
    a.ty = a.tx + n_tgt;
    a.tz = a.tx + 2 * n_tgt;
    a.tstride = 1;
    a.tperm = t->tgt.perm.as<int32_t>();
    a.nt = n_tgt;
    a.batch = B;
    a.nb = t->lists.nb;
    a.bctr = t->lists.bctr.as<dvec4>();
    if (t->lists.forest) {
        a.bstart = t->lists.bdesc.as<int32_t>();
        a.bcount = a.bstart + t->lists.nb;
    }
    a.far_off = t->lists.far_off.as<int64_t>();
    a.near_off = t->lists.near_off.as<int64_t>();
    a.far_id = t->lists.far_id.as<int32_t>();
    a.near_id = t->lists.near_id.as<int32_t>();
    a.far_mask = t->lists.far_mask.as<uint64_t>();
    a.near_mask = t->lists.near_mask.as<uint64_t>();
    a.src = t->wts.src.ptr;
    a.proxy = t->wts.proxy.ptr;
    a.clo = t->src.lo.as<dvec4>();
    a.chi = t->src.hi.as<dvec4>();
    a.cbegin = t->src.begin.as<int32_t>();
    a.cend = t->src.end.as<int32_t>();
    a.pbegin = t->wts.pbegin.as<int32_t>();
    a.out = out;
    fill_eval_common(a, p, t->flags.as<int>());
    if (t->var) {
        a.cdeg = t->cdeg.as<int32_t>();
        a.roff = t->roff.as<int64_t>();
        a.chebt = t->chebt.as<double>();
    }
    KITC_CUDA(cudaMemsetAsync(t->flags.ptr, 0, 4 * sizeof(int), s));
    KITC_TRY(evaluate_launch(p.kernel, is_mixed(p.precision), a, s));
    record(t, 6, s);
    t->last = a;
    KITC_TRY(read_error_flag(t->flags.as<int>() + 1, s));
    t->evaluated = true;
    t->stage_done[2] = t->stage_done[3] = true;
    return KITC_OK;
}

kitc_status kitc_evaluate(kitc_tree t, const double *tgt_xyz, int64_t n_tgt, double *out,
                          void *stream)
{
    if (t && t->src.nsys > 1) return KITC_ERR_STATE;
    return evaluate_impl(t, tgt_xyz, n_tgt, nullptr, 1, out, stream);
}

kitc_status kitc_evaluate_planned(kitc_tree t, double *out, void *stream)
{
    return evaluate_impl(t, nullptr, 0, nullptr, 1, out, stream);
}

kitc_status kitc_evaluate_forest(kitc_tree t, const double *tgt_xyz, const int64_t *tgt_counts,
                                 double *out, void *stream)
{
    if (!t || !tgt_counts) return KITC_ERR_INVALID_ARG;
    int nsys = t->src.nsys;
    int64_t tot = 0;
    for (int k = 0; k < nsys; ++k) {
        if (tgt_counts[k] < 1) return KITC_ERR_INVALID_ARG;
        tot += tgt_counts[k];
    }
    return evaluate_impl(t, tgt_xyz, tot, tgt_counts, nsys, out, stream);
}

kitc_status kitc_direct(const double *tgt_xyz, int64_t n_tgt, const double *src_xyz,
                        const double *w, int64_t n_src, const kitc_params *p, double *out,
                        void *stream)
{
    if (!valid_direct_params(p)) return KITC_ERR_INVALID_ARG;
    if (!valid_count(n_tgt) || !valid_count(n_src) || !device_accessible(tgt_xyz) ||
        !device_accessible(src_xyz) || !device_accessible(w) || !device_accessible(out))
        return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    bool mixed = is_mixed(p->precision);
    int win = kitc_kernel_win(p->kernel);
    int B = batch_of(*p);
    DevBuf rec, flags;
    kitc_status st = rec.reserve(direct_record_bytes(n_src, win, mixed, uses_pair_records(p->kernel, mixed)), s);
    if (st == KITC_OK)
        st = pack_direct_records(src_xyz, w, n_src, win, mixed, uses_pair_records(p->kernel, mixed),
                                 rec.ptr, s);
    if (st == KITC_OK) st = flags.reserve(4 * sizeof(int), s);
    if (st == KITC_OK) {
        EvalArgs a{};
        a.tx = tgt_xyz;
        a.ty = tgt_xyz + 1;
        a.tz = tgt_xyz + 2;
        a.tstride = 3;
        a.tperm = nullptr;
        a.nt = n_tgt;
        a.batch = B;
        a.nb = (n_tgt + B - 1) / B;
        a.direct_ns = n_src;
        a.src = rec.ptr;
        kitc_params q = *p;
        q.degree = 1;
        a.out = out;
        fill_eval_common(a, q, flags.as<int>());
        cudaError_t e = cudaMemsetAsync(flags.ptr, 0, 4 * sizeof(int), s);
        st = e == cudaSuccess ? evaluate_launch(p->kernel, mixed, a, s) : kitc_from_cuda(e);
        if (st == KITC_OK) st = read_error_flag(flags.as<int>() + 1, s);
    }
    rec.release(s);
    flags.release(s);
    return st;
}

kitc_status kitc_solve_host(const double *src_xyz, const double *w, int64_t n_src,
                            const double *tgt_xyz, int64_t n_tgt, const kitc_params *p,
                            double *out, void *stream)
{
    if (!src_xyz || !w || !out || !valid_params(p) || !valid_count(n_src)) return KITC_ERR_INVALID_ARG;
    if (tgt_xyz && !valid_count(n_tgt)) return KITC_ERR_INVALID_ARG;
    if (!tgt_xyz) n_tgt = n_src;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int win = kitc_kernel_win(p->kernel), wout = kitc_kernel_wout(p->kernel);
    DevBuf dx, dw, dt, dout;
    kitc_tree t = nullptr;
    kitc_status st = dx.reserve(sizeof(double) * 3 * n_src, s);
    if (st == KITC_OK) st = dw.reserve(sizeof(double) * win * n_src, s);
    if (st == KITC_OK && tgt_xyz) st = dt.reserve(sizeof(double) * 3 * n_tgt, s);
    if (st == KITC_OK) st = dout.reserve(sizeof(double) * wout * n_tgt, s);
    if (st == KITC_OK)
        st = kitc_from_cuda(cudaMemcpyAsync(dx.ptr, src_xyz, sizeof(double) * 3 * n_src,
                                            cudaMemcpyHostToDevice, s));
    if (st == KITC_OK)
        st = kitc_from_cuda(cudaMemcpyAsync(dw.ptr, w, sizeof(double) * win * n_src,
                                            cudaMemcpyHostToDevice, s));
    if (st == KITC_OK && tgt_xyz)
        st = kitc_from_cuda(cudaMemcpyAsync(dt.ptr, tgt_xyz, sizeof(double) * 3 * n_tgt,
                                            cudaMemcpyHostToDevice, s));
    if (st == KITC_OK) st = kitc_build_tree(dx.as<double>(), n_src, p, stream, &t);
    // The target tree and lists need only the source tree: they are built on a
    // second stream while the modified weights run on `stream`, and the
    // evaluation waits for both.
    cudaStream_t side = nullptr;
    cudaEvent_t built = nullptr, planned = nullptr;
    int prio_lo = 0, prio_hi = 0;  // the lists are the longer branch: highest priority
    if (st == KITC_OK) st = kitc_from_cuda(cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi));
    if (st == KITC_OK)
        st = kitc_from_cuda(cudaStreamCreateWithPriority(&side, cudaStreamNonBlocking, prio_hi));
    if (st == KITC_OK) st = kitc_from_cuda(cudaEventCreateWithFlags(&built, cudaEventDisableTiming));
    if (st == KITC_OK) st = kitc_from_cuda(cudaEventCreateWithFlags(&planned, cudaEventDisableTiming));
    if (st == KITC_OK) st = kitc_from_cuda(cudaEventRecord(built, s));
    if (st == KITC_OK) st = kitc_modified_weights(t, dw.as<double>(), stream);
    if (st == KITC_OK) st = kitc_from_cuda(cudaStreamWaitEvent(side, built, 0));
    if (st == KITC_OK)
        st = kitc_plan_targets(t, tgt_xyz ? dt.as<double>() : dx.as<double>(), n_tgt, side);
    if (st == KITC_OK) st = kitc_from_cuda(cudaEventRecord(planned, side));
    if (st == KITC_OK) st = kitc_from_cuda(cudaStreamWaitEvent(s, planned, 0));
    if (st == KITC_OK) st = kitc_evaluate_planned(t, dout.as<double>(), stream);
    if (side) {
        cudaStreamSynchronize(side);  // nothing of this call may still run on it
        cudaStreamDestroy(side);
    }
    if (built) cudaEventDestroy(built);
    if (planned) cudaEventDestroy(planned);
    if (st == KITC_OK)
        st = kitc_from_cuda(cudaMemcpyAsync(out, dout.ptr, sizeof(double) * wout * n_tgt,
                                            cudaMemcpyDeviceToHost, s));
    if (st == KITC_OK) st = kitc_from_cuda(cudaStreamSynchronize(s));
    if (t) kitc_free_tree(t);
    for (DevBuf *b : {&dx, &dw, &dt, &dout}) b->release(s);
    return st;
}

kitc_status kitc_get_stats(kitc_tree t, kitc_stats *s)
{
    if (!t || !s) return KITC_ERR_INVALID_ARG;
    memset(s, 0, sizeof(*s));
    s->n_sources = t->src.n;
    s->n_clusters = t->src.nclus;
    s->n_leaves = t->src.nleaves;
    s->depth = t->src.depth;
    s->degree = t->p.degree;
    if (t->evaluated || t->lists_ready) {
        s->n_targets = t->lists.nt;
        s->n_batches = t->lists.nb;
        s->far_entries = t->lists.nfar;
        s->near_entries = t->lists.nnear;
        s->near_pairs = t->lists.near_pairs;
        s->far_points = t->lists.far_points;
        s->near_exec = t->lists.near_exec;
        s->far_exec = t->lists.far_exec;
    }
    s->device_bytes = (int64_t)(t->src.bytes() + t->tgt.bytes() + t->wts.bytes() +
                                t->lists.bytes() + t->flags.bytes);
    if (t->ev_ok) {
        float *ms[4] = {&s->ms_tree, &s->ms_weights, &s->ms_lists, &s->ms_evaluate};
        int pairs[4][2] = {{0, 1}, {2, 3}, {4, 5}, {5, 6}};
        for (int i = 0; i < 4; ++i) {
            if (!t->stage_done[i]) continue;
            KITC_CUDA(cudaEventSynchronize(t->ev[pairs[i][1]]));
            KITC_CUDA(cudaEventElapsedTime(ms[i], t->ev[pairs[i][0]], t->ev[pairs[i][1]]));
        }
    }
    return KITC_OK;
}

kitc_status kitc_tree_download(kitc_tree t, int64_t *perm, double *lo, double *hi,
                               int64_t *begin, int64_t *end, int32_t *first_child,
                               int32_t *n_child, int32_t *level, int32_t *parent, void *stream)
{
    if (!t) return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int m = t->src.nclus;
    int64_t n = t->src.n;
    std::vector<int32_t> tmp((size_t)std::max<int64_t>(n, m));
    if (perm) {
        KITC_CUDA(cudaMemcpyAsync(tmp.data(), t->src.perm.ptr, sizeof(int32_t) * n,
                                  cudaMemcpyDeviceToHost, s));
        KITC_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < n; ++i) perm[i] = tmp[i];
    }
    std::vector<dvec4> b4(m);
    for (int side = 0; side < 2; ++side) {
        double *dst = side ? hi : lo;
        if (!dst) continue;
        KITC_CUDA(cudaMemcpyAsync(b4.data(), (side ? t->src.hi : t->src.lo).ptr,
                                  sizeof(dvec4) * m, cudaMemcpyDeviceToHost, s));
        KITC_CUDA(cudaStreamSynchronize(s));
        for (int c = 0; c < m; ++c) {
            dst[3 * c] = b4[c].x;
            dst[3 * c + 1] = b4[c].y;
            dst[3 * c + 2] = b4[c].z;
        }
    }
    const DevBuf *src64[2] = {&t->src.begin, &t->src.end};
    int64_t *dst64[2] = {begin, end};
    for (int i = 0; i < 2; ++i) {
        if (!dst64[i]) continue;
        KITC_CUDA(cudaMemcpyAsync(tmp.data(), src64[i]->ptr, sizeof(int32_t) * m,
                                  cudaMemcpyDeviceToHost, s));
        KITC_CUDA(cudaStreamSynchronize(s));
        for (int c = 0; c < m; ++c) dst64[i][c] = tmp[c];
    }
    const DevBuf *src32[4] = {&t->src.first_child, &t->src.n_child, &t->src.level, &t->src.parent};
    int32_t *dst32[4] = {first_child, n_child, level, parent};
    for (int i = 0; i < 4; ++i)
        if (dst32[i])
            KITC_CUDA(cudaMemcpyAsync(dst32[i], src32[i]->ptr, sizeof(int32_t) * m,
                                      cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    return KITC_OK;
}

kitc_status kitc_weights_download(kitc_tree t, double *fhat, void *stream)
{
    if (!t || !fhat) return KITC_ERR_INVALID_ARG;
    if (!t->has_weights) return KITC_ERR_STATE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (t->var) {  // gather each cluster's weights, in cluster order
        const int m = t->src.nclus;
        std::vector<double> all((size_t)std::max<int64_t>(t->wts.fhat_len, 1));
        std::vector<int64_t> fo(m);
        const int64_t *d_f = weights_foff(t->src, t->wts);
        if (!d_f) return KITC_ERR_STATE;
        KITC_CUDA(cudaMemcpyAsync(all.data(), t->wts.fhat.ptr, sizeof(double) * t->wts.fhat_len,
                                  cudaMemcpyDeviceToHost, s));
        KITC_CUDA(cudaMemcpyAsync(fo.data(), d_f, sizeof(int64_t) * m, cudaMemcpyDeviceToHost, s));
        KITC_CUDA(cudaStreamSynchronize(s));
        size_t o = 0;
        for (int c = 0; c < m; ++c) {
            int d = t->hdeg[c];
            if (d <= 0) continue;
            size_t k = (size_t)(d + 1) * (d + 1) * (d + 1) * t->win;
            memcpy(fhat + o, all.data() + fo[c], sizeof(double) * k);
            o += k;
        }
        return KITC_OK;
    }
    int np = t->p.degree + 1;
    size_t bytes = sizeof(double) * (size_t)t->src.nclus * np * np * np * t->win;
    KITC_CUDA(cudaMemcpyAsync(fhat, t->wts.fhat.ptr, bytes, cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    return KITC_OK;
}

kitc_status kitc_lists_download(kitc_tree t, int64_t *tperm, int64_t *nfar, int64_t *nnear,
                                int32_t *far, uint64_t *far_mask, int32_t *near,
                                uint64_t *near_mask, void *stream)
{
    if (!t) return KITC_ERR_INVALID_ARG;
    if (!t->evaluated) return KITC_ERR_STATE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const ListsDev &L = t->lists;
    if (tperm) {
        std::vector<int32_t> tmp(L.nt);
        KITC_CUDA(cudaMemcpyAsync(tmp.data(), t->tgt.perm.ptr, sizeof(int32_t) * L.nt,
                                  cudaMemcpyDeviceToHost, s));
        KITC_CUDA(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < L.nt; ++i) tperm[i] = tmp[i];
    }
    std::vector<int64_t> off(L.nb + 1);
    for (int k = 0; k < 2; ++k) {
        int64_t *dst = k ? nnear : nfar;
        if (!dst) continue;
        KITC_CUDA(cudaMemcpyAsync(off.data(), (k ? L.near_off : L.far_off).ptr,
                                  sizeof(int64_t) * (L.nb + 1), cudaMemcpyDeviceToHost, s));
        KITC_CUDA(cudaStreamSynchronize(s));
        for (int64_t b = 0; b < L.nb; ++b) dst[b] = off[b + 1] - off[b];
    }
    if (far) KITC_CUDA(cudaMemcpyAsync(far, L.far_id.ptr, sizeof(int32_t) * L.nfar, cudaMemcpyDeviceToHost, s));
    if (far_mask)
        KITC_CUDA(cudaMemcpyAsync(far_mask, L.far_mask.ptr, sizeof(uint64_t) * L.nfar, cudaMemcpyDeviceToHost, s));
    if (near) KITC_CUDA(cudaMemcpyAsync(near, L.near_id.ptr, sizeof(int32_t) * L.nnear, cudaMemcpyDeviceToHost, s));
    if (near_mask)
        KITC_CUDA(cudaMemcpyAsync(near_mask, L.near_mask.ptr, sizeof(uint64_t) * L.nnear, cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    return KITC_OK;
}

void kitc_free_tree(kitc_tree t)
{
    if (t) free_handle(t);
}

int64_t kitc_launch_count(void) { return g_launches.load(); }

kitc_status kitc_apply(kitc_tree t, const double *w, double *out, void *stream)
{
    if (!t || !device_accessible(w) || !device_accessible(out)) return KITC_ERR_INVALID_ARG;
    if (!t->evaluated) return KITC_ERR_STATE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    t->stream = s;
    EvalArgs a = t->last;
    a.out = out;
    const bool mixed = is_mixed(t->p.precision);
    auto body = [&]() -> kitc_status {
        KITC_TRY(launch_weights(t, w, s));
        KITC_CUDA(cudaMemsetAsync(t->flags.ptr, 0, 4 * sizeof(int), s));
        return evaluate_launch(t->p.kernel, mixed, a, s);
    };
    KITC_TRY(prepare_weights(t, s));
    if (!s) {  // the legacy default stream cannot be captured: launch directly
        KITC_TRY(body());
    } else {
        if (!t->graph || t->graph_w != w || t->graph_out != out || t->graph_stream != s) {
            if (t->graph) {
                cudaGraphExecDestroy(t->graph);
                t->graph = nullptr;
            }
            KITC_TRY(body());  // eager run: sets every kernel attribute before the capture
            int64_t l0 = g_launches.load();
            KITC_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            kitc_status st = body();
            cudaGraph_t g = nullptr;
            cudaError_t e = cudaStreamEndCapture(s, &g);
            if (st != KITC_OK || e != cudaSuccess) {
                if (g) cudaGraphDestroy(g);
                return st != KITC_OK ? st : kitc_from_cuda(e);
            }
            e = cudaGraphInstantiate(&t->graph, g, 0);
            cudaGraphDestroy(g);
            if (e != cudaSuccess) {
                t->graph = nullptr;
                return kitc_from_cuda(e);
            }
            t->graph_launches = g_launches.load() - l0;
            t->graph_w = w;
            t->graph_out = out;
            t->graph_stream = s;
        } else {
            g_launches.fetch_add(t->graph_launches);
        }
        KITC_CUDA(cudaGraphLaunch(t->graph, s));
    }
    t->has_weights = true;
    return read_error_flag(t->flags.as<int>() + 1, s);
}

kitc_status kitc_watchdog_selftest(int limit_ms, void *stream)
{
    if (limit_ms < 1 || limit_ms > 10000) return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    DevBuf flag;
    KITC_TRY(flag.reserve(sizeof(int), s));
    kitc_status st = kitc_from_cuda(cudaMemsetAsync(flag.ptr, 0, sizeof(int), s));
    if (st == KITC_OK) st = watchdog_launch((unsigned long long)limit_ms * 1000000ull, flag.as<int>(), s);
    if (st == KITC_OK) st = read_error_flag(flag.as<int>(), s);
    flag.release(s);
    return st;
}


kitc_status kitc_set_degrees(kitc_tree t, const int32_t *degrees, void *stream)
{
    if (!t) return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int m = t->src.nclus;
    std::vector<int32_t> h;
    if (degrees) {
        h.resize(m);
        KITC_CUDA(cudaMemcpyAsync(h.data(), degrees, sizeof(int32_t) * m, cudaMemcpyDefault, s));
        KITC_CUDA(cudaStreamSynchronize(s));
        for (int c = 0; c < m; ++c)
            if (h[c] < 0 || h[c] > KITC_MAX_DEGREE) return KITC_ERR_INVALID_ARG;
    }
    // a new degree map invalidates the weights, the lists and the captured graph
    if (t->graph) {
        cudaGraphExecDestroy(t->graph);
        t->graph = nullptr;
    }
    t->has_weights = t->evaluated = false;
    t->wts.planned = false;
    t->var = false;
    if (!degrees) return KITC_OK;
    const bool mixed = is_mixed(t->p.precision);
    const bool pairs = uses_pair_records(t->p.kernel, mixed);
    std::vector<int64_t> ro;
    t->proxy_bytes = proxy_offsets_var(h, t->win, mixed, pairs, pairs && uses_row_pairs(t->p.kernel), ro);
    std::vector<double> tab((KITC_MAX_DEGREE + 1) * (KITC_MAX_DEGREE + 1), 0.0);
    for (int d = 1; d <= KITC_MAX_DEGREE; ++d) cheb_cos_table(d, &tab[(size_t)d * (KITC_MAX_DEGREE + 1)]);
    KITC_TRY(t->cdeg.reserve(sizeof(int32_t) * m, s));
    KITC_TRY(t->roff.reserve(sizeof(int64_t) * m, s));
    KITC_TRY(t->chebt.reserve(sizeof(double) * tab.size(), s));
    KITC_CUDA(cudaMemcpyAsync(t->cdeg.ptr, h.data(), sizeof(int32_t) * m, cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(t->roff.ptr, ro.data(), sizeof(int64_t) * m, cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaMemcpyAsync(t->chebt.ptr, tab.data(), sizeof(double) * tab.size(),
                              cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaStreamSynchronize(s));  // the host vectors must outlive the copies
    t->hdeg.swap(h);
    t->var = true;
    return KITC_OK;
}


kitc_status kitc_plan_targets(kitc_tree t, const double *tgt_xyz, int64_t n_tgt, void *stream)
{
    if (!t || !valid_count(n_tgt) || !device_accessible(tgt_xyz)) return KITC_ERR_INVALID_ARG;
    if (t->src.nsys > 1) return KITC_ERR_STATE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    t->stream = s;
    t->evaluated = false;
    return plan_impl(t, tgt_xyz, n_tgt, nullptr, 1, s);
}

kitc_status kitc_plan_targets_forest(kitc_tree t, const double *tgt_xyz, const int64_t *tgt_counts,
                                     void *stream)
{
    if (!t || !tgt_counts || !device_accessible(tgt_xyz)) return KITC_ERR_INVALID_ARG;
    const int nsys = t->src.nsys;
    int64_t tot = 0;
    for (int k = 0; k < nsys; ++k) {
        if (tgt_counts[k] < 1) return KITC_ERR_INVALID_ARG;
        tot += tgt_counts[k];
    }
    if (!valid_count(tot)) return KITC_ERR_INVALID_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    t->stream = s;
    t->evaluated = false;
    return plan_impl(t, tgt_xyz, tot, tgt_counts, nsys, s);
}

static kitc_status ensure_cheb_table(kitc_tree t, cudaStream_t s)
{
    if (t->chebt.ptr) return KITC_OK;
    std::vector<double> tab((KITC_MAX_DEGREE + 1) * (KITC_MAX_DEGREE + 1), 0.0);
    for (int d = 1; d <= KITC_MAX_DEGREE; ++d) cheb_cos_table(d, &tab[(size_t)d * (KITC_MAX_DEGREE + 1)]);
    KITC_TRY(t->chebt.reserve(sizeof(double) * tab.size(), s));
    KITC_CUDA(cudaMemcpyAsync(t->chebt.ptr, tab.data(), sizeof(double) * tab.size(),
                              cudaMemcpyHostToDevice, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    return KITC_OK;
}

static LearnArgs learn_args(kitc_tree t)
{
    LearnArgs a;
    a.nclus = t->src.nclus;
    a.win = t->win;
    a.degree = t->p.degree;
    a.eps = t->p.eps;
    a.cbegin = t->src.begin.as<int32_t>();
    a.cend = t->src.end.as<int32_t>();
    a.perm = t->src.perm.as<int32_t>();
    a.level = t->src.level.as<int32_t>();
    a.first_child = t->src.first_child.as<int32_t>();
    a.n_child = t->src.n_child.as<int32_t>();
    a.cdeg = t->var ? t->cdeg.as<int32_t>() : nullptr;
    a.ctr = t->src.ctr.as<dvec4>();
    a.clo = t->src.lo.as<dvec4>();
    a.chi = t->src.hi.as<dvec4>();
    a.sxs = t->src.xs.as<double>();
    a.ns = t->src.n;
    a.txs = t->tgt.xs.as<double>();
    a.nt = t->lists.nt;
    a.nb = t->lists.nb;
    a.batch = t->lists.batch;
    a.bdesc = t->lists.forest ? t->lists.bdesc.as<int32_t>() : nullptr;
    a.far_off = t->lists.far_off.as<int64_t>();
    a.far_id = t->lists.far_id.as<int32_t>();
    a.far_mask = t->lists.far_mask.as<uint64_t>();
    a.fhat = t->wts.fhat.as<double>();
    a.foff = t->var ? weights_foff(t->src, t->wts) : nullptr;
    a.chebt = t->chebt.as<double>();
    a.err = t->flags.as<int>() + 1;
    return a;
}

kitc_status kitc_cluster_features(kitc_tree t, const double *w, float *features, void *stream)
{
    if (!t || !device_accessible(w) || !device_accessible(features)) return KITC_ERR_INVALID_ARG;
    if (!t->lists_ready) return KITC_ERR_STATE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    KITC_TRY(ensure_cheb_table(t, s));
    return learn_features(learn_args(t), t->src.level_start, w, features, t->learn, s);
}

kitc_status kitc_cluster_far_errors(kitc_tree t, const double *w, int max_samples, uint64_t seed,
                                    double *err2, int32_t *n_samples, void *stream)
{
    if (!t || !device_accessible(w) || !device_accessible(err2) || !device_accessible(n_samples) ||
        max_samples < 1 || t->p.kernel == KITC_TEST_POLY)
        return KITC_ERR_INVALID_ARG;
    if (!t->lists_ready || !t->has_weights) return KITC_ERR_STATE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    KITC_TRY(ensure_cheb_table(t, s));
    LearnArgs a = learn_args(t);
    if (t->var && !a.foff) return KITC_ERR_STATE;
    KITC_CUDA(cudaMemsetAsync(t->flags.ptr, 0, 4 * sizeof(int), s));
    KITC_TRY(learn_far_errors(t->p.kernel, a, w, max_samples, (unsigned long long)seed, err2,
                              n_samples, t->learn, s));
    int *h = nullptr;
    KITC_TRY(host_readback_buffer(reinterpret_cast<void **>(&h)));
    KITC_CUDA(cudaMemcpyAsync(h, t->flags.as<int>() + 1, sizeof(int), cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    return h[0] ? KITC_ERR_INVALID_ARG : KITC_OK;
}

}  // extern "C"
