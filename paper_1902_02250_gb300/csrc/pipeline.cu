// The treecode as one queue of device work (kitc_pipeline.h): source tree,
// modified weights and records, target tree, interaction lists and the
// evaluator, with every size read on the device instead of the host, in
// buffers reserved once.  The target tree and the lists run on a second
// stream while the weights pass runs (they need only the source tree), joined
// before the evaluator; under capture the fork and the join become graph
// edges.
#include <math.h>
#include <string.h>

#include <algorithm>

#include "common.cuh"
#include "kitc_pipeline.h"

namespace {

// flags: [evaluator work counter | evaluator error | pipeline error word | 0]
constexpr int FLAG_ERR = 2;

}  // namespace

struct kitc_pipeline_s {
    kitc_params p{};
    int win = 3, wout = 3, device = 0;
    int nsys = 1;
    bool self_targets = false;
    TreeAsync src, tgt;
    WeightsDev wts;
    ListsDev lists;
    DevBuf flags;
    EvalArgs a{};
    // second stream and fork/join events of a run: [0] eager runs, [1] the
    // capture of kitc_pipeline_replay (which starts on its own stream cap)
    cudaStream_t side[2] = {nullptr, nullptr}, cap = nullptr;
    cudaEvent_t ev[2][3] = {};
    // graph of kitc_pipeline_replay
    cudaGraphExec_t graph = nullptr;
    const void *g_src = nullptr, *g_w = nullptr, *g_tgt = nullptr, *g_out = nullptr;
    int64_t graph_launches = 0;
};

namespace {

void destroy(kitc_pipeline h)
{
    cudaStream_t s = nullptr;
    if (h->side[0]) cudaStreamSynchronize(h->side[0]);
    if (h->graph) cudaGraphExecDestroy(h->graph);
    h->src.release(s);
    h->tgt.release(s);
    h->wts.release(s);
    h->lists.release(s);
    h->flags.release(s);
    for (auto &row : h->ev)
        for (cudaEvent_t e : row)
            if (e) cudaEventDestroy(e);
    for (cudaStream_t q : {h->side[0], h->side[1], h->cap})
        if (q) cudaStreamDestroy(q);
    delete h;
}

// Room for ceil(slack * used) + margin, at least minimum.
int64_t room(int64_t used, double slack, int64_t margin, int64_t minimum)
{
    return std::max<int64_t>(minimum, (int64_t)ceil(slack * (double)used) + margin);
}

// One run queued on s, with its second stream and events from set k.
kitc_status run_impl(kitc_pipeline h, const double *src_xyz, const double *w, const double *tgt_xyz,
                     double *out, cudaStream_t s, int k)
{
    const kitc_params &p = h->p;
    const bool mixed = is_mixed(p.precision);
    const bool pairs = uses_pair_records(p.kernel, mixed);
    int *flags = h->flags.as<int>();
    int *err = flags + FLAG_ERR;
    cudaStream_t side = h->side[k];
    cudaEvent_t *ev = h->ev[k];  // fork, source tree done, join
    if (!tgt_xyz) tgt_xyz = src_xyz;
    KITC_CUDA(cudaMemsetAsync(flags, 0, 4 * sizeof(int), s));
    KITC_CUDA(cudaEventRecord(ev[0], s));
    KITC_CUDA(cudaStreamWaitEvent(side, ev[0], 0));
    // second stream: target tree, then (after the source tree) the lists
    KITC_TRY(tree_async_launch(h->tgt, tgt_xyz, err, side));
    // first stream: source tree, weights and records
    KITC_TRY(tree_async_launch(h->src, src_xyz, err, s));
    KITC_CUDA(cudaEventRecord(ev[1], s));
    KITC_CUDA(cudaStreamWaitEvent(side, ev[1], 0));
    KITC_TRY(lists_async_launch(h->src, h->tgt, p.theta, p.degree, p.mac, err, side, h->lists));
    KITC_CUDA(cudaEventRecord(ev[2], side));
    KITC_TRY(weights_async_launch(h->src, w, h->wts, mixed, pairs, err, s));
    KITC_CUDA(cudaStreamWaitEvent(s, ev[2], 0));
    EvalArgs a = h->a;
    a.out = out;
    return evaluate_launch(p.kernel, mixed, a, s);
}

// The handle's buffers live on the device that was current at creation.
bool on_device(kitc_pipeline h)
{
    int d = -1;
    return cudaGetDevice(&d) == cudaSuccess && d == h->device;
}

}  // namespace

extern "C" {

kitc_status kitc_pipeline_create(const double *src_xyz, const int64_t *src_counts,
                                 const double *tgt_xyz, const int64_t *tgt_counts, int num_systems,
                                 const kitc_params *p, double slack, void *stream, kitc_pipeline *out)
{
    if (!out) return KITC_ERR_INVALID_ARG;
    *out = nullptr;
    if (!valid_params(p) || !src_counts || num_systems < 1 || !(slack >= 1.0) || !isfinite(slack) ||
        !device_accessible(src_xyz) || (tgt_xyz && (!tgt_counts || !device_accessible(tgt_xyz))))
        return KITC_ERR_INVALID_ARG;
    const int nsys = num_systems;
    int64_t ns = 0, nt = 0;
    for (int k = 0; k < nsys; ++k) {
        if (src_counts[k] < 1 || (tgt_xyz && tgt_counts[k] < 1)) return KITC_ERR_INVALID_ARG;
        ns += src_counts[k];
        nt += tgt_xyz ? tgt_counts[k] : src_counts[k];
    }
    if (!valid_count(ns) || !valid_count(nt)) return KITC_ERR_INVALID_ARG;
    const int64_t *tc = tgt_xyz ? tgt_counts : src_counts;
    const double *txyz = tgt_xyz ? tgt_xyz : src_xyz;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    kitc_pipeline h = new kitc_pipeline_s();
    h->p = *p;
    h->p.target_batch = batch_of(*p);
    h->win = kitc_kernel_win(p->kernel);
    h->wout = kitc_kernel_wout(p->kernel);
    h->nsys = nsys;
    h->self_targets = tgt_xyz == nullptr;
    cudaGetDevice(&h->device);
    const int B = h->p.target_batch;
    const bool mixed = is_mixed(p->precision);
    const bool pairs = uses_pair_records(p->kernel, mixed);
    auto fail = [&](kitc_status st) {
        destroy(h);
        return st;
    };
    // one eager build on the example inputs: the sizes to reserve
    TreeDev es, et;
    ListsDev el;
    const int64_t *sc = nsys > 1 ? src_counts : nullptr;
    const int64_t *tcc = nsys > 1 ? tc : nullptr;
    kitc_status st = tree_build(src_xyz, ns, p->leaf_size, s, es, sc, nsys);
    if (st == KITC_OK) st = tree_build(txyz, nt, B, s, et, tcc, nsys);
    if (st == KITC_OK) st = lists_build(es, et, B, p->theta, p->degree, nullptr, p->mac, s, el);
    if (st != KITC_OK) {
        es.release(s);
        et.release(s);
        el.release(s);
        return fail(st);
    }
    const int cap_s = (int)std::min<int64_t>(INT32_MAX / 4, room(es.nclus, slack, 64, nsys));
    const int cap_t = (int)std::min<int64_t>(INT32_MAX / 4, room(et.nclus, slack, 64, nsys));
    const int lev_s = std::min(KITC_MAX_LEVEL + 1, es.depth + 2);
    const int lev_t = std::min(KITC_MAX_LEVEL + 1, et.depth + 2);
    const int64_t cap_far = room(el.nfar, slack, 1024, 1024);
    const int64_t cap_near = room(el.nnear, slack, 1024, 1024);
    es.release(s);
    et.release(s);
    el.release(s);
    st = tree_async_reserve(h->src, ns, p->leaf_size, sc, nsys, cap_s, lev_s, s);
    if (st == KITC_OK) st = tree_async_reserve(h->tgt, nt, B, tcc, nsys, cap_t, lev_t, s);
    if (st == KITC_OK)
        st = weights_async_reserve(h->src, h->win, p->degree, p->weights, mixed && weights_split_enabled(),
                                   mixed, pairs, pairs && uses_row_pairs(p->kernel),
                                   uses_leaf_offsets(*p), s, h->wts);
    if (st == KITC_OK) st = lists_async_reserve(h->src, h->tgt, B, cap_far, cap_near, s, h->lists);
    if (st == KITC_OK) st = h->flags.reserve(4 * sizeof(int), s);
    for (cudaStream_t *q : {&h->side[0], &h->side[1], &h->cap})
        if (st == KITC_OK) st = kitc_from_cuda(cudaStreamCreateWithFlags(q, cudaStreamNonBlocking));
    for (auto &row : h->ev)
        for (cudaEvent_t &e : row)
            if (st == KITC_OK) st = kitc_from_cuda(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
    // a status read before any run finds no error and zero counts
    if (st == KITC_OK) st = kitc_from_cuda(cudaMemsetAsync(h->flags.ptr, 0, 4 * sizeof(int), s));
    if (st == KITC_OK) st = kitc_from_cuda(cudaMemsetAsync(h->lists.totals.ptr, 0, h->lists.totals.bytes, s));
    if (st == KITC_OK) st = kitc_from_cuda(cudaMemsetAsync(h->src.sc.state(), 0, sizeof(BuildState), s));
    if (st == KITC_OK) st = kitc_from_cuda(cudaStreamSynchronize(s));
    if (st != KITC_OK) return fail(st);
    // evaluator arguments: every pointer is fixed but the output
    EvalArgs &a = h->a;
    const TreeDev &S = h->src.t, &T = h->tgt.t;
    const ListsDev &L = h->lists;
    a.tx = T.xs.as<double>();
    a.ty = a.tx + nt;
    a.tz = a.tx + 2 * nt;
    a.tstride = 1;
    a.tperm = T.perm.as<int32_t>();
    a.nt = nt;
    a.batch = B;
    a.nb = L.nb;
    a.bctr = L.bctr.as<dvec4>();
    if (L.forest) {
        a.bstart = L.bdesc.as<int32_t>();
        a.bcount = a.bstart + L.nb;
    }
    a.far_off = L.far_off.as<int64_t>();
    a.near_off = L.near_off.as<int64_t>();
    a.far_id = L.far_id.as<int32_t>();
    a.near_id = L.near_id.as<int32_t>();
    a.far_mask = L.far_mask.as<uint64_t>();
    a.near_mask = L.near_mask.as<uint64_t>();
    a.src = h->wts.src.ptr;
    a.proxy = h->wts.proxy.ptr;
    a.clo = S.lo.as<dvec4>();
    a.chi = S.hi.as<dvec4>();
    a.cbegin = S.begin.as<int32_t>();
    a.cend = S.end.as<int32_t>();
    a.pbegin = pairs ? h->wts.pbegin.as<int32_t>() : nullptr;
    fill_eval_common(a, h->p, h->flags.as<int>());
    *out = h;
    return KITC_OK;
}

kitc_status kitc_pipeline_run(kitc_pipeline h, const double *src_xyz, const double *w,
                              const double *tgt_xyz, double *out, void *stream)
{
    if (!h || !src_xyz || !w || !out || (tgt_xyz != nullptr) == h->self_targets)
        return KITC_ERR_INVALID_ARG;
    if (!on_device(h)) return KITC_ERR_STATE;
    return run_impl(h, src_xyz, w, tgt_xyz, out, reinterpret_cast<cudaStream_t>(stream), 0);
}

kitc_status kitc_pipeline_replay(kitc_pipeline h, const double *src_xyz, const double *w,
                                 const double *tgt_xyz, double *out, void *stream)
{
    if (!h || !src_xyz || !w || !out || (tgt_xyz != nullptr) == h->self_targets)
        return KITC_ERR_INVALID_ARG;
    if (!on_device(h)) return KITC_ERR_STATE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (h->graph && h->g_src == src_xyz && h->g_w == w && h->g_tgt == tgt_xyz && h->g_out == out) {
        for (int64_t i = 0; i < h->graph_launches; ++i) kitc_count_launch();
        KITC_CUDA(cudaGraphLaunch(h->graph, s));
        return KITC_OK;
    }
    if (h->graph) {
        cudaGraphExecDestroy(h->graph);
        h->graph = nullptr;
    }
    // this call's result comes from a run on the caller's stream, which also
    // loads and configures every kernel before the capture
    KITC_TRY(run_impl(h, src_xyz, w, tgt_xyz, out, s, 0));
    // the capture starts on the handle's own stream, so that any stream of
    // the caller (the legacy default stream too) can launch the graph
    const int64_t l0 = kitc_launch_count();
    KITC_CUDA(cudaStreamBeginCapture(h->cap, cudaStreamCaptureModeThreadLocal));
    kitc_status st = run_impl(h, src_xyz, w, tgt_xyz, out, h->cap, 1);
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->cap, &g);
    if (st != KITC_OK || e != cudaSuccess) {
        if (g) cudaGraphDestroy(g);
        return st != KITC_OK ? st : kitc_from_cuda(e);
    }
    e = cudaGraphInstantiate(&h->graph, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        h->graph = nullptr;
        return kitc_from_cuda(e);
    }
    h->graph_launches = kitc_launch_count() - l0;
    h->g_src = src_xyz;
    h->g_w = w;
    h->g_tgt = tgt_xyz;
    h->g_out = out;
    return KITC_OK;
}

kitc_status kitc_pipeline_status(kitc_pipeline h, kitc_stats *st, void *stream)
{
    if (!h) return KITC_ERR_INVALID_ARG;
    if (!on_device(h)) return KITC_ERR_STATE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int hf[4] = {0, 0, 0, 0};
    BuildState bs{};
    int64_t tot[8] = {};
    KITC_CUDA(cudaMemcpyAsync(hf, h->flags.ptr, sizeof(hf), cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaMemcpyAsync(&bs, h->src.state(), sizeof(bs), cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaMemcpyAsync(tot, h->lists.totals.ptr, sizeof(tot), cudaMemcpyDeviceToHost, s));
    KITC_CUDA(cudaStreamSynchronize(s));
    if (st) {
        memset(st, 0, sizeof(*st));
        st->n_sources = h->src.t.n;
        st->n_clusters = bs.nclus;
        st->n_leaves = bs.nleaves;
        st->depth = bs.depth;
        st->degree = h->p.degree;
        st->n_targets = h->lists.nt;
        st->n_batches = h->lists.nb;
        st->near_pairs = tot[0];
        st->far_points = tot[1];
        st->far_entries = tot[2];
        st->near_entries = tot[3];
        st->near_exec = tot[4];
        st->far_exec = tot[5];
        st->device_bytes = (int64_t)(h->src.bytes() + h->tgt.bytes() + h->wts.bytes() +
                                     h->lists.bytes() + h->flags.bytes);
    }
    const int perr = hf[FLAG_ERR];
    if (perr & (ASYNC_TREE_OVERFLOW | ASYNC_LIST_OVERFLOW | ASYNC_RECORD_OVERFLOW))
        return KITC_ERR_TOO_LARGE;
    if (perr & ASYNC_TRAVERSAL) return KITC_ERR_INVALID_ARG;
    if (hf[1]) return KITC_ERR_TIMEOUT;
    return KITC_OK;
}

int64_t kitc_pipeline_graph_launches(kitc_pipeline h) { return h ? h->graph_launches : 0; }

kitc_status kitc_pipeline_free(kitc_pipeline h)
{
    if (!h) return KITC_ERR_INVALID_ARG;
    destroy(h);
    return KITC_OK;
}

}  // extern "C"
