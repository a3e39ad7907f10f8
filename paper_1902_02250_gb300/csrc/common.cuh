// Internal declarations of libkitc (GB300 / sm_103a).  Not part of the ABI.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "kitc.h"

// Four doubles, 32-byte aligned (box corners, centre + radius).
struct alignas(32) dvec4 {
    double x, y, z, w;
};
__host__ __device__ inline dvec4 make_dvec4(double x, double y, double z, double w)
{
    dvec4 v;
    v.x = x;
    v.y = y;
    v.z = z;
    v.w = w;
    return v;
}

#define KITC_MAX_DEGREE 16
#define KITC_MAX_LEVEL 40      // splitting stops at this depth (degenerate inputs only)
#define KITC_MAX_BATCH 64      // targets per batch: two per lane of a warp

// ---------------------------------------------------------------------------
// Status plumbing: every CUDA call goes through KITC_CUDA, which turns an error
// into a kitc_status returned by the enclosing function.
// ---------------------------------------------------------------------------
kitc_status kitc_from_cuda(cudaError_t e);

#define KITC_CUDA(call)                                   \
    do {                                                  \
        cudaError_t _e = (call);                          \
        if (_e != cudaSuccess) return kitc_from_cuda(_e); \
    } while (0)

#define KITC_TRY(call)                      \
    do {                                    \
        kitc_status _s = (call);            \
        if (_s != KITC_OK) return _s;       \
    } while (0)

// A small pinned host buffer (64 bytes, per device and process) for
// read-backs of counts; callers synchronize the stream before reading it.
kitc_status host_readback_buffer(void **p);

// Stream-ordered device allocation from the device's default pool.
kitc_status dev_alloc(void **p, size_t bytes, cudaStream_t s);
void dev_free(void *p, cudaStream_t s);

template <typename T>
inline kitc_status dev_alloc_t(T **p, size_t count, cudaStream_t s)
{
    return dev_alloc(reinterpret_cast<void **>(p), count * sizeof(T), s);
}

// Device buffer owned by a handle; grows on demand, freed in the destructor
// of the owner through release().
struct DevBuf {
    void *ptr = nullptr;
    size_t bytes = 0;
    kitc_status reserve(size_t b, cudaStream_t s, bool keep = false);
    void release(cudaStream_t s);
    template <typename T> T *as() const { return reinterpret_cast<T *>(ptr); }
};

// ---------------------------------------------------------------------------
// Sec. 6 tree on the device.  Clusters are numbered breadth first; the
// children of a cluster are contiguous and ordered by octant code.
// ---------------------------------------------------------------------------
struct TreeDev {
    int64_t n = 0;          // particles
    int leaf = 0;           // N0
    int32_t nclus = 0, cap = 0, depth = 0, nleaves = 0;
    int32_t nsys = 1;       // independent systems; cluster s < nsys is the root of system s
    DevBuf perm;            // int32 [n]: perm[slot] = caller index
    DevBuf xs;              // double [3][n]: coordinates in tree order (SoA)
    DevBuf lo, hi;          // dvec4 [cap]: box corners (w unused)
    DevBuf ctr;             // dvec4 [cap]: centre xyz, radius in w (Fig. 1)
    DevBuf ctrf;            // float4 [2 cap]: centre as FP32 hi (+ radius) and lo parts
    DevBuf begin, end;      // int32 [cap]: slot range
    DevBuf first_child, n_child, level, parent;  // int32 [cap]
    std::vector<int32_t> level_start;            // host: first cluster of each level
    std::vector<int64_t> sys_off;                // host: first slot of each system (+ n)
    void release(cudaStream_t s);
    size_t bytes() const;
};

// State of the device-side level loop of the tree build.  Level l reads
// st[l & 1]; its children kernels write st[(l + 1) & 1].  Slots, permutation
// and cluster ids of the slots live in the first buffers while cur = 0 and in
// the second ones while cur = 1; a level that scatters sets flip, and the next
// level's split kernel applies it (after the scatter has read cur).
// level_start[d] is the first cluster of level d for d < depth; nclus ends the
// last level.  overflow: a level's children did not fit the cluster capacity
// (the tree then stops there, its clusters of that level staying leaves).
struct LevelState {
    int lb, nl;  // clusters [lb, lb + nl) of one level
};
struct BuildState {
    LevelState st[2];
    int nclus, depth, nleaves, overflow, cur, flip;
    int level_start[KITC_MAX_LEVEL + 2];
};

// Scratch of one tree build: the second buffers of the slot arrays, the
// per-block and per-level scratch, the root chunks and the state block.
struct TreeScratch {
    DevBuf perm2, xs2, node, node2, offs, bcount, lvl;
    int nblk = 0, nc = 0, nsys = 1, cap = 0;
    int64_t max_nl = 0;
    size_t n64 = 0, n32 = 0;       // int64 and int32 entries at the start of offs
    std::vector<int64_t> hoff;     // first slot of each system (+ n)
    BuildState *state() const;
    void release(cudaStream_t s);
};

// A tree whose build runs without any host read-back, so that it can be
// captured in a CUDA graph: buffers for cap clusters and `levels` levels are
// reserved once (tree_async_reserve); tree_async_launch queues the whole
// build.  The host never learns nclus, depth or the level starts: kernels
// downstream read them from state().  If the tree needs more clusters than cap
// or more levels than `levels`, bit ASYNC_TREE_OVERFLOW is set in *err; the
// arrays still hold a valid (coarser) tree, so every later kernel stays in
// bounds.
struct TreeAsync {
    TreeDev t;
    TreeScratch sc;
    int levels = 0;
    const BuildState *state() const { return sc.state(); }
    void release(cudaStream_t s);
    size_t bytes() const;
};
constexpr int ASYNC_TREE_OVERFLOW = 1;   // bits of the pipeline's error word
constexpr int ASYNC_LIST_OVERFLOW = 2;
constexpr int ASYNC_RECORD_OVERFLOW = 4;
constexpr int ASYNC_TRAVERSAL = 8;       // a traversal stack overflowed (lists)

kitc_status tree_async_reserve(TreeAsync &a, int64_t n, int leaf, const int64_t *counts, int nsys,
                               int cap, int levels, cudaStream_t s);
kitc_status tree_async_launch(TreeAsync &a, const double *xyz, int *err, cudaStream_t s);

// Builds the tree of the n points xyz (device, n x 3 row-major), or a forest
// with one tree per system when counts (host, nsys entries summing to n) is
// given: system k owns rows [sum_{j<k} counts[j], ...).  Reads back the child
// count of every level (one synchronization per level).
kitc_status tree_build(const double *xyz, int64_t n, int leaf, cudaStream_t s, TreeDev &t,
                       const int64_t *counts = nullptr, int nsys = 1);

// ---------------------------------------------------------------------------
// Modified weights (Eq. modified_weights / Algorithm 1) and the packed
// records the evaluator streams.
// ---------------------------------------------------------------------------
struct WeightsDev {
    int degree = 0, win = 0, mode = 0;
    // plan of the weights pass (weights_plan), reused by weights_launch
    bool planned = false, upward = false;
    size_t nitems = 0;
    int pair_ranges = 0;  // ranges of the paired records (pack_pairs_plan)
    // degree per cluster (weights_plan_var): one Algorithm 1 launch per degree
    struct Group {
        int degree = 0;
        size_t item0 = 0, nitems = 0;
        int64_t pofs = 0;
    };
    std::vector<Group> groups;
    bool split = false;       // split-precision products (mixed form)
    bool var = false;
    bool var_upward = false;  // degree map: upward form (else Algorithm 1 on every cluster)
    int var_pmax = 0;         // degree map: largest grid size of the upward form
    int64_t fhat_len = 0;     // doubles of fhat in use
    bool rowpairs = false;    // paired grid records in the row-pair form (uses_row_pairs)
    bool leaf = false;        // paired source records as leaf offsets (uses_leaf_offsets)
    bool async = false;       // device-planned (weights_async_reserve): nitems is the item capacity
    int64_t paircap = 0;      // device-planned paired records: capacity in pairs
    DevBuf fhat;      // double [nclus][P][win]
    DevBuf proxy;     // evaluator records of fhat (FP32 or FP64, padded)
    DevBuf src;       // evaluator records of the sources in tree order
    DevBuf pbegin;    // int32 [nclus]: first source pair of each leaf (paired records)
    DevBuf partial;   // scratch of the weights pass
    DevBuf items;     // scratch: work items of the weights pass
    void release(cudaStream_t s);
    size_t bytes() const;
};

int proxy_record_bytes(int win, bool mixed);
int source_record_bytes(int win, bool mixed);

// cos(k pi / n), k = 0..n (Eq. Chebyshev_points), computed on the host.
void cheb_cos_table(int n, double *t);

kitc_status weights_compute(const TreeDev &t, const double *w_user, int win, int degree, int mode,
                            cudaStream_t s, WeightsDev &wd);
kitc_status weights_plan(const TreeDev &t, int win, int degree, int mode, cudaStream_t s,
                         WeightsDev &wd);
kitc_status weights_launch(const TreeDev &t, const double *w_user, WeightsDev &wd, cudaStream_t s);
kitc_status pack_sources(const TreeDev *t, const double *xyz_user, const double *w_user,
                         int64_t n, int win, bool mixed, cudaStream_t s, DevBuf &out);
kitc_status pack_proxies(const TreeDev &t, WeightsDev &wd, bool mixed, cudaStream_t s);
// The FP32x2 evaluator (mixed precision, three weight components: the
// Stokeslet and the rotlet) reads paired source and grid records.
constexpr bool uses_pair_records(int kernel, bool mixed)
{
    return mixed && (kernel == KITC_STOKESLET || kernel == KITC_ROTLET);
}
// Both mixed forms (FP32 kernel values, FP64 sums).
constexpr bool is_mixed(int precision) { return precision == KITC_MIXED || precision == KITC_MIXED_LEAF; }
// A tree's paired source records hold offsets from the leaf's box centre
// (KITC_MIXED_LEAF with eps > 0: at eps = 0 nothing bounds the kernel of a
// close pair, whose difference would then carry the offsets' rounding).
inline bool uses_leaf_offsets(const kitc_params &p)
{
    return p.precision == KITC_MIXED_LEAF && uses_pair_records(p.kernel, true) && p.eps > 0.0;
}
// Paired FP32x2 grid records of the modified weights.
kitc_status pack_proxy_pairs(const TreeDev &t, WeightsDev &wd, cudaStream_t s);
// Paired grid records of one cluster with np points per axis, 32 bytes each.
// Each grid row (k1, k2) holds ceil(np / 2) records of consecutive k3 points,
// a missing last point with zero weight.  With row pairs (the rotlet's form)
// and odd np, each record instead holds one k3 point of two consecutive grid
// rows (row index k1 np + k2), the last row of the odd count paired with a
// zero-weight row.
constexpr bool uses_row_pairs(int kernel) { return kernel == KITC_ROTLET; }
__host__ __device__ inline int64_t pair_records(int np, bool rowpairs)
{
    return (rowpairs && (np & 1)) ? (int64_t)((np * np + 1) / 2) * np
                                  : (int64_t)np * np * ((np + 1) / 2);
}
kitc_status weights_plan_var(const TreeDev &t, int win, const std::vector<int32_t> &hdeg,
                             cudaStream_t s, WeightsDev &wd);
kitc_status weights_launch_var(const TreeDev &t, const double *w_user, WeightsDev &wd,
                               cudaStream_t s);
int64_t proxy_offsets_var(const std::vector<int32_t> &hdeg, int win, bool mixed, bool pairs,
                          bool rowpairs, std::vector<int64_t> &roff);
kitc_status pack_proxies_var(const TreeDev &t, WeightsDev &wd, const int32_t *d_deg,
                             const int64_t *d_roff, bool mixed, bool pairs, cudaStream_t s);
// Weights pass and evaluator records of an asynchronously built tree, planned
// on the device (no read-back, no allocation in the launch).  Reserve once;
// each launch recomputes everything from the tree's state block.  Bits of
// *err: ASYNC_RECORD_OVERFLOW (cannot happen for a valid tree; the records
// then stay in bounds but are not the weights).
int64_t weights_async_itemcap(int cap, int levels, int64_t n, int mode);
kitc_status weights_async_reserve(const TreeAsync &a, int win, int degree, int mode, bool split,
                                  bool mixed, bool pairs, bool rowpairs, bool leaf, cudaStream_t s,
                                  WeightsDev &wd);
kitc_status weights_async_launch(const TreeAsync &a, const double *w_user, WeightsDev &wd,
                                 bool mixed, bool pairs, int *err, cudaStream_t s);
// Paired FP32 records of a tree's leaves for the FP32x2 evaluator
// (pack_pairs_plan once per tree, then pack_pairs_launch): hi/lo coordinates
// (80 bytes a pair), or with leaf offsets (KITC_MIXED_LEAF) the offsets from
// the leaf's box centre (48 bytes); pbegin receives the first pair of every
// leaf (-1 for other clusters), followed by the ranges of the packing launch.
constexpr int LEAF_PAIR_BYTES = 48;
// The leaf-offset arithmetic shared by the record packing and the evaluator:
// c = the box centre as FP32 hi/lo parts, and the FP32 offset of a point p
// given as hi/lo parts, (ph - ch) + (pl - cl) (rounded at each step, no
// contraction), within about 2^-23 of |p - c|.
__host__ __device__ inline void leaf_centre(const dvec4 &lo, const dvec4 &hi, float *ch, float *cl)
{
    const double c[3] = {0.5 * (lo.x + hi.x), 0.5 * (lo.y + hi.y), 0.5 * (lo.z + hi.z)};
    for (int l = 0; l < 3; ++l) {
        ch[l] = (float)c[l];
        cl[l] = (float)(c[l] - (double)ch[l]);
    }
}
__device__ __forceinline__ float leaf_offset(float ph, float pl, float ch, float cl)
{
    return __fadd_rn(__fsub_rn(ph, ch), __fsub_rn(pl, cl));
}
constexpr size_t pair_record_bytes(bool leaf) { return leaf ? LEAF_PAIR_BYTES : 80; }
kitc_status pack_pairs_plan(const TreeDev *t, int64_t n, bool leaf, cudaStream_t s, DevBuf &out,
                            DevBuf &pbegin, int *nranges);
kitc_status pack_pairs_launch(const TreeDev *t, const double *w_user, int64_t n, int nranges,
                              bool leaf, cudaStream_t s, DevBuf &out, DevBuf &pbegin);
// Direct-sum source records in the caller's order, written to caller-provided
// device memory of direct_record_bytes() bytes (no allocation, no host copy);
// pairs selects the paired FP32x2 format.
size_t direct_record_bytes(int64_t n, int win, bool mixed, bool pairs);
kitc_status pack_direct_records(const double *xyz, const double *w, int64_t n, int win, bool mixed,
                                bool pairs, void *out, cudaStream_t s);
// Loads every kernel pack_direct_records may launch on the current device
// (lazy module loading defers that to the first launch otherwise) and raises
// *lmem to the largest per-thread local memory among them.
kitc_status pack_direct_preload(size_t *lmem);
// The same for every evaluator instantiation evaluate_launch may run, which
// also get their shared-memory attribute set.
kitc_status evaluate_preload(size_t *lmem);

// Argument checks shared by the entry points.
bool valid_count(int64_t n);              // 1 <= n <= INT32_MAX - 1024
// A pointer the kernels may read or write: device, managed or registered host memory.
bool device_accessible(const void *ptr);
// kitc_params fields used by the direct sums (kernel, eps, precision, batch).
bool valid_direct_params(const kitc_params *p);

// ---------------------------------------------------------------------------
// Interaction lists of target batches (Algorithm 2 traversal).
// ---------------------------------------------------------------------------
struct ListsDev {
    int64_t nb = 0, nt = 0;
    int batch = 0;
    bool forest = false;
    int64_t nfar = 0, nnear = 0;
    DevBuf bctr;                 // dvec4 [nb]: batch box centre
    DevBuf bdesc;                // forests: int32 [3][nb] first slot, size, source root
    DevBuf far_off, near_off;    // int64 [nb+1]
    DevBuf far_id, near_id;      // int32 [entries]
    DevBuf far_mask, near_mask;  // uint64 [entries]
    DevBuf counts;               // int64 scratch [nb*2] + totals
    DevBuf totals;               // int64 [8]
    int64_t near_pairs = 0, far_points = 0, near_exec = 0, far_exec = 0;
    bool async = false;                  // capacity-sized (lists_async_reserve)
    int64_t cap_far = 0, cap_near = 0;   // its room for far and near entries
    void release(cudaStream_t s);
    size_t bytes() const;
};

kitc_status lists_build(const TreeDev &src, const TreeDev &tgt, int batch, double theta,
                        int degree, const int32_t *cdeg, int mac, cudaStream_t s, ListsDev &L);
// Lists of two asynchronously built trees in buffers sized once for cap_far
// and cap_near entries (forests: batches from the target systems' sizes).
// The launch reads nothing back; lists that exceed their room are not written,
// every batch's lists are emptied and ASYNC_LIST_OVERFLOW is set in *err.
// Totals (as in lists_build) stay in L.totals on the device.
kitc_status lists_async_reserve(const TreeAsync &src, const TreeAsync &tgt, int batch, int64_t cap_far,
                                int64_t cap_near, cudaStream_t s, ListsDev &L);
kitc_status lists_async_launch(const TreeAsync &src, const TreeAsync &tgt, double theta, int degree,
                               int mac, int *err, cudaStream_t s, ListsDev &L);
// Far-field point counts of existing lists under the degree map cdeg;
// KITC_ERR_INVALID_ARG if an accepted cluster has degree 0.
kitc_status lists_recount(const int32_t *cdeg, cudaStream_t s, ListsDev &L);

// ---------------------------------------------------------------------------
// Fused near/far evaluator.
// ---------------------------------------------------------------------------
struct EvalArgs {
    // targets: slot -> coordinates (x[slot*stride], y[..], z[..]) and caller index
    const double *tx, *ty, *tz;
    int64_t tstride;
    const int32_t *tperm;        // NULL: slot == caller index
    int64_t nt;
    int batch;                   // targets per batch
    int64_t nb;
    const dvec4 *bctr;           // batch centres (mixed far field frame); may be NULL if no far
    const int32_t *bstart, *bcount;  // forests: first slot and size of each batch (else NULL)
    // lists (NULL near_off = direct mode: one near range [0, direct_ns) per batch)
    const int64_t *far_off, *near_off;
    const int32_t *far_id, *near_id;
    const uint64_t *far_mask, *near_mask;
    int64_t direct_ns;
    // sources / clusters
    const void *src;             // source records (tree order, or caller order in direct mode)
    const void *proxy;           // proxy records [cluster][P]
    const dvec4 *clo, *chi;    // cluster boxes (far field grid points)
    const int32_t *cbegin, *cend;
    const int32_t *pbegin;       // paired records: first pair of each leaf
    int leaf;                    // tree's paired records hold leaf offsets (KITC_MIXED_LEAF)
    int degree;
    double cheb[KITC_MAX_DEGREE + 1];  // cos(k pi / n)
    // degree per cluster (NULL: degree everywhere); then cluster c's grid
    // records start roff[c] bytes into proxy and chebt[n][k] = cos(k pi / n)
    const int32_t *cdeg;
    const int64_t *roff;
    const double *chebt;
    double eps;
    // set by evaluate_launch from eps: eps^2, eps^4 in FP64 and the FP32 kernel
    // coefficients eps^2, eps^4, 1.5 eps^2, 3.75 eps^2, 3.75 eps^4, -0.75 eps^2
    double e2d, e4d;
    float ecf[6];
    double *out;                 // caller order, n x wout
    int *queue;                  // work counter, zero at launch
    int *err;                    // error flag (nonzero on a timed-out wait)
    unsigned long long wait_ns;  // bound of every barrier wait
};

kitc_status evaluate_launch(int kernel, bool mixed, const EvalArgs &a, cudaStream_t s);
// Evaluator arguments common to every call: degree, Chebyshev table, eps, the
// work counter (flags[0]), the error flag (flags[1]) and the wait bound.
void fill_eval_common(EvalArgs &a, const kitc_params &p, int *flags);
// kitc_params checks of the treecode entry points; the target batch in use.
bool valid_params(const kitc_params *p);
int batch_of(const kitc_params &p);
// Split-precision weight products in the mixed form (a build-time choice).
bool weights_split_enabled();
// Reads the evaluator's error flag (synchronizes s): KITC_ERR_TIMEOUT if set.
kitc_status read_error_flag(int *d_err, cudaStream_t s);

// ---------------------------------------------------------------------------
// Per-cluster degree selection: features and measured far-field errors.
// ---------------------------------------------------------------------------
struct LearnArgs {
    int nclus = 0, win = 3, degree = 1;
    double eps = 0.0;
    const int32_t *cbegin = nullptr, *cend = nullptr, *perm = nullptr, *level = nullptr;
    const int32_t *cdeg = nullptr;           // degree map (NULL: degree everywhere)
    const int32_t *first_child = nullptr, *n_child = nullptr;
    const dvec4 *ctr = nullptr, *clo = nullptr, *chi = nullptr;
    const double *sxs = nullptr;             // sources, SoA [3][ns] in tree order
    int64_t ns = 0;
    const double *txs = nullptr;             // targets, SoA [3][nt] in target-tree order
    int64_t nt = 0, nb = 0;
    int batch = 0;
    const int32_t *bdesc = nullptr;          // forests: first slot, size, root per batch
    const int64_t *far_off = nullptr;
    const int32_t *far_id = nullptr;
    const uint64_t *far_mask = nullptr;
    const double *fhat = nullptr;            // FP64 modified weights
    const int64_t *foff = nullptr;           // with a degree map: offset of each cluster's weights
    const double *chebt = nullptr;           // [17][17] cos(k pi / n)
    int *err = nullptr;
};

kitc_status learn_features(const LearnArgs &a, const std::vector<int32_t> &level_start,
                           const double *w, float *feat, DevBuf &scratch, cudaStream_t s);
kitc_status learn_far_errors(int kernel, const LearnArgs &a, const double *w, int S,
                             unsigned long long seed, double *err2, int *nsamp, DevBuf &scratch,
                             cudaStream_t s);
const int64_t *weights_foff(const TreeDev &t, const WeightsDev &wd);

// Counts one kernel launch of this library (see kitc_launch_count).
void kitc_count_launch();

kitc_status watchdog_launch(unsigned long long limit_ns, int *err, cudaStream_t s);

extern int g_wait_limit_ms;
