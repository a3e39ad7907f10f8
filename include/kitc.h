/*
 * kitc.h -- C ABI of libkitc, a GB300 (sm_103a) implementation of the
 * kernel-independent treecode (KITC) of Wang, Krasny & Tlupova, "A
 * kernel-independent treecode based on barycentric Lagrange interpolation"
 * (arXiv 1902.02250).
 *
 * The library evaluates the sum of Eq. N-body,
 *     u(x_i) = sum_j k(x_i, y_j) f_j,
 * for the regularized Stokes kernels of Sec. 7, either directly or with the
 * treecode of Algorithm 2: a tree of clusters (Sec. 6), modified weights at
 * the (n+1)^3 Chebyshev points of each cluster (Eq. modified_weights,
 * Algorithm 1), and a MAC-driven traversal (Eq. MAC) that sums far clusters
 * through Eq. pc_approximation_3D and near leaves through Eq.
 * pc_interaction_3D.
 *
 * Conventions shared by every call:
 *   - Arrays are row-major.  Coordinates are n x 3 doubles; weights are
 *     n x w_in doubles; outputs are n x w_out doubles (w_in, w_out per
 *     kernel below).  Inputs and outputs are in the caller's order.
 *   - A pointer documented as "device" must point to memory of the current
 *     CUDA device; "host" pointers are ordinary process memory.  The caller
 *     owns every buffer it passes and keeps it alive until the work queued on
 *     `stream` is complete.  The library owns what a kitc_tree holds.
 *   - `stream` is a cudaStream_t (NULL = the legacy default stream).  Work is
 *     queued on it in order; only the calls that say so synchronize it.
 *   - Every call returns a kitc_status; nothing is thrown across the ABI.
 *     Argument errors are reported before any GPU work is queued.  After
 *     KITC_ERR_CUDA the handle must only be freed.
 *   - There is no CPU fallback: without a usable CUDA device the calls fail
 *     with KITC_ERR_CUDA.
 */
#ifndef KITC_H
#define KITC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    KITC_OK = 0,
    KITC_ERR_INVALID_ARG = 1, /* a null pointer, a size or parameter out of range */
    KITC_ERR_CUDA = 2,        /* a CUDA runtime call failed                       */
    KITC_ERR_OOM = 3,         /* device memory could not be allocated             */
    KITC_ERR_TIMEOUT = 4,     /* a bounded device-side wait ran out               */
    KITC_ERR_STATE = 5,       /* call out of order (e.g. evaluate before weights) */
    KITC_ERR_TOO_LARGE = 6    /* size beyond the fixed scratch of kitc_direct_noalloc,
                                 or beyond the room of a kitc_pipeline handle      */
} kitc_status;

/* Kernels of Sec. 7.  d = x - y, r = |d|, H1, H2, Q, D1, D2 of Eq. MRS_kernels. */
typedef enum {
    KITC_STOKESLET = 0,        /* Eq. Velocity_1; w_in 3 (force f), w_out 3 (u)          */
    KITC_ROTLET = 1,           /* torque terms of Eq. MRS_2; w_in 3 (torque n), w_out 6 (u, w) */
    KITC_STOKESLET_ROTLET = 2, /* Eq. MRS_2; w_in 6 (f then n), w_out 6 (u then w)       */
    KITC_TEST_POLY = 99        /* test kernel prod_l (1 + x_l y_l / 2)^3 times f; 3 -> 3  */
} kitc_kernel;

/* Arithmetic of the evaluation.  KITC_FP64: everything in FP64.
 * KITC_MIXED: kernel evaluations in FP32 (coordinate differences formed
 * from hi/lo FP32 pairs, far-field points taken relative to the target
 * batch's centre), FP32 partial sums over short runs, FP64 accumulation
 * of the per-leaf and per-cluster sums.  The tree, the MAC decisions, the
 * differences y - s_k of the barycentric basis and the modified-weight sums
 * are FP64 in both; the mixed form takes the basis's quotients and the
 * modified-weight products in split precision (FP32 hi/lo pairs, about
 * 2^-45 and 2^-47 relative error).
 * KITC_MIXED_LEAF: KITC_MIXED, except that the tree's near field of the
 * Stokeslet and the rotlet forms x - y = (x - c) - (y - c) from FP32 offsets
 * to the leaf's box centre c, each within about 2^-23 of its magnitude and
 * formed by the same arithmetic for targets and sources (a target on a
 * source gives exactly 0), one FP32 subtraction per coordinate instead of
 * three.  A pair's difference then carries an absolute error of about 2^-24
 * times the leaf's extent, which matters only for pairs much closer than
 * that: on a uniform cube (Stokeslet, N = 10^6, N0 = 4000) it changes the
 * output by about 1e-7 relative L2; on clustered inputs (dipole pairs,
 * points on a surface, the rotlet's 1/r^2 near field) by up to ~1e-6.
 * Direct sums, the other kernels and eps = 0 (where nothing bounds the
 * kernel of a close pair) are the same as KITC_MIXED. */
typedef enum { KITC_FP64 = 0, KITC_MIXED = 1, KITC_MIXED_LEAF = 2 } kitc_precision;

/* Traversal.  KITC_MAC_PARTICLE takes Algorithm 2's decision for every
 * target: cluster C is used through its grid points iff r_C <= theta * R
 * with R = |x - y_C| (Eq. MAC), and the target then skips C's subtree.
 * KITC_MAC_BATCH takes one decision per target batch: C is accepted iff
 * r_C <= theta * dist(box_B, y_C), box_B the smallest box enclosing the
 * batch; every accepted C then also passes Eq. MAC for each target.
 * KITC_MAC_ALL also takes one decision per batch: C is accepted iff every
 * target of the batch accepts it by Eq. MAC (weaker than the box rule, so
 * fewer interactions; each accepted interaction is one Algorithm 2 takes). */
typedef enum { KITC_MAC_PARTICLE = 0, KITC_MAC_BATCH = 1, KITC_MAC_ALL = 2 } kitc_mac;

/* How the modified weights of Eq. modified_weights are formed.  Both give the
 * same values up to rounding.  KITC_WEIGHTS_ALGORITHM1 runs Algorithm 1 on
 * every cluster from its particles.  KITC_WEIGHTS_UPWARD runs Algorithm 1 on
 * the leaves only and forms each parent from its children's weights through
 * the parent's barycentric basis at the children's Chebyshev points (exact,
 * Sec. 2: the parent's Lagrange polynomials have degree n); it falls back to
 * Algorithm 1 when (n+1)^3 w_in is too large for its shared-memory buffers. */
typedef enum { KITC_WEIGHTS_UPWARD = 0, KITC_WEIGHTS_ALGORITHM1 = 1 } kitc_weights_mode;

typedef struct {
    double theta;      /* MAC parameter of Eq. MAC, >= 0 (0: direct sum through the tree) */
    int degree;        /* interpolation degree n, 1..16; (n+1)^3 grid points per cluster  */
    int leaf_size;     /* N0: a cluster with <= N0 particles is a leaf (Sec. 6), >= 1     */
    double eps;        /* MRS regularization epsilon (Sec. 7), >= 0; with eps = 0 a pair
                          at r = 0 contributes nothing (Sec. 1)                          */
    int kernel;        /* kitc_kernel                                                     */
    int precision;     /* kitc_precision                                                  */
    int mac;           /* kitc_mac                                                        */
    int target_batch;  /* targets per batch, 1..64 (0 = 64).  Targets are ordered by the
                          Sec. 6 tree built on them with leaf size target_batch; batch b
                          is the slots [b*B, (b+1)*B) of that order.  The evaluator holds
                          two targets per lane; the mixed Stokeslet with B <= 32 holds
                          one, other forms leave the second slot idle              */
    int weights;       /* kitc_weights_mode                                               */
} kitc_params;

/* Per-cluster degree selector (kitc_cluster_features, kitc_mlp_*). */
#define KITC_NFEAT 12        /* features per cluster                          */
#define KITC_MLP_HIDDEN 64   /* units of each of the two hidden layers        */
#define KITC_MLP_CLASSES 6   /* outputs: degree classes                       */
/* parameters: mu[12] sd[12] W1[64][12] b1[64] W2[64][64] b2[64] W3[6][64] b3[6] */
#define KITC_MLP_NPARAM (2 * 12 + 64 * 12 + 64 + 64 * 64 + 64 + 6 * 64 + 6)

typedef struct kitc_tree_s *kitc_tree; /* opaque; owned by the library */

typedef struct {
    int64_t n_sources, n_clusters, n_leaves;
    int32_t depth, degree;
    int64_t n_targets, n_batches;          /* of the last kitc_evaluate or plan        */
    int64_t far_entries, near_entries;     /* interaction-list entries (batch, cluster) */
    int64_t near_pairs, far_points;        /* (target, source) and (target, grid point)
                                              kernel evaluations that count toward u   */
    int64_t device_bytes;                  /* device memory held by the handle         */
    float ms_tree, ms_weights, ms_lists, ms_evaluate; /* device time of the last calls */
    int64_t near_exec, far_exec;           /* evaluations the GPU performs: every entry
                                              is computed for all targets of its batch;
                                              near_pairs / near_exec is the lane use   */
} kitc_stats;

/* Sec. 6 tree build.  src_xyz: device, n_src x 3.  Copies the sources into
 * tree order inside the handle, so src_xyz may be reused once the stream has
 * passed this call.  The levels run on the device, each reading the cluster
 * range the previous one wrote; the host queues them in rounds and
 * synchronizes `stream` once per round to read the cluster count back.  One
 * round covers the depth of a uniform tree with leaves of N0 plus four
 * levels, so the usual trees take one synchronization; deeper trees (strongly
 * clustered points, coincident points) take one per further round, and a tree
 * with more clusters than the room first reserved (16 per N0 + 1 particles)
 * is built again with twice the room.  On success *out holds a new handle;
 * free it with kitc_free_tree. */
kitc_status kitc_build_tree(const double *src_xyz, int64_t n_src, const kitc_params *p,
                            void *stream, kitc_tree *out);

/* Many independent systems in one handle: a forest with one Sec. 6 tree per
 * system, built in the same level-synchronous passes.  src_xyz: device,
 * n_src x 3, system k owning the counts[k] rows after those of systems < k;
 * counts: host, num_systems entries >= 1 summing to n_src.  The handle is used
 * with kitc_modified_weights (one pass over every cluster of every system) and
 * kitc_evaluate_forest; kitc_evaluate is refused (KITC_ERR_STATE). */
kitc_status kitc_build_forest(const double *src_xyz, const int64_t *counts, int num_systems,
                              const kitc_params *p, void *stream, kitc_tree *out);

/* Eq. modified_weights (Algorithm 1) for every cluster of the tree, in
 * FP64.  w: device, n_src x w_in, in the order of src_xyz.  Replaces any
 * weights set before.  Stream-ordered and without host synchronization: the
 * work items and the evaluator's record ranges are planned on the device.
 * With a degree map (kitc_set_degrees), the first call after it plans the
 * degree groups on the host and synchronizes `stream` once. */
kitc_status kitc_modified_weights(kitc_tree t, const double *w, void *stream);

/* Algorithm 2: u at n_tgt targets.  tgt_xyz: device, n_tgt x 3; out: device,
 * n_tgt x w_out, overwritten.  Builds the target order, the interaction
 * lists and runs the fused near/far evaluator.  Synchronizes `stream` for the
 * target tree (as kitc_build_tree), once to size the lists and once to read
 * the evaluator's error flag.
 * KITC_ERR_STATE if kitc_modified_weights was not called. */
kitc_status kitc_evaluate(kitc_tree t, const double *tgt_xyz, int64_t n_tgt, double *out,
                          void *stream);

/* Algorithm 2 for every system of a forest: the targets of system k (rows of
 * tgt_xyz after those of systems < k, tgt_counts[k] >= 1 of them, host array of
 * num_systems entries) interact with system k's sources only.  Target batches
 * never span two systems; all batches of all systems go through one persistent
 * evaluator launch.  Synchronizes like kitc_evaluate. */
kitc_status kitc_evaluate_forest(kitc_tree t, const double *tgt_xyz, const int64_t *tgt_counts,
                                 double *out, void *stream);

/* Applies the treecode again with new weights, for the same sources and the
 * targets of the last kitc_evaluate / kitc_evaluate_forest (an iterative
 * solver's repeated products with one geometry): modified weights of w, then
 * the evaluator over the stored target order and interaction lists.  w: device,
 * n_src x w_in; out: device, n_tgt x w_out.  On a non-default stream the launch
 * sequence is captured into a CUDA graph at the first call for a given (w, out,
 * stream) and replayed afterwards (the first call also runs it once without
 * capture).  Synchronizes `stream` once to read the evaluator's error flag.
 * KITC_ERR_STATE if no evaluation has been done on the handle. */
kitc_status kitc_apply(kitc_tree t, const double *w, double *out, void *stream);

/* Gives every cluster c its own interpolation degree n_c = degrees[c]
 * (n_clusters int32 values in 0..16, host or device memory; NULL returns to
 * the uniform degree of kitc_params).  The paper uses one n for all clusters
 * (Sec. 3, Eq. pc_approximation_3D); the MAC of Eq. MAC does not involve n, so
 * the same interaction lists serve any degree map, and cluster c's far field
 * takes its own (n_c+1)^3 Chebyshev grid with the modified weights of
 * Eq. modified_weights at that degree (Algorithm 1 per cluster; the upward
 * pass is not used).  n_c = 0 means "no modified weights": a later
 * kitc_evaluate returns KITC_ERR_INVALID_ARG if any target accepts such a
 * cluster by the MAC.  Discards the weights, the lists and a captured graph
 * of the handle (call kitc_modified_weights and kitc_evaluate again).
 * kitc_weights_download then returns, cluster by cluster in cluster order,
 * (n_c+1)^3 x w_in values for every cluster with n_c > 0.  Synchronizes
 * `stream`.  KITC_ERR_INVALID_ARG for a degree outside 0..16. */
kitc_status kitc_set_degrees(kitc_tree t, const int32_t *degrees, void *stream);

/* Builds the target tree and the interaction lists of Algorithm 2 for the
 * targets tgt_xyz (device, n_tgt x 3) without evaluating anything: the MAC of
 * Eq. MAC does not involve the degree, so the lists exist before the degrees
 * are chosen.  Feeds kitc_cluster_features / kitc_cluster_far_errors.
 * KITC_ERR_STATE on a forest.  Synchronizes `stream`. */
kitc_status kitc_plan_targets(kitc_tree t, const double *tgt_xyz, int64_t n_tgt, void *stream);

/* kitc_plan_targets for a forest: tgt_counts[k] (host) rows of tgt_xyz are
 * the targets of system k, ordered and batched per system as in
 * kitc_evaluate_forest.  kitc_evaluate_planned then evaluates them. */
kitc_status kitc_plan_targets_forest(kitc_tree t, const double *tgt_xyz, const int64_t *tgt_counts,
                                     void *stream);

/* Algorithm 2 at the targets of the last kitc_plan_targets (or evaluation),
 * reusing its target tree and lists (the target coordinates were copied at
 * planning): the evaluation of kitc_evaluate without the list build.  Under a
 * degree map set after planning, the far-field counts are recomputed and
 * KITC_ERR_INVALID_ARG is returned if an accepted cluster has degree 0.
 * out: device, n_tgt x w_out in the planned targets' order.  KITC_ERR_STATE
 * without lists or weights. */
kitc_status kitc_evaluate_planned(kitc_tree t, double *out, void *stream);

/* Features of every source cluster c for the degree selector, written as
 * FP32 row c of features (device, n_clusters x KITC_NFEAT):
 *   0 log(1 + N_c)            1 log r_c (cluster radius, Sec. 6)
 *   2..4 min, mean, max of r_c / |x - y_c| over the targets x that accept c
 *        in the lists of the last kitc_plan_targets / kitc_evaluate (0 if none)
 *   5 min(eps / r_c, 10)      6 log |sum_j f_j|   7 log sum_j |f_j|
 *   8 log max_j |f_j|         (sums over c's sources, w: device n_src x w_in)
 *   9, 10 middle / longest and shortest / longest side of c's box
 *   11 level of c in the tree.
 * The paper has no degree selector; the features describe the quantities its
 * error analysis involves (Sec. 3 and the MAC of Algorithm 2).
 * KITC_ERR_STATE without lists. */
kitc_status kitc_cluster_features(kitc_tree t, const double *w, float *features, void *stream);

/* Measured far-field error of every cluster at its current modified weights
 * (uniform degree or the map of kitc_set_degrees): of the targets that accept
 * cluster c in the current lists, a sample of about max_samples (each taken
 * with probability min(1, max_samples / accepting targets) by a counter-based
 * hash of (seed, c, target slot)) is evaluated both with the cluster's far field
 * (Eq. pc_approximation_3D, FP64) and with the direct sum over c's sources
 * (Eq. pc_interaction_3D, FP64, w: device n_src x w_in).  err2[c] (device,
 * double) = sum over the samples of |difference|^2 (velocity units, 1/(8 pi)
 * included), n_samples[c] (device, int32) = their number.  KITC_ERR_STATE
 * without lists or weights.  Synchronizes `stream`. */
kitc_status kitc_cluster_far_errors(kitc_tree t, const double *w, int max_samples, uint64_t seed,
                                    double *err2, int32_t *n_samples, void *stream);

/* The degree selector network (FP32, parameters in the KITC_MLP_NPARAM
 * layout above; all pointers device memory unless stated).  The paper has no
 * counterpart: it fixes one degree n for every cluster.
 *
 * kitc_mlp_forward: logits (m x KITC_MLP_CLASSES, may be NULL) of the rows of
 * features (m x KITC_NFEAT) and, when degrees is not NULL, degrees[i] =
 * class_degree[argmax_o logits[i][o]] (class_degree: HOST array of
 * KITC_MLP_CLASSES degrees in 0..16; the first maximum wins ties); with
 * zero_unused, a row whose features 2, 3 and 4 are all 0 (a cluster no
 * target accepts, see kitc_cluster_features) gets degree 0 instead.
 *
 * kitc_mlp_loss_grad: loss[0] = mean softmax cross-entropy of the rows
 * against labels (int32 in 0..KITC_MLP_CLASSES-1), loss[1] = number of rows
 * whose label is out of range (left out of the sums), grad = gradient of
 * loss[0] (KITC_MLP_NPARAM floats; zero for mu and sd).  work: device scratch
 * of kitc_mlp_workspace_bytes(m) bytes, 16-byte aligned.  Fixed summation
 * order: the same inputs give the same bits.
 *
 * kitc_mlp_adam_step: one bias-corrected Adam update (step counts from 1) of
 * params with first and second moments m1, m2 (KITC_MLP_NPARAM floats each,
 * zero before step 1); mu and sd are not updated. */
size_t kitc_mlp_workspace_bytes(int64_t m);
kitc_status kitc_mlp_forward(const float *params, const float *features, int64_t m, float *logits,
                             const int32_t *class_degree, int zero_unused, int32_t *degrees,
                             void *stream);
kitc_status kitc_mlp_loss_grad(const float *params, const float *features, const int32_t *labels,
                               int64_t m, float *loss, float *grad, void *work, void *stream);
kitc_status kitc_mlp_adam_step(float *params, const float *grad, float *m1, float *m2, int step,
                               float lr, float beta1, float beta2, float eps, void *stream);

/* Eq. N-body by direct summation over all sources (self term included;
 * with eps = 0 a pair at r = 0 is skipped).  All pointers device.  Uses
 * p->kernel, p->eps, p->precision and p->target_batch; the tree
 * parameters are ignored.  Allocates and frees its own scratch. */
kitc_status kitc_direct(const double *tgt_xyz, int64_t n_tgt, const double *src_xyz,
                        const double *w, int64_t n_src, const kitc_params *p, double *out,
                        void *stream);

/* kitc_direct without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that must not allocate device memory --
 * latency-critical loops where an allocation may stall or fail, embeddings
 * whose own allocator owns all of the device's memory, or error handling that
 * runs when memory is already exhausted.  Arguments and results are those of
 * kitc_direct; the caller still passes (device) inputs and outputs.
 * Scratch is one file-scope device array of 8 MiB; n_src is limited to 100000
 * sources (KITC_ERR_TOO_LARGE beyond).
 * Set-up: the first call on a device, with that device current, looks up the
 * array's device address (cudaGetSymbolAddress) and loads every kernel this
 * call can launch.  With lazy module loading (the CUDA default) that loading
 * allocates device memory, and from then on the device holds the array until
 * the process exits; so make one call per device at initialisation, before any
 * stream capture.  Every later call on that device allocates nothing.
 * All calls share the array: each call clears the flags it needs and rewrites
 * the records, and calls that overlap on the GPU (other streams, other
 * threads) race on it.  Synchronizes `stream` (the error flag is read back). */
kitc_status kitc_direct_noalloc(const double *tgt_xyz, int64_t n_tgt, const double *src_xyz,
                                const double *w, int64_t n_src, const kitc_params *p, double *out,
                                void *stream);

/* End to end from host memory: copies the sources, weights and targets to
 * the device, builds the tree, computes the modified weights while building
 * the target tree and lists on a second stream (they need only the source
 * tree), evaluates, and copies u back.  All pointers host; tgt_xyz = NULL
 * means the targets are the sources (n_tgt ignored).  Synchronizes `stream`
 * before returning. */
kitc_status kitc_solve_host(const double *src_xyz, const double *w, int64_t n_src,
                            const double *tgt_xyz, int64_t n_tgt, const kitc_params *p,
                            double *out, void *stream);

/* Statistics of the handle; waits for the handle's timing events. */
kitc_status kitc_get_stats(kitc_tree t, kitc_stats *s);

/* Copies the tree to host arrays (any pointer may be NULL; sizes from
 * kitc_get_stats): perm[n_sources] (perm[slot] = caller index), lo/hi
 * [n_clusters][3], begin/end [n_clusters], first_child, n_child, level,
 * parent [n_clusters].  Clusters are numbered breadth first; the children
 * of a cluster are contiguous and ordered by octant code (bit 0 = upper x,
 * bit 1 = upper y, bit 2 = upper z).  Synchronizes `stream`. */
kitc_status kitc_tree_download(kitc_tree t, int64_t *perm, double *lo, double *hi,
                               int64_t *begin, int64_t *end, int32_t *first_child,
                               int32_t *n_child, int32_t *level, int32_t *parent,
                               void *stream);

/* Copies the FP64 modified weights to a host array
 * fhat[n_clusters][n+1][n+1][n+1][w_in].  Synchronizes `stream`. */
kitc_status kitc_weights_download(kitc_tree t, double *fhat, void *stream);

/* Copies the interaction lists of the last kitc_evaluate to host arrays
 * (any may be NULL): tperm[n_targets] (target order), nfar/nnear
 * [n_batches], far/near [far_entries / near_entries] cluster ids in
 * traversal order, far_mask/near_mask (bit k = the batch's k-th target
 * uses the entry).  Synchronizes `stream`. */
kitc_status kitc_lists_download(kitc_tree t, int64_t *tperm, int64_t *nfar, int64_t *nnear,
                                int32_t *far, uint64_t *far_mask, int32_t *near,
                                uint64_t *near_mask, void *stream);

void kitc_free_tree(kitc_tree t);

const char *kitc_status_string(kitc_status s);

/* Number of w_in / w_out components of a kernel, or -1 if unknown. */
int kitc_kernel_win(int kernel);
int kitc_kernel_wout(int kernel);

/* Device-side wait limit in milliseconds for the evaluator's pipeline
 * barriers (default 2000).  A wait that runs out makes the call return
 * KITC_ERR_TIMEOUT.  Returns the previous value. */
int kitc_set_wait_limit_ms(int ms);

/* Number of kernels this library has launched in this process (all devices). */
int64_t kitc_launch_count(void);

/* Failure-detection self test: launches one CTA whose thread waits, with the
 * same bounded wait the evaluator uses, on a shared-memory barrier that
 * nothing completes.  Returns KITC_ERR_TIMEOUT once limit_ms (1..10000) has
 * passed -- the path a stuck evaluator pipeline takes -- and leaves the CUDA
 * context usable.  Synchronizes `stream`. */
kitc_status kitc_watchdog_selftest(int limit_ms, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* KITC_H */
