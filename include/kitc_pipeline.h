/* The whole treecode as one queue of device work: a handle whose calls build
 * the source tree (Sec. 6), the modified weights (Eq. modified_weights,
 * Algorithm 1 and the upward pass), the target tree, the interaction lists
 * (Algorithm 2's traversal) and evaluate u (Eq. Velocity_1 / Eq. MRS_2)
 * without any host read-back, host synchronization or device allocation, so
 * that the sequence can be captured in a CUDA graph and replayed on new
 * coordinates and weights.
 *
 * The paper has no counterpart: it describes one serial treecode call.  The
 * eager entry points of kitc.h size every buffer from counts read back from
 * the device (clusters per level, work items, list lengths).  Here the sizes
 * are fixed when the handle is created, from one eager build on example
 * inputs times a slack factor; each run recomputes everything on the device
 * and checks it against that room.  A run that does not fit still stays in
 * bounds: the tree stops splitting, or the lists are left empty, and
 * kitc_pipeline_status reports KITC_ERR_TOO_LARGE.  Results of a run that
 * fits are bit-identical to kitc_build_tree / kitc_build_forest +
 * kitc_modified_weights + kitc_evaluate / kitc_evaluate_forest on the same
 * inputs and parameters.
 *
 * All pointers given to a run are device pointers (n x 3 row-major
 * coordinates, n x w_in weights, n_tgt x w_out output in the caller's target
 * order); the library copies what it needs, and they may be reused once the
 * stream has passed the run.  Handles are not thread-safe, and belong to the
 * device that was current at creation: a run, replay or status call made with
 * another device current returns KITC_ERR_STATE. */
#pragma once
#include "kitc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct kitc_pipeline_s *kitc_pipeline; /* opaque; owned by the library */

/* Creates a pipeline for num_systems independent systems (a forest when > 1,
 * as kitc_build_forest / kitc_evaluate_forest): system k has src_counts[k]
 * sources and tgt_counts[k] targets (host arrays, every count >= 1).
 * src_xyz and tgt_xyz (device) are example inputs of those sizes: the source
 * and target trees and the lists are built once eagerly on them, and the
 * handle reserves slack (>= 1) times their cluster and list-entry counts plus
 * a margin, and the depth of each tree plus two levels.  tgt_xyz = NULL: the
 * targets are the sources (tgt_counts ignored, and NULL is then allowed).
 * Parameters as in kitc_params; the uniform degree only.  Synchronizes
 * `stream`.  KITC_ERR_INVALID_ARG for bad sizes or parameters. */
kitc_status kitc_pipeline_create(const double *src_xyz, const int64_t *src_counts,
                                 const double *tgt_xyz, const int64_t *tgt_counts,
                                 int num_systems, const kitc_params *p, double slack,
                                 void *stream, kitc_pipeline *out);

/* Queues one whole treecode on `stream`: u (out) of the targets tgt_xyz
 * (NULL: the sources) from the sources src_xyz with weights w.  Launches
 * kernels and stream-ordered memsets only: no synchronization, no allocation,
 * no host copy, so the call may be captured in a CUDA graph (run it once
 * outside a capture first, so that every kernel is loaded and configured).
 * The targets of the sources-as-targets form must be passed as NULL here too
 * (the handle was created that way).  Errors that only the device sees are
 * recorded for kitc_pipeline_status.  Returns KITC_ERR_INVALID_ARG for a null
 * pointer, else the status of the launches. */
kitc_status kitc_pipeline_run(kitc_pipeline h, const double *src_xyz, const double *w,
                              const double *tgt_xyz, double *out, void *stream);

/* kitc_pipeline_run through a CUDA graph owned by the handle.  The first call
 * for a set of pointers runs the pipeline on `stream` (its result is that
 * call's output) and captures it, on a stream of the handle, into the graph;
 * later calls with the same pointers launch the graph on `stream` (any
 * stream, the legacy default stream included), reading the values the
 * buffers hold then.  No synchronization, no allocation after the first
 * call. */
kitc_status kitc_pipeline_replay(kitc_pipeline h, const double *src_xyz, const double *w,
                                 const double *tgt_xyz, double *out, void *stream);

/* Waits for `stream` and reports the last run (before any run: KITC_OK and
 * zero counts): KITC_ERR_TOO_LARGE if the
 * trees, the work items or the lists needed more room than the handle holds
 * (create the handle again from inputs like these, or with more slack),
 * KITC_ERR_INVALID_ARG if a traversal stack overflowed (as kitc_evaluate),
 * KITC_ERR_TIMEOUT if an evaluator wait ran out, else KITC_OK.  st (may be
 * NULL) receives the run's counts as kitc_get_stats gives them (no stage
 * times). */
kitc_status kitc_pipeline_status(kitc_pipeline h, kitc_stats *st, void *stream);

/* Launches captured in the handle's graph (0 before the first replay). */
int64_t kitc_pipeline_graph_launches(kitc_pipeline h);

/* Frees the handle.  Waits for the handle's own second stream only: every
 * stream the caller ran or replayed the handle on must be done with it. */
kitc_status kitc_pipeline_free(kitc_pipeline h);

#ifdef __cplusplus
}
#endif
