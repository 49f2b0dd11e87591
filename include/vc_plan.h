/*
 * vc_plan.h - batched MVC as a reusable plan captured as one CUDA graph (libvc).
 *
 * The batch is the same as vc_mvc_batch (vc.h): many independent graphs searched by one persistent
 * launch of the hybrid traversal (Sec. IV-A), worklist entries tagged with their graph.  A plan
 * does the per-batch set-up once -- copies the graphs into plan-owned device memory, checks them,
 * picks the variant, allocates stacks and worklist -- and captures the launch sequence
 *   reset problem records -> reset counters -> worklist init -> greedy bound (Sec. II-B)
 *   -> traversal -> gather the answers
 * as one CUDA graph.  Each vc_plan_launch replays it without a host synchronisation, so it can be
 * queued behind other work or captured into a caller's own graph.  The paper launches one search
 * per graph; the plan is this library's own deployment pattern.
 *
 * Memory: the plan owns its device memory until vc_plan_destroy; the caller's input buffers may
 * be freed once vc_plan_create_mvc_batch returns.  A plan must not be launched again before the
 * previous launch has finished (it reuses one set of buffers).  Errors as in vc.h.
 */
#ifndef VC_PLAN_H
#define VC_PLAN_H

#include <stdint.h>

#include "vc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vc_plan vc_plan;

/* Builds a plan for a packed batch laid out as for vc_mvc_batch (graph_vtx_offsets and
 * graph_edge_offsets are host arrays; packed arrays host or device per on_device).  Checks the
 * graphs (VC_EINVAL if malformed) and synchronises once. */
int vc_plan_create_mvc_batch(int32_t num_graphs, const int32_t *graph_vtx_offsets, const int32_t *graph_edge_offsets,
                             const int32_t *packed_offsets, const int32_t *packed_neighbors, int32_t on_device,
                             const vc_config *cfg, vc_plan **plan);

/* Enqueues one solve of the whole batch on `stream` (a single graph launch; no synchronisation). */
int vc_plan_launch(vc_plan *plan, void *stream);

/* Waits for `stream`, then copies the minimum sizes (host, num_graphs entries) and, if covers_out
 * is not NULL, the Σn cover masks (host or device per covers_on_device).  stats may be NULL. */
int vc_plan_results(vc_plan *plan, void *stream, int32_t *sizes_out, int32_t *covers_out, int32_t covers_on_device,
                    vc_stats *stats);

/* Per-graph completion of the last launch: waits for `stream`, then writes to done_ns_out (host,
 * num_graphs entries) when each graph was answered, in nanoseconds of the GPU's global timer after
 * the greedy pass's start (Sec. II-B); the time of the step's first kernel is the same up to a few
 * microseconds.  A graph is answered when the greedy bound settles it or when the last piece of its
 * search (root, worklist entry or local stack) is released (Sec. IV-C).  Every graph of a batched
 * launch is returned with the whole launch: these times show how long each graph's own search
 * lasted within it.  VC_EINVAL for a NULL argument. */
int vc_plan_completion_ns(vc_plan *plan, void *stream, int64_t *done_ns_out);

int vc_plan_destroy(vc_plan *plan);

#ifdef __cplusplus
}
#endif

#endif /* VC_PLAN_H */
