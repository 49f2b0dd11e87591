/*
 * vc_server.h - serving exact vertex cover with continuous batching (libvc).
 *
 * A server keeps a persistent traversal launch (the hybrid stack + worklist search of Sec. IV-A,
 * rules of Sec. II-B / IV-D, termination of Sec. IV-C) running per size class while requests
 * arrive.  Requests admitted while others are being searched join the running launch of their
 * class: idle workers claim them, run their greedy bound (Sec. II-B) and search them through the
 * class's worklist, whose entries carry the request's slot, so the work of many requests overlaps
 * on the device.  The paper solves one graph per launch; the serving layer is this library's own.
 *
 * Size classes (cfg->bit_rows = 1): graphs of at most 128 vertices run on one-warp bit-row workers
 * (the node in registers, the adjacency as bit rows in shared memory), larger ones on CSR-walk
 * workers sized for max_n.  The two classes' launches run side by side, the CSR-walk class on three
 * quarters of every SM's thread slots and the bit-row class on the rest, each with its own stacks,
 * worklist and arena.  By default (bit_rows 0 or -1) every request runs on CSR-walk workers sized
 * for max_n: one class.  cfg->worker_threads, width, worklist_capacity and donate_threshold apply
 * to the CSR-walk class.
 *
 * Admission: every request reserves a slot and a range of its class's device graph arena (its
 * CSR, its cover mask and one entry for its reduced root node).  Stacks and worklist are reserved
 * per class at creation for the class's largest graph (depth n + 3 entries of the degree-array
 * size per worker, n = 128 or max_n), so any accepted request fits them.  A request whose bytes do not fit the arena right now waits in a
 * host queue and is admitted when earlier requests of its class finish; it is never refused for
 * lack of room unless it alone is larger than the whole arena.
 *
 * Graphs are copied at submission (host pointers only; same CSR rules as vc.h, checked on the host);
 * the caller's buffers can be reused as soon as vc_server_submit returns.  All functions are safe
 * to call from several host threads.  Errors as in vc.h.
 */
#ifndef VC_SERVER_H
#define VC_SERVER_H

#include <stddef.h>
#include <stdint.h>

#include "vc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct vc_server vc_server;

/* State of one request.  Times are steady-clock nanoseconds (same clock for all requests). */
typedef struct {
    int32_t done;       /* 1 once the answer is known */
    int32_t answer;     /* MVC: minimum cover size; PVC: 1 if a cover of size <= k exists, else 0 */
    int32_t status;     /* VC_OK or the error that ended the request */
    int32_t greedy;     /* greedy upper bound computed for the request (-1 if none) */
    int64_t submit_ns;  /* vc_server_submit was called */
    int64_t admit_ns;   /* the request was uploaded and published to the device */
    int64_t done_ns;    /* the host saw the device's completion record */
} vc_request_info;

typedef struct {
    int64_t completed, pending, in_flight;  /* requests */
    int64_t launches;                       /* persistent launches started so far */
    int64_t epochs;                         /* arena / slot epochs completed */
    int64_t nodes_visited;                  /* tree nodes over all finished launches */
    int32_t workers, worker_threads, slots_per_epoch;
    int64_t arena_bytes;
    int64_t records;                        /* requests whose records the server still holds (not yet
                                               released with vc_server_release) */
    int32_t classes;                        /* size classes, each its own persistent launch (1 or 2) */
    int32_t small_max_n;                    /* largest graph of the bit-row class (0: no such class) */
    int32_t small_workers;                  /* one-warp workers of the bit-row class (also in workers) */
    int32_t reserved;
} vc_server_counters;

/* Creates a server on the current device.  device_bytes_budget (0 = 8 GiB) bounds the device
 * memory it holds: an eighth goes to the bit-row class when there are two, the rest to the other;
 * within a class, half goes to the per-worker stacks (which sets the worker count, up to the SM
 * slots the class has), a quarter to the graph arena (and, in the bit-row class, the bit rows).
 * max_n is the largest graph it accepts.  cfg (may be NULL) picks the CSR-walk class's worker size,
 * width, worklist capacity and donation threshold as in vc.h; node_in_global = 1 is VC_EINVAL.
 * With two classes, cfg->num_workers (if given) sets the CSR-walk class's worker
 * count instead of its three quarters of the SMs' thread slots; the bit-row class gets the slots
 * that remain (VC_EINVAL if none do). */
int vc_server_create(const vc_config *cfg, size_t device_bytes_budget, int32_t max_n, vc_server **server);

/* Queues a request: kind 0 = MVC, 1 = PVC with parameter k.  Returns at once with its id.  The
 * graph must be on the host (on_device = 0) with n <= max_n; it is copied before the call returns,
 * so the caller may free it then.  The CSR is checked on the host against the rules of vc.h (the
 * running launch never sees a malformed graph), and a malformed one is rejected here with
 * VC_EINVAL.  PVC with k < 0 is answered at once (no). */
int vc_server_submit(vc_server *server, const vc_graph *g, int32_t kind, int32_t k, uint64_t *request_id);

/* Reads a request's state (see vc_request_info). */
int vc_server_poll(vc_server *server, uint64_t request_id, vc_request_info *info);

/* Forgets a finished request: its record is freed and its id becomes unknown (a later poll or
 * release of it returns VC_EINVAL).  A request that has not finished cannot be released
 * (VC_EINVAL).  A long-running server should release every request once its answer has been read;
 * records that are never released are freed by vc_server_destroy. */
int vc_server_release(vc_server *server, uint64_t request_id);

/* Waits until every submitted request has finished (timeout_ms <= 0: no limit; VC_ETIMEOUT if the
 * limit passes first). */
int vc_server_drain(vc_server *server, int64_t timeout_ms);

/* Server-wide counters. */
int vc_server_stats(vc_server *server, vc_server_counters *out);

/* Finishes the requests still queued or in flight, stops the launch and frees everything. */
int vc_server_destroy(vc_server *server);

#ifdef __cplusplus
}
#endif

#endif /* VC_SERVER_H */
