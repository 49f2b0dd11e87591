/*
 * vc.h - C ABI of libvc: exact vertex cover on one GB300 (sm_103a) by data-parallel traversal of
 * the branch-and-reduce search tree.
 *
 * Method: Yamout, Barada, Jaljuli, Mouawad, El Hajj, "Parallel Vertex Cover Algorithms on GPUs"
 * (arXiv 2204.10402).
 *   - Problems (Sec. II-A): MVC finds a minimum vertex cover; PVC decides whether a cover of size
 *     <= k exists.
 *   - Search (Sec. II-B): at every tree node the degree-one, degree-two-triangle and high-degree
 *     reduction rules run to a fixpoint, then a stop check, then a solution check, then a branch on
 *     the maximum-degree vertex v into "v into S" and "N(v) into S".  The incumbent starts at the
 *     greedy upper bound.
 *   - Parallel traversal (Sec. IV-A, IV-C): each worker (a CUDA thread block) walks a sub-tree from
 *     a local stack and donates the N(v) child to a device-wide worklist while the worklist holds
 *     fewer entries than a threshold; idle workers take entries from the worklist; the search ends
 *     when the worklist is empty and every worker is idle.
 *   - State (Sec. IV-B): an intermediate graph is a degree array (one entry per original vertex,
 *     -1 once the vertex is in S) plus |S| and the remaining edge count, next to one read-only CSR.
 *
 * Graph input (all entry points): an undirected simple graph in CSR form.  offsets has n+1
 * int32 entries with offsets[0] = 0 and offsets[n] = 2m; neighbors has 2m int32 entries; each
 * undirected edge appears in both endpoint lists; every list is sorted strictly ascending; no
 * self-loops.  A graph that breaks any of these rules is rejected with VC_EINVAL (checked on the
 * GPU before any search).
 *
 * Memory: the caller owns every input and output buffer.  Host pointers are accepted when
 * on_device = 0 and device pointers (for example torch CUDA tensors) when on_device = 1; the
 * cover output follows the same flag, scalar outputs are always host pointers.  The library keeps
 * no pointer to caller memory after a call returns.  Device scratch (the copy of the graph,
 * stacks, worklist, counters) is allocated with cudaMalloc on first use, cached per device, grown
 * when a larger problem arrives, and released by vc_release() or at process exit.
 *
 * Streams: every call enqueues its work on `stream` (a cudaStream_t; NULL = the legacy default
 * stream), waits for that stream, and returns.  Calls from several host threads are serialised by
 * an internal lock.
 *
 * Errors: every function returns VC_OK (0) or a negative code below; on error the outputs are
 * unspecified.  vc_strerror() names a code.
 */
#ifndef VC_H
#define VC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VC_OK 0
#define VC_EINVAL (-1)      /* bad argument or malformed CSR */
#define VC_ENOMEM (-2)      /* device or pinned host allocation failed */
#define VC_ETIMEOUT (-3)    /* a device wait ran past its time limit; the search was abandoned */
#define VC_ESTACK (-4)      /* a local stack would have grown past its provisioned depth */
#define VC_ECUDA (-5)       /* a CUDA runtime call failed */
#define VC_ECANCELLED (-6)  /* the caller's cancel flag was raised */

/* An undirected graph in CSR form (see the input rules above). */
typedef struct {
    int32_t n;                 /* number of vertices, >= 0 */
    const int32_t *offsets;    /* n+1 entries (may be NULL when n = 0) */
    const int32_t *neighbors;  /* offsets[n] entries (may be NULL when there are none) */
    int32_t on_device;         /* 0: host pointers, 1: device pointers */
} vc_graph;

/* Launch configuration.  Zero in any field selects the library's choice for it. */
typedef struct {
    int32_t worker_threads;     /* threads per worker (one worker = one thread block): 32..512, power of 2 */
    int32_t num_workers;        /* persistent workers (thread blocks); 0 = SMs x resident blocks per SM */
    int32_t width;              /* degree-array entry width in bits: 16 or 32 */
    int32_t worklist_capacity;  /* worklist entries */
    float donate_threshold;     /* donate while the worklist holds fewer than this fraction of its capacity */
    int64_t idle_timeout_ns;    /* VC_ETIMEOUT once an idle worker saw no progress anywhere for this long (default 20 s) */
    int32_t skip_validation;    /* 1: trust the CSR and skip the device check */
    int32_t stage_csr;          /* shared-memory copy of each worker's current graph: 0 = its offsets when
                                   n <= 1024, 1 = offsets and neighbour lists when they fit (fewer resident
                                   workers), -1 = nothing (all CSR reads through L1) */
    const volatile int32_t *cancel;  /* optional host-mapped or device flag; nonzero aborts with VC_ECANCELLED */
    int32_t node_in_global;     /* placement of each worker's current node (degree array, marks, removal
                                   list), Sec. IV-E's two kernel versions: 0 = shared memory when it fits,
                                   else global memory; 1 = always global memory; -1 = shared memory only
                                   (VC_EINVAL when it does not fit).  The global version keeps a private
                                   region of about 2 x n x 4 bytes per worker and reads it through L2.
                                   vc_mvc, vc_pvc, vc_mvc_batch, vc_greedy and vc_reduce_node honour it;
                                   the server, the batch plan and vc_mvc_noalloc keep the node in shared
                                   memory. */
    int32_t bit_rows;           /* adjacency lookups of one-warp, shared-memory workers: 0 = bit rows of the
                                   adjacency matrix in shared memory for graphs of at most 256 vertices,
                                   else CSR walks; 1 = bit rows required (VC_EINVAL when the launch does
                                   not qualify); -1 = CSR walks.  Same answers and reduced
                                   degree arrays either way.  vc_mvc, vc_pvc, vc_mvc_batch, vc_greedy,
                                   vc_reduce_node and the batch plan honour it; the server walks the
                                   CSR unless bit_rows = 1 (then graphs of at most 128 vertices run on
                                   bit rows, see vc_server.h); vc_mvc_noalloc walks the CSR. */
} vc_config;

/* Counters of one call (all filled by the device except kernel_ms and the sizes). */
typedef struct {
    int64_t nodes_visited;      /* search-tree nodes expanded by the traversal kernel */
    int64_t stack_pushes;       /* N(v) children pushed on a local stack */
    int64_t stack_pops;         /* local stack pops */
    int64_t donations;          /* N(v) children put on the worklist */
    int64_t worklist_pops;      /* worklist entries taken */
    int64_t rule_passes;        /* reduction-rule passes (each scans one degree array) */
    int64_t csr_words;          /* CSR neighbour words read during the search */
    int64_t entry_bytes_moved;  /* entry bytes copied between shared and global memory: entry size x (pops + pushes +
                                   donations + worklist pops) */
    int32_t max_depth;          /* deepest local stack seen */
    int32_t greedy_ub;          /* greedy upper bound (single-graph calls; batch: sum over graphs) */
    int32_t workers;            /* persistent workers launched */
    int32_t worker_threads;     /* threads per worker */
    int32_t width;              /* 16 or 32 */
    int32_t csr_staged;         /* 1 if the workers read the CSR from shared memory */
    int32_t status;             /* device status word (VC_OK or an error code) */
    float kernel_ms;            /* traversal kernel time (CUDA events on the call's stream) */
    float total_ms;             /* whole call (validation, greedy, traversal, copies) */
    int64_t trace_ns[4];        /* builds with -DVC_TRACE: worker time waiting for work, in reduction rules and
                                   stop checks, branching, recording solutions (Sec. V-D breakdown); else 0 */
    int64_t idle_polls;         /* builds with -DVC_TRACE: idle-loop iterations; else 0 */
    int32_t node_in_global;     /* 1 if the workers kept their current node in global memory */
    int32_t stack_depth;        /* entries provisioned per local stack */
    int32_t bit_rows;           /* words per adjacency bit row the workers used (0: CSR walks) */
    int64_t trace_cycles[16];   /* builds with -DVC_TRACE: SM cycles of each worker's first thread, summed
                                   over workers, in: [0] per-node snapshot, [1] degree-one, [2] degree-two-
                                   triangle and [3] high-degree pass scans, [4] removals applied by the
                                   passes, [5] stop checks, [6] argmax, [7] donate or push, [8] the "v"
                                   child, [9] stack pops, [10] N(v) children applied by their takers,
                                   [11] acquiring work, [12] solutions; [13]-[15] the number of degree-one,
                                   triangle and high-degree passes; else 0 */
} vc_stats;

/* Minimum Vertex Cover (Sec. II-A, II-B, IV).
 * cover_out: n int32 entries (host or device per g->on_device), receives 1 for vertices of a
 * minimum cover and 0 elsewhere; may be NULL.  *cover_size_out receives the minimum size.
 * cfg and stats may be NULL. */
int vc_mvc(const vc_graph *g, const vc_config *cfg, void *stream,
           int32_t *cover_out, int32_t *cover_size_out, vc_stats *stats);

/* Parameterized Vertex Cover (Sec. II-A, II-B last paragraph, IV-A last paragraph).
 * *found_out = 1 iff a cover of size <= k exists; then cover_out (n entries, may be NULL)
 * receives such a cover as a 0/1 mask and *cover_size_out its size (else -1).  k < 0 is answered
 * "no" without touching the GPU.  When the greedy bound is already <= k the answer is "yes" with
 * the greedy cover and no search runs. */
int vc_pvc(const vc_graph *g, int32_t k, const vc_config *cfg, void *stream,
           int32_t *found_out, int32_t *cover_out, int32_t *cover_size_out, vc_stats *stats);

/* Batched MVC: num_graphs independent graphs solved by one persistent launch whose worklist
 * entries carry their graph's index.  Graph g has graph_vtx_offsets[g+1]-graph_vtx_offsets[g]
 * vertices; its own n_g+1 offsets (starting at 0) sit at packed_offsets[graph_vtx_offsets[g] + g],
 * its neighbours (numbered 0..n_g-1) at packed_neighbors[graph_edge_offsets[g] ...].
 * sizes_out (host, num_graphs) receives each minimum size; covers_out (Σ n_g entries laid out by
 * graph_vtx_offsets, host or device per on_device, may be NULL) receives 0/1 cover masks.
 * graph_vtx_offsets and graph_edge_offsets are host arrays of num_graphs+1 entries. */
int vc_mvc_batch(int32_t num_graphs, const int32_t *graph_vtx_offsets, const int32_t *graph_edge_offsets,
                 const int32_t *packed_offsets, const int32_t *packed_neighbors, int32_t on_device,
                 const vc_config *cfg, void *stream, int32_t *sizes_out, int32_t *covers_out,
                 vc_stats *stats);

/* Greedy upper bound on the GPU (Sec. II-B): repeat { degree-one and degree-two-triangle rules to a
 * fixpoint; stop when edgeless; put the maximum-degree vertex (lowest id on ties) into S }.
 * *size_out receives |S|; cover_out (n entries, may be NULL) the cover mask. */
int vc_greedy(const vc_graph *g, const vc_config *cfg, void *stream, int32_t *cover_out, int32_t *size_out);

/* One tree node's reduction on the GPU (Sec. II-B rules with the Sec. IV-D tie-breaks), for
 * testing.  deg (n entries, host or device per g->on_device) holds the degree array (-1 = in S) and
 * is reduced in place; *S and *m hold |S| and the edge count and are updated.  problem: 0 = MVC
 * (bound = best), 1 = PVC (bound = k).  rules: bit 0 degree-one, bit 1 degree-two-triangle,
 * bit 2 high-degree.  *pruned_out receives 1 iff the stop check prunes the reduced node.
 * Every rule pass is one simultaneous round: vertices that meet the rule at the start of the pass
 * are found, then all of them enter S together.
 * branch = -1 reduces the given state.  branch = v >= 0 (or -2-v) treats the given state as a
 * fixpoint of the rules, first puts v (or every live neighbour of v) into S, and then reduces the
 * child the way the traversal does, re-examining only vertices whose degree changed. */
int vc_reduce_node(const vc_graph *g, int32_t *deg, int32_t *S, int32_t *m, int32_t problem,
                   int32_t bound, int32_t rules, int32_t branch, const vc_config *cfg, void *stream,
                   int32_t *pruned_out);

/* MVC without any allocation (the paper has no counterpart: this is a deployment variant).
 * For callers that cannot let a library allocate device memory, e.g. code that runs under a
 * memory pool or arena owning all device memory, processes that lock their allocator after
 * start-up, or request paths where cudaMalloc/cudaFree (and the synchronisation they imply) are
 * not allowed.  The search runs the same kernels as vc_mvc, but all of its scratch lives in one
 * fixed array of VC_NOALLOC_SCRATCH_BYTES bytes that is part of the library image: every device
 * that loads the library holds that array until the process exits, and this call allocates
 * nothing (no cudaMalloc, cudaFree or pinned host memory).
 *   - g must be on the device (on_device = 1) with n <= VC_NOALLOC_MAX_N; larger graphs and host
 *     pointers are rejected with VC_EINVAL.  cover_out (n int32, device, may be NULL) and
 *     *cover_size_out (host) receive the result; cfg and stats may be NULL.
 *   - The first call on a device does a one-time set-up: it looks up the array's device address
 *     (cudaGetSymbolAddress) with that device current.  Make that first call before any stream
 *     capture begins on the device.
 *   - cfg fields it reads: worker_threads, num_workers, donate_threshold, idle_timeout_ns,
 *     skip_validation, cancel, and stage_csr 0 or -1.  Entries are always 16-bit, the node stays
 *     in shared memory, the workers walk the CSR and the worklist is a fixed ring of 1024 entries:
 *     width 32, node_in_global 1, bit_rows 1, stage_csr 1 or any other worklist_capacity return
 *     VC_EINVAL.
 *   - All calls of a process share the one array, and each call resets what must start from a
 *     known value.  Calls are serialised: each holds a process-wide lock until its GPU work has
 *     finished, error returns included, so calls from any host threads and streams of one process
 *     never overlap on the array.  Each process has its own array.
 *   - The call synchronises `stream` twice (after the greedy bound, which sizes the stacks, and at
 *     the end). */
#define VC_NOALLOC_MAX_N 512
#define VC_NOALLOC_SCRATCH_BYTES (32u << 20)
int vc_mvc_noalloc(const vc_graph *g, const vc_config *cfg, void *stream, int32_t *cover_out,
                   int32_t *cover_size_out, vc_stats *stats);

/* Per-SM search-tree node counts of the last traversal on the current device (Sec. V-C load
 * measure): counts_out receives min(capacity, SM count) entries; returns the SM count or an
 * error code. */
int vc_last_sm_nodes(int64_t *counts_out, int32_t capacity);

/* Measurement helper (no counterpart in the paper): copies `bytes` from src to dst `passes` times in
 * one launch on `stream`, with every load and store through L2 only.  With a working set well
 * below the L2 size (for example 2 x 16 MiB) the launch time gives the L2 bandwidth that the
 * traversal's roofline is stated against (2 * bytes * passes moved).  dst and src are device
 * pointers, 16-byte aligned, bytes a multiple of 16, passes >= 1; VC_EINVAL otherwise.  Does not
 * wait for the stream. */
int vc_l2_copy_probe(void *dst, const void *src, size_t bytes, int32_t passes, void *stream);

/* Releases the cached device scratch of the current device. */
int vc_release(void);
/* Short name of a status code. */
const char *vc_strerror(int code);
/* Library version: major * 10000 + minor * 100 + patch. */
int vc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* VC_H */
