// vc_kernels.cuh - kernels of libvc, templated on the degree-array width W, the worker size WT,
// the node placement GM (shared or global memory) and the bit-row words NW (0: CSR walks).
//
//   validate_kernel     checks the CSR rules of vc.h (one thread per vertex)
//   greedy_kernel       greedy upper bound per problem (Sec. II-B): seeds best, the cover and the
//                       problem's work unit
//   traverse_kernel     persistent hybrid traversal (Sec. IV-A): local stack + device worklist
//                       with termination (Sec. IV-C), rules (Sec. IV-D), branch (Sec. IV-B)
//   reduce_node_kernel  one node's fixpoint reduction (rule tests)
//
// Every wait is bounded by %globaltimer: an idle worker that finds no work for idle_timeout_ns,
// or a cover-lock wait that lasts as long, records VC_ETIMEOUT and returns.
#pragma once

#include "vc_device.cuh"
#include "vc_rows.cuh"

namespace vc {

// The worker a kernel instance uses: bit rows (NW > 0: one-warp RowWorker, node in registers) or
// CSR walks (Worker of WT threads, node in shared or, GM, global memory).
template <typename W, int WT, bool GM, int NW, bool ROWS = (NW > 0)>
struct WorkerSel {
    using type = Worker<W, WT, GM>;
};
template <typename W, int WT, bool GM, int NW>
struct WorkerSel<W, WT, GM, NW, true> {
    static_assert(WT == 32 && !GM, "bit rows are for one-warp shared-memory workers");
    using type = RowWorker<W, NW>;
};

// ------------------------------------------------------------------------------------------------
// CSR validation: offsets monotone from 0, neighbours in range, sorted strictly ascending, no
// self-loops, every edge listed at both endpoints, offsets[n] equal to the expected length.
// ------------------------------------------------------------------------------------------------
__global__ void validate_kernel(const int32_t *offsets, const int32_t *neighbors, const Problem *probs,
                                const int64_t *adj_len, int32_t num_problems, int64_t total_vertices,
                                Control *ctrl);

__global__ void init_worklist_kernel(uint32_t *seq, int32_t capacity, Control *ctrl,
                                     unsigned long long *claim_state);

// ------------------------------------------------------------------------------------------------
// Greedy upper bound (Sec. II-B; the oracle's reading R5): repeat {degree-one and
// degree-two-triangle rules to a fixpoint; stop when edgeless; put the maximum-degree vertex into
// S}.  Leaves the greedy cover in the problem's cover mask and best / greedy / cover_size (and the
// PVC found flag when the greedy cover already fits) in its record.  Returns whether a search is
// still needed (uniform across the block).
// ------------------------------------------------------------------------------------------------
// Where a problem's bit rows live in global memory (bit-row kernels), or null.
template <int NW>
__device__ __forceinline__ uint32_t *rows_of(const Params &P, const Ctx &c) {
    if constexpr (NW == 0) return nullptr;
    else return P.rows ? P.rows + (size_t)(c.cover - P.cover) * NW : nullptr;
}

// A problem's root entry (Params::roots), written by the greedy pass.
__device__ __forceinline__ uint8_t *root_entry(const Params &P, int32_t p) {
    return P.roots + __ldcg(&P.problems[p].root_base);
}

// The root node of problem p: the greedy pass's first fixpoint when it was kept, else the whole
// graph from the CSR.
template <class Wk>
__device__ __forceinline__ void load_root_node(const Params &P, Wk &w, int32_t p) {
    if (P.roots) w.load_entry(root_entry(P, p), P.entry_bytes, P.n_max);
    else w.load_root(make_ctx(P, p));
}

template <class Wk>
__device__ bool greedy_solve(const Params &P, Wk &w, Ctx &c) {
    w.cur_n = c.n;
    if (c.n == 0) {
        w.sync();
        if (w.tid == 0) {
            c.prob->greedy = c.prob->cover_size = c.prob->best = 0;
            c.prob->m = 0;
            if (c.kind == kPVC && c.k >= 0) c.prob->found = 1;
        }
        w.sync();
        return false;
    }
    w.stage(c, rows_of<Wk::kRowWords>(P, c));
    w.load_root(c);
    const int32_t m0 = w.node_m();
    for (bool first = true;; first = false) {
        reduce_fixpoint(w, c, 0, kRuleDeg1 | kRuleDeg2Tri, false);
        // The first fixpoint is the root node with its degree-one and triangle vertices in S: the
        // traversal starts from it instead of reducing the whole graph again (reading R13).
        if (first && P.roots) {
            w.store_entry(root_entry(P, c.index), P.entry_bytes, -1);
            w.sync();
        }
        if (w.node_m() == 0) break;
        int dv;
        const int v = w.argmax(c, dv);
        if (v < 0) break;  // unreachable: m > 0 implies a live vertex of degree >= 1
        w.take_vertex(c, v);
    }
    w.write_cover(c);
    const int32_t S = w.node_S();
    w.sync();
    if (w.tid == 0) {
        __threadfence();
        Problem *pr = c.prob;
        pr->m = m0;
        pr->greedy = S;
        pr->best = S;
        pr->cover_size = S;
        if (c.kind == kPVC && c.k >= 0 && S <= c.k) pr->found = 1;  // greedy already fits (reading R6)
    }
    w.sync();
    // An edgeless graph needs no search; PVC needs none when k < 0 or the greedy cover fits.
    return c.kind == kMVC ? S > 0 : (c.k >= 0 && S > c.k);
}

template <typename W, int WT, bool GM, int NW>
__global__ void __launch_bounds__(WT) greedy_kernel(Params P) {
    extern __shared__ __align__(16) uint8_t smem[];
    typename WorkerSel<W, WT, GM, NW>::type w(smem, P.n_max, P.csr_words,
                                              P.gstate + (size_t)blockIdx.x * (size_t)P.gstate_bytes);
    w.init_scratch(P.n_max);
    if (w.tid == 0) w.sc[kScB0] = ld_relaxed(&P.ctrl->status);
    w.sync();
    if (w.sc[kScB0] != VC_OK) return;
    w.dbg = P.ctrl;
    if (blockIdx.x == 0 && w.tid == 0) P.ctrl->t_launch_ns = globaltimer_ns();
    for (int p = blockIdx.x; p < P.num_problems; p += gridDim.x) {
        Ctx c = make_ctx(P, p);
        const bool search = greedy_solve(P, w, c);
        if (w.tid == 0) {
            c.prob->units = search ? 1 : 0;
            c.prob->done = search ? 0 : 1;
            if (!search) c.prob->t_done_ns = (int64_t)globaltimer_ns();  // answered by the greedy bound
            if (search) atomicAdd(&P.ctrl->units_total, 1);
        }
    }
}

// ------------------------------------------------------------------------------------------------
// Worklist (Sec. IV-A, IV-C): a ring of `capacity` entry slots (a power of two) with one sequence
// word per slot, and four counters on separate lines:
//   wl_space  free slots            producers reserve one before taking a ticket
//   wl_tail   producer tickets      ticket t writes slot t mod capacity
//   wl_count  published entries     consumers reserve one before taking a ticket
//   wl_head   consumer tickets      ticket t reads slot t mod capacity
// Slot s is writable for producer ticket t when seq[s] == t and readable for consumer ticket t
// when seq[s] == t + 1; the consumer frees it for the next lap with seq[s] = t + capacity.
// A reservation on wl_space / wl_count guarantees that the slot's previous user (or its producer)
// already holds its ticket, so the only waits are for operations already in progress; they are
// still bounded by idle_timeout_ns.  An idle poll is one relaxed load of wl_count.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ bool wait_seq(const Params &P, uint32_t slot, uint32_t want) {
    uint64_t t0 = 0;
    while (ld_acquire_u32(&P.wl_seq[slot]) != want) {
        const uint64_t now = globaltimer_ns();
        if (t0 == 0) {
            t0 = now;
        } else if (now - t0 > (uint64_t)P.idle_timeout_ns) {
            raise_status(P.ctrl, VC_ETIMEOUT);
            return false;
        }
        __nanosleep(20);
    }
    return true;
}

// Producer side: a ticket whose slot is ready for writing, or -1 (worklist at its threshold or
// full: the caller pushes on its local stack instead), or -2 (timed out).  `fill` is the
// worklist count the caller saw (read with the node's snapshot, so that the threshold test costs
// no extra round trip to L2; the free-slot reservation below is what bounds the ring).
__device__ __forceinline__ long long wl_reserve(const Params &P, int32_t fill) {
    Control *c = P.ctrl;
    if (fill >= P.wl_threshold) return -1;
    if (atomicSub(&c->wl_space, 1) <= 0) {
        atomicAdd(&c->wl_space, 1);
        return -1;
    }
    const uint32_t t = atomicAdd(&c->wl_tail, 1u);
    if (!wait_seq(P, t & ((uint32_t)P.wl_capacity - 1u), t)) return -2;
    return (long long)t;
}

// Consumer side: a ticket whose slot holds a published entry, or -1 (nothing published), or -2.
__device__ __forceinline__ long long wl_take(const Params &P) {
    Control *c = P.ctrl;
    if (ld_relaxed(&c->wl_count) <= 0) return -1;
    if (atomicSub(&c->wl_count, 1) <= 0) {
        atomicAdd(&c->wl_count, 1);
        return -1;
    }
    const uint32_t t = atomicAdd(&c->wl_head, 1u);
    if (!wait_seq(P, t & ((uint32_t)P.wl_capacity - 1u), t + 1u)) return -2;
    return (long long)t;
}

// Gives back the work unit a worker held for problem p (its node and local stack are finished).
// The worker that releases a problem's last unit completes it; a serving launch then writes the
// answer into the host-visible completion record, tag last.
__device__ __forceinline__ void release_unit(const Params &P, int32_t p) {
    Problem *pr = P.problems + p;
    __threadfence();
    if (atomicSub(&pr->units, 1) == 1) {
        pr->t_done_ns = (int64_t)globaltimer_ns();
        st_release(&pr->done, 1);
        if (P.completion) {
            volatile int32_t *rec = P.completion + 4 * (size_t)p;
            rec[1] = __ldcg(&pr->kind) == kMVC ? ld_relaxed(&pr->best) : ld_relaxed(&pr->found);
            rec[2] = ld_relaxed(&P.ctrl->status);
            rec[3] = ld_relaxed(&pr->greedy);
            __threadfence_system();
            rec[0] = __ldcg(&pr->tag);
        }
    }
    atomicSub(&P.ctrl->units_total, 1);
}

__device__ __forceinline__ bool cover_lock(const Params &P, Problem *pr) {
    const uint64_t t0 = globaltimer_ns();
    while (atomicCAS(&pr->lock, 0, 1) != 0) {
        if (globaltimer_ns() - t0 > (uint64_t)P.idle_timeout_ns) {
            raise_status(P.ctrl, VC_ETIMEOUT);
            return false;
        }
        __nanosleep(64);
    }
    __threadfence();
    return true;
}

// An edgeless node passed the stop check: MVC lowers best (atomicMin) and, if it still holds the
// smallest size under the cover lock, writes its cover; PVC raises the found flag and the first
// worker to raise it writes the cover (Sec. IV-A).
template <class Wk>
__device__ void record_solution(const Params &P, Wk &w, const Ctx &c) {
    const int32_t S = w.node_S();
    bool locked = false, write = false;
    if (w.tid == 0) {
        if (c.kind == kMVC) {
            const int32_t old = atomicMin(&c.prob->best, S);
            if (S < old) {
                locked = cover_lock(P, c.prob);
                write = locked && S < ld_relaxed(&c.prob->cover_size);
            }
        } else {
            write = atomicCAS(&c.prob->found, 0, 1) == 0;
        }
        w.sc[kScB3] = write;
    }
    w.sync();
    if (w.sc[kScB3]) w.write_cover(c);
    w.sync();
    if (w.tid == 0) {
        if (write) {
            __threadfence();
            st_release(&c.prob->cover_size, S);
        }
        if (locked) {
            __threadfence();
            atomicExch(&c.prob->lock, 0);
        }
    }
}

// Serving idle loop (thread 0): a worklist entry (returns 2, ticket in arg), a newly admitted
// request (returns 3, slot in arg; the caller holds its unit and runs its greedy bound), or 0 when
// the launch closes.  Claiming and closing go through one 64-bit word (closing bit | claimed
// count), so a claim and a close can never both succeed; a claimer counts its unit before it
// claims, so a closer that saw no unit left cannot overtake a claim in progress.  An empty launch
// closes after linger_ns idle (or at once when the host asks), and the host relaunches when new
// requests arrive.
__device__ __forceinline__ int serve_wait(const Params &P, int &arg) {
    Control *ctrl = P.ctrl;
    uint64_t t0 = globaltimer_ns();
    uint32_t beat = ld_relaxed_u32(&ctrl->heartbeat);
    unsigned sleep_ns = 64 + (blockIdx.x & 63);
    for (;;) {
        if (ld_relaxed(&ctrl->status) != VC_OK) return 0;
        const long long pos = wl_take(P);
        if (pos >= 0) {
            arg = (int)(uint32_t)pos;
            return 2;
        }
        if (pos == -2) return 0;
        const unsigned long long st = ld_relaxed_u64(P.claim_state);
        if (st >> 32) return 0;  // the launch is closing
        const uint32_t claimed = (uint32_t)st;
        if (claimed < ld_relaxed_u32(P.sub_tail)) {
            atomicAdd(&ctrl->units_total, 1);
            if (atomicCAS(P.claim_state, st, st + 1ull) == st) {
                const uint32_t slot = ld_relaxed_u32(&P.sub_ring[claimed & P.sub_mask]);
                atomicExch(&P.problems[slot].units, 1);
                arg = (int)slot;
                return 3;
            }
            atomicSub(&ctrl->units_total, 1);
            continue;
        }
        const uint64_t now = globaltimer_ns();
        if (ld_acquire(&ctrl->units_total) == 0) {
            if (ld_relaxed(P.close_now) != 0 || now - t0 > (uint64_t)P.linger_ns) {
                if (atomicCAS(P.claim_state, st, st | (1ull << 32)) == st) return 0;
                continue;
            }
        } else {
            const uint32_t b = ld_relaxed_u32(&ctrl->heartbeat);
            if (b != beat) {
                beat = b;
                t0 = now;
            } else if (now - t0 > (uint64_t)P.idle_timeout_ns) {
                raise_status(ctrl, VC_ETIMEOUT);
                return 0;
            }
        }
        if (P.cancel && *P.cancel) {
            raise_status(ctrl, VC_ECANCELLED);
            return 0;
        }
        __nanosleep(sleep_ns);
        if (sleep_ns < 8192) sleep_ns += sleep_ns >> 1;
    }
}

// Finds the next node for a worker whose local stack is empty: an unclaimed root first, then the
// worklist; idles with a growing sleep while other workers still hold work.  Returns 0 (stop),
// 1 (a root is loaded), 2 (a worklist entry is loaded) or, in serving launches, 3 (a new request
// is claimed; see serve_wait).  Sec. IV-C: the search is over when
// the worklist is empty and no worker holds work, i.e. when no work unit is left.
constexpr int kAwakeWorkers = 608;       // idle bit-row workers that poll at once in a small search
constexpr uint32_t kParkBeats = 64;      // heartbeat (busy workers bump it every 32 nodes) that ends parking
constexpr unsigned kParkNs = 16384;      // a parked worker's poll interval
template <bool SERVE, class Wk>
__device__ int acquire(const Params &P, Wk &w) {
    Control *ctrl = P.ctrl;
    if (w.tid == 0) {
        int result = 0, arg = 0;
        // Unclaimed roots; a serving launch gets its problems through serve_wait instead (its slots
        // hold no work until a request is claimed, and sweeping them cost every launch 16 K atomics).
        if (!(SERVE && P.serving)) {
            while (ld_relaxed(&ctrl->next_root) < P.num_problems) {
                const int r = atomicAdd(&ctrl->next_root, 1);
                if (r >= P.num_problems) break;
                if (ld_relaxed(&P.problems[r].units) > 0) {
                    result = 1;
                    arg = r;
                    break;
                }
            }
        }
        if (SERVE && !result && P.serving) {
            result = serve_wait(P, arg);
        } else if (!result) {
            // The wait ends with work, with the end of the search, or after idle_timeout_ns during
            // which no busy worker showed progress (heartbeat unchanged): a stalled launch reports
            // VC_ETIMEOUT instead of spinning forever.  Sleeps grow geometrically (with a per-worker
            // offset) so that thousands of idle workers do not flood the worklist counters.
            uint64_t t0 = globaltimer_ns();
            uint32_t beat = ld_relaxed_u32(&ctrl->heartbeat);
            unsigned sleep_ns = 64 + (blockIdx.x & 63);
            if constexpr (Wk::kRowWords > 0) {
                // While the search is small (heartbeat below 64: fewer than about 2 K nodes so far),
                // bit-row workers beyond the first kAwakeWorkers start parked, polling every 16 us:
                // thousands of pollers racing for the few entries of a small search slowed the
                // workers that had work (G(60, 0.10): 113 -> 80 us of traversal; the 4096-graph
                // batch and the planted cliques unchanged).  They join once the heartbeat grows.
                if ((int)blockIdx.x >= kAwakeWorkers && beat < kParkBeats) sleep_ns = kParkNs;
            }
            for (;;) {
                const long long pos = wl_take(P);
                if (pos >= 0) {
                    result = 2;
                    arg = (int)(uint32_t)pos;
                    break;
                }
                if (pos == -2) break;
                if (ld_relaxed(&ctrl->status) != VC_OK) break;
                if (ld_acquire(&ctrl->units_total) == 0) break;
                if (P.cancel && *P.cancel) {
                    raise_status(ctrl, VC_ECANCELLED);
                    break;
                }
                const uint64_t now = globaltimer_ns();
                const uint32_t b = ld_relaxed_u32(&ctrl->heartbeat);
                if (b != beat) {
                    beat = b;
                    t0 = now;
                } else if (now - t0 > (uint64_t)P.idle_timeout_ns) {
                    raise_status(ctrl, VC_ETIMEOUT);
                    break;
                }
#ifdef VC_TRACE
                w.tally[kTIdlePolls] += 1;
#endif
                __nanosleep(sleep_ns);
                if (sleep_ns < 8192) sleep_ns += sleep_ns >> 1;
                if constexpr (Wk::kRowWords > 0) {
                    if (sleep_ns > 8192 && b >= kParkBeats) sleep_ns = 8192;
                }
            }
        }
        w.sc[kScB4] = result;
        w.sc[kScB5] = arg;
    }
    w.sync();
    const int result = w.sc[kScB4];
    const int arg = w.sc[kScB5];
    if (result == 1) {
        VC_CHECK(ctrl, arg >= 0 && arg < P.num_problems, 12, arg, return 0);
        load_root_node(P, w, arg);
    } else if (result == 3) {
        VC_CHECK(ctrl, arg >= 0 && arg < P.num_problems, 18, arg, return 0);
    } else if (result == 2) {
        const uint32_t pos = (uint32_t)arg;
        const uint32_t slot = pos & ((uint32_t)P.wl_capacity - 1u);
        w.load_entry(P.wl_slots + (size_t)slot * P.entry_bytes, P.entry_bytes, P.n_max);
        if (w.tid == 0) {
            st_release_u32(&P.wl_seq[slot], pos + (uint32_t)P.wl_capacity);
            atomicAdd(&ctrl->wl_space, 1);
            w.tally[kTDequeues] += 1;
        }
    }
    return result;
}

// ------------------------------------------------------------------------------------------------
// Persistent hybrid traversal (Sec. IV-A): one worker per thread block.
// ------------------------------------------------------------------------------------------------
// At most 64 registers per thread, so every worker size keeps 1024 threads resident per SM
// (measured: the uncapped build used 72 registers, fit 28 one-warp blocks per SM and ran 4 % slower).
// One-warp workers declare 64 threads / 16 blocks, the same 64-register cap; with the worker's
// compile-time warp indices this build ran the 4096-graph batch in 174 ms against 180 ms for
// (32, 32) on one GB300.  More resident warps did not pay: 48, 40 and 32 registers with two or
// four workers per block (40 to 64 warps per SM) ran 171, 180 and 250 ms against 171 ms for the
// same build at 64 registers.  Eight-word bit-row workers (graphs of 129-256 vertices) declare 32
// threads / 28 blocks instead: their node needs more registers, and at the 64-register cap they
// spilled 136 bytes and ran the planted clique G(200, 0.05) + K_12 in 1420 ms; at 128 / 96 / 85
// registers (16 / 20 / 24 workers per SM) it took 1080 / 991 / 964 ms, against 1255 ms for CSR walks.
// With the passes' dynamic candidate loops, 22 / 24 / 28 blocks (80, 80, 72 registers; 16-96 bytes
// of spills) took 849 / 848 / 835 ms.
constexpr int kMaxThreads(int wt) { return wt == 32 ? 64 : wt; }
constexpr unsigned kSnapshotEvery = 16;  // nodes per re-read of the shared bounds (a power of two)
constexpr int kMinBlocks(int wt) { return wt == 32 ? 16 : 1024 / wt; }
// SERVE: the launch also takes requests from a server's ring (the instance the server launches);
// batch launches use the instance without that path, which keeps their code smaller.
template <typename W, int WT, bool GM, int NW, bool SERVE>
__global__ void __launch_bounds__(NW == 8 ? 32 : kMaxThreads(WT), NW == 8 ? 28 : kMinBlocks(WT)) traverse_kernel(Params P) {
    extern __shared__ __align__(16) uint8_t smem[];
    using Wk = typename WorkerSel<W, WT, GM, NW>::type;
    Wk w(smem, P.n_max, P.csr_words, P.gstate + (size_t)blockIdx.x * (size_t)P.gstate_bytes);
    w.init_scratch(P.n_max);
    Control *ctrl = P.ctrl;
    w.dbg = ctrl;
    const int32_t eb = P.entry_bytes;
    uint8_t *stack = P.stacks + (size_t)blockIdx.x * (size_t)P.stack_depth * (size_t)eb;
    const uint32_t wl_mask = (uint32_t)P.wl_capacity - 1u;
    int top = 0;
    int cur = -1;
    bool stop = false;
    bool fresh = true;  // the next node needs a fresh snapshot (its problem may be new)
    uint32_t nn = 0;    // bit-row workers: nodes expanded (its low bits pace the periodic work)
    int32_t bound = 0;  // snapshot: best (MVC) or k (PVC), one value for a whole node (reading R3)
    int32_t fill = 0;   // snapshot: worklist entries waiting
    Ctx c;
    c.n = 0;

    if (w.tid == 0) w.sc[kScB0] = ld_relaxed(&ctrl->status);
    w.sync();
    if (w.sc[kScB0] != VC_OK) return;

    while (!stop) {
        // Every warp must have finished reading the previous node (its prune / stop / solution
        // decision reads the header) before any warp overwrites it with the next one.
        w.sync();
        // ---- acquire: local stack first (Sec. IV-A), then a root or the worklist ----
        if (top > 0) {
            const long long t_pop = VC_CYC();
            --top;
            w.load_entry(stack + (size_t)top * eb, eb, P.n_max);
            w.node_loaded(c);
            if (w.tid == 0) w.tally[kTPops] += 1;
            VC_CYC_ADD(w, kPPop, t_pop);
        } else {
            if (cur >= 0 && w.tid == 0) release_unit(P, cur);
            cur = -1;
            const unsigned long long t_wait = VC_TRACE_NOW();
            const long long t_acq = VC_CYC();
            int got = acquire<SERVE>(P, w);
            fresh = true;
            VC_TRACE_ADD(w, kTWaitNs, t_wait);
            VC_CYC_ADD(w, kPAcquire, t_acq);
            if (got == 0) break;
            if (SERVE && got == 3) {  // serving: a new request; this worker holds its unit
                if constexpr (SERVE) {
                    cur = w.sc[kScB5];
                    c = make_ctx(P, cur);
                    VC_CHECK(ctrl, c.n >= 0 && c.n <= P.n_max, 19, c.n, { stop = true; break; });
                    if (!greedy_solve(P, w, c)) continue;  // answered by the greedy bound: release
                    load_root_node(P, w, cur);
                    w.node_loaded(c);
                }
            } else {
                cur = w.node_problem();
                VC_CHECK(ctrl, cur >= 0 && cur < P.num_problems, 1, cur, { stop = true; break; });
                c = make_ctx(P, cur);
                VC_CHECK(ctrl, c.n >= 0 && c.n <= P.n_max, 14, c.n, { stop = true; break; });
                w.cur_n = c.n;
                w.template stage<false>(c, rows_of<Wk::kRowWords>(P, c));
                w.node_loaded(c);
            }
        }
        const int32_t br = w.node_branch();
        VC_CHECK(ctrl, br < c.n, 13, br, { stop = true; break; });
        if (br >= 0) {  // a lazily stored N(v) child: apply the removal now
            const long long t_tn = VC_CYC();
            w.take_neighbourhood(c, br);
            w.clear_branch();
            VC_CYC_ADD(w, kPTakeN, t_tn);
        }

        // ---- expand nodes, continuing into the "v" child after each branch ----
        for (;;) {
            const long long t_hdr = VC_CYC();
            // The snapshot of best / found / status / worklist fill is re-read for every 16th node
            // and for the first node after acquiring work (reading R3: a stale, larger best only
            // weakens pruning).  Re-reading it for every node cost 2.5 % of the batch time, and for
            // every fourth node 0.5 %.  Busy workers bump the heartbeat every 32 nodes and honour
            // the caller's cancel flag every 1024 (the flag may live in host memory; the status
            // read of the next snapshot then stops the worker).
            if constexpr (Wk::kRowWords > 0) {
                // One warp, node in registers: the node count and the snapshot live in registers,
                // every lane reads the shared words itself, and the found flag and the status are
                // looked at only when they are re-read.
                ++nn;
                if ((nn & 31u) == 0u && w.tid == 0) atomicAdd(&ctrl->heartbeat, 1u);
                if ((nn & 1023u) == 0u) {
                    w.flush_counts();  // statistics kept in registers go to the shared tallies
                    if (w.tid == 0) {
                        w.tally[kTNodes] += 1024ull;
                        if (P.cancel && *P.cancel) raise_status(ctrl, VC_ECANCELLED);
                    }
                }
                if (fresh || (nn & (kSnapshotEvery - 1u)) == 0u) {
                    bound = (c.kind == kMVC) ? ld_relaxed(&c.prob->best) : c.k;
                    const int32_t found = (c.kind == kPVC) ? ld_relaxed(&c.prob->found) : 0;
                    const int32_t status = ld_relaxed(&ctrl->status);
                    fill = ld_relaxed(&ctrl->wl_count);
                    fresh = false;
                    if (status != VC_OK) {
                        stop = true;
                        break;
                    }
                    if (found) {  // PVC already answered: drop this problem's remaining work
                        w.discard_pending();
                        top = 0;
                        break;
                    }
                }
            } else {
                // Node in shared memory: thread 0 keeps the count and the snapshot in shared
                // memory (registers are scarcer here), and the worker reads them after a barrier.
                if (w.tid == 0) {
                    const unsigned long long n64 = ++w.tally[kTNodes];
                    if ((n64 & 31) == 0) atomicAdd(&ctrl->heartbeat, 1u);
                    if ((n64 & 1023) == 0 && P.cancel && *P.cancel) raise_status(ctrl, VC_ECANCELLED);
                    if (fresh || (n64 & (kSnapshotEvery - 1)) == 0) {
                        w.sc[kScB0] = (c.kind == kMVC) ? ld_relaxed(&c.prob->best) : c.k;
                        w.sc[kScB1] = (c.kind == kPVC) ? ld_relaxed(&c.prob->found) : 0;
                        w.sc[kScB2] = ld_relaxed(&ctrl->status);
                        w.sc[kScWlHint] = ld_relaxed(&ctrl->wl_count);
                    }
                }
                fresh = false;
                w.sync();
                bound = w.sc[kScB0];
                if (w.sc[kScB2] != VC_OK) {
                    stop = true;
                    break;
                }
                if (w.sc[kScB1]) {  // PVC already answered: drop this problem's remaining work
                    w.discard_pending();
                    top = 0;
                    break;
                }
            }
            VC_CYC_ADD(w, kPHeader, t_hdr);
            const unsigned long long t_red = VC_TRACE_NOW();
            const bool reduced_out = reduce_fixpoint(w, c, bound, kRuleAll, true);
            const long long t_stop = VC_CYC();
            const bool pruned = reduced_out || w.must_stop(c, bound);
            VC_CYC_ADD(w, kPStop, t_stop);
            VC_TRACE_ADD(w, kTReduceNs, t_red);
            if (pruned) break;
            if (w.node_m() == 0) {
                const unsigned long long t_sol = VC_TRACE_NOW();
                const long long t_solc = VC_CYC();
                record_solution(P, w, c);
                VC_TRACE_ADD(w, kTSolutionNs, t_sol);
                VC_CYC_ADD(w, kPSolution, t_solc);
                break;
            }
            const unsigned long long t_br = VC_TRACE_NOW();
            const long long t_am = VC_CYC();
            int dv;
            const int v = w.argmax(c, dv);
            VC_CYC_ADD(w, kPArgmax, t_am);
            const long long t_store = VC_CYC();
            if (v < 0) {  // unreachable: m > 0 implies a live vertex of degree >= 1
                if (w.tid == 0) raise_status(ctrl, VC_EINVAL);
                stop = true;
                break;
            }
            const int32_t S = w.node_S();
            // The N(v) child puts dv vertices into S; skip it when that alone prunes it.
            const bool keep = (c.kind == kMVC) ? (S + dv < bound) : (S + dv <= c.k);
            if (keep) {
                int32_t donate, pos;
                if constexpr (Wk::kRowWords > 0) {
                    long long t = -1;
                    if (w.tid == 0) t = wl_reserve(P, fill);
                    donate = __shfl_sync(kFull, t >= 0 ? 1 : 0, 0);
                    pos = __shfl_sync(kFull, (int32_t)(uint32_t)(t >= 0 ? t : 0), 0);
                } else {
                    if (w.tid == 0) {
                        const long long t = wl_reserve(P, w.sc[kScWlHint]);
                        w.sc[kScB3] = t >= 0;
                        w.sc[kScB4] = (int32_t)(uint32_t)(t >= 0 ? t : 0);
                    }
                    w.sync();
                    donate = w.sc[kScB3];
                    pos = w.sc[kScB4];
                }
                if (donate) {  // donate (Sec. IV-A: the worklist is below its threshold)
                    const uint32_t ticket = (uint32_t)pos;
                    w.store_entry(P.wl_slots + (size_t)(ticket & wl_mask) * eb, eb, v);
                    w.sync();  // every thread's part of the entry is written ...
                    if (w.tid == 0) {
                        __threadfence();  // ... and ordered before the publication below
                        atomicAdd(&c.prob->units, 1);
                        atomicAdd(&ctrl->units_total, 1);
                        st_release_u32(&P.wl_seq[ticket & wl_mask], ticket + 1u);
                        atomicAdd(&ctrl->wl_count, 1);
                        w.tally[kTDonations] += 1;
                    }
                } else {  // push on the local stack
                    if (top >= P.stack_depth) {
                        if (w.tid == 0) raise_status(ctrl, VC_ESTACK);
                        stop = true;
                        break;
                    }
                    w.store_entry(stack + (size_t)top * eb, eb, v);
                    ++top;
                    if (w.tid == 0) {
                        w.tally[kTPushes] += 1;
                        if ((unsigned long long)top > w.tally[kTMaxDepth]) w.tally[kTMaxDepth] = top;
                    }
                    w.sync();
                }
            }
            VC_CYC_ADD(w, kPStore, t_store);
            const long long t_tv = VC_CYC();
            w.take_vertex(c, v);
            VC_CYC_ADD(w, kPTakeV, t_tv);
            VC_TRACE_ADD(w, kTBranchNs, t_br);
        }
    }

    // ---- statistics ----
    w.flush_counts();
    w.sync();
    if (w.tid == 0) {
        if constexpr (Wk::kRowWords > 0) w.tally[kTNodes] += (unsigned long long)(nn & 1023u);
        const unsigned long long *T = w.tally;
#ifndef VC_TRACE
        // A worker that expanded no node has nothing to add (every tally counts node work): the
        // idle workers of a small search skip their 9 atomics on the same few counters.
        if (T[kTNodes] == 0) return;
#endif
        atomicAdd(&ctrl->nodes, T[kTNodes]);
        atomicAdd(&ctrl->stack_pushes, T[kTPushes]);
        atomicAdd(&ctrl->stack_pops, T[kTPops]);
        atomicAdd(&ctrl->donations, T[kTDonations]);
        atomicAdd(&ctrl->worklist_pops, T[kTDequeues]);
        atomicAdd(&ctrl->rule_passes, T[kTPasses]);
        atomicAdd(&ctrl->csr_words, T[kTCsr]);
#ifdef VC_TRACE
        atomicAdd(&ctrl->trace_ns[0], T[kTWaitNs]);
        atomicAdd(&ctrl->trace_ns[1], T[kTReduceNs]);
        atomicAdd(&ctrl->trace_ns[2], T[kTBranchNs]);
        atomicAdd(&ctrl->trace_ns[3], T[kTSolutionNs]);
        atomicAdd(&ctrl->idle_polls, T[kTIdlePolls]);
        for (int i = 0; i < kProfSlots; ++i) atomicAdd(&ctrl->trace_cycles[i], w.prof()[i]);
#endif
        atomicMax(&ctrl->max_depth, (int32_t)T[kTMaxDepth]);
        if (P.sm_nodes) atomicAdd(&P.sm_nodes[smid() & (kSmSlots - 1)], T[kTNodes]);
    }
}

// ------------------------------------------------------------------------------------------------
// One node's reduction (tests): reads an int32 degree array, reduces it to the fixpoint (no early
// exit, like the oracle), writes it back with |S|, m and the stop verdict.
// ------------------------------------------------------------------------------------------------
template <typename W, int WT, bool GM, int NW>
__global__ void __launch_bounds__(WT) reduce_node_kernel(ReduceParams R) {
    extern __shared__ __align__(16) uint8_t smem[];
    typename WorkerSel<W, WT, GM, NW>::type w(smem, R.n, 0, R.gstate);
    w.init_scratch(R.n);
    Ctx c;
    c.off = R.offsets;
    c.adj = R.neighbors;
    c.prob = nullptr;
    c.cover = nullptr;
    c.n = R.n;
    c.kind = R.problem;
    c.k = R.bound;
    c.index = 0;
    w.cur_n = R.n;
    w.stage(c, nullptr);  // bit rows built from the CSR (CSR-walk workers stage nothing here)
    // A state from outside has every vertex looked at; a branch from a fixpoint state starts
    // clean, like a stored node in the traversal.
    w.load_plain(c, R.deg, R.io[0], R.io[1], R.branch == -1);
    if (R.branch >= 0) w.take_vertex(c, R.branch);
    else if (R.branch <= -2) w.take_neighbourhood(c, -2 - R.branch);
    reduce_fixpoint(w, c, R.bound, R.rules, false);
    const bool pruned = w.must_stop(c, R.bound);
    w.save_plain(c, R.deg);
    if (w.tid == 0) {
        R.io[0] = w.node_S();
        R.io[1] = w.node_m();
        R.io[2] = pruned ? 1 : 0;
    }
}

}  // namespace vc
