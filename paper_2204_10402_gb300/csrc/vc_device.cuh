// vc_device.cuh - device building blocks of the traversal: the CSR-walk worker (a thread block
// of WT threads) holds the current tree node in shared memory and applies the reduction rules,
// the maximum-degree selection and the two branch removals to it by walking the CSR.  (Graphs of
// at most 256 vertices may use the bit-row worker of vc_rows.cuh instead, which has the same
// interface.)
//
// Shared-memory layout of a worker (all offsets 16-byte aligned):
//   [entry]  EntryHeader (16 B) + degree array W[n_max] padded to 16 B   <- copied to/from stacks
//   [marks]  CSR-walk workers: one bit per vertex, chosen for S in the current pass
//   [dirty]  one 64-bit word per 32 vertices: low half = degree changed to one since the degree-one
//            pass last looked at the vertex, high half = changed to two since the degree-two-triangle
//            pass last looked at it
//   [list]   CSR-walk workers: int32[n_max], the vertices chosen in the current pass (each once)
//   [sc]     kScratchWords int32: tallies, broadcasts, per-warp reduction keys, trace slots
//   [csr]    optional copy of the current graph's CSR (offsets, then neighbours), so that the
//            adjacency walks of the rules and branches cost shared-memory latency
// The global-memory version (GM) keeps [entry]'s degree array, [marks], [dirty] and [list] in a
// per-worker global region instead; the header and [sc] stay in shared memory.
//
// Degree-array semantics (Sec. IV-B): d[v] >= 0 is v's degree in G - S, d[v] = -1 means v is in S.
// W is int16_t or int32_t; -1 is the sentinel at both widths.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "vc_internal.h"

namespace vc {

constexpr unsigned kFull = 0xffffffffu;


// Scratch word indices.
enum : int {
    kScCount = 0,   // entries in the removal list
    kScEdges = 1,   // edges removed by the current removal
    kScB0 = 2,      // broadcast slots
    kScB1 = 3,
    kScB2 = 4,
    kScB3 = 5,
    kScB4 = 6,
    kScB5 = 7,
    kScWlHint = 40, // worklist fill seen by the node's snapshot
    kScMaxDeg = 41, // an upper bound on the current node's largest live degree (degrees only fall)
    kScMaxDegNext = 42, // CSR-walk workers: the bound a running high-degree pass collects
    kScKeys = 48,   // 16 x u64 per-warp argmax keys (words 48..79)
};

// ------------------------------------------------------------------------------------------------
// Memory-model helpers (PTX acquire/release at GPU scope)
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ int32_t ld_acquire(const int32_t *p) {
    int32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_acquire_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ int32_t ld_relaxed(const int32_t *p) {
    int32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint32_t ld_relaxed_u32(const uint32_t *p) {
    uint32_t v;
    asm volatile("ld.relaxed.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_u32(uint32_t *p, uint32_t v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void st_release(int32_t *p, int32_t v) {
    asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}
__device__ __forceinline__ uint32_t smid() {
    uint32_t s;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(s));
    return s;
}

// Records the first error of the launch.
__device__ __forceinline__ void raise_status(Control *ctrl, int32_t code) {
    atomicCAS(&ctrl->status, VC_OK, code);
}

// Debug builds (-DVC_DEBUG_CHECKS) check indices on the traversal's paths and, instead of making a
// bad access, record the first failing site and value and raise VC_EINVAL.
#ifdef VC_DEBUG_CHECKS
#define VC_CHECK(ctrl, cond, site, value, on_fail)                                  \
    do {                                                                            \
        if (!(cond)) {                                                              \
            if ((ctrl) && atomicCAS(&(ctrl)->dbg_site, 0, (site)) == 0)             \
                (ctrl)->dbg_value = (int32_t)(value);                               \
            if (ctrl) raise_status((ctrl), VC_EINVAL);                              \
            on_fail;                                                                \
        }                                                                           \
    } while (0)
#else
#define VC_CHECK(ctrl, cond, site, value, on_fail) \
    do {                                           \
    } while (0)
#endif

// Maximum of 64-bit keys across a warp (two 32-bit warp reductions).
__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long k) {
    uint32_t hi = (uint32_t)(k >> 32), lo = (uint32_t)k;
    uint32_t mhi = __reduce_max_sync(kFull, hi);
    uint32_t mlo = __reduce_max_sync(kFull, hi == mhi ? lo : 0u);
    return ((unsigned long long)mhi << 32) | mlo;
}

// ------------------------------------------------------------------------------------------------
// The problem a worker is currently working on (uniform across the block).
// ------------------------------------------------------------------------------------------------
struct Ctx {
    const int32_t *off;  // n+1 offsets of this graph (global, or the worker's shared-memory copy)
    const int32_t *adj;  // its neighbours
    Problem *prob;
    int32_t *cover;      // its cover mask (n entries)
    int32_t n;
    int32_t kind;
    int32_t k;
    int32_t index;
};

// The problem record's constants are read through L2 (.cg): a serving launch receives records
// written by the host while it runs, which no L1 may hold stale.
__device__ __forceinline__ Ctx make_ctx(const Params &P, int32_t p) {
    Ctx c;
    Problem *pr = P.problems + p;
    c.off = P.offsets + __ldcg(&pr->off_base);
    c.adj = P.neighbors + __ldcg(&pr->adj_base);
    c.prob = pr;
    c.cover = P.cover + __ldcg(&pr->cover_base);
    c.n = __ldcg(&pr->n);
    c.kind = __ldcg(&pr->kind);
    c.k = __ldcg(&pr->k);
    c.index = p;
    return c;
}

// Per-worker statistics, kept in shared memory (sc words 8..39) so they cost no registers.
enum TallySlot : int {
    kTNodes = 0,
    kTPushes,
    kTPops,
    kTDonations,
    kTDequeues,
    kTPasses,
    kTCsr,
    kTMaxDepth,
    kTWaitNs,     // VC_TRACE: time spent waiting for work (worklist, roots, idle)
    kTReduceNs,   // VC_TRACE: reduction rules and stop check
    kTBranchNs,   // VC_TRACE: argmax, donate / push, child construction
    kTSolutionNs, // VC_TRACE: solution capture
    kTIdlePolls,  // VC_TRACE: idle-loop iterations
    kTallySlots
};
constexpr int kScTally = 8;  // first scratch word of the tally (8-byte aligned, 16 slots)
static_assert(kScTally + 2 * kTallySlots <= 40, "tally overlaps the argmax keys");

// Finer breakdown in VC_TRACE builds: SM cycles (clock64) of thread 0 per activity, plus pass
// counts, accumulated in scratch words kScProf.. and summed over workers at the end.
enum ProfSlot {
    kPHeader = 0,  // per-node snapshot of best / found / status
    kPDeg1,        // degree-one pass scans (incl. their closing vote)
    kPTri,         // degree-two-triangle pass scans
    kPHigh,        // high-degree pass scans
    kPApply,       // removals applied by rule passes
    kPStop,        // |S| and m > t^2 checks
    kPArgmax,      // argmax
    kPStore,       // donate (reserve + entry copy + publish) or push
    kPTakeV,       // the "v" child: v into S
    kPPop,         // local stack pop (entry copy)
    kPTakeN,       // lazily stored N(v) child applied by its taker
    kPAcquire,     // roots and worklist (incl. idle waiting)
    kPSolution,    // solution capture
    kPDeg1Count,   // number of degree-one passes
    kPTriCount,    // number of degree-two-triangle passes
    kPHighCount,   // number of high-degree passes
    kProfSlots
};
constexpr int kScProf = 80;  // 16 u64 after the argmax keys (at most 16 warps)
static_assert(kScProf + 2 * kProfSlots <= kScratchWords, "profile slots exceed the scratch words");

// VC_TRACE builds time the activities of Sec. V-D (thread 0 of each worker, %globaltimer).
#ifdef VC_TRACE
#define VC_CYC() clock64()
#define VC_CYC_ADD(w, slot, t0)                                                      \
    do {                                                                             \
        if ((w).tid == 0) (w).prof()[slot] += (unsigned long long)(clock64() - (t0)); \
    } while (0)
#define VC_CYC_INC(w, slot)                       \
    do {                                          \
        if ((w).tid == 0) (w).prof()[slot] += 1; \
    } while (0)
#else
#define VC_CYC() 0ll
#define VC_CYC_ADD(w, slot, t0) \
    do {                        \
        (void)(t0);             \
    } while (0)
#define VC_CYC_INC(w, slot) \
    do {                    \
    } while (0)
#endif

#ifdef VC_TRACE
#define VC_TRACE_NOW() globaltimer_ns()
#define VC_TRACE_ADD(w, slot, t0)                                         \
    do {                                                                  \
        if ((w).tid == 0) (w).tally[slot] += globaltimer_ns() - (t0);    \
    } while (0)
#else
#define VC_TRACE_NOW() 0ull
#define VC_TRACE_ADD(w, slot, t0) \
    do {                          \
        (void)(t0);               \
    } while (0)
#endif

// NW-word bit rows as one vector load / store (two 16-byte halves for 8 words).
template <int NW> struct RowVec;
template <> struct RowVec<1> {
    using type = uint32_t;
    static __device__ __forceinline__ type pack(const uint32_t (&b)[1]) { return b[0]; }
    static __device__ __forceinline__ void unpack(type q, uint32_t (&b)[1]) { b[0] = q; }
    static __device__ __forceinline__ type load_cg(const type *p) { return __ldcg(p); }
    static __device__ __forceinline__ void store_cg(type *p, type q) { __stcg(p, q); }
};
template <> struct RowVec<2> {
    using type = uint2;
    static __device__ __forceinline__ type pack(const uint32_t (&b)[2]) { return make_uint2(b[0], b[1]); }
    static __device__ __forceinline__ void unpack(type q, uint32_t (&b)[2]) {
        b[0] = q.x;
        b[1] = q.y;
    }
    static __device__ __forceinline__ type load_cg(const type *p) { return __ldcg(p); }
    static __device__ __forceinline__ void store_cg(type *p, type q) { __stcg(p, q); }
};
template <> struct RowVec<4> {
    using type = uint4;
    static __device__ __forceinline__ type pack(const uint32_t (&b)[4]) { return make_uint4(b[0], b[1], b[2], b[3]); }
    static __device__ __forceinline__ void unpack(type q, uint32_t (&b)[4]) {
        b[0] = q.x;
        b[1] = q.y;
        b[2] = q.z;
        b[3] = q.w;
    }
    static __device__ __forceinline__ type load_cg(const type *p) { return __ldcg(p); }
    static __device__ __forceinline__ void store_cg(type *p, type q) { __stcg(p, q); }
};
struct alignas(16) Row8 {
    uint4 lo, hi;
};
template <> struct RowVec<8> {
    using type = Row8;
    static __device__ __forceinline__ type pack(const uint32_t (&b)[8]) {
        return Row8{make_uint4(b[0], b[1], b[2], b[3]), make_uint4(b[4], b[5], b[6], b[7])};
    }
    static __device__ __forceinline__ void unpack(const type &q, uint32_t (&b)[8]) {
        b[0] = q.lo.x;
        b[1] = q.lo.y;
        b[2] = q.lo.z;
        b[3] = q.lo.w;
        b[4] = q.hi.x;
        b[5] = q.hi.y;
        b[6] = q.hi.z;
        b[7] = q.hi.w;
    }
    static __device__ __forceinline__ type load_cg(const type *p) { return Row8{__ldcg(&p->lo), __ldcg(&p->hi)}; }
    static __device__ __forceinline__ void store_cg(type *p, const type &q) {
        __stcg(&p->lo, q.lo);
        __stcg(&p->hi, q.hi);
    }
};

// ------------------------------------------------------------------------------------------------
// Worker
// ------------------------------------------------------------------------------------------------
// GM = false: the node lives in shared memory.  GM = true: the degree array, marks, dirty bits and
// removal list live in a global-memory region of this worker (the header and scratch stay in
// shared memory); their reads go through L2 (.cg) because the atomics that change them act there.
//
// The kernels use a worker through this interface (shared with RowWorker, vc_rows.cuh): node
// accessors (node_S, node_m, node_branch, node_problem), loading and storing (load_root,
// load_entry, node_loaded, store_entry, load_plain, save_plain), the rule passes, apply,
// size_exceeded and must_stop, argmax, the two branches (take_vertex, take_neighbourhood) and
// write_cover.
template <typename W, int WT, bool GM = false>
struct Worker {
    static constexpr int kWT = WT;
    static constexpr int kWarps = WT / 32;
    static constexpr int kRowWords = 0;  // no bit rows
    EntryHeader *hdr;
    W *d;
    uint32_t *marks;
    unsigned long long *dirty;
    int32_t *list;
    int32_t *sc;
    unsigned long long *keys;
    unsigned long long *tally;
    int32_t *csr;
    int tid, lane, warp;
    int32_t entry_bytes;
    int32_t csr_words;
    int32_t staged;  // problem whose CSR is in csr, or -1
    bool staged_full;  // the neighbour lists are staged too
    Control *dbg;    // where debug builds report failed checks (may be null)
    int32_t cur_n;   // vertices of the current graph (for the debug checks)
    int32_t n_cap;   // shared-memory capacity in vertices

    __device__ Worker(uint8_t *smem, int32_t n_max, int32_t csr_capacity = 0, uint8_t *gstate = nullptr) {
        const int32_t eb = entry_bytes_for(n_max, (int32_t)sizeof(W));
        const int32_t mark_bytes = pad16(((int64_t)n_max + 31) / 32 * 4);
        const int32_t dirty_bytes = pad16(((int64_t)n_max + 31) / 32 * 8);
        hdr = reinterpret_cast<EntryHeader *>(smem);
        if constexpr (GM) {
            uint8_t *g = gstate;
            d = reinterpret_cast<W *>(g);
            g += pad16((int64_t)n_max * sizeof(W));
            marks = reinterpret_cast<uint32_t *>(g);
            dirty = reinterpret_cast<unsigned long long *>(g + mark_bytes);
            list = reinterpret_cast<int32_t *>(g + mark_bytes + dirty_bytes);
            sc = reinterpret_cast<int32_t *>(smem + 16);
        } else {
            d = reinterpret_cast<W *>(smem + 16);
            marks = reinterpret_cast<uint32_t *>(smem + eb);
            dirty = reinterpret_cast<unsigned long long *>(smem + eb + mark_bytes);
            list = reinterpret_cast<int32_t *>(smem + eb + mark_bytes + dirty_bytes);
            sc = list + pad16((int64_t)n_max * 4) / 4;
        }
        keys = reinterpret_cast<unsigned long long *>(sc + kScKeys);
        tally = reinterpret_cast<unsigned long long *>(sc + kScTally);
        csr = sc + kScratchWords;
        csr_words = csr_capacity;
        staged = -1;
        staged_full = false;
        dbg = nullptr;
        cur_n = n_max;
        n_cap = n_max;
        // One-warp workers: tid < 32 and warp = 0 are compile-time facts for the code generator.
        tid = (WT == 32) ? (int)(threadIdx.x & 31) : (int)threadIdx.x;
        lane = tid & 31;
        warp = (WT == 32) ? 0 : tid >> 5;
        entry_bytes = eb;
    }

    __device__ __forceinline__ unsigned long long *prof() const {
        return reinterpret_cast<unsigned long long *>(sc + kScProf);
    }

    // Worker-wide barriers: a one-warp worker needs only a warp barrier (and a warp vote).
    __device__ __forceinline__ void sync() const {
        if constexpr (WT == 32) __syncwarp();
        else __syncthreads();
    }
    __device__ __forceinline__ bool sync_or(bool p) const {
        if constexpr (WT == 32) return __any_sync(kFull, p);
        else return __syncthreads_or(p);
    }

    __device__ __forceinline__ int deg(int v) const {
        if constexpr (GM) return (int)__ldcg(d + v);
        else return (int)d[v];
    }
    __device__ __forceinline__ unsigned long long ld_dirty(int i) const {
        if constexpr (GM) return __ldcg(dirty + i);
        else return dirty[i];
    }
    __device__ __forceinline__ int ld_list(int i) const {
        if constexpr (GM) return __ldcg(list + i);
        else return list[i];
    }

    // Atomic decrement of d[u] in shared memory.  For 16-bit entries the containing 32-bit word
    // is decremented in the right half; a live vertex with a removed neighbour has degree >= 1, so
    // the half never borrows from its neighbour.
    // Returns the new degree.
    __device__ __forceinline__ int dec(int u) {
        if constexpr (sizeof(W) == 4) {
            return atomicSub(reinterpret_cast<int *>(d) + u, 1) - 1;
        } else {
            int *word = reinterpret_cast<int *>(d) + (u >> 1);
            const int old = atomicSub(word, (u & 1) ? 0x10000 : 1);
            return (int)(int16_t)((u & 1) ? (old >> 16) : old) - 1;
        }
    }

    __device__ __forceinline__ bool marked(int u) const {
        const uint32_t word = GM ? __ldcg(marks + (u >> 5)) : marks[u >> 5];
        return (word >> (u & 31)) & 1u;
    }

    // Choose u for S in the current pass (once, however many proposers).
    __device__ __forceinline__ void propose(int u) {
        VC_CHECK(dbg, u >= 0 && u < cur_n, 2, u, return);
        const uint32_t bit = 1u << (u & 31);
        const uint32_t old = atomicOr(&marks[u >> 5], bit);
        if (!(old & bit)) list[atomicAdd(&sc[kScCount], 1)] = u;
    }

    // Dirty tracking.  A degree-one or degree-two-triangle pass only looks at vertices whose degree
    // changed since that pass last ran, which finds exactly the vertices a full scan would: at the
    // end of a pass every vertex it looked at that still meets its rule has been dealt with, and a
    // vertex whose degree did not change since then kept its live neighbourhood (any removed
    // neighbour lowers the degree), so it still does not meet the rule.  A change marks a vertex
    // only for the pass its new degree concerns (low bit: degree 1; high bit: degree 2): a vertex
    // of any other degree is no candidate of either pass, and reaching degree 1 or 2 later is
    // itself a change that marks it.  A root, or a state given from outside, starts with every
    // vertex dirty; a stored node is a fixpoint of the rules and starts clean, and its pending
    // removal marks the neighbours of what it removes.
    __device__ __forceinline__ void touch(int x, int nd) {
        if (nd == 1 || nd == 2) atomicOr(&dirty[x >> 5], (nd == 1 ? 1ull : 0x100000000ull) << (x & 31));
    }
    __device__ void dirty_all(int n) {
        for (int i = tid; i < (n + 31) / 32; i += WT) {
            const int rem = n - 32 * i;
            const unsigned long long m = rem >= 32 ? 0xffffffffull : ((1ull << rem) - 1ull);
            dirty[i] = m | (m << 32);
        }
    }
    __device__ void dirty_none(int n) {
        for (int i = tid; i < (n + 31) / 32; i += WT) dirty[i] = 0ull;
    }

    // Clears scratch state; call once per kernel before any pass.
    __device__ void init_scratch(int32_t n_max) {
        for (int i = tid; i < (n_max + 31) / 32; i += WT) {
            marks[i] = 0;
            dirty[i] = 0ull;
        }
        for (int i = tid; i < kScratchWords; i += WT) sc[i] = (i == kScMaxDeg) ? INT32_MAX : 0;
        sync();
    }

    // Points c at a shared-memory copy of its graph's offsets -- and of its neighbour lists too
    // when the launch reserved room for them -- copied when the problem changes.  (BUILD and
    // grows concern bit-row workers only.)
    template <bool BUILD = true>
    __device__ void stage(Ctx &c, uint32_t * = nullptr) {
        const int n1 = c.n + 1;
        const bool copy_csr = csr_words > 0 && n1 <= csr_words;
        if (!copy_csr) return;  // nothing to stage: read global memory
        if (c.index == staged) {
            if (copy_csr) {
                c.off = csr;
                if (staged_full) c.adj = csr + n1;
            }
            return;
        }
        sync();  // nobody still reads the previous copy
        bool full = false;
        if (copy_csr) {
            const int len = c.off[c.n];
            full = n1 + len <= csr_words;
            for (int i = tid; i < n1; i += WT) csr[i] = c.off[i];
            if (full)
                for (int i = tid; i < len; i += WT) csr[n1 + i] = c.adj[i];
        }
        staged = c.index;
        staged_full = full;
        sync();
        if (copy_csr) {
            c.off = csr;
            if (full) c.adj = csr + n1;
        }
    }

    // ---- node loading / storing ---------------------------------------------------------------

    // Root node of a problem (Sec. IV-A: the search starts from the whole graph): degrees from the
    // CSR, |S| = 0, m = offsets[n] / 2.
    __device__ void load_root(const Ctx &c) {
        sync();  // no warp still reads the node being replaced
        for (int v = tid; v < c.n; v += WT) d[v] = (W)(c.off[v + 1] - c.off[v]);
        dirty_all(c.n);
        if (tid == 0) sc[kScMaxDeg] = INT32_MAX;  // unknown until a high-degree pass or a recount
        if (tid == 0) {
            hdr->problem = c.index;
            hdr->S = 0;
            hdr->m = c.off[c.n] / 2;
            hdr->branch = -1;
        }
        sync();
    }

    // Copies an entry of `bytes` (header + degree array of the entry's graph) from global memory.
    // Loads go through L2 only (.cg) because the producer may be another SM.
    __device__ void load_entry(const uint8_t *src, int32_t bytes, int32_t n_max) {
        sync();  // no warp still reads the node being replaced
        const int4 *s = reinterpret_cast<const int4 *>(src);
        if constexpr (GM) {
            int4 *dg = reinterpret_cast<int4 *>(d);
            for (int i = tid; i < bytes / 16; i += WT) {
                const int4 v = __ldcg(s + i);
                if (i == 0) *reinterpret_cast<int4 *>(hdr) = v;
                else __stcg(dg + (i - 1), v);
            }
        } else {
            int4 *t = reinterpret_cast<int4 *>(hdr);
            for (int i = tid; i < bytes / 16; i += WT) t[i] = __ldcg(s + i);
        }
        dirty_none(n_max);
        if (tid == 0) sc[kScMaxDeg] = INT32_MAX;
        sync();
    }

    // Copies the current node to global memory with its header's branch field set to `branch`.
    __device__ void store_entry(uint8_t *dst, int32_t bytes, int32_t branch) {
        int4 *t = reinterpret_cast<int4 *>(dst);
        for (int i = tid; i < bytes / 16; i += WT) {
            int4 v;
            if constexpr (GM) v = i == 0 ? *reinterpret_cast<const int4 *>(hdr) : __ldcg(reinterpret_cast<const int4 *>(d) + (i - 1));
            else v = reinterpret_cast<const int4 *>(hdr)[i];
            if (i == 0) v.w = branch;
            __stcg(t + i, v);
        }
    }

    // ---- removal (Sec. IV-B) --------------------------------------------------------------------

    // Moves every vertex of the removal list into S: each listed vertex's live neighbours outside
    // the list lose one degree, m loses every edge with a listed endpoint (an edge between two
    // listed vertices once), |S| grows by the list length.  One warp per listed vertex, its lanes
    // splitting the vertex's adjacency list.  Must follow a barrier that ended the proposals.
    // (A flattened walk over all listed vertices' lists at once issues fewer dependent loads but
    // measured slower: the traversal is bound by instruction issue, not by load latency.)
    __device__ __forceinline__ void apply_list(const Ctx &c) {
        int cnt = sc[kScCount];
        VC_CHECK(dbg, cnt >= 0 && cnt <= c.n, 3, cnt, cnt = 0);
        int edges = 0, words = 0;
        for (int i = warp; i < cnt; i += kWarps) {
            const int u = ld_list(i);
            VC_CHECK(dbg, u >= 0 && u < c.n, 4, u, continue);
            const int b = c.off[u], e = c.off[u + 1];
            VC_CHECK(dbg, b >= 0 && e >= b, 15, u, continue);
            words += e - b;
            for (int j = b + lane; j < e; j += 32) {
                const int x = c.adj[j];
                VC_CHECK(dbg, x >= 0 && x < c.n, 9, x, continue);
                if (deg(x) == -1) continue;
                if (marked(x)) {
                    if (x > u) edges++;
                } else {
                    touch(x, dec(x));
                    edges++;
                }
            }
        }
        edges = __reduce_add_sync(kFull, edges);
        if (lane == 0 && edges) atomicAdd(&sc[kScEdges], edges);
        if (lane == 0 && words) atomicAdd(&tally[kTCsr], (unsigned long long)words);
        sync();
        for (int i = tid; i < cnt; i += WT) {
            const int u = ld_list(i);
            VC_CHECK(dbg, u >= 0 && u < c.n, 16, u, continue);
            d[u] = (W)-1;
            marks[u >> 5] = 0u;
        }
        if (tid == 0) {
            hdr->S += cnt;
            hdr->m -= sc[kScEdges];
            sc[kScEdges] = 0;
            sc[kScCount] = 0;
        }
        sync();
    }

    // Ends a scan: returns whether some thread proposed a vertex (the proposals wait in the
    // removal list).  (slot, t0: VC_TRACE accounting of the scan.)
    __device__ __forceinline__ bool finish_pass(bool proposed, int slot, long long t0) {
        if (tid == 0) tally[kTPasses] += 1;
        const bool any = sync_or(proposed);
        VC_CYC_ADD(*this, slot, t0);
        VC_CYC_INC(*this, slot + (kPDeg1Count - kPDeg1));
        return any;
    }

    // Whether a branch left a removal waiting (uniform; take_vertex / take_neighbourhood end with
    // a barrier).
    __device__ __forceinline__ bool has_pending() const { return sc[kScCount] != 0; }

    // Drops a pending removal (a node abandoned before its reduction).
    __device__ void discard_pending() {
        const int cnt = sc[kScCount];
        for (int i = tid; i < cnt; i += WT) marks[ld_list(i) >> 5] = 0u;
        sync();
        if (tid == 0) sc[kScCount] = 0;
        sync();
    }

    __device__ __forceinline__ void apply(const Ctx &c) {
        const long long t1 = VC_CYC();
        apply_list(c);
        VC_CYC_ADD(*this, kPApply, t1);
    }

    // ---- warp-cooperative adjacency scans --------------------------------------------------------

    // The first `want` (1 or 2) live neighbours of v in id order; the whole warp participates and
    // every lane gets the answer.  Neighbour lists are sorted, so the first live ones found in
    // chunk order are the smallest ids.
    __device__ __forceinline__ void live_neighbours(const Ctx &c, int v, int want, int &a, int &b,
                                                     int &words) const {
        a = -1;
        b = -1;
        VC_CHECK(dbg, v >= 0 && v < c.n, 17, v, return);
        const int lo = c.off[v], hi = c.off[v + 1];
        VC_CHECK(dbg, lo >= 0 && hi >= lo, 7, v, return);
        for (int j = lo; j < hi; j += 32) {
            const bool in = j + lane < hi;
            int x = in ? c.adj[j + lane] : 0;
            VC_CHECK(dbg, x >= 0 && x < c.n, 10, x, x = 0);
            unsigned live = __ballot_sync(kFull, in && deg(x) != -1);
            words += min(32, hi - j);
            while (live) {
                const int src = __ffs(live) - 1;
                live &= live - 1;
                const int y = __shfl_sync(kFull, x, src);
                if (a < 0) {
                    a = y;
                } else {
                    b = y;
                    break;
                }
            }
            if (a >= 0 && (want == 1 || b >= 0)) break;
        }
    }

    // Whether u and w are adjacent in the input graph: the warp scans the shorter sorted list.
    __device__ __forceinline__ bool adjacent(const Ctx &c, int u, int w, int &words) const {
        VC_CHECK(dbg, u >= 0 && u < c.n && w >= 0 && w < c.n, 8, u, return false);
        int lo_u = c.off[u], hi_u = c.off[u + 1];
        int lo_w = c.off[w], hi_w = c.off[w + 1];
        int lo = lo_u, hi = hi_u, target = w;
        if (hi_w - lo_w < hi_u - lo_u) {
            lo = lo_w;
            hi = hi_w;
            target = u;
        }
        for (int j = lo; j < hi; j += 32) {
            const bool in = j + lane < hi;
            const int x = in ? c.adj[j + lane] : 0x7fffffff;
            words += min(32, hi - j);
            if (__ballot_sync(kFull, x == target)) return true;
            if (__ballot_sync(kFull, x > target)) return false;
        }
        return false;
    }

    // ---- reduction rules (Sec. II-B; tie-breaks of Sec. IV-D) -----------------------------------
    // Each pass reads the degree array without changing it while it proposes, then applies all
    // proposals at once, so the outcome does not depend on thread timing.

    // Degree-one: the live neighbour u of a degree-one vertex v enters S; if u also has degree one
    // (an isolated edge) only the smaller id of the pair enters.
    __device__ bool pass_degree_one(const Ctx &c) {
        const long long t0 = VC_CYC();
        bool proposed = false;
        int words = 0;
        for (int base = warp * 32; base < c.n; base += WT) {
            const unsigned long long dw = ld_dirty(base >> 5);
            const unsigned bits = (unsigned)dw;
            if (bits == 0u) continue;
            if (lane == 0) dirty[base >> 5] = dw & 0xffffffff00000000ull;
            const int v = base + lane;
            const int dv = v < c.n ? deg(v) : -1;
            unsigned cand = __ballot_sync(kFull, dv == 1) & bits;
            while (cand) {
                const int cv = base + __ffs(cand) - 1;
                cand &= cand - 1;
                int u, unused;
                live_neighbours(c, cv, 1, u, unused, words);
                if (u < 0) continue;  // unreachable for a consistent degree array
                if (lane == 0 && !(deg(u) == 1 && u > cv)) {
                    propose(u);
                    proposed = true;
                }
            }
        }
        if (lane == 0 && words) atomicAdd(&tally[kTCsr], (unsigned long long)words);
        return finish_pass(proposed, kPDeg1, t0);
    }

    // Degree-two-triangle: if N(v) = {u, w} and uw is an edge, u and w enter S; among degree-two
    // vertices of one triangle only the smallest id applies the rule.
    __device__ bool pass_degree_two_triangle(const Ctx &c) {
        const long long t0 = VC_CYC();
        bool proposed = false;
        int words = 0;
        for (int base = warp * 32; base < c.n; base += WT) {
            const unsigned long long dw = ld_dirty(base >> 5);
            const unsigned bits = (unsigned)(dw >> 32);
            if (bits == 0u) continue;
            if (lane == 0) dirty[base >> 5] = dw & 0xffffffffull;
            const int v = base + lane;
            const int dv = v < c.n ? deg(v) : -1;
            unsigned cand = __ballot_sync(kFull, dv == 2) & bits;
            while (cand) {
                const int cv = base + __ffs(cand) - 1;
                cand &= cand - 1;
                int u, w;
                live_neighbours(c, cv, 2, u, w, words);
                if (u < 0 || w < 0) continue;  // unreachable for a consistent degree array
                if (!adjacent(c, u, w, words)) continue;
                if (lane == 0 && !((deg(u) == 2 && u < cv) || (deg(w) == 2 && w < cv))) {
                    propose(u);
                    propose(w);
                    proposed = true;
                }
            }
        }
        if (lane == 0 && words) atomicAdd(&tally[kTCsr], (unsigned long long)words);
        return finish_pass(proposed, kPTri, t0);
    }

    // High-degree: a vertex whose degree exceeds the threshold enters S.  Threshold best-|S|-1
    // for MVC, k-|S| for PVC (`bound` is best or k).  (Computing argmax keys in this scan, to
    // spare argmax() its own scan after the last pass, measured 5 % slower: every pass paid for
    // keys only the last one needs.)
    // Skipped while the bound on the largest live degree is at most the threshold.  A pass that
    // runs leaves as the new bound the largest degree it did not choose (the chosen vertices
    // leave the graph and the rest only lose degree).
    __device__ bool pass_high_degree(const Ctx &c, int32_t bound) {
        const long long t0 = VC_CYC();
        const int thr = (c.kind == kMVC) ? bound - hdr->S - 1 : bound - hdr->S;
        if (sc[kScMaxDeg] <= thr) return false;
        bool proposed = false;
        int mx = 0;
        for (int v = tid; v < c.n; v += WT) {
            const int dv = deg(v);
            if (dv != -1 && dv > thr) {
                propose(v);
                proposed = true;
            } else if (dv > mx) {
                mx = dv;
            }
        }
        mx = (int)__reduce_max_sync(kFull, (unsigned)mx);
        if (lane == 0 && mx > 0) atomicMax(&sc[kScMaxDegNext], mx);
        const bool any = finish_pass(proposed, kPHigh, t0);  // ends with a barrier
        if (tid == 0) {  // read by the next high-degree pass, after further barriers
            sc[kScMaxDeg] = sc[kScMaxDegNext];
            sc[kScMaxDegNext] = 0;
        }
        return any;
    }

    // |S| part of the stop check: MVC needs |S| < best, PVC needs |S| <= k.
    __device__ __forceinline__ bool size_exceeded(const Ctx &c, int32_t bound) const {
        return (c.kind == kMVC) ? hdr->S >= bound : hdr->S > bound;
    }

    // Stop check (Sec. II-B): prune when |S| is too large or m > t^2 with t = best-|S|-1 (MVC) or
    // k-|S| (PVC).
    __device__ __forceinline__ bool must_stop(const Ctx &c, int32_t bound) const {
        if (size_exceeded(c, bound)) return true;
        const long long t = (c.kind == kMVC) ? (long long)bound - hdr->S - 1 : (long long)bound - hdr->S;
        return (long long)hdr->m > t * t;
    }

    // Maximum-degree live vertex, lowest id on ties (Sec. II-B, IV-B), and its degree dv.
    // Key = (d+1, ~v) so removed vertices (key 0) never win; returns -1 when no vertex is live.
    __device__ int argmax(const Ctx &c, int &dv) {
        unsigned long long key = 0ull;
        for (int v = tid; v < c.n; v += WT) {
            const int dv = deg(v);
            if (dv >= 0) {
                const unsigned long long k = ((unsigned long long)(dv + 1) << 32) | (0xffffffffu - (uint32_t)v);
                key = k > key ? k : key;
            }
        }
        key = warp_max_u64(key);
        if constexpr (kWarps > 1) {
            if (lane == 0) keys[warp] = key;
            sync();
            unsigned long long k2 = lane < kWarps ? keys[lane] : 0ull;
            key = warp_max_u64(k2);
        }
        dv = (int)(key >> 32) - 1;
        return key == 0ull ? -1 : (int)(0xffffffffu - (uint32_t)key);
    }

    // Puts the single vertex v into S (the "v" child of Sec. II-B).  The removal is left pending
    // and applied by the next reduce().
    __device__ void take_vertex(const Ctx &c, int v) {
        VC_CHECK(dbg, v >= 0 && v < c.n, 5, v, return);
        if (tid == 0) propose(v);
        sync();
    }

    // Puts every live neighbour of v into S (the "N(v)" child of Sec. II-B).  The removal is left
    // pending and applied by the next reduce().
    __device__ void take_neighbourhood(const Ctx &c, int v) {
        VC_CHECK(dbg, v >= 0 && v < c.n, 6, v, return);
        const int lo = c.off[v], hi = c.off[v + 1];
        for (int j = lo + tid; j < hi; j += WT) {
            const int x = c.adj[j];
            if (deg(x) != -1) propose(x);
        }
        if (tid == 0) atomicAdd(&tally[kTCsr], (unsigned long long)(hi - lo));
        sync();
    }

    // Node accessors (the header lives in shared memory; uniform after the worker's barriers).
    __device__ __forceinline__ int32_t node_S() const { return hdr->S; }
    __device__ __forceinline__ int32_t node_m() const { return hdr->m; }
    __device__ __forceinline__ int32_t node_branch() const { return hdr->branch; }
    __device__ __forceinline__ int32_t node_problem() const { return hdr->problem; }
    __device__ __forceinline__ void clear_branch() {
        if (tid == 0) hdr->branch = -1;
    }
    __device__ __forceinline__ void node_loaded(const Ctx &) {}  // the node is complete as loaded
    __device__ __forceinline__ void flush_counts() {}            // statistics live in shared memory

    // A degree array given from outside (rule tests): every vertex dirty unless the state is a
    // fixpoint that a branch is about to change.
    __device__ void load_plain(const Ctx &c, const int32_t *deg_in, int32_t S0, int32_t m0, bool all_dirty) {
        for (int v = tid; v < c.n; v += WT) {
            if constexpr (GM) __stcg(d + v, (W)deg_in[v]);
            else d[v] = (W)deg_in[v];
        }
        if (all_dirty) dirty_all(c.n);
        if (tid == 0) {
            hdr->problem = c.index;
            hdr->S = S0;
            hdr->m = m0;
            hdr->branch = -1;
        }
        sync();
    }
    __device__ void save_plain(const Ctx &c, int32_t *deg_out) const {
        for (int v = tid; v < c.n; v += WT) deg_out[v] = deg(v);
    }

    // Writes the current node's S as a 0/1 mask.
    __device__ void write_cover(const Ctx &c) {
        for (int v = tid; v < c.n; v += WT) __stcg(c.cover + v, deg(v) == -1 ? 1 : 0);
    }
};

// Applies a pending branch removal, then the chosen rules in the order degree-one,
// degree-two-triangle, high-degree, cyclically, until every chosen rule in a row has found
// nothing.  This is the fixpoint of repeating whole rounds until a round changes nothing: a rule
// that found nothing in a state finds nothing in it again, so the passes a round-based loop would
// add after that point cannot change the state.  With early_exit, returns true as soon as |S|
// alone prunes the node (sound: |S| only grows).  The removal is applied at this one place, which
// keeps the kernel's code small.  (Any worker type: Worker or RowWorker.)
template <class Wk>
__device__ bool reduce_fixpoint(Wk &w, const Ctx &c, int32_t bound, int rules, bool early_exit) {
    const int nrules = __popc(rules & kRuleAll);
    int quiet = 0, r = 0;
    bool pend = w.has_pending();
    if (early_exit && w.size_exceeded(c, bound)) {  // best fell since the node was made
        if (pend) w.discard_pending();
        return true;
    }
    for (;;) {
        if (pend) {
            w.apply(c);
            quiet = 0;
            if (early_exit && w.size_exceeded(c, bound)) return true;
        }
        if (quiet >= nrules) return false;
        const bool on = (rules >> r) & 1;
        pend = false;
        if (on) {
            if (r == 0) pend = w.pass_degree_one(c);
            else if (r == 1) pend = w.pass_degree_two_triangle(c);
            else pend = w.pass_high_degree(c, bound);
            if (!pend) ++quiet;
        }
        r = (r == 2) ? 0 : r + 1;
    }
}

}  // namespace vc
