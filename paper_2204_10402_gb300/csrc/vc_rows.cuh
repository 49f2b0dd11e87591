// vc_rows.cuh - the bit-row worker: one warp per worker, graphs of at most 32*NW vertices
// (NW = 1, 2, 4 or 8 words per adjacency row), the current tree node held in registers.
//
// The node is the paper's degree array (Sec. IV-B): stack and worklist entries are the same
// 16-byte header + degree array as for the CSR-walk worker.  While a worker expands a node, lane l
// keeps the degrees of its vertices l, l+32, ..., l+32(NW-1) in registers, and the warp keeps
// uniform bit masks over all vertices:
//   live    vertices not in S
//   pend    vertices chosen to enter S and not yet removed (a pass's proposals, a branch)
// Each lane also keeps one bit per own vertex (bit k: vertex 32k + l) marking a degree change since
// the last degree-two-triangle pass; kept per lane instead of as NW uniform words, it frees NW - 1
// registers (with it, 24 instead of 20 eight-word workers per SM ran the planted clique n = 200
// 3 % faster).
// The read-only adjacency is staged in shared memory as one NW-word bit row per vertex, with each
// vertex's input degree beside it.  Rule scans, removals and the argmax are lane-parallel bit
// operations closed by warp votes and reductions: no degree array in shared memory, no atomics.
//
// The rounds, tie-breaks (Sec. IV-D) and resulting degree arrays are exactly those of the CSR-walk
// worker and of the oracle (vc_reduce_node compares them entry by entry).
//
// Shared memory: [sc: kScratchWords int32][deg0: n_max bytes, padded to 16][rows: n_max x NW words]
#pragma once

#include "vc_device.cuh"

namespace vc {

template <typename W, int NW>
struct RowWorker {
    static_assert(NW == 1 || NW == 2 || NW == 4 || NW == 8, "bit rows of 1, 2, 4 or 8 words");
    static constexpr int kWT = 32;
    static constexpr int kWarps = 1;
    static constexpr int kRowWords = NW;
    using V = typename RowVec<NW>::type;

    int32_t *sc;
    unsigned long long *tally;
    uint8_t *deg0;   // input degree of each vertex of the staged graph (n <= 256)
    uint32_t *rows;  // adjacency bit rows of the staged graph, NW words per vertex
    // ---- the node ----
    int32_t dg[NW];        // degree of vertex 32k + lane; -1 once in S (and beyond n)
    uint32_t live[NW];     // uniform
    uint32_t pend[NW];     // uniform
    uint32_t dl;           // per lane: bit k set when vertex 32k + lane changed since the last triangle pass
    int32_t S, m, branch, problem;
    int32_t maxdeg;        // an upper bound on the largest live degree (degrees only fall)
    // ---- statistics since the last flush into the shared tallies ----
    uint32_t passes;       // rule passes (uniform)
    uint32_t words;        // this lane's share of the adjacency-list words of removed vertices
    int tid, lane, warp;
    int32_t staged;        // problem whose rows are staged, or -1
    int32_t n_cap;         // vertices per entry (the launch's n_max)
    int32_t cur_n;
    Control *dbg;

    __device__ RowWorker(uint8_t *smem, int32_t n_max, int32_t = 0, uint8_t * = nullptr) {
        sc = reinterpret_cast<int32_t *>(smem);
        tally = reinterpret_cast<unsigned long long *>(sc + kScTally);
        deg0 = smem + kScratchWords * 4;
        rows = reinterpret_cast<uint32_t *>(deg0 + pad16(n_max));
        tid = lane = (int)(threadIdx.x & 31);
        warp = 0;
        staged = -1;
        n_cap = n_max;
        cur_n = n_max;
        dbg = nullptr;
        passes = 0u;
        words = 0u;
        S = m = 0;
        branch = -1;
        problem = 0;
        maxdeg = 0;
        dl = 0u;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            dg[k] = -1;
            live[k] = pend[k] = 0u;
        }
    }

    __device__ __forceinline__ unsigned long long *prof() const {
        return reinterpret_cast<unsigned long long *>(sc + kScProf);
    }
    __device__ __forceinline__ void sync() const { __syncwarp(); }
    __device__ __forceinline__ bool sync_or(bool p) const { return __any_sync(kFull, p); }

    __device__ void init_scratch(int32_t) {
        for (int i = lane; i < kScratchWords; i += 32) sc[i] = 0;
        __syncwarp();
    }

    // Adds the statistics kept in registers to the shared tallies.
    __device__ void flush_counts() {
        const unsigned wsum = __reduce_add_sync(kFull, words);
        if (lane == 0) {
            tally[kTPasses] += passes;
            tally[kTCsr] += wsum;
        }
        passes = 0u;
        words = 0u;
        __syncwarp();
    }

    __device__ __forceinline__ int32_t node_S() const { return S; }
    __device__ __forceinline__ int32_t node_m() const { return m; }
    __device__ __forceinline__ int32_t node_branch() const { return branch; }
    __device__ __forceinline__ int32_t node_problem() const { return problem; }
    __device__ __forceinline__ void clear_branch() { branch = -1; }

    __device__ __forceinline__ void row(int v, uint32_t (&b)[NW]) const {
        RowVec<NW>::unpack(reinterpret_cast<const V *>(rows)[v], b);
    }

    // Copies (BUILD = false: from `grows`, where the greedy pass left them) or builds from the CSR
    // (BUILD = true; also written to `grows` when given) the bit rows of c's graph, with each
    // vertex's input degree, when the worker's problem changes.
    template <bool BUILD = true>
    __device__ void stage(Ctx &c, uint32_t *grows = nullptr) {
        if (c.index == staged) return;
        __syncwarp();  // nobody still reads the previous graph's rows
        V *r = reinterpret_cast<V *>(rows);
        if constexpr (!BUILD) {
            if (!grows) {  // the host always gives bit-row traversals their rows
                if (lane == 0 && dbg) raise_status(dbg, VC_EINVAL);
                for (int v = lane; v < c.n; v += 32) {
                    r[v] = V{};
                    deg0[v] = 0;
                }
            } else {
                const V *g = reinterpret_cast<const V *>(grows);
                for (int v = lane; v < c.n; v += 32) {
                    const V q = RowVec<NW>::load_cg(g + v);
                    uint32_t b[NW];
                    RowVec<NW>::unpack(q, b);
                    int d = 0;
#pragma unroll
                    for (int w = 0; w < NW; ++w) d += __popc(b[w]);
                    r[v] = q;
                    deg0[v] = (uint8_t)d;
                }
            }
        } else {
            for (int v = lane; v < c.n; v += 32) {
                uint32_t b[NW];
#pragma unroll
                for (int w = 0; w < NW; ++w) b[w] = 0u;
                const int lo = c.off[v], hi = c.off[v + 1];
                for (int j = lo; j < hi; ++j) {
                    const int x = c.adj[j];
                    VC_CHECK(dbg, x >= 0 && x < 32 * NW, 21, x, continue);
#pragma unroll
                    for (int w = 0; w < NW; ++w) b[w] |= ((x >> 5) == w) ? (1u << (x & 31)) : 0u;
                }
                const V q = RowVec<NW>::pack(b);
                r[v] = q;
                deg0[v] = (uint8_t)(hi - lo);
                if (grows) RowVec<NW>::store_cg(reinterpret_cast<V *>(grows) + v, q);
            }
        }
        staged = c.index;
        __syncwarp();
    }

    // ---- node loading / storing ---------------------------------------------------------------

    // Live mask and degree bound of a node whose degrees were just loaded.  Every node holds -1 at
    // the vertices beyond its graph's n: roots and plain states are loaded so, and entries are
    // written from such nodes.
    __device__ void node_loaded(const Ctx &c) {
        int mx = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            live[k] = __ballot_sync(kFull, dg[k] >= 0);
            mx = max(mx, dg[k]);
        }
        maxdeg = (int)__reduce_max_sync(kFull, (unsigned)mx);
        cur_n = c.n;
    }

    // Root node of a problem (Sec. IV-A): degrees from the CSR, |S| = 0, m = offsets[n] / 2;
    // every vertex is looked at by the first triangle pass.
    __device__ void load_root(const Ctx &c) {
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int v = 32 * k + lane;
            dg[k] = v < c.n ? c.off[v + 1] - c.off[v] : -1;
            pend[k] = 0u;
        }
        S = 0;
        m = c.off[c.n] / 2;
        branch = -1;
        problem = c.index;
        node_loaded(c);
        dl = 0u;
#pragma unroll
        for (int k = 0; k < NW; ++k) dl |= (uint32_t)(dg[k] >= 0) << k;
    }

    // An entry from a stack or the worklist (loads through L2: the producer may be another SM).
    // A stored node is a fixpoint of the rules, so nothing is dirty; its pending N(v) removal
    // (header branch) marks what it changes.
    __device__ void load_entry(const uint8_t *src, int32_t, int32_t) {
        const int4 h = __ldcg(reinterpret_cast<const int4 *>(src));
        problem = h.x;
        S = h.y;
        m = h.z;
        branch = h.w;
        const W *s = reinterpret_cast<const W *>(src + 16);
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int v = 32 * k + lane;
            dg[k] = v < n_cap ? (int)__ldcg(s + v) : -1;
            pend[k] = 0u;
        }
        dl = 0u;
    }

    // Writes the node as an entry whose header's branch field is `br`.
    __device__ void store_entry(uint8_t *dst, int32_t, int32_t br) {
        if (lane == 0) __stcg(reinterpret_cast<int4 *>(dst), make_int4(problem, S, m, br));
        W *d = reinterpret_cast<W *>(dst + 16);
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int v = 32 * k + lane;
            if (v < n_cap) __stcg(d + v, (W)dg[k]);
        }
    }

    // A degree array given from outside (rule tests): every vertex dirty unless the state is a
    // fixpoint that a branch is about to change.
    __device__ void load_plain(const Ctx &c, const int32_t *deg, int32_t S0, int32_t m0, bool all_dirty) {
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int v = 32 * k + lane;
            dg[k] = v < c.n ? deg[v] : -1;
            pend[k] = 0u;
        }
        S = S0;
        m = m0;
        branch = -1;
        problem = c.index;
        node_loaded(c);
        dl = 0u;
#pragma unroll
        for (int k = 0; k < NW; ++k) dl |= (uint32_t)(all_dirty && dg[k] >= 0) << k;
    }
    __device__ void save_plain(const Ctx &c, int32_t *deg) const {
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int v = 32 * k + lane;
            if (v < c.n) deg[v] = dg[k];
        }
    }

    // ---- removal (Sec. IV-B) --------------------------------------------------------------------

    __device__ __forceinline__ bool has_pending() const {
        uint32_t any = 0u;
#pragma unroll
        for (int k = 0; k < NW; ++k) any |= pend[k];
        return any != 0u;
    }
    __device__ __forceinline__ void discard_pending() {
#pragma unroll
        for (int k = 0; k < NW; ++k) pend[k] = 0u;
    }

    // Moves the chosen set into S.  One chosen vertex u (most single rule removals): u's live
    // neighbours lose one degree each and m loses deg(u); the degree bound still holds.  Several: every live vertex outside the set recounts its degree as
    // popc(row & live'), m = (sum of live degrees) / 2 and the degree bound is recomputed.  Every
    // vertex whose degree changed becomes dirty.  (Removing two or three chosen vertices one row at
    // a time instead of recounting measured 2-4 % slower on the batch.)
    __device__ void apply(const Ctx &c) {
        const long long t1 = VC_CYC();
        uint32_t nl[NW];
        int cnt = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            nl[k] = live[k] & ~pend[k];
            cnt += __popc(pend[k]);
        }
        if (cnt == 1) {
            int u = 0;
#pragma unroll
            for (int w = NW - 1; w >= 0; --w)
                if (pend[w]) u = 32 * w + __ffs(pend[w]) - 1;
            uint32_t r[NW];
            row(u, r);
            int du = 0;
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                const uint32_t hit = r[k] & nl[k];
                const bool mine = (pend[k] >> lane) & 1u;
                const uint32_t b = (hit >> lane) & 1u;
                dg[k] = mine ? -1 : dg[k] - (int)b;
                dl |= b << k;
                du += __popc(hit);
                live[k] = nl[k];
                pend[k] = 0u;
            }
            if (lane == 0) words += deg0[u];
            m -= du;
            S += 1;
            VC_CYC_ADD(*this, kPApply, t1);
            return;
        }
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            bool changed = false;
            if (dg[k] >= 0 && !((pend[k] >> lane) & 1u)) {
                uint32_t r[NW];
                row(32 * k + lane, r);
                int nd = 0;
#pragma unroll
                for (int w = 0; w < NW; ++w) nd += __popc(r[w] & nl[w]);
                changed = nd != dg[k];
                dg[k] = nd;
            }
            dl |= (uint32_t)changed << k;
        }
        int sum = 0, mx = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            if ((pend[k] >> lane) & 1u) {
                words += deg0[32 * k + lane];
                dg[k] = -1;
            }
            sum += max(dg[k], 0);
            mx = max(mx, dg[k]);
            live[k] = nl[k];
            pend[k] = 0u;
        }
        m = (int)(__reduce_add_sync(kFull, (unsigned)sum) >> 1);
        maxdeg = (int)__reduce_max_sync(kFull, (unsigned)mx);
        S += cnt;
        VC_CYC_ADD(*this, kPApply, t1);
    }

    // ---- reduction rules (Sec. II-B; tie-breaks of Sec. IV-D) -----------------------------------
    // A pass only reads the node while it decides; its choices become `pend` (a warp OR of every
    // lane's proposals), applied together by the caller.

    __device__ __forceinline__ bool finish(const uint32_t (&prop)[NW], int slot, long long t0) {
        uint32_t any = 0u;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            pend[w] = __reduce_or_sync(kFull, prop[w]);
            any |= pend[w];
        }
        VC_CYC_ADD(*this, slot, t0);
        return any != 0u;
    }

    // Degree-one: the live neighbour u of a degree-one vertex v enters S (the lowest bit of
    // row(v) & live); if u also has degree one (an isolated edge) only the smaller id enters.
    // Every degree-one vertex is a candidate.  (The CSR-walk worker looks only at vertices that
    // reached degree one since its last degree-one pass; those are all of them, because such a
    // pass leaves no vertex of degree one behind: each one's neighbour, or the vertex itself,
    // enters S.)
    __device__ bool pass_degree_one(const Ctx &) {
        const long long t0 = VC_CYC();
        uint32_t d1[NW], any = 0u;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            d1[k] = __ballot_sync(kFull, dg[k] == 1);
            any |= d1[k];
        }
        ++passes;
        VC_CYC_INC(*this, kPDeg1Count);
        if (any == 0u) {  // nothing to look at: pend stays empty
            VC_CYC_ADD(*this, kPDeg1, t0);
            return false;
        }
        uint32_t prop[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) prop[w] = 0u;
        if constexpr (NW >= 8) {
            // Eight-word rows: a dynamic loop over this lane's candidates (bit k: vertex 32k +
            // lane) keeps the pass's code O(NW) instead of O(NW^2).  Unrolled, the rule passes
            // missed the instruction cache (ncu: 3.1 no_instruction stalls per issue on the
            // planted clique n = 160) and the planted clique n = 200 took 975 against 842 ms;
            // for four-word rows the unrolled loop is 3 % faster on the 4096-graph batch.
            uint32_t mine = 0u;
#pragma unroll
            for (int k = 0; k < NW; ++k) mine |= ((d1[k] >> lane) & 1u) << k;
            while (mine) {
                const int k = __ffs(mine) - 1;
                mine &= mine - 1u;
                degree_one_candidate(k, d1, prop);
            }
        } else {
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                if (d1[k] == 0u) continue;
                if ((d1[k] >> lane) & 1u) degree_one_candidate(k, d1, prop);
            }
        }
        return finish(prop, kPDeg1, t0);
    }

    // Degree-one candidate 32k + lane: proposes its live neighbour unless that is a degree-one
    // vertex of smaller id.
    __device__ __forceinline__ void degree_one_candidate(int k, const uint32_t (&d1)[NW], uint32_t (&prop)[NW]) const {
        uint32_t r[NW];
        row(32 * k + lane, r);
        uint32_t nb_d1 = 0u, above = 0u;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            r[w] &= live[w];  // exactly one bit in all: u
            nb_d1 |= r[w] & d1[w];
            if (w > k) above |= r[w];
            else if (w == k) above |= r[w] & ~((2u << lane) - 1u);
        }
        if (!(nb_d1 && above))
#pragma unroll
            for (int w = 0; w < NW; ++w) prop[w] |= r[w];
    }

    // Degree-two-triangle: if N(v) = {u, x} (the two bits of row(v) & live) and ux is an edge (row(u)
    // has bit x), u and x enter S; among degree-two vertices of one triangle only the smallest id
    // applies the rule.  Candidates are the degree-two vertices whose degree changed since the last
    // such pass: a vertex whose degree did not change kept its live neighbourhood.
    __device__ bool pass_degree_two_triangle(const Ctx &) {
        const long long t0 = VC_CYC();
        uint32_t d2[NW], cand[NW], any = 0u;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            d2[k] = __ballot_sync(kFull, dg[k] == 2);
            cand[k] = __ballot_sync(kFull, dg[k] == 2 && ((dl >> k) & 1u));
            any |= cand[k];
        }
        dl = 0u;
        ++passes;
        VC_CYC_INC(*this, kPTriCount);
        if (any == 0u) {  // nothing to look at: pend stays empty
            VC_CYC_ADD(*this, kPTri, t0);
            return false;
        }
        uint32_t prop[NW];
#pragma unroll
        for (int w = 0; w < NW; ++w) prop[w] = 0u;
        if constexpr (NW >= 8) {  // one loop over this lane's candidates, as in the degree-one pass
            uint32_t mine = 0u;
#pragma unroll
            for (int k = 0; k < NW; ++k) mine |= ((cand[k] >> lane) & 1u) << k;
            while (mine) {
                const int k = __ffs(mine) - 1;
                mine &= mine - 1u;
                triangle_candidate(k, d2, prop);
            }
        } else {
#pragma unroll
            for (int k = 0; k < NW; ++k) {
                if (cand[k] == 0u) continue;
                if ((cand[k] >> lane) & 1u) triangle_candidate(k, d2, prop);
            }
        }
        return finish(prop, kPTri, t0);
    }

    // Triangle candidate 32k + lane: proposes its two live neighbours when they are adjacent and no
    // degree-two vertex of the triangle has a smaller id.
    __device__ __forceinline__ void triangle_candidate(int k, const uint32_t (&d2)[NW], uint32_t (&prop)[NW]) const {
        uint32_t r[NW];
        row(32 * k + lane, r);
        uint32_t tie = 0u;
        int u = -1;
#pragma unroll
        for (int w = 0; w < NW; ++w) {
            r[w] &= live[w];  // exactly two bits in all: u < x
            const uint32_t below = w < k ? ~0u : (w == k ? (1u << lane) - 1u : 0u);
            tie |= r[w] & d2[w] & below;
        }
#pragma unroll
        for (int w = NW - 1; w >= 0; --w)
            if (r[w]) u = 32 * w + __ffs(r[w]) - 1;
        if (!tie && u >= 0) {
            // ux is an edge iff row(u) meets {u, x} = r (u has no bit of its own): one row
            // load, no search for x (2 % faster on the batch than testing bit x of row(u))
            uint32_t ru[NW], hit = 0u;
            row(u, ru);
#pragma unroll
            for (int w = 0; w < NW; ++w) hit |= ru[w] & r[w];
            if (hit)
#pragma unroll
                for (int w = 0; w < NW; ++w) prop[w] |= r[w];
        }
    }

    // High-degree: a vertex whose degree exceeds best-|S|-1 (MVC) or k-|S| (PVC) enters S.  Skipped
    // while the degree bound is at most the threshold; a pass that runs leaves as the new bound the
    // largest degree it did not choose.
    __device__ bool pass_high_degree(const Ctx &c, int32_t bound) {
        const long long t0 = VC_CYC();
        const int thr = (c.kind == kMVC) ? bound - S - 1 : bound - S;
        if (maxdeg <= thr) return false;
        ++passes;
        VC_CYC_INC(*this, kPHighCount);
        uint32_t any = 0u;
        int mx = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const bool hi = dg[k] >= 0 && dg[k] > thr;
            pend[k] = __ballot_sync(kFull, hi);
            any |= pend[k];
            if (!hi) mx = max(mx, dg[k]);
        }
        maxdeg = (int)__reduce_max_sync(kFull, (unsigned)mx);
        VC_CYC_ADD(*this, kPHigh, t0);
        return any != 0u;
    }

    // |S| part of the stop check: MVC needs |S| < best, PVC needs |S| <= k.
    __device__ __forceinline__ bool size_exceeded(const Ctx &c, int32_t bound) const {
        return (c.kind == kMVC) ? S >= bound : S > bound;
    }

    // Stop check (Sec. II-B): prune when |S| is too large or m > t^2 with t = best-|S|-1 (MVC) or
    // k-|S| (PVC).
    __device__ __forceinline__ bool must_stop(const Ctx &c, int32_t bound) const {
        if (size_exceeded(c, bound)) return true;
        // 32-bit arithmetic: m < n^2 / 2 <= 2^15 here, so a t clamped to 2^15 decides the same.
        const int t = min((c.kind == kMVC) ? bound - S - 1 : bound - S, 1 << 15);
        return m > t * t;
    }

    // Maximum-degree live vertex, lowest id on ties (Sec. II-B, IV-B), and its degree: one warp
    // maximum over 32-bit keys (d+1) << 8 | (255 - v) (v < 256, so removed vertices, key 0, never
    // win); returns -1 when no vertex is live.
    __device__ int argmax(const Ctx &, int &dv) const {
        unsigned key = 0u;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const unsigned kk = dg[k] >= 0 ? ((unsigned)(dg[k] + 1) << 8) | (unsigned)(255 - (32 * k + lane)) : 0u;
            key = max(key, kk);
        }
        key = __reduce_max_sync(kFull, key);
        dv = (int)(key >> 8) - 1;
        return key == 0u ? -1 : 255 - (int)(key & 255u);
    }

    // The "v" child (Sec. II-B): v enters S at once, by the single-vertex removal of apply() with v
    // known (pend is empty between passes): 2 % faster on the 4096-graph batch than marking v in
    // pend for the next reduction, which had to find it there again.
    __device__ void take_vertex(const Ctx &, int v) {
        VC_CHECK(dbg, v >= 0 && v < cur_n, 5, v, return);
        uint32_t r[NW];
        row(v, r);
        const int kv = v >> 5;
        const uint32_t bv = 1u << (v & 31);
        int du = 0;
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const uint32_t hit = r[k] & live[k];  // v is not in its own row
            const uint32_t b = (hit >> lane) & 1u;
            dg[k] = (k == kv && lane == (v & 31)) ? -1 : dg[k] - (int)b;
            dl |= b << k;
            du += __popc(hit);
            if (k == kv) live[k] &= ~bv;
        }
        if (lane == 0) words += deg0[v];
        m -= du;
        S += 1;
    }

    // The "N(v)" child (Sec. II-B): every live neighbour of v enters S by the next reduction.
    __device__ void take_neighbourhood(const Ctx &, int v) {
        VC_CHECK(dbg, v >= 0 && v < cur_n, 6, v, return);
        uint32_t r[NW];
        row(v, r);
#pragma unroll
        for (int k = 0; k < NW; ++k) pend[k] = r[k] & live[k];
        if (lane == 0) words += deg0[v];
    }

    // Writes the current node's S as a 0/1 mask.
    __device__ void write_cover(const Ctx &c) const {
#pragma unroll
        for (int k = 0; k < NW; ++k) {
            const int v = 32 * k + lane;
            if (v < c.n) __stcg(c.cover + v, dg[k] == -1 ? 1 : 0);
        }
    }
};

}  // namespace vc
