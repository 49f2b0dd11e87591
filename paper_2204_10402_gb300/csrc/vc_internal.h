// vc_internal.h - layouts shared by the host side and the kernels of libvc.
//
// One launch solves one or more independent problems (graphs).  A problem is MVC or PVC(k).
// Device memory of a launch (all owned by the library's cached workspace):
//
//   CSR          packed offsets / neighbours of every problem (read-only, one copy, Sec. IV-B)
//   Problem[G]   per-problem constants and mutable search state (best, found flag, work units)
//   Control      launch-wide status word, termination counter, worklist tickets, statistics
//   cover        Σ n_g int32 0/1 masks: the best cover found so far per problem
//   stacks       workers x depth x entry_bytes: one local stack per worker (Sec. IV-A, IV-E)
//   worklist     capacity x entry_bytes slots + capacity sequence words (Sec. IV-A, IV-C)
//
// An entry (stack or worklist) is a 16-byte header followed by the degree array of the problem,
// padded to a multiple of 16 bytes:
//   header { problem index, |S|, m, pending branch vertex }
// The pending branch vertex makes the entry a lazily built child: an entry with branch = v >= 0
// stands for its degree array with every live neighbour of v moved into S (the "N(v)" child of
// Sec. II-B); the worker that takes the entry applies that removal first.  branch = -1 means the
// degree array is the node itself.
#pragma once

#include <stdint.h>

#include "../../include/vc.h"

namespace vc {

enum ProblemKind : int32_t { kMVC = 0, kPVC = 1 };
enum RuleBits : int32_t { kRuleDeg1 = 1, kRuleDeg2Tri = 2, kRuleHigh = 4, kRuleAll = 7 };

struct alignas(16) EntryHeader {
    int32_t problem;  // index into the Problem table
    int32_t S;        // |S|
    int32_t m;        // edges of G - S
    int32_t branch;   // pending N(branch) removal, or -1
};

// One record per problem, each on its own 128-byte line: records of different problems never
// share a line (no false sharing between their atomics, no stale neighbours in a serving launch).
struct alignas(128) Problem {
    // constants, written by the host
    int64_t off_base;    // first offset of this graph in the packed offsets array
    int64_t adj_base;    // first neighbour of this graph in the packed neighbour array
    int64_t cover_base;  // first entry of this graph's cover mask
    int32_t n;           // vertices
    int32_t m;           // edges
    int32_t kind;        // kMVC or kPVC
    int32_t k;           // PVC parameter
    // search state, written by the kernels
    int32_t best;        // MVC: size of the best cover found so far (greedy bound first)
    int32_t found;       // PVC: 1 once a cover of size <= k was found
    int32_t cover_size;  // size of the cover currently held in the cover mask
    int32_t lock;        // cover-capture lock (0 free, 1 held)
    int32_t greedy;      // greedy upper bound
    int32_t units;       // work units alive: unclaimed root + worklist entries + workers holding work
    int32_t done;        // 1 once the last unit was released
    int32_t tag;         // serving: completion tag the host waits for (0 otherwise)
    int64_t root_base;   // byte offset of this problem's root entry in Params::roots
    int64_t t_done_ns;   // %globaltimer when the problem was answered (0 until then)
};

// Launch-wide control block.  Words that many workers hit with atomics or polls each own a
// 128-byte line, so traffic on one never queues behind traffic on another.
struct alignas(128) Control {
    alignas(128) int32_t wl_count;     // published worklist entries no consumer has reserved yet
    alignas(128) int32_t wl_space;     // free worklist slots (initialised to the capacity)
    alignas(128) uint32_t wl_head;     // consumer tickets
    alignas(128) uint32_t wl_tail;     // producer tickets
    alignas(128) int32_t units_total;  // Σ units over problems; 0 means the whole launch is finished
    alignas(128) uint32_t heartbeat;   // bumped by busy workers; idle workers time out only while it stands still
    alignas(128) int32_t next_root;    // next problem whose root node has not been claimed
    alignas(128) int32_t status;       // VC_OK, or the first error code raised by any worker
    int32_t num_problems;
    int32_t max_depth;
    uint64_t t_launch_ns;  // %globaltimer at the greedy kernel's start (the reference of Problem::t_done_ns)
    int32_t dbg_site;     // debug builds (VC_DEBUG_CHECKS): first failed bounds check ...
    int32_t dbg_value;    // ... and the offending value
    unsigned long long nodes;
    unsigned long long stack_pushes;
    unsigned long long stack_pops;
    unsigned long long donations;
    unsigned long long worklist_pops;
    unsigned long long rule_passes;
    unsigned long long csr_words;
    unsigned long long trace_ns[4];  // VC_TRACE builds: ns waiting for work, reducing, branching, solutions
    unsigned long long idle_polls;   // VC_TRACE builds: idle-loop iterations
    unsigned long long trace_cycles[16];  // VC_TRACE builds: SM cycles per activity (ProfSlot)
};

// Kernel arguments (passed by value).
struct Params {
    const int32_t *offsets;
    const int32_t *neighbors;
    Problem *problems;
    int32_t num_problems;
    int32_t n_max;           // largest n of the launch (sizes the degree-array buffers)
    int32_t entry_bytes;     // 16 + degree-array bytes padded to 16
    int32_t stack_depth;     // entries per local stack
    Control *ctrl;
    int32_t *cover;          // Σ n cover masks
    uint8_t *stacks;         // workers x stack_depth x entry_bytes
    uint8_t *wl_slots;       // wl_capacity x entry_bytes
    uint32_t *wl_seq;        // wl_capacity sequence words
    int32_t wl_capacity;
    int32_t wl_threshold;    // donate while fewer than this many entries wait in the worklist
    int32_t csr_words;       // shared-memory CSR staging capacity in int32 words (0 = read the CSR from global)
    uint8_t *gstate;         // global-memory node state, gstate_bytes per worker (global-state kernels)
    int32_t gstate_bytes;
    uint32_t *rows;          // bit-row kernels: NW words per vertex, at cover_base * NW per problem
                             // (written by the greedy pass); null = each worker builds its own
    uint8_t *roots;          // one entry (entry_bytes) per problem at its root_base: the root node
                             // reduced by the greedy pass's first fixpoint; null = roots from the CSR
    int64_t idle_timeout_ns;
    const volatile int32_t *cancel;
    unsigned long long *sm_nodes;  // per-SM node counters
    // Serving (a persistent launch that takes requests while it runs); all zero otherwise.
    int32_t serving;
    uint32_t sub_mask;               // submission ring capacity - 1 (a power of two)
    const uint32_t *sub_ring;        // slot indices of admitted requests, written by the host's copies
    const uint32_t *sub_tail;        // number of published submissions
    unsigned long long *claim_state; // bit 32: the launch is closing; low 32 bits: requests claimed
    const int32_t *close_now;        // nonzero: idle workers close the launch at once
    int32_t *completion;             // host-mapped, 4 ints per slot: {tag, answer, status, greedy}
    int64_t linger_ns;               // idle time after which an empty launch closes
};

// Debug single-node reduction arguments.
struct ReduceParams {
    const int32_t *offsets;
    const int32_t *neighbors;
    int32_t n;
    int32_t problem;  // kMVC / kPVC
    int32_t bound;    // best (MVC) or k (PVC)
    int32_t rules;
    int32_t branch;   // -1: reduce as given; v >= 0: put v into S first; -2-v: put N(v) into S first
    int32_t *deg;     // n entries, in/out (device)
    int32_t *io;      // [0] = S, [1] = m, [2] = pruned (out)
    uint8_t *gstate;  // global-state kernels: one worker's node state
};

#ifdef __CUDACC__
#define VC_HD __host__ __device__
#else
#define VC_HD
#endif

// Shared-memory bytes one worker needs for a launch whose largest graph has n_max vertices.
VC_HD inline int32_t pad16(int64_t b) { return (int32_t)((b + 15) & ~int64_t(15)); }
VC_HD inline int32_t entry_bytes_for(int32_t n_max, int32_t width_bytes) {
    return 16 + pad16((int64_t)n_max * width_bytes);
}
// Scratch after the entry: marks bitmask, dirty bitmasks, removal list, counters and reduction
// slots, then an optional copy of the current graph's CSR (offsets followed by neighbours).
constexpr int kScratchWords = 112;
// Per-SM node counters are indexed by %smid modulo this power of two.
constexpr int kSmSlots = 1024;
// Bit-row workers (nw > 0 words per row) hold the node in registers and keep only the scratch
// words, each vertex's input degree (a byte) and the bit rows; they stage no CSR.
VC_HD inline int32_t smem_bytes_for(int32_t n_max, int32_t width_bytes, int32_t csr_words = 0, int32_t nw = 0) {
    if (nw > 0) return kScratchWords * 4 + pad16(n_max) + pad16((int64_t)n_max * nw * 4);
    int64_t b = entry_bytes_for(n_max, width_bytes);
    b += pad16(((int64_t)n_max + 31) / 32 * 4);  // marks
    b += pad16((int64_t)n_max * 4);             // removal list
    b += pad16(((int64_t)n_max + 31) / 32 * 8);  // dirty bits (two per vertex)
    b += kScratchWords * 4;
    b += pad16((int64_t)csr_words * 4);         // staged CSR
    return (int32_t)b;
}

// Global-state variant (Sec. IV-E: the paper's kernel version that keeps the current intermediate
// graph in global memory): shared memory keeps only the 16-byte header, the scratch words and any
// staged CSR; the degree array, marks, dirty bits and removal list live in a per-worker region.
VC_HD inline int32_t smem_bytes_gm(int32_t csr_words) {
    return 16 + kScratchWords * 4 + pad16((int64_t)csr_words * 4);
}
VC_HD inline int32_t gstate_bytes_for(int32_t n_max, int32_t width_bytes) {
    int64_t b = pad16((int64_t)n_max * width_bytes);
    b += pad16(((int64_t)n_max + 31) / 32 * 4);
    b += pad16(((int64_t)n_max + 31) / 32 * 8);
    b += pad16((int64_t)n_max * 4);
    return (int32_t)b;
}

}  // namespace vc
