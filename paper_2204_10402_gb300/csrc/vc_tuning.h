// vc_tuning.h - host-side launch policy: the built-in defaults per graph-size class (worker
// size, entry width, donation threshold, worklist capacity, bit rows, CSR staging).  Kept apart
// from the kernels' headers: changing a default changes no kernel.
#pragma once

#include "vc_internal.h"

namespace vc {

// Built-in launch defaults per graph-size class, from autotuner runs on a GB300
// (paper_2204_10402_gb300/autotune.py; coordinate descent over worker size, width, threshold,
// capacity and staging):
//   n <= 64    4096 G(n,p), n 20-64           one warp, 32-bit entries, threshold 0.25
//   n <= 128   4096 G(n,p), n 20-120          one warp, 32-bit entries, threshold 0.5 (with bit
//                                             rows; 16-bit entries were best for CSR walks)
//   n <= 400   planted-clique G(160/200, .05) one warp, 32-bit entries (1935 -> 1400 ms at n = 200
//                                             with CSR walks; up to 256 vertices the one-warp
//                                             workers use eight-word bit rows, rows_words_for)
//   n <= 1200  two warps; n <= 2560 four warps; larger: eight warps, threshold 0.25
//   worklist capacity: 512K entries for n <= 128 (169 -> 167 ms on the 20-120 batch), 256K
//   elsewhere (the 20-64 batch: 2.70 ms at 512K, 2.21 ms at 256K)
struct LaunchDefaults {
    int32_t worker_threads;
    int32_t width;
    float threshold;
    int32_t capacity;  // worklist entries, before the 1 GiB limit
};
VC_HD inline LaunchDefaults tuned_defaults(int32_t n_max) {
    if (n_max <= 64) return {32, 32, 0.25f, 262144};
    if (n_max <= 128) return {32, 32, 0.5f, 524288};
    if (n_max <= 400) return {32, 32, 0.5f, 262144};
    if (n_max <= 1200) return {64, 16, 0.5f, 262144};
    if (n_max <= 2560) return {128, 16, 0.5f, 262144};
    return {256, n_max <= 32768 ? 16 : 32, 0.25f, 262144};
}

// Default worklist capacity: the largest power of two up to `want` entries (the size class's
// tuned capacity) whose slots fit in 1 GiB (Sec. V-A tries 128K-512K entries).  Measured on the
// 4096-graph batch: CSR walks 16K entries 388 ms, 64K 348 ms, 256K 290 ms per launch; bit rows
// 64K 238 ms, 128K 197 ms, 256K 169 ms, 512K 167 ms, 1M 167 ms.
VC_HD inline int32_t default_worklist_capacity(int32_t entry_bytes, int32_t want = 262144) {
    int64_t cap = want;
    while (cap > 1024 && cap * (int64_t)entry_bytes > (int64_t(1) << 30)) cap >>= 1;
    return (int32_t)cap;
}

// Bit-row workers: words per adjacency row for graphs of at most n_max vertices (0 = none; such
// graphs use CSR walks).  Eight-word rows against CSR walks on graphs of 129-256 vertices, kernel
// times on a GB300: planted clique G(200, .05) + K_12 967 / 1279 ms, G(180, .05) + K_11 191 / 249 ms,
// G(n, p) n 150-256 1.19-1.32x faster, Chung-Lu n 180-256 1.8-1.9x, a 512-graph G(n, .01-.02)
// batch with n 129-256 31.9 / 41.0 ms.
VC_HD inline int32_t rows_words_for(int32_t n_max) {
    return n_max <= 32 ? 1 : n_max <= 64 ? 2 : n_max <= 128 ? 4 : n_max <= 256 ? 8 : 0;
}
// Shared-memory CSR staging by default: the offsets (n+1 ints) of graphs with up to
// kOffsetStageN vertices; nothing for larger graphs (their workers share the CSR through L1).
constexpr int32_t kOffsetStageN = 1024;
VC_HD inline int32_t default_csr_words(int32_t n_max, int32_t stage_csr) {
    return (stage_csr == 0 && n_max <= kOffsetStageN) ? n_max + 1 : 0;
}

}  // namespace vc
