// Internal definitions shared by the CUDA translation units of wt_gb300.
//
// Construction is organised in rounds of at most 8 levels (the first round takes
// L mod 8 levels, the others 8; see round_first_level).  Round r works on "jobs":
// contiguous runs of symbols of one text whose remaining rb code bits are still
// to be split.  Round 0 has one job per text.  For the wavelet matrix every round
// has one job per text (the text stably re-sorted by the reversed prefix of the
// levels done, Obs. 2).  For the wavelet tree, round r >= 1 has one job per
// prefix of the levels done: the independent subtree below that prefix (Sec. 2,
// node definition), stored contiguously because the previous round wrote the text
// stably sorted by prefix (Obs. 1).
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

#include "../../include/wt_gb300.h"

namespace wtg {

constexpr int kMaxRounds = 4;         // L <= 32
constexpr int kChunk = 8;             // levels per round
constexpr int kThreads = 512;         // build / histogram block size
constexpr int kWarps = kThreads / 32;
constexpr int kRowsPerBlock = 64;     // groups per block of the segmented scan
constexpr int kCols = 256;            // histogram columns (2^8 classes per round)
constexpr int kMaxTreeSigmaLog = 24;  // WT alphabets up to 2^24
constexpr int kTileSyms = 32768;      // symbols per tile of the bit-sliced build; groups are multiples

// RoundArgs::kind besides WT_TREE / WT_MATRIX: the WT and the WM of the same
// texts in one pass (texts with L <= 8 and more than kSmallJob symbols).  Within a
// tile both are the same stable splits (WM order); only the intervals' places
// in the levels differ, so every class run is written twice.
constexpr uint32_t kBoth = 2;
constexpr uint32_t kSmallJob = 4096;  // jobs of the last round up to this size: one warp each

// Default symbols per build block: four tiles (a block finishes the words that its
// tiles' runs share, so fewer blocks means fewer words updated in place).
constexpr uint32_t kDefaultGroup = 4 * 32768;

// Round geometry.  A text of L levels is built in ceil(L / 8) rounds; the first
// takes the L mod 8 top levels (8 when L is a multiple of 8) and every later round
// 8, so that the last round, where the wavelet tree has one job per subtree, has
// the fewest and largest subtrees.
__host__ __device__ inline uint32_t round_count(uint32_t L) { return (L + kChunk - 1) / kChunk; }
__host__ __device__ inline uint32_t first_round_levels(uint32_t L) { return L ? (L - 1) % kChunk + 1 : 0; }
__host__ __device__ inline uint32_t round_first_level(uint32_t L, uint32_t r)
{
    return r ? first_round_levels(L) + kChunk * (r - 1) : 0;
}
__host__ __device__ inline uint32_t round_levels(uint32_t L, uint32_t r)
{
    return r ? kChunk : first_round_levels(L);
}

// Smallest storage width (bytes) that holds b-bit codes.
__host__ __device__ inline uint32_t width_for_bits(uint32_t b) { return b <= 8 ? 1u : (b <= 16 ? 2u : 4u); }

struct TextInfo {
    const void *text;        // caller's symbols (round 0 input)
    void *buf[2];            // re-sorted symbols: round r writes buf[r & 1]
    uint64_t *bv;            // L * W words (the WT's when kind == kBoth)
    uint64_t *bv2;           // kBoth: the WM's L * W words
    uint64_t *zeros;         // WM (and kBoth): L values
    uint32_t *perm;          // optional: text position of every symbol in the order after the last level
    uint32_t *pbuf[2];       // perm: text positions in the re-sorted order, round r writes pbuf[r & 1]
    uint64_t n;
    uint64_t W;
    uint64_t sigma;
    uint32_t L;
    uint32_t in_w;
    uint32_t slot_base[kMaxRounds];   // first job slot of this text in round r
    uint32_t nslots[kMaxRounds];      // job slots of this text in round r (0: not taking part)
};

struct Job {
    uint32_t n;              // symbols of this job
    uint32_t off;            // first symbol inside the text's round buffer == first bit inside its levels
    uint32_t text;
    uint32_t g0;             // first group (build block) of this job in the round
    uint32_t ng;             // groups of this job
    uint32_t tile0;          // first row of this job in the tile histograms (kTileSyms symbols per row)
};

struct Ctl {
    uint32_t status;                      // first device-detected error (wt_status)
    uint32_t total_groups[kMaxRounds];
    uint32_t pad[11];
};

struct RoundArgs {
    Ctl *ctl;
    const TextInfo *texts;
    Job *jobs;               // this round's slots
    const Job *pjobs;        // previous round's slots (WT children)
    uint32_t *jobhist;       // [slots][256]: class totals of each job
    const uint32_t *pjobhist;
    uint32_t *ghist;         // [groups][256]: class counts of each group
    uint32_t *gexcl;         // [groups][256]: count of the class in earlier groups of the job
    uint32_t *thist;         // [tiles][256]: class counts of every kTileSyms symbols of a job
    uint32_t *btail;         // [blocks][256]: segmented-scan block summaries
    uint32_t *bflag;         // [blocks]
    uint32_t *bcarry;        // [blocks][256]
    uint32_t ntexts;
    uint32_t nslots;         // slots in this round
    uint32_t pnslots;        // slots in the previous round
    uint32_t round;
    uint32_t kind;           // WT_TREE / WT_MATRIX / kBoth
    uint32_t gelems;         // symbols per group in this round
    uint32_t groups_ub;      // grid bound for per-group kernels
    uint32_t blocks_ub;      // grid bound for per-block kernels
    uint32_t any_cut;        // some job of the round writes a re-sorted text
    uint32_t any_plain;      // some job of the round has no cut (its text's last round)
    uint32_t any_order;      // some text of the round wants its stable order (perm)
    uint32_t any_small;      // some job of the round may be small (one warp each)
    uint32_t all_h8;         // every job of the round splits 8 levels
    uint32_t *cscan;         // [2 * chunks]: group and tile totals per 4096 slots (many-slot rounds)
};

// sorted[j] = text[perm[j]] for j < n (symbols of width w).
cudaError_t launch_gather(const void *text, uint32_t w, const uint32_t *perm, uint64_t n, void *sorted,
                          cudaStream_t s);

// sorted for a text built in one round (L <= 8) from its class totals: count[c]
// copies of c, runs in id order (WT) or reversed-code order (WM).
cudaError_t launch_fill_runs(const uint32_t *count, uint32_t L, bool matrix, uint64_t n, void *sorted, uint32_t w,
                             cudaStream_t s);

// counts[c] += number of symbols with low 8 bits c (zeroed by the caller).
cudaError_t launch_class_counts(const void *text, uint32_t w, uint64_t n, uint32_t *counts, cudaStream_t s);

// A one-round build (L <= 8) of one text that also leaves its 256 class totals in
// d_counts (device).  Used by the builds of texts of any length.
wt_status build_with_counts(wt_kind kind, const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma,
                            uint64_t *d_bv, uint64_t *d_zeros, void *d_ws, size_t ws_bytes, uint32_t *d_counts,
                            cudaStream_t s);

// perm[j] = j and sorted = text (texts with a single symbol value, L = 0).
cudaError_t launch_identity_order(const void *text, uint32_t w, uint64_t n, uint32_t *perm, void *sorted,
                                  cudaStream_t s);

// Launches one round on the stream; in_w: the widest symbol (bytes) the round reads.
// Returns a CUDA error code.
cudaError_t launch_round(const RoundArgs &a, uint32_t in_w, cudaStream_t s);

// Device pass that marks every text's Z as zero (WM) before round 0.
cudaError_t launch_zero_z(const TextInfo *texts, uint32_t ntexts, cudaStream_t s);

cudaError_t configure_kernels();

// Diagnostics: events around kernel families (see wt_profile in the header).
void profile_mark(int family, bool begin, cudaStream_t s, uint32_t launches = 0);
bool profile_on();

}  // namespace wtg
