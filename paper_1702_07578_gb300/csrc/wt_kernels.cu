// Kernels of the bottom-up prefix-counting construction (arXiv:1702.07578).
//
// Per round (at most 8 levels, see wt_internal.h) the work is:
//   k_root_jobs / k_child_jobs   job list of the round
//   k_scan_groups                groups (build blocks) per job -> first group index
//   k_hist        (a1)           class histogram of every group; symbol range check
//   k_blocksum, k_blockscan, k_groupexcl  (a3)
//                                zero-based prefix sum over groups of the same job in
//                                (class-major, group-minor) order (Alg. 2, Sec. 3.2.1);
//                                job totals
//   k_build_bs    (a2-a5)        per group of tiles: fold the histograms to every level
//                                and take the interval starts (id or bit-reversal order,
//                                Sec. 3.1 / 5.1); the tile as bit planes in shared
//                                memory; per level, a stable split of the later planes
//                                (compress to the zero and to the one positions) and a
//                                copy of each class run to its interval start; in
//                                rounds that cut, the tile stably sorted by its 8-bit
//                                class for the next round (and, when asked, the text
//                                positions in the order after the last level)
//   k_build_small (a2-a4)        the same for jobs of at most 4096 symbols, one warp each
//   k_gather / k_identity_order  the sorted text from the stable order
#include <algorithm>
#include <cstdio>

#include "wt_internal.h"

namespace wtg {

// ---------------------------------------------------------------------------
// Bounds checks, compiled in with -DWT_DEBUG_BOUNDS (the default build has
// none: WT_IN is the constant true).  WT_IN(site, i, b) holds when i < b; a
// failure counts, keeps the first site / index / bound, and the caller skips
// the access it guards.
#ifdef WT_DEBUG_BOUNDS
__device__ wt_bounds_report g_bounds;

__device__ __noinline__ bool bounds_fail(uint32_t site, uint64_t i, uint64_t b)
{
    if (atomicAdd(&g_bounds.failures, 1u) == 0u) {
        g_bounds.site = site;
        g_bounds.index = i;
        g_bounds.bound = b;
    }
    return false;
}
#define WT_IN(site, i, b) ((uint64_t)(i) < (uint64_t)(b) || bounds_fail((site), (uint64_t)(i), (uint64_t)(b)))
#else
#define WT_IN(site, i, b) true
#endif

namespace {

constexpr uint32_t kFull = 0xffffffffu;

__device__ __forceinline__ uint32_t load_sym(const void *base, uint32_t w, uint64_t i)
{
    if (w == 1) return static_cast<const uint8_t *>(base)[i];
    if (w == 2) return static_cast<const uint16_t *>(base)[i];
    return static_cast<const uint32_t *>(base)[i];
}

__device__ __forceinline__ void store_sym(void *base, uint32_t w, uint64_t i, uint32_t v)
{
    if (w == 1) static_cast<uint8_t *>(base)[i] = static_cast<uint8_t>(v);
    else if (w == 2) static_cast<uint16_t *>(base)[i] = static_cast<uint16_t>(v);
    else static_cast<uint32_t *>(base)[i] = v;
}

// pi_l(q): the l-bit reversal of q (Sec. 5).
__device__ __forceinline__ uint32_t rev_bits(uint32_t q, uint32_t l)
{
    return l ? (__brev(q) >> (32u - l)) : 0u;
}

__device__ __forceinline__ uint32_t lanemask_lt()
{
    uint32_t m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

struct RoundText {
    const void *in;   // first symbol of the text in this round's input
    uint32_t in_w;
    void *cut;        // re-sorted output of this round (nullptr in the last round)
    uint32_t cut_w;
    uint32_t rb;      // code bits still to split
    uint32_t h;       // levels in this round
    uint32_t c;       // first level of this round
};

__device__ __forceinline__ RoundText round_text(const TextInfo &t, uint32_t r)
{
    RoundText x;
    x.c = round_first_level(t.L, r);
    x.rb = t.L - x.c;
    x.h = round_levels(t.L, r);
    x.in = r == 0 ? t.text : t.buf[(r - 1) & 1];
    x.in_w = r == 0 ? t.in_w : width_for_bits(x.rb);
    x.cut = x.rb > x.h ? t.buf[r & 1] : nullptr;
    x.cut_w = width_for_bits(x.rb - x.h);
    return x;
}

// Jobs of the last round of their text with at most kSmallJob symbols are built
// by one warp each (k_build_small) and get no groups.
constexpr uint32_t kSmallWords = 4;                  // words per lane of the warp build
constexpr int kSmallWarps = 8;                        // warps per block of the 4-row instantiation
constexpr int kTinyWarps = 16;                        // warps per block of the 1-row instantiation
constexpr uint32_t kLaneJob = 256;                    // small jobs up to this size: one thread each
static_assert(kSmallJob == 32 * 32 * kSmallWords, "a small job is one warp's 32 x 32 x kSmallWords bits");

__device__ __forceinline__ bool small_job(const TextInfo &t, uint32_t round, uint64_t n)
{
    // texts that want the stable order take the block path, which ranks it
    return n > 0 && n <= kSmallJob && t.L - round_first_level(t.L, round) <= (uint32_t)kChunk && t.perm == nullptr;
}

// Lanes whose key (< 2^8) equals this lane's, among the lanes with ok set, all
// lanes taking part: one warp match (lanes without a key all carry 0xffffffff,
// which no key equals).  Measured faster than the AND of eight bit ballots.
__device__ __forceinline__ uint32_t class_peers(uint32_t key, bool ok)
{
    return __match_any_sync(kFull, ok ? key : 0xffffffffu);
}

// The slot owning group g: the last slot whose first group is <= g (slots are
// in increasing g0 order; empty slots share g0 with their successor).
__device__ __forceinline__ uint32_t find_slot(const Job *jobs, uint32_t nslots, uint32_t g)
{
    uint32_t lo = 0, hi = nslots;           // first slot with g0 > g
    while (lo < hi) {
        uint32_t mid = (lo + hi) >> 1;
        if (jobs[mid].g0 <= g) lo = mid + 1; else hi = mid;
    }
    return lo - 1;
}

// Calls f(local_index, symbol) for the symbols [i0, i1) of base, spread over the
// block; full 16-byte chunks are read with vector loads.
template <typename F>
__device__ __forceinline__ void for_range(const void *base, uint32_t w, uint64_t i0, uint64_t i1, F f)
{
    const uint8_t *b = static_cast<const uint8_t *>(base);
    uintptr_t lo = reinterpret_cast<uintptr_t>(b) + i0 * w;
    uintptr_t hi = reinterpret_cast<uintptr_t>(b) + i1 * w;
    uintptr_t alo = (lo + 15) & ~uintptr_t(15), ahi = hi & ~uintptr_t(15);
    if (alo >= ahi) {
        for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) f(uint32_t(i - i0), load_sym(base, w, i));
        return;
    }
    uint64_t head = (alo - lo) / w;          // symbols before the first full chunk
    uint64_t tail0 = (ahi - reinterpret_cast<uintptr_t>(b)) / w;   // first symbol after the last chunk
    for (uint64_t i = i0 + threadIdx.x; i < i0 + head; i += blockDim.x) f(uint32_t(i - i0), load_sym(base, w, i));
    for (uint64_t i = tail0 + threadIdx.x; i < i1; i += blockDim.x) f(uint32_t(i - i0), load_sym(base, w, i));
    const uint4 *v = reinterpret_cast<const uint4 *>(alo);
    uint64_t nchunks = (ahi - alo) >> 4;
    uint32_t per = 16u / w;
    for (uint64_t k = threadIdx.x; k < nchunks; k += blockDim.x) {
        uint4 q = __ldg(v + k);
        uint32_t words[4] = {q.x, q.y, q.z, q.w};
        uint32_t li = uint32_t(head + k * per);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            uint32_t x = words[j];
            if (w == 1) {
                f(li + 4 * j + 0, x & 0xffu);
                f(li + 4 * j + 1, (x >> 8) & 0xffu);
                f(li + 4 * j + 2, (x >> 16) & 0xffu);
                f(li + 4 * j + 3, x >> 24);
            } else if (w == 2) {
                f(li + 2 * j + 0, x & 0xffffu);
                f(li + 2 * j + 1, x >> 16);
            } else {
                f(li + j, x);
            }
        }
    }
}

// Exclusive scan of n <= 256 values by one warp: out[map(i)] = sum of
// val(map(j)) for j < i.  Each lane takes 8 consecutive positions.
template <bool FLEX, class V, class M, class O>
__device__ __forceinline__ uint32_t warp_scan_t(uint32_t n, V val, M map, O out)
{
    // element i = lane * per + k: as many elements per lane as n needs (FLEX), or
    // always 8 (fewer registers, for the kernel instantiations that are short of them)
    const uint32_t lane = threadIdx.x & 31u, per = FLEX ? (n + 31u) >> 5 : 8u;
    uint32_t loc[8];
    uint32_t sum = 0;
#pragma unroll
    for (uint32_t k = 0; k < 8; ++k) {
        if (k >= per) break;
        const uint32_t i = lane * per + k;
        loc[k] = i < n ? val(map(i)) : 0u;
        sum += loc[k];
    }
    uint32_t inc = sum;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        uint32_t y = __shfl_up_sync(kFull, inc, d);
        if (lane >= (uint32_t)d) inc += y;
    }
    uint32_t run = inc - sum;
#pragma unroll
    for (uint32_t k = 0; k < 8; ++k) {
        if (k >= per) break;
        const uint32_t i = lane * per + k;
        if (i < n) out(map(i), run);
        run += loc[k];
    }
    return __shfl_sync(kFull, inc, 31);
}

template <class V, class M, class O>
__device__ __forceinline__ uint32_t warp_scan_256(uint32_t n, V val, M map, O out)
{
    return warp_scan_t<true>(n, val, map, out);
}

}  // namespace

// ---------------------------------------------------------------------------
// job lists

__global__ void k_zero_z(const TextInfo *texts, uint32_t ntexts)
{
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= ntexts) return;
    const TextInfo &x = texts[t];
    if (x.zeros)
        for (uint32_t l = 0; l < x.L; ++l) x.zeros[l] = 0;
}

// One job per taking-part text (round 0, and every WM round).
__global__ void k_root_jobs(RoundArgs a)
{
    uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= a.ntexts) return;
    const TextInfo &x = a.texts[t];
    if (x.nslots[a.round] == 0) return;
    Job j;
    j.n = (uint32_t)x.n;
    j.off = 0;
    j.text = t;
    j.g0 = 0;
    j.ng = small_job(x, a.round, x.n) ? 0u : (uint32_t)((x.n + a.gelems - 1) / a.gelems);
    j.tile0 = 0;
    a.jobs[x.slot_base[a.round]] = j;
}

// WT round r >= 1: parent job p splits into 2^h children (h: the levels of the
// parent's round), one per class of the parent's last level; child q starts at
// the parent's start plus the zero-based prefix sum of the parent's class totals
// in id order (Sec. 3.1).
__global__ void __launch_bounds__(256) k_child_jobs(RoundArgs a)
{
    __shared__ uint32_t s[256];
    uint32_t p = blockIdx.x;
    const Job pj = a.pjobs[p];
    const TextInfo &x = a.texts[pj.text];
    if (x.nslots[a.round] == 0) return;
    uint32_t q = threadIdx.x;
    uint32_t cnt = pj.ng ? a.pjobhist[(size_t)p * kCols + q] : 0u;
    s[q] = cnt;
    __syncthreads();
    if (q < 32) {
        warp_scan_256(256, [&](uint32_t i) { return s[i]; }, [](uint32_t i) { return i; },
                      [&](uint32_t i, uint32_t v) { s[i] = v; });
    }
    __syncthreads();
    const uint32_t hp = round_levels(x.L, a.round - 1);
    if (q >= (1u << hp)) return;                      // the parent has 2^hp classes
    const uint32_t cb = x.slot_base[a.round] + ((p - x.slot_base[a.round - 1]) << hp);
    Job j;
    j.n = cnt;
    j.off = pj.off + s[q];
    j.text = pj.text;
    j.g0 = 0;
    j.ng = small_job(x, a.round, cnt) ? 0u : (cnt + a.gelems - 1) / a.gelems;
    j.tile0 = 0;
    a.jobs[cb + q] = j;
}

// Exclusive scans over all slots of the group counts -> g0 (total groups) and
// of the tile counts -> tile0, in chunks of 4096 slots (4 per thread).  One
// block walks the chunks when there are few; with many (the wavelet tree's
// rounds >= 1 of many texts) the chunks' totals are taken by one block each,
// scanned, and every chunk is then written by its own block.
constexpr uint32_t kScanChunk = 4096;
constexpr uint32_t kScanOneBlock = 4 * kScanChunk;   // up to this many slots: one block

// Scans chunk c0 .. c0 + 4095 with the carries in; writes g0 / tile0 when `write`.
// Returns the chunk's totals through tg / tt (all threads).
__device__ __forceinline__ void scan_chunk(const RoundArgs &a, uint32_t c0, uint32_t carry_g, uint32_t carry_t,
                                           bool write, uint32_t *wg, uint32_t *wt, uint32_t &tg, uint32_t &tt)
{
    const uint32_t n = a.nslots, tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    uint32_t ng[4], nt[4], sg = 0, st = 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        const uint32_t i = c0 + 4u * tid + j;
        ng[j] = i < n ? a.jobs[i].ng : 0u;
        nt[j] = i < n ? (a.jobs[i].n + kTileSyms - 1) / kTileSyms : 0u;
        sg += ng[j];
        st += nt[j];
    }
    uint32_t ig = sg, it = st;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t yg = __shfl_up_sync(kFull, ig, d), yt = __shfl_up_sync(kFull, it, d);
        if (lane >= (uint32_t)d) { ig += yg; it += yt; }
    }
    if (lane == 31) { wg[warp] = ig; wt[warp] = it; }
    __syncthreads();
    const uint32_t xg = wg[lane], xt = wt[lane];
    uint32_t pg = xg, pt = xt;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t yg = __shfl_up_sync(kFull, pg, d), yt = __shfl_up_sync(kFull, pt, d);
        if (lane >= (uint32_t)d) { pg += yg; pt += yt; }
    }
    tg = __shfl_sync(kFull, pg, 31);
    tt = __shfl_sync(kFull, pt, 31);
    if (write) {
        uint32_t rg = carry_g + __shfl_sync(kFull, pg - xg, warp) + ig - sg;
        uint32_t rt_ = carry_t + __shfl_sync(kFull, pt - xt, warp) + it - st;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const uint32_t i = c0 + 4u * tid + j;
            if (i < n) {
                a.jobs[i].g0 = rg;
                a.jobs[i].tile0 = rt_;
            }
            rg += ng[j];
            rt_ += nt[j];
        }
    }
    __syncthreads();
}

// one block: every chunk in turn (few slots); or, with many slots, the scan of the
// chunks' totals in a.cscan (exclusive, in place)
__global__ void __launch_bounds__(1024) k_scan_groups(RoundArgs a)
{
    __shared__ uint32_t wg[32], wt[32];
    const uint32_t n = a.nslots;
    uint32_t carry_g = 0, carry_t = 0;
    if (n <= kScanOneBlock) {
        for (uint32_t c0 = 0; c0 < n; c0 += kScanChunk) {
            uint32_t tg, tt;
            scan_chunk(a, c0, carry_g, carry_t, true, wg, wt, tg, tt);
            carry_g += tg;
            carry_t += tt;
        }
    } else if (threadIdx.x == 0) {
        const uint32_t chunks = (n + kScanChunk - 1) / kScanChunk;
        for (uint32_t c = 0; c < chunks; ++c) {
            const uint32_t g = a.cscan[2 * c], t = a.cscan[2 * c + 1];
            a.cscan[2 * c] = carry_g;
            a.cscan[2 * c + 1] = carry_t;
            carry_g += g;
            carry_t += t;
        }
    }
    if (threadIdx.x == 0) a.ctl->total_groups[a.round] = carry_g;
}

// many slots: chunk blockIdx.x's totals (pass 0) or its slots written (pass 1)
__global__ void __launch_bounds__(1024) k_scan_chunks(RoundArgs a, uint32_t pass)
{
    __shared__ uint32_t wg[32], wt[32];
    const uint32_t c = blockIdx.x;
    uint32_t tg, tt;
    if (pass == 0) {
        scan_chunk(a, c * kScanChunk, 0, 0, false, wg, wt, tg, tt);
        if (threadIdx.x == 0) {
            a.cscan[2 * c] = tg;
            a.cscan[2 * c + 1] = tt;
        }
    } else {
        scan_chunk(a, c * kScanChunk, a.cscan[2 * c], a.cscan[2 * c + 1], true, wg, wt, tg, tt);
    }
}

// ---------------------------------------------------------------------------
// a1: class histogram of every group (the first counting-sort phase)

// One histogram per block, shared by all its warps.  Measured on the byte
// workload: per-warp copies cost more in their per-tile reduction (every tile
// row sums all copies) and in shared memory per block than they save in
// same-class atomics, and small blocks (8 per SM) keep more loads in flight.
// Rounds whose symbols are all bytes use per-lane columns instead (LC): class q
// of lane i is word 32q + i, so the 32 atomics of a warp instruction always fall
// in 32 different banks and never on one address, whatever the skew; a tile's
// row sums the 32 columns of each class with a rotated read.  That takes 32 KB
// per block, which the passes over 2- and 4-byte symbols (fewer symbols per
// byte read) do not repay.  Warp-aggregated counting (one atomic per distinct
// class of a warp instruction, found with a warp match) was measured 15 times
// slower: the match costs far more than the atomics it saves.
constexpr int kHistThreads = 256;
constexpr size_t kHistSmem = sizeof(uint32_t) * kCols;
constexpr size_t kHistSmemLC = sizeof(uint32_t) * kCols * 32;

template <bool LC>
__global__ void __launch_bounds__(kHistThreads, LC ? 6 : 8) k_hist(RoundArgs a)
{
    extern __shared__ __align__(16) uint32_t wh[];
    const uint32_t g = blockIdx.x;
    if (g >= a.ctl->total_groups[a.round]) return;
    const uint32_t slot = find_slot(a.jobs, a.nslots, g);
    if (!WT_IN(WT_BOUNDS_TABLE, slot, a.nslots)) return;
    const Job jb = a.jobs[slot];
    if (!WT_IN(WT_BOUNDS_TABLE, jb.text, a.ntexts)) return;
    const TextInfo &t = a.texts[jb.text];
    const RoundText rt = round_text(t, a.round);
    const uint64_t g0 = (uint64_t)(g - jb.g0) * a.gelems;
    const uint64_t g1 = min((uint64_t)jb.n, g0 + a.gelems);
    if (!WT_IN(WT_BOUNDS_TEXT, (uint64_t)jb.off + g1, t.n + 1)) return;
    [[maybe_unused]] const uint32_t job_rows = jb.tile0 + (uint32_t)(((uint64_t)jb.n + kTileSyms - 1) / kTileSyms);
    const uint32_t shift = rt.rb - rt.h, mask = (1u << rt.h) - 1u;
    const bool check = a.round == 0 && t.sigma < (1ull << t.L);
    const uint32_t sig = (uint32_t)min(t.sigma, (uint64_t)0xffffffffu);
    uint32_t *mine = wh;
    const uint32_t col = LC ? threadIdx.x & 31u : 0u;   // this lane's column
    constexpr uint32_t stride = LC ? 32u : 1u;          // words per class
    bool bad = false;
    const uint8_t *base = static_cast<const uint8_t *>(rt.in) + (size_t)jb.off * rt.in_w;
    const uint32_t top = a.round == 0 && t.L < 8 ? (0xffu << t.L) & 0xffu : 0u;
    const uint32_t top4 = top * 0x01010101u;
    const uint32_t tile_first = jb.tile0 + (uint32_t)(g0 / kTileSyms);
    uint32_t gsum = 0;                                   // running group count of column threadIdx.x
    // byte rounds over all 256 classes whose symbols cannot be out of range (the
    // one round of sigma = 2^8, or an 8-level last round of a larger alphabet): the
    // class is the byte itself
    const bool fullbyte = shift == 0 && mask == 0xffu && top == 0 && !check;
    uint32_t *colp = wh + col;
    for (uint32_t i = threadIdx.x; i < (uint32_t)kCols * stride; i += kHistThreads) wh[i] = 0;
    __syncthreads();
    // one tile (kTileSyms symbols) at a time; a tile's row is the difference of
    // the running counts after and before it
    for (uint64_t i0 = g0, tix = 0; i0 < g1; i0 += kTileSyms, ++tix) {
        const uint64_t i1 = min(g1, i0 + kTileSyms);
        const uint8_t *lo = base + i0, *hi = base + i1;
        if (rt.in_w == 1 && (reinterpret_cast<uintptr_t>(lo) & 15u) == 0) {
            // bytes: whole 16-byte chunks, range checks on whole words
            const uint4 *v = reinterpret_cast<const uint4 *>(lo);
            const uint64_t nchunks = (uint64_t)(hi - lo) >> 4;
            // four 16-byte loads in flight per thread before their counts
            for (uint64_t k0 = threadIdx.x; k0 < nchunks; k0 += 4 * kHistThreads) {
                uint4 q[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const uint64_t k = k0 + (uint64_t)u * kHistThreads;
                    q[u] = k < nchunks ? __ldg(v + k) : make_uint4(0u, 0u, 0u, 0u);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    if (k0 + (uint64_t)u * kHistThreads >= nchunks) break;
                    const uint32_t words[4] = {q[u].x, q[u].y, q[u].z, q[u].w};
                    if (LC && fullbyte) {
                        // the class is the byte: one byte permute and one address per
                        // symbol (2^30 bytes: 0.286 against 0.324 ms)
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t x = words[j];
#pragma unroll
                            for (int b = 0; b < 4; ++b)
                                atomicAdd(colp + (__byte_perm(x, 0u, 0x4440u + (uint32_t)b) << 5), 1u);
                        }
                    } else {
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const uint32_t x = words[j];
                            bad |= (x & top4) != 0u;
                            if (check) bad |= __vcmpgeu4(x, sig * 0x01010101u) != 0u;
#pragma unroll
                            for (int b = 0; b < 4; ++b)
                                atomicAdd(&mine[stride * ((x >> (8 * b + shift)) & mask) + col], 1u);
                        }
                    }
                }
            }
            for (uint64_t i = i0 + nchunks * 16 + threadIdx.x; i < i1; i += kHistThreads) {
                const uint32_t x = base[i];
                bad |= (check && x >= sig) || (x & top) != 0u;
                atomicAdd(&mine[stride * ((x >> shift) & mask) + col], 1u);
            }
        } else {
            for_range(base, rt.in_w, i0, i1, [&](uint32_t, uint32_t v) {
                bad |= check && v >= sig;
                bad |= a.round == 0 && t.L < 32 && (v >> t.L) != 0;
                atomicAdd(&mine[stride * ((v >> shift) & mask) + col], 1u);
            });
        }
        __syncthreads();
        static_assert(kHistThreads == kCols, "one column per thread");
        {
            uint32_t s = 0;
            if (LC) {
#pragma unroll 8
                for (uint32_t j = 0; j < 32u; ++j) s += wh[32u * threadIdx.x + ((j + threadIdx.x) & 31u)];
            } else {
                s = wh[threadIdx.x];
            }
            if (WT_IN(WT_BOUNDS_TABLE, tile_first + tix, job_rows))
                a.thist[((size_t)tile_first + tix) * kCols + threadIdx.x] = s - gsum;
            gsum = s;
        }
        __syncthreads();
    }
    if (bad) atomicCAS(&a.ctl->status, 0u, (uint32_t)WT_ERR_SYMBOL_RANGE);
    a.ghist[(size_t)g * kCols + threadIdx.x] = gsum;
}

// ---------------------------------------------------------------------------
// a3: segmented exclusive scan of the group histograms (segments = jobs)

__global__ void __launch_bounds__(256) k_blocksum(RoundArgs a)
{
    __shared__ uint8_t first[kRowsPerBlock];
    const uint32_t total = a.ctl->total_groups[a.round];
    const uint32_t b = blockIdx.x, r0 = b * kRowsPerBlock;
    if (r0 >= total) return;
    const uint32_t rows = min((uint32_t)kRowsPerBlock, total - r0);
    if (threadIdx.x < rows) {
        uint32_t g = r0 + threadIdx.x;
        first[threadIdx.x] = a.jobs[find_slot(a.jobs, a.nslots, g)].g0 == g;
    }
    __syncthreads();
    const uint32_t col = threadIdx.x;
    uint32_t tail = 0, has = 0;
    for (uint32_t r = 0; r < rows; ++r) {
        if (first[r]) { tail = 0; has = 1; }
        tail += a.ghist[(size_t)(r0 + r) * kCols + col];
    }
    a.btail[(size_t)b * kCols + col] = tail;
    if (col == 0) a.bflag[b] = has;
}

__global__ void __launch_bounds__(256) k_blockscan(RoundArgs a)
{
    const uint32_t total = a.ctl->total_groups[a.round];
    const uint32_t nb = (total + kRowsPerBlock - 1) / kRowsPerBlock;
    const uint32_t col = threadIdx.x;
    uint32_t carry = 0;
    uint32_t b = 0;
    for (; b + 8 <= nb; b += 8) {
        uint32_t t[8], f[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            t[k] = a.btail[(size_t)(b + k) * kCols + col];
            f[k] = a.bflag[b + k];
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
            a.bcarry[(size_t)(b + k) * kCols + col] = carry;
            carry = f[k] ? t[k] : carry + t[k];
        }
    }
    for (; b < nb; ++b) {
        a.bcarry[(size_t)b * kCols + col] = carry;
        uint32_t t = a.btail[(size_t)b * kCols + col];
        carry = a.bflag[b] ? t : carry + t;
    }
}

__global__ void __launch_bounds__(256) k_groupexcl(RoundArgs a)
{
    __shared__ uint32_t slot_of[kRowsPerBlock];
    __shared__ uint8_t first[kRowsPerBlock], last[kRowsPerBlock];
    const uint32_t total = a.ctl->total_groups[a.round];
    const uint32_t b = blockIdx.x, r0 = b * kRowsPerBlock;
    if (r0 >= total) return;
    const uint32_t rows = min((uint32_t)kRowsPerBlock, total - r0);
    if (threadIdx.x < rows) {
        uint32_t g = r0 + threadIdx.x;
        uint32_t s = find_slot(a.jobs, a.nslots, g);
        const Job j = a.jobs[s];
        slot_of[threadIdx.x] = s;
        first[threadIdx.x] = j.g0 == g;
        last[threadIdx.x] = j.g0 + j.ng - 1 == g;
    }
    __syncthreads();
    const uint32_t col = threadIdx.x;
    uint32_t run = a.bcarry[(size_t)b * kCols + col];
    for (uint32_t r = 0; r < rows; ++r) {
        if (first[r]) run = 0;
        a.gexcl[(size_t)(r0 + r) * kCols + col] = run;
        run += a.ghist[(size_t)(r0 + r) * kCols + col];
        if (last[r]) a.jobhist[(size_t)slot_of[r] * kCols + col] = run;
    }
}

// ---------------------------------------------------------------------------
// a2, a4, a5: shared pieces of the build kernels

namespace {

// Heap layout of per-level class tables: entry (1 << l) + q for class q of level l.
constexpr int kHeap = 512;

// Up to 64 bits of the tile's packed level starting at bit p.
__device__ __forceinline__ uint64_t extract_bits(const uint32_t *lvl, uint32_t p, uint32_t k)
{
    uint32_t w0 = p >> 5, s = p & 31u;
    uint64_t lo = ((uint64_t)lvl[w0 + 1] << 32) | lvl[w0];
    uint64_t r = lo >> s;
    if (s) r |= (uint64_t)lvl[w0 + 2] << (64u - s);
    if (k < 64) r &= (1ull << k) - 1ull;
    return r;
}

// k (1..64) bits of a tile's level plane starting at bit p (p + k <= kBsTile; the
// plane has two spare words past its end, so the third word read stays inside).
__device__ __forceinline__ uint64_t run_bits(const uint32_t *lvl, uint32_t p, uint32_t k)
{
    const uint32_t w = p >> 5, s = p & 31u;
    const uint32_t a = lvl[w], b = lvl[w + 1], c = lvl[w + 2];
    const uint64_t r = ((uint64_t)__funnelshift_r(b, c, s) << 32) | __funnelshift_r(a, b, s);
    return k < 64 ? r & ((1ull << k) - 1ull) : r;
}

}  // namespace

// ---------------------------------------------------------------------------
// Bit-sliced variant of a2-a4 for rounds without a cut (every text with sigma
// <= 256, and the last round of larger alphabets).  The tile is held as bit
// planes: bit e of word w of plane k is bit k (counted from the most significant
// of the round's code bits) of symbol 32w + e.  Thread t owns words 2t and
// 2t + 1.  The stable split of the tile by plane l (zeros keep their order,
// then ones; Sec. 5) is, for each word, a compress of every later plane to the
// zero positions and to the one positions of plane l (Hacker's Delight,
// "compress"), placed at the word's exclusive zero count and at Z plus its
// exclusive one count.  Plane l itself, in that order, is level l.

namespace {

constexpr int kBsWords = 2 * kThreads;        // words per plane
constexpr int kBsTile = kBsWords * 32;        // 32768 symbols per tile
constexpr int kRangeBits = 64 * 32;           // positions of one warp's words (2048)
static_assert(kBsTile == kTileSyms, "tile histograms are written per kTileSyms symbols");
static_assert(kRangeBits * kWarps == kBsTile, "each warp owns one range of the tile");
static_assert(kWarps >= 2 * kChunk, "two warps per level build the tile tables");

// Destination words of one level of a tile: at most kBsTile / 64 whole words
// plus, per class, the partial words at both ends of its run.
constexpr uint32_t kWcap = kBsWords / 2 + 2 * kCols;

struct BsSmem {
    uint32_t plane[2][kChunk][kBsWords + 2];  // current / next planes (+ overflow words)
    uint64_t pend[2][kCols];                  // per level and class: bits of the group's earlier tiles in
                                              // the word the class's run goes on in (tile parity)
    uint32_t gst[kCols];                      // per level and class: the group's first bit in the level
    uint32_t wz[kChunk][kWarps];              // zeros of level l's plane in each warp's range
    uint32_t thc[kCols];                      // class counts of the tile (histogram pass)
    union {
        uint32_t cntw[kWarps][kCols];         // cut: class counts / offsets per warp chunk
        struct {                              // kBoth: the WM's wcls, jspos, glo, wpre
            uint8_t wcls2[kChunk][kWcap];
            uint32_t jspos2[kHeap];
            uint32_t glo2[kHeap];
            uint32_t wpre2[kHeap];
        };
    };
    uint8_t wcls[kChunk][kWcap];              // destination word -> class, per level
    uint32_t tP[kCols + 1];
    uint32_t offq[kCols];                     // class counts of the job before this tile
    uint32_t jP[kCols + 1];
    uint32_t oP[kCols + 1];
    uint32_t jcnt[kHeap];                     // job class totals per level
    uint32_t jspos[kHeap];                    // interval starts inside the job per level
    uint32_t cnt[kHeap];                      // tile class counts per level
    uint32_t loc[kHeap];                      // class start in tile order per level
    uint32_t glo[kHeap];                      // class start inside the text's level (bits)
    uint32_t wpre[kHeap];                     // destination words before each class
    uint32_t wtot[kChunk + 2];
    uint32_t wtot2[kChunk + 2];               // kBoth: the WM's wtot
};

// Two blocks per SM: each block's shared memory (plus the 1 KB the hardware
// reserves per block) must fit in half of the SM's 228 KB.
static_assert(sizeof(BsSmem) + 1024 <= 114 * 1024, "k_build_bs needs two blocks per SM");

// x * c as an integer multiply.  The left shifts of the move-vector computation
// are written this way so that they issue on the multiply-add pipe, which this
// kernel leaves mostly idle, instead of the integer ALU pipe that bounds it.
__device__ __forceinline__ uint32_t mul_lo(uint32_t x, uint32_t c)
{
    uint32_t r;
    asm("mul.lo.u32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(c));
    return r;
}

// x >> s (1 <= s <= 31) as the high word of x * 2^(32-s): a multiply, so that it
// issues on the multiply-add pipe instead of the integer ALU pipe.
__device__ __forceinline__ uint32_t shr_hi(uint32_t x, uint32_t s)
{
    uint32_t r;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(1u << (32 - s)));
    return r;
}

// high word of x * c
__device__ __forceinline__ uint32_t mul_hi(uint32_t x, uint32_t c)
{
    uint32_t r;
    asm("mul.hi.u32 %0, %1, %2;" : "=r"(r) : "r"(x), "r"(c));
    return r;
}

// x * c + a (low word)
__device__ __forceinline__ uint32_t mad_lo(uint32_t x, uint32_t c, uint32_t a)
{
    uint32_t r;
    asm("mad.lo.u32 %0, %1, %2, %3;" : "=r"(r) : "r"(x), "r"(c), "r"(a));
    return r;
}

// compress(x, m) (Hacker's Delight, Sec. 7-4) keeps the bits of x under the ones
// of m and packs them towards bit 0 in their order.  Here it is done inside each
// byte of a word at once, for the splits.  Three rounds move bits 1, 2 and 4
// places towards bit 0 of their byte (the moves never leave the byte: a selected
// bit moves by the number of unselected bits below it in its byte); the receive
// mask of a round holds the positions bits arrive at, and the bits that move in
// round i are those under a one of the prefix XOR of the unselected positions
// below them (after the earlier rounds).  Afterwards byte b holds its c_b
// selected bits in its low c_b bits.  A join then puts byte b's run at bit
// c_0 + .. + c_(b-1) of the word, with multiplies (below).  Per word and level
// this costs far fewer operations for the masks than the five-round compress of a
// whole word, whose move masks depend on prefix XORs across all 32 positions
// (measured: about 80 instructions against 135 per word and level).
struct ByteSplit {
    uint32_t rz[3], ro[3];      // receive masks of rounds 0..2: zeros side, ones side
    uint32_t kz, ko;            // selected bits after the rounds: the low c_b bits of each byte
    uint32_t jz[3], jo[3];      // join multipliers (byte_join)
};

// prefix XOR inside every byte, from bit 0 up
__device__ __forceinline__ uint32_t pxor8(uint32_t k)
{
    uint32_t p = k ^ (mul_lo(k, 2u) & 0xFEFEFEFEu);
    p ^= mul_lo(p, 4u) & 0xFCFCFCFCu;
    p ^= mul_lo(p, 16u) & 0xF0F0F0F0u;
    return p;
}

// Join multipliers of a kept word whose byte b holds c_b bits (keep has the low c_b
// bits of byte b set).  With M_b = 2^(c_0 + .. + c_(b-1)), byte b must be multiplied
// by M_b; written as x + (x >> 8) K1 + (x >> 16) K2 + (x >> 24) K3 this holds for
// K1 = M1 - 2^8, K2 = M2 - 2^8 M1, K3 = M3 - 2^8 M2 (all modulo 2^32).
__device__ __forceinline__ void join_consts(uint32_t keep, uint32_t j[3])
{
    const uint32_t M1 = 1u << __popc(keep & 0xFFu);
    const uint32_t M2 = 1u << __popc(keep & 0xFFFFu);
    const uint32_t M3 = 1u << __popc(keep & 0xFFFFFFu);
    j[0] = M1 - 256u;
    j[1] = mad_lo(M1, 0xFFFFFF00u, M2);
    j[2] = mad_lo(M2, 0xFFFFFF00u, M3);
}

// Byte-wise compress masks of a word for both sides (zeros of m, ones of m).
// Round 0 of the ones side reuses the zeros side's prefix XOR: inside a byte the
// two start masks differ by 0xFE and the prefix XOR is linear, so the prefix XORs
// differ by that of 0xFE, 0xAA.
__device__ __forceinline__ void byte_split(uint32_t m, ByteSplit &b)
{
    uint32_t kz = mul_lo(m, 2u) & 0xFEFEFEFEu;    // ones of m below, inside the byte
    uint32_t ko = kz ^ 0xFEFEFEFEu;               // zeros of m below, inside the byte
    uint32_t sz = ~m, so = m;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        const uint32_t pz = pxor8(kz);
        const uint32_t po = i == 0 ? pz ^ 0xAAAAAAAAu : pxor8(ko);
        const uint32_t vz = pz & sz, vo = po & so;
        const uint32_t rz = shr_hi(vz, 1u << i), ro = shr_hi(vo, 1u << i);
        sz = (sz ^ vz) | rz;
        so = (so ^ vo) | ro;
        b.rz[i] = rz;
        b.ro[i] = ro;
        if (i < 2) {
            kz &= ~pz;
            ko &= ~po;
        }
    }
    b.kz = sz;
    b.ko = so;
    join_consts(sz, b.jz);
    join_consts(so, b.jo);
}

// compress of x inside its bytes (receive masks r, kept bits keep), then the
// byte runs joined into one run from bit 0.  The rounds shift on the integer ALU,
// the join multiplies on the multiply-add pipe, so that the two pipes share the
// work of every plane split.
__device__ __forceinline__ uint32_t byte_compress(uint32_t x, const uint32_t r[3], uint32_t keep, const uint32_t j[3])
{
    x = ((x >> 1) & r[0]) | (x & ~r[0]);
    x = ((x >> 2) & r[1]) | (x & ~r[1]);
    x = ((x >> 4) & r[2]) | (x & ~r[2]);
    x &= keep;
    uint32_t y = mad_lo(shr_hi(x, 8u), j[0], x);
    y = mad_lo(shr_hi(x, 16u), j[1], y);
    return mad_lo(shr_hi(x, 24u), j[2], y);
}

// The output levels are written with global-space stores and reductions.  Through
// a generic pointer the compiler must keep each store in order with the
// shared-memory loads after it (they could alias), which stalls the copy loop.
__device__ __forceinline__ void st_out(uint64_t *p, uint64_t v)
{
    asm volatile("st.global.u64 [%0], %1;" ::"l"(__cvta_generic_to_global(p)), "l"(v));
}

// The bits `clear` of the word replaced by v's (v has no bits outside clear):
// and-not, then or, so that other blocks may update their own bits of the word
// at the same time.
__device__ __forceinline__ void red_out(uint64_t *p, uint64_t clear, uint64_t v)
{
    const size_t g = __cvta_generic_to_global(p);
    asm volatile("red.global.and.b64 [%0], %1;" ::"l"(g), "l"(~clear));
    asm volatile("red.global.or.b64 [%0], %1;" ::"l"(g), "l"(v));
}

// OR the low `len` (<= 64) bits of `part` into a plane at bit offset d.
__device__ __forceinline__ void place_bits(uint32_t *plane, uint32_t d, uint64_t part, uint32_t len)
{
    if (len == 0) return;
    const uint32_t w = d >> 5, s = d & 31u;
    const uint64_t lo = part << s;
    atomicOr(plane + w, (uint32_t)lo);
    if (s + len > 32u) atomicOr(plane + w + 1, (uint32_t)(lo >> 32));
    if (s + len > 64u) atomicOr(plane + w + 2, (uint32_t)(part >> (64u - s)));
}

// Where a thread's part of a split goes: its bit offset in the next plane, its
// length, and the multipliers that spread it over the (up to three) words it
// touches.  Shared by every plane split at one level.
struct Dest {
    uint32_t *row0;     // word of the first bit (in plane 0 of the buffer; add the plane's stride)
    uint32_t ms;        // 2^(d mod 32)
    uint32_t len;
    bool w1, w2;        // the part reaches the second / third word
};

__device__ __forceinline__ Dest make_dest(uint32_t (*buf)[kBsWords + 2], uint32_t d, uint32_t len)
{
    Dest r;
    const uint32_t s = d & 31u;
    r.row0 = &buf[0][d >> 5];
    r.ms = 1u << s;
    r.len = len;
    r.w1 = s + len > 32u;
    r.w2 = s + len > 64u;
    if (len != 0 && !WT_IN(WT_BOUNDS_SHARED, (d >> 5) + (r.w2 ? 2u : r.w1 ? 1u : 0u), kBsWords + 2)) r.len = 0;
    return r;
}

// OR the part (lo, hi: its low len bits) into plane k of the buffer.  The shift by
// d mod 32 is done with multiplies (low and high words of part * 2^s).  Storing
// the words a part covers entirely instead of or-ing them was measured slower
// (4.53 against 4.11 ms per 2^30-symbol build): the per-lane choice costs more
// than the atomics it saves.
__device__ __forceinline__ void place_part(const Dest &d, uint32_t k, uint32_t lo, uint32_t hi)
{
    if (d.len == 0) return;
    uint32_t *p = d.row0 + (size_t)k * (kBsWords + 2);
    atomicOr(p, lo * d.ms);
    if (d.w1) atomicOr(p + 1, mad_lo(hi, d.ms, mul_hi(lo, d.ms)));
    if (d.w2) atomicOr(p + 2, mul_hi(hi, d.ms));
}

// Zeros of plane bits `part` (len bits at bit offset d of the next order) counted
// into the two warp ranges the warp's run can touch: r0 (the range of the run's
// first bit) and r0 + 1.  Returns the two counts of this thread.
__device__ __forceinline__ void range_zeros(uint32_t d, uint32_t len, uint64_t part, uint32_t r0, uint32_t &a,
                                            uint32_t &b)
{
    const uint32_t r = d / kRangeBits, room = kRangeBits - d % kRangeBits;
    uint32_t za, zb = 0;
    if (len <= room) {
        za = len - __popcll(part);
    } else {                                        // room < 64: the part ends in the next range
        za = room - __popcll(part & ((1ull << room) - 1ull));
        zb = (len - room) - __popcll(part >> room);
    }
    if (len == 0) za = 0;
    if (r == r0) { a = za; b = zb; }
    else { a = 0; b = za; }
}

// 8x8 bit transpose of the bytes of (lo, hi): afterwards byte j holds bit j of
// input byte i at bit i.
__device__ __forceinline__ void transpose8(uint32_t &lo, uint32_t &hi)
{
    uint32_t t;
    t = (lo ^ (lo >> 7)) & 0x00AA00AAu; lo = lo ^ t ^ (t << 7);
    t = (hi ^ (hi >> 7)) & 0x00AA00AAu; hi = hi ^ t ^ (t << 7);
    t = (lo ^ (lo >> 14)) & 0x0000CCCCu; lo = lo ^ t ^ (t << 14);
    t = (hi ^ (hi >> 14)) & 0x0000CCCCu; hi = hi ^ t ^ (t << 14);
    t = (lo ^ (hi << 4)) & 0xF0F0F0F0u; lo = lo ^ t; hi = hi ^ (t >> 4);
}

// Symbols [e0, e0 + 32) of the tile as 8 words of 4 bytes, byte = bits
// [shift, shift + 8) of the symbol (its round's 8 top code bits, or all of them
// when it has fewer); symbols at or beyond m read as 0xff, all ones, so that
// padding stays at the end of every stable split.
__device__ __forceinline__ void load32(const uint8_t *tile, uint32_t w, uint32_t e0, uint32_t m, uint32_t shift,
                                       uint32_t x[8])
{
    const uint8_t *p = tile + (size_t)e0 * w;
    if (e0 + 32u <= m && (reinterpret_cast<uintptr_t>(p) & 15u) == 0) {
        const uint4 *q = reinterpret_cast<const uint4 *>(p);
        if (w == 1) {
            const uint4 a = __ldg(q), b = __ldg(q + 1);
            x[0] = a.x; x[1] = a.y; x[2] = a.z; x[3] = a.w;
            x[4] = b.x; x[5] = b.y; x[6] = b.z; x[7] = b.w;
        } else if (w == 2) {
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint4 a = __ldg(q + k);
                const uint32_t v[4] = {a.x, a.y, a.z, a.w};
                uint32_t lo = 0, hi = 0;
#pragma unroll
                for (int j = 0; j < 2; ++j) {
                    lo |= ((v[j] >> shift) & 0xffu) << (16 * j);
                    lo |= ((v[j] >> (16 + shift)) & 0xffu) << (16 * j + 8);
                    hi |= ((v[2 + j] >> shift) & 0xffu) << (16 * j);
                    hi |= ((v[2 + j] >> (16 + shift)) & 0xffu) << (16 * j + 8);
                }
                x[2 * k] = lo;
                x[2 * k + 1] = hi;
            }
        } else {
#pragma unroll
            for (int k = 0; k < 8; ++k) {
                const uint4 a = __ldg(q + k);
                x[k] = ((a.x >> shift) & 0xffu) | ((a.y >> shift) & 0xffu) << 8 |
                       ((a.z >> shift) & 0xffu) << 16 | ((a.w >> shift) & 0xffu) << 24;
            }
        }
        return;
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
        uint32_t word = 0;
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint32_t e = e0 + 4u * k + b;
            const uint32_t v = e < m ? ((load_sym(tile, w, e) >> shift) & 0xffu) : 0xffu;
            word |= v << (8 * b);
        }
        x[k] = word;
    }
}

// Class counts for the counting sort of rounds that cut: the h-bit class of
// symbols e0 .. e0 + 31 (bytes of x, in load32's layout; symbols at or beyond m
// are not counted) on the warp's row of counters.  Thread t loads symbols
// [64t, 64t + 64), so warp w counts exactly the symbols [2048w, 2048w + 2048) it
// ranks after the levels.
__device__ __forceinline__ void count_classes(const uint32_t x[8], uint32_t e0, uint32_t m, uint32_t h,
                                              uint32_t *row)
{
    const uint32_t cmask = (1u << h) - 1u;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
#pragma unroll
        for (int b = 0; b < 4; ++b) {
            const uint32_t q = (x[k] >> (8 * b)) & cmask;
            if (e0 + 4u * k + b < m) atomicAdd(&row[q], 1u);
        }
    }
}

// Transposes 32 symbols and stores plane k (code bit rb-1-k) of word w; returns
// plane 0's word.
__device__ __forceinline__ uint32_t store_planes(uint32_t x[8], uint32_t rb, uint32_t h,
                                                 uint32_t (*planes)[kBsWords + 2], uint32_t w)
{
#pragma unroll
    for (int b = 0; b < 4; ++b) transpose8(x[2 * b], x[2 * b + 1]);
    uint32_t first = 0;
    for (uint32_t k = 0; k < h; ++k) {
        const uint32_t j = rb - 1u - k;               // bit position inside the byte
        const uint32_t sel = (j & 3u) | ((j & 3u) + 4u) << 4;
        const bool hi = j >= 4u;
        const uint32_t t01 = __byte_perm(hi ? x[1] : x[0], hi ? x[3] : x[2], sel);
        const uint32_t t23 = __byte_perm(hi ? x[5] : x[4], hi ? x[7] : x[6], sel);
        const uint32_t v = __byte_perm(t01, t23, 0x5410);
        planes[k][w] = v;
        if (k == 0) first = v;
    }
    return first;
}

}  // namespace

// BOTH: kind kBoth (two sets of destinations).  CUT: the round runs the cut pass
// (some job cuts, or some text wants its stable order); the plain build of texts
// with sigma <= 256 is the instantiation without either.  H: the levels of every
// job of the round when that is 8 (the loops over planes then have fixed bounds),
// 0 for any number.
//
// One block barrier per level.  The zero offsets of level l need the zeros of
// plane l in every warp's range of the tile; they are counted while plane l is
// placed at level l - 1 (each warp adds its parts' zeros per destination range),
// so a level starts right after the previous level's barrier.  Level l's bits are
// copied out from plane l of the current buffer, which the level's splits leave
// untouched.
template <bool BOTH, bool CUT, int H>
__global__ void __launch_bounds__(kThreads, 2) k_build_bs(RoundArgs a)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    BsSmem &sm = *reinterpret_cast<BsSmem *>(smem_raw);

    const uint32_t g = blockIdx.x;
    if (g >= a.ctl->total_groups[a.round]) return;
    const uint32_t tid = threadIdx.x, lane = tid & 31u, warp = tid >> 5;
    const uint32_t slot = find_slot(a.jobs, a.nslots, g);
    if (!WT_IN(WT_BOUNDS_TABLE, slot, a.nslots)) return;
    const Job jb = a.jobs[slot];
    if (!WT_IN(WT_BOUNDS_TABLE, jb.text, a.ntexts)) return;
    const TextInfo &t = a.texts[jb.text];
    const RoundText rt = round_text(t, a.round);
    const uint32_t h = H ? (uint32_t)H : rt.h, rb = rt.rb;
    if (!WT_IN(WT_BOUNDS_LEVEL, rt.c + h, t.L + 1)) return;
    const uint32_t shift = rb - h;                   // > 0 in rounds with a cut
    const uint32_t gi = g - jb.g0;
    const bool matrix = a.kind == WT_MATRIX;
    constexpr bool both = BOTH;

    // job totals -> class totals and interval starts of every level (fold,
    // Alg. 1; zero-based prefix sums in id or pi_l order, Sec. 3.1 / 5.1)
    for (uint32_t q = tid; q < kCols; q += kThreads) {
        sm.cnt[q] = a.jobhist[(size_t)slot * kCols + q];      // scratch for the scan below
        sm.offq[q] = a.gexcl[(size_t)g * kCols + q];
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t tot = warp_scan_t<!CUT>(256, [&](uint32_t i) { return sm.cnt[i]; }, [](uint32_t i) { return i; },
                                     [&](uint32_t i, uint32_t v) { sm.jP[i] = v; });
        if (lane == 0) sm.jP[256] = tot;
    }
    __syncthreads();
    for (uint32_t idx = tid; idx < kHeap; idx += kThreads) {
        if (idx == 0) continue;
        const uint32_t l = 31u - __clz(idx), q = idx - (1u << l);
        if (l <= h) sm.jcnt[idx] = sm.jP[(q + 1) << (h - l)] - sm.jP[q << (h - l)];
    }
    __syncthreads();
    for (uint32_t j = warp; j < (h + 1) * (both ? 2u : 1u); j += kWarps) {
        const uint32_t l = j % (h + 1), base = 1u << l;   // j > h: the WM's starts (kBoth)
        const bool rv = matrix || j > h;
        uint32_t *dst = j > h ? sm.jspos2 : sm.jspos;
        warp_scan_t<!CUT>(base, [&](uint32_t q) { return sm.jcnt[base + q]; },
                      [&](uint32_t i) { return rv ? rev_bits(i, l) : i; },
                      [&](uint32_t q, uint32_t v) { dst[base + q] = v; });
    }
    if ((matrix || both) && gi == 0 && tid < h) {    // Z[c + l]: even (l+1)-prefixes
        const uint32_t l = tid, base = 2u << l;
        uint32_t z = 0;
        for (uint32_t p = 0; p < base; p += 2) z += sm.jcnt[base + p];
        t.zeros[rt.c + l] = z;
    }
    __syncthreads();

    const uint64_t g_begin = (uint64_t)gi * a.gelems;
    const uint64_t g_end = min((uint64_t)jb.n, g_begin + a.gelems);
    if (!WT_IN(WT_BOUNDS_TEXT, (uint64_t)jb.off + g_end, t.n + 1)) return;
    [[maybe_unused]] const uint32_t job_rows = jb.tile0 + (uint32_t)(((uint64_t)jb.n + kTileSyms - 1) / kTileSyms);
    const uint8_t *in_base = static_cast<const uint8_t *>(rt.in) + (size_t)jb.off * rt.in_w;
    const uint32_t w0 = 2u * tid;                    // this thread's words: w0, w0 + 1

    const uint32_t tile_first = jb.tile0 + (uint32_t)(g_begin / kTileSyms);
    // the tile is stably sorted by its class after the levels (the next round's text,
    // or the stable order).  In rounds of fewer than 8 levels its classes are counted
    // per warp while it is loaded; 8-level rounds count them after the levels, where
    // a second read of the tile costs less than the atomic rank updates below
    const bool cuts = CUT && (rt.cut != nullptr || t.perm != nullptr);
    const bool load_count = cuts && h < (uint32_t)kChunk;
    uint32_t tix = 0;
    for (uint64_t t0 = g_begin; t0 < g_end; t0 += kBsTile, ++tix) {
        const uint32_t m = (uint32_t)min((uint64_t)kBsTile, g_end - t0);
        // ---- class counts of the tile (from the histogram pass); clear the next-plane
        //      buffer and the zero counts of the levels after the first
        {
            uint4 *p1 = reinterpret_cast<uint4 *>(&sm.plane[1][0][0]);
            constexpr uint32_t n4 = kChunk * (kBsWords + 2) / 4;
            static_assert(kChunk * (kBsWords + 2) % 4 == 0, "plane buffer in 16-byte pieces");
            for (uint32_t i = tid; i < n4; i += kThreads) p1[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        if (tid < (uint32_t)kChunk) sm.plane[0][tid][kBsWords] = sm.plane[0][tid][kBsWords + 1] = 0;
        if (tid < (uint32_t)(kChunk * kWarps)) (&sm.wz[0][0])[tid] = 0;
        if (load_count)
            for (uint32_t i = tid; i < (uint32_t)(kWarps * kCols); i += kThreads) (&sm.cntw[0][0])[i] = 0;
        for (uint32_t q = tid; q < kCols; q += kThreads)
            sm.thc[q] = WT_IN(WT_BOUNDS_TABLE, tile_first + tix, job_rows)
                            ? a.thist[((size_t)tile_first + tix) * kCols + q] : 0u;
        __syncthreads();
        if (warp == 0) {
            uint32_t tot = warp_scan_t<!CUT>(256, [&](uint32_t i) { return sm.thc[i]; }, [](uint32_t i) { return i; },
                                         [&](uint32_t i, uint32_t v) { sm.tP[i] = v; });
            if (lane == 0) sm.tP[256] = tot;
        } else if (warp == 1) {
            uint32_t tot = warp_scan_t<!CUT>(256, [&](uint32_t i) { return sm.offq[i]; }, [](uint32_t i) { return i; },
                                         [&](uint32_t i, uint32_t v) { sm.oP[i] = v; });
            if (lane == 0) sm.oP[256] = tot;
        }
        __syncthreads();
        // every level's class counts and interval starts in the level (fold of the
        // tile counts and of the job offsets; Alg. 1 fold, Sec. 3.1)
        for (uint32_t idx = tid; idx < kHeap; idx += kThreads) {
            if (idx == 0) continue;
            const uint32_t l = 31u - __clz(idx), q = idx - (1u << l);
            if (l <= h) {
                const uint32_t s = h - l, lo = q << s, hi = (q + 1) << s;
                const uint32_t c = sm.tP[hi] - sm.tP[lo], gs = jb.off + sm.jspos[idx] + (sm.oP[hi] - sm.oP[lo]);
                sm.cnt[idx] = c;
                sm.glo[idx] = gs;
                if (both) sm.glo2[idx] = jb.off + sm.jspos2[idx] + (sm.oP[hi] - sm.oP[lo]);
                if (!both && l < h) {                    // the group's runs (see the copy below)
                    if (tix == 0) {
                        sm.gst[idx] = gs;
                        sm.pend[0][idx] = 0;
                    } else if (c == 0) {
                        const uint64_t v = sm.pend[(tix - 1) & 1][idx];
                        sm.pend[tix & 1][idx] = v;
                        // the group's last tile has no run of this class: the bits its
                        // earlier tiles left in the word gs / 64 are written now (none
                        // are left when the class's run ended on a word boundary, or
                        // at n, where the word was finished with the bits past n)
                        if (t0 + kBsTile >= g_end && (gs & 63u) != 0 && (uint64_t)gs != t.n) {
                            const uint32_t gq = sm.gst[idx];
                            const uint32_t lo = (gs >> 6) == (gq >> 6) ? (gq & 63u) : 0u;
                            const uint64_t msk = ((1ull << (gs & 63u)) - 1ull) & ~((1ull << lo) - 1ull);
                            if (msk != 0 && WT_IN(WT_BOUNDS_LEVEL, gs >> 6, t.W)) {
                                red_out(t.bv + (uint64_t)(rt.c + l) * t.W + (gs >> 6), msk, v);
                            }
                        }
                    }
                }
            }
        }
        __syncthreads();
        // the leaf counts of this tile advance the job offsets for the next tile
        // (oP, read above, is not needed again in this tile)
        for (uint32_t q = tid; q < (1u << h); q += kThreads) sm.offq[q] += sm.cnt[(1u << h) + q];
        // per level (one warp each): class starts in tile order (reversed
        // prefixes, Obs. 2) and destination words of every class
        if (CUT && warp == h && (rt.cut != nullptr || t.perm != nullptr)) {   // class starts after the last split
            const uint32_t base = 1u << h;
            warp_scan_t<!CUT>(base, [&](uint32_t q) { return sm.cnt[base + q]; },
                          [&](uint32_t i) { return rev_bits(i, h); },
                          [&](uint32_t q, uint32_t v) { sm.loc[base + q] = v; });
        }
        if (warp < h) {                             // class starts in tile order (shared by kBoth)
            const uint32_t l = warp, base = 1u << l;
            warp_scan_t<!CUT>(base, [&](uint32_t q) { return sm.cnt[base + q]; },
                          [&](uint32_t i) { return rev_bits(i, l); },
                          [&](uint32_t q, uint32_t v) { sm.loc[base + q] = v; });
        }
        // destination words: warp 8 + l for level l, so that the table work of the
        // tile start is spread over all warps (kBoth: warp l the WT's, warp h + l the WM's)
        if (both ? warp < 2 * h : (warp >= (uint32_t)kChunk && warp - (uint32_t)kChunk < h)) {
            const bool second = both && warp >= h;
            const uint32_t l = both ? (second ? warp - h : warp) : warp - (uint32_t)kChunk, base = 1u << l;
            const uint32_t *glo = second ? sm.glo2 : sm.glo;
            uint32_t *wpre = second ? sm.wpre2 : sm.wpre;
            uint32_t wt = warp_scan_t<!CUT>(
                base,
                [&](uint32_t q) {
                    const uint32_t c = sm.cnt[base + q];
                    if (c == 0) return 0u;
                    const uint32_t gs = glo[base + q];
                    return ((gs + c - 1) >> 6) - (gs >> 6) + 1u;
                },
                [](uint32_t i) { return i; }, [&](uint32_t q, uint32_t v) { wpre[base + q] = v; });
            if (!WT_IN(WT_BOUNDS_SHARED, wt, kWcap + 1)) wt = 0;      // (the level is then not copied)
            if (lane == 0) (second ? sm.wtot2 : sm.wtot)[l] = wt;
            // word -> class map of level l: every nonempty class marks its first
            // destination word, a running maximum fills the words after it
            uint8_t *wc = second ? sm.wcls2[l] : sm.wcls[l];
            for (uint32_t k = lane; k < wt; k += 32) wc[k] = 0;
            __syncwarp();
            for (uint32_t q = lane; q < base; q += 32)
                if (sm.cnt[base + q]) wc[wpre[base + q]] = (uint8_t)q;
            __syncwarp();
            const uint32_t per = (wt + 31) / 32, b0 = lane * per, b1 = min(wt, b0 + per);
            uint32_t mx = 0;
            for (uint32_t k = b0; k < b1; ++k) mx = max(mx, (uint32_t)wc[k]);
            uint32_t inc = mx;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, inc, d);
                if (lane >= (uint32_t)d) inc = max(inc, y);
            }
            uint32_t run = __shfl_up_sync(kFull, inc, 1);
            if (lane == 0) run = 0;
            for (uint32_t k = b0; k < b1; ++k) {
                run = max(run, (uint32_t)wc[k]);
                wc[k] = (uint8_t)run;
            }
        }
        // ---- the next tile of the group is fetched into L2 while this one is built
        if (tid == 0 && t0 + kBsTile < g_end) {
            const uintptr_t b = reinterpret_cast<uintptr_t>(in_base + (size_t)(t0 + kBsTile) * rt.in_w);
            const uintptr_t e = reinterpret_cast<uintptr_t>(in_base + (size_t)min(g_end, t0 + 2 * (uint64_t)kBsTile) * rt.in_w);
            const uintptr_t b16 = (b + 15) & ~uintptr_t(15), e16 = e & ~uintptr_t(15);   // inside the job's symbols
            if (e16 > b16)
                asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b16), "r"((uint32_t)(e16 - b16)) : "memory");
        }
        // ---- load and transpose: plane k holds code bit rb-1-k of every symbol;
        //      the zeros of plane 0 in this warp's range
        {
            const uint8_t *tile = in_base + (size_t)t0 * rt.in_w;
            uint32_t x[8];
            load32(tile, rt.in_w, 32u * w0, m, shift, x);
            if (load_count) count_classes(x, 32u * w0, m, h, sm.cntw[warp]);
            const uint32_t f0 = store_planes(x, h, h, sm.plane[0], w0);
            load32(tile, rt.in_w, 32u * w0 + 32u, m, shift, x);
            if (load_count) count_classes(x, 32u * w0 + 32u, m, h, sm.cntw[warp]);
            const uint32_t f1 = store_planes(x, h, h, sm.plane[0], w0 + 1);
            const uint32_t z = __reduce_add_sync(kFull, __popc(~f0) + __popc(~f1));
            if (lane == 0) sm.wz[0][warp] = z;
        }
        __syncthreads();

#pragma unroll(H == 8 ? 8 : 1)
        for (uint32_t l = 0; l < h; ++l) {
            uint32_t(*cur)[kBsWords + 2] = sm.plane[l & 1];
            uint32_t(*nxt)[kBsWords + 2] = sm.plane[(l + 1) & 1];
            const uint32_t base = 1u << l;
            // plane l in tile order is level l; zero counts of this thread's words
            const uint2 mm = *reinterpret_cast<const uint2 *>(&cur[l][w0]);
            const uint32_t m0 = mm.x, m1 = mm.y;
            const uint32_t z0 = __popc(~m0), z1 = __popc(~m1);
            uint32_t inc = z0 + z1;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, inc, d);
                if (lane >= (uint32_t)d) inc += y;
            }
            const uint32_t zl = inc - z0 - z1;             // zeros before word w0 inside the warp
            // zeros before each warp's range (counted when plane l was placed); total Z
            const uint32_t ws = lane < (uint32_t)kWarps ? sm.wz[l][lane] : 0u;
            uint32_t wex = ws;
#pragma unroll
            for (int d = 1; d < kWarps; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, wex, d);
                if (lane >= (uint32_t)d) wex += y;
            }
            const uint32_t zt = __shfl_sync(kFull, wex, kWarps - 1);
            const uint32_t zw = __shfl_sync(kFull, wex - ws, warp);   // zeros before this warp's range
            const uint32_t zo = zw + zl;

            // copy every class's bits to its interval start in level c + l (for
            // kBoth: in the WT's levels, then in the WM's).  Consecutive tiles of the
            // group put a class's runs one after the other, so a word shared by two
            // tiles' runs is finished by the later tile: the earlier one leaves its
            // bits in pend and the later one stores the whole word.  Only words shared
            // with another group's runs are updated in place (and-not, then or), the
            // bits of this group only (single output; kBoth updates every partial word
            // in place).
            const uint32_t *lvl = cur[l];
            const bool first_tile = tix == 0, last_tile = t0 + kBsTile >= g_end;
            for (uint32_t out = 0; out < (both ? 2u : 1u); ++out) {
                const uint32_t wt = out ? sm.wtot2[l] : sm.wtot[l];
                const uint8_t *wc = out ? sm.wcls2[l] : sm.wcls[l];
                const uint32_t *glo = out ? sm.glo2 : sm.glo;
                const uint32_t *wpre = out ? sm.wpre2 : sm.wpre;
                uint64_t *lv = (out ? t.bv2 : t.bv) + (uint64_t)(rt.c + l) * t.W;
                for (uint32_t k = tid; k < wt; k += kThreads) {
                    // word `rel` of the class's run; positions relative to bit 0 of
                    // that word fit in 32 bits (a run has at most kBsTile bits)
                    const uint32_t idx = base + wc[k];
                    const uint32_t gs = glo[idx], c = sm.cnt[idx];
                    const uint32_t rel = k - wpre[idx], g0 = gs & 63u;
                    const uint32_t blo = rel ? 0u : g0;
                    uint32_t bhi = min(c + g0 - 64u * rel, 64u);
                    const uint32_t src = sm.loc[idx] + 64u * rel + blo - g0;
                    const uint64_t val = WT_IN(WT_BOUNDS_SHARED, src, kBsTile) ? run_bits(lvl, src, bhi - blo) << blo : 0u;
                    const uint64_t word = (uint64_t)(gs >> 6) + rel;
                    if (!WT_IN(WT_BOUNDS_LEVEL, word, t.W)) continue;
                    if ((uint64_t)gs + c == t.n) bhi = 64;   // bits past n belong to the last interval
                    if (both) {
                        if (blo == 0 && bhi == 64) {
                            st_out(lv + word, val);
                        } else {
                            const uint64_t msk = (bhi == 64 ? ~0ull : ((1ull << bhi) - 1ull)) & ~((1ull << blo) - 1ull);
                            red_out(lv + word, msk, val);
                        }
                        continue;
                    }
                    const uint32_t gq = sm.gst[idx];
                    const bool tail = ((gs + c - 1u) >> 6) == (gs >> 6) + rel;
                    uint64_t v = val;
                    if (rel == 0 && !first_tile) v |= sm.pend[(tix - 1) & 1][idx];
                    // this group's bits in the word start at lo (> 0 only in the group's first
                    // word of the class, when an earlier group's run ends in it)
                    const uint32_t lo = word == (uint64_t)(gq >> 6) ? (gq & 63u) : 0u;
                    if (bhi < 64 && !last_tile) {
                        sm.pend[tix & 1][idx] = v;            // the next tile finishes the word
                    } else if (lo == 0 && bhi == 64) {
                        st_out(lv + word, v);
                        if (tail) sm.pend[tix & 1][idx] = 0;
                    } else {
                        const uint64_t msk = (bhi == 64 ? ~0ull : ((1ull << bhi) - 1ull)) & ~((1ull << lo) - 1ull);
                        red_out(lv + word, msk, v);
                        if (tail) sm.pend[tix & 1][idx] = 0;
                    }
                }
            }

            // stable split of every later plane by plane l
            if (l + 1 < h) {
                ByteSplit s0, s1;
                byte_split(m0, s0);
                byte_split(m1, s1);
                const uint32_t nz = z0 + z1, no = 64u - nz;
                const uint32_t dz = zo, d1 = zt + w0 * 32u - zo;
                const Dest dzs = make_dest(nxt, dz, nz), dos = make_dest(nxt, d1, no);
                // the second word's part follows the first's z0 (32 - z0) bits
                const uint32_t o0 = 32u - z0;
                const uint32_t mz = z0 < 32u ? 1u << z0 : 0u, mo = o0 < 32u ? 1u << o0 : 0u;
                // the warp's zeros run starts in range zw / kRangeBits, its ones run in
                // range (zt + 2048 warp - zw) / kRangeBits; each spans at most two ranges
                const uint32_t rz0 = zw / kRangeBits, ro0 = (zt + (uint32_t)kRangeBits * warp - zw) / kRangeBits;
                const uint32_t nk = H ? (uint32_t)H : h;
#pragma unroll
                for (uint32_t k = 1; k < (H ? (uint32_t)H : (uint32_t)kChunk); ++k) {
                    if (k <= l || k >= nk) continue;
                    const uint2 xx = *reinterpret_cast<const uint2 *>(&cur[k][w0]);
                    *reinterpret_cast<uint2 *>(&cur[k][w0]) = make_uint2(0u, 0u);
                    const uint32_t cz0 = byte_compress(xx.x, s0.rz, s0.kz, s0.jz);
                    const uint32_t cz1 = byte_compress(xx.y, s1.rz, s1.kz, s1.jz);
                    const uint32_t co0 = byte_compress(xx.x, s0.ro, s0.ko, s0.jo);
                    const uint32_t co1 = byte_compress(xx.y, s1.ro, s1.ko, s1.jo);
                    const uint32_t zlo = mad_lo(cz1, mz, cz0), zhi = z0 < 32u ? mul_hi(cz1, mz) : cz1;
                    const uint32_t olo = mad_lo(co1, mo, co0), ohi = o0 < 32u ? mul_hi(co1, mo) : co1;
                    place_part(dzs, k, zlo, zhi);
                    place_part(dos, k, olo, ohi);
                    if (k == l + 1) {                   // the next level's zeros per warp range
                        uint32_t a0, b0, a1, b1;
                        range_zeros(dz, nz, ((uint64_t)zhi << 32) | zlo, rz0, a0, b0);
                        range_zeros(d1, no, ((uint64_t)ohi << 32) | olo, ro0, a1, b1);
                        a0 = __reduce_add_sync(kFull, a0);
                        b0 = __reduce_add_sync(kFull, b0);
                        a1 = __reduce_add_sync(kFull, a1);
                        b1 = __reduce_add_sync(kFull, b1);
                        if (lane == 0) {
                            if (a0 && WT_IN(WT_BOUNDS_SHARED, rz0, kWarps)) atomicAdd(&sm.wz[k][rz0], a0);
                            if (b0 && WT_IN(WT_BOUNDS_SHARED, rz0 + 1, kWarps)) atomicAdd(&sm.wz[k][rz0 + 1], b0);
                            if (a1 && WT_IN(WT_BOUNDS_SHARED, ro0, kWarps)) atomicAdd(&sm.wz[k][ro0], a1);
                            if (b1 && WT_IN(WT_BOUNDS_SHARED, ro0 + 1, kWarps)) atomicAdd(&sm.wz[k][ro0 + 1], b1);
                        }
                    }
                }
            }
            __syncthreads();
        }
        // ---- re-sorted symbols for the next round: the tile stably sorted by its
        //      h-bit class (the counting sort of Alg. 2), each class's run written
        //      at its interval start of level h (id order for the WT, reversed for
        //      the WM, Obs. 2); only the low rb - h bits go on.  Ranks: warp w
        //      takes symbols [2048w, 2048w + 2048) in text order, equal classes
        //      within a step are ranked by lane, chunks by a scan over warps.  The
        //      values are staged in sorted order in the (now idle) plane buffers
        //      so that every class run is written with consecutive stores.
        //      When the text wants its stable order, the same ranks place every
        //      symbol's text position: in the next round's position buffer, or,
        //      in the last round, in the order after the last level.
        if (cuts) {
            constexpr uint32_t kPer = kBsTile / kWarps;
            const uint8_t *tile = in_base + (size_t)t0 * rt.in_w;
            const uint32_t low = (1u << shift) - 1u;
            const uint32_t cmask = (1u << h) - 1u;       // classes of this round (k_hist counts the same)
            const uint32_t e_end = min(m, warp * kPer + kPer);
            const uint32_t base_h = 1u << h;
            uint32_t *cw = sm.cntw[warp];
            uint8_t *stage8 = reinterpret_cast<uint8_t *>(&sm.plane[0][0][0]);
            uint16_t *stage16 = reinterpret_cast<uint16_t *>(&sm.plane[0][0][0]);
            const bool staged = rt.cut != nullptr && rt.cut_w <= 2;   // 32768 values fit the plane buffers
            // last round: the 15-bit tile offsets of the symbols are staged in sorted
            // order instead (64 KB), and every class run of positions is written with
            // consecutive stores
            const bool pstaged = t.perm != nullptr && rt.cut == nullptr;
            const uint64_t pos0 = (uint64_t)jb.off + t0;             // round-buffer position of symbol 0
            const uint32_t *pin = a.round ? t.pbuf[(a.round - 1) & 1] : nullptr;
            uint32_t *pout = t.perm == nullptr ? nullptr : (rt.cut != nullptr ? t.pbuf[a.round & 1] : t.perm);
            // symbols in chunks of 8 steps of 32: the 8 loads of a lane are issued
            // together, so a chunk waits for memory once
            constexpr uint32_t kSteps = 8;
            static_assert(kPer % (32 * kSteps) == 0, "whole chunks per warp");
            if (!load_count) {
                // 8-level rounds: the counts of each warp's symbols, read again, on
                // 32-bit counters in the second half of the plane buffers (16 warps x
                // 256 words = 16 KB, idle between the level loop and the staging)
                uint32_t *cwc = reinterpret_cast<uint32_t *>(&sm.plane[1][0][0]) + warp * kCols;
                for (uint32_t q = lane; q < kCols; q += 32) cwc[q] = 0;
                __syncwarp();
                for (uint32_t c0 = warp * kPer; c0 < e_end; c0 += 32 * kSteps) {
                    uint32_t vs[kSteps];
#pragma unroll
                    for (uint32_t k = 0; k < kSteps; ++k) {
                        const uint32_t e = c0 + 32 * k + lane;
                        vs[k] = e < e_end ? load_sym(tile, rt.in_w, e) : 0u;
                    }
#pragma unroll
                    for (uint32_t k = 0; k < kSteps; ++k)
                        if (c0 + 32 * k + lane < e_end) atomicAdd(&cwc[((vs[k] >> shift) & cmask)], 1u);
                }
                __syncwarp();
                for (uint32_t q = lane; q < kCols; q += 32) cw[q] = cwc[q];
                __syncthreads();
            }
            // per-warp class counts -> offsets of each warp's symbols among the
            // tile's symbols of the class
            for (uint32_t q = tid; q < kCols; q += kThreads) {
                uint32_t run = 0;
                for (int w = 0; w < kWarps; ++w) {
                    const uint32_t c = sm.cntw[w][q];
                    sm.cntw[w][q] = run;
                    run += c;
                }
            }
            __syncthreads();
            const uint32_t lt = lanemask_lt();
            for (uint32_t c0 = warp * kPer; c0 < e_end; c0 += 32 * kSteps) {
                uint32_t vs[kSteps];
#pragma unroll
                for (uint32_t k = 0; k < kSteps; ++k) {
                    const uint32_t e = c0 + 32 * k + lane;
                    vs[k] = e < e_end ? load_sym(tile, rt.in_w, e) : 0u;
                }
#pragma unroll
                for (uint32_t k = 0; k < kSteps; ++k) {
                    const uint32_t e = c0 + 32 * k + lane;
                    const bool ok = e < e_end;
                    const uint32_t v = vs[k];
                    const uint32_t q = ok ? (v >> shift) & cmask : 0u;
                    const uint32_t peers = class_peers(q, ok);
                    const uint32_t rank = ok ? cw[q] + __popc(peers & lt) : 0u;
                    __syncwarp();
                    if (ok) {
                        // the last lane of each class advances its counter by the class's
                        // lanes in this step.  With the counts taken at load time this is an
                        // atomic: a plain store there gave wrong ranks in the normal build
                        // (measured; cause not found), while every build with the atomic and
                        // every build counting after the levels with the plain store was right
                        if ((peers >> lane) == 1u) {
                            if (load_count) atomicAdd(&cw[q], (uint32_t)__popc(peers));
                            else cw[q] = rank + 1u;
                        }
                        const uint64_t dst = (uint64_t)sm.glo[base_h + q] + rank;
                        if (pstaged) {
                            if (WT_IN(WT_BOUNDS_SHARED, sm.loc[base_h + q] + rank, kBsTile))
                                stage16[sm.loc[base_h + q] + rank] = (uint16_t)e;
                        }
                        else if (pout != nullptr && dst < t.n)
                            pout[dst] = pin ? pin[pos0 + e] : (uint32_t)(pos0 + e);
                        if (rt.cut == nullptr) {
                        } else if (!staged) {
                            if (WT_IN(WT_BOUNDS_NEXT, dst, t.n)) store_sym(rt.cut, rt.cut_w, dst, v & low);
                        } else {
                            const uint32_t pos = sm.loc[base_h + q] + rank;   // place in the sorted tile
                            if (!WT_IN(WT_BOUNDS_SHARED, pos, kBsTile)) {
                            } else if (rt.cut_w == 1) stage8[pos] = (uint8_t)(v & low);
                            else stage16[pos] = (uint16_t)(v & low);
                        }
                    }
                    __syncwarp();
                }
            }
            __syncthreads();
            if (staged) {                               // class runs, one warp per class
                for (uint32_t q = warp; q < base_h; q += kWarps) {
                    const uint32_t c = sm.cnt[base_h + q], src = sm.loc[base_h + q];
                    const uint64_t dst = sm.glo[base_h + q];
                    for (uint32_t i = lane; i < c; i += 32)
                        if (WT_IN(WT_BOUNDS_NEXT, dst + i, t.n) && WT_IN(WT_BOUNDS_SHARED, src + i, kBsTile))
                            store_sym(rt.cut, rt.cut_w, dst + i, rt.cut_w == 1 ? stage8[src + i] : stage16[src + i]);
                }
                __syncthreads();
            }
            if (pstaged) {                              // class runs of text positions
                for (uint32_t q = warp; q < base_h; q += kWarps) {
                    const uint32_t c = sm.cnt[base_h + q], src = sm.loc[base_h + q];
                    const uint64_t dst = sm.glo[base_h + q];
                    for (uint32_t i = lane; i < c; i += 32) {
                        const uint32_t e = stage16[src + i];
                        if (dst + i < t.n) pout[dst + i] = pin ? pin[pos0 + e] : (uint32_t)(pos0 + e);
                    }
                }
                __syncthreads();
            }
        }
    }
}

// ---------------------------------------------------------------------------
// Small jobs (at most kSmallJob symbols, last round of their text): one warp
// builds a whole job with the same bit-sliced splits as k_build_bs, with no
// block-wide barrier.  Lane i owns words i, 32 + i, 64 + i, 96 + i (row j holds
// words 32j .. 32j + 31), and a job runs only the rows its symbols fill, so a job
// of a few hundred symbols costs one row.  Wavelet
// tree rounds >= 1 split every text into one job per prefix (Sec. 2: the
// independent subtrees), most of them small.

namespace {

// Two instantiations: KW = 1 (jobs of at most 1024 symbols, most of the wavelet
// tree's subtrees: 6 KB per warp, 16 warps per block) and KW = kSmallWords (the
// rest, 8 warps per block).
template <int KW>
struct SmallSmem {
    uint32_t plane[2][kChunk][32 * KW + 1];   // current / next planes (+ overflow word)
    uint32_t lvl[32 * KW + 4];                // the current level's plane
    uint32_t lvl2[32 * KW + 4];               // WT: the level's plane in id order
    uint32_t hist[kCols];              // class counts of the job (leaf level)
    uint32_t P[kCols + 1];             // prefix sums of hist
    uint32_t cnt[kCols / 2];           // class counts of the current level
    uint32_t loc[kCols / 2];           // class start in job order (reversed prefixes)
    uint32_t glo[kCols / 2];           // class start inside the text's level
};

}  // namespace

template <int KW, int WARPS>
__global__ void __launch_bounds__(WARPS * 32, 2) k_build_small(RoundArgs a)
{
    constexpr uint32_t NW = 32 * KW;
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    SmallSmem<KW> &sm = reinterpret_cast<SmallSmem<KW> *>(smem_raw)[warp];
    const uint32_t slot = blockIdx.x * WARPS + warp;
    if (slot >= a.nslots) return;
    const Job jb = a.jobs[slot];
    if (!WT_IN(WT_BOUNDS_TABLE, jb.text, a.ntexts)) return;
    const TextInfo &t = a.texts[jb.text];
    if (!small_job(t, a.round, jb.n)) return;
    if ((KW == 1) != (jb.n <= 1024u)) return;        // the other instantiation takes it
    if (jb.n <= kLaneJob) return;                     // one thread each (k_build_lane)
    const RoundText rt = round_text(t, a.round);
    const uint32_t h = rt.h, rb = rt.rb, n = jb.n;
    if (!WT_IN(WT_BOUNDS_TEXT, (uint64_t)jb.off + n, t.n + 1)) return;
    if (!WT_IN(WT_BOUNDS_LEVEL, rt.c + h, t.L + 1)) return;
    if (!WT_IN(WT_BOUNDS_SHARED, n, (uint32_t)(32 * NW) + 1)) return;
    const bool matrix = a.kind == WT_MATRIX;
    const uint8_t *in = static_cast<const uint8_t *>(rt.in) + (size_t)jb.off * rt.in_w;
    const uint32_t nj = (n + 1023u) / 1024u;          // rows of 32 words in use (1 .. KW)
    const uint32_t nwu = 32u * nj;                    // words in use; word nwu takes overflow bits
    if (a.round == 0) {                               // symbols >= sigma, as in the histogram pass
        const bool check = t.sigma < (1ull << t.L);
        const uint32_t sig = (uint32_t)min(t.sigma, (uint64_t)0xffffffffu);
        bool bad = false;
        for (uint32_t i = lane; i < n; i += 32) {
            const uint32_t v = load_sym(in, rt.in_w, i);
            bad |= (check && v >= sig) || (t.L < 32 && (v >> t.L) != 0);
        }
        if (__any_sync(kFull, bad) && lane == 0) atomicCAS(&a.ctl->status, 0u, (uint32_t)WT_ERR_SYMBOL_RANGE);
    }

    // ---- clear, load and transpose (plane k = code bit rb-1-k), class counts
    for (uint32_t k = 0; k < 2 * kChunk; ++k)
        for (uint32_t i = lane; i <= nwu; i += 32) (&sm.plane[0][0][0])[k * (NW + 1) + i] = 0;
    for (uint32_t i = lane; i < kCols; i += 32) sm.hist[i] = 0;
    __syncwarp();
    for (uint32_t j = 0; j < nj; ++j) {
        const uint32_t wj = 32u * j + lane;           // this lane's word of row j
        uint32_t x[8];
        load32(in, rt.in_w, 32u * wj, n, 0u, x);
#pragma unroll
        for (int k = 0; k < 8; ++k) {
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                const uint32_t e = 32u * wj + 4u * k + b;
                if (e < n) atomicAdd(&sm.hist[(x[k] >> (8 * b)) & ((1u << h) - 1u)], 1u);
            }
        }
#pragma unroll
        for (int b = 0; b < 4; ++b) transpose8(x[2 * b], x[2 * b + 1]);
        for (uint32_t k = 0; k < h; ++k) {
            const uint32_t jb8 = rb - 1u - k;
            const uint32_t sel = (jb8 & 3u) | ((jb8 & 3u) + 4u) << 4;
            const bool hi = jb8 >= 4u;
            const uint32_t t01 = __byte_perm(hi ? x[1] : x[0], hi ? x[3] : x[2], sel);
            const uint32_t t23 = __byte_perm(hi ? x[5] : x[4], hi ? x[7] : x[6], sel);
            sm.plane[0][k][wj] = __byte_perm(t01, t23, 0x5410);
        }
    }
    __syncwarp();
    {
        const uint32_t tot = warp_scan_256(256, [&](uint32_t i) { return sm.hist[i]; }, [](uint32_t i) { return i; },
                                           [&](uint32_t i, uint32_t v) { sm.P[i] = v; });
        if (lane == 0) sm.P[256] = tot;
    }
    if (matrix) {                                     // Z[c + l]: zeros of level l, any order
        for (uint32_t l = 0; l < h; ++l) {
            uint32_t z = 0;
            for (uint32_t j = 0; j < nj; ++j) z += __popc(~sm.plane[0][l][32u * j + lane]);
#pragma unroll
            for (int d = 16; d >= 1; d >>= 1) z += __shfl_xor_sync(kFull, z, d);
            if (lane == 0) t.zeros[rt.c + l] = z;
        }
    }
    __syncwarp();

    uint64_t *bv = t.bv;
    for (uint32_t l = 0; l < h; ++l) {
        uint32_t(*cur)[NW + 1] = sm.plane[l & 1];
        uint32_t(*nxt)[NW + 1] = sm.plane[(l + 1) & 1];
        const uint32_t base = 1u << l, s = h - l;
        // ---- class tables of level l (fold of the counts; starts in job order
        //      by reversed prefixes; interval starts in id (WT) / pi_l (WM) order)
        for (uint32_t q = lane; q < base; q += 32) sm.cnt[q] = sm.P[(q + 1) << s] - sm.P[q << s];
        __syncwarp();
        warp_scan_256(base, [&](uint32_t q) { return sm.cnt[q]; }, [&](uint32_t i) { return rev_bits(i, l); },
                      [&](uint32_t q, uint32_t v) { sm.loc[q] = v; });
        __syncwarp();
        // interval starts: the job's order for the WM; id order for the WT, where the
        // symbols before prefix q are those with leaf codes below q << s
        for (uint32_t q = lane; q < base; q += 32) sm.glo[q] = jb.off + (matrix ? sm.loc[q] : sm.P[q << s]);
        __syncwarp();
        // zeros before each of this lane's words (row by row: a warp scan plus
        // the zeros of the rows before), and the total zt
        uint32_t mw[KW], zw[KW], zb[KW], zt = 0;
#pragma unroll
        for (uint32_t j = 0; j < KW; ++j) {
            if (j >= nj) break;
            mw[j] = cur[l][32u * j + lane];
            sm.lvl[32u * j + lane] = mw[j];
            zw[j] = __popc(~mw[j]);
            uint32_t inc = zw[j];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(kFull, inc, d);
                if (lane >= (uint32_t)d) inc += y;
            }
            zb[j] = zt + inc - zw[j];
            zt += __shfl_sync(kFull, inc, 31);
        }
        if (lane < 4) sm.lvl[nwu + lane] = 0;
        __syncwarp();
        // ---- the job's bits of level c + l are the range [off, off + n) of the level:
        //      for the WM in the job's order of classes (reversed prefixes, the
        //      level's interval order); for the WT in id order, which differs from the
        //      job's order from level 2 on: there the class runs are first moved to
        //      their id-order places in lvl2
        const uint32_t *src = sm.lvl;
        if (!matrix && l >= 2) {
            for (uint32_t i = lane; i < nwu + 4; i += 32) sm.lvl2[i] = 0;
            __syncwarp();
            for (uint32_t q = lane; q < base; q += 32) {
                const uint32_t c = sm.cnt[q], from = sm.loc[q], to = sm.glo[q] - jb.off;
                for (uint32_t i = 0; i < c; i += 64) {
                    const uint32_t len = min(64u, c - i);
                    if (WT_IN(WT_BOUNDS_SHARED, (to + i + len - 1) >> 5, 32 * KW + 4) &&
                        WT_IN(WT_BOUNDS_SHARED, ((from + i) >> 5) + 2, 32 * KW + 4))
                        place_bits(sm.lvl2, to + i, extract_bits(sm.lvl, from + i, len), len);
                }
            }
            __syncwarp();
            src = sm.lvl2;
        }
        {
            uint64_t *lv = bv + (uint64_t)(rt.c + l) * t.W;
            const uint64_t off = jb.off, end = off + n;
            for (uint64_t d = (off >> 6) + lane; d <= (end - 1) >> 6; d += 32) {
                if (!WT_IN(WT_BOUNDS_LEVEL, d, t.W)) break;
                const uint64_t wb = d << 6;
                const uint64_t lo = wb > off ? wb : off, hi = end < wb + 64 ? end : wb + 64;
                const uint32_t blo = (uint32_t)(lo - wb);
                uint32_t bhi = (uint32_t)(hi - wb);
                const uint64_t val = extract_bits(src, (uint32_t)(lo - off), bhi - blo) << blo;
                if (end == t.n) bhi = 64;                  // bits past n belong to the last job
                if (blo == 0 && bhi == 64) {
                    lv[d] = val;
                } else {
                    const uint64_t msk = (bhi == 64 ? ~0ull : ((1ull << bhi) - 1ull)) & ~((1ull << blo) - 1ull);
                    atomicAnd(reinterpret_cast<unsigned long long *>(lv + d), ~msk);
                    atomicOr(reinterpret_cast<unsigned long long *>(lv + d), val);
                }
            }
        }
        // ---- stable split of every later plane by plane l, word by word
        if (l + 1 < h) {
#pragma unroll
            for (uint32_t j = 0; j < KW; ++j) {
                if (j >= nj) break;
                const uint32_t wj = 32u * j + lane;
                const uint32_t m0 = mw[j], z0 = zw[j], zo = zb[j];
                ByteSplit bs;                             // the in-byte compress of the tile kernel
                byte_split(m0, bs);
                const uint32_t d1 = zt + 32u * wj - zo;
                const bool in_z = z0 == 0u || WT_IN(WT_BOUNDS_SHARED, (zo + z0 - 1u) >> 5, NW + 1);
                const bool in_o = z0 == 32u || WT_IN(WT_BOUNDS_SHARED, (d1 + 31u - z0) >> 5, NW + 1);
                for (uint32_t k = l + 1; k < h; ++k) {
                    const uint32_t x = cur[k][wj];
                    if (in_z) place_bits(nxt[k], zo, byte_compress(x, bs.rz, bs.kz, bs.jz), z0);
                    if (in_o) place_bits(nxt[k], d1, byte_compress(x, bs.ro, bs.ko, bs.jo), 32u - z0);
                    cur[k][wj] = 0;
                }
            }
            if (lane == 0)
                for (uint32_t k = l + 1; k < h; ++k) cur[k][nwu] = 0;
        }
        __syncwarp();
    }
}


// ---------------------------------------------------------------------------
// The smallest jobs (at most kLaneJob symbols, last round of their text): one
// thread builds a whole job.  Most of them are the wavelet tree's subtrees of
// short texts with large alphabets, a few dozen symbols each, where a warp would
// spend its instructions on 32 mostly empty words.  Per level l the thread counts
// its symbols' l-bit prefixes, takes the node starts by an exclusive scan of the
// counts (id order for the WT, reversed prefixes for the WM: Sec. 3.1 / 5.1), and
// sets every symbol's level bit at its node's next position, in text order (the
// stable scatter of Alg. 1).  Element k of lane i's arrays is at index 32k + i, so
// that the lanes of a warp touch consecutive addresses.

namespace {

constexpr int kLaneWarps = 2;                         // warps per block of k_build_lane (13.6 KB of shared
                                                      // memory per warp: 8 blocks, 16 warps per SM)
constexpr uint32_t kLaneWords = kLaneJob / 32 + 2;    // bit buffer words per lane (+ two spare words)

struct LaneSmem {                                     // per warp
    uint8_t sym[kLaneJob * 32];                       // the job's symbols in text order
    uint8_t ctr[(kCols / 2) * 32];                    // node counters of level l (2^l <= 128): positions
                                                      // below n <= 256 fit in a byte; a count of 256 (one
                                                      // node holding every symbol) wraps to 0, which is
                                                      // then the start of empty nodes only
    uint32_t bits[kLaneWords * 32];                   // the level's bits in node order
};

}  // namespace

__global__ void __launch_bounds__(kLaneWarps * 32) k_build_lane(RoundArgs a)
{
    extern __shared__ __align__(16) uint8_t smem_raw[];
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    LaneSmem &sm = reinterpret_cast<LaneSmem *>(smem_raw)[warp];
    const uint32_t slot = blockIdx.x * blockDim.x + threadIdx.x;
    if (slot >= a.nslots) return;
    const Job jb = a.jobs[slot];
    if (jb.n > kLaneJob) return;
    if (!WT_IN(WT_BOUNDS_TABLE, jb.text, a.ntexts)) return;
    const TextInfo &t = a.texts[jb.text];
    if (!small_job(t, a.round, jb.n)) return;
    const RoundText rt = round_text(t, a.round);
    const uint32_t h = rt.h, n = jb.n;
    if (!WT_IN(WT_BOUNDS_TEXT, (uint64_t)jb.off + n, t.n + 1)) return;
    if (!WT_IN(WT_BOUNDS_LEVEL, rt.c + h, t.L + 1)) return;
    const bool matrix = a.kind == WT_MATRIX;
    const uint8_t *in = static_cast<const uint8_t *>(rt.in) + (size_t)jb.off * rt.in_w;
    // the last round's symbols have h <= 8 code bits (rb == h); like the warp
    // kernel, only their low h bits are used, so every prefix indexes a node of
    // its level and every position stays below n
    const uint32_t hmask = (1u << h) - 1u;
    // first round: symbols >= sigma (or beyond the L code bits) are reported, as in
    // the histogram pass, which has no group of a small job to look at
    const bool first = a.round == 0;
    const bool check = first && t.sigma < (1ull << t.L);
    const uint32_t sig = (uint32_t)min(t.sigma, (uint64_t)0xffffffffu);
    bool bad = false;
    for (uint32_t i = 0; i < n; ++i) {
        const uint32_t v = load_sym(in, rt.in_w, i);
        bad |= (check && v >= sig) || (first && t.L < 32 && (v >> t.L) != 0);
        sm.sym[32u * i + lane] = (uint8_t)(v & hmask);
    }
    if (bad) atomicCAS(&a.ctl->status, 0u, (uint32_t)WT_ERR_SYMBOL_RANGE);
    for (uint32_t l = 0; l < h; ++l) {
        const uint32_t base = 1u << l, sh = h - l;
        for (uint32_t q = 0; q < base; ++q) sm.ctr[32u * q + lane] = 0;
        for (uint32_t i = 0; i < n; ++i) ++sm.ctr[32u * (sm.sym[32u * i + lane] >> sh) + lane];
        uint32_t run = 0;
        for (uint32_t k = 0; k < base; ++k) {
            const uint32_t q = matrix ? rev_bits(k, l) : k;
            const uint32_t c = sm.ctr[32u * q + lane];
            sm.ctr[32u * q + lane] = (uint8_t)run;
            run += c;
        }
        const uint32_t nw = (n + 31u) / 32u;
        for (uint32_t w = 0; w < nw + 2u; ++w) sm.bits[32u * w + lane] = 0;
        uint32_t z = 0;
        for (uint32_t i = 0; i < n; ++i) {
            const uint32_t v = sm.sym[32u * i + lane];
            const uint32_t q = v >> sh, b = (v >> (sh - 1u)) & 1u;
            const uint32_t d = sm.ctr[32u * q + lane];
            sm.ctr[32u * q + lane] = (uint8_t)(d + 1u);
            sm.bits[32u * (d >> 5) + lane] |= b << (d & 31u);
            z += b ^ 1u;
        }
        if (matrix) t.zeros[rt.c + l] = z;              // Z[c + l]: zeros of level l (the whole text)
        // the job's bits are the range [off, off + n) of level c + l
        uint64_t *lv = t.bv + (uint64_t)(rt.c + l) * t.W;
        const uint64_t off = jb.off, end = off + n;
        for (uint64_t dw = off >> 6; dw <= (end - 1) >> 6; ++dw) {
            if (!WT_IN(WT_BOUNDS_LEVEL, dw, t.W)) break;
            const uint64_t wb = dw << 6;
            const uint64_t lo = wb > off ? wb : off, hi = end < wb + 64 ? end : wb + 64;
            const uint32_t blo = (uint32_t)(lo - wb);
            uint32_t bhi = (uint32_t)(hi - wb);
            const uint32_t src = (uint32_t)(lo - off), len = bhi - blo;
            const uint32_t w0 = src >> 5, s0 = src & 31u;
            const uint64_t pair = ((uint64_t)sm.bits[32u * (w0 + 1u) + lane] << 32) | sm.bits[32u * w0 + lane];
            uint64_t val = pair >> s0;
            if (s0) val |= (uint64_t)sm.bits[32u * (w0 + 2u) + lane] << (64u - s0);
            if (len < 64u) val &= (1ull << len) - 1ull;
            val <<= blo;
            if (end == t.n) bhi = 64;                  // bits past n belong to the last job
            if (blo == 0 && bhi == 64) {
                lv[dw] = val;
            } else {
                const uint64_t msk = (bhi == 64 ? ~0ull : ((1ull << bhi) - 1ull)) & ~((1ull << blo) - 1ull);
                atomicAnd(reinterpret_cast<unsigned long long *>(lv + dw), ~msk);
                atomicOr(reinterpret_cast<unsigned long long *>(lv + dw), val);
            }
        }
    }
}

// ---------------------------------------------------------------------------

cudaError_t configure_kernels()
{
    cudaError_t e;
    e = cudaFuncSetAttribute(k_build_small<1, kTinyWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(SmallSmem<1>) * kTinyWarps));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_build_small<kSmallWords, kSmallWarps>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(SmallSmem<kSmallWords>) * kSmallWarps));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_build_lane, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(sizeof(LaneSmem) * kLaneWarps));
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_hist<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHistSmem);
    if (e != cudaSuccess) return e;
    e = cudaFuncSetAttribute(k_hist<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kHistSmemLC);
    if (e != cudaSuccess) return e;
    for (auto k : {k_build_bs<false, false, 0>, k_build_bs<false, true, 0>, k_build_bs<true, false, 0>,
                   k_build_bs<false, false, 8>, k_build_bs<false, true, 8>, k_build_bs<true, false, 8>}) {
        e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sizeof(BsSmem));
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

__global__ void k_gather(const void *text, uint32_t w, const uint32_t *perm, uint64_t n, void *sorted)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n; j += (uint64_t)gridDim.x * blockDim.x)
        store_sym(sorted, w, j, load_sym(text, w, perm[j]));
}

__global__ void k_identity_order(const void *text, uint32_t w, uint64_t n, uint32_t *perm, void *sorted)
{
    for (uint64_t j = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; j < n;
         j += (uint64_t)gridDim.x * blockDim.x) {
        if (perm) perm[j] = (uint32_t)j;
        if (sorted) store_sym(sorted, w, j, load_sym(text, w, j));
    }
}

// A text built in one round: its symbols after the last level are runs of equal
// symbols, c repeated count[c] times, the runs in id order (WT) or in the order of
// the reversed L-bit codes (WM).  Each block fills one contiguous chunk of the
// output; a thread keeps the run it is in and searches again (binary search over
// the run starts) only when it passes the run's end.
__global__ void __launch_bounds__(256) k_fill_runs(const uint32_t *count, uint32_t L, uint32_t matrix, uint64_t n,
                                                   void *sorted, uint32_t w)
{
    __shared__ uint32_t start[kCols + 1];
    __shared__ uint32_t sym[kCols];
    const uint32_t nc = 1u << L;
    if (threadIdx.x < 32) {
        const uint32_t tot = warp_scan_256(nc, [&](uint32_t c) { return count[c]; },
                                           [&](uint32_t i) { return matrix ? rev_bits(i, L) : i; },
                                           [&](uint32_t c, uint32_t v) {
                                               const uint32_t i = matrix ? rev_bits(c, L) : c;   // c's run
                                               start[i] = v;
                                               sym[i] = c;
                                           });
        if (threadIdx.x == 0) start[nc] = tot;
    }
    __syncthreads();
    const uint64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t j0 = (uint64_t)blockIdx.x * chunk, j1 = min(n, j0 + chunk);
    uint64_t end = 0;                                // end of the current run (0: none yet)
    uint32_t cur = 0;
    for (uint64_t j = j0 + threadIdx.x; j < j1; j += blockDim.x) {
        if (j >= end) {
            uint32_t lo = 0, hi = nc;                // last run starting at or before j
            while (hi - lo > 1) {
                const uint32_t mid = (lo + hi) >> 1;
                if (start[mid] <= j) lo = mid; else hi = mid;
            }
            cur = sym[lo];
            end = start[lo + 1];
        }
        store_sym(sorted, w, j, cur);
    }
}

cudaError_t launch_fill_runs(const uint32_t *count, uint32_t L, bool matrix, uint64_t n, void *sorted, uint32_t w,
                             cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 152ull * 16);
    k_fill_runs<<<(uint32_t)blocks, 256, 0, s>>>(count, L, matrix ? 1u : 0u, n, sorted, w);
    return cudaGetLastError();
}

cudaError_t launch_gather(const void *text, uint32_t w, const uint32_t *perm, uint64_t n, void *sorted,
                          cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 152ull * 16);
    k_gather<<<(uint32_t)blocks, 256, 0, s>>>(text, w, perm, n, sorted);
    return cudaGetLastError();
}

cudaError_t launch_identity_order(const void *text, uint32_t w, uint64_t n, uint32_t *perm, void *sorted,
                                  cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    const uint64_t blocks = std::min<uint64_t>((n + 255) / 256, 152ull * 16);
    k_identity_order<<<(uint32_t)blocks, 256, 0, s>>>(text, w, n, perm, sorted);
    return cudaGetLastError();
}

cudaError_t launch_zero_z(const TextInfo *texts, uint32_t ntexts, cudaStream_t s)
{
    if (ntexts == 0) return cudaSuccess;
    k_zero_z<<<(ntexts + 255) / 256, 256, 0, s>>>(texts, ntexts);
    return cudaGetLastError();
}

cudaError_t launch_round(const RoundArgs &a, uint32_t in_w, cudaStream_t s)
{
    if (a.nslots == 0) return cudaSuccess;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    cudaStreamIsCapturing(s, &cap);
    const bool prof = profile_on() && cap == cudaStreamCaptureStatusNone;
    const bool root = a.round == 0 || a.kind == WT_MATRIX;
    if (prof) profile_mark(3, true, s);
    if (root) k_root_jobs<<<(a.ntexts + 255) / 256, 256, 0, s>>>(a);
    else k_child_jobs<<<a.pnslots, 256, 0, s>>>(a);
    if (a.nslots <= kScanOneBlock) {
        k_scan_groups<<<1, 1024, 0, s>>>(a);
    } else {
        const uint32_t chunks = (a.nslots + kScanChunk - 1) / kScanChunk;
        k_scan_chunks<<<chunks, 1024, 0, s>>>(a, 0u);
        k_scan_groups<<<1, 1024, 0, s>>>(a);
        k_scan_chunks<<<chunks, 1024, 0, s>>>(a, 1u);
    }
    if (prof) profile_mark(3, false, s);
    if (a.groups_ub == 0) return cudaGetLastError();
    if (prof) profile_mark(1, true, s);
    if (in_w == 1) k_hist<true><<<a.groups_ub, kHistThreads, kHistSmemLC, s>>>(a);   // byte rounds
    else k_hist<false><<<a.groups_ub, kHistThreads, kHistSmem, s>>>(a);
    if (prof) { profile_mark(1, false, s); profile_mark(2, true, s); }
    k_blocksum<<<a.blocks_ub, 256, 0, s>>>(a);
    k_blockscan<<<1, 256, 0, s>>>(a);
    k_groupexcl<<<a.blocks_ub, 256, 0, s>>>(a);
    if (prof) { profile_mark(2, false, s); profile_mark(0, true, s); }
    // every job of the round splits 8 levels: the instantiation with fixed loop bounds
    const bool h8 = a.all_h8 != 0;
    if (a.kind == kBoth) {
        if (h8) k_build_bs<true, false, 8><<<a.groups_ub, kThreads, sizeof(BsSmem), s>>>(a);
        else k_build_bs<true, false, 0><<<a.groups_ub, kThreads, sizeof(BsSmem), s>>>(a);
    } else if (a.any_cut || a.any_order) {
        // rounds that write the stable order take the instantiation with loop bounds for
        // any number of levels: in the unrolled one, the order's ranking and staging run
        // short of registers (13.5 against 10.4 ms for the order of a 2^30-symbol WM)
        if (h8 && !a.any_order) k_build_bs<false, true, 8><<<a.groups_ub, kThreads, sizeof(BsSmem), s>>>(a);
        else k_build_bs<false, true, 0><<<a.groups_ub, kThreads, sizeof(BsSmem), s>>>(a);
    } else {
        if (h8) k_build_bs<false, false, 8><<<a.groups_ub, kThreads, sizeof(BsSmem), s>>>(a);
        else k_build_bs<false, false, 0><<<a.groups_ub, kThreads, sizeof(BsSmem), s>>>(a);
    }
    if (a.any_small && a.kind != kBoth)           // kBoth has no small jobs
    {
        k_build_lane<<<(a.nslots + kLaneWarps * 32 - 1) / (kLaneWarps * 32), kLaneWarps * 32,
                       sizeof(LaneSmem) * kLaneWarps, s>>>(a);
        k_build_small<1, kTinyWarps><<<(a.nslots + kTinyWarps - 1) / kTinyWarps, kTinyWarps * 32,
                                      sizeof(SmallSmem<1>) * kTinyWarps, s>>>(a);
        k_build_small<kSmallWords, kSmallWarps><<<(a.nslots + kSmallWarps - 1) / kSmallWarps, kSmallWarps * 32,
                                                  sizeof(SmallSmem<kSmallWords>) * kSmallWarps, s>>>(a);
    }
    if (prof) profile_mark(0, false, s, (a.any_small && a.kind != kBoth) ? 4 : 1);
    return cudaGetLastError();
}

}  // namespace wtg

// ---------------------------------------------------------------------------
// Report of the bounds checks (a build with -DWT_DEBUG_BOUNDS), see the header.

#ifdef WT_DEBUG_BOUNDS
namespace wtg {
namespace {

__global__ void k_bounds_selftest()
{
    // two checks with nothing behind them: the first fails, the second holds
    const uint64_t one = threadIdx.x + 1u;
    if (!WT_IN(WT_BOUNDS_SELFTEST, one, 1u)) {
    }
    if (!WT_IN(WT_BOUNDS_SELFTEST, one - 1u, 1u)) {
    }
}

}  // namespace
}  // namespace wtg
#endif

extern "C" wt_status wt_debug_bounds_read(wt_bounds_report *out, int reset)
{
    if (out == nullptr) return WT_ERR_INVALID_ARG;
    *out = wt_bounds_report{};
#ifdef WT_DEBUG_BOUNDS
    if (cudaDeviceSynchronize() != cudaSuccess) return WT_ERR_CUDA;
    if (cudaMemcpyFromSymbol(out, wtg::g_bounds, sizeof(*out)) != cudaSuccess) return WT_ERR_CUDA;
    out->enabled = 1;
    if (reset) {
        const wt_bounds_report zero{};
        if (cudaMemcpyToSymbol(wtg::g_bounds, &zero, sizeof(zero)) != cudaSuccess) return WT_ERR_CUDA;
    }
#else
    (void)reset;
#endif
    return WT_OK;
}

extern "C" wt_status wt_debug_bounds_selftest(void *stream)
{
#ifdef WT_DEBUG_BOUNDS
    wtg::k_bounds_selftest<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>();
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
#else
    (void)stream;
    return WT_ERR_INVALID_ARG;
#endif
}
