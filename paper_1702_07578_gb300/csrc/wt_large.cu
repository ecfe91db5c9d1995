// Texts of any length (see the "texts of any length" section of include/wt_gb300.h):
// domain decomposition (Sec. 3.3).  Consecutive slices of the text, each shorter
// than 2^32 symbols, are built on their own (wt_build / wm_build) into partial
// levels in the workspace; then, level by level, the merged level is the
// concatenation, prefix by prefix (id order for the WT, bit-reversal order for the
// WM, Sec. 5.1), of the slices' intervals in slice order.  A zero-based prefix sum
// of the interval sizes gives where each run lands; one thread per output word
// assembles the word from the runs that cover it.  Z[l] of the WM is the sum of the
// slices' Z[l].
#include <cstdint>

#include "wt_internal.h"

namespace wtg {
namespace {

constexpr uint64_t kDefaultSlice = 1ull << 31;

struct Run {
    uint64_t dst;     // first bit in the merged level
    uint32_t src;     // first bit in the slice's level
    uint32_t len;
    uint32_t slice;
    uint32_t pad;
};

struct LargePlan {
    uint32_t L = 0;
    uint64_t n = 0, slice = 0, nslices = 0, Ws = 0;
    size_t slice_ws = 0;
    size_t off_ws = 0, off_partial = 0, off_counts = 0, off_zp = 0, off_runs = 0, off_status = 0, bytes = 0;
};

size_t al(size_t x) { return (x + 255) / 256 * 256; }

uint32_t nlevels(uint64_t sigma)
{
    uint32_t L = 0;
    while (L < 64 && (1ull << L) < sigma) ++L;
    return L;
}

wt_status large_plan(wt_kind kind, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t slice, LargePlan &p)
{
    if (kind != WT_TREE && kind != WT_MATRIX) return WT_ERR_INVALID_ARG;
    if (type != WT_U8 && type != WT_U16 && type != WT_U32) return WT_ERR_INVALID_ARG;
    if (sigma == 0 || sigma > 256 || n >= (1ull << 40)) return WT_ERR_INVALID_ARG;
    if (slice == 0) slice = kDefaultSlice;
    if (slice >= (1ull << 32)) return WT_ERR_INVALID_ARG;
    p.L = nlevels(sigma);
    p.n = n;
    p.slice = slice;
    p.nslices = (n + slice - 1) / slice;
    if (p.nslices > (1u << 16)) return WT_ERR_INVALID_ARG;     // run tables of at most 2^23 entries
    p.Ws = (slice + 63) / 64;
    const uint64_t first = n < slice ? n : slice;
    wt_status st = wt_workspace_size(kind, type, first, sigma, &p.slice_ws);
    if (st != WT_OK) return st;
    size_t off = 0;
    p.off_ws = off;
    off = al(off + p.slice_ws);
    p.off_partial = off;
    off = al(off + 8 * p.nslices * p.L * p.Ws);
    p.off_counts = off;
    off = al(off + 4 * p.nslices * kCols);
    p.off_zp = off;
    off = al(off + 8 * p.nslices * (p.L ? p.L : 1));
    p.off_runs = off;
    off = al(off + sizeof(Run) * p.nslices * (p.L ? (1ull << (p.L - 1)) : 1));
    p.off_status = off;
    off = al(off + sizeof(uint32_t));
    p.bytes = off;
    return WT_OK;
}

// class counts of a text (its symbols' low 8 bits), one shared histogram per block
__global__ void __launch_bounds__(256) k_slice_counts(const void *text, uint32_t w, uint64_t n, uint32_t *counts)
{
    __shared__ uint32_t h[kCols];
    h[threadIdx.x] = 0;
    __syncthreads();
    const uint64_t chunk = (n + gridDim.x - 1) / gridDim.x;
    const uint64_t i0 = (uint64_t)blockIdx.x * chunk, i1 = min(n, i0 + chunk);
    for (uint64_t i = i0 + threadIdx.x; i < i1; i += blockDim.x) {
        const uint32_t v = w == 1 ? static_cast<const uint8_t *>(text)[i]
                                  : (w == 2 ? static_cast<const uint16_t *>(text)[i]
                                            : static_cast<const uint32_t *>(text)[i]);
        atomicAdd(&h[v & 0xffu], 1u);
    }
    __syncthreads();
    if (h[threadIdx.x]) atomicAdd(&counts[threadIdx.x], h[threadIdx.x]);
}

}  // namespace

cudaError_t launch_class_counts(const void *text, uint32_t w, uint64_t n, uint32_t *counts, cudaStream_t s)
{
    if (n == 0) return cudaSuccess;
    k_slice_counts<<<(uint32_t)((n + 65535) / 65536), 256, 0, s>>>(text, w, n, counts);
    return cudaGetLastError();
}

namespace {

__device__ __forceinline__ uint32_t rev_l(uint32_t q, uint32_t l) { return l ? (__brev(q) >> (32u - l)) : 0u; }

// Runs of level l in merged order: run r = i * nslices + c is the interval of the
// i-th prefix of the level's order (q = i, or rho_l(i) for the WM) in slice c.
__global__ void __launch_bounds__(1024) k_runs(const uint32_t *counts, uint32_t nslices, uint32_t L, uint32_t l,
                                               uint32_t matrix, Run *runs)
{
    __shared__ uint64_t ws[32];
    __shared__ uint64_t carry;
    const uint32_t nq = 1u << l, R = nq * nslices, span = 1u << (L - l);
    for (uint32_t r = threadIdx.x; r < R; r += blockDim.x) {
        const uint32_t i = r / nslices, c = r % nslices;
        const uint32_t q = matrix ? rev_l(i, l) : i;
        uint32_t s = 0;
        for (uint32_t a = q * span; a < (q + 1) * span; ++a) s += counts[(size_t)c * kCols + a];
        runs[r].len = s;
        runs[r].slice = c;
        runs[r].pad = 0;
    }
    __syncthreads();
    // slice-local interval starts: per slice, a running sum in the level's order
    for (uint32_t c = threadIdx.x; c < nslices; c += blockDim.x) {
        uint32_t s = 0;
        for (uint32_t i = 0; i < nq; ++i) {
            Run &x = runs[(size_t)i * nslices + c];
            x.src = s;
            s += x.len;
        }
    }
    // merged starts: exclusive scan over all runs in order
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    for (uint32_t r0 = 0; r0 < R; r0 += blockDim.x) {
        const uint32_t r = r0 + threadIdx.x;
        const uint64_t v = r < R ? runs[r].len : 0;
        uint64_t inc = v;
        for (int d = 1; d < 32; d <<= 1) {
            const uint64_t y = __shfl_up_sync(0xffffffffu, inc, d);
            if (lane >= (uint32_t)d) inc += y;
        }
        if (lane == 31) ws[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const uint64_t x = ws[lane];
            uint64_t p = x;
            for (int d = 1; d < 32; d <<= 1) {
                const uint64_t y = __shfl_up_sync(0xffffffffu, p, d);
                if (lane >= (uint32_t)d) p += y;
            }
            ws[lane] = p - x;
        }
        __syncthreads();
        if (r < R) runs[r].dst = carry + ws[warp] + inc - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry += ws[warp] + inc;
        __syncthreads();
    }
}

// `len` (<= 64) bits of a level starting at bit `pos`
__device__ __forceinline__ uint64_t read_bits(const uint64_t *lv, uint64_t words, uint64_t pos, uint32_t len)
{
    const uint64_t w = pos >> 6;
    const uint32_t s = (uint32_t)(pos & 63);
    uint64_t v = lv[w] >> s;
    if (s && s + len > 64 && w + 1 < words) v |= lv[w + 1] << (64 - s);
    return len == 64 ? v : (v & ((1ull << len) - 1ull));
}

// One thread per word of the merged level l.
__global__ void __launch_bounds__(256) k_merge(const Run *runs, uint32_t R, const uint64_t *partial, uint64_t Ws,
                                               uint32_t L, uint32_t l, uint64_t slice, uint64_t n, uint64_t *out,
                                               uint64_t W)
{
    __shared__ uint32_t first;
    const uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (threadIdx.x == 0) {                           // last run starting at or before the block's first bit
        const uint64_t p0 = (uint64_t)blockIdx.x * blockDim.x * 64;
        uint32_t lo = 0, hi = R;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (runs[mid].dst <= p0) lo = mid; else hi = mid;
        }
        first = lo;
    }
    __syncthreads();
    if (w >= W) return;
    uint64_t pos = w * 64;
    const uint64_t end = min(n, pos + 64);
    uint32_t lo = first;                              // forward to the run holding pos
    while (lo + 1 < R && runs[lo + 1].dst <= pos) ++lo;
    uint64_t word = 0;
    for (uint32_t r = lo; pos < end && r < R; ++r) {
        const Run x = runs[r];
        if (x.len == 0 || x.dst + x.len <= pos) continue;
        const uint64_t into = pos - x.dst;
        const uint32_t take = (uint32_t)min(end - pos, (uint64_t)x.len - into);
        const uint64_t nc = min(slice, n - (uint64_t)x.slice * slice);
        const uint64_t wc = (nc + 63) / 64;          // the slice build's words per level
        const uint64_t *lv = partial + (uint64_t)x.slice * L * Ws + (uint64_t)l * wc;
        word |= read_bits(lv, wc, x.src + into, take) << (pos - w * 64);
        pos += take;
    }
    out[w] = word;
}

// The slice workspace's status word (offset 0, the first field of its control
// block) is cleared by every slice build: keep the first error seen, and put it
// back at the end for wt_sync_status.
__global__ void k_keep_status(uint32_t *ctl_status, uint32_t *saved, uint32_t restore)
{
    if (restore) {
        if (*saved) *ctl_status = *saved;
    } else if (*saved == 0) {
        *saved = *ctl_status;
    }
}

__global__ void k_sum_z(const uint64_t *zp, uint32_t nslices, uint32_t L, uint64_t *z)
{
    const uint32_t l = threadIdx.x;
    if (l >= L) return;
    uint64_t s = 0;
    for (uint32_t c = 0; c < nslices; ++c) s += zp[(size_t)c * L + l];
    z[l] = s;
}

}  // namespace
}  // namespace wtg

using namespace wtg;

extern "C" {

wt_status wt_large_workspace_size(wt_kind kind, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t slice,
                                  size_t *bytes)
{
    if (bytes == nullptr) return WT_ERR_INVALID_ARG;
    LargePlan p;
    wt_status st = large_plan(kind, type, n, sigma, slice, p);
    if (st == WT_OK) *bytes = p.bytes;
    return st;
}

wt_status wt_build_large(wt_kind kind, const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma,
                         uint64_t slice, uint64_t *d_bv, uint64_t *d_zeros, void *d_ws, size_t ws_bytes,
                         void *stream)
{
    LargePlan p;
    wt_status st = large_plan(kind, type, n, sigma, slice, p);
    if (st != WT_OK) return st;
    if (d_ws == nullptr || ws_bytes < p.bytes) return WT_ERR_OUT_OF_MEMORY;
    if (reinterpret_cast<uintptr_t>(d_ws) % 256) return WT_ERR_INVALID_ARG;
    const bool matrix = kind == WT_MATRIX;
    if (p.L > 0 && n > 0 && (d_text == nullptr || d_bv == nullptr || (matrix && d_zeros == nullptr)))
        return WT_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    // the status word wt_sync_status reads (offset 0 of the workspace) starts clear
    if (cudaMemsetAsync(d_ws, 0, sizeof(uint32_t), s) != cudaSuccess) return WT_ERR_CUDA;
    if (p.L == 0) return WT_OK;
    if (n == 0) {
        if (matrix && cudaMemsetAsync(d_zeros, 0, 8 * p.L, s) != cudaSuccess) return WT_ERR_CUDA;
        return WT_OK;
    }
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    void *sws = ws + p.off_ws;
    uint64_t *partial = reinterpret_cast<uint64_t *>(ws + p.off_partial);
    uint32_t *counts = reinterpret_cast<uint32_t *>(ws + p.off_counts);
    uint64_t *zp = reinterpret_cast<uint64_t *>(ws + p.off_zp);
    Run *runs = reinterpret_cast<Run *>(ws + p.off_runs);
    const uint32_t w = (uint32_t)type;
    uint32_t *saved = reinterpret_cast<uint32_t *>(ws + p.off_status);
    uint32_t *ctl_status = reinterpret_cast<uint32_t *>(sws);
    if (cudaMemsetAsync(counts, 0, 4 * p.nslices * kCols, s) != cudaSuccess ||
        cudaMemsetAsync(saved, 0, sizeof(uint32_t), s) != cudaSuccess)
        return WT_ERR_CUDA;
    // partial levels of every slice
    for (uint64_t c = 0; c < p.nslices; ++c) {
        const uint64_t nc = n - c * p.slice < p.slice ? n - c * p.slice : p.slice;
        const uint8_t *tc = static_cast<const uint8_t *>(d_text) + c * p.slice * w;
        uint64_t *bc = partial + c * p.L * p.Ws;
        st = build_with_counts(kind, tc, type, nc, sigma, bc, matrix ? zp + c * p.L : nullptr, sws, p.slice_ws,
                               counts + c * kCols, s);
        if (st != WT_OK) return st;
        k_keep_status<<<1, 1, 0, s>>>(ctl_status, saved, 0u);
    }
    const uint64_t W = (n + 63) / 64;
    for (uint32_t l = 0; l < p.L; ++l) {
        const uint32_t R = (uint32_t)(p.nslices << l);
        k_runs<<<1, 1024, 0, s>>>(counts, (uint32_t)p.nslices, p.L, l, matrix ? 1u : 0u, runs);
        const uint64_t blocks = (W + 255) / 256;
        k_merge<<<(uint32_t)blocks, 256, 0, s>>>(runs, R, partial, p.Ws, p.L, l, p.slice, n, d_bv + (uint64_t)l * W,
                                                 W);
    }
    if (matrix) k_sum_z<<<1, 32, 0, s>>>(zp, (uint32_t)p.nslices, p.L, d_zeros);
    k_keep_status<<<1, 1, 0, s>>>(ctl_status, saved, 1u);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

}  // extern "C"
