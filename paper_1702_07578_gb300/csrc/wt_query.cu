// access / rank / select on built wavelet trees and matrices (see the "queries"
// section of include/wt_gb300.h).  The bit vectors of every level get a rank
// directory: the number of ones before each 256-bit block.  The wavelet tree also
// gets, per level, every node's start and the ones before it, so that a query
// follows a root-to-leaf (or leaf-to-root) path with one rank or select per level
// (Sec. 2 for the tree, Sec. 5 for the matrix navigation: position i of level l
// moves to rank0(i), or to Z[l] + rank1(i)).
#include <cstdint>

#include "wt_internal.h"

namespace wtg {
namespace {

constexpr uint32_t kDirChunk = 4096;       // directory entries per scan chunk
constexpr uint32_t kSampleLog = 13;        // select samples: every 8192nd one / zero of a level
constexpr uint64_t kNone = ~0ull;

struct RsLayout {
    uint32_t L = 0;
    uint64_t W = 0, NB = 0, nchunks = 0;
    uint64_t NS = 0;                        // select samples per level and bit value
    size_t off_dir = 0, off_csum = 0, off_S = 0, off_R = 0, off_smp = 0, bytes = 0;
};

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

uint32_t lvls(uint64_t sigma)
{
    uint32_t L = 0;
    while (L < 64 && (1ull << L) < sigma) ++L;
    return L;
}

wt_status layout(wt_kind kind, uint64_t n, uint64_t sigma, RsLayout &r)
{
    if (kind != WT_TREE && kind != WT_MATRIX) return WT_ERR_INVALID_ARG;
    if (sigma == 0 || sigma > (1ull << 32) || n >= (1ull << 32)) return WT_ERR_INVALID_ARG;
    r.L = lvls(sigma);
    if (kind == WT_TREE && r.L > (uint32_t)kMaxTreeSigmaLog) return WT_ERR_INVALID_ARG;
    r.W = (n + 63) / 64;
    r.NB = (r.W + 3) / 4 + 1;                               // last entry: total ones
    r.nchunks = (r.NB + kDirChunk - 1) / kDirChunk;
    size_t off = 0;
    r.off_dir = off;
    off = align256(off + sizeof(uint32_t) * r.L * r.NB);
    r.off_csum = off;
    off = align256(off + sizeof(uint32_t) * r.L * r.nchunks);
    const size_t tbl = kind == WT_TREE && r.L > 0 ? (size_t)((1ull << r.L) - 1 + r.L) : 0;
    r.off_S = off;
    off = align256(off + sizeof(uint32_t) * tbl);
    r.off_R = off;
    off = align256(off + sizeof(uint32_t) * tbl);
    // block of the (k * 8192)-th one and zero of every level (the zeros counted over
    // whole blocks, the padding past n last)
    r.NS = ((r.NB - 1) * 256 >> kSampleLog) + 2;
    r.off_smp = off;
    off = align256(off + sizeof(uint32_t) * 2 * r.L * r.NS);
    r.bytes = off > 0 ? off : 256;
    return WT_OK;
}

struct QArgs {
    const uint64_t *bv;       // L * W words
    const uint64_t *zeros;    // WM
    const uint32_t *dir;      // L * NB
    uint32_t *dirw;           // same, writable (build)
    uint32_t *csum;           // L * nchunks
    uint32_t *S, *R;          // WT node starts / ones before them, level l at (2^l - 1 + l)
    uint32_t *smp;            // select samples [level][bit value][NS] (null: search the whole directory)
    uint64_t n, W, NB, nchunks, NS;
    uint32_t L;
    uint32_t kind;
};

__device__ __forceinline__ size_t tbl_off(uint32_t l) { return ((size_t)1 << l) - 1 + l; }

// ones in bits [0, i) of level l
__device__ __forceinline__ uint32_t rank1(const QArgs &a, uint32_t l, uint64_t i)
{
    const uint64_t *bv = a.bv + (uint64_t)l * a.W;
    const uint64_t b = i >> 8, w = i >> 6;
    uint32_t r = a.dir[(uint64_t)l * a.NB + b];
    for (uint64_t k = b * 4; k < w; ++k) r += __popcll(bv[k]);
    if (i & 63) r += __popcll(bv[w] & ((1ull << (i & 63)) - 1ull));
    return r;
}

// position of the t-th (0-based) set bit of x
__device__ __forceinline__ uint32_t select_in_word(uint64_t x, uint32_t t)
{
    uint32_t pos = 0, v = (uint32_t)x, c = __popc(v);
    if (t >= c) {
        t -= c;
        v = (uint32_t)(x >> 32);
        pos = 32;
    }
    c = __popc(v & 0xffffu);
    if (t >= c) { t -= c; v >>= 16; pos += 16; }
    c = __popc(v & 0xffu);
    if (t >= c) { t -= c; v >>= 8; pos += 8; }
    c = __popc(v & 0xfu);
    if (t >= c) { t -= c; v >>= 4; pos += 4; }
    c = __popc(v & 0x3u);
    if (t >= c) { t -= c; v >>= 2; pos += 2; }
    if (t >= (v & 1u)) pos += 1;
    return pos;
}

// position of the j-th (0-based) bit equal to `one` in level l (j must exist)
__device__ __forceinline__ uint64_t select_bit(const QArgs &a, uint32_t l, uint64_t j, bool one)
{
    const uint64_t *bv = a.bv + (uint64_t)l * a.W;
    const uint32_t *dir = a.dir + (uint64_t)l * a.NB;
    uint64_t lo = 0, hi = a.NB - 1;                         // last block with count-before <= j
    if (a.smp != nullptr) {                                 // the samples around j bound the search
        const uint32_t *sm = a.smp + ((uint64_t)l * 2 + (one ? 1 : 0)) * a.NS;
        const uint64_t k = j >> kSampleLog;
        lo = sm[k];
        const uint64_t total = one ? dir[a.NB - 1] : (a.NB - 1) * 256 - dir[a.NB - 1];
        if (((k + 1) << kSampleLog) < total) hi = (uint64_t)sm[k + 1] + 1;
    }
    while (hi - lo > 1) {
        const uint64_t mid = (lo + hi) >> 1;
        const uint64_t before = one ? dir[mid] : mid * 256 - dir[mid];
        if (before <= j) lo = mid; else hi = mid;
    }
    uint64_t rem = j - (one ? dir[lo] : lo * 256 - dir[lo]);
    for (uint64_t k = lo * 4;; ++k) {
        const uint64_t x = one ? bv[k] : ~bv[k];
        const uint32_t c = __popcll(x);
        if (rem < c) return k * 64 + select_in_word(x, (uint32_t)rem);
        rem -= c;
    }
}

// ---- directory: counts of every 256-bit block, scanned per level ------------

__device__ __forceinline__ uint32_t block_ones(const QArgs &a, uint32_t l, uint64_t b)
{
    const uint64_t *bv = a.bv + (uint64_t)l * a.W;
    uint32_t c = 0;
    for (uint64_t k = b * 4; k < b * 4 + 4 && k < a.W; ++k) c += __popcll(bv[k]);
    return c;
}

__device__ __forceinline__ uint32_t block_scan_1024(uint32_t v, uint32_t *ws, uint32_t *total)
{
    const uint32_t lane = threadIdx.x & 31u, warp = threadIdx.x >> 5;
    uint32_t inc = v;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, inc, d);
        if (lane >= (uint32_t)d) inc += y;
    }
    if (lane == 31) ws[warp] = inc;
    __syncthreads();
    const uint32_t x = ws[lane];
    uint32_t p = x;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, p, d);
        if (lane >= (uint32_t)d) p += y;
    }
    *total = __shfl_sync(0xffffffffu, p, 31);
    const uint32_t before = __shfl_sync(0xffffffffu, p - x, warp);
    __syncthreads();
    return before + inc - v;
}

// ones of 256-bit block b of level l: two 16-byte loads when the block is whole and
// the level row is 16-byte aligned, else word by word
__device__ __forceinline__ uint32_t block_ones_v(const QArgs &a, uint32_t l, uint64_t b, bool vec)
{
    if (vec && b * 4 + 4 <= a.W) {
        const uint4 *q = reinterpret_cast<const uint4 *>(a.bv + (uint64_t)l * a.W + b * 4);
        const uint4 x = __ldg(q), y = __ldg(q + 1);
        return __popc(x.x) + __popc(x.y) + __popc(x.z) + __popc(x.w) + __popc(y.x) + __popc(y.y) +
               __popc(y.z) + __popc(y.w);
    }
    return block_ones(a, l, b);
}

// Block b0 + 1024 j + t of a chunk belongs to thread t (j = 0..3): a warp reads 32
// consecutive blocks (1 KB) per j.
__device__ __forceinline__ bool rows_aligned(const QArgs &a)
{
    return (a.W % 2 == 0) && (reinterpret_cast<uintptr_t>(a.bv) % 16 == 0);
}

// grid (nchunks, L), 1024 threads: ones of each chunk of 4096 blocks
__global__ void __launch_bounds__(1024) k_dir_chunks(QArgs a)
{
    __shared__ uint32_t ws[32];
    const uint32_t l = blockIdx.y;
    const uint64_t b0 = (uint64_t)blockIdx.x * kDirChunk;
    const bool vec = rows_aligned(a);
    uint32_t s = 0;
    for (uint32_t j = 0; j < 4; ++j) {
        const uint64_t b = b0 + j * 1024 + threadIdx.x;
        if (b + 1 < a.NB) s += block_ones_v(a, l, b, vec);
    }
    uint32_t total;
    block_scan_1024(s, ws, &total);
    if (threadIdx.x == 0) a.csum[(uint64_t)l * a.nchunks + blockIdx.x] = total;
}

// grid (L), 1024 threads: exclusive scan of the chunk sums of a level
__global__ void __launch_bounds__(1024) k_dir_chunk_scan(QArgs a)
{
    __shared__ uint32_t ws[32];
    uint32_t *c = a.csum + (uint64_t)blockIdx.x * a.nchunks;
    uint32_t carry = 0;
    for (uint64_t c0 = 0; c0 < a.nchunks; c0 += 1024) {
        const uint64_t i = c0 + threadIdx.x;
        const uint32_t v = i < a.nchunks ? c[i] : 0u;
        uint32_t total;
        const uint32_t ex = block_scan_1024(v, ws, &total);
        if (i < a.nchunks) c[i] = carry + ex;
        carry += total;
    }
}

// grid (nchunks, L), 1024 threads: exclusive prefix of every block (blocks in
// order: row j of 1024, then thread t)
__global__ void __launch_bounds__(1024) k_dir_apply(QArgs a)
{
    __shared__ uint32_t ws[32];
    const uint32_t l = blockIdx.y;
    const uint64_t b0 = (uint64_t)blockIdx.x * kDirChunk;
    const bool vec = rows_aligned(a);
    uint32_t run = a.csum[(uint64_t)l * a.nchunks + blockIdx.x];
    for (uint32_t j = 0; j < 4; ++j) {
        const uint64_t b = b0 + j * 1024 + threadIdx.x;
        const uint32_t c = b + 1 < a.NB ? block_ones_v(a, l, b, vec) : 0u;
        uint32_t total;
        const uint32_t ex = block_scan_1024(c, ws, &total);
        if (b < a.NB) a.dirw[(uint64_t)l * a.NB + b] = run + ex;
        run += total;
    }
}

// grid (blocks, L): block b records itself as the sample of every (k * 8192)-th one
// and zero it holds
__global__ void k_select_samples(QArgs a)
{
    const uint32_t l = blockIdx.y;
    const uint64_t b = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (b + 1 >= a.NB) return;
    const uint32_t *dir = a.dir + (uint64_t)l * a.NB;
    const uint64_t o0 = dir[b], o1 = dir[b + 1];
    const uint64_t z0 = b * 256 - o0, z1 = (b + 1) * 256 - o1;
    uint32_t *s1 = a.smp + ((uint64_t)l * 2 + 1) * a.NS, *s0 = a.smp + (uint64_t)l * 2 * a.NS;
    const uint64_t S = 1ull << kSampleLog;
    for (uint64_t k = (o0 + S - 1) >> kSampleLog; (k << kSampleLog) < o1; ++k) s1[k] = (uint32_t)b;
    for (uint64_t k = (z0 + S - 1) >> kSampleLog; (k << kSampleLog) < z1; ++k) s0[k] = (uint32_t)b;
}

// WT node tables, level l: node p covers [S[p], S[p+1]); R[p] = ones before S[p]
__global__ void k_tree_nodes(QArgs a, uint32_t l)
{
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t nodes = 1ull << l;
    if (l == 0 && p == 0) {
        a.S[tbl_off(0)] = 0;
        a.S[tbl_off(0) + 1] = (uint32_t)a.n;
    }
    if (p > nodes) return;
    const uint32_t *S = a.S + tbl_off(l);
    uint32_t *R = a.R + tbl_off(l);
    if (p == nodes) {                                         // end of the level
        R[p] = rank1(a, l, a.n);
        if (l + 1 < a.L) a.S[tbl_off(l + 1) + 2 * nodes] = (uint32_t)a.n;
        return;
    }
    const uint32_t s = l == 0 ? 0u : S[p], e = l == 0 ? (uint32_t)a.n : S[p + 1];
    const uint32_t rs = rank1(a, l, s);
    R[p] = rs;
    if (l + 1 < a.L) {
        const uint32_t ones = rank1(a, l, e) - rs;
        const uint32_t z = (e - s) - ones;
        a.S[tbl_off(l + 1) + 2 * p] = s;
        a.S[tbl_off(l + 1) + 2 * p + 1] = s + z;
    }
}

}  // namespace
}  // namespace wtg

// ---- queries: one thread per query ------------------------------------------

namespace wtg {
namespace {

__device__ __forceinline__ uint32_t cbit(uint32_t c, uint32_t l, uint32_t L) { return (c >> (L - 1u - l)) & 1u; }

// number of c in T[0, i)
__device__ uint64_t rank_sym(const QArgs &a, uint32_t c, uint64_t i)
{
    if (a.kind == WT_TREE) {
        // the node path is c's prefixes: each level's node entries are loaded one
        // level ahead, so a level waits for its rank only
        uint64_t k = i, p = 0;
        uint32_t s = a.S[tbl_off(0)], r = a.R[tbl_off(0)];
        for (uint32_t l = 0; l < a.L; ++l) {
            const uint32_t b = cbit(c, l, a.L);
            const uint64_t pn = 2 * p + b;
            uint32_t sn = 0, rn = 0;
            if (l + 1 < a.L) {
                sn = a.S[tbl_off(l + 1) + pn];
                rn = a.R[tbl_off(l + 1) + pn];
            }
            const uint64_t ones = rank1(a, l, s + k) - r;
            k = b ? ones : k - ones;
            p = pn;
            s = sn;
            r = rn;
        }
        return k;
    }
    uint64_t s = 0, e = i;
    for (uint32_t l = 0; l < a.L; ++l) {
        const uint64_t rs = rank1(a, l, s), re = rank1(a, l, e);
        if (cbit(c, l, a.L)) {
            s = a.zeros[l] + rs;
            e = a.zeros[l] + re;
        } else {
            s -= rs;
            e -= re;
        }
    }
    return e - s;
}

__global__ void k_access(QArgs a, const uint64_t *pos, uint32_t count, uint32_t *out)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    uint64_t i = pos[k];
    if (i >= a.n) { out[k] = 0xffffffffu; return; }
    uint32_t sym = 0;
    if (a.kind == WT_TREE) {
        // both children's starts and ones-before are loaded with the level's own
        // reads, so a level costs one round trip to memory
        uint64_t p = 0;
        uint32_t s = a.S[tbl_off(0)], r = a.R[tbl_off(0)];
        for (uint32_t l = 0; l < a.L; ++l) {
            const uint64_t *bv = a.bv + (uint64_t)l * a.W;
            uint32_t s0 = 0, s1 = 0, r0 = 0, r1 = 0;
            if (l + 1 < a.L) {
                const size_t o = tbl_off(l + 1) + 2 * p;
                s0 = a.S[o];
                s1 = a.S[o + 1];
                r0 = a.R[o];
                r1 = a.R[o + 1];
            }
            const uint32_t b = (uint32_t)(bv[i >> 6] >> (i & 63)) & 1u;
            const uint64_t ones = rank1(a, l, i) - r;
            sym = (sym << 1) | b;
            if (l + 1 < a.L) {
                i = (b ? s1 : s0) + (b ? ones : (i - s) - ones);
                p = 2 * p + b;
                s = b ? s1 : s0;
                r = b ? r1 : r0;
            }
        }
    } else {
        for (uint32_t l = 0; l < a.L; ++l) {
            const uint64_t *bv = a.bv + (uint64_t)l * a.W;
            const uint32_t b = (uint32_t)(bv[i >> 6] >> (i & 63)) & 1u;
            const uint64_t r1 = rank1(a, l, i);
            sym = (sym << 1) | b;
            i = b ? a.zeros[l] + r1 : i - r1;
        }
    }
    out[k] = sym;
}

__global__ void k_rank(QArgs a, const uint32_t *sym, const uint64_t *pos, uint32_t count, uint64_t *out)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const uint32_t c = sym[k];
    const uint64_t i = pos[k];
    if (i > a.n || (a.L < 32 && (c >> a.L) != 0)) { out[k] = kNone; return; }
    out[k] = rank_sym(a, c, i);
}

__global__ void k_select(QArgs a, const uint32_t *sym, const uint64_t *jj, uint32_t count, uint64_t *out)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const uint32_t c = sym[k];
    const uint64_t j = jj[k];
    if (j == 0 || (a.L < 32 && (c >> a.L) != 0)) { out[k] = kNone; return; }
    if (j > rank_sym(a, c, a.n)) { out[k] = kNone; return; }
    uint64_t pos = j - 1;
    if (a.kind == WT_TREE) {
        for (uint32_t l = a.L; l-- > 0;) {                     // from the leaf up
            const uint64_t p = (uint64_t)c >> (a.L - l);       // node of c at level l
            const uint32_t b = cbit(c, l, a.L);
            const uint32_t s = a.S[tbl_off(l) + p], r = a.R[tbl_off(l) + p];
            const uint64_t before = b ? r : s - r;             // b-bits before the node
            pos = select_bit(a, l, before + pos, b != 0) - s;
        }
    } else {
        uint64_t s = 0;                                        // start of c's interval below the last level
        for (uint32_t l = 0; l < a.L; ++l) {
            const uint64_t rs = rank1(a, l, s);
            s = cbit(c, l, a.L) ? a.zeros[l] + rs : s - rs;
        }
        pos += s;
        for (uint32_t l = a.L; l-- > 0;) {
            if (cbit(c, l, a.L)) pos = select_bit(a, l, pos - a.zeros[l], true);
            else pos = select_bit(a, l, pos, false);
        }
    }
    out[k] = pos;
}

QArgs make_args(const RsLayout &r, wt_kind kind, const uint64_t *bv, const uint64_t *zeros, const void *rs,
                uint64_t n)
{
    QArgs a{};
    uint8_t *base = const_cast<uint8_t *>(static_cast<const uint8_t *>(rs));
    a.bv = bv;
    a.zeros = zeros;
    a.dir = reinterpret_cast<const uint32_t *>(base + r.off_dir);
    a.dirw = reinterpret_cast<uint32_t *>(base + r.off_dir);
    a.csum = reinterpret_cast<uint32_t *>(base + r.off_csum);
    a.S = reinterpret_cast<uint32_t *>(base + r.off_S);
    a.R = reinterpret_cast<uint32_t *>(base + r.off_R);
    a.smp = reinterpret_cast<uint32_t *>(base + r.off_smp);
    a.NS = r.NS;
    a.n = n;
    a.W = r.W;
    a.NB = r.NB;
    a.nchunks = r.nchunks;
    a.L = r.L;
    a.kind = (uint32_t)kind;
    return a;
}

wt_status check_query(wt_kind kind, const uint64_t *bv, const uint64_t *zeros, const void *rs, uint64_t n,
                      uint64_t sigma, RsLayout &r)
{
    wt_status st = layout(kind, n, sigma, r);
    if (st != WT_OK) return st;
    if (rs == nullptr) return WT_ERR_INVALID_ARG;
    if (r.L > 0 && n > 0 && bv == nullptr) return WT_ERR_INVALID_ARG;
    if (kind == WT_MATRIX && r.L > 0 && zeros == nullptr) return WT_ERR_INVALID_ARG;
    return WT_OK;
}

}  // namespace
}  // namespace wtg

using namespace wtg;

extern "C" {

wt_status wt_rank_support_size(wt_kind kind, uint64_t n, uint64_t sigma, size_t *bytes)
{
    if (bytes == nullptr) return WT_ERR_INVALID_ARG;
    RsLayout r;
    wt_status st = layout(kind, n, sigma, r);
    if (st == WT_OK) *bytes = r.bytes;
    return st;
}

wt_status wt_rank_support_build(wt_kind kind, const uint64_t *d_bv, const uint64_t *d_zeros, uint64_t n,
                                uint64_t sigma, void *d_rs, size_t rs_bytes, void *stream)
{
    RsLayout r;
    wt_status st = check_query(kind, d_bv, d_zeros, d_rs, n, sigma, r);
    if (st != WT_OK) return st;
    if (rs_bytes < r.bytes) return WT_ERR_OUT_OF_MEMORY;
    if (r.L == 0) return WT_OK;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    QArgs a = make_args(r, kind, d_bv, d_zeros, d_rs, n);
    const dim3 grid((uint32_t)r.nchunks, r.L);
    k_dir_chunks<<<grid, 1024, 0, s>>>(a);
    k_dir_chunk_scan<<<r.L, 1024, 0, s>>>(a);
    k_dir_apply<<<grid, 1024, 0, s>>>(a);
    k_select_samples<<<dim3((uint32_t)((r.NB + 255) / 256), r.L), 256, 0, s>>>(a);
    if (kind == WT_TREE)
        for (uint32_t l = 0; l < r.L; ++l) {
            const uint64_t threads = (1ull << l) + 1;
            k_tree_nodes<<<(uint32_t)((threads + 255) / 256), 256, 0, s>>>(a, l);
        }
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

wt_status wt_access(wt_kind kind, const uint64_t *d_bv, const uint64_t *d_zeros, const void *d_rs, uint64_t n,
                    uint64_t sigma, const uint64_t *d_pos, uint32_t count, uint32_t *d_out, void *stream)
{
    RsLayout r;
    wt_status st = check_query(kind, d_bv, d_zeros, d_rs, n, sigma, r);
    if (st != WT_OK) return st;
    if (count == 0) return WT_OK;
    if (d_pos == nullptr || d_out == nullptr) return WT_ERR_INVALID_ARG;
    QArgs a = make_args(r, kind, d_bv, d_zeros, d_rs, n);
    k_access<<<(count + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(a, d_pos, count, d_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

wt_status wt_rank(wt_kind kind, const uint64_t *d_bv, const uint64_t *d_zeros, const void *d_rs, uint64_t n,
                  uint64_t sigma, const uint32_t *d_sym, const uint64_t *d_pos, uint32_t count, uint64_t *d_out,
                  void *stream)
{
    RsLayout r;
    wt_status st = check_query(kind, d_bv, d_zeros, d_rs, n, sigma, r);
    if (st != WT_OK) return st;
    if (count == 0) return WT_OK;
    if (d_sym == nullptr || d_pos == nullptr || d_out == nullptr) return WT_ERR_INVALID_ARG;
    QArgs a = make_args(r, kind, d_bv, d_zeros, d_rs, n);
    k_rank<<<(count + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(a, d_sym, d_pos, count, d_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

wt_status wt_select(wt_kind kind, const uint64_t *d_bv, const uint64_t *d_zeros, const void *d_rs, uint64_t n,
                    uint64_t sigma, const uint32_t *d_sym, const uint64_t *d_j, uint32_t count, uint64_t *d_out,
                    void *stream)
{
    RsLayout r;
    wt_status st = check_query(kind, d_bv, d_zeros, d_rs, n, sigma, r);
    if (st != WT_OK) return st;
    if (count == 0) return WT_OK;
    if (d_sym == nullptr || d_j == nullptr || d_out == nullptr) return WT_ERR_INVALID_ARG;
    QArgs a = make_args(r, kind, d_bv, d_zeros, d_rs, n);
    k_select<<<(count + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(a, d_sym, d_j, count, d_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Lemma 3: WT position -> WM position.  U = 1^Hist[0] 0 1^Hist[1] 0 ... (one run
// of ones per character of [0, 2^L), each followed by a zero) with rank/select,
// and X = the WM interval starts of levels 1 .. L-1, level l at X[2^l - 2 + p]
// (the proof's indexing; the statement's 2^(l-1) - 2 disagrees with the stated
// storage range X[2^l - 2, 2^(l+1))).  The histogram is read off the WT's node
// tables: node p of level L-1 holds characters 2p and 2p+1.

namespace wtg {
namespace {

struct MapLayout {
    RsLayout wt;                  // the WT rank support this map is built from
    uint32_t L = 0;
    uint64_t ubits = 0, uW = 0, uNB = 0, unchunks = 0;
    size_t off_u = 0, off_udir = 0, off_ucsum = 0, off_x = 0, off_xsum = 0, bytes = 0;
};

constexpr uint32_t kXChunk = 4096;     // nodes per block of the X scan of a large level

wt_status map_layout(uint64_t n, uint64_t sigma, MapLayout &m)
{
    wt_status st = layout(WT_TREE, n, sigma, m.wt);
    if (st != WT_OK) return st;
    m.L = m.wt.L;
    m.ubits = n + (1ull << m.L);
    m.uW = (m.ubits + 63) / 64;
    m.uNB = (m.uW + 3) / 4 + 1;
    m.unchunks = (m.uNB + kDirChunk - 1) / kDirChunk;
    size_t off = 0;
    m.off_u = off;
    off = align256(off + 8 * m.uW);
    m.off_udir = off;
    off = align256(off + 4 * m.uNB);
    m.off_ucsum = off;
    off = align256(off + 4 * m.unchunks);
    m.off_x = off;
    off = align256(off + 4 * (m.L >= 1 ? (1ull << m.L) : 1ull));
    m.off_xsum = off;                  // chunk totals of the largest level's scan
    off = align256(off + 4 * ((m.L >= 2 ? (1ull << (m.L - 1)) : 1ull) / kXChunk + 1));
    m.bytes = off;
    return WT_OK;
}

QArgs u_args(const MapLayout &m, void *d_map)
{
    uint8_t *b = static_cast<uint8_t *>(d_map);
    QArgs a{};
    a.bv = reinterpret_cast<const uint64_t *>(b + m.off_u);
    a.dir = reinterpret_cast<const uint32_t *>(b + m.off_udir);
    a.dirw = reinterpret_cast<uint32_t *>(b + m.off_udir);
    a.csum = reinterpret_cast<uint32_t *>(b + m.off_ucsum);
    a.n = m.ubits;
    a.W = m.uW;
    a.NB = m.uNB;
    a.nchunks = m.unchunks;
    a.L = 1;
    return a;
}

// U: ones everywhere below ubits, zeros above
__global__ void k_u_fill(uint64_t *u, uint64_t uW, uint64_t ubits)
{
    const uint64_t w = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (w >= uW) return;
    const uint64_t lo = w * 64;
    u[w] = lo + 64 <= ubits ? ~0ull : (ubits > lo ? (1ull << (ubits - lo)) - 1ull : 0ull);
}

// the zero after character c's run: position (characters <= c) + c
__global__ void k_u_zeros(QArgs wt, uint64_t *u)
{
    const uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;   // node of level L-1
    const uint32_t l = wt.L - 1;
    if (p >= (1ull << l)) return;
    const uint32_t s = wt.S[tbl_off(l) + p], e = wt.S[tbl_off(l) + p + 1];
    const uint32_t ones = wt.R[tbl_off(l) + p + 1] - wt.R[tbl_off(l) + p];
    const uint64_t c0 = 2 * p, c1 = 2 * p + 1;
    const uint64_t end0 = (uint64_t)s + ((e - s) - ones);               // characters <= c0
    const uint64_t end1 = e;                                            // characters <= c1
    const uint64_t z0 = end0 + c0, z1 = end1 + c1;
    atomicAnd(reinterpret_cast<unsigned long long *>(u + (z0 >> 6)), ~(1ull << (z0 & 63)));
    atomicAnd(reinterpret_cast<unsigned long long *>(u + (z1 >> 6)), ~(1ull << (z1 & 63)));
}

// X of level l: the exclusive scan of the level's interval sizes in bit-reversal
// order (Sec. 5.1); sizes from the WT node starts.  Node r of the scan order is
// p = rho_l(r); X[2^l - 2 + p] receives its start.  Levels with more than kXChunk
// nodes are scanned by one block per chunk of the order: the chunk totals first
// (pass 0), their scan, then the chunks with their carries (pass 1).
__device__ __forceinline__ uint32_t x_size(const QArgs &wt, uint32_t l, uint64_t r)
{
    const uint32_t p = __brev((uint32_t)r) >> (32 - l);
    const uint32_t *S = wt.S + tbl_off(l);
    return S[p + 1] - S[p];
}

// chunk c of level l (kXChunk nodes, 4 per thread): totals (pass 0) or starts (pass 1)
__global__ void __launch_bounds__(1024) k_x_chunks(QArgs wt, uint32_t *X, uint32_t *xsum, uint32_t l, uint32_t pass)
{
    __shared__ uint32_t ws[32];
    const uint64_t cnt = 1ull << l, r0 = (uint64_t)blockIdx.x * kXChunk + 4ull * threadIdx.x;
    uint32_t v[4], t = 0;
    for (int j = 0; j < 4; ++j) {
        v[j] = r0 + j < cnt ? x_size(wt, l, r0 + j) : 0u;
        t += v[j];
    }
    uint32_t total;
    uint32_t run = block_scan_1024(t, ws, &total);
    if (pass == 0) {
        if (threadIdx.x == 0) xsum[blockIdx.x] = total;
        return;
    }
    run += xsum[blockIdx.x];
    for (int j = 0; j < 4; ++j) {
        if (r0 + j < cnt) X[cnt - 2 + (__brev((uint32_t)(r0 + j)) >> (32 - l))] = run;
        run += v[j];
    }
}

// one block: a whole small level (pass 0), or the exclusive scan of xsum (pass 1)
__global__ void __launch_bounds__(1024) k_x_level(QArgs wt, uint32_t *X, uint32_t *xsum, uint32_t l, uint32_t nchunks)
{
    __shared__ uint32_t ws[32];
    const uint64_t cnt = 1ull << l;
    if (nchunks == 0) {
        uint32_t carry = 0;
        for (uint64_t r0 = 0; r0 < cnt; r0 += 1024) {
            const uint64_t r = r0 + threadIdx.x;
            const uint32_t sz = r < cnt ? x_size(wt, l, r) : 0u;
            uint32_t total;
            const uint32_t ex = block_scan_1024(sz, ws, &total);
            if (r < cnt) X[cnt - 2 + (__brev((uint32_t)r) >> (32 - l))] = carry + ex;
            carry += total;
        }
        return;
    }
    uint32_t carry = 0;
    for (uint32_t c0 = 0; c0 < nchunks; c0 += 1024) {
        const uint32_t c = c0 + threadIdx.x;
        const uint32_t v = c < nchunks ? xsum[c] : 0u;
        uint32_t total;
        const uint32_t ex = block_scan_1024(v, ws, &total);
        if (c < nchunks) xsum[c] = carry + ex;
        carry += total;
    }
}

__global__ void k_wt2wm(QArgs u, const uint32_t *X, uint32_t L, uint64_t n, const uint32_t *lvl, const uint64_t *pos,
                        uint32_t count, uint64_t *out)
{
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= count) return;
    const uint32_t l = lvl[k];
    const uint64_t i = pos[k];
    if (l >= L || i >= n) { out[k] = kNone; return; }
    if (l <= 1) { out[k] = i; return; }
    const uint64_t t = select_bit(u, 0, i, true);            // the (i+1)-th one
    const uint64_t ch = t - i;                                 // rank0(U, t): its character
    const uint64_t bp = ch >> (L - l);
    const uint64_t first = bp << (L - l);                      // smallest character with prefix bp
    const uint64_t start = first == 0 ? 0 : select_bit(u, 0, first - 1, false) - (first - 1);
    out[k] = X[(1ull << l) - 2 + bp] + (i - start);
}

}  // namespace
}  // namespace wtg

extern "C" {

wt_status wt_wt2wm_size(uint64_t n, uint64_t sigma, size_t *bytes)
{
    if (bytes == nullptr) return WT_ERR_INVALID_ARG;
    wtg::MapLayout m;
    wt_status st = wtg::map_layout(n, sigma, m);
    if (st == WT_OK) *bytes = m.bytes;
    return st;
}

wt_status wt_wt2wm_build(const uint64_t *d_bv, const void *d_rs, uint64_t n, uint64_t sigma, void *d_map,
                         size_t map_bytes, void *stream)
{
    using namespace wtg;
    MapLayout m;
    wt_status st = map_layout(n, sigma, m);
    if (st != WT_OK) return st;
    if (d_rs == nullptr || d_map == nullptr || (n > 0 && d_bv == nullptr)) return WT_ERR_INVALID_ARG;
    if (map_bytes < m.bytes) return WT_ERR_OUT_OF_MEMORY;
    if (m.L < 2) return WT_OK;                                  // levels 0 and 1 map to themselves
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    QArgs wt = make_args(m.wt, WT_TREE, d_bv, nullptr, d_rs, n);
    QArgs u = u_args(m, d_map);
    uint64_t *ubits = const_cast<uint64_t *>(u.bv);
    k_u_fill<<<(uint32_t)((m.uW + 255) / 256), 256, 0, s>>>(ubits, m.uW, m.ubits);
    k_u_zeros<<<(uint32_t)(((1ull << (m.L - 1)) + 255) / 256), 256, 0, s>>>(wt, ubits);
    const dim3 grid((uint32_t)m.unchunks, 1);
    k_dir_chunks<<<grid, 1024, 0, s>>>(u);
    k_dir_chunk_scan<<<1, 1024, 0, s>>>(u);
    k_dir_apply<<<grid, 1024, 0, s>>>(u);
    uint32_t *X = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(d_map) + m.off_x);
    uint32_t *xsum = reinterpret_cast<uint32_t *>(static_cast<uint8_t *>(d_map) + m.off_xsum);
    for (uint32_t l = 1; l < m.L; ++l) {
        const uint64_t cnt = 1ull << l;
        if (cnt <= kXChunk) {
            k_x_level<<<1, 1024, 0, s>>>(wt, X, xsum, l, 0u);
        } else {
            const uint32_t chunks = (uint32_t)(cnt / kXChunk);
            k_x_chunks<<<chunks, 1024, 0, s>>>(wt, X, xsum, l, 0u);
            k_x_level<<<1, 1024, 0, s>>>(wt, X, xsum, l, chunks);
            k_x_chunks<<<chunks, 1024, 0, s>>>(wt, X, xsum, l, 1u);
        }
    }
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

wt_status wt_wt2wm(const void *d_map, uint64_t n, uint64_t sigma, const uint32_t *d_level, const uint64_t *d_pos,
                   uint32_t count, uint64_t *d_out, void *stream)
{
    using namespace wtg;
    MapLayout m;
    wt_status st = map_layout(n, sigma, m);
    if (st != WT_OK) return st;
    if (count == 0) return WT_OK;
    if (d_map == nullptr || d_level == nullptr || d_pos == nullptr || d_out == nullptr) return WT_ERR_INVALID_ARG;
    QArgs u = u_args(m, const_cast<void *>(d_map));
    const uint32_t *X = reinterpret_cast<const uint32_t *>(static_cast<const uint8_t *>(d_map) + m.off_x);
    k_wt2wm<<<(count + 255) / 256, 256, 0, static_cast<cudaStream_t>(stream)>>>(u, X, m.L, n, d_level, d_pos, count,
                                                                               d_out);
    return cudaGetLastError() == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

}  // extern "C"
