/*
 * Reference oracle for wavelet tree (WT) and wavelet matrix (WM) construction.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only the test suite, the smoke check and the CPU-baseline leg of
 * the benchmark do.  It shares no code, header or table with the CUDA library.
 *
 * Everything here is plain, single-threaded and slow on purpose.  It follows
 * Fischer, Kurpicz, Loebel, "Simple, Fast and Lightweight Parallel Wavelet Tree
 * Construction" (arXiv:1702.07578):
 *
 *   bit(k, a)     k-th most significant bit of the L-bit code of a (Sec. 2)
 *   prefix(k, a)  the k most significant bits of a (Sec. 2)
 *   WT            level-wise wavelet tree (Sec. 2, "Wavelet Trees", Obs. 1)
 *   WM            wavelet matrix with zero counts Z (Sec. 5, "Wavelet Matrices")
 *
 * Output convention (the paper leaves the bit order inside a word open):
 * level l occupies words [l*W, (l+1)*W) with W = ceil(n/64); bit j of a level
 * is bit (j & 63) of word (j >> 6), least significant bit first; bits >= n in
 * the last word are zero.
 *
 * Functions:
 *   oracle_wt_topdown  WT straight from the node definition (Sec. 2)
 *   oracle_wm_topdown  WM straight from its definition (Sec. 5)
 *   oracle_pc          Algorithm 1 (pcWT; pcWM with the bit-reversal order, Sec. 5.1)
 *   oracle_ps          Algorithm 2 (psWT/psWM) executed slice after slice
 *
 * Readings of the paper taken here (each is listed with its reason in the
 * design notes of the repository):
 *   - levels are 0-based and level l is keyed by prefix(l, .) as in Alg. 1 and
 *     Obs. 1 (the prose of Sec. 3.1 counts from 1);
 *   - Alg. 1 never resets the start of the first interval although the scan
 *     post-increments it and the array is reused: the start of the first
 *     interval is set to 0 at every level;
 *   - the alphabet is treated as [0, 2^L) with L = ceil(lg sigma): every node
 *     splits on one bit (the bit-prefix definition of Obs. 1), and the
 *     histogram has 2^L zero-initialised entries;
 *   - Z[l] is the number of zeros of level l, which equals the number of
 *     symbols whose prefix(l+1, .) is even (Sec. 5.1); all L entries are given.
 *
 * Return value of every function: 0 on success, -1 on an argument error
 * (null pointer, bad width, L > 32), -2 when a symbol is >= 2^L, -3 when
 * memory for the scratch arrays cannot be obtained.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- symbol access and bit helpers (Sec. 2) ---------------------------- */

static uint32_t sym_at(const void *T, int w, uint64_t i)
{
    if (w == 1) return ((const uint8_t *)T)[i];
    if (w == 2) return ((const uint16_t *)T)[i];
    return ((const uint32_t *)T)[i];
}

/* bit(k, a): k counts from the most significant of the L code bits. */
static uint32_t bit_of(uint32_t a, uint32_t k, uint32_t L)
{
    return (a >> (L - 1u - k)) & 1u;
}

/* prefix(k, a): the k most significant of the L code bits. */
static uint32_t prefix_of(uint32_t a, uint32_t k, uint32_t L)
{
    if (k == 0) return 0;
    return (uint32_t)((uint64_t)a >> (L - k));
}

/* pi_k(i): reverse the k-bit binary representation of i (Sec. 5). */
static uint32_t bit_reverse(uint32_t i, uint32_t k)
{
    uint32_t r = 0;
    for (uint32_t b = 0; b < k; ++b) r |= ((i >> b) & 1u) << (k - 1u - b);
    return r;
}

static uint64_t words_per_level(uint64_t n) { return (n + 63u) >> 6; }

static void set_bit(uint64_t *level, uint64_t j, uint32_t v)
{
    if (v) level[j >> 6] |= (uint64_t)1 << (j & 63u);
}

static int check_args(const void *T, int w, uint64_t n, uint32_t L, const uint64_t *bv)
{
    if (w != 1 && w != 2 && w != 4) return -1;
    if (L > 32) return -1;
    if (n > 0 && L > 0 && (T == NULL || bv == NULL)) return -1;
    for (uint64_t i = 0; i < n; ++i)
        if (L < 32 && (uint64_t)sym_at(T, w, i) >> L) return -2;
    return 0;
}

uint32_t oracle_levels(uint64_t sigma)
{
    uint32_t L = 0;
    while (L < 64 && ((uint64_t)1 << L) < sigma) ++L;
    return L;
}

/* ---- WT from the node definition (Sec. 2) ------------------------------
 * The root holds T.  A node at depth d stores bit(d, .) of its symbols in
 * their order, and hands the symbols whose bit is 0 (kept in order) to its
 * left child and the others (kept in order) to its right child.  Concatenating
 * the node bit vectors of depth d from left to right gives level d.
 * Nodes are kept as explicit [begin, end) ranges of the current sequence. */
int oracle_wt_topdown(const void *T, int w, uint64_t n, uint32_t L, uint64_t *bv)
{
    int rc = check_args(T, w, n, L, bv);
    if (rc) return rc;
    uint64_t W = words_per_level(n);
    if (L == 0 || n == 0) return 0;
    memset(bv, 0, (size_t)(L * W) * sizeof(uint64_t));

    uint32_t *seq = malloc(n * sizeof(uint32_t));
    uint32_t *nxt = malloc(n * sizeof(uint32_t));
    uint64_t *node_b = malloc(((size_t)1 << (L < 31 ? L : 31)) * 2 * sizeof(uint64_t));
    if (!seq || !nxt || !node_b) { free(seq); free(nxt); free(node_b); return -3; }
    uint64_t *node_e = node_b + ((size_t)1 << (L < 31 ? L : 31));
    for (uint64_t i = 0; i < n; ++i) seq[i] = sym_at(T, w, i);

    uint64_t nodes = 1;
    node_b[0] = 0;
    node_e[0] = n;
    for (uint32_t d = 0; d < L; ++d) {
        uint64_t *level = bv + (uint64_t)d * W;
        for (uint64_t j = 0; j < n; ++j) set_bit(level, j, bit_of(seq[j], d, L));
        if (d + 1 == L) break;
        /* split every node: zeros first, then ones, each in their order */
        uint64_t child = 2 * nodes;
        for (uint64_t v = nodes; v-- > 0;) {
            uint64_t b = node_b[v], e = node_e[v], out = b;
            for (uint64_t j = b; j < e; ++j)
                if (bit_of(seq[j], d, L) == 0) nxt[out++] = seq[j];
            uint64_t mid = out;
            for (uint64_t j = b; j < e; ++j)
                if (bit_of(seq[j], d, L) == 1) nxt[out++] = seq[j];
            node_b[2 * v] = b;   node_e[2 * v] = mid;
            node_b[2 * v + 1] = mid; node_e[2 * v + 1] = e;
        }
        nodes = child;
        uint32_t *t = seq; seq = nxt; nxt = t;
    }
    free(seq); free(nxt); free(node_b);
    return 0;
}

/* ---- WM from its definition (Sec. 5) -----------------------------------
 * Level 0 holds bit(0, .) of T in text order.  A symbol at position i of
 * level l moves to position rank0(BV_l, i) of level l+1 when its bit is 0,
 * and to Z[l] + rank1(BV_l, i) otherwise; Z[l] is the number of zeros of
 * level l. */
int oracle_wm_topdown(const void *T, int w, uint64_t n, uint32_t L, uint64_t *bv, uint64_t *Z)
{
    int rc = check_args(T, w, n, L, bv);
    if (rc) return rc;
    if (L > 0 && Z == NULL) return -1;
    uint64_t W = words_per_level(n);
    for (uint32_t d = 0; d < L; ++d) Z[d] = 0;
    if (L == 0 || n == 0) return 0;
    memset(bv, 0, (size_t)(L * W) * sizeof(uint64_t));

    uint32_t *seq = malloc(n * sizeof(uint32_t));
    uint32_t *nxt = malloc(n * sizeof(uint32_t));
    if (!seq || !nxt) { free(seq); free(nxt); return -3; }
    for (uint64_t i = 0; i < n; ++i) seq[i] = sym_at(T, w, i);

    for (uint32_t d = 0; d < L; ++d) {
        uint64_t *level = bv + (uint64_t)d * W;
        uint64_t zeros = 0;
        for (uint64_t j = 0; j < n; ++j) {
            uint32_t b = bit_of(seq[j], d, L);
            set_bit(level, j, b);
            zeros += (b == 0);
        }
        Z[d] = zeros;
        if (d + 1 == L) break;
        uint64_t rank0 = 0, rank1 = 0;
        for (uint64_t j = 0; j < n; ++j) {
            if (bit_of(seq[j], d, L) == 0) nxt[rank0++] = seq[j];
            else nxt[zeros + rank1++] = seq[j];
        }
        uint32_t *t = seq; seq = nxt; nxt = t;
    }
    free(seq); free(nxt);
    return 0;
}

/* ---- Algorithm 1: pcWT, and pcWM with id = pi_l (Sec. 3.1, Sec. 5.1) ----
 * One scan fills the leaf histogram and level 0.  Then, from the last level
 * up to level 1: fold the histogram to prefixes of length l, compute the
 * interval starts in id order, and scan T once more, writing bit(l, T[i]) at
 * the start of the interval of prefix(l, T[i]) and advancing that start. */
int oracle_pc(int matrix, const void *T, int w, uint64_t n, uint32_t L, uint64_t *bv, uint64_t *Z)
{
    int rc = check_args(T, w, n, L, bv);
    if (rc) return rc;
    if (matrix && L > 0 && Z == NULL) return -1;
    if (L > 30) return -1;
    uint64_t W = words_per_level(n);
    if (matrix) for (uint32_t d = 0; d < L; ++d) Z[d] = 0;
    if (L == 0 || n == 0) return 0;
    memset(bv, 0, (size_t)(L * W) * sizeof(uint64_t));

    size_t H = (size_t)1 << L;
    uint64_t *hist = calloc(H, sizeof(uint64_t));
    uint64_t *spos = calloc(H, sizeof(uint64_t));
    if (!hist || !spos) { free(hist); free(spos); return -3; }

    for (uint64_t i = 0; i < n; ++i) {
        uint32_t a = sym_at(T, w, i);
        hist[a]++;
        set_bit(bv, i, bit_of(a, 0, L));
    }
    for (uint32_t l = L - 1; l >= 1; --l) {
        uint32_t cnt = 1u << l;
        if (matrix) {               /* zeros of level l: even (l+1)-prefixes */
            uint64_t z = 0;
            for (uint32_t p = 0; p < 2u * cnt; p += 2) z += hist[p];
            Z[l] = z;
        }
        for (uint32_t i = 0; i < cnt; ++i) hist[i] = hist[2 * i] + hist[2 * i + 1];
        spos[matrix ? bit_reverse(0, l) : 0] = 0;
        for (uint32_t i = 1; i < cnt; ++i) {
            uint32_t cur = matrix ? bit_reverse(i, l) : i;
            uint32_t prv = matrix ? bit_reverse(i - 1, l) : i - 1;
            spos[cur] = spos[prv] + hist[prv];
        }
        uint64_t *level = bv + (uint64_t)l * W;
        for (uint64_t i = 0; i < n; ++i) {
            uint32_t a = sym_at(T, w, i);
            uint64_t pos = spos[prefix_of(a, l, L)]++;
            set_bit(level, pos, bit_of(a, l, L));
        }
    }
    if (matrix) Z[0] = hist[0];      /* hist now holds the 1-prefix counts */
    free(hist); free(spos);
    return 0;
}

/* ---- Algorithm 2: psWT / psWM (Sec. 3.2.1, Sec. 5.1) ----------------------
 * The text is cut into p slices of (nearly) equal length.  Slice c keeps its
 * own histogram Hist_c.  At each level the per-slice interval starts SPos_c
 * are one zero-based prefix sum over the sequence
 *   Hist_0[id(0)], ..., Hist_{p-1}[id(0)], Hist_0[id(1)], ...,
 * the text is counting-sorted by its l-prefixes with these starts (slice c
 * placing its symbols in its order), and level l is bit(l, .) of the sorted
 * text in order.  The slices are processed one after the other here. */
int oracle_ps(int matrix, const void *T, int w, uint64_t n, uint32_t L, uint32_t p,
              uint64_t *bv, uint64_t *Z)
{
    int rc = check_args(T, w, n, L, bv);
    if (rc) return rc;
    if (p == 0 || L > 24) return -1;
    if (matrix && L > 0 && Z == NULL) return -1;
    uint64_t W = words_per_level(n);
    if (matrix) for (uint32_t d = 0; d < L; ++d) Z[d] = 0;
    if (L == 0 || n == 0) return 0;
    memset(bv, 0, (size_t)(L * W) * sizeof(uint64_t));

    size_t H = (size_t)1 << L;
    uint64_t *hist = calloc(H * p, sizeof(uint64_t));
    uint64_t *spos = calloc(H * p, sizeof(uint64_t));
    uint32_t *sorted = malloc(n * sizeof(uint32_t));
    if (!hist || !spos || !sorted) { free(hist); free(spos); free(sorted); return -3; }

    uint64_t *sb = malloc((size_t)(p + 1) * sizeof(uint64_t));
    if (!sb) { free(hist); free(spos); free(sorted); return -3; }
    for (uint32_t c = 0; c <= p; ++c) sb[c] = n * c / p;

    for (uint32_t c = 0; c < p; ++c)
        for (uint64_t i = sb[c]; i < sb[c + 1]; ++i) {
            uint32_t a = sym_at(T, w, i);
            hist[(size_t)c * H + a]++;
            set_bit(bv, i, bit_of(a, 0, L));
        }
    for (uint32_t l = L - 1; l >= 1; --l) {
        uint32_t cnt = 1u << l;
        if (matrix) {
            uint64_t z = 0;
            for (uint32_t c = 0; c < p; ++c)
                for (uint32_t q = 0; q < 2u * cnt; q += 2) z += hist[(size_t)c * H + q];
            Z[l] = z;
        }
        for (uint32_t c = 0; c < p; ++c)
            for (uint32_t i = 0; i < cnt; ++i)
                hist[(size_t)c * H + i] = hist[(size_t)c * H + 2 * i] + hist[(size_t)c * H + 2 * i + 1];
        uint64_t run = 0;            /* zero-based prefix sum, interleaved order */
        for (uint32_t i = 0; i < cnt; ++i) {
            uint32_t key = matrix ? bit_reverse(i, l) : i;
            for (uint32_t c = 0; c < p; ++c) {
                spos[(size_t)c * H + key] = run;
                run += hist[(size_t)c * H + key];
            }
        }
        for (uint32_t c = 0; c < p; ++c)  /* counting sort by l-prefix */
            for (uint64_t i = sb[c]; i < sb[c + 1]; ++i) {
                uint32_t a = sym_at(T, w, i);
                sorted[spos[(size_t)c * H + prefix_of(a, l, L)]++] = a;
            }
        uint64_t *level = bv + (uint64_t)l * W;
        for (uint64_t i = 0; i < n; ++i) set_bit(level, i, bit_of(sorted[i], l, L));
    }
    if (matrix) {
        uint64_t z = 0;
        for (uint32_t c = 0; c < p; ++c) z += hist[(size_t)c * H + 0];
        Z[0] = z;
    }
    free(hist); free(spos); free(sorted); free(sb);
    return 0;
}
