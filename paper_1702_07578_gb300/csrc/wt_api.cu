// C ABI of wt_gb300: argument checks, workspace planning and round launches
// for wt_build / wm_build / wt_build_batched.  See include/wt_gb300.h.
#include <algorithm>
#include <mutex>
#include <vector>

#include "wt_internal.h"

namespace wtg {
namespace {

struct HostText {
    const void *text;
    uint64_t n;
    uint64_t sigma;
    uint64_t *bv;
    uint64_t *zeros;
    uint64_t *bv2 = nullptr;     // kBoth: the WM's levels (bv holds the WT's)
    uint32_t *perm = nullptr;    // the stable order after the last level
    bool order = false;          // perm is wanted (size queries pass no pointer)
};

struct Plan {
    uint32_t count = 0;
    uint32_t rounds = 0;
    uint32_t nslots[kMaxRounds] = {};
    uint32_t groups_ub[kMaxRounds] = {};
    uint32_t blocks_ub[kMaxRounds] = {};
    uint32_t width[kMaxRounds] = {};
    uint32_t gelems[kMaxRounds] = {};     // symbols per build block in each round
    size_t off_ctl = 0, off_texts = 0, off_jobs[2] = {}, off_jobhist[2] = {};
    size_t off_ghist = 0, off_gexcl = 0, off_thist = 0, off_btail = 0, off_bflag = 0, off_bcarry = 0, off_cscan = 0;
    std::vector<size_t> off_buf[2];
    std::vector<size_t> off_pbuf[2];      // text positions carried through cut rounds (perm)
    std::vector<TextInfo> texts;
    size_t bytes = 0;
};

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

uint32_t levels_of(uint64_t sigma)
{
    uint32_t L = 0;
    while (L < 64 && (1ull << L) < sigma) ++L;
    return L;
}

// Smallest symbols-per-block choice; workspace sizes are computed with it, so any
// choice (a multiple of it) fits in a workspace of the reported size.
constexpr uint32_t kMinSpb = 32768;

// Rounds with fewer symbols than this many default groups (one wave of two build
// blocks per SM on 152 SMs) get one-tile groups, so that more blocks share the work.
constexpr uint32_t kSmallRoundGroups = 2 * 152;

bool valid_spb(uint32_t spb) { return spb == 0 || (spb % kMinSpb == 0 && spb <= (1u << 24)); }

// Checks the texts and lays out the workspace.  With check_ptrs == false only
// sizes are validated (workspace queries).  spb: symbols per build block
// (0 = the default for the round's symbol width).
wt_status make_plan(wt_kind kind, wt_symtype type, const HostText *t, uint32_t count, bool check_ptrs,
                    Plan &p, uint32_t spb = 0)
{
    if (!valid_spb(spb)) return WT_ERR_INVALID_ARG;
    const bool both = (uint32_t)kind == kBoth;
    if (kind != WT_TREE && kind != WT_MATRIX && !both) return WT_ERR_INVALID_ARG;
    if (type != WT_U8 && type != WT_U16 && type != WT_U32) return WT_ERR_INVALID_ARG;
    if (count > 0 && t == nullptr) return WT_ERR_INVALID_ARG;
    const uint32_t w = (uint32_t)type;
    p.count = count;
    p.texts.assign(count, TextInfo{});
    uint32_t max_slots = 0, max_groups = 0;
    uint64_t max_tiles = 0;
    uint64_t slot_acc[kMaxRounds] = {}, group_acc[kMaxRounds] = {};
    uint32_t width[kMaxRounds] = {};
    for (uint32_t i = 0; i < count; ++i) {
        const HostText &x = t[i];
        if (x.sigma == 0) return WT_ERR_INVALID_ARG;
        if (x.n >= (1ull << 32)) return WT_ERR_INVALID_ARG;
        if (w < 4 && x.sigma > (1ull << (8 * w))) return WT_ERR_INVALID_ARG;
        if (x.sigma > (1ull << 32)) return WT_ERR_INVALID_ARG;
        const uint32_t L = levels_of(x.sigma);
        if (kind == WT_TREE && L > (uint32_t)kMaxTreeSigmaLog) return WT_ERR_INVALID_ARG;
        if (both && (L > (uint32_t)kChunk || (x.n > 0 && x.n <= kSmallJob))) return WT_ERR_INVALID_ARG;
        if (both && x.order) return WT_ERR_INVALID_ARG;
        if (check_ptrs && x.order && x.n > 0 && (x.perm == nullptr || reinterpret_cast<uintptr_t>(x.perm) % 4))
            return WT_ERR_INVALID_ARG;
        if (check_ptrs && L > 0) {
            if (x.n > 0 && (x.text == nullptr || x.bv == nullptr)) return WT_ERR_INVALID_ARG;
            if ((kind == WT_MATRIX || both) && x.zeros == nullptr) return WT_ERR_INVALID_ARG;
            if (both && (x.bv2 == nullptr || reinterpret_cast<uintptr_t>(x.bv2) % 8)) return WT_ERR_INVALID_ARG;
            if (reinterpret_cast<uintptr_t>(x.text) % w) return WT_ERR_INVALID_ARG;
            if (reinterpret_cast<uintptr_t>(x.bv) % 8) return WT_ERR_INVALID_ARG;
        }
        TextInfo &ti = p.texts[i];
        ti.text = x.text;
        ti.bv = x.bv;
        ti.bv2 = both ? x.bv2 : nullptr;
        ti.perm = x.order ? x.perm : nullptr;
        ti.zeros = (kind == WT_MATRIX || both) ? x.zeros : nullptr;
        ti.n = x.n;
        ti.W = (x.n + 63) / 64;
        ti.sigma = x.sigma;
        ti.L = L;
        ti.in_w = w;
        const uint32_t rounds = round_count(L);
        if (rounds > p.rounds) p.rounds = rounds;
        for (uint32_t r = 0; r < kMaxRounds; ++r) {
            uint32_t ns = 0;                          // WT: one slot per prefix of the levels done
            if (x.n > 0 && r < rounds) ns = (kind == WT_TREE) ? (1u << round_first_level(L, r)) : 1u;
            ti.nslots[r] = ns;
            ti.slot_base[r] = (uint32_t)slot_acc[r];
            slot_acc[r] += ns;
            if (ns) {
                uint32_t wr = width_for_bits(L - round_first_level(L, r));
                if (wr > width[r]) width[r] = wr;
            }
        }
    }
    for (uint32_t r = 0; r < p.rounds; ++r) {
        if (slot_acc[r] >= (1ull << 31)) return WT_ERR_INVALID_ARG;
        p.width[r] = width[r] ? width[r] : 1;
        p.gelems[r] = spb ? spb : kDefaultGroup;
        if (!spb) {                   // less than one wave of default groups: one tile per group
            uint64_t syms = 0;
            for (uint32_t i = 0; i < count; ++i)
                if (p.texts[i].nslots[r]) syms += p.texts[i].n;
            if (syms < (uint64_t)kSmallRoundGroups * kDefaultGroup) p.gelems[r] = kMinSpb;
        }
        const uint64_t ge = p.gelems[r];
        for (uint32_t i = 0; i < count; ++i) {
            const TextInfo &ti = p.texts[i];
            const uint32_t ns = ti.nslots[r];
            if (!ns) continue;
            group_acc[r] += ns == 1 ? (ti.n + ge - 1) / ge : ti.n / ge + ns;
        }
        if (group_acc[r] >= (1ull << 31)) return WT_ERR_INVALID_ARG;
        p.nslots[r] = (uint32_t)slot_acc[r];
        p.groups_ub[r] = (uint32_t)group_acc[r];
        p.blocks_ub[r] = (p.groups_ub[r] + kRowsPerBlock - 1) / kRowsPerBlock;
        if (p.nslots[r] > max_slots) max_slots = p.nslots[r];
        if (p.groups_ub[r] > max_groups) max_groups = p.groups_ub[r];
        uint64_t tiles = 0;                       // rows of the tile histograms
        for (uint32_t i = 0; i < count; ++i) {
            const TextInfo &ti = p.texts[i];
            const uint32_t ns = ti.nslots[r];
            if (ns) tiles += ns == 1 ? (ti.n + kTileSyms - 1) / kTileSyms : ti.n / kTileSyms + ns;
        }
        if (tiles > max_tiles) max_tiles = tiles;
    }
    const uint32_t max_blocks = (max_groups + kRowsPerBlock - 1) / kRowsPerBlock;
    size_t off = 0;
    auto take = [&](size_t bytes) {
        size_t o = off;
        off = align_up(off + bytes, 256);
        return o;
    };
    p.off_ctl = take(sizeof(Ctl));
    p.off_texts = take(sizeof(TextInfo) * count);
    for (int k = 0; k < 2; ++k) p.off_jobs[k] = take(sizeof(Job) * max_slots);
    for (int k = 0; k < 2; ++k) p.off_jobhist[k] = take(sizeof(uint32_t) * kCols * (size_t)max_slots);
    p.off_ghist = take(sizeof(uint32_t) * kCols * (size_t)max_groups);
    p.off_gexcl = take(sizeof(uint32_t) * kCols * (size_t)max_groups);
    p.off_thist = take(sizeof(uint32_t) * kCols * (size_t)max_tiles);
    p.off_btail = take(sizeof(uint32_t) * kCols * (size_t)max_blocks);
    p.off_bcarry = take(sizeof(uint32_t) * kCols * (size_t)max_blocks);
    p.off_bflag = take(sizeof(uint32_t) * (size_t)max_blocks);
    p.off_cscan = take(sizeof(uint32_t) * 2 * ((size_t)max_slots / 4096 + 1));
    p.off_buf[0].assign(count, 0);
    p.off_buf[1].assign(count, 0);
    p.off_pbuf[0].assign(count, 0);
    p.off_pbuf[1].assign(count, 0);
    for (uint32_t i = 0; i < count; ++i) {
        const TextInfo &ti = p.texts[i];
        if (ti.n == 0) continue;
        // round r's re-sorted output (r = 0, 1; later rounds reuse them) holds the
        // code bits still to split after it
        const uint32_t R = round_count(ti.L);
        if (R > 1) p.off_buf[0][i] = take(ti.n * width_for_bits(ti.L - round_first_level(ti.L, 1)));
        if (R > 2) p.off_buf[1][i] = take(ti.n * width_for_bits(ti.L - round_first_level(ti.L, 2)));
        if (t[i].order && R > 1) p.off_pbuf[0][i] = take(ti.n * sizeof(uint32_t));
        if (t[i].order && R > 2) p.off_pbuf[1][i] = take(ti.n * sizeof(uint32_t));
    }
    p.bytes = off;
    return WT_OK;
}

std::mutex g_cfg_mu;
bool g_cfg_done[64] = {};

wt_status ensure_configured()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return WT_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_cfg_mu);
    if (dev >= 0 && dev < 64 && g_cfg_done[dev]) return WT_OK;
    if (configure_kernels() != cudaSuccess) return WT_ERR_CUDA;
    if (dev >= 0 && dev < 64) g_cfg_done[dev] = true;
    return WT_OK;
}

// Points the re-sorted text buffers of the plan into the workspace.
wt_status prepare(Plan &p, void *d_ws, size_t ws_bytes)
{
    if (d_ws == nullptr || ws_bytes < p.bytes) return WT_ERR_OUT_OF_MEMORY;
    if (reinterpret_cast<uintptr_t>(d_ws) % 256) return WT_ERR_INVALID_ARG;
    wt_status st = ensure_configured();
    if (st != WT_OK) return st;
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    for (uint32_t i = 0; i < p.count; ++i) {
        TextInfo &ti = p.texts[i];
        const uint32_t R = round_count(ti.L);
        ti.buf[0] = R > 1 ? ws + p.off_buf[0][i] : nullptr;
        ti.buf[1] = R > 2 ? ws + p.off_buf[1][i] : nullptr;
        ti.pbuf[0] = ti.perm && R > 1 ? reinterpret_cast<uint32_t *>(ws + p.off_pbuf[0][i]) : nullptr;
        ti.pbuf[1] = ti.perm && R > 2 ? reinterpret_cast<uint32_t *>(ws + p.off_pbuf[1][i]) : nullptr;
    }
    return WT_OK;
}

// Copies the text descriptors into the workspace (from `src`, host memory).
wt_status upload(const Plan &p, const TextInfo *src, void *d_ws, cudaStream_t s)
{
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    TextInfo *dtexts = reinterpret_cast<TextInfo *>(ws + p.off_texts);
    if (cudaMemcpyAsync(dtexts, src, sizeof(TextInfo) * p.count, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return WT_ERR_CUDA;
    return WT_OK;
}

// Every kernel of the build, in stream order; reads the descriptors from the
// workspace.  Nothing here touches host memory, so it can be captured in a graph.
wt_status launch(wt_kind kind, const Plan &p, void *d_ws, cudaStream_t s)
{
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    Ctl *ctl = reinterpret_cast<Ctl *>(ws + p.off_ctl);
    TextInfo *dtexts = reinterpret_cast<TextInfo *>(ws + p.off_texts);
    if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), s) != cudaSuccess) return WT_ERR_CUDA;
    if ((kind == WT_MATRIX || (uint32_t)kind == kBoth) && launch_zero_z(dtexts, p.count, s) != cudaSuccess)
        return WT_ERR_CUDA;
    for (uint32_t r = 0; r < p.rounds; ++r) {
        RoundArgs a{};
        a.ctl = ctl;
        a.texts = dtexts;
        a.jobs = reinterpret_cast<Job *>(ws + p.off_jobs[r & 1]);
        a.pjobs = reinterpret_cast<const Job *>(ws + p.off_jobs[(r + 1) & 1]);
        a.jobhist = reinterpret_cast<uint32_t *>(ws + p.off_jobhist[r & 1]);
        a.pjobhist = reinterpret_cast<const uint32_t *>(ws + p.off_jobhist[(r + 1) & 1]);
        a.ghist = reinterpret_cast<uint32_t *>(ws + p.off_ghist);
        a.gexcl = reinterpret_cast<uint32_t *>(ws + p.off_gexcl);
        a.thist = reinterpret_cast<uint32_t *>(ws + p.off_thist);
        a.btail = reinterpret_cast<uint32_t *>(ws + p.off_btail);
        a.bflag = reinterpret_cast<uint32_t *>(ws + p.off_bflag);
        a.bcarry = reinterpret_cast<uint32_t *>(ws + p.off_bcarry);
        a.cscan = reinterpret_cast<uint32_t *>(ws + p.off_cscan);
        a.ntexts = p.count;
        a.nslots = p.nslots[r];
        a.pnslots = r ? p.nslots[r - 1] : 0;
        a.round = r;
        a.kind = (uint32_t)kind;
        a.gelems = p.gelems[r];
        a.groups_ub = p.groups_ub[r];
        a.blocks_ub = p.blocks_ub[r];
        a.all_h8 = 1;
        uint32_t in_w = 1;                          // widest symbol read by the round
        for (uint32_t i = 0; i < p.count; ++i) {
            const TextInfo &ti = p.texts[i];
            if (ti.nslots[r] == 0) continue;
            if (round_levels(ti.L, r) != (uint32_t)kChunk) a.all_h8 = 0;
            const uint32_t w = r == 0 ? ti.in_w : width_for_bits(ti.L - round_first_level(ti.L, r));
            if (w > in_w) in_w = w;
            const bool last = r + 1 == round_count(ti.L);
            if (!last) a.any_cut = 1; else a.any_plain = 1;
            if (ti.perm != nullptr) a.any_order = 1;
            // small jobs (one warp each): the last round of a text that does not want its
            // order, where the WT's subtrees (r >= 1) may be small, or the whole text is
            if (last && ti.perm == nullptr &&
                ((kind == WT_TREE && r > 0) || (ti.n > 0 && ti.n <= kSmallJob)))
                a.any_small = 1;
        }
        if (launch_round(a, in_w, s) != cudaSuccess) return WT_ERR_CUDA;
    }
    return WT_OK;
}

wt_status run_plan(wt_kind kind, Plan &p, void *d_ws, size_t ws_bytes, cudaStream_t s)
{
    if (p.count == 0) return WT_OK;
    wt_status st = prepare(p, d_ws, ws_bytes);
    if (st == WT_OK) st = upload(p, p.texts.data(), d_ws, s);
    if (st == WT_OK) st = launch(kind, p, d_ws, s);
    return st;
}

wt_status single(wt_kind kind, const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *d_bv,
                 uint64_t *d_zeros, void *d_ws, size_t ws_bytes, void *stream)
{
    HostText h{d_text, n, sigma, d_bv, d_zeros};
    Plan p;
    wt_status st = make_plan(kind, type, &h, 1, true, p);
    if (st != WT_OK) return st;
    return run_plan(kind, p, d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

}  // namespace
}  // namespace wtg

using namespace wtg;

extern "C" {

uint32_t wt_levels(uint64_t sigma) { return levels_of(sigma); }

uint64_t wt_words_per_level(uint64_t n) { return (n + 63) / 64; }

const char *wt_status_string(wt_status s)
{
    switch (s) {
    case WT_OK: return "ok";
    case WT_ERR_INVALID_ARG: return "invalid argument";
    case WT_ERR_SYMBOL_RANGE: return "symbol out of range";
    case WT_ERR_OUT_OF_MEMORY: return "out of memory";
    case WT_ERR_CUDA: return "CUDA error";
    case WT_ERR_TIMEOUT: return "timeout";
    case WT_ERR_BUSY: return "busy";
    case WT_ERR_NOT_FOUND: return "not found";
    }
    return "unknown status";
}

wt_status wt_workspace_size(wt_kind kind, wt_symtype type, uint64_t n, uint64_t sigma, size_t *bytes)
{
    if (bytes == nullptr) return WT_ERR_INVALID_ARG;
    HostText h{nullptr, n, sigma, nullptr, nullptr};
    Plan p;
    wt_status st = make_plan(kind, type, &h, 1, false, p, kMinSpb);
    if (st == WT_OK) *bytes = p.bytes;
    return st;
}

wt_status wt_build(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *d_bv, void *d_ws,
                   size_t ws_bytes, void *stream)
{
    return single(WT_TREE, d_text, type, n, sigma, d_bv, nullptr, d_ws, ws_bytes, stream);
}

wt_status wm_build(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *d_bv,
                   uint64_t *d_zeros, void *d_ws, size_t ws_bytes, void *stream)
{
    return single(WT_MATRIX, d_text, type, n, sigma, d_bv, d_zeros, d_ws, ws_bytes, stream);
}

namespace {

// The fused pass applies to a text with L <= 8 and more than kSmallJob symbols.
bool fused_fits(uint64_t n, uint64_t sigma) { return levels_of(sigma) <= (uint32_t)kChunk && n > kSmallJob; }

}  // namespace

wt_status wt_wm_workspace_size(wt_symtype type, uint64_t n, uint64_t sigma, size_t *bytes)
{
    if (bytes == nullptr) return WT_ERR_INVALID_ARG;
    if (sigma > 0 && n < (1ull << 32) && fused_fits(n, sigma)) {
        HostText h{nullptr, n, sigma, nullptr, nullptr};
        Plan p;
        wt_status st = make_plan(static_cast<wt_kind>(kBoth), type, &h, 1, false, p, kMinSpb);
        if (st == WT_OK) *bytes = p.bytes;
        return st;
    }
    size_t a = 0, b = 0;
    wt_status st = wt_workspace_size(WT_TREE, type, n, sigma, &a);
    if (st == WT_OK) st = wt_workspace_size(WT_MATRIX, type, n, sigma, &b);
    if (st == WT_OK) *bytes = a > b ? a : b;
    return st;
}

wt_status wt_wm_build(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *d_bv_wt,
                      uint64_t *d_bv_wm, uint64_t *d_zeros, void *d_ws, size_t ws_bytes, void *stream)
{
    if (sigma == 0 || n >= (1ull << 32) || !fused_fits(n, sigma)) {
        wt_status st = single(WT_TREE, d_text, type, n, sigma, d_bv_wt, nullptr, d_ws, ws_bytes, stream);
        if (st != WT_OK) return st;
        return single(WT_MATRIX, d_text, type, n, sigma, d_bv_wm, d_zeros, d_ws, ws_bytes, stream);
    }
    HostText h{d_text, n, sigma, d_bv_wt, d_zeros, d_bv_wm};
    Plan p;
    wt_status st = make_plan(static_cast<wt_kind>(kBoth), type, &h, 1, true, p);
    if (st != WT_OK) return st;
    return run_plan(static_cast<wt_kind>(kBoth), p, d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

namespace {

wt_status build_order(wt_kind kind, const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma,
                      uint64_t *d_bv, uint64_t *d_zeros, uint32_t *d_perm, void *d_sorted, void *d_ws,
                      size_t ws_bytes, void *stream)
{
    HostText h{d_text, n, sigma, d_bv, d_zeros};
    h.perm = d_perm;
    h.order = true;
    Plan p;
    wt_status st = make_plan(kind, type, &h, 1, true, p);
    if (st != WT_OK) return st;
    if (n == 0) return WT_OK;
    if (d_perm == nullptr || d_text == nullptr) return WT_ERR_INVALID_ARG;
    if (d_sorted != nullptr && reinterpret_cast<uintptr_t>(d_sorted) % (uint32_t)type) return WT_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (levels_of(sigma) == 0) {                 // one symbol value: the text order
        if (ensure_configured() != WT_OK) return WT_ERR_CUDA;
        return launch_identity_order(d_text, (uint32_t)type, n, d_perm, d_sorted, s) == cudaSuccess ? WT_OK
                                                                                                    : WT_ERR_CUDA;
    }
    st = run_plan(kind, p, d_ws, ws_bytes, s);
    if (st != WT_OK || d_sorted == nullptr) return st;
    cudaError_t e;
    if (p.rounds == 1) {      // runs of equal symbols, lengths from the job's class totals
        const uint32_t *count = reinterpret_cast<const uint32_t *>(static_cast<uint8_t *>(d_ws) + p.off_jobhist[0]);
        e = launch_fill_runs(count, levels_of(sigma), kind == WT_MATRIX, n, d_sorted, (uint32_t)type, s);
    } else {
        e = launch_gather(d_text, (uint32_t)type, d_perm, n, d_sorted, s);
    }
    return e == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

}  // namespace

wt_status wt_order_workspace_size(wt_kind kind, wt_symtype type, uint64_t n, uint64_t sigma, size_t *bytes)
{
    if (bytes == nullptr) return WT_ERR_INVALID_ARG;
    HostText h{nullptr, n, sigma, nullptr, nullptr};
    h.order = true;
    Plan p;
    wt_status st = make_plan(kind, type, &h, 1, false, p, kMinSpb);
    if (st == WT_OK) *bytes = p.bytes;
    return st;
}

wt_status wt_build_order(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *d_bv,
                         uint32_t *d_perm, void *d_sorted, void *d_ws, size_t ws_bytes, void *stream)
{
    return build_order(WT_TREE, d_text, type, n, sigma, d_bv, nullptr, d_perm, d_sorted, d_ws, ws_bytes, stream);
}

wt_status wm_build_order(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *d_bv,
                         uint64_t *d_zeros, uint32_t *d_perm, void *d_sorted, void *d_ws, size_t ws_bytes,
                         void *stream)
{
    return build_order(WT_MATRIX, d_text, type, n, sigma, d_bv, d_zeros, d_perm, d_sorted, d_ws, ws_bytes,
                       stream);
}

}  // extern "C"

namespace {

// Device workspace of wt_build_host: the build workspace (the largest of the WT,
// WM and one-pass builds) at offset 0, then the text, the WT and WM levels and Z.
struct HostLayout {
    size_t text = 0, bv_wt = 0, bv_wm = 0, zeros = 0, bytes = 0;
};

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

wt_status host_layout(wt_symtype type, uint64_t n, uint64_t sigma, HostLayout &h)
{
    size_t a = 0, b = 0, c = 0;
    wt_status st = wt_workspace_size(WT_MATRIX, type, n, sigma, &b);
    if (st != WT_OK) return st;
    if (wt_workspace_size(WT_TREE, type, n, sigma, &a) != WT_OK) a = 0;    // alphabet beyond the WT's limit
    if (wt_wm_workspace_size(type, n, sigma, &c) != WT_OK) c = 0;
    const uint64_t L = levels_of(sigma), W = (n + 63) / 64;
    size_t off = align256(std::max(a, std::max(b, c)));
    h.text = off;
    off = align256(off + (size_t)n * (uint32_t)type);
    h.bv_wt = off;
    off = align256(off + (size_t)(L * W * 8));
    h.bv_wm = off;
    off = align256(off + (size_t)(L * W * 8));
    h.zeros = off;
    h.bytes = align256(off + 8 * (size_t)(L ? L : 1));
    return WT_OK;
}

}  // namespace

extern "C" {

wt_status wt_host_workspace_size(wt_symtype type, uint64_t n, uint64_t sigma, size_t *bytes)
{
    if (bytes == nullptr) return WT_ERR_INVALID_ARG;
    HostLayout h;
    wt_status st = host_layout(type, n, sigma, h);
    if (st == WT_OK) *bytes = h.bytes;
    return st;
}

wt_status wt_build_host(const void *h_text, wt_symtype type, uint64_t n, uint64_t sigma, uint64_t *h_bv_wt,
                        uint64_t *h_bv_wm, uint64_t *h_zeros, int one_pass, void *d_ws, size_t ws_bytes,
                        void *stream)
{
    if (d_ws == nullptr || (h_bv_wt == nullptr && h_bv_wm == nullptr)) return WT_ERR_INVALID_ARG;
    HostLayout h;
    wt_status st = host_layout(type, n, sigma, h);
    if (st != WT_OK) return st;
    if (ws_bytes < h.bytes) return WT_ERR_OUT_OF_MEMORY;
    const uint64_t L = levels_of(sigma), W = (n + 63) / 64;
    if (n > 0 && h_text == nullptr) return WT_ERR_INVALID_ARG;
    if (h_bv_wm != nullptr && L > 0 && h_zeros == nullptr) return WT_ERR_INVALID_ARG;
    if (h_bv_wt != nullptr && sigma > (1ull << 24)) return WT_ERR_INVALID_ARG;
    uint8_t *base = static_cast<uint8_t *>(d_ws);
    void *d_text = base + h.text;
    uint64_t *d_bv_wt = reinterpret_cast<uint64_t *>(base + h.bv_wt);
    uint64_t *d_bv_wm = reinterpret_cast<uint64_t *>(base + h.bv_wm);
    uint64_t *d_zeros = reinterpret_cast<uint64_t *>(base + h.zeros);
    const size_t bws = h.text;                   // the build workspace ends where the text starts
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (n > 0 && cudaMemcpyAsync(d_text, h_text, (size_t)n * (uint32_t)type, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return WT_ERR_CUDA;
    if (h_bv_wt != nullptr && h_bv_wm != nullptr && one_pass) {
        st = wt_wm_build(d_text, type, n, sigma, d_bv_wt, d_bv_wm, d_zeros, d_ws, bws, stream);
    } else {
        if (h_bv_wt != nullptr) st = wt_build(d_text, type, n, sigma, d_bv_wt, d_ws, bws, stream);
        if (st == WT_OK && h_bv_wm != nullptr) st = wm_build(d_text, type, n, sigma, d_bv_wm, d_zeros, d_ws, bws, stream);
    }
    if (st != WT_OK) return st;
    const size_t lvl = (size_t)(L * W * 8);
    if (lvl > 0 && h_bv_wt != nullptr && cudaMemcpyAsync(h_bv_wt, d_bv_wt, lvl, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return WT_ERR_CUDA;
    if (lvl > 0 && h_bv_wm != nullptr && cudaMemcpyAsync(h_bv_wm, d_bv_wm, lvl, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return WT_ERR_CUDA;
    if (L > 0 && h_bv_wm != nullptr && cudaMemcpyAsync(h_zeros, d_zeros, 8 * L, cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return WT_ERR_CUDA;
    return WT_OK;
}

}  // extern "C"

namespace wtg {

// One text of at most 8 levels built into d_bv (and d_zeros); its class totals
// (256 u32) are copied to d_counts from the build's job totals, or counted by a
// separate pass when the text is a small job (which has no totals).
wt_status build_with_counts(wt_kind kind, const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma,
                            uint64_t *d_bv, uint64_t *d_zeros, void *d_ws, size_t ws_bytes, uint32_t *d_counts,
                            cudaStream_t s)
{
    HostText h{d_text, n, sigma, d_bv, d_zeros};
    Plan p;
    wt_status st = make_plan(kind, type, &h, 1, true, p);
    if (st != WT_OK) return st;
    if (p.rounds != 1) return WT_ERR_INVALID_ARG;
    st = run_plan(kind, p, d_ws, ws_bytes, s);
    if (st != WT_OK) return st;
    if (n > kSmallJob) {
        const void *tot = static_cast<uint8_t *>(d_ws) + p.off_jobhist[0];
        return cudaMemcpyAsync(d_counts, tot, sizeof(uint32_t) * kCols, cudaMemcpyDeviceToDevice, s) == cudaSuccess
                   ? WT_OK
                   : WT_ERR_CUDA;
    }
    return launch_class_counts(d_text, (uint32_t)type, n, d_counts, s) == cudaSuccess ? WT_OK : WT_ERR_CUDA;
}

}  // namespace wtg

extern "C" {

wt_status wt_sync_status(void *d_ws, void *stream)
{
    if (d_ws == nullptr) return WT_ERR_INVALID_ARG;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return WT_ERR_CUDA;
    uint32_t st = 0;
    Ctl *ctl = static_cast<Ctl *>(d_ws);        // the control block sits at offset 0
    if (cudaMemcpy(&st, &ctl->status, sizeof(st), cudaMemcpyDeviceToHost) != cudaSuccess) return WT_ERR_CUDA;
    if (st != 0 && cudaMemset(&ctl->status, 0, sizeof(uint32_t)) != cudaSuccess) return WT_ERR_CUDA;
    return static_cast<wt_status>(st);
}

wt_status wt_batched_workspace_size(wt_kind kind, wt_symtype type, const wt_text_desc *h_descs, uint32_t count,
                                    size_t *bytes)
{
    if (bytes == nullptr || (count > 0 && h_descs == nullptr)) return WT_ERR_INVALID_ARG;
    std::vector<HostText> h(count);
    for (uint32_t i = 0; i < count; ++i)
        h[i] = HostText{nullptr, h_descs[i].n, h_descs[i].sigma, nullptr, nullptr};
    Plan p;
    wt_status st = make_plan(kind, type, h.data(), count, false, p, kMinSpb);
    if (st == WT_OK) *bytes = p.bytes;
    return st;
}

wt_status wt_build_batched(wt_kind kind, wt_symtype type, const wt_text_desc *h_descs, uint32_t count, void *d_ws,
                           size_t ws_bytes, void *stream)
{
    if (count > 0 && h_descs == nullptr) return WT_ERR_INVALID_ARG;
    std::vector<HostText> h(count);
    for (uint32_t i = 0; i < count; ++i)
        h[i] = HostText{h_descs[i].d_text, h_descs[i].n, h_descs[i].sigma, h_descs[i].d_bv, h_descs[i].d_zeros};
    Plan p;
    wt_status st = make_plan(kind, type, h.data(), count, true, p);
    if (st != WT_OK) return st;
    return run_plan(kind, p, d_ws, ws_bytes, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

// ---------------------------------------------------------------------------
// diagnostics: CUDA events around kernel families

namespace wtg {
namespace {

struct ProfRec {
    cudaEvent_t begin, end;
    int family;
    uint32_t launches;
};

std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof_recs;
std::vector<cudaEvent_t> g_prof_pool;
cudaEvent_t g_prof_open[4] = {};
double g_prof_ms[4] = {};
uint64_t g_prof_launches[4] = {};
const uint32_t kFamilyLaunches[4] = {1, 1, 3, 2};

cudaEvent_t take_event()
{
    if (!g_prof_pool.empty()) {
        cudaEvent_t e = g_prof_pool.back();
        g_prof_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

}  // namespace

bool profile_on() { return g_prof_on; }

void profile_mark(int family, bool begin, cudaStream_t s, uint32_t launches)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEvent_t e = take_event();
    cudaEventRecord(e, s);
    if (begin) {
        g_prof_open[family] = e;
    } else {
        g_prof_recs.push_back(ProfRec{g_prof_open[family], e, family, launches ? launches : kFamilyLaunches[family]});
        g_prof_open[family] = nullptr;
    }
}

}  // namespace wtg

extern "C" {

void wt_profile_enable(int on)
{
    std::lock_guard<std::mutex> lk(wtg::g_prof_mu);
    wtg::g_prof_on = on != 0;
}

wt_status wt_profile_read(wt_profile *out, int reset)
{
    using namespace wtg;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto &r : g_prof_recs) {
        if (cudaEventSynchronize(r.end) != cudaSuccess) return WT_ERR_CUDA;
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, r.begin, r.end) != cudaSuccess) return WT_ERR_CUDA;
        g_prof_ms[r.family] += ms;
        g_prof_launches[r.family] += r.launches;
        g_prof_pool.push_back(r.begin);
        g_prof_pool.push_back(r.end);
    }
    g_prof_recs.clear();
    if (out) {
        for (int k = 0; k < 4; ++k) {
            out->ms[k] = g_prof_ms[k];
            out->launches[k] = g_prof_launches[k];
        }
    }
    if (reset)
        for (int k = 0; k < 4; ++k) {
            g_prof_ms[k] = 0;
            g_prof_launches[k] = 0;
        }
    return WT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Wavelet tree build that allocates nothing (see wt_build_static_ws in the
// header).  Its scratch is a fixed array in device memory, so callers that are
// not allowed to allocate device memory can still build small texts.

namespace wtg {
namespace {

constexpr size_t kStaticScratchBytes = size_t(1) << 20;   // 1 MiB per device

// One copy per device that loads this library; it lives until the process exits.
__device__ __align__(256) uint8_t g_static_scratch[kStaticScratchBytes];

std::mutex g_static_mu;
void *g_static_ptr[64] = {};

// The text's descriptor written into the scratch from a kernel argument, so that
// the call reads no host memory on the stream.
__global__ void k_put_text(TextInfo *dst, TextInfo v)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) *dst = v;
}

// Device address of g_static_scratch on the current device (looked up once per device).
wt_status static_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return WT_ERR_CUDA;
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (g_static_ptr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_static_scratch) != cudaSuccess || p == nullptr) return WT_ERR_CUDA;
        g_static_ptr[dev] = p;
    }
    *out = g_static_ptr[dev];
    return WT_OK;
}

}  // namespace
}  // namespace wtg

extern "C" wt_status wt_build_static_ws(const void *d_text, wt_symtype type, uint64_t n, uint64_t sigma,
                                        uint64_t *d_bv, void *stream)
{
    using namespace wtg;
    HostText h{d_text, n, sigma, d_bv, nullptr};
    Plan p;
    wt_status st = make_plan(WT_TREE, type, &h, 1, true, p);
    if (st != WT_OK) return st;
    if (p.bytes > kStaticScratchBytes) return WT_ERR_OUT_OF_MEMORY;
    void *ws = nullptr;
    st = static_scratch(&ws);
    if (st != WT_OK) return st;
    st = prepare(p, ws, kStaticScratchBytes);
    if (st != WT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    TextInfo *dtexts = reinterpret_cast<TextInfo *>(static_cast<uint8_t *>(ws) + p.off_texts);
    k_put_text<<<1, 32, 0, s>>>(dtexts, p.texts[0]);
    if (cudaGetLastError() != cudaSuccess) return WT_ERR_CUDA;
    return launch(WT_TREE, p, ws, s);
}

// ---------------------------------------------------------------------------
// Batched build recorded once into a CUDA graph and replayed; autotuner for the
// symbols per build block with a JSON cache file.

#include <chrono>
#include <cstdio>
#include <cstdlib>
#include <map>
#include <string>

namespace wtg {
namespace {

struct BatchPlanImpl {
    wt_kind kind = WT_TREE;
    wt_symtype type = WT_U8;
    Plan plan;
    void *ws = nullptr;
    size_t ws_bytes = 0;
    TextInfo *h_desc = nullptr;        // pinned copy of the descriptors (upload source)
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<uint64_t> n, sigma;
    uint32_t spb = 0;
};

const uint32_t kSpbCandidates[] = {32768, 65536, 131072, 262144};

uint32_t ilog2(uint64_t x)
{
    uint32_t r = 0;
    while (x > 1) { x >>= 1; ++r; }
    return r;
}

// Cache key: kind, storage width, and buckets of the batch's shape.
std::string tune_key(wt_kind kind, wt_symtype type, const wt_text_desc *d, uint32_t count)
{
    uint64_t total = 0, maxn = 0;
    uint32_t maxL = 0;
    for (uint32_t i = 0; i < count; ++i) {
        total += d[i].n;
        maxn = d[i].n > maxn ? d[i].n : maxn;
        uint32_t L = levels_of(d[i].sigma);
        maxL = L > maxL ? L : maxL;
    }
    char buf[128];
    snprintf(buf, sizeof(buf), "k%d_w%d_c%u_t%u_m%u_L%u", (int)kind, (int)type, ilog2(count + 1), ilog2(total + 1),
             ilog2(maxn + 1), (maxL + 7) / 8);
    return buf;
}

std::mutex g_tune_mu;

std::map<std::string, uint32_t> read_cache(const char *path)
{
    std::map<std::string, uint32_t> m;
    FILE *f = path ? fopen(path, "r") : nullptr;
    if (!f) return m;
    std::string s;
    char chunk[4096];
    size_t k;
    while ((k = fread(chunk, 1, sizeof(chunk), f)) > 0) s.append(chunk, k);
    fclose(f);
    size_t pos = 0;
    while ((pos = s.find('"', pos)) != std::string::npos) {      // "key": value pairs
        size_t end = s.find('"', pos + 1);
        if (end == std::string::npos) break;
        std::string key = s.substr(pos + 1, end - pos - 1);
        size_t colon = s.find(':', end);
        if (colon == std::string::npos) break;
        m[key] = (uint32_t)strtoul(s.c_str() + colon + 1, nullptr, 10);
        pos = colon + 1;
    }
    return m;
}

void write_cache(const char *path, const std::map<std::string, uint32_t> &m)
{
    if (!path) return;
    std::string tmp = std::string(path) + ".tmp";
    FILE *f = fopen(tmp.c_str(), "w");
    if (!f) return;
    fprintf(f, "{");
    bool first = true;
    for (auto &kv : m) {
        fprintf(f, "%s\n  \"%s\": %u", first ? "" : ",", kv.first.c_str(), kv.second);
        first = false;
    }
    fprintf(f, "\n}\n");
    fclose(f);
    rename(tmp.c_str(), path);
}

uint32_t cached_spb(wt_kind kind, wt_symtype type, const wt_text_desc *d, uint32_t count)
{
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto m = read_cache(getenv("WT_TUNE_CACHE"));
    auto it = m.find(tune_key(kind, type, d, count));
    return it == m.end() || !valid_spb(it->second) ? 0u : it->second;
}

wt_status to_host_texts(const wt_text_desc *d, uint32_t count, std::vector<HostText> &h)
{
    if (count > 0 && d == nullptr) return WT_ERR_INVALID_ARG;
    h.resize(count);
    for (uint32_t i = 0; i < count; ++i) h[i] = HostText{d[i].d_text, d[i].n, d[i].sigma, d[i].d_bv, d[i].d_zeros};
    return WT_OK;
}

}  // namespace
}  // namespace wtg

struct wt_batch_plan {
    wtg::BatchPlanImpl impl;
};

extern "C" {

wt_status wt_batch_plan_create(wt_kind kind, wt_symtype type, const wt_text_desc *h_descs, uint32_t count,
                               uint32_t symbols_per_block, void *d_ws, size_t ws_bytes, void *stream,
                               wt_batch_plan **out)
{
    using namespace wtg;
    if (out == nullptr || stream == nullptr) return WT_ERR_INVALID_ARG;
    *out = nullptr;
    std::vector<HostText> h;
    wt_status st = to_host_texts(h_descs, count, h);
    if (st != WT_OK) return st;
    const uint32_t spb = symbols_per_block ? symbols_per_block : cached_spb(kind, type, h_descs, count);
    wt_batch_plan *bp = new wt_batch_plan();
    BatchPlanImpl &b = bp->impl;
    b.kind = kind;
    b.type = type;
    b.ws = d_ws;
    b.ws_bytes = ws_bytes;
    b.spb = spb;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    st = make_plan(kind, type, h.data(), count, true, b.plan, spb);
    if (st == WT_OK && count > 0) st = prepare(b.plan, d_ws, ws_bytes);
    if (st == WT_OK && count > 0) {
        if (cudaMallocHost(reinterpret_cast<void **>(&b.h_desc), sizeof(TextInfo) * count) != cudaSuccess)
            st = WT_ERR_OUT_OF_MEMORY;
    }
    if (st == WT_OK && count > 0) {
        for (uint32_t i = 0; i < count; ++i) {
            b.h_desc[i] = b.plan.texts[i];
            b.n.push_back(h_descs[i].n);
            b.sigma.push_back(h_descs[i].sigma);
        }
        st = upload(b.plan, b.h_desc, d_ws, s);
    }
    if (st == WT_OK && count > 0) {
        if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            st = WT_ERR_CUDA;
        } else {
            wt_status ls = launch(kind, b.plan, d_ws, s);
            cudaError_t e = cudaStreamEndCapture(s, &b.graph);
            if (ls != WT_OK) st = ls;
            else if (e != cudaSuccess) st = WT_ERR_CUDA;
            else if (cudaGraphInstantiate(&b.exec, b.graph, 0) != cudaSuccess) st = WT_ERR_CUDA;
        }
    }
    if (st != WT_OK) {
        wt_batch_plan_destroy(bp);
        return st;
    }
    *out = bp;
    return WT_OK;
}

wt_status wt_batch_plan_update(wt_batch_plan *bp, const wt_text_desc *h_descs, void *stream)
{
    using namespace wtg;
    if (bp == nullptr || stream == nullptr) return WT_ERR_INVALID_ARG;
    BatchPlanImpl &b = bp->impl;
    const uint32_t count = b.plan.count;
    if (count == 0) return WT_OK;
    if (h_descs == nullptr) return WT_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < count; ++i) {
        if (h_descs[i].n != b.n[i] || h_descs[i].sigma != b.sigma[i]) return WT_ERR_INVALID_ARG;
        const uint32_t L = b.plan.texts[i].L;
        if (L > 0 && h_descs[i].n > 0 && (h_descs[i].d_text == nullptr || h_descs[i].d_bv == nullptr))
            return WT_ERR_INVALID_ARG;
        if (b.kind == WT_MATRIX && L > 0 && h_descs[i].d_zeros == nullptr) return WT_ERR_INVALID_ARG;
    }
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (cudaStreamSynchronize(s) != cudaSuccess) return WT_ERR_CUDA;   // the pinned copy may still be read
    for (uint32_t i = 0; i < count; ++i) {
        b.h_desc[i].text = h_descs[i].d_text;
        b.h_desc[i].bv = h_descs[i].d_bv;
        b.h_desc[i].zeros = b.kind == WT_MATRIX ? h_descs[i].d_zeros : nullptr;
    }
    return upload(b.plan, b.h_desc, b.ws, s);
}

wt_status wt_batch_plan_launch(wt_batch_plan *bp, void *stream)
{
    if (bp == nullptr) return WT_ERR_INVALID_ARG;
    if (bp->impl.exec == nullptr) return WT_OK;                       // empty batch
    if (cudaGraphLaunch(bp->impl.exec, static_cast<cudaStream_t>(stream)) != cudaSuccess) return WT_ERR_CUDA;
    return WT_OK;
}

uint32_t wt_batch_plan_symbols_per_block(const wt_batch_plan *bp) { return bp ? bp->impl.spb : 0; }

void wt_batch_plan_destroy(wt_batch_plan *bp)
{
    if (bp == nullptr) return;
    if (bp->impl.exec) cudaGraphExecDestroy(bp->impl.exec);
    if (bp->impl.graph) cudaGraphDestroy(bp->impl.graph);
    if (bp->impl.h_desc) cudaFreeHost(bp->impl.h_desc);
    delete bp;
}

wt_status wt_autotune_batched(wt_kind kind, wt_symtype type, const wt_text_desc *h_descs, uint32_t count, void *d_ws,
                              size_t ws_bytes, void *stream, uint32_t *best_symbols_per_block)
{
    using namespace wtg;
    if (best_symbols_per_block == nullptr) return WT_ERR_INVALID_ARG;
    std::vector<HostText> h;
    wt_status st = to_host_texts(h_descs, count, h);
    if (st != WT_OK) return st;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return WT_ERR_CUDA;
    float best_ms = 0.f;
    uint32_t best = 0;
    for (uint32_t spb : kSpbCandidates) {
        Plan p;
        st = make_plan(kind, type, h.data(), count, true, p, spb);
        if (st != WT_OK) break;
        st = run_plan(kind, p, d_ws, ws_bytes, s);                      // warm-up
        if (st != WT_OK) break;
        cudaEventRecord(e0, s);
        for (int rep = 0; rep < 3 && st == WT_OK; ++rep) st = run_plan(kind, p, d_ws, ws_bytes, s);
        cudaEventRecord(e1, s);
        if (st != WT_OK || cudaEventSynchronize(e1) != cudaSuccess) { st = st == WT_OK ? WT_ERR_CUDA : st; break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (best == 0 || ms < best_ms) { best_ms = ms; best = spb; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != WT_OK) return st;
    *best_symbols_per_block = best;
    const char *path = getenv("WT_TUNE_CACHE");
    if (path) {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        auto m = read_cache(path);
        m[tune_key(kind, type, h_descs, count)] = best;
        write_cache(path, m);
    }
    return WT_OK;
}

}  // extern "C"
