// C ABI of wt_gb300: argument checks, workspace planning and round launches
// for wt_build / wm_build / wt_build_batched.  See include/wt_gb300.h.
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
};

struct Plan {
    uint32_t count = 0;
    uint32_t rounds = 0;
    uint32_t nslots[kMaxRounds] = {};
    uint32_t groups_ub[kMaxRounds] = {};
    uint32_t blocks_ub[kMaxRounds] = {};
    uint32_t width[kMaxRounds] = {};
    size_t off_ctl = 0, off_texts = 0, off_jobs[2] = {}, off_jobhist[2] = {};
    size_t off_ghist = 0, off_gexcl = 0, off_btail = 0, off_bflag = 0, off_bcarry = 0;
    std::vector<size_t> off_buf[2];
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

// Checks the texts and lays out the workspace.  With check_ptrs == false only
// sizes are validated (workspace queries).
wt_status make_plan(wt_kind kind, wt_symtype type, const HostText *t, uint32_t count, bool check_ptrs,
                    Plan &p)
{
    if (kind != WT_TREE && kind != WT_MATRIX) return WT_ERR_INVALID_ARG;
    if (type != WT_U8 && type != WT_U16 && type != WT_U32) return WT_ERR_INVALID_ARG;
    if (count > 0 && t == nullptr) return WT_ERR_INVALID_ARG;
    const uint32_t w = (uint32_t)type;
    p.count = count;
    p.texts.assign(count, TextInfo{});
    uint32_t max_slots = 0, max_groups = 0;
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
        if (check_ptrs && L > 0) {
            if (x.n > 0 && (x.text == nullptr || x.bv == nullptr)) return WT_ERR_INVALID_ARG;
            if (kind == WT_MATRIX && x.zeros == nullptr) return WT_ERR_INVALID_ARG;
            if (reinterpret_cast<uintptr_t>(x.text) % w) return WT_ERR_INVALID_ARG;
            if (reinterpret_cast<uintptr_t>(x.bv) % 8) return WT_ERR_INVALID_ARG;
        }
        TextInfo &ti = p.texts[i];
        ti.text = x.text;
        ti.bv = x.bv;
        ti.zeros = kind == WT_MATRIX ? x.zeros : nullptr;
        ti.n = x.n;
        ti.W = (x.n + 63) / 64;
        ti.sigma = x.sigma;
        ti.L = L;
        ti.in_w = w;
        const uint32_t rounds = (L + kChunk - 1) / kChunk;
        if (rounds > p.rounds) p.rounds = rounds;
        for (uint32_t r = 0; r < kMaxRounds; ++r) {
            uint32_t ns = 0;
            if (x.n > 0 && L > kChunk * r) ns = (kind == WT_TREE) ? (1u << (8 * r)) : 1u;
            ti.nslots[r] = ns;
            ti.slot_base[r] = (uint32_t)slot_acc[r];
            slot_acc[r] += ns;
            if (ns) {
                uint32_t wr = width_for_bits(L - kChunk * r);
                if (wr > width[r]) width[r] = wr;
            }
        }
    }
    for (uint32_t r = 0; r < p.rounds; ++r) {
        if (slot_acc[r] >= (1ull << 31)) return WT_ERR_INVALID_ARG;
        p.width[r] = width[r] ? width[r] : 1;
        const uint64_t ge = (uint64_t)group_elems(p.width[r]);
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
    p.off_btail = take(sizeof(uint32_t) * kCols * (size_t)max_blocks);
    p.off_bcarry = take(sizeof(uint32_t) * kCols * (size_t)max_blocks);
    p.off_bflag = take(sizeof(uint32_t) * (size_t)max_blocks);
    p.off_buf[0].assign(count, 0);
    p.off_buf[1].assign(count, 0);
    for (uint32_t i = 0; i < count; ++i) {
        const TextInfo &ti = p.texts[i];
        if (ti.n == 0) continue;
        if (ti.L > kChunk) p.off_buf[0][i] = take(ti.n * width_for_bits(ti.L - kChunk));
        if (ti.L > 2 * kChunk) p.off_buf[1][i] = take(ti.n * width_for_bits(ti.L - 2 * kChunk));
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

wt_status run_plan(wt_kind kind, Plan &p, void *d_ws, size_t ws_bytes, cudaStream_t s)
{
    if (p.count == 0) return WT_OK;
    if (d_ws == nullptr || ws_bytes < p.bytes) return WT_ERR_OUT_OF_MEMORY;
    if (reinterpret_cast<uintptr_t>(d_ws) % 256) return WT_ERR_INVALID_ARG;
    wt_status st = ensure_configured();
    if (st != WT_OK) return st;
    uint8_t *ws = static_cast<uint8_t *>(d_ws);
    for (uint32_t i = 0; i < p.count; ++i) {
        TextInfo &ti = p.texts[i];
        ti.buf[0] = ti.L > kChunk ? ws + p.off_buf[0][i] : nullptr;
        ti.buf[1] = ti.L > 2 * kChunk ? ws + p.off_buf[1][i] : nullptr;
    }
    Ctl *ctl = reinterpret_cast<Ctl *>(ws + p.off_ctl);
    TextInfo *dtexts = reinterpret_cast<TextInfo *>(ws + p.off_texts);
    if (cudaMemsetAsync(ctl, 0, sizeof(Ctl), s) != cudaSuccess) return WT_ERR_CUDA;
    if (cudaMemcpyAsync(dtexts, p.texts.data(), sizeof(TextInfo) * p.count, cudaMemcpyHostToDevice, s) !=
        cudaSuccess)
        return WT_ERR_CUDA;
    if (kind == WT_MATRIX && launch_zero_z(dtexts, p.count, s) != cudaSuccess) return WT_ERR_CUDA;
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
        a.btail = reinterpret_cast<uint32_t *>(ws + p.off_btail);
        a.bflag = reinterpret_cast<uint32_t *>(ws + p.off_bflag);
        a.bcarry = reinterpret_cast<uint32_t *>(ws + p.off_bcarry);
        a.ntexts = p.count;
        a.nslots = p.nslots[r];
        a.pnslots = r ? p.nslots[r - 1] : 0;
        a.round = r;
        a.kind = (uint32_t)kind;
        a.gelems = (uint32_t)group_elems(p.width[r]);
        a.groups_ub = p.groups_ub[r];
        a.blocks_ub = p.blocks_ub[r];
        for (uint32_t i = 0; i < p.count; ++i) {
            const TextInfo &ti = p.texts[i];
            if (ti.nslots[r] == 0) continue;
            if (ti.L - kChunk * r > (uint32_t)kChunk) a.any_cut = 1; else a.any_plain = 1;
        }
        if (launch_round(a, p.width[r], s) != cudaSuccess) return WT_ERR_CUDA;
    }
    return WT_OK;
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
    wt_status st = make_plan(kind, type, &h, 1, false, p);
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
    wt_status st = make_plan(kind, type, h.data(), count, false, p);
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
    return run_plan(WT_TREE, p, ws, kStaticScratchBytes, static_cast<cudaStream_t>(stream));
}
