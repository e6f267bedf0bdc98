// gsr_api.cu -- the C ABI of libgsr (declared in include/gsr.h).
//
// Host orchestration only: argument checks, the per-call view table,
// workspace sizing, the launch sequence and the status read-back.  Every
// step of the rasterizer runs in the kernels of gsr_preprocess.cu,
// gsr_sort.cu and gsr_blend.cu.
//
// Forward launch sequence (all on the caller's stream, no host sync inside):
//   memset control block and tile ranges
//   preprocess (project + compact visible records, look-back scan)
//   radix sort of visible records by depth bits (4 passes x 3 launches)
//   duplicate (tile instances in depth order, look-back scan)
//   radix sort of instances by tile id (ceil(log2 tiles)/8 passes)
//   ranges
//   blend forward (persistent over all (view, tile))
// Backward:
//   zero per-record and parameter gradients
//   blend backward (persistent), preprocess backward (one launch per view
//   group, in order)
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <vector>

#include "gsr.h"
#include "gsr_kernels.h"

using namespace gsr;

namespace {

struct DevMem {
    void* p = nullptr;
    size_t bytes = 0;
    ~DevMem() { if (p) cudaFree(p); }
    cudaError_t ensure(size_t need)
    {
        if (need <= bytes) return cudaSuccess;
        if (p) cudaFree(p);
        p = nullptr;
        bytes = 0;
        cudaError_t e = cudaMalloc(&p, need);
        if (e == cudaSuccess) bytes = need;
        return e;
    }
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

// control block: counters[kCntSlots] (u64) | status u32 | tickets ... |
// saturation histogram | look-back words (preprocess, emission, second-round
// emission)
constexpr size_t kCtrlCounters = 0;
constexpr size_t kCtrlStatus = 128;
constexpr size_t kCtrlTicketPre = 132;
constexpr size_t kCtrlTicketDup = 136;
constexpr size_t kCtrlWorkFwd = 140;
constexpr size_t kCtrlWorkBwd = 144;
constexpr size_t kCtrlQueueBwd = 148;
constexpr size_t kCtrlTicketDup2 = 152;   // the second round's emission
constexpr size_t kCtrlWorkFwd2 = 156;     // the second round's blend
constexpr size_t kCtrlGradRows = 160;     // u64: gradient rows written by the backward
constexpr size_t kCtrlRowTotal = 168;     // u64: kept tile rows of the forward's instance emission
constexpr size_t kCtrlRowTotal2 = 176;    // u64: the same for the second round
constexpr size_t kCtrlSatHist = 192;      // u64[kSatBuckets + 1]
constexpr size_t kCtrlInstHist = 768;     // u64[kSatBuckets]
constexpr size_t kCtrlHead = 1280;
static_assert(kCtrlCounters + 8 * kCntSlots <= kCtrlStatus, "counters overlap the status word");
static_assert(kCtrlSatHist + 8 * (kSatBuckets + 1) <= kCtrlInstHist, "histograms overlap");
static_assert(kCtrlInstHist + 8 * kSatBuckets <= kCtrlHead, "histogram overlaps the look-back words");

}  // namespace

namespace gsr {
std::atomic<long long> g_launches{0};
}

// One profiled call: events bracketing consecutive phases [first, first + n).
struct ProfRecord {
    static constexpr int kMax = 16;
    cudaEvent_t ev[kMax + 1] = {};
    int phase[kMax] = {};   // phase of the interval between marks i and i + 1
    int n = 0;
    bool pending = false;
};

struct gsr_ctx {
    gsr_config cfg;
    int device = 0;
    int num_sms = 0;
    std::string err;
    DevMem tmp_keys, tmp_vals, hist, grad_rec, bwd_queue, dup_rows, ins_scratch, freq_scratch, merge_scratch;
    std::map<int, DevMem> fft_twiddles;   // transform length -> W_n^t table
    int hist_blocks = 2048;
    std::map<std::string, gsr_config> tune_cache;
    static constexpr int kProfRing = 64;
    ProfRecord prof[kProfRing];
    int prof_next = 0;
    double phase_ms[GSR_NUM_PHASES] = {};
    int64_t phase_calls[GSR_NUM_PHASES] = {};
    // the backward clears the parameter gradients on this stream while the
    // backward blend runs (fork and join through the two events)
    cudaStream_t side = nullptr;
    cudaEvent_t fork = nullptr, join = nullptr;
    // limit of every device wait of this context's calls, and test-only
    // flags (gsr_debug_set_wait)
    uint64_t wait_ns = kWaitLimitNs;
    uint32_t debug_flags = 0;
    // the first-round fraction of the automatic list mode, chosen from the
    // saturation histogram of the last forward that synchronised
    float auto_prefix = 1.0f;
    ~gsr_ctx()
    {
        for (auto& r : prof)
            for (auto& e : r.ev)
                if (e) cudaEventDestroy(e);
        if (fork) cudaEventDestroy(fork);
        if (join) cudaEventDestroy(join);
        if (side) cudaStreamDestroy(side);
    }
};

static void prof_collect(gsr_ctx* ctx, ProfRecord& r)
{
    if (!r.pending) return;
    cudaEventSynchronize(r.ev[r.n]);
    for (int i = 0; i < r.n; ++i) {
        float ms = 0.0f;
        if (cudaEventElapsedTime(&ms, r.ev[i], r.ev[i + 1]) == cudaSuccess) {
            ctx->phase_ms[r.phase[i]] += ms;
            // a phase taken twice in one call (the two rounds) counts once
            bool again = false;
            for (int j = 0; j < i; ++j) again = again || r.phase[j] == r.phase[i];
            if (!again) ctx->phase_calls[r.phase[i]] += 1;
        }
    }
    r.pending = false;
}

// Start a profiled call covering phases [first, first + n); returns nullptr
// when profiling is off.  Mark phase boundaries with prof_mark(rec, i, s).
static ProfRecord* prof_begin(gsr_ctx* ctx, int first, int n, cudaStream_t s)
{
    if (!(ctx->cfg.flags & GSR_FLAG_PROFILE)) return nullptr;
    ProfRecord& r = ctx->prof[ctx->prof_next];
    ctx->prof_next = (ctx->prof_next + 1) % gsr_ctx::kProfRing;
    prof_collect(ctx, r);
    for (int i = 0; i <= ProfRecord::kMax; ++i)
        if (!r.ev[i] && cudaEventCreate(&r.ev[i]) != cudaSuccess) return nullptr;
    for (int i = 0; i < n; ++i) r.phase[i] = first + i;
    r.n = n;
    r.pending = true;
    cudaEventRecord(r.ev[0], s);
    return &r;
}

static inline void prof_mark(ProfRecord* r, int i, cudaStream_t s)
{
    if (r) cudaEventRecord(r->ev[i], s);
}

// Append intervals of the given phases to a profiled call (marks n + 1 ...).
static inline void prof_extend(ProfRecord* r, std::initializer_list<int> phases)
{
    if (!r) return;
    for (int p : phases)
        if (r->n < ProfRecord::kMax) r->phase[r->n++] = p;
}

struct gsr_saved {
    gsr_ctx* ctx = nullptr;
    Table table;
    int batch = 256;
    uint32_t flags = 0;
    bool filled = false;
    bool have_grads = false;
    int64_t rec_cap = 0, inst_cap = 0, row_cap = 0;   // visible records, kept instances, kept tile rows
    int64_t lb_pre_words = 0, lb_dup_words = 0;
    DevMem rec, vis_key, sorted_k, vis_aux, kstart, tile_key, tile_val, ranges, tfinal, ncontrib, wmask, ctrl;
    DevMem open_tiles, depthpos;         // two-round lists: open-tile bits, record depth positions
    // Two-round lists.  prefix: the first round's record fraction of the
    // last forward (1: one round); region2: where its second list region
    // starts (-1: one region).
    float prefix = 1.0f;
    int64_t region2 = -1;
    unsigned char* host_ctrl = nullptr;  // pinned mirror of the control block head
    ~gsr_saved() { if (host_ctrl) cudaFreeHost(host_ctrl); }
};

static gsr_status fail(gsr_ctx* ctx, gsr_status code, const std::string& msg)
{
    if (ctx) ctx->err = msg;
    return code;
}

static gsr_status cuda_fail(gsr_ctx* ctx, cudaError_t e, const char* where)
{
    return fail(ctx, e == cudaErrorMemoryAllocation ? GSR_ERR_OUT_OF_MEMORY : GSR_ERR_CUDA,
                std::string(where) + ": " + cudaGetErrorString(e));
}

static bool config_ok(const gsr_config* c, std::string& why)
{
    if (!blend_supported(c->tile_w, c->tile_h, c->blend_batch)) {
        why = "tile must be 16x16, 32x8 or 8x32 and blend_batch 128, 256 or 512";
        return false;
    }
    if (c->blend_batch_bwd != 0 && !blend_supported(c->tile_w, c->tile_h, c->blend_batch_bwd)) {
        why = "blend_batch_bwd must be 0, 128, 256 or 512";
        return false;
    }
    if (c->sh_degree < 0 || c->sh_degree > 3) { why = "sh_degree must be 0..3"; return false; }
    if (!(c->list_prefix >= 0.0f) || !std::isfinite(c->list_prefix)) {
        why = "list_prefix must be a finite number >= 0";
        return false;
    }
    if (!(c->near_plane > 0.0f) || !std::isfinite(c->near_plane)) { why = "near_plane must be > 0"; return false; }
    return true;
}

extern "C" {

const char* gsr_version(void) { return "gsr 0.1 (sm_103a)"; }

void gsr_config_default(gsr_config* cfg)
{
    if (!cfg) return;
    cfg->tile_w = 16;
    cfg->tile_h = 16;
    cfg->blend_batch = 256;
    cfg->sh_degree = 3;
    cfg->near_plane = 0.2f;
    cfg->bg[0] = cfg->bg[1] = cfg->bg[2] = 0.0f;
    cfg->flags = 0;
    cfg->blend_batch_bwd = 128;   // measured faster than 256 for the backward on every rig workload
    cfg->list_prefix = 1.0f;      // one round
}

gsr_status gsr_create(gsr_ctx** out, const gsr_config* cfg)
{
    if (!out) return GSR_ERR_INVALID_ARG;
    *out = nullptr;
    gsr_config c;
    if (cfg) c = *cfg; else gsr_config_default(&c);
    std::string why;
    if (!config_ok(&c, why)) return GSR_ERR_INVALID_ARG;
    gsr_ctx* ctx = new (std::nothrow) gsr_ctx();
    if (!ctx) return GSR_ERR_OUT_OF_MEMORY;
    ctx->cfg = c;
    cudaError_t e = cudaGetDevice(&ctx->device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, ctx->device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&ctx->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->fork, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ctx->join, cudaEventDisableTiming);
    if (e != cudaSuccess) { delete ctx; return GSR_ERR_CUDA; }
    *out = ctx;
    return GSR_OK;
}

void gsr_destroy(gsr_ctx* ctx) { delete ctx; }

const char* gsr_last_error(const gsr_ctx* ctx) { return ctx ? ctx->err.c_str() : "null context"; }

gsr_status gsr_set_config(gsr_ctx* ctx, const gsr_config* cfg)
{
    if (!ctx || !cfg) return GSR_ERR_INVALID_ARG;
    std::string why;
    if (!config_ok(cfg, why)) return fail(ctx, GSR_ERR_INVALID_ARG, why);
    ctx->cfg = *cfg;
    return GSR_OK;
}

gsr_status gsr_get_config(const gsr_ctx* ctx, gsr_config* cfg)
{
    if (!ctx || !cfg) return GSR_ERR_INVALID_ARG;
    *cfg = ctx->cfg;
    return GSR_OK;
}

gsr_status gsr_saved_create(gsr_ctx* ctx, gsr_saved** out)
{
    if (!ctx || !out) return GSR_ERR_INVALID_ARG;
    *out = nullptr;
    gsr_saved* s = new (std::nothrow) gsr_saved();
    if (!s) return fail(ctx, GSR_ERR_OUT_OF_MEMORY, "saved state");
    s->ctx = ctx;
    std::memset(&s->table, 0, sizeof(Table));
    cudaError_t e = cudaMallocHost((void**)&s->host_ctrl, kCtrlHead);
    if (e != cudaSuccess) { delete s; return cuda_fail(ctx, e, "cudaMallocHost"); }
    std::memset(s->host_ctrl, 0, kCtrlHead);
    *out = s;
    return GSR_OK;
}

void gsr_saved_destroy(gsr_saved* s) { delete s; }

gsr_status gsr_saved_get_info(const gsr_saved* s, gsr_saved_info* info)
{
    if (!s || !info) return GSR_ERR_INVALID_ARG;
    const unsigned long long* c = reinterpret_cast<const unsigned long long*>(s->host_ctrl + kCtrlCounters);
    info->n_records = s->table.n_records;
    info->n_visible = (int64_t)c[kCntVisible];
    info->n_instances = (int64_t)(c[kCntInstances] + c[kCntInstances2]);
    info->n_tiles = s->table.n_tiles;
    info->n_pixels = s->table.n_pixels;
    info->fwd_pairs = (int64_t)c[kCntFwdPairs];
    info->bwd_pairs = (int64_t)c[kCntBwdPairs];
    info->tile_w = s->table.tile_w;
    info->tile_h = s->table.tile_h;
    info->blend_batch = s->batch;
    info->blended_pairs = (int64_t)c[kCntBlended];
    info->warp_entries_fwd = (int64_t)c[kCntWarpFwd];
    info->warp_entries_bwd = (int64_t)c[kCntWarpBwd];
    info->n_instances_full = (int64_t)c[kCntFullInst];
    info->grad_rows = (int64_t)*reinterpret_cast<const unsigned long long*>(s->host_ctrl + kCtrlGradRows);
    info->list_prefix = s->prefix;
    info->n_instances_second = (int64_t)c[kCntInstances2];
    info->open_tiles = (int64_t)c[kCntOpenTiles];
    info->list_span = s->region2 >= 0 ? s->region2 + (int64_t)c[kCntInstances2] : (int64_t)c[kCntInstances];
    return GSR_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// table + sizing
// ---------------------------------------------------------------------------
// The launch table of a batch under configuration c; on failure *why names
// the reason.  Shared by gsr_forward/gsr_backward (through build_table, which
// records the reason in the context) and by the allocation-free forward.
static gsr_status build_table_cfg(const gsr_config& c, const gsr_gaussians* g, const gsr_view* views, int nv,
                                  Table& T, const char** why)
{
    auto fail_why = [why](gsr_status st, const char* msg) { *why = msg; return st; };
    if (!g || !views) return fail_why(GSR_ERR_INVALID_ARG, "null gaussians or views");
    if (nv < 1) return fail_why(GSR_ERR_INVALID_ARG, "n_views must be >= 1");
    if (nv > kMaxViews) return fail_why(GSR_ERR_NOT_SUPPORTED, "more than GSR_MAX_VIEWS views");
    if (g->n < 0 || g->n > 0xffffffffll) return fail_why(GSR_ERR_INVALID_ARG, "Gaussian count out of range");
    if (g->n > 0 && (!g->means || !g->log_scales || !g->quats || !g->opacity_logits || !g->sh))
        return fail_why(GSR_ERR_INVALID_ARG, "null Gaussian parameter pointer");
    if (((uintptr_t)g->quats & 15u) != 0) return fail_why(GSR_ERR_INVALID_ARG, "quats must be 16-byte aligned");
    std::memset(&T, 0, sizeof(Table));
    T.n_views = nv;
    T.tile_w = c.tile_w;
    T.tile_h = c.tile_h;
    T.inv_tile_w = 1.0f / (float)c.tile_w;   // exact: 8, 16 or 32
    T.inv_tile_h = 1.0f / (float)c.tile_h;
    T.sh_degree = c.sh_degree;
    T.near_plane = c.near_plane;
    for (int i = 0; i < 3; ++i) T.bg[i] = c.bg[i];
    int64_t tile_base = 0, pix_base = 0, vm_base = 0;
    for (int v = 0; v < nv; ++v) {
        const gsr_view& src = views[v];
        if (src.width <= 0 || src.height <= 0) return fail_why(GSR_ERR_INVALID_ARG, "view size must be positive");
        if (!(src.fx > 0.0f) || !(src.fy > 0.0f)) return fail_why(GSR_ERR_INVALID_ARG, "focal lengths must be > 0");
        const int64_t cnt = src.subset ? src.subset_count : g->n;
        if (cnt < 0 || cnt > g->n) return fail_why(GSR_ERR_INVALID_ARG, "subset_count out of range");
        DevView& d = T.v[v];
        for (int i = 0; i < 3; ++i) {
            for (int j = 0; j < 3; ++j) d.R[3 * i + j] = src.viewmat[4 * i + j];
            d.t[i] = src.viewmat[4 * i + 3];
        }
        d.fx = src.fx; d.fy = src.fy; d.cx = src.cx; d.cy = src.cy;
        d.W = src.width; d.H = src.height;
        d.TX = (src.width + c.tile_w - 1) / c.tile_w;
        d.TY = (src.height + c.tile_h - 1) / c.tile_h;
        if (d.TX > 65535 || d.TY > 65535) return fail_why(GSR_ERR_NOT_SUPPORTED, "tile grid wider than 65535");
        d.tile_base = tile_base;
        d.pix_base = pix_base;
        d.vm_base = vm_base;
        tile_base += (int64_t)d.TX * d.TY;
        pix_base += (int64_t)src.width * src.height;
        vm_base += cnt;
        // view groups: runs of consecutive views with the same subset
        const bool same = v > 0 && views[v - 1].subset == src.subset &&
                          (src.subset == nullptr || views[v - 1].subset_count == src.subset_count);
        if (!same) {
            DevGroup& G = T.g[T.n_groups++];
            G.subset = src.subset;
            G.n = cnt;
            G.first_view = v;
            G.nv = 0;
        }
        DevGroup& G = T.g[T.n_groups - 1];
        d.group = T.n_groups - 1;
        d.vl = G.nv++;
    }
    int64_t rec = 0, slot = 0;
    for (int gi = 0; gi < T.n_groups; ++gi) {
        DevGroup& G = T.g[gi];
        G.rec_base = rec;
        G.slot_base = slot;
        rec += G.n * G.nv;
        slot += G.n;
    }
    if (tile_base >= 0xffffffffll) return fail_why(GSR_ERR_NOT_SUPPORTED, "too many tiles");
    if (rec >= 0xffffffffll) return fail_why(GSR_ERR_NOT_SUPPORTED, "too many (view, Gaussian) records");
    T.n_records = rec;
    T.n_slots = slot;
    T.n_tiles = tile_base;
    T.n_pixels = pix_base;
    return GSR_OK;
}

static gsr_status build_table(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_view* views, int nv, Table& T)
{
    const char* why = "";
    const gsr_status st = build_table_cfg(ctx->cfg, g, views, nv, T, &why);
    return st == GSR_OK ? GSR_OK : fail(ctx, st, why);
}

// Two-round lists are possible under this configuration (list_prefix < 1:
// a fixed first-round fraction, or 0 for the automatic choice).
static bool two_rounds_configured(const gsr_config& c) { return c.list_prefix < 1.0f; }

// First position of the second list region: past the first region's
// inst_cap positions, rounded up to 64 so that the region's arrays start on
// 256-byte boundaries (the sort's bulk copies and the vector loads of the
// emission and the ranges need 16).
static int64_t region2_start(int64_t inst_cap) { return (inst_cap + 63) / 64 * 64; }

// The first round's record fraction of the next forward (1: one round).
// Both list regions' positions must fit the 32-bit ranges.
static float forward_prefix(const gsr_ctx* ctx, const gsr_saved* s)
{
    const float f = ctx->cfg.list_prefix;
    if (f >= 1.0f || region2_start(s->inst_cap) + s->inst_cap > (int64_t)0xffffffffll) return 1.0f;
    return f > 0.0f ? f : ctx->auto_prefix;
}

// The automatic first-round fraction, from a forward's two histograms over
// the share x of the depth-ordered records: H, list lengths of the tiles by
// the share they needed before every pixel stopped (last bucket: never), and
// J, kept instances by their record's share.  In units of one instance's
// emission and sort, with R visible records (a record's walk costs about
// kRec instances), one round costs I + kRec R (I = sum J).  A first round
// over the share f = sat_edge(b) costs I1 = (instances of shares < f) +
// kRec f R; the tiles that need more (buckets >= b of H) cost their full
// lists T once more, their first-round blend about kBlend T I1 / I, and, if
// there are any, the second round walks every record again (kWalk R).  Two
// rounds are taken when they cost at most kTake of one.  The constants are
// measured on the 1080p single view, the rig and the road corridor.
static float choose_prefix(const unsigned long long* H, const unsigned long long* J, unsigned long long R)
{
    constexpr double kRec = 4.5, kWalk = 4.0, kBlend = 4.0, kTake = 0.6;
    double I = 0.0;
    for (int b = 0; b < kSatBuckets; ++b) I += (double)J[b];
    if (I <= 0.0) return -1.0f;   // no measurement
    const double one = I + kRec * (double)R;
    double best = one, I1 = (double)J[0], T = 0.0;
    for (int b = 0; b <= kSatBuckets; ++b) T += (double)H[b];
    int best_b = kSatBuckets;
    for (int b = 1; b < kSatBuckets; ++b) {
        T -= (double)H[b - 1];          // tiles that finish within the share sat_edge(b)
        const double f = sat_edge(b);
        const double cost = I1 + kRec * f * (double)R +
                            (T > 0.0 ? T + kBlend * T * I1 / I + kWalk * (double)R : 0.0);
        if (cost < best) { best = cost; best_b = b; }
        I1 += (double)J[b];
    }
    return best_b < kSatBuckets && best <= kTake * one ? (float)sat_edge(best_b) : 1.0f;
}

static gsr_status size_saved(gsr_ctx* ctx, gsr_saved* s, const Table& T)
{
    cudaError_t e;
    if (s->rec_cap == 0) {
        int64_t cap = T.n_records;
        if (cap > (64ll << 20)) cap = std::max<int64_t>(64ll << 20, cap / 3);
        s->rec_cap = std::max<int64_t>(cap, 1);
    }
    if (s->inst_cap == 0) s->inst_cap = std::max<int64_t>(4 * s->rec_cap, 1 << 20);
    // the emission keeps two counts per record in the tile-sort destination
    // keys while they are free
    s->inst_cap = std::max<int64_t>(s->inst_cap, 2 * s->rec_cap);
    // a kept tile row holds >= 1 instance; rows are typically a third of them
    if (s->row_cap == 0) s->row_cap = std::max<int64_t>(std::max<int64_t>(s->inst_cap / 2, 2 * s->rec_cap), 1 << 18);
    const int64_t rc = s->rec_cap, ic = s->inst_cap;
    if ((e = s->rec.ensure((size_t)rc * kRecordBytes)) != cudaSuccess) return cuda_fail(ctx, e, "alloc records");
    if ((e = s->vis_key.ensure((size_t)rc * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc keys");
    if ((e = s->sorted_k.ensure((size_t)rc * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc order");
    if ((e = s->vis_aux.ensure((size_t)rc * 16)) != cudaSuccess) return cuda_fail(ctx, e, "alloc aux");
    if ((e = s->kstart.ensure((size_t)(T.n_slots + 1) * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc kstart");
    // two list regions of inst_cap positions each (the second from
    // region2_start) when two rounds may run
    const bool two = two_rounds_configured(ctx->cfg);
    const int64_t span = two ? region2_start(ic) + ic : ic;
    if ((e = s->tile_key.ensure((size_t)span * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc tile keys");
    if ((e = s->tile_val.ensure((size_t)span * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc tile vals");
    if (two) {
        if ((e = s->open_tiles.ensure((size_t)((std::max<int64_t>(T.n_tiles, 1) + 31) / 32) * 4)) != cudaSuccess)
            return cuda_fail(ctx, e, "alloc open tiles");
        if ((e = s->depthpos.ensure((size_t)rc * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc depth positions");
    }
    if ((e = s->ranges.ensure((size_t)std::max<int64_t>(T.n_tiles, 1) * 8)) != cudaSuccess) return cuda_fail(ctx, e, "alloc ranges");
    if ((e = s->tfinal.ensure((size_t)T.n_pixels * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc tfinal");
    if ((e = s->ncontrib.ensure((size_t)T.n_pixels * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc ncontrib");
    if ((e = s->wmask.ensure((size_t)span)) != cudaSuccess) return cuda_fail(ctx, e, "alloc warp masks");
    s->lb_pre_words = std::max<int64_t>(preprocess_blocks(T), 1);
    s->lb_dup_words = std::max<int64_t>(duplicate_blocks(rc), 1);
    const size_t ctrl = kCtrlHead + 8 * (size_t)(s->lb_pre_words + 2 * s->lb_dup_words);
    if ((e = s->ctrl.ensure(ctrl)) != cudaSuccess) return cuda_fail(ctx, e, "alloc control");
    const int64_t tmp = std::max(rc, ic);
    if ((e = ctx->tmp_keys.ensure((size_t)tmp * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc sort scratch");
    if ((e = ctx->tmp_vals.ensure((size_t)tmp * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc sort scratch");
    if ((e = ctx->hist.ensure((size_t)256 * (ctx->hist_blocks + 1) * 4)) != cudaSuccess) return cuda_fail(ctx, e, "alloc histogram");
    if ((e = ctx->dup_rows.ensure((size_t)s->row_cap * 16)) != cudaSuccess) return cuda_fail(ctx, e, "alloc tile rows");
    return GSR_OK;
}

static int tile_bits(int64_t n_tiles)
{
    if (n_tiles <= 1) return 1;
    int b = 0;
    uint64_t v = (uint64_t)(n_tiles - 1);
    while (v) { ++b; v >>= 1; }
    return b;
}

static void enqueue_forward(gsr_ctx* ctx, gsr_saved* s, const gsr_gaussians* g, const gsr_outputs* out,
                            cudaStream_t st)
{
    const Table& T = s->table;
    unsigned char* ctrl = s->ctrl.as<unsigned char>();
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(ctrl + kCtrlCounters);
    uint32_t* status = reinterpret_cast<uint32_t*>(ctrl + kCtrlStatus);
    unsigned long long* lb_pre = reinterpret_cast<unsigned long long*>(ctrl + kCtrlHead);
    unsigned long long* lb_dup = lb_pre + s->lb_pre_words;
    ProfRecord* pr = prof_begin(ctx, GSR_PHASE_PREPROCESS, 6, st);
    cudaMemsetAsync(ctrl, 0, kCtrlHead + 8 * (size_t)(s->lb_pre_words + 2 * s->lb_dup_words), st);
    cudaMemsetAsync(s->ranges.p, 0, (size_t)std::max<int64_t>(T.n_tiles, 1) * 8, st);

    PreprocessArgs pa;
    pa.means = g->means; pa.log_scales = g->log_scales; pa.quats = g->quats;
    pa.opacity = g->opacity_logits; pa.sh = g->sh;
    pa.rec = s->rec.as<float4>();
    pa.vis_key = s->vis_key.as<uint32_t>();
    pa.vis_aux = s->vis_aux.as<uint4>();
    pa.kstart = s->kstart.as<uint32_t>();
    pa.lb_status = lb_pre;
    pa.ticket = reinterpret_cast<unsigned int*>(ctrl + kCtrlTicketPre);
    pa.rec_cap = s->rec_cap;
    pa.status = status;
    pa.counters = counters;
    pa.wait_ns = ctx->wait_ns;
    pa.debug_flags = (ctx->debug_flags & GSR_DEBUG_WITHHOLD_PREFIX) ? kDebugWithholdFirstPrefix : 0u;
    launch_preprocess_fwd(T, pa, ctx->num_sms, st);
    prof_mark(pr, 1, st);

    RadixScratch rs{ctx->hist.as<uint32_t>(), ctx->hist.as<uint32_t>() + 256 * (size_t)ctx->hist_blocks,
                    ctx->hist_blocks, ctx->num_sms, status};
    rs.wait_ns = ctx->wait_ns;
    radix_sort_pairs(s->vis_key.as<uint32_t>(), s->sorted_k.as<uint32_t>(), ctx->tmp_keys.as<uint32_t>(),
                     ctx->tmp_vals.as<uint32_t>(), true, counters + kCntVisible, s->rec_cap, 32, rs, st);

    // Lists: one round, or two (a first round over a depth prefix of the
    // records, then the tiles it left open over all of them, listed in a
    // second region of the list arrays from region2_start(inst_cap) on).
    const float prefix = forward_prefix(ctx, s);
    const bool two = prefix < 1.0f;
    s->prefix = prefix;
    s->region2 = two ? region2_start(s->inst_cap) : -1;
    if (two) cudaMemsetAsync(s->open_tiles.p, 0, (size_t)((std::max<int64_t>(T.n_tiles, 1) + 31) / 32) * 4, st);
    // the automatic fraction's statistics (depth positions, the two
    // histograms): taken by forwards that synchronise, the only ones whose
    // statistics are read back
    const bool hist = ctx->cfg.list_prefix == 0.0f && !(ctx->cfg.flags & GSR_FLAG_NO_SYNC);
    const int bits = tile_bits(T.n_tiles);
    const int passes = (bits + 7) / 8;
    BlendFwdArgs ba;
    ba.rec = s->rec.as<float4>();
    ba.vals = s->tile_val.as<uint32_t>();
    ba.ranges = s->ranges.as<uint2>();
    ba.rgb = out->rgb;
    ba.depth = out->depth;
    ba.alpha = out->alpha;
    ba.tfinal = s->tfinal.as<float>();
    ba.ncontrib = s->ncontrib.as<uint32_t>();
    ba.wmask = s->wmask.as<uint8_t>();
    ba.status = status;
    ba.counters = counters;
    ba.wait_ns = ctx->wait_ns;
    ba.count_pairs = !(ctx->cfg.flags & GSR_FLAG_NO_PAIR_COUNTS);
    ba.prefix = prefix;
    ba.open_tiles = two ? s->open_tiles.as<uint32_t>() : nullptr;
    ba.depthpos = hist ? s->depthpos.as<uint32_t>() : nullptr;
    ba.hist = hist ? reinterpret_cast<unsigned long long*>(ctrl + kCtrlSatHist) : nullptr;
    // each list round (r = 0 alone, or r = 1 then r = 2): emission into the
    // region at `base`, tile sort, ranges, blend
    for (int r = two ? 1 : 0; r <= (two ? 2 : 0); ++r) {
        const bool second = r == 2;
        const int64_t base = second ? s->region2 : 0;
        uint32_t* rk = s->tile_key.as<uint32_t>() + base;
        uint32_t* rv = s->tile_val.as<uint32_t>() + base;
        uint32_t *xk, *xv, *yk, *yv;
        if (passes & 1) { xk = ctx->tmp_keys.as<uint32_t>(); xv = ctx->tmp_vals.as<uint32_t>(); yk = rk; yv = rv; }
        else { xk = rk; xv = rv; yk = ctx->tmp_keys.as<uint32_t>(); yv = ctx->tmp_vals.as<uint32_t>(); }
        unsigned long long* inst_count = counters + (second ? kCntInstances2 : kCntInstances);
        DuplicateArgs da;
        da.sorted_k = s->sorted_k.as<uint32_t>();
        da.vis_aux = s->vis_aux.as<uint4>();
        da.rec = s->rec.as<float4>();
        da.tile_key = xk;
        da.tile_val = xv;
        da.counts = reinterpret_cast<uint2*>(yk);       // inst_cap >= 2 rec_cap words
        da.rows = ctx->dup_rows.as<uint4>();
        da.win_first = yv;                              // inst_cap >= win_cap words
        da.rec_cap = s->rec_cap;
        da.inst_cap = s->inst_cap;
        da.row_cap = s->row_cap;
        da.win_cap = duplicate_windows(s->inst_cap);
        da.lb_inst = lb_dup + (second ? s->lb_dup_words : 0);
        da.row_total = reinterpret_cast<unsigned long long*>(ctrl + (second ? kCtrlRowTotal2 : kCtrlRowTotal));
        da.ticket = reinterpret_cast<unsigned int*>(ctrl + (second ? kCtrlTicketDup2 : kCtrlTicketDup));
        da.status = status;
        da.counters = counters;
        da.inst_count = inst_count;
        // the rectangles of every record are counted by the first emission
        da.full_count = second ? nullptr : counters + kCntFullInst;
        da.wait_ns = ctx->wait_ns;
        da.prefix = r == 1 ? prefix : 1.0f;
        da.open_tiles = second ? s->open_tiles.as<uint32_t>() : nullptr;
        da.depthpos = hist ? s->depthpos.as<uint32_t>() : nullptr;
        da.inst_hist = hist && r == 0 ? reinterpret_cast<unsigned long long*>(ctrl + kCtrlInstHist) : nullptr;
        if (second) prof_extend(pr, {GSR_PHASE_DUPLICATE, GSR_PHASE_TILE_SORT, GSR_PHASE_RANGES, GSR_PHASE_BLEND_FWD});
        const int m0 = second ? 6 : 2;   // first profiling mark of these phases
        prof_mark(pr, m0, st);
        launch_duplicate(T, da, ctx->num_sms, st);
        prof_mark(pr, m0 + 1, st);
        radix_sort_pairs(xk, xv, yk, yv, false, inst_count, s->inst_cap, bits, rs, st);
        prof_mark(pr, m0 + 2, st);
        launch_ranges(rk, inst_count, s->inst_cap, s->ranges.as<uint2>(), T.n_tiles, base, status, ctx->num_sms, st);
        ba.round = r;
        ba.work = reinterpret_cast<unsigned int*>(ctrl + (second ? kCtrlWorkFwd2 : kCtrlWorkFwd));
        prof_mark(pr, m0 + 3, st);
        launch_blend_fwd(T, s->batch, ba, ctx->num_sms, st);
        prof_mark(pr, m0 + 4, st);
    }
}

// The join of a side stream forked from `cs`: record() marks the end of the
// side stream's work, wait() makes `cs` wait for it.  If the scope is left
// before wait() (an early error return), the destructor does both.
struct SideJoin {
    cudaStream_t cs, side;
    cudaEvent_t join;
    bool recorded = false, joined = false;
    cudaError_t record()
    {
        const cudaError_t e = cudaEventRecord(join, side);
        recorded = e == cudaSuccess;
        return e;
    }
    cudaError_t wait()
    {
        const cudaError_t e = cudaStreamWaitEvent(cs, join, 0);
        joined = e == cudaSuccess;
        return e;
    }
    ~SideJoin()
    {
        if (joined) return;
        if (!recorded) record();
        wait();
    }
};

// Kept tile rows and instances the last forward's larger list round needed
// (valid after a status read-back).
static unsigned long long row_total(const gsr_saved* s)
{
    const unsigned long long r1 = *reinterpret_cast<const unsigned long long*>(s->host_ctrl + kCtrlRowTotal);
    const unsigned long long r2 = *reinterpret_cast<const unsigned long long*>(s->host_ctrl + kCtrlRowTotal2);
    return std::max(r1, r2);
}

static unsigned long long inst_total(const gsr_saved* s)
{
    const unsigned long long* c = reinterpret_cast<const unsigned long long*>(s->host_ctrl + kCtrlCounters);
    return std::max(c[kCntInstances], c[kCntInstances2]);
}

// Capacities for the exact kept-instance and row counts of an emission that
// overflowed them.
static void grow_emission(gsr_saved* s, unsigned long long inst, unsigned long long rows, uint32_t status)
{
    if (status & kErrInstCapacity) s->inst_cap = std::max<int64_t>(s->inst_cap, (int64_t)(inst + inst / 8 + 4096));
    if (status & kErrFullCapacity) s->row_cap = std::max<int64_t>(s->row_cap, (int64_t)(rows + rows / 8 + 4096));
}

// After a read-back of a complete forward: the automatic mode's next
// first-round fraction from its saturation histogram.
static void update_auto_prefix(gsr_ctx* ctx, const gsr_saved* s)
{
    if (!s->filled || ctx->cfg.list_prefix != 0.0f) return;
    const unsigned long long* c = reinterpret_cast<const unsigned long long*>(s->host_ctrl + kCtrlCounters);
    // J is measured by one-round forwards only: after two rounds the choice
    // stays as it was
    const float f = choose_prefix(reinterpret_cast<const unsigned long long*>(s->host_ctrl + kCtrlSatHist),
                                  reinterpret_cast<const unsigned long long*>(s->host_ctrl + kCtrlInstHist),
                                  c[kCntVisible]);
    if (f > 0.0f) ctx->auto_prefix = f;
}

static gsr_status read_status(gsr_ctx* ctx, gsr_saved* s, cudaStream_t st, uint32_t* status_out)
{
    cudaError_t e = cudaMemcpyAsync(s->host_ctrl, s->ctrl.p, kCtrlHead, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "status read-back");
    *status_out = *reinterpret_cast<const uint32_t*>(s->host_ctrl + kCtrlStatus);
    return GSR_OK;
}

extern "C" {

gsr_status gsr_reserve(gsr_ctx* ctx, gsr_saved* s, int64_t visible, int64_t instances)
{
    if (!ctx || !s || s->ctx != ctx || visible < 0 || instances < 0) return fail(ctx, GSR_ERR_INVALID_ARG, "reserve");
    s->rec_cap = std::max(s->rec_cap, visible);
    s->inst_cap = std::max(s->inst_cap, instances);
    s->row_cap = std::max(s->row_cap, instances);   // a kept tile row holds >= 1 instance
    return GSR_OK;
}

gsr_status gsr_forward(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_view* views, int n_views,
                       const gsr_outputs* out, gsr_saved* s, void* stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (!s || s->ctx != ctx) return fail(ctx, GSR_ERR_INVALID_ARG, "saved state missing or from another context");
    if (!out || !out->rgb || !out->depth || !out->alpha) return fail(ctx, GSR_ERR_INVALID_ARG, "null output");
    Table T;
    gsr_status st = build_table(ctx, g, views, n_views, T);
    if (st != GSR_OK) return st;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    s->table = T;
    s->batch = ctx->cfg.blend_batch;
    s->flags = ctx->cfg.flags;
    s->filled = false;
    s->have_grads = false;
    for (int attempt = 0; attempt < 4; ++attempt) {
        if ((st = size_saved(ctx, s, T)) != GSR_OK) return st;
        enqueue_forward(ctx, s, g, out, cs);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(ctx, e, "forward launch");
        s->filled = true;
        if (ctx->cfg.flags & GSR_FLAG_NO_SYNC) return GSR_OK;
        uint32_t status = 0;
        if ((st = read_status(ctx, s, cs, &status)) != GSR_OK) return st;
        if (status & kErrTimeout) { s->filled = false; return fail(ctx, GSR_ERR_TIMEOUT, "device wait timed out"); }
        if (status & kErrOverflow32) { s->filled = false; return fail(ctx, GSR_ERR_NOT_SUPPORTED, "more than 2^32 instances"); }
        if (status & kErrInternal) { s->filled = false; return fail(ctx, GSR_ERR_CUDA, "internal consistency check failed"); }
        if (!(status & (kErrRecCapacity | kErrInstCapacity | kErrFullCapacity))) {
            update_auto_prefix(ctx, s);
            return GSR_OK;
        }
        const unsigned long long* c = reinterpret_cast<const unsigned long long*>(s->host_ctrl + kCtrlCounters);
        if (status & kErrRecCapacity) {
            // later counts are of a truncated record set: grow the others in proportion
            const int64_t old = std::max<int64_t>(s->rec_cap, 1);
            s->rec_cap = (int64_t)(c[kCntVisible] + c[kCntVisible] / 8 + 1024);
            s->inst_cap = std::max<int64_t>(s->inst_cap, s->inst_cap / old * s->rec_cap);
            s->row_cap = std::max<int64_t>(s->row_cap, s->row_cap / old * s->rec_cap);
        } else {
            // the emission counts kept instances and rows exactly
            grow_emission(s, inst_total(s), row_total(s), status);
        }
    }
    s->filled = false;
    return fail(ctx, GSR_ERR_CAPACITY, "capacity did not converge");
}

float gsr_list_prefix_choice(const uint64_t* sat_hist, const uint64_t* inst_hist, uint64_t visible)
{
    static_assert(GSR_LIST_BUCKETS == kSatBuckets, "the header's bucket count is the kernels'");
    if (!sat_hist || !inst_hist) return -1.0f;
    return choose_prefix(reinterpret_cast<const unsigned long long*>(sat_hist),
                         reinterpret_cast<const unsigned long long*>(inst_hist), (unsigned long long)visible);
}

double gsr_list_bucket_edge(int b) { return sat_edge(b); }

gsr_status gsr_check(gsr_ctx* ctx, gsr_saved* s, void* stream)
{
    if (!ctx || !s) return GSR_ERR_INVALID_ARG;
    uint32_t status = 0;
    gsr_status st = read_status(ctx, s, static_cast<cudaStream_t>(stream), &status);
    if (st != GSR_OK) return st;
    if (status & kErrTimeout) return fail(ctx, GSR_ERR_TIMEOUT, "device wait timed out");
    if (status & kErrOverflow32) return fail(ctx, GSR_ERR_NOT_SUPPORTED, "more than 2^32 instances");
    if (status & kErrInternal) return fail(ctx, GSR_ERR_CUDA, "internal consistency check failed");
    if (status & (kErrRecCapacity | kErrInstCapacity | kErrFullCapacity)) {
        const unsigned long long* c = reinterpret_cast<const unsigned long long*>(s->host_ctrl + kCtrlCounters);
        if (status & kErrRecCapacity) s->rec_cap = std::max<int64_t>(s->rec_cap, (int64_t)(c[kCntVisible] * 9 / 8 + 1024));
        grow_emission(s, inst_total(s), row_total(s), status);
        return fail(ctx, GSR_ERR_CAPACITY, "internal capacity exceeded; capacities grown, call again");
    }
    update_auto_prefix(ctx, s);
    return GSR_OK;
}

}  // extern "C"

namespace gsr {
__global__ void zero_grad_rec_kernel(float4* g, const unsigned long long* n_dev, int64_t cap)
{
    const unsigned long long nv = *n_dev;
    const int64_t n = 3 * (int64_t)(nv < (unsigned long long)cap ? nv : (unsigned long long)cap);
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        g[i] = make_float4(0.f, 0.f, 0.f, 0.f);
}
}  // namespace gsr

extern "C" {

gsr_status gsr_backward(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_view* views, int n_views,
                        gsr_saved* s, const float* dl_drgb, const float* dl_ddepth, const float* dl_dalpha,
                        const gsr_grads* grads, void* stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (!s || s->ctx != ctx || !s->filled) return fail(ctx, GSR_ERR_INVALID_ARG, "backward needs a filled saved state");
    if (!dl_drgb || !grads) return fail(ctx, GSR_ERR_INVALID_ARG, "null upstream gradient or grads");
    if (!g || n_views != s->table.n_views) return fail(ctx, GSR_ERR_INVALID_ARG, "views differ from the forward");
    (void)views;
    if (g->n > 0 && (!grads->means || !grads->log_scales || !grads->quats || !grads->opacity_logits || !grads->sh))
        return fail(ctx, GSR_ERR_INVALID_ARG, "null gradient pointer");
    if (((uintptr_t)grads->quats & 15u) != 0) return fail(ctx, GSR_ERR_INVALID_ARG, "grad quats must be 16-byte aligned");
    const Table& T = s->table;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaError_t e = ctx->grad_rec.ensure((size_t)s->rec_cap * kGradFloats * 4);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "alloc record gradients");
    if ((e = ctx->bwd_queue.ensure((size_t)s->rec_cap * 4)) != cudaSuccess)
        return cuda_fail(ctx, e, "alloc extended-precision queue");
    unsigned char* ctrl = s->ctrl.as<unsigned char>();
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(ctrl + kCtrlCounters);
    uint32_t* status = reinterpret_cast<uint32_t*>(ctrl + kCtrlStatus);

    const int K = (T.sh_degree + 1) * (T.sh_degree + 1);
    const size_t n = (size_t)g->n;
    // The parameter gradients are first written by the preprocess backward, so
    // they are cleared on the side stream, after everything already queued on
    // the caller's stream, while the backward blend runs; the caller's stream
    // waits for the clear before the preprocess backward.  (Both events are
    // recorded in stream order, so this also holds under graph capture.)
    if ((e = cudaEventRecord(ctx->fork, cs)) != cudaSuccess) return cuda_fail(ctx, e, "backward fork");
    if ((e = cudaStreamWaitEvent(ctx->side, ctx->fork, 0)) != cudaSuccess) return cuda_fail(ctx, e, "backward fork");
    // from here on every exit joins the side stream back into the caller's
    // (an unjoined fork would also invalidate a graph capture of the call)
    SideJoin joiner{cs, ctx->side, ctx->join};
    {
        cudaError_t ce = cudaSuccess;
        auto clear = [&](void* p, size_t bytes) {
            if (p && ce == cudaSuccess) ce = cudaMemsetAsync(p, 0, bytes, ctx->side);
        };
        clear(grads->means, n * 12);
        clear(grads->log_scales, n * 12);
        clear(grads->quats, n * 16);
        clear(grads->opacity_logits, n * 4);
        clear(grads->sh, n * K * 12);
        clear(grads->pose, (size_t)T.n_views * 24);
        clear(grads->focal, (size_t)T.n_views * 8);
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "backward gradient clear");
    }
    if ((e = joiner.record()) != cudaSuccess) return cuda_fail(ctx, e, "backward join");
    ProfRecord* pr = prof_begin(ctx, GSR_PHASE_BWD_CLEAR, 3, cs);
    cudaMemsetAsync(ctrl + kCtrlWorkBwd, 0, 8, cs);   // blend tile counter and extended-precision queue count
    cudaMemsetAsync(counters + kCntBwdPairs, 0, 8, cs);
    cudaMemsetAsync(counters + kCntWarpBwd, 0, 8, cs);
    cudaMemsetAsync(ctrl + kCtrlGradRows, 0, 8, cs);
    GSR_COUNT_LAUNCH();
    zero_grad_rec_kernel<<<(unsigned)std::max(1, ctx->num_sms * 8), 256, 0, cs>>>(ctx->grad_rec.as<float4>(),
                                                                                  counters + kCntVisible, s->rec_cap);

    BlendBwdArgs bb;
    bb.rec = s->rec.as<float4>();
    bb.vals = s->tile_val.as<uint32_t>();
    bb.ranges = s->ranges.as<uint2>();
    bb.tfinal = s->tfinal.as<float>();
    bb.ncontrib = s->ncontrib.as<uint32_t>();
    bb.wmask = s->wmask.as<uint8_t>();
    bb.dl_rgb = dl_drgb;
    bb.dl_depth = dl_ddepth;
    bb.dl_alpha = dl_dalpha;
    bb.grad_rec = ctx->grad_rec.as<float4>();
    bb.work = reinterpret_cast<unsigned int*>(ctrl + kCtrlWorkBwd);
    bb.status = status;
    bb.counters = counters;
    bb.wait_ns = ctx->wait_ns;
    prof_mark(pr, 1, cs);
    // the backward's staging batch is free (it reads wmask by list position)
    launch_blend_bwd(T, ctx->cfg.blend_batch_bwd ? ctx->cfg.blend_batch_bwd : s->batch, bb, ctx->num_sms, cs);
    prof_mark(pr, 2, cs);

    PreprocessBwdArgs pb;
    pb.means = g->means; pb.log_scales = g->log_scales; pb.quats = g->quats;
    pb.opacity = g->opacity_logits; pb.sh = g->sh;
    pb.vis_aux = s->vis_aux.as<uint4>();
    pb.kstart = s->kstart.as<uint32_t>();
    pb.grad_rec = ctx->grad_rec.as<float4>();
    pb.grad_means = grads->means; pb.grad_log_scales = grads->log_scales; pb.grad_quats = grads->quats;
    pb.grad_opacity = grads->opacity_logits; pb.grad_sh = grads->sh; pb.grad_pose = grads->pose;
    pb.grad_focal = grads->focal;
    pb.queue = ctx->bwd_queue.as<uint32_t>();
    pb.queue_count = reinterpret_cast<unsigned int*>(ctrl + kCtrlQueueBwd);
    pb.queue_cap = s->rec_cap;
    pb.status = status;
    pb.grad_rows = reinterpret_cast<unsigned long long*>(ctrl + kCtrlGradRows);
    if ((e = joiner.wait()) != cudaSuccess) return cuda_fail(ctx, e, "backward join");
    for (int gi = 0; gi < T.n_groups; ++gi) launch_preprocess_bwd(T, gi, pb, ctx->num_sms, cs);
    launch_preprocess_bwd64(T, pb, ctx->num_sms, cs);
    prof_mark(pr, 3, cs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "backward launch");
    s->have_grads = true;
    if (ctx->cfg.flags & GSR_FLAG_NO_SYNC) return GSR_OK;
    uint32_t st = 0;
    gsr_status r = read_status(ctx, s, cs, &st);
    if (r != GSR_OK) return r;
    if (st & kErrTimeout) return fail(ctx, GSR_ERR_TIMEOUT, "device wait timed out");
    if (st & kErrInternal) return fail(ctx, GSR_ERR_CUDA, "internal consistency check failed");
    return GSR_OK;
}

gsr_status gsr_get_stats(gsr_ctx* ctx, gsr_stats* out)
{
    if (!ctx || !out) return GSR_ERR_INVALID_ARG;
    for (auto& r : ctx->prof) prof_collect(ctx, r);
    out->launches = g_launches.load();
    for (int i = 0; i < GSR_NUM_PHASES; ++i) {
        out->phase_ms[i] = ctx->phase_ms[i];
        out->calls[i] = ctx->phase_calls[i];
        ctx->phase_ms[i] = 0.0;
        ctx->phase_calls[i] = 0;
    }
    return GSR_OK;
}

gsr_status gsr_l1_loss_grad(const float* rgb, const float* target, int64_t n, float* dl, float* loss, void* stream)
{
    if (n < 0 || (n > 0 && (!rgb || !target || !dl))) return GSR_ERR_INVALID_ARG;
    launch_l1_loss_grad(rgb, target, n, dl, loss, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

void gsr_insert_params_default(gsr_insert_params* p)
{
    if (!p) return;
    p->sigma = 1.0f;
    p->tau_a = 0.2f;
}

gsr_status gsr_insertion(gsr_ctx* ctx, const gsr_insert_params* p, const gsr_view* views, int n_views,
                         const float* gt, const float* rendered, const float* depth, float* p_a, float* scale,
                         uint32_t* index, int64_t index_cap, unsigned long long* count, void* stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (!p || !views || n_views < 1) return fail(ctx, GSR_ERR_INVALID_ARG, "insertion: params and views required");
    if (n_views > kMaxViews) return fail(ctx, GSR_ERR_NOT_SUPPORTED, "insertion: too many views");
    if (!(p->sigma > 0.0f) || p->sigma > 7.0f / 3.0f) return fail(ctx, GSR_ERR_NOT_SUPPORTED, "insertion: sigma out of (0, 7/3]");
    if (index_cap < 0 || (count && index_cap > 0 && !index)) return fail(ctx, GSR_ERR_INVALID_ARG, "insertion: index buffer");
    InsertTable T;
    std::memset(&T, 0, sizeof(T));
    T.n_views = n_views;
    T.tau = p->tau_a;
    int64_t tiles = 0, pix = 0;
    for (int v = 0; v < n_views; ++v) {
        const gsr_view& src = views[v];
        if (src.width <= 0 || src.height <= 0 || !(src.fx > 0.0f)) return fail(ctx, GSR_ERR_INVALID_ARG, "insertion: view size");
        T.W[v] = src.width; T.H[v] = src.height; T.f[v] = src.fx;
        T.TX[v] = (src.width + 31) / 32;
        T.tile_base[v] = tiles;
        T.pix_base[v] = pix;
        tiles += (int64_t)T.TX[v] * ((src.height + 31) / 32);   // 32 x 32 pixel tiles
        pix += (int64_t)src.width * src.height;
    }
    T.tile_base[n_views] = tiles;
    T.pix_base[n_views] = pix;
    if (pix > 0xffffffffll) return fail(ctx, GSR_ERR_NOT_SUPPORTED, "insertion: more than 2^32 pixels");
    if (pix > 0 && (!gt || !rendered || !depth || !p_a || !scale)) return fail(ctx, GSR_ERR_INVALID_ARG, "insertion: null array");
    insertion_taps((double)p->sigma, &T.r, T.taps);
    // scratch: status word, ticket, look-back words (all start at zero)
    const int64_t words = insertion_lb_words(pix);
    cudaError_t e = ctx->ins_scratch.ensure(16 + 8 * (size_t)words);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "alloc insertion scratch");
    unsigned char* sc = ctx->ins_scratch.as<unsigned char>();
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(sc, 0, 16 + 8 * (size_t)words, cs);
    if (count) cudaMemsetAsync(count, 0, sizeof(unsigned long long), cs);
    uint32_t* status = reinterpret_cast<uint32_t*>(sc);
    launch_insertion(T, gt, rendered, depth, p_a, scale, index, index_cap, count,
                     reinterpret_cast<unsigned long long*>(sc + 16), reinterpret_cast<unsigned int*>(sc + 4), status,
                     ctx->wait_ns, ctx->num_sms, cs);
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "insertion launch");
    if (ctx->cfg.flags & GSR_FLAG_NO_SYNC) return GSR_OK;
    uint32_t st = 0;
    if ((e = cudaMemcpyAsync(&st, status, 4, cudaMemcpyDeviceToHost, cs)) != cudaSuccess ||
        (e = cudaStreamSynchronize(cs)) != cudaSuccess)
        return cuda_fail(ctx, e, "insertion status");
    if (st & kErrTimeout) return fail(ctx, GSR_ERR_TIMEOUT, "device wait timed out");
    return GSR_OK;
}

gsr_status gsr_rig_chain(gsr_ctx* ctx, int n_views, const float* pose_grads, const float* focal_grads,
                         const int32_t* keyframe_of_view, const int32_t* camera_of_view, const float* rel,
                         int n_keyframes, int n_cameras, float* central, float* camera_rel, float* camera_focal,
                         void* stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (n_views < 1 || n_keyframes < 1 || n_cameras < 0) return fail(ctx, GSR_ERR_INVALID_ARG, "rig chain: sizes");
    if (n_views > kMaxViews || n_keyframes > kMaxViews || n_cameras > kMaxViews)
        return fail(ctx, GSR_ERR_NOT_SUPPORTED, "rig chain: more than GSR_MAX_VIEWS");
    if (!pose_grads || !keyframe_of_view || !rel) return fail(ctx, GSR_ERR_INVALID_ARG, "rig chain: null input");
    const bool per_camera = camera_rel || camera_focal;
    if (per_camera && (!camera_of_view || n_cameras < 1))
        return fail(ctx, GSR_ERR_INVALID_ARG, "rig chain: camera outputs need camera_of_view");
    if (camera_focal && !focal_grads) return fail(ctx, GSR_ERR_INVALID_ARG, "rig chain: camera_focal needs focal_grads");
    RigTable T;
    std::memset(&T, 0, sizeof(T));
    T.n_views = n_views; T.n_keyframes = n_keyframes; T.n_cameras = per_camera ? n_cameras : 0;
    for (int i = 0; i < n_views; ++i) {
        if (keyframe_of_view[i] < 0 || keyframe_of_view[i] >= n_keyframes)
            return fail(ctx, GSR_ERR_INVALID_ARG, "rig chain: keyframe index out of range");
        T.kf[i] = keyframe_of_view[i];
        T.cam[i] = -1;
        if (per_camera) {
            if (camera_of_view[i] < 0 || camera_of_view[i] >= n_cameras)
                return fail(ctx, GSR_ERR_INVALID_ARG, "rig chain: camera index out of range");
            T.cam[i] = camera_of_view[i];
        }
        std::memcpy(T.rel[i], rel + 12 * (size_t)i, 12 * sizeof(float));
    }
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    launch_rig_chain(T, pose_grads, focal_grads, central, camera_rel, camera_focal, cs);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "rig chain launch");
    return GSR_OK;
}

void gsr_merge_params_default(gsr_merge_params* p)
{
    if (!p) return;
    p->tau_d = 0.5f;
    p->near_plane = 0.2f;
}

gsr_status gsr_merge(gsr_ctx* ctx, const gsr_merge_params* p, const gsr_view* view, int64_t n_existing,
                     const float* means, const float* log_scales, const float* sh, int64_t sh_stride,
                     int64_t n_samples, const uint32_t* sample_pixels, const float* scale_map,
                     const float* depth_map, const float* gt, const gsr_merge_outputs* out, void* stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (!p || !view || !out) return fail(ctx, GSR_ERR_INVALID_ARG, "merge: params, view and outputs required");
    if (n_existing < 0 || n_samples < 0 || n_existing >= ((int64_t)1 << 31))
        return fail(ctx, GSR_ERR_INVALID_ARG, "merge: sizes");
    if (view->width <= 0 || view->height <= 0 || !(view->fx > 0.0f) || !(view->fy > 0.0f))
        return fail(ctx, GSR_ERR_INVALID_ARG, "merge: view");
    const int64_t npix = (int64_t)view->width * view->height;
    if (npix > 0x7fffffffll) return fail(ctx, GSR_ERR_NOT_SUPPORTED, "merge: view larger than 2^31 pixels");
    if (n_samples > npix) return fail(ctx, GSR_ERR_INVALID_ARG, "merge: more samples than pixels");
    if (n_samples > 0 && (!sample_pixels || !scale_map || !depth_map || !gt || !out->sample_action))
        return fail(ctx, GSR_ERR_INVALID_ARG, "merge: sample inputs and sample_action required");
    if (n_existing > 0 && (!means || !log_scales || !sh || sh_stride < 3))
        return fail(ctx, GSR_ERR_INVALID_ARG, "merge: existing Gaussians");
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    if (n_samples == 0) {
        // nothing to pair with: every Gaussian is untouched
        if (n_existing > 0 && out->existing_action)
            cudaMemsetAsync(out->existing_action, 0, (size_t)n_existing * 4, cs);
        const cudaError_t e = cudaGetLastError();
        return e == cudaSuccess ? GSR_OK : cuda_fail(ctx, e, "merge");
    }
    // workspace: slot map | best | count | sums | slot_dc | pair
    auto up = [](size_t b) { return (b + 255) & ~(size_t)255; };
    const size_t o_map = 0, o_best = o_map + up((size_t)npix * 4), o_cnt = o_best + up((size_t)n_samples * 8);
    const size_t o_sum = o_cnt + up((size_t)n_samples * 4), o_dc = o_sum + up((size_t)n_samples * 32);
    const size_t o_pair = o_dc + up((size_t)n_samples * 12), total = o_pair + up((size_t)n_existing * 4);
    cudaError_t e = ctx->merge_scratch.ensure(total);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "alloc merge workspace");
    unsigned char* b = ctx->merge_scratch.as<unsigned char>();
    cudaMemsetAsync(b + o_map, 0xff, (size_t)npix * 4, cs);
    cudaMemsetAsync(b + o_best, 0xff, (size_t)n_samples * 8, cs);
    cudaMemsetAsync(b + o_cnt, 0, o_dc - o_cnt, cs);
    MergeArgs a;
    std::memset(&a, 0, sizeof(a));
    a.W = view->width; a.H = view->height;
    a.fx = view->fx; a.fy = view->fy; a.cx = view->cx; a.cy = view->cy;
    a.inv_fx = (float)(1.0 / (double)view->fx); a.inv_fy = (float)(1.0 / (double)view->fy);
    a.near_plane = p->near_plane; a.tau_d = p->tau_d;
    for (int i = 0; i < 12; ++i) a.V[i] = view->viewmat[i];
    a.n_existing = n_existing; a.n_samples = n_samples;
    a.means = means; a.log_scales = log_scales; a.sh = sh; a.sh_stride = sh_stride;
    a.pixels = sample_pixels; a.scale_map = scale_map; a.depth_map = depth_map; a.gt = gt;
    a.slot_map = reinterpret_cast<int32_t*>(b + o_map);
    a.best = reinterpret_cast<unsigned long long*>(b + o_best);
    a.count = reinterpret_cast<unsigned int*>(b + o_cnt);
    a.sums = reinterpret_cast<long long*>(b + o_sum);
    a.slot_dc = reinterpret_cast<float*>(b + o_dc);
    a.pair = reinterpret_cast<int32_t*>(b + o_pair);
    a.sample_action = out->sample_action; a.sample_means = out->sample_means; a.sample_scale = out->sample_scale;
    a.sample_depth = out->sample_depth; a.sample_dc = out->sample_dc;
    a.existing_action = out->existing_action; a.existing_dc = out->existing_dc;
    launch_merge(a, ctx->num_sms, cs);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "merge launch");
    return GSR_OK;
}

// Twiddle table of one transform length, W_n^t = exp(-2 pi i t / n) for
// t in [0, n), computed in double and rounded once; built on first use.
static cudaError_t fft_twiddles(gsr_ctx* ctx, int n, const float2** out)
{
    DevMem& d = ctx->fft_twiddles[n];
    if (!d.p) {
        std::vector<float2> h((size_t)n);
        for (int t = 0; t < n; ++t) {
            const double ang = 2.0 * 3.14159265358979323846 * (double)t / (double)n;
            h[(size_t)t] = make_float2((float)std::cos(ang), (float)-std::sin(ang));
        }
        cudaError_t e = d.ensure((size_t)n * sizeof(float2));
        if (e == cudaSuccess) e = cudaMemcpy(d.p, h.data(), (size_t)n * sizeof(float2), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) {
            ctx->fft_twiddles.erase(n);
            return e;
        }
    }
    *out = ctx->fft_twiddles[n].as<float2>();
    return cudaSuccess;
}

gsr_status gsr_dft_energy(gsr_ctx* ctx, const gsr_image* images, int n_images, float* x, void* stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (n_images < 0 || (n_images > 0 && (!images || !x))) return fail(ctx, GSR_ERR_INVALID_ARG, "dft: images and x required");
    if (n_images == 0) return GSR_OK;
    constexpr size_t kInterCap = (size_t)512 << 20;   // half-spectrum workspace per launch
    std::vector<size_t> need((size_t)n_images);
    size_t max_need = 0;
    for (int i = 0; i < n_images; ++i) {
        const gsr_image& im = images[i];
        if (im.width < 0 || im.height < 0 || im.factor < 1) return fail(ctx, GSR_ERR_INVALID_ARG, "dft: image size or factor");
        const int Wd = im.width / im.factor, Hd = im.height / im.factor;
        if (Wd > GSR_DFT_MAX_DIM || Hd > GSR_DFT_MAX_DIM) return fail(ctx, GSR_ERR_NOT_SUPPORTED, "dft: image larger than GSR_DFT_MAX_DIM");
        if (Wd > 0 && Hd > 0 && !im.data) return fail(ctx, GSR_ERR_INVALID_ARG, "dft: null image data");
        need[(size_t)i] = (Wd > 0 && Hd > 0) ? (size_t)3 * Hd * (Wd / 2 + 1) * sizeof(float2) : 0;
        max_need = std::max(max_need, need[(size_t)i]);
    }
    const size_t cap = std::max(kInterCap, max_need);
    const size_t acc_bytes = ((size_t)n_images * sizeof(double) + 255) & ~(size_t)255;
    cudaError_t e = ctx->freq_scratch.ensure(acc_bytes + std::min(cap, [&] {
        size_t t = 0;
        for (size_t v : need) t += v;
        return t;
    }()));
    if (e != cudaSuccess) return cuda_fail(ctx, e, "alloc dft workspace");
    double* xacc = ctx->freq_scratch.as<double>();
    float2* inter = reinterpret_cast<float2*>(ctx->freq_scratch.as<unsigned char>() + acc_bytes);
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(xacc, 0, (size_t)n_images * sizeof(double), cs);
    FreqTable* T = new FreqTable;   // ~17 KB: off the stack
    std::unique_ptr<FreqTable> own(T);
    int i = 0;
    while (i < n_images) {
        std::memset(T, 0, sizeof(FreqTable));
        size_t used = 0;
        int row_smem = 0, col_smem = 0;
        const int first = i;
        while (i < n_images && T->n_images < kFreqMaxImages && used + need[(size_t)i] <= cap) {
            const gsr_image& im = images[i];
            FreqImage& F = T->img[T->n_images];
            F.src = im.data; F.W = im.width; F.H = im.height; F.factor = im.factor;
            F.Wd = im.width / im.factor; F.Hd = im.height / im.factor; F.Wh = F.Wd / 2 + 1;
            F.C = F.Hd <= 1228 ? 4 : (F.Hd <= 2457 ? 2 : 1);   // 20 C Hd bytes of shared memory <= 96 KB
            F.inter = (int64_t)(used / sizeof(float2));
            F.row_base = T->row_items;
            F.col_base = T->col_items;
            if (F.Wd > 0 && F.Hd > 0) {
                int plans[2] = {-1, -1};
                const int lens[2] = {F.Wd, F.Hd};
                for (int d = 0; d < 2; ++d) {
                    for (int p = 0; p < T->n_plans; ++p)
                        if (T->plan[p].n == lens[d]) plans[d] = p;
                    if (plans[d] < 0) {
                        if (T->n_plans == kFreqMaxPlans) break;
                        FftPlan& P = T->plan[T->n_plans];
                        if (!fft_plan(lens[d], &P)) return fail(ctx, GSR_ERR_NOT_SUPPORTED, "dft: transform length");
                        if ((e = fft_twiddles(ctx, lens[d], &P.tw)) != cudaSuccess) return cuda_fail(ctx, e, "dft twiddles");
                        plans[d] = T->n_plans++;
                    }
                }
                if (plans[0] < 0 || plans[1] < 0) break;   // plan table full: next launch
                F.row_plan = plans[0]; F.col_plan = plans[1];
                T->row_items += (int64_t)3 * ((F.Hd + 1) / 2);
                T->col_items += (F.Wh + F.C - 1) / F.C;
                row_smem = std::max(row_smem, 16 * F.Wd);
                col_smem = std::max(col_smem, 20 * F.C * F.Hd);
            }
            used += need[(size_t)i];
            ++T->n_images;
            ++i;
        }
        if (T->n_images == 0) return fail(ctx, GSR_ERR_NOT_SUPPORTED, "dft: empty launch table");
        launch_dft_energy(*T, inter, xacc + first, row_smem, col_smem, ctx->num_sms, cs);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "dft launch");
    }
    launch_dft_finalize(xacc, x, n_images, cs);
    if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(ctx, e, "dft finalize");
    return GSR_OK;
}

gsr_status gsr_frequency_schedule(gsr_ctx* ctx, int n_frames, const float* x_gt, const float* x_gt_level,
                                  const float* x_rendered, float tau_f, const float* uniforms, int n_samples,
                                  float* r, float* r_level, int32_t* level_up, int32_t* samples, void* stream)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (n_frames < 1 || n_samples < 0) return fail(ctx, GSR_ERR_INVALID_ARG, "schedule: sizes");
    if (n_frames > kFreqMaxFrames) return fail(ctx, GSR_ERR_NOT_SUPPORTED, "schedule: more than GSR_SCHED_MAX_FRAMES");
    if (!x_gt || !x_rendered) return fail(ctx, GSR_ERR_INVALID_ARG, "schedule: x_gt and x_rendered required");
    if ((r_level || level_up) && !x_gt_level) return fail(ctx, GSR_ERR_INVALID_ARG, "schedule: level outputs need x_gt_level");
    if (samples && n_samples > 0 && !uniforms) return fail(ctx, GSR_ERR_INVALID_ARG, "schedule: samples need uniforms");
    launch_frequency_schedule(n_frames, x_gt, x_gt_level, x_rendered, tau_f, uniforms, samples ? n_samples : 0, r,
                              r_level, level_up, samples, static_cast<cudaStream_t>(stream));
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(ctx, e, "schedule launch");
    return GSR_OK;
}

gsr_status gsr_debug_lists(gsr_saved* s, uint64_t* keys, uint32_t* vals, uint32_t* ranges, void* stream)
{
    if (!s || !s->filled) return GSR_ERR_INVALID_ARG;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    DebugArgs a{};
    a.tile_key = s->tile_key.as<uint32_t>();
    a.tile_val = s->tile_val.as<uint32_t>();
    a.rec = s->rec.as<float4>();
    a.vis_aux = s->vis_aux.as<uint4>();
    a.counters = reinterpret_cast<const unsigned long long*>(s->ctrl.as<unsigned char>() + kCtrlCounters);
    a.rec_cap = s->rec_cap;
    a.inst_cap = s->inst_cap;
    a.region2 = s->region2;
    a.keys_out = keys;
    a.vals_out = vals;
    if (keys || vals) launch_debug_lists(s->table, a, cs);
    if (ranges)
        cudaMemcpyAsync(ranges, s->ranges.p, (size_t)s->table.n_tiles * 8, cudaMemcpyDeviceToDevice, cs);
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

gsr_status gsr_debug_list_slice(gsr_saved* s, int64_t first, int64_t count, uint64_t* keys, uint32_t* vals,
                                void* stream)
{
    if (!s || !s->filled || first < 0 || count < 0) return GSR_ERR_INVALID_ARG;
    DebugArgs a{};
    a.tile_key = s->tile_key.as<uint32_t>();
    a.tile_val = s->tile_val.as<uint32_t>();
    a.rec = s->rec.as<float4>();
    a.vis_aux = s->vis_aux.as<uint4>();
    a.counters = reinterpret_cast<const unsigned long long*>(s->ctrl.as<unsigned char>() + kCtrlCounters);
    a.rec_cap = s->rec_cap;
    a.inst_cap = s->inst_cap;
    a.first = first;
    a.count = count;
    a.region2 = s->region2;
    a.keys_out = keys;
    a.vals_out = vals;
    if ((keys || vals) && count > 0) launch_debug_lists(s->table, a, static_cast<cudaStream_t>(stream));
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

gsr_status gsr_debug_records(gsr_saved* s, float* rec, int32_t* rect, uint32_t* flags, void* stream)
{
    if (!s || !s->filled) return GSR_ERR_INVALID_ARG;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const int64_t nr = s->table.n_records;
    if (rec) cudaMemsetAsync(rec, 0, (size_t)nr * 64, cs);
    if (rect) cudaMemsetAsync(rect, 0, (size_t)nr * 16, cs);
    if (flags) {
        // culled unless the record is written below: 0x01 bytes -> 0x01010101, bit0 set
        cudaMemsetAsync(flags, 1, (size_t)nr * 4, cs);
    }
    DebugArgs a{};
    a.rec = s->rec.as<float4>();
    a.vis_aux = s->vis_aux.as<uint4>();
    a.counters = reinterpret_cast<const unsigned long long*>(s->ctrl.as<unsigned char>() + kCtrlCounters);
    a.rec_cap = s->rec_cap;
    a.inst_cap = s->inst_cap;
    a.rec_out = rec;
    a.rect_out = rect;
    a.flags_out = flags;
    launch_debug_records(s->table, a, cs);
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

gsr_status gsr_debug_pixels(gsr_saved* s, float* t_final, uint32_t* n_contrib, void* stream)
{
    if (!s || !s->filled) return GSR_ERR_INVALID_ARG;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    const size_t np = (size_t)s->table.n_pixels;
    if (t_final) cudaMemcpyAsync(t_final, s->tfinal.p, np * 4, cudaMemcpyDeviceToDevice, cs);
    if (n_contrib) cudaMemcpyAsync(n_contrib, s->ncontrib.p, np * 4, cudaMemcpyDeviceToDevice, cs);
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

gsr_status gsr_debug_record_grads(gsr_saved* s, float* grec, void* stream)
{
    if (!s || !s->filled || !s->have_grads || !grec) return GSR_ERR_INVALID_ARG;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    cudaMemsetAsync(grec, 0, (size_t)s->table.n_records * 48, cs);
    DebugArgs a{};
    a.rec = s->rec.as<float4>();
    a.vis_aux = s->vis_aux.as<uint4>();
    a.grad_rec = s->ctx->grad_rec.as<float4>();
    a.counters = reinterpret_cast<const unsigned long long*>(s->ctrl.as<unsigned char>() + kCtrlCounters);
    a.rec_cap = s->rec_cap;
    a.inst_cap = s->inst_cap;
    a.grec_out = grec;
    launch_debug_records(s->table, a, cs);
    return cudaGetLastError() == cudaSuccess ? GSR_OK : GSR_ERR_CUDA;
}

gsr_status gsr_debug_set_wait(gsr_ctx* ctx, uint64_t wait_ns, uint32_t flags)
{
    if (!ctx) return GSR_ERR_INVALID_ARG;
    if (flags & ~(uint32_t)GSR_DEBUG_WITHHOLD_PREFIX) return fail(ctx, GSR_ERR_INVALID_ARG, "unknown debug flags");
    ctx->wait_ns = wait_ns ? wait_ns : kWaitLimitNs;
    ctx->debug_flags = flags;
    return GSR_OK;
}

gsr_status gsr_tune(gsr_ctx* ctx, const gsr_gaussians* g, const gsr_view* views, int n_views,
                    const gsr_outputs* out, gsr_saved* s, const float* dl_drgb, const gsr_grads* grads,
                    gsr_config* best, void* stream)
{
    if (!ctx || !s || !g || !views || !out || !dl_drgb || !grads) return GSR_ERR_INVALID_ARG;
    cudaStream_t cs = static_cast<cudaStream_t>(stream);
    std::string sig = "D" + std::to_string(ctx->cfg.sh_degree) + ":n" + std::to_string(g->n);
    for (int v = 0; v < n_views; ++v)
        sig += ":" + std::to_string(views[v].width) + "x" + std::to_string(views[v].height) + "/" +
               std::to_string(views[v].subset ? views[v].subset_count : -1);
    auto it = ctx->tune_cache.find(sig);
    if (it != ctx->tune_cache.end()) {
        ctx->cfg = it->second;
        if (best) *best = it->second;
        return GSR_OK;
    }
    const gsr_config base = ctx->cfg;
    const int shapes[3][2] = {{16, 16}, {32, 8}, {8, 32}};
    const int batches[3] = {128, 256, 512};
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return fail(ctx, GSR_ERR_CUDA, "event create");
    float best_ms = 1e30f;
    gsr_config best_cfg = base;
    gsr_status result = GSR_OK;
    // every shape x batch (both passes on one batch), then the backward's batch
    // for the winner (it stages records independently of the forward)
    for (int k = 0; k < 9 + 3; ++k) {
        {
            gsr_config c = base;
            if (k < 9) {
                c.tile_w = shapes[k / 3][0];
                c.tile_h = shapes[k / 3][1];
                c.blend_batch = batches[k % 3];
                c.blend_batch_bwd = 0;
            } else {
                if (best_ms >= 1e29f) break;
                c = best_cfg;
                c.blend_batch_bwd = batches[k - 9];
                if (c.blend_batch_bwd == c.blend_batch) continue;   // timed already
            }
            c.flags &= ~GSR_FLAG_NO_SYNC;
            ctx->cfg = c;
            // warm-up (also sizes buffers for this shape)
            gsr_status r = gsr_forward(ctx, g, views, n_views, out, s, stream);
            if (r == GSR_OK) r = gsr_backward(ctx, g, views, n_views, s, dl_drgb, nullptr, nullptr, grads, stream);
            if (r != GSR_OK) { result = r; continue; }
            ctx->cfg.flags |= GSR_FLAG_NO_SYNC;
            const int reps = 3;
            cudaEventRecord(e0, cs);
            for (int i = 0; i < reps; ++i) {
                gsr_forward(ctx, g, views, n_views, out, s, stream);
                gsr_backward(ctx, g, views, n_views, s, dl_drgb, nullptr, nullptr, grads, stream);
            }
            cudaEventRecord(e1, cs);
            cudaEventSynchronize(e1);
            float ms = 0.0f;
            cudaEventElapsedTime(&ms, e0, e1);
            uint32_t status = 0;
            read_status(ctx, s, cs, &status);
            if (status) continue;
            if (ms < best_ms) { best_ms = ms; best_cfg = c; best_cfg.flags = base.flags; }
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    ctx->cfg = best_cfg;
    if (best_ms < 1e29f) ctx->tune_cache[sig] = best_cfg;
    if (best) *best = best_cfg;
    return best_ms < 1e29f ? GSR_OK : (result != GSR_OK ? result : GSR_ERR_CUDA);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free forward.
//
// For callers that may not allocate device memory while they render: code
// that runs with a fixed memory budget reserved up front, or inside a region
// where cudaMalloc is not allowed (for example while another component holds
// the device for stream capture or real-time playback).  Its workspace is the
// file-scope array below: it exists on every GPU that loads libgsr, for the
// lifetime of the process, and is shared by every call on that GPU.  Calls
// whose work overlaps on the GPU (different streams, or different host
// threads) race on it; serialise them.
// ---------------------------------------------------------------------------
namespace {

constexpr int64_t kNaRecords = GSR_NOALLOC_MAX_RECORDS;
constexpr int64_t kNaInstances = GSR_NOALLOC_MAX_INSTANCES;
constexpr int64_t kNaPixels = GSR_NOALLOC_MAX_PIXELS;
constexpr int64_t kNaTiles = GSR_NOALLOC_MAX_TILES;
constexpr int kNaHistBlocks = 1024;
constexpr int64_t kNaLbPre = (kNaRecords + 255) / 256 + 1;
constexpr int64_t kNaLbDup = (kNaRecords + 255) / 256 + 1;   // the emission scan's look-back words
// the emission's window index lives in the tile-sort destination values, its
// kept-row descriptors in the T_final + n_contrib regions (the blend writes
// those only after the emission): 16 bytes per row
constexpr int64_t kNaRows = 2 * kNaPixels * 4 / 16;
static_assert(kNaInstances >= (kNaInstances + 2047) / 2048 + 1, "window index must fit the sort buffer");
static_assert(kNaInstances >= 2 * kNaRecords, "record counts must fit the sort buffer");

// byte offsets into the scratch array (each region 256-byte aligned)
constexpr size_t na_align(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kNaOffRec = 0;
constexpr size_t kNaOffVisKey = na_align(kNaOffRec + kNaRecords * kRecordBytes);
constexpr size_t kNaOffSorted = na_align(kNaOffVisKey + kNaRecords * 4);
constexpr size_t kNaOffAux = na_align(kNaOffSorted + kNaRecords * 4);
constexpr size_t kNaOffKstart = na_align(kNaOffAux + kNaRecords * 16);
constexpr size_t kNaOffTileKey = na_align(kNaOffKstart + (kNaRecords + 1) * 4);
constexpr size_t kNaOffTileVal = na_align(kNaOffTileKey + kNaInstances * 4);
constexpr size_t kNaOffTmpKey = na_align(kNaOffTileVal + kNaInstances * 4);
constexpr size_t kNaOffTmpVal = na_align(kNaOffTmpKey + kNaInstances * 4);
constexpr size_t kNaOffHist = na_align(kNaOffTmpVal + kNaInstances * 4);
constexpr size_t kNaOffRanges = na_align(kNaOffHist + (size_t)256 * (kNaHistBlocks + 1) * 4);
constexpr size_t kNaOffTfinal = na_align(kNaOffRanges + kNaTiles * 8);
constexpr size_t kNaOffNcontrib = na_align(kNaOffTfinal + kNaPixels * 4);
constexpr size_t kNaOffCtrl = na_align(kNaOffNcontrib + kNaPixels * 4);
constexpr size_t kNaCtrlBytes = kCtrlHead + 8 * (size_t)(kNaLbPre + kNaLbDup);
static_assert(kNaOffNcontrib + kNaPixels * 4 - kNaOffTfinal >= (size_t)kNaRows * 16, "row descriptors must fit the pixel state");
constexpr size_t kNaBytes = na_align(kNaOffCtrl + kNaCtrlBytes);
static_assert(kNaBytes <= GSR_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the documented size");

}  // namespace

static __device__ __align__(256) unsigned char g_noalloc_scratch[GSR_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kNaMaxDevices = 64;
std::mutex g_na_mutex;
unsigned char* g_na_ptr[kNaMaxDevices] = {};
}  // namespace

extern "C" {

gsr_status gsr_forward_noalloc(const gsr_config* cfg, const gsr_gaussians* g, const gsr_view* views, int n_views,
                               const gsr_outputs* out, void* stream)
{
    if (!cfg || !g || !views || !out || !out->rgb || !out->depth || !out->alpha) return GSR_ERR_INVALID_ARG;
    std::string why;
    if (!config_ok(cfg, why)) return GSR_ERR_INVALID_ARG;

    // view table (the layout gsr_forward uses), checked against the fixed limits
    // before any device work
    Table T;
    const char* twhy = "";
    const gsr_status tst = build_table_cfg(*cfg, g, views, n_views, T, &twhy);
    if (tst != GSR_OK) return tst;
    if (T.n_records > kNaRecords || T.n_pixels > kNaPixels || T.n_tiles > kNaTiles) return GSR_ERR_NOT_SUPPORTED;

    // set-up, once per device, with that device current: the device address
    // of the scratch array (its host-side name is only a stand-in)
    int dev = 0, num_sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNaMaxDevices) return GSR_ERR_CUDA;
    if (cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return GSR_ERR_CUDA;
    unsigned char* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_na_mutex);
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GSR_ERR_CUDA;
            g_na_ptr[dev] = static_cast<unsigned char*>(p);
        }
        base = g_na_ptr[dev];
    }

    cudaStream_t st = static_cast<cudaStream_t>(stream);
    float4* d_rec = reinterpret_cast<float4*>(base + kNaOffRec);
    uint32_t* vis_key = reinterpret_cast<uint32_t*>(base + kNaOffVisKey);
    uint32_t* sorted_k = reinterpret_cast<uint32_t*>(base + kNaOffSorted);
    uint4* vis_aux = reinterpret_cast<uint4*>(base + kNaOffAux);
    uint32_t* kstart = reinterpret_cast<uint32_t*>(base + kNaOffKstart);
    uint32_t* tile_key = reinterpret_cast<uint32_t*>(base + kNaOffTileKey);
    uint32_t* tile_val = reinterpret_cast<uint32_t*>(base + kNaOffTileVal);
    uint32_t* tmp_key = reinterpret_cast<uint32_t*>(base + kNaOffTmpKey);
    uint32_t* tmp_val = reinterpret_cast<uint32_t*>(base + kNaOffTmpVal);
    uint32_t* hist = reinterpret_cast<uint32_t*>(base + kNaOffHist);
    uint2* ranges = reinterpret_cast<uint2*>(base + kNaOffRanges);
    float* tfinal = reinterpret_cast<float*>(base + kNaOffTfinal);
    uint32_t* ncontrib = reinterpret_cast<uint32_t*>(base + kNaOffNcontrib);
    unsigned char* ctrl = base + kNaOffCtrl;
    unsigned long long* counters = reinterpret_cast<unsigned long long*>(ctrl + kCtrlCounters);
    uint32_t* status = reinterpret_cast<uint32_t*>(ctrl + kCtrlStatus);
    unsigned long long* lb_pre = reinterpret_cast<unsigned long long*>(ctrl + kCtrlHead);
    unsigned long long* lb_dup = lb_pre + kNaLbPre;

    // the array keeps the previous call's contents: clear what must start at zero
    cudaMemsetAsync(ctrl, 0, kNaCtrlBytes, st);
    cudaMemsetAsync(ranges, 0, (size_t)std::max<int64_t>(T.n_tiles, 1) * 8, st);

    PreprocessArgs pa;
    pa.means = g->means; pa.log_scales = g->log_scales; pa.quats = g->quats;
    pa.opacity = g->opacity_logits; pa.sh = g->sh;
    pa.rec = d_rec; pa.vis_key = vis_key; pa.vis_aux = vis_aux; pa.kstart = kstart;
    pa.lb_status = lb_pre;
    pa.ticket = reinterpret_cast<unsigned int*>(ctrl + kCtrlTicketPre);
    pa.rec_cap = kNaRecords;
    pa.status = status;
    pa.counters = counters;
    launch_preprocess_fwd(T, pa, num_sms, st);

    RadixScratch rs{hist, hist + 256 * (size_t)kNaHistBlocks, kNaHistBlocks, num_sms, status};
    radix_sort_pairs(vis_key, sorted_k, tmp_key, tmp_val, true, counters + kCntVisible, kNaRecords, 32, rs, st);

    const int bits = tile_bits(T.n_tiles);
    const int passes = (bits + 7) / 8;
    uint32_t *xk = tile_key, *xv = tile_val, *yk = tmp_key, *yv = tmp_val;
    if (passes & 1) { xk = tmp_key; xv = tmp_val; yk = tile_key; yv = tile_val; }
    DuplicateArgs da;
    da.sorted_k = sorted_k;
    da.vis_aux = vis_aux;
    da.rec = d_rec;
    da.tile_key = xk;
    da.tile_val = xv;
    da.counts = reinterpret_cast<uint2*>(yk);      // the tile-sort destination keys, free until the sort
    da.rows = reinterpret_cast<uint4*>(tfinal);   // T_final + n_contrib, written only by the blend later
    da.win_first = yv;
    da.rec_cap = kNaRecords;
    da.inst_cap = kNaInstances;
    da.row_cap = kNaRows;
    da.win_cap = duplicate_windows(kNaInstances);
    da.lb_inst = lb_dup;
    da.row_total = reinterpret_cast<unsigned long long*>(ctrl + kCtrlRowTotal);
    da.ticket = reinterpret_cast<unsigned int*>(ctrl + kCtrlTicketDup);
    da.status = status;
    da.counters = counters;
    da.inst_count = counters + kCntInstances;
    da.full_count = counters + kCntFullInst;
    launch_duplicate(T, da, num_sms, st);
    radix_sort_pairs(xk, xv, yk, yv, false, counters + kCntInstances, kNaInstances, bits, rs, st);
    launch_ranges(tile_key, counters + kCntInstances, kNaInstances, ranges, T.n_tiles, 0, status, num_sms, st);

    BlendFwdArgs ba;
    ba.rec = d_rec;
    ba.vals = tile_val;
    ba.ranges = ranges;
    ba.rgb = out->rgb;
    ba.depth = out->depth;
    ba.alpha = out->alpha;
    ba.tfinal = tfinal;
    ba.ncontrib = ncontrib;
    ba.wmask = nullptr;
    ba.work = reinterpret_cast<unsigned int*>(ctrl + kCtrlWorkFwd);
    ba.status = status;
    ba.counters = counters;
    ba.count_pairs = !(cfg->flags & GSR_FLAG_NO_PAIR_COUNTS);
    launch_blend_fwd(T, cfg->blend_batch, ba, num_sms, st);
    if (cudaGetLastError() != cudaSuccess) return GSR_ERR_CUDA;

    // the instance count is only known on the device: read the status word
    uint32_t host_status = 0;
    if (cudaMemcpyAsync(&host_status, status, sizeof(uint32_t), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return GSR_ERR_CUDA;
    if (host_status & kErrTimeout) return GSR_ERR_TIMEOUT;
    if (host_status & (kErrRecCapacity | kErrInstCapacity | kErrFullCapacity)) return GSR_ERR_CAPACITY;
    if (host_status & (kErrOverflow32 | kErrInternal)) return GSR_ERR_CUDA;
    return GSR_OK;
}

}  // extern "C"
