// gsr_kernels.h -- launch interface between the C ABI (gsr_api.cu) and the
// kernels.  Internal to libgsr.
#pragma once

#include <atomic>
#include <cstdint>
#include <cuda_runtime.h>

#include "gsr_common.cuh"

namespace gsr {

// number of kernels launched by the library in this process
extern std::atomic<long long> g_launches;

// A per-device value computed on first use (function attributes, occupancy):
// slots[device] holds it, 0 until set.  Host threads that race on the first
// use may both compute it (the computations are idempotent and give the same
// value); every read sees either 0 or the whole value.
constexpr int kMaxDevices = 64;
template <typename F>
inline int per_device_once(std::atomic<int>* slots, F compute)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) dev = 0;
    int v = slots[dev].load(std::memory_order_acquire);
    if (v == 0) {
        v = compute();
        slots[dev].store(v, std::memory_order_release);
    }
    return v;
}
#define GSR_COUNT_LAUNCH() (::gsr::g_launches.fetch_add(1, std::memory_order_relaxed))

// counters[] slots (uint64, device)
enum : int {
    kCntVisible = 0,     // visible records
    kCntInstances = 1,   // M
    kCntFwdPairs = 2,    // (pixel, entry) pairs examined by the forward
    kCntBwdPairs = 3,    // sum of per-pixel contributor counts
    kCntBlended = 4,     // (pixel, entry) pairs blended by the forward
    kCntWarpFwd = 5,     // (warp, entry) iterations of the forward after culling
    kCntWarpBwd = 6,     // (warp, entry) iterations of the backward after culling
    kCntFullInst = 7,    // instances of the 3-sigma rectangles (the lists before tile culling)
    kCntInstances2 = 8,  // kept instances of the second round of a two-round forward
    kCntOpenTiles = 9,   // tiles the first round of a two-round forward left open
    kCntSlots = 16,
};

// Two-round lists.  The first round lists, for every tile, only the records
// among the first prefix_records(n, f) of the n depth-ordered visible
// records: every such list is a prefix of the tile's full list (the lists
// are ordered by depth position).  A tile whose pixels all stop within that
// prefix is final; the others are left open and the second round lists them
// again over all n records.  f >= 1 is the plain single round.
__host__ __device__ inline int64_t prefix_records(int64_t n, float f)
{
    if (!(f < 1.0f) || n <= 0) return n;
    const double p = ceil((double)f * (double)n);
    return p < 1.0 ? 1 : (p >= (double)n ? n : (int64_t)p);
}

// Saturation histogram of the forward: bucket b < kSatBuckets collects the
// (estimated full) list lengths of the tiles whose pixels all stopped within
// the first x n depth-ordered records, x in [sat_edge(b), sat_edge(b + 1))
// (geometric edges from 2^-kSatOctaves to 1; bucket 0 also takes anything
// smaller), bucket kSatBuckets those of the tiles that never saturate.
constexpr int kSatBuckets = 64;
constexpr int kSatOctaves = 12;
__host__ __device__ inline double sat_edge(int b)
{
    return exp2(-(double)kSatOctaves + (double)kSatOctaves * (double)b / (double)kSatBuckets);
}
// The bucket of x = needed records / visible records (binary32 with the
// approximate base-2 logarithm: a bucket edge may move by a rounding, which
// only shifts a list length to the neighbouring bucket of a heuristic).
__device__ inline int sat_bucket(float x)
{
    if (!(x < 1.0f)) return kSatBuckets - 1;
    if (!(x > 0.0f)) return 0;
    const float t = (__log2f(x) + (float)kSatOctaves) * ((float)kSatBuckets / (float)kSatOctaves);
    const int b = (int)floorf(t);
    return b < 0 ? 0 : (b > kSatBuckets - 1 ? kSatBuckets - 1 : b);
}

// PreprocessArgs::debug_flags: the first look-back ticket keeps its prefix
// to itself, so every later ticket's wait runs out (timeout tests only).
constexpr uint32_t kDebugWithholdFirstPrefix = 1u;

struct PreprocessArgs {
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* opacity;
    const float* sh;
    float4* rec;                   // [rec_cap][4]
    uint32_t* vis_key;             // [rec_cap] float bits of camera z
    uint4* vis_aux;                // [rec_cap] (x0 | y0 << 16, x1 | y1 << 16, subset position, view)
    uint32_t* kstart;              // [n_slots + 1] first compact record of each Gaussian slot
    unsigned long long* lb_status; // [blocks] look-back words, zeroed
    unsigned int* ticket;          // zeroed
    int64_t rec_cap;
    uint32_t* status;
    unsigned long long* counters;
    int sub;                       // records per thread and ticket (1..8), set by launch_preprocess_fwd
    uint64_t wait_ns = kWaitLimitNs;  // limit of each look-back wait
    uint32_t debug_flags = 0;      // kDebugWithholdFirstPrefix (tests only): ticket 0 never publishes
};

struct PreprocessBwdArgs {
    const float* means;
    const float* log_scales;
    const float* quats;
    const float* opacity;
    const float* sh;
    const uint4* vis_aux;
    const uint32_t* kstart;
    const float4* grad_rec;        // [n_vis][3]
    float* grad_means;
    float* grad_log_scales;
    float* grad_quats;
    float* grad_opacity;
    float* grad_sh;
    float* grad_pose;              // [n_views][6] or nullptr
    float* grad_focal;             // [n_views][2] (fx, fy) or nullptr
    uint32_t* queue;               // [queue_cap] records whose geometry adjoint runs in double-float
    unsigned int* queue_count;     // zeroed before the group passes
    int64_t queue_cap;             // >= visible records
    uint32_t* status;              // the forward's: the kernels skip their work after a timed-out wait
    unsigned long long* grad_rows; // += gradient rows written (one per Gaussian and view group)
};

void launch_preprocess_fwd(const Table& T, const PreprocessArgs& a, int num_sms, cudaStream_t s);
void launch_preprocess_bwd(const Table& T, int group, const PreprocessBwdArgs& a, int num_sms, cudaStream_t s);
void launch_preprocess_bwd64(const Table& T, const PreprocessBwdArgs& a, int num_sms, cudaStream_t s);
int64_t preprocess_blocks(const Table& T);   // look-back words the forward may use (its largest ticket count)

// Rig chain: per-keyframe central-pose and per-camera focal gradients from
// the per-view ones (one block; binary64 sums in view order).
struct RigTable {
    int n_views, n_keyframes, n_cameras;
    int kf[kMaxViews], cam[kMaxViews];
    float rel[kMaxViews][12];   // row-major [R | t]
};
void launch_rig_chain(const RigTable& T, const float* pose_grads, const float* focal_grads, float* central,
                      float* camera_rel, float* camera_focal, cudaStream_t s);

// ---- sort -----------------------------------------------------------------
struct RadixScratch {
    uint32_t* hist;   // [256 * max_blocks]
    uint32_t* dtot;   // [256]
    int max_blocks;
    int num_sms;
    uint32_t* status; // device status word (kErrInternal on an out-of-range position)
    uint64_t wait_ns = kWaitLimitNs;   // limit of each mbarrier wait
};

// Stable LSD sort of `bits` low bits of (key, val) pairs; the count is read
// on the device from *n_dev (clamped to cap).  vals_in == nullptr means the
// values are the input positions 0..n-1.  Ping-pongs between (k0, v0) and
// (k1, v1); returns 0 if the result is in (k0, v0), 1 if in (k1, v1).
int radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, bool implicit_vals,
                     const unsigned long long* n_dev, int64_t cap, int bits, const RadixScratch& rs,
                     cudaStream_t s);

struct DuplicateArgs {
    const uint32_t* sorted_k;      // depth-ordered compact record ids
    const uint4* vis_aux;
    const float4* rec;             // projected records (the tile culling reads u, v, conic, sigma)
    uint32_t* tile_key;            // [inst_cap] kept instances: global tile id
    uint32_t* tile_val;            // [inst_cap] kept instances: compact record id
    uint2* counts;                 // [rec_cap] scratch: per depth-ordered record (kept instances, kept rows)
    uint4* rows;                   // [row_cap] scratch: per kept tile row {record, first tile id, count, first instance}
    uint32_t* win_first;           // [win_cap] scratch: the row holding each window's first instance
    int64_t rec_cap, inst_cap;     // visible records; kept instances
    int64_t row_cap, win_cap;      // row descriptors; duplicate_windows(inst_cap)
    unsigned long long* lb_inst;   // [duplicate_blocks(rec_cap)] zeroed: look-back of the (row, instance) counts
    unsigned long long* row_total; // zeroed: kept rows of the batch (exact, summed by dup_count)
    unsigned int* ticket;          // zeroed
    uint32_t* status;
    unsigned long long* counters;  // counters[kCntVisible] = n; counters[kCntOpenTiles] read by a second round
    unsigned long long* inst_count;  // zeroed: kept instances of this emission (exact)
    unsigned long long* full_count = nullptr;  // += 3-sigma rectangle instances (nullptr: not counted)
    uint64_t wait_ns = kWaitLimitNs;   // limit of each look-back wait
    // Two-round lists: this emission covers the first prefix_records(n,
    // prefix) depth-ordered records; open_tiles != nullptr makes it a second
    // round, which lists only the tiles whose bit is set (nothing at all when
    // counters[kCntOpenTiles] is 0).
    float prefix = 1.0f;
    const uint32_t* open_tiles = nullptr;   // [ceil(n_tiles / 32)] bit t: tile t is open
    uint32_t* depthpos = nullptr;           // [rec_cap] if set: each covered record's depth position
    // [kSatBuckets] if set (an unfiltered emission of every record): the
    // kept instances of the records of depth share in each saturation bucket
    unsigned long long* inst_hist = nullptr;
};
void launch_duplicate(const Table& T, const DuplicateArgs& a, int num_sms, cudaStream_t s);
int64_t duplicate_blocks(int64_t rec_cap);     // look-back words of the scan
int64_t duplicate_windows(int64_t inst_cap);   // win_cap for inst_cap kept instances

// A key outside [0, n_tiles) sets kErrInternal and is skipped.  Positions
// are written as offset + index (the list region's start).
void launch_ranges(const uint32_t* sorted_tile_keys, const unsigned long long* m_dev, int64_t cap, uint2* ranges,
                   int64_t n_tiles, int64_t offset, uint32_t* status, int num_sms, cudaStream_t s);

// ---- blend ----------------------------------------------------------------
struct BlendFwdArgs {
    const float4* rec;
    const uint32_t* vals;
    const uint2* ranges;
    float* rgb;
    float* depth;
    float* alpha;
    float* tfinal;
    uint32_t* ncontrib;
    uint8_t* wmask;                // [inst_cap] bit w: warp w composited this list entry (may be nullptr)
    unsigned int* work;            // zeroed tile counter
    uint32_t* status;
    unsigned long long* counters;
    uint64_t wait_ns = kWaitLimitNs;   // limit of each mbarrier wait
    bool count_pairs = true;       // examined and composited pair counters
    // Two-round lists.  round: 0 for a forward of one round; 1 for the
    // first of two, which renders the prefix lists (the first
    // prefix_records(n, prefix) records), finishes the tiles whose pixels
    // all stop there and sets the others' bits in open_tiles (counting them
    // in counters[kCntOpenTiles]); 2 for the second of two, which renders
    // only the open tiles, over their full lists.  Outputs and statistics
    // are written by the pass that finishes a tile.
    int round = 0;
    float prefix = 1.0f;
    uint32_t* open_tiles = nullptr;
    const uint32_t* depthpos = nullptr;     // with hist: record -> depth position
    unsigned long long* hist = nullptr;     // [kSatBuckets + 1] saturation histogram, or nullptr
};

struct BlendBwdArgs {
    const float4* rec;
    const uint32_t* vals;
    const uint2* ranges;
    const float* tfinal;
    const uint32_t* ncontrib;
    const float* dl_rgb;
    const float* dl_depth;         // may be nullptr
    const float* dl_alpha;         // may be nullptr
    const uint8_t* wmask;          // written by the forward that filled the saved state
    float4* grad_rec;              // [n_vis][3], zeroed
    unsigned int* work;            // zeroed tile counter
    uint32_t* status;
    unsigned long long* counters;
    uint64_t wait_ns = kWaitLimitNs;   // limit of each mbarrier wait
};

bool blend_supported(int tile_w, int tile_h, int batch);
void launch_blend_fwd(const Table& T, int batch, const BlendFwdArgs& a, int num_sms, cudaStream_t s);
void launch_blend_bwd(const Table& T, int batch, const BlendBwdArgs& a, int num_sms, cudaStream_t s);

// ---- insertion probability (Sec. 3.2, Eq. 4-6) -------------------------------
constexpr int kInsMaxRadius = 7;
constexpr int kInsMaxTaps = (2 * kInsMaxRadius + 1) * (2 * kInsMaxRadius + 1);

struct InsertTable {
    int n_views, r;
    float tau;
    int W[kMaxViews], H[kMaxViews], TX[kMaxViews];   // TX: 32x32-pixel tiles per row
    float f[kMaxViews];                              // focal length (fx) of each view
    int64_t tile_base[kMaxViews + 1];                // first 32x32 tile of each view
    int64_t pix_base[kMaxViews + 1];                 // first pixel of each view
    float taps[kInsMaxTaps];                         // (2r+1)^2 zero-mean LoG taps, row-major
};

// Zero-mean LoG taps for sigma (host, double, rounded once to binary32).
void insertion_taps(double sigma, int* radius, float* taps);
int64_t insertion_lb_words(int64_t n_pixels);
// count == nullptr skips the compaction; *count, lb and *ticket start at zero.
void launch_insertion(const InsertTable& T, const float* gt, const float* rendered, const float* depth, float* p_a,
                      float* scale, uint32_t* index, int64_t index_cap, unsigned long long* count,
                      unsigned long long* lb, unsigned int* ticket, uint32_t* status, uint64_t wait_ns, int num_sms,
                      cudaStream_t s);

// ---- frequency scheduler (Sec. 3.3, Eq. 9-12) -------------------------------
constexpr int kFreqMaxImages = 192;     // images per launch table
constexpr int kFreqMaxDim = 4096;       // width and height after downsampling
constexpr int kFreqMaxPlans = 32;       // distinct transform lengths per table
constexpr int kFftMaxStages = 8;        // lengths <= 4096 need at most 7 passes
constexpr int kFreqMaxFrames = 4096;

// One Stockham pass: radix R, Ns = product of the earlier radices, m = n / R
// butterflies per sequence, twiddle stride n / (Ns R), and multiply-high
// reciprocals ceil(2^32 / d) of m, Ns and R (exact quotients of x < 2^16).
struct FftStage {
    int R, Ns, m, step;
    uint32_t mag_m, mag_ns, mag_r, pad;
};

// Mixed-radix Stockham plan of one transform length: passes in order and the
// table of W_n^t = exp(-2 pi i t / n), t in [0, n) (device).
struct FftPlan {
    int n, n_stages;
    FftStage st[kFftMaxStages];
    const float2* tw;
};

struct FreqImage {
    const float* src;            // planar RGB [3][H][W]
    int W, H, factor;            // source size and box-downsampling factor
    int Wd, Hd, Wh, C;           // transformed size, Wh = Wd/2 + 1, columns per column item
    int row_plan, col_plan;      // plans of length Wd and Hd
    int64_t inter;               // offset (float2) of the half spectra [3][Hd][Wh]
    int64_t row_base, col_base;  // first row-pass / column-pass item
};

struct FreqTable {
    int n_images, n_plans;
    int64_t row_items, col_items;
    FftPlan plan[kFreqMaxPlans];
    FreqImage img[kFreqMaxImages];
};

bool fft_plan(int n, FftPlan* plan);   // passes of length n (tw left to the caller); false if unsupported
void launch_dft_energy(const FreqTable& T, float2* inter, double* xacc, int row_smem, int col_smem, int num_sms,
                       cudaStream_t s);
void launch_dft_finalize(const double* xacc, float* x, int n, cudaStream_t s);
void launch_frequency_schedule(int n_frames, const float* x_gt, const float* x_gt_level, const float* x_rendered,
                               float tau_f, const float* uniforms, int n_samples, float* r, float* r_level,
                               int32_t* level_up, int32_t* samples, cudaStream_t s);

// ---- inter-camera merging (Sec. 3.2, Eq. 7-8) --------------------------------
enum : int32_t { kMergeInsert = 0, kMergeMerged = 1, kMergeReplaces = 2 };    // sample actions
enum : int32_t { kMergeUntouched = 0, kMergeRemoved = 1, kMergeKept = 2 };    // existing actions

struct MergeArgs {
    int W, H;
    float fx, fy, cx, cy, near_plane, tau_d;
    float inv_fx, inv_fy;               // 1 / fx, 1 / fy (rounded once from double)
    float V[12];                        // row-major [R | t], world to camera i
    int64_t n_existing, n_samples;
    const float* means;                 // [n_existing][3]
    const float* log_scales;            // [n_existing][3]
    const float* sh;                    // DC of Gaussian g at sh + g * sh_stride
    int64_t sh_stride;
    const uint32_t* pixels;             // [n_samples] sampled pixel indices of camera i
    const float* scale_map;             // [H][W] S of Eq. 6
    const float* depth_map;             // [H][W] camera depth
    const float* gt;                    // [3][H][W]
    int32_t* slot_map;                  // [H][W] scratch, -1 = no sample
    unsigned long long* best;           // [n_samples] scratch, ~0
    unsigned int* count;                // [n_samples] scratch, 0
    long long* sums;                    // [n_samples][4] scratch, 0: DC x 2^32, z x 2^24
    float* slot_dc;                     // [n_samples][3] scratch
    int32_t* pair;                      // [n_existing] scratch
    int32_t* sample_action;             // [n_samples]
    float* sample_means;                // [n_samples][3] or nullptr
    float* sample_scale;                // [n_samples] or nullptr
    float* sample_depth;                // [n_samples] or nullptr
    float* sample_dc;                   // [n_samples][3] or nullptr
    int32_t* existing_action;           // [n_existing] or nullptr
    float* existing_dc;                 // [n_existing][3] or nullptr; KEPT rows written
};
void launch_merge(const MergeArgs& a, int num_sms, cudaStream_t s);

// ---- misc -----------------------------------------------------------------
void launch_l1_loss_grad(const float* rgb, const float* target, int64_t n, float* dl, float* loss, cudaStream_t s);

struct DebugArgs {
    const uint32_t* tile_key;
    const uint32_t* tile_val;
    const float4* rec;
    const uint4* vis_aux;
    const float4* grad_rec;
    const unsigned long long* counters;
    int64_t rec_cap, inst_cap;
    int64_t first = 0, count = INT64_MAX;   // list positions exported by launch_debug_lists
    // a two-round forward's second list region starts at position region2
    // (-1: one region); positions in neither region's filled part export zeros
    int64_t region2 = -1;
    uint64_t* keys_out;
    uint32_t* vals_out;
    float* rec_out;                // [n_records][16]
    int32_t* rect_out;             // [n_records][4]
    uint32_t* flags_out;           // [n_records]
    float* grec_out;               // [n_records][12]
};
void launch_debug_lists(const Table& T, const DebugArgs& a, cudaStream_t s);
void launch_debug_records(const Table& T, const DebugArgs& a, cudaStream_t s);

}  // namespace gsr
