// gsr_radix.cu -- the project's stable LSD radix sort of (u32 key, u32 value)
// pairs, used twice per forward (visible records by depth bits, instances by
// tile id).
//
// One pass over a digit of <= 8 bits is three launches:
//   upsweep   G blocks, each counts the digits of its contiguous chunk
//             (warp-aggregated shared-memory histogram) -> hist[digit][block];
//   scan      256 blocks, block d turns row d of hist into exclusive offsets
//             along the blocks and writes the digit total;
//   scatter   G blocks walk their chunk in sub-tiles of 2048 items, each
//             gathered into shared memory by bulk asynchronous copies on an
//             mbarrier, double-buffered (the next sub-tile streams in while
//             the current one is ranked): ranks
//             within a warp come from one ballot per digit bit, ranks within the
//             sub-tile from per-digit prefix sums over the warps; the sub-tile
//             is reordered by digit in shared memory and written out as
//             contiguous per-digit runs (coalesced), each run continuing where
//             the block's previous sub-tile of that digit ended.
// Chunks are contiguous and processed in order, ranks follow input order:
// the sort is stable.  The item count is read on the device (so no host
// synchronisation is needed between producing the items and sorting them).
#include <algorithm>

#include "gsr_common.cuh"
#include "gsr_kernels.h"

namespace gsr {

constexpr int kRT = 256;                // threads per block = digit bins
constexpr int kRounds = 8;               // 32-item rounds per warp per sub-tile
constexpr int kSub = kRT * kRounds;      // items per sub-tile

__device__ __forceinline__ int64_t radix_count(const unsigned long long* n_dev, int64_t cap)
{
    const unsigned long long n = *n_dev;
    return n < (unsigned long long)cap ? (int64_t)n : cap;
}

__device__ __forceinline__ void radix_chunk(int64_t n, int G, int b, int64_t& start, int64_t& end)
{
    // chunk length rounded up to whole sub-tiles
    int64_t chunk = (n + G - 1) / G;
    chunk = (chunk + kSub - 1) / kSub * kSub;
    start = (int64_t)b * chunk;
    end = min(n, start + chunk);
}

// Block-wide exclusive scan of one value per thread (kRT threads).
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t* s_warp, uint32_t& total)
{
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[w] = incl;
    __syncthreads();
    if (w == 0) {
        const uint32_t x = lane < kRT / 32 ? s_warp[lane] : 0u;
        uint32_t ix = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, ix, o);
            if (lane >= o) ix += t;
        }
        if (lane < kRT / 32) s_warp[lane] = ix - x;
        if (lane == kRT / 32 - 1) s_warp[kRT / 32] = ix;
    }
    __syncthreads();
    const uint32_t r = s_warp[w] + incl - v;
    total = s_warp[kRT / 32];
    __syncthreads();
    return r;
}

__global__ void __launch_bounds__(kRT)
radix_upsweep_kernel(const uint32_t* __restrict__ keys, const unsigned long long* n_dev, int64_t cap, int shift,
                     uint32_t mask, uint32_t* __restrict__ hist, int G)
{
    // one private histogram per warp: shared atomics contend only within a warp
    __shared__ uint32_t h[kRT / 32][256];
    const int tid = threadIdx.x, w = tid >> 5;
#pragma unroll
    for (int i = 0; i < kRT / 32; ++i) h[i][tid] = 0;
    __syncthreads();
    int64_t start, end;
    radix_chunk(radix_count(n_dev, cap), G, blockIdx.x, start, end);
    uint32_t* hw = h[w];
    if (start < end) {
        // start is a multiple of the sub-tile: 16-byte aligned vector loads,
        // four in flight per thread, scalar tail
        const int64_t v0 = start >> 2, v1 = end >> 2;
        const uint4* k4 = reinterpret_cast<const uint4*>(keys);
        for (int64_t v = v0 + tid; v < v1; v += 4 * kRT) {
            uint4 q[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) q[u] = v + u * kRT < v1 ? k4[v + u * kRT] : make_uint4(0, 0, 0, 0);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                if (v + u * kRT < v1) {
                    atomicAdd(&hw[(q[u].x >> shift) & mask], 1u);
                    atomicAdd(&hw[(q[u].y >> shift) & mask], 1u);
                    atomicAdd(&hw[(q[u].z >> shift) & mask], 1u);
                    atomicAdd(&hw[(q[u].w >> shift) & mask], 1u);
                }
            }
        }
        const int64_t i = (v1 << 2) + tid;
        if (tid < 4 && i < end) atomicAdd(&hw[(keys[i] >> shift) & mask], 1u);
    }
    __syncthreads();
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < kRT / 32; ++i) s += h[i][tid];
    hist[(size_t)tid * G + blockIdx.x] = s;
}

// Block d: exclusive scan of hist[d][0..G) in place; dtot[d] = row total.
__global__ void __launch_bounds__(kRT)
radix_scan_kernel(uint32_t* __restrict__ hist, int G, uint32_t* __restrict__ dtot)
{
    __shared__ uint32_t s_warp[kRT / 32 + 1];
    uint32_t* row = hist + (size_t)blockIdx.x * G;
    const int per = (G + kRT - 1) / kRT;
    const int s = threadIdx.x * per, e = min(G, s + per);
    uint32_t sum = 0;
    for (int i = s; i < e; ++i) sum += row[i];
    uint32_t total;
    uint32_t run = block_excl_scan(sum, s_warp, total);
    for (int i = s; i < e; ++i) {
        const uint32_t v = row[i];
        row[i] = run;
        run += v;
    }
    if (threadIdx.x == 0) dtot[blockIdx.x] = total;
}

// Dynamic shared memory of the scatter: two stages of one sub-tile's keys
// and values, filled by bulk asynchronous copies (the TMA engine) so that the
// next sub-tile streams in while the current one is ranked.
constexpr size_t kScatterStageBytes = (size_t)2 * 2 * kSub * sizeof(uint32_t);

__global__ void __launch_bounds__(kRT)
radix_scatter_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, bool implicit_vals,
                     uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const unsigned long long* n_dev,
                     int64_t cap, int shift, uint32_t mask, const uint32_t* __restrict__ hist,
                     const uint32_t* __restrict__ dtot, int G, uint32_t* status, uint64_t wait_ns)
{
    extern __shared__ __align__(128) uint32_t s_stage[];   // [2 stages][keys, values][kSub]
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ uint32_t whist[kRT / 32][256];
    __shared__ uint32_t s_run[256], s_start[256], s_tot[256];
    __shared__ uint32_t s_warp[kRT / 32 + 1];
    __shared__ uint32_t sk[kSub], sv[kSub];
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    int64_t start, end;
    const int64_t n_items = radix_count(n_dev, cap);
    radix_chunk(n_items, G, blockIdx.x, start, end);
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    {
        uint32_t t;   // (the scan's barriers also publish the mbarrier initialisation)
        const uint32_t dbase = block_excl_scan(dtot[tid], s_warp, t);
        s_run[tid] = dbase + hist[(size_t)tid * G + blockIdx.x];
    }
    const int nsub = start < end ? (int)((end - start + kSub - 1) / kSub) : 0;
    // thread 0: gather sub-tile t into stage t & 1 (whole 16-byte words only;
    // sub-tiles start on 8 KB boundaries of the arrays)
    auto issue = [&](int t) {
        const int64_t sub = start + (int64_t)t * kSub;
        const int cnt = (int)min((int64_t)kSub, end - sub);
        const uint32_t bulk = (uint32_t)(cnt & ~3) * 4u;
        uint32_t* dk = s_stage + (size_t)(t & 1) * 2 * kSub;
        mbar_arrive_expect_tx(&s_bar[t & 1], implicit_vals ? bulk : 2u * bulk);
        if (bulk) {
            bulk_g2s(dk, kin + sub, bulk, &s_bar[t & 1]);
            if (!implicit_vals) bulk_g2s(dk + kSub, vin + sub, bulk, &s_bar[t & 1]);
        }
    };
    if (tid == 0 && nsub > 0) issue(0);
    uint32_t par0 = 0u, par1 = 0u;
    const uint32_t lt = (1u << lane) - 1u;
    const int width = __popc(mask);
    for (int t = 0; t < nsub; ++t) {
        const int s = t & 1;
        const int64_t sub = start + (int64_t)t * kSub;
        const int cnt = (int)min((int64_t)kSub, end - sub);
        uint32_t* stk = s_stage + (size_t)s * 2 * kSub;
        uint32_t* stv = stk + kSub;
        // the other stage was last read before the previous iteration's final barrier
        if (tid == 0 && t + 1 < nsub) issue(t + 1);
        // the last (< 4) items of a ragged sub-tile are read directly
        const int tail0 = cnt & ~3;
        if (tid < cnt - tail0) {
            stk[tail0 + tid] = kin[sub + tail0 + tid];
            if (!implicit_vals) stv[tail0 + tid] = vin[sub + tail0 + tid];
        }
#pragma unroll
        for (int i = 0; i < kRT / 32; ++i) whist[i][tid] = 0;
        const bool ok = mbar_wait_bounded(&s_bar[s], s ? par1 : par0, status, wait_ns);
        if (s) par1 ^= 1u; else par0 ^= 1u;
        if (__syncthreads_or(!ok)) {
            // leave no copy in flight into this block's shared memory
            if (t + 1 < nsub) mbar_wait_bounded(&s_bar[s ^ 1], s ? par0 : par1, status, wait_ns);
            return;
        }
        uint32_t local[kRounds];
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const int idx = w * (32 * kRounds) + r * 32 + lane;
            const bool valid = idx < cnt;
            const uint32_t d = valid ? (stk[idx] >> shift) & mask : 0u;
            // lanes holding the same digit: one ballot per digit bit
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                if (bit >= width) break;   // digits of fewer than 8 bits
                const bool on = (d >> bit) & 1u;
                const uint32_t bb = __ballot_sync(0xffffffffu, on);
                peers &= on ? bb : ~bb;
            }
            local[r] = 0u;
            const uint32_t prior = valid ? whist[w][d] : 0u;
            const uint32_t rank = __popc(peers & lt);
            __syncwarp();
            if (valid && rank == 0) whist[w][d] = prior + __popc(peers);
            __syncwarp();
            if (valid) local[r] = prior + rank;
        }
        __syncthreads();
        // thread tid = digit: prefix over warps, sub-tile total, digit start in the sub-tile
        uint32_t acc = 0;
#pragma unroll
        for (int ww = 0; ww < kRT / 32; ++ww) {
            const uint32_t c = whist[ww][tid];
            whist[ww][tid] = acc;
            acc += c;
        }
        s_tot[tid] = acc;
        uint32_t tot_all;
        const uint32_t my_start = block_excl_scan(acc, s_warp, tot_all);
        s_start[tid] = my_start;
        __syncthreads();   // every digit's start is visible before any thread uses it
        // reorder the sub-tile by digit in shared memory
#pragma unroll
        for (int r = 0; r < kRounds; ++r) {
            const int idx = w * (32 * kRounds) + r * 32 + lane;
            if (idx < cnt) {
                const uint32_t key = stk[idx];
                const uint32_t d = (key >> shift) & mask;
                const uint32_t lpos = s_start[d] + whist[w][d] + local[r];
                if (lpos < (uint32_t)kSub) {
                    sk[lpos] = key;
                    sv[lpos] = implicit_vals ? (uint32_t)(sub + idx) : stv[idx];
                } else {
                    atomicOr(status, kErrInternal);
                }
            }
        }
        __syncthreads();
        // contiguous per-digit runs to global memory
        for (uint32_t i = tid; i < tot_all; i += kRT) {
            const uint32_t k = sk[i];
            const uint32_t d = (k >> shift) & mask;
            const uint32_t g = s_run[d] + (i - s_start[d]);
            if ((int64_t)g < n_items) {
                kout[g] = k;
                vout[g] = sv[i];
            } else {
                atomicOr(status, kErrInternal);
            }
        }
        __syncthreads();
        s_run[tid] += s_tot[tid];
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// Small sorts in one launch: up to kSmallN items, one block of kSmallThreads,
// keys and values ping-ponging in shared memory.  Per pass of 8 bits, warp w
// owns the contiguous slice [w S, (w + 1) S) of the current order and ranks
// it in rounds of 32 consecutive items: the lanes holding the same digit come
// from one ballot per digit bit (cheaper here than the hardware match), a
// lane's rank is its warp's running count of the digit plus the matching lanes
// before it; a digit's place is the total of smaller digits plus the counts of
// the earlier warps.  Slices, rounds and lanes follow
// the current order, so each pass is stable.
// ---------------------------------------------------------------------------
constexpr int kSmallThreads = 1024;
constexpr int kSmallWarps = kSmallThreads / 32;
constexpr int kSmallN = 10240;
constexpr int kSmallPer = kSmallN / kSmallThreads;   // items per lane per pass
constexpr size_t kSmallSmem = (size_t)4 * kSmallN * 4 + (size_t)kSmallWarps * 256 * 4 + (256 + 8) * 4;

__global__ void __launch_bounds__(kSmallThreads)
radix_small_kernel(const uint32_t* __restrict__ kin, const uint32_t* __restrict__ vin, bool implicit_vals,
                   uint32_t* __restrict__ kout, uint32_t* __restrict__ vout, const unsigned long long* n_dev,
                   int64_t cap, int bits, int passes, int digit)
{
    extern __shared__ __align__(16) uint32_t sm[];
    uint32_t* sk0 = sm;
    uint32_t* sv0 = sk0 + kSmallN;
    uint32_t* sk1 = sv0 + kSmallN;
    uint32_t* sv1 = sk1 + kSmallN;
    uint32_t* whist = sv1 + kSmallN;                 // [kSmallWarps][256]
    uint32_t* dbase = whist + kSmallWarps * 256;     // [256]
    uint32_t* dwarp = dbase + 256;                   // [8] digit-scan carries
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    const int n = (int)radix_count(n_dev, cap < kSmallN ? cap : kSmallN);
    for (int i = tid; i < n; i += kSmallThreads) {
        sk0[i] = kin[i];
        sv0[i] = implicit_vals ? (uint32_t)i : vin[i];
    }
    const int S = (n + kSmallWarps - 1) / kSmallWarps;   // slice per warp
    const uint32_t lt = (1u << lane) - 1u;
    int shift = 0;
    for (int p = 0; p < passes; ++p) {
        const int width = (shift + digit > bits) ? bits - shift : digit;
        const uint32_t mask = (1u << width) - 1u;
        for (int i = tid; i < kSmallWarps * 256; i += kSmallThreads) whist[i] = 0u;
        __syncthreads();
        uint32_t* wh = whist + w * 256;
        uint32_t dg[kSmallPer], rk[kSmallPer];
#pragma unroll
        for (int r = 0; r < kSmallPer; ++r) {
            const int o = r * 32 + lane;
            const int i = w * S + o;
            const bool valid = o < S && i < n;
            const uint32_t d = valid ? (sk0[i] >> shift) & mask : 0xffffffffu;
            uint32_t peers = __ballot_sync(0xffffffffu, valid);
#pragma unroll
            for (int bit = 0; bit < 8; ++bit) {
                const bool on = (d >> bit) & 1u;
                const uint32_t bb = __ballot_sync(0xffffffffu, on);
                peers &= on ? bb : ~bb;
            }
            const uint32_t prior = valid ? wh[d] : 0u;
            __syncwarp();
            if (valid && (peers & lt) == 0u) wh[d] = prior + __popc(peers);
            __syncwarp();
            dg[r] = d;
            rk[r] = prior + __popc(peers & lt);
        }
        __syncthreads();
        // digit t: its total over the warps (the warps' exclusive prefix left
        // in whist), then the exclusive scan of the totals over the digits:
        // within each of the first eight warps by shuffles, then across them
        uint32_t dex = 0;
        if (tid < 256) {
            uint32_t acc = 0;
            for (int ww = 0; ww < kSmallWarps; ++ww) {
                const uint32_t c = whist[ww * 256 + tid];
                whist[ww * 256 + tid] = acc;
                acc += c;
            }
            uint32_t incl = acc;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            if (lane == 31) dwarp[w] = incl;
            dex = incl - acc;
        }
        __syncthreads();
        if (tid < 256) {
            uint32_t carry = 0;
            for (int ww = 0; ww < w; ++ww) carry += dwarp[ww];
            dbase[tid] = carry + dex;
        }
        __syncthreads();
#pragma unroll
        for (int r = 0; r < kSmallPer; ++r) {
            const int o = r * 32 + lane;
            const int i = w * S + o;
            if (o < S && i < n) {
                const uint32_t pos = dbase[dg[r]] + wh[dg[r]] + rk[r];
                sk1[pos] = sk0[i];
                sv1[pos] = sv0[i];
            }
        }
        __syncthreads();
        uint32_t* t = sk0; sk0 = sk1; sk1 = t;
        t = sv0; sv0 = sv1; sv1 = t;
        shift += width;
    }
    for (int i = tid; i < n; i += kSmallThreads) {
        kout[i] = sk0[i];
        vout[i] = sv0[i];
    }
}

int radix_sort_pairs(uint32_t* k0, uint32_t* v0, uint32_t* k1, uint32_t* v1, bool implicit_vals,
                     const unsigned long long* n_dev, int64_t cap, int bits, const RadixScratch& rs,
                     cudaStream_t s)
{
    if (cap <= 0 || bits <= 0) return 0;
    const int passes = (bits + 7) / 8;
    const int digit = (bits + passes - 1) / passes;
    if (cap <= kSmallN) {
        // one launch; the result goes where the multi-pass sort would leave it
        static std::atomic<int> attr_set[kMaxDevices];
        per_device_once(attr_set, [] {
            cudaFuncSetAttribute(radix_small_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmallSmem);
            return 1;
        });
        uint32_t* ko = (passes & 1) ? k1 : k0;
        uint32_t* vo = (passes & 1) ? v1 : v0;
        GSR_COUNT_LAUNCH();
        radix_small_kernel<<<1, kSmallThreads, kSmallSmem, s>>>(k0, v0, implicit_vals, ko, vo, n_dev, cap, bits,
                                                                passes, digit);
        return (passes & 1) ? 1 : 0;
    }
    // at least two sub-tiles per block, at most one resident wave of scatter
    // blocks (their shared-memory stages limit residency); the shared-memory
    // opt-in is a per-device setting.  (Eight sub-tiles per block left the
    // depth sorts of 0.5-1.5 M records on 31-90 blocks: 0.18 ms where two
    // take 0.09-0.10.)
    static std::atomic<int> per_sm_dev[kMaxDevices];
    const int per_sm = per_device_once(per_sm_dev, [] {
        int n = 0;
        cudaFuncSetAttribute(radix_scatter_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kScatterStageBytes);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, radix_scatter_kernel, kRT, kScatterStageBytes);
        return n < 1 ? 1 : n;
    });
    int64_t g = (cap + 2 * kSub - 1) / (2 * kSub);
    g = std::max<int64_t>(1, std::min<int64_t>(g, std::min<int64_t>(rs.max_blocks, (int64_t)per_sm * rs.num_sms)));
    const int G = (int)g;
    uint32_t *ki = k0, *vi = v0, *ko = k1, *vo = v1;
    int shift = 0;
    for (int p = 0; p < passes; ++p) {
        const int width = (shift + digit > bits) ? bits - shift : digit;
        const uint32_t mask = (1u << width) - 1u;
        GSR_COUNT_LAUNCH();
        radix_upsweep_kernel<<<G, kRT, 0, s>>>(ki, n_dev, cap, shift, mask, rs.hist, G);
        GSR_COUNT_LAUNCH();
        radix_scan_kernel<<<256, kRT, 0, s>>>(rs.hist, G, rs.dtot);
        GSR_COUNT_LAUNCH();
        radix_scatter_kernel<<<G, kRT, kScatterStageBytes, s>>>(ki, vi, implicit_vals && p == 0, ko, vo, n_dev, cap, shift, mask,
                                               rs.hist, rs.dtot, G, rs.status, rs.wait_ns);
        uint32_t* t;
        t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
        shift += width;
    }
    return (passes & 1) ? 1 : 0;
}

}  // namespace gsr
