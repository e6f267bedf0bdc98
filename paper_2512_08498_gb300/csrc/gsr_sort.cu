// gsr_sort.cu -- ordering of the tile lists.
//
// The lists are the instances (view, tile, depth) sorted by the 64-bit key
// (global tile << 32 | float bits of camera z) with ties broken by record
// index.  Instead of radix-sorting 64-bit keys over M instances, the order is
// produced in two stable LSD radix sorts over 32-bit keys:
//   1. visible records (n_vis << M) sorted by depth bits; the compact order
//      is the record order, so ties stay in record order;
//   2. instances emitted in that depth order, then stably sorted by the
//      global tile id (ceil(log2 n_tiles) bits).
// Stability of the second sort gives exactly the (tile, depth, record)
// order of the 64-bit key sort while moving 8 bytes per instance per pass
// over 16-19 bits instead of 12 bytes over 48-51 bits.
//
// The radix passes are in gsr_radix.cu.  The instance emission uses a
// single-pass decoupled look-back scan over the tile counts and spreads each
// block's instances evenly over its threads.
#include "gsr_common.cuh"
#include "gsr_kernels.h"

namespace gsr {

__device__ __forceinline__ int64_t clamped_count(const unsigned long long* n_dev, int64_t cap)
{
    const unsigned long long n = *n_dev;
    return n < (unsigned long long)cap ? (int64_t)n : cap;
}

// ---------------------------------------------------------------------------
// instance emission
//
// Two launches, so that the work follows the instances and not the records
// (in depth order the nearest records cover the most tiles, and a single
// block expanding a chunk of them was the tail of the old one-kernel form):
//   dup_scan    persistent, chunks of 1024 depth-ordered records in ticket
//               order: tile counts, block scan, decoupled look-back; writes a
//               descriptor per record {record id, first tile id, rect width |
//               tiles per row << 16, first instance} and, for every window of
//               kWin instances, the record holding the window's first instance;
//   dup_expand  windows of kWin rectangle instances in ticket order over a
//               persistent grid: the window's records come from the window
//               index, each thread walks eight consecutive instances (owner
//               by binary search, then along the rectangle) and keeps the
//               tiles that pass the record's tile culling (tile_cull_keep:
//               some pixel centre can reach alpha >= 1/255); the kept ones
//               are compacted by a block scan and a decoupled look-back over
//               the windows, staged in shared memory and written coalesced,
//               so the lists are the culled rectangles in depth order.
// ---------------------------------------------------------------------------
constexpr int kDupThreads = 256;
constexpr int kDupItems = 8;
constexpr int kDupChunk = kDupThreads * kDupItems;
constexpr int kWin = 2048;                        // instances per expansion window
constexpr int kWinPer = kWin / kDupThreads;       // per thread
static_assert(kWinPer == 8, "eight instances per thread");

__device__ __forceinline__ int pad32(int x) { return x + (x >> 5); }

__global__ void __launch_bounds__(kDupThreads)
dup_scan_kernel(const __grid_constant__ Table Tb, DuplicateArgs a)
{
    if (earlier_wait_timed_out(a.status)) return;
    __shared__ long long s_blk;
    __shared__ uint32_t s_warp[kDupThreads / 32];
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t n = clamped_count(a.counters + kCntVisible, a.rec_cap);
    const int64_t nchunks = (n + kDupChunk - 1) / kDupChunk;
    for (;;) {
        if (tid == 0) s_blk = (long long)atomicAdd(a.ticket, 1u);
        __syncthreads();
        const long long blk = s_blk;
        if (blk >= nchunks) break;
        const int64_t i0 = blk * kDupChunk + (int64_t)tid * kDupItems;
        uint4 d[kDupItems];
        uint32_t cnt[kDupItems], sum = 0;
#pragma unroll
        for (int j = 0; j < kDupItems; ++j) {
            const int64_t i = i0 + j;
            cnt[j] = 0;
            d[j] = make_uint4(0, 0, 0, 0);
            if (i < n) {
                const uint32_t k = a.sorted_k[i];
                const uint4 aux = a.vis_aux[k];
                const uint32_t x0 = aux.x & 0xffffu, y0 = aux.x >> 16, x1 = aux.y & 0xffffu, y1 = aux.y >> 16;
                const DevView& V = Tb.v[aux.w];
                cnt[j] = (x1 - x0) * (y1 - y0);
                d[j] = make_uint4(k, (uint32_t)(V.tile_base + (int64_t)y0 * V.TX + x0),
                                  (x1 - x0) | ((uint32_t)V.TX << 16), 0u);
                // the record's tile culling set-up, read by the expansion with the descriptor
                const float4 q0 = a.rec[4 * (size_t)k], q1 = a.rec[4 * (size_t)k + 1];
                const TileCull tc = tile_cull_setup(q0.x, q0.y, q0.z, q0.w, q1.x, q1.y);
                float4* cw = a.cull + 3 * i;
                cw[0] = make_float4(tc.u, tc.v, tc.qa, tc.qb);
                cw[1] = make_float4(tc.qc, tc.sig, tc.m, tc.kx);
                cw[2] = make_float4(tc.ky, __int_as_float(tc.mode), __uint_as_float(aux.x), tc.lo);
            }
            sum += cnt[j];
        }
        // block exclusive scan of the per-thread sums
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const uint32_t c = lane < kDupThreads / 32 ? s_warp[lane] : 0u;
            uint32_t wi = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, wi, o);
                if (lane >= o) wi += t;
            }
            const uint32_t acc = __shfl_sync(0xffffffffu, wi, 31);
            if (lane < kDupThreads / 32) s_warp[lane] = wi - c;
            const unsigned long long base = lookback_exclusive_warp(a.lb_status, blk, acc, a.status, a.wait_ns);
            if (lane == 0) {
                s_base = base;
                if (blk == nchunks - 1) {
                    // instances of the full rectangles (the window space of the expansion)
                    const unsigned long long total = base + acc;
                    a.counters[kCntFullInst] = total;
                    if (total > (unsigned long long)a.full_cap) atomicOr(a.status, kErrFullCapacity);
                    if (total > 0xffffffffull) atomicOr(a.status, kErrOverflow32);
                }
            }
        }
        __syncthreads();
        unsigned long long run = s_base + s_warp[wid] + incl - sum;
#pragma unroll
        for (int j = 0; j < kDupItems; ++j) {
            const int64_t i = i0 + j;
            if (i < n) {
                d[j].w = (uint32_t)run;
                a.desc[i] = d[j];
                // windows whose first instance lies in [run, run + cnt)
                if (cnt[j] > 0) {
                    const unsigned long long m0 = (run + kWin - 1) / kWin, m1 = (run + cnt[j] - 1) / kWin;
                    for (unsigned long long m = m0; m <= m1 && m < (unsigned long long)a.win_cap; ++m)
                        a.win_first[m] = (uint32_t)i;
                }
            }
            run += cnt[j];
        }
        __syncthreads();   // s_blk, s_warp, s_base are rewritten by the next chunk
    }
}

// Window wi of the rectangle instances: [w0, w1) and the records holding them.
struct WinInfo {
    int64_t w0, w1, r_lo, nr;
    bool bad;
};

__device__ __forceinline__ WinInfo window_info(const DuplicateArgs& a, int64_t wi, int64_t n,
                                               unsigned long long total, int64_t m_all)
{
    WinInfo W;
    W.w0 = wi * kWin;
    W.w1 = min(m_all, W.w0 + kWin);
    W.r_lo = a.win_first[wi];
    // the record holding the next window's first instance, if there is one
    const bool next = (unsigned long long)(W.w0 + kWin) < total && wi + 1 < a.win_cap;
    const int64_t r_hi = next ? (int64_t)a.win_first[wi + 1] : n - 1;
    W.nr = r_hi - W.r_lo + 1;
    // every visible record covers >= 1 tile, so a window holds <= kWin + 1 records
    W.bad = W.nr < 1 || W.nr > kWin + 1 || r_hi >= n;
    return W;
}

// This thread's eight consecutive instances of window W (owner by binary
// search over s_off, then along the rectangle).  TEST: returns the mask of
// the instances whose tile passes the record's tile culling.  !TEST: writes
// the tile id and record of the instances set in `mask` to tk / tv.
template <bool TEST>
__device__ __forceinline__ uint32_t walk8(const Table& Tb, const DuplicateArgs& a, const uint32_t* s_off,
                                          const WinInfo& W, uint32_t mask, uint32_t* tk, uint32_t* tv)
{
    const uint32_t e0 = (uint32_t)(W.w0 + threadIdx.x * kWinPer);
    if ((int64_t)e0 >= W.w1) return 0u;
    int lo = 0, hi = (int)W.nr - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (s_off[mid] <= e0) lo = mid; else hi = mid - 1;
    }
    int o = lo;
    uint4 d;
    uint32_t wdt = 1, txr = 0, ty = 0, tx = 0, rx0 = 0, ry0 = 0, row_ty = 0xffffffffu;
    TileCull tc;
    TileRow row;
    // walking consecutively, a new owner is entered at its first instance
    // (every record covers >= 1 tile), so only the first owner needs the
    // division
    auto owner = [&](uint32_t e, bool first) {
        d = a.desc[W.r_lo + o];
        wdt = d.z & 0xffffu; txr = d.z >> 16;
        if (first) {
            const uint32_t local = e - d.w;
            ty = local / wdt; tx = local - ty * wdt;
        } else {
            ty = 0; tx = 0;
        }
        if (TEST) {
            // the record's tile culling set-up, stored by the scan beside the descriptor
            const float4* cw = a.cull + 3 * (W.r_lo + o);
            const float4 c0 = cw[0], c1 = cw[1], c2 = cw[2];
            const uint32_t rect0 = __float_as_uint(c2.z);
            rx0 = rect0 & 0xffffu; ry0 = rect0 >> 16;
            tc.u = c0.x; tc.v = c0.y; tc.qa = c0.z; tc.qb = c0.w;
            tc.qc = c1.x; tc.sig = c1.y; tc.m = c1.z; tc.kx = c1.w;
            tc.ky = c2.x; tc.mode = __float_as_int(c2.y);
            tc.lo = c2.w; tc.hi = c2.w + 2e-3f;
            row_ty = 0xffffffffu;
        }
    };
    owner(e0, true);
    uint32_t keep = 0u;
#pragma unroll
    for (int j = 0; j < kWinPer; ++j) {
        const uint32_t e = e0 + j;
        if ((int64_t)e >= W.w1) break;
        if (e >= s_off[o + 1]) {
            do { ++o; } while (e >= s_off[o + 1]);
            owner(e, false);
        }
        if (TEST) {
            if (ty != row_ty) {
                const int Y0 = (int)(ry0 + ty) * Tb.tile_h;
                row = tile_cull_row(tc, (float)Y0, (float)(Y0 + Tb.tile_h - 1));
                row_ty = ty;
            }
            const int X0 = (int)(rx0 + tx) * Tb.tile_w;
            if (tile_cull_keep_row(tc, row, (float)X0, (float)(X0 + Tb.tile_w - 1))) keep |= 1u << j;
        } else if (mask & (1u << j)) {
            tk[j] = d.y + ty * txr + tx;
            tv[j] = d.x;
        }
        if (++tx == wdt) { tx = 0; ++ty; }
    }
    return keep;
}

__device__ __forceinline__ void window_offsets(const DuplicateArgs& a, const WinInfo& W, uint32_t* s_off)
{
    if (W.bad) return;
    for (int t = threadIdx.x; t < W.nr; t += kDupThreads) s_off[t] = a.desc[W.r_lo + t].w;
    if (threadIdx.x == 0) s_off[W.nr] = 0xffffffffu;
}

// Pass 1: per window, which instances are kept (one mask byte per thread)
// and how many.
__global__ void __launch_bounds__(kDupThreads)
dup_test_kernel(const __grid_constant__ Table Tb, DuplicateArgs a)
{
    if (earlier_wait_timed_out(a.status)) return;
    __shared__ uint32_t s_off[kWin + 2];
    __shared__ uint32_t s_part[kDupThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t n = clamped_count(a.counters + kCntVisible, a.rec_cap);
    const unsigned long long total = a.counters[kCntFullInst];
    const int64_t m_all = clamped_count(a.counters + kCntFullInst, a.full_cap);
    const int64_t nwin = (m_all + kWin - 1) / kWin;
    for (int64_t wi = blockIdx.x; wi < nwin; wi += gridDim.x) {
        const WinInfo W = window_info(a, wi, n, total, m_all);
        if (W.bad && tid == 0) atomicOr(a.status, kErrInternal);
        window_offsets(a, W, s_off);
        __syncthreads();
        const uint32_t mask = W.bad ? 0u : walk8<true>(Tb, a, s_off, W, 0u, nullptr, nullptr);
        a.keep[wi * kDupThreads + tid] = (uint8_t)mask;
        const uint32_t c = warp_sum((uint32_t)__popc(mask));
        if (lane == 0) s_part[wid] = c;
        __syncthreads();
        if (tid == 0) {
            uint32_t t = 0;
#pragma unroll
            for (int w = 0; w < kDupThreads / 32; ++w) t += s_part[w];
            a.win_count[wi] = t;
        }
        __syncthreads();   // s_off, s_part are rewritten by the next window
    }
}

// Pass 2: exclusive scan of the window counts in place (chunks of 1024
// windows in ticket order, decoupled look-back); the last chunk publishes
// the number of kept instances.
constexpr int kWinScan = 1024;

__global__ void __launch_bounds__(kWinScan)
dup_winscan_kernel(DuplicateArgs a)
{
    if (earlier_wait_timed_out(a.status)) return;
    __shared__ long long s_blk;
    __shared__ uint32_t s_warp[kWinScan / 32];
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t m_all = clamped_count(a.counters + kCntFullInst, a.full_cap);
    const int64_t nwin = (m_all + kWin - 1) / kWin;
    const int64_t nchunks = (nwin + kWinScan - 1) / kWinScan;
    for (;;) {
        if (tid == 0) s_blk = (long long)atomicAdd(a.win_ticket, 1u);
        __syncthreads();
        const long long blk = s_blk;
        if (blk >= nchunks) break;
        const int64_t i = blk * kWinScan + tid;
        const uint32_t v = i < nwin ? a.win_count[i] : 0u;
        uint32_t incl = v;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const uint32_t c = s_warp[lane];
            uint32_t ws = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += t;
            }
            const uint32_t acc = __shfl_sync(0xffffffffu, ws, 31);
            s_warp[lane] = ws - c;
            const unsigned long long base = lookback_exclusive_warp(a.lb_win, blk, acc, a.status, a.wait_ns);
            if (lane == 0) {
                s_base = base;
                if (blk == nchunks - 1) {
                    const unsigned long long kept = base + acc;
                    a.counters[kCntInstances] = kept;
                    if (kept > (unsigned long long)a.inst_cap) atomicOr(a.status, kErrInstCapacity);
                }
            }
        }
        __syncthreads();
        if (i < nwin) a.win_count[i] = (uint32_t)(s_base + s_warp[wid] + incl - v);
        __syncthreads();   // s_blk, s_warp, s_base are rewritten by the next chunk
    }
}

// Pass 3: the kept instances of every window at its offset, compacted in
// shared memory and written coalesced (over capacity, the positions below
// inst_cap are still written, so every list position holds a valid pair).
__global__ void __launch_bounds__(kDupThreads)
dup_emit_kernel(const __grid_constant__ Table Tb, DuplicateArgs a)
{
    if (earlier_wait_timed_out(a.status)) return;
    __shared__ uint32_t s_off[kWin + 2];
    __shared__ uint32_t sk[kWin + kWin / 32], sv[kWin + kWin / 32];
    __shared__ uint32_t s_warp[kDupThreads / 32 + 1];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t n = clamped_count(a.counters + kCntVisible, a.rec_cap);
    const unsigned long long total = a.counters[kCntFullInst];
    const int64_t m_all = clamped_count(a.counters + kCntFullInst, a.full_cap);
    const int64_t nwin = (m_all + kWin - 1) / kWin;
    for (int64_t wi = blockIdx.x; wi < nwin; wi += gridDim.x) {
        const WinInfo W = window_info(a, wi, n, total, m_all);
        window_offsets(a, W, s_off);
        const uint32_t mask = W.bad ? 0u : (uint32_t)a.keep[wi * kDupThreads + tid];
        __syncthreads();
        uint32_t tk[kWinPer], tv[kWinPer];
        if (mask) walk8<false>(Tb, a, s_off, W, mask, tk, tv);
        // block exclusive scan of the kept counts: compact positions
        const uint32_t cnt = __popc(mask);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        if (tid == 0) {
            uint32_t acc = 0;
#pragma unroll
            for (int w = 0; w < kDupThreads / 32; ++w) {
                const uint32_t c = s_warp[w];
                s_warp[w] = acc;
                acc += c;
            }
            s_warp[kDupThreads / 32] = acc;
        }
        __syncthreads();
        uint32_t q = s_warp[wid] + incl - cnt;
#pragma unroll
        for (int j = 0; j < kWinPer; ++j) {
            if (mask & (1u << j)) {
                sk[pad32((int)q)] = tk[j];
                sv[pad32((int)q)] = tv[j];
                ++q;
            }
        }
        __syncthreads();
        const unsigned long long base = a.win_count[wi];
        const int kept = (int)s_warp[kDupThreads / 32];
        for (int t = tid; t < kept; t += kDupThreads) {
            const unsigned long long pos = base + (unsigned long long)t;
            if (pos < (unsigned long long)a.inst_cap) {
                a.tile_key[pos] = sk[pad32(t)];
                a.tile_val[pos] = sv[pad32(t)];
            }
        }
        __syncthreads();   // s_off, sk, sv, s_warp are rewritten by the next window
    }
}

int64_t duplicate_blocks(int64_t rec_cap) { return (rec_cap + kDupChunk - 1) / kDupChunk; }
int64_t duplicate_windows(int64_t full_cap) { return (full_cap + kWin - 1) / kWin + 1; }

void launch_duplicate(const Table& T, const DuplicateArgs& a, int num_sms, cudaStream_t s)
{
    int64_t blocks = duplicate_blocks(a.rec_cap);
    if (blocks == 0) return;
    // one resident wave (3 blocks of 256 threads per SM at 80 registers): more
    // blocks in flight only lengthen the look-back walks
    if (blocks > (int64_t)num_sms * 3) blocks = (int64_t)num_sms * 3;
    GSR_COUNT_LAUNCH();
    dup_scan_kernel<<<(unsigned)blocks, kDupThreads, 0, s>>>(T, a);
    int64_t wblocks = duplicate_windows(a.full_cap);
    if (wblocks > (int64_t)num_sms * 8) wblocks = (int64_t)num_sms * 8;
    GSR_COUNT_LAUNCH();
    dup_test_kernel<<<(unsigned)wblocks, kDupThreads, 0, s>>>(T, a);
    int64_t sblocks = (duplicate_windows(a.full_cap) + kWinScan - 1) / kWinScan;
    if (sblocks > (int64_t)num_sms) sblocks = num_sms;
    GSR_COUNT_LAUNCH();
    dup_winscan_kernel<<<(unsigned)sblocks, kWinScan, 0, s>>>(a);
    GSR_COUNT_LAUNCH();
    dup_emit_kernel<<<(unsigned)wblocks, kDupThreads, 0, s>>>(T, a);
}

// Four keys per thread (one 16-byte load, the keys array starts 16-byte
// aligned) plus the neighbour on each side.
__global__ void ranges_kernel(const uint32_t* __restrict__ keys, const unsigned long long* m_dev, int64_t cap,
                              uint2* __restrict__ ranges, int64_t n_tiles, uint32_t* status)
{
    const int64_t m = clamped_count(m_dev, cap);
    const int64_t nq = (m + 3) / 4;
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nq; q += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i0 = 4 * q;
        uint32_t k[6];
        if (i0 + 4 <= m) {
            const uint4 v = reinterpret_cast<const uint4*>(keys)[q];
            k[1] = v.x; k[2] = v.y; k[3] = v.z; k[4] = v.w;
        } else {
#pragma unroll
            for (int u = 0; u < 4; ++u) k[1 + u] = i0 + u < m ? keys[i0 + u] : 0u;
        }
        k[0] = i0 > 0 ? keys[i0 - 1] : 0u;
        k[5] = i0 + 4 < m ? keys[i0 + 4] : 0u;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const int64_t i = i0 + u;
            if (i >= m) break;
            const uint32_t t = k[1 + u];
            const bool first = i == 0 || k[u] != t;
            const bool lastk = i == m - 1 || k[2 + u] != t;
            if (!first && !lastk) continue;
            if ((int64_t)t >= n_tiles) {
                atomicOr(status, kErrInternal);
                continue;
            }
            if (first) ranges[t].x = (uint32_t)i;
            if (lastk) ranges[t].y = (uint32_t)(i + 1);
        }
    }
}

void launch_ranges(const uint32_t* sorted_tile_keys, const unsigned long long* m_dev, int64_t cap, uint2* ranges,
                   int64_t n_tiles, uint32_t* status, int num_sms, cudaStream_t s)
{
    if (cap <= 0) return;
    int64_t blocks = (cap / 4 + 255) / 256 + 1;
    if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
    GSR_COUNT_LAUNCH();
    ranges_kernel<<<(unsigned)blocks, 256, 0, s>>>(sorted_tile_keys, m_dev, cap, ranges, n_tiles, status);
}

// ---------------------------------------------------------------------------
// parity exports
// ---------------------------------------------------------------------------
__global__ void debug_lists_kernel(const __grid_constant__ Table Tb, DebugArgs a)
{
    const int64_t m_all = clamped_count(a.counters + kCntInstances, a.inst_cap);
    const int64_t m = min(m_all, a.first + a.count);
    for (int64_t i = a.first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t k = a.tile_val[i];
        const uint4 aux = a.vis_aux[k];
        const DevView& V = Tb.v[aux.w];
        const uint32_t zb = __float_as_uint(a.rec[4 * (size_t)k + 1].z);
        if (a.keys_out) a.keys_out[i - a.first] = ((uint64_t)a.tile_key[i] << 32) | zb;
        if (a.vals_out) a.vals_out[i - a.first] = (uint32_t)(V.vm_base + aux.z);
    }
}

__global__ void debug_records_kernel(const __grid_constant__ Table Tb, DebugArgs a)
{
    const int64_t nv = clamped_count(a.counters + kCntVisible, a.rec_cap);
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < nv; k += (int64_t)gridDim.x * blockDim.x) {
        const uint4 aux = a.vis_aux[k];
        const DevView& V = Tb.v[aux.w];
        const int64_t r = V.vm_base + aux.z;
        if (a.rec_out) {
            const float4 r0 = a.rec[4 * k], r1 = a.rec[4 * k + 1], r2 = a.rec[4 * k + 2];
            float* o = a.rec_out + 16 * r;
            o[0] = r0.x; o[1] = r0.y; o[2] = r0.z; o[3] = r0.w;
            o[4] = r1.x; o[5] = r1.y; o[6] = r1.z; o[7] = 0.0f;
            o[8] = r2.x; o[9] = r2.y; o[10] = r2.z;
            for (int i = 11; i < 16; ++i) o[i] = 0.0f;
        }
        if (a.rect_out) {
            int32_t* o = a.rect_out + 4 * r;
            o[0] = aux.x & 0xffff; o[1] = aux.x >> 16; o[2] = aux.y & 0xffff; o[3] = aux.y >> 16;
        }
        if (a.flags_out) a.flags_out[r] = 0u;
        if (a.grec_out && a.grad_rec) {
            float* o = a.grec_out + 12 * r;
            const float4 g0 = a.grad_rec[3 * k], g1 = a.grad_rec[3 * k + 1], g2 = a.grad_rec[3 * k + 2];
            o[0] = g0.x; o[1] = g0.y; o[2] = g0.z; o[3] = g0.w;
            o[4] = g1.x; o[5] = g1.y; o[6] = g1.z; o[7] = g1.w;
            o[8] = g2.x; o[9] = g2.y; o[10] = g2.z; o[11] = g2.w;
        }
    }
}

void launch_debug_lists(const Table& T, const DebugArgs& a, cudaStream_t s)
{
    GSR_COUNT_LAUNCH();
    debug_lists_kernel<<<1024, 256, 0, s>>>(T, a);
}

void launch_debug_records(const Table& T, const DebugArgs& a, cudaStream_t s)
{
    GSR_COUNT_LAUNCH();
    debug_records_kernel<<<1024, 256, 0, s>>>(T, a);
}

// ---------------------------------------------------------------------------
// L1 loss helper
// ---------------------------------------------------------------------------
__global__ void l1_loss_grad_kernel(const float* __restrict__ rgb, const float* __restrict__ tgt, int64_t n,
                                    float* __restrict__ dl, float* loss)
{
    const float inv = 1.0f / (float)n;
    float acc = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t t0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool vec = ((reinterpret_cast<uintptr_t>(rgb) | reinterpret_cast<uintptr_t>(tgt) |
                       reinterpret_cast<uintptr_t>(dl)) & 15u) == 0;
    int64_t done = 0;
    if (vec) {
        // 16-byte loads and stores; the scalar loop below takes the tail
        const int64_t n4 = n / 4;
        for (int64_t q = t0; q < n4; q += stride) {
            const float4 a = reinterpret_cast<const float4*>(rgb)[q];
            const float4 b = reinterpret_cast<const float4*>(tgt)[q];
            const float d0 = a.x - b.x, d1 = a.y - b.y, d2 = a.z - b.z, d3 = a.w - b.w;
            acc += fabsf(d0) + fabsf(d1) + fabsf(d2) + fabsf(d3);
            float4 g;
            g.x = d0 > 0.0f ? inv : (d0 < 0.0f ? -inv : 0.0f);
            g.y = d1 > 0.0f ? inv : (d1 < 0.0f ? -inv : 0.0f);
            g.z = d2 > 0.0f ? inv : (d2 < 0.0f ? -inv : 0.0f);
            g.w = d3 > 0.0f ? inv : (d3 < 0.0f ? -inv : 0.0f);
            reinterpret_cast<float4*>(dl)[q] = g;
        }
        done = 4 * n4;
    }
    for (int64_t i = done + t0; i < n; i += stride) {
        const float d = rgb[i] - tgt[i];
        acc += fabsf(d);
        dl[i] = d > 0.0f ? inv : (d < 0.0f ? -inv : 0.0f);
    }
    if (loss) {
        // one atomic per block: per-warp atomics on a single address serialise
        __shared__ float s_part[32];
        acc = warp_sum(acc);
        const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
        if (lane == 0) s_part[w] = acc;
        __syncthreads();
        if (w == 0) {
            float t = lane < (int)(blockDim.x >> 5) ? s_part[lane] : 0.0f;
            t = warp_sum(t);
            if (lane == 0) atomicAdd(loss, t * inv);
        }
    }
}

void launch_l1_loss_grad(const float* rgb, const float* target, int64_t n, float* dl, float* loss, cudaStream_t s)
{
    if (n <= 0) return;
    if (loss) cudaMemsetAsync(loss, 0, sizeof(float), s);
    int64_t blocks = (n + 255) / 256;
    if (blocks > 4096) blocks = 4096;
    GSR_COUNT_LAUNCH();
    l1_loss_grad_kernel<<<(unsigned)blocks, 256, 0, s>>>(rgb, target, n, dl, loss);
}

}  // namespace gsr
