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

// The depth-ordered records an emission covers: a prefix of the visible ones.
__device__ __forceinline__ int64_t emission_records(const DuplicateArgs& a)
{
    return prefix_records(clamped_count(a.counters + kCntVisible, a.rec_cap), a.prefix);
}

// A second-round emission with no open tile has nothing to list.
__device__ __forceinline__ bool emission_idle(const DuplicateArgs& a)
{
    return a.open_tiles != nullptr && a.counters[kCntOpenTiles] == 0ull;
}

// Open tiles among the c consecutive tile ids from t0 (one tile row).
__device__ __forceinline__ int open_count(const uint32_t* __restrict__ m, uint32_t t0, int c)
{
    int n = 0;
    uint32_t t = t0;
    const uint32_t e = t0 + (uint32_t)c;
    while (t < e) {
        const uint32_t b = t & 31u;
        const uint32_t take = min(32u - b, e - t);
        uint32_t bits = m[t >> 5] >> b;
        if (take < 32u) bits &= (1u << take) - 1u;
        n += __popc(bits);
        t += take;
    }
    return n;
}

// The first open tile id >= t (t_end if there is none below t_end).
__device__ __forceinline__ uint32_t open_next(const uint32_t* __restrict__ m, uint32_t t, uint32_t t_end)
{
    while (t < t_end) {
        const uint32_t bits = m[t >> 5] >> (t & 31u);
        if (bits) return min(t_end, t + (uint32_t)(__ffs(bits) - 1));
        t = (t | 31u) + 1u;
    }
    return t_end;
}

// ---------------------------------------------------------------------------
// instance emission
//
// Four launches:
//   dup_count   one thread per depth-ordered record: its kept tiles row by
//               row (row_cull_run: one contiguous run per tile row of the
//               rectangle), written as (kept instances, kept rows);
//   dup_scan    their exclusive scan in place (chunks of 2048 records in
//               ticket order, decoupled look-backs; a chunk does nothing but
//               load, scan and store, so the look-back chain is never held up
//               by a row walk);
//   dup_rows    one thread per record again: a descriptor per kept row
//               {record, first global tile id, count, first instance} and,
//               for every window of kWin kept instances, the row holding its
//               first instance;
//   dup_expand  windows of kWin kept instances over a persistent grid: the
//               window's rows come from the window index, each thread writes
//               eight consecutive instances (owner row by binary search, then
//               consecutive tiles of the row), staged in shared memory and
//               written coalesced at their final positions.
// The instances come out in depth order (records) and row-major order within
// a record; only kept instances are walked.
// ---------------------------------------------------------------------------
constexpr int kDupThreads = 256;
constexpr int kWin = 2048;                        // instances per expansion window
constexpr int kWinPer = kWin / kDupThreads;       // per thread
static_assert(kWinPer == 8, "eight instances per thread");

__device__ __forceinline__ int pad32(int x) { return x + (x >> 5); }

// Exclusive block scan of one 64-bit value per thread; *total gets the sum.
__device__ __forceinline__ unsigned long long block_excl_scan64(unsigned long long v, unsigned long long* s_warp,
                                                                 unsigned long long* total)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    unsigned long long incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    unsigned long long before = 0, sum = 0;
#pragma unroll
    for (int w = 0; w < kDupThreads / 32; ++w) {
        const unsigned long long x = s_warp[w];
        before += w < wid ? x : 0ull;
        sum += x;
    }
    *total = sum;
    return before + incl - v;
}

// The record's rectangle and culling set-up.
struct DupRec {
    RowCull rc;
    int x0, y0, x1, y1;   // rectangle (tiles)
    int ty0, ty1;         // its rows that can meet the ellipse
    uint32_t view;
};

__device__ __forceinline__ DupRec dup_rec(const Table& Tb, const DuplicateArgs& a, uint32_t k)
{
    DupRec r;
    const uint4 aux = a.vis_aux[k];
    r.x0 = (int)(aux.x & 0xffffu); r.y0 = (int)(aux.x >> 16);
    r.x1 = (int)(aux.y & 0xffffu); r.y1 = (int)(aux.y >> 16);
    r.view = (uint32_t)aux_view(aux.w);
    const float4 q0 = a.rec[4 * (size_t)k], q1 = a.rec[4 * (size_t)k + 1];
    r.rc = row_cull_setup(q0.x, q0.y, q0.z, q0.w, q1.x, q1.y);
    row_cull_rows(r.rc, r.y0, r.y1, Tb.tile_h, r.ty0, r.ty1);
    return r;
}

// Kept run of row ty of record d.
__device__ __forceinline__ int dup_run(const Table& Tb, const DupRec& d, int ty, int& first)
{
    const float Y0 = (float)(ty * Tb.tile_h);
    const float y0 = (Y0 + 0.5f) - d.rc.v, y1 = (Y0 + (float)Tb.tile_h - 0.5f) - d.rc.v;
    return row_cull_run(d.rc, y0, y1, d.x0, d.x1, Tb.tile_w, first);
}

// The views' tile bases and widths in shared memory: a warp's records come
// from many views, and indexing the parameter table by view would serialise
// the warp's loads.
struct ViewTiles {
    int64_t base[kMaxViews];
    uint32_t tx[kMaxViews];
};

__device__ __forceinline__ void load_view_tiles(const Table& Tb, ViewTiles& vt)
{
    for (int v = threadIdx.x; v < Tb.n_views; v += kDupThreads) {
        vt.base[v] = Tb.v[v].tile_base;
        vt.tx[v] = (uint32_t)Tb.v[v].TX;
    }
    __syncthreads();
}

__global__ void __launch_bounds__(kDupThreads)
dup_count_kernel(const __grid_constant__ Table Tb, DuplicateArgs a)
{
    if (earlier_wait_timed_out(a.status) || emission_idle(a)) return;
    __shared__ ViewTiles s_vt;
    if (a.open_tiles) load_view_tiles(Tb, s_vt);
    const int64_t n_all = clamped_count(a.counters + kCntVisible, a.rec_cap);
    const int64_t n = emission_records(a);
    // the rectangles of every visible record, counted in the walk when it
    // covers them all, else in a pass of its own over the records' rectangles
    const bool rect_in_walk = n == n_all && !a.open_tiles;
    unsigned long long rect = 0, tot_inst = 0, tot_rows = 0;
    if (a.full_count && !rect_in_walk) {
        for (int64_t k = (int64_t)blockIdx.x * kDupThreads + threadIdx.x; k < n_all;
             k += (int64_t)gridDim.x * kDupThreads) {
            const uint4 aux = a.vis_aux[k];
            rect += (unsigned long long)(((aux.y & 0xffffu) - (aux.x & 0xffffu)) * ((aux.y >> 16) - (aux.x >> 16)));
        }
    }
    for (int64_t i = (int64_t)blockIdx.x * kDupThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDupThreads) {
        const uint32_t k = a.sorted_k[i];
        if (a.depthpos) a.depthpos[k] = (uint32_t)i;
        const DupRec d = dup_rec(Tb, a, k);
        if (rect_in_walk) rect += (unsigned long long)((d.x1 - d.x0) * (d.y1 - d.y0));
        uint32_t inst = 0, rows = 0;
        for (int ty = d.ty0; ty < d.ty1; ++ty) {
            int first;
            int c = dup_run(Tb, d, ty, first);
            if (a.open_tiles && c > 0)
                c = open_count(a.open_tiles, (uint32_t)(s_vt.base[d.view] + (int64_t)ty * s_vt.tx[d.view] + first), c);
            inst += (uint32_t)c;
            rows += c > 0 ? 1u : 0u;
        }
        a.counts[i] = make_uint2(inst, rows);
        tot_inst += inst;
        tot_rows += rows;
    }
    // exact totals (the scan packs both prefixes into one 64-bit word, valid
    // only while they fit)
    rect = warp_sum(rect);
    tot_inst = warp_sum(tot_inst);
    tot_rows = warp_sum(tot_rows);
    if ((threadIdx.x & 31) == 0) {
        if (rect && a.full_count) atomicAdd(a.full_count, rect);
        if (tot_inst) atomicAdd(a.inst_count, tot_inst);
        if (tot_rows) atomicAdd(a.row_total, tot_rows);
    }
}

// Exclusive scan of the records' (kept instances, kept rows) in depth order,
// in place: counts[i] becomes the record's first instance and first row.
// Both are summed in one 64-bit word (rows << 32 | instances), exact while
// the instance total stays below 2^32 and the row total below 2^30 (the
// look-back word holds 62 bits); dup_count's exact totals say when they do
// not, and then the scan and the row pass leave the counts alone and the call
// reports the overflow.  Chunks of kScanChunk records in ticket order, 16
// consecutive records per thread, one decoupled look-back: a chunk does
// nothing but load, scan and store, so the chain moves at memory speed.
constexpr int kScanItems = 16;
constexpr int kScanChunk = kDupThreads * kScanItems;

__device__ __forceinline__ bool emission_overflows(const DuplicateArgs& a)
{
    return *a.inst_count > 0xffffffffull || *a.row_total >= (1ull << 30);
}

__global__ void __launch_bounds__(kDupThreads)
dup_scan_kernel(DuplicateArgs a)
{
    if (earlier_wait_timed_out(a.status) || emission_idle(a)) return;
    __shared__ long long s_blk;
    __shared__ unsigned long long s_warp[kDupThreads / 32];
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x;
    if (blockIdx.x == 0 && tid == 0) {
        const unsigned long long ti = *a.inst_count, tr = *a.row_total;
        if (ti > (unsigned long long)a.inst_cap) atomicOr(a.status, kErrInstCapacity);
        if (tr > (unsigned long long)a.row_cap) atomicOr(a.status, kErrFullCapacity);
        if (emission_overflows(a)) atomicOr(a.status, kErrOverflow32);
    }
    if (emission_overflows(a)) return;
    const int64_t n = emission_records(a);
    const int64_t nchunks = (n + kScanChunk - 1) / kScanChunk;
    for (;;) {
        if (tid == 0) s_blk = (long long)atomicAdd(a.ticket, 1u);
        __syncthreads();
        const long long blk = s_blk;
        if (blk >= nchunks) break;
        const int64_t i0 = blk * kScanChunk + (int64_t)tid * kScanItems;
        uint2 c[kScanItems];
        unsigned long long sum = 0;
        if (i0 + kScanItems <= n) {
            // 16-byte loads: counts starts 16-byte aligned and i0 is even
            const uint4* c4 = reinterpret_cast<const uint4*>(a.counts + i0);
#pragma unroll
            for (int j = 0; j < kScanItems / 2; ++j) {
                const uint4 q = c4[j];
                c[2 * j] = make_uint2(q.x, q.y);
                c[2 * j + 1] = make_uint2(q.z, q.w);
            }
        } else {
#pragma unroll
            for (int j = 0; j < kScanItems; ++j) c[j] = i0 + j < n ? a.counts[i0 + j] : make_uint2(0u, 0u);
        }
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) sum += ((unsigned long long)c[j].y << 32) | c[j].x;
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan64(sum, s_warp, &tot);
        if (tid < 32) {
            const unsigned long long b = lookback_exclusive_warp(a.lb_inst, blk, tot, a.status, a.wait_ns);
            if (tid == 0) s_base = b;
        }
        __syncthreads();
        unsigned long long v = s_base + ex;
#pragma unroll
        for (int j = 0; j < kScanItems; ++j) {
            const unsigned long long cj = ((unsigned long long)c[j].y << 32) | c[j].x;
            c[j] = make_uint2((uint32_t)v, (uint32_t)(v >> 32));
            v += cj;
        }
        if (i0 + kScanItems <= n) {
            uint4* c4 = reinterpret_cast<uint4*>(a.counts + i0);
#pragma unroll
            for (int j = 0; j < kScanItems / 2; ++j) c4[j] = make_uint4(c[2 * j].x, c[2 * j].y, c[2 * j + 1].x, c[2 * j + 1].y);
        } else {
#pragma unroll
            for (int j = 0; j < kScanItems; ++j)
                if (i0 + j < n) a.counts[i0 + j] = c[j];
        }
        __syncthreads();   // s_blk, s_warp and the base are rewritten by the next chunk
    }
}

// One thread per depth-ordered record: its kept rows' descriptors at its row
// base and the window index (bases from dup_scan; instance and row positions
// stay below 2^32 or the call reports an overflow).
__global__ void __launch_bounds__(kDupThreads)
dup_rows_kernel(const __grid_constant__ Table Tb, DuplicateArgs a)
{
    if (earlier_wait_timed_out(a.status) || emission_idle(a)) return;
    __shared__ ViewTiles s_vt;
    load_view_tiles(Tb, s_vt);
    if (emission_overflows(a)) return;
    const int64_t n = emission_records(a);
    const unsigned long long total_rows = *a.row_total;
    if (a.inst_hist && blockIdx.x == 0 && threadIdx.x < kSatBuckets) {
        // kept instances of the records in each depth-share bucket, from the
        // scanned instance offsets at the buckets' first records
        const int b = threadIdx.x;
        const unsigned long long total = *a.inst_count;
        auto offset_at = [&](int e) -> unsigned long long {
            if (e <= 0) return 0ull;
            if (e >= kSatBuckets) return total;
            const float lo = exp2f(-(float)kSatOctaves + (float)kSatOctaves * (float)e / (float)kSatBuckets);
            int64_t i = (int64_t)ceilf(lo * (float)n) - 1;   // first i with (i + 1) / n >= lo
            i = i < 0 ? 0 : i;
            return i < n ? (unsigned long long)a.counts[i].x : total;
        };
        const unsigned long long o0 = offset_at(b), o1 = offset_at(b + 1);
        if (o1 > o0) a.inst_hist[b] = o1 - o0;
    }
    for (int64_t i = (int64_t)blockIdx.x * kDupThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kDupThreads) {
        const uint2 base = a.counts[i];
        const unsigned long long next_row = i + 1 < n ? (unsigned long long)a.counts[i + 1].y : total_rows;
        if (next_row == base.y) continue;   // no kept row
        const uint32_t k = a.sorted_k[i];
        const DupRec d = dup_rec(Tb, a, k);
        const int64_t tbase = s_vt.base[d.view];
        const uint32_t TX = s_vt.tx[d.view];
        unsigned long long ib = base.x, rb = base.y;
        for (int ty = d.ty0; ty < d.ty1; ++ty) {
            int first;
            int cnt = dup_run(Tb, d, ty, first);
            if (cnt == 0) continue;
            const uint32_t t0 = (uint32_t)(tbase + (int64_t)ty * TX + first);
            // a second round's row lists the open tiles of the run only; its
            // descriptor keeps the run's first tile id
            if (a.open_tiles) cnt = open_count(a.open_tiles, t0, cnt);
            if (cnt == 0) continue;
            if (rb < (unsigned long long)a.row_cap) {
                a.rows[rb] = make_uint4(k, t0, (uint32_t)cnt, (uint32_t)ib);
                // windows whose first instance lies in [ib, ib + cnt)
                const unsigned long long m0 = (ib + kWin - 1) / kWin, m1 = (ib + cnt - 1) / kWin;
                for (unsigned long long m = m0; m <= m1 && m < (unsigned long long)a.win_cap; ++m)
                    a.win_first[m] = (uint32_t)rb;
            }
            ib += (unsigned long long)cnt;
            ++rb;
        }
    }
}

// Window wi of the kept instances: [w0, w1) and the rows holding them.
struct WinInfo {
    int64_t w0, w1, r_lo, nr;
    bool ok;
};

__device__ __forceinline__ WinInfo window_info(const DuplicateArgs& a, int64_t wi, int64_t m_all, int64_t R)
{
    WinInfo W;
    W.w0 = wi * kWin;
    W.w1 = min(m_all, W.w0 + kWin);
    W.r_lo = a.win_first[wi];
    const bool next = W.w0 + kWin < m_all && wi + 1 < a.win_cap;
    const int64_t r_hi = next ? (int64_t)a.win_first[wi + 1] : R - 1;
    W.nr = r_hi - W.r_lo + 1;
    // every kept row holds >= 1 instance, so a window's rows, with the row
    // of the next window's first instance, number <= kWin + 1
    W.ok = W.nr >= 1 && W.nr <= kWin + 1 && r_hi < R;
    return W;
}

__global__ void __launch_bounds__(kDupThreads)
dup_expand_kernel(DuplicateArgs a, uint32_t n_tiles)
{
    if (earlier_wait_timed_out(a.status) || emission_idle(a)) return;
    __shared__ uint32_t s_off[kWin + 2];
    __shared__ uint32_t sk[kWin + kWin / 32], sv[kWin + kWin / 32];
    __shared__ int s_capacity;
    const int tid = threadIdx.x;
    if (tid == 0) s_capacity = (*reinterpret_cast<const volatile uint32_t*>(a.status) &
                                (kErrInstCapacity | kErrFullCapacity | kErrOverflow32)) != 0;
    __syncthreads();
    // over capacity the counts still cover every position below inst_cap, but
    // rows past row_cap were not written (nor any, after an overflow): such
    // windows get valid placeholder pairs (tile 0, record 0) and the call
    // reports the error
    const bool over = s_capacity != 0;
    const int64_t m_all = clamped_count(a.inst_count, a.inst_cap);
    const int64_t R = clamped_count(a.row_total, a.row_cap);
    const int64_t nwin = (m_all + kWin - 1) / kWin;
    for (int64_t wi = blockIdx.x; wi < nwin; wi += gridDim.x) {
        const WinInfo W = window_info(a, wi, m_all, R);
        if (!W.ok && !over && tid == 0) atomicOr(a.status, kErrInternal);
        if (W.ok) {
            for (int t = tid; t < W.nr; t += kDupThreads) s_off[t] = a.rows[W.r_lo + t].w;
            if (tid == 0) s_off[W.nr] = 0xffffffffu;
        }
        __syncthreads();
        const int64_t e0 = W.w0 + (int64_t)tid * kWinPer;
        if (W.ok && e0 < W.w1) {
            int lo = 0, hi = (int)W.nr - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_off[mid] <= (uint32_t)e0) lo = mid; else hi = mid - 1;
            }
            int o = lo;
            uint4 d = a.rows[W.r_lo + o];
            if (a.open_tiles) {
                // a second round's row: its instances are the open tiles of
                // the run from d.y, in order; the (e0 - d.w)-th of them first
                uint32_t t = open_next(a.open_tiles, d.y, n_tiles);
                for (uint32_t r = (uint32_t)e0 - d.w; r > 0u && t < n_tiles; --r)
                    t = open_next(a.open_tiles, t + 1u, n_tiles);
                for (int j = 0; j < kWinPer; ++j) {
                    const int64_t e = e0 + j;
                    if (e >= W.w1) break;
                    if ((uint32_t)e >= s_off[o + 1]) {
                        do { ++o; } while ((uint32_t)e >= s_off[o + 1]);
                        d = a.rows[W.r_lo + o];
                        t = open_next(a.open_tiles, d.y, n_tiles);
                    } else if (j > 0) {
                        t = open_next(a.open_tiles, t + 1u, n_tiles);
                    }
                    if (t >= n_tiles) {
                        atomicOr(a.status, kErrInternal);
                        t = 0u;
                    }
                    const int q = pad32((int)(e - W.w0));
                    sk[q] = t;
                    sv[q] = d.x;
                }
            } else {
#pragma unroll
                for (int j = 0; j < kWinPer; ++j) {
                    const int64_t e = e0 + j;
                    if (e >= W.w1) break;
                    if ((uint32_t)e >= s_off[o + 1]) {
                        do { ++o; } while ((uint32_t)e >= s_off[o + 1]);
                        d = a.rows[W.r_lo + o];
                    }
                    const int q = pad32((int)(e - W.w0));
                    sk[q] = d.y + ((uint32_t)e - d.w);
                    sv[q] = d.x;
                }
            }
        } else if (e0 < W.w1) {
            for (int j = 0; j < kWinPer && e0 + j < W.w1; ++j) {
                const int q = pad32((int)(e0 + j - W.w0));
                sk[q] = 0u;
                sv[q] = 0u;
            }
        }
        __syncthreads();
        for (int t = tid; t < (int)(W.w1 - W.w0); t += kDupThreads) {
            a.tile_key[W.w0 + t] = sk[pad32(t)];
            a.tile_val[W.w0 + t] = sv[pad32(t)];
        }
        __syncthreads();   // s_off, sk, sv are rewritten by the next window
    }
}

int64_t duplicate_blocks(int64_t rec_cap) { return (rec_cap + kScanChunk - 1) / kScanChunk; }
int64_t duplicate_windows(int64_t inst_cap) { return (inst_cap + kWin - 1) / kWin + 1; }

void launch_duplicate(const Table& T, const DuplicateArgs& a, int num_sms, cudaStream_t s)
{
    if (duplicate_blocks(a.rec_cap) == 0) return;
    int64_t cblocks = (a.rec_cap + kDupThreads - 1) / kDupThreads;
    if (cblocks > (int64_t)num_sms * 8) cblocks = (int64_t)num_sms * 8;
    GSR_COUNT_LAUNCH();
    dup_count_kernel<<<(unsigned)cblocks, kDupThreads, 0, s>>>(T, a);
    int64_t sblocks = (a.rec_cap + kScanChunk - 1) / kScanChunk;
    // one resident wave: more blocks in flight only lengthen the look-back walks
    if (sblocks > (int64_t)num_sms * 2) sblocks = (int64_t)num_sms * 2;
    GSR_COUNT_LAUNCH();
    dup_scan_kernel<<<(unsigned)sblocks, kDupThreads, 0, s>>>(a);
    GSR_COUNT_LAUNCH();
    dup_rows_kernel<<<(unsigned)cblocks, kDupThreads, 0, s>>>(T, a);
    int64_t wblocks = duplicate_windows(a.inst_cap);
    if (wblocks > (int64_t)num_sms * 8) wblocks = (int64_t)num_sms * 8;
    GSR_COUNT_LAUNCH();
    dup_expand_kernel<<<(unsigned)wblocks, kDupThreads, 0, s>>>(a, (uint32_t)T.n_tiles);
}

// Four keys per thread (one 16-byte load, the keys array starts 16-byte
// aligned) plus the neighbour on each side.
__global__ void ranges_kernel(const uint32_t* __restrict__ keys, const unsigned long long* m_dev, int64_t cap,
                              uint2* __restrict__ ranges, int64_t n_tiles, int64_t offset, uint32_t* status)
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
            if (first) ranges[t].x = (uint32_t)(offset + i);
            if (lastk) ranges[t].y = (uint32_t)(offset + i + 1);
        }
    }
}

void launch_ranges(const uint32_t* sorted_tile_keys, const unsigned long long* m_dev, int64_t cap, uint2* ranges,
                   int64_t n_tiles, int64_t offset, uint32_t* status, int num_sms, cudaStream_t s)
{
    if (cap <= 0) return;
    int64_t blocks = (cap / 4 + 255) / 256 + 1;
    if (blocks > (int64_t)num_sms * 8) blocks = (int64_t)num_sms * 8;
    GSR_COUNT_LAUNCH();
    ranges_kernel<<<(unsigned)blocks, 256, 0, s>>>(sorted_tile_keys, m_dev, cap, ranges, n_tiles, offset, status);
}

// ---------------------------------------------------------------------------
// parity exports
// ---------------------------------------------------------------------------
__global__ void debug_lists_kernel(const __grid_constant__ Table Tb, DebugArgs a)
{
    const int64_t m1 = clamped_count(a.counters + kCntInstances, a.inst_cap);
    const int64_t m2 = a.region2 >= 0 ? clamped_count(a.counters + kCntInstances2, a.inst_cap) : 0;
    const int64_t span = a.region2 >= 0 ? a.region2 + m2 : m1;
    const int64_t m = min(span, a.first + a.count);
    for (int64_t i = a.first + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m;
         i += (int64_t)gridDim.x * blockDim.x) {
        if (i >= m1 && (a.region2 < 0 || i < a.region2)) {
            // between the first region's filled part and the second region
            if (a.keys_out) a.keys_out[i - a.first] = 0ull;
            if (a.vals_out) a.vals_out[i - a.first] = 0xffffffffu;
            continue;
        }
        const uint32_t k = a.tile_val[i];
        const uint4 aux = a.vis_aux[k];
        const DevView& V = Tb.v[aux_view(aux.w)];
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
        const DevView& V = Tb.v[aux_view(aux.w)];
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
