// gsr_blend.cu -- per-pixel compositing (forward) and its adjoint (backward).
//
// One persistent launch covers every (view, tile) of the batch: each CTA
// takes the next global tile from an atomic counter, so views of uneven size
// and tiles of uneven list length share one grid of (SMs x resident CTAs).
// A CTA has one thread per pixel (256 = tile_w x tile_h, warps laid out as
// 8x4 pixel blocks).  The tile's sorted list is walked in batches of BATCH
// records; each batch is gathered into shared memory with one bulk async copy
// (cp.async.bulk, the TMA engine) per record (64 bytes; the backward stages
// only the 48 it reads), completing on an mbarrier, double-buffered so the
// gather of batch b+1 overlaps the arithmetic of batch b.
//
// Warp culling: every record carries a conservative box outside which its
// binary32 alpha is certainly below 1/255 (see alpha_box in
// gsr_preprocess.cu).  After a batch lands, each record's box is tested
// against the eight warps' 8x4 pixel blocks, and each warp walks only the
// entries that can touch its pixels, in list order.  Skipped pairs would
// have been skipped by the 1/255 rule anyway, so every decision (blend, skip,
// stop, contributor count) is unchanged.
//
// Forward, front to back (binary32 decisions per the contract):
//   P2 = dx (qa dx + qb dy) + qc dy^2           (= log2 of the Gaussian)
//   skip if P2 > 0; alpha = min(0.99, sigma 2^P2); skip if alpha < 1/255;
//   T' = T (1 - alpha); stop (entry not blended) if T' < 1e-4;
//   C += c alpha T, D += z alpha T, T = T'.
// Backward, back to front from the saved T_final and contributor count:
//   T_k = T_{k+1} / (1 - alpha_k) and suffix sums S of the later terms give
//   dL/dalpha_k = sum_ch dC (c T_k - S_C / (1 - alpha_k))
//               + dD (z T_k - S_D / (1 - alpha_k)) + dA T_final / (1 - alpha_k),
//   evaluated as T_k (dC . c + dD z) - X / (1 - alpha_k) with the single
//   running scalar X = dC . S_C + dD S_D - dA T_final;
//   then the chain to (u, v, qa, qb, qc, sigma, colour, z), reduced over the
//   warp through per-warp slot buffers (one entry per lane pair, see
//   slots_reduce), over the CTA in shared memory, and added to the
//   per-record gradient with one vector atomic per 16 bytes.
#include <type_traits>

#include "gsr_common.cuh"
#include "gsr_kernels.h"

namespace gsr {

constexpr int kBlendThreads = 256;
constexpr int kWarps = kBlendThreads / 32;

template <int BX, int BY>
struct TileShape {
    static_assert(BX * BY == kBlendThreads, "tile must hold 256 pixels");
    static constexpr int WX = 8, WY = 4;          // warp footprint
    static constexpr int WPR = BX / WX;           // warps per tile row
    __device__ static int lx(int tid) { return ((tid >> 5) % WPR) * WX + (tid & 7); }
    __device__ static int ly(int tid) { return ((tid >> 5) / WPR) * WY + ((tid & 31) >> 3); }
};

// Gather `cnt` records (list positions [first, first + cnt)) into dst.
template <int NQ>
__device__ __forceinline__ void issue_batch(const uint32_t* vals, const float4* rec, uint32_t first, int cnt,
                                            float4* dst, uint64_t* bar, uint32_t* idx_out)
{
    const int tid = threadIdx.x;
    if (tid == 0) mbar_arrive_expect_tx(bar, (uint32_t)cnt * NQ * 16u);
    for (int t = tid; t < cnt; t += kBlendThreads) {
        const uint32_t k = vals[first + t];
        if (idx_out) idx_out[t] = k;
        bulk_g2s(dst + NQ * t, rec + 4 * (size_t)k, NQ * 16, bar);
    }
}

// Largest value of the quadratic form P(x, y) = x (qa x + qb y) + qc y^2
// (negative definite) over the rectangle [x0, x1] x [y0, y1] of pixel
// offsets, up to rounding.  The unconstrained maximum is at the origin; when
// the origin lies outside, the maximum lies on a face that faces it, and
// along a face P is a parabola with its vertex at y = ky x (x = kx y), so two
// clamped candidates cover every case: each is a point of the rectangle, and
// together they include the maximiser.
__device__ __forceinline__ float rect_max_form(float x0, float x1, float y0, float y1, float qa, float qb, float qc,
                                               float kx, float ky)
{
    const float xe = fminf(fmaxf(0.0f, x0), x1);
    const float y1c = fminf(fmaxf(ky * xe, y0), y1);
    const float ye = fminf(fmaxf(0.0f, y0), y1);
    const float x2c = fminf(fmaxf(kx * ye, x0), x1);
    const float p1 = __fmaf_rn(xe, __fmaf_rn(qa, xe, __fmul_rn(qb, y1c)), __fmul_rn(__fmul_rn(qc, y1c), y1c));
    const float p2 = __fmaf_rn(x2c, __fmaf_rn(qa, x2c, __fmul_rn(qb, ye)), __fmul_rn(__fmul_rn(qc, ye), ye));
    return fmaxf(p1, p2);
}

// Bit w of mask[t]: record t can reach alpha >= 1/255 at a pixel centre of
// warp w.  Two conservative tests: the record's alpha box against the warp's
// block, then the maximum of the record's exponent over the block against
// its culling threshold (record slot 11).  The corner offsets are rounded
// exactly as the blend rounds each pixel's offset, so every pixel's rounded
// offset lies in the tested rectangle.
template <int BX, int BY>
__device__ __forceinline__ void warp_masks(const float4* B, int cnt, int tx0, int ty0, uint8_t* s_mask)
{
    using TS = TileShape<BX, BY>;
    for (int t = threadIdx.x; t < cnt; t += kBlendThreads) {
        const float4 r0 = B[4 * t];
        const float qc = B[4 * t + 1].x;
        const float thr_cull = B[4 * t + 2].w;
        const float4 bb = B[4 * t + 3];
        const float kx = -r0.w / (2.0f * r0.z), ky = -r0.w / (2.0f * qc);
        uint32_t m = 0;
#pragma unroll 1
        for (int w = 0; w < kWarps; ++w) {
            const float X0 = (float)(tx0 + (w % TS::WPR) * TS::WX);
            const float Y0 = (float)(ty0 + (w / TS::WPR) * TS::WY);
            bool hit = bb.x <= X0 + (TS::WX - 0.5f) && bb.y >= X0 + 0.5f && bb.z <= Y0 + (TS::WY - 0.5f) &&
                       bb.w >= Y0 + 0.5f;
            if (hit && thr_cull > -3.0e38f) {
                const float x0 = __fsub_rn(__fadd_rn(X0, 0.5f), r0.x);
                const float x1 = __fsub_rn(__fadd_rn(X0, TS::WX - 0.5f), r0.x);
                const float y0 = __fsub_rn(__fadd_rn(Y0, 0.5f), r0.y);
                const float y1 = __fsub_rn(__fadd_rn(Y0, TS::WY - 0.5f), r0.y);
                hit = rect_max_form(x0, x1, y0, y1, r0.z, r0.w, qc, kx, ky) >= thr_cull;
            }
            m |= (uint32_t)hit << w;
        }
        s_mask[t] = (uint8_t)m;
    }
}

// This warp's entries of the batch, in list order; returns their number.
__device__ __forceinline__ int warp_list(const uint8_t* s_mask, int cnt, int w, int lane, uint16_t* list)
{
    int nl = 0;
    const uint32_t lt = (1u << lane) - 1u;
    for (int base = 0; base < cnt; base += 32) {
        const int t = base + lane;
        const bool bit = t < cnt && ((s_mask[t] >> w) & 1u);
        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
        if (bit) list[nl + __popc(bal & lt)] = (uint16_t)t;
        nl += __popc(bal);
    }
    __syncwarp();
    return nl;
}

// One (pixel, entry) pair of the forward up to alpha (independent of T).
struct FwdPair {
    int k;
    float P2, al;
    float4 c;      // colour, depth
};

__device__ __forceinline__ FwdPair fwd_pair(const float4* B, int k, float pxf, float pyf)
{
    FwdPair e;
    e.k = k;
    const float4 r0 = B[4 * k];
    const float4 r1 = B[4 * k + 1];
    const float4 r2 = B[4 * k + 2];
    const float dx = __fsub_rn(pxf, r0.x), dy = __fsub_rn(pyf, r0.y);
    e.P2 = __fmaf_rn(dx, __fmaf_rn(r0.z, dx, __fmul_rn(r0.w, dy)), __fmul_rn(__fmul_rn(r1.x, dy), dy));
    e.al = fminf(GSR_ALPHA_MAX, __fmul_rn(r1.y, exp2_nonpos(fminf(e.P2, 0.0f))));
    e.c = make_float4(r2.x, r2.y, r2.z, r1.z);
    return e;
}

// Backward reduction over a warp's 32 pixels, transposed.  For each walked
// entry every lane stores two scalars in its warp's slot buffer -- gP =
// dL/dP2 and w = alpha T (both zero where the pixel does not composite the
// entry) -- and every kSlots entries the warp reduces the buffer with one
// entry per lane pair, so a lane sums over pixels serially instead of the
// warp summing ten values per entry with shuffles.  The record gradient needs
//   sum gP dx, sum gP dy, sum gP dx^2, sum gP dx dy, sum gP dy^2,
//   sum gP / sigma (= sum dL/dalpha G where alpha is not clamped),
//   sum w dD, sum w dC (three channels),
// with dx = px - u the same for every pixel up to the pixel's offset inside
// the 8x4 block: dx = xo - ux, xo = x - 3.5 (x = lane & 7), ux = u minus the
// block centre (same for y with yo = (lane >> 3) - 1.5).  So the warp keeps
// the six moments M = sum gP {1, xo, yo, xo^2, xo yo, yo^2} (constant
// weights) and shifts them once per entry:
//   sum gP dx = Mx - ux M0, sum gP dx^2 = Mxx - 2 ux Mx + ux^2 M0,
//   sum gP dx dy = Mxy - ux My - uy Mx + ux uy M0 (and y alike).
// The shifted form has the rounding error of the direct sums (bounded by
// the sums of |gP| dx^2 both ways).  Per-pixel dC, dD come from s_dcd.
constexpr int kSlots = 16;
// Shared record sums: 10 floats per record at an odd stride, so lanes
// adding to (or flushing) different records hit different banks.
constexpr int kSumStride = 11;
constexpr int kSlotStride = 32;   // floats per slot row: 32 pixels
// 16-byte chunk c of slot row r is stored at chunk c ^ (r & 7): a row's
// stores stay a permutation of its 32 banks, and the 16-byte reads of the
// same chunk from eight different rows land in eight different bank groups.
__device__ __forceinline__ int slot_chunk(int c, int r) { return c ^ (r & 7); }
// The float of slot row r that holds pixel (lane) l: chunk l / 4, element l % 4.
__device__ __forceinline__ int slot_col(int l, int r) { return l ^ ((r & 7) << 2); }

// Slot j holds the entry at position i0 - j of the warp's walk list L.
template <typename LT>
__device__ __forceinline__ void slots_reduce(const float* __restrict__ sgp, const float* __restrict__ swg,
                                             const float4* __restrict__ sdcd, int n, int lane, const LT* L,
                                             int i0, const float4* B, float cxw, float cyw, float* s_grad)
{
    const int e = lane & (kSlots - 1), h = lane >> 4;     // entry slot, pixel half (block rows 2h, 2h + 1)
    const float* gp = sgp + e * kSlotStride;
    const float* wg = swg + e * kSlotStride;
    float g[16];
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 t = *reinterpret_cast<const float4*>(gp + 4 * slot_chunk(4 * h + c, e));
        g[4 * c] = t.x; g[4 * c + 1] = t.y; g[4 * c + 2] = t.z; g[4 * c + 3] = t.w;
    }
    float r0 = 0.0f, r1 = 0.0f, mxx = 0.0f, mx0 = 0.0f, mx1 = 0.0f;
#pragma unroll
    for (int x = 0; x < 8; ++x) {
        const float xo = (float)x - 3.5f;
        r0 += g[x];
        r1 += g[8 + x];
        mxx = fmaf(xo * xo, g[x] + g[8 + x], mxx);
        mx0 = fmaf(xo, g[x], mx0);
        mx1 = fmaf(xo, g[8 + x], mx1);
    }
    const float y0 = 2.0f * (float)h - 1.5f, y1 = y0 + 1.0f;
    float v[10];
    v[0] = r0 + r1;
    v[1] = mx0 + mx1;
    v[2] = fmaf(y0, r0, y1 * r1);
    v[3] = mxx;
    v[4] = fmaf(y0, mx0, y1 * mx1);
    v[5] = fmaf(y0 * y0, r0, (y1 * y1) * r1);
    float sd = 0.0f, s0 = 0.0f, s1 = 0.0f, s2 = 0.0f;
    const float4* dcd = sdcd + 16 * h;
#pragma unroll
    for (int c = 0; c < 4; ++c) {
        const float4 t = *reinterpret_cast<const float4*>(wg + 4 * slot_chunk(4 * h + c, e));
        const float w4[4] = {t.x, t.y, t.z, t.w};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const float4 d = dcd[4 * c + j];
            s0 = fmaf(w4[j], d.x, s0);
            s1 = fmaf(w4[j], d.y, s1);
            s2 = fmaf(w4[j], d.z, s2);
            sd = fmaf(w4[j], d.w, sd);
        }
    }
    v[6] = sd; v[7] = s0; v[8] = s1; v[9] = s2;
#pragma unroll
    for (int j = 0; j < 10; ++j) v[j] += __shfl_xor_sync(0xffffffffu, v[j], 16);
    if (e >= n) return;
    const uint32_t k = L[i0 - e];
    // layout of a record's sums: du dv dqa dqb dqc dsig dz dr dg db
    float* sg = s_grad + k * kSumStride;
    if (h == 0) {
        const float4 r = B[3 * k];
        const float ux = r.x - cxw, uy = r.y - cyw;
        const float m0 = v[0];
        atomicAdd(sg + 0, fmaf(-ux, m0, v[1]));
        atomicAdd(sg + 1, fmaf(-uy, m0, v[2]));
        atomicAdd(sg + 2, fmaf(ux * ux, m0, fmaf(-2.0f * ux, v[1], v[3])));
        atomicAdd(sg + 3, fmaf(ux * uy, m0, fmaf(-ux, v[2], fmaf(-uy, v[1], v[4]))));
        atomicAdd(sg + 4, fmaf(uy * uy, m0, fmaf(-2.0f * uy, v[2], v[5])));
    } else {
        atomicAdd(sg + 5, v[0]);
        atomicAdd(sg + 6, v[6]);
        atomicAdd(sg + 7, v[7]);
        atomicAdd(sg + 8, v[8]);
        atomicAdd(sg + 9, v[9]);
    }
}

// four blocks per SM: 64 registers (the two-entry walk would otherwise take
// 72 and leave room for three).  COUNT: keep the per-pixel examined and
// composited counts (statistics only; a separate instantiation because the
// two running counts cost about 6 % of the walk).
template <int BX, int BY, int BATCH, bool COUNT>
__global__ void __launch_bounds__(kBlendThreads, 4)
blend_fwd_kernel(const __grid_constant__ Table Tb, BlendFwdArgs a)
{
    if (earlier_wait_timed_out(a.status)) return;
    using TS = TileShape<BX, BY>;
    extern __shared__ __align__(128) float4 s_buf[];     // [2][BATCH][4]
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ unsigned int s_item;
    __shared__ uint8_t s_mask[BATCH];
    __shared__ uint16_t s_list[kWarps][BATCH];
    __shared__ __align__(16) uint8_t s_wb[kWarps][BATCH]; // per warp: composited each entry of the batch
    // per tile (kept in shared memory, off the walk's registers): the warps'
    // walked entries, and the list entries up to the end of the batch in
    // which every pixel had stopped (0: they did not)
    __shared__ unsigned int s_witer[kWarps];
    __shared__ int s_satpos;
    __shared__ int s_prefix_all;   // the first round's lists are the full ones
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        const int64_t n_vis = (int64_t)a.counters[kCntVisible];
        s_prefix_all = prefix_records(n_vis, a.prefix) == n_vis;
    }
    for (int t = tid; t < kWarps * BATCH / 4; t += kBlendThreads) reinterpret_cast<uint32_t*>(&s_wb[0][0])[t] = 0u;
    __syncthreads();
    uint32_t par0 = 0u, par1 = 0u;
    const int lx = TS::lx(tid), ly = TS::ly(tid);
    unsigned long long exam_total = 0, blended_total = 0;
    unsigned int witer = 0;
    bool failed = false;
    uint16_t* L = s_list[w];
    if (a.round == 2 && a.counters[kCntOpenTiles] == 0ull) return;

    for (;;) {
        if (tid == 0) s_item = atomicAdd(a.work, 1u);
        __syncthreads();
        const unsigned int item = s_item;
        __syncthreads();
        if ((int64_t)item >= Tb.n_tiles || failed) break;
        if (a.round == 2 && !((a.open_tiles[item >> 5] >> (item & 31u)) & 1u)) continue;
        if (lane == 0) s_witer[w] = 0u;
        if (tid == 0) s_satpos = 0;
        const int view = find_view_of_tile(Tb, item);
        const DevView& V = Tb.v[view];
        const int lt = (int)(item - V.tile_base);
        const int tx0 = (lt % V.TX) * BX, ty0 = (lt / V.TX) * BY;
        const int px = tx0 + lx, py = ty0 + ly;
        const bool inside = px < V.W && py < V.H;
        const uint2 rg = a.ranges[item];
        const int n = (int)(rg.y - rg.x);
        const int nb = (n + BATCH - 1) / BATCH;
        const float pxf = __fadd_rn((float)px, 0.5f), pyf = __fadd_rn((float)py, 0.5f);
        float T = 1.0f, C0 = 0.0f, C1 = 0.0f, C2 = 0.0f, D = 0.0f;
        uint32_t last = 0, exam = (uint32_t)n, nblend = 0;
        bool done = !inside;

        if (nb > 0) issue_batch<4>(a.vals, a.rec, rg.x, min(BATCH, n), s_buf, &s_bar[0], nullptr);
        for (int b = 0; b < nb; ++b) {
            const int s = b & 1;
            if (b + 1 < nb)
                issue_batch<4>(a.vals, a.rec, rg.x + (b + 1) * BATCH, min(BATCH, n - (b + 1) * BATCH),
                            s_buf + (size_t)(s ^ 1) * BATCH * 4, &s_bar[s ^ 1], nullptr);
            const bool ok = mbar_wait_bounded(&s_bar[s], s ? par1 : par0, a.status, a.wait_ns);
            if (s) par1 ^= 1u; else par0 ^= 1u;
            if (__syncthreads_or(!ok)) {
                failed = true;
                if (b + 1 < nb) mbar_wait_bounded(&s_bar[s ^ 1], s ? par0 : par1, a.status, a.wait_ns);
                break;
            }
            const int cnt = min(BATCH, n - b * BATCH);
            const float4* B = s_buf + (size_t)s * BATCH * 4;
            warp_masks<BX, BY>(B, cnt, tx0, ty0, s_mask);
            __syncthreads();
            const int nl = warp_list(s_mask, cnt, w, lane, L);
            // Structured body and a warp vote per entry: the vote reconverges
            // the warp every iteration (lanes would otherwise drift apart under
            // independent thread scheduling) and ends the batch for the warp
            // once all of its pixels are done.
            if (!__all_sync(0xffffffffu, done)) {
                // Branch-free: after exact culling nearly every walked entry
                // composites somewhere in the warp, so every lane evaluates it
                // and the decisions select the updates (a zero weight leaves C
                // and D bit-identical).  Entries are taken two at a time: the
                // second's alpha does not depend on T, so it overlaps the
                // first's update; the warp vote that ends the walk once every
                // pixel has stopped is taken after every second pair (a done
                // pixel passes nothing, so the extra entries change no result).
                // Returns whether this pixel composited the entry.
                auto step = [&](const FwdPair& e) {
                    const float Tn = __fmul_rn(T, __fsub_rn(1.0f, e.al));
                    const bool pass = !done && e.P2 <= 0.0f && e.al >= GSR_ALPHA_MIN;
                    const bool stop = pass && Tn < GSR_T_STOP;
                    const bool blended_now = pass && !stop;
                    const float wgt = blended_now ? e.al * T : 0.0f;
                    C0 = fmaf(e.c.x, wgt, C0);
                    C1 = fmaf(e.c.y, wgt, C1);
                    C2 = fmaf(e.c.z, wgt, C2);
                    D = fmaf(e.c.w, wgt, D);
                    T = blended_now ? Tn : T;
                    if constexpr (COUNT) {
                        exam = stop ? (uint32_t)(b * BATCH + e.k + 1) : exam;
                        nblend += blended_now ? 1u : 0u;
                    }
                    done = done || stop;
                    return blended_now;
                };
                // Bit p of a lane's wb is its own decision for the p-th entry of
                // a group of 32.  Per group: the pixel's last composited entry
                // is the highest set bit, and one OR over the warp publishes
                // which entries some pixel of the warp composited (entry
                // L[i0 + l] by lane l).
                auto publish = [&](uint32_t wb, int i0, int cnt) {
                    if (wb) last = (uint32_t)(b * BATCH + L[i0 + 31 - __clz(wb)] + 1);
                    const uint32_t any = __reduce_or_sync(0xffffffffu, wb);
                    if (lane < cnt && ((any >> lane) & 1u)) s_wb[w][L[i0 + lane]] = 1;
                };
                int i = 0;
                bool all = false;
                // whole groups of 32 entries, bit positions fixed at compile time
                for (; i + 32 <= nl; i += 32) {
                    uint32_t wb = 0;
                    int p = 0;
#pragma unroll
                    for (; p < 32; p += 2) {
                        const FwdPair e0 = fwd_pair(B, L[i + p], pxf, pyf);
                        const FwdPair e1 = fwd_pair(B, L[i + p + 1], pxf, pyf);
                        if (step(e0)) wb |= 1u << p;
                        if (step(e1)) wb |= 2u << p;
                        if ((p & 2) && __all_sync(0xffffffffu, done)) { p += 2; all = true; break; }
                    }
                    publish(wb, i, p);
                    if (all) { i += p; break; }
                }
                if (!all) {
                    // the last (fewer than 32) entries
                    uint32_t wb = 0;
                    int p = 0;
                    for (; i + p + 1 < nl; p += 2) {
                        const FwdPair e0 = fwd_pair(B, L[i + p], pxf, pyf);
                        const FwdPair e1 = fwd_pair(B, L[i + p + 1], pxf, pyf);
                        if (step(e0)) wb |= 1u << p;
                        if (step(e1)) wb |= 2u << p;
                        if (__all_sync(0xffffffffu, done)) { p += 2; all = true; break; }
                    }
                    if (!all && i + p < nl) {
                        if (step(fwd_pair(B, L[i + p], pxf, pyf))) wb |= 1u << p;
                        ++p;
                    }
                    publish(wb, i, p);
                    i += p;
                }
                if (lane == 0) s_witer[w] += (unsigned)i;
            }
            const bool all_done = __syncthreads_and(done);
            // publish which warps composited each entry (the backward walks only those)
            for (int t = tid; t < cnt; t += kBlendThreads) {
                uint32_t m = 0;
#pragma unroll
                for (int ww = 0; ww < kWarps; ++ww) {
                    m |= (uint32_t)s_wb[ww][t] << ww;
                    s_wb[ww][t] = 0;
                }
                if (a.wmask) a.wmask[rg.x + (size_t)b * BATCH + t] = (uint8_t)m;
            }
            if (all_done) {
                if (tid == 0) s_satpos = b * BATCH + cnt;
                // drain the prefetched batch before leaving the tile
                if (b + 1 < nb) {
                    const bool ok2 = mbar_wait_bounded(&s_bar[s ^ 1], s ? par0 : par1, a.status, a.wait_ns);
                    if (s) par0 ^= 1u; else par1 ^= 1u;
                    if (__syncthreads_or(!ok2)) failed = true;
                }
                break;
            }
        }
        // A first round's tile is final when its pixels all stopped within
        // the prefix lists (or those were the full lists); otherwise the
        // second round renders it again over its full list.
        const bool saturated = __syncthreads_and(done);   // (also publishes s_witer and s_satpos)
        const bool final_tile = a.round != 1 || saturated || s_prefix_all;
        // (thread 0 re-reads the tile and its range: nothing of them stays
        // live in registers across the walk)
        if (!final_tile) {
            if (tid == 0 && !failed) {
                const unsigned int it = s_item;
                atomicOr(a.open_tiles + (it >> 5), 1u << (it & 31u));
                atomicAdd(a.counters + kCntOpenTiles, 1ull);
            }
            continue;
        }
        if (lane == 0) witer += s_witer[w];
        if (tid == 0 && a.hist && !failed) {
            // the share of the depth-ordered records the tile needed before
            // every pixel stopped, weighted by its (estimated full) list length
            const uint2 r = a.ranges[s_item];
            const unsigned long long n_vis = a.counters[kCntVisible];
            int bucket = kSatBuckets;
            if (saturated && s_satpos > 0 && n_vis > 0ull) {
                const uint32_t k = a.vals[r.x + s_satpos - 1];
                bucket = sat_bucket((float)(a.depthpos[k] + 1u) / (float)n_vis);
            }
            unsigned long long len = r.y - r.x;
            if (a.round == 1) {
                const unsigned long long n_pre = (unsigned long long)prefix_records((int64_t)n_vis, a.prefix);
                if (n_pre > 0ull) len = len * n_vis / n_pre;
            }
            if (len) atomicAdd(a.hist + bucket, len);
        }
        if (inside) {
            const int64_t hw = (int64_t)V.W * V.H;
            const int64_t off = (int64_t)py * V.W + px;
            const int64_t pix = V.pix_base + off;
            float* rgb = a.rgb + 3 * V.pix_base;
            rgb[off] = C0 + T * Tb.bg[0];
            rgb[hw + off] = C1 + T * Tb.bg[1];
            rgb[2 * hw + off] = C2 + T * Tb.bg[2];
            a.depth[pix] = D;
            a.alpha[pix] = 1.0f - T;
            a.tfinal[pix] = T;
            a.ncontrib[pix] = last;
            if constexpr (COUNT) {
                exam_total += exam;
                blended_total += nblend;
            }
        }
    }
    exam_total = warp_sum(exam_total);
    blended_total = warp_sum(blended_total);
    if (lane == 0 && exam_total) atomicAdd(a.counters + kCntFwdPairs, exam_total);
    if (lane == 0 && blended_total) atomicAdd(a.counters + kCntBlended, blended_total);
    if (lane == 0 && witer) atomicAdd(a.counters + kCntWarpFwd, (unsigned long long)witer);
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
// The part of one (pixel, entry) pair of the backward that does not depend
// on the running T and X: alpha, its decisions and the colour/depth dot.
struct BwdPair {
    int k;
    bool front;    // P2 <= 0
    bool near;     // alpha within 1e-6 relative of a threshold (see bwd_refine)
    bool contrib;
    float P2m, sa, al, iom, cdot;
};

__device__ __forceinline__ BwdPair bwd_pair(const float4* B, int k, float pxf, float pyf, float dC0, float dC1,
                                            float dC2, float dD)
{
    BwdPair e;
    e.k = k;
    const float4 r0 = B[3 * k];
    const float4 r1 = B[3 * k + 1];
    const float4 r2 = B[3 * k + 2];
    const float dx = __fsub_rn(pxf, r0.x), dy = __fsub_rn(pyf, r0.y);
    const float P2 = __fmaf_rn(dx, __fmaf_rn(r0.z, dx, __fmul_rn(r0.w, dy)), __fmul_rn(__fmul_rn(r1.x, dy), dy));
    // The value of 2^P2 here only feeds the adjoint, so the hardware
    // approximation (ex2.approx, a few ulp from 2^x, as is the contract's
    // polynomial) serves; the two decisions that must be the forward's --
    // alpha >= 1/255 and the 0.99 clamp -- are re-taken with the contract's
    // exponential whenever alpha lies near either threshold.  One test covers
    // both: (sa - 1/255)(sa - 0.99) is within 1.1e-6 of zero for sa within
    // about 1.1e-6 of either root (0.99 - 1/255 = 0.986), i.e. 1.1e-6 relative
    // at 0.99 and 3e-4 relative at 1/255 -- several times what the two
    // approximations can differ by (the rounding of the product is below
    // 3e-8 there).
    e.front = P2 <= 0.0f;
    e.P2m = fminf(P2, 0.0f);
    float G;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(G) : "f"(e.P2m));
    e.sa = __fmul_rn(r1.y, G);
    e.near = fabsf(__fmaf_rn(e.sa, __fsub_rn(e.sa, GSR_ALPHA_MIN + GSR_ALPHA_MAX), GSR_ALPHA_MIN * GSR_ALPHA_MAX)) <=
             1.1e-6f;
    e.cdot = dC0 * r2.x + dC1 * r2.y + dC2 * r2.z + dD * r1.z;
    return e;
}

// The contract's exponential for the (rare) pairs near a threshold.  Taken
// once per pair of entries on a warp vote, so the common case pays one vote
// instead of a divergent branch per entry.
__device__ __forceinline__ void bwd_refine(const float4* B, BwdPair& e1, BwdPair& e0)
{
    if (__any_sync(0xffffffffu, e1.near || e0.near)) {
        if (e1.near) e1.sa = __fmul_rn(B[3 * e1.k + 1].y, exp2_nonpos(e1.P2m));
        if (e0.near) e0.sa = __fmul_rn(B[3 * e0.k + 1].y, exp2_nonpos(e0.P2m));
    }
}

// The decisions and 1 / (1 - alpha) from the (refined) alpha.
__device__ __forceinline__ void bwd_finish(BwdPair& e, int lim)
{
    e.al = fminf(GSR_ALPHA_MAX, e.sa);
    e.contrib = e.k < lim && e.front && e.al >= GSR_ALPHA_MIN;
    e.iom = __fdividef(1.0f, 1.0f - e.al);   // 1 - al >= 0.01
}

// Dynamic shared memory of the backward: [2][BATCH][3] float4 records (the
// first 48 bytes of each: mean, conic, opacity, depth, colour),
// [BATCH][kSumStride] record sums, then per warp the slot buffers of gP and
// w ([kSlots][kSlotStride] floats each) and the pixels' (dC, dD) (32 float4):
// 55 KB at BATCH = 128, so four blocks share an SM.
template <int BATCH>
constexpr size_t bwd_smem_bytes()
{
    return (size_t)2 * BATCH * 48 + (size_t)BATCH * kSumStride * sizeof(float) +
           (size_t)kWarps * (2 * kSlots * kSlotStride * sizeof(float) + 32 * sizeof(float4));
}

template <int BX, int BY, int BATCH>
__global__ void __launch_bounds__(kBlendThreads, 4)
blend_bwd_kernel(const __grid_constant__ Table Tb, BlendBwdArgs a)
{
    if (earlier_wait_timed_out(a.status)) return;
    using TS = TileShape<BX, BY>;
    extern __shared__ __align__(128) float4 s_buf[];     // layout: see bwd_smem_bytes
    __shared__ __align__(8) uint64_t s_bar[2];
    __shared__ unsigned int s_item;
    __shared__ uint32_t s_idx[2][BATCH];
    __shared__ uint32_t s_maxlast;
    using ListT = typename std::conditional<(BATCH <= 256), uint8_t, uint16_t>::type;
    __shared__ ListT s_list[kWarps][BATCH];
    float* s_grad = reinterpret_cast<float*>(s_buf + 2 * BATCH * 3);
    const int tid = threadIdx.x, lane = tid & 31, w = tid >> 5;
    float* s_slots = s_grad + BATCH * kSumStride;
    float* sgp = s_slots + (size_t)w * 2 * kSlots * kSlotStride;   // this warp's gP slots
    float* swg = sgp + kSlots * kSlotStride;                          // and its w slots
    float4* sdcd = reinterpret_cast<float4*>(s_slots + (size_t)kWarps * 2 * kSlots * kSlotStride) + 32 * w;
    if (tid == 0) {
        mbar_init(&s_bar[0], 1);
        mbar_init(&s_bar[1], 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    for (int i = tid; i < BATCH * kSumStride; i += kBlendThreads) s_grad[i] = 0.0f;
    __syncthreads();
    uint32_t par0 = 0u, par1 = 0u;
    const int lx = TS::lx(tid), ly = TS::ly(tid);
    unsigned long long pairs_total = 0, witer = 0;
    bool failed = false;
    ListT* L = s_list[w];

    for (;;) {
        if (tid == 0) { s_item = atomicAdd(a.work, 1u); s_maxlast = 0; }
        __syncthreads();
        const unsigned int item = s_item;
        if ((int64_t)item >= Tb.n_tiles || failed) break;
        const int view = find_view_of_tile(Tb, item);
        const DevView& V = Tb.v[view];
        const int lt = (int)(item - V.tile_base);
        const int tx0 = (lt % V.TX) * BX, ty0 = (lt / V.TX) * BY;
        const int px = tx0 + lx, py = ty0 + ly;
        const bool inside = px < V.W && py < V.H;
        const uint2 rg = a.ranges[item];
        const float pxf = __fadd_rn((float)px, 0.5f), pyf = __fadd_rn((float)py, 0.5f);
        float Tcur = 1.0f, Tf = 1.0f, dC0 = 0, dC1 = 0, dC2 = 0, dD = 0, dA = 0;
        uint32_t mylast = 0;
        if (inside) {
            const int64_t hw = (int64_t)V.W * V.H;
            const int64_t off = (int64_t)py * V.W + px;
            const int64_t pix = V.pix_base + off;
            Tf = a.tfinal[pix];
            Tcur = Tf;
            mylast = a.ncontrib[pix];
            const float* g = a.dl_rgb + 3 * V.pix_base;
            dC0 = g[off]; dC1 = g[hw + off]; dC2 = g[2 * hw + off];
            if (a.dl_depth) dD = a.dl_depth[pix];
            if (a.dl_alpha) dA = a.dl_alpha[pix];
        }
        pairs_total += mylast;
        sdcd[lane] = make_float4(dC0, dC1, dC2, dD);   // read by the slot reduction (after __syncwarp)
        const float cxw = (float)(tx0 + (w % TS::WPR) * TS::WX + TS::WX / 2);
        const float cyw = (float)(ty0 + (w / TS::WPR) * TS::WY + TS::WY / 2);
        {
            uint32_t m = mylast;
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) m = max(m, __shfl_xor_sync(0xffffffffu, m, o));
            if (lane == 0 && m) atomicMax(&s_maxlast, m);
        }
        __syncthreads();
        const int maxlast = (int)s_maxlast;
        const int nb = (maxlast + BATCH - 1) / BATCH;
        // X = dC . S_C + dD S_D - dA T_final, S the suffix sums of the later
        // colour and depth terms (S_C starts at T_final bg): then
        // dL/dalpha_k = T_k (dC . c_k + dD z_k) - X / (1 - alpha_k).
        float X = Tf * (dC0 * Tb.bg[0] + dC1 * Tb.bg[1] + dC2 * Tb.bg[2] - dA);

        // batches from the back: the q-th processed batch covers list positions [bb*BATCH, ...)
        if (nb > 0) {
            const int bb = nb - 1;
            issue_batch<3>(a.vals, a.rec, rg.x + bb * BATCH, min(BATCH, maxlast - bb * BATCH), s_buf, &s_bar[0],
                        s_idx[0]);
        }
        for (int q = 0; q < nb; ++q) {
            const int s = q & 1;
            const int bb = nb - 1 - q;
            const int cnt = min(BATCH, maxlast - bb * BATCH);
            // exactly the (warp, entry) pairs the forward composited: lane l
            // holds the mask bytes of entries l + 32 j, read before the wait
            uint32_t mw[(BATCH + 127) / 128];
            {
                const uint8_t* wm = a.wmask + rg.x + (size_t)bb * BATCH;
#pragma unroll
                for (int j = 0; j < (BATCH + 127) / 128; ++j) mw[j] = 0u;
#pragma unroll
                for (int j = 0; j < BATCH / 32; ++j) {
                    const int t = lane + 32 * j;
                    if (t < cnt) mw[j >> 2] |= (uint32_t)wm[t] << (8 * (j & 3));
                }
            }
            const bool ok = mbar_wait_bounded(&s_bar[s], s ? par1 : par0, a.status, a.wait_ns);
            if (s) par1 ^= 1u; else par0 ^= 1u;
            // (this barrier also orders the previous batch's flush before the
            // reuse of its buffers and sums)
            if (__syncthreads_or(!ok)) {
                failed = true;
                break;
            }
            if (q + 1 < nb) {
                const int nbb = bb - 1;
                issue_batch<3>(a.vals, a.rec, rg.x + nbb * BATCH, min(BATCH, maxlast - nbb * BATCH),
                            s_buf + (size_t)(s ^ 1) * BATCH * 3, &s_bar[s ^ 1], s_idx[s ^ 1]);
            }
            const float4* B = s_buf + (size_t)s * BATCH * 3;
            int nl = 0;
            {
                const uint32_t lt = (1u << lane) - 1u;
#pragma unroll
                for (int j = 0; j < BATCH / 32; ++j) {
                    if (32 * j < cnt) {
                        const bool bit = (mw[j >> 2] >> (8 * (j & 3) + w)) & 1u;
                        const uint32_t bal = __ballot_sync(0xffffffffu, bit);
                        if (bit) L[nl + __popc(bal & lt)] = (ListT)(32 * j + lane);
                        nl += __popc(bal);
                    }
                }
                __syncwarp();
            }
            witer += nl;
            const int lim = (int)mylast - bb * BATCH;   // this pixel's entries k < lim
            // The walk is back to front: each entry's adjoint needs T and X as
            // left by the entry after it.  Branch-free: every lane evaluates
            // the pair, and a lane that does not composite it stores zero gP
            // and w into slot s of its warp's buffers.  Entries are taken two
            // at a time so that the second's alpha (independent of T and X)
            // overlaps the first's.
            auto step = [&](const BwdPair& e, int s) {
                const float Tk = Tcur * e.iom;
                const float wgt = e.contrib ? e.al * Tk : 0.0f;
                // the clamped alpha (sa >= 0.99) has no derivative
                const float ga = (e.contrib && e.sa < GSR_ALPHA_MAX) ? Tk * e.cdot - e.iom * X : 0.0f;
                // dL/dP2 / ln2; the record's coefficients, ln2 and the sign of
                // the mean gradient are applied once per record when the
                // shared sums are flushed
                const float gP = ga * e.al;
                X = fmaf(wgt, e.cdot, X);
                Tcur = e.contrib ? Tk : Tcur;
                const int at = s * kSlotStride + slot_col(lane, s);
                sgp[at] = gP;
                swg[at] = wgt;
            };
            auto pair = [&](int i1, int s) {
                BwdPair e1 = bwd_pair(B, L[i1], pxf, pyf, dC0, dC1, dC2, dD);
                BwdPair e0 = bwd_pair(B, L[i1 - 1], pxf, pyf, dC0, dC1, dC2, dD);
                bwd_refine(B, e1, e0);
                bwd_finish(e1, lim);
                bwd_finish(e0, lim);
                step(e1, s);
                step(e0, s + 1);
            };
            int i = nl - 1;
            // whole groups of kSlots entries, slot indices fixed at compile time
            for (; i >= kSlots - 1; i -= kSlots) {
#pragma unroll
                for (int p = 0; p < kSlots; p += 2) pair(i - p, p);
                __syncwarp();
                slots_reduce(sgp, swg, sdcd, kSlots, lane, L, i, B, cxw, cyw, s_grad);
                __syncwarp();
            }
            // the last (fewer than kSlots) entries
            const int i0 = i;      // list position of slot 0's entry
            int slot = 0;          // entries in the slot buffers (warp-uniform)
            for (; i >= 1; i -= 2, slot += 2) pair(i, slot);
            if (i == 0) {
                BwdPair e = bwd_pair(B, L[0], pxf, pyf, dC0, dC1, dC2, dD);
                if (__any_sync(0xffffffffu, e.near) && e.near) e.sa = __fmul_rn(B[3 * e.k + 1].y, exp2_nonpos(e.P2m));
                bwd_finish(e, lim);
                step(e, slot);
                ++slot;
            }
            if (slot) {
                __syncwarp();
                slots_reduce(sgp, swg, sdcd, slot, lane, L, i0, B, cxw, cyw, s_grad);
                __syncwarp();
            }
            __syncthreads();
            for (int t = tid; t < cnt; t += kBlendThreads) {
                float* sg = s_grad + t * kSumStride;
                // sums of gP dx, gP dy -> d(u, v); gP dx^2, gP dx dy, gP dy^2 -> d(qa, qb, qc)
                const float4 q0 = B[3 * t];
                const float qc = B[3 * t + 1].x, sig = B[3 * t + 1].y;
                const float sx = sg[0], sy = sg[1];
                const float4 v0 = make_float4(-GSR_LN2 * (2.0f * q0.z * sx + q0.w * sy),
                                              -GSR_LN2 * (q0.w * sx + 2.0f * qc * sy), GSR_LN2 * sg[2],
                                              GSR_LN2 * sg[3]);
                // sum dL/dalpha G over the pixels where alpha is not clamped = sum gP / sigma
                const float4 v1 = make_float4(GSR_LN2 * sg[4], sg[5] / sig, sg[6], 0.0f);
                const float4 v2 = make_float4(sg[7], sg[8], sg[9], 0.0f);
                const uint32_t k = s_idx[s][t];
                if (v0.x != 0.0f || v0.y != 0.0f || v0.z != 0.0f || v0.w != 0.0f || v1.x != 0.0f || v1.y != 0.0f ||
                    v1.z != 0.0f || v2.x != 0.0f || v2.y != 0.0f || v2.z != 0.0f) {
                    atomicAdd(a.grad_rec + 3 * (size_t)k, v0);
                    atomicAdd(a.grad_rec + 3 * (size_t)k + 1, v1);
                    atomicAdd(a.grad_rec + 3 * (size_t)k + 2, v2);
                }
#pragma unroll
                for (int c = 0; c < 10; ++c) sg[c] = 0.0f;
            }
        }
        __syncthreads();   // every thread has read s_item / s_maxlast of this tile; the flush is done
    }
    pairs_total = warp_sum(pairs_total);
    if (lane == 0 && pairs_total) atomicAdd(a.counters + kCntBwdPairs, pairs_total);
    if (lane == 0 && witer) atomicAdd(a.counters + kCntWarpBwd, witer);
}

// ---------------------------------------------------------------------------
// dispatch
// ---------------------------------------------------------------------------
template <int BX, int BY, int BATCH, bool COUNT>
static void fwd_launch(const Table& T, const BlendFwdArgs& a, int num_sms, cudaStream_t s)
{
    auto kern = blend_fwd_kernel<BX, BY, BATCH, COUNT>;
    const size_t smem = (size_t)2 * BATCH * kRecordBytes;
    // function attributes and occupancy are per device
    static std::atomic<int> per_sm_dev[kMaxDevices];
    const int per_sm = per_device_once(per_sm_dev, [&] {
        int n = 0;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kBlendThreads, smem);
        return n < 1 ? 1 : n;
    });
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > T.n_tiles) grid = T.n_tiles;
    if (grid < 1) return;
    GSR_COUNT_LAUNCH();
    kern<<<(unsigned)grid, kBlendThreads, smem, s>>>(T, a);
}

template <int BX, int BY, int BATCH>
static void fwd_one(const Table& T, const BlendFwdArgs& a, int num_sms, cudaStream_t s)
{
    if (a.count_pairs) fwd_launch<BX, BY, BATCH, true>(T, a, num_sms, s);
    else fwd_launch<BX, BY, BATCH, false>(T, a, num_sms, s);
}

template <int BX, int BY, int BATCH>
static void bwd_one(const Table& T, const BlendBwdArgs& a, int num_sms, cudaStream_t s)
{
    auto kern = blend_bwd_kernel<BX, BY, BATCH>;
    const size_t smem = bwd_smem_bytes<BATCH>();
    // function attributes and occupancy are per device
    static std::atomic<int> per_sm_dev[kMaxDevices];
    const int per_sm = per_device_once(per_sm_dev, [&] {
        int n = 0;
        cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        // all of the unified L1 as shared memory: four blocks of the
        // 128-record variant fit (the kernel keeps records in shared memory,
        // not in L1)
        cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, (int)cudaSharedmemCarveoutMaxShared);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kern, kBlendThreads, smem);
        return n < 1 ? 1 : n;
    });
    int64_t grid = (int64_t)num_sms * per_sm;
    if (grid > T.n_tiles) grid = T.n_tiles;
    if (grid < 1) return;
    GSR_COUNT_LAUNCH();
    kern<<<(unsigned)grid, kBlendThreads, smem, s>>>(T, a);
}

bool blend_supported(int tw, int th, int batch)
{
    const bool shape = (tw == 16 && th == 16) || (tw == 32 && th == 8) || (tw == 8 && th == 32);
    const bool b = batch == 128 || batch == 256 || batch == 512;
    return shape && b;
}

#define GSR_DISPATCH(FN, T, batch, ...)                                                          \
    do {                                                                                         \
        const int tw_ = (T).tile_w, th_ = (T).tile_h;                                            \
        if (tw_ == 16 && th_ == 16) {                                                            \
            if (batch == 128) FN<16, 16, 128>(T, __VA_ARGS__);                                   \
            else if (batch == 256) FN<16, 16, 256>(T, __VA_ARGS__);                              \
            else FN<16, 16, 512>(T, __VA_ARGS__);                                                \
        } else if (tw_ == 32 && th_ == 8) {                                                      \
            if (batch == 128) FN<32, 8, 128>(T, __VA_ARGS__);                                    \
            else if (batch == 256) FN<32, 8, 256>(T, __VA_ARGS__);                               \
            else FN<32, 8, 512>(T, __VA_ARGS__);                                                 \
        } else {                                                                                 \
            if (batch == 128) FN<8, 32, 128>(T, __VA_ARGS__);                                    \
            else if (batch == 256) FN<8, 32, 256>(T, __VA_ARGS__);                               \
            else FN<8, 32, 512>(T, __VA_ARGS__);                                                 \
        }                                                                                        \
    } while (0)

void launch_blend_fwd(const Table& T, int batch, const BlendFwdArgs& a, int num_sms, cudaStream_t s)
{
    GSR_DISPATCH(fwd_one, T, batch, a, num_sms, s);
}

void launch_blend_bwd(const Table& T, int batch, const BlendBwdArgs& a, int num_sms, cudaStream_t s)
{
    GSR_DISPATCH(bwd_one, T, batch, a, num_sms, s);
}

}  // namespace gsr
