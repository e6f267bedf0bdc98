// gsr_insert.cu -- insertion probability and scale initialisation of new
// Gaussians (Sec. 3.2, Eq. 4-6) on a batch of views.
//
//   P(I)(u, v) = min(|| LoG_sigma * I (u, v) ||, 1)   (norm over RGB)
//   P_a = max(P(I) - P(I~), 0)   I: ground truth, I~: rendering
//   inserted where P_a > tau_a, with scale S = d / (2 sqrt(P(I)) f)
//
// LoG: the Laplacian of Gaussian sampled at integer offsets within
// r = ceil(3 sigma), shifted to zero mean (taps computed on the host in
// double, rounded to binary32); image edges clamped.  The insertion decision
// is integer output, so it is taken in binary32 with a fixed order: per
// channel, acc = fma(tap, pixel, acc) over dy = -r..r, dx = -r..r from 0;
// n2 = fma(a0, a0, fma(a1, a1, a2 a2)); P = min(sqrt(n2), 1);
// P_a = max(P_I - P_R, 0).
//
// Two launches: a stencil kernel per 32x32 pixel tile (the channel planes of
// the tile and its halo staged in shared memory) writing P_a and S, and an
// order-preserving compaction of the inserted pixel indices (chunks of 1024
// pixels in ticket order, decoupled look-back).  HBM-bound: 2 x 12 B of
// colour + 4 B depth read, 8 B written per pixel.
#include <cmath>

#include "gsr_common.cuh"
#include "gsr_kernels.h"

namespace gsr {

constexpr int kInsTW = 32, kInsTH = 32;  // pixels per tile; a warp covers 32 columns x 4 rows
constexpr int kInsThreads = 256;
static_assert(kInsTH % (kInsThreads / kInsTW) == 0, "whole rows per thread");

void insertion_taps(double sigma, int* radius, float* taps)
{
    const int r = (int)std::ceil(3.0 * sigma), K = 2 * r + 1;
    double t[kInsMaxTaps];
    double sum = 0.0;
    const double s2 = sigma * sigma;
    for (int y = -r; y <= r; ++y) {
        for (int x = -r; x <= r; ++x) {
            const double q = (double)(x * x + y * y);
            const double v = (q - 2.0 * s2) / (s2 * s2) * std::exp(-q / (2.0 * s2)) / (2.0 * 3.14159265358979323846 * s2);
            t[(y + r) * K + (x + r)] = v;
            sum += v;
        }
    }
    const double mean = sum / (double)(K * K);
    for (int i = 0; i < K * K; ++i) taps[i] = (float)(t[i] - mean);
    *radius = r;
}

// One 32x32 tile per block iteration: a thread owns four vertically adjacent
// pixels of one column and walks the 2R+4 halo rows it needs once, feeding
// each row to every output that uses it.  Every output still accumulates its
// taps in the fixed order (dy ascending, then dx), so the result is that of
// the one-pixel loop.  The three channels of one image are staged at a time.
template <int R>
__global__ void __launch_bounds__(kInsThreads)
insert_prob_kernel(const __grid_constant__ InsertTable T, const float* __restrict__ gt, const float* __restrict__ ren,
                   const float* __restrict__ depth, float* __restrict__ p_a, float* __restrict__ scale)
{
    constexpr int K = 2 * R + 1, HW = kInsTW + 2 * R, HH = kInsTH + 2 * R, PLANE = HW * HH;
    constexpr int RPT = kInsTH / (kInsThreads / kInsTW);   // rows per thread
    __shared__ float s_img[3 * PLANE];
    const int tid = threadIdx.x, lx = tid % kInsTW, lg = tid / kInsTW;
    for (int64_t tile = blockIdx.x; tile < T.tile_base[T.n_views]; tile += gridDim.x) {
        int v = 0;
        while (tile >= T.tile_base[v + 1]) ++v;
        const int W = T.W[v], H = T.H[v];
        const int64_t lt = tile - T.tile_base[v];
        const int tx0 = (int)(lt % T.TX[v]) * kInsTW, ty0 = (int)(lt / T.TX[v]) * kInsTH;
        const int64_t hw = (int64_t)W * H;
        float P[2][RPT];
#pragma unroll
        for (int img = 0; img < 2; ++img) {
            const float* src0 = (img ? ren : gt) + 3 * T.pix_base[v];
            // the tile and its halo, edges clamped
#pragma unroll
            for (int c = 0; c < 3; ++c) {
                const float* __restrict__ plane = src0 + c * hw;
                for (int i = tid; i < PLANE; i += kInsThreads) {
                    const int row = i / HW, col = i - row * HW;
                    const int y = min(max(ty0 - R + row, 0), H - 1), x = min(max(tx0 - R + col, 0), W - 1);
                    s_img[c * PLANE + i] = __ldg(plane + (int64_t)y * W + x);
                }
            }
            __syncthreads();
            float n2[RPT];
#pragma unroll
            for (int j = 0; j < RPT; ++j) n2[j] = 0.0f;
            float a[3][RPT];
#pragma unroll
            for (int c = 0; c < 3; ++c) {
#pragma unroll
                for (int j = 0; j < RPT; ++j) a[c][j] = 0.0f;
                const float* s = s_img + c * PLANE + (lg * RPT) * HW + lx;
#pragma unroll
                for (int ir = 0; ir < K + RPT - 1; ++ir) {
#pragma unroll
                    for (int dx = 0; dx < K; ++dx) {
                        const float px = s[ir * HW + dx];
#pragma unroll
                        for (int j = 0; j < RPT; ++j) {
                            const int dy = ir - j;
                            if (dy >= 0 && dy < K) a[c][j] = __fmaf_rn(T.taps[dy * K + dx], px, a[c][j]);
                        }
                    }
                }
            }
#pragma unroll
            for (int j = 0; j < RPT; ++j) {
                n2[j] = __fmaf_rn(a[0][j], a[0][j], __fmaf_rn(a[1][j], a[1][j], __fmul_rn(a[2][j], a[2][j])));
                P[img][j] = fminf(__fsqrt_rn(n2[j]), 1.0f);
            }
            __syncthreads();   // s_img is rewritten by the next image or tile
        }
        const int x = tx0 + lx;
#pragma unroll
        for (int j = 0; j < RPT; ++j) {
            const int y = ty0 + lg * RPT + j;
            if (x < W && y < H) {
                const int64_t pix = T.pix_base[v] + (int64_t)y * W + x;
                const float pa = fmaxf(__fsub_rn(P[0][j], P[1][j]), 0.0f);
                p_a[pix] = pa;
                float sc = 0.0f;
                if (pa > T.tau)
                    sc = __fdiv_rn(depth[pix], __fmul_rn(__fmul_rn(2.0f, __fsqrt_rn(P[0][j])), T.f[v]));
                scale[pix] = sc;
            }
        }
    }
}

constexpr int kInsCompactItems = 16;
constexpr int kInsChunk = kInsThreads * kInsCompactItems;

// Indices of the pixels with P_a > tau (the stencil's decision, re-read from
// the stored binary32 P_a), ascending; the total goes to *count.
__global__ void __launch_bounds__(kInsThreads)
insert_compact_kernel(const float* __restrict__ p_a, int64_t n, float tau, uint32_t* __restrict__ index,
                      int64_t cap, unsigned long long* count, unsigned long long* lb, unsigned int* ticket,
                      uint32_t* status, uint64_t wait_ns)
{
    __shared__ long long s_blk;
    __shared__ uint32_t s_warp[kInsThreads / 32];
    __shared__ unsigned long long s_base;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const int64_t nchunks = (n + kInsChunk - 1) / kInsChunk;
    const bool vec = (reinterpret_cast<uintptr_t>(p_a) & 15u) == 0u;
    for (;;) {
        if (tid == 0) s_blk = (long long)atomicAdd(ticket, 1u);
        __syncthreads();
        const long long blk = s_blk;
        if (blk >= nchunks) break;
        const int64_t i0 = blk * kInsChunk + (int64_t)tid * kInsCompactItems;
        uint32_t keep = 0u;
        if (vec && i0 + kInsCompactItems <= n) {
            // 16-byte loads: i0 is a multiple of 16 floats and p_a 16-byte aligned
            const float4* q = reinterpret_cast<const float4*>(p_a + i0);
#pragma unroll
            for (int u = 0; u < kInsCompactItems / 4; ++u) {
                const float4 v = q[u];
                keep |= (v.x > tau ? 1u : 0u) << (4 * u);
                keep |= (v.y > tau ? 1u : 0u) << (4 * u + 1);
                keep |= (v.z > tau ? 1u : 0u) << (4 * u + 2);
                keep |= (v.w > tau ? 1u : 0u) << (4 * u + 3);
            }
        } else {
#pragma unroll
            for (int j = 0; j < kInsCompactItems; ++j)
                if (i0 + j < n && p_a[i0 + j] > tau) keep |= 1u << j;
        }
        const uint32_t cnt = __popc(keep);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_warp[wid] = incl;
        __syncthreads();
        if (wid == 0) {
            const uint32_t c = lane < kInsThreads / 32 ? s_warp[lane] : 0u;
            uint32_t ws = c;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const uint32_t t = __shfl_up_sync(0xffffffffu, ws, o);
                if (lane >= o) ws += t;
            }
            const uint32_t acc = __shfl_sync(0xffffffffu, ws, 31);
            if (lane < kInsThreads / 32) s_warp[lane] = ws - c;
            const unsigned long long base = lookback_exclusive_warp(lb, blk, acc, status, wait_ns);
            if (lane == 0) {
                s_base = base;
                if (blk == nchunks - 1) *count = base + acc;
            }
        }
        __syncthreads();
        unsigned long long pos = s_base + s_warp[wid] + incl - cnt;
#pragma unroll
        for (int j = 0; j < kInsCompactItems; ++j) {
            if (keep & (1u << j)) {
                if (pos < (unsigned long long)cap) index[pos] = (uint32_t)(i0 + j);
                ++pos;
            }
        }
        __syncthreads();   // s_blk, s_warp, s_base are rewritten by the next chunk
    }
}

int64_t insertion_lb_words(int64_t n_pixels) { return (n_pixels + kInsChunk - 1) / kInsChunk + 1; }

void launch_insertion(const InsertTable& T, const float* gt, const float* rendered, const float* depth, float* p_a,
                      float* scale, uint32_t* index, int64_t index_cap, unsigned long long* count,
                      unsigned long long* lb, unsigned int* ticket, uint32_t* status, uint64_t wait_ns, int num_sms,
                      cudaStream_t s)
{
    const int64_t tiles = T.tile_base[T.n_views];
    if (tiles <= 0) return;
    int64_t grid = tiles < (int64_t)num_sms * 8 ? tiles : (int64_t)num_sms * 8;
    GSR_COUNT_LAUNCH();
    switch (T.r) {
    case 1: insert_prob_kernel<1><<<(unsigned)grid, kInsThreads, 0, s>>>(T, gt, rendered, depth, p_a, scale); break;
    case 2: insert_prob_kernel<2><<<(unsigned)grid, kInsThreads, 0, s>>>(T, gt, rendered, depth, p_a, scale); break;
    case 3: insert_prob_kernel<3><<<(unsigned)grid, kInsThreads, 0, s>>>(T, gt, rendered, depth, p_a, scale); break;
    case 4: insert_prob_kernel<4><<<(unsigned)grid, kInsThreads, 0, s>>>(T, gt, rendered, depth, p_a, scale); break;
    case 5: insert_prob_kernel<5><<<(unsigned)grid, kInsThreads, 0, s>>>(T, gt, rendered, depth, p_a, scale); break;
    case 6: insert_prob_kernel<6><<<(unsigned)grid, kInsThreads, 0, s>>>(T, gt, rendered, depth, p_a, scale); break;
    default: insert_prob_kernel<7><<<(unsigned)grid, kInsThreads, 0, s>>>(T, gt, rendered, depth, p_a, scale); break;
    }
    if (!count) return;
    const int64_t n = T.pix_base[T.n_views];
    int64_t cgrid = insertion_lb_words(n) - 1;
    // one resident wave: more chunks in flight only lengthen the look-back walks
    if (cgrid > (int64_t)num_sms * 4) cgrid = (int64_t)num_sms * 4;
    if (cgrid < 1) cgrid = 1;
    GSR_COUNT_LAUNCH();
    insert_compact_kernel<<<(unsigned)cgrid, kInsThreads, 0, s>>>(p_a, n, T.tau, index, index_cap, count, lb, ticket,
                                                                status, wait_ns);
}

}  // namespace gsr
