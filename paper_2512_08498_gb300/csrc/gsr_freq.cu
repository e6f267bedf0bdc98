// gsr_freq.cu -- frequency-based scheduling (Sec. 3.3, Eq. 9-12) for a batch
// of images.
//
//   X(I) = sum over frequencies (i, j) of || DFT(I)(i, j) ||_2     (Eq. 10, 11)
//
// the unnormalised 2-D DFT of each colour channel, the norm taken over the
// three channels at each frequency.  Then r = X(I) / X(I~) (Eq. 9) weights
// the frames drawn for optimisation and r' = X(I^n) / X(I~) (Eq. 12), I^n the
// ground truth at downsampling factor n, raises the level when below tau_f.
//
// The DFT is a mixed-radix Stockham transform (radix 4, 2, 3, 5 butterflies
// and a direct radix-p pass for any other prime) run in shared memory, in two
// passes over each image:
//   rows     two real rows of one channel packed as one complex sequence;
//            after the transform the Hermitian split gives both rows' spectra
//            for k = 0 .. W/2 (the other half is their conjugate mirror),
//            written to a half-spectrum buffer [3][H][W/2 + 1];
//   columns  C adjacent columns of that buffer, one channel after the other,
//            transformed along y; |F_c|^2 summed over the channels in shared
//            memory, then sqrt and summed with weight 2 for the columns whose
//            mirror k' = W - k is not stored (1 for k = 0 and k = W/2).
// Box downsampling (I^n) is applied while loading the rows.  Values are FP32
// (twiddles from a host table computed in double); the magnitudes are summed
// per thread in FP32 and across threads and blocks in FP64.
#include <cmath>

#include "gsr_common.cuh"
#include "gsr_kernels.h"

namespace gsr {

constexpr int kRowThreads = 128;
constexpr int kColThreads = 256;

static uint32_t recip32(int d) { return d <= 1 ? 0u : (uint32_t)((((uint64_t)1 << 32) + (uint64_t)d - 1) / (uint64_t)d); }

bool fft_plan(int n, FftPlan* P)
{
    int radix[2 * kFftMaxStages];
    int k = 0, rest = n;
    while (rest % 4 == 0 && k < kFftMaxStages) { radix[k++] = 4; rest /= 4; }
    for (int p = 2; p <= 5 && rest > 1; ++p)
        while (rest % p == 0 && k < kFftMaxStages) { radix[k++] = p; rest /= p; }
    for (int p = 7; rest > 1 && k < kFftMaxStages; p += 2)
        while (rest % p == 0 && k < kFftMaxStages) { radix[k++] = p; rest /= p; }
    if (rest != 1 || n < 1 || n > kFreqMaxDim) return false;
    P->n = n;
    P->n_stages = k;
    int Ns = 1;
    for (int i = 0; i < k; ++i) {
        FftStage& S = P->st[i];
        S.R = radix[i]; S.Ns = Ns; S.m = n / S.R; S.step = n / (Ns * S.R);
        S.mag_m = recip32(S.m); S.mag_ns = recip32(Ns); S.mag_r = recip32(S.R); S.pad = 0;
        Ns *= S.R;
    }
    return true;
}

// x / d for x < 2^16, d < 2^16, by the reciprocal ceil(2^32 / d) (0 for d = 1)
__device__ __forceinline__ int udiv16(int x, uint32_t mag) { return mag ? (int)__umulhi((uint32_t)x, mag) : x; }

__device__ __forceinline__ float2 cmul(float2 a, float2 b)
{
    return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 mul_ni(float2 a) { return make_float2(a.y, -a.x); }   // -i a

// R-point forward DFTs, y_q = sum_r v_r exp(-2 pi i q r / R), in place.
template <int R> __device__ __forceinline__ void butterfly(float2* v);

template <> __device__ __forceinline__ void butterfly<2>(float2* v)
{
    const float2 a = v[0], b = v[1];
    v[0] = cadd(a, b); v[1] = csub(a, b);
}

template <> __device__ __forceinline__ void butterfly<4>(float2* v)
{
    const float2 t0 = cadd(v[0], v[2]), t1 = csub(v[0], v[2]);
    const float2 t2 = cadd(v[1], v[3]), t3 = mul_ni(csub(v[1], v[3]));
    v[0] = cadd(t0, t2); v[2] = csub(t0, t2);
    v[1] = cadd(t1, t3); v[3] = csub(t1, t3);
}

template <> __device__ __forceinline__ void butterfly<3>(float2* v)
{
    constexpr float h = 0.8660254037844386f;   // sin(2 pi / 3)
    const float2 s = cadd(v[1], v[2]), d = csub(v[1], v[2]);
    const float2 m = make_float2(v[0].x - 0.5f * s.x, v[0].y - 0.5f * s.y);
    const float2 rot = mul_ni(make_float2(h * d.x, h * d.y));   // -i sin(2 pi/3) d
    v[0] = cadd(v[0], s);
    v[1] = cadd(m, rot);
    v[2] = csub(m, rot);
}

template <> __device__ __forceinline__ void butterfly<5>(float2* v)
{
    constexpr float c1 = 0.30901699437494745f, c2 = -0.8090169943749475f;   // cos(2 pi k / 5), k = 1, 2
    constexpr float s1 = 0.9510565162951535f, s2 = 0.5877852522924731f;     // sin(2 pi k / 5)
    const float2 a0 = v[0];
    const float2 p1 = cadd(v[1], v[4]), d1 = csub(v[1], v[4]);
    const float2 p2 = cadd(v[2], v[3]), d2 = csub(v[2], v[3]);
    const float2 m1 = make_float2(a0.x + c1 * p1.x + c2 * p2.x, a0.y + c1 * p1.y + c2 * p2.y);
    const float2 m2 = make_float2(a0.x + c2 * p1.x + c1 * p2.x, a0.y + c2 * p1.y + c1 * p2.y);
    const float2 r1 = mul_ni(make_float2(s1 * d1.x + s2 * d2.x, s1 * d1.y + s2 * d2.y));
    const float2 r2 = mul_ni(make_float2(s2 * d1.x - s1 * d2.x, s2 * d1.y - s1 * d2.y));
    v[0] = cadd(a0, cadd(p1, p2));
    v[1] = cadd(m1, r1); v[4] = csub(m1, r1);
    v[2] = cadd(m2, r2); v[3] = csub(m2, r2);
}

// One Stockham pass over nseq sequences of length n stored back to back.
// Butterfly j (of m = n / R) reads src[j + r m], r < R, twiddled by
// W_{Ns R}^{r (j mod Ns)}, and writes its R outputs to
// dst[(j - j mod Ns) R + j mod Ns + q Ns], q < R; Ns is the product of the
// radices of the earlier passes.  One twiddle is loaded per butterfly, its
// powers formed by complex products.
template <int R>
__device__ __forceinline__ void fft_pass(const float2* __restrict__ src, float2* __restrict__ dst, int nseq, int n,
                                         const FftStage& S, const float2* __restrict__ tw)
{
    const int m = S.m, Ns = S.Ns, step = S.step;
    const uint32_t mag_m = S.mag_m, mag_ns = S.mag_ns;
    for (int t = threadIdx.x; t < nseq * m; t += blockDim.x) {
        const int s = udiv16(t, mag_m), j = t - s * m;
        const int jb = udiv16(j, mag_ns), jm = j - jb * Ns;
        const float2* in = src + s * n + j;
        float2 v[R];
#pragma unroll
        for (int r = 0; r < R; ++r) v[r] = in[r * m];
        if (jm != 0) {
            const float2 w1 = __ldg(tw + jm * step);
            float2 w = w1;
#pragma unroll
            for (int r = 1; r < R; ++r) {
                v[r] = cmul(v[r], w);
                if (r + 1 < R) w = cmul(w, w1);
            }
        }
        butterfly<R>(v);
        float2* out = dst + s * n + jb * Ns * R + jm;
#pragma unroll
        for (int q = 0; q < R; ++q) out[q * Ns] = v[q];
    }
}

// The same pass for a prime radix R > 5: one thread per output, the R-point
// DFT by its definition; the combined twiddle of input r for output q is
// W_{Ns R}^{r (j mod Ns + q Ns)}.
__device__ void fft_pass_direct(const float2* __restrict__ src, float2* __restrict__ dst, int nseq, int n,
                                const FftStage& S, const float2* __restrict__ tw)
{
    const int R = S.R, m = S.m, Ns = S.Ns, NsR = Ns * R, step = S.step;
    for (int t = threadIdx.x; t < nseq * n; t += blockDim.x) {
        const int s = t / n, u = t - s * n;
        const int j = udiv16(u, S.mag_r), q = u - j * R;
        const int jb = udiv16(j, S.mag_ns), jm = j - jb * Ns;
        const float2* in = src + s * n;
        const int e = jm + q * Ns;   // < Ns R
        float2 acc = in[j];
        int idx = 0;
        for (int r = 1; r < R; ++r) {
            idx += e;
            if (idx >= NsR) idx -= NsR;
            acc = cadd(acc, cmul(in[j + r * m], __ldg(tw + idx * step)));
        }
        dst[s * n + jb * NsR + jm + q * Ns] = acc;
    }
}

// Transform nseq sequences held in a; b is scratch of the same size.
// Returns the buffer that holds the result.  All threads of the block call it.
__device__ float2* fft_run(float2* a, float2* b, int nseq, const FftPlan& P)
{
    for (int st = 0; st < P.n_stages; ++st) {
        const FftStage& S = P.st[st];
        switch (S.R) {
        case 4: fft_pass<4>(a, b, nseq, P.n, S, P.tw); break;
        case 2: fft_pass<2>(a, b, nseq, P.n, S, P.tw); break;
        case 3: fft_pass<3>(a, b, nseq, P.n, S, P.tw); break;
        case 5: fft_pass<5>(a, b, nseq, P.n, S, P.tw); break;
        default: fft_pass_direct(a, b, nseq, P.n, S, P.tw); break;
        }
        __syncthreads();
        float2* t = a; a = b; b = t;
    }
    return a;
}

__device__ __forceinline__ int image_of(const FreqTable& T, int64_t item, bool rows)
{
    int lo = 0, hi = T.n_images - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        const int64_t base = rows ? T.img[mid].row_base : T.img[mid].col_base;
        if (base <= item) lo = mid; else hi = mid - 1;
    }
    return lo;
}

// Row pass: item = (image, row pair, channel).  Rows y0 = 2p and y0 + 1 of
// channel c (box-averaged over factor x factor source pixels) are the real
// and imaginary parts of one sequence Z; their spectra are
// A(k) = (Z(k) + conj Z(-k)) / 2 and B(k) = (Z(k) - conj Z(-k)) / (2i).
__global__ void __launch_bounds__(kRowThreads)
dft_rows_kernel(const __grid_constant__ FreqTable T, float2* __restrict__ inter)
{
    extern __shared__ float2 sm[];
    for (int64_t item = blockIdx.x; item < T.row_items; item += gridDim.x) {
        const FreqImage& I = T.img[image_of(T, item, true)];
        const int64_t local = item - I.row_base;
        const int c = (int)(local % 3), y0 = 2 * (int)(local / 3);
        const int Wd = I.Wd, f = I.factor;
        const bool two = y0 + 1 < I.Hd;
        const float* __restrict__ plane = I.src + (int64_t)c * I.H * I.W;
        float2* a = sm;
        float2* b = sm + Wd;
        if (f == 1) {
            // four loads per row in flight per thread
            const float* __restrict__ r0 = plane + (int64_t)y0 * I.W;
            const float* __restrict__ r1 = r0 + (two ? I.W : 0);
            for (int x = threadIdx.x; x < Wd; x += 4 * kRowThreads) {
                float p0[4], p1[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int xi = x + u * kRowThreads;
                    p0[u] = xi < Wd ? __ldg(r0 + xi) : 0.0f;
                    p1[u] = xi < Wd ? __ldg(r1 + xi) : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int xi = x + u * kRowThreads;
                    if (xi < Wd) a[xi] = make_float2(p0[u], two ? p1[u] : 0.0f);
                }
            }
        } else {
            const float inv = 1.0f / (float)(f * f);
            for (int x = threadIdx.x; x < Wd; x += kRowThreads) {
                float p0 = 0.0f, p1 = 0.0f;
                for (int dy = 0; dy < f; ++dy) {
                    const float* r0 = plane + (int64_t)(y0 * f + dy) * I.W + (int64_t)x * f;
                    for (int dx = 0; dx < f; ++dx) p0 += __ldg(r0 + dx);
                    if (two) {
                        const float* r1 = plane + (int64_t)((y0 + 1) * f + dy) * I.W + (int64_t)x * f;
                        for (int dx = 0; dx < f; ++dx) p1 += __ldg(r1 + dx);
                    }
                }
                a[x] = make_float2(p0 * inv, p1 * inv);
            }
        }
        __syncthreads();
        const float2* z = fft_run(a, b, 1, T.plan[I.row_plan]);
        float2* o = inter + I.inter + ((int64_t)c * I.Hd + y0) * I.Wh;
        for (int k = threadIdx.x; k < I.Wh; k += blockDim.x) {
            const float2 z1 = z[k], z2 = z[k == 0 ? 0 : Wd - k];
            o[k] = make_float2(0.5f * (z1.x + z2.x), 0.5f * (z1.y - z2.y));
            if (two) o[I.Wh + k] = make_float2(0.5f * (z1.y + z2.y), 0.5f * (z2.x - z1.x));
        }
        __syncthreads();   // the buffers are rewritten by the next item
    }
}

// Column pass: item = (image, C adjacent half-spectrum columns).  Shared
// memory: two C x Hd complex buffers and C x Hd floats of sum_c |F_c|^2.
__global__ void __launch_bounds__(kColThreads)
dft_cols_kernel(const __grid_constant__ FreqTable T, const float2* __restrict__ inter, double* __restrict__ xacc)
{
    extern __shared__ float2 sm[];
    __shared__ double s_red[kColThreads / 32];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    for (int64_t item = blockIdx.x; item < T.col_items; item += gridDim.x) {
        const int ii = image_of(T, item, false);
        const FreqImage& I = T.img[ii];
        const int Hd = I.Hd, Wh = I.Wh;
        const int k0 = (int)(item - I.col_base) * I.C;
        const int nc = min(I.C, Wh - k0), ne = nc * Hd;
        float2* a = sm;
        float2* b = sm + I.C * Hd;
        float* acc = reinterpret_cast<float*>(sm + 2 * I.C * Hd);
        for (int e = tid; e < ne; e += blockDim.x) acc[e] = 0.0f;
        // loads: thread = (row group, column kk), C a power of two
        const int lc = I.C == 4 ? 2 : (I.C == 2 ? 1 : 0);
        const int kk = tid & (I.C - 1), ty = tid >> lc, ystep = kColThreads >> lc;
        for (int c = 0; c < 3; ++c) {
            const float2* __restrict__ plane = inter + I.inter + (int64_t)c * Hd * Wh + k0 + kk;
            if (kk < nc) {
                for (int y = ty; y < Hd; y += 4 * ystep) {
                    float2 v[4];
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int yi = y + u * ystep;
                        v[u] = yi < Hd ? plane[(int64_t)yi * Wh] : make_float2(0.0f, 0.0f);
                    }
#pragma unroll
                    for (int u = 0; u < 4; ++u) {
                        const int yi = y + u * ystep;
                        if (yi < Hd) a[kk * Hd + yi] = v[u];
                    }
                }
            }
            __syncthreads();
            const float2* F = fft_run(a, b, nc, T.plan[I.col_plan]);
            for (int e = tid; e < ne; e += blockDim.x) {
                const float2 v = F[e];
                acc[e] += v.x * v.x + v.y * v.y;
            }
            __syncthreads();
        }
        float part = 0.0f;
        for (int q = 0; q < nc; ++q) {
            const int k = k0 + q;
            const float w = (k == 0 || 2 * k == I.Wd) ? 1.0f : 2.0f;
            float sq = 0.0f;
            for (int y = tid; y < Hd; y += kColThreads) sq += sqrtf(acc[q * Hd + y]);
            part += w * sq;
        }
        double d = (double)part;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(0xffffffffu, d, o);
        if (lane == 0) s_red[wid] = d;
        __syncthreads();
        if (tid == 0) {
            double s = 0.0;
#pragma unroll
            for (int w = 0; w < kColThreads / 32; ++w) s += s_red[w];
            atomicAdd(xacc + ii, s);
        }
        __syncthreads();   // s_red and the buffers are rewritten by the next item
    }
}

__global__ void dft_finalize_kernel(const double* __restrict__ xacc, float* __restrict__ x, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) x[i] = (float)xacc[i];
}

// Scheduler decisions in binary32 (one block): r = x_gt / x_rendered,
// r' = x_gt_level / x_rendered, level-up iff r' < tau_f; frame weights r
// (NaN -> 0, capped at 1e30; all 1 if none is positive), cumulative sums in
// frame order, and for each uniform u the first frame whose cumulative weight
// exceeds u * total (else the last frame of positive weight).
__global__ void __launch_bounds__(256)
frequency_schedule_kernel(int n, const float* __restrict__ x_gt, const float* __restrict__ x_gl,
                          const float* __restrict__ x_r, float tau, const float* __restrict__ u, int ns,
                          float* __restrict__ r, float* __restrict__ rl, int32_t* __restrict__ up,
                          int32_t* __restrict__ samples)
{
    __shared__ float s_c[kFreqMaxFrames];
    __shared__ int s_last;
    const int tid = threadIdx.x;
    for (int f = tid; f < n; f += blockDim.x) {
        const float rv = __fdiv_rn(x_gt[f], x_r[f]);
        if (r) r[f] = rv;
        if (x_gl) {
            const float lv = __fdiv_rn(x_gl[f], x_r[f]);
            if (rl) rl[f] = lv;
            if (up) up[f] = lv < tau ? 1 : 0;
        }
        s_c[f] = isnan(rv) ? 0.0f : fminf(rv, 1e30f);
    }
    __syncthreads();
    if (tid == 0) {
        bool any = false;
        for (int f = 0; f < n; ++f) any = any || s_c[f] > 0.0f;
        float c = 0.0f;
        int last = -1;
        for (int f = 0; f < n; ++f) {
            const float w = any ? s_c[f] : 1.0f;
            if (w > 0.0f) last = f;
            c = __fadd_rn(c, w);
            s_c[f] = c;
        }
        s_last = last;
    }
    __syncthreads();
    if (!samples) return;
    const float total = s_c[n - 1];
    for (int k = tid; k < ns; k += blockDim.x) {
        const float t = __fmul_rn(u[k], total);
        int lo = 0, hi = n;   // first f with c_f > t (cumulative sums do not decrease)
        while (lo < hi) {
            const int mid = (lo + hi) >> 1;
            if (s_c[mid] > t) hi = mid; else lo = mid + 1;
        }
        samples[k] = lo < n ? lo : s_last;
    }
}

template <typename K>
static int resident_blocks(K kernel, int threads, int smem)
{
    int n = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kernel, threads, smem) != cudaSuccess || n < 1) n = 1;
    return n;
}

void launch_dft_energy(const FreqTable& T, float2* inter, double* xacc, int row_smem, int col_smem, int num_sms,
                       cudaStream_t s)
{
    static std::atomic<int> attr_set[kMaxDevices];
    per_device_once(attr_set, [] {
        cudaFuncSetAttribute(dft_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, kFreqMaxDim * 16);
        cudaFuncSetAttribute(dft_cols_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 100 * 1024);
        return 1;
    });
    if (T.row_items > 0) {
        int64_t grid = (int64_t)num_sms * resident_blocks(dft_rows_kernel, kRowThreads, row_smem);
        if (grid > T.row_items) grid = T.row_items;
        GSR_COUNT_LAUNCH();
        dft_rows_kernel<<<(unsigned)grid, kRowThreads, row_smem, s>>>(T, inter);
    }
    if (T.col_items > 0) {
        int64_t grid = (int64_t)num_sms * resident_blocks(dft_cols_kernel, kColThreads, col_smem);
        if (grid > T.col_items) grid = T.col_items;
        GSR_COUNT_LAUNCH();
        dft_cols_kernel<<<(unsigned)grid, kColThreads, col_smem, s>>>(T, inter, xacc);
    }
}

void launch_dft_finalize(const double* xacc, float* x, int n, cudaStream_t s)
{
    if (n <= 0) return;
    GSR_COUNT_LAUNCH();
    dft_finalize_kernel<<<(n + 255) / 256, 256, 0, s>>>(xacc, x, n);
}

void launch_frequency_schedule(int n_frames, const float* x_gt, const float* x_gt_level, const float* x_rendered,
                               float tau_f, const float* uniforms, int n_samples, float* r, float* r_level,
                               int32_t* level_up, int32_t* samples, cudaStream_t s)
{
    GSR_COUNT_LAUNCH();
    frequency_schedule_kernel<<<1, 256, 0, s>>>(n_frames, x_gt, x_gt_level, x_rendered, tau_f, uniforms, n_samples,
                                                r, r_level, level_up, samples);
}

}  // namespace gsr
