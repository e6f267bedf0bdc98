// gsr_common.cuh -- shared device definitions of libgsr (sm_103a).
//
// The rasterizer is the 3D Gaussian Splatting renderer that the paper's
// per-keyframe optimisation runs (Sec. 3.3): Gaussians and camera poses are
// optimised jointly, SH gradients detached for the pose.  This header holds
//   * the binary32 "decision contract": every operation that feeds a discrete
//     decision (cull, radius, tile rectangle, depth key, alpha skip/clamp,
//     early stop, colour clamp) is written with explicitly rounded intrinsics
//     (__fmul_rn, __fadd_rn, __fdiv_rn, __fsqrt_rn, __fmaf_rn) in a fixed
//     order, so the compiler cannot contract or reorder it;
//   * the library's own binary32 exponentials (Cody-Waite reduction and a
//     degree-7 Taylor polynomial; no CUDA math-library exp);
//   * PTX wrappers for mbarriers and bulk (TMA) global->shared copies with
//     bounded waits that report a timeout instead of hanging;
//   * the per-call view table passed by value to every kernel.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace gsr {

constexpr int kMaxViews = 64;
constexpr int kRecordBytes = 64;        // projected record: 4 x float4
constexpr int kGradFloats = 12;         // per-record 2D gradient: 3 x float4

// status word bits (device)
constexpr uint32_t kErrRecCapacity = 1u;
constexpr uint32_t kErrInstCapacity = 2u;
constexpr uint32_t kErrTimeout = 4u;
constexpr uint32_t kErrOverflow32 = 8u;
constexpr uint32_t kErrInternal = 16u;   // an internal consistency check failed (access skipped)
constexpr uint32_t kErrFullCapacity = 32u;  // more kept tile rows than the row descriptors hold

// decision constants (binary32)
#define GSR_ALPHA_MAX 0x1.fae148p-1f    // 0.99
#define GSR_ALPHA_MIN 0x1.010102p-8f    // 1/255
#define GSR_T_STOP    0x1.a36e2ep-14f   // 1e-4
#define GSR_NHALF_L2E (-0x1.715476p-1f) // -log2(e)/2
#define GSR_NL2E      (-0x1.715476p+0f) // -log2(e)
#define GSR_LN2       0x1.62e430p-1f

// ---------------------------------------------------------------------------
// view table (kernel parameter, by value)
// ---------------------------------------------------------------------------
struct DevView {
    float R[9];          // world-to-camera rotation, row-major
    float t[3];
    float fx, fy, cx, cy;
    int W, H, TX, TY;    // image and tile-grid size
    int group, vl;       // view group and position inside it
    int64_t tile_base;   // first global tile id
    int64_t pix_base;    // first pixel of the view in the output images
    int64_t vm_base;     // first record of the view in view-major numbering
};

struct DevGroup {
    const uint32_t* subset;  // ascending Gaussian indices or nullptr (= all)
    int64_t n;               // Gaussians in the group
    int64_t rec_base;        // first flat record (flat = rec_base + j * nv + vl)
    int64_t slot_base;       // first Gaussian slot (slot = slot_base + j)
    int first_view, nv;
};

// vis_aux.w of a visible record: its view (bits 0-7) and the forward's
// decisions that the backward reuses -- the frustum guard on x/z and y/z
// (bits 8-9 and 10-11, each -1, 0 or 1 stored plus one) and the clamp of
// each colour channel at zero (bits 12-14).
__device__ __forceinline__ uint32_t aux_pack(int view, int clx, int cly, uint32_t cclamp)
{
    return (uint32_t)view | ((uint32_t)(clx + 1) << 8) | ((uint32_t)(cly + 1) << 10) | (cclamp << 12);
}
__device__ __forceinline__ int aux_view(uint32_t w) { return (int)(w & 0xffu); }
__device__ __forceinline__ int aux_clx(uint32_t w) { return (int)((w >> 8) & 3u) - 1; }
__device__ __forceinline__ int aux_cly(uint32_t w) { return (int)((w >> 10) & 3u) - 1; }
__device__ __forceinline__ uint32_t aux_cclamp(uint32_t w) { return (w >> 12) & 7u; }

struct Table {
    int n_views, n_groups, tile_w, tile_h, sh_degree, pad0;
    float near_plane, bg[3];
    float inv_tile_w, inv_tile_h;   // 1 / tile size, exact (the sizes are powers of two)
    int64_t n_records, n_slots, n_tiles, n_pixels;
    DevView v[kMaxViews];
    DevGroup g[kMaxViews];
};

// ---------------------------------------------------------------------------
// Camera of one view, as the per-record kernels use it.  Kernels whose lanes
// hold records of different views (the preprocess: one Gaussian's records
// are consecutive) read it from a shared-memory copy of the view table --
// the kernel-parameter bank would serialise those reads per distinct
// address.  21 four-byte words per view: an odd stride, so lanes reading the
// same field of different views hit different banks.
// ---------------------------------------------------------------------------
struct Cam {
    float R[9], t[3];
    float fx, fy, cx, cy;
    int W, H, TX, TY, group;
    float lx, ly;   // frustum-guard limits on x/z and y/z (see chain_forward)
    float cp[3];    // camera centre -R^T t
    float pad;
};
static_assert(sizeof(Cam) == 27 * 4, "odd word stride");

__device__ __forceinline__ void cam_table_fill(Cam* s, const Table& Tb)
{
    for (int v = threadIdx.x; v < Tb.n_views; v += blockDim.x) {
        const DevView& V = Tb.v[v];
        Cam c;
#pragma unroll
        for (int i = 0; i < 9; ++i) c.R[i] = V.R[i];
#pragma unroll
        for (int i = 0; i < 3; ++i) c.t[i] = V.t[i];
        c.fx = V.fx; c.fy = V.fy; c.cx = V.cx; c.cy = V.cy;
        c.W = V.W; c.H = V.H; c.TX = V.TX; c.TY = V.TY; c.group = V.group;
        // 1.3 times the larger half-extent of the image over the focal length
        c.lx = __fmul_rn(1.3f, __fdiv_rn(fmaxf(V.cx, __fsub_rn((float)V.W, V.cx)), V.fx));
        c.ly = __fmul_rn(1.3f, __fdiv_rn(fmaxf(V.cy, __fsub_rn((float)V.H, V.cy)), V.fy));
#pragma unroll
        for (int j = 0; j < 3; ++j)
            c.cp[j] = -__fmaf_rn(V.R[j], V.t[0], __fmaf_rn(V.R[3 + j], V.t[1], __fmul_rn(V.R[6 + j], V.t[2])));
        c.pad = 0.0f;
        s[v] = c;
    }
}

// ---------------------------------------------------------------------------
// binary32 exponentials
// ---------------------------------------------------------------------------

// 2^y for y <= 0: clamp y to >= -126; n = nearest integer (1.5*2^23
// shifter); f = y - n exact in [-1/2, 1/2]; 2^f = exp(f ln2) by the degree-7
// Taylor series (coefficients (ln2)^k / k! in binary32), Horner with fused
// multiply-add; times 2^n built from exponent bits.
__device__ __forceinline__ float exp2_poly(float f)
{
    float p = 0x1.ffcbfcp-17f;
    p = __fmaf_rn(p, f, 0x1.430912p-13f);
    p = __fmaf_rn(p, f, 0x1.5d87fep-10f);
    p = __fmaf_rn(p, f, 0x1.3b2ab6p-7f);
    p = __fmaf_rn(p, f, 0x1.c6b08ep-5f);
    p = __fmaf_rn(p, f, 0x1.ebfbe0p-3f);
    p = __fmaf_rn(p, f, 0x1.62e430p-1f);
    p = __fmaf_rn(p, f, 1.0f);
    return p;
}

__device__ __forceinline__ float exp2_nonpos(float y)
{
    y = fmaxf(y, -126.0f);
    const float j = __fadd_rn(y, 0x1.8p23f);
    const float nf = __fsub_rn(j, 0x1.8p23f);
    const float f = __fsub_rn(y, nf);
    const int n = __float_as_int(j) - __float_as_int(0x1.8p23f);
    return __fmul_rn(exp2_poly(f), __int_as_float((n + 127) << 23));
}

// e^x: clamp x to [-87, 88]; n = nearest integer to x log2(e) (fused, with the
// shifter); r = x - n ln2 in two Cody-Waite steps; e^r by the degree-7 Taylor
// series (1/k! in binary32), Horner with fused multiply-add; times 2^n.
__device__ __forceinline__ float exp_contract(float x)
{
    x = fmaxf(x, -87.0f);
    x = fminf(x, 88.0f);
    const float j = __fmaf_rn(x, 0x1.715476p+0f, 0x1.8p23f);
    const float nf = __fsub_rn(j, 0x1.8p23f);
    float r = __fmaf_rn(nf, -0x1.62e430p-1f, x);
    r = __fmaf_rn(nf, 0x1.05c610p-29f, r);
    float p = 0x1.a01a02p-13f;
    p = __fmaf_rn(p, r, 0x1.6c16c2p-10f);
    p = __fmaf_rn(p, r, 0x1.111112p-7f);
    p = __fmaf_rn(p, r, 0x1.555556p-5f);
    p = __fmaf_rn(p, r, 0x1.555556p-3f);
    p = __fmaf_rn(p, r, 0.5f);
    p = __fmaf_rn(p, r, 1.0f);
    p = __fmaf_rn(p, r, 1.0f);
    const int n = __float2int_rz(nf);
    return __fmul_rn(p, __int_as_float((n + 127) << 23));
}

// ---------------------------------------------------------------------------
// Tile culling of the lists (a GPU optimisation: the lists of the definition
// are the full 3-sigma rectangles; any list that keeps every record that
// composites or stops some pixel gives the same images).  A record keeps a
// tile of its rectangle only if some pixel centre of the tile can reach
// alpha >= 1/255, judged conservatively:
//   sigma < 1/255 -> no tile (alpha <= sigma);
//   the form A = -[[qa, qb/2], [qb/2, qc]] (log2 units) not positive
//   definite, or cond(A) >= 1e5 -> every tile of the rectangle;
//   else the pixel offsets (x, y) with P(x, y) = -(x, y) A (x, y)^T >= t,
//   t = log2(1 / (255 sigma)) - m - 1e-4, form an ellipse: m = 9e-5 cond +
//   1e-4 bounds the binary32 error of the blend's P at any pixel that can
//   composite, 1e-4 that of sigma 2^P.  Over a tile row's band of pixel
//   centres [y0, y1] the ellipse's x-extent is one interval [xl, xr] (the
//   right boundary is concave in y and peaks at the ellipse's rightmost
//   point, the left one mirrors it), so the row keeps the contiguous run of
//   tiles whose pixel-centre columns meet it.  Intervals and bands are padded
//   by more than the binary32 error of this evaluation and of the blend's
//   pixel offsets.
// ---------------------------------------------------------------------------
struct RowCull {
    float u, v;          // the mean (pixels)
    float i2a, b, det4;  // 1 / (2a) with a = -qa, b = qb, det4 = 4 a c - b^2 (c = -qc)
    float s4a;           // 4 a s, s = -t > 0
    float ymax, yr;      // the ellipse's y half-extent; y of its rightmost point
    float pad;           // padding of bands and intervals (pixels)
    int mode;            // 0: no tile, 1: every tile of the rectangle, 2: per-row intervals
};

__device__ __forceinline__ RowCull row_cull_setup(float u, float v, float qa, float qb, float qc, float sig)
{
    RowCull r;
    r.u = u; r.v = v; r.i2a = -0.5f / qa; r.b = qb; r.det4 = 0.0f; r.s4a = 0.0f; r.ymax = 0.0f; r.yr = 0.0f;
    r.pad = 0.0f;
    if (!(sig >= GSR_ALPHA_MIN)) { r.mode = 0; return r; }
    const float a = -qa, c = -qc;
    const float det = a * c - 0.25f * qb * qb;
    const float mid = 0.5f * (a + c);
    const float lmax = mid + sqrtf(fmaxf(mid * mid - det, 0.0f));
    if (!(det > 0.0f) || !(lmax > 0.0f) || !(lmax * lmax < 1e5f * det)) { r.mode = 1; return r; }
    const float cond = lmax * lmax / det;
    const float s = log2f(255.0f * sig) + fmaf(9e-5f, cond, 1e-4f) + 1e-4f;   // -t
    r.mode = 2;
    r.det4 = 4.0f * det;
    r.s4a = 4.0f * a * s;
    r.ymax = sqrtf(r.s4a / r.det4);
    const float xmax = sqrtf(4.0f * c * s / r.det4);
    r.yr = qb * xmax / (2.0f * c);
    r.pad = 0.02f + 1e-5f * (fabsf(u) + fabsf(v)) + 1e-4f * (xmax + r.ymax);
    return r;
}

// The rows [*ty0, *ty1) of a rectangle [y0r, y1r) whose bands of pixel
// centres (tiles th high) can meet the ellipse.
__device__ __forceinline__ void row_cull_rows(const RowCull& r, int y0r, int y1r, int th, int& ty0, int& ty1)
{
    ty0 = y0r; ty1 = y1r;
    if (r.mode == 0) { ty1 = y0r; return; }
    if (r.mode != 2) return;
    // row ty's band of offsets is [ty th + 0.5 - v, ty th + th - 0.5 - v]
    const float ith = 1.0f / (float)th;   // exact: th is a power of two
    const float lo = ceilf((r.v - r.ymax - r.pad - 0.5f) * ith - 1.0f) - 1.0f;
    const float hi = floorf((r.v + r.ymax + r.pad - 0.5f) * ith) + 1.0f;
    ty0 = (int)fminf(fmaxf(lo, (float)y0r), (float)y1r);
    ty1 = (int)fminf(fmaxf(hi + 1.0f, (float)ty0), (float)y1r);
}

// The kept tiles of the rectangle row whose pixel centres span the offsets
// [y0, y1] (relative to the mean), as the first tile column and a count
// (0: none), within the rectangle's columns [x0, x1) of tiles tw wide
// (tw a power of two).
__device__ __forceinline__ int row_cull_run(const RowCull& r, float y0, float y1, int x0, int x1, int tw, int& first)
{
    first = x0;
    if (r.mode != 2) return r.mode == 1 ? x1 - x0 : 0;
    const float lo = fmaxf(y0 - r.pad, -r.ymax), hi = fminf(y1 + r.pad, r.ymax);
    if (!(lo <= hi)) return 0;
    const float yc = fminf(fmaxf(r.yr, lo), hi);
    const float xr = (r.b * yc + sqrtf(fmaxf(r.s4a - r.det4 * yc * yc, 0.0f))) * r.i2a + r.pad;
    const float yl = fminf(fmaxf(-r.yr, lo), hi);
    const float xl = (r.b * yl - sqrtf(fmaxf(r.s4a - r.det4 * yl * yl, 0.0f))) * r.i2a - r.pad;
    // tile tx spans pixel-centre offsets [tx tw + 0.5 - u, tx tw + tw - 0.5 - u]
    const float itw = 1.0f / (float)tw;   // exact: tw is a power of two
    const float flo = ceilf((xl + r.u + 0.5f) * itw - 1.0f), fhi = floorf((xr + r.u - 0.5f) * itw);
    const int tlo = (int)fminf(fmaxf(flo, (float)x0), (float)x1);
    const int thi = (int)fmaxf(fminf(fhi, (float)(x1 - 1)), (float)(x0 - 1));
    first = tlo;
    return thi >= tlo ? thi - tlo + 1 : 0;
}

// ---------------------------------------------------------------------------
// real spherical harmonics, l <= 3, basis order m = -l..l, with the
// Condon-Shortley sign (-1)^m; binary32 with a fixed operation order
// ---------------------------------------------------------------------------
#define GSR_SH0  0.28209479177387814    // 1/(2 sqrt pi)
#define GSR_SH1  0.4886025119029199     // sqrt(3/(4 pi))
#define GSR_SH2A 1.0925484305920792     // sqrt(15/pi)/2
#define GSR_SH2B 0.31539156525252005    // sqrt(5/pi)/4
#define GSR_SH2C 0.5462742152960396     // sqrt(15/pi)/4
#define GSR_SH3A 0.5900435899266435     // sqrt(35/(2 pi))/4
#define GSR_SH3B 2.890611442640554      // sqrt(105/pi)/2
#define GSR_SH3C 0.4570457994644658     // sqrt(21/(2 pi))/4
#define GSR_SH3D 0.3731763325901154     // sqrt(7/pi)/4
#define GSR_SH3E 1.445305721320277      // sqrt(105/pi)/4

__device__ __forceinline__ void sh_basis(int deg, float x, float y, float z, float* b)
{
    b[0] = (float)GSR_SH0;
    if (deg < 1) return;
    b[1] = __fmul_rn((float)(-GSR_SH1), y);
    b[2] = __fmul_rn((float)GSR_SH1, z);
    b[3] = __fmul_rn((float)(-GSR_SH1), x);
    if (deg < 2) return;
    const float xx = __fmul_rn(x, x), yy = __fmul_rn(y, y), zz = __fmul_rn(z, z);
    const float xy = __fmul_rn(x, y), yz = __fmul_rn(y, z), xz = __fmul_rn(x, z);
    b[4] = __fmul_rn((float)GSR_SH2A, xy);
    b[5] = __fmul_rn((float)(-GSR_SH2A), yz);
    b[6] = __fmul_rn((float)GSR_SH2B, __fsub_rn(__fsub_rn(__fmul_rn(2.0f, zz), xx), yy));
    b[7] = __fmul_rn((float)(-GSR_SH2A), xz);
    b[8] = __fmul_rn((float)GSR_SH2C, __fsub_rn(xx, yy));
    if (deg < 3) return;
    const float f4z = __fsub_rn(__fsub_rn(__fmul_rn(4.0f, zz), xx), yy);
    b[9]  = __fmul_rn(__fmul_rn((float)(-GSR_SH3A), y), __fsub_rn(__fmul_rn(3.0f, xx), yy));
    b[10] = __fmul_rn(__fmul_rn((float)GSR_SH3B, xy), z);
    b[11] = __fmul_rn(__fmul_rn((float)(-GSR_SH3C), y), f4z);
    b[12] = __fmul_rn(__fmul_rn((float)GSR_SH3D, z),
                      __fsub_rn(__fsub_rn(__fmul_rn(2.0f, zz), __fmul_rn(3.0f, xx)), __fmul_rn(3.0f, yy)));
    b[13] = __fmul_rn(__fmul_rn((float)(-GSR_SH3C), x), f4z);
    b[14] = __fmul_rn(__fmul_rn((float)GSR_SH3E, z), __fsub_rn(xx, yy));
    b[15] = __fmul_rn(__fmul_rn((float)(-GSR_SH3A), x), __fsub_rn(xx, __fmul_rn(3.0f, yy)));
}

// sum_i w_i d b_i / d(x, y, z) for the basis above, accumulated term by term
// (value path of the adjoint; plain fp32): the direction gradient of a
// colour whose channel-weighted coefficients are w_i.
__device__ __forceinline__ void sh_dir_grad(int deg, float x, float y, float z, const float* w, float* g)
{
    float g0 = 0.0f, g1 = 0.0f, g2 = 0.0f;
    if (deg >= 1) {
        const float C1 = (float)GSR_SH1;
        g1 -= C1 * w[1]; g2 += C1 * w[2]; g0 -= C1 * w[3];
    }
    if (deg >= 2) {
        const float A = (float)GSR_SH2A, B = (float)GSR_SH2B, Cc = (float)GSR_SH2C;
        g0 += A * y * w[4]; g1 += A * x * w[4];
        g1 -= A * z * w[5]; g2 -= A * y * w[5];
        g0 -= 2.0f * B * x * w[6]; g1 -= 2.0f * B * y * w[6]; g2 += 4.0f * B * z * w[6];
        g0 -= A * z * w[7]; g2 -= A * x * w[7];
        g0 += 2.0f * Cc * x * w[8]; g1 -= 2.0f * Cc * y * w[8];
    }
    if (deg >= 3) {
        const float a3 = (float)GSR_SH3A, b3 = (float)GSR_SH3B, c3 = (float)GSR_SH3C;
        const float d3 = (float)GSR_SH3D, e3 = (float)GSR_SH3E;
        const float xx = x * x, yy = y * y, zz = z * z;
        const float xy = x * y, yz = y * z, xz = x * z;
        const float t1 = 3.0f * xx - 3.0f * yy;
        g0 -= a3 * 6.0f * xy * w[9]; g1 -= a3 * t1 * w[9];
        g0 += b3 * yz * w[10]; g1 += b3 * xz * w[10]; g2 += b3 * xy * w[10];
        g0 += c3 * 2.0f * xy * w[11]; g1 -= c3 * (4.0f * zz - xx - 3.0f * yy) * w[11]; g2 -= c3 * 8.0f * yz * w[11];
        g0 -= d3 * 6.0f * xz * w[12]; g1 -= d3 * 6.0f * yz * w[12];
        g2 += d3 * (6.0f * zz - 3.0f * xx - 3.0f * yy) * w[12];
        g0 -= c3 * (4.0f * zz - 3.0f * xx - yy) * w[13]; g1 += c3 * 2.0f * xy * w[13]; g2 -= c3 * 8.0f * xz * w[13];
        g0 += e3 * 2.0f * xz * w[14]; g1 -= e3 * 2.0f * yz * w[14]; g2 += e3 * (xx - yy) * w[14];
        g0 -= a3 * t1 * w[15]; g1 += a3 * 6.0f * xy * w[15];
    }
    g[0] = g0; g[1] = g1; g[2] = g2;
}

// d b_i / d(x, y, z) of the basis above (value path of the adjoint; plain fp32)
__device__ __forceinline__ void sh_basis_grad(int deg, float x, float y, float z, float (*db)[3])
{
    for (int i = 0; i < 16; ++i) db[i][0] = db[i][1] = db[i][2] = 0.0f;
    if (deg < 1) return;
    db[1][1] = -(float)GSR_SH1; db[2][2] = (float)GSR_SH1; db[3][0] = -(float)GSR_SH1;
    if (deg < 2) return;
    const float A = (float)GSR_SH2A, B = (float)GSR_SH2B, Cc = (float)GSR_SH2C;
    db[4][0] = A * y;  db[4][1] = A * x;
    db[5][1] = -A * z; db[5][2] = -A * y;
    db[6][0] = -2.0f * B * x; db[6][1] = -2.0f * B * y; db[6][2] = 4.0f * B * z;
    db[7][0] = -A * z; db[7][2] = -A * x;
    db[8][0] = 2.0f * Cc * x; db[8][1] = -2.0f * Cc * y;
    if (deg < 3) return;
    const float a3 = (float)GSR_SH3A, b3 = (float)GSR_SH3B, c3 = (float)GSR_SH3C;
    const float d3 = (float)GSR_SH3D, e3 = (float)GSR_SH3E;
    const float xx = x * x, yy = y * y, zz = z * z;
    db[9][0] = -a3 * 6.0f * x * y;
    db[9][1] = -a3 * (3.0f * xx - 3.0f * yy);
    db[10][0] = b3 * y * z; db[10][1] = b3 * x * z; db[10][2] = b3 * x * y;
    db[11][0] = c3 * 2.0f * x * y;
    db[11][1] = -c3 * (4.0f * zz - xx - 3.0f * yy);
    db[11][2] = -c3 * 8.0f * y * z;
    db[12][0] = -d3 * 6.0f * x * z;
    db[12][1] = -d3 * 6.0f * y * z;
    db[12][2] = d3 * (6.0f * zz - 3.0f * xx - 3.0f * yy);
    db[13][0] = -c3 * (4.0f * zz - 3.0f * xx - yy);
    db[13][1] = c3 * 2.0f * x * y;
    db[13][2] = -c3 * 8.0f * x * z;
    db[14][0] = e3 * 2.0f * x * z;
    db[14][1] = -e3 * 2.0f * y * z;
    db[14][2] = e3 * (xx - yy);
    db[15][0] = -a3 * (3.0f * xx - 3.0f * yy);
    db[15][1] = a3 * 6.0f * x * y;
}

// ---------------------------------------------------------------------------
// PTX: mbarrier + bulk copies, bounded waits
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ uint64_t global_timer_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

constexpr uint64_t kWaitLimitNs = 2000000000ull;   // 2 s: the default limit of every device wait

// Wait for phase `parity` of an mbarrier; gives up after limit_ns and sets
// kErrTimeout in *status.  Returns false on timeout.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint32_t* status,
                                                  uint64_t limit_ns)
{
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_timer_ns();
    for (;;) {
        for (int i = 0; i < 32; ++i)
            if (mbar_try_wait(bar, parity)) return true;
        if (global_timer_ns() - t0 > limit_ns) {
            atomicOr(status, kErrTimeout);
            return false;
        }
    }
}

// Bulk asynchronous copy global -> shared (TMA engine), completion counted
// in bytes on the mbarrier.  Addresses 16-byte aligned, size multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst_smem, const void* src_gmem, uint32_t bytes, uint64_t* bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst_smem)),
        "l"(src_gmem), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// decoupled look-back (single-pass scan across blocks of one launch)
// status word: bits 63..62 = 0 not ready, 1 aggregate, 2 inclusive prefix
// ---------------------------------------------------------------------------
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v)
{
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p)
{
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

constexpr unsigned long long kLbAgg = 1ull << 62;
constexpr unsigned long long kLbInc = 2ull << 62;
constexpr unsigned long long kLbMask = (1ull << 62) - 1;

// Called by one thread of block `b` (blocks numbered in launch-ticket order)
// with the block's own total; returns the exclusive prefix of the totals of
// blocks 0..b-1.  Waits on predecessors are bounded by limit_ns (kErrTimeout).
__device__ __forceinline__ unsigned long long lookback_exclusive(unsigned long long* st, long long b,
                                                                 unsigned long long total, uint32_t* status,
                                                                 uint64_t limit_ns)
{
    if (b == 0) {
        st_release_u64(st, kLbInc | total);
        return 0ull;
    }
    st_release_u64(st + b, kLbAgg | total);
    unsigned long long excl = 0;
    long long p = b - 1;
    const uint64_t t0 = global_timer_ns();
    while (p >= 0) {
        const unsigned long long s = ld_acquire_u64(st + p);
        const unsigned long long flag = s & ~kLbMask;
        if (flag == kLbInc) { excl += s & kLbMask; break; }
        if (flag == kLbAgg) { excl += s & kLbMask; --p; continue; }
        if (global_timer_ns() - t0 > limit_ns) { atomicOr(status, kErrTimeout); break; }
        __nanosleep(64);
    }
    st_release_u64(st + b, kLbInc | (excl + total));
    return excl;
}

// Warp-wide version, called by all 32 lanes of one warp of block `b`: the
// lanes inspect 32 predecessors at a time, add up their aggregates back to the
// nearest inclusive prefix, and publish this block's inclusive prefix.
// Returns the exclusive prefix in every lane.  Waits are bounded by limit_ns.
__device__ __forceinline__ unsigned long long lookback_exclusive_warp(unsigned long long* st, long long b,
                                                                      unsigned long long total, uint32_t* status,
                                                                      uint64_t limit_ns)
{
    const int lane = threadIdx.x & 31;
    if (b == 0) {
        if (lane == 0) st_release_u64(st, kLbInc | total);
        return 0ull;
    }
    if (lane == 0) st_release_u64(st + b, kLbAgg | total);
    unsigned long long excl = 0;
    long long p = b - 1;
    const uint64_t t0 = global_timer_ns();
    while (true) {
        const long long i = p - lane;
        const unsigned long long s = i >= 0 ? ld_acquire_u64(st + i) : (kLbInc | 0ull);
        const unsigned long long flag = s & ~kLbMask;
        if (__any_sync(0xffffffffu, flag == 0ull)) {
            if (global_timer_ns() - t0 > limit_ns) {
                if (lane == 0) atomicOr(status, kErrTimeout);
                break;
            }
            __nanosleep(32);
            continue;
        }
        const uint32_t inc = __ballot_sync(0xffffffffu, flag == kLbInc);
        unsigned long long v = s & kLbMask;
        if (inc) {
            const int first = __ffs(inc) - 1;
            if (lane > first) v = 0ull;
            excl += warp_sum(v);
            break;
        }
        excl += warp_sum(v);
        p -= 32;
    }
    if (lane == 0) st_release_u64(st + b, kLbInc | (excl + total));
    return excl;
}

// A kernel that follows a look-back in the same call starts only if no wait
// of an earlier kernel gave up: after a timeout, prefix offsets (and so the
// records they place) are unreliable, and nothing may index through them.
// One thread reads the status word (set by earlier launches, so stable for
// this one); the block takes the decision together.  Call at kernel entry,
// from every thread of the block.
__device__ __forceinline__ bool earlier_wait_timed_out(const uint32_t* status)
{
    __shared__ int s_timed_out;
    if (threadIdx.x == 0) s_timed_out = (*reinterpret_cast<const volatile uint32_t*>(status) & kErrTimeout) != 0;
    __syncthreads();
    return s_timed_out != 0;
}

// ---------------------------------------------------------------------------
// small helpers
// ---------------------------------------------------------------------------
__device__ __forceinline__ int find_group(const Table& T, int64_t rec)
{
    int lo = 0, hi = T.n_groups - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.g[mid].rec_base <= rec) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ int find_view_of_tile(const Table& T, int64_t tile)
{
    int lo = 0, hi = T.n_views - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (T.v[mid].tile_base <= tile) lo = mid; else hi = mid - 1;
    }
    return lo;
}

}  // namespace gsr
