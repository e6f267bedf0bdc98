// gsr_preprocess.cu -- projection of (view, Gaussian) records and its adjoint.
//
// Forward (one thread per flat record, Gaussian-major inside each run of
// views that share a subset, so the views of one Gaussian are adjacent
// threads and its 236 parameter bytes are fetched from HBM once):
//   EWA splatting of the 3D covariance R S S^T R^T to a 2D conic with the
//   frustum guard and a 0.3 px^2 low-pass, sigmoid opacity, colour from SH
//   along the camera-centre -> mean direction, radius 3 sqrt(lambda_max) and
//   tile rectangle.  All decision-feeding arithmetic follows the binary32
//   contract in gsr_common.cuh.  Visible records are compacted in flat order
//   with a single-pass decoupled look-back scan.
//
// Backward (one thread per visible record, Gaussian-major like the forward, so
// the views of one Gaussian are adjacent lanes and a segmented warp sum adds
// them before one write per Gaussian): exact adjoint of the forward with the
// forward's decisions (the frustum guard and colour clamp bits it stores per
// record) and its values recomputed, giving the parameter gradients summed over views
// and the per-view se(3) pose gradient (left perturbation of the
// world-to-camera matrix; the SH viewing direction is held constant for the
// pose, as the paper's joint optimisation detaches the SH gradients for the
// camera update, Sec. 3.3).
#include "gsr_common.cuh"
#include "gsr_kernels.h"

namespace gsr {

// Intermediates of the binary32 forward chain of one record.
struct Chain {
    float pc[3];
    float s[3];
    float rn, qh[4];
    float Rq[3][3], M[3][3], S[3][3];
    float lx, ly;
    int clx, cly;
    float J00, J02, J11, J12;
    float T[2][3];
    float a, b, c, det;
    float u, v, c0, c1, c2;
    float rad;
    int x0, y0, x1, y1;
    float sig;
    float dir[3], idn;
    float basis[16];
    float col[3];
    uint32_t cclamp;
};

// Coefficients c0 .. c0+3 of one Gaussian's SH row [K][3] (twelve floats,
// zero past the row's end).  Rows of K = 4 and 16 coefficients are 48 and 192
// bytes long, so when the row starts on a 16-byte boundary the chunk is three
// 16-byte loads: adjacent lanes hold different Gaussians, so each scalar load
// of a row touches one cache line per lane, and the vector loads cut those
// requests fourfold.
template <int K>
__device__ __forceinline__ void sh_chunk(const float* row, int c0, bool vec, float (&v)[12])
{
    if (K % 4 == 0 && vec) {
        const float4* p = reinterpret_cast<const float4*>(row + 3 * c0);
        const float4 a = p[0], b = p[1], c = p[2];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
        v[8] = c.x; v[9] = c.y; v[10] = c.z; v[11] = c.w;
    } else {
#pragma unroll
        for (int i = 0; i < 12; ++i) v[i] = 3 * c0 + i < 3 * K ? row[3 * c0 + i] : 0.0f;
    }
}

template <int K>
__device__ __forceinline__ bool sh_row_vec(const float* row)
{
    return K % 4 == 0 && (reinterpret_cast<uintptr_t>(row) & 15u) == 0u;
}

// The binary32 contract.  Returns false if the record is culled (z <= near,
// degenerate quaternion, non-positive determinant, empty tile rectangle).
// with_colour = false stops after the rectangle (visibility only).
template <int DEG>
__device__ __forceinline__ bool chain_forward(const Table& Tb, const Cam& V, const float* mu, const float* ls,
                                              const float* q, float ologit, const float* kk, bool with_colour,
                                              Chain& f)
{
    const float* R = V.R;
#pragma unroll
    for (int i = 0; i < 3; ++i)
        f.pc[i] = __fmaf_rn(R[3 * i], mu[0], __fmaf_rn(R[3 * i + 1], mu[1], __fmaf_rn(R[3 * i + 2], mu[2], V.t[i])));
    const float x = f.pc[0], y = f.pc[1], z = f.pc[2];
    if (!(z > Tb.near_plane)) return false;

#pragma unroll
    for (int i = 0; i < 3; ++i) f.s[i] = exp_contract(ls[i]);
    const float n2 = __fmaf_rn(q[0], q[0], __fmaf_rn(q[1], q[1], __fmaf_rn(q[2], q[2], __fmul_rn(q[3], q[3]))));
    if (!(n2 > 0.0f)) return false;
    f.rn = __fdiv_rn(1.0f, __fsqrt_rn(n2));
    const float qw = __fmul_rn(q[0], f.rn), qx = __fmul_rn(q[1], f.rn);
    const float qy = __fmul_rn(q[2], f.rn), qz = __fmul_rn(q[3], f.rn);
    f.qh[0] = qw; f.qh[1] = qx; f.qh[2] = qy; f.qh[3] = qz;
    const float xx = __fmul_rn(qx, qx), yy = __fmul_rn(qy, qy), zz = __fmul_rn(qz, qz);
    const float xy = __fmul_rn(qx, qy), xz = __fmul_rn(qx, qz), yz = __fmul_rn(qy, qz);
    const float wx = __fmul_rn(qw, qx), wy = __fmul_rn(qw, qy), wz = __fmul_rn(qw, qz);
    f.Rq[0][0] = __fmaf_rn(-2.0f, __fadd_rn(yy, zz), 1.0f);
    f.Rq[0][1] = __fmul_rn(2.0f, __fsub_rn(xy, wz));
    f.Rq[0][2] = __fmul_rn(2.0f, __fadd_rn(xz, wy));
    f.Rq[1][0] = __fmul_rn(2.0f, __fadd_rn(xy, wz));
    f.Rq[1][1] = __fmaf_rn(-2.0f, __fadd_rn(xx, zz), 1.0f);
    f.Rq[1][2] = __fmul_rn(2.0f, __fsub_rn(yz, wx));
    f.Rq[2][0] = __fmul_rn(2.0f, __fsub_rn(xz, wy));
    f.Rq[2][1] = __fmul_rn(2.0f, __fadd_rn(yz, wx));
    f.Rq[2][2] = __fmaf_rn(-2.0f, __fadd_rn(xx, yy), 1.0f);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) f.M[i][j] = __fmul_rn(f.Rq[i][j], f.s[j]);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            f.S[i][j] = __fmaf_rn(f.M[i][0], f.M[j][0], __fmaf_rn(f.M[i][1], f.M[j][1], __fmul_rn(f.M[i][2], f.M[j][2])));
            f.S[j][i] = f.S[i][j];
        }

    f.lx = V.lx;   // per view, the same binary32 expression (cam_table_fill)
    f.ly = V.ly;
    const float iz = __fdiv_rn(1.0f, z);
    const float xr = __fmul_rn(x, iz), yr = __fmul_rn(y, iz);
    f.clx = xr < -f.lx ? -1 : (xr > f.lx ? 1 : 0);
    f.cly = yr < -f.ly ? -1 : (yr > f.ly ? 1 : 0);
    const float tx = __fmul_rn(z, fminf(f.lx, fmaxf(-f.lx, xr)));
    const float ty = __fmul_rn(z, fminf(f.ly, fmaxf(-f.ly, yr)));
    const float iz2 = __fmul_rn(iz, iz);
    f.J00 = __fmul_rn(V.fx, iz);
    f.J02 = -__fmul_rn(__fmul_rn(V.fx, tx), iz2);
    f.J11 = __fmul_rn(V.fy, iz);
    f.J12 = -__fmul_rn(__fmul_rn(V.fy, ty), iz2);
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        f.T[0][j] = __fmaf_rn(f.J00, R[j], __fmul_rn(f.J02, R[6 + j]));
        f.T[1][j] = __fmaf_rn(f.J11, R[3 + j], __fmul_rn(f.J12, R[6 + j]));
    }
    float U[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j)
            U[i][j] = __fmaf_rn(f.T[i][0], f.S[0][j], __fmaf_rn(f.T[i][1], f.S[1][j], __fmul_rn(f.T[i][2], f.S[2][j])));
    f.a = __fadd_rn(__fmaf_rn(U[0][0], f.T[0][0], __fmaf_rn(U[0][1], f.T[0][1], __fmul_rn(U[0][2], f.T[0][2]))), 0.3f);
    f.b = __fmaf_rn(U[0][0], f.T[1][0], __fmaf_rn(U[0][1], f.T[1][1], __fmul_rn(U[0][2], f.T[1][2])));
    f.c = __fadd_rn(__fmaf_rn(U[1][0], f.T[1][0], __fmaf_rn(U[1][1], f.T[1][1], __fmul_rn(U[1][2], f.T[1][2]))), 0.3f);
    f.det = __fmaf_rn(f.a, f.c, -__fmul_rn(f.b, f.b));
    if (!(f.det > 0.0f)) return false;
    const float idet = __fdiv_rn(1.0f, f.det);
    f.c0 = __fmul_rn(f.c, idet);
    f.c1 = -__fmul_rn(f.b, idet);
    f.c2 = __fmul_rn(f.a, idet);
    f.u = __fmaf_rn(__fmul_rn(V.fx, x), iz, V.cx);
    f.v = __fmaf_rn(__fmul_rn(V.fy, y), iz, V.cy);

    const float mid = __fmul_rn(0.5f, __fadd_rn(f.a, f.c));
    const float lam = __fadd_rn(mid, __fsqrt_rn(fmaxf(0.1f, __fmaf_rn(mid, mid, -f.det))));
    f.rad = ceilf(__fmul_rn(3.0f, __fsqrt_rn(lam)));
    // division by the tile size: the tile sizes are powers of two, so the
    // product with the exact reciprocal is the correctly rounded quotient
    const float bx = (float)Tb.tile_w, by = (float)Tb.tile_h, ibx = Tb.inv_tile_w, iby = Tb.inv_tile_h;
    const float TXf = (float)V.TX, TYf = (float)V.TY;
    f.x0 = __float2int_rz(fminf(fmaxf(__fmul_rn(__fsub_rn(f.u, f.rad), ibx), 0.0f), TXf));
    f.x1 = __float2int_rz(fminf(fmaxf(__fmul_rn(__fadd_rn(__fadd_rn(f.u, f.rad), __fsub_rn(bx, 1.0f)), ibx), 0.0f), TXf));
    f.y0 = __float2int_rz(fminf(fmaxf(__fmul_rn(__fsub_rn(f.v, f.rad), iby), 0.0f), TYf));
    f.y1 = __float2int_rz(fminf(fmaxf(__fmul_rn(__fadd_rn(__fadd_rn(f.v, f.rad), __fsub_rn(by, 1.0f)), iby), 0.0f), TYf));
    if ((f.x1 - f.x0) * (f.y1 - f.y0) == 0) return false;
    if (!with_colour) return true;

    f.sig = __fdiv_rn(1.0f, __fadd_rn(1.0f, exp_contract(-ologit)));
    const float* cp = V.cp;   // per view, the same binary32 expression (cam_table_fill)
    const float d0 = __fsub_rn(mu[0], cp[0]), d1 = __fsub_rn(mu[1], cp[1]), d2 = __fsub_rn(mu[2], cp[2]);
    const float dn = __fsqrt_rn(__fmaf_rn(d0, d0, __fmaf_rn(d1, d1, __fmul_rn(d2, d2))));
    f.idn = __fdiv_rn(1.0f, dn);
    f.dir[0] = __fmul_rn(d0, f.idn);
    f.dir[1] = __fmul_rn(d1, f.idn);
    f.dir[2] = __fmul_rn(d2, f.idn);
    sh_basis(DEG, f.dir[0], f.dir[1], f.dir[2], f.basis);
    constexpr int K = (DEG + 1) * (DEG + 1);
    f.cclamp = 0;
    // per channel: basis_0 k_0 rounded, then fused adds in ascending i (the
    // chunks interleave the channels, not the order within one)
    float acc[3] = {0.0f, 0.0f, 0.0f};
    const bool vec = sh_row_vec<K>(kk);
#pragma unroll
    for (int c0 = 0; c0 < K; c0 += 4) {
        float kv[12];
        sh_chunk<K>(kk, c0, vec, kv);
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            if (c0 + i < K) {
#pragma unroll
                for (int ch = 0; ch < 3; ++ch)
                    acc[ch] = c0 + i == 0 ? __fmul_rn(f.basis[0], kv[ch])
                                          : __fmaf_rn(f.basis[c0 + i], kv[3 * i + ch], acc[ch]);
            }
        }
    }
#pragma unroll
    for (int ch = 0; ch < 3; ++ch) {
        float col = __fadd_rn(acc[ch], 0.5f);
        if (col < 0.0f) { f.cclamp |= 1u << ch; col = 0.0f; }
        f.col[ch] = col;
    }
    return true;
}

// The values of a visible record's forward chain that its adjoint reads,
// for the backward.  Every decision of the chain (visibility, the frustum
// guard, the colour clamp) is the forward's, read from the record's aux word,
// so only values are recomputed here, and with the fast hardware exponential,
// reciprocal and reciprocal square root: their few-ulp differences from the
// forward's binary32 values are far below the gradients' tolerance.
__device__ __forceinline__ void chain_values(const Cam& V, const float* mu, const float* ls, const float* q,
                                             float ologit, uint32_t auxw, Chain& f)
{
    const float* R = V.R;
#pragma unroll
    for (int i = 0; i < 3; ++i) f.pc[i] = fmaf(R[3 * i], mu[0], fmaf(R[3 * i + 1], mu[1], fmaf(R[3 * i + 2], mu[2], V.t[i])));
    const float x = f.pc[0], y = f.pc[1], z = f.pc[2];
#pragma unroll
    for (int i = 0; i < 3; ++i) f.s[i] = __expf(ls[i]);
    f.rn = rsqrtf(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);   // > 0: the record is visible
    const float qw = q[0] * f.rn, qx = q[1] * f.rn, qy = q[2] * f.rn, qz = q[3] * f.rn;
    f.qh[0] = qw; f.qh[1] = qx; f.qh[2] = qy; f.qh[3] = qz;
    f.Rq[0][0] = 1.0f - 2.0f * (qy * qy + qz * qz);
    f.Rq[0][1] = 2.0f * (qx * qy - qw * qz);
    f.Rq[0][2] = 2.0f * (qx * qz + qw * qy);
    f.Rq[1][0] = 2.0f * (qx * qy + qw * qz);
    f.Rq[1][1] = 1.0f - 2.0f * (qx * qx + qz * qz);
    f.Rq[1][2] = 2.0f * (qy * qz - qw * qx);
    f.Rq[2][0] = 2.0f * (qx * qz - qw * qy);
    f.Rq[2][1] = 2.0f * (qy * qz + qw * qx);
    f.Rq[2][2] = 1.0f - 2.0f * (qx * qx + qy * qy);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) f.M[i][j] = f.Rq[i][j] * f.s[j];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = i; j < 3; ++j) {
            f.S[i][j] = f.M[i][0] * f.M[j][0] + f.M[i][1] * f.M[j][1] + f.M[i][2] * f.M[j][2];
            f.S[j][i] = f.S[i][j];
        }
    f.lx = V.lx;
    f.ly = V.ly;
    f.clx = aux_clx(auxw);
    f.cly = aux_cly(auxw);
    const float iz = __fdividef(1.0f, z), iz2 = iz * iz;
    // J02 = -fx x~ / z^2 with x~ = z clamp(x / z, -lx, lx)
    const float tx = f.clx == 0 ? x : z * ((float)f.clx * f.lx);
    const float ty = f.cly == 0 ? y : z * ((float)f.cly * f.ly);
    f.J00 = V.fx * iz;
    f.J02 = -(V.fx * tx) * iz2;
    f.J11 = V.fy * iz;
    f.J12 = -(V.fy * ty) * iz2;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        f.T[0][j] = f.J00 * R[j] + f.J02 * R[6 + j];
        f.T[1][j] = f.J11 * R[3 + j] + f.J12 * R[6 + j];
    }
    float U[2][3];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) U[i][j] = f.T[i][0] * f.S[0][j] + f.T[i][1] * f.S[1][j] + f.T[i][2] * f.S[2][j];
    f.a = U[0][0] * f.T[0][0] + U[0][1] * f.T[0][1] + U[0][2] * f.T[0][2] + 0.3f;
    f.b = U[0][0] * f.T[1][0] + U[0][1] * f.T[1][1] + U[0][2] * f.T[1][2];
    f.c = U[1][0] * f.T[1][0] + U[1][1] * f.T[1][1] + U[1][2] * f.T[1][2] + 0.3f;
    f.det = f.a * f.c - f.b * f.b;
    const float idet = __fdividef(1.0f, f.det);
    f.c0 = f.c * idet;
    f.c1 = -f.b * idet;
    f.c2 = f.a * idet;
    f.sig = __fdividef(1.0f, 1.0f + __expf(-ologit));
    const float d0 = mu[0] - V.cp[0], d1 = mu[1] - V.cp[1], d2 = mu[2] - V.cp[2];
    f.idn = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
    f.dir[0] = d0 * f.idn;
    f.dir[1] = d1 * f.idn;
    f.dir[2] = d2 * f.idn;
    f.cclamp = aux_cclamp(auxw);
}

// Conservative box (x0, x1, y0, y1 in pixel-centre coordinates) outside which
// the blend's binary32 evaluation of alpha = sigma 2^P2 is certainly below
// 1/255, so skipping those (pixel, entry) pairs changes no decision.
//   P2 = -Q(d), Q(d) = d^T A d, A = [[-qa, -qb/2], [-qb/2, -qc]] (positive
//   definite).  alpha >= 1/255 needs P2 >= log2(1/(255 sigma)) = -q_max.
//   The binary32 P2 differs from the exact quadratic form of the same
//   coefficients by at most 8 * 2^-24 * cond(A) * Q (six roundings on terms
//   bounded by 2 cond(A) Q), and the 2^x polynomial by 2 ulp; the box is the
//   bounding box of Q <= q_max (1 + 1e-3) (1 + 1e-6 cond(A) + 1e-4) + slack,
//   so outside it the binary32 alpha is below (1/255) 2^-0.001 (1 + 4e-7).
//   Above cond(A) = 1e5 the bound is not used (box = whole plane).
// Records that can never reach 1/255 (sigma < 1/255) get an empty box.
// The box itself is computed in binary32: det(A) carries a relative error of
// at most ~cond(A) 2^-22 and the square roots halve it, so every factor below
// is widened by (1 + 2e-6 cond(A) + 1e-3) and the half-widths by 0.02 px.
//
// thr_cull (out) is the threshold of the blend kernels' exact warp test:
// a warp's 8x4 block of pixel centres can hold a pixel with binary32
// P2 >= thr only if the maximum of the exact quadratic form over the block,
// evaluated in binary32, is >= thr_cull = thr - margin.  Worked in the
// rounded pixel offsets (the block's corner offsets are rounded exactly as
// the blend rounds each pixel's), the evaluation error of the form at a point
// is at most ~5 2^-24 (|qa| dx^2 + |qb dx dy| + |qc| dy^2) <= 5 2^-24 4 cond |P2|
// on either side, so margin = 1e-5 cond (|thr| + 1) + 1e-4 covers both with
// room to spare.  Forms that are not negative definite or have cond >= 1e5
// get -inf (the warp test always passes).
__device__ __forceinline__ float4 alpha_box(float u, float v, float qa, float qb, float qc, float sig, float thr,
                                            float& thr_cull)
{
    const float inf = __int_as_float(0x7f800000);
    thr_cull = -inf;
    // sigma < 1/255: 2^P2 <= 1 for P2 <= 0, so alpha < 1/255 everywhere
    if (!(sig >= GSR_ALPHA_MIN)) return make_float4(inf, -inf, inf, -inf);
    const float a11 = -qa, a12 = -0.5f * qb, a22 = -qc;
    const float det = fmaf(a11, a22, -a12 * a12);
    const float mid = 0.5f * (a11 + a22);
    const float lmax = mid + sqrtf(fmaxf(fmaf(mid, mid, -det), 0.0f));
    if (!(det > 0.0f) || !(lmax > 0.0f)) return make_float4(-inf, inf, -inf, inf);
    const float cond = lmax * lmax / det;                      // lmax / lmin
    if (!(cond < 1e5f)) return make_float4(-inf, inf, -inf, inf);
    thr_cull = thr - (1e-5f * cond * (fabsf(thr) + 1.0f) + 1e-4f);
    const float widen = 1.0f + 2e-6f * cond + 1e-3f;
    const float qmax = log2f(255.0f * sig) + 1e-3f;            // > 0 since sigma >= 1/255
    const float qb_ = qmax * widen * (1.0f + 1e-6f * cond + 1e-4f);
    const float ex = sqrtf(qb_ * a22 / det) * widen + 2e-2f;
    const float ey = sqrtf(qb_ * a11 / det) * widen + 2e-2f;
    // edges rounded outwards, so the box stays conservative at any |u|, |v|
    return make_float4(__fsub_rd(u, ex), __fadd_ru(u, ex), __fsub_rd(v, ey), __fadd_ru(v, ey));
}

// Exponent threshold of the 1/255 test: P2 < thr implies
// min(0.99, sigma 2^P2) < 1/255 under the blend's binary32 arithmetic, so the
// blend kernels may skip the exponential there without changing a decision.
// The 1e-3 margin in log2 units (a factor 0.9993) dwarfs the errors of log2f
// (~1e-6 absolute here), of the 2^x polynomial and of the product rounding.
// sigma = 0 never blends (+inf); a NaN or negative sigma keeps the full test.
__device__ __forceinline__ float alpha_threshold(float sig)
{
    const float inf = __int_as_float(0x7f800000);
    if (sig > 0.0f) return -log2f(255.0f * sig) - 1e-3f;
    return sig == 0.0f ? inf : -inf;
}

// ---------------------------------------------------------------------------
// forward
// ---------------------------------------------------------------------------
constexpr int kPreThreads = 256;

// Per view: K = (fx (|R_0| + lx |R_2|))^2 + (fy (|R_1| + ly |R_2|))^2 (1 + 1e-4),
// R_i the rows of the world-to-camera rotation and lx, ly the frustum-guard
// limits.  With |J02| <= fx lx / z (the guard clamps x~) the rows of T = J R
// have |T_0| <= fx (|R_0| + lx |R_2|) / z, likewise T_1, so the EWA terms obey
// a + c <= s_max^2 K / z^2 + 0.6 and the radius eigenvalue
// lam = mid + sqrt(max(0.1, mid^2 - det)) <= a + c + 0.32.
__device__ __forceinline__ float cull_bound_coeff(const Cam& V)
{
    const float n0 = sqrtf(V.R[0] * V.R[0] + V.R[1] * V.R[1] + V.R[2] * V.R[2]);
    const float n1 = sqrtf(V.R[3] * V.R[3] + V.R[4] * V.R[4] + V.R[5] * V.R[5]);
    const float n2 = sqrtf(V.R[6] * V.R[6] + V.R[7] * V.R[7] + V.R[8] * V.R[8]);
    const float lx = 1.3f * fmaxf(V.cx, (float)V.W - V.cx) / V.fx;
    const float ly = 1.3f * fmaxf(V.cy, (float)V.H - V.cy) / V.fy;
    const float ax = V.fx * (n0 + lx * n2), ay = V.fy * (n1 + ly * n2);
    return (ax * ax + ay * ay) * 1.0001f;
}

// Conservative pre-cull: true only if chain_forward certainly culls the
// record -- z <= near (the same binary32 expression), or a tile rectangle that
// is empty even for the radius bound rb >= ceil(3 sqrt(lam)) (x1 = 0 needs
// u + rad < 1; x0 = TX needs u - rad >= TX bx; slack covers the rounding of
// this coarser evaluation, which also takes 1/z and the square root from the
// approximate hardware functions: their relative errors, below 1e-6, are far
// inside the slack).  A NaN in the bound keeps the record.  smax is the
// Gaussian's largest axis scale, exp(max log-scale).
__device__ __forceinline__ bool surely_culled(const Cam& V, float K, float near_plane, float bx, float by,
                                              const float* mu, float smax, float& z_out)
{
    const float* R = V.R;
    float pc[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
        pc[i] = __fmaf_rn(R[3 * i], mu[0], __fmaf_rn(R[3 * i + 1], mu[1], __fmaf_rn(R[3 * i + 2], mu[2], V.t[i])));
    z_out = pc[2];
    if (!(pc[2] > near_plane)) return true;   // chain_forward's own test, bit for bit
    const float iz = __fdividef(1.0f, pc[2]);
    const float lam = smax * smax * K * iz * iz + 1.0f;
    const float rb = 3.03f * (lam * rsqrtf(lam)) + 2.0f;
    const float u = V.fx * (pc[0] * iz) + V.cx, v = V.fy * (pc[1] * iz) + V.cy;
    const float sx = 1e-4f * (fabsf(u) + rb) + 2.0f, sy = 1e-4f * (fabsf(v) + rb) + 2.0f;
    const bool cx = (u + rb + sx < 0.0f) || (u - rb - sx > (float)V.TX * bx);
    const bool cy = (v + rb + sy < 0.0f) || (v - rb - sy > (float)V.TY * by);
    return cx || cy;
}

// Record r -> (group, Gaussian j of the group, view); records are view-minor
// within a group (r = rec_base + j nv + view - first_view).
__device__ __forceinline__ void record_map(const Table& Tb, int64_t r, int& gi, int64_t& j, int& view)
{
    gi = find_group(Tb, r);
    const DevGroup& G = Tb.g[gi];
    const int64_t off = r - G.rec_base;
    if (off < ((int64_t)1 << 32)) {
        const uint32_t o = (uint32_t)off, jj = o / (uint32_t)G.nv;
        j = jj;
        view = G.first_view + (int)(o - jj * (uint32_t)G.nv);
    } else {
        j = off / G.nv;
        view = G.first_view + (int)(off - j * G.nv);
    }
}

constexpr int kPreSub = 8;                          // most records per thread and ticket
constexpr int kPreTicket = kPreThreads * kPreSub;   // most records per ticket (one look-back each)

// Persistent: tickets of 256 sub records in order (sub = a.sub, up to 8:
// fewer on small batches, so that enough tickets run at once).  Per ticket:
//   1. each thread pre-culls sub consecutive records (surely_culled), and a
//      block scan packs the candidates in record order;
//   2. the candidates' visibility (the binary32 chain up to the tile
//      rectangle), one candidate per thread in turn, as bits in record order;
//   3. one decoupled look-back for the ticket's visible count;
//   4. each Gaussian's first record offset (kstart);
//   5. the full chain on the visible records, written at their rank.
// Visible geometry is evaluated twice (2 and 5), which costs less than the
// look-backs a 256-record ticket needs: with hundreds of tickets in flight a
// look-back walks past that many unresolved predecessors.
template <int DEG>
__global__ void __launch_bounds__(kPreThreads, 3)
preprocess_fwd_kernel(const __grid_constant__ Table Tb, PreprocessArgs a)
{
    __shared__ long long s_block;
    __shared__ unsigned long long s_base;
    __shared__ uint32_t s_wcnt[kPreThreads / 32];
    __shared__ uint32_t s_vis[kPreTicket / 32];
    __shared__ uint32_t s_vpre[kPreTicket / 32];
    __shared__ uint16_t s_cand[kPreTicket];
    __shared__ uint16_t s_vlist[kPreTicket];
    __shared__ Cam s_cam[kMaxViews];
    __shared__ float s_kb[kMaxViews];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    cam_table_fill(s_cam, Tb);
    __syncthreads();
    for (int v = tid; v < Tb.n_views; v += kPreThreads) s_kb[v] = cull_bound_coeff(s_cam[v]);
    const float bx = (float)Tb.tile_w, by = (float)Tb.tile_h;
    const int sub = a.sub, ticket = kPreThreads * sub;
    const int64_t nblk = (Tb.n_records + ticket - 1) / ticket;
    constexpr int K = (DEG + 1) * (DEG + 1);
    for (;;) {
    __syncthreads();   // tables filled; the shared scratch of the previous ticket is free
    if (tid == 0) s_block = (long long)atomicAdd(a.ticket, 1u);
    for (int i = tid; i < kPreTicket / 32; i += kPreThreads) s_vis[i] = 0u;
    __syncthreads();
    const long long blk = s_block;
    if (blk >= nblk) break;
    const int64_t base = blk * ticket;

    // 1. pre-cull; remember the first-view records' Gaussian slots for kstart.
    // A thread's records are consecutive, so after the first one the next
    // (group, Gaussian, view) is a step of the view, and a Gaussian's mean and
    // largest scale are loaded once for all of its views.
    uint32_t cmask = 0u, fmask = 0u;
    uint32_t kslot[kPreSub];
    {
        const int64_t r0 = base + (int64_t)tid * sub;
        int gi = 0, view = 0;
        int64_t j = 0, gauss = -1;
        if (r0 < Tb.n_records) record_map(Tb, r0, gi, j, view);
        float mu[3] = {0.0f, 0.0f, 0.0f}, smax = 0.0f;
#pragma unroll
        for (int k = 0; k < kPreSub; ++k) {
            kslot[k] = 0u;
            const int64_t r = r0 + k;
            if (k < sub && r < Tb.n_records) {
                const DevGroup& G = Tb.g[gi];
                if (view == G.first_view) { fmask |= 1u << k; kslot[k] = (uint32_t)(G.slot_base + j); }
                const int64_t gk = G.subset ? (int64_t)G.subset[j] : j;
                if (gk != gauss) {
                    gauss = gk;
                    float ls[3];
#pragma unroll
                    for (int i = 0; i < 3; ++i) { mu[i] = a.means[3 * gauss + i]; ls[i] = a.log_scales[3 * gauss + i]; }
                    smax = expf(fmaxf(fmaxf(ls[0], ls[1]), ls[2]));
                }
                float z;
                if (!surely_culled(s_cam[view], s_kb[view], Tb.near_plane, bx, by, mu, smax, z)) cmask |= 1u << k;
                // the next record: the next view, else the next Gaussian, else the next group
                if (++view == G.first_view + G.nv) {
                    view -= G.nv;
                    if (++j == G.n) {
                        // (groups of an empty subset hold no record)
                        do { ++gi; } while (gi < Tb.n_groups && Tb.g[gi].n == 0);
                        j = 0;
                        if (gi < Tb.n_groups) view = Tb.g[gi].first_view;
                    }
                }
            }
        }
    }
    {
        const uint32_t cnt = __popc(cmask);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        if (lane == 31) s_wcnt[wid] = incl;
        __syncthreads();
        uint32_t pos = incl - cnt;
#pragma unroll
        for (int w = 0; w < kPreThreads / 32; ++w) pos += w < wid ? s_wcnt[w] : 0u;
#pragma unroll
        for (int k = 0; k < kPreSub; ++k)
            if (cmask & (1u << k)) s_cand[pos++] = (uint16_t)(tid * sub + k);
    }
    __syncthreads();
    uint32_t n_cand = 0;
#pragma unroll
    for (int w = 0; w < kPreThreads / 32; ++w) n_cand += s_wcnt[w];

    // 2. visibility of the candidates (geometry only)
    for (uint32_t c = tid; c < n_cand; c += kPreThreads) {
        const int loc = s_cand[c];
        int gi, view;
        int64_t j;
        record_map(Tb, base + loc, gi, j, view);
        const DevGroup& G = Tb.g[gi];
        const int64_t gauss = G.subset ? (int64_t)G.subset[j] : j;
        float mu[3], ls[3], q[4];
#pragma unroll
        for (int i = 0; i < 3; ++i) { mu[i] = a.means[3 * gauss + i]; ls[i] = a.log_scales[3 * gauss + i]; }
        const float4 q4 = reinterpret_cast<const float4*>(a.quats)[gauss];
        q[0] = q4.x; q[1] = q4.y; q[2] = q4.z; q[3] = q4.w;
        Chain f;
        if (chain_forward<DEG>(Tb, s_cam[view], mu, ls, q, 0.0f, nullptr, false, f))
            atomicOr(&s_vis[loc >> 5], 1u << (loc & 31));
    }
    __syncthreads();

    // 3. exclusive prefix of the visibility words, then the ticket's look-back
    if (wid == 0) {
        static_assert(kPreTicket / 32 == 64, "two words per lane");
        const uint32_t c0 = __popc(s_vis[2 * lane]), c1 = __popc(s_vis[2 * lane + 1]);
        const uint32_t t = c0 + c1;
        uint32_t incl = t;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t u = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += u;
        }
        s_vpre[2 * lane] = incl - t;
        s_vpre[2 * lane + 1] = incl - t + c0;
        const uint32_t acc = __shfl_sync(0xffffffffu, incl, 31);
        // (tests only: with kDebugWithholdFirstPrefix the first ticket never
        // publishes, so every later ticket's wait runs out)
        const unsigned long long lb = (blk == 0 && (a.debug_flags & kDebugWithholdFirstPrefix))
                                          ? 0ull
                                          : lookback_exclusive_warp(a.lb_status, blk, acc, a.status, a.wait_ns);
        if (lane == 0) {
            s_base = lb;
            if (base + ticket >= Tb.n_records) {
                // the ticket holding the last record publishes the total
                const unsigned long long total = lb + acc;
                a.counters[0] = total;
                a.kstart[Tb.n_slots] = (uint32_t)total;
                if (total > (unsigned long long)a.rec_cap) atomicOr(a.status, kErrRecCapacity);
            }
        }
    }
    __syncthreads();
    const unsigned long long tbase = s_base;

    // 4. kstart, and the visible candidates listed densely in rank order
#pragma unroll
    for (int k = 0; k < kPreSub; ++k) {
        if (fmask & (1u << k)) {
            const int loc = tid * sub + k;
            a.kstart[kslot[k]] =
                (uint32_t)(tbase + s_vpre[loc >> 5] + __popc(s_vis[loc >> 5] & ((1u << (loc & 31)) - 1u)));
        }
    }
    for (uint32_t c = tid; c < n_cand; c += kPreThreads) {
        const int loc = s_cand[c];
        const uint32_t word = s_vis[loc >> 5], bit = 1u << (loc & 31);
        if (word & bit) s_vlist[s_vpre[loc >> 5] + __popc(word & (bit - 1u))] = (uint16_t)loc;
    }
    __syncthreads();
    const uint32_t n_vis = s_vpre[kPreTicket / 32 - 1] + __popc(s_vis[kPreTicket / 32 - 1]);

    // 5. the full chain on the visible records, written at their rank
    for (uint32_t c = tid; c < n_vis; c += kPreThreads) {
        const unsigned long long excl = tbase + c;
        if (excl >= (unsigned long long)a.rec_cap) continue;
        const int loc = s_vlist[c];
        int gi, view;
        int64_t j;
        record_map(Tb, base + loc, gi, j, view);
        const DevGroup& G = Tb.g[gi];
        const int64_t gauss = G.subset ? (int64_t)G.subset[j] : j;
        float mu[3], ls[3], q[4];
#pragma unroll
        for (int i = 0; i < 3; ++i) { mu[i] = a.means[3 * gauss + i]; ls[i] = a.log_scales[3 * gauss + i]; }
        const float4 q4 = reinterpret_cast<const float4*>(a.quats)[gauss];
        q[0] = q4.x; q[1] = q4.y; q[2] = q4.z; q[3] = q4.w;
        Chain f;
        chain_forward<DEG>(Tb, s_cam[view], mu, ls, q, a.opacity[gauss], a.sh + (size_t)gauss * K * 3, true, f);
        float4* out = a.rec + 4 * excl;
        const float qa = __fmul_rn(f.c0, GSR_NHALF_L2E), qb = __fmul_rn(f.c1, GSR_NL2E);
        const float qc = __fmul_rn(f.c2, GSR_NHALF_L2E);
        out[0] = make_float4(f.u, f.v, qa, qb);
        const float thr = alpha_threshold(f.sig);
        float thr_cull;
        out[3] = alpha_box(f.u, f.v, qa, qb, qc, f.sig, thr, thr_cull);
        out[1] = make_float4(qc, f.sig, f.pc[2], thr);
        out[2] = make_float4(f.col[0], f.col[1], f.col[2], thr_cull);
        a.vis_key[excl] = __float_as_uint(f.pc[2]);
        a.vis_aux[excl] = make_uint4((uint32_t)f.x0 | ((uint32_t)f.y0 << 16), (uint32_t)f.x1 | ((uint32_t)f.y1 << 16),
                                     (uint32_t)j, aux_pack(view, f.clx, f.cly, f.cclamp));
    }
    }
}

// ---------------------------------------------------------------------------
// backward
// ---------------------------------------------------------------------------
__device__ __forceinline__ void cross3(const float* a, const float* b, float* o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

// Double-float arithmetic: a value is the unevaluated sum hi + lo of two
// binary32 numbers with |lo| <= ulp(hi) / 2, about 48 significant bits.
// Sums use Knuth's two-sum (the exact rounding error of a + b from six
// additions) in the accurate form that renormalises after adding the low
// parts, so cancelling operands keep their low-order digits; products use
// the fused multiply-add to get the exact error of hi * hi (Dekker's product
// without splitting).  On a part whose binary64 rate is 1/64 of binary32 this
// costs a few times fewer issue slots than binary64 for the same adjoint.
struct df64 {
    float hi, lo;
    __device__ __forceinline__ df64() {}
    __device__ __forceinline__ df64(float h, float l) : hi(h), lo(l) {}
    __device__ __forceinline__ df64(float x) : hi(x), lo(0.0f) {}
    __device__ __forceinline__ df64(int x) : hi((float)x), lo(0.0f) {}   // small integers only
    __device__ __forceinline__ df64(double x) : hi((float)x), lo((float)(x - (double)(float)x)) {}
    __device__ __forceinline__ explicit operator float() const { return __fadd_rn(hi, lo); }
    __device__ __forceinline__ explicit operator double() const { return (double)hi + (double)lo; }
};

__device__ __forceinline__ df64 df_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    return df64(s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb)));
}

// |a| >= |b| (or a = 0)
__device__ __forceinline__ df64 df_fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    return df64(s, __fsub_rn(b, __fsub_rn(s, a)));
}

__device__ __forceinline__ df64 operator+(df64 x, df64 y)
{
    df64 s = df_two_sum(x.hi, y.hi);
    const df64 t = df_two_sum(x.lo, y.lo);
    s = df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
    return df_fast_two_sum(s.hi, __fadd_rn(s.lo, t.lo));
}
__device__ __forceinline__ df64 operator-(df64 x) { return df64(-x.hi, -x.lo); }
__device__ __forceinline__ df64 operator-(df64 x, df64 y) { return x + (-y); }
__device__ __forceinline__ df64 operator*(df64 x, df64 y)
{
    const float p = __fmul_rn(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.hi, -p);
    e = __fmaf_rn(x.hi, y.lo, e);
    e = __fmaf_rn(x.lo, y.hi, e);
    return df_fast_two_sum(p, e);
}
__device__ __forceinline__ df64 operator/(df64 x, df64 y)
{
    // two quotient digits: q1 from the high parts, q2 from the remainder
    const float q1 = __fdiv_rn(x.hi, y.hi);
    const df64 r = x - y * df64(q1);
    const float q2 = __fdiv_rn(r.hi, y.hi);
    return df_fast_two_sum(q1, q2);
}
__device__ __forceinline__ df64& operator+=(df64& x, df64 y) { x = x + y; return x; }

// Adjoint of the EWA projection for one visible record, in the scalar type
// Rl: conic -> 2D covariance (dSigma = -C dC C, no 1/det cancellation),
// Sigma2D = T S3 T^T with T = J R, J(p) with the frozen guard decisions,
// p = R mu + t, S3 = M M^T with M = Rq diag(s), the quaternion and its
// normalisation; and, if want_cam, the camera gradients pose[8]: the
// left-perturbation pose gradient
// (rho = dL/dp, omega = p x dL/dp + sum_j R_:j x (J^T gT)_:j).  Adds into
// gmu, gls, gq; writes pose.
template <typename Rl>
__device__ __forceinline__ void geom_adjoint(const Chain& f, const Cam& V, float gu, float gv, float gc0, float gc1,
                                             float gc2, float gz, bool want_cam, Rl* gmu, Rl* gls, Rl* gq, Rl* pose)
{
    const Rl two = Rl(2), four = Rl(4), half = Rl(0.5);
    const Rl c0 = f.c0, c1 = f.c1, c2 = f.c2;
    const Rl dgc0 = gc0, dgc1 = gc1, dgc2 = gc2;
    const Rl gS00 = -(dgc0 * c0 * c0 + dgc1 * c0 * c1 + dgc2 * c1 * c1);
    const Rl gS11 = -(dgc0 * c1 * c1 + dgc1 * c1 * c2 + dgc2 * c2 * c2);
    const Rl gS01 = -(two * dgc0 * c0 * c1 + dgc1 * (c0 * c2 + c1 * c1) + two * dgc2 * c1 * c2);
    const Rl Gm[2][2] = {{gS00, half * gS01}, {half * gS01, gS11}};
    Rl T[2][3], S[3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        T[0][i] = f.T[0][i]; T[1][i] = f.T[1][i];
        S[i][0] = f.S[i][0]; S[i][1] = f.S[i][1]; S[i][2] = f.S[i][2];
    }
    Rl gT[2][3], gS3[3][3];
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) {
        const Rl ts0 = T[0][0] * S[0][jj] + T[0][1] * S[1][jj] + T[0][2] * S[2][jj];
        const Rl ts1 = T[1][0] * S[0][jj] + T[1][1] * S[1][jj] + T[1][2] * S[2][jj];
        gT[0][jj] = two * (Gm[0][0] * ts0 + Gm[0][1] * ts1);
        gT[1][jj] = two * (Gm[1][0] * ts0 + Gm[1][1] * ts1);
    }
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int jj = 0; jj < 3; ++jj)
            gS3[i][jj] = T[0][i] * (Gm[0][0] * T[0][jj] + Gm[0][1] * T[1][jj]) +
                         T[1][i] * (Gm[1][0] * T[0][jj] + Gm[1][1] * T[1][jj]);

    // T = J R
    const float* R = V.R;
    Rl gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0;
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) {
        gJ00 += gT[0][jj] * (Rl)R[jj];
        gJ02 += gT[0][jj] * (Rl)R[6 + jj];
        gJ11 += gT[1][jj] * (Rl)R[3 + jj];
        gJ12 += gT[1][jj] * (Rl)R[6 + jj];
    }

    // J(p) with the frozen guard decisions, mean2D and depth
    const Rl x = f.pc[0], y = f.pc[1], z = f.pc[2];
    const Rl fx = V.fx, fy = V.fy;
    const Rl iz = Rl(1) / z, iz2 = iz * iz, iz3 = iz2 * iz;
    Rl gp[3] = {0, 0, 0};
    gp[2] += gJ00 * (-fx * iz2) + gJ11 * (-fy * iz2);
    if (f.clx == 0) { gp[0] += gJ02 * (-fx * iz2); gp[2] += gJ02 * (two * fx * x * iz3); }
    else gp[2] += gJ02 * (fx * (Rl)f.clx * (Rl)f.lx * iz2);
    if (f.cly == 0) { gp[1] += gJ12 * (-fy * iz2); gp[2] += gJ12 * (two * fy * y * iz3); }
    else gp[2] += gJ12 * (fy * (Rl)f.cly * (Rl)f.ly * iz2);
    gp[0] += (Rl)gu * fx * iz;
    gp[1] += (Rl)gv * fy * iz;
    gp[2] += -(Rl)gu * fx * x * iz2 - (Rl)gv * fy * y * iz2 + (Rl)gz;

    // p = R mu + t
#pragma unroll
    for (int jj = 0; jj < 3; ++jj)
        gmu[jj] += (Rl)R[jj] * gp[0] + (Rl)R[3 + jj] * gp[1] + (Rl)R[6 + jj] * gp[2];

    // S3 = M M^T, M = Rq diag(s)
    Rl gRq[3][3];
#pragma unroll
    for (int jj = 0; jj < 3; ++jj) {
        Rl gs = 0;
        const Rl sj = f.s[jj];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            const Rl gM = two * (gS3[i][0] * (Rl)f.M[0][jj] + gS3[i][1] * (Rl)f.M[1][jj] + gS3[i][2] * (Rl)f.M[2][jj]);
            gs += gM * (Rl)f.Rq[i][jj];
            gRq[i][jj] = gM * sj;
        }
        gls[jj] += gs * sj;
    }

    // R(q^), normalisation
    const Rl w = f.qh[0], qa = f.qh[1], qb = f.qh[2], qc = f.qh[3];
    Rl gqh[4];
    gqh[0] = two * (-qc * gRq[0][1] + qb * gRq[0][2] + qc * gRq[1][0] - qa * gRq[1][2] - qb * gRq[2][0] + qa * gRq[2][1]);
    gqh[1] = two * (qb * gRq[0][1] + qc * gRq[0][2] + qb * gRq[1][0] - w * gRq[1][2] + qc * gRq[2][0] + w * gRq[2][1]) -
             four * qa * (gRq[1][1] + gRq[2][2]);
    gqh[2] = two * (qa * gRq[0][1] + w * gRq[0][2] + qa * gRq[1][0] + qc * gRq[1][2] - w * gRq[2][0] + qc * gRq[2][1]) -
             four * qb * (gRq[0][0] + gRq[2][2]);
    gqh[3] = two * (-w * gRq[0][1] + qa * gRq[0][2] + w * gRq[1][0] + qb * gRq[1][2] + qa * gRq[2][0] + qb * gRq[2][1]) -
             four * qc * (gRq[0][0] + gRq[1][1]);
    const Rl qd = w * gqh[0] + qa * gqh[1] + qb * gqh[2] + qc * gqh[3];
    const Rl rn = f.rn;
    gq[0] += (gqh[0] - w * qd) * rn;
    gq[1] += (gqh[1] - qa * qd) * rn;
    gq[2] += (gqh[2] - qb * qd) * rn;
    gq[3] += (gqh[3] - qc * qd) * rn;

    if (want_cam) {
        Rl om[3] = {y * gp[2] - z * gp[1], z * gp[0] - x * gp[2], x * gp[1] - y * gp[0]};
#pragma unroll
        for (int jj = 0; jj < 3; ++jj) {
            const Rl r0 = R[jj], r1 = R[3 + jj], r2 = R[6 + jj];
            const Rl g0 = (Rl)f.J00 * gT[0][jj];
            const Rl g1 = (Rl)f.J11 * gT[1][jj];
            const Rl g2 = (Rl)f.J02 * gT[0][jj] + (Rl)f.J12 * gT[1][jj];
            om[0] += r1 * g2 - r2 * g1;
            om[1] += r2 * g0 - r0 * g2;
            om[2] += r0 * g1 - r1 * g0;
        }
        pose[0] = gp[0]; pose[1] = gp[1]; pose[2] = gp[2];
        pose[3] = om[0]; pose[4] = om[1]; pose[5] = om[2];
        // focal lengths: u = fx x/z + cx, J00 = fx/z, J02 = -fx x~/z^2 (under the
        // frustum guard fx x~ does not depend on fx)
        pose[6] = (Rl)gu * x * iz + gJ00 * iz + (f.clx == 0 ? -gJ02 * x * iz2 : Rl(0));
        pose[7] = (Rl)gv * y * iz + gJ11 * iz + (f.cly == 0 ? -gJ12 * y * iz2 : Rl(0));
    }
}

// Records whose geometry adjoint runs in extended precision (double-float,
// about 48 significant bits).  The binary32 adjoint loses digits where terms
// of the chain cancel, and that happens for Gaussians that are large relative
// to their distance (max scale / z): the 1/z^2 and 1/z^3 terms of J(p) and
// the covariance terms grow together.  Measured against the binary64 oracle on
// the 1M-Gaussian street rig, the binary32 adjoint alone gave 1.3e-3 relative
// L2 on the mean gradients, concentrated in a handful of near-camera
// Gaussians; a binary64 adjoint for the records above 0.1 brought it to 1e-5
// (0.5% of the records), and 0.05 is used here (3.5% of the records) for
// margin; double-float in place of binary64 meets the same bars.
__device__ __forceinline__ bool needs_binary64(const Chain& f)
{
    const float smax = fmaxf(f.s[0], fmaxf(f.s[1], f.s[2]));
    return smax > 0.05f * f.pc[2];
}

// Segmented sum over the warp: after it, the first lane of each segment
// [lane, nxt) holds the segment's sum (steps up to the longest segment).
template <int N>
__device__ __forceinline__ void seg_sum(float (&v)[N], int lane, int nxt, int span)
{
    for (int o = 1; o < span; o <<= 1) {
        const bool take = lane + o < nxt;
#pragma unroll
        for (int c = 0; c < N; ++c) {
            const float t = __shfl_down_sync(0xffffffffu, v[c], o);
            if (take) v[c] += t;
        }
    }
}

// Per-group backward, one thread per visible record of the group.  The
// group's records are Gaussian-major, so the records of one Gaussian are
// consecutive: a segmented reduction over the warp sums each Gaussian's
// partials into the first lane of its segment, which adds them to the
// Gaussian's gradient row -- with a plain read-modify-write when the segment
// lies inside the warp (groups run in stream order and hold each Gaussian
// once), with atomics when it continues into a neighbouring warp.  The 11
// geometry/opacity partials are reduced that way.  The 3K SH partials (the
// basis times the colour gradient) are too in groups of few views (short
// runs); in groups of many views (runs of about ten records on a road batch)
// they are summed transposed, one coefficient pair per lane over the warp's
// records, through a per-warp staging row in shared memory.
constexpr int kTransposedViews = 12;

template <int DEG, bool TRANSPOSED_SH>
__global__ void __launch_bounds__(kPreThreads, 2)
preprocess_bwd_kernel(const __grid_constant__ Table Tb, int gi, PreprocessBwdArgs a)
{
    if (earlier_wait_timed_out(a.status)) return;
    constexpr int K = (DEG + 1) * (DEG + 1);
    // per-warp pose partials: shared atomics then collide only within a warp
    __shared__ float s_pose[kPreThreads / 32][kMaxViews][8];   // pose (6) and focal (2)
    // per warp and lane: the record's SH basis (16) and colour gradient (3, +1);
    // rows of 20 floats, so that the lanes' 16-byte stores fall in distinct
    // bank groups
    __shared__ __align__(16) float s_shb[kPreThreads / 32][32][20];
    __shared__ Cam s_cam[kMaxViews];
    const DevGroup& G = Tb.g[gi];
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    cam_table_fill(s_cam, Tb);
    for (int i = tid; i < (kPreThreads / 32) * kMaxViews * 8; i += kPreThreads) (&s_pose[0][0][0])[i] = 0.0f;
    __syncthreads();
    const bool want_cam = a.grad_pose != nullptr || a.grad_focal != nullptr;
    // Rows are cleared before the first group's launch; a Gaussian appears at
    // most once per group, so in group 0 a segment that stays inside its warp
    // is the only writer of its row (segments across warps add atomically).
    const bool first_group = gi == 0;
    const int64_t kb = a.kstart[G.slot_base], ke = a.kstart[G.slot_base + G.n];

    for (int64_t base = kb + (int64_t)blockIdx.x * kPreThreads; base < ke; base += (int64_t)gridDim.x * kPreThreads) {
        const int64_t k = base + tid;
        const bool has = k < ke;
        uint4 aux = make_uint4(0, 0, 0xffffffffu - lane, 0);
        if (has) aux = a.vis_aux[k];
        const uint32_t j = aux.z;
        float v[11];   // mean 3, log-scale 3, quaternion 4, opacity 1
#pragma unroll
        for (int c = 0; c < 11; ++c) v[c] = 0.0f;
        float dir[3] = {0.0f, 0.0f, 1.0f}, gcol[3] = {0.0f, 0.0f, 0.0f};
        int64_t gauss = 0;
        if (has) {
            const int view = aux_view(aux.w);
            const Cam& V = s_cam[view];
            gauss = G.subset ? (int64_t)G.subset[j] : (int64_t)j;
            float mu[3], ls[3], q[4];
#pragma unroll
            for (int i = 0; i < 3; ++i) { mu[i] = a.means[3 * gauss + i]; ls[i] = a.log_scales[3 * gauss + i]; }
            const float4 q4 = reinterpret_cast<const float4*>(a.quats)[gauss];
            q[0] = q4.x; q[1] = q4.y; q[2] = q4.z; q[3] = q4.w;
            const float* kk = a.sh + (size_t)gauss * K * 3;
            Chain f;
            chain_values(V, mu, ls, q, a.opacity[gauss], aux.w, f);
            const float4 g0 = a.grad_rec[3 * k], g1 = a.grad_rec[3 * k + 1], g2 = a.grad_rec[3 * k + 2];
            gcol[0] = (f.cclamp & 1u) ? 0.0f : g2.x;
            gcol[1] = (f.cclamp & 2u) ? 0.0f : g2.y;
            gcol[2] = (f.cclamp & 4u) ? 0.0f : g2.z;

            // Geometry adjoint.  Records of large angular size go to the
            // extended-precision queue (see needs_binary64); the rest are evaluated here
            // in binary32.
            if (needs_binary64(f)) {
                const unsigned int slot = atomicAdd(a.queue_count, 1u);
                if ((int64_t)slot < a.queue_cap) a.queue[slot] = (uint32_t)k;
                else atomicOr(a.status, kErrInternal);
            } else {
                float pose[8];
                geom_adjoint<float>(f, V, g0.x, g0.y, g0.z * GSR_NHALF_L2E, g0.w * GSR_NL2E, g1.x * GSR_NHALF_L2E,
                                    g1.z, want_cam, v, v + 3, v + 6, pose);
                if (want_cam) {
                    float* sp = s_pose[wid][view - G.first_view];
#pragma unroll
                    for (int c = 0; c < 8; ++c) atomicAdd(sp + c, pose[c]);
                }
            }

            // colour: the viewing direction (Gaussian only), from the SH row
            // read once here; the SH partials basis_i gcol_ch are formed
            // below from the direction
            float wsh[K], gdir[3];
            {
                const bool vec = sh_row_vec<K>(kk);
#pragma unroll
                for (int c0 = 0; c0 < K; c0 += 4) {
                    float kv[12];
                    sh_chunk<K>(kk, c0, vec, kv);
#pragma unroll
                    for (int i = 0; i < 4; ++i)
                        if (c0 + i < K) wsh[c0 + i] = kv[3 * i] * gcol[0] + kv[3 * i + 1] * gcol[1] + kv[3 * i + 2] * gcol[2];
                }
            }
            sh_dir_grad(DEG, f.dir[0], f.dir[1], f.dir[2], wsh, gdir);
            dir[0] = f.dir[0]; dir[1] = f.dir[1]; dir[2] = f.dir[2];
            const float dd = f.dir[0] * gdir[0] + f.dir[1] * gdir[1] + f.dir[2] * gdir[2];
#pragma unroll
            for (int i = 0; i < 3; ++i) v[i] += (gdir[i] - f.dir[i] * dd) * f.idn;
            // opacity
            v[10] = g1.y * f.sig * (1.0f - f.sig);
        }

        // segments of equal j (lanes without a record have unique sentinels)
        const uint32_t jprev = __shfl_up_sync(0xffffffffu, j, 1);
        const bool head = lane == 0 || jprev != j;
        const uint32_t heads = __ballot_sync(0xffffffffu, head);
        const uint32_t after = lane < 31 ? heads >> (lane + 1) : 0u;
        const int nxt = after ? lane + __ffs(after) : 32;       // first lane of the next segment
        int span = head ? nxt - lane : 0;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) span = max(span, __shfl_xor_sync(0xffffffffu, span, o));
        // does the Gaussian continue into the previous or the next warp?
        bool shared_seg = false, cont_prev = false;
        if (head && has) {
            if (lane == 0 && k > kb) cont_prev = a.vis_aux[k - 1].z == j;
            const int64_t klast = k + (nxt - 1 - lane);
            shared_seg = cont_prev;
            if (nxt == 32 && klast + 1 < ke) shared_seg = shared_seg || a.vis_aux[klast + 1].z == j;
        }
        const bool writer = head && has;
        // rows written: one per Gaussian of this group (its first segment)
        const uint32_t firsts = __ballot_sync(0xffffffffu, writer && !cont_prev);
        if (lane == 0 && firsts) atomicAdd(a.grad_rows, (unsigned long long)__popc(firsts));

        seg_sum(v, lane, nxt, span);
        if (writer) {
            float* gm = a.grad_means + 3 * gauss;
            float* gl = a.grad_log_scales + 3 * gauss;
            float* gq = a.grad_quats + 4 * gauss;
            if (shared_seg) {
#pragma unroll
                for (int i = 0; i < 3; ++i) { atomicAdd(gm + i, v[i]); atomicAdd(gl + i, v[3 + i]); }
#pragma unroll
                for (int i = 0; i < 4; ++i) atomicAdd(gq + i, v[6 + i]);
                atomicAdd(a.grad_opacity + gauss, v[10]);
            } else if (first_group) {
                // the first group to reach the row: a plain store (no read)
#pragma unroll
                for (int i = 0; i < 3; ++i) { gm[i] = v[i]; gl[i] = v[3 + i]; }
                *reinterpret_cast<float4*>(gq) = make_float4(v[6], v[7], v[8], v[9]);
                a.grad_opacity[gauss] = v[10];
            } else {
#pragma unroll
                for (int i = 0; i < 3; ++i) { gm[i] += v[i]; gl[i] += v[3 + i]; }
                float4 o4 = *reinterpret_cast<float4*>(gq);
                o4.x += v[6]; o4.y += v[7]; o4.z += v[8]; o4.w += v[9];
                *reinterpret_cast<float4*>(gq) = o4;
                a.grad_opacity[gauss] += v[10];
            }
        }
        if constexpr (TRANSPOSED_SH) {
            // SH gradients, transposed: every lane stages its record's basis (the
            // same binary32 values as the forward's) and colour gradient, then the
            // warp walks its 32 records in order with lane l accumulating
            // coefficients l and l + 32 of the 3K-float row (coefficient f / 3,
            // channel f % 3) and writes them at each segment's end: one coalesced
            // row write per Gaussian instead of per-lane segmented sums of 3K values.
            {
                float basis[16];
                sh_basis(DEG, dir[0], dir[1], dir[2], basis);
#pragma unroll
                for (int i = K; i < 16; ++i) basis[i] = 0.0f;
                float4* sb = reinterpret_cast<float4*>(s_shb[wid][lane]);
                sb[0] = make_float4(basis[0], basis[1], basis[2], basis[3]);
                sb[1] = make_float4(basis[4], basis[5], basis[6], basis[7]);
                sb[2] = make_float4(basis[8], basis[9], basis[10], basis[11]);
                sb[3] = make_float4(basis[12], basis[13], basis[14], basis[15]);
                sb[4] = make_float4(gcol[0], gcol[1], gcol[2], 0.0f);
            }
            __syncwarp();
            {
                const uint32_t wmask = __ballot_sync(0xffffffffu, writer);
                const uint32_t smask = __ballot_sync(0xffffffffu, writer && shared_seg);
                const uint32_t ends = (heads >> 1) | 0x80000000u;   // last lane of each segment
                const uint32_t glo = (uint32_t)gauss, ghi = (uint32_t)((uint64_t)gauss >> 32);
                const int f1 = lane, f2 = lane + 32;
                const bool has1 = f1 < 3 * K, has2 = f2 < 3 * K;
                const int i1 = min(f1 / 3, K - 1), c1 = f1 % 3;
                const int i2 = min(f2 / 3, K - 1), c2 = f2 % 3;
                float acc1 = 0.0f, acc2 = 0.0f;
#pragma unroll
                for (int r = 0; r < 32; ++r) {
                    const float* row = s_shb[wid][r];
                    acc1 = fmaf(row[i1], row[16 + c1], acc1);
                    acc2 = fmaf(row[i2], row[16 + c2], acc2);
                    if ((ends >> r) & 1u) {
                        // the segment [h, r]: written if its head holds a record
                        const int h = 31 - __clz(heads & (0xffffffffu >> (31 - r)));
                        if ((wmask >> h) & 1u) {
                            const uint32_t lo = __shfl_sync(0xffffffffu, glo, r), hi = __shfl_sync(0xffffffffu, ghi, r);
                            float* gs = a.grad_sh + (size_t)(((uint64_t)hi << 32) | lo) * K * 3;
                            // the first group's own rows: plain stores; otherwise
                            // reductions (fire-and-forget: a read-modify-write here
                            // would wait out one memory round trip per segment)
                            if (first_group && !((smask >> h) & 1u)) {
                                if (has1) gs[f1] = acc1;
                                if (has2) gs[f2] = acc2;
                            } else {
                                if (has1) atomicAdd(gs + f1, acc1);
                                if (has2) atomicAdd(gs + f2, acc2);
                            }
                        }
                        acc1 = 0.0f;
                        acc2 = 0.0f;
                    }
                }
            }
            __syncwarp();   // the staging rows are rewritten by the next pass
        } else {
            // short runs (few views per group): segmented warp sums in chunks of
            // four coefficients regenerated from the basis
            float* gs = a.grad_sh + (size_t)gauss * K * 3;
            const bool gvec = sh_row_vec<K>(gs);
            // the basis regenerated from the direction (the same binary32 values as
            // the forward's); only the chunk's coefficients stay live
            float basis[16];
            sh_basis(DEG, dir[0], dir[1], dir[2], basis);
#pragma unroll
            for (int c0 = 0; c0 < K; c0 += 4) {
                constexpr int C = K < 4 ? K : 4;
                float u[3 * C];
#pragma unroll
                for (int i = 0; i < C; ++i)
#pragma unroll
                    for (int ch = 0; ch < 3; ++ch) u[3 * i + ch] = c0 + i < K ? basis[c0 + i] * gcol[ch] : 0.0f;
                seg_sum(u, lane, nxt, span);
                if constexpr (K % 4 == 0) {
                    if (writer && gvec) {
                        // whole chunks of a 16-byte aligned row: three 16-byte accesses
                        float4* p = reinterpret_cast<float4*>(gs + 3 * c0);
                        const float4 d0 = make_float4(u[0], u[1], u[2], u[3]);
                        const float4 d1 = make_float4(u[4], u[5], u[6], u[7]);
                        const float4 d2 = make_float4(u[8], u[9], u[10], u[11]);
                        if (shared_seg) {
                            atomicAdd(p, d0);
                            atomicAdd(p + 1, d1);
                            atomicAdd(p + 2, d2);
                        } else if (first_group) {
                            p[0] = d0; p[1] = d1; p[2] = d2;
                        } else {
                            float4 o0 = p[0], o1 = p[1], o2 = p[2];
                            o0.x += d0.x; o0.y += d0.y; o0.z += d0.z; o0.w += d0.w;
                            o1.x += d1.x; o1.y += d1.y; o1.z += d1.z; o1.w += d1.w;
                            o2.x += d2.x; o2.y += d2.y; o2.z += d2.z; o2.w += d2.w;
                            p[0] = o0; p[1] = o1; p[2] = o2;
                        }
                        continue;
                    }
                }
                if (writer) {
                    // (the last chunk may be short: K = 9 at degree 2)
                    if (shared_seg) {
#pragma unroll
                        for (int i = 0; i < 3 * C; ++i)
                            if (3 * c0 + i < 3 * K) atomicAdd(gs + 3 * c0 + i, u[i]);
                    } else if (first_group) {
#pragma unroll
                        for (int i = 0; i < 3 * C; ++i)
                            if (3 * c0 + i < 3 * K) gs[3 * c0 + i] = u[i];
                    } else {
#pragma unroll
                        for (int i = 0; i < 3 * C; ++i)
                            if (3 * c0 + i < 3 * K) gs[3 * c0 + i] += u[i];
                    }
                }
            }
        }
    }
    if (want_cam) {
        __syncthreads();
        for (int i = tid; i < G.nv * 8; i += kPreThreads) {
            const int vl = i / 8, c = i % 8;
            double acc = 0.0;
#pragma unroll
            for (int w = 0; w < kPreThreads / 32; ++w) acc += (double)s_pose[w][vl][c];
            const float pv = (float)acc;
            if (pv == 0.0f) continue;
            if (c < 6 && a.grad_pose) atomicAdd(a.grad_pose + (size_t)(G.first_view + vl) * 6 + c, pv);
            if (c >= 6 && a.grad_focal) atomicAdd(a.grad_focal + (size_t)(G.first_view + vl) * 2 + (c - 6), pv);
        }
    }
}

// The queued records (double-float geometry adjoint), after every group pass:
// the contributions are added with atomics on top of the groups' sums.  Two
// blocks per SM (128 registers, an 8-byte spill): at the 172 registers it
// takes unbounded, one block per SM left the dependent double-float chains
// eight warps to hide their latency.
__global__ void __launch_bounds__(kPreThreads, 2)
preprocess_bwd64_kernel(const __grid_constant__ Table Tb, PreprocessBwdArgs a)
{
    if (earlier_wait_timed_out(a.status)) return;
    __shared__ double s_pose[kPreThreads / 32][kMaxViews][8];   // per warp, as above
    __shared__ Cam s_cam[kMaxViews];
    const int tid = threadIdx.x, wid = tid >> 5;
    cam_table_fill(s_cam, Tb);
    for (int i = tid; i < (kPreThreads / 32) * kMaxViews * 8; i += kPreThreads) (&s_pose[0][0][0])[i] = 0.0;
    const bool want_cam = a.grad_pose != nullptr || a.grad_focal != nullptr;
    __syncthreads();
    const unsigned int qn = *a.queue_count;
    const int64_t nq = (int64_t)qn < a.queue_cap ? (int64_t)qn : a.queue_cap;
    for (int64_t q = (int64_t)blockIdx.x * kPreThreads + tid; q < nq; q += (int64_t)gridDim.x * kPreThreads) {
        const uint32_t k = a.queue[q];
        const uint4 aux = a.vis_aux[k];
        const int view = aux_view(aux.w);
        const Cam& V = s_cam[view];
        const DevGroup& G = Tb.g[V.group];
        const int64_t gauss = G.subset ? (int64_t)G.subset[aux.z] : (int64_t)aux.z;
        float mu[3], ls[3], qq[4];
#pragma unroll
        for (int i = 0; i < 3; ++i) { mu[i] = a.means[3 * gauss + i]; ls[i] = a.log_scales[3 * gauss + i]; }
        const float4 q4 = reinterpret_cast<const float4*>(a.quats)[gauss];
        qq[0] = q4.x; qq[1] = q4.y; qq[2] = q4.z; qq[3] = q4.w;
        Chain f;
        chain_values(V, mu, ls, qq, a.opacity[gauss], aux.w, f);
        const float4 g0 = a.grad_rec[3 * (size_t)k], g1 = a.grad_rec[3 * (size_t)k + 1];
        df64 gmu[3] = {0, 0, 0}, gls[3] = {0, 0, 0}, gq[4] = {0, 0, 0, 0}, pose[8];
        geom_adjoint<df64>(f, V, g0.x, g0.y, g0.z * GSR_NHALF_L2E, g0.w * GSR_NL2E, g1.x * GSR_NHALF_L2E, g1.z,
                           want_cam, gmu, gls, gq, pose);
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            atomicAdd(a.grad_means + 3 * gauss + i, (float)gmu[i]);
            atomicAdd(a.grad_log_scales + 3 * gauss + i, (float)gls[i]);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) atomicAdd(a.grad_quats + 4 * gauss + i, (float)gq[i]);
        if (want_cam) {
#pragma unroll
            for (int c = 0; c < 8; ++c) atomicAdd(&s_pose[wid][view][c], (double)pose[c]);
        }
    }
    if (want_cam) {
        __syncthreads();
        for (int i = tid; i < Tb.n_views * 8; i += kPreThreads) {
            const int vw = i / 8, c = i % 8;
            double acc = 0.0;
#pragma unroll
            for (int w = 0; w < kPreThreads / 32; ++w) acc += s_pose[w][vw][c];
            const float v = (float)acc;
            if (v == 0.0f) continue;
            if (c < 6 && a.grad_pose) atomicAdd(a.grad_pose + (size_t)vw * 6 + c, v);
            if (c >= 6 && a.grad_focal) atomicAdd(a.grad_focal + (size_t)vw * 2 + (c - 6), v);
        }
    }
}

void launch_preprocess_bwd64(const Table& T, const PreprocessBwdArgs& a, int num_sms, cudaStream_t s)
{
    if (a.queue_cap <= 0) return;
    int64_t blocks = (a.queue_cap + kPreThreads - 1) / kPreThreads;
    if (blocks > (int64_t)num_sms * 2) blocks = (int64_t)num_sms * 2;
    GSR_COUNT_LAUNCH();
    preprocess_bwd64_kernel<<<(unsigned)blocks, kPreThreads, 0, s>>>(T, a);
}

// Rig chain (Sec. 3.1, 3.3).  V_i = A_i V_m(k): a left perturbation delta of
// the central pose reaches view i as Ad(A_i) delta, so the central gradient
// is Ad(A_i)^T g_i = (R^T g_rho, R^T (g_omega - t x g_rho)); a left
// perturbation of A_c reaches each of its views unchanged.  One thread per
// output component, summing in binary64 over the views in ascending order.
constexpr int kRigThreads = kMaxViews * 14;   // 6 central + 6 relative + 2 focal per index
__global__ void __launch_bounds__(kRigThreads)
rig_chain_kernel(const __grid_constant__ RigTable T, const float* __restrict__ pose_grads,
                 const float* __restrict__ focal_grads, float* __restrict__ central, float* __restrict__ camera_rel,
                 float* __restrict__ camera_focal)
{
    const int t = threadIdx.x;
    if (t < kMaxViews * 6) {
        const int k = t / 6, c = t % 6;
        if (!central || k >= T.n_keyframes) return;
        double acc = 0.0;
        for (int i = 0; i < T.n_views; ++i) {
            if (T.kf[i] != k) continue;
            const float* g = pose_grads + (size_t)i * 6;
            const float* A = T.rel[i];
            const double gr[3] = {g[0], g[1], g[2]};
            double w[3];
            if (c < 3) {
                w[0] = gr[0]; w[1] = gr[1]; w[2] = gr[2];
            } else {
                const double tx = A[3], ty = A[7], tz = A[11];
                w[0] = (double)g[3] - (ty * gr[2] - tz * gr[1]);
                w[1] = (double)g[4] - (tz * gr[0] - tx * gr[2]);
                w[2] = (double)g[5] - (tx * gr[1] - ty * gr[0]);
            }
            const int col = c % 3;   // (R^T w)_col = sum_r R[r][col] w_r
            acc += (double)A[col] * w[0] + (double)A[4 + col] * w[1] + (double)A[8 + col] * w[2];
        }
        central[k * 6 + c] = (float)acc;
    } else if (t < kMaxViews * 12) {
        const int u = t - kMaxViews * 6, cam = u / 6, c = u % 6;
        if (!camera_rel || cam >= T.n_cameras) return;
        double acc = 0.0;
        for (int i = 0; i < T.n_views; ++i)
            if (T.cam[i] == cam) acc += (double)pose_grads[(size_t)i * 6 + c];
        camera_rel[cam * 6 + c] = (float)acc;
    } else {
        const int u = t - kMaxViews * 12, cam = u / 2, c = u % 2;
        if (!camera_focal || cam >= T.n_cameras) return;
        double acc = 0.0;
        for (int i = 0; i < T.n_views; ++i)
            if (T.cam[i] == cam) acc += (double)focal_grads[(size_t)i * 2 + c];
        camera_focal[cam * 2 + c] = (float)acc;
    }
}

void launch_rig_chain(const RigTable& T, const float* pose_grads, const float* focal_grads, float* central,
                      float* camera_rel, float* camera_focal, cudaStream_t s)
{
    GSR_COUNT_LAUNCH();
    rig_chain_kernel<<<1, kRigThreads, 0, s>>>(T, pose_grads, focal_grads, central, camera_rel, camera_focal);
}

// Persistent grid: one resident wave, each block taking tickets of 256 sub records.
template <int DEG>
static void pre_fwd_launch(const Table& T, const PreprocessArgs& a, int64_t blocks, int num_sms, cudaStream_t s)
{
    static std::atomic<int> per_sm_dev[kMaxDevices];
    const int per_sm = per_device_once(per_sm_dev, [] {
        int n = 0;
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, preprocess_fwd_kernel<DEG>, kPreThreads, 0);
        return n < 1 ? 1 : n;
    });
    const int64_t grid = blocks < (int64_t)num_sms * per_sm ? blocks : (int64_t)num_sms * per_sm;
    preprocess_fwd_kernel<DEG><<<(unsigned)grid, kPreThreads, 0, s>>>(T, a);
}

static int preprocess_sub(const Table& T, int num_sms);

void launch_preprocess_fwd(const Table& T, const PreprocessArgs& a, int num_sms, cudaStream_t s)
{
    PreprocessArgs b = a;
    b.sub = preprocess_sub(T, num_sms);
    const int64_t blocks = (T.n_records + (int64_t)kPreThreads * b.sub - 1) / ((int64_t)kPreThreads * b.sub);   // tickets
    if (blocks == 0) return;
    GSR_COUNT_LAUNCH();
    switch (T.sh_degree) {
    case 0: pre_fwd_launch<0>(T, b, blocks, num_sms, s); break;
    case 1: pre_fwd_launch<1>(T, b, blocks, num_sms, s); break;
    case 2: pre_fwd_launch<2>(T, b, blocks, num_sms, s); break;
    default: pre_fwd_launch<3>(T, b, blocks, num_sms, s); break;
    }
}

void launch_preprocess_bwd(const Table& T, int group, const PreprocessBwdArgs& a, int num_sms, cudaStream_t s)
{
    // grid-stride over the group's visible records (their count is on the device)
    const int64_t n = T.g[group].n * (int64_t)T.g[group].nv;
    int64_t blocks = (n + kPreThreads - 1) / kPreThreads;
    if (blocks > (int64_t)num_sms * 2) blocks = (int64_t)num_sms * 2;
    if (blocks == 0) return;
    GSR_COUNT_LAUNCH();
    // Long runs of records per Gaussian (groups of many views) sum the SH
    // partials transposed; short runs keep the segmented warp sums, which then
    // cost fewer steps than the transposed walk over all 32 records.
    if (T.g[group].nv >= kTransposedViews) {
        switch (T.sh_degree) {
        case 0: preprocess_bwd_kernel<0, true><<<(unsigned)blocks, kPreThreads, 0, s>>>(T, group, a); break;
        case 1: preprocess_bwd_kernel<1, true><<<(unsigned)blocks, kPreThreads, 0, s>>>(T, group, a); break;
        case 2: preprocess_bwd_kernel<2, true><<<(unsigned)blocks, kPreThreads, 0, s>>>(T, group, a); break;
        default: preprocess_bwd_kernel<3, true><<<(unsigned)blocks, kPreThreads, 0, s>>>(T, group, a); break;
        }
    } else {
        switch (T.sh_degree) {
        case 0: preprocess_bwd_kernel<0, false><<<(unsigned)blocks, kPreThreads, 0, s>>>(T, group, a); break;
        case 1: preprocess_bwd_kernel<1, false><<<(unsigned)blocks, kPreThreads, 0, s>>>(T, group, a); break;
        case 2: preprocess_bwd_kernel<2, false><<<(unsigned)blocks, kPreThreads, 0, s>>>(T, group, a); break;
        default: preprocess_bwd_kernel<3, false><<<(unsigned)blocks, kPreThreads, 0, s>>>(T, group, a); break;
        }
    }
}

int64_t preprocess_blocks(const Table& T) { return (T.n_records + kPreThreads - 1) / kPreThreads; }

// Records per thread: the largest of 8, 4, 2, 1 that still gives two
// resident waves of tickets (a ticket's work runs on one block).
static int preprocess_sub(const Table& T, int num_sms)
{
    const int64_t want = (int64_t)num_sms * 3 * 2;
    int sub = kPreSub;
    while (sub > 1 && (T.n_records + (int64_t)kPreThreads * sub - 1) / ((int64_t)kPreThreads * sub) < want) sub >>= 1;
    return sub;
}

}  // namespace gsr
