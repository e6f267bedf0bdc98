/*
 * gsr_oracle.c -- CPU reference of the differentiable tile-based Gaussian
 * splatting rasterizer (3DGS, cited by the paper as the renderer it optimises
 * in Sec. 3.3 "Optimization": Gaussians and camera poses updated jointly, SH
 * gradients detached for the camera update).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links or calls this
 * file; only the tests, the package smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code, header or constant table with the CUDA
 * library: every formula below is written out here from the definition.
 *
 * Two layers:
 *
 *   1. The binary32 decision mirror.  Every discrete result of the renderer
 *      (near cull, determinant cull, screen radius, tile rectangle, the 64-bit
 *      (view, tile, depth) sort key, the alpha-clamp / 1/255-skip / 1e-4-stop
 *      decisions of the blend, the colour clamp) is a function of binary32
 *      arithmetic.  The mirror evaluates those quantities in binary32 with a
 *      fixed, documented operation order (fmaf where a fused multiply-add is
 *      written, every other operation rounded to nearest), so that a GPU
 *      implementation following the same order reproduces the decisions bit
 *      for bit.  The exponentials are this project's own binary32 routines
 *      (Cody-Waite argument reduction followed by a degree-7 Taylor
 *      polynomial), not a C library function.
 *
 *   2. The FP64 value path.  Images and gradients are computed in double
 *      precision, taking every discrete decision from the mirror ("decisions
 *      in the kernel's precision, values exact").  The backward pass is the
 *      exact adjoint of the forward with those decisions frozen, including the
 *      se(3) camera-pose gradient under a left perturbation exp(delta^) V with
 *      the SH viewing direction held constant for the pose.
 *
 * Compile with -ffp-contract=off (no implicit fusion) and without fast-math.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_API __attribute__((visibility("default")))

/* ------------------------------------------------------------------------- */
/* binary32 helpers                                                           */
/* ------------------------------------------------------------------------- */

static inline float u2f(uint32_t b) { float f; memcpy(&f, &b, 4); return f; }
static inline uint32_t f2u(float f) { uint32_t b; memcpy(&b, &f, 4); return b; }

/* 2^y in binary32.  y is clamped to [-126, 127]; n = round-to-nearest-even(y)
 * by adding and subtracting 1.5*2^23; f = y - n is exact and |f| <= 1/2;
 * 2^f = exp(f ln 2) by the degree-7 Taylor polynomial with coefficients
 * (ln 2)^k / k! rounded to binary32, evaluated by Horner's rule with fmaf; the
 * result is scaled by 2^n built directly from exponent bits. */
ORC_API float orc_exp2_f32(float y)
{
    y = fmaxf(y, -126.0f);
    y = fminf(y, 127.0f);
    float j = y + 0x1.8p23f;
    float nf = j - 0x1.8p23f;
    float f = y - nf;
    float p = 0x1.ffcbfcp-17f;           /* ln2^7/7! */
    p = fmaf(p, f, 0x1.430912p-13f);     /* ln2^6/6! */
    p = fmaf(p, f, 0x1.5d87fep-10f);     /* ln2^5/5! */
    p = fmaf(p, f, 0x1.3b2ab6p-7f);      /* ln2^4/4! */
    p = fmaf(p, f, 0x1.c6b08ep-5f);      /* ln2^3/3! */
    p = fmaf(p, f, 0x1.ebfbe0p-3f);      /* ln2^2/2! */
    p = fmaf(p, f, 0x1.62e430p-1f);      /* ln2     */
    p = fmaf(p, f, 1.0f);
    int n = (int)nf;
    return p * u2f((uint32_t)(n + 127) << 23);
}

/* e^x in binary32.  x is clamped to [-87, 88]; n = nearest integer to
 * x*log2(e) (fused, 1.5*2^23 shifter); r = x - n*ln2 in two Cody-Waite steps
 * (ln2 split into a binary32 head and tail); e^r by the degree-7 Taylor
 * polynomial (coefficients 1/k! rounded to binary32), Horner with fmaf;
 * scaled by 2^n from exponent bits. */
ORC_API float orc_exp_f32(float x)
{
    x = fmaxf(x, -87.0f);
    x = fminf(x, 88.0f);
    float j = fmaf(x, 0x1.715476p+0f, 0x1.8p23f);
    float nf = j - 0x1.8p23f;
    float r = fmaf(nf, -0x1.62e430p-1f, x);
    r = fmaf(nf, 0x1.05c610p-29f, r);    /* -(ln2 tail); the tail is negative */
    float p = 0x1.a01a02p-13f;           /* 1/7! */
    p = fmaf(p, r, 0x1.6c16c2p-10f);     /* 1/6! */
    p = fmaf(p, r, 0x1.111112p-7f);      /* 1/5! */
    p = fmaf(p, r, 0x1.555556p-5f);      /* 1/4! */
    p = fmaf(p, r, 0x1.555556p-3f);      /* 1/3! */
    p = fmaf(p, r, 0.5f);
    p = fmaf(p, r, 1.0f);
    p = fmaf(p, r, 1.0f);
    int n = (int)nf;
    return p * u2f((uint32_t)(n + 127) << 23);
}

/* Real spherical-harmonic constants, l <= 3, from the normalisation formulas
 * sqrt((2l+1)/(4 pi) * (l-|m|)!/(l+|m|)!) (times sqrt 2 for m != 0); the sign
 * convention carries the Condon-Shortley factor (-1)^m, basis order
 * m = -l .. l within each band. */
#define SH_C0   0.28209479177387814   /* 1/(2 sqrt(pi))          */
#define SH_C1   0.4886025119029199    /* sqrt(3/(4 pi))          */
#define SH_C2A  1.0925484305920792    /* sqrt(15/pi)/2           */
#define SH_C2B  0.31539156525252005   /* sqrt(5/pi)/4            */
#define SH_C2C  0.5462742152960396    /* sqrt(15/pi)/4           */
#define SH_C3A  0.5900435899266435    /* sqrt(35/(2 pi))/4       */
#define SH_C3B  2.890611442640554     /* sqrt(105/pi)/2          */
#define SH_C3C  0.4570457994644658    /* sqrt(21/(2 pi))/4       */
#define SH_C3D  0.3731763325901154    /* sqrt(7/pi)/4            */
#define SH_C3E  1.445305721320277     /* sqrt(105/pi)/4          */

/* binary32 basis, fixed operation order (the mirror's contract) */
ORC_API void orc_sh_basis_f32(int degree, float x, float y, float z, float* b)
{
    b[0] = (float)SH_C0;
    if (degree < 1) return;
    b[1] = (float)(-SH_C1) * y;
    b[2] = (float)SH_C1 * z;
    b[3] = (float)(-SH_C1) * x;
    if (degree < 2) return;
    float xx = x * x, yy = y * y, zz = z * z;
    float xy = x * y, yz = y * z, xz = x * z;
    b[4] = (float)SH_C2A * xy;
    b[5] = (float)(-SH_C2A) * yz;
    b[6] = (float)SH_C2B * ((2.0f * zz - xx) - yy);
    b[7] = (float)(-SH_C2A) * xz;
    b[8] = (float)SH_C2C * (xx - yy);
    if (degree < 3) return;
    b[9]  = ((float)(-SH_C3A) * y) * ((3.0f * xx) - yy);
    b[10] = ((float)SH_C3B * xy) * z;
    b[11] = ((float)(-SH_C3C) * y) * (((4.0f * zz) - xx) - yy);
    b[12] = ((float)SH_C3D * z) * (((2.0f * zz) - (3.0f * xx)) - (3.0f * yy));
    b[13] = ((float)(-SH_C3C) * x) * (((4.0f * zz) - xx) - yy);
    b[14] = ((float)SH_C3E * z) * (xx - yy);
    b[15] = ((float)(-SH_C3A) * x) * (xx - (3.0f * yy));
}

/* FP64 basis and its Jacobian d b_i / d(x, y, z) (for the direction path). */
ORC_API void orc_sh_basis_f64(int degree, double x, double y, double z, double* b, double* db /* [16][3] or NULL */)
{
    int K = (degree + 1) * (degree + 1);
    if (db) memset(db, 0, sizeof(double) * 3 * K);
    b[0] = SH_C0;
    if (degree < 1) return;
    b[1] = -SH_C1 * y;  b[2] = SH_C1 * z;  b[3] = -SH_C1 * x;
    if (db) { db[1*3+1] = -SH_C1; db[2*3+2] = SH_C1; db[3*3+0] = -SH_C1; }
    if (degree < 2) return;
    double xx = x * x, yy = y * y, zz = z * z;
    b[4] = SH_C2A * x * y;
    b[5] = -SH_C2A * y * z;
    b[6] = SH_C2B * (2 * zz - xx - yy);
    b[7] = -SH_C2A * x * z;
    b[8] = SH_C2C * (xx - yy);
    if (db) {
        db[4*3+0] = SH_C2A * y;  db[4*3+1] = SH_C2A * x;
        db[5*3+1] = -SH_C2A * z; db[5*3+2] = -SH_C2A * y;
        db[6*3+0] = -2 * SH_C2B * x; db[6*3+1] = -2 * SH_C2B * y; db[6*3+2] = 4 * SH_C2B * z;
        db[7*3+0] = -SH_C2A * z; db[7*3+2] = -SH_C2A * x;
        db[8*3+0] = 2 * SH_C2C * x; db[8*3+1] = -2 * SH_C2C * y;
    }
    if (degree < 3) return;
    b[9]  = -SH_C3A * y * (3 * xx - yy);
    b[10] = SH_C3B * x * y * z;
    b[11] = -SH_C3C * y * (4 * zz - xx - yy);
    b[12] = SH_C3D * z * (2 * zz - 3 * xx - 3 * yy);
    b[13] = -SH_C3C * x * (4 * zz - xx - yy);
    b[14] = SH_C3E * z * (xx - yy);
    b[15] = -SH_C3A * x * (xx - 3 * yy);
    if (db) {
        db[9*3+0] = -SH_C3A * 6 * x * y;
        db[9*3+1] = -SH_C3A * (3 * xx - 3 * yy);
        db[10*3+0] = SH_C3B * y * z; db[10*3+1] = SH_C3B * x * z; db[10*3+2] = SH_C3B * x * y;
        db[11*3+0] = -SH_C3C * (-2 * x * y);
        db[11*3+1] = -SH_C3C * (4 * zz - xx - 3 * yy);
        db[11*3+2] = -SH_C3C * (8 * y * z);
        db[12*3+0] = SH_C3D * (-6 * x * z);
        db[12*3+1] = SH_C3D * (-6 * y * z);
        db[12*3+2] = SH_C3D * (6 * zz - 3 * xx - 3 * yy);
        db[13*3+0] = -SH_C3C * (4 * zz - 3 * xx - yy);
        db[13*3+1] = -SH_C3C * (-2 * x * y);
        db[13*3+2] = -SH_C3C * (8 * x * z);
        db[14*3+0] = SH_C3E * 2 * x * z;
        db[14*3+1] = -SH_C3E * 2 * y * z;
        db[14*3+2] = SH_C3E * (xx - yy);
        db[15*3+0] = -SH_C3A * (3 * xx - 3 * yy);
        db[15*3+1] = -SH_C3A * (-6 * x * y);
    }
}

/* ------------------------------------------------------------------------- */
/* scene description shared by the entry points                               */
/* ------------------------------------------------------------------------- */

typedef struct {
    int64_t n;                 /* Gaussians */
    int sh_degree;
    const float* means;        /* [n][3] binary32 inputs for the mirror */
    const float* log_scales;   /* [n][3] */
    const float* quats;        /* [n][4] (w, x, y, z) */
    const float* opac;         /* [n] */
    const float* sh;           /* [n][K][3] */
    const double* means64;     /* same parameters in double for the value path (may be perturbed) */
    const double* log_scales64;
    const double* quats64;
    const double* opac64;
    const double* sh64;
    int nv;                    /* views */
    const int32_t* wh;         /* [nv][2] width, height */
    const float* intr;         /* [nv][4] fx, fy, cx, cy */
    const float* viewmats;     /* [nv][16] row-major world-to-camera (binary32, for the mirror) */
    const double* viewmats64;  /* [nv][16] for the value path (may be perturbed) */
    const double* campos64;    /* [nv][3] SH camera centre override, or NULL = -R^T t of viewmats64 */
    const uint32_t* subset_data;
    const int64_t* subset_off; /* [nv] offset into subset_data, or -1 = all n Gaussians */
    const int64_t* counts;     /* [nv] records per view */
    int tile_w, tile_h;
    float near_plane;
    double bg[3];
    const double* intr64;      /* [nv][4] intrinsics for the value path (may be perturbed), or NULL = intr */
} orc_scene;

/* decision mirror, one entry per (view, record) */
typedef struct {
    uint32_t* flags;   /* bit0 culled; bit1/bit2 guard clamp x low/high; bit3/bit4 y low/high; bit5..7 colour clamp */
    uint32_t* zbits;   /* binary32 bits of camera-space z */
    int32_t* radius;
    int32_t* rect;     /* [4] x0, y0, x1, y1 (tile units, half open) */
    int32_t* tiles;
    float* blend;      /* [6] u, v, qa, qb, qc, sigma: the blend's binary32 inputs */
    float* colour;     /* [3] */
    float* conic;      /* [3] c0, c1, c2 (binary32) */
} orc_mirror;

#define F_CULLED 1u
#define F_CLX_LO 2u
#define F_CLX_HI 4u
#define F_CLY_LO 8u
#define F_CLY_HI 16u
#define F_CCLAMP0 32u

static int64_t rec_base_of(const orc_scene* s, int v)
{
    int64_t b = 0;
    for (int w = 0; w < v; ++w) b += s->counts[w];
    return b;
}

static int64_t total_records(const orc_scene* s) { return rec_base_of(s, s->nv); }

static inline int tiles_x(const orc_scene* s, int v) { return (s->wh[2*v] + s->tile_w - 1) / s->tile_w; }
static inline int tiles_y(const orc_scene* s, int v) { return (s->wh[2*v+1] + s->tile_h - 1) / s->tile_h; }

static int64_t tile_base_of(const orc_scene* s, int v)
{
    int64_t b = 0;
    for (int w = 0; w < v; ++w) b += (int64_t)tiles_x(s, w) * tiles_y(s, w);
    return b;
}

static inline int64_t gaussian_of(const orc_scene* s, int v, int64_t j)
{
    return s->subset_off[v] < 0 ? j : (int64_t)s->subset_data[s->subset_off[v] + j];
}

/* ------------------------------------------------------------------------- */
/* 1. binary32 decision mirror of the preprocess step                         */
/* ------------------------------------------------------------------------- */

static void mirror_one(const orc_scene* s, int v, int64_t g, int64_t r, orc_mirror* m)
{
    const float* V = s->viewmats + 16 * v;
    const float R[3][3] = {{V[0], V[1], V[2]}, {V[4], V[5], V[6]}, {V[8], V[9], V[10]}};
    const float t[3] = {V[3], V[7], V[11]};
    const float fx = s->intr[4*v], fy = s->intr[4*v+1], cx = s->intr[4*v+2], cy = s->intr[4*v+3];
    const int W = s->wh[2*v], H = s->wh[2*v+1];
    const int TX = tiles_x(s, v), TY = tiles_y(s, v);
    const float* mu = s->means + 3 * g;
    uint32_t flags = 0;

    m->tiles[r] = 0; m->radius[r] = 0;
    for (int k = 0; k < 4; ++k) m->rect[4*r+k] = 0;
    for (int k = 0; k < 6; ++k) m->blend[6*r+k] = 0.0f;
    for (int k = 0; k < 3; ++k) { m->colour[3*r+k] = 0.0f; m->conic[3*r+k] = 0.0f; }

    /* camera-space position */
    float pc[3];
    for (int i = 0; i < 3; ++i)
        pc[i] = fmaf(R[i][0], mu[0], fmaf(R[i][1], mu[1], fmaf(R[i][2], mu[2], t[i])));
    const float x = pc[0], y = pc[1], z = pc[2];
    m->zbits[r] = f2u(z);
    if (!(z > s->near_plane)) { m->flags[r] = F_CULLED; return; }

    /* scales and normalised quaternion */
    const float* ls = s->log_scales + 3 * g;
    float sc[3] = {orc_exp_f32(ls[0]), orc_exp_f32(ls[1]), orc_exp_f32(ls[2])};
    const float* q = s->quats + 4 * g;
    float n2 = fmaf(q[0], q[0], fmaf(q[1], q[1], fmaf(q[2], q[2], q[3] * q[3])));
    if (!(n2 > 0.0f)) { m->flags[r] = F_CULLED; return; }
    float rn = 1.0f / sqrtf(n2);
    float qw = q[0] * rn, qx = q[1] * rn, qy = q[2] * rn, qz = q[3] * rn;

    float xx = qx * qx, yy = qy * qy, zz = qz * qz;
    float xy = qx * qy, xz = qx * qz, yz = qy * qz;
    float wx = qw * qx, wy = qw * qy, wz = qw * qz;
    float Rq[3][3];
    Rq[0][0] = fmaf(-2.0f, yy + zz, 1.0f);
    Rq[0][1] = 2.0f * (xy - wz);
    Rq[0][2] = 2.0f * (xz + wy);
    Rq[1][0] = 2.0f * (xy + wz);
    Rq[1][1] = fmaf(-2.0f, xx + zz, 1.0f);
    Rq[1][2] = 2.0f * (yz - wx);
    Rq[2][0] = 2.0f * (xz - wy);
    Rq[2][1] = 2.0f * (yz + wx);
    Rq[2][2] = fmaf(-2.0f, xx + yy, 1.0f);

    float M[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) M[i][j] = Rq[i][j] * sc[j];
    float S[3][3];
    for (int i = 0; i < 3; ++i)
        for (int j = i; j < 3; ++j) {
            S[i][j] = fmaf(M[i][0], M[j][0], fmaf(M[i][1], M[j][1], M[i][2] * M[j][2]));
            S[j][i] = S[i][j];
        }

    /* EWA Jacobian with the frustum guard */
    const float lx = 1.3f * (fmaxf(cx, (float)W - cx) / fx);
    const float ly = 1.3f * (fmaxf(cy, (float)H - cy) / fy);
    const float iz = 1.0f / z;
    const float xr = x * iz, yr = y * iz;
    if (xr < -lx) flags |= F_CLX_LO;
    if (xr > lx) flags |= F_CLX_HI;
    if (yr < -ly) flags |= F_CLY_LO;
    if (yr > ly) flags |= F_CLY_HI;
    const float tx = z * fminf(lx, fmaxf(-lx, xr));
    const float ty = z * fminf(ly, fmaxf(-ly, yr));
    const float iz2 = iz * iz;
    const float J00 = fx * iz, J02 = -((fx * tx) * iz2);
    const float J11 = fy * iz, J12 = -((fy * ty) * iz2);

    float T[2][3];
    for (int j = 0; j < 3; ++j) {
        T[0][j] = fmaf(J00, R[0][j], J02 * R[2][j]);
        T[1][j] = fmaf(J11, R[1][j], J12 * R[2][j]);
    }
    float U[2][3];
    for (int i = 0; i < 2; ++i)
        for (int j = 0; j < 3; ++j)
            U[i][j] = fmaf(T[i][0], S[0][j], fmaf(T[i][1], S[1][j], T[i][2] * S[2][j]));
    float a = fmaf(U[0][0], T[0][0], fmaf(U[0][1], T[0][1], U[0][2] * T[0][2])) + 0.3f;
    float b = fmaf(U[0][0], T[1][0], fmaf(U[0][1], T[1][1], U[0][2] * T[1][2]));
    float c = fmaf(U[1][0], T[1][0], fmaf(U[1][1], T[1][1], U[1][2] * T[1][2])) + 0.3f;

    float det = fmaf(a, c, -(b * b));
    if (!(det > 0.0f)) { m->flags[r] = F_CULLED | flags; return; }
    float idet = 1.0f / det;
    float c0 = c * idet, c1 = -(b * idet), c2 = a * idet;

    float u = fmaf(fx * x, iz, cx);
    float vv = fmaf(fy * y, iz, cy);

    /* screen radius: 3 sqrt of the larger eigenvalue, lower discriminant 0.1 */
    float mid = 0.5f * (a + c);
    float lam = mid + sqrtf(fmaxf(0.1f, fmaf(mid, mid, -det)));
    float rad = ceilf(3.0f * sqrtf(lam));

    /* tile rectangle, half open, clamped to the view's tile grid */
    const float bxf = (float)s->tile_w, byf = (float)s->tile_h;
    int x0 = (int)fminf(fmaxf((u - rad) / bxf, 0.0f), (float)TX);
    int x1 = (int)fminf(fmaxf(((u + rad) + (bxf - 1.0f)) / bxf, 0.0f), (float)TX);
    int y0 = (int)fminf(fmaxf((vv - rad) / byf, 0.0f), (float)TY);
    int y1 = (int)fminf(fmaxf(((vv + rad) + (byf - 1.0f)) / byf, 0.0f), (float)TY);
    int tiles = (x1 - x0) * (y1 - y0);
    m->radius[r] = (int32_t)rad;
    m->rect[4*r] = x0; m->rect[4*r+1] = y0; m->rect[4*r+2] = x1; m->rect[4*r+3] = y1;
    if (tiles == 0) { m->flags[r] = F_CULLED | flags; return; }
    m->tiles[r] = tiles;

    /* opacity */
    float sig = 1.0f / (1.0f + orc_exp_f32(-s->opac[g]));

    /* colour from SH along the camera-centre -> mean direction */
    float cp[3];
    for (int j = 0; j < 3; ++j)
        cp[j] = -fmaf(R[0][j], t[0], fmaf(R[1][j], t[1], R[2][j] * t[2]));
    float d0 = mu[0] - cp[0], d1 = mu[1] - cp[1], d2 = mu[2] - cp[2];
    float dn = sqrtf(fmaf(d0, d0, fmaf(d1, d1, d2 * d2)));
    float idn = 1.0f / dn;
    float bs[16];
    orc_sh_basis_f32(s->sh_degree, d0 * idn, d1 * idn, d2 * idn, bs);
    const int K = (s->sh_degree + 1) * (s->sh_degree + 1);
    const float* kk = s->sh + (size_t)g * K * 3;
    for (int ch = 0; ch < 3; ++ch) {
        float acc = bs[0] * kk[ch];
        for (int i = 1; i < K; ++i) acc = fmaf(bs[i], kk[3*i+ch], acc);
        float col = acc + 0.5f;
        if (col < 0.0f) { flags |= (F_CCLAMP0 << ch); col = 0.0f; }
        m->colour[3*r+ch] = col;
    }

    m->conic[3*r] = c0; m->conic[3*r+1] = c1; m->conic[3*r+2] = c2;
    float* bl = m->blend + 6 * r;
    bl[0] = u; bl[1] = vv;
    bl[2] = c0 * -0x1.715476p-1f;   /* -log2(e)/2 */
    bl[3] = c1 * -0x1.715476p+0f;   /* -log2(e)   */
    bl[4] = c2 * -0x1.715476p-1f;
    bl[5] = sig;
    m->flags[r] = flags;
}

ORC_API int orc_mirror_preprocess(const orc_scene* s, orc_mirror* m)
{
    for (int v = 0; v < s->nv; ++v) {
        const int64_t base = rec_base_of(s, v);
        const int64_t cnt = s->counts[v];
        #pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < cnt; ++j) mirror_one(s, v, gaussian_of(s, v, j), base + j, m);
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 2. tile lists: 64-bit keys (global tile << 32 | depth bits), sorted ranges */
/* ------------------------------------------------------------------------- */

/*
 * The list of a tile is every record that is not culled and whose tile
 * rectangle (the 3-sigma screen radius, Sec. 3.3 renders with the 3DGS tile
 * rasterizer) holds the tile, ordered by the binary32 bits of its camera-space
 * depth and, for equal depths, by record index.  Nothing else removes an
 * entry: a renderer may list fewer records as long as each pixel still
 * composites the same records in the same order (the tests check a GPU's
 * shorter lists against these with orc_tile_reach below).
 */

typedef struct { uint64_t key; uint32_t val; } orc_pair;

static int cmp_pair(const void* a, const void* b)
{
    const orc_pair* x = (const orc_pair*)a;
    const orc_pair* y = (const orc_pair*)b;
    if (x->key != y->key) return x->key < y->key ? -1 : 1;
    if (x->val != y->val) return x->val < y->val ? -1 : 1;
    return 0;
}

/* Instances whose global tile is selected by mask (NULL = every tile). */
ORC_API int64_t orc_count_instances(const orc_scene* s, const orc_mirror* m, const uint8_t* mask)
{
    int64_t total = 0;
    for (int v = 0; v < s->nv; ++v) {
        const int64_t rb = rec_base_of(s, v), tb = tile_base_of(s, v);
        const int TX = tiles_x(s, v);
        for (int64_t j = 0; j < s->counts[v]; ++j) {
            const int64_t r = rb + j;
            if (m->flags[r] & F_CULLED) continue;
            const int32_t* rc = m->rect + 4 * r;
            for (int ty = rc[1]; ty < rc[3]; ++ty)
                for (int tx = rc[0]; tx < rc[2]; ++tx)
                    total += !mask || mask[tb + (int64_t)ty * TX + tx];
        }
    }
    return total;
}

/* The sorted lists restricted to the tiles selected by mask (NULL = all):
 * keys/vals: M entries (M = orc_count_instances); ranges: [total tiles][2],
 * (0, 0) for unselected or empty tiles. */
ORC_API int orc_build_lists_masked(const orc_scene* s, const orc_mirror* m, const uint8_t* mask, int64_t M,
                                   uint64_t* keys, uint32_t* vals, uint32_t* ranges)
{
    orc_pair* P = (orc_pair*)malloc(sizeof(orc_pair) * (size_t)(M > 0 ? M : 1));
    if (!P) return 1;
    int64_t w = 0;
    for (int v = 0; v < s->nv; ++v) {
        const int64_t rb = rec_base_of(s, v), tb = tile_base_of(s, v);
        const int TX = tiles_x(s, v);
        for (int64_t j = 0; j < s->counts[v]; ++j) {
            const int64_t r = rb + j;
            if (m->flags[r] & F_CULLED) continue;
            const int32_t* rc = m->rect + 4 * r;
            for (int ty = rc[1]; ty < rc[3]; ++ty)
                for (int tx = rc[0]; tx < rc[2]; ++tx) {
                    const int64_t gt = tb + (int64_t)ty * TX + tx;
                    if (mask && !mask[gt]) continue;
                    if (w >= M) { free(P); return 2; }
                    P[w].key = ((uint64_t)gt << 32) | (uint64_t)m->zbits[r];
                    P[w].val = (uint32_t)r;
                    ++w;
                }
        }
    }
    if (w != M) { free(P); return 3; }
    qsort(P, (size_t)M, sizeof(orc_pair), cmp_pair);
    const int64_t nt = tile_base_of(s, s->nv);
    memset(ranges, 0, sizeof(uint32_t) * 2 * (size_t)nt);
    for (int64_t i = 0; i < M; ++i) {
        keys[i] = P[i].key;
        vals[i] = P[i].val;
        const uint64_t t = P[i].key >> 32;
        if (i == 0 || (P[i-1].key >> 32) != t) ranges[2*t] = (uint32_t)i;
        if (i == M - 1 || (P[i+1].key >> 32) != t) ranges[2*t+1] = (uint32_t)(i + 1);
    }
    free(P);
    return 0;
}

/* keys/vals: M entries (M = sum of tiles); ranges: [total tiles][2]. */
ORC_API int orc_build_lists(const orc_scene* s, const orc_mirror* m, int64_t M,
                            uint64_t* keys, uint32_t* vals, uint32_t* ranges)
{
    return orc_build_lists_masked(s, m, NULL, M, keys, vals, ranges);
}

/* ------------------------------------------------------------------------- */
/* 3. FP64 preprocess (values), decisions taken from the mirror               */
/* ------------------------------------------------------------------------- */

/* per record: u, v, c0, c1, c2, sigma, r, g, b, z */
#define R64 10

typedef struct {
    /* forward intermediates needed by the adjoint */
    double R[3][3], t[3], p[3], s[3], qn, qh[4], Rq[3][3], M[3][3], S3[3][3];
    double J00, J02, J11, J12, T[2][3], S2[3], det;
    double u, v, c[3], sig, col[3], dir[3], dn, bsh[16], z;
    int clx, cly;         /* -1, 0, +1 */
    double lx, ly;
    uint32_t flags;
} orc_fwd64;

static void pre64(const orc_scene* s, int v, int64_t g, uint32_t flags, orc_fwd64* f)
{
    const double* V = s->viewmats64 + 16 * v;
    for (int i = 0; i < 3; ++i) { for (int j = 0; j < 3; ++j) f->R[i][j] = V[4*i+j]; f->t[i] = V[4*i+3]; }
    const double* in = s->intr64 ? s->intr64 + 4 * v : NULL;
    const double fx = in ? in[0] : s->intr[4*v], fy = in ? in[1] : s->intr[4*v+1];
    const double cx = in ? in[2] : s->intr[4*v+2], cy = in ? in[3] : s->intr[4*v+3];
    const double W = s->wh[2*v], H = s->wh[2*v+1];
    const double* mu = s->means64 + 3 * g;
    f->flags = flags;
    for (int i = 0; i < 3; ++i)
        f->p[i] = f->R[i][0] * mu[0] + f->R[i][1] * mu[1] + f->R[i][2] * mu[2] + f->t[i];
    const double x = f->p[0], y = f->p[1], z = f->p[2];
    f->z = z;
    const double* ls = s->log_scales64 + 3 * g;
    for (int i = 0; i < 3; ++i) f->s[i] = exp(ls[i]);
    const double* q = s->quats64 + 4 * g;
    f->qn = sqrt(q[0]*q[0] + q[1]*q[1] + q[2]*q[2] + q[3]*q[3]);
    for (int i = 0; i < 4; ++i) f->qh[i] = q[i] / f->qn;
    const double w = f->qh[0], a = f->qh[1], b = f->qh[2], c = f->qh[3];
    f->Rq[0][0] = 1 - 2*(b*b + c*c); f->Rq[0][1] = 2*(a*b - w*c);     f->Rq[0][2] = 2*(a*c + w*b);
    f->Rq[1][0] = 2*(a*b + w*c);     f->Rq[1][1] = 1 - 2*(a*a + c*c); f->Rq[1][2] = 2*(b*c - w*a);
    f->Rq[2][0] = 2*(a*c - w*b);     f->Rq[2][1] = 2*(b*c + w*a);     f->Rq[2][2] = 1 - 2*(a*a + b*b);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) f->M[i][j] = f->Rq[i][j] * f->s[j];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j)
        f->S3[i][j] = f->M[i][0]*f->M[j][0] + f->M[i][1]*f->M[j][1] + f->M[i][2]*f->M[j][2];

    f->lx = 1.3 * fmax(cx, W - cx) / fx;
    f->ly = 1.3 * fmax(cy, H - cy) / fy;
    f->clx = (flags & F_CLX_LO) ? -1 : (flags & F_CLX_HI) ? 1 : 0;
    f->cly = (flags & F_CLY_LO) ? -1 : (flags & F_CLY_HI) ? 1 : 0;
    const double xt = f->clx ? f->clx * f->lx * z : x;
    const double yt = f->cly ? f->cly * f->ly * z : y;
    f->J00 = fx / z; f->J02 = -fx * xt / (z * z);
    f->J11 = fy / z; f->J12 = -fy * yt / (z * z);
    for (int j = 0; j < 3; ++j) {
        f->T[0][j] = f->J00 * f->R[0][j] + f->J02 * f->R[2][j];
        f->T[1][j] = f->J11 * f->R[1][j] + f->J12 * f->R[2][j];
    }
    double TS[2][3];
    for (int i = 0; i < 2; ++i) for (int j = 0; j < 3; ++j)
        TS[i][j] = f->T[i][0]*f->S3[0][j] + f->T[i][1]*f->S3[1][j] + f->T[i][2]*f->S3[2][j];
    f->S2[0] = TS[0][0]*f->T[0][0] + TS[0][1]*f->T[0][1] + TS[0][2]*f->T[0][2] + 0.3;
    f->S2[1] = TS[0][0]*f->T[1][0] + TS[0][1]*f->T[1][1] + TS[0][2]*f->T[1][2];
    f->S2[2] = TS[1][0]*f->T[1][0] + TS[1][1]*f->T[1][1] + TS[1][2]*f->T[1][2] + 0.3;
    f->det = f->S2[0] * f->S2[2] - f->S2[1] * f->S2[1];
    f->c[0] = f->S2[2] / f->det;
    f->c[1] = -f->S2[1] / f->det;
    f->c[2] = f->S2[0] / f->det;
    f->u = fx * x / z + cx;
    f->v = fy * y / z + cy;
    f->sig = 1.0 / (1.0 + exp(-s->opac64[g]));

    double cp[3];
    if (s->campos64) { for (int j = 0; j < 3; ++j) cp[j] = s->campos64[3*v+j]; }
    else for (int j = 0; j < 3; ++j) cp[j] = -(f->R[0][j]*f->t[0] + f->R[1][j]*f->t[1] + f->R[2][j]*f->t[2]);
    double d[3] = {mu[0] - cp[0], mu[1] - cp[1], mu[2] - cp[2]};
    f->dn = sqrt(d[0]*d[0] + d[1]*d[1] + d[2]*d[2]);
    for (int j = 0; j < 3; ++j) f->dir[j] = d[j] / f->dn;
    orc_sh_basis_f64(s->sh_degree, f->dir[0], f->dir[1], f->dir[2], f->bsh, NULL);
    const int K = (s->sh_degree + 1) * (s->sh_degree + 1);
    const double* kk = s->sh64 + (size_t)g * K * 3;
    for (int ch = 0; ch < 3; ++ch) {
        double acc = 0.5;
        for (int i = 0; i < K; ++i) acc += f->bsh[i] * kk[3*i+ch];
        f->col[ch] = (flags & (F_CCLAMP0 << ch)) ? 0.0 : acc;
    }
}

/* rec64: [N_vg][R64].  Culled records are zero. */
ORC_API int orc_preprocess64(const orc_scene* s, const orc_mirror* m, double* rec64)
{
    for (int v = 0; v < s->nv; ++v) {
        const int64_t base = rec_base_of(s, v);
        #pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < s->counts[v]; ++j) {
            const int64_t r = base + j;
            double* o = rec64 + R64 * r;
            if (m->flags[r] & F_CULLED) { for (int k = 0; k < R64; ++k) o[k] = 0.0; continue; }
            orc_fwd64 f;
            pre64(s, v, gaussian_of(s, v, j), m->flags[r], &f);
            o[0] = f.u; o[1] = f.v; o[2] = f.c[0]; o[3] = f.c[1]; o[4] = f.c[2];
            o[5] = f.sig; o[6] = f.col[0]; o[7] = f.col[1]; o[8] = f.col[2]; o[9] = f.z;
        }
    }
    return 0;
}

/* FP64 screen radius and tile rectangle from the FP64 covariance, for the
 * decision cross-check (mirror vs. double precision).  out: [N_vg][6] =
 * radius, x0, y0, x1, y1, tiles (0 for mirror-culled records). */
ORC_API int orc_rect64(const orc_scene* s, const orc_mirror* m, int32_t* out)
{
    for (int v = 0; v < s->nv; ++v) {
        const int64_t base = rec_base_of(s, v);
        const int TX = tiles_x(s, v), TY = tiles_y(s, v);
        #pragma omp parallel for schedule(static)
        for (int64_t j = 0; j < s->counts[v]; ++j) {
            const int64_t r = base + j;
            int32_t* o = out + 6 * r;
            for (int k = 0; k < 6; ++k) o[k] = 0;
            if (m->flags[r] & F_CULLED) continue;
            orc_fwd64 f;
            pre64(s, v, gaussian_of(s, v, j), m->flags[r], &f);
            double mid = 0.5 * (f.S2[0] + f.S2[2]);
            double lam = mid + sqrt(fmax(0.1, mid * mid - f.det));
            double rad = ceil(3.0 * sqrt(lam));
            double bx = s->tile_w, by = s->tile_h;
            int x0 = (int)fmin(fmax((f.u - rad) / bx, 0.0), TX);
            int x1 = (int)fmin(fmax((f.u + rad + bx - 1) / bx, 0.0), TX);
            int y0 = (int)fmin(fmax((f.v - rad) / by, 0.0), TY);
            int y1 = (int)fmin(fmax((f.v + rad + by - 1) / by, 0.0), TY);
            o[0] = (int32_t)rad; o[1] = x0; o[2] = y0; o[3] = x1; o[4] = y1; o[5] = (x1 - x0) * (y1 - y0);
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 4. per-pixel compositing                                                   */
/* ------------------------------------------------------------------------- */

typedef struct { int view, x0, y0, w, h; } orc_block;

typedef struct {
    const uint32_t* vals;    /* sorted record indices */
    const uint32_t* ranges;  /* [tiles][2] */
    int brute;               /* 1: ignore the lists, walk every non-culled record of the view */
    int decide64;            /* 1: take the blend decisions in double precision instead of the mirror */
} orc_lists;

typedef struct { int64_t rec; double alpha, G, dx, dy; int clamped; } orc_entry;

#define ALPHA_MAX_F 0x1.fae148p-1f   /* 0.99  */
#define ALPHA_MIN_F 0x1.010102p-8f   /* 1/255 */
#define T_STOP_F    0x1.a36e2ep-14f  /* 1e-4  */

/* Brute-force list for one pixel: all non-culled records of view v whose tile
 * rectangle contains the pixel's tile (brute = 1), or every non-culled record
 * of the view (brute = 2), ordered by (depth bits, record index). */
typedef struct { uint32_t zb; uint32_t r; } orc_zr;
static int cmp_zr(const void* a, const void* b)
{
    const orc_zr* x = (const orc_zr*)a; const orc_zr* y = (const orc_zr*)b;
    if (x->zb != y->zb) return x->zb < y->zb ? -1 : 1;
    return x->r < y->r ? -1 : (x->r > y->r);
}

/* The blend's per-entry test at pixel centre (pxf, pyf), in binary32
 * (Sec. 3.3's renderer; the thresholds 0.99, 1/255 and 1e-4 of the 3DGS
 * blend): the form P2 = log2(e) * P at the pixel offset, skipped if P2 > 0;
 * alpha = min(0.99, sigma 2^P2); the entry composites only if alpha >= 1/255.
 * Returns 1 if it passes, with *alpha and *clamped set. */
static int blend_test_f32(const float* bl, float pxf, float pyf, float* alpha, int* clamped)
{
    const float fdx = pxf - bl[0], fdy = pyf - bl[1];
    const float P2 = fmaf(fdx, fmaf(bl[2], fdx, bl[3] * fdy), (bl[4] * fdy) * fdy);
    if (P2 > 0.0f) return 0;
    const float sa = bl[5] * orc_exp2_f32(P2);
    *alpha = fminf(ALPHA_MAX_F, sa);
    *clamped = !(sa < ALPHA_MAX_F);
    return *alpha >= ALPHA_MIN_F;
}

/* Walk the list of pixel (px, py) of view v front to back.  Writes the
 * blended entries to ent (capacity cap), returns their number; *ncontrib =
 * list position of the last blended entry + 1; *nexam = entries examined;
 * *stoprec = the record at which the walk stopped (transmittance would fall
 * below 1e-4), or UINT32_MAX if it reached the end of the list. */
static int walk_pixel(const orc_scene* s, const orc_mirror* m, const double* rec64, const orc_lists* L,
                      int v, int px, int py, orc_entry* ent, int64_t cap, orc_zr* scratch,
                      uint32_t* ncontrib, uint32_t* nexam, uint32_t* stoprec)
{
    const int TX = tiles_x(s, v);
    const int tx = px / s->tile_w, ty = py / s->tile_h;
    const int64_t gt = tile_base_of(s, v) + (int64_t)ty * TX + tx;
    int64_t start, end;
    const uint32_t* list;
    if (L->brute) {
        const int64_t rb = rec_base_of(s, v);
        int64_t n = 0;
        for (int64_t j = 0; j < s->counts[v]; ++j) {
            const int64_t r = rb + j;
            if (m->flags[r] & F_CULLED) continue;
            const int32_t* rc = m->rect + 4 * r;
            if (L->brute == 1 && !(tx >= rc[0] && tx < rc[2] && ty >= rc[1] && ty < rc[3]))
                continue;
            scratch[n].zb = m->zbits[r]; scratch[n].r = (uint32_t)r; ++n;
        }
        qsort(scratch, (size_t)n, sizeof(orc_zr), cmp_zr);
        start = 0; end = n; list = NULL;
    } else {
        start = L->ranges[2*gt]; end = L->ranges[2*gt+1]; list = L->vals;
    }
    const float pxf = (float)px + 0.5f, pyf = (float)py + 0.5f;
    const double pxd = px + 0.5, pyd = py + 0.5;
    float T32 = 1.0f;
    double T64 = 1.0;
    int nb = 0;
    uint32_t last = 0, exam = 0;
    *stoprec = UINT32_MAX;
    for (int64_t k = start; k < end; ++k) {
        const int64_t r = list ? (int64_t)list[k] : (int64_t)scratch[k].r;
        exam = (uint32_t)(k - start + 1);
        const double* o = rec64 + R64 * r;
        const double dx = pxd - o[0], dy = pyd - o[1];
        const double P = -0.5 * (o[2] * dx * dx + o[4] * dy * dy) - o[3] * dx * dy;
        const double G = exp(P);
        int clamped;
        if (L->decide64) {
            double a = o[5] * G;
            clamped = !(a < 0.99);
            if (clamped) a = 0.99;
            if (a < 1.0 / 255.0) continue;
            double Tn = T64 * (1.0 - a);
            if (Tn < 1e-4) { *stoprec = (uint32_t)r; break; }
            T64 = Tn;
        } else {
            float a;
            if (!blend_test_f32(m->blend + 6 * r, pxf, pyf, &a, &clamped)) continue;
            const float Tn = T32 * (1.0f - a);
            if (Tn < T_STOP_F) { *stoprec = (uint32_t)r; break; }
            T32 = Tn;
        }
        if (nb < cap) {
            ent[nb].rec = r; ent[nb].G = G; ent[nb].dx = dx; ent[nb].dy = dy; ent[nb].clamped = clamped;
            ent[nb].alpha = clamped ? 0.99 : o[5] * G;
        }
        ++nb;
        last = (uint32_t)(k - start + 1);
    }
    *ncontrib = last;
    *nexam = exam;
    return nb;
}

/* For each entry k of the lists (every tile's range), reach[k] = 1 iff the
 * record passes the blend's test (blend_test_f32) at one or more pixel
 * centres of its tile that lie inside the view, by brute force over the
 * tile's pixels.  An entry with reach 0 composites at no pixel and stops no
 * pixel's walk, so a list without it composites the same records in the same
 * order; reach 1 entries must stay in any such list.  reach: [M]. */
ORC_API int orc_tile_reach(const orc_scene* s, const orc_mirror* m, const orc_lists* L, int64_t M, uint8_t* reach)
{
    memset(reach, 0, (size_t)(M > 0 ? M : 0));
    for (int v = 0; v < s->nv; ++v) {
        const int TX = tiles_x(s, v), TY = tiles_y(s, v);
        const int W = s->wh[2*v], H = s->wh[2*v+1];
        const int64_t tb = tile_base_of(s, v);
        #pragma omp parallel for schedule(dynamic, 4)
        for (int64_t t = 0; t < (int64_t)TX * TY; ++t) {
            const int tx = (int)(t % TX), ty = (int)(t / TX);
            const int x0 = tx * s->tile_w, y0 = ty * s->tile_h;
            const int x1 = x0 + s->tile_w < W ? x0 + s->tile_w : W;
            const int y1 = y0 + s->tile_h < H ? y0 + s->tile_h : H;
            const uint32_t a = L->ranges[2*(tb + t)], b = L->ranges[2*(tb + t) + 1];
            for (uint32_t k = a; k < b && (int64_t)k < M; ++k) {
                const float* bl = m->blend + 6 * (int64_t)L->vals[k];
                int hit = 0;
                for (int py = y0; py < y1 && !hit; ++py)
                    for (int px = x0; px < x1 && !hit; ++px) {
                        float al; int cl;
                        hit = blend_test_f32(bl, (float)px + 0.5f, (float)py + 0.5f, &al, &cl);
                    }
                reach[k] = (uint8_t)hit;
            }
        }
    }
    return 0;
}

static int64_t max_list_len(const orc_scene* s, const orc_lists* L)
{
    int64_t mx = 1;
    if (L->brute) { for (int v = 0; v < s->nv; ++v) if (s->counts[v] > mx) mx = s->counts[v]; return mx; }
    const int64_t nt = tile_base_of(s, s->nv);
    for (int64_t t = 0; t < nt; ++t) { int64_t l = (int64_t)L->ranges[2*t+1] - L->ranges[2*t]; if (l > mx) mx = l; }
    return mx;
}

static int64_t block_pixels(const orc_block* b, int nb)
{
    int64_t n = 0;
    for (int i = 0; i < nb; ++i) n += (int64_t)b[i].w * b[i].h;
    return n;
}

/* Outputs are compact per block, blocks concatenated: rgb [3][h][w] per
 * block, depth/alpha/tfinal/ncontrib/nexam/nblend/stoprec [h][w] per block
 * (nblend: entries composited; stoprec: see walk_pixel; both may be NULL). */
ORC_API int orc_forward(const orc_scene* s, const orc_mirror* m, const double* rec64, const orc_lists* L,
                        const orc_block* blocks, int nblocks,
                        double* rgb, double* depth, double* alpha, double* tfinal,
                        uint32_t* ncontrib, uint32_t* nexam, uint32_t* nblend, uint32_t* stoprec)
{
    const int64_t cap = max_list_len(s, L);
    int64_t off = 0;
    for (int bi = 0; bi < nblocks; ++bi) {
        const orc_block B = blocks[bi];
        const int64_t np = (int64_t)B.w * B.h;
        #pragma omp parallel
        {
            orc_entry* ent = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)cap);
            orc_zr* scr = L->brute ? (orc_zr*)malloc(sizeof(orc_zr) * (size_t)cap) : NULL;
            #pragma omp for schedule(dynamic, 16)
            for (int64_t i = 0; i < np; ++i) {
                const int px = B.x0 + (int)(i % B.w), py = B.y0 + (int)(i / B.w);
                uint32_t nc, ne, sr;
                const int nbl = walk_pixel(s, m, rec64, L, B.view, px, py, ent, cap, scr, &nc, &ne, &sr);
                double T = 1.0, C[3] = {0, 0, 0}, D = 0.0;
                for (int k = 0; k < nbl; ++k) {
                    const double* o = rec64 + R64 * ent[k].rec;
                    const double w = ent[k].alpha * T;
                    for (int ch = 0; ch < 3; ++ch) C[ch] += o[6+ch] * w;
                    D += o[9] * w;
                    T *= 1.0 - ent[k].alpha;
                }
                for (int ch = 0; ch < 3; ++ch) rgb[3*off + ch*np + i] = C[ch] + T * s->bg[ch];
                depth[off + i] = D;
                alpha[off + i] = 1.0 - T;
                tfinal[off + i] = T;
                ncontrib[off + i] = nc;
                nexam[off + i] = ne;
                if (nblend) nblend[off + i] = (uint32_t)nbl;
                if (stoprec) stoprec[off + i] = sr;
            }
            free(ent); free(scr);
        }
        off += np;
    }
    return 0;
}

/* ------------------------------------------------------------------------- */
/* 5. backward: blend adjoint (back to front) and preprocess adjoint          */
/* ------------------------------------------------------------------------- */

/* per-record 2D gradient: du, dv, dc0, dc1, dc2, dsigma, dr, dg, db, dz */
#define G2 10

static inline void atomic_add(double* p, double v)
{
    #pragma omp atomic
    *p += v;
}

static void blend_backward(const orc_scene* s, const orc_mirror* m, const double* rec64, const orc_lists* L,
                           const orc_block* blocks, int nblocks,
                           const double* dl_rgb, const double* dl_depth, const double* dl_alpha, double* grec)
{
    const int64_t cap = max_list_len(s, L);
    int64_t off = 0;
    for (int bi = 0; bi < nblocks; ++bi) {
        const orc_block B = blocks[bi];
        const int64_t np = (int64_t)B.w * B.h;
        #pragma omp parallel
        {
            orc_entry* ent = (orc_entry*)malloc(sizeof(orc_entry) * (size_t)cap);
            double* Tb = (double*)malloc(sizeof(double) * (size_t)cap);
            orc_zr* scr = L->brute ? (orc_zr*)malloc(sizeof(orc_zr) * (size_t)cap) : NULL;
            #pragma omp for schedule(dynamic, 16)
            for (int64_t i = 0; i < np; ++i) {
                const int px = B.x0 + (int)(i % B.w), py = B.y0 + (int)(i / B.w);
                const double dC[3] = {dl_rgb[3*off + i], dl_rgb[3*off + np + i], dl_rgb[3*off + 2*np + i]};
                const double dD = dl_depth ? dl_depth[off + i] : 0.0;
                const double dA = dl_alpha ? dl_alpha[off + i] : 0.0;
                uint32_t nc, ne, sr;
                const int nbl = walk_pixel(s, m, rec64, L, B.view, px, py, ent, cap, scr, &nc, &ne, &sr);
                double T = 1.0;
                for (int k = 0; k < nbl; ++k) { Tb[k] = T; T *= 1.0 - ent[k].alpha; }
                const double Tf = T;
                double SC[3] = {Tf * s->bg[0], Tf * s->bg[1], Tf * s->bg[2]}, SD = 0.0;
                for (int k = nbl - 1; k >= 0; --k) {
                    const orc_entry* e = ent + k;
                    const double* o = rec64 + R64 * e->rec;
                    const double a = e->alpha, Tk = Tb[k], om = 1.0 - a;
                    double ga = dA * Tf / om;
                    for (int ch = 0; ch < 3; ++ch) ga += dC[ch] * (o[6+ch] * Tk - SC[ch] / om);
                    ga += dD * (o[9] * Tk - SD / om);
                    double* gr = grec + G2 * e->rec;
                    for (int ch = 0; ch < 3; ++ch) atomic_add(gr + 6 + ch, dC[ch] * a * Tk);
                    atomic_add(gr + 9, dD * a * Tk);
                    if (!e->clamped) {
                        const double dP = ga * a;
                        atomic_add(gr + 5, ga * e->G);
                        atomic_add(gr + 0, dP * (o[2] * e->dx + o[3] * e->dy));
                        atomic_add(gr + 1, dP * (o[3] * e->dx + o[4] * e->dy));
                        atomic_add(gr + 2, dP * (-0.5 * e->dx * e->dx));
                        atomic_add(gr + 3, dP * (-e->dx * e->dy));
                        atomic_add(gr + 4, dP * (-0.5 * e->dy * e->dy));
                    }
                    for (int ch = 0; ch < 3; ++ch) SC[ch] += o[6+ch] * a * Tk;
                    SD += o[9] * a * Tk;
                }
            }
            free(ent); free(Tb); free(scr);
        }
        off += np;
    }
}

static inline void cross3(const double* a, const double* b, double* o)
{
    o[0] = a[1]*b[2] - a[2]*b[1];
    o[1] = a[2]*b[0] - a[0]*b[2];
    o[2] = a[0]*b[1] - a[1]*b[0];
}

/* Adjoint of pre64 for one record.  g: the record's 2D gradient.  Adds to the
 * Gaussian's parameter gradients and to the view's gpose[8]: pose (rho, omega)
 * and focal lengths (fx, fy). */
static void pre64_backward(const orc_scene* s, int v, int64_t g, const orc_fwd64* f, const double* gr,
                           double* gm, double* gl, double* gq, double* go, double* gsh, double* gpose)
{
    const double fx = s->intr64 ? s->intr64[4*v] : s->intr[4*v];
    const double fy = s->intr64 ? s->intr64[4*v+1] : s->intr[4*v+1];
    const int K = (s->sh_degree + 1) * (s->sh_degree + 1);
    const double x = f->p[0], y = f->p[1], z = f->p[2];
    double gmu[3] = {0, 0, 0};

    /* colour: SH coefficients and the viewing direction (Gaussian only) */
    double gcol[3];
    for (int ch = 0; ch < 3; ++ch) gcol[ch] = (f->flags & (F_CCLAMP0 << ch)) ? 0.0 : gr[6+ch];
    double bsh[16], dbsh[48];
    orc_sh_basis_f64(s->sh_degree, f->dir[0], f->dir[1], f->dir[2], bsh, dbsh);
    const double* kk = s->sh64 + (size_t)g * K * 3;
    double gdir[3] = {0, 0, 0};
    for (int i = 0; i < K; ++i)
        for (int ch = 0; ch < 3; ++ch) {
            atomic_add(gsh + ((size_t)g * K + i) * 3 + ch, bsh[i] * gcol[ch]);
            for (int j = 0; j < 3; ++j) gdir[j] += dbsh[3*i+j] * kk[3*i+ch] * gcol[ch];
        }
    const double dd = f->dir[0]*gdir[0] + f->dir[1]*gdir[1] + f->dir[2]*gdir[2];
    for (int j = 0; j < 3; ++j) gmu[j] += (gdir[j] - f->dir[j] * dd) / f->dn;

    /* opacity */
    atomic_add(go + g, gr[5] * f->sig * (1.0 - f->sig));

    /* conic -> 2D covariance (S00, S01, S11) */
    const double S00 = f->S2[0], S01 = f->S2[1], S11 = f->S2[2], det = f->det, d2 = det * det;
    const double gc0 = gr[2], gc1 = gr[3], gc2 = gr[4];
    const double gS00 = gc0 * (-S11 * S11 / d2) + gc1 * (S01 * S11 / d2) + gc2 * (1.0 / det - S00 * S11 / d2);
    const double gS11 = gc0 * (1.0 / det - S11 * S00 / d2) + gc1 * (S01 * S00 / d2) + gc2 * (-S00 * S00 / d2);
    const double gS01 = gc0 * (2.0 * S11 * S01 / d2) + gc1 * (-1.0 / det - 2.0 * S01 * S01 / d2) + gc2 * (2.0 * S00 * S01 / d2);
    const double G[2][2] = {{gS00, 0.5 * gS01}, {0.5 * gS01, gS11}};

    /* S2 = T S3 T^T: gT = 2 G T S3, gS3 = T^T G T */
    double TS[2][3];
    for (int i = 0; i < 2; ++i) for (int j = 0; j < 3; ++j)
        TS[i][j] = f->T[i][0]*f->S3[0][j] + f->T[i][1]*f->S3[1][j] + f->T[i][2]*f->S3[2][j];
    double gT[2][3], gS3[3][3];
    for (int i = 0; i < 2; ++i) for (int j = 0; j < 3; ++j)
        gT[i][j] = 2.0 * (G[i][0] * TS[0][j] + G[i][1] * TS[1][j]);
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j) {
        double acc = 0.0;
        for (int a = 0; a < 2; ++a) for (int b = 0; b < 2; ++b) acc += f->T[a][i] * G[a][b] * f->T[b][j];
        gS3[i][j] = acc;
    }

    /* T = J R: gJ = gT R^T; gRcov = J^T gT */
    double gJ00 = 0, gJ02 = 0, gJ11 = 0, gJ12 = 0;
    for (int j = 0; j < 3; ++j) {
        gJ00 += gT[0][j] * f->R[0][j];
        gJ02 += gT[0][j] * f->R[2][j];
        gJ11 += gT[1][j] * f->R[1][j];
        gJ12 += gT[1][j] * f->R[2][j];
    }
    double gRc[3][3];
    for (int j = 0; j < 3; ++j) {
        gRc[0][j] = f->J00 * gT[0][j];
        gRc[1][j] = f->J11 * gT[1][j];
        gRc[2][j] = f->J02 * gT[0][j] + f->J12 * gT[1][j];
    }

    /* J(x, y, z) with the frozen guard decisions */
    double gp[3] = {0, 0, 0};
    const double iz = 1.0 / z, iz2 = iz * iz, iz3 = iz2 * iz;
    gp[2] += gJ00 * (-fx * iz2) + gJ11 * (-fy * iz2);
    if (f->clx == 0) { gp[0] += gJ02 * (-fx * iz2); gp[2] += gJ02 * (2.0 * fx * x * iz3); }
    else gp[2] += gJ02 * (fx * f->clx * f->lx * iz2);
    if (f->cly == 0) { gp[1] += gJ12 * (-fy * iz2); gp[2] += gJ12 * (2.0 * fy * y * iz3); }
    else gp[2] += gJ12 * (fy * f->cly * f->ly * iz2);

    /* mean2D and depth */
    gp[0] += gr[0] * fx * iz;
    gp[2] += -gr[0] * fx * x * iz2;
    gp[1] += gr[1] * fy * iz;
    gp[2] += -gr[1] * fy * y * iz2;
    gp[2] += gr[9];

    /* p = R mu + t */
    for (int j = 0; j < 3; ++j) gmu[j] += f->R[0][j]*gp[0] + f->R[1][j]*gp[1] + f->R[2][j]*gp[2];
    for (int j = 0; j < 3; ++j) atomic_add(gm + 3*g + j, gmu[j]);

    /* S3 = M M^T, M = Rq diag(s) */
    double gM[3][3];
    for (int i = 0; i < 3; ++i) for (int j = 0; j < 3; ++j)
        gM[i][j] = (gS3[i][0] + gS3[0][i]) * f->M[0][j] + (gS3[i][1] + gS3[1][i]) * f->M[1][j]
                 + (gS3[i][2] + gS3[2][i]) * f->M[2][j];
    double gRq[3][3];
    for (int j = 0; j < 3; ++j) {
        double gs = 0.0;
        for (int i = 0; i < 3; ++i) { gs += gM[i][j] * f->Rq[i][j]; gRq[i][j] = gM[i][j] * f->s[j]; }
        atomic_add(gl + 3*g + j, gs * f->s[j]);
    }

    /* R(q^) and the normalisation */
    const double w = f->qh[0], a = f->qh[1], b = f->qh[2], c = f->qh[3];
    double gqh[4];
    gqh[0] = 2 * (-c * gRq[0][1] + b * gRq[0][2] + c * gRq[1][0] - a * gRq[1][2] - b * gRq[2][0] + a * gRq[2][1]);
    gqh[1] = 2 * (b * gRq[0][1] + c * gRq[0][2] + b * gRq[1][0] - w * gRq[1][2] + c * gRq[2][0] + w * gRq[2][1])
           - 4 * a * (gRq[1][1] + gRq[2][2]);
    gqh[2] = 2 * (a * gRq[0][1] + w * gRq[0][2] + a * gRq[1][0] + c * gRq[1][2] - w * gRq[2][0] + c * gRq[2][1])
           - 4 * b * (gRq[0][0] + gRq[2][2]);
    gqh[3] = 2 * (-w * gRq[0][1] + a * gRq[0][2] + w * gRq[1][0] + b * gRq[1][2] + a * gRq[2][0] + b * gRq[2][1])
           - 4 * c * (gRq[0][0] + gRq[1][1]);
    const double qd = w * gqh[0] + a * gqh[1] + b * gqh[2] + c * gqh[3];
    for (int i = 0; i < 4; ++i) atomic_add(gq + 4*g + i, (gqh[i] - f->qh[i] * qd) / f->qn);

    /* focal lengths: u = fx x / z + cx, J00 = fx / z, J02 = -fx x~ / z^2; with the
     * frustum guard active fx x~ = clx 1.3 max(cx, W - cx) z no longer depends on fx */
    if (gpose) {
        gpose[6] += gr[0] * x * iz + gJ00 * iz + (f->clx == 0 ? gJ02 * (-x * iz2) : 0.0);
        gpose[7] += gr[1] * y * iz + gJ11 * iz + (f->cly == 0 ? gJ12 * (-y * iz2) : 0.0);
    }

    /* camera pose, left perturbation V <- exp(delta^) V, delta = (rho, omega) */
    if (gpose) {
        double o1[3], o2[3];
        for (int i = 0; i < 3; ++i) gpose[i] += gp[i];
        cross3(f->p, gp, o1);
        for (int i = 0; i < 3; ++i) gpose[3+i] += o1[i];
        for (int j = 0; j < 3; ++j) {
            const double col[3] = {f->R[0][j], f->R[1][j], f->R[2][j]};
            const double gcolj[3] = {gRc[0][j], gRc[1][j], gRc[2][j]};
            cross3(col, gcolj, o2);
            for (int i = 0; i < 3; ++i) gpose[3+i] += o2[i];
        }
    }
}

/* Full backward.  dl_*: upstream gradients in the block layout of
 * orc_forward (dl_depth, dl_alpha may be NULL).  Outputs are overwritten.
 * grec (optional, [N_vg][10]) receives the per-record 2D gradients. */
ORC_API int orc_backward(const orc_scene* s, const orc_mirror* m, const double* rec64, const orc_lists* L,
                         const orc_block* blocks, int nblocks,
                         const double* dl_rgb, const double* dl_depth, const double* dl_alpha,
                         double* g_means, double* g_log_scales, double* g_quats, double* g_opac,
                         double* g_sh, double* g_pose, double* grec_out, double* g_focal)
{
    const int64_t nvg = total_records(s);
    const int K = (s->sh_degree + 1) * (s->sh_degree + 1);
    double* grec = grec_out ? grec_out : (double*)malloc(sizeof(double) * G2 * (size_t)(nvg > 0 ? nvg : 1));
    if (!grec) return 1;
    memset(grec, 0, sizeof(double) * G2 * (size_t)nvg);
    memset(g_means, 0, sizeof(double) * 3 * s->n);
    memset(g_log_scales, 0, sizeof(double) * 3 * s->n);
    memset(g_quats, 0, sizeof(double) * 4 * s->n);
    memset(g_opac, 0, sizeof(double) * s->n);
    memset(g_sh, 0, sizeof(double) * 3 * K * s->n);
    if (g_pose) memset(g_pose, 0, sizeof(double) * 6 * s->nv);

    blend_backward(s, m, rec64, L, blocks, nblocks, dl_rgb, dl_depth, dl_alpha, grec);

    for (int v = 0; v < s->nv; ++v) {
        const int64_t base = rec_base_of(s, v);
        double pose[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        #pragma omp parallel
        {
            double lp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            #pragma omp for schedule(static)
            for (int64_t j = 0; j < s->counts[v]; ++j) {
                const int64_t r = base + j;
                if (m->flags[r] & F_CULLED) continue;
                const double* gr = grec + G2 * r;
                int any = 0;
                for (int k = 0; k < G2; ++k) any |= (gr[k] != 0.0);
                if (!any) continue;
                const int64_t g = gaussian_of(s, v, j);
                orc_fwd64 f;
                pre64(s, v, g, m->flags[r], &f);
                pre64_backward(s, v, g, &f, gr, g_means, g_log_scales, g_quats, g_opac, g_sh, lp);
            }
            #pragma omp critical
            for (int k = 0; k < 8; ++k) pose[k] += lp[k];
        }
        if (g_pose) for (int k = 0; k < 6; ++k) g_pose[6*v+k] = pose[k];
        if (g_focal) for (int k = 0; k < 2; ++k) g_focal[2*v+k] = pose[6+k];
    }
    if (!grec_out) free(grec);
    return 0;
}

/* Only the preprocess adjoint: parameter and pose gradients from given
 * per-record 2D gradients grec [N_vg][10] (du, dv, dc0, dc1, dc2, dsigma,
 * dr, dg, db, dz).  Outputs are overwritten. */
ORC_API int orc_chain_backward(const orc_scene* s, const orc_mirror* m, const double* grec,
                               double* g_means, double* g_log_scales, double* g_quats, double* g_opac,
                               double* g_sh, double* g_pose, double* g_focal)
{
    const int K = (s->sh_degree + 1) * (s->sh_degree + 1);
    memset(g_means, 0, sizeof(double) * 3 * s->n);
    memset(g_log_scales, 0, sizeof(double) * 3 * s->n);
    memset(g_quats, 0, sizeof(double) * 4 * s->n);
    memset(g_opac, 0, sizeof(double) * s->n);
    memset(g_sh, 0, sizeof(double) * 3 * K * s->n);
    if (g_pose) memset(g_pose, 0, sizeof(double) * 6 * s->nv);
    for (int v = 0; v < s->nv; ++v) {
        const int64_t base = rec_base_of(s, v);
        double pose[8] = {0, 0, 0, 0, 0, 0, 0, 0};
        #pragma omp parallel
        {
            double lp[8] = {0, 0, 0, 0, 0, 0, 0, 0};
            #pragma omp for schedule(static)
            for (int64_t j = 0; j < s->counts[v]; ++j) {
                const int64_t r = base + j;
                if (m->flags[r] & F_CULLED) continue;
                const double* gr = grec + G2 * r;
                int any = 0;
                for (int k = 0; k < G2; ++k) any |= (gr[k] != 0.0);
                if (!any) continue;
                const int64_t g = gaussian_of(s, v, j);
                orc_fwd64 f;
                pre64(s, v, g, m->flags[r], &f);
                pre64_backward(s, v, g, &f, gr, g_means, g_log_scales, g_quats, g_opac, g_sh, lp);
            }
            #pragma omp critical
            for (int k = 0; k < 8; ++k) pose[k] += lp[k];
        }
        if (g_pose) for (int k = 0; k < 6; ++k) g_pose[6*v+k] = pose[k];
        if (g_focal) for (int k = 0; k < 2; ++k) g_focal[2*v+k] = pose[6+k];
    }
    return 0;
}

ORC_API int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Threads of the parallel loops that follow (timing on one core or all). */
ORC_API void orc_set_num_threads(int n)
{
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------------- */
/* 5. insertion probability and scale initialisation (Sec. 3.2, Eq. 4-6)      */
/* ------------------------------------------------------------------------- */

/*
 * P(I)(u, v) = min(|| LoG_sigma * I (u, v) ||, 1) over the three colour
 * channels, P_a = max(P(I) - P(I~), 0) for the ground truth I and the
 * rendering I~ (Eq. 4-5); a Gaussian is inserted where P_a > tau_a, with
 * scale S = d / (2 sqrt(P(I)) f) (Eq. 6).  Readings: the Laplacian of
 * Gaussian LoG(x, y) = (x^2 + y^2 - 2 s^2) / s^4 * exp(-(x^2 + y^2) / (2 s^2))
 * / (2 pi s^2) sampled at integer offsets |x|, |y| <= r = ceil(3 s), shifted to
 * zero mean (a constant image responds 0); image edges clamped; the norm is
 * the Euclidean norm of the three channel responses.
 *
 * Taps: t computed in double, mean over the (2r+1)^2 taps summed row-major,
 * taps64 = t - mean, taps32 = (float)(t - mean).  The insertion decision is
 * taken in binary32 (the mirror): per channel acc = fma(tap, I, acc) over
 * dy = -r..r, dx = -r..r; n2 = fma(a0, a0, fma(a1, a1, a2 a2));
 * P = min(sqrt(n2), 1); P_a = max(P_I - P_R, 0); inserted iff P_a > tau_a.
 * Values (P, P_a, S) in double.
 */
ORC_API int orc_log_taps(double sigma, int* radius, float* taps32, double* taps64)
{
    if (!(sigma > 0.0) || sigma > 7.0 / 3.0) return 1;
    const int r = (int)ceil(3.0 * sigma), K = 2 * r + 1;
    double t[15 * 15];
    double sum = 0.0;
    const double s2 = sigma * sigma;
    for (int y = -r; y <= r; ++y)
        for (int x = -r; x <= r; ++x) {
            const double q = (double)(x * x + y * y);
            const double v = (q - 2.0 * s2) / (s2 * s2) * exp(-q / (2.0 * s2)) / (2.0 * 3.14159265358979323846 * s2);
            t[(y + r) * K + (x + r)] = v;
            sum += v;
        }
    const double mean = sum / (double)(K * K);
    for (int i = 0; i < K * K; ++i) {
        if (taps64) taps64[i] = t[i] - mean;
        if (taps32) taps32[i] = (float)(t[i] - mean);
    }
    *radius = r;
    return 0;
}

static inline int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

ORC_API int orc_insertion(int W, int H, const float* gt, const float* ren, const float* depth, float focal,
                          double sigma, float tau_a, double* p_gt, double* p_ren, double* p_a, double* scale,
                          uint8_t* inserted)
{
    int r;
    float k32[15 * 15];
    double k64[15 * 15];
    if (orc_log_taps(sigma, &r, k32, k64)) return 1;
    const int K = 2 * r + 1;
    const int64_t hw = (int64_t)W * H;
    #pragma omp parallel for schedule(static)
    for (int y = 0; y < H; ++y)
        for (int x = 0; x < W; ++x) {
            float P32[2];
            double P64[2];
            for (int img = 0; img < 2; ++img) {
                const float* I = img ? ren : gt;
                float a32[3];
                double a64[3];
                for (int c = 0; c < 3; ++c) {
                    float acc = 0.0f;
                    double accd = 0.0;
                    for (int dy = -r; dy <= r; ++dy) {
                        const int yy = clampi(y + dy, 0, H - 1);
                        for (int dx = -r; dx <= r; ++dx) {
                            const int xx = clampi(x + dx, 0, W - 1);
                            const float px = I[c * hw + (int64_t)yy * W + xx];
                            const int ti = (dy + r) * K + (dx + r);
                            acc = fmaf(k32[ti], px, acc);
                            accd += k64[ti] * (double)px;
                        }
                    }
                    a32[c] = acc;
                    a64[c] = accd;
                }
                const float n2 = fmaf(a32[0], a32[0], fmaf(a32[1], a32[1], a32[2] * a32[2]));
                P32[img] = fminf(sqrtf(n2), 1.0f);
                const double n = sqrt(a64[0] * a64[0] + a64[1] * a64[1] + a64[2] * a64[2]);
                P64[img] = n < 1.0 ? n : 1.0;
            }
            const int64_t i = (int64_t)y * W + x;
            const float pa32 = fmaxf(P32[0] - P32[1], 0.0f);
            const int ins = pa32 > tau_a;
            const double pa = P64[0] - P64[1] > 0.0 ? P64[0] - P64[1] : 0.0;
            if (p_gt) p_gt[i] = P64[0];
            if (p_ren) p_ren[i] = P64[1];
            if (p_a) p_a[i] = pa;
            if (scale) scale[i] = ins ? (double)depth[i] / (2.0 * sqrt(P64[0]) * (double)focal) : 0.0;
            if (inserted) inserted[i] = (uint8_t)ins;
        }
    return 0;
}
