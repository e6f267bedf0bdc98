// gsr_merge.cu -- inter-camera Gaussian merging (Sec. 3.2, Eq. 7-8).
//
// Camera i's sampled pixels (those of Eq. 4-5 above tau_a, scales S of Eq. 6)
// meet the Gaussians already built from cameras 0 .. i-1:
//   1. each existing Gaussian is reprojected into camera i and paired with
//      the sampled pixel containing its mean, if |z' - d_i| <= tau_d;
//   2. each sampled pixel's group (the sample and its paired Gaussians) keeps
//      the primitive of smallest image-space scale -- S f / z for both sides
//      (Eq. 7 and Eq. 8 agree on a sample of Eq. 6 under this reading), ties
//      to the existing Gaussian of lowest index -- and the group's mean
//      colour (SH DC coefficients); a kept sample moves to the group's mean
//      depth, its scale following the depth as in Eq. 6.
// Pairing, the depth gate and the choice are integer results: they are taken
// in binary32 with the operation order written in the kernels (the projection
// sums left to right, no contraction; the scale through the decision
// contract's exponential).  Group sums are fixed-point 64-bit atomics, so the
// results do not depend on the order of the atomics.
//
// Four launches: slot scatter (pixel -> sample), pairing (one thread per
// existing Gaussian: argmin key = (scale bits, index) by 64-bit atomicMin,
// fixed-point sums), per-sample resolution (one thread per sample), and
// per-Gaussian resolution.
#include "gsr_common.cuh"
#include "gsr_kernels.h"

namespace gsr {

constexpr int kMergeThreads = 256;
constexpr float kDcFix = 4294967296.0f;    // 2^32: DC coefficients in fixed point
constexpr float kZFix = 16777216.0f;       // 2^24: depths in fixed point

__global__ void merge_scatter_kernel(const uint32_t* __restrict__ pixels, int64_t n, int32_t* __restrict__ slot_map,
                                     int64_t n_pix)
{
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < n; s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t p = pixels[s];
        if (p < n_pix) slot_map[p] = (int32_t)s;
    }
}

__global__ void __launch_bounds__(kMergeThreads)
merge_pair_kernel(const __grid_constant__ MergeArgs a)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.n_existing;
         g += (int64_t)gridDim.x * blockDim.x) {
        const float mx = a.means[3 * g], my = a.means[3 * g + 1], mz = a.means[3 * g + 2];
        float pc[3];
#pragma unroll
        for (int r = 0; r < 3; ++r)
            pc[r] = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(a.V[4 * r], mx), __fmul_rn(a.V[4 * r + 1], my)),
                                        __fmul_rn(a.V[4 * r + 2], mz)), a.V[4 * r + 3]);
        int32_t slot = -1;
        if (pc[2] > a.near_plane) {
            const float u = __fadd_rn(__fmul_rn(a.fx, __fdiv_rn(pc[0], pc[2])), a.cx);
            const float v = __fadd_rn(__fmul_rn(a.fy, __fdiv_rn(pc[1], pc[2])), a.cy);
            if (u >= 0.0f && u < (float)a.W && v >= 0.0f && v < (float)a.H) {
                const int64_t pix = (int64_t)floorf(v) * a.W + (int64_t)floorf(u);
                const int32_t s = a.slot_map[pix];
                if (s >= 0 && fabsf(__fsub_rn(pc[2], a.depth_map[pix])) <= a.tau_d) {
                    const float* ls = a.log_scales + 3 * g;
                    const float S = exp_contract(fmaxf(fmaxf(ls[0], ls[1]), ls[2]));
                    const float sc = __fdiv_rn(__fmul_rn(S, a.fx), pc[2]);
                    const unsigned long long key =
                        ((unsigned long long)__float_as_uint(sc) << 32) | (unsigned long long)(uint32_t)g;
                    atomicMin(a.best + s, key);
                    atomicAdd(a.count + s, 1u);
                    const float* dc = a.sh + (int64_t)a.sh_stride * g;
                    long long* sum = a.sums + 4 * (int64_t)s;
#pragma unroll
                    for (int c = 0; c < 3; ++c)
                        atomicAdd(reinterpret_cast<unsigned long long*>(sum + c),
                                  (unsigned long long)__float2ll_rn(dc[c] * kDcFix));
                    atomicAdd(reinterpret_cast<unsigned long long*>(sum + 3),
                              (unsigned long long)__float2ll_rn(pc[2] * kZFix));
                    slot = s;
                }
            }
        }
        a.pair[g] = slot;
    }
}

// Values here are FP32 (GB300 runs FP64 at a small fraction of the FP32
// rate): the colour, depth and position of a sample carry ~1e-7 relative
// error, the decision s_new < s_best is the binary32 one of the contract.
__global__ void __launch_bounds__(kMergeThreads)
merge_sample_kernel(const __grid_constant__ MergeArgs a)
{
    const int64_t npix = (int64_t)a.W * a.H;
    const float inv_sh0 = (float)(1.0 / GSR_SH0);
    for (int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; s < a.n_samples;
         s += (int64_t)gridDim.x * blockDim.x) {
        const uint32_t pix = a.pixels[s];
        if ((int64_t)pix >= npix) {   // a pixel index outside the view: no outputs but the action
            a.sample_action[s] = -1;
            continue;
        }
        const float d = a.depth_map[pix], Sp = a.scale_map[pix];
        float dc[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) dc[c] = (a.gt[(int64_t)c * npix + pix] - 0.5f) * inv_sh0;
        float depth = d;
        int32_t action = kMergeInsert;
        const unsigned n = a.count[s];
        if (n > 0) {
            const unsigned long long key = a.best[s];
            const float s_best = __uint_as_float((uint32_t)(key >> 32));
            const float s_new = __fdiv_rn(__fmul_rn(Sp, a.fx), d);
            const longlong4_32a sum = *reinterpret_cast<const longlong4_32a*>(a.sums + 4 * s);   // 32-byte aligned rows
            const float inv = 1.0f / (float)(n + 1);
            float mean[3] = {(dc[0] + (float)sum.x * 0x1p-32f) * inv, (dc[1] + (float)sum.y * 0x1p-32f) * inv,
                             (dc[2] + (float)sum.z * 0x1p-32f) * inv};
            if (s_new < s_best) {
                action = kMergeReplaces;
                depth = (d + (float)sum.w * 0x1p-24f) * inv;
#pragma unroll
                for (int c = 0; c < 3; ++c) dc[c] = mean[c];
            } else {
                action = kMergeMerged;
                a.slot_dc[3 * s] = mean[0];
                a.slot_dc[3 * s + 1] = mean[1];
                a.slot_dc[3 * s + 2] = mean[2];
            }
        }
        a.sample_action[s] = action;
        // the sample as a Gaussian: its pixel centre unprojected at `depth`
        const float px = (float)(pix % (uint32_t)a.W) + 0.5f, py = (float)(pix / (uint32_t)a.W) + 0.5f;
        const float q[3] = {(px - a.cx) * a.inv_fx * depth - a.V[3], (py - a.cy) * a.inv_fy * depth - a.V[7],
                            depth - a.V[11]};
        if (a.sample_means) {
#pragma unroll
            for (int c = 0; c < 3; ++c)
                a.sample_means[3 * s + c] = a.V[c] * q[0] + a.V[4 + c] * q[1] + a.V[8 + c] * q[2];
        }
        if (a.sample_depth) a.sample_depth[s] = depth;
        if (a.sample_scale) a.sample_scale[s] = d > 0.0f ? Sp * (depth / d) : Sp * depth;
        if (a.sample_dc) {
#pragma unroll
            for (int c = 0; c < 3; ++c) a.sample_dc[3 * s + c] = dc[c];
        }
    }
}

// Per existing Gaussian: its action; the group's mean colour for the kept
// ones only (the others keep the colour the caller holds, so their SH rows
// are not read).
__global__ void __launch_bounds__(kMergeThreads)
merge_existing_kernel(const __grid_constant__ MergeArgs a)
{
    for (int64_t g = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; g < a.n_existing;
         g += (int64_t)gridDim.x * blockDim.x) {
        const int32_t s = a.pair[g];
        int32_t action = kMergeUntouched;
        if (s >= 0) {
            action = kMergeRemoved;
            if (a.sample_action[s] == kMergeMerged && (uint32_t)(a.best[s] & 0xffffffffu) == (uint32_t)g) {
                action = kMergeKept;
                if (a.existing_dc) {
                    a.existing_dc[3 * g] = a.slot_dc[3 * s];
                    a.existing_dc[3 * g + 1] = a.slot_dc[3 * s + 1];
                    a.existing_dc[3 * g + 2] = a.slot_dc[3 * s + 2];
                }
            }
        }
        if (a.existing_action) a.existing_action[g] = action;
    }
}

static unsigned merge_grid(int64_t n, int num_sms)
{
    int64_t g = (n + kMergeThreads - 1) / kMergeThreads;
    const int64_t cap = (int64_t)num_sms * 8;
    if (g > cap) g = cap;
    return (unsigned)(g < 1 ? 1 : g);
}

void launch_merge(const MergeArgs& a, int num_sms, cudaStream_t s)
{
    if (a.n_samples > 0) {
        GSR_COUNT_LAUNCH();
        merge_scatter_kernel<<<merge_grid(a.n_samples, num_sms), kMergeThreads, 0, s>>>(
            a.pixels, a.n_samples, a.slot_map, (int64_t)a.W * a.H);
    }
    if (a.n_existing > 0) {
        GSR_COUNT_LAUNCH();
        merge_pair_kernel<<<merge_grid(a.n_existing, num_sms), kMergeThreads, 0, s>>>(a);
    }
    if (a.n_samples > 0) {
        GSR_COUNT_LAUNCH();
        merge_sample_kernel<<<merge_grid(a.n_samples, num_sms), kMergeThreads, 0, s>>>(a);
    }
    if (a.n_existing > 0) {
        GSR_COUNT_LAUNCH();
        merge_existing_kernel<<<merge_grid(a.n_existing, num_sms), kMergeThreads, 0, s>>>(a);
    }
}

}  // namespace gsr
