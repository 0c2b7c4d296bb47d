// voge_sample.cu -- the neural sampler of Sec. 3.4 (Eq. 10): per-kernel
// attributes from per-pixel features through the renderer's kept lists,
//   alpha_k = sum_p W_pk phi_p / sum_p W_pk,
// the sums running over the pixels whose kept list holds k (the renderer's
// W_pk, Eq. 8, is zero for every other pixel).  A kernel no pixel keeps gets
// alpha_k = 0.
//
// The sums are a transpose of the forward pass's scatter: each (pixel, list
// slot) adds W phi_p to its kernel's row.  One warp handles 32 consecutive
// pixels, one list slot at a time; the lanes cover (source, channel group)
// pairs, so one 16-byte vector reduction adds four channels of a row.  For
// wide rows (k_sample_grouped) the warp first groups its lanes by kernel
// (match.any), since neighbouring pixels often keep the same kernel in the
// same slot; each group adds one summed row and one summed weight.  For
// narrow rows the grouping costs more than the reductions it saves.
#include "../../include/voge.h"
#include "voge_device.cuh"
#include "voge_trace.cuh"

namespace voge {
namespace {

// Rows of any width: one (pixel, slot) entry adds its W-weighted feature row.
__global__ void __launch_bounds__(256) k_sample(int64_t P, int L, int N, int C, const int32_t* __restrict__ idx,
                                                const float* __restrict__ W, const float* __restrict__ phi,
                                                float* num, float* wsum) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const bool rv4 = (C & 3) == 0 && ((reinterpret_cast<uintptr_t>(phi) | reinterpret_cast<uintptr_t>(num)) & 15) == 0;
    const int cw = rv4 ? C >> 2 : C;         // row width in reduction units
    const int spi = cw <= 32 ? 32 / cw : 1;  // source pixels per step
    const int sub = cw <= 32 ? lane / cw : 0;
    const int cc = cw <= 32 ? lane - sub * cw : lane;
    for (int64_t wb = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); wb * 32 < P; wb += nwarps) {
        const int64_t p = wb * 32 + lane;
        for (int k = 0; k < L; ++k) {
            int32_t g = -1;
            float w = 0.0f;
            if (p < P) {
                g = __ldg(idx + p * L + k);
                if (g >= N) g = -1;
                if (g >= 0) w = __ldg(W + p * L + k);
            }
            const unsigned m = __ballot_sync(0xffffffffu, g >= 0);
            if (m == 0) continue;  // no kept kernel in this slot of the warp's pixels
            if (g >= 0) atomicAdd(wsum + g, w);
            const int top = 32 - __clz(m);
            for (int s0 = 0; s0 < top; s0 += spi) {
                const int src = s0 + sub;
                const int32_t gs = __shfl_sync(0xffffffffu, g, src & 31);
                const float ws = __shfl_sync(0xffffffffu, w, src & 31);
                if (sub < spi && src < 32 && gs >= 0) {
                    const float* f = phi + (wb * 32 + src) * C;
                    float* dst = num + (int64_t)gs * C;
                    if (rv4) {
                        for (int c = cc; c < cw; c += 32) {
                            const float4 x = __ldg(reinterpret_cast<const float4*>(f) + c);
                            red_add_v4(dst + 4 * c, ws * x.x, ws * x.y, ws * x.z, ws * x.w);
                        }
                    } else {
                        for (int c = cc; c < C; c += 32) atomicAdd(dst + c, ws * __ldg(f + c));
                    }
                }
            }
        }
    }
}

// Wide 16-byte rows: lanes holding the same kernel in a slot add one summed row.
__global__ void __launch_bounds__(256) k_sample_grouped(int64_t P, int L, int N, int C,
                                                        const int32_t* __restrict__ idx, const float* __restrict__ W,
                                                        const float* __restrict__ phi, float* num, float* wsum) {
    // per warp of the 256-thread block: the slot's weights, kernels and same-kernel lane masks
    __shared__ float s_w[8][32];
    __shared__ int32_t s_g[8][32];
    __shared__ unsigned s_grp[8][32];
    __shared__ int32_t s_ld[8][32];  // lanes of the group leaders, in lane order
    const int lane = threadIdx.x & 31, wi = threadIdx.x >> 5;
    const int64_t nwarps = (int64_t)gridDim.x * (blockDim.x >> 5);
    const bool rv4 = (C & 3) == 0 && ((reinterpret_cast<uintptr_t>(phi) | reinterpret_cast<uintptr_t>(num)) & 15) == 0;
    const int cw = rv4 ? C >> 2 : C;         // row width in reduction units
    const int spi = cw <= 32 ? 32 / cw : 1;  // kernels per step
    const int sub = cw <= 32 ? lane / cw : 0;
    const int cc = cw <= 32 ? lane - sub * cw : lane;
    for (int64_t wb = (int64_t)blockIdx.x * (blockDim.x >> 5) + wi; wb * 32 < P; wb += nwarps) {
        const int64_t p = wb * 32 + lane;
        for (int k = 0; k < L; ++k) {
            int32_t g = -1;
            float w = 0.0f;
            if (p < P) {
                g = __ldg(idx + p * L + k);
                if (g >= N) g = -1;
                if (g >= 0) w = __ldg(W + p * L + k);
            }
            if (__ballot_sync(0xffffffffu, g >= 0) == 0) continue;  // no kept kernel in this slot of the warp
            // neighbouring pixels often keep the same kernel in the same slot:
            // each group of equal kernels adds one summed row and one weight
            const unsigned grp = __match_any_sync(0xffffffffu, g);
            const bool leader = g >= 0 && __ffs(grp) - 1 == lane;
            s_w[wi][lane] = w;
            s_g[wi][lane] = g;
            s_grp[wi][lane] = grp;
            __syncwarp();
            const unsigned lead = __ballot_sync(0xffffffffu, leader);
            const int nlead = __popc(lead);
            if (leader) {
                s_ld[wi][__popc(lead & ((1u << lane) - 1u))] = lane;
                float ws = 0.0f;
                for (unsigned b = grp; b; b &= b - 1) ws += s_w[wi][__ffs(b) - 1];
                atomicAdd(wsum + g, ws);
            }
            __syncwarp();
            for (int s0 = 0; s0 < nlead; s0 += spi) {
                const int li = s0 + sub;
                if (sub < spi && li < nlead) {
                    const int ld = s_ld[wi][li];
                    const unsigned gm = s_grp[wi][ld];
                    float* dst = num + (int64_t)s_g[wi][ld] * C;
                    const float* f0 = phi + wb * 32 * C;
                    if (rv4) {
                        for (int c = cc; c < cw; c += 32) {
                            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                            for (unsigned b = gm; b; b &= b - 1) {
                                const int q = __ffs(b) - 1;
                                const float wq = s_w[wi][q];
                                const float4 x = __ldg(reinterpret_cast<const float4*>(f0 + (int64_t)q * C) + c);
                                acc.x = fmaf(wq, x.x, acc.x);
                                acc.y = fmaf(wq, x.y, acc.y);
                                acc.z = fmaf(wq, x.z, acc.z);
                                acc.w = fmaf(wq, x.w, acc.w);
                            }
                            red_add_v4(dst + 4 * c, acc.x, acc.y, acc.z, acc.w);
                        }
                    } else {
                        for (int c = cc; c < C; c += 32) {
                            float acc = 0.0f;
                            for (unsigned b = gm; b; b &= b - 1) {
                                const int q = __ffs(b) - 1;
                                acc = fmaf(s_w[wi][q], __ldg(f0 + (int64_t)q * C + c), acc);
                            }
                            atomicAdd(dst + c, acc);
                        }
                    }
                }
            }
            __syncwarp();  // the slot's shared entries are read; the next slot overwrites them
        }
    }
}

// alpha = num / wsum per kernel (0 where no pixel keeps the kernel), in place.
__global__ void __launch_bounds__(256) k_sample_norm(int N, int C, float* alpha, const float* __restrict__ wsum) {
    const int64_t n = (int64_t)N * C;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const float d = __ldg(wsum + e / C);
        alpha[e] = d > 0.0f ? alpha[e] / d : 0.0f;
    }
}

}  // namespace
}  // namespace voge

using namespace voge;

extern "C" int voge_sample(int64_t pixels, int32_t L, int32_t N, int32_t C, const int32_t* index, const float* weights,
                           const float* features, float* alpha, float* wsum, voge_stream_t stream_) {
    if (pixels < 0 || L < 0 || N < 0 || C < 1) return VOGE_ERR_ARG;
    if (N > 0 && (!alpha || !wsum)) return VOGE_ERR_ARG;
    if (pixels > 0 && L > 0 && (!index || !weights || !features)) return VOGE_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    if (N == 0) return VOGE_OK;
    if (cudaMemsetAsync(alpha, 0, sizeof(float) * (size_t)N * (size_t)C, s) != cudaSuccess ||
        cudaMemsetAsync(wsum, 0, sizeof(float) * (size_t)N, s) != cudaSuccess)
        return VOGE_ERR_CUDA;
    if (pixels > 0 && L > 0) {
        int64_t nb = (pixels + 255) / 256;
        if (nb > 152 * 16) nb = 152 * 16;
        // the kernels test the same alignment for their 16-byte rows
        const bool wide = (C & 3) == 0 && C >= 64 &&
                          ((reinterpret_cast<uintptr_t>(features) | reinterpret_cast<uintptr_t>(alpha)) & 15) == 0;
        if (wide) {
            TraceScope tr("k_sample_grouped", s);
            k_sample_grouped<<<(unsigned)nb, 256, 0, s>>>(pixels, L, N, C, index, weights, features, alpha, wsum);
        } else {
            TraceScope tr("k_sample", s);
            k_sample<<<(unsigned)nb, 256, 0, s>>>(pixels, L, N, C, index, weights, features, alpha, wsum);
        }
        if (cudaPeekAtLastError() != cudaSuccess) return VOGE_ERR_CUDA;
    }
    int64_t nb = ((int64_t)N * C + 255) / 256;
    if (nb > 152 * 16) nb = 152 * 16;
    TraceScope tr("k_sample_norm", s);
    k_sample_norm<<<(unsigned)nb, 256, 0, s>>>(N, C, alpha, wsum);
    return cudaPeekAtLastError() == cudaSuccess ? VOGE_OK : VOGE_ERR_CUDA;
}
