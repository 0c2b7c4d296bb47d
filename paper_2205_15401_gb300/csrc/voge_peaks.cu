// voge_peaks.cu -- measured arithmetic ceilings for the roofline of the tile
// kernels.  Nothing on the render path is a dense contraction or bound by
// HBM: the pair terms of Eq. 7 (forward) and their adjoint (backward) run on
// the FP32 and MUFU pipes.  Four register-only loops measure, on every SM of
// the current device:
//   - the FP32 FMA rate (eight independent chains per thread),
//   - the MUFU ex2.approx rate,
//   - the rate of the forward pair term exactly as the fine pass evaluates
//     it (u, erf by A&S 7.1.28, A_k += copysign(m_j, u) erf|u|),
//   - the rate of the backward pair adjoint exactly as k_backward evaluates
//     it (A&S 7.1.26 with e^{-u^2}, the four accumulations).
// The pair loops keep the k side in registers like the tile kernels and
// advance the j side with one FMA per row of pairs instead of a shared-memory
// read, so they bound what the pair loops can reach on this GPU.
#include <cstring>

#include "../../include/voge.h"
#include "voge_device.cuh"

namespace voge {
namespace {

__device__ float g_peak_sink;  // written only if a result hits an impossible value

constexpr int kFmaIters = 40000, kEx2Iters = 5000, kFwdIters = 25000, kBwdIters = 20000;
constexpr int kPairKM = 20;  // list capacity of the benchmark's tile kernels
constexpr float kTwoOverSqrtPi = 1.1283791670955126f;

__global__ void __launch_bounds__(256, 4) k_peak_fma(int iters, float seed) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = seed + (float)(threadIdx.x + 32 * i) * 1e-7f;
    const float m = 0.9999999f, c = 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = fmaf(x[i], m, c);
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == -1.2345678f) g_peak_sink = s;
}

__global__ void __launch_bounds__(256, 4) k_peak_ex2(int iters, float seed) {
    float x[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = seed + (float)(threadIdx.x + 32 * i) * 1e-7f;
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int r = 0; r < 16; ++r) {
#pragma unroll
            for (int i = 0; i < 8; ++i) x[i] = ex2_approx(-x[i]);  // stays in [0.5, 1]
        }
    }
    float s = 0.0f;
#pragma unroll
    for (int i = 0; i < 8; ++i) s += x[i];
    if (s == -1.2345678f) g_peak_sink = s;
}

// Forward pair term: the k_render<20, 16> occupancy (three CTAs of 256 per SM).
__global__ void __launch_bounds__(256, 3) k_peak_pair_fwd(int iters, float seed) {
    float hi[kPairKM], lo[kPairKM], A[kPairKM];
#pragma unroll
    for (int s = 0; s < kPairKM; ++s) {
        hi[s] = seed + 0.03f * (float)s + 1e-6f * (float)threadIdx.x;
        lo[s] = 1e-8f * (float)s;
        A[s] = 0.0f;
    }
    float4 J = make_float4(seed + 0.2f, 3e-9f, 40.0f, 0.25f);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int s = 0; s < kPairKM; ++s) {
            const float u = ((hi[s] - J.x) + (lo[s] - J.y)) * J.z;
            A[s] = fmaf(copysignf(J.w, u), 1.0f - erfc_as28(fabsf(u)), A[s]);
        }
        J.x = fmaf(J.x, 0.9999f, 1.5e-4f);  // the next j (drifts towards 1.5)
    }
    float s = 0.0f;
#pragma unroll
    for (int k = 0; k < kPairKM; ++k) s += A[k];
    if (s == -1.2345678f) g_peak_sink = s;
}

// Backward pair adjoint: the k_backward<20, 8> occupancy (four CTAs of 128 per SM).
__global__ void __launch_bounds__(128, 4) k_peak_pair_bwd(int iters, float seed) {
    float hi[kPairKM], lo[kPairKM], dA[kPairKM], dl[kPairKM];
#pragma unroll
    for (int s = 0; s < kPairKM; ++s) {
        hi[s] = seed + 0.03f * (float)s + 1e-6f * (float)threadIdx.x;
        lo[s] = 1e-8f * (float)s;
        dA[s] = -0.01f * (float)(s + 1);
        dl[s] = 0.0f;
    }
    float4 J = make_float4(seed + 0.2f, 3e-9f, 40.0f, 0.25f);
    float tot = 0.0f;
    for (int it = 0; it < iters; ++it) {
        const float mj = J.w * kTwoOverSqrtPi;
        float acc_dm = 0.0f, acc_s = 0.0f, acc_dr = 0.0f;
#pragma unroll
        for (int s = 0; s < kPairKM; ++s) {
            const float d = (hi[s] - J.x) + (lo[s] - J.y);
            const float u = d * J.z;
            float g2;
            const float ec = erfc_as26(fabsf(u), g2);
            const float E = copysignf(1.0f - ec, u);
            acc_dm = fmaf(dA[s], 1.0f + E, acc_dm);
            const float du = dA[s] * mj * g2;
            dl[s] = fmaf(du, J.z, dl[s]);
            acc_s += du;
            acc_dr = fmaf(du, d, acc_dr);
        }
        tot += acc_dm + acc_s + acc_dr;
        J.x = fmaf(J.x, 0.9999f, 1.5e-4f);
    }
#pragma unroll
    for (int k = 0; k < kPairKM; ++k) tot += dl[k];
    if (tot == -1.2345678f) g_peak_sink = tot;
}

// One untimed and one timed launch; milliseconds of the timed one.
template <typename Launch>
cudaError_t timed(Launch launch, cudaStream_t s, float* ms) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e == cudaSuccess) {
        launch();
        e = cudaPeekAtLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e0, s);
    if (e == cudaSuccess) {
        launch();
        e = cudaPeekAtLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, s);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    if (e == cudaSuccess) e = cudaEventElapsedTime(ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return e;
}

}  // namespace
}  // namespace voge

using namespace voge;

extern "C" int voge_measure_alu_peaks(voge_alu_peaks* out, voge_stream_t stream) {
    if (!out) return VOGE_ERR_ARG;
    memset(out, 0, sizeof(*out));
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    int dev = 0, nsm = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return VOGE_ERR_CUDA;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) return VOGE_ERR_CUDA;
    out->sms = nsm;
    const float seed = 0.5f;
    float ms[4] = {0, 0, 0, 0};
    const int g4 = 4 * nsm, g3 = 3 * nsm;
    cudaError_t e = timed([&] { k_peak_fma<<<g4, 256, 0, s>>>(kFmaIters, seed); }, s, &ms[0]);
    if (e == cudaSuccess) e = timed([&] { k_peak_ex2<<<g4, 256, 0, s>>>(kEx2Iters, seed); }, s, &ms[1]);
    if (e == cudaSuccess) e = timed([&] { k_peak_pair_fwd<<<g3, 256, 0, s>>>(kFwdIters, seed); }, s, &ms[2]);
    if (e == cudaSuccess) e = timed([&] { k_peak_pair_bwd<<<g4, 128, 0, s>>>(kBwdIters, seed); }, s, &ms[3]);
    if (e != cudaSuccess) return VOGE_ERR_CUDA;
    for (int i = 0; i < 4; ++i) {
        if (!(ms[i] > 0.0f)) return VOGE_ERR_CUDA;
        out->ms[i] = ms[i];
    }
    const double t256x4 = 256.0 * g4, t256x3 = 256.0 * g3, t128x4 = 128.0 * g4;
    out->fma_tflops = t256x4 * kFmaIters * 128.0 * 2.0 / (ms[0] * 1e-3) / 1e12;
    out->ex2_tops = t256x4 * kEx2Iters * 128.0 / (ms[1] * 1e-3) / 1e12;
    out->fwd_gpairs = t256x3 * kFwdIters * (double)kPairKM / (ms[2] * 1e-3) / 1e9;
    out->bwd_gpairs = t128x4 * kBwdIters * (double)kPairKM / (ms[3] * 1e-3) / 1e9;
    return VOGE_OK;
}
