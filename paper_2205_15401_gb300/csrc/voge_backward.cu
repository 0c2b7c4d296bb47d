// voge_backward.cu -- adjoint of the forward pass with the kept lists frozen.
//
// Only the per-pixel index lists come from the forward pass; l, e^{q},
// sigma, T(l_k) and every erf term of Eq. 7 are recomputed here.  For a pixel
// with list L_p and upstream gradient g_p = dLoss/dimage_p:
//   dc_k += W_k g_p,  G_k = g_p . c_k,  dA_k = -tau G_k W_k
//   dm_j += dA_k (1 + erf u_kj),  du_kj = dA_k m_j (2/sqrt(pi)) e^{-u_kj^2}
//   dl_k += du r_j,  dl_j -= du r_j,  dr_j += du (l_k - l_j)
//   dqt_k = dA_k / (2 tau) - a_k dm_k / 4   (from W = T a, m = a/2, a = e^{-qt/2})
//   db_k  = dr_k / (4 r_k)                  (r = sqrt(b/2))
// and then (qt, l, b) -> camera-space mean and inverse covariance:
//   dM += 2 dqt P V + dl P D / b,
//   dP_ab += dqt V_a V_b + dl (V_a D_b + D_a V_b) / (2b) + db D_a D_b,
// with V = M - l D (App. A.1: VᵀPD = 0, so l's own dependence drops out of qt).
// Camera-space sums per (view, Gaussian) are rotated to world space and
// reduced into the camera pose by k_grad_finalize.
#include "voge_device.cuh"
#include "voge_trace.cuh"

namespace voge {

constexpr float kTwoOverSqrtPi = 1.1283791670955126f;

// Camera-space gradient of one (pixel, kept Gaussian) pair: out[0..2] = dM,
// out[3..8] = G (xx, xy, xz, yy, yz, zz) with entries of P treated as independent.
__device__ __forceinline__ void chain_to_camera(const Args& a, int64_t o, float px, float py, float invF, float dqt,
                                                float dl, float db, float out[9]) {
    float4 r0, r1, r2, r3;
    load_rec(a.ws.rec, o, r0, r1, r2, r3);
    const float4 s0 = __ldg(a.ws.rec2 + 2 * o), s1 = __ldg(a.ws.rec2 + 2 * o + 1);
    const Trace t = trace_px(r0, r1, r2, r3, px, py);
    const float ib = 1.0f / t.b;
    const float Mz = r3.y;
    const float dlt = -Mz * t.num * ib;  // l - Mz
    const float dx = t.du * invF, dy = t.dv * invF;
    const float D0 = s1.z + dx, D1 = s1.w + dy;  // D = (D0, D1, 1)
    // V = M - l D = -Mz D' - (l - Mz) D
    const float V0 = fmaf(-Mz, dx, -dlt * D0), V1 = fmaf(-Mz, dy, -dlt * D1), V2 = -dlt;
    const float Pxx = s0.x, Pxy = s0.y, Pxz = s0.z, Pyy = s0.w, Pyz = s1.x, Pzz = s1.y;
    const float PV0 = fmaf(Pxx, V0, fmaf(Pxy, V1, Pxz * V2));
    const float PV1 = fmaf(Pxy, V0, fmaf(Pyy, V1, Pyz * V2));
    const float PV2 = fmaf(Pxz, V0, fmaf(Pyz, V1, Pzz * V2));
    const float PD0 = fmaf(Pxx, D0, fmaf(Pxy, D1, Pxz));
    const float PD1 = fmaf(Pxy, D0, fmaf(Pyy, D1, Pyz));
    const float PD2 = fmaf(Pxz, D0, fmaf(Pyz, D1, Pzz));
    const float q2 = 2.0f * dqt, lb = dl * ib, lh = 0.5f * lb;
    out[0] = fmaf(q2, PV0, lb * PD0);
    out[1] = fmaf(q2, PV1, lb * PD1);
    out[2] = fmaf(q2, PV2, lb * PD2);
    out[3] = fmaf(dqt, V0 * V0, fmaf(lb, V0 * D0, db * D0 * D0));
    out[4] = fmaf(dqt, V0 * V1, fmaf(lh, fmaf(V0, D1, D0 * V1), db * D0 * D1));
    out[5] = fmaf(dqt, V0 * V2, fmaf(lh, fmaf(V0, 1.0f, D0 * V2), db * D0));
    out[6] = fmaf(dqt, V1 * V1, fmaf(lb, V1 * D1, db * D1 * D1));
    out[7] = fmaf(dqt, V1 * V2, fmaf(lh, fmaf(V1, 1.0f, D1 * V2), db * D1));
    out[8] = fmaf(dqt, V2 * V2, fmaf(lb, V2, db));
}

template <int KM, int TH>
__global__ void __launch_bounds__(16 * TH, TH == 16 ? 2 : 3) k_backward(Args a) {
    constexpr int NT = 16 * TH;
    extern __shared__ float4 smem[];
    float4* jst = smem;  // [KM][NT]

    const CamDev* cams = a.ws.cams;
    const int t = blockIdx.x;
    const int v = find_view(cams, a.B, t);
    const int lt = t - __ldg(&cams[v].tile_base);
    const int tiles_x = __ldg(&cams[v].tiles_x);
    const int tx = lt % tiles_x, ty = lt / tiles_x;
    const int H = __ldg(&cams[v].H), W = __ldg(&cams[v].W);
    const float invF = __ldg(&cams[v].invF);
    const int tid = threadIdx.x;
    const int j = tx * kTileW + (tid & 15);
    const int i = ty * TH + (tid >> 4);
    const bool valid = (i < H) && (j < W);
    const float px = (float)j + 0.5f, py = (float)i + 0.5f;
    const int64_t pix = __ldg(&cams[v].pix_base) + (int64_t)i * W + j;
    const int64_t vb = (int64_t)v * a.N;
    const int L = a.L, K = a.L, C = a.C;

    int32_t id[KM];
    float hi[KM], lo[KM], dA[KM], dl[KM];
    if (!valid) return;  // no block-wide barriers in this kernel
    int n = 0;
    bool open = true;
#pragma unroll
    for (int s = 0; s < KM; ++s) {
        id[s] = -1;
        hi[s] = 0.0f;
        lo[s] = 0.0f;
        dA[s] = 0.0f;
        dl[s] = 0.0f;
        if (s >= KM - K && open) {
            const int32_t g = __ldg(a.index_in + pix * L + (s - (KM - K)));
            if (g >= 0 && g < a.N) {
                float4 r0, r1, r2, r3;
                load_rec(a.ws.rec, vb + g, r0, r1, r2, r3);
                const Entry e = entry_px(r0, r1, r2, r3, px, py);
                hi[s] = e.hi;
                lo[s] = e.lo;
                id[s] = g;
                jst[n * NT + tid] = make_float4(e.hi, e.lo, e.r, 0.5f * e.a);
                ++n;
            } else {
                open = false;
            }
        }
    }
    // loop 1: A_k
    float A[KM];
#pragma unroll
    for (int s = 0; s < KM; ++s) A[s] = 0.0f;
    for (int e = 0; e < n; ++e) {
        const float4 J = jst[e * NT + tid];
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            const float u = ((hi[s] - J.x) + (lo[s] - J.y)) * J.z;
            const float q = erfc_as28(fabsf(u));
            const float sm = copysignf(J.w, u);
            A[s] = fmaf(-sm, q, A[s] + (J.w + sm));
        }
    }
    // T, W, attribute gradient, dA
    const float ntl = -a.tau * kLog2e;
    const float* gp = a.grad_image + pix * C;
    {
        int e = 0;
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            if (id[s] >= 0) {
                const float am = jst[e * NT + tid].w;
                const float Wk = ex2_approx(ntl * A[s]) * (2.0f * am);
                const float* ck = a.attr + (int64_t)id[s] * C;
                float G = 0.0f;
                for (int c = 0; c < C; ++c) {
                    const float gc = __ldg(gp + c);
                    G = fmaf(gc, __ldg(ck + c), G);
                    if (a.grad_attr) atomicAdd(a.grad_attr + (int64_t)id[s] * C + c, Wk * gc);
                }
                dA[s] = -a.tau * G * Wk;
                ++e;
            }
        }
    }
    // loop 2: adjoint of the pair terms
    for (int e = 0; e < n; ++e) {
        const float4 J = jst[e * NT + tid];
        const float mj = J.w * kTwoOverSqrtPi;
        float acc_dm = 0.0f, acc_s = 0.0f, acc_dr = 0.0f;
#pragma unroll
        for (int s = 0; s < KM; ++s) {
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
        jst[e * NT + tid] = make_float4(acc_dm, -acc_s * J.z, acc_dr, 0.0f);
    }
    // chain rule to camera space
    const float inv2tau = 0.5f / a.tau;
    {
        int e = 0;
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            if (id[s] >= 0) {
                const float4 J = jst[e * NT + tid];
                float4 r0, r1, r2, r3;
                const int64_t o = vb + id[s];
                load_rec(a.ws.rec, o, r0, r1, r2, r3);
                const Entry en = entry_px(r0, r1, r2, r3, px, py);
                const float dqt = fmaf(dA[s], inv2tau, -0.25f * en.a * J.x);
                const float db = J.z / (4.0f * en.r);
                float gv[9];
                chain_to_camera(a, o, px, py, invF, dqt, dl[s] + J.y, db, gv);
                float* gc = a.ws.gcam + 9 * o;
#pragma unroll
                for (int q = 0; q < 9; ++q) atomicAdd(gc + q, gv[q]);
                ++e;
            }
        }
    }
}

// Generic backward for list lengths above the register lists (L > 32).
// Per-pixel scratch in the workspace: [L][8] floats = hi, lo, r, m, A->dA, dl, dm, dr.
__global__ void __launch_bounds__(256) k_backward_generic(Args a) {
    constexpr int TH = 16;
    const CamDev* cams = a.ws.cams;
    const int t = blockIdx.x;
    const int v = find_view(cams, a.B, t);
    const int lt = t - __ldg(&cams[v].tile_base);
    const int tiles_x = __ldg(&cams[v].tiles_x);
    const int tx = lt % tiles_x, ty = lt / tiles_x;
    const int H = __ldg(&cams[v].H), W = __ldg(&cams[v].W);
    const float invF = __ldg(&cams[v].invF);
    const int tid = threadIdx.x;
    const int j = tx * kTileW + (tid & 15);
    const int i = ty * TH + (tid >> 4);
    if (i >= H || j >= W) return;
    const float px = (float)j + 0.5f, py = (float)i + 0.5f;
    const int64_t pix = __ldg(&cams[v].pix_base) + (int64_t)i * W + j;
    const int64_t vb = (int64_t)v * a.N;
    const int L = a.L, C = a.C;
    const int32_t* li = a.index_in + pix * L;
    float* S = a.ws.gkey + pix * (int64_t)L * 8;
    int n = 0;
    while (n < L) {
        const int32_t g = li[n];
        if (g < 0 || g >= a.N) break;
        float4 r0, r1, r2, r3;
        load_rec(a.ws.rec, vb + g, r0, r1, r2, r3);
        const Entry e = entry_px(r0, r1, r2, r3, px, py);
        float* s = S + 8 * n;
        s[0] = e.hi; s[1] = e.lo; s[2] = e.r; s[3] = 0.5f * e.a;
        s[4] = 0.0f; s[5] = 0.0f; s[6] = 0.0f; s[7] = 0.0f;
        ++n;
    }
    const float* gp = a.grad_image + pix * C;
    for (int k = 0; k < n; ++k) {
        float* sk = S + 8 * k;
        float A = 0.0f;
        for (int jj = 0; jj < n; ++jj) {
            const float* sj = S + 8 * jj;
            const float u = ((sk[0] - sj[0]) + (sk[1] - sj[1])) * sj[2];
            const float q = erfc_as28(fabsf(u));
            const float sm = copysignf(sj[3], u);
            A = fmaf(-sm, q, A + (sj[3] + sm));
        }
        const float Wk = ex2_approx(-a.tau * kLog2e * A) * (2.0f * sk[3]);
        const int32_t g = li[k];
        float G = 0.0f;
        for (int c = 0; c < C; ++c) {
            const float gc = gp[c];
            G = fmaf(gc, __ldg(a.attr + (int64_t)g * C + c), G);
            if (a.grad_attr) atomicAdd(a.grad_attr + (int64_t)g * C + c, Wk * gc);
        }
        sk[4] = -a.tau * G * Wk;
    }
    for (int k = 0; k < n; ++k) {
        float* sk = S + 8 * k;
        for (int jj = 0; jj < n; ++jj) {
            float* sj = S + 8 * jj;
            const float d = (sk[0] - sj[0]) + (sk[1] - sj[1]);
            const float u = d * sj[2];
            float g2;
            const float ec = erfc_as26(fabsf(u), g2);
            const float E = copysignf(1.0f - ec, u);
            sj[6] = fmaf(sk[4], 1.0f + E, sj[6]);
            const float du = sk[4] * sj[3] * kTwoOverSqrtPi * g2;
            sk[5] = fmaf(du, sj[2], sk[5]);
            sj[5] = fmaf(-du, sj[2], sj[5]);
            sj[7] = fmaf(du, d, sj[7]);
        }
    }
    const float inv2tau = 0.5f / a.tau;
    for (int k = 0; k < n; ++k) {
        const float* sk = S + 8 * k;
        const float dqt = fmaf(sk[4], inv2tau, -0.5f * sk[3] * sk[6]);  // a/4 = m/2
        const float db = sk[7] / (4.0f * sk[2]);
        float gv[9];
        chain_to_camera(a, vb + li[k], px, py, invF, dqt, sk[5], db, gv);
        float* gc = a.ws.gcam + 9 * (vb + li[k]);
        for (int q = 0; q < 9; ++q) atomicAdd(gc + q, gv[q]);
    }
}

// Camera-space accumulators -> world-space gradients of means and inverse
// covariances (M = R M_w + T, P = R P_w Rᵀ), and dL/dR = dM M_wᵀ + 2 G R P_w,
// dL/dT = dM reduced over Gaussians per view.
__global__ void __launch_bounds__(256) k_grad_finalize(Args a, float* grad_means, float* grad_inv_cov, float* grad_cam) {
    __shared__ float red[8][12];
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = g < a.N;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    float gm[3] = {0.f, 0.f, 0.f}, gw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    float Mw[3] = {0.f, 0.f, 0.f}, Pw[9];
    if (live) {
        for (int q = 0; q < 3; ++q) Mw[q] = __ldg(a.means + 3 * (int64_t)g + q);
        const float* p6 = a.inv_cov + 6 * (int64_t)g;
        Pw[0] = __ldg(p6 + 0); Pw[1] = __ldg(p6 + 1); Pw[2] = __ldg(p6 + 2);
        Pw[3] = Pw[1]; Pw[4] = __ldg(p6 + 3); Pw[5] = __ldg(p6 + 4);
        Pw[6] = Pw[2]; Pw[7] = Pw[5]; Pw[8] = __ldg(p6 + 5);
    } else {
        for (int q = 0; q < 9; ++q) Pw[q] = 0.0f;
    }
    for (int v = 0; v < a.B; ++v) {
        float R[9];
        for (int q = 0; q < 9; ++q) R[q] = __ldg(&a.ws.cams[v].R[q]);
        float dM[3] = {0.f, 0.f, 0.f}, G[9];
        for (int q = 0; q < 9; ++q) G[q] = 0.0f;
        if (live) {
            const float* gc = a.ws.gcam + 9 * ((int64_t)v * a.N + g);
            dM[0] = gc[0]; dM[1] = gc[1]; dM[2] = gc[2];
            G[0] = gc[3]; G[1] = gc[4]; G[2] = gc[5];
            G[3] = gc[4]; G[4] = gc[6]; G[5] = gc[7];
            G[6] = gc[5]; G[7] = gc[7]; G[8] = gc[8];
        }
        // world mean gradient Rᵀ dM
        for (int q = 0; q < 3; ++q) gm[q] += R[q] * dM[0] + R[3 + q] * dM[1] + R[6 + q] * dM[2];
        // world P gradient Rᵀ G R
        float GR[9];
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) GR[3 * x + y] = G[3 * x] * R[y] + G[3 * x + 1] * R[3 + y] + G[3 * x + 2] * R[6 + y];
        float Gw[9];
        for (int x = 0; x < 3; ++x)
            for (int y = 0; y < 3; ++y) Gw[3 * x + y] = R[x] * GR[y] + R[3 + x] * GR[3 + y] + R[6 + x] * GR[6 + y];
        gw[0] += Gw[0]; gw[1] += Gw[1] + Gw[3]; gw[2] += Gw[2] + Gw[6];
        gw[3] += Gw[4]; gw[4] += Gw[5] + Gw[7]; gw[5] += Gw[8];
        if (grad_cam) {
            // pose: dR = dM Mwᵀ + 2 G (R Pw), dT = dM
            float RP[9];
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y) RP[3 * x + y] = R[3 * x] * Pw[y] + R[3 * x + 1] * Pw[3 + y] + R[3 * x + 2] * Pw[6 + y];
            float p[12];
            for (int x = 0; x < 3; ++x)
                for (int y = 0; y < 3; ++y)
                    p[3 * x + y] = dM[x] * Mw[y] + 2.0f * (G[3 * x] * RP[y] + G[3 * x + 1] * RP[3 + y] + G[3 * x + 2] * RP[6 + y]);
            p[9] = dM[0]; p[10] = dM[1]; p[11] = dM[2];
            for (int q = 0; q < 12; ++q) {
                float x = p[q];
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                p[q] = x;
            }
            if (lane == 0)
                for (int q = 0; q < 12; ++q) red[wid][q] = p[q];
            __syncthreads();
            if (threadIdx.x < 12) {
                float s = 0.0f;
                for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w][threadIdx.x];
                atomicAdd(grad_cam + 12 * v + threadIdx.x, s);
            }
            __syncthreads();
        }
    }
    if (!live) return;
    if (grad_means)
        for (int q = 0; q < 3; ++q) grad_means[3 * (int64_t)g + q] += gm[q];
    if (grad_inv_cov)
        for (int q = 0; q < 6; ++q) grad_inv_cov[6 * (int64_t)g + q] += gw[q];
}

template <typename Kern>
static cudaError_t launch_tiles(Kern k, const char* name, int nblocks, int nthreads, size_t smem, cudaStream_t s,
                                const Args& a) {
    TraceScope tr(name, s);
    if (smem > 48 * 1024) {
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<nblocks, nthreads, smem, s>>>(a);
    return cudaPeekAtLastError();
}

template <int KM, int TH>
static size_t backward_smem_bytes() {
    return (size_t)KM * 16 * TH * 16;
}

// Launch the backward tile kernel for register-list capacity KM (0 = generic).
cudaError_t launch_backward_tiles(int KM, int nblocks, cudaStream_t s, const Args& a) {
    switch (KM) {
        case 8: return launch_tiles(k_backward<8, 16>, "k_backward<8>", nblocks, 256, backward_smem_bytes<8, 16>(), s, a);
        case 16: return launch_tiles(k_backward<16, 16>, "k_backward<16>", nblocks, 256, backward_smem_bytes<16, 16>(), s, a);
        case 20: return launch_tiles(k_backward<20, 16>, "k_backward<20>", nblocks, 256, backward_smem_bytes<20, 16>(), s, a);
        case 24: return launch_tiles(k_backward<24, 16>, "k_backward<24>", nblocks, 256, backward_smem_bytes<24, 16>(), s, a);
        case 32: return launch_tiles(k_backward<32, 8>, "k_backward<32>", nblocks, 128, backward_smem_bytes<32, 8>(), s, a);
        default: return launch_tiles(k_backward_generic, "k_backward_generic", nblocks, 256, 0, s, a);
    }
}

cudaError_t launch_grad_finalize(int N, cudaStream_t s, const Args& a, float* grad_means, float* grad_inv_cov,
                                 float* grad_cam) {
    TraceScope tr("k_grad_finalize", s);
    k_grad_finalize<<<(unsigned)((N + 255) / 256), 256, 0, s>>>(a, grad_means, grad_inv_cov, grad_cam);
    return cudaPeekAtLastError();
}

}  // namespace voge
