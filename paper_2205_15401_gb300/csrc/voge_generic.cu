// voge_generic.cu -- forward and backward for kept lists longer than the
// register lists (L > 32, including K = all): one warp per pixel.
//
// Selection (Sec. 3.3, App. A.3): the lanes trace the pixel's candidates 32
// at a time (Eq. 6: l, e^{q}; keep e^{q} > eta, l > 0).  The chunk's kept
// candidates are sorted by (l, index) with a warp bitonic network and merged
// into the pixel's sorted list, which lives in the workspace (two buffers,
// ping-pong): every output position finds its co-rank by binary search, so
// the merge is spread over the lanes.  Candidates sorted by a depth lower
// bound stop once the list is full and the next chunk starts beyond it.
//
// Fine pass (Eq. 7-8): the lanes take the list's entries; each sets up its
// entries (l as two floats, r = sqrt(b/2), m = a/2), then sums its A_k over
// the whole list, read back from the workspace with every lane on the same
// entry (one broadcast load per step).
//
// Backward (frozen lists): the same entries; the pair adjoint runs with the
// j side as the outer loop, each lane adding its k entries' terms, and the
// j-side sums (dm_j, dl_j, dr_j) reduced over the warp by shuffles; the
// chain rule to camera space then takes one entry per lane.
//
// Per-pixel scratch: the workspace's [pixels][L][8] floats.
//   forward:  [0] [1] list key / id (buffer 0), [2] [3] (buffer 1), [4..7] entry
//   backward: [0..3] entry (hi, lo, r, m), [4] dA, [5] dl, [6] dm, [7] dr
#include "voge_device.cuh"
#include "voge_trace.cuh"

namespace voge {

namespace {

constexpr unsigned kFull = 0xffffffffu;
constexpr float kTwoOverSqrtPiG = 1.1283791670955126f;

// (l, g) strictly before (l2, g2) in list order
__device__ __forceinline__ bool before(float l, int32_t g, float l2, int32_t g2) {
    return l < l2 || (l == l2 && g < g2);
}

// Warp bitonic sort of 32 (key, id) pairs, one per lane, ascending in lane order.
__device__ __forceinline__ void warp_sort32(float& key, int32_t& id, int lane) {
#pragma unroll
    for (int size = 2; size <= 32; size <<= 1) {
#pragma unroll
        for (int stride = size >> 1; stride > 0; stride >>= 1) {
            const float ok = __shfl_xor_sync(kFull, key, stride);
            const int32_t oi = __shfl_xor_sync(kFull, id, stride);
            const bool up = (lane & size) == 0;        // this block sorts ascending
            const bool lower = (lane & stride) == 0;   // this lane keeps the smaller one
            const bool other_first = before(ok, oi, key, id);
            const bool take = (lower == up) ? other_first : !other_first;
            if (take) {
                key = ok;
                id = oi;
            }
        }
    }
}

// Pixel of a global pixel index: its view (binary search over pix_base).
__device__ __forceinline__ int view_of_pixel(const ViewDesc* __restrict__ vd, int nv, int64_t p) {
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&vd[mid].pix_base) <= p) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

struct GenPixel {
    int v, i, j, tile;
};
__device__ __forceinline__ GenPixel gen_pixel(const Args& a, int64_t gp) {
    GenPixel q;
    q.v = view_of_pixel(a.views, a.hdr->nviews, gp);
    const ViewDesc& vd = a.views[q.v];
    const int64_t lp = gp - vd.pix_base;
    q.i = (int)(lp / vd.W);
    q.j = (int)(lp - (int64_t)q.i * vd.W);
    q.tile = vd.tile_base + (q.i / vd.tile_h) * vd.tiles_x + q.j / kTileW;
    return q;
}

__device__ __forceinline__ float* scratch_of(const Args& a, const ViewDesc& vd, int64_t pix) {
    return a.ws.gkey + (vd.pix_base + pix) * (int64_t)a.ws.gen_L * 8;
}

}  // namespace

// ---------------------------------------------------------------------------
// Forward: one warp per pixel (eight per CTA).
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_render_generic(Args a, int64_t total_pixels) {
    const int lane = threadIdx.x & 31;
    const int64_t gp = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (gp >= total_pixels) return;  // whole warp
    const GenPixel q = gen_pixel(a, gp);
    const ViewDesc& vd = a.views[q.v];
    const int W = vd.W, L = vd.L, C = vd.C, N = vd.N;
    const int64_t pix = (int64_t)q.i * W + q.j;
    const int64_t vb = vd.rec_base;
    const float px = (float)q.j + 0.5f, py = (float)q.i + 0.5f;
    float* S = scratch_of(a, vd, pix);
    if (VOGE_IDX(a.hdr, L, (int64_t)a.ws.gen_L + 1, kChkScratch) != L) return;  // scratch laid out for shorter lists

    // candidate source of the pixel's tile
    int mode, count, start = 0, filter_box = 0;
    const int tx = q.j / kTileW, ty = q.i / vd.tile_h;
    if (vd.plain) {
        mode = 2;
        count = N;
    } else {
        const int tc = (int)VOGE_IDX(a.hdr, q.tile, a.hdr->total_tiles, kChkTile);
        const int cnt = a.ws.tile_cnt[tc], off = a.ws.tile_off[tc];
        if ((int64_t)off + cnt > a.ws.bin_cap) {
            mode = 2;
            count = N;
            filter_box = 1;
        } else {
            mode = (vd.use_thresh && cnt > 1 && cnt <= kSortMax) ? 1 : 0;
            count = cnt;
            start = off;
        }
    }

    int n = 0, cur = 0;  // list length, current buffer
    float kmax = INFINITY;
    int32_t gmax = INT32_MAX;
    unsigned traced = 0;
    for (int base = 0; base < count; base += 32) {
        const int qi = base + lane;
        float l = 0.0f;
        int32_t g = -1;
        float lmin = INFINITY;
        if (qi < count) {
            g = mode == 2 ? qi : a.ws.tile_gauss[VOGE_IDX(a.hdr, start + qi, a.ws.bin_cap, kChkTileList)];
            g = (int32_t)VOGE_IDX(a.hdr, g, N, kChkRecord);
            float4 r0, r1, r2, r3;
            load_rec(a.ws.rec, vb + g, r0, r1, r2, r3);
            lmin = r3.w;
            bool outside = false;
            if (filter_box) {
                const int4 tb = a.ws.tbox[vb + g];
                outside = tx < tb.x || tx > tb.y || ty < tb.z || ty > tb.w;
            }
            if (!outside) {
                l = candidate_key(r0, r1, r2, r3, px, py, vd.Qeta);
                ++traced;
            }
        }
        // sorted by the depth lower bound: a full list ends the walk once the
        // chunk's first candidate starts beyond its last entry
        if (mode == 1 && n == L && __shfl_sync(kFull, lmin, 0) > kmax) break;
        const bool keep = l > 0.0f && (n < L || before(l, g, kmax, gmax));
        const unsigned ballot = __ballot_sync(kFull, keep);
        if (ballot == 0u) continue;
        const int m = __popc(ballot);
        float bk = keep ? l : INFINITY;
        int32_t bi = keep ? g : INT32_MAX;
        warp_sort32(bk, bi, lane);  // lanes [0, m) hold the chunk's kept candidates in order
        // merge the sorted list (n, buffer cur) with the chunk (m): output
        // position o takes a of its first o from the list, by binary search
        const int nc = min(L, n + m);
        float* A = S + 2 * cur;
        float* Cb = S + 2 * (cur ^ 1);
        for (int o0 = 0; o0 < nc; o0 += 32) {
            const int o = o0 + lane;
            int lo = max(0, o - m), hi = min(o, n);
            bool busy = o < nc;
            // uniform loop: every lane joins the shuffles
            while (__any_sync(kFull, busy && lo < hi)) {
                const bool act = busy && lo < hi;
                const int mid = act ? (lo + hi) >> 1 : 0;
                const int bidx = act ? o - mid - 1 : 0;
                const float kb = __shfl_sync(kFull, bk, bidx & 31);
                const int32_t ib = __shfl_sync(kFull, bi, bidx & 31);
                if (act) {
                    const float ka = A[8 * mid];
                    const int32_t ia = __float_as_int(A[8 * mid + 1]);
                    if (before(ka, ia, kb, ib)) lo = mid + 1;
                    else hi = mid;
                }
            }
            const int ai = lo, bidx = o - lo;
            const float kb = __shfl_sync(kFull, bk, min(bidx, 31) & 31);
            const int32_t ib = __shfl_sync(kFull, bi, min(bidx, 31) & 31);
            if (busy) {
                float ko;
                int32_t io;
                if (bidx >= m || (ai < n && before(A[8 * ai], __float_as_int(A[8 * ai + 1]), kb, ib))) {
                    ko = A[8 * ai];
                    io = __float_as_int(A[8 * ai + 1]);
                } else {
                    ko = kb;
                    io = ib;
                }
                Cb[8 * o] = ko;
                Cb[8 * o + 1] = __int_as_float(io);
            }
        }
        __syncwarp();
        cur ^= 1;
        n = nc;
        if (n == L) {
            kmax = S[8 * (n - 1) + 2 * cur];
            gmax = __float_as_int(S[8 * (n - 1) + 2 * cur + 1]);
        }
    }
    {
        const unsigned w_traced = __reduce_add_sync(kFull, traced);
        if (lane == 0) {
            atomicAdd(&a.hdr->traces, (unsigned long long)w_traced);
            atomicAdd(&a.hdr->entries, (unsigned long long)n);
            atomicAdd(&a.hdr->pairs, (unsigned long long)n * (unsigned long long)n);
        }
    }
    const float* LS = S + 2 * cur;  // the sorted list: key at [8k], id at [8k + 1]

    // entries
    for (int k = lane; k < n; k += 32) {
        float4 r0, r1, r2, r3;
        load_rec(a.ws.rec, vb + VOGE_IDX(a.hdr, __float_as_int(LS[8 * k + 1]), N, kChkRecord), r0, r1, r2, r3);
        const Entry en = entry_px(r0, r1, r2, r3, px, py);
        *reinterpret_cast<float4*>(S + 8 * k + 4) = make_float4(en.hi, en.lo, en.r, 0.5f * en.a);
    }
    __syncwarp();
    // A_k over the whole list (one broadcast load per j), W_k into the free key slot
    float msum = 0.0f;
    for (int k = lane; k < n; k += 32) msum += S[8 * k + 7];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(kFull, msum, o);
    const float ntl = -vd.tau * kLog2e;
    float* WS = S + 2 * (cur ^ 1);  // W_k at [8k]
    for (int k0 = 0; k0 < n; k0 += 32) {
        const int k = k0 + lane;
        float A0 = 0.0f, A1 = 0.0f;
        float4 Kq = make_float4(0.f, 0.f, 0.f, 0.f);
        if (k < n) Kq = *reinterpret_cast<const float4*>(S + 8 * k + 4);
        int jj = 0;
        for (; jj + 1 < n; jj += 2) {
            const float4 J0 = *reinterpret_cast<const float4*>(S + 8 * jj + 4);
            const float4 J1 = *reinterpret_cast<const float4*>(S + 8 * (jj + 1) + 4);
            const float u0 = ((Kq.x - J0.x) + (Kq.y - J0.y)) * J0.z;
            const float u1 = ((Kq.x - J1.x) + (Kq.y - J1.y)) * J1.z;
            A0 = fmaf(copysignf(J0.w, u0), 1.0f - erfc_as28(fabsf(u0)), A0);
            A1 = fmaf(copysignf(J1.w, u1), 1.0f - erfc_as28(fabsf(u1)), A1);
        }
        if (jj < n) {
            const float4 J0 = *reinterpret_cast<const float4*>(S + 8 * jj + 4);
            const float u0 = ((Kq.x - J0.x) + (Kq.y - J0.y)) * J0.z;
            A0 = fmaf(copysignf(J0.w, u0), 1.0f - erfc_as28(fabsf(u0)), A0);
        }
        if (k < n) WS[8 * k] = ex2_approx(ntl * (msum + (A0 + A1))) * (2.0f * Kq.w);
    }
    __syncwarp();
    // outputs: index and weights in list order (padded), image = sum_k W_k c_k
    for (int k = lane; k < L; k += 32) {
        const bool in = k < n;
        const int64_t o = VOGE_IDX(a.hdr, pix * L + k, (int64_t)vd.H * W * L, kChkOutput);
        vd.index[o] = in ? __float_as_int(LS[8 * k + 1]) : -1;
        if (vd.weights) vd.weights[o] = in ? WS[8 * k] : 0.0f;
    }
    float* img = vd.image + pix * C;
    if (C <= 32) {
        for (int c = 0; c < C; ++c) {
            float acc = 0.0f;
            for (int k = lane; k < n; k += 32)
                acc = fmaf(WS[8 * k], __ldg(vd.attr + (int64_t)__float_as_int(LS[8 * k + 1]) * C + c), acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
            if (lane == 0) img[c] = acc;
        }
    } else {
        for (int c0 = 0; c0 < C; c0 += 32) {
            const int c = c0 + lane;
            float acc = 0.0f;
            for (int k = 0; k < n; ++k)
                if (c < C) acc = fmaf(WS[8 * k], __ldg(vd.attr + (int64_t)__float_as_int(LS[8 * k + 1]) * C + c), acc);
            if (c < C) img[c] = acc;
        }
    }
}

// ---------------------------------------------------------------------------
// Backward with frozen lists: one warp per pixel (eight per CTA).
//   dc_k += W_k g_p,  G_k = g_p . c_k,  dA_k = -tau G_k W_k,
//   dm_j += dA_k (1 + erf u_kj),  du_kj = dA_k m_j (2/sqrt(pi)) e^{-u_kj^2},
//   dl_k += du r_j,  dl_j -= du r_j,  dr_j += du (l_k - l_j),
// then the chain to camera space as in the tile kernels.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_backward_generic(Args a, int64_t total_pixels) {
    constexpr int kT = 8;  // k entries per lane and block: 256 per block
    const int lane = threadIdx.x & 31;
    const int64_t gp = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
    if (gp >= total_pixels) return;  // whole warp
    const GenPixel q = gen_pixel(a, gp);
    const ViewDesc& vd = a.views[q.v];
    const int W = vd.W, L = vd.L, C = vd.C, N = vd.N;
    const int64_t pix = (int64_t)q.i * W + q.j;
    const int64_t vb = vd.rec_base;
    const float px = (float)q.j + 0.5f, py = (float)q.i + 0.5f;
    const float tau = vd.tau, invF = vd.invF;
    float* S = scratch_of(a, vd, pix);
    const int32_t* li = vd.index_in + pix * L;
    if (VOGE_IDX(a.hdr, L, (int64_t)a.ws.gen_L + 1, kChkScratch) != L) return;  // scratch laid out for shorter lists

    // the list: entries before the first one outside [0, N)
    int n = L;
    for (int k0 = 0; k0 < L; k0 += 32) {
        const int k = k0 + lane;
        const int32_t g = k < L ? __ldg(li + k) : 0;
        const unsigned bad = __ballot_sync(kFull, k < L && !(g >= 0 && g < N));
        if (bad) {
            n = k0 + __ffs(bad) - 1;
            break;
        }
    }
    if (n == 0) return;
    for (int k = lane; k < n; k += 32) {
        float4 r0, r1, r2, r3;
        load_rec(a.ws.rec, vb + VOGE_IDX(a.hdr, __ldg(li + k), N, kChkRecord), r0, r1, r2, r3);
        const Entry en = entry_px(r0, r1, r2, r3, px, py);
        *reinterpret_cast<float4*>(S + 8 * k) = make_float4(en.hi, en.lo, en.r, 0.5f * en.a);
        *reinterpret_cast<float4*>(S + 8 * k + 4) = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    __syncwarp();
    // W_k (from the forward, else recomputed), G_k, dA_k and the attribute gradient
    const float* gpx = vd.grad_image + pix * C;
    const float* wi = vd.weights_in ? vd.weights_in + pix * L : nullptr;
    float msum = 0.0f;
    if (!wi) {
        for (int k = lane; k < n; k += 32) msum += S[8 * k + 3];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) msum += __shfl_xor_sync(kFull, msum, o);
    }
    const float ntl = -tau * kLog2e;
    for (int k = lane; k < n; k += 32) {
        const float4 Kq = *reinterpret_cast<const float4*>(S + 8 * k);
        float Wk;
        if (wi) {
            Wk = __ldg(wi + k);
        } else {
            float A0 = 0.0f;
            for (int jj = 0; jj < n; ++jj) {
                const float4 J = *reinterpret_cast<const float4*>(S + 8 * jj);
                const float u = ((Kq.x - J.x) + (Kq.y - J.y)) * J.z;
                A0 = fmaf(copysignf(J.w, u), 1.0f - erfc_as28(fabsf(u)), A0);
            }
            Wk = ex2_approx(ntl * (msum + A0)) * (2.0f * Kq.w);
        }
        const int32_t g = __ldg(li + k);
        const float* ck = vd.attr + (int64_t)g * C;
        float G = 0.0f;
        for (int c = 0; c < C; ++c) {
            const float gc = __ldg(gpx + c);
            G = fmaf(gc, __ldg(ck + c), G);
            if (vd.grad_attr) atomicAdd(vd.grad_attr + (int64_t)g * C + c, Wk * gc);
        }
        S[8 * k + 4] = -tau * G * Wk;
    }
    __syncwarp();
    // pair adjoint: the j side outer, each lane's k entries (blocks of 256) in registers
    for (int kb0 = 0; kb0 < n; kb0 += 32 * kT) {
        const int T = min(kT, (n - kb0 + 31) / 32);  // warp-uniform
        float hk[kT], lk[kT], dAk[kT], dlk[kT];
#pragma unroll
        for (int t = 0; t < kT; ++t) {
            const int k = kb0 + 32 * t + lane;
            const bool in = t < T && k < n;
            hk[t] = in ? S[8 * k] : 0.0f;
            lk[t] = in ? S[8 * k + 1] : 0.0f;
            dAk[t] = in ? S[8 * k + 4] : 0.0f;  // zero dA: no contribution
            dlk[t] = 0.0f;
        }
        for (int jj = 0; jj < n; ++jj) {
            const float4 J = *reinterpret_cast<const float4*>(S + 8 * jj);
            const float mj = J.w * kTwoOverSqrtPiG;
            float acc_dm = 0.0f, acc_s = 0.0f, acc_dr = 0.0f;
#pragma unroll
            for (int t = 0; t < kT; ++t) {
                if (t < T) {
                    const float d = (hk[t] - J.x) + (lk[t] - J.y);
                    const float u = d * J.z;
                    float g2;
                    const float ec = erfc_as26(fabsf(u), g2);
                    const float E = copysignf(1.0f - ec, u);
                    acc_dm = fmaf(dAk[t], 1.0f + E, acc_dm);
                    const float du = dAk[t] * mj * g2;
                    dlk[t] = fmaf(du, J.z, dlk[t]);
                    acc_s += du;
                    acc_dr = fmaf(du, d, acc_dr);
                }
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) {
                acc_dm += __shfl_xor_sync(kFull, acc_dm, o);
                acc_s += __shfl_xor_sync(kFull, acc_s, o);
                acc_dr += __shfl_xor_sync(kFull, acc_dr, o);
            }
            if (lane == 0) {
                S[8 * jj + 5] -= acc_s * J.z;
                S[8 * jj + 6] += acc_dm;
                S[8 * jj + 7] += acc_dr;
            }
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < kT; ++t) {
            const int k = kb0 + 32 * t + lane;
            if (t < T && k < n) S[8 * k + 5] += dlk[t];
        }
        __syncwarp();
    }
    // chain rule to camera space, one entry per lane
    const float inv2tau = 0.5f / tau;
    for (int k = lane; k < n; k += 32) {
        const float4 e0 = *reinterpret_cast<const float4*>(S + 8 * k);
        const float4 e1 = *reinterpret_cast<const float4*>(S + 8 * k + 4);
        const float dqt = fmaf(e1.x, inv2tau, -0.5f * e0.w * e1.z);  // a/4 = m/2
        const float db = e1.w / (4.0f * e0.z);
        const int64_t o = vb + __ldg(li + k);
        float4 r0, r1, r2, r3;
        load_rec(a.ws.rec, o, r0, r1, r2, r3);
        const Trace tr = trace_px(r0, r1, r2, r3, px, py);
        float gv[9];
        chain_to_camera(__ldg(a.ws.rec2 + 2 * o), __ldg(a.ws.rec2 + 2 * o + 1), tr, r3, invF, dqt, e1.y, db, gv);
        float* gc = a.ws.gcam + kGcamStride * o;
        red_add_v4(gc, gv[0], gv[1], gv[2], gv[3]);
        red_add_v4(gc + 4, gv[4], gv[5], gv[6], gv[7]);
        red_add_v4(gc + 8, gv[8], 0.0f, 0.0f, 0.0f);
    }
}

// One warp per pixel, eight pixels per CTA.
cudaError_t launch_render_generic(int64_t total_pixels, cudaStream_t s, const Args& a) {
    if (total_pixels <= 0) return cudaSuccess;
    TraceScope tr("k_render_generic", s);
    k_render_generic<<<(unsigned)((total_pixels + 7) / 8), 256, 0, s>>>(a, total_pixels);
    return cudaPeekAtLastError();
}

cudaError_t launch_backward_generic(int64_t total_pixels, cudaStream_t s, const Args& a) {
    if (total_pixels <= 0) return cudaSuccess;
    TraceScope tr("k_backward_generic", s);
    k_backward_generic<<<(unsigned)((total_pixels + 7) / 8), 256, 0, s>>>(a, total_pixels);
    return cudaPeekAtLastError();
}

}  // namespace voge
