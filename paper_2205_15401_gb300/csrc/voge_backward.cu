// voge_backward.cu -- adjoint of the forward pass with the kept lists frozen.
//
// The per-pixel index lists come from the forward pass, and its weights W_k
// when the caller passes them (voge_render_bwd_w); l, e^{q}, sigma, every erf
// term of Eq. 7 and, without the weights, T(l_k) are recomputed here.  For a pixel
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
// reduced into the camera pose by the finalize kernels at the end of this
// file.
#include "voge_device.cuh"
#include "voge_trace.cuh"

namespace voge {

constexpr float kTwoOverSqrtPi = 1.1283791670955126f;

// Entries per step of the chain rule's loop (their gathers are in flight
// together; 4 measured faster than 2 or 3), and entries per lane per step of
// the packed set-up (2 measured faster than 3 or 4).
#ifndef VOGE_CHAIN_STEP
#define VOGE_CHAIN_STEP 4
#endif
constexpr int kChainStep = VOGE_CHAIN_STEP;
#ifndef VOGE_SETUP_STEP
#define VOGE_SETUP_STEP 2
#endif
constexpr int kSetupStep = VOGE_SETUP_STEP;
// Matching lane pairs a warp needs before it aggregates its reductions.
#ifndef VOGE_AGG_PAIRS
#define VOGE_AGG_PAIRS 4
#endif
constexpr int kAggPairs = VOGE_AGG_PAIRS;

// How a tile adds the attribute gradient dL/dc_g += W_k dL/dI:
//   kAttrLane:  one reduction per lane and channel (4 <= C < 8),
//   kAttrWarp:  warp-cooperative rows, lanes over (source pixel, channel) (C >= 8),
//   kAttrChain: C <= 3, W_k (the forward's weights when supplied, else kept
//               in shared memory) added with the third camera-space vector
//               reduction of the chain rule (slots 9..11 of the record's 12
//               floats, free otherwise), folded into grad_attr by the
//               finalize kernel,
//   kAttrSlot:  C <= 3 for classes without room for W_k in shared memory: the
//               same slots, with one vector reduction of their own.
//   kAttrPacked: kAttrChain with the forward's W_k supplied, the entries set
//               up packed over the lanes (k_backward_packed, its own kernel
//               so that its registers do not weigh on the other forms).
constexpr int kAttrLane = 0, kAttrWarp = 1, kAttrChain = 2, kAttrSlot = 3, kAttrPacked = 4;

// Classes whose W_k buffer fits next to the stream without losing a block per SM.
template <int KM, int TH>
__host__ __device__ constexpr bool wk_in_smem() { return KM <= 20; }

// Packed backward: index lists staged per warp as [pixel of the row pair]
// [stride], stride = L rounded up to odd, so that lanes reading one list
// position of their pixels hit distinct banks.
__host__ __device__ constexpr int packed_stride(int L) { return L | 1; }
template <int KM>
__host__ __device__ constexpr int packed_warp_words() { return 32 * packed_stride(KM); }

// The calling warp's asynchronous copies of the index lists of unit
// (t, hb, q) of view v into its staging rows sw: consecutive lanes take
// consecutive words of a row segment's [16][L] block (word x is list position
// x % L of column x / L; L <= 20 < 32, so one carry per step), landing on
// consecutive words of sw.  Pixels outside the image are never read.  One
// commit group.
__device__ __forceinline__ void stage_lists_packed(const Args& a, int32_t* sw, int v, int t, int hb, int q) {
    constexpr int TH = 8;
    const ViewDesc& vd = a.views[v];
    const int lt = t - vd.tile_base;
    const int tx = lt % vd.tiles_x, ty = lt / vd.tiles_x;
    const int H = vd.H, W = vd.W, L = vd.L, S = packed_stride(L);
    const int row0 = ty * vd.tile_h + hb * TH + 2 * q;
    const int lane = threadIdx.x & 31;
    const int ncols = min(kTileW, W - tx * kTileW);
    const int dc = 32 / L, dk = 32 - dc * L;
#pragma unroll
    for (int rw = 0; rw < 2; ++rw) {
        const int irow = row0 + rw;
        const int cnt = irow < H ? ncols * L : 0;
        int64_t o0 = ((int64_t)irow * W + tx * kTileW) * L;
        if (cnt > 0) o0 = VOGE_IDX(a.hdr, o0 + cnt - 1, (int64_t)H * W * L, kChkListRead) - (cnt - 1);
        const int32_t* src = vd.index_in + o0;
        int col = lane / L, k = lane - col * L;
        int32_t* dst = sw + 16 * rw * S;
        for (int x = lane; x < cnt; x += 32) {
            cp_async4(dst + col * S + k, src + x);
            k += dk;
            col += dc;
            if (k >= L) {
                k -= L;
                ++col;
            }
        }
    }
    cp_async_commit();
}

struct NoHook {
    __device__ void operator()() const {}
};

// Rows 2q and 2q + 1 of one backward tile, rows [hb TH, hb TH + TH) of
// binning tile t of view v (v < 0: looked up) -- the backward reads the index
// lists, not the tile lists, so it may split the forward's tiles into shorter
// ones -- for the calling warp, in its warp's shared-memory columns.  The
// packed form finds its lists already staged in its warp's rows of the W_k
// buffer (stage_lists_packed).  The set-up replaces them with the entries'
// dA_k; once those are in registers, restage() copies this unit's lists in
// again (they arrive during the pair terms), and once the chain rule has
// taken the indices into the stream, next() may stage the caller's next unit.
template <int KM, int TH, int AM, typename Restage = NoHook, typename Hook = NoHook>
__device__ __forceinline__ void backward_tile(const Args& a, int t, int hb, int q, int v = -1,
                                              Restage restage = Restage(), Hook next = Hook()) {
    constexpr int NT = 16 * TH;
    extern __shared__ float4 smem[];
    float4* jst = smem;  // [KM][NT]
    float* swk = reinterpret_cast<float*>(jst + KM * NT);  // [KM][NT] W_k (kAttrChain)

    if (v < 0) v = view_of_tile(a.views, a.hdr->nviews, t);
    const ViewDesc& vd = a.views[v];
    const int lt = t - vd.tile_base;
    const int tiles_x = vd.tiles_x;
    const int tx = lt % tiles_x, ty = lt / tiles_x;
    const int H = vd.H, W = vd.W;
    const float invF = vd.invF;
    const int tid = threadIdx.x;
    const int row0 = ty * vd.tile_h + hb * TH + 2 * q;  // first pixel row of this warp's pair
    const int j = tx * kTileW + (tid & 15);
    const int i = row0 + ((tid >> 4) & 1);
    const bool valid = (i < H) && (j < W);
    const float px = (float)j + 0.5f, py = (float)i + 0.5f;
    const int64_t pix = (int64_t)i * W + j;
    const int64_t vb = vd.rec_base;
    const int L = vd.L, K = vd.L, C = vd.C, N = vd.N;
    const float tau = vd.tau;
    const float* attr = vd.attr;
    float* grad_attr = vd.grad_attr;

    constexpr bool packed = AM == kAttrPacked;
    // staged index lists of the packed set-up, in the layout of the W_k
    // buffer, which takes each entry's dA_k in place of its index once the
    // entry is set up
    const int lane = tid & 31, warp = tid >> 5;
    const int S = packed_stride(L);
    int32_t* sw = reinterpret_cast<int32_t*>(swk) + warp * packed_warp_words<KM>();  // this warp's rows
    auto stg = [&](int x) -> int32_t* {
        return reinterpret_cast<int32_t*>(jst + (x >> 7) * NT + 32 * warp) + (x & 127);
    };
    if constexpr (packed) {
        cp_async_wait<0>();
    } else {
        // each warp reads its two 16-pixel row segments (contiguous [16][L]
        // blocks) with consecutive lanes on consecutive words
        const int ncols = min(kTileW, W - tx * kTileW);
#pragma unroll
        for (int rw = 0; rw < 2; ++rw) {
            const int irow = row0 + rw;
            const int cnt = irow < H ? ncols * L : 0;
            int64_t o0 = ((int64_t)irow * W + tx * kTileW) * L;
            if (cnt > 0) o0 = VOGE_IDX(a.hdr, o0 + cnt - 1, (int64_t)H * W * L, kChkListRead) - (cnt - 1);
            const int32_t* src = vd.index_in + o0;
            for (int x = lane; x < 16 * L; x += 32) *stg(rw * 16 * L + x) = x < cnt ? __ldg(src + x) : -1;
        }
    }
    __syncwarp();
    // a warp whose 32 lists are all empty has nothing to add
    if (!__any_sync(0xffffffffu, valid && (packed ? sw[lane * S] : *stg(lane * L)) >= 0)) {
        if constexpr (packed) {
            __syncwarp();  // every lane has read its row
            next();
        }
        return;
    }
    // Kept entries occupy slots [KM - K, KM - K + n); slot s holds list
    // position k = s - (KM - K).  The indices live in registers only while
    // the entries are set up; later stages reload them from the list (the
    // rows were just read, so these hit in cache).
    float hi[KM], lo[KM], dA[KM], dl[KM];
    int n = 0;
    // With the forward's weights and narrow attributes, dA_k is formed while
    // the entries are set up (the index is in a register there).
    const float* wi = vd.weights_in ? vd.weights_in + pix * L : nullptr;
    constexpr bool kChain = AM == kAttrChain || AM == kAttrPacked;
    const bool early = wi != nullptr && C <= 3 && AM != kAttrWarp && AM != kAttrLane;
    float ga0 = 0.0f, ga1 = 0.0f, ga2 = 0.0f;
    if constexpr (packed) {
        // Set-up with the entries packed over the lanes (the forward's W_k are
        // supplied and C <= 3).  The warp's kept entries are enumerated by
        // list position first: row k holds the pixels whose lists are longer
        // than k (mask M_k, nested since lists are prefixes), so consecutive
        // lanes take neighbouring pixels at one position -- distinct shared-
        // memory banks, and often the same record.  Each entry's (l, r, m)
        // goes to the stream and dA_k replaces its staged index.
        float* sdA = reinterpret_cast<float*>(sw);
        {
            bool open = valid;
#pragma unroll
            for (int s = 0; s < KM; ++s) {
                if (s < K) {
                    const int32_t g = sw[lane * S + s];
                    open = open && g >= 0 && g < N;
                    n += open ? 1 : 0;
                }
            }
        }
        // lane k < KM holds M_k and the number of entries before row k
        unsigned mrow = 0u;
#pragma unroll
        for (int k = 0; k < KM; ++k) {
            const unsigned m = __ballot_sync(0xffffffffu, n > k);
            if (lane == k) mrow = m;
        }
        const int cnt = __popc(mrow);
        int incl = cnt;
#pragma unroll
        for (int d = 1; d < 32; d <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, d);
            if (lane >= d) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31), excl = incl - cnt;
        // every row full (all 32 pixels keep L entries): entry i is (i / 32, i % 32)
        const bool rows_full = total == 32 * K;
        for (int i0 = 0; i0 < total; i0 += 32 * kSetupStep) {
            int pp[kSetupStep], kk[kSetupStep];
            int32_t gg[kSetupStep];
            int64_t px2[kSetupStep];
#pragma unroll
            for (int h = 0; h < kSetupStep; ++h) {
                const int i = min(i0 + 32 * h + lane, total - 1);
                int k = i >> 5, p = i & 31;
                if (!rows_full) {
                    k = 0;  // the last row whose first entry is at or before i
#pragma unroll
                    for (int step = 16; step >= 1; step >>= 1) {
                        const int b = __shfl_sync(0xffffffffu, excl, k + step);
                        if (k + step < KM && b <= i) k += step;
                    }
                    // the (i - first)-th set bit of M_k, by halving popcounts
                    unsigned m = __shfl_sync(0xffffffffu, mrow, k);
                    int r = i - __shfl_sync(0xffffffffu, excl, k);
                    p = 0;
#pragma unroll
                    for (int w = 16; w >= 1; w >>= 1) {
                        const int c = __popc(m & ((1u << w) - 1u));
                        if (r >= c) {
                            r -= c;
                            m >>= w;
                            p += w;
                        }
                    }
                }
                pp[h] = p;
                kk[h] = k;
                px2[h] = (int64_t)(row0 + (p >> 4)) * W + tx * kTileW + (p & 15);
                // a lane past the last entry reads no staged index (its owner
                // may already have replaced it) and gathers record 0
                gg[h] = i0 + 32 * h + lane < total
                            ? (int32_t)VOGE_IDX(a.hdr, sw[p * S + k], N, kChkRecord)
                            : 0;
            }
            float4 r[kSetupStep][4];
            float c[kSetupStep][3], gq[kSetupStep][3], wk[kSetupStep];
#pragma unroll
            for (int h = 0; h < kSetupStep; ++h) {
                load_rec(a.ws.rec, vb + gg[h], r[h][0], r[h][1], r[h][2], r[h][3]);
                const float* ck = attr + (int64_t)gg[h] * C;
                const float* gp0 = vd.grad_image + px2[h] * C;
                c[h][0] = __ldg(ck);
                gq[h][0] = __ldg(gp0);
                c[h][1] = C > 1 ? __ldg(ck + 1) : 0.0f;
                gq[h][1] = C > 1 ? __ldg(gp0 + 1) : 0.0f;
                c[h][2] = C > 2 ? __ldg(ck + 2) : 0.0f;
                gq[h][2] = C > 2 ? __ldg(gp0 + 2) : 0.0f;
                wk[h] = __ldg(vd.weights_in + px2[h] * L + kk[h]);
            }
#pragma unroll
            for (int h = 0; h < kSetupStep; ++h) {
                if (i0 + 32 * h + lane < total) {
                    const int p = pp[h];
                    const float pxp = (float)(tx * kTileW + (p & 15)) + 0.5f;
                    const float pyp = (float)(row0 + (p >> 4)) + 0.5f;
                    const Entry e = entry_px(r[h][0], r[h][1], r[h][2], r[h][3], pxp, pyp);
                    const float G = fmaf(gq[h][2], c[h][2], fmaf(gq[h][1], c[h][1], gq[h][0] * c[h][0]));
                    jst[kk[h] * NT + 32 * warp + p] = make_float4(e.hi, e.lo, e.r, 0.5f * e.a);
                    sdA[p * S + kk[h]] = -tau * G * wk[h];
                }
            }
        }
        __syncwarp();
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            const int e = s - (KM - K);
            dl[s] = 0.0f;
            if (e >= 0 && e < n) {
                const float4 J = jst[e * NT + tid];
                hi[s] = J.x;
                lo[s] = J.y;
                dA[s] = sdA[lane * S + e];
            } else {
                hi[s] = 0.0f;
                lo[s] = 0.0f;
                dA[s] = 0.0f;
            }
        }
        __syncwarp();  // every lane has read its dA_k: the rows are free
        restage();
    } else if (early && valid) {
        const float* gp0 = vd.grad_image + pix * C;
        ga0 = __ldg(gp0);
        if (C > 1) ga1 = __ldg(gp0 + 1);
        if (C > 2) ga2 = __ldg(gp0 + 2);
    }
    if constexpr (!packed) {
        int32_t id[KM];
#pragma unroll
        for (int s = 0; s < KM; ++s) id[s] = (s >= KM - K) ? *stg(lane * L + (s - (KM - K))) : -1;
        __syncwarp();
        bool open = valid;  // lanes outside the image keep no entries but stay for the warp-wide steps
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            hi[s] = 0.0f;
            lo[s] = 0.0f;
            dA[s] = 0.0f;
            dl[s] = 0.0f;
            const int32_t g = id[s];
            if (s >= KM - K && open && g >= 0 && g < N) {
                float4 r0, r1, r2, r3;
                load_rec(a.ws.rec, vb + g, r0, r1, r2, r3);
                const Entry e = entry_px(r0, r1, r2, r3, px, py);
                hi[s] = e.hi;
                lo[s] = e.lo;
                jst[n * NT + tid] = make_float4(e.hi, e.lo, e.r, 0.5f * e.a);
                if (early) {
                    const float* ck = attr + (int64_t)g * C;
                    float G = ga0 * __ldg(ck);
                    if (C > 1) G = fmaf(ga1, __ldg(ck + 1), G);
                    if (C > 2) G = fmaf(ga2, __ldg(ck + 2), G);
                    const float Wk = __ldg(wi + (s - (KM - K)));
                    dA[s] = -tau * G * Wk;
                    if (kChain && !wi) swk[n * NT + tid] = Wk;
                    if (AM == kAttrSlot) red_add_v4(a.ws.gcam + kGcamStride * (vb + g) + 8, 0.0f, Wk * ga0, Wk * ga1, Wk * ga2);
                }
                ++n;
            } else if (s >= KM - K) {
                open = false;
            }
        }
    }
    const int32_t* li = vd.index_in + pix * L;
    auto kept = [&](int s) { return s >= KM - K && s - (KM - K) < n; };
    // depths relative to the pixel's nearest kept entry, l - l0 = (hi - l0) + lo
    // with l0 = hi of list position 0: the pair terms take l_k - l_j as one
    // difference of these, and the k side holds one register per slot (a lane
    // with an empty list runs no pair loop, so its l0 is never used)
    const float l0 = jst[tid].x;
    float dk[KM];
#pragma unroll
    for (int s = 0; s < KM; ++s) dk[s] = (hi[s] - l0) + lo[s];
    // loop 1: A_k (skipped when the forward's W_k are supplied)
    float A[KM];
#pragma unroll
    for (int s = 0; s < KM; ++s) A[s] = 0.0f;
    for (int e = 0; e < (wi ? 0 : n); ++e) {
        const float4 J = jst[e * NT + tid];
        const float dj = (J.x - l0) + J.y;
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            const float u = (dk[s] - dj) * J.z;
            const float q = erfc_as28(fabsf(u));
            const float sm = copysignf(J.w, u);
            A[s] = fmaf(-sm, q, A[s] + (J.w + sm));
        }
    }
    // T, W, dA and the attribute gradient (see kAttr*)
    const float ntl = -tau * kLog2e;
    const float* gp = vd.grad_image + pix * C;
    constexpr bool coop = AM == kAttrWarp;
    // rows of 16-byte vectors when the widths and addresses allow
    const bool rv4 = (C & 3) == 0 && ((reinterpret_cast<uintptr_t>(grad_attr) |
                                       reinterpret_cast<uintptr_t>(vd.grad_image)) & 15) == 0;
    const int cw = rv4 ? C >> 2 : C;         // row width in scatter units
    const int spi = cw <= 32 ? 32 / cw : 1;  // source lanes per step
    const int sub = cw <= 32 ? lane / cw : 0;
    const int cc = cw <= 32 ? lane - sub * cw : lane;
    const int64_t pbase = (int64_t)(row0) * W + tx * kTileW;
    if (!early) {
        int e = 0;
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            float Wk = 0.0f;
            int32_t g = -1;
            if (kept(s)) {
                g = __ldg(li + (s - (KM - K)));
                Wk = wi ? __ldg(wi + (s - (KM - K))) : ex2_approx(ntl * A[s]) * (2.0f * jst[e * NT + tid].w);
                const float* ck = attr + (int64_t)g * C;
                float G = 0.0f;
                if (AM == kAttrWarp && ((C & 3) | ((reinterpret_cast<uintptr_t>(attr) |
                                                     reinterpret_cast<uintptr_t>(vd.grad_image)) & 15)) == 0) {
                    for (int c = 0; c < (C >> 2); ++c) {
                        const float4 x = __ldg(reinterpret_cast<const float4*>(gp) + c);
                        const float4 y = __ldg(reinterpret_cast<const float4*>(ck) + c);
                        G = fmaf(x.x, y.x, fmaf(x.y, y.y, fmaf(x.z, y.z, fmaf(x.w, y.w, G))));
                    }
                } else {
                    for (int c = 0; c < C; ++c) {
                        const float gc = __ldg(gp + c);
                        G = fmaf(gc, __ldg(ck + c), G);
                        if (AM == kAttrLane && grad_attr) atomicAdd(grad_attr + (int64_t)g * C + c, Wk * gc);
                    }
                }
                dA[s] = -tau * G * Wk;
                if (kChain && !wi) swk[e * NT + tid] = Wk;
                if (AM == kAttrSlot) {
                    const float g0 = __ldg(gp), g1 = C > 1 ? __ldg(gp + 1) : 0.0f, g2 = C > 2 ? __ldg(gp + 2) : 0.0f;
                    red_add_v4(a.ws.gcam + kGcamStride * (vb + g) + 8, 0.0f, Wk * g0, Wk * g1, Wk * g2);
                }
                ++e;
            }
            if (grad_attr && coop) {
                const unsigned m = __ballot_sync(0xffffffffu, g >= 0);
                const int top = 32 - __clz(m);
#pragma unroll 1
                for (int s0 = 0; s0 < top; s0 += spi) {
                    const int src = s0 + sub;
                    const int32_t gs = __shfl_sync(0xffffffffu, g, src & 31);
                    const float ws = __shfl_sync(0xffffffffu, Wk, src & 31);
                    if (sub < spi && src < 32 && gs >= 0) {
                        const float* gsrc = vd.grad_image + (pbase + (src >> 4) * W + (src & 15)) * C;
                        float* dst = grad_attr + (int64_t)gs * C;
                        if (rv4) {
                            for (int c = cc; c < cw; c += 32) {
                                const float4 x = __ldg(reinterpret_cast<const float4*>(gsrc) + c);
                                red_add_v4(dst + 4 * c, ws * x.x, ws * x.y, ws * x.z, ws * x.w);
                            }
                        } else {
                            for (int c = cc; c < C; c += 32) atomicAdd(dst + c, ws * __ldg(gsrc + c));
                        }
                    }
                }
            }
        }
    }
    if (!packed && n == 0) return;  // no warp-wide steps below (the packed form has some)
    // loop 2: adjoint of the pair terms.  1 + erf u is formed as 1 + E with
    // E = copysign(1 - erfc|u|, u), so that a k in front of j adds dA_k
    // erfc|u| without cancellation.  The factor m_j 2/sqrt(pi) of du is
    // applied once per j to the j-side sums, and folded into the k side's
    // per-j factor mz.
    for (int e = 0; e < n; ++e) {
        const float4 J = jst[e * NT + tid];
        const float mj = J.w * kTwoOverSqrtPi;
        const float mz = mj * J.z;
        const float dj = (J.x - l0) + J.y;
        float acc_dm = 0.0f, acc_s = 0.0f, acc_dr = 0.0f;
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            const float d = dk[s] - dj;
            const float u = d * J.z;
            float g2;
            const float ec = erfc_as26(fabsf(u), g2);
            const float E = copysignf(1.0f - ec, u);
            acc_dm = fmaf(dA[s], 1.0f + E, acc_dm);
            const float du = dA[s] * g2;  // du_kj / (m_j 2/sqrt(pi))
            dl[s] = fmaf(du, mz, dl[s]);
            acc_s += du;
            acc_dr = fmaf(du, d, acc_dr);
        }
        acc_s *= mj;
        acc_dr *= mj;
        // j-side parts of dqt_j = dA_j / (2 tau) - a_j dm_j / 4 (a_j = 2 m_j)
        // and of dl_j; db_j = dr_j / (4 r_j) in full
        jst[e * NT + tid] = make_float4(-0.5f * J.w * acc_dm, -acc_s * J.z, acc_dr * rcp_approx(4.0f * J.z), 0.0f);
    }
    // the chain rule reads each entry's (dqt, dl, db, index) from the stream:
    // .x gets the k-side dA_k / (2 tau), .y the k-side dl, .w the index (all
    // of the pixel's indices are loaded at once here, so that the chain's
    // record gathers wait on shared memory only)
    const float inv2tau = 0.5f / tau;
    {
        int32_t gid[KM];
        if constexpr (packed) {
            cp_async_wait<0>();  // this unit's lists, staged again
            __syncwarp();
#pragma unroll
            for (int s = 0; s < KM; ++s) gid[s] = kept(s) ? sw[lane * S + (s - (KM - K))] : 0;
            __syncwarp();  // every lane has its indices: the rows are free
            next();
        } else {
#pragma unroll
            for (int s = 0; s < KM; ++s) gid[s] = kept(s) ? __ldg(li + (s - (KM - K))) : 0;
        }
        int e = 0;
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            if (kept(s)) {
                float4 J = jst[e * NT + tid];
                J.x = fmaf(dA[s], inv2tau, J.x);
                J.y += dl[s];
                J.w = __int_as_float(gid[s]);
                jst[e * NT + tid] = J;
                ++e;
            }
        }
    }
    // chain rule to camera space: a run-time loop over the entries, so that
    // it holds no per-slot registers
    float gi0 = 0.0f, gi1 = 0.0f, gi2 = 0.0f;  // dL/dI of this pixel (kAttrChain)
    if (kChain) {
        gi0 = __ldg(gp);
        if (C > 1) gi1 = __ldg(gp + 1);
        if (C > 2) gi2 = __ldg(gp + 2);
    }
    // kChainStep entries at a time: their records and second records.  The
    // packed form runs the loop over the warp's longest list, so that the
    // whole warp can aggregate its reductions: lanes 2i and 2i + 1 are
    // horizontally adjacent pixels, which often keep the same Gaussian at the
    // same list position.  When at least kAggPairs such pairs do, lane 2i adds
    // lane 2i + 1's twelve sums to its own and only lane 2i issues the three
    // reductions (the twelve shuffles cost about what four pairs' reductions
    // save).  Past the end of its list a lane computes on record 0 and issues
    // nothing.
    const int nloop = packed ? (int)__reduce_max_sync(0xffffffffu, (unsigned)n) : n;
    for (int e0 = 0; e0 < nloop; e0 += kChainStep) {
        float4 J[kChainStep];
        int64_t o[kChainStep];
        int32_t gk[kChainStep];
#pragma unroll
        for (int h = 0; h < kChainStep; ++h) {
            J[h] = jst[max(min(e0 + h, n - 1), 0) * NT + tid];
            gk[h] = e0 + h < n ? (int32_t)VOGE_IDX(a.hdr, __float_as_int(J[h].w), N, kChkRecord) : 0;
            o[h] = vb + gk[h];
        }
        float4 r[kChainStep][4], q[kChainStep][2];
        float wk[kChainStep];
#pragma unroll
        for (int h = 0; h < kChainStep; ++h) {
            load_rec(a.ws.rec, o[h], r[h][0], r[h][1], r[h][2], r[h][3]);
            q[h][0] = __ldg(a.ws.rec2 + 2 * o[h]);
            q[h][1] = __ldg(a.ws.rec2 + 2 * o[h] + 1);
            const int e = max(min(e0 + h, n - 1), 0);
            wk[h] = kChain ? (wi ? __ldg(wi + e) : swk[e * NT + tid]) : 0.0f;
        }
#pragma unroll
        for (int h = 0; h < kChainStep; ++h) {
            const bool live = e0 + h < n;
            float gv[12];
            const Trace tr = trace_px(r[h][0], r[h][1], r[h][2], r[h][3], px, py);
            chain_to_camera(q[h][0], q[h][1], tr, r[h][3], invF, J[h].x, J[h].y, J[h].z, gv);
            gv[9] = kChain ? wk[h] * gi0 : 0.0f;
            gv[10] = kChain ? wk[h] * gi1 : 0.0f;
            gv[11] = kChain ? wk[h] * gi2 : 0.0f;
            bool issue = live;
            if constexpr (packed) {
                const int key = live ? gk[h] : -1 - lane;
                const bool odd = (lane & 1) != 0;
                const bool pair = __shfl_xor_sync(0xffffffffu, key, 1) == key;
                if (__popc(__ballot_sync(0xffffffffu, pair && !odd)) >= kAggPairs) {
#pragma unroll
                    for (int x = 0; x < 12; ++x) {
                        const float t = __shfl_down_sync(0xffffffffu, gv[x], 1);
                        if (pair && !odd) gv[x] += t;
                    }
                    issue = live && !(pair && odd);
                }
            }
            if (issue) {
                float* gc = a.ws.gcam + kGcamStride * o[h];
                red_add_v4(gc, gv[0], gv[1], gv[2], gv[3]);
                red_add_v4(gc + 4, gv[4], gv[5], gv[6], gv[7]);
                red_add_v4(gc + 8, gv[8], gv[9], gv[10], gv[11]);
            }
        }
    }
}

// Backward tiles are 16 x TH (TH = 8): each binning tile of tile_h rows is
// split into tile_h / TH of them, so CTAs of 128 threads use less shared
// memory each (more L1) than one per binning tile; lists of up to 20 entries
// run four CTAs per SM, longer ones three with more registers.  WIDE kernels take the views with C >= 8 (warp-cooperative
// attribute rows), the others the rest; they are separate kernels so that
// each gets its own register allocation.  Each skips the other's tiles.
template <int KM, int TH, bool WIDE>
__global__ void __launch_bounds__(16 * TH, TH == 16 ? 2 : (KM <= 20 ? 4 : 3)) k_backward(Args a) {
    __shared__ int s_slot;
    // every view of one class launch has the same tile height (a serving tick
    // mixes classes, so take it from this class's first tile)
    const int R = max(1, a.views[view_of_tile(a.views, a.hdr->nviews, a.hdr->class_begin[a.cls])].tile_h / TH);
    for (;;) {
        if (threadIdx.x == 0) s_slot = atomicAdd(&a.hdr->counters[a.cls + (WIDE ? 2 : 1) * kMaxClasses], 1);
        __syncthreads();
        const int tb = R * a.hdr->class_begin[a.cls] + s_slot;
        __syncthreads();
        if (tb >= R * a.hdr->class_end[a.cls]) return;
        const int t = tb / R, hb = tb - t * R;
        const ViewDesc& vd = a.views[view_of_tile(a.views, a.hdr->nviews, t)];
        const int C = vd.C;
        if ((C >= 8) != WIDE) continue;
        if (WIDE) backward_tile<KM, TH, kAttrWarp>(a, t, hb, threadIdx.x >> 5);
        else if (C >= 4) backward_tile<KM, TH, kAttrLane>(a, t, hb, threadIdx.x >> 5);
        else if (vd.weights_in || (wk_in_smem<KM, TH>() && a.wk_smem)) backward_tile<KM, TH, kAttrChain>(a, t, hb, threadIdx.x >> 5);
        else backward_tile<KM, TH, kAttrSlot>(a, t, hb, threadIdx.x >> 5);
    }
}

// The fitting step's backward (the forward's W_k supplied, C <= 3, lists of
// up to 20): every tile takes the packed set-up.
// Row pairs (units) of a backward tile with at least one kept entry, for the
// packed form.  A block takes 256 consecutive units, each of its warps 32 of
// them: lane x first works out where unit x's lists are, then the warp reads
// the first list entry of each unit's 32 pixels, all 32 units at once, and a
// ballot tells whether any is kept.  The block appends its live units in
// order with one atomic.
__global__ void __launch_bounds__(256) k_live_units(Args a) {
    constexpr int TH = 8, Q = TH / 2, kAhead = 32;
    __shared__ unsigned s_mask[8];
    __shared__ int s_base;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int R = max(1, a.views[view_of_tile(a.views, a.hdr->nviews, a.hdr->class_begin[a.cls])].tile_h / TH);
    const int first = Q * R * a.hdr->class_begin[a.cls], end = Q * R * a.hdr->class_end[a.cls];
    const int r = lane >> 4, c = lane & 15;
    for (int ub = first + 256 * blockIdx.x; ub < end; ub += 256 * gridDim.x) {
        // this lane's unit: view, first list word, row stride, rows and columns inside the image
        const int u = ub + 32 * w + lane;
        int v = 0, Wu = 0, Lu = 0, nrows = 0, ncols = 0;
        const int32_t* base = nullptr;
        if (u < end) {
            const int tb = u / Q, q = u - tb * Q, t = tb / R, hb = tb - t * R;
            v = view_of_tile(a.views, a.hdr->nviews, t);
            const ViewDesc& vd = a.views[v];
            const int lt = t - vd.tile_base;
            const int tx = lt % vd.tiles_x, ty = lt / vd.tiles_x;
            const int row0 = ty * vd.tile_h + hb * TH + 2 * q, col0 = tx * kTileW;
            Wu = vd.W;
            Lu = vd.L;
            nrows = max(0, min(2, vd.H - row0));
            ncols = min(kTileW, vd.W - col0);
            base = vd.index_in + ((int64_t)row0 * vd.W + col0) * vd.L;
        }
        unsigned mask = 0u;  // bit x: unit ub + 32 w + x is live
#pragma unroll 1
        for (int x0 = 0; x0 < 32; x0 += kAhead) {
            int32_t g[kAhead];
#pragma unroll
            for (int h = 0; h < kAhead; ++h) {
                const int x = x0 + h;
                const int32_t* bx = reinterpret_cast<const int32_t*>(
                    __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(base), x));
                const int wx = __shfl_sync(0xffffffffu, Wu, x), lx = __shfl_sync(0xffffffffu, Lu, x);
                const int nr = __shfl_sync(0xffffffffu, nrows, x), nc = __shfl_sync(0xffffffffu, ncols, x);
                g[h] = (r < nr && c < nc) ? __ldg(bx + ((int64_t)r * wx + c) * lx) : -1;
            }
#pragma unroll
            for (int h = 0; h < kAhead; ++h)
                if (__any_sync(0xffffffffu, g[h] >= 0)) mask |= 1u << (x0 + h);
        }
        if (lane == 0) s_mask[w] = mask;
        __syncthreads();
        if (threadIdx.x == 0) {
            int n = 0;
#pragma unroll
            for (int x = 0; x < 8; ++x) n += __popc(s_mask[x]);
            s_base = n ? atomicAdd(&a.ws.live_hdr->n[a.cls], n) : 0;
        }
        __syncthreads();
        if ((mask >> lane) & 1u) {
            int pos = s_base + __popc(mask & ((1u << lane) - 1u));
            for (int x = 0; x < w; ++x) pos += __popc(s_mask[x]);
            a.ws.live[first + pos] = make_int2(u, v);
        }
        __syncthreads();
    }
}

// Warp-persistent over the units: each warp claims units one at a time (two
// claims ahead), with no block barriers, and stages the next unit's lists
// while the current one's pair terms and chain rule run.  When the call's
// record of live units describes these lists (the forward's, or
// k_live_units'), only those are visited; otherwise every unit of the class
// is, and the empty ones cost their list read.
template <int KM>
__global__ void __launch_bounds__(128, 4) k_backward_packed(Args a) {
    constexpr int TH = 8, Q = TH / 2;
    extern __shared__ float4 smem[];
    int32_t* sw = reinterpret_cast<int32_t*>(smem + KM * 16 * TH) + (threadIdx.x >> 5) * packed_warp_words<KM>();
    const int lane = threadIdx.x & 31;
    const int R = max(1, a.views[view_of_tile(a.views, a.hdr->nviews, a.hdr->class_begin[a.cls])].tile_h / TH);
    int* counter = &a.hdr->counters[a.cls + kMaxClasses];
    const int first = Q * R * a.hdr->class_begin[a.cls];
    const LiveHdr* lh = a.ws.live_hdr;
    const bool rec = lh->index_fwd != nullptr && lh->index_fwd == a.views[0].index_in;
    const int count = rec ? lh->n[a.cls] : Q * R * a.hdr->class_end[a.cls] - first;
    const int2* live = a.ws.live + first;
    auto unit = [&](int x) -> int2 {
        if (rec) return __ldg(live + x);
        return make_int2(first + x, view_of_tile(a.views, a.hdr->nviews, (first + x) / (Q * R)));
    };
    auto stage = [&](int2 un) {
        const int tb = un.x / Q, t = tb / R;
        stage_lists_packed(a, sw, un.y, t, tb - t * R, un.x - tb * Q);
    };
    int cur = __shfl_sync(0xffffffffu, lane == 0 ? atomicAdd(counter, 1) : 0, 0);
    int2 cu = make_int2(0, 0);
    if (cur < count) {
        cu = unit(cur);
        stage(cu);
    }
    int claim = lane == 0 ? atomicAdd(counter, 1) : 0;
    while (cur < count) {
        const int nx = __shfl_sync(0xffffffffu, claim, 0);
        const int2 nu = nx < count ? unit(nx) : make_int2(0, 0);
        claim = lane == 0 ? atomicAdd(counter, 1) : 0;
        const int tb = cu.x / Q, t = tb / R;
        backward_tile<KM, TH, kAttrPacked>(
            a, t, tb - t * R, cu.x - tb * Q, cu.y, [&]() { stage(cu); },
            [&]() {
                if (nx < count) stage(nu);
            });
        cur = nx;
        cu = nu;
    }
}

// Camera-space accumulators -> world-space gradients of each view's scene
// (M = R M_w + T, P = R P_w Rᵀ): dM_w = Rᵀ dM, dP_w = Rᵀ G R, and the camera
// pose dL/dR = dM M_wᵀ + 2 G R P_w, dL/dT = dM summed over the view's
// Gaussians.  One thread per (view, Gaussian) record; the accumulators are
// cleared once read.
__global__ void __launch_bounds__(256) k_grad_finalize(Args a) {
    const int nv = a.hdr->nviews;
    const int64_t total = a.hdr->total_records;
    const int lane = threadIdx.x & 31;
    for (int64_t tb = (int64_t)blockIdx.x * blockDim.x; tb < total; tb += (int64_t)gridDim.x * blockDim.x) {
        const int64_t t = tb + threadIdx.x;
        const bool live = t < total;
        const int v = live ? view_of_record(a.views, nv, t) : -1;
        float p[12];
#pragma unroll
        for (int q = 0; q < 12; ++q) p[q] = 0.0f;
        float* gcam_out = nullptr;
        if (live) {
            const ViewDesc& vd = a.views[v];
            const int64_t g = t - vd.rec_base;
            float* gc = a.ws.gcam + kGcamStride * t;
            const float dM[3] = {gc[0], gc[1], gc[2]};
            const float G[9] = {gc[3], gc[4], gc[5], gc[4], gc[6], gc[7], gc[5], gc[7], gc[8]};
            if (vd.C <= 3 && vd.grad_attr)  // narrow attribute gradients ride in slots 9..11
                for (int c = 0; c < vd.C; ++c) atomicAdd(vd.grad_attr + (int64_t)vd.C * g + c, gc[9 + c]);
#pragma unroll
            for (int q = 0; q < 12; ++q) gc[q] = 0.0f;
            float R[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) R[q] = vd.R[q];
            if (vd.grad_means) {
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    atomicAdd(vd.grad_means + 3 * g + q, R[q] * dM[0] + R[3 + q] * dM[1] + R[6 + q] * dM[2]);
            }
            float GR[9];
#pragma unroll
            for (int x = 0; x < 3; ++x)
#pragma unroll
                for (int y = 0; y < 3; ++y) GR[3 * x + y] = G[3 * x] * R[y] + G[3 * x + 1] * R[3 + y] + G[3 * x + 2] * R[6 + y];
            if (vd.grad_inv_cov) {
                float Gw[9];
#pragma unroll
                for (int x = 0; x < 3; ++x)
#pragma unroll
                    for (int y = 0; y < 3; ++y) Gw[3 * x + y] = R[x] * GR[y] + R[3 + x] * GR[3 + y] + R[6 + x] * GR[6 + y];
                float* gp = vd.grad_inv_cov + 6 * g;
                atomicAdd(gp + 0, Gw[0]);
                atomicAdd(gp + 1, Gw[1] + Gw[3]);
                atomicAdd(gp + 2, Gw[2] + Gw[6]);
                atomicAdd(gp + 3, Gw[4]);
                atomicAdd(gp + 4, Gw[5] + Gw[7]);
                atomicAdd(gp + 5, Gw[8]);
            }
            if (vd.grad_cam) {
                gcam_out = vd.grad_cam;
                float Mw[3], Pw[9];
#pragma unroll
                for (int q = 0; q < 3; ++q) Mw[q] = __ldg(vd.means + 3 * g + q);
                const float* p6 = vd.inv_cov + 6 * g;
                Pw[0] = __ldg(p6 + 0); Pw[1] = __ldg(p6 + 1); Pw[2] = __ldg(p6 + 2);
                Pw[3] = Pw[1]; Pw[4] = __ldg(p6 + 3); Pw[5] = __ldg(p6 + 4);
                Pw[6] = Pw[2]; Pw[7] = Pw[5]; Pw[8] = __ldg(p6 + 5);
                float RP[9];
#pragma unroll
                for (int x = 0; x < 3; ++x)
#pragma unroll
                    for (int y = 0; y < 3; ++y) RP[3 * x + y] = R[3 * x] * Pw[y] + R[3 * x + 1] * Pw[3 + y] + R[3 * x + 2] * Pw[6 + y];
#pragma unroll
                for (int x = 0; x < 3; ++x)
#pragma unroll
                    for (int y = 0; y < 3; ++y)
                        p[3 * x + y] = dM[x] * Mw[y] + 2.0f * (G[3 * x] * RP[y] + G[3 * x + 1] * RP[3 + y] + G[3 * x + 2] * RP[6 + y]);
                p[9] = dM[0];
                p[10] = dM[1];
                p[11] = dM[2];
            }
        }
        // pose sums: one warp reduction when the warp's records share a view
        const int v0 = __shfl_sync(0xffffffffu, v, 0);
        float* out0 = reinterpret_cast<float*>(__shfl_sync(0xffffffffu, reinterpret_cast<uintptr_t>(gcam_out), 0));
        const bool uniform = __all_sync(0xffffffffu, v == v0 || v < 0) && v0 >= 0;
        if (uniform) {
#pragma unroll
            for (int q = 0; q < 12; ++q) {
                float x = p[q];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
                p[q] = x;
            }
            if (lane == 0 && out0)
#pragma unroll
                for (int q = 0; q < 12; ++q) atomicAdd(out0 + q, p[q]);
        } else if (gcam_out) {
#pragma unroll
            for (int q = 0; q < 12; ++q) atomicAdd(gcam_out + q, p[q]);
        }
    }
}

template <typename Kern>
static cudaError_t launch_tiles(Kern k, const char* name, int nblocks, int nthreads, size_t smem, cudaStream_t s,
                                const Args& a) {
    TraceScope tr(name, s);
    if (smem > 32 * 1024) {  // opt in well below 48 KB: the kernels' static shared memory counts too
        cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    k<<<nblocks, nthreads, smem, s>>>(a);
    return cudaPeekAtLastError();
}

// The stream, plus the W_k buffer where it fits (it holds W_k when the
// backward recomputes them, dA_k when the forward's W_k are supplied).
template <int KM, int TH>
static size_t backward_smem_bytes(bool = true) {
    return (size_t)KM * 16 * TH * (wk_in_smem<KM, TH>() ? 20 : 16);
}

// The packed form: the stream, then each warp's staging rows.
template <int KM>
static size_t packed_smem_bytes() {
    return (size_t)KM * 16 * 8 * 16 + 4 * (size_t)packed_warp_words<KM>() * 4;
}

template <typename Kern>
static int blocks_per_sm(Kern k, int nthreads, size_t smem) {
    if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, nthreads, smem) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

// Resident CTAs per SM of the backward tile kernel for capacity KM.
int backward_blocks_per_sm(int KM) {
    switch (KM) {
        case 8: return blocks_per_sm(k_backward<8, 8, false>, 128, backward_smem_bytes<8, 8>());
        case 16: return blocks_per_sm(k_backward<16, 8, false>, 128, backward_smem_bytes<16, 8>());
        case 20: return blocks_per_sm(k_backward<20, 8, false>, 128, backward_smem_bytes<20, 8>());
        case 24: return blocks_per_sm(k_backward<24, 8, false>, 128, backward_smem_bytes<24, 8>());
        case 32: return blocks_per_sm(k_backward<32, 8, false>, 128, backward_smem_bytes<32, 8>());
        default: return 1;  // lists longer than 32: voge_generic.cu
    }
}

// Launch the backward tile kernel for register-list capacity KM (8..32).
template <int KM>
static cudaError_t launch_backward_pair(const char* name, const char* wname, int nblocks, bool w, int kinds,
                                        cudaStream_t s, const Args& a) {
    cudaError_t e = cudaSuccess;
    if (kinds & 1) e = launch_tiles(k_backward<KM, 8, false>, name, nblocks, 128, backward_smem_bytes<KM, 8>(w), s, a);
    if (e == cudaSuccess && (kinds & 2))
        e = launch_tiles(k_backward<KM, 8, true>, wname, nblocks, 128, backward_smem_bytes<KM, 8>(w), s, a);
    return e;
}

// The packed form (k_backward_packed) for capacities up to 20, when every
// view brings the forward's weights and C <= 3.
cudaError_t launch_backward_packed(int KM, int nblocks, int live_tiles, cudaStream_t s, const Args& a) {
    if (live_tiles > 0) {  // find the live units of given lists
        TraceScope tr("k_live_units", s);
        const int nb = (8 * live_tiles + 255) / 256;  // at most 8 units per tile
        k_live_units<<<nb < 1024 ? nb : 1024, 256, 0, s>>>(a);
        const cudaError_t e = cudaPeekAtLastError();
        if (e != cudaSuccess) return e;
    }
    switch (KM) {
        case 8: return launch_tiles(k_backward_packed<8>, "k_backward<8>", nblocks, 128, packed_smem_bytes<8>(), s, a);
        case 16: return launch_tiles(k_backward_packed<16>, "k_backward<16>", nblocks, 128, packed_smem_bytes<16>(), s, a);
        case 20: return launch_tiles(k_backward_packed<20>, "k_backward<20>", nblocks, 128, packed_smem_bytes<20>(), s, a);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_backward_tiles(int KM, int nblocks, int with_wk, int kinds, cudaStream_t s, const Args& a0) {
    // with_wk = 0: every view brings the forward's weights, so the W_k buffer
    // is left out and its shared memory goes to L1 (the chain's record reads).
    // kinds: bit 0 launches the kernel for C < 8, bit 1 the one for C >= 8.
    Args a = a0;
    a.wk_smem = with_wk ? 1 : 0;
    const bool w = with_wk != 0;
    switch (KM) {
        case 8: return launch_backward_pair<8>("k_backward<8>", "k_backward<8,wide>", nblocks, w, kinds, s, a);
        case 16: return launch_backward_pair<16>("k_backward<16>", "k_backward<16,wide>", nblocks, w, kinds, s, a);
        case 20: return launch_backward_pair<20>("k_backward<20>", "k_backward<20,wide>", nblocks, w, kinds, s, a);
        case 24: return launch_backward_pair<24>("k_backward<24>", "k_backward<24,wide>", nblocks, w, kinds, s, a);
        case 32: return launch_backward_pair<32>("k_backward<32>", "k_backward<32,wide>", nblocks, w, kinds, s, a);
        default: return cudaErrorInvalidValue;  // lists longer than 32: launch_backward_generic
    }
}

// Shared-scene form (every view renders the same N Gaussians), in two
// kernels.  k_pose_grad_shared: one thread per (view, Gaussian) turns the
// camera-space sums into that view's pose gradient (Sec. 3.3 chain through
// M = R M_w + T, P = R P_w R^T), reduced per block.  k_grad_finalize_shared:
// one thread per Gaussian rotates the sums of every view into world space and
// adds them up, so world gradients are written once without atomics; it also
// clears the sums for the next call.
__global__ void __launch_bounds__(256) k_pose_grad_shared(Args a) {
    __shared__ float red[8][12];
    const int v = blockIdx.y;
    const ViewDesc& vd = a.views[v];
    if (!vd.grad_cam) return;  // uniform in the block
    const int N = vd.N;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int g = blockIdx.x * blockDim.x + threadIdx.x;
    float p[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) p[q] = 0.0f;
    if (g < N) {
        const float4* gc4 = reinterpret_cast<const float4*>(a.ws.gcam + kGcamStride * (vd.rec_base + g));
        const float4 c0 = gc4[0], c1 = gc4[1], c2 = gc4[2];
        const float dM[3] = {c0.x, c0.y, c0.z};
        const float G[9] = {c0.w, c1.x, c1.y, c1.x, c1.z, c1.w, c1.y, c1.w, c2.x};
        float R[9], Mw[3], Pw[9];
#pragma unroll
        for (int q = 0; q < 9; ++q) R[q] = vd.R[q];
#pragma unroll
        for (int q = 0; q < 3; ++q) Mw[q] = __ldg(vd.means + 3 * (int64_t)g + q);
        const float* p6 = vd.inv_cov + 6 * (int64_t)g;
        Pw[0] = __ldg(p6 + 0); Pw[1] = __ldg(p6 + 1); Pw[2] = __ldg(p6 + 2);
        Pw[3] = Pw[1]; Pw[4] = __ldg(p6 + 3); Pw[5] = __ldg(p6 + 4);
        Pw[6] = Pw[2]; Pw[7] = Pw[5]; Pw[8] = __ldg(p6 + 5);
        float RP[9];
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int y = 0; y < 3; ++y) RP[3 * x + y] = R[3 * x] * Pw[y] + R[3 * x + 1] * Pw[3 + y] + R[3 * x + 2] * Pw[6 + y];
#pragma unroll
        for (int x = 0; x < 3; ++x)
#pragma unroll
            for (int y = 0; y < 3; ++y)
                p[3 * x + y] = dM[x] * Mw[y] + 2.0f * (G[3 * x] * RP[y] + G[3 * x + 1] * RP[3 + y] + G[3 * x + 2] * RP[6 + y]);
        p[9] = dM[0];
        p[10] = dM[1];
        p[11] = dM[2];
    }
#pragma unroll
    for (int q = 0; q < 12; ++q) {
        float x = p[q];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if (lane == 0) red[wid][q] = x;
    }
    __syncthreads();
    if (threadIdx.x < 12) {
        float sum = 0.0f;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w][threadIdx.x];
        atomicAdd(vd.grad_cam + threadIdx.x, sum);
    }
}

__global__ void __launch_bounds__(256) k_grad_finalize_shared(Args a) {
    const int nv = a.hdr->nviews;
    const ViewDesc& v0 = a.views[0];
    const int N = v0.N, C = v0.C;
    for (int g = blockIdx.x * blockDim.x + threadIdx.x; g < N; g += gridDim.x * blockDim.x) {
        float gm[3] = {0.f, 0.f, 0.f}, gw[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f}, ga[3] = {0.f, 0.f, 0.f};
        for (int v = 0; v < nv; ++v) {
            const ViewDesc& vd = a.views[v];
            float4* gc4 = reinterpret_cast<float4*>(a.ws.gcam + kGcamStride * (vd.rec_base + g));
            const float4 c0 = gc4[0], c1 = gc4[1], c2 = gc4[2];
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            gc4[0] = z;
            gc4[1] = z;
            gc4[2] = z;
            float R[9];
#pragma unroll
            for (int q = 0; q < 9; ++q) R[q] = vd.R[q];
            const float dM[3] = {c0.x, c0.y, c0.z};
            const float G[9] = {c0.w, c1.x, c1.y, c1.x, c1.z, c1.w, c1.y, c1.w, c2.x};
            ga[0] += c2.y;  // narrow attribute gradients (slots 9..11)
            ga[1] += c2.z;
            ga[2] += c2.w;
#pragma unroll
            for (int q = 0; q < 3; ++q) gm[q] += R[q] * dM[0] + R[3 + q] * dM[1] + R[6 + q] * dM[2];
            float GR[9];
#pragma unroll
            for (int x = 0; x < 3; ++x)
#pragma unroll
                for (int y = 0; y < 3; ++y) GR[3 * x + y] = G[3 * x] * R[y] + G[3 * x + 1] * R[3 + y] + G[3 * x + 2] * R[6 + y];
            float Gw[9];
#pragma unroll
            for (int x = 0; x < 3; ++x)
#pragma unroll
                for (int y = 0; y < 3; ++y) Gw[3 * x + y] = R[x] * GR[y] + R[3 + x] * GR[3 + y] + R[6 + x] * GR[6 + y];
            gw[0] += Gw[0]; gw[1] += Gw[1] + Gw[3]; gw[2] += Gw[2] + Gw[6];
            gw[3] += Gw[4]; gw[4] += Gw[5] + Gw[7]; gw[5] += Gw[8];
        }
        if (v0.grad_means)
            for (int q = 0; q < 3; ++q) v0.grad_means[3 * (int64_t)g + q] += gm[q];
        if (v0.grad_inv_cov)
            for (int q = 0; q < 6; ++q) v0.grad_inv_cov[6 * (int64_t)g + q] += gw[q];
        if (C <= 3 && v0.grad_attr)
            for (int c = 0; c < C; ++c) v0.grad_attr[(int64_t)C * g + c] += ga[c];
    }
}

cudaError_t launch_grad_finalize(int grid, int nviews, int N, int shared_scene, cudaStream_t s, const Args& a) {
    TraceScope tr("k_grad_finalize", s);
    if (shared_scene) {
        if (N > 0 && nviews > 0) {
            k_pose_grad_shared<<<dim3((N + 255) / 256, nviews), 256, 0, s>>>(a);
            k_grad_finalize_shared<<<grid, 256, 0, s>>>(a);
        }
    } else {
        k_grad_finalize<<<grid, 256, 0, s>>>(a);
    }
    return cudaPeekAtLastError();
}

}  // namespace voge
