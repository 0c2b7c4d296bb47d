// voge_forward.cu -- fused coarse + fine forward pass: persistent CTAs over
// tiles of 16 x TH pixels, one thread per pixel.
//
// Coarse pass (Sec. 3.3, App. A.3): the tile's candidate Gaussians (binned
// and, when eta > 0, sorted by a lower bound of l by k_sort_tiles) are staged
// in shared memory in chunks of 16 TH.  While staging, each candidate's
// threshold conic gives a 16-bit pixel mask per tile row; every pixel traces
// (Eq. 6) only the candidates whose mask covers it, keeps those with
// e^{q} > eta and l > 0, and holds the K nearest by (l, index) in its own
// shared-memory column.  A pixel stops once no later candidate can enter.
//
// Fine pass (Eq. 7-8): with the kept list L_p,
//   A_k = sum_{j in L_p} (a_j/2)(1 + erf((l_k - l_j) sqrt(b_j/2))),
//   T_k = exp(-tau A_k),  W_k = T_k a_k,  image = sum_k W_k c_k.
// The list's (l, r, a/2) are streamed from shared memory over j while the k
// side stays in registers; erf is Abramowitz & Stegun 7.1.28 on the FMA pipe
// plus one MUFU reciprocal.
#include "voge_device.cuh"
#include "voge_trace.cuh"

namespace voge {

// Candidate source of one tile.
struct TileSrc {
    int mode;          // 0 = binned list, 1 = binned list sorted by depth bound, 2 = every Gaussian (plain/overflow)
    int filter_box;    // mode 2: test the Gaussian's tile box
    int count;
    int start;
};

// Candidate source of a tile.  mode 1: the binned list, sorted by depth lower
// bound (early exit allowed); mode 0: the binned list unsorted; mode 2: every
// Gaussian of the view (plain, or the tile's list overflowed the bins).
template <int NT>
__device__ __forceinline__ TileSrc tile_source(const Args& a, const ViewDesc& vd, int t) {
    TileSrc src;
    src.filter_box = 0;
    const int N = vd.N;
    if (vd.plain) {
        src.mode = 2;
        src.count = N;
        src.start = 0;
        return src;
    }
    const int cnt = a.ws.tile_cnt[t];
    const int off = a.ws.tile_off[t];
    if ((int64_t)off + cnt > a.ws.bin_cap) {  // binning overflowed: test every Gaussian against its box
        src.mode = 2;
        src.filter_box = 1;
        src.count = N;
        src.start = 0;
        return src;
    }
    src.count = cnt;
    src.start = off;
    src.mode = (vd.use_thresh && cnt > 1 && cnt <= kSortMax) ? 1 : 0;
    return src;
}

// Transpose a 32 x 32 bit matrix held one row per lane (bit c of lane r is
// entry (r, c)): afterwards lane c holds column c.  Each butterfly stage swaps
// the off-diagonal blocks of size j inside the blocks of size 2j (Hacker's
// Delight, 7-3, with the row exchanges done by warp shuffles).
__device__ __forceinline__ uint32_t warp_transpose32(uint32_t x, int lane) {
#pragma unroll
    for (int j = 16; j >= 1; j >>= 1) {
        const uint32_t m = j == 16 ? 0x0000ffffu : j == 8 ? 0x00ff00ffu : j == 4 ? 0x0f0f0f0fu : j == 2 ? 0x33333333u
                                                                                                     : 0x55555555u;
        const uint32_t y = __shfl_xor_sync(0xffffffffu, x, j);
        // the lower lane of a pair keeps its low blocks and takes the partner's
        // low blocks into its high ones; the upper lane the reverse
        x = (lane & j) ? ((x & ~m) | ((y >> j) & m)) : ((x & m) | ((y << j) & ~m));
    }
    return x;
}

template <int KM, int TH>
__device__ __forceinline__ void render_tile(const Args& a, int t) {
    constexpr int NT = 16 * TH;
    extern __shared__ float4 smem[];
    // phase 1 layout: stage[4][NT] float4 | sgid[NT] | siv[TH][NT] | smask[NT/32][NT] | slk, sli [KM][NT]
    float4* stage = smem;
    int32_t* sgid = reinterpret_cast<int32_t*>(stage + 4 * NT);
    uint16_t* siv = reinterpret_cast<uint16_t*>(sgid + NT);
    uint32_t* smask = reinterpret_cast<uint32_t*>(siv + TH * NT);  // [NT/32][NT] per-lane hit masks
    float* slk = reinterpret_cast<float*>(smask + (NT / 32) * NT);  // [KM][NT] per-lane kept depths
    int32_t* sli = reinterpret_cast<int32_t*>(slk + KM * NT);      // [KM][NT] per-lane kept indices
    // phase 2 layout: jst[KM][NT] float4 (aliases phase 1)
    float4* jst = smem;

    const int v = view_of_tile(a.views, a.hdr->nviews, t);
    const ViewDesc& vd = a.views[v];
    const int lt = t - vd.tile_base;
    const int tiles_x = vd.tiles_x;
    const int tx = lt % tiles_x, ty = lt / tiles_x;
    const int H = vd.H, W = vd.W;
    const int tid = threadIdx.x;
    const int j = tx * kTileW + (tid & 15);
    const int i = ty * TH + (tid >> 4);
    const bool valid = (i < H) && (j < W);
    const float px = (float)j + 0.5f, py = (float)i + 0.5f;
    const int64_t pix = (int64_t)i * W + j;  // pixel within the view
    const int64_t vb = vd.rec_base;
    const int K = vd.L;  // list length (<= KM)
    const float Qeta = vd.Qeta;

    // The kept list of this pixel lives in its own shared-memory column: new
    // candidates are appended while it fills; once it holds K entries a
    // nearer candidate replaces the farthest one (kmax, gmax at slot smax).
    // It is sorted once at the end.
    int n = 0, smax = 0;
    float kmax = INFINITY;
    int32_t gmax = INT32_MAX;

    const TileSrc src = tile_source<NT>(a, vd, t);
    if (src.count == 0) {
        // no candidate reaches this tile: empty lists, zero weights and image,
        // each warp writing its two row segments
        const int lane = tid & 31, warp = tid >> 5;
        const int L = vd.L, C = vd.C;
        const int ncols = min(kTileW, W - tx * kTileW);
#pragma unroll
        for (int rw = 0; rw < 2; ++rw) {
            const int irow = ty * TH + 2 * warp + rw;
            if (irow >= H) continue;
            const int64_t p0 = (int64_t)irow * W + tx * kTileW;
            for (int x = lane; x < ncols * L; x += 32) {
                vd.index[p0 * L + x] = -1;
                if (vd.weights) vd.weights[p0 * L + x] = 0.0f;
            }
            for (int x = lane; x < ncols * C; x += 32) vd.image[p0 * C + x] = 0.0f;
        }
        return;
    }
    bool active = valid;
    for (int base = 0; base < src.count; base += NT) {
        const int nc = min(NT, src.count - base);
        if (tid < nc) {
            int32_t g;
            if (src.mode != 2) g = a.ws.tile_gauss[src.start + base + tid];
            else g = base + tid;
            float4 r0, r1, r2, r3;
            load_rec(a.ws.rec, vb + g, r0, r1, r2, r3);
            bool outside = false;
            if (src.filter_box) {
                const int4 tb = a.ws.tbox[vb + g];
                outside = tx < tb.x || tx > tb.y || ty < tb.z || ty > tb.w;
                if (outside) {
                    r1 = make_float4(0.f, 0.f, 0.f, 0.f);
                    r2 = r1;
                }
            }
            stage[0 * NT + tid] = r0;
            stage[1 * NT + tid] = r1;
            stage[2 * NT + tid] = r2;
            stage[3 * NT + tid] = r3;
            sgid[tid] = g;
            if (outside) {
#pragma unroll
                for (int rr = 0; rr < TH; ++rr) siv[rr * NT + tid] = kRowEmpty;
            } else {
                row_masks<TH>(r0, r1, r2, r3, Qeta, tx, ty, siv + tid, NT);
            }
        }
        __syncthreads();
        constexpr int NW = NT / 32;
        if (__any_sync(0xffffffffu, active)) {
            // 1) the hit masks of the warp's 32 pixels (two tile rows), one
            //    32-bit word per 32 candidates: lane q supplies candidate q's
            //    coverage of the two rows (its row masks, 16 bits each) and a
            //    bit transpose hands each lane its pixel's bits
            const int lane = tid & 31, r2 = 2 * (tid >> 5);
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                uint32_t m = 0;
                if (w * 32 < nc) {  // uniform
                    const int q = w * 32 + lane;
                    const uint32_t x = q < nc ? (uint32_t)siv[r2 * NT + q] | ((uint32_t)siv[(r2 + 1) * NT + q] << 16) : 0u;
                    m = warp_transpose32(x, lane);
                }
                smask[w * NT + tid] = m;
            }
        }
        if (active) {
            // 2) each lane walks its own hits: lanes of a warp trace different
            //    candidates at the same time instead of the union of all hits.
            //    One cursor runs over all mask words, so the warp iterates as
            //    often as its busiest lane has hits in the chunk.
            int w = 0;
            uint32_t m = smask[tid];
            for (;;) {
                while (m == 0 && w < NW - 1) m = smask[++w * NT + tid];
                if (m == 0) break;
                const int q = w * 32 + __ffs(m) - 1;
                m &= m - 1;
                const float4 r3 = stage[3 * NT + q];  // .w: the candidate's depth lower bound
                if (src.mode == 1 && r3.w > kmax) {
                    active = false;  // sorted by lower bound: nothing later can enter
                    break;
                }
                const float4 r0 = stage[q], r1 = stage[NT + q], r2 = stage[2 * NT + q];
                const float l = candidate_key(r0, r1, r2, r3, px, py, Qeta);
                if (l > 0.0f) {
                    const int32_t g = sgid[q];
                    int slot = -1;
                    if (n < K) {
                        slot = n++;
                    } else if (l < kmax || (l == kmax && g < gmax)) {
                        slot = smax;
                    }
                    if (slot >= 0) {
                        slk[slot * NT + tid] = l;
                        sli[slot * NT + tid] = g;
                        if (n == K) {  // full: find the farthest entry, the bar for later candidates
                            kmax = -INFINITY;
                            gmax = -1;
                            for (int s2 = 0; s2 < K; ++s2) {
                                const float x = slk[s2 * NT + tid];
                                const int32_t y = sli[s2 * NT + tid];
                                if (x > kmax || (x == kmax && y > gmax)) {
                                    kmax = x;
                                    gmax = y;
                                    smax = s2;
                                }
                            }
                        }
                    }
                }
            }
            // a pixel whose list is full and whose next candidate (in sorted
            // order) starts beyond its K-th depth can stop for good
            if (active && src.mode == 1 && nc == NT && base + NT < src.count) {
                // the first candidate of the next chunk bounds everything after it
                const int32_t gn = __ldg(a.ws.tile_gauss + src.start + base + NT);
                const float nxt = __ldg(&a.ws.rec[4 * (vb + gn) + 3].w);
                if (nxt > kmax) active = false;
            }
        }
        if (__syncthreads_and(!active)) break;
    }
    // sort the kept list by (l, index).  Short lists (KM <= 20): in registers,
    // entries at slots [KM - K, KM - K + n), the slots before them padded with
    // (-inf, min) and after them with (+inf, max) so that they stay put;
    // odd-even transposition sort, and since candidates arrive nearly in
    // depth order the warp stops after a few passes, once no lane swapped in
    // two passes.  Longer lists: insertion sort in the shared-memory columns.
    int32_t id[KM];
    if constexpr (KM <= 20) {
        float xk[KM];
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            const int k = s - (KM - K);
            const bool in = k >= 0 && k < n;
            xk[s] = in ? slk[k * NT + tid] : (k < 0 ? -INFINITY : INFINITY);
            id[s] = in ? sli[k * NT + tid] : (k < 0 ? INT32_MIN : INT32_MAX);
        }
        auto cmpx = [&](float& ka, int32_t& ia, float& kb, int32_t& ib) -> bool {
            const bool gt = ka > kb || (ka == kb && ia > ib);
            const float k0 = gt ? kb : ka, k1 = gt ? ka : kb;
            const int32_t i0 = gt ? ib : ia, i1 = gt ? ia : ib;
            ka = k0;
            kb = k1;
            ia = i0;
            ib = i1;
            return gt;
        };
        bool prev = true;
        for (int pass = 0; pass < KM; ++pass) {
            bool sw = false;
            if (pass & 1) {
#pragma unroll
                for (int s = 1; s + 1 < KM; s += 2) sw |= cmpx(xk[s], id[s], xk[s + 1], id[s + 1]);
            } else {
#pragma unroll
                for (int s = 0; s + 1 < KM; s += 2) sw |= cmpx(xk[s], id[s], xk[s + 1], id[s + 1]);
            }
            const bool any = __any_sync(0xffffffffu, sw);
            if (!any && !prev) break;
            prev = any;
        }
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            const int k = s - (KM - K);
            if (!(k >= 0 && k < n)) id[s] = -1;
        }
    } else {
        for (int i = 1; i < n; ++i) {
            const float x = slk[i * NT + tid];
            const int32_t y = sli[i * NT + tid];
            int j = i - 1;
            while (j >= 0) {
                const float xj = slk[j * NT + tid];
                const int32_t yj = sli[j * NT + tid];
                if (!(xj > x || (xj == x && yj > y))) break;
                slk[(j + 1) * NT + tid] = xj;
                sli[(j + 1) * NT + tid] = yj;
                --j;
            }
            slk[(j + 1) * NT + tid] = x;
            sli[(j + 1) * NT + tid] = y;
        }
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            const int k = s - (KM - K);
            id[s] = (k >= 0 && k < n) ? sli[k * NT + tid] : -1;
        }
    }
    __syncthreads();  // selection buffers are free from here on

    // ---------------- index output ----------------
    // Each warp covers two 16-pixel row segments of the tile; a segment's
    // lists are contiguous in memory ([pixel][L]).  The warp stages its 32
    // lists in its own shared-memory columns (blocks of 32 float4) and writes
    // each segment with consecutive lanes on consecutive words.
    const int L = vd.L, C = vd.C;
    const int lane = tid & 31, warp = tid >> 5;
    auto stg = [&](int x) -> float* { return reinterpret_cast<float*>(jst + (x >> 7) * NT + 32 * warp) + (x & 127); };
    const int ncols = min(kTileW, W - tx * kTileW);
#pragma unroll
    for (int s = 0; s < KM; ++s)
        if (s >= KM - K) *reinterpret_cast<int32_t*>(stg(lane * L + (s - (KM - K)))) = id[s];
    __syncwarp();
#pragma unroll
    for (int rw = 0; rw < 2; ++rw) {
        const int irow = ty * TH + 2 * warp + rw;
        if (irow >= H) continue;
        int32_t* di = vd.index + ((int64_t)irow * W + tx * kTileW) * L;
        for (int x = lane; x < ncols * L; x += 32) di[x] = *reinterpret_cast<const int32_t*>(stg(rw * 16 * L + x));
    }
    __syncwarp();

    // ---------------- fine pass ----------------
    // kept entries occupy slots [KM - K, KM - K + n) in ascending (l, index)
    float hi[KM], lo[KM], A[KM];
#pragma unroll
    for (int s = 0; s < KM; ++s) {
        hi[s] = 0.0f;
        lo[s] = 0.0f;
        A[s] = 0.0f;
        const int e = s - (KM - K);
        if (e >= 0 && e < n) {
            float4 r0, r1, r2, r3;
            load_rec(a.ws.rec, vb + id[s], r0, r1, r2, r3);
            const Entry en = entry_px(r0, r1, r2, r3, px, py);
            hi[s] = en.hi;
            lo[s] = en.lo;
            jst[e * NT + tid] = make_float4(en.hi, en.lo, en.r, 0.5f * en.a);
        }
    }
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
    // W_k = T_k a_k, written over A_k
    const float ntl = -vd.tau * kLog2e;
    {
        int e = 0;
#pragma unroll
        for (int s = 0; s < KM; ++s) {
            if (s >= KM - K && s - (KM - K) < n) {
                const float am = jst[e * NT + tid].w;
                A[s] = ex2_approx(ntl * A[s]) * (2.0f * am);
                ++e;
            } else {
                A[s] = 0.0f;
            }
        }
    }
    // ---------------- weights and image ----------------
    __syncwarp();
#pragma unroll
    for (int s = 0; s < KM; ++s)
        if (s >= KM - K) *stg(lane * L + (s - (KM - K))) = A[s];
    __syncwarp();
    if (vd.weights) {
#pragma unroll
        for (int rw = 0; rw < 2; ++rw) {
            const int irow = ty * TH + 2 * warp + rw;
            if (irow >= H) continue;
            float* dw = vd.weights + ((int64_t)irow * W + tx * kTileW) * L;
            for (int x = lane; x < ncols * L; x += 32) dw[x] = *stg(rw * 16 * L + x);
        }
    }
    // the blend reads the lists back from the index output this warp wrote
    if (C >= 64) {
        // wide attributes: the warp blends one pixel at a time, lanes over channels
        for (int p = 0; p < 32; ++p) {
            const int irow = ty * TH + 2 * warp + (p >> 4), jcol = tx * kTileW + (p & 15);
            if (irow >= H || jcol >= W) continue;
            const int64_t pp = (int64_t)irow * W + jcol;
            for (int c0 = 0; c0 < C; c0 += 32) {
                const int c = c0 + lane;
                float acc = 0.0f;
                for (int k = 0; k < L; ++k) {
                    const int32_t g = vd.index[pp * L + k];
                    if (g < 0) break;
                    if (c < C) acc = fmaf(*stg(p * L + k), __ldg(vd.attr + (int64_t)g * C + c), acc);
                }
                if (c < C) vd.image[pp * C + c] = acc;
            }
        }
    } else if (valid && C <= 4) {
        // narrow attributes: one pass over the list, all channels at once
        float acc0 = 0.0f, acc1 = 0.0f, acc2 = 0.0f, acc3 = 0.0f;
        const int32_t* li = vd.index + pix * L;
        for (int k = 0; k < n; ++k) {
            const float w = *stg(lane * L + k);
            const float* ap = vd.attr + (int64_t)li[k] * C;
            acc0 = fmaf(w, __ldg(ap), acc0);
            if (C > 1) acc1 = fmaf(w, __ldg(ap + 1), acc1);
            if (C > 2) acc2 = fmaf(w, __ldg(ap + 2), acc2);
            if (C > 3) acc3 = fmaf(w, __ldg(ap + 3), acc3);
        }
        float* ip = vd.image + pix * C;
        ip[0] = acc0;
        if (C > 1) ip[1] = acc1;
        if (C > 2) ip[2] = acc2;
        if (C > 3) ip[3] = acc3;
    } else if (valid) {
        // this lane's list: indices from the index output, weights from the staging area
        const bool v4 = (C & 3) == 0 && ((reinterpret_cast<uintptr_t>(vd.attr) |
                                          reinterpret_cast<uintptr_t>(vd.image)) & 15) == 0;
        if (v4) {
            for (int c = 0; c < C; c += 4) {
                float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
                for (int k = 0; k < n; ++k) {
                    const int32_t g = vd.index[pix * L + k];
                    const float w = *stg(lane * L + k);
                    const float4 a4 = __ldg(reinterpret_cast<const float4*>(vd.attr + (int64_t)g * C + c));
                    acc.x = fmaf(w, a4.x, acc.x);
                    acc.y = fmaf(w, a4.y, acc.y);
                    acc.z = fmaf(w, a4.z, acc.z);
                    acc.w = fmaf(w, a4.w, acc.w);
                }
                *reinterpret_cast<float4*>(vd.image + pix * C + c) = acc;
            }
        } else {
            for (int c = 0; c < C; ++c) {
                float acc = 0.0f;
                for (int k = 0; k < n; ++k) {
                    const int32_t g = vd.index[pix * L + k];
                    acc = fmaf(*stg(lane * L + k), __ldg(vd.attr + (int64_t)g * C + c), acc);
                }
                vd.image[pix * C + c] = acc;
            }
        }
    }
}

template <int KM, int TH>
__global__ void __launch_bounds__(16 * TH, TH == 16 ? 2 : 3) k_render(Args a) {
    __shared__ int s_slot;
    for (;;) {
        const int t = next_tile(a, 1, &s_slot);
        if (t < 0) return;
        render_tile<KM, TH>(a, t);
    }
}

// ---------------------------------------------------------------------------
// Generic path for list lengths above the register lists (L > 32): same tile
// staging, the per-pixel list kept sorted in the workspace.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void render_tile_generic(const Args& a, int t) {
    constexpr int NT = 256, TH = 16;
    extern __shared__ float4 smem[];
    float4* stage = smem;
    int32_t* sgid = reinterpret_cast<int32_t*>(stage + 4 * NT);

    const int v = view_of_tile(a.views, a.hdr->nviews, t);
    const ViewDesc& vd = a.views[v];
    const int lt = t - vd.tile_base;
    const int tiles_x = vd.tiles_x;
    const int tx = lt % tiles_x, ty = lt / tiles_x;
    const int H = vd.H, W = vd.W;
    const int tid = threadIdx.x;
    const int j = tx * kTileW + (tid & 15);
    const int i = ty * TH + (tid >> 4);
    const bool valid = (i < H) && (j < W);
    const float px = (float)j + 0.5f, py = (float)i + 0.5f;
    const int64_t pix = (int64_t)i * W + j;
    const int64_t vb = vd.rec_base;
    const int L = vd.L;
    const int64_t gpix = vd.pix_base + pix;
    float* lk = a.ws.gkey + gpix * (int64_t)a.ws.gen_L * 8;
    int32_t* li = a.ws.gid + gpix * (int64_t)a.ws.gen_L;
    int n = 0;

    const TileSrc src = tile_source<NT>(a, vd, t);
    bool active = valid;
    for (int base = 0; base < src.count; base += NT) {
        const int nc = min(NT, src.count - base);
        if (tid < nc) {
            int32_t g;
            if (src.mode != 2) g = a.ws.tile_gauss[src.start + base + tid];
            else g = base + tid;
            float4 r0, r1, r2, r3;
            load_rec(a.ws.rec, vb + g, r0, r1, r2, r3);
            if (src.filter_box) {
                const int4 tb = a.ws.tbox[vb + g];
                if (tx < tb.x || tx > tb.y || ty < tb.z || ty > tb.w) {
                    r1 = make_float4(0.f, 0.f, 0.f, 0.f);
                    r2 = r1;
                }
            }
            stage[tid] = r0;
            stage[NT + tid] = r1;
            stage[2 * NT + tid] = r2;
            stage[3 * NT + tid] = r3;
            sgid[tid] = g;
        }
        __syncthreads();
        if (active) {
            for (int q = 0; q < nc; ++q) {
                const float4 r3 = stage[3 * NT + q];
                const float kth = (n == L) ? lk[L - 1] : INFINITY;
                if (src.mode == 1 && r3.w > kth) {
                    active = false;
                    break;
                }
                const float l = candidate_key(stage[q], stage[NT + q], stage[2 * NT + q], r3, px, py, vd.Qeta);
                if (l > 0.0f) {
                    const int32_t g = sgid[q];
                    if (n < L || l < lk[L - 1] || (l == lk[L - 1] && g < li[L - 1])) {
                        int p = (n < L) ? n : L - 1;
                        while (p > 0 && (lk[p - 1] > l || (lk[p - 1] == l && li[p - 1] > g))) {
                            lk[p] = lk[p - 1];
                            li[p] = li[p - 1];
                            --p;
                        }
                        lk[p] = l;
                        li[p] = g;
                        if (n < L) ++n;
                    }
                }
            }
        }
        if (__syncthreads_and(!active)) break;
    }
    if (valid) {
        // fine pass with both loops over the list in global memory (L1 resident)
        float* lw = vd.weights ? vd.weights + pix * L : nullptr;
        for (int k = 0; k < n; ++k) {
            float4 r0, r1, r2, r3;
            load_rec(a.ws.rec, vb + li[k], r0, r1, r2, r3);
            const Entry ek = entry_px(r0, r1, r2, r3, px, py);
            float A = 0.0f;
            for (int jj = 0; jj < n; ++jj) {
                load_rec(a.ws.rec, vb + li[jj], r0, r1, r2, r3);
                const Entry ej = entry_px(r0, r1, r2, r3, px, py);
                const float u = ((ek.hi - ej.hi) + (ek.lo - ej.lo)) * ej.r;
                const float q = erfc_as28(fabsf(u));
                const float m = 0.5f * ej.a;
                const float sm = copysignf(m, u);
                A = fmaf(-sm, q, A + (m + sm));
            }
            lk[L + k] = ex2_approx(-vd.tau * kLog2e * A) * ek.a;  // W_k
        }
        for (int k = 0; k < L; ++k) {
            const bool real = k < n;
            vd.index[pix * L + k] = real ? li[k] : -1;
            if (lw) lw[k] = real ? lk[L + k] : 0.0f;
        }
        for (int c = 0; c < vd.C; ++c) {
            float acc = 0.0f;
            for (int k = 0; k < n; ++k) acc = fmaf(lk[L + k], __ldg(vd.attr + (int64_t)li[k] * vd.C + c), acc);
            vd.image[pix * vd.C + c] = acc;
        }
    }
    __syncthreads();
}

__global__ void __launch_bounds__(256) k_render_generic(Args a) {
    __shared__ int s_slot;
    for (;;) {
        const int t = next_tile(a, 1, &s_slot);
        if (t < 0) return;
        render_tile_generic(a, t);
    }
}

size_t render_smem_bytes(int KM, int TH) {
    const int NT = 16 * TH;
    const size_t phase1 = (size_t)NT * 64 + (size_t)NT * 4 + (size_t)NT * TH * 2 + (size_t)NT * (NT / 32) * 4 +
                          (size_t)KM * NT * 8;
    const size_t phase2 = (size_t)KM * NT * 16;
    return phase1 > phase2 ? phase1 : phase2;
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

template <typename Kern>
static int blocks_per_sm(Kern k, int nthreads, size_t smem) {
    if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, nthreads, smem) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

// Resident CTAs per SM of the forward tile kernel for capacity KM.
int render_blocks_per_sm(int KM) {
    switch (KM) {
        case 8: return blocks_per_sm(k_render<8, 16>, 256, render_smem_bytes(8, 16));
        case 16: return blocks_per_sm(k_render<16, 16>, 256, render_smem_bytes(16, 16));
        case 20: return blocks_per_sm(k_render<20, 16>, 256, render_smem_bytes(20, 16));
        case 24: return blocks_per_sm(k_render<24, 16>, 256, render_smem_bytes(24, 16));
        case 32: return blocks_per_sm(k_render<32, 8>, 128, render_smem_bytes(32, 8));
        default: return blocks_per_sm(k_render_generic, 256, render_smem_bytes(0, 16));
    }
}

// Launch the forward tile kernel for register-list capacity KM (0 = generic):
// `nblocks` persistent CTAs that take tiles of class a.cls from the header.
cudaError_t launch_render_tiles(int KM, int nblocks, cudaStream_t s, const Args& a) {
    switch (KM) {
        case 8: return launch_tiles(k_render<8, 16>, "k_render<8>", nblocks, 256, render_smem_bytes(8, 16), s, a);
        case 16: return launch_tiles(k_render<16, 16>, "k_render<16>", nblocks, 256, render_smem_bytes(16, 16), s, a);
        case 20: return launch_tiles(k_render<20, 16>, "k_render<20>", nblocks, 256, render_smem_bytes(20, 16), s, a);
        case 24: return launch_tiles(k_render<24, 16>, "k_render<24>", nblocks, 256, render_smem_bytes(24, 16), s, a);
        case 32: return launch_tiles(k_render<32, 8>, "k_render<32>", nblocks, 128, render_smem_bytes(32, 8), s, a);
        default: return launch_tiles(k_render_generic, "k_render_generic", nblocks, 256, render_smem_bytes(0, 16), s, a);
    }
}

}  // namespace voge
