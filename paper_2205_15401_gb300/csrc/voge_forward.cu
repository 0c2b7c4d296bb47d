// voge_forward.cu -- the forward pass: coarse selection and fine pass, fused
// in one persistent kernel (k_render) or split into a selection kernel and a
// standalone fine kernel (k_fine, also behind voge_render_fine).
//
// Coarse pass (Sec. 3.3, App. A.3), one thread per pixel of a 16 x TH tile:
// the tile's candidate Gaussians (binned and, when eta > 0, sorted by a lower
// bound of l by k_sort_tiles) are staged in shared memory in chunks of 16 TH.
// While staging, each candidate's threshold conic gives a 16-bit pixel mask
// per tile row; a warp bit transpose turns these into per-pixel hit words.
// Every pixel traces (Eq. 6) only the candidates whose mask covers it, keeps
// those with e^{q} > eta and l > 0, and holds the K nearest by (l, index) in
// its own shared-memory column, kept sorted by insertion (candidates arrive
// nearly in depth order, so an insertion mostly appends or moves one entry).
// A pixel stops once no later candidate can enter.
//
// Fine pass (Eq. 7-8), one warp per 16-pixel row segment: with the kept list
// S_p of each pixel,
//   A_k = sum_{j in S_p} (a_j/2)(1 + erf((l_k - l_j) sqrt(b_j/2))),
//   T_k = exp(-tau A_k),  W_k = T_k a_k,  image = sum_k W_k c_k.
// The segment's entries (pixel, slot) are packed over the lanes: a lane sets
// up one entry (l as two floats, r = sqrt(b/2), m = a/2) from the kernel's
// record, then sums its A_k over its pixel's list, so that lanes stay busy
// whatever the lists' lengths.  erf is Abramowitz & Stegun 7.1.28 on the FMA
// pipe plus one MUFU reciprocal.
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
    const int tc = (int)VOGE_IDX(a.hdr, t, a.hdr->total_tiles, kChkTile);
    const int cnt = a.ws.tile_cnt[tc];
    const int off = a.ws.tile_off[tc];
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

// ---------------------------------------------------------------------------
// Fine pass (Eq. 7-8), weights and blend of one 16-pixel row segment by one
// warp, with the entries packed over the lanes:
//   A_k = sum_{j in S_p} (a_j/2)(1 + erf((l_k - l_j) sqrt(b_j/2))),
//   W_k = e^{-tau A_k} a_k,  image_p = sum_k W_k c_k.
// The segment's kept entries (pixel p, slot k < n_p) are numbered pixel after
// pixel; lane i of a step takes entry i.  A lane first sets up its entry from
// the kernel's record (l = hi + lo, r = sqrt(b/2), m = a/2 for this pixel),
// then sums its A_k over its pixel's list, so that lists of any length keep
// every lane busy and the record gathers of 32 entries are in flight at once.
// ---------------------------------------------------------------------------
template <int KM>
struct SegScratch {  // per warp
    static constexpr int kItems = 16 * KM;
    static constexpr size_t e_off = 0;                            // float4 E[KM][16]: (hi, lo, r, m)
    static constexpr size_t w_off = (size_t)kItems * 16;          // float Wst[16][L]
    static constexpr size_t b_off = w_off + (size_t)kItems * 4;   // int pbase[16], pcnt[16]; float msum[16]
    static constexpr size_t bytes = b_off + 192;
};

// irow: the segment's image row; its pixels are columns 16 tx + p, p < 16.
// Lane p < 16 passes n_p in np_lane; id_of(p, k) is entry k of pixel p's
// list (k < n_p).  scratch: this warp's SegScratch.  The weights (W_k, then
// zeros up to L) and the image of the segment's pixels are written.
template <int KM, typename IdFn>
__device__ __forceinline__ void fine_segment(const Args& a, const ViewDesc& vd, int tx, int irow, int np_lane,
                                             IdFn id_of, char* scratch) {
    using S = SegScratch<KM>;
    float4* E = reinterpret_cast<float4*>(scratch + S::e_off);
    float* Wst = reinterpret_cast<float*>(scratch + S::w_off);
    int* pbase = reinterpret_cast<int*>(scratch + S::b_off);
    int* pcnt = pbase + 16;
    float* msum = reinterpret_cast<float*>(pcnt + 16);
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const int H = vd.H, W = vd.W, L = vd.L, C = vd.C;
    const int64_t vb = vd.rec_base;
    if (irow >= H) return;
    const int col0 = tx * kTileW;
    const int ncols = min(kTileW, W - col0);
    const float py = (float)irow + 0.5f;
    const bool px_ok = lane < ncols;  // lanes 0..15 are the segment's pixels
    float* dw = vd.weights ? vd.weights + ((int64_t)irow * W + col0) * L : nullptr;
    float* img = vd.image + (VOGE_IDX(a.hdr, ((int64_t)irow * W + col0 + ncols) * C - 1, (int64_t)H * W * C, kChkOutput) -
                             ((int64_t)ncols * C - 1));

    // entry numbering: pixel p's entries are [pbase[p], pbase[p] + n_p)
    const int n = (lane < 16 && px_ok) ? np_lane : 0;
    int incl = n;
#pragma unroll
    for (int d = 1; d < 16; d <<= 1) {
        const int t = __shfl_up_sync(FULL, incl, d);
        if (lane >= d) incl += t;
    }
    const int total = __shfl_sync(FULL, incl, 15);
    if (total == 0) {  // no pixel of the segment keeps anything: zero weights and image
        if (dw)
            for (int x = lane; x < ncols * L; x += 32) dw[x] = 0.0f;
        for (int x = lane; x < ncols * C; x += 32) img[x] = 0.0f;
        return;
    }
    const int excl = incl - n;
    // the pixel of entry i: the last p < 16 with pbase[p] <= i (pixels with
    // no entries share the next one's base, so the last such p owns i)
    auto pixel_of = [&](int i) -> int {
        int p = 0;
#pragma unroll
        for (int step = 8; step >= 1; step >>= 1) {
            const int b = __shfl_sync(FULL, excl, p + step);
            if (b <= i) p += step;
        }
        return p;
    };
    if (lane < 16) {
        pbase[lane] = excl;
        pcnt[lane] = n;
    }
    __syncwarp();
    // Set-up, 64 entries at a time (two per lane, their records in flight
    // together).  The entries are taken by list position first -- row k holds
    // the pixels whose lists are longer than k (mask M_k, lane k holds it and
    // the number of entries before row k) -- so that neighbouring lanes take
    // neighbouring pixels at one position, which often keep the same kernel:
    // their record gathers share lines.  E is stored the same way, E[k][p].
    unsigned mrow = 0u;
#pragma unroll
    for (int k = 0; k < KM; ++k) {
        const unsigned m = __ballot_sync(FULL, n > k);
        if (lane == k) mrow = m;
    }
    const int crow = __popc(mrow);
    int rincl = crow;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) {
        const int t = __shfl_up_sync(FULL, rincl, d);
        if (lane >= d) rincl += t;
    }
    const int rexcl = rincl - crow;
    // every row full (all 16 pixels keep L entries): entry i is (i / 16, i % 16)
    const bool rows_full = total == 16 * L;
    for (int i0 = 0; i0 < total; i0 += 64) {
        float4 r[2][4];
        int pp[2], kk[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int i = min(i0 + 32 * h + lane, total - 1);
            int k = i >> 4, p = i & 15;
            if (!rows_full) {
                k = 0;  // the last row whose first entry is at or before i
#pragma unroll
                for (int step = 16; step >= 1; step >>= 1) {
                    const int b = __shfl_sync(FULL, rexcl, k + step);
                    if (k + step < KM && b <= i) k += step;
                }
                unsigned m = __shfl_sync(FULL, mrow, k);
                int rr = i - __shfl_sync(FULL, rexcl, k);  // the rr-th set bit of M_k
                p = 0;
#pragma unroll
                for (int w = 8; w >= 1; w >>= 1) {
                    const int c = __popc(m & ((1u << w) - 1u));
                    if (rr >= c) {
                        rr -= c;
                        m >>= w;
                        p += w;
                    }
                }
            }
            pp[h] = p;
            kk[h] = k;
            const int64_t g = VOGE_IDX(a.hdr, id_of(p, k), vd.N, kChkRecord);
            load_rec(a.ws.rec, vb + g, r[h][0], r[h][1], r[h][2], r[h][3]);
        }
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            if (i0 + 32 * h + lane < total) {
                const Entry en = entry_px(r[h][0], r[h][1], r[h][2], r[h][3], (float)(col0 + pp[h]) + 0.5f, py);
                E[kk[h] * 16 + pp[h]] = make_float4(en.hi, en.lo, en.r, 0.5f * en.a);
            }
        }
    }
    __syncwarp();
    // sum of m_j over each pixel's list: 1 + erf(u) = 1 + sign(u) erf|u|, so
    // A_k = sum_j m_j + sum_j copysign(m_j, u_kj) (1 - erfc|u_kj|)
    {
        // two lanes per pixel (even and odd list positions), one shuffle
        const int pp = lane & 15;
        const int np = __shfl_sync(FULL, n, pp);
        float ms = 0.0f;
        for (int k = lane >> 4; k < np; k += 2) ms += E[k * 16 + pp].w;
        ms += __shfl_down_sync(FULL, ms, 16);
        if (lane < 16) msum[lane] = ms;
    }
    __syncwarp();
    const bool narrow = C <= 4;
    const float ntl = -vd.tau * kLog2e;
    auto pair = [](const float4& Kq, const float4& J, float& A) {
        const float u = ((Kq.x - J.x) + (Kq.y - J.y)) * J.z;
        A = fmaf(copysignf(J.w, u), 1.0f - erfc_as28(fabsf(u)), A);
    };
    // with every list full, pixel i / L (a multiply and a shift: exact for
    // i < 32 L <= 1024 and L <= 32) replaces the search over the bases
    const int div_mul = (65536 + L - 1) / L;
    for (int i0 = 0; i0 < total; i0 += 32) {
        const int i = i0 + lane;
        const int p = rows_full ? (min(i, total - 1) * div_mul) >> 16 : pixel_of(i < total ? i : total - 1);
        if (i < total) {
            const int base = rows_full ? p * L : pbase[p], np = rows_full ? L : pcnt[p];
            const float4 Kq = E[(i - base) * 16 + p];
            const float4* Jp = E + p;  // entry j of pixel p: Jp[16 j]
            float A0 = 0.0f, A1 = 0.0f;
            int j = 0;
            for (; j + 3 < np; j += 4) {
                const float4 J0 = Jp[16 * j], J1 = Jp[16 * (j + 1)], J2 = Jp[16 * (j + 2)], J3 = Jp[16 * (j + 3)];
                pair(Kq, J0, A0);
                pair(Kq, J1, A1);
                pair(Kq, J2, A0);
                pair(Kq, J3, A1);
            }
            for (; j < np; ++j) pair(Kq, Jp[16 * j], A0);
            Wst[p * L + (i - base)] = ex2_approx(ntl * (msum[p] + (A0 + A1))) * (2.0f * Kq.w);
        }
    }
    if (lane < 16)
        for (int k = n; k < L; ++k) Wst[lane * L + k] = 0.0f;
    __syncwarp();
    if (dw)  // [16][L] is the segment's layout: one coalesced copy
        for (int x = lane; x < ncols * L; x += 32)
            vd.weights[VOGE_IDX(a.hdr, ((int64_t)irow * W + col0) * L + x, (int64_t)H * W * L, kChkOutput)] = Wst[x];
    if (narrow) {
        // image: two lanes per pixel (lane p and p + 16 take its even and odd
        // list positions), eight rows each in flight, added by one shuffle
        const int pp = lane & 15, h = lane >> 4;
        const int np = __shfl_sync(FULL, n, pp);
        float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
        if (pp < ncols) {
            for (int k0 = h; k0 < np; k0 += 16) {
                float4 c[8];
                float w[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int kk = k0 + 2 * u;
                    const int k = min(kk, np - 1);
                    w[u] = kk < np ? Wst[pp * L + k] : 0.0f;
                    const float* ap = vd.attr + VOGE_IDX(a.hdr, id_of(pp, k), vd.N, kChkRecord) * C;
                    c[u].x = __ldg(ap);
                    c[u].y = C > 1 ? __ldg(ap + 1) : 0.0f;
                    c[u].z = C > 2 ? __ldg(ap + 2) : 0.0f;
                    c[u].w = C > 3 ? __ldg(ap + 3) : 0.0f;
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    acc.x = fmaf(w[u], c[u].x, acc.x);
                    acc.y = fmaf(w[u], c[u].y, acc.y);
                    acc.z = fmaf(w[u], c[u].z, acc.z);
                    acc.w = fmaf(w[u], c[u].w, acc.w);
                }
            }
        }
        acc.x += __shfl_down_sync(FULL, acc.x, 16);
        acc.y += __shfl_down_sync(FULL, acc.y, 16);
        acc.z += __shfl_down_sync(FULL, acc.z, 16);
        acc.w += __shfl_down_sync(FULL, acc.w, 16);
        if (h == 0 && pp < ncols) {
            float* ip = img + pp * C;
            ip[0] = acc.x;
            if (C > 1) ip[1] = acc.y;
            if (C > 2) ip[2] = acc.z;
            if (C > 3) ip[3] = acc.w;
        }
        return;
    }
    // wider attributes: lanes over (entry group, 16-byte channel group or
    // channel); G groups of cw lanes take entries k = grp, grp + G, ... of a
    // pixel, four each in flight, and a shuffle reduction adds the groups up
    const bool v4 = (C & 3) == 0 && ((reinterpret_cast<uintptr_t>(vd.attr) | reinterpret_cast<uintptr_t>(img)) & 15) == 0;
    const int cw = v4 ? C >> 2 : C;  // row width in units of one lane's load
    const int G = cw >= 32 ? 1 : 1 << (31 - __clz(32 / cw));  // power of two, G cw <= 32
    const int grp = cw >= 32 ? 0 : lane / cw;
    const int cl = cw >= 32 ? lane : lane - grp * cw;
    const bool lane_on = grp < G;
    for (int cu0 = 0; cu0 < cw; cu0 += 32) {
        const int cu = cu0 + cl;
        const bool on = lane_on && cu < cw;
        for (int p = 0; p < ncols; ++p) {
            const int np = pcnt[p];
            float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
            for (int k0 = 0; k0 < np; k0 += 4 * G) {
                float4 x[4];
                float w[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const int kk = k0 + u * G + grp;
                    const int k = min(kk, np - 1);
                    w[u] = (on && kk < np) ? Wst[p * L + k] : 0.0f;
                    const float* ap = vd.attr + VOGE_IDX(a.hdr, id_of(p, k), vd.N, kChkRecord) * C;
                    if (!on) x[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                    else if (v4) x[u] = __ldg(reinterpret_cast<const float4*>(ap) + cu);
                    else x[u] = make_float4(__ldg(ap + cu), 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    acc.x = fmaf(w[u], x[u].x, acc.x);
                    acc.y = fmaf(w[u], x[u].y, acc.y);
                    acc.z = fmaf(w[u], x[u].z, acc.z);
                    acc.w = fmaf(w[u], x[u].w, acc.w);
                }
            }
            for (int off = cw; off < G * cw; off <<= 1) {
                acc.x += __shfl_down_sync(FULL, acc.x, off);
                acc.y += __shfl_down_sync(FULL, acc.y, off);
                acc.z += __shfl_down_sync(FULL, acc.z, off);
                acc.w += __shfl_down_sync(FULL, acc.w, off);
            }
            if (on && grp == 0) {
                if (v4) reinterpret_cast<float4*>(img + p * C)[cu] = acc;
                else img[p * C + cu] = acc.x;
            }
        }
    }
}

// Shared memory of one forward tile (NT = 16 TH threads, NW = NT / 32 warps):
//   selection: stage[4][NT] float4 | sgid[NT] | siv[TH][NT] u16 | smask[NT/32][NT] | slk[KM][NT]
//   after it:  one SegScratch per warp (over the selection buffers): the
//              index output's staging and the packed fine pass
//   sli[KM][NT], the sorted index lists: past both
template <int KM, int TH>
struct FwdSmem {
    static constexpr int NT = 16 * TH;
    static constexpr size_t sel0 = (size_t)NT * 64 + (size_t)NT * 4 + (size_t)NT * TH * 2 +
                                   (size_t)NT * (NT / 32) * 4 + (size_t)KM * NT * 4;
    static constexpr size_t fine = (size_t)(NT / 32) * SegScratch<KM>::bytes;
    static constexpr size_t ids_off = sel0 > fine ? sel0 : fine;
    static constexpr size_t bytes = ids_off + (size_t)KM * NT * 4;
};

// One forward tile: selection, index output and, with FINE, the fine pass,
// weights and image (without FINE, k_fine does those from the index output).
template <int KM, int TH, bool FINE>
__device__ __forceinline__ void render_tile(const Args& a, int t) {
    constexpr int NT = 16 * TH;
    using SM = FwdSmem<KM, TH>;
    extern __shared__ float4 smem[];
    float4* stage = smem;
    int32_t* sgid = reinterpret_cast<int32_t*>(stage + 4 * NT);
    uint16_t* siv = reinterpret_cast<uint16_t*>(sgid + NT);
    uint32_t* smask = reinterpret_cast<uint32_t*>(siv + TH * NT);  // [NT/32][NT] per-lane hit masks
    float* slk = reinterpret_cast<float*>(smask + (NT / 32) * NT);  // [KM][NT] per-lane kept depths
    int32_t* sli = reinterpret_cast<int32_t*>(reinterpret_cast<char*>(smem) + SM::ids_off);  // [KM][NT]

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
    const int64_t vb = vd.rec_base;
    const int K = vd.L;  // list length (<= KM)
    const float Qeta = vd.Qeta;

    // The kept list of this pixel lives in its own shared-memory column,
    // always sorted by (l, index).  Its last entry (lk_last, li_last), the
    // current maximum, is also held in registers: candidates arrive nearly
    // in depth order, so most insertions append after it (no shared-memory
    // read) or go just before it.  Once the list holds K entries, a nearer
    // candidate drops the last one.  kbar is the bar a candidate must pass
    // (+inf while the list is filling).
    int n = 0;
    float lk_last = -INFINITY, kbar = INFINITY;
    int32_t li_last = INT32_MIN;
    unsigned traced = 0;  // candidates this pixel traced (Eq. 6)

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
                if (FINE && vd.weights) vd.weights[p0 * L + x] = 0.0f;
            }
            if (FINE)
                for (int x = lane; x < ncols * C; x += 32) vd.image[p0 * C + x] = 0.0f;
        }
        return;
    }
    bool active = valid;
    // depth bound of the first candidate after the current chunk (sorted
    // order: it bounds every later one), staged with the chunk by thread 0
    __shared__ float s_next_bound;
    for (int base = 0; base < src.count; base += NT) {
        const int nc = min(NT, src.count - base);
        const bool has_next = src.mode == 1 && nc == NT && base + NT < src.count;
        if (tid < nc) {
            int32_t g, gn = 0;
            if (src.mode != 2) g = a.ws.tile_gauss[VOGE_IDX(a.hdr, src.start + base + tid, a.ws.bin_cap, kChkTileList)];
            else g = base + tid;
            if (tid == 0 && has_next)
                gn = (int32_t)VOGE_IDX(
                    a.hdr, __ldg(a.ws.tile_gauss + VOGE_IDX(a.hdr, src.start + base + NT, a.ws.bin_cap, kChkTileList)), vd.N,
                    kChkRecord);
            g = (int32_t)VOGE_IDX(a.hdr, g, vd.N, kChkRecord);
            float4 r0, r1, r2, r3;
            load_rec(a.ws.rec, vb + g, r0, r1, r2, r3);
            if (tid == 0 && has_next) s_next_bound = __ldg(&a.ws.rec[4 * (vb + gn) + 3].w);
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
        uint32_t words = 0;  // bit w: this lane has hits in mask word w
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
                words |= (m != 0u ? 1u : 0u) << w;
            }
        }
        if (active) {
            // 2) each lane walks its own hits: lanes of a warp trace different
            //    candidates at the same time instead of the union of all hits.
            //    One cursor runs over the non-empty mask words, so the warp
            //    iterates as often as its busiest lane has hits in the chunk.
            int w = 0;
            uint32_t m = 0;
            for (;;) {
                if (m == 0) {
                    if (words == 0) break;
                    w = __ffs(words) - 1;
                    words &= words - 1;
                    m = smask[w * NT + tid];
                }
                const int q = w * 32 + __ffs(m) - 1;
                m &= m - 1;
                const float4 r3 = stage[3 * NT + q];  // .w: the candidate's depth lower bound
                if (src.mode == 1 && r3.w > kbar) {
                    active = false;  // sorted by lower bound: nothing later can enter
                    break;
                }
                const float4 r0 = stage[q], r1 = stage[NT + q], r2 = stage[2 * NT + q];
                const float l = candidate_key(r0, r1, r2, r3, px, py, Qeta);
                ++traced;
                if (!(l > 0.0f)) continue;
                const int32_t g = sgid[q];
                const bool full = n == K;
                if (full && !(l < lk_last || (l == lk_last && g < li_last))) continue;
                // insertion: p is the slot to fill (append, or the last one,
                // which drops out); larger entries move up by one
                int p = full ? K - 1 : n;
                float x = lk_last;  // entry p - 1: the cached last one when appending
                int32_t y = li_last;
                if (full && p > 0) {
                    x = slk[(p - 1) * NT + tid];
                    y = sli[(p - 1) * NT + tid];
                }
                bool moved = false;
                while (p > 0 && (x > l || (x == l && y > g))) {
                    slk[p * NT + tid] = x;
                    sli[p * NT + tid] = y;
                    if (!moved) {  // the first entry moved lands in the last slot
                        lk_last = x;
                        li_last = y;
                        moved = true;
                    }
                    --p;
                    if (p > 0) {
                        x = slk[(p - 1) * NT + tid];
                        y = sli[(p - 1) * NT + tid];
                    }
                }
                slk[p * NT + tid] = l;
                sli[p * NT + tid] = g;
                if (!moved) {
                    lk_last = l;
                    li_last = g;
                }
                if (!full) ++n;
                if (n == K) kbar = lk_last;
            }
            // a pixel whose list is full and whose next candidate (in sorted
            // order) starts beyond its K-th depth can stop for good
            if (active && has_next && s_next_bound > kbar) active = false;
        }
        if (__syncthreads_and(!active)) break;
    }
    // the call's counts: one addition per warp
    {
        const unsigned w_traced = __reduce_add_sync(0xffffffffu, traced);
        const unsigned w_entries = __reduce_add_sync(0xffffffffu, (unsigned)n);
        const unsigned w_pairs = __reduce_add_sync(0xffffffffu, (unsigned)(n * n));
        if ((tid & 31) == 0) {
            atomicAdd(&a.hdr->traces, (unsigned long long)w_traced);
            atomicAdd(&a.hdr->entries, (unsigned long long)w_entries);
            atomicAdd(&a.hdr->pairs, (unsigned long long)w_pairs);
            // this warp's row pair is a live unit of the backward (unit
            // numbering: TH / 2 per tile, the warps of a tile in order)
            if (w_entries > 0 && a.ws.live_hdr) {
                const int pos = atomicAdd(&a.ws.live_hdr->n[a.cls], 1);
                a.ws.live[(TH / 2) * a.hdr->class_begin[a.cls] + pos] = make_int2((TH / 2) * t + (tid >> 5), v);
            }
        }
    }
    // The lists are sorted; the selection buffers are free from here on.
    // Each warp holds two 16-pixel row segments of the tile (lanes 0-15 and
    // 16-31).  Per segment: the index output, staged in the warp's scratch as
    // the segment's [16][L] layout and copied out with coalesced stores; then
    // (FINE) the packed fine pass over the same lists.
    const int L = vd.L;
    const int lane = tid & 31, warp = tid >> 5;
    const int ncols = min(kTileW, W - tx * kTileW);
    char* scratch = reinterpret_cast<char*>(smem) + (size_t)warp * SegScratch<KM>::bytes;
    int32_t* istg = reinterpret_cast<int32_t*>(scratch + SegScratch<KM>::w_off);
#pragma unroll
    for (int rw = 0; rw < 2; ++rw) {
        const int irow = ty * TH + 2 * warp + rw;
        const int colb = 32 * warp + 16 * rw;  // sli column of the segment's pixel 0
        const int np_lane = __shfl_sync(0xffffffffu, n, 16 * rw + (lane & 15));
        {
            // two lanes per pixel (even and odd list positions)
            const int pp = lane & 15;
            for (int k = lane >> 4; k < L; k += 2) istg[pp * L + k] = k < np_lane ? sli[k * NT + colb + pp] : -1;
        }
        __syncwarp();
        if (irow < H) {
            const int64_t o0 = ((int64_t)irow * W + tx * kTileW) * L;
            for (int x = lane; x < ncols * L; x += 32)
                vd.index[VOGE_IDX(a.hdr, o0 + x, (int64_t)H * W * L, kChkOutput)] = istg[x];
        }
        __syncwarp();
        if constexpr (FINE) {
            auto id_of = [&](int p, int k) -> int32_t { return sli[k * NT + colb + p]; };
            fine_segment<KM>(a, vd, tx, irow, np_lane, id_of, scratch);
            __syncwarp();
        }
    }
}

// CTAs per SM of the tile kernels (three of 256 threads or four of 128):
// enough warps to hide the latency of the selection walk.
template <int TH, bool FINE>
__host__ __device__ constexpr int render_ctas() { return TH == 16 ? 3 : 4; }

template <int KM, int TH, bool FINE>
__global__ void __launch_bounds__(16 * TH, render_ctas<TH, FINE>()) k_render(Args a) {
    __shared__ int s_slot;
    for (;;) {
        const int t = next_tile(a, 1, &s_slot);
        if (t < 0) return;
        render_tile<KM, TH, FINE>(a, t);
    }
}

// Standalone fine pass over given index lists (voge_render_fine, and the
// split forward).  Each CTA is one warp, persistent.  It takes groups of
// kFineRows consecutive 16-pixel row segments of one binning tile from a work
// counter (neighbouring rows keep mostly the same kernels, whose records then
// stay in L1) and runs the packed fine pass on them one after another; while
// it works on one segment, the index row of the next is already on its way
// into shared memory (cp.async, double-buffered).  Nothing is shared between
// warps: there is no CTA barrier.
constexpr int kFineRows = 4;
template <int KM>
struct FineSmem {
    static constexpr size_t buf = (size_t)16 * KM * 4;  // one segment's lists: [16][L <= KM] int32
    static constexpr size_t bytes = SegScratch<KM>::bytes + 2 * buf;
};


// Row r of group g: its view, tile column and image row.
struct FineRow {
    int v, tx, irow;
};
__device__ __forceinline__ FineRow fine_row(const Args& a, int g, int r, int gpt) {
    const int t = g / gpt, gi = g - t * gpt;
    FineRow f;
    f.v = view_of_tile(a.views, a.hdr->nviews, t);
    const ViewDesc& vd = a.views[f.v];
    const int lt = t - vd.tile_base;
    f.tx = lt % vd.tiles_x;
    f.irow = (lt / vd.tiles_x) * vd.tile_h + gi * kFineRows + r;
    return f;
}

// Start the copy of a segment's lists ([16][L], -1 where the image ends) into
// buf; a group past the end only commits an empty copy group.
__device__ __forceinline__ void fine_prefetch(const Args& a, int g, int r, int ngroups, int gpt, bool v16,
                                              int32_t* buf) {
    const int lane = threadIdx.x & 31;
    if (g < ngroups) {
        const FineRow f = fine_row(a, g, r, gpt);
        const ViewDesc& vd = a.views[f.v];
        const int L = vd.L, W = vd.W;
        const int cnt = f.irow < vd.H ? min(kTileW, W - f.tx * kTileW) * L : 0;
        int64_t o0 = ((int64_t)f.irow * W + f.tx * kTileW) * L;
        if (cnt > 0) o0 = VOGE_IDX(a.hdr, o0 + cnt - 1, (int64_t)vd.H * W * L, kChkListRead) - (cnt - 1);
        const int32_t* src = vd.index_in + o0;
        if (v16) {
            for (int x = 4 * lane; x < cnt; x += 128) cp_async16(buf + x, src + x);
        } else {
            for (int x = lane; x < cnt; x += 32) cp_async4(buf + x, src + x);
        }
        for (int x = cnt + lane; x < 16 * L; x += 32) buf[x] = -1;
    }
    cp_async_commit();
}

template <int KM>
__global__ void __launch_bounds__(32, KM <= 20 ? 24 : 16) k_fine(Args a, int ngroups, int gpt, int v16) {
    extern __shared__ float4 smem[];
    char* scratch = reinterpret_cast<char*>(smem);
    int32_t* bufs = reinterpret_cast<int32_t*>(scratch + SegScratch<KM>::bytes);
    constexpr int kBuf = (int)(FineSmem<KM>::buf / 4);
    const int lane = threadIdx.x;
    int* ctr = &a.hdr->counters[3 * kMaxClasses + a.cls];
    auto claim = [&]() -> int {
        int u = 0;
        if (lane == 0) u = atomicAdd(ctr, 1);
        return __shfl_sync(0xffffffffu, u, 0);
    };
    int g = claim(), r = 0;   // the segment being processed
    int gn = g, rn = 1;       // the next one (kFineRows >= 2)
    fine_prefetch(a, g, r, ngroups, gpt, v16 != 0, bufs);
    fine_prefetch(a, gn, rn, ngroups, gpt, v16 != 0, bufs + kBuf);
    int slot = 0;
    while (g < ngroups) {
        cp_async_wait<1>();  // this lane's copies of the current segment are done
        __syncwarp();        // ... and every lane's
        int32_t* buf = bufs + slot * kBuf;
        const FineRow f = fine_row(a, g, r, gpt);
        const ViewDesc& vd = a.views[f.v];
        const int L = vd.L, N = vd.N;
        // lane p < 16: pixel p's list, the entries before the first one outside [0, N)
        int np = 0;
        if (lane < 16) {
            bool open = true;
            if (v16) {  // L is a multiple of 4: the row starts 16-byte aligned
                const int4* row = reinterpret_cast<const int4*>(buf + lane * L);
#pragma unroll
                for (int s4 = 0; s4 < KM / 4; ++s4) {
                    const int4 q = s4 < L / 4 ? row[s4] : make_int4(-1, -1, -1, -1);
                    open = open && (unsigned)q.x < (unsigned)N;
                    np += open ? 1 : 0;
                    open = open && (unsigned)q.y < (unsigned)N;
                    np += open ? 1 : 0;
                    open = open && (unsigned)q.z < (unsigned)N;
                    np += open ? 1 : 0;
                    open = open && (unsigned)q.w < (unsigned)N;
                    np += open ? 1 : 0;
                }
            } else {
#pragma unroll
                for (int s = 0; s < KM; ++s) {
                    const int32_t id = s < L ? buf[lane * L + s] : -1;
                    open = open && (unsigned)id < (unsigned)N;
                    np += open ? 1 : 0;
                }
            }
        }
        auto id_of = [&](int p, int k) -> int32_t { return buf[p * L + k]; };
        fine_segment<KM>(a, vd, f.tx, f.irow, np, id_of, scratch);
        __syncwarp();  // every lane is done with buf and the scratch
        g = gn;
        r = rn;
        if (g < ngroups) {
            rn = r + 1;
            if (rn == kFineRows) {
                gn = claim();
                rn = 0;
            }
        }
        fine_prefetch(a, gn, rn, ngroups, gpt, v16 != 0, buf);
        slot ^= 1;
    }
    cp_async_wait<0>();
}

size_t render_smem_bytes(int KM, int fine) {
    (void)fine;  // the fused and the selection-only kernel share one layout
    switch (KM) {
        case 8: return FwdSmem<8, 16>::bytes;
        case 16: return FwdSmem<16, 16>::bytes;
        case 20: return FwdSmem<20, 16>::bytes;
        case 24: return FwdSmem<24, 8>::bytes;
        case 32: return FwdSmem<32, 8>::bytes;
        default: return 0;  // lists longer than 32: voge_generic.cu
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

template <typename Kern>
static int blocks_per_sm(Kern k, int nthreads, size_t smem) {
    if (smem > 32 * 1024) cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, nthreads, smem) != cudaSuccess || nb < 1) nb = 1;
    return nb;
}

// Resident CTAs per SM of the forward tile kernel for capacity KM (fine:
// fused with the fine pass, else selection only).
int render_blocks_per_sm(int KM, int fine) {
    if (fine) {
        switch (KM) {
            case 8: return blocks_per_sm(k_render<8, 16, true>, 256, render_smem_bytes(8, 1));
            case 16: return blocks_per_sm(k_render<16, 16, true>, 256, render_smem_bytes(16, 1));
            case 20: return blocks_per_sm(k_render<20, 16, true>, 256, render_smem_bytes(20, 1));
            case 24: return blocks_per_sm(k_render<24, 8, true>, 128, render_smem_bytes(24, 1));
            case 32: return blocks_per_sm(k_render<32, 8, true>, 128, render_smem_bytes(32, 1));
            default: return 1;
        }
    }
    switch (KM) {
        case 8: return blocks_per_sm(k_render<8, 16, false>, 256, render_smem_bytes(8, 0));
        case 16: return blocks_per_sm(k_render<16, 16, false>, 256, render_smem_bytes(16, 0));
        case 20: return blocks_per_sm(k_render<20, 16, false>, 256, render_smem_bytes(20, 0));
        case 24: return blocks_per_sm(k_render<24, 8, false>, 128, render_smem_bytes(24, 0));
        case 32: return blocks_per_sm(k_render<32, 8, false>, 128, render_smem_bytes(32, 0));
        default: return 1;
    }
}

// Launch the forward tile kernel for register-list capacity KM (8..32):
// `nblocks` persistent CTAs that take tiles of class a.cls from the header.
// fine = 0 launches the selection-only form (index lists only).
cudaError_t launch_render_tiles(int KM, int nblocks, cudaStream_t s, const Args& a, int fine) {
    if (fine) {
        switch (KM) {
            case 8: return launch_tiles(k_render<8, 16, true>, "k_render<8>", nblocks, 256, render_smem_bytes(8, 1), s, a);
            case 16: return launch_tiles(k_render<16, 16, true>, "k_render<16>", nblocks, 256, render_smem_bytes(16, 1), s, a);
            case 20: return launch_tiles(k_render<20, 16, true>, "k_render<20>", nblocks, 256, render_smem_bytes(20, 1), s, a);
            case 24: return launch_tiles(k_render<24, 8, true>, "k_render<24>", nblocks, 128, render_smem_bytes(24, 1), s, a);
            case 32: return launch_tiles(k_render<32, 8, true>, "k_render<32>", nblocks, 128, render_smem_bytes(32, 1), s, a);
            default: return cudaErrorInvalidValue;  // lists longer than 32: launch_render_generic
        }
    }
    switch (KM) {
        case 8: return launch_tiles(k_render<8, 16, false>, "k_select<8>", nblocks, 256, render_smem_bytes(8, 0), s, a);
        case 16: return launch_tiles(k_render<16, 16, false>, "k_select<16>", nblocks, 256, render_smem_bytes(16, 0), s, a);
        case 20: return launch_tiles(k_render<20, 16, false>, "k_select<20>", nblocks, 256, render_smem_bytes(20, 0), s, a);
        case 24: return launch_tiles(k_render<24, 8, false>, "k_select<24>", nblocks, 128, render_smem_bytes(24, 0), s, a);
        case 32: return launch_tiles(k_render<32, 8, false>, "k_select<32>", nblocks, 128, render_smem_bytes(32, 0), s, a);
        default: return cudaErrorInvalidValue;
    }
}

// Launch the standalone fine pass over a.views[*].index_in for capacity KM
// (8..32): one warp per CTA, as many as can be resident, over groups of
// kFineRows row segments of every binning tile (tile_h / kFineRows per tile).
// v16: the lists can be copied in 16-byte pieces (L a multiple of 4, a
// 16-byte aligned index).
template <int KM>
static cudaError_t launch_fine_km(const char* name, int ngroups, int gpt, int v16, cudaStream_t s, const Args& a) {
    const size_t smem = FineSmem<KM>::bytes;
    static int per_sm[64] = {0};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    if (per_sm[dev] == 0) {
        int nb = 0, nsm = 1;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fine<KM>, 32, smem) != cudaSuccess || nb < 1) nb = 1;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
        per_sm[dev] = nb * nsm;
    }
    const int grid = ngroups < per_sm[dev] ? ngroups : per_sm[dev];
    TraceScope tr(name, s);
    k_fine<KM><<<grid, 32, smem, s>>>(a, ngroups, gpt, v16);
    return cudaPeekAtLastError();
}

cudaError_t launch_fine(int KM, int total_tiles, int tile_h, int L, const void* index, cudaStream_t s,
                        const Args& a) {
    const int gpt = tile_h / kFineRows;
    const int ngroups = total_tiles * gpt;
    if (ngroups <= 0) return cudaSuccess;
    const int v16 = (L % 4 == 0 && (reinterpret_cast<uintptr_t>(index) & 15) == 0) ? 1 : 0;
    switch (KM) {
        case 8: return launch_fine_km<8>("k_fine<8>", ngroups, gpt, v16, s, a);
        case 16: return launch_fine_km<16>("k_fine<16>", ngroups, gpt, v16, s, a);
        case 20: return launch_fine_km<20>("k_fine<20>", ngroups, gpt, v16, s, a);
        case 24: return launch_fine_km<24>("k_fine<24>", ngroups, gpt, v16, s, a);
        case 32: return launch_fine_km<32>("k_fine<32>", ngroups, gpt, v16, s, a);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace voge
