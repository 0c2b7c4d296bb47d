// voge_project.cu -- viewing transform, per-(view, Gaussian) records and
// tile binning (the coarse stage's culling).
//
// Sec. 3.3 (viewing transformation): M = R M_w + T, P = R P_w Rᵀ.
// App. A.3 (coarse rasterisation role): the paper rasterises a per-ellipsoid
// screen box at 1/8 resolution into a pixel->kernel assignment.  Here the box
// is the exact bounding box of the conic {pixels : e^{q} > eta} (plus a
// safety margin), binned into 16 x TH pixel tiles with a count / scan /
// scatter, so that a pixel only traces the Gaussians of its tile and the
// culling never changes a result.
#include "voge_device.cuh"
#include "voge_trace.cuh"

namespace voge {

__device__ __forceinline__ void project_one(const Args& a, int v, int64_t t, int count_tiles) {
    const ViewDesc& c = a.views[v];
    const int g = (int)(t - __ldg(&c.rec_base));
    const float* means = c.means;
    const float* inv_cov = c.inv_cov;
    const int use_thresh = __ldg(&c.use_thresh);
    const float Qeta = __ldg(&c.Qeta);
    float R[9], T[3];
#pragma unroll
    for (int q = 0; q < 9; ++q) R[q] = __ldg(&c.R[q]);
#pragma unroll
    for (int q = 0; q < 3; ++q) T[q] = __ldg(&c.T[q]);
    const float F = __ldg(&c.F), Ox = __ldg(&c.Ox), Oy = __ldg(&c.Oy), invF = __ldg(&c.invF);
    const int H = __ldg(&c.H), W = __ldg(&c.W), tiles_x = __ldg(&c.tiles_x), tile_h = __ldg(&c.tile_h);
    const int tile_base = __ldg(&c.tile_base);
    const int plain = __ldg(&c.plain);

    const float X = __ldg(means + 3 * (int64_t)g), Y = __ldg(means + 3 * (int64_t)g + 1),
                Z = __ldg(means + 3 * (int64_t)g + 2);
    float pw[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) pw[q] = __ldg(inv_cov + 6 * (int64_t)g + q);

    // camera-space mean in double-float
    dfl Mx = df_dot3_add(R[0], X, R[1], Y, R[2], Z, T[0]);
    dfl My = df_dot3_add(R[3], X, R[4], Y, R[5], Z, T[1]);
    dfl Mz = df_dot3_add(R[6], X, R[7], Y, R[8], Z, T[2]);

    // camera-space inverse covariance P = R Pw Rᵀ
    const float Pw[9] = {pw[0], pw[1], pw[2], pw[1], pw[3], pw[4], pw[2], pw[4], pw[5]};
    float A[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) A[3 * i + j] = fmaf(R[3 * i], Pw[j], fmaf(R[3 * i + 1], Pw[3 + j], R[3 * i + 2] * Pw[6 + j]));
    float P[6];  // xx xy xz yy yz zz
    P[0] = fmaf(A[0], R[0], fmaf(A[1], R[1], A[2] * R[2]));
    P[1] = fmaf(A[0], R[3], fmaf(A[1], R[4], A[2] * R[5]));
    P[2] = fmaf(A[0], R[6], fmaf(A[1], R[7], A[2] * R[8]));
    P[3] = fmaf(A[3], R[3], fmaf(A[4], R[4], A[5] * R[5]));
    P[4] = fmaf(A[3], R[6], fmaf(A[4], R[7], A[5] * R[8]));
    P[5] = fmaf(A[6], R[6], fmaf(A[7], R[7], A[8] * R[8]));

    float4 r0 = make_float4(0.f, 0.f, 0.f, 0.f), r1 = r0, r2 = r0, r3 = r0;
    float4 s0 = make_float4(P[0], P[1], P[2], P[3]);
    float4 s1 = make_float4(P[4], P[5], 0.f, 0.f);
    int4 tb = make_int4(1, 0, 1, 0);  // empty

    bool valid = Mz.hi > 0.0f && isfinite(Mz.hi) && isfinite(Mx.hi) && isfinite(My.hi);
#pragma unroll
    for (int q = 0; q < 6; ++q) valid = valid && isfinite(P[q]);
    if (valid) {
        const dfl xh = df_div(Mx, Mz), yh = df_div(My, Mz);
        const dfl uc = df_add(df_mul_f(xh, F), dfl{Ox, 0.0f});
        const dfl vc = df_add(df_mul_f(yh, F), dfl{Oy, 0.0f});
        const float x = xh.hi, y = yh.hi;
        // g = P Mh, beta0 = Mhᵀ P Mh
        const float gx = fmaf(P[0], x, fmaf(P[1], y, P[2]));
        const float gy = fmaf(P[1], x, fmaf(P[3], y, P[4]));
        const float gz = fmaf(P[2], x, fmaf(P[4], y, P[5]));
        const float beta0 = fmaf(gx, x, fmaf(gy, y, gz));
        const float invF2 = invF * invF;
        // adjugate of P (symmetric)
        const float a00 = fmaf(P[3], P[5], -P[4] * P[4]);
        const float a01 = fmaf(P[2], P[4], -P[1] * P[5]);
        const float a02 = fmaf(P[1], P[4], -P[2] * P[3]);
        const float a11 = fmaf(P[0], P[5], -P[2] * P[2]);
        const float a12 = fmaf(P[1], P[2], -P[0] * P[4]);
        const float a22 = fmaf(P[0], P[3], -P[1] * P[1]);
        // (M x D') = Mz (du c1 + dv c2)/F with c1 = (0, 1, -y), c2 = (-1, 0, x)
        const float c11 = fmaf(y, fmaf(a22, y, -2.0f * a12), a11);
        const float c22 = fmaf(x, fmaf(a22, x, -2.0f * a02), a00);
        const float c12 = fmaf(a12, x, fmaf(a02, y, fmaf(-a22 * x, y, -a01)));
        const float mzf = Mz.hi * invF;
        const float s2 = mzf * mzf;
        r0 = make_float4(uc.hi, uc.lo, vc.hi, vc.lo);
        r1 = make_float4(beta0, gx * invF, gy * invF, P[0] * invF2);
        r2 = make_float4(2.0f * P[1] * invF2, P[3] * invF2, s2 * c11, 2.0f * s2 * c12);
        // depth bound: l D is inside the ellipsoid (X-M)ᵀP(X-M) <= Qeta, so
        // |l - Mz| <= sqrt(Qeta Sigma_zz), Sigma_zz = a22 / det P.
        const float detP = fmaf(P[0], a00, fmaf(P[1], a01, P[2] * a02));
        float lmin = -INFINITY;
        if (use_thresh && detP > 0.0f && a22 > 0.0f) {
            const float h = sqrtf(Qeta * a22 / detP);
            lmin = Mz.hi - (1.001f * h + 1e-6f * Mz.hi);
            // snapped down to a multiple of 2^11 in the order-preserving
            // integer map: still a lower bound, and the tile sort keys the
            // list position into the freed low bits
            lmin = order_float(float_order(lmin) & ~((1u << kSortPosBits) - 1u));
        }
        r3 = make_float4(s2 * c22, Mz.hi, Mz.lo, lmin);
        s1.z = x;
        s1.w = y;

        // tile box of the conic qb - Qeta b < 0 (pixel units)
        int j0 = 0, j1 = W - 1, i0 = 0, i1 = H - 1;
        bool empty = false;
        if (use_thresh) {
            const float Q = Qeta;
            const float h00 = fmaf(-Q, r1.w, r2.z);
            const float h01 = fmaf(-Q, 0.5f * r2.x, 0.5f * r2.w);
            const float h11 = fmaf(-Q, r2.y, r3.x);
            const float hx = -Q * r1.y, hy = -Q * r1.z, h22 = -Q * beta0;
            const float det = fmaf(h00, h11, -h01 * h01);
            if (h00 > 0.0f && det > 1e-12f * h00 * h11 && isfinite(det)) {
                const float id = 1.0f / det;
                const float cx = -(h11 * hx - h01 * hy) * id;
                const float cy = -(h00 * hy - h01 * hx) * id;
                const float f0 = h22 + hx * cx + hy * cy;
                if (!(f0 < 0.0f)) {
                    empty = true;
                } else {
                    const float xr = sqrtf(-f0 * h11 * id) * 1.02f + 1.0f;
                    const float yr = sqrtf(-f0 * h00 * id) * 1.02f + 1.0f;
                    const float ucx = uc.hi + cx - 0.5f, vcy = vc.hi + cy - 0.5f;
                    const float fj0 = floorf(ucx - xr), fj1 = ceilf(ucx + xr);
                    const float fi0 = floorf(vcy - yr), fi1 = ceilf(vcy + yr);
                    if (isfinite(fj0) && isfinite(fj1) && isfinite(fi0) && isfinite(fi1)) {
                        if (fj1 < 0.0f || fi1 < 0.0f || fj0 > (float)(W - 1) || fi0 > (float)(H - 1)) {
                            empty = true;
                        } else {
                            j0 = max(0, (int)fmaxf(fj0, -1.0f));
                            j1 = min(W - 1, (int)fminf(fj1, (float)W));
                            i0 = max(0, (int)fmaxf(fi0, -1.0f));
                            i1 = min(H - 1, (int)fminf(fi1, (float)H));
                        }
                    }
                }
            }
        }
        if (!empty && W > 0 && H > 0) tb = make_int4(j0 / kTileW, j1 / kTileW, i0 / tile_h, i1 / tile_h);
    }
    a.ws.rec[4 * t + 0] = r0;
    a.ws.rec[4 * t + 1] = r1;
    a.ws.rec[4 * t + 2] = r2;
    a.ws.rec[4 * t + 3] = r3;
    a.ws.rec2[2 * t + 0] = s0;
    a.ws.rec2[2 * t + 1] = s1;
    a.ws.tbox[t] = tb;
    if (count_tiles && !plain) {
        // one of kTileSub counters per tile, picked by the Gaussian index, so
        // that the many Gaussians of a busy tile do not all hit one address
        const int sub = g & (kTileSub - 1);
        for (int ty = tb.z; ty <= tb.w; ++ty)
            for (int tx = tb.x; tx <= tb.y; ++tx)
                atomicAdd(&a.ws.tile_sub[VOGE_IDX(a.hdr, tile_base + ty * tiles_x + tx, a.hdr->total_tiles, kChkTile) * kTileSub +
                                         sub], 1);
    }
}

__global__ void __launch_bounds__(256) k_project(Args a, int count_tiles) {
    const int nv = a.hdr->nviews;
    const int64_t total = a.hdr->total_records;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        project_one(a, view_of_record(a.views, nv, t), t, count_tiles);
    }
}

// Per tile: the total of its sub-counts (tile_cnt) and their exclusive
// prefix within the tile (in place: the scatter cursors relative to the
// tile's first entry).  One thread per tile.
__global__ void __launch_bounds__(256) k_tile_totals(Args a) {
    static_assert(kTileSub == 8, "two 16-byte vectors of sub-counts per tile");
    const int n = a.hdr->total_tiles;
    int4* sub4 = reinterpret_cast<int4*>(a.ws.tile_sub);
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n; t += gridDim.x * blockDim.x) {
        const int4 u = sub4[2 * t], v = sub4[2 * t + 1];
        int4 cu, cv;
        cu.x = 0;
        cu.y = u.x;
        cu.z = cu.y + u.y;
        cu.w = cu.z + u.z;
        cv.x = cu.w + u.w;
        cv.y = cv.x + v.x;
        cv.z = cv.y + v.y;
        cv.w = cv.z + v.z;
        sub4[2 * t] = cu;
        sub4[2 * t + 1] = cv;
        a.ws.tile_cnt[t] = cv.w + v.w;
    }
}

// Exclusive scan of tile_cnt into tile_off (one CTA of 1024 threads, rounds
// of 4096 tiles, four consecutive tiles per thread).
__global__ void __launch_bounds__(1024) k_scan_tiles(Args a) {
    __shared__ int32_t warp_sums[32];
    const int n = a.hdr->total_tiles;
    const int tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    int32_t carry = 0;
    for (int base = 0; base < n; base += 4 * 1024) {
        const int q = base + 4 * tid;
        int4 c = make_int4(0, 0, 0, 0);
        if (q + 3 < n) {
            c = *reinterpret_cast<const int4*>(a.ws.tile_cnt + q);
        } else {
            if (q < n) c.x = a.ws.tile_cnt[q];
            if (q + 1 < n) c.y = a.ws.tile_cnt[q + 1];
            if (q + 2 < n) c.z = a.ws.tile_cnt[q + 2];
        }
        const int32_t s = (c.x + c.y) + (c.z + c.w);
        int32_t x = s;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[wid] = x;
        __syncthreads();
        if (wid == 0) {
            int32_t w = warp_sums[lane];
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int32_t y = __shfl_up_sync(0xffffffffu, w, o);
                if (lane >= o) w += y;
            }
            warp_sums[lane] = w;
        }
        __syncthreads();
        const int32_t first = carry + x - s + (wid > 0 ? warp_sums[wid - 1] : 0);
        const int4 o4 = make_int4(first, first + c.x, first + c.x + c.y, first + c.x + c.y + c.z);
        if (q + 3 < n) {
            *reinterpret_cast<int4*>(a.ws.tile_off + q) = o4;
        } else {
            if (q < n) a.ws.tile_off[q] = o4.x;
            if (q + 1 < n) a.ws.tile_off[q + 1] = o4.y;
            if (q + 2 < n) a.ws.tile_off[q + 2] = o4.z;
        }
        carry += warp_sums[31];
        __syncthreads();  // warp_sums is rewritten by the next round
    }
}

__global__ void __launch_bounds__(256) k_scatter(Args a) {
    const int nv = a.hdr->nviews;
    const int64_t total = a.hdr->total_records;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += (int64_t)gridDim.x * blockDim.x) {
        const int4 tb = a.ws.tbox[t];
        if (tb.x > tb.y) continue;
        const int v = view_of_record(a.views, nv, t);
        if (__ldg(&a.views[v].plain)) continue;
        const int g = (int)(t - __ldg(&a.views[v].rec_base));
        const int tiles_x = __ldg(&a.views[v].tiles_x), tile_base = __ldg(&a.views[v].tile_base);
        const int sub = g & (kTileSub - 1);
        for (int ty = tb.z; ty <= tb.w; ++ty)
            for (int tx = tb.x; tx <= tb.y; ++tx) {
                const int tile = (int)VOGE_IDX(a.hdr, tile_base + ty * tiles_x + tx, a.hdr->total_tiles, kChkTile);
                const int pos = __ldg(a.ws.tile_off + tile) + atomicAdd(&a.ws.tile_sub[tile * kTileSub + sub], 1);
                if (pos < a.ws.bin_cap) a.ws.tile_gauss[VOGE_IDX(a.hdr, pos, a.ws.bin_cap, kChkBin)] = g;
            }
    }
}

// Depth order of each tile's candidate list (ascending lower bound of l), so
// that a pixel can stop once no later candidate can enter its list.  Lists of
// at most kSortMax entries are sorted (one CTA per list, below); longer lists
// stay unsorted and are traced in full.
__device__ __forceinline__ bool tile_sorted(int use_thresh, int plain, int cnt, int64_t off, int64_t cap) {
    return use_thresh && !plain && cnt > 1 && cnt <= kSortMax && off + cnt <= cap;
}

// One block sorts one tile list at a time.  Each entry is one 32-bit word,
// (order-preserving bits of lmin, whose low kSortPosBits bits k_project
// cleared) | (the entry's position in the unsorted list), so one compare
// orders by (lmin, position) and the sorted words give back the Gaussians
// through a table of the unsorted list.  The list is padded with all-ones
// words to a power of two n and sorted by the bitonic network with the words
// in registers: thread t holds words [tE, tE + E) (E = n / 256, at least 1).
// Exchanges at distance j < E stay inside a thread, E <= j < 32E go through
// warp shuffles and only j >= 32E through shared memory, with a block barrier
// on each side.
constexpr int kSortThreads = 256;

// Keeps the smaller (take_min) or the larger of (mine, other).
__device__ __forceinline__ uint32_t keep(uint32_t mine, uint32_t other, bool take_min) {
    return take_min ? min(mine, other) : max(mine, other);
}

template <int E>
__device__ __forceinline__ void sort_tile_block(const Args& a, uint32_t* sw, int32_t* sg, int cnt, int off, int n2,
                                                int64_t vb, int vd_N) {
    const int tid = threadIdx.x;
    const int nthr = n2 / E;  // threads holding entries (a multiple of 32 or all of n2 < 32)
    const bool act = tid < nthr;
    uint32_t w[E];
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int x = tid * E + r;
        w[r] = ~0u;
        if (act && x < cnt) {
            const int32_t g = (int32_t)VOGE_IDX(a.hdr, a.ws.tile_gauss[VOGE_IDX(a.hdr, off + x, a.ws.bin_cap, kChkTileList)],
                                                vd_N, kChkRecord);
            sg[x] = g;
            w[r] = (float_order(__ldg(&a.ws.rec[4 * (vb + g) + 3].w)) & ~((1u << kSortPosBits) - 1u)) | (uint32_t)x;
        }
    }
    for (int k = 2; k <= n2; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j < E) {
#pragma unroll
                for (int b = 1; b < E; b <<= 1) {
                    if (j == b) {
#pragma unroll
                        for (int r = 0; r < E; ++r) {
                            if (r & b) continue;
                            const bool up = ((tid * E + r) & k) == 0;
                            const uint32_t lo = w[r], hi = w[r | b];
                            w[r] = up ? min(lo, hi) : max(lo, hi);
                            w[r | b] = up ? max(lo, hi) : min(lo, hi);
                        }
                    }
                }
            } else if (j < 32 * E && nthr >= 32) {
                const int lm = j / E;  // partner lane distance
#pragma unroll
                for (int r = 0; r < E; ++r) {
                    const uint32_t o = __shfl_xor_sync(0xffffffffu, w[r], lm);
                    const int x = tid * E + r;
                    w[r] = keep(w[r], o, ((x & j) == 0) == ((x & k) == 0));
                }
            } else {
                // partner in another warp (or lists shorter than a warp)
                if (act)
#pragma unroll
                    for (int r = 0; r < E; ++r) sw[tid * E + r] = w[r];
                __syncthreads();
                if (act)
#pragma unroll
                    for (int r = 0; r < E; ++r) {
                        const int x = tid * E + r;
                        w[r] = keep(w[r], sw[x ^ j], ((x & j) == 0) == ((x & k) == 0));
                    }
                __syncthreads();
            }
        }
    }
    __syncthreads();  // sg complete (written above by every thread)
#pragma unroll
    for (int r = 0; r < E; ++r) {
        const int x = tid * E + r;
        if (act && x < cnt) a.ws.tile_gauss[off + x] = sg[w[r] & ((1u << kSortPosBits) - 1u)];
    }
}

__global__ void __launch_bounds__(kSortThreads) k_sort_tiles(Args a) {
    __shared__ uint32_t sw[kSortMax];
    __shared__ int32_t sg[kSortMax];
    const int nv = a.hdr->nviews, total = a.hdr->total_tiles;
    for (int t = blockIdx.x; t < total; t += gridDim.x) {
        const int cnt = a.ws.tile_cnt[t];
        const int off = a.ws.tile_off[t];
        const ViewDesc& vd = a.views[view_of_tile(a.views, nv, t)];
        if (!tile_sorted(vd.use_thresh, vd.plain, cnt, off, a.ws.bin_cap)) continue;  // uniform in the block
        int n2 = 2;
        while (n2 < cnt) n2 <<= 1;
        const int64_t vb = vd.rec_base;
        if (n2 <= 256) sort_tile_block<1>(a, sw, sg, cnt, off, n2, vb, vd.N);
        else if (n2 == 512) sort_tile_block<2>(a, sw, sg, cnt, off, n2, vb, vd.N);
        else if (n2 == 1024) sort_tile_block<4>(a, sw, sg, cnt, off, n2, vb, vd.N);
        else sort_tile_block<8>(a, sw, sg, cnt, off, n2, vb, vd.N);
        __syncthreads();  // the next tile reuses sw and sg
    }
}

// Projection of every (view, Gaussian) record, then (with count_tiles) the
// tile scan and scatter.  Grid-stride kernels: `grid` blocks of 256 threads
// cover any number of records read from the batch header.
cudaError_t launch_project(int grid, int tiles, int count_tiles, cudaStream_t s, const Args& a) {
    {
        TraceScope tr("k_project", s);
        k_project<<<grid, 256, 0, s>>>(a, count_tiles);
        cudaError_t e = cudaPeekAtLastError();
        if (e != cudaSuccess) return e;
    }
    if (count_tiles) {
        {
            TraceScope tr("k_scan_tiles", s);
            k_tile_totals<<<tiles < 1 ? 1 : (tiles + 255) / 256, 256, 0, s>>>(a);
            k_scan_tiles<<<1, 1024, 0, s>>>(a);
        }
        {
            TraceScope tr("k_scatter", s);
            k_scatter<<<grid, 256, 0, s>>>(a);
        }
        {
            // one block per tile (grid-stride beyond 8 blocks per SM)
            TraceScope tr("k_sort_tiles", s);
            const int sgrid = tiles < 1 ? 1 : (tiles < 152 * 8 ? tiles : 152 * 8);
            k_sort_tiles<<<sgrid, kSortThreads, 0, s>>>(a);
        }
        return cudaPeekAtLastError();
    }
    return cudaSuccess;
}

}  // namespace voge
