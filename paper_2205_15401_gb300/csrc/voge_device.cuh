// voge_device.cuh -- device-side types and helpers of libvoge (sm_103a).
//
// Geometry of one Gaussian seen from one view (Eq. 6 of the paper, rewritten
// around the ray through the Gaussian's centre so that FP32 keeps the
// precision the FP64 reference has):
//
//   M = (Mx, My, Mz) camera-space mean, P camera-space inverse covariance,
//   Mh = M / Mz = (xh, yh, 1) its centre ray, D = Mh + D' with
//   D' = (du/F, dv/F, 0), (du, dv) = pixel-centre offset from the projected
//   centre (uc, vc) = (F xh + Ox, F yh + Oy).
//
//   b   = DᵀPD               = beta0 + 2 lin + quad
//   lin = Mhᵀ P D'            = beta1 du + beta2 dv
//   quad= D'ᵀ P D'            = g00 du^2 + 2 g01 du dv + g11 dv^2
//   l   = MᵀPD / b            = Mz - Mz (quad + lin) / b        (peak depth)
//   qt  = (M - lD)ᵀP(M - lD)  = Mz^2 (M x D')ᵀ adj(P) (M x D') / (Mz^2 b)
//                             = (q00 du^2 + 2 q01 du dv + q11 dv^2) / b
//   a   = e^{q} = exp(-qt/2), sigma^2 = 1/b.
//
// The qt form is the Lagrange identity (MᵀPM)(DᵀPD) - (MᵀPD)^2 =
// (M x D)ᵀ adj(P) (M x D): it has no cancellation, unlike MᵀPM - (MᵀPD)^2/b.
// The depth l is kept as two floats (Mz_hi, Mz_lo + dl) so that l_k - l_j in
// the erf argument of Eq. 7 is exact to FP32 rounding of the difference.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace voge {

constexpr int kTileW = 16;     // tile width in pixels (one warp covers 16 x 2 pixels)
constexpr int kSortMax = 2048; // tiles with more candidates are processed unsorted
constexpr int kTileSub = 8;    // counters per tile for binning (spreads same-address atomics)
constexpr int kSortPosBits = 11;  // list positions of a sorted tile (kSortMax = 2^11)
static_assert(kSortMax == 1 << kSortPosBits, "sort words hold a list position in their low bits");

// Order-preserving map between floats and unsigned integers: a < b exactly
// when float_order(a) < float_order(b) (for non-NaN a, b).
__device__ __forceinline__ uint32_t float_order(float x) {
    const uint32_t b = __float_as_uint(x);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}
__device__ __forceinline__ float order_float(uint32_t o) {
    return __uint_as_float((o & 0x80000000u) ? (o & 0x7fffffffu) : ~o);
}
constexpr float kLog2e = 1.4426950408889634f;

// One view as the kernels read it: the camera, the scene this view renders
// (its own Gaussians, attribute width, list length) and where its outputs go.
// A render call fills one per view, all pointing at the same scene; a serving
// tick fills one per admitted request, each with its own scene, so that one
// launch covers every request.
struct ViewDesc {
    float R[9];
    float T[3];
    float F, Ox, Oy, invF;
    int32_t H, W, tiles_x, tiles_y;
    int32_t tile_base;  // first global tile id of this view
    int32_t tile_h;     // tile height in pixels
    int32_t N, C;       // Gaussians and attribute channels of this view's scene
    int32_t L;          // list length (<= the register capacity of the launch)
    int32_t use_thresh, plain, pad0;
    float tau, Qeta;    // Qeta = 2 ln(1/eta) or +inf
    float pad1, pad2;
    int64_t rec_base;   // record of (this view, Gaussian g) is rec_base + g
    int64_t elem_base;  // first image element of this view in the batch (for per-element kernels)
    int64_t pix_base;   // first pixel of this view in the batch (generic-path scratch)
    int64_t pad3;
    const float* means;
    const float* inv_cov;
    const float* attr;
    float* image;       // this view's first pixel: [H*W][C]
    float* weights;     // [H*W][L] or null
    int32_t* index;     // [H*W][L]
    const int32_t* index_in;
    const float* grad_image;  // [H*W][C]
    const float* target;      // [H*W][C] (loss helper)
    float* loss;              // one float (loss helper)
    float* grad_means;        // [N][3] or null
    float* grad_inv_cov;      // [N][6] or null
    float* grad_attr;         // [N][C] or null
    float* grad_cam;          // [12] or null
    const float* weights_in;  // [H*W][L] W_k of the forward pass, or null (backward recomputes them)
    const void* pad4;
};
static_assert(sizeof(ViewDesc) % 16 == 0, "ViewDesc layout");

// Per-call (or per-tick) totals and work counters, in device memory next to
// the view table.  The counters start at zero on every upload.
constexpr int kMaxClasses = 8;
struct BatchHdr {
    int64_t total_records;  // sum over views of N
    int64_t total_elems;    // sum over views of H*W*C
    int32_t total_tiles;
    int32_t nviews;
    int32_t class_begin[kMaxClasses];  // tile ranges of the list-capacity classes
    int32_t class_end[kMaxClasses];
    int32_t counters[4 * kMaxClasses]; // persistent-launch work counters (forward, backward, wide backward,
                                       // standalone fine pass)
    int32_t shared_scene;   // 1: every view renders the same Gaussians (records rec_base = v * N)
    int32_t pad[1];
    // what the forward pass of this call did (voge_render_stats): Gaussian-ray
    // traces of the coarse pass (Eq. 6 evaluations), kept entries, and the
    // fine pass's (k, j) pairs (sum over pixels of n_p^2)
    unsigned long long traces, entries, pairs;
    int32_t check_site;     // checked builds: the first index check that failed (0: none)
    int32_t pad3;
};
static_assert(sizeof(BatchHdr) % 16 == 0, "BatchHdr layout");

// A record of the row pairs (units: rows 2q, 2q + 1 of a 16 x 8 backward
// tile, one warp of a tile launch) whose index lists keep an entry, in device
// memory just after the view table: written by the forward pass as it
// selects, or by k_live_units from given lists.  Every upload clears it and
// names the lists it will describe (null: none); a backward that reuses the
// forward's projection uploads only the header and view table, so it finds
// the forward's record, and uses it when it reads those same lists.
struct LiveHdr {
    int32_t n[kMaxClasses];      // units in the list, per class
    const int32_t* index_fwd;    // the lists they describe (view 0's first word)
    int64_t pad;
};
static_assert(sizeof(LiveHdr) % 16 == 0, "LiveHdr layout");

// ------------------------------------------------------------------------
// Checked builds (-DVOGE_CHECKED, build.py's checked library): every gather
// and scatter index of the tile kernels goes through VOGE_IDX.  An index
// outside [0, n) records its site in *site (the first one wins) and is
// replaced by 0, a valid element, so the kernel reads or writes in bounds,
// finishes, and the C ABI reports VOGE_ERR_CHECK.  Normal builds compile the
// checks away.
// ------------------------------------------------------------------------
enum : int32_t {
    kChkTileList = 1,  // candidate list of a tile (tile_gauss)
    kChkRecord = 2,    // Gaussian index into records, attributes, gradients
    kChkTile = 3,      // tile index (counts, offsets, boxes)
    kChkListRead = 4,  // a pixel's index / weight list read back
    kChkOutput = 5,    // image, weight or index output element
    kChkScratch = 6,   // per-pixel scratch of the generic path
    kChkBin = 7        // binning cursor
};

__host__ __device__ __forceinline__ bool in_bounds(int64_t i, int64_t n) { return (uint64_t)i < (uint64_t)n; }

// i if 0 <= i < n, else 0 with the site recorded (first failure kept).
__host__ __device__ __forceinline__ int64_t checked_index(int32_t* site, int64_t i, int64_t n, int32_t where) {
    if (in_bounds(i, n)) return i;
#ifdef __CUDA_ARCH__
    atomicCAS(site, 0, where);
#else
    if (*site == 0) *site = where;
#endif
    return 0;
}

#ifdef VOGE_CHECKED
#define VOGE_IDX(hdr, i, n, where) ::voge::checked_index(&(hdr)->check_site, (int64_t)(i), (int64_t)(n), (where))
#else
#define VOGE_IDX(hdr, i, n, where) (i)
#endif

// Projected record of one (view, Gaussian): 4 x float4 = 64 bytes.
//   r0 = (uc_hi, uc_lo, vc_hi, vc_lo)   centre, pixel units (u = column + 0.5)
//   r1 = (beta0, beta1, beta2, g00)
//   r2 = (2 g01, g11, q00, 2 q01)
//   r3 = (q11, Mz_hi, Mz_lo, lmin)      lmin: lower bound of l over the pixels
//                                       where the Gaussian is a candidate
// An invalid Gaussian (behind the camera, non-finite) has r1 = r2 = 0 so that
// b = 0 and it never passes the b > 0 test.
// Second record (backward only): 2 x float4 = (Pxx, Pxy, Pxz, Pyy), (Pyz, Pzz, xh, yh).

// ------------------------------------------------------------------------
// Hardware approximations (PTX ISA: ex2.approx, rcp.approx).
// ------------------------------------------------------------------------
__device__ __forceinline__ float ex2_approx(float x) {
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rcp_approx(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// erfc(x) for x >= 0 by Abramowitz & Stegun (1964), eq. 7.1.28:
//   erf(x) = 1 - (1 + a1 x + a2 x^2 + ... + a6 x^6)^-16,  |error| <= 3e-7.
// Returns the (...)^-16 term.  For large x the power overflows to +inf and
// the reciprocal is 0, i.e. erf = 1.
__device__ __forceinline__ float erfc_as28(float x) {
    float p = fmaf(4.30638e-5f, x, 2.765672e-4f);
    p = fmaf(p, x, 1.520143e-4f);
    p = fmaf(p, x, 9.2705272e-3f);
    p = fmaf(p, x, 4.22820123e-2f);
    p = fmaf(p, x, 7.05230784e-2f);
    p = fmaf(p, x, 1.0f);
    p = p * p;
    p = p * p;
    p = p * p;
    p = p * p;
    return rcp_approx(p);
}

// erfc(x) for x >= 0 by Abramowitz & Stegun (1964), eq. 7.1.26:
//   erf(x) = 1 - t (a1 + t (a2 + t (a3 + t (a4 + t a5)))) e^{-x^2},
//   t = 1 / (1 + p x),  |error| <= 1.5e-7.
// Also returns g = e^{-x^2}, which the backward pass needs for d erf/dx.
__device__ __forceinline__ float erfc_as26(float x, float& g) {
    float t = rcp_approx(fmaf(0.3275911f, x, 1.0f));
    float s = fmaf(t, 1.061405429f, -1.453152027f);
    s = fmaf(s, t, 1.421413741f);
    s = fmaf(s, t, -0.284496736f);
    s = fmaf(s, t, 0.254829592f);
    s = s * t;
    g = ex2_approx(x * (x * -kLog2e));
    return s * g;
}

// ------------------------------------------------------------------------
// Double-float (unevaluated sum of two floats) helpers for the camera
// transform and the projected centre.
// ------------------------------------------------------------------------
struct dfl {
    float hi, lo;
};
__device__ __forceinline__ dfl two_prod(float a, float b) {
    float p = a * b;
    return {p, fmaf(a, b, -p)};
}
__device__ __forceinline__ dfl two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    float bb = __fsub_rn(s, a);
    float e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return {s, e};
}
__device__ __forceinline__ dfl fast_two_sum(float a, float b) {
    float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ dfl df_add(dfl x, dfl y) {
    dfl s = two_sum(x.hi, y.hi);
    float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}
__device__ __forceinline__ dfl df_mul_f(dfl x, float y) {
    dfl p = two_prod(x.hi, y);
    float e = fmaf(x.lo, y, p.lo);
    return fast_two_sum(p.hi, e);
}
__device__ __forceinline__ dfl df_div(dfl x, dfl y) {
    float q1 = __fdiv_rn(x.hi, y.hi);
    dfl p = two_prod(q1, y.hi);
    float r = __fsub_rn(__fadd_rn(__fsub_rn(__fsub_rn(x.hi, p.hi), p.lo), x.lo), __fmul_rn(q1, y.lo));
    float q2 = __fdiv_rn(r, y.hi);
    return fast_two_sum(q1, q2);
}
// exact-ish a.x + b.y + c.z + d with a, x... floats
__device__ __forceinline__ dfl df_dot3_add(float a0, float x0, float a1, float x1, float a2, float x2, float d) {
    dfl s = two_prod(a0, x0);
    s = df_add(s, two_prod(a1, x1));
    s = df_add(s, two_prod(a2, x2));
    return df_add(s, dfl{d, 0.0f});
}

// ------------------------------------------------------------------------
// Per-pixel trace of one Gaussian from its record (Eq. 6).
// ------------------------------------------------------------------------
struct Trace {
    float du, dv, b, num, qb;
};

__device__ __forceinline__ Trace trace_px(const float4& r0, const float4& r1, const float4& r2, const float4& r3,
                                          float px, float py) {
    Trace t;
    t.du = __fsub_rn(__fsub_rn(px, r0.x), r0.y);
    t.dv = __fsub_rn(__fsub_rn(py, r0.z), r0.w);
    float dv2 = t.dv * t.dv;
    float lin = fmaf(r1.y, t.du, r1.z * t.dv);
    float quad = fmaf(t.du, fmaf(r1.w, t.du, r2.x * t.dv), r2.y * dv2);
    t.num = quad + lin;
    t.b = (r1.x + lin) + t.num;
    t.qb = fmaf(t.du, fmaf(r2.z, t.du, r2.w * t.dv), r3.x * dv2);
    return t;
}

// Candidate test of App. A.3 (e^{q} > eta, i.e. qt < Qeta = 2 ln(1/eta)) plus
// b > 0 and l > 0; returns the sort key l (> 0) or 0 when rejected.
__device__ __forceinline__ float candidate_key(const float4& r0, const float4& r1, const float4& r2, const float4& r3,
                                               float px, float py, float Qeta) {
    Trace t = trace_px(r0, r1, r2, r3, px, py);
    if (!(t.b > 0.0f) || !(t.qb < Qeta * t.b)) return 0.0f;
    float dl = -r3.y * t.num * rcp_approx(t.b);
    float l = r3.y + (r3.z + dl);
    return l > 0.0f ? l : 0.0f;
}

// Fine-pass values of a kept Gaussian: l = hi + lo, r = sqrt(b/2) = 1/(sqrt2 sigma), a = e^{q}.
struct Entry {
    float hi, lo, r, a;
};
__device__ __forceinline__ Entry entry_px(const float4& r0, const float4& r1, const float4& r2, const float4& r3,
                                          float px, float py) {
    Trace t = trace_px(r0, r1, r2, r3, px, py);
    float ib = rcp_approx(t.b);
    Entry e;
    e.hi = r3.y;
    e.lo = r3.z - r3.y * t.num * ib;
    e.r = sqrtf(0.5f * t.b);
    e.a = ex2_approx(-0.5f * kLog2e * t.qb * ib);
    return e;
}

__device__ __forceinline__ void load_rec(const float4* __restrict__ rec, int64_t o, float4& r0, float4& r1,
                                         float4& r2, float4& r3) {
    r0 = __ldg(rec + 4 * o + 0);
    r1 = __ldg(rec + 4 * o + 1);
    r2 = __ldg(rec + 4 * o + 2);
    r3 = __ldg(rec + 4 * o + 3);
}

// Sorted insertion into a register list of KM (key, id) pairs, ascending by
// (key, id).  The caller has checked that (l, g) beats the last entry.  All
// comparisons are made against the old list first (the flags are monotone in
// s because the list is sorted), then every slot is updated independently, so
// the insertion has no serial dependency chain through the list.
template <int KM>
__device__ __forceinline__ void topk_insert(float (&key)[KM], int32_t (&id)[KM], float l, int32_t g) {
    bool lt[KM];
#pragma unroll
    for (int s = 0; s < KM; ++s) lt[s] = (l < key[s]) || (l == key[s] && g < id[s]);
#pragma unroll
    for (int s = KM - 1; s >= 1; --s) {
        key[s] = lt[s] ? (lt[s - 1] ? key[s - 1] : l) : key[s];
        id[s] = lt[s] ? (lt[s - 1] ? id[s - 1] : g) : id[s];
    }
    key[0] = lt[0] ? l : key[0];
    id[0] = lt[0] ? g : id[0];
}

// Pixels of each tile row in which the candidate test can pass.  Per row
// the test qb < Qeta b is the quadratic inequality
//   h00 du^2 + 2 (h01 dv + hx) du + (h11 dv^2 + 2 hy dv + h22) < 0,
// an interval of du whenever h00 > 0.  The interval is widened by 1 pixel
// plus 2% of its half-width, so it never excludes a pixel that the exact
// per-pixel test keeps (this margin also covers the approximate square root
// and reciprocal used here); rows with h00 <= 0 (or no threshold) are left
// whole.  Output: one 16-bit mask per row, bit c set for tile column c.
constexpr uint16_t kRowEmpty = 0x0000u;
constexpr uint16_t kRowFull = 0xffffu;

__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

template <int TH>
__device__ __forceinline__ void row_masks(const float4& r0, const float4& r1, const float4& r2, const float4& r3,
                                          float Q, int tx, int ty, uint16_t* out, int stride) {
    const float h00 = fmaf(-Q, r1.w, r2.z);
    if (!(h00 > 0.0f) || !(Q < INFINITY)) {
#pragma unroll
        for (int rr = 0; rr < TH; ++rr) out[rr * stride] = kRowFull;
        return;
    }
    const float h01 = 0.5f * fmaf(-Q, r2.x, r2.w);
    const float h11 = fmaf(-Q, r2.y, r3.x);
    const float hx = -Q * r1.y, hy2 = -2.0f * Q * r1.z, h22 = -Q * r1.x;
    const float ih = rcp_approx(h00);
    const float uoff = r0.x - ((float)(tx * kTileW) + 0.5f);  // centre relative to tile column 0
    const float row0 = (float)(ty * TH) + 0.5f;
#pragma unroll
    for (int rr = 0; rr < TH; ++rr) {
        const float dv = ((row0 + (float)rr) - r0.z) - r0.w;
        const float Bp = fmaf(h01, dv, hx);
        const float Cp = fmaf(fmaf(h11, dv, hy2), dv, h22);
        const float disc = fmaf(Bp, Bp, -h00 * Cp);
        const float scale = fmaf(Bp, Bp, fabsf(h00 * Cp));
        const float w = sqrt_approx(fmaxf(disc, 0.0f)) * ih;
        const float c = uoff - Bp * ih;
        const float m = fmaf(0.02f, w, 1.0f);
        const int lo = (int)fminf(fmaxf(ceilf(c - w - m), 0.0f), 16.0f);
        const int hi = (int)fmaxf(fminf(floorf(c + w + m), 15.0f), -1.0f);
        const uint32_t bits = (0xffffu >> (15 - max(hi, 0))) & (0xffffu << lo);
        out[rr * stride] = (disc > -1e-3f * scale && lo <= hi) ? (uint16_t)bits : kRowEmpty;
    }
}

// Camera-space gradient of one (pixel, kept Gaussian) pair: out[0..2] = dM,
// out[3..8] = G (xx, xy, xz, yy, yz, zz) with entries of P treated as independent.
// s0, s1: the pair's second record (camera-space P and centre ray).
__device__ __forceinline__ void chain_to_camera(const float4& s0, const float4& s1, const Trace& t, const float4& r3,
                                                float invF, float dqt, float dl, float db, float out[9]) {
    const float ib = rcp_approx(t.b);
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

// Camera-space gradient sums per record: 12 floats = three 16-byte groups
// (dM0 dM1 dM2 G0 | G1 G2 G3 G4 | G5 0 0 0), G = (xx, xy, xz, yy, yz, zz).
constexpr int kGcamStride = 12;

// Vector reduction into global memory (PTX red.global.add.v4.f32, sm_90+):
// one operation adds four consecutive floats; the address is 16-byte aligned.
__device__ __forceinline__ void red_add_v4(float* addr, float a, float b, float c, float d) {
    asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c), "f"(d)
                 : "memory");
}

// Asynchronous global -> shared copies (PTX cp.async, sm_80+): 16 bytes
// through L2 only, or 4 bytes through L1; a thread waits for its own groups.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async4(void* sdst, const void* gsrc) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(sdst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(d), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }

// View of a global tile / record / image element (binary searches over the
// view table's monotone bases).
__device__ __forceinline__ int view_of_tile(const ViewDesc* __restrict__ vd, int nv, int tile) {
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&vd[mid].tile_base) <= tile) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int view_of_record(const ViewDesc* __restrict__ vd, int nv, int64_t r) {
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&vd[mid].rec_base) <= r) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}
__device__ __forceinline__ int view_of_elem(const ViewDesc* __restrict__ vd, int nv, int64_t e) {
    int lo = 0, hi = nv - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (__ldg(&vd[mid].elem_base) <= e) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

// Workspace arrays shared by the launches of one call / tick.
struct Ws {
    float4* rec;      // [records][4]
    float4* rec2;     // [records][2]
    int4* tbox;       // [records]: tile range tx0, tx1, ty0, ty1 (tx0 > tx1: none)
    int32_t* tile_cnt;  // [tiles] candidates per tile (written by the scan)
    int32_t* tile_off;  // [tiles] first list entry of each tile
    int32_t* tile_sub;  // [tiles][kTileSub] counts per sub-counter, then scatter cursors
    int32_t* tile_gauss;
    int64_t bin_cap;
    float* gcam;      // [records][12] backward accumulators: dM (3), G (6), narrow attribute gradient (3)
    float* gkey;      // generic-path per-pixel scratch
    int32_t* gid;
    int2* live;       // (unit, view) of each row pair with a kept entry (class c from (TH/2) class_begin[c])
    LiveHdr* live_hdr;  // their count (null: not recorded)
    int32_t gen_L;    // list length the generic scratch is laid out for
};

struct Args {
    const ViewDesc* views;
    BatchHdr* hdr;
    Ws ws;
    int32_t cls;      // list-capacity class of a tile launch (index into class_begin/end)
    int32_t wk_smem;  // backward launches: the W_k buffer follows the stream in shared memory
};

// Next tile of a persistent tile launch (dynamic: CTAs take tiles as they
// free up).  Returns a global tile id or -1 when the class range is done.
__device__ __forceinline__ int next_tile(const Args& a, int fwd, int* s_slot) {
    if (threadIdx.x == 0) *s_slot = atomicAdd(&a.hdr->counters[a.cls + (fwd ? 0 : kMaxClasses)], 1);
    __syncthreads();
    const int t = a.hdr->class_begin[a.cls] + *s_slot;
    __syncthreads();
    return t < a.hdr->class_end[a.cls] ? t : -1;
}

}  // namespace voge
