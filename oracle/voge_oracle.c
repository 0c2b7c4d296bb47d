/*
 * voge_oracle.c -- plain, slow, FP64 CPU reference of the VoGE renderer
 * (Wang et al., "VoGE: A Differentiable Volume Renderer using Gaussian
 * Ellipsoids for Analysis-by-Synthesis", ICLR 2023).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker for the CUDA path, not
 * part of it: only tests/, __graft_entry__.smoke() and bench.py's CPU
 * baseline leg may build, load or call it.  It shares no code, header, table
 * or helper with the CUDA library, and the CUDA library never calls it.
 *
 * Every step follows the paper's definitions directly, in double precision,
 * with no blocking, fusion or reordering:
 *   - viewing transform, Sec. 3.3 (M = R M_o + T; the inverse covariance is
 *     carried to camera space as P_cam = R P Rᵀ, the column-vector reading);
 *   - perspective rays, Eq. 5 (pixel centres, x = column, y = row, D_z = 1);
 *   - ray tracing of one ellipsoid, Eq. 6 and App. A.1 (l, q, sigma);
 *   - selection, Sec. 3.3 and App. A.3 (keep e^{q} > eta, sort by l, keep
 *     the K' nearest; ties broken by Gaussian index);
 *   - closed-form transmittance, Eq. 7 (sum over the pixel's kept list);
 *   - weights and blend, Eq. 8 (W_k = T(l_k) e^{q_k}, C = sum W_k c_k);
 *   - backward: the chain rule of the steps above with the lists frozen;
 *   - the exact outer integral of Eq. 1 by adaptive quadrature (to bound the
 *     approximation of Eq. 8; App. A.2, Fig. 6);
 *   - the neural sampler, Sec. 3.4 Eq. 10: alpha_k = sum_p W_pk phi_p /
 *     sum_p W_pk over the pixels whose kept list holds k (W_pk = 0
 *     elsewhere); a kernel no pixel keeps gets alpha_k = 0.
 * Notation: a = e^{q} is the peak density on the ray, qt = -2q >= 0,
 * b = DᵀPD = 1/sigma^2, m = a/2 so that tau*sum m(1+erf) is Eq. 7's exponent.
 *
 * Pins: tests/test_oracle_*.py check this file against closed forms,
 * invariants, the paper's printed 0.0256 and finite differences.
 */
#define _GNU_SOURCE
#include <complex.h>
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

typedef struct {
    double R[9];   /* row-major rotation, M_cam = R M + T */
    double T[3];
    double F, Ox, Oy;
    int H, W;
} vo_camera;

typedef struct {
    int B, N, C, K;   /* K <= 0 or K >= N: keep every candidate */
    double tau, eta;  /* eta <= 0: no threshold */
} vo_params;

static int list_cap(const vo_params* p) {
    return (p->K <= 0 || p->K >= p->N) ? p->N : p->K;
}

/* ---------------------------------------------------------------------- */
/* Camera pose (azimuth, elevation, distance, roll) -> R, T.               */
/* Look-at construction: camera centre on a sphere of radius dist, looking */
/* at the origin, world up +y, camera axes x right, y down, z forward,    */
/* then a roll about the optical axis.  Written for complex arguments so   */
/* that its derivative can be taken by the complex step.                   */
/* ---------------------------------------------------------------------- */
static void pose_to_RT_c(const double complex pose[4], double complex R[9], double complex T[3]) {
    double complex a = pose[0], e = pose[1], dist = pose[2], roll = pose[3];
    double complex C[3] = {dist * ccos(e) * csin(a), dist * csin(e), dist * ccos(e) * ccos(a)};
    double complex n = csqrt(C[0] * C[0] + C[1] * C[1] + C[2] * C[2]);
    double complex f[3] = {-C[0] / n, -C[1] / n, -C[2] / n};
    const double up[3] = {0.0, 1.0, 0.0};
    double complex r[3] = {f[1] * up[2] - f[2] * up[1], f[2] * up[0] - f[0] * up[2], f[0] * up[1] - f[1] * up[0]};
    double complex rn = csqrt(r[0] * r[0] + r[1] * r[1] + r[2] * r[2]);
    for (int i = 0; i < 3; i++) r[i] /= rn;
    double complex d[3] = {f[1] * r[2] - f[2] * r[1], f[2] * r[0] - f[0] * r[2], f[0] * r[1] - f[1] * r[0]};
    double complex R0[9] = {r[0], r[1], r[2], d[0], d[1], d[2], f[0], f[1], f[2]};
    double complex c = ccos(roll), s = csin(roll);
    double complex Rz[9] = {c, -s, 0, s, c, 0, 0, 0, 1};
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double complex acc = 0;
            for (int k = 0; k < 3; k++) acc += Rz[3 * i + k] * R0[3 * k + j];
            R[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; i++) T[i] = -(R[3 * i] * C[0] + R[3 * i + 1] * C[1] + R[3 * i + 2] * C[2]);
}

void vo_pose_to_RT(const double pose[4], double R[9], double T[3]) {
    double complex pc[4] = {pose[0], pose[1], pose[2], pose[3]};
    double complex Rc[9], Tc[3];
    pose_to_RT_c(pc, Rc, Tc);
    for (int i = 0; i < 9; i++) R[i] = creal(Rc[i]);
    for (int i = 0; i < 3; i++) T[i] = creal(Tc[i]);
}

/* dL/dpose from dL/dR (9, row-major) and dL/dT (3): dRT = [dR | dT].
 * Derivative of the look-at by the complex step (exact to rounding). */
void vo_pose_grad(const double pose[4], const double dRT[12], double dpose[4]) {
    const double h = 1e-30;
    for (int q = 0; q < 4; q++) {
        double complex pc[4] = {pose[0], pose[1], pose[2], pose[3]};
        pc[q] += I * h;
        double complex Rc[9], Tc[3];
        pose_to_RT_c(pc, Rc, Tc);
        double g = 0.0;
        for (int i = 0; i < 9; i++) g += dRT[i] * cimag(Rc[i]) / h;
        for (int i = 0; i < 3; i++) g += dRT[9 + i] * cimag(Tc[i]) / h;
        dpose[q] = g;
    }
}

/* ---------------------------------------------------------------------- */
/* Viewing transform (Sec. 3.3) and rays (Eq. 5).                          */
/* ---------------------------------------------------------------------- */
static void sym_from6(const double* p6, double P[9]) {
    /* parameter order xx, xy, xz, yy, yz, zz */
    P[0] = p6[0]; P[1] = p6[1]; P[2] = p6[2];
    P[3] = p6[1]; P[4] = p6[3]; P[5] = p6[4];
    P[6] = p6[2]; P[7] = p6[4]; P[8] = p6[5];
}

static void to_camera(const vo_camera* c, const double* Mw, const double* Pw6, double M[3], double P[9]) {
    double Pw[9], RP[9];
    sym_from6(Pw6, Pw);
    for (int i = 0; i < 3; i++) M[i] = c->R[3 * i] * Mw[0] + c->R[3 * i + 1] * Mw[1] + c->R[3 * i + 2] * Mw[2] + c->T[i];
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += c->R[3 * i + k] * Pw[3 * k + j];
            RP[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double acc = 0;
            for (int k = 0; k < 3; k++) acc += RP[3 * i + k] * c->R[3 * j + k];
            P[3 * i + j] = acc;
        }
}

static void ray_dir(const vo_camera* c, int i, int j, double D[3]) {
    D[0] = ((double)j + 0.5 - c->Ox) / c->F;
    D[1] = ((double)i + 0.5 - c->Oy) / c->F;
    D[2] = 1.0;
}

static double quad3(const double* x, const double P[9], const double* y) {
    double s = 0;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) s += x[a] * P[3 * a + b] * y[b];
    return s;
}

/* Ray tracing of one ellipsoid along r(t) = tD (Eq. 6, App. A.1):
 *   b = DᵀPD,  l = (MᵀPD + DᵀPM) / (2b),  V = M - lD,  qt = VᵀPV = -2q. */
static void trace(const double M[3], const double P[9], const double D[3], double* l, double* qt, double* b) {
    double bb = quad3(D, P, D);
    double ll = (quad3(M, P, D) + quad3(D, P, M)) / (2.0 * bb);
    double V[3] = {M[0] - ll * D[0], M[1] - ll * D[1], M[2] - ll * D[2]};
    *b = bb;
    *l = ll;
    *qt = quad3(V, P, V);
}

/* exposed for the closed-form pins */
void vo_trace_dir(const double M[3], const double P6[6], const double D[3], double out[3]) {
    double P[9];
    sym_from6(P6, P);
    trace(M, P, D, &out[0], &out[1], &out[2]);
}

/* ---------------------------------------------------------------------- */
/* Per-view camera-space copies of the scene.                              */
/* ---------------------------------------------------------------------- */
typedef struct {
    const vo_camera* cams;
    const vo_params* p;
    const double *means, *P6, *attr;
    double* Mc; /* [B][N][3] */
    double* Pc; /* [B][N][9] */
    int32_t* bbox; /* [B][N][4] (x0, x1, y0, y1) or NULL */
} scene_t;

static void scene_init(scene_t* s, const vo_camera* cams, const vo_params* p, const double* means,
                       const double* P6, const double* attr) {
    s->cams = cams; s->p = p; s->means = means; s->P6 = P6; s->attr = attr;
    size_t BN = (size_t)p->B * (size_t)p->N;
    s->Mc = (double*)malloc(sizeof(double) * 3 * (BN ? BN : 1));
    s->Pc = (double*)malloc(sizeof(double) * 9 * (BN ? BN : 1));
    s->bbox = NULL;
    for (int v = 0; v < p->B; v++)
        for (int g = 0; g < p->N; g++) {
            size_t o = (size_t)v * p->N + g;
            to_camera(&cams[v], means + 3 * (size_t)g, P6 + 6 * (size_t)g, s->Mc + 3 * o, s->Pc + 9 * o);
        }
}

static void scene_free(scene_t* s) {
    free(s->Mc); free(s->Pc); free(s->bbox);
}

/* Exact pixel bounding box of the region e^{q} > eta (culled mode).
 * qt(D) = DᵀQD / DᵀPD with Q = (MᵀPM) P - (PM)(PM)ᵀ (Lagrange identity in the
 * P inner product), so qt < r2 = 2 ln(1/eta) is the conic Dᵀ(Q - r2 P)D < 0 in
 * D = (x, y, 1).  If its upper 2x2 block is not positive definite the region
 * is unbounded on the image plane and the whole image is kept. */
static void bbox_one(const vo_camera* c, const vo_params* p, const double M[3], const double P[9], int32_t out[4]) {
    out[0] = 0; out[1] = c->W - 1; out[2] = 0; out[3] = c->H - 1;
    if (p->eta <= 0.0 || !(M[2] > 0.0)) {
        if (!(M[2] > 0.0)) { out[0] = 1; out[1] = 0; } /* never a candidate */
        return;
    }
    double r2 = 2.0 * log(1.0 / p->eta);
    double PM[3];
    for (int a = 0; a < 3; a++) PM[a] = P[3 * a] * M[0] + P[3 * a + 1] * M[1] + P[3 * a + 2] * M[2];
    double mpm = M[0] * PM[0] + M[1] * PM[1] + M[2] * PM[2];
    double Hm[9];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) Hm[3 * a + b] = (mpm - r2) * P[3 * a + b] - PM[a] * PM[b];
    double h00 = Hm[0], h01 = Hm[1], h11 = Hm[4], h02 = Hm[2], h12 = Hm[5], h22 = Hm[8];
    double det = h00 * h11 - h01 * h01;
    if (!(h00 > 0.0) || !(det > 0.0)) return; /* unbounded: whole image */
    double i00 = h11 / det, i01 = -h01 / det, i11 = h00 / det;
    double cx = -(i00 * h02 + i01 * h12), cy = -(i01 * h02 + i11 * h12);
    double f0 = h22 + h02 * cx + h12 * cy;
    if (!(f0 < 0.0)) { out[0] = 1; out[1] = 0; return; } /* empty */
    double xh = sqrt(-f0 * i00), yh = sqrt(-f0 * i11);
    /* pixel centre of column j is x = (j + 0.5 - Ox)/F; one pixel of margin */
    double jx0 = c->F * (cx - xh) + c->Ox - 0.5, jx1 = c->F * (cx + xh) + c->Ox - 0.5;
    double iy0 = c->F * (cy - yh) + c->Oy - 0.5, iy1 = c->F * (cy + yh) + c->Oy - 0.5;
    double lo_x = floor(jx0) - 1, hi_x = ceil(jx1) + 1, lo_y = floor(iy0) - 1, hi_y = ceil(iy1) + 1;
    if (lo_x < 0) lo_x = 0;
    if (lo_y < 0) lo_y = 0;
    if (hi_x > c->W - 1) hi_x = c->W - 1;
    if (hi_y > c->H - 1) hi_y = c->H - 1;
    out[0] = (int32_t)lo_x; out[1] = (int32_t)hi_x; out[2] = (int32_t)lo_y; out[3] = (int32_t)hi_y;
}

void vo_bbox(const vo_camera* cams, const vo_params* p, const double* means, const double* P6, int32_t* bbox) {
    for (int v = 0; v < p->B; v++)
        for (int g = 0; g < p->N; g++) {
            double M[3], P[9];
            to_camera(&cams[v], means + 3 * (size_t)g, P6 + 6 * (size_t)g, M, P);
            bbox_one(&cams[v], p, M, P, bbox + 4 * ((size_t)v * p->N + g));
        }
}

/* ---------------------------------------------------------------------- */
/* Selection (Sec. 3.3, App. A.3).                                         */
/* ---------------------------------------------------------------------- */
typedef struct { double l, a, b; int32_t g; } cand_t;

static int cand_cmp(const void* x, const void* y) {
    const cand_t* u = (const cand_t*)x;
    const cand_t* w = (const cand_t*)y;
    if (u->l < w->l) return -1;
    if (u->l > w->l) return 1;
    return (u->g < w->g) ? -1 : (u->g > w->g);
}

/* All Gaussians with M_z > 0, b > 0, l > 0 and (eta <= 0 or a > eta), sorted by
 * (l, index), truncated to the list capacity.  Returns the list length. */
static int select_list(const scene_t* s, int v, int i, int j, int culled, cand_t* buf) {
    const vo_params* p = s->p;
    const vo_camera* c = &s->cams[v];
    double D[3];
    ray_dir(c, i, j, D);
    int n = 0;
    for (int g = 0; g < p->N; g++) {
        size_t o = (size_t)v * p->N + g;
        if (culled) {
            const int32_t* bb = s->bbox + 4 * o;
            if (j < bb[0] || j > bb[1] || i < bb[2] || i > bb[3]) continue;
        }
        const double* M = s->Mc + 3 * o;
        const double* P = s->Pc + 9 * o;
        if (!(M[2] > 0.0)) continue;
        double l, qt, b;
        trace(M, P, D, &l, &qt, &b);
        if (!(b > 0.0) || !(l > 0.0)) continue;
        double a = exp(-0.5 * qt);
        if (p->eta > 0.0 && !(a > p->eta)) continue;
        buf[n].l = l; buf[n].a = a; buf[n].b = b; buf[n].g = g;
        n++;
    }
    qsort(buf, (size_t)n, sizeof(cand_t), cand_cmp);
    int cap = list_cap(p);
    return n < cap ? n : cap;
}

/* Re-trace a given list (frozen selection). Entries < 0 end the list. */
static int given_list(const scene_t* s, int v, int i, int j, const int32_t* idx, int Kc, cand_t* buf) {
    const vo_params* p = s->p;
    double D[3];
    ray_dir(&s->cams[v], i, j, D);
    int n = 0;
    for (int k = 0; k < Kc; k++) {
        int g = idx[k];
        if (g < 0) break;
        size_t o = (size_t)v * p->N + g;
        double l, qt, b;
        trace(s->Mc + 3 * o, s->Pc + 9 * o, D, &l, &qt, &b);
        buf[n].l = l; buf[n].a = exp(-0.5 * qt); buf[n].b = b; buf[n].g = g;
        n++;
    }
    return n;
}

/* ---------------------------------------------------------------------- */
/* Closed-form transmittance (Eq. 7) and blend (Eq. 8).                    */
/*   A_k = sum_j (a_j/2)(1 + erf((l_k - l_j) sqrt(b_j/2))),               */
/*   T_k = exp(-tau A_k),  W_k = T_k a_k,  C = sum_k W_k c_k.              */
/* ---------------------------------------------------------------------- */
static void fine(const vo_params* p, const cand_t* L, int n, const double* attr, double* T, double* W, double* img) {
    for (int k = 0; k < n; k++) {
        double A = 0.0;
        for (int j = 0; j < n; j++) A += 0.5 * L[j].a * (1.0 + erf((L[k].l - L[j].l) * sqrt(0.5 * L[j].b)));
        T[k] = exp(-p->tau * A);
        W[k] = T[k] * L[k].a;
    }
    for (int c = 0; c < p->C; c++) {
        double acc = 0.0;
        for (int k = 0; k < n; k++) acc += W[k] * attr[(size_t)L[k].g * p->C + c];
        img[c] = acc;
    }
}

/* ---------------------------------------------------------------------- */
/* Threaded drivers.                                                       */
/* ---------------------------------------------------------------------- */
typedef struct {
    const scene_t* s;
    const int32_t* pix; /* [npix][3]: view, row, col */
    int64_t p0, p1;
    int culled;
    const int32_t* idx_in; /* frozen lists or NULL */
    int Kc;
    double *image, *weights, *ldepth, *aval;
    int32_t* idx_out;
    int32_t* count;
    /* backward */
    const double* gimg;
    double *gM, *gP6, *gattr, *gRT; /* per-thread accumulators */
} job_t;

static void* fwd_worker(void* arg) {
    job_t* jb = (job_t*)arg;
    const scene_t* s = jb->s;
    const vo_params* p = s->p;
    int Kc = jb->Kc;
    cand_t* buf = (cand_t*)malloc(sizeof(cand_t) * (p->N > 0 ? p->N : 1));
    double* T = (double*)malloc(sizeof(double) * (Kc > 0 ? Kc : 1));
    double* W = (double*)malloc(sizeof(double) * (Kc > 0 ? Kc : 1));
    for (int64_t q = jb->p0; q < jb->p1; q++) {
        int v = jb->pix[3 * q], i = jb->pix[3 * q + 1], j = jb->pix[3 * q + 2];
        int n = jb->idx_in ? given_list(s, v, i, j, jb->idx_in + (size_t)q * Kc, Kc, buf)
                           : select_list(s, v, i, j, jb->culled, buf);
        fine(p, buf, n, s->attr, T, W, jb->image + (size_t)q * p->C);
        for (int k = 0; k < Kc; k++) {
            int in = k < n;
            if (jb->weights) jb->weights[(size_t)q * Kc + k] = in ? W[k] : 0.0;
            if (jb->idx_out) jb->idx_out[(size_t)q * Kc + k] = in ? buf[k].g : -1;
            if (jb->ldepth) jb->ldepth[(size_t)q * Kc + k] = in ? buf[k].l : 0.0;
            if (jb->aval) jb->aval[(size_t)q * Kc + k] = in ? buf[k].a : 0.0;
        }
        if (jb->count) jb->count[q] = n;
    }
    free(buf); free(T); free(W);
    return NULL;
}

static void run_threads(job_t* base, int64_t npix, int nthreads, void* (*fn)(void*), job_t* jobs) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = *base;
        jobs[t].p0 = npix * t / nthreads;
        jobs[t].p1 = npix * (t + 1) / nthreads;
    }
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, fn, &jobs[t]);
    fn(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
}

/* Forward render of a list of pixels.  Outputs (any may be NULL except image):
 * image [npix][C], weights/ldepth/aval [npix][Kc], idx [npix][Kc] (-1 pad),
 * count [npix].  Kc = K if 0 < K < N else N.  culled: 1 uses the exact conic
 * bounding boxes to skip Gaussians (must not change any result). */
int vo_render(const vo_camera* cams, const vo_params* p, const double* means, const double* P6, const double* attr,
              const int32_t* pix, int64_t npix, int culled, int nthreads, double* image, double* weights,
              int32_t* idx, int32_t* count, double* ldepth, double* aval) {
    scene_t s;
    scene_init(&s, cams, p, means, P6, attr);
    if (culled) {
        size_t BN = (size_t)p->B * p->N;
        s.bbox = (int32_t*)malloc(sizeof(int32_t) * 4 * (BN ? BN : 1));
        vo_bbox(cams, p, means, P6, s.bbox);
    }
    job_t base;
    memset(&base, 0, sizeof(base));
    base.s = &s; base.pix = pix; base.culled = culled; base.Kc = list_cap(p);
    base.image = image; base.weights = weights; base.idx_out = idx; base.count = count;
    base.ldepth = ldepth; base.aval = aval;
    job_t jobs[256];
    run_threads(&base, npix, nthreads, fwd_worker, jobs);
    scene_free(&s);
    return 0;
}

/* Fine pass (Eq. 7-8) over given, frozen lists idx [npix][Kc]. */
int vo_fine(const vo_camera* cams, const vo_params* p, const double* means, const double* P6, const double* attr,
            const int32_t* pix, int64_t npix, const int32_t* idx, int Kc, int nthreads, double* image,
            double* weights) {
    scene_t s;
    scene_init(&s, cams, p, means, P6, attr);
    job_t base;
    memset(&base, 0, sizeof(base));
    base.s = &s; base.pix = pix; base.idx_in = idx; base.Kc = Kc;
    base.image = image; base.weights = weights;
    job_t jobs[256];
    run_threads(&base, npix, nthreads, fwd_worker, jobs);
    scene_free(&s);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Backward: chain rule of Eq. 5-8 with the lists frozen.                  */
/* ---------------------------------------------------------------------- */
static void* bwd_worker(void* arg) {
    job_t* jb = (job_t*)arg;
    const scene_t* s = jb->s;
    const vo_params* p = s->p;
    int Kc = jb->Kc, C = p->C;
    cand_t* L = (cand_t*)malloc(sizeof(cand_t) * (Kc > 0 ? Kc : 1));
    size_t nk = (size_t)(Kc > 0 ? Kc : 1);
    double *T = calloc(nk, 8), *W = calloc(nk, 8), *img = calloc((size_t)(C > 0 ? C : 1), 8);
    double *dA = calloc(nk, 8), *da = calloc(nk, 8), *dl = calloc(nk, 8), *dr = calloc(nk, 8), *dm = calloc(nk, 8);
    const double two_over_sqrtpi = 2.0 / sqrt(M_PI);
    for (int64_t q = jb->p0; q < jb->p1; q++) {
        int v = jb->pix[3 * q], i = jb->pix[3 * q + 1], j = jb->pix[3 * q + 2];
        const vo_camera* c = &s->cams[v];
        int n = given_list(s, v, i, j, jb->idx_in + (size_t)q * Kc, Kc, L);
        if (n == 0) continue;
        fine(p, L, n, s->attr, T, W, img);
        const double* g = jb->gimg + (size_t)q * C;
        /* C = sum_k W_k c_k */
        for (int k = 0; k < n; k++) {
            double dW = 0.0;
            const double* ck = s->attr + (size_t)L[k].g * C;
            for (int cc = 0; cc < C; cc++) {
                dW += g[cc] * ck[cc];
                jb->gattr[(size_t)L[k].g * C + cc] += W[k] * g[cc];
            }
            /* W_k = T_k a_k,  T_k = exp(-tau A_k) */
            da[k] = dW * T[k];
            dA[k] = -p->tau * T[k] * (dW * L[k].a);
            dl[k] = 0.0; dr[k] = 0.0; dm[k] = 0.0;
        }
        /* A_k = sum_j m_j (1 + erf(u_kj)),  u_kj = (l_k - l_j) r_j */
        for (int k = 0; k < n; k++)
            for (int jj = 0; jj < n; jj++) {
                double rj = sqrt(0.5 * L[jj].b);
                double u = (L[k].l - L[jj].l) * rj;
                double mj = 0.5 * L[jj].a;
                dm[jj] += dA[k] * (1.0 + erf(u));
                double du = dA[k] * mj * two_over_sqrtpi * exp(-u * u);
                dl[k] += du * rj;
                dl[jj] -= du * rj;
                dr[jj] += du * (L[k].l - L[jj].l);
            }
        double D[3];
        ray_dir(c, i, j, D);
        for (int k = 0; k < n; k++) {
            double a = L[k].a, b = L[k].b, l = L[k].l;
            double da_tot = da[k] + 0.5 * dm[k];            /* m = a/2 */
            double dqt = da_tot * (-0.5 * a);               /* a = exp(-qt/2) */
            double rk = sqrt(0.5 * b);
            double db = dr[k] / (4.0 * rk);                 /* r = sqrt(b/2) */
            size_t o = (size_t)v * p->N + L[k].g;
            const double* M = s->Mc + 3 * o;
            const double* P = s->Pc + 9 * o;
            double V[3] = {M[0] - l * D[0], M[1] - l * D[1], M[2] - l * D[2]};
            double PV[3], PD[3];
            for (int a3 = 0; a3 < 3; a3++) {
                PV[a3] = P[3 * a3] * V[0] + P[3 * a3 + 1] * V[1] + P[3 * a3 + 2] * V[2];
                PD[a3] = P[3 * a3] * D[0] + P[3 * a3 + 1] * D[1] + P[3 * a3 + 2] * D[2];
            }
            /* camera-space gradients:
             *   dqt/dM = 2PV, dl/dM = PD/b, db/dM = 0
             *   dqt/dP_ab = V_a V_b, dl/dP_ab = (M_a D_b + D_a M_b)/(2b) - l D_a D_b / b,
             *   db/dP_ab = D_a D_b  (P entries treated as independent; result symmetric) */
            double gM[3], G[9];
            for (int a3 = 0; a3 < 3; a3++) gM[a3] = dqt * 2.0 * PV[a3] + dl[k] * PD[a3] / b;
            for (int a3 = 0; a3 < 3; a3++)
                for (int b3 = 0; b3 < 3; b3++)
                    G[3 * a3 + b3] = dqt * V[a3] * V[b3] +
                                     dl[k] * ((M[a3] * D[b3] + D[a3] * M[b3]) / (2.0 * b) - l * D[a3] * D[b3] / b) +
                                     db * D[a3] * D[b3];
            /* world space: M_cam = R M_w + T, P_cam = R P_w Rᵀ */
            const double* R = c->R;
            double* gMw = jb->gM + 3 * (size_t)L[k].g;
            for (int a3 = 0; a3 < 3; a3++) gMw[a3] += R[a3] * gM[0] + R[3 + a3] * gM[1] + R[6 + a3] * gM[2];
            double Gw[9];
            for (int x = 0; x < 3; x++)
                for (int y = 0; y < 3; y++) {
                    double acc = 0.0;
                    for (int a3 = 0; a3 < 3; a3++)
                        for (int b3 = 0; b3 < 3; b3++) acc += R[3 * a3 + x] * G[3 * a3 + b3] * R[3 * b3 + y];
                    Gw[3 * x + y] = acc;
                }
            double* gp = jb->gP6 + 6 * (size_t)L[k].g;
            gp[0] += Gw[0];
            gp[1] += Gw[1] + Gw[3];
            gp[2] += Gw[2] + Gw[6];
            gp[3] += Gw[4];
            gp[4] += Gw[5] + Gw[7];
            gp[5] += Gw[8];
            /* camera: dL/dR = gM Mwᵀ + G R Pwᵀ + Gᵀ R Pw,  dL/dT = gM */
            const double* Mw = s->means + 3 * (size_t)L[k].g;
            double Pw[9];
            sym_from6(s->P6 + 6 * (size_t)L[k].g, Pw);
            double RP[9];
            for (int x = 0; x < 3; x++)
                for (int y = 0; y < 3; y++) {
                    double acc = 0.0;
                    for (int z = 0; z < 3; z++) acc += R[3 * x + z] * Pw[3 * z + y];
                    RP[3 * x + y] = acc;
                }
            double* gRT = jb->gRT + 12 * (size_t)v;
            for (int x = 0; x < 3; x++)
                for (int y = 0; y < 3; y++) {
                    double acc = gM[x] * Mw[y];
                    for (int z = 0; z < 3; z++) acc += (G[3 * x + z] + G[3 * z + x]) * RP[3 * z + y];
                    gRT[3 * x + y] += acc;
                }
            for (int x = 0; x < 3; x++) gRT[9 + x] += gM[x];
        }
    }
    free(L); free(T); free(W); free(img); free(dA); free(da); free(dl); free(dr); free(dm);
    return NULL;
}

/* Backward with frozen lists idx [npix][Kc].  Gradients are written (not
 * accumulated): g_means [N][3], g_P6 [N][6] (derivative w.r.t. the six
 * parameters xx,xy,xz,yy,yz,zz), g_attr [N][C], g_RT [B][12] = (dL/dR row-major,
 * dL/dT).  grad_image [npix][C]. */
int vo_render_bwd(const vo_camera* cams, const vo_params* p, const double* means, const double* P6,
                  const double* attr, const int32_t* pix, int64_t npix, const int32_t* idx, int Kc,
                  const double* grad_image, int nthreads, double* g_means, double* g_P6, double* g_attr,
                  double* g_RT) {
    scene_t s;
    scene_init(&s, cams, p, means, P6, attr);
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    size_t N = (size_t)p->N, C = (size_t)p->C, B = (size_t)p->B;
    job_t base;
    memset(&base, 0, sizeof(base));
    base.s = &s; base.pix = pix; base.idx_in = idx; base.Kc = Kc; base.gimg = grad_image;
    job_t jobs[256];
    for (int t = 0; t < nthreads; t++) {
        jobs[t] = base;
        jobs[t].p0 = npix * t / nthreads;
        jobs[t].p1 = npix * (t + 1) / nthreads;
        jobs[t].gM = calloc(3 * N + 1, 8);
        jobs[t].gP6 = calloc(6 * N + 1, 8);
        jobs[t].gattr = calloc(C * N + 1, 8);
        jobs[t].gRT = calloc(12 * B + 1, 8);
    }
    pthread_t th[256];
    for (int t = 1; t < nthreads; t++) pthread_create(&th[t], NULL, bwd_worker, &jobs[t]);
    bwd_worker(&jobs[0]);
    for (int t = 1; t < nthreads; t++) pthread_join(th[t], NULL);
    memset(g_means, 0, 8 * 3 * N);
    memset(g_P6, 0, 8 * 6 * N);
    memset(g_attr, 0, 8 * C * N);
    memset(g_RT, 0, 8 * 12 * B);
    for (int t = 0; t < nthreads; t++) {
        for (size_t x = 0; x < 3 * N; x++) g_means[x] += jobs[t].gM[x];
        for (size_t x = 0; x < 6 * N; x++) g_P6[x] += jobs[t].gP6[x];
        for (size_t x = 0; x < C * N; x++) g_attr[x] += jobs[t].gattr[x];
        for (size_t x = 0; x < 12 * B; x++) g_RT[x] += jobs[t].gRT[x];
        free(jobs[t].gM); free(jobs[t].gP6); free(jobs[t].gattr); free(jobs[t].gRT);
    }
    scene_free(&s);
    return 0;
}

/* ---------------------------------------------------------------------- */
/* Exact outer integral of Eq. 1 for one ray, by adaptive Simpson.         */
/* Along the ray each kept kernel contributes density                      */
/*   rho_k(t) = a_k * sqrt(b_k/(2 pi)) * exp(-b_k (t - l_k)^2 / 2)         */
/* (a 1D Gaussian of mass a_k, the reading under which Eq. 7 is exact),    */
/* T(t) = exp(-tau sum_j (a_j/2)(1 + erf((t - l_j) sqrt(b_j/2)))) exactly, */
/* and W_k^exact = int T(t) rho_k(t) dt.  Eq. 8 replaces T(t) by T(l_k).   */
/* ---------------------------------------------------------------------- */
typedef struct { const double *l, *a, *b; int n, k; double tau; } qctx_t;

static double q_integrand(const qctx_t* q, double x) {
    /* x = (t - l_k) sqrt(b_k): unit-variance coordinate of kernel k */
    double t = q->l[q->k] + x / sqrt(q->b[q->k]);
    double A = 0.0;
    for (int j = 0; j < q->n; j++) A += 0.5 * q->a[j] * (1.0 + erf((t - q->l[j]) * sqrt(0.5 * q->b[j])));
    return exp(-q->tau * A) * q->a[q->k] * exp(-0.5 * x * x) / sqrt(2.0 * M_PI);
}

static double simpson_rec(const qctx_t* q, double lo, double hi, double flo, double fmid, double fhi, double whole,
                          double eps, int depth) {
    double mid = 0.5 * (lo + hi);
    double lm = 0.5 * (lo + mid), rm = 0.5 * (mid + hi);
    double flm = q_integrand(q, lm), frm = q_integrand(q, rm);
    double left = (mid - lo) / 6.0 * (flo + 4.0 * flm + fmid);
    double right = (hi - mid) / 6.0 * (fmid + 4.0 * frm + fhi);
    double d = left + right - whole;
    if (depth <= 0 || fabs(d) <= 15.0 * eps) return left + right + d / 15.0;
    return simpson_rec(q, lo, mid, flo, flm, fmid, left, 0.5 * eps, depth - 1) +
           simpson_rec(q, mid, hi, fmid, frm, fhi, right, 0.5 * eps, depth - 1);
}

/* W_exact of kernel k among the n kernels (l, a, b) of one ray. */
double vo_quad_weight(const double* l, const double* a, const double* b, int n, double tau, int k) {
    qctx_t q = {l, a, b, n, k, tau};
    /* integrate x in [-14, 14] as 28 unit panels, each adaptively */
    double acc = 0.0;
    for (int s = -14; s < 14; s++) {
        double lo = s, hi = s + 1.0;
        double flo = q_integrand(&q, lo), fhi = q_integrand(&q, hi), fmid = q_integrand(&q, 0.5 * (lo + hi));
        double whole = (hi - lo) / 6.0 * (flo + 4.0 * fmid + fhi);
        acc += simpson_rec(&q, lo, hi, flo, fmid, fhi, whole, 1e-14, 40);
    }
    return acc;
}

/* W_exact[k] for the n kernels (l, a, b) of one ray. */
void vo_quad_weights(const double* l, const double* a, const double* b, int n, double tau, double* W_exact) {
    for (int k = 0; k < n; k++) W_exact[k] = vo_quad_weight(l, a, b, n, tau, k);
}

/* Neural sampler, Sec. 3.4 Eq. 10, on given per-pixel lists and weights:
 * idx [P][L] (negative = empty slot), W [P][L], phi [P][C] ->
 * alpha [N][C] = sum_p W_pk phi_p / sum_p W_pk and wsum [N] = sum_p W_pk
 * (alpha_k = 0 where wsum_k = 0).  Plain loops in pixel order. */
int vo_sample(int64_t P, int L, int N, int C, const int32_t* idx, const double* W, const double* phi, double* alpha,
              double* wsum) {
    if (P < 0 || L < 0 || N < 0 || C < 0) return -1;
    memset(alpha, 0, sizeof(double) * (size_t)N * (size_t)C);
    memset(wsum, 0, sizeof(double) * (size_t)N);
    for (int64_t p = 0; p < P; ++p) {
        for (int k = 0; k < L; ++k) {
            const int32_t g = idx[p * L + k];
            if (g < 0 || g >= N) continue;
            const double w = W[p * L + k];
            wsum[g] += w;
            for (int c = 0; c < C; ++c) alpha[(int64_t)g * C + c] += w * phi[p * C + c];
        }
    }
    for (int g = 0; g < N; ++g)
        for (int c = 0; c < C; ++c) alpha[(int64_t)g * C + c] = wsum[g] > 0.0 ? alpha[(int64_t)g * C + c] / wsum[g] : 0.0;
    return 0;
}
