/*
 * voge.h -- C ABI of libvoge.so, the GB300 (sm_103a) implementation of the
 * VoGE renderer's hot path (Wang et al., "VoGE: A Differentiable Volume
 * Renderer using Gaussian Ellipsoids for Analysis-by-Synthesis", ICLR 2023).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * - Pointers marked "device" are CUDA device pointers on the current device;
 *   pointers marked "host" are ordinary host memory.  The caller owns every
 *   buffer, including the workspace.  No entry point allocates device memory.
 * - All device work is enqueued on `stream` (0 = legacy default stream) and
 *   is asynchronous with respect to the host, except voge_render_fwd /
 *   voge_render_bwd, which copy the B camera structs from host memory into the
 *   workspace with cudaMemcpyAsync before their first launch (the host array
 *   may be reused as soon as the call returns).
 * - Return value: VOGE_OK (0) or a negative VOGE_ERR_* code; nothing aborts.
 *   A launch error is reported as VOGE_ERR_CUDA; the CUDA error itself can be
 *   read with cudaGetLastError() by the caller.
 * - Camera model (Sec. 3.3 and Eq. 5 of the paper): a Gaussian with world mean
 *   M_w and world inverse covariance P_w is seen at M = R M_w + T with inverse
 *   covariance R P_w Rᵀ.  The ray of pixel (row i, column j) is r(t) = tD with
 *   D = ((j + 0.5 - Ox)/F, (i + 0.5 - Oy)/F, 1): x right, y down, z forward.
 * - Pixels: views are stored back to back, view v holding H_v x W_v pixels in
 *   row-major order.  When every view has the same H, W this is [B][H][W].
 * - Gaussians: means [N][3] (x, y, z); inverse covariances P = Sigma^-1 as six
 *   floats per Gaussian in the order (xx, xy, xz, yy, yz, zz) of the symmetric
 *   matrix; attributes [N][C] (RGB when C = 3, or C-channel features).
 */
#ifndef VOGE_H
#define VOGE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st* voge_stream_t; /* same type as cudaStream_t */

enum {
    VOGE_OK = 0,
    VOGE_ERR_ARG = -1,        /* a size, pointer or parameter is invalid */
    VOGE_ERR_WORKSPACE = -2,  /* workspace NULL or smaller than voge_workspace_bytes() */
    VOGE_ERR_CUDA = -3,       /* a CUDA call or kernel launch failed */
    VOGE_ERR_UNSUPPORTED = -4,/* a combination the library does not implement */
    VOGE_ERR_TIMEOUT = -5,    /* a bounded wait ran out (serving) */
    VOGE_ERR_ADMISSION = -6,  /* request larger than the server's memory budget */
    VOGE_ERR_BUSY = -7,       /* no free slot / queue full (serving) */
    VOGE_ERR_CHECK = -8       /* checked builds only (libvoge_checked.so): a kernel caught an index
                                 outside its array; the access was redirected to element 0 and the
                                 outputs of the call are not valid */
};

/* One view.  R row-major; M_cam = R M_world + T (Sec. 3.3).  F, Ox, Oy in
 * pixels (Eq. 5).  H, W: image size of this view. */
typedef struct {
    float R[9];
    float T[3];
    float F, Ox, Oy;
    int32_t H, W;
} voge_camera;

/* Render parameters.
 *   B       number of views (>= 1)
 *   N       number of Gaussians (>= 0)
 *   C       attribute channels (>= 1)
 *   K       length of each pixel's kept list: the K' nearest kernels of
 *           Sec. 3.3 / App. A.3.  K <= 0 or K >= N keeps every candidate.
 *   tau     absorption coefficient of Eq. 1 / Eq. 7 (> 0)
 *   thresh  eta of App. A.3: a kernel is a candidate for a pixel only if its
 *           peak density e^{q} on that ray is > thresh.  thresh <= 0: no cut.
 *   flags   VOGE_FLAG_* bits
 *   bin_capacity  average number of 16x16 screen tiles per Gaussian that the
 *           workspace reserves for tile binning (0 = default 8).  Overflow never
 *           changes a result: the tiles whose lists overflowed fall back to
 *           testing every Gaussian. */
typedef struct {
    int32_t B, N, C, K;
    float tau, thresh;
    int32_t flags;
    int32_t bin_capacity;
} voge_params;

enum {
    /* Comparator path: every pixel tests every Gaussian (no tile binning). */
    VOGE_FLAG_PLAIN = 1,
    /* voge_render_bwd only: reuse the projection that the matching
     * voge_render_fwd call left in the same workspace (same cams, params and
     * Gaussians, workspace untouched in between) instead of recomputing it.
     * When index is that call's index output (the same buffer, unchanged),
     * its record of which 16 x 2-pixel row pairs kept an entry is reused
     * too, so that the backward skips the others without reading them. */
    VOGE_FLAG_REUSE_PROJECTION = 2,
    /* voge_render_fwd only: run the coarse pass (selection) and the fine pass
     * as two kernels -- the selection writes the index lists, then the fine
     * pass of voge_render_fine reads them -- instead of one fused kernel.
     * Same outputs up to the rounding of W (identical arithmetic); lists
     * longer than 32 always take the fused path. */
    VOGE_FLAG_SPLIT_FORWARD = 4
};

/* Library version (major*10000 + minor*100 + patch). */
int voge_version(void);

/* Human-readable text for a VOGE_* code (static storage). */
const char* voge_strerror(int code);

/* Effective list length: K if 0 < K < N, else N (and 0 when N == 0). */
int voge_list_length(const voge_params* p);

/* Bytes of device workspace that voge_render_fwd / voge_render_bwd need for
 * these cameras (host, B entries) and parameters.  Query, allocate, then call.
 * Returns 0 if the arguments are invalid. */
size_t voge_workspace_bytes(const voge_camera* cams, const voge_params* p);

/*
 * Forward render: coarse pass (ray tracing of each ellipsoid, Eq. 6; keep
 * kernels with e^{q} > thresh and l > 0, sort by peak depth l, keep the K
 * nearest -- Sec. 3.3, App. A.3) and fine pass (closed-form transmittance of
 * Eq. 7 over the kept list, weights W_k = T(l_k) e^{q_k} and blend of Eq. 8).
 *
 *   cams     host, [B]
 *   means    device, [N][3] float
 *   inv_cov  device, [N][6] float (xx, xy, xz, yy, yz, zz of Sigma^-1)
 *   attr     device, [N][C] float
 *   image    device, [pixels][C] float, written: sum_k W_k c_k (no background)
 *   weights  device, [pixels][L] float, written: W_k in list order, 0 padded;
 *            may be NULL
 *   index    device, [pixels][L] int32, written: Gaussian index of each kept
 *            kernel, ascending (l, index), -1 padded.  Required (the backward
 *            pass reads it).
 *   L = voge_list_length(p).  Every output element is written.
 *   workspace  device, >= voge_workspace_bytes(cams, p) bytes, 256-byte aligned.
 */
int voge_render_fwd(const voge_camera* cams, const voge_params* p, const float* means, const float* inv_cov,
                    const float* attr, float* image, float* weights, int32_t* index, void* workspace,
                    size_t workspace_bytes, voge_stream_t stream);

/*
 * What the last forward pass run in a workspace did, counted on the device
 * while it ran (one addition per warp and tile):
 *   traces   Gaussian-ray traces of the coarse pass: evaluations of Eq. 6
 *            (l, e^{q}, sigma) for a (pixel, candidate kernel), including the
 *            candidates the threshold or the list then rejects
 *   entries  kept (pixel, kernel) entries: the sum of the list lengths
 *   pairs    (k, j) pairs of the fine pass's transmittance sums (Eq. 7): the
 *            sum over pixels of the squared list length
 * `workspace` is the one passed to voge_render_fwd; the counts stay valid
 * until the next call that uses the workspace (voge_render_bwd resets them).
 * Copies 24 bytes to `out` (host) on `stream` and waits for the stream.
 * VOGE_ERR_ARG for NULL or misaligned pointers, VOGE_ERR_CUDA on a CUDA failure.
 * Not a step of the paper: an aid for measurement.
 */
typedef struct {
    int64_t traces, entries, pairs;
} voge_render_stats_t;
int voge_render_stats(const void* workspace, voge_render_stats_t* out, voge_stream_t stream);

/*
 * Fine pass alone (Eq. 7 and 8) over given per-pixel lists: for each pixel
 * with list S_p (the entries before the first slot outside [0, N)),
 *   A_k = sum_{j in S_p} (a_j/2)(1 + erf((l_k - l_j) sqrt(b_j/2))),
 *   W_k = exp(-tau A_k) e^{q_k},  image_p = sum_k W_k c_k,
 * with l, e^{q} = a and b = DᵀPD of each listed kernel on the pixel's ray
 * (Eq. 6).  The sum is over the list in any order; it includes k itself.
 * The selection (thresh, K) is not applied: the lists are taken as given.
 * This is the second half of voge_render_fwd, for re-rendering from saved
 * lists (new attributes or tau, same selection) and for checking the fine
 * pass on its own.
 *
 *   cams, p    as voge_render_fwd; L = voge_list_length(p) must be <= 32
 *              (VOGE_ERR_UNSUPPORTED otherwise)
 *   index      device, [pixels][L] int32: each pixel's list, ended by the
 *              first entry < 0 or >= N (typically voge_render_fwd's output)
 *   image      device, [pixels][C] float, written
 *   weights    device, [pixels][L] float, written: W_k in list order, 0 after
 *              the list's end; may be NULL
 *   workspace  device, >= voge_workspace_bytes(cams, p), 256-byte aligned
 * Asynchronous on `stream`; allocates nothing.  VOGE_ERR_ARG / _WORKSPACE as
 * voge_render_fwd.
 */
int voge_render_fine(const voge_camera* cams, const voge_params* p, const float* means, const float* inv_cov,
                     const float* attr, const int32_t* index, float* image, float* weights, void* workspace,
                     size_t workspace_bytes, voge_stream_t stream);

/*
 * Backward pass of voge_render_fwd with the kept lists frozen (the selection
 * is piecewise constant; no gradient flows through it).  Recomputes l, e^{q},
 * sigma, T(l_k) and every erf term from `index` (nothing else is saved), then
 * applies the chain rule of Eq. 5-8.
 *
 *   index       device, [pixels][L] int32 from voge_render_fwd
 *   grad_image  device, [pixels][C] float: dLoss/dimage
 *   grad_means  device, [N][3] float or NULL      -- ACCUMULATED into (+=)
 *   grad_inv_cov device, [N][6] float or NULL    -- ACCUMULATED; derivative
 *               with respect to the six stored parameters (so an off-diagonal
 *               entry receives dL/dP_xy + dL/dP_yx)
 *   grad_attr   device, [N][C] float or NULL     -- ACCUMULATED
 *   grad_cam    device, [B][12] float or NULL    -- ACCUMULATED: dL/dR (9,
 *               row-major) then dL/dT (3) of each view
 *   The caller zeroes the gradient buffers before the first accumulation.
 *   Floating-point atomics make the last bits of the gradients depend on
 *   scheduling.
 */
int voge_render_bwd(const voge_camera* cams, const voge_params* p, const float* means, const float* inv_cov,
                    const float* attr, const int32_t* index, const float* grad_image, float* grad_means,
                    float* grad_inv_cov, float* grad_attr, float* grad_cam, void* workspace,
                    size_t workspace_bytes, voge_stream_t stream);

/*
 * voge_render_bwd with the forward's weights supplied.  W_k = T(l_k) e^{q_k}
 * of Eq. 7 is the only quantity of the backward pass that needs the
 * transmittance sum over the whole list; taking it from the forward pass
 * removes that recomputation.  Same results as voge_render_bwd up to the
 * rounding of W (the forward computes it with the same arithmetic).
 *
 *   weights  device, [pixels][L] float: the `weights` output of the
 *            voge_render_fwd call that produced `index` (same cameras,
 *            parameters and scene), or NULL to recompute W from `index`.
 *   All other arguments, ownership and errors as voge_render_bwd.
 */
int voge_render_bwd_w(const voge_camera* cams, const voge_params* p, const float* means, const float* inv_cov,
                      const float* attr, const int32_t* index, const float* weights, const float* grad_image,
                      float* grad_means, float* grad_inv_cov, float* grad_attr, float* grad_cam, void* workspace,
                      size_t workspace_bytes, voge_stream_t stream);

/*
 * Neural sampler of Sec. 3.4 (Eq. 10): per-kernel attributes from per-pixel
 * features (image values, deep features) through the renderer's kept lists,
 *   alpha_k = sum_p W_pk phi_p / sum_p W_pk,
 * the sums over the pixels whose list holds k (W_pk of Eq. 8 is zero for the
 * others).  A kernel that no pixel keeps gets alpha_k = 0.
 *
 *   pixels    number of pixels P (all views of a voge_render_fwd call: the
 *             sum of H*W)
 *   L         list length of `index` and `weights` (voge_list_length)
 *   N, C      kernels and feature channels
 *   index     device, [P][L] int32 from voge_render_fwd (negative = empty
 *             slot; indices >= N are ignored)
 *   weights   device, [P][L] float from voge_render_fwd
 *   features  device, [P][C] float: phi_p
 *   alpha     device, [N][C] float, written (overwritten, not accumulated)
 *   wsum      device, [N] float, written: sum_p W_pk
 *   Asynchronous on `stream`; allocates nothing.  VOGE_ERR_ARG for negative
 *   sizes, C < 1 or a missing pointer.  Floating-point atomics make the last
 *   bits depend on scheduling.
 */
int voge_sample(int64_t pixels, int32_t L, int32_t N, int32_t C, const int32_t* index, const float* weights,
                const float* features, float* alpha, float* wsum, voge_stream_t stream);

/*
 * Mesh and point-cloud converters (App. A.4): one isotropic Gaussian per
 * vertex or point, centred on it, with the variance on the diagonal
 *   sigma_k = (d_k / 2)^2 / log(1 / zeta),
 * zeta in (0, 1) the coverage rate (0.5 standard).  Outputs are the renderer's
 * inputs: means [V][3] and inverse covariances [V][6] (xx, xy, xz, yy, yz, zz),
 * device float, written.  Asynchronous on `stream`.
 *
 * Mesh: d_k is the mean length of the distinct edges at vertex k.
 *   verts  device, [V][3] float;  faces  device, [F][3] int32 vertex indices
 *          (faces with an index outside [0, V) or a repeated vertex are
 *          skipped; a vertex on no edge gets NaN inverse covariances).
 *   flatten  0: isotropic.  f > 0: flattened along the vertex normal n (the
 *          normalised sum of the adjacent faces' area-weighted normals), the
 *          variant App. B describes: Sigma = sigma (I - n nᵀ) + f sigma n nᵀ.
 *   workspace  device, >= voge_mesh_workspace_bytes(V, F), 256-byte aligned
 *          (an edge set and per-vertex sums); VOGE_ERR_WORKSPACE otherwise.
 * Points: d_k is the mean distance from point k to its m nearest other
 *   points, 1 <= m <= 32 and m < V (brute force over all points).
 * VOGE_ERR_ARG for negative sizes, zeta outside (0, 1), a negative flatten,
 * m out of range or a missing pointer.
 */
size_t voge_mesh_workspace_bytes(int32_t V, int32_t F);
int voge_mesh_to_gaussians(int32_t V, int32_t F, const float* verts, const int32_t* faces, float zeta, float flatten,
                           float* means, float* inv_cov, void* workspace, size_t workspace_bytes,
                           voge_stream_t stream);
int voge_points_to_gaussians(int32_t V, int32_t m, float zeta, const float* points, float* means, float* inv_cov,
                             voge_stream_t stream);

/*
 * Camera pose (azimuth, elevation, distance, roll), radians -> R, T (host).
 * Look-at camera: centre dist*(cos e sin a, sin e, cos e cos a), looking at
 * the world origin, world up +y, then a roll about the optical axis.  The
 * paper's render-and-compare pose estimation (Sec. 4.1) does not fix a pose
 * parameterisation; this look-at form is the library's choice.
 *   pose  host [4];  R host [9] row-major;  T host [3].
 */
void voge_pose_to_RT(const double pose[4], float R[9], float T[3]);

/*
 * Chain rule of voge_pose_to_RT on the device: grad_pose[v] += d(R,T)/d(pose)ᵀ
 * grad_cam[v] for v < B.
 *   pose       device [B][4] float
 *   grad_cam   device [B][12] float (dL/dR row-major, dL/dT), as voge_render_bwd writes
 *   grad_pose  device [B][4] float, ACCUMULATED
 */
int voge_pose_grad(const float* pose, const float* grad_cam, float* grad_pose, int32_t B, voge_stream_t stream);

/*
 * Mean-squared-error helper for render-and-compare loops (Sec. 4.3 fits a
 * render to target images): loss[0] += sum((image - target)^2) / n and
 * grad_image = 2 (image - target) / n, n = count.  All device pointers.
 */
int voge_mse_grad(const float* image, const float* target, int64_t count, float* grad_image, float* loss,
                  voge_stream_t stream);

/* ------------------------------------------------------------------------
 * Serving: render-and-compare requests with continuous batching.
 *
 * Not a step of the paper: the paper's analysis-by-synthesis loops (pose
 * estimation, Sec. 4.1; shape fitting, Sec. 4.3) issue one render + gradient
 * per optimisation step.  The server runs many such steps for many scenes at
 * once.  A request renders one view of its own scene (voge_render_fwd), takes
 * the mean squared error against a target image and returns the image, the
 * loss and the gradients (voge_render_bwd), exactly as those calls would.
 *
 * Requests are admitted in arrival order whenever a slot and enough of the
 * server's device memory are free; their inputs are copied in on a copy
 * stream while earlier work runs.  Each tick takes every admitted request
 * whose inputs have arrived and runs them together: one persistent launch
 * per list-length class covers all of them.  With use_graphs, a tick is the
 * replay of a CUDA graph captured once per set of classes present.  Up to
 * inflight_ticks ticks run at once on separate streams.  With batching = 0
 * every request runs alone (one request per tick): the plain comparator.
 *
 * Ownership: the server allocates its device memory (mem_budget_bytes, one
 * allocation) and pinned staging at creation, and nothing afterwards.  Host
 * buffers of a request (inputs and outputs) must stay valid until
 * voge_server_wait returns for its ticket; page-locked host buffers keep the
 * copies asynchronous (pageable ones make the scheduler thread wait).
 * ------------------------------------------------------------------------ */
typedef struct voge_server voge_server;

typedef struct {
    int32_t device;            /* CUDA device ordinal */
    int32_t max_slots;         /* requests resident on the device at once (>= 1) */
    int32_t max_queue;         /* pending requests before submit returns VOGE_ERR_BUSY (<= 0: 65536) */
    int32_t use_graphs;        /* 1: each tick is a CUDA-graph replay */
    int32_t batching;          /* 1: continuous batching; 0: one request per tick */
    int32_t inflight_ticks;    /* ticks running at once, 1..4 (<= 0: 2) */
    int64_t max_tick_gaussians;/* Gaussians summed over one tick's requests (<= 0: what a quarter of
                                  the budget holds, between 64 Ki and 4 Mi) */
    int64_t max_tick_pixels;   /* pixels summed over one tick's requests (<= 0: 16 Mi) */
    size_t mem_budget_bytes;   /* device memory of the server (>= 1 MiB) */
} voge_server_config;

typedef struct {
    voge_camera cam;           /* the view to render */
    int32_t scene;             /* resident scene id (voge_server_add_scene), or -1: parameters below */
    int32_t N, C, K;           /* Gaussians, attribute channels (ignored for a resident scene), list
                                  length (K <= 32 once clipped to N) */
    float tau, thresh;         /* as voge_params */
    const float* means;        /* host [N][3] (inline scene only) */
    const float* inv_cov;      /* host [N][6] (inline scene only) */
    const float* attr;         /* host [N][C] (inline scene only) */
    const float* target;       /* host [H][W][C]: the image to match */
    float* image;              /* host [H][W][C] out, or NULL */
    float* grad_means;         /* host [N][3] out (dLoss/dmeans), or NULL */
    float* grad_inv_cov;       /* host [N][6] out, or NULL */
    float* grad_attr;          /* host [N][C] out, or NULL */
    float* grad_cam;           /* host [12] out: dLoss/dR (row-major), dLoss/dT, or NULL */
    float* loss;               /* host [1] out: mean squared error, or NULL */
} voge_request;

typedef struct {
    double submit_us, admit_us, start_us, done_us; /* server clock, microseconds */
    int32_t tick;              /* tick the request ran in */
    int32_t status;            /* VOGE_OK or the error that ended it */
} voge_request_timing;

typedef struct {
    int64_t submitted, completed, rejected, ticks, requests_in_ticks, graphs_captured, queued;
    int32_t resident, pad;
} voge_server_stats;

/* Create a server (allocates its device memory and starts its scheduler
 * thread).  VOGE_ERR_ARG for a bad config, VOGE_ERR_ADMISSION if the budget
 * cannot hold the tick workspaces, VOGE_ERR_CUDA on a CUDA failure. */
int voge_server_create(const voge_server_config* cfg, voge_server** out);

/* Queue a request (host descriptor copied; buffers referenced).  *ticket
 * identifies it.  VOGE_ERR_ADMISSION if it can never fit the server,
 * VOGE_ERR_BUSY if the queue is full, VOGE_ERR_UNSUPPORTED for lists longer
 * than 32, VOGE_ERR_ARG for invalid fields. */
int voge_server_submit(voge_server* s, const voge_request* req, uint64_t* ticket);

/* Wait until the request's outputs are in its host buffers.  timeout_ms < 0
 * waits without limit; on timeout returns VOGE_ERR_TIMEOUT and the ticket
 * stays valid.  Otherwise returns the request's status and retires the ticket;
 * `timing` (may be NULL) receives its timestamps. */
int voge_server_wait(voge_server* s, uint64_t ticket, int32_t timeout_ms, voge_request_timing* timing);

/* Copy a scene into the server's memory once; requests then name it by
 * *scene_id instead of sending its parameters.  Host arrays may be freed on
 * return.  VOGE_ERR_ADMISSION if it does not fit. */
int voge_server_add_scene(voge_server* s, int32_t N, int32_t C, const float* means, const float* inv_cov,
                          const float* attr, int32_t* scene_id);

/* Free a resident scene; VOGE_ERR_BUSY while a request that uses it is pending. */
int voge_server_remove_scene(voge_server* s, int32_t scene_id);

/* Hold (paused = 1) or release (0) the start of new ticks.  Admission and
 * input copies go on while held, so releasing starts one tick over every
 * request admitted meanwhile. */
int voge_server_pause(voge_server* s, int32_t paused);

/* Counters of the server (host memory). */
int voge_server_get_stats(voge_server* s, voge_server_stats* out);

/* Finish the queued work, stop the scheduler and free everything. */
int voge_server_destroy(voge_server* s);

/*
 * Forward render that allocates nothing and takes no workspace.  The paper
 * has no counterpart: this entry point exists for callers that cannot
 * allocate device memory where they render -- a real-time loop whose device
 * memory budget is fixed up front and must not grow, or a program that links
 * only this library and has no allocator of its own.
 *
 * It behaves as voge_render_fwd (same arguments and outputs, minus the
 * workspace) but uses a workspace of VOGE_STATIC_WORKSPACE_BYTES that lives
 * in the library: a device array that every GPU loading libvoge.so holds
 * until the process exits.
 *   - Returns VOGE_ERR_WORKSPACE, and launches nothing, if
 *     voge_workspace_bytes(cams, p) exceeds VOGE_STATIC_WORKSPACE_BYTES.
 *   - Each call looks up the array's device address on the current device
 *     (cudaGetSymbolAddress, which allocates nothing) and passes it on.
 *   - Every call on a device shares the one array, which keeps the previous
 *     call's contents (each call clears what must start at zero).  Calls whose
 *     work overlaps on the GPU -- for example on two streams -- race on it:
 *     order them on one stream or synchronise between them.
 *   - The caller still provides every input and output buffer (device).
 */
#define VOGE_STATIC_WORKSPACE_BYTES (32u << 20)
int voge_render_fwd_static(const voge_camera* cams, const voge_params* p, const float* means, const float* inv_cov,
                           const float* attr, float* image, float* weights, int32_t* index, voge_stream_t stream);

/*
 * One Adam step over `count` floats, in place (the optimiser of the paper's
 * shape fitting, Sec. 4.3):  m = b1 m + (1-b1) g,  v = b2 v + (1-b2) g^2,
 * param -= lr (m / (1 - b1^step)) / (sqrt(v / (1 - b2^step)) + eps).
 * All pointers device, [count] float; step >= 1 is the 1-based step number.
 * `grad` is set to zero after it is read, ready for the next accumulation by
 * voge_render_bwd.
 */
int voge_adam_step(float* param, float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                   float beta2, float eps, int32_t step, voge_stream_t stream);

/*
 * Kernel timing (tracing).  While enabled, every kernel launch of the library
 * is bracketed by two CUDA events on its stream.  voge_trace_read() waits for
 * the recorded events, adds their device time per kernel name into the
 * running totals, and copies up to max_entries totals into `out` (host
 * memory); it returns the number of distinct kernel names seen.
 * voge_trace_reset() zeroes the totals.  Do not enable while a stream is being
 * captured into a CUDA graph.  Not part of the paper: an aid for measurement.
 */
typedef struct {
    char name[48];
    int64_t launches;
    double total_ms;
} voge_trace_entry;

int voge_trace_enable(int on); /* returns the previous state */
int voge_trace_read(voge_trace_entry* out, int max_entries);
void voge_trace_reset(void);

/*
 * Measured arithmetic ceilings (an aid for measurement, not a paper step).
 * The render path runs on the FP32 and MUFU pipes: the pair term of Eq. 7 in
 * the forward pass and its adjoint in the backward pass.  This call measures,
 * on every SM of the current device, the rates of register-only loops:
 *   fma_tflops  FP32 fused multiply-add, 2 FLOP each, in TFLOP/s;
 *   ex2_tops    ex2.approx on the MUFU pipe, in 10^12 per second;
 *   fwd_gpairs  the forward pair term (u, erf by A&S 7.1.28 and the signed
 *               accumulation into A_k, exactly as the forward kernel does it),
 *               in 10^9 pairs per second, at the forward kernel's occupancy;
 *   bwd_gpairs  the backward pair adjoint (A&S 7.1.26 with e^{-u^2} and the
 *               four accumulations), in 10^9 pairs per second, at the backward
 *               kernel's occupancy;
 *   ms[4]       the timed launch of each, in milliseconds; sms the SM count.
 * Each loop runs once untimed and once timed between CUDA events on
 * `stream`, about 20 ms each; the call returns after the stream has finished
 * them.  Allocates nothing.  VOGE_ERR_ARG for a NULL `out`, VOGE_ERR_CUDA on a
 * CUDA failure.
 */
typedef struct {
    double fma_tflops, ex2_tops, fwd_gpairs, bwd_gpairs;
    double ms[4];
    int32_t sms, pad;
} voge_alu_peaks;

int voge_measure_alu_peaks(voge_alu_peaks* out, voge_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* VOGE_H */
