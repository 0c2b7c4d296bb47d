// voge_api.cu -- the C ABI of libvoge.so (declared in include/voge.h):
// argument checks, workspace layout and the launch sequence of one render.
#include <math.h>
#include <stddef.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "../../include/voge.h"
#include "voge_device.cuh"
#include "voge_trace.cuh"

namespace voge {
cudaError_t launch_project(int grid, int tiles, int count_tiles, cudaStream_t s, const Args& a);
cudaError_t launch_render_tiles(int KM, int nblocks, cudaStream_t s, const Args& a, int fine);
cudaError_t launch_fine(int KM, int total_tiles, int tile_h, int L, const void* index, cudaStream_t s,
                        const Args& a);
cudaError_t launch_backward_tiles(int KM, int nblocks, int with_wk, int kinds, cudaStream_t s, const Args& a);
cudaError_t launch_backward_packed(int KM, int nblocks, int live_tiles, cudaStream_t s, const Args& a);
cudaError_t launch_grad_finalize(int grid, int nviews, int N, int shared_scene, cudaStream_t s, const Args& a);
int render_blocks_per_sm(int KM, int fine);
cudaError_t launch_render_generic(int64_t total_pixels, cudaStream_t s, const Args& a);
cudaError_t launch_backward_generic(int64_t total_pixels, cudaStream_t s, const Args& a);
int backward_blocks_per_sm(int KM);

// Persistent tile launches: as many CTAs as can be resident at once (cached
// per device and variant), never more than there are tiles.  fwd: 0 the
// backward, 1 the fused forward, 2 the selection-only forward.
int tile_grid(int KM, int fwd, int total_tiles) {
    static std::mutex mu;
    static int cache[64][3][6];
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64) dev = 0;
    const int vi = KM == 8 ? 0 : KM == 16 ? 1 : KM == 20 ? 2 : KM == 24 ? 3 : KM == 32 ? 4 : 5;
    int g;
    {
        std::lock_guard<std::mutex> lk(mu);
        g = cache[dev][fwd][vi];
    }
    if (g == 0) {
        int nsm = 0;
        if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || nsm < 1) nsm = 1;
        g = nsm * (fwd ? render_blocks_per_sm(KM, fwd == 1) : backward_blocks_per_sm(KM));
        std::lock_guard<std::mutex> lk(mu);
        cache[dev][fwd][vi] = g;
    }
    return total_tiles < g ? total_tiles : g;
}
}  // namespace voge

using namespace voge;

namespace {

constexpr int kMaxRegisterList = 32;

int list_length(const voge_params* p) {
    if (p->N <= 0) return 0;
    return (p->K <= 0 || p->K >= p->N) ? p->N : p->K;
}

// Register-list capacity and tile height chosen for a list length.
void pick_variant(int L, int* KM, int* TH) {
    if (L <= 8) { *KM = 8; *TH = 16; }
    else if (L <= 16) { *KM = 16; *TH = 16; }
    else if (L <= 20) { *KM = 20; *TH = 16; }
    else if (L <= 24) { *KM = 24; *TH = 8; }
    else if (L <= kMaxRegisterList) { *KM = 32; *TH = 8; }
    else { *KM = 0; *TH = 16; }  // generic path
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

struct Layout {
    size_t desc, live_hdr, rec, rec2, tbox, tile_cnt, tile_off, tile_sub, tile_gauss, gcam, live, gkey, gid, total;
    int64_t pixels, bin_cap;
    int32_t total_tiles, TH, KM, L;
};

bool valid_params(const voge_camera* cams, const voge_params* p) {
    if (!cams || !p) return false;
    if (p->B < 1 || p->N < 0 || p->C < 1) return false;
    if (!(p->tau > 0.0f) || !isfinite(p->tau) || isnan(p->thresh)) return false;
    if (p->bin_capacity < 0) return false;
    for (int v = 0; v < p->B; ++v) {
        const voge_camera& c = cams[v];
        if (c.H < 1 || c.W < 1 || !(c.F > 0.0f) || !isfinite(c.F) || !isfinite(c.Ox) || !isfinite(c.Oy)) return false;
        for (int q = 0; q < 9; ++q)
            if (!isfinite(c.R[q])) return false;
        for (int q = 0; q < 3; ++q)
            if (!isfinite(c.T[q])) return false;
    }
    return true;
}

Layout make_layout(const voge_camera* cams, const voge_params* p) {
    Layout l;
    l.L = list_length(p);
    pick_variant(l.L, &l.KM, &l.TH);
    int64_t tiles = 0, pixels = 0;
    for (int v = 0; v < p->B; ++v) {
        const int tx = (cams[v].W + kTileW - 1) / kTileW, ty = (cams[v].H + l.TH - 1) / l.TH;
        tiles += (int64_t)tx * ty;
        pixels += (int64_t)cams[v].H * cams[v].W;
    }
    l.total_tiles = (int32_t)tiles;
    l.pixels = pixels;
    const int64_t BN = (int64_t)p->B * p->N;
    const int cap = p->bin_capacity > 0 ? p->bin_capacity : 8;
    l.bin_cap = BN * cap;
    if (l.bin_cap > (int64_t)INT32_MAX) l.bin_cap = INT32_MAX;
    size_t o = 0;
    l.live_hdr = o + sizeof(BatchHdr) + sizeof(ViewDesc) * p->B;
    l.desc = o; o = align256(o + sizeof(BatchHdr) + sizeof(ViewDesc) * p->B + sizeof(LiveHdr));
    l.rec = o; o = align256(o + 64 * (size_t)BN);
    l.rec2 = o; o = align256(o + 32 * (size_t)BN);
    l.tbox = o; o = align256(o + 16 * (size_t)BN);
    l.tile_cnt = o; o = align256(o + 4 * (size_t)(tiles + 1));
    l.tile_off = o; o = align256(o + 4 * (size_t)(tiles + 1));
    l.tile_sub = o; o = align256(o + 4 * (size_t)kTileSub * (size_t)(tiles + 1));
    l.tile_gauss = o; o = align256(o + 4 * (size_t)l.bin_cap);
    l.gcam = o; o = align256(o + 4 * kGcamStride * (size_t)BN);
    // packed backward's live row pairs: at most 4 row pairs x 2 backward tiles per tile
    l.live = o; o = align256(o + 8 * 8 * (size_t)(tiles + 1));
    if (l.KM == 0 && l.L > 0) {
        l.gkey = o; o = align256(o + 32 * (size_t)pixels * l.L);  // 8 floats per entry
        l.gid = o; o = align256(o + 4 * (size_t)pixels * l.L);
    } else {
        l.gkey = l.gid = o;
    }
    l.total = o + 256;
    return l;
}

Ws make_ws(const Layout& l, void* base) {
    char* b = static_cast<char*>(base);
    Ws w;
    w.rec = reinterpret_cast<float4*>(b + l.rec);
    w.rec2 = reinterpret_cast<float4*>(b + l.rec2);
    w.tbox = reinterpret_cast<int4*>(b + l.tbox);
    w.tile_cnt = reinterpret_cast<int32_t*>(b + l.tile_cnt);
    w.tile_off = reinterpret_cast<int32_t*>(b + l.tile_off);
    w.tile_sub = reinterpret_cast<int32_t*>(b + l.tile_sub);
    w.tile_gauss = reinterpret_cast<int32_t*>(b + l.tile_gauss);
    w.bin_cap = l.bin_cap;
    w.gcam = reinterpret_cast<float*>(b + l.gcam);
    w.live = reinterpret_cast<int2*>(b + l.live);
    w.live_hdr = reinterpret_cast<LiveHdr*>(b + l.live_hdr);
    w.gkey = reinterpret_cast<float*>(b + l.gkey);
    w.gid = reinterpret_cast<int32_t*>(b + l.gid);
    w.gen_L = l.L;
    return w;
}

struct Buffers {
    const float *means, *inv_cov, *attr;
    float *image, *weights;
    int32_t* index;
    const int32_t* index_in;
    const float* weights_in;
    const float* grad_image;
    float *grad_means, *grad_inv_cov, *grad_attr, *grad_cam;
    const int32_t* live_for;  // the lists whose live row pairs this call records (null: none)
};

// View table of a render call: every view shares the scene; outputs are
// laid out view after view.
void build_views(const voge_camera* cams, const voge_params* p, const Layout& l, const Buffers& b,
                 std::vector<unsigned char>& blob) {
    blob.assign(sizeof(BatchHdr) + sizeof(ViewDesc) * p->B + sizeof(LiveHdr), 0);
    BatchHdr* h = reinterpret_cast<BatchHdr*>(blob.data());
    ViewDesc* vd = reinterpret_cast<ViewDesc*>(blob.data() + sizeof(BatchHdr));
    LiveHdr* lh = reinterpret_cast<LiveHdr*>(blob.data() + sizeof(BatchHdr) + sizeof(ViewDesc) * p->B);
    lh->index_fwd = b.live_for;
    const int use_thresh = p->thresh > 0.0f ? 1 : 0;
    const float Qeta = use_thresh ? (p->thresh >= 1.0f ? 0.0f : (float)(2.0 * log(1.0 / (double)p->thresh))) : INFINITY;
    int32_t tile_base = 0;
    int64_t pix_base = 0;
    for (int v = 0; v < p->B; ++v) {
        ViewDesc& d = vd[v];
        memcpy(d.R, cams[v].R, sizeof(d.R));
        memcpy(d.T, cams[v].T, sizeof(d.T));
        d.F = cams[v].F;
        d.Ox = cams[v].Ox;
        d.Oy = cams[v].Oy;
        d.invF = (float)(1.0 / (double)cams[v].F);
        d.H = cams[v].H;
        d.W = cams[v].W;
        d.tiles_x = (cams[v].W + kTileW - 1) / kTileW;
        d.tiles_y = (cams[v].H + l.TH - 1) / l.TH;
        d.tile_h = l.TH;
        d.tile_base = tile_base;
        d.N = p->N;
        d.C = p->C;
        d.L = l.L;
        d.use_thresh = use_thresh;
        d.plain = (p->flags & VOGE_FLAG_PLAIN) ? 1 : 0;
        d.tau = p->tau;
        d.Qeta = Qeta;
        d.rec_base = (int64_t)v * p->N;
        d.pix_base = pix_base;
        d.elem_base = pix_base * p->C;
        d.means = b.means;
        d.inv_cov = b.inv_cov;
        d.attr = b.attr;
        d.image = b.image ? b.image + pix_base * p->C : nullptr;
        d.weights = b.weights ? b.weights + pix_base * l.L : nullptr;
        d.index = b.index ? b.index + pix_base * l.L : nullptr;
        d.index_in = b.index_in ? b.index_in + pix_base * l.L : nullptr;
        d.weights_in = b.weights_in ? b.weights_in + pix_base * l.L : nullptr;
        d.grad_image = b.grad_image ? b.grad_image + pix_base * p->C : nullptr;
        d.grad_means = b.grad_means;
        d.grad_inv_cov = b.grad_inv_cov;
        d.grad_attr = b.grad_attr;
        d.grad_cam = b.grad_cam ? b.grad_cam + 12 * v : nullptr;
        tile_base += d.tiles_x * d.tiles_y;
        pix_base += (int64_t)cams[v].H * cams[v].W;
    }
    h->total_records = (int64_t)p->B * p->N;
    h->total_elems = pix_base * p->C;
    h->total_tiles = tile_base;
    h->nviews = p->B;
    h->class_begin[0] = 0;
    h->class_end[0] = tile_base;
    h->shared_scene = 1;
}

Args make_args(const Layout& l, void* ws) {
    Args a;
    memset(&a, 0, sizeof(a));
    char* b = static_cast<char*>(ws);
    a.hdr = reinterpret_cast<BatchHdr*>(b + l.desc);
    a.views = reinterpret_cast<const ViewDesc*>(b + l.desc + sizeof(BatchHdr));
    a.ws = make_ws(l, ws);
    a.cls = 0;
    return a;
}

#ifdef VOGE_CHECKED
// Checked builds: wait for the call's kernels and report a failed index check
// (the first failing site is in the call header).
int finish_call(const Args& a, cudaStream_t s, int rc) {
    if (rc != VOGE_OK) return rc;
    int32_t site = 0;
    if (cudaMemcpyAsync(&site, &a.hdr->check_site, sizeof(site), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return VOGE_ERR_CUDA;
    return site ? VOGE_ERR_CHECK : VOGE_OK;
}
#else
inline int finish_call(const Args&, cudaStream_t, int rc) { return rc; }
#endif

int record_grid(int64_t records) {
    int64_t g = (records + 255) / 256;
    if (g > 152 * 16) g = 152 * 16;
    return (int)(g < 1 ? 1 : g);
}

// Upload the view table and header, project every (view, Gaussian); with
// `bin` also build the tile lists.
int upload_and_project(const voge_camera* cams, const voge_params* p, const Layout& l, const Args& a,
                       const Buffers& b, int project, int bin, cudaStream_t s) {
    std::vector<unsigned char> blob;
    build_views(cams, p, l, b, blob);
    // a call that reuses the forward's projection keeps its record of live
    // row pairs (the blob's tail) as well
    const size_t bytes = blob.size() - (project ? 0 : sizeof(LiveHdr));
    if (cudaMemcpyAsync(a.hdr, blob.data(), bytes, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return VOGE_ERR_CUDA;
    if (!project) return VOGE_OK;
    const int count_tiles = bin && !(p->flags & VOGE_FLAG_PLAIN);
    if (count_tiles && cudaMemsetAsync(a.ws.tile_sub, 0, 4 * (size_t)kTileSub * (size_t)(l.total_tiles + 1), s) != cudaSuccess)
        return VOGE_ERR_CUDA;
    return launch_project(record_grid((int64_t)p->B * p->N), l.total_tiles, count_tiles, s, a) == cudaSuccess ? VOGE_OK
                                                                                                : VOGE_ERR_CUDA;
}

__global__ void k_pose_grad(const float* pose, const float* gcam, float* gpose, int B) {
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= B) return;
    const float az = pose[4 * v], el = pose[4 * v + 1], ro = pose[4 * v + 3];
    float sa, ca, se, ce, sr, cr;
    sincosf(az, &sa, &ca);
    sincosf(el, &se, &ce);
    sincosf(ro, &sr, &cr);
    // R = Rz(roll) R0(az, el), rows of R0: right, down, forward; T = (0, 0, dist)
    const float rt[3] = {ca, 0.f, -sa}, dn[3] = {se * sa, -ce, se * ca};
    const float drt_a[3] = {-sa, 0.f, -ca};
    const float ddn_a[3] = {se * ca, 0.f, -se * sa}, ddn_e[3] = {ce * sa, se, ce * ca};
    const float dfw_a[3] = {-ce * ca, 0.f, ce * sa}, dfw_e[3] = {se * sa, -ce, se * ca};
    const float* g = gcam + 12 * v;
    float ga = 0.f, ge = 0.f, gr = 0.f;
    for (int q = 0; q < 3; ++q) {
        // row0 = cr rt - sr dn ; row1 = sr rt + cr dn ; row2 = fw
        ga += g[q] * (cr * drt_a[q] - sr * ddn_a[q]) + g[3 + q] * (sr * drt_a[q] + cr * ddn_a[q]) + g[6 + q] * dfw_a[q];
        ge += g[q] * (-sr * ddn_e[q]) + g[3 + q] * (cr * ddn_e[q]) + g[6 + q] * dfw_e[q];
        gr += g[q] * (-sr * rt[q] - cr * dn[q]) + g[3 + q] * (cr * rt[q] - sr * dn[q]);
    }
    gpose[4 * v + 0] += ga;
    gpose[4 * v + 1] += ge;
    gpose[4 * v + 2] += g[11];
    gpose[4 * v + 3] += gr;
}

__global__ void __launch_bounds__(256) k_mse(const float* x, const float* y, int64_t n, float* gx, float* loss) {
    __shared__ float red[8];
    const float inv = 1.0f / (float)n;
    float acc = 0.0f;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool v4 = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(gx)) & 15) == 0;
    int64_t done = 0;
    if (v4) {  // 16-byte rows of four elements, then the tail
        const int64_t n4 = n >> 2;
        for (int64_t q = first; q < n4; q += stride) {
            const float4 a = __ldg(reinterpret_cast<const float4*>(x) + q), b = __ldg(reinterpret_cast<const float4*>(y) + q);
            const float4 d = make_float4(a.x - b.x, a.y - b.y, a.z - b.z, a.w - b.w);
            acc = fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, fmaf(d.w, d.w, acc))));
            reinterpret_cast<float4*>(gx)[q] = make_float4(2.0f * d.x * inv, 2.0f * d.y * inv, 2.0f * d.z * inv, 2.0f * d.w * inv);
        }
        done = n4 << 2;
    }
    for (int64_t q = done + first; q < n; q += stride) {
        const float d = x[q] - y[q];
        acc = fmaf(d, d, acc);
        gx[q] = 2.0f * d * inv;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        float s = 0.0f;
        for (int w = 0; w < 8; ++w) s += red[w];
        atomicAdd(loss, s * inv);
    }
}

// One Adam step (Kingma & Ba 2015) over n parameters, bias-corrected with
// the 1-based step count; the gradient is zeroed once read.
__device__ __forceinline__ void adam_one(float& x, float& g, float& m, float& v, float lr, float b1, float b2,
                                         float eps, float c1, float c2) {
    const float gq = g;
    g = 0.0f;  // consumed: ready for the next accumulation
    m = fmaf(b1, m - gq, gq);
    v = fmaf(b2, v - gq * gq, gq * gq);
    x -= lr * (m * c1) / (sqrtf(v * c2) + eps);
}

__global__ void __launch_bounds__(256) k_adam(float* x, float* g, float* m, float* v, int64_t n, float lr,
                                              float b1, float b2, float eps, float c1, float c2) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool v4 = ((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(g) | reinterpret_cast<uintptr_t>(m) |
                      reinterpret_cast<uintptr_t>(v)) & 15) == 0;
    int64_t done = 0;
    if (v4) {  // four parameters per thread and step, then the tail
        const int64_t n4 = n >> 2;
        for (int64_t q = first; q < n4; q += stride) {
            float4 xq = reinterpret_cast<float4*>(x)[q], gq = reinterpret_cast<float4*>(g)[q];
            float4 mq = reinterpret_cast<float4*>(m)[q], vq = reinterpret_cast<float4*>(v)[q];
            adam_one(xq.x, gq.x, mq.x, vq.x, lr, b1, b2, eps, c1, c2);
            adam_one(xq.y, gq.y, mq.y, vq.y, lr, b1, b2, eps, c1, c2);
            adam_one(xq.z, gq.z, mq.z, vq.z, lr, b1, b2, eps, c1, c2);
            adam_one(xq.w, gq.w, mq.w, vq.w, lr, b1, b2, eps, c1, c2);
            reinterpret_cast<float4*>(x)[q] = xq;
            reinterpret_cast<float4*>(g)[q] = gq;
            reinterpret_cast<float4*>(m)[q] = mq;
            reinterpret_cast<float4*>(v)[q] = vq;
        }
        done = n4 << 2;
    }
    for (int64_t q = done + first; q < n; q += stride) adam_one(x[q], g[q], m[q], v[q], lr, b1, b2, eps, c1, c2);
}

}  // namespace

extern "C" {

int voge_version(void) { return 100; }

const char* voge_strerror(int code) {
    switch (code) {
        case VOGE_OK: return "ok";
        case VOGE_ERR_ARG: return "invalid argument";
        case VOGE_ERR_WORKSPACE: return "workspace missing or too small";
        case VOGE_ERR_CUDA: return "CUDA call or kernel launch failed";
        case VOGE_ERR_UNSUPPORTED: return "unsupported combination";
        case VOGE_ERR_TIMEOUT: return "bounded wait ran out";
        case VOGE_ERR_ADMISSION: return "request exceeds the memory budget";
        case VOGE_ERR_BUSY: return "no free slot";
        case VOGE_ERR_CHECK: return "checked build: a kernel caught an out-of-range index";
        default: return "unknown error";
    }
}

int voge_list_length(const voge_params* p) { return p ? list_length(p) : 0; }

size_t voge_workspace_bytes(const voge_camera* cams, const voge_params* p) {
    if (!valid_params(cams, p)) return 0;
    return make_layout(cams, p).total;
}

int voge_render_fwd(const voge_camera* cams, const voge_params* p, const float* means, const float* inv_cov,
                    const float* attr, float* image, float* weights, int32_t* index, void* workspace,
                    size_t workspace_bytes, voge_stream_t stream_) {
    if (!valid_params(cams, p) || !image) return VOGE_ERR_ARG;
    if (p->N > 0 && (!means || !inv_cov || !attr || !index)) return VOGE_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    const Layout l = make_layout(cams, p);
    if (!workspace || workspace_bytes < l.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return VOGE_ERR_WORKSPACE;
    if (p->N == 0) {
        return cudaMemsetAsync(image, 0, sizeof(float) * (size_t)l.pixels * p->C, s) == cudaSuccess ? VOGE_OK
                                                                                                    : VOGE_ERR_CUDA;
    }
    const Args a = make_args(l, workspace);
    Buffers b;
    memset(&b, 0, sizeof(b));
    b.means = means;
    b.inv_cov = inv_cov;
    b.attr = attr;
    b.image = image;
    b.weights = weights;
    b.index = index;
    if (l.KM > 0) b.live_for = index;  // the tile kernels record the row pairs that keep an entry
    const bool split = (p->flags & VOGE_FLAG_SPLIT_FORWARD) && l.KM != 0;
    if (split) b.index_in = index;  // the fine kernel reads the lists the selection kernel wrote
    int rc = upload_and_project(cams, p, l, a, b, 1, 1, s);
    if (rc != VOGE_OK) return rc;
    if (l.total_tiles == 0) return VOGE_OK;
    cudaError_t e;
    if (l.KM == 0) {
        e = launch_render_generic(l.pixels, s, a);
    } else if (!split) {
        e = launch_render_tiles(l.KM, tile_grid(l.KM, 1, l.total_tiles), s, a, 1);
    } else {
        e = launch_render_tiles(l.KM, tile_grid(l.KM, 2, l.total_tiles), s, a, 0);
        if (e == cudaSuccess) e = launch_fine(l.KM, l.total_tiles, l.TH, l.L, index, s, a);
    }
    return finish_call(a, s, e == cudaSuccess ? VOGE_OK : VOGE_ERR_CUDA);
}

int voge_render_fine(const voge_camera* cams, const voge_params* p, const float* means, const float* inv_cov,
                     const float* attr, const int32_t* index, float* image, float* weights, void* workspace,
                     size_t workspace_bytes, voge_stream_t stream_) {
    if (!valid_params(cams, p) || !image) return VOGE_ERR_ARG;
    if (p->N > 0 && (!means || !inv_cov || !attr || !index)) return VOGE_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    const Layout l = make_layout(cams, p);
    if (!workspace || workspace_bytes < l.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return VOGE_ERR_WORKSPACE;
    if (p->N == 0) {
        if (weights && l.L > 0 &&
            cudaMemsetAsync(weights, 0, sizeof(float) * (size_t)l.pixels * l.L, s) != cudaSuccess)
            return VOGE_ERR_CUDA;
        return cudaMemsetAsync(image, 0, sizeof(float) * (size_t)l.pixels * p->C, s) == cudaSuccess ? VOGE_OK
                                                                                                    : VOGE_ERR_CUDA;
    }
    if (l.KM == 0) return VOGE_ERR_UNSUPPORTED;  // lists longer than 32
    const Args a = make_args(l, workspace);
    Buffers b;
    memset(&b, 0, sizeof(b));
    b.means = means;
    b.inv_cov = inv_cov;
    b.attr = attr;
    b.image = image;
    b.weights = weights;
    b.index_in = index;
    int rc = upload_and_project(cams, p, l, a, b, 1, 0, s);
    if (rc != VOGE_OK) return rc;
    return finish_call(a, s, launch_fine(l.KM, l.total_tiles, l.TH, l.L, index, s, a) == cudaSuccess ? VOGE_OK
                                                                                                   : VOGE_ERR_CUDA);
}

int voge_render_bwd(const voge_camera* cams, const voge_params* p, const float* means, const float* inv_cov,
                    const float* attr, const int32_t* index, const float* grad_image, float* grad_means,
                    float* grad_inv_cov, float* grad_attr, float* grad_cam, void* workspace, size_t workspace_bytes,
                    voge_stream_t stream_) {
    return voge_render_bwd_w(cams, p, means, inv_cov, attr, index, nullptr, grad_image, grad_means, grad_inv_cov,
                             grad_attr, grad_cam, workspace, workspace_bytes, stream_);
}

int voge_render_bwd_w(const voge_camera* cams, const voge_params* p, const float* means, const float* inv_cov,
                      const float* attr, const int32_t* index, const float* weights, const float* grad_image,
                      float* grad_means, float* grad_inv_cov, float* grad_attr, float* grad_cam, void* workspace,
                      size_t workspace_bytes, voge_stream_t stream_) {
    if (!valid_params(cams, p) || !grad_image) return VOGE_ERR_ARG;
    if (p->N == 0) return VOGE_OK;
    if (!means || !inv_cov || !attr || !index) return VOGE_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    const Layout l = make_layout(cams, p);
    if (!workspace || workspace_bytes < l.total || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return VOGE_ERR_WORKSPACE;
    const Args a = make_args(l, workspace);
    Buffers b;
    memset(&b, 0, sizeof(b));
    b.means = means;
    b.inv_cov = inv_cov;
    b.attr = attr;
    b.index_in = index;
    b.weights_in = weights;
    b.grad_image = grad_image;
    b.grad_means = grad_means;
    b.grad_inv_cov = grad_inv_cov;
    b.grad_attr = grad_attr;
    b.grad_cam = grad_cam;
    const int project = (p->flags & VOGE_FLAG_REUSE_PROJECTION) ? 0 : 1;
    // the packed form works through the row pairs that keep an entry: from the
    // forward's record when the projection (and so the record) is reused,
    // else found here by k_live_units
    const bool packed = weights && p->C <= 3 && l.KM > 0 && l.KM <= 20;
    if (packed && project) b.live_for = index;
    int rc = upload_and_project(cams, p, l, a, b, project, 0, s);
    if (rc != VOGE_OK) return rc;
    if (cudaMemsetAsync(a.ws.gcam, 0, 4 * kGcamStride * (size_t)p->B * p->N, s) != cudaSuccess) return VOGE_ERR_CUDA;
    if (l.total_tiles > 0) {
        const cudaError_t e =
            l.KM == 0 ? launch_backward_generic(l.pixels, s, a)
            : packed  ? launch_backward_packed(l.KM, tile_grid(l.KM, 0, 2 * l.total_tiles), project ? l.total_tiles : 0,
                                               s, a)
                      : launch_backward_tiles(l.KM, tile_grid(l.KM, 0, l.total_tiles), weights ? 0 : 1,
                                              p->C >= 8 ? 2 : 1, s, a);
        if (e != cudaSuccess) return VOGE_ERR_CUDA;
    }
    // the finalize also folds in attribute gradients of up to three channels
    if ((grad_means || grad_inv_cov || grad_cam || grad_attr) &&
        launch_grad_finalize(record_grid(p->N), p->B, p->N, 1, s, a) != cudaSuccess)
        return VOGE_ERR_CUDA;
    return finish_call(a, s, VOGE_OK);
}

int voge_render_stats(const void* workspace, voge_render_stats_t* out, voge_stream_t stream_) {
    if (!workspace || !out || (reinterpret_cast<uintptr_t>(workspace) & 255)) return VOGE_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    unsigned long long c[3] = {0, 0, 0};
    // the call header sits at the start of every workspace layout
    const char* h = static_cast<const char*>(workspace) + offsetof(BatchHdr, traces);
    if (cudaMemcpyAsync(c, h, sizeof(c), cudaMemcpyDeviceToHost, s) != cudaSuccess) return VOGE_ERR_CUDA;
    if (cudaStreamSynchronize(s) != cudaSuccess) return VOGE_ERR_CUDA;
    out->traces = (int64_t)c[0];
    out->entries = (int64_t)c[1];
    out->pairs = (int64_t)c[2];
    return VOGE_OK;
}

void voge_pose_to_RT(const double pose[4], float R[9], float T[3]) {
    const double sa = sin(pose[0]), ca = cos(pose[0]), se = sin(pose[1]), ce = cos(pose[1]);
    const double sr = sin(pose[3]), cr = cos(pose[3]);
    const double rt[3] = {ca, 0.0, -sa}, dn[3] = {se * sa, -ce, se * ca}, fw[3] = {-ce * sa, -se, -ce * ca};
    for (int q = 0; q < 3; ++q) {
        R[q] = (float)(cr * rt[q] - sr * dn[q]);
        R[3 + q] = (float)(sr * rt[q] + cr * dn[q]);
        R[6 + q] = (float)fw[q];
    }
    T[0] = 0.0f;
    T[1] = 0.0f;
    T[2] = (float)pose[2];
}

int voge_pose_grad(const float* pose, const float* grad_cam, float* grad_pose, int32_t B, voge_stream_t stream_) {
    if (B < 0 || (B > 0 && (!pose || !grad_cam || !grad_pose))) return VOGE_ERR_ARG;
    if (B == 0) return VOGE_OK;
    TraceScope tr("k_pose_grad", reinterpret_cast<cudaStream_t>(stream_));
    k_pose_grad<<<(B + 127) / 128, 128, 0, reinterpret_cast<cudaStream_t>(stream_)>>>(pose, grad_cam, grad_pose, B);
    return cudaPeekAtLastError() == cudaSuccess ? VOGE_OK : VOGE_ERR_CUDA;
}

int voge_mse_grad(const float* image, const float* target, int64_t count, float* grad_image, float* loss,
                  voge_stream_t stream_) {
    if (count < 0 || (count > 0 && (!image || !target || !grad_image || !loss))) return VOGE_ERR_ARG;
    if (count == 0) return VOGE_OK;
    int64_t nb = (count + 255) / 256;
    if (nb > 152 * 8) nb = 152 * 8;
    TraceScope tr("k_mse", reinterpret_cast<cudaStream_t>(stream_));
    k_mse<<<(unsigned)nb, 256, 0, reinterpret_cast<cudaStream_t>(stream_)>>>(image, target, count, grad_image, loss);
    return cudaPeekAtLastError() == cudaSuccess ? VOGE_OK : VOGE_ERR_CUDA;
}

int voge_adam_step(float* param, float* grad, float* m, float* v, int64_t count, float lr, float beta1,
                   float beta2, float eps, int32_t step, voge_stream_t stream_) {
    if (count < 0 || step < 1 || (count > 0 && (!param || !grad || !m || !v))) return VOGE_ERR_ARG;
    if (count == 0) return VOGE_OK;
    const float c1 = (float)(1.0 / (1.0 - pow((double)beta1, (double)step)));
    const float c2 = (float)(1.0 / (1.0 - pow((double)beta2, (double)step)));
    int64_t nb = (count + 255) / 256;
    if (nb > 152 * 8) nb = 152 * 8;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    TraceScope tr("k_adam", s);
    k_adam<<<(unsigned)nb, 256, 0, s>>>(param, grad, m, v, count, lr, beta1, beta2, eps, c1, c2);
    return cudaPeekAtLastError() == cudaSuccess ? VOGE_OK : VOGE_ERR_CUDA;
}

}  // extern "C"
