// voge_serve.cu -- render-and-compare serving with continuous batching.
//
// A request is one analysis-by-synthesis step on its own scene: render one
// view (forward pass of Sec. 3.3 / Eq. 6-8), compare with a target image
// (mean squared error) and return the image, the loss and the gradients of
// the scene and camera (backward pass).  The server keeps admitted requests'
// inputs, outputs and K-lists resident in one device arena and runs them in
// ticks: every request whose inputs are on the device when a tick starts joins
// it, and the tick runs one persistent launch per list-capacity class over all
// of its requests (projection, binning, coarse + fine forward, loss, adjoint,
// gradient finalisation).  Requests that arrive while a tick runs are admitted
// as slots and arena space free up and join the next tick; their host-to-device
// copies overlap the running tick.  With graphs on, each tick is the replay of
// a CUDA graph captured once per set of classes present.
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/voge.h"
#include "voge_device.cuh"
#include "voge_trace.cuh"

namespace voge {
cudaError_t launch_project(int grid, int tiles, int count_tiles, cudaStream_t s, const Args& a);
cudaError_t launch_render_tiles(int KM, int nblocks, cudaStream_t s, const Args& a, int fine);
cudaError_t launch_backward_tiles(int KM, int nblocks, int with_wk, int kinds, cudaStream_t s, const Args& a);
cudaError_t launch_grad_finalize(int grid, int nviews, int N, int shared_scene, cudaStream_t s, const Args& a);
int tile_grid(int KM, int fwd, int total_tiles);

// Loss helper over a batch: per view, grad_image = 2 (image - target) / n and
// loss += sum (image - target)^2 / n with n = H W C of that view.
__global__ void __launch_bounds__(256) k_mse_batch(Args a) {
    // One view after another; within a view the blocks stride over its
    // image in 16-byte vectors (scalar when the view's arrays are not
    // aligned), and each block adds its share of the view's loss once.
    __shared__ float red[8];
    const int nv = a.hdr->nviews;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t first = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (int v = 0; v < nv; ++v) {
        const ViewDesc& vd = a.views[v];
        const int64_t n = (int64_t)vd.H * vd.W * vd.C;
        const float inv = 1.0f / (float)n;
        const float* x = vd.image;
        const float* y = vd.target;
        float* gx = const_cast<float*>(vd.grad_image);
        float acc = 0.0f;
        int64_t done = 0;
        if (((reinterpret_cast<uintptr_t>(x) | reinterpret_cast<uintptr_t>(y) | reinterpret_cast<uintptr_t>(gx)) & 15) == 0) {
            const int64_t n4 = n >> 2;
            for (int64_t q = first; q < n4; q += stride) {
                const float4 p = reinterpret_cast<const float4*>(x)[q];
                const float4 t = __ldg(reinterpret_cast<const float4*>(y) + q);
                const float4 d = make_float4(p.x - t.x, p.y - t.y, p.z - t.z, p.w - t.w);
                acc = fmaf(d.x, d.x, fmaf(d.y, d.y, fmaf(d.z, d.z, fmaf(d.w, d.w, acc))));
                reinterpret_cast<float4*>(gx)[q] =
                    make_float4(2.0f * d.x * inv, 2.0f * d.y * inv, 2.0f * d.z * inv, 2.0f * d.w * inv);
            }
            done = n4 << 2;
        }
        for (int64_t q = done + first; q < n; q += stride) {
            const float d = x[q] - __ldg(y + q);
            acc = fmaf(d, d, acc);
            gx[q] = 2.0f * d * inv;
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        if (lane == 0) red[wid] = acc;
        __syncthreads();
        if (threadIdx.x == 0 && vd.loss) {
            float sum = 0.0f;
            for (int w = 0; w < (int)(blockDim.x >> 5); ++w) sum += red[w];
            atomicAdd(vd.loss, sum * inv);
        }
        __syncthreads();  // red is reused by the next view
    }
}
}  // namespace voge

using namespace voge;

namespace {

using Clock = std::chrono::steady_clock;

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// First-fit allocator over one device buffer (offsets only).
class Arena {
   public:
    void init(size_t bytes) {
        free_.clear();
        free_[0] = bytes;
        size_ = bytes;
    }
    bool alloc(size_t bytes, size_t* off) {
        bytes = up256(bytes);
        for (auto it = free_.begin(); it != free_.end(); ++it) {
            if (it->second >= bytes) {
                *off = it->first;
                const size_t rest = it->second - bytes, start = it->first + bytes;
                free_.erase(it);
                if (rest) free_[start] = rest;
                return true;
            }
        }
        return false;
    }
    void release(size_t off, size_t bytes) {
        bytes = up256(bytes);
        auto it = free_.emplace(off, bytes).first;
        auto nx = std::next(it);
        if (nx != free_.end() && it->first + it->second == nx->first) {
            it->second += nx->second;
            free_.erase(nx);
        }
        if (it != free_.begin()) {
            auto pv = std::prev(it);
            if (pv->first + pv->second == it->first) {
                pv->second += it->second;
                free_.erase(it);
            }
        }
    }
   private:
    std::map<size_t, size_t> free_;
    size_t size_ = 0;
};

int list_len(int K, int N) { return N <= 0 ? 0 : ((K <= 0 || K >= N) ? N : K); }

// capacity class of a list length: 0..4 register lists 8/16/20/24/32, 5 generic
int class_of(int L) {
    if (L <= 8) return 0;
    if (L <= 16) return 1;
    if (L <= 20) return 2;
    if (L <= 24) return 3;
    if (L <= 32) return 4;
    return 5;
}
const int kClassKM[6] = {8, 16, 20, 24, 32, 0};
const int kClassTH[6] = {16, 16, 16, 8, 8, 16};
constexpr int kClasses = 6;

struct Scene {
    int32_t N = 0, C = 0;
    size_t off = 0, bytes = 0;
    float *means = nullptr, *inv_cov = nullptr, *attr = nullptr;
    int users = 0;  // requests that reference it and have not finished
};

struct Req {
    uint64_t ticket;
    Scene* scene = nullptr;  // resident scene, or null for inline parameters
    voge_request r;
    int L = 0, cls = 0;
    int64_t pixels = 0;
    size_t off = 0, bytes = 0;  // arena block
    // device pointers inside the block
    float *means, *inv_cov, *attr, *target, *image, *grad_image, *weights, *gmeans, *ginv, *gattr, *gcam, *loss;
    int32_t* index;
    cudaEvent_t ready = nullptr;
    int state = 0;  // 0 queued, 1 admitted (copying), 2 in a tick, 3 done
    int status = VOGE_OK;
    int tick = -1;
    double t_submit = 0, t_admit = 0, t_start = 0, t_done = 0;
};

struct TickSlot {
    void* ws = nullptr;  // device: [hdr | views] | records ... (fixed layout)
    size_t desc_bytes = 0;
    unsigned char* host_desc = nullptr;  // pinned mirror of [hdr | views]
    Args args;
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    std::vector<Req*> reqs;
    bool busy = false;
    int id = 0;
    std::unordered_map<uint32_t, cudaGraphExec_t> graphs;  // per class-set
};

}  // namespace

struct voge_server {
    voge_server_config cfg;
    int device = 0;
    void* arena_base = nullptr;
    Arena arena;
    cudaStream_t copy_stream = nullptr;
    std::vector<TickSlot> slots;
    int64_t max_records = 0, max_tiles = 0, max_elems = 0;
    int max_views = 0;
    int grid_records = 0;
    size_t ws_rec = 0, ws_rec2 = 0, ws_tbox = 0, ws_cnt = 0, ws_off = 0, ws_sub = 0, ws_gauss = 0, ws_gcam = 0;
    int64_t bin_cap = 0;
    size_t request_capacity = 0;  // arena bytes left for requests

    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<Req*> queue;         // submitted, not admitted
    std::vector<Req*> admitted;     // admitted, not yet in a tick
    std::unordered_map<uint64_t, Req*> all;
    std::unordered_map<int32_t, Scene*> scenes;
    int32_t next_scene = 0;
    uint64_t next_ticket = 1;
    int resident = 0;
    bool stop = false;
    bool paused = false;
    std::thread worker;
    Clock::time_point t0;
    voge_server_stats st;
    int tick_counter = 0;

    double now_us() const { return std::chrono::duration<double, std::micro>(Clock::now() - t0).count(); }
};

namespace {

size_t request_bytes(const voge_request& r, int L, bool resident) {
    const int64_t P = (int64_t)r.cam.H * r.cam.W;
    const size_t N = (size_t)r.N, C = (size_t)r.C;
    size_t b = 0;
    if (!resident) b += up256(4 * 3 * N) + up256(4 * 6 * N) + up256(4 * C * N);  // means, inv_cov, attr
    b += 3 * up256(4 * (size_t)P * C);                             // target, image, grad_image
    b += 2 * up256(4 * (size_t)P * std::max(L, 1));                // weights, index
    b += up256(4 * 3 * N) + up256(4 * 6 * N) + up256(4 * C * N);  // gradients
    b += up256(4 * 16);                                            // grad_cam (12) + loss
    return b;
}

void carve(Req* q, char* base) {
    const int64_t P = q->pixels;
    const size_t N = (size_t)q->r.N, C = (size_t)q->r.C, L = (size_t)std::max(q->L, 1);
    char* p = base + q->off;
    auto take = [&](size_t bytes) {
        char* x = p;
        p += up256(bytes);
        return x;
    };
    if (q->scene) {
        q->means = q->scene->means;
        q->inv_cov = q->scene->inv_cov;
        q->attr = q->scene->attr;
    } else {
        q->means = (float*)take(4 * 3 * N);
        q->inv_cov = (float*)take(4 * 6 * N);
        q->attr = (float*)take(4 * C * N);
    }
    q->target = (float*)take(4 * (size_t)P * C);
    q->image = (float*)take(4 * (size_t)P * C);
    q->grad_image = (float*)take(4 * (size_t)P * C);
    q->weights = (float*)take(4 * (size_t)P * L);
    q->index = (int32_t*)take(4 * (size_t)P * L);
    q->gmeans = (float*)take(4 * 3 * N);
    q->ginv = (float*)take(4 * 6 * N);
    q->gattr = (float*)take(4 * C * N);
    q->gcam = (float*)take(4 * 16);
    q->loss = q->gcam + 12;
}

bool valid_request(const voge_request* r) {
    if (!r || !(r->tau > 0.0f) || isnan(r->thresh) || !r->target) return false;
    if (r->scene < 0 && (r->N < 1 || r->C < 1 || !r->means || !r->inv_cov || !r->attr)) return false;
    const voge_camera& c = r->cam;
    if (c.H < 1 || c.W < 1 || !(c.F > 0.0f) || !isfinite(c.F)) return false;
    return true;
}

// Build the tick's view table (views sorted by class) into the slot's pinned
// mirror; returns the class-set bit mask.
uint32_t build_tick(voge_server* S, TickSlot& ts) {
    std::sort(ts.reqs.begin(), ts.reqs.end(), [](const Req* x, const Req* y) {
        return x->cls != y->cls ? x->cls < y->cls : x->ticket < y->ticket;
    });
    memset(ts.host_desc, 0, ts.desc_bytes);
    BatchHdr* h = reinterpret_cast<BatchHdr*>(ts.host_desc);
    ViewDesc* vd = reinterpret_cast<ViewDesc*>(ts.host_desc + sizeof(BatchHdr));
    int32_t tile_base = 0;
    int64_t rec_base = 0, elem_base = 0, pix_base = 0;
    uint32_t mask = 0;
    for (int c = 0; c < kMaxClasses; ++c) h->class_begin[c] = h->class_end[c] = 0;
    int cur = -1;
    for (size_t v = 0; v < ts.reqs.size(); ++v) {
        Req* q = ts.reqs[v];
        const voge_request& r = q->r;
        ViewDesc& d = vd[v];
        const int TH = kClassTH[q->cls];
        if (q->cls != cur) {
            if (cur >= 0) h->class_end[cur] = tile_base;
            cur = q->cls;
            h->class_begin[cur] = tile_base;
            mask |= 1u << cur;
        }
        memcpy(d.R, r.cam.R, sizeof(d.R));
        memcpy(d.T, r.cam.T, sizeof(d.T));
        d.F = r.cam.F;
        d.Ox = r.cam.Ox;
        d.Oy = r.cam.Oy;
        d.invF = (float)(1.0 / (double)r.cam.F);
        d.H = r.cam.H;
        d.W = r.cam.W;
        d.tiles_x = (r.cam.W + kTileW - 1) / kTileW;
        d.tiles_y = (r.cam.H + TH - 1) / TH;
        d.tile_h = TH;
        d.tile_base = tile_base;
        d.N = r.N;
        d.C = r.C;
        d.L = q->L;
        d.use_thresh = r.thresh > 0.0f ? 1 : 0;
        d.plain = 0;
        d.tau = r.tau;
        d.Qeta = d.use_thresh ? (r.thresh >= 1.0f ? 0.0f : (float)(2.0 * log(1.0 / (double)r.thresh))) : INFINITY;
        d.rec_base = rec_base;
        d.elem_base = elem_base;
        d.pix_base = pix_base;
        d.means = q->means;
        d.inv_cov = q->inv_cov;
        d.attr = q->attr;
        d.image = q->image;
        d.weights = q->weights;
        d.index = q->index;
        d.index_in = q->index;
        d.weights_in = q->weights;  // the tick's own forward pass wrote them
        d.grad_image = q->grad_image;
        d.target = q->target;
        d.loss = q->loss;
        d.grad_means = q->gmeans;
        d.grad_inv_cov = q->ginv;
        d.grad_attr = q->gattr;
        d.grad_cam = q->gcam;
        tile_base += d.tiles_x * d.tiles_y;
        rec_base += r.N;
        elem_base += q->pixels * r.C;
        pix_base += q->pixels;
    }
    if (cur >= 0) h->class_end[cur] = tile_base;
    h->total_records = rec_base;
    h->total_elems = elem_base;
    h->total_tiles = tile_base;
    h->nviews = (int32_t)ts.reqs.size();
    h->shared_scene = 0;
    return mask;
}

// The launch sequence of one tick (captured into a graph or issued directly).
cudaError_t issue_tick(voge_server* S, TickSlot& ts, uint32_t mask) {
    cudaStream_t s = ts.stream;
    const Args& a = ts.args;
    cudaError_t e = cudaMemcpyAsync(a.hdr, ts.host_desc, ts.desc_bytes, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemsetAsync(a.ws.tile_sub, 0, 4 * (size_t)kTileSub * (size_t)(S->max_tiles + 1), s);
    if (e != cudaSuccess) return e;
    e = launch_project(S->grid_records, (int)std::min<int64_t>(S->max_tiles, (int64_t)S->grid_records * 8), 1, s, a);
    if (e != cudaSuccess) return e;
    for (int c = 0; c < kClasses; ++c) {
        if (!(mask & (1u << c))) continue;
        Args ac = a;
        ac.cls = c;
        e = launch_render_tiles(kClassKM[c], tile_grid(kClassKM[c], 1, 1 << 30), s, ac, 1);
        if (e != cudaSuccess) return e;
    }
    k_mse_batch<<<S->grid_records, 256, 0, s>>>(a);
    e = cudaPeekAtLastError();
    if (e != cudaSuccess) return e;
    for (int c = 0; c < kClasses; ++c) {
        if (!(mask & (1u << c))) continue;
        Args ac = a;
        ac.cls = c;
        // ticks pass their weights; requests of both attribute kinds may share a class
        e = launch_backward_tiles(kClassKM[c], tile_grid(kClassKM[c], 0, 1 << 30), 0, 3, s, ac);
        if (e != cudaSuccess) return e;
    }
    return launch_grad_finalize(S->grid_records, 0, 0, 0, s, a);
}

int run_tick(voge_server* S, TickSlot& ts) {
    const uint32_t mask = build_tick(S, ts);
    cudaError_t e = cudaSuccess;
    if (S->cfg.use_graphs) {
        cudaGraphExec_t exec = nullptr;
        auto it = ts.graphs.find(mask);
        if (it != ts.graphs.end()) {
            exec = it->second;
        } else {
            const int tr = voge_trace_enable(0);  // no event nodes inside the graph
            cudaGraph_t g = nullptr;
            e = cudaStreamBeginCapture(ts.stream, cudaStreamCaptureModeThreadLocal);
            if (e == cudaSuccess) {
                cudaError_t e2 = issue_tick(S, ts, mask);
                e = cudaStreamEndCapture(ts.stream, &g);
                if (e2 != cudaSuccess) e = e2;
            }
            if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, g, 0);
            if (g) cudaGraphDestroy(g);
            voge_trace_enable(tr);
            if (e != cudaSuccess) return VOGE_ERR_CUDA;
            ts.graphs[mask] = exec;
            S->st.graphs_captured += 1;
        }
        e = cudaGraphLaunch(exec, ts.stream);
    } else {
        e = issue_tick(S, ts, mask);
    }
    if (e != cudaSuccess) return VOGE_ERR_CUDA;
    // results back to the callers' host buffers, in stream order after the tick
    for (Req* q : ts.reqs) {
        const voge_request& r = q->r;
        const size_t P = (size_t)q->pixels, N = (size_t)r.N, C = (size_t)r.C;
        if (r.image) cudaMemcpyAsync(r.image, q->image, 4 * P * C, cudaMemcpyDeviceToHost, ts.stream);
        if (r.grad_means) cudaMemcpyAsync(r.grad_means, q->gmeans, 4 * 3 * N, cudaMemcpyDeviceToHost, ts.stream);
        if (r.grad_inv_cov) cudaMemcpyAsync(r.grad_inv_cov, q->ginv, 4 * 6 * N, cudaMemcpyDeviceToHost, ts.stream);
        if (r.grad_attr) cudaMemcpyAsync(r.grad_attr, q->gattr, 4 * C * N, cudaMemcpyDeviceToHost, ts.stream);
        if (r.grad_cam) cudaMemcpyAsync(r.grad_cam, q->gcam, 4 * 12, cudaMemcpyDeviceToHost, ts.stream);
        if (r.loss) cudaMemcpyAsync(r.loss, q->loss, 4, cudaMemcpyDeviceToHost, ts.stream);
    }
    if (cudaEventRecord(ts.done, ts.stream) != cudaSuccess) return VOGE_ERR_CUDA;
    return VOGE_OK;
}

void finish(voge_server* S, Req* q, int status) {
    q->status = status;
    q->state = 3;
    q->t_done = S->now_us();
    if (q->ready) {
        cudaEventDestroy(q->ready);
        q->ready = nullptr;
    }
    if (q->bytes) {
        S->arena.release(q->off, q->bytes);
        q->bytes = 0;
    }
    if (q->scene) q->scene->users -= 1;
    S->resident -= 1;
    S->st.completed += 1;
}

void worker_loop(voge_server* S) {
    cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    while (true) {
        bool progressed = false;
        // 1) completed ticks
        for (TickSlot& ts : S->slots) {
            if (ts.busy && cudaEventQuery(ts.done) == cudaSuccess) {
                for (Req* q : ts.reqs) finish(S, q, VOGE_OK);
                ts.reqs.clear();
                ts.busy = false;
                progressed = true;
                S->cv_done.notify_all();
            }
        }
        // 2) admission, in arrival order, while a slot and arena space are free
        while (!S->queue.empty() && S->resident < S->cfg.max_slots) {
            Req* q = S->queue.front();
            if (!S->arena.alloc(q->bytes, &q->off)) break;
            S->queue.pop_front();
            S->resident += 1;
            carve(q, static_cast<char*>(S->arena_base));
            const voge_request& r = q->r;
            const size_t P = (size_t)q->pixels, N = (size_t)r.N, C = (size_t)r.C;
            cudaStream_t cs = S->copy_stream;
            if (!q->scene) {
                cudaMemcpyAsync(q->means, r.means, 4 * 3 * N, cudaMemcpyHostToDevice, cs);
                cudaMemcpyAsync(q->inv_cov, r.inv_cov, 4 * 6 * N, cudaMemcpyHostToDevice, cs);
                cudaMemcpyAsync(q->attr, r.attr, 4 * C * N, cudaMemcpyHostToDevice, cs);
            }
            cudaMemcpyAsync(q->target, r.target, 4 * P * C, cudaMemcpyHostToDevice, cs);
            cudaMemsetAsync(q->gmeans, 0, (char*)(q->gcam + 16) - (char*)q->gmeans, cs);
            cudaEventCreateWithFlags(&q->ready, cudaEventDisableTiming);
            cudaEventRecord(q->ready, cs);
            q->state = 1;
            q->t_admit = S->now_us();
            S->admitted.push_back(q);
            progressed = true;
        }
        // 3) a tick over every admitted request whose inputs have arrived
        TickSlot* free_slot = nullptr;
        for (TickSlot& ts : S->slots)
            if (!ts.busy) {
                free_slot = &ts;
                break;
            }
        if (free_slot && !S->admitted.empty() && !S->paused) {
            int64_t recs = 0, tiles = 0, elems = 0;
            std::vector<Req*> keep;
            for (Req* q : S->admitted) {
                const int TH = kClassTH[q->cls];
                const int64_t qt = (int64_t)((q->r.cam.W + kTileW - 1) / kTileW) * ((q->r.cam.H + TH - 1) / TH);
                const bool fits = (int)free_slot->reqs.size() < S->max_views && recs + q->r.N <= S->max_records &&
                                  tiles + qt <= S->max_tiles && elems + q->pixels * q->r.C <= S->max_elems;
                const bool one_per_tick = !S->cfg.batching && !free_slot->reqs.empty();
                if (fits && !one_per_tick && cudaEventQuery(q->ready) == cudaSuccess) {
                    free_slot->reqs.push_back(q);
                    recs += q->r.N;
                    tiles += qt;
                    elems += q->pixels * q->r.C;
                } else {
                    keep.push_back(q);
                }
            }
            if (!free_slot->reqs.empty()) {
                S->admitted.swap(keep);
                const int tick = S->tick_counter++;
                const double t = S->now_us();
                for (Req* q : free_slot->reqs) {
                    q->state = 2;
                    q->tick = tick;
                    q->t_start = t;
                }
                const int rc = run_tick(S, *free_slot);
                if (rc != VOGE_OK) {
                    for (Req* q : free_slot->reqs) finish(S, q, rc);
                    free_slot->reqs.clear();
                    S->cv_done.notify_all();
                } else {
                    free_slot->busy = true;
                    S->st.ticks += 1;
                    S->st.requests_in_ticks += (int64_t)free_slot->reqs.size();
                }
                progressed = true;
            }
        }
        if (S->stop && S->queue.empty() && S->admitted.empty()) {
            bool idle = true;
            for (TickSlot& ts : S->slots) idle = idle && !ts.busy;
            if (idle) break;
        }
        if (!progressed) {
            // nothing moved: sleep briefly (new submissions wake us at once)
            S->cv_work.wait_for(lk, std::chrono::microseconds(50));
        }
    }
}

}  // namespace

extern "C" {

int voge_server_create(const voge_server_config* cfg, voge_server** out) {
    if (!cfg || !out || cfg->mem_budget_bytes < (1u << 20) || cfg->max_slots < 1) return VOGE_ERR_ARG;
    voge_server* S = new voge_server();
    S->cfg = *cfg;
    if (S->cfg.max_queue < 1) S->cfg.max_queue = 1 << 16;
    if (S->cfg.inflight_ticks < 1 || S->cfg.inflight_ticks > 4) S->cfg.inflight_ticks = 2;
    if (S->cfg.max_tick_gaussians <= 0) {
        // tick workspaces (about 180 bytes per Gaussian) take at most a quarter of the budget
        const int64_t g = (int64_t)(cfg->mem_budget_bytes / (4 * 180 * (size_t)S->cfg.inflight_ticks));
        S->cfg.max_tick_gaussians = std::max<int64_t>(1 << 16, std::min<int64_t>(g, 4 << 20));
    }
    if (S->cfg.max_tick_pixels <= 0) S->cfg.max_tick_pixels = 16 << 20;
    memset(&S->st, 0, sizeof(S->st));
    S->device = cfg->device;
    S->t0 = Clock::now();
    if (cudaSetDevice(S->device) != cudaSuccess) {
        delete S;
        return VOGE_ERR_CUDA;
    }
    int nsm = 152;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, S->device);
    S->grid_records = nsm * 8;
    S->max_views = std::max(1, std::min(cfg->max_slots, 4096));
    S->max_records = S->cfg.max_tick_gaussians;
    S->max_elems = (int64_t)S->cfg.max_tick_pixels * 128;
    S->max_tiles = S->cfg.max_tick_pixels / 128 + 4 * S->max_views;  // 16 x 8 tiles at worst, plus ragged edges
    S->bin_cap = std::min<int64_t>(S->max_records * 8, INT32_MAX);
    // tick workspace layout
    size_t o = 0;
    const size_t desc = up256(sizeof(BatchHdr) + sizeof(ViewDesc) * S->max_views);
    o += desc;
    S->ws_rec = o; o += up256(64 * (size_t)S->max_records);
    S->ws_rec2 = o; o += up256(32 * (size_t)S->max_records);
    S->ws_tbox = o; o += up256(16 * (size_t)S->max_records);
    S->ws_cnt = o; o += up256(4 * (size_t)(S->max_tiles + 1));
    S->ws_off = o; o += up256(4 * (size_t)(S->max_tiles + 1));
    S->ws_sub = o; o += up256(4 * (size_t)kTileSub * (size_t)(S->max_tiles + 1));
    S->ws_gauss = o; o += up256(4 * (size_t)S->bin_cap);
    S->ws_gcam = o; o += up256(4 * kGcamStride * (size_t)S->max_records);
    const size_t tick_bytes = o;
    const size_t total = (size_t)S->cfg.inflight_ticks * tick_bytes;
    if (total >= cfg->mem_budget_bytes) {
        delete S;
        return VOGE_ERR_ADMISSION;
    }
    bool ok = cudaMalloc(&S->arena_base, cfg->mem_budget_bytes) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking) == cudaSuccess;
    S->arena.init(cfg->mem_budget_bytes);
    S->slots.resize(S->cfg.inflight_ticks);
    for (int k = 0; ok && k < S->cfg.inflight_ticks; ++k) {
        TickSlot& ts = S->slots[k];
        ts.id = k;
        size_t off = 0;
        ok = ok && S->arena.alloc(tick_bytes, &off);
        ts.ws = static_cast<char*>(S->arena_base) + off;
        ts.desc_bytes = sizeof(BatchHdr) + sizeof(ViewDesc) * S->max_views;
        ok = ok && cudaMallocHost((void**)&ts.host_desc, ts.desc_bytes) == cudaSuccess;
        ok = ok && cudaStreamCreateWithFlags(&ts.stream, cudaStreamNonBlocking) == cudaSuccess;
        ok = ok && cudaEventCreateWithFlags(&ts.done, cudaEventDisableTiming) == cudaSuccess;
        if (!ok) break;
        char* b = static_cast<char*>(ts.ws);
        Args& a = ts.args;
        memset(&a, 0, sizeof(a));
        a.hdr = reinterpret_cast<BatchHdr*>(b);
        a.views = reinterpret_cast<const ViewDesc*>(b + sizeof(BatchHdr));
        a.ws.rec = reinterpret_cast<float4*>(b + S->ws_rec);
        a.ws.rec2 = reinterpret_cast<float4*>(b + S->ws_rec2);
        a.ws.tbox = reinterpret_cast<int4*>(b + S->ws_tbox);
        a.ws.tile_cnt = reinterpret_cast<int32_t*>(b + S->ws_cnt);
        a.ws.tile_off = reinterpret_cast<int32_t*>(b + S->ws_off);
        a.ws.tile_sub = reinterpret_cast<int32_t*>(b + S->ws_sub);
        a.ws.tile_gauss = reinterpret_cast<int32_t*>(b + S->ws_gauss);
        a.ws.bin_cap = S->bin_cap;
        a.ws.gcam = reinterpret_cast<float*>(b + S->ws_gcam);
        a.ws.gkey = nullptr;  // lists longer than 32 are not served
        a.ws.gid = nullptr;
        a.ws.gen_L = 0;
        ok = ok && cudaMemset(a.ws.gcam, 0, 4 * kGcamStride * (size_t)S->max_records) == cudaSuccess;  // finalize keeps it zeroed
    }
    if (!ok) {
        voge_server_destroy(S);
        return VOGE_ERR_CUDA;
    }
    S->request_capacity = cfg->mem_budget_bytes - total;
    // occupancy queries and kernel attributes now, outside any stream capture
    for (int c = 0; c < kClasses; ++c) {
        tile_grid(kClassKM[c], 1, 1 << 30);
        tile_grid(kClassKM[c], 0, 1 << 30);
    }
    S->worker = std::thread(worker_loop, S);
    *out = S;
    return VOGE_OK;
}

int voge_server_submit(voge_server* S, const voge_request* req, uint64_t* ticket) {
    if (!S || !ticket || !valid_request(req)) return VOGE_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    Scene* sc = nullptr;
    voge_request rr = *req;
    if (req->scene >= 0) {
        auto it = S->scenes.find(req->scene);
        if (it == S->scenes.end()) return VOGE_ERR_ARG;
        sc = it->second;
        rr.N = sc->N;
        rr.C = sc->C;
    }
    const int L = list_len(rr.K, rr.N);
    if (L > 32) return VOGE_ERR_UNSUPPORTED;
    Req* q = new Req();
    q->r = rr;
    q->scene = sc;
    q->L = L;
    q->cls = class_of(L);
    q->pixels = (int64_t)rr.cam.H * rr.cam.W;
    q->bytes = request_bytes(rr, L, sc != nullptr);
    const int TH = kClassTH[q->cls];
    const int64_t qt = (int64_t)((rr.cam.W + kTileW - 1) / kTileW) * ((rr.cam.H + TH - 1) / TH);
    if (q->bytes > S->request_capacity || rr.N > S->max_records || qt > S->max_tiles || q->pixels * rr.C > S->max_elems) {
        delete q;
        S->st.rejected += 1;
        return VOGE_ERR_ADMISSION;
    }
    if ((int)S->queue.size() >= S->cfg.max_queue) {
        delete q;
        S->st.rejected += 1;
        return VOGE_ERR_BUSY;
    }
    if (sc) sc->users += 1;
    q->ticket = S->next_ticket++;
    q->t_submit = S->now_us();
    S->queue.push_back(q);
    S->all[q->ticket] = q;
    S->st.submitted += 1;
    *ticket = q->ticket;
    S->cv_work.notify_one();
    return VOGE_OK;
}

int voge_server_wait(voge_server* S, uint64_t ticket, int32_t timeout_ms, voge_request_timing* timing) {
    if (!S) return VOGE_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->all.find(ticket);
    if (it == S->all.end()) return VOGE_ERR_ARG;
    Req* q = it->second;
    const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms < 0 ? 0 : timeout_ms);
    while (q->state != 3) {
        if (timeout_ms >= 0 && S->cv_done.wait_until(lk, deadline) == std::cv_status::timeout && q->state != 3)
            return VOGE_ERR_TIMEOUT;
        if (timeout_ms < 0) S->cv_done.wait(lk);
    }
    if (timing) {
        timing->submit_us = q->t_submit;
        timing->admit_us = q->t_admit;
        timing->start_us = q->t_start;
        timing->done_us = q->t_done;
        timing->tick = q->tick;
        timing->status = q->status;
    }
    const int status = q->status;
    S->all.erase(it);
    delete q;
    return status;
}

int voge_server_add_scene(voge_server* S, int32_t N, int32_t C, const float* means, const float* inv_cov,
                          const float* attr, int32_t* scene_id) {
    if (!S || !scene_id || N < 1 || C < 1 || !means || !inv_cov || !attr) return VOGE_ERR_ARG;
    std::unique_lock<std::mutex> lk(S->mu);
    Scene* sc = new Scene();
    sc->N = N;
    sc->C = C;
    sc->bytes = up256(4 * 3 * (size_t)N) + up256(4 * 6 * (size_t)N) + up256(4 * (size_t)C * N);
    if (sc->bytes > S->request_capacity || !S->arena.alloc(sc->bytes, &sc->off)) {
        delete sc;
        return VOGE_ERR_ADMISSION;
    }
    char* p = static_cast<char*>(S->arena_base) + sc->off;
    sc->means = reinterpret_cast<float*>(p);
    sc->inv_cov = reinterpret_cast<float*>(p + up256(4 * 3 * (size_t)N));
    sc->attr = reinterpret_cast<float*>(p + up256(4 * 3 * (size_t)N) + up256(4 * 6 * (size_t)N));
    cudaStream_t cs = S->copy_stream;
    bool ok = cudaMemcpyAsync(sc->means, means, 4 * 3 * (size_t)N, cudaMemcpyHostToDevice, cs) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(sc->inv_cov, inv_cov, 4 * 6 * (size_t)N, cudaMemcpyHostToDevice, cs) == cudaSuccess;
    ok = ok && cudaMemcpyAsync(sc->attr, attr, 4 * (size_t)C * N, cudaMemcpyHostToDevice, cs) == cudaSuccess;
    ok = ok && cudaStreamSynchronize(cs) == cudaSuccess;  // the host arrays may go away after return
    if (!ok) {
        S->arena.release(sc->off, sc->bytes);
        delete sc;
        return VOGE_ERR_CUDA;
    }
    *scene_id = S->next_scene++;
    S->scenes[*scene_id] = sc;
    return VOGE_OK;
}

int voge_server_remove_scene(voge_server* S, int32_t scene_id) {
    if (!S) return VOGE_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    auto it = S->scenes.find(scene_id);
    if (it == S->scenes.end()) return VOGE_ERR_ARG;
    if (it->second->users > 0) return VOGE_ERR_BUSY;
    S->arena.release(it->second->off, it->second->bytes);
    delete it->second;
    S->scenes.erase(it);
    return VOGE_OK;
}

int voge_server_pause(voge_server* S, int32_t paused) {
    if (!S) return VOGE_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    S->paused = paused != 0;
    S->cv_work.notify_all();
    return VOGE_OK;
}

int voge_server_get_stats(voge_server* S, voge_server_stats* out) {
    if (!S || !out) return VOGE_ERR_ARG;
    std::lock_guard<std::mutex> lk(S->mu);
    *out = S->st;
    out->queued = (int64_t)S->queue.size();
    out->resident = S->resident;
    return VOGE_OK;
}

int voge_server_destroy(voge_server* S) {
    if (!S) return VOGE_ERR_ARG;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        S->paused = false;
        S->cv_work.notify_all();
    }
    if (S->worker.joinable()) S->worker.join();
    for (TickSlot& ts : S->slots) {
        for (auto& kv : ts.graphs) cudaGraphExecDestroy(kv.second);
        if (ts.stream) cudaStreamDestroy(ts.stream);
        if (ts.done) cudaEventDestroy(ts.done);
        if (ts.host_desc) cudaFreeHost(ts.host_desc);
    }
    for (auto& kv : S->all) {
        if (kv.second->ready) cudaEventDestroy(kv.second->ready);
        delete kv.second;
    }
    for (auto& kv : S->scenes) delete kv.second;
    for (Req* q : S->queue) (void)q;  // owned by `all`
    if (S->copy_stream) cudaStreamDestroy(S->copy_stream);
    if (S->arena_base) cudaFree(S->arena_base);
    delete S;
    return VOGE_OK;
}

}  // extern "C"
