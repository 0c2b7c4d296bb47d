// voge_convert.cu -- mesh and point-cloud converters (App. A.4): one
// isotropic Gaussian per vertex or point, with the variance on the diagonal
//   sigma_k = (d_k / 2)^2 / log(1 / zeta),
// d_k the mean length of the distinct edges at vertex k (mesh) or the mean
// distance to the m nearest other points (point cloud), zeta the coverage
// rate.  Optionally (the variant App. B describes) a mesh Gaussian is
// flattened along its vertex normal n (the normalised sum of the adjacent
// faces' area-weighted normals): Sigma = sigma (I - n nᵀ) + f sigma n nᵀ.
#include <math.h>

#include "../../include/voge.h"
#include "voge_device.cuh"
#include "voge_trace.cuh"

namespace voge {
namespace {

constexpr unsigned long long kEmptyEdge = ~0ull;

size_t up256(size_t x) { return (x + 255) & ~(size_t)255; }

// Workspace of the mesh converter: an open-addressing set of edges
// (capacity a power of two >= 2 x 3F), per-vertex edge-length sums, edge
// counts and normal sums.
struct MeshWs {
    unsigned long long* keys;
    float* sum;
    int32_t* cnt;
    float* nrm;
    int64_t cap;
    size_t bytes;
};

MeshWs mesh_ws(int32_t V, int32_t F, void* base) {
    MeshWs w{};
    int64_t cap = 2;
    while (cap < 6 * (int64_t)F) cap <<= 1;
    w.cap = cap;
    size_t o = 0;
    char* b = static_cast<char*>(base);
    const size_t keys = o; o = up256(o + 8 * (size_t)cap);
    const size_t sum = o; o = up256(o + 4 * (size_t)V);
    const size_t cnt = o; o = up256(o + 4 * (size_t)V);
    const size_t nrm = o; o = up256(o + 12 * (size_t)V);
    w.bytes = o;
    if (b) {
        w.keys = reinterpret_cast<unsigned long long*>(b + keys);
        w.sum = reinterpret_cast<float*>(b + sum);
        w.cnt = reinterpret_cast<int32_t*>(b + cnt);
        w.nrm = reinterpret_cast<float*>(b + nrm);
    }
    return w;
}

// Per face: its three edges enter the set; the thread that inserts an edge
// first adds its length to both end vertices.  Faces with an index outside
// [0, V) or a repeated vertex are skipped.  With `normals`, the face's
// area-weighted normal (the cross product of two edges) is added to its
// three vertices.
__global__ void __launch_bounds__(256) k_mesh_edges(int32_t V, int32_t F, const float* __restrict__ verts,
                                                    const int32_t* __restrict__ faces, MeshWs w, int normals) {
    for (int64_t f = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; f < F; f += (int64_t)gridDim.x * blockDim.x) {
        const int32_t v[3] = {faces[3 * f], faces[3 * f + 1], faces[3 * f + 2]};
        if (v[0] < 0 || v[1] < 0 || v[2] < 0 || v[0] >= V || v[1] >= V || v[2] >= V) continue;
        if (v[0] == v[1] || v[1] == v[2] || v[0] == v[2]) continue;
        float p[3][3];
#pragma unroll
        for (int c = 0; c < 3; ++c)
#pragma unroll
            for (int q = 0; q < 3; ++q) p[c][q] = verts[3 * (int64_t)v[c] + q];
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            const int32_t a = v[e], b = v[(e + 1) % 3];
            const uint32_t lo = (uint32_t)min(a, b), hi = (uint32_t)max(a, b);
            const unsigned long long key = ((unsigned long long)lo << 32) | hi;
            unsigned long long h = (key * 0x9E3779B97F4A7C15ull) & (unsigned long long)(w.cap - 1);
            bool first = false;
            for (int64_t probe = 0; probe < w.cap; ++probe) {  // bounded: the set is at most half full
                const unsigned long long old = atomicCAS(w.keys + h, kEmptyEdge, key);
                if (old == kEmptyEdge) {
                    first = true;
                    break;
                }
                if (old == key) break;
                h = (h + 1) & (unsigned long long)(w.cap - 1);
            }
            if (first) {
                const float dx = p[e][0] - p[(e + 1) % 3][0], dy = p[e][1] - p[(e + 1) % 3][1],
                            dz = p[e][2] - p[(e + 1) % 3][2];
                const float len = sqrtf(dx * dx + dy * dy + dz * dz);
                atomicAdd(w.sum + a, len);
                atomicAdd(w.sum + b, len);
                atomicAdd(w.cnt + a, 1);
                atomicAdd(w.cnt + b, 1);
            }
        }
        if (normals) {
            const float e1[3] = {p[1][0] - p[0][0], p[1][1] - p[0][1], p[1][2] - p[0][2]};
            const float e2[3] = {p[2][0] - p[0][0], p[2][1] - p[0][1], p[2][2] - p[0][2]};
            const float n[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                e1[0] * e2[1] - e1[1] * e2[0]};
#pragma unroll
            for (int c = 0; c < 3; ++c)
#pragma unroll
                for (int q = 0; q < 3; ++q) atomicAdd(w.nrm + 3 * (int64_t)v[c] + q, n[q]);
        }
    }
}

__device__ __forceinline__ void write_gaussian(int64_t k, const float* x, float sig, const float* n, float flatten,
                                               float* means, float* inv_cov) {
    means[3 * k] = x[0];
    means[3 * k + 1] = x[1];
    means[3 * k + 2] = x[2];
    const float is = 1.0f / sig;
    float P[6] = {is, 0.0f, 0.0f, is, 0.0f, is};
    if (n) {  // (I - n nᵀ) / sigma + n nᵀ / (f sigma)
        const float c = is / flatten - is;
        P[0] += c * n[0] * n[0];
        P[1] += c * n[0] * n[1];
        P[2] += c * n[0] * n[2];
        P[3] += c * n[1] * n[1];
        P[4] += c * n[1] * n[2];
        P[5] += c * n[2] * n[2];
    }
    const bool sized = sig > 0.0f;  // no edges / no size: every entry NaN
#pragma unroll
    for (int q = 0; q < 6; ++q) inv_cov[6 * k + q] = sized ? P[q] : NAN;
}

__global__ void __launch_bounds__(256) k_mesh_finish(int32_t V, const float* __restrict__ verts, MeshWs w,
                                                     float inv_log, float flatten, float* means, float* inv_cov) {
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < V; k += (int64_t)gridDim.x * blockDim.x) {
        const float x[3] = {verts[3 * k], verts[3 * k + 1], verts[3 * k + 2]};
        const int32_t c = w.cnt[k];
        const float d = c > 0 ? w.sum[k] / (float)c : NAN;  // a vertex on no edge has no size
        const float sig = 0.25f * d * d * inv_log;
        float n[3];
        bool use_n = false;
        if (flatten > 0.0f) {
            n[0] = w.nrm[3 * k];
            n[1] = w.nrm[3 * k + 1];
            n[2] = w.nrm[3 * k + 2];
            const float len = sqrtf(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
            if (len > 0.0f) {
                n[0] /= len;
                n[1] /= len;
                n[2] /= len;
                use_n = true;
            }
        }
        write_gaussian(k, x, sig, use_n ? n : nullptr, flatten, means, inv_cov);
    }
}

// Point clouds: one thread per point scans all points in shared-memory tiles
// and keeps its M smallest squared distances (ascending) in registers; d_k is
// the mean of the first m of their square roots.
template <int M>
__global__ void __launch_bounds__(256) k_points(int32_t V, int32_t m, const float* __restrict__ pts, float inv_log,
                                                float* means, float* inv_cov) {
    __shared__ float tile[256 * 3];
    const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = k < V;
    float x[3] = {0.0f, 0.0f, 0.0f};
    if (live) {
        x[0] = pts[3 * k];
        x[1] = pts[3 * k + 1];
        x[2] = pts[3 * k + 2];
    }
    float best[M];
#pragma unroll
    for (int s = 0; s < M; ++s) best[s] = INFINITY;
    for (int64_t base = 0; base < V; base += 256) {
        const int64_t j = base + threadIdx.x;
        __syncthreads();
        if (j < V) {
            tile[3 * threadIdx.x] = pts[3 * j];
            tile[3 * threadIdx.x + 1] = pts[3 * j + 1];
            tile[3 * threadIdx.x + 2] = pts[3 * j + 2];
        }
        __syncthreads();
        const int nt = (int)min((int64_t)256, V - base);
        for (int t = 0; t < nt; ++t) {
            const float dx = tile[3 * t] - x[0], dy = tile[3 * t + 1] - x[1], dz = tile[3 * t + 2] - x[2];
            const float d2 = dx * dx + dy * dy + dz * dz;
            if (d2 < best[M - 1] && base + t != k) {
                // insert into the ascending list: every slot compares against
                // the old list, then takes its neighbour, the new value or itself
                bool lt[M];
#pragma unroll
                for (int s = 0; s < M; ++s) lt[s] = d2 < best[s];
#pragma unroll
                for (int s = M - 1; s >= 1; --s) best[s] = lt[s] ? (lt[s - 1] ? best[s - 1] : d2) : best[s];
                best[0] = lt[0] ? d2 : best[0];
            }
        }
    }
    if (!live) return;
    float acc = 0.0f;
#pragma unroll
    for (int s = 0; s < M; ++s)
        if (s < m) acc += sqrtf(best[s]);
    const float d = acc / (float)m;
    write_gaussian(k, x, 0.25f * d * d * inv_log, nullptr, 0.0f, means, inv_cov);
}

}  // namespace
}  // namespace voge

using namespace voge;

extern "C" size_t voge_mesh_workspace_bytes(int32_t V, int32_t F) {
    if (V < 0 || F < 0) return 0;
    return mesh_ws(V, F, nullptr).bytes;
}

extern "C" int voge_mesh_to_gaussians(int32_t V, int32_t F, const float* verts, const int32_t* faces, float zeta,
                                      float flatten, float* means, float* inv_cov, void* workspace,
                                      size_t workspace_bytes, voge_stream_t stream_) {
    if (V < 0 || F < 0 || !(zeta > 0.0f && zeta < 1.0f) || flatten < 0.0f) return VOGE_ERR_ARG;
    if (V == 0) return VOGE_OK;
    if (!verts || !means || !inv_cov || (F > 0 && !faces)) return VOGE_ERR_ARG;
    const MeshWs probe = mesh_ws(V, F, nullptr);
    if (!workspace || workspace_bytes < probe.bytes || (reinterpret_cast<uintptr_t>(workspace) & 255))
        return VOGE_ERR_WORKSPACE;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    const MeshWs w = mesh_ws(V, F, workspace);
    if (cudaMemsetAsync(w.keys, 0xff, 8 * (size_t)w.cap, s) != cudaSuccess ||
        cudaMemsetAsync(w.sum, 0, (char*)(w.nrm + 3 * (size_t)V) - (char*)w.sum, s) != cudaSuccess)
        return VOGE_ERR_CUDA;
    const float inv_log = (float)(1.0 / log(1.0 / (double)zeta));
    {
        TraceScope tr("k_mesh_edges", s);
        if (F > 0) {
            const int64_t nb = (F + 255) / 256;
            k_mesh_edges<<<(unsigned)(nb > 152 * 16 ? 152 * 16 : nb), 256, 0, s>>>(V, F, verts, faces, w,
                                                                                  flatten > 0.0f ? 1 : 0);
            if (cudaPeekAtLastError() != cudaSuccess) return VOGE_ERR_CUDA;
        }
    }
    TraceScope tr("k_mesh_finish", s);
    const int64_t nb = (V + 255) / 256;
    k_mesh_finish<<<(unsigned)(nb > 152 * 16 ? 152 * 16 : nb), 256, 0, s>>>(V, verts, w, inv_log, flatten, means,
                                                                             inv_cov);
    return cudaPeekAtLastError() == cudaSuccess ? VOGE_OK : VOGE_ERR_CUDA;
}

extern "C" int voge_points_to_gaussians(int32_t V, int32_t m, float zeta, const float* points, float* means,
                                        float* inv_cov, voge_stream_t stream_) {
    if (V < 0 || m < 1 || m > 32 || (V > 0 && m >= V) || !(zeta > 0.0f && zeta < 1.0f)) return VOGE_ERR_ARG;
    if (V == 0) return VOGE_OK;
    if (!points || !means || !inv_cov) return VOGE_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream_);
    const float inv_log = (float)(1.0 / log(1.0 / (double)zeta));
    const unsigned nb = (unsigned)((V + 255) / 256);
    TraceScope tr("k_points", s);
    if (m <= 4) k_points<4><<<nb, 256, 0, s>>>(V, m, points, inv_log, means, inv_cov);
    else if (m <= 8) k_points<8><<<nb, 256, 0, s>>>(V, m, points, inv_log, means, inv_cov);
    else if (m <= 16) k_points<16><<<nb, 256, 0, s>>>(V, m, points, inv_log, means, inv_cov);
    else k_points<32><<<nb, 256, 0, s>>>(V, m, points, inv_log, means, inv_cov);
    return cudaPeekAtLastError() == cudaSuccess ? VOGE_OK : VOGE_ERR_CUDA;
}
