"""FP64 CPU oracle of the VoGE renderer (test infrastructure only).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library never calls it and shares no
code with it.  ``voge_oracle.c`` holds the arithmetic; this module only builds
it with gcc and marshals numpy arrays through ctypes.

Functions and the passages they follow:
  pose_to_RT / pose_grad   camera pose -> (R, T), look-at; Sec. 3.3 viewing transform
  trace_dir                Eq. 6 / App. A.1 (l, qt = -2q, b = 1/sigma^2)
  render                   Eq. 5-8 with the selection of Sec. 3.3 / App. A.3
  fine                     Eq. 7-8 on given (frozen) per-pixel lists
  render_bwd               chain rule of Eq. 5-8 with frozen lists
  bbox                     exact conic bounding box of e^{q} > eta (App. A.3 role)
  quad_weights             exact outer integral of Eq. 1 by adaptive quadrature
  sample                   neural sampler, Sec. 3.4 Eq. 10 (lists and weights -> per-kernel attributes)
  mesh_to_gaussians        mesh converter of App. A.4: isotropic, optionally flattened along normals
  points_to_gaussians      point-cloud converter of App. A.4 (the same sigma from the m nearest points)
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "voge_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None


class Camera(ctypes.Structure):
    _fields_ = [("R", ctypes.c_double * 9), ("T", ctypes.c_double * 3), ("F", ctypes.c_double),
                ("Ox", ctypes.c_double), ("Oy", ctypes.c_double), ("H", ctypes.c_int), ("W", ctypes.c_int)]


class Params(ctypes.Structure):
    _fields_ = [("B", ctypes.c_int), ("N", ctypes.c_int), ("C", ctypes.c_int), ("K", ctypes.c_int),
                ("tau", ctypes.c_double), ("eta", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (IEEE double, no fast-math)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d, i32, i64 = ctypes.c_double, ctypes.c_int32, ctypes.c_int64
            lib.vo_pose_to_RT.argtypes = [P(d), P(d), P(d)]
            lib.vo_sample.argtypes = [i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, P(i32), P(d), P(d), P(d), P(d)]
            lib.vo_sample.restype = ctypes.c_int
            lib.vo_pose_grad.argtypes = [P(d), P(d), P(d)]
            lib.vo_trace_dir.argtypes = [P(d), P(d), P(d), P(d)]
            lib.vo_bbox.argtypes = [P(Camera), P(Params), P(d), P(d), P(i32)]
            lib.vo_render.argtypes = [P(Camera), P(Params), P(d), P(d), P(d), P(i32), i64, ctypes.c_int, ctypes.c_int,
                                      P(d), P(d), P(i32), P(i32), P(d), P(d)]
            lib.vo_render.restype = ctypes.c_int
            lib.vo_fine.argtypes = [P(Camera), P(Params), P(d), P(d), P(d), P(i32), i64, P(i32), ctypes.c_int,
                                    ctypes.c_int, P(d), P(d)]
            lib.vo_render_bwd.argtypes = [P(Camera), P(Params), P(d), P(d), P(d), P(i32), i64, P(i32), ctypes.c_int,
                                          P(d), ctypes.c_int, P(d), P(d), P(d), P(d)]
            lib.vo_quad_weights.argtypes = [P(d), P(d), P(d), ctypes.c_int, d, P(d)]
            lib.vo_quad_weight.argtypes = [P(d), P(d), P(d), ctypes.c_int, d, ctypes.c_int]
            lib.vo_quad_weight.restype = d
            _lib = lib
    return _lib


def _ptr(a, ctype):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctype))


def _f64(a, shape_tail=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape_tail is not None:
        a = a.reshape((-1,) + tuple(shape_tail))
    return a


def make_cameras(cams):
    """cams: list of dicts with R (3x3), T (3), F, Ox, Oy, H, W."""
    arr = (Camera * max(1, len(cams)))()
    for v, c in enumerate(cams):
        R = np.asarray(c["R"], dtype=np.float64).reshape(9)
        T = np.asarray(c["T"], dtype=np.float64).reshape(3)
        for q in range(9):
            arr[v].R[q] = float(R[q])
        for q in range(3):
            arr[v].T[q] = float(T[q])
        arr[v].F, arr[v].Ox, arr[v].Oy = float(c["F"]), float(c["Ox"]), float(c["Oy"])
        arr[v].H, arr[v].W = int(c["H"]), int(c["W"])
    return arr


def list_cap(K, N):
    return N if (K <= 0 or K >= N) else K


def pose_to_RT(pose):
    lib = _load()
    p = _f64(pose).reshape(4)
    R = np.zeros(9)
    T = np.zeros(3)
    lib.vo_pose_to_RT(_ptr(p, ctypes.c_double), _ptr(R, ctypes.c_double), _ptr(T, ctypes.c_double))
    return R.reshape(3, 3), T


def pose_grad(pose, dR, dT):
    lib = _load()
    p = _f64(pose).reshape(4)
    dRT = np.concatenate([np.asarray(dR, np.float64).reshape(9), np.asarray(dT, np.float64).reshape(3)])
    out = np.zeros(4)
    lib.vo_pose_grad(_ptr(p, ctypes.c_double), _ptr(dRT, ctypes.c_double), _ptr(out, ctypes.c_double))
    return out


def trace_dir(M, P6, D):
    """Eq. 6: returns (l, qt, b) for mean M (3), inverse covariance P6 (6) and ray direction D (3)."""
    lib = _load()
    M, P6, D = _f64(M).reshape(3), _f64(P6).reshape(6), _f64(D).reshape(3)
    out = np.zeros(3)
    lib.vo_trace_dir(_ptr(M, ctypes.c_double), _ptr(P6, ctypes.c_double), _ptr(D, ctypes.c_double),
                     _ptr(out, ctypes.c_double))
    return float(out[0]), float(out[1]), float(out[2])


def all_pixels(cams):
    out = []
    for v, c in enumerate(cams):
        H, W = int(c["H"]), int(c["W"])
        ii, jj = np.meshgrid(np.arange(H), np.arange(W), indexing="ij")
        out.append(np.stack([np.full(H * W, v), ii.reshape(-1), jj.reshape(-1)], 1))
    return np.ascontiguousarray(np.concatenate(out, 0).astype(np.int32))


def _params(B, N, C, K, tau, eta):
    return Params(int(B), int(N), int(C), int(K), float(tau), float(eta))


def render(cams, means, inv_cov, attr, K, tau, eta, pix=None, culled=False, nthreads=None):
    """Forward render of pixels ``pix`` [n][3] = (view, row, col) (all pixels if None).

    Returns dict with image [n][C], weights [n][Kc], idx [n][Kc] (-1 pad), count [n],
    l [n][Kc] (peak depths) and a [n][Kc] (peak densities e^{q})."""
    lib = _load()
    means = _f64(means, (3,))
    inv_cov = _f64(inv_cov, (6,))
    N = means.shape[0]
    attr = _f64(attr).reshape(N, -1) if N else np.zeros((0, np.asarray(attr).shape[-1]))
    C = attr.shape[1]
    attr = np.ascontiguousarray(attr)
    camarr = make_cameras(cams)
    if pix is None:
        pix = all_pixels(cams)
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int32).reshape(-1, 3))
    n = pix.shape[0]
    Kc = list_cap(K, N)
    image = np.zeros((n, C))
    W = np.zeros((n, Kc))
    idx = np.zeros((n, Kc), np.int32)
    cnt = np.zeros(n, np.int32)
    L = np.zeros((n, Kc))
    A = np.zeros((n, Kc))
    p = _params(len(cams), N, C, K, tau, eta)
    nt = nthreads or os.cpu_count() or 1
    lib.vo_render(camarr, ctypes.byref(p), _ptr(means, ctypes.c_double), _ptr(inv_cov, ctypes.c_double),
                  _ptr(attr, ctypes.c_double), _ptr(pix, ctypes.c_int32), n, int(bool(culled)), int(nt),
                  _ptr(image, ctypes.c_double), _ptr(W, ctypes.c_double), _ptr(idx, ctypes.c_int32),
                  _ptr(cnt, ctypes.c_int32), _ptr(L, ctypes.c_double), _ptr(A, ctypes.c_double))
    return {"image": image, "weights": W, "idx": idx, "count": cnt, "l": L, "a": A, "pix": pix}


def fine(cams, means, inv_cov, attr, tau, pix, idx, nthreads=None):
    """Eq. 7-8 on the given lists idx [n][Kc] (-1 terminated)."""
    lib = _load()
    means = _f64(means, (3,))
    inv_cov = _f64(inv_cov, (6,))
    N = means.shape[0]
    attr = np.ascontiguousarray(_f64(attr).reshape(N, -1))
    C = attr.shape[1]
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int32).reshape(-1, 3))
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32).reshape(pix.shape[0], -1))
    n, Kc = idx.shape
    image = np.zeros((n, C))
    W = np.zeros((n, Kc))
    p = _params(len(cams), N, C, Kc, tau, 0.0)
    nt = nthreads or os.cpu_count() or 1
    lib.vo_fine(make_cameras(cams), ctypes.byref(p), _ptr(means, ctypes.c_double), _ptr(inv_cov, ctypes.c_double),
                _ptr(attr, ctypes.c_double), _ptr(pix, ctypes.c_int32), n, _ptr(idx, ctypes.c_int32), Kc, int(nt),
                _ptr(image, ctypes.c_double), _ptr(W, ctypes.c_double))
    return {"image": image, "weights": W}


def render_bwd(cams, means, inv_cov, attr, tau, pix, idx, grad_image, nthreads=None):
    """Analytic gradients with frozen lists.  Returns dict of g_means [N][3], g_inv_cov [N][6],
    g_attr [N][C], g_R [B][3][3], g_T [B][3]."""
    lib = _load()
    means = _f64(means, (3,))
    inv_cov = _f64(inv_cov, (6,))
    N = means.shape[0]
    attr = np.ascontiguousarray(_f64(attr).reshape(N, -1))
    C = attr.shape[1]
    pix = np.ascontiguousarray(np.asarray(pix, dtype=np.int32).reshape(-1, 3))
    idx = np.ascontiguousarray(np.asarray(idx, dtype=np.int32).reshape(pix.shape[0], -1))
    n, Kc = idx.shape
    gimg = np.ascontiguousarray(_f64(grad_image).reshape(n, C))
    B = len(cams)
    gM = np.zeros((N, 3))
    gP = np.zeros((N, 6))
    gA = np.zeros((N, C))
    gRT = np.zeros((B, 12))
    p = _params(B, N, C, Kc, tau, 0.0)
    nt = nthreads or os.cpu_count() or 1
    lib.vo_render_bwd(make_cameras(cams), ctypes.byref(p), _ptr(means, ctypes.c_double),
                      _ptr(inv_cov, ctypes.c_double), _ptr(attr, ctypes.c_double), _ptr(pix, ctypes.c_int32), n,
                      _ptr(idx, ctypes.c_int32), Kc, _ptr(gimg, ctypes.c_double), int(nt),
                      _ptr(gM, ctypes.c_double), _ptr(gP, ctypes.c_double), _ptr(gA, ctypes.c_double),
                      _ptr(gRT, ctypes.c_double))
    return {"g_means": gM, "g_inv_cov": gP, "g_attr": gA, "g_R": gRT[:, :9].reshape(B, 3, 3), "g_T": gRT[:, 9:]}


def bbox(cams, means, inv_cov, eta):
    """[B][N][4] inclusive pixel boxes (x0, x1, y0, y1); x0 > x1 means empty."""
    lib = _load()
    means = _f64(means, (3,))
    inv_cov = _f64(inv_cov, (6,))
    N = means.shape[0]
    B = len(cams)
    out = np.zeros((B, N, 4), np.int32)
    p = _params(B, N, 1, 0, 1.0, eta)
    lib.vo_bbox(make_cameras(cams), ctypes.byref(p), _ptr(means, ctypes.c_double), _ptr(inv_cov, ctypes.c_double),
                _ptr(out, ctypes.c_int32))
    return out


def quad_weights(l, a, b, tau, k=None):
    """Exact W_k = int T(t) rho_k(t) dt along one ray for kernels (l, a, b):
    every kernel's, or kernel k's alone (a float) when k is given."""
    lib = _load()
    l, a, b = _f64(l).reshape(-1), _f64(a).reshape(-1), _f64(b).reshape(-1)
    if k is not None:
        return float(lib.vo_quad_weight(_ptr(l, ctypes.c_double), _ptr(a, ctypes.c_double),
                                        _ptr(b, ctypes.c_double), int(l.shape[0]), float(tau), int(k)))
    out = np.zeros(l.shape[0])
    lib.vo_quad_weights(_ptr(l, ctypes.c_double), _ptr(a, ctypes.c_double), _ptr(b, ctypes.c_double),
                        int(l.shape[0]), float(tau), _ptr(out, ctypes.c_double))
    return out


def sample(idx, weights, phi, N):
    """Sec. 3.4 Eq. 10 on given lists: (alpha [N][C], wsum [N]) from idx [P][L]
    (negative = empty), weights [P][L] and features phi [P][C]."""
    lib = _load()
    idx = np.ascontiguousarray(idx, dtype=np.int32)
    P, L = idx.shape
    W = _f64(weights)
    phi = _f64(phi)
    C = phi.shape[1]
    assert W.shape == (P, L) and phi.shape[0] == P
    alpha = np.zeros((N, C))
    wsum = np.zeros(N)
    rc = lib.vo_sample(P, L, N, C, _ptr(idx, ctypes.c_int32), _ptr(W, ctypes.c_double), _ptr(phi, ctypes.c_double),
                       _ptr(alpha, ctypes.c_double), _ptr(wsum, ctypes.c_double))
    assert rc == 0
    return alpha, wsum


def _iso_sigma(d, zeta):
    """App. A.4: sigma_k = (d_k / 2)^2 / log(1 / zeta), the variance on the
    diagonal of the isotropic Sigma_k."""
    return (np.asarray(d, np.float64) / 2.0) ** 2 / np.log(1.0 / zeta)


def _pack_inverse(Pm):
    """[n][3][3] symmetric -> [n][6] (xx, xy, xz, yy, yz, zz)."""
    return np.stack([Pm[:, 0, 0], Pm[:, 0, 1], Pm[:, 0, 2], Pm[:, 1, 1], Pm[:, 1, 2], Pm[:, 2, 2]], 1)


def mesh_to_gaussians(verts, faces, zeta=0.5, flatten=None):
    """Mesh converter (App. A.4): one Gaussian per vertex; d_k is the mean
    length of the distinct edges at vertex k; Sigma_k = sigma_k I.
    With `flatten` = f (the variant App. B describes), the Gaussian is
    flattened along the vertex normal (the normalised sum of the adjacent
    faces' area-weighted normals):
    Sigma_k = sigma_k (I - n nᵀ) + f sigma_k n nᵀ.  Returns (means [V][3],
    inv_cov [V][6]) in FP64; a vertex on no edge has no d_k and gets an
    inverse covariance of nan."""
    V = np.asarray(verts, np.float64)
    Fc = np.asarray(faces, np.int64)
    edges = set()
    for a, b, c in Fc:
        for i, j in ((a, b), (b, c), (c, a)):
            edges.add((min(i, j), max(i, j)))
    total = np.zeros(len(V))
    count = np.zeros(len(V))
    for i, j in sorted(edges):
        length = np.linalg.norm(V[i] - V[j])
        total[i] += length
        total[j] += length
        count[i] += 1
        count[j] += 1
    d = np.where(count > 0, total / np.where(count > 0, count, 1), np.nan)
    sig = _iso_sigma(d, zeta)
    Pm = np.tile(np.eye(3), (len(V), 1, 1)) / sig[:, None, None]
    if flatten is not None:
        nrm = np.zeros_like(V)
        for a, b, c in Fc:
            fn = np.cross(V[b] - V[a], V[c] - V[a])  # length = twice the area
            nrm[a] += fn
            nrm[b] += fn
            nrm[c] += fn
        nrm /= np.linalg.norm(nrm, axis=1, keepdims=True)
        nn = nrm[:, :, None] * nrm[:, None, :]
        Pm = (np.eye(3)[None] - nn) / sig[:, None, None] + nn / (flatten * sig[:, None, None])
    return V.copy(), _pack_inverse(Pm)


def points_to_gaussians(points, m=4, zeta=0.5):
    """Point-cloud converter (App. A.4): the same sigma_k with d_k the mean
    distance from point k to its m nearest other points (brute force)."""
    X = np.asarray(points, np.float64)
    n = len(X)
    d = np.zeros(n)
    for k in range(n):
        dist = np.sqrt(((X - X[k]) ** 2).sum(1))
        dist[k] = np.inf
        d[k] = np.sort(dist)[:m].mean()
    sig = _iso_sigma(d, zeta)
    Pm = np.tile(np.eye(3), (n, 1, 1)) / sig[:, None, None]
    return X.copy(), _pack_inverse(Pm)
