"""CPU FP64 oracle for the sparse-dense SDF renderer -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline / reference arm
may import this package.  The product library (paper_2305_13220_b300) never
imports it and shares no code with it.

The arithmetic lives in sdg_oracle.cpp (plain single-threaded C++17, FP64
except for FP32 block activation); this module only builds it with g++ and
marshals numpy arrays through ctypes.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sdg_oracle.cpp")
_LIB = os.path.join(_HERE, "libsdg_oracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with g++ (no FMA contraction, so FP32 activation follows its stated op order)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
                               "-shared", _SRC, "-o", tmp])
        os.replace(tmp, _LIB)
    return _LIB


class use_library:
    """Context manager that routes every call through another build of the oracle (a test plants a
    mistake in a copy of sdg_oracle.cpp and checks that the pins catch it)."""

    def __init__(self, path):
        self.path = path

    def __enter__(self):
        global _lib
        lib()
        self._old = _lib
        L = C.CDLL(self.path)
        _declare(L)
        _lib = L
        return L

    def __exit__(self, *a):
        global _lib
        _lib = self._old


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _declare(_lib)
    return _lib


_p = C.c_void_p
_i64 = C.c_int64
_u32 = C.c_uint32
_d = C.c_double


def _declare(L):
    sig = {
        "orc_unproject": (_i64, [_p, C.c_int, C.c_int, _p, _p, _p, _p]),
        "orc_keyset_new": (_p, []),
        "orc_keyset_free": (None, [_p]),
        "orc_keyset_add_points": (None, [_p, _p, _p, _i64, C.c_float, C.c_int]),
        "orc_keyset_size": (_i64, [_p]),
        "orc_keyset_get": (None, [_p, _p]),
        "orc_grid_new": (_p, [_d, _d, C.c_int]),
        "orc_grid_free": (None, [_p]),
        "orc_grid_set": (C.c_int, [_p, _p, _i64, _p, _p, _p]),
        "orc_grid_lookup": (None, [_p, _p, _i64, _p]),
        "orc_traverse": (C.c_int, [_p, _p, _p, _p, C.c_int]),
        "orc_sample_hash": (_u32, [_u32, _u32, _u32]),
        "orc_sample_u": (_d, [_u32, _u32, _u32]),
        "orc_density": (_d, [_d, _d]),
        "orc_density_deriv": (_d, [_d, _d]),
        "orc_query": (None, [_p, _p, _i64, _p, _p, _p]),
        "orc_query_grad": (None, [_p, _p, _i64, _p, _p, _p]),
        "orc_eikonal": (_d, [_p, _p, _i64, _d, _p, _p]),
        "orc_crf_loss": (_d, [_p, C.c_int, _p, _i64, _p, _d, _p, _p]),
        "orc_render": (None, [_p, _p, _i64, C.c_int, _u32, _u32, C.c_int, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p]),
        "orc_loss_normal": (_d, [_i64, _p, _p, _d, _p]),
        "orc_lattice_simplex": (None, [_p, C.c_int, _p, _p]),
        "orc_lattice_filter": (_i64, [_i64, C.c_int, _p, C.c_int, _p, _p, C.c_int]),
        "orc_crf_meanfield": (None, [_i64, C.c_int, _p, C.c_int, _p, _p, _d, _p]),
        "orc_trace": (C.c_int, [_p, _p, C.c_int, _u32, _u32, C.c_int, _p]),
        "orc_render_backward": (None, [_p, _p, _i64, C.c_int, _u32, _u32, C.c_int, _p, _p, _p, _p, _p, _p, _p,
                                       _p, _p, _p, _p, _p, _p]),
        "orc_depth_ssi": (_d, [_i64, _p, _p, _d, _p, _p]),
        "orc_count_touched": (None, [_p, _p, _i64, C.c_int, _u32, _u32, C.c_int, _p, _p]),
        "orc_loss": (_d, [_i64, C.c_int, _p, _p, _p, _p, _p, _p, _d, _d, _p, _p, _p]),
        "orc_adam": (None, [_p, _p, _p, _p, _i64, _d, _d, _d, _d, C.c_int]),
        "orc_rmsprop": (None, [_p, _p, _p, _i64, _d, _d, _d]),
        "orc_view_rays": (None, [C.c_int, C.c_int, _p, _p, C.c_float, C.c_float, _p]),
        "orc_fuse": (None, [_p, _i64, C.c_float, C.c_int, C.c_int, C.c_int, _p, _p, _p, C.c_int, _p, _p, C.c_float,
                            _p, _p, _p, _p]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def _arr(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data_as(C.c_void_p)


def _np(x, dtype):
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    return np.ascontiguousarray(x, dtype=dtype)


# ----------------------------------------------------------------------------
# Activation (Eq. 7-8), FP32
# ----------------------------------------------------------------------------


def unproject(depth, K, Twc):
    """Depth map (H, W) -> (xyz (H*W, 3) float32, valid (H*W,) uint8)."""
    depth = _np(depth, np.float32)
    H, W = depth.shape
    Kf, pK = _arr(np.asarray(K, dtype=np.float32), np.float32)
    Tf, pT = _arr(np.asarray(Twc, dtype=np.float32).reshape(12), np.float32)
    xyz = np.empty((H * W, 3), np.float32)
    valid = np.empty(H * W, np.uint8)
    lib().orc_unproject(depth.ctypes.data, H, W, pK, pT, xyz.ctypes.data, valid.ctypes.data)
    return xyz, valid


class KeySet:
    """Exact set of active block keys (std::set), iterated in ascending (z, y, x) order."""

    def __init__(self):
        self._h = lib().orc_keyset_new()

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_keyset_free(self._h)
            self._h = None

    def add_points(self, xyz, voxel_size: float, dilate_voxels: int, valid=None):
        xyz = _np(xyz, np.float32).reshape(-1, 3)
        vp = None
        if valid is not None:
            valid = _np(valid, np.uint8)
            vp = valid.ctypes.data
        lib().orc_keyset_add_points(self._h, xyz.ctypes.data, vp, xyz.shape[0], C.c_float(voxel_size),
                                    int(dilate_voxels))

    def add_depth(self, depth, K, Twc, voxel_size: float, dilate_voxels: int):
        xyz, valid = unproject(depth, K, Twc)
        self.add_points(xyz, voxel_size, dilate_voxels, valid)

    def keys(self) -> np.ndarray:
        n = lib().orc_keyset_size(self._h)
        out = np.empty((n, 3), np.int32)
        if n:
            lib().orc_keyset_get(self._h, out.ctypes.data)
        return out


# ----------------------------------------------------------------------------
# Grid + rendering
# ----------------------------------------------------------------------------


class Grid:
    """FP64 oracle grid: block map + per-voxel sdf / rgb / sem arrays (float64 copies)."""

    def __init__(self, voxel_size: float, beta: float, n_sem: int = 0):
        self.vs, self.beta, self.n_sem = float(voxel_size), float(beta), int(n_sem)
        self._h = lib().orc_grid_new(self.vs, self.beta, self.n_sem)

    def __del__(self):
        if getattr(self, "_h", None):
            lib().orc_grid_free(self._h)
            self._h = None

    def set(self, keys, sdf, rgb, sem=None):
        self.keys = _np(keys, np.int32).reshape(-1, 3)
        N = self.keys.shape[0]
        self.sdf = _np(sdf, np.float64).reshape(N, 512)
        self.rgb = _np(rgb, np.float64).reshape(N, 512, 3)
        self.sem = _np(sem, np.float64).reshape(N, 512, self.n_sem) if self.n_sem else None
        sp = self.sem.ctypes.data if self.n_sem else None
        rc = lib().orc_grid_set(self._h, self.keys.ctypes.data, N, self.sdf.ctypes.data, self.rgb.ctypes.data, sp)
        if rc != 0:
            raise ValueError("duplicate block key")
        return self

    @property
    def n_blocks(self):
        return self.keys.shape[0]

    def lookup(self, keys):
        keys = _np(keys, np.int32).reshape(-1, 3)
        out = np.empty(keys.shape[0], np.int32)
        lib().orc_grid_lookup(self._h, keys.ctypes.data, keys.shape[0], out.ctypes.data)
        return out

    def traverse(self, ray, cap: int = 4096):
        ray = _np(ray, np.float32).reshape(8)
        a = np.empty(cap)
        b = np.empty(cap)
        n = lib().orc_traverse(self._h, ray.ctypes.data, a.ctypes.data, b.ctypes.data, cap)
        return np.stack([a[:n], b[:n]], axis=-1)

    def query(self, x):
        x = _np(x, np.float64).reshape(-1, 3)
        n = x.shape[0]
        sdf, rgb, valid = np.empty(n), np.empty((n, 3)), np.empty(n, np.uint8)
        lib().orc_query(self._h, x.ctypes.data, n, sdf.ctypes.data, rgb.ctypes.data, valid.ctypes.data)
        return sdf, rgb, valid.astype(bool)

    def query_grad(self, x):
        """SDF and its closed-form gradient (Eq. 16-17) at points x (n,3): sdf (n), grad (n,3), valid (n)."""
        x = _np(x, np.float64).reshape(-1, 3)
        n = x.shape[0]
        sdf, grad, valid = np.empty(n), np.empty((n, 3)), np.empty(n, np.uint8)
        lib().orc_query_grad(self._h, x.ctypes.data, n, sdf.ctypes.data, grad.ctypes.data, valid.ctypes.data)
        return sdf, grad, valid.astype(bool)

    def eikonal(self, x, lam: float):
        """Eikonal loss (lambda/n) sum (|grad f| - 1)^2 at points x (n,3); returns (loss, per-point terms,
        dL/dtheta_d [N,512])."""
        x = _np(x, np.float64).reshape(-1, 3)
        n = x.shape[0]
        g = np.zeros((self.n_blocks, 512))
        terms = np.empty(n)
        L = lib().orc_eikonal(self._h, x.ctypes.data, n, float(lam), g.ctypes.data, terms.ctypes.data)
        return L, terms, g

    def crf_loss(self, prop: str, x, target, lam: float):
        """CRF loss of a property ("label", "color", "normal") at points x (n,3) against fixed targets; returns
        (loss, per-point terms, dL/d(stored values): [N,512,n_sem], [N,512,3] or [N,512])."""
        x = _np(x, np.float64).reshape(-1, 3)
        n = x.shape[0]
        pid = {"label": 0, "color": 1, "normal": 2}[prop]
        ch = self.n_sem if pid == 0 else 3
        t = _np(target, np.float64).reshape(n, ch)
        shape = (self.n_blocks, 512) + ((ch,) if pid < 2 else ())
        g = np.zeros(shape)
        terms = np.empty(n)
        L = lib().orc_crf_loss(self._h, pid, x.ctypes.data, n, t.ctypes.data, float(lam), g.ctypes.data,
                               terms.ctypes.data)
        return L, terms, g

    def render(self, rays, n_samples: int, seed: int = 0, ray_id0: int = 0, stratified: bool = True, bg=(0, 0, 0),
               given=None):
        """Forward render.  given: None, or a dict with the samples of every ray fixed by the caller -- "S" [n],
        "t" [n, N] (float32) and "cell" [n, N, 3] (int32, base corner of each sample's trilinear cell); then s_k,
        delta_k and everything after the placement are computed here, in FP64, from those samples."""
        rays = _np(rays, np.float32).reshape(-1, 8)
        n = rays.shape[0]
        gS, gt, gc = _given(given, n, n_samples)
        bgv = np.asarray(bg, np.float64)
        out = {"rgb": np.empty((n, 3)), "depth": np.empty(n), "opac": np.empty(n), "diag": np.empty((n, 4)),
               "normal": np.empty((n, 3))}
        semp = None
        if self.n_sem:
            out["sem"] = np.empty((n, self.n_sem))
            semp = out["sem"].ctypes.data
        lib().orc_render(self._h, rays.ctypes.data, n, int(n_samples), _u32(seed), _u32(ray_id0), int(stratified),
                         bgv.ctypes.data, out["rgb"].ctypes.data, out["depth"].ctypes.data, out["opac"].ctypes.data,
                         semp, out["diag"].ctypes.data, out["normal"].ctypes.data, _ptr_or_none(gS),
                         _ptr_or_none(gt), _ptr_or_none(gc))
        out["S"] = out["diag"][:, 0]
        out["n_valid"] = out["diag"][:, 1]
        out["degenerate"] = out["diag"][:, 2] > 0
        out["T_N"] = out["diag"][:, 3]
        return out

    def trace(self, ray, n_samples: int, seed: int = 0, ray_id: int = 0, stratified: bool = True):
        """Per-sample columns s, t, delta, valid, d, sigma, T, w of one ray."""
        ray = _np(ray, np.float32).reshape(8)
        out = np.zeros((n_samples, 8))
        k = lib().orc_trace(self._h, ray.ctypes.data, int(n_samples), _u32(seed), _u32(ray_id), int(stratified),
                            out.ctypes.data)
        cols = ["s", "t", "delta", "valid", "d", "sigma", "T", "w"]
        return {c: out[:k, i] for i, c in enumerate(cols)}

    def backward(self, rays, n_samples: int, g_rgb, g_depth=None, g_opac=None, g_sem=None, seed: int = 0,
                 ray_id0: int = 0, stratified: bool = True, bg=(0, 0, 0), g_normal=None, given=None):
        """Accumulated dL/dtheta for the given seeds (see render for `given`)."""
        rays = _np(rays, np.float32).reshape(-1, 8)
        n = rays.shape[0]
        gS, gt, gc = _given(given, n, n_samples)
        g_rgb = _np(g_rgb, np.float64).reshape(n, 3)
        gd = _np(g_depth, np.float64) if g_depth is not None else None
        go = _np(g_opac, np.float64) if g_opac is not None else None
        gs = _np(g_sem, np.float64).reshape(n, self.n_sem) if (g_sem is not None and self.n_sem) else None
        N = self.n_blocks
        grad = {"sdf": np.zeros((N, 512)), "rgb": np.zeros((N, 512, 3)), "beta_per_ray": np.zeros(n)}
        gsp = None
        if self.n_sem:
            grad["sem"] = np.zeros((N, 512, self.n_sem))
            gsp = grad["sem"].ctypes.data
        bgv = np.asarray(bg, np.float64)
        gn = _np(g_normal, np.float64).reshape(n, 3) if g_normal is not None else None
        lib().orc_render_backward(self._h, rays.ctypes.data, n, int(n_samples), _u32(seed), _u32(ray_id0),
                                  int(stratified), bgv.ctypes.data, g_rgb.ctypes.data,
                                  gd.ctypes.data if gd is not None else None,
                                  go.ctypes.data if go is not None else None,
                                  gs.ctypes.data if gs is not None else None,
                                  grad["sdf"].ctypes.data, grad["rgb"].ctypes.data, gsp,
                                  grad["beta_per_ray"].ctypes.data, gn.ctypes.data if gn is not None else None,
                                  _ptr_or_none(gS), _ptr_or_none(gt), _ptr_or_none(gc))
        grad["beta"] = float(grad["beta_per_ray"].sum())
        return grad

    def count_touched(self, rays, n_samples: int, seed: int = 0, ray_id0: int = 0, stratified: bool = True):
        rays = _np(rays, np.float32).reshape(-1, 8)
        n = rays.shape[0]
        vx = np.empty(n, np.int64)
        bl = np.empty(n, np.int64)
        lib().orc_count_touched(self._h, rays.ctypes.data, n, int(n_samples), _u32(seed), _u32(ray_id0),
                                int(stratified), vx.ctypes.data, bl.ctypes.data)
        return vx, bl


def _ptr_or_none(a):
    return None if a is None else a.ctypes.data


def _given(given, n, N):
    """Contiguous (S float64 [n], t float32 [n, N], cell int32 [n, N, 3]) of a caller-fixed sample set, or Nones."""
    if given is None:
        return None, None, None
    S = _np(given["S"], np.float64).reshape(n)
    t = _np(given["t"], np.float32).reshape(n, N)
    c = _np(given["cell"], np.int32).reshape(n, N, 3)
    return S, t, c


def sample_hash(seed, ray, k) -> int:
    return int(lib().orc_sample_hash(_u32(seed), _u32(ray), _u32(k)))


def sample_u(seed, ray, k) -> float:
    return float(lib().orc_sample_u(_u32(seed), _u32(ray), _u32(k)))


def density(d, beta):
    return float(lib().orc_density(float(d), float(beta)))


def density_deriv(d, beta):
    return float(lib().orc_density_deriv(float(d), float(beta)))


def loss(rgb, depth, t_rgb, t_depth, lam_d=0.1, sem=None, t_sem=None, lam_s=0.1):
    rgb = _np(rgb, np.float64).reshape(-1, 3)
    n = rgb.shape[0]
    depth = _np(depth, np.float64)
    t_rgb = _np(t_rgb, np.float64).reshape(n, 3)
    t_depth = _np(t_depth, np.float64)
    ns = 0 if sem is None else int(np.asarray(sem).reshape(n, -1).shape[1])
    g_rgb, g_depth = np.empty((n, 3)), np.empty(n)
    g_sem = np.empty((n, ns)) if ns else None
    sp = tp = gp = None
    if ns:
        sem = _np(sem, np.float64).reshape(n, ns)
        t_sem = _np(t_sem, np.float64).reshape(n, ns)
        sp, tp, gp = sem.ctypes.data, t_sem.ctypes.data, g_sem.ctypes.data
    L = lib().orc_loss(n, ns, rgb.ctypes.data, depth.ctypes.data, sp, t_rgb.ctypes.data, t_depth.ctypes.data, tp,
                       float(lam_d), float(lam_s), g_rgb.ctypes.data, g_depth.ctypes.data, gp)
    return L, {"rgb": g_rgb, "depth": g_depth, "sem": g_sem}


def adam(theta, grad, m, v, lr=1e-3, b1=0.9, b2=0.999, eps=1e-8, step=1):
    """In-place Adam step on float64 numpy arrays (grad is zeroed)."""
    for a in (theta, grad, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_adam(theta.ctypes.data, grad.ctypes.data, m.ctypes.data, v.ctypes.data, theta.size, lr, b1, b2, eps,
                   int(step))


def rmsprop(theta, grad, v, lr=1e-3, alpha=0.99, eps=1e-8):
    for a in (theta, grad, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    lib().orc_rmsprop(theta.ctypes.data, grad.ctypes.data, v.ctypes.data, theta.size, lr, alpha, eps)


def view_rays(H, W, K, Twc, tnear=0.05, tfar=1.0e3):
    Kd = np.ascontiguousarray(K, np.float64)
    Td = np.ascontiguousarray(np.asarray(Twc, np.float64).reshape(12))
    rays = np.empty((H * W, 8), np.float32)
    lib().orc_view_rays(H, W, Kd.ctypes.data, Td.ctypes.data, C.c_float(tnear), C.c_float(tfar), rays.ctypes.data)
    return rays


def fuse(keys, voxel_size: float, depth, K, Twc, mu: float, rgb=None, sem=None):
    """Volumetric fusion (Eq. 9-11): frames depth [F,H,W] (z-depth), optional rgb [F,H,W,3] and logits
    [F,H,W,ns], intrinsics K [4] or [F,4] (fx, fy, cx, cy), camera-to-world Twc [3,4] or [F,3,4].  Returns
    float64 sdf [N,512], rgb [N,512,3], sem [N,512,ns] (normalised) and weight [N,512] (association counts)."""
    keys, kp = _arr(keys, np.int32)
    depth = np.asarray(_np(depth, np.float32), dtype=np.float32)
    if depth.ndim == 2:
        depth = depth[None]
    F, H, W = depth.shape
    depth, dp = _arr(depth, np.float32)
    K = np.broadcast_to(np.asarray(_np(K, np.float32), np.float32).reshape(-1, 4), (F, 4))
    K, Kp = _arr(K, np.float32)
    T = np.asarray(_np(Twc, np.float32), np.float32).reshape(-1, 12)
    T = np.broadcast_to(T, (F, 12))
    T, Tp = _arr(T, np.float32)
    N = keys.shape[0]
    ns = 0
    rp = sp = None
    if rgb is not None:
        rgb, rp = _arr(_np(rgb, np.float32), np.float32)
    if sem is not None:
        sem, sp = _arr(_np(sem, np.float32), np.float32)
        ns = sem.shape[-1]
    out = {"sdf": np.zeros((N, 512)), "rgb": np.zeros((N, 512, 3)), "sem": np.zeros((N, 512, max(ns, 1))),
           "weight": np.zeros((N, 512))}
    lib().orc_fuse(kp, N, float(voxel_size), F, H, W, dp, rp, sp, ns, Kp, Tp, float(mu),
                   out["sdf"].ctypes.data_as(_p), out["rgb"].ctypes.data_as(_p), out["sem"].ctypes.data_as(_p),
                   out["weight"].ctypes.data_as(_p))
    if not ns:
        del out["sem"]
    return out


def depth_ssi(depth, t_depth, lam: float = 0.1):
    """Scale/shift-invariant depth loss: (loss, dL/dD (n), (a, b)) with (a, b) the least-squares alignment of the
    targets to the rendered depths."""
    D = _np(depth, np.float64).reshape(-1)
    t = _np(t_depth, np.float64).reshape(-1)
    g = np.empty_like(D)
    ab = np.empty(2)
    L = lib().orc_depth_ssi(D.shape[0], D.ctypes.data, t.ctypes.data, float(lam), g.ctypes.data, ab.ctypes.data)
    return L, g, (float(ab[0]), float(ab[1]))


def loss_normal(normal, t_normal, lam: float = 0.05):
    """L1 normal loss (Eq. 14): (loss, dL/dN (n,3))."""
    N = _np(normal, np.float64).reshape(-1, 3)
    Nt = _np(t_normal, np.float64).reshape(-1, 3)
    g = np.empty_like(N)
    L = lib().orc_loss_normal(N.shape[0], N.ctypes.data, Nt.ctypes.data, float(lam), g.ctypes.data)
    return L, g


def lattice_simplex(p):
    """Enclosing simplex of one scaled feature p (d,) in the permutohedral lattice: vertices ((d+1), (d+1)) int64
    and barycentric weights (d+1,)."""
    p = _np(p, np.float64).reshape(-1)
    d = p.shape[0]
    vert = np.empty((d + 1, d + 1), np.int64)
    bary = np.empty(d + 1)
    lib().orc_lattice_simplex(p.ctypes.data, d, vert.ctypes.data, bary.ctypes.data)
    return vert, bary


def lattice_filter(pos, val, normalize: bool = False):
    """Permutohedral-lattice Gaussian filter of val (n, c) at scaled features pos (n, d); returns (out, lattice
    points)."""
    pos = _np(pos, np.float64)
    val = _np(val, np.float64)
    n, d = pos.shape
    c = val.shape[1]
    out = np.empty((n, c))
    M = lib().orc_lattice_filter(n, d, pos.ctypes.data, c, val.ctypes.data, out.ctypes.data, int(normalize))
    return out, M


def crf_meanfield(pos, unary, Q, w: float):
    """One Potts mean-field update of label distributions Q (n, L) with unaries (n, L) and pairwise weight w."""
    pos = _np(pos, np.float64)
    unary = _np(unary, np.float64)
    Q = _np(Q, np.float64)
    n, d = pos.shape
    L = Q.shape[1]
    out = np.empty((n, L))
    lib().orc_crf_meanfield(n, d, pos.ctypes.data, L, unary.ctypes.data, Q.ctypes.data, float(w), out.ctypes.data)
    return out
