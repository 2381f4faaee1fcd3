"""Python view of an sdg grid: marshals torch tensors (device memory, streams) to the C ABI."""
from __future__ import annotations

import ctypes as C
from typing import Optional, Sequence

import torch

from . import _abi as A


def _ptr(t: Optional[torch.Tensor], dtype=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if dtype is not None and t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    return t.data_ptr() if t.numel() else None


class _DevArray:
    """__cuda_array_interface__ wrapper so torch can view grid-owned memory without a copy."""

    def __init__(self, ptr: int, shape, typestr: str, owner):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 3, "strides": None}
        self._owner = owner


_CHANNEL_SHAPES = {
    # (group, kind) -> (lanes per voxel, typestr); None lanes -> n_sem
    (A.GROUP_GEO, A.KIND_VALUE): (4, "<f4"), (A.GROUP_GEO, A.KIND_GRAD): (4, "<f4"),
    (A.GROUP_GEO, A.KIND_ADAM_M): (4, "<f4"), (A.GROUP_GEO, A.KIND_ADAM_V): (4, "<f4"),
    (A.GROUP_SDF, A.KIND_VALUE): (1, "<f4"), (A.GROUP_SDF, A.KIND_GRAD): (1, "<f4"),
    (A.GROUP_SDF, A.KIND_ADAM_M): (1, "<f4"), (A.GROUP_SDF, A.KIND_ADAM_V): (1, "<f4"),
    (A.GROUP_RGB, A.KIND_VALUE): (4, "<i2"), (A.GROUP_RGB, A.KIND_GRAD): (4, "<f4"),
    (A.GROUP_RGB, A.KIND_ADAM_M): (4, "<f4"), (A.GROUP_RGB, A.KIND_ADAM_V): (4, "<f4"),
    (A.GROUP_SEM, A.KIND_VALUE): (None, "<i2"), (A.GROUP_SEM, A.KIND_GRAD): (None, "<f4"),
    (A.GROUP_SEM, A.KIND_ADAM_M): (None, "<f4"), (A.GROUP_SEM, A.KIND_ADAM_V): (None, "<f4"),
    (A.GROUP_WEIGHT, A.KIND_VALUE): (1, "<f4"),
}


class Grid:
    """A globally sparse, locally dense SDF/colour/semantic grid living on one GPU.

    All work is enqueued on `stream` (default: torch's current stream on `device` at creation)."""

    def __init__(self, voxel_size: float, max_blocks: int, beta: float = 0.0, rgb_dtype: str = "f32", n_sem: int = 0,
                 device: int = 0, stream: Optional[torch.cuda.Stream] = None, _handle=None):
        self.device = device
        if stream is None:
            stream = torch.cuda.current_stream(device)
        self.stream = stream
        if _handle is not None:
            self._h = _handle
        else:
            d = A.GridDesc(voxel_size=voxel_size, beta=beta, max_blocks=max_blocks,
                           rgb_dtype=A.F32 if rgb_dtype == "f32" else A.BF16, n_sem=n_sem, device=device,
                           reserved=0, stream=stream.cuda_stream)
            h = C.c_void_p()
            A.call("sdg_grid_create", C.byref(d), C.byref(h))
            self._h = h
        self.voxel_size = voxel_size
        self.max_blocks = max_blocks
        self.rgb_dtype = rgb_dtype
        self.n_sem = n_sem

    # -- life cycle ---------------------------------------------------------
    def set_pass_events(self, start=None, stop=None):
        """Makes every later render pass on this grid record the torch.cuda.Event pair around its render kernels
        (sdg_grid_set_pass_events); no arguments stop the recording."""
        A.call("sdg_grid_set_pass_events", self._h, None if start is None else C.c_void_p(start.cuda_event),
               None if stop is None else C.c_void_p(stop.cuda_event))

    def close(self):
        """Destroys the grid (SdgError with SDG_ERR_BUSY, the grid kept, while a server still holds it)."""
        if getattr(self, "_h", None) is not None and self._h.value:
            A.call("sdg_grid_destroy", self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    # -- activation (Eq. 7-8) ----------------------------------------------
    def activate_points(self, xyz: torch.Tensor, dilate_voxels: int) -> int:
        n = C.c_int64()
        A.call("sdg_grid_activate_points", self._h, _ptr(xyz, torch.float32, "xyz"), xyz.shape[0],
               int(dilate_voxels), C.byref(n))
        return n.value

    def activate_depth(self, depth: torch.Tensor, K: Sequence[float], Twc, dilate_voxels: int) -> int:
        H, W = depth.shape
        Kc = (C.c_float * 4)(*[float(v) for v in K])
        Tc = (C.c_float * 12)(*[float(v) for v in torch.as_tensor(Twc, dtype=torch.float64).reshape(12).tolist()])
        n = C.c_int64()
        A.call("sdg_grid_activate_depth", self._h, _ptr(depth, torch.float32, "depth"), H, W, Kc, Tc,
               int(dilate_voxels), C.byref(n))
        return n.value

    def activate_depth_frames(self, depth: torch.Tensor, K, Twc, dilate_voxels: int) -> int:
        """activate_depth over F maps as one activation batch: depth [F,H,W] on the grid's device, K [4] or [F,4],
        Twc [3,4] or [F,3,4] camera-to-world.  Returns the number of blocks added."""
        F, H, W = depth.shape
        Kt = torch.as_tensor(K, dtype=torch.float64).reshape(-1, 4).expand(F, 4)
        Tt = torch.as_tensor(Twc, dtype=torch.float64).reshape(-1, 12).expand(F, 12)
        Kc = (C.c_float * max(4 * F, 1))(*[float(v) for v in Kt.reshape(-1).tolist()])
        Tc = (C.c_float * max(12 * F, 1))(*[float(v) for v in Tt.reshape(-1).tolist()])
        n = C.c_int64()
        A.call("sdg_grid_activate_depth_frames", self._h, _ptr(depth, torch.float32, "depth"), F, H, W, Kc, Tc,
               int(dilate_voxels), C.byref(n))
        return n.value

    def fuse(self, depth: torch.Tensor, K, Twc, mu: float, rgb: Optional[torch.Tensor] = None,
             sem: Optional[torch.Tensor] = None):
        """Volumetric fusion (Eq. 9-11) of F frames: depth [F,H,W] or [H,W] (z-depth), optional rgb [F,H,W,3] and
        logits [F,H,W,n_sem] on the grid's device; K [4] or [F,4]; Twc [3,4] or [F,3,4] camera-to-world.
        Running means over calls; call fuse_finalize() once all frames are in (before training)."""
        if depth.dim() == 2:
            depth = depth[None]
            rgb = rgb[None] if rgb is not None else None
            sem = sem[None] if sem is not None else None
        F, H, W = depth.shape
        Kt = torch.as_tensor(K, dtype=torch.float32).reshape(-1, 4).expand(F, 4).contiguous()
        Tt = torch.as_tensor(Twc, dtype=torch.float32).reshape(-1, 12).expand(F, 12).contiguous()
        A.call("sdg_fuse_frames", self._h, F, H, W, _ptr(depth, torch.float32, "depth"),
               _ptr(rgb, torch.float32, "rgb") if rgb is not None else None,
               _ptr(sem, torch.float32, "sem") if sem is not None else None,
               Kt.data_ptr(), Tt.data_ptr(), float(mu))

    def lattice_filter(self, pos: torch.Tensor, val: torch.Tensor, normalize: bool = False):
        """Permutohedral-lattice Gaussian filter (the CRF's message passing): val (n, c) at scaled features
        pos (n, d); returns (out (n, c), number of lattice points).  Uses this grid's stream and scratch."""
        out = torch.empty_like(val)
        m = C.c_int64()
        A.call("sdg_lattice_filter", self._h, pos.shape[0], pos.shape[1], _ptr(pos, torch.float32, "pos"),
               val.shape[1], _ptr(val, torch.float32, "val"), _ptr(out), 1 if normalize else 0, C.byref(m))
        return out, m.value

    def crf_meanfield(self, pos: torch.Tensor, unary: torch.Tensor, q: torch.Tensor, w: float):
        """One Potts mean-field update (Eq. 22) of label distributions q (n, L) with unaries (n, L)."""
        out = torch.empty_like(q)
        A.call("sdg_crf_meanfield", self._h, pos.shape[0], pos.shape[1], _ptr(pos, torch.float32, "pos"),
               q.shape[1], _ptr(unary, torch.float32, "unary"), _ptr(q, torch.float32, "q"), float(w), _ptr(out))
        return out

    def crf_loss(self, prop: str, xyz: torch.Tensor, target: torch.Tensor, lam: float,
                 terms: Optional[torch.Tensor] = None, loss_sum: Optional[torch.Tensor] = None):
        """CRF loss of a property ("label", "color", "normal") at points xyz (n, 3) against fixed targets; the
        gradient is ADDED into the property's gradient channel."""
        pid = {"label": 0, "color": 1, "normal": 2}[prop]
        A.call("sdg_crf_loss", self._h, pid, xyz.shape[0], _ptr(xyz, torch.float32, "xyz"),
               _ptr(target, torch.float32, "target"), float(lam), _ptr(terms), _ptr(loss_sum))

    def fuse_finalize(self):
        A.call("sdg_fuse_finalize", self._h)

    def query(self, xyz: torch.Tensor, want_sdf: bool = True, want_grad: bool = True):
        """SDF (n) and closed-form gradient (n, 3) at points xyz (n, 3) float32 in one pass (Eq. 16-17); NaN
        where a grid point of the cell is not allocated."""
        n = xyz.shape[0]
        sdf = torch.empty(n, device=xyz.device) if want_sdf else None
        grad = torch.empty((n, 3), device=xyz.device) if want_grad else None
        A.call("sdg_query", self._h, _ptr(xyz, torch.float32, "xyz"), n, _ptr(sdf), _ptr(grad))
        return sdf, grad

    def eikonal(self, xyz: torch.Tensor, lam: float = 0.1, terms: Optional[torch.Tensor] = None,
                loss_sum: Optional[torch.Tensor] = None):
        """Eikonal loss (lam/n) sum (|grad f| - 1)^2 at points xyz (n, 3); its gradient is ADDED into the SDF
        gradient channel.  Per-point terms to `terms` (n) and their sum to `loss_sum` (1) when given."""
        A.call("sdg_eikonal", self._h, _ptr(xyz, torch.float32, "xyz"), xyz.shape[0], float(lam), _ptr(terms),
               _ptr(loss_sum))

    def activate_keys(self, keys: torch.Tensor) -> int:
        n = C.c_int64()
        A.call("sdg_grid_activate_keys", self._h, _ptr(keys, torch.int32, "keys"), keys.shape[0], C.byref(n))
        return n.value

    @property
    def num_blocks(self) -> int:
        n = C.c_int64()
        A.call("sdg_grid_num_blocks", self._h, C.byref(n))
        return n.value

    def keys(self) -> torch.Tensor:
        n = self.num_blocks
        out = torch.empty((n, 3), dtype=torch.int32, device=f"cuda:{self.device}")
        A.call("sdg_grid_keys", self._h, _ptr(out))
        return out

    def lookup(self, keys: torch.Tensor) -> torch.Tensor:
        out = torch.empty(keys.shape[0], dtype=torch.int32, device=keys.device)
        A.call("sdg_grid_lookup", self._h, _ptr(keys, torch.int32, "keys"), keys.shape[0], _ptr(out))
        return out

    # -- channels -----------------------------------------------------------
    def channel(self, group: int, kind: int = A.KIND_VALUE) -> torch.Tensor:
        """Zero-copy tensor view [max_blocks, 512, lanes] of a grid channel (bf16 values as torch.bfloat16)."""
        p = C.c_void_p()
        nbytes = C.c_int64()
        A.call("sdg_grid_channel", self._h, group, kind, C.byref(p), C.byref(nbytes))
        lanes, ts = _CHANNEL_SHAPES[(group, kind)]
        if lanes is None:
            lanes = self.n_sem
        shape = (self.max_blocks, 512, lanes)
        with torch.cuda.device(self.device):
            t = torch.as_tensor(_DevArray(p.value, shape, ts, self), device=f"cuda:{self.device}")
        if ts == "<i2":
            t = t.view(torch.bfloat16)
        return t

    def zero_grad(self):
        A.call("sdg_grid_zero_grad", self._h)

    def sync(self):
        A.call("sdg_grid_sync", self._h)

    @property
    def beta(self) -> float:
        """Laplace scale of the SDF-to-density transform (learnable through train_step_rays(learn_beta=True))."""
        b = C.c_float()
        A.call("sdg_grid_get_beta", self._h, C.byref(b))
        return b.value

    @beta.setter
    def beta(self, v: float):
        A.call("sdg_grid_set_beta", self._h, float(v))

    def beta_grad(self) -> float:
        """dL/dbeta accumulated since the last optimiser step (synchronises)."""
        b = C.c_float()
        A.call("sdg_grid_beta_grad", self._h, C.byref(b))
        return b.value

    @property
    def step(self) -> int:
        s = C.c_int32()
        A.call("sdg_grid_get_step", self._h, C.byref(s))
        return s.value

    @step.setter
    def step(self, v: int):
        A.call("sdg_grid_set_step", self._h, int(v))

    # -- optimiser ----------------------------------------------------------
    def adam_step(self, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, step: int = 0, algo: str = "adam"):
        o = A.AdamOpts(lr=lr, beta1=beta1, beta2=beta2, eps=eps, step=step,
                       algo=A.OPT_ADAM if algo == "adam" else A.OPT_RMSPROP)
        A.call("sdg_adam_step", self._h, C.byref(o))

    # -- checkpoint ---------------------------------------------------------
    def save(self, path: str):
        A.call("sdg_grid_save", self._h, path.encode())

    @classmethod
    def load(cls, path: str, max_blocks: Optional[int] = None, device: int = 0, stream=None) -> "Grid":
        if stream is None:
            stream = torch.cuda.current_stream(device)
        h = C.c_void_p()
        d = None
        if max_blocks is not None:
            d = A.GridDesc(voxel_size=0.0, beta=0.0, max_blocks=max_blocks, rgb_dtype=0, n_sem=0, device=device,
                           reserved=0, stream=stream.cuda_stream)
        A.call("sdg_grid_load", path.encode(), C.byref(d) if d is not None else None, C.byref(h))
        g = cls.__new__(cls)
        g._h = h
        g.device = device
        g.stream = stream
        # read back layout from the file header through the channel API
        import struct
        with open(path, "rb") as f:
            hdr = f.read(40)
        vs, beta, dt, ns, nb, step, _ = struct.unpack("<8xffiiqii", hdr)
        g.voxel_size, g.rgb_dtype, g.n_sem = vs, ("f32" if dt == A.F32 else "bf16"), ns
        g.max_blocks = max_blocks if max_blocks is not None else max(nb, 1)
        return g


def render_opts(n_samples: int, seed: int = 0, ray_id0: int = 0, stratified: bool = True, mode: str = "recompute",
                bg=(0.0, 0.0, 0.0)) -> A.RenderOpts:
    o = A.RenderOpts(n_samples=n_samples, seed=seed, ray_id0=ray_id0, stratified=int(stratified),
                     mode=A.MODE_STORE if mode == "store" else A.MODE_RECOMPUTE)
    o.bg[0], o.bg[1], o.bg[2] = (float(v) for v in bg)
    return o
