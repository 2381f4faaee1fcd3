"""Rendering calls and the autograd wrapper (argument marshalling over the C ABI; all compute is in libsdg)."""
from __future__ import annotations

import ctypes as C
from typing import Optional

import torch

from . import _abi as A
from .grid import Grid, _ptr, render_opts


class RenderContext:
    """Saved state of one forward for its backward (owns the ABI context; rays are kept alive)."""

    def __init__(self, handle: C.c_void_p, grid: Grid, rays: torch.Tensor):
        self._h = handle
        self.grid = grid
        self.rays = rays

    def release(self):
        if self._h is not None and self._h.value:
            A.lib().sdg_ctx_release(self._h)
        self._h = None

    def __del__(self):
        try:
            self.release()
        except Exception:
            pass


def render(grid: Grid, rays: torch.Tensor, n_samples: int, seed: int = 0, ray_id0: int = 0, stratified: bool = True,
           mode: str = "recompute", bg=(0.0, 0.0, 0.0), want_ctx: bool = False, want_sem: bool = True):
    """Forward render (Eq. 12-15) of rays [n, 8] -> dict(rgb [n,3], depth [n], opac [n], sem [n,n_sem], ctx)."""
    n = rays.shape[0]
    dev = rays.device
    out = {"rgb": torch.empty((n, 3), device=dev), "depth": torch.empty(n, device=dev),
           "opac": torch.empty(n, device=dev)}
    sem_p = None
    if grid.n_sem and want_sem:
        out["sem"] = torch.empty((n, grid.n_sem), device=dev)
        sem_p = _ptr(out["sem"])
    ro = A.RenderOut(rgb=_ptr(out["rgb"]), depth=_ptr(out["depth"]), opac=_ptr(out["opac"]), sem=sem_p)
    o = render_opts(n_samples, seed, ray_id0, stratified, mode, bg)
    h = C.c_void_p()
    A.call("sdg_render_forward", grid.handle, _ptr(rays, torch.float32, "rays"), n, C.byref(o), C.byref(ro),
           C.byref(h) if want_ctx else None)
    out["ctx"] = RenderContext(h, grid, rays) if want_ctx else None
    return out


def _trace_buffers(n: int, n_samples: int, dev):
    out = {"n_cells": torch.empty(n, dtype=torch.int32, device=dev), "S": torch.empty(n, device=dev),
           "t": torch.empty((n, n_samples), device=dev),
           "cell": torch.empty((n, n_samples, 3), dtype=torch.int32, device=dev),
           "block": torch.empty((n, n_samples), dtype=torch.int32, device=dev),
           "valid": torch.empty((n, n_samples), dtype=torch.uint8, device=dev),
           "seg": torch.zeros((n, A.TRACE_CELLS, 2), device=dev),
           "rgb": torch.empty((n, 3), device=dev), "depth": torch.empty(n, device=dev),
           "opac": torch.empty(n, device=dev)}
    to = A.TraceOut(**{k: _ptr(v) for k, v in out.items()})
    return out, to


def trace(grid: Grid, rays: torch.Tensor, n_samples: int, seed: int = 0, ray_id0: int = 0, stratified: bool = True,
          bg=(0.0, 0.0, 0.0), walk: str = "pass"):
    """Debug export of the sample placement of a forward render (sdg_debug_trace): per ray n_cells, S, seg; per
    sample t, cell [.., 3], block, valid; and the forward outputs rgb, depth, opac.  walk: "pass" (as the forward,
    backward and training passes) or "in_warp" (as the serving loop and the allocation-free training pass)."""
    walks = {"pass": A.WALK_PASS, "in_warp": A.WALK_IN_WARP}
    n = rays.shape[0]
    out, to = _trace_buffers(n, n_samples, rays.device)
    o = render_opts(n_samples, seed, ray_id0, stratified, "recompute", bg)
    A.call("sdg_debug_trace", grid.handle, _ptr(rays, torch.float32, "rays"), n, C.byref(o), walks[walk],
           C.byref(to))
    return out


def trace_view(grid: Grid, H: int, W: int, K, Twc, n_samples: int, seed: int = 0, stratified: bool = True,
               tnear: float = 0.05, tfar: float = 1.0e3):
    """Debug export of a served H x W view (sdg_debug_trace_view): the trace() outputs plus the rays [H*W, 8] the
    serving kernel forms for it."""
    n = H * W
    dev = f"cuda:{grid.device}"
    out, to = _trace_buffers(n, n_samples, dev)
    out["rays"] = torch.empty((n, 8), device=dev)
    o = render_opts(n_samples, seed, 0, stratified, "recompute", (0.0, 0.0, 0.0))
    Kc = (C.c_float * 4)(*[float(x) for x in K])
    Tc = (C.c_float * 12)(*torch.as_tensor(Twc, dtype=torch.float64).reshape(12).tolist())
    A.call("sdg_debug_trace_view", grid.handle, H, W, Kc, Tc, float(tnear), float(tfar), C.byref(o),
           _ptr(out["rays"]), C.byref(to))
    return out


def backward(ctx: RenderContext, g_rgb: torch.Tensor, g_depth: Optional[torch.Tensor] = None,
             g_opac: Optional[torch.Tensor] = None, g_sem: Optional[torch.Tensor] = None):
    """Accumulates dL/dtheta into the grid's gradient channels."""
    A.call("sdg_render_backward", ctx._h, _ptr(g_rgb.contiguous(), torch.float32, "g_rgb"),
           _ptr(None if g_depth is None else g_depth.contiguous()),
           _ptr(None if g_opac is None else g_opac.contiguous()),
           _ptr(None if g_sem is None else g_sem.contiguous()))


def loss_l1(grid: Grid, rgb, depth, t_rgb, t_depth, sem=None, t_sem=None, lambda_depth=0.1, lambda_sem=0.1):
    """Per-ray L1 colour / depth (+ squared L2 logits) loss terms and their gradient seeds."""
    n = rgb.shape[0]
    g = {"rgb": torch.empty_like(rgb), "depth": torch.empty_like(depth)}
    if sem is not None:
        g["sem"] = torch.empty_like(sem)
    loss = torch.empty(n, device=rgb.device)
    lo = A.LossOpts(lambda_depth=lambda_depth, lambda_sem=lambda_sem)
    A.call("sdg_loss_l1", grid.handle, n, _ptr(rgb), _ptr(depth), _ptr(sem), _ptr(t_rgb), _ptr(t_depth), _ptr(t_sem),
           C.byref(lo), _ptr(g["rgb"]), _ptr(g["depth"]), _ptr(g.get("sem")), _ptr(loss))
    return loss, g


def train_step_rays_normal(grid: Grid, rays: torch.Tensor, t_rgb: torch.Tensor, t_depth: torch.Tensor,
                           t_normal: torch.Tensor, n_samples: int = 128, seed: int = 0, ray_id0: int = 0,
                           stratified: bool = True, bg=(0.0, 0.0, 0.0), lambda_depth: float = 0.1,
                           lambda_normal: float = 0.05, loss: Optional[torch.Tensor] = None,
                           loss_sum: Optional[torch.Tensor] = None, ray_order: str = "auto"):
    """Fused training pass with the L1 normal loss of Eq. 14 on the rendered normal sum_k w_k grad f(x_k)."""
    o = render_opts(n_samples, seed, ray_id0, stratified, "recompute", bg)
    orders = {"auto": A.ORDER_AUTO, "given": A.ORDER_GIVEN, "surface": A.ORDER_SURFACE}
    lo = A.LossOpts(lambda_depth=lambda_depth, lambda_sem=0.0, ray_order=orders[ray_order], learn_beta=0)
    A.call("sdg_train_step_rays_normal", grid.handle, _ptr(rays, torch.float32, "rays"), rays.shape[0],
           _ptr(t_rgb, torch.float32, "t_rgb"), _ptr(t_depth, torch.float32, "t_depth"),
           _ptr(t_normal, torch.float32, "t_normal"), C.byref(o), C.byref(lo), float(lambda_normal), _ptr(loss),
           _ptr(loss_sum))


def loss_depth_ssi(grid: Grid, depth, t_depth, lam: float = 0.1, want_ab: bool = False):
    """Scale/shift-invariant depth loss: per-ray terms, depth seeds dL/dD and, if want_ab, the fitted (a, b)."""
    n = depth.shape[0]
    g = torch.empty_like(depth)
    loss = torch.empty(n, device=depth.device)
    ab = (C.c_double * 2)()
    A.call("sdg_loss_depth_ssi", grid.handle, n, _ptr(depth, torch.float32, "depth"),
           _ptr(t_depth, torch.float32, "t_depth"), float(lam), _ptr(g), _ptr(loss), None, ab if want_ab else None)
    return (loss, g, (ab[0], ab[1])) if want_ab else (loss, g)


def train_step_rays(grid: Grid, rays: torch.Tensor, t_rgb: torch.Tensor, t_depth: torch.Tensor,
                    t_sem: Optional[torch.Tensor] = None, n_samples: int = 128, seed: int = 0, ray_id0: int = 0,
                    stratified: bool = True, bg=(0.0, 0.0, 0.0), lambda_depth: float = 0.1, lambda_sem: float = 0.1,
                    loss: Optional[torch.Tensor] = None, loss_sum: Optional[torch.Tensor] = None,
                    ray_order: str = "auto", learn_beta: bool = False, norm_rays: int = 0,
                    prepared: Optional[int] = None):
    """Fused forward + L1 losses + backward; gradients accumulate into the grid.

    ray_order: "auto" (surface order for batches of 65536 rays or more), "given" or "surface" (rays grouped by
    the coarse cell of their target surface point; per-ray results are unchanged).  learn_beta: also accumulate
    dL/dbeta for the next optimiser step, which then updates the grid's Laplace scale.  norm_rays: the n of the
    means over rays (0: these rays' count; a data-parallel shard passes the whole batch's).  prepared: the slot
    train_prepare prepared these rays in (their ordering and traversal then ran ahead)."""
    o = render_opts(n_samples, seed, ray_id0, stratified, "recompute", bg)
    orders = {"auto": A.ORDER_AUTO, "given": A.ORDER_GIVEN, "surface": A.ORDER_SURFACE}
    if ray_order not in orders:
        raise ValueError(f"ray_order must be one of {sorted(orders)}")
    lo = A.LossOpts(lambda_depth=lambda_depth, lambda_sem=lambda_sem, ray_order=orders[ray_order],
                    learn_beta=1 if learn_beta else 0, norm_rays=int(norm_rays),
                    prepared=0 if prepared is None else int(prepared) + 1)
    A.call("sdg_train_step_rays", grid.handle, _ptr(rays, torch.float32, "rays"), rays.shape[0],
           _ptr(t_rgb, torch.float32, "t_rgb"), _ptr(t_depth, torch.float32, "t_depth"), _ptr(t_sem), C.byref(o),
           C.byref(lo), _ptr(loss), _ptr(loss_sum))


def train_prepare(grid: Grid, rays: torch.Tensor, t_depth: torch.Tensor, slot: int, ray_order: str = "auto"):
    """Enqueues the ordering and traversal of a training batch on the grid's auxiliary stream into `slot` (0, 1):
    called after one step's train_step_rays and before its optimiser step, the next batch's traversal runs beside
    the optimiser; pass prepared=slot to the train_step_rays of these rays."""
    orders = {"auto": A.ORDER_AUTO, "given": A.ORDER_GIVEN, "surface": A.ORDER_SURFACE}
    lo = A.LossOpts(ray_order=orders[ray_order])
    A.call("sdg_train_prepare", grid.handle, _ptr(rays, torch.float32, "rays"), rays.shape[0],
           _ptr(t_depth, torch.float32, "t_depth"), C.byref(lo), int(slot))


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(fctx, anchor, grid, rays, n_samples, seed, ray_id0, stratified, mode, bg):
        out = render(grid, rays, n_samples, seed, ray_id0, stratified, mode, bg, want_ctx=True)
        fctx.sdg = out["ctx"]
        fctx.has_sem = "sem" in out
        res = [out["rgb"], out["depth"], out["opac"]]
        if fctx.has_sem:
            res.append(out["sem"])
        return tuple(res)

    @staticmethod
    def backward(fctx, g_rgb, g_depth, g_opac, *rest):
        g_sem = rest[0] if fctx.has_sem and rest else None
        backward(fctx.sdg, g_rgb, g_depth, g_opac, g_sem)
        fctx.sdg.release()
        return (None,) * 9


class DifferentiableRenderer:
    """torch.autograd entry: outputs are differentiable w.r.t. the grid's voxels; loss.backward() ACCUMULATES
    dL/dtheta into the grid's gradient channels (read them with Grid.channel(group, KIND_GRAD)).  The anchor
    tensor only connects the outputs to the autograd graph; it receives no gradient."""

    def __init__(self, grid: Grid):
        self.grid = grid
        self.anchor = torch.zeros(1, device=f"cuda:{grid.device}", requires_grad=True)

    def __call__(self, rays, n_samples: int, seed: int = 0, ray_id0: int = 0, stratified: bool = True,
                 mode: str = "recompute", bg=(0.0, 0.0, 0.0)):
        return _RenderFn.apply(self.anchor, self.grid, rays, n_samples, seed, ray_id0, stratified, mode, tuple(bg))
