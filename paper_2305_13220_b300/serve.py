"""Thin wrapper of the continuous-batching render server (sdg_server_* in include/sdg.h)."""
from __future__ import annotations

import ctypes as C
from typing import Sequence

import torch

from . import _abi as A
from .grid import Grid


class Server:
    def __init__(self, hbm_budget_bytes: int = 1 << 30, max_slots: int = 16, n_streams: int = 4,
                 chunk_rays: int = 4096, max_batch_rays: int = 1 << 18, device: int = 0):
        o = A.ServerOpts(hbm_budget_bytes=hbm_budget_bytes, max_slots=max_slots, n_streams=n_streams,
                         chunk_rays=chunk_rays, max_batch_rays=max_batch_rays, device=device, reserved=0)
        h = C.c_void_p()
        A.call("sdg_server_create", C.byref(o), C.byref(h))
        self._h = h
        self.device = device
        self._scenes = []

    def add_scene(self, grid: Grid) -> int:
        i = C.c_int32()
        A.call("sdg_server_add_scene", self._h, grid.handle, C.byref(i))
        self._scenes.append(grid)
        return i.value

    def submit(self, scene_id: int, H: int, W: int, K: Sequence[float], Twc, n_samples: int = 128, seed: int = 0,
               stratified: bool = True, tnear: float = 0.05, tfar: float = 1.0e3) -> int:
        q = A.Request(scene_id=scene_id, H=H, W=W, n_samples=n_samples, seed=seed, stratified=int(stratified),
                      tnear=tnear, tfar=tfar)
        for i, v in enumerate(K):
            q.K[i] = float(v)
        for i, v in enumerate(torch.as_tensor(Twc, dtype=torch.float64).reshape(12).tolist()):
            q.Twc[i] = v
        t = C.c_uint64()
        A.call("sdg_server_submit", self._h, C.byref(q), C.byref(t))
        return t.value

    def poll(self, ticket: int):
        r = A.Result()
        code = A.lib().sdg_server_poll(self._h, ticket, C.byref(r))
        if code == A.ERR_BUSY:
            return None
        A.check(code, "sdg_server_poll")
        return r

    def wait(self, ticket: int, timeout_ms: int = 60000) -> A.Result:
        r = A.Result()
        A.call("sdg_server_wait", self._h, ticket, int(timeout_ms), C.byref(r))
        return r

    def result_tensors(self, r: A.Result, copy: bool = True):
        """(rgb [H*W,3], depth [H*W], opac [H*W]) views of a finished result (copied unless copy=False)."""
        from .grid import _DevArray
        n = r.H * r.W
        dev = f"cuda:{self.device}"
        mk = lambda p, shape: torch.as_tensor(_DevArray(p, shape, "<f4", self), device=dev)
        out = mk(r.rgb, (n, 3)), mk(r.depth, (n,)), mk(r.opac, (n,))
        return tuple(t.clone() for t in out) if copy else out

    def release(self, ticket: int):
        A.call("sdg_server_release", self._h, ticket)

    def stats(self) -> A.ServerStats:
        s = A.ServerStats()
        A.call("sdg_server_get_stats", self._h, C.byref(s))
        return s

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            A.lib().sdg_server_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
