"""sdg: differentiable volume rendering of SDF + colour + semantic channels in a globally sparse, locally
dense voxel-block grid (arXiv 2305.13220), as hand-written sm_103a CUDA behind a C ABI (include/sdg.h).

This package is a thin binding: it marshals torch tensors (device memory, streams) to libsdg.so.  Importing it
loads libsdg.so and raises ImportError if the library has not been built -- there is no CPU fallback."""
from . import _abi
from ._abi import SdgError

_abi.lib()  # fail loudly at import when the CUDA library is missing

from .grid import Grid, render_opts  # noqa: E402
from .render import (DifferentiableRenderer, RenderContext, backward, loss_depth_ssi, loss_l1,  # noqa: E402
                     render, trace, trace_view, train_prepare, train_step_rays, train_step_rays_normal)
from .serve import Server  # noqa: E402

__all__ = ["Grid", "render_opts", "render", "trace", "trace_view", "train_prepare", "backward", "loss_l1", "loss_depth_ssi", "train_step_rays",
           "train_step_rays_normal",
           "DifferentiableRenderer", "RenderContext", "SdgError", "Server"]
