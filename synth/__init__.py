"""Seeded synthetic inputs for the sparse-dense SDF renderer.

This module is the only code shared by the CUDA path's tests/bench and the CPU
oracle.  It produces INPUTS only: analytic indoor scenes (a signed distance
field, a smooth colour field and per-primitive labels), camera poses, analytic
depth maps, pinhole ray batches with their analytic targets, and per-voxel
grid contents for a given set of active blocks.  It contains none of the
method's arithmetic (no unprojection, quantisation, hashing, traversal,
sampling, interpolation, density transform, compositing, loss or optimiser).

The scenes stand in for the paper's ScanNet / 7-Scenes rooms, which are not
available: boxes, capped z-cylinders and spheres inside box-shaped rooms, with
metric sizes like the paper's indoor scenes (Sec. 4 "Setup": 8^3 blocks,
1-1.5 cm voxels, 640x480 images).

All arithmetic is float64 torch on the requested device, so the same code can
fill a room-scale grid on a GPU quickly and a tiny grid on the CPU.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional, Sequence, Tuple

import numpy as np
import torch

F64 = torch.float64

# ----------------------------------------------------------------------------
# Scene description
# ----------------------------------------------------------------------------


@dataclasses.dataclass
class Primitive:
    kind: str                      # "sphere" | "box" | "cylinder"
    center: Tuple[float, float, float]
    size: Tuple[float, float, float]  # sphere: (r,_,_); box: half extents; cylinder: (r, half_height, _)
    label: int


@dataclasses.dataclass
class Scene:
    name: str
    lo: Tuple[float, float, float]   # room interior min corner (m)
    hi: Tuple[float, float, float]   # room interior max corner (m)
    prims: List[Primitive]
    omega: np.ndarray                # (3, 3) colour spatial frequencies (rad/m), row = channel
    phase: np.ndarray                # (3,) colour phases
    seed: int

    @property
    def n_labels(self) -> int:
        return 1 + len(self.prims)


def _colour_params(rng: np.random.Generator):
    omega = rng.uniform(1.5, 6.0, size=(3, 3)) * rng.choice([-1.0, 1.0], size=(3, 3))
    phase = rng.uniform(0.0, 2.0 * math.pi, size=3)
    return omega, phase


def scene_tiny_room(seed: int = 0) -> Scene:
    """2x2x2 m cube room with a 0.5 m sphere at its centre (tiny analytic scene)."""
    rng = np.random.default_rng(seed)
    omega, phase = _colour_params(rng)
    return Scene("tiny_room", (0.0, 0.0, 0.0), (2.0, 2.0, 2.0),
                 [Primitive("sphere", (1.0, 1.0, 1.0), (0.5, 0.0, 0.0), 1)], omega, phase, seed)


def _floor_objects(rng, n, lo, hi, label0=1, size_range=(0.2, 1.2)):
    prims = []
    for i in range(n):
        kind = "box" if rng.random() < 0.6 else "cylinder"
        w = rng.uniform(*size_range, size=3)
        w[2] = min(w[2], (hi[2] - lo[2]) * 0.6)
        cx = rng.uniform(lo[0] + 0.3 + w[0] / 2, hi[0] - 0.3 - w[0] / 2)
        cy = rng.uniform(lo[1] + 0.3 + w[1] / 2, hi[1] - 0.3 - w[1] / 2)
        cz = lo[2] + w[2] / 2
        if kind == "box":
            prims.append(Primitive("box", (cx, cy, cz), (w[0] / 2, w[1] / 2, w[2] / 2), label0 + i))
        else:
            r = min(w[0], w[1]) / 2
            prims.append(Primitive("cylinder", (cx, cy, cz), (r, w[2] / 2, 0.0), label0 + i))
    return prims


def scene_room(seed: int = 0, size=(6.0, 6.0, 3.0), n_objects: int = 10) -> Scene:
    """Room of `size` metres with `n_objects` seeded boxes / z-cylinders (0.2-1.2 m) on the floor."""
    rng = np.random.default_rng(1000 + seed)
    omega, phase = _colour_params(rng)
    lo, hi = (0.0, 0.0, 0.0), tuple(float(s) for s in size)
    return Scene(f"room{seed}", lo, hi, _floor_objects(rng, n_objects, lo, hi), omega, phase, seed)


def scene_apartment(seed: int = 0, size=(20.0, 15.0, 3.0), n_furniture: int = 60) -> Scene:
    """20x15x3 m apartment: 6 rooms separated by 10 cm interior walls with 1 m door gaps,
    plus `n_furniture` seeded primitives."""
    rng = np.random.default_rng(5000 + seed)
    omega, phase = _colour_params(rng)
    lo, hi = (0.0, 0.0, 0.0), tuple(float(s) for s in size)
    H = hi[2]
    prims: List[Primitive] = []
    label = 1
    # 3 x 2 rooms: two interior x-walls and one interior y-wall, each with door gaps.
    xs = [hi[0] / 3 + rng.uniform(-1, 1), 2 * hi[0] / 3 + rng.uniform(-1, 1)]
    ymid = hi[1] / 2 + rng.uniform(-1, 1)
    t = 0.05  # half thickness
    for x in xs:          # wall along y at x, door gaps in each half
        cuts = [0.0]
        for (a, b) in ((0.0, ymid), (ymid, hi[1])):
            g = rng.uniform(a + 0.5, b - 1.5)
            cuts += [g, g + 1.0]
        cuts.append(hi[1])
        for k in range(0, len(cuts), 2):
            y0, y1 = cuts[k], cuts[k + 1]
            prims.append(Primitive("box", (x, (y0 + y1) / 2, H / 2), (t, (y1 - y0) / 2, H / 2), label))
            label += 1
    bounds = [0.0] + xs + [hi[0]]
    for k in range(3):    # wall along x at ymid, one door per room
        x0, x1 = bounds[k], bounds[k + 1]
        g = rng.uniform(x0 + 0.5, x1 - 1.5)
        for (a, b) in ((x0, g), (g + 1.0, x1)):
            prims.append(Primitive("box", ((a + b) / 2, ymid, H / 2), ((b - a) / 2, t, H / 2), label))
            label += 1
    rooms = [((bounds[i], y0), (bounds[i + 1], y1)) for i in range(3) for (y0, y1) in ((0.0, ymid), (ymid, hi[1]))]
    per_room = [n_furniture // 6 + (1 if i < n_furniture % 6 else 0) for i in range(6)]
    for (rlo, rhi), n in zip(rooms, per_room):
        sub = _floor_objects(rng, n, (rlo[0] + 0.15, rlo[1] + 0.15, 0.0), (rhi[0] - 0.15, rhi[1] - 0.15, H),
                             label0=label, size_range=(0.2, 1.0))
        prims += sub
        label += n
    return Scene(f"apartment{seed}", lo, hi, prims, omega, phase, seed)


# ----------------------------------------------------------------------------
# Analytic fields (inputs: the "true" scene the grid is filled from)
# ----------------------------------------------------------------------------


def _prim_sdf(p: Primitive, x: torch.Tensor) -> torch.Tensor:
    c = torch.tensor(p.center, dtype=F64, device=x.device)
    q = x - c
    if p.kind == "sphere":
        return q.norm(dim=-1) - p.size[0]
    if p.kind == "box":
        h = torch.tensor(p.size, dtype=F64, device=x.device)
        a = q.abs() - h
        outside = a.clamp(min=0).norm(dim=-1)
        inside = a.max(dim=-1).values.clamp(max=0)
        return outside + inside
    if p.kind == "cylinder":
        r, hh = p.size[0], p.size[1]
        dx = q[..., :2].norm(dim=-1) - r
        dz = q[..., 2].abs() - hh
        a = torch.stack([dx, dz], dim=-1)
        return a.clamp(min=0).norm(dim=-1) + a.max(dim=-1).values.clamp(max=0)
    raise ValueError(p.kind)


def scene_sdf(scene: Scene, x: torch.Tensor, with_label: bool = False):
    """Signed distance of free space (positive inside the room and outside every primitive).

    Room term: distance to the nearest wall, min over axes of (x-lo, hi-x).  Returns the SDF and,
    optionally, the label of the closest surface (0 = room shell, primitive label otherwise)."""
    lo = torch.tensor(scene.lo, dtype=F64, device=x.device)
    hi = torch.tensor(scene.hi, dtype=F64, device=x.device)
    d = torch.minimum(x - lo, hi - x).min(dim=-1).values
    lab = torch.zeros(d.shape, dtype=torch.int64, device=x.device) if with_label else None
    for p in scene.prims:
        dp = _prim_sdf(p, x)
        if with_label:
            lab = torch.where(dp < d, torch.full_like(lab, p.label), lab)
        d = torch.minimum(d, dp)
    return (d, lab) if with_label else d


def scene_colour(scene: Scene, x: torch.Tensor) -> torch.Tensor:
    """Smooth seeded colour field c(x) = 0.5 + 0.5 sin(omega_ch . x + phase_ch), in [0, 1]."""
    om = torch.tensor(scene.omega, dtype=F64, device=x.device)
    ph = torch.tensor(scene.phase, dtype=F64, device=x.device)
    return 0.5 + 0.5 * torch.sin(x @ om.T + ph)


# ----------------------------------------------------------------------------
# Grids: which blocks are active (analytic mode) and their voxel contents
# ----------------------------------------------------------------------------

def _local_offsets(device) -> torch.Tensor:
    """(512, 3) local voxel offsets in storage order: linear = lz*64 + ly*8 + lx."""
    i = torch.arange(512, device=device)
    return torch.stack([i % 8, (i // 8) % 8, i // 64], dim=-1)


def band_blocks(scene: Scene, voxel_size: float, band_voxels: int, device="cpu", chunk=1 << 14) -> np.ndarray:
    """Analytic block set: a block is active iff min over its 512 grid points of |sdf| <= band*vs.

    Returns int32 keys (M, 3) sorted by (z, y, x)."""
    L = 8 * voxel_size
    lo = np.floor((np.array(scene.lo) - 2 * L) / L).astype(np.int64)
    hi = np.floor((np.array(scene.hi) + 2 * L) / L).astype(np.int64)
    axes = [torch.arange(lo[a], hi[a] + 1, device=device) for a in range(3)]
    bz, by, bx = torch.meshgrid(axes[2], axes[1], axes[0], indexing="ij")
    cand = torch.stack([bx.reshape(-1), by.reshape(-1), bz.reshape(-1)], dim=-1)
    loc = _local_offsets(device)
    keep = []
    thr = band_voxels * voxel_size
    for s in range(0, cand.shape[0], chunk):
        k = cand[s:s + chunk]
        v = (k[:, None, :] * 8 + loc[None]).to(F64) * voxel_size
        d = scene_sdf(scene, v.reshape(-1, 3)).reshape(k.shape[0], 512)
        keep.append(k[(d.abs() <= thr).any(dim=1)])
    keys = torch.cat(keep).cpu().numpy().astype(np.int32)
    return keys


def voxel_positions(keys: np.ndarray, voxel_size: float, device="cpu") -> torch.Tensor:
    """World positions (N, 512, 3) of the grid points of each block (grid point v sits at v*vs)."""
    k = torch.as_tensor(np.asarray(keys), dtype=torch.int64, device=device)
    v = k[:, None, :] * 8 + _local_offsets(device)[None]
    return v.to(F64) * voxel_size


def fill_grid(scene: Scene, keys: np.ndarray, voxel_size: float, band_voxels: Optional[float], n_sem: int = 0,
              device="cpu", seed: int = 0, chunk_blocks: int = 8192):
    """Per-voxel grid contents for the blocks `keys` (in index order).

    Returns dict with float64 tensors: sdf (N,512), rgb (N,512,3) and, if n_sem, sem (N,512,n_sem).
    sdf is clamped to +-band*vs (truncation) unless band_voxels is None.
    Semantic logits: 4*onehot(label mod n_sem) + N(0, 0.5^2), seeded."""
    N = int(np.asarray(keys).shape[0])
    sdf = torch.empty((N, 512), dtype=F64, device=device)
    rgb = torch.empty((N, 512, 3), dtype=F64, device=device)
    sem = torch.empty((N, 512, n_sem), dtype=F64, device=device) if n_sem else None
    gen = torch.Generator(device=device)
    gen.manual_seed(7919 + seed)
    keys_t = np.asarray(keys)
    for s in range(0, N, chunk_blocks):
        x = voxel_positions(keys_t[s:s + chunk_blocks], voxel_size, device)
        d, lab = scene_sdf(scene, x.reshape(-1, 3), with_label=True)
        d = d.reshape(x.shape[:2])
        if band_voxels is not None:
            t = band_voxels * voxel_size
            d = d.clamp(-t, t)
        sdf[s:s + chunk_blocks] = d
        rgb[s:s + chunk_blocks] = scene_colour(scene, x.reshape(-1, 3)).reshape(x.shape)
        if n_sem:
            oh = torch.nn.functional.one_hot(lab.reshape(x.shape[:2]) % n_sem, n_sem).to(F64)
            noise = torch.randn(oh.shape, generator=gen, dtype=F64, device=device) * 0.5
            sem[s:s + chunk_blocks] = 4.0 * oh + noise
    out = {"sdf": sdf, "rgb": rgb}
    if n_sem:
        out["sem"] = sem
    return out


def plane_grid(normal, offset: float, voxel_size: float, extent_blocks=((-2, 2), (-2, 2), (-2, 2)),
               slab_blocks: int = 1):
    """Blocks around the plane n.x = offset with an UNCLAMPED linear field theta(v) = n.(v vs) - offset.

    A block is kept when its centre is within slab_blocks block-lengths of the plane.  Returns (keys, sdf, rgb)
    with rgb a constant-free linear colour a.x + b (float64)."""
    n = np.asarray(normal, dtype=np.float64)
    n = n / np.linalg.norm(n)
    L = 8 * voxel_size
    rng = [np.arange(a, b + 1) for a, b in extent_blocks]
    keys = []
    for bz in rng[2]:
        for by in rng[1]:
            for bx in rng[0]:
                c = (np.array([bx, by, bz]) + 0.5) * L
                if abs(c @ n - offset) <= slab_blocks * L:
                    keys.append((bx, by, bz))
    keys = np.array(keys, dtype=np.int32)
    x = voxel_positions(keys, voxel_size).numpy()
    sdf = x @ n - offset
    rgb = np.stack([0.3 + 0.1 * x[..., 0], 0.5 + 0.05 * x[..., 1], 0.2 + 0.07 * x[..., 2]], axis=-1)
    return keys, sdf, rgb


# ----------------------------------------------------------------------------
# Cameras, depth maps, rays
# ----------------------------------------------------------------------------


def intrinsics(W: int, H: int, fov_deg: float = 60.0):
    """Pinhole (fx, fy, cx, cy) with horizontal field of view fov_deg."""
    fx = 0.5 * W / math.tan(math.radians(fov_deg) / 2)
    return (fx, fx, W / 2.0, H / 2.0)


def look_at(eye, target, up=(0.0, 0.0, 1.0)) -> np.ndarray:
    """Camera-to-world 3x4 [R|t], OpenCV axes (x right, y down, z forward)."""
    eye, target, up = (np.asarray(v, dtype=np.float64) for v in (eye, target, up))
    f = target - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, up)
    if np.linalg.norm(r) < 1e-6:
        r = np.cross(f, np.array([0.0, 1.0, 0.0]))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    R = np.stack([r, d, f], axis=1)
    return np.concatenate([R, eye[:, None]], axis=1)


def random_poses(scene: Scene, n: int, seed: int = 0, clearance: float = 0.3, max_tries: int = 100000):
    """n seeded camera poses inside the room, >= clearance from every surface, looking at a seeded point."""
    rng = np.random.default_rng(20000 + seed)
    lo, hi = np.array(scene.lo), np.array(scene.hi)
    poses = []
    tries = 0
    while len(poses) < n and tries < max_tries:
        tries += 1
        eye = rng.uniform(lo + clearance, hi - clearance)
        eye[2] = rng.uniform(lo[2] + 0.8, min(hi[2] - clearance, lo[2] + 2.0))
        if float(scene_sdf(scene, torch.tensor(eye[None]))[0]) < clearance:
            continue
        tgt = rng.uniform(lo + 0.2, hi - 0.2)
        tgt[2] = rng.uniform(lo[2] + 0.2, hi[2] - 0.5)
        if np.linalg.norm(tgt - eye) < 0.5:
            continue
        poses.append(look_at(eye, tgt))
    if len(poses) < n:
        raise RuntimeError("could not place cameras")
    return np.stack(poses)


def _ray_box_exit_inside(o, d, lo, hi):
    inv = 1.0 / d
    t1 = (lo - o) * inv
    t2 = (hi - o) * inv
    return torch.maximum(t1, t2).min(dim=-1).values


def _ray_prim(p: Primitive, o, d):
    """Nearest positive hit distance of rays o + t d (|d| arbitrary) with primitive p; inf if none."""
    inf = torch.full(o.shape[:-1], float("inf"), dtype=F64, device=o.device)
    c = torch.tensor(p.center, dtype=F64, device=o.device)
    q = o - c
    if p.kind == "sphere":
        a = (d * d).sum(-1)
        b = (q * d).sum(-1)
        cc = (q * q).sum(-1) - p.size[0] ** 2
        disc = b * b - a * cc
        s = torch.sqrt(disc.clamp(min=0))
        t = (-b - s) / a
        return torch.where((disc >= 0) & (t > 0), t, inf)
    if p.kind == "box":
        h = torch.tensor(p.size, dtype=F64, device=o.device)
        inv = 1.0 / d
        t1 = (-h - q) * inv
        t2 = (h - q) * inv
        tn = torch.minimum(t1, t2).max(dim=-1).values
        tf = torch.maximum(t1, t2).min(dim=-1).values
        return torch.where((tn <= tf) & (tn > 0), tn, inf)
    if p.kind == "cylinder":
        r, hh = p.size[0], p.size[1]
        a = (d[..., :2] ** 2).sum(-1)
        b = (q[..., :2] * d[..., :2]).sum(-1)
        cc = (q[..., :2] ** 2).sum(-1) - r * r
        disc = b * b - a * cc
        s = torch.sqrt(disc.clamp(min=0))
        ts = (-b - s) / a.clamp(min=1e-300)
        z = q[..., 2] + ts * d[..., 2]
        side = torch.where((disc >= 0) & (ts > 0) & (z.abs() <= hh) & (a > 0), ts, inf)
        best = side
        for zc in (hh, -hh):
            tc = (zc - q[..., 2]) / d[..., 2]
            xy = q[..., :2] + tc[..., None] * d[..., :2]
            ok = (tc > 0) & ((xy ** 2).sum(-1) <= r * r) & ((q[..., 2] - zc) * d[..., 2] < 0)
            best = torch.minimum(best, torch.where(ok, tc, inf))
        return best
    raise ValueError(p.kind)


def ray_hit(scene: Scene, o: torch.Tensor, d: torch.Tensor) -> torch.Tensor:
    """Distance t (in units of |d|) to the first surface along o + t d, for rays starting inside the room."""
    lo = torch.tensor(scene.lo, dtype=F64, device=o.device)
    hi = torch.tensor(scene.hi, dtype=F64, device=o.device)
    t = _ray_box_exit_inside(o, d, lo, hi)
    for p in scene.prims:
        t = torch.minimum(t, _ray_prim(p, o, d))
    return t


def pixel_dirs_cam(W: int, H: int, K, device="cpu") -> torch.Tensor:
    """(H*W, 3) camera-frame directions ((u+0.5-cx)/fx, (v+0.5-cy)/fy, 1), row-major over (v, u)."""
    fx, fy, cx, cy = K
    v, u = torch.meshgrid(torch.arange(H, device=device, dtype=F64), torch.arange(W, device=device, dtype=F64),
                          indexing="ij")
    return torch.stack([(u + 0.5 - cx) / fx, (v + 0.5 - cy) / fy, torch.ones_like(u)], dim=-1).reshape(-1, 3)


def depth_map(scene: Scene, Twc: np.ndarray, W: int, H: int, K, device="cpu") -> torch.Tensor:
    """Analytic z-depth map (H, W) float32 of the scene seen from camera-to-world pose Twc."""
    R = torch.tensor(Twc[:, :3], dtype=F64, device=device)
    t = torch.tensor(Twc[:, 3], dtype=F64, device=device)
    dc = pixel_dirs_cam(W, H, K, device)
    dw = dc @ R.T                      # z-component of dc is 1, so the hit t is the z-depth
    o = t.expand_as(dw)
    z = ray_hit(scene, o, dw)
    return z.reshape(H, W).to(torch.float32)


def rgbd_frame(scene: Scene, Twc: np.ndarray, W: int, H: int, K, n_sem: int = 0, seed: int = 0, device="cpu"):
    """One analytic RGB-D(-logit) frame: z-depth (H, W), the colour at each pixel's first hit (H, W, 3) and, if
    n_sem, logits 4*onehot(hit label mod n_sem) + N(0, 0.5^2) (H, W, n_sem), all float32.  Pixels whose ray
    leaves the scene get depth inf and colour 0."""
    R = torch.tensor(Twc[:, :3], dtype=F64, device=device)
    t = torch.tensor(Twc[:, 3], dtype=F64, device=device)
    dc = pixel_dirs_cam(W, H, K, device)
    dw = dc @ R.T
    o = t.expand_as(dw)
    z = ray_hit(scene, o, dw)
    hit = torch.isfinite(z)
    x = o + torch.where(hit, z, torch.zeros_like(z))[:, None] * dw
    rgb = torch.where(hit[:, None], scene_colour(scene, x), torch.zeros_like(x))
    out = {"depth": z.reshape(H, W).to(torch.float32), "rgb": rgb.reshape(H, W, 3).to(torch.float32)}
    if n_sem:
        _, lab = scene_sdf(scene, x, with_label=True)
        g = torch.Generator(device="cpu")
        g.manual_seed(70000 + seed)
        noise = torch.randn((H * W, n_sem), generator=g, dtype=F64).to(device) * 0.5
        logits = 4.0 * torch.nn.functional.one_hot(lab % n_sem, n_sem).to(F64) + noise
        out["sem"] = logits.reshape(H, W, n_sem).to(torch.float32)
    return out


def pack_rays(o: torch.Tensor, d: torch.Tensor, tnear: float = 0.05, tfar: float = 1.0e3) -> torch.Tensor:
    """Ray records (n, 8) float32: ox, oy, oz, tnear, dx, dy, dz, tfar."""
    n = o.shape[0]
    r = torch.empty((n, 8), dtype=torch.float32, device=o.device)
    r[:, 0:3] = o.to(torch.float32)
    r[:, 3] = tnear
    r[:, 4:7] = d.to(torch.float32)
    r[:, 7] = tfar
    return r


def view_rays(Twc: np.ndarray, W: int, H: int, K, device="cpu", tnear=0.05, tfar=1.0e3) -> torch.Tensor:
    """All pixels of one view as unit-direction rays (H*W, 8) float32."""
    R = torch.tensor(Twc[:, :3], dtype=F64, device=device)
    t = torch.tensor(Twc[:, 3], dtype=F64, device=device)
    dw = pixel_dirs_cam(W, H, K, device) @ R.T
    dw = dw / dw.norm(dim=-1, keepdim=True)
    return pack_rays(t.expand_as(dw), dw, tnear, tfar)


def training_batch(scene: Scene, poses: np.ndarray, W: int, H: int, K, n_rays: int, seed: int = 0,
                   device="cpu", n_sem: int = 0, tnear=0.05, tfar=1.0e3, order: str = "drawn"):
    """n_rays rays drawn uniformly (seeded) over the pixels of the given views, with analytic targets.

    order="drawn" keeps the draw order; order="pixel" lists the same rays grouped by view and sorted by pixel
    index, as a loader that draws rays per image would hand them over (same set of rays, other order).
    Returns dict: rays (n,8) f32, rgb (n,3) f32 = colour at the first hit, depth (n,) f32 = hit distance
    along the unit ray, and, if n_sem, sem (n, n_sem) f32 = 4*onehot(hit label mod n_sem)."""
    g = torch.Generator(device="cpu")
    g.manual_seed(40000 + seed)
    view = torch.randint(0, poses.shape[0], (n_rays,), generator=g)
    pix = torch.randint(0, W * H, (n_rays,), generator=g)
    if order == "pixel":
        perm = torch.argsort(view * (W * H) + pix, stable=True)
        view, pix = view[perm], pix[perm]
    elif order != "drawn":
        raise ValueError(order)
    u = (pix % W).to(F64)
    v = (pix // W).to(F64)
    fx, fy, cx, cy = K
    dc = torch.stack([(u + 0.5 - cx) / fx, (v + 0.5 - cy) / fy, torch.ones_like(u)], dim=-1).to(device)
    P = torch.tensor(poses, dtype=F64, device=device)[view.to(device)]
    dw = torch.einsum("nij,nj->ni", P[:, :, :3], dc)
    dw = dw / dw.norm(dim=-1, keepdim=True)
    o = P[:, :, 3]
    th = ray_hit(scene, o, dw)
    x = o + th[:, None] * dw
    out = {"rays": pack_rays(o, dw, tnear, tfar), "rgb": scene_colour(scene, x).to(torch.float32),
           "depth": th.to(torch.float32)}
    if n_sem:
        _, lab = scene_sdf(scene, x, with_label=True)
        out["sem"] = (4.0 * torch.nn.functional.one_hot(lab % n_sem, n_sem)).to(torch.float32)
    return out


def random_rays_through(keys: np.ndarray, voxel_size: float, n: int, seed: int = 0, tnear=0.0, tfar=1.0e3):
    """n seeded rays that start outside the AABB of `keys` and aim at random points inside it (unit dirs)."""
    rng = np.random.default_rng(60000 + seed)
    L = 8 * voxel_size
    lo = keys.min(axis=0) * L
    hi = (keys.max(axis=0) + 1) * L
    c = (lo + hi) / 2
    rad = np.linalg.norm(hi - lo) * 0.75 + L
    tgt = rng.uniform(lo, hi, size=(n, 3))
    dirn = rng.normal(size=(n, 3))
    dirn /= np.linalg.norm(dirn, axis=1, keepdims=True)
    o = c + dirn * rad
    d = tgt - o
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    return pack_rays(torch.tensor(o), torch.tensor(d), tnear, tfar)
