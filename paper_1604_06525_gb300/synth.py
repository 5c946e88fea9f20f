"""Seeded synthetic problem instances shaped like the paper's workloads.

The paper's own images and meshes (Sec. 8, Fig. 21) are not available, so every
input is generated here from a seed.  This module only builds *inputs*: grids,
rest shapes, handle lists, masks, noise images and icosphere meshes.  It holds
none of the solver's arithmetic (no residuals, no derivatives, no PCG), and it
is the only module that both the FP64 CPU oracle and the CUDA path use.

Conventions shared by both sides (each one is a reading of the paper):

* ARAP image warping (Fig. 24): unknowns per pixel are the displacement
  (dx, dy) of the pixel from its rest position UrShape plus a rotation angle
  theta; Offset = UrShape + (dx, dy).  UrShape(x, y) = (x, y) in pixel units,
  but it is stored as an array and must be read as one.  Handles are distinct
  pixels drawn without replacement; each handle's target is a displacement.
* Poisson image editing (Fig. 27): four channels; the mask is nonzero on the
  fixed (excluded) pixels; the free region is one random rectangle covering
  30% of the image.  X0 is the target image, T the guidance image.
* ARAP mesh deformation (Fig. 25): a subdivided icosphere of unit radius with
  every undirected edge present in both directions, sorted by (v0, v1).
  Unknowns per vertex are the displacement from UrShape and three Euler angles.

All arrays are float32 / int32 / uint8 and laid out as planes (struct of
arrays): a grid plane is (H, W) row-major, a mesh plane has V entries.
"""
from __future__ import annotations

from dataclasses import dataclass, field
import math

import numpy as np

BASE_SEED = 1604


# ----------------------------------------------------------------------------
# problem containers (plain data)
# ----------------------------------------------------------------------------
@dataclass
class WarpProblem:
    """ARAP image warping instance (Fig. 24).

    x0 planes: 0 = dx, 1 = dy, 2 = theta; each (H, W) float32.
    urshape planes: 0 = rest x, 1 = rest y; each (H, W) float32.
    mask: (H, W) uint8, nonzero = pixel excluded, or None (all pixels free).
    handle_idx: (n,) int32 pixel indices y * W + x (distinct).
    handle_target: (n, 2) float32 target displacements.
    """
    W: int
    H: int
    urshape: np.ndarray
    x0: np.ndarray
    handle_idx: np.ndarray
    handle_target: np.ndarray
    mask: np.ndarray | None = None
    w_reg: float = 1.0
    w_fit: float = 100.0
    seed: int = BASE_SEED
    kind: str = field(default="warp", init=False)

    @property
    def n_unknowns(self) -> int:
        return 3 * self.W * self.H


@dataclass
class PoissonProblem:
    """Poisson image editing instance (Fig. 27), C = 4 channels.

    x0: (4, H, W) float32 initial image (the target image everywhere).
    guide: (4, H, W) float32 guidance image T.
    mask: (H, W) uint8, nonzero = fixed pixel (excluded from the solve).
    """
    W: int
    H: int
    x0: np.ndarray
    guide: np.ndarray
    mask: np.ndarray
    seed: int = BASE_SEED
    kind: str = field(default="poisson", init=False)

    @property
    def n_unknowns(self) -> int:
        return 4 * self.W * self.H


@dataclass
class MeshProblem:
    """ARAP mesh deformation instance (Fig. 25).

    urshape: (3, V) float32 rest positions.
    v0, v1: (E,) int32 directed edges, sorted by (v0, v1).
    x0 planes: 0..2 = displacement, 3..5 = Euler angles; (6, V) float32.
    handle_idx: (n,) int32 vertex ids (distinct); handle_target: (n, 3)
    float32 target displacements.
    """
    V: int
    urshape: np.ndarray
    v0: np.ndarray
    v1: np.ndarray
    x0: np.ndarray
    handle_idx: np.ndarray
    handle_target: np.ndarray
    w_reg: float = 1.0
    w_fit: float = 100.0
    level: int = -1
    seed: int = BASE_SEED
    kind: str = field(default="mesh", init=False)

    @property
    def E(self) -> int:
        return int(self.v0.shape[0])

    @property
    def n_unknowns(self) -> int:
        return 6 * self.V


@dataclass
class WarpGraphProblem:
    """ARAP image warping written on an explicit graph (the explicit side of
    the implicit-grid vs explicit-graph comparison, Fig. 18): one vertex per
    pixel, the stencil neighbourhood as directed edges.

    urshape: (2, V) float32 rest positions.
    v0, v1: (E,) int32 directed edges, sorted by (v0, v1).
    x0 planes: 0 = dx, 1 = dy, 2 = theta; (3, V) float32.
    handle_idx: (n,) int32 vertex ids (distinct); handle_target: (n, 2)
    float32 target displacements.
    """
    V: int
    urshape: np.ndarray
    v0: np.ndarray
    v1: np.ndarray
    x0: np.ndarray
    handle_idx: np.ndarray
    handle_target: np.ndarray
    w_reg: float = 1.0
    w_fit: float = 100.0
    seed: int = BASE_SEED
    kind: str = field(default="warp_graph", init=False)

    @property
    def E(self) -> int:
        return int(self.v0.shape[0])

    @property
    def n_unknowns(self) -> int:
        return 3 * self.V


@dataclass
class VolumeProblem:
    """Volumetric ARAP deformation instance (Fig. 31): a W x H x D voxel grid,
    7-point stencil.  Voxel index (z * H + y) * W + x.

    urshape: (3, V) float32 rest positions (read as an array).
    x0 planes: 0..2 = displacement, 3..5 = Euler angles; (6, V) float32.
    handle_idx: (n,) int32 voxel ids (distinct); handle_target: (n, 3)
    float32 target displacements (the constrained voxels of Fig. 31).
    """
    W: int
    H: int
    D: int
    urshape: np.ndarray
    x0: np.ndarray
    handle_idx: np.ndarray
    handle_target: np.ndarray
    w_reg: float = 1.0
    w_fit: float = 100.0
    seed: int = BASE_SEED
    kind: str = field(default="volume", init=False)

    @property
    def V(self) -> int:
        return self.W * self.H * self.D

    @property
    def n_unknowns(self) -> int:
        return 6 * self.V


# ----------------------------------------------------------------------------
# image warping
# ----------------------------------------------------------------------------
def warp_problem(W: int, H: int, n_handles: int, seed: int = BASE_SEED,
                 max_disp: float = 8.0, mask: np.ndarray | None = None,
                 w_reg: float = 1.0, w_fit: float = 100.0,
                 x0_noise: float = 0.0) -> WarpProblem:
    """ARAP warp on a W x H grid with `n_handles` seeded handle constraints.

    Handle pixels are distinct (drawn without replacement) and avoid masked
    pixels; target displacements are uniform in [-max_disp, max_disp]^2.
    The initial state is the rest shape (dx = dy = theta = 0) unless
    x0_noise > 0, which draws dx, dy, theta uniform in +-x0_noise (tests).
    """
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:H, 0:W]
    urshape = np.stack([xs, ys]).astype(np.float32)
    free = np.arange(W * H) if mask is None else np.flatnonzero(mask.reshape(-1) == 0)
    n_handles = min(n_handles, free.size)
    hidx = np.sort(rng.choice(free, size=n_handles, replace=False)).astype(np.int32)
    htgt = rng.uniform(-max_disp, max_disp, size=(n_handles, 2)).astype(np.float32)
    x0 = np.zeros((3, H, W), np.float32)
    if x0_noise > 0:
        x0[:] = rng.uniform(-x0_noise, x0_noise, size=x0.shape).astype(np.float32)
    m = None if mask is None else np.ascontiguousarray(mask, dtype=np.uint8)
    return WarpProblem(W, H, urshape, x0, hidx, htgt, m, float(w_reg), float(w_fit), seed)


def random_mask(W: int, H: int, frac: float, seed: int) -> np.ndarray:
    """Bernoulli(frac) mask of excluded pixels (tests of the masked stencil)."""
    rng = np.random.default_rng(seed)
    return (rng.random((H, W)) < frac).astype(np.uint8)


def warp_graph_from_grid(prob: WarpProblem) -> WarpGraphProblem:
    """The same warp as an explicit graph: vertex y * W + x per pixel, a
    directed edge (k, k + d) for every stencil direction d whose neighbour is
    inside the image with both pixels unmasked; handles on masked pixels are
    dropped (their pixels carry no unknowns in the grid form either)."""
    W, H = prob.W, prob.H
    mask = np.zeros((H, W), bool) if prob.mask is None else (prob.mask != 0)
    ys, xs = np.mgrid[0:H, 0:W]
    a, b = [], []
    for ox, oy in ((1, 0), (-1, 0), (0, 1), (0, -1)):
        nx, ny = xs + ox, ys + oy
        inb = (nx >= 0) & (nx < W) & (ny >= 0) & (ny < H)
        nxc, nyc = np.clip(nx, 0, W - 1), np.clip(ny, 0, H - 1)
        ok = inb & ~mask & ~mask[nyc, nxc]
        a.append((ys * W + xs)[ok])
        b.append((nyc * W + nxc)[ok])
    v0 = np.concatenate(a).astype(np.int64)
    v1 = np.concatenate(b).astype(np.int64)
    order = np.lexsort((v1, v0))
    keep = ~mask.reshape(-1)[prob.handle_idx]
    return WarpGraphProblem(V=W * H, urshape=prob.urshape.reshape(2, -1).astype(np.float32).copy(),
                            v0=v0[order].astype(np.int32), v1=v1[order].astype(np.int32),
                            x0=prob.x0.reshape(3, -1).astype(np.float32).copy(),
                            handle_idx=prob.handle_idx[keep].astype(np.int32).copy(),
                            handle_target=prob.handle_target[keep].astype(np.float32).copy(),
                            w_reg=prob.w_reg, w_fit=prob.w_fit, seed=prob.seed)


def warp_handle_count(W: int, H: int) -> int:
    """Handles for the batched warps: max(8, round(64 * px / 1024^2))."""
    return max(8, int(round(64.0 * W * H / float(1024 * 1024))))


# ----------------------------------------------------------------------------
# Poisson image editing
# ----------------------------------------------------------------------------
def smooth_noise(W: int, H: int, channels: int, seed: int, cell: int = 32) -> np.ndarray:
    """Uniform [0,1] noise on a coarse lattice (one node per `cell` pixels),
    bilinearly upsampled to (channels, H, W) float32."""
    rng = np.random.default_rng(seed)
    gh = max(2, -(-H // cell) + 1)
    gw = max(2, -(-W // cell) + 1)
    lat = rng.random((channels, gh, gw))
    fy = np.arange(H, dtype=np.float64) / cell
    fx = np.arange(W, dtype=np.float64) / cell
    y0 = np.minimum(np.floor(fy).astype(np.int64), gh - 2)
    x0 = np.minimum(np.floor(fx).astype(np.int64), gw - 2)
    ty = (fy - y0)[:, None]
    tx = (fx - x0)[None, :]
    out = np.empty((channels, H, W), np.float32)
    for c in range(channels):
        a = lat[c][y0][:, x0]
        b = lat[c][y0][:, x0 + 1]
        cc = lat[c][y0 + 1][:, x0]
        d = lat[c][y0 + 1][:, x0 + 1]
        out[c] = ((1 - ty) * ((1 - tx) * a + tx * b) + ty * ((1 - tx) * cc + tx * d)).astype(np.float32)
    return out


def free_rectangle_mask(W: int, H: int, frac: float, rng: np.random.Generator) -> np.ndarray:
    """Mask with one free (zero) rectangle of area round(frac*W*H); aspect
    ratio log-uniform in [1/2, 2]; position uniform inside the image."""
    area = max(1, int(round(frac * W * H)))
    aspect = math.exp(rng.uniform(math.log(0.5), math.log(2.0)))
    rw = int(min(W, max(1, round(math.sqrt(area * aspect)))))
    rh = int(min(H, max(1, round(area / rw))))
    x0 = int(rng.integers(0, W - rw + 1))
    y0 = int(rng.integers(0, H - rh + 1))
    mask = np.ones((H, W), np.uint8)
    mask[y0:y0 + rh, x0:x0 + rw] = 0
    return mask


def poisson_problem(W: int, H: int, seed: int = BASE_SEED, free_frac: float = 0.3,
                    mask: np.ndarray | None = None) -> PoissonProblem:
    """Poisson editing on W x H x 4: target = smooth noise (seed), guidance =
    smooth noise (seed + 1), free region = random rectangle (30% of pixels)."""
    rng = np.random.default_rng(seed + 2)
    x0 = smooth_noise(W, H, 4, seed)
    guide = smooth_noise(W, H, 4, seed + 1)
    m = free_rectangle_mask(W, H, free_frac, rng) if mask is None else np.ascontiguousarray(mask, np.uint8)
    return PoissonProblem(W, H, x0, guide, m, seed)


# ----------------------------------------------------------------------------
# icosphere mesh
# ----------------------------------------------------------------------------
def _icosahedron():
    phi = (1.0 + math.sqrt(5.0)) / 2.0
    v = []
    for a in (-1.0, 1.0):
        for b in (-phi, phi):
            v += [(a, b, 0.0), (0.0, a, b), (b, 0.0, a)]
    v = np.array(v, np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    # the 20 faces are the triangles of the convex hull of the 12 vertices
    from scipy.spatial import ConvexHull
    faces = np.sort(ConvexHull(v).simplices.astype(np.int64), axis=1)
    faces = faces[np.lexsort((faces[:, 2], faces[:, 1], faces[:, 0]))]
    return v, faces


def icosphere(level: int):
    """Unit icosphere after `level` midpoint subdivisions.

    V = 10 * 4^level + 2 vertices.  New vertices are appended per level in the
    order of their edge key (min endpoint, max endpoint).  Returns (verts
    (V, 3) float64, faces (F, 3) int64)."""
    verts, faces = _icosahedron()
    for _ in range(level):
        nv = verts.shape[0]
        e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
        key = np.minimum(e[:, 0], e[:, 1]) * nv + np.maximum(e[:, 0], e[:, 1])
        ukey, inv = np.unique(key, return_inverse=True)
        a = ukey // nv
        b = ukey % nv
        mid = verts[a] + verts[b]
        mid /= np.linalg.norm(mid, axis=1, keepdims=True)
        nf = faces.shape[0]
        m01 = nv + inv[0:nf]
        m12 = nv + inv[nf:2 * nf]
        m20 = nv + inv[2 * nf:3 * nf]
        f0, f1, f2 = faces[:, 0], faces[:, 1], faces[:, 2]
        faces = np.concatenate([
            np.stack([f0, m01, m20], 1), np.stack([f1, m12, m01], 1),
            np.stack([f2, m20, m12], 1), np.stack([m01, m12, m20], 1)])
        verts = np.concatenate([verts, mid])
    return verts, faces


def directed_edges(faces: np.ndarray, n_vertices: int):
    """Every undirected mesh edge in both directions, sorted by (v0, v1)."""
    e = np.concatenate([faces[:, [0, 1]], faces[:, [1, 2]], faces[:, [2, 0]]])
    key = np.unique(np.minimum(e[:, 0], e[:, 1]) * n_vertices + np.maximum(e[:, 0], e[:, 1]))
    a = key // n_vertices
    b = key % n_vertices
    v0 = np.concatenate([a, b])
    v1 = np.concatenate([b, a])
    order = np.lexsort((v1, v0))
    return v0[order].astype(np.int32), v1[order].astype(np.int32)


@dataclass
class EmbeddedProblem:
    """Embedded deformation instance (Fig. 28): a mesh whose vertices carry a
    displacement and a full 3x3 matrix.

    urshape: (3, V) float32 rest positions; v0, v1: (E,) int32 directed edges
    sorted by (v0, v1).  x0 planes: 0..2 = displacement, 3..11 = the matrix
    row-major (R00, R01, R02, R10, ..., R22); (12, V) float32, identity
    matrices at the start.  handle_idx / handle_target as MeshProblem.
    """
    V: int
    urshape: np.ndarray
    v0: np.ndarray
    v1: np.ndarray
    x0: np.ndarray
    handle_idx: np.ndarray
    handle_target: np.ndarray
    w_reg: float = 1.0
    w_fit: float = 100.0
    w_rot: float = 1.0
    level: int = -1
    seed: int = BASE_SEED
    kind: str = field(default="embedded", init=False)

    @property
    def E(self) -> int:
        return int(self.v0.shape[0])

    @property
    def n_unknowns(self) -> int:
        return 12 * self.V


def embedded_problem(level: int, seed: int = BASE_SEED, handle_frac: float = 0.01, max_off: float = 0.1,
                     w_reg: float = 1.0, w_fit: float = 100.0, w_rot: float = 1.0,
                     x0_noise: float = 0.0) -> EmbeddedProblem:
    """Embedded deformation on a level-`level` icosphere: the handles of
    mesh_problem(level, seed, handle_frac, max_off), displacement 0 and
    identity matrices at the start (optionally perturbed by x0_noise)."""
    m = mesh_problem(level, seed=seed, handle_frac=handle_frac, max_off=max_off, w_reg=w_reg, w_fit=w_fit)
    x0 = np.zeros((12, m.V), np.float32)
    x0[3] = x0[7] = x0[11] = 1.0
    if x0_noise > 0:
        rng = np.random.default_rng(seed + 7)
        x0 += rng.uniform(-x0_noise, x0_noise, size=x0.shape).astype(np.float32)
    return EmbeddedProblem(m.V, m.urshape, m.v0, m.v1, x0, m.handle_idx, m.handle_target, float(w_reg),
                           float(w_fit), float(w_rot), level, seed)


def mesh_problem(level: int, seed: int = BASE_SEED, handle_frac: float = 0.01,
                 max_off: float = 0.1, w_reg: float = 1.0, w_fit: float = 100.0,
                 x0_noise: float = 0.0) -> MeshProblem:
    """ARAP mesh deformation on a level-`level` icosphere with
    round(handle_frac * V) seeded handles (at least 1) displaced uniformly in
    [-max_off, max_off]^3."""
    verts, faces = icosphere(level)
    V = verts.shape[0]
    v0, v1 = directed_edges(faces, V)
    rng = np.random.default_rng(seed)
    n_h = max(1, int(round(handle_frac * V)))
    hidx = np.sort(rng.choice(V, size=n_h, replace=False)).astype(np.int32)
    htgt = rng.uniform(-max_off, max_off, size=(n_h, 3)).astype(np.float32)
    x0 = np.zeros((6, V), np.float32)
    if x0_noise > 0:
        x0[:] = rng.uniform(-x0_noise, x0_noise, size=x0.shape).astype(np.float32)
    urshape = np.ascontiguousarray(verts.T.astype(np.float32))
    return MeshProblem(V, urshape, v0, v1, x0, hidx, htgt, float(w_reg), float(w_fit), level, seed)


def graph_problem(urshape: np.ndarray, v0: np.ndarray, v1: np.ndarray, n_handles: int,
                  seed: int = BASE_SEED, max_off: float = 0.1,
                  x0_noise: float = 0.0) -> MeshProblem:
    """ARAP mesh deformation on a caller-given directed edge list (any order).
    Used for small hand-built graphs in tests."""
    V = urshape.shape[1]
    rng = np.random.default_rng(seed)
    hidx = np.sort(rng.choice(V, size=n_handles, replace=False)).astype(np.int32)
    htgt = rng.uniform(-max_off, max_off, size=(n_handles, 3)).astype(np.float32)
    x0 = np.zeros((6, V), np.float32)
    if x0_noise > 0:
        x0[:] = rng.uniform(-x0_noise, x0_noise, size=x0.shape).astype(np.float32)
    return MeshProblem(V, np.ascontiguousarray(urshape, np.float32), np.asarray(v0, np.int32),
                       np.asarray(v1, np.int32), x0, hidx, htgt, 1.0, 100.0, -1, seed)


# ----------------------------------------------------------------------------
# volumetric deformation
# ----------------------------------------------------------------------------
def volume_problem(W: int, H: int, D: int, n_handles: int, seed: int = BASE_SEED, spacing: float = 1.0,
                   max_off: float = 2.0, w_reg: float = 1.0, w_fit: float = 100.0,
                   x0_noise: float = 0.0) -> VolumeProblem:
    """Volumetric ARAP on a W x H x D grid with rest positions at the voxel
    centres (spacing apart), `n_handles` distinct seeded constrained voxels
    displaced uniformly in [-max_off, max_off]^3."""
    zs, ys, xs = np.mgrid[0:D, 0:H, 0:W]
    urshape = (spacing * np.stack([xs, ys, zs]).reshape(3, -1)).astype(np.float32)
    V = W * H * D
    rng = np.random.default_rng(seed)
    hidx = np.sort(rng.choice(V, size=n_handles, replace=False)).astype(np.int32)
    htgt = rng.uniform(-max_off, max_off, size=(n_handles, 3)).astype(np.float32)
    x0 = np.zeros((6, V), np.float32)
    if x0_noise > 0:
        x0[:] = rng.uniform(-x0_noise, x0_noise, size=x0.shape).astype(np.float32)
    return VolumeProblem(W, H, D, urshape, x0, hidx, htgt, float(w_reg), float(w_fit), seed)


def volume_edges(W: int, H: int, D: int):
    """The 7-point stencil of a W x H x D grid as directed edges (k, k + d)
    with both voxels inside the grid, sorted by (v0, v1)."""
    zs, ys, xs = np.mgrid[0:D, 0:H, 0:W]
    a, b = [], []
    for ox, oy, oz in ((1, 0, 0), (-1, 0, 0), (0, 1, 0), (0, -1, 0), (0, 0, 1), (0, 0, -1)):
        nx, ny, nz = xs + ox, ys + oy, zs + oz
        ok = (nx >= 0) & (nx < W) & (ny >= 0) & (ny < H) & (nz >= 0) & (nz < D)
        a.append(((zs * H + ys) * W + xs)[ok])
        b.append(((nz * H + ny) * W + nx)[ok])
    v0 = np.concatenate(a)
    v1 = np.concatenate(b)
    order = np.lexsort((v1, v0))
    return v0[order].astype(np.int32), v1[order].astype(np.int32)


# ----------------------------------------------------------------------------
# batched and serving workloads
# ----------------------------------------------------------------------------
def batch_sides(n: int, lo: int = 32, hi: int = 512, seed: int = BASE_SEED) -> np.ndarray:
    """n square image sides, log-uniform in [lo, hi] (rounded)."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), size=n))
    return np.clip(np.rint(s).astype(np.int64), lo, hi)


def batch_warps(n: int, lo: int = 32, hi: int = 512, seed: int = BASE_SEED):
    """The batched precision workload: n square ARAP warps of uneven sides."""
    sides = batch_sides(n, lo, hi, seed)
    return [warp_problem(int(s), int(s), warp_handle_count(int(s), int(s)), seed=seed + 1000 + i)
            for i, s in enumerate(sides)]


def arrival_times(n: int, rate_per_s: float, seed: int = BASE_SEED) -> np.ndarray:
    """Poisson-process arrival times (seconds) of n requests."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=n))
