"""Seeded synthetic inputs shared by the CUDA path, the CPU oracle, the tests and the bench.

This module holds only the *inputs*: grid node coordinates, random right-hand sides,
the synthetic extruded-airfoil point cloud and its triangulation, and the named workload
shapes.  It holds none of the method's arithmetic (no operator coefficients, no SpMM, no
solver step), so that the oracle and the GPU path stay independent of each other.

Workload shapes follow the paper's test cases (Sec. 4):
  * channel flow, Sec. 4.1: tanh wall-normal refinement with factor 1.5;
  * Rayleigh-Benard, Sec. 4.2: walls in one direction, tanh refinement;
  * 30P30N airfoil, Sec. 4.3: an unstructured mesh extruded along a periodic span
    (150c x 150c x 2c); the real mesh is not available, so a seeded Delaunay mesh
    clustered around a NACA-0012 profile stands in for it.
"""
from __future__ import annotations

import dataclasses
import math
from typing import Sequence

import numpy as np

# --------------------------------------------------------------------------------------
# Random numbers
# --------------------------------------------------------------------------------------


def rng(seed: int) -> np.random.Generator:
    """Seeded generator used for every synthetic input."""
    return np.random.default_rng(seed)


def normal(shape, seed: int, dtype=np.float64) -> np.ndarray:
    """N(0,1) values, generated in float64 and then cast (RNE) to ``dtype``."""
    return rng(seed).standard_normal(shape).astype(dtype)


# --------------------------------------------------------------------------------------
# Structured grids: node coordinates per axis
# --------------------------------------------------------------------------------------


@dataclasses.dataclass(frozen=True)
class Axis:
    """One grid direction: ``n`` cells bounded by ``n + 1`` increasing nodes."""

    nodes: np.ndarray  # float64, shape (n + 1,)
    periodic: bool

    @property
    def n(self) -> int:
        return int(self.nodes.shape[0] - 1)


def uniform_axis(n: int, length: float = 1.0, periodic: bool = True) -> Axis:
    return Axis(np.linspace(0.0, length, n + 1), periodic)


def tanh_axis(n: int, gamma: float, lo: float = -1.0, hi: float = 1.0) -> Axis:
    """Wall-bounded axis refined towards both walls by a hyperbolic tangent.

    Node j sits at tanh(gamma (2j/n - 1)) / tanh(gamma), mapped from [-1, 1] to
    [lo, hi].  The paper gives only the factor gamma (Sec. 4.1, Sec. 4.2); this is the
    usual symmetric two-wall form of that refinement.
    """
    j = np.arange(n + 1, dtype=np.float64)
    s = np.tanh(gamma * (2.0 * j / n - 1.0)) / np.tanh(gamma)
    s[0], s[-1] = -1.0, 1.0
    return Axis(lo + (hi - lo) * 0.5 * (s + 1.0), False)


@dataclasses.dataclass(frozen=True)
class Grid:
    """Cartesian staggered grid; unknowns are ordered with x fastest: id = i + nx (j + ny k)."""

    axes: tuple  # (Axis x, Axis y, Axis z)
    name: str = ""

    @property
    def shape(self) -> tuple:
        return tuple(a.n for a in self.axes)

    @property
    def n_cells(self) -> int:
        nx, ny, nz = self.shape
        return nx * ny * nz


def unit_periodic_grid(n: int) -> Grid:
    """Periodic unit cube with n^3 cells (h = 1/n)."""
    return Grid((uniform_axis(n), uniform_axis(n), uniform_axis(n)), f"periodic-{n}^3")


def channel_grid(nx: int, ny: int, nz: int, gamma: float = 1.5) -> Grid:
    """Plane channel 2pi x 2 x pi: periodic in x and z, walls at y = -1 and y = +1."""
    return Grid(
        (uniform_axis(nx, 2.0 * math.pi), tanh_axis(ny, gamma, -1.0, 1.0), uniform_axis(nz, math.pi)),
        f"channel-{nx}x{ny}x{nz}",
    )


def rbc_grid(n: int = 128, gamma: float = 1.4) -> Grid:
    """Unit box, periodic in x and y, walls at z = 0 and z = 1 refined by tanh."""
    return Grid((uniform_axis(n), uniform_axis(n), tanh_axis(n, gamma, 0.0, 1.0)), f"rbc-{n}^3")


# --------------------------------------------------------------------------------------
# Synthetic extruded airfoil: seeded points around a NACA-0012 profile, Delaunay mesh
# --------------------------------------------------------------------------------------


def naca0012_half_thickness(x: np.ndarray) -> np.ndarray:
    """Half thickness of the symmetric NACA 4-digit section with 12 % thickness, chord 1."""
    x = np.clip(x, 0.0, 1.0)
    return 0.6 * (0.2969 * np.sqrt(x) - 0.1260 * x - 0.3516 * x**2 + 0.2843 * x**3 - 0.1036 * x**4)


def _inside_profile(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    return (x > 0.0) & (x < 1.0) & (np.abs(y) < naca0012_half_thickness(x))


@dataclasses.dataclass(frozen=True)
class TriMesh:
    points: np.ndarray  # float64 (n_vert, 2)
    triangles: np.ndarray  # int32 (n_tri, 3), counter-clockwise


def airfoil_mesh(n_points: int = 150_000, seed: int = 3000, box: float = 20.0, near_frac: float = 0.5,
                 near_dist: float = 0.05) -> TriMesh:
    """Seeded point cloud clustered within ``near_dist`` chord of the profile, Delaunay meshed.

    A fraction ``near_frac`` of the points lies within ``near_dist`` of the profile
    surface, the rest is uniform in a ``box`` x ``box`` square centred on the chord.
    Points inside the profile are dropped; triangles whose centroid is inside the
    profile are removed, so the body is a hole in the mesh.  Unused vertices are
    dropped and the rest renumbered in (x, y)-sorted order along a coarse raster, which
    keeps neighbouring vertices close in memory.
    """
    from scipy.spatial import Delaunay

    g = rng(seed)
    n_near = int(n_points * near_frac)
    n_far = n_points - n_near
    # far field: uniform in the box centred at the mid-chord
    far = (g.random((n_far, 2)) - 0.5) * box
    far[:, 0] += 0.5
    # near field: a point on the profile surface, displaced along y by up to near_dist
    t = g.random(n_near)
    xs = 0.5 * (1.0 - np.cos(math.pi * t))  # cosine clustering towards the edges
    side = np.where(g.random(n_near) < 0.5, -1.0, 1.0)
    off = g.random(n_near) * near_dist
    near = np.stack([xs + (g.random(n_near) - 0.5) * near_dist, side * (naca0012_half_thickness(xs) + off)], axis=1)
    # surface points so that the hole is well resolved
    ns = max(64, int(math.sqrt(n_points)))
    ts = 0.5 * (1.0 - np.cos(math.pi * np.linspace(0.0, 1.0, ns)))
    surf = np.concatenate([np.stack([ts, naca0012_half_thickness(ts)], 1), np.stack([ts[1:-1], -naca0012_half_thickness(ts[1:-1])], 1)])
    pts = np.concatenate([surf, near, far])
    keep = ~_inside_profile(pts[:, 0], pts[:, 1] * 1.0000001)
    pts = pts[keep]
    # deterministic de-duplication
    pts = np.unique(np.round(pts, 12), axis=0)
    tri = Delaunay(pts).simplices.astype(np.int64)
    c = pts[tri].mean(axis=1)
    tri = tri[~_inside_profile(c[:, 0], c[:, 1])]
    # orient counter-clockwise
    a, b, cc = pts[tri[:, 0]], pts[tri[:, 1]], pts[tri[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (cc[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (cc[:, 0] - a[:, 0])
    flip = cross < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    tri = tri[np.abs(cross) > 1e-14]
    # drop unused vertices, renumber along a raster of cells
    used = np.unique(tri)
    p = pts[used]
    cell = 0.05
    key_y = np.floor((p[:, 1] + box) / cell).astype(np.int64)
    order = np.lexsort((p[:, 0], key_y))
    new_id = np.empty(pts.shape[0], dtype=np.int64)
    new_id[used[order]] = np.arange(used.shape[0])
    return TriMesh(p[order].copy(), new_id[tri].astype(np.int32))


def mesh_adjacency(mesh: TriMesh):
    """Vertex adjacency of a triangle mesh as a CSR pattern (row_ptr, col_idx), diagonal included,
    columns sorted within each row.  Pure topology: the sparsity pattern of any vertex-centred
    operator on the mesh."""
    n = mesh.points.shape[0]
    t = mesh.triangles.astype(np.int64)
    a = np.concatenate([t[:, 0], t[:, 1], t[:, 2], t[:, 1], t[:, 2], t[:, 0], np.arange(n)])
    b = np.concatenate([t[:, 1], t[:, 2], t[:, 0], t[:, 0], t[:, 1], t[:, 2], np.arange(n)])
    key = np.unique(a * n + b)
    rows = key // n
    cols = (key % n).astype(np.int32)
    row_ptr = np.zeros(n + 1, dtype=np.int32)
    np.add.at(row_ptr, rows + 1, 1)
    return np.cumsum(row_ptr).astype(np.int32), cols


def grid_trimesh(nx: int, ny: int, h: float = 1.0) -> TriMesh:
    """Regular right-triangle mesh of an nx x ny block of squares (a test fixture)."""
    xs, ys = np.meshgrid(np.arange(nx + 1) * h, np.arange(ny + 1) * h)
    pts = np.stack([xs.ravel(), ys.ravel()], 1)
    tris = []
    for j in range(ny):
        for i in range(nx):
            v0 = i + (nx + 1) * j
            v1, v2, v3 = v0 + 1, v0 + nx + 1, v0 + nx + 2
            tris.append((v0, v1, v3))
            tris.append((v0, v3, v2))
    return TriMesh(pts, np.array(tris, dtype=np.int32))


def random_trimesh(n: int, seed: int) -> TriMesh:
    """Delaunay mesh of n seeded uniform points in the unit square (a test fixture)."""
    from scipy.spatial import Delaunay

    pts = rng(seed).random((n, 2))
    tri = Delaunay(pts).simplices.astype(np.int64)
    a, b, c = pts[tri[:, 0]], pts[tri[:, 1]], pts[tri[:, 2]]
    cross = (b[:, 0] - a[:, 0]) * (c[:, 1] - a[:, 1]) - (b[:, 1] - a[:, 1]) * (c[:, 0] - a[:, 0])
    flip = cross < 0
    tri[flip, 1], tri[flip, 2] = tri[flip, 2].copy(), tri[flip, 1].copy()
    return TriMesh(pts, tri.astype(np.int32))


# --------------------------------------------------------------------------------------
# Named workloads (sizes of the paper-shaped synthetic cases)
# --------------------------------------------------------------------------------------

CHANNEL_SHAPE = (192, 128, 96)  # channel-flow shaped case, n = 2,359,296
SMALL_PERIODIC_N = 32  # 32^3 uniform periodic correctness case
EXTRUDED_NZ = 64  # periodic planes of the extruded airfoil
EXTRUDED_SPAN = 2.0  # span in chords, as the airfoil domain of Sec. 4.3
BATCH_SHAPES = (("periodic", 64), ("periodic", 128), ("channel", (96, 64, 48)), ("channel", (96, 64, 48)),
                ("channel", (96, 64, 48)))
BATCH_K_DEFAULT = (8, 1, 3, 3, 3)


def batch_grids() -> list:
    out = []
    for kind, s in BATCH_SHAPES:
        out.append(unit_periodic_grid(s) if kind == "periodic" else channel_grid(*s, gamma=1.5))
    return out


def seed_for(cfg: int, k: int, salt: int = 0) -> int:
    return 1000 * cfg + k + 100_000 * salt


def zero_mean(b: np.ndarray) -> np.ndarray:
    """Remove each column's mean (makes a right-hand side compatible with a singular Neumann/periodic problem)."""
    return b - b.mean(axis=0, keepdims=True)


def face_field(n_faces: int, k: int, seed: int, dtype=np.float64) -> np.ndarray:
    """N(0,1) face velocities (k columns) used to build compatible right-hand sides b = M u."""
    return normal((n_faces, k), seed, dtype)


# Learned-guess data: a Rayleigh-Benard-shaped 128^3 grid, 8 independent forcing sequences
# (the k = 8 columns of each solve) of 252 steps; pairs start at step 2 (two previous
# pressures), the last 25 steps of every sequence are held out: 8 x 225 = 1800 training and
# 8 x 25 = 200 test pairs.
GUESS_N = 128
GUESS_CHAINS = 8
GUESS_STEPS = 252
GUESS_HOLDOUT = 25
GUESS_KMAX = 4
GUESS_RHO = 0.95


def forcing_spectra(steps: int, chains: int, kmax: int = GUESS_KMAX, rho: float = GUESS_RHO,
                    seed: int = 5000) -> np.ndarray:
    """Seeded random amplitudes of the Fourier modes 0 < |kappa| <= kmax of three smooth scalar
    fields (one per face direction) for `chains` independent sequences, AR(1) in time:
    a_t = rho a_{t-1} + sqrt(1 - rho^2) xi_t, xi complex N(0, 1).  Shape
    [steps, chains, 3, 2 kmax + 1, 2 kmax + 1, kmax + 1] (z, y wavenumbers -kmax..kmax, x 0..kmax)."""
    g = rng(seed)
    m = 2 * kmax + 1
    kz, ky, kx = np.meshgrid(np.arange(-kmax, kmax + 1), np.arange(-kmax, kmax + 1), np.arange(kmax + 1),
                             indexing="ij")
    mask = (kz**2 + ky**2 + kx**2 <= kmax * kmax) & ((kz != 0) | (ky != 0) | (kx != 0))
    shape = (chains, 3, m, m, kmax + 1)
    out = np.zeros((steps,) + shape, dtype=np.complex128)
    a = (g.standard_normal(shape) + 1j * g.standard_normal(shape)) * mask
    s = np.sqrt(1.0 - rho * rho)
    for t in range(steps):
        if t:
            a = rho * a + s * (g.standard_normal(shape) + 1j * g.standard_normal(shape)) * mask
        out[t] = a
    return out


def face_fields(spec_t: np.ndarray, cells: tuple, torch_mod, device) -> "object":
    """Synthesise the face velocities of one step from its spectra (inverse real FFT on the
    cell-index grid, scaled to unit rms per mode count): returns a float64 tensor
    [n_faces, chains] in the face order x faces, y faces, z faces (each x fastest), with
    periodic x and y (nx, ny faces per line) and walls in z (nz - 1 interior z faces)."""
    torch = torch_mod
    nx, ny, nz = cells
    chains, _, m, _, kx1 = spec_t.shape
    kmax = (m - 1) // 2
    full = torch.zeros((chains, 3, nz, ny, nx // 2 + 1), dtype=torch.complex128, device=device)
    sp = torch.as_tensor(spec_t, device=device)
    zi = torch.as_tensor(np.arange(-kmax, kmax + 1) % nz, device=device)
    yi = torch.as_tensor(np.arange(-kmax, kmax + 1) % ny, device=device)
    full[:, :, zi[:, None], yi[None, :], :kx1] = sp
    f = torch.fft.irfftn(full, s=(nz, ny, nx), dim=(2, 3, 4)) * (nx * ny * nz / np.sqrt(4.0 * m * m * kx1))
    fx = f[:, 0].reshape(chains, -1)
    fy = f[:, 1].reshape(chains, -1)
    fz = f[:, 2, : nz - 1].reshape(chains, -1)
    return torch.cat([fx, fy, fz], dim=1).t().contiguous()


def as_columns(x: np.ndarray) -> np.ndarray:
    return x.reshape(x.shape[0], -1)


def ks_sweep() -> Sequence[int]:
    return (1, 2, 3, 4, 8, 16, 32)
