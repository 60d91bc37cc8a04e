"""Seeded synthetic workloads for thin plate / shell time stepping.

This module only generates inputs: triangle meshes, rest and initial shapes, material draws, boundary
conditions and request arrival times. It contains no mechanics (no curvature operator, energy, force,
matrix or solver), so both the CUDA library's callers and the independent FP64 oracle can use it
without sharing any of the method's arithmetic.

Conventions (shared by every generator):

* A regular grid of ``nx`` x ``ny`` cells has ``(nx+1)*(ny+1)`` vertices numbered row-major,
  ``index = j*(nx+1) + i``. Each cell ``[i,i+1] x [j,j+1]`` is split along the diagonal from
  ``(i,j)`` to ``(i+1,j+1)``; both triangles are counter-clockwise seen from +z.
* Plates rest in the z = 0 plane. Cylinder panels have their axis along x, the panel on top
  (around +z), and triangle normals pointing away from the axis.
* Every random draw is made from ``numpy.random.default_rng(seed)`` in a fixed order.

The benchmark scenarios mirror the paper's workloads in size and material only (51 to 88K-node meshes,
Section 6); none of the paper's meshes ship with it, so every mesh here is generated.
"""
from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

MODELS = ("EP", "ES", "FP", "FS", "SP", "SS")
MODEL_ID = {m: i for i, m in enumerate(MODELS)}
PLATE_MODELS = ("EP", "FP", "SP")
SHELL_MODELS = ("ES", "FS", "SS")


# --------------------------------------------------------------------------------------------
# meshes
# --------------------------------------------------------------------------------------------
def grid(nx: int, ny: int, lx: float = 1.0, ly: float = 1.0):
    """Regular right-triangle grid on [0,lx] x [0,ly].

    Returns ``(xy, tris)``: ``xy`` float64 [V,2], ``tris`` int32 [2*nx*ny, 3].
    """
    xs = np.linspace(0.0, lx, nx + 1)
    ys = np.linspace(0.0, ly, ny + 1)
    gx, gy = np.meshgrid(xs, ys)  # [ny+1, nx+1]
    xy = np.stack([gx.ravel(), gy.ravel()], axis=1)
    i, j = np.meshgrid(np.arange(nx), np.arange(ny))
    i = i.ravel()
    j = j.ravel()
    v00 = j * (nx + 1) + i
    v10 = v00 + 1
    v01 = v00 + (nx + 1)
    v11 = v01 + 1
    t1 = np.stack([v00, v10, v11], axis=1)
    t2 = np.stack([v00, v11, v01], axis=1)
    tris = np.empty((2 * nx * ny, 3), dtype=np.int32)
    tris[0::2] = t1
    tris[1::2] = t2
    return xy, tris


def equilateral_grid(nx: int, ny: int, side: float = 1.0):
    """Grid of equilateral triangles: rows of ``nx+1`` points spaced ``side``, odd rows shifted by
    ``side/2``, row spacing ``side*sqrt(3)/2``. Triangles counter-clockwise seen from +z.

    Returns ``(xy, tris)``.
    """
    h = side * math.sqrt(3.0) / 2.0
    pts = []
    for j in range(ny + 1):
        off = 0.5 * side if (j % 2) else 0.0
        for i in range(nx + 1):
            pts.append((i * side + off, j * h))
    xy = np.asarray(pts, dtype=np.float64)
    tris = []
    for j in range(ny):
        for i in range(nx):
            a = j * (nx + 1) + i
            b = a + 1
            c = a + (nx + 1)
            d = c + 1
            if j % 2 == 0:
                # row j unshifted, row j+1 shifted right
                tris.append((a, b, c))
                tris.append((b, d, c))
            else:
                # row j shifted right, row j+1 unshifted
                tris.append((a, d, c))
                tris.append((a, b, d))
    return xy, np.asarray(tris, dtype=np.int32)


def grid_interior_mask(nx: int, ny: int) -> np.ndarray:
    """Boolean [V]: vertex is not on the outer boundary of an ``nx`` x ``ny`` cell grid."""
    i, j = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1))
    return ((i > 0) & (i < nx) & (j > 0) & (j < ny)).ravel()


def grid_side_vertices(nx: int, ny: int, side: str) -> np.ndarray:
    """Vertex indices on one side of the grid: ``'x0'`` (i=0), ``'x1'`` (i=nx), ``'y0'``, ``'y1'``."""
    i, j = np.meshgrid(np.arange(nx + 1), np.arange(ny + 1))
    i = i.ravel()
    j = j.ravel()
    sel = {"x0": i == 0, "x1": i == nx, "y0": j == 0, "y1": j == ny}[side]
    return np.nonzero(sel)[0].astype(np.int32)


def grid_side_edges(nx: int, ny: int, side: str) -> np.ndarray:
    """Boundary edges [n,2] (vertex pairs, unordered) along one side of the grid."""
    v = grid_side_vertices(nx, ny, side)
    return np.stack([v[:-1], v[1:]], axis=1).astype(np.int32)


def jitter(xy: np.ndarray, spacing: float, amount: float, movable: np.ndarray, seed: int) -> np.ndarray:
    """Move the ``movable`` vertices in-plane by U(-amount*spacing, amount*spacing) per coordinate."""
    rng = np.random.default_rng(seed)
    d = rng.uniform(-amount * spacing, amount * spacing, size=xy.shape)
    out = xy.copy()
    out[movable] += d[movable]
    return out


def flat3(xy: np.ndarray) -> np.ndarray:
    """Lift 2D points into the z = 0 plane."""
    return np.concatenate([xy, np.zeros((xy.shape[0], 1))], axis=1)


def roll_to_cylinder(xy: np.ndarray, radius: float, width: float) -> np.ndarray:
    """Map a flat strip (x along the axis, y in [0,width] across) isometrically onto a cylinder of the
    given radius whose axis is the x axis; the strip's centre line y = width/2 lands on top (+z)."""
    phi = (xy[:, 1] - 0.5 * width) / radius
    return np.stack([xy[:, 0], radius * np.sin(phi), radius * np.cos(phi)], axis=1)


# --------------------------------------------------------------------------------------------
# scenarios
# --------------------------------------------------------------------------------------------
@dataclasses.dataclass
class Scenario:
    """One simulation: mesh, material, bending model, boundary conditions and stepping options.

    Arrays use the library's layouts: ``tris`` int32 [T,3] (consistently oriented), ``rest``/``x0``/``v0``
    float64 [V,3], ``pinned`` uint8 [V], ``clamped_edges`` int32 [n,2], ``load_vtx`` int32 [m],
    ``load_f`` float64 [m,3].
    """

    name: str
    tris: np.ndarray
    rest: np.ndarray
    x0: np.ndarray
    v0: np.ndarray
    model: str
    E: float
    nu: float
    thickness: float
    density: float
    pinned: np.ndarray
    clamped_edges: np.ndarray
    gravity: tuple
    load_vtx: np.ndarray
    load_f: np.ndarray
    dt: float
    steps: int
    seed: Optional[int] = None
    # per-vertex bit mask of fixed displacement components (bit 0 x, bit 1 y, bit 2 z), uint8 [V], or None;
    # a vertex with all three bits set is pinned
    fixed_dofs: Optional[np.ndarray] = None

    @property
    def n_verts(self) -> int:
        return int(self.rest.shape[0])

    @property
    def n_tris(self) -> int:
        return int(self.tris.shape[0])


def _no_loads():
    return np.zeros((0,), np.int32), np.zeros((0, 3), np.float64)


def plate_clamped_x0(n: int, model: str = "EP", E: float = 1e6, nu: float = 0.3, thickness: float = 1e-3,
                     density: float = 1000.0, dt: float = 1e-2, steps: int = 100, size: float = 1.0,
                     gravity=(0.0, 0.0, -9.81)) -> Scenario:
    """Rest-flat horizontal square plate, ``n`` x ``n`` right-triangle cells, edge x = 0 clamped, gravity.

    With the defaults this is the 16 x 16 (289 vertices, 512 triangles) edge-hinge plate workload.
    """
    xy, tris = grid(n, n, size, size)
    rest = flat3(xy)
    pinned = np.zeros(rest.shape[0], np.uint8)
    pinned[grid_side_vertices(n, n, "x0")] = 1
    lv, lf = _no_loads()
    return Scenario(f"plate{n}_{model}", tris, rest, rest.copy(), np.zeros_like(rest), model, E, nu, thickness,
                    density, pinned, grid_side_edges(n, n, "x0"), tuple(gravity), lv, lf, dt, steps)


def cylinder_panel(n: int, model: str, radius: float = 0.5, arc: float = math.pi / 2, length: float = 1.0,
                   E: float = 1e6, nu: float = 0.3, thickness: float = 1e-3, density: float = 1000.0,
                   dt: float = 5e-3, steps: int = 200, load: float = 1.0, gravity=(0.0, 0.0, 0.0),
                   ny: Optional[int] = None) -> Scenario:
    """Rest-curved cylindrical panel (axis along x), ``n`` x ``ny`` cells, both straight edges (parallel to
    the axis) clamped, a point load of ``load`` newtons at the centre vertex pointing at the axis.

    Shell models rest on the cylinder. Plate models rest on the unrolled flat strip and start on the
    cylinder (a rest-flat shell relaxes towards flat).
    """
    ny = n if ny is None else ny
    width = radius * arc
    xy, tris = grid(n, ny, length, width)
    curved = roll_to_cylinder(xy, radius, width)
    rest = curved.copy() if model in SHELL_MODELS else flat3(xy)
    pinned = np.zeros(rest.shape[0], np.uint8)
    clamped = np.concatenate([grid_side_edges(n, ny, "y0"), grid_side_edges(n, ny, "y1")])
    pinned[np.unique(clamped)] = 1
    centre = (ny // 2) * (n + 1) + n // 2
    if load != 0.0:
        p = curved[centre]
        radial = np.array([0.0, p[1], p[2]]) / math.hypot(p[1], p[2])
        lv = np.array([centre], np.int32)
        lf = (-load * radial)[None, :]
    else:
        lv, lf = _no_loads()
    return Scenario(f"cyl{n}_{model}", tris, rest, curved, np.zeros_like(curved), model, E, nu, thickness, density,
                    pinned, clamped.astype(np.int32), tuple(gravity), lv, lf, dt, steps)


def jittered_plate(n_side_verts: int = 512, model: str = "SP", seed: int = 2502, E: float = 1e7, nu: float = 0.3,
                   thickness: float = 5e-4, density: float = 1000.0, dt: float = 1.0 / 60.0, steps: int = 1000,
                   amount: float = 0.2, size: float = 1.0) -> Scenario:
    """Rest-flat horizontal plate on a jittered grid of ``n_side_verts``^2 vertices: interior vertices move
    in-plane by U(-amount*s, amount*s); the two corners at y = size are pinned; gravity -z."""
    n = n_side_verts - 1
    s = size / n
    xy, tris = grid(n, n, size, size)
    xy = jitter(xy, s, amount, grid_interior_mask(n, n), seed)
    rest = flat3(xy)
    pinned = np.zeros(rest.shape[0], np.uint8)
    pinned[n * (n + 1)] = 1          # (0, size)
    pinned[n * (n + 1) + n] = 1      # (size, size)
    lv, lf = _no_loads()
    return Scenario(f"jitter{n_side_verts}_{model}", tris, rest, rest.copy(), np.zeros_like(rest), model, E, nu,
                    thickness, density, pinned, np.zeros((0, 2), np.int32), (0.0, 0.0, -9.81), lv, lf, dt, steps,
                    seed)


def random_instance(rng: np.random.Generator, side_lo: int = 8, side_hi: int = 128, dt: float = 1e-2,
                    steps: int = 500, name: str = "inst") -> Scenario:
    """One instance of the mixed batch: side log-uniform in [side_lo, side_hi] cells, half plates (1 m square,
    one edge clamped, gravity) and half cylinder panels (radius U(0.3, 2), 90 degree arc, 1 m long, both
    straight edges clamped, gravity), model uniform over the six, E log-uniform in [1e5, 1e8] Pa,
    nu uniform in [0.2, 0.45], thickness 1e-3 m, density 1000 kg/m^3.

    Draw order (fixed): side, shape, model, E, nu, radius.
    """
    side = int(round(math.exp(rng.uniform(math.log(side_lo), math.log(side_hi)))))
    curved = bool(rng.uniform() < 0.5)
    model = MODELS[int(rng.integers(0, 6))]
    E = float(math.exp(rng.uniform(math.log(1e5), math.log(1e8))))
    nu = float(rng.uniform(0.2, 0.45))
    radius = float(rng.uniform(0.3, 2.0))
    if curved:
        sc = cylinder_panel(side, model, radius=radius, E=E, nu=nu, thickness=1e-3, density=1000.0, dt=dt,
                            steps=steps, load=0.0, gravity=(0.0, 0.0, -9.81))
    else:
        sc = plate_clamped_x0(side, model=model, E=E, nu=nu, thickness=1e-3, density=1000.0, dt=dt, steps=steps)
    sc.name = f"{name}_{'cyl' if curved else 'plate'}{side}_{model}"
    return sc


def mixed_batch(n_instances: int = 256, seed: int = 4, side_lo: int = 8, side_hi: int = 128, dt: float = 1e-2,
                steps: int = 500) -> List[Scenario]:
    """The batched workload: ``n_instances`` independent instances drawn by :func:`random_instance`."""
    rng = np.random.default_rng(seed)
    out = []
    for k in range(n_instances):
        sc = random_instance(rng, side_lo, side_hi, dt, steps, name=f"b{k:03d}")
        sc.seed = seed
        out.append(sc)
    return out


def serving_requests(n_requests: int, rate_hz: float = 200.0, seed: int = 5, v_lo: int = 1000,
                     v_hi: int = 250000, steps_lo: int = 50, steps_hi: int = 500, dt: float = 1e-2):
    """Poisson arrivals of simulation requests: returns a list of ``(arrival_s, Scenario)``.

    Each request: vertex count log-uniform in [v_lo, v_hi] as a jittered square grid with side
    round(sqrt(V)) vertices, model uniform over the six, step count uniform in [steps_lo, steps_hi],
    E log-uniform [1e5, 1e8], nu U(0.2, 0.45), thickness 1e-3, density 1000, one edge clamped, gravity.
    Draw order per request (fixed): gap, V, model, steps, E, nu, jitter seed.
    """
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for k in range(n_requests):
        t += float(rng.exponential(1.0 / rate_hz))
        v = float(math.exp(rng.uniform(math.log(v_lo), math.log(v_hi))))
        side_v = max(3, int(round(math.sqrt(v))))
        model = MODELS[int(rng.integers(0, 6))]
        steps = int(rng.integers(steps_lo, steps_hi + 1))
        E = float(math.exp(rng.uniform(math.log(1e5), math.log(1e8))))
        nu = float(rng.uniform(0.2, 0.45))
        jseed = int(rng.integers(0, 2**31 - 1))
        n = side_v - 1
        s = 1.0 / n
        xy, tris = grid(n, n)
        xy = jitter(xy, s, 0.2, grid_interior_mask(n, n), jseed)
        rest = flat3(xy)
        pinned = np.zeros(rest.shape[0], np.uint8)
        pinned[grid_side_vertices(n, n, "x0")] = 1
        lv, lf = _no_loads()
        sc = Scenario(f"req{k:05d}_{side_v}_{model}", tris, rest, rest.copy(), np.zeros_like(rest), model, E, nu,
                      1e-3, 1000.0, pinned, grid_side_edges(n, n, "x0"), (0.0, 0.0, -9.81), lv, lf, dt, steps,
                      jseed)
        out.append((t, sc))
    return out


def simply_supported_square(n: int, size: float = 8.0, mesh: str = "regular"):
    """Square plate for the static uniform-load benchmark (Section 6.1): side ``size``, every boundary vertex
    pinned, every boundary edge free for bending. ``mesh`` is ``'regular'`` (right triangles, ``n`` x ``n``
    cells) or ``'equilateral'`` (``n`` columns of equilateral triangles, rows fitted to the square, then
    the y coordinate rescaled onto [0, size]).

    Returns ``(rest [V,3], tris, boundary_mask [V])``.
    """
    if mesh == "regular":
        xy, tris = grid(n, n, size, size)
        bmask = ~grid_interior_mask(n, n)
    elif mesh == "equilateral":
        side = size / n
        ny = max(2, int(round(size / (side * math.sqrt(3) / 2))))
        xy, tris = equilateral_grid(n, ny, side)
        # shifted rows start at side/2 and end at size + side/2: pull their end points onto x = 0 and
        # x = size so the outline is a rectangle, then fit y onto [0, size]
        row_first = np.arange(ny + 1) * (n + 1)
        odd = (np.arange(ny + 1) % 2) == 1
        xy[row_first[odd], 0] = 0.0
        xy[:, 0] = np.minimum(xy[:, 0], size)
        xy[:, 1] *= size / xy[:, 1].max()
        eps = 1e-9 * size
        bmask = (xy[:, 0] < eps) | (xy[:, 0] > size - eps) | (xy[:, 1] < eps) | (xy[:, 1] > size - eps)
    else:
        raise ValueError(mesh)
    return flat3(xy), tris, bmask


def cantilever(model: str = "FP", nx: int = 16, ny: int = 2, length: float = 10.0, width: float = 1.0,
               E: float = 1.2e6, nu: float = 0.1, thickness: float = 0.1, total_load: float = 4.0,
               density: float = 1.0, dt: float = 1.0) -> Scenario:
    """Cantilever under end shear (Section 6.1, geometrically non-linear benchmark): a flat ``length`` x
    ``width`` plate meshed with (nx + 1) x (ny + 1) nodes (17 x 3 = 51 by default; cells split along
    (i, j) -> (i + 1, j + 1)), the two node columns at x = 0 pinned, ``total_load`` shared equally by the
    right-edge nodes along +z, no gravity, no clamped edges (all boundary edges are free for bending).
    ``density`` and ``dt`` only enter a quasi-static solve through the mass shift M / dt^2 of its linear
    systems (negligible by default: about 1e-7 of the stiffness)."""
    xy, tris = grid(nx, ny, length, width)
    rest = flat3(xy)
    V = rest.shape[0]
    pinned = (xy[:, 0] < length / nx * (1.0 + 1e-9)).astype(np.uint8)
    right = np.flatnonzero(np.abs(xy[:, 0] - length) < 1e-9 * length).astype(np.int32)
    lf = np.tile([0.0, 0.0, total_load / len(right)], (len(right), 1))
    return Scenario(f"cantilever_{model}", tris, rest, rest.copy(), np.zeros_like(rest), model, E, nu, thickness,
                    density, pinned, np.zeros((0, 2), np.int32), (0.0, 0.0, 0.0), right, lf, dt, 1)


def cantilever_tip(sc: Scenario) -> int:
    """Index of the mid node of the cantilever's loaded edge (where w_tip is read)."""
    right = np.asarray(sc.load_vtx)
    return int(right[np.argsort(sc.rest[right, 1])[len(right) // 2]])


def hemisphere(model: str = "SS", n_around: int = 64, n_rings: int = 17, radius: float = 10.0,
               cut_deg: float = 18.0, E: float = 6.825e7, nu: float = 0.3, thickness: float = 0.04,
               load: float = 200.0, density: float = 1.0, dt: float = 1.0) -> Scenario:
    """Hemispherical shell under alternating radial point loads (Section 6.1, geometrically non-linear
    benchmark), the whole shell: radius ``radius``, a circular hole of half-angle ``cut_deg`` at the pole,
    ``n_rings`` rings of ``n_around`` nodes from the equator (latitude 0) to the hole's edge (latitude
    90 - cut_deg), 64 x 17 = 1088 nodes by default. Ring k, node j sits at latitude k (90 - cut_deg) /
    (n_rings - 1) and longitude 2 pi j / n_around. Each quadrilateral cell is split into two triangles along
    the diagonal that makes the mesh symmetric under the reflections x -> -x and y -> -y (from (j, k) to
    (j + 1, k + 1) where j lies in the first or third quadrant of longitudes, the other diagonal in the
    second and fourth), so the loaded problem has both symmetries. Triangles are counter-clockwise seen from
    outside. Loads on the equator: ``load`` towards the centre at (+-radius, 0, 0) and away from it at
    (0, +-radius, 0). Constraints (``fixed_dofs``): x fixed on the nodes of the y-z plane, y fixed on the
    nodes of the x-z plane, and z also fixed on the hole's edge in the y-z plane. No gravity, no clamped
    edges. ``n_around`` must be a multiple of 4. ``density`` and ``dt`` only enter a quasi-static solve
    through the mass shift M / dt^2 of its linear systems."""
    if n_around % 4 or n_around < 8 or n_rings < 2:
        raise ValueError("n_around must be a multiple of 4 (>= 8) and n_rings >= 2")
    lat = np.radians(90.0 - cut_deg) * np.arange(n_rings) / (n_rings - 1)
    lon = 2.0 * np.pi * np.arange(n_around) / n_around
    k, j = np.meshgrid(np.arange(n_rings), np.arange(n_around), indexing="ij")
    k, j = k.ravel(), j.ravel()
    rest = np.stack([radius * np.cos(lat[k]) * np.cos(lon[j]), radius * np.cos(lat[k]) * np.sin(lon[j]),
                     radius * np.sin(lat[k])], axis=1)
    q = n_around // 4
    for jj, c in ((0, 0), (q, 1), (2 * q, 0), (3 * q, 1)):   # exact zeros on the symmetry planes
        rest[j == jj, 1 - c] = 0.0
    vid = lambda kk, jj: kk * n_around + (jj % n_around)
    tris = []
    for kk in range(n_rings - 1):
        for jj in range(n_around):
            a, b, c, d = vid(kk, jj), vid(kk, jj + 1), vid(kk + 1, jj + 1), vid(kk + 1, jj)
            if (jj // q) % 2 == 0:
                tris += [(a, b, c), (a, c, d)]
            else:
                tris += [(a, b, d), (b, c, d)]
    tris = np.asarray(tris, np.int32)
    fixed = np.zeros(rest.shape[0], np.uint8)
    fixed[(j == q) | (j == 3 * q)] |= 1
    fixed[(j == 0) | (j == 2 * q)] |= 2
    fixed[((j == q) | (j == 3 * q)) & (k == n_rings - 1)] |= 4
    lv = np.array([vid(0, 0), vid(0, 2 * q), vid(0, q), vid(0, 3 * q)], np.int32)
    lf = load * np.array([[-1.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, -1.0, 0.0]])
    return Scenario(f"hemisphere_{model}", tris, rest, rest.copy(), np.zeros_like(rest), model, E, nu, thickness,
                    density, np.zeros(rest.shape[0], np.uint8), np.zeros((0, 2), np.int32), (0.0, 0.0, 0.0), lv,
                    lf, dt, 1, fixed_dofs=fixed)


def hemisphere_probes(sc: Scenario):
    """Indices of the equator nodes at (radius, 0, 0) (loaded towards the centre: u_min is read there) and
    at (0, radius, 0) (loaded outwards: v_max)."""
    return int(sc.load_vtx[0]), int(sc.load_vtx[2])


def linear_plate(model: str = "FP", n: int = 32, mesh: str = "regular", size: float = 8.0,
                 pressure: float = 9.81e-3, E: float = 2e11, nu: float = 0.3, thickness: float = 0.01,
                 density: float = 1.0, dt: float = 1.0) -> Scenario:
    """Linear plate bending benchmark (Section 6.1): the simply supported ``size`` x ``size`` square of
    :func:`simply_supported_square` under a uniform transverse pressure, applied as point loads pressure x
    (a third of the incident triangles' areas) at the free vertices along +z. The default pressure is the
    benchmark's 9.81 scaled by 1e-3, so the centre deflection (about 9e-6) stays far below the thickness and a
    quasi-static solve, which carries the corotated membrane, gives the linear bending response (the
    deflection scales with the pressure). n = 85 on the regular mesh gives 7,396 vertices (the paper times
    7,459). ``density`` and ``dt`` only enter through the mass shift of a quasi-static solve."""
    rest, tris, bmask = simply_supported_square(n, size, mesh)
    t = np.asarray(tris, np.int64)
    area = 0.5 * np.linalg.norm(np.cross(rest[t[:, 1]] - rest[t[:, 0]], rest[t[:, 2]] - rest[t[:, 0]]), axis=1)
    nodal = np.zeros(rest.shape[0])
    np.add.at(nodal, t.ravel(), np.repeat(area / 3.0, 3))
    lv = np.flatnonzero(~bmask).astype(np.int32)
    lf = np.zeros((len(lv), 3))
    lf[:, 2] = pressure * nodal[lv]
    return Scenario(f"linear_plate_{mesh}{n}_{model}", tris.astype(np.int32), rest, rest.copy(), np.zeros_like(rest),
                    model, E, nu, thickness, density, bmask.astype(np.uint8), np.zeros((0, 2), np.int32),
                    (0.0, 0.0, 0.0), lv, lf, dt, 1)
