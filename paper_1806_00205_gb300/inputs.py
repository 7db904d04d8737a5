"""Seeded synthetic inputs for the RTMC secondary-electron-yield path.

This module only *prepares data*: triangle meshes in a periodic cell and the
flat-surface yield table.  It holds none of the method's arithmetic (no ray
tracing, no sampling, no tallies), so both the CUDA path and the CPU oracle
may consume what it produces.

Geometry conventions (Section 2.1 of the paper, Fig. 1 "Geometry" box):
  * a mesh is a float32 array ``tri[n, 3, 3]`` of vertices V0, V1, V2;
  * the facet normal (V1-V0) x (V2-V0) points from solid into vacuum
    (counter-clockwise vertices seen from the vacuum side);
  * the cell is periodic in x in [0, lx] and y in [0, ly]; the substrate
    sits at the bottom and the escape plane is z = z_top (Section 2.2, last
    paragraph: periodic x/y, flat boundary at z_min, emission at z_max).

The paper builds its foams from X-ray tomography voxels (Section 3).  Those
images are not available, so a Gaussian random field thresholded at the
requested porosity stands in for them, and the isosurface is extracted with
a marching-cubes variant whose case table is generated here from the corner
sign pattern (see ``_mc_case_table``).
"""
from __future__ import annotations

import dataclasses
import math
from functools import lru_cache

import numpy as np

__all__ = [
    "Box", "Mesh", "SeeTable", "grf_field", "marching_cubes_periodic",
    "grf_foam", "flat_plane", "square_well", "see_table",
]


@dataclasses.dataclass(frozen=True)
class Box:
    """Periodic cell: x in [0, lx), y in [0, ly); z in [z_min, z_top]."""
    lx: float
    ly: float
    z_min: float
    z_top: float

    def as_tuple(self):
        return (float(self.lx), float(self.ly), float(self.z_min), float(self.z_top))


@dataclasses.dataclass
class Mesh:
    tri: np.ndarray          # float32 [n, 3, 3], C-contiguous
    box: Box
    name: str = ""
    porosity: float = float("nan")

    @property
    def n_tri(self) -> int:
        return int(self.tri.shape[0])


@dataclasses.dataclass
class SeeTable:
    """Flat-surface yield table delta(E, theta) on a log-E x linear-theta grid.

    ``delta[i, j]`` is the yield at E_i = e_lo * (e_hi/e_lo)**(i/(n_e-1)) and
    theta_j = j * theta_step_deg (row-major, energy-major, float32).
    """
    delta: np.ndarray
    e_lo_ev: float
    e_hi_ev: float
    theta_step_deg: float

    @property
    def n_e(self) -> int:
        return int(self.delta.shape[0])

    @property
    def n_theta(self) -> int:
        return int(self.delta.shape[1])

    def energy_grid(self) -> np.ndarray:
        i = np.arange(self.n_e, dtype=np.float64)
        return self.e_lo_ev * (self.e_hi_ev / self.e_lo_ev) ** (i / (self.n_e - 1))


# ----------------------------------------------------------------------------
# Yield tables
# ----------------------------------------------------------------------------

def lin_joy_delta(e_ev, theta_rad, delta_max=1.4, e_max_ev=650.0):
    """Universal-curve yield with the 1 + theta^2/(2 pi) angular factor.

    delta = delta_max (1 + theta^2 / (2 pi)) 1.28 (E/Em)^-0.67
            (1 - exp(-1.614 (E/Em)^1.67)), theta in radians.
    """
    x = np.asarray(e_ev, dtype=np.float64) / e_max_ev
    th = np.asarray(theta_rad, dtype=np.float64)
    return (delta_max * (1.0 + th * th / (2.0 * math.pi)) * 1.28 * x ** -0.67
            * (1.0 - np.exp(-1.614 * x ** 1.67)))


def see_table(n_e=64, n_theta=18, e_lo_ev=1.0, e_hi_ev=2000.0, theta_step_deg=5.0,
              delta_max=1.4, e_max_ev=650.0) -> SeeTable:
    """Tabulate the universal-curve yield on the 64 x 18 grid used by the runs."""
    e = e_lo_ev * (e_hi_ev / e_lo_ev) ** (np.arange(n_e) / (n_e - 1))
    th = np.deg2rad(np.arange(n_theta) * theta_step_deg)
    d = lin_joy_delta(e[:, None], th[None, :], delta_max, e_max_ev)
    return SeeTable(np.ascontiguousarray(d.astype(np.float32)), float(e_lo_ev),
                    float(e_hi_ev), float(theta_step_deg))


# ----------------------------------------------------------------------------
# Gaussian random field foams
# ----------------------------------------------------------------------------

def grf_field(n: int, corr_len_vox: float, seed: int) -> np.ndarray:
    """Periodic n^3 Gaussian random field, unit variance, float64.

    White noise (numpy Philox stream keyed by ``seed``) filtered in Fourier
    space by exp(-|k|^2 l^2 / 2) with l in voxels.
    """
    rng = np.random.Generator(np.random.Philox(seed))
    w = rng.standard_normal((n, n, n))
    k = 2.0 * np.pi * np.fft.fftfreq(n)
    k2 = k[:, None, None] ** 2 + k[None, :, None] ** 2 + k[None, None, :] ** 2
    f = np.fft.ifftn(np.fft.fftn(w) * np.exp(-0.5 * k2 * corr_len_vox ** 2)).real
    f -= f.mean()
    f /= f.std()
    return f


def _corner_offsets():
    return np.array([[(c >> 0) & 1, (c >> 1) & 1, (c >> 2) & 1] for c in range(8)], dtype=np.int64)


def _edges():
    """The 12 cube edges as (lower corner, upper corner, axis)."""
    out = []
    for axis in range(3):
        for a in range(8):
            if not (a >> axis) & 1:
                out.append((a, a | (1 << axis), axis))
    return out


@lru_cache(maxsize=None)
def _mc_case_table():
    """Triangles (as triples of edge ids) for each of the 256 sign patterns.

    Construction: on each cube face, walk its corners counter-clockwise as
    seen from outside the cube and record the edges where the solid/vacuum
    state changes.  Every crossing where the walk enters solid is joined to
    the next crossing (where it leaves solid); on a face with four crossings
    this cuts each solid corner off on its own, a rule that depends on the
    face alone, so two cubes sharing a face make the same (opposite-directed)
    segments and the surface closes.  Each crossing edge starts one segment
    and ends another, so the segments chain into closed loops; each loop is
    fanned into triangles.  The loop direction makes (V1-V0) x (V2-V0) point
    out of the solid.
    """
    off = _corner_offsets()
    edges = _edges()
    edge_of = {}
    for e, (a, b, _) in enumerate(edges):
        edge_of[(a, b)] = e
        edge_of[(b, a)] = e
    faces = []
    for axis in range(3):
        for side in (0, 1):
            cs = [c for c in range(8) if ((c >> axis) & 1) == side]
            p = off[cs].astype(np.float64)
            ctr = p.mean(axis=0)
            u, v = [ax for ax in range(3) if ax != axis]
            ang = np.arctan2(p[:, v] - ctr[v], p[:, u] - ctr[u])
            order = [cs[i] for i in np.argsort(ang)]
            q = off[order].astype(np.float64)
            nrm = np.cross(q[1] - q[0], q[2] - q[0])
            outward = np.zeros(3)
            outward[axis] = 1.0 if side else -1.0
            if np.dot(nrm, outward) < 0:
                order = order[::-1]
            faces.append(order)
    table = []
    for case in range(256):
        solid = [(case >> c) & 1 for c in range(8)]
        nxt = {}
        for order in faces:
            cross = []
            for i in range(4):
                a, b = order[i], order[(i + 1) % 4]
                if solid[a] != solid[b]:
                    cross.append((edge_of[(a, b)], bool(solid[b])))  # True = entering solid
            for i, (e, entering) in enumerate(cross):
                if entering:
                    e_next = cross[(i + 1) % len(cross)][0]
                    assert e not in nxt
                    nxt[e] = e_next
        tris = []
        seen = set()
        for start in sorted(nxt):
            if start in seen:
                continue
            loop = [start]
            seen.add(start)
            e = nxt[start]
            while e != start:
                loop.append(e)
                seen.add(e)
                e = nxt[e]
            for i in range(1, len(loop) - 1):
                tris.append((loop[0], loop[i], loop[i + 1]))
        table.append(tris)
    max_t = max(len(t) for t in table)
    arr = -np.ones((256, max_t, 3), dtype=np.int64)
    cnt = np.zeros(256, dtype=np.int64)
    for c, tris in enumerate(table):
        cnt[c] = len(tris)
        if tris:
            arr[c, :len(tris)] = np.array(tris)
    return arr, cnt


def marching_cubes_periodic(f: np.ndarray, thr: float, h: float,
                            frac_clamp: float = 1e-3) -> np.ndarray:
    """Isosurface {f = thr} of a sample grid periodic in x and y.

    ``f`` has shape (nx, ny, nz); sample (i, j, k) sits at (i h, j h, k h).
    In x and y sample nx wraps to sample 0, so cube i spans [i h, (i+1) h]
    for i < nx and every vertex lies in [0, nx h].  In z the grid is open
    (cubes k < nz-1).  Solid is ``f > thr``.  Edge crossings are clamped to
    [frac_clamp, 1 - frac_clamp] of the edge to avoid slivers.  Returns a
    float32 triangle soup [n, 3, 3] with normals pointing out of the solid.
    """
    table, cnt = _mc_case_table()
    off = _corner_offsets()
    edges = np.array(_edges(), dtype=np.int64)
    nx, ny, nz = f.shape
    out = []
    for k0 in range(0, nz - 1, 16):
        k1 = min(nz - 1, k0 + 16)
        ii, jj, kk = np.meshgrid(np.arange(nx), np.arange(ny), np.arange(k0, k1), indexing="ij")
        ii, jj, kk = ii.ravel(), jj.ravel(), kk.ravel()
        vals = np.empty((ii.size, 8), dtype=np.float64)
        for c in range(8):
            vals[:, c] = f[(ii + off[c, 0]) % nx, (jj + off[c, 1]) % ny, kk + off[c, 2]]
        case = np.zeros(ii.size, dtype=np.int64)
        for c in range(8):
            case |= (vals[:, c] > thr).astype(np.int64) << c
        nt = cnt[case]
        keep = nt > 0
        ii, jj, kk, vals, case, nt = ii[keep], jj[keep], kk[keep], vals[keep], case[keep], nt[keep]
        base = np.stack([ii, jj, kk], axis=1)
        for s in range(table.shape[1]):
            m = nt > s
            if not m.any():
                break
            tv = np.empty((int(m.sum()), 3, 3), dtype=np.float64)
            for v in range(3):
                e = table[case[m], s, v]
                a, b, axis = edges[e, 0], edges[e, 1], edges[e, 2]
                sel = np.arange(e.size)
                fa = vals[m][sel, a]
                fb = vals[m][sel, b]
                frac = np.clip((thr - fa) / (fb - fa), frac_clamp, 1.0 - frac_clamp)
                p = (base[m] + off[a]).astype(np.float64)
                p[sel, axis] += frac
                tv[:, v, :] = p * h
            out.append(tv)
    if not out:
        return np.zeros((0, 3, 3), dtype=np.float32)
    tri = np.concatenate(out).astype(np.float32)
    e1 = tri[:, 1] - tri[:, 0]
    e2 = tri[:, 2] - tri[:, 0]
    area2 = np.linalg.norm(np.cross(e1, e2), axis=1)
    tri = tri[area2 > 1e-12 * h * h]
    return np.ascontiguousarray(tri)


def grf_foam(n: int, porosity: float, corr_len_vox: float = 2.0, seed: int = 1806,
             h: float = 10.0, substrate_layers: int = 2, vacuum_layers: int = 1) -> Mesh:
    """Periodic foam: n^3 random field, void fraction ``porosity``.

    Solid voxels are those above the porosity quantile of the field; the
    threshold sits halfway between two neighbouring sorted samples so no
    sample lies on the isosurface.  ``substrate_layers`` solid sample layers
    are added below the foam (z = 0 ...) and ``vacuum_layers`` void layers
    above it; the escape plane z_top is the top sample layer.  Units of h are
    nanometres (10 nm voxels by default).
    """
    f = grf_field(n, corr_len_vox, seed)
    s = np.sort(f.ravel())
    m = int(round(porosity * s.size))
    m = min(max(m, 1), s.size - 1)
    thr = 0.5 * (s[m - 1] + s[m])
    nz = substrate_layers + n + vacuum_layers
    g = np.empty((n, n, nz), dtype=np.float64)
    g[:, :, :substrate_layers] = thr + 1.0
    g[:, :, substrate_layers:substrate_layers + n] = f
    g[:, :, substrate_layers + n:] = thr - 1.0
    tri = marching_cubes_periodic(g, thr, h)
    box = Box(n * h, n * h, 0.0, (nz - 1) * h)
    return Mesh(tri, box, name=f"grf{n}_p{porosity:g}_l{corr_len_vox:g}_s{seed}",
                porosity=float(m) / s.size)


def flat_plane(length: float = 160.0, height: float | None = None) -> Mesh:
    """Two triangles covering [0, L]^2 at z = 0, normal +z.

    The escape plane is z_top = L/16 by default (a thin slab keeps grazing
    secondaries from needing thousands of periodic wraps before escaping).
    """
    L = float(length)
    tri = np.array([[[0, 0, 0], [L, 0, 0], [L, L, 0]],
                    [[0, 0, 0], [L, L, 0], [0, L, 0]]], dtype=np.float32)
    ztop = L / 16.0 if height is None else float(height)
    return Mesh(tri, Box(L, L, -L, ztop), name=f"flat{L:g}")


def _quad(p0, p1, p2, p3):
    """Two CCW triangles of the planar quad p0 p1 p2 p3 (normal by right hand)."""
    return [[p0, p1, p2], [p0, p2, p3]]


def square_well(a: float = 100.0, depth: float = 100.0, rim: float | None = None) -> Mesh:
    """Square pit a x a, ``depth`` deep, in a periodic cell of side a + 2 rim.

    Floor at z = 0 (normal +z), four walls facing into the pit, plateau at
    z = depth split on a 3 x 3 grid so every edge is shared by exactly two
    triangles (no T-junctions).  The pit opening is [rim, rim + a]^2; the
    escape plane sits a/4 above the plateau.
    """
    r = a / 16.0 if rim is None else float(rim)
    L = a + 2 * r
    x = [0.0, r, r + a, L]
    h = float(depth)
    tris = []
    # floor
    tris += _quad((r, r, 0), (r + a, r, 0), (r + a, r + a, 0), (r, r + a, 0))
    # walls, normals into the pit
    tris += _quad((r, r, 0), (r, r + a, 0), (r, r + a, h), (r, r, h))              # x = r, +x
    tris += _quad((r + a, r, 0), (r + a, r, h), (r + a, r + a, h), (r + a, r + a, 0))  # x = r+a, -x
    tris += _quad((r, r, 0), (r, r, h), (r + a, r, h), (r + a, r, 0))              # y = r, +y
    tris += _quad((r, r + a, 0), (r + a, r + a, 0), (r + a, r + a, h), (r, r + a, h))  # y = r+a, -y
    # plateau (3 x 3 grid minus the centre)
    for i in range(3):
        for j in range(3):
            if i == 1 and j == 1:
                continue
            tris += _quad((x[i], x[j], h), (x[i + 1], x[j], h), (x[i + 1], x[j + 1], h), (x[i], x[j + 1], h))
    tri = np.ascontiguousarray(np.array(tris, dtype=np.float32))
    return Mesh(tri, Box(L, L, -h, h + a / 4.0), name=f"well{a:g}x{h:g}")


def opening_window(a: float = 100.0, rim: float | None = None):
    """Source window (x0, x1, y0, y1) covering exactly the pit opening."""
    r = a / 16.0 if rim is None else float(rim)
    return (r, r + a, r, r + a)


def batched_foams(n_foams: int = 16, p_lo: float = 0.30, p_hi: float = 0.90, g_lo: int = 48, g_hi: int = 128,
                  seed: int = 1806):
    """The batched workload's foams: porosity linspace(p_lo, p_hi, n) and grid
    sizes linspace(g_lo, g_hi, n) rounded to multiples of 16, paired by a
    seeded shuffle.  Returns a list of (grid, porosity, seed)."""
    por = np.linspace(p_lo, p_hi, n_foams)
    grids = (np.round(np.linspace(g_lo, g_hi, n_foams) / 16.0) * 16).astype(int)
    rng = np.random.Generator(np.random.Philox(seed))
    grids = grids[rng.permutation(n_foams)]
    return [(int(g), float(p), int(seed + k)) for k, (g, p) in enumerate(zip(grids, por))]


def gibson_ashby_cage(v_f: float, cell: float = 1000.0, C: float = 28.0, res: int = 128) -> Mesh:
    """Cubic open-cell cage on a flat substrate (the verification geometry of Section 3.1).

    Ligament thickness t from the Gibson-Ashby relation v_f = C (t/l)^2 with the
    paper's C = 28 and l = `cell` (nm).  The periodic cell (l x l, periodic in x
    and y) holds square-section ligaments of side t centred on the cube edges:
    a vertical ligament on the cell corner, and two horizontal ligaments (along
    x and along y) on the top edges at z = l; the bottom edges lie in the solid
    substrate (z < 0).  The solid is meshed by the periodic marching cubes on a
    `res` samples-per-cell grid of the field max(substrate, ligaments), each
    term the signed Chebyshev distance to a ligament's surface.
    """
    l = float(cell)
    t = l * math.sqrt(v_f / C)
    h = l / res
    n_below, n_above = 2, int(math.ceil((0.5 * t) / h)) + 3
    nz = n_below + res + n_above
    x = np.arange(res) * h
    z = (np.arange(nz) - n_below + 0.5) * h            # half-voxel shift: no sample on z = 0
    dx = np.minimum(x, l - x)                            # periodic distance to the corner line x = 0
    X = dx[:, None, None]
    Y = dx[None, :, None]
    Z = z[None, None, :]
    f_sub = -Z + 0.0 * X + 0.0 * Y
    f_vert = np.minimum(0.5 * t - np.maximum(X, Y), l + 0.5 * t - Z)
    f_top_x = 0.5 * t - np.maximum(Y, np.abs(Z - l)) + 0.0 * X
    f_top_y = 0.5 * t - np.maximum(X, np.abs(Z - l)) + 0.0 * Y
    f = np.maximum(np.maximum(f_sub, f_vert), np.maximum(f_top_x, f_top_y))
    thr = 1e-7 * h                                      # no sample exactly on the surface
    tri = marching_cubes_periodic(f, thr, h, frac_clamp=1e-4)
    tri[..., 2] += np.float32(z[0])
    box = Box(l, l, float(z[0]), float(z[-1]))
    m = Mesh(np.ascontiguousarray(tri), box, name=f"cage_vf{v_f:g}_l{l:g}")
    m.porosity = 1.0 - (3 * (t / l) ** 2 - 2 * (t / l) ** 3)   # solid fraction of the ligament frame
    return m
