"""Checks of the seeded input generators (meshes and tables)."""
import collections
import math

import numpy as np
import pytest
from scipy.ndimage import map_coordinates

from paper_1806_00205_gb300 import inputs as I


def _directed_edges(mesh):
    """Directed edges with vertices identified across the periodic x/y faces."""
    v = mesh.tri.astype(np.float64).copy()
    for ax, L in ((0, mesh.box.lx), (1, mesh.box.ly)):
        v[..., ax] = np.where(v[..., ax] == np.float32(L), 0.0, v[..., ax])
    cnt = collections.Counter()
    for t in v:
        for i in range(3):
            a, b = tuple(t[i]), tuple(t[(i + 1) % 3])
            cnt[(a, b)] += 1
    return cnt


def _is_closed(mesh):
    cnt = _directed_edges(mesh)
    return all(n == 1 and cnt.get((b, a), 0) == 1 for (a, b), n in cnt.items())


@pytest.mark.parametrize("n,p,seed", [(8, 0.5, 1), (16, 0.5, 1806), (16, 0.8, 3), (12, 0.3, 9)])
def test_foam_is_closed_and_oriented(n, p, seed):
    m = I.grf_foam(n, p, 2.0, seed)
    assert m.tri.dtype == np.float32 and m.tri.flags.c_contiguous
    assert _is_closed(m), "every directed edge must meet its reverse exactly once"
    assert abs(m.porosity - p) < 1.0 / n ** 3 + 1e-12
    # normals point from solid (field > threshold) into vacuum
    f = I.grf_field(n, 2.0, seed)
    s = np.sort(f.ravel())
    k = int(round(p * s.size))
    thr = 0.5 * (s[k - 1] + s[k])
    core = np.empty((n, n, n + 3))
    core[:, :, :2] = thr + 1
    core[:, :, 2:n + 2] = f
    core[:, :, n + 2:] = thr - 1
    g = np.empty((n + 1, n + 1, n + 3))
    g[:n, :n] = core
    g[n, :n] = core[0]
    g[:n, n] = core[:, 0]
    g[n, n] = core[0, 0]
    c = m.tri.astype(np.float64).mean(axis=1) / 10.0
    nr = np.cross(m.tri[:, 1] - m.tri[:, 0], m.tri[:, 2] - m.tri[:, 0]).astype(np.float64)
    nr /= np.linalg.norm(nr, axis=1)[:, None]
    fo = map_coordinates(g, (c + 0.05 * nr).T, order=1, mode="nearest")
    fi = map_coordinates(g, (c - 0.05 * nr).T, order=1, mode="nearest")
    # (a trilinear probe of the field, so a few slivers in folds may disagree)
    assert np.mean(fo < fi) > 0.99
    # inside the cell, below the escape plane
    assert m.tri[..., 0].min() >= 0 and m.tri[..., 0].max() <= m.box.lx
    assert m.tri[..., 2].max() < m.box.z_top and m.tri[..., 2].min() > m.box.z_min


def test_tiny_foam_size():
    m = I.grf_foam(16, 0.5)           # 16^3 voxels of 10 nm, correlation 2 voxels
    assert 2500 < m.n_tri < 6000
    assert m.box.lx == 160.0 and m.box.z_top == 180.0


def test_well_and_plane():
    w = I.square_well(100.0, 50.0)
    assert _is_closed(w) and w.n_tri == 26
    fp = I.flat_plane(160.0)
    n = np.cross(fp.tri[:, 1] - fp.tri[:, 0], fp.tri[:, 2] - fp.tri[:, 0])
    assert np.all(n[:, 2] > 0) and np.all(n[:, :2] == 0)


def test_see_table():
    t = I.see_table()
    assert t.delta.shape == (64, 18) and t.delta.dtype == np.float32
    g = t.energy_grid()
    assert math.isclose(g[0], 1.0) and math.isclose(g[-1], 2000.0)
    # the universal curve at 300 eV, normal incidence
    assert abs(float(I.lin_joy_delta(300.0, 0.0)) - 1.078076) < 1e-6
    assert np.all(np.diff(t.delta, axis=1) > 0)          # grows with angle


def test_grf_is_seeded():
    a = I.grf_field(8, 2.0, 5)
    b = I.grf_field(8, 2.0, 5)
    c = I.grf_field(8, 2.0, 6)
    assert np.array_equal(a, b) and not np.array_equal(a, c)


@pytest.mark.parametrize("v_f", [0.01, 0.04])
def test_gibson_ashby_cage(v_f):
    m = I.gibson_ashby_cage(v_f, res=96)
    assert _is_closed(m)
    t = 1000.0 * math.sqrt(v_f / 28.0)           # v_f = C (t/l)^2, C = 28 (Section 3.1)
    # the vertical ligament's cross-section at mid height spans t (up to a voxel)
    mid = m.tri[(np.abs(m.tri[..., 2] - 500.0) < 30.0).all(axis=1)]
    xs = mid[..., 0].ravel()
    near = np.minimum(xs, 1000.0 - xs)
    assert abs(2 * near.max() - t) < 2 * 1000.0 / 96
    # normals of the substrate point up, the top plane is above everything
    flat = m.tri[(np.abs(m.tri[..., 2]) < 1e-3).all(axis=1)]
    n = np.cross(flat[:, 1] - flat[:, 0], flat[:, 2] - flat[:, 0])
    assert np.all(n[:, 2] > 0)
    assert m.tri[..., 2].max() < m.box.z_top
