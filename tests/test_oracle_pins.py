"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: published
known-answer vectors, closed forms (view factors, spectrum moments, the flat
surface's exact expectation), textbook distributions, brute force on tiny
inputs, and conservation identities.  None of these need a GPU.
"""
import math
import os

import numpy as np
import pytest
from scipy import integrate, stats

import oracle as O
from paper_1806_00205_gb300 import inputs as I

HERE = os.path.dirname(os.path.abspath(__file__))
TABLE = I.see_table()
E47 = float(TABLE.energy_grid()[47])          # a grid energy (about 290.6 eV)


def _kat_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "philox4x32_10_kat.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = [int(x, 16) for x in line.split()]
                rows.append((w[0:4], w[4:6], w[6:10]))
    return rows


@pytest.mark.parametrize("ctr,key,expect", _kat_rows())
def test_philox_known_answers(ctr, key, expect):
    # Salmon et al. SC'11; vectors shipped with Random123 (tests/golden)
    assert list(O.philox(ctr, key)) == expect


# ---------------------------------------------------------------- geometry --

def test_flat_plane_closed_form_hit():
    """A vertical ray onto the 2-triangle plane: t, triangle and (u, v) are known."""
    fp = I.flat_plane(160.0)
    L = 160.0
    rng = np.random.default_rng(3)
    for _ in range(200):
        x, y = rng.uniform(0, L, 2)
        z0 = rng.uniform(1, 5)
        t, j, u, v = O.closest_hit(fp, [x, y, z0], [0, 0, -1])
        assert math.isclose(t, z0, rel_tol=1e-14)
        if y < x:    # triangle 0: (0,0) (L,0) (L,L); P = u V1 + v V2
            assert j == 0
            assert math.isclose(v, y / L, abs_tol=1e-13) and math.isclose(u, (x - y) / L, abs_tol=1e-13)
        else:        # triangle 1: (0,0) (L,L) (0,L)
            assert j == 1
            assert math.isclose(u, x / L, abs_tol=1e-13) and math.isclose(v, (y - x) / L, abs_tol=1e-13)
        # back-face culling (Section 2.1 check 1): from below the plane the ray sees nothing
        t2, j2, _, _ = O.closest_hit(fp, [x, y, -z0], [0, 0, 1])
        assert j2 == -1 and math.isinf(t2)


def test_watertight_matches_paper_moller_trumbore_on_foam():
    """Watertight FP64 scan vs the paper's M-T solve with its four checks."""
    mesh = I.grf_foam(8, 0.5, 1.5, seed=11)
    rng = np.random.default_rng(5)
    box = mesh.box
    agree = 0
    n = 400
    for _ in range(n):
        o = np.array([rng.uniform(0, box.lx), rng.uniform(0, box.ly), box.z_top])
        d = rng.normal(size=3)
        d[2] = -abs(d[2]) - 0.2
        d /= np.linalg.norm(d)
        a = O.closest_hit(mesh, o, d)
        b = O.closest_hit(mesh, o, d, method="mt", eps=1e-12)
        if a[1] == b[1]:
            agree += 1
            if a[1] >= 0:
                assert math.isclose(a[0], b[0], rel_tol=1e-10)
                assert abs(a[2] - b[2]) < 1e-9 and abs(a[3] - b[3]) < 1e-9
    assert agree >= n - 1


def test_hit_point_lies_on_ray_and_facet():
    mesh = I.grf_foam(8, 0.5, 1.5, seed=12)
    rng = np.random.default_rng(6)
    tri = mesh.tri.astype(np.float64)
    hits = 0
    for _ in range(300):
        o = np.array([rng.uniform(0, mesh.box.lx), rng.uniform(0, mesh.box.ly), mesh.box.z_top])
        d = np.array([rng.normal(), rng.normal(), -3.0])
        d /= np.linalg.norm(d)
        t, j, u, v = O.closest_hit(mesh, o, d)
        if j < 0:
            continue
        hits += 1
        p = (1 - u - v) * tri[j, 0] + u * tri[j, 1] + v * tri[j, 2]
        assert np.allclose(o + t * d, p, atol=1e-9)
        assert u >= 0 and v >= 0 and u + v <= 1 + 1e-12
        # no other front-facing triangle is hit closer (brute force over all of them)
        n = np.cross(tri[:, 1] - tri[:, 0], tri[:, 2] - tri[:, 0])
        assert np.dot(n[j], d) < 0
    assert hits > 50


def test_closest_hit_is_minimum_over_single_triangles():
    """Brute force on a tiny mesh: the scan's answer is the min over one-triangle scans."""
    mesh = I.grf_foam(6, 0.5, 1.2, seed=13)
    rng = np.random.default_rng(7)
    for _ in range(40):
        o = np.array([rng.uniform(0, mesh.box.lx), rng.uniform(0, mesh.box.ly), mesh.box.z_top * 0.7])
        d = rng.normal(size=3)
        d /= np.linalg.norm(d)
        t, j, _, _ = O.closest_hit(mesh, o, d)
        best, bj = math.inf, -1
        for k in range(mesh.n_tri):
            one = I.Mesh(mesh.tri[k:k + 1], mesh.box)
            tk, jk, _, _ = O.closest_hit(one, o, d)
            if jk == 0 and tk < best:
                best, bj = tk, k
        assert bj == j and (j < 0 or best == t)


def test_periodic_walk_counts_wraps():
    """A daughter leaving the flat plane crosses the lateral faces a known number of times."""
    fp = I.flat_plane(160.0)        # z_top = 10
    L, H = 160.0, 10.0
    for dx, dy, dz in [(3.0, 0.5, 0.01), (-2.0, 1.0, 0.05), (0.3, -4.0, 0.02), (1.0, 1.0, 2.0)]:
        d = np.array([dx, dy, dz]) / math.sqrt(dx * dx + dy * dy + dz * dz)
        o = np.array([17.0, 33.0, 0.0])
        r = O.trace_ray(fp, o, d, origin_tri=0, max_wraps=100000)
        assert r["fate"] == O.ESCAPED
        t_top = H / d[2]
        xf, yf = o[0] + t_top * d[0], o[1] + t_top * d[1]
        expect = abs(math.floor(xf / L)) + abs(math.floor(yf / L))
        assert r["wraps"] == expect
        # the last segment ends on z_top at the wrapped exit point
        end = r["o_last"] + r["t"] * d
        assert math.isclose(end[2], H, abs_tol=1e-9)
        assert math.isclose(end[0], xf - L * math.floor(xf / L), abs_tol=1e-6)
        assert math.isclose(end[1], yf - L * math.floor(yf / L), abs_tol=1e-6)
    # too many wraps -> lost
    d = np.array([1.0, 0.0, 1e-4]); d /= np.linalg.norm(d)
    r = O.trace_ray(fp, [5.0, 5.0, 0.0], d, origin_tri=0, max_wraps=8)
    assert r["fate"] == O.LOST and r["wraps"] == 9


def test_record_incidence_cosine_and_flight_length():
    """The records' error-bound fields on a flat plane in closed form: a primary
    at polar angle theta meets the plane with -d.n = cos(theta) after a flight of
    z_top / cos(theta), wraps included; an escaping daughter records d_z and a
    flight of z_top / d_z from its start on the plane."""
    fp = I.flat_plane(160.0, height=400.0)      # tall slab: steep primaries wrap several times
    for theta in (0.0, 37.0, 75.0):
        r = O.run(fp, TABLE, E47, theta, 3000, seed=31, records=True)
        rec = r["records"]
        prim, dau = rec[rec["gen"] == 0], rec[rec["gen"] == 1]
        c = math.cos(math.radians(theta))
        assert np.allclose(prim["cos_in"], c, rtol=0, atol=1e-12)
        assert np.allclose(prim["flight"], 400.0 / c, rtol=1e-12, atol=0)
        if theta == 75.0:
            assert prim["wraps"].max() >= 5
        esc = dau[dau["fate"] == O.ESCAPED]
        assert esc.size > 1000
        assert np.allclose(esc["flight"] * esc["cos_in"], 400.0, rtol=1e-9, atol=0)
        assert np.all((esc["cos_in"] > 0) & (esc["cos_in"] <= 1))


# ---------------------------------------------------------------- sampling --

def test_delta_lookup_grid_nodes_and_bilinearity():
    g = TABLE.energy_grid()
    for i in (0, 10, 47, 63):
        for j in (0, 7, 17):
            val = O.lookup_delta(TABLE, g[i], math.radians(5.0 * j))
            assert math.isclose(val, float(TABLE.delta[i, j]), rel_tol=1e-9)
    # midpoint in (ln E, theta) is the mean of the four corners
    e_mid = math.sqrt(g[20] * g[21])
    val = O.lookup_delta(TABLE, e_mid, math.radians(12.5))
    corners = TABLE.delta[20:22, 2:4].astype(np.float64).mean()
    assert math.isclose(val, corners, rel_tol=1e-9)
    # interpolation error against the analytic curve is small off-grid
    for e in (55.0, 300.0, 777.0):
        for th in (0.0, 33.0, 71.0):
            exact = float(I.lin_joy_delta(e, math.radians(th)))
            assert abs(O.lookup_delta(TABLE, e, math.radians(th)) - exact) < 4e-3
    # clamping outside the grid
    assert math.isclose(O.lookup_delta(TABLE, 1e4, math.radians(89.0)),
                        float(TABLE.delta[63, 17]), rel_tol=1e-9)


def test_poisson_inversion_matches_pmf():
    m = 200000
    u = (np.arange(m) + 0.5) / m
    for lam in (0.3, 1.078, 3.7):
        ks = np.array([O.poisson(lam, x)[0] for x in u])
        freq = np.bincount(ks, minlength=16)[:16] / m
        pmf = stats.poisson.pmf(np.arange(16), lam)
        assert np.abs(freq - pmf).max() < 2.0 / m
    k, capped = O.poisson(40.0, 0.999)
    assert k == 15 and capped == 1
    k, capped = O.poisson(1.0, 0.5)
    assert capped == 0


def test_energy_sampler_inverts_the_spectrum_cdf():
    phi, ecut = 4.55, 50.0
    pdf = lambda e: e / (e + phi) ** 4
    z = integrate.quad(pdf, 0, ecut)[0]
    for u in (1e-6, 0.01, 0.25, 0.5, 0.9, 0.999999):
        e = O.sample_energy(u)
        assert 0.0 <= e <= ecut
        assert math.isclose(integrate.quad(pdf, 0, e, epsabs=1e-14, epsrel=1e-12)[0] / z, u,
                            rel_tol=1e-9, abs_tol=1e-12)


def test_cosine_direction_law_and_basis():
    rng = np.random.default_rng(9)
    normals = [np.array([0, 0, 1.0]), np.array([0, 0, -1.0]), np.array([1.0, 0, 0])]
    normals += [v / np.linalg.norm(v) for v in rng.normal(size=(20, 3))]
    m = 64
    for n in normals:
        cos_sum = 0.0
        for i in range(m):
            for j in range(m):
                u1, u2 = (i + 0.5) / m, (j + 0.5) / m
                d = O.cosine_dir(n, u1, u2)
                assert math.isclose(np.linalg.norm(d), 1.0, rel_tol=1e-12)
                assert math.isclose(float(d @ n), math.sqrt(1 - u1), rel_tol=1e-9, abs_tol=1e-12)
                cos_sum += float(d @ n)
        # Malley: <cos theta'> = 2/3 under the cosine law
        assert abs(cos_sum / (m * m) - 2.0 / 3.0) < 1e-3


# ------------------------------------------------------------ whole runs --

def test_flat_plane_reproduces_table_yield():
    """Section 3.1: on a flat surface RTMC returns the sampling function exactly."""
    fp = I.flat_plane(160.0)
    for theta, j in ((0.0, 0), (60.0, 12)):
        r = O.run(fp, TABLE, E47, theta, 400000, seed=2024, item=j)
        lam = float(TABLE.delta[47, j])
        assert r["lost"] == 0 and r["absorbed_low"] == 0 and r["absorbed_other"] == 0
        assert r["escaped"] == r["emitted"] == r["sum_k"]      # every daughter escapes
        assert abs(r["sey"] - lam) < 3.0 * r["sey_se"], (r["sey"], lam, r["sey_se"])
        # Poisson counts: variance equals the mean
        assert abs(r["sey_se"] ** 2 * r["n_primaries"] / lam - 1.0) < 0.02


def test_flat_plane_spectra():
    fp = I.flat_plane(160.0)
    r = O.run(fp, TABLE, E47, 0.0, 300000, seed=99)
    n = r["escaped"]
    phi, ecut = 4.55, 50.0
    pdf = lambda e: e / (e + phi) ** 4
    z = integrate.quad(pdf, 0, ecut)[0]
    edges = np.linspace(0, ecut, 65)
    pe = np.array([integrate.quad(pdf, a, b)[0] for a, b in zip(edges[:-1], edges[1:])]) / z
    assert stats.chisquare(r["hist_e"], pe * n).pvalue > 1e-3
    th = np.radians(np.linspace(0, 90, 19))
    pa = np.diff(np.sin(th) ** 2)                        # cosine law about +z
    assert stats.chisquare(r["hist_a"], pa * n).pvalue > 1e-3
    mean = integrate.quad(lambda e: e * pdf(e), 0, ecut)[0] / z
    m2 = integrate.quad(lambda e: e * e * pdf(e), 0, ecut)[0] / z
    se = math.sqrt((m2 - mean * mean) / n)
    assert abs(r["e_sum"] / n - mean) < 3 * se
    assert math.isclose(mean, 7.148468, rel_tol=1e-6)


def view_factor_squares(x):
    """Parallel, coaxial equal squares, side a, gap h, X = a/h (textbook closed form)."""
    s = math.sqrt(1 + x * x)
    return (2.0 / (math.pi * x * x)) * (math.log((1 + x * x) / math.sqrt(1 + 2 * x * x))
                                        + 2 * x * s * math.atan(x / s) - 2 * x * math.atan(x))


@pytest.mark.parametrize("a_over_h", [0.5, 1.0, 2.0])
def test_square_well_view_factor(a_over_h):
    a = 100.0
    well = I.square_well(a, a / a_over_h)
    r = O.run(well, TABLE, E47, 0.0, 300000, seed=31, window=I.opening_window(a))
    lam = float(TABLE.delta[47, 0])
    expect = lam * view_factor_squares(a_over_h)
    assert r["lost"] == 0
    assert abs(r["sey"] - expect) < 3.0 * r["sey_se"], (r["sey"], expect, r["sey_se"])
    # every daughter either escapes or is absorbed by a wall
    assert r["emitted"] == r["escaped"] + r["absorbed_low"] + r["absorbed_other"]


def test_view_factor_reference_values():
    # tabulated values of the closed form (X = 0.5, 1, 2, 4)
    for x, f in ((0.5, 0.068590), (1.0, 0.199825), (2.0, 0.415253), (4.0, 0.632036)):
        assert abs(view_factor_squares(x) - f) < 2e-6


def _conservation(r, n):
    assert r["n_primaries"] == n
    assert r["rays"] == n + r["emitted"]
    assert r["rays"] == (r["escaped"] + r["absorbed_low"] + r["absorbed_other"]
                         + r["emitters"] + r["lost"])
    assert r["sum_k"] == r["escaped"]
    assert r["hist_e"].sum() == r["escaped"] == r["hist_a"].sum()


def test_foam_conservation_and_records():
    mesh = I.grf_foam(16, 0.5)
    n = 3000
    r = O.run(mesh, TABLE, 300.0, 0.0, n, seed=5, records=True)
    _conservation(r, n)
    assert r["lost"] == 0                          # closed mesh: nothing leaks
    assert 0.2 < r["sey"] < 1.0                    # a foam traps part of the yield
    rec = r["records"]
    assert rec.size == r["rays"]
    # tree structure: one primary per id, daughters j < k of their parent
    prim = rec[rec["gen"] == 0]
    assert prim.size == n and np.all(prim["path"] == 1)
    kids = {}
    for x in rec[rec["gen"] == 1]:
        kids.setdefault(int(x["prim"]), []).append(int(x["path"]) - 16)
    for p in prim:
        got = sorted(kids.get(int(p["prim"]), []))
        assert got == list(range(int(p["k"])))
    esc = rec[rec["fate"] == O.ESCAPED]
    assert np.bincount(esc["e_bin"], minlength=64).tolist() == r["hist_e"].tolist()


def test_foam_results_independent_of_threads():
    mesh = I.grf_foam(16, 0.5)
    a = O.run(mesh, TABLE, 500.0, 30.0, 1500, seed=8, n_threads=1)
    b = O.run(mesh, TABLE, 500.0, 30.0, 1500, seed=8, n_threads=4)
    for k in ("rays", "escaped", "sum_k2", "wraps", "e_sum"):
        assert a[k] == b[k]
    assert (a["hist_a"] == b["hist_a"]).all()


def test_tertiaries_conserve():
    mesh = I.grf_foam(16, 0.7, seed=4)
    em = O.Emission(regen_min_ev=20.0, max_generation=2)
    n = 3000
    r = O.run(mesh, TABLE, 500.0, 0.0, n, seed=6, emission=em, records=True)
    _conservation(r, n)
    assert r["regenerated"] > 0
    rec = r["records"]
    assert (rec["gen"] == 2).any() and rec["gen"].max() == 2
    regen = rec[(rec["gen"] == 1) & (rec["fate"] == O.EMITTER)]
    assert np.all(regen["energy"] >= 20.0)


def test_primary_ids_replay_the_same_trees():
    """Counter-based streams: a subset of primaries replays exactly."""
    mesh = I.grf_foam(16, 0.5)
    full = O.run(mesh, TABLE, 300.0, 0.0, 400, seed=5, records=True)["records"]
    ids = np.array([3, 77, 150, 399], dtype=np.uint64)
    sub = O.run(mesh, TABLE, 300.0, 0.0, 0, seed=5, prim_ids=ids, records=True)["records"]
    want = full[np.isin(full["prim"], ids)]
    assert sub.tobytes() == want.tobytes()


# ------------------------------------------ random incidence and depth --

def test_random_incidence_is_cosine_law():
    """Reading R14: an isotropic beam crossing the top plane has cos^2(theta) uniform on (0, 1).

    On a flat plane a primary that does not wrap hits after t = h / cos(theta);
    a thin slab (h = 0.1 nm over a 160 nm cell) keeps wraps rare."""
    h = 0.1
    fp = I.flat_plane(160.0, height=h)
    n = 20000
    r = O.run(fp, TABLE, E47, 37.0, n, seed=77, random_polar=True, records=True)
    rec = r["records"]
    prim = rec[rec["gen"] == 0]
    assert prim.size == n and np.all(prim["fate"] == O.EMITTER)
    direct = prim[prim["wraps"] == 0]
    assert direct.size > 0.99 * n
    c2 = (h / direct["t"]) ** 2
    assert stats.kstest(c2, "uniform").pvalue > 1e-3
    # a mistaken law (cos theta uniform, or theta uniform) is far off: mean cos theta is 2/3 here
    assert abs(np.mean(np.sqrt(c2)) - 2.0 / 3.0) < 0.01


def test_random_incidence_flat_yield():
    """Flat plane, cosine-law incidence: E[SEY] = int_0^{pi/2} delta(E, theta) sin(2 theta) d theta.

    At a grid energy delta is linear in theta between the 5-degree nodes and
    constant past 85 degrees (the table's last node)."""
    fp = I.flat_plane(160.0)
    r = O.run(fp, TABLE, E47, 0.0, 400000, seed=4242, random_polar=True)
    th = np.radians(5.0 * np.arange(TABLE.delta.shape[1]))
    row = TABLE.delta[47].astype(np.float64)
    expect = integrate.quad(lambda a: np.interp(a, th, row) * math.sin(2.0 * a), 0.0, math.pi / 2,
                            points=list(th[1:]), limit=200)[0]
    assert r["lost"] == 0 and r["escaped"] == r["emitted"]
    assert abs(r["sey"] - expect) < 3.0 * r["sey_se"], (r["sey"], expect, r["sey_se"])
    # differs from normal incidence by far more than the error
    assert r["sey"] - float(row[0]) > 10.0 * r["sey_se"]


def test_depth_tally_flat_plane():
    """Reading R15: every primary stops on the plane, 10 nm below z_top (box 170 nm deep, 16 bins)."""
    fp = I.flat_plane(160.0)
    n = 20000
    for polar in (False, True):
        r = O.run(fp, TABLE, E47, 30.0, n, seed=5, random_polar=polar, n_zbins=16)
        hz = r["hist_z"]
        assert hz[0] == n and hz.sum() == n == r["emitters"]


def test_depth_tally_square_well_view_factors():
    """Depth profile in a square well with absorbing walls.

    Cosine-law emission from the uniformly lit a x a floor crosses the
    coaxial square at height z with probability F(a/z) (parallel-squares view
    factor), so the walls between heights z1 < z2 take F(a/z1) - F(a/z2) of
    the daughters and the opening passes F(a/h).  Each primary stops on the
    floor at depth z_top - 0."""
    a, hw, nz = 100.0, 100.0, 40
    well = I.square_well(a, hw)
    box = well.box
    n = 200000
    r = O.run(well, TABLE, E47, 0.0, n, seed=8, window=I.opening_window(a), n_zbins=nz)
    hz = r["hist_z"].astype(np.int64)
    assert hz.sum() == r["emitters"] + r["absorbed_low"] + r["absorbed_other"]
    dz = (box.z_top - box.z_min) / nz
    floor_bin = int((box.z_top - 0.0) // dz)

    def cross(z):                       # fraction of floor emission passing height z
        return 1.0 if z <= 0.0 else view_factor_squares(a / z)

    p = np.zeros(nz)
    for b in range(nz):
        z_hi = min(hw, box.z_top - b * dz)
        z_lo = max(0.0, box.z_top - (b + 1) * dz)
        if z_hi > z_lo:
            p[b] = cross(z_lo) - cross(z_hi)
    walls = hz.copy()
    walls[floor_bin] -= n
    assert walls[floor_bin] >= 0 and np.all(walls[p == 0.0] == 0)
    nd = r["emitted"]
    assert walls.sum() + r["escaped"] == nd
    obs = np.append(walls[p > 0], r["escaped"])
    exp = np.append(p[p > 0], cross(hw)) * nd
    assert abs(exp.sum() - nd) < 1e-6 * nd
    assert stats.chisquare(obs, exp).pvalue > 1e-3


# ------------------------------------------------- paper-fit emission --

PAPER = O.paper_emission()


def test_paper_fit_peak_matches_printed_value():
    """Section 3.2 quotes a maximum flat-tungsten yield of about 1.49; Eq. 6 at
    normal incidence (alpha in degrees, reading R16) peaks there near 416 eV."""
    e = np.arange(100.0, 1500.0, 0.5)
    g = np.array([O.gamma_fit(x, 0.0) for x in e])
    assert abs(g.max() - 1.49) < 0.005
    assert 380.0 < e[g.argmax()] < 450.0


def test_stochastic_rounding_footnote_example():
    """Section 2.2 footnote: gamma = 1.2 rounds down when xi >= 0.2, up otherwise."""
    assert O.round_stochastic(1.2, 0.25) == (1, 0)
    assert O.round_stochastic(1.2, 0.15) == (2, 0)
    assert O.round_stochastic(-0.3, 0.01) == (0, 0)
    assert O.round_stochastic(16.5, 0.9) == (15, 1)


def _paper_fit_rows():
    rows = []
    with open(os.path.join(HERE, "golden", "paper_fits.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                w = line.split()
                rows.append((w[0], [float(x) for x in w[1:]]))
    return rows


@pytest.mark.parametrize("which,cols", _paper_fit_rows())
def test_paper_fits_match_term_by_term_table(which, cols):
    """Eq. 6 and Eq. 7 (Section 2.2) at points where every term matters.

    tests/golden/paper_fits.txt lists each printed term of the two equations
    worked out on its own (alpha != 0, the alpha^7 term, sin(E) < 0, a negative
    E_SEE), so a dropped term, a wrong sign or a mistyped coefficient in the
    oracle's transcription changes the value by far more than the tolerance."""
    e, a = cols[0], cols[1]
    if which == "gamma":
        terms, total = [cols[i - 1] for i in (3, 4, 5, 7, 8, 11)], cols[11]
        got = O.gamma_fit(e, a)
    else:
        terms, total = [cols[i - 1] for i in (3, 4, 6, 8, 9)], cols[9]
        got = O.esee_fit(e, a)
    assert math.isclose(math.fsum(terms), total, rel_tol=0, abs_tol=1e-12 * max(1.0, abs(total)))
    assert math.isclose(got, total, rel_tol=0, abs_tol=1e-11 * max(1.0, abs(total))), (which, e, a, got, total)


@pytest.mark.parametrize("energy,theta", [(416.0, 0.0), (150.0, 40.0), (1200.0, 75.0)])
def test_paper_fit_flat_plane_yield_is_gamma(energy, theta):
    """On a flat surface every daughter escapes, so E[SEY] = gamma(E, theta)
    and the count variance is f (1 - f), f = frac(gamma) (not Poisson's gamma)."""
    fp = I.flat_plane(160.0)
    n = 200000
    r = O.run(fp, TABLE, energy, theta, n, seed=3, emission=PAPER)
    g = O.gamma_fit(energy, theta)
    f = g - math.floor(g)
    assert r["lost"] == 0 and r["escaped"] == r["emitted"] == r["sum_k"]
    assert r["absorbed_low"] == 0 and r["absorbed_other"] == 0
    assert abs(r["sey"] - g) < 3.5 * math.sqrt(f * (1 - f) / n) + 1e-9
    var = r["sey_se"] ** 2 * n
    assert abs(var - f * (1 - f)) < 0.02 * f * (1 - f) + 1e-6


def test_paper_fit_pair_rule_on_flat_plane():
    """Two daughters of one emission (Section 2.2): beta_2 = pi/2 - beta_1, so
    cos^2(beta_1) + cos^2(beta_2) = 1, with E_1 = E_SEE sin(beta_1) and
    E_2 = E_SEE cos^2(beta_1); a single daughter carries E_SEE.  On a thin flat
    slab an escaping daughter that does not wrap travels t = h / cos(beta)."""
    h = 0.1
    fp = I.flat_plane(160.0, height=h)
    energy, theta = 1200.0, 60.0                    # gamma about 1.5: one or two daughters
    esee = O.esee_fit(energy, theta)
    r = O.run(fp, TABLE, energy, theta, 20000, seed=19, emission=PAPER, records=True)
    rec = r["records"]
    d = rec[rec["gen"] == 1]
    assert np.all(d["fate"] == O.ESCAPED)
    k = np.bincount(d["prim"].astype(np.int64), minlength=20000)
    pairs = np.flatnonzero(k == 2)
    singles = np.flatnonzero(k == 1)
    assert pairs.size > 4000 and singles.size > 4000
    by_prim = {}
    for row in d:
        by_prim.setdefault(int(row["prim"]), {})[int(row["path"]) - 16] = row
    checked = 0
    for p in pairs[:3000]:
        a, b = by_prim[p][0], by_prim[p][1]
        if a["wraps"] or b["wraps"]:
            continue
        c1, c2 = h / a["t"], h / b["t"]
        assert abs(c1 * c1 + c2 * c2 - 1.0) < 1e-6
        s1 = math.sqrt(max(0.0, 1.0 - c1 * c1))
        assert abs(a["energy"] - esee * s1) < 1e-6 * esee
        assert abs(b["energy"] - esee * c1 * c1) < 1e-6 * esee
        checked += 1
    assert checked > 2500
    one = np.array([by_prim[p][0]["energy"] for p in singles])
    assert np.all(np.abs(one - esee) < 1e-9 * esee)
    c2s = np.array([(h / by_prim[p][0]["t"]) ** 2 for p in singles if not by_prim[p][0]["wraps"]])
    assert stats.kstest(c2s, "uniform").pvalue > 1e-3       # unpaired: cosine law


def test_paper_fit_foam_generations_and_conservation():
    """Unbounded generations above E_c on a 4 % solid foam: the energy falls
    each generation, trees end well before the 6-generation path limit, and
    every ray is accounted for."""
    mesh = I.grf_foam(24, 0.96)
    n = 6000
    r = O.run(mesh, TABLE, 2000.0, 0.0, n, seed=4, emission=PAPER, records=True)
    rec = r["records"]
    assert r["rays"] == n + r["emitted"] == rec.size
    assert r["rays"] == (r["escaped"] + r["absorbed_low"] + r["absorbed_other"] + r["emitters"] + r["lost"])
    assert r["regenerated"] > 0 and rec["gen"].max() < 6
    mean_e = [rec["energy"][rec["gen"] == g].mean() for g in range(rec["gen"].max() + 1)]
    assert all(b < a for a, b in zip(mean_e, mean_e[1:])), mean_e
    # a ray re-emits exactly when it is below the cap and at or above E_c
    hit = rec[(rec["fate"] != O.ESCAPED) & (rec["fate"] != O.LOST)]
    emit = hit["fate"] == O.EMITTER
    assert np.array_equal(emit, (hit["gen"] == 0) | (hit["energy"] >= PAPER.regen_min_ev))
