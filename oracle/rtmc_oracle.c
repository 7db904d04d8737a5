/*
 * rtmc_oracle.c -- plain, slow FP64 CPU oracle for RTMC secondary-electron
 * yield (Alvarado et al., "Monte Carlo Raytracing Method for Calculating
 * Secondary Electron Emission from Micro-Architected Surfaces").
 *
 * TEST INFRASTRUCTURE ONLY: loaded by the tests, the smoke check and the
 * benchmark's CPU-baseline leg; never by the product path.  It shares no
 * code with the CUDA path.  Everything is written for clarity: brute force
 * over every triangle for every ray segment (Section 2.1), one FIFO ray tree
 * per primary (Section 2.2), FP64 throughout.
 *
 * Readings of the paper used here (each is listed in the design notes):
 *  R1 Eq. 5 prints the determinant as (D x L2) . L2, which is identically 0;
 *     the Moller-Trumbore determinant (D x L2) . L1 is meant, and the
 *     barycentric condition "u^2 + v^2 <= 1" below Eq. 2 is read as u + v <= 1.
 *  R2 The closest-hit scan uses the watertight ray/triangle test of Woop,
 *     Benthin and Wald (JCGT 2013) in FP64; it is the same predicate as the
 *     M-T checks of Section 2.1 away from exact edges, and orc_closest_hit_mt
 *     gives the paper's form for comparison.  Ties in t go to the lowest id.
 *  R3 The incidence angle of Section 2.2 is acos(-D.n): D points into the
 *     surface and n out of it, so the printed acos(D.n) would exceed 90 deg.
 *  R4 Periodic x/y boundaries (Section 2.2, last paragraph) are a cell walk:
 *     a ray that leaves the cell laterally re-enters on the opposite face
 *     (x before y on an exact corner); more than max_wraps wraps, or leaving
 *     through z_min, is counted as lost.  The origin triangle is skipped only
 *     before the first wrap.
 *  R5 Number of daughters: Poisson(delta(E, alpha)) by sequential inversion,
 *     capped at k_max; daughter energy from the pdf E/(E+phi)^4 on
 *     [0, E_cut]; direction cosine-law about the facet normal in the
 *     orthonormal basis of Duff et al. (JCGT 2017).
 *  R6 A primary always emits at its first hit; a daughter of generation g
 *     emits only when g < max_generation and E >= regen_min; otherwise it is absorbed
 *     (absorbed_low below absorb_min).  A daughter of any energy that
 *     reaches z_top moving up is emitted (Section 2.2, last paragraph).
 *  R7 Random streams: Philox4x32-10, key = (seed lo, seed hi), counter =
 *     (prim lo, prim hi, path, item).  Primary path = 1; daughter j of a ray
 *     with path p has path 16 p + j.  The four words w0..w3 of a ray's block
 *     map to uniforms u = ((w >> 9) + 0.5) 2^-23, a 24-bit odd multiple of
 *     2^-24 and so exact in FP32 as in FP64.  Primary: u0, u1 -> (x, y)
 *     in the source window, u2 -> azimuth when random, u3 -> its Poisson
 *     draw.  Daughter: u0 -> energy, u1, u2 -> direction, u3 -> its own
 *     Poisson draw if it re-emits.
 *  R8 delta(E, theta) is bilinear in (ln E, theta) on the table grid, with
 *     E and theta clamped to the grid.
 *  R14 Random primary incidence (Section 3.2, normal versus random
 *     incidence) is the flux of an isotropic beam through the top plane:
 *     the polar angle follows the cosine law, sin^2 theta = u0 of a second
 *     Philox block (path 0, never a daughter path), and the azimuth is
 *     uniform (u2 of the primary's block).  The item angle is then unused.
 *  R15 The penetration profile (Section 3.2) tallies the depth z_top - z of
 *     the point where each ray's flight ends on a facet, of any generation,
 *     whether it re-emits or not: the electron itself stops there.  Bins
 *     split [0, z_top - z_min] evenly, clamped at both ends.
 *  R16 Paper-fit emission (model ORC_MODEL_PAPER_FIT), Section 2.2: the
 *     angle in Eq. 6 and Eq. 7 is the local incidence angle in degrees, E in
 *     eV, and sin(E) takes E as radians, as printed.  gamma < 0 counts as 0
 *     and E_SEE < 0 as 0 eV.  The count is gamma rounded stochastically
 *     (the footnote): floor(gamma) + 1 when u3 < gamma - floor(gamma).
 *  R17 Daughters of one emission come in pairs (0,1), (2,3), ...: a pair
 *     shares xi = u1 of its first daughter's block; the first takes
 *     E_SEE sqrt(xi) at polar angle asin(sqrt(xi)), the second
 *     (1 - xi) E_SEE at pi/2 minus that angle.  An unpaired daughter (a
 *     single emission, or the last of an odd count) takes E_SEE at a
 *     cosine-law angle (sin^2 = its own u1).  Every azimuth is uniform
 *     (u2 of the daughter's own block) in the Duff et al. basis.
 *  R18 E_c = phi + E_F is regen_min: a daughter below it still flies (and
 *     escapes through z_top) but stops at the facet it hits, so on a flat
 *     surface E[SEY] = gamma exactly (Section 3.1).  "Unbounded"
 *     generations end at max_generation (at most 6, the depth the 32-bit
 *     ray path holds); the fits shrink the energy each generation, so the
 *     cap is rarely reached.
 *
 * Eq. 6 and Eq. 7 are pinned by a table of their printed terms worked out
 * one by one at sixteen (E, alpha) points (alpha != 0, sin E < 0, a negative
 * E_SEE), and Eq. 6's maximum by the 1.49 that Section 3.2 quotes for flat W.
 */
#include "rtmc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11, Section 4)             */
/* ------------------------------------------------------------------------ */

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    /* multipliers and Weyl key increments from the Philox paper */
    const uint64_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u;
    const uint32_t W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t p0 = M0 * (uint64_t)c0;
        uint64_t p1 = M1 * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* The four uniforms of the ray (prim, path) in stream `item` (reading R7). */
static void ray_uniforms(uint64_t seed, uint64_t prim, uint32_t path, uint32_t item, double u[4])
{
    uint32_t ctr[4] = { (uint32_t)prim, (uint32_t)(prim >> 32), path, item };
    uint32_t key[2] = { (uint32_t)seed, (uint32_t)(seed >> 32) };
    uint32_t w[4];
    orc_philox4x32_10(ctr, key, w);
    for (int i = 0; i < 4; ++i)
        u[i] = ((double)(w[i] >> 9) + 0.5) * (1.0 / 8388608.0);
}

/* ------------------------------------------------------------------------ */
/* Geometry (Section 2.1)                                                    */
/* ------------------------------------------------------------------------ */

static void vert(const float* tri, int64_t j, int v, double p[3])
{
    const float* q = tri + 9 * j + 3 * v;
    p[0] = q[0]; p[1] = q[1]; p[2] = q[2];
}

static void sub3(const double a[3], const double b[3], double r[3])
{
    r[0] = a[0] - b[0]; r[1] = a[1] - b[1]; r[2] = a[2] - b[2];
}

static void cross3(const double a[3], const double b[3], double r[3])
{
    r[0] = a[1] * b[2] - a[2] * b[1];
    r[1] = a[2] * b[0] - a[0] * b[2];
    r[2] = a[0] * b[1] - a[1] * b[0];
}

static double dot3(const double a[3], const double b[3])
{
    return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

/* unit facet normal n = s/|s|, s = (V1-V0) x (V2-V0)  (Section 2.1) */
static void facet_normal(const float* tri, int64_t j, double n[3])
{
    double v0[3], v1[3], v2[3], l1[3], l2[3];
    vert(tri, j, 0, v0); vert(tri, j, 1, v1); vert(tri, j, 2, v2);
    sub3(v1, v0, l1); sub3(v2, v0, l2);
    cross3(l1, l2, n);
    double s = sqrt(dot3(n, n));
    n[0] /= s; n[1] /= s; n[2] /= s;
}

/* Watertight ray/triangle test (reading R2).  Accepts front-facing hits only
   (check 1), rejects a zero determinant (check 2), keeps points with all
   three barycentric weights >= 0 (check 3) and t > 0.  Returns 1 on a hit. */
typedef struct { int kx, ky, kz; double sx, sy, sz; } shear_t;

static shear_t make_shear(const double d[3])
{
    shear_t s;
    int kz = 0;
    if (fabs(d[1]) > fabs(d[kz])) kz = 1;
    if (fabs(d[2]) > fabs(d[kz])) kz = 2;
    int kx = (kz + 1) % 3, ky = (kx + 1) % 3;
    if (d[kz] < 0.0) { int tmp = kx; kx = ky; ky = tmp; }   /* keep the winding */
    s.kx = kx; s.ky = ky; s.kz = kz;
    s.sx = d[kx] / d[kz];
    s.sy = d[ky] / d[kz];
    s.sz = 1.0 / d[kz];
    return s;
}

static int watertight(const float* tri, int64_t j, const double o[3], const shear_t* s,
                      double* t, double* u, double* v)
{
    double v0[3], v1[3], v2[3], a[3], b[3], c[3];
    vert(tri, j, 0, v0); vert(tri, j, 1, v1); vert(tri, j, 2, v2);
    sub3(v0, o, a); sub3(v1, o, b); sub3(v2, o, c);
    double ax = a[s->kx] - s->sx * a[s->kz], ay = a[s->ky] - s->sy * a[s->kz];
    double bx = b[s->kx] - s->sx * b[s->kz], by = b[s->ky] - s->sy * b[s->kz];
    double cx = c[s->kx] - s->sx * c[s->kz], cy = c[s->ky] - s->sy * c[s->kz];
    double U = cx * by - cy * bx;   /* weight of V0 */
    double V = ax * cy - ay * cx;   /* weight of V1 */
    double W = bx * ay - by * ax;   /* weight of V2 */
    if (U < 0.0 || V < 0.0 || W < 0.0) return 0;   /* outside, or back-facing */
    double det = U + V + W;
    if (det == 0.0) return 0;                       /* parallel / degenerate  */
    double az = s->sz * a[s->kz], bz = s->sz * b[s->kz], cz = s->sz * c[s->kz];
    double T = U * az + V * bz + W * cz;
    if (T <= 0.0) return 0;                         /* behind the origin      */
    *t = T / det;
    *u = V / det;
    *v = W / det;
    return 1;
}

void orc_closest_hit(const float* tri, int64_t n_tri, const double o[3], const double d[3],
                     int64_t exclude, double* t, int64_t* tri_id, double* u, double* v)
{
    shear_t s = make_shear(d);
    double best = INFINITY, bu = 0.0, bv = 0.0;
    int64_t bj = -1;
    for (int64_t j = 0; j < n_tri; ++j) {           /* every element (Section 2.1) */
        if (j == exclude) continue;
        double n[3];
        facet_normal(tri, j, n);
        if (dot3(n, d) >= 0.0) continue;            /* check 1: back-face culling  */
        double tj, uj, vj;
        if (!watertight(tri, j, o, &s, &tj, &uj, &vj)) continue;
        if (tj < best) { best = tj; bj = j; bu = uj; bv = vj; }   /* check 4 */
    }
    *t = best; *tri_id = bj; *u = bu; *v = bv;
}

/* The paper's Moller-Trumbore form, Eq. 5 with the determinant read as
   (D x L2) . L1 (reading R1) and the four checks of Section 2.1. */
void orc_closest_hit_mt(const float* tri, int64_t n_tri, const double o[3], const double d[3],
                        int64_t exclude, double eps, double* t, int64_t* tri_id,
                        double* u, double* v)
{
    double best = INFINITY, bu = 0.0, bv = 0.0;
    int64_t bj = -1;
    for (int64_t j = 0; j < n_tri; ++j) {
        if (j == exclude) continue;
        double v0[3], v1[3], v2[3], l1[3], l2[3], tt[3], n[3], p[3], q[3];
        vert(tri, j, 0, v0); vert(tri, j, 1, v1); vert(tri, j, 2, v2);
        sub3(v1, v0, l1); sub3(v2, v0, l2);
        cross3(l1, l2, n);
        if (dot3(n, d) >= 0.0) continue;                 /* check 1 */
        cross3(d, l2, p);                                /* D x L2 */
        double det = dot3(p, l1);
        if (fabs(det) < eps) continue;                   /* check 2 */
        sub3(o, v0, tt);                                 /* T = O - V0 */
        cross3(tt, l1, q);                               /* T x L1 */
        double tj = dot3(q, l2) / det;
        double uj = dot3(p, tt) / det;
        double vj = dot3(q, d) / det;
        if (uj < 0.0 || vj < 0.0 || uj + vj > 1.0) continue;   /* check 3 */
        if (tj <= 0.0) continue;
        if (tj < best) { best = tj; bj = j; bu = uj; bv = vj; }   /* check 4 */
    }
    *t = best; *tri_id = bj; *u = bu; *v = bv;
}

/* Periodic cell walk (reading R4).  Returns ORC_EMITTER for "hit a facet",
   ORC_ESCAPED or ORC_LOST. */
/* The periodic walk; *flight gets the length of the whole path (every
   segment, the last one included), used only to state error bounds. */
static int walk_ray(const float* tri, int64_t n_tri, const orc_box* box, const double o_in[3],
                    const double d[3], int64_t origin_tri, int32_t max_wraps,
                    int64_t* tri_id, double* t, double* u, double* v, int32_t* wraps,
                    double o_last[3], double* flight)
{
    double o[3] = { o_in[0], o_in[1], o_in[2] };
    int64_t excl = origin_tri;
    int32_t nw = 0;
    double run_len = 0.0;
    for (;;) {
        double th, uh, vh;
        int64_t j;
        orc_closest_hit(tri, n_tri, o, d, excl, &th, &j, &uh, &vh);
        if (j >= 0) {
            *tri_id = j; *t = th; *u = uh; *v = vh; *wraps = nw;
            memcpy(o_last, o, sizeof o);
            *flight = run_len + th;
            return ORC_EMITTER;
        }
        /* no facet in this cell: find the face the ray leaves through */
        double tx = INFINITY, ty = INFINITY, tz = INFINITY;
        if (d[0] > 0.0) tx = (box->lx - o[0]) / d[0];
        else if (d[0] < 0.0) tx = (0.0 - o[0]) / d[0];
        if (d[1] > 0.0) ty = (box->ly - o[1]) / d[1];
        else if (d[1] < 0.0) ty = (0.0 - o[1]) / d[1];
        if (d[2] > 0.0) tz = (box->z_top - o[2]) / d[2];
        else if (d[2] < 0.0) tz = (box->z_min - o[2]) / d[2];
        *tri_id = -1; *u = 0.0; *v = 0.0; *wraps = nw;
        memcpy(o_last, o, sizeof o);
        if (tz < tx && tz < ty) {
            *t = tz;
            *flight = run_len + tz;
            return d[2] > 0.0 ? ORC_ESCAPED : ORC_LOST;  /* top: emission; bottom: leak */
        }
        if (++nw > max_wraps) { *t = fmin(tx, ty); *wraps = nw; *flight = run_len + *t; return ORC_LOST; }
        run_len += fmin(tx, ty);
        if (tx <= ty) {
            o[1] = o[1] + tx * d[1]; o[2] = o[2] + tx * d[2];
            o[0] = d[0] > 0.0 ? 0.0 : box->lx;      /* re-enter on the opposite face */
        } else {
            o[0] = o[0] + ty * d[0]; o[2] = o[2] + ty * d[2];
            o[1] = d[1] > 0.0 ? 0.0 : box->ly;
        }
        excl = -1;
    }
}

int orc_trace_ray(const float* tri, int64_t n_tri, const orc_box* box, const double o_in[3],
                  const double d[3], int64_t origin_tri, int32_t max_wraps,
                  int64_t* tri_id, double* t, double* u, double* v, int32_t* wraps,
                  double o_last[3])
{
    double flight;
    return walk_ray(tri, n_tri, box, o_in, d, origin_tri, max_wraps, tri_id, t, u, v, wraps, o_last, &flight);
}

/* ------------------------------------------------------------------------ */
/* Sampling (Section 2.2)                                                    */
/* ------------------------------------------------------------------------ */

/* delta(E, alpha): bilinear in (ln E, angle) on the table grid (reading R8). */
double orc_lookup_delta(const orc_physics* ph, double e_ev, double alpha_rad)
{
    double x = log(e_ev / ph->e_lo_ev) / log(ph->e_hi_ev / ph->e_lo_ev) * (ph->n_e - 1);
    if (x < 0.0) x = 0.0;
    if (x > ph->n_e - 1) x = ph->n_e - 1;
    int i = (int)floor(x);
    if (i > ph->n_e - 2) i = ph->n_e - 2;
    double fx = x - i;
    double y = alpha_rad * (180.0 / ORC_PI) / ph->theta_step_deg;
    if (y < 0.0) y = 0.0;
    if (y > ph->n_theta - 1) y = ph->n_theta - 1;
    int j = (int)floor(y);
    if (j > ph->n_theta - 2) j = ph->n_theta - 2;
    double fy = y - j;
    const float* T = ph->delta;
    int nt = ph->n_theta;
    double t00 = T[i * nt + j], t10 = T[(i + 1) * nt + j];
    double t01 = T[i * nt + j + 1], t11 = T[(i + 1) * nt + j + 1];
    return (1 - fx) * (1 - fy) * t00 + fx * (1 - fy) * t10 + (1 - fx) * fy * t01 + fx * fy * t11;
}

/* k = min{k : u < P(K <= k)} for K ~ Poisson(lambda), capped at k_max. */
int orc_poisson(double lambda, double u, int32_t k_max, int* capped)
{
    double p = exp(-lambda);
    double cdf = p;
    *capped = 0;
    for (int k = 0; k < k_max; ++k) {
        if (u < cdf) return k;
        p *= lambda / (k + 1);
        cdf += p;
    }
    if (!(u < cdf)) *capped = 1;
    return k_max;
}

/* normalised CDF of the pdf E/(E+phi)^4 on [0, inf): 1 - 3 s^2 + 2 s^3, s = phi/(E+phi) */
static double spectrum_cdf(double e, double phi)
{
    double s = phi / (e + phi);
    return 1.0 - 3.0 * s * s + 2.0 * s * s * s;
}

/* Daughter energy: inverse of the spectrum CDF truncated to [0, E_cut],
   found by bisection (reading R5). */
double orc_sample_energy(const orc_physics* ph, double u)
{
    double target = u * spectrum_cdf(ph->e_cut_ev, ph->phi_ev);
    double lo = 0.0, hi = ph->e_cut_ev;
    for (int it = 0; it < 200; ++it) {
        double mid = 0.5 * (lo + hi);
        if (mid <= lo || mid >= hi) break;
        if (spectrum_cdf(mid, ph->phi_ev) < target) lo = mid; else hi = mid;
    }
    return 0.5 * (lo + hi);
}

/* Eq. 6 (Section 2.2): SEE yield of flat tungsten, E in eV, alpha in
   degrees (reading R16). */
double orc_gamma_fit(double e, double a)
{
    return 3.05 + 1.7949e-5 * a * a + 6.15e-7 * e * e
           - (371.317 - exp(0.04826 * a)) / (87.602 + e)
           - 1.974e-3 * e - 0.1097 * cos(0.1201 + 2.469 * a);
}

/* Eq. 7 (Section 2.2): energy of an emitted secondary, eV. */
double orc_esee_fit(double e, double a)
{
    return 0.195 * e + 1.6e-4 * e * e + 0.148 * a * sin(e) + 3.44e-15 * e * pow(a, 7.0) - 6.54;
}

/* Section 2.2 footnote: a fractional yield is rounded up when u falls below
   its fractional part, down otherwise; negative yields emit nothing. */
int orc_round_stochastic(double gamma, double u, int32_t k_max, int* capped)
{
    if (gamma < 0.0) gamma = 0.0;
    double fl = floor(gamma);
    int k = (int)fl + (u < gamma - fl ? 1 : 0);
    *capped = k > k_max;
    return k > k_max ? k_max : k;
}

/* Cosine-law direction about the unit normal n: sin^2(theta') = u1,
   phi' = 2 pi u2, in the orthonormal basis of Duff et al. (JCGT 2017). */
void orc_cosine_dir(const double n[3], double u1, double u2, double d[3])
{
    double sgn = n[2] >= 0.0 ? 1.0 : -1.0;
    double a = -1.0 / (sgn + n[2]);
    double b = n[0] * n[1] * a;
    double t1[3] = { 1.0 + sgn * n[0] * n[0] * a, sgn * b, -sgn * n[0] };
    double t2[3] = { b, sgn + n[1] * n[1] * a, -n[1] };
    double st = sqrt(u1), ct = sqrt(1.0 - u1);
    double x = st * cos(2.0 * ORC_PI * u2), y = st * sin(2.0 * ORC_PI * u2);
    for (int i = 0; i < 3; ++i) d[i] = x * t1[i] + y * t2[i] + ct * n[i];
}

/* ------------------------------------------------------------------------ */
/* The ray tree of one primary (Section 2.2, Fig. 1)                         */
/* ------------------------------------------------------------------------ */

typedef struct {
    double o[3], d[3], e;
    uint32_t path;
    int32_t gen;
    int64_t origin_tri;
} orc_ray;

typedef struct {
    orc_result r;
    int64_t *he, *ha, *hz;
    orc_record* rec;
    int64_t nrec, caprec;
} orc_local;

static void push_record(orc_local* L, const orc_record* r)
{
    if (L->nrec == L->caprec) {
        L->caprec = L->caprec ? 2 * L->caprec : 1024;
        L->rec = (orc_record*)realloc(L->rec, (size_t)L->caprec * sizeof(orc_record));
    }
    L->rec[L->nrec++] = *r;
}

static void run_primary(const float* tri, int64_t n_tri, const orc_box* box,
                        const orc_physics* ph, const orc_run* run, uint64_t prim,
                        orc_local* L, int want_rec, int64_t* k_out, double* es_out, double* e2_out)
{
    double x0 = run->src_x0, x1 = run->src_x1, y0 = run->src_y0, y1 = run->src_y1;
    if (x0 == 0.0 && x1 == 0.0 && y0 == 0.0 && y1 == 0.0) { x1 = box->lx; y1 = box->ly; }

    int64_t cap = 16, head = 0, tail = 0;
    orc_ray* q = (orc_ray*)malloc((size_t)cap * sizeof(orc_ray));

    /* primary ray (Fig. 1 "Generate primary rays"; fixed or random incidence) */
    double u[4];
    ray_uniforms(run->seed, prim, 1u, run->item, u);
    double th = run->theta_deg * (ORC_PI / 180.0);
    double sin_t = sin(th), cos_t = cos(th);
    int random_az = run->random_azimuth;
    if (run->random_polar) {                  /* reading R14: cosine-law incidence */
        double v[4];
        ray_uniforms(run->seed, prim, 0u, run->item, v);
        sin_t = sqrt(v[0]);
        cos_t = sqrt(1.0 - v[0]);
        random_az = 1;
    }
    double ph_az = random_az ? 2.0 * ORC_PI * u[2] : 0.0;
    orc_ray r0;
    r0.o[0] = x0 + u[0] * (x1 - x0);
    r0.o[1] = y0 + u[1] * (y1 - y0);
    r0.o[2] = box->z_top;
    r0.d[0] = sin_t * cos(ph_az);
    r0.d[1] = sin_t * sin(ph_az);
    r0.d[2] = -cos_t;
    r0.e = run->energy_ev;
    r0.path = 1u;
    r0.gen = 0;
    r0.origin_tri = -1;
    q[tail++] = r0;

    int64_t kp = 0;
    double es = 0.0, e2 = 0.0;
    double de = run->hist_e_max_ev / run->n_ebins;
    double da = 90.0 / run->n_abins;

    while (head < tail) {                      /* "until a tree has no further branches" */
        orc_ray ray = q[head++];
        L->r.rays++;
        orc_record rc;
        memset(&rc, 0, sizeof rc);
        rc.prim = prim; rc.path = ray.path; rc.gen = ray.gen; rc.tri = -1;
        rc.k = 0; rc.e_bin = -1; rc.a_bin = -1; rc.energy = ray.e;

        int64_t j; double t, uh, vh, olast[3], flight;
        int32_t nw;
        int fate = walk_ray(tri, n_tri, box, ray.o, ray.d, ray.origin_tri, run->max_wraps,
                            &j, &t, &uh, &vh, &nw, olast, &flight);
        L->r.wraps += nw;
        rc.wraps = nw; rc.t = t; rc.flight = flight;

        if (fate == ORC_ESCAPED && ray.gen > 0) {
            /* emission event: reached z_max moving up */
            rc.fate = ORC_ESCAPED;
            L->r.escaped++;
            kp++;
            int eb = (int)floor(ray.e / de);
            if (eb > run->n_ebins - 1) eb = run->n_ebins - 1;
            if (eb < 0) eb = 0;
            double pol = acos(fmin(1.0, ray.d[2])) * (180.0 / ORC_PI);
            int ab = (int)floor(pol / da);
            if (ab > run->n_abins - 1) ab = run->n_abins - 1;
            if (ab < 0) ab = 0;
            L->he[eb]++; L->ha[ab]++;
            rc.e_bin = eb; rc.a_bin = ab;
            rc.cos_in = ray.d[2];
            es += ray.e; e2 += ray.e * ray.e;
        } else if (fate == ORC_ESCAPED || fate == ORC_LOST) {
            /* a primary that never meets the surface, a leak, or too many wraps */
            rc.fate = ORC_LOST;
            L->r.lost++;
        } else {
            rc.tri = (int32_t)j;
            {
                double nf[3];
                facet_normal(tri, j, nf);
                rc.cos_in = -dot3(ray.d, nf);
            }
            if (run->n_zbins > 0) {               /* reading R15: where the flight ends */
                double v0[3], v1[3], v2[3];
                vert(tri, j, 0, v0); vert(tri, j, 1, v1); vert(tri, j, 2, v2);
                double z = (1.0 - uh - vh) * v0[2] + uh * v1[2] + vh * v2[2];
                double dz = (box->z_top - box->z_min) / run->n_zbins;
                int zb = (int)floor((box->z_top - z) / dz);
                if (zb > run->n_zbins - 1) zb = run->n_zbins - 1;
                if (zb < 0) zb = 0;
                L->hz[zb]++;
            }
            int emits = ray.gen == 0 ||
                        (ray.gen < ph->max_generation && ray.e >= ph->regen_min_ev);
            if (!emits) {
                if (ray.e < ph->absorb_min_ev) { rc.fate = ORC_ABSORBED_LOW; L->r.absorbed_low++; }
                else { rc.fate = ORC_ABSORBED_OTHER; L->r.absorbed_other++; }
            } else {
                rc.fate = ORC_EMITTER;
                L->r.emitters++;
                if (ray.gen > 0) L->r.regenerated++;
                double n[3];
                facet_normal(tri, j, n);
                double cosa = -dot3(ray.d, n);
                double alpha = acos(fmin(1.0, cosa));          /* reading R3 */
                double ur[4];
                ray_uniforms(run->seed, prim, ray.path, run->item, ur);
                int capped, k;
                double esee = 0.0;
                if (ph->model == ORC_MODEL_PAPER_FIT) {          /* readings R16-R18 */
                    double a_deg = alpha * (180.0 / ORC_PI);
                    k = orc_round_stochastic(orc_gamma_fit(ray.e, a_deg), ur[3], ph->k_max, &capped);
                    esee = fmax(0.0, orc_esee_fit(ray.e, a_deg));
                } else {
                    double lam = orc_lookup_delta(ph, ray.e, alpha);
                    k = orc_poisson(lam, ur[3], ph->k_max, &capped);
                }
                L->r.capped += capped;
                L->r.emitted += k;
                rc.k = k;
                /* hit point on the facet from its barycentric coordinates, Eq. 2 */
                double v0[3], v1[3], v2[3], p[3];
                vert(tri, j, 0, v0); vert(tri, j, 1, v1); vert(tri, j, 2, v2);
                for (int c = 0; c < 3; ++c)
                    p[c] = (1.0 - uh - vh) * v0[c] + uh * v1[c] + vh * v2[c];
                for (int jj = 0; jj < k; ++jj) {
                    orc_ray dr;
                    dr.path = ray.path * 16u + (uint32_t)jj;
                    dr.gen = ray.gen + 1;
                    dr.origin_tri = j;
                    double ud[4];
                    ray_uniforms(run->seed, prim, dr.path, run->item, ud);
                    if (ph->model == ORC_MODEL_PAPER_FIT) {
                        int first = jj & ~1;
                        if (first + 1 < k) {                      /* one of a pair (R17) */
                            double uf[4];
                            ray_uniforms(run->seed, prim, ray.path * 16u + (uint32_t)first, run->item, uf);
                            double xi = uf[1];
                            if (jj == first) { dr.e = esee * sqrt(xi); orc_cosine_dir(n, xi, ud[2], dr.d); }
                            else { dr.e = (1.0 - xi) * esee; orc_cosine_dir(n, 1.0 - xi, ud[2], dr.d); }
                        } else {                                  /* unpaired */
                            dr.e = esee;
                            orc_cosine_dir(n, ud[1], ud[2], dr.d);
                        }
                    } else {
                        dr.e = orc_sample_energy(ph, ud[0]);
                        orc_cosine_dir(n, ud[1], ud[2], dr.d);
                    }
                    memcpy(dr.o, p, sizeof p);
                    if (tail == cap) {
                        cap *= 2;
                        q = (orc_ray*)realloc(q, (size_t)cap * sizeof(orc_ray));
                    }
                    q[tail++] = dr;                  /* appended to the end of the tree */
                }
            }
        }
        if (want_rec) push_record(L, &rc);
    }
    free(q);
    *k_out = kp; *es_out = es; *e2_out = e2;
}

int orc_run_rtmc(const float* tri, int64_t n_tri, const orc_box* box,
                 const orc_physics* ph, const orc_run* run, orc_result* out,
                 int64_t* hist_e, int64_t* hist_a, int64_t* hist_z,
                 orc_record* rec, int64_t rec_cap, int64_t* n_rec)
{
    if (!tri || n_tri <= 0 || !box || !ph || !run || !out || run->n_primaries < 0 ||
        run->n_ebins <= 0 || run->n_abins <= 0 || ph->n_e < 2 || ph->n_theta < 2 ||
        run->n_zbins < 0 || (run->n_zbins > 0 && !hist_z))
        return -1;
    int64_t N = run->n_primaries;
    int64_t* kp = (int64_t*)calloc((size_t)(N > 0 ? N : 1), sizeof(int64_t));
    double* es = (double*)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    double* e2 = (double*)calloc((size_t)(N > 0 ? N : 1), sizeof(double));
    int nthr = 1;
#ifdef _OPENMP
    nthr = run->n_threads > 0 ? run->n_threads : omp_get_max_threads();
#endif
    orc_local* loc = (orc_local*)calloc((size_t)nthr, sizeof(orc_local));
    for (int i = 0; i < nthr; ++i) {
        loc[i].he = (int64_t*)calloc((size_t)run->n_ebins, sizeof(int64_t));
        loc[i].ha = (int64_t*)calloc((size_t)run->n_abins, sizeof(int64_t));
        loc[i].hz = (int64_t*)calloc((size_t)(run->n_zbins > 0 ? run->n_zbins : 1), sizeof(int64_t));
    }
    int want_rec = rec != NULL;

#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthr)
#endif
    for (int64_t i = 0; i < N; ++i) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        uint64_t prim = run->prim_ids ? run->prim_ids[i] : run->primary_offset + (uint64_t)i;
        run_primary(tri, n_tri, box, ph, run, prim, &loc[tid], want_rec, &kp[i], &es[i], &e2[i]);
    }

    memset(out, 0, sizeof *out);
    memset(hist_e, 0, (size_t)run->n_ebins * sizeof(int64_t));
    memset(hist_a, 0, (size_t)run->n_abins * sizeof(int64_t));
    if (run->n_zbins > 0) memset(hist_z, 0, (size_t)run->n_zbins * sizeof(int64_t));
    int64_t nr = 0;
    for (int i = 0; i < nthr; ++i) {
        orc_result* r = &loc[i].r;
        out->rays += r->rays; out->escaped += r->escaped;
        out->absorbed_low += r->absorbed_low; out->absorbed_other += r->absorbed_other;
        out->emitters += r->emitters; out->emitted += r->emitted;
        out->regenerated += r->regenerated; out->capped += r->capped;
        out->lost += r->lost; out->wraps += r->wraps;
        for (int b = 0; b < run->n_ebins; ++b) hist_e[b] += loc[i].he[b];
        for (int b = 0; b < run->n_abins; ++b) hist_a[b] += loc[i].ha[b];
        for (int b = 0; b < run->n_zbins; ++b) hist_z[b] += loc[i].hz[b];
        if (want_rec) {
            for (int64_t k = 0; k < loc[i].nrec && nr < rec_cap; ++k) rec[nr++] = loc[i].rec[k];
        }
        free(loc[i].he); free(loc[i].ha); free(loc[i].hz); free(loc[i].rec);
    }
    if (n_rec) *n_rec = nr;
    /* per-primary sums in primary order: the same result for any thread count */
    for (int64_t i = 0; i < N; ++i) {
        out->sum_k += kp[i];
        out->sum_k2 += kp[i] * kp[i];
        out->e_sum += es[i];
        out->e2_sum += e2[i];
    }
    out->n_primaries = N;
    if (N > 0) out->sey = (double)out->sum_k / (double)N;
    if (N > 1) {
        double var = ((double)out->sum_k2 / (double)N - out->sey * out->sey) / (double)(N - 1);
        out->sey_se = var > 0.0 ? sqrt(var) : 0.0;
    }
    free(loc); free(kp); free(es); free(e2);
    return 0;
}
