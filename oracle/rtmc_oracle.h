/*
 * rtmc_oracle.h -- plain FP64 CPU oracle for ray-tracing Monte Carlo (RTMC)
 * secondary-electron yield.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library; the product path never
 * calls it.  It shares no code, header or constant table with the CUDA path.
 *
 * What it computes (Alvarado et al., Sections 2.1-2.2 and Fig. 1):
 *   a primary ray enters the periodic cell from the top plane, the closest
 *   front-facing triangle is found by a brute-force scan over every element
 *   (Section 2.1, the four checks), the local incidence angle sets the
 *   expected yield from a flat-surface table (Section 2.2), daughters are
 *   appended to the end of the primary's ray tree and traced in turn, and a
 *   ray leaving through z_top is counted as emitted (Section 2.2, last
 *   paragraph; Fig. 1 gamma_eff).
 *
 * All geometry and sampling arithmetic is FP64.  Random numbers come from
 * Philox4x32-10 (Salmon et al., SC'11) keyed as described in rtmc_oracle.c.
 */
#ifndef RTMC_ORACLE_H
#define RTMC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct { double lx, ly, z_min, z_top; } orc_box;

typedef struct {
    const float* delta;      /* n_e * n_theta, energy-major */
    int32_t n_e, n_theta;
    double e_lo_ev, e_hi_ev, theta_step_deg;
    double phi_ev;           /* secondary-spectrum parameter (4.55 eV)      */
    double e_cut_ev;         /* secondary-spectrum cut (50 eV)              */
    double absorb_min_ev;    /* below: absorbed_low on a facet hit (10 eV)  */
    double regen_min_ev;     /* daughters at/above may re-emit              */
    int32_t max_generation;  /* daughters of generation g < this re-emit    */
    int32_t k_max;           /* daughter count cap (15)                     */
    int32_t model;           /* ORC_MODEL_TABLE or ORC_MODEL_PAPER_FIT      */
} orc_physics;

/* emission models: the yield table with Poisson counts and the truncated
   spectrum, or the paper's own fits (Eq. 6, Eq. 7, stochastic rounding and
   the two-daughter split of Section 2.2; readings R16-R18) */
enum { ORC_MODEL_TABLE = 0, ORC_MODEL_PAPER_FIT = 1 };

typedef struct {
    double energy_ev, theta_deg;
    uint64_t seed;
    uint32_t item;                 /* Philox counter word 3                  */
    int32_t random_azimuth;
    int64_t n_primaries;
    uint64_t primary_offset;       /* ids are offset + i ...                 */
    const uint64_t* prim_ids;      /* ... unless this list is given          */
    double src_x0, src_x1, src_y0, src_y1;   /* all 0 -> whole cell          */
    int32_t n_ebins, n_abins;
    double hist_e_max_ev;
    int32_t max_wraps;
    int32_t n_threads;             /* 0 -> OpenMP default                    */
    int32_t random_polar;          /* 1: cosine-law polar angle (reading R14) */
    int32_t n_zbins;               /* penetration-depth bins (reading R15)    */
} orc_run;

typedef struct {
    int64_t n_primaries, rays, escaped, absorbed_low, absorbed_other;
    int64_t emitters, emitted, regenerated, capped, lost, wraps;
    int64_t sum_k, sum_k2;
    double e_sum, e2_sum, sey, sey_se;
} orc_result;

/* fate of one ray */
enum { ORC_ESCAPED = 0, ORC_EMITTER = 1, ORC_ABSORBED_LOW = 2,
       ORC_ABSORBED_OTHER = 3, ORC_LOST = 4 };

typedef struct {
    uint64_t prim;
    uint32_t path;
    int32_t gen, fate, tri, k, e_bin, a_bin, wraps;
    double t;        /* length parameter of the final segment (hit or exit) */
    double energy;   /* ray energy, eV                                      */
    double cos_in;   /* -d.n at a facet hit, d_z at an escape, 0 if lost    */
    double flight;   /* path length over every segment (wraps included)     */
} orc_record;        /* 72 bytes */

int orc_run_rtmc(const float* tri, int64_t n_tri, const orc_box* box,
                 const orc_physics* phys, const orc_run* run, orc_result* out,
                 int64_t* hist_e, int64_t* hist_a, int64_t* hist_z,
                 orc_record* rec, int64_t rec_cap, int64_t* n_rec);

/* Closest front-facing hit in one cell (no periodic walk); tri_id = -1 on a miss. */
void orc_closest_hit(const float* tri, int64_t n_tri, const double o[3], const double d[3],
                     int64_t exclude, double* t, int64_t* tri_id, double* u, double* v);

/* Same scan with the paper's Moller-Trumbore solve (Eq. 5, determinant read as
   (D x L2) . L1) and the four checks of Section 2.1; eps = parallel tolerance. */
void orc_closest_hit_mt(const float* tri, int64_t n_tri, const double o[3], const double d[3],
                        int64_t exclude, double eps, double* t, int64_t* tri_id,
                        double* u, double* v);

/* Periodic walk of one ray: fate (ORC_ESCAPED / ORC_EMITTER meaning "hit" / ORC_LOST). */
int orc_trace_ray(const float* tri, int64_t n_tri, const orc_box* box, const double o[3],
                  const double d[3], int64_t origin_tri, int32_t max_wraps,
                  int64_t* tri_id, double* t, double* u, double* v, int32_t* wraps,
                  double o_last[3]);

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
double orc_lookup_delta(const orc_physics* phys, double e_ev, double alpha_rad);
int orc_poisson(double lambda, double u, int32_t k_max, int* capped);
double orc_sample_energy(const orc_physics* phys, double u);
void orc_cosine_dir(const double n[3], double u1, double u2, double d[3]);
double orc_gamma_fit(double e_ev, double alpha_deg);
double orc_esee_fit(double e_ev, double alpha_deg);
int orc_round_stochastic(double gamma, double u, int32_t k_max, int* capped);

#ifdef __cplusplus
}
#endif
#endif
