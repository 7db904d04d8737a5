/*
 * rtmc.h -- C ABI of librtmc, a GB300 (sm_103a) implementation of ray-tracing
 * Monte Carlo (RTMC) secondary-electron yield from triangulated surfaces
 * (Alvarado, Chang, Nadvornick, Ghoniem, Marian: "Monte Carlo Raytracing
 * Method for Calculating Secondary Electron Emission from Micro-Architected
 * Surfaces").
 *
 * Method (Sections 2.1-2.2, Fig. 1): primary rays start on the top plane and
 * travel into a periodic triangle mesh; the closest front-facing facet is
 * found (Section 2.1, four checks; here through a linear BVH); at a hit the
 * local incidence angle and energy give the expected number of secondaries
 * from a flat-surface yield table (Section 2.2); each daughter gets an energy
 * and a cosine-law direction and is traced in turn; a ray that reaches the
 * top plane moving up is an emission event, and the yield is
 * emissions / primaries (Fig. 1, gamma_eff).
 *
 * Conventions for every entry point:
 *  - return 0 on success or a negative RTMC_ERR_* code; rtmc_last_error()
 *    then holds a one-line message for that context;
 *  - input pointers may be host or device memory (unified addressing decides)
 *    and are copied before the call returns; the caller keeps ownership;
 *  - outputs go to caller-owned host memory unless stated otherwise;
 *  - work is ordered on the context's stream and the call synchronises that
 *    stream before it returns;
 *  - a context is used by one host thread at a time.
 */
#ifndef RTMC_H
#define RTMC_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RTMC_OK                 0
#define RTMC_ERR_INVALID_ARG   -1
#define RTMC_ERR_OOM           -2
#define RTMC_ERR_CUDA          -3
#define RTMC_ERR_NOT_LOADED    -4
#define RTMC_ERR_NOT_BUILT     -5
#define RTMC_ERR_CAPACITY      -6
#define RTMC_ERR_TIMEOUT       -7
#define RTMC_ERR_DEVICE_CHECK  -8

#define RTMC_BVH_FP32 0     /* 64-byte nodes with FP32 child boxes */
#define RTMC_BVH_Q8   1     /* 32-byte nodes with 8-bit outward-rounded child boxes */
#define RTMC_BVH_W4   2     /* 128-byte 4-wide nodes with FP32 child boxes, collapsed from the binary hierarchy */
#define RTMC_BVH_Q4   3     /* 64-byte 4-wide nodes with 8-bit outward-rounded child boxes (the RTMC_BVH_W4 hierarchy, quantised) */
/* bvh_kind = node format | RTMC_BVH_LEAF(n): leaves of up to n (1..8) triangles, default 4 */
#define RTMC_BVH_LEAF(n) ((n) << 8)
/* ... | RTMC_BVH_PLOC: build the hierarchy by locally-ordered clustering
   (Meister & Bittner 2018) instead of the Karras split of the sorted codes */
#define RTMC_BVH_PLOC (1 << 16)

/* Ray fates (per-ray records) */
#define RTMC_ESCAPED        0
#define RTMC_EMITTER        1
#define RTMC_ABSORBED_LOW   2
#define RTMC_ABSORBED_OTHER 3
#define RTMC_LOST           4

typedef struct rtmc_ctx rtmc_ctx;

/* Periodic cell (Section 2.2, last paragraph): x in [0, lx), y in [0, ly)
   periodic; the substrate lies above z_min; z_top is the escape plane. */
typedef struct { double lx, ly, z_min, z_top; } rtmc_box;

/* Yield-table grid: E_i = e_lo * (e_hi/e_lo)^(i/(n_e-1)), theta_j = j * step. */
typedef struct {
    int32_t n_e, n_theta;
    double e_lo_ev, e_hi_ev, theta_step_deg;
} rtmc_grid;

/* Secondary emission (Section 2.2).  A primary always emits at its first hit;
   a daughter of generation g re-emits when g < max_generation (<= 6, the
   depth a 32-bit ray path holds) and E >= regen_min_ev, else it is absorbed
   (absorbed_low below absorb_min_ev).  Counts are capped at k_max (<= 15).
   model RTMC_EMISSION_TABLE: count ~ Poisson(delta(E, alpha)) from the
     loaded table; daughter energies follow E/(E+phi)^4 on [0, e_cut_ev];
     directions cosine-law about the facet normal.
   model RTMC_EMISSION_PAPER_FIT: the paper's own rules -- the yield gamma of
     Eq. 6 (alpha in degrees) rounded stochastically (floor(gamma) + 1 with
     probability gamma - floor(gamma)); the energy E_SEE of Eq. 7; daughters
     in pairs sharing xi, the first with E_SEE sqrt(xi) at polar angle
     asin(sqrt(xi)), the second with (1 - xi) E_SEE at pi/2 minus that angle;
     an unpaired daughter with E_SEE at a cosine-law angle; uniform azimuths.
     regen_min_ev plays E_c = phi + E_F.  The table is still loaded (its
     grid is validated) but not read; phi_ev and e_cut_ev are unused. */
#define RTMC_EMISSION_TABLE 0
#define RTMC_EMISSION_PAPER_FIT 1
typedef struct {
    double phi_ev, e_cut_ev, absorb_min_ev, regen_min_ev;
    int32_t max_generation, k_max;
    int32_t model;                 /* RTMC_EMISSION_TABLE or RTMC_EMISSION_PAPER_FIT */
} rtmc_emission;

typedef struct {
    int32_t n_ebins, n_abins;      /* escaped-energy bins on [0, hist_e_max); polar bins on [0, 90 deg) */
    double hist_e_max_ev;
    uint64_t primary_offset;       /* primary ids are offset .. offset + n - 1 */
    int32_t random_azimuth;        /* 0: incidence in the x-z plane; 1: uniform azimuth */
    int32_t max_wraps;             /* lateral re-entries before a ray counts as lost (0 -> 1024) */
    double src_x0, src_x1, src_y0, src_y1;   /* primary source window; all 0 -> whole cell */
    int64_t chunk;                 /* primaries per wavefront chunk (0 -> automatic) */
    int32_t block_threads;         /* traversal block size (0 -> 64) */
    int32_t blocks_per_sm;         /* persistent traversal blocks per SM (0 -> occupancy) */
    uint64_t* prim_hash;           /* optional DEVICE array [n_primaries]: per-primary
                                      sum of record hashes (see rtmc_record_hash) */
    int32_t profile;               /* 1: time every kernel launch with CUDA events */
    int32_t count_visits;          /* 1: count BVH node visits and triangle tests */
    int32_t traversal;             /* 0: default (2, and the column grid for generation 0
                                      at normal incidence, see rtmc_build_bvh); 1: one ray
                                      per lane per 32-ray tile; 2: while-while loop with
                                      per-lane ray refill, the hierarchy for every ray */
    int32_t fp64_retest;           /* 1: decide in FP64 every facet whose FP32 edge
                                      functions lie within 1e-5 (relative to their sum)
                                      of an edge, hit or miss, and take the distance of a
                                      closest hit with cos(incidence) < 1e-3 from the FP64
                                      test (while-while traversal only) */
    uint32_t item_base;            /* added to every item index (Philox counter word 3) */
    int32_t no_graph;              /* rtmc_run_batch: 1 = launch eagerly, no CUDA graph */
    int32_t stack_depth;           /* shared-memory traversal stack entries: 8, 16 or 32 (0 -> 16) */
    int32_t fetch_threshold;       /* warp refills rays when fewer lanes than this are busy (0 -> 28) */
    int32_t random_polar;          /* 1: random incidence -- polar angle from the cosine law
                                      (sin^2 theta = u of a second Philox block, path 0) and
                                      uniform azimuth; the item angle is ignored */
    int32_t n_zbins;               /* penetration-depth bins over [0, z_top - z_min] below
                                      z_top: every ray whose flight ends on a facet (0: off) */
    uint64_t* hist_z;              /* host [n_items][n_zbins] when n_zbins > 0 */
    int32_t id_order;              /* 1: queue primaries in id order; 0: order them by a
                                      Morton-ordered 128 x 128 grid of entry points
                                      (coherent traversal; results do not depend on order) */
    int32_t max_visits;            /* failure-detection bound: inner-node visits one cell
                                      traversal may make before its ray is abandoned and
                                      the call fails with RTMC_ERR_DEVICE_CHECK.  The
                                      library always applies the tree's own bound (its
                                      inner-node count + 1: a correct traversal visits each
                                      inner node at most once); a value > 0 lowers it */
    double queue_factor;           /* daughter-queue capacity of a chunk's first attempt,
                                      in rays per primary (0: twice the largest expected
                                      yield of the loaded emission, at least 2, at most
                                      k_max); if any chunk's daughters overflow their queue,
                                      the item (rtmc_run) or the batch (rtmc_run_batch) is
                                      run again from the start with twice the capacity, up
                                      to six times, then the call fails with
                                      RTMC_ERR_CAPACITY */
} rtmc_run_desc;

typedef struct {
    int64_t n_primaries, rays, escaped, absorbed_low, absorbed_other;
    int64_t emitters, emitted, regenerated, capped, lost, wraps;
    int64_t sum_k, sum_k2;                     /* per-primary escape count k: sum, sum of squares */
    double e_sum, e2_sum;                      /* escaped energy moments (eV, eV^2) */
    double sey, sey_se;                        /* sum_k / N and its standard error */
    double gpu_ms;                             /* device time of this (E, theta) item */
    int64_t launches;                          /* kernels launched for this item */
    int64_t node_visits, tri_tests;            /* with count_visits */
    double ms_generate, ms_traverse, ms_shade, ms_finalize;   /* with profile */
    int64_t traverse_launches;                 /* hierarchy traversal launches */
    int64_t retested;                          /* rays with a facet decided in FP64 */
    double ms_column;                          /* with profile: the column-grid launches */
    int64_t column_rays;                       /* rays traced through the column grid (not
                                                  counted in node_visits / tri_tests) */
    int64_t queue_retries;                     /* times the item (or batch) was run again
                                                  after a daughter-queue overflow */
} rtmc_result;

/* One traced ray: the integer event sequence used for parity checks. */
typedef struct {
    uint64_t prim;
    uint32_t path;            /* primary 1; daughter j of path p: 16 p + j */
    int32_t gen, fate, tri;   /* tri: original triangle id of the final hit or -1 */
    int32_t k, e_bin, a_bin, wraps;
    double t;                 /* length parameter of the final segment */
    double energy;            /* eV */
} rtmc_record;                /* 56 bytes */

/* Closest-hit query result (rtmc_trace_rays). */
typedef struct { float t, u, v; int32_t tri; } rtmc_hit;

/* Create a context on CUDA `device`.  `cuda_stream` is a cudaStream_t to
   order all work on, or NULL for a context-owned stream. */
int rtmc_create(rtmc_ctx** out, int32_t device, void* cuda_stream);
void rtmc_destroy(rtmc_ctx* ctx);
const char* rtmc_last_error(const rtmc_ctx* ctx);

/* Copy a triangle soup tri[n_tri][3][3] (FP32, vertices V0 V1 V2 with
   (V1-V0) x (V2-V0) pointing into vacuum, Section 2.1) into the context.
   All vertices must lie in [0,lx] x [0,ly] x (z_min, z_top).
   Writes the new mesh id. */
int rtmc_load_mesh(rtmc_ctx* ctx, const float* tri, int64_t n_tri, const rtmc_box* box,
                   int32_t* mesh_id);

/* Free the device memory of a mesh and its BVH; the id becomes invalid. */
int rtmc_unload_mesh(rtmc_ctx* ctx, int32_t mesh_id);

/* Copy the flat-surface yield table delta[n_e][n_theta] (FP32, energy-major;
   Section 2.2 "pre-calculated tables") and the emission parameters. */
int rtmc_load_see_tables(rtmc_ctx* ctx, const float* delta, const rtmc_grid* grid,
                         const rtmc_emission* emission);

/* Build the linear BVH of a loaded mesh on the device: Morton codes of the
   triangle centroids, radix sort, Karras hierarchy, bottom-up box refit,
   triangle repack; RTMC_BVH_Q8 also quantises each node's two child boxes to
   8 bits per coordinate in the node's own frame (origin + q 2^e, rounded
   outward).  `bvh_kind` is RTMC_BVH_FP32 or RTMC_BVH_Q8, optionally or-ed with
   RTMC_BVH_LEAF(n) to cap leaves at n triangles (subtrees with at most n
   triangles become one leaf).  With RTMC_BVH_PLOC the hierarchy comes from
   locally-ordered clustering instead (Meister & Bittner 2018: mutually
   nearest clusters by merged-box surface area within 16 positions of the
   Morton order merge, round by round), rewritten into the same node layout;
   it is deterministic and synchronises with the host once per round.
   RTMC_BVH_W4 builds the binary hierarchy and then collapses it into 4-wide
   nodes (each opens the inner child of largest surface area until it holds
   four children; leaves are those of the binary hierarchy), level by level,
   one host synchronisation per level.  RTMC_BVH_Q4 builds that 4-wide
   hierarchy and quantises every node to 64 bytes: per axis a quantum
   s = 2^e and a frame origin, and per child and plane one byte: each plane is
   moved outward by M 2^-21 + s 2^-7 beyond the 4-wide box (M the largest cell
   coordinate), then rounded outward to the quantum grid, so that the
   traversal may evaluate each plane with one FMA.  RTMC_ERR_INVALID_ARG if a
   node would need a quantum above 2^40 (coordinates beyond about 2^47).
   Every kind also gets a column grid for rays parallel to z (generation 0 at
   normal incidence): about n_tri / 5 pixels over [0, lx) x [0, ly), each
   listing the facets whose xy box meets it, sorted by top z (descending, then
   index).  Such a ray tests its pixel's facets in that order and stops when
   no facet further down the list can be closer than its best hit; the facet
   tests are the hierarchy's, so every hit record is the same.  A facet over
   more than 64 pixels makes the build retry with a quarter of the pixels (up
   to four times); a mesh the grid still does not suit (a pixel with more than
   2048 facets, more than 2^24 facets, or no device memory for it) gets none. */
int rtmc_build_bvh(rtmc_ctx* ctx, int32_t mesh_id, int32_t bvh_kind);

/* Run RTMC for every (energy, angle) pair: n_e * n_theta items, item
   ie * n_theta + it.  Each item traces n_primaries primaries with seed `seed`
   (Philox4x32-10 streams keyed by seed and indexed by primary id, ray path and
   item).  Writes out[n_e * n_theta] and, when non-NULL, hist_e[item][n_ebins]
   and hist_a[item][n_abins] (host memory); with desc->n_zbins > 0 also
   desc->hist_z[item][n_zbins], the penetration profile of Section 3.2: the
   depth z_top - z of every point where a ray's flight ends on a facet (any
   generation, re-emitting or absorbed), in n_zbins equal bins over
   [0, z_top - z_min], clamped.  desc may be NULL (defaults). */
int rtmc_run(rtmc_ctx* ctx, int32_t mesh_id, const double* energies_ev, int32_t n_e,
             const double* theta_deg, int32_t n_theta, int64_t n_primaries, uint64_t seed,
             const rtmc_run_desc* desc, rtmc_result* out, uint64_t* hist_e, uint64_t* hist_a);

/* Batched form: every (mesh, energy, angle) combination of the batch as one
   item, item = (m * n_e + ie) * n_theta + it (plus desc->item_base), each with
   n_primaries primaries.  The rays of all items of a mesh share the wavefront
   queues (a chunk spans items), and the whole launch sequence over all meshes
   is captured once into a CUDA graph and replayed on later calls with the same
   batch shape (desc->no_graph = 1 launches eagerly instead).  Item k uses the
   same random streams as rtmc_run with item_base = k, so its tallies are
   identical to that run's.  Every generation the loaded emission allows
   (max_generation <= 6) is traced, one traversal and one shade launch per
   generation and chunk; a generation with no rays ends its launches at once.
   With desc->chunk = 0 a chunk is the largest power of two up to 2^26
   primaries whose queues take at most a quarter of the free device memory
   (the queues the context already holds counted as free), and at most 15
   items' worth of primaries.
   Queues are sized as in rtmc_run (desc->queue_factor); if a chunk overflows,
   the whole batch is recorded again with twice the capacity and run again
   (up to six times; queue_retries counts the repeats).  Writes
   out[n_items]; hist_e / hist_a / desc->hist_z as in rtmc_run, with
   n_ebins + n_abins + n_zbins <= 512.  gpu_ms of every result is
   the device time of the whole batch, and node_visits / tri_tests / retested
   are batch totals (the traversal does not tell items apart); launches counts
   the batch's kernels; with no_graph and profile the ms_* fields hold the
   batch's per-kernel totals. */
typedef struct {
    const int32_t* mesh_ids;
    int32_t n_meshes;
    const double* energies_ev;
    int32_t n_e;
    const double* theta_deg;
    int32_t n_theta;
    int64_t n_primaries;           /* per item */
    uint64_t seed;
} rtmc_batch;
int rtmc_run_batch(rtmc_ctx* ctx, const rtmc_batch* batch, const rtmc_run_desc* desc,
                   rtmc_result* out, uint64_t* hist_e, uint64_t* hist_a);

/* As rtmc_run for one (energy, angle) item with index `item`, also writing one
   record per traced ray (any order) into rec[rec_cap] (host memory); *n_rec
   receives the count.  Fails with RTMC_ERR_CAPACITY when rec_cap is too small. */
int rtmc_run_records(rtmc_ctx* ctx, int32_t mesh_id, double energy_ev, double theta_deg,
                     uint32_t item, int64_t n_primaries, uint64_t seed,
                     const rtmc_run_desc* desc, rtmc_result* out, rtmc_record* rec,
                     int64_t rec_cap, int64_t* n_rec);

/* Closest front-facing hit of n rays in the cell (no periodic walk) through
   the BVH: origins o[n][3], directions d[n][3] (FP32), origin triangle ids
   to skip (original ids, -1 = none, may be NULL).  hits[n] gets t, the
   barycentrics (u, v) of V1 and V2, and the original triangle id (-1 on a
   miss).  Section 2.1. */
int rtmc_trace_rays(rtmc_ctx* ctx, int32_t mesh_id, const float* o, const float* d,
                    const int32_t* skip_tri, int64_t n, rtmc_hit* hits);

/* Copy a built BVH to host memory for inspection: which = 0 FP32 nodes
   (n_nodes x 64 B; every child box widened outward by M 2^-22, M the
   largest coordinate of the cell, so that a ray with a zero direction
   component lying in a face plane of the exact box is still inside it),
   1 Q8 nodes (n_nodes x 32 B, RTMC_BVH_Q8 meshes only; the widened boxes,
   quantised outward),
   2 triangles in leaf order (n_tri x 48 B), 3 4-wide nodes (RTMC_BVH_W4
   meshes only, n_w4 x 128 B: rows lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of the
   four child boxes, each widened outward by M 2^-22 with M the largest
   coordinate of the cell, then the four child refs; an empty slot has ref
   INT_MIN and the box [+inf, +inf]^3), 4 quantised 4-wide nodes
   (RTMC_BVH_Q4 meshes only, n_w4 x 64 B: floats o'.x, o'.y, o'.z, S.x | S.y,
   S.z, then six words lo.x, hi.x, lo.y, hi.y, lo.z, hi.z whose byte c is
   child c's code q, then the four child refs; S = 2^15 s with s the quantum,
   a plane is o' + (1 + q 2^-15) S, an empty slot has codes lo 255, hi 0 and
   ref INT_MIN).  Layouts as in the library's
   device code; a Q8 node holds per axis a shifted origin o' (float) and a
   biased exponent byte b (scale s = 2^(b - 127)), and child bound q decodes
   as fmaf(2^23 + q, s, o') in FP32.  With out == NULL only *bytes_needed is written; otherwise
   bytes must be at least that size. */
int rtmc_export_bvh(rtmc_ctx* ctx, int32_t mesh_id, int32_t which, void* out, int64_t bytes,
                    int64_t* bytes_needed);

/* Read-bandwidth probe used as a roofline denominator: `iters` launches of a
   kernel that streams `bytes` (a context-owned buffer, zero-filled) with
   128-bit loads from every SM, repeating the pass so that each launch reads
   at least 2 GiB; *gbs receives bytes read / device time.  32 MiB stays in
   L2 after the first pass; a few GiB measures HBM. */
int rtmc_probe_bandwidth(rtmc_ctx* ctx, int64_t bytes, int32_t iters, double* gbs);

/* Philox4x32-10 on the device: out[i][4] = philox(ctr[i][4], key), for
   checking the device generator against the published vectors. */
int rtmc_philox(rtmc_ctx* ctx, const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out);

/* Scratch-free run of one (energy, angle) item.  The paper has no
   counterpart: this entry point serves callers that must not allocate device
   memory while they run, for example a process whose allocator reserved the
   whole device up front so that nothing can fail for lack of memory later, or
   a latency-bound loop that cannot afford cudaMalloc/cudaFree, which may
   synchronise the device and stall other streams.  It computes what rtmc_run
   computes for one item (same kernels, same random streams, same outputs)
   but allocates nothing: it calls no cudaMalloc, cudaFree or allocating
   library routine.  Its scratch (ray queues, hits, counters, histograms,
   about 4.5 MiB) is one static device array compiled into librtmc, which
   every GPU that loads the library keeps until the process exits.  The mesh,
   BVH and tables still come from the context (loaded beforehand).
   Limits, rejected with RTMC_ERR_INVALID_ARG and a message:
     n_primaries <= RTMC_NOALLOC_MAX_PRIMARIES per call (advance
       desc->primary_offset and call again for more primaries);
     the loaded emission parameters must have max_generation == 1;
     n_ebins + n_abins + n_zbins <= 1024.
   desc is checked as rtmc_run checks it.  desc->profile, desc->chunk and
   desc->queue_factor are ignored (the static queues hold k_max daughters per
   primary); desc->prim_hash (device, n_primaries entries), desc->count_visits,
   desc->fp64_retest (it runs inside the traversal kernel and needs no
   scratch) and the traversal controls (traversal, stack_depth,
   fetch_threshold, block_threads, blocks_per_sm, max_visits) work as in
   rtmc_run.
   The first call in a context looks up the array's device address
   (cudaGetSymbolAddress) with the context's device current and keeps it in
   the context; make that first call before any stream capture.  A device
   reset ends the context's use, as for every other entry point: destroy the
   context and create a new one.  Every call on a device uses the same array and
   clears the counters it needs before it starts; calls whose GPU work
   overlaps (other host threads, other contexts or streams on the same
   device) race on the array and must be serialised by the caller.
   Writes *out and, when non-NULL, hist_e[n_ebins] / hist_a[n_abins] (host),
   and desc->hist_z[n_zbins] when n_zbins > 0. */
#define RTMC_NOALLOC_MAX_PRIMARIES 4096
int rtmc_run_noalloc(rtmc_ctx* ctx, int32_t mesh_id, double energy_ev, double theta_deg,
                     uint32_t item, int64_t n_primaries, uint64_t seed,
                     const rtmc_run_desc* desc, rtmc_result* out, uint64_t* hist_e,
                     uint64_t* hist_a);

/* Hash of one record (the per-primary hash is the sum mod 2^64 of the hashes
   of that primary's records): h = sm(prim); h = sm(h ^ (path | fate << 32));
   h = sm(h ^ (uint32 tri | uint32 k << 32)); h = sm(h ^ (uint32 e_bin |
   uint32 a_bin << 32)); h = sm(h ^ uint32 wraps), sm = splitmix64. */
uint64_t rtmc_record_hash(const rtmc_record* r);

#ifdef __cplusplus
}
#endif
#endif
