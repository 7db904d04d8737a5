// rtmc_internal.h -- host-side state shared by the translation units of librtmc.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/rtmc.h"
#include "rtmc_device.cuh"

namespace rtmc {

// A slanted column grid (rays of one fixed oblique direction, see GridDev),
// built on first use by a run at that incidence and kept with the mesh.
struct SlantGrid {
    float dx = 0.f, dz = -1.f;     // the FP32 direction it serves (d.y = 0)
    int gx = 0, gy = 0;
    float iwx = 0.f, iwy = 0.f;
    unsigned* off = nullptr;
    uint2* ent = nullptr;
    int64_t entries = 0;
};

struct DeviceMesh {
    int64_t n_tri = 0;
    rtmc_box box{};
    float* tri_in = nullptr;       // n_tri * 9, original order
    bool built = false;
    int kind = RTMC_BVH_FP32;
    int64_t n_nodes = 0;
    float4* nodes = nullptr;       // n_nodes * 4 float4 (64 B each)
    float4* tris = nullptr;        // n_tri * 3 float4, BVH leaf order
    float4* normals = nullptr;     // n_tri float4
    int* inv_order = nullptr;      // original id -> leaf-order index
    void* q8 = nullptr;            // n_nodes * 32 B quantised nodes (RTMC_BVH_Q8)
    void* w4 = nullptr;            // n_w4 * 128 B 4-wide nodes (RTMC_BVH_W4, RTMC_BVH_Q4)
    void* q4 = nullptr;            // n_w4 * 64 B quantised 4-wide nodes (RTMC_BVH_Q4)
    int64_t n_w4 = 0;
    int depth_w4 = 0;              // levels of the 4-wide hierarchy
    int depth = 0;                 // hierarchy depth (root = 1)
    int leaf_max = 4;              // triangles per leaf (1..8)
    bool ploc = false;             // hierarchy from locally-ordered clustering
    double build_ms = 0.0;
    // Column grid for rays parallel to z (generation 0 at normal incidence),
    // col_gx x col_gy pixels over [0, lx) x [0, ly); pixel p lists the facets
    // whose xy box (widened by col_margin) meets it, as (leaf-order index, top z
    // bits) pairs col_ent[col_off[p] .. col_off[p + 1]) sorted by top z
    // descending, then index ascending.
    bool col_ok = false;
    int col_gx = 0, col_gy = 0;
    float col_inv_wx = 0.f, col_inv_wy = 0.f;
    unsigned* col_off = nullptr;   // col_gx * col_gy + 1
    uint2* col_ent = nullptr;
    int64_t col_entries = 0;
    std::vector<SlantGrid> slant;  // slanted grids built so far (freed with the column grid)
    size_t slant_bytes = 0;
    std::vector<float2> slant_failed;   // directions whose grid could not be built (not retried)
};

// Growable device scratch owned by the context.
struct Scratch {
    void* ptr = nullptr;
    size_t bytes = 0;
};

struct Tuning {
    int block_threads = 64;
    int blocks_per_sm = 0;         // 0: from occupancy
    int traversal = 0;             // 0/2: while-while with ray refill, 1: one ray per lane per tile
    int stack_depth = 16;          // shared-memory stack entries per ray (8, 16, 32)
    int fetch_threshold = 0;       // refill when fewer lanes are active (0: default 28)
    int max_visits = 0;            // lower bound on inner-node visits per cell traversal (0: the tree's own)
};

// Tuning of a run from its descriptor (the controls rtmc_run honours).
inline Tuning tuning_from(const rtmc_run_desc& d)
{
    Tuning t;
    if (d.block_threads > 0) t.block_threads = d.block_threads;
    t.blocks_per_sm = d.blocks_per_sm;
    t.traversal = d.traversal;
    if (d.stack_depth > 0) t.stack_depth = d.stack_depth;
    t.fetch_threshold = d.fetch_threshold;
    t.max_visits = d.max_visits;
    return t;
}

// Daughter-queue capacities per primary of a chunk, for the buffer of even
// generations (index 0, generation 0 included) and of odd ones (index 1).
// First attempt: from the largest expected yield y of the loaded emission at
// energies up to e_max_ev, a margin of two over the expectation per generation
// (generation g of a tree holds at most about y^g rays per primary, and for
// chunks of thousands of primaries the count stays far below twice that),
// capped at k_max for generation 1 and 16 beyond; desc.queue_factor > 0
// replaces the odd buffer's factor (test hook).  A chunk that still overflows sets ST_QUEUE_OVERFLOW and
// is run again with both factors doubled.
struct QueueFactors {
    double f[2] = {1.0, 1.0};
};
QueueFactors queue_factors(const rtmc_ctx* ctx, const rtmc_run_desc& d, double e_max_ev);
// Default primaries per chunk: the largest power of two up to 2^26 whose queues
// (capacities f[0], f[1] per primary) take at most a quarter of the device memory
// not held by other buffers; the queues the context already holds count as free,
// so the choice is the same from call to call.
int64_t default_chunk(const rtmc_ctx* ctx, const QueueFactors& qf);

}  // namespace rtmc

struct rtmc_ctx {
    int device = 0;
    int num_sms = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    std::vector<rtmc::DeviceMesh> meshes;
    float* delta = nullptr;
    rtmc_grid grid{};
    rtmc_emission emission{};
    bool table_loaded = false;
    // run buffers
    rtmc::Scratch q_oe[2], q_dt[2], q_id[2], hits, kcount, ctl, tally, hist, wraps, records, tmp;
    rtmc::Scratch items;                      // batched item table
    rtmc::Scratch sort_counts;                // spatial sort of primaries
    rtmc::Scratch grids;                      // column-grid descriptors of the items (GridDev)
    cudaGraphExec_t batch_graph = nullptr;    // captured batch launch sequence
    std::string batch_key;                    // what the captured graph was built for
    int64_t batch_launches = 0;               // kernel launches in the captured graph
    void* noalloc_scratch = nullptr;          // device address of rtmc_run_noalloc's static array
    double yield_max = 1.0;                   // largest expected daughter count per emission (loaded emission)
    std::string err;
    int fail(int code, const std::string& msg) { err = msg; return code; }
};

namespace rtmc {

struct RunParams;
RunParams make_params(const DeviceMesh& m, const rtmc_run_desc& d, uint64_t seed, unsigned item, double energy,
                      double theta_deg);
TableDesc make_table(const rtmc_ctx* ctx);
Emission make_emission(const rtmc_emission& em);
void fill_result(rtmc_result& r, const Tally& t, int64_t n_prim);
int check_run_desc(rtmc_ctx* ctx, const rtmc_run_desc& d);

// Ensure a scratch buffer holds at least `bytes`; returns cudaSuccess or the error.
cudaError_t scratch_reserve(Scratch& s, size_t bytes);
void scratch_free(Scratch& s);

// LBVH build (rtmc_bvh.cu).
int build_lbvh(rtmc_ctx* ctx, DeviceMesh& m);

// Device-wide exclusive scan of 32-bit counts: out[i] = in[0] + ... + in[i-1]
// (in == out allowed), *total (device, optional) = the sum of all n.  part:
// device scratch of scan_parts(n) words.  Three launches on s.
long long scan_parts(long long n);
void scan_exclusive(const unsigned* in, unsigned* out, long long n, unsigned* total, unsigned* part, cudaStream_t s);

// Wavefront launchers (rtmc_trace.cu).
struct RunParams {
    unsigned long long seed = 0;
    unsigned item = 0;
    float energy = 0.f;
    int random_azimuth = 0;
    int random_polar = 0;        // 1: cosine-law polar angle of incidence (second Philox block, path 0)
    float src_x0 = 0.f, src_x1 = 0.f, src_y0 = 0.f, src_y1 = 0.f;
    float lx = 0.f, ly = 0.f, z_min = 0.f, z_top = 0.f;
    int max_wraps = 1024;
    int n_ebins = 0, n_abins = 0;
    int n_zbins = 0;             // penetration-depth bins over [0, z_top - z_min] below z_top
    float ebin_w = 1.f;          // eV per energy bin
    float inv_abin = 0.f;        // bins per radian of polar angle
    float inv_zbin = 0.f;        // bins per nm of depth
    unsigned long long prim_offset = 0;
    float sin_t = 0.f, cos_t = 1.f;   // incidence (single-item runs): the FP64 angle's sine and cosine, rounded once
};

struct Queues {
    float4* oe[2];
    float4* dt[2];
    uint4* id[2];
    float4* hits;
    int* wraps;                  // record mode only
    unsigned* kcount;
    unsigned* sort_counts;       // spatial sort of primaries: per-bucket counts / cursors
    Control* ctl;
    Tally* tally;
    unsigned long long* hist_e;  // device, n_ebins
    unsigned long long* hist_a;  // device, n_abins
    unsigned long long* prim_hash;  // optional
    rtmc_record* records;        // optional (device)
    unsigned long long rec_cap;
    unsigned cap[2];
};

cudaError_t launch_generate(const RunParams& p, const Queues& q, int buf, unsigned long long first,
                            unsigned n, cudaStream_t s);
cudaError_t launch_traverse(const DeviceMesh& m, const RunParams& p, const Queues& q, int buf,
                            int gen, int num_sms, const Tuning& tune, bool record, bool count,
                            bool retest, cudaStream_t s);
cudaError_t launch_shade(const DeviceMesh& m, const RunParams& p, const TableDesc& tab,
                         const Emission& em, const Queues& q, int buf, int gen,
                         unsigned long long chunk_first, int num_sms, bool record, cudaStream_t s);
cudaError_t launch_finalize(const Queues& q, unsigned n, cudaStream_t s);
cudaError_t launch_generate_items(const RunParams& p, const ItemCtx& ic, const Queues& q, unsigned n,
                                  cudaStream_t s);
// Spatially sorted primaries (Morton-ordered 512 x 512 entry cells; per item in
// multi-item chunks, at most kChunkItems items).  The sort scratch holds the
// counts of up to `items` items followed by the scan's tile sums.
constexpr unsigned kSortBucketsPerItem = 1u << 18;
inline size_t sort_scratch_bytes(unsigned items)
{
    const long long b = (long long)items * kSortBucketsPerItem;
    return (size_t)(b + scan_parts(b)) * 4;
}
cudaError_t launch_generate_sorted(const RunParams& p, const Queues& q, unsigned long long first, unsigned n,
                                   cudaStream_t s);
cudaError_t launch_generate_items_sorted(const RunParams& p, const ItemCtx& ic, const Queues& q, unsigned n,
                                         cudaStream_t s);
cudaError_t launch_shade_items(const DeviceMesh& m, const RunParams& p, const TableDesc& tab, const Emission& em,
                               const ItemCtx& ic, const Queues& q, int buf, int gen, int num_sms, cudaStream_t s);
cudaError_t launch_finalize_items(const ItemCtx& ic, const Queues& q, unsigned n, int num_sms, cudaStream_t s);
// Generation `gen` of rays parallel to z (all of them) through the column grid
// instead of the hierarchy: the same facet tests, so the same hit records.
cudaError_t launch_columns(const DeviceMesh& m, const RunParams& p, const Queues& q, int buf, int gen,
                           int num_sms, bool record, bool retest, cudaStream_t s);
int build_columns(rtmc_ctx* ctx, DeviceMesh& m);
void free_columns(DeviceMesh& m);
// The slanted grid for primaries of direction (dx, 0, dz), dx > 0 > dz, built on
// first use (synchronises the context's stream; never call it inside a stream
// capture); its descriptor goes to `out`.  false when the mesh has none and
// cannot get one: no column grid, too many facets, a footprint too wide even
// for coarse pixels, more than 255 wraps before a facet, or the slanted grids'
// memory cap -- such rays take the hierarchy.
bool slant_grid(rtmc_ctx* ctx, DeviceMesh& m, float dx, float dz, GridDev& out);
GridDev grid_dev(const DeviceMesh& m, const SlantGrid* g);   // g == nullptr: the vertical grid
// Generation `gen` of primaries of fixed directions (one per item when `items`)
// through their grids (device array; entry 0, or one per item of the mesh).
cudaError_t launch_slant(const DeviceMesh& m, const RunParams& p, const GridDev* grids, bool items, const Queues& q,
                         int buf, int gen, int num_sms, bool record, cudaStream_t s);
cudaError_t launch_trace_rays(const DeviceMesh& m, const float* o, const float* d, const int* skip,
                              int64_t n, rtmc_hit* hits, unsigned* status, cudaStream_t s);
cudaError_t launch_read_probe(const void* buf, size_t bytes, int passes, int num_sms, float* sink, cudaStream_t s);
cudaError_t launch_philox(const uint32_t* ctr, int64_t n, unsigned long long key, uint32_t* out,
                          cudaStream_t s);

}  // namespace rtmc
