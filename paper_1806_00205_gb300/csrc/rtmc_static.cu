// rtmc_static.cu -- rtmc_run_noalloc: one (energy, angle) item whose scratch
// lives in a static device array, for callers that must not allocate device
// memory.  It launches the same kernels as rtmc_run.
//
// Layout of the static array (each part 256-byte aligned):
//   queue 0  (oe, dt, id)        3 x 16 B x kMaxPrim
//   queue 1  (oe, dt, id)        3 x 16 B x kMaxPrim x 15
//   hits                         16 B x kMaxPrim x 15
//   wraps                        4 B x kMaxPrim x 15   (per-primary hashing)
//   per-primary escape counts    4 B x kMaxPrim
//   Control, Tally, histograms   (n_ebins + n_abins + n_zbins <= kMaxBins) x 8 B
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>

#include "rtmc_internal.h"

namespace {

constexpr int64_t kMaxPrim = RTMC_NOALLOC_MAX_PRIMARIES;
constexpr int64_t kMaxDaughters = kMaxPrim * 15;     // k_max <= 15, one generation of daughters
constexpr int kMaxBins = 1024;

constexpr size_t al(size_t x) { return (x + 255) & ~(size_t)255; }
constexpr size_t kQ0 = 0;
constexpr size_t kQ1 = kQ0 + 3 * al(16 * kMaxPrim);
constexpr size_t kHits = kQ1 + 3 * al(16 * kMaxDaughters);
constexpr size_t kWraps = kHits + al(16 * kMaxDaughters);
constexpr size_t kKcount = kWraps + al(4 * kMaxDaughters);
constexpr size_t kCtl = kKcount + al(4 * kMaxPrim);
constexpr size_t kTally = kCtl + al(sizeof(rtmc::Control));
constexpr size_t kHist = kTally + al(sizeof(rtmc::Tally));
constexpr size_t kBytes = kHist + al(8 * kMaxBins);

// The scratch: one copy per device that loads the library, held until exit.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kBytes];

// Device address of the static array, looked up with the context's device
// current on the context's first call and kept in the context: a device reset
// ends the context's other device state too, so the cache never outlives the
// module load it came from while the context is usable.
cudaError_t scratch_address(rtmc_ctx* ctx, void** out)
{
    if (!ctx->noalloc_scratch) {
        void* p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        ctx->noalloc_scratch = p;
    }
    *out = ctx->noalloc_scratch;
    return cudaSuccess;
}

struct CurrentDevice {
    int prev = -1;
    explicit CurrentDevice(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~CurrentDevice()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

double spectrum_cdf(double e, double phi)
{
    const double s = phi / (e + phi);
    return 1.0 - 3.0 * s * s + 2.0 * s * s * s;
}

}  // namespace

extern "C" int rtmc_run_noalloc(rtmc_ctx* ctx, int32_t mesh_id, double energy_ev, double theta_deg, uint32_t item,
                                int64_t n_primaries, uint64_t seed, const rtmc_run_desc* desc, rtmc_result* out,
                                uint64_t* hist_e, uint64_t* hist_a)
{
    using namespace rtmc;
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (mesh_id < 0 || mesh_id >= (int)ctx->meshes.size() || !ctx->meshes[mesh_id].tri_in)
        return ctx->fail(RTMC_ERR_NOT_LOADED, "run_noalloc: unknown mesh id");
    if (!ctx->meshes[mesh_id].built) return ctx->fail(RTMC_ERR_NOT_BUILT, "run_noalloc: build_bvh first");
    if (!ctx->table_loaded) return ctx->fail(RTMC_ERR_NOT_LOADED, "run_noalloc: load_see_tables first");
    if (!out || !(energy_ev > 0.0) || !(theta_deg >= 0.0 && theta_deg < 90.0))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run_noalloc: bad arguments");
    if (n_primaries < 0 || n_primaries > kMaxPrim)
        return ctx->fail(RTMC_ERR_INVALID_ARG,
                         "run_noalloc: n_primaries must be in [0, 4096] (the static scratch holds 4096 primaries "
                         "per call; advance primary_offset and call again for more)");
    if (ctx->emission.max_generation != 1)
        return ctx->fail(RTMC_ERR_INVALID_ARG,
                         "run_noalloc: only max_generation == 1 fits the static scratch (one generation of daughters)");
    rtmc_run_desc d;
    std::memset(&d, 0, sizeof d);
    if (desc) {
        d = *desc;
    } else {
        d.n_ebins = 64;
        d.n_abins = 18;
        d.hist_e_max_ev = 50.0;
    }
    const int vrc = check_run_desc(ctx, d);     // the descriptor contract of rtmc_run
    if (vrc) return vrc;
    if (d.n_ebins + d.n_abins + d.n_zbins > kMaxBins)
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run_noalloc: histogram bins must satisfy n_ebins + n_abins + n_zbins <= 1024");

    CurrentDevice guard(ctx->device);
    void* base_v = nullptr;
    cudaError_t ce = scratch_address(ctx, &base_v);
    if (ce != cudaSuccess)
        return ctx->fail(RTMC_ERR_CUDA, std::string("run_noalloc: cudaGetSymbolAddress: ") + cudaGetErrorString(ce));
    char* base = static_cast<char*>(base_v);
    const DeviceMesh& m = ctx->meshes[mesh_id];
    const rtmc_emission& em = ctx->emission;
    cudaStream_t s = ctx->stream;
    const double kPi = 3.14159265358979323846;

    RunParams p;
    p.seed = seed;
    p.item = item;
    p.energy = (float)energy_ev;
    p.sin_t = (float)std::sin(theta_deg * kPi / 180.0);
    p.cos_t = (float)std::cos(theta_deg * kPi / 180.0);
    p.random_azimuth = d.random_azimuth;
    p.random_polar = d.random_polar;
    const bool full = d.src_x0 == 0.0 && d.src_x1 == 0.0 && d.src_y0 == 0.0 && d.src_y1 == 0.0;
    p.src_x0 = full ? 0.f : (float)d.src_x0;
    p.src_x1 = full ? (float)m.box.lx : (float)d.src_x1;
    p.src_y0 = full ? 0.f : (float)d.src_y0;
    p.src_y1 = full ? (float)m.box.ly : (float)d.src_y1;
    p.lx = (float)m.box.lx;
    p.ly = (float)m.box.ly;
    p.z_min = (float)m.box.z_min;
    p.z_top = (float)m.box.z_top;
    p.max_wraps = d.max_wraps > 0 ? d.max_wraps : 1024;
    p.n_ebins = d.n_ebins;
    p.n_abins = d.n_abins;
    p.ebin_w = (float)(d.hist_e_max_ev / d.n_ebins);
    p.inv_abin = (float)(d.n_abins / (0.5 * kPi));
    p.n_zbins = d.n_zbins;
    p.inv_zbin = (float)(d.n_zbins / (m.box.z_top - m.box.z_min));
    p.prim_offset = d.primary_offset;

    TableDesc tab;
    tab.delta = ctx->delta;
    tab.n_e = ctx->grid.n_e;
    tab.n_theta = ctx->grid.n_theta;
    tab.inv_log_span = (float)((ctx->grid.n_e - 1) / std::log(ctx->grid.e_hi_ev / ctx->grid.e_lo_ev));
    tab.log_e_lo = (float)std::log(ctx->grid.e_lo_ev);
    tab.inv_theta_step_deg = (float)(1.0 / ctx->grid.theta_step_deg);

    Emission e;
    e.phi = (float)em.phi_ev;
    e.e_cut = (float)em.e_cut_ev;
    e.absorb_min = (float)em.absorb_min_ev;
    e.regen_min = std::isinf(em.regen_min_ev) ? INFINITY : (float)em.regen_min_ev;
    e.max_generation = em.max_generation;
    e.k_max = em.k_max;
    e.spec_norm = (float)spectrum_cdf(em.e_cut_ev, em.phi_ev);
    e.model = em.model;

    Queues q;
    for (int b = 0; b < 2; ++b) {
        const size_t qb = b ? kQ1 : kQ0;
        const size_t len = b ? al(16 * kMaxDaughters) : al(16 * kMaxPrim);
        q.oe[b] = reinterpret_cast<float4*>(base + qb);
        q.dt[b] = reinterpret_cast<float4*>(base + qb + len);
        q.id[b] = reinterpret_cast<uint4*>(base + qb + 2 * len);
    }
    q.cap[0] = (unsigned)kMaxPrim;
    q.cap[1] = (unsigned)kMaxDaughters;
    q.hits = reinterpret_cast<float4*>(base + kHits);
    const bool hashing = d.prim_hash != nullptr;
    q.wraps = hashing ? reinterpret_cast<int*>(base + kWraps) : nullptr;
    q.kcount = reinterpret_cast<unsigned*>(base + kKcount);
    q.sort_counts = nullptr;   // primaries stay in id order here (no sort scratch)
    q.ctl = reinterpret_cast<Control*>(base + kCtl);
    q.tally = reinterpret_cast<Tally*>(base + kTally);
    q.hist_e = reinterpret_cast<unsigned long long*>(base + kHist);
    q.hist_a = q.hist_e + d.n_ebins;
    q.prim_hash = reinterpret_cast<unsigned long long*>(d.prim_hash);
    q.records = nullptr;
    q.rec_cap = 0;

    const Tuning tune = tuning_from(d);

    // The array keeps the previous call's contents: clear everything that must start at zero.
    ce = cudaMemsetAsync(base + kCtl, 0, sizeof(Control), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(base + kTally, 0, sizeof(Tally), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(base + kHist, 0, 8 * (size_t)(d.n_ebins + d.n_abins + d.n_zbins), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(base + kKcount, 0, 4 * (size_t)kMaxPrim, s);
    if (ce == cudaSuccess && hashing) ce = cudaMemsetAsync(d.prim_hash, 0, 8 * (size_t)n_primaries, s);
    const unsigned n = (unsigned)n_primaries;
    if (ce == cudaSuccess) ce = launch_generate(p, q, 0, 0ull, n, s);
    const bool columns = m.col_ok && d.traversal == 0 && theta_deg == 0.0 && !d.random_polar;
    for (int g = 0; g <= 1 && ce == cudaSuccess; ++g) {
        ce = columns && g == 0
                 ? launch_columns(m, p, q, g, g, ctx->num_sms, hashing, d.fp64_retest != 0, s)
                 : launch_traverse(m, p, q, g, g, ctx->num_sms, tune, hashing, d.count_visits != 0,
                                   d.fp64_retest != 0, s);
        if (ce == cudaSuccess) ce = launch_shade(m, p, tab, e, q, g, g, 0ull, ctx->num_sms, false, s);
    }
    if (ce == cudaSuccess) ce = launch_finalize(q, n, s);
    Tally t;
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(&t, base + kTally, sizeof t, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess && hist_e)
        ce = cudaMemcpyAsync(hist_e, base + kHist, 8 * (size_t)d.n_ebins, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess && hist_a)
        ce = cudaMemcpyAsync(hist_a, base + kHist + 8 * (size_t)d.n_ebins, 8 * (size_t)d.n_abins,
                             cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess && d.n_zbins > 0)
        ce = cudaMemcpyAsync(d.hist_z, base + kHist + 8 * (size_t)(d.n_ebins + d.n_abins), 8 * (size_t)d.n_zbins,
                             cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) return ctx->fail(RTMC_ERR_CUDA, std::string("run_noalloc: ") + cudaGetErrorString(ce));
    if (t.status & ST_QUEUE_OVERFLOW) return ctx->fail(RTMC_ERR_CAPACITY, "run_noalloc: daughter queue overflow");
    if (t.status & (ST_STACK_OVERFLOW | ST_LOOP_LIMIT | ST_COLUMN))
        return ctx->fail(RTMC_ERR_DEVICE_CHECK, "run_noalloc: traversal stack overflow or iteration bound");

    rtmc_result& r = *out;
    std::memset(&r, 0, sizeof r);
    r.n_primaries = n_primaries;
    r.rays = (int64_t)t.rays;
    r.escaped = (int64_t)t.escaped;
    r.absorbed_low = (int64_t)t.absorbed_low;
    r.absorbed_other = (int64_t)t.absorbed_other;
    r.emitters = (int64_t)t.emitters;
    r.emitted = (int64_t)t.emitted;
    r.regenerated = (int64_t)t.regenerated;
    r.capped = (int64_t)t.capped;
    r.lost = (int64_t)t.lost;
    r.wraps = (int64_t)t.wraps;
    r.sum_k = (int64_t)t.sum_k;
    r.sum_k2 = (int64_t)t.sum_k2;
    r.e_sum = t.e_sum;
    r.e2_sum = t.e2_sum;
    r.node_visits = (int64_t)t.node_visits;
    r.tri_tests = (int64_t)t.tri_tests;
    r.retested = (int64_t)t.retested;
    r.column_rays = (int64_t)t.col_rays;
    r.launches = 6;
    r.traverse_launches = columns ? 1 : 2;
    if (n_primaries > 0) r.sey = (double)r.sum_k / (double)n_primaries;
    if (n_primaries > 1) {
        const double var = ((double)r.sum_k2 / (double)n_primaries - r.sey * r.sey) / (double)(n_primaries - 1);
        r.sey_se = var > 0.0 ? std::sqrt(var) : 0.0;
    }
    return RTMC_OK;
}
