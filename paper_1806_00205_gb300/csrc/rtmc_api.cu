// rtmc_api.cu -- the C ABI of librtmc: contexts, mesh and table upload, BVH
// build, and the host orchestration of the wavefront RTMC loop.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "rtmc_internal.h"

using rtmc::DeviceMesh;

namespace rtmc {

cudaError_t scratch_reserve(Scratch& s, size_t bytes)
{
    if (bytes <= s.bytes && s.ptr) return cudaSuccess;
    if (s.ptr) { cudaFree(s.ptr); s.ptr = nullptr; s.bytes = 0; }
    bytes = std::max<size_t>(bytes, 256);
    cudaError_t e = cudaMalloc(&s.ptr, bytes);
    if (e == cudaSuccess) s.bytes = bytes;
    return e;
}

void scratch_free(Scratch& s)
{
    if (s.ptr) cudaFree(s.ptr);
    s.ptr = nullptr;
    s.bytes = 0;
}

}  // namespace rtmc

namespace {

constexpr double kPi = 3.14159265358979323846;

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev)
    {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard()
    {
        int cur = -1;
        cudaGetDevice(&cur);
        if (prev >= 0 && cur != prev) cudaSetDevice(prev);
    }
};

int cuda_fail(rtmc_ctx* ctx, cudaError_t e, const char* where)
{
    return ctx->fail(RTMC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

rtmc_run_desc default_desc()
{
    rtmc_run_desc d;
    std::memset(&d, 0, sizeof d);
    d.n_ebins = 64;
    d.n_abins = 18;
    d.hist_e_max_ev = 50.0;
    return d;
}

}  // namespace

namespace rtmc {

RunParams make_params(const DeviceMesh& m, const rtmc_run_desc& d, uint64_t seed, unsigned item, double energy,
                      double theta_deg)
{
    RunParams p;
    p.seed = seed;
    p.item = item;
    p.energy = (float)energy;
    // the FP32 direction nearest the exact one: sin and cos of the FP64 angle, rounded once
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
    return p;
}

TableDesc make_table(const rtmc_ctx* ctx)
{
    TableDesc tab;
    tab.delta = ctx->delta;
    tab.n_e = ctx->grid.n_e;
    tab.n_theta = ctx->grid.n_theta;
    tab.inv_log_span = (float)((ctx->grid.n_e - 1) / std::log(ctx->grid.e_hi_ev / ctx->grid.e_lo_ev));
    tab.log_e_lo = (float)std::log(ctx->grid.e_lo_ev);
    tab.inv_theta_step_deg = (float)(1.0 / ctx->grid.theta_step_deg);
    return tab;
}

Emission make_emission(const rtmc_emission& em)
{
    Emission e;
    e.phi = (float)em.phi_ev;
    e.e_cut = (float)em.e_cut_ev;
    e.absorb_min = (float)em.absorb_min_ev;
    e.regen_min = std::isinf(em.regen_min_ev) ? INFINITY : (float)em.regen_min_ev;
    e.max_generation = em.max_generation;
    e.k_max = em.k_max;
    e.model = em.model;
    const double sn = em.phi_ev / (em.e_cut_ev + em.phi_ev);
    e.spec_norm = (float)(1.0 - 3.0 * sn * sn + 2.0 * sn * sn * sn);
    return e;
}

// Eq. 6 (Section 2.2) on the host, alpha in degrees: only to size queues.
static double paper_yield(double e, double a)
{
    return 3.05 + 1.7949e-5 * a * a + 6.15e-7 * e * e - (371.317 - std::exp(0.04826 * a)) / (87.602 + e) -
           1.974e-3 * e - 0.1097 * std::cos(0.1201 + 2.469 * a);
}

QueueFactors queue_factors(const rtmc_ctx* ctx, const rtmc_run_desc& d, double e_max_ev)
{
    const rtmc_emission& em = ctx->emission;
    double y = ctx->yield_max;
    if (em.model == RTMC_EMISSION_PAPER_FIT) {        // daughters never exceed the primary energy by much
        y = 0.0;
        const double top = std::max(e_max_ev, 10.0) * 1.05;
        for (int i = 0; i <= 256; ++i)
            for (int a = 0; a <= 90; ++a) y = std::max(y, paper_yield(top * i / 256.0, (double)a));
    }
    y = std::max(y, 1.0);
    const double kmax = std::max(1, em.k_max);
    QueueFactors q;
    double yg = 1.0;
    for (int g = 1; g <= em.max_generation; ++g) {
        yg *= y;
        const double need = g == 1 ? std::min(kmax, std::max(2.0, 2.0 * y)) : std::min(16.0, 2.0 * yg);
        q.f[g & 1] = std::max(q.f[g & 1], need);
    }
    if (d.queue_factor > 0.0) q.f[1] = d.queue_factor;
    return q;
}

int64_t default_chunk(const rtmc_ctx* ctx, const QueueFactors& qf)
{
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) { cudaGetLastError(); free_b = 0; }
    double avail = (double)free_b;
    for (int b = 0; b < 2; ++b) avail += (double)(ctx->q_oe[b].bytes + ctx->q_dt[b].bytes + ctx->q_id[b].bytes);
    avail += (double)(ctx->hits.bytes + ctx->wraps.bytes + ctx->kcount.bytes);
    // queue entries (48 B) in both buffers, hit record and wrap count per slot, escape count per primary
    const double per_primary = 48.0 * (qf.f[0] + qf.f[1]) + 20.0 * std::max(qf.f[0], qf.f[1]) + 4.0;
    int64_t chunk = (int64_t)1 << 26;
    while (chunk > ((int64_t)1 << 20) && per_primary * (double)chunk > 0.25 * avail) chunk >>= 1;
    return chunk;
}

void fill_result(rtmc_result& r, const Tally& t, int64_t n_prim)
{
    std::memset(&r, 0, sizeof r);
    r.n_primaries = n_prim;
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
    if (n_prim > 0) r.sey = (double)r.sum_k / (double)n_prim;
    if (n_prim > 1) {
        const double var = ((double)r.sum_k2 / (double)n_prim - r.sey * r.sey) / (double)(n_prim - 1);
        r.sey_se = var > 0.0 ? std::sqrt(var) : 0.0;
    }
}

}  // namespace rtmc

namespace {

using rtmc::make_params;
using rtmc::make_table;
using rtmc::make_emission;

struct ItemOut {
    rtmc_result* res;
    uint64_t* hist_e;   // host, n_ebins or NULL
    uint64_t* hist_a;
    uint64_t* hist_z;   // host, n_zbins or NULL
    rtmc_record* rec;   // host or NULL
    int64_t rec_cap;
    int64_t* n_rec;
};

// Run one (energy, angle) item through the wavefront loop.
int run_item(rtmc_ctx* ctx, DeviceMesh& m, double energy, double theta_deg, unsigned item,
             int64_t n_prim, uint64_t seed, const rtmc_run_desc& d, ItemOut o)
{
    using namespace rtmc;
    cudaStream_t s = ctx->stream;
    const rtmc_emission& em = ctx->emission;
    const bool record = o.rec != nullptr;
    const bool need_wraps = record || d.prim_hash != nullptr;   // wrap counts enter records and hashes

    const RunParams p = make_params(m, d, seed, item, energy, theta_deg);
    const TableDesc tab = make_table(ctx);
    // generation 0 at normal incidence runs parallel to z: the column grid;
    // at a fixed oblique incidence (azimuth 0) the slanted grid of that direction
    const bool columns = m.col_ok && d.traversal == 0 && theta_deg == 0.0 && !d.random_polar;
    GridDev slant{};
    const bool slanted = !columns && m.col_ok && d.traversal == 0 && !d.random_polar && !d.random_azimuth &&
                         !d.fp64_retest && theta_deg > 0.0 && n_prim > 0 &&
                         slant_grid(ctx, m, p.sin_t, -p.cos_t, slant);
    const Emission e = make_emission(em);

    // Queue capacities: buffer 0 holds even generations, buffer 1 odd ones,
    // sized from the expected yield (queue_factors); a chunk whose daughters
    // overflow is run again with doubled capacities.
    const QueueFactors qf = queue_factors(ctx, d, energy);
    int64_t chunk = d.chunk > 0 ? d.chunk : default_chunk(ctx, qf);
    chunk = std::min<int64_t>(chunk, std::max<int64_t>(n_prim, 1));
    double mult[2] = {qf.f[0], qf.f[1]};
    const Tuning tune = tuning_from(d);
    int64_t retries = 0;

    for (int attempt = 0;; ++attempt) {
        const int64_t cap0 = (int64_t)std::ceil((double)chunk * mult[0]) + 256;
        const int64_t cap1 = (int64_t)std::ceil((double)chunk * mult[1]) + 256;
        if (cap0 > 0xFFFFFFF0ll || cap1 > 0xFFFFFFF0ll)
            return ctx->fail(RTMC_ERR_CAPACITY, "run: queue capacity exceeds 2^32 rays; lower chunk");
        const int64_t capmax = std::max(cap0, cap1);
        cudaError_t ce = cudaSuccess;
        for (int b = 0; b < 2 && ce == cudaSuccess; ++b) {
            const int64_t c = b ? cap1 : cap0;
            ce = scratch_reserve(ctx->q_oe[b], (size_t)c * 16);
            if (ce == cudaSuccess) ce = scratch_reserve(ctx->q_dt[b], (size_t)c * 16);
            if (ce == cudaSuccess) ce = scratch_reserve(ctx->q_id[b], (size_t)c * 16);
        }
        if (ce == cudaSuccess) ce = scratch_reserve(ctx->hits, (size_t)capmax * 16);
        if (ce == cudaSuccess && need_wraps) ce = scratch_reserve(ctx->wraps, (size_t)capmax * 4);
        const bool kc_new = ctx->kcount.bytes < (size_t)chunk * 4;
        if (ce == cudaSuccess) ce = scratch_reserve(ctx->kcount, (size_t)chunk * 4);
        if (ce == cudaSuccess && kc_new) ce = cudaMemsetAsync(ctx->kcount.ptr, 0, ctx->kcount.bytes, s);
        if (ce == cudaSuccess) ce = scratch_reserve(ctx->ctl, sizeof(Control));
        if (ce == cudaSuccess && !d.id_order) ce = scratch_reserve(ctx->sort_counts, sort_scratch_bytes(1));
        if (ce == cudaSuccess) ce = scratch_reserve(ctx->tally, sizeof(Tally));
        if (ce == cudaSuccess) ce = scratch_reserve(ctx->hist, (size_t)(d.n_ebins + d.n_abins + d.n_zbins) * 8);
        if (ce == cudaSuccess && record) ce = scratch_reserve(ctx->records, (size_t)std::max<int64_t>(o.rec_cap, 1) * sizeof(rtmc_record));
        if (ce == cudaSuccess && slanted) ce = scratch_reserve(ctx->grids, sizeof(GridDev));
        if (ce == cudaSuccess && slanted)
            ce = cudaMemcpyAsync(ctx->grids.ptr, &slant, sizeof(GridDev), cudaMemcpyHostToDevice, s);
        if (ce != cudaSuccess) return ctx->fail(RTMC_ERR_OOM, std::string("run: scratch: ") + cudaGetErrorString(ce));

        Queues q;
        for (int b = 0; b < 2; ++b) {
            q.oe[b] = (float4*)ctx->q_oe[b].ptr;
            q.dt[b] = (float4*)ctx->q_dt[b].ptr;
            q.id[b] = (uint4*)ctx->q_id[b].ptr;
        }
        q.cap[0] = (unsigned)cap0;
        q.cap[1] = (unsigned)cap1;
        q.hits = (float4*)ctx->hits.ptr;
        q.wraps = need_wraps ? (int*)ctx->wraps.ptr : nullptr;
        q.kcount = (unsigned*)ctx->kcount.ptr;
        q.sort_counts = d.id_order ? nullptr : (unsigned*)ctx->sort_counts.ptr;
        q.ctl = (Control*)ctx->ctl.ptr;
        q.tally = (Tally*)ctx->tally.ptr;
        q.hist_e = (unsigned long long*)ctx->hist.ptr;
        q.hist_a = q.hist_e + d.n_ebins;
        q.prim_hash = (unsigned long long*)d.prim_hash;
        q.records = record ? (rtmc_record*)ctx->records.ptr : nullptr;
        q.rec_cap = record ? (unsigned long long)o.rec_cap : 0ull;

        cudaEvent_t ev0, ev1;
        cudaEventCreate(&ev0);
        cudaEventCreate(&ev1);
        cudaMemsetAsync(q.tally, 0, sizeof(Tally), s);
        cudaMemsetAsync(q.hist_e, 0, (size_t)(d.n_ebins + d.n_abins + d.n_zbins) * 8, s);
        if (d.prim_hash) cudaMemsetAsync(d.prim_hash, 0, (size_t)n_prim * 8, s);
        // per-kernel timing (profile): one event pair per launch, kind 0..4 (4: column grid)
        std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> kev;
        auto tick = [&](int kind) -> int {
            if (!d.profile) return -1;
            cudaEvent_t a, b;
            cudaEventCreate(&a);
            cudaEventCreate(&b);
            cudaEventRecord(a, s);
            kev.push_back({kind, {a, b}});
            return (int)kev.size() - 1;
        };
        auto tock = [&](int h) { if (h >= 0) cudaEventRecord(kev[h].second.second, s); };
        int64_t launches = 0, trav_launches = 0;
        cudaEventRecord(ev0, s);
        for (int64_t first = 0; first < n_prim && ce == cudaSuccess; first += chunk) {
            const unsigned nc = (unsigned)std::min<int64_t>(chunk, n_prim - first);
            ce = cudaMemsetAsync(q.ctl, 0, sizeof(Control), s);
            int h = tick(0);
            if (ce == cudaSuccess)
                ce = d.id_order ? launch_generate(p, q, 0, (unsigned long long)first, nc, s)
                                : launch_generate_sorted(p, q, (unsigned long long)first, nc, s);
            tock(h);
            launches += d.id_order ? 1 : 6;      // sorted: count, scan (three kernels), scatter, write
            for (int g = 0; g <= em.max_generation && ce == cudaSuccess; ++g) {
                const int buf = g & 1;
                const bool col = (columns || slanted) && g == 0;
                h = tick(col ? 4 : 1);
                if (columns && g == 0)
                    ce = launch_columns(m, p, q, buf, g, ctx->num_sms, need_wraps, d.fp64_retest != 0, s);
                else if (slanted && g == 0)
                    ce = launch_slant(m, p, (const GridDev*)ctx->grids.ptr, false, q, buf, g, ctx->num_sms,
                                      need_wraps, s);
                else
                    ce = launch_traverse(m, p, q, buf, g, ctx->num_sms, tune, need_wraps, d.count_visits != 0,
                                         d.fp64_retest != 0, s);
                tock(h);
                h = tick(2);
                if (ce == cudaSuccess)
                    ce = launch_shade(m, p, tab, e, q, buf, g, (unsigned long long)first, ctx->num_sms, record, s);
                tock(h);
                launches += 2;
                if (!col) ++trav_launches;
            }
            h = tick(3);
            if (ce == cudaSuccess) ce = launch_finalize(q, nc, s);
            tock(h);
            ++launches;
        }
        cudaEventRecord(ev1, s);
        Tally t;
        std::vector<unsigned long long> hist((size_t)(d.n_ebins + d.n_abins + d.n_zbins));
        if (ce == cudaSuccess) ce = cudaMemcpyAsync(&t, q.tally, sizeof t, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess)
            ce = cudaMemcpyAsync(hist.data(), q.hist_e, hist.size() * 8, cudaMemcpyDeviceToHost, s);
        if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
        float ms = 0.f;
        if (ce == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
        cudaEventDestroy(ev0);
        cudaEventDestroy(ev1);
        double kms[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
        for (auto& k : kev) {
            float x = 0.f;
            if (ce == cudaSuccess && cudaEventElapsedTime(&x, k.second.first, k.second.second) == cudaSuccess)
                kms[k.first] += x;
            cudaEventDestroy(k.second.first);
            cudaEventDestroy(k.second.second);
        }
        if (ce != cudaSuccess) return cuda_fail(ctx, ce, "run");
        const unsigned long long status_all = t.status;
        if (status_all & ST_QUEUE_OVERFLOW) {
            if (attempt >= 6) return ctx->fail(RTMC_ERR_CAPACITY, "run: daughter queue overflow after six retries");
            mult[0] *= 2; mult[1] *= 2;
            ++retries;
            // the per-primary counts of the aborted chunk must start from zero again
            cudaMemsetAsync(ctx->kcount.ptr, 0, ctx->kcount.bytes, s);
            continue;
        }
        if (status_all & (ST_STACK_OVERFLOW | ST_LOOP_LIMIT | ST_COLUMN))
            return ctx->fail(RTMC_ERR_DEVICE_CHECK, "run: traversal stack overflow, iteration bound or a non-vertical ray in the column grid");
        if (record && (status_all & ST_RECORD_OVERFLOW))
            return ctx->fail(RTMC_ERR_CAPACITY, "run_records: record buffer too small");

        rtmc_result& r = *o.res;
        rtmc::fill_result(r, t, n_prim);
        r.queue_retries = retries;
        r.gpu_ms = ms;
        r.launches = launches;
        r.traverse_launches = trav_launches;
        r.ms_generate = kms[0];
        r.ms_traverse = kms[1];
        r.ms_shade = kms[2];
        r.ms_finalize = kms[3];
        r.ms_column = kms[4];
        if (o.hist_e) for (int b = 0; b < d.n_ebins; ++b) o.hist_e[b] = hist[b];
        if (o.hist_a) for (int b = 0; b < d.n_abins; ++b) o.hist_a[b] = hist[d.n_ebins + b];
        if (o.hist_z) for (int b = 0; b < d.n_zbins; ++b) o.hist_z[b] = hist[d.n_ebins + d.n_abins + b];
        if (record) {
            const int64_t nrec = (int64_t)std::min<unsigned long long>(t.rays_recorded, (unsigned long long)o.rec_cap);
            ce = cudaMemcpyAsync(o.rec, q.records, (size_t)nrec * sizeof(rtmc_record), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) return cuda_fail(ctx, ce, "run_records: copy");
            if (o.n_rec) *o.n_rec = nrec;
        }
        return RTMC_OK;
    }
}

int check_run_args(rtmc_ctx* ctx, int32_t mesh_id, int64_t n_primaries, const rtmc_run_desc& d)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (mesh_id < 0 || mesh_id >= (int)ctx->meshes.size() || !ctx->meshes[mesh_id].tri_in)
        return ctx->fail(RTMC_ERR_NOT_LOADED, "run: unknown mesh id");
    if (!ctx->meshes[mesh_id].built) return ctx->fail(RTMC_ERR_NOT_BUILT, "run: build_bvh first");
    if (!ctx->table_loaded) return ctx->fail(RTMC_ERR_NOT_LOADED, "run: load_see_tables first");
    if (n_primaries < 0 || n_primaries > ((int64_t)1 << 40)) return ctx->fail(RTMC_ERR_INVALID_ARG, "run: n_primaries out of range");
    return rtmc::check_run_desc(ctx, d);
}

}  // namespace

int rtmc::check_run_desc(rtmc_ctx* ctx, const rtmc_run_desc& d)
{
    if (d.n_ebins <= 0 || d.n_ebins > 4096 || d.n_abins <= 0 || d.n_abins > 4096 || !(d.hist_e_max_ev > 0.0))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run: histogram shape");
    if (d.block_threads != 0 && (d.block_threads % 32 != 0 || d.block_threads < 32 || d.block_threads > 128))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run: block_threads must be a multiple of 32 in [32, 128]");
    if (d.traversal < 0 || d.traversal > 2) return ctx->fail(RTMC_ERR_INVALID_ARG, "run: unknown traversal variant");
    if (d.n_zbins < 0 || d.n_zbins > 4096 || (d.n_zbins > 0 && !d.hist_z))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run: n_zbins in [0, 4096] and hist_z needed when n_zbins > 0");
    if (d.stack_depth != 0 && d.stack_depth != 8 && d.stack_depth != 16 && d.stack_depth != 32)
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run: stack_depth must be 8, 16 or 32");
    if (d.fetch_threshold < 0 || d.fetch_threshold > 32)
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run: fetch_threshold must be in [0, 32]");
    if (d.fp64_retest && d.traversal == 1)
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run: fp64_retest needs the while-while traversal");
    if (d.chunk < 0 || d.chunk > ((int64_t)1 << 28)) return ctx->fail(RTMC_ERR_INVALID_ARG, "run: chunk out of range");
    if (d.max_wraps < 0 || d.max_wraps > (1 << 20)) return ctx->fail(RTMC_ERR_INVALID_ARG, "run: max_wraps out of range");
    if (d.blocks_per_sm < 0 || d.blocks_per_sm > 64) return ctx->fail(RTMC_ERR_INVALID_ARG, "run: blocks_per_sm out of range");
    if (d.max_visits < 0) return ctx->fail(RTMC_ERR_INVALID_ARG, "run: max_visits must be >= 0");
    if (!(d.queue_factor >= 0.0 && d.queue_factor <= 64.0))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run: queue_factor must be in [0, 64]");
    return RTMC_OK;
}

extern "C" {

int rtmc_create(rtmc_ctx** out, int32_t device, void* cuda_stream)
{
    if (!out) return RTMC_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return RTMC_ERR_CUDA;
    rtmc_ctx* ctx = new (std::nothrow) rtmc_ctx;
    if (!ctx) return RTMC_ERR_OOM;
    ctx->device = device;
    DeviceGuard g(device);
    cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (cuda_stream) {
        ctx->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
            delete ctx;
            return RTMC_ERR_CUDA;
        }
        ctx->own_stream = true;
    }
    *out = ctx;
    return RTMC_OK;
}

void rtmc_destroy(rtmc_ctx* ctx)
{
    if (!ctx) return;
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto& m : ctx->meshes) {
        cudaFree(m.tri_in);
        cudaFree(m.nodes);
        cudaFree(m.tris);
        cudaFree(m.normals);
        cudaFree(m.inv_order);
        cudaFree(m.q8);
        cudaFree(m.w4);
        cudaFree(m.q4);
        rtmc::free_columns(m);
    }
    cudaFree(ctx->delta);
    if (ctx->batch_graph) cudaGraphExecDestroy(ctx->batch_graph);
    rtmc::Scratch* all[] = {&ctx->q_oe[0], &ctx->q_oe[1], &ctx->q_dt[0], &ctx->q_dt[1], &ctx->q_id[0],
                            &ctx->q_id[1], &ctx->hits, &ctx->kcount, &ctx->ctl, &ctx->tally, &ctx->hist,
                            &ctx->wraps, &ctx->records, &ctx->tmp, &ctx->items,
                            &ctx->sort_counts, &ctx->grids};
    for (auto* s : all) rtmc::scratch_free(*s);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    delete ctx;
}

const char* rtmc_last_error(const rtmc_ctx* ctx)
{
    return ctx ? ctx->err.c_str() : "null context";
}

int rtmc_load_mesh(rtmc_ctx* ctx, const float* tri, int64_t n_tri, const rtmc_box* box, int32_t* mesh_id)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (!tri || !box || !mesh_id || n_tri <= 0 || n_tri >= ((int64_t)1 << 30))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "load_mesh: bad arguments");
    if (!(box->lx > 0.0) || !(box->ly > 0.0) || !(box->z_top > box->z_min))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "load_mesh: degenerate cell");
    DeviceGuard g(ctx->device);
    DeviceMesh m;
    m.n_tri = n_tri;
    m.box = *box;
    cudaError_t e = cudaMalloc(&m.tri_in, (size_t)n_tri * 36);
    if (e != cudaSuccess) return ctx->fail(RTMC_ERR_OOM, std::string("load_mesh: ") + cudaGetErrorString(e));
    e = cudaMemcpyAsync(m.tri_in, tri, (size_t)n_tri * 36, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
        cudaFree(m.tri_in);
        return cuda_fail(ctx, e, "load_mesh");
    }
    ctx->meshes.push_back(m);
    *mesh_id = (int32_t)ctx->meshes.size() - 1;
    return RTMC_OK;
}

int rtmc_unload_mesh(rtmc_ctx* ctx, int32_t mesh_id)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (mesh_id < 0 || mesh_id >= (int)ctx->meshes.size() || !ctx->meshes[mesh_id].tri_in)
        return ctx->fail(RTMC_ERR_NOT_LOADED, "unload_mesh: unknown mesh id");
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    DeviceMesh& m = ctx->meshes[mesh_id];
    cudaFree(m.tri_in);
    cudaFree(m.nodes);
    cudaFree(m.tris);
    cudaFree(m.normals);
    cudaFree(m.inv_order);
    cudaFree(m.q8);
    cudaFree(m.w4);
    cudaFree(m.q4);
    rtmc::free_columns(m);
    m = DeviceMesh();
    return RTMC_OK;
}

int rtmc_load_see_tables(rtmc_ctx* ctx, const float* delta, const rtmc_grid* grid, const rtmc_emission* em)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (!delta || !grid || !em || grid->n_e < 2 || grid->n_theta < 2 || grid->n_e > 65536 || grid->n_theta > 4096 ||
        !(grid->e_lo_ev > 0.0) || !(grid->e_hi_ev > grid->e_lo_ev) || !(grid->theta_step_deg > 0.0))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "load_see_tables: bad grid");
    if (em->k_max < 0 || em->k_max > 15 || em->max_generation < 1 || em->max_generation > 6 || !(em->phi_ev > 0.0) ||
        !(em->e_cut_ev > 0.0) || (em->model != RTMC_EMISSION_TABLE && em->model != RTMC_EMISSION_PAPER_FIT))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "load_see_tables: bad emission parameters");
    DeviceGuard g(ctx->device);
    const size_t bytes = (size_t)grid->n_e * grid->n_theta * sizeof(float);
    if (ctx->delta) { cudaFree(ctx->delta); ctx->delta = nullptr; }
    cudaError_t e = cudaMalloc(&ctx->delta, bytes);
    if (e == cudaSuccess) e = cudaMemcpyAsync(ctx->delta, delta, bytes, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "load_see_tables");
    {   // the largest tabulated yield sizes the daughter queues
        std::vector<float> h((size_t)grid->n_e * grid->n_theta);
        e = cudaMemcpy(h.data(), ctx->delta, bytes, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(ctx, e, "load_see_tables");
        double y = 0.0;
        for (float v : h) if (std::isfinite(v)) y = std::max(y, (double)v);
        ctx->yield_max = y;
    }
    ctx->grid = *grid;
    ctx->emission = *em;
    ctx->table_loaded = true;
    return RTMC_OK;
}

int rtmc_build_bvh(rtmc_ctx* ctx, int32_t mesh_id, int32_t bvh_kind)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (mesh_id < 0 || mesh_id >= (int)ctx->meshes.size() || !ctx->meshes[mesh_id].tri_in)
        return ctx->fail(RTMC_ERR_NOT_LOADED, "build_bvh: unknown mesh id");
    const int format = bvh_kind & 0xFF, leaf = (bvh_kind >> 8) & 0xFF, builder = bvh_kind >> 16;
    if ((format != RTMC_BVH_FP32 && format != RTMC_BVH_Q8 && format != RTMC_BVH_W4 && format != RTMC_BVH_Q4) ||
        (builder != 0 && builder != 1) ||
        leaf > 8)
        return ctx->fail(RTMC_ERR_INVALID_ARG, "build_bvh: unknown bvh kind or leaf size > 8");
    DeviceGuard g(ctx->device);
    DeviceMesh& m = ctx->meshes[mesh_id];
    m.kind = format;
    m.leaf_max = leaf ? leaf : 4;
    m.ploc = builder == 1;
    return rtmc::build_lbvh(ctx, m);
}

int rtmc_run(rtmc_ctx* ctx, int32_t mesh_id, const double* energies_ev, int32_t n_e, const double* theta_deg,
             int32_t n_theta, int64_t n_primaries, uint64_t seed, const rtmc_run_desc* desc, rtmc_result* out,
             uint64_t* hist_e, uint64_t* hist_a)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    const rtmc_run_desc d = desc ? *desc : default_desc();
    int rc = check_run_args(ctx, mesh_id, n_primaries, d);
    if (rc) return rc;
    if (!energies_ev || !theta_deg || !out || n_e <= 0 || n_theta <= 0)
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run: empty energy or angle list");
    if (d.prim_hash && n_e * n_theta != 1)
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run: prim_hash needs a single (energy, angle) item");
    for (int i = 0; i < n_e; ++i)
        if (!(energies_ev[i] > 0.0)) return ctx->fail(RTMC_ERR_INVALID_ARG, "run: energies must be > 0");
    for (int i = 0; i < n_theta; ++i)
        if (!(theta_deg[i] >= 0.0 && theta_deg[i] < 90.0))
            return ctx->fail(RTMC_ERR_INVALID_ARG, "run: incidence angles must be in [0, 90) degrees");
    DeviceGuard g(ctx->device);
    DeviceMesh& m = ctx->meshes[mesh_id];
    for (int ie = 0; ie < n_e; ++ie) {
        for (int it = 0; it < n_theta; ++it) {
            const int item = ie * n_theta + it;
            ItemOut o{&out[item], hist_e ? hist_e + (size_t)item * d.n_ebins : nullptr,
                      hist_a ? hist_a + (size_t)item * d.n_abins : nullptr,
                      d.n_zbins ? d.hist_z + (size_t)item * d.n_zbins : nullptr, nullptr, 0, nullptr};
            rc = run_item(ctx, m, energies_ev[ie], theta_deg[it], d.item_base + (unsigned)item, n_primaries, seed,
                          d, o);
            if (rc) return rc;
        }
    }
    return RTMC_OK;
}

int rtmc_run_records(rtmc_ctx* ctx, int32_t mesh_id, double energy_ev, double theta_deg, uint32_t item,
                     int64_t n_primaries, uint64_t seed, const rtmc_run_desc* desc, rtmc_result* out,
                     rtmc_record* rec, int64_t rec_cap, int64_t* n_rec)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    const rtmc_run_desc d = desc ? *desc : default_desc();
    int rc = check_run_args(ctx, mesh_id, n_primaries, d);
    if (rc) return rc;
    if (!out || !rec || rec_cap <= 0 || !n_rec || !(energy_ev > 0.0) || !(theta_deg >= 0.0 && theta_deg < 90.0))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run_records: bad arguments");
    DeviceGuard g(ctx->device);
    ItemOut o{out, nullptr, nullptr, d.n_zbins ? d.hist_z : nullptr, rec, rec_cap, n_rec};
    return run_item(ctx, ctx->meshes[mesh_id], energy_ev, theta_deg, item, n_primaries, seed, d, o);
}

int rtmc_trace_rays(rtmc_ctx* ctx, int32_t mesh_id, const float* o, const float* d, const int32_t* skip_tri,
                    int64_t n, rtmc_hit* hits)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (mesh_id < 0 || mesh_id >= (int)ctx->meshes.size() || !ctx->meshes[mesh_id].tri_in)
        return ctx->fail(RTMC_ERR_NOT_LOADED, "trace_rays: unknown mesh id");
    if (!ctx->meshes[mesh_id].built) return ctx->fail(RTMC_ERR_NOT_BUILT, "trace_rays: build_bvh first");
    if (n < 0 || (n > 0 && (!o || !d || !hits))) return ctx->fail(RTMC_ERR_INVALID_ARG, "trace_rays: bad arguments");
    if (n == 0) return RTMC_OK;
    DeviceGuard g(ctx->device);
    const size_t nb3 = (size_t)n * 12;
    auto align = [](size_t x) { return (x + 255) & ~(size_t)255; };
    const size_t off_d = align(nb3), off_skip = off_d + align(nb3), off_h = off_skip + align((size_t)n * 4);
    const size_t off_st = off_h + align((size_t)n * sizeof(rtmc_hit));
    cudaError_t e = rtmc::scratch_reserve(ctx->tmp, off_st + 256);
    if (e != cudaSuccess) return ctx->fail(RTMC_ERR_OOM, "trace_rays: scratch");
    char* base = (char*)ctx->tmp.ptr;
    float* d_o = (float*)base;
    float* d_d = (float*)(base + off_d);
    int* d_skip = (int*)(base + off_skip);
    rtmc_hit* d_h = (rtmc_hit*)(base + off_h);
    unsigned* d_status = (unsigned*)(base + off_st);
    cudaStream_t s = ctx->stream;
    e = cudaMemcpyAsync(d_o, o, nb3, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d_d, d, nb3, cudaMemcpyDefault, s);
    if (e == cudaSuccess && skip_tri) e = cudaMemcpyAsync(d_skip, skip_tri, (size_t)n * 4, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_status, 0, 4, s);
    if (e == cudaSuccess)
        e = rtmc::launch_trace_rays(ctx->meshes[mesh_id], d_o, d_d, skip_tri ? d_skip : nullptr, n, d_h, d_status, s);
    unsigned status = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(hits, d_h, (size_t)n * sizeof(rtmc_hit), cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, 4, cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "trace_rays");
    if (status) return ctx->fail(RTMC_ERR_DEVICE_CHECK, "trace_rays: traversal stack overflow");
    return RTMC_OK;
}

int rtmc_export_bvh(rtmc_ctx* ctx, int32_t mesh_id, int32_t which, void* out, int64_t bytes, int64_t* bytes_needed)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (mesh_id < 0 || mesh_id >= (int)ctx->meshes.size() || !ctx->meshes[mesh_id].tri_in)
        return ctx->fail(RTMC_ERR_NOT_LOADED, "export_bvh: unknown mesh id");
    const DeviceMesh& m = ctx->meshes[mesh_id];
    if (!m.built) return ctx->fail(RTMC_ERR_NOT_BUILT, "export_bvh: build_bvh first");
    const void* src = nullptr;
    int64_t need = 0;
    if (which == 0) { src = m.nodes; need = m.n_nodes * 64; }
    else if (which == 1 && m.q8) { src = m.q8; need = m.n_nodes * 32; }
    else if (which == 2) { src = m.tris; need = m.n_tri * 48; }
    else if (which == 3 && m.w4) { src = m.w4; need = m.n_w4 * 128; }
    else if (which == 4 && m.q4) { src = m.q4; need = m.n_w4 * 64; }
    else return ctx->fail(RTMC_ERR_INVALID_ARG, "export_bvh: unknown array or not built in this format");
    if (bytes_needed) *bytes_needed = need;
    if (!out) return RTMC_OK;
    if (bytes < need) return ctx->fail(RTMC_ERR_INVALID_ARG, "export_bvh: output buffer too small");
    DeviceGuard g(ctx->device);
    cudaError_t e = cudaMemcpyAsync(out, src, (size_t)need, cudaMemcpyDefault, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "export_bvh");
    return RTMC_OK;
}

int rtmc_probe_bandwidth(rtmc_ctx* ctx, int64_t bytes, int32_t iters, double* gbs)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (!gbs || bytes < (1 << 20) || bytes > ((int64_t)64 << 30) || iters < 1 || iters > 10000)
        return ctx->fail(RTMC_ERR_INVALID_ARG, "probe_bandwidth: bytes in [1 MiB, 64 GiB], iters in [1, 10000]");
    DeviceGuard g(ctx->device);
    bytes &= ~(int64_t)255;
    cudaError_t e = rtmc::scratch_reserve(ctx->tmp, (size_t)bytes + 256);
    if (e != cudaSuccess) return ctx->fail(RTMC_ERR_OOM, "probe_bandwidth: scratch");
    cudaStream_t s = ctx->stream;
    float* sink = reinterpret_cast<float*>(static_cast<char*>(ctx->tmp.ptr) + bytes);
    const int passes = (int)std::max<int64_t>(1, ((int64_t)2 << 30) / bytes);   // >= 2 GiB per launch
    e = cudaMemsetAsync(ctx->tmp.ptr, 0, (size_t)bytes, s);
    if (e == cudaSuccess) e = rtmc::launch_read_probe(ctx->tmp.ptr, (size_t)bytes, passes, ctx->num_sms, sink, s);
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaEventRecord(a, s);
    for (int i = 0; i < iters && e == cudaSuccess; ++i)
        e = rtmc::launch_read_probe(ctx->tmp.ptr, (size_t)bytes, passes, ctx->num_sms, sink, s);
    cudaEventRecord(b, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    float ms = 0.f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "probe_bandwidth");
    *gbs = (double)bytes * passes * iters / (ms / 1e3) / 1e9;
    return RTMC_OK;
}

int rtmc_philox(rtmc_ctx* ctx, const uint32_t* ctr, int64_t n, uint64_t key, uint32_t* out)
{
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (n < 0 || (n > 0 && (!ctr || !out))) return ctx->fail(RTMC_ERR_INVALID_ARG, "philox: bad arguments");
    if (n == 0) return RTMC_OK;
    DeviceGuard g(ctx->device);
    const size_t bytes = (size_t)n * 16;
    cudaError_t e = rtmc::scratch_reserve(ctx->tmp, 2 * bytes + 512);
    if (e != cudaSuccess) return ctx->fail(RTMC_ERR_OOM, "philox: scratch");
    uint32_t* d_c = (uint32_t*)ctx->tmp.ptr;
    uint32_t* d_o = (uint32_t*)((char*)ctx->tmp.ptr + ((bytes + 255) & ~(size_t)255));
    cudaStream_t s = ctx->stream;
    e = cudaMemcpyAsync(d_c, ctr, bytes, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = rtmc::launch_philox(d_c, n, key, d_o, s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, d_o, bytes, cudaMemcpyDefault, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "philox");
    return RTMC_OK;
}

uint64_t rtmc_record_hash(const rtmc_record* r)
{
    if (!r) return 0;
    return rtmc::record_hash_fields(r->prim, r->path, r->fate, r->tri, r->k, r->e_bin, r->a_bin, r->wraps);
}

}  // extern "C"
