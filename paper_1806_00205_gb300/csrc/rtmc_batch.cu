// rtmc_batch.cu -- rtmc_run_batch: many (mesh, energy, angle) items in one
// captured CUDA graph.
//
// Items of one mesh share the wavefront queues: the chunk-linear index g runs
// over (item, primary) pairs, item-major, so a chunk can span several items
// and the persistent traversal kernels stay full up to the last item.  The
// whole launch sequence (per mesh, per chunk: generate, traverse [+ FP64
// re-test] and shade per generation, finalize) is recorded once by stream
// capture and replayed as one graph launch on later calls with the same batch
// shape and the same scratch buffers.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "rtmc_internal.h"

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

// Per-kernel CUDA-event timing of an eager batch (kind 0 generate, 1
// traverse, 2 shade, 3 finalize, 4 column grid).
struct KernelTimer {
    bool on = false;
    std::vector<std::pair<int, std::pair<cudaEvent_t, cudaEvent_t>>> ev;
    int tick(int kind, cudaStream_t s)
    {
        if (!on) return -1;
        cudaEvent_t a, b;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        cudaEventRecord(a, s);
        ev.push_back({kind, {a, b}});
        return (int)ev.size() - 1;
    }
    void tock(int h, cudaStream_t s) { if (h >= 0) cudaEventRecord(ev[h].second.second, s); }
    void collect(double ms[5], int64_t& trav_launches)
    {
        for (auto& k : ev) {
            float x = 0.f;
            if (cudaEventElapsedTime(&x, k.second.first, k.second.second) == cudaSuccess) ms[k.first] += x;
            if (k.first == 1) ++trav_launches;
            cudaEventDestroy(k.second.first);
            cudaEventDestroy(k.second.second);
        }
        ev.clear();
    }
};

// Chunks of one mesh's items over the item-major linear index of (item,
// primary) pairs.  Generation 0 of an item at normal incidence can run parallel
// to z through the column grid, one at a fixed oblique incidence through the
// slanted grid of its direction (class 1 and 2; class 0: the hierarchy).  A
// chunk whose items all have a grid traces generation 0 through the grids (the
// vertical kernel when all are at normal incidence), else through the
// hierarchy; so that neither holds the other back, the chunks are cut where an
// item without a grid follows one with a grid or the reverse, then into pieces
// of at most `chunk` pairs.
struct BatchChunk {
    int64_t g0;
    unsigned n;
    int method;          // generation 0: 0 hierarchy, 1 vertical column grid, 2 per-item grids
};

std::vector<BatchChunk> batch_chunks(const rtmc_batch& b, const int* cls, int64_t chunk)
{
    const int64_t per_mesh = (int64_t)b.n_e * b.n_theta;
    std::vector<BatchChunk> out;
    int64_t i0 = 0;
    while (i0 < per_mesh) {
        const bool grid = cls[i0] != 0;
        int64_t i1 = i0 + 1;
        while (i1 < per_mesh && (cls[i1] != 0) == grid) ++i1;
        const int64_t lo = i0 * b.n_primaries, hi = i1 * b.n_primaries;
        for (int64_t g0 = lo; g0 < hi; g0 += chunk) {
            const unsigned n = (unsigned)std::min<int64_t>(chunk, hi - g0);
            int method = 0;
            if (grid && n > 0) {
                const int64_t a = g0 / b.n_primaries, z = (g0 + n - 1) / b.n_primaries;
                method = 1;
                for (int64_t it = a; it <= z; ++it) if (cls[it] != 1) method = 2;
            }
            out.push_back({g0, n, method});
        }
        i0 = i1;
    }
    return out;
}

// Record the launch sequence of the whole batch on `s`.
cudaError_t record_batch(rtmc_ctx* ctx, const rtmc_batch& b, const rtmc_run_desc& d, const rtmc::Queues& q,
                         rtmc::ItemDev* d_items, rtmc::Tally* d_tallies, unsigned long long* d_hists,
                         const std::vector<int>& cls, const rtmc::GridDev* d_grids,
                         int64_t chunk, const rtmc::Tuning& tune, int64_t n_items, cudaStream_t s,
                         KernelTimer& kt, int64_t& launches)
{
    using namespace rtmc;
    const int nbins = d.n_ebins + d.n_abins + d.n_zbins;
    cudaError_t ce = cudaMemsetAsync(d_tallies, 0, (size_t)(n_items + 1) * sizeof(Tally), s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(d_hists, 0, (size_t)n_items * nbins * 8, s);
    const TableDesc tab = make_table(ctx);
    const Emission em = make_emission(ctx->emission);
    const int64_t per_mesh = (int64_t)b.n_e * b.n_theta;
    for (int mi = 0; mi < b.n_meshes && ce == cudaSuccess; ++mi) {
        const DeviceMesh& m = ctx->meshes[b.mesh_ids[mi]];
        const RunParams p = make_params(m, d, b.seed, 0u, 1.0, 0.0);
        ItemCtx ic;
        ic.items = d_items + mi * per_mesh;
        ic.n_per_item = (unsigned long long)b.n_primaries;
        ic.tallies = d_tallies;
        ic.hists = d_hists;
        for (const BatchChunk& c : batch_chunks(b, cls.data() + mi * per_mesh, chunk)) {
            if (ce != cudaSuccess) break;
            const int64_t g0 = c.g0;
            const unsigned n = c.n;
            ic.g0 = (unsigned long long)g0;
            ic.it_lo = (unsigned)(g0 / b.n_primaries);
            ic.n_items = (unsigned)((g0 + n - 1) / b.n_primaries) - ic.it_lo + 1;
            Queues qq = q;
            qq.tally = d_tallies + n_items;   // traversal-side counters and status: the batch slot
            ce = cudaMemsetAsync(q.ctl, 0, sizeof(Control), s);
            int h = kt.tick(0, s);
            const bool sorted = !d.id_order && ic.n_items <= (unsigned)kChunkItems;
            if (ce == cudaSuccess)
                ce = sorted ? launch_generate_items_sorted(p, ic, qq, n, s) : launch_generate_items(p, ic, qq, n, s);
            kt.tock(h, s);
            launches += sorted ? 6 : 1;          // sorted: count, scan (three kernels), scatter, write
            for (int g = 0; g <= ctx->emission.max_generation && ce == cudaSuccess; ++g) {
                const int buf = g & 1;
                const int method = g == 0 ? c.method : 0;
                h = kt.tick(method ? 4 : 1, s);
                if (method == 1)
                    ce = launch_columns(m, p, qq, buf, g, ctx->num_sms, true, d.fp64_retest != 0, s);
                else if (method == 2)
                    ce = launch_slant(m, p, d_grids + mi * per_mesh, true, qq, buf, g, ctx->num_sms, true, s);
                else
                    ce = launch_traverse(m, p, qq, buf, g, ctx->num_sms, tune, true, d.count_visits != 0,
                                         d.fp64_retest != 0, s);
                kt.tock(h, s);
                h = kt.tick(2, s);
                if (ce == cudaSuccess) ce = launch_shade_items(m, p, tab, em, ic, qq, buf, g, ctx->num_sms, s);
                kt.tock(h, s);
                launches += 2;
            }
            h = kt.tick(3, s);
            if (ce == cudaSuccess) ce = launch_finalize_items(ic, qq, n, ctx->num_sms, s);
            kt.tock(h, s);
            launches += 1;
        }
    }
    return ce;
}

}  // namespace

extern "C" int rtmc_run_batch(rtmc_ctx* ctx, const rtmc_batch* batch, const rtmc_run_desc* desc, rtmc_result* out,
                              uint64_t* hist_e, uint64_t* hist_a)
{
    using namespace rtmc;
    if (!ctx) return RTMC_ERR_INVALID_ARG;
    if (!batch || !out || !batch->mesh_ids || !batch->energies_ev || !batch->theta_deg || batch->n_meshes <= 0 ||
        batch->n_e <= 0 || batch->n_theta <= 0 || batch->n_primaries < 0 ||
        batch->n_primaries > ((int64_t)1 << 32))
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run_batch: bad batch description");
    rtmc_run_desc d;
    std::memset(&d, 0, sizeof d);
    if (desc) {
        d = *desc;
    } else {
        d.n_ebins = 64;
        d.n_abins = 18;
        d.hist_e_max_ev = 50.0;
    }
    int rc = check_run_desc(ctx, d);
    if (rc) return rc;
    if (!ctx->table_loaded) return ctx->fail(RTMC_ERR_NOT_LOADED, "run_batch: load_see_tables first");
    if (d.prim_hash) return ctx->fail(RTMC_ERR_INVALID_ARG, "run_batch: per-primary hashes are not supported");
    if (d.n_ebins + d.n_abins + d.n_zbins > 512)
        return ctx->fail(RTMC_ERR_INVALID_ARG, "run_batch: n_ebins + n_abins + n_zbins must be <= 512");
    for (int i = 0; i < batch->n_meshes; ++i) {
        const int mid = batch->mesh_ids[i];
        if (mid < 0 || mid >= (int)ctx->meshes.size() || !ctx->meshes[mid].tri_in)
            return ctx->fail(RTMC_ERR_NOT_LOADED, "run_batch: unknown mesh id");
        if (!ctx->meshes[mid].built) return ctx->fail(RTMC_ERR_NOT_BUILT, "run_batch: build_bvh first");
    }
    for (int i = 0; i < batch->n_e; ++i)
        if (!(batch->energies_ev[i] > 0.0)) return ctx->fail(RTMC_ERR_INVALID_ARG, "run_batch: energies must be > 0");
    for (int i = 0; i < batch->n_theta; ++i)
        if (!(batch->theta_deg[i] >= 0.0 && batch->theta_deg[i] < 90.0))
            return ctx->fail(RTMC_ERR_INVALID_ARG, "run_batch: incidence angles must be in [0, 90) degrees");

    DeviceGuard guard(ctx->device);
    cudaStream_t s = ctx->stream;
    const int64_t per_mesh = (int64_t)batch->n_e * batch->n_theta;
    const int64_t n_items = per_mesh * batch->n_meshes;
    const int nbins = d.n_ebins + d.n_abins + d.n_zbins;

    // item table (host -> device every call: energies and angles may change)
    std::vector<ItemDev> items((size_t)n_items);
    for (int mi = 0; mi < batch->n_meshes; ++mi)
        for (int ie = 0; ie < batch->n_e; ++ie)
            for (int it = 0; it < batch->n_theta; ++it) {
                const int64_t k = (mi * (int64_t)batch->n_e + ie) * batch->n_theta + it;
                ItemDev& x = items[(size_t)k];
                const double th = batch->theta_deg[it] * kPi / 180.0;
                x.energy = (float)batch->energies_ev[ie];
                x.sin_t = (float)std::sin(th);
                x.cos_t = (float)std::cos(th);
                x.philox_item = d.item_base + (unsigned)k;
                x.prim_offset = d.primary_offset;
                x.tally = (int)k;
                x.pad = 0;
            }

    // generation 0 of each item: the column grid (normal incidence), the slanted
    // grid of its direction (fixed oblique incidence), or the hierarchy; slanted
    // grids are built here, before any capture
    std::vector<int> cls((size_t)n_items, 0);
    std::vector<GridDev> gdev((size_t)n_items);
    for (int mi = 0; mi < batch->n_meshes; ++mi) {
        DeviceMesh& m = ctx->meshes[batch->mesh_ids[mi]];
        if (d.traversal != 0 || d.random_polar || !m.col_ok) continue;
        for (int64_t j = 0; j < per_mesh; ++j) {
            const int64_t k = mi * per_mesh + j;
            const ItemDev& x = items[(size_t)k];
            if (batch->theta_deg[j % batch->n_theta] == 0.0) {
                cls[(size_t)k] = 1;
                gdev[(size_t)k] = grid_dev(m, nullptr);
            } else if (!d.random_azimuth && !d.fp64_retest && slant_grid(ctx, m, x.sin_t, -x.cos_t, gdev[(size_t)k])) {
                cls[(size_t)k] = 2;
            }
        }
    }

    // scratch: queues for one chunk, sized from the expected yield as in rtmc_run;
    // an overflow records the batch again with doubled capacities
    double e_max = 0.0;
    for (int i = 0; i < batch->n_e; ++i) e_max = std::max(e_max, batch->energies_ev[i]);
    const QueueFactors qf = queue_factors(ctx, d, e_max);
    double mult[2] = {qf.f[0], qf.f[1]};
    int64_t chunk = d.chunk;
    if (chunk <= 0) {
        // longer chunks mean fewer launches and shorter launch tails: 2^26 against
        // 2^23 traced a 9e8-primary step 6 % faster
        chunk = default_chunk(ctx, qf);
        // and at most kChunkItems items per chunk (a chunk may start inside an item), so that
        // shade keeps its per-item shared accumulators and the primaries stay spatially sorted
        chunk = std::min<int64_t>(chunk, std::max<int64_t>((int64_t)(kChunkItems - 1) * batch->n_primaries,
                                                           batch->n_primaries));
    }
    chunk = std::min<int64_t>(chunk, std::max<int64_t>(per_mesh * batch->n_primaries, 1));
    const Tuning tune = tuning_from(d);
    int64_t retries = 0;
    std::vector<Tally> t((size_t)n_items + 1);
    std::vector<unsigned long long> h((size_t)n_items * nbins);
    float ms = 0.f;
    double kms[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    int64_t launches = 0, trav_launches = 0;
    for (int attempt = 0;; ++attempt) {
    const int64_t cap0 = (int64_t)std::ceil((double)chunk * mult[0]) + 256;
    const int64_t cap1 = (int64_t)std::ceil((double)chunk * mult[1]) + 256;
    if (cap0 > 0xFFFFFFF0ll || cap1 > 0xFFFFFFF0ll)
        return ctx->fail(RTMC_ERR_CAPACITY, "run_batch: queue capacity exceeds 2^32 rays; lower chunk");
    const int64_t capmax = std::max(cap0, cap1);
    cudaError_t ce = cudaSuccess;
    const void* before[15] = {ctx->q_oe[0].ptr, ctx->q_oe[1].ptr, ctx->q_dt[0].ptr, ctx->q_dt[1].ptr,
                              ctx->q_id[0].ptr, ctx->q_id[1].ptr, ctx->hits.ptr, ctx->kcount.ptr,
                              ctx->ctl.ptr, ctx->tally.ptr, ctx->hist.ptr, ctx->items.ptr, ctx->wraps.ptr,
                              ctx->sort_counts.ptr, ctx->grids.ptr};
    for (int bb = 0; bb < 2 && ce == cudaSuccess; ++bb) {
        const int64_t c = bb ? cap1 : cap0;
        ce = scratch_reserve(ctx->q_oe[bb], (size_t)c * 16);
        if (ce == cudaSuccess) ce = scratch_reserve(ctx->q_dt[bb], (size_t)c * 16);
        if (ce == cudaSuccess) ce = scratch_reserve(ctx->q_id[bb], (size_t)c * 16);
    }
    if (ce == cudaSuccess) ce = scratch_reserve(ctx->hits, (size_t)capmax * 16);
    const bool kc_new = ctx->kcount.bytes < (size_t)chunk * 4;
    if (ce == cudaSuccess) ce = scratch_reserve(ctx->kcount, (size_t)chunk * 4);
    if (ce == cudaSuccess && (kc_new || attempt > 0)) ce = cudaMemsetAsync(ctx->kcount.ptr, 0, ctx->kcount.bytes, s);
    if (ce == cudaSuccess) ce = scratch_reserve(ctx->ctl, sizeof(Control));
    if (ce == cudaSuccess) ce = scratch_reserve(ctx->tally, (size_t)(n_items + 1) * sizeof(Tally));
    if (ce == cudaSuccess) ce = scratch_reserve(ctx->wraps, (size_t)capmax * 4);
    if (ce == cudaSuccess) ce = scratch_reserve(ctx->hist, (size_t)n_items * nbins * 8);
    if (ce == cudaSuccess) ce = scratch_reserve(ctx->items, (size_t)n_items * sizeof(ItemDev));
    if (ce == cudaSuccess && !d.id_order)
        ce = scratch_reserve(ctx->sort_counts, sort_scratch_bytes(kChunkItems));
    if (ce == cudaSuccess) ce = scratch_reserve(ctx->grids, (size_t)n_items * sizeof(GridDev));
    if (ce != cudaSuccess) return ctx->fail(RTMC_ERR_OOM, std::string("run_batch: scratch: ") + cudaGetErrorString(ce));
    const void* after[15] = {ctx->q_oe[0].ptr, ctx->q_oe[1].ptr, ctx->q_dt[0].ptr, ctx->q_dt[1].ptr,
                             ctx->q_id[0].ptr, ctx->q_id[1].ptr, ctx->hits.ptr, ctx->kcount.ptr,
                             ctx->ctl.ptr, ctx->tally.ptr, ctx->hist.ptr, ctx->items.ptr, ctx->wraps.ptr,
                             ctx->sort_counts.ptr, ctx->grids.ptr};
    const bool moved = std::memcmp(before, after, sizeof before) != 0;

    Queues q;
    for (int bb = 0; bb < 2; ++bb) {
        q.oe[bb] = (float4*)ctx->q_oe[bb].ptr;
        q.dt[bb] = (float4*)ctx->q_dt[bb].ptr;
        q.id[bb] = (uint4*)ctx->q_id[bb].ptr;
    }
    q.cap[0] = (unsigned)cap0;
    q.cap[1] = (unsigned)cap1;
    q.hits = (float4*)ctx->hits.ptr;
    q.wraps = (int*)ctx->wraps.ptr;
    q.kcount = (unsigned*)ctx->kcount.ptr;
    q.sort_counts = d.id_order ? nullptr : (unsigned*)ctx->sort_counts.ptr;
    q.ctl = (Control*)ctx->ctl.ptr;
    q.tally = (Tally*)ctx->tally.ptr;
    q.hist_e = nullptr;
    q.hist_a = nullptr;
    q.prim_hash = nullptr;
    q.records = nullptr;
    q.rec_cap = 0;

    ce = cudaMemcpyAsync(ctx->items.ptr, items.data(), items.size() * sizeof(ItemDev), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess)
        ce = cudaMemcpyAsync(ctx->grids.ptr, gdev.data(), gdev.size() * sizeof(GridDev), cudaMemcpyHostToDevice, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);     // the host copies of the tables go out of scope
    if (ce != cudaSuccess) return ctx->fail(RTMC_ERR_CUDA, std::string("run_batch: ") + cudaGetErrorString(ce));

    // graph key: everything the recorded launch parameters depend on
    std::string key;
    {
        char buf[512];
        std::snprintf(buf, sizeof buf, "%d|%d|%d|%lld|%llu|%lld|%d|%d|%d|%d|%d|%d|%d|%d|%u|%.17g|%llu|%.17g|%.17g|%.17g|%.17g|z%d|rp%d|c%lld:%lld|mv%d|g%d",
                      batch->n_meshes, batch->n_e, batch->n_theta, (long long)batch->n_primaries,
                      (unsigned long long)batch->seed, (long long)chunk, d.n_ebins, d.n_abins, d.random_azimuth,
                      d.max_wraps, d.block_threads, d.blocks_per_sm, d.traversal * 10000 + d.stack_depth * 100 + d.fetch_threshold, d.fp64_retest, d.item_base,
                      d.hist_e_max_ev, (unsigned long long)d.primary_offset, d.src_x0, d.src_x1, d.src_y0, d.src_y1,
                      d.n_zbins, d.random_polar, (long long)cap0, (long long)cap1, d.max_visits,
                      ctx->emission.max_generation);
        key = buf;
        for (int i = 0; i < batch->n_meshes; ++i) {      // every mesh array a recorded launch reads
            const DeviceMesh& m = ctx->meshes[batch->mesh_ids[i]];
            std::snprintf(buf, sizeof buf, "|%d:%p:%p:%p:%p:%p:%p:%p:%p:%d:%d", batch->mesh_ids[i],
                          (const void*)m.nodes, m.q8, m.w4, m.q4, (const void*)m.tris, (const void*)m.normals,
                          (const void*)m.col_off, (const void*)m.col_ent, m.kind, (int)m.col_ok);
            key += buf;
        }
        key += "|g";                                      // which grid generation 0 of each item takes
        for (size_t k = 0; k < cls.size(); ++k) {
            std::snprintf(buf, sizeof buf, "%d:%p,", cls[k], cls[k] ? (const void*)gdev[k].ent : nullptr);
            key += buf;
        }
        std::snprintf(buf, sizeof buf, "|cv%d|io%d|%p", d.count_visits, d.id_order, (const void*)ctx->delta);
        key += buf;
    }
    if (moved || key != ctx->batch_key) {
        if (ctx->batch_graph) { cudaGraphExecDestroy(ctx->batch_graph); ctx->batch_graph = nullptr; }
        ctx->batch_key.clear();
        ctx->batch_launches = 0;
    }

    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    KernelTimer kt;
    kt.on = d.no_graph && d.profile;
    launches = 0;
    cudaEventRecord(ev0, s);
    if (d.no_graph) {
        ce = record_batch(ctx, *batch, d, q, (ItemDev*)ctx->items.ptr, (Tally*)ctx->tally.ptr,
                          (unsigned long long*)ctx->hist.ptr, cls, (const GridDev*)ctx->grids.ptr, chunk, tune,
                          n_items, s, kt, launches);
    } else {
        if (!ctx->batch_graph) {
            cudaGraph_t graph = nullptr;
            ce = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
            if (ce == cudaSuccess) {
                KernelTimer none;
                const cudaError_t rec = record_batch(ctx, *batch, d, q, (ItemDev*)ctx->items.ptr,
                                                     (Tally*)ctx->tally.ptr, (unsigned long long*)ctx->hist.ptr,
                                                     cls, (const GridDev*)ctx->grids.ptr, chunk, tune, n_items, s,
                                                     none, ctx->batch_launches);
                ce = cudaStreamEndCapture(s, &graph);
                if (ce == cudaSuccess) ce = rec;
            }
            if (ce == cudaSuccess) ce = cudaGraphInstantiate(&ctx->batch_graph, graph, 0);
            if (ce != cudaSuccess) ctx->batch_launches = 0;
            if (graph) cudaGraphDestroy(graph);
            if (ce == cudaSuccess) ctx->batch_key = key;
            else ctx->batch_graph = nullptr;
        }
        if (ce == cudaSuccess) ce = cudaGraphLaunch(ctx->batch_graph, s);
        launches = ctx->batch_launches;
    }
    cudaEventRecord(ev1, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(t.data(), ctx->tally.ptr, t.size() * sizeof(Tally), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaMemcpyAsync(h.data(), ctx->hist.ptr, h.size() * 8, cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce == cudaSuccess) cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    trav_launches = 0;
    for (double& x : kms) x = 0.0;
    kt.collect(kms, trav_launches);
    if (ce != cudaSuccess) return ctx->fail(RTMC_ERR_CUDA, std::string("run_batch: ") + cudaGetErrorString(ce));
    unsigned long long status = 0;
    for (const Tally& x : t) status |= x.status;
    if (status & ST_QUEUE_OVERFLOW) {
        if (attempt >= 6)
            return ctx->fail(RTMC_ERR_CAPACITY, "run_batch: daughter queue overflow after six retries");
        mult[0] *= 2; mult[1] *= 2;
        ++retries;
        continue;                        // new capacities change the key: the batch is recorded again
    }
    if (status & (ST_STACK_OVERFLOW | ST_LOOP_LIMIT | ST_COLUMN))
        return ctx->fail(RTMC_ERR_DEVICE_CHECK, "run_batch: traversal stack overflow or iteration bound");
    break;
    }
    const Tally& all = t[(size_t)n_items];
    for (int64_t k = 0; k < n_items; ++k) {
        fill_result(out[k], t[(size_t)k], batch->n_primaries);
        out[k].gpu_ms = ms;
        out[k].node_visits = (int64_t)all.node_visits;     // traversal counters: batch totals
        out[k].tri_tests = (int64_t)all.tri_tests;
        out[k].retested = (int64_t)all.retested;
        out[k].column_rays = (int64_t)all.col_rays;
        out[k].launches = launches;
        out[k].queue_retries = retries;
        out[k].traverse_launches = trav_launches;
        out[k].ms_generate = kms[0];
        out[k].ms_traverse = kms[1];
        out[k].ms_shade = kms[2];
        out[k].ms_finalize = kms[3];
        out[k].ms_column = kms[4];
        if (hist_e)
            for (int bb = 0; bb < d.n_ebins; ++bb) hist_e[k * d.n_ebins + bb] = h[(size_t)k * nbins + bb];
        if (hist_a)
            for (int bb = 0; bb < d.n_abins; ++bb) hist_a[k * d.n_abins + bb] = h[(size_t)k * nbins + d.n_ebins + bb];
        if (d.n_zbins)
            for (int bb = 0; bb < d.n_zbins; ++bb)
                d.hist_z[k * d.n_zbins + bb] = h[(size_t)k * nbins + d.n_ebins + d.n_abins + bb];
    }
    return RTMC_OK;
}
