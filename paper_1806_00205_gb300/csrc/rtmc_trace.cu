// rtmc_trace.cu -- wavefront RTMC kernels (sm_103a).
//
// One chunk of primaries is processed as generations of rays held in
// structure-of-arrays queues in HBM (paper Section 2.2: daughters are
// appended to the end of the ray tree; here a whole generation is one queue):
//   generate  : primaries from Philox streams           -> queue 0
//   traverse  : (rtmc_traverse.cu) BVH closest hit, periodic cell walk -> hits
//   shade     : escape tallies / yield-table lookup / Poisson count; a block
//               prefix over the counts compacts the daughters, which are then
//               expanded one per thread into queue g+1
//   finalize  : per-primary escape counts -> sum k, sum k^2
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "rtmc_internal.h"

namespace rtmc {
namespace {

constexpr int kShadeThreads = 128;
constexpr int kShadeBlocksPerSm = 1024 / kShadeThreads;   // resident blocks per SM at 64 registers
constexpr size_t kShadeDefaultSmem = 24 * 1024;   // dynamic bytes that fit beside the static arrays

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// --------------------------------------------------------------------------
// generate
// --------------------------------------------------------------------------
// Direction of a primary.  Fixed incidence: the item's polar angle, azimuth 0
// or uniform (u2 of the primary's block).  Random incidence (Section 3.2):
// the flux of an isotropic beam through the top plane, a cosine-law polar
// angle with sin^2 theta = u0 of the path-0 block (no daughter uses path 0)
// and a uniform azimuth.  u0 is an odd multiple of 2^-24, so 1 - u0 is exact.
__device__ __forceinline__ float4 primary_dir(const RunParams& p, float sin_t, float cos_t, unsigned plo,
                                              unsigned phi, unsigned pitem, unsigned wz)
{
    bool random_az = p.random_azimuth != 0;
    if (p.random_polar) {
        const float u = u01(ray_block(p.seed, plo, phi, 0u, pitem).x);
        sin_t = sqrtf(u);
        cos_t = sqrtf(1.f - u);
        random_az = true;
    }
    float ca = 1.f, sa = 0.f;
    if (random_az) sincospif(2.0f * u01(wz), &sa, &ca);
    return make_float4(sin_t * ca, sin_t * sa, -cos_t, __int_as_float(-1));
}

__global__ void k_generate(RunParams p, float sin_t, float cos_t, unsigned long long first,
                           unsigned n, float4* __restrict__ oe, float4* __restrict__ dt,
                           uint4* __restrict__ id, Control* __restrict__ ctl)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) ctl->count[0] = n;
    if (i >= n) return;
    const unsigned long long prim = p.prim_offset + first + i;
    const unsigned plo = (unsigned)prim, phi = (unsigned)(prim >> 32);
    const uint4 w = ray_block(p.seed, plo, phi, 1u, p.item);
    const float x = p.src_x0 + u01(w.x) * (p.src_x1 - p.src_x0);
    const float y = p.src_y0 + u01(w.y) * (p.src_y1 - p.src_y0);
    oe[i] = make_float4(x, y, p.z_top, p.energy);
    dt[i] = primary_dir(p, sin_t, cos_t, plo, phi, p.item, w.z);
    id[i] = make_uint4(plo, phi, 1u, 0u);
}

// Multi-item chunk: slot i is local primary (g0 + i) % N of item (g0 + i) / N.
// Ray id = (local primary, item index, path, generation).
__global__ void k_generate_items(RunParams p, ItemCtx ic, unsigned n, float4* __restrict__ oe,
                                 float4* __restrict__ dt, uint4* __restrict__ id, Control* __restrict__ ctl)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) ctl->count[0] = n;
    if (i >= n) return;
    const unsigned long long g = ic.g0 + i;
    const unsigned it = (unsigned)(g / ic.n_per_item);
    const unsigned pl = (unsigned)(g - (unsigned long long)it * ic.n_per_item);
    const ItemDev item = ic.items[it];
    const unsigned long long prim = item.prim_offset + pl;
    const uint4 w = ray_block(p.seed, (unsigned)prim, (unsigned)(prim >> 32), 1u, item.philox_item);
    const float x = p.src_x0 + u01(w.x) * (p.src_x1 - p.src_x0);
    const float y = p.src_y0 + u01(w.y) * (p.src_y1 - p.src_y0);
    oe[i] = make_float4(x, y, p.z_top, item.energy);
    dt[i] = primary_dir(p, item.sin_t, item.cos_t, (unsigned)prim, (unsigned)(prim >> 32), item.philox_item, w.z);
    id[i] = make_uint4(pl, it, 1u, 0u);
}

// Spatially ordered generation: primaries are counting-sorted by a
// Morton-ordered 512 x 512 grid cell of their entry point (per item), so a
// warp's lanes start close together and fetch the same BVH nodes.  The sort
// is not stable (slots come from atomic cursors); per-ray results do not
// depend on queue order because each ray's random numbers are keyed by its
// identity.  Pass 1 counts, a device-wide scan turns counts into cursors,
// pass 2 writes each ray at its cursor.  Cells of 5 nm on the 256^3 foam: finer
// cells (fewer collisions on the counters' atomics, closer neighbours for the
// grid kernels) measured faster than 128 x 128 and no slower than 256 x 256.
constexpr int kSortCellBits = 9;                        // 512 x 512 cells
constexpr unsigned kSortCells = 1u << (2 * kSortCellBits);
static_assert(kSortCells == kSortBucketsPerItem, "sort scratch sized for these cells");

__device__ __forceinline__ unsigned spread9(unsigned v)   // bits 0..8 -> even bit positions
{
    v &= 0x1FFu;
    v = (v | (v << 8)) & 0x00FF00FFu;
    v = (v | (v << 4)) & 0x0F0F0F0Fu;
    v = (v | (v << 2)) & 0x33333333u;
    v = (v | (v << 1)) & 0x55555555u;
    return v;
}

template <bool ITEMS>
__device__ __forceinline__ void primary_of(const RunParams& p, const ItemCtx& ic, unsigned long long first,
                                           unsigned i, float4& oe, float4& dt, uint4& id, unsigned& bucket)
{
    unsigned long long prim;
    unsigned pitem, it_rel = 0;
    float energy, sin_t, cos_t;
    uint2 idxy;
    if (ITEMS) {
        const unsigned long long g = ic.g0 + i;
        const unsigned it = (unsigned)(g / ic.n_per_item);
        const unsigned pl = (unsigned)(g - (unsigned long long)it * ic.n_per_item);
        const ItemDev item = ic.items[it];
        prim = item.prim_offset + pl;
        pitem = item.philox_item;
        energy = item.energy; sin_t = item.sin_t; cos_t = item.cos_t;
        idxy = make_uint2(pl, it);
        it_rel = it - ic.it_lo;
    } else {
        prim = p.prim_offset + first + i;
        pitem = p.item;
        energy = p.energy; sin_t = p.sin_t; cos_t = p.cos_t;
        idxy = make_uint2((unsigned)prim, (unsigned)(prim >> 32));
    }
    const uint4 w = ray_block(p.seed, (unsigned)prim, (unsigned)(prim >> 32), 1u, pitem);
    const float ux = u01(w.x), uy = u01(w.y);
    const float x = p.src_x0 + ux * (p.src_x1 - p.src_x0);
    const float y = p.src_y0 + uy * (p.src_y1 - p.src_y0);
    oe = make_float4(x, y, p.z_top, energy);
    dt = primary_dir(p, sin_t, cos_t, (unsigned)prim, (unsigned)(prim >> 32), pitem, w.z);
    id = make_uint4(idxy.x, idxy.y, 1u, 0u);
    const unsigned cx = min((unsigned)(ux * (1 << kSortCellBits)), (1u << kSortCellBits) - 1);
    const unsigned cy = min((unsigned)(uy * (1 << kSortCellBits)), (1u << kSortCellBits) - 1);
    bucket = it_rel * kSortCells + (spread9(cx) | (spread9(cy) << 1));
}

template <bool ITEMS>
__global__ void k_prim_count(RunParams p, ItemCtx ic, unsigned long long first, unsigned n,
                             unsigned* __restrict__ counts)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 a, b;
    uint4 c;
    unsigned bucket;
    primary_of<ITEMS>(p, ic, first, i, a, b, c, bucket);
    atomicAdd(&counts[bucket], 1u);
}

// Pass 2 places only the primary's 4-byte index (scattered); pass 3 then
// writes the 48-byte queue entries in sorted order, coalesced, recomputing
// each primary from its Philox stream.
template <bool ITEMS>
__global__ void k_scatter_perm(RunParams p, ItemCtx ic, unsigned long long first, unsigned n,
                               unsigned* __restrict__ cursor, unsigned* __restrict__ perm)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float4 a, b;
    uint4 c;
    unsigned bucket;
    primary_of<ITEMS>(p, ic, first, i, a, b, c, bucket);
    const unsigned slot = atomicAdd(&cursor[bucket], 1u);
    if (slot < n) perm[slot] = i;
}

template <bool ITEMS>
__global__ void k_generate_sorted(RunParams p, ItemCtx ic, unsigned long long first, unsigned n,
                                  const unsigned* __restrict__ perm, float4* __restrict__ oe, float4* __restrict__ dt,
                                  uint4* __restrict__ id, Control* __restrict__ ctl)
{
    const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i == 0) ctl->count[0] = n;
    if (i >= n) return;
    const unsigned j = perm[i];
    float4 a, b;
    uint4 c;
    unsigned bucket;
    primary_of<ITEMS>(p, ic, first, j, a, b, c, bucket);
    oe[i] = a;
    dt[i] = b;
    id[i] = c;
}

// --------------------------------------------------------------------------
// shade
// --------------------------------------------------------------------------
__device__ __forceinline__ float lookup_delta(const TableDesc& t, float e, float alpha)
{
    float x = (__logf(e) - t.log_e_lo) * t.inv_log_span;
    x = fminf(fmaxf(x, 0.f), (float)(t.n_e - 1));
    int i = min((int)x, t.n_e - 2);
    const float fx = x - (float)i;
    float y = alpha * 57.295779513082321f * t.inv_theta_step_deg;
    y = fminf(fmaxf(y, 0.f), (float)(t.n_theta - 1));
    const int j = min((int)y, t.n_theta - 2);
    const float fy = y - (float)j;
    const float* r0 = t.delta + i * t.n_theta + j;
    const float* r1 = r0 + t.n_theta;
    const float t00 = __ldg(r0), t01 = __ldg(r0 + 1), t10 = __ldg(r1), t11 = __ldg(r1 + 1);
    return (1.f - fx) * ((1.f - fy) * t00 + fy * t01) + fx * ((1.f - fy) * t10 + fy * t11);
}

__device__ __forceinline__ int poisson_inv(float lam, float u, int k_max, int& capped)
{
    float p = expf(-lam);
    float cdf = p;
    capped = 0;
    for (int k = 0; k < k_max; ++k) {
        if (u < cdf) return k;
        p *= lam / (float)(k + 1);
        cdf += p;
    }
    if (!(u < cdf)) capped = 1;
    return k_max;
}

// Inverse of the truncated spectrum CDF 1 - 3 s^2 + 2 s^3, s = phi/(E+phi):
// smoothstep(s) = 3 s^2 - 2 s^3 = 1 - y, solved as s = 1/2 - sin(asin(2y - 1)/3).
__device__ __forceinline__ float sample_energy(const Emission& em, float u)
{
    const float y = u * em.spec_norm;
    const float s = 0.5f - sinf(asinf(fmaf(2.f, y, -1.f)) * (1.0f / 3.0f));
    return fminf(em.phi * (1.0f / s - 1.0f), em.e_cut);
}

// Section 2.2, Eq. 6: SEE yield of flat tungsten; e in eV, a (local incidence) in degrees.
__device__ __forceinline__ float gamma_fit(float e, float a)
{
    return 3.05f + 1.7949e-5f * a * a + 6.15e-7f * e * e - (371.317f - expf(0.04826f * a)) / (87.602f + e) -
           1.974e-3f * e - 0.1097f * cosf(0.1201f + 2.469f * a);
}

// Section 2.2, Eq. 7: energy (eV) of an emitted secondary; sin takes e as radians, as printed.
__device__ __forceinline__ float esee_fit(float e, float a)
{
    const float a2 = a * a, a7 = a2 * a2 * a2 * a;
    return 0.195f * e + 1.6e-4f * e * e + 0.148f * a * sinf(e) + 3.44e-15f * e * a7 - 6.54f;
}

// Section 2.2 footnote: round the fractional yield up when u falls below its
// fractional part (g - floor(g) is exact in binary floating point).
__device__ __forceinline__ int round_stochastic(float g, float u, int k_max, int& capped)
{
    g = fmaxf(g, 0.f);
    const float fl = floorf(g);
    const int k = (int)fl + (u < g - fl ? 1 : 0);
    capped = k > k_max;
    return min(k, k_max);
}

// Cosine-law direction about n in the basis of Duff et al. (JCGT 2017).
__device__ __forceinline__ float3 cosine_dir(float3 n, float u1, float u2)
{
    const float sgn = n.z >= 0.f ? 1.f : -1.f;
    const float a = -1.0f / (sgn + n.z);
    const float b = n.x * n.y * a;
    const float3 t1 = make_float3(1.f + sgn * n.x * n.x * a, sgn * b, -sgn * n.x);
    const float3 t2 = make_float3(b, sgn + n.y * n.y * a, -n.y);
    const float st = sqrtf(u1), ct = sqrtf(1.f - u1);
    float sp, cp;
    sincospif(2.0f * u2, &sp, &cp);
    const float x = st * cp, y = st * sp;
    return make_float3(x * t1.x + y * t2.x + ct * n.x, x * t1.y + y * t2.y + ct * n.y,
                       x * t1.z + y * t2.z + ct * n.z);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v)
{
    for (int off = 16; off; off >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
    return v;
}

struct ShadeOut {
    float4* oe;
    float4* dt;
    uint4* id;
    unsigned cap;
};

// Per-ray contribution to the tallies.
// Energy moments as unevaluated float pairs (hi + lo): FP64 is a small
// fraction of the FP32 rate on this GPU, so per-ray and per-warp sums stay in
// FP32 and become FP64 only where they enter an FP64 atomic.  E^2 splits
// exactly (E E rounded plus its FMA remainder); a pair sum is Knuth's TwoSum of
// the high parts with the error and the low parts carried in the low word
// (relative error a few 2^-48, far below the FP64 moments' needs).  The
// round-to-nearest intrinsics keep the compiler from contracting the steps.
struct FF {
    float hi = 0.f, lo = 0.f;
};

__device__ __forceinline__ FF ff_add(FF a, FF b)
{
    const float s = __fadd_rn(a.hi, b.hi);
    const float bv = __fsub_rn(s, a.hi);
    const float err = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bv)), __fsub_rn(b.hi, bv));
    const float lo = __fadd_rn(__fadd_rn(a.lo, b.lo), err);
    FF r;
    r.hi = __fadd_rn(s, lo);
    r.lo = __fsub_rn(lo, __fsub_rn(r.hi, s));
    return r;
}

__device__ __forceinline__ FF ff_warp_sum(FF v)
{
    for (int off = 16; off; off >>= 1) {
        FF o;
        o.hi = __shfl_xor_sync(0xFFFFFFFFu, v.hi, off);
        o.lo = __shfl_xor_sync(0xFFFFFFFFu, v.lo, off);
        v = ff_add(v, o);
    }
    return v;
}

__device__ __forceinline__ double ff_double(FF v) { return (double)v.hi + (double)v.lo; }
__device__ __forceinline__ bool ff_nonzero(FF v) { return v.hi != 0.f || v.lo != 0.f; }

struct Acc {
    unsigned rays = 0, esc = 0, lost = 0, low = 0, other = 0, emit = 0, regen = 0, emitted = 0, capped = 0;
    unsigned wraps = 0;               // multi-item chunks only (the traversal cannot tell items apart)
    FF es, e2;                        // sum E, sum E^2
    __device__ void add(const Acc& a)
    {
        rays += a.rays; esc += a.esc; lost += a.lost; low += a.low; other += a.other; emit += a.emit;
        regen += a.regen; emitted += a.emitted; capped += a.capped; wraps += a.wraps;
        es = ff_add(es, a.es);
        e2 = ff_add(e2, a.e2);
    }
};

__device__ __forceinline__ void acc_atomic(Tally* t, const Acc& a)
{
    if (a.rays) atomicAdd(&t->rays, (unsigned long long)a.rays);
    if (a.esc) atomicAdd(&t->escaped, (unsigned long long)a.esc);
    if (a.lost) atomicAdd(&t->lost, (unsigned long long)a.lost);
    if (a.low) atomicAdd(&t->absorbed_low, (unsigned long long)a.low);
    if (a.other) atomicAdd(&t->absorbed_other, (unsigned long long)a.other);
    if (a.emit) atomicAdd(&t->emitters, (unsigned long long)a.emit);
    if (a.regen) atomicAdd(&t->regenerated, (unsigned long long)a.regen);
    if (a.emitted) atomicAdd(&t->emitted, (unsigned long long)a.emitted);
    if (a.capped) atomicAdd(&t->capped, (unsigned long long)a.capped);
    if (a.wraps) atomicAdd(&t->wraps, (unsigned long long)a.wraps);
    if (ff_nonzero(a.es)) atomicAdd(&t->e_sum, ff_double(a.es));
    if (ff_nonzero(a.e2)) atomicAdd(&t->e2_sum, ff_double(a.e2));
}

// With ITEMS the queue holds rays of several items (ray id.y is the item
// index in ic.items).  Daughters of different items interleave in the next
// queue tile by tile, so each block keeps per-item counters and histograms
// in shared memory for every item the chunk touches (at most kChunkItems);
// a warp whose rays share one item (the common case) adds one reduced value
// per counter.  The block flushes to global memory once, at its end.
template <bool RECORD, bool ITEMS>
__global__ void __launch_bounds__(kShadeThreads, kShadeBlocksPerSm)
k_shade(const float4* __restrict__ tris, const float4* __restrict__ normals, TableDesc tab, Emission em,
        RunParams p, ItemCtx ic, const float4* __restrict__ oe, const float4* __restrict__ dt,
        const uint4* __restrict__ id, const float4* __restrict__ hits, const int* __restrict__ wraps_in,
        ShadeOut out, Control* __restrict__ ctl, int gen, unsigned cap_in, Tally* __restrict__ tally,
        unsigned long long* __restrict__ hist_e, unsigned long long* __restrict__ hist_a,
        unsigned* __restrict__ kcount, unsigned long long chunk_first,
        unsigned long long* __restrict__ prim_hash, rtmc_record* __restrict__ records,
        unsigned long long rec_cap)
{
    extern __shared__ unsigned s_hist[];              // [ITEMS ? kChunkItems : 1][n_ebins + n_abins + n_zbins]
    __shared__ unsigned s_excl[kShadeThreads + 1];
    __shared__ unsigned s_warp[kShadeThreads / 32];
    __shared__ float s_px[kShadeThreads], s_py[kShadeThreads], s_pz[kShadeThreads];
    __shared__ float s_nx[kShadeThreads], s_ny[kShadeThreads], s_nz[kShadeThreads];
    __shared__ uint4 s_id[kShadeThreads];             // child id: (x, y, parent path, gen + 1)
    __shared__ uint3 s_key[kShadeThreads];            // Philox: (prim lo, prim hi, item)
    __shared__ int s_tri[kShadeThreads];
    __shared__ float s_esee[kShadeThreads];           // paper-fit model: E_SEE of the emission
    __shared__ unsigned s_base;
    __shared__ unsigned long long s_red[10][kShadeThreads / 32];
    __shared__ double s_dred[2][kShadeThreads / 32];
    __shared__ unsigned s_icnt[kChunkItems][10];      // multi-item chunks: per-item counters
    __shared__ double s_isum[kChunkItems][2];       // multi-item warps (rare): FP64 shared atomics
    __shared__ float s_iff[kShadeThreads / 32][kChunkItems][4];   // per warp and item: sum E, sum E^2 as float pairs

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nbins = p.n_ebins + p.n_abins + p.n_zbins;
    const int zbase = p.n_ebins + p.n_abins;
    // multi-item chunks touching at most kChunkItems items accumulate per item in
    // shared memory; wider chunks (tiny items) send every ray to global atomics
    const bool shared_items = ITEMS && ic.n_items <= (unsigned)kChunkItems;
    const int hist_rows = ITEMS ? (shared_items ? (int)ic.n_items : 0) : 1;
    for (int b = tid; b < hist_rows * nbins; b += kShadeThreads) s_hist[b] = 0u;
    if (ITEMS)
        for (int b = tid; b < kChunkItems * 10; b += kShadeThreads) {
            (&s_icnt[0][0])[b] = 0u;
            if (b < kChunkItems * 2) (&s_isum[0][0])[b] = 0.0;
            if (b < kChunkItems * 4) for (int w = 0; w < kShadeThreads / 32; ++w) s_iff[w][0][b] = 0.f;
        }
    unsigned *sh_e = s_hist, *sh_a = s_hist + p.n_ebins;
    const unsigned n = min(*((volatile unsigned*)&ctl->count[gen]), cap_in);
    Acc acc;                                          // single-item runs: this thread's share
    Tally* home_tally = tally;
    unsigned long long* home_he = hist_e;
    __syncthreads();

    // block reduction of `acc` and the shared histogram into the home item
    auto flush = [&]() {
        const unsigned cs[10] = {acc.rays, acc.esc, acc.lost, acc.low, acc.other, acc.emit, acc.regen,
                                 acc.emitted, acc.capped, acc.wraps};
#pragma unroll
        for (int q = 0; q < 10; ++q) {
            const unsigned v = warp_sum(cs[q]);
            if (lane == 0) s_red[q][warp] = v;
        }
        const FF es = ff_warp_sum(acc.es), e2 = ff_warp_sum(acc.e2);
        if (lane == 0) { s_dred[0][warp] = ff_double(es); s_dred[1][warp] = ff_double(e2); }
        __syncthreads();
        if (tid < 10) {
            unsigned long long v = 0;
            for (int w = 0; w < kShadeThreads / 32; ++w) v += s_red[tid][w];
            if (v) {
                unsigned long long* dst[10] = {&home_tally->rays, &home_tally->escaped, &home_tally->lost,
                                               &home_tally->absorbed_low, &home_tally->absorbed_other,
                                               &home_tally->emitters, &home_tally->regenerated,
                                               &home_tally->emitted, &home_tally->capped, &home_tally->wraps};
                atomicAdd(dst[tid], v);
            }
        } else if (tid >= 32 && tid < 34) {
            double v = 0.0;
            for (int w = 0; w < kShadeThreads / 32; ++w) v += s_dred[tid - 32][w];
            if (v != 0.0) atomicAdd(tid == 32 ? &home_tally->e_sum : &home_tally->e2_sum, v);
        }
        for (int b = tid; b < nbins; b += kShadeThreads) {
            if (s_hist[b]) atomicAdd(&home_he[b], (unsigned long long)s_hist[b]);
            s_hist[b] = 0u;
        }
        acc = Acc();
        __syncthreads();
    };

    for (unsigned tile = blockIdx.x; tile * kShadeThreads < n; tile += gridDim.x) {
        const unsigned i = tile * kShadeThreads + tid;
        unsigned k = 0;
        Acc r;
        int jslot = -1;                               // multi-item: item index - ic.it_lo
        if (i < n) {
            const float4 a = oe[i], b = dt[i], h = hits[i];
            const uint4 rid = id[i];
            const int tri = __float_as_int(h.w);
            const unsigned g = rid.w;
            const float E = a.w;
            unsigned long long prim;
            unsigned pitem;
            int slot = 0;
            if (ITEMS) {
                const ItemDev item = ic.items[rid.y];
                prim = item.prim_offset + rid.x;
                pitem = item.philox_item;
                slot = item.tally;
                jslot = (int)(rid.y - ic.it_lo);
            } else {
                prim = ((unsigned long long)rid.y << 32) | rid.x;
                pitem = p.item;
            }
            int fate, orig = -1, e_bin = -1, a_bin = -1, kk = 0;
            r.rays = 1;
            if (ITEMS && wraps_in) r.wraps = (unsigned)wraps_in[i];
            if (tri == HIT_ESCAPE && g > 0) {
                fate = RTMC_ESCAPED;
                r.esc = 1;
                e_bin = max(0, min((int)(E / p.ebin_w), p.n_ebins - 1));
                const float pol = acosf(fminf(1.f, b.z));
                a_bin = max(0, min((int)(pol * p.inv_abin), p.n_abins - 1));
                if (!ITEMS) {
                    atomicAdd(&sh_e[e_bin], 1u);
                    atomicAdd(&sh_a[a_bin], 1u);
                } else if (shared_items) {
                    atomicAdd(&s_hist[jslot * nbins + e_bin], 1u);
                    atomicAdd(&s_hist[jslot * nbins + p.n_ebins + a_bin], 1u);
                } else {
                    unsigned long long* hh = ic.hists + (size_t)slot * nbins;
                    atomicAdd(&hh[e_bin], 1ull);
                    atomicAdd(&hh[p.n_ebins + a_bin], 1ull);
                }
                const unsigned long long ks = ITEMS ? (unsigned long long)rid.y * ic.n_per_item + rid.x - ic.g0
                                                    : prim - p.prim_offset - chunk_first;
                atomicAdd(&kcount[ks], 1u);
                r.es.hi = E;
                r.e2.hi = __fmul_rn(E, E);
                r.e2.lo = __fmaf_rn(E, E, -r.e2.hi);     // exact remainder of E^2
            } else if (tri < 0) {
                fate = RTMC_LOST;
                r.lost = 1;
            } else {
                const float4 w0 = ldg4(tris + 3ll * tri);
                orig = __float_as_int(w0.w);
                const float bw = 1.f - h.y - h.z;
                if (p.n_zbins > 0) {
                    // penetration depth: the flight of every ray that meets a facet ends there
                    const float z1 = ldg4(tris + 3ll * tri + 1).z, z2 = ldg4(tris + 3ll * tri + 2).z;
                    const float pz = bw * w0.z + h.y * z1 + h.z * z2;
                    const int z_bin = max(0, min((int)floorf((p.z_top - pz) * p.inv_zbin), p.n_zbins - 1));
                    if (!ITEMS) atomicAdd(&s_hist[zbase + z_bin], 1u);
                    else if (shared_items) atomicAdd(&s_hist[jslot * nbins + zbase + z_bin], 1u);
                    else atomicAdd(&ic.hists[(size_t)slot * nbins + zbase + z_bin], 1ull);
                }
                const bool emits = g == 0 || ((int)g < em.max_generation && E >= em.regen_min);
                if (!emits) {
                    if (E < em.absorb_min) { fate = RTMC_ABSORBED_LOW; r.low = 1; }
                    else { fate = RTMC_ABSORBED_OTHER; r.other = 1; }
                } else {
                    fate = RTMC_EMITTER;
                    r.emit = 1;
                    if (g > 0) r.regen = 1;
                    const float4 nr = ldg4(normals + tri);
                    const float cosa = -(b.x * nr.x + b.y * nr.y + b.z * nr.z);
                    const float alpha = acosf(fminf(1.f, cosa));
                    const uint4 w = ray_block(p.seed, (unsigned)prim, (unsigned)(prim >> 32), rid.z, pitem);
                    int capped;
                    if (em.model == RTMC_EMISSION_PAPER_FIT) {
                        const float a_deg = alpha * 57.295779513082321f;
                        kk = round_stochastic(gamma_fit(E, a_deg), u01(w.w), em.k_max, capped);
                        s_esee[tid] = fmaxf(esee_fit(E, a_deg), 0.f);
                    } else {
                        kk = poisson_inv(lookup_delta(tab, E, alpha), u01(w.w), em.k_max, capped);
                    }
                    r.capped = capped;
                    r.emitted = kk;
                    k = kk;
                    const float4 w1 = ldg4(tris + 3ll * tri + 1), w2 = ldg4(tris + 3ll * tri + 2);
                    s_px[tid] = bw * w0.x + h.y * w1.x + h.z * w2.x;
                    s_py[tid] = bw * w0.y + h.y * w1.y + h.z * w2.y;
                    s_pz[tid] = bw * w0.z + h.y * w1.z + h.z * w2.z;
                    s_nx[tid] = nr.x; s_ny[tid] = nr.y; s_nz[tid] = nr.z;
                    s_id[tid] = make_uint4(rid.x, rid.y, rid.z, g + 1);
                    s_key[tid] = make_uint3((unsigned)prim, (unsigned)(prim >> 32), pitem);
                    s_tri[tid] = tri;
                }
            }
            if (!ITEMS) acc.add(r);
            else if (!shared_items) acc_atomic(ic.tallies + slot, r);
            if (!ITEMS && (RECORD || prim_hash)) {
                const int wr = wraps_in ? wraps_in[i] : 0;
                if (prim_hash)
                    atomicAdd(&prim_hash[prim - p.prim_offset],
                              record_hash_fields(prim, rid.z, fate, orig, kk, e_bin, a_bin, wr));
                if (RECORD) {
                    const unsigned long long rs = atomicAdd(&tally->rays_recorded, 1ull);
                    if (rs < rec_cap) {
                        rtmc_record rec;
                        rec.prim = prim; rec.path = rid.z; rec.gen = (int)g; rec.fate = fate; rec.tri = orig;
                        rec.k = kk; rec.e_bin = e_bin; rec.a_bin = a_bin; rec.wraps = wr;
                        rec.t = (double)h.x; rec.energy = (double)E;
                        records[rs] = rec;
                    } else {
                        atomicOr(&tally->status, (unsigned long long)ST_RECORD_OVERFLOW);
                    }
                }
            }
        }
        if (ITEMS && shared_items) {
            // warps are almost always single-item: reduce the warp, one shared add per counter
            const int j0 = __shfl_sync(0xFFFFFFFFu, jslot, 0);
            if (__all_sync(0xFFFFFFFFu, jslot == j0 || jslot < 0) && j0 >= 0) {
                const unsigned cs[10] = {r.rays, r.esc, r.lost, r.low, r.other, r.emit, r.regen, r.emitted,
                                         r.capped, r.wraps};
#pragma unroll
                for (int c = 0; c < 10; ++c) {
                    const unsigned v = __reduce_add_sync(0xFFFFFFFFu, cs[c]);
                    if (lane == 0 && v) atomicAdd(&s_icnt[j0][c], v);
                }
                if (__any_sync(0xFFFFFFFFu, r.esc != 0u)) {
                    const FF es = ff_warp_sum(r.es), e2 = ff_warp_sum(r.e2);
                    if (lane == 0) {
                        // the warp's own slots: no atomics, and FP64 only once per item at the end
                        float* f = s_iff[warp][j0];
                        FF a, b;
                        a.hi = f[0]; a.lo = f[1]; b.hi = f[2]; b.lo = f[3];
                        a = ff_add(a, es);
                        b = ff_add(b, e2);
                        f[0] = a.hi; f[1] = a.lo; f[2] = b.hi; f[3] = b.lo;
                    }
                }
            } else if (jslot >= 0) {
                const unsigned cs[10] = {r.rays, r.esc, r.lost, r.low, r.other, r.emit, r.regen, r.emitted,
                                         r.capped, r.wraps};
#pragma unroll
                for (int c = 0; c < 10; ++c)
                    if (cs[c]) atomicAdd(&s_icnt[jslot][c], cs[c]);
                if (ff_nonzero(r.es)) {
                    atomicAdd(&s_isum[jslot][0], ff_double(r.es));
                    atomicAdd(&s_isum[jslot][1], ff_double(r.e2));
                }
            }
        }
        // block exclusive prefix of the daughter counts (warp shuffles + warp totals)
        unsigned incl = k;
        for (int off = 1; off < 32; off <<= 1) {
            const unsigned v = __shfl_up_sync(0xFFFFFFFFu, incl, off);
            if (lane >= off) incl += v;
        }
        if (lane == 31) s_warp[warp] = incl;
        // the barrier also tells whether the tile has any daughter: one without
        // (every tile of the last generation) skips the scan and the expansion
        if (!__syncthreads_or(k != 0u)) continue;
        if (warp == 0) {
            unsigned v = lane < kShadeThreads / 32 ? s_warp[lane] : 0u;
            for (int off = 1; off < 32; off <<= 1) {
                const unsigned u = __shfl_up_sync(0xFFFFFFFFu, v, off);
                if (lane >= off) v += u;
            }
            if (lane < kShadeThreads / 32) s_warp[lane] = v;     // inclusive warp totals
        }
        __syncthreads();
        const unsigned warp_off = warp ? s_warp[warp - 1] : 0u;
        s_excl[tid] = warp_off + incl - k;
        const unsigned total = s_warp[kShadeThreads / 32 - 1];
        if (tid == 0) {
            s_excl[kShadeThreads] = total;
            s_base = total ? atomicAdd(&ctl->count[gen + 1], total) : 0u;
        }
        __syncthreads();
        // expand: daughter slot s belongs to the last parent with excl <= s
        const unsigned base = s_base;
        for (unsigned s = tid; s < total; s += kShadeThreads) {
            int lo = 0, hi = kShadeThreads - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_excl[mid] <= s) lo = mid; else hi = mid - 1;
            }
            const int par = lo;
            const unsigned j = s - s_excl[par];
            const uint4 pid = s_id[par];
            const uint3 key = s_key[par];
            const unsigned path = pid.z * 16u + j;
            const uint4 w = ray_block(p.seed, key.x, key.y, path, key.z);
            float e, sb2 = u01(w.y);                  // energy; sin^2 of the polar angle
            if (em.model == RTMC_EMISSION_PAPER_FIT) {
                // pairs (0,1), (2,3), ... share xi = u1 of the pair's first daughter;
                // an unpaired daughter takes E_SEE at a cosine-law angle
                const unsigned kpar = s_excl[par + 1] - s_excl[par];
                const unsigned first = j & ~1u;
                const float esee = s_esee[par];
                e = esee;
                if (first + 1 < kpar) {
                    if (j & 1) {
                        const float xi = u01(ray_block(p.seed, key.x, key.y, pid.z * 16u + first, key.z).y);
                        e = (1.f - xi) * esee;        // cos^2(beta_1) E_SEE at beta_2 = pi/2 - beta_1
                        sb2 = 1.f - xi;
                    } else {
                        e = esee * sqrtf(sb2);        // E_SEE sqrt(xi) at beta_1 = asin(sqrt(xi))
                    }
                }
            } else {
                e = sample_energy(em, u01(w.x));
            }
            const float3 dd = cosine_dir(make_float3(s_nx[par], s_ny[par], s_nz[par]), sb2, u01(w.z));
            const unsigned slot = base + s;
            if (slot < out.cap) {
                out.oe[slot] = make_float4(s_px[par], s_py[par], s_pz[par], e);
                out.dt[slot] = make_float4(dd.x, dd.y, dd.z, __int_as_float(s_tri[par]));
                out.id[slot] = make_uint4(pid.x, pid.y, path, pid.w);
            } else {
                atomicOr(&tally->status, (unsigned long long)ST_QUEUE_OVERFLOW);
            }
        }
        __syncthreads();
    }
    if (!ITEMS) {
        flush();
    } else if (shared_items) {
        __syncthreads();
        for (int j = 0; j < (int)ic.n_items; ++j) {
            const int slot = ic.items[ic.it_lo + j].tally;
            Tally* t = ic.tallies + slot;
            if (tid < 10) {
                const unsigned v = s_icnt[j][tid];
                if (v) {
                    unsigned long long* dst[10] = {&t->rays, &t->escaped, &t->lost, &t->absorbed_low,
                                                   &t->absorbed_other, &t->emitters, &t->regenerated, &t->emitted,
                                                   &t->capped, &t->wraps};
                    atomicAdd(dst[tid], (unsigned long long)v);
                }
            } else if (tid == 32 || tid == 33) {
                double v = s_isum[j][tid - 32];
                for (int w = 0; w < kShadeThreads / 32; ++w) {
                    FF x;
                    x.hi = s_iff[w][j][2 * (tid - 32)];
                    x.lo = s_iff[w][j][2 * (tid - 32) + 1];
                    v += ff_double(x);
                }
                if (v != 0.0) atomicAdd(tid == 32 ? &t->e_sum : &t->e2_sum, v);
            }
            unsigned long long* hh = ic.hists + (size_t)slot * nbins;
            for (int b = tid; b < nbins; b += kShadeThreads)
                if (s_hist[j * nbins + b]) atomicAdd(&hh[b], (unsigned long long)s_hist[j * nbins + b]);
        }
    }
}

// --------------------------------------------------------------------------
// finalize: per-primary escape counts -> sum k, sum k^2; resets the counts
// --------------------------------------------------------------------------
__global__ void k_finalize(unsigned* __restrict__ kcount, unsigned n, Tally* __restrict__ tally)
{
    unsigned long long s1 = 0, s2 = 0;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const unsigned k = kcount[i];
        if (k) {
            s1 += k;
            s2 += (unsigned long long)k * k;
            kcount[i] = 0u;
        }
    }
    s1 = warp_sum(s1);
    s2 = warp_sum(s2);
    __shared__ unsigned long long r1[8], r2[8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) { r1[warp] = s1; r2[warp] = s2; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long a = 0, b = 0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) { a += r1[w]; b += r2[w]; }
        if (a) { atomicAdd(&tally->sum_k, a); atomicAdd(&tally->sum_k2, b); }
    }
}

// Multi-item finalize: per-block shared sums per item of the chunk (at most
// kChunkItems; wider chunks add per lane straight to global memory).
__global__ void k_finalize_items(unsigned* __restrict__ kcount, unsigned n, ItemCtx ic)
{
    __shared__ unsigned long long s_sum[kChunkItems][2];
    __shared__ unsigned s_end[kChunkItems];           // chunk-relative end of item it_lo + j
    const bool shared_items = ic.n_items <= (unsigned)kChunkItems;
    for (int b = threadIdx.x; b < kChunkItems * 2; b += blockDim.x) (&s_sum[0][0])[b] = 0ull;
    if (shared_items && threadIdx.x < ic.n_items) {
        const unsigned long long e = (unsigned long long)(ic.it_lo + threadIdx.x + 1) * ic.n_per_item - ic.g0;
        s_end[threadIdx.x] = (unsigned)min(e, (unsigned long long)n);
    }
    __syncthreads();
    const unsigned lane = threadIdx.x & 31;
    const unsigned stride = gridDim.x * blockDim.x;
    for (unsigned base = blockIdx.x * blockDim.x; base < n; base += stride) {   // warp-uniform trip count
        const unsigned i = base + threadIdx.x;
        unsigned k = 0;
        if (i < n) {
            k = kcount[i];
            if (k) kcount[i] = 0u;
        }
        if (shared_items) {
            unsigned j = 0;
            if (i < n) while (j + 1 < ic.n_items && i >= s_end[j]) ++j;
            const unsigned j0 = __shfl_sync(0xFFFFFFFFu, j, 0);
            if (__all_sync(0xFFFFFFFFu, j == j0 || i >= n)) {          // one item in this warp
                const unsigned s1 = __reduce_add_sync(0xFFFFFFFFu, k);
                const unsigned s2 = __reduce_add_sync(0xFFFFFFFFu, k * k);
                if (lane == 0 && s1) {
                    atomicAdd(&s_sum[j0][0], (unsigned long long)s1);
                    atomicAdd(&s_sum[j0][1], (unsigned long long)s2);
                }
            } else if (k) {
                atomicAdd(&s_sum[j][0], (unsigned long long)k);
                atomicAdd(&s_sum[j][1], (unsigned long long)k * k);
            }
        } else if (k) {
            const unsigned it = (unsigned)((ic.g0 + i) / ic.n_per_item);
            Tally* t = ic.tallies + ic.items[it].tally;
            atomicAdd(&t->sum_k, (unsigned long long)k);
            atomicAdd(&t->sum_k2, (unsigned long long)k * k);
        }
    }
    __syncthreads();
    if (shared_items && threadIdx.x < ic.n_items) {
        const unsigned j = threadIdx.x;
        if (s_sum[j][0]) {
            Tally* t = ic.tallies + ic.items[ic.it_lo + j].tally;
            atomicAdd(&t->sum_k, s_sum[j][0]);
            atomicAdd(&t->sum_k2, s_sum[j][1]);
        }
    }
}

// --------------------------------------------------------------------------
// test hooks
// --------------------------------------------------------------------------
// Streaming read of n float4, `passes` times over (bandwidth probe); the sum
// keeps the loads alive.  Several passes per launch keep launch overhead out
// of the L2-resident measurement.
__global__ void __launch_bounds__(256) k_read_probe(const float4* __restrict__ a, size_t n, int passes,
                                                    float* __restrict__ sink)
{
    float acc = 0.f;
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    for (int pass = 0; pass < passes; ++pass) {
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n; i += 4 * stride) {
        const float4 x = __ldcg(a + i), y = __ldcg(a + i + stride), z = __ldcg(a + i + 2 * stride),
                     w = __ldcg(a + i + 3 * stride);
        acc += x.x + x.y + x.z + x.w + y.x + y.y + y.z + y.w + z.x + z.y + z.z + z.w + w.x + w.y + w.z + w.w;
    }
    for (; i < n; i += stride) {
        const float4 x = __ldcg(a + i);
        acc += x.x + x.y + x.z + x.w;
    }
    }
    if (acc == 1234.5f) sink[0] = acc;   // never true for the zero-filled buffer
}

__global__ void k_philox(const uint4* __restrict__ ctr, int64_t n, unsigned long long key, uint4* __restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    out[i] = philox4x32_10(ctr[i], make_uint2((unsigned)key, (unsigned)(key >> 32)));
}

}  // namespace

// ----------------------------------------------------------------------------
// launchers
// ----------------------------------------------------------------------------
cudaError_t launch_generate(const RunParams& p, const Queues& q, int buf, unsigned long long first,
                            unsigned n, cudaStream_t s)
{
    const int tb = 256;
    const unsigned gb = n ? (n + tb - 1) / tb : 1;
    k_generate<<<gb, tb, 0, s>>>(p, p.sin_t, p.cos_t, first, n, q.oe[buf], q.dt[buf], q.id[buf], q.ctl);
    return cudaGetLastError();
}

cudaError_t launch_shade(const DeviceMesh& m, const RunParams& p, const TableDesc& tab, const Emission& em,
                         const Queues& q, int buf, int gen, unsigned long long chunk_first, int num_sms,
                         bool record, cudaStream_t s)
{
    const int nb = 1 - buf;
    const ShadeOut out{q.oe[nb], q.dt[nb], q.id[nb], q.cap[nb]};
    const size_t smem = (size_t)(p.n_ebins + p.n_abins + p.n_zbins) * sizeof(unsigned);
    const int blocks = num_sms * kShadeBlocksPerSm;
    const ItemCtx ic{};
    if (smem > kShadeDefaultSmem) {
        // up to 3 x 4096 bins: past the default dynamic shared-memory limit
        cudaError_t e = cudaFuncSetAttribute(record ? k_shade<true, false> : k_shade<false, false>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    if (record)
        k_shade<true, false><<<blocks, kShadeThreads, smem, s>>>(m.tris, m.normals, tab, em, p, ic, q.oe[buf],
                                                                 q.dt[buf], q.id[buf], q.hits, q.wraps, out, q.ctl,
                                                                 gen, q.cap[buf], q.tally, q.hist_e, q.hist_a,
                                                                 q.kcount, chunk_first, q.prim_hash, q.records,
                                                                 q.rec_cap);
    else
        k_shade<false, false><<<blocks, kShadeThreads, smem, s>>>(m.tris, m.normals, tab, em, p, ic, q.oe[buf],
                                                                  q.dt[buf], q.id[buf], q.hits,
                                                                  q.prim_hash ? q.wraps : nullptr, out, q.ctl, gen,
                                                                  q.cap[buf], q.tally, q.hist_e, q.hist_a, q.kcount,
                                                                  chunk_first, q.prim_hash, nullptr, 0);
    return cudaGetLastError();
}

template <bool ITEMS>
static cudaError_t generate_sorted(const RunParams& p, const ItemCtx& ic, const Queues& q,
                                   unsigned long long first, unsigned n, unsigned buckets, cudaStream_t s)
{
    const int tb = 256;
    const unsigned gb = n ? (n + tb - 1) / tb : 1;
    cudaError_t e = cudaMemsetAsync(q.sort_counts, 0, (size_t)buckets * 4, s);
    if (e == cudaSuccess && n) k_prim_count<ITEMS><<<gb, tb, 0, s>>>(p, ic, first, n, q.sort_counts);
    if (e == cudaSuccess) scan_exclusive(q.sort_counts, q.sort_counts, buckets, nullptr, q.sort_counts + buckets, s);
    // the hit records are idle until this chunk's first traversal: they hold the permutation
    unsigned* perm = reinterpret_cast<unsigned*>(q.hits);
    if (e == cudaSuccess && n) k_scatter_perm<ITEMS><<<gb, tb, 0, s>>>(p, ic, first, n, q.sort_counts, perm);
    if (e == cudaSuccess)
        k_generate_sorted<ITEMS><<<gb, tb, 0, s>>>(p, ic, first, n, perm, q.oe[0], q.dt[0], q.id[0], q.ctl);
    return e == cudaSuccess ? cudaGetLastError() : e;
}

cudaError_t launch_generate_sorted(const RunParams& p, const Queues& q, unsigned long long first, unsigned n,
                                   cudaStream_t s)
{
    return generate_sorted<false>(p, ItemCtx{}, q, first, n, kSortCells, s);
}

cudaError_t launch_generate_items_sorted(const RunParams& p, const ItemCtx& ic, const Queues& q, unsigned n,
                                         cudaStream_t s)
{
    return generate_sorted<true>(p, ic, q, 0ull, n, ic.n_items * kSortCells, s);
}

cudaError_t launch_generate_items(const RunParams& p, const ItemCtx& ic, const Queues& q, unsigned n,
                                  cudaStream_t s)
{
    const int tb = 256;
    const unsigned gb = n ? (n + tb - 1) / tb : 1;
    k_generate_items<<<gb, tb, 0, s>>>(p, ic, n, q.oe[0], q.dt[0], q.id[0], q.ctl);
    return cudaGetLastError();
}

cudaError_t launch_shade_items(const DeviceMesh& m, const RunParams& p, const TableDesc& tab, const Emission& em,
                               const ItemCtx& ic, const Queues& q, int buf, int gen, int num_sms, cudaStream_t s)
{
    const int nb = 1 - buf;
    const ShadeOut out{q.oe[nb], q.dt[nb], q.id[nb], q.cap[nb]};
    const size_t smem = (size_t)kChunkItems * (p.n_ebins + p.n_abins + p.n_zbins) * sizeof(unsigned);
    k_shade<false, true><<<num_sms * kShadeBlocksPerSm, kShadeThreads, smem, s>>>(m.tris, m.normals, tab, em, p, ic, q.oe[buf],
                                                                  q.dt[buf], q.id[buf], q.hits, q.wraps, out, q.ctl,
                                                                  gen, q.cap[buf], q.tally, nullptr, nullptr, q.kcount,
                                                                  0ull, nullptr, nullptr, 0);
    return cudaGetLastError();
}

cudaError_t launch_finalize_items(const ItemCtx& ic, const Queues& q, unsigned n, int num_sms, cudaStream_t s)
{
    int gb = (int)((n + 255) / 256);
    gb = std::max(1, std::min(gb, num_sms * 8));
    k_finalize_items<<<gb, 256, 0, s>>>(q.kcount, n, ic);
    return cudaGetLastError();
}

cudaError_t launch_finalize(const Queues& q, unsigned n, cudaStream_t s)
{
    const int tb = 256;
    int gb = (int)((n + tb - 1) / tb);
    if (gb > 4096) gb = 4096;
    if (gb < 1) gb = 1;
    k_finalize<<<gb, tb, 0, s>>>(q.kcount, n, q.tally);
    return cudaGetLastError();
}

cudaError_t launch_read_probe(const void* buf, size_t bytes, int passes, int num_sms, float* sink, cudaStream_t s)
{
    k_read_probe<<<num_sms * 8, 256, 0, s>>>(reinterpret_cast<const float4*>(buf), bytes / 16, passes, sink);
    return cudaGetLastError();
}

cudaError_t launch_philox(const uint32_t* ctr, int64_t n, unsigned long long key, uint32_t* out, cudaStream_t s)
{
    const int tb = 256;
    const int64_t gb = (n + tb - 1) / tb;
    if (gb > 0)
        k_philox<<<(unsigned)gb, tb, 0, s>>>(reinterpret_cast<const uint4*>(ctr), n, key,
                                             reinterpret_cast<uint4*>(out));
    return cudaGetLastError();
}

}  // namespace rtmc
