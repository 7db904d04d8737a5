// rtmc_device.cuh -- device-side building blocks of the RTMC path (sm_103a).
//
// Layouts in HBM (all 16-byte aligned, read with 128-bit loads):
//   BVH node (64 B): float4 a = (c0.lo.x, c0.hi.x, c0.lo.y, c0.hi.y)
//                    float4 b = (c1.lo.x, c1.hi.x, c1.lo.y, c1.hi.y)
//                    float4 c = (c0.lo.z, c0.hi.z, c1.lo.z, c1.hi.z)
//                    int4   d = (child0, child1, 0, 0); child >= 0: inner node,
//                               child < 0: leaf holding sorted triangle ~child.
//   Q8 node (32 B): float4 (frame origin xyz, packed: ex | ey << 8 | ez << 16 | meta << 24)
//                   uint4  (12 quantised bytes: c0 lo.xyz hi.xyz, c1 lo.xyz hi.xyz; gamma)
//                   a child coordinate decodes to fmaf(q, 2^e, origin) (outward rounded);
//                   children are gamma and gamma + 1: inner node indices, or leaves
//                   ending at gamma / starting at gamma + 1 (meta: leaf bit + count - 1).
//   triangle (48 B): float4 V0 (w = original id bits), float4 V1, float4 V2
//   normal   (16 B): float4 (unit normal, 0)
//   ray queue (SoA, 48 B per ray):
//     float4 o_e   = (ox, oy, oz, E)
//     float4 d_ot  = (dx, dy, dz, origin triangle as int bits; -1 = none)
//     uint4  id    = (prim lo, prim hi, path, generation)
//   hit (16 B): float4 (t, u, v, tri as int bits); tri >= 0 sorted triangle,
//               HIT_ESCAPE or HIT_LOST.
#pragma once
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

namespace rtmc {

constexpr int HIT_ESCAPE = -1;
constexpr int HIT_LOST = -2;
constexpr int kStackMax = 128;    // binary: depth <= 62 (30-bit codes + index); 4-wide: 3 entries per level

// device status word bits
constexpr unsigned ST_STACK_OVERFLOW = 1u;
constexpr unsigned ST_QUEUE_OVERFLOW = 2u;
constexpr unsigned ST_RECORD_OVERFLOW = 4u;
constexpr unsigned ST_LOOP_LIMIT = 8u;     // a traversal exceeded its iteration bound
constexpr unsigned ST_COLUMN = 16u;        // the column kernel got a ray not parallel to z
constexpr int kMaxVisits = 1 << 22;        // node visits per ray segment before giving up

struct Tally {                    // one (energy, angle) item, device resident
    unsigned long long rays, escaped, absorbed_low, absorbed_other, emitters, emitted,
        regenerated, capped, lost, wraps, sum_k, sum_k2;
    double e_sum, e2_sum;
    unsigned long long rays_recorded;
    unsigned long long status;    // ST_* bits raised by any kernel of the item
    unsigned long long node_visits, tri_tests;   // counting variant of traverse only
    unsigned long long retested;                 // rays with a facet decided in FP64
    unsigned long long col_rays;                 // rays traced through the column grid
};

struct Control {                  // per chunk
    unsigned int count[8];        // rays in queue of generation g
    unsigned int next[8];         // persistent-traversal work counter per generation
};

// One (energy, angle) item of a batched launch.
struct ItemDev {
    float energy, sin_t, cos_t;
    unsigned philox_item;            // Philox counter word 3
    unsigned long long prim_offset;  // global id of the item's primary 0
    int tally;                       // slot in the tally / histogram arrays
    int pad;
};

// Where the rays of a multi-item chunk come from: chunk-linear index g (from
// g0) is local primary g % n_per_item of item g / n_per_item.
struct ItemCtx {
    const ItemDev* items;
    unsigned long long n_per_item;
    unsigned long long g0;
    Tally* tallies;
    unsigned long long* hists;       // [slot][n_ebins + n_abins]
    unsigned it_lo, n_items;         // items this chunk touches: it_lo .. it_lo + n_items - 1
};

constexpr int kChunkItems = 16;      // per-block shared accumulators for up to this many items

// A column grid as the traversal kernels read it.  Rays of direction
// (dx, 0, dz), dz < 0, dx >= 0, enter through z_top; pixel p of the gx x gy grid
// over [0, lx) x [0, ly) lists ent[off[p] .. off[p+1]) = (facet | k << 24, top z
// bits), sorted by top z descending: the facets a ray entering in p can meet,
// with the lateral wraps k it makes before it meets them (k = 0 when dx = 0).
struct GridDev {
    const unsigned* off;
    const uint2* ent;
    int gx, gy;
    float iwx, iwy;
    float dx, dz;
};
constexpr unsigned kSlantFacetBits = 24;    // facet index bits of a grid entry; the wrap count sits above

struct Emission {
    float phi, e_cut, absorb_min, regen_min;
    int max_generation, k_max;
    float spec_norm;              // spectrum CDF at e_cut
    int model;                    // RTMC_EMISSION_TABLE or RTMC_EMISSION_PAPER_FIT
};

struct TableDesc {
    const float* delta;
    int n_e, n_theta;
    float inv_log_span;           // (n_e - 1) / ln(e_hi / e_lo)
    float log_e_lo;
    float inv_theta_step_deg;
};

constexpr int FMT_FP32 = 0;
constexpr int FMT_Q8 = 1;
constexpr int FMT_W4 = 2;         // 4-wide nodes, FP32 child boxes (128 B)
constexpr int FMT_Q4 = 3;         // 4-wide nodes, 8-bit child boxes (64 B)
// A 4-wide 8-bit node keeps its shifted frame origin (|o'| below 2^24 quanta)
// finite after the slab test multiplies it by 1/d: the quantum stays below
// 2^kQ4MaxExp and the traversal clamps |1/d| to 2^kQ4MaxInvExp.
constexpr int kQ4MaxExp = 40;
constexpr int kQ4MaxInvExp = 64;
constexpr int kEmptyChild = INT_MIN;   // unused slot of a 4-wide node (its box is never hit)

// Leaf reference used by both node formats: ~((first << 3) | (count - 1)).
__host__ __device__ inline int leaf_ref(int first, int count) { return ~((first << 3) | (count - 1)); }

// 2^e for e in [-126, 127] (a normal float built from its exponent field).
__device__ __forceinline__ float exp2_int(int e) { return __int_as_float((e + 127) << 23); }

// Byte q = byte k of w as the float 0x4B0000qq, i.e. 2^23 + q (exact).
__device__ __forceinline__ float byte_m(unsigned w, int k)
{
    return __int_as_float(__byte_perm(w, 0x4B000000u, (unsigned)k | 0x7540u));
}

// Byte q = byte k of w as the float 0x3F80qq00, i.e. 1 + q 2^-15 (exact).
__device__ __forceinline__ float byte_f(unsigned w, int k)
{
    return __int_as_float(__byte_perm(w, 0x3F800000u, 0x7604u | ((unsigned)k << 4)));
}

// --------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11).  Counter (prim lo, prim hi, path,
// item), key (seed lo, seed hi); uniforms ((w >> 9) + 0.5) 2^-23, which are
// exact in FP32.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        if (r) { k.x += 0x9E3779B9u; k.y += 0xBB67AE85u; }
        const unsigned hi0 = __umulhi(0xD2511F53u, c.x), lo0 = 0xD2511F53u * c.x;
        const unsigned hi1 = __umulhi(0xCD9E8D57u, c.z), lo1 = 0xCD9E8D57u * c.z;
        c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
    }
    return c;
}

__device__ __forceinline__ float u01(unsigned w)
{
    return (float)(w >> 9) * 1.1920928955078125e-07f + 5.9604644775390625e-08f;
}

__device__ __forceinline__ uint4 ray_block(unsigned long long seed, unsigned prim_lo,
                                           unsigned prim_hi, unsigned path, unsigned item)
{
    return philox4x32_10(make_uint4(prim_lo, prim_hi, path, item),
                         make_uint2((unsigned)seed, (unsigned)(seed >> 32)));
}

// --------------------------------------------------------------------------
// small vector helpers
// --------------------------------------------------------------------------
__device__ __forceinline__ float3 f3(float4 v) { return make_float3(v.x, v.y, v.z); }
__device__ __forceinline__ float3 operator-(float3 a, float3 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// The facet test's arithmetic with its rounding spelled out (one product, then
// fused multiply-adds, in a fixed order): every kernel that inlines the test
// rounds alike, so a ray through an edge shared by two facets gets the same
// decision whichever traversal tests it.
__device__ __forceinline__ float dot3_fixed(float3 a, float3 b)
{
    return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}
__device__ __forceinline__ float cross2_fixed(float a, float b, float c, float d)   // a b - c d
{
    return __fmaf_rn(a, b, -__fmul_rn(c, d));
}

__host__ __device__ inline unsigned long long splitmix64(unsigned long long x)
{
    unsigned long long z = x + 0x9E3779B97F4A7C15ull;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// Hash of one ray's integer event record; a primary's hash is the sum over its rays.
__host__ __device__ inline unsigned long long record_hash_fields(
    unsigned long long prim, unsigned path, int fate, int tri, int k, int e_bin, int a_bin, int wraps)
{
    unsigned long long h = splitmix64(prim);
    h = splitmix64(h ^ ((unsigned long long)path | ((unsigned long long)(unsigned)fate << 32)));
    h = splitmix64(h ^ ((unsigned long long)(unsigned)tri | ((unsigned long long)(unsigned)k << 32)));
    h = splitmix64(h ^ ((unsigned long long)(unsigned)e_bin | ((unsigned long long)(unsigned)a_bin << 32)));
    h = splitmix64(h ^ (unsigned long long)(unsigned)wraps);
    return h;
}

// --------------------------------------------------------------------------
// Per-ray set-up of the watertight test (Woop, Benthin, Wald, JCGT 2013):
// the ray is sheared onto +z; rows of that shear are kept as three vectors so
// no per-triangle index selects are needed.
// --------------------------------------------------------------------------
struct RaySetup {
    float3 o;
    float3 mx, my, mz;       // shear rows: e_kx - Sx e_kz, e_ky - Sy e_kz, Sz e_kz
    float3 inv;              // reciprocal direction for slab tests (zeros replaced)
};

__device__ __forceinline__ float3 axis_vec(int k, float s)
{
    return make_float3(k == 0 ? s : 0.f, k == 1 ? s : 0.f, k == 2 ? s : 0.f);
}

__device__ __forceinline__ RaySetup setup_ray(float3 o, float3 d)
{
    RaySetup r;
    r.o = o;
    const float ax = fabsf(d.x), ay = fabsf(d.y), az = fabsf(d.z);
    int kz = 0;
    if (ay > ax) kz = 1;
    if (az > fmaxf(ax, ay)) kz = 2;
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    const float dkz = kz == 0 ? d.x : (kz == 1 ? d.y : d.z);
    if (dkz < 0.f) { const int t = kx; kx = ky; ky = t; }
    const float dkx = kx == 0 ? d.x : (kx == 1 ? d.y : d.z);
    const float dky = ky == 0 ? d.x : (ky == 1 ? d.y : d.z);
    const float sx = dkx / dkz, sy = dky / dkz, sz = 1.0f / dkz;
    const float3 ex = axis_vec(kx, 1.f), ey = axis_vec(ky, 1.f), ez = axis_vec(kz, 1.f);
    r.mx = make_float3(ex.x - sx * ez.x, ex.y - sx * ez.y, ex.z - sx * ez.z);
    r.my = make_float3(ey.x - sy * ez.x, ey.y - sy * ez.y, ey.z - sy * ez.z);
    r.mz = make_float3(sz * ez.x, sz * ez.y, sz * ez.z);
    const float tiny = 1e-30f;
    r.inv = make_float3(1.0f / (fabsf(d.x) > tiny ? d.x : copysignf(tiny, d.x)),
                        1.0f / (fabsf(d.y) > tiny ? d.y : copysignf(tiny, d.y)),
                        1.0f / (fabsf(d.z) > tiny ? d.z : copysignf(tiny, d.z)));
    return r;
}

// Watertight FP32 test, front faces only.  On a hit with t < *t_best (or a
// tie broken towards the lower original id) updates t_best/u/v and returns true.
__device__ __forceinline__ bool intersect_tri(const RaySetup& r, float4 w0, float4 w1, float4 w2,
                                              float& t_best, int& best_orig, float& bu, float& bv)
{
    const float3 A = f3(w0) - r.o, B = f3(w1) - r.o, C = f3(w2) - r.o;
    const float ax = dot3_fixed(A, r.mx), ay = dot3_fixed(A, r.my);
    const float bx = dot3_fixed(B, r.mx), by = dot3_fixed(B, r.my);
    const float cx = dot3_fixed(C, r.mx), cy = dot3_fixed(C, r.my);
    float U = cross2_fixed(cx, by, cy, bx);
    float V = cross2_fixed(ax, cy, ay, cx);
    float W = cross2_fixed(bx, ay, by, ax);
    if (U == 0.f || V == 0.f || W == 0.f) {            // exact edge: decide in FP64
        U = (float)((double)cx * (double)by - (double)cy * (double)bx);
        V = (float)((double)ax * (double)cy - (double)ay * (double)cx);
        W = (float)((double)bx * (double)ay - (double)by * (double)ax);
    }
    if (U < 0.f || V < 0.f || W < 0.f) return false;   // outside or back-facing
    const float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.f) return false;
    const float az = dot3_fixed(A, r.mz), bz = dot3_fixed(B, r.mz), cz = dot3_fixed(C, r.mz);
    const float T = __fmaf_rn(W, cz, __fmaf_rn(V, bz, __fmul_rn(U, az)));
    if (T <= 0.f) return false;
    const float t = T / det;
    const int orig = __float_as_int(w0.w);
    if (t < t_best || (t == t_best && orig < best_orig)) {
        t_best = t;
        best_orig = orig;
        bu = V / det;
        bv = W / det;
        return true;
    }
    return false;
}

}  // namespace rtmc
