// rtmc_traverse.cu -- ray traversal of the wavefront RTMC loop (sm_103a):
// closest front-facing facet through the BVH (FP32 or Q8 nodes) with the
// periodic cell walk, the FP64 re-test of flagged hits, and the closest-hit
// query hook.  Section 2.1 of the paper (the four checks of the element scan)
// and Section 2.2, last paragraph (periodic x/y, escape through z_max).
#include <cuda_runtime.h>

#include <algorithm>
#include <climits>
#include <cstdint>

#include "rtmc_internal.h"

namespace rtmc {
namespace {

constexpr int kSmemStack = 16;        // default stack entries held in shared memory per ray
constexpr float kRobust = 1.0000004f; // 1 + 2 gamma_3 (Ize 2013): conservative slab test
// Boxes are culled against the best facet distance widened by 2^-16: the FP32
// facet test rounds too, and a box whose facet would tie the best FP32 distance
// (met on a shared edge) must still be entered so the tie goes to the lower id.
constexpr float kTieSlack = 1.0000152587890625f;

__device__ __forceinline__ float4 ldg4(const float4* p) { return __ldg(p); }

// One 256-bit read-only load (sm_100+ `ld.global.nc.v8`); p must be 32-byte aligned.
// Node fetches use it so a 64-byte node costs two L1 requests instead of four.
__device__ __forceinline__ void ldg8(const void* p, float4& a, float4& b)
{
    asm("ld.global.nc.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
        : "=f"(a.x), "=f"(a.y), "=f"(a.z), "=f"(a.w), "=f"(b.x), "=f"(b.y), "=f"(b.z), "=f"(b.w)
        : "l"(p));
}

// --------------------------------------------------------------------------
// traverse: BVH closest hit in one cell + periodic walk
// --------------------------------------------------------------------------
struct StackRef {
    int2* smem;       // [kSmemStack][blockDim]
    int stride;
    int tid;
};

// Distance bound before any hit: finite, so that tmax = min(.., t_best) stays
// finite and a box whose entry distance is +inf -- the empty slot of a 4-wide
// node, [+inf, +inf]^3 -- is never hit.  Every real slab distance is far below
// it (box coordinates are finite and |1/d| <= 1e30).
constexpr float kNoHit = 1e37f;

// Slab test of one box (Ize 2013 form: difference first, then the reciprocal,
// tmax widened by 1 + 2 gamma_3 so the test is conservative).
__device__ __forceinline__ void slab_box(float lox, float hix, float loy, float hiy, float loz, float hiz,
                                         const RaySetup& r, float t_best, float& tmin, bool& hit)
{
    const float lx = (lox - r.o.x) * r.inv.x, hx = (hix - r.o.x) * r.inv.x;
    const float ly = (loy - r.o.y) * r.inv.y, hy = (hiy - r.o.y) * r.inv.y;
    const float lz = (loz - r.o.z) * r.inv.z, hz = (hiz - r.o.z) * r.inv.z;
    tmin = fmaxf(fmaxf(fminf(lx, hx), fminf(ly, hy)), fmaxf(fminf(lz, hz), 0.f));
    const float tmax = fminf(fminf(fmaxf(lx, hx), fmaxf(ly, hy)), fminf(fmaxf(lz, hz), t_best));
    hit = tmin <= tmax * kRobust;
}

// Fetch node `node` and test its two child boxes; c0/c1 get the child refs
// (inner node index >= 0 or leaf_ref(first, count) < 0).
template <int FMT>
__device__ __forceinline__ void node_children(const void* __restrict__ nodes, int node, const RaySetup& r,
                                              float t_best, float& tmin0, float& tmin1, bool& h0, bool& h1,
                                              int& c0, int& c1)
{
    if (FMT == FMT_FP32) {
        const float4* np = reinterpret_cast<const float4*>(nodes) + 4ll * node;
        float4 n0, n1, n2, n3;
        ldg8(np, n0, n1);
        ldg8(np + 2, n2, n3);
        slab_box(n0.x, n0.y, n0.z, n0.w, n2.x, n2.y, r, t_best, tmin0, h0);
        slab_box(n1.x, n1.y, n1.z, n1.w, n2.z, n2.w, r, t_best, tmin1, h1);
        c0 = __float_as_int(n3.x);
        c1 = __float_as_int(n3.y);
    } else {
        const uint4* np = reinterpret_cast<const uint4*>(nodes) + 2ll * node;
        float4 f0, f1;
        ldg8(np, f0, f1);
        const uint4 w0 = make_uint4(__float_as_uint(f0.x), __float_as_uint(f0.y), __float_as_uint(f0.z),
                                    __float_as_uint(f0.w));
        const uint4 w1 = make_uint4(__float_as_uint(f1.x), __float_as_uint(f1.y), __float_as_uint(f1.z),
                                    __float_as_uint(f1.w));
        // shifted frame origin o', scales 2^e from biased exponent bytes; a bound
        // decodes as fmaf(M(q), s, o') with M(q) the float 0x4B0000qq = 2^23 + q
        const float ox = __uint_as_float(w0.x), oy = __uint_as_float(w0.y), oz = __uint_as_float(w0.z);
        const unsigned pk = w0.w;
        const float sx = __uint_as_float((pk << 23) & 0x7F800000u);
        const float sy = __uint_as_float((pk << 15) & 0x7F800000u);
        const float sz = __uint_as_float((pk << 7) & 0x7F800000u);
        const unsigned meta = pk >> 24;
        slab_box(fmaf(byte_m(w1.x, 0), sx, ox), fmaf(byte_m(w1.x, 3), sx, ox),
                 fmaf(byte_m(w1.x, 1), sy, oy), fmaf(byte_m(w1.y, 0), sy, oy),
                 fmaf(byte_m(w1.x, 2), sz, oz), fmaf(byte_m(w1.y, 1), sz, oz), r, t_best, tmin0, h0);
        slab_box(fmaf(byte_m(w1.y, 2), sx, ox), fmaf(byte_m(w1.z, 1), sx, ox),
                 fmaf(byte_m(w1.y, 3), sy, oy), fmaf(byte_m(w1.z, 2), sy, oy),
                 fmaf(byte_m(w1.z, 0), sz, oz), fmaf(byte_m(w1.z, 3), sz, oz), r, t_best, tmin1, h1);
        const int g = (int)w1.w;
        c0 = (meta & 1u) ? leaf_ref(g - (int)((meta >> 1) & 7u), (int)((meta >> 1) & 7u) + 1) : g;
        c1 = (meta & 16u) ? leaf_ref(g + 1, (int)((meta >> 5) & 7u) + 1) : g + 1;
    }
}

// Slab test of a 4-wide child with the planes already ordered per axis (near
// first), one FMA per plane: t = fmaf(plane, inv, -o * inv).  The product
// plane * inv is exact inside the FMA; the rounding of o * inv moves a plane
// by at most |o| 2^-24, and 4-wide boxes are stored widened outward by
// M 2^-22 (M the largest cell coordinate), so the planes tested still enclose
// the exact box.  The reciprocal and the FMA's own rounding are covered, as
// in slab_box, by widening tmax by 1 + 2 gamma_3.  Rounding is monotonic, so
// the near plane stays the nearer.
__device__ __forceinline__ void slab_near_far(float nxp, float fxp, float nyp, float fyp, float nzp, float fzp,
                                              const RaySetup& r, float3 oi, float t_best, float& tmin, bool& hit)
{
    const float nx = fmaf(nxp, r.inv.x, -oi.x), fx = fmaf(fxp, r.inv.x, -oi.x);
    const float ny = fmaf(nyp, r.inv.y, -oi.y), fy = fmaf(fyp, r.inv.y, -oi.y);
    const float nz = fmaf(nzp, r.inv.z, -oi.z), fz = fmaf(fzp, r.inv.z, -oi.z);
    tmin = fmaxf(fmaxf(nx, ny), fmaxf(nz, 0.f));
    const float tmax = fminf(fminf(fx, fy), fminf(fz, t_best));
    hit = tmin <= tmax * kRobust;
}

// 4-wide node (128 B): rows lo.x, hi.x, lo.y, hi.y, lo.z, hi.z of the four
// child boxes, then the four child refs.  The 8-bit form (64 B) holds per
// axis a frame origin o' and a scale S = 2^15 s, then the same six rows as one
// code byte per child, then the refs.  The hit children come back sorted by
// entry distance (nearest first); *nh is their number.  An empty slot holds
// the box [+inf, +inf]^3 (FP32) or the codes lo 255, hi 0 (8-bit), never hit.
template <int FMT>
__device__ __forceinline__ void node4_children(const void* __restrict__ nodes, int node, const RaySetup& r,
                                               float t_best, float (&tk)[4], int (&ck)[4], int& nh)
{
    bool h0, h1, h2, h3;
    if constexpr (FMT == FMT_Q4) {
        // Plane (m + q) s evaluated as fmaf(1 + q 2^-15, S / d, (o' - o) / d)
        // with S = 2^15 s and o' = (m - 2^15) s: one FMA per plane on the code
        // byte made a float by __byte_perm.  The codes are rounded outward far
        // enough to cover the rounding of (o' - o) / d (see the quantiser); the
        // near row of each axis is chosen by the sign of the direction, as for
        // FP32 nodes.
        const float4* np = reinterpret_cast<const float4*>(nodes) + 4ll * node;
        float4 a, b, c, cr;
        ldg8(np, a, b);                          // o'.xyz, S.x | S.y, S.z, row lo.x, row hi.x
        ldg8(np + 2, c, cr);                     // rows lo.y, hi.y, lo.z, hi.z | refs
        const float kx = a.w * r.inv.x, ky = b.x * r.inv.y, kz = b.y * r.inv.z;
        const float ox = (a.x - r.o.x) * r.inv.x, oy = (a.y - r.o.y) * r.inv.y, oz = (a.z - r.o.z) * r.inv.z;
        const unsigned lx = __float_as_uint(b.z), hx = __float_as_uint(b.w);
        const unsigned ly = __float_as_uint(c.x), hy = __float_as_uint(c.y);
        const unsigned lz = __float_as_uint(c.z), hz = __float_as_uint(c.w);
        const bool gx = r.inv.x < 0.f, gy = r.inv.y < 0.f, gz = r.inv.z < 0.f;
        const unsigned nxw = gx ? hx : lx, fxw = gx ? lx : hx;
        const unsigned nyw = gy ? hy : ly, fyw = gy ? ly : hy;
        const unsigned nzw = gz ? hz : lz, fzw = gz ? lz : hz;
        ck[0] = __float_as_int(cr.x); ck[1] = __float_as_int(cr.y);
        ck[2] = __float_as_int(cr.z); ck[3] = __float_as_int(cr.w);
        auto child = [&](int j, float& tmin, bool& hit) {
            const float tnx = fmaf(byte_f(nxw, j), kx, ox), tfx = fmaf(byte_f(fxw, j), kx, ox);
            const float tny = fmaf(byte_f(nyw, j), ky, oy), tfy = fmaf(byte_f(fyw, j), ky, oy);
            const float tnz = fmaf(byte_f(nzw, j), kz, oz), tfz = fmaf(byte_f(fzw, j), kz, oz);
            tmin = fmaxf(fmaxf(tnx, tny), fmaxf(tnz, 0.f));
            const float tmax = fminf(fminf(tfx, tfy), fminf(tfz, t_best));
            hit = tmin <= tmax * kRobust;
        };
        child(0, tk[0], h0);
        child(1, tk[1], h1);
        child(2, tk[2], h2);
        child(3, tk[3], h3);
        // an empty slot (codes lo 255, hi 0) is never hit: its near plane lies beyond its far
        // plane along the ray whatever the direction's sign, also where both saturate to +-inf
    } else {
        // Per axis the lane loads the near row first (lo when the direction is
        // positive, hi when negative), so (near - o) * inv <= (far - o) * inv and no
        // min / max is needed to order the two planes: the same values as the
        // two-plane slab test, three more loads, 24 fewer ALU operations.
        const float4* np = reinterpret_cast<const float4*>(nodes) + 8ll * node;
        const int sx = (int)(__float_as_uint(r.inv.x) >> 31), sy = (int)(__float_as_uint(r.inv.y) >> 31),
                  sz = (int)(__float_as_uint(r.inv.z) >> 31);
        const float4 nx = ldg4(np + sx), fx = ldg4(np + 1 - sx);
        const float4 ny = ldg4(np + 2 + sy), fy = ldg4(np + 3 - sy);
        const float4 nz = ldg4(np + 4 + sz), fz = ldg4(np + 5 - sz);
        const float4 cr = ldg4(np + 6);
        const float3 oi = make_float3(r.o.x * r.inv.x, r.o.y * r.inv.y, r.o.z * r.inv.z);
        slab_near_far(nx.x, fx.x, ny.x, fy.x, nz.x, fz.x, r, oi, t_best, tk[0], h0);
        slab_near_far(nx.y, fx.y, ny.y, fy.y, nz.y, fz.y, r, oi, t_best, tk[1], h1);
        slab_near_far(nx.z, fx.z, ny.z, fy.z, nz.z, fz.z, r, oi, t_best, tk[2], h2);
        slab_near_far(nx.w, fx.w, ny.w, fy.w, nz.w, fz.w, r, oi, t_best, tk[3], h3);
        ck[0] = __float_as_int(cr.x); ck[1] = __float_as_int(cr.y);
        ck[2] = __float_as_int(cr.z); ck[3] = __float_as_int(cr.w);
    }
    if (!h0) tk[0] = INFINITY;
    if (!h1) tk[1] = INFINITY;
    if (!h2) tk[2] = INFINITY;
    if (!h3) tk[3] = INFINITY;
    nh = (int)h0 + (int)h1 + (int)h2 + (int)h3;
    auto cswap = [&](int a, int b) {
        if (tk[b] < tk[a]) {
            const float t = tk[a]; tk[a] = tk[b]; tk[b] = t;
            const int c = ck[a]; ck[a] = ck[b]; ck[b] = c;
        }
    };
    cswap(0, 1); cswap(2, 3); cswap(0, 2); cswap(1, 3); cswap(1, 2);
}

// The 8-bit 4-wide nodes multiply their shifted origin by 1/d: |1/d| is
// clamped to 2^kQ4MaxInvExp there so the product stays finite.  Only a
// direction component below 2^-64 in magnitude (in practice an exact zero,
// whose 1/d the ray set-up makes 1e30) changes, and for it any magnitude this
// large keeps each slab either all-pass or all-miss.
__device__ __forceinline__ RaySetup q4_setup(RaySetup r)
{
    const float lim = 0x1p64f;
    r.inv = make_float3(fminf(fmaxf(r.inv.x, -lim), lim), fminf(fmaxf(r.inv.y, -lim), lim),
                        fminf(fmaxf(r.inv.z, -lim), lim));
    return r;
}

struct Counts { unsigned visits = 0, tests = 0; };

// FP64 form of the watertight test on the same (FP32-valued) ray: used to
// re-test hits the FP32 pass flags as near an edge or grazing.
struct RaySetup64 {
    double ox, oy, oz;
    int kx, ky, kz;
    double sx, sy, sz;
};

__device__ __forceinline__ RaySetup64 setup_ray64(float3 o, float3 d)
{
    RaySetup64 r;
    r.ox = o.x; r.oy = o.y; r.oz = o.z;
    const double dv[3] = {d.x, d.y, d.z};
    int kz = 0;
    if (fabs(dv[1]) > fabs(dv[kz])) kz = 1;
    if (fabs(dv[2]) > fabs(dv[kz])) kz = 2;
    int kx = kz == 2 ? 0 : kz + 1;
    int ky = kx == 2 ? 0 : kx + 1;
    if (dv[kz] < 0.0) { const int t = kx; kx = ky; ky = t; }
    r.kx = kx; r.ky = ky; r.kz = kz;
    r.sx = dv[kx] / dv[kz];
    r.sy = dv[ky] / dv[kz];
    r.sz = 1.0 / dv[kz];
    return r;
}

__device__ __forceinline__ double comp(double x, double y, double z, int k) { return k == 0 ? x : (k == 1 ? y : z); }

__device__ __forceinline__ bool intersect_tri64(const RaySetup64& r, float4 w0, float4 w1, float4 w2, double& t_best,
                                                int& best_orig, float& bu, float& bv)
{
    const double a0 = w0.x - r.ox, a1 = w0.y - r.oy, a2 = w0.z - r.oz;
    const double b0 = w1.x - r.ox, b1 = w1.y - r.oy, b2 = w1.z - r.oz;
    const double c0 = w2.x - r.ox, c1 = w2.y - r.oy, c2 = w2.z - r.oz;
    const double akz = comp(a0, a1, a2, r.kz), bkz = comp(b0, b1, b2, r.kz), ckz = comp(c0, c1, c2, r.kz);
    const double ax = comp(a0, a1, a2, r.kx) - r.sx * akz, ay = comp(a0, a1, a2, r.ky) - r.sy * akz;
    const double bx = comp(b0, b1, b2, r.kx) - r.sx * bkz, by = comp(b0, b1, b2, r.ky) - r.sy * bkz;
    const double cx = comp(c0, c1, c2, r.kx) - r.sx * ckz, cy = comp(c0, c1, c2, r.ky) - r.sy * ckz;
    const double U = cx * by - cy * bx, V = ax * cy - ay * cx, W = bx * ay - by * ax;
    if (U < 0.0 || V < 0.0 || W < 0.0) return false;
    const double det = U + V + W;
    if (det == 0.0) return false;
    const double T = U * (r.sz * akz) + V * (r.sz * bkz) + W * (r.sz * ckz);
    if (T <= 0.0) return false;
    if (T > t_best * det * (1.0 + 1e-12)) return false;     // cannot beat the best hit (det > 0)
    const double t = T / det;                               // divisions only for candidates
    const int orig = __float_as_int(w0.w);
    if (t < t_best || (t == t_best && orig < best_orig)) {
        t_best = t;
        best_orig = orig;
        const double inv = 1.0 / det;
        bu = (float)(V * inv);
        bv = (float)(W * inv);
        return true;
    }
    return false;
}

// Test the triangles of a leaf ref.
template <bool COUNT, bool TRI64>
__device__ __forceinline__ void test_leaf(const float4* __restrict__ tris, const RaySetup& r, const RaySetup64& r64,
                                          int code, int skip, float& t_best, double& t_best64, int& best,
                                          int& best_orig, float& bu, float& bv, Counts* cnt)
{
    const int v = ~code;
    const int first = v >> 3, count = (v & 7) + 1;
    for (int k = 0; k < count; ++k) {
        const int j = first + k;
        if (j == skip) continue;
        if (COUNT) ++cnt->tests;
        const float4* tp = tris + 3ll * j;
        if (TRI64) {
            if (intersect_tri64(r64, ldg4(tp), ldg4(tp + 1), ldg4(tp + 2), t_best64, best_orig, bu, bv)) {
                best = j;
                t_best = (float)t_best64;
            }
        } else {
            if (intersect_tri(r, ldg4(tp), ldg4(tp + 1), ldg4(tp + 2), t_best, best_orig, bu, bv)) best = j;
        }
    }
}

// Closest front-facing triangle (leaf order index) with t > 0, skipping
// `skip`: one ray per lane, leaves tested as soon as their box is hit.
// SMEM: stack entries per ray held in shared memory (the rest in local memory).
template <int FMT, bool COUNT = false, bool TRI64 = false, int SMEM = kSmemStack>
__device__ __forceinline__ int bvh_closest(const void* __restrict__ nodes, const float4* __restrict__ tris,
                                           const RaySetup& r, const RaySetup64& r64, int skip, StackRef st,
                                           float& t_best, float& bu, float& bv, unsigned& status, int max_iter,
                                           Counts* cnt = nullptr)
{
    int2 lstack[kStackMax - SMEM];
    int sp = 0;
    int node = 0;
    int best = -1, best_orig = INT_MAX;
    double t_best64 = INFINITY;
    t_best = kNoHit;
    bu = bv = 0.f;
    auto push = [&](int ref, float tmin) {
        const int2 e = make_int2(ref, __float_as_int(tmin));
        if (sp < SMEM) st.smem[sp * st.stride + st.tid] = e;
        else if (sp < kStackMax) lstack[sp - SMEM] = e;
        else { status |= ST_STACK_OVERFLOW; sp = kStackMax - 1; }
        ++sp;
    };
    auto pop = [&]() -> bool {
        while (sp > 0) {
            --sp;
            const int2 e = sp < SMEM ? st.smem[sp * st.stride + st.tid] : lstack[sp - SMEM];
            if (__int_as_float(e.y) <= t_best * kTieSlack * kRobust) { node = e.x; return true; }
        }
        return false;
    };
    for (int visits = 0;; ++visits) {
        if (visits >= max_iter) { status |= ST_LOOP_LIMIT; break; }
        if constexpr (FMT == FMT_W4 || FMT == FMT_Q4) {
            if (node < 0) {                                  // a leaf: test it now
                test_leaf<COUNT, TRI64>(tris, r, r64, node, skip, t_best, t_best64, best, best_orig, bu, bv, cnt);
                if (!pop()) break;
                continue;
            }
            if (COUNT) ++cnt->visits;
            float tk[4];
            int ck[4], nh;
            node4_children<FMT>(nodes, node, FMT == FMT_Q4 ? q4_setup(r) : r, t_best * kTieSlack, tk, ck, nh);
            if (nh > 3) push(ck[3], tk[3]);
            if (nh > 2) push(ck[2], tk[2]);
            if (nh > 1) push(ck[1], tk[1]);
            if (nh > 0) node = ck[0];
            else if (!pop()) break;
            continue;
        }
        if (COUNT) ++cnt->visits;
        float tmin0, tmin1;
        bool h0, h1;
        int c0, c1;
        node_children<FMT>(nodes, node, r, t_best * kTieSlack, tmin0, tmin1, h0, h1, c0, c1);
        if (h0 && c0 < 0) {
            test_leaf<COUNT, TRI64>(tris, r, r64, c0, skip, t_best, t_best64, best, best_orig, bu, bv, cnt);
            h0 = false;
        }
        if (h1 && c1 < 0) {
            test_leaf<COUNT, TRI64>(tris, r, r64, c1, skip, t_best, t_best64, best, best_orig, bu, bv, cnt);
            h1 = false;
        }
        if (h0 && h1) {
            int near = c0, far = c1;
            float tfar = tmin1;
            if (tmin1 < tmin0) { near = c1; far = c0; tfar = tmin0; }
            const int2 e = make_int2(far, __float_as_int(tfar));
            if (sp < SMEM) st.smem[sp * st.stride + st.tid] = e;
            else if (sp < kStackMax) lstack[sp - SMEM] = e;
            else { status |= ST_STACK_OVERFLOW; sp = kStackMax - 1; }
            ++sp;
            node = near;
            continue;
        }
        if (h0) { node = c0; continue; }
        if (h1) { node = c1; continue; }
        bool found = false;
        while (sp > 0) {
            --sp;
            const int2 e = sp < SMEM ? st.smem[sp * st.stride + st.tid] : lstack[sp - SMEM];
            if (__int_as_float(e.y) <= t_best * kTieSlack * kRobust) { node = e.x; found = true; break; }
        }
        if (!found) break;
    }
    if (TRI64 && best >= 0) t_best = (float)t_best64;
    return best;
}

struct Cell {
    float lx, ly, z_min, z_top;
    int max_wraps;
    float eps;      // 2^-20 M, M the largest cell coordinate: bound on FP32 face-distance errors
    int max_visits; // inner-node visits of one cell traversal before the ray is abandoned (ST_LOOP_LIMIT)
};

// A ray that meets no facet in the cell leaves it through a face (reading R4).
// The distances to the three faces ahead are estimated in FP32 from the FP32
// origin o (slab reciprocals inv); they pick the face unless the two nearest
// lie closer than the estimates' error bound (2^-20 M per unit of |1/d|, plus
// 1e-5 relative), when the FP64 quotients from the FP64 origin (ox, oy, oz)
// decide (the reference rule: z first if strictly nearest, then x on a tie
// with y).  An exit through z_top or z_min returns HIT_ESCAPE / HIT_LOST with
// its distance from the FP64 offset in tout; so does a wrap past max_wraps
// (HIT_LOST).  A lateral wrap returns 0 with the FP64 re-entry point, the same
// FP64 quotient as the reference, in (ox, oy, oz) and one more in wraps.  (FP64
// is slow on this GPU; most daughters leave a cell at least once.)
__device__ __forceinline__ int cell_exit(float3 o, float3 d, float3 inv, const Cell& cell, double& ox, double& oy,
                                         double& oz, int& wraps, float& tout)
{
    const float ax = fabsf(inv.x), ay = fabsf(inv.y), az = fabsf(inv.z);
    const float fx = d.x != 0.f ? (d.x > 0.f ? cell.lx - o.x : o.x) * ax : INFINITY;
    const float fy = d.y != 0.f ? (d.y > 0.f ? cell.ly - o.y : o.y) * ay : INFINITY;
    const float fz = d.z != 0.f ? (d.z > 0.f ? cell.z_top - o.z : o.z - cell.z_min) * az : INFINITY;
    const float m1 = fminf(fx, fminf(fy, fz));
    const float m2 = fmaxf(fminf(fx, fy), fminf(fmaxf(fx, fy), fz));   // second smallest
    int face;                                                           // 0 x, 1 y, 2 z
    if (m2 - m1 <= 1e-5f * m2 + cell.eps * (ax + ay + az)) {
        double tx = INFINITY, ty = INFINITY, tz = INFINITY;
        if (d.x > 0.f) tx = ((double)cell.lx - ox) / d.x; else if (d.x < 0.f) tx = (0.0 - ox) / d.x;
        if (d.y > 0.f) ty = ((double)cell.ly - oy) / d.y; else if (d.y < 0.f) ty = (0.0 - oy) / d.y;
        if (d.z > 0.f) tz = ((double)cell.z_top - oz) / d.z; else if (d.z < 0.f) tz = ((double)cell.z_min - oz) / d.z;
        face = (tz < tx && tz < ty) ? 2 : (tx <= ty ? 0 : 1);
    } else {
        face = fz == m1 ? 2 : (fx == m1 ? 0 : 1);
    }
    if (face == 2) {
        tout = (float)(d.z > 0.f ? (double)cell.z_top - oz : oz - (double)cell.z_min) * az;
        return d.z > 0.f ? HIT_ESCAPE : HIT_LOST;
    }
    if (++wraps > cell.max_wraps) {
        tout = fminf(fx, fy);
        return HIT_LOST;
    }
    if (face == 0) {
        const double tx = d.x > 0.f ? ((double)cell.lx - ox) / d.x : (0.0 - ox) / d.x;
        oy = oy + tx * d.y; oz = oz + tx * d.z; ox = d.x > 0.f ? 0.0 : (double)cell.lx;
    } else {
        const double ty = d.y > 0.f ? ((double)cell.ly - oy) / d.y : (0.0 - oy) / d.y;
        ox = ox + ty * d.x; oz = oz + ty * d.z; oy = d.y > 0.f ? 0.0 : (double)cell.ly;
    }
    tout = 0.f;
    return 0;
}

// Trace one ray segment by segment through the periodic cell (Section 2.2,
// last paragraph).  Returns the hit record; *wraps gets the lateral re-entries.
// The re-entry point is carried in FP64 (a few operations per wrap) so a ray
// that wraps many times does not accumulate FP32 rounding in its origin; each
// cell query uses that point rounded to FP32.
template <int FMT, bool COUNT, bool TRI64, int SMEM = kSmemStack>
__device__ __forceinline__ float4 trace_ray(const void* __restrict__ nodes, const float4* __restrict__ tris,
                                            const float3 o32, const float3 d, int skip, const Cell& c, StackRef st,
                                            int& wraps, unsigned& status, Counts* cnt)
{
    wraps = 0;
    double ox = o32.x, oy = o32.y, oz = o32.z;
    float3 o = o32;
    for (;;) {
        const RaySetup rs = setup_ray(o, d);
        RaySetup64 r64;
        if (TRI64) r64 = setup_ray64(o, d);
        float t, u, v;
        // loop passes of one cell: inner-node visits plus leaf tests (at most 4 per 4-wide node)
        const int j = bvh_closest<FMT, COUNT, TRI64, SMEM>(nodes, tris, rs, r64, skip, st, t, u, v, status,
                                                           5 * c.max_visits, cnt);
        if (j >= 0) return make_float4(t, u, v, __int_as_float(j));
        double tx = INFINITY, ty = INFINITY, tz = INFINITY;
        if (d.x > 0.f) tx = ((double)c.lx - ox) / d.x; else if (d.x < 0.f) tx = (0.0 - ox) / d.x;
        if (d.y > 0.f) ty = ((double)c.ly - oy) / d.y; else if (d.y < 0.f) ty = (0.0 - oy) / d.y;
        if (d.z > 0.f) tz = ((double)c.z_top - oz) / d.z; else if (d.z < 0.f) tz = ((double)c.z_min - oz) / d.z;
        if (tz < tx && tz < ty)
            return make_float4((float)tz, 0.f, 0.f, __int_as_float(d.z > 0.f ? HIT_ESCAPE : HIT_LOST));
        if (++wraps > c.max_wraps) return make_float4((float)fmin(tx, ty), 0.f, 0.f, __int_as_float(HIT_LOST));
        if (tx <= ty) {
            oy = oy + tx * d.y;
            oz = oz + tx * d.z;
            ox = d.x > 0.f ? 0.0 : (double)c.lx;
        } else {
            ox = ox + ty * d.x;
            oz = oz + ty * d.z;
            oy = d.y > 0.f ? 0.0 : (double)c.ly;
        }
        o = make_float3((float)ox, (float)oy, (float)oz);
        skip = -1;
    }
}

template <int FMT, bool RECORD, bool COUNT>
__global__ void __launch_bounds__(128)
k_traverse(const void* __restrict__ nodes, const float4* __restrict__ tris, Cell cell,
           const float4* __restrict__ oe, const float4* __restrict__ dt, float4* __restrict__ hits,
           int* __restrict__ wraps_out, Control* __restrict__ ctl, int gen, unsigned cap,
           Tally* __restrict__ tally)
{
    extern __shared__ int2 s_stack[];
    const StackRef st{s_stack, (int)blockDim.x, (int)threadIdx.x};
    const unsigned n = min(*((volatile unsigned*)&ctl->count[gen]), cap);
    const int lane = threadIdx.x & 31;
    unsigned long long my_wraps = 0;
    unsigned status = 0;
    Counts cnt;
    for (;;) {
        unsigned base = 0;
        if (lane == 0) base = atomicAdd(&ctl->next[gen], 32u);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        if (base >= n) break;
        const unsigned i = base + lane;
        if (i < n) {
            const float4 a = oe[i], b = dt[i];
            int w;
            const float4 h = trace_ray<FMT, COUNT, false>(nodes, tris, make_float3(a.x, a.y, a.z),
                                                          make_float3(b.x, b.y, b.z), __float_as_int(b.w), cell,
                                                          st, w, status, &cnt);
            hits[i] = h;
            my_wraps += (unsigned)w;
            if (RECORD) wraps_out[i] = w;
        }
    }
    for (int off = 16; off; off >>= 1) {
        my_wraps += __shfl_xor_sync(0xFFFFFFFFu, my_wraps, off);
        status |= __shfl_xor_sync(0xFFFFFFFFu, status, off);
    }
    if (COUNT) {
        unsigned long long v = cnt.visits, t = cnt.tests;
        for (int off = 16; off; off >>= 1) {
            v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
            t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
        }
        if (lane == 0) { atomicAdd(&tally->node_visits, v); atomicAdd(&tally->tri_tests, t); }
    }
    if (lane == 0) {
        if (my_wraps) atomicAdd(&tally->wraps, my_wraps);
        if (status) atomicOr(&tally->status, (unsigned long long)status);
    }
}

// Re-test form of the FP32 watertight test: besides a new closest hit (1) or
// none (0) it answers 2 when the facet's smallest edge function lies within
// edge_eps (relative to |U| + |V| + |W|) of zero -- a hit or a miss too close
// to an edge for FP32 to decide -- and leaves that facet to the FP64 test.
// With edge_eps = 0 every facet gets the plain FP32 decision.
__device__ __forceinline__ int intersect_tri_rt(const RaySetup& r, float4 w0, float4 w1, float4 w2, float edge_eps,
                                                float& t_best, int& best_orig, float& bu, float& bv)
{
    const float3 A = f3(w0) - r.o, B = f3(w1) - r.o, C = f3(w2) - r.o;
    const float ax = dot3_fixed(A, r.mx), ay = dot3_fixed(A, r.my);
    const float bx = dot3_fixed(B, r.mx), by = dot3_fixed(B, r.my);
    const float cx = dot3_fixed(C, r.mx), cy = dot3_fixed(C, r.my);
    const float U = cross2_fixed(cx, by, cy, bx), V = cross2_fixed(ax, cy, ay, cx), W = cross2_fixed(bx, ay, by, ax);
    const float m = fminf(fminf(U, V), W);
    const float e = edge_eps * (fabsf(U) + fabsf(V) + fabsf(W));
    if (m < -e) return 0;                          // clearly outside or back-facing
    if (m <= e && edge_eps > 0.f) return 2;        // near an edge: FP64 decides
    const float det = __fadd_rn(__fadd_rn(U, V), W);
    if (det == 0.f) return 0;
    const float az = dot3_fixed(A, r.mz), bz = dot3_fixed(B, r.mz), cz = dot3_fixed(C, r.mz);
    const float T = __fmaf_rn(W, cz, __fmaf_rn(V, bz, __fmul_rn(U, az)));
    if (T <= 0.f) return 0;
    const float t = T / det;
    const int orig = __float_as_int(w0.w);
    if (t < t_best || (t == t_best && orig < best_orig)) {
        t_best = t;
        best_orig = orig;
        bu = V / det;
        bv = W / det;
        return 1;
    }
    return 0;
}

// FP64 test of one facet against the best hit so far (state in and out by
// value).  Out of line, so its double-precision registers never press on the
// traversal loop that calls it for the rare ambiguous facet.
struct Hit64 {
    double t;             // best distance so far
    float u, v;
    int orig;             // original index of the best facet
    bool won;             // this facet is the new best
};

__device__ __noinline__ Hit64 facet_fp64(float3 o, float3 d, float4 w0, float4 w1, float4 w2, Hit64 cur)
{
    const RaySetup64 r64 = setup_ray64(o, d);
    cur.won = intersect_tri64(r64, w0, w1, w2, cur.t, cur.orig, cur.u, cur.v);
    return cur;
}

// --------------------------------------------------------------------------
// traverse, while-while form (Aila & Laine, HPG 2009): inner nodes and leaf
// triangles run in separate loops so the lanes of a warp stay in the same
// phase; the first leaf a lane meets is postponed until every active lane
// has one.  A lane whose ray finishes takes a new ray from the generation's
// queue (one atomic per warp refill) instead of idling until the whole tile
// is done.  The FP64 re-entry point of each lane lives in shared memory.
// With RETEST, a facet whose FP32 edge functions cannot decide it (within
// kEdgeEps of an edge, hit or miss) is set aside -- up to kAmbMax per cell
// traversal, in the lane's shared-memory list -- and decided by the FP64 test
// once the cell's traversal ends; a closest hit meeting its facet with
// cos(incidence) below kGrazeCos gets its distance from the FP64 test too.
// Setting a facet aside only weakens the culling meanwhile, so none is
// missed.  The FP64 work is per ambiguous facet, in the same launch, and its
// call stays out of the inner loops (a call there costs registers on every
// iteration).  Ambiguous facets beyond kAmbMax in one cell (expected about
// once in 1e17 cells at the measured rate of 1e-4 per test) keep the FP32
// decision.
// --------------------------------------------------------------------------
constexpr int kEntrySentinel = 0x76543210;   // "stack empty" (never a node index)
constexpr int kFetchThreshold = 28;          // default: refill when fewer lanes than this are active
constexpr float kEdgeEps = 1e-5f;
constexpr float kGrazeCos = 1e-3f;
constexpr int kAmbMax = 4;

template <int FMT, bool RECORD, bool COUNT, bool RETEST, int SSTACK>
__global__ void __launch_bounds__(128, 8)
k_traverse_ww(const void* __restrict__ nodes, const float4* __restrict__ tris, const float4* __restrict__ normals,
              Cell cell, const float4* __restrict__ oe, const float4* __restrict__ dt, float4* __restrict__ hits,
              int* __restrict__ wraps_out, Control* __restrict__ ctl, int gen, unsigned cap,
              Tally* __restrict__ tally, int fetch_threshold)
{
    extern __shared__ int2 s_stack[];                                   // [SSTACK][blockDim]
    const int B = blockDim.x, tid = threadIdx.x, lane = tid & 31;
    double* s_o = reinterpret_cast<double*>(s_stack + SSTACK * B);       // [3][blockDim]
    double* s_t64 = s_o + 3 * B;                                         // RETEST: [blockDim]
    int* s_b64 = reinterpret_cast<int*>(s_t64 + B);                      // RETEST: [blockDim]
    int* s_amb = s_b64 + B;                                              // RETEST: [kAmbMax][blockDim]
    const unsigned lt = (1u << lane) - 1u;
    const unsigned n = min(*((volatile unsigned*)&ctl->count[gen]), cap);
    int2 lstack[kStackMax - SSTACK];

    int ray = -1;
    bool exhausted = false, drained = false;
    float3 o = make_float3(0.f, 0.f, 0.f), d = make_float3(0.f, 0.f, 1.f);
    RaySetup rs = setup_ray(o, d);
    float t_best = kNoHit, bu = 0.f, bv = 0.f;
    double t_best64 = INFINITY;
    int best = -1, best_orig = INT_MAX, node = kEntrySentinel, leaf = 0, sp = 0, skip = -1, wraps = 0, visits = 0;
    unsigned status = 0;
    unsigned long long my_wraps = 0;
    unsigned my_retested = 0;
    bool used64 = false;                 // RETEST: the current ray had a facet decided in FP64
    int namb = 0;                        // RETEST: facets set aside for FP64 in this cell
    Counts cnt;

    auto push = [&](int node_ref, float tmin) {
        const int2 e = make_int2(node_ref, __float_as_int(tmin));
        if (sp < SSTACK) s_stack[sp * B + tid] = e;
        else if (sp < kStackMax) lstack[sp - SSTACK] = e;
        else { status |= ST_STACK_OVERFLOW; sp = kStackMax - 1; }
        ++sp;
    };
    auto pop = [&]() -> int {
        while (sp > 0) {
            --sp;
            const int2 e = sp < SSTACK ? s_stack[sp * B + tid] : lstack[sp - SSTACK];
            if (__int_as_float(e.y) <= t_best * kTieSlack * kRobust) return e.x;
        }
        return kEntrySentinel;
    };
    auto restart = [&]() {      // new cell traversal from the current origin
        rs = setup_ray(o, d);
        if constexpr (FMT == FMT_Q4) rs = q4_setup(rs);   // the cell exit reads only finite 1/d
        node = 0; leaf = 0; sp = 0; visits = 0;
        t_best = kNoHit; best = -1; best_orig = INT_MAX; bu = bv = 0.f;
        if (RETEST) { s_b64[tid] = -1; namb = 0; }   // s_t64: FP64 distance of facet s_b64 (if the best)
    };

    for (;;) {
        const bool need = ray < 0 && !exhausted;
        const unsigned m = __ballot_sync(0xFFFFFFFFu, need);
        if (m) {
            const int leader = __ffs(m) - 1;
            unsigned base = 0;
            if (lane == leader) base = atomicAdd(&ctl->next[gen], (unsigned)__popc(m));
            base = __shfl_sync(0xFFFFFFFFu, base, leader);
            if (base + (unsigned)__popc(m) >= n) drained = true;
            if (need) {
                const unsigned idx = base + __popc(m & lt);
                if (idx < n) {
                    ray = (int)idx;
                    const float4 a = oe[idx], b = dt[idx];
                    o = make_float3(a.x, a.y, a.z);
                    d = make_float3(b.x, b.y, b.z);
                    skip = __float_as_int(b.w);
                    s_o[tid] = a.x; s_o[B + tid] = a.y; s_o[2 * B + tid] = a.z;
                    wraps = 0;
                    restart();
                } else {
                    exhausted = true;
                }
            }
        }
        if (__all_sync(0xFFFFFFFFu, ray < 0)) break;
        if (ray < 0) continue;

        bool cell_done = false;
        for (;;) {
            while (node >= 0 && node != kEntrySentinel) {
                if (++visits > cell.max_visits) { status |= ST_LOOP_LIMIT; node = kEntrySentinel; leaf = 0; sp = 0; break; }
                if (COUNT) ++cnt.visits;
                if constexpr (FMT == FMT_W4 || FMT == FMT_Q4) {
                    float tk[4];
                    int ck[4], nh;
                    node4_children<FMT>(nodes, node, rs, t_best * kTieSlack, tk, ck, nh);
                    if (nh > 3) push(ck[3], tk[3]);           // farthest first: the nearest stays on top
                    if (nh > 2) push(ck[2], tk[2]);
                    if (nh > 1) push(ck[1], tk[1]);
                    node = nh > 0 ? ck[0] : pop();
                } else {
                    float tmin0, tmin1;
                    bool h0, h1;
                    int c0, c1;
                    node_children<FMT>(nodes, node, rs, t_best * kTieSlack, tmin0, tmin1, h0, h1, c0, c1);
                    if (h0 && h1) {
                        const bool first0 = tmin0 <= tmin1;
                        push(first0 ? c1 : c0, first0 ? tmin1 : tmin0);
                        node = first0 ? c0 : c1;
                    } else if (h0 || h1) {
                        node = h0 ? c0 : c1;
                    } else {
                        node = pop();
                    }
                }
                if (node < 0 && leaf == 0) { leaf = node; node = pop(); }
                if (!__any_sync(__activemask(), leaf == 0)) break;
            }
            while (leaf < 0) {
                if (RETEST) {
                    const int v = ~leaf;
                    const int first = v >> 3, count = (v & 7) + 1;
                    for (int k = 0; k < count; ++k) {
                        const int j = first + k;
                        if (j == skip) continue;
                        if (COUNT) ++cnt.tests;
                        const float4* tp = tris + 3ll * j;
                        const float4 w0 = ldg4(tp), w1 = ldg4(tp + 1), w2 = ldg4(tp + 2);
                        const int r = intersect_tri_rt(rs, w0, w1, w2, namb < kAmbMax ? kEdgeEps : 0.f, t_best,
                                                       best_orig, bu, bv);
                        if (r == 1) best = j;
                        else if (r == 2) s_amb[(namb++) * B + tid] = j;
                    }
                } else {
                    test_leaf<COUNT, false>(tris, rs, RaySetup64{}, leaf, skip, t_best, t_best64, best, best_orig,
                                            bu, bv, &cnt);
                }
                leaf = 0;
                if (node < 0) { leaf = node; node = pop(); }
            }
            if (node == kEntrySentinel) { cell_done = true; break; }
            if (!drained && __popc(__activemask()) < fetch_threshold) break;
        }
        if (!cell_done) continue;

        if (RETEST && namb > 0) {        // the facets set aside, against the FP32 best, in FP64
            for (int k = 0; k < namb; ++k) {
                const int j = s_amb[k * B + tid];
                const float4* tp = tris + 3ll * j;
                const double ref = (best >= 0 && s_b64[tid] == best) ? s_t64[tid] : (double)t_best;
                const Hit64 h = facet_fp64(o, d, ldg4(tp), ldg4(tp + 1), ldg4(tp + 2),
                                           Hit64{ref, bu, bv, best_orig, false});
                if (h.won) {
                    best = j; best_orig = h.orig; bu = h.u; bv = h.v;
                    t_best = (float)h.t;
                    s_t64[tid] = h.t; s_b64[tid] = j;
                }
            }
            namb = 0;
            used64 = true;
        }

        if (best >= 0) {
            if (RETEST && s_b64[tid] != best) {
                const float4 nr = ldg4(normals + best);
                if (-(d.x * nr.x + d.y * nr.y + d.z * nr.z) < kGrazeCos) {   // grazing: distance in FP64
                    const float4* tp = tris + 3ll * best;
                    const Hit64 h = facet_fp64(o, d, ldg4(tp), ldg4(tp + 1), ldg4(tp + 2),
                                               Hit64{INFINITY, bu, bv, INT_MAX, false});
                    if (h.won) { t_best = (float)h.t; bu = h.u; bv = h.v; }
                    used64 = true;
                }
            }
            hits[ray] = make_float4(t_best, bu, bv, __int_as_float(best));
        } else {
            double ox = s_o[tid], oy = s_o[B + tid], oz = s_o[2 * B + tid];
            float tout;
            const int code = cell_exit(o, d, rs.inv, cell, ox, oy, oz, wraps, tout);
            if (code) {
                hits[ray] = make_float4(tout, 0.f, 0.f, __int_as_float(code));
            } else {
                s_o[tid] = ox; s_o[B + tid] = oy; s_o[2 * B + tid] = oz;
                o = make_float3((float)ox, (float)oy, (float)oz);
                skip = -1;
                restart();
                continue;
            }
        }
        my_wraps += (unsigned)wraps;
        if (RECORD) wraps_out[ray] = wraps;
        if (RETEST) { my_retested += used64 ? 1u : 0u; used64 = false; }
        ray = -1;
    }
    for (int off = 16; off; off >>= 1) {
        my_wraps += __shfl_xor_sync(0xFFFFFFFFu, my_wraps, off);
        status |= __shfl_xor_sync(0xFFFFFFFFu, status, off);
        if (RETEST) my_retested += __shfl_xor_sync(0xFFFFFFFFu, my_retested, off);
    }
    if (COUNT) {
        unsigned long long v = cnt.visits, t = cnt.tests;
        for (int off = 16; off; off >>= 1) {
            v += __shfl_xor_sync(0xFFFFFFFFu, v, off);
            t += __shfl_xor_sync(0xFFFFFFFFu, t, off);
        }
        if (lane == 0) { atomicAdd(&tally->node_visits, v); atomicAdd(&tally->tri_tests, t); }
    }
    if (lane == 0) {
        if (my_wraps) atomicAdd(&tally->wraps, my_wraps);
        if (status) atomicOr(&tally->status, (unsigned long long)status);
        if (RETEST && my_retested) atomicAdd(&tally->retested, (unsigned long long)my_retested);
    }
}

// --------------------------------------------------------------------------
// a generation of rays parallel to z through the column grid
// --------------------------------------------------------------------------
// A ray with direction (0, 0, d_z) meets a facet only inside the facet's xy
// box and, going down, at or below the facet's top z.  It tests the facets
// listed for its pixel in order of decreasing top z and stops when even the
// next top z lies farther than the best hit (margins 1 + 2^-12 relative and
// 2^-16 M absolute, M the largest cell coordinate, far above the rounding of
// a facet distance), so no facet it skips could have won.  The facet tests,
// the FP64 re-test and the tie rule are those of the hierarchy's traversal,
// so the hit record is the same; a ray that meets no facet leaves through
// z_min (z_top going up) as in the hierarchy's cell exit.  It never wraps.
constexpr float kColRel = 1.000244140625f;     // 1 + 2^-12

template <bool RECORD, bool RETEST>
__global__ void __launch_bounds__(128)
k_trace_columns(const unsigned* __restrict__ col_off, const uint2* __restrict__ col_ent, int gx, int gy, float iwx,
                float iwy, const float4* __restrict__ tris, const float4* __restrict__ normals, Cell cell,
                const float4* __restrict__ oe, const float4* __restrict__ dt, float4* __restrict__ hits,
                int* __restrict__ wraps_out, Control* __restrict__ ctl, int gen, unsigned cap,
                Tally* __restrict__ tally)
{
    const unsigned n = min(*((volatile unsigned*)&ctl->count[gen]), cap);
    const float eps_abs = cell.eps * 16.f;
    unsigned status = 0, my_rays = 0, my_retested = 0;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 a = oe[i], b = dt[i];
        const float3 o = make_float3(a.x, a.y, a.z), d = make_float3(b.x, b.y, b.z);
        const int skip = __float_as_int(b.w);
        ++my_rays;
        if (RECORD) wraps_out[i] = 0;
        if (d.x != 0.f || d.y != 0.f || !(d.z != 0.f)) {      // not a column ray: the caller chose wrongly
            status |= ST_COLUMN;
            hits[i] = make_float4(0.f, 0.f, 0.f, __int_as_float(HIT_LOST));
            continue;
        }
        const RaySetup rs = setup_ray(o, d);
        const float az = fabsf(rs.inv.z);
        const int px = min(max((int)floorf(o.x * iwx), 0), gx - 1);
        const int py = min(max((int)floorf(o.y * iwy), 0), gy - 1);
        const unsigned e0 = col_off[py * gx + px], e1 = col_off[py * gx + px + 1];
        float t_best = kNoHit, bu = 0.f, bv = 0.f;
        int best = -1, best_orig = INT_MAX;
        int amb[kAmbMax];
        int namb = 0;
        // Two entries per pass: both stop checks use the best distance before the
        // pass, which can only test a facet more (never skip one that could win),
        // and both facets' loads are in flight together.
        auto test = [&](int j) {
            if (j == skip) return;
            const float4* tp = tris + 3ll * j;
            const float4 w0 = ldg4(tp), w1 = ldg4(tp + 1), w2 = ldg4(tp + 2);
            if (RETEST) {
                const int r = intersect_tri_rt(rs, w0, w1, w2, namb < kAmbMax ? kEdgeEps : 0.f, t_best, best_orig,
                                               bu, bv);
                if (r == 1) best = j;
                else if (r == 2) amb[namb++] = j;
            } else {
                if (intersect_tri(rs, w0, w1, w2, t_best, best_orig, bu, bv)) best = j;
            }
        };
        uint2 nx0 = e0 < e1 ? col_ent[e0] : make_uint2(0u, 0u);
        uint2 nx1 = e0 + 1 < e1 ? col_ent[e0 + 1] : make_uint2(0u, 0u);
        for (unsigned e = e0; e < e1; e += 2) {
            const uint2 ea = nx0, eb = nx1;
            if (e + 2 < e1) nx0 = col_ent[e + 2];        // the next pair loads while these facets are tested
            if (e + 3 < e1) nx1 = col_ent[e + 3];
            const float lim = t_best * kColRel + eps_abs;
            if (d.z < 0.f && (o.z - __uint_as_float(ea.y)) * az > lim) break;
            const bool second = e + 1 < e1 && !(d.z < 0.f && (o.z - __uint_as_float(eb.y)) * az > lim);
            test((int)ea.x);
            if (!second) break;
            test((int)eb.x);
        }
        bool used64 = false;
        int b64 = -1;
        double t64 = 0.0;
        if (RETEST && namb > 0) {                 // the facets set aside, against the FP32 best, in FP64
            for (int k = 0; k < namb; ++k) {
                const int j = amb[k];
                const float4* tp = tris + 3ll * j;
                const double ref = (best >= 0 && b64 == best) ? t64 : (double)t_best;
                const Hit64 h = facet_fp64(o, d, ldg4(tp), ldg4(tp + 1), ldg4(tp + 2),
                                           Hit64{ref, bu, bv, best_orig, false});
                if (h.won) {
                    best = j; best_orig = h.orig; bu = h.u; bv = h.v;
                    t_best = (float)h.t;
                    t64 = h.t; b64 = j;
                }
            }
            used64 = true;
        }
        if (best >= 0) {
            if (RETEST && b64 != best) {
                const float4 nr = ldg4(normals + best);
                if (-(d.x * nr.x + d.y * nr.y + d.z * nr.z) < kGrazeCos) {   // grazing: distance in FP64
                    const float4* tp = tris + 3ll * best;
                    const Hit64 h = facet_fp64(o, d, ldg4(tp), ldg4(tp + 1), ldg4(tp + 2),
                                               Hit64{INFINITY, bu, bv, INT_MAX, false});
                    if (h.won) { t_best = (float)h.t; bu = h.u; bv = h.v; }
                    used64 = true;
                }
            }
            hits[i] = make_float4(t_best, bu, bv, __int_as_float(best));
        } else {
            const double oz = (double)o.z;
            const float tout = (float)(d.z > 0.f ? (double)cell.z_top - oz : oz - (double)cell.z_min) * az;
            hits[i] = make_float4(tout, 0.f, 0.f, __int_as_float(d.z > 0.f ? HIT_ESCAPE : HIT_LOST));
        }
        if (RETEST && used64) ++my_retested;
    }
    const int lane = threadIdx.x & 31;
    for (int off = 16; off; off >>= 1) {
        my_rays += __shfl_xor_sync(0xFFFFFFFFu, my_rays, off);
        status |= __shfl_xor_sync(0xFFFFFFFFu, status, off);
        if (RETEST) my_retested += __shfl_xor_sync(0xFFFFFFFFu, my_retested, off);
    }
    if (lane == 0) {
        if (my_rays) atomicAdd(&tally->col_rays, (unsigned long long)my_rays);
        if (status) atomicOr(&tally->status, (unsigned long long)status);
        if (RETEST && my_retested) atomicAdd(&tally->retested, (unsigned long long)my_retested);
    }
}

// --------------------------------------------------------------------------
// a generation of rays of one fixed oblique direction through a slanted grid
// --------------------------------------------------------------------------
// Primaries at fixed incidence (dx, 0, dz) travel in straight lines through
// the periodic images of the cell.  Projected along that direction onto the
// top plane, every facet image covers the entry points of the rays that can
// meet it, and the image fixes how many lateral wraps k the ray has made by
// then.  The slanted grid lists, per pixel of entry points, those (facet, k)
// pairs sorted by top z (their along-ray distance from the entry is at least
// (z_top - top z) / |dz|).  A ray tests them in that order against the FP32 ray
// of its segment k -- the FP32 re-entry point after k wraps, replayed with the
// hierarchy's own cell exit -- keeps the best (k, t, original id) in that
// order (the hierarchy ends at the first segment with a hit and takes the
// nearest, then the lowest id, within it), and stops when the next facet lies
// beyond the best hit by the column grid's margins.  The facet tests, wrap
// replay and tie rule are the hierarchy's, so the hit record, wrap count
// included, is the same.  With no facet met the replay carries the ray to its
// exit, as the hierarchy does.
template <bool RECORD, bool ITEMS>
__global__ void __launch_bounds__(128, 6)      // 6 blocks per SM (80 registers, under 100 B of spills): 18 % faster than 4
k_trace_slant(const GridDev* __restrict__ grids, const float4* __restrict__ tris, Cell cell,
              const float4* __restrict__ oe, const float4* __restrict__ dt, const uint4* __restrict__ id,
              float4* __restrict__ hits, int* __restrict__ wraps_out, Control* __restrict__ ctl, int gen,
              unsigned cap, Tally* __restrict__ tally)
{
    const unsigned n = min(*((volatile unsigned*)&ctl->count[gen]), cap);
    const float eps_abs = cell.eps * 16.f;
    unsigned status = 0, my_rays = 0;
    unsigned long long my_wraps = 0;
    for (unsigned i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const float4 a = oe[i], b = dt[i];
        const float3 o = make_float3(a.x, a.y, a.z), d = make_float3(b.x, b.y, b.z);
        const GridDev g = grids[ITEMS ? id[i].y : 0u];
        ++my_rays;
        if (d.y != 0.f || d.x != g.dx || d.z != g.dz || !(d.z < 0.f) || __float_as_int(b.w) != -1 ||
            o.z != cell.z_top) {
            status |= ST_COLUMN;           // not a ray this grid serves: the caller chose wrongly
            hits[i] = make_float4(0.f, 0.f, 0.f, __int_as_float(HIT_LOST));
            if (RECORD) wraps_out[i] = 0;
            continue;
        }
        const float az = fabsf(1.0f / d.z);
        const int px = min(max((int)floorf(o.x * g.iwx), 0), g.gx - 1);
        const int py = min(max((int)floorf(o.y * g.iwy), 0), g.gy - 1);
        const unsigned e0 = g.off[py * g.gx + px], e1 = g.off[py * g.gx + px + 1];
        // segment state: the ray after kc wraps (FP32 origin oc, FP64 origin sx/sy/sz);
        // k_end: the last segment the ray reaches (its exit or wrap limit ends it there)
        int kc = 0, wr = 0, k_end = INT_MAX, end_code = 0;
        float end_tout = 0.f;
        float3 oc = o;
        float drop = 0.f;                           // z of the entry minus z of the segment's origin
        double sx = o.x, sy = o.y, sz = o.z;
        RaySetup rs = setup_ray(oc, d);
        auto advance = [&](int k) {                 // replay the wraps up to segment k
            if (k < kc) { kc = 0; wr = 0; oc = o; sx = o.x; sy = o.y; sz = o.z; rs = setup_ray(oc, d); drop = 0.f; }
            while (kc < k && kc < k_end) {
                float tout;
                const int code = cell_exit(oc, d, rs.inv, cell, sx, sy, sz, wr, tout);
                if (code) { k_end = kc; end_code = code; end_tout = tout; break; }
                oc = make_float3((float)sx, (float)sy, (float)sz);
                rs = setup_ray(oc, d);
                drop = (float)((double)o.z - sz);
                ++kc;
            }
        };
        float t_best = kNoHit, bu = 0.f, bv = 0.f, reach = kNoHit;
        int best = -1, best_orig = INT_MAX, k_best = INT_MAX;
        for (unsigned e = e0; e < e1; ++e) {
            const uint2 ent = g.ent[e];
            if ((o.z - __uint_as_float(ent.y)) * az > reach) break;
            const int k = (int)(ent.x >> kSlantFacetBits);
            const int j = (int)(ent.x & ((1u << kSlantFacetBits) - 1u));
            if (k > k_best || k > k_end) continue;             // a later segment cannot win
            if (k != kc) advance(k);
            if (kc != k) continue;                             // the ray ends before segment k
            float t = k == k_best ? t_best : kNoHit, u = 0.f, v = 0.f;
            int orig = k == k_best ? best_orig : INT_MAX;
            const float4* tp = tris + 3ll * j;
            if (intersect_tri(rs, ldg4(tp), ldg4(tp + 1), ldg4(tp + 2), t, orig, u, v)) {
                t_best = t; best_orig = orig; bu = u; bv = v; best = j; k_best = k;
                // along-ray distance of the best hit from the entry point, with the grid margins
                reach = (drop * az + t_best) * kColRel + eps_abs;
            }
        }
        int w;
        if (best >= 0) {
            hits[i] = make_float4(t_best, bu, bv, __int_as_float(best));
            w = k_best;
        } else {
            advance(INT_MAX);                                   // no facet: replay to the exit
            hits[i] = make_float4(end_tout, 0.f, 0.f, __int_as_float(end_code ? end_code : HIT_LOST));
            w = wr;
        }
        my_wraps += (unsigned)w;
        if (RECORD) wraps_out[i] = w;
    }
    const int lane = threadIdx.x & 31;
    for (int off = 16; off; off >>= 1) {
        my_rays += __shfl_xor_sync(0xFFFFFFFFu, my_rays, off);
        my_wraps += __shfl_xor_sync(0xFFFFFFFFu, my_wraps, off);
        status |= __shfl_xor_sync(0xFFFFFFFFu, status, off);
    }
    if (lane == 0) {
        if (my_rays) atomicAdd(&tally->col_rays, (unsigned long long)my_rays);
        if (my_wraps) atomicAdd(&tally->wraps, my_wraps);
        if (status) atomicOr(&tally->status, (unsigned long long)status);
    }
}

template <int FMT>
__global__ void __launch_bounds__(128)
k_trace_rays(const void* __restrict__ nodes, const float4* __restrict__ tris, const int* __restrict__ inv_order,
             int n_tri, const float* __restrict__ o, const float* __restrict__ d, const int* __restrict__ skip,
             int64_t n, rtmc_hit* __restrict__ hits, unsigned* __restrict__ status_out, int max_iter)
{
    extern __shared__ int2 s_stack[];
    const StackRef st{s_stack, (int)blockDim.x, (int)threadIdx.x};
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float3 oo = make_float3(o[3 * i], o[3 * i + 1], o[3 * i + 2]);
    const float3 dd = make_float3(d[3 * i], d[3 * i + 1], d[3 * i + 2]);
    const int sk = (skip && skip[i] >= 0 && skip[i] < n_tri) ? inv_order[skip[i]] : -1;
    unsigned status = 0;
    float t, u, v;
    RaySetup64 r64;
    const int j = bvh_closest<FMT>(nodes, tris, setup_ray(oo, dd), r64, sk, st, t, u, v, status, max_iter);
    rtmc_hit h;
    h.t = j >= 0 ? t : INFINITY;
    h.u = u; h.v = v;
    h.tri = j >= 0 ? __float_as_int(__ldg(tris + 3ll * j).w) : -1;
    hits[i] = h;
    if (status) atomicOr(status_out, status);
}

}  // namespace

// Inner-node visits one cell traversal may make: in a tree every inner node is
// pushed by its one parent at most once, so a correct traversal visits each at
// most once; more means a broken hierarchy, and the ray is abandoned with
// ST_LOOP_LIMIT instead of looping.  `cap` > 0 lowers the bound (test hook).
static int visit_bound(const DeviceMesh& m, int cap)
{
    const int64_t inner = (m.kind == FMT_W4 || m.kind == FMT_Q4) ? m.n_w4 : m.n_nodes;
    int64_t b = std::min<int64_t>(inner + 1, (int64_t)kMaxVisits);
    if (cap > 0) b = std::min<int64_t>(b, cap);
    return (int)b;
}

template <int F, bool R, bool C, int SS>
static cudaError_t ww_launch(const DeviceMesh& m, const Cell& cell, const Queues& q, int buf, int gen, int num_sms,
                             const Tuning& tune, bool retest, const void* nodes, cudaStream_t s)
{
    const int bt = tune.block_threads;
    int per_sm = tune.blocks_per_sm;
    const int thr = tune.fetch_threshold > 0 ? tune.fetch_threshold : kFetchThreshold;
    const size_t smem = (size_t)SS * bt * sizeof(int2) + 3 * (size_t)bt * sizeof(double);
    if (retest) {
        const size_t smem_rt = smem + (size_t)bt * (sizeof(double) + (1 + kAmbMax) * sizeof(int));
        if (per_sm <= 0)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse_ww<F, R, C, true, SS>, bt, smem_rt);
        k_traverse_ww<F, R, C, true, SS><<<num_sms * (per_sm > 0 ? per_sm : 1), bt, smem_rt, s>>>(
            nodes, m.tris, m.normals, cell, q.oe[buf], q.dt[buf], q.hits, R ? q.wraps : nullptr, q.ctl, gen,
            q.cap[buf], q.tally, thr);
    } else {
        if (per_sm <= 0)
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse_ww<F, R, C, false, SS>, bt, smem);
        k_traverse_ww<F, R, C, false, SS><<<num_sms * (per_sm > 0 ? per_sm : 1), bt, smem, s>>>(
            nodes, m.tris, m.normals, cell, q.oe[buf], q.dt[buf], q.hits, R ? q.wraps : nullptr, q.ctl, gen,
            q.cap[buf], q.tally, thr);
    }
    return cudaGetLastError();
}

template <int F, bool R, bool C>
static cudaError_t traverse_t(const DeviceMesh& m, const RunParams& p, const Queues& q, int buf, int gen,
                              int num_sms, const Tuning& tune, bool retest, cudaStream_t s)
{
    const float big = fmaxf(fmaxf(fabsf(p.lx), fabsf(p.ly)), fmaxf(fabsf(p.z_min), fabsf(p.z_top)));
    const Cell cell{p.lx, p.ly, p.z_min, p.z_top, p.max_wraps, ldexpf(big, -20), visit_bound(m, tune.max_visits)};
    const void* nodes = F == FMT_Q8 ? m.q8 : (F == FMT_W4 ? m.w4 : (F == FMT_Q4 ? m.q4 : (const void*)m.nodes));
    const int bt = tune.block_threads;
    int per_sm = tune.blocks_per_sm;
    if (tune.traversal == 1) {
        const size_t smem = (size_t)kSmemStack * bt * sizeof(int2);
        if (per_sm <= 0) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_traverse<F, R, C>, bt, smem);
        k_traverse<F, R, C><<<num_sms * (per_sm > 0 ? per_sm : 1), bt, smem, s>>>(
            nodes, m.tris, cell, q.oe[buf], q.dt[buf], q.hits, R ? q.wraps : nullptr, q.ctl, gen, q.cap[buf],
            q.tally);
    } else {
        const int depth = tune.stack_depth;
        if (C || depth == 16) return ww_launch<F, R, C, 16>(m, cell, q, buf, gen, num_sms, tune, retest, nodes, s);
        if (depth == 8) return ww_launch<F, R, false, 8>(m, cell, q, buf, gen, num_sms, tune, retest, nodes, s);
        return ww_launch<F, R, false, 32>(m, cell, q, buf, gen, num_sms, tune, retest, nodes, s);
    }
    return cudaGetLastError();
}

template <int F>
static cudaError_t traverse_f(const DeviceMesh& m, const RunParams& p, const Queues& q, int buf, int gen,
                              int num_sms, const Tuning& tune, bool record, bool count, bool retest, cudaStream_t s)
{
    if (record) return count ? traverse_t<F, true, true>(m, p, q, buf, gen, num_sms, tune, retest, s)
                             : traverse_t<F, true, false>(m, p, q, buf, gen, num_sms, tune, retest, s);
    return count ? traverse_t<F, false, true>(m, p, q, buf, gen, num_sms, tune, retest, s)
                 : traverse_t<F, false, false>(m, p, q, buf, gen, num_sms, tune, retest, s);
}

cudaError_t launch_traverse(const DeviceMesh& m, const RunParams& p, const Queues& q, int buf, int gen,
                            int num_sms, const Tuning& tune, bool record, bool count, bool retest, cudaStream_t s)
{
    if (m.kind == FMT_Q8) return traverse_f<FMT_Q8>(m, p, q, buf, gen, num_sms, tune, record, count, retest, s);
    if (m.kind == FMT_W4) return traverse_f<FMT_W4>(m, p, q, buf, gen, num_sms, tune, record, count, retest, s);
    if (m.kind == FMT_Q4) return traverse_f<FMT_Q4>(m, p, q, buf, gen, num_sms, tune, record, count, retest, s);
    return traverse_f<FMT_FP32>(m, p, q, buf, gen, num_sms, tune, record, count, retest, s);
}

cudaError_t launch_columns(const DeviceMesh& m, const RunParams& p, const Queues& q, int buf, int gen,
                           int num_sms, bool record, bool retest, cudaStream_t s)
{
    if (!m.col_ok) return cudaErrorInvalidValue;
    const float big = fmaxf(fmaxf(fabsf(p.lx), fabsf(p.ly)), fmaxf(fabsf(p.z_min), fabsf(p.z_top)));
    const Cell cell{p.lx, p.ly, p.z_min, p.z_top, p.max_wraps, ldexpf(big, -20), visit_bound(m, 0)};
    const int tb = 128;
    int per_sm = 0;
    if (record) cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, retest ? k_trace_columns<true, true>
                                                                              : k_trace_columns<true, false>, tb, 0);
    else cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, retest ? k_trace_columns<false, true>
                                                                       : k_trace_columns<false, false>, tb, 0);
    const unsigned gb = (unsigned)num_sms * (unsigned)(per_sm > 0 ? per_sm : 1);   // one wave, grid-stride
    int* wr = record ? q.wraps : nullptr;
#define RTMC_COLUMNS(R, T)                                                                                      \
    k_trace_columns<R, T><<<gb, tb, 0, s>>>(m.col_off, m.col_ent, m.col_gx, m.col_gy, m.col_inv_wx, m.col_inv_wy, \
                                            m.tris, m.normals, cell, q.oe[buf], q.dt[buf], q.hits, wr, q.ctl, gen, \
                                            q.cap[buf], q.tally)
    if (record) { if (retest) RTMC_COLUMNS(true, true); else RTMC_COLUMNS(true, false); }
    else { if (retest) RTMC_COLUMNS(false, true); else RTMC_COLUMNS(false, false); }
#undef RTMC_COLUMNS
    return cudaGetLastError();
}

cudaError_t launch_slant(const DeviceMesh& m, const RunParams& p, const GridDev* grids, bool items, const Queues& q,
                         int buf, int gen, int num_sms, bool record, cudaStream_t s)
{
    const float big = fmaxf(fmaxf(fabsf(p.lx), fabsf(p.ly)), fmaxf(fabsf(p.z_min), fabsf(p.z_top)));
    const Cell cell{p.lx, p.ly, p.z_min, p.z_top, p.max_wraps, ldexpf(big, -20), visit_bound(m, 0)};
    const int tb = 128;
    int per_sm = 0;
    int* wr = record ? q.wraps : nullptr;
#define RTMC_SLANT(R, I)                                                                                        \
    do {                                                                                                        \
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_trace_slant<R, I>, tb, 0);                     \
        k_trace_slant<R, I><<<(unsigned)num_sms * (unsigned)(per_sm > 0 ? per_sm : 1), tb, 0, s>>>(            \
            grids, m.tris, cell, q.oe[buf], q.dt[buf], q.id[buf], q.hits, wr, q.ctl, gen, q.cap[buf], q.tally); \
    } while (0)
    if (record) { if (items) RTMC_SLANT(true, true); else RTMC_SLANT(true, false); }
    else { if (items) RTMC_SLANT(false, true); else RTMC_SLANT(false, false); }
#undef RTMC_SLANT
    return cudaGetLastError();
}

cudaError_t launch_trace_rays(const DeviceMesh& m, const float* o, const float* d, const int* skip, int64_t n,
                              rtmc_hit* hits, unsigned* status, cudaStream_t s)
{
    const int tb = 128;
    const size_t smem = (size_t)kSmemStack * tb * sizeof(int2);
    const int64_t gb = (n + tb - 1) / tb;
    if (gb > 0 && m.kind == FMT_Q8)
        k_trace_rays<FMT_Q8><<<(unsigned)gb, tb, smem, s>>>(m.q8, m.tris, m.inv_order, (int)m.n_tri, o, d, skip, n,
                                                            hits, status, 5 * visit_bound(m, 0));
    else if (gb > 0 && m.kind == FMT_W4)
        k_trace_rays<FMT_W4><<<(unsigned)gb, tb, smem, s>>>(m.w4, m.tris, m.inv_order, (int)m.n_tri, o, d, skip, n,
                                                            hits, status, 5 * visit_bound(m, 0));
    else if (gb > 0 && m.kind == FMT_Q4)
        k_trace_rays<FMT_Q4><<<(unsigned)gb, tb, smem, s>>>(m.q4, m.tris, m.inv_order, (int)m.n_tri, o, d, skip, n,
                                                            hits, status, 5 * visit_bound(m, 0));
    else if (gb > 0)
        k_trace_rays<FMT_FP32><<<(unsigned)gb, tb, smem, s>>>(m.nodes, m.tris, m.inv_order, (int)m.n_tri, o, d, skip,
                                                              n, hits, status, 5 * visit_bound(m, 0));
    return cudaGetLastError();
}

}  // namespace rtmc
