// rtmc_bvh.cu -- linear BVH construction on the device (sm_103a).
//
// The paper scans every element per ray (Section 2.1: "must scan through all
// elements ... rapidly become prohibitive"); this library replaces the scan
// by a binary BVH so a ray visits O(log n) boxes.  Construction follows the
// Karras (HPG 2012) formulation:
//   1. 30-bit Morton code of each triangle centroid, quantised on the cell box;
//   2. stable LSD radix sort of (code, triangle id), 4 passes of 8 bits;
//   3. one thread per inner node finds its key range and split (Karras);
//   4. bottom-up box refit: one thread per leaf climbs, the second thread to
//      reach a node (atomic counter) writes it;
//   5. triangles and normals repacked in leaf order as 16-byte aligned float4.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>

#include "rtmc_internal.h"

namespace rtmc {
namespace {

constexpr int kSortThreads = 256;
constexpr int kSortItems = 4;
constexpr int kSortTile = kSortThreads * kSortItems;

__device__ __forceinline__ unsigned expand_bits10(unsigned v)
{
    v = (v * 0x00010001u) & 0xFF0000FFu;
    v = (v * 0x00000101u) & 0x0F00F00Fu;
    v = (v * 0x00000011u) & 0xC30C30C3u;
    v = (v * 0x00000005u) & 0x49249249u;
    return v;
}

__device__ __forceinline__ unsigned quant10(float x)
{
    float q = fminf(fmaxf(x * 1024.0f, 0.0f), 1023.0f);
    return (unsigned)q;
}

__global__ void k_morton(const float* __restrict__ tri, int n, float4 box_lo, float4 box_inv,
                         unsigned* __restrict__ keys, unsigned* __restrict__ vals)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float* t = tri + 9ll * i;
    const float cx = (t[0] + t[3] + t[6]) * (1.0f / 3.0f);
    const float cy = (t[1] + t[4] + t[7]) * (1.0f / 3.0f);
    const float cz = (t[2] + t[5] + t[8]) * (1.0f / 3.0f);
    const unsigned x = quant10((cx - box_lo.x) * box_inv.x);
    const unsigned y = quant10((cy - box_lo.y) * box_inv.y);
    const unsigned z = quant10((cz - box_lo.z) * box_inv.z);
    keys[i] = (expand_bits10(x) << 2) | (expand_bits10(y) << 1) | expand_bits10(z);
    vals[i] = (unsigned)i;
}

// ---- radix sort: per-tile digit histogram --------------------------------
__global__ void k_radix_hist(const unsigned* __restrict__ keys, int n, int shift, int n_tiles,
                             unsigned* __restrict__ hist)
{
    __shared__ unsigned cnt[256];
    cnt[threadIdx.x] = 0;
    __syncthreads();
    const long long base = (long long)blockIdx.x * kSortTile;
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const long long e = base + it * kSortThreads + threadIdx.x;
        if (e < n) atomicAdd(&cnt[(keys[e] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(long long)threadIdx.x * n_tiles + blockIdx.x] = cnt[threadIdx.x];
}

// ---- device-wide exclusive scan of 32-bit counts --------------------------
// Tiles of kScanThreads threads x kScanPer consecutive elements.  Pass 1 sums
// each tile, pass 2 scans the tile sums in one block, pass 3 rescans every tile
// from its offset.  A whole tile moves as 16-byte vectors (the arrays come from
// cudaMalloc, so a tile start is 16-byte aligned).  In place (in == out) is
// fine: a tile is read before it is written, and only by its own block.
constexpr int kScanThreads = 256, kScanPer = 16, kScanTile = kScanThreads * kScanPer;

__device__ __forceinline__ void scan_load(const unsigned* __restrict__ in, long long n, long long i0,
                                          unsigned (&v)[kScanPer])
{
    if (i0 + kScanPer <= n) {
        const uint4* p = reinterpret_cast<const uint4*>(in + i0);
#pragma unroll
        for (int q = 0; q < kScanPer / 4; ++q) {
            const uint4 w = p[q];
            v[4 * q] = w.x; v[4 * q + 1] = w.y; v[4 * q + 2] = w.z; v[4 * q + 3] = w.w;
        }
    } else {
#pragma unroll
        for (int k = 0; k < kScanPer; ++k) v[k] = i0 + k < n ? in[i0 + k] : 0u;
    }
}

// Exclusive prefix of x over the block (kScanThreads threads); *sum gets the block total.
__device__ __forceinline__ unsigned block_exclusive(unsigned x, unsigned* s_warp, unsigned& sum)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned incl = x;
    for (int off = 1; off < 32; off <<= 1) {
        const unsigned y = __shfl_up_sync(0xFFFFFFFFu, incl, off);
        if (lane >= off) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    unsigned before = 0, tot = 0;
    for (int w = 0; w < kScanThreads / 32; ++w) {
        const unsigned t = s_warp[w];
        before += w < warp ? t : 0u;
        tot += t;
    }
    sum = tot;
    return before + incl - x;
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_tiles(const unsigned* __restrict__ in, long long n, unsigned* __restrict__ part)
{
    __shared__ unsigned s_warp[kScanThreads / 32];
    unsigned v[kScanPer];
    scan_load(in, n, (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanPer, v);
    unsigned t = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) t += v[k];
    unsigned sum;
    block_exclusive(t, s_warp, sum);
    if (threadIdx.x == 0) part[blockIdx.x] = sum;
}

// One block: exclusive scan of the nb tile sums in place; the grand total to *total.
__global__ void k_scan_parts(unsigned* __restrict__ part, long long nb, unsigned* __restrict__ total)
{
    __shared__ unsigned sums[1024];
    const long long per = (nb + blockDim.x - 1) / blockDim.x;
    const long long lo = threadIdx.x * per, hi = lo + per < nb ? lo + per : nb;
    unsigned t = 0;
    for (long long i = lo; i < hi; ++i) t += part[i];
    sums[threadIdx.x] = t;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const unsigned v = threadIdx.x >= (unsigned)off ? sums[threadIdx.x - off] : 0u;
        __syncthreads();
        sums[threadIdx.x] += v;
        __syncthreads();
    }
    unsigned run = sums[threadIdx.x] - t;
    for (long long i = lo; i < hi; ++i) {
        const unsigned v = part[i];
        part[i] = run;
        run += v;
    }
    if (total && threadIdx.x == blockDim.x - 1) *total = sums[threadIdx.x];
}

__global__ void __launch_bounds__(kScanThreads)
k_scan_apply(const unsigned* in, unsigned* out, long long n, const unsigned* __restrict__ part)
{
    __shared__ unsigned s_warp[kScanThreads / 32];
    const long long i0 = (long long)blockIdx.x * kScanTile + (long long)threadIdx.x * kScanPer;
    unsigned v[kScanPer];
    scan_load(in, n, i0, v);
    unsigned t = 0;
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) t += v[k];
    unsigned sum;
    unsigned run = part[blockIdx.x] + block_exclusive(t, s_warp, sum);
#pragma unroll
    for (int k = 0; k < kScanPer; ++k) {
        const unsigned x = v[k];
        v[k] = run;
        run += x;
    }
    if (i0 + kScanPer <= n) {
        uint4* p = reinterpret_cast<uint4*>(out + i0);
#pragma unroll
        for (int q = 0; q < kScanPer / 4; ++q) p[q] = make_uint4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < kScanPer; ++k)
            if (i0 + k < n) out[i0 + k] = v[k];
    }
}

// ---- radix sort: stable scatter ------------------------------------------
// Element e = tile*1024 + it*256 + warp*32 + lane.  Its rank among equal
// digits of the tile = (equal digits in earlier (it, warp) slots) + (equal
// digits in lower lanes of its own warp, from __match_any_sync).
__global__ void __launch_bounds__(kSortThreads)
k_radix_scatter(const unsigned* __restrict__ kin, const unsigned* __restrict__ vin,
                unsigned* __restrict__ kout, unsigned* __restrict__ vout, int n, int shift,
                int n_tiles, const unsigned* __restrict__ hist)
{
    constexpr int kSlots = kSortItems * (kSortThreads / 32);
    __shared__ unsigned cnt[kSlots][256];
    for (int i = threadIdx.x; i < kSlots * 256; i += kSortThreads) (&cnt[0][0])[i] = 0u;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    const long long base = (long long)blockIdx.x * kSortTile;
    unsigned key[kSortItems], val[kSortItems], dig[kSortItems], rank[kSortItems];
    bool ok[kSortItems];
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        const long long e = base + it * kSortThreads + threadIdx.x;
        ok[it] = e < n;
        key[it] = ok[it] ? kin[e] : 0u;
        val[it] = ok[it] ? vin[e] : 0u;
        dig[it] = (key[it] >> shift) & 255u;
        const unsigned tag = ok[it] ? dig[it] : 0x100u;
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, tag);
        rank[it] = __popc(peers & lt);
        if (ok[it] && (peers & lt) == 0u) cnt[it * (kSortThreads / 32) + warp][dig[it]] = __popc(peers);
    }
    __syncthreads();
    {   // exclusive prefix over the (it, warp) slots, one digit per thread
        const int d = threadIdx.x;
        unsigned run = 0;
        for (int s = 0; s < kSlots; ++s) {
            const unsigned v = cnt[s][d];
            cnt[s][d] = run;
            run += v;
        }
    }
    __syncthreads();
#pragma unroll
    for (int it = 0; it < kSortItems; ++it) {
        if (!ok[it]) continue;
        const unsigned pos = hist[(long long)dig[it] * n_tiles + blockIdx.x] +
                             cnt[it * (kSortThreads / 32) + warp][dig[it]] + rank[it];
        kout[pos] = key[it];
        vout[pos] = val[it];
    }
}

// ---- Karras hierarchy ------------------------------------------------------
__device__ __forceinline__ int common_prefix(const unsigned* __restrict__ k, int n, int i, int j)
{
    if (j < 0 || j >= n) return -1;
    const unsigned a = k[i], b = k[j];
    if (a == b) return 32 + __clz((unsigned)(i ^ j));
    return __clz(a ^ b);
}

__global__ void k_karras(const unsigned* __restrict__ keys, int n, int2* __restrict__ child,
                         int2* __restrict__ range, int* __restrict__ parent, int* __restrict__ leaf_parent)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n - 1) return;
    const int d = (common_prefix(keys, n, i, i + 1) - common_prefix(keys, n, i, i - 1)) >= 0 ? 1 : -1;
    const int dmin = common_prefix(keys, n, i, i - d);
    int lmax = 2;
    while (common_prefix(keys, n, i, i + lmax * d) > dmin) lmax *= 2;
    int l = 0;
    for (int t = lmax / 2; t >= 1; t /= 2)
        if (common_prefix(keys, n, i, i + (l + t) * d) > dmin) l += t;
    const int j = i + l * d;
    const int dnode = common_prefix(keys, n, i, j);
    int s = 0;
    for (int div = 2;; div *= 2) {
        const int t = (l + div - 1) / div;
        if (common_prefix(keys, n, i, i + (s + t) * d) > dnode) s += t;
        if (t <= 1) break;
    }
    const int gamma = i + s * d + min(d, 0);
    const int lo = min(i, j), hi = max(i, j);
    const int left = (lo == gamma) ? ~gamma : gamma;
    const int right = (hi == gamma + 1) ? ~(gamma + 1) : gamma + 1;
    child[i] = make_int2(left, right);
    range[i] = make_int2(lo, hi);
    if (left < 0) leaf_parent[~left] = i; else parent[left] = i;
    if (right < 0) leaf_parent[~right] = i; else parent[right] = i;
    if (i == 0) parent[0] = -1;
}

struct Box3 { float3 lo, hi; };

// A box widened outward by m on every face, rounded outward.  Every stored
// child box carries m = M 2^-22 (M the largest cell coordinate): the 4-wide
// slab test evaluates planes with one FMA and relies on it, and for every
// format it keeps a ray with a zero direction component that lies in a face
// plane of a box inside the box (a slab test of such a ray sees the face at
// distance 0 and would reject the box).
__device__ __forceinline__ Box3 widen(const Box3& b, float m)
{
    Box3 w;
    w.lo = make_float3(__fsub_rd(b.lo.x, m), __fsub_rd(b.lo.y, m), __fsub_rd(b.lo.z, m));
    w.hi = make_float3(__fadd_ru(b.hi.x, m), __fadd_ru(b.hi.y, m), __fadd_ru(b.hi.z, m));
    return w;
}

__device__ __forceinline__ Box3 tri_box(const float* __restrict__ tri, unsigned t)
{
    const float* p = tri + 9ll * t;
    Box3 b;
    b.lo = make_float3(fminf(fminf(p[0], p[3]), p[6]), fminf(fminf(p[1], p[4]), p[7]),
                       fminf(fminf(p[2], p[5]), p[8]));
    b.hi = make_float3(fmaxf(fmaxf(p[0], p[3]), p[6]), fmaxf(fmaxf(p[1], p[4]), p[7]),
                       fmaxf(fmaxf(p[2], p[5]), p[8]));
    return b;
}

__device__ __forceinline__ void store_node(float4* __restrict__ nodes, int i, const Box3& b0,
                                           const Box3& b1, int c0, int c1)
{
    float4* nd = nodes + 4ll * i;
    nd[0] = make_float4(b0.lo.x, b0.hi.x, b0.lo.y, b0.hi.y);
    nd[1] = make_float4(b1.lo.x, b1.hi.x, b1.lo.y, b1.hi.y);
    nd[2] = make_float4(b0.lo.z, b0.hi.z, b1.lo.z, b1.hi.z);
    nd[3] = make_float4(__int_as_float(c0), __int_as_float(c1), 0.f, 0.f);
}

// Child reference stored in a node: an inner node index (>= 0), or a leaf
// ~((first << 3) | (count - 1)) covering `count` <= 8 consecutive triangles of
// the leaf order.  A Karras inner node covers a contiguous key range, so an
// inner child whose range holds at most `leaf_max` triangles is stored as one
// leaf over that range.
__device__ __forceinline__ int child_ref(int c, const int2* __restrict__ range, int leaf_max)
{
    if (c < 0) return ~((~c) << 3);
    const int2 r = range[c];
    const int cnt = r.y - r.x + 1;
    if (cnt <= leaf_max) return ~((r.x << 3) | (cnt - 1));
    return c;
}

__global__ void k_refit(const float* __restrict__ tri, const unsigned* __restrict__ order, int n,
                        const int2* __restrict__ child, const int2* __restrict__ range,
                        const int* __restrict__ parent, const int* __restrict__ leaf_parent,
                        unsigned* __restrict__ flag, float4* __restrict__ aabb, float4* __restrict__ nodes,
                        int leaf_max, float margin)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int node = leaf_parent[j];
    for (int level = 0; node >= 0 && level < 256; ++level) {   // depth is far below 256
        if (atomicAdd(&flag[node], 1u) == 0u) return;    // the sibling is not done yet
        const int2 c = child[node];
        Box3 b[2];
        const int cc[2] = {c.x, c.y};
#pragma unroll
        for (int s = 0; s < 2; ++s) {
            if (cc[s] < 0) {
                b[s] = tri_box(tri, order[~cc[s]]);
            } else {
                const float4 lo = __ldcg(aabb + 2ll * cc[s]);
                const float4 hi = __ldcg(aabb + 2ll * cc[s] + 1);
                b[s].lo = make_float3(lo.x, lo.y, lo.z);
                b[s].hi = make_float3(hi.x, hi.y, hi.z);
            }
        }
        store_node(nodes, node, widen(b[0], margin), widen(b[1], margin), child_ref(c.x, range, leaf_max),
                   child_ref(c.y, range, leaf_max));
        __stcg(aabb + 2ll * node, make_float4(fminf(b[0].lo.x, b[1].lo.x), fminf(b[0].lo.y, b[1].lo.y),
                                              fminf(b[0].lo.z, b[1].lo.z), 0.f));
        __stcg(aabb + 2ll * node + 1, make_float4(fmaxf(b[0].hi.x, b[1].hi.x), fmaxf(b[0].hi.y, b[1].hi.y),
                                                  fmaxf(b[0].hi.z, b[1].hi.z), 0.f));
        __threadfence();
        node = parent[node];
    }
}

// A one-triangle mesh: the root's two children are the same leaf (the repeat
// test cannot change the closest hit).
__global__ void k_single_leaf(const float* __restrict__ tri, float4* __restrict__ nodes, float margin)
{
    const Box3 b = widen(tri_box(tri, 0), margin);
    store_node(nodes, 0, b, b, ~0, ~0);
}

// ---- Q8 nodes: 8-bit child boxes, outward rounded -------------------------
// The frame of node i is its own box.  Per axis it stores a power-of-two
// scale s = 2^e (biased exponent e + 127 in one byte) and a shifted origin
// o' = lo - 2^23 s rounded down.  A child bound q decodes with one FMA,
// fmaf(M(q), s, o'), where M(q) = 2^23 + q is the float with bit pattern
// 0x4B0000qq, so the traversal needs one byte permute and one FMA per bound.
// Decode(0) <= lo by construction; e is the smallest exponent with
// decode(255) >= hi.  Lower bounds are rounded down and upper bounds up,
// checked with this same FP32 decode, so a decoded child box always contains
// the exact one.
__device__ __forceinline__ float q8_decode(unsigned q, float s, float o_shift)
{
    return fmaf(__int_as_float(0x4B000000 | (int)q), s, o_shift);
}

__device__ __forceinline__ float q8_shift(float lo, float s) { return __fsub_rd(lo, 8388608.0f * s); }

// 2^23 s stays finite (coordinates up to about 2^100 fit a frame)
constexpr int kQ8MaxExp = 100;

__device__ int frame_exponent(float lo, float hi)
{
    const float ext = hi - lo;
    int e = -126;
    if (ext > 0.f) {
        e = (int)ceilf(log2f(ext / 255.0f));
        e = max(-126, min(e, kQ8MaxExp));
    }
    while (e < kQ8MaxExp && q8_decode(255u, exp2_int(e), q8_shift(lo, exp2_int(e))) < hi) ++e;
    return e;
}

__device__ unsigned quant_lo(float v, float o_shift, float sc)
{
    int q = (int)floorf((v - q8_decode(0u, sc, o_shift)) / sc);
    q = max(0, min(q, 255));
    while (q > 0 && q8_decode((unsigned)q, sc, o_shift) > v) --q;
    return (unsigned)q;
}

__device__ unsigned quant_hi(float v, float o_shift, float sc)
{
    int q = (int)ceilf((v - q8_decode(0u, sc, o_shift)) / sc);
    q = max(0, min(q, 255));
    while (q < 255 && q8_decode((unsigned)q, sc, o_shift) < v) ++q;
    return (unsigned)q;
}

__device__ void child_info(int raw, const float* __restrict__ tri, const unsigned* __restrict__ order,
                           const int2* __restrict__ range, const float4* __restrict__ aabb, int leaf_max,
                           float margin, Box3& b, bool& leaf, int& count)
{
    if (raw < 0) {
        b = widen(tri_box(tri, order[~raw]), margin);
        leaf = true;
        count = 1;
        return;
    }
    const float4 lo = __ldcg(aabb + 2ll * raw), hi = __ldcg(aabb + 2ll * raw + 1);
    b.lo = make_float3(lo.x, lo.y, lo.z);
    b.hi = make_float3(hi.x, hi.y, hi.z);
    b = widen(b, margin);
    const int2 r = range[raw];
    count = r.y - r.x + 1;
    leaf = count <= leaf_max;
}

__global__ void k_quantize(const float* __restrict__ tri, const unsigned* __restrict__ order, int n_inner,
                           const int2* __restrict__ child, const int2* __restrict__ range,
                           const float4* __restrict__ aabb, int leaf_max, float margin, uint4* __restrict__ q8)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n_inner) return;
    const int2 c = child[i];
    Box3 b[2];
    bool leaf[2];
    int count[2];
    child_info(c.x, tri, order, range, aabb, leaf_max, margin, b[0], leaf[0], count[0]);
    child_info(c.y, tri, order, range, aabb, leaf_max, margin, b[1], leaf[1], count[1]);
    const int gamma = c.x < 0 ? ~c.x : c.x;
    const float3 plo = make_float3(fminf(b[0].lo.x, b[1].lo.x), fminf(b[0].lo.y, b[1].lo.y), fminf(b[0].lo.z, b[1].lo.z));
    const float3 phi = make_float3(fmaxf(b[0].hi.x, b[1].hi.x), fmaxf(b[0].hi.y, b[1].hi.y), fmaxf(b[0].hi.z, b[1].hi.z));
    const int ex = frame_exponent(plo.x, phi.x), ey = frame_exponent(plo.y, phi.y), ez = frame_exponent(plo.z, phi.z);
    const float sx = exp2_int(ex), sy = exp2_int(ey), sz = exp2_int(ez);
    const float ox = q8_shift(plo.x, sx), oy = q8_shift(plo.y, sy), oz = q8_shift(plo.z, sz);
    unsigned qb[12];
    for (int k = 0; k < 2; ++k) {
        qb[6 * k + 0] = quant_lo(b[k].lo.x, ox, sx);
        qb[6 * k + 1] = quant_lo(b[k].lo.y, oy, sy);
        qb[6 * k + 2] = quant_lo(b[k].lo.z, oz, sz);
        qb[6 * k + 3] = quant_hi(b[k].hi.x, ox, sx);
        qb[6 * k + 4] = quant_hi(b[k].hi.y, oy, sy);
        qb[6 * k + 5] = quant_hi(b[k].hi.z, oz, sz);
    }
    const unsigned meta = (leaf[0] ? 1u : 0u) | ((unsigned)(leaf[0] ? count[0] - 1 : 0) << 1) |
                          (leaf[1] ? 16u : 0u) | ((unsigned)(leaf[1] ? count[1] - 1 : 0) << 5);
    const unsigned packed = (unsigned)(ex + 127) | ((unsigned)(ey + 127) << 8) | ((unsigned)(ez + 127) << 16) |
                            (meta << 24);
    q8[2ll * i] = make_uint4(__float_as_uint(ox), __float_as_uint(oy), __float_as_uint(oz), packed);
    q8[2ll * i + 1] = make_uint4(qb[0] | qb[1] << 8 | qb[2] << 16 | qb[3] << 24,
                                 qb[4] | qb[5] << 8 | qb[6] << 16 | qb[7] << 24,
                                 qb[8] | qb[9] << 8 | qb[10] << 16 | qb[11] << 24, (unsigned)gamma);
}

// One-triangle mesh in Q8 form: left leaf = triangle 0, right leaf = the
// degenerate padding triangle 1 (never hit).
__global__ void k_quantize_single(const float* __restrict__ tri, float margin, uint4* __restrict__ q8)
{
    const Box3 b = widen(tri_box(tri, 0), margin);
    const int ex = frame_exponent(b.lo.x, b.hi.x), ey = frame_exponent(b.lo.y, b.hi.y), ez = frame_exponent(b.lo.z, b.hi.z);
    const unsigned meta = 1u | 16u;
    const unsigned packed = (unsigned)(ex + 127) | ((unsigned)(ey + 127) << 8) | ((unsigned)(ez + 127) << 16) |
                            (meta << 24);
    q8[0] = make_uint4(__float_as_uint(q8_shift(b.lo.x, exp2_int(ex))), __float_as_uint(q8_shift(b.lo.y, exp2_int(ey))),
                       __float_as_uint(q8_shift(b.lo.z, exp2_int(ez))), packed);
    q8[1] = make_uint4(0xFF000000u, 0x0000FFFFu, 0x00000000u, 0u);   // c0 = [0,255]^3, c1 = [0,0]^3
}

__global__ void k_pack(const float* __restrict__ tri, const unsigned* __restrict__ order, int n,
                       float4* __restrict__ tris, float4* __restrict__ normals,
                       int* __restrict__ inv_order)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j == n) {   // degenerate padding triangle after the last leaf (never hit)
        const float* p0 = tri;
        const float4 v = make_float4(p0[0], p0[1], p0[2], __int_as_float(-1));
        tris[3ll * n + 0] = v;
        tris[3ll * n + 1] = make_float4(v.x, v.y, v.z, 0.f);
        tris[3ll * n + 2] = make_float4(v.x, v.y, v.z, 0.f);
        normals[n] = make_float4(0.f, 0.f, 1.f, 0.f);
        return;
    }
    if (j >= n) return;
    const unsigned i = order[j];
    const float* p = tri + 9ll * i;
    tris[3ll * j + 0] = make_float4(p[0], p[1], p[2], __int_as_float((int)i));
    tris[3ll * j + 1] = make_float4(p[3], p[4], p[5], 0.f);
    tris[3ll * j + 2] = make_float4(p[6], p[7], p[8], 0.f);
    const float l1x = p[3] - p[0], l1y = p[4] - p[1], l1z = p[5] - p[2];
    const float l2x = p[6] - p[0], l2y = p[7] - p[1], l2z = p[8] - p[2];
    const float nx = l1y * l2z - l1z * l2y, ny = l1z * l2x - l1x * l2z, nz = l1x * l2y - l1y * l2x;
    const float inv = 1.0f / sqrtf(nx * nx + ny * ny + nz * nz);
    normals[j] = make_float4(nx * inv, ny * inv, nz * inv, 0.f);
    inv_order[i] = j;
}

__global__ void k_depth(const int* __restrict__ parent, const int* __restrict__ leaf_parent, int n,
                        int* __restrict__ depth)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int d = 1, node = leaf_parent[j];
    while (node >= 0 && d < 1000) { ++d; node = parent[node]; }
    atomicMax(depth, d);
}

// ---- PLOC hierarchy (Meister & Bittner, "Parallel Locally-Ordered
// Clustering for Bounding Volume Hierarchy Construction", TVCG 2018) --------
// Clusters start as the Morton-sorted triangles.  Each round, every cluster
// finds the neighbour within +-kPlocRadius positions whose union box has the
// smallest surface area (ties: the lower position, which makes the choice a
// total order on pairs, so the globally best pair is always mutual and every
// round merges at least once); mutual pairs merge into a new node kept at the
// lower position, and the surviving clusters are compacted in order.  Node
// ids: leaves 0..n-1 (sorted positions), inner nodes n..2n-2 in creation
// order, so the root is 2n-2.  The finished tree is rewritten into the Karras
// layout the rest of the builder consumes (see k_ploc_emit).
constexpr int kPlocRadius = 16;
constexpr int kPlocBlock = 256;

struct PlocState {
    int count;      // clusters after the round
    int created;    // inner nodes created so far
};

__device__ __forceinline__ float half_area(float3 lo, float3 hi)
{
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

__global__ void k_ploc_init(const float* __restrict__ tri, const unsigned* __restrict__ sorted, int n,
                            int* __restrict__ cl_node, float4* __restrict__ cl_lo, float4* __restrict__ cl_hi,
                            int* __restrict__ cnt)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const Box3 b = tri_box(tri, sorted[i]);
    cl_node[i] = i;
    cl_lo[i] = make_float4(b.lo.x, b.lo.y, b.lo.z, 0.f);
    cl_hi[i] = make_float4(b.hi.x, b.hi.y, b.hi.z, 0.f);
    cnt[i] = 1;
}

__global__ void __launch_bounds__(kPlocBlock)
k_ploc_nn(const float4* __restrict__ cl_lo, const float4* __restrict__ cl_hi, int c, int* __restrict__ nn)
{
    __shared__ float4 s_lo[kPlocBlock + 2 * kPlocRadius], s_hi[kPlocBlock + 2 * kPlocRadius];
    const int b0 = blockIdx.x * kPlocBlock;
    for (int t = threadIdx.x; t < kPlocBlock + 2 * kPlocRadius; t += kPlocBlock) {
        const int g = b0 - kPlocRadius + t;
        if (g >= 0 && g < c) { s_lo[t] = cl_lo[g]; s_hi[t] = cl_hi[g]; }
    }
    __syncthreads();
    const int i = b0 + threadIdx.x;
    if (i >= c) return;
    const int li = threadIdx.x + kPlocRadius;
    const float4 alo = s_lo[li], ahi = s_hi[li];
    float best = INFINITY;
    int bj = -1;
    for (int dj = -kPlocRadius; dj <= kPlocRadius; ++dj) {
        const int j = i + dj;
        if (dj == 0 || j < 0 || j >= c) continue;
        const float4 blo = s_lo[li + dj], bhi = s_hi[li + dj];
        const float a = half_area(make_float3(fminf(alo.x, blo.x), fminf(alo.y, blo.y), fminf(alo.z, blo.z)),
                                  make_float3(fmaxf(ahi.x, bhi.x), fmaxf(ahi.y, bhi.y), fmaxf(ahi.z, bhi.z)));
        if (a < best) { best = a; bj = j; }       // increasing j: ties keep the lower position
    }
    nn[i] = bj;
}

// Per block: number of surviving clusters and of merges it starts.
__device__ __forceinline__ void ploc_flags(const int* __restrict__ nn, int c, int i, bool& keep, bool& make)
{
    keep = false;
    make = false;
    if (i >= c) return;
    const int j = nn[i];
    const bool mutual = j >= 0 && nn[j] == i;
    keep = !(mutual && j < i);        // the upper member of a mutual pair is absorbed
    make = mutual && i < j;
}

__global__ void __launch_bounds__(kPlocBlock)
k_ploc_count(const int* __restrict__ nn, int c, int2* __restrict__ block_counts)
{
    __shared__ int s_k[kPlocBlock / 32], s_m[kPlocBlock / 32];
    const int i = blockIdx.x * kPlocBlock + threadIdx.x;
    bool keep, make;
    ploc_flags(nn, c, i, keep, make);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int k = __popc(__ballot_sync(0xFFFFFFFFu, keep)), m = __popc(__ballot_sync(0xFFFFFFFFu, make));
    if (lane == 0) { s_k[w] = k; s_m[w] = m; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int tk = 0, tm = 0;
        for (int q = 0; q < kPlocBlock / 32; ++q) { tk += s_k[q]; tm += s_m[q]; }
        block_counts[blockIdx.x] = make_int2(tk, tm);
    }
}

// Exclusive scan of the per-block (keep, make) counts, one block; the totals
// go to the state (new cluster count; inner nodes created).
__global__ void k_ploc_scan(int2* __restrict__ block_counts, int n_blocks, PlocState* __restrict__ st)
{
    __shared__ int2 sums[1024];
    const int per = (n_blocks + (int)blockDim.x - 1) / (int)blockDim.x;
    const int lo = threadIdx.x * per, hi = min(lo + per, n_blocks);
    int2 s = make_int2(0, 0);
    for (int b = lo; b < hi; ++b) { s.x += block_counts[b].x; s.y += block_counts[b].y; }
    sums[threadIdx.x] = s;
    __syncthreads();
    for (int off = 1; off < (int)blockDim.x; off <<= 1) {
        const int2 v = threadIdx.x >= (unsigned)off ? sums[threadIdx.x - off] : make_int2(0, 0);
        __syncthreads();
        sums[threadIdx.x].x += v.x;
        sums[threadIdx.x].y += v.y;
        __syncthreads();
    }
    int2 run = make_int2(sums[threadIdx.x].x - s.x, sums[threadIdx.x].y - s.y);
    for (int b = lo; b < hi; ++b) {
        const int2 v = block_counts[b];
        block_counts[b] = run;
        run.x += v.x;
        run.y += v.y;
    }
    if (threadIdx.x == blockDim.x - 1) {
        st->count = sums[threadIdx.x].x;
        st->created += sums[threadIdx.x].y;
    }
}

__global__ void __launch_bounds__(kPlocBlock)
k_ploc_merge(const int* __restrict__ nn, int c, const int2* __restrict__ block_off, int first_id,
             const int* __restrict__ cl_node, const float4* __restrict__ cl_lo, const float4* __restrict__ cl_hi,
             int* __restrict__ out_node, float4* __restrict__ out_lo, float4* __restrict__ out_hi,
             int2* __restrict__ kids, int* __restrict__ parent, int* __restrict__ cnt)
{
    __shared__ int s_k[kPlocBlock / 32], s_m[kPlocBlock / 32];
    const int i = blockIdx.x * kPlocBlock + threadIdx.x;
    bool keep, make;
    ploc_flags(nn, c, i, keep, make);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned bk = __ballot_sync(0xFFFFFFFFu, keep), bm = __ballot_sync(0xFFFFFFFFu, make);
    if (lane == 0) { s_k[w] = __popc(bk); s_m[w] = __popc(bm); }
    __syncthreads();
    int ok = block_off[blockIdx.x].x, om = block_off[blockIdx.x].y;
    for (int q = 0; q < w; ++q) { ok += s_k[q]; om += s_m[q]; }
    const unsigned lt = (1u << lane) - 1u;
    ok += __popc(bk & lt);
    om += __popc(bm & lt);
    if (!keep) return;
    if (make) {
        const int j = nn[i];
        const int a = cl_node[i], b = cl_node[j], id = first_id + om;
        const float4 alo = cl_lo[i], ahi = cl_hi[i], blo = cl_lo[j], bhi = cl_hi[j];
        kids[id] = make_int2(a, b);               // lower position on the left: leaves stay in Morton order
        parent[a] = id;
        parent[b] = id;
        cnt[id] = cnt[a] + cnt[b];
        out_node[ok] = id;
        out_lo[ok] = make_float4(fminf(alo.x, blo.x), fminf(alo.y, blo.y), fminf(alo.z, blo.z), 0.f);
        out_hi[ok] = make_float4(fmaxf(ahi.x, bhi.x), fmaxf(ahi.y, bhi.y), fmaxf(ahi.z, bhi.z), 0.f);
    } else {
        out_node[ok] = cl_node[i];
        out_lo[ok] = cl_lo[i];
        out_hi[ok] = cl_hi[i];
    }
}

// First leaf position (depth-first, left to right) of every node: the sum of
// the left-sibling counts along the path to the root.  The climb is bounded;
// a longer path sets *bad.
__global__ void k_ploc_first(const int2* __restrict__ kids, const int* __restrict__ parent,
                             const int* __restrict__ cnt, int n_all, int root, int* __restrict__ first,
                             int* __restrict__ bad)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= n_all) return;
    int lo = 0, x = v, steps = 0;
    while (x != root) {
        const int p = parent[x];
        const int2 k = kids[p];
        if (x == k.y) lo += cnt[k.x];
        x = p;
        if (++steps > 4096) { atomicExch(bad, 1); break; }
    }
    first[v] = lo;
}

// Rewrite into the Karras layout: leaves by depth-first position; an inner
// node with leaf range [lo, hi] gets index hi if it is a left child, lo if it
// is a right child, 0 if it is the root.  For any binary tree these indices
// are distinct and fill [0, n-2], and the children of index g are g and g+1
// (as leaves or inner nodes) -- the Karras (HPG 2012) numbering, which the
// refit, the Q8 quantiser and the traversal rely on.
__device__ __forceinline__ int karras_index(const int2* __restrict__ kids, const int* __restrict__ parent,
                                            const int* __restrict__ cnt, const int* __restrict__ first,
                                            int v, int root)
{
    if (v == root) return 0;
    const int p = parent[v];
    return kids[p].x == v ? first[v] + cnt[v] - 1 : first[v];
}

__global__ void k_ploc_emit(const int2* __restrict__ kids, const int* __restrict__ parent_all,
                            const int* __restrict__ cnt, const int* __restrict__ first,
                            const unsigned* __restrict__ sorted, int n, int root,
                            int2* __restrict__ child, int2* __restrict__ range, int* __restrict__ parent,
                            int* __restrict__ leaf_parent, unsigned* __restrict__ order)
{
    const int v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < n) {                                   // leaf: its triangle at its depth-first position
        order[first[v]] = sorted[v];
        return;
    }
    if (v >= 2 * n - 1) return;
    const int g = karras_index(kids, parent_all, cnt, first, v, root);
    const int2 k = kids[v];
    int ref[2];
    const int cs[2] = {k.x, k.y};
#pragma unroll
    for (int s = 0; s < 2; ++s) {
        const int c = cs[s];
        if (c < n) {
            ref[s] = ~first[c];
            leaf_parent[first[c]] = g;
        } else {
            ref[s] = karras_index(kids, parent_all, cnt, first, c, root);
            parent[ref[s]] = g;
        }
    }
    child[g] = make_int2(ref[0], ref[1]);
    range[g] = make_int2(first[v], first[v] + cnt[v] - 1);
    if (v == root) parent[0] = -1;
}

// ---- 4-wide nodes, collapsed from the finished binary hierarchy ------------
// Each 4-wide node stands for one binary inner node b: it starts from b's two
// children and, while it has fewer than four, opens the inner child with the
// largest box surface area (a child that collapses into a leaf stays closed).
// Level by level: count the inner children of every node of the frontier,
// scan, then write the nodes and the next frontier, so the numbering is
// deterministic (root 0, then level order).
constexpr int kW4Block = 256;

__device__ __forceinline__ float box_area(float4 lo, float4 hi)
{
    const float dx = hi.x - lo.x, dy = hi.y - lo.y, dz = hi.z - lo.z;
    return dx * dy + dy * dz + dz * dx;
}

__device__ __forceinline__ bool w4_open(int raw, const int2* __restrict__ range, int leaf_max)
{
    if (raw < 0) return false;
    const int2 r = range[raw];
    return r.y - r.x + 1 > leaf_max;
}

__device__ int w4_expand(int b, const int2* __restrict__ child, const int2* __restrict__ range,
                         const float4* __restrict__ aabb, int leaf_max, int (&raw)[4])
{
    const int2 c = child[b];
    raw[0] = c.x;
    raw[1] = c.y;
    raw[2] = raw[3] = -1;
    int n = 2;
    while (n < 4) {
        int best = -1;
        float ba = -1.f;
        for (int k = 0; k < n; ++k) {
            if (!w4_open(raw[k], range, leaf_max)) continue;
            const float a = box_area(aabb[2ll * raw[k]], aabb[2ll * raw[k] + 1]);
            if (a > ba) { ba = a; best = k; }
        }
        if (best < 0) break;
        const int2 cc = child[raw[best]];
        raw[best] = cc.x;
        raw[n++] = cc.y;
    }
    return n;
}

__global__ void k_w4_count(const int2* __restrict__ front, int nf, const int2* __restrict__ child,
                           const int2* __restrict__ range, const float4* __restrict__ aabb, int leaf_max,
                           int* __restrict__ cnt)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    int raw[4];
    const int n = w4_expand(front[f].x, child, range, aabb, leaf_max, raw);
    int m = 0;
    for (int k = 0; k < n; ++k) m += w4_open(raw[k], range, leaf_max) ? 1 : 0;
    cnt[f] = m;
}

__device__ __forceinline__ void w4_store(float4* __restrict__ w4, int w, const Box3 (&b)[4], const int (&ref)[4])
{
    float4* nd = w4 + 8ll * w;
    nd[0] = make_float4(b[0].lo.x, b[1].lo.x, b[2].lo.x, b[3].lo.x);
    nd[1] = make_float4(b[0].hi.x, b[1].hi.x, b[2].hi.x, b[3].hi.x);
    nd[2] = make_float4(b[0].lo.y, b[1].lo.y, b[2].lo.y, b[3].lo.y);
    nd[3] = make_float4(b[0].hi.y, b[1].hi.y, b[2].hi.y, b[3].hi.y);
    nd[4] = make_float4(b[0].lo.z, b[1].lo.z, b[2].lo.z, b[3].lo.z);
    nd[5] = make_float4(b[0].hi.z, b[1].hi.z, b[2].hi.z, b[3].hi.z);
    nd[6] = make_float4(__int_as_float(ref[0]), __int_as_float(ref[1]), __int_as_float(ref[2]),
                        __int_as_float(ref[3]));
    nd[7] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_w4_emit(const int2* __restrict__ front, int nf, const int* __restrict__ off, int base,
                          const int2* __restrict__ child, const int2* __restrict__ range,
                          const float4* __restrict__ aabb, const float* __restrict__ tri,
                          const unsigned* __restrict__ order, int leaf_max, float margin, float4* __restrict__ w4,
                          int2* __restrict__ next)
{
    const int f = blockIdx.x * blockDim.x + threadIdx.x;
    if (f >= nf) return;
    const int2 fw = front[f];
    int raw[4];
    const int n = w4_expand(fw.x, child, range, aabb, leaf_max, raw);
    Box3 b[4];
    int ref[4];
    int j = 0;
    for (int k = 0; k < 4; ++k) {
        if (k >= n) {                                  // empty slot: a box no ray can hit
            b[k].lo = b[k].hi = make_float3(INFINITY, INFINITY, INFINITY);
            ref[k] = kEmptyChild;
            continue;
        }
        const int r = raw[k];
        if (r < 0) {                                   // single triangle at leaf position ~r
            b[k] = widen(tri_box(tri, order[~r]), margin);
            ref[k] = ~((~r) << 3);
            continue;
        }
        const float4 lo = aabb[2ll * r], hi = aabb[2ll * r + 1];
        b[k].lo = make_float3(lo.x, lo.y, lo.z);
        b[k].hi = make_float3(hi.x, hi.y, hi.z);
        b[k] = widen(b[k], margin);
        const int2 rg = range[r];
        const int c = rg.y - rg.x + 1;
        if (c <= leaf_max) {
            ref[k] = ~((rg.x << 3) | (c - 1));
        } else {
            const int slot = off[f] + j++;
            ref[k] = base + slot;
            next[slot] = make_int2(r, base + slot);
        }
    }
    w4_store(w4, fw.y, b, ref);
}

// One-triangle mesh: the root holds the single leaf.
__global__ void k_w4_single(const float* __restrict__ tri, float margin, float4* __restrict__ w4)
{
    Box3 b[4];
    int ref[4];
    b[0] = widen(tri_box(tri, 0), margin);
    ref[0] = ~0;
    for (int k = 1; k < 4; ++k) {
        b[k].lo = b[k].hi = make_float3(INFINITY, INFINITY, INFINITY);
        ref[k] = kEmptyChild;
    }
    w4_store(w4, 0, b, ref);
}

// ---- 4-wide nodes quantised to 8 bits ---------------------------------------
// Per axis a quantum s = 2^e and an integer frame start m (origin m s); child
// plane codes q in [0, 255] stand for (m + q) s.  The traversal evaluates a
// plane as fmaf(1 + q 2^-15, S / d, (o' - o) / d) with S = 2^15 s and
// o' = (m - 2^15) s, both exact in FP32 (|m - 2^15| < 2^24).  The product
// (1 + q 2^-15) S / d is exact inside the FMA (S is a power of two); the
// rounding of o' - o and of its quotient moves a plane by at most
// |o' - o| 2^-23 <= M 2^-22 + s 2^-8 (|m s| <= M, |o| <= M), so every plane
// is rounded outward from the FP32 4-wide box by twice that, M 2^-21 + s 2^-7,
// before it is rounded to the quantum grid -- a small fraction of a quantum
// where the shifted origin (m - 2^23) s of the 0x4B0000qq decode needed one
// whole quantum.  All of it is exact in FP64: s is a power of two, |m| < 2^23.
// Returns false when no quantum up to 2^kQ4MaxExp fits (coordinates too large).
__device__ bool q4_axis(const float4& lo_row, const float4& hi_row, const bool (&real)[4], double big,
                        float& o_shift, float& scale, unsigned& w_lo, unsigned& w_hi)
{
    const float lo[4] = {lo_row.x, lo_row.y, lo_row.z, lo_row.w};
    const float hi[4] = {hi_row.x, hi_row.y, hi_row.z, hi_row.w};
    double L = INFINITY, H = -INFINITY;
    for (int c = 0; c < 4; ++c)
        if (real[c]) { L = fmin(L, (double)lo[c]); H = fmax(H, (double)hi[c]); }
    const double span = fmax(H - L, 0.0), mag = fmax(fabs(L), fabs(H));
    int e = -126;
    if (span > 0.0) e = max(e, ilogb(span / 250.0));
    if (mag > 0.0) e = max(e, ilogb(mag) - 22);
    for (; e <= kQ4MaxExp; ++e) {
        const double sc = ldexp(1.0, e);
        const double margin = big * 0x1p-21 + sc * 0x1p-7;
        const double m = floor((L - margin) / sc);
        if (!(fabs(m) < 0x1p23) || ceil((H + margin - m * sc) / sc) > 255.0) continue;
        w_lo = w_hi = 0u;
        for (int c = 0; c < 4; ++c) {
            unsigned ql = 255u, qh = 0u;                 // empty slot: lo above hi
            if (real[c]) {
                ql = (unsigned)floor(((double)lo[c] - margin - m * sc) / sc);
                qh = (unsigned)ceil(((double)hi[c] + margin - m * sc) / sc);
            }
            w_lo |= ql << (8 * c);
            w_hi |= qh << (8 * c);
        }
        o_shift = (float)((m - 0x1p15) * sc);
        scale = (float)(sc * 0x1p15);
        return true;
    }
    return false;
}

__global__ void k_q4_quantize(const float4* __restrict__ w4, int n, double big, uint4* __restrict__ q4,
                              int* __restrict__ bad)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const float4* nd = w4 + 8ll * i;
    const float4 cr = nd[6];
    const int ref[4] = {__float_as_int(cr.x), __float_as_int(cr.y), __float_as_int(cr.z), __float_as_int(cr.w)};
    const bool real[4] = {ref[0] != kEmptyChild, ref[1] != kEmptyChild, ref[2] != kEmptyChild,
                          ref[3] != kEmptyChild};
    float o[3], sc[3];
    unsigned wl[3], wh[3];
    bool ok = true;
    for (int a = 0; a < 3; ++a) ok = q4_axis(nd[2 * a], nd[2 * a + 1], real, big, o[a], sc[a], wl[a], wh[a]) && ok;
    if (!ok) {
        atomicExch(bad, 1);
        for (int a = 0; a < 3; ++a) { o[a] = 0.f; sc[a] = 1.f; wl[a] = 0u; wh[a] = 0xFFFFFFFFu; }
    }
    q4[4ll * i + 0] = make_uint4(__float_as_uint(o[0]), __float_as_uint(o[1]), __float_as_uint(o[2]),
                                 __float_as_uint(sc[0]));
    q4[4ll * i + 1] = make_uint4(__float_as_uint(sc[1]), __float_as_uint(sc[2]), wl[0], wh[0]);
    q4[4ll * i + 2] = make_uint4(wl[1], wh[1], wl[2], wh[2]);
    q4[4ll * i + 3] = make_uint4((unsigned)ref[0], (unsigned)ref[1], (unsigned)ref[2], (unsigned)ref[3]);
}

// ---- column grid -----------------------------------------------------------
// A ray parallel to z meets only facets whose xy box contains its xy point, and
// none above its first hit: per pixel of an xy grid the facets whose box meets
// the pixel, sorted by top z, let it test those in order and stop.
constexpr int kColMaxSpan = 64;      // pixels per facet; a larger facet disables the grid
constexpr int kColSortMax = 2048;    // facets per pixel; more disables the grid

__device__ __forceinline__ bool col_range(const float4* __restrict__ tris, int j, int gx, int gy, float iwx,
                                          float iwy, int& x0, int& x1, int& y0, int& y1, float& ztop)
{
    const float4 a = tris[3ll * j], b = tris[3ll * j + 1], c = tris[3ll * j + 2];
    const float lox = fminf(a.x, fminf(b.x, c.x)), hix = fmaxf(a.x, fmaxf(b.x, c.x));
    const float loy = fminf(a.y, fminf(b.y, c.y)), hiy = fmaxf(a.y, fmaxf(b.y, c.y));
    // floor(v * iw) is monotonic in v, so a ray's pixel lies inside the range of
    // every facet whose box contains the ray's xy point (every facet it can hit)
    x0 = min(max((int)floorf(lox * iwx), 0), gx - 1);
    x1 = min(max((int)floorf(hix * iwx), 0), gx - 1);
    y0 = min(max((int)floorf(loy * iwy), 0), gy - 1);
    y1 = min(max((int)floorf(hiy * iwy), 0), gy - 1);
    ztop = fmaxf(a.z, fmaxf(b.z, c.z));
    return (x1 - x0 + 1) * (y1 - y0 + 1) <= kColMaxSpan;
}

__global__ void k_col_count(const float4* __restrict__ tris, int n, int gx, int gy, float iwx, float iwy,
                            int* __restrict__ cnt, int* __restrict__ bad)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int x0, x1, y0, y1;
    float zt;
    if (!col_range(tris, j, gx, gy, iwx, iwy, x0, x1, y0, y1, zt)) { atomicOr(bad, 1); return; }
    for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) atomicAdd(&cnt[y * gx + x], 1);
}

__global__ void k_col_fill(const float4* __restrict__ tris, int n, int gx, int gy, float iwx, float iwy,
                           int* __restrict__ cursor, uint2* __restrict__ ent)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    int x0, x1, y0, y1;
    float zt;
    if (!col_range(tris, j, gx, gy, iwx, iwy, x0, x1, y0, y1, zt)) return;
    for (int y = y0; y <= y1; ++y)
        for (int x = x0; x <= x1; ++x) {
            const int slot = atomicAdd(&cursor[y * gx + x], 1);
            ent[slot] = make_uint2((unsigned)j, __float_as_uint(zt));
        }
}

// Sort key: top z descending, then facet index ascending (a total order, so the
// lists do not depend on the order of the fill's atomics).
__device__ __forceinline__ unsigned long long col_key(uint2 e)
{
    const unsigned u = e.y;
    const unsigned ord = u ^ ((u & 0x80000000u) ? 0xFFFFFFFFu : 0x80000000u);   // float order as unsigned
    return ((unsigned long long)(~ord) << 32) | e.x;
}

__device__ __forceinline__ uint2 col_unkey(unsigned long long k)
{
    const unsigned ord = ~(unsigned)(k >> 32);
    const unsigned u = (ord & 0x80000000u) ? (ord ^ 0x80000000u) : ~ord;
    return make_uint2((unsigned)k, u);
}

// Pixel lists of up to kRankSortMax entries: one warp per pixel (grid-stride,
// pixels in order) loads the list into shared memory and every lane ranks its
// R keys against all of them (rank = number of smaller keys; the keys are
// distinct, so the ranks are a permutation), then writes each entry to its
// rank.  About L^2 / 32 comparisons per lane and no block barrier.  Longer
// lists are left to k_col_sort_long.
constexpr int kRankSortMax = 256;
constexpr int kRankWarps = 4;                 // warps per block

template <int R>
__device__ __forceinline__ void rank_list(const unsigned long long* key, uint2* __restrict__ ent, int b, int L,
                                          int lane)
{
    unsigned long long mine[R];
    int rank[R];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        const int e = lane + 32 * r;
        mine[r] = e < L ? key[e] : ~0ull;
        rank[r] = 0;
    }
    for (int j = 0; j < L; ++j) {
        const unsigned long long kj = key[j];         // the same word for every lane: a broadcast
#pragma unroll
        for (int r = 0; r < R; ++r) rank[r] += kj < mine[r] ? 1 : 0;
    }
#pragma unroll
    for (int r = 0; r < R; ++r)
        if (lane + 32 * r < L) ent[b + rank[r]] = col_unkey(mine[r]);
}

__global__ void __launch_bounds__(32 * kRankWarps) k_col_rank_sort(const int* __restrict__ off,
                                                                   uint2* __restrict__ ent, int np)
{
    __shared__ unsigned long long s_key[kRankWarps][kRankSortMax];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    unsigned long long* key = s_key[w];
    for (int p = blockIdx.x * kRankWarps + w; p < np; p += gridDim.x * kRankWarps) {
        const int b = off[p], L = off[p + 1] - b;
        if (L <= 1 || L > kRankSortMax) continue;
        __syncwarp();                                  // the previous list's ranks are read
        for (int i = lane; i < L; i += 32) key[i] = col_key(ent[b + i]);
        __syncwarp();
        if (L <= 32) rank_list<1>(key, ent, b, L, lane);
        else if (L <= 64) rank_list<2>(key, ent, b, L, lane);
        else if (L <= 128) rank_list<4>(key, ent, b, L, lane);
        else rank_list<8>(key, ent, b, L, lane);
    }
}

// Lists longer than kRankSortMax, one block per pixel: bitonic sort in shared
// memory; lists beyond kColSortMax refuse the grid (*bad |= 2).
__global__ void __launch_bounds__(128) k_col_sort_long(const int* __restrict__ off, uint2* __restrict__ ent,
                                                      int* __restrict__ bad)
{
    __shared__ unsigned long long key[kColSortMax];
    const int p = blockIdx.x;
    const int b = off[p], L = off[p + 1] - b;
    if (L <= kRankSortMax) return;
    if (L > kColSortMax) { if (threadIdx.x == 0) atomicOr(bad, 2); return; }
    int m = 1;
    while (m < L) m <<= 1;
    for (int i = threadIdx.x; i < m; i += blockDim.x) key[i] = i < L ? col_key(ent[b + i]) : ~0ull;
    __syncthreads();
    for (int k = 2; k <= m; k <<= 1)
        for (int jj = k >> 1; jj > 0; jj >>= 1) {
            for (int i = threadIdx.x; i < m; i += blockDim.x) {
                const int ixj = i ^ jj;
                if (ixj > i) {
                    const unsigned long long x = key[i], y = key[ixj];
                    if ((x > y) == ((i & k) == 0)) { key[i] = y; key[ixj] = x; }
                }
            }
            __syncthreads();
        }
    for (int i = threadIdx.x; i < L; i += blockDim.x) ent[b + i] = col_unkey(key[i]);
}

// Sort every pixel list of a grid by col_key.
void sort_lists(const int* off, uint2* ent, int np, int* bad, int num_sms, cudaStream_t s)
{
    k_col_rank_sort<<<num_sms * 16, 32 * kRankWarps, 0, s>>>(off, ent, np);
    k_col_sort_long<<<np, 128, 0, s>>>(off, ent, bad);
}

// ---- slanted column grid ---------------------------------------------------
// Rays of direction (dx, 0, dz), dz < 0, entering through z_top at x0 reach the
// point (x, y, z) of the unwrapped line when x0 = x - (z_top - z) dx / |dz| + k lx
// for the image k (the lateral wraps before that point).  A facet's footprint
// is its vertices' sheared x' = x - (z_top - z) s, s = dx / |dz|, and y; it is
// listed, with k, in every pixel its footprint shifted by k lx meets inside
// [0, lx), for every k >= 0 that does.  The bounds are taken in FP64, widened
// by `margin` (a bound on how far FP32 rounding moves the traced ray from the
// exact line) and rounded outward to FP32 before the monotonic pixel floor.
constexpr int kSlantMaxImages = 255;         // wraps a ray may make before its hit in a listed entry

struct SlantSpan {
    int k0, k1, y0, y1;
    double lo, hi;      // sheared x' range, widened
};

__device__ __forceinline__ SlantSpan slant_span(const float4* __restrict__ tris, int j, double lx, double z_top,
                                               double shear, double margin, int gy, float iwy, float& ztop)
{
    const float4 a = tris[3ll * j], b = tris[3ll * j + 1], c = tris[3ll * j + 2];
    const double xa = (double)a.x - (z_top - (double)a.z) * shear;
    const double xb = (double)b.x - (z_top - (double)b.z) * shear;
    const double xc = (double)c.x - (z_top - (double)c.z) * shear;
    SlantSpan sp;
    sp.lo = fmin(xa, fmin(xb, xc)) - margin;
    sp.hi = fmax(xa, fmax(xb, xc)) + margin;
    sp.k0 = max(0, (int)ceil(-sp.hi / lx));              // images whose shifted footprint reaches [0, lx)
    sp.k1 = (int)ceil((lx - sp.lo) / lx) - 1;
    const float loy = __double2float_rd((double)fminf(a.y, fminf(b.y, c.y)) - margin);
    const float hiy = __double2float_ru((double)fmaxf(a.y, fmaxf(b.y, c.y)) + margin);
    sp.y0 = min(max((int)floorf(loy * iwy), 0), gy - 1);
    sp.y1 = min(max((int)floorf(hiy * iwy), 0), gy - 1);
    ztop = fmaxf(a.z, fmaxf(b.z, c.z));
    return sp;
}

__device__ __forceinline__ void slant_xrange(const SlantSpan& sp, int k, double lx, int gx, float iwx, int& x0,
                                             int& x1)
{
    const float lo = __double2float_rd(fmax(sp.lo + k * lx, 0.0));
    const float hi = __double2float_ru(fmin(sp.hi + k * lx, lx));
    x0 = min(max((int)floorf(lo * iwx), 0), gx - 1);
    x1 = min(max((int)floorf(hi * iwx), 0), gx - 1);
}

__global__ void k_slant_count(const float4* __restrict__ tris, int n, int gx, int gy, float iwx, float iwy, double lx,
                              double z_top, double shear, double margin, int* __restrict__ cnt, int* __restrict__ bad)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float zt;
    const SlantSpan sp = slant_span(tris, j, lx, z_top, shear, margin, gy, iwy, zt);
    if (sp.k1 > kSlantMaxImages) { atomicOr(bad, 4); return; }
    int total = 0;
    for (int k = sp.k0; k <= sp.k1; ++k) {
        int x0, x1;
        slant_xrange(sp, k, lx, gx, iwx, x0, x1);
        total += (x1 - x0 + 1) * (sp.y1 - sp.y0 + 1);
    }
    if (total > 4 * kColMaxSpan) { atomicOr(bad, 1); return; }
    for (int k = sp.k0; k <= sp.k1; ++k) {
        int x0, x1;
        slant_xrange(sp, k, lx, gx, iwx, x0, x1);
        for (int y = sp.y0; y <= sp.y1; ++y)
            for (int x = x0; x <= x1; ++x) atomicAdd(&cnt[y * gx + x], 1);
    }
}

__global__ void k_slant_fill(const float4* __restrict__ tris, int n, int gx, int gy, float iwx, float iwy, double lx,
                             double z_top, double shear, double margin, int* __restrict__ cursor,
                             uint2* __restrict__ ent)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    float zt;
    const SlantSpan sp = slant_span(tris, j, lx, z_top, shear, margin, gy, iwy, zt);
    if (sp.k1 > kSlantMaxImages) return;
    for (int k = sp.k0; k <= sp.k1; ++k) {
        int x0, x1;
        slant_xrange(sp, k, lx, gx, iwx, x0, x1);
        for (int y = sp.y0; y <= sp.y1; ++y)
            for (int x = x0; x <= x1; ++x) {
                const int slot = atomicAdd(&cursor[y * gx + x], 1);
                ent[slot] = make_uint2((unsigned)j | ((unsigned)k << kSlantFacetBits), __float_as_uint(zt));
            }
    }
}

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { if (p) cudaFree(p); }
    cudaError_t alloc(size_t bytes) { return cudaMalloc(&p, bytes ? bytes : 16); }
    template <class T> T* as() const { return static_cast<T*>(p); }
};

}  // namespace

// Tile sums needed by scan_exclusive for n elements.
long long scan_parts(long long n) { return std::max<long long>((n + kScanTile - 1) / kScanTile, 1); }

// out[i] = in[0] + ... + in[i-1] for i < n (in == out allowed); *total (device,
// optional) = the sum of all n.  part: device scratch of scan_parts(n) words.
void scan_exclusive(const unsigned* in, unsigned* out, long long n, unsigned* total, unsigned* part, cudaStream_t s)
{
    const long long nb = (n + kScanTile - 1) / kScanTile;
    if (nb > 0) k_scan_tiles<<<(unsigned)nb, kScanThreads, 0, s>>>(in, n, part);
    k_scan_parts<<<1, 1024, 0, s>>>(part, nb, total);
    if (nb > 0) k_scan_apply<<<(unsigned)nb, kScanThreads, 0, s>>>(in, out, n, part);
}

int build_lbvh(rtmc_ctx* ctx, DeviceMesh& m)
{
    cudaStream_t s = ctx->stream;
    const int n = (int)m.n_tri;
    if (m.n_tri <= 0 || m.n_tri >= (int64_t)1 << 28)
        return ctx->fail(RTMC_ERR_INVALID_ARG, "build_bvh: triangle count out of range");
    if (m.nodes) { cudaFree(m.nodes); m.nodes = nullptr; }
    if (m.tris) { cudaFree(m.tris); m.tris = nullptr; }
    if (m.normals) { cudaFree(m.normals); m.normals = nullptr; }
    if (m.inv_order) { cudaFree(m.inv_order); m.inv_order = nullptr; }
    if (m.q8) { cudaFree(m.q8); m.q8 = nullptr; }
    if (m.w4) { cudaFree(m.w4); m.w4 = nullptr; }
    if (m.q4) { cudaFree(m.q4); m.q4 = nullptr; }
    m.n_w4 = 0;
    m.depth_w4 = 0;
    m.built = false;
    free_columns(m);
    const int64_t n_nodes = n > 1 ? n - 1 : 1;
    cudaError_t e = cudaMalloc(&m.nodes, n_nodes * 64);
    if (e == cudaSuccess) e = cudaMalloc(&m.tris, (size_t)(n + 1) * 48);
    if (e == cudaSuccess) e = cudaMalloc(&m.normals, (size_t)(n + 1) * 16);
    if (e == cudaSuccess && m.kind == FMT_Q8) e = cudaMalloc(&m.q8, n_nodes * 32);
    const bool wide = m.kind == FMT_W4 || m.kind == FMT_Q4;
    if (e == cudaSuccess && wide) e = cudaMalloc(&m.w4, n_nodes * 128);   // one per binary inner node at most
    if (e == cudaSuccess && m.kind == FMT_Q4) e = cudaMalloc(&m.q4, n_nodes * 64);
    if (e == cudaSuccess) e = cudaMalloc(&m.inv_order, (size_t)n * 4);
    if (e != cudaSuccess) return ctx->fail(RTMC_ERR_OOM, std::string("build_bvh: ") + cudaGetErrorString(e));
    m.n_nodes = n_nodes;

    cudaEvent_t ev0, ev1;
    cudaEventCreate(&ev0);
    cudaEventCreate(&ev1);
    cudaEventRecord(ev0, s);

    const int n_tiles = (n + kSortTile - 1) / kSortTile;
    DevBuf k0, k1, v0, v1, hist, part, child, range, parent, leafp, flag, aabb, depth;
    e = k0.alloc(4ull * n);
    if (e == cudaSuccess) e = k1.alloc(4ull * n);
    if (e == cudaSuccess) e = v0.alloc(4ull * n);
    if (e == cudaSuccess) e = v1.alloc(4ull * n);
    if (e == cudaSuccess) e = hist.alloc(4ull * 256 * n_tiles);
    if (e == cudaSuccess) e = part.alloc(4ull * scan_parts(256ll * n_tiles));
    if (e == cudaSuccess) e = child.alloc(8ull * n_nodes);
    if (e == cudaSuccess) e = range.alloc(8ull * n_nodes);
    if (e == cudaSuccess) e = parent.alloc(4ull * n_nodes);
    if (e == cudaSuccess) e = leafp.alloc(4ull * n);
    if (e == cudaSuccess) e = flag.alloc(4ull * n_nodes);
    if (e == cudaSuccess) e = aabb.alloc(32ull * n_nodes);
    if (e == cudaSuccess) e = depth.alloc(4);
    if (e != cudaSuccess) return ctx->fail(RTMC_ERR_OOM, std::string("build_bvh scratch: ") + cudaGetErrorString(e));

    const rtmc_box& bx = m.box;
    // outward margin of every stored child box (all node formats): M 2^-22, M the largest coordinate a
    // ray origin in the cell can have (the FMA slab test's o * inv rounding moves
    // a plane by at most |o| 2^-24)
    const double big = std::max(std::max(std::fabs(bx.lx), std::fabs(bx.ly)),
                                std::max(std::fabs(bx.z_min), std::fabs(bx.z_top)));
    const float w4_margin = (float)std::ldexp(big, -22);
    const float4 lo = make_float4(0.f, 0.f, (float)bx.z_min, 0.f);
    const float4 inv = make_float4((float)(1.0 / bx.lx), (float)(1.0 / bx.ly),
                                   (float)(1.0 / (bx.z_top - bx.z_min)), 0.f);
    const int tb = 256, gb = (n + tb - 1) / tb;
    k_morton<<<gb, tb, 0, s>>>(m.tri_in, n, lo, inv, k0.as<unsigned>(), v0.as<unsigned>());
    unsigned *ki = k0.as<unsigned>(), *ko = k1.as<unsigned>();
    unsigned *vi = v0.as<unsigned>(), *vo = v1.as<unsigned>();
    for (int pass = 0; pass < 4; ++pass) {
        const int shift = 8 * pass;
        k_radix_hist<<<n_tiles, kSortThreads, 0, s>>>(ki, n, shift, n_tiles, hist.as<unsigned>());
        scan_exclusive(hist.as<unsigned>(), hist.as<unsigned>(), 256ll * n_tiles, nullptr, part.as<unsigned>(), s);
        k_radix_scatter<<<n_tiles, kSortThreads, 0, s>>>(ki, vi, ko, vo, n, shift, n_tiles, hist.as<unsigned>());
        unsigned* t = ki; ki = ko; ko = t;
        t = vi; vi = vo; vo = t;
    }
    // after 4 passes the sorted data is back in (k0, v0)
    cudaMemsetAsync(depth.p, 0, 4, s);
    const unsigned* order = vi;                  // leaf position -> triangle id
    DevBuf ord;
    if (n > 1 && m.ploc) {
        const int n_all = 2 * n - 1;
        const int max_blocks = (n + kPlocBlock - 1) / kPlocBlock;
        DevBuf cn[2], clo[2], chi[2], nn, bc, kids, pall, cnt, first, st, bad;
        for (int b = 0; b < 2 && e == cudaSuccess; ++b) {
            e = cn[b].alloc(4ull * n);
            if (e == cudaSuccess) e = clo[b].alloc(16ull * n);
            if (e == cudaSuccess) e = chi[b].alloc(16ull * n);
        }
        if (e == cudaSuccess) e = nn.alloc(4ull * n);
        if (e == cudaSuccess) e = bc.alloc(8ull * max_blocks);
        if (e == cudaSuccess) e = kids.alloc(8ull * n_all);
        if (e == cudaSuccess) e = pall.alloc(4ull * n_all);
        if (e == cudaSuccess) e = cnt.alloc(4ull * n_all);
        if (e == cudaSuccess) e = first.alloc(4ull * n_all);
        if (e == cudaSuccess) e = st.alloc(sizeof(PlocState));
        if (e == cudaSuccess) e = bad.alloc(4);
        if (e == cudaSuccess) e = ord.alloc(4ull * n);
        if (e != cudaSuccess) return ctx->fail(RTMC_ERR_OOM, std::string("build_bvh (PLOC) scratch: ") + cudaGetErrorString(e));
        k_ploc_init<<<gb, tb, 0, s>>>(m.tri_in, vi, n, cn[0].as<int>(), clo[0].as<float4>(), chi[0].as<float4>(),
                                      cnt.as<int>());
        cudaMemsetAsync(st.p, 0, sizeof(PlocState), s);
        cudaMemsetAsync(bad.p, 0, 4, s);
        int c = n, created = 0, cur = 0;
        for (int round = 0; c > 1; ++round) {
            if (round >= n) return ctx->fail(RTMC_ERR_DEVICE_CHECK, "build_bvh (PLOC): clustering made no progress");
            const int nb = (c + kPlocBlock - 1) / kPlocBlock;
            k_ploc_nn<<<nb, kPlocBlock, 0, s>>>(clo[cur].as<float4>(), chi[cur].as<float4>(), c, nn.as<int>());
            k_ploc_count<<<nb, kPlocBlock, 0, s>>>(nn.as<int>(), c, bc.as<int2>());
            k_ploc_scan<<<1, 1024, 0, s>>>(bc.as<int2>(), nb, st.as<PlocState>());
            k_ploc_merge<<<nb, kPlocBlock, 0, s>>>(nn.as<int>(), c, bc.as<int2>(), n + created, cn[cur].as<int>(),
                                                   clo[cur].as<float4>(), chi[cur].as<float4>(), cn[1 - cur].as<int>(),
                                                   clo[1 - cur].as<float4>(), chi[1 - cur].as<float4>(),
                                                   kids.as<int2>(), pall.as<int>(), cnt.as<int>());
            PlocState h{};
            e = cudaMemcpyAsync(&h, st.p, sizeof h, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            if (e != cudaSuccess) return ctx->fail(RTMC_ERR_CUDA, std::string("build_bvh (PLOC): ") + cudaGetErrorString(e));
            if (h.count >= c || h.created != n - h.count)
                return ctx->fail(RTMC_ERR_DEVICE_CHECK, "build_bvh (PLOC): inconsistent cluster counts");
            c = h.count;
            created = h.created;
            cur = 1 - cur;
        }
        const int root = n_all - 1;
        const int ga = (n_all + tb - 1) / tb;
        k_ploc_first<<<ga, tb, 0, s>>>(kids.as<int2>(), pall.as<int>(), cnt.as<int>(), n_all, root, first.as<int>(),
                                       bad.as<int>());
        k_ploc_emit<<<ga, tb, 0, s>>>(kids.as<int2>(), pall.as<int>(), cnt.as<int>(), first.as<int>(), vi, n, root,
                                      child.as<int2>(), range.as<int2>(), parent.as<int>(), leafp.as<int>(),
                                      ord.as<unsigned>());
        int h_bad = 0;
        e = cudaMemcpyAsync(&h_bad, bad.p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return ctx->fail(RTMC_ERR_CUDA, std::string("build_bvh (PLOC): ") + cudaGetErrorString(e));
        if (h_bad) return ctx->fail(RTMC_ERR_DEVICE_CHECK, "build_bvh (PLOC): hierarchy too deep");
        order = ord.as<unsigned>();
    }
    if (n == 1) {
        k_single_leaf<<<1, 1, 0, s>>>(m.tri_in, m.nodes, w4_margin);
        if (m.kind == FMT_Q8) k_quantize_single<<<1, 1, 0, s>>>(m.tri_in, w4_margin, reinterpret_cast<uint4*>(m.q8));
        if (wide) {
            k_w4_single<<<1, 1, 0, s>>>(m.tri_in, w4_margin, reinterpret_cast<float4*>(m.w4));
            m.n_w4 = 1;
            m.depth_w4 = 1;
        }
        int one = 1;
        cudaMemcpyAsync(depth.p, &one, 4, cudaMemcpyHostToDevice, s);
    } else {
        cudaMemsetAsync(flag.p, 0, 4ull * n_nodes, s);
        const int gi = (n - 1 + tb - 1) / tb;
        if (!m.ploc)
            k_karras<<<gi, tb, 0, s>>>(ki, n, child.as<int2>(), range.as<int2>(), parent.as<int>(), leafp.as<int>());
        k_refit<<<gb, tb, 0, s>>>(m.tri_in, order, n, child.as<int2>(), range.as<int2>(), parent.as<int>(),
                                  leafp.as<int>(), flag.as<unsigned>(), aabb.as<float4>(), m.nodes, m.leaf_max,
                                  w4_margin);
        k_depth<<<gb, tb, 0, s>>>(parent.as<int>(), leafp.as<int>(), n, depth.as<int>());
        if (m.kind == FMT_Q8)
            k_quantize<<<gi, tb, 0, s>>>(m.tri_in, order, n - 1, child.as<int2>(), range.as<int2>(), aabb.as<float4>(),
                                         m.leaf_max, w4_margin, reinterpret_cast<uint4*>(m.q8));
        if (wide) {
            DevBuf fr[2], cnt, off, tot, part;
            e = fr[0].alloc(8ull * n_nodes);
            if (e == cudaSuccess) e = fr[1].alloc(8ull * n_nodes);
            if (e == cudaSuccess) e = cnt.alloc(4ull * n_nodes);
            if (e == cudaSuccess) e = off.alloc(4ull * n_nodes);
            if (e == cudaSuccess) e = tot.alloc(4);
            if (e == cudaSuccess) e = part.alloc(4ull * scan_parts(n_nodes));
            if (e != cudaSuccess)
                return ctx->fail(RTMC_ERR_OOM, std::string("build_bvh (4-wide) scratch: ") + cudaGetErrorString(e));
            const int2 root = make_int2(0, 0);
            e = cudaMemcpyAsync(fr[0].p, &root, sizeof root, cudaMemcpyHostToDevice, s);
            int nf = 1, base = 1, levels = 0, cur = 0;
            while (nf > 0 && e == cudaSuccess) {
                if (++levels > 1000) return ctx->fail(RTMC_ERR_DEVICE_CHECK, "build_bvh (4-wide): runaway collapse");
                const int gf = (nf + kW4Block - 1) / kW4Block;
                k_w4_count<<<gf, kW4Block, 0, s>>>(fr[cur].as<int2>(), nf, child.as<int2>(), range.as<int2>(),
                                                   aabb.as<float4>(), m.leaf_max, cnt.as<int>());
                scan_exclusive(cnt.as<unsigned>(), off.as<unsigned>(), nf, tot.as<unsigned>(), part.as<unsigned>(), s);
                k_w4_emit<<<gf, kW4Block, 0, s>>>(fr[cur].as<int2>(), nf, off.as<int>(), base, child.as<int2>(),
                                                  range.as<int2>(), aabb.as<float4>(), m.tri_in, order, m.leaf_max,
                                                  w4_margin, reinterpret_cast<float4*>(m.w4), fr[1 - cur].as<int2>());
                int h_tot = 0;
                e = cudaMemcpyAsync(&h_tot, tot.p, 4, cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
                if (e == cudaSuccess && (h_tot < 0 || (int64_t)base + h_tot > n_nodes))
                    return ctx->fail(RTMC_ERR_DEVICE_CHECK, "build_bvh (4-wide): node count out of range");
                base += h_tot;
                nf = h_tot;
                cur = 1 - cur;
            }
            if (e != cudaSuccess) return ctx->fail(RTMC_ERR_CUDA, std::string("build_bvh (4-wide): ") + cudaGetErrorString(e));
            m.n_w4 = base;
            m.depth_w4 = levels;
        }
    }
    DevBuf qbad;
    int h_qbad = 0;
    if (m.kind == FMT_Q4) {
        e = qbad.alloc(4);
        if (e == cudaSuccess) e = cudaMemsetAsync(qbad.p, 0, 4, s);
        if (e != cudaSuccess) return ctx->fail(RTMC_ERR_OOM, std::string("build_bvh (Q4): ") + cudaGetErrorString(e));
        k_q4_quantize<<<(unsigned)((m.n_w4 + tb - 1) / tb), tb, 0, s>>>(reinterpret_cast<const float4*>(m.w4),
                                                                       (int)m.n_w4, big, reinterpret_cast<uint4*>(m.q4),
                                                                       qbad.as<int>());
        cudaMemcpyAsync(&h_qbad, qbad.p, 4, cudaMemcpyDeviceToHost, s);
    }
    const int gp = (n + 1 + tb - 1) / tb;
    k_pack<<<gp, tb, 0, s>>>(m.tri_in, order, n, m.tris, m.normals, m.inv_order);
    int h_depth = 0;
    cudaMemcpyAsync(&h_depth, depth.p, 4, cudaMemcpyDeviceToHost, s);
    cudaEventRecord(ev1, s);
    e = cudaStreamSynchronize(s);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    cudaEventDestroy(ev0);
    cudaEventDestroy(ev1);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return ctx->fail(RTMC_ERR_CUDA, std::string("build_bvh: ") + cudaGetErrorString(e));
    m.depth = h_depth;
    m.build_ms = ms;
    if (h_depth >= kStackMax)
        return ctx->fail(RTMC_ERR_DEVICE_CHECK, "build_bvh: hierarchy deeper than the traversal stack");
    if (h_qbad) return ctx->fail(RTMC_ERR_INVALID_ARG, "build_bvh (Q4): coordinates too large for 8-bit 4-wide nodes");
    if (wide && 3 * m.depth_w4 >= kStackMax)
        return ctx->fail(RTMC_ERR_DEVICE_CHECK, "build_bvh: 4-wide hierarchy deeper than the traversal stack");
    const int rc = build_columns(ctx, m);
    if (rc != RTMC_OK) return rc;
    m.built = true;
    return RTMC_OK;
}

void free_columns(DeviceMesh& m)
{
    for (SlantGrid& g : m.slant) {
        if (g.off) cudaFree(g.off);
        if (g.ent) cudaFree(g.ent);
    }
    m.slant.clear();
    m.slant_failed.clear();
    m.slant_bytes = 0;
    if (m.col_off) cudaFree(m.col_off);
    if (m.col_ent) cudaFree(m.col_ent);
    m.col_off = nullptr;
    m.col_ent = nullptr;
    m.col_ok = false;
    m.col_gx = m.col_gy = 0;
    m.col_entries = 0;
}

// The column grid over the leaf-order facets.  About 5 facets per pixel (2.4 nm
// pixels on a 128^3 foam of 10 nm voxels; finer pixels cut the facet tests per
// vertical ray, 5 -> 2.4 nm took a fifth off the column kernel).  A facet over
// more than kColMaxSpan pixels makes the build retry with a quarter of the
// pixels; a pixel with more than kColSortMax facets, more than 2^24 facets or
// no room on the device leave the mesh without a grid, and its vertical rays
// take the hierarchy.
int build_columns(rtmc_ctx* ctx, DeviceMesh& m)
{
    free_columns(m);
    const int n = (int)m.n_tri;
    const double lx = m.box.lx, ly = m.box.ly;
    if (n <= 0 || n > (1 << 24) || !(lx > 0.0) || !(ly > 0.0)) return RTMC_OK;
    cudaStream_t s = ctx->stream;
    double pix = std::max(1.0, (double)n / 5.0);
    for (int attempt = 0; attempt < 5; ++attempt, pix = std::max(1.0, pix / 4.0)) {
        free_columns(m);
        const int gx = std::min(2048, std::max(1, (int)std::lround(std::sqrt(pix * lx / ly))));
        const int gy = std::min(2048, std::max(1, (int)std::lround(pix / gx)));
        const int np = gx * gy;
        const float iwx = (float)(gx / lx), iwy = (float)(gy / ly);
        DevBuf cnt, tot, bad, part;
        cudaError_t e = cnt.alloc(4ull * np);
        if (e == cudaSuccess) e = tot.alloc(4);
        if (e == cudaSuccess) e = bad.alloc(4);
        if (e == cudaSuccess) e = part.alloc(4ull * scan_parts(np));
        if (e == cudaSuccess) e = cudaMalloc(&m.col_off, 4ull * (np + 1));
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt.p, 0, 4ull * np, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(bad.p, 0, 4, s);
        const int tb = 256, gb = (n + tb - 1) / tb;
        if (e == cudaSuccess) {
            k_col_count<<<gb, tb, 0, s>>>(m.tris, n, gx, gy, iwx, iwy, cnt.as<int>(), bad.as<int>());
            scan_exclusive(cnt.as<unsigned>(), reinterpret_cast<unsigned*>(m.col_off), np, tot.as<unsigned>(),
                           part.as<unsigned>(), s);
            e = cudaGetLastError();
        }
        int h_tot = 0, h_bad = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(m.col_off + np, tot.p, 4, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_tot, tot.p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad.p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e == cudaSuccess && (h_bad & 1)) continue;          // a facet too wide for these pixels
        if (e == cudaSuccess && h_tot > 0) {
            e = cudaMalloc(&m.col_ent, 8ull * h_tot);
            if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.p, m.col_off, 4ull * np, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) {
                k_col_fill<<<gb, tb, 0, s>>>(m.tris, n, gx, gy, iwx, iwy, cnt.as<int>(), m.col_ent);
                sort_lists(reinterpret_cast<const int*>(m.col_off), m.col_ent, np, bad.as<int>(), ctx->num_sms, s);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad.p, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e == cudaErrorMemoryAllocation) {      // no room: the hierarchy serves every ray
            cudaGetLastError();
            free_columns(m);
            return RTMC_OK;
        }
        if (e != cudaSuccess)
            return ctx->fail(RTMC_ERR_CUDA, std::string("build_bvh: column grid: ") + cudaGetErrorString(e));
        if (h_bad || h_tot <= 0) { free_columns(m); return RTMC_OK; }
        m.col_gx = gx;
        m.col_gy = gy;
        m.col_inv_wx = iwx;
        m.col_inv_wy = iwy;
        m.col_entries = h_tot;
        m.col_ok = true;
        return RTMC_OK;
    }
    free_columns(m);
    return RTMC_OK;
}

GridDev grid_dev(const DeviceMesh& m, const SlantGrid* g)
{
    GridDev d;
    if (g) {
        d.off = g->off; d.ent = g->ent; d.gx = g->gx; d.gy = g->gy; d.iwx = g->iwx; d.iwy = g->iwy;
        d.dx = g->dx; d.dz = g->dz;
    } else {
        d.off = m.col_off; d.ent = m.col_ent; d.gx = m.col_gx; d.gy = m.col_gy; d.iwx = m.col_inv_wx;
        d.iwy = m.col_inv_wy; d.dx = 0.f; d.dz = -1.f;
    }
    return d;
}

// The slanted grid keeps the vertical grid's y pixels and widens its x pixels
// by 1 + s (s = dx / |dz|), so a facet's sheared footprint (x extent plus z
// extent times s) covers about as many pixels as its vertical footprint; a
// footprint over more than 4 x 64 pixels makes the build retry with half the x
// pixels (up to four times).  All slanted grids of a mesh together stay below
// a quarter of the free device memory and 32 GiB.
bool slant_grid(rtmc_ctx* ctx, DeviceMesh& m, float dx, float dz, GridDev& out)
{
    for (const SlantGrid& g : m.slant)
        if (g.dx == dx && g.dz == dz) { out = grid_dev(m, &g); return true; }
    for (const float2& f : m.slant_failed)
        if (f.x == dx && f.y == dz) return false;
    auto fail = [&]() { m.slant_failed.push_back(make_float2(dx, dz)); return false; };
    const int n = (int)m.n_tri;
    if (!m.col_ok || !(dx > 0.f) || !(dz < 0.f) || n <= 0 || n > (1 << kSlantFacetBits)) return fail();
    cudaStream_t s = ctx->stream;
    const double lx = m.box.lx, ly = m.box.ly, z_top = m.box.z_top, z_min = m.box.z_min;
    const double shear = (double)dx / -(double)dz;
    const double big = std::max(std::max(std::fabs(lx), std::fabs(ly)), std::max(std::fabs(z_min), std::fabs(z_top)));
    const double flight = (z_top - z_min) * std::sqrt(1.0 + shear * shear);
    const double margin = std::ldexp(big + flight, -16);   // FP32 rounding of the traced ray, with room to spare
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const size_t cap = std::min<size_t>((size_t)32 << 30, free_b / 4);
    const int gy = m.col_gy;
    int gx = std::max(1, (int)std::lround(m.col_gx / (1.0 + shear)));
    for (int attempt = 0; attempt < 5; ++attempt, gx = std::max(1, gx / 2)) {
        const int np = gx * gy;
        const float iwx = (float)(gx / lx), iwy = (float)(gy / ly);
        SlantGrid g;
        g.dx = dx; g.dz = dz; g.gx = gx; g.gy = gy; g.iwx = iwx; g.iwy = iwy;
        DevBuf cnt, tot, bad, part;
        cudaError_t e = cnt.alloc(4ull * np);
        if (e == cudaSuccess) e = tot.alloc(4);
        if (e == cudaSuccess) e = bad.alloc(4);
        if (e == cudaSuccess) e = part.alloc(4ull * scan_parts(np));
        if (e == cudaSuccess) e = cudaMalloc(&g.off, 4ull * (np + 1));
        if (e == cudaSuccess) e = cudaMemsetAsync(cnt.p, 0, 4ull * np, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(bad.p, 0, 4, s);
        const int tb = 256, gb = (n + tb - 1) / tb;
        if (e == cudaSuccess) {
            k_slant_count<<<gb, tb, 0, s>>>(m.tris, n, gx, gy, iwx, iwy, lx, z_top, shear, margin, cnt.as<int>(),
                                            bad.as<int>());
            scan_exclusive(cnt.as<unsigned>(), reinterpret_cast<unsigned*>(g.off), np, tot.as<unsigned>(),
                           part.as<unsigned>(), s);
            e = cudaGetLastError();
        }
        int h_tot = 0, h_bad = 0;
        if (e == cudaSuccess) e = cudaMemcpyAsync(g.off + np, tot.p, 4, cudaMemcpyDeviceToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_tot, tot.p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad.p, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        const size_t bytes = 8ull * (size_t)std::max(h_tot, 0) + 4ull * (np + 1);
        if (e == cudaSuccess && (h_bad & 1) == 0 && (h_bad || h_tot <= 0 || m.slant_bytes + bytes > cap)) {
            cudaFree(g.off);
            return fail();                              // too many wraps, nothing listed, or no room
        }
        if (e == cudaSuccess && (h_bad & 1)) { cudaFree(g.off); continue; }   // a footprint too wide
        if (e == cudaSuccess) {
            e = cudaMalloc(&g.ent, 8ull * h_tot);
            if (e == cudaSuccess) e = cudaMemcpyAsync(cnt.p, g.off, 4ull * np, cudaMemcpyDeviceToDevice, s);
            if (e == cudaSuccess) {
                k_slant_fill<<<gb, tb, 0, s>>>(m.tris, n, gx, gy, iwx, iwy, lx, z_top, shear, margin, cnt.as<int>(),
                                               g.ent);
                sort_lists(reinterpret_cast<const int*>(g.off), g.ent, np, bad.as<int>(), ctx->num_sms, s);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) e = cudaMemcpyAsync(&h_bad, bad.p, 4, cudaMemcpyDeviceToHost, s);
            if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        }
        if (e != cudaSuccess || h_bad) {             // no memory, or a pixel list too long to sort
            if (e != cudaSuccess) cudaGetLastError();
            if (g.off) cudaFree(g.off);
            if (g.ent) cudaFree(g.ent);
            return fail();
        }
        g.entries = h_tot;
        m.slant_bytes += bytes;
        m.slant.push_back(g);
        out = grid_dev(m, &g);
        return true;
    }
    return fail();
}

}  // namespace rtmc
