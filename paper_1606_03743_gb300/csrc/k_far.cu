// k_far.cu -- far-field point-charge cubature (Eq. 4.1) with distance-ratio
// rule bands (Sec. 4) and compaction of the near-field pairs.
//
// Work decomposition:
//  * Field points arrive sorted by spatial cell.  A work item is one warp's
//    tile of 32 * PT neighbouring points times one chunk of the elements;
//    every point of the tile is owned by one lane (PT points per lane).  The
//    elements are cut into a number of chunks fixed by the mesh alone, so a
//    point's sum is always split the same way whatever batch it came in.
//  * The kernel is persistent: a grid that fills the GPU once, whose warps
//    take work items from a global counter until none is left.  Warps never
//    wait for one another (no CTA barrier inside the loop).
//  * Each warp streams its chunk in batches of 32 elements, one element per
//    lane: the lane stages the element's centroid, frame and charge in the
//    warp's shared memory and tests, conservatively, whether every point of
//    the warp lies in one distance-ratio band of that element.
//  * Per element the warp expands only the rule it needs (lane i computes
//    node i from the element frame: Eq. 3.2 / Eq. 3.3), as (offset, w_i q)
//    records in a double-buffered shared-memory slot, then every lane runs
//    the node loop for its PT points reading the records by broadcast.
//    Elements whose band differs between points of the warp fall back to
//    per-point bands: the warp runs each band present with the other
//    points' charges masked.  Either way a point always gets exactly the
//    band of its own distance ratio, so its result does not depend on which
//    points share its warp.
//  * Pairs in the analytic band are appended to a compacted list by warp
//    ballots, with a (point, chunk, ordinal) tag so that the analytic pass
//    adds them back in element order.
//
// Arithmetic:
//  * FP64 path: everything in double precision.
//  * Mixed path: points and centroids are split into FP32 hi + lo parts, and
//    P - Q_i is formed as ((P_hi - C_hi) + P_lo) - (o_i + C_lo): the small
//    lo part of the centroid rides with the node offset o_i (both are small),
//    so the difference keeps FP32 relative accuracy anywhere in space.  Node
//    offsets, rsqrt and the sums are FP32: each element's node terms (at
//    most 33) are summed on their own, eight such element sums are added up,
//    and that sum is flushed into FP64 accumulators in shared memory.  No
//    FP32 sum runs over more than 33 terms; the FP64 pipe sees two adds per
//    element and point.
#include <stdio.h>

#include <type_traits>

#include "bem_internal.cuh"

namespace bem {

// field points per lane of the mixed and FP64 paths (a warp's tile is 32 x PT points)
#ifndef BEM_MIXED_PT
#define BEM_MIXED_PT 4
#endif
#ifndef BEM_FP64_PT
#define BEM_FP64_PT 2
#endif
constexpr int kPtMixed = BEM_MIXED_PT, kPtFp64 = BEM_FP64_PT;
// node-loop unroll depth
#ifndef BEM_NODE_UNROLL
#define BEM_NODE_UNROLL 4
#endif
constexpr int kNodeUnroll = BEM_NODE_UNROLL;

constexpr int kSlots = 76;    // rule-table slots per element type (75 used at most)
constexpr int kWarps = 4;     // warps per CTA
constexpr int kNodeBuf = 36;  // node records per buffer (33 used at most)

__constant__ float c_alpha_f[2 * kSlots], c_beta_f[2 * kSlots], c_w_f[2 * kSlots];
__constant__ double c_alpha_d[2 * kSlots], c_beta_d[2 * kSlots], c_w_d[2 * kSlots];
__constant__ int c_rule_n[10], c_rule_start[10];

struct FarK {
    const double* pts;
    const int* perm;
    int n_pts, n_el;
    int n_chunks, chunk_len, n_items;
    int* work;  // work-item counter (zeroed before the launch)
    const float4 *chi, *clo, *e0f, *e1f;  // mixed element records
    const double *cen, *fr, *geo;         // FP64 element data
    const int* type;
    const double* sigma;  // nullptr: unit density (assembly)
    double4* part;        // per (point, chunk) far sums, [n_pts][n_chunks]
    int* near_cnt;        // per (point, chunk) near pairs, [n_pts][n_chunks]
    int4* near_rec;
    unsigned long long* counters;
    unsigned long long near_cap;
    double* A;
    double kc;
    float tau2f[2][5];
    double tau2d[2][5];
    const unsigned* bbox;  // field-point bounding box (order-preserving float bits: min xyz, max xyz)
    float coord_max;       // largest |coordinate| of the mesh
    const int* n_dev;      // if set: the point count is read here (n_pts is then the capacity)
    int tile_pts;          // points per work-item tile (32 x PT)
};

__device__ __forceinline__ float ord_to_float(unsigned u) {
    return __uint_as_float((u & 0x80000000u) ? (u & 0x7fffffffu) : ~u);
}

// ------------------------------------------------------------ helpers
__device__ __forceinline__ float warp_min(float v) {
    for (int o = 16; o; o >>= 1) v = fminf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}
__device__ __forceinline__ float warp_max(float v) {
    for (int o = 16; o; o >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, o));
    return v;
}

template <typename R>
__device__ __forceinline__ int band_of(R d2, const R* thr) {
    return (d2 >= thr[0]) + (d2 >= thr[1]) + (d2 >= thr[2]) + (d2 >= thr[3]) + (d2 >= thr[4]);
}

// code of an element for a warp: 0..5 = every point in that band, 7 = mixed, 15 = past the end
constexpr int kMixedCode = 7, kEndCode = 15;

__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }

// Warp-cooperative append of near pairs; want[q] marks point q of this lane.
template <int PT>
__device__ __forceinline__ void append_near(const FarK& p, const bool (&want)[PT], const int (&sidx)[PT], int elem,
                                            int chunk, int (&ncnt)[PT], int lane) {
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const unsigned m = __ballot_sync(0xffffffffu, want[q]);
        if (!m) continue;
        const int leader = __ffs(m) - 1;
        unsigned long long base = 0;
        if (lane == leader) base = atomicAdd(p.counters, (unsigned long long)__popc(m));
        base = __shfl_sync(0xffffffffu, base, leader);
        if (want[q]) {
            const unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
            if (idx < p.near_cap) p.near_rec[idx] = make_int4(sidx[q], elem, ncnt[q], chunk);
            ++ncnt[q];
        }
    }
}

// One point charge (offset o, charge o.w) at the PT points of a lane.
// MASKED: point q's charge is scaled by mq[q] (1 or 0); masked-off points
// have been moved far away by the caller, so r^2 > 0 and their terms are
// exact zeros, while an active point's arithmetic is bit-for-bit that of
// the unmasked path.  INIT: the sums start from this term.
template <typename R, typename R4, int PT, bool WANT_E, bool MASKED, bool INIT>
__device__ __forceinline__ void node(const R4 o, const R (&dx)[PT], const R (&dy)[PT], const R (&dz)[PT],
                                     R (&acc)[PT][4], const R (&mq)[PT]) {
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const R rx = dx[q] - o.x, ry = dy[q] - o.y, rz = dz[q] - o.z;
        const R r2 = fmad(rx, rx, fmad(ry, ry, rz * rz));
        R wq = o.w;
        if (MASKED) wq *= mq[q];
        const R inv = rsq(r2);
        const R a = wq * inv;          // q_i / r_i
        const R b = a * (inv * inv);   // q_i / r_i^3
        if (INIT) {
            acc[q][0] = a;
            if (WANT_E) { acc[q][1] = b * rx; acc[q][2] = b * ry; acc[q][3] = b * rz; }
        } else {
            acc[q][0] += a;
            if (WANT_E) {
                acc[q][1] = fmad(b, rx, acc[q][1]);
                acc[q][2] = fmad(b, ry, acc[q][2]);
                acc[q][3] = fmad(b, rz, acc[q][3]);
            }
        }
    }
}

// Accumulate the point charges of one rule of one element into
// acc[q] = (phi, Ex, Ey, Ez) sums.  nd: the rule's (offset, w_i q) records in
// shared memory (warp-uniform addresses: broadcast).  MASKED: point q counts
// with weight mq[q].  INIT: the first node starts the sums.
template <typename R, typename R4, int PT, bool WANT_E, bool MASKED, bool INIT>
__device__ __forceinline__ void nodes(const R4* __restrict__ nd, int n, const R (&dx)[PT], const R (&dy)[PT],
                                      const R (&dz)[PT], R (&acc)[PT][4], const R (&mq)[PT]) {
    int i = 0;
    if (INIT) {  // every rule has at least four nodes
        node<R, R4, PT, WANT_E, MASKED, true>(nd[0], dx, dy, dz, acc, mq);
        i = 1;
    }
#pragma unroll kNodeUnroll
    for (; i < n; ++i) node<R, R4, PT, WANT_E, MASKED, false>(nd[i], dx, dy, dz, acc, mq);
}

// Shared memory of one warp.
template <typename R, typename R4, int PT, bool ACC64>
struct WarpSmem {
    R4 c[32];    // centroid (hi part for mixed), w = type
    R4 cl[32];   // centroid lo part (mixed), w = L
    R4 e0[32];   // frame e0, w = q (element charge)
    R4 e1[32];   // frame e1
    R thr[32 * 5];
    R4 nd[2][kNodeBuf];
    double acc64[ACC64 ? PT * 4 * 32 : 1];
};

template <typename R>
struct RuleSmem {
    R al[2 * kSlots], be[2 * kSlots], w[2 * kSlots];
    int n[10], start[10];
    unsigned long long stat[15];  // 12 band counts, uniform / mixed (warp, element) pairs, node evaluations
};

template <bool F64, int PT, bool WANT_E, int MODE>
constexpr size_t far_smem_bytes() {
    using R = typename std::conditional<F64, double, float>::type;
    using R4 = typename std::conditional<F64, double4, float4>::type;
    constexpr bool ACC64 = !F64 && MODE == 0;
    return ((sizeof(RuleSmem<R>) + 15) / 16) * 16 + kWarps * sizeof(WarpSmem<R, R4, PT, ACC64>);
}

// ------------------------------------------------------------ the kernel
// MODE 0: evaluation (sum over elements); MODE 1: assembly (one value per
// (point, element) pair written to A, potential only, sigma = 1).
// STATS: count pairs per (type, band) into counters[2 + 6 type + band], and
// into counters[16..18] the (warp, element) pairs that ran one band for the
// whole warp, those that fell back to per-point bands, and the node
// evaluations executed (lanes x points x nodes, masked ones included).
// CTAs per SM the register allocation must allow (4 x 4 warps)
#ifndef BEM_MIN_BLOCKS
#define BEM_MIN_BLOCKS 4
#endif
template <bool F64, int PT, bool WANT_E, int MODE, bool STATS>
__global__ void __launch_bounds__(kWarps * 32, BEM_MIN_BLOCKS) k_far(const FarK p) {
    using R = typename std::conditional<F64, double, float>::type;
    using R4 = typename std::conditional<F64, double4, float4>::type;
    constexpr bool ACC64 = !F64 && MODE == 0;  // FP64 accumulators in shared memory
    using WS = WarpSmem<R, R4, PT, ACC64>;

    extern __shared__ __align__(16) unsigned char smem_raw[];
    RuleSmem<R>& rs = *reinterpret_cast<RuleSmem<R>*>(smem_raw);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    WS& ws = reinterpret_cast<WS*>(smem_raw + ((sizeof(RuleSmem<R>) + 15) / 16) * 16)[warp];
    int n_pts = p.n_pts, n_items = p.n_items;
    if (p.n_dev) {
        n_pts = min(n_pts, *p.n_dev);
        n_items = (n_pts + p.tile_pts - 1) / p.tile_pts * p.n_chunks;
    }

    for (int i = tid; i < 2 * kSlots; i += blockDim.x) {
        if constexpr (F64) {
            rs.al[i] = c_alpha_d[i]; rs.be[i] = c_beta_d[i]; rs.w[i] = c_w_d[i];
        } else {
            rs.al[i] = c_alpha_f[i]; rs.be[i] = c_beta_f[i]; rs.w[i] = c_w_f[i];
        }
    }
    if (tid < 10) {
        rs.n[tid] = c_rule_n[tid];
        rs.start[tid] = c_rule_start[tid];
    }
    if (STATS && tid < 15) rs.stat[tid] = 0ull;
    // absolute margin of the warp band test: coordinates enter it rounded to
    // FP32 (relative 6e-8); 1e-6 of the largest magnitude in play bounds that
    // rounding with a wide margin
    float slack_abs;
    {
        float pm = 0.0f;
#pragma unroll
        for (int k = 0; k < 6; ++k) pm = fmaxf(pm, fabsf(ord_to_float(p.bbox[k])));
        slack_abs = 1e-6f * (3.0f * p.coord_max + pm);
    }
    __syncthreads();

    R ones[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) ones[q] = (R)1;
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(p.work, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        const int tile = item / p.n_chunks, chunk = item - tile * p.n_chunks;
        const int base = tile * (32 * PT);

        // ---- field points of this lane
        R px[PT], py[PT], pz[PT];      // FP64: the point; mixed: hi part
        float lx[PT], ly[PT], lz[PT];  // mixed: lo part
        int sidx[PT];
        bool valid[PT];
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            int i = base + q * 32 + lane;
            valid[q] = i < n_pts;
            if (!valid[q]) i = base;  // duplicate a live point of the tile
            sidx[q] = i;
            const int src = p.perm[i];
            const double X = p.pts[3 * (size_t)src], Y = p.pts[3 * (size_t)src + 1], Z = p.pts[3 * (size_t)src + 2];
            if constexpr (F64) {
                px[q] = X; py[q] = Y; pz[q] = Z;
                lx[q] = ly[q] = lz[q] = 0.0f;
            } else {
                const float hx = (float)X, hy = (float)Y, hz = (float)Z;
                px[q] = hx; py[q] = hy; pz[q] = hz;
                lx[q] = (float)(X - (double)hx); ly[q] = (float)(Y - (double)hy); lz[q] = (float)(Z - (double)hz);
            }
        }
        // ---- bounding sphere of the tile (FP32, only for the band test)
        float wcx, wcy, wcz, wrad, wmag;
        {
            float mn[3] = {1e30f, 1e30f, 1e30f}, mx[3] = {-1e30f, -1e30f, -1e30f};
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const float v[3] = {(float)px[q], (float)py[q], (float)pz[q]};
#pragma unroll
                for (int k = 0; k < 3; ++k) { mn[k] = fminf(mn[k], v[k]); mx[k] = fmaxf(mx[k], v[k]); }
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) { mn[k] = warp_min(mn[k]); mx[k] = warp_max(mx[k]); }
            wcx = 0.5f * (mn[0] + mx[0]); wcy = 0.5f * (mn[1] + mx[1]); wcz = 0.5f * (mn[2] + mx[2]);
            float r2 = 0.0f;
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const float ax = (float)px[q] - wcx, ay = (float)py[q] - wcy, az = (float)pz[q] - wcz;
                r2 = fmaxf(r2, ax * ax + ay * ay + az * az);
            }
            wrad = sqrtf(warp_max(r2));
            wmag = sqrtf(wcx * wcx + wcy * wcy + wcz * wcz) + wrad;
        }
        int nvalid = 0;  // valid points of the tile (for the statistics)
        if (STATS) nvalid = min(32 * PT, n_pts - base);

        // ---- accumulators
        R acc[PT][4];  // FP64 path: the sums; mixed: FP32 sum of up to 8 element sums
        int ncnt[PT];
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            ncnt[q] = 0;
#pragma unroll
            for (int c = 0; c < 4; ++c) {
                acc[q][c] = (R)0;
                if constexpr (ACC64) ws.acc64[(q * 4 + c) * 32 + lane] = 0.0;
            }
        }

        const int el0 = chunk * p.chunk_len, el1 = min(p.n_el, el0 + p.chunk_len);
        int par = 0;  // node buffer parity
        for (int b0 = el0; b0 < el1; b0 += 32) {
            // ---- stage the batch: one element per lane
            __syncwarp();
            int code = kEndCode;
            {
                const int j = b0 + lane;
                if (j < el1) {
                    const int ty = p.type[j];
                    const double sg = p.sigma ? p.sigma[j] : 1.0;
                    const double area = p.geo[2 * j + 1];
                    R4 c, cl;
                    float th[5];
                    if constexpr (F64) {
                        const double L = p.geo[2 * j];
                        c = R4{p.cen[3 * j], p.cen[3 * j + 1], p.cen[3 * j + 2], (double)ty};
                        cl = R4{0, 0, 0, L};
                        ws.e0[lane] = R4{p.fr[6 * j], p.fr[6 * j + 1], p.fr[6 * j + 2], sg * area};
                        ws.e1[lane] = R4{p.fr[6 * j + 3], p.fr[6 * j + 4], p.fr[6 * j + 5], 0.0};
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            const double t = p.tau2d[ty][k] * L * L;
                            ws.thr[lane * 5 + k] = t;
                            th[k] = (float)t;
                        }
                    } else {
                        c = p.chi[j];  // w: the element type as int bits
                        cl = p.clo[j];
                        const float4 a = p.e0f[j], b = p.e1f[j];
                        ws.e0[lane] = R4{a.x, a.y, a.z, (float)(sg * area)};
                        ws.e1[lane] = R4{b.x, b.y, b.z, 0.0f};
                        const float L = cl.w;
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            th[k] = p.tau2f[ty][k] * L * L;
                            ws.thr[lane * 5 + k] = th[k];
                        }
                    }
                    ws.c[lane] = c;
                    ws.cl[lane] = cl;
                    // conservative band test of the whole tile against this element
                    const float dx = ((float)(wcx - (float)c.x)) - (float)cl.x;
                    const float dy = ((float)(wcy - (float)c.y)) - (float)cl.y;
                    const float dz = ((float)(wcz - (float)c.z)) - (float)cl.z;
                    const float Dc = sqrtf(dx * dx + dy * dy + dz * dz);
                    const float slack = fmaf(1e-5f, Dc + wrad, slack_abs);
                    const float dmin = fmaxf(Dc - wrad - slack, 0.0f), dmax = Dc + wrad + slack;
                    const int blo = band_of<float>(dmin * dmin, th), bhi = band_of<float>(dmax * dmax, th);
                    code = blo == bhi ? blo : kMixedCode;
                }
            }
            __syncwarp();

            const int nb = min(32, el1 - b0);
            for (int e = 0; e < nb; ++e) {
                const int cd = __shfl_sync(0xffffffffu, code, e);
                const R4 c = ws.c[e];
                int ty;
                if constexpr (F64) ty = (int)c.w;
                else ty = __float_as_int(c.w);
                // (P_hi - C_hi) + P_lo; the centroid's lo part is in the node offsets
                R dx[PT], dy[PT], dz[PT];
#pragma unroll
                for (int q = 0; q < PT; ++q) {
                    if constexpr (F64) {
                        dx[q] = px[q] - c.x; dy[q] = py[q] - c.y; dz[q] = pz[q] - c.z;
                    } else {
                        dx[q] = (px[q] - c.x) + lx[q];
                        dy[q] = (py[q] - c.y) + ly[q];
                        dz[q] = (pz[q] - c.z) + lz[q];
                    }
                }
                // per-element sums (mixed path, assembly; started by the element's
                // first rule pass) or the running sums (FP64 evaluation)
                constexpr bool kElemSum = MODE == 1 || !F64;
                R eacc[PT][4];
                R(&dst)[PT][4] = kElemSum ? eacc : acc;

                // expand rule r of element e into the free node buffer (lane i: node i)
                auto expand = [&](int r) -> int {
                    const int n = rs.n[ty * 5 + r], st = ty * kSlots + rs.start[ty * 5 + r];
                    const R4 a = ws.e0[e], b = ws.e1[e];
                    R ox = 0, oy = 0, oz = 0;  // mixed path: the centroid's lo part
                    if constexpr (!F64) {
                        const R4 cl = ws.cl[e];
                        ox = cl.x; oy = cl.y; oz = cl.z;
                    }
                    for (int i = lane; i < n; i += 32) {
                        const R al = rs.al[st + i], be = rs.be[st + i];
                        ws.nd[par][i] = R4{fmad(al, a.x, fmad(be, b.x, ox)), fmad(al, a.y, fmad(be, b.y, oy)),
                                           fmad(al, a.z, fmad(be, b.z, oz)), rs.w[st + i] * a.w};
                    }
                    __syncwarp();
                    return n;
                };

                if (cd >= 1 && cd <= 5) {
                    const int n = expand(band_rule(cd));
                    nodes<R, R4, PT, WANT_E, false, kElemSum>(ws.nd[par], n, dx, dy, dz, dst, ones);
                    par ^= 1;
                    if (STATS && lane == 0) {
                        atomicAdd(&rs.stat[6 * ty + cd], (unsigned long long)nvalid);
                        atomicAdd(&rs.stat[12], 1ull);
                        atomicAdd(&rs.stat[14], (unsigned long long)n * 32 * PT);
                    }
                } else {
                    // per-point bands
                    int bq[PT];
                    const R* th = ws.thr + e * 5;
                    unsigned mask = 0;
#pragma unroll
                    for (int q = 0; q < PT; ++q) {
                        const R d2 = dx[q] * dx[q] + dy[q] * dy[q] + dz[q] * dz[q];
                        bq[q] = band_of<R>(d2, th);
                        if (valid[q]) mask |= 1u << bq[q];
                    }
                    mask = __reduce_or_sync(0xffffffffu, mask);
                    if (mask & 1u) {
                        bool want[PT];
#pragma unroll
                        for (int q = 0; q < PT; ++q) want[q] = valid[q] && bq[q] == 0;
                        append_near<PT>(p, want, sidx, b0 + e, chunk, ncnt, lane);
                    }
                    if (kElemSum) {  // near-only points get zero far sums
#pragma unroll
                        for (int q = 0; q < PT; ++q)
#pragma unroll
                            for (int k = 0; k < 4; ++k) eacc[q][k] = (R)0;
                    }
#pragma unroll 1
                    for (int band = 1; band <= 5; ++band) {
                        if (!(mask & (1u << band))) continue;
                        // points of other bands: zero charge, parked far from every node
                        // (the active points' differences are formed afresh, exactly as above)
                        R mq[PT];
                        {
                            const R4 cc = ws.c[e];
#pragma unroll
                            for (int q = 0; q < PT; ++q) {
                                const bool on = bq[q] == band;
                                mq[q] = on ? (R)1 : (R)0;
                                R ax, ay, az;
                                if constexpr (F64) {
                                    ax = px[q] - cc.x; ay = py[q] - cc.y; az = pz[q] - cc.z;
                                } else {
                                    ax = (px[q] - cc.x) + lx[q];
                                    ay = (py[q] - cc.y) + ly[q];
                                    az = (pz[q] - cc.z) + lz[q];
                                }
                                dx[q] = on ? ax : (R)1e3;
                                dy[q] = on ? ay : (R)1e3;
                                dz[q] = on ? az : (R)1e3;
                            }
                        }
                        const int n = expand(band_rule(band));
                        nodes<R, R4, PT, WANT_E, true, false>(ws.nd[par], n, dx, dy, dz, dst, mq);
                        par ^= 1;
                        if (STATS && lane == 0) atomicAdd(&rs.stat[14], (unsigned long long)n * 32 * PT);
                    }
                    if (STATS) {
                        if (lane == 0) atomicAdd(&rs.stat[13], 1ull);
#pragma unroll
                        for (int q = 0; q < PT; ++q) {
                            for (int band = 0; band <= 5; ++band) {
                                const unsigned m = __ballot_sync(0xffffffffu, valid[q] && bq[q] == band);
                                if (lane == 0 && m) atomicAdd(&rs.stat[6 * ty + band], (unsigned long long)__popc(m));
                            }
                        }
                    }
                }

                if constexpr (MODE == 0 && !F64) {
                    // add the element sums; every 8 elements move the FP32 sum into FP64
#pragma unroll
                    for (int q = 0; q < PT; ++q)
#pragma unroll
                        for (int k = 0; k < 4; ++k) acc[q][k] += eacc[q][k];
                    if (((b0 + e) & 7) == 7 || e == nb - 1) {
#pragma unroll
                        for (int q = 0; q < PT; ++q)
#pragma unroll
                            for (int k = 0; k < 4; ++k) {
                                ws.acc64[(q * 4 + k) * 32 + lane] += (double)acc[q][k];
                                acc[q][k] = (R)0;
                            }
                    }
                }
                if constexpr (MODE == 1) {
                    // assembly: one potential per pair, times 1/(4 pi eps0); near pairs are filled later
#pragma unroll
                    for (int q = 0; q < PT; ++q)
                        if (valid[q]) p.A[(size_t)p.perm[sidx[q]] * p.n_el + (b0 + e)] = p.kc * (double)eacc[q][0];
                }
            }
        }

        if constexpr (MODE == 0) {
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                if (!valid[q]) continue;
                double4 o;
                if constexpr (F64) o = make_double4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
                else
                    o = make_double4(ws.acc64[(q * 4) * 32 + lane], ws.acc64[(q * 4 + 1) * 32 + lane],
                                     ws.acc64[(q * 4 + 2) * 32 + lane], ws.acc64[(q * 4 + 3) * 32 + lane]);
                const size_t slot = (size_t)sidx[q] * p.n_chunks + chunk;
                p.part[slot] = o;
                p.near_cnt[slot] = ncnt[q];
            }
        }
    }
    if (STATS) {
        __syncthreads();
        if (tid < 12 && rs.stat[tid]) atomicAdd(&p.counters[2 + tid], rs.stat[tid]);
        if (tid >= 12 && tid < 15 && rs.stat[tid]) atomicAdd(&p.counters[16 + tid - 12], rs.stat[tid]);
    }
}

// ------------------------------------------------------------ host side
namespace {
int uploaded_mask = 0;  // devices whose constant rule tables are loaded

int upload_rules(int dev) {
    if (dev < 32 && (uploaded_mask >> dev) & 1) return BEM_OK;
    const RuleSet& rs = rules();
    float af[2 * kSlots], bf[2 * kSlots], wf[2 * kSlots];
    double ad[2 * kSlots], bd[2 * kSlots], wd[2 * kSlots];
    for (int t = 0; t < 2; ++t)
        for (int s = 0; s < kSlots; ++s) {
            ad[t * kSlots + s] = rs.alpha[t][s];
            bd[t * kSlots + s] = rs.beta[t][s];
            wd[t * kSlots + s] = rs.w[t][s];
            af[t * kSlots + s] = (float)rs.alpha[t][s];
            bf[t * kSlots + s] = (float)rs.beta[t][s];
            wf[t * kSlots + s] = (float)rs.w[t][s];
        }
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_alpha_f, af, sizeof af));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_beta_f, bf, sizeof bf));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_w_f, wf, sizeof wf));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_alpha_d, ad, sizeof ad));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_beta_d, bd, sizeof bd));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_w_d, wd, sizeof wd));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_rule_n, rs.n, sizeof rs.n));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_rule_start, rs.start, sizeof rs.start));
    if (dev < 32) uploaded_mask |= 1 << dev;
    return BEM_OK;
}

template <bool F64, int PT, bool WANT_E, int MODE, bool STATS>
int launch_one(const FarK& k, cudaStream_t s) {
    constexpr size_t sm = far_smem_bytes<F64, PT, WANT_E, MODE>();
    auto fn = k_far<F64, PT, WANT_E, MODE, STATS>;
    static int per_sm = 0, sms = 0;  // per instantiation
    if (!per_sm) {
        BEM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        int dev = 0;
        BEM_CUDA_TRY(cudaGetDevice(&dev));
        BEM_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        BEM_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kWarps * 32, sm));
        if (per_sm < 1) per_sm = 1;
    }
    if (k.n_items == 0) return BEM_OK;
    const int want = (k.n_items + kWarps - 1) / kWarps;
    const int grid = want < per_sm * sms ? want : per_sm * sms;
    fn<<<grid, kWarps * 32, sm, s>>>(k);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}

template <bool F64, int PT, bool WANT_E, int MODE>
int launch_stats(const FarK& k, cudaStream_t s, bool stats) {
    return stats ? launch_one<F64, PT, WANT_E, MODE, true>(k, s) : launch_one<F64, PT, WANT_E, MODE, false>(k, s);
}
}  // namespace

int far_points_per_tile(int precision) { return 32 * (precision == kFP64 ? kPtFp64 : kPtMixed); }

int launch_far(bem_mesh* m, const FarArgs& a, cudaStream_t s) {
    int rc = upload_rules(m->device);
    if (rc) return rc;
    FarK k;
    k.pts = a.pts;
    k.perm = a.perm;
    k.n_pts = a.n_pts;
    k.n_el = m->d.n;
    k.work = a.work;
    k.chi = m->d.chi; k.clo = m->d.clo; k.e0f = m->d.e0; k.e1f = m->d.e1;
    k.cen = m->d.cen; k.fr = m->d.fr; k.geo = m->d.geo;
    k.type = m->d.type;
    k.sigma = a.sigma;
    k.part = a.part;
    k.near_cnt = a.near_cnt;
    k.near_rec = a.near_rec;
    k.counters = a.counters;
    k.near_cap = a.near_cap;
    k.A = a.A;
    k.kc = a.kc;
    k.bbox = a.bbox;
    k.coord_max = (float)m->coord_max;
    k.n_dev = a.n_dev;
    for (int t = 0; t < 2; ++t)
        for (int i = 0; i < 5; ++i) {
            k.tau2d[t][i] = m->limits[t][i] * m->limits[t][i];
            k.tau2f[t][i] = (float)k.tau2d[t][i];
        }
    const bool f64 = m->precision == kFP64;
    const int tile = far_points_per_tile(m->precision);
    const int n_tiles = (a.n_pts + tile - 1) / tile;
    if (a.A) {
        // assembly has no reduction over elements: cut them finely enough to fill the GPU
        const int chunks = (152 * 16 * 2 + n_tiles - 1) / n_tiles;
        int len = (m->d.n + chunks - 1) / chunks;
        len = ((len + 31) / 32) * 32;
        k.chunk_len = len;
        k.n_chunks = (m->d.n + len - 1) / len;
    } else {
        k.chunk_len = m->chunk_len;
        k.n_chunks = m->n_chunks;
    }
    k.n_items = n_tiles * k.n_chunks;
    k.tile_pts = tile;
    const bool st = a.stats != 0;
    if (a.A) {
        if (f64) return launch_stats<true, kPtFp64, false, 1>(k, s, st);
        return launch_stats<false, kPtMixed, false, 1>(k, s, st);
    }
    if (f64) {
        if (a.want_e) return launch_stats<true, kPtFp64, true, 0>(k, s, st);
        return launch_stats<true, kPtFp64, false, 0>(k, s, st);
    }
    if (a.want_e) return launch_stats<false, kPtMixed, true, 0>(k, s, st);
    return launch_stats<false, kPtMixed, false, 0>(k, s, st);
}

}  // namespace bem
