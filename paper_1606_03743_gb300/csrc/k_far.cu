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
//    node record i from the element frame: Eq. 3.2 / Eq. 3.3; a record is
//    one node, or on rectangles the pair of nodes o, -o), as offset and
//    weight records in a double-buffered shared-memory slot, then every lane runs
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
//  * FP64 path: everything in double precision, in the frame form below
//    (r_i^2 = s + |o_i|^2 + A_i u + B_i v, the field or its gradient rebuilt
//    per element, rectangle nodes in pairs o, -o).
//  * Mixed path: points and centroids are split into FP32 hi + lo parts with
//    the hi parts on one power-of-two grid fixed by the mesh, so that in
//    d = P - C = (P_hi - C_hi) + (P_lo - C_lo) the first difference is exact
//    and d is rounded once: FP32 relative accuracy anywhere in space, with
//    rounding errors that differ from element to element instead of one
//    common shift of the point.  The node offsets lie in the
//    element plane, o_i = alpha_i e0 + beta_i e1, so with u = d.e0, v = d.e1
//    and s = |d|^2 (once per point and element) each node needs only
//      r_i^2 = s + |o_i|^2 - 2 (alpha_i u + beta_i v),
//    and the field sum_i b_i (d - o_i) (b_i = w_i q / r_i^3) is rebuilt per
//    element from B = sum b_i, sum b_i alpha_i, sum b_i beta_i:
//      d B - e0 sum b_i alpha_i - e1 sum b_i beta_i.
//    With the node's weight also stored premultiplied by alpha_i and beta_i,
//    every sum takes one FMA: 9 FP32 operations and one rsqrt per node and
//    point instead of 13; two points of a lane go through packed f32x2
//    instructions together.  The rectangle rules (App. B) are centrally
//    symmetric: their nodes o and -o (equal weights) share s + |o|^2 and the
//    projection, r_+-^2 = s + |o|^2 -+ (alpha u + beta v), and their two
//    alpha, beta moments combine into one, w alpha (1/r_+^3 - 1/r_-^3): 16
//    operations for the two nodes.  A rule's centre node (alpha = beta = 0,
//    several rules of both types) needs r^2 = s only: 4 operations.
//    At DR >= 3 the terms of r_i^2 cancel by at most a factor of about 4, so
//    the split costs about two bits of an FP32 result.  rsqrt and the sums
//    are FP32: each element's node terms (at most 33) are summed on their
//    own, eight such element sums are added up, and that sum is added into
//    running sums kept in shared memory as unevaluated FP32 pairs hi + lo
//    (an exact two-sum: about 48 significant bits), so the FP64 pipe, slow
//    on this GPU, stays out of the loop.  No plain FP32 sum runs over more
//    than 33 terms.
#include <math.h>
#include <stdio.h>

#include <type_traits>

#include "bem_internal.cuh"
#include "bem_test.h"

namespace bem {

// field points per lane of the mixed and FP64 paths (a warp's tile is 32 x PT points)
#ifndef BEM_MIXED_PT
#define BEM_MIXED_PT 4
#endif
#ifndef BEM_FP64_PT
#define BEM_FP64_PT 2
#endif
constexpr int kPtMixed = BEM_MIXED_PT, kPtFp64 = BEM_FP64_PT;
#ifndef BEM_GRAD_PT
#define BEM_GRAD_PT 2
#endif
constexpr int kPtGradMixed = BEM_GRAD_PT;  // mixed gradient: seven sums per point pair and node
// mixed potential-only passes (assembly rows; matvec and phi-only evaluation)
#ifndef BEM_ASM_PT
#define BEM_ASM_PT BEM_MIXED_PT
#endif
#ifndef BEM_PHI_PT
#define BEM_PHI_PT BEM_MIXED_PT
#endif
constexpr int kPtAsm = BEM_ASM_PT, kPtPhi = BEM_PHI_PT;
// node-loop unroll depth
#ifndef BEM_NODE_UNROLL
#define BEM_NODE_UNROLL 4
#endif
constexpr int kNodeUnroll = BEM_NODE_UNROLL;
// mixed path: elements per FP32 sum before it moves into the hi + lo running sums (a power of two)
#ifndef BEM_FLUSH
#define BEM_FLUSH 8
#endif
constexpr int kFlush = BEM_FLUSH;
// the per-band (masked) passes of straddling elements run one generic node
// loop per element type (unrolled BEM_MASKED_UNROLL deep) instead of loops
// compiled per rule: the kernel is large enough for its code size to cost
// instruction-fetch stalls
#ifndef BEM_MASKED_UNROLL
#define BEM_MASKED_UNROLL 2
#endif
constexpr int kMaskedUnroll = BEM_MASKED_UNROLL;


static_assert((kFlush & (kFlush - 1)) == 0 && kFlush <= 32, "flush interval: a power of two up to 32");

constexpr int kSlots = 76;    // rule-table slots per element type (75 used at most)
constexpr int kWarps = 4;     // warps per CTA
constexpr int kNodeBuf = 33;  // nodes per buffer (the largest rule)
constexpr int kAsmGroup = 4;  // mixed assembly: elements per staged group (a 32-byte row segment)
// assembly work items per resident warp (elements are chunked finely enough for this many)
#ifndef BEM_ASM_ITEMS
#define BEM_ASM_ITEMS 32
#endif

__constant__ float c_alpha_f[2 * kSlots], c_beta_f[2 * kSlots], c_w_f[2 * kSlots];
__constant__ double c_alpha_d[2 * kSlots], c_beta_d[2 * kSlots], c_w_d[2 * kSlots];
__constant__ int c_rule_n[10];
// the rules as node records (FP32: c_alpha_f, c_beta_f, c_w_f; FP64: c_alpha_d, ...): per rule the
// centre node (if any), then one record per pair (o, -o) on rectangles or per node on triangles; the
// first record of each rule and its shape (centre records | other records << 1)
__constant__ int c_rec_start[10], c_rule_shape[10];

struct FarK {
    const double* pts;
    const int* perm;
    int n_pts, n_el;
    int n_chunks, chunk_len, n_items;
    int* work;  // work-item counter (zeroed before the launch)
    const float4 *chi, *clo, *e0f, *e1f;  // mixed element records
    const float4* nodes;                  // node table (BEM_FLAG_NODE_TABLE) or nullptr
    const double *cen, *fr, *geo;         // FP64 element data
    const int* type;
    const double* sigma;  // nullptr: unit density (assembly)
    const double* slope;  // linear densities: [n_el][2] slopes in the element frame, or nullptr
    const double* curv;   // quadratic densities: [n_el][3] alpha^2, alpha beta, beta^2 coefficients, or nullptr
    double4* part;        // per (tile, chunk, point of the tile) far sums (transient)
    double4* part_g;      // gradient pass: the same, 6 sums as two double4
    int* near_cnt;        // per (tile, chunk, point of the tile) near pairs (transient)
    double4* far;         // per sorted point: far sums over all chunks (gradient: far_g, two double4)
    double4* far_g;
    int* near_tot;        // per sorted point: near pairs over all chunks
    int* near_row;        // per sorted point with near pairs: its row of near_rows
    int* near_rows;       // [row][chunk]: near pairs of the point in the chunks before
    int* tile_done;       // [tile] finished work items; [n_tiles] the near_rows row counter
    unsigned long long part_cap, pts_cap;  // capacities (checked build): see FarArgs
    int4* near_rec;
    unsigned long long* counters;
    unsigned long long near_cap;
    double* A;
    double kc;
    float tau2f[2][5];
    double tau2d[2][5];
    const unsigned* bbox;  // field-point bounding box (order-preserving float bits: min xyz, max xyz)
    float coord_max;       // largest |coordinate| of the mesh
    double grid, inv_grid; // mixed path: grid of the hi parts (a power of two) and its inverse
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
// Near pairs are recorded as runs: a run is a sequence of consecutive elements
// of one chunk that are all in the analytic band for one point, recorded as
// (sorted point, first element, ordinal of its first pair among the point's
// near pairs in the chunk, number of pairs).  Point q of a lane is sorted point
// tile_base + 32 q + lane; its open run (first element, length) and its pair
// counter (the next ordinal) live in the warp's shared memory.
constexpr int kMaxRun = 1 << 20;  // a longer run is split

// Append the runs of the lanes marked in `emit` (point q) to the list.
__device__ __forceinline__ void emit_runs(const FarK& p, bool emit, int sp, int first, int ord, int len, int lane) {
    const unsigned m = __ballot_sync(0xffffffffu, emit);
    if (!m) return;
    const int leader = __ffs(m) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(p.counters, (unsigned long long)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (emit) {
        const unsigned long long idx = base + __popc(m & ((1u << lane) - 1u));
        if (idx < p.near_cap) p.near_rec[idx] = make_int4(sp, first, ord, len);
    }
}

// Element `elem` is in the analytic band for the points marked in want[q]:
// extend their open runs, or close them (append) and open new ones.
template <int PT>
__device__ __forceinline__ void note_near(const FarK& p, const bool (&want)[PT], int tile_base, int elem, int* run_first,
                                          int* run_len, int* ncnt, int lane) {
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int i = q * 32 + lane;
        int first = 0, len = 0, cnt = 0;
        bool close = false;
        if (want[q]) {  // only live points want pairs
            first = run_first[i];
            len = run_len[i];
            cnt = ncnt[i];
            close = len > 0 && (first + len != elem || len == kMaxRun);
        }
        emit_runs(p, close, tile_base + i, first, cnt - len, len, lane);
        if (want[q]) {
            if (len == 0 || close) {
                run_first[i] = elem;
                run_len[i] = 1;
            } else {
                run_len[i] = len + 1;
            }
            ncnt[i] = cnt + 1;
        }
    }
}

// End of a work item: append every open run; add the item's pairs to the pair counter.
template <int PT>
__device__ __forceinline__ void close_runs(const FarK& p, int tile_base, int n_pts, int* run_first, int* run_len,
                                           const int* ncnt, int lane) {
    int pairs = 0;
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int i = q * 32 + lane;
        const bool live = tile_base + i < n_pts;
        const int len = live ? run_len[i] : 0;
        const int cnt = live ? ncnt[i] : 0;
        pairs += cnt;
        emit_runs(p, len > 0, tile_base + i, live ? run_first[i] : 0, cnt - len, len, lane);
    }
    for (int o = 16; o; o >>= 1) pairs += __shfl_xor_sync(0xffffffffu, pairs, o);
    if (lane == 0 && pairs) atomicAdd(p.counters + kPairCounter, (unsigned long long)pairs);
}

// ---- FP64 path, frame form.  A node record is (A, B, |o|^2, w q) with
// A = -2 alpha, B = -2 beta, and per point s = |d|^2, u = d.e0, v = d.e1, so
// r^2 = s + |o|^2 + A u + B v.  The element's sums per point are
// (sum w q / r, sum b, sum b A, sum b B) with b = w q / r^3, and its field is
// d sum b + (e0 / 2) sum b A + (e1 / 2) sum b B.  A point that must not take
// part carries s = +inf: r^2 = +inf, rsqrt gives +0 and its terms are exact
// zeros.
template <int PT, bool WANT_E>
__device__ __forceinline__ void node64(const double4 o, const double (&s)[PT], const double (&u)[PT],
                                       const double (&v)[PT], double (&acc)[PT][4]) {
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const double r2 = fma(o.x, u[q], fma(o.y, v[q], s[q] + o.z));
        const double inv = rsqrt(r2);
        acc[q][0] = fma(o.w, inv, acc[q][0]);
        if (WANT_E) {
            const double b = o.w * (inv * (inv * inv));
            acc[q][1] += b;
            acc[q][2] = fma(o.x, b, acc[q][2]);
            acc[q][3] = fma(o.y, b, acc[q][3]);
        }
    }
}

// Nodes o and -o of equal weight (rectangle rules, App. B), record of the node
// at o: they share s + |o|^2 and m = A u + B v (r_+-^2 = s + |o|^2 +- m), and
// their A, B moments combine into A (b_+ - b_-).
template <int PT, bool WANT_E>
__device__ __forceinline__ void node64_pair(const double4 o, const double (&s)[PT], const double (&u)[PT],
                                            const double (&v)[PT], double (&acc)[PT][4]) {
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const double t = s[q] + o.z, m = fma(o.x, u[q], o.y * v[q]);
        const double ip = rsqrt(t + m), im = rsqrt(t - m);
        acc[q][0] = fma(o.w, im, fma(o.w, ip, acc[q][0]));
        if (WANT_E) {
            const double bp = o.w * (ip * (ip * ip)), bm = o.w * (im * (im * im));
            acc[q][1] = (acc[q][1] + bp) + bm;
            const double bd = bp - bm;
            acc[q][2] = fma(o.x, bd, acc[q][2]);
            acc[q][3] = fma(o.y, bd, acc[q][3]);
        }
    }
}

// A rule's centre node (alpha = beta = 0): r^2 = s.
template <int PT, bool WANT_E>
__device__ __forceinline__ void node64_centre(const double4 o, const double (&s)[PT], double (&acc)[PT][4]) {
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const double inv = rsqrt(s[q]);
        acc[q][0] = fma(o.w, inv, acc[q][0]);
        if (WANT_E) acc[q][1] += o.w * (inv * (inv * inv));
    }
}

// All records of one rule (shape = c | r << 1): the centre node, then pairs
// (rectangles, PAIRS) or single nodes.
template <int PT, bool WANT_E, bool PAIRS>
__device__ __forceinline__ void nodes64(const double4* __restrict__ nd, int ty, int shape, const double (&s)[PT],
                                        const double (&u)[PT], const double (&v)[PT], double (&acc)[PT][4]) {
    const int c = shape & 1, n = c + (shape >> 1);
    int i = 0;
    if (c) {
        node64_centre<PT, WANT_E>(nd[0], s, acc);
        i = 1;
    }
    if (PAIRS && ty == BEM_RECTANGLE) {
#pragma unroll 2
        for (; i < n; ++i) node64_pair<PT, WANT_E>(nd[i], s, u, v, acc);
    } else {
#pragma unroll 4
        for (; i < n; ++i) node64<PT, WANT_E>(nd[i], s, u, v, acc);
    }
}

// ---- FP64 field gradient, frame form (records as node64).  Per point the
// element's sums are g = (sum b, sum c, sum c A, sum c B, sum c A^2,
// sum c A B, sum c B^2) with b = w q / r^3, c = w q / r^5, from which the
// rebuild forms sum w q (I / r^3 - 3 r r^T / r^5) (the point-charge
// derivatives of Sec. 7), r = d - alpha e0 - beta e1.  Points that must not
// take part carry s = +inf.
template <int PT>
__device__ __forceinline__ void grad64_terms(double A, double B, double w, double inv, double (&g)[7]) {
    const double i2 = inv * inv, b = w * inv * i2, c = b * i2, ca = c * A, cb = c * B;
    g[0] += b;
    g[1] += c;
    g[2] += ca;
    g[3] += cb;
    g[4] = fma(ca, A, g[4]);
    g[5] = fma(ca, B, g[5]);
    g[6] = fma(cb, B, g[6]);
}

template <int PT, bool PAIRS>
__device__ __forceinline__ void nodes64_grad(const double4* __restrict__ nd, int ty, int shape, const double (&s)[PT],
                                             const double (&u)[PT], const double (&v)[PT], double (&g)[PT][7]) {
    const int c = shape & 1, n = c + ((shape >> 1) & 127);
    int i = 0;
    if (c) {  // centre node: r^2 = s, no alpha, beta moments
        const double w = nd[0].w;
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const double inv = rsqrt(s[q]), i2 = inv * inv, b = w * inv * i2;
            g[q][0] += b;
            g[q][1] += b * i2;
        }
        i = 1;
    }
    if (PAIRS && ty == BEM_RECTANGLE) {
        // nodes o, -o: b and c add up, the odd moments take c_+ - c_-, the even ones the sum
#pragma unroll 2
        for (; i < n; ++i) {
            const double4 o = nd[i];
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const double t = s[q] + o.z, m = fma(o.x, u[q], o.y * v[q]);
                const double ip = rsqrt(t + m), im = rsqrt(t - m);
                const double i2p = ip * ip, i2m = im * im;
                const double bp = o.w * ip * i2p, bm = o.w * im * i2m, cp = bp * i2p, cm = bm * i2m;
                const double cs = cp + cm, cd = cp - cm, ta = cs * o.x, tb = cs * o.y;
                g[q][0] += bp + bm;
                g[q][1] += cs;
                g[q][2] = fma(cd, o.x, g[q][2]);
                g[q][3] = fma(cd, o.y, g[q][3]);
                g[q][4] = fma(ta, o.x, g[q][4]);
                g[q][5] = fma(ta, o.y, g[q][5]);
                g[q][6] = fma(tb, o.y, g[q][6]);
            }
        }
    } else {
#pragma unroll 2
        for (; i < n; ++i) {
            const double4 o = nd[i];
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const double r2 = fma(o.x, u[q], fma(o.y, v[q], s[q] + o.z));
                grad64_terms<PT>(o.x, o.y, o.w, rsqrt(r2), g[q]);
            }
        }
    }
}

// ---- mixed path: two field points per packed f32x2 operation
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

// 16-byte asynchronous copy global -> shared (no registers), and its group fences
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    const unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(sa), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// hi + lo += x exactly up to the rounding of lo: the two addends ordered by
// magnitude (selects, off the FP32 pipe), then Dekker's fast two-sum, whose
// error term is exact for ordered addends -- the same hi and lo as Knuth's
// branch-free two-sum with two FP32 operations fewer (fma(a, -1, b) is b - a
// rounded once).  It keeps the running sums of the mixed path on the FP32
// pipe: a warp-wide FP64 add occupies this GPU's FP64 pipe for tens of cycles.
__device__ __forceinline__ void two_sum_add(float2& hi, float2& lo, float2 x) {
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const bool ox = fabsf(hi.x) >= fabsf(x.x), oy = fabsf(hi.y) >= fabsf(x.y);
    const float2 a = make_float2(ox ? hi.x : x.x, oy ? hi.y : x.y);  // the larger magnitude
    const float2 b = make_float2(ox ? x.x : hi.x, oy ? x.y : hi.y);
    const float2 sm = add2(a, b);
    const float2 z = fma2(a, m1, sm);  // sm - a, exact since |a| >= |b|
    const float2 er = fma2(z, m1, b);  // b - z: the exact rounding error of sm
    hi = sm;
    lo = add2(lo, er);
}

// One node of an element at the NP point pairs of a lane, in the frame form:
// ab = (-alpha, -alpha, -beta, -beta), ow = (|o|^2, |o|^2, w q, w q),
// wab = (-w q alpha, -w q alpha, -w q beta, -w q beta) / 2;
// s, u, v = |d|^2, 2 d.e0, 2 d.e1 per point (r^2 = s + |o|^2 - alpha u -
// beta v).  acc[k] = (sum a, sum b, -sum b alpha / 2, -sum b beta / 2) with
// a = w q / r, b = a / r^2 (phi only: sum a).  A point that must not take
// part carries s = +inf: then r^2 = +inf,
// rsqrt gives +0 and its terms are exact zeros, while the other points'
// arithmetic is bit-for-bit that of a pass without it.  INIT: the sums start
// from this term.
//
// GRAD (field gradient): acc[k] = (sum b, sum c, -sum c alpha, -sum c beta,
// sum c alpha^2, sum c alpha beta, sum c beta^2) with c = b / r^2 = w q / r^5,
// from which the rebuild forms sum q (I / r^3 - 3 r r^T / r^5) with
// r = d - alpha e0 - beta e1.
template <int NP, bool WANT_E, bool GRAD, bool INIT, int NS>
__device__ __forceinline__ void node2(const float4 ab, const float4 ow, const float4 wab, const float2 (&s)[NP],
                                      const float2 (&u)[NP], const float2 (&v)[NP], float2 (&acc)[NP][NS]) {
    const float2 al = make_float2(ab.x, ab.y), be = make_float2(ab.z, ab.w);
    const float2 oo = make_float2(ow.x, ow.y), w = make_float2(ow.z, ow.w);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float2 r2 = fma2(al, u[k], fma2(be, v[k], add2(s[k], oo)));
        const float2 inv = make_float2(rsqrtf(r2.x), rsqrtf(r2.y));
        if constexpr (GRAD) {
            static_assert(NS == 7, "gradient sums");
            const float2 i2 = mul2(inv, inv);
            const float2 b = mul2(mul2(w, inv), i2);  // q_i / r_i^3
            const float2 c = mul2(b, i2);             // q_i / r_i^5
            const float2 ca = mul2(c, al), cb = mul2(c, be);
            if (INIT) {
                acc[k][0] = b; acc[k][1] = c; acc[k][2] = ca; acc[k][3] = cb;
                acc[k][4] = mul2(ca, al); acc[k][5] = mul2(ca, be); acc[k][6] = mul2(cb, be);
            } else {
                acc[k][0] = add2(acc[k][0], b);
                acc[k][1] = add2(acc[k][1], c);
                acc[k][2] = add2(acc[k][2], ca);
                acc[k][3] = add2(acc[k][3], cb);
                acc[k][4] = fma2(ca, al, acc[k][4]);
                acc[k][5] = fma2(ca, be, acc[k][5]);
                acc[k][6] = fma2(cb, be, acc[k][6]);
            }
            continue;
        }
        // the third record, (-w alpha / 2, -w beta / 2): every sum is one FMA of its weight and
        // 1/r or 1/r^3
        if (INIT) acc[k][0] = mul2(w, inv);
        else acc[k][0] = fma2(w, inv, acc[k][0]);
        if (WANT_E) {
            const float2 i3 = mul2(inv, mul2(inv, inv));  // 1 / r_i^3
            const float2 wa = make_float2(wab.x, wab.y), wb = make_float2(wab.z, wab.w);
            if (INIT) {
                acc[k][1] = mul2(w, i3); acc[k][2] = mul2(wa, i3); acc[k][3] = mul2(wb, i3);
            } else {
                acc[k][1] = fma2(w, i3, acc[k][1]);
                acc[k][2] = fma2(wa, i3, acc[k][2]);
                acc[k][3] = fma2(wb, i3, acc[k][3]);
            }
        }
    }
}

// The centre node of a rule (alpha = beta = 0, so |o|^2 = 0 and r^2 = s):
// the point charge w q at the centroid.  ow = (0, 0, w q, w q).
template <int NP, bool WANT_E, bool GRAD, bool INIT, int NS>
__device__ __forceinline__ void node2_centre(const float4 ow, const float2 (&s)[NP], float2 (&acc)[NP][NS]) {
    const float2 w = make_float2(ow.z, ow.w), z = make_float2(0.0f, 0.0f);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float2 inv = make_float2(rsqrtf(s[k].x), rsqrtf(s[k].y));
        if constexpr (GRAD) {
            static_assert(NS == 7, "gradient sums");
            const float2 i2 = mul2(inv, inv);
            const float2 b = mul2(mul2(w, inv), i2);  // q / r^3
            const float2 c = mul2(b, i2);             // q / r^5
            if (INIT) {
                acc[k][0] = b; acc[k][1] = c;
#pragma unroll
                for (int j = 2; j < 7; ++j) acc[k][j] = z;
            } else {
                acc[k][0] = add2(acc[k][0], b);
                acc[k][1] = add2(acc[k][1], c);
            }
            continue;
        }
        if (INIT) acc[k][0] = mul2(w, inv);
        else acc[k][0] = fma2(w, inv, acc[k][0]);
        if (WANT_E) {
            const float2 i3 = mul2(inv, mul2(inv, inv));
            if (INIT) {
                acc[k][1] = mul2(w, i3); acc[k][2] = z; acc[k][3] = z;
            } else {
                acc[k][1] = fma2(w, i3, acc[k][1]);
            }
        }
    }
}

// The gradient sums of one node with its own (-alpha, -beta) = (al, be), weight w and 1 / r.
template <bool INIT>
__device__ __forceinline__ void grad_terms(const float2 al, const float2 be, const float2 w, const float2 inv,
                                           float2 (&acc)[7]) {
    const float2 i2 = mul2(inv, inv);
    const float2 b = mul2(mul2(w, inv), i2);  // q_i / r_i^3
    const float2 c = mul2(b, i2);             // q_i / r_i^5
    const float2 ca = mul2(c, al), cb = mul2(c, be);
    if (INIT) {
        acc[0] = b; acc[1] = c; acc[2] = ca; acc[3] = cb;
        acc[4] = mul2(ca, al); acc[5] = mul2(ca, be); acc[6] = mul2(cb, be);
    } else {
        acc[0] = add2(acc[0], b);
        acc[1] = add2(acc[1], c);
        acc[2] = add2(acc[2], ca);
        acc[3] = add2(acc[3], cb);
        acc[4] = fma2(ca, al, acc[4]);
        acc[5] = fma2(ca, be, acc[5]);
        acc[6] = fma2(cb, be, acc[6]);
    }
}

// Two nodes at o and -o with the same weight (the rectangle rules of App. B
// are centrally symmetric), records as node2() for the node at o.  They share
// s + |o|^2 and the projection m = -(alpha u + beta v):
//   r_+^2 = s + |o|^2 + m,  r_-^2 = s + |o|^2 - m,
// and the two alpha, beta moments combine: w alpha (1/r_+^3 - 1/r_-^3).
// 16 packed operations for the two nodes instead of 18.
template <int NP, bool WANT_E, bool GRAD, bool INIT, int NS>
__device__ __forceinline__ void node2_pair(const float4 ab, const float4 ow, const float4 wab, const float2 (&s)[NP],
                                           const float2 (&u)[NP], const float2 (&v)[NP], float2 (&acc)[NP][NS]) {
    const float2 al = make_float2(ab.x, ab.y), be = make_float2(ab.z, ab.w);
    const float2 oo = make_float2(ow.x, ow.y), w = make_float2(ow.z, ow.w);
    const float2 m1 = make_float2(-1.0f, -1.0f);
#pragma unroll
    for (int k = 0; k < NP; ++k) {
        const float2 t = add2(s[k], oo);
        const float2 m = fma2(al, u[k], mul2(be, v[k]));
        const float2 rp = add2(t, m), rm = fma2(m, m1, t);
        const float2 ip = make_float2(rsqrtf(rp.x), rsqrtf(rp.y)), im = make_float2(rsqrtf(rm.x), rsqrtf(rm.y));
        if constexpr (GRAD) {
            // the two nodes' sums: b = w/r^3 and c = w/r^5 add up, the odd moments
            // (c alpha, c beta) take the difference c_+ - c_-, the even ones the sum
            static_assert(NS == 7, "gradient sums");
            const float2 i2p = mul2(ip, ip), i2m = mul2(im, im);
            const float2 bp = mul2(mul2(w, ip), i2p), bm = mul2(mul2(w, im), i2m);
            const float2 cp = mul2(bp, i2p), cm = mul2(bm, i2m);
            const float2 bs = add2(bp, bm), cs = add2(cp, cm), cd = fma2(cm, m1, cp);
            const float2 ta = mul2(cs, al), tb = mul2(cs, be);
            if (INIT) {
                acc[k][0] = bs; acc[k][1] = cs; acc[k][2] = mul2(al, cd); acc[k][3] = mul2(be, cd);
                acc[k][4] = mul2(ta, al); acc[k][5] = mul2(ta, be); acc[k][6] = mul2(tb, be);
            } else {
                acc[k][0] = add2(acc[k][0], bs);
                acc[k][1] = add2(acc[k][1], cs);
                acc[k][2] = fma2(al, cd, acc[k][2]);
                acc[k][3] = fma2(be, cd, acc[k][3]);
                acc[k][4] = fma2(ta, al, acc[k][4]);
                acc[k][5] = fma2(ta, be, acc[k][5]);
                acc[k][6] = fma2(tb, be, acc[k][6]);
            }
            continue;
        }
        if (INIT) acc[k][0] = mul2(w, ip);
        else acc[k][0] = fma2(w, ip, acc[k][0]);
        acc[k][0] = fma2(w, im, acc[k][0]);
        if (WANT_E) {
            const float2 i3p = mul2(ip, mul2(ip, ip)), i3m = mul2(im, mul2(im, im));
            const float2 dd = fma2(i3m, m1, i3p);  // 1/r_+^3 - 1/r_-^3
            const float2 wa = make_float2(wab.x, wab.y), wb = make_float2(wab.z, wab.w);
            if (INIT) {
                acc[k][1] = mul2(w, i3p); acc[k][2] = mul2(wa, dd); acc[k][3] = mul2(wb, dd);
            } else {
                acc[k][1] = fma2(w, i3p, acc[k][1]);
                acc[k][2] = fma2(wa, dd, acc[k][2]);
                acc[k][3] = fma2(wb, dd, acc[k][3]);
            }
            acc[k][1] = fma2(w, i3m, acc[k][1]);
        }
    }
}

// Shape of a rule's node records: c centre records (0 or 1) | r other records << 1
__host__ __device__ inline int shape_c(int sh) { return sh & 1; }
__host__ __device__ inline int shape_r(int sh) { return sh >> 1; }

// Record i of a node buffer (kNodeRecs float4 per record).
#define BEM_REC(nd, i) (nd)[kNodeRecs * (i)], (nd)[kNodeRecs * (i) + 1], (nd)[kNodeRecs * (i) + kNodeRecs - 1]

// One node record of a rule: a pair (o, -o) on rectangles, a single node on triangles.
template <bool PAIR, int NP, bool WANT_E, bool GRAD, bool INIT, int NS>
__device__ __forceinline__ void node2_rec(const float4* __restrict__ nd, int i, const float2 (&s)[NP],
                                          const float2 (&u)[NP], const float2 (&v)[NP], float2 (&acc)[NP][NS]) {
    if constexpr (PAIR) node2_pair<NP, WANT_E, GRAD, INIT>(BEM_REC(nd, i), s, u, v, acc);
    else node2<NP, WANT_E, GRAD, INIT>(BEM_REC(nd, i), s, u, v, acc);
}

// All records of one rule with the shape known at compile time: C centre
// records (0 or 1) first, then R other records (pairs if PAIR), fully unrolled.
template <int C, int R, bool PAIR, int NP, bool WANT_E, bool GRAD, bool INIT, int NS>
__device__ __forceinline__ void nodes2_shape(const float4* __restrict__ nd, const float2 (&s)[NP],
                                             const float2 (&u)[NP], const float2 (&v)[NP], float2 (&acc)[NP][NS]) {
    if constexpr (C) {
        node2_centre<NP, WANT_E, GRAD, INIT>(nd[1], s, acc);
    } else {
        node2_rec<PAIR, NP, WANT_E, GRAD, INIT>(nd, 0, s, u, v, acc);
    }
#pragma unroll
    for (int i = 1; i < C + R; ++i) node2_rec<PAIR, NP, WANT_E, GRAD, false>(nd, i, s, u, v, acc);
}

// The same with the shape read at run time (c centre records, r others).
template <int UNROLL, bool PAIR, int NP, bool WANT_E, bool GRAD, bool INIT, int NS>
__device__ __forceinline__ void nodes2_loop(const float4* __restrict__ nd, int c, int r, const float2 (&s)[NP],
                                            const float2 (&u)[NP], const float2 (&v)[NP], float2 (&acc)[NP][NS]) {
    int i = 0;
    if (c) {
        node2_centre<NP, WANT_E, GRAD, INIT>(nd[1], s, acc);
        i = 1;
    } else if (INIT) {  // every rule has at least two records
        node2_rec<PAIR, NP, WANT_E, GRAD, true>(nd, 0, s, u, v, acc);
        i = 1;
    }
#pragma unroll UNROLL
    for (; i < c + r; ++i) node2_rec<PAIR, NP, WANT_E, GRAD, false>(nd, i, s, u, v, acc);
}

// All records of one rule of an element of type ty, shape = c | r << 1.  The
// rules with 7 and 12 nodes, which carry most of the work, get their own
// fully unrolled code; the per-band passes of straddling elements (INIT
// false) share one loop per element type.  PAIRS false (varying densities,
// whose paired nodes carry different charges): every record is one node.
template <int NP, bool WANT_E, bool GRAD, bool INIT, bool PAIRS, int NS>
__device__ __forceinline__ void nodes2(const float4* __restrict__ nd, int ty, int shape, const float2 (&s)[NP],
                                       const float2 (&u)[NP], const float2 (&v)[NP], float2 (&acc)[NP][NS]) {
    const int c = shape_c(shape), r = shape_r(shape);
    if (PAIRS && ty == BEM_RECTANGLE) {
        if constexpr (INIT) {
            if (shape == (1 | 3 << 1)) return nodes2_shape<1, 3, true, NP, WANT_E, GRAD, INIT>(nd, s, u, v, acc);
            if (shape == (0 | 6 << 1)) return nodes2_shape<0, 6, true, NP, WANT_E, GRAD, INIT>(nd, s, u, v, acc);
            return nodes2_loop<1, true, NP, WANT_E, GRAD, INIT>(nd, c, r, s, u, v, acc);
        }
        return nodes2_loop<1, true, NP, WANT_E, GRAD, INIT>(nd, c, r, s, u, v, acc);
    }
    if constexpr (INIT) {
        if (shape == (1 | 6 << 1)) return nodes2_shape<1, 6, false, NP, WANT_E, GRAD, INIT>(nd, s, u, v, acc);
        if (shape == (0 | 12 << 1)) return nodes2_shape<0, 12, false, NP, WANT_E, GRAD, INIT>(nd, s, u, v, acc);
        return nodes2_loop<kNodeUnroll, false, NP, WANT_E, GRAD, INIT>(nd, c, r, s, u, v, acc);
    }
    return nodes2_loop<kMaskedUnroll, false, NP, WANT_E, GRAD, INIT>(nd, c, r, s, u, v, acc);
}

// Shared memory of one warp.
template <typename R, typename R4, int PT, int NACC, bool ATILE = false>
struct WarpSmem {
    static constexpr bool kMixed = sizeof(R) == 4;
    // mixed assembly: kc x potential of kAsmGroup elements for the warp's points, written out
    // as short contiguous row segments; and the matrix row of each point of the tile
    double at[ATILE ? kAsmGroup * PT * 32 : 1];
    int rows[ATILE ? PT * 32 : 1];
    R4 c[kMixed ? 1 : 32];   // FP64: centroid, w = type
    R4 e0[kMixed ? 1 : 32];  // FP64: frame e0, w = q (element charge)
    R4 e1[kMixed ? 1 : 32];  // FP64: frame e1
    float2 qt[kMixed ? 32 : 1];  // mixed: element charge q, type (int bits); the frame is in pr
    R thr[32 * 5];           // squared band limits (tau L)^2
    R sl[2 * 32];            // linear densities: area x (d sigma / d alpha, d sigma / d beta), else 0
    // mixed: per element, the values each node pass and the field rebuild
    // read, duplicated into (x, x, y, y) pairs for the packed f32x2 arithmetic:
    // -C_hi, -C_lo, 2 e0, 2 e1 (six float4; the doubling is exact and makes the
    // projections 2 d.e0, 2 d.e1 of the node loop one FMA chain each)
    float4 pr[kMixed ? 32 * 6 : 1];

    R4 nd[2][kMixed ? kNodeRecs * kNodeBuf : kNodeBuf];  // node records (FP64: one per node; mixed: kNodeRecs)
    // mixed evaluation (NACC = 4: phi, E) and gradient (NACC = 6): per point pair,
    // component and lane, the running sum as an unevaluated FP32 pair hi + lo
    // (hi.x, hi.y, lo.x, lo.y)
    float4 accdf[NACC ? (PT / 2) * NACC * 32 : 1];
    int ncnt[PT * 32];  // near pairs found so far per point of the tile (their ordinals)
    int run_first[PT * 32], run_len[PT * 32];  // each point's open run of near pairs
};

template <typename R>
struct RuleSmem {
    R al[2 * kSlots], be[2 * kSlots], w[2 * kSlots];
    int n[10], start[10], shape[10];  // nodes, first slot (mixed: first record), shape (mixed)
    unsigned long long stat[15];  // 12 band counts, uniform / mixed (warp, element) pairs, node evaluations
};

template <bool F64, int PT, bool WANT_E, int MODE>
constexpr size_t far_smem_bytes() {
    using R = typename std::conditional<F64, double, float>::type;
    using R4 = typename std::conditional<F64, double4, float4>::type;
    constexpr int NACC = F64 ? 0 : MODE == 0 ? 4 : MODE == 3 ? 6 : 0;
    return ((sizeof(RuleSmem<R>) + 15) / 16) * 16 + kWarps * sizeof(WarpSmem<R, R4, PT, NACC, !F64 && MODE == 1>);
}

// A double4 read at L2 (past L1, which may hold stale lines of other SMs' writes).
__device__ __forceinline__ double4 ldcg4(const double4* a) {
    const double2 lo = __ldcg(reinterpret_cast<const double2*>(a));
    const double2 hi = __ldcg(reinterpret_cast<const double2*>(a) + 1);
    return make_double4(lo.x, lo.y, hi.x, hi.y);
}

// Drop a 128-byte line from L2 without writing it back (its data is used up).
__device__ __forceinline__ void discard_l2(const void* line) {
    asm volatile("discard.global.L2 [%0], 128;" ::"l"(line) : "memory");
}

// End of a work item that wrote its partial sums (NPART double4 per point) and
// near-pair counts into the item's slots of the tile-major areas.  The tile's
// last item to finish -- told by a per-tile counter -- sums every chunk's
// partials in chunk order (the same additions, in the same order, whatever
// batch the points came in: the results stay batch-independent), counts the
// near pairs per point with their per-chunk prefix, and then discards the
// tile's slots from L2: they are never read again, so they need no write-back
// to HBM.  The usual split-phase pattern: stores, a device fence, the counter;
// the last item fences again and reads past L1.
template <int NPART, int PT>
__device__ __forceinline__ void finish_tile(const FarK& p, const double4* part, double4* far, int tile, int base,
                                            int n_pts, int n_tiles, int lane) {
    __threadfence();
    __syncwarp();
    int last = 0;
    if (lane == 0) last = atomicAdd(p.tile_done + tile, 1) == p.n_chunks - 1;
    last = __shfl_sync(0xffffffffu, last, 0);
    if (!last) return;
    __threadfence();
    const int nc = p.n_chunks, tp = p.tile_pts;
    const size_t tbase = (size_t)tile * nc * tp;
    const bool slots_ok = check_ok(tbase + (size_t)nc * tp <= p.part_cap, p.counters, kCheckPart);
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        const int sp = base + q * 32 + lane;
        if (sp >= n_pts || !slots_ok || !check_ok((unsigned long long)sp < p.pts_cap, p.counters, kCheckPoint)) continue;
        double s[4 * NPART];
#pragma unroll
        for (int k = 0; k < 4 * NPART; ++k) s[k] = 0.0;
        int tot = 0;
        for (int c = 0; c < nc; ++c) {
            const size_t slot = tbase + (size_t)c * tp + q * 32 + lane;
#pragma unroll
            for (int j = 0; j < NPART; ++j) {
                const double4 v = ldcg4(part + NPART * slot + j);
                if (NPART == 1 && c == 0) {  // the evaluation's sum starts from the first chunk
                    s[0] = v.x; s[1] = v.y; s[2] = v.z; s[3] = v.w;
                } else {
                    s[4 * j] += v.x; s[4 * j + 1] += v.y; s[4 * j + 2] += v.z; s[4 * j + 3] += v.w;
                }
            }
            tot += __ldcg(p.near_cnt + slot);
        }
#pragma unroll
        for (int j = 0; j < NPART; ++j) far[NPART * (size_t)sp + j] = make_double4(s[4 * j], s[4 * j + 1], s[4 * j + 2], s[4 * j + 3]);
        p.near_tot[sp] = tot;
        if (tot > 0) {
            const int r = atomicAdd(p.tile_done + n_tiles, 1);
            if (!check_ok((unsigned long long)r < p.pts_cap, p.counters, kCheckRow)) continue;
            p.near_row[sp] = r;
            int run = 0;
            for (int c = 0; c < nc; ++c) {
                p.near_rows[(size_t)r * nc + c] = run;
                run += __ldcg(p.near_cnt + tbase + (size_t)c * tp + q * 32 + lane);
            }
        }
    }
    if (!slots_ok) return;
    const char* pa = reinterpret_cast<const char*>(part + NPART * tbase);
    const size_t pbytes = sizeof(double4) * NPART * (size_t)nc * tp;
    for (size_t off = (size_t)lane * 128; off < pbytes; off += 32 * 128) discard_l2(pa + off);
    const char* pc = reinterpret_cast<const char*>(p.near_cnt + tbase);
    const size_t cbytes = sizeof(int) * (size_t)nc * tp;
    for (size_t off = (size_t)lane * 128; off < cbytes; off += 32 * 128) discard_l2(pc + off);
}

// ------------------------------------------------------------ the kernel
// MODE 0: evaluation (sum over elements); MODE 1: assembly (one value per
// (point, element) pair written to A, potential only, sigma = 1); MODE 2
// (FP64) and MODE 3 (mixed): field gradient sums.
// STATS: count pairs per (type, band) into counters[2 + 6 type + band], and
// into counters[16..18] the (warp, element) pairs that ran one band for the
// whole warp, those that fell back to per-point bands, and the node
// evaluations executed (lanes x points x nodes, masked ones included).
// VAR: 0 constant densities, nodes formed on the fly; 1 the node table
// (BEM_FLAG_NODE_TABLE); 2 linear / quadratic densities (sigma at every node,
// formed on the fly).  Each variant carries only its own expansion code: the
// kernel is large enough for extra code to cost instruction-fetch stalls.
// CTAs per SM the register allocation must allow (4 x 4 warps)
#ifndef BEM_MIN_BLOCKS
#define BEM_MIN_BLOCKS 4
#endif
template <bool F64, int PT, bool WANT_E, int MODE, bool STATS, int VAR>
__global__ void __launch_bounds__(kWarps * 32, BEM_MIN_BLOCKS) k_far(const FarK p) {
    constexpr bool PRE = VAR == 1, VARY = VAR == 2;
    using R = typename std::conditional<F64, double, float>::type;
    using R4 = typename std::conditional<F64, double4, float4>::type;
    // running sums in shared memory (mixed evaluation: phi, E; mixed gradient: 6 components)
    constexpr int NACC = F64 ? 0 : MODE == 0 ? 4 : MODE == 3 ? 6 : 0;
    constexpr bool ATILE = !F64 && MODE == 1;  // mixed assembly: row segments staged in shared memory
    static_assert(MODE != 3 || !F64, "MODE 3 is the mixed gradient");
    static_assert(MODE != 2 || F64, "MODE 2 is the FP64 gradient");
    constexpr bool GRAD3 = MODE == 3;
    constexpr int NE = GRAD3 ? 7 : 4;  // per-element sums of a point pair (mixed path)
    using WS = WarpSmem<R, R4, PT, NACC, ATILE>;

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
        rs.start[tid] = c_rec_start[tid];
        rs.shape[tid] = c_rule_shape[tid];
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

    static_assert(F64 || PT % 2 == 0, "the mixed path works on point pairs");
    constexpr int NP = F64 ? 1 : PT / 2;  // point pairs of a lane (mixed path)
    for (;;) {
        int item = 0;
        if (lane == 0) item = atomicAdd(p.work, 1);
        item = __shfl_sync(0xffffffffu, item, 0);
        if (item >= n_items) break;
        // on-the-fly nodes: the chunks of one tile are neighbours; node table: the
        // tiles of one chunk are (so that the chunk's records stay in L2)
        int tile, chunk;
        if (PRE) {
            const int n_tiles = (n_pts + p.tile_pts - 1) / p.tile_pts;
            chunk = item / n_tiles;
            tile = item - chunk * n_tiles;
        } else {
            tile = item / p.n_chunks;
            chunk = item - tile * p.n_chunks;
        }
        const int base = tile * (32 * PT);

        // ---- field points of this lane
        R px[PT], py[PT], pz[PT];      // FP64: the point; mixed: hi part
        float lx[PT], ly[PT], lz[PT];  // mixed: lo part
        // point q of this lane: sorted point base + 32 q + lane; a slot past the end takes a
        // live point of the tile (its results are not stored).  Formed when needed rather
        // than held in registers through the element loop.
        auto valid = [&](int q) { return base + q * 32 + lane < n_pts; };
        auto sidx = [&](int q) { return valid(q) ? base + q * 32 + lane : base; };
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const int i = sidx(q);
            ws.ncnt[q * 32 + lane] = 0;
            ws.run_len[q * 32 + lane] = 0;
            const int src = p.perm[i];
            const double X = p.pts[3 * (size_t)src], Y = p.pts[3 * (size_t)src + 1], Z = p.pts[3 * (size_t)src + 2];
            if constexpr (F64) {
                px[q] = X; py[q] = Y; pz[q] = Z;
                lx[q] = ly[q] = lz[q] = 0.0f;
            } else {
                // hi part on the centroids' grid (exact differences P_hi - C_hi), lo part the rest
                const double hX = rint(X * p.inv_grid) * p.grid, hY = rint(Y * p.inv_grid) * p.grid,
                             hZ = rint(Z * p.inv_grid) * p.grid;
                px[q] = (float)hX; py[q] = (float)hY; pz[q] = (float)hZ;
                lx[q] = (float)(X - (double)px[q]); ly[q] = (float)(Y - (double)py[q]);
                lz[q] = (float)(Z - (double)pz[q]);
            }
        }
        // ---- bounding sphere of the tile (FP32, only for the band test)
        float wcx, wcy, wcz, wrad, wmag;
        {
            float mn[3] = {1e30f, 1e30f, 1e30f}, mx[3] = {-1e30f, -1e30f, -1e30f};
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const float v[3] = {(float)px[q] + lx[q], (float)py[q] + ly[q], (float)pz[q] + lz[q]};
#pragma unroll
                for (int k = 0; k < 3; ++k) { mn[k] = fminf(mn[k], v[k]); mx[k] = fmaxf(mx[k], v[k]); }
            }
#pragma unroll
            for (int k = 0; k < 3; ++k) { mn[k] = warp_min(mn[k]); mx[k] = warp_max(mx[k]); }
            wcx = 0.5f * (mn[0] + mx[0]); wcy = 0.5f * (mn[1] + mx[1]); wcz = 0.5f * (mn[2] + mx[2]);
            float r2 = 0.0f;
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                const float ax = ((float)px[q] + lx[q]) - wcx, ay = ((float)py[q] + ly[q]) - wcy,
                            az = ((float)pz[q] + lz[q]) - wcz;
                r2 = fmaxf(r2, ax * ax + ay * ay + az * az);
            }
            wrad = sqrtf(warp_max(r2));
            wmag = sqrtf(wcx * wcx + wcy * wcy + wcz * wcz) + wrad;
        }
        int nvalid = 0;  // valid points of the tile (for the statistics)
        if (STATS) nvalid = min(32 * PT, n_pts - base);
        // mixed path: points 2k and 2k+1 of the lane as packed pairs (hi, lo parts)
        float2 P2[3][NP], L2[3][NP];
#pragma unroll
        for (int k = 0; k < NP; ++k) {
            if constexpr (!F64) {
                P2[0][k] = make_float2(px[2 * k], px[2 * k + 1]);
                P2[1][k] = make_float2(py[2 * k], py[2 * k + 1]);
                P2[2][k] = make_float2(pz[2 * k], pz[2 * k + 1]);
                L2[0][k] = make_float2(lx[2 * k], lx[2 * k + 1]);
                L2[1][k] = make_float2(ly[2 * k], ly[2 * k + 1]);
                L2[2][k] = make_float2(lz[2 * k], lz[2 * k + 1]);
            }
        }

        // ---- accumulators
        R acc[F64 ? PT : 1][4];  // FP64 evaluation: the running sums
        R accg[MODE == 2 ? PT : 1][6];  // gradient pass: the running sums
        constexpr int NA = GRAD3 ? 6 : 4;
        float2 acc8[NP][NA];  // mixed: FP32 sum of up to 8 element results (point pairs)
#pragma unroll
        for (int q = 0; q < PT; ++q) {
#pragma unroll
            for (int c = 0; c < 4; ++c)
                if constexpr (F64) acc[q][c] = (R)0;
            if constexpr (MODE == 2) {
#pragma unroll
                for (int c = 0; c < 6; ++c) accg[q][c] = (R)0;
            }
        }
        if constexpr (NACC > 0) {
#pragma unroll
            for (int k = 0; k < NP * NACC; ++k) ws.accdf[k * 32 + lane] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
        }
#pragma unroll
        for (int k = 0; k < NP; ++k)
#pragma unroll
            for (int c = 0; c < NA; ++c) acc8[k][c] = make_float2(0.0f, 0.0f);

        const int el0 = chunk * p.chunk_len, el1 = min(p.n_el, el0 + p.chunk_len);
        if constexpr (ATILE) {
#pragma unroll
            for (int q = 0; q < PT; ++q) ws.rows[q * 32 + lane] = valid(q) ? p.perm[sidx(q)] : -1;
            __syncwarp();
        }
        int par = 0;    // node buffer parity
        int pre_n = 0;  // node table: node count of the next element's records already in flight
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
                    if constexpr (VARY) {
                        ws.sl[2 * lane] = (R)(p.slope[2 * j] * area);
                        ws.sl[2 * lane + 1] = (R)(p.slope[2 * j + 1] * area);
                    }
                    R4 c, cl;
                    float th[5];
                    if constexpr (F64) {
                        const double L = p.geo[2 * j];
                        c = R4{p.cen[3 * j], p.cen[3 * j + 1], p.cen[3 * j + 2], (double)ty};
                        cl = R4{0, 0, 0, L};
                        ws.e0[lane] = R4{p.fr[6 * j], p.fr[6 * j + 1], p.fr[6 * j + 2], sg * area};
                        ws.e1[lane] = R4{p.fr[6 * j + 3], p.fr[6 * j + 4], p.fr[6 * j + 5], 0.0};
                        ws.c[lane] = c;
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            const double t = p.tau2d[ty][k] * L * L;
                            ws.thr[lane * 5 + k] = t;
                            th[k] = (float)t;
                        }
                    } else {
                        c = p.chi[j];
                        cl = p.clo[j];
                        const float4 a = p.e0f[j], b = p.e1f[j];
                        ws.qt[lane] = make_float2((float)(sg * area), __int_as_float(ty));
                        float4* pr = ws.pr + lane * 6;
                        pr[0] = make_float4(-c.x, -c.x, -c.y, -c.y);
                        pr[1] = make_float4(-c.z, -c.z, -cl.x, -cl.x);
                        pr[2] = make_float4(-cl.y, -cl.y, -cl.z, -cl.z);
                        pr[3] = make_float4(2.0f * a.x, 2.0f * a.x, 2.0f * a.y, 2.0f * a.y);
                        pr[4] = make_float4(2.0f * a.z, 2.0f * a.z, 2.0f * b.x, 2.0f * b.x);
                        pr[5] = make_float4(2.0f * b.y, 2.0f * b.y, 2.0f * b.z, 2.0f * b.z);
                        const float L = cl.w;
#pragma unroll
                        for (int k = 0; k < 5; ++k) {
                            th[k] = p.tau2f[ty][k] * L * L;
                            ws.thr[lane * 5 + k] = th[k];
                        }
                    }
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
                int ty;
                if constexpr (F64) ty = (int)ws.c[e].w;
                else ty = __float_as_int(ws.qt[e].y);

                if constexpr (F64) {
                    // ---------------- FP64 path: d = P - C, the frame form (node64, nodes64_grad)
                    const R4 c = ws.c[e];
                    R dx[PT], dy[PT], dz[PT];
#pragma unroll
                    for (int q = 0; q < PT; ++q) {
                        dx[q] = px[q] - c.x; dy[q] = py[q] - c.y; dz[q] = pz[q] - c.z;
                    }
                    constexpr bool kGrad = MODE == 2;
                    // varying densities: the two nodes of a rectangle's pair as two records
                    const bool split = VARY && ty == BEM_RECTANGLE;
                    auto rule_shape64 = [&](int r) -> int {
                        const int sh = rs.shape[ty * 5 + r];
                        return split ? shape_c(sh) | shape_r(sh) << 2 : sh;
                    };
                    // expand rule r of element e into the free node buffer (lane k: output record k);
                    // returns the rule's node count
                    auto expand = [&](int r) -> int {
                        const int n = rs.n[ty * 5 + r], st = ty * kSlots + rs.start[ty * 5 + r];
                        const int shape = rs.shape[ty * 5 + r], c0 = shape_c(shape), nrec = c0 + shape_r(shape);
                        const int nout = split ? 2 * nrec - c0 : nrec;
                        const R4 a = ws.e0[e], b = ws.e1[e];
                        R ca = (R)0, cb = (R)0, cc = (R)0;
                        if (VARY && p.curv) {  // quadratic densities: area x second-order coefficients
                            const size_t j = (size_t)(b0 + e);
                            const double ar = p.geo[2 * j + 1];
                            ca = (R)(p.curv[3 * j] * ar);
                            cb = (R)(p.curv[3 * j + 1] * ar);
                            cc = (R)(p.curv[3 * j + 2] * ar);
                        }
                        for (int k = lane; k < nout; k += 32) {
                            // output record k: table record i, its node o or (odd split records) -o
                            const int i = split && k >= c0 ? c0 + ((k - c0) >> 1) : k;
                            const bool neg = split && k >= c0 && ((k - c0) & 1);
                            const R al = neg ? -rs.al[st + i] : rs.al[st + i];
                            const R be = neg ? -rs.be[st + i] : rs.be[st + i];
                            // charge w_i area sigma(Q_i) (linear / quadratic densities: sigma at the node)
                            R qi = a.w;
                            if constexpr (VARY) {
                                qi = fmad(al, ws.sl[2 * e], fmad(be, ws.sl[2 * e + 1], qi));
                                if (p.curv) qi = fmad(al, fmad(al, ca, be * cb), fmad(be * be, cc, qi));
                            }
                            const R ox = fmad(al, a.x, be * b.x), oy = fmad(al, a.y, be * b.y), oz = fmad(al, a.z, be * b.z);
                            const R wq = rs.w[st + i] * qi;
                            ws.nd[par][k] = R4{-2.0 * al, -2.0 * be, fmad(ox, ox, fmad(oy, oy, oz * oz)), wq};
                        }
                        __syncwarp();
                        return n;
                    };

                    // frame form: s = |d|^2, u = d.e0, v = d.e1; the element's sums (eacc, gacc)
                    R sv[PT], uv[PT], vv[PT];
                    R eacc[kGrad ? 1 : PT][4], gacc[kGrad ? PT : 1][7];
                    {
                        const R4 a = ws.e0[e], b = ws.e1[e];
#pragma unroll
                        for (int q = 0; q < PT; ++q) {
                            sv[q] = fmad(dx[q], dx[q], fmad(dy[q], dy[q], dz[q] * dz[q]));
                            uv[q] = fmad(dx[q], a.x, fmad(dy[q], a.y, dz[q] * a.z));
                            vv[q] = fmad(dx[q], b.x, fmad(dy[q], b.y, dz[q] * b.z));
                            if constexpr (kGrad) {
#pragma unroll
                                for (int k = 0; k < 7; ++k) gacc[q][k] = (R)0;
                            } else {
#pragma unroll
                                for (int k = 0; k < 4; ++k) eacc[q][k] = (R)0;
                            }
                        }
                    }

                    if (cd >= 1 && cd <= 5) {
                        const int n = expand(band_rule(cd));
                        if constexpr (kGrad) nodes64_grad<PT, !VARY>(ws.nd[par], ty, rule_shape64(band_rule(cd)), sv, uv, vv, gacc);
                        else nodes64<PT, WANT_E, !VARY>(ws.nd[par], ty, rule_shape64(band_rule(cd)), sv, uv, vv, eacc);
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
                            const R d2 = fmad(dx[q], dx[q], fmad(dy[q], dy[q], dz[q] * dz[q]));
                            bq[q] = band_of<R>(d2, th);
                            if (valid(q)) mask |= 1u << bq[q];
                        }
                        mask = __reduce_or_sync(0xffffffffu, mask);
                        if (mask & 1u) {
                            bool want[PT];
#pragma unroll
                            for (int q = 0; q < PT; ++q) want[q] = valid(q) && bq[q] == 0;
                            note_near<PT>(p, want, base, b0 + e, ws.run_first, ws.run_len, ws.ncnt, lane);
                        }
#pragma unroll 1
                        for (int band = 1; band <= 5; ++band) {
                            if (!(mask & (1u << band))) continue;
                            const int n = expand(band_rule(band));
                            // points of other bands sit at infinite distance in this pass
                            R sm[PT];
#pragma unroll
                            for (int q = 0; q < PT; ++q) sm[q] = bq[q] == band ? sv[q] : (R)INFINITY;
                            if constexpr (kGrad) nodes64_grad<PT, !VARY>(ws.nd[par], ty, rule_shape64(band_rule(band)), sm, uv, vv, gacc);
                            else nodes64<PT, WANT_E, !VARY>(ws.nd[par], ty, rule_shape64(band_rule(band)), sm, uv, vv, eacc);
                            par ^= 1;
                            if (STATS && lane == 0) atomicAdd(&rs.stat[14], (unsigned long long)n * 32 * PT);
                        }
                        if (STATS) {
                            if (lane == 0) atomicAdd(&rs.stat[13], 1ull);
#pragma unroll
                            for (int q = 0; q < PT; ++q) {
                                for (int band = 0; band <= 5; ++band) {
                                    const unsigned m = __ballot_sync(0xffffffffu, valid(q) && bq[q] == band);
                                    if (lane == 0 && m) atomicAdd(&rs.stat[6 * ty + band], (unsigned long long)__popc(m));
                                }
                            }
                        }
                    }
                    if constexpr (MODE == 0) {
                        // the element's phi and E = d B + (e0 / 2) sum b A + (e1 / 2) sum b B into the running sums
                        const R4 a = ws.e0[e], b = ws.e1[e];
#pragma unroll
                        for (int q = 0; q < PT; ++q) {
                            acc[q][0] += eacc[q][0];
                            if (WANT_E) {
                                const R ha = 0.5 * eacc[q][2], hb = 0.5 * eacc[q][3];
                                acc[q][1] += fmad(dx[q], eacc[q][1], fmad(a.x, ha, b.x * hb));
                                acc[q][2] += fmad(dy[q], eacc[q][1], fmad(a.y, ha, b.y * hb));
                                acc[q][3] += fmad(dz[q], eacc[q][1], fmad(a.z, ha, b.z * hb));
                            }
                        }
                    }
                    if constexpr (MODE == 1) {
                        // assembly: one potential per pair, times 1/(4 pi eps0); near pairs are filled later
#pragma unroll
                        for (int q = 0; q < PT; ++q)
                            if (valid(q)) {
                                const int row = p.perm[sidx(q)];
                                if (check_ok(row >= 0 && row < p.n_pts && b0 + e < p.n_el, p.counters, kCheckMatrix))
                                    p.A[(size_t)row * p.n_el + (b0 + e)] = p.kc * (double)eacc[q][0];
                            }
                    }
                    if constexpr (kGrad) {
                        // the element's sum w q (I / r^3 - 3 r r^T / r^5), r = d - alpha e0 - beta e1:
                        // with S = sum c, S_a = sum c alpha, ... (alpha = -A / 2), it is
                        // sum b I - 3 (M d^T + N0 e0^T + N1 e1^T), M = S d - S_a e0 - S_b e1,
                        // N0 = -S_a d + S_aa e0 + S_ab e1, N1 = -S_b d + S_ab e0 + S_bb e1
                        const R4 a = ws.e0[e], b = ws.e1[e];
                        const R f0[3] = {a.x, a.y, a.z}, f1[3] = {b.x, b.y, b.z};
#pragma unroll
                        for (int q = 0; q < PT; ++q) {
                            const R* G = gacc[q];
                            const R Sa = -0.5 * G[2], Sb = -0.5 * G[3], Saa = 0.25 * G[4], Sab = 0.25 * G[5],
                                    Sbb = 0.25 * G[6];
                            const R dv[3] = {dx[q], dy[q], dz[q]};
                            R M[3], N0[3], N1[3];
#pragma unroll
                            for (int k = 0; k < 3; ++k) {
                                M[k] = fmad(G[1], dv[k], fmad(-Sa, f0[k], -Sb * f1[k]));
                                N0[k] = fmad(-Sa, dv[k], fmad(Saa, f0[k], Sab * f1[k]));
                                N1[k] = fmad(-Sb, dv[k], fmad(Sab, f0[k], Sbb * f1[k]));
                            }
                            auto T = [&](int i, int j) { return fmad(M[i], dv[j], fmad(N0[i], f0[j], N1[i] * f1[j])); };
                            accg[q][0] += fmad(-3.0, T(0, 0), G[0]);
                            accg[q][1] += fmad(-3.0, T(1, 1), G[0]);
                            accg[q][2] += fmad(-3.0, T(2, 2), G[0]);
                            accg[q][3] -= 3.0 * T(0, 1);
                            accg[q][4] -= 3.0 * T(0, 2);
                            accg[q][5] -= 3.0 * T(1, 2);
                        }
                    }
                } else {
                    // ---------------- mixed path (frame form, point pairs)
                    // d = (P_hi - C_hi) + (P_lo - C_lo) of pair k, the first difference exact
                    const float4* pr = ws.pr + e * 6;
                    auto lo2 = [](float4 v) { return make_float2(v.x, v.y); };
                    auto hi2 = [](float4 v) { return make_float2(v.z, v.w); };
                    auto diff = [&](int k, float2& dx, float2& dy, float2& dz) {
                        const float4 r0 = pr[0], r1 = pr[1], r2 = pr[2];
                        dx = add2(add2(P2[0][k], lo2(r0)), add2(L2[0][k], hi2(r1)));
                        dy = add2(add2(P2[1][k], hi2(r0)), add2(L2[1][k], lo2(r2)));
                        dz = add2(add2(P2[2][k], lo2(r1)), add2(L2[2][k], hi2(r2)));
                    };
                    // s = |d|^2, u = d.e0, v = d.e1 of every pair
                    float2 sv[NP], uv[NP], vv[NP];
                    float2 dxk[NP], dyk[NP], dzk[NP];  // d, held for the field rebuild
                    {
                        const float4 r3 = pr[3], r4 = pr[4], r5 = pr[5];
#pragma unroll
                        for (int k = 0; k < NP; ++k) {
                            float2 dx, dy, dz;
                            diff(k, dx, dy, dz);
                            dxk[k] = dx; dyk[k] = dy; dzk[k] = dz;
                            sv[k] = fma2(dx, dx, fma2(dy, dy, mul2(dz, dz)));
                            const float2 u = fma2(dx, lo2(r3), fma2(dy, hi2(r3), mul2(dz, lo2(r4))));
                            const float2 v = fma2(dx, hi2(r4), fma2(dy, lo2(r5), mul2(dz, hi2(r5))));
                            uv[k] = u;  // 2 d.e0, 2 d.e1 (the frame records hold 2 e0, 2 e1)
                            vv[k] = v;
                        }
                    }
                    float2 eacc[NP][NE];  // this element's sums (started by its first rule pass)
                    // shape of rule r's records in the node buffer (varying densities: rectangle pairs split)
                    auto rule_shape = [&](int r) -> int {
                        const int sh = rs.shape[ty * 5 + r];
                        return VARY && ty == BEM_RECTANGLE ? shape_c(sh) | shape_r(sh) << 2 : sh;
                    };
                    // expand rule r of element e into the free node buffer (lane i: node i)
                    auto expand = [&](int r) -> int {
                        const int n = rs.n[ty * 5 + r], st = ty * kSlots + rs.start[ty * 5 + r];
                        const int shape = rs.shape[ty * 5 + r], nrec = shape_c(shape) + shape_r(shape);
                        // the doubled frame from the duplicated records: 2 (e0x, e0x, e0y, e0y),
                        // 2 (e0z, e0z, e1x, e1x), 2 (e1y, e1y, e1z, e1z), taken with alpha / 2 and
                        // beta / 2 (exact scalings); the charge from qt
                        const float4 r3 = pr[3], r4 = pr[4], r5 = pr[5];
                        const float4 f0 = make_float4(r3.x, r3.z, r4.x, ws.qt[e].x), f1 = make_float4(r4.z, r5.x, r5.z, 0.0f);
                        float ca = 0.0f, cb = 0.0f, cc = 0.0f;
                        if (VARY && p.curv) {  // quadratic densities: area x second-order coefficients
                            const size_t j = (size_t)(b0 + e);
                            const double ar = p.geo[2 * j + 1];
                            ca = (float)(p.curv[3 * j] * ar);
                            cb = (float)(p.curv[3 * j + 1] * ar);
                            cc = (float)(p.curv[3 * j + 2] * ar);
                        }
                        // varying densities: the two nodes of a pair carry different charges, so a
                        // rectangle's pair record i >= c becomes the single records c + 2 (i - c) (node
                        // o) and the one after it (node -o)
                        const bool split = VARY && ty == BEM_RECTANGLE;
                        const int c = shape_c(shape), nout = split ? 2 * nrec - c : nrec;
                        for (int k = lane; k < nout; k += 32) {
                            // output record k: table record i, its node o or (odd split records) -o
                            const int i = split && k >= c ? c + ((k - c) >> 1) : k;
                            const bool neg = split && k >= c && ((k - c) & 1);
                            const float al = neg ? -rs.al[st + i] : rs.al[st + i];
                            const float be = neg ? -rs.be[st + i] : rs.be[st + i];
                            const float ah = 0.5f * al, bh = 0.5f * be;
                            const float ox = fmaf(ah, f0.x, bh * f1.x), oy = fmaf(ah, f0.y, bh * f1.y),
                                        oz = fmaf(ah, f0.z, bh * f1.z);
                            const float oo = fmaf(ox, ox, fmaf(oy, oy, oz * oz));
                            // charge w_i area sigma(Q_i) (linear / quadratic densities: sigma at the node)
                            float qi = f0.w;
                            if constexpr (VARY) {
                                qi = fmaf(al, ws.sl[2 * e], fmaf(be, ws.sl[2 * e + 1], qi));
                                if (p.curv) qi = fmaf(al, fmaf(al, ca, be * cb), fmaf(be * be, cc, qi));
                            }
                            const float am = -al, bm = -be, wq = rs.w[st + i] * qi, wh = 0.5f * wq;
                            ws.nd[par][kNodeRecs * k] = make_float4(am, am, bm, bm);
                            ws.nd[par][kNodeRecs * k + 1] = make_float4(oo, oo, wq, wq);
                            const float wa = wh * am, wb = wh * bm;  // halved: times the doubled frame
                            ws.nd[par][kNodeRecs * k + 2] = make_float4(wa, wa, wb, wb);
                        }
                        __syncwarp();
                        return n;
                    };
                    // node table: copy rule r of element el (type t) into buffer buf
                    // asynchronously (lane i: node i); the caller waits and syncs
                    auto fetch = [&](int el, int t, int r, int buf) -> int {
                        const int n = rs.n[t * 5 + r], shape = rs.shape[t * 5 + r];
                        const float4* src = p.nodes + ((size_t)el * kTableSlots + rs.start[t * 5 + r]) * kNodeRecs;
                        for (int i = lane; i < shape_c(shape) + shape_r(shape); i += 32) {
#pragma unroll
                            for (int k = 0; k < kNodeRecs; ++k)
                                cp_async16(&ws.nd[buf][kNodeRecs * i + k], src + kNodeRecs * i + k);
                        }
                        cp_async_commit();
                        return n;
                    };

                    if (cd >= 1 && cd <= 5) {
                        int n;
                        if constexpr (PRE) {
                            // this element's records (fetched during the previous element if
                            // that was a one-band element), then the next element's, whose
                            // copy runs while this element's node loop does
                            n = pre_n ? pre_n : fetch(b0 + e, ty, band_rule(cd), par);
                            cp_async_wait_all();
                            __syncwarp();
                            pre_n = 0;
                            if (e + 1 < nb) {
                                const int cdn = __shfl_sync(0xffffffffu, code, e + 1);
                                if (cdn >= 1 && cdn <= 5)
                                    pre_n = fetch(b0 + e + 1, __float_as_int(ws.qt[e + 1].y), band_rule(cdn), par ^ 1);
                            }
                        } else {
                            n = expand(band_rule(cd));
                        }
                        // the element's first node starts its sums
                        nodes2<NP, WANT_E, GRAD3, true, !VARY>(ws.nd[par], ty, rule_shape(band_rule(cd)), sv, uv, vv, eacc);
                        par ^= 1;
                        if (STATS && lane == 0) {
                            atomicAdd(&rs.stat[6 * ty + cd], (unsigned long long)nvalid);
                            atomicAdd(&rs.stat[12], 1ull);
                            atomicAdd(&rs.stat[14], (unsigned long long)n * 32 * PT);
                        }
                    } else {
                        // per-point bands
                        int bq[PT];
                        const float* th = ws.thr + e * 5;
                        unsigned mask = 0;
#pragma unroll
                        for (int k = 0; k < NP; ++k) {
                            bq[2 * k] = band_of<float>(sv[k].x, th);
                            bq[2 * k + 1] = band_of<float>(sv[k].y, th);
                        }
#pragma unroll
                        for (int q = 0; q < PT; ++q)
                            if (valid(q)) mask |= 1u << bq[q];
                        mask = __reduce_or_sync(0xffffffffu, mask);
                        if (mask & 1u) {
                            bool want[PT];
#pragma unroll
                            for (int q = 0; q < PT; ++q) want[q] = valid(q) && bq[q] == 0;
                            note_near<PT>(p, want, base, b0 + e, ws.run_first, ws.run_len, ws.ncnt, lane);
                        }
#pragma unroll
                        for (int k = 0; k < NP; ++k)
#pragma unroll
                            for (int j = 0; j < NE; ++j) eacc[k][j] = make_float2(0.0f, 0.0f);  // near-only points
#pragma unroll 1
                        for (int band = 1; band <= 5; ++band) {
                            if (!(mask & (1u << band))) continue;
                            // points of other bands sit at infinite distance in this pass
                            constexpr float kInf = __builtin_huge_valf();
                            float2 sm[NP];
#pragma unroll
                            for (int k = 0; k < NP; ++k)
                                sm[k] = make_float2(bq[2 * k] == band ? sv[k].x : kInf,
                                                    bq[2 * k + 1] == band ? sv[k].y : kInf);
                            int n;
                            if constexpr (PRE) {
                                n = fetch(b0 + e, ty, band_rule(band), par);
                                cp_async_wait_all();
                                __syncwarp();
                            } else {
                                n = expand(band_rule(band));
                            }
                            nodes2<NP, WANT_E, GRAD3, false, !VARY>(ws.nd[par], ty, rule_shape(band_rule(band)), sm, uv, vv, eacc);
                            par ^= 1;
                            if (STATS && lane == 0) atomicAdd(&rs.stat[14], (unsigned long long)n * 32 * PT);
                        }
                        if (STATS) {
                            if (lane == 0) atomicAdd(&rs.stat[13], 1ull);
#pragma unroll
                            for (int q = 0; q < PT; ++q) {
                                for (int band = 0; band <= 5; ++band) {
                                    const unsigned m = __ballot_sync(0xffffffffu, valid(q) && bq[q] == band);
                                    if (lane == 0 && m) atomicAdd(&rs.stat[6 * ty + band], (unsigned long long)__popc(m));
                                }
                            }
                        }
                    }

                    if constexpr (PRE) {  // the table's weights carry no charge: scale the element's sums
                        const float q = ws.qt[e].x;
                        const float2 q2 = make_float2(q, q);
#pragma unroll
                        for (int k = 0; k < NP; ++k)
#pragma unroll
                            for (int j = 0; j < (WANT_E ? 4 : 1); ++j) eacc[k][j] = mul2(eacc[k][j], q2);
                    }
                    if constexpr (MODE == 0) {
                        // the element's phi and E = d B - e0 sum b alpha - e1 sum b beta (the
                        // records hold 2 e0, 2 e1 and the sums half of sum b alpha, sum b beta)
                        // into the FP32 sums; every kFlush elements move those into the hi + lo sums
                        const float4 r3 = pr[3], r4 = pr[4], r5 = pr[5];
                        const float2 h0x = lo2(r3), h0y = hi2(r3), h0z = lo2(r4);
                        const float2 h1x = hi2(r4), h1y = lo2(r5), h1z = hi2(r5);
#pragma unroll
                        for (int k = 0; k < NP; ++k) {
                            acc8[k][0] = add2(acc8[k][0], eacc[k][0]);
                            if (WANT_E) {
                                const float2 dx = dxk[k], dy = dyk[k], dz = dzk[k];
                                acc8[k][1] = fma2(dx, eacc[k][1], fma2(h0x, eacc[k][2], fma2(h1x, eacc[k][3], acc8[k][1])));
                                acc8[k][2] = fma2(dy, eacc[k][1], fma2(h0y, eacc[k][2], fma2(h1y, eacc[k][3], acc8[k][2])));
                                acc8[k][3] = fma2(dz, eacc[k][1], fma2(h0z, eacc[k][2], fma2(h1z, eacc[k][3], acc8[k][3])));
                            }
                        }
                        if (((b0 + e) & (kFlush - 1)) == kFlush - 1 || e == nb - 1) {
#pragma unroll
                            for (int k = 0; k < NP; ++k)
#pragma unroll
                                for (int j = 0; j < 4; ++j) {
                                    float4& slot = ws.accdf[(k * 4 + j) * 32 + lane];
                                    const float4 v = slot;
                                    float2 hi = make_float2(v.x, v.y), lo = make_float2(v.z, v.w);
                                    two_sum_add(hi, lo, acc8[k][j]);
                                    slot = make_float4(hi.x, hi.y, lo.x, lo.y);
                                    acc8[k][j] = make_float2(0.0f, 0.0f);
                                }
                        }
                    }
                    if constexpr (GRAD3) {
                        // the element's gradient sum q (I / r^3 - 3 r r^T / r^5), r = d - alpha e0 -
                        // beta e1: with M = C0 d + Ca e0 + Cb e1, N0 = Ca d + Caa e0 + Cab e1,
                        // N1 = Cb d + Cab e0 + Cbb e1 (C the sums of node2, Ca = -sum c alpha, ...)
                        // it is B I - 3 (M d^T + N0 e0^T + N1 e1^T)
                        const float4 r3 = pr[3], r4 = pr[4], r5 = pr[5];
                        const float2 hf = make_float2(0.5f, 0.5f);  // the records hold 2 e0, 2 e1
                        const float2 h0x = mul2(hf, lo2(r3)), h0y = mul2(hf, hi2(r3)), h0z = mul2(hf, lo2(r4));
                        const float2 h1x = mul2(hf, hi2(r4)), h1y = mul2(hf, lo2(r5)), h1z = mul2(hf, hi2(r5));
                        const float2 m3 = make_float2(-3.0f, -3.0f);
#pragma unroll
                        for (int k = 0; k < NP; ++k) {
                            float2 dx, dy, dz;
                            diff(k, dx, dy, dz);
                            const float2* c = eacc[k];
                            const float2 mx = fma2(c[1], dx, fma2(c[2], h0x, mul2(c[3], h1x)));
                            const float2 my = fma2(c[1], dy, fma2(c[2], h0y, mul2(c[3], h1y)));
                            const float2 mz = fma2(c[1], dz, fma2(c[2], h0z, mul2(c[3], h1z)));
                            const float2 ax = fma2(c[2], dx, fma2(c[4], h0x, mul2(c[5], h1x)));
                            const float2 ay = fma2(c[2], dy, fma2(c[4], h0y, mul2(c[5], h1y)));
                            const float2 az = fma2(c[2], dz, fma2(c[4], h0z, mul2(c[5], h1z)));
                            const float2 bx = fma2(c[3], dx, fma2(c[5], h0x, mul2(c[6], h1x)));
                            const float2 by = fma2(c[3], dy, fma2(c[5], h0y, mul2(c[6], h1y)));
                            const float2 bz = fma2(c[3], dz, fma2(c[5], h0z, mul2(c[6], h1z)));
                            // (xx, yy, zz, xy, xz, yz)
                            const float2 txx = fma2(mx, dx, fma2(ax, h0x, mul2(bx, h1x)));
                            const float2 tyy = fma2(my, dy, fma2(ay, h0y, mul2(by, h1y)));
                            const float2 tzz = fma2(mz, dz, fma2(az, h0z, mul2(bz, h1z)));
                            const float2 txy = fma2(mx, dy, fma2(ax, h0y, mul2(bx, h1y)));
                            const float2 txz = fma2(mx, dz, fma2(ax, h0z, mul2(bx, h1z)));
                            const float2 tyz = fma2(my, dz, fma2(ay, h0z, mul2(by, h1z)));
                            acc8[k][0] = add2(acc8[k][0], fma2(m3, txx, c[0]));
                            acc8[k][1] = add2(acc8[k][1], fma2(m3, tyy, c[0]));
                            acc8[k][2] = add2(acc8[k][2], fma2(m3, tzz, c[0]));
                            acc8[k][3] = fma2(m3, txy, acc8[k][3]);
                            acc8[k][4] = fma2(m3, txz, acc8[k][4]);
                            acc8[k][5] = fma2(m3, tyz, acc8[k][5]);
                        }
                        if (((b0 + e) & (kFlush - 1)) == kFlush - 1 || e == nb - 1) {
#pragma unroll
                            for (int k = 0; k < NP; ++k)
#pragma unroll
                                for (int j = 0; j < 6; ++j) {
                                    float4& slot = ws.accdf[(k * 6 + j) * 32 + lane];
                                    const float4 v = slot;
                                    float2 hi = make_float2(v.x, v.y), lo = make_float2(v.z, v.w);
                                    two_sum_add(hi, lo, acc8[k][j]);
                                    slot = make_float4(hi.x, hi.y, lo.x, lo.y);
                                    acc8[k][j] = make_float2(0.0f, 0.0f);
                                }
                        }
                    }
                    if constexpr (MODE == 1) {
                        // assembly: one potential per pair, times 1/(4 pi eps0), staged for a group
                        // of kAsmGroup elements and written as row segments (near pairs are
                        // filled later)
                        const int g = e & (kAsmGroup - 1);
#pragma unroll
                        for (int k = 0; k < NP; ++k) {
                            ws.at[g * (PT * 32) + (2 * k) * 32 + lane] = p.kc * (double)eacc[k][0].x;
                            ws.at[g * (PT * 32) + (2 * k + 1) * 32 + lane] = p.kc * (double)eacc[k][0].y;
                        }
                        if (g == kAsmGroup - 1 || e == nb - 1) {
                            __syncwarp();
                            const int gn = g + 1, col0 = b0 + e - g;
                            // lane l: point slot 8 j + l / 4, column l % 4 of the group
                            const int sub = lane & (kAsmGroup - 1);
#pragma unroll 4
                            for (int j = 0; j < PT * 32 / 8; ++j) {
                                const int ps = j * 8 + (lane >> 2);
                                const int row = ws.rows[ps];
                                if (row >= 0 && sub < gn &&
                                    check_ok(row < p.n_pts && col0 + sub < p.n_el, p.counters, kCheckMatrix))
                                    p.A[(size_t)row * p.n_el + (col0 + sub)] = ws.at[sub * (PT * 32) + ps];
                            }
                            __syncwarp();
                        }
                    }
                }
            }
        }

        // ---- the item's open near-pair runs
        close_runs<PT>(p, base, n_pts, ws.run_first, ws.run_len, ws.ncnt, lane);
        // ---- this item's partial sums and near-pair counts, then the tile's reduction
        constexpr int NPART = MODE == 0 ? 1 : (MODE == 2 || MODE == 3) ? 2 : 0;
        if constexpr (NPART > 0) {
            double4* part = NPART == 1 ? p.part : p.part_g;
            const size_t ibase = ((size_t)tile * p.n_chunks + chunk) * p.tile_pts;
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                if (!valid(q)) continue;
                const size_t slot = ibase + q * 32 + lane;
                if (!check_ok(slot < p.part_cap, p.counters, kCheckPart)) continue;
                if constexpr (MODE == 0) {
                    double4 o;
                    if constexpr (F64) {
                        o = make_double4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
                    } else {
                        double c4[4];
#pragma unroll
                        for (int j = 0; j < 4; ++j) {
                            const float4 v = ws.accdf[((q >> 1) * 4 + j) * 32 + lane];
                            c4[j] = (q & 1) ? (double)v.y + (double)v.w : (double)v.x + (double)v.z;
                        }
                        o = make_double4(c4[0], c4[1], c4[2], c4[3]);
                    }
                    part[slot] = o;
                } else {
                    double g6[6];
#pragma unroll
                    for (int j = 0; j < 6; ++j) {
                        if constexpr (MODE == 2) {
                            g6[j] = accg[q][j];
                        } else {
                            const float4 v = ws.accdf[((q >> 1) * 6 + j) * 32 + lane];
                            g6[j] = (q & 1) ? (double)v.y + (double)v.w : (double)v.x + (double)v.z;
                        }
                    }
                    part[2 * slot] = make_double4(g6[0], g6[1], g6[2], g6[3]);
                    part[2 * slot + 1] = make_double4(g6[4], g6[5], 0.0, 0.0);
                }
                p.near_cnt[slot] = ws.ncnt[q * 32 + lane];
            }
            const int n_tiles = (p.n_pts + p.tile_pts - 1) / p.tile_pts;  // capacity tiles (counter layout)
            finish_tile<NPART, PT>(p, part, NPART == 1 ? p.far : p.far_g, tile, base, n_pts, n_tiles, lane);
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

// FP32 copies of one rule's n weights whose exact sum is one as closely as
// one-ulp nudges of single weights get it (within one ulp of the smallest
// weight).  Rounding each weight on its own leaves the sum off by up to a few
// 1e-8, which scales the charge of every element that uses the rule by the
// same factor: a systematic error that, unlike independent rounding errors,
// does not average out over many elements.
// A record that stands for a pair of nodes (mult 2) counts twice.
void round_weights(const double* w, const int* mult, int n, float* out) {
    for (int i = 0; i < n; ++i) out[i] = (float)w[i];
    for (int it = 0; it < 4 * n; ++it) {
        double sum = 0.0;  // exact: at most 33 floats within a few binades
        for (int i = 0; i < n; ++i) sum += mult[i] * (double)out[i];
        const double res = 1.0 - sum;
        if (res == 0.0) break;
        int best = -1;
        double best_err = fabs(res);
        float best_val = 0.0f;
        for (int i = 0; i < n; ++i) {
            const float c = nextafterf(out[i], res > 0.0 ? INFINITY : -INFINITY);
            const double err = fabs(res - mult[i] * ((double)c - (double)out[i]));
            if (err < best_err) {
                best_err = err;
                best = i;
                best_val = c;
            }
        }
        if (best < 0) break;
        out[best] = best_val;
    }
}

// The mixed path's node records of every rule: the centre node first (alpha =
// beta = 0, if the rule has one), then on rectangles one record per pair of
// nodes o, -o of equal weight (every rule of App. B is centrally symmetric),
// on triangles one record per node.  The FP32 weights are rounded so that the
// rule's weights, pairs counted twice, still sum to one.
int build_records(const RuleSet& rs, float* af, float* bf, float* wf, double* ad, double* bd, double* wd,
                  int* rec_start, int* shape) {
    for (int t = 0; t < 2; ++t) {
        int slot = 0;
        for (int r = 0; r < 5; ++r) {
            const int s0 = rs.start[t][r], n = rs.n[t][r];
            const double *al = &rs.alpha[t][s0], *be = &rs.beta[t][s0], *w = &rs.w[t][s0];
            double rw[kSlots];
            int idx[kSlots], mult[kSlots], nrec = 0, ncen = 0;
            bool used[kSlots] = {};
            for (int i = 0; i < n; ++i)
                if (al[i] == 0.0 && be[i] == 0.0) { idx[nrec] = i; mult[nrec++] = 1; used[i] = true; ++ncen; }
            for (int i = 0; i < n; ++i) {
                if (used[i]) continue;
                used[i] = true;
                int mate = -1;
                if (t == BEM_RECTANGLE)
                    for (int j = i + 1; j < n && mate < 0; ++j)
                        if (!used[j] && al[j] == -al[i] && be[j] == -be[i] && w[j] == w[i]) mate = j;
                if (t == BEM_RECTANGLE && mate < 0) {
                    set_error("rule tables: rectangle rule %d is not centrally symmetric", r);
                    return BEM_ERR_INVALID;
                }
                if (mate >= 0) used[mate] = true;
                idx[nrec] = i;
                mult[nrec++] = mate >= 0 ? 2 : 1;
            }
            if (ncen > 1 || nrec - ncen < 1) {
                set_error("rule tables: unexpected shape of rule %d", r);
                return BEM_ERR_INVALID;
            }
            for (int k = 0; k < nrec; ++k) {
                af[t * kSlots + slot + k] = (float)al[idx[k]];
                bf[t * kSlots + slot + k] = (float)be[idx[k]];
                rw[k] = w[idx[k]];
                ad[t * kSlots + slot + k] = al[idx[k]];
                bd[t * kSlots + slot + k] = be[idx[k]];
                wd[t * kSlots + slot + k] = w[idx[k]];
            }
            round_weights(rw, mult, nrec, &wf[t * kSlots + slot]);
            rec_start[t * 5 + r] = slot;
            shape[t * 5 + r] = ncen | (nrec - ncen) << 1;
            slot += nrec;
        }
    }
    return BEM_OK;
}

int upload_rules(int dev) {
    if (dev < 32 && (uploaded_mask >> dev) & 1) return BEM_OK;
    const RuleSet& rs = rules();
    float af[2 * kSlots] = {}, bf[2 * kSlots] = {}, wf[2 * kSlots] = {};
    double ad[2 * kSlots] = {}, bd[2 * kSlots] = {}, wd[2 * kSlots] = {};
    int rec_start[10], shape[10];
    const int rc = build_records(rs, af, bf, wf, ad, bd, wd, rec_start, shape);
    if (rc) return rc;
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_rec_start, rec_start, sizeof rec_start));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_rule_shape, shape, sizeof shape));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_alpha_f, af, sizeof af));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_beta_f, bf, sizeof bf));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_w_f, wf, sizeof wf));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_alpha_d, ad, sizeof ad));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_beta_d, bd, sizeof bd));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_w_d, wd, sizeof wd));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_rule_n, rs.n, sizeof rs.n));
    if (dev < 32) uploaded_mask |= 1 << dev;
    return BEM_OK;
}

template <bool F64, int PT, bool WANT_E, int MODE, bool STATS, int VAR>
int launch_one(const FarK& k, cudaStream_t s) {
    constexpr size_t sm = far_smem_bytes<F64, PT, WANT_E, MODE>();
    auto fn = k_far<F64, PT, WANT_E, MODE, STATS, VAR>;
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
    if constexpr (!F64 && MODE != 3) {
        if (k.nodes)
            return stats ? launch_one<F64, PT, WANT_E, MODE, true, 1>(k, s)
                         : launch_one<F64, PT, WANT_E, MODE, false, 1>(k, s);
    }
    if constexpr (MODE != 1) {  // linear / quadratic densities: evaluation and gradients
        if (k.slope)
            return stats ? launch_one<F64, PT, WANT_E, MODE, true, 2>(k, s)
                         : launch_one<F64, PT, WANT_E, MODE, false, 2>(k, s);
    }
    return stats ? launch_one<F64, PT, WANT_E, MODE, true, 0>(k, s)
                 : launch_one<F64, PT, WANT_E, MODE, false, 0>(k, s);
}

// Node records of every rule for every element (BEM_FLAG_NODE_TABLE): thread
// (element j, record slot) writes what the kernel's on-the-fly expansion
// writes, with the bare weight w in place of w q (rectangles use fewer slots:
// one record per pair of nodes).
__global__ void k_fill_nodes(int n, const float4* __restrict__ e0f, const float4* __restrict__ e1f,
                             const int* __restrict__ type, float4* __restrict__ out) {
    const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (long long)n * kTableSlots) return;
    const int j = (int)(id / kTableSlots), slot = (int)(id - (long long)j * kTableSlots);
    const int t = type[j];
    const float al = c_alpha_f[t * kSlots + slot], be = c_beta_f[t * kSlots + slot], w = c_w_f[t * kSlots + slot];
    const float4 f0 = e0f[j], f1 = e1f[j];
    const float ox = fmaf(al, f0.x, be * f1.x), oy = fmaf(al, f0.y, be * f1.y), oz = fmaf(al, f0.z, be * f1.z);
    const float oo = fmaf(ox, ox, fmaf(oy, oy, oz * oz));
    out[kNodeRecs * id] = make_float4(-al, -al, -be, -be);
    out[kNodeRecs * id + 1] = make_float4(oo, oo, w, w);
    const float wa = 0.5f * (w * -al), wb = 0.5f * (w * -be);  // halved: times the doubled frame
    out[kNodeRecs * id + 2] = make_float4(wa, wa, wb, wb);
}
}  // namespace

int launch_fill_nodes(bem_mesh* m, cudaStream_t s) {
    int rc = upload_rules(m->device);
    if (rc) return rc;
    const long long total = (long long)m->d.n * kTableSlots;
    if (total == 0) return BEM_OK;
    k_fill_nodes<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(m->d.n, m->d.e0, m->d.e1, m->d.type, m->d.nodes);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}


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
    // the node table's weights carry the element charge as one factor: constant densities only
    k.nodes = (m->precision == kFP64 || a.slope || a.part_g) ? nullptr : m->d.nodes;
    k.slope = a.slope;
    k.curv = eval_curv(m, a.slope);
    k.cen = m->d.cen; k.fr = m->d.fr; k.geo = m->d.geo;
    k.type = m->d.type;
    k.sigma = a.sigma;
    k.part = a.part;
    k.part_g = a.part_g;
    k.near_cnt = a.near_cnt;
    k.far = a.far;
    k.far_g = a.far_g;
    k.near_tot = a.near_tot;
    k.near_row = a.near_row;
    k.near_rows = a.near_rows;
    k.tile_done = a.tile_done;
    k.part_cap = a.part_cap;
    k.pts_cap = a.pts_cap;
    k.near_rec = a.near_rec;
    k.counters = a.counters;
    k.near_cap = a.near_cap;
    k.A = a.A;
    k.kc = a.kc;
    k.bbox = a.bbox;
    k.coord_max = (float)m->coord_max;
    k.grid = m->grid;
    k.inv_grid = 1.0 / m->grid;
    k.n_dev = a.n_dev;
    for (int t = 0; t < 2; ++t)
        for (int i = 0; i < 5; ++i) {
            k.tau2d[t][i] = m->limits[t][i] * m->limits[t][i];
            k.tau2f[t][i] = (float)k.tau2d[t][i];
        }
    const bool f64 = m->precision == kFP64;
    const int pt = f64 ? kPtFp64 : a.part_g ? kPtGradMixed : a.A ? kPtAsm : a.want_e ? kPtMixed : kPtPhi;
    const int tile = 32 * pt;
    const int n_tiles = (a.n_pts + tile - 1) / tile;
    if (a.A) {
        // assembly has no reduction over elements: cut them finely enough to fill the GPU
        const int chunks = (152 * 16 * BEM_ASM_ITEMS + n_tiles - 1) / n_tiles;
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
    if (!a.A) {  // per-tile item counters and the near_rows row counter start at zero
        if (!a.tile_done) {
            set_error("launch_far: no tile counters");
            return BEM_ERR_INVALID;
        }
        BEM_CUDA_TRY(cudaMemsetAsync(a.tile_done, 0, sizeof(int) * ((size_t)n_tiles + 1), s));
    }
    const bool st = a.stats != 0;
    if (a.part_g) {  // field gradient: the mesh's precision
        if (f64) return launch_stats<true, kPtFp64, true, 2>(k, s, st);
        return launch_stats<false, kPtGradMixed, true, 3>(k, s, st);
    }
    if (a.A) {
        if (f64) return launch_stats<true, kPtFp64, false, 1>(k, s, st);
        return launch_stats<false, kPtAsm, false, 1>(k, s, st);
    }
    if (f64) {
        if (a.want_e) return launch_stats<true, kPtFp64, true, 0>(k, s, st);
        return launch_stats<true, kPtFp64, false, 0>(k, s, st);
    }
    if (a.want_e) return launch_stats<false, kPtMixed, true, 0>(k, s, st);
    return launch_stats<false, kPtPhi, false, 0>(k, s, st);
}

}  // namespace bem

extern "C" int32_t bem_test_rule_records(int32_t type, int32_t r, int32_t precision, double* out, int32_t* shape) {
    using namespace bem;
    if ((type != BEM_TRIANGLE && type != BEM_RECTANGLE) || r < 0 || r > 4 || !out || !shape ||
        (precision != 0 && precision != 1)) {
        set_error("bem_test_rule_records: bad arguments");
        return BEM_ERR_INVALID;
    }
    float af[2 * kSlots] = {}, bf[2 * kSlots] = {}, wf[2 * kSlots] = {};
    double ad[2 * kSlots] = {}, bd[2 * kSlots] = {}, wd[2 * kSlots] = {};
    int rec_start[10], sh[10];
    const int rc = build_records(rules(), af, bf, wf, ad, bd, wd, rec_start, sh);
    if (rc) return rc;
    const int k = type * 5 + r, n = shape_c(sh[k]) + shape_r(sh[k]);
    for (int i = 0; i < n; ++i) {
        const int j = type * kSlots + rec_start[k] + i;
        out[4 * i] = precision ? (double)af[j] : ad[j];
        out[4 * i + 1] = precision ? (double)bf[j] : bd[j];
        out[4 * i + 2] = precision ? (double)wf[j] : wd[j];
        out[4 * i + 3] = (type == BEM_RECTANGLE && !(i == 0 && shape_c(sh[k]))) ? 2.0 : 1.0;
    }
    *shape = sh[k];
    return n;
}
