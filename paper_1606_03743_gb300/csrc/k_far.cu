// k_far.cu -- far-field point-charge cubature (Eq. 4.1) with distance-ratio
// rule bands (Sec. 4) and compaction of the near-field pairs.
//
// Work decomposition (one launch covers every field point x every element):
//  * Field points arrive sorted by spatial cell; a CTA of NT threads owns
//    NT * PT consecutive points, each thread PT of them (a warp owns 32 * PT
//    neighbouring points).
//  * Elements stream through shared memory in tiles of TE.  For each tile the
//    CTA expands the nodes of all five rules of each element's type on the
//    fly (Eq. 3.2 / Eq. 3.3 from the element frame) into (offset, w_i q)
//    records, where q = sigma A is the element charge (Eq. 4.1).
//  * Band choice: one lane per element tests, conservatively, whether every
//    point of its warp falls into one distance-ratio band of that element;
//    if so the warp runs that rule with no per-point test (the common case
//    for sorted points).  Otherwise each point picks its own band and the
//    warp runs every band present with the other points' weights masked.
//    Either way a point always gets exactly the band of its own distance
//    ratio, so its result does not depend on which points share its warp.
//  * Pairs in the analytic band (DR below the near limit) are appended to a
//    compacted list with warp-aggregated atomics, with a per-point ordinal so
//    that the analytic pass can add them back in element order.
//
// Arithmetic:
//  * FP64 path: everything in double precision.
//  * Mixed path: the point-to-centroid difference is formed from FP32 hi/lo
//    splits of both points, (P_hi - C_hi) + (P_lo - C_lo), so it keeps FP32
//    relative accuracy even for points far from the origin; node offsets,
//    rsqrt and the sums are FP32: each element's node terms (at most 33) are
//    summed on their own, eight such element sums are added up, and that
//    sum is flushed into FP64 accumulators (kept in shared memory).  No FP32
//    sum therefore runs over more than 33 terms; the FP64 pipe sees two adds
//    per element and point.
#include <stdio.h>

#include <type_traits>

#include "bem_internal.cuh"

namespace bem {

constexpr int kSlots = 76;  // node slots per element in shared memory (75 used at most)

__constant__ float c_alpha_f[2][kMaxSlots], c_beta_f[2][kMaxSlots], c_w_f[2][kMaxSlots];
__constant__ double c_alpha_d[2][kMaxSlots], c_beta_d[2][kMaxSlots], c_w_d[2][kMaxSlots];
__constant__ int c_nslot[2], c_rule_n[2][5], c_rule_start[2][5];

struct FarK {
    const double* pts;
    const int* perm;
    int n_pts, n_el;
    int el_chunk;  // elements per CTA column (grid.y); a multiple of the tile, = n_el for evaluation
    const float4 *chi, *clo, *e0f, *e1f;                // mixed element records
    const double *cen, *fr, *geo;                         // FP64 element data
    const int* type;
    const double* sigma;
    double4* far;
    int* near_cnt;
    int4* near_rec;
    unsigned long long* counters;
    unsigned long long near_cap;
    double* A;
    double kc;
    float tau2f[2][5];
    double tau2d[2][5];
};

// ------------------------------------------------------------ warp helpers
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

// Warp-cooperative append of near pairs; want[q] marks point q of this lane.
template <int PT>
__device__ __forceinline__ void append_near(const FarK& p, const bool (&want)[PT], const int (&sidx)[PT], int elem,
                                            int (&ncnt)[PT], int lane) {
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
            if (idx < p.near_cap) p.near_rec[idx] = make_int4(sidx[q], elem, ncnt[q], 0);
            ++ncnt[q];
        }
    }
}

// ------------------------------------------------------------ node loops
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ float fmad(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double fmad(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tiny_floor(float x) { return fmaxf(x, 1e-30f); }
__device__ __forceinline__ double tiny_floor(double x) { return fmax(x, 1e-300); }

// Accumulate the point charges of one rule of one element into
// acc[q] = (phi, Ex, Ey, Ez) sums.  nd points at the rule's first
// (offset, w_i q) record in shared memory (warp-uniform address: a
// broadcast).  MASKED: only points q with bq[q] == band contribute.
template <typename R, typename R4, int PT, bool WANT_E, bool MASKED>
__device__ __forceinline__ void nodes(const R4* __restrict__ nd, int n, const R (&dx)[PT], const R (&dy)[PT],
                                      const R (&dz)[PT], R (&acc)[PT][4], const int (&bq)[PT], int band) {
#pragma unroll 4
    for (int i = 0; i < n; ++i) {
        const R4 o = nd[i];
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            const R rx = dx[q] - o.x, ry = dy[q] - o.y, rz = dz[q] - o.z;
            R r2 = fmad(rx, rx, fmad(ry, ry, rz * rz));
            R wq = o.w;
            if (MASKED) {
                wq = (bq[q] == band) ? wq : R(0);
                r2 = tiny_floor(r2);  // a masked-off point may sit on a node
            }
            const R inv = rsq(r2);
            const R a = wq * inv;  // q_i / r_i
            acc[q][0] += a;
            if (WANT_E) {
                const R b = a * inv * inv;  // q_i / r_i^3
                acc[q][1] = fmad(b, rx, acc[q][1]);
                acc[q][2] = fmad(b, ry, acc[q][2]);
                acc[q][3] = fmad(b, rz, acc[q][3]);
            }
        }
    }
}

// ------------------------------------------------------------ the kernel
// MODE 0: evaluation (sum over elements); MODE 1: assembly (one value per
// (point, element) pair written to A, potential only, sigma = 1).
// STATS: count pairs per (type, band) into counters[2 + 6 type + band].
template <bool F64, int PT, int TE, bool WANT_E, int MODE, bool STATS>
__global__ void __launch_bounds__(128) k_far(const FarK p) {
    constexpr int NT = 128;
    using R = typename std::conditional<F64, double, float>::type;
    using R4 = typename std::conditional<F64, double4, float4>::type;
    static_assert(TE == 16 || TE == 32, "one lane per element in the band test");

    extern __shared__ __align__(16) unsigned char smem_raw[];
    R4* s_node = reinterpret_cast<R4*>(smem_raw);                    // [TE][kSlots]
    R4* s_c = s_node + TE * kSlots;                                  // centroid (hi part for mixed), w = type
    R4* s_cl = s_c + TE;                                             // centroid lo part (mixed), w = L
    R4* s_e0 = s_cl + TE;                                            // e0, w = q (charge)
    R4* s_e1 = s_e0 + TE;                                            // e1
    R* s_thr = reinterpret_cast<R*>(s_e1 + TE);                      // [TE][5] (tau_k L)^2
    unsigned long long* s_stat = reinterpret_cast<unsigned long long*>(s_thr + TE * 5);  // 8-byte aligned
    double* s_acc64 = reinterpret_cast<double*>(s_stat + 16);  // [PT * 4][NT] FP64 sums of the mixed path

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wbase = blockIdx.x * (NT * PT) + warp * (32 * PT);
    const bool warp_live = wbase < p.n_pts;

    if (STATS) {
        if (tid < 12) s_stat[tid] = 0ull;
    }

    // ---- field points of this thread
    R px[PT], py[PT], pz[PT];            // FP64: the point; mixed: hi part
    float lx[PT], ly[PT], lz[PT];        // mixed: lo part
    int sidx[PT];
    bool valid[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        int i = wbase + q * 32 + lane;
        valid[q] = i < p.n_pts;
        if (!valid[q]) i = warp_live ? wbase : 0;  // duplicate a live point of the warp
        sidx[q] = i;
        const int src = p.perm[i];
        const double X = p.pts[3 * src], Y = p.pts[3 * src + 1], Z = p.pts[3 * src + 2];
        if constexpr (F64) {
            px[q] = (R)X; py[q] = (R)Y; pz[q] = (R)Z;
            lx[q] = ly[q] = lz[q] = 0.0f;
        } else {
            const float hx = (float)X, hy = (float)Y, hz = (float)Z;
            px[q] = hx; py[q] = hy; pz[q] = hz;
            lx[q] = (float)(X - (double)hx); ly[q] = (float)(Y - (double)hy); lz[q] = (float)(Z - (double)hz);
        }
    }

    // ---- bounding sphere of the warp's points (FP32, used only for the band test)
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

    // ---- accumulators
    R acc[PT][4];  // FP64 path: the sums; mixed path: FP32 sum of up to 8 element sums
    int ncnt[PT];
#pragma unroll
    for (int q = 0; q < PT; ++q) {
        ncnt[q] = 0;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            acc[q][c] = (R)0;
            if (!F64 && MODE == 0) s_acc64[(q * 4 + c) * NT + tid] = 0.0;
        }
    }
    const int dummy_b[PT] = {};

    const int el0 = blockIdx.y * p.el_chunk, el1 = min(p.n_el, el0 + p.el_chunk);
    for (int t0 = el0; t0 < el1; t0 += TE) {
        __syncthreads();
        // ---- stage element data of the tile
        if (tid < TE) {
            const int j = t0 + tid;
            if (j < el1) {
                const int ty = p.type[j];
                const double sg = p.sigma ? p.sigma[j] : 1.0;  // assembly: unit density
                const double area = p.geo[2 * j + 1];
                if constexpr (F64) {
                    const double L = p.geo[2 * j];
                    s_c[tid] = R4{(R)p.cen[3 * j], (R)p.cen[3 * j + 1], (R)p.cen[3 * j + 2], (R)ty};
                    s_cl[tid] = R4{0, 0, 0, (R)L};
                    s_e0[tid] = R4{(R)p.fr[6 * j], (R)p.fr[6 * j + 1], (R)p.fr[6 * j + 2], (R)(sg * area)};
                    s_e1[tid] = R4{(R)p.fr[6 * j + 3], (R)p.fr[6 * j + 4], (R)p.fr[6 * j + 5], (R)0};
#pragma unroll
                    for (int k = 0; k < 5; ++k) s_thr[tid * 5 + k] = (R)(p.tau2d[ty][k] * L * L);
                } else {
                    const float4 ch = p.chi[j], cl = p.clo[j], a = p.e0f[j], b = p.e1f[j];
                    s_c[tid] = R4{ch.x, ch.y, ch.z, ch.w};
                    s_cl[tid] = R4{cl.x, cl.y, cl.z, cl.w};
                    s_e0[tid] = R4{a.x, a.y, a.z, (float)(sg * area)};
                    s_e1[tid] = R4{b.x, b.y, b.z, 0.0f};
                    const float L = cl.w;
#pragma unroll
                    for (int k = 0; k < 5; ++k) s_thr[tid * 5 + k] = p.tau2f[ty][k] * L * L;
                }
            }
        }
        __syncthreads();
        // ---- expand all rule nodes of the tile: offset = alpha e0 + beta e1, weight w q
        for (int s = tid; s < TE * kSlots; s += NT) {
            const int e = s / kSlots, slot = s - e * kSlots;
            if (t0 + e >= el1) continue;
            const int ty = (int)s_c[e].w;
            if (slot >= c_nslot[ty]) continue;
            const R4 a = s_e0[e], b = s_e1[e];
            R al, be, w;
            if constexpr (F64) { al = c_alpha_d[ty][slot]; be = c_beta_d[ty][slot]; w = c_w_d[ty][slot]; }
            else { al = (R)c_alpha_f[ty][slot]; be = (R)c_beta_f[ty][slot]; w = (R)c_w_f[ty][slot]; }
            s_node[e * kSlots + slot] = R4{al * a.x + be * b.x, al * a.y + be * b.y, al * a.z + be * b.z, w * a.w};
        }
        __syncthreads();
        if (!warp_live) continue;

        // ---- conservative warp band test, one lane per element
        int code = kEndCode;
        {
            const int e = lane;
            if (e < TE && t0 + e < el1) {
                const R4 c = s_c[e], cl = s_cl[e];
                const float dx = ((float)(wcx - (float)c.x)) - (float)cl.x;
                const float dy = ((float)(wcy - (float)c.y)) - (float)cl.y;
                const float dz = ((float)(wcz - (float)c.z)) - (float)cl.z;
                const float Dc = sqrtf(dx * dx + dy * dy + dz * dz);
                const float cmag = fabsf((float)c.x) + fabsf((float)c.y) + fabsf((float)c.z);
                const float slack = 1e-5f * (Dc + wrad) + 1e-6f * (wmag + cmag);
                const float dmin = fmaxf(Dc - wrad - slack, 0.0f), dmax = Dc + wrad + slack;
                float th[5];
#pragma unroll
                for (int i = 0; i < 5; ++i) th[i] = (float)s_thr[e * 5 + i];
                const int blo = band_of<float>(dmin * dmin, th), bhi = band_of<float>(dmax * dmax, th);
                code = blo == bhi ? blo : kMixedCode;
            }
        }

        const int tend = min(TE, el1 - t0);
        for (int e = 0; e < tend; ++e) {
            const int cd = __shfl_sync(0xffffffffu, code, e);
            const R4 c = s_c[e], cl = s_cl[e];
            const int ty = (int)c.w;
            R dx[PT], dy[PT], dz[PT];
#pragma unroll
            for (int q = 0; q < PT; ++q) {
                if constexpr (F64) {
                    dx[q] = px[q] - c.x; dy[q] = py[q] - c.y; dz[q] = pz[q] - c.z;
                } else {
                    dx[q] = (px[q] - c.x) + (lx[q] - cl.x);
                    dy[q] = (py[q] - c.y) + (ly[q] - cl.y);
                    dz[q] = (pz[q] - c.z) + (lz[q] - cl.z);
                }
            }
            // per-element sums (assembly, mixed path) or the running sums (FP64 evaluation)
            R eacc[PT][4];
            constexpr bool kElemSum = MODE == 1 || !F64;
            if (kElemSum) {
#pragma unroll
                for (int q = 0; q < PT; ++q)
#pragma unroll
                    for (int k = 0; k < 4; ++k) eacc[q][k] = (R)0;
            }
            R(&dst)[PT][4] = kElemSum ? eacc : acc;
            const R4* nd0 = s_node + e * kSlots;

            if (cd >= 1 && cd <= 5) {
                const int r = band_rule(cd);
                nodes<R, R4, PT, WANT_E, false>(nd0 + c_rule_start[ty][r], c_rule_n[ty][r], dx, dy, dz, dst,
                                                dummy_b, 0);
                if (STATS && lane == 0) {
                    int nv = 0;
                    for (int q = 0; q < PT; ++q) nv += min(32, max(0, p.n_pts - (wbase + q * 32)));
                    atomicAdd(&s_stat[6 * ty + cd], (unsigned long long)nv);
                }
            } else {
                // per-point bands
                int bq[PT];
                const R* th = s_thr + e * 5;
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
                    append_near<PT>(p, want, sidx, t0 + e, ncnt, lane);
                }
#pragma unroll 1
                for (int band = 1; band <= 5; ++band) {
                    if (!(mask & (1u << band))) continue;
                    const int r = band_rule(band);
                    nodes<R, R4, PT, WANT_E, true>(nd0 + c_rule_start[ty][r], c_rule_n[ty][r], dx, dy, dz, dst,
                                                   bq, band);
                }
                if (STATS) {
#pragma unroll
                    for (int q = 0; q < PT; ++q) {
                        for (int band = 0; band <= 5; ++band) {
                            const unsigned m = __ballot_sync(0xffffffffu, valid[q] && bq[q] == band);
                            if (lane == 0 && m) atomicAdd(&s_stat[6 * ty + band], (unsigned long long)__popc(m));
                        }
                    }
                }
            }
            if (MODE == 0 && !F64) {
                // add the element sums; every 8 elements move the FP32 sum into FP64
#pragma unroll
                for (int q = 0; q < PT; ++q)
#pragma unroll
                    for (int c = 0; c < 4; ++c) acc[q][c] += eacc[q][c];
                if ((e & 7) == 7 || e == tend - 1) {
#pragma unroll
                    for (int q = 0; q < PT; ++q)
#pragma unroll
                        for (int c = 0; c < 4; ++c) {
                            s_acc64[(q * 4 + c) * NT + tid] += (double)acc[q][c];
                            acc[q][c] = (R)0;
                        }
                }
            }
            if (MODE == 1) {
                // assembly: one potential per pair, scaled by 1/(4 pi eps0); near pairs are filled later
                const int col = t0 + e;
#pragma unroll
                for (int q = 0; q < PT; ++q)
                    if (valid[q]) p.A[(size_t)p.perm[sidx[q]] * p.n_el + col] = p.kc * (double)eacc[q][0];
            }
        }
    }

    if (warp_live && MODE == 0) {
#pragma unroll
        for (int q = 0; q < PT; ++q) {
            if (!valid[q]) continue;
            double4 o;
            if constexpr (F64) o = make_double4(acc[q][0], acc[q][1], acc[q][2], acc[q][3]);
            else
                o = make_double4(s_acc64[(q * 4) * NT + tid], s_acc64[(q * 4 + 1) * NT + tid],
                                 s_acc64[(q * 4 + 2) * NT + tid], s_acc64[(q * 4 + 3) * NT + tid]);
            p.far[sidx[q]] = o;
            p.near_cnt[sidx[q]] = ncnt[q];
        }
    }
    if (STATS) {
        __syncthreads();
        if (tid < 12 && s_stat[tid]) atomicAdd(&p.counters[2 + tid], s_stat[tid]);
    }
}

// ------------------------------------------------------------ host side
namespace {
int uploaded_mask = 0;  // devices whose constant rule tables are loaded

int upload_rules(int dev) {
    if (dev < 32 && (uploaded_mask >> dev) & 1) return BEM_OK;
    const RuleSet& rs = rules();
    float af[2][kMaxSlots], bf[2][kMaxSlots], wf[2][kMaxSlots];
    for (int t = 0; t < 2; ++t)
        for (int s = 0; s < kMaxSlots; ++s) {
            af[t][s] = (float)rs.alpha[t][s];
            bf[t][s] = (float)rs.beta[t][s];
            wf[t][s] = (float)rs.w[t][s];
        }
    int nslot[2];
    for (int t = 0; t < 2; ++t) nslot[t] = rs.start[t][4] + rs.n[t][4];
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_alpha_f, af, sizeof af));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_beta_f, bf, sizeof bf));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_w_f, wf, sizeof wf));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_alpha_d, rs.alpha, sizeof rs.alpha));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_beta_d, rs.beta, sizeof rs.beta));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_w_d, rs.w, sizeof rs.w));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_nslot, nslot, sizeof nslot));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_rule_n, rs.n, sizeof rs.n));
    BEM_CUDA_TRY(cudaMemcpyToSymbol(c_rule_start, rs.start, sizeof rs.start));
    if (dev < 32) uploaded_mask |= 1 << dev;
    return BEM_OK;
}

template <bool F64, int PT, int TE>
constexpr size_t far_smem() {
    using R4 = typename std::conditional<F64, double4, float4>::type;
    using R = typename std::conditional<F64, double, float>::type;
    return sizeof(R4) * (TE * kSlots + 4 * TE) + sizeof(R) * (TE * 5) + 16 * sizeof(unsigned long long) +
           (F64 ? 0 : sizeof(double) * 4 * PT * 128);
}

template <bool F64, int PT, int TE, bool WANT_E, int MODE, bool STATS>
int launch_one(const FarK& k, cudaStream_t s) {
    constexpr size_t sm = far_smem<F64, PT, TE>();
    auto fn = k_far<F64, PT, TE, WANT_E, MODE, STATS>;
    static bool attr_set = false;  // per instantiation; the attribute is per function
    if (!attr_set) {
        BEM_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
        attr_set = true;
    }
    const int per_cta = 128 * PT;
    const int grid = (k.n_pts + per_cta - 1) / per_cta;
    if (grid == 0 || k.n_el == 0) return BEM_OK;
    FarK kk = k;
    int gy = 1;
    if (MODE == 1) {
        // assembly has no reduction over elements: split them so that the grid
        // holds at least four CTAs per SM
        gy = (152 * 4 + grid - 1) / grid;
        int chunk = (k.n_el + gy - 1) / gy;
        chunk = ((chunk + TE - 1) / TE) * TE;
        gy = (k.n_el + chunk - 1) / chunk;
        kk.el_chunk = chunk;
    } else {
        kk.el_chunk = k.n_el;
    }
    fn<<<dim3(grid, gy), 128, sm, s>>>(kk);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}

template <bool F64, int PT, int TE, bool WANT_E, int MODE>
int launch_stats(const FarK& k, cudaStream_t s, bool stats) {
    return stats ? launch_one<F64, PT, TE, WANT_E, MODE, true>(k, s) : launch_one<F64, PT, TE, WANT_E, MODE, false>(k, s);
}
}  // namespace

int launch_far(bem_mesh* m, const FarArgs& a, cudaStream_t s) {
    int rc = upload_rules(m->device);
    if (rc) return rc;
    FarK k;
    k.pts = a.pts;
    k.perm = a.perm;
    k.n_pts = a.n_pts;
    k.n_el = m->d.n;
    k.chi = m->d.chi; k.clo = m->d.clo; k.e0f = m->d.e0; k.e1f = m->d.e1;
    k.cen = m->d.cen; k.fr = m->d.fr; k.geo = m->d.geo;
    k.type = m->d.type;
    k.sigma = a.sigma;
    k.far = a.far;
    k.near_cnt = a.near_cnt;
    k.near_rec = a.near_rec;
    k.counters = a.counters;
    k.near_cap = a.near_cap;
    k.A = a.A;
    k.kc = a.kc;
    for (int t = 0; t < 2; ++t)
        for (int i = 0; i < 5; ++i) {
            k.tau2d[t][i] = m->limits[t][i] * m->limits[t][i];
            k.tau2f[t][i] = (float)k.tau2d[t][i];
        }
    const bool f64 = m->precision == kFP64;
    const bool st = a.stats != 0;
    if (a.A) {
        if (f64) return launch_stats<true, 2, 16, false, 1>(k, s, st);
        return launch_stats<false, 4, 32, false, 1>(k, s, st);
    }
    if (f64) {
        if (a.want_e) return launch_stats<true, 2, 16, true, 0>(k, s, st);
        return launch_stats<true, 2, 16, false, 0>(k, s, st);
    }
    if (a.want_e) return launch_stats<false, 4, 32, true, 0>(k, s, st);
    return launch_stats<false, 4, 32, false, 0>(k, s, st);
}

}  // namespace bem
