// k_prep.cu -- per-element preprocessing and validation (one thread per element).
//
// From the corners it derives what the method needs (Sec. 2, Eq. 3.2, Eq. 3.3):
//   triangle A, B, C:   Q_cen = (A + B + C) / 3, L = (|AB| + |BC| + |CA|) / 3,
//                       area = |AB x AC| / 2, frame e0 = A - Q_cen, e1 = B - Q_cen
//   rectangle P0..P3:   Q_cen = (P0 + P1 + P2 + P3) / 4, a = |P1 - P0|, b = |P3 - P0|,
//                       L = (a + b) / 2, area = a b, e0 = (P1 - P0) / 2 = (a/2) u_x,
//                       e1 = (P3 - P0) / 2 = (b/2) u_y
// and writes the FP64 arrays (centroid, frame, L, area) plus the FP32
// records of the mixed path.  The centroid is split as C = C_hi + C_lo with
// C_hi a multiple of a power-of-two grid g = 2^(e - 12), 2^e >= the largest
// corner coordinate; the far-field kernel splits field points on the same
// grid, so P_hi - C_hi is exact in FP32 and d = (P_hi - C_hi) + (P_lo - C_lo)
// takes a single rounding.  (Rounding both to the nearest float instead
// would round every P - C of a point on one common grid, a shift of the
// point that is the same for all elements and is not averaged away.)
#include <string.h>

#include "bem_internal.cuh"

namespace bem {

namespace {

struct V3 {
    double x, y, z;
};
__device__ __forceinline__ V3 ld3(const double* p) { return V3{p[0], p[1], p[2]}; }
__device__ __forceinline__ V3 operator-(V3 a, V3 b) { return V3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ V3 operator+(V3 a, V3 b) { return V3{a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ __forceinline__ V3 operator*(double s, V3 a) { return V3{s * a.x, s * a.y, s * a.z}; }
__device__ __forceinline__ double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ V3 cross(V3 a, V3 b) {
    return V3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ double len(V3 a) { return sqrt(dot(a, a)); }

// error codes written with the element index
enum { kBadType = 1, kNotFinite = 2, kDegenerate = 3, kNotRectangle = 4 };

__global__ void k_prep(int n, const int* __restrict__ type, const double* __restrict__ verts,
                       const double* __restrict__ sigma, MeshDev d, unsigned long long* bad, unsigned* cmax) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    {
        // largest |coordinate| (float bits of a non-negative float order like unsigned ints)
        float m = 0.0f;
        for (int k = 0; k < 12; ++k) m = fmaxf(m, (float)fabs(verts[12 * (size_t)j + k]));
        if (isfinite(m)) atomicMax(cmax, __float_as_uint(m));
    }
    const int ty = type[j];
    const double* v = verts + 12 * (size_t)j;
    int code = 0;
    if (ty != BEM_TRIANGLE && ty != BEM_RECTANGLE) code = kBadType;
    const int nv = ty == BEM_RECTANGLE ? 4 : 3;
    for (int k = 0; k < 3 * nv && !code; ++k)
        if (!isfinite(v[k])) code = kNotFinite;
    if (!code && !isfinite(sigma[j])) code = kNotFinite;

    V3 cen = {0, 0, 0}, e0 = {0, 0, 0}, e1 = {0, 0, 0};
    double L = 0.0, area = 0.0;
    if (!code && ty == BEM_TRIANGLE) {
        const V3 A = ld3(v), B = ld3(v + 3), C = ld3(v + 6);
        const V3 ab = B - A, ac = C - A, bc = C - B;
        const double lab = len(ab), lac = len(ac), lbc = len(bc);
        area = 0.5 * len(cross(ab, ac));
        const double smax = fmax(lab, fmax(lac, lbc));
        if (!(area > 1e-14 * smax * smax)) code = kDegenerate;
        cen = (1.0 / 3.0) * (A + B + C);
        L = (lab + lbc + lac) / 3.0;
        e0 = A - cen;
        e1 = B - cen;
    } else if (!code) {
        const V3 P0 = ld3(v), P1 = ld3(v + 3), P2 = ld3(v + 6), P3 = ld3(v + 9);
        const V3 s1 = P1 - P0, s3 = P3 - P0;
        const double a = len(s1), b = len(s3);
        if (!(a > 0.0 && b > 0.0)) code = kDegenerate;
        else {
            const double gap = len(P2 - (P1 + s3));
            if (gap > 1e-9 * fmax(a, b) || fabs(dot(s1, s3)) > 1e-9 * a * b) code = kNotRectangle;
        }
        cen = 0.25 * (P0 + P1 + P2 + P3);
        L = 0.5 * (a + b);
        area = a * b;
        e0 = 0.5 * s1;
        e1 = 0.5 * s3;
    }
    if (code) {
        atomicMin(bad, ((unsigned long long)j << 8) | (unsigned long long)code);
        return;
    }
    d.type[j] = ty;
    d.sigma[j] = sigma[j];
    for (int k = 0; k < 12; ++k) d.verts[12 * (size_t)j + k] = k < 3 * nv ? v[k] : 0.0;
    {
        // near-field geometry: the unit normal, per edge the unit tangent and the in-plane outward
        // normal, the mean side
        double* g = d.egeo + (size_t)kEgeo * j;
        const V3 c0 = ld3(v), c1 = ld3(v + 3), c2 = ld3(v + 6);
        V3 nrm = cross(c1 - c0, c2 - c0);
        nrm = (1.0 / len(nrm)) * nrm;
        g[0] = nrm.x; g[1] = nrm.y; g[2] = nrm.z;
        double perim = 0.0;
        for (int k = 0; k < 4; ++k) {
            V3 t = {0, 0, 0}, m = {0, 0, 0};
            if (k < nv) {
                t = ld3(v + 3 * ((k + 1) % nv)) - ld3(v + 3 * k);
                const double l = len(t);
                perim += l;
                t = (1.0 / l) * t;
                m = cross(t, nrm);
            }
            g[3 + 6 * k] = t.x; g[4 + 6 * k] = t.y; g[5 + 6 * k] = t.z;
            g[6 + 6 * k] = m.x; g[7 + 6 * k] = m.y; g[8 + 6 * k] = m.z;
        }
        g[27] = perim / nv;
    }
    d.cen[3 * j] = cen.x; d.cen[3 * j + 1] = cen.y; d.cen[3 * j + 2] = cen.z;
    d.fr[6 * j] = e0.x; d.fr[6 * j + 1] = e0.y; d.fr[6 * j + 2] = e0.z;
    d.fr[6 * j + 3] = e1.x; d.fr[6 * j + 4] = e1.y; d.fr[6 * j + 5] = e1.z;
    d.geo[2 * j] = L;
    d.geo[2 * j + 1] = area;
    // xyz of chi / clo: written by k_split once the grid is known
    d.chi[j] = make_float4(0.0f, 0.0f, 0.0f, __int_as_float(ty));  // w: type as int bits
    d.clo[j] = make_float4(0.0f, 0.0f, 0.0f, (float)L);
    d.e0[j] = make_float4((float)e0.x, (float)e0.y, (float)e0.z, (float)area);
    d.e1[j] = make_float4((float)e1.x, (float)e1.y, (float)e1.z, 0.0f);
}

// Centroid hi / lo parts on the grid g (a power of two, so c / g and the
// products are exact): hi = rint(c / g) g, lo = c - hi.
__global__ void k_split(int n, const double* __restrict__ cen, double g, double inv_g, float4* chi, float4* clo) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double h[3];
    float lo[3];
    for (int k = 0; k < 3; ++k) {
        const double c = cen[3 * j + k];
        h[k] = rint(c * inv_g) * g;
        lo[k] = (float)(c - h[k]);
    }
    const float4 a = chi[j], b = clo[j];
    chi[j] = make_float4((float)h[0], (float)h[1], (float)h[2], a.w);
    clo[j] = make_float4(lo[0], lo[1], lo[2], b.w);
}

const char* code_name(int c) {
    switch (c) {
        case kBadType: return "element type is neither triangle (0) nor rectangle (1)";
        case kNotFinite: return "non-finite corner coordinate or charge density";
        case kDegenerate: return "degenerate element (zero area or zero side)";
        case kNotRectangle: return "corners do not form a rectangle (P2 != P1 + P3 - P0 or sides not orthogonal)";
        default: return "invalid element";
    }
}

}  // namespace

// types/verts/sigma are device arrays (staged by the caller).
int launch_prep(bem_mesh* m, const int* types, const double* verts, const double* sigma, cudaStream_t s,
                int64_t* bad_index, int* bad_code, double* coord_max) {
    unsigned long long* dbad = m->w.counters + 1;
    unsigned* dmax = reinterpret_cast<unsigned*>(m->w.counters + 2);
    const unsigned long long init[2] = {~0ull, 0ull};
    BEM_CUDA_TRY(cudaMemcpyAsync(dbad, init, sizeof init, cudaMemcpyHostToDevice, s));
    const int n = m->d.n;
    k_prep<<<(n + 255) / 256, 256, 0, s>>>(n, types, verts, sigma, m->d, dbad, dmax);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    unsigned long long hbad = 0;
    unsigned hmax = 0;
    BEM_CUDA_TRY(cudaMemcpyAsync(&hbad, dbad, sizeof hbad, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaMemcpyAsync(&hmax, dmax, sizeof hmax, cudaMemcpyDeviceToHost, s));
    BEM_CUDA_TRY(cudaStreamSynchronize(s));
    float fm;
    memcpy(&fm, &hmax, sizeof fm);
    *coord_max = fm;
    if (hbad != ~0ull) {
        *bad_index = (int64_t)(hbad >> 8);
        *bad_code = (int)(hbad & 0xff);
        set_error("bem_create: element %lld: %s", (long long)*bad_index, code_name(*bad_code));
        return BEM_ERR_INVALID;
    }
    *bad_index = -1;
    *bad_code = 0;
    int e = 0;
    if (fm > 0.0f) frexp((double)fm, &e);  // 2^e > the largest coordinate
    m->grid = ldexp(1.0, e - 12);
    k_split<<<(n + 255) / 256, 256, 0, s>>>(n, m->d.cen, m->grid, 1.0 / m->grid, m->d.chi, m->d.clo);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}

}  // namespace bem
