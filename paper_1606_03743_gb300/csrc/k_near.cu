// k_near.cu -- analytic near field (FP64) over the compacted near-pair list,
// and the per-point finalisation.
//
// Below the near limit (by default DR < 4.5 for triangles and 6 for
// rectangles, Sec. 4) the element is integrated analytically; the paper
// cites the formulas without printing them.  For a
// uniformly charged planar polygon with unit normal n (corners counter-
// clockwise about n) and field point P at signed height h = (P - V)·n:
//   int dA / R         = sum_e d_e l_e - h Omega
//   int (P - Q)/R^3 dA = sum_e m_e l_e + n Omega
// where for edge e: t_e its unit direction, m_e = t_e x n the outward
// in-plane normal, d_e = (V1 - P)·m_e, l_e = int_e ds / R = ln((s2 + R2) /
// (s1 + R1)) with s_k = (V_k - P)·t_e, R_k = |V_k - P|, and Omega the solid
// angle of the polygon seen from P with the sign of h (Van Oosterom and
// Strackee's formula on each triangle).  The edge logarithm is evaluated in
// whichever of its three equivalent forms has no cancellation.
#include <algorithm>
#include <climits>

#include "bem_internal.cuh"

namespace bem {

namespace {

struct D3 {
    double x, y, z;
};
__device__ __forceinline__ D3 sub(D3 a, D3 b) { return D3{a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ __forceinline__ double dot(D3 a, D3 b) { return fma(a.x, b.x, fma(a.y, b.y, a.z * b.z)); }
__device__ __forceinline__ D3 cross(D3 a, D3 b) {
    return D3{a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
}
__device__ __forceinline__ D3 scale(D3 a, double s) { return D3{a.x * s, a.y * s, a.z * s}; }

// Van Oosterom and Strackee: the solid angle of triangle (a, b, c) is
// -2 atan2(y, x) with y = a.(b x c) and x = |a||b||c| + (a.b)|c| + (a.c)|b| + (b.c)|a|.
__device__ __forceinline__ void solid_angle_args(D3 a, D3 b, D3 c, double la, double lb, double lc, double& y,
                                                 double& x) {
    y = dot(a, cross(b, c));  // = -2 area h
    x = la * lb * lc + dot(a, b) * lc + dot(a, c) * lb + dot(b, c) * la;
}

// Signed solid angle of triangle (a, b, c) (relative positions from P, at
// distances la, lb, lc), with the sign of h for a triangle counter-clockwise
// about the normal.
__device__ double solid_angle(D3 a, D3 b, D3 c, double la, double lb, double lc) {
    double y, x;
    solid_angle_args(a, b, c, la, lb, lc, y, x);
    return -2.0 * atan2(y, x);
}

// phi and E (unit sigma, without 1/(4 pi eps0)) of element with corners V
// (3 for a triangle, 4 for a rectangle) at P; G: the element's normal, edge
// tangents and outward normals and mean side (kEgeo doubles, from bem_create).
__device__ void polygon_field(int nv, const double* __restrict__ V, const double* __restrict__ G, D3 P,
                              double out[4]) {
    D3 c[4];
    for (int k = 0; k < nv; ++k) c[k] = sub(D3{V[3 * k], V[3 * k + 1], V[3 * k + 2]}, P);  // corners relative to P
    const D3 nrm{G[0], G[1], G[2]};
    const double h = -dot(c[0], nrm);  // (P - V0)·n
    double phi = 0.0, ex = 0.0, ey = 0.0, ez = 0.0;
    double r[4];
    for (int k = 0; k < nv; ++k) r[k] = sqrt(dot(c[k], c[k]));
    for (int k = 0; k < nv; ++k) {
        const int k2 = (k + 1 == nv) ? 0 : k + 1;
        const D3 t{G[3 + 6 * k], G[4 + 6 * k], G[5 + 6 * k]}, m{G[6 + 6 * k], G[7 + 6 * k], G[8 + 6 * k]};
        const double s1 = dot(c[k], t), s2 = dot(c[k2], t);
        const double d = dot(c[k], m);
        double num, den;
        if (s1 >= 0.0) {
            num = r[k2] + s2;
            den = r[k] + s1;
        } else if (s2 <= 0.0) {
            num = r[k] - s1;
            den = r[k2] - s2;
        } else {  // the foot of the perpendicular lies inside the edge
            num = (r[k2] + s2) * (r[k] - s1);
            den = fma(d, d, h * h);
        }
        // a point on the closed edge: the edge adds d l -> 0 to the potential
        // and its (log-singular) in-plane field is left out
        const double l = den == 0.0 ? 0.0 : log(num / den);
        phi = fma(d, l, phi);
        ex = fma(m.x, l, ex);
        ey = fma(m.y, l, ey);
        ez = fma(m.z, l, ez);
    }
    // in the element plane to 1e-12 of the mean side (a point computed to lie on the element,
    // such as its centroid, counts as on it whatever the rounding of h): h Omega = 0, and on the
    // element the mean of both sides of the normal-field jump (0)
    double om = 0.0;
    if (fabs(h) > 1e-12 * G[27]) {
        if (nv == 3) om = solid_angle(c[0], c[1], c[2], r[0], r[1], r[2]);
        else {
            // the rectangle's two triangles: their half-angles add up as the arguments of the
            // complex numbers (x1 + i y1)(x2 + i y2); one atan2 does while the sum stays within
            // +-pi/2 (real part positive), away from atan2's branch cut
            double y1, x1, y2, x2;
            solid_angle_args(c[0], c[1], c[3], r[0], r[1], r[3], y1, x1);
            solid_angle_args(c[1], c[2], c[3], r[1], r[2], r[3], y2, x2);
            const double xr = fma(x1, x2, -y1 * y2), yr = fma(y1, x2, y2 * x1);
            om = xr > 0.0 ? -2.0 * atan2(yr, xr) : -2.0 * (atan2(y1, x1) + atan2(y2, x2));
        }
    }
    out[0] = phi - h * om;
    out[1] = fma(nrm.x, om, ex);
    out[2] = fma(nrm.y, om, ey);
    out[3] = fma(nrm.z, om, ez);
}

// Field of an edge V1 -> V2 as a unit line charge at P: J = int (P - Q)/R^3 ds
// = -rho (u2/R2 - u1/R1) / |rho|^2 + t (1/R2 - 1/R1), with t the unit tangent,
// u_k = (V_k - P)·t, rho = (V1 - P) - u1 t; the differences are rewritten as
// quotients without cancellation.  A point on the closed edge gives 0.
// (corners c1, c2 relative to P at distances R1, R2; t the edge's unit tangent)
__device__ D3 edge_line_field(D3 c1, D3 c2, D3 t, double R1, double R2) {
    const double u1 = dot(c1, t), u2 = dot(c2, t);
    const D3 rho = sub(c1, scale(t, u1));
    const double rho2 = dot(rho, rho);
    if (R1 == 0.0 || R2 == 0.0) return D3{0.0, 0.0, 0.0};
    double f;
    if (u1 >= 0.0) f = (u2 - u1) * (u2 + u1) / (R1 * R2 * (u2 * R1 + u1 * R2));
    else if (u2 <= 0.0) f = (u1 - u2) * (u1 + u2) / (R1 * R2 * (-u1 * R2 - u2 * R1));
    else if (rho2 > 0.0) f = (u2 / R2 - u1 / R1) / rho2;
    else return D3{0.0, 0.0, 0.0};
    const double g = (u1 - u2) * (u1 + u2) / (R1 * R2 * (R1 + R2));  // 1/R2 - 1/R1
    return D3{fma(-rho.x, f, t.x * g), fma(-rho.y, f, t.y * g), fma(-rho.z, f, t.z * g)};
}

// Field gradient dE_i/dx_j (xx, yy, zz, xy, xz, yz; unit sigma, without
// 1/(4 pi eps0)) of the polygon at P, from the decomposition above: the
// gradient of l_e is -J_e and that of Omega is -sum_e t_e x J_e, so
//   dE/dx = -sum_e m_e J_e^T - n (sum_e t_e x J_e)^T.
// Eg: the element's normal, edge tangents and outward normals (kEgeo doubles, from bem_create).
__device__ void polygon_grad(int nv, const double* __restrict__ V, const double* __restrict__ Eg, D3 P,
                             double out[6]) {
    D3 c[4];
    double r[4];
    for (int k = 0; k < nv; ++k) {
        c[k] = sub(D3{V[3 * k], V[3 * k + 1], V[3 * k + 2]}, P);
        r[k] = sqrt(dot(c[k], c[k]));
    }
    const D3 nrm{Eg[0], Eg[1], Eg[2]};
    double G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}};
    D3 w{0.0, 0.0, 0.0};
    for (int k = 0; k < nv; ++k) {
        const int k2 = (k + 1 == nv) ? 0 : k + 1;
        const D3 t{Eg[3 + 6 * k], Eg[4 + 6 * k], Eg[5 + 6 * k]}, m{Eg[6 + 6 * k], Eg[7 + 6 * k], Eg[8 + 6 * k]};
        const D3 J = edge_line_field(c[k], c[k2], t, r[k], r[k2]);
        const double mv[3] = {m.x, m.y, m.z}, Jv[3] = {J.x, J.y, J.z};
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a][b] = fma(-mv[a], Jv[b], G[a][b]);
        const D3 tj = cross(t, J);
        w = D3{w.x + tj.x, w.y + tj.y, w.z + tj.z};
    }
    const double nv3[3] = {nrm.x, nrm.y, nrm.z}, wv[3] = {w.x, w.y, w.z};
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) G[a][b] = fma(-nv3[a], wv[b], G[a][b]);
    out[0] = G[0][0];
    out[1] = G[1][1];
    out[2] = G[2][2];
    out[3] = G[0][1];
    out[4] = G[0][2];
    out[5] = G[1][2];
}

// Slot, among all near values, of the first pair of near-pair run r =
// (sorted point, first element, ordinal of its first pair in its chunk, pairs):
// the point's first slot, plus its near pairs in the chunks before the run's
// chunk (the element's chunk), plus the ordinal -- so a point's values sit in
// element order.  The run's other pairs follow in the next slots.
__device__ __forceinline__ unsigned long long near_slot(const int4 r, const int* __restrict__ near_off,
                                                        const int* __restrict__ near_row,
                                                        const int* __restrict__ near_rows, int n_chunks,
                                                        int chunk_len) {
    const int chunk = r.y / chunk_len;
    return (unsigned long long)near_off[r.x] + (unsigned long long)near_rows[(size_t)near_row[r.x] * n_chunks + chunk] +
           (unsigned long long)r.z;
}

// What the checked build checks near-pair runs against: the point capacity,
// the element count, and the counters that take the flag.
struct NearBounds {
    int n_pts, n_el;
    unsigned long long* counters;
};

// The near-pair passes run with blocks of kNearThreads threads.
constexpr int kNearThreads = 128;
constexpr int kNearWarps = kNearThreads / 32;

// Calls f(run, k, P, slot) for pair k of every near-pair run: each warp takes
// 32 runs at a time, lays their pairs end to end (a warp prefix sum of the run
// lengths) and deals them out to its lanes, so that a long run does not leave
// the warp's other lanes idle.  P is the run's field point; slot its pair's
// slot among the near values (slot_of(run) + k), or the run's index when
// slot_of is null (assembly writes no values).
//
// A run whose point or elements fall outside [0, n_pts) x [0, n_el) is a
// corrupt record: the checked build skips it and flags kCheckElement.
template <typename SlotOf, typename F>
__device__ __forceinline__ void for_each_near_pair(const int4* __restrict__ rec, unsigned long long n_runs,
                                                   const double* __restrict__ pts, const int* __restrict__ perm,
                                                   const NearBounds nb, SlotOf slot_of, F f) {
    __shared__ int4 s_rec[kNearWarps][32];
    __shared__ int s_first[kNearWarps][32];
    __shared__ unsigned long long s_slot[kNearWarps][32];
    __shared__ double s_P[kNearWarps][32][3];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned long long stride = (unsigned long long)gridDim.x * kNearWarps * 32;
    for (unsigned long long b = ((unsigned long long)blockIdx.x * kNearWarps + warp) * 32; b < n_runs; b += stride) {
        const unsigned long long i = b + lane;
        int4 r = i < n_runs ? rec[i] : make_int4(0, 0, 0, 0);
        if (!check_ok(r.w == 0 || (r.x >= 0 && r.x < nb.n_pts && r.y >= 0 && r.w > 0 && r.y + r.w <= nb.n_el),
                      nb.counters, kCheckElement))
            r.w = 0;
        int incl = r.w;  // inclusive prefix sum of the run lengths over the lanes
        for (int o = 1; o < 32; o <<= 1) {
            const int t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += t;
        }
        const int total = __shfl_sync(0xffffffffu, incl, 31);
        s_rec[warp][lane] = r;
        s_first[warp][lane] = incl - r.w;
        if (r.w > 0) {
            const int src = perm[r.x];
            s_P[warp][lane][0] = pts[3 * (size_t)src];
            s_P[warp][lane][1] = pts[3 * (size_t)src + 1];
            s_P[warp][lane][2] = pts[3 * (size_t)src + 2];
            s_slot[warp][lane] = slot_of(r);
        }
        __syncwarp();
        for (int j = lane; j < total; j += 32) {
            int lo = 0, hi = 31;  // the last run whose first pair is at or before j (lengths are >= 1)
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_first[warp][mid] <= j) lo = mid;
                else hi = mid - 1;
            }
            const int k = j - s_first[warp][lo];
            const D3 P{s_P[warp][lo][0], s_P[warp][lo][1], s_P[warp][lo][2]};
            f(s_rec[warp][lo], k, P, s_slot[warp][lo] + (unsigned long long)k);
        }
        __syncwarp();
    }
}

// far gradient sums (the chunks already summed in chunk order) + near pairs in
// element order, times 1/(4 pi eps0), written at the point's original position.
__global__ void k_finalize_grad(int n, const int* __restrict__ perm, const double4* __restrict__ far_g,
                                const int* __restrict__ near_tot, const int* __restrict__ near_off,
                                const double4* __restrict__ gval, unsigned long long gcap, double kc,
                                double* __restrict__ G) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double4 a0 = far_g[2 * (size_t)i], b0 = far_g[2 * (size_t)i + 1];
    double s[6] = {a0.x, a0.y, a0.z, a0.w, b0.x, b0.y};
    const int cnt = near_tot[i];
    const unsigned long long off = (unsigned long long)near_off[i];
    for (int k = 0; k < cnt; ++k) {
        if (off + k >= gcap) break;
        const double4 a = gval[2 * (off + k)], b = gval[2 * (off + k) + 1];
        s[0] += a.x; s[1] += a.y; s[2] += a.z; s[3] += a.w; s[4] += b.x; s[5] += b.y;
    }
    const int o = perm[i];
    for (int k = 0; k < 6; ++k) G[6 * (size_t)o + k] = kc * s[k];
}

// phi and E (without 1/(4 pi eps0)) of the polygon with the linear density
// sigma(Q) = sc + g.(Q - C) (g in the element plane).  With P' the foot of P
// in the plane (P = P' + h n), w = Q - P' and the constant-density results
// I0 = int dA / R, E0 (polygon_field):
//   phi = sigma(P') I0 + g . sum_e m_e (s2 R2 - s1 R1 + rho_e^2 l_e) / 2
//   E   = sigma(P') E0 - g I0 - h n sum_e (g.m_e) l_e
//         + sum_e (g.m_e) (d_e l_e m_e + (R2 - R1) t_e)
// (the in-plane divergence theorem on grad R = w / R, grad (1/R) = -w / R^3
// and on w / R; rho_e^2 = d_e^2 + h^2 is the squared distance of P from the
// edge line).
__device__ void polygon_field_lin(int nv, const double* __restrict__ V, const double* __restrict__ G, D3 P, double sc, D3 g,
                                  D3 C, double out[4]) {
    double f0[4];
    polygon_field(nv, V, G, P, f0);
    D3 c[4];
    for (int k = 0; k < nv; ++k) c[k] = sub(D3{V[3 * k], V[3 * k + 1], V[3 * k + 2]}, P);
    D3 nrm = cross(sub(c[1], c[0]), sub(c[2], c[0]));
    nrm = scale(nrm, 1.0 / sqrt(dot(nrm, nrm)));
    const double h = -dot(c[0], nrm);
    const D3 Pp = sub(P, scale(nrm, h));
    const double sP = sc + dot(g, sub(Pp, C));
    double r[4];
    for (int k = 0; k < nv; ++k) r[k] = sqrt(dot(c[k], c[k]));
    double i1 = 0.0, hsum = 0.0;
    D3 ec = scale(g, -f0[0]);
    for (int k = 0; k < nv; ++k) {
        const int k2 = (k + 1 == nv) ? 0 : k + 1;
        D3 t = sub(c[k2], c[k]);
        t = scale(t, 1.0 / sqrt(dot(t, t)));
        const D3 m = cross(t, nrm);
        const double s1 = dot(c[k], t), s2 = dot(c[k2], t);
        const double d = dot(c[k], m);
        double num, den;
        if (s1 >= 0.0) {
            num = r[k2] + s2;
            den = r[k] + s1;
        } else if (s2 <= 0.0) {
            num = r[k] - s1;
            den = r[k2] - s2;
        } else {
            num = (r[k2] + s2) * (r[k] - s1);
            den = fma(d, d, h * h);
        }
        const double l = den == 0.0 ? 0.0 : log(num / den);
        const double gm = dot(g, m);
        i1 = fma(gm, 0.5 * (s2 * r[k2] - s1 * r[k] + fma(d, d, h * h) * l), i1);
        hsum = fma(gm, l, hsum);
        const double a = gm * d * l, b = gm * (r[k2] - r[k]);
        ec = D3{ec.x + a * m.x + b * t.x, ec.y + a * m.y + b * t.y, ec.z + a * m.z + b * t.z};
    }
    out[0] = fma(sP, f0[0], i1);
    out[1] = fma(sP, f0[1], fma(-h * nrm.x, hsum, ec.x));
    out[2] = fma(sP, f0[2], fma(-h * nrm.y, hsum, ec.y));
    out[3] = fma(sP, f0[3], fma(-h * nrm.z, hsum, ec.z));
}

// x^T H y for the symmetric H stored as (xx, yy, zz, xy, xz, yz)
__device__ __forceinline__ double hform(const double* H, D3 x, D3 y) {
    return x.x * (H[0] * y.x + H[3] * y.y + H[4] * y.z) + x.y * (H[3] * y.x + H[1] * y.y + H[5] * y.z) +
           x.z * (H[4] * y.x + H[5] * y.y + H[2] * y.z);
}
__device__ __forceinline__ D3 hmul(const double* H, D3 x) {
    return D3{H[0] * x.x + H[3] * x.y + H[4] * x.z, H[3] * x.x + H[1] * x.y + H[5] * x.z,
              H[4] * x.x + H[5] * x.y + H[2] * x.z};
}

// phi and E (without 1/(4 pi eps0)) of the polygon with the quadratic density
// sigma(Q) = sc + g.(Q - C) + (Q - C)^T H (Q - C) / 2 (g and H in the element
// plane).  About the foot P' of P (w = Q - P'): sigma = sP + gP.w + w^T H w / 2
// with gP = g + H (P' - C).  Beyond the linear terms, per edge e (J_e =
// int_e R ds = (s2 R2 - s1 R1 + rho_e^2 l_e) / 2):
//   H : int w w^T / R dA   = sum_e (d_e J_e m^T H m + (R2^3 - R1^3)/3 t^T H m) - tr(H) int R dA,
//                            int R dA = (sum_e d_e J_e + h^2 I0) / 3
//   H : int w w^T / R^3 dA = tr(H) I0 - sum_e (d_e l_e m^T H m + (R2 - R1) t^T H m)
//   int (w^T H w) w / R^3 dA = 2 H int w / R dA - sum_e m_e q_e,
//   q_e = int_e w^T H w / R ds = d_e^2 m^T H m l_e + 2 d_e m^T H t (R2 - R1)
//         + t^T H t (s2 R2 - s1 R1 - rho_e^2 l_e) / 2
// (the in-plane divergence theorem on w R, w w^T / R and (w^T H w) / R, with
// w = d_e m_e + s t_e on the edge); then
//   phi = sP I0 + gP . int w / R dA + (H : int w w^T / R dA) / 2
//   E   = sP E0 + [linear terms with gP] + [h n (H : int w w^T / R^3 dA) - int (w^T H w) w / R^3 dA] / 2.
__device__ void polygon_field_quad(int nv, const double* __restrict__ V, const double* __restrict__ G, D3 P, double sc, D3 g,
                                   const double* H, D3 C,
                                   double out[4]) {
    double f0[4];
    polygon_field(nv, V, G, P, f0);
    D3 c[4];
    for (int k = 0; k < nv; ++k) c[k] = sub(D3{V[3 * k], V[3 * k + 1], V[3 * k + 2]}, P);
    D3 nrm = cross(sub(c[1], c[0]), sub(c[2], c[0]));
    nrm = scale(nrm, 1.0 / sqrt(dot(nrm, nrm)));
    const double h = -dot(c[0], nrm);
    const D3 dl = sub(sub(P, scale(nrm, h)), C);
    const D3 Hd = hmul(H, dl);
    const double sP = sc + dot(g, dl) + 0.5 * dot(dl, Hd);
    const D3 gP{g.x + Hd.x, g.y + Hd.y, g.z + Hd.z};
    const double trH = H[0] + H[1] + H[2];
    double r[4];
    for (int k = 0; k < nv; ++k) r[k] = sqrt(dot(c[k], c[k]));
    D3 i1{0.0, 0.0, 0.0}, ec = scale(gP, -f0[0]), qm{0.0, 0.0, 0.0};
    double hsum = 0.0, sdj = 0.0, hi2 = 0.0, hk2 = trH * f0[0];
    for (int k = 0; k < nv; ++k) {
        const int k2 = (k + 1 == nv) ? 0 : k + 1;
        D3 t = sub(c[k2], c[k]);
        t = scale(t, 1.0 / sqrt(dot(t, t)));
        const D3 m = cross(t, nrm);
        const double s1 = dot(c[k], t), s2 = dot(c[k2], t);
        const double d = dot(c[k], m);
        const double rho2 = fma(d, d, h * h);
        double num, den;
        if (s1 >= 0.0) {
            num = r[k2] + s2;
            den = r[k] + s1;
        } else if (s2 <= 0.0) {
            num = r[k] - s1;
            den = r[k2] - s2;
        } else {
            num = (r[k2] + s2) * (r[k] - s1);
            den = rho2;
        }
        const double l = den == 0.0 ? 0.0 : log(num / den);
        const double sr = s2 * r[k2] - s1 * r[k];
        const double J = 0.5 * fma(rho2, l, sr);
        const double dR = r[k2] - r[k];
        const double cub = (r[k2] * r[k2] * r[k2] - r[k] * r[k] * r[k]) / 3.0;
        const double mHm = hform(H, m, m), tHm = hform(H, t, m), tHt = hform(H, t, t);
        i1 = D3{fma(m.x, J, i1.x), fma(m.y, J, i1.y), fma(m.z, J, i1.z)};
        sdj = fma(d, J, sdj);
        hi2 += d * J * mHm + cub * tHm;
        hk2 -= d * l * mHm + dR * tHm;
        const double q = d * d * mHm * l + 2.0 * d * tHm * dR + 0.5 * tHt * fma(-rho2, l, sr);
        qm = D3{fma(m.x, q, qm.x), fma(m.y, q, qm.y), fma(m.z, q, qm.z)};
        const double gm = dot(gP, m);
        hsum = fma(gm, l, hsum);
        const double a = gm * d * l, b = gm * dR;
        ec = D3{ec.x + a * m.x + b * t.x, ec.y + a * m.y + b * t.y, ec.z + a * m.z + b * t.z};
    }
    hi2 -= trH * (sdj + h * h * f0[0]) / 3.0;
    const D3 Hi1 = hmul(H, i1);
    // (h n hk2 - (2 H I1 - qm)) / 2
    const D3 qt{0.5 * (h * nrm.x * hk2 + qm.x) - Hi1.x, 0.5 * (h * nrm.y * hk2 + qm.y) - Hi1.y,
                0.5 * (h * nrm.z * hk2 + qm.z) - Hi1.z};
    out[0] = fma(sP, f0[0], dot(gP, i1) + 0.5 * hi2);
    out[1] = fma(sP, f0[1], fma(-h * nrm.x, hsum, ec.x) + qt.x);
    out[2] = fma(sP, f0[2], fma(-h * nrm.y, hsum, ec.y) + qt.y);
    out[3] = fma(sP, f0[3], fma(-h * nrm.z, hsum, ec.z) + qt.z);
}

// The density of element j in space: sigma(Q) = sc + g.(Q - C) + (Q - C)^T H (Q - C) / 2
// from its frame coefficients: g = s_a grad(alpha) + s_b grad(beta) and H = 2 c3 d0 d0^T +
// c4 (d0 d1^T + d1 d0^T) + 2 c5 d1 d1^T, with d0 = grad(alpha), d1 = grad(beta) the in-plane
// duals of the frame vectors e0, e1 (H = 0 for a linear density).
struct Density {
    double sc;
    D3 g, C;
    double H[6];  // xx, yy, zz, xy, xz, yz
};
__device__ void element_density(int j, double sc, const double* __restrict__ slope, const double* __restrict__ curv,
                                const double* __restrict__ fr, const double* __restrict__ cen, Density& dn) {
    const double* F = fr + 6 * (size_t)j;
    const D3 e0{F[0], F[1], F[2]}, e1{F[3], F[4], F[5]};
    const double g00 = dot(e0, e0), g01 = dot(e0, e1), g11 = dot(e1, e1);
    const double det = g00 * g11 - g01 * g01;
    const double sa = slope[2 * (size_t)j] / det, sb = slope[2 * (size_t)j + 1] / det;
    const double c0 = sa * g11 - sb * g01, c1 = sb * g00 - sa * g01;
    dn.sc = sc;
    dn.g = D3{c0 * e0.x + c1 * e1.x, c0 * e0.y + c1 * e1.y, c0 * e0.z + c1 * e1.z};
    dn.C = D3{cen[3 * (size_t)j], cen[3 * (size_t)j + 1], cen[3 * (size_t)j + 2]};
    for (int k = 0; k < 6; ++k) dn.H[k] = 0.0;
    if (curv) {
        const double ig = 1.0 / det;
        const D3 d0{(g11 * e0.x - g01 * e1.x) * ig, (g11 * e0.y - g01 * e1.y) * ig, (g11 * e0.z - g01 * e1.z) * ig};
        const D3 d1{(g00 * e1.x - g01 * e0.x) * ig, (g00 * e1.y - g01 * e0.y) * ig, (g00 * e1.z - g01 * e0.z) * ig};
        const double* cq = curv + 3 * (size_t)j;
        const double a2 = 2.0 * cq[0], ab = cq[1], b2 = 2.0 * cq[2];
        dn.H[0] = a2 * d0.x * d0.x + 2.0 * ab * d0.x * d1.x + b2 * d1.x * d1.x;
        dn.H[1] = a2 * d0.y * d0.y + 2.0 * ab * d0.y * d1.y + b2 * d1.y * d1.y;
        dn.H[2] = a2 * d0.z * d0.z + 2.0 * ab * d0.z * d1.z + b2 * d1.z * d1.z;
        dn.H[3] = a2 * d0.x * d0.y + ab * (d0.x * d1.y + d1.x * d0.y) + b2 * d1.x * d1.y;
        dn.H[4] = a2 * d0.x * d0.z + ab * (d0.x * d1.z + d1.x * d0.z) + b2 * d1.x * d1.z;
        dn.H[5] = a2 * d0.y * d0.z + ab * (d0.y * d1.z + d1.y * d0.z) + b2 * d1.y * d1.z;
    }
}

// Line integral over the edge c1 -> c2 (corners relative to P) of sigma(Q) (P - Q) / R^3 ds.
// With F the foot of the perpendicular from P on the edge line, s the coordinate along t
// from F and rho = |F - P|, sigma = b0 + b1 s + b2 s^2 on the edge and
//   int = -(F - P) (b0 M0 + b1 M1 + b2 M2) - t (b0 M1 + b1 M2 + b2 M3),
//   M0 = [s / (rho^2 R)], M1 = [-1/R], M2 = [ln(s + R) - s/R] = l - rho^2 M0,
//   M3 = [R + rho^2 / R] = (R2 - R1) - rho^2 M1
// (the brackets differences between the edge ends; M0 and M1 in cancellation-free
// quotient forms).  A point on the closed edge gives 0.
__device__ D3 edge_density_field(D3 c1, D3 c2, D3 P, const Density& dn) {
    D3 t = sub(c2, c1);
    t = scale(t, 1.0 / sqrt(dot(t, t)));
    const double u1 = dot(c1, t), u2 = dot(c2, t);
    const double R1 = sqrt(dot(c1, c1)), R2 = sqrt(dot(c2, c2));
    const D3 rho = sub(c1, scale(t, u1));  // F - P
    const double rho2 = dot(rho, rho);
    if (R1 == 0.0 || R2 == 0.0) return D3{0.0, 0.0, 0.0};
    double M0;
    if (u1 >= 0.0) M0 = (u2 - u1) * (u2 + u1) / (R1 * R2 * (u2 * R1 + u1 * R2));
    else if (u2 <= 0.0) M0 = (u1 - u2) * (u1 + u2) / (R1 * R2 * (-u1 * R2 - u2 * R1));
    else if (rho2 > 0.0) M0 = (u2 / R2 - u1 / R1) / rho2;
    else return D3{0.0, 0.0, 0.0};
    const double M1 = (u2 - u1) * (u2 + u1) / (R1 * R2 * (R1 + R2));
    double num, den;
    if (u1 >= 0.0) {
        num = R2 + u2;
        den = R1 + u1;
    } else if (u2 <= 0.0) {
        num = R1 - u1;
        den = R2 - u2;
    } else {
        num = (R2 + u2) * (R1 - u1);
        den = rho2;
    }
    const double l = den == 0.0 ? 0.0 : log(num / den);
    const double M2 = l - rho2 * M0;
    const double M3 = (u2 - u1) * (u2 + u1) / (R1 + R2) - rho2 * M1;
    // sigma, its slope along t and half its curvature along t at the foot
    const D3 dF = sub(D3{P.x + rho.x, P.y + rho.y, P.z + rho.z}, dn.C);
    const D3 HdF = hmul(dn.H, dF);
    const double b0 = dn.sc + dot(dn.g, dF) + 0.5 * dot(dF, HdF);
    const double b1 = dot(dn.g, t) + dot(HdF, t);
    const double b2 = 0.5 * hform(dn.H, t, t);
    const double a = fma(b0, M0, fma(b1, M1, b2 * M2)), b = fma(b0, M1, fma(b1, M2, b2 * M3));
    return D3{-rho.x * a - t.x * b, -rho.y * a - t.y * b, -rho.z * a - t.z * b};
}

// Field gradient (xx, yy, zz, xy, xz, yz; without 1/(4 pi eps0)) of the polygon with the
// density dn at P.  For an in-plane unit vector tau the derivative moves from P onto the
// density (dK(P - Q)/dP = -dK(P - Q)/dQ for K(x) = x / |x|^3, then the divergence theorem
// in the plane):
//   dE/dtau = E[d sigma / dtau] - sum_e (tau.m_e) int_e sigma (P - Q) / R^3 ds,
// with E[d sigma / dtau] the field of the linear density tau.g + (H tau).(Q - C).  The
// normal column follows from the symmetry of the tensor and its zero trace off the element.
__device__ void polygon_grad_var(int nv, const double* __restrict__ V, const double* __restrict__ G, D3 P, const Density& dn,
                                 double out[6]) {
    D3 c[4];
    for (int k = 0; k < nv; ++k) c[k] = sub(D3{V[3 * k], V[3 * k + 1], V[3 * k + 2]}, P);
    D3 nrm = cross(sub(c[1], c[0]), sub(c[2], c[0]));
    nrm = scale(nrm, 1.0 / sqrt(dot(nrm, nrm)));
    D3 tau[2];
    tau[0] = sub(c[1], c[0]);
    tau[0] = scale(tau[0], 1.0 / sqrt(dot(tau[0], tau[0])));
    tau[1] = cross(nrm, tau[0]);
    D3 col[3];
    for (int q = 0; q < 2; ++q) {
        double f[4];
        polygon_field_lin(nv, V, G, P, dot(tau[q], dn.g), hmul(dn.H, tau[q]), dn.C, f);
        D3 v{f[1], f[2], f[3]};
        for (int k = 0; k < nv; ++k) {
            const int k2 = (k + 1 == nv) ? 0 : k + 1;
            D3 t = sub(c[k2], c[k]);
            t = scale(t, 1.0 / sqrt(dot(t, t)));
            const double tm = dot(tau[q], cross(t, nrm));
            const D3 L = edge_density_field(c[k], c[k2], P, dn);
            v = D3{fma(-tm, L.x, v.x), fma(-tm, L.y, v.y), fma(-tm, L.z, v.z)};
        }
        col[q] = v;
    }
    const double n0 = dot(nrm, col[0]), n1 = dot(nrm, col[1]);
    const double nn = -(dot(tau[0], col[0]) + dot(tau[1], col[1]));
    col[2] = D3{n0 * tau[0].x + n1 * tau[1].x + nn * nrm.x, n0 * tau[0].y + n1 * tau[1].y + nn * nrm.y,
                n0 * tau[0].z + n1 * tau[1].z + nn * nrm.z};
    // G = col_0 tau_0^T + col_1 tau_1^T + col_2 n^T, symmetrised
    auto Gab = [&](int a, int b) {
        const double ca[3] = {a == 0 ? col[0].x : a == 1 ? col[0].y : col[0].z,
                              a == 0 ? col[1].x : a == 1 ? col[1].y : col[1].z,
                              a == 0 ? col[2].x : a == 1 ? col[2].y : col[2].z};
        const double rb[3] = {b == 0 ? tau[0].x : b == 1 ? tau[0].y : tau[0].z,
                              b == 0 ? tau[1].x : b == 1 ? tau[1].y : tau[1].z,
                              b == 0 ? nrm.x : b == 1 ? nrm.y : nrm.z};
        return ca[0] * rb[0] + ca[1] * rb[1] + ca[2] * rb[2];
    };
    out[0] = Gab(0, 0);
    out[1] = Gab(1, 1);
    out[2] = Gab(2, 2);
    out[3] = 0.5 * (Gab(0, 1) + Gab(1, 0));
    out[4] = 0.5 * (Gab(0, 2) + Gab(2, 0));
    out[5] = 0.5 * (Gab(1, 2) + Gab(2, 1));
}

// Gradient of each near-pair run's pairs, times sigma, at the pairs' slots (two double4
// each); linear / quadratic densities (slope set) by polygon_grad_var.
__global__ void k_near_grad(const int4* __restrict__ rec, const unsigned long long* counters, unsigned long long cap,
                            const NearBounds nb, unsigned long long gcap, const double* __restrict__ pts, const int* __restrict__ perm,
                            const int* __restrict__ near_off, const int* __restrict__ near_row,
                            const int* __restrict__ near_rows, int n_chunks, int chunk_len,
                            const int* __restrict__ type, const double* __restrict__ verts,
                            const double* __restrict__ sigma, const double* __restrict__ slope,
                            const double* __restrict__ curv, const double* __restrict__ fr,
                            const double* __restrict__ cen, const double* __restrict__ egeo, double4* __restrict__ gval) {
    const unsigned long long n = min(counters[0], cap);
    auto slot_of = [&](const int4 r) { return near_slot(r, near_off, near_row, near_rows, n_chunks, chunk_len); };
    for_each_near_pair(rec, n, pts, perm, nb, slot_of, [&](const int4 r, int k, const D3 P, unsigned long long slot) {
        if (slot >= gcap) return;
        const int el = r.y + k;
        const int nv = type[el] == BEM_RECTANGLE ? 4 : 3;
        double f[6];
        double sg = sigma[el];
        if (slope) {
            Density dn;
            element_density(el, sg, slope, curv, fr, cen, dn);
            polygon_grad_var(nv, verts + 12 * (size_t)el, egeo + (size_t)kEgeo * el, P, dn, f);
            sg = 1.0;
        } else {
            polygon_grad(nv, verts + 12 * (size_t)el, egeo + (size_t)kEgeo * el, P, f);
        }
        gval[2 * slot] = make_double4(sg * f[0], sg * f[1], sg * f[2], sg * f[3]);
        gval[2 * slot + 1] = make_double4(sg * f[4], sg * f[5], 0.0, 0.0);
    });
}

// phi and E of each near-pair run's pairs, times sigma, at the pairs' slots;
// linear / quadratic densities (slope set) by the analytic integral of the density.
__global__ void k_near_eval(const int4* __restrict__ rec, const unsigned long long* counters, unsigned long long cap,
                            const NearBounds nb, const double* __restrict__ pts, const int* __restrict__ perm,
                            const int* __restrict__ near_off, const int* __restrict__ near_row,
                            const int* __restrict__ near_rows, int n_chunks, int chunk_len,
                            const int* __restrict__ type, const double* __restrict__ verts,
                            const double* __restrict__ sigma, const double* __restrict__ slope,
                            const double* __restrict__ curv, const double* __restrict__ fr,
                            const double* __restrict__ cen, const double* __restrict__ egeo, double4* __restrict__ val) {
    const unsigned long long n = min(counters[0], cap);
    auto slot_of = [&](const int4 r) { return near_slot(r, near_off, near_row, near_rows, n_chunks, chunk_len); };
    for_each_near_pair(rec, n, pts, perm, nb, slot_of, [&](const int4 r, int k, const D3 P, unsigned long long slot) {
        if (slot >= cap) return;
        const int el = r.y + k;
        double f[4];
        const int nv = type[el] == BEM_RECTANGLE ? 4 : 3;
        double sg = sigma[el];
        if (slope) {
            Density dn;
            element_density(el, sg, slope, curv, fr, cen, dn);
            const double* G = egeo + (size_t)kEgeo * el;
            if (curv) polygon_field_quad(nv, verts + 12 * (size_t)el, G, P, dn.sc, dn.g, dn.H, dn.C, f);
            else polygon_field_lin(nv, verts + 12 * (size_t)el, G, P, dn.sc, dn.g, dn.C, f);
            sg = 1.0;
        } else {
            polygon_field(nv, verts + 12 * (size_t)el, egeo + (size_t)kEgeo * el, P, f);
        }
        val[slot] = make_double4(sg * f[0], sg * f[1], sg * f[2], sg * f[3]);
    });
}

// far sums (the element chunks already summed in chunk order) + near
// contributions in element order, times 1/(4 pi eps0), written at the point's
// original position.
__global__ void k_finalize(int n, const int* n_dev, const int* __restrict__ perm, const double4* __restrict__ far,
                           const int* __restrict__ near_tot, const int* __restrict__ near_off,
                           const double4* __restrict__ val, unsigned long long cap, double kc, double* phi, double* E,
                           int stride4) {
    if (n_dev) n = min(n, *n_dev);
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double4 s = far[i];
    const int cnt = near_tot[i];
    const unsigned long long off = (unsigned long long)near_off[i];
    for (int k = 0; k < cnt; ++k) {
        if (off + k >= cap) break;
        const double4 v = val[off + k];
        s.x += v.x;
        s.y += v.y;
        s.z += v.z;
        s.w += v.w;
    }
    const int o = perm[i];
    if (stride4) {  // packed (phi, Ex, Ey, Ez) per point
        phi[4 * (size_t)o] = kc * s.x;
        phi[4 * (size_t)o + 1] = kc * s.y;
        phi[4 * (size_t)o + 2] = kc * s.z;
        phi[4 * (size_t)o + 3] = kc * s.w;
        return;
    }
    if (phi) phi[o] = kc * s.x;
    if (E) {
        E[3 * (size_t)o] = kc * s.y;
        E[3 * (size_t)o + 1] = kc * s.z;
        E[3 * (size_t)o + 2] = kc * s.w;
    }
}

__global__ void k_near_assemble(const int4* __restrict__ rec, const unsigned long long* counters,
                                unsigned long long cap, const NearBounds nb, const double* __restrict__ pts, const int* __restrict__ perm,
                                const int* __restrict__ type, const double* __restrict__ verts,
                                const double* __restrict__ egeo, int n_el, double kc, double* __restrict__ A) {
    const unsigned long long n = min(counters[0], cap);
    auto no_slot = [](const int4) { return 0ull; };
    for_each_near_pair(rec, n, pts, perm, nb, no_slot, [&](const int4 r, int k, const D3 P, unsigned long long) {
        const int el = r.y + k;
        double f[4];
        polygon_field(type[el] == BEM_RECTANGLE ? 4 : 3, verts + 12 * (size_t)el, egeo + (size_t)kEgeo * el, P, f);
        A[(size_t)perm[r.x] * n_el + el] = kc * f[0];
    });
}

// Self potential of each element at its own centroid (unit sigma), times kc:
// the diagonal of the collocation matrix at the centroids.
__global__ void k_self_potential(int n, const int* __restrict__ type, const double* __restrict__ verts,
                                 const double* __restrict__ egeo, const double* __restrict__ cen, double kc,
                                 double* __restrict__ out) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    double f[4];
    polygon_field(type[j] == BEM_RECTANGLE ? 4 : 3, verts + 12 * (size_t)j, egeo + (size_t)kEgeo * j,
                  D3{cen[3 * j], cen[3 * j + 1], cen[3 * j + 2]}, f);
    out[j] = kc * f[0];
}

}  // namespace

int launch_self_potential(bem_mesh* m, double* out, cudaStream_t s) {
    const int n = m->d.n;
    if (n == 0) return BEM_OK;
    k_self_potential<<<(n + 255) / 256, 256, 0, s>>>(n, m->d.type, m->d.verts, m->d.egeo, m->d.cen, m->kc, out);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}

static NearBounds near_bounds(bem_mesh* m) {
    return NearBounds{(int)std::min<size_t>(m->w.cap_pts, INT_MAX), m->d.n, m->w.counters};
}

int launch_near_eval(bem_mesh* m, const double* pts, const int* perm, int n_pts, const double* sigma,
                     unsigned long long /*n_near_hint*/, cudaStream_t s, const double* slope) {
    (void)n_pts;
    Work& w = m->w;
    k_near_eval<<<152 * 8, kNearThreads, 0, s>>>(w.near_rec, w.counters, (unsigned long long)w.cap_near,
                                        near_bounds(m), pts, perm, w.near_off,
                                        w.near_row, w.near_rows, m->n_chunks, m->chunk_len, m->d.type, m->d.verts,
                                        sigma, slope, eval_curv(m, slope),
                                        m->d.fr, m->d.cen, m->d.egeo, w.near_val);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}

int launch_finalize(bem_mesh* m, const int* perm, int n_pts, double* phi, double* E, int stride4, cudaStream_t s,
                    const int* n_dev) {
    Work& w = m->w;
    k_finalize<<<(n_pts + 255) / 256, 256, 0, s>>>(n_pts, n_dev, perm, w.far, w.near_tot, w.near_off, w.near_val,
                                                   (unsigned long long)w.cap_near, m->kc, phi, E, stride4);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}

int launch_near_grad(bem_mesh* m, const double* pts, const int* perm, const double* sigma, double4* gval,
                     unsigned long long gcap, cudaStream_t s, const double* slope) {
    Work& w = m->w;
    k_near_grad<<<152 * 8, kNearThreads, 0, s>>>(w.near_rec, w.counters, (unsigned long long)w.cap_near,
                                        near_bounds(m), gcap, pts, perm,
                                        w.near_off, w.near_row, w.near_rows, m->n_chunks, m->chunk_len, m->d.type,
                                        m->d.verts, sigma, slope,
                                        eval_curv(m, slope), m->d.fr, m->d.cen, m->d.egeo, gval);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}

int launch_finalize_grad(bem_mesh* m, const int* perm, int n_pts, const double4* far_g, const double4* gval,
                         unsigned long long gcap, double* G, cudaStream_t s) {
    Work& w = m->w;
    k_finalize_grad<<<(n_pts + 255) / 256, 256, 0, s>>>(n_pts, perm, far_g, w.near_tot, w.near_off,
                                                        gval, gcap, m->kc, G);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}

int launch_near_assemble(bem_mesh* m, const double* pts, const int* perm, double* A, unsigned long long,
                         cudaStream_t s) {
    Work& w = m->w;
    k_near_assemble<<<152 * 8, kNearThreads, 0, s>>>(w.near_rec, w.counters, (unsigned long long)w.cap_near,
                                            near_bounds(m), pts, perm,
                                            m->d.type, m->d.verts, m->d.egeo, m->d.n, m->kc, A);
    BEM_CUDA_TRY(cudaGetLastError());
    count_launches(1);
    return BEM_OK;
}

}  // namespace bem
