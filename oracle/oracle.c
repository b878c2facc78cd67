/*
 * oracle.c -- plain FP64 CPU oracle for the potential and field of charged
 * constant-density BEM triangles and rectangles (Glueck & Hilk,
 * "Electric potential and field calculation of charged BEM triangles and
 * rectangles by Gaussian cubature", arXiv:1606.03743).
 *
 * TEST INFRASTRUCTURE, NOT PRODUCT CODE.  Only the test suite, the smoke
 * check and the CPU-baseline leg of the benchmark load this file.  It shares
 * no code, header, table or constant with the CUDA library: every number
 * below is typed in here from the paper's appendix tables, and every formula
 * is written out from the equation or section it cites.
 *
 * It is deliberately plain: one field point at a time, every element in
 * index order, every step in the paper's order and notation, double
 * precision throughout (the paper's own arithmetic, Sec. 2 and Sec. 6).
 * The only parallelism is over independent field points, which does not
 * change any per-point arithmetic.
 *
 * Layers (the paper's):
 *   rule tables ........ App. A (Tables A1-A5), App. B (Tables B1-B5)
 *   natural coords ..... Eq. 3.2 (rectangle), Eq. 3.3 (barycentric, triangle)
 *   cubature formula ... Eq. 3.1
 *   point charges ...... Eq. 4.1
 *   distance ratio ..... Sec. 2 (DR = D / L)
 *   rule bands ......... Sec. 4 (DR-banded choice, analytic below DR = 3)
 *   analytic near field  Sec. 2 cites it without printing it; written here
 *                        from the divergence-theorem decomposition of a
 *                        uniformly charged planar polygon (edge logarithms
 *                        plus the solid angle, Van Oosterom & Strackee 1983).
 *   GL2 reference ...... Sec. 2 (two nested 16-node Gauss-Legendre rules)
 *
 * Pinned by tests/test_oracle_*.py against what the paper and mathematics
 * fix (rule exactness, closed forms, point-charge limit, E = -grad phi,
 * brute-force subdivision, Gauss's law, symmetry, the paper's printed rule
 * bands).  Nothing here is "parity unpinned".
 */
#include <math.h>
#include <stddef.h>
#include <stdint.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------ */
/* small vector helpers                                                */
/* ------------------------------------------------------------------ */
static double dot3(const double a[3], const double b[3]) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void sub3(const double a[3], const double b[3], double o[3]) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static void cross3(const double a[3], const double b[3], double o[3])
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double norm3(const double a[3]) { return sqrt(dot3(a, a)); }

/* ------------------------------------------------------------------ */
/* Cubature rules, App. A and App. B                                   */
/* ------------------------------------------------------------------ */
/* Rule index 0..4 <-> N = 4, 7, 12, 19, 33 (triangles, Tables A1-A5)
 *                 <-> N = 4, 7, 12, 17, 33 (rectangles, Tables B1-B5).
 * Triangle nodes are barycentric (lambda_A, lambda_B, lambda_C), Eq. 3.3.
 * Rectangle nodes are natural coordinates (x, y) in [-1, 1]^2, Eq. 3.2.
 * Weights sum to 1 (Eq. 3.1). */
#define MAXN 33
typedef struct {
    int n;
    double a[MAXN], b[MAXN], c[MAXN], w[MAXN];
} rule_t;

static rule_t TRI[5], RECT[5];
static int rules_ready = 0;

static void tri_add(rule_t* r, double la, double lb, double lc, double w)
{
    r->a[r->n] = la; r->b[r->n] = lb; r->c[r->n] = lc; r->w[r->n] = w; r->n++;
}
/* the three points with lambda_A = p and lambda_B = lambda_C = q, permuted
 * (caption of Table A2: "all possible different permutations of lambda_A
 * and lambda_B = lambda_C") */
static void tri_perm3(rule_t* r, double p, double q, double w)
{
    tri_add(r, p, q, q, w);
    tri_add(r, q, p, q, w);
    tri_add(r, q, q, p, w);
}
/* cyclic permutations (A,B,C) -> (B,C,A) -> (C,A,B), caption of Table A3 */
static void tri_cyc3(rule_t* r, double la, double lb, double lc, double w)
{
    tri_add(r, la, lb, lc, w);
    tri_add(r, lb, lc, la, w);
    tri_add(r, lc, la, lb, w);
}
/* all six permutations, captions of Tables A4 and A5 */
static void tri_perm6(rule_t* r, double la, double lb, double lc, double w)
{
    tri_add(r, la, lb, lc, w);
    tri_add(r, la, lc, lb, w);
    tri_add(r, lb, la, lc, w);
    tri_add(r, lb, lc, la, w);
    tri_add(r, lc, la, lb, w);
    tri_add(r, lc, lb, la, w);
}
static void rect_add(rule_t* r, double x, double y, double w)
{
    r->a[r->n] = x; r->b[r->n] = y; r->c[r->n] = 0.0; r->w[r->n] = w; r->n++;
}
/* all sign changes (x,y),(x,-y),(-x,y),(-x,-y), captions of Tables B2, B3 */
static void rect_sign4(rule_t* r, double x, double y, double w)
{
    rect_add(r, x, y, w);
    rect_add(r, x, -y, w);
    rect_add(r, -x, y, w);
    rect_add(r, -x, -y, w);
}
/* rotations by 0, 180, +90, -90 degrees: (x,y) -> +-(x,y), +-(-y,x),
 * captions of Tables B4 and B5 */
static void rect_rot4(rule_t* r, double x, double y, double w)
{
    rect_add(r, x, y, w);
    rect_add(r, -x, -y, w);
    rect_add(r, -y, x, w);
    rect_add(r, y, -x, w);
}

static void build_rules(void)
{
    rule_t* r;
    if (rules_ready) return;
    memset(TRI, 0, sizeof TRI);
    memset(RECT, 0, sizeof RECT);

    /* Table A1: 4 points, degree 3 */
    r = &TRI[0];
    tri_add(r, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, -9.0 / 16.0);
    tri_perm3(r, 3.0 / 5.0, 1.0 / 5.0, 25.0 / 48.0);

    /* Table A2: 7 points, degree 5; t = 1/3, s = (1-sqrt15)/7, r = (1+sqrt15)/7 */
    {
        const double q15 = sqrt(15.0), t = 1.0 / 3.0;
        const double s = (1.0 - q15) / 7.0, rr = (1.0 + q15) / 7.0;
        r = &TRI[1];
        tri_add(r, t, t, t, 9.0 / 40.0);
        tri_perm3(r, t + 2.0 * t * s, t - t * s, (155.0 + q15) / 1200.0);
        tri_perm3(r, t + 2.0 * t * rr, t - t * rr, (155.0 - q15) / 1200.0);
    }

    /* Table A3: 12 points, degree 7 (cyclic permutations) */
    r = &TRI[2];
    tri_cyc3(r, 0.06238226509439084, 0.06751786707392436, 0.8700998678316848, 0.05303405631486900);
    tri_cyc3(r, 0.05522545665692000, 0.3215024938520156, 0.6232720494910644, 0.08776281742889622);
    tri_cyc3(r, 0.03432430294509488, 0.6609491961867980, 0.3047265008681072, 0.05755008556995056);
    tri_cyc3(r, 0.5158423343536001, 0.2777161669764050, 0.2064414986699949, 0.13498637401961758);

    /* Table A4: 19 points, degree 9 */
    r = &TRI[3];
    tri_add(r, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, 0.09713579628279610);
    tri_perm3(r, 0.02063496160252593, 0.48968251919873704, 0.03133470022713983);
    tri_perm3(r, 0.1258208170141290, 0.4370895914929355, 0.07782754100477543);
    tri_perm3(r, 0.6235929287619356, 0.18820353561903219, 0.07964773892720910);
    tri_perm3(r, 0.9105409732110941, 0.04472951339445297, 0.02557767565869810);
    tri_perm6(r, 0.03683841205473626, 0.7411985987844980, 0.22196298916076573, 0.04328353937728940);

    /* Table A5: 33 points, degree 12 */
    r = &TRI[4];
    tri_perm3(r, 0.4570749859701478, 0.27146250701492611, 0.06254121319590276);
    tri_perm3(r, 0.1197767026828138, 0.44011164865859310, 0.04991833492806094);
    tri_perm3(r, 0.0235924981089169, 0.48820375094554155, 0.02426683808145203);
    tri_perm3(r, 0.7814843446812914, 0.10925782765935432, 0.02848605206887754);
    tri_perm3(r, 0.9507072731273288, 0.02464636343633558, 0.00793164250997364);
    tri_perm6(r, 0.1162960196779266, 0.2554542286385173, 0.62824975168355610, 0.04322736365941421);
    tri_perm6(r, 0.02303415635526714, 0.2916556797383410, 0.68531016390639186, 0.02178358503860756);
    tri_perm6(r, 0.02138249025617059, 0.1272797172335894, 0.85133779251024000, 0.01508367757651144);

    /* Table B1: 4 points, degree 3; s = 1/sqrt3 */
    r = &RECT[0];
    rect_sign4(r, 1.0 / sqrt(3.0), 1.0 / sqrt(3.0), 0.25);

    /* Table B2: 7 points, degree 5; t = sqrt(14/15), r = sqrt(3/5), s = sqrt(1/3).
     * The (0, +-t) nodes lie on the local y axis exactly as printed. */
    r = &RECT[1];
    rect_add(r, 0.0, 0.0, 2.0 / 7.0);
    rect_add(r, 0.0, sqrt(14.0 / 15.0), 5.0 / 63.0);
    rect_add(r, 0.0, -sqrt(14.0 / 15.0), 5.0 / 63.0);
    rect_sign4(r, sqrt(3.0 / 5.0), sqrt(1.0 / 3.0), 5.0 / 36.0);

    /* Table B3: 12 points, degree 7 */
    {
        const double q583 = sqrt(583.0);
        const double rr = sqrt(6.0 / 7.0);
        const double s = sqrt((114.0 - 3.0 * q583) / 287.0);
        const double t = sqrt((114.0 + 3.0 * q583) / 287.0);
        const double B1 = 49.0 / 810.0;
        const double B2 = (178981.0 + 2769.0 * q583) / 1888920.0;
        const double B3 = (178981.0 - 2769.0 * q583) / 1888920.0;
        r = &RECT[2];
        rect_add(r, rr, 0.0, B1);
        rect_add(r, -rr, 0.0, B1);
        rect_add(r, 0.0, rr, B1);
        rect_add(r, 0.0, -rr, B1);
        rect_sign4(r, s, s, B2);
        rect_sign4(r, t, t, B3);
    }

    /* Table B4: 17 points, degree 9 */
    r = &RECT[3];
    rect_add(r, 0.0, 0.0, 0.131687242798353921);
    rect_rot4(r, 0.968849966361977720, 0.630680119731668854, 0.022219844542549678);
    rect_rot4(r, 0.750277099978900533, 0.927961645959569667, 0.028024900532399120);
    rect_rot4(r, 0.523735820214429336, 0.453339821135647190, 0.099570609815517519);
    rect_rot4(r, 0.076208328192617173, 0.852615729333662307, 0.067262834409945196);

    /* Table B5: 33 points, degree 13 */
    r = &RECT[4];
    rect_add(r, 0.0, 0.0, 0.075095528857806335);
    rect_rot4(r, 0.778809711554419422, 0.983486682439872263, 0.007497959716124783);
    rect_rot4(r, 0.957297699786307365, 0.859556005641638928, 0.009543605329270918);
    rect_rot4(r, 0.138183459862465353, 0.958925170287534857, 0.015106230954437494);
    rect_rot4(r, 0.941327225872925236, 0.390736216129461000, 0.019373184633276336);
    rect_rot4(r, 0.475808625218275905, 0.850076673699748575, 0.029711166825148901);
    rect_rot4(r, 0.755805356572081436, 0.647821637187010732, 0.032440887592500675);
    rect_rot4(r, 0.696250078491749413, 0.070741508996444936, 0.053335395364297350);
    rect_rot4(r, 0.342716556040406789, 0.409304561694038843, 0.064217687370491966);

    rules_ready = 1;
}

/* ------------------------------------------------------------------ */
/* Element geometry: Sec. 2 (centroid, L), Eq. 3.2, Eq. 3.3              */
/* ------------------------------------------------------------------ */
/* type 0 = triangle with corners A, B, C (v[0..2]);
 * type 1 = rectangle with corners P0, P1, P2, P3 in order around the
 * boundary, side a along P0->P1 (u_x), side b along P0->P3 (u_y). */
typedef struct {
    int type;
    double v[4][3];
    double cen[3];   /* Q_cen */
    double L;        /* average side length */
    double area;     /* cal A */
    double ux[3], uy[3], a, b; /* rectangle frame, Eq. 3.2 */
} elem_t;

static void elem_setup(elem_t* e, int type, const double* verts)
{
    int i, k;
    e->type = type;
    for (i = 0; i < 4; ++i)
        for (k = 0; k < 3; ++k) e->v[i][k] = verts[3 * i + k];
    if (type == 0) {
        double ab[3], ac[3], bc[3], cr[3];
        sub3(e->v[1], e->v[0], ab);
        sub3(e->v[2], e->v[0], ac);
        sub3(e->v[2], e->v[1], bc);
        cross3(ab, ac, cr);
        e->area = 0.5 * norm3(cr);
        for (k = 0; k < 3; ++k) e->cen[k] = (e->v[0][k] + e->v[1][k] + e->v[2][k]) / 3.0;
        /* L = (a + b + c) / 3, Sec. 2 */
        e->L = (norm3(ab) + norm3(bc) + norm3(ac)) / 3.0;
    } else {
        double d1[3], d3[3];
        sub3(e->v[1], e->v[0], d1);
        sub3(e->v[3], e->v[0], d3);
        e->a = norm3(d1);
        e->b = norm3(d3);
        for (k = 0; k < 3; ++k) {
            e->ux[k] = d1[k] / e->a;
            e->uy[k] = d3[k] / e->b;
            e->cen[k] = (e->v[0][k] + e->v[1][k] + e->v[2][k] + e->v[3][k]) / 4.0;
        }
        e->area = e->a * e->b;
        /* mean of the four side lengths (the paper states L for the triangle
         * only; the rectangle reading is (a + b) / 2) */
        e->L = 0.5 * (e->a + e->b);
    }
}

/* i-th node of a rule, Eq. 3.3 (triangle) or Eq. 3.2 (rectangle) */
static void rule_node(const elem_t* e, const rule_t* r, int i, double Q[3])
{
    int k;
    if (e->type == 0) {
        for (k = 0; k < 3; ++k) Q[k] = r->a[i] * e->v[0][k] + r->b[i] * e->v[1][k] + r->c[i] * e->v[2][k];
    } else {
        for (k = 0; k < 3; ++k)
            Q[k] = e->cen[k] + 0.5 * e->a * r->a[i] * e->ux[k] + 0.5 * e->b * r->b[i] * e->uy[k];
    }
}

/* ------------------------------------------------------------------ */
/* Point-charge cubature, Eq. 4.1 (unit sigma; 1/(4 pi eps0) applied by  */
/* the caller)                                                          */
/* ------------------------------------------------------------------ */
static void cubature_field(const elem_t* e, int rule, const double P[3], double out[4])
{
    const rule_t* r = e->type == 0 ? &TRI[rule] : &RECT[rule];
    double phi = 0.0, Ex = 0.0, Ey = 0.0, Ez = 0.0;
    int i;
    for (i = 0; i < r->n; ++i) {
        double Q[3], d[3], dist, qi;
        rule_node(e, r, i, Q);
        sub3(P, Q, d);
        dist = norm3(d);
        qi = r->w[i] * e->area; /* q_i = w_i q with q = sigma * area, sigma = 1 */
        phi += qi / dist;
        Ex += qi * d[0] / (dist * dist * dist);
        Ey += qi * d[1] / (dist * dist * dist);
        Ez += qi * d[2] / (dist * dist * dist);
    }
    out[0] = phi; out[1] = Ex; out[2] = Ey; out[3] = Ez;
}

/* ------------------------------------------------------------------ */
/* Analytic near field of a uniformly charged planar polygon (unit       */
/* sigma, no 1/(4 pi eps0)).                                            */
/*                                                                      */
/* The paper uses analytical integration below DR = 3 (Sec. 4) and      */
/* cites the formulas without printing them.  This is the standard      */
/* decomposition from potential theory.  With n the unit normal of the  */
/* polygon (corners counter-clockwise seen from +n), h = (P - V)·n the  */
/* signed height, and for each edge e from V1 to V2 the unit tangent t,  */
/* the in-plane outward normal m = t x n, d = (V1 - P)·m, s_k = (V_k-P)·t,*/
/* R_k = |P - V_k| and l = ln((s2 + R2) / (s1 + R1)) = integral of ds/R  */
/* along the edge:                                                      */
/*   int dA / R            = sum_e d_e l_e - h Omega                    */
/*   int (P-Q) / R^3 dA    = sum_e m_e l_e + n Omega                    */
/* where Omega is the solid angle of the polygon seen from P, signed     */
/* like h.  (The first line is the 2-D divergence theorem applied to the */
/* in-plane field rho (R - |h|) / rho^2; the second follows from         */
/* grad_Q (1/R) on the edges and from h / R^3 being the solid-angle      */
/* density.)                                                            */
/* ------------------------------------------------------------------ */

/* integral of ds / R over an edge, written so that no sum of nearly
 * opposite terms occurs: s1 < s2 always (s grows along the edge).
 * A field point ON the closed edge makes the integral diverge (only
 * logarithmically); the edge then contributes d l -> 0 to the potential
 * (d = 0 there) and its singular in-plane field is left out: 0 is
 * returned.  (The paper does not treat field points on an element.) */
static double edge_log(double s1, double s2, double R1, double R2, double perp2)
{
    double num, den;
    if (s1 >= 0.0) { num = R2 + s2; den = R1 + s1; }
    else if (s2 <= 0.0) { num = R1 - s1; den = R2 - s2; }
    else { num = (R2 + s2) * (R1 - s1); den = perp2; } /* s1 < 0 < s2: R1 + s1 = perp^2 / (R1 - s1) */
    if (den == 0.0) return 0.0;
    return log(num / den);
}

/* solid angle of triangle (a, b, c) seen from P, Van Oosterom & Strackee
 * (1983), returned with the sign of h for a triangle that is counter-
 * clockwise about n. */
static double tri_solid_angle(const double a[3], const double b[3], const double c[3], const double P[3])
{
    double Ra[3], Rb[3], Rc[3], bxc[3], num, den, ra, rb, rc;
    sub3(a, P, Ra);
    sub3(b, P, Rb);
    sub3(c, P, Rc);
    ra = norm3(Ra); rb = norm3(Rb); rc = norm3(Rc);
    cross3(Rb, Rc, bxc);
    num = dot3(Ra, bxc);
    den = ra * rb * rc + dot3(Ra, Rb) * rc + dot3(Ra, Rc) * rb + dot3(Rb, Rc) * ra;
    /* num = -2 * area * h for a counter-clockwise triangle */
    return 2.0 * atan2(-num, den);
}

static void analytic_field(const elem_t* e, const double P[3], double out[4])
{
    const int nv = e->type == 0 ? 3 : 4;
    double n[3], e1[3], e2[3], nl, h, phi = 0.0, E[3] = {0.0, 0.0, 0.0}, omega;
    int k, j;
    sub3(e->v[1], e->v[0], e1);
    sub3(e->v[2], e->v[0], e2);
    cross3(e1, e2, n);
    nl = norm3(n);
    for (k = 0; k < 3; ++k) n[k] /= nl;
    {
        double pv[3];
        sub3(P, e->v[0], pv);
        h = dot3(pv, n);
    }
    for (j = 0; j < nv; ++j) {
        const double* V1 = e->v[j];
        const double* V2 = e->v[(j + 1) % nv];
        double t[3], m[3], r1[3], r2[3], len, s1, s2, R1, R2, d, perp2, l;
        sub3(V2, V1, t);
        len = norm3(t);
        for (k = 0; k < 3; ++k) t[k] /= len;
        cross3(t, n, m);
        sub3(V1, P, r1);
        sub3(V2, P, r2);
        s1 = dot3(r1, t);
        s2 = dot3(r2, t);
        R1 = norm3(r1);
        R2 = norm3(r2);
        d = dot3(r1, m);
        perp2 = d * d + h * h;
        l = edge_log(s1, s2, R1, R2, perp2);
        phi += d * l;
        for (k = 0; k < 3; ++k) E[k] += m[k] * l;
    }
    if (fabs(h) <= 1e-12 * e->L) {
        /* field point in the element plane (to 1e-12 of the mean side, so
         * that a point computed to lie on the element, such as its centroid,
         * counts as on it whatever the rounding of h): h * Omega = 0; on the
         * element the normal field jumps, and the mean of both sides (0) is used */
        omega = 0.0;
    } else {
        omega = tri_solid_angle(e->v[0], e->v[1], e->v[2], P);
        if (nv == 4) omega += tri_solid_angle(e->v[0], e->v[2], e->v[3], P);
    }
    phi -= h * omega;
    for (k = 0; k < 3; ++k) E[k] += n[k] * omega;
    out[0] = phi; out[1] = E[0]; out[2] = E[1]; out[3] = E[2];
}

/* ------------------------------------------------------------------ */
/* GL2 reference integrator, Sec. 2: two nested 16-node Gauss-Legendre   */
/* quadratures.                                                         */
/* ------------------------------------------------------------------ */
#define NGL_MAX 64
/* Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on P_n */
static void gauss_legendre(int n, double* x, double* w)
{
    int i, it, j;
    for (i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), pp = 0.0;
        for (it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z, z1;
            for (j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            /* p1 = P_n(z), p0 = P_{n-1}(z) */
            pp = n * (z * p1 - p0) / (z * z - 1.0);
            z1 = z;
            z = z1 - p1 / pp;
            if (fabs(z - z1) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (j = 2; j <= n; ++j) {
                double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            pp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = -z;
        w[i] = 2.0 / ((1.0 - z * z) * pp * pp);
    }
}

/* GL2 over one element with n x n nodes.  Rectangle: tensor product over
 * (x, y) in [-1,1]^2 of Eq. 3.2, Jacobian a b / 4.  Triangle: collapsed map
 * Q(u, v) = A + u (B - A) + u v (C - B), (u, v) in [0,1]^2, Jacobian
 * 2 area u (the paper does not state its triangle mapping). */
static void gl2_field(const elem_t* e, int n, const double P[3], double out[4])
{
    double x[NGL_MAX], w[NGL_MAX], acc[4] = {0.0, 0.0, 0.0, 0.0};
    int i, j, k;
    gauss_legendre(n, x, w);
    for (i = 0; i < n; ++i) {
        for (j = 0; j < n; ++j) {
            double Q[3], d[3], dist, wt;
            if (e->type == 1) {
                for (k = 0; k < 3; ++k)
                    Q[k] = e->cen[k] + 0.5 * e->a * x[i] * e->ux[k] + 0.5 * e->b * x[j] * e->uy[k];
                wt = w[i] * w[j] * e->a * e->b / 4.0;
            } else {
                const double u = 0.5 * (x[i] + 1.0), v = 0.5 * (x[j] + 1.0);
                for (k = 0; k < 3; ++k)
                    Q[k] = e->v[0][k] + u * (e->v[1][k] - e->v[0][k]) + u * v * (e->v[2][k] - e->v[1][k]);
                wt = 0.25 * w[i] * w[j] * 2.0 * e->area * u;
            }
            sub3(P, Q, d);
            dist = norm3(d);
            acc[0] += wt / dist;
            for (k = 0; k < 3; ++k) acc[k + 1] += wt * d[k] / (dist * dist * dist);
        }
    }
    for (k = 0; k < 4; ++k) out[k] = acc[k];
}

/* Brute force: split the element into 2^level x 2^level congruent pieces
 * (triangle: midpoint subdivision into 4 per level; rectangle: quadrants)
 * and sum GL2 over the pieces. */
static void subdiv_field(const elem_t* e, int level, int n, const double P[3], double out[4])
{
    int k;
    if (level == 0) {
        gl2_field(e, n, P, out);
        return;
    }
    for (k = 0; k < 4; ++k) out[k] = 0.0;
    if (e->type == 0) {
        double m01[3], m12[3], m20[3], tris[4][4][3], part[4];
        int c, t;
        for (k = 0; k < 3; ++k) {
            m01[k] = 0.5 * (e->v[0][k] + e->v[1][k]);
            m12[k] = 0.5 * (e->v[1][k] + e->v[2][k]);
            m20[k] = 0.5 * (e->v[2][k] + e->v[0][k]);
        }
        for (k = 0; k < 3; ++k) {
            tris[0][0][k] = e->v[0][k]; tris[0][1][k] = m01[k];     tris[0][2][k] = m20[k];
            tris[1][0][k] = m01[k];     tris[1][1][k] = e->v[1][k]; tris[1][2][k] = m12[k];
            tris[2][0][k] = m20[k];     tris[2][1][k] = m12[k];     tris[2][2][k] = e->v[2][k];
            tris[3][0][k] = m12[k];     tris[3][1][k] = m20[k];     tris[3][2][k] = m01[k];
            for (c = 0; c < 4; ++c) tris[c][3][k] = 0.0;
        }
        for (t = 0; t < 4; ++t) {
            elem_t sub;
            elem_setup(&sub, 0, &tris[t][0][0]);
            subdiv_field(&sub, level - 1, n, P, part);
            for (c = 0; c < 4; ++c) out[c] += part[c];
        }
    } else {
        int qx, qy, c;
        for (qx = 0; qx < 2; ++qx) {
            for (qy = 0; qy < 2; ++qy) {
                double corners[4][3], part[4];
                const double x0 = qx - 1.0, y0 = qy - 1.0; /* quadrant [x0, x0+1] x [y0, y0+1] */
                const double xs[4] = {x0, x0 + 1.0, x0 + 1.0, x0};
                const double ys[4] = {y0, y0, y0 + 1.0, y0 + 1.0};
                elem_t sub;
                for (c = 0; c < 4; ++c)
                    for (k = 0; k < 3; ++k)
                        corners[c][k] = e->cen[k] + 0.5 * e->a * xs[c] * e->ux[k] + 0.5 * e->b * ys[c] * e->uy[k];
                elem_setup(&sub, 1, &corners[0][0]);
                subdiv_field(&sub, level - 1, n, P, part);
                for (c = 0; c < 4; ++c) out[c] += part[c];
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* Rule bands by distance ratio, Sec. 4                                 */
/* ------------------------------------------------------------------ */
/* lim[type][0..4] ascending DR limits.  DR < lim[0]: analytic;
 * lim[0] <= DR < lim[1]: 33 points; lim[1] <= DR < lim[2]: 19 (triangle) or
 * 17 (rectangle) points; lim[2] <= DR < lim[3]: 12 points;
 * lim[3] <= DR < lim[4]: 7 points; DR >= lim[4]: 4 points.
 * Sec. 4 prints the triangle-potential limits for 2e-15 (3, 8, 20, 80, 1500)
 * and says the field needs slightly higher ones, which then serve potential
 * and field together.  No field or rectangle limits are printed: the default
 * table below is the smallest DR per rule at which the mean err(phi) and
 * err(E) of the paper's experiment (oracle/dr_experiment.py, 2000 random
 * unit-cube elements per DR) stay below 2e-15, rounded up.  That includes
 * the near limit, the lower limit of the 33-point rule: for the triangle
 * potential alone the experiment puts it at DR 3, as printed; the field
 * needs DR 4.1 (triangles) and 5.3 (rectangles), taken as 4.5 and 6. */
static const double DEFAULT_LIMITS[2][5] = {
    {4.5, 12.0, 30.0, 120.0, 2250.0}, /* triangles */
    {6.0, 18.0, 45.0, 160.0, 2800.0}, /* rectangles */
};

/* band: 0 = analytic, else the rule index (4 = 33 points ... 0 = 4 points)
 * encoded as 1 + rule index */
static int choose_band(const elem_t* e, const double P[3], const double* lim, double* dr_out)
{
    double d[3], D, DR;
    int nb = 0, k;
    sub3(P, e->cen, d);
    D = norm3(d);          /* D = |P - Q_cen|, Sec. 2 */
    DR = D / e->L;         /* DR = D / L */
    if (dr_out) *dr_out = DR;
    for (k = 0; k < 5; ++k)
        if (DR >= lim[k]) nb++;
    if (nb == 0) return 0;
    return 1 + (5 - nb); /* nb = 1 -> 33 points (rule 4), nb = 5 -> 4 points (rule 0) */
}

/* ------------------------------------------------------------------ */
/* Neumaier-compensated summation (the element sum of Sec. 5 evaluated   */
/* as accurately as double precision allows)                            */
/* ------------------------------------------------------------------ */
static void nsum_add(double* s, double* c, double x)
{
    const double t = *s + x;
    if (fabs(*s) >= fabs(x)) *c += (*s - t) + x;
    else *c += (x - t) + *s;
    *s = t;
}

#define EPS0_SI 8.8541878128e-12 /* CODATA 2018 vacuum permittivity, F/m */

static double coulomb_k(double eps0)
{
    if (!(eps0 > 0.0)) eps0 = EPS0_SI;
    return 1.0 / (4.0 * M_PI * eps0);
}

/* ------------------------------------------------------------------ */
/* Public entry points (ctypes)                                         */
/* ------------------------------------------------------------------ */

/* method codes for single-element and field evaluations */
#define OR_METHOD_PAPER 0    /* rule bands + analytic near field (the method) */
#define OR_METHOD_GL2 1      /* GL2 with n nodes per dimension */
#define OR_METHOD_ANALYTIC 2 /* analytic everywhere */
#define OR_METHOD_RULE 3     /* one fixed cubature rule (param = rule index) */
#define OR_METHOD_SUBDIV 4   /* 2^param x 2^param pieces, 16 x 16 GL2 on each */

int oracle_rule(int type, int rule, double* nodes /* 33 x 4 */)
{
    const rule_t* r;
    int i;
    build_rules();
    if (type < 0 || type > 1 || rule < 0 || rule > 4) return -1;
    r = type == 0 ? &TRI[rule] : &RECT[rule];
    for (i = 0; i < r->n; ++i) {
        nodes[4 * i + 0] = r->a[i];
        nodes[4 * i + 1] = r->b[i];
        nodes[4 * i + 2] = r->c[i];
        nodes[4 * i + 3] = r->w[i];
    }
    return r->n;
}

void oracle_gauss_legendre(int n, double* x, double* w) { gauss_legendre(n, x, w); }

void oracle_default_limits(double* out /* 10 */)
{
    int t, k;
    for (t = 0; t < 2; ++t)
        for (k = 0; k < 5; ++k) out[5 * t + k] = DEFAULT_LIMITS[t][k];
}

/* centroid (3), L, area of one element */
void oracle_element_geometry(int type, const double* verts, double* out /* 5 */)
{
    elem_t e;
    elem_setup(&e, type, verts);
    out[0] = e.cen[0]; out[1] = e.cen[1]; out[2] = e.cen[2];
    out[3] = e.L;
    out[4] = e.area;
}

/* phi and E of ONE element with sigma = 1 and without 1/(4 pi eps0) */
int oracle_element(int type, const double* verts, const double* P, int method, int param,
                   const double* limits, double* out /* 4 */, int* band_out)
{
    elem_t e;
    int band = -1;
    build_rules();
    elem_setup(&e, type, verts);
    switch (method) {
    case OR_METHOD_PAPER:
        band = choose_band(&e, P, limits ? limits + 5 * type : DEFAULT_LIMITS[type], NULL);
        if (band == 0) analytic_field(&e, P, out);
        else cubature_field(&e, band - 1, P, out);
        break;
    case OR_METHOD_GL2:
        if (param < 1 || param > NGL_MAX) return -1;
        gl2_field(&e, param, P, out);
        break;
    case OR_METHOD_ANALYTIC:
        analytic_field(&e, P, out);
        break;
    case OR_METHOD_RULE:
        if (param < 0 || param > 4) return -1;
        cubature_field(&e, param, P, out);
        break;
    case OR_METHOD_SUBDIV:
        if (param < 0 || param > 12) return -1;
        subdiv_field(&e, param, 16, P, out);
        break;
    default:
        return -1;
    }
    if (band_out) *band_out = band;
    return 0;
}

/* phi and E at n_pts field points, summed over n_el elements in index
 * order (Sec. 5), each element with constant sigma, times 1/(4 pi eps0).
 *   verts:  n_el x 4 x 3 (triangles use the first three corners)
 *   method: OR_METHOD_PAPER (the method) or OR_METHOD_GL2 (param nodes)
 *   hist:   optional 2 x 6 pair counts per (type, band) -- band 0 is the
 *           analytic branch, band 1 + r is cubature rule r
 *   min_dr: optional per-point minimum distance ratio over all elements
 *   esum:   optional per-point sum over elements of |E_j| (times
 *           1/(4 pi eps0)); esum / |E| is the condition number of the field
 *           sum, the factor by which cancellation magnifies rounding
 */
int oracle_eval(int64_t n_el, const int32_t* type, const double* verts, const double* sigma,
                const double* limits, double eps0, int64_t n_pts, const double* pts,
                double* phi, double* E, int method, int param, int nthreads,
                int64_t* hist, double* min_dr, double* esum)
{
    const double kc = coulomb_k(eps0);
    int64_t p, j;
    int64_t hist_local[12];
    build_rules();
    if (n_el < 0 || n_pts < 0) return -1;
    for (j = 0; j < n_el; ++j)
        if (type[j] != 0 && type[j] != 1) return -1;
    memset(hist_local, 0, sizeof hist_local);
    if (nthreads < 1) nthreads = 1;

#pragma omp parallel num_threads(nthreads)
    {
        int64_t h_thr[12];
        memset(h_thr, 0, sizeof h_thr);
#pragma omp for schedule(dynamic, 4)
        for (p = 0; p < n_pts; ++p) {
            const double* P = pts + 3 * p;
            double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0}, mdr = INFINITY, eabs = 0.0;
            int64_t jj;
            int k;
            for (jj = 0; jj < n_el; ++jj) {
                elem_t e;
                double f[4], dr;
                elem_setup(&e, type[jj], verts + 12 * jj);
                if (method == OR_METHOD_GL2) {
                    gl2_field(&e, param, P, f);
                    {
                        double d[3];
                        sub3(P, e.cen, d);
                        dr = norm3(d) / e.L;
                    }
                } else {
                    const int band = choose_band(&e, P, limits ? limits + 5 * type[jj] : DEFAULT_LIMITS[type[jj]], &dr);
                    if (band == 0) analytic_field(&e, P, f);
                    else cubature_field(&e, band - 1, P, f);
                    h_thr[6 * type[jj] + band]++;
                }
                if (dr < mdr) mdr = dr;
                for (k = 0; k < 4; ++k) nsum_add(&s[k], &c[k], sigma[jj] * f[k]);
                eabs += fabs(sigma[jj]) * sqrt(f[1] * f[1] + f[2] * f[2] + f[3] * f[3]);
            }
            phi[p] = kc * (s[0] + c[0]);
            for (k = 0; k < 3; ++k) E[3 * p + k] = kc * (s[k + 1] + c[k + 1]);
            if (min_dr) min_dr[p] = mdr;
            if (esum) esum[p] = kc * eabs;
        }
#pragma omp critical
        for (j = 0; j < 12; ++j) hist_local[j] += h_thr[j];
    }
    if (hist)
        for (j = 0; j < 12; ++j) hist[j] = hist_local[j];
    return 0;
}

/* BEM collocation coefficients (the sigma-to-potential matrix of the
 * charge-density solve that the paper's BEM context describes, Sec. 5):
 * A[i][j] = potential at colloc point i of element j with sigma = 1, by the
 * same rule bands and analytic near field, times 1/(4 pi eps0).
 * rows [row0, row0 + n_rows) only; A is n_rows x n_el, row-major. */
int oracle_assemble(int64_t n_el, const int32_t* type, const double* verts, const double* limits,
                    double eps0, int64_t row0, int64_t n_rows, const double* colloc, double* A,
                    int nthreads)
{
    const double kc = coulomb_k(eps0);
    int64_t i;
    build_rules();
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
    for (i = 0; i < n_rows; ++i) {
        const double* P = colloc + 3 * (row0 + i);
        int64_t j;
        for (j = 0; j < n_el; ++j) {
            elem_t e;
            double f[4];
            int band;
            elem_setup(&e, type[j], verts + 12 * j);
            band = choose_band(&e, P, limits ? limits + 5 * type[j] : DEFAULT_LIMITS[type[j]], NULL);
            if (band == 0) analytic_field(&e, P, f);
            else cubature_field(&e, band - 1, P, f);
            A[i * n_el + j] = kc * f[0];
        }
    }
    return 0;
}

int oracle_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* oracle_element for n independent (element, point) pairs: verts n x 4 x 3,
 * P n x 3, out n x 4 (used by the distance-ratio experiment of Sec. 4) */
int oracle_element_batch(int64_t n, const int32_t* type, const double* verts, const double* P, int method,
                         int param, const double* limits, double* out, int32_t* band, int nthreads)
{
    int64_t i;
    int bad = 0;
    build_rules();
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(static) num_threads(nthreads) reduction(| : bad)
    for (i = 0; i < n; ++i) {
        int b = -1;
        if (oracle_element(type[i], verts + 12 * i, P + 3 * i, method, param, limits, out + 4 * i, &b) != 0) bad |= 1;
        if (band) band[i] = b;
    }
    return bad ? -1 : 0;
}

/* ------------------------------------------------------------------ */
/* Field gradient dE_i / dx_j, output as (xx, yy, zz, xy, xz, yz), unit  */
/* sigma, without 1/(4 pi eps0).                                        */
/*                                                                      */
/* Sec. 7 notes that point charges give higher derivatives of the field */
/* directly: a charge q at Q adds q (delta_ij / r^3 - 3 r_i r_j / r^5)  */
/* with r = P - Q.  The analytic branch differentiates the near-field    */
/* decomposition E = sum_e m_e l_e + n Omega used above: the gradient of */
/* the edge integral l_e is -J_e, J_e = int_e (P - Q) / R^3 ds (the     */
/* field of the edge as a unit line charge), and the gradient of the    */
/* solid angle is -sum_e t_e x J_e (the Biot-Savart field of the         */
/* boundary), so                                                        */
/*   dE_i / dx_j = - sum_e m_e,i J_e,j - n_i (sum_e t_e x J_e)_j .      */
/* ------------------------------------------------------------------ */
static void charge_grad(double q, const double r[3], double g[6])
{
    const double r2 = dot3(r, r), inv = 1.0 / sqrt(r2);
    const double inv3 = inv * inv * inv, c = 3.0 * q * inv3 / r2;
    g[0] += q * inv3 - c * r[0] * r[0];
    g[1] += q * inv3 - c * r[1] * r[1];
    g[2] += q * inv3 - c * r[2] * r[2];
    g[3] -= c * r[0] * r[1];
    g[4] -= c * r[0] * r[2];
    g[5] -= c * r[1] * r[2];
}

static void cubature_grad(const elem_t* e, int rule, const double P[3], double g[6])
{
    const rule_t* r = e->type == 0 ? &TRI[rule] : &RECT[rule];
    int i;
    for (i = 0; i < 6; ++i) g[i] = 0.0;
    for (i = 0; i < r->n; ++i) {
        double Q[3], d[3];
        rule_node(e, r, i, Q);
        sub3(P, Q, d);
        charge_grad(r->w[i] * e->area, d, g);
    }
}

static void gl2_grad(const elem_t* e, int n, const double P[3], double g[6])
{
    double x[NGL_MAX], w[NGL_MAX];
    int i, j, k;
    gauss_legendre(n, x, w);
    for (k = 0; k < 6; ++k) g[k] = 0.0;
    for (i = 0; i < n; ++i) {
        for (j = 0; j < n; ++j) {
            double Q[3], d[3], wt;
            if (e->type == 1) {
                for (k = 0; k < 3; ++k)
                    Q[k] = e->cen[k] + 0.5 * e->a * x[i] * e->ux[k] + 0.5 * e->b * x[j] * e->uy[k];
                wt = w[i] * w[j] * e->a * e->b / 4.0;
            } else {
                const double u = 0.5 * (x[i] + 1.0), v = 0.5 * (x[j] + 1.0);
                for (k = 0; k < 3; ++k)
                    Q[k] = e->v[0][k] + u * (e->v[1][k] - e->v[0][k]) + u * v * (e->v[2][k] - e->v[1][k]);
                wt = 0.25 * w[i] * w[j] * 2.0 * e->area * u;
            }
            sub3(P, Q, d);
            charge_grad(wt, d, g);
        }
    }
}

/* J = int over the edge V1 -> V2 of (P - Q) / R^3 ds.  With t the unit
 * tangent, u_k = (V_k - P)·t and rho = (V1 - P) - u1 t (from P to the edge
 * line, perpendicular):  J = -rho (u2/R2 - u1/R1) / |rho|^2 + t (1/R2 - 1/R1).
 * The two differences are rewritten as quotients without cancellation; a
 * point on the closed edge (a singularity of the edge's field) gives 0. */
static void edge_line_field(const double V1[3], const double V2[3], const double P[3], double J[3])
{
    double t[3], r1[3], r2[3], rho[3], len, u1, u2, R1, R2, rho2, f, g;
    int k;
    sub3(V2, V1, t);
    len = norm3(t);
    for (k = 0; k < 3; ++k) t[k] /= len;
    sub3(V1, P, r1);
    sub3(V2, P, r2);
    u1 = dot3(r1, t);
    u2 = dot3(r2, t);
    R1 = norm3(r1);
    R2 = norm3(r2);
    for (k = 0; k < 3; ++k) rho[k] = r1[k] - u1 * t[k];
    rho2 = dot3(rho, rho);
    J[0] = J[1] = J[2] = 0.0;
    if (R1 == 0.0 || R2 == 0.0) return;
    if (u1 >= 0.0) {        /* the edge lies ahead of the foot of the perpendicular */
        f = (u2 - u1) * (u2 + u1) / (R1 * R2 * (u2 * R1 + u1 * R2));
    } else if (u2 <= 0.0) { /* ... or behind it */
        f = (u1 - u2) * (u1 + u2) / (R1 * R2 * (-u1 * R2 - u2 * R1));
    } else {                /* the foot lies on the edge */
        if (rho2 == 0.0) return;
        f = (u2 / R2 - u1 / R1) / rho2;
    }
    g = (u1 - u2) * (u1 + u2) / (R1 * R2 * (R1 + R2)); /* 1/R2 - 1/R1 */
    for (k = 0; k < 3; ++k) J[k] = -rho[k] * f + t[k] * g;
}

static void analytic_grad(const elem_t* e, const double P[3], double g[6])
{
    const int nv = e->type == 0 ? 3 : 4;
    double n[3], e1[3], e2[3], nl, G[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, gw[3] = {0, 0, 0};
    int j, a, b;
    sub3(e->v[1], e->v[0], e1);
    sub3(e->v[2], e->v[0], e2);
    cross3(e1, e2, n);
    nl = norm3(n);
    for (a = 0; a < 3; ++a) n[a] /= nl;
    for (j = 0; j < nv; ++j) {
        const double* V1 = e->v[j];
        const double* V2 = e->v[(j + 1) % nv];
        double t[3], m[3], J[3], tj[3], len;
        sub3(V2, V1, t);
        len = norm3(t);
        for (a = 0; a < 3; ++a) t[a] /= len;
        cross3(t, n, m);
        edge_line_field(V1, V2, P, J);
        for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b) G[a][b] -= m[a] * J[b];
        cross3(t, J, tj);
        for (a = 0; a < 3; ++a) gw[a] += tj[a];
    }
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) G[a][b] -= n[a] * gw[b];
    g[0] = G[0][0]; g[1] = G[1][1]; g[2] = G[2][2];
    g[3] = G[0][1]; g[4] = G[0][2]; g[5] = G[1][2];
}

/* gradient of ONE element, sigma = 1, without 1/(4 pi eps0); methods as
 * oracle_element (SUBDIV not offered) */
int oracle_element_grad(int type, const double* verts, const double* P, int method, int param,
                        const double* limits, double* out /* 6 */, int* band_out)
{
    elem_t e;
    int band = -1;
    build_rules();
    elem_setup(&e, type, verts);
    switch (method) {
    case OR_METHOD_PAPER:
        band = choose_band(&e, P, limits ? limits + 5 * type : DEFAULT_LIMITS[type], NULL);
        if (band == 0) analytic_grad(&e, P, out);
        else cubature_grad(&e, band - 1, P, out);
        break;
    case OR_METHOD_GL2:
        if (param < 1 || param > NGL_MAX) return -1;
        gl2_grad(&e, param, P, out);
        break;
    case OR_METHOD_ANALYTIC:
        analytic_grad(&e, P, out);
        break;
    case OR_METHOD_RULE:
        if (param < 0 || param > 4) return -1;
        cubature_grad(&e, param, P, out);
        break;
    default:
        return -1;
    }
    if (band_out) *band_out = band;
    return 0;
}

/* field gradient at n_pts points, summed over all elements in index order
 * by the method (rule bands, analytic near field), times 1/(4 pi eps0);
 * G is n_pts x 6 (xx, yy, zz, xy, xz, yz) */
/* gsum (optional, n_pts): the sum over elements of the largest |component|
 * of each element's contribution, times 1/(4 pi eps0): the scale against
 * which cancellation in G is measured */
int oracle_eval_grad(int64_t n_el, const int32_t* type, const double* verts, const double* sigma,
                     const double* limits, double eps0, int64_t n_pts, const double* pts, double* G, double* gsum,
                     int nthreads)
{
    const double kc = coulomb_k(eps0);
    int64_t p, j;
    build_rules();
    if (n_el < 0 || n_pts < 0) return -1;
    for (j = 0; j < n_el; ++j)
        if (type[j] != 0 && type[j] != 1) return -1;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (p = 0; p < n_pts; ++p) {
        const double* P = pts + 3 * p;
        double s[6] = {0, 0, 0, 0, 0, 0}, c[6] = {0, 0, 0, 0, 0, 0}, am = 0.0;
        int64_t jj;
        int k;
        for (jj = 0; jj < n_el; ++jj) {
            elem_t e;
            double f[6], mx = 0.0;
            int band;
            elem_setup(&e, type[jj], verts + 12 * jj);
            band = choose_band(&e, P, limits ? limits + 5 * type[jj] : DEFAULT_LIMITS[type[jj]], NULL);
            if (band == 0) analytic_grad(&e, P, f);
            else cubature_grad(&e, band - 1, P, f);
            for (k = 0; k < 6; ++k) {
                nsum_add(&s[k], &c[k], sigma[jj] * f[k]);
                if (fabs(sigma[jj] * f[k]) > mx) mx = fabs(sigma[jj] * f[k]);
            }
            am += mx;
        }
        for (k = 0; k < 6; ++k) G[6 * p + k] = kc * (s[k] + c[k]);
        if (gsum) gsum[p] = kc * am;
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Linear charge density (Sec. 7: the cubature applies unchanged to     */
/* non-constant densities; the paper treats constant ones).             */
/*                                                                      */
/* sigma(Q) = s_c + s_a alpha + s_b beta, with (alpha, beta) the         */
/* element's coordinates Q - Q_cen = alpha e0 + beta e1 (triangle: e0 =  */
/* A - Q_cen, e1 = B - Q_cen, i.e. alpha = lambda_A - lambda_C, beta =   */
/* lambda_B - lambda_C of Eq. 3.3; rectangle: e0 = (a/2) u_x, e1 =        */
/* (b/2) u_y, i.e. the natural coordinates x, y of Eq. 3.2).  Written as */
/* sigma(Q) = s_c + g·(Q - Q_cen) with g = s_a grad(alpha) + s_b         */
/* grad(beta), the in-plane dual vectors of e0, e1.                      */
/* ------------------------------------------------------------------ */
typedef struct {
    double sc, g[3], C[3];
    double H[3][3]; /* quadratic densities: the in-plane Hessian (0 for linear ones) */
} lin_t;

static void linear_density(const elem_t* e, const double* coef, lin_t* s)
{
    double e0[3], e1[3], g00, g01, g11, det, d0[3], d1[3];
    int k;
    if (e->type == 0) {
        sub3(e->v[0], e->cen, e0);
        sub3(e->v[1], e->cen, e1);
    } else {
        for (k = 0; k < 3; ++k) {
            e0[k] = 0.5 * e->a * e->ux[k];
            e1[k] = 0.5 * e->b * e->uy[k];
        }
    }
    g00 = dot3(e0, e0);
    g01 = dot3(e0, e1);
    g11 = dot3(e1, e1);
    det = g00 * g11 - g01 * g01;
    for (k = 0; k < 3; ++k) {
        d0[k] = (g11 * e0[k] - g01 * e1[k]) / det; /* grad(alpha) */
        d1[k] = (g00 * e1[k] - g01 * e0[k]) / det; /* grad(beta) */
    }
    s->sc = coef[0];
    for (k = 0; k < 3; ++k) {
        s->g[k] = coef[1] * d0[k] + coef[2] * d1[k];
        s->C[k] = e->cen[k];
    }
    memset(s->H, 0, sizeof s->H);
}

/* quadratic density sigma = c0 + c1 alpha + c2 beta + c3 alpha^2 + c4 alpha beta
 * + c5 beta^2: with grad(alpha) = d0, grad(beta) = d1 the Hessian in space is
 * H = 2 c3 d0 d0^T + c4 (d0 d1^T + d1 d0^T) + 2 c5 d1 d1^T */
static void quadratic_density(const elem_t* e, const double* coef, lin_t* s)
{
    double e0[3], e1[3], g00, g01, g11, det, d0[3], d1[3];
    int a, b;
    linear_density(e, coef, s);
    if (e->type == 0) {
        sub3(e->v[0], e->cen, e0);
        sub3(e->v[1], e->cen, e1);
    } else {
        for (a = 0; a < 3; ++a) {
            e0[a] = 0.5 * e->a * e->ux[a];
            e1[a] = 0.5 * e->b * e->uy[a];
        }
    }
    g00 = dot3(e0, e0);
    g01 = dot3(e0, e1);
    g11 = dot3(e1, e1);
    det = g00 * g11 - g01 * g01;
    for (a = 0; a < 3; ++a) {
        d0[a] = (g11 * e0[a] - g01 * e1[a]) / det;
        d1[a] = (g00 * e1[a] - g01 * e0[a]) / det;
    }
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b)
            s->H[a][b] = 2.0 * coef[3] * d0[a] * d0[b] + coef[4] * (d0[a] * d1[b] + d1[a] * d0[b]) +
                         2.0 * coef[5] * d1[a] * d1[b];
}

static double quad_form(const double H[3][3], const double x[3], const double y[3])
{
    int a, b;
    double r = 0.0;
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) r += x[a] * H[a][b] * y[b];
    return r;
}

static double lin_sigma(const lin_t* s, const double Q[3])
{
    double d[3];
    sub3(Q, s->C, d);
    return s->sc + dot3(s->g, d) + 0.5 * quad_form(s->H, d, d);
}

/* Eq. 4.1 with q_i = w_i area sigma(Q_i) */
static void cubature_field_lin(const elem_t* e, int rule, const double P[3], const lin_t* s, double out[4])
{
    const rule_t* r = e->type == 0 ? &TRI[rule] : &RECT[rule];
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    int i, k;
    for (i = 0; i < r->n; ++i) {
        double Q[3], d[3], dist, qi;
        rule_node(e, r, i, Q);
        sub3(P, Q, d);
        dist = norm3(d);
        qi = r->w[i] * e->area * lin_sigma(s, Q);
        acc[0] += qi / dist;
        for (k = 0; k < 3; ++k) acc[k + 1] += qi * d[k] / (dist * dist * dist);
    }
    for (k = 0; k < 4; ++k) out[k] = acc[k];
}

static void gl2_field_lin(const elem_t* e, int n, const double P[3], const lin_t* s, double out[4])
{
    double x[NGL_MAX], w[NGL_MAX], acc[4] = {0.0, 0.0, 0.0, 0.0};
    int i, j, k;
    gauss_legendre(n, x, w);
    for (i = 0; i < n; ++i) {
        for (j = 0; j < n; ++j) {
            double Q[3], d[3], dist, wt;
            if (e->type == 1) {
                for (k = 0; k < 3; ++k)
                    Q[k] = e->cen[k] + 0.5 * e->a * x[i] * e->ux[k] + 0.5 * e->b * x[j] * e->uy[k];
                wt = w[i] * w[j] * e->a * e->b / 4.0;
            } else {
                const double u = 0.5 * (x[i] + 1.0), v = 0.5 * (x[j] + 1.0);
                for (k = 0; k < 3; ++k)
                    Q[k] = e->v[0][k] + u * (e->v[1][k] - e->v[0][k]) + u * v * (e->v[2][k] - e->v[1][k]);
                wt = 0.25 * w[i] * w[j] * 2.0 * e->area * u;
            }
            wt *= lin_sigma(s, Q);
            sub3(P, Q, d);
            dist = norm3(d);
            acc[0] += wt / dist;
            for (k = 0; k < 3; ++k) acc[k + 1] += wt * d[k] / (dist * dist * dist);
        }
    }
    for (k = 0; k < 4; ++k) out[k] = acc[k];
}

/* brute force as subdiv_field, with the parent element's density */
static void subdiv_field_lin(const elem_t* e, int level, int n, const double P[3], const lin_t* s, double out[4])
{
    int k, c;
    if (level == 0) {
        gl2_field_lin(e, n, P, s, out);
        return;
    }
    for (k = 0; k < 4; ++k) out[k] = 0.0;
    if (e->type == 0) {
        double m01[3], m12[3], m20[3], tris[4][4][3], part[4];
        int t;
        for (k = 0; k < 3; ++k) {
            m01[k] = 0.5 * (e->v[0][k] + e->v[1][k]);
            m12[k] = 0.5 * (e->v[1][k] + e->v[2][k]);
            m20[k] = 0.5 * (e->v[2][k] + e->v[0][k]);
        }
        for (k = 0; k < 3; ++k) {
            tris[0][0][k] = e->v[0][k]; tris[0][1][k] = m01[k];     tris[0][2][k] = m20[k];
            tris[1][0][k] = m01[k];     tris[1][1][k] = e->v[1][k]; tris[1][2][k] = m12[k];
            tris[2][0][k] = m20[k];     tris[2][1][k] = m12[k];     tris[2][2][k] = e->v[2][k];
            tris[3][0][k] = m12[k];     tris[3][1][k] = m20[k];     tris[3][2][k] = m01[k];
            for (c = 0; c < 4; ++c) tris[c][3][k] = 0.0;
        }
        for (t = 0; t < 4; ++t) {
            elem_t sub;
            elem_setup(&sub, 0, &tris[t][0][0]);
            subdiv_field_lin(&sub, level - 1, n, P, s, part);
            for (c = 0; c < 4; ++c) out[c] += part[c];
        }
    } else {
        int qx, qy;
        for (qx = 0; qx < 2; ++qx) {
            for (qy = 0; qy < 2; ++qy) {
                double corners[4][3], part[4];
                const double x0 = qx - 1.0, y0 = qy - 1.0;
                const double xs[4] = {x0, x0 + 1.0, x0 + 1.0, x0};
                const double ys[4] = {y0, y0, y0 + 1.0, y0 + 1.0};
                elem_t sub;
                for (c = 0; c < 4; ++c)
                    for (k = 0; k < 3; ++k)
                        corners[c][k] = e->cen[k] + 0.5 * e->a * xs[c] * e->ux[k] + 0.5 * e->b * ys[c] * e->uy[k];
                elem_setup(&sub, 1, &corners[0][0]);
                subdiv_field_lin(&sub, level - 1, n, P, s, part);
                for (c = 0; c < 4; ++c) out[c] += part[c];
            }
        }
    }
}

/* Analytic near field for the linear density.  With P' the foot of P in
 * the element plane (P = P' + h n) and w = Q - P', sigma(Q) = sigma(P') +
 * g·w, and
 *   int sigma / R dA = sigma(P') I0 + g · int w / R dA
 *   int w / R dA     = sum_e m_e int_e R ds          (in-plane grad R = w / R)
 *   int_e R ds       = (s2 R2 - s1 R1 + rho_e^2 l_e) / 2,  rho_e^2 = d_e^2 + h^2
 *   int sigma (P - Q) / R^3 dA = sigma(P') E0 + h n (g · int w / R^3 dA)
 *                                - (int w w^T / R^3 dA) g
 *   int w / R^3 dA      = - sum_e m_e l_e           (grad (1/R) = -w / R^3)
 *   int w w^T / R^3 dA  = Pi I0 - sum_e (int_e w / R ds) m_e^T,
 *   int_e w / R ds      = d_e l_e m_e + (R2 - R1) t_e
 * (the divergence theorem in the plane on w / R; Pi the in-plane
 * projector), where I0, E0 are the constant-density results of
 * analytic_field and d_e, l_e, s_k, R_k, m_e, t_e are as defined there. */
static void analytic_field_lin(const elem_t* e, const double P[3], const lin_t* s, double out[4])
{
    const int nv = e->type == 0 ? 3 : 4;
    double f0[4], n[3], e1[3], e2[3], nl, h, Pp[3], sP, I1[3] = {0.0, 0.0, 0.0}, Ec[3], hsum = 0.0;
    int k, j;
    analytic_field(e, P, f0);
    sub3(e->v[1], e->v[0], e1);
    sub3(e->v[2], e->v[0], e2);
    cross3(e1, e2, n);
    nl = norm3(n);
    for (k = 0; k < 3; ++k) n[k] /= nl;
    {
        double pv[3];
        sub3(P, e->v[0], pv);
        h = dot3(pv, n);
    }
    for (k = 0; k < 3; ++k) Pp[k] = P[k] - h * n[k];
    sP = lin_sigma(s, Pp);
    for (k = 0; k < 3; ++k) Ec[k] = -s->g[k] * f0[0];
    for (j = 0; j < nv; ++j) {
        const double* V1 = e->v[j];
        const double* V2 = e->v[(j + 1) % nv];
        double t[3], m[3], r1[3], r2[3], len, s1, s2, R1, R2, d, perp2, l, gm;
        sub3(V2, V1, t);
        len = norm3(t);
        for (k = 0; k < 3; ++k) t[k] /= len;
        cross3(t, n, m);
        sub3(V1, P, r1);
        sub3(V2, P, r2);
        s1 = dot3(r1, t);
        s2 = dot3(r2, t);
        R1 = norm3(r1);
        R2 = norm3(r2);
        d = dot3(r1, m);
        perp2 = d * d + h * h;
        l = edge_log(s1, s2, R1, R2, perp2);
        for (k = 0; k < 3; ++k) I1[k] += m[k] * 0.5 * (s2 * R2 - s1 * R1 + perp2 * l);
        gm = dot3(s->g, m);
        hsum += gm * l;
        for (k = 0; k < 3; ++k) Ec[k] += gm * (d * l * m[k] + (R2 - R1) * t[k]);
    }
    out[0] = sP * f0[0] + dot3(s->g, I1);
    for (k = 0; k < 3; ++k) out[k + 1] = sP * f0[k + 1] - h * n[k] * hsum + Ec[k];
}

/* phi and E of ONE element with linear density coef = (s_c, s_a, s_b),
 * without 1/(4 pi eps0); methods as oracle_element */
int oracle_element_linear(int type, const double* verts, const double* coef, const double* P, int method, int param,
                          const double* limits, double* out /* 4 */, int* band_out)
{
    elem_t e;
    lin_t s;
    int band = -1;
    build_rules();
    elem_setup(&e, type, verts);
    linear_density(&e, coef, &s);
    switch (method) {
    case OR_METHOD_PAPER:
        band = choose_band(&e, P, limits ? limits + 5 * type : DEFAULT_LIMITS[type], NULL);
        if (band == 0) analytic_field_lin(&e, P, &s, out);
        else cubature_field_lin(&e, band - 1, P, &s, out);
        break;
    case OR_METHOD_GL2:
        if (param < 1 || param > NGL_MAX) return -1;
        gl2_field_lin(&e, param, P, &s, out);
        break;
    case OR_METHOD_ANALYTIC:
        analytic_field_lin(&e, P, &s, out);
        break;
    case OR_METHOD_RULE:
        if (param < 0 || param > 4) return -1;
        cubature_field_lin(&e, param, P, &s, out);
        break;
    case OR_METHOD_SUBDIV:
        if (param < 0 || param > 12) return -1;
        subdiv_field_lin(&e, param, 16, P, &s, out);
        break;
    default:
        return -1;
    }
    if (band_out) *band_out = band;
    return 0;
}

/* phi and E at n_pts points for elements with linear densities coef
 * (n_el x 3), by the method, summed in index order, times 1/(4 pi eps0) */
int oracle_eval_linear(int64_t n_el, const int32_t* type, const double* verts, const double* coef,
                       const double* limits, double eps0, int64_t n_pts, const double* pts, double* phi, double* E,
                       int nthreads)
{
    const double kc = coulomb_k(eps0);
    int64_t p, j;
    build_rules();
    if (n_el < 0 || n_pts < 0) return -1;
    for (j = 0; j < n_el; ++j)
        if (type[j] != 0 && type[j] != 1) return -1;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (p = 0; p < n_pts; ++p) {
        const double* P = pts + 3 * p;
        double sm[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
        int64_t jj;
        int k;
        for (jj = 0; jj < n_el; ++jj) {
            elem_t e;
            lin_t s;
            double f[4];
            int band;
            elem_setup(&e, type[jj], verts + 12 * jj);
            linear_density(&e, coef + 3 * jj, &s);
            band = choose_band(&e, P, limits ? limits + 5 * type[jj] : DEFAULT_LIMITS[type[jj]], NULL);
            if (band == 0) analytic_field_lin(&e, P, &s, f);
            else cubature_field_lin(&e, band - 1, P, &s, f);
            for (k = 0; k < 4; ++k) nsum_add(&sm[k], &c[k], f[k]);
        }
        phi[p] = kc * (sm[0] + c[0]);
        for (k = 0; k < 3; ++k) E[3 * p + k] = kc * (sm[k + 1] + c[k + 1]);
    }
    return 0;
}

/* Analytic near field for the quadratic density sigma(Q) = sigma(P') + g·w +
 * w^T H w / 2 (w = Q - P', P' the foot of P in the plane, g and H the
 * gradient and Hessian there).  Besides the integrals of the linear case:
 *   int w w^T / R dA   = sum_e (d_e J_e m_e + (R2^3 - R1^3)/3 t_e) m_e^T - Pi int R dA
 *   int R dA           = (sum_e d_e J_e + h^2 I0) / 3,      J_e = int_e R ds
 *   int (w^T H w) w / R^3 dA = 2 H int w / R dA - sum_e m_e int_e (w^T H w) / R ds
 *   int_e (w^T H w) / R ds = d_e^2 m^T H m l_e + 2 d_e m^T H t (R2 - R1)
 *                            + t^T H t (s2 R2 - s1 R1 - rho_e^2 l_e) / 2
 * (the in-plane divergence theorem on w R, w_i w_j / R and the edge
 * parametrisation w = d_e m_e + u t_e), so that
 *   phi = sigma(P') I0 + g·I1 + (H : I2) / 2
 *   E   = sigma(P') E0 + [h n (g·K1) - K2 g] + [h n (H : K2) - T] / 2
 * with I1 = int w / R, I2 = int w w^T / R, K1 = int w / R^3, K2 = int w w^T / R^3,
 * T = int (w^T H w) w / R^3 (all dA). */
static void analytic_field_quad(const elem_t* e, const double P[3], const lin_t* s, double out[4])
{
    const int nv = e->type == 0 ? 3 : 4;
    double f0[4], n[3], e1[3], e2[3], nl, h, Pp[3], dl[3], sP, g[3], I1[3] = {0, 0, 0};
    double K2[3][3], I2[3][3], Qm[3] = {0, 0, 0}, sumdJ = 0.0, hsum = 0.0, intR, HI2 = 0.0, HK2 = 0.0, T[3];
    int k, j, a, b;
    analytic_field(e, P, f0);
    sub3(e->v[1], e->v[0], e1);
    sub3(e->v[2], e->v[0], e2);
    cross3(e1, e2, n);
    nl = norm3(n);
    for (k = 0; k < 3; ++k) n[k] /= nl;
    {
        double pv[3];
        sub3(P, e->v[0], pv);
        h = dot3(pv, n);
    }
    for (k = 0; k < 3; ++k) Pp[k] = P[k] - h * n[k];
    sub3(Pp, s->C, dl);
    sP = s->sc + dot3(s->g, dl) + 0.5 * quad_form(s->H, dl, dl);
    for (a = 0; a < 3; ++a) {
        g[a] = s->g[a];
        for (b = 0; b < 3; ++b) g[a] += s->H[a][b] * dl[b];
    }
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) {
            const double pi = (a == b ? 1.0 : 0.0) - n[a] * n[b];
            K2[a][b] = pi * f0[0];
            I2[a][b] = 0.0;
        }
    for (j = 0; j < nv; ++j) {
        const double* V1 = e->v[j];
        const double* V2 = e->v[(j + 1) % nv];
        double t[3], m[3], r1[3], r2[3], len, s1, s2, R1, R2, d, perp2, l, J, wR[3], cub, Qe;
        sub3(V2, V1, t);
        len = norm3(t);
        for (k = 0; k < 3; ++k) t[k] /= len;
        cross3(t, n, m);
        sub3(V1, P, r1);
        sub3(V2, P, r2);
        s1 = dot3(r1, t);
        s2 = dot3(r2, t);
        R1 = norm3(r1);
        R2 = norm3(r2);
        d = dot3(r1, m);
        perp2 = d * d + h * h;
        l = edge_log(s1, s2, R1, R2, perp2);
        J = 0.5 * (s2 * R2 - s1 * R1 + perp2 * l);
        for (k = 0; k < 3; ++k) I1[k] += m[k] * J;
        sumdJ += d * J;
        for (k = 0; k < 3; ++k) wR[k] = d * l * m[k] + (R2 - R1) * t[k];
        cub = (R2 * R2 * R2 - R1 * R1 * R1) / 3.0;
        for (a = 0; a < 3; ++a)
            for (b = 0; b < 3; ++b) {
                K2[a][b] -= wR[a] * m[b];
                I2[a][b] += (d * J * m[a] + cub * t[a]) * m[b];
            }
        Qe = d * d * quad_form(s->H, m, m) * l + 2.0 * d * quad_form(s->H, m, t) * (R2 - R1) +
             quad_form(s->H, t, t) * 0.5 * (s2 * R2 - s1 * R1 - perp2 * l);
        for (k = 0; k < 3; ++k) Qm[k] += m[k] * Qe;
        hsum += dot3(g, m) * l;
    }
    intR = (sumdJ + h * h * f0[0]) / 3.0;
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) {
            I2[a][b] -= ((a == b ? 1.0 : 0.0) - n[a] * n[b]) * intR;
            HI2 += s->H[a][b] * I2[a][b];
            HK2 += s->H[a][b] * K2[a][b];
        }
    for (a = 0; a < 3; ++a) {
        T[a] = -Qm[a];
        for (b = 0; b < 3; ++b) T[a] += 2.0 * s->H[a][b] * I1[b];
    }
    out[0] = sP * f0[0] + dot3(g, I1) + 0.5 * HI2;
    for (a = 0; a < 3; ++a) {
        double Kg = 0.0;
        for (b = 0; b < 3; ++b) Kg += K2[a][b] * g[b];
        out[a + 1] = sP * f0[a + 1] - h * n[a] * hsum - Kg + 0.5 * (h * n[a] * HK2 - T[a]);
    }
}

/* phi and E of ONE element with the quadratic density coef = (c0, ..., c5),
 * sigma = c0 + c1 alpha + c2 beta + c3 alpha^2 + c4 alpha beta + c5 beta^2,
 * without 1/(4 pi eps0); methods as oracle_element */
int oracle_element_quad(int type, const double* verts, const double* coef, const double* P, int method, int param,
                        const double* limits, double* out /* 4 */, int* band_out)
{
    elem_t e;
    lin_t s;
    int band = -1;
    build_rules();
    elem_setup(&e, type, verts);
    quadratic_density(&e, coef, &s);
    switch (method) {
    case OR_METHOD_PAPER:
        band = choose_band(&e, P, limits ? limits + 5 * type : DEFAULT_LIMITS[type], NULL);
        if (band == 0) analytic_field_quad(&e, P, &s, out);
        else cubature_field_lin(&e, band - 1, P, &s, out);
        break;
    case OR_METHOD_GL2:
        if (param < 1 || param > NGL_MAX) return -1;
        gl2_field_lin(&e, param, P, &s, out);
        break;
    case OR_METHOD_ANALYTIC:
        analytic_field_quad(&e, P, &s, out);
        break;
    case OR_METHOD_RULE:
        if (param < 0 || param > 4) return -1;
        cubature_field_lin(&e, param, P, &s, out);
        break;
    case OR_METHOD_SUBDIV:
        if (param < 0 || param > 12) return -1;
        subdiv_field_lin(&e, param, 16, P, &s, out);
        break;
    default:
        return -1;
    }
    if (band_out) *band_out = band;
    return 0;
}

/* phi and E at n_pts points for elements with quadratic densities coef
 * (n_el x 6), by the method, summed in index order, times 1/(4 pi eps0) */
int oracle_eval_quad(int64_t n_el, const int32_t* type, const double* verts, const double* coef,
                     const double* limits, double eps0, int64_t n_pts, const double* pts, double* phi, double* E,
                     int nthreads)
{
    const double kc = coulomb_k(eps0);
    int64_t p, j;
    build_rules();
    if (n_el < 0 || n_pts < 0) return -1;
    for (j = 0; j < n_el; ++j)
        if (type[j] != 0 && type[j] != 1) return -1;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (p = 0; p < n_pts; ++p) {
        const double* P = pts + 3 * p;
        double sm[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
        int64_t jj;
        int k;
        for (jj = 0; jj < n_el; ++jj) {
            elem_t e;
            lin_t s;
            double f[4];
            int band;
            elem_setup(&e, type[jj], verts + 12 * jj);
            quadratic_density(&e, coef + 6 * jj, &s);
            band = choose_band(&e, P, limits ? limits + 5 * type[jj] : DEFAULT_LIMITS[type[jj]], NULL);
            if (band == 0) analytic_field_quad(&e, P, &s, f);
            else cubature_field_lin(&e, band - 1, P, &s, f);
            for (k = 0; k < 4; ++k) nsum_add(&sm[k], &c[k], f[k]);
        }
        phi[p] = kc * (sm[0] + c[0]);
        for (k = 0; k < 3; ++k) E[3 * p + k] = kc * (sm[k + 1] + c[k + 1]);
    }
    return 0;
}

/* ------------------------------------------------------------------ */
/* Field gradient for linear and quadratic densities.                   */
/*                                                                      */
/* The cubature branch takes q_i = w_i area sigma(Q_i) in the point-     */
/* charge derivative above.  The analytic branch moves the derivative   */
/* along an in-plane unit vector tau from the field point onto the      */
/* density (dK(P - Q)/dP = -dK(P - Q)/dQ for K(x) = x / |x|^3, then the  */
/* divergence theorem in the plane):                                    */
/*   dE/dtau = E[d sigma / dtau] - sum_e (tau·m_e) int_e sigma (P - Q) / R^3 ds */
/* where E[d sigma / dtau] is the field of the density d sigma / dtau    */
/* (constant for a linear sigma, linear for a quadratic one).  On an     */
/* edge, sigma = b0 + b1 s + b2 s^2 in the coordinate s along t_e from   */
/* the foot F of the perpendicular from P (P - Q = (P - F) - s t_e), so  */
/* the edge integral is                                                 */
/*   (P - F) (b0 M0 + b1 M1 + b2 M2) - t_e (b0 M1 + b1 M2 + b2 M3),     */
/*   M_k = int s^k / R^3 ds:  M0 = [s / (rho^2 R)], M1 = [-1/R],         */
/*   M2 = [ln(s + R) - s / R] = l_e - rho^2 M0, M3 = [R + rho^2 / R]     */
/* (rho = |P - F|).  The two in-plane columns of G follow; the normal    */
/* column from the symmetry of G and Laplace's equation (zero trace).    */
/* ------------------------------------------------------------------ */
static void cubature_grad_var(const elem_t* e, int rule, const double P[3], const lin_t* s, double g[6])
{
    const rule_t* r = e->type == 0 ? &TRI[rule] : &RECT[rule];
    int i;
    for (i = 0; i < 6; ++i) g[i] = 0.0;
    for (i = 0; i < r->n; ++i) {
        double Q[3], d[3];
        rule_node(e, r, i, Q);
        sub3(P, Q, d);
        charge_grad(r->w[i] * e->area * lin_sigma(s, Q), d, g);
    }
}

static void gl2_grad_var(const elem_t* e, int n, const double P[3], const lin_t* s, double g[6])
{
    double x[NGL_MAX], w[NGL_MAX];
    int i, j, k;
    gauss_legendre(n, x, w);
    for (k = 0; k < 6; ++k) g[k] = 0.0;
    for (i = 0; i < n; ++i) {
        for (j = 0; j < n; ++j) {
            double Q[3], d[3], wt;
            if (e->type == 1) {
                for (k = 0; k < 3; ++k)
                    Q[k] = e->cen[k] + 0.5 * e->a * x[i] * e->ux[k] + 0.5 * e->b * x[j] * e->uy[k];
                wt = w[i] * w[j] * e->a * e->b / 4.0;
            } else {
                const double u = 0.5 * (x[i] + 1.0), v = 0.5 * (x[j] + 1.0);
                for (k = 0; k < 3; ++k)
                    Q[k] = e->v[0][k] + u * (e->v[1][k] - e->v[0][k]) + u * v * (e->v[2][k] - e->v[1][k]);
                wt = 0.25 * w[i] * w[j] * 2.0 * e->area * u;
            }
            sub3(P, Q, d);
            charge_grad(wt * lin_sigma(s, Q), d, g);
        }
    }
}

/* int over the edge V1 -> V2 of sigma(Q) (P - Q) / R^3 ds for the density s */
static void edge_density_field(const double V1[3], const double V2[3], const double P[3], const lin_t* s,
                               double L[3])
{
    double t[3], r1[3], r2[3], rho[3], F[3], dF[3], gF[3], len, u1, u2, R1, R2, rho2, M0, M1, M2, M3, l, b0, b1, b2;
    int k, a;
    sub3(V2, V1, t);
    len = norm3(t);
    for (k = 0; k < 3; ++k) t[k] /= len;
    sub3(V1, P, r1);
    sub3(V2, P, r2);
    u1 = dot3(r1, t);
    u2 = dot3(r2, t);
    R1 = norm3(r1);
    R2 = norm3(r2);
    for (k = 0; k < 3; ++k) rho[k] = r1[k] - u1 * t[k]; /* F - P */
    rho2 = dot3(rho, rho);
    L[0] = L[1] = L[2] = 0.0;
    if (R1 == 0.0 || R2 == 0.0) return;
    if (u1 >= 0.0) {
        M0 = (u2 - u1) * (u2 + u1) / (R1 * R2 * (u2 * R1 + u1 * R2));
    } else if (u2 <= 0.0) {
        M0 = (u1 - u2) * (u1 + u2) / (R1 * R2 * (-u1 * R2 - u2 * R1));
    } else {
        if (rho2 == 0.0) return; /* on the closed edge */
        M0 = (u2 / R2 - u1 / R1) / rho2;
    }
    M1 = (u2 - u1) * (u2 + u1) / (R1 * R2 * (R1 + R2)); /* 1/R1 - 1/R2 */
    l = edge_log(u1, u2, R1, R2, rho2);
    M2 = l - rho2 * M0;
    M3 = (u2 - u1) * (u2 + u1) / (R1 + R2) - rho2 * M1; /* (R2 - R1) + rho^2 (1/R2 - 1/R1) */
    /* sigma along the edge about the foot F */
    for (k = 0; k < 3; ++k) F[k] = P[k] + rho[k];
    sub3(F, s->C, dF);
    for (a = 0; a < 3; ++a) {
        gF[a] = s->g[a];
        for (k = 0; k < 3; ++k) gF[a] += s->H[a][k] * dF[k];
    }
    b0 = lin_sigma(s, F);
    b1 = dot3(gF, t);
    b2 = 0.5 * quad_form(s->H, t, t);
    for (k = 0; k < 3; ++k)
        L[k] = -rho[k] * (b0 * M0 + b1 * M1 + b2 * M2) - t[k] * (b0 * M1 + b1 * M2 + b2 * M3);
}

static void analytic_grad_var(const elem_t* e, const double P[3], const lin_t* s, double g[6])
{
    const int nv = e->type == 0 ? 3 : 4;
    double n[3], e1[3], e2[3], nl, tau[2][3], col[3][3], G[3][3];
    int j, a, b, c;
    sub3(e->v[1], e->v[0], e1);
    sub3(e->v[2], e->v[0], e2);
    cross3(e1, e2, n);
    nl = norm3(n);
    for (a = 0; a < 3; ++a) n[a] /= nl;
    for (a = 0; a < 3; ++a) tau[0][a] = e1[a] / norm3(e1);
    cross3(n, tau[0], tau[1]);
    for (c = 0; c < 2; ++c) {
        /* E of the density d sigma / d tau = tau·g + (H tau)·(Q - C) */
        lin_t ds;
        double f[4];
        ds.sc = dot3(tau[c], s->g);
        for (a = 0; a < 3; ++a) {
            ds.g[a] = 0.0;
            for (b = 0; b < 3; ++b) ds.g[a] += s->H[a][b] * tau[c][b];
            ds.C[a] = s->C[a];
        }
        memset(ds.H, 0, sizeof ds.H);
        analytic_field_lin(e, P, &ds, f);
        for (a = 0; a < 3; ++a) col[c][a] = f[a + 1];
        for (j = 0; j < nv; ++j) {
            const double* V1 = e->v[j];
            const double* V2 = e->v[(j + 1) % nv];
            double t[3], m[3], L[3], len, tm;
            sub3(V2, V1, t);
            len = norm3(t);
            for (a = 0; a < 3; ++a) t[a] /= len;
            cross3(t, n, m);
            tm = dot3(tau[c], m);
            edge_density_field(V1, V2, P, s, L);
            for (a = 0; a < 3; ++a) col[c][a] -= tm * L[a];
        }
    }
    /* normal column: tau_k·(G n) = n·(G tau_k), n·(G n) = -(tau_1·G tau_1 + tau_2·G tau_2) */
    {
        const double c0 = dot3(n, col[0]), c1 = dot3(n, col[1]);
        const double nn = -(dot3(tau[0], col[0]) + dot3(tau[1], col[1]));
        for (a = 0; a < 3; ++a) col[2][a] = c0 * tau[0][a] + c1 * tau[1][a] + nn * n[a];
    }
    for (a = 0; a < 3; ++a)
        for (b = 0; b < 3; ++b) G[a][b] = col[0][a] * tau[0][b] + col[1][a] * tau[1][b] + col[2][a] * n[b];
    g[0] = G[0][0]; g[1] = G[1][1]; g[2] = G[2][2];
    g[3] = 0.5 * (G[0][1] + G[1][0]);
    g[4] = 0.5 * (G[0][2] + G[2][0]);
    g[5] = 0.5 * (G[1][2] + G[2][1]);
}

/* gradient of ONE element with the quadratic density coef = (c0 .. c5)
 * (linear: c3 = c4 = c5 = 0), without 1/(4 pi eps0); methods PAPER, GL2,
 * ANALYTIC, RULE as oracle_element_grad */
int oracle_element_grad_var(int type, const double* verts, const double* coef, const double* P, int method,
                            int param, const double* limits, double* out /* 6 */, int* band_out)
{
    elem_t e;
    lin_t s;
    int band = -1;
    build_rules();
    elem_setup(&e, type, verts);
    quadratic_density(&e, coef, &s);
    switch (method) {
    case OR_METHOD_PAPER:
        band = choose_band(&e, P, limits ? limits + 5 * type : DEFAULT_LIMITS[type], NULL);
        if (band == 0) analytic_grad_var(&e, P, &s, out);
        else cubature_grad_var(&e, band - 1, P, &s, out);
        break;
    case OR_METHOD_GL2:
        if (param < 1 || param > NGL_MAX) return -1;
        gl2_grad_var(&e, param, P, &s, out);
        break;
    case OR_METHOD_ANALYTIC:
        analytic_grad_var(&e, P, &s, out);
        break;
    case OR_METHOD_RULE:
        if (param < 0 || param > 4) return -1;
        cubature_grad_var(&e, param, P, &s, out);
        break;
    default:
        return -1;
    }
    if (band_out) *band_out = band;
    return 0;
}

/* field gradient at n_pts points for elements with quadratic densities
 * coef (n_el x 6), by the method, summed in index order, times 1/(4 pi eps0) */
int oracle_eval_grad_var(int64_t n_el, const int32_t* type, const double* verts, const double* coef,
                         const double* limits, double eps0, int64_t n_pts, const double* pts, double* G,
                         double* gsum, int nthreads)
{
    const double kc = coulomb_k(eps0);
    int64_t p, j;
    build_rules();
    if (n_el < 0 || n_pts < 0) return -1;
    for (j = 0; j < n_el; ++j)
        if (type[j] != 0 && type[j] != 1) return -1;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
    for (p = 0; p < n_pts; ++p) {
        const double* P = pts + 3 * p;
        double sm[6] = {0, 0, 0, 0, 0, 0}, c[6] = {0, 0, 0, 0, 0, 0}, am = 0.0;
        int64_t jj;
        int k;
        for (jj = 0; jj < n_el; ++jj) {
            elem_t e;
            lin_t s;
            double f[6], mx = 0.0;
            int band;
            elem_setup(&e, type[jj], verts + 12 * jj);
            quadratic_density(&e, coef + 6 * jj, &s);
            band = choose_band(&e, P, limits ? limits + 5 * type[jj] : DEFAULT_LIMITS[type[jj]], NULL);
            if (band == 0) analytic_grad_var(&e, P, &s, f);
            else cubature_grad_var(&e, band - 1, P, &s, f);
            for (k = 0; k < 6; ++k) {
                nsum_add(&sm[k], &c[k], f[k]);
                if (fabs(f[k]) > mx) mx = fabs(f[k]);
            }
            am += mx;
        }
        for (k = 0; k < 6; ++k) G[6 * p + k] = kc * (sm[k] + c[k]);
        if (gsum) gsum[p] = kc * am;
    }
    return 0;
}
