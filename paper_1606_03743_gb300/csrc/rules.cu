// rules.cu -- the ten Gaussian cubature rules of the paper's appendices,
// expanded on the host into the library's node representation.
//
// Triangle rules (App. A, Tables A1-A5) list barycentric rows (lambda_A,
// lambda_B, lambda_C, w) that expand by permutation; rectangle rules
// (App. B, Tables B1-B5) list natural-coordinate rows (x, y, w) that expand
// by sign changes or rotations.  A node is stored as (alpha, beta, w) with
//   Q = Q_cen + alpha e0 + beta e1,
// where for a triangle e0 = A - Q_cen, e1 = B - Q_cen and, since
// C - Q_cen = -e0 - e1 and the lambdas sum to one (Eq. 3.3),
// alpha = lambda_A - lambda_C, beta = lambda_B - lambda_C; for a rectangle
// e0 = (a/2) u_x, e1 = (b/2) u_y and (alpha, beta) = (x, y) (Eq. 3.2).
#include <math.h>
#include <string.h>

#include <mutex>

#include "bem_internal.cuh"

namespace bem {
namespace {

enum Expand {
    kCentre,      // one node at the centroid (triangle) or (0, 0) (rectangle)
    kTriPerm3,    // (p, q, q) and its two other distinct permutations
    kTriCyclic,   // (a, b, c), (b, c, a), (c, a, b)
    kTriPerm6,    // all six permutations of (a, b, c)
    kRectAxisY,   // (0, +t), (0, -t)
    kRectAxes,    // (+r, 0), (-r, 0), (0, +r), (0, -r)
    kRectSigns,   // (+-x, +-y)
    kRectRot,     // (x, y), (-x, -y), (-y, x), (y, -x)
};

struct Row {
    Expand how;
    double a, b, c, w;
};

struct Builder {
    RuleSet* rs;
    int type, slot;
    void tri(double la, double lb, double lc, double w) {
        rs->alpha[type][slot] = la - lc;
        rs->beta[type][slot] = lb - lc;
        rs->w[type][slot] = w;
        ++slot;
    }
    void rect(double x, double y, double w) {
        rs->alpha[type][slot] = x;
        rs->beta[type][slot] = y;
        rs->w[type][slot] = w;
        ++slot;
    }
    void row(const Row& r) {
        switch (r.how) {
            case kCentre:
                if (type == BEM_TRIANGLE) tri(1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0, r.w);
                else rect(0.0, 0.0, r.w);
                break;
            case kTriPerm3:
                tri(r.a, r.b, r.b, r.w);
                tri(r.b, r.a, r.b, r.w);
                tri(r.b, r.b, r.a, r.w);
                break;
            case kTriCyclic:
                tri(r.a, r.b, r.c, r.w);
                tri(r.b, r.c, r.a, r.w);
                tri(r.c, r.a, r.b, r.w);
                break;
            case kTriPerm6: {
                const double v[3] = {r.a, r.b, r.c};
                const int p[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
                for (auto& q : p) tri(v[q[0]], v[q[1]], v[q[2]], r.w);
                break;
            }
            case kRectAxisY:
                rect(0.0, r.a, r.w);
                rect(0.0, -r.a, r.w);
                break;
            case kRectAxes:
                rect(r.a, 0.0, r.w);
                rect(-r.a, 0.0, r.w);
                rect(0.0, r.a, r.w);
                rect(0.0, -r.a, r.w);
                break;
            case kRectSigns:
                rect(r.a, r.b, r.w);
                rect(r.a, -r.b, r.w);
                rect(-r.a, r.b, r.w);
                rect(-r.a, -r.b, r.w);
                break;
            case kRectRot:
                rect(r.a, r.b, r.w);
                rect(-r.a, -r.b, r.w);
                rect(-r.b, r.a, r.w);
                rect(r.b, -r.a, r.w);
                break;
        }
    }
};

void build(RuleSet* rs) {
    memset(rs, 0, sizeof(*rs));
    const double s15 = sqrt(15.0), s583 = sqrt(583.0);

    // ---- triangles -------------------------------------------------------
    // Table A1 (N = 4, degree 3)
    const Row t4[] = {{kCentre, 0, 0, 0, -9.0 / 16.0}, {kTriPerm3, 0.6, 0.2, 0, 25.0 / 48.0}};
    // Table A2 (N = 7, degree 5): t = 1/3, s = (1 - sqrt15)/7, r = (1 + sqrt15)/7
    const double t = 1.0 / 3.0, s7 = (1.0 - s15) / 7.0, r7 = (1.0 + s15) / 7.0;
    const Row t7[] = {{kCentre, 0, 0, 0, 9.0 / 40.0},
                      {kTriPerm3, t + 2 * t * s7, t - t * s7, 0, (155.0 + s15) / 1200.0},
                      {kTriPerm3, t + 2 * t * r7, t - t * r7, 0, (155.0 - s15) / 1200.0}};
    // Table A3 (N = 12, degree 7), cyclic permutations
    const Row t12[] = {
        {kTriCyclic, 0.06238226509439084, 0.06751786707392436, 0.8700998678316848, 0.05303405631486900},
        {kTriCyclic, 0.05522545665692000, 0.3215024938520156, 0.6232720494910644, 0.08776281742889622},
        {kTriCyclic, 0.03432430294509488, 0.6609491961867980, 0.3047265008681072, 0.05755008556995056},
        {kTriCyclic, 0.5158423343536001, 0.2777161669764050, 0.2064414986699949, 0.13498637401961758}};
    // Table A4 (N = 19, degree 9)
    const Row t19[] = {{kCentre, 0, 0, 0, 0.09713579628279610},
                       {kTriPerm3, 0.02063496160252593, 0.48968251919873704, 0, 0.03133470022713983},
                       {kTriPerm3, 0.1258208170141290, 0.4370895914929355, 0, 0.07782754100477543},
                       {kTriPerm3, 0.6235929287619356, 0.18820353561903219, 0, 0.07964773892720910},
                       {kTriPerm3, 0.9105409732110941, 0.04472951339445297, 0, 0.02557767565869810},
                       {kTriPerm6, 0.03683841205473626, 0.7411985987844980, 0.22196298916076573,
                        0.04328353937728940}};
    // Table A5 (N = 33, degree 12)
    const Row t33[] = {
        {kTriPerm3, 0.4570749859701478, 0.27146250701492611, 0, 0.06254121319590276},
        {kTriPerm3, 0.1197767026828138, 0.44011164865859310, 0, 0.04991833492806094},
        {kTriPerm3, 0.0235924981089169, 0.48820375094554155, 0, 0.02426683808145203},
        {kTriPerm3, 0.7814843446812914, 0.10925782765935432, 0, 0.02848605206887754},
        {kTriPerm3, 0.9507072731273288, 0.02464636343633558, 0, 0.00793164250997364},
        {kTriPerm6, 0.1162960196779266, 0.2554542286385173, 0.62824975168355610, 0.04322736365941421},
        {kTriPerm6, 0.02303415635526714, 0.2916556797383410, 0.68531016390639186, 0.02178358503860756},
        {kTriPerm6, 0.02138249025617059, 0.1272797172335894, 0.85133779251024000, 0.01508367757651144}};

    // ---- rectangles -------------------------------------------------------
    // Table B1 (N = 4, degree 3): s = 1/sqrt3
    const Row r4[] = {{kRectSigns, 1.0 / sqrt(3.0), 1.0 / sqrt(3.0), 0, 0.25}};
    // Table B2 (N = 7, degree 5): t = sqrt(14/15), r = sqrt(3/5), s = sqrt(1/3)
    const Row r7r[] = {{kCentre, 0, 0, 0, 2.0 / 7.0},
                       {kRectAxisY, sqrt(14.0 / 15.0), 0, 0, 5.0 / 63.0},
                       {kRectSigns, sqrt(3.0 / 5.0), sqrt(1.0 / 3.0), 0, 5.0 / 36.0}};
    // Table B3 (N = 12, degree 7)
    const double rr = sqrt(6.0 / 7.0), ss = sqrt((114.0 - 3.0 * s583) / 287.0),
                 tt = sqrt((114.0 + 3.0 * s583) / 287.0);
    const Row r12[] = {{kRectAxes, rr, 0, 0, 49.0 / 810.0},
                       {kRectSigns, ss, ss, 0, (178981.0 + 2769.0 * s583) / 1888920.0},
                       {kRectSigns, tt, tt, 0, (178981.0 - 2769.0 * s583) / 1888920.0}};
    // Table B4 (N = 17, degree 9)
    const Row r17[] = {{kCentre, 0, 0, 0, 0.131687242798353921},
                       {kRectRot, 0.968849966361977720, 0.630680119731668854, 0, 0.022219844542549678},
                       {kRectRot, 0.750277099978900533, 0.927961645959569667, 0, 0.028024900532399120},
                       {kRectRot, 0.523735820214429336, 0.453339821135647190, 0, 0.099570609815517519},
                       {kRectRot, 0.076208328192617173, 0.852615729333662307, 0, 0.067262834409945196}};
    // Table B5 (N = 33, degree 13)
    const Row r33[] = {{kCentre, 0, 0, 0, 0.075095528857806335},
                       {kRectRot, 0.778809711554419422, 0.983486682439872263, 0, 0.007497959716124783},
                       {kRectRot, 0.957297699786307365, 0.859556005641638928, 0, 0.009543605329270918},
                       {kRectRot, 0.138183459862465353, 0.958925170287534857, 0, 0.015106230954437494},
                       {kRectRot, 0.941327225872925236, 0.390736216129461000, 0, 0.019373184633276336},
                       {kRectRot, 0.475808625218275905, 0.850076673699748575, 0, 0.029711166825148901},
                       {kRectRot, 0.755805356572081436, 0.647821637187010732, 0, 0.032440887592500675},
                       {kRectRot, 0.696250078491749413, 0.070741508996444936, 0, 0.053335395364297350},
                       {kRectRot, 0.342716556040406789, 0.409304561694038843, 0, 0.064217687370491966}};

    struct Span {
        const Row* rows;
        int n;
    };
    const Span tri_rules[5] = {{t4, 2}, {t7, 3}, {t12, 4}, {t19, 6}, {t33, 8}};
    const Span rect_rules[5] = {{r4, 1}, {r7r, 3}, {r12, 3}, {r17, 5}, {r33, 9}};
    for (int type = 0; type < 2; ++type) {
        Builder b{rs, type, 0};
        for (int r = 0; r < 5; ++r) {
            const Span& sp = type == BEM_TRIANGLE ? tri_rules[r] : rect_rules[r];
            rs->start[type][r] = b.slot;
            for (int k = 0; k < sp.n; ++k) b.row(sp.rows[k]);
            rs->n[type][r] = b.slot - rs->start[type][r];
        }
    }
}

}  // namespace

const RuleSet& rules() {
    static RuleSet rs;
    static std::once_flag once;
    std::call_once(once, [] { build(&rs); });
    return rs;
}

}  // namespace bem

extern "C" int bem_rule(int32_t type, int32_t r, double* out) {
    if ((type != BEM_TRIANGLE && type != BEM_RECTANGLE) || r < 0 || r > 4 || !out) {
        bem::set_error("bem_rule: bad arguments (type %d, rule %d)", (int)type, (int)r);
        return BEM_ERR_INVALID;
    }
    const bem::RuleSet& rs = bem::rules();
    const int s = rs.start[type][r], n = rs.n[type][r];
    for (int i = 0; i < n; ++i) {
        out[3 * i + 0] = rs.alpha[type][s + i];
        out[3 * i + 1] = rs.beta[type][s + i];
        out[3 * i + 2] = rs.w[type][s + i];
    }
    return n;
}
