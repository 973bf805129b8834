// Device-side setup: geometry upload, FP64 near-field Galerkin integrals with
// singularity extraction, leaf radiation/receive patterns, translation operators,
// interpolation tables and shift tables.
//
// Near-field entries (Eqs. 43-46 restricted to RWG pairs in touching leaf boxes):
//   P_mn = 1/2 <f_m, L f_n> + 1/2 <f_m, n x Kbar f_n>,  Q_mn = 1/2 <f_m, n x L f_n> - 1/2 <f_m, Kbar f_n>,
// with L and Kbar as defined below Eq. 22 (Sec. II.C).  Each entry is a sum over the
// four triangle pairs of the two RWG supports.  Per triangle pair, the outer integral
// runs over the test triangle, the inner one over the source triangle:
//   - separated pairs: 7-point Radon rules on both triangles;
//   - close pairs: the inner integrals of 1/R, R, (r'-r)/R, (r'-r) R and grad(1/R) are
//     closed forms (Wilton et al. 1984; Graglia 1993), the bounded remainder of G and
//     grad G uses the 7-point rule; the outer rule is a composite rule, or a product
//     Gauss rule graded toward the shared edge/vertex, or (same triangle) three
//     sub-triangles graded toward the triangle's own edges;
//   - the grad-Phi part of <f_m, n x L f_n> is integrated by parts onto the edges of the
//     test triangle for close pairs (n x f_m is divergence free on a flat triangle).
#include <algorithm>
#include <chrono>
#include <cmath>
#include <complex>
#include <cstdlib>
#include <vector>

#include "bi_internal.h"

namespace {

constexpr double kPiD = 3.14159265358979323846;

// ------------------------------------------------------------- rules (constant memory)
constexpr int kNearQ = 28, kEdgeQ = 64, kVertQ = 64, kLineQ = 8;
struct rules_c {
    double near_b[kNearQ][3], near_w[kNearQ];
    double edge_b[kEdgeQ][3], edge_w[kEdgeQ];
    double vert_b[kVertQ][3], vert_w[kVertQ];
    double line_x[kLineQ], line_w[kLineQ];
};
__constant__ rules_c c_rules;

// 7-point rule of degree 5 (Radon 1948): centroid, and two orbits of three points.
__device__ __forceinline__ void radon7(int q, double& b0, double& b1, double& b2, double& w) {
    const double s15 = 3.872983346207417;  // sqrt(15)
    const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
    if (q == 0) { b0 = b1 = b2 = 1.0 / 3.0; w = 9.0 / 40.0; return; }
    double a = (q <= 3) ? a1 : a2;
    w = (q <= 3) ? (155.0 - s15) / 1200.0 : (155.0 + s15) / 1200.0;
    int r = (q - 1) % 3;
    b0 = b1 = b2 = a;
    double c = 1.0 - 2.0 * a;
    if (r == 0) b0 = c; else if (r == 1) b1 = c; else b2 = c;
}

struct dtri {
    double p[3][3];
    double n[3];
    double area, diam, c[3];
    int vid[3];
};

__device__ __forceinline__ double dot3(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
__device__ __forceinline__ void cross3(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

__device__ void load_tri(const double* tri, const double* nrm, const double* area, const int* vid, int t, dtri& T) {
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) T.p[a][d] = tri[9 * t + 3 * a + d];
    for (int d = 0; d < 3; ++d) {
        T.n[d] = nrm[3 * t + d];
        T.c[d] = (T.p[0][d] + T.p[1][d] + T.p[2][d]) / 3.0;
    }
    T.area = area[t];
    double m = 0;
    for (int e = 0; e < 3; ++e) {
        double s = 0;
        for (int d = 0; d < 3; ++d) {
            double x = T.p[(e + 1) % 3][d] - T.p[e][d];
            s += x * x;
        }
        m = fmax(m, s);
    }
    T.diam = sqrt(m);
    for (int a = 0; a < 3; ++a) T.vid[a] = vid[3 * t + a];
}

// complex double helpers
struct zd {
    double x, y;
};
__device__ __forceinline__ zd zmk(double a, double b) { return zd{a, b}; }
__device__ __forceinline__ zd zadd(zd a, zd b) { return zd{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ zd zmul(zd a, zd b) { return zd{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ zd zscale(zd a, double s) { return zd{a.x * s, a.y * s}; }
__device__ __forceinline__ zd zexpj(double ph) {  // exp(j ph)
    double s, c;
    sincos(ph, &s, &c);
    return zd{c, s};
}
__device__ __forceinline__ zd zsub(zd a, zd b) { return zd{a.x - b.x, a.y - b.y}; }
__device__ __forceinline__ zd zinv(zd a) {
    const double d = 1.0 / (a.x * a.x + a.y * a.y);
    return zd{a.x * d, -a.y * d};
}

// Wavenumber arithmetic.  KT = double: a real wavenumber (the exterior free space, the paths
// used before complex wavenumbers existed, compiled unchanged); KT = zd: a complex wavenumber
// k = k' + j k'' of a lossy medium (k'' <= 0 with exp(j w t)), where every kernel is the
// analytic continuation of the real-k one.
template <typename KT>
constexpr bool kReal = sizeof(KT) == sizeof(double);
__device__ __forceinline__ zd kz(double k) { return zd{k, 0.0}; }
__device__ __forceinline__ zd kz(zd k) { return k; }
// exp(-j k R) for real R
__device__ __forceinline__ zd zexp_mjk(zd k, double R) { return zscale(zexpj(-k.x * R), exp(k.y * R)); }

// Closed-form integrals over triangle S seen from r (in the plane: principal values):
//   I1 = int 1/R, IR = int R, Irho = int (rho'-rho)/R, IrhoR = int (rho'-rho) R, Ig = int grad_r(1/R)
struct statics {
    double I1, IR, h;
    double Irho[3], IrhoR[3], Ig[3];
};

__device__ void static_parts(const dtri& S, const double* r, statics& o) {
    double v0[3] = {r[0] - S.p[0][0], r[1] - S.p[0][1], r[2] - S.p[0][2]};
    double h = dot3(S.n, v0);
    double rho[3] = {r[0] - h * S.n[0], r[1] - h * S.n[1], r[2] - h * S.n[2]};
    double ah = fabs(h);
    double tiny = 1e-12 * S.diam;
    double sum1 = 0, sumR = 0, om = 0;
    for (int d = 0; d < 3; ++d) { o.Irho[d] = 0; o.IrhoR[d] = 0; o.Ig[d] = 0; }
    for (int e = 0; e < 3; ++e) {
        const double* A = S.p[e];
        const double* B = S.p[(e + 1) % 3];
        double t[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double len = sqrt(dot3(t, t));
        for (int d = 0; d < 3; ++d) t[d] /= len;
        double u[3];
        cross3(t, S.n, u);
        double qa[3] = {A[0] - rho[0], A[1] - rho[1], A[2] - rho[2]};
        double qb[3] = {B[0] - rho[0], B[1] - rho[1], B[2] - rho[2]};
        double lm = dot3(qa, t), lp = dot3(qb, t), d0 = dot3(qa, u);
        double R02 = d0 * d0 + h * h;
        double Rp = sqrt(lp * lp + R02), Rm = sqrt(lm * lm + R02);
        bool online = sqrt(R02) < tiny;
        // log((Rp + lp)/(Rm + lm)), with R + l = R0^2 / (R - l) when l < 0
        double f = 0;
        bool finite = true;
        if (online) {
            finite = !(lm <= 0.0 && lp >= 0.0);
            if (finite) f = (lp > 0) ? log((Rp + lp) / (Rm + lm)) : log((Rm - lm) / (Rp - lp));
        } else {
            double num = (lp >= 0) ? (Rp + lp) : R02 / (Rp - lp);
            double den = (lm >= 0) ? (Rm + lm) : R02 / (Rm - lm);
            f = log(num / den);
        }
        double beta = 0;
        if (!online) beta = atan(d0 * lp / (R02 + ah * Rp)) - atan(d0 * lm / (R02 + ah * Rm));
        double eR = 0.5 * (lp * Rp - lm * Rm + (online ? 0.0 : R02 * f));  // int_edge R dl
        double eR3 = 0.25 * (lp * Rp * Rp * Rp - lm * Rm * Rm * Rm) + 0.375 * R02 * (lp * Rp - lm * Rm) +
                     (online ? 0.0 : 0.375 * R02 * R02 * f);                 // int_edge R^3 dl
        if (!online) sum1 += d0 * f - ah * beta;
        sumR += d0 * eR;
        om += beta;
        for (int d = 0; d < 3; ++d) {
            o.Irho[d] += u[d] * eR;
            o.IrhoR[d] += u[d] * eR3 / 3.0;
            o.Ig[d] -= finite ? u[d] * f : 0.0;  // the log singularity on the edge line only occurs where it is not used
        }
    }
    double sg = (h > 0) ? 1.0 : ((h < 0) ? -1.0 : 0.0);
    for (int d = 0; d < 3; ++d) o.Ig[d] -= S.n[d] * sg * om;
    o.I1 = sum1;
    o.IR = (sumR + h * h * sum1) / 3.0;
    o.h = h;
}

// inner integrals: Sg = int G, Sr = int (r'-r) G, Kv = int grad_r G   (complex, 1 + 3 + 3)
struct inner_res {
    zd Sg;
    zd Sr[3];
    zd Kv[3];
};

template <typename KT>
__device__ void inner_regular(const dtri& S, KT k, const double* r, inner_res& o) {
    o.Sg = zmk(0, 0);
    for (int d = 0; d < 3; ++d) { o.Sr[d] = zmk(0, 0); o.Kv[d] = zmk(0, 0); }
    const double i4pi = 1.0 / (4.0 * kPiD);
    for (int q = 0; q < 7; ++q) {
        double b0, b1, b2, w;
        radon7(q, b0, b1, b2, w);
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = b0 * S.p[0][c] + b1 * S.p[1][c] + b2 * S.p[2][c] - r[c];
        double R = sqrt(dot3(d, d));
        double ww = w * S.area;
        zd e, jkr;   // exp(-jkR), 1 + jkR
        if constexpr (kReal<KT>) {
            e = zexpj(-k * R);
            jkr = zmk(1.0, k * R);
        } else {
            e = zexp_mjk(k, R);
            jkr = zmk(1.0 - k.y * R, k.x * R);
        }
        zd G = zscale(e, i4pi / R * ww);
        // (1 + jkR) e / (4 pi R^3)
        zd gt = zscale(zmul(jkr, e), i4pi / (R * R * R) * ww);
        o.Sg = zadd(o.Sg, G);
        for (int c = 0; c < 3; ++c) {
            o.Sr[c] = zadd(o.Sr[c], zscale(G, d[c]));
            o.Kv[c] = zadd(o.Kv[c], zscale(gt, d[c]));
        }
    }
}

template <typename KT>
__device__ void inner_singular(const dtri& S, KT k, const double* r, inner_res& o, bool need_kv) {
    statics st;
    static_parts(S, r, st);
    const double i4pi = 1.0 / (4.0 * kPiD);
    // int (r'-r)/R = Irho - h n I1 ;  int (r'-r) R = IrhoR - h n IR
    double rr1[3], rrR[3];
    for (int c = 0; c < 3; ++c) {
        rr1[c] = st.Irho[c] - st.h * S.n[c] * st.I1;
        rrR[c] = st.IrhoR[c] - st.h * S.n[c] * st.IR;
    }
    // static parts of G = 1/(4 pi R) - k^2 R/(8 pi) + smooth, grad G = (r'-r)[1/R^3 + k^2/(2R)]/(4 pi) + smooth
    if constexpr (kReal<KT>) {
        const double k2 = k * k;
        o.Sg = zmk((st.I1 - 0.5 * k2 * st.IR) * i4pi, 0.0);
        for (int c = 0; c < 3; ++c) {
            o.Sr[c] = zmk((rr1[c] - 0.5 * k2 * rrR[c]) * i4pi, 0.0);
            o.Kv[c] = need_kv ? zmk((st.Ig[c] + 0.5 * k2 * rr1[c]) * i4pi, 0.0) : zmk(0, 0);
        }
    } else {
        const zd h2 = zscale(zmul(k, k), 0.5 * i4pi);   // k^2 / (8 pi)
        o.Sg = zsub(zmk(st.I1 * i4pi, 0.0), zscale(h2, st.IR));
        for (int c = 0; c < 3; ++c) {
            o.Sr[c] = zsub(zmk(rr1[c] * i4pi, 0.0), zscale(h2, rrR[c]));
            o.Kv[c] = need_kv ? zadd(zmk(st.Ig[c] * i4pi, 0.0), zscale(h2, rr1[c])) : zmk(0, 0);
        }
    }
    for (int q = 0; q < 7; ++q) {
        double b0, b1, b2, w;
        radon7(q, b0, b1, b2, w);
        double d[3];
        for (int c = 0; c < 3; ++c) d[c] = b0 * S.p[0][c] + b1 * S.p[1][c] + b2 * S.p[2][c] - r[c];
        double R = sqrt(dot3(d, d));
        double ww = w * S.area * i4pi;
        zd gr, gtr;
        if constexpr (kReal<KT>) {
            double x = k * R;
            if (x < 1e-2) {
                // series of the remainders
                gr = zmk(k * x * x * x / 24.0, -k + k * x * x / 6.0 - k * x * x * x * x / 120.0);
                gtr = (R > 0) ? zmk((-x * x * x * x / 8.0 + x * x * x * x * x * x / 144.0) / (R * R * R),
                                    (-x * x * x / 3.0 + x * x * x * x * x / 30.0) / (R * R * R))
                              : zmk(0, -k * k * k / 3.0);
            } else {
                zd e = zexpj(-x);
                gr = zscale(zmk(e.x - 1.0 + 0.5 * x * x, e.y), 1.0 / R);
                zd t = zmul(zmk(1.0, x), e);
                gtr = zscale(zmk(t.x - 1.0 - 0.5 * x * x, t.y), 1.0 / (R * R * R));
            }
        } else {
            // the same remainders at complex x = kR:
            //   (exp(-jx) - 1 + x^2/2) / R,   ((1 + jx) exp(-jx) - 1 - x^2/2) / R^3
            const zd x = zscale(k, R);
            const zd x2 = zmul(x, x), x3 = zmul(x2, x), x4 = zmul(x2, x2);
            if (sqrt(x.x * x.x + x.y * x.y) < 1e-2) {
                // k (x^3/24 + j(-1 + x^2/6 - x^4/120)),  (-j x^3/3 - x^4/8 + j x^5/30 + x^6/144) / R^3
                const zd a = zmk(-1.0 + x2.x / 6.0 - x4.x / 120.0, x2.y / 6.0 - x4.y / 120.0);
                gr = zmul(k, zadd(zscale(x3, 1.0 / 24.0), zmk(-a.y, a.x)));
                if (R > 0) {
                    const zd x5 = zmul(x4, x), x6 = zmul(x3, x3);
                    const zd im = zadd(zscale(x3, -1.0 / 3.0), zscale(x5, 1.0 / 30.0));   // times j
                    const zd re = zadd(zscale(x4, -1.0 / 8.0), zscale(x6, 1.0 / 144.0));
                    gtr = zscale(zadd(re, zmk(-im.y, im.x)), 1.0 / (R * R * R));
                } else {
                    const zd k3 = zmul(zmul(k, k), k);
                    gtr = zmk(k3.y / 3.0, -k3.x / 3.0);   // -j k^3 / 3
                }
            } else {
                const zd e = zexp_mjk(k, R);
                gr = zscale(zadd(zsub(e, zmk(1.0, 0.0)), zscale(x2, 0.5)), 1.0 / R);
                const zd t = zmul(zmk(1.0 - x.y, x.x), e);   // (1 + jx) e
                gtr = zscale(zsub(zsub(t, zmk(1.0, 0.0)), zscale(x2, 0.5)), 1.0 / (R * R * R));
            }
        }
        gr = zscale(gr, ww);
        gtr = zscale(gtr, ww);
        o.Sg = zadd(o.Sg, gr);
        for (int c = 0; c < 3; ++c) {
            o.Sr[c] = zadd(o.Sr[c], zscale(gr, d[c]));
            if (need_kv) o.Kv[c] = zadd(o.Kv[c], zscale(gtr, d[c]));
        }
    }
}

// accumulate the four raw integrands for test half-basis g_i = r - v_i and source g_j = r' - v_j
struct raw4 {
    zd L, NL, K, NK;
};

template <typename KT>
__device__ void outer_point(const dtri& Tm, const dtri& Tn, int i, int j, const double* r, double W, const inner_res& in,
                            KT k, bool surface_nl, raw4& acc) {
    double gi[3], gj[3], ngi[3], ngj[3];
    for (int c = 0; c < 3; ++c) { gi[c] = r[c] - Tm.p[i][c]; gj[c] = r[c] - Tn.p[j][c]; }
    cross3(Tm.n, gi, ngi);
    cross3(Tm.n, gj, ngj);
    // g_j(r') = (r' - r) + (r - v_j)
    zd giSr = zmk(0, 0), ngiSr = zmk(0, 0), ngiKv = zmk(0, 0);
    for (int c = 0; c < 3; ++c) {
        giSr = zadd(giSr, zscale(in.Sr[c], gi[c]));
        ngiSr = zadd(ngiSr, zscale(in.Sr[c], ngi[c]));
        ngiKv = zadd(ngiKv, zscale(in.Kv[c], ngi[c]));
    }
    double gg = dot3(gi, gj), gngj = dot3(gi, ngj);
    // L: -jk [ g_i.Sr + (g_i.g_j) Sg - (4/k^2) Sg ]
    // NL surface part: -jk [ -(n x g_i).Sr + (g_i.(n x g_j)) Sg ] (+ (2j/k)(n x g_i).Kv when separated)
    zd tN = zadd(zscale(ngiSr, -1.0), zscale(in.Sg, gngj));
    if constexpr (kReal<KT>) {
        zd tL = zadd(giSr, zscale(in.Sg, gg - 4.0 / (k * k)));
        acc.L = zadd(acc.L, zscale(zmul(zmk(0, -k), tL), W));
        zd nl = zmul(zmk(0, -k), tN);
        if (surface_nl) nl = zadd(nl, zmul(zmk(0, 2.0 / k), ngiKv));
        acc.NL = zadd(acc.NL, zscale(nl, W));
    } else {
        const zd ik = zinv(k), mjk = zmk(k.y, -k.x);
        zd tL = zadd(zadd(giSr, zscale(in.Sg, gg)), zscale(zmul(in.Sg, zmul(ik, ik)), -4.0));
        acc.L = zadd(acc.L, zscale(zmul(mjk, tL), W));
        zd nl = zmul(mjk, tN);
        if (surface_nl) nl = zadd(nl, zmul(zmk(-2.0 * ik.y, 2.0 * ik.x), ngiKv));
        acc.NL = zadd(acc.NL, zscale(nl, W));
    }
    // K: g_i.(Kv x g_j) = Kv.(g_j x g_i) ; NK: g_i.(n x (Kv x g_j)) = (Kv.g_i)(n.g_j) - (g_i.g_j)(n.Kv)
    double gjxgi[3];
    cross3(gj, gi, gjxgi);
    zd kk = zmk(0, 0), kgi = zmk(0, 0), kn = zmk(0, 0);
    for (int c = 0; c < 3; ++c) {
        kk = zadd(kk, zscale(in.Kv[c], gjxgi[c]));
        kgi = zadd(kgi, zscale(in.Kv[c], gi[c]));
        kn = zadd(kn, zscale(in.Kv[c], Tm.n[c]));
    }
    acc.K = zadd(acc.K, zscale(kk, W));
    zd nk = zadd(zscale(kgi, dot3(Tm.n, gj)), zscale(kn, -gg));
    acc.NK = zadd(acc.NK, zscale(nk, W));
}

// grad-Phi part of NL on the edges of the test triangle: -(j/k) sum_e int_e Phi (g_i . tau) dl, Phi = 2 int G
template <typename KT>
__device__ void nl_edges(const dtri& Tm, const dtri& Tn, int i, KT k, raw4& acc) {
    for (int e = 0; e < 3; ++e) {
        const double* A = Tm.p[e];
        const double* B = Tm.p[(e + 1) % 3];
        double t[3] = {B[0] - A[0], B[1] - A[1], B[2] - A[2]};
        double len = sqrt(dot3(t, t));
        for (int c = 0; c < 3; ++c) t[c] /= len;
        for (int q = 0; q < kLineQ; ++q) {
            double s = c_rules.line_x[q];
            double r[3] = {A[0] + s * (B[0] - A[0]), A[1] + s * (B[1] - A[1]), A[2] + s * (B[2] - A[2])};
            inner_res in;
            inner_singular(Tn, k, r, in, false);
            double gt = (r[0] - Tm.p[i][0]) * t[0] + (r[1] - Tm.p[i][1]) * t[1] + (r[2] - Tm.p[i][2]) * t[2];
            double wl = c_rules.line_w[q] * len * gt;
            // -(j/k) * 2 Sg * wl
            if constexpr (kReal<KT>) {
                acc.NL = zadd(acc.NL, zmul(zmk(0, -2.0 * wl / k), in.Sg));
            } else {
                const zd ik = zinv(k);
                acc.NL = zadd(acc.NL, zmul(zmk(2.0 * wl * ik.y, -2.0 * wl * ik.x), in.Sg));
            }
        }
    }
}

template <typename KT>
__device__ raw4 tri_pair(const dtri& Tm, int i, const dtri& Tn, int j, KT k) {
    raw4 acc{zmk(0, 0), zmk(0, 0), zmk(0, 0), zmk(0, 0)};
    int sa[3], ns = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (Tm.vid[a] == Tn.vid[b]) sa[ns++] = a;
    double dc[3] = {Tm.c[0] - Tn.c[0], Tm.c[1] - Tn.c[1], Tm.c[2] - Tn.c[2]};
    double dist = sqrt(dot3(dc, dc));
    double dm = fmax(Tm.diam, Tn.diam);
    if (ns == 0 && dist >= 2.0 * dm) {
        for (int q = 0; q < 7; ++q) {
            double b0, b1, b2, w;
            radon7(q, b0, b1, b2, w);
            double r[3];
            for (int c = 0; c < 3; ++c) r[c] = b0 * Tm.p[0][c] + b1 * Tm.p[1][c] + b2 * Tm.p[2][c];
            inner_res in;
            inner_regular(Tn, k, r, in);
            outer_point(Tm, Tn, i, j, r, w * Tm.area, in, k, true, acc);
        }
        return acc;
    }
    if (ns == 3) {
        // same triangle: three sub-triangles (v_e, v_e+1, centroid) graded toward their base
        for (int e = 0; e < 3; ++e)
            for (int q = 0; q < kEdgeQ; ++q) {
                double bb[3] = {0, 0, 0};
                bb[e] += c_rules.edge_b[q][0];
                bb[(e + 1) % 3] += c_rules.edge_b[q][1];
                for (int c = 0; c < 3; ++c) bb[c] += c_rules.edge_b[q][2] / 3.0;
                double r[3];
                for (int c = 0; c < 3; ++c) r[c] = bb[0] * Tm.p[0][c] + bb[1] * Tm.p[1][c] + bb[2] * Tm.p[2][c];
                inner_res in;
                inner_singular(Tn, k, r, in, false);
                outer_point(Tm, Tn, i, j, r, c_rules.edge_w[q] * Tm.area / 3.0, in, k, false, acc);
            }
        nl_edges(Tm, Tn, i, k, acc);
        acc.K = zmk(0, 0);  // principal value on one flat triangle
        acc.NK = zmk(0, 0);
        return acc;
    }
    int map[3] = {0, 1, 2};
    int nq = kNearQ;
    const double(*rb)[3] = c_rules.near_b;
    const double* rw = c_rules.near_w;
    if (ns == 2) {
        map[0] = sa[0];
        map[1] = sa[1];
        map[2] = 3 - sa[0] - sa[1];
        nq = kEdgeQ;
        rb = c_rules.edge_b;
        rw = c_rules.edge_w;
    } else if (ns == 1) {
        map[0] = sa[0];
        map[1] = (sa[0] + 1) % 3;
        map[2] = (sa[0] + 2) % 3;
        nq = kVertQ;
        rb = c_rules.vert_b;
        rw = c_rules.vert_w;
    }
    for (int q = 0; q < nq; ++q) {
        double bb[3];
        bb[map[0]] = rb[q][0];
        bb[map[1]] = rb[q][1];
        bb[map[2]] = rb[q][2];
        double r[3];
        for (int c = 0; c < 3; ++c) r[c] = bb[0] * Tm.p[0][c] + bb[1] * Tm.p[1][c] + bb[2] * Tm.p[2][c];
        inner_res in;
        inner_singular(Tn, k, r, in, true);
        outer_point(Tm, Tn, i, j, r, rw[q] * Tm.area, in, k, false, acc);
    }
    nl_edges(Tm, Tn, i, k, acc);
    return acc;
}

// Regular triangle pairs (no shared vertex, centroids at least three diameters apart): plain
// 7-point rules on both triangles, evaluated in FP32.
// Triangle-pair classes of the near-field fill:
//   0 separated by >= 4 diameters: 7 x 7 point rules, FP32
//   1 separated by 2..4 diameters: 28 x 28 point composite rules, FP32
//   2 closer than 2 diameters, no shared vertex: singularity subtraction, FP64
//   3 one shared vertex, 4 shared edge, 5 same triangle: singularity subtraction with graded rules, FP64
__device__ __forceinline__ int pair_class(const dtri& Tm, const dtri& Tn) {
    int ns = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (Tm.vid[a] == Tn.vid[b]) ++ns;
    if (ns > 0) return 2 + ns;
    double dc[3] = {Tm.c[0] - Tn.c[0], Tm.c[1] - Tn.c[1], Tm.c[2] - Tn.c[2]};
    const double d = sqrt(dot3(dc, dc)), dm = fmax(Tm.diam, Tn.diam);
    return d >= 4.0 * dm ? 0 : (d >= 2.0 * dm ? 1 : 2);
}

struct zf {
    float x, y;
};
__device__ __forceinline__ zf fadd(zf a, zf b) { return zf{a.x + b.x, a.y + b.y}; }
__device__ __forceinline__ zf fmul(zf a, zf b) { return zf{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x}; }
__device__ __forceinline__ zf fsc(zf a, float s) { return zf{a.x * s, a.y * s}; }

// returns (P_raw, Q_raw) = (1/2)(L + NK), (1/2)(NL - K) for half-bases g_i (test), g_j (source)
template <int NSUB>
__device__ void tri_pair_regular_f32(const dtri& Tm, int i, const dtri& Tn, int j, float k, zf& Pr, zf& Qr) {
    // coordinates relative to the test centroid keep FP32 accurate for large meshes
    float pm[3][3], pn[3][3], nm[3];
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) {
            pm[a][d] = (float)(Tm.p[a][d] - Tm.c[d]);
            pn[a][d] = (float)(Tn.p[a][d] - Tm.c[d]);
        }
    for (int d = 0; d < 3; ++d) nm[d] = (float)Tm.n[d];
    const float Am = (float)Tm.area, An = (float)Tn.area;
    const float i4pi = 0.0795774715459477f;
    const float s15 = 3.8729833f;
    const float a1 = (6.0f - s15) / 21.0f, a2 = (6.0f + s15) / 21.0f;
    const float w1 = (155.0f - s15) / 1200.0f, w2 = (155.0f + s15) / 1200.0f;
    // 7-point rule on NSUB sub-triangles (midpoint subdivision when NSUB = 4)
    constexpr int NQ = 7 * NSUB;
    float bq[NQ][3], wq[NQ];
    {
        float b7[7][3], w7[7];
        b7[0][0] = b7[0][1] = b7[0][2] = 1.0f / 3.0f;
        w7[0] = 9.0f / 40.0f;
        for (int q = 1; q < 7; ++q) {
            const float a = (q <= 3) ? a1 : a2;
            w7[q] = (q <= 3) ? w1 : w2;
            b7[q][0] = b7[q][1] = b7[q][2] = a;
            b7[q][(q - 1) % 3] = 1.0f - 2.0f * a;
        }
        const float sub[4][3][3] = {{{1, 0, 0}, {.5f, .5f, 0}, {.5f, 0, .5f}},
                                    {{.5f, .5f, 0}, {0, 1, 0}, {0, .5f, .5f}},
                                    {{.5f, 0, .5f}, {0, .5f, .5f}, {0, 0, 1}},
                                    {{.5f, .5f, 0}, {0, .5f, .5f}, {.5f, 0, .5f}}};
        for (int sb = 0; sb < NSUB; ++sb)
            for (int q = 0; q < 7; ++q) {
                for (int d = 0; d < 3; ++d)
                    bq[sb * 7 + q][d] = NSUB == 1 ? b7[q][d]
                                                   : b7[q][0] * sub[sb][0][d] + b7[q][1] * sub[sb][1][d] + b7[q][2] * sub[sb][2][d];
                wq[sb * 7 + q] = w7[q] / NSUB;
            }
    }
    zf L = {0, 0}, NL = {0, 0}, K = {0, 0}, NK = {0, 0};
    for (int qo = 0; qo < NQ; ++qo) {
        float r[3];
        for (int d = 0; d < 3; ++d) r[d] = bq[qo][0] * pm[0][d] + bq[qo][1] * pm[1][d] + bq[qo][2] * pm[2][d];
        zf Sg = {0, 0}, Sr[3] = {{0, 0}, {0, 0}, {0, 0}}, Kv[3] = {{0, 0}, {0, 0}, {0, 0}};
        for (int qi = 0; qi < NQ; ++qi) {
            float dd[3];
            for (int d = 0; d < 3; ++d)
                dd[d] = bq[qi][0] * pn[0][d] + bq[qi][1] * pn[1][d] + bq[qi][2] * pn[2][d] - r[d];
            const float R2 = dd[0] * dd[0] + dd[1] * dd[1] + dd[2] * dd[2];
            const float iR = rsqrtf(R2);
            const float R = R2 * iR;
            float sn, cs;
            sincosf(-k * R, &sn, &cs);
            const float ww = wq[qi] * An * i4pi * iR;
            const zf G = {cs * ww, sn * ww};
            // (1 + jkR) e^{-jkR} / R^2 (times the 1/R of ww)
            const zf gt = fsc(fmul(zf{1.0f, k * R}, zf{cs, sn}), ww * iR * iR);
            Sg = fadd(Sg, G);
            for (int d = 0; d < 3; ++d) {
                Sr[d] = fadd(Sr[d], fsc(G, dd[d]));
                Kv[d] = fadd(Kv[d], fsc(gt, dd[d]));
            }
        }
        const float W = wq[qo] * Am;
        float gi[3], gj[3], ngi[3], ngj[3];
        for (int d = 0; d < 3; ++d) { gi[d] = r[d] - pm[i][d]; gj[d] = r[d] - pn[j][d]; }
        ngi[0] = nm[1] * gi[2] - nm[2] * gi[1]; ngi[1] = nm[2] * gi[0] - nm[0] * gi[2]; ngi[2] = nm[0] * gi[1] - nm[1] * gi[0];
        ngj[0] = nm[1] * gj[2] - nm[2] * gj[1]; ngj[1] = nm[2] * gj[0] - nm[0] * gj[2]; ngj[2] = nm[0] * gj[1] - nm[1] * gj[0];
        zf giSr = {0, 0}, ngiSr = {0, 0}, ngiKv = {0, 0}, kk = {0, 0}, kgi = {0, 0}, kn = {0, 0};
        float gjxgi[3] = {gj[1] * gi[2] - gj[2] * gi[1], gj[2] * gi[0] - gj[0] * gi[2], gj[0] * gi[1] - gj[1] * gi[0]};
        for (int d = 0; d < 3; ++d) {
            giSr = fadd(giSr, fsc(Sr[d], gi[d]));
            ngiSr = fadd(ngiSr, fsc(Sr[d], ngi[d]));
            ngiKv = fadd(ngiKv, fsc(Kv[d], ngi[d]));
            kk = fadd(kk, fsc(Kv[d], gjxgi[d]));
            kgi = fadd(kgi, fsc(Kv[d], gi[d]));
            kn = fadd(kn, fsc(Kv[d], nm[d]));
        }
        const float gg = gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2];
        const float gngj = gi[0] * ngj[0] + gi[1] * ngj[1] + gi[2] * ngj[2];
        const zf tL = fadd(giSr, fsc(Sg, gg - 4.0f / (k * k)));
        L = fadd(L, fsc(fmul(zf{0.0f, -k}, tL), W));
        const zf tN = fadd(fsc(ngiSr, -1.0f), fsc(Sg, gngj));
        NL = fadd(NL, fsc(fadd(fmul(zf{0.0f, -k}, tN), fmul(zf{0.0f, 2.0f / k}, ngiKv)), W));
        K = fadd(K, fsc(kk, W));
        const float ngjn = nm[0] * gj[0] + nm[1] * gj[1] + nm[2] * gj[2];
        NK = fadd(NK, fsc(fadd(fsc(kgi, ngjn), fsc(kn, -gg)), W));
    }
    Pr = fsc(fadd(L, NK), 0.5f);
    Qr = fsc(fadd(NL, fsc(K, -1.0f)), 0.5f);
}

// Pass 1: one CTA per near block, one thread per entry: the separated triangle pairs
// (classes 0, 1) in FP32; every other triangle pair of the entry is appended to the list of
// its class for pass 2.  Entry = (A, B) with A = P, B = Q at this point.
struct special_item {
    int lo, hi;   // entry offset (split in two 31-bit halves)
    int m, n;     // tree RWG indices
    int sides;    // sm | (sn << 1)
    int pad;
};
template <typename T>
__global__ void __launch_bounds__(128) k_near_regular(int nblk, const int* __restrict__ blk_box, const int* __restrict__ near_ptr,
                                                      const int* __restrict__ near_src, const int64_t* __restrict__ near_blk,
                                                      const int* __restrict__ leaf_start, const int* __restrict__ rwg_t,
                                                      const int* __restrict__ rwg_l, const double* __restrict__ rwg_len,
                                                      const double* __restrict__ tri, const double* __restrict__ nrm,
                                                      const double* __restrict__ area, const int* __restrict__ vid, double k,
                                                      int mode, T* __restrict__ out, special_item* __restrict__ lists,
                                                      unsigned long long* __restrict__ count,
                                                      const unsigned long long* __restrict__ cap,
                                                      const unsigned long long* __restrict__ base) {
    int q = blockIdx.x;
    if (q >= nblk) return;
    int b = blk_box[q], s = near_src[q];
    int m0 = leaf_start[b], mb = leaf_start[b + 1] - m0;
    int n0 = leaf_start[s], nbs = leaf_start[s + 1] - n0;
    const int64_t seg = near_blk[near_ptr[b]];
    const int ncol = (int)((near_blk[near_ptr[b + 1]] - seg) / mb);
    const int c0 = (int)((near_blk[q] - seg) / mb);
    for (int e = threadIdx.x; e < mb * nbs; e += blockDim.x) {
        const int ml = e % mb, nl = e / mb;
        const int m = m0 + ml, n = n0 + nl;
        const int64_t o = seg + (int64_t)ml * ncol + c0 + nl;
        zf P = {0, 0}, Q = {0, 0};
        for (int sm = 0; sm < 2; ++sm) {
            dtri Tm;
            load_tri(tri, nrm, area, vid, rwg_t[2 * m + sm], Tm);
            const int i = rwg_l[2 * m + sm];
            const float cm = (float)((sm == 0 ? 1.0 : -1.0) * rwg_len[m] / (2.0 * Tm.area));
            for (int sn = 0; sn < 2; ++sn) {
                dtri Tn;
                load_tri(tri, nrm, area, vid, rwg_t[2 * n + sn], Tn);
                const int cls = pair_class(Tm, Tn);
                if (cls >= 2) {
                    const unsigned long long slot = atomicAdd(count + (cls - 2), 1ull);
                    if (slot < cap[cls - 2]) {
                        special_item it;
                        it.lo = (int)(o & 0x7fffffff);
                        it.hi = (int)(o >> 31);
                        it.m = m;
                        it.n = n;
                        it.sides = sm | (sn << 1);
                        it.pad = 0;
                        lists[base[cls - 2] + slot] = it;
                    }
                    continue;
                }
                const int j = rwg_l[2 * n + sn];
                const float cn = (float)((sn == 0 ? 1.0 : -1.0) * rwg_len[n] / (2.0 * Tn.area));
                zf pr, qr;
                if (cls == 0) tri_pair_regular_f32<1>(Tm, i, Tn, j, (float)k, pr, qr);
                else tri_pair_regular_f32<4>(Tm, i, Tn, j, (float)k, pr, qr);
                P = fadd(P, fsc(pr, cm * cn));
                Q = fadd(Q, fsc(qr, cm * cn));
            }
        }
        if (mode == 0) {
            out[4 * o + 0] = (T)P.x;
            out[4 * o + 1] = (T)P.y;
            out[4 * o + 2] = (T)Q.x;
            out[4 * o + 3] = (T)Q.y;
        } else {
            out[2 * o + 0] = (T)P.x;
            out[2 * o + 1] = (T)P.y;
        }
    }
}

// Counting pass: how many triangle pairs of each special class (2..5) the near entries hold,
// so the lists of pass 1 are allocated exactly.
__global__ void __launch_bounds__(128) k_near_count(int nblk, const int* __restrict__ blk_box, const int* __restrict__ near_src,
                                                    const int* __restrict__ leaf_start, const int* __restrict__ rwg_t,
                                                    const double* __restrict__ tri, const double* __restrict__ nrm,
                                                    const double* __restrict__ area, const int* __restrict__ vid,
                                                    unsigned long long* __restrict__ count) {
    int q = blockIdx.x;
    if (q >= nblk) return;
    int b = blk_box[q], s = near_src[q];
    int m0 = leaf_start[b], mb = leaf_start[b + 1] - m0;
    int n0 = leaf_start[s], nbs = leaf_start[s + 1] - n0;
    unsigned long long c[4] = {0, 0, 0, 0};
    for (int e = threadIdx.x; e < mb * nbs; e += blockDim.x) {
        const int m = m0 + e % mb, n = n0 + e / mb;
        for (int sm = 0; sm < 2; ++sm) {
            dtri Tm;
            load_tri(tri, nrm, area, vid, rwg_t[2 * m + sm], Tm);
            for (int sn = 0; sn < 2; ++sn) {
                dtri Tn;
                load_tri(tri, nrm, area, vid, rwg_t[2 * n + sn], Tn);
                const int cls = pair_class(Tm, Tn);
                if (cls >= 2) ++c[cls - 2];
            }
        }
    }
    for (int k = 0; k < 4; ++k)
        if (c[k]) atomicAdd(count + k, c[k]);
}

// Pass 2: one thread per listed triangle pair of one class (so a warp follows one path):
// the pair's contribution in FP64 with singularity extraction, plus its Gram terms for the
// same-triangle class, added atomically to the entry (at most four pairs per entry):
// A += P - g G, B += Q - X/2.
template <typename T>
__global__ void __launch_bounds__(128) k_near_special(unsigned long long nlist, const special_item* __restrict__ list,
                                                      const int* __restrict__ rwg_t, const int* __restrict__ rwg_l,
                                                      const double* __restrict__ rwg_len, const double* __restrict__ tri,
                                                      const double* __restrict__ nrm, const double* __restrict__ area,
                                                      const int* __restrict__ vid, double k, int mode, T* __restrict__ out) {
    const unsigned long long it = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= nlist) return;
    const special_item w = list[it];
    const int64_t o = (int64_t)(unsigned)w.lo | ((int64_t)w.hi << 31);
    const int m = w.m, n = w.n, sm = w.sides & 1, sn = (w.sides >> 1) & 1;
    dtri Tm, Tn;
    const int tm = rwg_t[2 * m + sm], i = rwg_l[2 * m + sm];
    const int tn = rwg_t[2 * n + sn], j = rwg_l[2 * n + sn];
    load_tri(tri, nrm, area, vid, tm, Tm);
    load_tri(tri, nrm, area, vid, tn, Tn);
    const double cm = (sm == 0 ? 1.0 : -1.0) * rwg_len[m] / (2.0 * Tm.area);
    const double cn = (sn == 0 ? 1.0 : -1.0) * rwg_len[n] / (2.0 * Tn.area);
    raw4 r = tri_pair(Tm, i, Tn, j, k);
    const double c = 0.5 * cm * cn;
    zd P = zscale(zadd(r.L, r.NK), c);
    zd Q = zscale(zadd(r.NL, zscale(r.K, -1.0)), c);
    double G = 0, X = 0;
    if (tm == tn) {
        double gg = 0, gx = 0;
        for (int e2 = 0; e2 < 3; ++e2) {
            double x[3], gi[3], gj[3], ngj[3];
            for (int d = 0; d < 3; ++d) {
                x[d] = 0.5 * (Tm.p[e2][d] + Tm.p[(e2 + 1) % 3][d]);
                gi[d] = x[d] - Tm.p[i][d];
                gj[d] = x[d] - Tm.p[j][d];
            }
            cross3(Tm.n, gj, ngj);
            gg += dot3(gi, gj) / 3.0;
            gx += dot3(gi, ngj) / 3.0;
        }
        G = cm * cn * gg * Tm.area;
        X = cm * cn * gx * Tm.area;
    }
    const double gA = (mode == 0) ? 1.0 : 0.25;
    if (mode == 0) {
        atomicAdd(out + 4 * o + 0, (T)(P.x - gA * G));
        atomicAdd(out + 4 * o + 1, (T)P.y);
        atomicAdd(out + 4 * o + 2, (T)(Q.x - 0.5 * X));
        atomicAdd(out + 4 * o + 3, (T)Q.y);
    } else {
        atomicAdd(out + 2 * o + 0, (T)(P.x - gA * G));
        atomicAdd(out + 2 * o + 1, (T)P.y);
    }
}

// One CTA per near block (test leaf box b, source box s); threads loop over the block's
// entries, column-major (source column outer, test row inner).
template <typename T, typename KT>
__global__ void k_near_fill(int nblk, const int* __restrict__ blk_box, const int* __restrict__ near_ptr,
                            const int* __restrict__ near_src,
                            const int64_t* __restrict__ near_blk, const int* __restrict__ leaf_start,
                            const int* __restrict__ rwg_t, const int* __restrict__ rwg_l, const double* __restrict__ rwg_len,
                            const double* __restrict__ tri, const double* __restrict__ nrm, const double* __restrict__ area,
                            const int* __restrict__ vid, KT k, int mode, T* __restrict__ out) {
    int q = blockIdx.x;
    if (q >= nblk) return;
    int b = blk_box[q], s = near_src[q];
    int m0 = leaf_start[b], mb = leaf_start[b + 1] - m0;
    int n0 = leaf_start[s], nbs = leaf_start[s + 1] - n0;
    // the test box's blocks form one row-major mb x ncol segment (columns: near source RWGs)
    const int64_t seg = near_blk[near_ptr[b]];
    const int ncol = (int)((near_blk[near_ptr[b + 1]] - seg) / mb);
    const int c0 = (int)((near_blk[q] - seg) / mb);
    int cnt = mb * nbs;
    for (int e = threadIdx.x; e < cnt; e += blockDim.x) {
        int ml = e % mb, nl = e / mb;
        int m = m0 + ml, n = n0 + nl;
        zd P = zmk(0, 0), Q = zmk(0, 0), Lm = zmk(0, 0), Km = zmk(0, 0);
        double G = 0, X = 0;
        for (int sm = 0; sm < 2; ++sm) {
            dtri Tm;
            int tm = rwg_t[2 * m + sm], i = rwg_l[2 * m + sm];
            load_tri(tri, nrm, area, vid, tm, Tm);
            double cm = (sm == 0 ? 1.0 : -1.0) * rwg_len[m] / (2.0 * Tm.area);
            for (int sn = 0; sn < 2; ++sn) {
                dtri Tn;
                int tn = rwg_t[2 * n + sn], j = rwg_l[2 * n + sn];
                load_tri(tri, nrm, area, vid, tn, Tn);
                double cn = (sn == 0 ? 1.0 : -1.0) * rwg_len[n] / (2.0 * Tn.area);
                raw4 r = tri_pair(Tm, i, Tn, j, k);
                double c = 0.5 * cm * cn;
                P = zadd(P, zscale(zadd(r.L, r.NK), c));
                Q = zadd(Q, zscale(zadd(r.NL, zscale(r.K, -1.0)), c));
                Lm = zadd(Lm, zscale(r.L, cm * cn));
                Km = zadd(Km, zscale(r.K, cm * cn));
                if (tm == tn) {
                    // Gram integrals are exact with the edge-midpoint rule (degree-2 integrand)
                    double gg = 0, gx = 0;
                    for (int e2 = 0; e2 < 3; ++e2) {
                        double x[3], gi[3], gj[3], ngj[3];
                        for (int d = 0; d < 3; ++d) {
                            x[d] = 0.5 * (Tm.p[e2][d] + Tm.p[(e2 + 1) % 3][d]);
                            gi[d] = x[d] - Tm.p[i][d];
                            gj[d] = x[d] - Tm.p[j][d];
                        }
                        cross3(Tm.n, gj, ngj);
                        gg += dot3(gi, gj) / 3.0;
                        gx += dot3(gi, ngj) / 3.0;
                    }
                    G += cm * cn * gg * Tm.area;
                    X += cm * cn * gx * Tm.area;
                }
            }
        }
        // A = P - g G,  B = Q - X/2  (g = 1 for the C block, 1/4 for PEC); one medium of the
        // two-region form (mode 3): A = <f_m, L f_n>, B = <f_m, Kbar f_n>, no identity terms
        double gA = (mode == 0) ? 1.0 : 0.25;
        zd A = zmk(P.x - gA * G, P.y);
        zd B = zmk(Q.x - 0.5 * X, Q.y);
        if (mode == 3) {
            A = Lm;
            B = Km;
        }
        int64_t o = seg + (int64_t)ml * ncol + c0 + nl;
        if (mode == 0 || mode == 3) {
            out[4 * o + 0] = (T)A.x;
            out[4 * o + 1] = (T)A.y;
            out[4 * o + 2] = (T)B.x;
            out[4 * o + 3] = (T)B.y;
        } else {
            out[2 * o + 0] = (T)A.x;
            out[2 * o + 1] = (T)A.y;
        }
    }
}

// Leaf patterns, one thread per (tree RWG n, direction kk):
//   F_n(k)  = int f_n exp(+jk khat.(r - c)) ds,  RX_n(k) = int (n x f_n) exp(-jk khat.(r - c)) ds,
// theta and phi components, c = center of the RWG's leaf box.  f_n is real, so the pattern at
// the antipode -khat is the conjugate vector, and theta-hat(-khat) = theta-hat(khat),
// phi-hat(-khat) = -phi-hat(khat): only the first K/2 directions (theta-major: one of each
// antipodal pair) are stored, [N][K/2][2].
// With a complex wavenumber (ki != 0) the identities behind the packing fail (R_n is no longer
// conj F_n): every direction is stored, Kh = K, and exp(+-jk khat.(r - c)) carries the decay.
template <typename T>
__global__ void k_patterns(int N, int K, int nph, const double* __restrict__ theta, const int* __restrict__ leaf_of,
                           const double* __restrict__ centers, const int* __restrict__ rwg_t, const int* __restrict__ rwg_l,
                           const double* __restrict__ rwg_len, const double* __restrict__ tri, const double* __restrict__ nrm,
                           const double* __restrict__ area, double k, double ki, int full, T* __restrict__ F,
                           T* __restrict__ RX) {
    const int Kh = full ? K : K / 2;
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)N * Kh) return;
    int n = (int)(idx / Kh), kk = (int)(idx % Kh);
    int it = kk / nph, jp = kk % nph;
    double th = theta[it], ph = 2.0 * kPiD * jp / nph;
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    double kh[3] = {st * cp, st * sp, ct}, tv[3] = {ct * cp, ct * sp, -st}, pv[3] = {-sp, cp, 0.0};
    const double* c = centers + 3 * leaf_of[n];
    zd Ft = zmk(0, 0), Fp = zmk(0, 0), Rt = zmk(0, 0), Rp = zmk(0, 0);
    for (int s = 0; s < 2; ++s) {
        int t = rwg_t[2 * n + s], l = rwg_l[2 * n + s];
        const double* P = tri + 9 * t;
        const double* nn = nrm + 3 * t;
        double cf = (s == 0 ? 1.0 : -1.0) * rwg_len[n] / (2.0 * area[t]) * area[t];
        for (int q = 0; q < 7; ++q) {
            double b0, b1, b2, w;
            radon7(q, b0, b1, b2, w);
            double r[3], f[3];
            for (int d = 0; d < 3; ++d) {
                r[d] = b0 * P[d] + b1 * P[3 + d] + b2 * P[6 + d];
                f[d] = cf * w * (r[d] - P[3 * l + d]);
            }
            double nf[3];
            cross3(nn, f, nf);
            const double a = kh[0] * (r[0] - c[0]) + kh[1] * (r[1] - c[1]) + kh[2] * (r[2] - c[2]);
            zd e = zexpj(k * a);
            zd ec = zmk(e.x, -e.y);
            if (ki != 0.0) {   // exp(+jka) = exp(jk'a) exp(-k''a), exp(-jka) = exp(-jk'a) exp(k''a)
                e = zscale(e, exp(-ki * a));
                ec = zscale(ec, exp(ki * a));
            }
            Ft = zadd(Ft, zscale(e, dot3(f, tv)));
            Fp = zadd(Fp, zscale(e, dot3(f, pv)));
            Rt = zadd(Rt, zscale(ec, dot3(nf, tv)));
            Rp = zadd(Rp, zscale(ec, dot3(nf, pv)));
        }
    }
    int64_t o = 2 * idx;
    F[2 * o + 0] = (T)Ft.x; F[2 * o + 1] = (T)Ft.y; F[2 * o + 2] = (T)Fp.x; F[2 * o + 3] = (T)Fp.y;
    RX[2 * o + 0] = (T)Rt.x; RX[2 * o + 1] = (T)Rt.y; RX[2 * o + 2] = (T)Rp.x; RX[2 * o + 3] = (T)Rp.y;
}

// Translation operators of one level with the quadrature weight folded in:
//   T(khat; X) = w(khat) sum_{l=0}^{L} (-j)^l (2l+1) h_l^(2)(k|X|) P_l(khat . Xhat),
// one thread per (offset code o in 7^3, direction kk); near offsets are left zero.
template <typename T>
__global__ void k_translations(int K, int nph, int L, const double* __restrict__ theta, const double* __restrict__ wth,
                               double a, const int* __restrict__ dist_idx, const double* __restrict__ hank, T* __restrict__ out) {
    int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= (int64_t)343 * K) return;
    int o = (int)(idx / K), kk = (int)(idx % K);
    int ox = o / 49 - 3, oy = (o / 7) % 7 - 3, oz = o % 7 - 3;
    zd acc = zmk(0, 0);
    int di = dist_idx[o];
    if (di >= 0) {
        int it = kk / nph, jp = kk % nph;
        double th = theta[it], ph = 2.0 * kPiD * jp / nph;
        double st, ct, sp, cp;
        sincos(th, &st, &ct);
        sincos(ph, &sp, &cp);
        double X[3] = {ox * a, oy * a, oz * a};
        double Xn = sqrt(dot3(X, X));
        double cg = (st * cp * X[0] + st * sp * X[1] + ct * X[2]) / Xn;
        const double* hk = hank + 2 * (size_t)di * (L + 1);
        double p0 = 1.0, p1 = cg;
        for (int l = 0; l <= L; ++l) {
            double pl = (l == 0) ? p0 : p1;
            if (l >= 2) {
                double pn = ((2.0 * l - 1.0) * cg * p1 - (l - 1.0) * p0) / l;
                p0 = p1;
                p1 = pn;
                pl = pn;
            }
            // (-j)^l
            zd ph_l = (l % 4 == 0) ? zmk(1, 0) : (l % 4 == 1) ? zmk(0, -1) : (l % 4 == 2) ? zmk(-1, 0) : zmk(0, 1);
            zd term = zmul(ph_l, zmk(hk[2 * l], hk[2 * l + 1]));
            acc = zadd(acc, zscale(term, (2.0 * l + 1.0) * pl));
        }
        double w = wth[it] * 2.0 * kPiD / nph;
        acc = zscale(acc, w);
    }
    out[2 * idx] = (T)acc.x;
    out[2 * idx + 1] = (T)acc.y;
}

// exp(+jk khat.(c_child - c_parent)) for the 8 child octants of a parent level
template <typename T>
__global__ void k_shifts(int K, int nph, const double* __restrict__ theta, double half_child, double k, double ki,
                         T* __restrict__ out) {
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 8 * K) return;
    int o = idx / K, kk = idx % K;
    int it = kk / nph, jp = kk % nph;
    double th = theta[it], ph = 2.0 * kPiD * jp / nph;
    double st, ct, sp, cp;
    sincos(th, &st, &ct);
    sincos(ph, &sp, &cp);
    double d[3] = {((o & 1) ? 1.0 : -1.0) * half_child, ((o & 2) ? 1.0 : -1.0) * half_child, ((o & 4) ? 1.0 : -1.0) * half_child};
    const double a = st * cp * d[0] + st * sp * d[1] + ct * d[2];
    zd e = zexpj(k * a);
    if (ki != 0.0) e = zscale(e, exp(-ki * a));
    out[2 * idx] = (T)e.x;
    out[2 * idx + 1] = (T)e.y;
}

// spherical Hankel functions of the second kind h_l^(2)(x) = j_l(x) - j y_l(x), l = 0..L
void hankel2(int L, double x, std::vector<double>& out) {
    out.assign(2 * (L + 1), 0.0);
    std::vector<double> y(L + 2), jv(L + 2);
    y[0] = -std::cos(x) / x;
    if (L >= 1) y[1] = -std::cos(x) / (x * x) - std::sin(x) / x;
    for (int l = 1; l < L; ++l) y[l + 1] = (2.0 * l + 1.0) / x * y[l] - y[l - 1];
    // j_l by downward recurrence (Miller), normalised with j_0 = sin x / x
    int start = L + 40 + (int)(1.2 * x);
    std::vector<double> f(start + 2, 0.0);
    f[start + 1] = 0.0;
    f[start] = 1.0;
    for (int l = start; l >= 1; --l) {
        f[l - 1] = (2.0 * l + 1.0) / x * f[l] - f[l + 1];
        if (std::fabs(f[l - 1]) > 1e100) {
            for (int m = l - 1; m <= start; ++m) f[m] *= 1e-100;
        }
    }
    // normalise with sum_l (2l+1) j_l(x)^2 = 1 (j_0 alone vanishes at x = n pi); the sign
    // follows whichever of j_0, j_1 is larger in magnitude
    double ss = 0.0;
    for (int l = 0; l <= start; ++l) ss += (2.0 * l + 1.0) * f[l] * f[l];
    double s = 1.0 / std::sqrt(ss);
    double j0 = std::sin(x) / x, j1 = std::sin(x) / (x * x) - std::cos(x) / x;
    if (std::fabs(j0) >= std::fabs(j1)) { if (j0 * f[0] < 0) s = -s; }
    else { if (j1 * f[1] < 0) s = -s; }
    for (int l = 0; l <= L; ++l) jv[l] = f[l] * s;
    for (int l = 0; l <= L; ++l) {
        out[2 * l] = jv[l];
        out[2 * l + 1] = -y[l];
    }
}

// h_l^(2)(z) for complex z (a lossy medium's k |X|): y_l by upward recurrence, j_l by Miller's
// downward recurrence normalised with the closed form of the larger of j_0, j_1 (neither
// vanishes off the real axis, and no sum that cancels is formed).
void hankel2c(int L, std::complex<double> z, std::vector<double>& out) {
    typedef std::complex<double> C;
    out.assign(2 * (L + 1), 0.0);
    const C sz = std::sin(z), cz = std::cos(z);
    std::vector<C> y(L + 2);
    y[0] = -cz / z;
    if (L >= 1) y[1] = -cz / (z * z) - sz / z;
    for (int l = 1; l < L; ++l) y[l + 1] = (2.0 * l + 1.0) / z * y[l] - y[l - 1];
    const int start = L + 40 + (int)(1.2 * std::abs(z));
    std::vector<C> f(start + 2, C(0.0));
    f[start] = 1.0;
    for (int l = start; l >= 1; --l) {
        f[l - 1] = (2.0 * l + 1.0) / z * f[l] - f[l + 1];
        if (std::abs(f[l - 1]) > 1e100)
            for (int m = l - 1; m <= start; ++m) f[m] *= 1e-100;
    }
    const C j0 = sz / z, j1 = sz / (z * z) - cz / z;
    const C s = std::abs(j0) >= std::abs(j1) ? j0 / f[0] : j1 / f[1];
    for (int l = 0; l <= L; ++l) {
        const C h = f[l] * s - C(0.0, 1.0) * y[l];
        out[2 * l] = h.real();
        out[2 * l + 1] = h.imag();
    }
}

}  // namespace

void bi_translation_series(const bi_handle_s* h, int l, std::vector<int>& dist_idx, std::vector<double>& hk) {
    const level_t& L = h->lev[l];
    // distinct offset lengths |X|^2 = a^2 (ox^2 + oy^2 + oz^2)
    dist_idx.assign(343, -1);
    std::vector<int> sq_of;
    for (int o = 0; o < 343; ++o) {
        int ox = o / 49 - 3, oy = (o / 7) % 7 - 3, oz = o % 7 - 3;
        if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) continue;
        int sq = ox * ox + oy * oy + oz * oz;
        auto it = std::find(sq_of.begin(), sq_of.end(), sq);
        if (it == sq_of.end()) {
            dist_idx[o] = (int)sq_of.size();
            sq_of.push_back(sq);
        } else {
            dist_idx[o] = (int)(it - sq_of.begin());
        }
    }
    hk.clear();
    hk.reserve(sq_of.size() * 2 * (L.L + 1));
    for (int sq : sq_of) {
        std::vector<double> one;
        const double X = L.a * std::sqrt((double)sq);
        if (h->ki != 0.0) hankel2c(L.L, std::complex<double>(h->k * X, h->ki * X), one);
        else hankel2(L.L, h->k * X, one);
        hk.insert(hk.end(), one.begin(), one.end());
    }
}

// ---------------------------------------------------------------------------------
void bi_device_geometry(bi_handle_s* h, const double* V, const int* Tm) {
    const int nt = h->nt, N = h->N;
    std::vector<double> tri(9 * (size_t)nt), nrm(3 * (size_t)nt), area(nt);
    for (int t = 0; t < nt; ++t) {
        for (int a = 0; a < 3; ++a)
            for (int d = 0; d < 3; ++d) tri[9 * t + 3 * a + d] = V[3 * Tm[3 * t + a] + d];
        double e1[3], e2[3], c[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = tri[9 * t + 3 + d] - tri[9 * t + d];
            e2[d] = tri[9 * t + 6 + d] - tri[9 * t + d];
        }
        c[0] = e1[1] * e2[2] - e1[2] * e2[1];
        c[1] = e1[2] * e2[0] - e1[0] * e2[2];
        c[2] = e1[0] * e2[1] - e1[1] * e2[0];
        double a2 = std::sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        for (int d = 0; d < 3; ++d) nrm[3 * t + d] = c[d] / a2;
        area[t] = 0.5 * a2;
    }
    std::vector<int> rt(2 * (size_t)N), rl(2 * (size_t)N), leaf_of(N);
    std::vector<double> len(N);
    for (int ti = 0; ti < N; ++ti) {
        int n = h->perm[ti];
        rt[2 * ti] = h->tplus[n];
        rt[2 * ti + 1] = h->tminus[n];
        rl[2 * ti] = h->lplus[n];
        rl[2 * ti + 1] = h->lminus[n];
        const double* a = V + 3 * h->edges[2 * n];
        const double* b = V + 3 * h->edges[2 * n + 1];
        len[ti] = std::sqrt((a[0] - b[0]) * (a[0] - b[0]) + (a[1] - b[1]) * (a[1] - b[1]) + (a[2] - b[2]) * (a[2] - b[2]));
    }
    const level_t& LF = h->lev[h->leaf];
    for (int b = 0; b < LF.nbox; ++b)
        for (int t = h->leaf_start[b]; t < h->leaf_start[b + 1]; ++t) leaf_of[t] = b;
    h->d_tri = h->upload(tri);
    h->d_tri_n = h->upload(nrm);
    h->d_tri_area = h->upload(area);
    h->d_tri_vid = h->upload(h->tri_vid_host);
    h->d_rwg_t = h->upload(rt);
    h->d_rwg_l = h->upload(rl);
    h->d_rwg_len = h->upload(len);
    h->d_leaf_of = h->upload(leaf_of);
    h->d_perm = h->upload(h->perm);
    h->d_leaf_start = h->upload(h->leaf_start);
    h->d_near_ptr = h->upload(h->near_ptr);
    h->d_near_src = h->upload(h->near_src);
    h->d_near_blk = h->upload(h->near_blk);
    {
        // streaming near kernel work items: up to 16 rows (8 warps x 2 rows) of one test box
        std::vector<int> work;
        for (int b = 0; b < LF.nbox; ++b)
            for (int r0 = 0; r0 < h->leaf_start[b + 1] - h->leaf_start[b]; r0 += 16) {
                work.push_back(b);
                work.push_back(r0);
            }
        h->near_nwork = (int)(work.size() / 2);
        h->d_near_work = h->upload(work);
        // column offset of every near entry inside its test box's segment, and the segment
        // width of every box (int32: the product kernels need no 64-bit division)
        std::vector<int> col0(h->near_src.size()), ncol(LF.nbox);
        for (int b = 0; b < LF.nbox; ++b) {
            const int mb = h->leaf_start[b + 1] - h->leaf_start[b];
            const int64_t seg = h->near_blk[h->near_ptr[b]];
            for (int q = h->near_ptr[b]; q < h->near_ptr[b + 1]; ++q) col0[q] = (int)((h->near_blk[q] - seg) / mb);
            ncol[b] = (int)((h->near_blk[h->near_ptr[b + 1]] - seg) / mb);
        }
        h->d_near_col0 = h->upload(col0);
        h->d_near_ncol = h->upload(ncol);
    }
    std::vector<double> cen = LF.center;
    h->d_leaf_center = h->upload(cen);
    h->tri_host = tri;
    h->tri_n_host = nrm;
    h->tri_area_host = area;
    h->rwg_len_user.resize(N);
    for (int ti = 0; ti < N; ++ti) h->rwg_len_user[h->perm[ti]] = len[ti];
}

static void upload_rules() {
    rules_c R{};
    std::vector<double> x, w;
    // composite rule: 4 sub-triangles (midpoint subdivision) x 7-point Radon
    {
        const double s15 = std::sqrt(15.0);
        const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
        double bb[7][3], ww[7];
        bb[0][0] = bb[0][1] = bb[0][2] = 1.0 / 3.0;
        ww[0] = 9.0 / 40.0;
        for (int q = 1; q < 7; ++q) {
            double a = (q <= 3) ? a1 : a2;
            ww[q] = (q <= 3) ? (155.0 - s15) / 1200.0 : (155.0 + s15) / 1200.0;
            int r = (q - 1) % 3;
            bb[q][0] = bb[q][1] = bb[q][2] = a;
            bb[q][r] = 1.0 - 2.0 * a;
        }
        // sub-triangles in barycentric coordinates of the parent
        const double sub[4][3][3] = {{{1, 0, 0}, {.5, .5, 0}, {.5, 0, .5}},
                                     {{.5, .5, 0}, {0, 1, 0}, {0, .5, .5}},
                                     {{.5, 0, .5}, {0, .5, .5}, {0, 0, 1}},
                                     {{.5, .5, 0}, {0, .5, .5}, {.5, 0, .5}}};
        int k = 0;
        for (int s = 0; s < 4; ++s)
            for (int q = 0; q < 7; ++q, ++k) {
                for (int d = 0; d < 3; ++d)
                    R.near_b[k][d] = bb[q][0] * sub[s][0][d] + bb[q][1] * sub[s][1][d] + bb[q][2] * sub[s][2][d];
                R.near_w[k] = ww[q] / 4.0;
            }
    }
    gauss_legendre(8, x, w);
    std::vector<double> g(8), gw(8);
    for (int i = 0; i < 8; ++i) { g[i] = 0.5 * (x[i] + 1.0); gw[i] = 0.5 * w[i]; }
    // graded toward the edge (v0, v1): distance t = s^3; along the edge a smoothstep map
    {
        int k = 0;
        for (int a = 0; a < 8; ++a)
            for (int c = 0; c < 8; ++c, ++k) {
                double s = g[a], t = s * s * s, jt = 3 * s * s;
                double u = g[c], sg = u * u * (3 - 2 * u), js = 6 * u * (1 - u);
                R.edge_b[k][2] = t;
                R.edge_b[k][1] = (1 - t) * sg;
                R.edge_b[k][0] = (1 - t) * (1 - sg);
                R.edge_w[k] = 2.0 * gw[a] * gw[c] * (1 - t) * jt * js;
            }
    }
    // graded toward vertex v0: radius u = s^2 (Duffy map with a square-root grading)
    {
        int k = 0;
        for (int a = 0; a < 8; ++a)
            for (int c = 0; c < 8; ++c, ++k) {
                double s = g[a], u = s * s, ju = 2 * s;
                double sg = g[c];
                R.vert_b[k][0] = 1 - u;
                R.vert_b[k][1] = u * (1 - sg);
                R.vert_b[k][2] = u * sg;
                R.vert_w[k] = 2.0 * gw[a] * gw[c] * u * ju;
            }
    }
    for (int q = 0; q < 8; ++q) {
        double u = g[q];
        R.line_x[q] = u * u * (3 - 2 * u);
        R.line_w[q] = gw[q] * 6 * u * (1 - u);
    }
    CU(cudaMemcpyToSymbol(c_rules, &R, sizeof(R)));
}

void bi_fill_near(bi_handle_s* h) {
    upload_rules();
    const level_t& LF = h->lev[h->leaf];
    int nblk = h->near_ptr[LF.nbox];
    std::vector<int> blk_box(nblk);
    for (int b = 0; b < LF.nbox; ++b)
        for (int q = h->near_ptr[b]; q < h->near_ptr[b + 1]; ++q) blk_box[q] = b;
    int* d_blk_box = h->upload(blk_box);
    size_t per = (h->prm.op_mode == 0 || h->prm.op_mode == 3 ? 2 : 1) * h->csize;
    h->d_near = h->alloc(per * (size_t)std::max<int64_t>(h->near_nnz, 1));
    const char* env_fill = std::getenv("BI_NEAR_FILL_SINGLE_PASS");
    const bool two_pass = !(env_fill && env_fill[0] == '1') && h->ki == 0.0 && h->prm.op_mode != 3;
    if (nblk > 0 && two_pass) {
        // per-class lists of singular / near-singular triangle pairs, counted first and sized exactly
        unsigned long long* d_count = nullptr;
        CU(cudaMallocAsync((void**)&d_count, 12 * sizeof(unsigned long long), h->stream));
        CU(cudaMemsetAsync(d_count, 0, 12 * sizeof(unsigned long long), h->stream));
        k_near_count<<<nblk, 128, 0, h->stream>>>(nblk, d_blk_box, h->d_near_src, h->d_leaf_start, h->d_rwg_t, h->d_tri,
                                                   h->d_tri_n, h->d_tri_area, h->d_tri_vid, d_count);
        CU(cudaGetLastError());
        unsigned long long capv[4], basev[4];
        CU(cudaMemcpyAsync(capv, d_count, sizeof(capv), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        unsigned long long tot_cap = 0;
        for (int c = 0; c < 4; ++c) { basev[c] = tot_cap; tot_cap += capv[c]; }
        CU(cudaMemcpyAsync(d_count + 4, capv, sizeof(capv), cudaMemcpyHostToDevice, h->stream));
        CU(cudaMemcpyAsync(d_count + 8, basev, sizeof(basev), cudaMemcpyHostToDevice, h->stream));
        CU(cudaMemsetAsync(d_count, 0, 4 * sizeof(unsigned long long), h->stream));
        special_item* d_list = nullptr;
        CU(cudaMallocAsync((void**)&d_list, sizeof(special_item) * std::max<unsigned long long>(tot_cap, 1), h->stream));
        auto t0 = std::chrono::steady_clock::now();
        if (h->prec == 0)
            k_near_regular<double><<<nblk, 128, 0, h->stream>>>(nblk, d_blk_box, h->d_near_ptr, h->d_near_src, h->d_near_blk,
                                                                 h->d_leaf_start, h->d_rwg_t, h->d_rwg_l, h->d_rwg_len,
                                                                 h->d_tri, h->d_tri_n, h->d_tri_area, h->d_tri_vid, h->k,
                                                                 h->prm.op_mode, (double*)h->d_near, d_list, d_count, d_count + 4, d_count + 8);
        else
            k_near_regular<float><<<nblk, 128, 0, h->stream>>>(nblk, d_blk_box, h->d_near_ptr, h->d_near_src, h->d_near_blk,
                                                                h->d_leaf_start, h->d_rwg_t, h->d_rwg_l, h->d_rwg_len,
                                                                h->d_tri, h->d_tri_n, h->d_tri_area, h->d_tri_vid, h->k,
                                                                h->prm.op_mode, (float*)h->d_near, d_list, d_count, d_count + 4, d_count + 8);
        CU(cudaGetLastError());
        unsigned long long nlist[4] = {0, 0, 0, 0};
        CU(cudaMemcpyAsync(nlist, d_count, sizeof(nlist), cudaMemcpyDeviceToHost, h->stream));
        CU(cudaStreamSynchronize(h->stream));
        auto t1 = std::chrono::steady_clock::now();
        unsigned long long total = 0;
        for (int c = 0; c < 4; ++c) {
            if (nlist[c] != capv[c]) throw bi_error{BI_ERR_CUDA, "near-field special list count mismatch"};
            total += nlist[c];
            if (nlist[c] == 0) continue;
            const unsigned nb = (unsigned)((nlist[c] + 127) / 128);
            if (h->prec == 0)
                k_near_special<double><<<nb, 128, 0, h->stream>>>(nlist[c], d_list + basev[c], h->d_rwg_t, h->d_rwg_l,
                                                                  h->d_rwg_len, h->d_tri, h->d_tri_n, h->d_tri_area,
                                                                  h->d_tri_vid, h->k, h->prm.op_mode, (double*)h->d_near);
            else
                k_near_special<float><<<nb, 128, 0, h->stream>>>(nlist[c], d_list + basev[c], h->d_rwg_t, h->d_rwg_l,
                                                                 h->d_rwg_len, h->d_tri, h->d_tri_n, h->d_tri_area,
                                                                 h->d_tri_vid, h->k, h->prm.op_mode, (float*)h->d_near);
            CU(cudaGetLastError());
        }
        CU(cudaStreamSynchronize(h->stream));
        auto t2 = std::chrono::steady_clock::now();
        CU(cudaFreeAsync(d_list, h->stream));
        CU(cudaFreeAsync(d_count, h->stream));
        h->info.setup_near_regular_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        h->info.setup_near_special_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
        h->info.near_special_entries = (int64_t)total;
    } else if (nblk > 0 && h->ki != 0.0) {
        // complex wavenumber: every triangle pair in FP64 (singularity extraction for close pairs)
        const zd kc{h->k, h->ki};
        if (h->prec == 0)
            k_near_fill<double, zd><<<nblk, 128, 0, h->stream>>>(nblk, d_blk_box, h->d_near_ptr, h->d_near_src, h->d_near_blk,
                                                                  h->d_leaf_start, h->d_rwg_t, h->d_rwg_l, h->d_rwg_len,
                                                                  h->d_tri, h->d_tri_n, h->d_tri_area, h->d_tri_vid, kc,
                                                                  h->prm.op_mode, (double*)h->d_near);
        else
            k_near_fill<float, zd><<<nblk, 128, 0, h->stream>>>(nblk, d_blk_box, h->d_near_ptr, h->d_near_src, h->d_near_blk,
                                                                 h->d_leaf_start, h->d_rwg_t, h->d_rwg_l, h->d_rwg_len,
                                                                 h->d_tri, h->d_tri_n, h->d_tri_area, h->d_tri_vid, kc,
                                                                 h->prm.op_mode, (float*)h->d_near);
        CU(cudaGetLastError());
    } else if (nblk > 0) {
        if (h->prec == 0)
            k_near_fill<double, double><<<nblk, 128, 0, h->stream>>>(nblk, d_blk_box, h->d_near_ptr, h->d_near_src, h->d_near_blk, h->d_leaf_start,
                                                              h->d_rwg_t, h->d_rwg_l, h->d_rwg_len, h->d_tri, h->d_tri_n,
                                                              h->d_tri_area, h->d_tri_vid, h->k, h->prm.op_mode,
                                                              (double*)h->d_near);
        else
            k_near_fill<float, double><<<nblk, 128, 0, h->stream>>>(nblk, d_blk_box, h->d_near_ptr, h->d_near_src, h->d_near_blk, h->d_leaf_start,
                                                             h->d_rwg_t, h->d_rwg_l, h->d_rwg_len, h->d_tri, h->d_tri_n,
                                                             h->d_tri_area, h->d_tri_vid, h->k, h->prm.op_mode,
                                                             (float*)h->d_near);
        CU(cudaGetLastError());
    }
    // Gram correction of the M rows (C block): (X/2) x_J - (G/2) x_M for RWGs sharing a triangle.
    // The Gram integrands are quadratic on a flat triangle: the edge-midpoint rule is exact.
    if (h->prm.op_mode == 0) {
        const int N = h->N;
        std::vector<int> inv(N);
        for (int t = 0; t < N; ++t) inv[h->perm[t]] = t;
        std::vector<int> trw(3 * (size_t)h->nt, -1);
        std::vector<double> tcf(3 * (size_t)h->nt, 0.0);
        for (int n = 0; n < N; ++n) {
            int t = h->tplus[n], a = h->lplus[n];
            trw[3 * t + a] = inv[n];
            tcf[3 * t + a] = h->rwg_len_user[n] / (2.0 * h->tri_area_host[t]);
            t = h->tminus[n];
            a = h->lminus[n];
            trw[3 * t + a] = inv[n];
            tcf[3 * t + a] = -h->rwg_len_user[n] / (2.0 * h->tri_area_host[t]);
        }
        std::vector<std::vector<int>> rc(N);
        std::vector<std::vector<double>> rg(N), rx(N);
        for (int t = 0; t < h->nt; ++t) {
            const double* P = &h->tri_host[9 * (size_t)t];
            const double* nn = &h->tri_n_host[3 * (size_t)t];
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    int m = trw[3 * t + i], n = trw[3 * t + j];
                    if (m < 0 || n < 0) continue;
                    double gg = 0, gx = 0;
                    for (int e = 0; e < 3; ++e) {
                        double x[3], gi[3], gj[3];
                        for (int d = 0; d < 3; ++d) {
                            x[d] = 0.5 * (P[3 * e + d] + P[3 * ((e + 1) % 3) + d]);
                            gi[d] = x[d] - P[3 * i + d];
                            gj[d] = x[d] - P[3 * j + d];
                        }
                        double ngj[3] = {nn[1] * gj[2] - nn[2] * gj[1], nn[2] * gj[0] - nn[0] * gj[2], nn[0] * gj[1] - nn[1] * gj[0]};
                        gg += (gi[0] * gj[0] + gi[1] * gj[1] + gi[2] * gj[2]) / 3.0;
                        gx += (gi[0] * ngj[0] + gi[1] * ngj[1] + gi[2] * ngj[2]) / 3.0;
                    }
                    double c = tcf[3 * t + i] * tcf[3 * t + j] * h->tri_area_host[t];
                    size_t pos = 0;
                    while (pos < rc[m].size() && rc[m][pos] != n) ++pos;
                    if (pos == rc[m].size()) { rc[m].push_back(n); rg[m].push_back(0); rx[m].push_back(0); }
                    rg[m][pos] += c * gg;
                    rx[m][pos] += c * gx;
                }
        }
        // column of each Gram neighbour inside its test box's near segment (x is staged there)
        const level_t& LFb = h->lev[h->leaf];
        std::vector<int> leaf_of_t(N);
        for (int b = 0; b < LFb.nbox; ++b)
            for (int t = h->leaf_start[b]; t < h->leaf_start[b + 1]; ++t) leaf_of_t[t] = b;
        std::vector<int> ptr(N + 1, 0), col, segc;
        std::vector<double> val;
        for (int m = 0; m < N; ++m) {
            const int b = leaf_of_t[m];
            const int mb = h->leaf_start[b + 1] - h->leaf_start[b];
            const int64_t seg = h->near_blk[h->near_ptr[b]];
            for (size_t q = 0; q < rc[m].size(); ++q) {
                const int n = rc[m][q], sb = leaf_of_t[n];
                int c = -1;
                for (int qq = h->near_ptr[b]; qq < h->near_ptr[b + 1]; ++qq)
                    if (h->near_src[qq] == sb) c = (int)((h->near_blk[qq] - seg) / mb) + (n - h->leaf_start[sb]);
                if (c < 0) throw bi_error{BI_ERR_MESH, "Gram neighbour outside the near field (mesh too coarse for the leaf box)"};
                col.push_back(n);
                segc.push_back(c);
                val.push_back(rg[m][q]);
                val.push_back(rx[m][q]);
            }
            ptr[m + 1] = (int)col.size();
        }
        h->d_gram_ptr = h->upload(ptr);
        h->d_gram_col = h->upload(col);
        h->d_gram_seg = h->upload(segc);
        if (h->prec == 0) {
            h->d_gram_val = h->upload(val);
        } else {
            std::vector<float> vf(val.begin(), val.end());
            h->d_gram_val = h->upload(vf);
        }
    }
}

void bi_fill_patterns(bi_handle_s* h) {
    if (h->leaf < 2) return;
    const level_t& LF = h->lev[h->leaf];
    double* d_theta = h->upload(LF.theta);
    // stored directions: all of them at complex k and for one medium of the two-region form
    const int full = (h->ki != 0.0 || h->prm.op_mode == 3) ? 1 : 0;
    const int Ks = full ? LF.K : LF.K / 2;
    size_t nel = (size_t)h->N * Ks * 2;
    h->d_F = h->alloc(nel * h->csize);
    h->d_RX = h->alloc(nel * h->csize);
    int64_t tot = (int64_t)h->N * Ks;
    int th = 256;
    int64_t nb = (tot + th - 1) / th;
    if (h->prec == 0)
        k_patterns<double><<<(unsigned)nb, th, 0, h->stream>>>(h->N, LF.K, LF.nph, d_theta, h->d_leaf_of, h->d_leaf_center,
                                                                h->d_rwg_t, h->d_rwg_l, h->d_rwg_len, h->d_tri, h->d_tri_n,
                                                                h->d_tri_area, h->k, h->ki, full, (double*)h->d_F, (double*)h->d_RX);
    else
        k_patterns<float><<<(unsigned)nb, th, 0, h->stream>>>(h->N, LF.K, LF.nph, d_theta, h->d_leaf_of, h->d_leaf_center,
                                                               h->d_rwg_t, h->d_rwg_l, h->d_rwg_len, h->d_tri, h->d_tri_n,
                                                               h->d_tri_area, h->k, h->ki, full, (float*)h->d_F, (float*)h->d_RX);
    CU(cudaGetLastError());
}

void bi_fill_translations(bi_handle_s* h) {
    for (int l = 2; l <= h->leaf; ++l) {
        level_t& L = h->lev[l];
        std::vector<int> dist_idx;
        std::vector<double> hk;
        bi_translation_series(h, l, dist_idx, hk);
        double* d_theta = h->upload(L.theta);
        double* d_wth = h->upload(L.wtheta);
        int* d_di = h->upload(dist_idx);
        double* d_hk = h->upload(hk);
        // 343 offset codes plus a zero row (code 343) that lets a translation kernel run every
        // child slot without a branch: a slot without an interaction reads zeros
        L.d_T = h->alloc((size_t)344 * L.K * h->csize);
        CU(cudaMemsetAsync((char*)L.d_T + (size_t)343 * L.K * h->csize, 0, (size_t)L.K * h->csize, h->stream));
        int64_t tot = (int64_t)343 * L.K;
        unsigned nb = (unsigned)((tot + 255) / 256);
        if (h->prec == 0)
            k_translations<double><<<nb, 256, 0, h->stream>>>(L.K, L.nph, L.L, d_theta, d_wth, L.a, d_di, d_hk, (double*)L.d_T);
        else
            k_translations<float><<<nb, 256, 0, h->stream>>>(L.K, L.nph, L.L, d_theta, d_wth, L.a, d_di, d_hk, (float*)L.d_T);
        CU(cudaGetLastError());
        L.d_il_ptr = h->upload(L.il_ptr);
        L.d_il_src = h->upload(L.il_src);
        L.d_il_off = h->upload(L.il_off);
        // shift tables of a parent level (children at l + 1)
        if (l < h->leaf) {
            L.d_shift = h->alloc((size_t)8 * L.K * h->csize);
            unsigned nb2 = (unsigned)((8 * L.K + 255) / 256);
            double half_child = 0.5 * h->lev[l + 1].a;
            if (h->prec == 0)
                k_shifts<double><<<nb2, 256, 0, h->stream>>>(L.K, L.nph, d_theta, half_child, h->k, h->ki, (double*)L.d_shift);
            else
                k_shifts<float><<<nb2, 256, 0, h->stream>>>(L.K, L.nph, d_theta, half_child, h->k, h->ki, (float*)L.d_shift);
            CU(cudaGetLastError());
            L.d_shift_dn = L.d_shift;
            if (h->ki != 0.0) {
                // downward factor exp(-jk khat.d) = exp(-jk'a) exp(k''a), stored conjugated
                // (exp(+jk'a) exp(k''a)) because the downward kernels conjugate what they read
                L.d_shift_dn = h->alloc((size_t)8 * L.K * h->csize);
                if (h->prec == 0)
                    k_shifts<double><<<nb2, 256, 0, h->stream>>>(L.K, L.nph, d_theta, half_child, h->k, -h->ki,
                                                                 (double*)L.d_shift_dn);
                else
                    k_shifts<float><<<nb2, 256, 0, h->stream>>>(L.K, L.nph, d_theta, half_child, h->k, -h->ki,
                                                                (float*)L.d_shift_dn);
                CU(cudaGetLastError());
            }
            L.d_child_ptr = h->upload(L.child_ptr);
        }
        // octant of each box of this level inside its parent
        std::vector<int> oct(L.nbox);
        for (int b = 0; b < L.nbox; ++b)
            oct[b] = (L.coords[3 * b] & 1) | ((L.coords[3 * b + 1] & 1) << 1) | ((L.coords[3 * b + 2] & 1) << 2);
        L.d_octant = h->upload(oct);
        L.d_parent = h->upload(L.parent);
        {
            // slot of each box among its siblings; order = by slot, then by parent
            std::vector<int> slot(L.nbox, 0), ord(L.nbox);
            for (int b = 1; b < L.nbox; ++b) slot[b] = (L.parent[b] == L.parent[b - 1]) ? slot[b - 1] + 1 : 0;
            for (int b = 0; b < L.nbox; ++b) ord[b] = b;
            std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return slot[x] < slot[y]; });
            L.d_child_order = h->upload(ord);
        }
    }
    // interpolation tables (weights in the handle precision)
    for (int l = 2; l + 1 <= h->leaf; ++l) {
        interp_t& I = h->itp[l];
        I.d_th_src = h->upload(I.th_src);
        I.d_th_flip = h->upload(I.th_flip);
        I.d_ph_src = h->upload(I.ph_src);
        I.d_tth_ptr = h->upload(I.tth_ptr);
        I.d_tth_dst = h->upload(I.tth_dst);
        I.d_tth_flip = h->upload(I.tth_flip);
        I.d_tph_ptr = h->upload(I.tph_ptr);
        I.d_tph_dst = h->upload(I.tph_dst);
        if (h->prec == 0) {
            I.d_th_w = h->upload(I.th_w);
            I.d_ph_w = h->upload(I.ph_w);
            I.d_tth_w = h->upload(I.tth_w);
            I.d_tph_w = h->upload(I.tph_w);
        } else {
            I.d_th_w = h->upload(std::vector<float>(I.th_w.begin(), I.th_w.end()));
            I.d_ph_w = h->upload(std::vector<float>(I.ph_w.begin(), I.ph_w.end()));
            I.d_tth_w = h->upload(std::vector<float>(I.tth_w.begin(), I.tth_w.end()));
            I.d_tph_w = h->upload(std::vector<float>(I.tph_w.begin(), I.tph_w.end()));
        }
    }
    bi_upload_taps(h);
}

void bi_alloc_work(bi_handle_s* h) {
    const int R = h->max_rhs;
    h->d_status = (int*)h->alloc(sizeof(int));
    CU(cudaMemset(h->d_status, 0, sizeof(int)));
    {
        // largest leaf boxes first: per-box CTAs then finish close together
        const int nb = (int)h->leaf_start.size() - 1;
        std::vector<int> order(std::max(nb, 0));
        for (int b = 0; b < nb; ++b) order[b] = b;
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
            return h->leaf_start[a + 1] - h->leaf_start[a] > h->leaf_start[b + 1] - h->leaf_start[b];
        });
        h->d_leaf_order = h->upload(order);
    }
    size_t vec = (size_t)h->N * h->nX * R * h->csize;
    h->d_xt = h->alloc(vec);
    h->d_yt = h->alloc(vec);
    h->d_yfar = h->alloc(vec);
    h->d_sx = h->alloc((size_t)h->nun * R * h->csize);
    h->d_sy = h->alloc((size_t)h->nun * R * h->csize);
    const int E = 2 * h->nF * R;
    for (int l = 2; l <= h->leaf; ++l) {
        level_t& L = h->lev[l];
        size_t sz = (size_t)L.nbox * L.K * E * h->csize;
        L.d_U = h->alloc(sz);
        L.d_V = h->alloc(sz);
    }
    for (int l = 2; l + 1 <= h->leaf; ++l) {
        const level_t& P = h->lev[l];
        const level_t& C = h->lev[l + 1];
        // theta-pass intermediate: per child box [nth_parent][nph_child][E]
        size_t sz = (size_t)C.nbox * P.nth * C.nph * E * h->csize;
        h->itp[l].d_tmp = h->alloc(sz);
    }
}
