/*
 * bi_oracle.c -- CPU FP64 oracle for the boundary-integral matrix C (Eqs. 42-46).
 *
 * TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
 * CPU-baseline leg load this library.  It shares no code, header, table or
 * constant generator with the CUDA path.
 *
 * What it computes (plain definitions, written out):
 *   - RWG basis functions on pairs of triangles (Sec. II.C, Eq. exp4-5, Rao-Wilton-
 *     Glisson 1982): f = (l / 2A+)(r - p+) on T+, (l / 2A-)(p- - r) on T-.
 *   - Free-space Green's function G = exp(-j k R) / (4 pi R), time convention
 *     exp(j w t) (Sec. II.A).  k may be complex (a lossy medium such as the coating of
 *     Sec. III.D, Im k < 0): every kernel piece below is analytic in k.
 *   - Operators L and K of Sec. II.C (Eq. 22 and the definitions below it),
 *     K-bar = principal value of K.
 *   - Galerkin primitives (inner product without conjugation, Eq. 10):
 *       Gram  G_mn  = <f_m, f_n>,   twisted Gram X_mn = <f_m, n x f_n>,
 *       P_mn = 1/2 <f_m, L f_n> + 1/2 <f_m, n x Kbar f_n>        (<f_m, C f_n>, Eq. 27, alpha = 1/2)
 *       Q_mn = 1/2 <f_m, n x L f_n> - 1/2 <f_m, Kbar f_n>        (<f_m, n x C f_n>)
 *   - Mode 0 (the C block of Eq. 42, entries Eqs. 43-46):
 *       [ G - P      X/2 - Q ]
 *       [   Q        G/2 - P ]
 *   - Mode 1 (PEC combined-field equation from Eqs. 24a/24b with M = 0 and
 *     alpha = 1/2):  G/4 - P.
 *   - Plane-wave right-hand sides (Eqs. 49-50, excitation of Sec. III) and the
 *     far field of the currents (Eq. 22a in the far zone) for the RCS of Eq. 5-25.
 *
 * Integration: all entries are double integrals over a test triangle (outer, r)
 * and a source triangle (inner, r').  Well separated pairs use plain product
 * Gauss rules.  Close pairs use singularity subtraction: the static parts 1/R,
 * (r'-r)/R and grad(1/R) of the inner integral are taken in closed form
 * (Wilton et al. 1984, Graglia 1993), the bounded remainder by quadrature.  Outer
 * rules are graded toward a shared edge or vertex, where the inner integral of
 * grad G has a logarithmic singularity.  The gradient part of <f_m, n x L f_n>
 * is moved onto the boundary of the test triangle (integration by parts, the
 * test field n x f_m is divergence free on a flat triangle) for close pairs.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cx;

#define PI 3.14159265358979323846

/* ------------------------------------------------------------------ vectors */
static inline void v_sub(const double* a, const double* b, double* o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static inline double v_dot(const double* a, const double* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static inline void v_cross(const double* a, const double* b, double* o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static inline double v_norm(const double* a) { return sqrt(v_dot(a, a)); }

/* complex 3-vectors */
typedef struct { cx x[3]; } cv3;
static inline cx cv_dot_r(const cv3* a, const double* b) { return a->x[0] * b[0] + a->x[1] * b[1] + a->x[2] * b[2]; }
static inline void cv_cross_rc(const double* a, const cv3* b, cv3* o) { /* a (real) x b (complex) */
    o->x[0] = a[1] * b->x[2] - a[2] * b->x[1];
    o->x[1] = a[2] * b->x[0] - a[0] * b->x[2];
    o->x[2] = a[0] * b->x[1] - a[1] * b->x[0];
}
static inline void cv_cross_cr(const cv3* a, const double* b, cv3* o) { /* a (complex) x b (real) */
    o->x[0] = a->x[1] * b[2] - a->x[2] * b[1];
    o->x[1] = a->x[2] * b[0] - a->x[0] * b[2];
    o->x[2] = a->x[0] * b[1] - a->x[1] * b[0];
}

/* --------------------------------------------------------------- quadrature */
/* Gauss-Legendre nodes/weights on [0,1] by Newton iteration on P_n. */
static void gauss01(int n, double* x, double* w) {
    for (int i = 0; i < n; ++i) {
        double z = cos(PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

#define MAXQ 4096
/* A triangle rule: barycentric coordinates of (v0, v1, v2) and weights summing to 1,
 * so that int_T f ds ~= area * sum_k w_k f(x_k). */
typedef struct { int n; double b[MAXQ][3]; double w[MAXQ]; } trirule;

/* Conical (collapsed) product rule: b1 = u, b2 = (1-u) v. */
static void rule_plain(int n, trirule* R) {
    double x[64], w[64];
    gauss01(n, x, w);
    R->n = 0;
    for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) {
            double u = x[a], v = x[c];
            double b1 = u, b2 = (1.0 - u) * v;
            int k = R->n++;
            R->b[k][0] = 1.0 - b1 - b2;
            R->b[k][1] = b1;
            R->b[k][2] = b2;
            R->w[k] = 2.0 * w[a] * w[c] * (1.0 - u);
        }
}
/* Rule graded toward the edge (v0, v1): distance parameter t = s^q. */
static void rule_edge(int n, int q, trirule* R) {
    double x[64], w[64];
    gauss01(n, x, w);
    R->n = 0;
    for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) {
            double s = x[a], sg0 = x[c];
            double t = pow(s, q), jt = q * pow(s, q - 1);
            /* also cluster toward both ends of the edge (the shared vertices) */
            double sig = sg0 * sg0 * (3.0 - 2.0 * sg0), js = 6.0 * sg0 * (1.0 - sg0);
            int k = R->n++;
            R->b[k][2] = t;
            R->b[k][1] = (1.0 - t) * sig;
            R->b[k][0] = (1.0 - t) * (1.0 - sig);
            R->w[k] = 2.0 * w[a] * w[c] * (1.0 - t) * jt * js;
        }
}
/* Rule graded toward vertex v0: radial parameter u = s^q. */
static void rule_vertex(int n, int q, trirule* R) {
    double x[64], w[64];
    gauss01(n, x, w);
    R->n = 0;
    for (int a = 0; a < n; ++a)
        for (int c = 0; c < n; ++c) {
            double s = x[a], sig = x[c];
            double u = pow(s, q), ju = q * pow(s, q - 1);
            int k = R->n++;
            R->b[k][0] = 1.0 - u;
            R->b[k][1] = u * (1.0 - sig);
            R->b[k][2] = u * sig;
            R->w[k] = 2.0 * w[a] * w[c] * u * ju;
        }
}

/* ------------------------------------------------------------------ mesh */
typedef struct {
    double p[3][3];
    double n[3];
    double area;
    double diam;
    double c[3];
    int vid[3];
} tri_t;

static void make_tri(const double* V, const int* t, tri_t* T) {
    for (int a = 0; a < 3; ++a) {
        T->vid[a] = t[a];
        for (int d = 0; d < 3; ++d) T->p[a][d] = V[3 * t[a] + d];
    }
    double e1[3], e2[3], nn[3];
    v_sub(T->p[1], T->p[0], e1);
    v_sub(T->p[2], T->p[0], e2);
    v_cross(e1, e2, nn);
    double a2 = v_norm(nn);
    T->area = 0.5 * a2;
    for (int d = 0; d < 3; ++d) {
        T->n[d] = nn[d] / a2;
        T->c[d] = (T->p[0][d] + T->p[1][d] + T->p[2][d]) / 3.0;
    }
    double d01[3], d12[3], d20[3];
    v_sub(T->p[1], T->p[0], d01);
    v_sub(T->p[2], T->p[1], d12);
    v_sub(T->p[0], T->p[2], d20);
    double m = v_norm(d01);
    if (v_norm(d12) > m) m = v_norm(d12);
    if (v_norm(d20) > m) m = v_norm(d20);
    T->diam = m;
}

static void bary_point(const tri_t* T, const double* b, double* r) {
    for (int d = 0; d < 3; ++d) r[d] = b[0] * T->p[0][d] + b[1] * T->p[1][d] + b[2] * T->p[2][d];
}

typedef struct { int64_t key; int a, b, tri, loc; } halfedge;
static int he_cmp(const void* x, const void* y) {
    const halfedge* p = (const halfedge*)x;
    const halfedge* q = (const halfedge*)y;
    if (p->key < q->key) return -1;
    if (p->key > q->key) return 1;
    return (p->a < q->a) ? -1 : (p->a > q->a);
}

/*
 * RWG functions from a closed triangle mesh.  Edges are numbered in increasing
 * (min vertex, max vertex) order.  T+ is the triangle in which the edge runs from
 * its smaller to its larger vertex index (counter-clockwise seen from outside).
 * Outputs per edge: the two vertex ids, T+, T-, and the local index (0..2) of the
 * free vertex in T+ and T-.  Returns the number of RWG functions, or a negative code:
 * -1 open or non-manifold edge, -2 inconsistent orientation, -3 degenerate triangle.
 */
int or_rwg(int nv, const double* V, int nt, const int* T, int* edges, int* tp, int* tm, int* lp, int* lm) {
    (void)nv;
    for (int t = 0; t < nt; ++t) {
        tri_t tt;
        make_tri(V, T + 3 * t, &tt);
        if (!(tt.area > 1e-14 * tt.diam * tt.diam)) return -3;
    }
    halfedge* h = (halfedge*)malloc(sizeof(halfedge) * 3 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = T[3 * t + k], b = T[3 * t + (k + 1) % 3];
            halfedge* e = &h[3 * t + k];
            int lo = a < b ? a : b, hi = a < b ? b : a;
            e->key = (int64_t)lo * 4294967296LL + hi;
            e->a = a;
            e->b = b;
            e->tri = t;
            e->loc = (k + 2) % 3; /* vertex opposite the half-edge (k, k+1) */
        }
    qsort(h, 3 * (size_t)nt, sizeof(halfedge), he_cmp);
    int ne = 0;
    size_t i = 0, n3 = 3 * (size_t)nt;
    int rc = 0;
    while (i < n3) {
        size_t j = i;
        while (j < n3 && h[j].key == h[i].key) ++j;
        if (j - i != 2) { rc = -1; break; }
        halfedge *x = &h[i], *y = &h[i + 1];
        halfedge *pl = NULL, *mi = NULL;
        if (x->a < x->b && y->a > y->b) { pl = x; mi = y; }
        else if (y->a < y->b && x->a > x->b) { pl = y; mi = x; }
        else { rc = -2; break; }
        edges[2 * ne] = pl->a;
        edges[2 * ne + 1] = pl->b;
        tp[ne] = pl->tri;
        tm[ne] = mi->tri;
        lp[ne] = pl->loc;
        lm[ne] = mi->loc;
        ++ne;
        i = j;
    }
    free(h);
    return rc ? rc : ne;
}

/* ------------------------------------------------- closed-form static parts */
/* ln((R+ + l+)/(R- + l-)) evaluated without cancellation. */
static double edge_log(double lp, double lm, double Rp, double Rm, double R02) {
    /* R + l for l < 0 is computed as R0^2 / (R - l) to avoid cancellation */
    double a = (lp >= 0.0) ? (Rp + lp) : R02 / (Rp - lp);
    double b = (lm >= 0.0) ? (Rm + lm) : R02 / (Rm - lm);
    return log(a) - log(b);
}

/*
 * Static integrals over triangle T for the observation point r:
 *   I1   = int_T 1/R ds'
 *   Ir   = int_T (rho' - rho)/R ds'             (in-plane vector, rho = projection of r)
 *   Ig   = int_T grad_r (1/R) ds' = int_T (r' - r)/R^3 ds'
 * Wilton et al., IEEE TAP 32(3) 1984; Graglia, IEEE TAP 41(10) 1993.
 * On the plane of T (h = 0) the normal part of Ig is the principal value, 0.
 */
void or_static_tri2(const double* P, const double* r, double* I1, double* Ir, double* Ig, double* IR, double* IrR) {
    tri_t T;
    double V[9];
    memcpy(V, P, sizeof(V));
    int id[3] = {0, 1, 2};
    make_tri(V, id, &T);
    double d0[3];
    v_sub(r, T.p[0], d0);
    double h = v_dot(T.n, d0);
    double rho[3];
    for (int d = 0; d < 3; ++d) rho[d] = r[d] - h * T.n[d];
    double ah = fabs(h);
    double scale = T.diam;
    double s1 = 0.0, sr[3] = {0, 0, 0}, sg[3] = {0, 0, 0}, sbeta = 0.0;
    double sR = 0.0, srR[3] = {0, 0, 0};
    for (int e = 0; e < 3; ++e) {
        const double* pa = T.p[e];
        const double* pb = T.p[(e + 1) % 3];
        double le[3];
        v_sub(pb, pa, le);
        double len = v_norm(le);
        for (int d = 0; d < 3; ++d) le[d] /= len;
        double u[3];
        v_cross(le, T.n, u); /* outward in-plane normal of the edge */
        double qa[3], qb[3];
        v_sub(pa, rho, qa);
        v_sub(pb, rho, qb);
        double lm = v_dot(qa, le), lp = v_dot(qb, le);
        double t0 = v_dot(qa, u);
        double R02 = t0 * t0 + h * h;
        double Rp = sqrt(lp * lp + R02), Rm = sqrt(lm * lm + R02);
        double f;
        int on_line = (sqrt(R02) < 1e-12 * scale);
        if (on_line) {
            /* observation point on the line of this edge: the log may be infinite but
               it only enters multiplied by t0 or R0^2 in I1, Ir; in Ig it is singular. */
            f = (lm > 0.0 || lp < 0.0) ? edge_log(lp, lm, Rp, Rm, R02) : INFINITY;
        } else {
            f = edge_log(lp, lm, Rp, Rm, R02);
        }
        double beta = 0.0;
        if (!on_line) beta = atan(t0 * lp / (R02 + ah * Rp)) - atan(t0 * lm / (R02 + ah * Rm));
        if (!on_line) s1 += t0 * f - ah * beta;
        double rr = (on_line ? 0.0 : R02 * f) + lp * Rp - lm * Rm;
        for (int d = 0; d < 3; ++d) {
            sr[d] += 0.5 * u[d] * rr;
            sg[d] -= u[d] * f;
        }
        sbeta += beta;
        /* int_edge R dl = (rr)/2 ; int_T R = (1/3)[sum t0 int_edge R + h^2 I1] */
        sR += t0 * 0.5 * rr;
        /* int_edge R^3 dl = [l R^3/4 + 3 R0^2 l R/8 + 3 R0^4/8 ln(l + R)] */
        double e3 = 0.25 * (lp * Rp * Rp * Rp - lm * Rm * Rm * Rm) + 0.375 * R02 * (lp * Rp - lm * Rm) +
                    (on_line ? 0.0 : 0.375 * R02 * R02 * f);
        for (int d = 0; d < 3; ++d) srR[d] += u[d] * e3 / 3.0;
    }
    double sgn = (h > 0.0) ? 1.0 : (h < 0.0 ? -1.0 : 0.0);
    *I1 = s1;
    for (int d = 0; d < 3; ++d) {
        Ir[d] = sr[d];
        Ig[d] = sg[d] - T.n[d] * sgn * sbeta;
    }
    *IR = (sR + h * h * s1) / 3.0;
    for (int d = 0; d < 3; ++d) IrR[d] = srR[d];
}

void or_static_tri(const double* P, const double* r, double* I1, double* Ir, double* Ig) {
    double IR, IrR[3];
    or_static_tri2(P, r, I1, Ir, Ig, &IR, IrR);
}

/* ----------------------------------------------------------- kernel pieces */
/* G - 1/(4 pi R) + k^2 R/(8 pi)  (smooth: -jk/(4 pi) + j k^3 R^2/(24 pi) + ...).  Every kernel
   piece is analytic in k, so a complex wavenumber (lossy medium, Im k < 0 with exp(j w t))
   goes through the same expressions. */
static inline cx g_rem(cx k, double R) {
    cx x = k * R;
    if (cabs(x) < 1e-2) return (-I * k + I * k * x * x / 6.0 + k * x * x * x / 24.0 - I * k * x * x * x * x / 120.0) / (4.0 * PI);
    return (cexp(-I * x) - 1.0 + 0.5 * x * x) / (4.0 * PI * R);
}
/* gt(R) with grad_r G = (r' - r) gt(R): gt = (1 + jkR) exp(-jkR) / (4 pi R^3) */
static inline cx gt_full(cx k, double R) { return (1.0 + I * k * R) * cexp(-I * k * R) / (4.0 * PI * R * R * R); }
/* gt - (1/R^3 + k^2/(2R))/(4 pi) */
static inline cx gt_rem(cx k, double R) {
    cx x = k * R;
    if (cabs(x) < 2e-2) {
        /* series of (1+jx)e^{-jx} = 1 + x^2/2 - j x^3/3 - x^4/8 + j x^5/30 + ... */
        cx s = -I * x * x * x / 3.0 - x * x * x * x / 8.0 + I * x * x * x * x * x / 30.0 + x * x * x * x * x * x / 144.0;
        return s / (4.0 * PI * R * R * R);
    }
    return ((1.0 + I * x) * cexp(-I * x) - 1.0 - 0.5 * x * x) / (4.0 * PI * R * R * R);
}

/* Inner integrals over source triangle S at observation point r:
 *   Sg = int_S G ds',  Sr = int_S (r' - r) G ds',  Kv = int_S grad_r G ds'. */
typedef struct { cx Sg; cv3 Sr; cv3 Kv; } inner_t;

static void inner_plain(const tri_t* S, const trirule* R, cx k, const double* r, inner_t* o) {
    o->Sg = 0;
    for (int d = 0; d < 3; ++d) { o->Sr.x[d] = 0; o->Kv.x[d] = 0; }
    for (int q = 0; q < R->n; ++q) {
        double rp[3], dr[3];
        bary_point(S, R->b[q], rp);
        v_sub(rp, r, dr);
        double Rl = v_norm(dr);
        double w = R->w[q] * S->area;
        cx G = cexp(-I * k * Rl) / (4.0 * PI * Rl);
        cx gt = gt_full(k, Rl);
        o->Sg += w * G;
        for (int d = 0; d < 3; ++d) {
            o->Sr.x[d] += w * G * dr[d];
            o->Kv.x[d] += w * gt * dr[d];
        }
    }
}

static void inner_sing(const tri_t* S, const trirule* R, cx k, const double* r, inner_t* o) {
    double I1, Ir[3], Ig[3], IR, IrR[3];
    double P[9];
    for (int a = 0; a < 3; ++a)
        for (int d = 0; d < 3; ++d) P[3 * a + d] = S->p[a][d];
    or_static_tri2(P, r, &I1, Ir, Ig, &IR, IrR);
    double d0[3];
    v_sub(r, S->p[0], d0);
    double h = v_dot(S->n, d0);
    /* int (r' - r)/R = Ir - h n I1 */
    double Irr[3];
    for (int d = 0; d < 3; ++d) Irr[d] = Ir[d] - h * S->n[d] * I1;
    /* int (r' - r) R = IrR - h n IR */
    o->Sg = (I1 - 0.5 * k * k * IR) / (4.0 * PI);
    for (int d = 0; d < 3; ++d) {
        o->Sr.x[d] = (Irr[d] - 0.5 * k * k * (IrR[d] - h * S->n[d] * IR)) / (4.0 * PI);
        o->Kv.x[d] = (Ig[d] + 0.5 * k * k * Irr[d]) / (4.0 * PI);
    }
    for (int q = 0; q < R->n; ++q) {
        double rp[3], dr[3];
        bary_point(S, R->b[q], rp);
        v_sub(rp, r, dr);
        double Rl = v_norm(dr);
        double w = R->w[q] * S->area;
        cx gr, gtr;
        if (Rl < 1e-14 * S->diam) { gr = -I * k / (4.0 * PI); gtr = 0; }  /* limits at R = 0 */
        else { gr = g_rem(k, Rl); gtr = gt_rem(k, Rl); }
        o->Sg += w * gr;
        for (int d = 0; d < 3; ++d) {
            o->Sr.x[d] += w * gr * dr[d];
            o->Kv.x[d] += w * gtr * dr[d];
        }
    }
}

/* ------------------------------------------------- per triangle-pair blocks */
/* Raw blocks with the half-basis g_i(r) = r - v_i (divergence 2) on both sides:
 *   L [i][j] = -jk [ int int g_i . g_j G - (4/k^2) int int G ]
 *   NL[i][j] = -jk int int g_i . (n_m x g_j) G  - (j/k) int g_i . (n_m x grad Phi_j)
 *              with Phi_j = int 2 G ds'
 *   K [i][j] = int int g_i . (grad_r G x g_j)
 *   NK[i][j] = int int g_i . (n_m x (grad_r G x g_j))
 * The RWG entry is the raw entry times (s l / 2A) of each side. */
typedef struct { cx L[3][3], NL[3][3], K[3][3], NK[3][3]; } blocks_t;

enum { REL_FAR = 0, REL_NEAR = 1, REL_VERTEX = 2, REL_EDGE = 3, REL_SAME = 4 };

typedef struct {
    int n_far_out, n_far_in;   /* plain rules for separated pairs */
    int n_near_out, n_near_in; /* singularity subtraction */
    int n_sing;                /* graded outer rules */
    int q_grade;
    int n_line;                /* Gauss points per edge for the boundary term */
    double near_factor;        /* near if centroid distance < near_factor * max diam */
} quality_t;

static void quality_set(int level, quality_t* q) {
    /* level 0: default; higher levels refine every rule (used to pin convergence). */
    q->n_far_out = 4 + level;
    q->n_far_in = 4 + level;
    q->n_near_out = 6 + 2 * level;
    q->n_near_in = 6 + 2 * level;
    q->n_sing = 10 + 4 * level;
    q->q_grade = 3;
    q->n_line = 10 + 4 * level;
    q->near_factor = 3.0;
}

/* permutation mapping the shared edge/vertex of the test triangle to local slots */
typedef struct { int perm[3]; } rot_t;

static void accumulate_outer(const tri_t* Tm, const tri_t* Tn, const double* r, double W, const inner_t* in,
                             cx k, int far_surface_nl, blocks_t* B) {
    cx jk = I * k;
    for (int i = 0; i < 3; ++i) {
        double gi[3];
        v_sub(r, Tm->p[i], gi);
        double ngi[3];
        v_cross(Tm->n, gi, ngi); /* n_m x g_i */
        /* g_i . Sr and g_i . (n x Sr) = -(n x g_i) . Sr */
        cx gi_Sr = cv_dot_r(&in->Sr, gi);
        cx ngi_Sr = cv_dot_r(&in->Sr, ngi);
        cx nl2 = 0;
        if (far_surface_nl) nl2 = (2.0 * I / k) * cv_dot_r(&in->Kv, ngi);
        for (int j = 0; j < 3; ++j) {
            double gj[3];
            v_sub(r, Tn->p[j], gj); /* g_j evaluated at the test point: g_j(r') = (r'-r) + (r - v_j) */
            double gg = v_dot(gi, gj);
            double ngj_gi = 0.0;
            {
                double ngj[3];
                v_cross(Tm->n, gj, ngj);
                ngj_gi = v_dot(gi, ngj);
            }
            /* L */
            cx t_gg = gi_Sr + gg * in->Sg;
            B->L[i][j] += W * (-jk) * (t_gg - (4.0 / (k * k)) * in->Sg);
            /* NL, surface part: g_i . (n x (Sr + (r - v_j) Sg)) */
            cx t_ng = -ngi_Sr + ngj_gi * in->Sg;
            B->NL[i][j] += W * ((-jk) * t_ng + nl2);
            /* K: g_i . (Kv x g_j(r)) ; NK: g_i . (n x (Kv x g_j(r))) */
            cv3 kx;
            cv_cross_cr(&in->Kv, gj, &kx);
            B->K[i][j] += W * cv_dot_r(&kx, gi);
            cv3 nkx;
            cv_cross_rc(Tm->n, &kx, &nkx);
            B->NK[i][j] += W * cv_dot_r(&nkx, gi);
        }
    }
}

/* Boundary form of the gradient part of NL:
 *   -(j/k) int_Tm g_i . (n x grad Phi) ds = (j/k) int_Tm (n x g_i) . grad Phi ds
 *   = (j/k) sum_edges int_e Phi (n x g_i) . nu dl = -(j/k) sum_e int_e Phi g_i . tau dl,
 * with Phi = 2 int_Tn G ds' and tau the counter-clockwise edge tangent. */
static void nl_boundary(const tri_t* Tm, const tri_t* Tn, const trirule* Rin, int nline, cx k, blocks_t* B) {
    double x[64], w[64];
    gauss01(nline, x, w);
    /* Phi has logarithmic derivative singularities at the vertices of the source triangle;
       the map x = s^2 (3 - 2 s) clusters the Gauss points toward both edge ends. */
    for (int q = 0; q < nline; ++q) {
        double s = x[q];
        x[q] = s * s * (3.0 - 2.0 * s);
        w[q] *= 6.0 * s * (1.0 - s);
    }
    for (int e = 0; e < 3; ++e) {
        const double* pa = Tm->p[e];
        const double* pb = Tm->p[(e + 1) % 3];
        double tv[3];
        v_sub(pb, pa, tv);
        double len = v_norm(tv);
        for (int d = 0; d < 3; ++d) tv[d] /= len;
        for (int q = 0; q < nline; ++q) {
            double r[3];
            for (int d = 0; d < 3; ++d) r[d] = pa[d] + x[q] * (pb[d] - pa[d]);
            inner_t in;
            inner_sing(Tn, Rin, k, r, &in);
            cx Phi = 2.0 * in.Sg;
            for (int i = 0; i < 3; ++i) {
                double gi[3];
                v_sub(r, Tm->p[i], gi);
                cx c = -(I / k) * Phi * v_dot(gi, tv) * w[q] * len;
                for (int j = 0; j < 3; ++j) B->NL[i][j] += c;
            }
        }
    }
}

typedef struct {
    trirule far_out, far_in, near_out, near_in, edge_r, vert_r;
    quality_t q;
} rules_t;

static rules_t* rules_make(int level) {
    rules_t* R = (rules_t*)malloc(sizeof(rules_t));
    quality_set(level, &R->q);
    rule_plain(R->q.n_far_out, &R->far_out);
    rule_plain(R->q.n_far_in, &R->far_in);
    rule_plain(R->q.n_near_out, &R->near_out);
    rule_plain(R->q.n_near_in, &R->near_in);
    rule_edge(R->q.n_sing, R->q.q_grade, &R->edge_r);
    rule_vertex(R->q.n_sing, R->q.q_grade, &R->vert_r);
    return R;
}

/* relation of two triangles by shared vertex ids */
static int tri_relation(const tri_t* A, const tri_t* B, int* sa, int* sb) {
    int ns = 0;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b)
            if (A->vid[a] == B->vid[b]) {
                sa[ns] = a;
                sb[ns] = b;
                ++ns;
            }
    return ns;
}

static void pair_blocks(const tri_t* Tm, const tri_t* Tn, const rules_t* R, cx k, blocks_t* B) {
    memset(B, 0, sizeof(*B));
    int sa[3], sb[3];
    int ns = tri_relation(Tm, Tn, sa, sb);
    double dc[3];
    v_sub(Tm->c, Tn->c, dc);
    double dist = v_norm(dc);
    double dm = Tm->diam > Tn->diam ? Tm->diam : Tn->diam;
    int rel;
    if (ns == 3) rel = REL_SAME;
    else if (ns == 2) rel = REL_EDGE;
    else if (ns == 1) rel = REL_VERTEX;
    else if (dist < R->q.near_factor * dm) rel = REL_NEAR;
    else rel = REL_FAR;

    if (rel == REL_FAR) {
        const trirule* ro = &R->far_out;
        for (int q = 0; q < ro->n; ++q) {
            double r[3];
            bary_point(Tm, ro->b[q], r);
            inner_t in;
            inner_plain(Tn, &R->far_in, k, r, &in);
            accumulate_outer(Tm, Tn, r, ro->w[q] * Tm->area, &in, k, 1, B);
        }
        return;
    }
    if (rel == REL_SAME) {
        /* the inner static integrals have x log x behaviour at the triangle's own edges:
           split the test triangle at its centroid and grade each piece toward its base edge */
        for (int e = 0; e < 3; ++e) {
            const trirule* re = &R->edge_r;
            for (int q = 0; q < re->n; ++q) {
                /* sub-triangle (v_e, v_{e+1}, centroid) with barycentrics (1/3,1/3,1/3) at the centroid */
                double b[3] = {0, 0, 0};
                b[e] += re->b[q][0];
                b[(e + 1) % 3] += re->b[q][1];
                for (int d = 0; d < 3; ++d) b[d] += re->b[q][2] / 3.0;
                double r[3];
                bary_point(Tm, b, r);
                inner_t in;
                inner_sing(Tn, &R->near_in, k, r, &in);
                accumulate_outer(Tm, Tn, r, re->w[q] * Tm->area / 3.0, &in, k, 0, B);
            }
        }
        nl_boundary(Tm, Tn, &R->near_in, R->q.n_line, k, B);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) { B->K[i][j] = 0; B->NK[i][j] = 0; }
        return;
    }
    /* outer rule for the test triangle, mapped so the singular feature sits at the graded spot */
    const trirule* ro = &R->near_out;
    int map[3] = {0, 1, 2};
    if (rel == REL_EDGE) {
        ro = &R->edge_r;
        int a0 = sa[0], a1 = sa[1];
        int a2 = 3 - a0 - a1;
        map[0] = a0;
        map[1] = a1;
        map[2] = a2;
    } else if (rel == REL_VERTEX) {
        ro = &R->vert_r;
        map[0] = sa[0];
        map[1] = (sa[0] + 1) % 3;
        map[2] = (sa[0] + 2) % 3;
    }
    for (int q = 0; q < ro->n; ++q) {
        double b[3];
        b[map[0]] = ro->b[q][0];
        b[map[1]] = ro->b[q][1];
        b[map[2]] = ro->b[q][2];
        double r[3];
        bary_point(Tm, b, r);
        inner_t in;
        inner_sing(Tn, &R->near_in, k, r, &in);
        accumulate_outer(Tm, Tn, r, ro->w[q] * Tm->area, &in, k, 0, B);
    }
    nl_boundary(Tm, Tn, &R->near_in, R->q.n_line, k, B);
    if (rel == REL_SAME) {
        /* principal value: both K-type kernels vanish on one flat triangle */
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) { B->K[i][j] = 0; B->NK[i][j] = 0; }
    }
}

/* exposed for tests: raw blocks of one triangle pair (row-major [4][3][3] complex) at the
   wavenumber k_re + j k_im */
void or_pair_blocks(const double* Pm, const double* Pn, const int* idm, const int* idn, double k_re, double k_im,
                    int level, double* out) {
    const cx k = k_re + I * k_im;
    tri_t Tm, Tn;
    make_tri(Pm, (int[]){0, 1, 2}, &Tm);
    make_tri(Pn, (int[]){0, 1, 2}, &Tn);
    for (int a = 0; a < 3; ++a) { Tm.vid[a] = idm[a]; Tn.vid[a] = idn[a]; }
    rules_t* R = rules_make(level);
    blocks_t B;
    pair_blocks(&Tm, &Tn, R, k, &B);
    free(R);
    cx* o = (cx*)out;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            o[0 * 9 + 3 * i + j] = B.L[i][j];
            o[1 * 9 + 3 * i + j] = B.NL[i][j];
            o[2 * 9 + 3 * i + j] = B.K[i][j];
            o[3 * 9 + 3 * i + j] = B.NK[i][j];
        }
}

/* ------------------------------------------------------------ assembly */
typedef struct {
    int nt, ne;
    tri_t* tris;
    int *tp, *tm, *lp, *lm;
    double* len;
    /* per triangle: RWG index of the function whose free vertex is local a, and its coefficient s l / 2A */
    int* t_rwg;   /* [nt][3] */
    double* t_cf; /* [nt][3] */
} mesh_t;

static int mesh_build(int nv, const double* V, int nt, const int* T, mesh_t* M) {
    memset(M, 0, sizeof(*M));
    M->nt = nt;
    int ne_max = 3 * nt / 2 + 1;
    int* edges = (int*)malloc(sizeof(int) * 2 * ne_max);
    M->tp = (int*)malloc(sizeof(int) * ne_max);
    M->tm = (int*)malloc(sizeof(int) * ne_max);
    M->lp = (int*)malloc(sizeof(int) * ne_max);
    M->lm = (int*)malloc(sizeof(int) * ne_max);
    int ne = or_rwg(nv, V, nt, T, edges, M->tp, M->tm, M->lp, M->lm);
    if (ne < 0) { free(edges); return ne; }
    M->ne = ne;
    M->tris = (tri_t*)malloc(sizeof(tri_t) * nt);
    for (int t = 0; t < nt; ++t) make_tri(V, T + 3 * t, &M->tris[t]);
    M->len = (double*)malloc(sizeof(double) * ne);
    M->t_rwg = (int*)malloc(sizeof(int) * 3 * nt);
    M->t_cf = (double*)malloc(sizeof(double) * 3 * nt);
    for (int i = 0; i < 3 * nt; ++i) { M->t_rwg[i] = -1; M->t_cf[i] = 0.0; }
    for (int e = 0; e < ne; ++e) {
        double d[3];
        v_sub(V + 3 * edges[2 * e + 1], V + 3 * edges[2 * e], d);
        M->len[e] = v_norm(d);
        int t = M->tp[e], a = M->lp[e];
        M->t_rwg[3 * t + a] = e;
        M->t_cf[3 * t + a] = M->len[e] / (2.0 * M->tris[t].area);
        t = M->tm[e];
        a = M->lm[e];
        M->t_rwg[3 * t + a] = e;
        M->t_cf[3 * t + a] = -M->len[e] / (2.0 * M->tris[t].area);
    }
    free(edges);
    return 0;
}
static void mesh_free(mesh_t* M) {
    free(M->tris); free(M->tp); free(M->tm); free(M->lp); free(M->lm);
    free(M->len); free(M->t_rwg); free(M->t_cf);
}

static inline void atomic_add_cx(cx* z, cx v) {
    double* p = (double*)z;
#pragma omp atomic
    p[0] += creal(v);
#pragma omp atomic
    p[1] += cimag(v);
}

/* raw Gram integrals on one triangle: int g_i . g_j and int g_i . (n x g_j), exact
   (degree-2 integrand) with the edge-midpoint rule */
static void gram_raw(const tri_t* T, double Gr[3][3], double Xr[3][3]) {
    double mid[3][3];
    for (int e = 0; e < 3; ++e)
        for (int d = 0; d < 3; ++d) mid[e][d] = 0.5 * (T->p[e][d] + T->p[(e + 1) % 3][d]);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double sg = 0, sx = 0;
            for (int q = 0; q < 3; ++q) {
                double gi[3], gj[3], ngj[3];
                v_sub(mid[q], T->p[i], gi);
                v_sub(mid[q], T->p[j], gj);
                v_cross(T->n, gj, ngj);
                sg += v_dot(gi, gj) / 3.0;
                sx += v_dot(gi, ngj) / 3.0;
            }
            Gr[i][j] = sg * T->area;
            Xr[i][j] = sx * T->area;
        }
}

/*
 * Rows of the matrix of mode 0 (2N x 2N, J rows then M rows) or mode 1 (N x N).
 * rows == NULL (nrows ignored) means all rows.  Z is row-major [nrows][ncols],
 * complex128.  'part' selects: 0 everything, 1 P only (as -P in the JJ slot),
 * 2 Q only (as -Q in the JM slot) -- parts are used by tests.
 * The wavenumber is k_re + j k_im (k_im <= 0 for a lossy medium).
 * Returns 0, or the negative mesh error of or_rwg.
 */
int or_fill_rows(int nv, const double* V, int nt, const int* T, double k_re, double k_im, int mode, int level,
                 int nrows, const int* rows, double* Zout) {
    const cx k = k_re + I * k_im;
    mesh_t M;
    int rc = mesh_build(nv, V, nt, T, &M);
    if (rc) return rc;
    int N = M.ne;
    int nun = (mode == 0) ? 2 * N : N;
    int all = (rows == NULL);
    if (all) nrows = nun;
    size_t ncols = (size_t)nun;
    cx* Z = (cx*)Zout;
    memset(Z, 0, sizeof(cx) * (size_t)nrows * ncols);
    /* map: RWG m -> output row for its J test (or PEC) and for its M test */
    int* rowJ = (int*)malloc(sizeof(int) * N);
    int* rowM = (int*)malloc(sizeof(int) * N);
    for (int m = 0; m < N; ++m) { rowJ[m] = -1; rowM[m] = -1; }
    for (int r = 0; r < nrows; ++r) {
        int g = all ? r : rows[r];
        if (g < N) rowJ[g] = r;
        else if (mode == 0 && g < 2 * N) rowM[g - N] = r;
    }
    /* test triangles that are needed */
    char* need = (char*)calloc(M.nt, 1);
    for (int m = 0; m < N; ++m)
        if (rowJ[m] >= 0 || rowM[m] >= 0) { need[M.tp[m]] = 1; need[M.tm[m]] = 1; }
    int* list = (int*)malloc(sizeof(int) * M.nt);
    int nl = 0;
    for (int t = 0; t < M.nt; ++t)
        if (need[t]) list[nl++] = t;
    rules_t* R = rules_make(level);

    /* work items: (test triangle, block of source triangles), so that a few rows of a large
       mesh still spread over all cores */
    const int sblk = 512;
    const int nsb = (M.nt + sblk - 1) / sblk;
#pragma omp parallel for schedule(dynamic, 1)
    for (long long item = 0; item < (long long)nl * nsb; ++item) {
        int li = (int)(item / nsb);
        int tmi = list[li];
        const tri_t* Tm = &M.tris[tmi];
        int t0 = (int)(item % nsb) * sblk;
        int t1 = t0 + sblk < M.nt ? t0 + sblk : M.nt;
        for (int tni = t0; tni < t1; ++tni) {
            const tri_t* Tn = &M.tris[tni];
            blocks_t B;
            pair_blocks(Tm, Tn, R, k, &B);
            for (int i = 0; i < 3; ++i) {
                int m = M.t_rwg[3 * tmi + i];
                if (m < 0 || (rowJ[m] < 0 && rowM[m] < 0)) continue;
                double cm = M.t_cf[3 * tmi + i];
                for (int j = 0; j < 3; ++j) {
                    int n = M.t_rwg[3 * tni + j];
                    if (n < 0) continue;
                    double cn = M.t_cf[3 * tni + j];
                    double c = cm * cn;
                    cx P = 0.5 * c * (B.L[i][j] + B.NK[i][j]);
                    cx Q = 0.5 * c * (B.NL[i][j] - B.K[i][j]);
                    if (mode == 0) {
                        if (rowJ[m] >= 0) {
                            atomic_add_cx(&Z[(size_t)rowJ[m] * ncols + n], -P);
                            atomic_add_cx(&Z[(size_t)rowJ[m] * ncols + N + n], -Q);
                        }
                        if (rowM[m] >= 0) {
                            atomic_add_cx(&Z[(size_t)rowM[m] * ncols + n], Q);
                            atomic_add_cx(&Z[(size_t)rowM[m] * ncols + N + n], -P);
                        }
                    } else {
                        if (rowJ[m] >= 0) atomic_add_cx(&Z[(size_t)rowJ[m] * ncols + n], -P);
                    }
                }
            }
        }
    }
    /* Gram parts (only pairs sharing a triangle) */
    for (int li = 0; li < nl; ++li) {
        int t = list[li];
        double Gr[3][3], Xr[3][3];
        gram_raw(&M.tris[t], Gr, Xr);
        for (int i = 0; i < 3; ++i) {
            int m = M.t_rwg[3 * t + i];
            if (m < 0 || (rowJ[m] < 0 && rowM[m] < 0)) continue;
            for (int j = 0; j < 3; ++j) {
                int n = M.t_rwg[3 * t + j];
                if (n < 0) continue;
                double c = M.t_cf[3 * t + i] * M.t_cf[3 * t + j];
                double g = c * Gr[i][j], x = c * Xr[i][j];
                if (mode == 0) {
                    if (rowJ[m] >= 0) {
                        Z[(size_t)rowJ[m] * ncols + n] += g;
                        Z[(size_t)rowJ[m] * ncols + N + n] += 0.5 * x;
                    }
                    if (rowM[m] >= 0) Z[(size_t)rowM[m] * ncols + N + n] += 0.5 * g;
                } else {
                    if (rowJ[m] >= 0) Z[(size_t)rowJ[m] * ncols + n] += 0.25 * g;
                }
            }
        }
    }
    free(R); free(list); free(need); free(rowJ); free(rowM);
    mesh_free(&M);
    return 0;
}

/* Gram and twisted Gram as dense N x N (for tests), complex128 row-major */
int or_gram(int nv, const double* V, int nt, const int* T, double* Gout, double* Xout) {
    mesh_t M;
    int rc = mesh_build(nv, V, nt, T, &M);
    if (rc) return rc;
    int N = M.ne;
    memset(Gout, 0, sizeof(double) * (size_t)N * N);
    memset(Xout, 0, sizeof(double) * (size_t)N * N);
    for (int t = 0; t < M.nt; ++t) {
        double Gr[3][3], Xr[3][3];
        gram_raw(&M.tris[t], Gr, Xr);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                int m = M.t_rwg[3 * t + i], n = M.t_rwg[3 * t + j];
                double c = M.t_cf[3 * t + i] * M.t_cf[3 * t + j];
                Gout[(size_t)m * N + n] += c * Gr[i][j];
                Xout[(size_t)m * N + n] += c * Xr[i][j];
            }
    }
    mesh_free(&M);
    return 0;
}

/* Raw operator matrices <f_m, L f_n>, <f_m, n x L f_n>, <f_m, Kbar f_n>, <f_m, n x Kbar f_n>
   (dense N x N each, complex128) at the wavenumber k_re + j k_im: the invariants' tests, and
   the operators of each region of a multi-region surface formulation. */
int or_operators(int nv, const double* V, int nt, const int* T, double k_re, double k_im, int level, double* Lo,
                 double* NLo, double* Ko, double* NKo) {
    const cx k = k_re + I * k_im;
    mesh_t M;
    int rc = mesh_build(nv, V, nt, T, &M);
    if (rc) return rc;
    int N = M.ne;
    cx *L = (cx*)Lo, *NL = (cx*)NLo, *K = (cx*)Ko, *NK = (cx*)NKo;
    memset(L, 0, sizeof(cx) * (size_t)N * N);
    memset(NL, 0, sizeof(cx) * (size_t)N * N);
    memset(K, 0, sizeof(cx) * (size_t)N * N);
    memset(NK, 0, sizeof(cx) * (size_t)N * N);
    rules_t* R = rules_make(level);
#pragma omp parallel for schedule(dynamic, 1)
    for (int a = 0; a < M.nt; ++a)
        for (int b = 0; b < M.nt; ++b) {
            blocks_t B;
            pair_blocks(&M.tris[a], &M.tris[b], R, k, &B);
            for (int i = 0; i < 3; ++i)
                for (int j = 0; j < 3; ++j) {
                    int m = M.t_rwg[3 * a + i], n = M.t_rwg[3 * b + j];
                    double c = M.t_cf[3 * a + i] * M.t_cf[3 * b + j];
                    size_t o = (size_t)m * N + n;
                    atomic_add_cx(&L[o], c * B.L[i][j]);
                    atomic_add_cx(&NL[o], c * B.NL[i][j]);
                    atomic_add_cx(&K[o], c * B.K[i][j]);
                    atomic_add_cx(&NK[o], c * B.NK[i][j]);
                }
        }
    free(R);
    mesh_free(&M);
    return 0;
}

/* ------------------------------------------------ excitation and far field */
/* Plane wave of Sec. III with normalised fields: E = p exp(-jk khat.r), H = (khat x p) exp(-jk khat.r).
 * b^J_m = <f_m, E/2 + n x H/2> (Eq. 49),  b^M_m = <f_m, H/2 - n x E/2> (Eq. 50).
 * Mode 2: the tested fields themselves, <f_m, E> then <f_m, H> (the excitation of a two-region
 * surface formulation, where the tangential traces of E and H are matched).
 * Output b: complex128 [nrhs][nun] (nun = 2N for modes 0 and 2: J block then M block; N for mode 1). */
int or_rhs_planewave(int nv, const double* V, int nt, const int* T, double k, int mode, int nrhs,
                     const double* khat, const double* phat, double* bout) {
    mesh_t M;
    int rc = mesh_build(nv, V, nt, T, &M);
    if (rc) return rc;
    int N = M.ne;
    int nun = mode == 1 ? N : 2 * N;
    cx* b = (cx*)bout;
    memset(b, 0, sizeof(cx) * (size_t)nun * nrhs);
    trirule Rq;
    rule_plain(7, &Rq);
    for (int s = 0; s < nrhs; ++s) {
        const double* kh = khat + 3 * s;
        const double* ph = phat + 3 * s;
        double hp[3];
        v_cross(kh, ph, hp);
        for (int t = 0; t < M.nt; ++t) {
            const tri_t* Tt = &M.tris[t];
            for (int q = 0; q < Rq.n; ++q) {
                double r[3];
                bary_point(Tt, Rq.b[q], r);
                cx ph_ = cexp(-I * k * v_dot(kh, r));
                double nE[3], nH[3];
                v_cross(Tt->n, ph, nE);
                v_cross(Tt->n, hp, nH);
                double w = Rq.w[q] * Tt->area;
                for (int i = 0; i < 3; ++i) {
                    int m = M.t_rwg[3 * t + i];
                    double gi[3];
                    v_sub(r, Tt->p[i], gi);
                    double c = M.t_cf[3 * t + i];
                    if (mode == 2) {
                        b[(size_t)s * nun + m] += v_dot(gi, ph) * ph_ * c * w;
                        b[(size_t)s * nun + N + m] += v_dot(gi, hp) * ph_ * c * w;
                        continue;
                    }
                    cx bj = 0.5 * (v_dot(gi, ph) + v_dot(gi, nH)) * ph_ * c * w;
                    b[(size_t)s * nun + m] += bj;
                    if (mode == 0) {
                        cx bm = 0.5 * (v_dot(gi, hp) - v_dot(gi, nE)) * ph_ * c * w;
                        b[(size_t)s * nun + N + m] += bm;
                    }
                }
            }
        }
    }
    mesh_free(&M);
    return 0;
}

/* Far-field vector F(rhat) such that E_sca ~ exp(-jkr)/r F and sigma = 4 pi |F|^2 for unit
 * incident amplitude:  F = -jk/(4 pi) [ (I - rr) N_J - rhat x N_M ],  N_X = sum_n x_n int f_n exp(jk rhat.r').
 * x: complex128 [nun] (mode 0: J then M; mode 1: J only).  out: complex128 [ndir][3]. */
int or_farfield(int nv, const double* V, int nt, const int* T, double k, int mode, const double* xin,
                int ndir, const double* dirs, double* out) {
    mesh_t M;
    int rc = mesh_build(nv, V, nt, T, &M);
    if (rc) return rc;
    int N = M.ne;
    const cx* x = (const cx*)xin;
    cx* F = (cx*)out;
    trirule Rq;
    rule_plain(7, &Rq);
#pragma omp parallel for
    for (int dI = 0; dI < ndir; ++dI) {
        const double* rh = dirs + 3 * dI;
        cx NJ[3] = {0, 0, 0}, NM[3] = {0, 0, 0};
        for (int t = 0; t < M.nt; ++t) {
            const tri_t* Tt = &M.tris[t];
            for (int q = 0; q < Rq.n; ++q) {
                double r[3];
                bary_point(Tt, Rq.b[q], r);
                cx ph = cexp(I * k * v_dot(rh, r)) * Rq.w[q] * Tt->area;
                for (int i = 0; i < 3; ++i) {
                    int m = M.t_rwg[3 * t + i];
                    double c = M.t_cf[3 * t + i];
                    double gi[3];
                    v_sub(r, Tt->p[i], gi);
                    cx aJ = x[m] * c * ph;
                    cx aM = (mode == 0) ? x[N + m] * c * ph : 0;
                    for (int d = 0; d < 3; ++d) { NJ[d] += aJ * gi[d]; NM[d] += aM * gi[d]; }
                }
            }
        }
        cx rN = NJ[0] * rh[0] + NJ[1] * rh[1] + NJ[2] * rh[2];
        cx cr[3];
        cr[0] = rh[1] * NM[2] - rh[2] * NM[1];
        cr[1] = rh[2] * NM[0] - rh[0] * NM[2];
        cr[2] = rh[0] * NM[1] - rh[1] * NM[0];
        for (int d = 0; d < 3; ++d) F[3 * dI + d] = (-I * k / (4.0 * PI)) * (NJ[d] - rh[d] * rN - cr[d]);
    }
    mesh_free(&M);
    return 0;
}

/* quadrature rule access for tests: writes barycentrics [n][3] and weights [n]; returns n */
int or_rule(int kind, int n, int q, double* bary, double* w) {
    trirule R;
    if (kind == 0) rule_plain(n, &R);
    else if (kind == 1) rule_edge(n, q, &R);
    else rule_vertex(n, q, &R);
    for (int i = 0; i < R.n; ++i) {
        for (int d = 0; d < 3; ++d) bary[3 * i + d] = R.b[i][d];
        w[i] = R.w[i];
    }
    return R.n;
}

int or_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
