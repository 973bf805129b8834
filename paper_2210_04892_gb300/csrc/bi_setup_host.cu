// Host-side setup: RWG functions, octree, near/interaction lists, angular sampling and
// Lagrange interpolation tables.  Integer and table work only; every integral is
// evaluated on the device (bi_setup_device.cu).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <unordered_map>

#include "bi_internal.h"

static const double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------------------------
// Gauss-Legendre nodes on (-1, 1) (Golub-Welsch is not needed at these orders: Newton
// on the three-term recurrence from the Chebyshev-like initial guess).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (i + 0.75) / (n + 0.5));
        double pd = 1.0;
        for (int it = 0; it < 200; ++it) {
            double pm = 1.0, p = z;
            for (int k = 2; k <= n; ++k) {
                double pn = ((2 * k - 1) * z * p - (k - 1) * pm) / k;
                pm = p;
                p = pn;
            }
            if (n == 1) { p = z; pm = 1.0; }
            pd = n * (z * p - pm) / (z * z - 1.0);
            double dz = p / pd;
            z -= dz;
            if (std::fabs(dz) < 1e-15) break;
        }
        double pm = 1.0, p = z;
        for (int k = 2; k <= n; ++k) {
            double pn = ((2 * k - 1) * z * p - (k - 1) * pm) / k;
            pm = p;
            p = pn;
        }
        if (n == 1) { p = z; pm = 1.0; }
        pd = n * (z * p - pm) / (z * z - 1.0);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * pd * pd);
    }
}

// ---------------------------------------------------------------------------------
// RWG functions (Sec. II.C; Rao, Wilton, Glisson 1982).  One function per interior
// edge, numbered by (min vertex, max vertex).  T+ is the triangle in which the edge
// runs from the smaller to the larger vertex index.
namespace {
struct half_edge {
    int lo, hi, from, tri, opp;
};
}  // namespace

void bi_build_rwg(bi_handle_s* h, const double* V, int nv, const int* T, int nt) {
    for (int t = 0; t < nt; ++t) {
        for (int a = 0; a < 3; ++a)
            if (T[3 * t + a] < 0 || T[3 * t + a] >= nv) throw bi_error{BI_ERR_MESH, "triangle vertex index out of range"};
        const double* p0 = V + 3 * T[3 * t];
        const double* p1 = V + 3 * T[3 * t + 1];
        const double* p2 = V + 3 * T[3 * t + 2];
        double e1[3], e2[3];
        for (int d = 0; d < 3; ++d) { e1[d] = p1[d] - p0[d]; e2[d] = p2[d] - p0[d]; }
        double c0 = e1[1] * e2[2] - e1[2] * e2[1], c1 = e1[2] * e2[0] - e1[0] * e2[2], c2 = e1[0] * e2[1] - e1[1] * e2[0];
        double a2 = std::sqrt(c0 * c0 + c1 * c1 + c2 * c2);
        double l2 = std::max(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2], e2[0] * e2[0] + e2[1] * e2[1] + e2[2] * e2[2]);
        if (!(a2 > 2e-14 * l2)) throw bi_error{BI_ERR_MESH, "degenerate triangle " + std::to_string(t)};
    }
    std::vector<half_edge> he(3 * (size_t)nt);
    for (int t = 0; t < nt; ++t)
        for (int k = 0; k < 3; ++k) {
            int a = T[3 * t + k], b = T[3 * t + (k + 1) % 3];
            he[3 * t + k] = {std::min(a, b), std::max(a, b), a, t, (k + 2) % 3};
        }
    std::sort(he.begin(), he.end(), [](const half_edge& p, const half_edge& q) {
        return p.lo != q.lo ? p.lo < q.lo : (p.hi != q.hi ? p.hi < q.hi : p.tri < q.tri);
    });
    h->edges.clear();
    h->tplus.clear(); h->tminus.clear(); h->lplus.clear(); h->lminus.clear();
    size_t i = 0;
    while (i < he.size()) {
        size_t j = i + 1;
        while (j < he.size() && he[j].lo == he[i].lo && he[j].hi == he[i].hi) ++j;
        if (j - i != 2)
            throw bi_error{BI_ERR_MESH, "edge (" + std::to_string(he[i].lo) + "," + std::to_string(he[i].hi) +
                                            ") has " + std::to_string(j - i) + " triangles (open or non-manifold surface)"};
        const half_edge& x = he[i];
        const half_edge& y = he[i + 1];
        bool xp = (x.from == x.lo), yp = (y.from == y.lo);
        if (xp == yp)
            throw bi_error{BI_ERR_MESH, "inconsistent orientation at edge (" + std::to_string(x.lo) + "," +
                                            std::to_string(x.hi) + ")"};
        const half_edge& P = xp ? x : y;
        const half_edge& M = xp ? y : x;
        h->edges.push_back(P.lo);
        h->edges.push_back(P.hi);
        h->tplus.push_back(P.tri);
        h->lplus.push_back(P.opp);
        h->tminus.push_back(M.tri);
        h->lminus.push_back(M.opp);
        i = j;
    }
    h->N = (int)h->tplus.size();
    h->nt = nt;
    h->nv = nv;
    h->tri_vid_host.assign(T, T + 3 * (size_t)nt);
}

// ---------------------------------------------------------------------------------
// Octree over RWG midpoints.
static inline uint64_t spread3(uint64_t v) {
    // 21 bits -> every third bit
    v &= 0x1fffff;
    v = (v | v << 32) & 0x1f00000000ffffULL;
    v = (v | v << 16) & 0x1f0000ff0000ffULL;
    v = (v | v << 8) & 0x100f00f00f00f00fULL;
    v = (v | v << 4) & 0x10c30c30c30c30c3ULL;
    v = (v | v << 2) & 0x1249249249249249ULL;
    return v;
}
static inline uint64_t morton(int i, int j, int k) { return spread3(i) | (spread3(j) << 1) | (spread3(k) << 2); }
static inline uint64_t coord_key(int i, int j, int k) { return ((uint64_t)i << 42) | ((uint64_t)j << 21) | (uint64_t)k; }

void bi_build_tree(bi_handle_s* h, const double* V) {
    const int N = h->N;
    const double lambda = 2.0 * kPi / h->k;
    std::vector<double> mid(3 * (size_t)N);
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
    for (int n = 0; n < N; ++n) {
        const double* a = V + 3 * h->edges[2 * n];
        const double* b = V + 3 * h->edges[2 * n + 1];
        for (int d = 0; d < 3; ++d) {
            mid[3 * n + d] = 0.5 * (a[d] + b[d]);
            lo[d] = std::min(lo[d], mid[3 * n + d]);
            hi[d] = std::max(hi[d], mid[3 * n + d]);
        }
    }
    double extent = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
    double a_leaf = h->prm.leaf_box * lambda;
    int nlev = h->prm.levels;
    if (nlev <= 0) {
        nlev = 1;
        while (a_leaf * std::ldexp(1.0, nlev - 1) < extent * (1.0 + 1e-12) && nlev < BI_MAXLEV) ++nlev;
    }
    double root = a_leaf * std::ldexp(1.0, nlev - 1);
    if (root < extent * (1.0 - 1e-12) || nlev > 21)
        throw bi_error{BI_ERR_ARG, "levels too small for the mesh extent or too many levels"};
    h->nlev = nlev;
    h->leaf = nlev - 1;
    double corner[3];
    for (int d = 0; d < 3; ++d) corner[d] = 0.5 * (lo[d] + hi[d]) - 0.5 * root;
    const int nside = 1 << h->leaf;
    std::vector<int> ci(3 * (size_t)N);
    std::vector<uint64_t> mk(N);
    for (int n = 0; n < N; ++n) {
        for (int d = 0; d < 3; ++d) {
            int c = (int)std::floor((mid[3 * n + d] - corner[d]) / a_leaf);
            ci[3 * n + d] = std::min(std::max(c, 0), nside - 1);
        }
        mk[n] = morton(ci[3 * n], ci[3 * n + 1], ci[3 * n + 2]);
    }
    // margin: twice the largest distance from an RWG midpoint to a vertex of its support
    {
        double ov = 0.0;
        for (int n = 0; n < N; ++n) {
            int tri[2] = {h->tplus[n], h->tminus[n]};
            for (int s = 0; s < 2; ++s)
                for (int a = 0; a < 3; ++a) {
                    const double* q = V + 3 * h->tri_vid_host[3 * tri[s] + a];
                    double d2 = 0.0;
                    for (int d = 0; d < 3; ++d) d2 += (q[d] - mid[3 * n + d]) * (q[d] - mid[3 * n + d]);
                    ov = std::max(ov, std::sqrt(d2));
                }
        }
        h->margin = 2.0 * ov;
    }
    h->perm.resize(N);
    for (int n = 0; n < N; ++n) h->perm[n] = n;
    std::stable_sort(h->perm.begin(), h->perm.end(), [&](int a, int b) { return mk[a] < mk[b]; });

    h->lev.assign(nlev, level_t());
    for (int l = 0; l < nlev; ++l) {
        level_t& L = h->lev[l];
        L.a = a_leaf * std::ldexp(1.0, h->leaf - l);
        int shift = 3 * (h->leaf - l);
        for (int t = 0; t < N; ++t) {
            uint64_t key = mk[h->perm[t]] >> shift;
            if (L.key.empty() || L.key.back() != key) {
                L.key.push_back(key);
                int n = h->perm[t];
                int c[3] = {ci[3 * n] >> (h->leaf - l), ci[3 * n + 1] >> (h->leaf - l), ci[3 * n + 2] >> (h->leaf - l)};
                for (int d = 0; d < 3; ++d) {
                    L.coords.push_back(c[d]);
                    L.center.push_back(corner[d] + (c[d] + 0.5) * L.a);
                }
            }
        }
        L.nbox = (int)L.key.size();
    }
    // leaf ranges
    level_t& LF = h->lev[h->leaf];
    h->leaf_start.assign(LF.nbox + 1, 0);
    {
        int b = 0;
        for (int t = 0; t < N; ++t) {
            uint64_t key = mk[h->perm[t]];
            while (LF.key[b] != key) {
                ++b;
                h->leaf_start[b] = t;
            }
        }
        h->leaf_start[LF.nbox] = N;
        h->max_leaf_count = 0;
        for (int b2 = 0; b2 < LF.nbox; ++b2)
            h->max_leaf_count = std::max(h->max_leaf_count, h->leaf_start[b2 + 1] - h->leaf_start[b2]);
    }
    // parent / child links (Morton order keeps children of one parent contiguous)
    for (int l = 1; l < nlev; ++l) {
        level_t& C = h->lev[l];
        level_t& P = h->lev[l - 1];
        C.parent.resize(C.nbox);
        P.child_ptr.assign(P.nbox + 1, 0);
        int p = 0;
        for (int b = 0; b < C.nbox; ++b) {
            uint64_t pk = C.key[b] >> 3;
            while (P.key[p] != pk) ++p;
            C.parent[b] = p;
            P.child_ptr[p + 1] = b + 1;
        }
        for (int q = 1; q <= P.nbox; ++q) P.child_ptr[q] = std::max(P.child_ptr[q], P.child_ptr[q - 1]);
    }
    // near lists at the leaf: same or touching boxes
    {
        std::unordered_map<uint64_t, int> idx;
        idx.reserve(LF.nbox * 2);
        for (int b = 0; b < LF.nbox; ++b) idx[coord_key(LF.coords[3 * b], LF.coords[3 * b + 1], LF.coords[3 * b + 2])] = b;
        h->near_ptr.assign(LF.nbox + 1, 0);
        h->near_src.clear();
        h->near_blk.clear();
        int64_t off = 0;
        for (int b = 0; b < LF.nbox; ++b) {
            std::vector<int> lst;
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        int x = LF.coords[3 * b] + dx, y = LF.coords[3 * b + 1] + dy, z = LF.coords[3 * b + 2] + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= nside || y >= nside || z >= nside) continue;
                        auto it = idx.find(coord_key(x, y, z));
                        if (it != idx.end()) lst.push_back(it->second);
                    }
            std::sort(lst.begin(), lst.end());
            int mb = h->leaf_start[b + 1] - h->leaf_start[b];
            for (int s : lst) {
                h->near_src.push_back(s);
                h->near_blk.push_back(off);
                off += (int64_t)mb * (h->leaf_start[s + 1] - h->leaf_start[s]);
            }
            h->near_ptr[b + 1] = (int)h->near_src.size();
        }
        h->near_nnz = off;
        h->near_blk.push_back(off);
        h->near_ncol_max = 0;
        for (int b = 0; b < LF.nbox; ++b) {
            int mb = h->leaf_start[b + 1] - h->leaf_start[b];
            int ncol = (int)((h->near_blk[h->near_ptr[b + 1]] - h->near_blk[h->near_ptr[b]]) / mb);
            h->near_ncol_max = std::max(h->near_ncol_max, ncol);
        }
    }
    // interaction lists on levels 2..leaf: children of the parent's neighbours that do not touch
    for (int l = 2; l < nlev; ++l) {
        level_t& C = h->lev[l];
        level_t& P = h->lev[l - 1];
        std::unordered_map<uint64_t, int> pidx;
        pidx.reserve(P.nbox * 2);
        for (int b = 0; b < P.nbox; ++b) pidx[coord_key(P.coords[3 * b], P.coords[3 * b + 1], P.coords[3 * b + 2])] = b;
        int pside = 1 << (l - 1);
        C.il_ptr.assign(C.nbox + 1, 0);
        C.il_src.clear();
        C.il_off.clear();
        for (int b = 0; b < C.nbox; ++b) {
            int p = C.parent[b];
            for (int dx = -1; dx <= 1; ++dx)
                for (int dy = -1; dy <= 1; ++dy)
                    for (int dz = -1; dz <= 1; ++dz) {
                        int x = P.coords[3 * p] + dx, y = P.coords[3 * p + 1] + dy, z = P.coords[3 * p + 2] + dz;
                        if (x < 0 || y < 0 || z < 0 || x >= pside || y >= pside || z >= pside) continue;
                        auto it = pidx.find(coord_key(x, y, z));
                        if (it == pidx.end()) continue;
                        int q = it->second;
                        for (int s = P.child_ptr[q]; s < P.child_ptr[q + 1]; ++s) {
                            int ox = C.coords[3 * b] - C.coords[3 * s];
                            int oy = C.coords[3 * b + 1] - C.coords[3 * s + 1];
                            int oz = C.coords[3 * b + 2] - C.coords[3 * s + 2];
                            if (std::abs(ox) <= 1 && std::abs(oy) <= 1 && std::abs(oz) <= 1) continue;
                            C.il_src.push_back(s);
                            C.il_off.push_back((ox + 3) * 49 + (oy + 3) * 7 + (oz + 3));
                        }
                    }
            C.il_ptr[b + 1] = (int)C.il_src.size();
        }
        C.n_inter = (int64_t)C.il_src.size();
    }
}

// ---------------------------------------------------------------------------------
// Angular sampling per level: L from the excess-bandwidth rule with the box diagonal
// enlarged by twice the largest RWG overhang; (L+1) Gauss-Legendre points in cos(theta)
// and 2(L+1) uniform points in phi.
void bi_build_sampling(bi_handle_s* h) {
    const double d0 = (double)h->prm.digits;
    for (int l = 2; l <= h->leaf; ++l) {
        level_t& L = h->lev[l];
        double d = std::sqrt(3.0) * L.a + h->margin;
        double kd = h->k * d;
        L.L = (int)std::ceil(kd + 1.8 * std::pow(d0, 2.0 / 3.0) * std::cbrt(kd));
        L.nth = L.L + 1;
        L.nph = 2 * (L.L + 1);
        L.K = L.nth * L.nph;
        std::vector<double> x, w;
        gauss_legendre(L.nth, x, w);
        // theta ascending <=> cos(theta) descending
        std::vector<int> ord(L.nth);
        for (int i = 0; i < L.nth; ++i) ord[i] = i;
        std::sort(ord.begin(), ord.end(), [&](int a, int b) { return x[a] > x[b]; });
        L.theta.resize(L.nth);
        L.wtheta.resize(L.nth);
        for (int i = 0; i < L.nth; ++i) {
            L.theta[i] = std::acos(std::max(-1.0, std::min(1.0, x[ord[i]])));
            L.wtheta[i] = w[ord[i]];
        }
    }
}

// Lagrange weights of nodes t[0..p) at x
static void lagrange(const double* t, int p, double x, double* w) {
    for (int a = 0; a < p; ++a) {
        double v = 1.0;
        for (int b = 0; b < p; ++b)
            if (b != a) v *= (x - t[b]) / (t[a] - t[b]);
        w[a] = v;
    }
}

void bi_build_interp(bi_handle_s* h) {
    h->itp.assign(h->nlev, interp_t());
    for (int l = 2; l + 1 <= h->leaf; ++l) {
        const level_t& P = h->lev[l];
        const level_t& C = h->lev[l + 1];
        interp_t& I = h->itp[l];
        int p = h->prm.interp_order;
        I.p_th = std::min(p, C.nth);
        I.p_ph = std::min(p, C.nph);
        // extended theta list across both poles: -theta (reversed), theta, 2 pi - theta (reversed)
        int nc = C.nth;
        std::vector<double> ext(3 * nc);
        std::vector<int> esrc(3 * nc), eflip(3 * nc);
        for (int i = 0; i < nc; ++i) {
            ext[i] = -C.theta[nc - 1 - i];
            esrc[i] = nc - 1 - i;
            eflip[i] = 1;
            ext[nc + i] = C.theta[i];
            esrc[nc + i] = i;
            eflip[nc + i] = 0;
            ext[2 * nc + i] = 2 * kPi - C.theta[nc - 1 - i];
            esrc[2 * nc + i] = nc - 1 - i;
            eflip[2 * nc + i] = 1;
        }
        I.th_src.resize((size_t)P.nth * I.p_th);
        I.th_flip.resize((size_t)P.nth * I.p_th);
        I.th_w.resize((size_t)P.nth * I.p_th);
        for (int ip = 0; ip < P.nth; ++ip) {
            double x = P.theta[ip];
            int pos = (int)(std::upper_bound(ext.begin(), ext.end(), x) - ext.begin());
            int s0 = pos - I.p_th / 2;
            s0 = std::max(0, std::min(s0, 3 * nc - I.p_th));
            std::vector<double> w(I.p_th);
            lagrange(&ext[s0], I.p_th, x, w.data());
            for (int t = 0; t < I.p_th; ++t) {
                I.th_src[(size_t)ip * I.p_th + t] = esrc[s0 + t];
                I.th_flip[(size_t)ip * I.p_th + t] = eflip[s0 + t];
                I.th_w[(size_t)ip * I.p_th + t] = w[t];
            }
        }
        double dph = 2 * kPi / C.nph;
        I.ph_src.resize((size_t)P.nph * I.p_ph);
        I.ph_w.resize((size_t)P.nph * I.p_ph);
        for (int jp = 0; jp < P.nph; ++jp) {
            double x = 2 * kPi * jp / P.nph;
            int c = (int)std::floor(x / dph + 1e-12);
            int s0 = c - (I.p_ph / 2 - 1);
            std::vector<double> t(I.p_ph), w(I.p_ph);
            for (int q = 0; q < I.p_ph; ++q) t[q] = (s0 + q) * dph;
            lagrange(t.data(), I.p_ph, x, w.data());
            for (int q = 0; q < I.p_ph; ++q) {
                int j = ((s0 + q) % C.nph + C.nph) % C.nph;
                I.ph_src[(size_t)jp * I.p_ph + q] = j;
                I.ph_w[(size_t)jp * I.p_ph + q] = w[q];
            }
        }
        // transposed lists
        I.tth_ptr.assign(C.nth + 1, 0);
        for (size_t e = 0; e < I.th_src.size(); ++e) I.tth_ptr[I.th_src[e] + 1]++;
        for (int i = 0; i < C.nth; ++i) I.tth_ptr[i + 1] += I.tth_ptr[i];
        I.tth_dst.resize(I.th_src.size());
        I.tth_flip.resize(I.th_src.size());
        I.tth_w.resize(I.th_src.size());
        {
            std::vector<int> fill(I.tth_ptr.begin(), I.tth_ptr.end() - 1);
            for (int ip = 0; ip < P.nth; ++ip)
                for (int t = 0; t < I.p_th; ++t) {
                    size_t e = (size_t)ip * I.p_th + t;
                    int pos = fill[I.th_src[e]]++;
                    I.tth_dst[pos] = ip;
                    I.tth_flip[pos] = I.th_flip[e];
                    I.tth_w[pos] = I.th_w[e];
                }
        }
        I.tph_ptr.assign(C.nph + 1, 0);
        for (size_t e = 0; e < I.ph_src.size(); ++e) I.tph_ptr[I.ph_src[e] + 1]++;
        for (int j = 0; j < C.nph; ++j) I.tph_ptr[j + 1] += I.tph_ptr[j];
        I.tph_dst.resize(I.ph_src.size());
        I.tph_w.resize(I.ph_src.size());
        {
            std::vector<int> fill(I.tph_ptr.begin(), I.tph_ptr.end() - 1);
            for (int jp = 0; jp < P.nph; ++jp)
                for (int q = 0; q < I.p_ph; ++q) {
                    size_t e = (size_t)jp * I.p_ph + q;
                    int pos = fill[I.ph_src[e]]++;
                    I.tph_dst[pos] = jp;
                    I.tph_w[pos] = I.ph_w[e];
                }
        }
    }
}
