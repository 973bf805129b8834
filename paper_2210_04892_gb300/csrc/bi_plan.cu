// Host-only plan of the multilevel product: RWG numbering, octree, near and interaction
// lists, parent-centred translation lists, angular sampling and interpolation tables, built by
// the same host code as bi_setup but without a device.  It lets the set-up logic be checked on
// a machine without a GPU.
#include <cstring>
#include <exception>
#include <new>
#include <string>
#include <vector>

#include "bi_internal.h"

struct bi_plan_s {
    bi_handle_s h;
};

static thread_local std::string g_plan_error;

namespace {

template <typename V>
int put(const std::vector<V>& v, void* out, int64_t bytes, int64_t* count) {
    if (count) *count = (int64_t)v.size();
    if (!out) return BI_OK;
    if (bytes < (int64_t)(v.size() * sizeof(V))) return BI_ERR_ARG;
    if (!v.empty()) std::memcpy(out, v.data(), v.size() * sizeof(V));
    return BI_OK;
}

}  // namespace

extern "C" int bi_plan_create(const double* verts, int nv, const int* tris, int nt, double k0, const bi_params* opt,
                              bi_plan* out) {
    if (!out) return BI_ERR_ARG;
    *out = nullptr;
    if (!verts || !tris || nv < 3 || nt < 4 || !(k0 > 0)) {
        g_plan_error = "bi_plan_create: null mesh, fewer than 4 triangles, or k0 <= 0";
        return BI_ERR_ARG;
    }
    bi_plan_s* p = new (std::nothrow) bi_plan_s();
    if (!p) return BI_ERR_OOM;
    bi_handle_s* h = &p->h;
    if (opt) h->prm = *opt;
    else bi_default_params(&h->prm);
    if (!bi_params_valid(h->prm) || h->prm.op_mode > 1) {
        g_plan_error = "bi_plan_create: parameter out of range (op_mode 0 or 1)";
        delete p;
        return BI_ERR_ARG;
    }
    if (h->prm.k_im < -k0) {
        g_plan_error = "bi_plan_create: k_im outside [-k0, 0]";
        delete p;
        return BI_ERR_ARG;
    }
    h->k = k0;
    h->ki = h->prm.k_im;
    h->nX = h->prm.op_mode == 0 ? 2 : 1;
    try {
        bi_build_rwg(h, verts, nv, tris, nt);
        h->nun = h->nX * h->N;
        bi_build_tree(h, verts);
        bi_build_sampling(h);
        bi_build_interp(h);
        bi_plan_translate_lists(h);
    } catch (const bi_error& e) {
        g_plan_error = e.msg;
        delete p;
        return e.code;
    } catch (const std::exception& e) {
        g_plan_error = std::string("bi_plan_create: ") + e.what();
        delete p;
        return BI_ERR_ARG;
    }
    *out = p;
    return BI_OK;
}

extern "C" int bi_plan_info(bi_plan p, bi_info_t* info) {
    if (!p || !info) return BI_ERR_ARG;
    const bi_handle_s& h = p->h;
    std::memset(info, 0, sizeof(*info));
    info->n_rwg = h.N;
    info->n_unknowns = h.nun;
    info->levels = h.nlev;
    info->leaf_level = h.leaf;
    for (int l = 0; l < h.nlev && l < 32; ++l) {
        info->boxes[l] = h.lev[l].nbox;
        info->L[l] = h.lev[l].L;
        info->K[l] = h.lev[l].K;
        info->interactions[l] = h.lev[l].n_inter;
    }
    info->near_pairs = h.near_nnz;
    info->root_size = h.lev[0].a;
    return BI_OK;
}

static int plan_get(const bi_plan_s* p, int what, int level, void* out, int64_t bytes, int64_t* count);

extern "C" int bi_plan_get(bi_plan p, int what, int level, void* out, int64_t bytes, int64_t* count) {
    if (!p) return BI_ERR_ARG;
    try {
        return plan_get(p, what, level, out, bytes, count);
    } catch (const std::exception&) {
        return BI_ERR_OOM;              // a converted copy (codes 11, 40, 41) did not fit
    }
}

static int plan_get(const bi_plan_s* p, int what, int level, void* out, int64_t bytes, int64_t* count) {
    const bi_handle_s& h = p->h;
    const bool lev_ok = level >= 0 && level < h.nlev;
    const bool far_ok = lev_ok && level >= 2 && level <= h.leaf;
    const bool itp_ok = level >= 2 && level + 1 <= h.leaf && (size_t)level < h.itp.size();
    switch (what) {
        case 0: return put(h.leaf_start, out, bytes, count);
        case 1: return put(h.near_ptr, out, bytes, count);
        case 2: return put(h.near_src, out, bytes, count);
        case 3: return lev_ok ? put(h.lev[level].coords, out, bytes, count) : BI_ERR_ARG;
        case 4: return lev_ok && level >= 1 ? put(h.lev[level].parent, out, bytes, count) : BI_ERR_ARG;
        case 5: return lev_ok && level + 1 < h.nlev ? put(h.lev[level].child_ptr, out, bytes, count) : BI_ERR_ARG;
        case 6: return far_ok ? put(h.lev[level].il_ptr, out, bytes, count) : BI_ERR_ARG;
        case 7: return far_ok ? put(h.lev[level].il_src, out, bytes, count) : BI_ERR_ARG;
        case 8: return far_ok ? put(h.lev[level].il_off, out, bytes, count) : BI_ERR_ARG;
        case 9: return far_ok ? put(h.lev[level].tp_ptr, out, bytes, count) : BI_ERR_ARG;
        case 10: return far_ok ? put(h.lev[level].tp_src, out, bytes, count) : BI_ERR_ARG;
        case 11: {
            if (!far_ok) return BI_ERR_ARG;
            std::vector<int> c(h.lev[level].tp_code.begin(), h.lev[level].tp_code.end());
            return put(c, out, bytes, count);
        }
        case 12: return put(h.perm, out, bytes, count);
        case 13: return put(h.edges, out, bytes, count);
        case 14: return put(h.tplus, out, bytes, count);
        case 15: return put(h.tminus, out, bytes, count);
        case 20: return far_ok ? put(h.lev[level].theta, out, bytes, count) : BI_ERR_ARG;
        case 21: return far_ok ? put(h.lev[level].wtheta, out, bytes, count) : BI_ERR_ARG;
        case 22: return itp_ok ? put(h.itp[level].th_src, out, bytes, count) : BI_ERR_ARG;
        case 23: return itp_ok ? put(h.itp[level].th_flip, out, bytes, count) : BI_ERR_ARG;
        case 24: return itp_ok ? put(h.itp[level].th_w, out, bytes, count) : BI_ERR_ARG;
        case 25: return itp_ok ? put(h.itp[level].ph_src, out, bytes, count) : BI_ERR_ARG;
        case 26: return itp_ok ? put(h.itp[level].ph_w, out, bytes, count) : BI_ERR_ARG;
        case 27: return itp_ok ? put(h.itp[level].tth_ptr, out, bytes, count) : BI_ERR_ARG;
        case 28: return itp_ok ? put(h.itp[level].tth_dst, out, bytes, count) : BI_ERR_ARG;
        case 29: return itp_ok ? put(h.itp[level].tth_flip, out, bytes, count) : BI_ERR_ARG;
        case 30: return itp_ok ? put(h.itp[level].tth_w, out, bytes, count) : BI_ERR_ARG;
        case 31: return itp_ok ? put(h.itp[level].tph_ptr, out, bytes, count) : BI_ERR_ARG;
        case 32: return itp_ok ? put(h.itp[level].tph_dst, out, bytes, count) : BI_ERR_ARG;
        case 33: return itp_ok ? put(h.itp[level].tph_w, out, bytes, count) : BI_ERR_ARG;
        case 40:
        case 41: {
            if (!far_ok) return BI_ERR_ARG;
            std::vector<int> di;
            std::vector<double> hk;
            bi_translation_series(&h, level, di, hk);
            return what == 40 ? put(di, out, bytes, count) : put(hk, out, bytes, count);
        }
        default: return BI_ERR_ARG;
    }
}

extern "C" const char* bi_plan_last_error(void) { return g_plan_error.c_str(); }

extern "C" void bi_plan_destroy(bi_plan p) { delete p; }
