// Complex arithmetic and pattern helpers shared by the product kernels.
#pragma once
#include <cstdint>

template <typename T>
struct cpx {
    T x, y;
};
template <typename T>
__device__ __forceinline__ cpx<T> cmul(cpx<T> a, cpx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> cmulc(cpx<T> a, cpx<T> b) {  // conj(a) * b
    return {a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename T>
__device__ __forceinline__ cpx<T> cadd(cpx<T> a, cpx<T> b) {
    return {a.x + b.x, a.y + b.y};
}
template <typename T>
__device__ __forceinline__ cpx<T> csub(cpx<T> a, cpx<T> b) {
    return {a.x - b.x, a.y - b.y};
}
template <typename T>
__device__ __forceinline__ cpx<T> cscale(cpx<T> a, T s) {
    return {a.x * s, a.y * s};
}
template <typename T>
__device__ __forceinline__ void cfma(cpx<T>& acc, cpx<T> a, cpx<T> b) {
    acc.x = fma(a.x, b.x, acc.x);
    acc.x = fma(-a.y, b.y, acc.x);
    acc.y = fma(a.x, b.y, acc.y);
    acc.y = fma(a.y, b.x, acc.y);
}
template <typename T>
__device__ __forceinline__ cpx<T> czero() {
    return {T(0), T(0)};
}

// Antipodal pairs of directions: (it, jp) <-> (nth - 1 - it, jp + nph/2 mod nph).  The leaf
// pattern arrays hold the first K/2 directions of the theta-major numbering, one of each pair;
// a stored (theta, phi) pair (a, b) reads (conj a, -conj b) at the antipode (real basis
// functions; the antipodal map keeps theta-hat and reverses phi-hat).
__device__ __forceinline__ int antipode(int kk, int K, int nph) {
    const int it = kk / nph, jp = kk - it * nph, jm = jp + (nph >> 1);
    return (K / nph - 1 - it) * nph + (jm >= nph ? jm - nph : jm);
}
template <typename T>
__device__ __forceinline__ cpx<T> cconj(cpx<T> a) {
    return {a.x, -a.y};
}
template <typename T>
__device__ __forceinline__ cpx<T> cnegconj(cpx<T> a) {
    return {-a.x, a.y};
}
// One direction's receive terms (R = conj(F), khat x V = (-V_phi, V_theta)):
//   J += R.V - RX.(khat x V),  M += -R.(khat x V) - RX.V
template <typename T, int MODE>
__device__ __forceinline__ void recv_terms(cpx<T> Ft, cpx<T> Fp, cpx<T> Xt, cpx<T> Xp, cpx<T> Vt, cpx<T> Vp, cpx<T>& sJ,
                                           cpx<T>& sM) {
    sJ = cadd(sJ, csub(cadd(cmulc(Ft, Vt), cmulc(Fp, Vp)), csub(cmul(Xp, Vt), cmul(Xt, Vp))));
    if (MODE == 0) {
        const cpx<T> t = csub(cmulc(Ft, Vp), cmulc(Fp, Vt));
        sM = cadd(sM, csub(t, cadd(cmul(Xt, Vt), cmul(Xp, Vp))));
    }
}

// The receive terms of one stored direction (V) and of its antipode (W, where the patterns
// read (conj F_theta, -conj F_phi), (conj X_theta, -conj X_phi)), written out as real fused
// multiply-adds into separate accumulators:
//   stored:   J += conj(Ft) Vt + conj(Fp) Vp - Xp Vt + Xt Vp,   M += conj(Ft) Vp - conj(Fp) Vt - Xt Vt - Xp Vp
//   antipode: J += Ft Wt - Fp Wp + conj(Xp) Wt + conj(Xt) Wp,   M += Ft Wp + Fp Wt - conj(Xt) Wt + conj(Xp) Wp
template <typename T, int MODE>
__device__ __forceinline__ void recv_pair(cpx<T> Ft, cpx<T> Fp, cpx<T> Xt, cpx<T> Xp, cpx<T> Vt, cpx<T> Vp, cpx<T> Wt,
                                          cpx<T> Wp, cpx<T>& sJ, cpx<T>& sM, cpx<T>& aJ, cpx<T>& aM) {
    sJ.x = fma(Ft.x, Vt.x, sJ.x); sJ.x = fma(Ft.y, Vt.y, sJ.x); sJ.x = fma(Fp.x, Vp.x, sJ.x); sJ.x = fma(Fp.y, Vp.y, sJ.x);
    sJ.x = fma(-Xp.x, Vt.x, sJ.x); sJ.x = fma(Xp.y, Vt.y, sJ.x); sJ.x = fma(Xt.x, Vp.x, sJ.x); sJ.x = fma(-Xt.y, Vp.y, sJ.x);
    sJ.y = fma(Ft.x, Vt.y, sJ.y); sJ.y = fma(-Ft.y, Vt.x, sJ.y); sJ.y = fma(Fp.x, Vp.y, sJ.y); sJ.y = fma(-Fp.y, Vp.x, sJ.y);
    sJ.y = fma(-Xp.x, Vt.y, sJ.y); sJ.y = fma(-Xp.y, Vt.x, sJ.y); sJ.y = fma(Xt.x, Vp.y, sJ.y); sJ.y = fma(Xt.y, Vp.x, sJ.y);
    aJ.x = fma(Ft.x, Wt.x, aJ.x); aJ.x = fma(-Ft.y, Wt.y, aJ.x); aJ.x = fma(-Fp.x, Wp.x, aJ.x); aJ.x = fma(Fp.y, Wp.y, aJ.x);
    aJ.x = fma(Xp.x, Wt.x, aJ.x); aJ.x = fma(Xp.y, Wt.y, aJ.x); aJ.x = fma(Xt.x, Wp.x, aJ.x); aJ.x = fma(Xt.y, Wp.y, aJ.x);
    aJ.y = fma(Ft.x, Wt.y, aJ.y); aJ.y = fma(Ft.y, Wt.x, aJ.y); aJ.y = fma(-Fp.x, Wp.y, aJ.y); aJ.y = fma(-Fp.y, Wp.x, aJ.y);
    aJ.y = fma(Xp.x, Wt.y, aJ.y); aJ.y = fma(-Xp.y, Wt.x, aJ.y); aJ.y = fma(Xt.x, Wp.y, aJ.y); aJ.y = fma(-Xt.y, Wp.x, aJ.y);
    if (MODE == 0) {
        sM.x = fma(Ft.x, Vp.x, sM.x); sM.x = fma(Ft.y, Vp.y, sM.x); sM.x = fma(-Fp.x, Vt.x, sM.x); sM.x = fma(-Fp.y, Vt.y, sM.x);
        sM.x = fma(-Xt.x, Vt.x, sM.x); sM.x = fma(Xt.y, Vt.y, sM.x); sM.x = fma(-Xp.x, Vp.x, sM.x); sM.x = fma(Xp.y, Vp.y, sM.x);
        sM.y = fma(Ft.x, Vp.y, sM.y); sM.y = fma(-Ft.y, Vp.x, sM.y); sM.y = fma(-Fp.x, Vt.y, sM.y); sM.y = fma(Fp.y, Vt.x, sM.y);
        sM.y = fma(-Xt.x, Vt.y, sM.y); sM.y = fma(-Xt.y, Vt.x, sM.y); sM.y = fma(-Xp.x, Vp.y, sM.y); sM.y = fma(-Xp.y, Vp.x, sM.y);
        aM.x = fma(Ft.x, Wp.x, aM.x); aM.x = fma(-Ft.y, Wp.y, aM.x); aM.x = fma(Fp.x, Wt.x, aM.x); aM.x = fma(-Fp.y, Wt.y, aM.x);
        aM.x = fma(-Xt.x, Wt.x, aM.x); aM.x = fma(-Xt.y, Wt.y, aM.x); aM.x = fma(Xp.x, Wp.x, aM.x); aM.x = fma(Xp.y, Wp.y, aM.x);
        aM.y = fma(Ft.x, Wp.y, aM.y); aM.y = fma(Ft.y, Wp.x, aM.y); aM.y = fma(Fp.x, Wt.y, aM.y); aM.y = fma(Fp.y, Wt.x, aM.y);
        aM.y = fma(-Xt.x, Wt.y, aM.y); aM.y = fma(Xt.y, Wt.x, aM.y); aM.y = fma(Xp.x, Wp.y, aM.y); aM.y = fma(-Xp.y, Wp.x, aM.y);
    }
}

// Aggregation terms of one RWG at a stored direction (u) and at its antipode (v):
//   u_theta -= xJ Ft + xM Fp,  u_phi += -xJ Fp + xM Ft,
//   v_theta += -conj(Ft) xJ + conj(Fp) xM,  v_phi += conj(Fp) xJ + conj(Ft) xM     (MODE 1: xM = 0)
template <typename T, int MODE>
__device__ __forceinline__ void agg_pair(cpx<T> Ft, cpx<T> Fp, cpx<T> xJ, cpx<T> xM, cpx<T>& ut, cpx<T>& up, cpx<T>& vt,
                                         cpx<T>& vp) {
    ut.x = fma(-xJ.x, Ft.x, ut.x); ut.x = fma(xJ.y, Ft.y, ut.x);
    ut.y = fma(-xJ.x, Ft.y, ut.y); ut.y = fma(-xJ.y, Ft.x, ut.y);
    up.x = fma(-xJ.x, Fp.x, up.x); up.x = fma(xJ.y, Fp.y, up.x);
    up.y = fma(-xJ.x, Fp.y, up.y); up.y = fma(-xJ.y, Fp.x, up.y);
    vt.x = fma(-Ft.x, xJ.x, vt.x); vt.x = fma(-Ft.y, xJ.y, vt.x);
    vt.y = fma(-Ft.x, xJ.y, vt.y); vt.y = fma(Ft.y, xJ.x, vt.y);
    vp.x = fma(Fp.x, xJ.x, vp.x); vp.x = fma(Fp.y, xJ.y, vp.x);
    vp.y = fma(Fp.x, xJ.y, vp.y); vp.y = fma(-Fp.y, xJ.x, vp.y);
    if (MODE == 0) {
        ut.x = fma(-xM.x, Fp.x, ut.x); ut.x = fma(xM.y, Fp.y, ut.x);
        ut.y = fma(-xM.x, Fp.y, ut.y); ut.y = fma(-xM.y, Fp.x, ut.y);
        up.x = fma(xM.x, Ft.x, up.x); up.x = fma(-xM.y, Ft.y, up.x);
        up.y = fma(xM.x, Ft.y, up.y); up.y = fma(xM.y, Ft.x, up.y);
        vt.x = fma(Fp.x, xM.x, vt.x); vt.x = fma(Fp.y, xM.y, vt.x);
        vt.y = fma(Fp.x, xM.y, vt.y); vt.y = fma(-Fp.y, xM.x, vt.y);
        vp.x = fma(Ft.x, xM.x, vp.x); vp.x = fma(Ft.y, xM.y, vp.x);
        vp.y = fma(Ft.x, xM.y, vp.y); vp.y = fma(-Ft.y, xM.x, vp.y);
    }
}

// 16-byte load of two adjacent complex floats (read-only path); two 16-byte loads for doubles.
__device__ __forceinline__ void load_pair(const cpx<float>* p, cpx<float>& A, cpx<float>& B) {
    const float4 v = __ldg(reinterpret_cast<const float4*>(p));
    A = {v.x, v.y};
    B = {v.z, v.w};
}
__device__ __forceinline__ void load_pair(const cpx<double>* p, cpx<double>& A, cpx<double>& B) {
    const double2 a = __ldg(reinterpret_cast<const double2*>(p));
    const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
    A = {a.x, a.y};
    B = {b.x, b.y};
}
// One complex value through the read-only path as a single vector load.
__device__ __forceinline__ cpx<float> ldg_cpx(const cpx<float>* p) {
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return {v.x, v.y};
}
__device__ __forceinline__ cpx<double> ldg_cpx(const cpx<double>* p) {
    const double2 v = __ldg(reinterpret_cast<const double2*>(p));
    return {v.x, v.y};
}
// Two adjacent complex values from 16-byte aligned shared memory (one vector load for floats).
__device__ __forceinline__ void lds_pair(const cpx<float>* p, cpx<float>& A, cpx<float>& B) {
    const float4 v = *reinterpret_cast<const float4*>(p);
    A = {v.x, v.y};
    B = {v.z, v.w};
}
__device__ __forceinline__ void lds_pair(const cpx<double>* p, cpx<double>& A, cpx<double>& B) {
    const double2 a = reinterpret_cast<const double2*>(p)[0];
    const double2 b = reinterpret_cast<const double2*>(p)[1];
    A = {a.x, a.y};
    B = {b.x, b.y};
}
template <typename T>
__device__ __forceinline__ cpx<T> warp_sum(cpx<T> v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
        v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
    }
    return v;
}

