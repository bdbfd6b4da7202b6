// roe.cuh -- Roe flux of the 1-D Euler equations on the GPU (§3.3).
//
// Textbook Roe flux, no entropy fix, gamma-law gas, conserved U = (rho, m, E):
//   iK = 1/rhoK, uK = mK*iK, pK = (g-1)*(EK - 0.5*(rhoK*(uK*uK))), HK = (EK+pK)*iK
//   sL = sqrt(rhoL), sR = sqrt(rhoR), w = sL + sR, iw = 1/w
//   (per cell, once: s, s*u, s*H and the physical flux components below)
//   ut = (sL*uL + sR*uR)*iw, Ht = (sL*HL + sR*HR)*iw
//   ct = sqrt((g-1)*(Ht - 0.5*(ut*ut)))
//   jumps d0, d1, d2 of rho, m, E; wave strengths
//   a2 = (g-1)/(ct*ct) * ((d0*(Ht - ut*ut) + ut*d1) - d2)
//   a1 = ((d0*(ut+ct) - d1) - ct*a2) / (2*ct),   a3 = d0 - (a1 + a2)
//   speeds |ut-ct|, |ut|, |ut+ct|; eigenvectors
//   r1 = (1, ut-ct, Ht-ut*ct), r2 = (1, ut, 0.5*(ut*ut)), r3 = (1, ut+ct, Ht+ut*ct)
//   F_k = 0.5*(fL_k + fR_k) - 0.5*((l1*a1*r1_k + l2*a2*r2_k) + l3*a3*r3_k)
// Every operation is an explicitly rounded IEEE operation (no contraction),
// in this order, so the double version is reproducible bit for bit.
#pragma once

#include <cuda_runtime.h>

namespace fqnm {

template <typename T> struct Ar;

// half_(x) = 0.5*x and twice(x) = 2*x are exact scalings by a power of two
// (a policy may form them on the exponent field instead).
template <> struct Ar<double> {
    static __device__ __forceinline__ double half_(double a) { return __dmul_rn(0.5, a); }
    static __device__ __forceinline__ double twice(double a) { return __dmul_rn(2.0, a); }
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    // mul2: a product that a policy may move off the FP64 unit (same result)
    static __device__ __forceinline__ double mul2(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double abs_(double a) { return fabs(a); }
};

template <> struct Ar<float> {
    static __device__ __forceinline__ float half_(float a) { return __fmul_rn(0.5f, a); }
    static __device__ __forceinline__ float twice(float a) { return __fmul_rn(2.0f, a); }
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float mul2(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
    static __device__ __forceinline__ float abs_(float a) { return fabsf(a); }
};

// The quantities of one cell that both of its faces use: the conserved
// state, s = sqrt(rho), the products s*u and s*H of the Roe averages, and
// the physical flux's momentum and energy components f1 = m*u + p and
// f2 = u*(E + p) (the same operations as in the flux, formed once per cell).
template <typename T>
struct RoeCell {
    T rho, m, E, s, su, sH, f1, f2;
};

// A: the arithmetic (Ar<T>, or a policy with the same members that forms
// some operations another way but with the same IEEE results).
template <typename T, class A = Ar<T>>
__device__ __forceinline__ RoeCell<T> roe_cell(T g, T rho, T m, T E)
{
    const T gm1 = A::sub(g, T(1));
    RoeCell<T> c;
    c.rho = rho;
    c.m = m;
    c.E = E;
    const T inv = A::div(T(1), rho);
    const T u = A::mul(m, inv);
    const T p = A::mul(gm1, A::sub(E, A::half_(A::mul(rho, A::mul(u, u)))));
    const T Ep = A::add(E, p);
    const T H = A::mul(Ep, inv);
    c.s = A::sqrt_(rho);
    c.su = A::mul(c.s, u);
    c.sH = A::mul(c.s, H);
    c.f1 = A::add(A::mul(m, u), p);
    c.f2 = A::mul(u, Ep);
    return c;
}

// A cell's quantities from the lane `delta` above (down = true) or below.
template <typename T>
__device__ __forceinline__ RoeCell<T> roe_shfl(const RoeCell<T>& c, int delta, bool down)
{
    RoeCell<T> r;
#define FQNM_SH(f) r.f = down ? __shfl_down_sync(0xffffffffu, c.f, delta) \
                              : __shfl_up_sync(0xffffffffu, c.f, delta)
    FQNM_SH(rho); FQNM_SH(m); FQNM_SH(E); FQNM_SH(s); FQNM_SH(su); FQNM_SH(sH);
    FQNM_SH(f1); FQNM_SH(f2);
#undef FQNM_SH
    return r;
}

// The Roe flux between two cells whose quantities are already formed (the
// same operations, in the same order, as roe_flux below).
template <typename T, class A = Ar<T>>
__device__ __forceinline__ void roe_flux_cells(T g, const RoeCell<T>& L, const RoeCell<T>& R, T* F)
{
    const T one = T(1), gm1 = A::sub(g, one);
    const T w = A::add(L.s, R.s), iw = A::div(one, w);
    const T ut = A::mul(A::add(L.su, R.su), iw);
    const T Ht = A::mul(A::add(L.sH, R.sH), iw);
    const T uu = A::mul(ut, ut);
    const T huu = A::half_(uu);
    const T ct = A::sqrt_(A::mul(gm1, A::sub(Ht, huu)));
    const T d0 = A::sub(R.rho, L.rho), d1 = A::sub(R.m, L.m), d2 = A::sub(R.E, L.E);
    const T a2 = A::mul(A::div(gm1, A::mul(ct, ct)),
                        A::sub(A::add(A::mul(d0, A::sub(Ht, uu)), A::mul(ut, d1)), d2));
    const T a1 = A::div(A::sub(A::sub(A::mul(d0, A::add(ut, ct)), d1), A::mul(ct, a2)),
                        A::twice(ct));
    const T a3 = A::sub(d0, A::add(a1, a2));
    const T l1 = A::abs_(A::sub(ut, ct)), l2 = A::abs_(ut), l3 = A::abs_(A::add(ut, ct));
    const T uct = A::mul(ut, ct);
    const T r1[3] = {one, A::sub(ut, ct), A::sub(Ht, uct)};
    const T r2[3] = {one, ut, huu};
    const T r3[3] = {one, A::add(ut, ct), A::add(Ht, uct)};
    const T fL[3] = {L.m, L.f1, L.f2};
    const T fR[3] = {R.m, R.f1, R.f2};
    const T la1 = A::mul(l1, a1), la2 = A::mul(l2, a2), la3 = A::mul(l3, a3);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        // the eigenvectors' first components are 1: x*1 = x exactly
        const T diss = k == 0 ? A::add(A::add(la1, la2), la3)
                              : A::add(A::add(A::mul2(la1, r1[k]), A::mul2(la2, r2[k])),
                                       A::mul2(la3, r3[k]));
        F[k] = A::sub(A::half_(A::add(fL[k], fR[k])), A::half_(diss));
    }
}

template <typename T>
__device__ __forceinline__ void roe_flux(T g, const T* UL, const T* UR, T* F)
{
    roe_flux_cells<T>(g, roe_cell<T>(g, UL[0], UL[1], UL[2]), roe_cell<T>(g, UR[0], UR[1], UR[2]), F);
}

}  // namespace fqnm
