// roe.cuh -- Roe flux of the 1-D Euler equations on the GPU (§3.3).
//
// Textbook Roe flux, no entropy fix, gamma-law gas, conserved U = (rho, m, E):
//   iK = 1/rhoK, uK = mK*iK, pK = (g-1)*(EK - 0.5*(rhoK*(uK*uK))), HK = (EK+pK)*iK
//   sL = sqrt(rhoL), sR = sqrt(rhoR), w = sL + sR, iw = 1/w
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

template <> struct Ar<double> {
    static __device__ __forceinline__ double add(double a, double b) { return __dadd_rn(a, b); }
    static __device__ __forceinline__ double sub(double a, double b) { return __dsub_rn(a, b); }
    static __device__ __forceinline__ double mul(double a, double b) { return __dmul_rn(a, b); }
    static __device__ __forceinline__ double div(double a, double b) { return __ddiv_rn(a, b); }
    static __device__ __forceinline__ double sqrt_(double a) { return __dsqrt_rn(a); }
    static __device__ __forceinline__ double abs_(double a) { return fabs(a); }
};

template <> struct Ar<float> {
    static __device__ __forceinline__ float add(float a, float b) { return __fadd_rn(a, b); }
    static __device__ __forceinline__ float sub(float a, float b) { return __fsub_rn(a, b); }
    static __device__ __forceinline__ float mul(float a, float b) { return __fmul_rn(a, b); }
    static __device__ __forceinline__ float div(float a, float b) { return __fdiv_rn(a, b); }
    static __device__ __forceinline__ float sqrt_(float a) { return __fsqrt_rn(a); }
    static __device__ __forceinline__ float abs_(float a) { return fabsf(a); }
};

// The quantities of one cell that both of its faces use.
template <typename T>
struct RoeCell {
    T rho, m, E, u, p, H, s;
};

// A: the arithmetic (Ar<T>, or a policy with the same members that forms
// some operations another way but with the same IEEE results).
template <typename T, class A = Ar<T>>
__device__ __forceinline__ RoeCell<T> roe_cell(T g, T rho, T m, T E)
{
    const T gm1 = A::sub(g, T(1)), half = T(0.5);
    RoeCell<T> c;
    c.rho = rho;
    c.m = m;
    c.E = E;
    const T inv = A::div(T(1), rho);
    c.u = A::mul(m, inv);
    c.p = A::mul(gm1, A::sub(E, A::mul(half, A::mul(rho, A::mul(c.u, c.u)))));
    c.H = A::mul(A::add(E, c.p), inv);
    c.s = A::sqrt_(rho);
    return c;
}

// The Roe flux between two cells whose quantities are already formed (the
// same operations, in the same order, as roe_flux below).
template <typename T, class A = Ar<T>>
__device__ __forceinline__ void roe_flux_cells(T g, const RoeCell<T>& L, const RoeCell<T>& R, T* F)
{
    const T one = T(1), half = T(0.5), gm1 = A::sub(g, one);
    const T rhoL = L.rho, mL = L.m, EL = L.E, uL = L.u, pL = L.p, HL = L.H, sL = L.s;
    const T rhoR = R.rho, mR = R.m, ER = R.E, uR = R.u, pR = R.p, HR = R.H, sR = R.s;
    const T w = A::add(sL, sR), iw = A::div(one, w);
    const T ut = A::mul(A::add(A::mul(sL, uL), A::mul(sR, uR)), iw);
    const T Ht = A::mul(A::add(A::mul(sL, HL), A::mul(sR, HR)), iw);
    const T uu = A::mul(ut, ut);
    const T ct = A::sqrt_(A::mul(gm1, A::sub(Ht, A::mul(half, uu))));
    const T d0 = A::sub(rhoR, rhoL), d1 = A::sub(mR, mL), d2 = A::sub(ER, EL);
    const T a2 = A::mul(A::div(gm1, A::mul(ct, ct)),
                        A::sub(A::add(A::mul(d0, A::sub(Ht, uu)), A::mul(ut, d1)), d2));
    const T a1 = A::div(A::sub(A::sub(A::mul(d0, A::add(ut, ct)), d1), A::mul(ct, a2)),
                        A::mul(T(2), ct));
    const T a3 = A::sub(d0, A::add(a1, a2));
    const T l1 = A::abs_(A::sub(ut, ct)), l2 = A::abs_(ut), l3 = A::abs_(A::add(ut, ct));
    const T uct = A::mul(ut, ct);
    const T r1[3] = {one, A::sub(ut, ct), A::sub(Ht, uct)};
    const T r2[3] = {one, ut, A::mul(half, uu)};
    const T r3[3] = {one, A::add(ut, ct), A::add(Ht, uct)};
    const T fL[3] = {mL, A::add(A::mul(mL, uL), pL), A::mul(uL, A::add(EL, pL))};
    const T fR[3] = {mR, A::add(A::mul(mR, uR), pR), A::mul(uR, A::add(ER, pR))};
    const T la1 = A::mul(l1, a1), la2 = A::mul(l2, a2), la3 = A::mul(l3, a3);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const T diss = A::add(A::add(A::mul(la1, r1[k]), A::mul(la2, r2[k])),
                              A::mul(la3, r3[k]));
        F[k] = A::sub(A::mul(half, A::add(fL[k], fR[k])), A::mul(half, diss));
    }
}

template <typename T>
__device__ __forceinline__ void roe_flux(T g, const T* UL, const T* UR, T* F)
{
    roe_flux_cells<T>(g, roe_cell<T>(g, UL[0], UL[1], UL[2]), roe_cell<T>(g, UR[0], UR[1], UR[2]), F);
}

}  // namespace fqnm
