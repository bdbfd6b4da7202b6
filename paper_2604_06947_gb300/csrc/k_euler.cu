// k_euler.cu -- integer Euler step with the Roe flux quantised per conserved
// component (§3.3; the two-point transfer of eq.
// transfer_operator_equivalence_definition applied to each of rho, m, E):
//     Phi^k_{i+1/2} = round( F^k_Roe(delta q_i, delta q_{i+1}) * dt/dx / delta_k )
//     q^k_i <- q^k_i - (Phi^k_{i+1/2} - Phi^k_{i-1/2})
// States are int64 [3][n]; ends are transmissive (ghost cell = edge cell).
// One thread per cell evaluates the face on its right; the face on its left
// comes from the neighbouring lane by a shuffle (lane 0 evaluates its own), so
// each face's double-precision Roe flux is evaluated once per warp.  The
// boundary transfers are accumulated exactly in int64 so that
// sum q^k(now) = sum q^k(load) - bflux^k.
#include "fqnm_internal.h"
#include "roe.cuh"

namespace fqnm {

namespace {

struct EulerParams {
    double g, lambda;
    double delta[3], inv_delta[3];
    int rounding;
};

__device__ __forceinline__ double round_mode(double v, int mode)
{
    if (mode == FQNM_ROUND_HALF_AWAY) return round(v);
    if (mode == FQNM_ROUND_FLOOR) return floor(v);
    return rint(v);
}

__device__ __forceinline__ void face_transfer(const int64_t* __restrict__ q,
                                              long long n, long long iL,
                                              long long iR, const EulerParams& P,
                                              long long* Phi, unsigned* err)
{
    double UL[3], UR[3], F[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        UL[k] = __dmul_rn(P.delta[k], (double)q[k * n + iL]);
        UR[k] = __dmul_rn(P.delta[k], (double)q[k * n + iR]);
    }
    roe_flux<double>(P.g, UL, UR, F);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        double r = round_mode(__dmul_rn(__dmul_rn(F[k], P.lambda), P.inv_delta[k]), P.rounding);
        if (!(fabs(r) < 4.0e18)) {                 // also NaN (negative pressure)
            atomicOr(err, ERRBIT_OVERFLOW);
            r = 0.0;
        }
        Phi[k] = (long long)r;
    }
}

__global__ void k_euler_step(const int64_t* __restrict__ qin,
                             int64_t* __restrict__ qout, long long n,
                             EulerParams P, unsigned* err, long long* bflux)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const long long c = i < n ? i : n - 1;           // tail lanes mirror the last cell
    long long Fr[3], Fl[3];
    face_transfer(qin, n, c, c + 1 < n ? c + 1 : n - 1, P, Fr, err);
#pragma unroll
    for (int k = 0; k < 3; ++k) Fl[k] = __shfl_up_sync(0xffffffffu, Fr[k], 1);
    if (lane == 0) face_transfer(qin, n, c > 0 ? c - 1 : 0, c, P, Fl, err);
    if (i < n) {
#pragma unroll
        for (int k = 0; k < 3; ++k) qout[k * n + i] = qin[k * n + i] - (Fr[k] - Fl[k]);
        if (i == 0)
            for (int k = 0; k < 3; ++k)
                atomicAdd((unsigned long long*)(bflux + k), (unsigned long long)(-Fl[k]));
        if (i == n - 1)
            for (int k = 0; k < 3; ++k)
                atomicAdd((unsigned long long*)(bflux + k), (unsigned long long)Fr[k]);
    }
}

}  // namespace

cudaError_t launch_euler_step(const int64_t* qin, int64_t* qout, int64_t n,
                              double gamma, const double* delta, double lambda,
                              int rounding, unsigned* err, long long* bflux,
                              cudaStream_t st)
{
    EulerParams P;
    P.g = gamma;
    P.lambda = lambda;
    for (int k = 0; k < 3; ++k) {
        P.delta[k] = delta[k];
        P.inv_delta[k] = 1.0 / delta[k];
    }
    P.rounding = rounding;
    const int block = 128;
    const long long grid = (n + block - 1) / block;
    k_euler_step<<<(unsigned)grid, block, 0, st>>>(qin, qout, n, P, err, bflux);
    note_launches();
    return cudaGetLastError();
}

}  // namespace fqnm
