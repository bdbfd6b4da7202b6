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
#include "fp64_int.cuh"

#include <cmath>
#include "roe.cuh"

namespace fqnm {

namespace {

// The FP64 instructions for operands outside the integer paths, as calls:
// inlined, their code was scheduled into the common path and executed
// whether or not a lane needed it (2^20-cell Sod step: 5.7 s against 3.8 s
// for 20,000 steps), while a call runs only when taken.
__device__ __noinline__ double fp64_div(double a, double b) { return __ddiv_rn(a, b); }
__device__ __noinline__ double fp64_sqrt(double a) { return __dsqrt_rn(a); }
__device__ __noinline__ double fp64_mul(double a, double b) { return __dmul_rn(a, b); }

// The Roe flux's arithmetic with division and square root on the integer
// pipes (fp64_int.cuh; the FP64 instruction for operands outside that path).
struct ArIntDivSqrt : Ar<double> {
    // The kernel's lanes run these in step (no lane-dependent branch around
    // the flux), so the FP64 call is a warp-uniform branch taken only when
    // some lane's operands fall outside the integer path.
    static __device__ __forceinline__ double div(double a, double b)
    {
        bool ok;
        double r = f64i::div_rn(a, b, ok);
        if (__any_sync(0xffffffffu, !ok)) {
            if (!ok) r = fp64_div(a, b);
        }
        return r;
    }
    static __device__ __forceinline__ double sqrt_(double a)
    {
        bool ok;
        double r = f64i::sqrt_rn(a, ok);
        if (__any_sync(0xffffffffu, !ok)) {
            if (!ok) r = fp64_sqrt(a);
        }
        return r;
    }
    // |a|: clear the sign bit (an integer operation; no FP64 instruction)
    static __device__ __forceinline__ double abs_(double a)
    {
        return __longlong_as_double(__double_as_longlong(a) & 0x7fffffffffffffffll);
    }
    static __device__ __forceinline__ double half_(double a)
    {
        bool ok;
        double r = f64i::scale2_rn(a, -1, ok);
        if (__any_sync(0xffffffffu, !ok)) {
            if (!ok) r = fp64_mul(0.5, a);
        }
        return r;
    }
    static __device__ __forceinline__ double twice(double a)
    {
        bool ok;
        double r = f64i::scale2_rn(a, 1, ok);
        if (__any_sync(0xffffffffu, !ok)) {
            if (!ok) r = fp64_mul(2.0, a);
        }
        return r;
    }
};

// ... and the products the flux marks as movable (mul2) on the integer pipes.
struct ArIntMul : ArIntDivSqrt {
    static __device__ __forceinline__ double mul2(double a, double b)
    {
        bool ok;
        double r = f64i::mul_rn(a, b, ok);
        if (__any_sync(0xffffffffu, !ok)) {
            if (!ok) r = fp64_mul(a, b);
        }
        return r;
    }
};

struct EulerParams {
    double g, lambda;
    double delta[3], inv_delta[3];
    int edelta[3];              // delta_k = 2^edelta[k]
    int rounding;
    int mask;                   // components evolved as integers (1 rho, 2 m, 4 E)
    int int_conv;               // conversions and rounding on the integer pipes
};

__device__ __forceinline__ double round_mode(double v, int mode)
{
    if (mode == FQNM_ROUND_HALF_AWAY) return round(v);
    if (mode == FQNM_ROUND_FLOOR) return floor(v);
    return rint(v);
}

// A component in the mask holds an integer state (value delta*q); one outside
// it holds the bits of its double value.  delta*q is formed on the integer
// pipes (the same double as the FP64 conversion and scaling: delta is a
// power of two) unless delta's exponent is out of that path's range.
__device__ __forceinline__ double comp_value(const int64_t* __restrict__ q, long long n,
                                             long long i, int k, const EulerParams& P)
{
    const long long v = q[k * n + i];
    if (!((P.mask >> k) & 1)) return __longlong_as_double(v);
    return P.int_conv ? f64i::i64_scaled_to_f64(v, P.edelta[k])
                      : __dmul_rn(P.delta[k], (double)v);
}

template <class A>
__device__ __forceinline__ RoeCell<double> load_cell(const int64_t* __restrict__ q, long long n,
                                                    long long i, const EulerParams& P)
{
    return roe_cell<double, A>(P.g, comp_value(q, n, i, 0, P), comp_value(q, n, i, 1, P),
                               comp_value(q, n, i, 2, P));
}

// The Roe flux of one face and, for the integer components, its quantised
// transfer round(F lambda / delta).
template <class A>
__device__ __forceinline__ void transfer(const RoeCell<double>& L, const RoeCell<double>& R,
                                         const EulerParams& P, long long* Phi, double* F,
                                         unsigned* err)
{
    roe_flux_cells<double, A>(P.g, L, R, F);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if (!((P.mask >> k) & 1)) { Phi[k] = 0; continue; }
        if (P.int_conv) {        // R(F lambda 2^-e): the scaling and rounding as integers
            bool bad = false;
            Phi[k] = f64i::f64_scaled_round_to_i64(__dmul_rn(F[k], P.lambda), -P.edelta[k],
                                                   P.rounding, bad);
            if (bad) atomicOr(err, ERRBIT_OVERFLOW);  // also NaN (negative pressure)
            continue;
        }
        double r = round_mode(__dmul_rn(__dmul_rn(F[k], P.lambda), P.inv_delta[k]), P.rounding);
        if (!(fabs(r) < 4.0e18)) {                 // also NaN (negative pressure)
            atomicOr(err, ERRBIT_OVERFLOW);
            r = 0.0;
        }
        Phi[k] = (long long)r;
    }
}

// Cells per warp: a warp loads 32 consecutive cells, the 30 it owns and one
// neighbour on each side, so that every lane runs the same instructions
// (a lane that computed an extra face alone would hold the FP64 pipe for a
// whole warp-instruction per operation).
constexpr int EULER_OWN = 30;

// Lane l holds cell c0 - 1 + l (clamped to [0, n-1]: the clamp is the
// transmissive ghost copy) and forms its quantities once; it evaluates the
// face to its right with its right neighbour's quantities by shuffle, and
// lanes 1..30 update their cells with the faces of lanes l-1 and l.
template <class A>
__global__ void k_euler_step(const int64_t* __restrict__ qin,
                             int64_t* __restrict__ qout, long long n,
                             EulerParams P, unsigned* err, long long* bflux)
{
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long c = warp * EULER_OWN - 1 + lane;
    const long long j = c < 0 ? 0 : (c >= n ? n - 1 : c);
    const RoeCell<double> me = load_cell<A>(qin, n, j, P);
    const RoeCell<double> right = roe_shfl<double>(me, 1, true);   // lane 31: unused face
    long long Fr[3], Fl[3];
    double Dr[3], Dl[3];
    transfer<A>(me, right, P, Fr, Dr, err);
    // each component's left face: the integer transfer, or for a component
    // kept in double its flux (a uniform branch on the mask)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if ((P.mask >> k) & 1) {
            Fl[k] = __shfl_up_sync(0xffffffffu, Fr[k], 1);
            Dl[k] = 0.0;
        } else {
            Fl[k] = 0;
            Dl[k] = __shfl_up_sync(0xffffffffu, Dr[k], 1);
        }
    }
    if (lane < 1 || lane > EULER_OWN || c >= n || !FQNM_IN_RANGE(c, n, err)) return;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        if ((P.mask >> k) & 1) {
            qout[k * n + c] = qin[k * n + c] - (Fr[k] - Fl[k]);
        } else {                                       // floating-point update
            const double u = __longlong_as_double(qin[k * n + c]);
            qout[k * n + c] = __double_as_longlong(
                __dsub_rn(u, __dmul_rn(P.lambda, __dsub_rn(Dr[k], Dl[k]))));
        }
    }
    if (c == 0)
        for (int k = 0; k < 3; ++k)
            if ((P.mask >> k) & 1)
                atomicAdd((unsigned long long*)(bflux + k), (unsigned long long)(-Fl[k]));
    if (c == n - 1)
        for (int k = 0; k < 3; ++k)
            if ((P.mask >> k) & 1)
                atomicAdd((unsigned long long*)(bflux + k), (unsigned long long)Fr[k]);
}

}  // namespace

cudaError_t launch_euler_step(const int64_t* qin, int64_t* qout, int64_t n,
                              double gamma, const double* delta, double lambda,
                              int rounding, int mask, int fp64_mode, unsigned* err,
                              long long* bflux, cudaStream_t st)
{
    EulerParams P;
    P.mask = mask;
    P.g = gamma;
    P.lambda = lambda;
    P.int_conv = fp64_mode >= 1;
    for (int k = 0; k < 3; ++k) {
        P.delta[k] = delta[k];
        P.inv_delta[k] = 1.0 / delta[k];
        P.edelta[k] = ilogb(delta[k]);
        if (std::ldexp(1.0, P.edelta[k]) != delta[k] || P.edelta[k] < -1022 ||
            P.edelta[k] > 960)
            P.int_conv = 0;          // not a power of two in the integer path's range
    }
    P.rounding = rounding;
    // one warp per block: the warps (segments of 30 cells) then spread over
    // the SMs one at a time, so a grid smaller than the GPU loads every SM
    // within one warp of the others (2^16 cells: 14 or 15 warps per SM,
    // against 12 or 16 with 4-warp blocks)
    const int block = 32;
    const long long warps = (n + EULER_OWN - 1) / EULER_OWN;
    const long long grid = (warps * 32 + block - 1) / block;
    if (fp64_mode >= 3)
        k_euler_step<ArIntMul><<<(unsigned)grid, block, 0, st>>>(qin, qout, n, P, err, bflux);
    else if (fp64_mode == 2)
        k_euler_step<ArIntDivSqrt><<<(unsigned)grid, block, 0, st>>>(qin, qout, n, P, err, bflux);
    else
        k_euler_step<Ar<double>><<<(unsigned)grid, block, 0, st>>>(qin, qout, n, P, err, bflux);
    note_launches();
    return cudaGetLastError();
}

}  // namespace fqnm
