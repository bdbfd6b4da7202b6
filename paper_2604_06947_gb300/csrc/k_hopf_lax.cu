// k_hopf_lax.cu -- the Hopf-Lax (Lax-Oleinik) entropy solution of inviscid
// Burgers on a candidate grid: the accuracy reference of the Burgers test
// (§3.2, the dense-grid entropy reference).
//
//   u(x, t) = (x - y*) / t,  y* = argmin_j  U0_j + ((x - y_j)^2) / (2 t)
//
// over candidates (y_j, U0_j = int_0^{y_j} u0), ties to the smallest j.  Each
// operation is rounded once in this order (d = x - y_j; d*d; * inv2t; + U0_j,
// inv2t = 1/(2t) formed once), so the result does not depend on how the
// candidates are split between lanes.
//
// A warp holds R rows (x values) in registers and its lanes stride over the
// candidates, each candidate load serving R evaluations; the warp then
// reduces each row's (value, index) pairs.  FP64-bound: the 4 FP64
// operations of an evaluation run on the FP64 pipe (2 per SM per cycle on
// this part); the comparison runs on the integer pipe, on keys that order
// as the doubles do (-0 folded onto +0, NaN never taken).
#include "fqnm_internal.h"
#include "hopf_lax.h"

#include <climits>

namespace fqnm {

namespace {

constexpr int HL_ROWS = 4;
constexpr int HL_THREADS = 256;
constexpr long long KEY_INF = 0x7ff0000000000000LL;     // key of +inf (its bits)
constexpr long long KEY_NEG_INF = (long long)0x8010000000000000ULL;   // key of -inf

// An int64 that orders as the double does: for non-NaN a, b,
// a < b <=> key(a) < key(b) and a == b <=> key(a) == key(b) (-0 and +0
// both map to 0).  Non-negative doubles keep their bits; negative ones map
// to (bits ^ 0x7fff...f) + 1.  A NaN maps above KEY_INF (positive sign) or
// below KEY_NEG_INF (negative sign), so `key < best && key >= KEY_NEG_INF`
// never takes a NaN.  All integer operations, off the FP64 pipe.
__device__ __forceinline__ long long order_key(double v)
{
    const long long b = __double_as_longlong(v);
    const long long m = b >> 63;                          // 0 or -1
    return (b ^ (m & 0x7fffffffffffffffLL)) - m;
}

__global__ void __launch_bounds__(HL_THREADS)
k_hopf_lax(const double* __restrict__ x, long long nx, const double* __restrict__ y,
           const double* __restrict__ U, long long ny, double t, double inv2t,
           double* __restrict__ u, long long* __restrict__ idx)
{
    const int lane = threadIdx.x & 31;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const long long r0 = warp * HL_ROWS;
    if (r0 >= nx) return;                               // the whole warp leaves
    double xr[HL_ROWS];
    long long best[HL_ROWS];                            // order keys
    long long bj[HL_ROWS];
#pragma unroll
    for (int r = 0; r < HL_ROWS; ++r) {
        xr[r] = x[r0 + r < nx ? r0 + r : r0];
        best[r] = KEY_INF;                              // +inf: never taken
        bj[r] = LLONG_MAX;
    }
    for (long long j = lane; j < ny; j += 32) {
        const double yj = y[j], Uj = U[j];
#pragma unroll
        for (int r = 0; r < HL_ROWS; ++r) {
            const double d = __dsub_rn(xr[r], yj);
            const long long o = order_key(__dadd_rn(Uj, __dmul_rn(__dmul_rn(d, d), inv2t)));
            if (o < best[r] && o >= KEY_NEG_INF) {      // first minimum of this lane
                best[r] = o;
                bj[r] = j;
            }
        }
    }
#pragma unroll
    for (int r = 0; r < HL_ROWS; ++r) {
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) {
            const long long ob = __shfl_down_sync(0xffffffffu, best[r], off);
            const long long oj = __shfl_down_sync(0xffffffffu, bj[r], off);
            if (ob < best[r] || (ob == best[r] && oj < bj[r])) {
                best[r] = ob;
                bj[r] = oj;
            }
        }
    }
    if (lane != 0) return;
#pragma unroll
    for (int r = 0; r < HL_ROWS; ++r) {
        if (r0 + r >= nx) break;
        const long long j = bj[r];
        if (j == LLONG_MAX) {                           // no finite candidate
            u[r0 + r] = __longlong_as_double(0x7ff8000000000000LL);
            if (idx) idx[r0 + r] = -1;
            continue;
        }
        u[r0 + r] = __ddiv_rn(__dsub_rn(xr[r], y[j]), t);
        if (idx) idx[r0 + r] = j;
    }
}

}  // namespace

cudaError_t launch_hopf_lax(const double* x, int64_t nx, const double* y, const double* U0y,
                            int64_t ny, double t, double* u, int64_t* idx, cudaStream_t st)
{
    const long long warps = (nx + HL_ROWS - 1) / HL_ROWS;
    const long long grid = (warps * 32 + HL_THREADS - 1) / HL_THREADS;
    const double inv2t = 1.0 / (2.0 * t);
    k_hopf_lax<<<(unsigned)grid, HL_THREADS, 0, st>>>(x, nx, y, U0y, ny, t, inv2t, u,
                                                     (long long*)idx);
    note_launches();
    return cudaGetLastError();
}

}  // namespace fqnm
