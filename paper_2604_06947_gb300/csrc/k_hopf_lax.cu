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
// Work items are (R rows, one chunk of the candidates): a warp holds the R
// rows (x values) in registers, its lanes stride over the chunk, each
// candidate load serving R evaluations, and the warp reduces each row's
// (key, index) pairs into a partial minimum.  Persistent warps take the
// items grid-stride, about 16 per resident warp, so every SM stays busy to
// the end whatever the number of rows; a second kernel takes each row's
// minimum over the chunks (the smallest index among equal keys, as within a
// chunk).  FP64-bound: the 4 FP64 operations of an evaluation run on the
// FP64 pipe (2 per SM per cycle on this part); the comparison runs on the
// integer pipe, on keys that order as the doubles do (-0 folded onto +0,
// NaN never taken).
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

// (key, j) < (key', j'): the smaller key, then the smaller index
__device__ __forceinline__ bool hl_less(long long k, long long j, long long k2, long long j2)
{
    return k < k2 || (k == k2 && j < j2);
}

__global__ void __launch_bounds__(HL_THREADS)
k_hopf_lax_part(const double* __restrict__ x, long long nx, const double* __restrict__ y,
                const double* __restrict__ U, long long ny, double inv2t, long long chunks,
                long long L, long long* __restrict__ pkey, long long* __restrict__ pj)
{
    const int lane = threadIdx.x & 31;
    const long long warps = ((long long)gridDim.x * blockDim.x) >> 5;
    const long long groups = (nx + HL_ROWS - 1) / HL_ROWS;
    for (long long item = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
         item < groups * chunks; item += warps) {
        const long long g = item / chunks, c = item - g * chunks;
        const long long r0 = g * HL_ROWS, j0 = c * L, j1 = j0 + L < ny ? j0 + L : ny;
        double xr[HL_ROWS];
        long long best[HL_ROWS];                        // order keys
        long long bj[HL_ROWS];
#pragma unroll
        for (int r = 0; r < HL_ROWS; ++r) {
            xr[r] = x[r0 + r < nx ? r0 + r : r0];
            best[r] = KEY_INF;                          // +inf: never taken
            bj[r] = LLONG_MAX;
        }
        for (long long j = j0 + lane; j < j1; j += 32) {
            const double yj = y[j], Uj = U[j];
#pragma unroll
            for (int r = 0; r < HL_ROWS; ++r) {
                const double d = __dsub_rn(xr[r], yj);
                const long long o = order_key(__dadd_rn(Uj, __dmul_rn(__dmul_rn(d, d), inv2t)));
                if (o < best[r] && o >= KEY_NEG_INF) {  // first minimum of this lane
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
                if (hl_less(ob, oj, best[r], bj[r])) {
                    best[r] = ob;
                    bj[r] = oj;
                }
            }
        }
        if (lane == 0) {
#pragma unroll
            for (int r = 0; r < HL_ROWS; ++r) {
                if (r0 + r >= nx) break;
                pkey[c * nx + r0 + r] = best[r];
                pj[c * nx + r0 + r] = bj[r];
            }
        }
    }
}

__global__ void k_hopf_lax_finish(const double* __restrict__ x, long long nx,
                                  const double* __restrict__ y, double t, long long chunks,
                                  const long long* __restrict__ pkey,
                                  const long long* __restrict__ pj, double* __restrict__ u,
                                  long long* __restrict__ idx)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nx;
         i += (long long)gridDim.x * blockDim.x) {
        long long bk = KEY_INF, bj = LLONG_MAX;
        for (long long c = 0; c < chunks; ++c) {
            const long long k = pkey[c * nx + i], j = pj[c * nx + i];
            if (hl_less(k, j, bk, bj)) {
                bk = k;
                bj = j;
            }
        }
        if (bj == LLONG_MAX) {                          // no finite candidate
            u[i] = __longlong_as_double(0x7ff8000000000000LL);
            if (idx) idx[i] = -1;
            continue;
        }
        u[i] = __ddiv_rn(__dsub_rn(x[i], y[bj]), t);
        if (idx) idx[i] = bj;
    }
}

}  // namespace

cudaError_t launch_hopf_lax(const double* x, int64_t nx, const double* y, const double* U0y,
                            int64_t ny, double t, double* u, int64_t* idx, cudaStream_t st)
{
    if (nx < 1 || ny < 1) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_hopf_lax_part, HL_THREADS, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) per_sm = 1;
    // chunks: about 16 items per resident warp, at least 256 candidates each
    const long long resident = (long long)sms * per_sm * (HL_THREADS / 32);
    const long long groups = (nx + HL_ROWS - 1) / HL_ROWS;
    long long chunks = (16 * resident + groups - 1) / groups;
    const long long max_chunks = (ny + 255) / 256;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    const long long L = (ny + chunks - 1) / chunks;
    chunks = (ny + L - 1) / L;
    long long* part = nullptr;
    e = cudaMallocAsync((void**)&part, 2 * chunks * nx * sizeof(long long), st);
    if (e != cudaSuccess) return e;
    const long long items = groups * chunks;
    const long long want = (items * 32 + HL_THREADS - 1) / HL_THREADS;
    const long long grid = want < (long long)sms * per_sm ? want : (long long)sms * per_sm;
    const double inv2t = 1.0 / (2.0 * t);
    k_hopf_lax_part<<<(unsigned)grid, HL_THREADS, 0, st>>>(x, nx, y, U0y, ny, inv2t, chunks, L,
                                                           part, part + chunks * nx);
    note_launches();
    e = cudaGetLastError();
    if (e == cudaSuccess) {
        k_hopf_lax_finish<<<grid_for(nx, 256), 256, 0, st>>>(x, nx, y, t, chunks, part,
                                                             part + chunks * nx, u,
                                                             (long long*)idx);
        note_launches();
        e = cudaGetLastError();
    }
    const cudaError_t f = cudaFreeAsync(part, st);
    return e != cudaSuccess ? e : f;
}

}  // namespace fqnm
