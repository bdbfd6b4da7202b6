// k_reduce.cu -- exact integer invariants and the reconstructed observable.
//
// Invariants (eq. exact_conservation; Lemma on CFL stability (ii), (iii)):
//     mass = sum_i q_i
//     TV   = sum_i |q_{i+1} - q_i|      (periodic: the wrap face included)
//     l1   = sum_i |q_i - other_i|
// Integer sums are exact and independent of the reduction order: each thread
// accumulates in int64, warps reduce by shuffles, blocks through shared
// memory, and one 64-bit atomic per block adds the block total.
//
// Observable (eq. reconstruction_operator): u_i = delta*q_i, exact in double
// for |q| < 2^53 and delta = 2^k; the float variant rounds once.
#include "fqnm_internal.h"

namespace fqnm {

namespace {

constexpr int RBLOCK = 256;

__device__ __forceinline__ long long warp_sum(long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <typename T>
__global__ void __launch_bounds__(RBLOCK)
k_invariants(const T* __restrict__ q, const T* __restrict__ other, long long n,
             int periodic, long long* acc)
{
    __shared__ long long sh[3][RBLOCK / 32];
    long long mass = 0, tv = 0, l1 = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const long long v = (long long)q[i];
        mass += v;
        long long nb;
        bool face = true;
        if (i + 1 < n) nb = (long long)q[i + 1];
        else if (periodic && n > 1) nb = (long long)q[0];
        else { nb = v; face = false; }
        if (face) tv += nb > v ? nb - v : v - nb;
        if (other) {
            const long long o = (long long)other[i];
            l1 += o > v ? o - v : v - o;
        }
    }
    mass = warp_sum(mass);
    tv = warp_sum(tv);
    l1 = warp_sum(l1);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][w] = mass; sh[1][w] = tv; sh[2][w] = l1; }
    __syncthreads();
    if (w == 0) {
        for (int k = 0; k < 3; ++k) {
            long long t = lane < RBLOCK / 32 ? sh[k][lane] : 0;
            t = warp_sum(t);
            if (lane == 0 && t != 0)
                atomicAdd((unsigned long long*)(acc + k), (unsigned long long)t);
        }
    }
}

template <typename T>
__global__ void k_observe(const T* __restrict__ q, long long n, double delta,
                          void* u, int fp32, int bits)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const double v = bits ? __longlong_as_double((long long)q[i])
                              : __dmul_rn(delta, (double)q[i]);
        if (fp32) static_cast<float*>(u)[i] = (float)v;
        else static_cast<double*>(u)[i] = v;
    }
}

}  // namespace

cudaError_t launch_invariants_i32(const int32_t* q, const int32_t* other,
                                  int64_t n, int periodic, long long* acc,
                                  cudaStream_t st)
{
    k_invariants<int32_t><<<grid_for(n, RBLOCK, 152 * 8), RBLOCK, 0, st>>>(q, other, n, periodic, acc);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_invariants_i64(const int64_t* q, const int64_t* other,
                                  int64_t n, int periodic, long long* acc,
                                  cudaStream_t st)
{
    k_invariants<int64_t><<<grid_for(n, RBLOCK, 152 * 8), RBLOCK, 0, st>>>(q, other, n, periodic, acc);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_observe_i32(const int32_t* q, int64_t n, double delta,
                               void* u, int fp32, cudaStream_t st)
{
    k_observe<int32_t><<<grid_for(n, 256), 256, 0, st>>>(q, n, delta, u, fp32, 0);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_observe_i64(const int64_t* q, int64_t n, double delta,
                               void* u, int fp32, cudaStream_t st, int bits)
{
    k_observe<int64_t><<<grid_for(n, 256), 256, 0, st>>>(q, n, delta, u, fp32, bits);
    note_launches();
    return cudaGetLastError();
}

}  // namespace fqnm
