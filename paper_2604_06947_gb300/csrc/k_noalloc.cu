// k_noalloc.cu -- exact invariants of a caller's int32 state without any
// device allocation (fqnm_invariants_noalloc).
//
// Some callers cannot let a library call cudaMalloc: processes that hand all
// free device memory to their own pool (a caching allocator such as
// PyTorch's keeps freed blocks, so an outside cudaMalloc can fail even though
// the pool has room), latency-critical loops (cudaFree waits for the whole
// device), and services that must not grow their device footprint after
// start-up.  This variant of the invariants reduction keeps its scratch -- the
// per-block partial sums and the three totals -- in one file-scope static
// device array, reserved on every GPU where the library's device code is
// loaded (under lazy module loading, at the first call there) until the
// process exits, and allocates nothing per call.
//
// Limits and sharing:
//   * at most NA_MAX_CELLS = 2^26 cells per call (4096 partial slots of
//     16384 cells each); larger n is rejected with FQNM_ERR_ARG before any
//     launch;
//   * every call on a device uses the same array, which keeps the contents of
//     the last call; each call overwrites every slot it reads (no slot
//     accumulates), so nothing has to be cleared first;
//   * calls whose work overlaps on the GPU (different streams, or different
//     host threads on one device) race on the array: serialise them;
//   * the first call on each device looks up the array's device address
//     (cudaGetSymbolAddress) with that device current; make that first call
//     before any stream capture on that device.
#include "fqnm_internal.h"

#include <mutex>

namespace fqnm {

namespace {

constexpr int NA_BLOCK = 256;
constexpr int NA_ITEMS = 64;                                  // cells per thread
constexpr long long NA_CELLS_PER_BLOCK = (long long)NA_BLOCK * NA_ITEMS;
constexpr int NA_MAX_BLOCKS = 4096;
constexpr long long NA_MAX_CELLS = NA_CELLS_PER_BLOCK * NA_MAX_BLOCKS;   // 2^26
constexpr int NA_TOTALS = 3 * NA_MAX_BLOCKS;                  // offset of the 3 totals
constexpr int NA_MAX_DEVICES = 64;

// [0, 3*NA_MAX_BLOCKS): partials as [variable][block]; then 3 totals.
static __device__ __align__(256) long long g_noalloc_scratch[3 * NA_MAX_BLOCKS + 32];

__device__ __forceinline__ long long na_warp_sum(long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

// Pass 1: block b sums mass, total variation and l1 distance over its chunk
// [b*16384, (b+1)*16384) and overwrites its three partial slots.
__global__ void __launch_bounds__(NA_BLOCK)
k_na_partials(const int32_t* __restrict__ q, const int32_t* __restrict__ other,
              long long n, int periodic, long long* __restrict__ scratch)
{
    __shared__ long long sh[3][NA_BLOCK / 32];
    const long long begin = (long long)blockIdx.x * NA_CELLS_PER_BLOCK;
    const long long end = begin + NA_CELLS_PER_BLOCK < n ? begin + NA_CELLS_PER_BLOCK : n;
    long long mass = 0, tv = 0, l1 = 0;
    for (long long i = begin + threadIdx.x; i < end; i += NA_BLOCK) {
        const long long v = q[i];
        mass += v;
        bool face = true;
        long long nb = v;
        if (i + 1 < n) nb = q[i + 1];
        else if (periodic && n > 1) nb = q[0];
        else face = false;
        if (face) tv += nb > v ? nb - v : v - nb;
        if (other) {
            const long long o = other[i];
            l1 += o > v ? o - v : v - o;
        }
    }
    mass = na_warp_sum(mass);
    tv = na_warp_sum(tv);
    l1 = na_warp_sum(l1);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][w] = mass; sh[1][w] = tv; sh[2][w] = l1; }
    __syncthreads();
    if (w == 0) {
        for (int k = 0; k < 3; ++k) {
            long long t = lane < NA_BLOCK / 32 ? sh[k][lane] : 0;
            t = na_warp_sum(t);
            if (lane == 0) scratch[k * NA_MAX_BLOCKS + blockIdx.x] = t;
        }
    }
}

// Pass 2: one block adds the first nblocks partials of each variable and
// overwrites the three totals.
__global__ void __launch_bounds__(NA_BLOCK)
k_na_total(long long* __restrict__ scratch, int nblocks)
{
    __shared__ long long sh[NA_BLOCK / 32];
    for (int k = 0; k < 3; ++k) {
        long long t = 0;
        for (int b = threadIdx.x; b < nblocks; b += NA_BLOCK) t += scratch[k * NA_MAX_BLOCKS + b];
        t = na_warp_sum(t);
        const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
        if (lane == 0) sh[w] = t;
        __syncthreads();
        if (w == 0) {
            long long s = lane < NA_BLOCK / 32 ? sh[lane] : 0;
            s = na_warp_sum(s);
            if (lane == 0) scratch[NA_TOTALS + k] = s;
        }
        __syncthreads();
    }
}

std::mutex g_na_mu;
long long* g_na_ptr[NA_MAX_DEVICES] = {};

// Device address of the scratch array on the current device, looked up once
// per device with that device current.
fqnm_status na_scratch(long long** out)
{
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_error(e, "cudaGetDevice");
    if (dev < 0 || dev >= NA_MAX_DEVICES)
        return set_error(FQNM_ERR_ARG, "device ordinal %d out of range", dev);
    std::lock_guard<std::mutex> g(g_na_mu);
    if (!g_na_ptr[dev]) {
        void* p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return cuda_error(e, "cudaGetSymbolAddress(g_noalloc_scratch)");
        g_na_ptr[dev] = (long long*)p;
    }
    *out = g_na_ptr[dev];
    return FQNM_OK;
}

}  // namespace

}  // namespace fqnm

using namespace fqnm;

extern "C" fqnm_status fqnm_invariants_noalloc(const int32_t* q, const int32_t* other,
                                               size_t n, int boundary, int64_t* out,
                                               void* stream)
{
    if (!q || !out) return set_error(FQNM_ERR_ARG, "null state or output pointer");
    if (n == 0) return set_error(FQNM_ERR_ARG, "n == 0");
    if ((long long)n > NA_MAX_CELLS || n > (size_t)NA_MAX_CELLS)
        return set_error(FQNM_ERR_ARG,
                         "n = %zu exceeds the %lld-cell limit of the allocation-free "
                         "invariants (use fqnm_invariants for larger states)",
                         n, NA_MAX_CELLS);
    if (boundary != FQNM_BC_PERIODIC && boundary != FQNM_BC_TRANSMISSIVE)
        return set_error(FQNM_ERR_ARG, "unknown boundary %d", boundary);
    long long* scratch = nullptr;
    fqnm_status st = na_scratch(&scratch);
    if (st != FQNM_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int nblocks = (int)(((long long)n + NA_CELLS_PER_BLOCK - 1) / NA_CELLS_PER_BLOCK);
    k_na_partials<<<nblocks, NA_BLOCK, 0, s>>>(q, other, (long long)n,
                                               boundary == FQNM_BC_PERIODIC, scratch);
    note_launches();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "k_na_partials");
    k_na_total<<<1, NA_BLOCK, 0, s>>>(scratch, nblocks);
    note_launches();
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_error(e, "k_na_total");
    e = cudaMemcpyAsync(out, scratch + NA_TOTALS, 3 * sizeof(long long),
                        cudaMemcpyDeviceToHost, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaMemcpyAsync totals");
    e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    return FQNM_OK;
}
