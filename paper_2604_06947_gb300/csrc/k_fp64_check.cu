// k_fp64_check.cu -- the integer-pipe IEEE double steps of fp64_int.cuh
// evaluated elementwise next to the FP64 instructions they stand in for
// (fqnm_fp64_check), so that tests can compare the two bit for bit on
// arbitrary operands.
#include "fqnm_internal.h"
#include "fp64_int.cuh"

namespace fqnm {
namespace {

__device__ __forceinline__ double round_fp64(double v, int mode)
{
    if (mode == FQNM_ROUND_HALF_AWAY) return round(v);
    if (mode == FQNM_ROUND_FLOOR) return floor(v);
    return rint(v);
}

__global__ void k_fp64_check(int op, int mode, const double* __restrict__ a,
                             const double* __restrict__ b, long long n,
                             long long* __restrict__ out_int, long long* __restrict__ out_fp64,
                             int* __restrict__ out_path)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const double x = a[i], y = b[i];
    long long ri = 0, rf = 0;
    int path = 0;
    if (op == 0) {                         // x / y
        bool ok;
        const double r = f64i::div_rn(x, y, ok);
        ri = __double_as_longlong(ok ? r : __ddiv_rn(x, y));
        rf = __double_as_longlong(__ddiv_rn(x, y));
        path = ok;
    } else if (op == 1) {                  // sqrt(x)
        bool ok;
        const double r = f64i::sqrt_rn(x, ok);
        ri = __double_as_longlong(ok ? r : __dsqrt_rn(x));
        rf = __double_as_longlong(__dsqrt_rn(x));
        path = ok;
    } else if (op == 2) {                  // (double)q * 2^e, q = bits of x, e = (int)y
        const long long q = __double_as_longlong(x);
        const int e = (int)y;
        ri = __double_as_longlong(f64i::i64_scaled_to_f64(q, e));
        rf = __double_as_longlong(__dmul_rn((double)q, ldexp(1.0, e)));
        path = 1;
    } else if (op == 5) {                  // x * y
        bool ok;
        const double r = f64i::mul_rn(x, y, ok);
        ri = __double_as_longlong(ok ? r : __dmul_rn(x, y));
        rf = __double_as_longlong(__dmul_rn(x, y));
        path = ok;
    } else if (op == 4) {                  // x * 2^k, k = (int)y in {-1, 1}
        const int k = (int)y;
        bool ok;
        const double r = f64i::scale2_rn(x, k, ok);
        const double f = __dmul_rn(x, k < 0 ? 0.5 : 2.0);
        ri = __double_as_longlong(ok ? r : f);
        rf = __double_as_longlong(f);
        path = ok;
    } else {                               // op 3: R(x * 2^e) as int64, e = (int)y
        const int e = (int)y;
        bool bad = false;
        ri = f64i::f64_scaled_round_to_i64(x, e, mode, bad);
        const double r = round_fp64(__dmul_rn(x, ldexp(1.0, e)), mode);
        const bool bad_f = !(fabs(r) < 4.0e18);
        rf = bad_f ? 0 : (long long)r;
        path = (bad ? 2 : 0) | (bad_f ? 4 : 0) | 1;
    }
    out_int[i] = ri;
    out_fp64[i] = rf;
    out_path[i] = path;
}

}  // namespace
}  // namespace fqnm

using namespace fqnm;

extern "C" fqnm_status fqnm_fp64_check(int op, int rounding, const double* a, const double* b,
                                       size_t n, int64_t* out_int, int64_t* out_fp64,
                                       int32_t* out_path, void* stream)
{
    if (op < 0 || op > 5) return set_error(FQNM_ERR_ARG, "op must be 0..5");
    if (rounding < 0 || rounding > 2) return set_error(FQNM_ERR_ARG, "rounding must be 0..2");
    if (n == 0) return FQNM_OK;
    if (!a || !b || !out_int || !out_fp64 || !out_path)
        return set_error(FQNM_ERR_ARG, "null pointer");
    const int block = 256;
    const long long grid = ((long long)n + block - 1) / block;
    if (grid > 0x7fffffffLL) return set_error(FQNM_ERR_ARG, "n too large");
    k_fp64_check<<<(unsigned)grid, block, 0, (cudaStream_t)stream>>>(
        op, rounding, a, b, (long long)n, (long long*)out_int, (long long*)out_fp64, out_path);
    note_launches();
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? FQNM_OK : cuda_error(e, "k_fp64_check");
}
