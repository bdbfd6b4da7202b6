// k_rule.cu -- building and checking the integer transfer rule on the GPU.
//
// eq. flux_table:  phi+-(q) = round( f+-(delta q) * dt/dx * delta^-1 ).
// The maps are tabulated once per problem over the visited state range (the
// only place where rounding enters, Table 1 "Rounding exposure") in double
// precision, one operation at a time with explicit round-to-nearest
// intrinsics so that no multiply-add is contracted:
//     u = delta*q (exact, delta = 2^k)
//     t = f+-(u)  (order below)
//     s = t*lambda, lambda = dt/dx
//     v = s*(1/delta) (exact)
//     phi = round(v)  (half-even default; half-away; floor)
// Split fluxes (eq. flux_splitting):
//     LINEAR_UPWIND  f+ = max(a,0)*u,   f- = min(a,0)*u
//     LINEAR_LF      f+- = 0.5*(a*u +- alpha*u)
//     BURGERS_LF     f+- = 0.5*(0.5*(u*u) +- alpha*u)
//     BURGERS_EO     f+ = 0.5*(w*w), w = max(u,0);  f- likewise with min(u,0)
#include "closed_form.cuh"

#include <climits>

namespace fqnm {

namespace {

__device__ __forceinline__ double split_flux(int kind, double a, double alpha,
                                             int sign, double u)
{
    switch (kind) {
    case FQNM_FLUX_LINEAR_UPWIND: {
        double c = sign > 0 ? (a > 0.0 ? a : 0.0) : (a < 0.0 ? a : 0.0);
        return __dmul_rn(c, u);
    }
    case FQNM_FLUX_LINEAR_LF:
    case FQNM_FLUX_BURGERS_LF: {
        double f = (kind == FQNM_FLUX_LINEAR_LF) ? __dmul_rn(a, u)
                                                 : __dmul_rn(0.5, __dmul_rn(u, u));
        double d = __dmul_rn(alpha, u);
        return __dmul_rn(0.5, sign > 0 ? __dadd_rn(f, d) : __dsub_rn(f, d));
    }
    case FQNM_FLUX_BURGERS_EO: {
        double w = sign > 0 ? (u > 0.0 ? u : 0.0) : (u < 0.0 ? u : 0.0);
        return __dmul_rn(0.5, __dmul_rn(w, w));
    }
    default:
        return 0.0;
    }
}

__device__ __forceinline__ double round_mode(double v, int mode)
{
    if (mode == FQNM_ROUND_HALF_AWAY) return round(v);
    if (mode == FQNM_ROUND_FLOOR) return floor(v);
    return rint(v);
}

__global__ void k_build_split_table(int kind, double a, double alpha,
                                    double delta, double lambda, int rounding,
                                    long long lo, long long count, int2* tab2,
                                    int32_t* tabp, unsigned* err)
{
    const double inv_delta = 1.0 / delta;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const double u = __dmul_rn(delta, (double)(lo + k));
        int out[2];
        for (int side = 0; side < 2; ++side) {
            const int sign = side == 0 ? +1 : -1;
            double t = split_flux(kind, a, alpha, sign, u);
            double v = __dmul_rn(__dmul_rn(t, lambda), inv_delta);
            double r = round_mode(v, rounding);
            if (!(fabs(r) <= 2147483647.0)) {     // also catches NaN
                atomicOr(err, ERRBIT_OVERFLOW);
                r = 0.0;
            }
            out[side] = (int)r;
        }
        tab2[k] = make_int2(out[0], out[1]);
        tabp[k] = out[0];
    }
}

__global__ void k_pack_tab16(const int2* tab2, long long count, int32_t* tab16)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const int2 v = tab2[k];
        tab16[k] = (int32_t)(((unsigned)v.x & 0xffffu) | ((unsigned)v.y << 16));
    }
}

__global__ void k_copy_user_table(const int32_t* p, const int32_t* m,
                                  long long count, int2* tab2, int32_t* tabp)
{
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        tab2[k] = make_int2(p[k], m[k]);
        tabp[k] = p[k];
    }
}



template <int BLOCK>
__device__ __forceinline__ unsigned long long block_sum_u64(unsigned long long v)
{
    __shared__ unsigned long long sh[BLOCK / 32];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (threadIdx.x < 32) {
        t = threadIdx.x < BLOCK / 32 ? sh[threadIdx.x] : 0ull;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    }
    __syncthreads();
    return t;
}

constexpr int CHECK_BLOCK = 256;

// Closed-form mismatches, the monotonicity certificate and max|phi|.
__global__ void __launch_bounds__(CHECK_BLOCK)
k_rule_check(const int2* tab2, long long lo, long long count, ClosedForm cf,
             int use_cf, unsigned long long* out)
{
    unsigned long long mism = 0, flags = 0, maxp = 0, maxm = 0;
    for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < count;
         k += (long long)gridDim.x * blockDim.x) {
        const int2 v = tab2[k];
        const long long q = lo + k;
        if (use_cf) {
            if (cf_eval(int(q), cf) != v.x || v.y != 0) ++mism;
        }
        if (v.x != 0) flags |= CERT_P_NONZERO;
        if (v.y != 0) flags |= CERT_M_NONZERO;
        unsigned long long ap = (unsigned long long)(v.x < 0 ? -(long long)v.x : v.x);
        unsigned long long am = (unsigned long long)(v.y < 0 ? -(long long)v.y : v.y);
        maxp = ap > maxp ? ap : maxp;
        maxm = am > maxm ? am : maxm;
        if (k + 1 < count) {
            const int2 w = tab2[k + 1];
            if (w.x < v.x) flags |= CERT_P_NOT_MONOTONE;
            if (w.y > v.y) flags |= CERT_M_NOT_MONOTONE;
            // H(q) = q - phi+(q) + phi-(q) must not decrease
            long long h0 = q - v.x + v.y, h1 = (q + 1) - w.x + w.y;
            if (h1 < h0) flags |= CERT_H_NOT_MONOTONE;
        }
    }
    // one atomic per block and result: reduce over the warp, then the block
    unsigned long long s = block_sum_u64<CHECK_BLOCK>(mism);
    __shared__ unsigned shf[CHECK_BLOCK / 32], shp[CHECK_BLOCK / 32], shm[CHECK_BLOCK / 32];
    const unsigned f = __reduce_or_sync(0xffffffffu, (unsigned)flags);
    const unsigned mp = __reduce_max_sync(0xffffffffu, (unsigned)maxp);
    const unsigned mm = __reduce_max_sync(0xffffffffu, (unsigned)maxm);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { shf[w] = f; shp[w] = mp; shm[w] = mm; }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned bf = 0, bp = 0, bm = 0;
        for (int i = 0; i < CHECK_BLOCK / 32; ++i) {
            bf |= shf[i];
            bp = bp > shp[i] ? bp : shp[i];
            bm = bm > shm[i] ? bm : shm[i];
        }
        if (s) atomicAdd(out + 0, s);
        if (bf) atomicOr(out + 1, (unsigned long long)bf);
        if (bp) atomicMax(out + 2, (unsigned long long)bp);
        if (bm) atomicMax(out + 3, (unsigned long long)bm);
    }
}

template <typename T>
__global__ void k_minmax(const T* q, long long n, long long* out)
{
    long long mn = LLONG_MAX, mx = LLONG_MIN;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        long long v = (long long)q[i];
        mn = v < mn ? v : mn;
        mx = v > mx ? v : mx;
    }
    for (int o = 16; o > 0; o >>= 1) {
        long long a = __shfl_down_sync(0xffffffffu, mn, o);
        long long b = __shfl_down_sync(0xffffffffu, mx, o);
        mn = a < mn ? a : mn;
        mx = b > mx ? b : mx;
    }
    if ((threadIdx.x & 31) == 0) {
        atomicMin(out + 0, mn);
        atomicMax(out + 1, mx);
    }
}

// eq. quantisation: q = round(u/delta), u*(1/delta) exact for delta = 2^k.
__global__ void k_quantise(const double* u, long long n, double inv_delta,
                           int rounding, int bits, void* qv, unsigned* err)
{
    const double lim = bits == 32 ? 2147483647.0 : 9.2e18;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        double r = round_mode(__dmul_rn(u[i], inv_delta), rounding);
        if (!(fabs(r) <= lim)) {
            atomicOr(err, ERRBIT_OVERFLOW);
            r = 0.0;
        }
        if (bits == 32) static_cast<int32_t*>(qv)[i] = (int32_t)r;
        else static_cast<int64_t*>(qv)[i] = (int64_t)r;
    }
}

}  // namespace

cudaError_t launch_build_split_table(int kind, double a, double alpha,
                                     double delta, double lambda, int rounding,
                                     int64_t lo, int64_t count, int2* tab2,
                                     int32_t* tabp, unsigned* err,
                                     cudaStream_t st)
{
    k_build_split_table<<<grid_for(count, 256), 256, 0, st>>>(
        kind, a, alpha, delta, lambda, rounding, lo, count, tab2, tabp, err);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_pack_tab16(const int2* tab2, int64_t count, int32_t* tab16,
                              cudaStream_t st)
{
    k_pack_tab16<<<grid_for(count, 256), 256, 0, st>>>(tab2, count, tab16);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_copy_user_table(const int32_t* p, const int32_t* m,
                                   int64_t count, int2* tab2, int32_t* tabp,
                                   cudaStream_t st)
{
    k_copy_user_table<<<grid_for(count, 256), 256, 0, st>>>(p, m, count, tab2, tabp);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_rule_check(const int2* tab2, int64_t lo, int64_t count,
                              const ClosedForm* cf, unsigned long long* out,
                              cudaStream_t st)
{
    ClosedForm c{};
    if (cf) c = *cf;
    k_rule_check<<<grid_for(count, CHECK_BLOCK), CHECK_BLOCK, 0, st>>>(
        tab2, lo, count, c, cf ? 1 : 0, out);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_minmax_i32(const int32_t* q, int64_t n, long long* out,
                              cudaStream_t st)
{
    k_minmax<int32_t><<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(q, n, out);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_minmax_i64(const int64_t* q, int64_t n, long long* out,
                              cudaStream_t st)
{
    k_minmax<int64_t><<<grid_for(n, 256, 152 * 8), 256, 0, st>>>(q, n, out);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_quantise(const double* u, int64_t n, double inv_delta,
                            int rounding, int bits, void* q, unsigned* err,
                            cudaStream_t st)
{
    k_quantise<<<grid_for(n, 256), 256, 0, st>>>(u, n, inv_delta, rounding, bits, q, err);
    note_launches();
    return cudaGetLastError();
}

void init_minmax(long long* host2)
{
    host2[0] = LLONG_MAX;
    host2[1] = LLONG_MIN;
}

}  // namespace fqnm
