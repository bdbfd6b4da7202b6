// k_fv.cu -- the floating-point finite-volume baseline with the same flux.
//
// eq. classical_operator_definition:
//     u_i <- u_i - lambda * (F_{i+1/2} - F_{i-1/2}),  F(uL,uR) = f+(uL) + f-(uR)
// in float or double, each operation explicitly rounded (no contraction) in
// the order
//     Fr = f+(u_i) + f-(u_{i+1}),  Fl = f+(u_{i-1}) + f-(u_i),
//     d = Fr - Fl,  u_i - lambda*d
// with the split fluxes of eq. flux_splitting written as in the rule builder.
// One step per launch, or (periodic scalar problems) K steps per launch in
// tiles with a K-cell halo, the execution strategy of the integer kernel:
// the same operations on the same values, so the two agree bit for bit.
// The Euler variant uses the Roe flux of roe.cuh on [3][n], transmissive ends.
#include "fqnm_internal.h"
#include "roe.cuh"

namespace fqnm {

namespace {

template <typename T>
struct FvParams {
    int kind;
    T a, alpha, lambda;
};

template <typename T, int KIND>
__device__ __forceinline__ T fsplit_k(const FvParams<T>& P, int sign, T u)
{
    using A = Ar<T>;
    if (KIND == FQNM_FLUX_LINEAR_UPWIND) {
        const T c = sign > 0 ? (P.a > T(0) ? P.a : T(0)) : (P.a < T(0) ? P.a : T(0));
        return A::mul(c, u);
    }
    if (KIND == FQNM_FLUX_LINEAR_LF || KIND == FQNM_FLUX_BURGERS_LF) {
        const T f = KIND == FQNM_FLUX_LINEAR_LF ? A::mul(P.a, u) : A::mul(T(0.5), A::mul(u, u));
        const T d = A::mul(P.alpha, u);
        return A::mul(T(0.5), sign > 0 ? A::add(f, d) : A::sub(f, d));
    }
    if (KIND == FQNM_FLUX_BURGERS_EO) {
        const T w = sign > 0 ? (u > T(0) ? u : T(0)) : (u < T(0) ? u : T(0));
        return A::mul(T(0.5), A::mul(w, w));
    }
    return T(0);
}

template <typename T>
__device__ __forceinline__ T fsplit(const FvParams<T>& P, int sign, T u)
{
    switch (P.kind) {
    case FQNM_FLUX_LINEAR_UPWIND: return fsplit_k<T, FQNM_FLUX_LINEAR_UPWIND>(P, sign, u);
    case FQNM_FLUX_LINEAR_LF: return fsplit_k<T, FQNM_FLUX_LINEAR_LF>(P, sign, u);
    case FQNM_FLUX_BURGERS_LF: return fsplit_k<T, FQNM_FLUX_BURGERS_LF>(P, sign, u);
    case FQNM_FLUX_BURGERS_EO: return fsplit_k<T, FQNM_FLUX_BURGERS_EO>(P, sign, u);
    default: return T(0);
    }
}

// K steps per launch on a periodic line: a block of FV_TB_BLOCK threads
// holds FV_TB_V consecutive cells per thread (a tile of FV_TB_TILE cells
// starting K cells before the S = FV_TB_TILE - 2K cells it writes), takes
// the neighbours' split fluxes by shuffle within a warp and through shared
// memory between warps (one barrier per step); the tile's two end cells use
// a ghost copy of themselves and lie outside the cells written.
constexpr int FV_TB_V = 8, FV_TB_BLOCK = 128, FV_TB_TILE = FV_TB_V * FV_TB_BLOCK;

template <typename T, int KIND>
__global__ void __launch_bounds__(FV_TB_BLOCK)
k_fv_tb(FvParams<T> P, const T* __restrict__ uin, T* __restrict__ uout, long long n, int K,
        long long S)
{
    using A = Ar<T>;
    constexpr int NW = FV_TB_BLOCK / 32;
    __shared__ T shp[2][NW], shm[2][NW];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long start = (long long)blockIdx.x * S - K;
    T u[FV_TB_V];
    // a thread's cells are consecutive: an aligned run inside [0, n) loads as
    // 16-byte vectors (as in the integer kernel), a wrapped one cell by cell
    constexpr int PER16 = 16 / (int)sizeof(T);
    const long long c0 = start + (long long)threadIdx.x * FV_TB_V;
    if (c0 >= 0 && c0 + FV_TB_V <= n && (reinterpret_cast<uintptr_t>(uin + c0) & 15) == 0) {
#pragma unroll
        for (int j = 0; j < FV_TB_V; j += PER16) {
            const uint4 v = __ldg(reinterpret_cast<const uint4*>(uin + c0 + j));
            const T* e = reinterpret_cast<const T*>(&v);
#pragma unroll
            for (int k = 0; k < PER16; ++k) u[j + k] = e[k];
        }
    } else {
#pragma unroll
        for (int j = 0; j < FV_TB_V; ++j) {
            long long g = (start + threadIdx.x * FV_TB_V + j) % n;
            if (g < 0) g += n;
            u[j] = uin[g];
        }
    }
    for (int s = 0; s < K; ++s) {
        T fp[FV_TB_V], fm[FV_TB_V];
#pragma unroll
        for (int j = 0; j < FV_TB_V; ++j) {
            fp[j] = fsplit_k<T, KIND>(P, +1, u[j]);
            fm[j] = fsplit_k<T, KIND>(P, -1, u[j]);
        }
        const int b = s & 1;
        if (lane == 31) shp[b][w] = fp[FV_TB_V - 1];
        if (lane == 0) shm[b][w] = fm[0];
        __syncthreads();
        T fpl = __shfl_up_sync(0xffffffffu, fp[FV_TB_V - 1], 1);
        T fmr = __shfl_down_sync(0xffffffffu, fm[0], 1);
        if (lane == 0) fpl = w > 0 ? shp[b][w - 1] : fp[0];
        if (lane == 31) fmr = w < NW - 1 ? shm[b][w + 1] : fm[FV_TB_V - 1];
        T Fl = A::add(fpl, fm[0]);
#pragma unroll
        for (int j = 0; j < FV_TB_V; ++j) {
            const T Fr = A::add(fp[j], j < FV_TB_V - 1 ? fm[j + 1] : fmr);
            u[j] = A::sub(u[j], A::mul(P.lambda, A::sub(Fr, Fl)));
            Fl = Fr;
        }
    }
#pragma unroll
    for (int j0 = 0; j0 < FV_TB_V; j0 += PER16) {
        const long long e = (long long)threadIdx.x * FV_TB_V + j0;
        const long long o = (long long)blockIdx.x * S + (e - K);
        if (e >= K && e + PER16 <= K + S && o + PER16 <= n &&
            (reinterpret_cast<uintptr_t>(uout + o) & 15) == 0) {
            uint4 v;
            T* w = reinterpret_cast<T*>(&v);
#pragma unroll
            for (int k = 0; k < PER16; ++k) w[k] = u[j0 + k];
            *reinterpret_cast<uint4*>(uout + o) = v;
            continue;
        }
#pragma unroll
        for (int j = j0; j < j0 + PER16; ++j) {
            const long long ej = (long long)threadIdx.x * FV_TB_V + j;
            const long long oj = (long long)blockIdx.x * S + (ej - K);
            if (ej >= K && ej < K + S && oj < n) uout[oj] = u[j];
        }
    }
}

template <typename T>
cudaError_t launch_fv_tb(const FvParams<T>& P, const T* uin, T* uout, long long n, int K,
                         cudaStream_t st)
{
    if (K < 1 || K > FV_TB_MAX_K || n < 1) return cudaErrorInvalidValue;
    const long long S = FV_TB_TILE - 2LL * K;
    const long long blocks = (n + S - 1) / S;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    switch (P.kind) {
    case FQNM_FLUX_LINEAR_UPWIND:
        k_fv_tb<T, FQNM_FLUX_LINEAR_UPWIND><<<(unsigned)blocks, FV_TB_BLOCK, 0, st>>>(P, uin, uout, n, K, S);
        break;
    case FQNM_FLUX_LINEAR_LF:
        k_fv_tb<T, FQNM_FLUX_LINEAR_LF><<<(unsigned)blocks, FV_TB_BLOCK, 0, st>>>(P, uin, uout, n, K, S);
        break;
    case FQNM_FLUX_BURGERS_LF:
        k_fv_tb<T, FQNM_FLUX_BURGERS_LF><<<(unsigned)blocks, FV_TB_BLOCK, 0, st>>>(P, uin, uout, n, K, S);
        break;
    case FQNM_FLUX_BURGERS_EO:
        k_fv_tb<T, FQNM_FLUX_BURGERS_EO><<<(unsigned)blocks, FV_TB_BLOCK, 0, st>>>(P, uin, uout, n, K, S);
        break;
    default:
        return cudaErrorInvalidValue;
    }
    note_launches();
    return cudaGetLastError();
}

template <typename T>
__global__ void k_fv_step(FvParams<T> P, const T* __restrict__ uin,
                          T* __restrict__ uout, long long n, int periodic)
{
    using A = Ar<T>;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        long long il = i - 1, ir = i + 1;
        if (periodic) {
            if (il < 0) il = n - 1;
            if (ir >= n) ir = 0;
        } else {
            if (il < 0) il = 0;
            if (ir >= n) ir = n - 1;
        }
        const T ul = uin[il], uc = uin[i], ur = uin[ir];
        const T Fr = A::add(fsplit(P, +1, uc), fsplit(P, -1, ur));
        const T Fl = A::add(fsplit(P, +1, ul), fsplit(P, -1, uc));
        uout[i] = A::sub(uc, A::mul(P.lambda, A::sub(Fr, Fl)));
    }
}

template <typename T>
__device__ __forceinline__ RoeCell<T> fv_cell(const T* __restrict__ u, long long n, long long i, T g)
{
    return roe_cell<T>(g, u[i], u[n + i], u[2 * n + i]);
}

// Cell quantities formed once per cell and shared with the neighbouring
// lanes, with the same warp layout as the integer Euler kernel: a warp loads
// 32 cells (its 30 and one on each side, clamped: the transmissive ghost),
// every lane evaluates the face to its right, lanes 1..30 update.
constexpr int EULER_FV_OWN = 30;

template <typename T>
__global__ void k_euler_fv(T g, T lambda, const T* __restrict__ uin,
                           T* __restrict__ uout, long long n)
{
    using A = Ar<T>;
    const long long warp = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    const long long c = warp * EULER_FV_OWN - 1 + lane;
    const long long j = c < 0 ? 0 : (c >= n ? n - 1 : c);
    const RoeCell<T> me = fv_cell<T>(uin, n, j, g);
    const RoeCell<T> right = roe_shfl<T>(me, 1, true);
    T Fr[3], Fl[3];
    roe_flux_cells<T>(g, me, right, Fr);
#pragma unroll
    for (int k = 0; k < 3; ++k) Fl[k] = __shfl_up_sync(0xffffffffu, Fr[k], 1);
    if (lane < 1 || lane > EULER_FV_OWN || c >= n) return;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        uout[k * n + c] = A::sub(uin[k * n + c], A::mul(lambda, A::sub(Fr[k], Fl[k])));
}

// one warp per block (as the integer Euler kernel): a grid smaller than the
// GPU then loads every SM within one warp of the others
static unsigned euler_fv_grid(long long n)
{
    return (unsigned)((n + EULER_FV_OWN - 1) / EULER_FV_OWN);
}

template <typename A, typename B>
__global__ void k_convert(const A* in, B* out, long long n)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        out[i] = (B)in[i];
}

}  // namespace

cudaError_t launch_fv_step_f64(int kind, double a, double alpha, double lambda,
                               const double* uin, double* uout, int64_t n,
                               int periodic, cudaStream_t st)
{
    FvParams<double> P{kind, a, alpha, lambda};
    k_fv_step<double><<<grid_for(n, 256), 256, 0, st>>>(P, uin, uout, n, periodic);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_fv_step_f32(int kind, double a, double alpha, double lambda,
                               const float* uin, float* uout, int64_t n,
                               int periodic, cudaStream_t st)
{
    FvParams<float> P{kind, (float)a, (float)alpha, (float)lambda};
    k_fv_step<float><<<grid_for(n, 256), 256, 0, st>>>(P, uin, uout, n, periodic);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_fv_tb_f64(int kind, double a, double alpha, double lambda, const double* uin,
                             double* uout, int64_t n, int K, cudaStream_t st)
{
    return launch_fv_tb<double>(FvParams<double>{kind, a, alpha, lambda}, uin, uout, n, K, st);
}

cudaError_t launch_fv_tb_f32(int kind, double a, double alpha, double lambda, const float* uin,
                             float* uout, int64_t n, int K, cudaStream_t st)
{
    return launch_fv_tb<float>(FvParams<float>{kind, (float)a, (float)alpha, (float)lambda}, uin,
                               uout, n, K, st);
}

cudaError_t launch_euler_fv_f64(double gamma, double lambda, const double* uin,
                                double* uout, int64_t n, cudaStream_t st)
{
    k_euler_fv<double><<<euler_fv_grid(n), 32, 0, st>>>(gamma, lambda, uin, uout, n);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_euler_fv_f32(double gamma, double lambda, const float* uin,
                                float* uout, int64_t n, cudaStream_t st)
{
    k_euler_fv<float><<<euler_fv_grid(n), 32, 0, st>>>((float)gamma, (float)lambda,
                                                      uin, uout, n);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_convert_f64_to_f32(const double* in, float* out, int64_t n,
                                      cudaStream_t st)
{
    k_convert<double, float><<<grid_for(n, 256), 256, 0, st>>>(in, out, n);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_convert_f32_to_f64(const float* in, double* out, int64_t n,
                                      cudaStream_t st)
{
    k_convert<float, double><<<grid_for(n, 256), 256, 0, st>>>(in, out, n);
    note_launches();
    return cudaGetLastError();
}

}  // namespace fqnm
