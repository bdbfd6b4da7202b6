// k_scalar.cu -- the quantised conservative step for scalar laws.
//
// eq. update_rule / numerical_count_flux_definition:
//     F_{i+1/2} = phi+(q_i) + phi-(q_{i+1})
//     q_i <- q_i - (F_{i+1/2} - F_{i-1/2})
// Per cell and step this is one transfer-map evaluation (a table gather or
// an integer closed form), one add per face and two subtractions per cell
// (§2.4 Complexity); the arithmetic is exact, so any execution order gives
// the same integers.
//
// Two kernels:
//  * k_step_naive: one thread per cell, one step per launch, periodic or
//    transmissive ends (ghost cell = edge cell).  Plain reference path.
//  * k_step_tb: temporal blocking.  A block holds E = blockDim*V cells in
//    registers, steps them K times and writes the E-2K cells whose
//    dependency cone stayed inside the block (the invalid margin grows by one
//    cell per side per step).  Neighbour values move between lanes by warp
//    shuffles and between warps through shared memory (one barrier per
//    step).  Periodic ends only.  HBM traffic is 8 bytes per cell per K
//    steps instead of per step.
//    Two register layouts of a warp's 32*V cells:
//      INTERLEAVED  lane l holds cells 32*j + l (j < V): a warp-wide table
//                   gather touches 32 neighbouring cells, whose states are
//                   close, so it hits one or two cache lines;
//      BLOCKED      lane l holds cells V*l + j: neighbours are mostly in the
//                   same thread (two shuffles per V cells), best when the
//                   map is a closed form and there is no gather.
#include "closed_form.cuh"

namespace fqnm {

namespace {

constexpr unsigned FULL = 0xffffffffu;

// ---- transfer-map evaluators ------------------------------------------------
// operator()(q, p, m, acc): p = phi+(q), m = phi-(q); acc tracks max(q - lo)
// as unsigned, so a state below lo or above hi shows up as acc > span.

struct EvTablePM {                    // both maps from the (phi+, phi-) table
    static constexpr bool HAS_M = true;
    const int2* __restrict__ tab;
    int lo;
    unsigned span;
    __device__ __forceinline__ void operator()(int q, int& p, int& m,
                                               unsigned& acc) const
    {
        unsigned i = (unsigned)(q - lo);
        acc = max(acc, i);
        i = min(i, span);               // never read outside the table
        const int2 v = __ldg(tab + i);
        p = v.x;
        m = v.y;
    }
};

struct EvTableP {                     // phi- == 0 on the range: phi+ only
    static constexpr bool HAS_M = false;
    const int* __restrict__ tab;
    int lo;
    unsigned span;
    __device__ __forceinline__ void operator()(int q, int& p, int& m,
                                               unsigned& acc) const
    {
        unsigned i = (unsigned)(q - lo);
        acc = max(acc, i);
        i = min(i, span);
        p = __ldg(tab + i);
        m = 0;
    }
};

struct EvClosedP {                    // phi+(q) = R(q num/den), phi- == 0
    static constexpr bool HAS_M = false;
    ClosedForm cf;
    int lo;
    unsigned span;
    __device__ __forceinline__ void operator()(int q, int& p, int& m,
                                               unsigned& acc) const
    {
        acc = max(acc, (unsigned)(q - lo));
        p = cf_eval(q, cf);
        m = 0;
    }
};

// ---- naive kernel -------------------------------------------------------------

__global__ void k_step_naive(RuleView r, const int* __restrict__ qin,
                             int* __restrict__ qout, long long n, int periodic,
                             unsigned* err, long long* bflux)
{
    EvTablePM ev{r.tab2, r.lo, r.span};
    unsigned acc = 0;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        long long il = i - 1, ir = i + 1;
        if (periodic) {
            if (il < 0) il = n - 1;
            if (ir >= n) ir = 0;
        } else {                                   // ghost = edge cell
            if (il < 0) il = 0;
            if (ir >= n) ir = n - 1;
        }
        int pl, ml, pc, mc, pr, mr;
        ev(qin[il], pl, ml, acc);
        ev(qin[i], pc, mc, acc);
        ev(qin[ir], pr, mr, acc);
        const int Fr = pc + mr;                    // F_{i+1/2}
        const int Fl = pl + mc;                    // F_{i-1/2}
        qout[i] = qin[i] - (Fr - Fl);
        if (!periodic && bflux) {
            if (i == 0) atomicAdd((unsigned long long*)bflux, (unsigned long long)(-(long long)Fl));
            if (i == n - 1) atomicAdd((unsigned long long*)bflux, (unsigned long long)(long long)Fr);
        }
    }
    if (acc > r.span) atomicOr(err, ERRBIT_RANGE);
}

// ---- temporal-blocked kernel -----------------------------------------------------

__device__ __forceinline__ long long wrap_index(long long g, long long n)
{
    if (g < 0) g += n;
    if (g >= n) g -= n;
    if (g < 0 || g >= n) {                         // tiny domains: several wraps
        g %= n;
        if (g < 0) g += n;
    }
    return g;
}

template <int LAYOUT, int V>
__device__ __forceinline__ long long cell_of(int j)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (LAYOUT == LAYOUT_INTERLEAVED) return (long long)w * 32 * V + j * 32 + lane;
    return (long long)threadIdx.x * V + j;
}

constexpr int TB_MAX_BLOCK = 512;

template <class Ev, int V, int LAYOUT>
__global__ void __launch_bounds__(TB_MAX_BLOCK)
k_step_tb(const int* __restrict__ qin, int* __restrict__ qout, long long n,
          int K, long long S, Ev ev, unsigned* __restrict__ err)
{
    __shared__ int shp[2][TB_MAX_BLOCK / 32];
    __shared__ int shm[2][TB_MAX_BLOCK / 32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const long long start = (long long)blockIdx.x * S - K;

    int q[V];
#pragma unroll
    for (int j = 0; j < V; ++j)
        q[j] = __ldg(qin + wrap_index(start + cell_of<LAYOUT, V>(j), n));

    unsigned acc = 0;
    for (int s = 0; s < K; ++s) {
        int p[V], m[V];
#pragma unroll
        for (int j = 0; j < V; ++j) ev(q[j], p[j], m[j], acc);

        // edge values of each warp for its neighbours: p of the last cell,
        // m of the first cell (double-buffered: one barrier per step)
        const int b = s & 1;
        if (lane == 31) shp[b][w] = p[V - 1];
        if (Ev::HAS_M && lane == 0) shm[b][w] = m[0];
        __syncthreads();
        const int pe = shp[b][w > 0 ? w - 1 : 0];            // block edge: invalid anyway
        const int me = Ev::HAS_M ? shm[b][w < nw - 1 ? w + 1 : w] : 0;

        // The block's two end cells have no neighbour in the block; they
        // use a ghost copy of themselves (a transmissive end).  Their values
        // are outside the exact region anyway, but this keeps them on a valid
        // scheme, so they stay in the range the maps are verified on.
        const bool first_owner = (w == 0 && lane == 0);
        const bool last_owner = (w == nw - 1 && lane == 31);
        if (LAYOUT == LAYOUT_INTERLEAVED) {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                // left neighbour of (j, lane) is (j, lane-1); of (j, 0) it is
                // (j-1, 31), offered by lane 31 to lane 0
                const int offp = (lane == 31) ? (j > 0 ? p[j - 1] : pe) : p[j];
                int pl = __shfl_sync(FULL, offp, (lane + 31) & 31);
                if (j == 0 && first_owner) pl = p[0];
                int d = pl - p[j];                            // F_{i-1/2} - F_{i+1/2}
                if (Ev::HAS_M) {
                    const int offm = (lane == 0) ? (j < V - 1 ? m[j + 1] : me) : m[j];
                    int mr = __shfl_sync(FULL, offm, (lane + 1) & 31);
                    if (j == V - 1 && last_owner) mr = m[V - 1];
                    d += m[j] - mr;
                }
                q[j] += d;
            }
        } else {
            int pl0 = __shfl_up_sync(FULL, p[V - 1], 1);
            if (lane == 0) pl0 = first_owner ? p[0] : pe;
            int mrV = 0;
            if (Ev::HAS_M) {
                mrV = __shfl_down_sync(FULL, m[0], 1);
                if (lane == 31) mrV = last_owner ? m[V - 1] : me;
            }
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int pl = j > 0 ? p[j - 1] : pl0;
                int d = pl - p[j];
                if (Ev::HAS_M) {
                    const int mr = j < V - 1 ? m[j + 1] : mrV;
                    d += m[j] - mr;
                }
                q[j] += d;
            }
        }
    }

    // cells [K, K+S) of the block are exact after K steps
#pragma unroll
    for (int j = 0; j < V; ++j) {
        const long long e = cell_of<LAYOUT, V>(j);
        if (e >= K && e < K + S) {
            const long long o = (long long)blockIdx.x * S + (e - K);
            if (o < n) qout[o] = q[j];
        }
    }
    if (acc > ev.span) atomicOr(err, ERRBIT_RANGE);
}

template <class Ev, int V, int LAYOUT>
cudaError_t launch_tb_t(const Ev& ev, int block, const int* qin, int* qout,
                        long long n, int k, unsigned* err, cudaStream_t st)
{
    const long long E = (long long)block * V;
    const long long S = E - 2LL * k;
    const long long grid = (n + S - 1) / S;
    k_step_tb<Ev, V, LAYOUT><<<(unsigned)grid, block, 0, st>>>(qin, qout, n, k, S, ev, err);
    note_launches();
    return cudaGetLastError();
}

template <class Ev>
cudaError_t dispatch_tb(const Ev& ev, const Plan& p, const int* qin, int* qout,
                        long long n, int k, unsigned* err, cudaStream_t st)
{
#define FQNM_TB_CASE(VV)                                                          \
    if (p.v == VV) {                                                              \
        if (p.layout == LAYOUT_INTERLEAVED)                                       \
            return launch_tb_t<Ev, VV, LAYOUT_INTERLEAVED>(ev, p.block, qin, qout, n, k, err, st); \
        return launch_tb_t<Ev, VV, LAYOUT_BLOCKED>(ev, p.block, qin, qout, n, k, err, st); \
    }
    FQNM_TB_CASE(4)
    FQNM_TB_CASE(8)
    FQNM_TB_CASE(16)
#undef FQNM_TB_CASE
    return cudaErrorInvalidValue;
}

}  // namespace

bool tb_plan_supported(const RuleView& r, const Plan& p)
{
    (void)r;
    if (p.v != 4 && p.v != 8 && p.v != 16) return false;
    if (p.block < 32 || p.block > TB_MAX_BLOCK || p.block % 32) return false;
    if (p.layout != LAYOUT_INTERLEAVED && p.layout != LAYOUT_BLOCKED) return false;
    return p.k >= 1 && 2LL * p.k < (long long)p.block * p.v;
}

cudaError_t launch_step_naive(const RuleView& r, const int32_t* qin,
                              int32_t* qout, int64_t n, int periodic,
                              unsigned* err, long long* bflux, cudaStream_t st)
{
    k_step_naive<<<grid_for(n, 256), 256, 0, st>>>(r, qin, qout, n, periodic, err, bflux);
    note_launches();
    return cudaGetLastError();
}

cudaError_t launch_step_tb(const RuleView& r, const Plan& p, const int32_t* qin,
                           int32_t* qout, int64_t n, int k, unsigned* err,
                           cudaStream_t st)
{
    if (!tb_plan_supported(r, p) || 2LL * k >= (long long)p.block * p.v)
        return cudaErrorInvalidValue;
    if (r.evaluator == EVAL_CLOSED_FORM && !r.has_m) {
        EvClosedP ev{r.cf, r.lo, r.span};
        return dispatch_tb(ev, p, qin, qout, n, k, err, st);
    }
    if (!r.has_m) {
        EvTableP ev{r.tabp, r.lo, r.span};
        return dispatch_tb(ev, p, qin, qout, n, k, err, st);
    }
    EvTablePM ev{r.tab2, r.lo, r.span};
    return dispatch_tb(ev, p, qin, qout, n, k, err, st);
}

}  // namespace fqnm
