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
//  * k_step_resident: a short periodic line held whole by one block (n/V
//    threads, V cells each), every step of the call in one launch: each
//    step is exact over the whole line (no halo), so the latency per step
//    is a few shuffles, one shared-memory exchange and one barrier.
#include "tile_step.cuh"

namespace fqnm {

namespace {

using tb::EvTablePM;
using tb::EvTableP;
using tb::EvClosedP;
using tb::TB_MAX_BLOCK;

// ---- naive kernel -------------------------------------------------------------

__global__ void k_step_naive(RuleView r, const int* __restrict__ qin,
                             int* __restrict__ qout, long long n, int periodic,
                             unsigned* err, long long* bflux)
{
    unsigned acc = 0;
    auto ev = [&](int q, int& p, int& m) {             // (phi+, phi-) table gather
        unsigned k = (unsigned)(q - r.lo);
        acc = max(acc, k);
        k = min(k, r.span);
        const int2 v = r.tab2[k];
        p = v.x;
        m = v.y;
    };
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
        ev(qin[il], pl, ml);
        ev(qin[i], pc, mc);
        ev(qin[ir], pr, mr);
        const int Fr = r.face_max ? max(pc, mr) : pc + mr;   // F_{i+1/2}
        const int Fl = r.face_max ? max(pl, mc) : pl + mc;   // F_{i-1/2}
        qout[i] = qin[i] - (Fr - Fl);
        if (!periodic && bflux) {
            if (i == 0) atomicAdd((unsigned long long*)bflux, (unsigned long long)(-(long long)Fl));
            if (i == n - 1) atomicAdd((unsigned long long*)bflux, (unsigned long long)(long long)Fr);
        }
    }
    if (acc > r.span) atomicOr(err, ERRBIT_RANGE);
}

// ---- temporal-blocked kernel -----------------------------------------------------

template <class Ev, int V, int LAYOUT, bool WARP>
__global__ void __launch_bounds__(tb::TB_MAX_BLOCK)
k_step_tb(const int* __restrict__ qin, int* __restrict__ qout, long long n,
          int K, long long S, Ev ev, unsigned* __restrict__ err)
{
    __shared__ tb::TileSmem sm;
    tb::tile_step<Ev, V, LAYOUT, WARP>(qin, qout, n, K, S, (long long)blockIdx.x, ev, err, sm);
}

template <class Ev, int V, int LAYOUT>
cudaError_t launch_tb_t(const Ev& ev, int block, int pdl, const int* qin, int* qout,
                        long long n, int k, unsigned* err, cudaStream_t st)
{
    const long long E = (long long)block * V;
    const long long S = E - 2LL * k;
    const long long grid = (n + S - 1) / S;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)grid);
    cfg.blockDim = dim3((unsigned)block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    cudaError_t e;
    if (block == 32)
        e = cudaLaunchKernelEx(&cfg, k_step_tb<Ev, V, LAYOUT, true>, qin, qout, n, k, S, ev, err);
    else
        e = cudaLaunchKernelEx(&cfg, k_step_tb<Ev, V, LAYOUT, false>, qin, qout, n, k, S, ev, err);
    if (e != cudaSuccess) return e;
    note_launches();
    return cudaGetLastError();
}

// ---- resident kernel ----------------------------------------------------------

// Thread t holds cells [tV, tV + V) of the n = blockDim.x * V cells.  The
// last warp may be partial: its shuffles use the mask of its lanes.  Warp
// edges and the periodic wrap go through shared memory: each warp publishes
// p of its last cell and m of its first (double-buffered by step parity, one
// barrier per step); warp 0's left neighbour is the last warp, and the last
// warp's right neighbour is warp 0.
template <class Ev, int V>
__global__ void __launch_bounds__(RESIDENT_MAX_THREADS)
k_step_resident(const int* __restrict__ qin, int* __restrict__ qout, long long steps, Ev ev,
                unsigned* __restrict__ err)
{
    __shared__ int shp[2][RESIDENT_MAX_THREADS / 32], shm[2][RESIDENT_MAX_THREADS / 32];
    const int t = threadIdx.x, lane = t & 31, w = t >> 5;
    const int nw = (blockDim.x + 31) >> 5;
    const int nl = w == nw - 1 ? (int)blockDim.x - 32 * (nw - 1) : 32;   // lanes of this warp
    const unsigned mask = nl == 32 ? 0xffffffffu : ((1u << nl) - 1u);
    const int wl = w == 0 ? nw - 1 : w - 1, wr = w == nw - 1 ? 0 : w + 1;
    int q[V];
#pragma unroll
    for (int j = 0; j < V; ++j) q[j] = __ldg(qin + t * V + j);
    unsigned acc = 0;
    for (long long s = 0; s < steps; ++s) {
        int p[V], m[V];
#pragma unroll
        for (int j = 0; j < V; ++j) ev(q[j], p[j], m[j], acc);
        const int b = (int)(s & 1);
        if (lane == nl - 1) shp[b][w] = p[V - 1];
        if (Ev::HAS_M && lane == 0) shm[b][w] = m[0];
        __syncthreads();
        int pl = __shfl_up_sync(mask, p[V - 1], 1);
        if (lane == 0) pl = shp[b][wl];
        int mr = 0;
        if (Ev::HAS_M) {
            mr = __shfl_down_sync(mask, m[0], 1);
            if (lane == nl - 1) mr = shm[b][wr];
        }
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int l = j > 0 ? p[j - 1] : pl;
            int d = l - p[j];
            if (Ev::HAS_M) {
                const int r = j < V - 1 ? m[j + 1] : mr;
                d = Ev::FACE_MAX ? max(l, m[j]) - max(p[j], r) : d + m[j] - r;
            }
            q[j] += d;
        }
    }
#pragma unroll
    for (int j = 0; j < V; ++j) qout[t * V + j] = q[j];
    if (acc > ev.span) atomicOr(err, ERRBIT_RANGE);
}

template <class Ev>
cudaError_t launch_resident_t(const Ev& ev, int v, const int* qin, int* qout, long long n,
                              long long steps, unsigned* err, cudaStream_t st)
{
    const unsigned threads = (unsigned)(n / v);
    switch (v) {
    case 1: k_step_resident<Ev, 1><<<1, threads, 0, st>>>(qin, qout, steps, ev, err); break;
    case 2: k_step_resident<Ev, 2><<<1, threads, 0, st>>>(qin, qout, steps, ev, err); break;
    case 4: k_step_resident<Ev, 4><<<1, threads, 0, st>>>(qin, qout, steps, ev, err); break;
    case 8: k_step_resident<Ev, 8><<<1, threads, 0, st>>>(qin, qout, steps, ev, err); break;
    default: return cudaErrorInvalidValue;
    }
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
            return launch_tb_t<Ev, VV, LAYOUT_INTERLEAVED>(ev, p.block, p.pdl, qin, qout, n, k, err, st); \
        return launch_tb_t<Ev, VV, LAYOUT_BLOCKED>(ev, p.block, p.pdl, qin, qout, n, k, err, st); \
    }
#define FQNM_TB_RUNS(VV, LL)                                                      \
    if (p.v == VV && p.layout == LL)                                              \
        return launch_tb_t<Ev, VV, LL>(ev, p.block, p.pdl, qin, qout, n, k, err, st);
    FQNM_TB_RUNS(8, LAYOUT_RUNS4)
    FQNM_TB_RUNS(16, LAYOUT_RUNS4)
    FQNM_TB_RUNS(32, LAYOUT_RUNS4)
    FQNM_TB_RUNS(16, LAYOUT_RUNS8)
    FQNM_TB_RUNS(32, LAYOUT_RUNS8)
    FQNM_TB_CASE(4)
    FQNM_TB_CASE(8)
    FQNM_TB_CASE(16)
    FQNM_TB_CASE(32)
#undef FQNM_TB_CASE
#undef FQNM_TB_RUNS
    return cudaErrorInvalidValue;
}

}  // namespace

bool tb_plan_supported(const RuleView& r, const Plan& p)
{
    (void)r;
    if (p.v != 4 && p.v != 8 && p.v != 16 && p.v != 32) return false;
    if (p.block < 32 || p.block > TB_MAX_BLOCK || p.block % 32) return false;
    if (p.layout < LAYOUT_INTERLEAVED || p.layout > LAYOUT_RUNS8) return false;
    // a runs layout needs at least two runs per lane (one run is BLOCKED)
    if (p.layout == LAYOUT_RUNS4 && p.v < 8) return false;
    if (p.layout == LAYOUT_RUNS8 && p.v < 16) return false;
    return p.k >= 1 && 2LL * p.k < (long long)p.block * p.v;
}

int resident_v(int64_t n)
{
    // at most 256 threads where that fits (a step's latency, about 300 to
    // 450 cycles, barely moves between 256 and 1024 threads), else the most
    // cells per thread that fit one block
    for (int v : {1, 2, 4, 8})
        if (n % v == 0 && n / v <= 256) return v;
    for (int v : {8, 4, 2, 1})
        if (n % v == 0 && n / v <= RESIDENT_MAX_THREADS) return v;
    return 0;
}

cudaError_t launch_step_resident(const RuleView& r, const int32_t* qin, int32_t* qout,
                                 int64_t n, int64_t steps, unsigned* err, cudaStream_t st)
{
    const int v = resident_v(n);
    if (v == 0 || n < 1 || steps < 1) return cudaErrorInvalidValue;
    if (r.evaluator == EVAL_CLOSED_FORM && !r.has_m)
        return launch_resident_t(EvClosedP{r.cf, r.lo, r.span}, v, qin, qout, n, steps, err, st);
    if (!r.has_m)
        return launch_resident_t(EvTableP{r.tabp, r.lo, r.span}, v, qin, qout, n, steps, err, st);
    if (r.face_max) {
        tb::EvTablePMMax ev;
        ev.tab = r.tab2;
        ev.lo = r.lo;
        ev.span = r.span;
        return launch_resident_t(ev, v, qin, qout, n, steps, err, st);
    }
    if (r.tab16)
        return launch_resident_t(tb::EvTablePM16{r.tab16, r.lo, r.span}, v, qin, qout, n, steps,
                                 err, st);
    return launch_resident_t(EvTablePM{r.tab2, r.lo, r.span}, v, qin, qout, n, steps, err, st);
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
    if (!r.has_m) {                              // phi- == 0: the max is the sum too
        EvTableP ev{r.tabp, r.lo, r.span};
        return dispatch_tb(ev, p, qin, qout, n, k, err, st);
    }
    if (r.face_max) {
        tb::EvTablePMMax ev;
        ev.tab = r.tab2;
        ev.lo = r.lo;
        ev.span = r.span;
        return dispatch_tb(ev, p, qin, qout, n, k, err, st);
    }
    if (r.tab16) {
        tb::EvTablePM16 ev{r.tab16, r.lo, r.span};
        return dispatch_tb(ev, p, qin, qout, n, k, err, st);
    }
    EvTablePM ev{r.tab2, r.lo, r.span};
    return dispatch_tb(ev, p, qin, qout, n, k, err, st);
}

}  // namespace fqnm
