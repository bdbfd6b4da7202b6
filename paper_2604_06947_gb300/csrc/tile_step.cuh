// tile_step.cuh -- one tile of the temporal-blocked quantised step.
//
// The block holds E = blockDim*V cells of one periodic problem in registers,
// starting K cells left of the tile's first output cell, applies K steps of
// eq. update_rule and writes the E-2K cells whose dependency cone stayed
// inside the block.  Used by the single-problem kernel (one tile per block)
// and by the batched serving kernel (tiles of many problems per launch).
// See k_scalar.cu for the layouts and the evaluators' contract.
#pragma once

#include "closed_form.cuh"

namespace fqnm {
namespace tb {

constexpr unsigned FULL = 0xffffffffu;

// ---- transfer-map evaluators ------------------------------------------------
// operator()(q, p, m, acc): p = phi+(q), m = phi-(q); acc tracks max(q - lo)
// as unsigned, so a state below lo or above hi shows up as acc > span.
// FACE_MAX: the face transfer is max(phi+(q_L), phi-(q_R)) (the Godunov flux
// of Burgers from its Engquist-Osher maps) instead of the sum.

struct EvTablePM {                    // both maps from the (phi+, phi-) table
    static constexpr bool FACE_MAX = false;
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

struct EvTablePM16 {                  // both maps packed as int16 halves of one word
    static constexpr bool FACE_MAX = false;
    static constexpr bool HAS_M = true;
    const int* __restrict__ tab;
    int lo;
    unsigned span;
    __device__ __forceinline__ void operator()(int q, int& p, int& m,
                                               unsigned& acc) const
    {
        unsigned i = (unsigned)(q - lo);
        acc = max(acc, i);
        i = min(i, span);
        const int v = __ldg(tab + i);
        p = (int)(short)(v & 0xffff);   // sign-extend the low half
        m = v >> 16;                    // arithmetic shift keeps the sign
    }
};

struct EvTableP {                     // phi- == 0 on the range: phi+ only
    static constexpr bool FACE_MAX = false;
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
    static constexpr bool FACE_MAX = false;
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

struct EvTablePMMax : EvTablePM {    // Godunov faces from the EO maps
    static constexpr bool FACE_MAX = true;
};

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

struct TileSmem {
    int shp[2][TB_MAX_BLOCK / 32];
    int shm[2][TB_MAX_BLOCK / 32];
};

// All threads of the block must call this with the same arguments.  WARP:
// the block is one warp (blockDim 32): no shared-memory edge exchange and no
// block barrier; its two end cells take ghost copies of themselves.
template <class Ev, int V, int LAYOUT, bool WARP = false>
__device__ __forceinline__ void tile_step(const int* __restrict__ qin,
                                          int* __restrict__ qout, long long n,
                                          int K, long long S, long long tile,
                                          const Ev& ev, unsigned* __restrict__ err,
                                          TileSmem& sm)
{
    int (&shp)[2][TB_MAX_BLOCK / 32] = sm.shp;
    int (&shm)[2][TB_MAX_BLOCK / 32] = sm.shm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int nw = blockDim.x >> 5;
    const long long start = tile * S - K;

    // Programmatic dependent launch: when the previous step launch was
    // launched as this one's programmatic predecessor, wait here until it has
    // completed and its stores are visible (a no-op otherwise).
    asm volatile("griddepcontrol.wait;" ::: "memory");
    int q[V];
    // blocked layout: a thread's V cells are consecutive, so an aligned run
    // inside [0, n) loads as int4 vectors (16-byte loads, fully used);
    // wrapped or misaligned runs load cell by cell
    const long long c0 = start + (long long)threadIdx.x * V;
    const bool vec = LAYOUT == LAYOUT_BLOCKED && V % 4 == 0 && c0 >= 0 && c0 + V <= n &&
                     (reinterpret_cast<uintptr_t>(qin + c0) & 15) == 0;
    if (vec) {
#pragma unroll
        for (int j = 0; j < V; j += 4) {
            const int4 v = __ldg(reinterpret_cast<const int4*>(qin + c0 + j));
            q[j] = v.x;
            q[j + 1] = v.y;
            q[j + 2] = v.z;
            q[j + 3] = v.w;
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const long long gi = wrap_index(start + cell_of<LAYOUT, V>(j), n);
            q[j] = FQNM_IN_RANGE(gi, n, err) ? __ldg(qin + gi) : 0;
        }
    }

    unsigned acc = 0;
    for (int s = 0; s < K; ++s) {
        int p[V], m[V];
#pragma unroll
        for (int j = 0; j < V; ++j) ev(q[j], p[j], m[j], acc);

        // edge values of each warp for its neighbours: p of the last cell,
        // m of the first cell (double-buffered: one barrier per step)
        // (lane 31's p and lane 0's m are broadcast by a shuffle and every
        // lane stores the same value: one slot per warp, no lane-dependent
        // branch, and the shared-memory footprint stays small so the L1 that
        // serves the table gathers keeps its capacity)
        int pe = 0, me = 0;
        if (!WARP) {
            const int b = s & 1;
            shp[b][w] = __shfl_sync(FULL, p[V - 1], 31);
            if (Ev::HAS_M) shm[b][w] = __shfl_sync(FULL, m[0], 0);
            __syncthreads();
            pe = shp[b][w > 0 ? w - 1 : 0];                   // block edge: invalid anyway
            me = Ev::HAS_M ? shm[b][w < nw - 1 ? w + 1 : w] : 0;
        }

        // The block's two end cells have no neighbour in the block; they
        // use a ghost copy of themselves (a transmissive end).  Their values
        // are outside the exact region anyway, but this keeps them on a valid
        // scheme, so they stay in the range the maps are verified on.
        const bool first_owner = WARP ? lane == 0 : (w == 0 && lane == 0);
        const bool last_owner = WARP ? lane == 31 : (w == nw - 1 && lane == 31);
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
                    d = Ev::FACE_MAX ? max(pl, m[j]) - max(p[j], mr) : d + m[j] - mr;
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
                    d = Ev::FACE_MAX ? max(pl, m[j]) - max(p[j], mr) : d + m[j] - mr;
                }
                q[j] += d;
            }
        }
    }

    // let the next step launch start its blocks (they wait for this grid)
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");

    // cells [K, K+S) of the block are exact after K steps; in the blocked
    // layout a thread's aligned groups of 4 inside that range and inside
    // [0, n) store as int4 vectors
#pragma unroll
    for (int j0 = 0; j0 < V; j0 += (LAYOUT == LAYOUT_BLOCKED && V % 4 == 0) ? 4 : 1) {
        if (LAYOUT == LAYOUT_BLOCKED && V % 4 == 0) {
            const long long e = (long long)threadIdx.x * V + j0;
            const long long o = tile * S + (e - K);
            if (e >= K && e + 4 <= K + S && o + 4 <= n &&
                (reinterpret_cast<uintptr_t>(qout + o) & 15) == 0) {
                if (FQNM_IN_RANGE(o + 3, n, err))
                    *reinterpret_cast<int4*>(qout + o) =
                        make_int4(q[j0], q[j0 + 1], q[j0 + 2], q[j0 + 3]);
                continue;
            }
#pragma unroll
            for (int j = j0; j < j0 + 4; ++j) {
                const long long ej = (long long)threadIdx.x * V + j;
                if (ej >= K && ej < K + S) {
                    const long long oj = tile * S + (ej - K);
                    if (oj < n && FQNM_IN_RANGE(oj, n, err)) qout[oj] = q[j];
                }
            }
        } else {
            const long long e = cell_of<LAYOUT, V>(j0);
            if (e >= K && e < K + S) {
                const long long o = tile * S + (e - K);
                if (o < n && FQNM_IN_RANGE(o, n, err)) qout[o] = q[j0];
            }
        }
    }
    if (acc > ev.span) atomicOr(err, ERRBIT_RANGE);
}


}  // namespace tb
}  // namespace fqnm
