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

// BIASED evaluators also offer at(i, p, m): the maps at table index
// i = q - lo (clamped to the table), for kernels that hold q - lo.
struct EvTablePM {                    // both maps from the (phi+, phi-) table
    static constexpr bool FACE_MAX = false;
    static constexpr bool HAS_M = true;
    static constexpr bool BIASED = true;
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
    __device__ __forceinline__ void at(unsigned i, int& p, int& m) const
    {
        const int2 v = __ldg(tab + min(i, span));
        p = v.x;
        m = v.y;
    }
};

struct EvTablePM16 {                  // both maps packed as int16 halves of one word
    static constexpr bool FACE_MAX = false;
    static constexpr bool HAS_M = true;
    static constexpr bool BIASED = true;
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
    __device__ __forceinline__ void at(unsigned i, int& p, int& m) const
    {
        const int v = __ldg(tab + min(i, span));
        p = (int)(short)(v & 0xffff);
        m = v >> 16;
    }
};

struct EvTableP {                     // phi- == 0 on the range: phi+ only
    static constexpr bool FACE_MAX = false;
    static constexpr bool HAS_M = false;
    static constexpr bool BIASED = true;
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
    __device__ __forceinline__ void at(unsigned i, int& p, int& m) const
    {
        p = __ldg(tab + min(i, span));
        m = 0;
    }
};

struct EvClosedP {                    // phi+(q) = R(q num/den), phi- == 0
    static constexpr bool FACE_MAX = false;
    static constexpr bool HAS_M = false;
    static constexpr bool BIASED = false;
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

// Run length of a layout: a lane holds V/R runs of R consecutive cells, run
// k of a warp's 32 lanes covering 32*R consecutive cells (INTERLEAVED: R = 1;
// BLOCKED: R = V, one run per lane; RUNS4 / RUNS8: R = 4 / 8, so that one
// warp-wide table gather touches 32*R neighbouring cells, while a cell's
// neighbours stay in the thread except at a run's two ends).
template <int LAYOUT, int V>
__device__ __host__ constexpr int run_len()
{
    return LAYOUT == LAYOUT_INTERLEAVED ? 1 : LAYOUT == LAYOUT_RUNS4 ? 4
                                            : LAYOUT == LAYOUT_RUNS8 ? 8 : V;
}

template <int LAYOUT, int V>
__device__ __forceinline__ long long cell_of(int j)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (LAYOUT == LAYOUT_INTERLEAVED) return (long long)w * 32 * V + j * 32 + lane;
    if (LAYOUT == LAYOUT_RUNS4 || LAYOUT == LAYOUT_RUNS8) {
        constexpr int R = run_len<LAYOUT, V>();
        return (long long)w * 32 * V + (j / R) * 32 * R + lane * R + (j % R);
    }
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
    constexpr bool RUNS = LAYOUT == LAYOUT_RUNS4 || LAYOUT == LAYOUT_RUNS8;
    constexpr int R = run_len<LAYOUT, V>();
    const long long c0 = start + (long long)threadIdx.x * V;
    const bool vec = LAYOUT == LAYOUT_BLOCKED && V % 4 == 0 && c0 >= 0 && c0 + V <= n &&
                     (reinterpret_cast<uintptr_t>(qin + c0) & 15) == 0;
    if (RUNS) {
        // each run of R cells loads as R/4 int4 vectors when aligned and
        // inside [0, n), else cell by cell (wrapped)
#pragma unroll
        for (int k = 0; k < V / R; ++k) {
            const long long r0 = start + cell_of<LAYOUT, V>(k * R);
            if (r0 >= 0 && r0 + R <= n && (reinterpret_cast<uintptr_t>(qin + r0) & 15) == 0) {
#pragma unroll
                for (int i = 0; i < R; i += 4) {
                    const int4 v = __ldg(reinterpret_cast<const int4*>(qin + r0 + i));
                    q[k * R + i] = v.x;
                    q[k * R + i + 1] = v.y;
                    q[k * R + i + 2] = v.z;
                    q[k * R + i + 3] = v.w;
                }
            } else {
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const long long gi = wrap_index(r0 + i, n);
                    q[k * R + i] = FQNM_IN_RANGE(gi, n, err) ? __ldg(qin + gi) : 0;
                }
            }
        }
    } else if (vec) {
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
    // A table evaluator's block holds q - lo (the update only moves
    // differences, so the offset is removed once here and restored at the
    // store): the state is then the table index itself, and the range
    // guard is one three-way maximum per two cells.
    constexpr bool BIASED = Ev::BIASED;
    const unsigned bias = BIASED ? (unsigned)ev.lo : 0u;
    if (BIASED) {
#pragma unroll
        for (int j = 0; j < V; ++j) q[j] = (int)((unsigned)q[j] - bias);
    }

    unsigned acc = 0;
    for (int s = 0; s < K; ++s) {
        int p[V], m[V];
        if constexpr (BIASED) {
#pragma unroll
            for (int j = 0; j + 1 < V; j += 2)
                acc = __vimax3_u32(acc, (unsigned)q[j], (unsigned)q[j + 1]);
            if (V & 1) acc = max(acc, (unsigned)q[V - 1]);
#pragma unroll
            for (int j = 0; j < V; ++j) ev.at((unsigned)q[j], p[j], m[j]);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) ev(q[j], p[j], m[j], acc);
        }

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
        if (RUNS) {
#pragma unroll
            for (int k = 0; k < V / R; ++k) {
                // the run's first cell: its left neighbour ends lane-1's run
                // k; lane 0's is the end of lane 31's run k-1 (or, for k = 0,
                // the previous warp's last cell); mirrored on the right
                const int offp = (lane == 31) ? (k > 0 ? p[k * R - 1] : pe) : p[k * R + R - 1];
                int pl = __shfl_sync(FULL, offp, (lane + 31) & 31);
                if (k == 0 && first_owner) pl = p[0];
                int mr = 0;
                if (Ev::HAS_M) {
                    const int offm = (lane == 0) ? (k < V / R - 1 ? m[(k + 1) * R] : me) : m[k * R];
                    mr = __shfl_sync(FULL, offm, (lane + 1) & 31);
                    if (k == V / R - 1 && last_owner) mr = m[V - 1];
                }
#pragma unroll
                for (int i = 0; i < R; ++i) {
                    const int j = k * R + i;
                    const int plj = i > 0 ? p[j - 1] : pl;
                    int d = plj - p[j];
                    if (Ev::HAS_M) {
                        const int mrj = i < R - 1 ? m[j + 1] : mr;
                        d = Ev::FACE_MAX ? max(plj, m[j]) - max(p[j], mrj) : d + m[j] - mrj;
                    }
                    q[j] += d;
                }
            }
        } else if (LAYOUT == LAYOUT_INTERLEAVED) {
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
    for (int j0 = 0; j0 < V; j0 += ((LAYOUT == LAYOUT_BLOCKED && V % 4 == 0) || RUNS) ? 4 : 1) {
        if ((LAYOUT == LAYOUT_BLOCKED && V % 4 == 0) || RUNS) {
            // (a run's groups of 4 are consecutive cells too)
            const long long e = cell_of<LAYOUT, V>(j0);
            const long long o = tile * S + (e - K);
            if (e >= K && e + 4 <= K + S && o + 4 <= n &&
                (reinterpret_cast<uintptr_t>(qout + o) & 15) == 0) {
                if (FQNM_IN_RANGE(o + 3, n, err))
                    *reinterpret_cast<int4*>(qout + o) =
                        make_int4((int)((unsigned)q[j0] + bias), (int)((unsigned)q[j0 + 1] + bias),
                                  (int)((unsigned)q[j0 + 2] + bias), (int)((unsigned)q[j0 + 3] + bias));
                continue;
            }
#pragma unroll
            for (int j = j0; j < j0 + 4; ++j) {
                const long long ej = e + (j - j0);
                if (ej >= K && ej < K + S) {
                    const long long oj = tile * S + (ej - K);
                    if (oj < n && FQNM_IN_RANGE(oj, n, err)) qout[oj] = (int)((unsigned)q[j] + bias);
                }
            }
        } else {
            const long long e = cell_of<LAYOUT, V>(j0);
            if (e >= K && e < K + S) {
                const long long o = tile * S + (e - K);
                if (o < n && FQNM_IN_RANGE(o, n, err)) qout[o] = (int)((unsigned)q[j0] + bias);
            }
        }
    }
    if (acc > ev.span) atomicOr(err, ERRBIT_RANGE);
}


}  // namespace tb
}  // namespace fqnm
