// k_nd.cu -- the d-dimensional quantised step by directional composition
// (Theorem, Cartesian extension; eqs. nd_transfer_rule, nd_flux_definition).
//
// On a periodic grid (d = 2 or 3, dims[0] fastest) with the same
// one-dimensional transfer rule along every axis:
//   F_{i+e_m/2} = phi+(q_i) + phi-(q_{i+e_m})
//   q_i <- q_i - sum_m (F_{i+e_m/2} - F_{i-e_m/2})
//        = q_i - d (phi+(q_i) - phi-(q_i)) + sum_m (phi+(q_{i-e_m}) - phi-(q_{i+e_m})).
// Kernels: one step per launch (2-D: warps marching y; 3-D: warps streaming
// z slabs), K steps per launch in register tiles (2-D) and K steps per
// launch by pipelined walks (2-D and 3-D).  The 2-D marching kernel sums
// updates in 64-bit and checks them against int32; the others sum in int32,
// which the rule build makes exact by refusing a range within
// 2 d (max|phi+| + max|phi-|) of the int32 limits.
#include "nd.h"
#include "tile_step.cuh"

#include <algorithm>
#include <climits>
#include <type_traits>

namespace fqnm {

namespace {

using tb::EvClosedP;
using tb::EvTableP;
using tb::EvTablePM;
using tb::EvTablePM16;

struct Strides {
    long long n, nx, ny, nz, sy, sz;
};

// ---- marching one-step kernels ---------------------------------------------------
// Each warp owns a strip of 32 consecutive x (lane = column) and walks along
// the slowest axis, keeping the row below and the current row in registers:
// every cell is loaded once, its maps are evaluated once, its x neighbours'
// values arrive by shuffle, and its update is stored once.  The lanes at the
// strip's two ends (and the columns next to the periodic seam) also load and
// evaluate the neighbouring column outside the strip.  Rows go in groups of
// MARCH_G: the group's loads (and edge loads) are issued together, then its
// maps evaluated, then its updates applied, so that MARCH_G loads and
// gathers are in flight per warp.  2-D walks y; 3-D walks z with the block's
// warps on consecutive y rows, exchanging y-edge values through shared
// memory (the block's first and last warp only supply halo rows).

constexpr int MARCH_G = 8;                // rows per group
constexpr int MARCH_ROWS = 32;            // rows of the walk per warp (2-D); a multiple of MARCH_G

struct EdgeCols {
    bool need_l, need_r;
    long long xl, xr;                     // neighbour columns outside the strip (or across the seam)
};

__device__ __forceinline__ EdgeCols edge_cols(long long x, long long nx, int lane)
{
    EdgeCols e;
    e.need_l = lane == 0 || x == 0;
    e.need_r = lane == 31 || x + 1 == nx;
    e.xl = x > 0 ? x - 1 : nx - 1;
    e.xr = x + 1 < nx ? x + 1 : 0;
    return e;
}

template <class Ev>
__global__ void __launch_bounds__(256)
k_march2d(const int* __restrict__ qin, int* __restrict__ qout, long long nx, long long ny,
          long long strips, long long chunks, Ev ev, unsigned* __restrict__ err)
{
    const int lane = threadIdx.x & 31;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (wid >= strips * chunks) return;                 // whole warp
    const long long strip = wid % strips, chunk = wid / strips;
    const long long x = strip * 32 + lane;
    const long long xc = x < nx ? x : nx - 1;           // idle lanes shadow a valid column
    const EdgeCols e = edge_cols(xc, nx, lane);
    const long long y0 = chunk * MARCH_ROWS;
    const long long y1 = y0 + MARCH_ROWS < ny ? y0 + MARCH_ROWS : ny;
    unsigned acc = 0;
    bool over = false;
    int pd, md, qc, pc, mc, plc = 0, mrc = 0;           // row y-1: p; row y: q, p, m, edges
    {
        const long long yd = y0 > 0 ? y0 - 1 : ny - 1;
        ev(__ldg(qin + yd * nx + xc), pd, md, acc);
        qc = __ldg(qin + y0 * nx + xc);
        ev(qc, pc, mc, acc);
        int t;
        if (e.need_l) ev(__ldg(qin + y0 * nx + e.xl), plc, t, acc);
        if (e.need_r) ev(__ldg(qin + y0 * nx + e.xr), t, mrc, acc);
    }
    for (long long y = y0; y < y1; y += MARCH_G) {
        int qn[MARCH_G], pn[MARCH_G], mn[MARCH_G], pl[MARCH_G], mr[MARCH_G];
#pragma unroll
        for (int g = 0; g < MARCH_G; ++g) {             // rows y+1 .. y+G, loads in flight together
            long long r = y + 1 + g;
            if (r >= ny) r -= ny;
            if (r >= ny) r %= ny;
            const int* row = qin + r * nx;
            qn[g] = __ldg(row + xc);
            pl[g] = e.need_l ? __ldg(row + e.xl) : 0;
            mr[g] = e.need_r ? __ldg(row + e.xr) : 0;
        }
#pragma unroll
        for (int g = 0; g < MARCH_G; ++g) {
            int t;
            ev(qn[g], pn[g], mn[g], acc);
            if (e.need_l) ev(pl[g], pl[g], t, acc);
            if (e.need_r) ev(mr[g], t, mr[g], acc);
        }
#pragma unroll
        for (int g = 0; g < MARCH_G; ++g) {             // update row y+g
            const int q0 = g == 0 ? qc : qn[g - 1];
            const int p0 = g == 0 ? pc : pn[g - 1];
            const int m0 = g == 0 ? mc : mn[g - 1];
            const int pdn = g == 0 ? pd : (g == 1 ? pc : pn[g - 2]);
            int l = __shfl_up_sync(0xffffffffu, p0, 1);
            int r = __shfl_down_sync(0xffffffffu, m0, 1);
            if (e.need_l) l = g == 0 ? plc : pl[g - 1];
            if (e.need_r) r = g == 0 ? mrc : mr[g - 1];
            const long long v = (long long)q0 - 2LL * ((long long)p0 - (long long)m0) + l + pdn
                                - (long long)r - (long long)mn[g];
            if (x < nx && y + g < y1 && FQNM_IN_RANGE((y + g) * nx + x, nx * ny, err)) {
                if (v < INT_MIN || v > INT_MAX) over = true;
                qout[(y + g) * nx + x] = (int)v;
            }
        }
        pd = pn[MARCH_G - 2];
        qc = qn[MARCH_G - 1];
        pc = pn[MARCH_G - 1];
        mc = mn[MARCH_G - 1];
        plc = pl[MARCH_G - 1];
        mrc = mr[MARCH_G - 1];
    }
    if (acc > ev.span) atomicOr(err, ERRBIT_RANGE);
    if (over) atomicOr(err, ERRBIT_OVERFLOW);
}

// ---- streaming one-step 3-D kernel ---------------------------------------------
// A warp owns STREAM_OWN = 30 consecutive x on R consecutive y rows and walks
// a chunk of z slabs.  Its 32 lanes hold columns x0-1 .. x0+30 (lanes 1..30
// update; lanes 0 and 31 supply the x neighbours by shuffle), and each lane
// also evaluates the row below and the row above its R rows, so the y
// neighbours stay in the thread.  No shared memory and no barrier: the warps
// are independent.  Slab z+3's states are loaded and slab z+2's maps
// gathered before slab z is updated, so their latency overlaps the update
// (the slabs then shift down one register set).  The update is summed in
// int32: the rule build checks
// that one d-D step from inside the table's range cannot overflow, and a
// state outside that range is a range error anyway (its maps are clamped).
constexpr int STREAM_OWN = 30;

template <class Ev, int R>
__global__ void __launch_bounds__(128)
k_stream3d(const int* __restrict__ qin, int* __restrict__ qout, long long nx, long long ny,
           long long nz, long long strips, long long rowblocks, long long zlen, long long items,
           Ev ev, unsigned* __restrict__ err)
{
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (wid >= items) return;                                  // whole warps
    const int lane = threadIdx.x & 31;
    const long long strip = wid % strips, rb = (wid / strips) % rowblocks;
    const long long zc = wid / (strips * rowblocks);
    const long long xu = strip * STREAM_OWN - 1 + lane;        // unwrapped column
    const long long x = tb::wrap_index(xu, nx);
    const long long y0 = rb * R;
    const long long sz = nx * ny;
    int yo[R + 2];                                             // rows y0-1 .. y0+R
#pragma unroll
    for (int r = 0; r < R + 2; ++r) yo[r] = (int)(tb::wrap_index(y0 - 1 + r, ny) * nx);
    const long long z0 = zc * zlen, z1 = z0 + zlen < nz ? z0 + zlen : nz;
    const bool xown = lane >= 1 && lane <= STREAM_OWN && xu < nx;
    unsigned acc = 0;
    auto load = [&](long long z, int (&q)[R + 2]) {
        const int* b = qin + tb::wrap_index(z, nz) * sz + x;
#pragma unroll
        for (int r = 0; r < R + 2; ++r) q[r] = __ldg(b + yo[r]);
    };
    auto eval = [&](const int (&q)[R + 2], int (&p)[R + 2], int (&m)[R + 2]) {
#pragma unroll
        for (int r = 0; r < R + 2; ++r) ev(q[r], p[r], m[r], acc);
    };
    int pp[R];                                                 // p of slab z-1, rows 0..R-1
    int qc[R + 2], pc[R + 2], mc[R + 2];                       // slab z
    int qn[R + 2], pn[R + 2], mn[R + 2];                       // slab z+1
    int qf[R + 2];                                             // slab z+2, loaded
    {
        int qd[R + 2], pd[R + 2], md[R + 2];
        load(z0 - 1, qd);
        load(z0, qc);
        load(z0 + 1, qn);
        load(z0 + 2, qf);
        eval(qd, pd, md);
        eval(qc, pc, mc);
        eval(qn, pn, mn);
#pragma unroll
        for (int r = 0; r < R; ++r) pp[r] = pd[r + 1];
    }
    for (long long z = z0; z < z1; ++z) {
        int qg[R + 2], pf[R + 2], mf[R + 2];
        if (z + 3 <= z1) load(z + 3, qg);                      // slab z+3: needed from z+2 on
        if (z + 2 <= z1) eval(qf, pf, mf);                     // slab z+2's maps
#pragma unroll
        for (int r = 0; r < R; ++r) {                          // update slab z, row y0 + r
            const int pcr = pc[r + 1], mcr = mc[r + 1];
            const int pl = __shfl_up_sync(0xffffffffu, pcr, 1);     // x - 1
            const int mr = __shfl_down_sync(0xffffffffu, mcr, 1);   // x + 1
            const int v = qc[r + 1] - 3 * (pcr - mcr) + pl + pc[r] + pp[r] - mr - mc[r + 2]
                          - mn[r + 1];
            const long long o = z * sz + (long long)yo[r + 1] + x;
            if (xown && y0 + r < ny && FQNM_IN_RANGE(o, nz * sz, err)) qout[o] = v;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) pp[r] = pc[r + 1];
#pragma unroll
        for (int r = 0; r < R + 2; ++r) {
            qc[r] = qn[r]; pc[r] = pn[r]; mc[r] = mn[r];
            qn[r] = qf[r]; pn[r] = pf[r]; mn[r] = mf[r];
            qf[r] = qg[r];
        }
    }
    if (acc > ev.span) atomicOr(err, ERRBIT_RANGE);
}

// The same walk for the packed table (both maps as int16 halves of one
// word): each cell's maps stay packed in one register and are unpacked where
// they are used, so a row of the pipeline holds 8 registers instead of 11;
// with 7 rows per warp and 32-bit offsets (a grid holds fewer than 2^31
// cells) four blocks fit an SM.
template <int R>
__global__ void __launch_bounds__(128, 4)
k_stream3d_pk(const int* __restrict__ qin, int* __restrict__ qout, int nx, int ny, int nz,
              int strips, int rowblocks, int zlen, int items, tb::EvTablePM16 ev,
              unsigned* __restrict__ err)
{
    const int wid = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    if (wid >= items) return;                                  // whole warps
    const int lane = threadIdx.x & 31;
    const int strip = wid % strips, rb = (wid / strips) % rowblocks;
    const int zc = wid / (strips * rowblocks);
    const int xu = strip * STREAM_OWN - 1 + lane;              // unwrapped column
    const int x = xu < 0 ? xu + nx : xu >= nx ? xu - nx : xu;  // |xu| < 2 nx
    const int y0 = rb * R;
    const int sz = nx * ny;
    int yo[R + 2];                                             // rows y0-1 .. y0+R
#pragma unroll
    for (int r = 0; r < R + 2; ++r) {
        int y = y0 - 1 + r;
        y = y < 0 ? y + ny : y;
        y = y >= ny ? y % ny : y;                              // a ragged block's rows wrap
        yo[r] = y * nx + x;
    }
    const int z0 = zc * zlen, z1 = z0 + zlen < nz ? z0 + zlen : nz;
    unsigned own = 0;                                          // bit r: row y0 + r is ours
    if (lane >= 1 && lane <= STREAM_OWN && xu < nx) {
#pragma unroll
        for (int r = 0; r < R; ++r) own |= (unsigned)(y0 + r < ny) << r;
    }
    unsigned acc = 0;
    auto slab = [&](int z) { z = z < 0 ? z + nz : z; return (z >= nz ? z - nz : z) * sz; };
    auto load = [&](int z, int (&q)[R + 2]) {
        const int* b = qin + slab(z);
#pragma unroll
        for (int r = 0; r < R + 2; ++r) q[r] = __ldg(b + yo[r]);
    };
    auto gather = [&](const int (&q)[R + 2], int (&w)[R + 2]) {
#pragma unroll
        for (int r = 0; r < R + 2; ++r) {
            const unsigned i = (unsigned)(q[r] - ev.lo);
            acc = max(acc, i);
            w[r] = __ldg(ev.tab + min(i, ev.span));            // never outside the table
        }
    };
    auto P = [](int w) { return (int)(short)(w & 0xffff); };   // phi+: the low half
    auto M = [](int w) { return w >> 16; };                    // phi-: the high half
    int wp[R];                                                 // slab z-1, rows 0..R-1
    int qc[R + 2], wc[R + 2];                                  // slab z
    int qn[R + 2], wn[R + 2];                                  // slab z+1
    int qf[R + 2];                                             // slab z+2, loaded
    {
        int qd[R + 2], wd[R + 2];
        load(z0 - 1, qd);
        load(z0, qc);
        load(z0 + 1, qn);
        load(z0 + 2, qf);
        gather(qd, wd);
        gather(qc, wc);
        gather(qn, wn);
#pragma unroll
        for (int r = 0; r < R; ++r) wp[r] = wd[r + 1];
    }
    for (int z = z0; z < z1; ++z) {
        int qg[R + 2], wf[R + 2];
        if (z + 3 <= z1) load(z + 3, qg);                      // slab z+3: needed from z+2 on
        if (z + 2 <= z1) gather(qf, wf);                       // slab z+2's maps
        int* const o = qout + z * sz;
#pragma unroll
        for (int r = 0; r < R; ++r) {                          // update slab z, row y0 + r
            const int pcr = P(wc[r + 1]), mcr = M(wc[r + 1]);
            const int pl = __shfl_up_sync(0xffffffffu, pcr, 1);     // x - 1
            const int mr = __shfl_down_sync(0xffffffffu, mcr, 1);   // x + 1
            const int v = qc[r + 1] - 3 * (pcr - mcr) + pl + P(wc[r]) + P(wp[r]) - mr
                          - M(wc[r + 2]) - M(wn[r + 1]);
            if (((own >> r) & 1) && FQNM_IN_RANGE((long long)z * sz + yo[r + 1],
                                                  (long long)nz * sz, err))
                o[yo[r + 1]] = v;
        }
#pragma unroll
        for (int r = 0; r < R; ++r) wp[r] = wc[r + 1];
#pragma unroll
        for (int r = 0; r < R + 2; ++r) {
            qc[r] = qn[r]; wc[r] = wn[r];
            qn[r] = qf[r]; wn[r] = wf[r];
            qf[r] = qg[r];
        }
    }
    if (acc > ev.span) atomicOr(err, ERRBIT_RANGE);
}

constexpr int STREAM_R_PK = 7;
constexpr int STREAM_R = 8;

template <class Ev>
cudaError_t launch_stream3d(const Ev& ev, const int32_t* qin, int32_t* qout, const NdGrid& g,
                            unsigned* err, cudaStream_t st)
{
    const long long nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
    constexpr bool packed = std::is_same<Ev, tb::EvTablePM16>::value;
    constexpr int R = packed ? STREAM_R_PK : STREAM_R;
    const long long strips = (nx + STREAM_OWN - 1) / STREAM_OWN;
    const long long rowblocks = (ny + R - 1) / R;
    // Blocks of four warps run in waves of `slots` (the SMs times the blocks
    // each holds), and a warp's chunk of c slabs costs c + 2 slab times (the
    // pipeline loads and evaluates the slab below and the slab above the
    // chunk): take the chunk length (4 slabs at least) whose waves x slab
    // times is least.
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) {
        if constexpr (packed)
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream3d_pk<R>, 128, 0);
        else
            e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_stream3d<Ev, STREAM_R>, 128, 0);
    }
    if (e != cudaSuccess) return e;
    const long long slots = (long long)sms * (per_sm > 0 ? per_sm : 1);
    const long long cols = strips * rowblocks;
    long long zlen = nz, best = -1;
    for (long long c = 1; c <= nz && c <= 1024; ++c) {
        const long long len = (nz + c - 1) / c, chunks = (nz + len - 1) / len;
        if (len < 4 && c > 1) break;
        const long long blocks = (cols * chunks + 3) / 4;
        const long long cost = ((blocks + slots - 1) / slots) * (len + 2);
        if (best < 0 || cost < best) { best = cost; zlen = len; }
    }
    const long long chunks = (nz + zlen - 1) / zlen;
    const long long items = cols * chunks;
    const long long blocks = (items * 32 + 127) / 128;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    if constexpr (packed)   // every count below fits int: the grid holds < 2^31 cells
        k_stream3d_pk<R><<<(unsigned)blocks, 128, 0, st>>>(qin, qout, (int)nx, (int)ny, (int)nz,
                                                           (int)strips, (int)rowblocks, (int)zlen,
                                                           (int)items, ev, err);
    else
        k_stream3d<Ev, STREAM_R><<<(unsigned)blocks, 128, 0, st>>>(qin, qout, nx, ny, nz, strips,
                                                                   rowblocks, zlen, items, ev, err);
    note_launches();
    return cudaGetLastError();
}

template <class Ev>
cudaError_t dispatch_march(const Ev& ev, const int32_t* qin, int32_t* qout, const NdGrid& g,
                           unsigned* err, cudaStream_t st)
{
    const long long nx = g.dims[0], ny = g.dims[1];
    const long long strips = (nx + 31) / 32;
    if (g.d == 2) {
        const long long chunks = (ny + MARCH_ROWS - 1) / MARCH_ROWS;
        const long long warps = strips * chunks;
        const long long blocks = (warps + 7) / 8;
        if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
        k_march2d<<<(unsigned)blocks, 256, 0, st>>>(qin, qout, nx, ny, strips, chunks, ev, err);
    } else {
        return launch_stream3d(ev, qin, qout, g, err, st);
    }
    note_launches();
    return cudaGetLastError();
}

// ---- 2-D temporal blocking ------------------------------------------------------
// A block of WX x WY warps holds a TX x TY tile (TX = 32 WX along x, TY =
// VY WY along y) in registers: lane l of warp (wx, wy) holds column
// 32 wx + l, rows VY wy .. VY wy + VY - 1.  The tile starts K cells left of
// and below its output region and applies K steps; the cells whose
// dependency cone (within K in x and in y) stayed inside the tile are exact
// and are written: (TX - 2K) x (TY - 2K) per tile.
//   x neighbours: shuffles inside a warp; a warp's edge columns (p of lane
//     31, m of lane 0) through shared memory to the warps left and right;
//   y neighbours: registers inside a thread; a warp's edge rows (p of the top
//     row, m of the bottom row) through shared memory to the warps above and
//     below.
// Edge arrays are double-buffered: one barrier per step.  The tile's outer
// cells use a ghost copy of themselves (values outside the exact region,
// kept on a valid scheme so they cannot trip the range guard).

template <int VY, int WX, int WY>
struct Tile2dSmem {
    int xp[2][WX * WY][VY];        // p of lane 31, per row
    int xm[2][WX * WY][VY];        // m of lane 0, per row
    int yp[2][WX * WY][32];        // p of the top row, per lane
    int ym[2][WX * WY][32];        // m of the bottom row, per lane
};

struct Tile2dArgs {
    long long nx, ny;
    int K;
    long long SX, SY;              // output cells per tile along x and y
    long long tiles_x;
};

using tb::wrap_index;           // one conditional add or subtract; a modulo only for tiny grids

template <class Ev, int VY, int WX, int WY>
__global__ void __launch_bounds__(32 * WX * WY)
k_step2d_tb(const int* __restrict__ qin, int* __restrict__ qout, Tile2dArgs a, Ev ev,
            unsigned* __restrict__ err)
{
    __shared__ Tile2dSmem<VY, WX, WY> sm;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int wx = w % WX, wy = w / WX;
    const long long tx = blockIdx.x % a.tiles_x, ty = blockIdx.x / a.tiles_x;
    const long long x0 = tx * a.SX - a.K, y0 = ty * a.SY - a.K;
    const int ex = 32 * wx + lane;                      // tile column
    const long long gx = wrap_index(x0 + ex, a.nx);
    int q[VY];
#pragma unroll
    for (int j = 0; j < VY; ++j)
    {
        const long long gi = wrap_index(y0 + VY * wy + j, a.ny) * a.nx + gx;
        q[j] = FQNM_IN_RANGE(gi, a.nx * a.ny, err) ? __ldg(qin + gi) : 0;
    }

    unsigned acc = 0;
    const int wl = wx > 0 ? w - 1 : w, wr = wx < WX - 1 ? w + 1 : w;
    const int wd = wy > 0 ? w - WX : w, wu = wy < WY - 1 ? w + WX : w;
    for (int s = 0; s < a.K; ++s) {
        int p[VY], m[VY];
#pragma unroll
        for (int j = 0; j < VY; ++j) ev(q[j], p[j], m[j], acc);
        const int b = s & 1;
        if (lane == 31)
#pragma unroll
            for (int j = 0; j < VY; ++j) sm.xp[b][w][j] = p[j];
        if (Ev::HAS_M && lane == 0)
#pragma unroll
            for (int j = 0; j < VY; ++j) sm.xm[b][w][j] = m[j];
        sm.yp[b][w][lane] = p[VY - 1];
        if (Ev::HAS_M) sm.ym[b][w][lane] = m[0];
        __syncthreads();
        // neighbours across warp edges (own value at the tile's outer edge)
        const int pd0 = wy > 0 ? sm.yp[b][wd][lane] : p[0];
        const int muT = (Ev::HAS_M && wy < WY - 1) ? sm.ym[b][wu][lane] : m[VY - 1];
#pragma unroll
        for (int j = 0; j < VY; ++j) {
            int pl = __shfl_up_sync(0xffffffffu, p[j], 1);
            if (lane == 0) pl = wx > 0 ? sm.xp[b][wl][j] : p[j];
            const int pd = j > 0 ? p[j - 1] : pd0;
            int d = pl + pd - 2 * p[j];
            if (Ev::HAS_M) {
                int mr = __shfl_down_sync(0xffffffffu, m[j], 1);
                if (lane == 31) mr = wx < WX - 1 ? sm.xm[b][wr][j] : m[j];
                const int mu = j < VY - 1 ? m[j + 1] : muT;
                d += 2 * m[j] - mr - mu;
            }
            q[j] += d;
        }
    }
    // the exact region: tile cells [K, K + SX) x [K, K + SY)
    if (ex >= a.K && ex < a.K + a.SX) {
        const long long ox = tx * a.SX + (ex - a.K);
        if (ox < a.nx) {
#pragma unroll
            for (int j = 0; j < VY; ++j) {
                const int ey = VY * wy + j;
                if (ey < a.K || ey >= a.K + a.SY) continue;
                const long long oy = ty * a.SY + (ey - a.K);
                if (oy < a.ny && FQNM_IN_RANGE(oy * a.nx + ox, a.nx * a.ny, err))
                    qout[oy * a.nx + ox] = q[j];
            }
        }
    }
    if (acc > ev.span) atomicOr(err, ERRBIT_RANGE);
}

template <class Ev, int VY, int WX, int WY>
cudaError_t launch_2d(const Ev& ev, const int32_t* qin, int32_t* qout, const NdGrid& g, int K,
                      unsigned* err, cudaStream_t st)
{
    constexpr int TX = 32 * WX, TY = VY * WY;
    if (2 * K >= TX || 2 * K >= TY) return cudaErrorInvalidValue;
    Tile2dArgs a;
    a.nx = g.dims[0];
    a.ny = g.dims[1];
    a.K = K;
    a.SX = TX - 2 * K;
    a.SY = TY - 2 * K;
    a.tiles_x = (a.nx + a.SX - 1) / a.SX;
    const long long tiles_y = (a.ny + a.SY - 1) / a.SY;
    const long long blocks = a.tiles_x * tiles_y;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_step2d_tb<Ev, VY, WX, WY><<<(unsigned)blocks, 32 * WX * WY, 0, st>>>(qin, qout, a, ev, err);
    note_launches();
    return cudaGetLastError();
}

template <class Ev>
cudaError_t dispatch_2d(const Ev& ev, const NdPlan& p, const int32_t* qin, int32_t* qout,
                        const NdGrid& g, int K, unsigned* err, cudaStream_t st)
{
    switch (p.shape) {
    case ND_TILE_64x64: return launch_2d<Ev, 16, 2, 4>(ev, qin, qout, g, K, err, st);
    case ND_TILE_128x64: return launch_2d<Ev, 16, 4, 4>(ev, qin, qout, g, K, err, st);
    case ND_TILE_64x32: return launch_2d<Ev, 8, 2, 4>(ev, qin, qout, g, K, err, st);
    case ND_TILE_128x32: return launch_2d<Ev, 8, 4, 4>(ev, qin, qout, g, K, err, st);
    case ND_TILE_32x128: return launch_2d<Ev, 16, 1, 8>(ev, qin, qout, g, K, err, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---- 2-D temporal walk ------------------------------------------------------------
// A warp holds a strip of 64 columns (lane l: columns 2l and 2l+1) and walks
// y, applying K steps as a skewed pipeline: at tick i, level l produces row
// i - 2l (level 0: the loaded row i) from level l-1's last three rows
// i-2l-1, i-2l, i-2l+1, all produced on earlier ticks.  The K levels of a
// tick are therefore independent of one another (2K independent table
// gathers per lane per tick), which hides the gather latency inside the
// warp.  Inside a lane the two columns see each other directly; across lanes
// one shuffle per cell.  The strip's two outer columns take ghost copies of
// themselves, so after K levels columns [K, 64-K) are exact, and rows
// [y0, y1) are exact once the walk has read rows y0-K .. y1+K-1.  No shared
// memory and no barrier; row loads are issued WALK_AHEAD rows ahead.

constexpr int WALK_COLS = 64;
constexpr int WALK_AHEAD = 4;             // rows loaded ahead of the walk

template <class Ev, int K>
__global__ void __launch_bounds__(256)
k_walk2d(const int* __restrict__ qin, int* __restrict__ qout, long long nx, long long ny,
         long long strips, long long chunks, long long R, Ev ev, unsigned* __restrict__ err)
{
    constexpr int SW = WALK_COLS - 2 * K;               // output columns per strip
    const int lane = threadIdx.x & 31;
    const long long wid = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5;
    if (wid >= strips * chunks) return;                 // whole warp
    const long long strip = wid % strips, chunk = wid / strips;
    const long long xs = strip * SW - K;                // column of strip index 0
    const long long xa = wrap_index(xs + 2 * lane, nx), xb = wrap_index(xs + 2 * lane + 1, nx);
    const long long y0 = chunk * R, y1 = y0 + R < ny ? y0 + R : ny;
    unsigned acc = 0;

    // per level l < K: its last three rows, two columns: up (q, p, m) = the
    // newest, center (q, p, m), down (p)
    int qU[K][2], pU[K][2], mU[K][2], qC[K][2], pC[K][2], mC[K][2], pD[K][2];
    {
        const int* row = qin + wrap_index(y0 - K - 1, ny) * nx;
        const int a = __ldg(row + xa), b = __ldg(row + xb);
        int pa, ma, pb, mb;
        ev(a, pa, ma, acc);
        ev(b, pb, mb, acc);
#pragma unroll
        for (int l = 0; l < K; ++l) {                   // ghosts: never reach an output
            qU[l][0] = qC[l][0] = a; pU[l][0] = pC[l][0] = pD[l][0] = pa; mU[l][0] = mC[l][0] = ma;
            qU[l][1] = qC[l][1] = b; pU[l][1] = pC[l][1] = pD[l][1] = pb; mU[l][1] = mC[l][1] = mb;
        }
    }
    int fa[WALK_AHEAD], fb[WALK_AHEAD];
#pragma unroll
    for (int a = 0; a < WALK_AHEAD; ++a) {
        const int* row = qin + wrap_index(y0 - K + a, ny) * nx;
        fa[a] = __ldg(row + xa);
        fb[a] = __ldg(row + xb);
    }
    const int ca = 2 * lane, cb = 2 * lane + 1;          // strip column indices
    const long long oa = strip * SW + (ca - K), ob = strip * SW + (cb - K);
    const bool wa = ca >= K && ca < WALK_COLS - K && oa < nx;
    const bool wb = cb >= K && cb < WALK_COLS - K && ob < nx;
    // level K row i - 2K lands in [y0, y1) for i in [y0 + 2K, y1 + 2K)
    for (long long i = y0 - K; i < y1 + 2 * K; ++i) {
        // new rows of every level this tick, from the windows as they stood
        int nq[K + 1][2];
        nq[0][0] = fa[0];
        nq[0][1] = fb[0];
#pragma unroll
        for (int a = 0; a + 1 < WALK_AHEAD; ++a) {
            fa[a] = fa[a + 1];
            fb[a] = fb[a + 1];
        }
        {
            const int* row = qin + wrap_index(i + WALK_AHEAD, ny) * nx;
            fa[WALK_AHEAD - 1] = __ldg(row + xa);
            fb[WALK_AHEAD - 1] = __ldg(row + xb);
        }
#pragma unroll
        for (int l = 0; l < K; ++l) {                   // level l+1 from level l's window
            int pl = __shfl_up_sync(0xffffffffu, pC[l][1], 1);
            int mr = __shfl_down_sync(0xffffffffu, mC[l][0], 1);
            if (lane == 0) pl = pC[l][0];               // ghost of the strip's first column
            if (lane == 31) mr = mC[l][1];              // ghost of the strip's last column
            nq[l + 1][0] = qC[l][0] - 2 * (pC[l][0] - mC[l][0]) + pl + pD[l][0] - mC[l][1] - mU[l][0];
            nq[l + 1][1] = qC[l][1] - 2 * (pC[l][1] - mC[l][1]) + pC[l][0] + pD[l][1] - mr - mU[l][1];
        }
        // shift every level's window by its new row (levels 0 .. K-1), evaluating it
#pragma unroll
        for (int l = 0; l < K; ++l) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                pD[l][c] = pC[l][c];
                qC[l][c] = qU[l][c];
                pC[l][c] = pU[l][c];
                mC[l][c] = mU[l][c];
                qU[l][c] = nq[l][c];
                ev(nq[l][c], pU[l][c], mU[l][c], acc);
            }
        }
        const long long r = i - 2 * K;                  // level-K row of this tick
        if (r >= y0 && r < y1) {
            if (wa && FQNM_IN_RANGE(r * nx + oa, nx * ny, err)) qout[r * nx + oa] = nq[K][0];
            if (wb && FQNM_IN_RANGE(r * nx + ob, nx * ny, err)) qout[r * nx + ob] = nq[K][1];
        }
    }
    if (acc > ev.span) atomicOr(err, ERRBIT_RANGE);
}

// Rows per warp R (at least 4K: a walk re-reads 2K halo rows and fills its
// pipeline for K more ticks per R rows) chosen against the waves the grid
// needs; see the cost rule below.
template <class Ev, int K>
cudaError_t launch_walk(const Ev& ev, const int32_t* qin, int32_t* qout, const NdGrid& g,
                        unsigned* err, cudaStream_t st)
{
    const long long nx = g.dims[0], ny = g.dims[1];
    const long long strips = (nx + (WALK_COLS - 2 * K) - 1) / (WALK_COLS - 2 * K);
    // One warp per block: the warps are independent, and the SMs then hold
    // as many as their registers allow.  A warp of R rows takes R + 3K ticks
    // and the warps run in waves of `slots`: take the chunk count whose
    // waves x ticks is least, with R >= 4K (the 3K fill ticks of shorter
    // walks cost more than the waves they save: 1024^2 ran 28 % slower at
    // R = 7 than at R = 16).
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk2d<Ev, K>, 32, 0);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)sms * (per_sm > 0 ? per_sm : 1);
    long long R = ny, best = -1;
    for (long long c = 1; c <= ny && c <= 2048; ++c) {
        const long long r = (ny + c - 1) / c, ch = (ny + r - 1) / r;
        if (c > 1 && r < 4 * K) break;                  // r only falls as c grows
        const long long cost = ((strips * ch + slots - 1) / slots) * (r + 3 * K);
        if (best < 0 || cost < best) { best = cost; R = r; }
    }
    const long long chunks = (ny + R - 1) / R;
    const long long blocks = strips * chunks;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_walk2d<Ev, K><<<(unsigned)blocks, 32, 0, st>>>(qin, qout, nx, ny, strips, chunks, R, ev, err);
    note_launches();
    return cudaGetLastError();
}

template <class Ev>
cudaError_t dispatch_walk(const Ev& ev, int K, const int32_t* qin, int32_t* qout,
                          const NdGrid& g, unsigned* err, cudaStream_t st)
{
    switch (K) {
    case 1: return launch_walk<Ev, 1>(ev, qin, qout, g, err, st);
    case 2: return launch_walk<Ev, 2>(ev, qin, qout, g, err, st);
    case 3: return launch_walk<Ev, 3>(ev, qin, qout, g, err, st);
    case 4: return launch_walk<Ev, 4>(ev, qin, qout, g, err, st);
    case 6: return launch_walk<Ev, 6>(ev, qin, qout, g, err, st);
    case 8: return launch_walk<Ev, 8>(ev, qin, qout, g, err, st);
    default: return cudaErrorInvalidValue;
    }
}

// ---- 3-D temporal walk ------------------------------------------------------------
// A block of ROWS warps holds a 64-column x strip (two columns per lane) of
// ROWS consecutive y rows (one per warp) and walks z with K
// steps in the skewed pipeline of the 2-D walk: at tick i level l produces
// slice i - 2l from level l-1's slices i-2l-1 .. i-2l+1 (z neighbours in
// registers), x neighbours within the warp, y neighbours from the warps
// above and below through shared memory.  The levels of a tick are
// independent, so one barrier per tick serves all of them (double-buffered
// by tick parity).  Outer columns and the block's first and last rows take
// ghost copies of themselves: columns [K, 64-K) and rows [K, ROWS-K) are
// exact after K levels.  ROWS = 32 (1024 threads, at most 64 registers)
// for K <= 2, where the y halo then costs 1/7 instead of 1/3.

template <int K, int ROWS>
struct Walk3Smem {
    int p[2][K][ROWS][WALK_COLS];         // level l's centre slice: p
    int m[2][K][ROWS][WALK_COLS];         // and m
};

template <class Ev, int K, int ROWS>
__global__ void __launch_bounds__(32 * ROWS)
k_walk3d(const int* __restrict__ qin, int* __restrict__ qout, long long nx, long long ny,
         long long nz, long long strips, long long rowblocks, long long chunks, long long R, Ev ev,
         unsigned* __restrict__ err)
{
    constexpr int SW = WALK_COLS - 2 * K, SR = ROWS - 2 * K;
    extern __shared__ __align__(16) unsigned char walk3_raw[];
    Walk3Smem<K, ROWS>& sm = *reinterpret_cast<Walk3Smem<K, ROWS>*>(walk3_raw);
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const long long b = blockIdx.x;
    const long long strip = b % strips, rb = (b / strips) % rowblocks, chunk = b / (strips * rowblocks);
    const long long xs = strip * SW - K;
    const long long xa = wrap_index(xs + 2 * lane, nx), xb = wrap_index(xs + 2 * lane + 1, nx);
    const long long yr = rb * SR - K + w;                 // this warp's row (unwrapped)
    const long long y = wrap_index(yr, ny);
    const long long sy = nx, sz = nx * ny;
    const long long z0 = chunk * R, z1 = z0 + R < nz ? z0 + R : nz;
    const int wd = w > 0 ? w - 1 : w, wu = w < ROWS - 1 ? w + 1 : w;
    unsigned acc = 0;

    int qU[K][2], pU[K][2], mU[K][2], qC[K][2], pC[K][2], mC[K][2], pD[K][2];
    {
        const int* row = qin + wrap_index(z0 - K - 1, nz) * sz + y * sy;
        const int a = __ldg(row + xa), c = __ldg(row + xb);
        int pa, ma, pc, mc;
        ev(a, pa, ma, acc);
        ev(c, pc, mc, acc);
#pragma unroll
        for (int l = 0; l < K; ++l) {
            qU[l][0] = qC[l][0] = a; pU[l][0] = pC[l][0] = pD[l][0] = pa; mU[l][0] = mC[l][0] = ma;
            qU[l][1] = qC[l][1] = c; pU[l][1] = pC[l][1] = pD[l][1] = pc; mU[l][1] = mC[l][1] = mc;
        }
    }
    int fa[WALK_AHEAD], fb[WALK_AHEAD];
#pragma unroll
    for (int a = 0; a < WALK_AHEAD; ++a) {
        const int* row = qin + wrap_index(z0 - K + a, nz) * sz + y * sy;
        fa[a] = __ldg(row + xa);
        fb[a] = __ldg(row + xb);
    }
    const int ca = 2 * lane, cb = 2 * lane + 1;
    const long long oa = strip * SW + (ca - K), ob = strip * SW + (cb - K);
    const bool rowok = w >= K && w < ROWS - K && yr < ny && yr >= 0;
    const bool wa = rowok && ca >= K && ca < WALK_COLS - K && oa < nx;
    const bool wb = rowok && cb >= K && cb < WALK_COLS - K && ob < nx;
    int par = 0;
    for (long long i = z0 - K; i < z1 + 2 * K; ++i, par ^= 1) {
        int nq[K + 1][2];
        nq[0][0] = fa[0];
        nq[0][1] = fb[0];
#pragma unroll
        for (int a = 0; a + 1 < WALK_AHEAD; ++a) {
            fa[a] = fa[a + 1];
            fb[a] = fb[a + 1];
        }
        {
            const int* row = qin + wrap_index(i + WALK_AHEAD, nz) * sz + y * sy;
            fa[WALK_AHEAD - 1] = __ldg(row + xa);
            fb[WALK_AHEAD - 1] = __ldg(row + xb);
        }
        // publish every level's centre slice for the rows above and below
#pragma unroll
        for (int l = 0; l < K; ++l) {
            sm.p[par][l][w][ca] = pC[l][0];
            sm.p[par][l][w][cb] = pC[l][1];
            sm.m[par][l][w][ca] = mC[l][0];
            sm.m[par][l][w][cb] = mC[l][1];
        }
        __syncthreads();
#pragma unroll
        for (int l = 0; l < K; ++l) {                   // level l+1 from level l's window
            int pl = __shfl_up_sync(0xffffffffu, pC[l][1], 1);
            int mr = __shfl_down_sync(0xffffffffu, mC[l][0], 1);
            if (lane == 0) pl = pC[l][0];
            if (lane == 31) mr = mC[l][1];
            const int pya = sm.p[par][l][wd][ca], pyb = sm.p[par][l][wd][cb];   // row below
            const int mya = sm.m[par][l][wu][ca], myb = sm.m[par][l][wu][cb];   // row above
            nq[l + 1][0] = qC[l][0] - 3 * (pC[l][0] - mC[l][0]) + pl + pya + pD[l][0]
                           - mC[l][1] - mya - mU[l][0];
            nq[l + 1][1] = qC[l][1] - 3 * (pC[l][1] - mC[l][1]) + pC[l][0] + pyb + pD[l][1]
                           - mr - myb - mU[l][1];
        }
#pragma unroll
        for (int l = 0; l < K; ++l) {
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                pD[l][c] = pC[l][c];
                qC[l][c] = qU[l][c];
                pC[l][c] = pU[l][c];
                mC[l][c] = mU[l][c];
                qU[l][c] = nq[l][c];
                ev(nq[l][c], pU[l][c], mU[l][c], acc);
            }
        }
        const long long r = i - 2 * K;                  // level-K slice of this tick
        if (r >= z0 && r < z1) {
            const long long base = r * sz + y * sy;
            if (wa && FQNM_IN_RANGE(base + oa, nz * sz, err)) qout[base + oa] = nq[K][0];
            if (wb && FQNM_IN_RANGE(base + ob, nz * sz, err)) qout[base + ob] = nq[K][1];
        }
    }
    if (acc > ev.span) atomicOr(err, ERRBIT_RANGE);
}

template <class Ev, int K, int ROWS>
cudaError_t launch_walk3(const Ev& ev, const int32_t* qin, int32_t* qout, const NdGrid& g,
                         unsigned* err, cudaStream_t st)
{
    const long long nx = g.dims[0], ny = g.dims[1], nz = g.dims[2];
    const long long strips = (nx + (WALK_COLS - 2 * K) - 1) / (WALK_COLS - 2 * K);
    const long long rowblocks = (ny + (ROWS - 2 * K) - 1) / (ROWS - 2 * K);
    // Blocks run in waves of `slots` (the SMs times the blocks each holds)
    // and a block of R slices takes R + 3K ticks: take the chunk count whose
    // waves x ticks is least.
    constexpr int smem = (int)sizeof(Walk3Smem<K, ROWS>);
    // opt in above the 48 KB default (a per-device attribute: set it for the
    // current device at every launch)
    cudaError_t e = cudaFuncSetAttribute(k_walk3d<Ev, K, ROWS>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    int dev = 0, sms = 0, per_sm = 0;
    if (e == cudaSuccess) e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_walk3d<Ev, K, ROWS>,
                                                          32 * ROWS, smem);
    if (e != cudaSuccess) return e;
    const long long slots = (long long)sms * (per_sm > 0 ? per_sm : 1);
    const long long xy = strips * rowblocks;
    long long R = nz, best = -1;
    for (long long c = 1; c <= nz && c <= 256; ++c) {
        const long long r = (nz + c - 1) / c, chunks = (nz + r - 1) / r;
        const long long cost = ((xy * chunks + slots - 1) / slots) * (r + 3 * K);
        if (best < 0 || cost < best) { best = cost; R = r; }
    }
    const long long chunks = (nz + R - 1) / R;
    const long long blocks = strips * rowblocks * chunks;
    if (blocks > 0x7fffffffLL) return cudaErrorInvalidValue;
    k_walk3d<Ev, K, ROWS><<<(unsigned)blocks, 32 * ROWS, smem, st>>>(qin, qout, nx, ny, nz, strips,
                                                                     rowblocks, chunks, R, ev, err);
    note_launches();
    return cudaGetLastError();
}

template <class Ev>
cudaError_t dispatch_walk3(const Ev& ev, int K, const int32_t* qin, int32_t* qout,
                           const NdGrid& g, unsigned* err, cudaStream_t st)
{
    switch (K) {
    case 1: return launch_walk3<Ev, 1, 32>(ev, qin, qout, g, err, st);
    case 2: return launch_walk3<Ev, 2, 32>(ev, qin, qout, g, err, st);
    case 3: return launch_walk3<Ev, 3, 16>(ev, qin, qout, g, err, st);
    case 4: return launch_walk3<Ev, 4, 16>(ev, qin, qout, g, err, st);
    default: return cudaErrorInvalidValue;
    }
}

constexpr int IBLOCK = 256;

__device__ __forceinline__ long long warp_sum64(long long v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(IBLOCK)
k_invariants_nd(const int* __restrict__ q, const int* __restrict__ other, Strides g, int d,
                long long* acc)
{
    __shared__ long long sh[3][IBLOCK / 32];
    long long mass = 0, tv = 0, l1 = 0;
    const long long x = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (x < g.nx) {
        const long long xr = x + 1 < g.nx ? x + 1 : 0;
        for (long long z = blockIdx.z; z < g.nz; z += gridDim.z) {
            const long long zr = z + 1 < g.nz ? z + 1 : 0;
            for (long long y = blockIdx.y; y < g.ny; y += gridDim.y) {
                const long long yr = y + 1 < g.ny ? y + 1 : 0;
                const long long row = z * g.sz + y * g.sy;
                const long long v = q[row + x];
                mass += v;
                long long w = q[row + xr];
                tv += w > v ? w - v : v - w;
                if (d >= 2) {
                    w = q[z * g.sz + yr * g.sy + x];
                    tv += w > v ? w - v : v - w;
                }
                if (d >= 3) {
                    w = q[zr * g.sz + y * g.sy + x];
                    tv += w > v ? w - v : v - w;
                }
                if (other) {
                    const long long o = other[row + x];
                    l1 += o > v ? o - v : v - o;
                }
            }
        }
    }
    mass = warp_sum64(mass);
    tv = warp_sum64(tv);
    l1 = warp_sum64(l1);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) { sh[0][w] = mass; sh[1][w] = tv; sh[2][w] = l1; }
    __syncthreads();
    if (w == 0) {
        for (int k = 0; k < 3; ++k) {
            long long t = lane < IBLOCK / 32 ? sh[k][lane] : 0;
            t = warp_sum64(t);
            if (lane == 0 && t != 0) atomicAdd((unsigned long long*)(acc + k), (unsigned long long)t);
        }
    }
}

}  // namespace

cudaError_t launch_step_nd(const RuleView& r, const int32_t* qin, int32_t* qout, const NdGrid& g,
                           unsigned* err, cudaStream_t st)
{
    if (g.d < 2 || g.d > 3 || g.cells() <= 0) return cudaErrorInvalidValue;
    if (r.evaluator == EVAL_CLOSED_FORM && !r.has_m)
        return dispatch_march(EvClosedP{r.cf, r.lo, r.span}, qin, qout, g, err, st);
    if (!r.has_m) return dispatch_march(EvTableP{r.tabp, r.lo, r.span}, qin, qout, g, err, st);
    if (r.tab16) return dispatch_march(EvTablePM16{r.tab16, r.lo, r.span}, qin, qout, g, err, st);
    return dispatch_march(EvTablePM{r.tab2, r.lo, r.span}, qin, qout, g, err, st);
}

int nd_tile_x(int shape)
{
    switch (shape) {
    case ND_TILE_64x64: case ND_TILE_64x32: return 64;
    case ND_TILE_128x64: case ND_TILE_128x32: return 128;
    case ND_TILE_32x128: return 32;
    default: return 0;
    }
}

int nd_tile_y(int shape)
{
    switch (shape) {
    case ND_TILE_64x64: case ND_TILE_128x64: return 64;
    case ND_TILE_64x32: case ND_TILE_128x32: return 32;
    case ND_TILE_32x128: return 128;
    default: return 0;
    }
}

cudaError_t launch_step2d_tb(const RuleView& r, const NdPlan& p, const int32_t* qin,
                             int32_t* qout, const NdGrid& g, int K, unsigned* err,
                             cudaStream_t st)
{
    if (g.d != 2 || K < 1) return cudaErrorInvalidValue;
    if (r.evaluator == EVAL_CLOSED_FORM && !r.has_m)
        return dispatch_2d(EvClosedP{r.cf, r.lo, r.span}, p, qin, qout, g, K, err, st);
    if (!r.has_m) return dispatch_2d(EvTableP{r.tabp, r.lo, r.span}, p, qin, qout, g, K, err, st);
    if (r.tab16) return dispatch_2d(EvTablePM16{r.tab16, r.lo, r.span}, p, qin, qout, g, K, err, st);
    return dispatch_2d(EvTablePM{r.tab2, r.lo, r.span}, p, qin, qout, g, K, err, st);
}

bool walk_k_supported(int K) { return K == 1 || K == 2 || K == 3 || K == 4 || K == 6 || K == 8; }

cudaError_t launch_walk2d(const RuleView& r, const int32_t* qin, int32_t* qout, const NdGrid& g,
                          int K, unsigned* err, cudaStream_t st)
{
    if (g.d != 2 || !walk_k_supported(K)) return cudaErrorInvalidValue;
    if (r.evaluator == EVAL_CLOSED_FORM && !r.has_m)
        return dispatch_walk(EvClosedP{r.cf, r.lo, r.span}, K, qin, qout, g, err, st);
    if (!r.has_m) return dispatch_walk(EvTableP{r.tabp, r.lo, r.span}, K, qin, qout, g, err, st);
    if (r.tab16) return dispatch_walk(EvTablePM16{r.tab16, r.lo, r.span}, K, qin, qout, g, err, st);
    return dispatch_walk(EvTablePM{r.tab2, r.lo, r.span}, K, qin, qout, g, err, st);
}

bool walk3_k_supported(int K) { return K >= 1 && K <= 4; }

cudaError_t launch_walk3d(const RuleView& r, const int32_t* qin, int32_t* qout, const NdGrid& g,
                          int K, unsigned* err, cudaStream_t st)
{
    if (g.d != 3 || !walk3_k_supported(K)) return cudaErrorInvalidValue;
    if (r.evaluator == EVAL_CLOSED_FORM && !r.has_m)
        return dispatch_walk3(EvClosedP{r.cf, r.lo, r.span}, K, qin, qout, g, err, st);
    if (!r.has_m) return dispatch_walk3(EvTableP{r.tabp, r.lo, r.span}, K, qin, qout, g, err, st);
    if (r.tab16) return dispatch_walk3(EvTablePM16{r.tab16, r.lo, r.span}, K, qin, qout, g, err, st);
    return dispatch_walk3(EvTablePM{r.tab2, r.lo, r.span}, K, qin, qout, g, err, st);
}

cudaError_t launch_invariants_nd(const int32_t* q, const int32_t* other, const NdGrid& gr,
                                 long long* acc, cudaStream_t st)
{
    Strides g{gr.cells(), gr.dims[0], gr.dims[1], gr.dims[2], gr.dims[0], gr.dims[0] * gr.dims[1]};
    const dim3 grid((unsigned)((g.nx + IBLOCK - 1) / IBLOCK),
                    (unsigned)std::min<long long>(g.ny, 1024), (unsigned)std::min<long long>(g.nz, 64));
    k_invariants_nd<<<grid, IBLOCK, 0, st>>>(q, other, g, gr.d, acc);
    note_launches();
    return cudaGetLastError();
}

}  // namespace fqnm
