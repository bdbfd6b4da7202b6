// k_levels.cu -- level statistics of integer states (Supplementary
// Information, Entropy and Statistical Structure).
//
// For a transition q^n -> q^{n+1} of one scalar problem:
//   c_k = #{i : q_i = k}, p_k = c_k / N                      eq. pk_definition
//   S = -sum_k p_k log p_k                                   eq. discrete_entropy
//   N_eff = exp(S)                                           eq. neff
//   N_{k'k} = #{i : q_i^n = k, q_i^{n+1} = k'}               (level-transition counts)
//   M_{k'k} = N_{k'k} / c_k^n                                eq. empirical_M
//   rho = max over occupied k' of p^{n+1} of |sum_k M_{k'k} - 1|   (row-sum defect)
//
// Levels are indexed densely over [lo, lo + W) (the min..max of the two
// states).  Counts and the transition matrix are exact integers.  The
// nonzero entries of N^n are found by sorting the cell pair keys
// (k - lo) * W + (k' - lo) with a stable LSD radix sort (8-bit digits) and
// run-length encoding the sorted keys.  The row sums sum_k N_{k'k} / c_k^n
// then take one term per nonzero entry, round(N_{k'k} 2^62 / c_k^n) (an
// exact 128-by-64-bit division, rounded to nearest), split into a high part
// (units of 2^-31) and a low part (units of 2^-62) summed in two unsigned
// 64-bit integer accumulators: an exact sum of the rounded terms, whatever
// the order of the atomics.  |error| <= (nonzero entries in row k') 2^-63,
// and a row whose terms are multiples of 2^-62 (a permutation, a column
// sent whole to one level, c_k a power of two) is exact.  S is reduced in
// double in a fixed order, so every result is reproducible.
#include "fqnm_internal.h"
#include "levels.h"

#include <algorithm>

namespace fqnm {

namespace {

constexpr unsigned FULLMASK = 0xffffffffu;
constexpr int SCAN_THREADS = 1024;
constexpr int SCAN_ITEMS = 4;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;     // elements per scan block
constexpr int RADIX_THREADS = 256;
constexpr int RADIX_WARPS = RADIX_THREADS / 32;
constexpr int RADIX_ROUNDS = 16;                            // 32-key rounds per warp
constexpr int RADIX_TILE = RADIX_THREADS * RADIX_ROUNDS;   // 4096 keys per tile
constexpr int RADIX_BITS = 8;
constexpr int RADIX_DIGITS = 1 << RADIX_BITS;
constexpr int REDUCE_BLOCKS = 512;                          // fixed: reproducible reductions
constexpr int REDUCE_THREADS = 256;
constexpr unsigned long long ONE_FIXED = 1ull << 62;        // 1.0 in units of 2^-62
constexpr int HI_SHIFT = 31;

// ---- histogram ---------------------------------------------------------------

// c[q - lo] += 1 for every cell; lanes of a warp that hit the same level
// add once (plateaus of equal states would otherwise serialise on one word).
__global__ void k_level_hist(const int32_t* __restrict__ q, long long n, long long lo,
                             unsigned long long W, unsigned* __restrict__ hist,
                             unsigned* __restrict__ err)
{
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long base = blockIdx.x * (long long)blockDim.x;
    const int lane = threadIdx.x & 31;
    for (long long i0 = base; i0 < n; i0 += stride) {         // warp-uniform trip count
        const long long i = i0 + threadIdx.x;
        unsigned long long key = ~0ull;
        if (i < n) {
            const unsigned long long d = (unsigned long long)((long long)q[i] - lo);
            if (d < W) key = d;
            else atomicOr(err, ERRBIT_RANGE);
        }
        const unsigned peers = __match_any_sync(FULLMASK, key);
        if (key != ~0ull && lane == __ffs(peers) - 1)
            atomicAdd(hist + key, (unsigned)__popc(peers));
    }
}

// ---- block reductions in a fixed order ------------------------------------------

template <typename T>
__device__ __forceinline__ T block_sum(T v, T* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(FULLMASK, v, o);
    if (lane == 0) sh[w] = v;
    __syncthreads();
    T r = 0;
    if (threadIdx.x == 0)
        for (int j = 0; j < (int)(blockDim.x >> 5); ++j) r += sh[j];
    __syncthreads();
    return r;                                   // valid in thread 0
}

// Per-block partial of -sum p log p and of the occupied count over the bins
// [0, W); the grid is fixed (REDUCE_BLOCKS), so the order is too.
__global__ void k_level_entropy(const unsigned* __restrict__ hist, unsigned long long W,
                                long long n, double* __restrict__ part_s,
                                unsigned long long* __restrict__ part_occ)
{
    __shared__ double shd[32];
    __shared__ unsigned long long shu[32];
    double s = 0.0;
    unsigned long long occ = 0;
    const double dn = (double)n;
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < W;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        const unsigned c = hist[k];
        if (c) {
            const double p = __ddiv_rn((double)c, dn);
            s = __dsub_rn(s, __dmul_rn(p, log(p)));
            ++occ;
        }
    }
    s = block_sum<double>(s, shd);
    occ = block_sum<unsigned long long>(occ, shu);
    if (threadIdx.x == 0) {
        part_s[blockIdx.x] = s;
        part_occ[blockIdx.x] = occ;
    }
}

// Row sums: nonzero entry j of N^n (sorted keys) adds round(N 2^62 / c_k)
// to row k'.  Also counts the cells that changed level.
__global__ void k_level_rowacc(const unsigned long long* __restrict__ head_key,
                               const unsigned* __restrict__ head_pos,
                               const unsigned* __restrict__ pairs, long long n,
                               unsigned long long W, const unsigned* __restrict__ hist_prev,
                               unsigned long long* __restrict__ acc_hi,
                               unsigned long long* __restrict__ acc_lo,
                               unsigned long long* __restrict__ moved)
{
    __shared__ unsigned long long shu[32];
    const long long m = *pairs;
    unsigned long long mv = 0;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
         j += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = head_key[j];
        const unsigned long long a = key / W, b = key % W;
        const long long end = j + 1 < m ? (long long)head_pos[j + 1] : n;
        const unsigned long long N = (unsigned long long)(end - (long long)head_pos[j]);
        if (a >= W) continue;                               // only from a flagged range error
        const unsigned long long c = hist_prev[a];          // >= N > 0
        if (c < N) continue;
        const unsigned __int128 num = ((unsigned __int128)N << 62) + (c >> 1);
        const unsigned long long t = (unsigned long long)(num / c);   // <= 2^62
        atomicAdd(acc_hi + b, t >> HI_SHIFT);
        atomicAdd(acc_lo + b, t & ((1ull << HI_SHIFT) - 1));
        if (a != b) mv += N;
    }
    mv = block_sum<unsigned long long>(mv, shu);
    if (threadIdx.x == 0 && mv) atomicAdd(moved, mv);
}

// |R - 2^62| for a row, R = acc_hi 2^31 + acc_lo (units of 2^-62), as a
// 128-bit magnitude in two words.
__device__ __forceinline__ void row_defect(unsigned long long h, unsigned long long l,
                                           unsigned long long& dh, unsigned long long& dl)
{
    const unsigned __int128 R = ((unsigned __int128)h << HI_SHIFT) + (unsigned __int128)l;
    const unsigned __int128 one = (unsigned __int128)ONE_FIXED;
    const unsigned __int128 D = R >= one ? R - one : one - R;
    dh = (unsigned long long)(D >> 64);
    dl = (unsigned long long)D;
}

struct DefectArg {
    unsigned long long dh, dl;     // defect magnitude
    unsigned long long k;          // row index (smallest wins ties)
};

__device__ __forceinline__ bool better(const DefectArg& a, const DefectArg& b)
{
    if (a.dh != b.dh) return a.dh > b.dh;
    if (a.dl != b.dl) return a.dl > b.dl;
    return a.k < b.k;
}

__device__ __forceinline__ DefectArg shfl_down_arg(const DefectArg& a, int o)
{
    DefectArg r;
    r.dh = __shfl_down_sync(FULLMASK, a.dh, o);
    r.dl = __shfl_down_sync(FULLMASK, a.dl, o);
    r.k = __shfl_down_sync(FULLMASK, a.k, o);
    return r;
}

__device__ DefectArg block_best(DefectArg v, DefectArg* sh)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const DefectArg u = shfl_down_arg(v, o);
        if (better(u, v)) v = u;
    }
    if (lane == 0) sh[w] = v;
    __syncthreads();
    DefectArg r = sh[0];
    if (threadIdx.x == 0)
        for (int j = 1; j < (int)(blockDim.x >> 5); ++j)
            if (better(sh[j], r)) r = sh[j];
    __syncthreads();
    return r;
}

constexpr unsigned long long NO_ROW = ~0ull;

// Per-block best (largest defect, then smallest level) over the occupied
// rows of p^{n+1}.
__global__ void k_level_defect(const unsigned* __restrict__ hist,
                               const unsigned long long* __restrict__ acc_hi,
                               const unsigned long long* __restrict__ acc_lo,
                               unsigned long long W, DefectArg* __restrict__ part)
{
    __shared__ DefectArg sh[32];
    DefectArg best{0, 0, NO_ROW};
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < W;
         k += (unsigned long long)gridDim.x * blockDim.x) {
        if (!hist[k]) continue;
        DefectArg v;
        row_defect(acc_hi[k], acc_lo[k], v.dh, v.dl);
        v.k = k;
        if (best.k == NO_ROW || better(v, best)) best = v;
    }
    // an empty slot never beats a real row
    if (best.k == NO_ROW) { best.dh = 0; best.dl = 0; }
    const DefectArg r = block_best(best, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = r;
}

// One block of REDUCE_BLOCKS threads: combine the partials (thread j holds
// partial j) by fixed-order block reductions into the record.
__global__ void __launch_bounds__(REDUCE_BLOCKS)
k_level_finish(const double* __restrict__ ps_prev, const unsigned long long* __restrict__ po_prev,
               const double* __restrict__ ps, const unsigned long long* __restrict__ po,
               const DefectArg* __restrict__ pd, const unsigned* __restrict__ pairs,
               const unsigned long long* __restrict__ moved, long long n, long long lo,
               LevelRecord* __restrict__ rec)
{
    __shared__ double shd[32];
    __shared__ unsigned long long shu[32];
    __shared__ DefectArg sha[32];
    const int j = threadIdx.x;
    const double s0 = block_sum<double>(ps_prev[j], shd);
    const double s1 = block_sum<double>(ps[j], shd);
    const unsigned long long o0 = block_sum<unsigned long long>(po_prev[j], shu);
    const unsigned long long o1 = block_sum<unsigned long long>(po[j], shu);
    DefectArg v = pd[j];
    if (v.k == NO_ROW) { v.dh = 0; v.dl = 0; }
    const DefectArg best = block_best(v, sha);
    if (j != 0) return;
    rec->n_cells = n;
    rec->occupied_prev = (long long)o0;
    rec->occupied = (long long)o1;
    rec->S_prev = s0;
    rec->S = s1;
    rec->n_eff = exp(s1);
    // defect = D 2^-62 with D = dh 2^64 + dl
    const double d = __dadd_rn(__dmul_rn((double)best.dh, 0x1p64), (double)best.dl);
    rec->rho = best.k == NO_ROW ? 0.0 : __dmul_rn(d, 0x1p-62);
    rec->rho_level = best.k == NO_ROW ? 0 : (long long)best.k + lo;
    rec->pairs = pairs ? (long long)*pairs : -1;
    rec->moved = (long long)*moved;
}

// ---- exclusive scan of unsigned counts (three phases) --------------------------

__device__ __forceinline__ unsigned block_exclusive_scan(unsigned v, unsigned* sh, unsigned& total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    unsigned x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned y = __shfl_up_sync(FULLMASK, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[w] = x;
    __syncthreads();
    if (w == 0) {
        unsigned t = lane < nw ? sh[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned y = __shfl_up_sync(FULLMASK, t, o);
            if (lane >= o) t += y;
        }
        if (lane < nw) sh[lane] = t;          // inclusive prefix of warp totals
    }
    __syncthreads();
    total = sh[nw - 1];
    const unsigned before = w > 0 ? sh[w - 1] : 0;
    __syncthreads();
    return before + x - v;
}

__global__ void k_scan_sums(const unsigned* __restrict__ in, long long m, unsigned* __restrict__ sums)
{
    __shared__ unsigned sh[32];
    const long long b0 = blockIdx.x * (long long)SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned v = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j)
        if (b0 + j < m) v += in[b0 + j];
    unsigned total;
    (void)block_exclusive_scan(v, sh, total);
    if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

// One block: exclusive scan of the block sums in place; the grand total to *total.
__global__ void k_scan_top(unsigned* __restrict__ sums, int nb, unsigned* __restrict__ total)
{
    __shared__ unsigned sh[32];
    unsigned carry = 0;
    for (int b0 = 0; b0 < nb; b0 += blockDim.x) {
        const int b = b0 + threadIdx.x;
        const unsigned v = b < nb ? sums[b] : 0;
        unsigned t;
        const unsigned ex = block_exclusive_scan(v, sh, t);
        if (b < nb) sums[b] = carry + ex;
        carry += t;
    }
    if (threadIdx.x == 0 && total) *total = carry;
}

__global__ void k_scan_apply(const unsigned* __restrict__ in, long long m,
                             const unsigned* __restrict__ sums, unsigned* __restrict__ out)
{
    __shared__ unsigned sh[32];
    const long long b0 = blockIdx.x * (long long)SCAN_TILE + threadIdx.x * SCAN_ITEMS;
    unsigned v[SCAN_ITEMS];
    unsigned tsum = 0;
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        v[j] = b0 + j < m ? in[b0 + j] : 0;
        tsum += v[j];
    }
    unsigned total;
    unsigned run = block_exclusive_scan(tsum, sh, total) + sums[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SCAN_ITEMS; ++j) {
        if (b0 + j < m) out[b0 + j] = run;
        run += v[j];
    }
}

// ---- stable LSD radix sort of 64-bit keys -------------------------------------------
// Tile t covers keys [t*4096, (t+1)*4096); warp w of the tile walks its 512
// keys in 16 rounds of 32 in index order, so ranks follow the input order.

__device__ __forceinline__ long long radix_index(long long tile, int w, int r, int lane)
{
    return tile * RADIX_TILE + (long long)w * (RADIX_ROUNDS * 32) + r * 32 + lane;
}

__global__ void k_pair_keys(const int32_t* __restrict__ qn, const int32_t* __restrict__ qn1,
                            long long n, long long lo, unsigned long long W,
                            unsigned long long* __restrict__ keys)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x) {
        const unsigned long long a = (unsigned long long)((long long)qn[i] - lo);
        const unsigned long long b = (unsigned long long)((long long)qn1[i] - lo);
        keys[i] = a * W + b;              // both < W (checked by the histogram pass)
    }
}

__global__ void __launch_bounds__(RADIX_THREADS)
k_radix_count(const unsigned long long* __restrict__ keys, long long n, int shift,
              long long ntiles, unsigned* __restrict__ counts)
{
    __shared__ unsigned hist[RADIX_DIGITS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    hist[threadIdx.x] = 0;
    __syncthreads();
    for (int r = 0; r < RADIX_ROUNDS; ++r) {
        const long long i = radix_index(blockIdx.x, w, r, lane);
        const unsigned d = i < n ? (unsigned)((keys[i] >> shift) & (RADIX_DIGITS - 1)) : RADIX_DIGITS;
        const unsigned peers = __match_any_sync(FULLMASK, d);
        if (d < RADIX_DIGITS && lane == __ffs(peers) - 1) atomicAdd(hist + d, (unsigned)__popc(peers));
    }
    __syncthreads();
    counts[(long long)threadIdx.x * ntiles + blockIdx.x] = hist[threadIdx.x];
}

__global__ void __launch_bounds__(RADIX_THREADS)
k_radix_scatter(const unsigned long long* __restrict__ in, unsigned long long* __restrict__ out,
                long long n, int shift, long long ntiles, const unsigned* __restrict__ offsets,
                unsigned* __restrict__ err)
{
    __shared__ unsigned whist[RADIX_WARPS][RADIX_DIGITS];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned lt = (1u << lane) - 1u;
    for (int j = 0; j < RADIX_WARPS; ++j) whist[j][threadIdx.x] = 0;
    __syncthreads();
    for (int r = 0; r < RADIX_ROUNDS; ++r) {                    // per-warp digit counts
        const long long i = radix_index(blockIdx.x, w, r, lane);
        const unsigned d = i < n ? (unsigned)((in[i] >> shift) & (RADIX_DIGITS - 1)) : RADIX_DIGITS;
        const unsigned peers = __match_any_sync(FULLMASK, d);
        if (d < RADIX_DIGITS && lane == __ffs(peers) - 1) whist[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    {                                                           // warp start positions
        const int d = threadIdx.x;
        unsigned run = offsets[(long long)d * ntiles + blockIdx.x];
        for (int j = 0; j < RADIX_WARPS; ++j) {
            const unsigned c = whist[j][d];
            whist[j][d] = run;
            run += c;
        }
    }
    __syncthreads();
    for (int r = 0; r < RADIX_ROUNDS; ++r) {
        const long long i = radix_index(blockIdx.x, w, r, lane);
        const unsigned long long key = i < n ? in[i] : 0;
        const unsigned d = i < n ? (unsigned)((key >> shift) & (RADIX_DIGITS - 1)) : RADIX_DIGITS;
        const unsigned peers = __match_any_sync(FULLMASK, d);
        const unsigned long long pos = (unsigned long long)whist[w][d] + __popc(peers & lt);
        if (d < RADIX_DIGITS && FQNM_IN_RANGE(pos, n, err)) out[pos] = key;
        __syncwarp();
        if (d < RADIX_DIGITS && lane == __ffs(peers) - 1) whist[w][d] += __popc(peers);
        __syncwarp();
    }
}

// ---- run-length encoding of the sorted keys ---------------------------------------

__global__ void k_heads(const unsigned long long* __restrict__ keys, long long n, unsigned* __restrict__ flags)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        flags[i] = (i == 0 || keys[i] != keys[i - 1]) ? 1u : 0u;
}

__global__ void k_compact_heads(const unsigned long long* __restrict__ keys, long long n,
                                const unsigned* __restrict__ flags, const unsigned* __restrict__ idx,
                                unsigned long long* __restrict__ head_key, unsigned* __restrict__ head_pos,
                                unsigned* __restrict__ err)
{
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
         i += (long long)gridDim.x * blockDim.x)
        if (flags[i] && FQNM_IN_RANGE(idx[i], n, err)) {
            head_key[idx[i]] = keys[i];
            head_pos[idx[i]] = (unsigned)i;
        }
}

__global__ void k_decode_pairs(const unsigned long long* __restrict__ head_key,
                               const unsigned* __restrict__ head_pos, const unsigned* __restrict__ pairs,
                               long long n, long long lo, unsigned long long W,
                               long long* __restrict__ k, long long* __restrict__ kn,
                               long long* __restrict__ cnt)
{
    const long long m = *pairs;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < m;
         j += (long long)gridDim.x * blockDim.x) {
        const unsigned long long key = head_key[j];
        k[j] = (long long)(key / W) + lo;
        kn[j] = (long long)(key % W) + lo;
        const long long end = j + 1 < m ? (long long)head_pos[j + 1] : n;
        cnt[j] = end - (long long)head_pos[j];
    }
}

__global__ void k_widen_counts(const unsigned* __restrict__ hist, unsigned long long W,
                               long long* __restrict__ out)
{
    for (unsigned long long k = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; k < W;
         k += (unsigned long long)gridDim.x * blockDim.x)
        out[k] = hist[k];
}

int grid_of(long long n, int threads, int cap = 152 * 16)
{
    long long g = (n + threads - 1) / threads;
    if (g < 1) g = 1;
    return (int)(g < cap ? g : cap);
}

}  // namespace

// ---- host side ---------------------------------------------------------------

struct LevelWork {
    size_t n_cap = 0, w_cap = 0;
    unsigned* hist[2] = {nullptr, nullptr};
    unsigned long long* acc = nullptr;          // [2][w_cap]: hi, lo
    unsigned long long* keys[2] = {nullptr, nullptr};
    unsigned* counts = nullptr;                 // radix digit counts, then flags
    unsigned* scan = nullptr;                   // scan output
    unsigned* sums = nullptr;                   // scan block sums
    size_t counts_cap = 0, scan_cap = 0, sums_cap = 0;
    unsigned long long* head_key = nullptr;
    unsigned* head_pos = nullptr;
    unsigned* pairs = nullptr;                  // [1]
    unsigned long long* moved = nullptr;        // [1]
    double* part_s = nullptr;                   // [2][REDUCE_BLOCKS]
    unsigned long long* part_occ = nullptr;     // [2][REDUCE_BLOCKS]
    DefectArg* part_def = nullptr;              // [REDUCE_BLOCKS]
    LevelRecord* rec = nullptr;                 // device record
    unsigned* err = nullptr;                    // [1] out-of-range levels
    int32_t* snap = nullptr;                    // q^n
    size_t snap_cap = 0;
    long long last_lo = 0;
    unsigned long long last_W = 0;
    long long last_n = 0;
    bool have_pairs = false;
};

static void free_all(LevelWork* w)
{
    void* ps[] = {w->hist[0], w->hist[1], w->acc, w->keys[0], w->keys[1], w->counts, w->scan,
                  w->sums, w->head_key, w->head_pos, w->pairs, w->moved, w->part_s,
                  w->part_occ, w->part_def, w->rec, w->err, w->snap};
    for (void* p : ps)
        if (p) cudaFree(p);
}

LevelWork* level_work_create() { return new LevelWork(); }

void level_work_destroy(LevelWork* w)
{
    if (!w) return;
    free_all(w);
    delete w;
}

#define LCK(x)                                   \
    do {                                         \
        cudaError_t e_ = (x);                    \
        if (e_ != cudaSuccess) return e_;        \
    } while (0)

template <typename T>
static cudaError_t grow(T*& p, size_t& cap, size_t want)
{
    if (p && cap >= want) return cudaSuccess;
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
    LCK(cudaMalloc((void**)&p, want * sizeof(T)));
    cap = want;
    return cudaSuccess;
}

static cudaError_t ensure(LevelWork* w, size_t n, size_t W)
{
    if (!w->rec) {
        LCK(cudaMalloc((void**)&w->rec, sizeof(LevelRecord)));
        LCK(cudaMalloc((void**)&w->err, sizeof(unsigned)));
        LCK(cudaMalloc((void**)&w->pairs, sizeof(unsigned)));
        LCK(cudaMalloc((void**)&w->moved, sizeof(unsigned long long)));
        LCK(cudaMalloc((void**)&w->part_s, 2 * REDUCE_BLOCKS * sizeof(double)));
        LCK(cudaMalloc((void**)&w->part_occ, 2 * REDUCE_BLOCKS * sizeof(unsigned long long)));
        LCK(cudaMalloc((void**)&w->part_def, REDUCE_BLOCKS * sizeof(DefectArg)));
    }
    if (W > w->w_cap) {
        for (int j = 0; j < 2; ++j)
            if (w->hist[j]) cudaFree(w->hist[j]);
        if (w->acc) cudaFree(w->acc);
        w->hist[0] = w->hist[1] = nullptr;
        w->acc = nullptr;
        w->w_cap = 0;
        LCK(cudaMalloc((void**)&w->hist[0], W * sizeof(unsigned)));
        LCK(cudaMalloc((void**)&w->hist[1], W * sizeof(unsigned)));
        LCK(cudaMalloc((void**)&w->acc, 2 * W * sizeof(unsigned long long)));
        w->w_cap = W;
    }
    if (n > w->n_cap) {
        void* ps[] = {w->keys[0], w->keys[1], w->head_key, w->head_pos};
        for (void* p : ps)
            if (p) cudaFree(p);
        w->keys[0] = w->keys[1] = w->head_key = nullptr;
        w->head_pos = nullptr;
        w->n_cap = 0;
        LCK(cudaMalloc((void**)&w->keys[0], n * sizeof(unsigned long long)));
        LCK(cudaMalloc((void**)&w->keys[1], n * sizeof(unsigned long long)));
        LCK(cudaMalloc((void**)&w->head_key, n * sizeof(unsigned long long)));
        LCK(cudaMalloc((void**)&w->head_pos, n * sizeof(unsigned)));
        w->n_cap = n;
    }
    const size_t ntiles = (n + RADIX_TILE - 1) / RADIX_TILE;
    const size_t m = std::max(n, (size_t)RADIX_DIGITS * ntiles);
    LCK(grow(w->counts, w->counts_cap, m));
    LCK(grow(w->scan, w->scan_cap, m));
    LCK(grow(w->sums, w->sums_cap, (m + SCAN_TILE - 1) / SCAN_TILE + 1));
    return cudaSuccess;
}

// exclusive scan of in[0, m) into out; the total to *total (device)
static cudaError_t scan_u32(LevelWork* w, const unsigned* in, long long m, unsigned* out,
                            unsigned* total, cudaStream_t st)
{
    const int nb = (int)((m + SCAN_TILE - 1) / SCAN_TILE);
    k_scan_sums<<<nb, SCAN_THREADS, 0, st>>>(in, m, w->sums);
    k_scan_top<<<1, SCAN_THREADS, 0, st>>>(w->sums, nb, total);
    k_scan_apply<<<nb, SCAN_THREADS, 0, st>>>(in, m, w->sums, out);
    note_launches(3);
    return cudaGetLastError();
}

cudaError_t level_transition(LevelWork* w, const int32_t* qn, const int32_t* qn1, int64_t n,
                             int64_t lo, int64_t W, cudaStream_t st)
{
    if (n <= 0 || W <= 0) return cudaErrorInvalidValue;
    LCK(ensure(w, (size_t)n, (size_t)W));
    unsigned* err = w->err;
    LCK(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
    const unsigned long long uW = (unsigned long long)W;
    w->last_lo = lo;
    w->last_W = uW;
    w->last_n = n;
    int launches = 0;

    // histograms of q^n and q^{n+1}
    for (int j = 0; j < 2; ++j) LCK(cudaMemsetAsync(w->hist[j], 0, W * sizeof(unsigned), st));
    LCK(cudaMemsetAsync(w->acc, 0, 2 * W * sizeof(unsigned long long), st));
    LCK(cudaMemsetAsync(w->moved, 0, sizeof(unsigned long long), st));
    const int g = grid_of(n, 256);
    k_level_hist<<<g, 256, 0, st>>>(qn, n, lo, uW, w->hist[0], err);
    k_level_hist<<<g, 256, 0, st>>>(qn1, n, lo, uW, w->hist[1], err);
    // entropy partials of both
    k_level_entropy<<<REDUCE_BLOCKS, REDUCE_THREADS, 0, st>>>(w->hist[0], uW, n, w->part_s,
                                                              w->part_occ);
    k_level_entropy<<<REDUCE_BLOCKS, REDUCE_THREADS, 0, st>>>(
        w->hist[1], uW, n, w->part_s + REDUCE_BLOCKS, w->part_occ + REDUCE_BLOCKS);
    launches += 4;

    // nonzero entries of N^n: sort the pair keys, run-length encode
    k_pair_keys<<<g, 256, 0, st>>>(qn, qn1, n, lo, uW, w->keys[0]);
    ++launches;
    const unsigned long long maxkey = uW * uW - 1;
    int bits = 0;
    while (bits < 64 && (maxkey >> bits)) ++bits;
    const long long ntiles = (n + RADIX_TILE - 1) / RADIX_TILE;
    int cur = 0;
    for (int shift = 0; shift < bits; shift += RADIX_BITS) {
        k_radix_count<<<(unsigned)ntiles, RADIX_THREADS, 0, st>>>(w->keys[cur], n, shift, ntiles,
                                                                  w->counts);
        LCK(scan_u32(w, w->counts, RADIX_DIGITS * ntiles, w->scan, nullptr, st));
        k_radix_scatter<<<(unsigned)ntiles, RADIX_THREADS, 0, st>>>(w->keys[cur], w->keys[1 - cur],
                                                                    n, shift, ntiles, w->scan, err);
        launches += 2;
        cur = 1 - cur;
    }
    k_heads<<<g, 256, 0, st>>>(w->keys[cur], n, w->counts);
    LCK(scan_u32(w, w->counts, n, w->scan, w->pairs, st));
    k_compact_heads<<<g, 256, 0, st>>>(w->keys[cur], n, w->counts, w->scan, w->head_key,
                                       w->head_pos, err);
    // row sums from the entries, then the defect
    k_level_rowacc<<<g, 256, 0, st>>>(w->head_key, w->head_pos, w->pairs, n, uW, w->hist[0],
                                      w->acc, w->acc + W, w->moved);
    k_level_defect<<<REDUCE_BLOCKS, REDUCE_THREADS, 0, st>>>(w->hist[1], w->acc, w->acc + W, uW,
                                                             w->part_def);
    launches += 4;
    k_level_finish<<<1, REDUCE_BLOCKS, 0, st>>>(w->part_s, w->part_occ, w->part_s + REDUCE_BLOCKS,
                                                w->part_occ + REDUCE_BLOCKS, w->part_def,
                                                w->pairs, w->moved, n, lo, w->rec);
    ++launches;
    note_launches(launches);
    w->have_pairs = true;
    return cudaGetLastError();
}

cudaError_t level_record(LevelWork* w, LevelRecord* host, unsigned* host_err, cudaStream_t st)
{
    LCK(cudaMemcpyAsync(host, w->rec, sizeof(LevelRecord), cudaMemcpyDeviceToHost, st));
    LCK(cudaMemcpyAsync(host_err, w->err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    return cudaStreamSynchronize(st);
}

cudaError_t level_export_pairs(LevelWork* w, int64_t pairs, int64_t* k, int64_t* kn, int64_t* cnt,
                               cudaStream_t st)
{
    if (!w->have_pairs) return cudaErrorInvalidValue;
    if (pairs <= 0) return cudaSuccess;
    long long* dk = nullptr;
    LCK(cudaMallocAsync((void**)&dk, 3 * pairs * sizeof(long long), st));
    k_decode_pairs<<<grid_of(pairs, 256), 256, 0, st>>>(w->head_key, w->head_pos, w->pairs,
                                                        w->last_n, w->last_lo, w->last_W, dk,
                                                        dk + pairs, dk + 2 * pairs);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(k, dk, pairs * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(kn, dk + pairs, pairs * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(cnt, dk + 2 * pairs, pairs * sizeof(long long), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dk, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

cudaError_t level_histogram(LevelWork* w, const int32_t* q, int64_t n, int64_t lo, int64_t W,
                            int64_t* counts, unsigned* host_err, cudaStream_t st)
{
    if (n <= 0 || W <= 0) return cudaErrorInvalidValue;
    LCK(ensure(w, (size_t)n, (size_t)W));
    unsigned* err = w->err;
    LCK(cudaMemsetAsync(err, 0, sizeof(unsigned), st));
    LCK(cudaMemsetAsync(w->hist[0], 0, W * sizeof(unsigned), st));
    k_level_hist<<<grid_of(n, 256), 256, 0, st>>>(q, n, lo, (unsigned long long)W, w->hist[0], err);
    long long* dc = nullptr;
    LCK(cudaMallocAsync((void**)&dc, W * sizeof(long long), st));
    k_widen_counts<<<grid_of(W, 256), 256, 0, st>>>(w->hist[0], (unsigned long long)W, dc);
    note_launches(2);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(counts, dc, W * sizeof(long long), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(host_err, err, sizeof(unsigned), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(dc, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

cudaError_t level_snapshot(LevelWork* w, const int32_t* q, int64_t n, cudaStream_t st)
{
    LCK(grow(w->snap, w->snap_cap, (size_t)n));
    LCK(cudaMemcpyAsync(w->snap, q, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, st));
    return cudaSuccess;
}

const int32_t* level_snap(const LevelWork* w) { return w->snap; }

}  // namespace fqnm
