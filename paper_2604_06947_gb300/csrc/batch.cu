// batch.cu -- continuous batching of many independent periodic scalar
// problems (the serving path).
//
// Requests of uneven size and step count are queued with their arrival time.
// Each epoch the host
//   1. admits waiting requests that have arrived, while a slot and arena
//      memory are free (first fit; a large request at the head does not block
//      smaller ones behind it), copies their initial states to the device
//      and builds their transfer maps there (eq. flux_table, as a single
//      solver would);
//   2. uploads the table of active problems (one copy of the bytes in use)
//      and launches one persistent batched kernel: every tile of every active
//      problem runs the same temporal-blocked tile code as the single-problem
//      kernel, advancing that problem by min(K, remaining) steps;
//   3. copies finished states to host memory, frees their memory and slots,
//      and records submit-to-result latency.
// Epochs are pipelined: epoch e is enqueued before the host waits for epoch
// e-1 and reads its retirements (finished states, error words, rule
// checks), so the GPU runs e while the host retires e-1 and admits for e+1.
// A problem's memory is released only once no enqueued epoch uses it; an
// error seen one epoch late restarts the problem after that epoch too.
// States stay resident on the device between epochs.  Problems are
// independent and the arithmetic is integer, so each result is bit-identical
// to solving the problem alone.  A range escape (error bit of that problem)
// restarts only that problem from its initial state with a wider map.
#include "tile_step.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cstring>
#include <deque>
#include <map>
#include <unordered_map>
#include <vector>

namespace fqnm {

namespace {

struct BatchDesc {             // one active problem as the batched kernel sees it
    const int* qin;
    int* qout;
    long long n;
    long long S;               // output cells per tile
    int k;                     // steps this epoch
    int evaluator;
    int has_m;
    int lo;
    unsigned span;
    const int2* tab2;
    const int* tabp;
    const int* tab16;          // packed (phi+, phi-) int16 pairs, or null
    unsigned* err;
    ClosedForm cf;
};

struct BatchHeader {
    int nprob;
    int pad;
    long long total_tiles;
};

template <int V, int LAYOUT, bool WARP>
__global__ void __launch_bounds__(tb::TB_MAX_BLOCK)
k_batch_step(const BatchDesc* __restrict__ d, const long long* __restrict__ prefix,
             const BatchHeader* __restrict__ hdr)
{
    __shared__ tb::TileSmem sm;
    const int np = hdr->nprob;
    const long long total = hdr->total_tiles;
    for (long long t = blockIdx.x; t < total; t += gridDim.x) {
        int lo = 0, hi = np - 1;                      // last p with prefix[p] <= t
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (prefix[mid] <= t) lo = mid; else hi = mid - 1;
        }
        const BatchDesc D = d[lo];
        const long long tile = t - prefix[lo];
        if (D.evaluator == EVAL_CLOSED_FORM) {
            tb::EvClosedP ev{D.cf, D.lo, D.span};
            tb::tile_step<tb::EvClosedP, V, LAYOUT, WARP>(D.qin, D.qout, D.n, D.k, D.S, tile, ev, D.err, sm);
        } else if (!D.has_m) {
            tb::EvTableP ev{D.tabp, D.lo, D.span};
            tb::tile_step<tb::EvTableP, V, LAYOUT, WARP>(D.qin, D.qout, D.n, D.k, D.S, tile, ev, D.err, sm);
        } else if (D.tab16) {
            tb::EvTablePM16 ev{D.tab16, D.lo, D.span};
            tb::tile_step<tb::EvTablePM16, V, LAYOUT, WARP>(D.qin, D.qout, D.n, D.k, D.S, tile, ev, D.err, sm);
        } else {
            tb::EvTablePM ev{D.tab2, D.lo, D.span};
            tb::tile_step<tb::EvTablePM, V, LAYOUT, WARP>(D.qin, D.qout, D.n, D.k, D.S, tile, ev, D.err, sm);
        }
        __syncthreads();                              // shared edges are reused by the next tile
    }
}

using BatchKernel = void (*)(const BatchDesc*, const long long*, const BatchHeader*);

BatchKernel batch_kernel(int v, int layout, int block)
{
    const bool w = block == 32;
    if (layout == LAYOUT_RUNS8) {
        if (v == 16) return w ? k_batch_step<16, LAYOUT_RUNS8, true> : k_batch_step<16, LAYOUT_RUNS8, false>;
        return nullptr;
    }
    if (layout == LAYOUT_RUNS4) {
        if (v == 8) return w ? k_batch_step<8, LAYOUT_RUNS4, true> : k_batch_step<8, LAYOUT_RUNS4, false>;
        if (v == 16) return w ? k_batch_step<16, LAYOUT_RUNS4, true> : k_batch_step<16, LAYOUT_RUNS4, false>;
        return nullptr;
    }
    if (layout == LAYOUT_BLOCKED) {
        if (v == 4) return w ? k_batch_step<4, LAYOUT_BLOCKED, true> : k_batch_step<4, LAYOUT_BLOCKED, false>;
        if (v == 8) return w ? k_batch_step<8, LAYOUT_BLOCKED, true> : k_batch_step<8, LAYOUT_BLOCKED, false>;
        if (v == 16) return w ? k_batch_step<16, LAYOUT_BLOCKED, true> : k_batch_step<16, LAYOUT_BLOCKED, false>;
    } else if (layout == LAYOUT_INTERLEAVED) {
        if (v == 4) return w ? k_batch_step<4, LAYOUT_INTERLEAVED, true> : k_batch_step<4, LAYOUT_INTERLEAVED, false>;
        if (v == 8) return w ? k_batch_step<8, LAYOUT_INTERLEAVED, true> : k_batch_step<8, LAYOUT_INTERLEAVED, false>;
        if (v == 16) return w ? k_batch_step<16, LAYOUT_INTERLEAVED, true> : k_batch_step<16, LAYOUT_INTERLEAVED, false>;
    }
    return nullptr;
}

uint64_t now_ns()
{
    return (uint64_t)std::chrono::duration_cast<std::chrono::nanoseconds>(
               std::chrono::steady_clock::now().time_since_epoch()).count();
}

size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }

}  // namespace

}  // namespace fqnm

using namespace fqnm;

#define BCK(call)                                                  \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);       \
    } while (0)

namespace {

struct Request {
    fqnm_problem_spec spec{};
    size_t n = 0;
    std::vector<int32_t> q0;           // host submission (copied)
    const int32_t* q0_dev = nullptr;   // device submission (caller's)
    int32_t* out_dev = nullptr;        // device result (caller's), else host
    std::vector<int32_t> result;
    uint64_t steps = 0;
    uint64_t arrival_ns = 0, done_ns = 0;
    int state = 0;            // 0 queued, 1 active, 2 done, 3 handed out
    int64_t margin = 1024;
    int32_t qmin = 0, qmax = 0;
};

struct Slot {
    int64_t req = -1;
    size_t off = 0, bytes = 0;       // arena block of the two state buffers
    size_t toff = 0, tbytes = 0;     // arena block of the tables
    bool range_pending = false;
    int32_t* q[2] = {nullptr, nullptr};
    int2* tab2 = nullptr;
    int32_t* tabp = nullptr;
    int32_t* tab16 = nullptr;
    bool use16 = false;
    int cur = 0;
    uint64_t done = 0;
    int32_t lo = 0;
    uint32_t span = 0;
    int evaluator = EVAL_TABLE;
    int has_m = 1;
    ClosedForm cf{};
    bool check_pending = false;
    bool cf_candidate = false;
    int k_this_epoch = 0;
    size_t out_off = 0;              // where its final state lands in the staging area
    long long first_epoch = -1;      // the first enqueued epoch that steps it
    long long last_epoch = -1;       // the last enqueued epoch that steps it
    long long check_epoch = -1;      // the epoch whose read-back carries its rule check
    long long finish_epoch = -1;     // the epoch that copies its final state out
    bool restarting = false;         // an error was seen: restart once no epoch uses it
};

constexpr int TUNE_MIN_ACTIVE = 16;  // problems stepping before tuning epochs count

struct Inflight {                    // an enqueued epoch not yet retired
    long long epoch = 0;
    int np = 0;                      // problems it steps
    uint64_t updates = 0;            // cell updates it performs
    uint64_t t0 = 0;                 // host clock when it was enqueued
    int cand = -1;                   // autotuning candidate it runs, or -1
    int k = 1;                       // steps per problem in this epoch (the plan's K)
};

}  // namespace

struct fqnm_batch {
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char* arena = nullptr;
    size_t budget = 0;
    std::map<size_t, size_t> free_blocks;     // offset -> size
    int max_slots = 0;
    std::vector<Slot> slots;
    std::vector<int> free_slots;
    std::vector<Request> reqs;                // indexed by id
    std::deque<int64_t> queue;
    std::deque<int64_t> completed;            // finished, not yet reported
    // device
    // the epoch's problem table, packed as [header | tile prefix (np+1) |
    // descriptors (np)] and uploaded in one copy of just the bytes in use
    char* d_tab = nullptr;
    size_t tab_bytes = 0;
    // error words and rule-check results, read back in one copy (the check
    // part only when a check is due)
    char* d_rb = nullptr;
    size_t rb_err_bytes = 0, rb_bytes = 0;
    unsigned* d_err = nullptr;                // into d_rb
    unsigned long long* d_check = nullptr;    // into d_rb
    long long* d_range = nullptr;             // [2*slot]: min, max of a device submission
    cudaStream_t side = nullptr;              // device submissions' state ranges
    double gpu_ms = 0.0;
    // per epoch parity (two epochs in flight): the pinned problem table and
    // read-back buffer and the events around the launch; the staging area
    // is split in two halves
    char* h_tab[2] = {nullptr, nullptr};
    std::vector<BatchDesc> desc_scratch;
    std::vector<long long> prefix_scratch;
    char* h_rb[2] = {nullptr, nullptr};
    Plan grid_plan;                           // the plan `grid` was sized for
    bool grid_valid = false;
    // ev0 / ev1 bracket the batched launch (GPU time); ev2 follows the
    // epoch's copies and read-backs (its retirement waits on it)
    cudaEvent_t ev0[2] = {nullptr, nullptr}, ev1[2] = {nullptr, nullptr}, ev2[2] = {nullptr, nullptr};
    long long* h_range = nullptr;
    int32_t* h_stage = nullptr;
    size_t stage_ints = 0;                    // per half
    // pipeline
    long long next_epoch = 0;
    std::deque<Inflight> inflight;
    uint64_t last_retire_ns = 0;
    // plan
    Plan plan;
    int grid = 0;
    // online autotuning: candidate plans tried in turn (round robin, so that
    // each sees the same mix of load) on the first epochs with work, scored
    // by the wall time between epoch retirements per time step: the time an
    // active problem waits for each of its steps, fixed costs per epoch
    // included (a long-running request's latency is its steps times this)
    bool tuning = false;
    std::vector<Plan> cands;
    std::vector<double> cand_ns;             // wall ns per time step, summed over epochs
    std::vector<uint64_t> cand_updates;
    std::vector<int> cand_retired;
    int tune_launch = 0, tune_per_plan = 3;
    Plan tune_default;                       // the plan run while tuning waits for load
    // counters
    uint64_t launches = 0, cell_updates = 0, epochs = 0;
    bool pack16 = false;                     // packed int16 tables (off: faster on GB300)
    int64_t margin = 1024;                   // initial map margin of new requests
};

static void batch_free_device(fqnm_batch* b)
{
    for (int pe = 0; pe < 2; ++pe) {
        if (b->ev0[pe]) cudaEventDestroy(b->ev0[pe]);
        if (b->ev1[pe]) cudaEventDestroy(b->ev1[pe]);
        if (b->ev2[pe]) cudaEventDestroy(b->ev2[pe]);
        cudaFreeHost(b->h_tab[pe]);
        cudaFreeHost(b->h_rb[pe]);
    }
    cudaFree(b->arena);
    cudaFree(b->d_tab);
    cudaFree(b->d_rb);
    cudaFree(b->d_range);
    cudaFreeHost(b->h_range);
    cudaFreeHost(b->h_stage);
    if (b->side) cudaStreamDestroy(b->side);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
}

static bool arena_alloc(fqnm_batch* b, size_t bytes, size_t* off)
{
    for (auto it = b->free_blocks.begin(); it != b->free_blocks.end(); ++it) {
        if (it->second >= bytes) {
            *off = it->first;
            const size_t rest = it->second - bytes;
            const size_t roff = it->first + bytes;
            b->free_blocks.erase(it);
            if (rest) b->free_blocks[roff] = rest;
            return true;
        }
    }
    return false;
}

static void arena_free(fqnm_batch* b, size_t off, size_t bytes)
{
    auto it = b->free_blocks.emplace(off, bytes).first;
    auto nx = std::next(it);
    if (nx != b->free_blocks.end() && it->first + it->second == nx->first) {
        it->second += nx->second;
        b->free_blocks.erase(nx);
    }
    if (it != b->free_blocks.begin()) {
        auto pv = std::prev(it);
        if (pv->first + pv->second == it->first) {
            pv->second += it->second;
            b->free_blocks.erase(it);
        }
    }
}

extern "C" uint64_t fqnm_clock_ns(void) { return now_ns(); }

extern "C" fqnm_status fqnm_batch_create(size_t mem_budget_bytes, int max_slots,
                                         void* stream, fqnm_batch** out)
{
    if (!out) return set_error(FQNM_ERR_ARG, "null out");
    *out = nullptr;
    if (max_slots < 1 || max_slots > 65536) return set_error(FQNM_ERR_ARG, "max_slots must be 1..65536");
    if (mem_budget_bytes < (1u << 20)) return set_error(FQNM_ERR_ARG, "memory budget below 1 MiB");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return set_error(FQNM_ERR_CUDA, "no CUDA device available");
    fqnm_batch* b = new (std::nothrow) fqnm_batch();
    if (!b) return set_error(FQNM_ERR_OOM, "host allocation failed");
    b->budget = align_up(mem_budget_bytes, 256);
    b->max_slots = max_slots;
    b->slots.resize(max_slots);
    for (int i = max_slots - 1; i >= 0; --i) b->free_slots.push_back(i);
    b->plan.kernel = 2;
    b->plan.layout = LAYOUT_BLOCKED;
    b->plan.v = 8;
    b->plan.block = 128;
    b->plan.k = 128;
    b->stage_ints = (size_t)32 << 20;                 // 2 x 128 MiB pinned staging
    cudaError_t e = cudaSuccess;
    if (stream) b->stream = (cudaStream_t)stream;
    else { e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking); b->own_stream = true; }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->side, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->arena, b->budget);
    b->tab_bytes = align_up(sizeof(BatchHeader) + (max_slots + 1) * sizeof(long long), 16) +
                   max_slots * sizeof(BatchDesc);
    b->rb_err_bytes = align_up(max_slots * sizeof(unsigned), 16);
    b->rb_bytes = b->rb_err_bytes + 4 * max_slots * sizeof(unsigned long long);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_tab, b->tab_bytes);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_rb, b->rb_bytes);
    if (e == cudaSuccess) {
        b->d_err = (unsigned*)b->d_rb;
        b->d_check = (unsigned long long*)(b->d_rb + b->rb_err_bytes);
    }
    for (int pe = 0; pe < 2 && e == cudaSuccess; ++pe) {
        e = cudaMallocHost((void**)&b->h_tab[pe], b->tab_bytes);
        if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_rb[pe], b->rb_bytes);
        if (e == cudaSuccess) e = cudaEventCreate(&b->ev0[pe]);
        if (e == cudaSuccess) e = cudaEventCreate(&b->ev1[pe]);
        if (e == cudaSuccess) e = cudaEventCreate(&b->ev2[pe]);
    }
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_stage, 2 * b->stage_ints * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_range, 2 * max_slots * sizeof(long long));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_range, 2 * max_slots * sizeof(long long));
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_rb, 0, b->rb_bytes, b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        fqnm_status st = (e == cudaErrorMemoryAllocation)
                             ? set_error(FQNM_ERR_OOM, "batch allocation failed: %s", cudaGetErrorString(e))
                             : cuda_error(e, "fqnm_batch_create");
        batch_free_device(b);
        delete b;
        return st;
    }
    for (int pe = 0; pe < 2; ++pe) {
        std::memset(b->h_tab[pe], 0, b->tab_bytes);
        std::memset(b->h_rb[pe], 0, b->rb_bytes);
    }
    b->free_blocks[0] = b->budget;
    *out = b;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_destroy(fqnm_batch* b)
{
    if (!b) return FQNM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->side) cudaStreamSynchronize(b->side);
    batch_free_device(b);
    delete b;
    return FQNM_OK;
}

static fqnm_status retire_oldest(fqnm_batch* b);

// Retire every enqueued epoch (before the plan changes).
static fqnm_status drain(fqnm_batch* b)
{
    while (!b->inflight.empty()) {
        fqnm_status st = retire_oldest(b);
        if (st != FQNM_OK) return st;
    }
    return FQNM_OK;
}

static void drop_grid(fqnm_batch* b)
{
    b->grid_valid = false;
}

extern "C" fqnm_status fqnm_batch_set_plan(fqnm_batch* b, int cells_per_thread, int block,
                                           int k, int layout)
{
    if (!b) return set_error(FQNM_ERR_ARG, "null handle");
    Plan p = b->plan;
    if (cells_per_thread) p.v = cells_per_thread;
    if (block) p.block = block;
    if (k) p.k = k;
    if (layout) p.layout = layout;
    RuleView dummy{};
    if (!tb_plan_supported(dummy, p) || !batch_kernel(p.v, p.layout, p.block))
        return set_error(FQNM_ERR_ARG, "unsupported batch plan (V=%d, block=%d, K=%d, layout=%d)",
                         p.v, p.block, p.k, p.layout);
    // the plan only decides how each epoch cuts problems into tiles, so it
    // may change between epochs
    fqnm_status st = drain(b);
    if (st != FQNM_OK) return st;
    b->plan = p;
    b->tuning = false;
    drop_grid(b);
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_autotune(fqnm_batch* b, int epochs_per_plan)
{
    if (!b) return set_error(FQNM_ERR_ARG, "null handle");
    if (epochs_per_plan < 1 || epochs_per_plan > 64)
        return set_error(FQNM_ERR_ARG, "epochs_per_plan must be 1..64");
    fqnm_status st = drain(b);
    if (st != FQNM_OK) return st;
    b->cands.clear();
    const int vs[2] = {8, 16}, blocks[3] = {32, 128, 256}, ks[3] = {32, 64, 128};
    RuleView dummy{};
    for (int L : {LAYOUT_BLOCKED, LAYOUT_RUNS8})
        for (int v : vs)
            for (int bl : blocks)
                for (int k : ks) {
                    Plan p;
                    p.kernel = 2; p.layout = L; p.v = v; p.block = bl; p.k = k;
                    if (4LL * k > (long long)bl * v) continue;      // > 50 % halo work
                    if (tb_plan_supported(dummy, p) && batch_kernel(v, L, bl))
                        b->cands.push_back(p);
                }
    b->cand_ns.assign(b->cands.size(), 0.0);
    b->cand_updates.assign(b->cands.size(), 0);
    b->cand_retired.assign(b->cands.size(), 0);
    b->tune_launch = 0;
    b->tune_per_plan = epochs_per_plan;
    b->tuning = !b->cands.empty();
    b->tune_default = b->plan;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_set_margin(fqnm_batch* b, int64_t margin)
{
    if (!b) return set_error(FQNM_ERR_ARG, "null handle");
    if (margin < 0 || margin > (INT32_MAX / 8)) return set_error(FQNM_ERR_ARG, "margin out of range");
    b->margin = margin;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_get_plan(fqnm_batch* b, int* cells_per_thread, int* block,
                                           int* k, int* layout, int* tuning)
{
    if (!b) return set_error(FQNM_ERR_ARG, "null handle");
    if (cells_per_thread) *cells_per_thread = b->plan.v;
    if (block) *block = b->plan.block;
    if (k) *k = b->plan.k;
    if (layout) *layout = b->plan.layout;
    if (tuning) *tuning = b->tuning ? 1 : 0;
    return FQNM_OK;
}

// Bytes a problem occupies on the device: two state buffers and its tables.
static size_t problem_bytes(size_t n, int64_t count)
{
    return align_up(n * sizeof(int32_t), 256) * 2 + align_up(count * sizeof(int2), 256) +
           2 * align_up(count * sizeof(int32_t), 256);
}

static fqnm_status validate_spec(const fqnm_problem_spec* spec, size_t n)
{
    if (n == 0 || n > (size_t)INT32_MAX / 2) return set_error(FQNM_ERR_ARG, "bad problem size");
    if (spec->boundary != FQNM_BC_PERIODIC)
        return set_error(FQNM_ERR_ARG, "the batch serves periodic problems");
    const fqnm_flux& f = spec->flux;
    if (f.kind != FQNM_FLUX_LINEAR_UPWIND && f.kind != FQNM_FLUX_LINEAR_LF &&
        f.kind != FQNM_FLUX_BURGERS_LF && f.kind != FQNM_FLUX_BURGERS_EO)
        return set_error(FQNM_ERR_ARG, "the batch serves scalar split fluxes");
    // the same validation as a single solver (Courant number, delta = 2^k)
    fqnm_solver* probe = nullptr;
    fqnm_status st = fqnm_create(&f, &spec->delta, spec->dx, spec->dt, spec->boundary, &probe);
    if (st != FQNM_OK) return st;
    fqnm_destroy(probe);
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_submit(fqnm_batch* b, const fqnm_problem_spec* spec,
                                         const int32_t* q0, size_t n, uint64_t steps,
                                         uint64_t arrival_ns, int64_t* id)
{
    if (!b || !spec || !q0 || !id) return set_error(FQNM_ERR_ARG, "null argument");
    fqnm_status st = validate_spec(spec, n);
    if (st != FQNM_OK) return st;
    Request r;
    r.spec = *spec;
    r.n = n;
    r.q0.assign(q0, q0 + n);
    r.steps = steps;
    r.arrival_ns = arrival_ns ? arrival_ns : now_ns();
    r.margin = b->margin;
    auto mm = std::minmax_element(r.q0.begin(), r.q0.end());
    r.qmin = *mm.first;
    r.qmax = *mm.second;
    const int64_t count = ((int64_t)r.qmax + r.margin) - ((int64_t)r.qmin - r.margin) + 1;
    if (problem_bytes(n, count) > b->budget)
        return set_error(FQNM_ERR_OOM, "problem needs %zu bytes of device memory, the batch "
                         "budget is %zu", problem_bytes(n, count), b->budget);
    *id = (int64_t)b->reqs.size();
    b->reqs.push_back(std::move(r));
    b->queue.push_back(*id);
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_submit_device(fqnm_batch* b, const fqnm_problem_spec* spec,
                                                const int32_t* q0, size_t n, uint64_t steps,
                                                uint64_t arrival_ns, int32_t* out,
                                                int64_t* id)
{
    if (!b || !spec || !q0 || !id) return set_error(FQNM_ERR_ARG, "null argument");
    fqnm_status st = validate_spec(spec, n);
    if (st != FQNM_OK) return st;
    if (problem_bytes(n, 1) > b->budget)
        return set_error(FQNM_ERR_OOM, "problem states alone exceed the batch budget");
    Request r;
    r.spec = *spec;
    r.n = n;
    r.q0_dev = q0;
    r.out_dev = out;
    r.steps = steps;
    r.arrival_ns = arrival_ns ? arrival_ns : now_ns();
    r.margin = b->margin;
    *id = (int64_t)b->reqs.size();
    b->reqs.push_back(std::move(r));
    b->queue.push_back(*id);
    return FQNM_OK;
}

// Phase 1 of admission: a slot, the state buffers and the initial state on
// the device; a device submission also gets its state range from the GPU.
static fqnm_status admit_state(fqnm_batch* b, int64_t rid, int32_t* stage_base,
                               size_t* stage_used, bool* admitted)
{
    *admitted = false;
    Request& r = b->reqs[rid];
    const size_t n = r.n;
    const bool host = r.q0_dev == nullptr;
    if (host && *stage_used + n > b->stage_ints) return FQNM_OK;          // next epoch
    if (b->free_slots.empty()) return FQNM_OK;
    const size_t sb = align_up(n * sizeof(int32_t), 256);
    size_t off = 0;
    if (!arena_alloc(b, 2 * sb, &off)) return FQNM_OK;
    const int si = b->free_slots.back();
    b->free_slots.pop_back();
    Slot& s = b->slots[si];
    s = Slot();
    s.req = rid;
    s.off = off;
    s.bytes = 2 * sb;
    s.q[0] = (int32_t*)(b->arena + off);
    s.q[1] = (int32_t*)(b->arena + off + sb);
    if (host) {
        int32_t* stage = stage_base + *stage_used;
        std::memcpy(stage, r.q0.data(), n * sizeof(int32_t));
        *stage_used += n;
        BCK(cudaMemcpyAsync(s.q[0], stage, n * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream));
    } else {
        // on the side stream: the host waits for the range without waiting
        // for the epoch in flight (the copy is complete before the state is
        // first stepped: that wait precedes the launch)
        BCK(cudaMemcpyAsync(s.q[0], r.q0_dev, n * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                            b->side));
        init_minmax(b->h_range + 2 * si);
        BCK(cudaMemcpyAsync(b->d_range + 2 * si, b->h_range + 2 * si, 2 * sizeof(long long),
                            cudaMemcpyHostToDevice, b->side));
        BCK(launch_minmax_i32(s.q[0], (int64_t)n, b->d_range + 2 * si, b->side));
        s.range_pending = true;
    }
    r.state = 1;
    *admitted = true;
    return FQNM_OK;
}

// Phase 2: the transfer tables over the state range, built and checked on
// the GPU.  False in *ok if the arena has no room yet (the caller requeues).
static fqnm_status admit_table(fqnm_batch* b, int si, bool* ok)
{
    *ok = false;
    Slot& s = b->slots[si];
    Request& r = b->reqs[s.req];
    const int64_t lo = std::max<int64_t>((int64_t)r.qmin - r.margin, INT32_MIN / 4);
    const int64_t hi = std::min<int64_t>((int64_t)r.qmax + r.margin, INT32_MAX / 4);
    const int64_t count = hi - lo + 1;
    if (problem_bytes(r.n, count) > b->budget)
        return set_error(FQNM_ERR_OOM, "problem %lld needs %zu bytes, the batch budget is %zu",
                         (long long)s.req, problem_bytes(r.n, count), b->budget);
    const size_t t2 = align_up(count * sizeof(int2), 256);
    const size_t tp = align_up(count * sizeof(int32_t), 256);
    const size_t tb = t2 + 2 * tp;
    size_t toff = 0;
    if (!arena_alloc(b, tb, &toff)) return FQNM_OK;
    s.toff = toff;
    s.tbytes = tb;
    s.tab2 = (int2*)(b->arena + toff);
    s.tabp = (int32_t*)(b->arena + toff + t2);
    s.tab16 = (int32_t*)(b->arena + toff + t2 + tp);
    s.lo = (int32_t)lo;
    s.span = (uint32_t)(count - 1);
    const fqnm_flux& f = r.spec.flux;
    s.has_m = !(f.kind == FQNM_FLUX_LINEAR_UPWIND && f.a >= 0.0);
    s.evaluator = EVAL_TABLE;
    BCK(cudaMemsetAsync(b->d_err + si, 0, sizeof(unsigned), b->stream));
    BCK(launch_build_split_table(f.kind, f.a, f.alpha, r.spec.delta, r.spec.dt / r.spec.dx,
                                 f.rounding, lo, count, s.tab2, s.tabp, b->d_err + si, b->stream));
    // certificate, phi- presence and, for a linear map, one closed-form
    // candidate are checked on the GPU; the table serves until the result is
    // read back at the end of the epoch
    BCK(cudaMemsetAsync(b->d_check + 4 * si, 0, 4 * sizeof(unsigned long long), b->stream));
    ClosedForm cf{};
    bool cand = false;
    if (f.kind == FQNM_FLUX_LINEAR_UPWIND && f.a > 0.0) {
        // the finest convergent of the multiplier is the candidate; the GPU
        // accepts it only if it equals the table at every entry
        const auto cv = convergents(f.a * (r.spec.dt / r.spec.dx), 1u << 12);
        if (!cv.empty())
            cand = make_closed_form(lo, hi, cv.back().first, cv.back().second, f.rounding, &cf);
    }
    BCK(launch_rule_check(s.tab2, lo, count, cand ? &cf : nullptr, b->d_check + 4 * si, b->stream));
    s.cf = cf;
    s.cf_candidate = cand;
    s.check_pending = true;
    *ok = true;
    return FQNM_OK;
}

static void release_slot(fqnm_batch* b, int si)
{
    Slot& s = b->slots[si];
    arena_free(b, s.off, s.bytes);
    if (s.tbytes) arena_free(b, s.toff, s.tbytes);
    s.tbytes = 0;
    s.req = -1;
    b->free_slots.push_back(si);
}

static bool same_plan(const Plan& a, const Plan& b)
{
    return a.layout == b.layout && a.v == b.v && a.block == b.block && a.k == b.k;
}

// The batched kernel's grid for the current plan: every SM filled with as
// many blocks as it holds (the kernel loops over the epoch's tiles).
static fqnm_status size_grid(fqnm_batch* b, BatchKernel* kern)
{
    *kern = batch_kernel(b->plan.v, b->plan.layout, b->plan.block);
    if (!*kern) return set_error(FQNM_ERR_ARG, "no batched kernel for this plan");
    if (b->grid_valid && same_plan(b->grid_plan, b->plan)) return FQNM_OK;
    int per_sm = 0, sms = 0, dev = 0;
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, *kern, b->plan.block, 0));
    b->grid = std::max(1, per_sm) * sms;
    b->grid_plan = b->plan;
    b->grid_valid = true;
    return FQNM_OK;
}

static fqnm_status run_epoch_body(fqnm_batch* b, bool* did_work);

// One serving epoch inside an NVTX range ("fqnm_batch_epoch").
static fqnm_status run_epoch(fqnm_batch* b, bool* did_work)
{
    nvtxRangePushA("fqnm_batch_epoch");
    const fqnm_status st = run_epoch_body(b, did_work);
    nvtxRangePop();
    return st;
}


// Admission: arrived requests into free slots (states first, then, after
// the state range of device submissions is known, their tables).
static fqnm_status admit_arrivals(fqnm_batch* b, int32_t* stage_base, size_t* stage_used)
{
    const uint64_t t = now_ns();
    std::vector<int> fresh;
    bool need_range = false;
    for (auto it = b->queue.begin(); it != b->queue.end();) {
        Request& r = b->reqs[*it];
        if (r.arrival_ns > t) { ++it; continue; }
        bool adm = false;
        const int64_t rid = *it;
        fqnm_status st = admit_state(b, rid, stage_base, stage_used, &adm);
        if (st != FQNM_OK) return st;
        if (adm) {
            it = b->queue.erase(it);
            for (int si = 0; si < b->max_slots; ++si)
                if (b->slots[si].req == rid && !b->slots[si].tbytes) {
                    fresh.push_back(si);
                    need_range = need_range || b->slots[si].range_pending;
                    break;
                }
        } else {
            ++it;
        }
        if (b->free_slots.empty()) break;
    }
    if (need_range) {
        BCK(cudaMemcpyAsync(b->h_range, b->d_range, 2 * b->max_slots * sizeof(long long),
                            cudaMemcpyDeviceToHost, b->side));
        BCK(cudaStreamSynchronize(b->side));
    }
    // tables in admission order; when one does not fit, the state blocks of
    // the later fresh requests are given back first (so that they cannot
    // starve the earlier one), and the request retries once
    std::vector<int64_t> requeue;
    for (size_t f = 0; f < fresh.size(); ++f) {
        const int si = fresh[f];
        Slot& s = b->slots[si];
        Request& r = b->reqs[s.req];
        if (s.range_pending) {
            r.qmin = (int32_t)b->h_range[2 * si];
            r.qmax = (int32_t)b->h_range[2 * si + 1];
            s.range_pending = false;
        }
        bool ok = false;
        fqnm_status st = admit_table(b, si, &ok);
        if (st != FQNM_OK) return st;
        if (!ok) {
            for (size_t g = f + 1; g < fresh.size(); ++g) {
                Slot& sg = b->slots[fresh[g]];
                b->reqs[sg.req].state = 0;
                requeue.push_back(sg.req);
                release_slot(b, fresh[g]);
            }
            fresh.resize(f + 1);
            st = admit_table(b, si, &ok);
            if (st != FQNM_OK) return st;
        }
        if (!ok) {                                    // no room for the tables yet
            r.state = 0;
            requeue.push_back(s.req);
            release_slot(b, si);
        }
    }
    for (auto it = requeue.rbegin(); it != requeue.rend(); ++it) b->queue.push_front(*it);
    // nothing on the device and an arrived request still waiting: it cannot
    // be admitted at all (report it rather than spin)
    if (b->free_slots.size() == (size_t)b->max_slots && b->inflight.empty()) {
        for (int64_t rid : b->queue)
            if (b->reqs[rid].arrival_ns <= t)
                return set_error(FQNM_ERR_OOM, "request %lld cannot be admitted into an empty "
                                 "batch (budget %zu bytes)", (long long)rid, b->budget);
    }
    return FQNM_OK;
}

// Enqueue the next epoch: one batched launch over every active problem with
// steps left, the copies of the states that this launch finishes (or that
// finished earlier and still wait for staging room), and the read-back of
// the error words and rule checks.  Nothing is enqueued when there is
// nothing to do.
static fqnm_status launch_epoch(fqnm_batch* b, int32_t* stage_base, size_t stage_used,
                                bool* launched)
{
    *launched = false;
    const long long ep = b->next_epoch;
    const int pe = (int)(ep & 1);
    Inflight f;
    f.epoch = ep;
    f.t0 = now_ns();
    if (b->tuning) {
        // candidates are timed only under load (at least TUNE_MIN_ACTIVE
        // problems stepping): the first epochs of a stream, with a handful of
        // small problems, would favour the smallest tiles
        int active = 0;
        for (int si = 0; si < b->max_slots; ++si) {
            const Slot& s = b->slots[si];
            active += s.req >= 0 && !s.restarting && s.done < b->reqs[s.req].steps;
        }
        const int nc = (int)b->cands.size();
        if (active >= TUNE_MIN_ACTIVE && b->tune_launch < nc * b->tune_per_plan) {
            const int c = b->tune_launch % nc;
            b->plan = b->cands[c];
            f.cand = c;
        } else {
            b->plan = b->tune_default;
        }
    }
    f.k = b->plan.k;
    const long long E = (long long)b->plan.block * b->plan.v;
    // descriptors first into a staging order, packed after the prefix below
    std::vector<BatchDesc>& hdv = b->desc_scratch;
    hdv.resize(b->max_slots);
    BatchDesc* hd = hdv.data();
    std::vector<long long>& hpv = b->prefix_scratch;
    hpv.resize(b->max_slots + 1);
    long long* hp = hpv.data();
    int np = 0;
    long long total = 0;
    bool pending = false;
    for (int si = 0; si < b->max_slots; ++si) {
        Slot& s = b->slots[si];
        s.k_this_epoch = 0;
        if (s.req < 0 || s.restarting) continue;
        Request& r = b->reqs[s.req];
        if (s.check_pending && s.check_epoch < 0) pending = true;
        if (s.done >= r.steps) {
            if (s.finish_epoch < 0) pending = true;       // its copy still to enqueue
            continue;
        }
        const int k = (int)std::min<uint64_t>((uint64_t)b->plan.k, r.steps - s.done);
        const long long S = E - 2LL * k;
        const long long n = (long long)r.n;
        BatchDesc& d = hd[np];
        d.qin = s.q[s.cur];
        d.qout = s.q[1 - s.cur];
        d.n = n;
        d.S = S;
        d.k = k;
        d.evaluator = s.evaluator;
        d.has_m = s.has_m;
        d.lo = s.lo;
        d.span = s.span;
        d.tab2 = s.tab2;
        d.tab16 = s.use16 ? s.tab16 : nullptr;
        d.tabp = s.tabp;
        d.err = b->d_err + si;
        d.cf = s.cf;
        hp[np] = total;
        total += (n + S - 1) / S;
        s.k_this_epoch = k;
        f.updates += (uint64_t)k * (uint64_t)n;
        ++np;
    }
    if (np == 0 && !pending) return FQNM_OK;
    hp[np] = total;
    f.np = np;
    if (np > 0) {
        BatchKernel kern = nullptr;
        fqnm_status st = size_grid(b, &kern);
        if (st != FQNM_OK) return st;
        // this parity's pinned table was last read by the copy of epoch
        // ep - 2, which has been retired
        char* h = b->h_tab[pe];
        BatchHeader hdr{};
        hdr.nprob = np;
        hdr.total_tiles = total;
        std::memcpy(h, &hdr, sizeof(hdr));
        const size_t off_prefix = sizeof(BatchHeader);
        const size_t off_desc = align_up(off_prefix + (size_t)(np + 1) * sizeof(long long), 16);
        std::memcpy(h + off_prefix, hp, (size_t)(np + 1) * sizeof(long long));
        std::memcpy(h + off_desc, hd, (size_t)np * sizeof(BatchDesc));
        const size_t bytes = off_desc + (size_t)np * sizeof(BatchDesc);
        BCK(cudaEventRecord(b->ev0[pe], b->stream));
        BCK(cudaMemcpyAsync(b->d_tab, h, bytes, cudaMemcpyHostToDevice, b->stream));
        kern<<<b->grid, b->plan.block, 0, b->stream>>>(
            (const BatchDesc*)(b->d_tab + off_desc), (const long long*)(b->d_tab + off_prefix),
            (const BatchHeader*)b->d_tab);
        BCK(cudaGetLastError());
        BCK(cudaEventRecord(b->ev1[pe], b->stream));
        note_launches();
        b->launches += 1;
        b->epochs += 1;
        if (f.cand >= 0) b->tune_launch += 1;
    }
    // bookkeeping; final states out
    size_t out_used = stage_used;
    for (int si = 0; si < b->max_slots; ++si) {
        Slot& s = b->slots[si];
        if (s.req < 0 || s.restarting) continue;
        Request& r = b->reqs[s.req];
        if (s.k_this_epoch) {
            s.done += s.k_this_epoch;
            s.cur = 1 - s.cur;
            if (s.first_epoch < 0) s.first_epoch = ep;
            s.last_epoch = ep;
            b->cell_updates += (uint64_t)s.k_this_epoch * r.n;
        }
        if (s.check_pending && s.check_epoch < 0) s.check_epoch = ep;
        if (s.done < r.steps || s.finish_epoch >= 0) continue;
        if (r.out_dev) {
            BCK(cudaMemcpyAsync(r.out_dev, s.q[s.cur], r.n * sizeof(int32_t),
                                cudaMemcpyDeviceToDevice, b->stream));
            s.finish_epoch = ep;
        } else if (out_used + r.n <= b->stage_ints) {
            BCK(cudaMemcpyAsync(stage_base + out_used, s.q[s.cur], r.n * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, b->stream));
            s.finish_epoch = ep;
            s.out_off = out_used;
            out_used += r.n;
        }
    }
    // one read-back: the error words, and the rule checks when one is due
    bool checks = false;
    for (int si = 0; si < b->max_slots && !checks; ++si)
        checks = b->slots[si].req >= 0 && b->slots[si].check_pending &&
                 b->slots[si].check_epoch == ep;
    BCK(cudaMemcpyAsync(b->h_rb[pe], b->d_rb, checks ? b->rb_bytes : b->rb_err_bytes,
                        cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaEventRecord(b->ev2[pe], b->stream));
    b->inflight.push_back(f);
    b->next_epoch += 1;
    *launched = true;
    return FQNM_OK;
}

// Wait for the oldest enqueued epoch and act on what it read back: GPU time
// and tuning, rule checks, errors (restart the problem once no enqueued
// epoch uses it), finished states (results, slots freed).
static fqnm_status retire_oldest(fqnm_batch* b)
{
    if (b->inflight.empty()) return FQNM_OK;
    const Inflight f = b->inflight.front();
    b->inflight.pop_front();
    const int pe = (int)(f.epoch & 1);
    BCK(cudaEventSynchronize(b->ev2[pe]));
    const uint64_t tdone = now_ns();
    if (f.np > 0) {
        float ms = 0.0f;
        BCK(cudaEventElapsedTime(&ms, b->ev0[pe], b->ev1[pe]));
        b->gpu_ms += ms;
    }
    // tuning: each candidate is scored by the wall time between retirements
    // (the epoch period the host sees, its own work included) per time step
    const uint64_t period = tdone - (b->last_retire_ns > f.t0 ? b->last_retire_ns : f.t0);
    b->last_retire_ns = tdone;
    if (b->tuning && f.cand >= 0 && f.np > 0) {
        b->cand_ns[f.cand] += (double)period / (double)f.k;
        b->cand_updates[f.cand] += f.updates;
        b->cand_retired[f.cand] += 1;
        bool all = true;
        for (size_t j = 0; j < b->cands.size(); ++j)
            all = all && b->cand_retired[j] >= b->tune_per_plan;
        if (all) {                                   // all tried: keep the fastest
            size_t best = 0;
            double best_v = 1e300;
            for (size_t j = 0; j < b->cands.size(); ++j) {
                if (!b->cand_retired[j]) continue;
                const double v = b->cand_ns[j] / (double)b->cand_retired[j];
                if (v < best_v) { best_v = v; best = j; }
            }
            b->plan = b->cands[best];
            b->tuning = false;
        }
    }
    const unsigned* herr = (const unsigned*)b->h_rb[pe];
    const unsigned long long* hcheck = (const unsigned long long*)(b->h_rb[pe] + b->rb_err_bytes);
    // rule checks read back by this epoch
    for (int si = 0; si < b->max_slots; ++si) {
        Slot& s = b->slots[si];
        if (s.req < 0 || !s.check_pending || s.check_epoch != f.epoch) continue;
        s.check_pending = false;
        const unsigned long long* c = hcheck + 4 * si;
        s.has_m = (c[1] & CERT_M_NONZERO) != 0;
        if (b->pack16 && c[2] <= 32767 && c[3] <= 32767) {   // both maps fit int16
            BCK(launch_pack_tab16(s.tab2, (int64_t)s.span + 1, s.tab16, b->stream));
            s.use16 = true;
        }
        if (s.cf_candidate && c[0] == 0 && !s.has_m) s.evaluator = EVAL_CLOSED_FORM;
    }
    // errors: the problem restarts from its initial state with a wider map
    for (int si = 0; si < b->max_slots; ++si) {
        Slot& s = b->slots[si];
        // (an error word read back before this problem's first epoch may
        // still be its slot's previous occupant's)
        if (s.req < 0 || s.restarting || herr[si] == 0 || s.first_epoch < 0 ||
            f.epoch < s.first_epoch)
            continue;
        Request& r = b->reqs[s.req];
        if (herr[si] & ERRBIT_OVERFLOW)
            return set_error(FQNM_ERR_OVERFLOW, "problem %lld: a transfer does not fit int32",
                             (long long)s.req);
        r.margin = std::max<int64_t>(4 * r.margin, 4096);
        s.restarting = true;
    }
    for (int si = 0; si < b->max_slots; ++si) {
        Slot& s = b->slots[si];
        if (s.req < 0) continue;
        Request& r = b->reqs[s.req];
        if (s.restarting) {
            if (s.last_epoch > f.epoch) continue;     // an enqueued epoch still steps it
            r.state = 0;
            b->queue.push_front(s.req);
            release_slot(b, si);
            BCK(cudaMemsetAsync(b->d_err + si, 0, sizeof(unsigned), b->stream));
            continue;
        }
        if (s.finish_epoch != f.epoch) continue;
        if (!r.out_dev) {
            const int32_t* stage = b->h_stage + (size_t)pe * b->stage_ints + s.out_off;
            r.result.assign(stage, stage + r.n);
        }
        r.done_ns = tdone;
        r.state = 2;
        b->completed.push_back(s.req);
        release_slot(b, si);
    }
    return FQNM_OK;
}

// One epoch: admit, enqueue epoch e, then retire epoch e-1 while e runs
// (with nothing to enqueue, retire what is in flight).
static fqnm_status run_epoch_body(fqnm_batch* b, bool* did_work)
{
    *did_work = false;
    const int pe = (int)(b->next_epoch & 1);
    int32_t* stage_base = b->h_stage + (size_t)pe * b->stage_ints;
    size_t stage_used = 0;
    fqnm_status st = admit_arrivals(b, stage_base, &stage_used);
    if (st != FQNM_OK) return st;
    bool launched = false;
    st = launch_epoch(b, stage_base, stage_used, &launched);
    if (st != FQNM_OK) return st;
    if (b->inflight.size() > 1 || (!launched && !b->inflight.empty())) {
        st = retire_oldest(b);
        if (st != FQNM_OK) return st;
        *did_work = true;
    }
    *did_work = *did_work || launched;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_progress(fqnm_batch* b, int max_epochs, int* n_active,
                                           int* n_queued)
{
    if (!b) return set_error(FQNM_ERR_ARG, "null handle");
    for (int e = 0; e < max_epochs; ++e) {
        bool work = false;
        fqnm_status st = run_epoch(b, &work);
        if (st != FQNM_OK) return st;
        if (!work) break;
    }
    if (n_active) *n_active = b->max_slots - (int)b->free_slots.size();
    if (n_queued) *n_queued = (int)b->queue.size();
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_poll(fqnm_batch* b, int64_t id, int32_t* q_out,
                                       size_t capacity, uint64_t* latency_ns, int* done)
{
    if (!b || !done) return set_error(FQNM_ERR_ARG, "null argument");
    if (id < 0 || id >= (int64_t)b->reqs.size()) return set_error(FQNM_ERR_ARG, "unknown id %lld", (long long)id);
    Request& r = b->reqs[id];
    *done = 0;
    if (r.state == 3) return set_error(FQNM_ERR_STATE, "result %lld already handed out", (long long)id);
    if (r.state != 2) return FQNM_OK;
    if (q_out && !r.out_dev && capacity < r.n)
        return set_error(FQNM_ERR_ARG, "result buffer holds %zu values, problem %lld has %zu",
                         capacity, (long long)id, r.n);
    if (q_out && !r.out_dev) std::memcpy(q_out, r.result.data(), r.result.size() * sizeof(int32_t));
    if (latency_ns) *latency_ns = r.done_ns - r.arrival_ns;
    *done = 1;
    r.state = 3;
    std::vector<int32_t>().swap(r.result);
    std::vector<int32_t>().swap(r.q0);
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_completed(fqnm_batch* b, int64_t* ids, int max_ids,
                                            int* n)
{
    if (!b || !n || (max_ids > 0 && !ids)) return set_error(FQNM_ERR_ARG, "null argument");
    int k = 0;
    while (k < max_ids && !b->completed.empty()) {
        ids[k++] = b->completed.front();
        b->completed.pop_front();
    }
    *n = k;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_stats(fqnm_batch* b, uint64_t* launches,
                                        uint64_t* cell_updates, uint64_t* epochs,
                                        double* gpu_ms)
{
    if (!b) return set_error(FQNM_ERR_ARG, "null handle");
    if (launches) *launches = b->launches;
    if (cell_updates) *cell_updates = b->cell_updates;
    if (epochs) *epochs = b->epochs;
    if (gpu_ms) *gpu_ms = b->gpu_ms;
    return FQNM_OK;
}
