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
//   2. replays a CUDA graph that uploads the table of active problems and
//      launches one persistent batched kernel: every tile of every active
//      problem runs the same temporal-blocked tile code as the single-problem
//      kernel, advancing that problem by min(K, remaining) steps;
//   3. copies finished states to host memory, frees their memory and slots,
//      and records submit-to-result latency.
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
    if (layout == LAYOUT_BLOCKED) {
        if (v == 4) return w ? k_batch_step<4, LAYOUT_BLOCKED, true> : k_batch_step<4, LAYOUT_BLOCKED, false>;
        if (v == 8) return w ? k_batch_step<8, LAYOUT_BLOCKED, true> : k_batch_step<8, LAYOUT_BLOCKED, false>;
        if (v == 16) return w ? k_batch_step<16, LAYOUT_BLOCKED, true> : k_batch_step<16, LAYOUT_BLOCKED, false>;
    } else {
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
    BatchDesc* d_desc = nullptr;
    long long* d_prefix = nullptr;
    BatchHeader* d_hdr = nullptr;
    unsigned* d_err = nullptr;
    unsigned long long* d_check = nullptr;
    long long* d_range = nullptr;             // [2*slot]: min, max of a device submission
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    double gpu_ms = 0.0;
    // pinned
    BatchDesc* h_desc = nullptr;
    long long* h_prefix = nullptr;
    BatchHeader* h_hdr = nullptr;
    unsigned* h_err = nullptr;
    unsigned long long* h_check = nullptr;
    long long* h_range = nullptr;
    int32_t* h_stage = nullptr;
    size_t stage_ints = 0;
    // plan and graph
    Plan plan;
    int grid = 0;
    cudaGraphExec_t gexec = nullptr;
    // online autotuning: candidate plans tried on the first epochs with work,
    // scored by the epochs' wall time (host admission, replay and sync
    // included: a fixed cost per epoch that small K pays more often) per
    // cell update
    bool tuning = false;
    std::vector<Plan> cands;
    std::vector<double> cand_ns;             // wall ns of the epochs, summed
    std::vector<uint64_t> cand_updates;
    int tune_epoch = 0, tune_per_plan = 3;
    // counters
    uint64_t launches = 0, cell_updates = 0, epochs = 0;
    bool pack16 = false;                     // packed int16 tables (off: faster on GB300)
};

static void batch_free_device(fqnm_batch* b)
{
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    cudaFree(b->arena);
    cudaFree(b->d_desc);
    cudaFree(b->d_prefix);
    cudaFree(b->d_hdr);
    cudaFree(b->d_err);
    cudaFree(b->d_check);
    cudaFree(b->d_range);
    cudaFreeHost(b->h_range);
    if (b->ev0) cudaEventDestroy(b->ev0);
    if (b->ev1) cudaEventDestroy(b->ev1);
    cudaFreeHost(b->h_desc);
    cudaFreeHost(b->h_prefix);
    cudaFreeHost(b->h_hdr);
    cudaFreeHost(b->h_err);
    cudaFreeHost(b->h_check);
    cudaFreeHost(b->h_stage);
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
    b->plan.k = 32;
    b->stage_ints = (size_t)64 << 20;                 // 256 MiB pinned staging
    cudaError_t e = cudaSuccess;
    if (stream) b->stream = (cudaStream_t)stream;
    else { e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking); b->own_stream = true; }
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->arena, b->budget);
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_desc, max_slots * sizeof(BatchDesc));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_prefix, (max_slots + 1) * sizeof(long long));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_hdr, sizeof(BatchHeader));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_err, max_slots * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_check, 4 * max_slots * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_desc, max_slots * sizeof(BatchDesc));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_prefix, (max_slots + 1) * sizeof(long long));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_hdr, sizeof(BatchHeader));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_err, max_slots * sizeof(unsigned));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_check, 4 * max_slots * sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_stage, b->stage_ints * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_range, 2 * max_slots * sizeof(long long));
    if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_range, 2 * max_slots * sizeof(long long));
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&b->ev1);
    if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, max_slots * sizeof(unsigned), b->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) {
        fqnm_status st = (e == cudaErrorMemoryAllocation)
                             ? set_error(FQNM_ERR_OOM, "batch allocation failed: %s", cudaGetErrorString(e))
                             : cuda_error(e, "fqnm_batch_create");
        batch_free_device(b);
        delete b;
        return st;
    }
    std::memset(b->h_desc, 0, max_slots * sizeof(BatchDesc));
    std::memset(b->h_prefix, 0, (max_slots + 1) * sizeof(long long));
    std::memset(b->h_hdr, 0, sizeof(BatchHeader));
    b->free_blocks[0] = b->budget;
    *out = b;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_destroy(fqnm_batch* b)
{
    if (!b) return FQNM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free_device(b);
    delete b;
    return FQNM_OK;
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
    b->plan = p;
    b->tuning = false;
    if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_batch_autotune(fqnm_batch* b, int epochs_per_plan)
{
    if (!b) return set_error(FQNM_ERR_ARG, "null handle");
    if (epochs_per_plan < 1 || epochs_per_plan > 64)
        return set_error(FQNM_ERR_ARG, "epochs_per_plan must be 1..64");
    b->cands.clear();
    const int vs[2] = {8, 16}, blocks[3] = {32, 128, 256}, ks[3] = {32, 64, 128};
    RuleView dummy{};
    for (int v : vs)
        for (int bl : blocks)
            for (int k : ks) {
                Plan p;
                p.kernel = 2; p.layout = LAYOUT_BLOCKED; p.v = v; p.block = bl; p.k = k;
                if (4LL * k > (long long)bl * v) continue;      // > 50 % halo work
                if (tb_plan_supported(dummy, p)) b->cands.push_back(p);
            }
    b->cand_ns.assign(b->cands.size(), 0.0);
    b->cand_updates.assign(b->cands.size(), 0);
    b->tune_epoch = 0;
    b->tune_per_plan = epochs_per_plan;
    b->tuning = !b->cands.empty();
    if (b->tuning) {
        b->plan = b->cands[0];
        if (b->gexec) { cudaGraphExecDestroy(b->gexec); b->gexec = nullptr; }
    }
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
    *id = (int64_t)b->reqs.size();
    b->reqs.push_back(std::move(r));
    b->queue.push_back(*id);
    return FQNM_OK;
}

// Phase 1 of admission: a slot, the state buffers and the initial state on
// the device; a device submission also gets its state range from the GPU.
static fqnm_status admit_state(fqnm_batch* b, int64_t rid, size_t* stage_used, bool* admitted)
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
        int32_t* stage = b->h_stage + *stage_used;
        std::memcpy(stage, r.q0.data(), n * sizeof(int32_t));
        *stage_used += n;
        BCK(cudaMemcpyAsync(s.q[0], stage, n * sizeof(int32_t), cudaMemcpyHostToDevice, b->stream));
    } else {
        BCK(cudaMemcpyAsync(s.q[0], r.q0_dev, n * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                            b->stream));
        init_minmax(b->h_range + 2 * si);
        BCK(cudaMemcpyAsync(b->d_range + 2 * si, b->h_range + 2 * si, 2 * sizeof(long long),
                            cudaMemcpyHostToDevice, b->stream));
        BCK(launch_minmax_i32(s.q[0], (int64_t)n, b->d_range + 2 * si, b->stream));
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

static fqnm_status build_epoch_graph(fqnm_batch* b)
{
    BatchKernel kern = batch_kernel(b->plan.v, b->plan.layout, b->plan.block);
    int per_sm = 0, sms = 0, dev = 0;
    BCK(cudaGetDevice(&dev));
    BCK(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    BCK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, b->plan.block, 0));
    b->grid = std::max(1, per_sm) * sms;
    cudaStream_t cap = nullptr;
    BCK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_desc, b->h_desc, b->max_slots * sizeof(BatchDesc),
                                              cudaMemcpyHostToDevice, cap);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_prefix, b->h_prefix,
                                              (b->max_slots + 1) * sizeof(long long),
                                              cudaMemcpyHostToDevice, cap);
    if (e == cudaSuccess) e = cudaMemcpyAsync(b->d_hdr, b->h_hdr, sizeof(BatchHeader),
                                              cudaMemcpyHostToDevice, cap);
    if (e == cudaSuccess) {
        kern<<<b->grid, b->plan.block, 0, cap>>>(b->d_desc, b->d_prefix, b->d_hdr);
        e = cudaGetLastError();
    }
    cudaError_t ee = cudaStreamEndCapture(cap, &g);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_error(e, "batch graph capture"); }
    if (ee != cudaSuccess) return cuda_error(ee, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) { b->gexec = nullptr; return cuda_error(e, "cudaGraphInstantiate"); }
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

static fqnm_status run_epoch_body(fqnm_batch* b, bool* did_work)
{
    *did_work = false;
    const uint64_t t = now_ns();
    // 1. admission: states first, then (after one sync if a device
    // submission needs its range) the tables
    size_t stage_used = 0;
    std::vector<int> fresh;
    bool need_range = false;
    for (auto it = b->queue.begin(); it != b->queue.end();) {
        Request& r = b->reqs[*it];
        if (r.arrival_ns > t) { ++it; continue; }
        bool adm = false;
        const int64_t rid = *it;
        fqnm_status st = admit_state(b, rid, &stage_used, &adm);
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
                            cudaMemcpyDeviceToHost, b->stream));
        BCK(cudaStreamSynchronize(b->stream));
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
    if (b->free_slots.size() == (size_t)b->max_slots) {
        for (int64_t rid : b->queue)
            if (b->reqs[rid].arrival_ns <= t)
                return set_error(FQNM_ERR_OOM, "request %lld cannot be admitted into an empty "
                                 "batch (budget %zu bytes)", (long long)rid, b->budget);
    }
    // 2. the epoch's launch over every active problem with steps left
    const long long E = (long long)b->plan.block * b->plan.v;
    int np = 0;
    long long total = 0;
    for (int si = 0; si < b->max_slots; ++si) {
        Slot& s = b->slots[si];
        s.k_this_epoch = 0;
        if (s.req < 0) continue;
        Request& r = b->reqs[s.req];
        if (s.done >= r.steps) continue;
        const int k = (int)std::min<uint64_t>((uint64_t)b->plan.k, r.steps - s.done);
        const long long S = E - 2LL * k;
        const long long n = (long long)r.n;
        BatchDesc& d = b->h_desc[np];
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
        b->h_prefix[np] = total;
        total += (n + S - 1) / S;
        s.k_this_epoch = k;
        ++np;
    }
    b->h_prefix[np] = total;
    b->h_hdr->nprob = np;
    b->h_hdr->total_tiles = total;
    if (np > 0) {
        if (!b->gexec) {
            fqnm_status st = build_epoch_graph(b);
            if (st != FQNM_OK) return st;
        }
        BCK(cudaEventRecord(b->ev0, b->stream));
        BCK(cudaGraphLaunch(b->gexec, b->stream));
        BCK(cudaEventRecord(b->ev1, b->stream));
        note_launches();
        b->launches += 1;
        b->epochs += 1;
        *did_work = true;
    }
    // 3. bookkeeping, copies of finished states, error words, rule checks
    size_t out_used = stage_used;
    std::vector<int> finished;
    for (int si = 0; si < b->max_slots; ++si) {
        Slot& s = b->slots[si];
        if (s.req < 0) continue;
        Request& r = b->reqs[s.req];
        if (s.k_this_epoch) {
            s.done += s.k_this_epoch;
            s.cur = 1 - s.cur;
            b->cell_updates += (uint64_t)s.k_this_epoch * r.n;
        }
        if (s.done >= r.steps && r.out_dev) {
            BCK(cudaMemcpyAsync(r.out_dev, s.q[s.cur], r.n * sizeof(int32_t),
                                cudaMemcpyDeviceToDevice, b->stream));
            finished.push_back(si);
        } else if (s.done >= r.steps && out_used + r.n <= b->stage_ints) {
            BCK(cudaMemcpyAsync(b->h_stage + out_used, s.q[s.cur], r.n * sizeof(int32_t),
                                cudaMemcpyDeviceToHost, b->stream));
            finished.push_back(si);
            s.out_off = out_used;
            out_used += r.n;
        }
        *did_work = *did_work || s.req >= 0;
    }
    BCK(cudaMemcpyAsync(b->h_err, b->d_err, b->max_slots * sizeof(unsigned),
                        cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaMemcpyAsync(b->h_check, b->d_check, 4 * b->max_slots * sizeof(unsigned long long),
                        cudaMemcpyDeviceToHost, b->stream));
    BCK(cudaStreamSynchronize(b->stream));
    const uint64_t tdone = now_ns();
    if (np > 0) {
        float ms = 0.0f;
        BCK(cudaEventElapsedTime(&ms, b->ev0, b->ev1));
        b->gpu_ms += ms;
        if (b->tuning) {
            uint64_t upd = 0;
            for (int i = 0; i < np; ++i) upd += (uint64_t)b->h_desc[i].n * b->h_desc[i].k;
            const size_t c = (size_t)(b->tune_epoch / b->tune_per_plan);
            b->cand_ns[c] += (double)(tdone - t);
            b->cand_updates[c] += upd;
            ++b->tune_epoch;
            const size_t nc = (size_t)(b->tune_epoch / b->tune_per_plan);
            if (nc >= b->cands.size()) {           // all tried: keep the fastest
                size_t best = 0;
                double best_v = 1e300;
                for (size_t j = 0; j < b->cands.size(); ++j) {
                    if (!b->cand_updates[j]) continue;
                    const double v = b->cand_ns[j] / (double)b->cand_updates[j];
                    if (v < best_v) { best_v = v; best = j; }
                }
                b->plan = b->cands[best];
                b->tuning = false;
            } else if (nc != c) {
                b->plan = b->cands[nc];
            }
            if (b->gexec && (nc != c || !b->tuning)) {
                cudaGraphExecDestroy(b->gexec);
                b->gexec = nullptr;
            }
        }
    }
    // rule checks of newly admitted problems
    for (int si = 0; si < b->max_slots; ++si) {
        Slot& s = b->slots[si];
        if (s.req < 0 || !s.check_pending) continue;
        s.check_pending = false;
        const unsigned long long* c = b->h_check + 4 * si;
        s.has_m = (c[1] & CERT_M_NONZERO) != 0;
        if (b->pack16 && c[2] <= 32767 && c[3] <= 32767) {   // both maps fit int16
            BCK(launch_pack_tab16(s.tab2, (int64_t)s.span + 1, s.tab16, b->stream));
            s.use16 = true;
        }
        if (s.cf_candidate && c[0] == 0 && !s.has_m) s.evaluator = EVAL_CLOSED_FORM;
    }
    // errors restart that problem alone from its initial state (wider map)
    for (int si = 0; si < b->max_slots; ++si) {
        Slot& s = b->slots[si];
        if (s.req < 0 || b->h_err[si] == 0) continue;
        Request& r = b->reqs[s.req];
        if (b->h_err[si] & ERRBIT_OVERFLOW)
            return set_error(FQNM_ERR_OVERFLOW, "problem %lld: a transfer does not fit int32",
                             (long long)s.req);
        finished.erase(std::remove(finished.begin(), finished.end(), si), finished.end());
        r.margin = std::max<int64_t>(4 * r.margin, 4096);
        r.state = 0;
        b->queue.push_front(s.req);
        release_slot(b, si);
        BCK(cudaMemsetAsync(b->d_err + si, 0, sizeof(unsigned), b->stream));
    }
    for (int si : finished) {
        Slot& s = b->slots[si];
        Request& r = b->reqs[s.req];
        if (!r.out_dev) r.result.assign(b->h_stage + s.out_off, b->h_stage + s.out_off + r.n);
        r.done_ns = tdone;
        r.state = 2;
        b->completed.push_back(s.req);
        release_slot(b, si);
    }
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
