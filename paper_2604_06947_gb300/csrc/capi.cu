// capi.cu -- the C ABI of libfqnm (include/fqnm.h): handle lifecycle, the
// transfer-rule builder, plan selection, the step loop, invariants and the
// floating-point baseline handle.
//
// Every compute step runs in the kernels of k_*.cu; this file only
// validates arguments, owns device memory and streams, and sequences
// launches.
#include "fqnm_internal.h"
#include "levels.h"
#include "hopf_lax.h"
#include "nd.h"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <map>
#include <mutex>
#include <tuple>
#include <vector>

namespace fqnm {

static thread_local char g_err[1024] = "";
std::atomic<unsigned long long> g_kernel_launches{0};

fqnm_status set_error(fqnm_status st, const char* fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof g_err, fmt, ap);
    va_end(ap);
    return st;
}

fqnm_status cuda_error(cudaError_t e, const char* where)
{
    return set_error(FQNM_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

static bool is_pow2(double d)
{
    if (!(d > 0.0) || !std::isfinite(d)) return false;
    int e;
    return std::frexp(d, &e) == 0.5;
}

static int64_t floor_div(int64_t a, int64_t b)
{
    int64_t q = a / b;
    if ((a % b != 0) && ((a < 0) != (b < 0))) --q;
    return q;
}

static int bit_length(uint64_t x)
{
    int b = 0;
    while (x) { ++b; x >>= 1; }
    return b;
}

// Build the closed form for phi(q) = R(q*num/den) on [lo, hi]; false if the
// 32-bit evaluation would not be exact there.
bool make_closed_form(int64_t lo, int64_t hi, uint32_t num, uint32_t den,
                             int rounding, ClosedForm* out)
{
    if (num == 0 || den == 0 || hi < lo) return false;
    const int64_t twoden = 2 * (int64_t)den;
    const int64_t base = floor_div(lo, twoden) * twoden;
    const int64_t xmax = hi - base;
    if (base < INT32_MIN || xmax > INT32_MAX) return false;
    if ((uint64_t)xmax * num >= (1ull << 31)) return false;
    const uint64_t tmax = (uint64_t)xmax * num;
    const int k = bit_length(tmax * den);           // tmax*den < 2^k
    if (k > 63) return false;
    const uint64_t magic = ((1ull << k) + den - 1) / den;
    if (magic >= (1ull << 32)) return false;
    const int64_t c0 = (base / (int64_t)den) * (int64_t)num;
    if (c0 < INT32_MIN || c0 > INT32_MAX) return false;
    out->base = (int32_t)base;
    out->num = num;
    out->den = den;
    out->magic = (uint32_t)magic;
    out->shift = k;
    out->c0 = (int32_t)c0;
    out->rounding = rounding;
    return true;
}

// Continued-fraction convergents of c > 0 with denominators <= maxden.
std::vector<std::pair<uint32_t, uint32_t>> convergents(double c, uint32_t maxden)
{
    std::vector<std::pair<uint32_t, uint32_t>> out;
    if (!(c > 0.0) || !std::isfinite(c)) return out;
    double x = c;
    long double h1 = 1, h2 = 0, k1 = 0, k2 = 1;
    for (int it = 0; it < 40; ++it) {
        const long double a = std::floor((long double)x);
        const long double h = a * h1 + h2, k = a * k1 + k2;
        if (k > maxden || h > 4.0e9) break;
        out.emplace_back((uint32_t)h, (uint32_t)k);
        const double frac = x - (double)a;
        if (frac < 1e-15) break;
        x = 1.0 / frac;
        h2 = h1; h1 = h; k2 = k1; k1 = k;
    }
    return out;
}

}  // namespace fqnm

using namespace fqnm;

// NVTX range for the duration of a call (tools such as ncu --nvtx see it).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
};

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_error(e_, #call);       \
    } while (0)

// A temporary device buffer, freed on every return path (CK returns early).
template <typename T>
struct DeviceScratch {
    T* p = nullptr;
    DeviceScratch() = default;
    DeviceScratch(const DeviceScratch&) = delete;
    DeviceScratch& operator=(const DeviceScratch&) = delete;
    cudaError_t alloc(size_t count) { return cudaMalloc((void**)&p, count * sizeof(T)); }
    ~DeviceScratch()
    {
        if (p) cudaFree(p);
    }
};

// ============================================================================
// solver handle
// ============================================================================

struct fqnm_solver {
    fqnm_flux flux{};
    int nvars = 1;
    double delta[3] = {1, 1, 1};
    double dx = 0, dt = 0, lambda = 0;
    int boundary = FQNM_BC_PERIODIC;
    bool user_table = false;
    // host callbacks of a custom monotone split, tabulated at load
    fqnm_split_fn fplus = nullptr, fminus = nullptr;
    void* fuser = nullptr;
    std::vector<int32_t> user_p, user_m;
    int64_t user_lo = 0;

    // options
    int opt_kernel = 0, opt_layout = 0, opt_v = 0, opt_block = 0, opt_k = 0, opt_pdl = -1;
    int64_t margin = 1024;
    int closed_form = 1, recover = 1, autotune = 0, use_graph = 1;
    int qmask = 7;                          // Euler: components evolved as integers
    int fp64_mode = 2;                      // Euler: FP64 steps on the integer pipes
    NdGrid grid{1, {0, 1, 1}};              // d > 1: the Cartesian step of Theorem (extension)
    int opt_nd_tile = 0;                    // 2-D tile shape (0: default)
    int nd_tuned_tile = -1, nd_tuned_k = 0; // d-D plan kept by the autotuner (-1: none)
    int verify = 0;                         // check the conserved totals at each sync
    long long mass0[3] = {0, 0, 0};         // totals the check expects (plus boundary transfer)

    // streams
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t cap_stream = nullptr;

    // state
    size_t n = 0, cap_n = 0;
    bool loaded = false;
    void* q[2] = {nullptr, nullptr};
    int cur = 0;
    void* ckpt = nullptr;
    uint64_t ckpt_step = 0;
    // device side of host fields (load_field, observe), kept between calls:
    // a stream-ordered allocation this large went back to the device at each
    // synchronisation and was mapped again by the next call (0.15 to 0.2 ms
    // per 8 MB call against a 0.05 ms copy)
    double* d_stage = nullptr;
    size_t stage_cap = 0;                   // doubles
    long long ckpt_bflux[3] = {0, 0, 0};

    // transfer rule
    int2* tab2 = nullptr;
    int32_t* tabp = nullptr;
    int32_t* tab16 = nullptr;
    int64_t tab_cap = 0;
    int pack16 = -1;                       // option: pack the maps as int16 pairs (-1 auto)
    RuleView rule{};
    fqnm_rule_info info{};
    // the last rule built, reused by a load whose range and settings match:
    // rule_gen counts the calls that can change a rule (options, grid)
    uint64_t rule_gen = 1, built_gen = 0;
    int64_t built_lo = 0, built_hi = -1;

    // device / pinned scratch
    unsigned* d_err = nullptr;
    // d_acc slots: [0,9) invariants of up to 3 variables, [9,12) boundary
    // transfer totals, [12,15) their value at the checkpoint, [16,18) min/max
    long long* d_acc = nullptr;
    unsigned long long* d_check = nullptr; // rule check results
    long long* h_acc = nullptr;            // pinned mirrors
    unsigned* h_err = nullptr;
    unsigned long long* h_check = nullptr;

    // plan and counters
    Plan plan;
    uint64_t step_count = 0, launches = 0, cell_updates = 0;

    // graph of a run of full-depth temporal-blocked launches
    cudaGraphExec_t gexec = nullptr;
    int g_launches = 0, g_k = 0, g_cur = -1;
    Plan g_plan;
    RuleView g_rule{};
    const void* g_q0 = nullptr;

    // level statistics (entropy diagnostics), allocated on first use
    LevelWork* levels = nullptr;
    LevelRecord level_last{};
    bool level_valid = false;

    size_t state_bytes() const { return nvars == 3 ? sizeof(int64_t) : sizeof(int32_t); }
};

enum { ACC_BFLUX = 9, ACC_BFLUX_CKPT = 12, ACC_MINMAX = 16, ACC_SLOTS = 24 };

static void replan(fqnm_solver* s);

static void destroy_graph(fqnm_solver* s)
{
    if (s->gexec) cudaGraphExecDestroy(s->gexec);
    s->gexec = nullptr;
    s->g_cur = -1;
}

static fqnm_status ensure_runtime(fqnm_solver* s)
{
    if (!s->d_err) {
        int ndev = 0;
        cudaError_t e = cudaGetDeviceCount(&ndev);
        if (e != cudaSuccess || ndev == 0)
            return set_error(FQNM_ERR_CUDA, "no CUDA device available (%s)",
                             cudaGetErrorString(e));
        CK(cudaMalloc(&s->d_err, sizeof(unsigned)));
        CK(cudaMalloc(&s->d_acc, ACC_SLOTS * sizeof(long long)));
        CK(cudaMalloc(&s->d_check, 4 * sizeof(unsigned long long)));
        CK(cudaMallocHost(&s->h_acc, ACC_SLOTS * sizeof(long long)));
        CK(cudaMallocHost(&s->h_err, sizeof(unsigned)));
        CK(cudaMallocHost(&s->h_check, 4 * sizeof(unsigned long long)));
        CK(cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking));
        if (!s->stream) {
            CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
            s->own_stream = true;
        }
        CK(cudaMemsetAsync(s->d_err, 0, sizeof(unsigned), s->stream));
        CK(cudaMemsetAsync(s->d_acc, 0, ACC_SLOTS * sizeof(long long), s->stream));
    }
    return FQNM_OK;
}

static fqnm_status check_flux(const fqnm_flux* f, const double* delta, double dx,
                              double dt, int boundary, int* nvars)
{
    if (!f || !delta) return set_error(FQNM_ERR_ARG, "null flux or delta");
    if (!(dx > 0) || !(dt > 0) || !std::isfinite(dx) || !std::isfinite(dt))
        return set_error(FQNM_ERR_ARG, "dx and dt must be positive and finite");
    if (boundary != FQNM_BC_PERIODIC && boundary != FQNM_BC_TRANSMISSIVE)
        return set_error(FQNM_ERR_ARG, "unknown boundary %d", boundary);
    if (f->rounding < FQNM_ROUND_HALF_EVEN || f->rounding > FQNM_ROUND_FLOOR)
        return set_error(FQNM_ERR_ARG, "unknown rounding %d", f->rounding);
    const double lam = dt / dx;
    double nu = 0;
    switch (f->kind) {
    case FQNM_FLUX_LINEAR_UPWIND:
        nu = std::fabs(f->a) * lam;
        *nvars = 1;
        break;
    case FQNM_FLUX_LINEAR_LF:
        if (!(f->alpha >= std::fabs(f->a)))
            return set_error(FQNM_ERR_ARG, "LF needs alpha >= |a| (alpha=%g, a=%g)", f->alpha, f->a);
        nu = f->alpha * lam;
        *nvars = 1;
        break;
    case FQNM_FLUX_BURGERS_LF:
        if (!(f->alpha > 0))
            return set_error(FQNM_ERR_ARG, "BURGERS_LF needs alpha > 0 (alpha >= max|u|)");
        nu = f->alpha * lam;
        *nvars = 1;
        break;
    case FQNM_FLUX_BURGERS_EO:
    case FQNM_FLUX_BURGERS_GODUNOV:
        if (!(f->alpha > 0))
            return set_error(FQNM_ERR_ARG, "BURGERS_EO/GODUNOV need alpha = max|u| > 0 for the CFL check");
        nu = f->alpha * lam;
        *nvars = 1;
        break;
    case FQNM_FLUX_EULER_ROE:
        if (!(f->gamma > 1.0)) return set_error(FQNM_ERR_ARG, "EULER_ROE needs gamma > 1");
        *nvars = 3;
        nu = 0;           // state dependent; not checked here
        break;
    default:
        return set_error(FQNM_ERR_ARG, "unknown flux kind %d", f->kind);
    }
    if (nu > 1.0)
        return set_error(FQNM_ERR_CFL, "Courant number %.17g > 1 (eq. cfl_number)", nu);
    for (int v = 0; v < *nvars; ++v)
        if (!is_pow2(delta[v]))
            return set_error(FQNM_ERR_ARG, "delta[%d] = %g is not a power of two", v, delta[v]);
    if (*nvars == 3 && boundary != FQNM_BC_TRANSMISSIVE)
        return set_error(FQNM_ERR_ARG, "EULER_ROE supports transmissive ends only");
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_create(const fqnm_flux* flux, const double* delta,
                                   double dx, double dt, int boundary,
                                   fqnm_solver** out)
{
    if (!out) return set_error(FQNM_ERR_ARG, "null out");
    *out = nullptr;
    int nvars = 1;
    fqnm_status st = check_flux(flux, delta, dx, dt, boundary, &nvars);
    if (st != FQNM_OK) return st;
    fqnm_solver* s = new (std::nothrow) fqnm_solver();
    if (!s) return set_error(FQNM_ERR_OOM, "host allocation failed");
    s->flux = *flux;
    s->nvars = nvars;
    for (int v = 0; v < nvars; ++v) s->delta[v] = delta[v];
    s->dx = dx;
    s->dt = dt;
    s->lambda = dt / dx;
    s->boundary = boundary;
    *out = s;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_create_custom(fqnm_split_fn fplus, fqnm_split_fn fminus, void* user,
                                          double alpha, double delta, double dx, double dt,
                                          int boundary, int rounding, fqnm_solver** out)
{
    if (!out) return set_error(FQNM_ERR_ARG, "null out");
    *out = nullptr;
    if (!fplus || !fminus) return set_error(FQNM_ERR_ARG, "null callback");
    // the CFL check of a split with max|f'| <= alpha
    fqnm_flux f{};
    f.kind = FQNM_FLUX_BURGERS_LF;
    f.alpha = alpha;
    f.rounding = rounding;
    int nvars = 1;
    fqnm_status st = check_flux(&f, &delta, dx, dt, boundary, &nvars);
    if (st != FQNM_OK) return st;
    fqnm_solver* s = new (std::nothrow) fqnm_solver();
    if (!s) return set_error(FQNM_ERR_OOM, "host allocation failed");
    f.kind = FQNM_FLUX_CUSTOM_SPLIT;
    s->flux = f;
    s->fplus = fplus;
    s->fminus = fminus;
    s->fuser = user;
    s->delta[0] = delta;
    s->dx = dx;
    s->dt = dt;
    s->lambda = dt / dx;
    s->boundary = boundary;
    *out = s;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_create_table(const int32_t* phi_p, const int32_t* phi_m,
                                         int64_t lo, int64_t count, double delta,
                                         int boundary, fqnm_solver** out)
{
    if (!out) return set_error(FQNM_ERR_ARG, "null out");
    *out = nullptr;
    if (!phi_p || !phi_m || count <= 0 || count > (1ll << 30))
        return set_error(FQNM_ERR_ARG, "bad table arguments");
    if (lo < INT32_MIN / 2 || lo + count > INT32_MAX / 2)
        return set_error(FQNM_ERR_ARG, "table range must lie within +-2^30");
    if (!is_pow2(delta)) return set_error(FQNM_ERR_ARG, "delta is not a power of two");
    if (boundary != FQNM_BC_PERIODIC && boundary != FQNM_BC_TRANSMISSIVE)
        return set_error(FQNM_ERR_ARG, "unknown boundary %d", boundary);
    fqnm_solver* s = new (std::nothrow) fqnm_solver();
    if (!s) return set_error(FQNM_ERR_OOM, "host allocation failed");
    s->flux.kind = FQNM_FLUX_TABLE;
    s->nvars = 1;
    s->delta[0] = delta;
    s->dx = s->dt = 1.0;
    s->lambda = 1.0;
    s->boundary = boundary;
    s->user_table = true;
    s->user_p.assign(phi_p, phi_p + count);
    s->user_m.assign(phi_m, phi_m + count);
    s->user_lo = lo;
    *out = s;
    return FQNM_OK;
}

// The staging buffer for `count` doubles (grown when needed; the stream is
// drained before an old buffer is released).
static fqnm_status stage_buffer(fqnm_solver* s, size_t count, double** out)
{
    if (count > s->stage_cap) {
        if (s->d_stage) {
            CK(cudaStreamSynchronize(s->stream));
            cudaFree(s->d_stage);
        }
        s->d_stage = nullptr;
        s->stage_cap = 0;
        CK(cudaMalloc((void**)&s->d_stage, count * sizeof(double)));
        s->stage_cap = count;
    }
    *out = s->d_stage;
    return FQNM_OK;
}

static void free_state(fqnm_solver* s)
{
    for (int b = 0; b < 2; ++b) {
        if (s->q[b]) cudaFree(s->q[b]);
        s->q[b] = nullptr;
    }
    if (s->ckpt) cudaFree(s->ckpt);
    s->ckpt = nullptr;
    s->cap_n = 0;
}

extern "C" fqnm_status fqnm_destroy(fqnm_solver* s)
{
    if (!s) return FQNM_OK;
    if (s->stream) cudaStreamSynchronize(s->stream);
    destroy_graph(s);
    level_work_destroy(s->levels);
    free_state(s);
    if (s->d_stage) cudaFree(s->d_stage);
    if (s->tab2) cudaFree(s->tab2);
    if (s->tabp) cudaFree(s->tabp);
    if (s->tab16) cudaFree(s->tab16);
    if (s->d_err) cudaFree(s->d_err);
    if (s->d_acc) cudaFree(s->d_acc);
    if (s->d_check) cudaFree(s->d_check);
    if (s->h_acc) cudaFreeHost(s->h_acc);
    if (s->h_err) cudaFreeHost(s->h_err);
    if (s->h_check) cudaFreeHost(s->h_check);
    if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    delete s;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_set_stream(fqnm_solver* s, void* stream)
{
    if (!s) return set_error(FQNM_ERR_ARG, "null handle");
    if (s->stream) {
        cudaError_t e = cudaStreamSynchronize(s->stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize");
    }
    if (s->own_stream && s->stream) cudaStreamDestroy(s->stream);
    s->own_stream = false;
    s->stream = (cudaStream_t)stream;
    if (!stream && s->d_err) {
        CK(cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking));
        s->own_stream = true;
    }
    return FQNM_OK;
}

static fqnm_status sync_and_check(fqnm_solver* s);
static fqnm_status set_expected_totals(fqnm_solver* s);

extern "C" fqnm_status fqnm_set_option(fqnm_solver* s, int option, int64_t value)
{
    if (!s) return set_error(FQNM_ERR_ARG, "null handle");
    ++s->rule_gen;                          // the next load builds its rule afresh
    switch (option) {
    case FQNM_OPT_KERNEL:
        if (value < 0 || value > 4 || value == 3)
            return set_error(FQNM_ERR_ARG, "kernel must be 0, 1, 2 or 4");
        s->opt_kernel = (int)value; break;
    case FQNM_OPT_LAYOUT:
        if (value < 0 || value > 4) return set_error(FQNM_ERR_ARG, "layout must be 0..4");
        s->opt_layout = (int)value; break;
    case FQNM_OPT_CELLS_PER_THREAD:
        if (value != 0 && value != 4 && value != 8 && value != 16 && value != 32)
            return set_error(FQNM_ERR_ARG, "cells per thread must be 0, 4, 8, 16 or 32");
        s->opt_v = (int)value; break;
    case FQNM_OPT_BLOCK:
        if (value != 0 && (value < 32 || value > 512 || value % 32))
            return set_error(FQNM_ERR_ARG, "block must be 0 or a multiple of 32 in [32, 512]");
        s->opt_block = (int)value; break;
    case FQNM_OPT_K:
        if (value < 0 || value > 4096) return set_error(FQNM_ERR_ARG, "K must be in [0, 4096]");
        s->opt_k = (int)value; break;
    case FQNM_OPT_MARGIN:
        if (value < 0 || value > (1ll << 28)) return set_error(FQNM_ERR_ARG, "margin out of range");
        s->margin = value; break;
    case FQNM_OPT_CLOSED_FORM: s->closed_form = value != 0; break;
    case FQNM_OPT_RECOVER: s->recover = value != 0; break;
    case FQNM_OPT_AUTOTUNE: s->autotune = value != 0; break;
    case FQNM_OPT_GRAPH: s->use_graph = value != 0; break;
    case FQNM_OPT_PACK16: s->pack16 = value < 0 ? -1 : value != 0; break;
    case FQNM_OPT_VERIFY: {
        s->verify = value != 0;
        if (s->verify && s->loaded) {            // expect the totals as they stand now
            fqnm_status st = sync_and_check(s);
            if (st != FQNM_OK) return st;
            st = set_expected_totals(s);
            if (st != FQNM_OK) return st;
        }
        break;
    }
    case FQNM_OPT_ND_TILE:
        if (value < 0 || value > ND_WALK) return set_error(FQNM_ERR_ARG, "2-D plan 0..6");
        s->opt_nd_tile = (int)value; break;
    case FQNM_OPT_QUANTISE_MASK:
        if (value < 0 || value > 7) return set_error(FQNM_ERR_ARG, "mask must be 0..7");
        if (s->nvars != 3) return set_error(FQNM_ERR_ARG, "the mask applies to EULER_ROE");
        if (s->loaded) return set_error(FQNM_ERR_STATE, "set the mask before loading");
        s->qmask = (int)value; break;
    case FQNM_OPT_PDL:
        if (value < 0 || value > 1) return set_error(FQNM_ERR_ARG, "pdl must be 0 or 1");
        s->opt_pdl = (int)value; break;
    case FQNM_OPT_FP64:
        if (value < 0 || value > 3) return set_error(FQNM_ERR_ARG, "fp64 mode must be 0..3");
        s->fp64_mode = (int)value; break;
    default: return set_error(FQNM_ERR_ARG, "unknown option %d", option);
    }
    if (s->loaded && s->nvars == 1 && option <= FQNM_OPT_K) {
        destroy_graph(s);
        replan(s);          // the new overrides take effect at the next step
    }
    return FQNM_OK;
}

// ============================================================================
// transfer-rule builder
// ============================================================================

static fqnm_status read_check(fqnm_solver* s, const ClosedForm* cf, int64_t lo,
                              int64_t count)
{
    CK(cudaMemsetAsync(s->d_check, 0, 4 * sizeof(unsigned long long), s->stream));
    CK(launch_rule_check(s->tab2, lo, count, cf, s->d_check, s->stream));
    CK(cudaMemcpyAsync(s->h_check, s->d_check, 4 * sizeof(unsigned long long),
                       cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    return FQNM_OK;
}

// Tabulate the maps over [lo, hi] and choose the evaluator.
// eq. flux_table for host callbacks, in the order of the built-in maps:
// u = delta*q (exact), t = f(u), s = t*lambda, phi = R(s*(1/delta)).
static fqnm_status tabulate_custom(fqnm_solver* s, int64_t lo, int64_t count)
{
    s->user_p.resize((size_t)count);
    s->user_m.resize((size_t)count);
    const double inv = 1.0 / s->delta[0];
    for (int64_t k = 0; k < count; ++k) {
        const double u = s->delta[0] * (double)(lo + k);
        double fp = s->fplus(u, s->fuser), fm = s->fminus(u, s->fuser);
        double vp = (fp * s->lambda) * inv, vm = (fm * s->lambda) * inv;
        switch (s->flux.rounding) {
        case FQNM_ROUND_HALF_AWAY: vp = std::round(vp); vm = std::round(vm); break;
        case FQNM_ROUND_FLOOR: vp = std::floor(vp); vm = std::floor(vm); break;
        default: vp = std::nearbyint(vp); vm = std::nearbyint(vm); break;
        }
        if (!(std::fabs(vp) < 1.0e9) || !(std::fabs(vm) < 1.0e9))
            return set_error(FQNM_ERR_OVERFLOW, "custom map at q = %lld is %g, %g",
                             (long long)(lo + k), vp, vm);
        s->user_p[(size_t)k] = (int32_t)vp;
        s->user_m[(size_t)k] = (int32_t)vm;
    }
    return FQNM_OK;
}

static fqnm_status build_rule(fqnm_solver* s, int64_t lo, int64_t hi)
{
    // the maps are functions of the state alone: the same range under the
    // same settings gives the same tables, checks and closed form (custom
    // split callbacks are tabulated again every time: they are the caller's)
    if (s->built_gen == s->rule_gen && lo == s->built_lo && hi == s->built_hi && !s->fplus)
        return FQNM_OK;
    s->built_gen = 0;
    const int64_t count = hi - lo + 1;
    if (count <= 0 || count > (1ll << 30))
        return set_error(FQNM_ERR_RANGE, "transfer-map range [%lld, %lld] too large",
                         (long long)lo, (long long)hi);
    if (lo < INT32_MIN || hi > INT32_MAX)
        return set_error(FQNM_ERR_OVERFLOW, "state range exceeds int32");
    if (count > s->tab_cap) {
        if (s->tab2) cudaFree(s->tab2);
        if (s->tabp) cudaFree(s->tabp);
        if (s->tab16) cudaFree(s->tab16);
        s->tab2 = nullptr;
        s->tabp = nullptr;
        s->tab16 = nullptr;
        s->tab_cap = 0;
        CK(cudaMalloc(&s->tab2, count * sizeof(int2)));
        CK(cudaMalloc(&s->tabp, count * sizeof(int32_t)));
        CK(cudaMalloc(&s->tab16, count * sizeof(int32_t)));
        s->tab_cap = count;
    }
    CK(cudaMemsetAsync(s->d_err, 0, sizeof(unsigned), s->stream));
    if (s->fplus) {                 // custom split: eq. flux_table on the host, same order
        fqnm_status st = tabulate_custom(s, lo, count);
        if (st != FQNM_OK) return st;
    }
    if (s->user_table || s->fplus) {
        DeviceScratch<int32_t> dp, dm;
        CK(dp.alloc(count));
        CK(dm.alloc(count));
        CK(cudaMemcpyAsync(dp.p, s->user_p.data(), count * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s->stream));
        CK(cudaMemcpyAsync(dm.p, s->user_m.data(), count * sizeof(int32_t),
                           cudaMemcpyHostToDevice, s->stream));
        CK(launch_copy_user_table(dp.p, dm.p, count, s->tab2, s->tabp, s->stream));
        CK(cudaStreamSynchronize(s->stream));
    } else {
        // Godunov steps with the Engquist-Osher maps (and a max at each face)
        const int table_kind = s->flux.kind == FQNM_FLUX_BURGERS_GODUNOV ? FQNM_FLUX_BURGERS_EO
                                                                        : s->flux.kind;
        CK(launch_build_split_table(table_kind, s->flux.a, s->flux.alpha, s->delta[0],
                                    s->lambda, s->flux.rounding, lo, count, s->tab2,
                                    s->tabp, s->d_err, s->stream));
    }
    CK(cudaMemcpyAsync(s->h_err, s->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
    fqnm_status st = read_check(s, nullptr, lo, count);
    if (st != FQNM_OK) return st;
    if (*s->h_err & ERRBIT_OVERFLOW)
        return set_error(FQNM_ERR_OVERFLOW, "a transfer-map value does not fit int32");
    const unsigned long long flags = s->h_check[1];
    const long long maxp = (long long)s->h_check[2], maxm = (long long)s->h_check[3];
    // one step from inside [lo, hi] must not overflow int32: an update moves a
    // state by at most 2 d (max|phi+| + max|phi-|) on a d-D grid (the d-D
    // kernels sum in int32 and rely on this)
    const long long reach = 2LL * std::max(1, s->grid.d) * (maxp + maxm);
    if (hi + reach >= INT32_MAX || lo - reach <= INT32_MIN)
        return set_error(FQNM_ERR_OVERFLOW, "state range too close to the int32 limits");

    RuleView r{};
    r.tab2 = s->tab2;
    r.tabp = s->tabp;
    r.tab16 = nullptr;
    // both maps fit int16: the packed table halves the gather footprint
    // (by default on d-D grids, whose gathers miss L1 more often)
    const bool pack = s->pack16 > 0 || (s->pack16 < 0 && s->grid.d > 1);
    if (pack && maxp <= 32767 && maxm <= 32767) {
        CK(launch_pack_tab16(s->tab2, count, s->tab16, s->stream));
        r.tab16 = s->tab16;
    }
    r.lo = (int32_t)lo;
    r.span = (uint32_t)(count - 1);
    r.evaluator = EVAL_TABLE;
    r.has_p = (flags & CERT_P_NONZERO) != 0;
    r.has_m = (flags & CERT_M_NONZERO) != 0;
    r.face_max = s->flux.kind == FQNM_FLUX_BURGERS_GODUNOV;

    fqnm_rule_info info{};
    info.lo = lo;
    info.hi = hi;
    info.evaluator = EVAL_TABLE;
    info.has_plus = r.has_p;
    info.has_minus = r.has_m;
    info.monotone = (flags & (CERT_P_NOT_MONOTONE | CERT_M_NOT_MONOTONE | CERT_H_NOT_MONOTONE)) == 0;
    info.recoveries = s->info.recoveries;

    // Integer closed form for a linear map (phi- == 0 on the range): propose
    // the convergents of the multiplier and keep the first one the GPU finds
    // identical to the table at every entry.
    const bool linear = s->flux.kind == FQNM_FLUX_LINEAR_UPWIND ||
                        s->flux.kind == FQNM_FLUX_LINEAR_LF;
    if (s->closed_form && linear && !r.has_m && r.has_p) {
        double c = s->flux.kind == FQNM_FLUX_LINEAR_UPWIND
                       ? std::max(s->flux.a, 0.0) * s->lambda
                       : 0.5 * (s->flux.a + s->flux.alpha) * s->lambda;
        for (auto& nd : convergents(c, 1u << 12)) {
            ClosedForm cf;
            if (!make_closed_form(lo, hi, nd.first, nd.second, s->flux.rounding, &cf)) continue;
            st = read_check(s, &cf, lo, count);
            if (st != FQNM_OK) return st;
            if (s->h_check[0] == 0) {
                r.evaluator = EVAL_CLOSED_FORM;
                r.cf = cf;
                info.evaluator = EVAL_CLOSED_FORM;
                info.num = nd.first;
                info.den = nd.second;
                info.closed_form_sign = +1;
                break;
            }
        }
    }
    s->rule = r;
    s->info = info;
    s->built_gen = s->rule_gen;
    s->built_lo = lo;
    s->built_hi = hi;
    return FQNM_OK;
}

// ============================================================================
// plans
// ============================================================================

static void replan(fqnm_solver* s)
{
    Plan p;
    const bool table = s->rule.evaluator == EVAL_TABLE;
    p.kernel = s->boundary == FQNM_BC_PERIODIC ? 2 : 1;
    if (s->opt_kernel == 1) p.kernel = 1;
    if (s->opt_kernel == 2 && s->boundary == FQNM_BC_PERIODIC) p.kernel = 2;
    // a short periodic line fits one block: every step of a call in one
    // launch.  Asked for, or by default up to RESIDENT_AUTO_CELLS when no
    // temporal-blocked plan parameter was set: one block's step latency
    // (about 140 ns at 256 cells, 210 ns at 1024) beats the tiled kernel's
    // launches (about 5 us per 32 steps) only on the shortest lines.
    const bool tb_opts = s->opt_layout || s->opt_v || s->opt_block || s->opt_k;
    if (s->boundary == FQNM_BC_PERIODIC && s->grid.d == 1 && s->nvars == 1 &&
        resident_v((int64_t)s->n) > 0 &&
        (s->opt_kernel == 4 ||
         (s->opt_kernel == 0 && !tb_opts && s->n <= (size_t)RESIDENT_AUTO_CELLS)))
        p.kernel = 4;
    // defaults, measured on the 2^20-cell Burgers line (table) and the
    // 2^24-cell upwind line (closed form): a table map gathers once per cell
    // and step, and a warp-wide gather over 256 neighbouring cells (runs of
    // 8, two per lane) keeps the L1 sectors per gather low while a cell's
    // neighbours stay mostly in the thread (1.89e12 against 1.78e12 cell
    // updates/s for 8 cells per lane, blocked, 4 warps); a closed form has no
    // gather, and the blocked layout's two shuffles per lane and step win
    // (a line of fewer than 2^18 cells fills few tiles; there the shorter
    // per-step latency of 8 cells per lane and 4-warp blocks wins)
    const bool runs = table && s->n >= ((size_t)1 << 18);
    p.layout = s->opt_layout ? s->opt_layout : (runs ? LAYOUT_RUNS8 : LAYOUT_BLOCKED);
    p.v = s->opt_v ? s->opt_v : (runs ? 16 : 8);
    p.block = s->opt_block ? s->opt_block : (runs ? 64 : 128);
    p.k = s->opt_k ? s->opt_k : 64;
    if (p.layout == LAYOUT_RUNS8 && p.v < 16) p.layout = LAYOUT_BLOCKED;
    if (p.layout == LAYOUT_RUNS4 && p.v < 8) p.layout = LAYOUT_BLOCKED;
    p.pdl = s->opt_pdl < 0 ? 1 : s->opt_pdl;
    const long long E = (long long)p.block * p.v;
    if (2LL * p.k >= E) p.k = (int)std::max(1LL, (E - 1) / 2);
    if (p.kernel == 2 && !tb_plan_supported(s->rule, p)) p.kernel = 1;
    s->plan = p;
}

// Time a candidate plan: `launches` launches that evolve a scratch copy of
// the current state (ping-pong between two scratch buffers); seconds per step.
static float time_plan(fqnm_solver* s, const Plan& p, int launches, int32_t* sa, int32_t* sb)
{
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    cudaMemcpyAsync(sa, s->q[s->cur], s->n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s->stream);
    launch_step_tb(s->rule, p, sa, sb, (int64_t)s->n, p.k, s->d_err, s->stream);   // warm-up
    cudaEventRecord(a, s->stream);
    for (int i = 0; i < launches; ++i) {
        launch_step_tb(s->rule, p, (i & 1) ? sb : sa, (i & 1) ? sa : sb, (int64_t)s->n, p.k,
                       s->d_err, s->stream);
    }
    cudaEventRecord(b, s->stream);
    cudaEventSynchronize(b);
    float ms = 0;
    cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return ms / (launches * (float)p.k);           // per step
}

struct TuneKey {
    int64_t nclass;
    int evaluator, has_m;
    bool operator<(const TuneKey& o) const
    {
        return std::tie(nclass, evaluator, has_m) < std::tie(o.nclass, o.evaluator, o.has_m);
    }
};
static std::mutex g_tune_mu;
static std::map<TuneKey, Plan> g_tune_cache;
static bool g_tune_file_read = false;

// FQNM_TUNE_CACHE=<file>: tuned plans persist across processes, one line per
// key: "nclass evaluator has_m layout v block k pdl".  Read once (lines that
// do not parse, or name an unsupported plan, are ignored); rewritten
// whenever a plan is tuned.  Called with g_tune_mu held.
static void read_tune_file()
{
    if (g_tune_file_read) return;
    g_tune_file_read = true;
    const char* path = std::getenv("FQNM_TUNE_CACHE");
    if (!path || !*path) return;
    FILE* f = std::fopen(path, "r");
    if (!f) return;
    long long nc;
    int ev, hm, layout, v, block, k, pdl;
    while (std::fscanf(f, "%lld %d %d %d %d %d %d %d", &nc, &ev, &hm, &layout, &v, &block, &k,
                       &pdl) == 8) {
        Plan p;
        p.kernel = 2;
        p.layout = layout;
        p.v = v;
        p.block = block;
        p.k = k;
        p.pdl = pdl != 0;
        RuleView none{};
        if (!tb_plan_supported(none, p)) continue;
        g_tune_cache[TuneKey{nc, ev, hm}] = p;
    }
    std::fclose(f);
}

static void write_tune_file()
{
    const char* path = std::getenv("FQNM_TUNE_CACHE");
    if (!path || !*path) return;
    const std::string tmp = std::string(path) + ".tmp";
    FILE* f = std::fopen(tmp.c_str(), "w");
    if (!f) return;
    for (const auto& kv : g_tune_cache)
        std::fprintf(f, "%lld %d %d %d %d %d %d %d\n", (long long)kv.first.nclass,
                     kv.first.evaluator, kv.first.has_m, kv.second.layout, kv.second.v,
                     kv.second.block, kv.second.k, kv.second.pdl ? 1 : 0);
    std::fclose(f);
    std::rename(tmp.c_str(), path);
}

// d-D plans: every walk depth the kernels support, (2-D) every register
// tile at K = 2, 3, 4 and (3-D) the one-step streaming kernel, each timed
// twice (interleaved) over about 32 steps that evolve scratch copies of the
// loaded state.  The default plan (the walk at K = 4 in 2-D, the one-step
// kernel in 3-D) stays unless another is more than 3 % faster per step:
// short timings on a large grid drift by about that much.
static fqnm_status autotune_nd(fqnm_solver* s)
{
    if (s->opt_kernel == 1 || s->opt_nd_tile != 0 || s->opt_k != 0) return FQNM_OK;
    struct Cand { int tile, k; };
    std::vector<Cand> cands;
    if (s->grid.d == 2) {
        for (int k : {2, 3, 4, 6, 8}) cands.push_back({ND_WALK, k});
        for (int t = 1; t <= 5; ++t)
            for (int k : {2, 3, 4}) cands.push_back({t, k});
    } else {
        cands.push_back({0, 1});                      // one step per launch
        for (int k = 1; k <= 4; ++k) cands.push_back({ND_WALK, k});
    }
    DeviceScratch<int32_t> scratch;
    CK(scratch.alloc(s->n));
    int32_t* sa = (int32_t*)s->ckpt;              // restored by the caller
    int32_t* sb = scratch.p;
    cudaEvent_t a, b;
    CK(cudaEventCreate(&a));
    CK(cudaEventCreate(&b));
    auto launch = [&](const Cand& c, const int32_t* in, int32_t* out) {
        if (c.tile == 0) return launch_step_nd(s->rule, in, out, s->grid, s->d_err, s->stream);
        if (c.tile == ND_WALK)
            return s->grid.d == 3 ? launch_walk3d(s->rule, in, out, s->grid, c.k, s->d_err, s->stream)
                                  : launch_walk2d(s->rule, in, out, s->grid, c.k, s->d_err, s->stream);
        NdPlan p;
        p.blocked = 1;
        p.walk = 0;
        p.shape = c.tile;
        p.k = c.k;
        return launch_step2d_tb(s->rule, p, in, out, s->grid, c.k, s->d_err, s->stream);
    };
    std::vector<float> best(cands.size(), 1e30f);
    cudaError_t e = cudaSuccess;
    for (int rep = 0; rep < 2 && e == cudaSuccess; ++rep)
        for (size_t i = 0; i < cands.size() && e == cudaSuccess; ++i) {
            const Cand& c = cands[i];
            const int launches = std::max(2, 32 / c.k);
            e = cudaMemcpyAsync(sa, s->q[s->cur], s->n * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                                s->stream);
            if (e == cudaSuccess) e = launch(c, sa, sb);                    // warm-up
            if (e == cudaSuccess) e = cudaEventRecord(a, s->stream);
            for (int j = 0; j < launches && e == cudaSuccess; ++j)
                e = launch(c, (j & 1) ? sb : sa, (j & 1) ? sa : sb);
            if (e == cudaSuccess) e = cudaEventRecord(b, s->stream);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0;
            if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
            if (e == cudaSuccess) best[i] = std::min(best[i], ms / (launches * (float)c.k));
        }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (e != cudaSuccess) return cuda_error(e, "autotune_nd");
    const Cand dc = s->grid.d == 3 ? Cand{0, 1} : Cand{ND_WALK, 4};
    size_t dflt = 0, pick = 0;
    for (size_t i = 0; i < cands.size(); ++i) {
        if (cands[i].tile == dc.tile && cands[i].k == dc.k) dflt = i;
        if (best[i] < best[pick]) pick = i;
    }
    if (best[pick] * 1.03f > best[dflt]) pick = dflt;
    s->nd_tuned_tile = cands[pick].tile;
    s->nd_tuned_k = cands[pick].k;
    CK(cudaMemsetAsync(s->d_err, 0, sizeof(unsigned), s->stream));
    return FQNM_OK;
}

static fqnm_status autotune(fqnm_solver* s)
{
    if (s->grid.d > 1) return autotune_nd(s);
    if (s->plan.kernel != 2) return FQNM_OK;
    TuneKey key{(int64_t)bit_length((uint64_t)s->n), s->rule.evaluator, s->rule.has_m};
    {
        std::lock_guard<std::mutex> g(g_tune_mu);
        read_tune_file();
        auto it = g_tune_cache.find(key);
        if (it != g_tune_cache.end()) {
            s->plan = it->second;
            return FQNM_OK;
        }
    }
    // stage 1: screen every candidate on a few launches from the loaded
    // state; stage 2: re-time the six fastest over about 1000 evolving steps
    DeviceScratch<int32_t> scratch;
    CK(scratch.alloc(s->n));
    int32_t* sb = scratch.p;
    int32_t* sa = (int32_t*)s->ckpt;              // restored by the caller
    std::vector<std::pair<float, Plan>> screened;
    const int layouts[4] = {LAYOUT_INTERLEAVED, LAYOUT_BLOCKED, LAYOUT_RUNS4, LAYOUT_RUNS8};
    const int vs[4] = {4, 8, 16, 32};
    const int blocks[5] = {32, 64, 128, 256, 512};
    const int ks[5] = {8, 16, 32, 64, 128};
    for (int L : layouts)
        for (int v : vs)
            for (int b : blocks)
                for (int k : ks) {
                    Plan p;
                    p.kernel = 2; p.layout = L; p.v = v; p.block = b; p.k = k;
                    p.pdl = s->plan.pdl;
                    if (!tb_plan_supported(s->rule, p)) continue;
                    if (4LL * k > (long long)b * v) continue;   // >50% redundant work
                    screened.emplace_back(time_plan(s, p, 3, sa, sb), p);
                }
    std::sort(screened.begin(), screened.end(),
              [](const std::pair<float, Plan>& x, const std::pair<float, Plan>& y) {
                  return x.first < y.first;
              });
    // finalists: the six fastest screened plans and the default plan, each
    // timed three times (interleaved) over ~2000 evolving steps; the default
    // stays unless another plan's median is more than 2 % faster
    const Plan dflt = s->plan;
    std::vector<Plan> fin;
    fin.push_back(dflt);
    for (size_t i = 0; i < screened.size() && fin.size() < 7; ++i) {
        const Plan& p = screened[i].second;
        if (p.layout == dflt.layout && p.v == dflt.v && p.block == dflt.block && p.k == dflt.k)
            continue;
        fin.push_back(p);
    }
    std::vector<std::vector<float>> ts(fin.size());
    for (int rep = 0; rep < 3; ++rep)
        for (size_t i = 0; i < fin.size(); ++i)
            ts[i].push_back(time_plan(s, fin[i], std::max(4, 2048 / fin[i].k), sa, sb));
    auto median = [](std::vector<float> v) {
        std::sort(v.begin(), v.end());
        return v[v.size() / 2];
    };
    Plan best = dflt;
    float best_t = median(ts[0]) / 1.02f;
    for (size_t i = 1; i < fin.size(); ++i) {
        const float t = median(ts[i]);
        if (t < best_t) { best_t = t; best = fin[i]; }
    }
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(s->d_err, 0, sizeof(unsigned), s->stream));
    s->plan = best;
    std::lock_guard<std::mutex> g(g_tune_mu);
    g_tune_cache[key] = best;
    write_tune_file();
    return FQNM_OK;
}

// ============================================================================
// loading, stepping, recovery
// ============================================================================

static fqnm_status alloc_state(fqnm_solver* s, size_t n)
{
    const size_t bytes = n * s->state_bytes() * s->nvars;
    if (n > s->cap_n) {
        destroy_graph(s);
        free_state(s);
        for (int b = 0; b < 2; ++b) CK(cudaMalloc(&s->q[b], bytes));
        CK(cudaMalloc(&s->ckpt, bytes));
        s->cap_n = n;
    }
    s->n = n;
    return FQNM_OK;
}

static fqnm_status state_range(fqnm_solver* s, const void* q, int64_t* lo, int64_t* hi)
{
    init_minmax(s->h_acc + ACC_MINMAX);
    CK(cudaMemcpyAsync(s->d_acc + ACC_MINMAX, s->h_acc + ACC_MINMAX, 2 * sizeof(long long),
                       cudaMemcpyHostToDevice, s->stream));
    CK(launch_minmax_i32((const int32_t*)q, (int64_t)s->n, s->d_acc + ACC_MINMAX, s->stream));
    CK(cudaMemcpyAsync(s->h_acc + ACC_MINMAX, s->d_acc + ACC_MINMAX, 2 * sizeof(long long),
                       cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    *lo = s->h_acc[ACC_MINMAX];
    *hi = s->h_acc[ACC_MINMAX + 1];
    return FQNM_OK;
}

static fqnm_status build_for_state(fqnm_solver* s, const void* q)
{
    int64_t lo = 0, hi = 0;
    fqnm_status st = state_range(s, q, &lo, &hi);
    if (st != FQNM_OK) return st;
    if (s->user_table) {
        const int64_t ulo = s->user_lo, uhi = s->user_lo + (int64_t)s->user_p.size() - 1;
        if (lo < ulo || hi > uhi)
            return set_error(FQNM_ERR_RANGE, "initial states [%lld, %lld] outside the table [%lld, %lld]",
                             (long long)lo, (long long)hi, (long long)ulo, (long long)uhi);
        return build_rule(s, ulo, uhi);
    }
    // the maps are built over [lo - margin, hi + margin] within +-2^30, which
    // leaves a step's transfers room below the int32 limits
    if (lo < INT32_MIN / 2 || hi > INT32_MAX / 2)
        return set_error(FQNM_ERR_OVERFLOW, "states [%lld, %lld] beyond +-2^30 (int32 headroom)",
                         (long long)lo, (long long)hi);
    const int64_t m = s->margin;
    return build_rule(s, std::max<int64_t>(lo - m, INT32_MIN / 2),
                      std::min<int64_t>(hi + m, INT32_MAX / 2));
}

static fqnm_status load_common(fqnm_solver* s, const void* q, size_t n, bool device)
{
    NvtxRange range("fqnm_load");
    if (!s) return set_error(FQNM_ERR_ARG, "null handle");
    if (!q || n == 0) return set_error(FQNM_ERR_ARG, "null states or n == 0");
    if (n > (size_t)INT32_MAX) return set_error(FQNM_ERR_ARG, "n too large");
    if (s->grid.d > 1 && (long long)n != s->grid.cells())
        return set_error(FQNM_ERR_ARG, "%zu states for a grid of %lld cells", n, s->grid.cells());
    fqnm_status st = ensure_runtime(s);
    if (st != FQNM_OK) return st;
    s->loaded = false;
    st = alloc_state(s, n);
    if (st != FQNM_OK) return st;
    const size_t bytes = n * s->state_bytes() * s->nvars;
    CK(cudaMemcpyAsync(s->q[0], q, bytes,
                       device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s->stream));
    s->cur = 0;
    CK(cudaMemsetAsync(s->d_err, 0, sizeof(unsigned), s->stream));
    CK(cudaMemsetAsync(s->d_acc, 0, ACC_SLOTS * sizeof(long long), s->stream));
    s->info.recoveries = 0;
    if (s->nvars == 1) {
        st = build_for_state(s, s->q[0]);
        if (st != FQNM_OK) return st;
        replan(s);
    }
    CK(cudaMemcpyAsync(s->ckpt, s->q[0], bytes, cudaMemcpyDeviceToDevice, s->stream));
    s->ckpt_step = 0;
    s->ckpt_bflux[0] = s->ckpt_bflux[1] = s->ckpt_bflux[2] = 0;
    s->step_count = s->launches = s->cell_updates = 0;
    if (s->nvars == 1 && s->autotune) {
        st = autotune(s);
        if (st != FQNM_OK) return st;
        CK(cudaMemcpyAsync(s->ckpt, s->q[0], bytes, cudaMemcpyDeviceToDevice, s->stream));
    }
    CK(cudaStreamSynchronize(s->stream));
    s->loaded = true;
    if (s->verify) return set_expected_totals(s);
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_load_states(fqnm_solver* s, const void* q, size_t n)
{
    return load_common(s, q, n, false);
}

extern "C" fqnm_status fqnm_load_states_device(fqnm_solver* s, const void* q, size_t n)
{
    return load_common(s, q, n, true);
}

extern "C" fqnm_status fqnm_load_field(fqnm_solver* s, const double* u, size_t n,
                                       int on_device)
{
    if (!s) return set_error(FQNM_ERR_ARG, "null handle");
    if (s->user_table) return set_error(FQNM_ERR_STATE, "a table solver loads integer states");
    if (!u || n == 0 || n > (size_t)INT32_MAX) return set_error(FQNM_ERR_ARG, "bad field");
    fqnm_status st = ensure_runtime(s);
    if (st != FQNM_OK) return st;
    st = alloc_state(s, n);
    if (st != FQNM_OK) return st;
    const size_t cnt = n * s->nvars;
    const double* src = u;
    if (!on_device) {
        double* stage = nullptr;
        st = stage_buffer(s, cnt, &stage);
        if (st != FQNM_OK) return st;
        CK(cudaMemcpyAsync(stage, u, cnt * sizeof(double), cudaMemcpyHostToDevice, s->stream));
        src = stage;
    }
    // quantise into the checkpoint buffer, then load from it
    CK(cudaMemsetAsync(s->d_err, 0, sizeof(unsigned), s->stream));
    for (int v = 0; v < s->nvars; ++v) {
        char* dst = (char*)s->ckpt + v * n * s->state_bytes();
        if (s->nvars == 3 && !((s->qmask >> v) & 1)) {     // kept as double bits
            CK(cudaMemcpyAsync(dst, src + v * n, n * sizeof(double), cudaMemcpyDeviceToDevice,
                               s->stream));
            continue;
        }
        CK(launch_quantise(src + v * n, (int64_t)n, 1.0 / s->delta[v], s->flux.rounding,
                           s->nvars == 3 ? 64 : 32, dst, s->d_err, s->stream));
    }
    CK(cudaMemcpyAsync(s->h_err, s->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (*s->h_err) return set_error(FQNM_ERR_OVERFLOW, "a quantised value does not fit the state type");
    return load_common(s, s->ckpt, n, true);
}

extern "C" uint64_t fqnm_kernel_launches(void) { return g_kernel_launches.load(); }

static fqnm_status enqueue_tb(fqnm_solver* s, int k)
{
    int32_t* in = (int32_t*)s->q[s->cur];
    int32_t* out = (int32_t*)s->q[1 - s->cur];
    CK(launch_step_tb(s->rule, s->plan, in, out, (int64_t)s->n, k, s->d_err, s->stream));
    s->cur = 1 - s->cur;
    s->launches += 1;
    return FQNM_OK;
}

static fqnm_status build_graph(fqnm_solver* s, int nlaunch)
{
    destroy_graph(s);
    cudaGraph_t g = nullptr;
    CK(cudaStreamBeginCapture(s->cap_stream, cudaStreamCaptureModeThreadLocal));
    int c = s->cur;
    cudaError_t le = cudaSuccess;
    for (int i = 0; i < nlaunch && le == cudaSuccess; ++i) {
        le = launch_step_tb(s->rule, s->plan, (int32_t*)s->q[c], (int32_t*)s->q[1 - c],
                            (int64_t)s->n, s->plan.k, s->d_err, s->cap_stream);
        c = 1 - c;
    }
    g_kernel_launches.fetch_sub((unsigned long long)nlaunch);   // captured, not run
    cudaError_t ee = cudaStreamEndCapture(s->cap_stream, &g);
    if (le != cudaSuccess) { if (g) cudaGraphDestroy(g); return cuda_error(le, "graph capture launch"); }
    if (ee != cudaSuccess) return cuda_error(ee, "cudaStreamEndCapture");
    cudaError_t ie = cudaGraphInstantiate(&s->gexec, g, 0);
    cudaGraphDestroy(g);
    if (ie != cudaSuccess) { s->gexec = nullptr; return cuda_error(ie, "cudaGraphInstantiate"); }
    s->g_launches = nlaunch;
    s->g_k = s->plan.k;
    s->g_cur = s->cur;
    s->g_plan = s->plan;
    s->g_rule = s->rule;
    s->g_q0 = s->q[0];
    return FQNM_OK;
}

// A captured graph bakes in buffers, the rule and the plan: reuse it only if
// none of them changed since the capture.
static bool graph_valid(const fqnm_solver* s)
{
    const RuleView &a = s->rule, &b = s->g_rule;
    const Plan &p = s->plan, &g = s->g_plan;
    return s->gexec && s->g_cur == s->cur && s->g_q0 == s->q[0] && s->g_k == p.k &&
           g.layout == p.layout && g.v == p.v && g.block == p.block && g.kernel == p.kernel &&
           g.pdl == p.pdl &&
           a.tab2 == b.tab2 && a.tabp == b.tabp && a.tab16 == b.tab16 && a.lo == b.lo &&
           a.span == b.span &&
           a.evaluator == b.evaluator && a.has_p == b.has_p && a.has_m == b.has_m &&
           a.cf.base == b.cf.base && a.cf.num == b.cf.num && a.cf.den == b.cf.den &&
           a.cf.magic == b.cf.magic && a.cf.shift == b.cf.shift && a.cf.c0 == b.cf.c0 &&
           a.cf.rounding == b.cf.rounding;
}

// The d-D plan.  2-D: K steps per launch (the walk, or register tiles)
// unless the one-step kernel was asked for (FQNM_OPT_KERNEL = 1).  3-D: the
// one-step kernel streaming z slabs, unless a walk was asked for (FQNM_OPT_K
// or FQNM_OPT_ND_TILE = 6): its single pass over the grid per step beats the
// K-step walk, whose shared-memory exchange and barrier per slab bound it.
static NdPlan nd_plan(const fqnm_solver* s)
{
    NdPlan p;
    p.blocked = s->opt_kernel != 1;
    // the autotuner's plan, unless a plan option was set explicitly
    if (p.blocked && s->nd_tuned_tile >= 0 && s->opt_nd_tile == 0 && s->opt_k == 0) {
        if (s->nd_tuned_tile == 0) {                  // the one-step kernel
            p.blocked = 0;
            return p;
        }
        p.walk = s->nd_tuned_tile == ND_WALK;
        if (!p.walk) p.shape = s->nd_tuned_tile;
        p.k = s->nd_tuned_k;
        return p;
    }
    if (s->grid.d == 3 && s->opt_k == 0 && s->opt_nd_tile == 0) p.blocked = 0;
    p.walk = s->grid.d == 3 || s->opt_nd_tile == 0 || s->opt_nd_tile == ND_WALK;
    if (!p.walk) p.shape = s->opt_nd_tile;
    const int lim = s->grid.d == 3 ? 4
                    : p.walk ? 8 : std::min(nd_tile_x(p.shape), nd_tile_y(p.shape)) / 2 - 1;
    const int dflt = s->grid.d == 3 ? 2 : 4;      // 3-D: K = 2 keeps 32-row blocks
    p.k = s->opt_k > 0 ? std::min(s->opt_k, lim) : std::min(dflt, lim);
    return p;
}

// The 2-D walk supports K in {1, 2, 3, 4, 6, 8}, the 3-D walk 1 .. 4: the
// largest of them <= k.
static int walk_k(int d, int k)
{
    while (k > 1 && !(d == 3 ? walk3_k_supported(k) : walk_k_supported(k))) --k;
    return k;
}

static fqnm_status step_scalar(fqnm_solver* s, uint64_t k)
{
    if (s->grid.d > 1) {
        // K steps per launch by the walk (or 2-D register tiles) unless the
        // one-step kernel is asked for
        const NdPlan np = nd_plan(s);
        uint64_t done = 0;
        while (done < k) {
            if (np.blocked && np.walk) {
                const int kk = walk_k(s->grid.d, (int)std::min<uint64_t>((uint64_t)np.k, k - done));
                if (s->grid.d == 3)
                    CK(launch_walk3d(s->rule, (const int32_t*)s->q[s->cur],
                                     (int32_t*)s->q[1 - s->cur], s->grid, kk, s->d_err, s->stream));
                else
                    CK(launch_walk2d(s->rule, (const int32_t*)s->q[s->cur],
                                     (int32_t*)s->q[1 - s->cur], s->grid, kk, s->d_err, s->stream));
                done += kk;
            } else if (np.blocked) {
                const int kk = (int)std::min<uint64_t>((uint64_t)np.k, k - done);
                CK(launch_step2d_tb(s->rule, np, (const int32_t*)s->q[s->cur],
                                    (int32_t*)s->q[1 - s->cur], s->grid, kk, s->d_err, s->stream));
                done += kk;
            } else {
                CK(launch_step_nd(s->rule, (const int32_t*)s->q[s->cur], (int32_t*)s->q[1 - s->cur],
                                  s->grid, s->d_err, s->stream));
                done += 1;
            }
            s->cur = 1 - s->cur;
            s->launches += 1;
        }
        return FQNM_OK;
    }
    if (s->plan.kernel == 4) {
        const uint64_t chunk = 1u << 16;               // steps per launch at most
        for (uint64_t done = 0; done < k;) {
            const uint64_t kk = std::min(chunk, k - done);
            CK(launch_step_resident(s->rule, (const int32_t*)s->q[s->cur],
                                    (int32_t*)s->q[1 - s->cur], (int64_t)s->n, (int64_t)kk,
                                    s->d_err, s->stream));
            s->cur = 1 - s->cur;
            s->launches += 1;
            done += kk;
        }
        return FQNM_OK;
    }
    if (s->plan.kernel == 1) {
        for (uint64_t i = 0; i < k; ++i) {
            CK(launch_step_naive(s->rule, (int32_t*)s->q[s->cur], (int32_t*)s->q[1 - s->cur],
                                 (int64_t)s->n, s->boundary == FQNM_BC_PERIODIC, s->d_err,
                                 s->d_acc + ACC_BFLUX, s->stream));
            s->cur = 1 - s->cur;
            s->launches += 1;
        }
        return FQNM_OK;
    }
    const uint64_t K = (uint64_t)s->plan.k;
    uint64_t full = k / K;
    const int rem = (int)(k % K);
    const int G = 64;                                  // launches per graph (even)
    if (s->use_graph && full >= (uint64_t)G) {
        if (!graph_valid(s)) {
            fqnm_status st = build_graph(s, G);
            if (st != FQNM_OK) return st;
        }
        while (full >= (uint64_t)G) {
            CK(cudaGraphLaunch(s->gexec, s->stream));
            note_launches(G);
            s->launches += G;
            full -= G;
        }
    }
    for (uint64_t i = 0; i < full; ++i) {
        fqnm_status st = enqueue_tb(s, (int)K);
        if (st != FQNM_OK) return st;
    }
    if (rem) return enqueue_tb(s, rem);
    return FQNM_OK;
}

static fqnm_status step_euler(fqnm_solver* s, uint64_t k)
{
    for (uint64_t i = 0; i < k; ++i) {
        CK(launch_euler_step((int64_t*)s->q[s->cur], (int64_t*)s->q[1 - s->cur],
                             (int64_t)s->n, s->flux.gamma, s->delta, s->lambda,
                             s->flux.rounding, s->qmask, s->fp64_mode, s->d_err,
                             s->d_acc + ACC_BFLUX, s->stream));
        s->cur = 1 - s->cur;
        s->launches += 1;
    }
    return FQNM_OK;
}

static fqnm_status step_any(fqnm_solver* s, uint64_t k)
{
    fqnm_status st = s->nvars == 3 ? step_euler(s, k) : step_scalar(s, k);
    if (st != FQNM_OK) return st;
    s->step_count += k;
    s->cell_updates += k * (uint64_t)s->n;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_step(fqnm_solver* s, uint64_t k)
{
    NvtxRange range("fqnm_step");
    if (!s) return set_error(FQNM_ERR_ARG, "null handle");
    if (!s->loaded) return set_error(FQNM_ERR_STATE, "fqnm_step before fqnm_load_states");
    if (k == 0) return FQNM_OK;
    return step_any(s, k);
}

// Wait for the stream; on a range escape rebuild a wider map from the last
// checkpoint and replay the steps since, so that the result is still exact.
// The exact conserved totals of every integer variable (eq. exact_conservation)
// and the boundary transfer accumulated since load; synchronises the stream.
static fqnm_status current_totals(fqnm_solver* s, long long mass[3], long long bflux[3])
{
    CK(cudaMemsetAsync(s->d_acc, 0, 9 * sizeof(long long), s->stream));
    for (int v = 0; v < s->nvars; ++v) {
        if (s->nvars == 3) {
            if (!((s->qmask >> v) & 1)) continue;
            CK(launch_invariants_i64((const int64_t*)s->q[s->cur] + v * s->n, nullptr,
                                     (int64_t)s->n, 0, s->d_acc + 3 * v, s->stream));
        } else if (s->grid.d > 1) {
            CK(launch_invariants_nd((const int32_t*)s->q[s->cur], nullptr, s->grid, s->d_acc,
                                    s->stream));
        } else {
            CK(launch_invariants_i32((const int32_t*)s->q[s->cur], nullptr, (int64_t)s->n, 0,
                                     s->d_acc, s->stream));
        }
    }
    CK(cudaMemcpyAsync(s->h_acc, s->d_acc, (ACC_BFLUX + 3) * sizeof(long long),
                       cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int v = 0; v < 3; ++v) {
        mass[v] = s->h_acc[3 * v];
        bflux[v] = s->h_acc[ACC_BFLUX + v];
    }
    return FQNM_OK;
}

// Expect mass + boundary transfer to stay what it is now.
static fqnm_status set_expected_totals(fqnm_solver* s)
{
    long long mass[3], bflux[3];
    fqnm_status st = current_totals(s, mass, bflux);
    if (st != FQNM_OK) return st;
    for (int v = 0; v < 3; ++v) s->mass0[v] = mass[v] + bflux[v];
    return FQNM_OK;
}

// FQNM_OPT_VERIFY: every step conserves sum q exactly, so sum q + the
// transfer through the ends must equal its value at load; a difference
// means the state changed outside the library (or was corrupted).
static fqnm_status verify_totals(fqnm_solver* s)
{
    long long mass[3], bflux[3];
    fqnm_status st = current_totals(s, mass, bflux);
    if (st != FQNM_OK) return st;
    for (int v = 0; v < s->nvars; ++v) {
        if (s->nvars == 3 && !((s->qmask >> v) & 1)) continue;
        if (mass[v] + bflux[v] != s->mass0[v])
            return set_error(FQNM_ERR_STATE,
                             "conservation check failed at step %llu: variable %d totals %lld, "
                             "expected %lld (the state changed outside the steps)",
                             (unsigned long long)s->step_count, v, mass[v] + bflux[v],
                             s->mass0[v]);
    }
    return FQNM_OK;
}

static fqnm_status sync_and_check(fqnm_solver* s)
{
    for (int attempt = 0;; ++attempt) {
        CK(cudaMemcpyAsync(s->h_err, s->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost,
                           s->stream));
        CK(cudaStreamSynchronize(s->stream));
        const unsigned e = *s->h_err;
        if (e == 0) break;
        if (e & ERRBIT_OVERFLOW)
            return set_error(FQNM_ERR_OVERFLOW, "a transfer does not fit its integer type");
        if (e & ERRBIT_BOUNDS)
            return set_error(FQNM_ERR_STATE, "checked build: a computed index left its buffer");
        if (!(e & ERRBIT_RANGE))
            return set_error(FQNM_ERR_TIMEOUT, "device error word 0x%x", e);
        if (!s->recover || s->nvars != 1 || s->user_table || attempt >= 4)
            return set_error(FQNM_ERR_RANGE,
                             "a state left the verified range [%lld, %lld] of the transfer map",
                             (long long)s->info.lo, (long long)s->info.hi);
        // replay from the checkpoint with a wider map
        const uint64_t replay = s->step_count - s->ckpt_step;
        CK(cudaMemcpyAsync(s->q[0], s->ckpt, s->n * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                           s->stream));
        CK(cudaMemcpyAsync(s->d_acc + ACC_BFLUX, s->d_acc + ACC_BFLUX_CKPT, 3 * sizeof(long long),
                           cudaMemcpyDeviceToDevice, s->stream));
        s->cur = 0;
        destroy_graph(s);
        CK(cudaMemsetAsync(s->d_err, 0, sizeof(unsigned), s->stream));
        s->margin = std::max<int64_t>(4 * s->margin, 4096);
        fqnm_status st = build_for_state(s, s->q[0]);
        if (st != FQNM_OK) return st;
        const Plan keep = s->plan;
        replan(s);
        if (s->autotune) s->plan = keep;
        s->info.recoveries += 1;
        s->step_count = s->ckpt_step;
        st = step_any(s, replay);
        if (st != FQNM_OK) return st;
    }
    if (s->verify) {
        fqnm_status st = verify_totals(s);
        if (st != FQNM_OK) return st;
    }
    // new checkpoint
    if (s->recover && s->nvars == 1 && s->step_count != s->ckpt_step) {
        CK(cudaMemcpyAsync(s->ckpt, s->q[s->cur], s->n * sizeof(int32_t),
                           cudaMemcpyDeviceToDevice, s->stream));
        CK(cudaMemcpyAsync(s->d_acc + ACC_BFLUX_CKPT, s->d_acc + ACC_BFLUX, 3 * sizeof(long long),
                           cudaMemcpyDeviceToDevice, s->stream));
        s->ckpt_step = s->step_count;
    }
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_sync(fqnm_solver* s)
{
    if (!s) return set_error(FQNM_ERR_ARG, "null handle");
    if (!s->loaded) return set_error(FQNM_ERR_STATE, "not loaded");
    return sync_and_check(s);
}

static fqnm_status observe_to(fqnm_solver* s, void* u, int fp32)
{
    for (int v = 0; v < s->nvars; ++v) {
        const size_t es = fp32 ? sizeof(float) : sizeof(double);
        char* dst = (char*)u + v * s->n * es;
        if (s->nvars == 3)
            CK(launch_observe_i64((const int64_t*)s->q[s->cur] + v * s->n, (int64_t)s->n,
                                  s->delta[v], dst, fp32, s->stream, !((s->qmask >> v) & 1)));
        else
            CK(launch_observe_i32((const int32_t*)s->q[s->cur], (int64_t)s->n, s->delta[0],
                                  dst, fp32, s->stream));
    }
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_observe_device(fqnm_solver* s, void* u, int fp32)
{
    if (!s || !u) return set_error(FQNM_ERR_ARG, "null argument");
    if (!s->loaded) return set_error(FQNM_ERR_STATE, "not loaded");
    return observe_to(s, u, fp32);
}

extern "C" fqnm_status fqnm_observe(fqnm_solver* s, double* u)
{
    NvtxRange range("fqnm_observe");
    if (!s || !u) return set_error(FQNM_ERR_ARG, "null argument");
    if (!s->loaded) return set_error(FQNM_ERR_STATE, "not loaded");
    fqnm_status st = sync_and_check(s);
    if (st != FQNM_OK) return st;
    const size_t bytes = s->n * s->nvars * sizeof(double);
    double* d = nullptr;
    st = stage_buffer(s, s->n * s->nvars, &d);
    if (st != FQNM_OK) return st;
    st = observe_to(s, d, 0);
    if (st == FQNM_OK) {
        cudaError_t e = cudaMemcpyAsync(u, d, bytes, cudaMemcpyDeviceToHost, s->stream);
        if (e != cudaSuccess) st = cuda_error(e, "cudaMemcpyAsync observe");
    }
    CK(cudaStreamSynchronize(s->stream));
    return st;
}

extern "C" fqnm_status fqnm_checkpoint(fqnm_solver* s, void* q, uint64_t* step)
{
    if (!s || !q) return set_error(FQNM_ERR_ARG, "null argument");
    if (!s->loaded) return set_error(FQNM_ERR_STATE, "not loaded");
    fqnm_status st = sync_and_check(s);
    if (st != FQNM_OK) return st;
    CK(cudaMemcpyAsync(q, s->q[s->cur], s->n * s->nvars * s->state_bytes(),
                       cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    if (step) *step = s->step_count;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_checkpoint_device(fqnm_solver* s, void* q)
{
    if (!s || !q) return set_error(FQNM_ERR_ARG, "null argument");
    if (!s->loaded) return set_error(FQNM_ERR_STATE, "not loaded");
    CK(cudaMemcpyAsync(q, s->q[s->cur], s->n * s->nvars * s->state_bytes(),
                       cudaMemcpyDeviceToDevice, s->stream));
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_invariants(fqnm_solver* s, const fqnm_solver* other,
                                       fqnm_invariants_t* out)
{
    if (!s || !out) return set_error(FQNM_ERR_ARG, "null argument");
    if (!s->loaded) return set_error(FQNM_ERR_STATE, "not loaded");
    if (other && (!other->loaded || other->n != s->n || other->nvars != s->nvars))
        return set_error(FQNM_ERR_ARG, "other solver has a different shape");
    fqnm_status st = sync_and_check(s);
    if (st != FQNM_OK) return st;
    if (other && other->stream != s->stream) {
        cudaError_t e = cudaStreamSynchronize(other->stream);
        if (e != cudaSuccess) return cuda_error(e, "cudaStreamSynchronize(other)");
    }
    CK(cudaMemsetAsync(s->d_acc, 0, 9 * sizeof(long long), s->stream));
    const int periodic = s->boundary == FQNM_BC_PERIODIC;
    for (int v = 0; v < s->nvars; ++v) {
        if (s->nvars == 3) {
            if (!((s->qmask >> v) & 1)) continue;     // a floating-point component
            const int64_t* q = (const int64_t*)s->q[s->cur] + v * s->n;
            const int64_t* o = other ? (const int64_t*)other->q[other->cur] + v * s->n : nullptr;
            CK(launch_invariants_i64(q, o, (int64_t)s->n, periodic, s->d_acc + 3 * v, s->stream));
        } else if (s->grid.d > 1) {
            const int32_t* o = other ? (const int32_t*)other->q[other->cur] : nullptr;
            CK(launch_invariants_nd((const int32_t*)s->q[s->cur], o, s->grid, s->d_acc,
                                    s->stream));
        } else {
            const int32_t* o = other ? (const int32_t*)other->q[other->cur] : nullptr;
            CK(launch_invariants_i32((const int32_t*)s->q[s->cur], o, (int64_t)s->n, periodic,
                                     s->d_acc, s->stream));
        }
    }
    CK(cudaMemcpyAsync(s->h_acc, s->d_acc, (ACC_BFLUX + 3) * sizeof(long long),
                       cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    std::memset(out, 0, sizeof *out);
    for (int v = 0; v < s->nvars; ++v) {
        out->mass[v] = s->h_acc[3 * v + 0];
        out->tv[v] = s->h_acc[3 * v + 1];
        out->l1[v] = s->h_acc[3 * v + 2];
        out->boundary_flux[v] = s->h_acc[ACC_BFLUX + v];
    }
    out->step = s->step_count;
    out->nvars = s->nvars;
    return FQNM_OK;
}

// ---- level statistics (Supplementary Information, entropy appendix) -------------

static fqnm_status level_check(fqnm_solver* s)
{
    if (!s) return set_error(FQNM_ERR_ARG, "null handle");
    if (s->nvars != 1) return set_error(FQNM_ERR_ARG, "level statistics are defined for scalar states");
    if (!s->loaded) return set_error(FQNM_ERR_STATE, "not loaded");
    if (!s->levels) s->levels = level_work_create();
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_level_step(fqnm_solver* s, fqnm_level_stats_t* out)
{
    NvtxRange range("fqnm_level_step");
    fqnm_status st = level_check(s);
    if (st != FQNM_OK) return st;
    if (!out) return set_error(FQNM_ERR_ARG, "null output");
    static_assert(sizeof(LevelRecord) == sizeof(fqnm_level_stats_t), "record layout");
    st = sync_and_check(s);
    if (st != FQNM_OK) return st;
    const uint64_t n0 = s->step_count;
    s->level_valid = false;
    CK(level_snapshot(s->levels, (const int32_t*)s->q[s->cur], (int64_t)s->n, s->stream));
    st = step_any(s, 1);
    if (st != FQNM_OK) return st;
    st = sync_and_check(s);                    // a range escape is recovered here
    if (st != FQNM_OK) return st;
    const int32_t* qn = level_snap(s->levels);
    const int32_t* qn1 = (const int32_t*)s->q[s->cur];
    int64_t lo0 = 0, hi0 = 0, lo1 = 0, hi1 = 0;
    st = state_range(s, qn, &lo0, &hi0);
    if (st != FQNM_OK) return st;
    st = state_range(s, qn1, &lo1, &hi1);
    if (st != FQNM_OK) return st;
    const int64_t lo = std::min(lo0, lo1), W = std::max(hi0, hi1) - lo + 1;
    CK(level_transition(s->levels, qn, qn1, (int64_t)s->n, lo, W, s->stream));
    unsigned e = 0;
    CK(level_record(s->levels, &s->level_last, &e, s->stream));
    if (e & ERRBIT_BOUNDS)
        return set_error(FQNM_ERR_STATE, "checked build: a computed index left its buffer");
    if (e) return set_error(FQNM_ERR_RANGE, "a level left [%lld, %lld]", (long long)lo,
                            (long long)(lo + W - 1));
    s->level_last.step = n0;
    s->level_valid = true;
    std::memcpy(out, &s->level_last, sizeof *out);
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_level_series(fqnm_solver* s, uint64_t records, uint64_t every,
                                         fqnm_level_stats_t* out)
{
    fqnm_status st = level_check(s);
    if (st != FQNM_OK) return st;
    if (every == 0) return set_error(FQNM_ERR_ARG, "every must be >= 1");
    if (records && !out) return set_error(FQNM_ERR_ARG, "null output");
    for (uint64_t r = 0; r < records; ++r) {
        if (every > 1) {
            st = step_any(s, every - 1);
            if (st != FQNM_OK) return st;
        }
        st = fqnm_level_step(s, out + r);
        if (st != FQNM_OK) return st;
    }
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_level_transitions(fqnm_solver* s, int64_t* k, int64_t* k_next,
                                              int64_t* count, size_t cap, size_t* pairs)
{
    fqnm_status st = level_check(s);
    if (st != FQNM_OK) return st;
    if (!s->level_valid) return set_error(FQNM_ERR_STATE, "no recorded transition (call fqnm_level_step)");
    const size_t m = (size_t)s->level_last.pairs;
    if (pairs) *pairs = m;
    if (cap < m) return set_error(FQNM_ERR_ARG, "capacity %zu below the %zu pairs", cap, m);
    if (m && (!k || !k_next || !count)) return set_error(FQNM_ERR_ARG, "null output");
    CK(level_export_pairs(s->levels, (int64_t)m, k, k_next, count, s->stream));
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_level_histogram(fqnm_solver* s, int64_t* lo, int64_t* counts,
                                            size_t cap, size_t* len)
{
    fqnm_status st = level_check(s);
    if (st != FQNM_OK) return st;
    st = sync_and_check(s);
    if (st != FQNM_OK) return st;
    int64_t l = 0, h = 0;
    st = state_range(s, s->q[s->cur], &l, &h);
    if (st != FQNM_OK) return st;
    const size_t W = (size_t)(h - l + 1);
    if (lo) *lo = l;
    if (len) *len = W;
    if (cap < W) return set_error(FQNM_ERR_ARG, "capacity %zu below the %zu levels", cap, W);
    if (!counts) return set_error(FQNM_ERR_ARG, "null output");
    unsigned e = 0;
    CK(level_histogram(s->levels, (const int32_t*)s->q[s->cur], (int64_t)s->n, l, (int64_t)W,
                       counts, &e, s->stream));
    if (e) return set_error(FQNM_ERR_RANGE, "a level left [%lld, %lld]", (long long)l, (long long)h);
    return FQNM_OK;
}

// ---- Hopf-Lax entropy reference of Burgers (§3.2) ----------------------------------

extern "C" fqnm_status fqnm_hopf_lax(const double* x, size_t nx, const double* y,
                                     const double* U0y, size_t ny, double t, double* u,
                                     int64_t* idx, int on_device, void* stream)
{
    NvtxRange range("fqnm_hopf_lax");
    if (!x || !y || !U0y || !u) return set_error(FQNM_ERR_ARG, "null array");
    if (nx == 0 || ny == 0) return set_error(FQNM_ERR_ARG, "empty points or candidates");
    if (nx > (size_t)INT32_MAX * 4 || ny > (size_t)INT64_MAX / 8)
        return set_error(FQNM_ERR_ARG, "too many points");
    if (!(t > 0.0) || !(t < 1e300)) return set_error(FQNM_ERR_ARG, "t must be positive and finite");
    cudaStream_t st = (cudaStream_t)stream;
    if (on_device) {
        CK(launch_hopf_lax(x, (int64_t)nx, y, U0y, (int64_t)ny, t, u, idx, st));
        return FQNM_OK;
    }
    double* d = nullptr;
    const size_t doubles = 2 * nx + 2 * ny;
    CK(cudaMallocAsync((void**)&d, doubles * sizeof(double) + nx * sizeof(int64_t), st));
    double* dx_ = d;
    double* dy = d + nx;
    double* dU = dy + ny;
    double* du = dU + ny;
    int64_t* di = (int64_t*)(du + nx);
    cudaError_t e = cudaMemcpyAsync(dx_, x, nx * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dy, y, ny * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dU, U0y, ny * sizeof(double), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = launch_hopf_lax(dx_, (int64_t)nx, dy, dU, (int64_t)ny, t, du, di, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(u, du, nx * sizeof(double), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && idx)
        e = cudaMemcpyAsync(idx, di, nx * sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    cudaFreeAsync(d, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return cuda_error(e, "fqnm_hopf_lax");
    return FQNM_OK;
}

// ---- Cartesian grids (Theorem, extension by directional composition) -------------

extern "C" fqnm_status fqnm_set_grid(fqnm_solver* s, int d, const size_t* dims)
{
    if (!s) return set_error(FQNM_ERR_ARG, "null handle");
    if (s->loaded) return set_error(FQNM_ERR_STATE, "set the grid before loading");
    if (d < 1 || d > 3 || (d > 1 && !dims)) return set_error(FQNM_ERR_ARG, "d must be 1, 2 or 3");
    if (s->nvars != 1) return set_error(FQNM_ERR_ARG, "grids are for scalar solvers");
    if (d > 1 && s->boundary != FQNM_BC_PERIODIC)
        return set_error(FQNM_ERR_ARG, "d > 1 grids are periodic");
    if (d > 1 && s->flux.kind == FQNM_FLUX_BURGERS_GODUNOV)
        return set_error(FQNM_ERR_ARG, "grids step split fluxes (the Godunov face is 1-D only)");
    NdGrid g{d, {1, 1, 1}};
    long long cells = 1;
    for (int m = 0; m < d && d > 1; ++m) {
        if (dims[m] == 0 || dims[m] > (size_t)INT32_MAX)
            return set_error(FQNM_ERR_ARG, "dims[%d] = %zu", m, dims[m]);
        g.dims[m] = (long long)dims[m];
        cells *= g.dims[m];
        if (cells > (long long)INT32_MAX) return set_error(FQNM_ERR_ARG, "too many cells");
    }
    // monotone (Lemma on CFL stability per axis summed): d nu <= 1
    if (d > 1 && !s->user_table) {
        double nu = 0;
        const double lam = s->lambda;
        if (s->flux.kind == FQNM_FLUX_LINEAR_UPWIND) nu = std::fabs(s->flux.a) * lam;
        else nu = s->flux.alpha * lam;
        if (d * nu > 1.0)
            return set_error(FQNM_ERR_CFL, "d * Courant number = %.17g > 1", d * nu);
    }
    if (d == 1) g = NdGrid{1, {0, 1, 1}};
    s->grid = g;
    ++s->rule_gen;
    destroy_graph(s);
    return FQNM_OK;
}

// ---- resume and the live state --------------------------------------------------

extern "C" fqnm_status fqnm_resume(fqnm_solver* s, const void* q, size_t n, uint64_t step,
                                   const int64_t* boundary_flux)
{
    fqnm_status st = load_common(s, q, n, false);
    if (st != FQNM_OK) return st;
    long long b[3] = {0, 0, 0};
    for (int v = 0; v < s->nvars && boundary_flux; ++v) b[v] = boundary_flux[v];
    CK(cudaMemcpyAsync(s->d_acc + ACC_BFLUX, b, 3 * sizeof(long long), cudaMemcpyHostToDevice,
                       s->stream));
    CK(cudaMemcpyAsync(s->d_acc + ACC_BFLUX_CKPT, b, 3 * sizeof(long long),
                       cudaMemcpyHostToDevice, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int v = 0; v < 3; ++v) s->ckpt_bflux[v] = b[v];
    s->step_count = step;
    s->ckpt_step = step;
    if (s->verify) return set_expected_totals(s);
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_state_device(fqnm_solver* s, void** q, size_t* n_cells)
{
    if (!s || !q) return set_error(FQNM_ERR_ARG, "null argument");
    if (!s->loaded) return set_error(FQNM_ERR_STATE, "not loaded");
    fqnm_status st = sync_and_check(s);
    if (st != FQNM_OK) return st;
    *q = s->q[s->cur];
    if (n_cells) *n_cells = s->n;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_get_size(fqnm_solver* s, size_t* n_cells, int* nvars)
{
    if (!s) return set_error(FQNM_ERR_ARG, "null handle");
    if (n_cells) *n_cells = s->loaded ? s->n : 0;
    if (nvars) *nvars = s->nvars;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_get_rule(fqnm_solver* s, fqnm_rule_info* out)
{
    if (!s || !out) return set_error(FQNM_ERR_ARG, "null argument");
    if (!s->loaded || s->nvars != 1) return set_error(FQNM_ERR_STATE, "no scalar rule loaded");
    *out = s->info;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_get_tables(fqnm_solver* s, int32_t* phi_p, int32_t* phi_m)
{
    if (!s || !phi_p || !phi_m) return set_error(FQNM_ERR_ARG, "null argument");
    if (!s->loaded || s->nvars != 1) return set_error(FQNM_ERR_STATE, "no scalar rule loaded");
    const int64_t count = s->info.hi - s->info.lo + 1;
    std::vector<int2> h((size_t)count);
    CK(cudaMemcpyAsync(h.data(), s->tab2, count * sizeof(int2), cudaMemcpyDeviceToHost, s->stream));
    CK(cudaStreamSynchronize(s->stream));
    for (int64_t k = 0; k < count; ++k) {
        phi_p[k] = h[k].x;
        phi_m[k] = h[k].y;
    }
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_get_stats(fqnm_solver* s, fqnm_stats* out, int reset)
{
    if (!s || !out) return set_error(FQNM_ERR_ARG, "null argument");
    std::memset(out, 0, sizeof *out);
    out->launches = s->launches;
    out->steps = s->step_count;
    out->cell_updates = s->cell_updates;
    out->kernel = s->nvars == 3 ? 3 : s->plan.kernel;
    out->layout = s->plan.layout;
    out->cells_per_thread = s->plan.v;
    out->block = s->plan.block;
    out->k = s->plan.k;
    if (s->nvars == 1 && s->grid.d > 1) {                // the d-D plan
        const NdPlan np = nd_plan(s);
        out->kernel = !np.blocked ? 1 : (np.walk ? 5 : 6);
        out->layout = np.walk ? ND_WALK : np.shape;
        out->cells_per_thread = 0;
        out->block = 0;
        out->k = np.blocked ? np.k : 1;
    }
    if (s->nvars == 1 && s->plan.kernel == 4) {          // one block holds the line
        out->layout = LAYOUT_BLOCKED;
        out->cells_per_thread = resident_v((int64_t)s->n);
        out->block = out->cells_per_thread ? (int32_t)(s->n / out->cells_per_thread) : 0;
        out->k = 0;
    }
    out->graph = s->use_graph;
    if (reset) {
        s->launches = 0;
        s->cell_updates = 0;
    }
    return FQNM_OK;
}

// ============================================================================
// quantisation helper (eq. quantisation on the GPU)
// ============================================================================

extern "C" fqnm_status fqnm_quantise_device(const double* u, size_t n, double delta,
                                           int rounding, int state_bits, void* q,
                                           void* stream)
{
    if (!u || !q || n == 0) return set_error(FQNM_ERR_ARG, "null argument or n == 0");
    if (!is_pow2(delta)) return set_error(FQNM_ERR_ARG, "delta is not a power of two");
    if (state_bits != 32 && state_bits != 64) return set_error(FQNM_ERR_ARG, "state_bits must be 32 or 64");
    if (rounding < 0 || rounding > 2) return set_error(FQNM_ERR_ARG, "unknown rounding");
    cudaStream_t st = (cudaStream_t)stream;
    unsigned* d_err = nullptr;
    CK(cudaMallocAsync((void**)&d_err, sizeof(unsigned), st));
    CK(cudaMemsetAsync(d_err, 0, sizeof(unsigned), st));
    CK(launch_quantise(u, (int64_t)n, 1.0 / delta, rounding, state_bits, q, d_err, st));
    unsigned h = 0;
    CK(cudaMemcpyAsync(&h, d_err, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(d_err, st));
    CK(cudaStreamSynchronize(st));
    if (h) return set_error(FQNM_ERR_OVERFLOW, "a quantised value does not fit %d bits", state_bits);
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_quantise(const double* u, size_t n, double delta, int rounding,
                                    int state_bits, void* q)
{
    if (!u || !q || n == 0) return set_error(FQNM_ERR_ARG, "null argument or n == 0");
    if (state_bits != 32 && state_bits != 64) return set_error(FQNM_ERR_ARG, "state_bits must be 32 or 64");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return set_error(FQNM_ERR_CUDA, "no CUDA device available");
    double* du = nullptr;
    void* dq = nullptr;
    const size_t qb = n * (state_bits / 8);
    CK(cudaMalloc((void**)&du, n * sizeof(double)));
    cudaError_t e = cudaMalloc(&dq, qb);
    if (e != cudaSuccess) { cudaFree(du); return cuda_error(e, "cudaMalloc"); }
    fqnm_status st = FQNM_OK;
    e = cudaMemcpy(du, u, n * sizeof(double), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_error(e, "cudaMemcpy");
    if (st == FQNM_OK) st = fqnm_quantise_device(du, n, delta, rounding, state_bits, dq, nullptr);
    if (st == FQNM_OK) {
        e = cudaMemcpy(q, dq, qb, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) st = cuda_error(e, "cudaMemcpy");
    }
    cudaFree(du);
    cudaFree(dq);
    return st;
}

// ============================================================================
// floating-point finite-volume baseline
// ============================================================================

struct fqnm_fv {
    fqnm_flux flux{};
    int nvars = 1, precision = 64, boundary = FQNM_BC_PERIODIC;
    double dx = 0, dt = 0, lambda = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    void* u[2] = {nullptr, nullptr};
    int cur = 0;
    size_t n = 0, cap_n = 0;
    bool loaded = false;
    uint64_t launches = 0;
    int k = 1;                              // time steps per launch
};

extern "C" fqnm_status fqnm_fv_create(const fqnm_flux* flux, double dx, double dt,
                                      int boundary, int precision, fqnm_fv** out)
{
    if (!out) return set_error(FQNM_ERR_ARG, "null out");
    *out = nullptr;
    if (precision != 32 && precision != 64) return set_error(FQNM_ERR_ARG, "precision must be 32 or 64");
    const double ones[3] = {1.0, 1.0, 1.0};
    int nvars = 1;
    fqnm_status st = check_flux(flux, ones, dx, dt, boundary, &nvars);
    if (st != FQNM_OK) return st;
    if (flux->kind == FQNM_FLUX_BURGERS_GODUNOV)
        return set_error(FQNM_ERR_ARG, "the FV baseline takes split fluxes (use BURGERS_EO)");
    fqnm_fv* f = new (std::nothrow) fqnm_fv();
    if (!f) return set_error(FQNM_ERR_OOM, "host allocation failed");
    f->flux = *flux;
    f->nvars = nvars;
    f->precision = precision;
    f->boundary = boundary;
    f->dx = dx;
    f->dt = dt;
    f->lambda = dt / dx;
    *out = f;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_fv_destroy(fqnm_fv* f)
{
    if (!f) return FQNM_OK;
    if (f->stream) cudaStreamSynchronize(f->stream);
    for (int b = 0; b < 2; ++b) if (f->u[b]) cudaFree(f->u[b]);
    if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
    delete f;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_fv_set_stream(fqnm_fv* f, void* stream)
{
    if (!f) return set_error(FQNM_ERR_ARG, "null handle");
    if (f->stream) cudaStreamSynchronize(f->stream);
    if (f->own_stream && f->stream) cudaStreamDestroy(f->stream);
    f->own_stream = false;
    f->stream = (cudaStream_t)stream;
    return FQNM_OK;
}

static fqnm_status fv_load(fqnm_fv* f, const double* u, size_t n, bool device)
{
    if (!f || !u || n == 0) return set_error(FQNM_ERR_ARG, "null argument or n == 0");
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0)
        return set_error(FQNM_ERR_CUDA, "no CUDA device available");
    if (!f->stream) {
        CK(cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking));
        f->own_stream = true;
    }
    const size_t cnt = n * f->nvars;
    const size_t es = f->precision == 64 ? sizeof(double) : sizeof(float);
    if (n > f->cap_n) {
        for (int b = 0; b < 2; ++b) { if (f->u[b]) cudaFree(f->u[b]); f->u[b] = nullptr; }
        for (int b = 0; b < 2; ++b) CK(cudaMalloc(&f->u[b], cnt * es));
        f->cap_n = n;
    }
    f->n = n;
    f->cur = 0;
    const double* src = u;
    DeviceScratch<double> tmp;
    if (!device) {
        CK(tmp.alloc(cnt));
        CK(cudaMemcpyAsync(tmp.p, u, cnt * sizeof(double), cudaMemcpyHostToDevice, f->stream));
        src = tmp.p;
    }
    if (f->precision == 64)
        CK(cudaMemcpyAsync(f->u[0], src, cnt * sizeof(double), cudaMemcpyDeviceToDevice, f->stream));
    else
        CK(launch_convert_f64_to_f32(src, (float*)f->u[0], (int64_t)cnt, f->stream));
    CK(cudaStreamSynchronize(f->stream));
    f->loaded = true;
    f->launches = 0;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_fv_load(fqnm_fv* f, const double* u, size_t n)
{
    return fv_load(f, u, n, false);
}

extern "C" fqnm_status fqnm_fv_load_device(fqnm_fv* f, const double* u, size_t n)
{
    return fv_load(f, u, n, true);
}

extern "C" fqnm_status fqnm_fv_set_k(fqnm_fv* f, int k)
{
    if (!f) return set_error(FQNM_ERR_ARG, "null handle");
    if (k < 1 || k > FV_TB_MAX_K) return set_error(FQNM_ERR_ARG, "K = %d outside 1..%d", k, FV_TB_MAX_K);
    if (k > 1 && (f->nvars != 1 || f->boundary != FQNM_BC_PERIODIC))
        return set_error(FQNM_ERR_ARG, "K > 1 needs a periodic scalar baseline");
    f->k = k;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_fv_step(fqnm_fv* f, uint64_t k)
{
    if (!f) return set_error(FQNM_ERR_ARG, "null handle");
    if (!f->loaded) return set_error(FQNM_ERR_STATE, "fqnm_fv_step before load");
    const int periodic = f->boundary == FQNM_BC_PERIODIC;
    if (f->k > 1) {
        for (uint64_t done = 0; done < k;) {
            const int kk = (int)std::min<uint64_t>((uint64_t)f->k, k - done);
            void* in = f->u[f->cur];
            void* out = f->u[1 - f->cur];
            if (f->precision == 64)
                CK(launch_fv_tb_f64(f->flux.kind, f->flux.a, f->flux.alpha, f->lambda,
                                    (const double*)in, (double*)out, (int64_t)f->n, kk, f->stream));
            else
                CK(launch_fv_tb_f32(f->flux.kind, f->flux.a, f->flux.alpha, f->lambda,
                                    (const float*)in, (float*)out, (int64_t)f->n, kk, f->stream));
            f->cur = 1 - f->cur;
            f->launches += 1;
            done += (uint64_t)kk;
        }
        return FQNM_OK;
    }
    for (uint64_t i = 0; i < k; ++i) {
        void* in = f->u[f->cur];
        void* out = f->u[1 - f->cur];
        if (f->nvars == 3) {
            if (f->precision == 64)
                CK(launch_euler_fv_f64(f->flux.gamma, f->lambda, (const double*)in, (double*)out,
                                       (int64_t)f->n, f->stream));
            else
                CK(launch_euler_fv_f32(f->flux.gamma, f->lambda, (const float*)in, (float*)out,
                                       (int64_t)f->n, f->stream));
        } else if (f->precision == 64) {
            CK(launch_fv_step_f64(f->flux.kind, f->flux.a, f->flux.alpha, f->lambda,
                                  (const double*)in, (double*)out, (int64_t)f->n, periodic,
                                  f->stream));
        } else {
            CK(launch_fv_step_f32(f->flux.kind, f->flux.a, f->flux.alpha, f->lambda,
                                  (const float*)in, (float*)out, (int64_t)f->n, periodic,
                                  f->stream));
        }
        f->cur = 1 - f->cur;
        f->launches += 1;
    }
    return FQNM_OK;
}

static fqnm_status fv_observe(fqnm_fv* f, double* u, bool device)
{
    if (!f || !u) return set_error(FQNM_ERR_ARG, "null argument");
    if (!f->loaded) return set_error(FQNM_ERR_STATE, "not loaded");
    const size_t cnt = f->n * f->nvars;
    double* dst = u;
    double* tmp = nullptr;
    if (!device) {
        CK(cudaMallocAsync((void**)&tmp, cnt * sizeof(double), f->stream));
        dst = tmp;
    }
    if (f->precision == 64)
        CK(cudaMemcpyAsync(dst, f->u[f->cur], cnt * sizeof(double), cudaMemcpyDeviceToDevice,
                           f->stream));
    else
        CK(launch_convert_f32_to_f64((const float*)f->u[f->cur], dst, (int64_t)cnt, f->stream));
    if (!device) {
        CK(cudaMemcpyAsync(u, tmp, cnt * sizeof(double), cudaMemcpyDeviceToHost, f->stream));
        CK(cudaFreeAsync(tmp, f->stream));
        CK(cudaStreamSynchronize(f->stream));
    }
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_fv_observe(fqnm_fv* f, double* u) { return fv_observe(f, u, false); }
extern "C" fqnm_status fqnm_fv_observe_device(fqnm_fv* f, double* u) { return fv_observe(f, u, true); }

extern "C" fqnm_status fqnm_fv_get_size(fqnm_fv* f, size_t* n_cells, int* nvars)
{
    if (!f) return set_error(FQNM_ERR_ARG, "null handle");
    if (n_cells) *n_cells = f->loaded ? f->n : 0;
    if (nvars) *nvars = f->nvars;
    return FQNM_OK;
}

extern "C" fqnm_status fqnm_fv_launches(fqnm_fv* f, uint64_t* launches)
{
    if (!f || !launches) return set_error(FQNM_ERR_ARG, "null argument");
    *launches = f->launches;
    return FQNM_OK;
}

// ============================================================================
// diagnostics
// ============================================================================

extern "C" const char* fqnm_last_error(void) { return g_err; }

extern "C" const char* fqnm_status_string(int st)
{
    switch (st) {
    case FQNM_OK: return "ok";
    case FQNM_ERR_ARG: return "invalid argument";
    case FQNM_ERR_CFL: return "Courant number above 1";
    case FQNM_ERR_RANGE: return "state left the verified range of the transfer map";
    case FQNM_ERR_OVERFLOW: return "integer overflow";
    case FQNM_ERR_OOM: return "out of memory";
    case FQNM_ERR_CUDA: return "CUDA error";
    case FQNM_ERR_TIMEOUT: return "timeout";
    case FQNM_ERR_STATE: return "call out of order";
    case FQNM_ERR_BUSY: return "busy";
    default: return "unknown status";
    }
}

extern "C" int fqnm_version(void) { return 100; }
