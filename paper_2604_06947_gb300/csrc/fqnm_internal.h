// fqnm_internal.h -- declarations shared by the libfqnm translation units.
// Nothing here is part of the C ABI (that is include/fqnm.h).
#pragma once

#include <cuda_runtime.h>
#include <atomic>
#include <cstddef>
#include <cstdint>
#include <utility>
#include <vector>

#include "../../include/fqnm.h"

// Checked builds (-DFQNM_CHECKED, the stand-in for a sanitizer): the index
// computations that are not bounded by construction are verified before the
// access; a bad one sets ERRBIT_BOUNDS and the access is skipped.  In the
// normal build the check is `true` and compiles away.
#ifdef FQNM_CHECKED
#define FQNM_IN_RANGE(i, n, err)                                                  \
    ((unsigned long long)(i) < (unsigned long long)(n)                             \
         ? true                                                                    \
         : (atomicOr((err), ERRBIT_BOUNDS), false))
#else
#define FQNM_IN_RANGE(i, n, err) true
#endif

namespace fqnm {

// Bits of the per-handle device error word.
enum : unsigned {
    ERRBIT_RANGE = 1u,      // a state left [lo, hi] of the verified transfer map
    ERRBIT_OVERFLOW = 2u,   // a value does not fit its integer type
    ERRBIT_TIMEOUT = 4u,    // a bounded device wait ran out
    ERRBIT_BOUNDS = 8u,     // (checked builds) a computed index left its buffer
};

enum Layout : int { LAYOUT_INTERLEAVED = 1, LAYOUT_BLOCKED = 2, LAYOUT_RUNS4 = 3, LAYOUT_RUNS8 = 4 };
enum Evaluator : int { EVAL_TABLE = 1, EVAL_CLOSED_FORM = 2 };

// Integer closed form phi(q) = R(q * num / den) for den > 0, num > 0,
// evaluated with 32-bit words: x = q - base (base a multiple of 2*den, so
// the shift keeps the parity that half-even rounding looks at),
// t = x*num < 2^31, d = floor(t/den) by a multiply-shift with magic
// (Granlund & Montgomery, "Division by invariant integers using
// multiplication", PLDI 1994), r = t - d*den, then the rounding decision.
struct ClosedForm {
    int32_t base;
    uint32_t num, den;
    uint32_t magic;
    int32_t shift;
    int32_t c0;         // base*num/den, an even multiple of num
    int32_t rounding;   // fqnm_rounding
};

// Transfer rule as the kernels see it.
struct RuleView {
    const int2* tab2;     // (phi+, phi-) for q = lo .. lo+span
    const int32_t* tabp;  // phi+ only (same range)
    const int32_t* tab16; // phi+ in the low, phi- in the high 16 bits, when both fit int16
    int32_t lo;
    uint32_t span;        // entries - 1
    int32_t evaluator;    // Evaluator
    int32_t has_p, has_m;
    int32_t face_max;     // face transfer max(phi+(qL), phi-(qR)) instead of the sum
    ClosedForm cf;        // valid when evaluator == EVAL_CLOSED_FORM (phi+ only)
};

// Execution plan of the scalar stepping kernels.
struct Plan {
    int kernel = 2;        // 1 naive, 2 temporal-blocked, 4 resident (one block)
    int layout = LAYOUT_INTERLEAVED;
    int v = 8;             // cells per thread
    int block = 256;
    int k = 32;            // steps per launch
    int pdl = 0;           // launch with programmatic dependent launch
};

// ---- k_rule.cu --------------------------------------------------------------
cudaError_t launch_build_split_table(int kind, double a, double alpha,
                                     double delta, double lambda, int rounding,
                                     int64_t lo, int64_t count, int2* tab2,
                                     int32_t* tabp, unsigned* err,
                                     cudaStream_t st);
// tab16[k] = (phi+ & 0xffff) | (phi- << 16); caller checks both fit int16
cudaError_t launch_pack_tab16(const int2* tab2, int64_t count, int32_t* tab16,
                              cudaStream_t st);
cudaError_t launch_copy_user_table(const int32_t* p, const int32_t* m,
                                   int64_t count, int2* tab2, int32_t* tabp,
                                   cudaStream_t st);
// out[0] closed-form mismatches (if cf != nullptr), out[1] certificate flags,
// out[2] max|phi+|, out[3] max|phi-|; out must be zeroed device memory.
enum : unsigned long long {
    CERT_P_NOT_MONOTONE = 1, CERT_M_NOT_MONOTONE = 2, CERT_H_NOT_MONOTONE = 4,
    CERT_P_NONZERO = 8, CERT_M_NONZERO = 16,
};
cudaError_t launch_rule_check(const int2* tab2, int64_t lo, int64_t count,
                              const ClosedForm* cf, unsigned long long* out,
                              cudaStream_t st);
// out[0] = min, out[1] = max over q (must be initialised to +inf/-inf).
cudaError_t launch_minmax_i32(const int32_t* q, int64_t n, long long* out,
                              cudaStream_t st);
cudaError_t launch_minmax_i64(const int64_t* q, int64_t n, long long* out,
                              cudaStream_t st);
cudaError_t launch_quantise(const double* u, int64_t n, double inv_delta,
                            int rounding, int bits, void* q, unsigned* err,
                            cudaStream_t st);
void init_minmax(long long* host2);

// ---- k_scalar.cu ------------------------------------------------------------
cudaError_t launch_step_naive(const RuleView& r, const int32_t* qin,
                              int32_t* qout, int64_t n, int periodic,
                              unsigned* err, long long* bflux, cudaStream_t st);
// One launch of `k` steps of the temporal-blocked kernel (periodic only).
cudaError_t launch_step_tb(const RuleView& r, const Plan& p, const int32_t* qin,
                           int32_t* qout, int64_t n, int k, unsigned* err,
                           cudaStream_t st);
bool tb_plan_supported(const RuleView& r, const Plan& p);
// A periodic line held whole by one block: cells per thread V (1, 2, 4, 8)
// with V | n and n / V <= RESIDENT_MAX_THREADS, or 0 if none fits.
constexpr int RESIDENT_MAX_THREADS = 1024;
constexpr int RESIDENT_AUTO_CELLS = 512;   // the default plan's limit (measured crossover)
int resident_v(int64_t n);
// `steps` steps of the whole line in one launch.
cudaError_t launch_step_resident(const RuleView& r, const int32_t* qin, int32_t* qout,
                                 int64_t n, int64_t steps, unsigned* err, cudaStream_t st);

// ---- k_reduce.cu ------------------------------------------------------------
// acc[0..2] += (mass, tv, l1) of one variable (int32 or int64 states).
cudaError_t launch_invariants_i32(const int32_t* q, const int32_t* other,
                                  int64_t n, int periodic, long long* acc,
                                  cudaStream_t st);
cudaError_t launch_invariants_i64(const int64_t* q, const int64_t* other,
                                  int64_t n, int periodic, long long* acc,
                                  cudaStream_t st);
cudaError_t launch_observe_i32(const int32_t* q, int64_t n, double delta,
                               void* u, int fp32, cudaStream_t st);
// bits != 0: q holds the bits of doubles (an unquantised Euler component)
cudaError_t launch_observe_i64(const int64_t* q, int64_t n, double delta,
                               void* u, int fp32, cudaStream_t st, int bits = 0);

// ---- k_euler.cu -------------------------------------------------------------
// mask: components evolved as integers (1 rho, 2 m, 4 E); the others hold
// the bits of a double and take the floating-point update with the same flux
cudaError_t launch_euler_step(const int64_t* qin, int64_t* qout, int64_t n,
                              double gamma, const double* delta,
                              double lambda, int rounding, int mask, int fp64_mode,
                              unsigned* err, long long* bflux, cudaStream_t st);

// ---- k_fv.cu ----------------------------------------------------------------
cudaError_t launch_fv_step_f64(int kind, double a, double alpha, double lambda,
                               const double* uin, double* uout, int64_t n,
                               int periodic, cudaStream_t st);
cudaError_t launch_fv_step_f32(int kind, double a, double alpha, double lambda,
                               const float* uin, float* uout, int64_t n,
                               int periodic, cudaStream_t st);
// K steps per launch (periodic scalar problems; 1 <= K <= FV_TB_MAX_K)
constexpr int FV_TB_MAX_K = 64;
cudaError_t launch_fv_tb_f64(int kind, double a, double alpha, double lambda, const double* uin,
                             double* uout, int64_t n, int K, cudaStream_t st);
cudaError_t launch_fv_tb_f32(int kind, double a, double alpha, double lambda, const float* uin,
                             float* uout, int64_t n, int K, cudaStream_t st);
cudaError_t launch_euler_fv_f64(double gamma, double lambda, const double* uin,
                                double* uout, int64_t n, cudaStream_t st);
cudaError_t launch_euler_fv_f32(double gamma, double lambda, const float* uin,
                                float* uout, int64_t n, cudaStream_t st);
cudaError_t launch_convert_f64_to_f32(const double* in, float* out, int64_t n,
                                      cudaStream_t st);
cudaError_t launch_convert_f32_to_f64(const float* in, double* out, int64_t n,
                                      cudaStream_t st);

// ---- capi.cu ----------------------------------------------------------------
// kernels launched by this library in this process
extern std::atomic<unsigned long long> g_kernel_launches;
inline void note_launches(unsigned long long k = 1) { g_kernel_launches.fetch_add(k); }
fqnm_status set_error(fqnm_status st, const char* fmt, ...);
// closed-form candidates of a linear map (rule builder)
bool make_closed_form(int64_t lo, int64_t hi, uint32_t num, uint32_t den, int rounding,
                      ClosedForm* out);
std::vector<std::pair<uint32_t, uint32_t>> convergents(double c, uint32_t maxden);
fqnm_status cuda_error(cudaError_t e, const char* where);

inline unsigned grid_for(int64_t n, int block, int max_blocks = 152 * 16)
{
    int64_t g = (n + block - 1) / block;
    if (g < 1) g = 1;
    if (g > max_blocks) g = max_blocks;
    return (unsigned)g;
}

}  // namespace fqnm
