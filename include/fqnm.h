/*
 * fqnm.h -- C ABI of libfqnm, the GB300 (sm_103a) implementation of the
 * quantised conservative step of the Fast Quantised Numerical Method
 * (Park, Ha & Kang, arXiv 2604.06947).
 *
 * The method (§2, eqs. quantisation, flux_table, update_rule):
 *   q_i = round(u_i / delta)                       integer state
 *   phi+-(q) = round(f+-(delta q) dt/dx / delta)   integer transfer maps
 *   F_{i+1/2} = phi+(q_i) + phi-(q_{i+1})          face count flux
 *   q_i <- q_i - (F_{i+1/2} - F_{i-1/2})           telescoping update
 *   u_i = delta q_i                                observable, on request
 *
 * Conventions for every call:
 *   - Every call returns an fqnm_status; no call aborts, traps or exits.
 *     On failure fqnm_last_error() holds a message (thread-local).
 *   - A handle is not thread-safe: use one handle per host thread.
 *   - "host" pointers are ordinary CPU memory owned by the caller; the call
 *     copies what it needs before returning.  "device" pointers are CUDA
 *     global memory owned by the caller (for example a torch tensor); the
 *     call only reads or writes them, in stream order on the handle's stream.
 *   - Device memory of a handle belongs to the library and is released by
 *     the matching destroy call.
 *   - Steps are enqueued asynchronously on the handle's stream; errors of the
 *     device work (a state leaving the verified range of the transfer map)
 *     surface at the next synchronising call (sync, observe, checkpoint,
 *     invariants).
 *   - delta must be a power of two (so delta*q and v/delta are exact in
 *     double); otherwise FQNM_ERR_ARG.
 *   - Integer states are int32 for scalar laws and int64 for the Euler
 *     system, laid out as [nvars][n] (structure of arrays).
 */
#ifndef FQNM_H
#define FQNM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    FQNM_OK = 0,
    FQNM_ERR_ARG = -1,       /* invalid argument (null, size, delta not 2^k) */
    FQNM_ERR_CFL = -2,       /* Courant number nu = alpha dt/dx > 1 (eq. cfl_number) */
    FQNM_ERR_RANGE = -3,     /* a state left the range on which the map is verified */
    FQNM_ERR_OVERFLOW = -4,  /* a state or transfer does not fit its integer type */
    FQNM_ERR_OOM = -5,       /* device memory or batch memory budget exhausted */
    FQNM_ERR_CUDA = -6,      /* CUDA runtime error (message in fqnm_last_error) */
    FQNM_ERR_TIMEOUT = -7,   /* a bounded device or host wait ran out */
    FQNM_ERR_STATE = -8,     /* call out of order (e.g. step before load) */
    FQNM_ERR_BUSY = -9       /* batch: no free slot for the request right now */
} fqnm_status;

typedef enum { FQNM_BC_PERIODIC = 0, FQNM_BC_TRANSMISSIVE = 1 } fqnm_boundary;

/* Rounding of round() in eqs. quantisation and flux_table.  The paper's
 * prototype rounds half to even (the default); floor is the mean-field
 * closure n = floor(Np) of eq. mean_field_closure. */
typedef enum {
    FQNM_ROUND_HALF_EVEN = 0,
    FQNM_ROUND_HALF_AWAY = 1,
    FQNM_ROUND_FLOOR = 2
} fqnm_rounding;

/* Flux kinds.  Split fluxes f = f+ + f- (eq. flux_splitting):
 *   LINEAR_UPWIND  f = a u,     f+ = max(a,0) u,  f- = min(a,0) u
 *   LINEAR_LF      f = a u,     f+- = (f(u) +- alpha u)/2
 *   BURGERS_LF     f = u^2/2,   f+- = (f(u) +- alpha u)/2
 *   BURGERS_EO     f = u^2/2,   f+ = max(u,0)^2/2, f- = min(u,0)^2/2
 *   TABLE          caller-supplied integer maps phi+- (fqnm_create_table):
 *                  the transfer rule as the primitive object (§2.2, scope of
 *                  transfer-operator equivalence)
 *   BURGERS_GODUNOV  Burgers, the two-point Godunov flux (the exact Riemann
 *                  flux of u^2/2, eq. transfer_operator_equivalence_definition
 *                  rounded once per face).  Both Engquist-Osher maps are >= 0
 *                  and one of them is 0 at every face but a transonic shock,
 *                  where Godunov takes the larger flux, and x -> R(x dt/dx/delta)
 *                  is monotone; so Phi(qL, qR) = max(phi+_EO(qL), phi-_EO(qR))
 *                  exactly, and the solver steps with the EO tables and that
 *                  max at every face.  1-D only (not on grids, in the batch or
 *                  in the FV baseline); alpha >= max|u| for the CFL check.
 *   EULER_ROE      1-D Euler, gamma-law gas, Roe flux quantised per
 *                  conserved component (§3.3); nvars = 3                    */
typedef enum {
    FQNM_FLUX_LINEAR_UPWIND = 0,
    FQNM_FLUX_LINEAR_LF = 1,
    FQNM_FLUX_BURGERS_LF = 2,
    FQNM_FLUX_BURGERS_EO = 3,
    FQNM_FLUX_BURGERS_GODUNOV = 4,
    FQNM_FLUX_CUSTOM_SPLIT = 5,  /* fqnm_create_custom */
    FQNM_FLUX_TABLE = 8,
    FQNM_FLUX_EULER_ROE = 16
} fqnm_flux_kind;

typedef struct {
    int kind;        /* fqnm_flux_kind */
    double a;        /* advection speed (linear kinds) */
    double alpha;    /* LF bound, alpha >= max|f'(u)| (§2, after eq. flux_splitting) */
    double gamma;    /* ratio of specific heats (EULER_ROE) */
    int rounding;    /* fqnm_rounding */
} fqnm_flux;

typedef struct fqnm_solver fqnm_solver;

/* ---- solver lifecycle ---------------------------------------------------- */

/* Create a solver for one problem (§2: grid spacing dx, step dt, quantum
 * delta).  delta points to nvars values (1 scalar, 3 Euler), each a power of
 * two.  The Courant number nu = alpha*dt/dx (LF kinds) or |a|*dt/dx (upwind)
 * must be <= 1 (eq. cfl_number), else FQNM_ERR_CFL.  Touches no GPU: the
 * transfer rule is built at load time, when the visited range is known.
 * *out receives a handle to release with fqnm_destroy. */
fqnm_status fqnm_create(const fqnm_flux* flux, const double* delta, double dx,
                        double dt, int boundary, fqnm_solver** out);

/* Create a solver whose transfer rule is given directly as integer maps
 * phi_p[k] = phi+(lo+k), phi_m[k] = phi-(lo+k), k < count (host arrays,
 * copied).  States must stay in [lo, lo+count-1]; leaving it is
 * FQNM_ERR_RANGE.  delta only scales the observable. */
fqnm_status fqnm_create_table(const int32_t* phi_p, const int32_t* phi_m,
                              int64_t lo, int64_t count, double delta,
                              int boundary, fqnm_solver** out);

/* A custom monotone split f = f+ + f- (f+ nondecreasing, f- nonincreasing)
 * given as host callbacks of u, evaluated only when the transfer maps are
 * tabulated (at load, over the states' range plus the margin, and again when
 * a range escape widens it): phi+-(q) = R((f+-(delta*q) * lambda) * (1/delta))
 * with lambda = dt/dx, the order of the built-in kinds (eq. flux_table).
 * alpha >= max|f'| is used for the CFL check alpha*dt/dx <= 1.  The
 * callbacks must be deterministic; they are called from the calling thread
 * of fqnm_load_* and fqnm_sync/fqnm_step (recovery).  A map value outside
 * +-1e9 gives FQNM_ERR_OVERFLOW. */
typedef double (*fqnm_split_fn)(double u, void* user);
fqnm_status fqnm_create_custom(fqnm_split_fn fplus, fqnm_split_fn fminus, void* user,
                               double alpha, double delta, double dx, double dt,
                               int boundary, int rounding, fqnm_solver** out);

fqnm_status fqnm_destroy(fqnm_solver* s);

/* Use the caller's CUDA stream (a cudaStream_t, e.g. torch's current stream)
 * for all later work of this handle.  NULL selects the library's own
 * non-blocking stream. */
fqnm_status fqnm_set_stream(fqnm_solver* s, void* stream);

/* Options (fqnm_option) that override the automatic execution plan.  Plans
 * differ in speed only: every plan gives bit-identical states. */
typedef enum {
    FQNM_OPT_KERNEL = 0,     /* 0 auto, 1 naive one-step, 2 temporal-blocked, 4 resident: a
                                periodic line held whole by one block (V cells per thread,
                                V in 1, 2, 4, 8 dividing n, n / V <= 1024 threads), every step
                                of a call in one launch.  Auto takes 4 for periodic lines of
                                at most 512 cells when no temporal-blocked plan option is set,
                                else 2 (periodic) or 1. */
    FQNM_OPT_LAYOUT = 1,     /* 0 auto, 1 interleaved, 2 blocked (cells per thread contiguous),
                                3 / 4 runs of 4 / 8 consecutive cells per lane (a warp-wide
                                table gather then covers 128 / 256 neighbouring cells; needs
                                at least two runs per lane) */
    FQNM_OPT_CELLS_PER_THREAD = 2, /* 4, 8, 16 or 32; 0 auto */
    FQNM_OPT_BLOCK = 3,      /* threads per block, multiple of 32, <= 512 (32: one warp, no barrier); 0 auto */
    FQNM_OPT_K = 4,          /* time steps per launch (temporal block depth); 0 auto */
    FQNM_OPT_MARGIN = 5,     /* quanta added on each side of the loaded range (default 1024) */
    FQNM_OPT_CLOSED_FORM = 6,/* 1 (default): use a verified integer closed form when one exists */
    FQNM_OPT_RECOVER = 7,    /* 1 (default): on range escape widen the map and replay */
    FQNM_OPT_AUTOTUNE = 8,   /* 1: time candidate plans at load and keep the fastest: 1-D
                                temporal-blocked plans (cached per size class), or on a
                                grid the walk depths, (2-D) the register tiles and (3-D) the
                                one-step kernel, unless a d-D plan option (FQNM_OPT_ND_TILE,
                                FQNM_OPT_K) was set */
    FQNM_OPT_GRAPH = 9,      /* 1 (default): replay long step loops from a CUDA graph */
    FQNM_OPT_PDL = 10,       /* 1 (default): chain step launches with programmatic dependent
                                launch (the next launch's blocks start while the previous
                                drains, and wait for its results before reading them) */
    FQNM_OPT_PACK16 = 11,    /* 1: when |phi+-| < 2^15 on the range, gather both maps from one
                                32-bit word (half the table footprint, two more instructions
                                per cell); 0: never; -1, the default: on d-D grids only (in 1-D
                                the unpacked table is faster while it fits L1/L2) */
    FQNM_OPT_QUANTISE_MASK = 12, /* EULER_ROE: components evolved by integer transfer, bits
                                1 rho, 2 m, 4 E (default 7, componentwise).  1 is the density-
                                channel prototype of §3.3: m and E evolve in double with the
                                same Roe flux.  A component outside the mask holds the bits of
                                its double in the int64 state slot (load, checkpoint); its
                                invariants are reported as 0.  Set before loading. */
    FQNM_OPT_ND_TILE = 13    /* 2-D grids, K steps per launch (FQNM_OPT_K, default 4):
                                0 or 6 (default) warps walking y with the K steps pipelined
                                (K in 1, 2, 3, 4, 6, 8; others round down); 1..5 register tiles
                                of x by y cells, 1 64x64, 2 128x64, 3 64x32, 4 128x32, 5 32x128
                                (K below half the smaller side).  FQNM_OPT_KERNEL = 1 selects one
                                step per launch.  3-D grids take one step per launch by
                                default (warps streaming z slabs), or, when FQNM_OPT_K is set
                                or this option is 6, K steps per launch (K in 1..4, default 2)
                                by blocks of rows walking z. */,
    FQNM_OPT_VERIFY = 14,    /* 1: at each synchronising call, check that every integer
                                variable's total plus its counted boundary transfer still
                                equals its value at load (eq. exact_conservation holds for
                                every step, so a difference means the state was changed
                                outside the steps); FQNM_ERR_STATE if not.  One reduction per
                                sync.  Default 0. */
    FQNM_OPT_FP64 = 15       /* EULER_ROE: which IEEE double steps of the integer Roe step
                                run on the integer pipes instead of the FP64 unit (same
                                results bit for bit; the GB300's FP64 unit executes 2
                                operations per SM per cycle).  0: none; 1: the state's
                                conversion delta*q and the transfer's scaling and rounding;
                                2 (default): also every division and square root of the
                                Roe flux, correctly rounded from an FP32 seed, Newton steps
                                in 64-bit fixed point and an exact integer remainder, and
                                its exact halvings and doublings on the exponent field;
                                3: also the products of the wave strengths with the
                                eigenvectors (the FP64 instruction takes over for operands
                                outside these paths: subnormals, infinities, NaN). */
} fqnm_option;
fqnm_status fqnm_set_option(fqnm_solver* s, int option, int64_t value);

/* ---- states --------------------------------------------------------------- */

/* eq. quantisation on the GPU: q_i = round(u_i/delta) with the given rounding.
 * u: n doubles; q_out: n int32 (state_bits = 32) or int64 (64).  _device
 * takes device pointers and runs on `stream` (NULL: legacy default stream);
 * the host variant stages through device memory.  A value that does not fit
 * the state type is FQNM_ERR_OVERFLOW. */
fqnm_status fqnm_quantise(const double* u, size_t n, double delta, int rounding,
                          int state_bits, void* q_out);
fqnm_status fqnm_quantise_device(const double* u, size_t n, double delta,
                                 int rounding, int state_bits, void* q_out,
                                 void* stream);

/* Load the initial integer state (host or device pointer; int32 [n] for
 * scalar laws, int64 [3][n] for EULER_ROE).  Builds the transfer rule over
 * the loaded range (eq. flux_table, on the GPU), verifies any integer closed
 * form against it, and resets the step counter and boundary-flux totals.
 * FQNM_ERR_ARG for n = 0; scalar states beyond +-2^30 (no headroom for a
 * step's transfers in int32) are FQNM_ERR_OVERFLOW. */
fqnm_status fqnm_load_states(fqnm_solver* s, const void* q, size_t n_cells);
fqnm_status fqnm_load_states_device(fqnm_solver* s, const void* q,
                                    size_t n_cells);

/* Quantise a double field u ([nvars][n], host or device pointer) on the GPU
 * with the flux's rounding (eq. quantisation, per-variable delta) and load
 * it as the initial state, exactly as fqnm_load_states would load the
 * quantised integers.  A host field passes through a device staging buffer
 * of nvars*n doubles that the handle keeps (shared with fqnm_observe) until
 * fqnm_destroy. */
fqnm_status fqnm_load_field(fqnm_solver* s, const double* u, size_t n_cells,
                            int on_device);

/* Advance k steps of eq. update_rule (asynchronous). */
fqnm_status fqnm_step(fqnm_solver* s, uint64_t k);

/* Wait for the handle's stream and report device-side errors. */
fqnm_status fqnm_sync(fqnm_solver* s);

/* Observable u = delta*q (eq. reconstruction_operator) as double, [nvars][n].
 * fqnm_observe writes a host buffer (through the handle's staging buffer)
 * and synchronises; _device writes a device buffer (fp32 != 0: float)
 * asynchronously. */
fqnm_status fqnm_observe(fqnm_solver* s, double* u_out);
fqnm_status fqnm_observe_device(fqnm_solver* s, void* u_out, int fp32);

/* Copy the integer state out (host: synchronises; device: asynchronous). */
fqnm_status fqnm_checkpoint(fqnm_solver* s, void* q_out, uint64_t* step);
fqnm_status fqnm_checkpoint_device(fqnm_solver* s, void* q_out);

/* Exact integer invariants (Lemma on telescoping conservation, eq.
 * exact_conservation; Lemma on CFL stability (ii)-(iii)):
 *   mass[v] = sum_i q^v_i
 *   tv[v]   = sum_i |q^v_{i+1} - q^v_i| (periodic: includes the wrap face)
 *   l1[v]   = sum_i |q^v_i - other^v_i| (0 when other is NULL)
 *   boundary_flux[v] = transfer out of the right end minus into the left end
 *                      since load; sum q^v(now) = sum q^v(load) - it.
 * other must have the same shape.  Synchronises. */
typedef struct {
    int64_t mass[3];
    int64_t tv[3];
    int64_t l1[3];
    int64_t boundary_flux[3];
    uint64_t step;
    int32_t nvars;
} fqnm_invariants_t;
fqnm_status fqnm_invariants(fqnm_solver* s, const fqnm_solver* other,
                            fqnm_invariants_t* out);

/* Allocation-free invariants of a caller's int32 state.  The paper has no
 * counterpart to this call; it exists for callers that cannot let a library
 * allocate device memory: processes whose free device memory is held by
 * their own pool (a caching allocator such as PyTorch's keeps freed blocks,
 * so an outside cudaMalloc can fail while the pool has room), latency-critical
 * loops (cudaFree waits for the whole device) and services that must not grow
 * their device footprint after start-up.
 * Computes, like fqnm_invariants for one variable, out[0] = sum q,
 * out[1] = total variation (boundary FQNM_BC_PERIODIC includes the wrap face),
 * out[2] = sum |q - other| (0 when other is NULL).  q and other are device
 * pointers to n int32 (caller-owned, only read); out is a host int64[3].  Runs
 * on `stream` (NULL: legacy default stream) and waits for it before returning.
 * Its scratch is one static device array (about 98 KB) reserved on each GPU
 * where the library's device code is loaded (with CUDA's lazy module loading,
 * at the first call on that device) until the process exits; it calls no
 * cudaMalloc or cudaFree.
 *   - n must be 1 .. FQNM_NOALLOC_MAX_CELLS, else FQNM_ERR_ARG (no launch).
 *   - The first call on each device looks up the array's address with that
 *     device current; make it before any stream capture on that device.
 *   - All calls on a device share the array and it keeps the last call's
 *     contents (every slot a call reads is overwritten by that call first).
 *     Calls whose GPU work overlaps race on it: serialise them. */
#define FQNM_NOALLOC_MAX_CELLS (1LL << 26)
fqnm_status fqnm_invariants_noalloc(const int32_t* q, const int32_t* other,
                                    size_t n, int boundary, int64_t* out,
                                    void* stream);

/* Diagnostics for FQNM_OPT_FP64 (the paper has no counterpart: these are the
 * GB300 execution strategy's own checks).  Evaluates, elementwise on device
 * arrays a, b of n doubles, an IEEE double step as the integer Roe step forms
 * it on the integer pipes and as the FP64 instruction forms it:
 *   op 0: a / b (round to nearest even)      op 1: sqrt(a)
 *   op 2: (double)q * 2^e, q = the bits of a as int64, e = (int)b
 *   op 3: R(a * 2^e) as int64 with `rounding`, e = (int)b (0 when NaN,
 *         infinite or |R| >= 4e18)
 *   op 4: a * 2^k, k = (int)b in {-1, 1} (the exact halving and doubling)
 *   op 5: a * b (round to nearest even)
 * out_int / out_fp64: n int64 (the result's bits for ops 0-2, the integer
 * for op 3), the integer-pipe result and the FP64 instruction's; out_path: n
 * int32, bit 0 set when the integer path applied (ops 0, 1, 4, 5: otherwise the
 * FP64 instruction's value is taken), for op 3 bit 1 / bit 2 the out-of-range
 * flag of either side.  Device pointers, caller-owned; asynchronous on
 * `stream` (NULL: the legacy default stream).  FQNM_ERR_ARG for op or
 * rounding out of range or a null pointer. */
fqnm_status fqnm_fp64_check(int op, int rounding, const double* a, const double* b,
                            size_t n, int64_t* out_int, int64_t* out_fp64,
                            int32_t* out_path, void* stream);

/* ---- Level statistics (Supplementary Information, Entropy and Statistical
 * Structure) ------------------------------------------------------------------
 * For one step q^n -> q^{n+1} of a scalar solver:
 *   c_k = #{i : q_i = k}, p_k = c_k / N              eq. pk_definition
 *   S = -sum_k p_k log p_k (natural log)             eq. discrete_entropy
 *   N_eff = exp(S)                                   eq. neff
 *   N_{k'k} = #{i : q_i^n = k, q_i^{n+1} = k'}       level-transition counts
 *   M_{k'k} = N_{k'k} / c_k^n                        eq. empirical_M
 *   rho = max_{k'} |sum_k M_{k'k} - 1|               row-sum defect
 * rho runs over the occupied levels k' of p^{n+1} (the only rows of M that
 * can be nonzero).  Counts are exact.  Each row sum is an exact sum of its
 * terms N_{k'k}/c_k^n, each rounded to a multiple of 2^-62 (|error| <=
 * (nonzero entries in the row) 2^-63; exact for a permutation or a column
 * sent whole to one level), then rounded to double; S is summed in double
 * in a fixed order.  All results are reproducible run to run.  Scalar (int32) solvers only: FQNM_ERR_ARG
 * for an Euler solver. */
typedef struct {
    uint64_t step;          /* n */
    int64_t n_cells;
    int64_t occupied_prev;  /* #{k : c_k^n > 0} */
    int64_t occupied;       /* #{k : c_k^{n+1} > 0} */
    double S_prev;          /* S(p^n) */
    double S;               /* S(p^{n+1}) */
    double n_eff;           /* exp(S(p^{n+1})) */
    double rho;             /* row-sum defect of M^n */
    int64_t rho_level;      /* the smallest k' attaining rho */
    int64_t pairs;          /* nonzero entries of N^n */
    int64_t moved;          /* cells with q_i^{n+1} != q_i^n */
} fqnm_level_stats_t;

/* Advance the solver by exactly one step (as fqnm_step(s, 1), including
 * range recovery) and compute the statistics of that transition.  Keeps a
 * device copy of q^n and the sorted nonzero entries of N^n for
 * fqnm_level_transitions.  Synchronises the solver's stream.  Device memory
 * is grown on first use (about 40 bytes per cell plus 24 bytes per level
 * between min and max of the two states) and released by fqnm_destroy. */
fqnm_status fqnm_level_step(fqnm_solver* s, fqnm_level_stats_t* out);

/* records times: advance every-1 steps, then fqnm_level_step into out[r]
 * (host array of `records`).  The entropy production rate of Definition
 * (discrete entropy production rate) is (S - S_prev) / dt of each record. */
fqnm_status fqnm_level_series(fqnm_solver* s, uint64_t records, uint64_t every,
                              fqnm_level_stats_t* out);

/* The nonzero entries of N^n of the last fqnm_level_step, sorted by k then k':
 * host arrays k, k_next, count of capacity cap.  *pairs receives the number
 * of entries; FQNM_ERR_ARG if cap is smaller (nothing copied), FQNM_ERR_STATE
 * if no transition was recorded. */
fqnm_status fqnm_level_transitions(fqnm_solver* s, int64_t* k, int64_t* k_next,
                                   int64_t* count, size_t cap, size_t* pairs);

/* Dense level counts c_k of the current state over [*lo, *lo + *len), where
 * lo and lo + len - 1 are the state's min and max, into the host array
 * counts of capacity cap (FQNM_ERR_ARG, with *lo and *len set, if smaller).
 * Synchronises the solver's stream. */
fqnm_status fqnm_level_histogram(fqnm_solver* s, int64_t* lo, int64_t* counts,
                                 size_t cap, size_t* len);

/* ---- Cartesian grids (Theorem, Cartesian extension by directional
 * composition; eqs. nd_transfer_rule, nd_flux_definition) ---------------------
 * Declare the loaded state a periodic d-dimensional grid (d = 2 or 3;
 * dims[0] fastest, n = dims[0] * ... * dims[d-1]; d = 1 restores the line).
 * Each step then applies the solver's one-dimensional rule along every axis:
 *   q_i <- q_i - sum_m (F_{i+e_m/2} - F_{i-e_m/2}),
 *   F_{i+e_m/2} = phi+(q_i) + phi-(q_{i+e_m}),
 * all fluxes from the state before the step.  Mass is conserved exactly;
 * fqnm_invariants reports TV summed over the axes.  Call before loading, on
 * a periodic scalar solver.  FQNM_ERR_CFL when d * (Courant number) > 1
 * (the monotonicity bound of the composed scheme), FQNM_ERR_ARG for a bad
 * shape, FQNM_ERR_STATE after loading. */
fqnm_status fqnm_set_grid(fqnm_solver* s, int d, const size_t* dims);

/* ---- Hopf-Lax entropy reference of inviscid Burgers (§3.2) ------------------
 * The dense-grid entropy reference of the Burgers test (Lax-Oleinik formula):
 *   u_i = (x_i - y_{j*}) / t,  j* = argmin_j  U0y_j + (x_i - y_j)^2 / (2 t)
 * over the candidates (y_j, U0y_j), U0y_j = int_0^{y_j} u0 (periodic data:
 * pass the periodic images y_j + m with U0y_j + m * mean(u0)).  Evaluated
 * as d = x_i - y_j; ((d*d) * inv2t) + U0y_j with inv2t = 1/(2t), each
 * operation rounded once; ties go to the smallest j (-0 and +0 tie); NaN
 * objectives are never the minimum, and a point whose objectives are all
 * NaN or +inf gets u = NaN and idx = -1.
 * x[nx], y[ny], U0y[ny] in; u[nx] and idx[nx] (int64, may be NULL) out.
 * on_device = 1: all arrays are device pointers and the call is
 * asynchronous on `stream` (NULL: the legacy default stream); 0: host arrays,
 * copied, and the call synchronises.  Partial minima over chunks of the
 * candidates take stream-ordered device scratch (16 bytes per point and
 * chunk, freed on the stream).  FQNM_ERR_ARG for a null array, empty input
 * or t not positive and finite. */
fqnm_status fqnm_hopf_lax(const double* x, size_t nx, const double* y,
                          const double* U0y, size_t ny, double t, double* u,
                          int64_t* idx, int on_device, void* stream);

/* Resume from a checkpoint: load the host states q (as fqnm_load_states),
 * then set the step counter to `step` and the accumulated boundary transfer
 * to boundary_flux[nvars] (NULL: zero), so that invariants, checkpoints and
 * FQNM_OPT_VERIFY continue as in an uninterrupted run.  A run resumed from
 * (fqnm_checkpoint, fqnm_invariants().boundary_flux) is bit-identical to the
 * uninterrupted one. */
fqnm_status fqnm_resume(fqnm_solver* s, const void* q, size_t n_cells, uint64_t step,
                        const int64_t* boundary_flux);

/* The solver's live device state (int32 [n] or int64 [3][n]) after a
 * synchronisation; valid until the next step, load or destroy.  Writing to
 * it bypasses the steps (FQNM_OPT_VERIFY reports a changed total). */
fqnm_status fqnm_state_device(fqnm_solver* s, void** q, size_t* n_cells);

/* Number of cells and of conserved variables of the loaded state (0 cells
 * before the first load). */
fqnm_status fqnm_get_size(fqnm_solver* s, size_t* n_cells, int* nvars);

/* Description of the transfer rule built at load (eq. flux_table). */
typedef struct {
    int64_t lo, hi;        /* q range the maps are tabulated and verified on */
    int32_t evaluator;     /* 1 table gather, 2 integer closed form */
    int32_t has_plus, has_minus;
    int32_t monotone;      /* certificate: phi+ nondecreasing, phi- nonincreasing
                              and q - phi+(q) + phi-(q) nondecreasing on the
                              range, so the integer update is a monotone scheme */
    int64_t num, den;      /* closed form phi+(q) = round(q*num/den) when evaluator = 2 */
    int32_t closed_form_sign; /* +1: closed form is phi+, -1: phi- */
    int32_t recoveries;    /* range escapes repaired by widening and replay */
} fqnm_rule_info;
fqnm_status fqnm_get_rule(fqnm_solver* s, fqnm_rule_info* out);

/* Copy the transfer tables (phi+ and phi- over [lo, hi]) to host arrays of
 * hi-lo+1 int32 each. */
fqnm_status fqnm_get_tables(fqnm_solver* s, int32_t* phi_p, int32_t* phi_m);

/* Execution statistics since load (or since the last reset). */
typedef struct {
    uint64_t launches;      /* kernels launched by step calls */
    uint64_t steps;
    uint64_t cell_updates;  /* n * steps */
    int32_t kernel;         /* 1 naive (or d-D one step), 2 temporal-blocked, 3 Euler,
                               4 resident (k = 0), 5 d-D walk, 6 d-D register tile (layout =
                               the FQNM_OPT_ND_TILE code, k = steps per launch) */
    int32_t layout, cells_per_thread, block, k;
    int32_t graph;          /* 1 if step loops are replayed from a CUDA graph */
} fqnm_stats;
fqnm_status fqnm_get_stats(fqnm_solver* s, fqnm_stats* out, int reset);

/* ---- floating-point finite-volume baseline -------------------------------- */

/* The classical split finite-volume operator of eq.
 * classical_operator_definition, u_i <- u_i - dt/dx (F(u_i,u_{i+1}) -
 * F(u_{i-1},u_i)), F(uL,uR) = f+(uL) + f-(uR), with the same flux as the
 * integer solver, in float (precision 32) or double (64), one step per
 * launch (or K, fqnm_fv_set_k), no FMA contraction.  EULER_ROE runs the Roe
 * flux on [3][n]. */
typedef struct fqnm_fv fqnm_fv;
fqnm_status fqnm_fv_create(const fqnm_flux* flux, double dx, double dt,
                           int boundary, int precision, fqnm_fv** out);
fqnm_status fqnm_fv_destroy(fqnm_fv* f);
fqnm_status fqnm_fv_set_stream(fqnm_fv* f, void* stream);
/* u: [nvars][n] doubles (host or device); converted to the precision. */
fqnm_status fqnm_fv_load(fqnm_fv* f, const double* u, size_t n_cells);
fqnm_status fqnm_fv_load_device(fqnm_fv* f, const double* u, size_t n_cells);
fqnm_status fqnm_fv_step(fqnm_fv* f, uint64_t k);
/* Time steps per launch of a periodic scalar baseline, 1..64 (default 1):
 * K > 1 runs the steps in tiles with a K-cell halo, the temporal blocking of
 * the integer kernel (an execution strategy: results are bit-identical to
 * K = 1).  FQNM_ERR_ARG for K outside 1..64, or K > 1 on a transmissive or
 * Euler baseline. */
fqnm_status fqnm_fv_set_k(fqnm_fv* f, int k);
fqnm_status fqnm_fv_observe(fqnm_fv* f, double* u_out);          /* host, syncs */
fqnm_status fqnm_fv_observe_device(fqnm_fv* f, double* u_out);   /* device */
fqnm_status fqnm_fv_launches(fqnm_fv* f, uint64_t* launches);
/* Cells and variables of the loaded field (0 cells before the first load). */
fqnm_status fqnm_fv_get_size(fqnm_fv* f, size_t* n_cells, int* nvars);

/* ---- batched serving ------------------------------------------------------ */

/* Continuous batching of many independent periodic scalar problems of uneven
 * size and step count (each one the method of §2 on its own grid).  Waiting
 * problems are admitted as slots and device memory (the budget, one arena
 * allocated at create) free up; every epoch one persistent launch, replayed
 * from a CUDA graph, advances every active problem by up to K steps of the
 * temporal-blocked update; finished states are copied to host memory.  Each
 * result is bit-identical to solving the problem alone with fqnm_step. */
typedef struct fqnm_batch fqnm_batch;
typedef struct {
    fqnm_flux flux;        /* a scalar split flux (not TABLE or EULER_ROE) */
    double delta, dx, dt;  /* as in fqnm_create; delta a power of two */
    int boundary;          /* FQNM_BC_PERIODIC */
} fqnm_problem_spec;

/* mem_budget_bytes: device arena for states and transfer tables (allocated
 * here); max_slots: problems on the device at once; stream: NULL for the
 * library's own.  FQNM_ERR_OOM if the arena cannot be allocated. */
fqnm_status fqnm_batch_create(size_t mem_budget_bytes, int max_slots,
                              void* stream, fqnm_batch** out);
fqnm_status fqnm_batch_destroy(fqnm_batch* b);
/* Execution plan of the batched launch (0 keeps a value): cells per thread
 * (4, 8, 16), threads per block, steps per epoch K, layout (1 interleaved, 2
 * blocked, 3 runs of 4 cells with 8 or 16 cells per thread, 4 runs of 8 with
 * 16).  Takes effect at the next epoch (epochs already enqueued finish
 * first); results do not depend on it. */
fqnm_status fqnm_batch_set_plan(fqnm_batch* b, int cells_per_thread, int block,
                                int k, int layout);
/* Autotune the plan online: the next epochs with work try the candidates
 * in turn (blocked or runs of 8 cells, cells per thread 8/16, 32/128/256
 * threads, K 32/64/128, halo work at most half the tile), epochs_per_plan
 * epochs each, and keep the one with the least wall time between epoch
 * retirements per time step (the wait of an active problem per step, the
 * epoch's fixed costs included; the host's admission and bookkeeping
 * overlap the GPU's epochs).  Candidates are timed only on epochs that step
 * at least 16 problems (the first epochs of a stream, with a few small
 * problems, would favour the smallest tiles); until then the current plan
 * runs.  The default plan is blocked, 8 cells per thread, 128 threads,
 * K = 128. */
fqnm_status fqnm_batch_autotune(fqnm_batch* b, int epochs_per_plan);
/* The quanta added on each side of a request's state range when its
 * transfer maps are built (default 1024), for requests submitted after this
 * call.  A state that leaves the maps restarts its problem with the margin
 * widened (x4, at least 4096); the result is the same.  FQNM_ERR_ARG for a
 * negative margin. */
fqnm_status fqnm_batch_set_margin(fqnm_batch* b, int64_t margin);
/* The current plan; *tuning = 1 while candidates are still being tried. */
fqnm_status fqnm_batch_get_plan(fqnm_batch* b, int* cells_per_thread, int* block,
                                int* k, int* layout, int* tuning);
/* Queue a problem: q0 is a host int32 [n] (copied), `steps` time steps.
 * arrival_ns (fqnm_clock_ns clock; 0 = now) is when the request arrives: it
 * is not admitted before, and its latency is measured from it.  Validates
 * like fqnm_create.  *id receives its ticket (0, 1, 2, ...). */
fqnm_status fqnm_batch_submit(fqnm_batch* b, const fqnm_problem_spec* spec,
                              const int32_t* q0, size_t n, uint64_t steps,
                              uint64_t arrival_ns, int64_t* id);
/* Queue a problem whose initial state is already on the device: q0 is a
 * device int32 [n] that must stay valid and unchanged until the problem has
 * finished (it is copied at admission, and again if a range escape restarts
 * the problem); out, if not NULL, is
 * a device int32 [n] that receives the final state (then poll returns no
 * host state).  The state range is taken on the GPU at admission. */
fqnm_status fqnm_batch_submit_device(fqnm_batch* b, const fqnm_problem_spec* spec,
                                     const int32_t* q0, size_t n, uint64_t steps,
                                     uint64_t arrival_ns, int32_t* out, int64_t* id);
/* Run up to max_epochs epochs (admission, one batched launch, retirement),
 * stopping early when nothing has arrived or is active.  Reports how many
 * problems are on the device and how many still wait. */
fqnm_status fqnm_batch_progress(fqnm_batch* b, int max_epochs, int* n_active,
                                int* n_queued);
/* If problem `id` is finished: copy its final state to q_out (host int32,
 * room for `capacity` values, at least the problem's n; may be NULL), its
 * arrival-to-result latency in ns, set *done = 1 and release the result (a
 * second poll is FQNM_ERR_STATE).  Else *done = 0.  A capacity below n is
 * FQNM_ERR_ARG and releases nothing. */
fqnm_status fqnm_batch_poll(fqnm_batch* b, int64_t id, int32_t* q_out,
                            size_t capacity, uint64_t* latency_ns, int* done);
/* Pop up to max_ids tickets of problems finished since the last call (in
 * completion order) into ids; *n receives how many. */
fqnm_status fqnm_batch_completed(fqnm_batch* b, int64_t* ids, int max_ids, int* n);
/* Batched launches, cell updates and epochs executed so far, and the GPU
 * time of the epochs' launches in ms (CUDA events around each epoch). */
fqnm_status fqnm_batch_stats(fqnm_batch* b, uint64_t* launches,
                             uint64_t* cell_updates, uint64_t* epochs, double* gpu_ms);
/* The monotonic clock (ns) the batch uses for arrivals and latencies. */
uint64_t fqnm_clock_ns(void);

/* ---- diagnostics ---------------------------------------------------------- */

const char* fqnm_last_error(void);
/* Number of CUDA kernels this library has launched in this process (kernels
 * inside a replayed CUDA graph count one each). */
uint64_t fqnm_kernel_launches(void);
const char* fqnm_status_string(int status);
/* Library version as major*10000 + minor*100 + patch. */
int fqnm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* FQNM_H */
