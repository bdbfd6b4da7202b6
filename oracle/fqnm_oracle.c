/*
 * fqnm_oracle.c -- plain, slow, single-threaded CPU oracle for the FQNM
 * quantised conservative step (arXiv 2604.06947).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * bench's CPU-baseline leg load this file.  It shares no code, header, table
 * or constant generator with the CUDA library; it is the definition of the
 * method written out, in the paper's notation, so that a reader can check it
 * against the paper by eye.
 *
 * Build: gcc -O2 -ffp-contract=off -fPIC -shared fqnm_oracle.c -lm
 * (no FMA contraction: every floating-point expression below is evaluated
 * operation by operation, left to right, in IEEE double unless stated.)
 *
 * Readings of the paper used here (where it is silent or ambiguous):
 *   R1  round() is round-half-to-even (C nearbyint in the default mode);
 *       half-away-from-zero and floor are selectable alternatives.
 *   R2  phi(q) = R( fl( fl(f(fl(delta*q))) * lambda ) * (1/delta) ) with
 *       lambda = fl(dt/dx); delta a power of two, so the scalings by delta and
 *       1/delta are exact.
 *   R3  the hot path uses split rounding (each phi rounded on its own,
 *       eq. update_rule); the two-point form of eq.
 *       transfer_operator_equivalence_definition rounds the joint flux.
 *   R4  transmissive ends copy the edge cell into a ghost cell.
 *   R5  the Euler/Roe flux is the textbook Roe flux without entropy fix,
 *       evaluated in the order written in orc_roe_flux().
 *
 * Parity pins for every function are in tests/test_oracle_*.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* Flux kinds (oracle numbering). */
enum {
    ORC_LINEAR_UPWIND = 0,  /* f+ = max(a,0) u,  f- = min(a,0) u            */
    ORC_LINEAR_LF = 1,      /* f = a u,    f+- = (f(u) +- alpha u)/2         */
    ORC_BURGERS_LF = 2,     /* f = u^2/2,  f+- = (f(u) +- alpha u)/2         */
    ORC_BURGERS_EO = 3,     /* f+ = max(u,0)^2/2, f- = min(u,0)^2/2          */
    ORC_BURGERS_GODUNOV = 4 /* two-point only: exact Riemann flux of u^2/2  */
};
enum { ORC_ROUND_HALF_EVEN = 0, ORC_ROUND_HALF_AWAY = 1, ORC_ROUND_FLOOR = 2 };
enum { ORC_PERIODIC = 0, ORC_TRANSMISSIVE = 1 };

/* ------------------------------------------------------------------------ */
/* Rounding, eq. quantisation and eq. flux_table (reading R1).               */
/* ------------------------------------------------------------------------ */
static double orc_round(double v, int mode)
{
    if (mode == ORC_ROUND_HALF_AWAY) return round(v);
    if (mode == ORC_ROUND_FLOOR) return floor(v);
    return nearbyint(v);                    /* half to even */
}

/* eq. quantisation: q = round(u/delta).  Returns 0, or -1 if some q does not
 * fit in 62 bits. */
int orc_quantise(const double* u, int64_t n, double delta, int rounding,
                 int64_t* q)
{
    int bad = 0;
    for (int64_t i = 0; i < n; i++) {
        double v = orc_round(u[i] / delta, rounding);
        if (!(fabs(v) < 4.0e18)) { bad = 1; q[i] = 0; continue; }
        q[i] = (int64_t)v;
    }
    return bad ? -1 : 0;
}

/* The physical flux f(u) of each kind. */
static double orc_f(int kind, double a, double u)
{
    if (kind == ORC_LINEAR_UPWIND || kind == ORC_LINEAR_LF) return a * u;
    return 0.5 * (u * u);
}

/* Split fluxes of eq. flux_splitting.  sign = +1 for f+, -1 for f-. */
static double orc_fsplit(int kind, double a, double alpha, int sign, double u)
{
    switch (kind) {
    case ORC_LINEAR_UPWIND:
        if (sign > 0) return (a > 0.0 ? a : 0.0) * u;
        return (a < 0.0 ? a : 0.0) * u;
    case ORC_LINEAR_LF:
    case ORC_BURGERS_LF: {
        double f = orc_f(kind, a, u);
        double d = alpha * u;
        return 0.5 * (sign > 0 ? f + d : f - d);
    }
    case ORC_BURGERS_EO: {
        double w = sign > 0 ? (u > 0.0 ? u : 0.0) : (u < 0.0 ? u : 0.0);
        return 0.5 * (w * w);
    }
    default:
        return 0.0;
    }
}

/* eq. flux_table: phi+-(q) = round( f+-(delta q) * (dt/dx) * delta^-1 ). */
static int64_t orc_phi(int kind, double a, double alpha, int sign, int64_t q,
                       double delta, double lambda, int rounding)
{
    double u = delta * (double)q;
    double t = orc_fsplit(kind, a, alpha, sign, u);
    double s = t * lambda;
    return (int64_t)orc_round(s * (1.0 / delta), rounding);
}

/* Tabulate phi+ and phi- for q = lo .. lo+count-1 (table construction is the
 * only place rounding enters, Table 1 "Rounding exposure"). */
int orc_split_table(int kind, double a, double alpha, double delta, double dx,
                    double dt, int rounding, int64_t lo, int64_t count,
                    int64_t* phi_p, int64_t* phi_m)
{
    double lambda = dt / dx;
    for (int64_t k = 0; k < count; k++) {
        phi_p[k] = orc_phi(kind, a, alpha, +1, lo + k, delta, lambda, rounding);
        phi_m[k] = orc_phi(kind, a, alpha, -1, lo + k, delta, lambda, rounding);
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* A memo of the split maps: a table over the range seen so far; values      */
/* outside it are evaluated from the definition directly.                    */
/* ------------------------------------------------------------------------ */
typedef struct {
    int kind, rounding;
    double a, alpha, delta, lambda;
    int64_t lo, count;
    int64_t* p;
    int64_t* m;
} orc_maps;

static int orc_maps_init(orc_maps* M, int kind, double a, double alpha,
                         double delta, double dx, double dt, int rounding,
                         const int64_t* q, int64_t n, int64_t margin)
{
    int64_t lo = q[0], hi = q[0];
    for (int64_t i = 1; i < n; i++) {
        if (q[i] < lo) lo = q[i];
        if (q[i] > hi) hi = q[i];
    }
    M->kind = kind; M->rounding = rounding; M->a = a; M->alpha = alpha;
    M->delta = delta; M->lambda = dt / dx;
    M->lo = lo - margin;
    M->count = hi - lo + 1 + 2 * margin;
    M->p = (int64_t*)malloc(sizeof(int64_t) * (size_t)M->count);
    M->m = (int64_t*)malloc(sizeof(int64_t) * (size_t)M->count);
    if (!M->p || !M->m) { free(M->p); free(M->m); return -1; }
    for (int64_t k = 0; k < M->count; k++) {
        M->p[k] = orc_phi(kind, a, alpha, +1, M->lo + k, delta, M->lambda, rounding);
        M->m[k] = orc_phi(kind, a, alpha, -1, M->lo + k, delta, M->lambda, rounding);
    }
    return 0;
}

static void orc_maps_free(orc_maps* M) { free(M->p); free(M->m); }

static int64_t orc_pp(const orc_maps* M, int64_t q)
{
    int64_t k = q - M->lo;
    if (k >= 0 && k < M->count) return M->p[k];
    return orc_phi(M->kind, M->a, M->alpha, +1, q, M->delta, M->lambda, M->rounding);
}

static int64_t orc_pm(const orc_maps* M, int64_t q)
{
    int64_t k = q - M->lo;
    if (k >= 0 && k < M->count) return M->m[k];
    return orc_phi(M->kind, M->a, M->alpha, -1, q, M->delta, M->lambda, M->rounding);
}

/* ------------------------------------------------------------------------ */
/* eq. update_rule / update_rule_conservative_form, cell form.               */
/*   F_{i+1/2} = phi+(q_i) + phi-(q_{i+1})                                   */
/*   q_i <- q_i - (F_{i+1/2} - F_{i-1/2})                                    */
/* Periodic: indices mod n.  Transmissive: ghosts q_{-1}=q_0, q_n=q_{n-1}.   */
/* bflux (may be NULL) accumulates F_{n-1/2} - F_{-1/2} over the steps, so  */
/* that sum(q) changes by exactly -bflux (zero for periodic).                */
/* ------------------------------------------------------------------------ */
int orc_step_split(int kind, double a, double alpha, double delta, double dx,
                   double dt, int rounding, int boundary, int64_t* q,
                   int64_t n, int64_t steps, int64_t* bflux)
{
    if (n <= 0) return 0;
    orc_maps M;
    if (orc_maps_init(&M, kind, a, alpha, delta, dx, dt, rounding, q, n, 64))
        return -1;
    int64_t* F = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!F) { orc_maps_free(&M); return -1; }
    /* F[i+1] holds F_{i+1/2}; F[0] holds F_{-1/2}. */
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t i = 0; i < n; i++) {
            int64_t right = (i + 1 < n) ? q[i + 1]
                          : (boundary == ORC_PERIODIC ? q[0] : q[n - 1]);
            F[i + 1] = orc_pp(&M, q[i]) + orc_pm(&M, right);
        }
        if (boundary == ORC_PERIODIC) F[0] = F[n];
        else F[0] = orc_pp(&M, q[0]) + orc_pm(&M, q[0]);
        for (int64_t i = 0; i < n; i++)
            q[i] = q[i] - (F[i + 1] - F[i]);
        if (bflux) *bflux += F[n] - F[0];
    }
    free(F);
    orc_maps_free(&M);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Theorem (Cartesian extension by directional composition), eqs.            */
/* nd_transfer_rule and nd_flux_definition: on a periodic d-dimensional grid */
/* (d = 1..3, dims[0] fastest), with the same one-dimensional rule along     */
/* every axis,                                                               */
/*   F_{i+e_m/2} = phi+(q_i) + phi-(q_{i+e_m})                               */
/*   q_i <- q_i - sum_m (F_{i+e_m/2} - F_{i-e_m/2}).                         */
/* All face fluxes of a step are taken from the state before the step.      */
/* ------------------------------------------------------------------------ */
int orc_step_nd(int kind, double a, double alpha, double delta, double dx,
                double dt, int rounding, int d, const int64_t* dims,
                int64_t* q, int64_t steps)
{
    if (d < 1 || d > 3) return -2;
    int64_t n = 1, stride[3] = {1, 1, 1}, ext[3] = {1, 1, 1};
    for (int m = 0; m < d; m++) {
        if (dims[m] <= 0) return -2;
        ext[m] = dims[m];
        stride[m] = n;
        n *= dims[m];
    }
    orc_maps M;
    if (orc_maps_init(&M, kind, a, alpha, delta, dx, dt, rounding, q, n, 64)) return -1;
    /* Fup[m*n + i] = F_{i + e_m/2} */
    int64_t* Fup = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n * d));
    if (!Fup) { orc_maps_free(&M); return -1; }
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t i = 0; i < n; i++) {
            int64_t c[3] = {0, 0, 0}, r = i;
            for (int m = 0; m < d; m++) { c[m] = r % ext[m]; r /= ext[m]; }
            for (int m = 0; m < d; m++) {
                int64_t up = (c[m] + 1 < ext[m]) ? i + stride[m]
                                                 : i - (ext[m] - 1) * stride[m];
                Fup[m * n + i] = orc_pp(&M, q[i]) + orc_pm(&M, q[up]);
            }
        }
        for (int64_t i = 0; i < n; i++) {
            int64_t c[3] = {0, 0, 0}, r = i;
            for (int m = 0; m < d; m++) { c[m] = r % ext[m]; r /= ext[m]; }
            int64_t div = 0;
            for (int m = 0; m < d; m++) {
                int64_t dn = (c[m] > 0) ? i - stride[m] : i + (ext[m] - 1) * stride[m];
                div += Fup[m * n + i] - Fup[m * n + dn];
            }
            q[i] = q[i] - div;
        }
    }
    free(Fup);
    orc_maps_free(&M);
    return 0;
}

/* The same step written face by face: each face moves F quanta from its left
 * cell to its right cell (q_i -= F, q_{i+1} += F), the pairwise exchange
 * J_{i,i+1} = -J_{i+1,i} behind the telescoping of Lemma (telescoping
 * conservation).  Kept independent of orc_step_split on purpose: it evaluates
 * phi straight from the definition, with no memo. */
int orc_step_split_faces(int kind, double a, double alpha, double delta,
                         double dx, double dt, int rounding, int boundary,
                         int64_t* q, int64_t n, int64_t steps)
{
    if (n <= 0) return 0;
    double lambda = dt / dx;
    int64_t* old = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!old) return -1;
    for (int64_t s = 0; s < steps; s++) {
        memcpy(old, q, sizeof(int64_t) * (size_t)n);
        int64_t nfaces = (boundary == ORC_PERIODIC) ? n : n - 1;
        for (int64_t f = 0; f < nfaces; f++) {
            int64_t L = f, R = (f + 1) % n;
            int64_t F = orc_phi(kind, a, alpha, +1, old[L], delta, lambda, rounding)
                      + orc_phi(kind, a, alpha, -1, old[R], delta, lambda, rounding);
            q[L] -= F;
            q[R] += F;
        }
        if (boundary == ORC_TRANSMISSIVE) {
            /* boundary faces: flux against the ghost copy of the edge cell */
            int64_t Fl = orc_phi(kind, a, alpha, +1, old[0], delta, lambda, rounding)
                       + orc_phi(kind, a, alpha, -1, old[0], delta, lambda, rounding);
            int64_t Fr = orc_phi(kind, a, alpha, +1, old[n - 1], delta, lambda, rounding)
                       + orc_phi(kind, a, alpha, -1, old[n - 1], delta, lambda, rounding);
            q[0] += Fl;
            q[n - 1] -= Fr;
        }
    }
    free(old);
    return 0;
}

/* Sampled parity: the value of one cell after `steps` steps depends only on
 * the 2*steps+1 cells around it (nearest-neighbour stencil).  Given that
 * window of the initial state, evolve the shrinking window (each step drops
 * one cell at either end, whose neighbour is unknown) down to one cell. */
int orc_cone(int kind, double a, double alpha, double delta, double dx,
             double dt, int rounding, const int64_t* window, int64_t len,
             int64_t steps, int64_t* out)
{
    if (len != 2 * steps + 1) return -1;
    orc_maps M;
    if (orc_maps_init(&M, kind, a, alpha, delta, dx, dt, rounding, window, len, 64))
        return -1;
    int64_t* w = (int64_t*)malloc(sizeof(int64_t) * (size_t)len);
    int64_t* F = (int64_t*)malloc(sizeof(int64_t) * (size_t)len);
    if (!w || !F) { free(w); free(F); orc_maps_free(&M); return -1; }
    memcpy(w, window, sizeof(int64_t) * (size_t)len);
    int64_t L = len;
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t j = 0; j + 1 < L; j++)          /* face between j, j+1 */
            F[j] = orc_pp(&M, w[j]) + orc_pm(&M, w[j + 1]);
        for (int64_t j = 1; j + 1 < L; j++)          /* interior cells */
            w[j - 1] = w[j] - (F[j] - F[j - 1]);
        L -= 2;
    }
    *out = w[0];
    free(w); free(F); orc_maps_free(&M);
    return 0;
}

/* Windowed parity, the same dependency argument for a run of cells: W
 * consecutive cells after `steps` steps depend only on the window of
 * W + 2*steps cells around them.  `window` holds that window of the initial
 * state (len = W + 2*steps, periodic wrap already applied by the caller);
 * each step evaluates eq. update_rule on the cells whose two faces lie in
 * the window and drops the two outermost cells.  `out` receives the W
 * cells.  This is orc_cone for W > 1. */
int orc_window(int kind, double a, double alpha, double delta, double dx,
               double dt, int rounding, const int64_t* window, int64_t len,
               int64_t steps, int64_t* out)
{
    if (steps < 0 || len < 2 * steps + 1) return -1;
    orc_maps M;
    if (orc_maps_init(&M, kind, a, alpha, delta, dx, dt, rounding, window, len, 64))
        return -1;
    int64_t* w = (int64_t*)malloc(sizeof(int64_t) * (size_t)len);
    int64_t* F = (int64_t*)malloc(sizeof(int64_t) * (size_t)len);
    if (!w || !F) { free(w); free(F); orc_maps_free(&M); return -1; }
    memcpy(w, window, sizeof(int64_t) * (size_t)len);
    int64_t L = len;
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t j = 0; j + 1 < L; j++)          /* F[j]: face between j, j+1 */
            F[j] = orc_pp(&M, w[j]) + orc_pm(&M, w[j + 1]);
        for (int64_t j = 1; j + 1 < L; j++)          /* cell j has faces j-1, j */
            w[j - 1] = w[j] - (F[j] - F[j - 1]);
        L -= 2;
    }
    memcpy(out, w, sizeof(int64_t) * (size_t)L);
    free(w); free(F); orc_maps_free(&M);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Two-point transfer of eq. transfer_operator_equivalence_definition:       */
/*   Phi(qL,qR) = round( F(delta qL, delta qR) * dt/dx * delta^-1 )          */
/* with the joint flux rounded once (reading R3).                            */
/* ------------------------------------------------------------------------ */
static double orc_two_point_flux(int kind, double a, double alpha, double uL,
                                 double uR)
{
    if (kind == ORC_BURGERS_GODUNOV) {
        double fL = 0.5 * (uL * uL), fR = 0.5 * (uR * uR);
        if (uL <= uR) {                       /* rarefaction: min of f */
            if (uL > 0.0) return fL;
            if (uR < 0.0) return fR;
            return 0.0;
        }
        return fL > fR ? fL : fR;             /* shock: max of f */
    }
    return orc_fsplit(kind, a, alpha, +1, uL) + orc_fsplit(kind, a, alpha, -1, uR);
}

int64_t orc_two_point_phi(int kind, double a, double alpha, double delta,
                          double dx, double dt, int rounding, int64_t qL,
                          int64_t qR)
{
    double lambda = dt / dx;
    double F = orc_two_point_flux(kind, a, alpha, delta * (double)qL,
                                  delta * (double)qR);
    return (int64_t)orc_round((F * lambda) * (1.0 / delta), rounding);
}

int orc_step_two_point(int kind, double a, double alpha, double delta,
                       double dx, double dt, int rounding, int boundary,
                       int64_t* q, int64_t n, int64_t steps)
{
    if (n <= 0) return 0;
    int64_t* F = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!F) return -1;
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t i = 0; i < n; i++) {
            int64_t right = (i + 1 < n) ? q[i + 1]
                          : (boundary == ORC_PERIODIC ? q[0] : q[n - 1]);
            F[i + 1] = orc_two_point_phi(kind, a, alpha, delta, dx, dt, rounding,
                                         q[i], right);
        }
        F[0] = (boundary == ORC_PERIODIC) ? F[n]
             : orc_two_point_phi(kind, a, alpha, delta, dx, dt, rounding, q[0], q[0]);
        for (int64_t i = 0; i < n; i++) q[i] = q[i] - (F[i + 1] - F[i]);
    }
    free(F);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Invariants: total mass (eq. exact_conservation), total variation and      */
/* l1 distance (Lemma on CFL stability, items (ii) and (iii)).               */
/* out[0] = sum q; out[1] = TV (periodic: includes the wrap face);           */
/* out[2] = sum |q - other| (0 when other is NULL).                          */
/* ------------------------------------------------------------------------ */
int orc_invariants(const int64_t* q, int64_t n, const int64_t* other,
                   int boundary, int64_t* out)
{
    int64_t mass = 0, tv = 0, l1 = 0;
    for (int64_t i = 0; i < n; i++) {
        mass += q[i];
        if (i + 1 < n) tv += llabs(q[i + 1] - q[i]);
        if (other) l1 += llabs(q[i] - other[i]);
    }
    if (boundary == ORC_PERIODIC && n > 1) tv += llabs(q[0] - q[n - 1]);
    out[0] = mass; out[1] = tv; out[2] = l1;
    return 0;
}

/* Discrete level entropy S = -sum_k p_k log p_k with p_k the fraction of
 * cells at level k (Supplementary eq. pk_definition, discrete_entropy).
 * Levels are counted by sorting a copy. */
static int orc_cmp64(const void* x, const void* y)
{
    int64_t a = *(const int64_t*)x, b = *(const int64_t*)y;
    return (a > b) - (a < b);
}

double orc_level_entropy(const int64_t* q, int64_t n)
{
    if (n <= 0) return 0.0;
    int64_t* c = (int64_t*)malloc(sizeof(int64_t) * (size_t)n);
    if (!c) return NAN;
    memcpy(c, q, sizeof(int64_t) * (size_t)n);
    qsort(c, (size_t)n, sizeof(int64_t), orc_cmp64);
    double S = 0.0;
    int64_t run = 1;
    for (int64_t i = 1; i <= n; i++) {
        if (i < n && c[i] == c[i - 1]) { run++; continue; }
        double p = (double)run / (double)n;
        S -= p * log(p);
        run = 1;
    }
    free(c);
    return S;
}

/* ------------------------------------------------------------------------ */
/* Classical split finite-volume operator, eq. classical_operator_definition */
/*   u_i <- u_i - lambda (F(u_i,u_{i+1}) - F(u_{i-1},u_i)),                  */
/*   F(uL,uR) = f+(uL) + f-(uR),                                             */
/* in double and in float with the same operation order.                     */
/* ------------------------------------------------------------------------ */
int orc_fv_step_f64(int kind, double a, double alpha, double dx, double dt,
                    int boundary, double* u, int64_t n, int64_t steps)
{
    if (n <= 0) return 0;
    double lambda = dt / dx;
    double* F = (double*)malloc(sizeof(double) * (size_t)(n + 1));
    if (!F) return -1;
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t i = 0; i < n; i++) {
            double right = (i + 1 < n) ? u[i + 1]
                         : (boundary == ORC_PERIODIC ? u[0] : u[n - 1]);
            F[i + 1] = orc_fsplit(kind, a, alpha, +1, u[i])
                     + orc_fsplit(kind, a, alpha, -1, right);
        }
        F[0] = (boundary == ORC_PERIODIC) ? F[n]
             : orc_fsplit(kind, a, alpha, +1, u[0]) + orc_fsplit(kind, a, alpha, -1, u[0]);
        for (int64_t i = 0; i < n; i++) {
            double d = F[i + 1] - F[i];
            u[i] = u[i] - lambda * d;
        }
    }
    free(F);
    return 0;
}

static float orc_fsplit_f32(int kind, float a, float alpha, int sign, float u)
{
    switch (kind) {
    case ORC_LINEAR_UPWIND:
        if (sign > 0) return (a > 0.0f ? a : 0.0f) * u;
        return (a < 0.0f ? a : 0.0f) * u;
    case ORC_LINEAR_LF:
    case ORC_BURGERS_LF: {
        float f = (kind == ORC_LINEAR_LF) ? a * u : 0.5f * (u * u);
        float d = alpha * u;
        return 0.5f * (sign > 0 ? f + d : f - d);
    }
    case ORC_BURGERS_EO: {
        float w = sign > 0 ? (u > 0.0f ? u : 0.0f) : (u < 0.0f ? u : 0.0f);
        return 0.5f * (w * w);
    }
    default:
        return 0.0f;
    }
}

int orc_fv_step_f32(int kind, double a, double alpha, double dx, double dt,
                    int boundary, float* u, int64_t n, int64_t steps)
{
    if (n <= 0) return 0;
    float lambda = (float)(dt / dx);
    float af = (float)a, alf = (float)alpha;
    float* F = (float*)malloc(sizeof(float) * (size_t)(n + 1));
    if (!F) return -1;
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t i = 0; i < n; i++) {
            float right = (i + 1 < n) ? u[i + 1]
                        : (boundary == ORC_PERIODIC ? u[0] : u[n - 1]);
            F[i + 1] = orc_fsplit_f32(kind, af, alf, +1, u[i])
                     + orc_fsplit_f32(kind, af, alf, -1, right);
        }
        F[0] = (boundary == ORC_PERIODIC) ? F[n]
             : orc_fsplit_f32(kind, af, alf, +1, u[0]) + orc_fsplit_f32(kind, af, alf, -1, u[0]);
        for (int64_t i = 0; i < n; i++) {
            float d = F[i + 1] - F[i];
            u[i] = u[i] - lambda * d;
        }
    }
    free(F);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* 1-D Euler, Roe flux (§3.3 "Sod shock tube under Roe flux quantisation").  */
/* Conserved U = (rho, m, E), p = (gamma-1)(E - m^2/(2 rho)).                */
/* Textbook Roe flux, no entropy fix (reading R5), evaluated in this order:  */
/*   iK = 1/rhoK; uK = mK*iK; pK = (g-1)*(EK - 0.5*(rhoK*(uK*uK)));          */
/*   HK = (EK+pK)*iK                                                         */
/*   sL = sqrt(rhoL); sR = sqrt(rhoR); w = sL + sR; iw = 1/w                 */
/*   ut = (sL*uL + sR*uR)*iw;  Ht = (sL*HL + sR*HR)*iw                       */
/*   ct = sqrt((g-1)*(Ht - 0.5*(ut*ut)))                                     */
/*   d0 = rhoR-rhoL; d1 = mR-mL; d2 = ER-EL                                  */
/*   a2 = (g-1)/(ct*ct) * ((d0*(Ht - ut*ut) + ut*d1) - d2)                   */
/*   a1 = ((d0*(ut+ct) - d1) - ct*a2) / (2*ct);  a3 = d0 - (a1 + a2)         */
/*   l1 = |ut-ct|, l2 = |ut|, l3 = |ut+ct|                                   */
/*   r1 = (1, ut-ct, Ht-ut*ct), r2 = (1, ut, 0.5*(ut*ut)),                    */
/*   r3 = (1, ut+ct, Ht+ut*ct)                                               */
/*   F_k = 0.5*(fL_k + fR_k) - 0.5*((l1*a1*r1_k + l2*a2*r2_k) + l3*a3*r3_k)  */
/* with f(U) = (m, m*u + p, u*(E + p)) and products grouped left to right.   */
/* ------------------------------------------------------------------------ */
void orc_roe_flux(double g, const double* UL, const double* UR, double* F)
{
    double rhoL = UL[0], mL = UL[1], EL = UL[2];
    double rhoR = UR[0], mR = UR[1], ER = UR[2];
    double iL = 1.0 / rhoL, iR = 1.0 / rhoR;
    double uL = mL * iL, uR = mR * iR;
    double pL = (g - 1.0) * (EL - 0.5 * (rhoL * (uL * uL)));
    double pR = (g - 1.0) * (ER - 0.5 * (rhoR * (uR * uR)));
    double HL = (EL + pL) * iL, HR = (ER + pR) * iR;
    double sL = sqrt(rhoL), sR = sqrt(rhoR), w = sL + sR, iw = 1.0 / w;
    double ut = (sL * uL + sR * uR) * iw;
    double Ht = (sL * HL + sR * HR) * iw;
    double ct = sqrt((g - 1.0) * (Ht - 0.5 * (ut * ut)));
    double d0 = rhoR - rhoL, d1 = mR - mL, d2 = ER - EL;
    double a2 = (g - 1.0) / (ct * ct) * ((d0 * (Ht - ut * ut) + ut * d1) - d2);
    double a1 = ((d0 * (ut + ct) - d1) - ct * a2) / (2.0 * ct);
    double a3 = d0 - (a1 + a2);
    double l1 = fabs(ut - ct), l2 = fabs(ut), l3 = fabs(ut + ct);
    double r1[3] = {1.0, ut - ct, Ht - ut * ct};
    double r2[3] = {1.0, ut, 0.5 * (ut * ut)};
    double r3[3] = {1.0, ut + ct, Ht + ut * ct};
    double fL[3] = {mL, mL * uL + pL, uL * (EL + pL)};
    double fR[3] = {mR, mR * uR + pR, uR * (ER + pR)};
    for (int k = 0; k < 3; k++) {
        double diss = (l1 * a1 * r1[k] + l2 * a2 * r2[k]) + l3 * a3 * r3[k];
        F[k] = 0.5 * (fL[k] + fR[k]) - 0.5 * diss;
    }
}

/* Integer Euler step: Phi^k_{i+1/2} = round( F^k_Roe(delta q_i, delta q_{i+1})
 * * dt/dx * delta_k^-1 ) for each conserved component k (the two-point
 * transfer of eq. transfer_operator_equivalence_definition applied per
 * component), then q^k_i -= Phi^k_{i+1/2} - Phi^k_{i-1/2}.  q is SoA
 * [3][n] int64; ends are transmissive (ghost = edge).  bflux[k] accumulates
 * Phi^k_{n-1/2} - Phi^k_{-1/2}, so sum_i q^k changes by exactly -bflux[k]. */
int orc_euler_roe_step(double g, const double* delta, double dx, double dt,
                       int rounding, int64_t* q, int64_t n, int64_t steps,
                       int64_t* bflux)
{
    if (n <= 0) return 0;
    double lambda = dt / dx;
    int64_t* Phi = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n + 1));
    if (!Phi) return -1;
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t f = 0; f <= n; f++) {          /* face f-1/2, f = 0..n */
            int64_t iL = f - 1 < 0 ? 0 : f - 1;
            int64_t iR = f < n ? f : n - 1;
            double UL[3], UR[3], F[3];
            for (int k = 0; k < 3; k++) {
                UL[k] = delta[k] * (double)q[k * n + iL];
                UR[k] = delta[k] * (double)q[k * n + iR];
            }
            orc_roe_flux(g, UL, UR, F);
            for (int k = 0; k < 3; k++)
                Phi[k * (n + 1) + f] =
                    (int64_t)orc_round((F[k] * lambda) * (1.0 / delta[k]), rounding);
        }
        for (int k = 0; k < 3; k++) {
            int64_t* P = Phi + k * (n + 1);
            for (int64_t i = 0; i < n; i++)
                q[k * n + i] = q[k * n + i] - (P[i + 1] - P[i]);
            if (bflux) bflux[k] += P[n] - P[0];
        }
    }
    free(Phi);
    return 0;
}

/* Windowed parity for the integer Euler step: after `steps` steps a cell
 * depends only on the cells within `steps` of it (each face reads its two
 * neighbours), or on the domain's edge cell through the transmissive ghost.
 * `qw` is [3][len] SoA: cells [a, a+len) of a domain [0, n); left_end says
 * a == 0 and right_end says a+len == n, where the ghost of
 * orc_euler_roe_step applies.  Each step evaluates the faces whose two
 * cells are known (plus the ghost faces at a domain end) and updates the
 * cells that have both faces, so a side that is not a domain end loses one
 * cell per step.  `out` ([3][W], W = len - steps*(2 - left_end - right_end))
 * receives the surviving cells, which equal cells
 * [a + (left_end ? 0 : steps), ...) of the full run. */
int orc_euler_window(double g, const double* delta, double dx, double dt,
                     int rounding, const int64_t* qw, int64_t len,
                     int left_end, int right_end, int64_t steps, int64_t* out)
{
    int64_t shrink = (left_end ? 0 : 1) + (right_end ? 0 : 1);
    if (steps < 0 || len < 1 || len - shrink * steps < 1) return -1;
    double lambda = dt / dx;
    int64_t* q = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)len);
    int64_t* Phi = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(len + 1));
    if (!q || !Phi) { free(q); free(Phi); return -1; }
    memcpy(q, qw, sizeof(int64_t) * 3 * (size_t)len);
    int64_t lo = 0, hi = len - 1;                   /* cells still exact */
    for (int64_t s = 0; s < steps; s++) {
        /* face f sits between cells f-1 and f (f = lo..hi+1); the outer
         * faces exist only at a domain end, against the ghost copy */
        int64_t f0 = left_end ? lo : lo + 1, f1 = right_end ? hi + 1 : hi;
        for (int64_t f = f0; f <= f1; f++) {
            int64_t iL = f - 1 < lo ? lo : f - 1;
            int64_t iR = f > hi ? hi : f;
            double UL[3], UR[3], F[3];
            for (int k = 0; k < 3; k++) {
                UL[k] = delta[k] * (double)q[k * len + iL];
                UR[k] = delta[k] * (double)q[k * len + iR];
            }
            orc_roe_flux(g, UL, UR, F);
            for (int k = 0; k < 3; k++)
                Phi[k * (len + 1) + f] =
                    (int64_t)orc_round((F[k] * lambda) * (1.0 / delta[k]), rounding);
        }
        int64_t c0 = left_end ? lo : lo + 1, c1 = right_end ? hi : hi - 1;
        for (int k = 0; k < 3; k++) {
            int64_t* P = Phi + k * (len + 1);
            for (int64_t i = c0; i <= c1; i++)
                q[k * len + i] = q[k * len + i] - (P[i + 1] - P[i]);
        }
        lo = c0;
        hi = c1;
    }
    int64_t W = hi - lo + 1;
    for (int k = 0; k < 3; k++)
        memcpy(out + k * W, q + k * len + lo, sizeof(int64_t) * (size_t)W);
    free(q);
    free(Phi);
    return 0;
}

/* The density-channel prototype of §3.3: only the components whose bit is
 * set in `mask` (1 rho, 2 m, 4 E) are quantised and updated by integer
 * transfer as in orc_euler_roe_step; the others are kept in double (uf,
 * [3][n]) and updated with the same Roe flux by the floating-point
 * finite-volume update u <- u - lambda (F_{i+1/2} - F_{i-1/2}).  The flux of
 * every face is evaluated on U = (quantised: delta q; otherwise: uf). */
int orc_euler_roe_step_mask(double g, const double* delta, double dx, double dt,
                            int rounding, int mask, int64_t* q, double* uf,
                            int64_t n, int64_t steps, int64_t* bflux)
{
    if (mask < 0 || mask > 7) return -2;
    if (n <= 0) return 0;
    double lambda = dt / dx;
    double* Fx = (double*)malloc(sizeof(double) * 3 * (size_t)(n + 1));
    int64_t* Phi = (int64_t*)malloc(sizeof(int64_t) * 3 * (size_t)(n + 1));
    if (!Fx || !Phi) { free(Fx); free(Phi); return -1; }
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t f = 0; f <= n; f++) {
            int64_t iL = f - 1 < 0 ? 0 : f - 1;
            int64_t iR = f < n ? f : n - 1;
            double UL[3], UR[3], F[3];
            for (int k = 0; k < 3; k++) {
                int quant = (mask >> k) & 1;
                UL[k] = quant ? delta[k] * (double)q[k * n + iL] : uf[k * n + iL];
                UR[k] = quant ? delta[k] * (double)q[k * n + iR] : uf[k * n + iR];
            }
            orc_roe_flux(g, UL, UR, F);
            for (int k = 0; k < 3; k++) {
                Fx[k * (n + 1) + f] = F[k];
                Phi[k * (n + 1) + f] =
                    ((mask >> k) & 1) ? (int64_t)orc_round((F[k] * lambda) * (1.0 / delta[k]), rounding) : 0;
            }
        }
        for (int k = 0; k < 3; k++) {
            if ((mask >> k) & 1) {
                int64_t* P = Phi + k * (n + 1);
                for (int64_t i = 0; i < n; i++) q[k * n + i] = q[k * n + i] - (P[i + 1] - P[i]);
                if (bflux) bflux[k] += P[n] - P[0];
            } else {
                double* Fk = Fx + k * (n + 1);
                for (int64_t i = 0; i < n; i++) {
                    double d = Fk[i + 1] - Fk[i];
                    uf[k * n + i] = uf[k * n + i] - lambda * d;
                }
            }
        }
    }
    free(Fx);
    free(Phi);
    return 0;
}

/* Floating-point Roe finite-volume step (the FP reference of the Sod test):
 * U_i <- U_i - lambda (F_{i+1/2} - F_{i-1/2}), same flux, transmissive. */
int orc_euler_fv_step_f64(double g, double dx, double dt, double* U, int64_t n,
                          int64_t steps)
{
    if (n <= 0) return 0;
    double lambda = dt / dx;
    double* Fx = (double*)malloc(sizeof(double) * 3 * (size_t)(n + 1));
    if (!Fx) return -1;
    for (int64_t s = 0; s < steps; s++) {
        for (int64_t f = 0; f <= n; f++) {
            int64_t iL = f - 1 < 0 ? 0 : f - 1;
            int64_t iR = f < n ? f : n - 1;
            double UL[3] = {U[iL], U[n + iL], U[2 * n + iL]};
            double UR[3] = {U[iR], U[n + iR], U[2 * n + iR]};
            double F[3];
            orc_roe_flux(g, UL, UR, F);
            for (int k = 0; k < 3; k++) Fx[k * (n + 1) + f] = F[k];
        }
        for (int k = 0; k < 3; k++)
            for (int64_t i = 0; i < n; i++) {
                double d = Fx[k * (n + 1) + i + 1] - Fx[k * (n + 1) + i];
                U[k * n + i] = U[k * n + i] - lambda * d;
            }
    }
    free(Fx);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Exact Riemann solution of the 1-D Euler equations for an ideal gas,       */
/* written from the standard construction: the star pressure p* is the      */
/* root of fL(p) + fR(p) + (uR - uL) = 0, where fK is the shock (Rankine-    */
/* Hugoniot) branch for p > pK and the rarefaction (isentropic, Riemann      */
/* invariant) branch otherwise; the solution is self-similar in x/t.         */
/* Used as the calibration reference of the Sod test (§3.3).                 */
/* ------------------------------------------------------------------------ */
static double orc_fK(double g, double p, double rK, double pK, double* dfdp)
{
    double cK = sqrt(g * pK / rK);
    if (p > pK) {
        double A = 2.0 / ((g + 1.0) * rK), B = (g - 1.0) / (g + 1.0) * pK;
        double s = sqrt(A / (p + B));
        *dfdp = s * (1.0 - 0.5 * (p - pK) / (p + B));
        return (p - pK) * s;
    }
    double e = (g - 1.0) / (2.0 * g);
    *dfdp = 1.0 / (rK * cK) * pow(p / pK, -(g + 1.0) / (2.0 * g));
    return 2.0 * cK / (g - 1.0) * (pow(p / pK, e) - 1.0);
}

/* star[0..3] = p*, u*, rho*L, rho*R.  Returns 0, -1 on vacuum generation. */
int orc_riemann_star(double g, double rL, double uL, double pL, double rR,
                     double uR, double pR, double* star)
{
    double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    if (2.0 / (g - 1.0) * (cL + cR) <= uR - uL) return -1;
    /* bisection on [lo, hi] bracketing the root, then Newton polish */
    double lo = 1e-14, hi = 10.0 * (pL > pR ? pL : pR) + 10.0;
    double d;
    for (int it = 0; it < 200; it++) {
        double mid = 0.5 * (lo + hi);
        double fm = orc_fK(g, mid, rL, pL, &d) + orc_fK(g, mid, rR, pR, &d) + (uR - uL);
        if (fm > 0.0) hi = mid; else lo = mid;
    }
    double p = 0.5 * (lo + hi);
    for (int it = 0; it < 4; it++) {
        double dL, dR;
        double f = orc_fK(g, p, rL, pL, &dL) + orc_fK(g, p, rR, pR, &dR) + (uR - uL);
        double np = p - f / (dL + dR);
        if (np > 0.0) p = np;
    }
    double dL, dR;
    double fL = orc_fK(g, p, rL, pL, &dL), fR = orc_fK(g, p, rR, pR, &dR);
    double us = 0.5 * (uL + uR) + 0.5 * (fR - fL);
    double gm = (g - 1.0) / (g + 1.0);
    double rsL = (p > pL) ? rL * ((p / pL + gm) / (gm * p / pL + 1.0))
                          : rL * pow(p / pL, 1.0 / g);
    double rsR = (p > pR) ? rR * ((p / pR + gm) / (gm * p / pR + 1.0))
                          : rR * pow(p / pR, 1.0 / g);
    star[0] = p; star[1] = us; star[2] = rsL; star[3] = rsR;
    return 0;
}

/* Sample the exact solution at positions x (interface at x0) and time t. */
int orc_riemann_sample(double g, double rL, double uL, double pL, double rR,
                       double uR, double pR, double x0, double t,
                       const double* x, int64_t n, double* rho, double* u,
                       double* p)
{
    double st[4];
    if (orc_riemann_star(g, rL, uL, pL, rR, uR, pR, st)) return -1;
    double ps = st[0], us = st[1], rsL = st[2], rsR = st[3];
    double cL = sqrt(g * pL / rL), cR = sqrt(g * pR / rR);
    for (int64_t i = 0; i < n; i++) {
        double S = (t > 0.0) ? (x[i] - x0) / t : (x[i] < x0 ? -INFINITY : INFINITY);
        double r, v, pr;
        if (S <= us) {                                  /* left of contact */
            if (ps > pL) {                              /* left shock */
                double SL = uL - cL * sqrt((g + 1.0) / (2.0 * g) * ps / pL
                                           + (g - 1.0) / (2.0 * g));
                if (S <= SL) { r = rL; v = uL; pr = pL; }
                else { r = rsL; v = us; pr = ps; }
            } else {                                    /* left rarefaction */
                double csL = cL * pow(ps / pL, (g - 1.0) / (2.0 * g));
                double SH = uL - cL, ST = us - csL;
                if (S <= SH) { r = rL; v = uL; pr = pL; }
                else if (S >= ST) { r = rsL; v = us; pr = ps; }
                else {
                    v = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * uL + S);
                    double c = 2.0 / (g + 1.0) * (cL + 0.5 * (g - 1.0) * (uL - S));
                    r = rL * pow(c / cL, 2.0 / (g - 1.0));
                    pr = pL * pow(c / cL, 2.0 * g / (g - 1.0));
                }
            }
        } else {                                        /* right of contact */
            if (ps > pR) {                              /* right shock */
                double SR = uR + cR * sqrt((g + 1.0) / (2.0 * g) * ps / pR
                                           + (g - 1.0) / (2.0 * g));
                if (S >= SR) { r = rR; v = uR; pr = pR; }
                else { r = rsR; v = us; pr = ps; }
            } else {                                    /* right rarefaction */
                double csR = cR * pow(ps / pR, (g - 1.0) / (2.0 * g));
                double SH = uR + cR, ST = us + csR;
                if (S >= SH) { r = rR; v = uR; pr = pR; }
                else if (S <= ST) { r = rsR; v = us; pr = ps; }
                else {
                    v = 2.0 / (g + 1.0) * (-cR + 0.5 * (g - 1.0) * uR + S);
                    double c = 2.0 / (g + 1.0) * (cR - 0.5 * (g - 1.0) * (uR - S));
                    r = rR * pow(c / cR, 2.0 / (g - 1.0));
                    pr = pR * pow(c / cR, 2.0 * g / (g - 1.0));
                }
            }
        }
        rho[i] = r; u[i] = v; p[i] = pr;
    }
    return 0;
}

/* Shock speed of the right-moving shock (for the calibration window test). */
double orc_riemann_right_shock_speed(double g, double rL, double uL, double pL,
                                     double rR, double uR, double pR)
{
    double st[4];
    if (orc_riemann_star(g, rL, uL, pL, rR, uR, pR, st)) return NAN;
    double cR = sqrt(g * pR / rR);
    return uR + cR * sqrt((g + 1.0) / (2.0 * g) * st[0] / pR + (g - 1.0) / (2.0 * g));
}
