// levels.h -- level statistics of integer states (entropy appendix); the
// kernels are in k_levels.cu.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace fqnm {

// Same layout as fqnm_level_stats_t in the public header.
struct LevelRecord {
    uint64_t step;
    long long n_cells, occupied_prev, occupied;
    double S_prev, S, n_eff, rho;
    long long rho_level, pairs, moved;
};

struct LevelWork;                 // device buffers, grown on demand

LevelWork* level_work_create();
void level_work_destroy(LevelWork* w);

// Copy of q^n kept for the next transition.
cudaError_t level_snapshot(LevelWork* w, const int32_t* q, int64_t n, cudaStream_t st);
const int32_t* level_snap(const LevelWork* w);

// Statistics of q^n -> q^{n+1} (device states of n cells, levels in
// [lo, lo + W)), enqueued on st; the record stays on the device until
// level_record.  An out-of-range level is skipped and sets ERRBIT_RANGE in
// the work's own error word (reported by level_record).
cudaError_t level_transition(LevelWork* w, const int32_t* qn, const int32_t* qn1, int64_t n,
                             int64_t lo, int64_t W, cudaStream_t st);
// Copies the record and the error word to the host; synchronises st.
cudaError_t level_record(LevelWork* w, LevelRecord* host, unsigned* host_err, cudaStream_t st);

// The nonzero entries of N^n of the last transition (host arrays of `pairs`
// entries each), sorted by k then k'.  Synchronises st.
cudaError_t level_export_pairs(LevelWork* w, int64_t pairs, int64_t* k, int64_t* kn, int64_t* cnt,
                               cudaStream_t st);

// Dense counts c_k of q over [lo, lo + W) into a host array, and the error
// word.  Synchronises st.
cudaError_t level_histogram(LevelWork* w, const int32_t* q, int64_t n, int64_t lo, int64_t W,
                            int64_t* counts, unsigned* host_err, cudaStream_t st);

}  // namespace fqnm
