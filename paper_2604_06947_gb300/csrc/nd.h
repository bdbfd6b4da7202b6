// nd.h -- the d-dimensional step by directional composition (k_nd.cu).
#pragma once

#include "fqnm_internal.h"

namespace fqnm {

// A periodic Cartesian grid, dims[0] fastest; unused dims are 1.
struct NdGrid {
    int d;
    long long dims[3];
    long long cells() const { return dims[0] * dims[1] * dims[2]; }
};

// One step of eq. nd_transfer_rule on an int32 state, d = 2 or 3 (the rule's
// maps on every axis).  A state outside the rule's range sets ERRBIT_RANGE,
// an update that leaves int32 ERRBIT_OVERFLOW.
cudaError_t launch_step_nd(const RuleView& r, const int32_t* qin, int32_t* qout, const NdGrid& g,
                           unsigned* err, cudaStream_t st);

// 2-D temporal-blocked plans: tile shape (x by y cells) and K steps per launch.
enum NdTile { ND_TILE_64x64 = 1, ND_TILE_128x64 = 2, ND_TILE_64x32 = 3, ND_TILE_128x32 = 4,
              ND_TILE_32x128 = 5, ND_WALK = 6 };
struct NdPlan {
    int blocked = 0;              // 0: one step per launch (walking kernels)
    int walk = 1;                 // blocked: 1 pipelined walk along y, 0 register tiles
    int shape = ND_TILE_64x32;
    int k = 4;
};
int nd_tile_x(int shape);
int nd_tile_y(int shape);

// K steps of eq. nd_transfer_rule on a 2-D grid in one launch (K < min(TX, TY) / 2).
cudaError_t launch_step2d_tb(const RuleView& r, const NdPlan& p, const int32_t* qin,
                             int32_t* qout, const NdGrid& g, int K, unsigned* err,
                             cudaStream_t st);

// K steps of eq. nd_transfer_rule on a 2-D grid in one launch by a pipelined
// walk along y (K in {1, 2, 3, 4, 6, 8}).
bool walk_k_supported(int K);
cudaError_t launch_walk2d(const RuleView& r, const int32_t* qin, int32_t* qout, const NdGrid& g,
                          int K, unsigned* err, cudaStream_t st);

// K steps of eq. nd_transfer_rule on a 3-D grid in one launch by a pipelined
// walk along z (K in 1 .. 4).
bool walk3_k_supported(int K);
cudaError_t launch_walk3d(const RuleView& r, const int32_t* qin, int32_t* qout, const NdGrid& g,
                          int K, unsigned* err, cudaStream_t st);

// mass, TV summed over the axes (periodic faces), l1 to other (may be null),
// added to acc[0..2].
cudaError_t launch_invariants_nd(const int32_t* q, const int32_t* other, const NdGrid& g,
                                 long long* acc, cudaStream_t st);

}  // namespace fqnm
