// woi_kernels.h -- launch parameters and launchers of the libwoi kernels
// (internal to the library; the public interface is include/woi.h).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "woi_layout.h"

namespace woi {

constexpr int kMixedMaxBlock = 256;
constexpr int kMixedMinBlocks = 3;    // resident blocks per SM the walk kernels are compiled for
// the general-surface kernels of 2D and 3D (star curves, meshes) wait on long dependent
// chains (root refinement, hierarchy loads) and gain more from a fourth resident block
// (64 registers) than they lose to spills: 9 % (star) and 15 % (meshes) faster; in 4-6D
// (ellipsoids) the spills cost more (12 % slower), and on spheres 2-4 % slower.  The
// variance-reduced kernels of 4-6D carry two chains of d-vectors and are compiled for two
// blocks (128 registers): 6D spheres 512 -> 417 ms (in 2-3D two blocks were slower)
template <int D, bool STAR, bool VR = false>
constexpr int mixed_min_blocks() { return (VR && D >= 4) ? 2 : ((STAR && D <= 3) ? 4 : kMixedMinBlocks); }
constexpr int kSharedBlock = 128;     // threads per block of the shared-trajectory kernel
constexpr int kTile = 32;             // points per shared-trajectory tile

struct MixedParams {
    const InstDesc *inst;              // device [n_inst]; units of instance k start at inst[k].unit_begin
    int n_inst;
    int64_t total_units;
    unsigned long long *queue;         // device work-queue head (batch: one per instance), zero before the launch
    int max_surf;                      // batch: the most surfaces of any instance (per-warp table size)
    double *partials;                  // device [total_units][2 (dim+1)]
    int walks_per_lane;
    uint64_t seed;
};

struct FinalizeParams {
    int dim;
    int64_t n_pts;
    int64_t n_walks;
    int sched_group;
    int64_t unit_begin;
    int64_t chunks_per_point;
    const double *partials;            // unit partials, or [n_pts][2 (dim+1)] accumulators
    int tile;                          // > 0: shared-trajectory rows [(tile, chunk)][tile points]
    double *u, *grad, *se_u, *se_grad; // device, each may be null
    double *moments;                   // device [n_pts][2][dim+1], may be null
};

struct Fp64PointParams {
    const DevGeom *geom;
    const double *x;                   // device [dim]
    uint32_t point_id, instance_id;
    int64_t walk_begin, n_walks;
    int sched_group;
    uint64_t seed;
    double *acc;                       // device [2 (dim+1)]
};

struct WalkValuesParams {
    const DevGeom *geom;
    const double *x;                   // device [dim]
    uint32_t point_id, instance_id;
    const uint64_t *walks;             // device [n]
    int64_t n;
    int sched_group;
    uint64_t seed;
    double *f_u, *f_grad;              // device [n], [n][dim]
    double *trace;                     // device [n][chains][M+1][dim+2] (y, Q, T per step) or null
};

// launchers of one dimension / star flag; defined in woi_kernels_impl.cuh and
// explicitly instantiated in woi_k<d>.cu
template <int D, bool STAR>
struct DimLaunchers {
    static cudaError_t mixed(bool vr, const MixedParams &p, int grid, int block, size_t smem, cudaStream_t s);
    static cudaError_t occupancy(bool vr, int block, size_t smem, int *blocks_per_sm);
    static cudaError_t mixed_warp(bool vr, const MixedParams &p, int grid, int block, size_t smem, cudaStream_t s);
    static cudaError_t occupancy_warp(bool vr, int block, size_t smem, int *blocks_per_sm);
    static cudaError_t shared(bool vr, const MixedParams &p, int grid, size_t smem, cudaStream_t s);
    static cudaError_t occupancy_shared(bool vr, size_t smem, int *blocks_per_sm);
    static cudaError_t fp64_point(bool vr, const Fp64PointParams &p, int grid, cudaStream_t s);
    static cudaError_t values(bool vr, bool fp64, const WalkValuesParams &p, cudaStream_t s);
};
template <int D, bool STAR> struct DimTag {
    using L = DimLaunchers<D, STAR>;
};
extern template struct DimLaunchers<2, false>;
extern template struct DimLaunchers<2, true>;
extern template struct DimLaunchers<3, false>;
extern template struct DimLaunchers<4, false>;
extern template struct DimLaunchers<5, false>;
extern template struct DimLaunchers<6, false>;
extern template struct DimLaunchers<3, true>;
extern template struct DimLaunchers<4, true>;
extern template struct DimLaunchers<5, true>;
extern template struct DimLaunchers<6, true>;

struct BatchFinalizeParams {
    const InstDesc *inst;              // device [n_inst], sorted by point_begin
    int n_inst;
    int dim;
    int64_t total_points;
    const double *partials;            // unit partials of all instances
};

// batched kernel: warp units of many instances, queue = one head per instance; dynamic shared
// memory (block / 32) * max_surf * kMaxDim floats
cudaError_t launch_mixed(int dim, bool vr, bool star, const MixedParams &p, int grid, int block, size_t smem,
                         cudaStream_t s);
cudaError_t launch_finalize_batch(const BatchFinalizeParams &p, cudaStream_t s);
cudaError_t mixed_occupancy(int dim, bool vr, bool star, int block, size_t smem, int *blocks_per_sm);
// single-instance kernel with warp-level work units of 32 x walks_per_lane walks;
// dynamic shared memory: (block / 32) * n_surf * kMaxDim floats
cudaError_t launch_mixed_warp(int dim, bool vr, bool star, const MixedParams &p, int grid, int block, size_t smem,
                              cudaStream_t s);
cudaError_t mixed_warp_occupancy(int dim, bool vr, bool star, int block, size_t smem, int *blocks_per_sm);
// shared-trajectory kernel (tiles of kTile points share walks); dynamic shared memory:
// (kSharedBlock / 32) * chains * (M + 1) * 32 * shared_record_floats(dim) * 4 bytes
// (a record: yhi, ylo and the coefficient; in odd dim padded to whole float4 vectors)
constexpr int shared_record_floats(int dim) { return dim % 2 == 0 ? 2 * dim + 1 : ((2 * dim + 1) + 3) / 4 * 4; }
cudaError_t launch_shared(int dim, bool vr, bool star, const MixedParams &p, int grid, size_t smem, cudaStream_t s);
cudaError_t shared_occupancy(int dim, bool vr, bool star, size_t smem, int *blocks_per_sm);
cudaError_t launch_finalize(const FinalizeParams &p, bool from_acc, cudaStream_t s);
cudaError_t launch_fp64_point(int dim, bool vr, bool star, const Fp64PointParams &p, cudaStream_t s);
cudaError_t launch_walk_values(int dim, bool vr, bool star, bool fp64, const WalkValuesParams &p, cudaStream_t s);

}  // namespace woi
