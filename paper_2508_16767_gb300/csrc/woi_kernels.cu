// woi_kernels.cu -- finalize kernels and the dispatch of the walk kernels
// over the dimension (the walk kernels are instantiated in woi_k<d>.cu).
#include <cuda_runtime.h>

#include "woi_kernels.h"

namespace woi {

// ---------------------------------------------------------------------------
// finalize: ordered sums of the unit partials -> mean, SE, raw moments
// ---------------------------------------------------------------------------
__global__ void k_finalize(FinalizeParams p)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int D = p.dim, C = D + 1;
    if (idx >= p.n_pts * C) return;
    const int64_t point = idx / C;
    const int c = (int)(idx - point * C);
    double S1 = 0.0, S2 = 0.0;
    if (p.tile > 0) {
        const int64_t t = point / p.tile, q = point - t * p.tile;
        for (int64_t ch = 0; ch < p.chunks_per_point; ++ch) {
            const double *row = p.partials + ((t * p.chunks_per_point + ch) * p.tile + q) * (2 * C);
            S1 += row[c];
            S2 += row[C + c];
        }
    } else {
        const double *src = p.partials + (p.unit_begin + point * p.chunks_per_point) * (2 * C);
        for (int64_t ch = 0; ch < p.chunks_per_point; ++ch) {
            S1 += src[ch * 2 * C + c];
            S2 += src[ch * 2 * C + C + c];
        }
    }
    if (p.moments) {
        p.moments[point * 2 * C + c] = S1;
        p.moments[point * 2 * C + C + c] = S2;
    }
    const double W = (double)p.n_walks;
    const double G = W / (double)p.sched_group;
    const double mean = S1 / W;
    double var = (S2 - G * mean * mean) / (G > 1.0 ? G - 1.0 : 1.0);
    var = var > 0.0 ? var : 0.0;
    const double se = sqrt(var / G);
    if (c == 0) {
        if (p.u) p.u[point] = mean;
        if (p.se_u) p.se_u[point] = se;
    } else {
        if (p.grad) p.grad[point * D + c - 1] = mean;
        if (p.se_grad) p.se_grad[point * D + c - 1] = se;
    }
}

// the per-point accumulators [n_pts][2(D+1)] -> outputs
__global__ void k_finalize_acc(FinalizeParams p)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int D = p.dim, C = D + 1;
    if (idx >= p.n_pts * C) return;
    const int64_t point = idx / C;
    const int c = (int)(idx - point * C);
    const double S1 = p.partials[point * 2 * C + c], S2 = p.partials[point * 2 * C + C + c];
    if (p.moments) {
        p.moments[point * 2 * C + c] = S1;
        p.moments[point * 2 * C + C + c] = S2;
    }
    const double W = (double)p.n_walks, G = W / (double)p.sched_group, mean = S1 / W;
    double var = (S2 - G * mean * mean) / (G > 1.0 ? G - 1.0 : 1.0);
    var = var > 0.0 ? var : 0.0;
    const double se = sqrt(var / G);
    if (c == 0) {
        if (p.u) p.u[point] = mean;
        if (p.se_u) p.se_u[point] = se;
    } else {
        if (p.grad) p.grad[point * D + c - 1] = mean;
        if (p.se_grad) p.se_grad[point * D + c - 1] = se;
    }
}

// batched finalize: one thread per (instance point, component)
__global__ void k_finalize_batch(BatchFinalizeParams p)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int D = p.dim, C = D + 1;
    if (idx >= p.total_points * C) return;
    const int64_t gp = idx / C;
    const int c = (int)(idx - gp * C);
    int lo = 0, hi = p.n_inst;  // last instance with point_begin <= gp
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (p.inst[m].point_begin <= gp) lo = m; else hi = m;
    }
    const InstDesc &id = p.inst[lo];
    const int64_t point = gp - id.point_begin;
    const double *src = p.partials + (id.unit_begin + point * id.chunks_per_point) * (2 * C);
    double S1 = 0.0, S2 = 0.0;
    for (int64_t ch = 0; ch < id.chunks_per_point; ++ch) {
        S1 += src[ch * 2 * C + c];
        S2 += src[ch * 2 * C + C + c];
    }
    const double W = (double)id.n_walks, G = W / (double)id.sched_group, mean = S1 / W;
    double var = (S2 - G * mean * mean) / (G > 1.0 ? G - 1.0 : 1.0);
    var = var > 0.0 ? var : 0.0;
    const double se = sqrt(var / G);
    if (c == 0) {
        if (id.u) id.u[point] = mean;
        if (id.se_u) id.se_u[point] = se;
    } else {
        if (id.grad) id.grad[point * D + c - 1] = mean;
        if (id.se_grad) id.se_grad[point * D + c - 1] = se;
    }
}

cudaError_t launch_finalize_batch(const BatchFinalizeParams &p, cudaStream_t s)
{
    const int64_t n = p.total_points * (p.dim + 1);
    if (n == 0) return cudaSuccess;
    k_finalize_batch<<<(int)((n + 255) / 256), 256, 0, s>>>(p);
    return cudaGetLastError();
}

template <typename F>
static cudaError_t by_dim(int dim, bool star, F &&f)
{
    switch (dim) {
    case 2: return star ? f(DimTag<2, true>{}) : f(DimTag<2, false>{});
    case 3: return star ? f(DimTag<3, true>{}) : f(DimTag<3, false>{});
    case 4: return star ? f(DimTag<4, true>{}) : f(DimTag<4, false>{});
    case 5: return star ? f(DimTag<5, true>{}) : f(DimTag<5, false>{});
    case 6: return star ? f(DimTag<6, true>{}) : f(DimTag<6, false>{});
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_mixed(int dim, bool vr, bool star, const MixedParams &p, int grid, int block, size_t smem,
                         cudaStream_t s)
{
    return by_dim(dim, star, [&](auto t) { return decltype(t)::L::mixed(vr, p, grid, block, smem, s); });
}

cudaError_t mixed_occupancy(int dim, bool vr, bool star, int block, size_t smem, int *blocks_per_sm)
{
    return by_dim(dim, star, [&](auto t) { return decltype(t)::L::occupancy(vr, block, smem, blocks_per_sm); });
}

cudaError_t launch_mixed_warp(int dim, bool vr, bool star, const MixedParams &p, int grid, int block, size_t smem,
                              cudaStream_t s)
{
    return by_dim(dim, star, [&](auto t) { return decltype(t)::L::mixed_warp(vr, p, grid, block, smem, s); });
}

cudaError_t mixed_warp_occupancy(int dim, bool vr, bool star, int block, size_t smem, int *blocks_per_sm)
{
    return by_dim(dim, star, [&](auto t) { return decltype(t)::L::occupancy_warp(vr, block, smem, blocks_per_sm); });
}

cudaError_t launch_shared(int dim, bool vr, bool star, const MixedParams &p, int grid, size_t smem, cudaStream_t s)
{
    return by_dim(dim, star, [&](auto t) { return decltype(t)::L::shared(vr, p, grid, smem, s); });
}

cudaError_t shared_occupancy(int dim, bool vr, bool star, size_t smem, int *blocks_per_sm)
{
    return by_dim(dim, star, [&](auto t) { return decltype(t)::L::occupancy_shared(vr, smem, blocks_per_sm); });
}

cudaError_t launch_finalize(const FinalizeParams &p, bool from_acc, cudaStream_t s)
{
    const int64_t n = p.n_pts * (p.dim + 1);
    if (n == 0) return cudaSuccess;
    const int grid = (int)((n + 255) / 256);
    if (from_acc) k_finalize_acc<<<grid, 256, 0, s>>>(p);
    else k_finalize<<<grid, 256, 0, s>>>(p);
    return cudaGetLastError();
}

cudaError_t launch_fp64_point(int dim, bool vr, bool star, const Fp64PointParams &p, cudaStream_t s)
{
    const int grid = (int)((p.n_walks + 255) / 256);
    if (grid == 0) return cudaSuccess;
    return by_dim(dim, star, [&](auto t) { return decltype(t)::L::fp64_point(vr, p, grid, s); });
}

cudaError_t launch_walk_values(int dim, bool vr, bool star, bool fp64, const WalkValuesParams &p, cudaStream_t s)
{
    if (p.n == 0) return cudaSuccess;
    return by_dim(dim, star, [&](auto t) { return decltype(t)::L::values(vr, fp64, p, s); });
}

}  // namespace woi
