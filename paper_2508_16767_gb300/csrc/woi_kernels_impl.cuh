// woi_kernels_impl.cuh -- Walk-on-Interfaces kernel templates for sm_103a
// (instantiated per dimension in woi_k<d>.cu).
//
//   k_walk_mixed      batched persistent kernel: FP32 walks, one walk per thread;
//                     warps take (point, walk-chunk) units of the instance their
//                     block serves from that instance's queue, accumulate
//                     compensated FP32 sums per lane and reduce them (TwoSum) to
//                     one partial per unit (deterministic order)
//   k_walk_mixed_warp the same for one instance (all blocks share one queue)
//   k_walk_shared     tiles of 32 points sharing their walks (Sec. 4.6)
//   k_finalize        per (instance, point, component): ordered sum of the unit
//                     partials, mean and standard error from the schedule-group
//                     means (Algorithm 1)
//   k_walk_fp64_point FP64 walks, one launch per evaluation point, FP64 atomics
//   k_walk_values     per-walk tallies (pathwise replay), FP32 or FP64
#pragma once

#include <cuda_runtime.h>

#include "woi_device.cuh"
#include "woi_kernels.h"

namespace woi {

// ---------------------------------------------------------------------------
// reductions
// ---------------------------------------------------------------------------
__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    return v;
}
__device__ __forceinline__ float warp_sum_all(float v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xFFFFFFFFu, v, o);
    return v;
}

// warp sum of (hi, lo) FP32 pairs with error-free additions (Knuth's TwoSum): the
// result in lane 0 keeps about twice the FP32 precision; no FP64 instruction
__device__ __forceinline__ void warp_sum_pair(float &hi, float &lo)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const float bh = __shfl_down_sync(0xFFFFFFFFu, hi, o), bl = __shfl_down_sync(0xFFFFFFFFu, lo, o);
        const float s = hi + bh, bb = s - hi;
        const float e = (hi - (s - bb)) + (bh - bb);
        hi = s;
        lo = lo + bl + e;
    }
}

// Neumaier (compensated) FP32 accumulation
__device__ __forceinline__ void kahan_add(float &s, float &c, float v)
{
    const float t = s + v;
    c += (fabsf(s) >= fabsf(v)) ? ((s - t) + v) : ((v - t) + s);
    s = t;
}

// ---------------------------------------------------------------------------
// one warp-level work unit: the walks [w_base, w_base + 32 L) of one point (lane l runs walks
// w_base + 32 j + l), summed per lane with compensation and reduced over the warp (TwoSum) into
// one partial row (sum of f, sum of squared schedule-group means) written by lane 0
// ---------------------------------------------------------------------------
template <int D, bool VR, bool STAR>
__device__ __forceinline__ void run_unit(const SGeomFor<float, D, STAR> &g, const DevGeom *geom,
                                         const float (*xc)[kMaxDim], Rng &rng, int64_t w_base, int64_t w_end, int L,
                                         int sched_group, int lane, double *row)
{
    float s1[D + 1], c1[D + 1], s2[D + 1];
#pragma unroll
    for (int c = 0; c <= D; ++c) s1[c] = c1[c] = s2[c] = 0.f;
    // the plain variant on spheres in d <= 3 with per-walk schedules advances rounds j and j + 1
    // together (two independent walks per lane overlap their dependency chains); in higher
    // dimensions, and with the larger code of stars, ellipsoids and meshes, the second walk's
    // state does not fit in the registers
    constexpr bool PAIR = !VR && !STAR && D <= 3;
    int j = 0;
    if (PAIR && sched_group == 1) {
        for (; j + 1 < L; j += 2) {
            const int64_t wa = w_base + (int64_t)j * 32 + lane, wb = wa + 32;
            float f2[2][D + 1];
            Rng r2[2] = {rng, rng};
            r2[0].w0 = (uint32_t)wa;
            r2[0].w1 = (uint32_t)((uint64_t)wa >> 32);
            r2[1].w0 = (uint32_t)wb;
            r2[1].w1 = (uint32_t)((uint64_t)wb >> 32);
            if (wa < w_end) walk_pair<float, D, STAR>(g, geom, xc, r2, f2);
#pragma unroll
            for (int q = 0; q < 2; ++q) {
                const bool valid = (q == 0 ? wa : wb) < w_end;
#pragma unroll
                for (int c = 0; c <= D; ++c) {
                    const float fv = valid ? f2[q][c] : 0.f;
                    kahan_add(s1[c], c1[c], fv);
                    s2[c] += fv * fv;
                }
            }
        }
    }
    for (; j < L; ++j) {
        const int64_t w = w_base + (int64_t)j * 32 + lane;
        float f[D + 1];
        const bool valid = w < w_end;
        if (valid) {
            rng.w0 = (uint32_t)w;
            rng.w1 = (uint32_t)((uint64_t)w >> 32);
            // a shared schedule: w_base is a multiple of 32 and a round is all valid or all past
            // the end, so lane 0 runs the first walk of the round's group; the general-surface
            // kernels take its word by a shuffle, the sphere kernels (whose workloads use
            // per-walk schedules, and whose code is timed to the instruction) draw it
            walk<float, D, VR, STAR, false, STAR>(g, geom, xc, rng, sched_group, (uint64_t)w / 32u, f);
        } else {
#pragma unroll
            for (int c = 0; c <= D; ++c) f[c] = 0.f;
        }
#pragma unroll
        for (int c = 0; c <= D; ++c) kahan_add(s1[c], c1[c], f[c]);
        if (sched_group == 1) {
#pragma unroll
            for (int c = 0; c <= D; ++c) s2[c] += f[c] * f[c];
        } else {
            // the 32 lanes share one schedule; a warp's round is all valid or all past the end
#pragma unroll
            for (int c = 0; c <= D; ++c) {
                const float gm = warp_sum_all(f[c]) * (1.0f / 32.0f);
                if (lane == 0 && valid) s2[c] += gm * gm;
            }
        }
    }
#pragma unroll
    for (int c = 0; c <= D; ++c) {
        float h1 = s1[c], l1 = c1[c], h2 = s2[c], l2 = 0.f;
        warp_sum_pair(h1, l1);
        warp_sum_pair(h2, l2);
        if (lane == 0) {
            row[c] = (double)h1 + (double)l1;
            row[D + 1 + c] = (double)h2 + (double)l2;
        }
    }
}

// ---------------------------------------------------------------------------
// batched walk kernel: warp-level work units (point, 32 x L walks) of many
// instances.  A block serves one instance at a time (its geometry staged in
// shared memory); its warps take units from that instance's own queue head
// until it is exhausted, then the block moves on.  Block b starts at instance
// b mod n and visits every instance once: an instance it leaves is exhausted
// for good, so one round covers all the work.
// ---------------------------------------------------------------------------
template <int D, bool VR, bool STAR>
__global__ void __launch_bounds__(256, mixed_min_blocks<D, STAR, VR>()) k_walk_mixed(MixedParams p)
{
    __shared__ SGeomFor<float, D, STAR> g;
    __shared__ int left_sh;
    extern __shared__ float xc_all[];   // [warps][max_surf][kMaxDim]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    float(*xc)[kMaxDim] = reinterpret_cast<float(*)[kMaxDim]>(xc_all + (size_t)warp * p.max_surf * kMaxDim);
    const int L = p.walks_per_lane;
    int k = blockIdx.x % p.n_inst;
    for (int visit = 0; visit < p.n_inst; ++visit, k = (k + 1 == p.n_inst) ? 0 : k + 1) {
        const InstDesc &id = p.inst[k];
        const unsigned long long units_k = (unsigned long long)(id.n_pts * id.chunks_per_point);
        if (tid == 0) left_sh = atomicAdd(p.queue + k, 0ull) < units_k;
        __syncthreads();
        const bool left = left_sh != 0;
        __syncthreads();
        if (!left) continue;
        load_geometry(g, id.geom);
        __syncthreads();
        Rng rng;
        rng.k1 = (uint32_t)(p.seed >> 32) ^ id.instance_id;
        const int64_t w_end = id.walk_begin + id.n_walks;
        for (;;) {
            unsigned long long u = 0;
            if (lane == 0) u = atomicAdd(p.queue + k, 1ull);
            u = __shfl_sync(0xFFFFFFFFu, u, 0);
            if (u >= units_k) break;
            const int64_t local = (int64_t)u;
            const int64_t point = local / id.chunks_per_point;
            const int64_t chunk = local - point * id.chunks_per_point;
            const double *x = id.points + point * D;
            for (int i = lane; i < g.n * D; i += 32) {
                const int sidx = i / D, c = i - sidx * D;
                xc[sidx][c] = (float)(x[c] - id.geom->center[sidx][c]);
            }
            __syncwarp();
            rng.k0 = (uint32_t)p.seed ^ (uint32_t)point;
            const int64_t w_base = id.walk_begin + chunk * 32LL * L;
            run_unit<D, VR, STAR>(g, id.geom, xc, rng, w_base, w_end, L, id.sched_group, lane,
                                  p.partials + (id.unit_begin + local) * (2 * (D + 1)));
            __syncwarp();   // the table is rewritten for the next unit
        }
        __syncthreads();    // every warp is done with this instance before its geometry is replaced
    }
}

// ---------------------------------------------------------------------------
// single-instance variant: warp-level work units (32 lanes x L walks of one
// point), each warp with its own x - c_s table, no block barrier per unit
// ---------------------------------------------------------------------------
template <int D, bool VR, bool STAR>
__global__ void __launch_bounds__(256, mixed_min_blocks<D, STAR, VR>()) k_walk_mixed_warp(MixedParams p)
{
    __shared__ SGeomFor<float, D, STAR> g;
    extern __shared__ float xc_all[];   // [warps][n][kMaxDim]
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const InstDesc &id = p.inst[0];
    load_geometry(g, id.geom);
    __syncthreads();
    float(*xc)[kMaxDim] = reinterpret_cast<float(*)[kMaxDim]>(xc_all + (size_t)warp * g.n * kMaxDim);
    const int L = p.walks_per_lane;
    const int64_t w_end = id.walk_begin + id.n_walks;
    Rng rng;
    rng.k1 = (uint32_t)(p.seed >> 32) ^ id.instance_id;
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(p.queue, 1ull);
        u = __shfl_sync(0xFFFFFFFFu, u, 0);
        if (u >= (unsigned long long)p.total_units) break;
        const int64_t unit = (int64_t)u;
        const int64_t point = unit / id.chunks_per_point;
        const int64_t chunk = unit - point * id.chunks_per_point;
        const double *x = id.points + point * D;
        for (int i = lane; i < g.n * D; i += 32) {
            const int sidx = i / D, k = i - sidx * D;
            xc[sidx][k] = (float)(x[k] - id.geom->center[sidx][k]);
        }
        __syncwarp();
        rng.k0 = (uint32_t)p.seed ^ (uint32_t)point;
        const int64_t w_base = id.walk_begin + chunk * 32LL * L;
        run_unit<D, VR, STAR>(g, id.geom, xc, rng, w_base, w_end, L, id.sched_group, lane,
                              p.partials + unit * (2 * (D + 1)));
        __syncwarp();   // the table is rewritten for the next unit
    }
}

// ---------------------------------------------------------------------------
// shared trajectories (Sec. 4.6): the 32 points of a tile share their walks.
// A warp unit is (tile, walk chunk): per round each lane runs one walk and
// records its states (surface, offset, coefficient) in shared memory, then each
// lane tallies its point against the 32 recorded walks (broadcast reads).
// ---------------------------------------------------------------------------
// record of one walk state for the tile: y = c_s + v as an unevaluated FP32 sum
// yhi + ylo (TwoSum, then c_lo), and the coefficient c. The vector part holds kRec<D>
// floats, 16-byte aligned, so that the 32 lanes read it with kRec<D> / 4 broadcast vector
// loads. In even d the 2d floats of yhi, ylo fill whole vectors and c goes to an array of
// its own after the vector parts (2d + 1 floats a record); in odd d c pads the last vector.
template <int D>
constexpr bool kRecSplit = D % 2 == 0;
template <int D>
constexpr int kRec = kRecSplit<D> ? 2 * D : ((2 * D + 1) + 3) / 4 * 4;
static_assert(shared_record_floats(2) == kRec<2> + 1 && shared_record_floats(3) == kRec<3> &&
                  shared_record_floats(4) == kRec<4> + 1 && shared_record_floats(5) == kRec<5> &&
                  shared_record_floats(6) == kRec<6> + 1,
              "host and kernel record sizes differ");

template <int D>
struct RecordSink {
    const SGeom<float> &g;
    float *rec;    // [chains][M+1][32 walks][kRec<D>]
    float *rec_c;  // [chains][M+1][32 walks] (even d)
    int M1, lane;
    __device__ __forceinline__ void operator()(int i, int k, const Chain<float, D> &ch, float c)
    {
        float *r = rec + ((size_t)(k * M1 + i) * 32 + lane) * kRec<D>;
        float out[kRec<D> + (kRecSplit<D> ? 1 : 0)];
#pragma unroll
        for (int q = 0; q < D; ++q) {
            const float a = g.c_hi[ch.s][q], b = ch.v[q];
            const float sum = a + b, bb = sum - a;
            out[q] = sum;
            out[D + q] = ((a - (sum - bb)) + (b - bb)) + g.c_lo[ch.s][q];
        }
        out[2 * D] = c;
#pragma unroll
        for (int q = 2 * D + 1; q < kRec<D>; ++q) out[q] = 0.f;
#pragma unroll
        for (int q = 0; q < kRec<D>; q += 4)
            *reinterpret_cast<float4 *>(r + q) = make_float4(out[q], out[q + 1], out[q + 2], out[q + 3]);
        if constexpr (kRecSplit<D>) rec_c[(size_t)(k * M1 + i) * 32 + lane] = c;
    }
};

template <int D, bool VR, bool STAR>
__global__ void __launch_bounds__(kSharedBlock) k_walk_shared(MixedParams p)
{
    __shared__ SGeomTile<float, D, STAR> g;
    extern __shared__ float4 rec_all4[];
    float *rec_all = reinterpret_cast<float *>(rec_all4);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const InstDesc &id = p.inst[0];
    load_geometry(g, id.geom);
    __syncthreads();
    constexpr int chains = VR ? 2 : 1;
    constexpr int R = kRec<D>;
    const int M1 = g.M + 1;
    const int n_rec = chains * M1;
    float *rec = rec_all + (size_t)warp * n_rec * 32 * (R + (kRecSplit<D> ? 1 : 0));
    float *rec_c = rec + (size_t)n_rec * 32 * R;   // (even d)
    RecordSink<D> sink{g, rec, rec_c, M1, lane};
    const int L = p.walks_per_lane;
    const int64_t w_end = id.walk_begin + id.n_walks;
    Rng rng;
    rng.k1 = (uint32_t)(p.seed >> 32) ^ id.instance_id;
    for (;;) {
        unsigned long long u = 0;
        if (lane == 0) u = atomicAdd(p.queue, 1ull);
        u = __shfl_sync(0xFFFFFFFFu, u, 0);
        if (u >= (unsigned long long)p.total_units) break;
        const int64_t unit = (int64_t)u;
        const int64_t tile = unit / id.chunks_per_point;
        const int64_t chunk = unit - tile * id.chunks_per_point;
        const int64_t point = tile * 32 + lane;
        const bool has_point = point < id.n_pts;
        float xhi[D], xlo[D];
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const double xv = has_point ? id.points[point * D + k] : 0.0;
            xhi[k] = (float)xv;
            xlo[k] = (float)(xv - (double)xhi[k]);
        }
        rng.k0 = (uint32_t)p.seed ^ (uint32_t)tile;
        const int64_t w_base = id.walk_begin + chunk * 32LL * L;
        float s1[D + 1], c1[D + 1], s2[D + 1];
#pragma unroll
        for (int c = 0; c <= D; ++c) s1[c] = c1[c] = s2[c] = 0.f;
        for (int j = 0; j < L; ++j) {
            const int64_t w0 = w_base + (int64_t)j * 32;
            if (w0 >= w_end) break;
            const int64_t w = w0 + lane;
            if (w < w_end) {
                rng.w0 = (uint32_t)w;
                rng.w1 = (uint32_t)((uint64_t)w >> 32);
                walk_steps<float, D, VR, STAR, STAR>(g, id.geom, rng, id.sched_group, (uint64_t)w / 32u, sink);
            }
            __syncwarp();
            const int n_valid = (int)min((int64_t)32, w_end - w0);
            float gs[D + 1];
#pragma unroll
            for (int c = 0; c <= D; ++c) gs[c] = 0.f;
            for (int ww = 0; ww < n_valid; ++ww) {
                float f[D + 1];
#pragma unroll
                for (int c = 0; c <= D; ++c) f[c] = 0.f;
                for (int e = 0; e < n_rec; ++e) {
                    const float *r = rec + ((size_t)e * 32 + ww) * R;
                    float y[R + (kRecSplit<D> ? 1 : 0)];
                    if constexpr (kRecSplit<D>) {   // the coefficient first: a zero skips the vector loads
                        y[2 * D] = rec_c[e * 32 + ww];
                        if (y[2 * D] == 0.f) continue;
                    }
#pragma unroll
                    for (int q = 0; q < R; q += 4) {
                        const float4 t = *reinterpret_cast<const float4 *>(r + q);
                        y[q] = t.x; y[q + 1] = t.y; y[q + 2] = t.z; y[q + 3] = t.w;
                    }
                    const float cc = y[2 * D];
                    if (cc == 0.f) continue;
                    float dx[D];
#pragma unroll
                    for (int q = 0; q < D; ++q) dx[q] = (xhi[q] - y[q]) + (xlo[q] - y[D + q]);
                    tally_dx<float, D>(dx, cc, f);
                }
#pragma unroll
                for (int c = 0; c <= D; ++c) {
                    kahan_add(s1[c], c1[c], f[c]);
                    if (id.sched_group == 1) s2[c] += f[c] * f[c];
                    else gs[c] += f[c];
                }
            }
            if (id.sched_group != 1) {
#pragma unroll
                for (int c = 0; c <= D; ++c) {
                    const float gm = gs[c] * (1.0f / 32.0f);
                    s2[c] += gm * gm;
                }
            }
            __syncwarp();
        }
        if (has_point) {
            double *row = p.partials + (unit * 32 + lane) * (2 * (D + 1));
#pragma unroll
            for (int c = 0; c <= D; ++c) {
                row[c] = (double)s1[c] + (double)c1[c];
                row[D + 1 + c] = (double)s2[c];
            }
        }
    }
}

// ---------------------------------------------------------------------------
// FP64 baseline: one launch per point, one walk per thread, FP64 atomics
// ---------------------------------------------------------------------------
template <int D, bool VR, bool STAR>
__global__ void __launch_bounds__(256) k_walk_fp64_point(Fp64PointParams p)
{
    __shared__ SGeomFor<double, D, STAR> g;
    __shared__ double xc[kMaxSurf][kMaxDim];
    __shared__ double red[8][2 * (D + 1)];
    load_geometry(g, p.geom);
    fill_xc<double>(xc, p.geom, p.geom->n, D, p.x);
    __syncthreads();
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int64_t w = p.walk_begin + (int64_t)blockIdx.x * blockDim.x + tid;
    const bool valid = w < p.walk_begin + p.n_walks;
    double f[D + 1];
    if (valid) {
        Rng rng;
        rng.k0 = (uint32_t)p.seed ^ p.point_id;
        rng.k1 = (uint32_t)(p.seed >> 32) ^ p.instance_id;
        rng.w0 = (uint32_t)w;
        rng.w1 = (uint32_t)((uint64_t)w >> 32);
        walk<double, D, VR, STAR, false, STAR>(g, p.geom, xc, rng, p.sched_group, (uint64_t)w / 32u, f);
    } else {
#pragma unroll
        for (int c = 0; c <= D; ++c) f[c] = 0.0;
    }
#pragma unroll
    for (int c = 0; c <= D; ++c) {
        const double v1 = warp_sum(f[c]);
        double v2;
        if (p.sched_group == 1) {
            v2 = warp_sum(f[c] * f[c]);
        } else {
            const double gm = v1 / 32.0;  // lane 0 holds the group sum
            v2 = (lane == 0 && valid) ? gm * gm : 0.0;
        }
        if (lane == 0) {
            red[warp][c] = v1;
            red[warp][D + 1 + c] = v2;
        }
    }
    __syncthreads();
    if (tid < 2 * (D + 1)) {
        double acc = 0.0;
        for (int wi = 0; wi < (int)(blockDim.x >> 5); ++wi) acc += red[wi][tid];
        atomicAdd(p.acc + tid, acc);
    }
}

// ---------------------------------------------------------------------------
// per-walk values (pathwise replay)
// ---------------------------------------------------------------------------
template <typename Real, int D, bool VR, bool STAR>
__global__ void __launch_bounds__(128) k_walk_values(WalkValuesParams p)
{
    __shared__ SGeomFor<Real, D, STAR> g;
    __shared__ Real xc[kMaxSurf][kMaxDim];
    load_geometry(g, p.geom);
    fill_xc<Real>(xc, p.geom, p.geom->n, D, p.x);
    __syncthreads();
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= p.n) return;
    const uint64_t w = p.walks[i];
    Rng rng;
    rng.k0 = (uint32_t)p.seed ^ p.point_id;
    rng.k1 = (uint32_t)(p.seed >> 32) ^ p.instance_id;
    rng.w0 = (uint32_t)w;
    rng.w1 = (uint32_t)(w >> 32);
    Real f[D + 1];
    walk<Real, D, VR, STAR, true>(g, p.geom, xc, rng, p.sched_group, w / 32u, f,
                                  p.trace ? p.trace + (size_t)i * (VR ? 2 : 1) * (g.M + 1) * (D + 2) : nullptr);
    p.f_u[i] = (double)f[0];
#pragma unroll
    for (int c = 0; c < D; ++c) p.f_grad[i * D + c] = (double)f[1 + c];
}

// launchers of one dimension / star flag (explicitly instantiated in woi_k<d>.cu)
template <int D, bool STAR>
cudaError_t DimLaunchers<D, STAR>::mixed(bool vr, const MixedParams &p, int grid, int block, size_t smem, cudaStream_t s)
{
    {
        if (vr) {
            k_walk_mixed<D, true, STAR><<<grid, block, smem, s>>>(p);
            return cudaGetLastError();
        }
    }
    k_walk_mixed<D, false, STAR><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}
template <int D, bool STAR>
cudaError_t DimLaunchers<D, STAR>::mixed_warp(bool vr, const MixedParams &p, int grid, int block, size_t smem,
                                             cudaStream_t s)
{
    {
        if (vr) {
            k_walk_mixed_warp<D, true, STAR><<<grid, block, smem, s>>>(p);
            return cudaGetLastError();
        }
    }
    k_walk_mixed_warp<D, false, STAR><<<grid, block, smem, s>>>(p);
    return cudaGetLastError();
}

template <int D, bool STAR>
cudaError_t DimLaunchers<D, STAR>::occupancy_warp(bool vr, int block, size_t smem, int *blocks_per_sm)
{
    {
        if (vr) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_walk_mixed_warp<D, true, STAR>, block, smem);
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_walk_mixed_warp<D, false, STAR>, block, smem);
}

// the static SGeom and the dynamic records together exceed the default 48 KB per
// block, so the dynamic limit is raised for every launch of the shared kernels
template <int D, bool STAR>
cudaError_t DimLaunchers<D, STAR>::shared(bool vr, const MixedParams &p, int grid, size_t smem, cudaStream_t s)
{
    {
        if (vr) {
            cudaError_t e = cudaFuncSetAttribute(k_walk_shared<D, true, STAR>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            k_walk_shared<D, true, STAR><<<grid, kSharedBlock, smem, s>>>(p);
            return cudaGetLastError();
        }
    }
    cudaError_t e = cudaFuncSetAttribute(k_walk_shared<D, false, STAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    k_walk_shared<D, false, STAR><<<grid, kSharedBlock, smem, s>>>(p);
    return cudaGetLastError();
}

template <int D, bool STAR>
cudaError_t DimLaunchers<D, STAR>::occupancy_shared(bool vr, size_t smem, int *blocks_per_sm)
{
    {
        if (vr) {
            cudaError_t e = cudaFuncSetAttribute(k_walk_shared<D, true, STAR>,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_walk_shared<D, true, STAR>, kSharedBlock, smem);
        }
    }
    cudaError_t e = cudaFuncSetAttribute(k_walk_shared<D, false, STAR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_walk_shared<D, false, STAR>, kSharedBlock, smem);
}

template <int D, bool STAR>
cudaError_t DimLaunchers<D, STAR>::occupancy(bool vr, int block, size_t smem, int *blocks_per_sm)
{
    {
        if (vr) return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_walk_mixed<D, true, STAR>, block, smem);
    }
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, k_walk_mixed<D, false, STAR>, block, smem);
}
template <int D, bool STAR>
cudaError_t DimLaunchers<D, STAR>::fp64_point(bool vr, const Fp64PointParams &p, int grid, cudaStream_t s)
    {
        {
            if (vr) {
                k_walk_fp64_point<D, true, STAR><<<grid, 256, 0, s>>>(p);
                return cudaGetLastError();
            }
        }
        k_walk_fp64_point<D, false, STAR><<<grid, 256, 0, s>>>(p);
        return cudaGetLastError();
    }
template <int D, bool STAR>
cudaError_t DimLaunchers<D, STAR>::values(bool vr, bool fp64, const WalkValuesParams &p, cudaStream_t s)
    {
        const int grid = (int)((p.n + 127) / 128);
        {
            if (vr) {
                if (fp64) k_walk_values<double, D, true, STAR><<<grid, 128, 0, s>>>(p);
                else k_walk_values<float, D, true, STAR><<<grid, 128, 0, s>>>(p);
                return cudaGetLastError();
            }
        }
        if (fp64) k_walk_values<double, D, false, STAR><<<grid, 128, 0, s>>>(p);
        else k_walk_values<float, D, false, STAR><<<grid, 128, 0, s>>>(p);
        return cudaGetLastError();
    }

}  // namespace woi
