// woi_device.cuh -- device side of the Walk-on-Interfaces walk (sm_103a).
//
// One walk per thread.  Everything here is templated on the arithmetic type
// Real (float for the mixed path, double for the FP64 path) and on the
// dimension D, so the same source is the FP32 walk and the FP64 baseline.
//
// The method (Ding & Stinchcombe, arXiv 2508.16767):
//   Sec. 3        alpha, beta, truncated Neumann series with w_i = 1 - delta_iM/2
//   Sec. 4.2      transition densities (Eqs. naive_woi_p0, naive_woi_p) and the
//                 Q / T factors (Eqs. naive_woi_Q, naive_woi_T)
//   Sec. 4.3      scheduled interfaces (Thm 4.2), Eq. woi_estimator, Algs. 1-2
//   Sec. 4.4      variance reduction (Alg. 3)
//   Sec. 4.5      gradient tally with grad_x Phi
// Readings: the alpha-sign product runs over m = 1..i (Thm 4.2); in the
// uniform ("otherwise") transition T is unchanged because Q already carries the
// signed K*(y_i, y_{i-1}) evaluated with the normal at y_i; "descendant" is a
// strict descendant at any depth; a line/ray with no admissible intersection
// ends the walk.
//
// Precision: a walk state is kept as (surface s, offset v = y - c_s) and
// surface centres as (hi, lo) pairs, so differences between points on nearby
// surfaces and x - y near a surface are formed without cancellation in FP32.
// Angles on curves are carried as (node j, small offset delta) with exact node
// cosines and sines, and arc-length targets are split in FP64 (two operations).
#pragma once

#include <type_traits>

#include <cstdint>

#include "woi_layout.h"

namespace woi {

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds, multipliers 0xD2511F53 and
// 0xCD9E8D57, Weyl key increments 0x9E3779B9 and 0xBB67AE85.
// ---------------------------------------------------------------------------
struct U4 {
    uint32_t x, y, z, w;
};

__device__ __forceinline__ U4 philox10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                                       uint32_t k1)
{
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
        const uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
        const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
        c0 = n0;
        c1 = lo1;
        c2 = n2;
        c3 = lo0;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    return {c0, c1, c2, c3};
}

// Random-number protocol: key = (seed_lo ^ point, seed_hi ^ instance);
// counter = (walk_lo, walk_hi, step, (chain << 4) | sub) for the walk's own
// words; on 2D instances of circles only, steps 2j and 2j + 1 share the call of
// step j (ChainWords).  A shared schedule (groups of 32 walks) takes, in step i,
// the schedule word of the group's first walk.
struct Rng {
    uint32_t k0, k1;
    uint32_t w0, w1;
    __device__ __forceinline__ U4 words(int step, int chain, int sub) const
    {
        return philox10(w0, w1, (uint32_t)step, (uint32_t)((chain << 4) | sub), k0, k1);
    }
    // the words of rejection attempt a >= 1 of a (step, chain) stream: (a << 9) in counter word 3
    __device__ __forceinline__ U4 words_at(int step, int chain, int attempt, int sub) const
    {
        return philox10(w0, w1, (uint32_t)step, ((uint32_t)attempt << 9) | (uint32_t)((chain << 4) | sub), k0, k1);
    }
};

// uniform on (0,1): ((w >> 9) + 0.5) / 2^23, exact in FP32 and FP64
template <typename Real>
__device__ __forceinline__ Real u01(uint32_t w)
{
    return ((Real)(w >> 9) + (Real)0.5) * (Real)(1.0 / 8388608.0);
}
// FP32: the same value without an int-to-float conversion: 1.m - (1 - 2^-24) = (2m + 1) / 2^24,
// exact (Sterbenz) since both operands lie in [1 - 2^-24, 2)
template <>
__device__ __forceinline__ float u01<float>(uint32_t w)
{
    return __uint_as_float(0x3F800000u | (w >> 9)) - 0.99999994039535522f;
}

template <typename Real> struct RealOps;
template <> struct RealOps<float> {
    // sin and cos of 2 pi u for a uniform u in (0, 1) (24-bit, exact in FP32): an exact
    // reduction to a quarter turn q and a remainder r = u - q/4 in [-1/8, 1/8], the Taylor
    // series of sin and cos at theta = 2 pi r (|theta| <= pi/4; the first omitted terms,
    // theta^11/11! and theta^12/12!, are below 2e-9), then the rotation by q quarter turns
    __device__ static __forceinline__ void sincos2pi(float u, float *s, float *c)
    {
        const float q = rintf(4.0f * u);
        const float r = fmaf(q, -0.25f, u);                    // exact
        const float t = r * 6.28318530717958648f;
        const float t2 = t * t;
        float ps = fmaf(t2, 1.0f / 362880.0f, -1.0f / 5040.0f);
        ps = fmaf(t2, ps, 1.0f / 120.0f);
        ps = fmaf(t2, ps, -1.0f / 6.0f);
        const float sn = fmaf(t * t2, ps, t);
        float pc = fmaf(t2, -1.0f / 3628800.0f, 1.0f / 40320.0f);
        pc = fmaf(t2, pc, -1.0f / 720.0f);
        pc = fmaf(t2, pc, 1.0f / 24.0f);
        pc = fmaf(t2, pc, -0.5f);
        const float cs = fmaf(t2, pc, 1.0f);
        const int k = (int)q & 3;
        const float a = (k & 1) ? cs : sn, b = (k & 1) ? sn : cs;
        *s = (k & 2) ? -a : a;
        *c = ((k + 1) & 2) ? -b : b;
    }
    // sin and cos of x radians: x / 2 pi rounded once (relative 6e-8, within the rounding of x
    // itself for |x| <= pi), then sincos2pi; no large-argument path
    __device__ static __forceinline__ void sincos_rad(float x, float *s, float *c)
    {
        sincos2pi(x * 0.159154943091895336f, s, c);
    }
    // sin and cos of a small angle: Taylor series to d^7 and d^8 for |d| <= 1/4 (the first
    // omitted terms, d^9/9! and d^10/10!, are below 4e-11 relative); larger d through sincos_rad
    __device__ static __forceinline__ void sincos_small(float d, float *s, float *c)
    {
        if (fabsf(d) <= 0.25f) {
            const float d2 = d * d;
            *s = fmaf(d * d2, fmaf(d2, fmaf(d2, -1.0f / 5040.0f, 1.0f / 120.0f), -1.0f / 6.0f), d);
            *c = fmaf(d2, fmaf(d2, fmaf(d2, fmaf(d2, 1.0f / 40320.0f, -1.0f / 720.0f), 1.0f / 24.0f), -0.5f), 1.0f);
        } else {
            sincos_rad(d, s, c);
        }
    }
    __device__ static __forceinline__ float sqrt_(float v) { return sqrtf(v); }
    // sqrt of a strictly positive argument through the reciprocal square root
    __device__ static __forceinline__ float sqrt_pos(float v) { return v * rsqrtf(v); }
    __device__ static __forceinline__ float div_(float a, float b) { return __fdividef(a, b); }
    __device__ static __forceinline__ float rsqrt_(float v) { return rsqrtf(v); }
    __device__ static __forceinline__ float log_(float v) { return logf(v); }
    __device__ static __forceinline__ float fast_log(float v) { return __logf(v); }
    __device__ static __forceinline__ float fabs_(float v) { return fabsf(v); }
    __device__ static __forceinline__ float rcp(float v) { return __fdividef(1.0f, v); }
    __device__ static __forceinline__ float atan2_(float y, float x) { return atan2f(y, x); }
};
template <> struct RealOps<double> {
    __device__ static __forceinline__ void sincos2pi(double u, double *s, double *c) { sincospi(2.0 * u, s, c); }
    __device__ static __forceinline__ double sqrt_(double v) { return sqrt(v); }
    __device__ static __forceinline__ double sqrt_pos(double v) { return sqrt(v); }
    __device__ static __forceinline__ double div_(double a, double b) { return a / b; }
    __device__ static __forceinline__ double rsqrt_(double v) { return 1.0 / sqrt(v); }
    __device__ static __forceinline__ double log_(double v) { return log(v); }
    __device__ static __forceinline__ double fast_log(double v) { return log(v); }
    __device__ static __forceinline__ void sincos_rad(double t, double *s, double *c) { sincos(t, s, c); }
    __device__ static __forceinline__ void sincos_small(double t, double *s, double *c) { sincos(t, s, c); }
    __device__ static __forceinline__ double fabs_(double v) { return fabs(v); }
    __device__ static __forceinline__ double rcp(double v) { return 1.0 / v; }
    __device__ static __forceinline__ double atan2_(double y, double x) { return atan2(y, x); }
};

// Newton step below which the iteration has converged (the last step is then taken:
// with quadratic convergence the result is accurate to the rounding noise of f)
template <typename Real> __host__ __device__ constexpr Real eps_tol() { return sizeof(Real) == 4 ? (Real)1e-6 : (Real)1e-10; }
// bracket width below which a bisection-safeguarded search stops
template <typename Real> __host__ __device__ constexpr Real bracket_tol() { return sizeof(Real) == 4 ? (Real)1e-9 : (Real)1e-17; }

// word k (k >= 1) of a (step, chain) stream: sub-call k / 4, lane k % 4
struct StepWords {
    U4 a, b;  // sub 0 and sub 1
    __device__ __forceinline__ uint32_t get(int k) const
    {
        const U4 &v = (k < 4) ? a : b;
        switch (k & 3) {
        case 0: return v.x;
        case 1: return v.y;
        case 2: return v.z;
        default: return v.w;
        }
    }
};

// isotropic unit vector from the words 1.. of a step (2D: one angle; 3D:
// z = 1 - 2u, azimuth 2 pi u'; d >= 4: Box-Muller pairs then normalise)
template <typename Real, int D>
__device__ __forceinline__ void direction(const StepWords &w, Real *z)
{
    using O = RealOps<Real>;
    if constexpr (D == 2) {
        O::sincos2pi(u01<Real>(w.a.y), &z[1], &z[0]);
    } else if constexpr (D == 3) {
        const Real u = u01<Real>(w.a.y);
        Real s, c;
        O::sincos2pi(u01<Real>(w.a.z), &s, &c);
        const Real rho = (Real)2 * O::sqrt_pos(u * ((Real)1 - u));  // sqrt(1 - (1-2u)^2); u in (0, 1)
        z[0] = rho * c;
        z[1] = rho * s;
        z[2] = (Real)1 - (Real)2 * u;
    } else {
        Real g[D + 1];
#pragma unroll
        for (int j = 0; 2 * j < D; ++j) {
            const Real ua = u01<Real>(w.get(1 + 2 * j));
            const Real ub = u01<Real>(w.get(2 + 2 * j));
            const Real rho = O::sqrt_pos((Real)-2 * O::log_(ua));   // ua < 1: log < 0
            Real s, c;
            O::sincos2pi(ub, &s, &c);
            g[2 * j] = rho * c;
            g[2 * j + 1] = rho * s;
        }
        Real n2 = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) n2 += g[k] * g[k];
        const Real inv = O::rsqrt_(n2);
#pragma unroll
        for (int k = 0; k < D; ++k) z[k] = g[k] * inv;
    }
}

template <int D> __host__ __device__ constexpr int choice_word() { return D == 2 ? 2 : (D == 3 ? 3 : (D == 4 ? 5 : 7)); }
template <int D> __host__ __device__ constexpr bool two_calls() { return D >= 4; }

// ---------------------------------------------------------------------------
// geometry staged in shared memory (one instance)
// ---------------------------------------------------------------------------
template <typename Real>
struct SGeom {
    int n, npad, M, star_idx, star_K;
    uint32_t sched_tm1[kMaxSurfPad];     // T_n - 1 (schedule thresholds), padded with 0xFFFFFFFF
    int sched_bucket[kSchedBuckets + 1]; // first n with T_n - 1 >= b 2^24
    Real c_hi[kMaxSurf][kMaxDim];        // centres as hi + lo
    Real c_lo[kMaxSurf][kMaxDim];
    Real radius[kMaxSurf];
    Real area[kMaxSurf];
    Real alpha_sign[kMaxSurf];
    Real beta_scale[kMaxSurf];
    int tin[kMaxSurf], tout[kMaxSurf];
    int type[kMaxSurf];
    Real coef[kMaxM + 1];                // N w_i ||alpha||_1^i
    Real node_cs[kNodes][2];             // cos, sin of t_j = 2 pi j / kNodes (circle arcs too)
};

// the star curve's tables (at most one star per instance)
template <typename Real>
struct SGeomS : SGeom<Real> {
    Real star_a[kMaxStar + 1], star_b[kMaxStar + 1];
    Real star_lmax;                      // bound on |gamma'|
    Real star_kpp;                       // bound on |gamma''|
    Real star_k3;                        // bound on |gamma'''|
    Real star_harm[kMaxStar + 2][4];     // gamma - centre = sum_m (X_m cos mt + Y_m sin mt, U_m cos mt + V_m sin mt)
    Real star_rmin, star_rmax;           // annulus that contains the star
    Real scan[kNodes][2];                // gamma(t_j) - centre
    Real scan_d[kNodes][2];              // gamma'(t_j)
    double panel_s[kNodes + 1];          // arc length at t_j
};

// the star view of a geometry that a 2D general-surface kernel staged as SGeomS
template <typename Real>
__device__ __forceinline__ const SGeomS<Real> &star_geom(const SGeom<Real> &g)
{
    return static_cast<const SGeomS<Real> &>(g);
}

// stages the common tables, and the star's with TABS (g is then an SGeomS)
template <typename Real, bool TABS>
__device__ void load_geometry_tables(SGeom<Real> &g, const DevGeom *src)
{
    const int tid = threadIdx.x, nt = blockDim.x;
    if (tid == 0) {
        g.n = src->n;
        g.npad = src->npad;
        g.M = src->M;
        g.star_idx = src->star_idx;
        g.star_K = src->star_K;
        if constexpr (TABS) {
            SGeomS<Real> &gs = static_cast<SGeomS<Real> &>(g);
            gs.star_lmax = (Real)src->star_lmax;
            gs.star_kpp = (Real)src->star_kpp;
            gs.star_k3 = (Real)src->star_k3;
            gs.star_rmin = (Real)src->star_rmin;
            gs.star_rmax = (Real)src->star_rmax;
        }
    }
    for (int i = tid; i < kMaxSurfPad; i += nt) g.sched_tm1[i] = src->sched_tm1[i];
    for (int i = tid; i <= kSchedBuckets; i += nt) g.sched_bucket[i] = src->sched_bucket[i];
    for (int i = tid; i < src->n; i += nt) {
        for (int k = 0; k < kMaxDim; ++k) {
            const double c = src->center[i][k];
            const Real hi = (Real)c;
            g.c_hi[i][k] = hi;
            g.c_lo[i][k] = (Real)(c - (double)hi);
        }
        g.radius[i] = (Real)src->radius[i];
        g.area[i] = (Real)src->area[i];
        g.alpha_sign[i] = (Real)src->alpha_sign[i];
        g.beta_scale[i] = (Real)src->beta_scale[i];
        g.tin[i] = src->tin[i];
        g.tout[i] = src->tout[i];
        g.type[i] = src->type[i];
    }
    for (int i = tid; i <= kMaxM; i += nt) g.coef[i] = (Real)src->coef[i];
    for (int j = tid; j < kNodes; j += nt) {
        g.node_cs[j][0] = (Real)src->node_cs[j][0];
        g.node_cs[j][1] = (Real)src->node_cs[j][1];
    }
    if constexpr (TABS) {
        SGeomS<Real> &gs = static_cast<SGeomS<Real> &>(g);
        if (src->star_idx >= 0) {
            for (int k = tid; k <= kMaxStar; k += nt) {
                gs.star_a[k] = (Real)src->star_a[k];
                gs.star_b[k] = (Real)src->star_b[k];
            }
            for (int j = tid; j < kNodes; j += nt) {
                gs.scan[j][0] = (Real)src->star_scan[j][0];
                gs.scan[j][1] = (Real)src->star_scan[j][1];
                gs.scan_d[j][0] = (Real)src->star_scan_d[j][0];
                gs.scan_d[j][1] = (Real)src->star_scan_d[j][1];
            }
            for (int j = tid; j <= kNodes; j += nt) gs.panel_s[j] = src->star_panel_s[j];
            for (int i = tid; i < (kMaxStar + 2) * 4; i += nt)
                gs.star_harm[i / 4][i % 4] = (Real)src->star_harm[i / 4][i % 4];
        }
    }
}

template <typename Real>
__device__ void load_geometry(SGeom<Real> &g, const DevGeom *src)
{
    load_geometry_tables<Real, false>(g, src);
}

template <typename Real>
__device__ void load_geometry(SGeomS<Real> &g, const DevGeom *src)
{
    load_geometry_tables<Real, true>(g, src);
}

// ellipsoids of an instance (d >= 3), staged only by kernels compiled for them
template <typename Real>
struct SEll {
    int slot[kMaxSurf];                  // slot of surface i, -1 if not an ellipsoid
    Real A[kMaxEll][kMaxDim][kMaxDim];   // (y - c)^T A (y - c) = 1
    Real map[kMaxEll][kMaxDim][kMaxDim]; // A^{-1/2}: unit sphere -> surface, area ratio sqrt(u^T A u)
    Real jmax[kMaxEll];                  // sqrt(max eigenvalue of A)
};

template <typename Real>
struct SGeomE : SGeomS<Real> {
    SEll<Real> ell;
};

// the staged geometry of a per-point kernel: every table, with the ellipsoids' when it serves
// general surfaces in d >= 3 (STAR is the kernels' flag for "not only spheres"). The sphere
// kernels run at the occupancy their registers allow, so the unused star tables cost them
// nothing; staging only the common tables there measured 1 % slower (its code differs).
template <typename Real, int D, bool STAR>
using SGeomFor = typename std::conditional<(STAR && D >= 3), SGeomE<Real>, SGeomS<Real>>::type;

// the staged geometry of a shared-trajectory kernel, whose occupancy is bounded by shared
// memory: spheres stage only the common tables
template <typename Real, int D, bool STAR>
using SGeomTile = typename std::conditional<STAR, SGeomFor<Real, D, STAR>, SGeom<Real>>::type;

template <typename Real>
__device__ void load_geometry(SGeomE<Real> &g, const DevGeom *src)
{
    load_geometry(static_cast<SGeomS<Real> &>(g), src);
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < kMaxSurf; i += nt) g.ell.slot[i] = i < src->n ? src->ell_slot[i] : -1;
    for (int i = tid; i < src->n_ell * kMaxDim * kMaxDim; i += nt) {
        const int e = i / (kMaxDim * kMaxDim), r = (i / kMaxDim) % kMaxDim, c = i % kMaxDim;
        g.ell.A[e][r][c] = (Real)src->ell_A[e][r][c];
        g.ell.map[e][r][c] = (Real)src->ell_map[e][r][c];
    }
    for (int i = tid; i < src->n_ell; i += nt) g.ell.jmax[i] = (Real)src->ell_jmax[i];
}

// H_i from a 32-bit word: i = 0 uniform over the N surfaces, i >= 1 the first n
// with w <= T_n - 1: a scan that starts at the first threshold of the word's top-8-bit
// bucket (no threshold before it can be the answer; T_N - 1 = 2^32 - 1 ends the scan)
template <typename Real>
__device__ __forceinline__ int schedule(const SGeom<Real> &g, int i, uint32_t w)
{
    if (i == 0) return (int)(((uint64_t)w * (uint64_t)g.n) >> 32);
    int n = g.sched_bucket[w >> 24];
#pragma unroll 1
    while (g.sched_tm1[n] < w) ++n;
    return n;
}

// 0: same surface, 1: prev is a strict descendant of cur, 2: otherwise
template <typename Real>
__device__ __forceinline__ int relation(const SGeom<Real> &g, int prev, int cur)
{
    if (prev == cur) return 0;
    return (g.tin[cur] < g.tin[prev] && g.tin[prev] < g.tout[cur]) ? 1 : 2;
}

// c_a - c_b without cancellation
template <typename Real, int D>
__device__ __forceinline__ void center_diff(const SGeom<Real> &g, int a, int b, Real *out)
{
#pragma unroll
    for (int k = 0; k < D; ++k) out[k] = (g.c_hi[a][k] - g.c_hi[b][k]) + (g.c_lo[a][k] - g.c_lo[b][k]);
}

// ---------------------------------------------------------------------------
// star curve about its centre: r(t) = R (1 + sum a_k cos kt + b_k sin kt).
// An angle is (node j, offset delta): t = 2 pi j / kNodes + delta.
// ---------------------------------------------------------------------------
template <typename Real>
__device__ __forceinline__ void angle_cs(const SGeom<Real> &g, int j, Real delta, Real *ct, Real *st)
{
    Real sd, cd;
    RealOps<Real>::sincos_small(delta, &sd, &cd);
    const Real cj = g.node_cs[j][0], sj = g.node_cs[j][1];
    *ct = cj * cd - sj * sd;
    *st = sj * cd + cj * sd;
}

template <typename Real>
__device__ __forceinline__ void star_eval(const SGeomS<Real> &g, Real ct, Real st, Real *r, Real *dr)
{
    Real ck = ct, sk = st, s = 1, ds = 0;
#pragma unroll 1
    for (int k = 1; k <= g.star_K; ++k) {
        const Real a = g.star_a[k], b = g.star_b[k];
        s += a * ck + b * sk;
        ds += (Real)k * (b * ck - a * sk);
        const Real cn = ck * ct - sk * st;  // cos((k+1)t), sin((k+1)t)
        sk = sk * ct + ck * st;
        ck = cn;
    }
    const Real R = g.radius[g.star_idx];
    *r = R * s;
    *dr = R * ds;
}

// local point r (cos t, sin t), outward unit normal and |gamma'| at the angle (ct, st)
template <typename Real>
__device__ __forceinline__ Real star_local(const SGeomS<Real> &g, Real ct, Real st, Real *v, Real *n)
{
    Real r, dr;
    star_eval(g, ct, st, &r, &dr);
    v[0] = r * ct;
    v[1] = r * st;
    const Real tx = dr * ct - r * st, ty = dr * st + r * ct;
    const Real sp = RealOps<Real>::sqrt_(tx * tx + ty * ty);
    if (n) {
        n[0] = ty / sp;
        n[1] = -tx / sp;
    }
    return sp;
}

template <typename Real>
__device__ __forceinline__ Real star_speed_at(const SGeomS<Real> &g, int j, Real delta)
{
    Real ct, st, r, dr;
    angle_cs(g, j, delta, &ct, &st);
    star_eval(g, ct, st, &r, &dr);
    return RealOps<Real>::sqrt_(r * r + dr * dr);
}

// Gauss-Legendre 8-point rule on [-1, 1] (positive half)
__device__ __forceinline__ double gl8_x(int q)
{
    const double x[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    return x[q];
}
__device__ __forceinline__ double gl8_w(int q)
{
    const double w[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    return w[q];
}

// Gauss-Legendre 4-point rule on [-1, 1] (positive half)
__device__ __forceinline__ float gl4_x(int q) { return q == 0 ? 0.33998104358485626f : 0.86113631159405258f; }
__device__ __forceinline__ float gl4_w(int q) { return q == 0 ? 0.65214515486254614f : 0.34785484513745386f; }

// arc length from node j to node j + delta (|delta| <= 2 pi / kNodes): Gauss-Legendre with 8
// points in FP64 and 4 in FP32, whose error on the panel, delta^9 (4!)^4 / (9 (8!)^3) times
// max |speed^(8)| (at most 16^8 times the curve's size for degree <= 16), is below 1e-10 of
// the panel's length, far below the FP32 rounding
template <typename Real>
__device__ Real star_local_arclen(const SGeomS<Real> &g, int j, Real delta)
{
    const Real half = (Real)0.5 * delta;
    Real s = 0;
    if constexpr (sizeof(Real) == 4) {
#pragma unroll 1
        for (int q = 0; q < 4; ++q) {   // nodes half -+ x_0 half, half -+ x_1 half
            const Real xq = gl4_x(q >> 1) * half;
            s += gl4_w(q >> 1) * star_speed_at(g, j, (q & 1) ? half + xq : half - xq);
        }
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const Real xq = (Real)gl8_x(q) * half;
            s += (Real)gl8_w(q) * (star_speed_at(g, j, half - xq) + star_speed_at(g, j, half + xq));
        }
    }
    return half * s;
}

// (node, offset) of the point at arc length s_abs (FP64 split of the target)
template <typename Real>
__device__ void star_at_arclen(const SGeomS<Real> &g, double s_abs, int *jo, Real *delta_o)
{
    int lo = 0, hi = kNodes;
    while (hi - lo > 1) {
        const int m = (lo + hi) >> 1;
        if (g.panel_s[m] <= s_abs) lo = m; else hi = m;
    }
    const Real H = (Real)(2.0 * 3.14159265358979323846 / kNodes);
    const Real ds = (Real)(s_abs - g.panel_s[lo]);
    Real d_lo = 0, d_hi = H;
    Real delta = ds / star_speed_at(g, lo, (Real)0);
    if (!(delta > d_lo && delta < d_hi)) delta = (Real)0.5 * H;
    const int iters = sizeof(Real) == 4 ? 12 : 30;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
        const Real f = star_local_arclen(g, lo, delta) - ds;
        if (f == (Real)0) break;
        if (f > 0) d_hi = delta; else d_lo = delta;
        const Real step = f / star_speed_at(g, lo, delta);
        if (RealOps<Real>::fabs_(step) <= eps_tol<Real>()) {   // converged: take the last Newton step
            delta -= step;
            break;
        }
        Real dn = delta - step;
        if (!(dn > d_lo && dn < d_hi)) dn = (Real)0.5 * (d_lo + d_hi);
        delta = dn;
    }
    *jo = lo;
    *delta_o = delta;
}

// f(delta) = (gamma_loc(t_j + delta) - yc) x z and its derivative
template <typename Real>
__device__ __forceinline__ void star_line_f(const SGeomS<Real> &g, int j, Real delta, const Real *yc, const Real *z,
                                            Real *f, Real *df)
{
    Real ct, st, r, dr;
    angle_cs(g, j, delta, &ct, &st);
    star_eval(g, ct, st, &r, &dr);
    const Real px = r * ct - yc[0], py = r * st - yc[1];
    *f = px * z[1] - py * z[0];
    const Real tx = dr * ct - r * st, ty = dr * st + r * ct;
    *df = tx * z[1] - ty * z[0];
}

// The line through the state y = gamma(s) on the star, in direction z: its other intersections
// are the roots of g(t) = [(gamma(t) - gamma(s)) / (t - s)] x z, the divided difference of the
// curve crossed with z (g(s) = gamma'(s) x z; no root at s itself).  With gamma a trigonometric
// polynomial of degree K + 1,
//   (cos mt - cos ms) / (t - s) = -m sin(m c) S(m h),  (sin mt - sin ms) / (t - s) = m cos(m c) S(m h),
// c = (t + s) / 2, h = (t - s) / 2, S(x) = sin(x) / x, so every term is formed to relative
// accuracy: no cancellation between gamma(t) and a rounded gamma(s) however close t is to s (a
// near-tangent line).  t = t_j + delta, s = t_js + ds.  Returns g and g' in *gv, *gd, and in
// *dz the divided difference dotted with z, so that t - s times it is the line parameter.
template <typename Real>
__device__ void star_dd(const SGeomS<Real> &g, int j, Real delta, int js, Real ds, const Real *z, Real *gv, Real *gd,
                        Real *dz)
{
    using O = RealOps<Real>;
    const Real H = (Real)(2.0 * 3.14159265358979323846 / kNodes);
    int dj = j - js;
    if (dj > kNodes / 2) dj -= kNodes;
    if (dj < -kNodes / 2) dj += kNodes;
    const Real h = (Real)0.5 * ((Real)dj * H + (delta - ds));
    Real cc, sc;                                             // c = t_j + (delta + ds - dj H) / 2
    angle_cs(g, j, (Real)0.5 * (delta + ds - (Real)dj * H), &cc, &sc);
    Real sh, ch;
    O::sincos_rad(h, &sh, &ch);
    Real cmc = cc, smc = sc, cmh = ch, smh = sh;             // cos / sin of m c and m h, m = 1
    Real Dx = 0, Dy = 0, dDx = 0, dDy = 0;
#pragma unroll 1
    for (int m = 1; m <= g.star_K + 1; ++m) {
        const Real x = (Real)m * h, x2 = x * x;
        Real S, Sp;                                          // S(x) and S'(x)
        if (O::fabs_(x) < (Real)0.1) {
            S = (Real)1 - x2 * ((Real)(1.0 / 6.0) - x2 * ((Real)(1.0 / 120.0) - x2 * (Real)(1.0 / 5040.0)));
            Sp = -x * ((Real)(1.0 / 3.0) - x2 * ((Real)(1.0 / 30.0) - x2 * (Real)(1.0 / 840.0)));
        } else {
            S = smh / x;
            Sp = (cmh - S) / x;
        }
        const Real *c = g.star_harm[m];
        const Real Fx = -c[0] * smc + c[1] * cmc, Fxp = -c[0] * cmc - c[1] * smc;
        const Real Fy = -c[2] * smc + c[3] * cmc, Fyp = -c[2] * cmc - c[3] * smc;
        const Real mh = (Real)0.5 * (Real)m;
        Dx += (Real)m * S * Fx;
        Dy += (Real)m * S * Fy;
        dDx += (Real)m * mh * (Sp * Fx + S * Fxp);
        dDy += (Real)m * mh * (Sp * Fy + S * Fyp);
        const Real cn = cmc * cc - smc * sc;                 // m + 1
        smc = smc * cc + cmc * sc;
        cmc = cn;
        const Real hn = cmh * ch - smh * sh;
        smh = smh * ch + cmh * sh;
        cmh = hn;
    }
    *gv = Dx * z[1] - Dy * z[0];
    *gd = dDx * z[1] - dDy * z[0];
    if (dz) *dz = Dx * z[0] + Dy * z[1];
}

// the function whose roots in scan interval j are the crossings: f(delta) = (gamma - yc) x z
// (a ray, or a line away from its start), or the divided difference g of the line through the
// state (js, ds) (DD = true); a compile-time choice, so that each search is compiled with
// its own evaluator only
template <typename Real, bool DD>
struct StarLineEval {
    const SGeomS<Real> &g;
    const Real *yc, *z;
    int j;
    int js;
    Real ds;
    __device__ __forceinline__ void operator()(Real delta, Real *v, Real *dv) const
    {
        if constexpr (DD) star_dd(g, j, delta, js, ds, z, v, dv, (Real *)nullptr);
        else star_line_f(g, j, delta, yc, z, v, dv);
    }
};

// root in (a, b) given sign(v(a)) (safeguarded Newton in delta)
template <typename Real, typename Ev>
__device__ Real star_refine(const Ev &ev, Real a, Real b, Real fa, Real t0 = (Real)-1)
{
    Real t = (t0 > a && t0 < b) ? t0 : (Real)0.5 * (a + b);
    const int iters = sizeof(Real) == 4 ? 40 : 90;
#pragma unroll 1
    for (int it = 0; it < iters; ++it) {
        Real f, df;
        ev(t, &f, &df);
        if (f == (Real)0) break;
        if ((f < 0) == (fa < 0)) a = t; else b = t;
        const Real step = f / df;
        if (RealOps<Real>::fabs_(step) <= eps_tol<Real>()) {   // converged: take the last Newton step
            t -= step;
            break;
        }
        Real tn = t - step;
        if (!(tn > a && tn < b)) tn = (Real)0.5 * (a + b);
        t = tn;
        if (b - a <= bracket_tol<Real>()) break;
    }
    return t;
}

// rounding level of f = (gamma - y) x z and of f' = gamma' x z in the kernel's precision
template <typename Real>
__device__ __forceinline__ Real star_f_noise(const SGeomS<Real> &g)
{
    return (sizeof(Real) == 4 ? (Real)2e-6 : (Real)1e-12) * g.star_rmax;
}
// |f| below which a computed value's sign is not trusted (a few units of the rounding of gamma)
template <typename Real>
__device__ __forceinline__ Real star_dip_noise(const SGeomS<Real> &g)
{
    return (sizeof(Real) == 4 ? (Real)1e-6 : (Real)1e-14) * g.star_rmax;
}
template <typename Real>
__device__ __forceinline__ Real star_df_noise(const SGeomS<Real> &g)
{
    return (sizeof(Real) == 4 ? (Real)2e-6 : (Real)1e-12) * g.star_lmax;
}

// f = (gamma - y) x z has |f''| <= |gamma''| <= K, so on a scan interval [0, H] f stays
// above the chord minus K H^2 / 8: with f(0), f(H) of one sign and both beyond that (plus
// the rounding of f), the interval holds no root; only the others need a search for a pair
template <typename Real>
__device__ __forceinline__ Real star_guard(const SGeomS<Real> &g)
{
    const Real H = (Real)(2.0 * 3.14159265358979323846 / kNodes);
    return g.star_kpp * H * H * (Real)0.125 + star_f_noise(g);
}

// The roots of f (the evaluator's function: (gamma - y) x z, or the divided difference g) in the
// scan interval [t_j, t_j+1] (j in [0, kNodes)), appended to cand in scan order (at most
// kIntervalRoots), by depth-first subdivision.  f'' is bounded by K (|gamma''| for f,
// |gamma'''| / 3 for g), so a piece of width w, with f and f' known at its ends,
//   - holds exactly one root if its end values differ in sign and f' has one sign at both
//     ends with min |f'| > K w (f' cannot change sign inside: f is monotone); it is refined;
//   - holds none if its end values share a sign and either min |f| > K w^2 / 8 (f stays above
//     its chord minus that) or f is monotone;
//   - is split at its midpoint otherwise; a midpoint of the other sign between ends of one sign
//     leaves a sign change in each half, unless |f| there is within the rounding of f (then
//     the piece is a tangency and holds no root).
// Any number of extrema in the interval is handled (a near-tangent line close to an inflection
// of the curve puts three roots in one interval, or two with two extrema of f).  Pieces narrower
// than pair_min_width (a tangency within the rounding of f) count one root for a sign change
// and none otherwise.  fa, fb and da, db are f and f' at the interval's ends; nf, nd and ndip
// the rounding levels of f and f' and the |f| below which a sign is not trusted.
// depth-first stack: one pending piece per level; pieces stop at pair_min_width, so
// log2(H / pair_min_width) + 1 levels suffice (13 + 1 in FP32, 35 + 1 in FP64)
template <typename Real> __host__ __device__ constexpr int pair_stack() { return sizeof(Real) == 4 ? 16 : 40; }
constexpr int kIntervalRoots = 4;
template <typename Real> __host__ __device__ constexpr Real pair_min_width() { return sizeof(Real) == 4 ? (Real)4e-6 : (Real)1e-12; }

// The piece under test is held in registers; the stack holds the right halves still pending
// (one per level), so a piece that needs no split touches no local memory.
template <typename Real, typename Ev>
__device__ int star_interval_roots(const Ev &ev, Real fa, Real fb, Real da, Real db, Real K,
                                   Real nf, Real nd, Real ndip, Real *cand)
{
    using O = RealOps<Real>;
    constexpr int kPairStack = pair_stack<Real>();
    Real lo_[kPairStack], hi_[kPairStack], flo_[kPairStack], fhi_[kPairStack], dlo_[kPairStack], dhi_[kPairStack];
    Real lo = 0, hi = (Real)(2.0 * 3.14159265358979323846 / kNodes), flo = fa, fhi = fb, dlo = da, dhi = db;
    int sp = 0, nc = 0;
    for (;;) {
        const Real w = hi - lo;
        const Real dmin = O::fabs_(dlo) < O::fabs_(dhi) ? O::fabs_(dlo) : O::fabs_(dhi);
        const bool mono = (dlo < 0) == (dhi < 0) && dmin > K * w + nd;
        const bool last = w <= pair_min_width<Real>() || sp + 1 > kPairStack;
        bool split = false;
        if ((flo < 0) == (fhi < 0)) {
            const Real fmin_ = O::fabs_(flo) < O::fabs_(fhi) ? O::fabs_(flo) : O::fabs_(fhi);
            split = !(mono || fmin_ > K * w * w * (Real)0.125 + nf || last);
        } else if (mono || last) {
            cand[nc++] = star_refine(ev, lo, hi, flo, lo + w * flo / (flo - fhi));   // secant start
        } else {
            split = true;
        }
        if (split) {
            const Real m = (Real)0.5 * (lo + hi);
            Real fm, dm;
            ev(m, &fm, &dm);
            // a dip through zero between ends of one sign brackets roots in both halves, unless
            // the dip is within the rounding of f (a tangency: no root)
            if (!((flo < 0) == (fhi < 0) && (fm < 0) != (flo < 0) && O::fabs_(fm) <= ndip)) {
                // the right half waits; the left one is searched first (scan order)
                lo_[sp] = m; hi_[sp] = hi; flo_[sp] = fm; fhi_[sp] = fhi; dlo_[sp] = dm; dhi_[sp] = dhi;
                ++sp;
                hi = m;
                fhi = fm;
                dhi = dm;
                continue;
            }
        }
        if (sp == 0 || nc >= kIntervalRoots) break;
        --sp;
        lo = lo_[sp]; hi = hi_[sp]; flo = flo_[sp]; fhi = fhi_[sp]; dlo = dlo_[sp]; dhi = dhi_[sp];
    }
    return nc;
}

// the scan intervals of the nodes whose angles lie between the polar angles of the points
// yc + sa z and yc + sb z (the angle is monotone along a line that misses the centre; it
// increases when e = yc x z > 0), padded by one node on each side: the cyclic node range
// [j0, j0 + count)
template <typename Real>
__device__ __forceinline__ void star_window(const Real *yc, const Real *z, Real e, Real sa, Real sb, int *j0,
                                            int *count)
{
    const Real H = (Real)(2.0 * 3.14159265358979323846 / kNodes), TWO_PI = (Real)(2.0 * 3.14159265358979323846);
    Real pa = RealOps<Real>::atan2_(yc[1] + sa * z[1], yc[0] + sa * z[0]);
    Real pb = RealOps<Real>::atan2_(yc[1] + sb * z[1], yc[0] + sb * z[0]);
    if (e < 0) {  // sweep from pb to pa instead
        const Real t = pa;
        pa = pb;
        pb = t;
    }
    if (pa < 0) pa += TWO_PI;
    if (pb < 0) pb += TWO_PI;
    Real span = pb - pa;
    if (span < 0) span += TWO_PI;
    *j0 = ((int)(pa / H) - 1) & (kNodes - 1);   // kNodes is a power of two
    const int c = (int)(span / H) + 3;
    *count = c < kNodes ? c : kNodes;
}

// Intersections of the line (ray = false) or ray (ray = true) yc + s z (yc
// relative to the star centre) with the star.  A root is a point of the curve on
// the line, so it lies where the line is inside the annulus rmin <= |p| <= rmax:
// at most two windows of polar angle (for a ray, their parts with s > 0; a window
// cut at s = 0 holds yc, so |yc| >= rmin > 0 and its polar angle is defined),
// scanned node by node (roots as in
// star_interval_roots, of f = (gamma - yc) x z).  For a line, whose start is the
// state itself on the curve at angle (sj, sd), the three scan intervals around that
// angle hold only the start unless the line is close to tangent there; then they are
// searched for the roots of the divided difference g of star_dd instead of f: g has no
// root at the start, and a crossing close to it is found to the accuracy of g's terms,
// not of f's cancelling difference.  Returns q;
// tt[] the line parameters, jj[] / dd[] the roots as (node, offset).
template <typename Real>
__device__ int star_intersections(const SGeomS<Real> &g, const Real *yc, const Real *z, bool ray, int sj, Real sd,
                                  Real *tt, int *jj, Real *dd)
{
    const Real e = yc[0] * z[1] - yc[1] * z[0];
    const Real H = (Real)(2.0 * 3.14159265358979323846 / kNodes);
    const Real tiny = sizeof(Real) == 4 ? (Real)1e-6 : (Real)1e-9;
    const Real ae = RealOps<Real>::fabs_(e);
    if (ae >= g.star_rmax) return 0;
    // the windows as at most two cyclic node ranges [s0, s0 + c0) and [s1, s1 + c1), merged where
    // they overlap or touch, so that every interval is scanned once
    int s0 = 0, c0 = 0, s1 = 0, c1 = 0, nr = 0;
    {
        const Real sf = -(yc[0] * z[0] + yc[1] * z[1]);          // foot of the perpendicular from the centre
        const Real outer = RealOps<Real>::sqrt_(g.star_rmax * g.star_rmax - e * e);
        const Real in2 = g.star_rmin * g.star_rmin - e * e;
        const Real inner = in2 > (Real)0 ? RealOps<Real>::sqrt_(in2) : (Real)0;
        Real a0 = sf - outer, a1 = sf + inner;
        const Real b0 = sf - inner, b1 = sf + outer;
        if (ray) {   // only s > 0 is on the ray: the windows are cut at the start
            a0 = a0 > (Real)0 ? a0 : (Real)0;
            a1 = a1 > (Real)0 ? a1 : (Real)0;
        }
#pragma unroll 1
        for (int k = 0; k < 2; ++k) {   // one copy of the window code
            const Real sa = k == 0 ? a0 : a1, sb = k == 0 ? b0 : b1;
            if (ray && !(sb > (Real)0)) continue;
            int jw, cw;
            star_window(yc, z, e, sa, sb, &jw, &cw);
            if (nr == 0) {
                s0 = jw;
                c0 = cw;
            } else {
                s1 = jw;
                c1 = cw;
            }
            ++nr;
        }
        if (nr == 2) {
            const int d01 = (s1 - s0) & (kNodes - 1), d10 = (s0 - s1) & (kNodes - 1);
            if (d01 <= c0) {            // the second starts inside the first or where it ends
                const int u = d01 + c1 > c0 ? d01 + c1 : c0;
                c0 = u < kNodes ? u : kNodes;
                nr = 1;
            } else if (d10 <= c1) {     // the first starts inside the second or where it ends
                const int u = d10 + c0 > c1 ? d10 + c0 : c1;
                s0 = s1;
                c0 = u < kNodes ? u : kNodes;
                nr = 1;
            }
        }
    }
    int q = 0;
    const Real unit = sizeof(Real) == 4 ? (Real)1e-6 : (Real)1e-14;    // sign trust, relative
    bool near_start = false;
    if (!ray) {
        // the intervals sj - 1, sj, sj + 1 around the start hold no crossing but the start itself
        // unless the line is close to tangent there: |g'| <= |gamma''| / 2 = K / 2, so g keeps the
        // sign of g(s) = gamma'(s) x z within 2 H of s when |g(s)| > K H (plus rounding); the
        // scan of f skips them
        Real ct, st, r, dr;
        angle_cs(g, sj, sd, &ct, &st);
        star_eval(g, ct, st, &r, &dr);
        const Real gs = (dr * ct - r * st) * z[1] - (dr * st + r * ct) * z[0];
        near_start = RealOps<Real>::fabs_(gs) <= g.star_kpp * H + star_df_noise(g);
    }
    if (near_start) {
        // near-tangent line: the roots of g in those intervals, with |g''| <= |gamma'''| / 3
        StarLineEval<Real, true> ev{g, yc, z, 0, sj, sd};
        Real gv[4], gd[4];
#pragma unroll 1
        for (int n = 0; n < 4; ++n) {
            ev.j = (sj - 1 + n) & (kNodes - 1);
            ev((Real)0, &gv[n], &gd[n]);
        }
        const Real nf = star_df_noise(g), nd = (sizeof(Real) == 4 ? (Real)2e-6 : (Real)1e-12) * g.star_kpp;
#pragma unroll 1
        for (int o = 0; o < 3; ++o) {
            ev.j = (sj - 1 + o) & (kNodes - 1);
            Real cand[kIntervalRoots];
            const int nc = star_interval_roots(ev, gv[o], gv[o + 1], gd[o], gd[o + 1], g.star_k3 * (Real)(1.0 / 3.0), nf,
                                               nd, unit * g.star_lmax, cand);
            for (int c = 0; c < nc && q < kMaxRoots; ++c) {
                Real gg, gdd, dz;
                star_dd(g, ev.j, cand[c], sj, sd, z, &gg, &gdd, &dz);
                tt[q] = dz * ((Real)(o - 1) * H + (cand[c] - sd));  // (gamma(t) - gamma(s)) . z
                jj[q] = ev.j;
                dd[q] = cand[c];
                ++q;
            }
        }
    }
    // the roots of one candidate interval of f, appended in scan order
    auto roots_of = [&](int j, Real fa, Real fb) {
        Real cand[kIntervalRoots];
        const int jn = (j + 1 == kNodes) ? 0 : j + 1;
        const Real da = g.scan_d[j][0] * z[1] - g.scan_d[j][1] * z[0];     // f' at the nodes
        const Real db = g.scan_d[jn][0] * z[1] - g.scan_d[jn][1] * z[0];
        const StarLineEval<Real, false> ev{g, yc, z, j, 0, (Real)0};
        const int nc = star_interval_roots(ev, fa, fb, da, db, g.star_kpp, star_f_noise(g), star_df_noise(g),
                                           star_dip_noise(g), cand);
        for (int c = 0; c < nc; ++c) {
            Real ct, st, p[2];
            angle_cs(g, j, cand[c], &ct, &st);
            star_local(g, ct, st, p, (Real *)nullptr);
            const Real s = (p[0] - yc[0]) * z[0] + (p[1] - yc[1]) * z[1];
            const bool ok = ray ? (s > tiny) : true;
            if (ok && q < kMaxRoots) {
                tt[q] = s;
                jj[q] = j;
                dd[q] = cand[c];
                ++q;
            }
        }
    };
    // two phases, so that the lanes of a warp refine their roots together: the scan (cheap,
    // of a different length in every lane) keeps up to kCand intervals that can hold a root
    // (a sign change, or an end within the guard); the refinement then runs candidate by
    // candidate in lock-step.  More candidates than that take further rounds, in scan order.
    constexpr int kCand = 8;
    int cj[kCand];
    Real cfa[kCand], cfb[kCand];
    const Real guard = star_guard(g);
    int r = 0, t = 0;   // the range being scanned and the position in it
    for (int round = 0; round <= kNodes / kCand; ++round) {
        int n_cand = 0;
        for (;;) {
            if (r >= nr || n_cand == kCand) break;
            if (t >= (r == 0 ? c0 : c1)) {
                ++r;
                t = 0;
                continue;
            }
            const int j = ((r == 0 ? s0 : s1) + t) & (kNodes - 1);
            ++t;
            if (!ray && ((j - sj + 1) & (kNodes - 1)) < 3) continue;   // the three around the start
            const int jn = (j + 1 == kNodes) ? 0 : j + 1;
            const Real fa = g.scan[j][0] * z[1] - g.scan[j][1] * z[0] - e;
            const Real fb = g.scan[jn][0] * z[1] - g.scan[jn][1] * z[0] - e;
            if ((fa < 0) != (fb < 0) || RealOps<Real>::fabs_(fa) < guard || RealOps<Real>::fabs_(fb) < guard) {
                cj[n_cand] = j;
                cfa[n_cand] = fa;
                cfb[n_cand] = fb;
                ++n_cand;
            }
        }
        for (int c = 0; c < n_cand; ++c) roots_of(cj[c], cfa[c], cfb[c]);
        if (r >= nr) break;   // the ranges are exhausted
    }
    return q;
}

// ---------------------------------------------------------------------------
// flux datum b_h(y) at the start point (Sec. 1); u = unit outward direction
// for spheres / (cos t, sin t) of the parameter for 2D curves; n = normal
// ---------------------------------------------------------------------------
template <typename Real> __device__ __forceinline__ const Real *flux_coefs(const DevGeom *gd);
template <> __device__ __forceinline__ const float *flux_coefs<float>(const DevGeom *gd) { return gd->flux_coef_f; }
template <> __device__ __forceinline__ const double *flux_coefs<double>(const DevGeom *gd) { return gd->flux_coef; }

// the general real spherical harmonics (3D) and harmonic polynomials (the workloads' degree-2
// data take the quadratic forms in flux_value; inlined, these loops are half of a kernel's
// code), with out-of-line copies
template <typename Real>
__device__ __forceinline__ Real flux_real_sh_body(const Real *c, int nc, const Real *u)
{
    // associated Legendre P_l^m(x) without the (-1)^m phase, x = cos(polar); the
    // coefficients already carry the normalisation of the real harmonics
    const Real x = u[2];
    Real sx2 = (Real)1 - x * x;
    sx2 = sx2 > (Real)0 ? sx2 : (Real)0;
    const Real sx = RealOps<Real>::sqrt_(sx2);
    Real ca = 1, sa = 0;  // cos / sin of the azimuth
    if (sx > (Real)0) {
        const Real inv = (Real)1 / sx;
        ca = u[0] * inv;
        sa = u[1] * inv;
    }
    int L = 0;
    while ((L + 2) * (L + 2) <= nc) ++L;
    Real v = 0;
    Real pmm = 1, cm = 1, sm = 0;  // P_m^m, cos(m az), sin(m az)
    for (int m = 0; m <= L; ++m) {
        if (m > 0) {
            pmm *= (Real)(2 * m - 1) * sx;
            const Real cn = cm * ca - sm * sa;
            sm = sm * ca + cm * sa;
            cm = cn;
        }
        Real p_prev = 0, p_cur = pmm;
        for (int l = m; l <= L; ++l) {
            if (l > m) {
                const Real p_next = (l == m + 1) ? x * (Real)(2 * m + 1) * pmm
                                                 : ((Real)(2 * l - 1) * x * p_cur - (Real)(l + m - 1) * p_prev) / (Real)(l - m);
                p_prev = p_cur;
                p_cur = p_next;
            }
            if (m == 0) v += c[l * l + l] * p_cur;
            else v += (c[l * l + l + m] * cm + c[l * l + l - m] * sm) * p_cur;
        }
    }
    return v;
}
template <typename Real, int D>
__device__ __forceinline__ Real flux_harmonic_poly_body(const Real *c, const Real *y, const Real *n)
{
    const Real s = c[0];
    const int T = (int)c[1];
    Real grad[D];
#pragma unroll
    for (int k = 0; k < D; ++k) grad[k] = 0;
    for (int t = 0; t < T; ++t) {
        const Real *row = c + 2 + t * (D + 1);
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const int ek = (int)row[1 + k];
            if (ek == 0) continue;
            Real term = row[0] * (Real)ek;
            for (int j = 0; j < D; ++j) {
                const int e = (int)row[1 + j] - (j == k ? 1 : 0);
                for (int p = 0; p < e; ++p) term *= y[j];
            }
            grad[k] += term;
        }
    }
    Real v = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) v += n[k] * grad[k];
    return s * v;
}
template <typename Real>
__device__ __noinline__ Real flux_real_sh(const Real *c, int nc, const Real *u) { return flux_real_sh_body<Real>(c, nc, u); }
template <typename Real, int D>
__device__ __noinline__ Real flux_harmonic_poly(const Real *c, const Real *y, const Real *n)
{
    return flux_harmonic_poly_body<Real, D>(c, y, n);
}

// OUT: the general real spherical harmonics and harmonic polynomials are called out of line
// (the plain general-surface kernels, which their instruction footprint bounds); elsewhere
// inlined (the sphere and variance-reduced kernels measured 1.5-15 % slower with the calls)
template <typename Real, int D, bool OUT = false>
__device__ Real flux_value(const DevGeom *gd, int h, const Real *y, const Real *u, const Real *n)
{
    const int basis = gd->flux_basis[h];
    const Real *c = flux_coefs<Real>(gd) + gd->flux_off[h];
    const int nc = gd->flux_n[h];
    if (basis == kFluxFourier) {
        Real v = c[0], ck = u[0], sk = u[1];
        for (int k = 1; 2 * k <= nc - 1; ++k) {
            v += c[2 * k - 1] * ck + c[2 * k] * sk;
            const Real cn = ck * u[0] - sk * u[1];
            sk = sk * u[0] + ck * u[1];
            ck = cn;
        }
        return v;
    }
    if (basis == kFluxRealSH) {
        if constexpr (D == 3) return OUT ? flux_real_sh<Real>(c, nc, u) : flux_real_sh_body<Real>(c, nc, u);
        return 0;
    }
    if (basis == kFluxHarmonicPoly)
        return OUT ? flux_harmonic_poly<Real, D>(c, y, n) : flux_harmonic_poly_body<Real, D>(c, y, n);
    if (basis == kFluxSphQuad) {
        if constexpr (D == 3) {
            const Real x = u[0], yv = u[1], z = u[2];
            return c[0] + c[1] * x + c[2] * yv + c[3] * z + x * (c[4] * x + c[5] * yv + c[6] * z) +
                   yv * (c[7] * yv + c[8] * z) + c[9] * z * z;
        }
        return 0;
    }
    if (basis == kFluxHarmonicQuad) {
        // s n . grad P with dP/dy_k = a_k + sum_j b_kj y_j + sum_{j<=l} c_kjl y_j y_l
        constexpr int per_k = 1 + D + D * (D + 1) / 2;
        Real yy[D * (D + 1) / 2];
        int t = 0;
#pragma unroll
        for (int j = 0; j < D; ++j)
#pragma unroll
            for (int l = j; l < D; ++l) yy[t++] = y[j] * y[l];
        Real v = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const Real *q = c + 1 + k * per_k;
            Real gk = q[0];
#pragma unroll
            for (int j = 0; j < D; ++j) gk += q[1 + j] * y[j];
#pragma unroll
            for (int m = 0; m < D * (D + 1) / 2; ++m) gk += q[1 + D + m] * yy[m];
            v += n[k] * gk;
        }
        return c[0] * v;
    }
    if (basis == kFluxPointCharge) {
        // s n . grad_y |y - x0|^{2-d} = s (2 - d) |y - x0|^{-d} (y - x0) . n
        Real r2 = 0, dot = 0;
#pragma unroll
        for (int k = 0; k < D; ++k) {
            const Real e = y[k] - c[1 + k];
            r2 += e * e;
            dot += e * n[k];
        }
        const Real ir = RealOps<Real>::rsqrt_(r2);
        Real ird = ir;
#pragma unroll
        for (int k = 1; k < D; ++k) ird *= ir;
        return c[0] * (Real)(2 - D) * ird * dot;
    }
    return 0;
}

// ---------------------------------------------------------------------------
// ellipsoids (Sec. 5, Example 2)
// ---------------------------------------------------------------------------
// uniform point by surface measure on ellipsoid slot e (Eq. naive_woi_p0): u uniform on
// the unit sphere from the words of attempt a of the (step, chain) stream, accepted when
// v^2 jmax^2 <= u^T A u (v the attempt's choice word; sqrt(u^T A u) is the area ratio of
// the map A^{-1/2}); y - c = A^{-1/2} u and the outward normal A (y - c) / |A (y - c)|.
// After kEllAttempts rejections the last attempt is kept (each attempt is accepted with
// probability at least sqrt(lambda_min / lambda_max)).
template <typename Real, int D>
__device__ void ell_uniform(const SEll<Real> &E, int e, const Rng &rng, int step, int chain, const StepWords &w0,
                            Real *v, Real *nrm)
{
    Real u[D];
    StepWords w = w0;
    const Real jm = E.jmax[e];
    for (int a = 0; a < kEllAttempts; ++a) {
        if (a > 0) {
            w.a = rng.words_at(step, chain, a, 0);
            if constexpr (two_calls<D>()) w.b = rng.words_at(step, chain, a, 1);
        }
        direction<Real, D>(w, u);
        Real J2 = 0;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            Real t = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) t += E.A[e][r][c] * u[c];
            J2 += u[r] * t;
        }
        const Real acc = u01<Real>(w.get(choice_word<D>()));
        if (acc * acc * jm * jm <= J2) break;
    }
#pragma unroll
    for (int r = 0; r < D; ++r) {
        Real t = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) t += E.map[e][r][c] * u[c];
        v[r] = t;
    }
    Real nn = 0;
#pragma unroll
    for (int r = 0; r < D; ++r) {
        Real t = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) t += E.A[e][r][c] * v[c];
        nrm[r] = t;
        nn += t * t;
    }
    const Real inv = RealOps<Real>::rsqrt_(nn);
#pragma unroll
    for (int r = 0; r < D; ++r) nrm[r] *= inv;
}

// c Phi(x, y) and c grad_x Phi(x, y) added to acc[0], acc[1..D], given dx = x - y
template <typename Real, int D>
__device__ __forceinline__ void tally_dx(const Real *dx, Real c, Real *acc)
{
    using O = RealOps<Real>;
    Real r2 = 0;
#pragma unroll
    for (int k = 0; k < D; ++k) r2 += dx[k] * dx[k];
    if (r2 <= (Real)0) return;  // x on a walk state exactly: measure zero, contributes nothing
    constexpr double PI = 3.14159265358979323846;
    if constexpr (D == 2) {
        const Real inv_r2 = O::rcp(r2);
        acc[0] += c * ((Real)(-1.0 / (4.0 * PI)) * O::fast_log(r2));
        const Real gc = c * (Real)(-1.0 / (2.0 * PI)) * inv_r2;
#pragma unroll
        for (int k = 0; k < D; ++k) acc[1 + k] += gc * dx[k];
    } else {
        // omega_d = 2 pi^{d/2} / Gamma(d/2)
        constexpr double omega = D == 3 ? 4.0 * PI : (D == 4 ? 2.0 * PI * PI : (D == 5 ? 8.0 * PI * PI / 3.0 : PI * PI * PI));
        const Real inv_r = O::rsqrt_(r2);
        Real inv_pow = inv_r;  // r^{-(d-2)}
#pragma unroll
        for (int k = 1; k < D - 2; ++k) inv_pow *= inv_r;
        acc[0] += c * (Real)(1.0 / ((D - 2) * omega)) * inv_pow;
        const Real gc = c * (Real)(-1.0 / omega) * inv_pow * inv_r * inv_r;
#pragma unroll
        for (int k = 0; k < D; ++k) acc[1 + k] += gc * dx[k];
    }
}

// the same with y = c_s + v and xc[s] = x - c_s formed in FP64 once per evaluation
// point (no cancellation near a surface)
template <typename Real, int D>
__device__ __forceinline__ void tally(const Real (*xc)[kMaxDim], int s, const Real *v, Real c, Real *acc)
{
    Real dx[D];
#pragma unroll
    for (int k = 0; k < D; ++k) dx[k] = xc[s][k] - v[k];
    tally_dx<Real, D>(dx, c, acc);
}

// x - c_s for every surface of the staged instance (all threads of the block)
template <typename Real>
__device__ __forceinline__ void fill_xc(Real (*xc)[kMaxDim], const DevGeom *gd, int n, int dim, const double *x)
{
    for (int i = threadIdx.x; i < n * dim; i += blockDim.x) {
        const int s = i / dim, k = i - s * dim;
        xc[s][k] = (Real)(x[k] - gd->center[s][k]);
    }
}

// ---------------------------------------------------------------------------
// one chain's state: surface s, offset v = y - c_s
// ---------------------------------------------------------------------------
template <typename Real, int D>
struct Chain {
    int s;
    Real v[D];
    Real Q, T;
    bool alive;
    int aj;       // on a star: the state's angle as node aj + offset ad; on a mesh: its triangle
    Real ad;
};

// ---------------------------------------------------------------------------
// triangle meshes (d = 3, Sec. 5): rows (v0, e1, e2, n) in the surface's local coordinates
// ---------------------------------------------------------------------------
template <typename Real> __device__ __forceinline__ const Real *tri_rows(const DevGeom *gd);
template <> __device__ __forceinline__ const float *tri_rows<float>(const DevGeom *gd) { return gd->tri_f; }
template <> __device__ __forceinline__ const double *tri_rows<double>(const DevGeom *gd) { return gd->tri_d; }

// uniform point by area on mesh slot m (Eq. naive_woi_p0): word 1 picks triangle j, the
// first with w1 <= T_j - 1; words 2 and 3 give barycentric (1 - s, s (1 - w), s w), s = sqrt(u)
template <typename Real>
__device__ void mesh_uniform(const DevGeom *gd, int m, const StepWords &w, Real *v, Real *nrm, int *tri)
{
    const uint32_t w1 = w.a.y;
    // the answer lies between the first triangles of the word's bucket and of the next one
    const int *bk = gd->tri_bucket + (size_t)m * (kTriBuckets + 1) + (w1 >> 22);
    int lo = __ldg(bk), hi = __ldg(bk + 1);
    const int last = gd->mesh_tri_off[m] + gd->mesh_ntri[m] - 1;
    hi = hi < last ? hi : last;
    while (lo < hi) {                       // first j in [lo, hi] with w1 <= tm1[j] (tm1[last] = 2^32 - 1)
        const int mid = (lo + hi) >> 1;
        if (__ldg(gd->tri_tm1 + mid) < w1) lo = mid + 1;
        else hi = mid;
    }
    const Real u = u01<Real>(w.a.z), ww = u01<Real>(w.a.w);
    const Real sq = RealOps<Real>::sqrt_(u), b1 = sq * ((Real)1 - ww), b2 = sq * ww;
    const Real *r = tri_rows<Real>(gd) + (size_t)lo * 12;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        v[k] = __ldg(r + k) + b1 * __ldg(r + 3 + k) + b2 * __ldg(r + 6 + k);
        nrm[k] = __ldg(r + 9 + k);
    }
    *tri = lo;
}

// crossings of the line (ray: t > 0) o + t z with mesh slot m, skipping triangle `exclude`,
// through the hierarchy; up to kMaxHits (t, triangle) pairs, a count above that is reported
// through the overflow counter and truncated
template <typename Real>
__device__ int mesh_hits(const DevGeom *gd, int m, const Real *o, const Real *z, bool ray, int exclude, Real *tt,
                         int *tri)
{
    const Real *rows = tri_rows<Real>(gd);
    const BvhWide *nodes = gd->bvh;
    const Real iz[3] = {(Real)1 / z[0], (Real)1 / z[1], (Real)1 / z[2]};
    const Real t_lo = ray ? (Real)0 : (Real)-1e30;
    // the padded box with corners (b0, b1, b2) and (b3, b4, b5) against the line (or the
    // ray's t >= 0 part)
    auto meets = [&](float b0, float b1, float b2, float b3, float b4, float b5) {
        const float lo[3] = {b0, b1, b2}, hi[3] = {b3, b4, b5};
        Real t0 = t_lo, t1 = (Real)1e30;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const Real ta = ((Real)lo[k] - o[k]) * iz[k], tb = ((Real)hi[k] - o[k]) * iz[k];
            const Real tmn = ta < tb ? ta : tb, tmx = ta < tb ? tb : ta;
            t0 = tmn > t0 ? tmn : t0;
            t1 = tmx < t1 ? tmx : t1;
        }
        return t0 <= t1;
    };
    int stack[kMeshStack];
    int sp = 0, q = 0;
    bool over = false;
    // the line starts on or inside the mesh, so it meets the root's box: the root is taken
    // without a test
    stack[sp++] = gd->mesh_node_off[m];
    // "while-while" order: each lane walks internal entries until it holds a leaf (or its
    // stack is empty), then the lanes test their leaves' triangles together, so that the leaf
    // code is not run once per lane while the other lanes wait in the node code. An entry
    // holds both children's boxes: one load per entry tests two boxes, and only the children
    // the line meets go on the stack (a leaf child as -(triangle + 1)).
    for (;;) {
        int t = -1;
        while (sp > 0) {
            const int ref = stack[--sp];
            if (ref < 0) {
                t = -ref - 1;
                break;
            }
            const float4 *np = reinterpret_cast<const float4 *>(nodes + ref);
            const float4 n0 = __ldg(np), n1 = __ldg(np + 1), n2 = __ldg(np + 2), n3 = __ldg(np + 3);
            const bool h0 = meets(n0.x, n0.y, n0.z, n0.w, n1.x, n1.y);
            const bool h1 = meets(n1.z, n1.w, n2.x, n2.y, n2.z, n2.w);
            // child 1 is taken first: the crossings come out in the depth-first order of the
            // build, right subtree first
            if (h0) {
                if (sp < kMeshStack) stack[sp++] = __float_as_int(n3.x);
                else over = true;
            }
            if (h1) {
                if (sp < kMeshStack) stack[sp++] = __float_as_int(n3.y);
                else over = true;
            }
        }
        if (t < 0) break;                        // the stack ran empty without another leaf
        {
            if (t == exclude) continue;
            const Real *r = rows + (size_t)t * 12;
            const Real e1[3] = {__ldg(r + 3), __ldg(r + 4), __ldg(r + 5)};
            const Real e2[3] = {__ldg(r + 6), __ldg(r + 7), __ldg(r + 8)};
            const Real p[3] = {z[1] * e2[2] - z[2] * e2[1], z[2] * e2[0] - z[0] * e2[2], z[0] * e2[1] - z[1] * e2[0]};
            const Real det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
            if (det == (Real)0) continue;
            const Real idet = (Real)1 / det;
            const Real sv[3] = {o[0] - __ldg(r), o[1] - __ldg(r + 1), o[2] - __ldg(r + 2)};
            const Real a = (sv[0] * p[0] + sv[1] * p[1] + sv[2] * p[2]) * idet;
            if (a < (Real)0 || a > (Real)1) continue;
            const Real qv[3] = {sv[1] * e1[2] - sv[2] * e1[1], sv[2] * e1[0] - sv[0] * e1[2], sv[0] * e1[1] - sv[1] * e1[0]};
            const Real b = (z[0] * qv[0] + z[1] * qv[1] + z[2] * qv[2]) * idet;
            if (b < (Real)0 || a + b > (Real)1) continue;
            const Real th = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) * idet;
            if (ray && !(th > (Real)0)) continue;
            if (q < kMaxHits) {
                tt[q] = th;
                tri[q] = t;
                ++q;
            } else {
                over = true;
            }
        }
    }
    if (over && gd->mesh_overflow) atomicAdd(gd->mesh_overflow, 1u);
    return q;
}

// transition i >= 1 to mesh h (relation rel); dy = y - c_h, the state's triangle in ch.aj.
// Line (same surface, skipping the state's own triangle) or ray (from a descendant): the
// pick-th crossing in line order (choice word 3), T *= q sign((y' - y).n(y')), Q *= 1/2 for the
// line.  Otherwise: uniform by area with Q *= K*(y', y) |dOmega_h|.
template <typename Real>
__device__ void mesh_step(const DevGeom *gd, Real area, int h, int rel, const StepWords &w, const Real *dy,
                          Chain<Real, 3> &ch)
{
    using O = RealOps<Real>;
    constexpr double PI = 3.14159265358979323846;
    const int m = gd->mesh_slot[h];
    if (rel == 2) {
        Real vn[3], nrm[3];
        int t;
        mesh_uniform<Real>(gd, m, w, vn, nrm, &t);
        Real r2 = 0, dot = 0;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
            const Real diff = vn[c] - dy[c];
            r2 += diff * diff;
            dot += diff * nrm[c];
            ch.v[c] = vn[c];
        }
        const Real ir = O::rsqrt_(r2);
        ch.Q *= dot * ir * ir * ir * (Real)(1.0 / (4.0 * PI)) * area;
        ch.aj = t;
    } else {
        Real z[3];
        direction<Real, 3>(w, z);
        Real tt[kMaxHits];
        int tri[kMaxHits];
        const int q = mesh_hits<Real>(gd, m, dy, z, rel == 1, rel == 0 ? ch.aj : -1, tt, tri);
        if (q == 0) {                          // no admissible crossing (tangent line): the walk ends
            ch.alive = false;
            ch.T = 0;
            return;
        }
        const int pick = (int)(((uint64_t)w.get(choice_word<3>()) * (uint64_t)q) >> 32);
        int sel = 0;
        for (int a = 0; a < q; ++a) {
            int rank = 0;
            for (int b = 0; b < q; ++b) rank += (tt[b] < tt[a]) || (tt[b] == tt[a] && b < a);
            if (rank == pick) sel = a;
        }
        const Real t = tt[sel];
        const Real *r = tri_rows<Real>(gd) + (size_t)tri[sel] * 12;
        const Real zn = z[0] * __ldg(r + 9) + z[1] * __ldg(r + 10) + z[2] * __ldg(r + 11);
        const Real dot = t * zn;               // (y' - y) . n(y')
#pragma unroll
        for (int c = 0; c < 3; ++c) ch.v[c] = dy[c] + t * z[c];
        if (rel == 0) ch.Q *= (Real)0.5;
        ch.T *= (Real)q * (dot > 0 ? (Real)1 : (dot < 0 ? (Real)-1 : (Real)0));
        ch.aj = tri[sel];
    }
    ch.s = h;
}

// the part (0: beta >= 0, 1: beta < 0) of a uniform start point on a circle or sphere, from
// its direction's words w and beta b evaluated in Real.  In FP32, where |b| is within the
// surface's tolerance of 0 (the FP32 error is far below it), the sign is taken again in
// FP64 from the same words, so that the part is the one an FP64 evaluation gives.
template <typename Real, int D>
__device__ __forceinline__ int vr_part(const DevGeom *gd, int h, const StepWords &w, Real b)
{
    if constexpr (sizeof(Real) == 4) {
        if (fabsf(b) < (float)gd->vr_tol[h]) {
            double u[D], y[D];
            direction<double, D>(w, u);
#pragma unroll
            for (int c = 0; c < D; ++c) y[c] = gd->center[h][c] + gd->radius[h] * u[c];
            return gd->beta_scale[h] * flux_value<double, D>(gd, h, y, u, u) >= 0.0 ? 0 : 1;
        }
    }
    return b >= (Real)0 ? 0 : 1;
}

// VR start where the parts have no closed form (d >= 3, and 2D data other than a Fourier
// series): kVrTrials uniform points on dOmega_h (the circle / sphere, star, ellipsoid or mesh
// sampler) shared by both chains (trial t draws the step-0 words of chain id t << 12; trial 0
// is chain 0's own).  Chain k starts at the first trial of
// its sign with Q = beta |dOmega| C_k / kVrTrials, C_k the trials of that sign: an unbiased
// estimate of |dOmega^+/-| / |dOmega| that is independent of where the first trial of that
// sign lies, so the chain's term has Algorithm 3's mean.  No trial of a sign: that chain is
// dead.  On stars, ellipsoids and meshes the sign is taken in the kernel's precision, like the
// ellipsoid sampler's acceptance test.
template <typename Real, int D, bool STAR>
__device__ void vr_trials_start(const SGeom<Real> &g, const DevGeom *gd, int h, const StepWords &w0, const Rng &rng,
                                Chain<Real, D> *ch)
{
    bool is_ell = false, is_mesh = false, is_star = false;
    if constexpr (STAR && D >= 3) is_ell = g.type[h] == kEllipsoid;
    if constexpr (STAR && D == 3) is_mesh = g.type[h] == kMesh;
    if constexpr (STAR && D == 2) is_star = g.type[h] == kStar;
    int n[2] = {0, 0}, af[2] = {0, 0};
    Real vf[2][D], nf[2][D], adf[2] = {0, 0};
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int c = 0; c < D; ++c) vf[k][c] = nf[k][c] = 0;
    for (int t = 0; t < kVrTrials; ++t) {
        const int cid = t << 12;
        StepWords w = w0;
        if (t > 0) {
            w.a = rng.words(0, cid, 0);
            if constexpr (two_calls<D>()) w.b = rng.words(0, cid, 1);
        }
        Real v[D], nrm[D], y[D], ad = 0;
        int aj = 0;
        if (is_star) {
            if constexpr (STAR && D == 2) {   // by arc length, as the plain start
                Real ct, st;
                const SGeomS<Real> &gs = star_geom(g);
                star_at_arclen(gs, (double)u01<Real>(w.a.y) * (double)g.area[h], &aj, &ad);
                angle_cs(g, aj, ad, &ct, &st);
                star_local(gs, ct, st, v, nrm);
            }
        } else if (is_mesh) {
            if constexpr (STAR && D == 3) mesh_uniform<Real>(gd, gd->mesh_slot[h], w, v, nrm, &aj);
        } else if (is_ell) {
            if constexpr (STAR && D >= 3) {
                const SEll<Real> &E = static_cast<const SGeomE<Real> &>(g).ell;
                ell_uniform<Real, D>(E, E.slot[h], rng, 0, cid, w, v, nrm);
            }
        } else {
            direction<Real, D>(w, nrm);
#pragma unroll
            for (int c = 0; c < D; ++c) v[c] = g.radius[h] * nrm[c];
        }
#pragma unroll
        for (int c = 0; c < D; ++c) y[c] = (g.c_hi[h][c] + g.c_lo[h][c]) + v[c];
        const Real b = g.beta_scale[h] * flux_value<Real, D>(gd, h, y, nrm, nrm);
        const int part = (is_ell || is_mesh || is_star) ? (b >= (Real)0 ? 0 : 1) : vr_part<Real, D>(gd, h, w, b);
        if (n[part] == 0) {
#pragma unroll
            for (int c = 0; c < D; ++c) {
                vf[part][c] = v[c];
                nf[part][c] = nrm[c];
            }
            af[part] = aj;
            adf[part] = ad;
        }
        ++n[part];
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        Chain<Real, D> &q = ch[k];
        q.T = 1;
        q.s = h;
        q.aj = af[k];
        q.ad = adf[k];
        q.alive = n[k] > 0 && gd->flux_basis[h] != kFluxZero;
        Real y[D];
#pragma unroll
        for (int c = 0; c < D; ++c) {
            q.v[c] = q.alive ? vf[k][c] : (Real)0;
            y[c] = (g.c_hi[h][c] + g.c_lo[h][c]) + q.v[c];
        }
        q.Q = q.alive ? g.beta_scale[h] * flux_value<Real, D>(gd, h, y, nf[k], nf[k]) *
                            (Real)(gd->area[h] * ((double)n[k] / kVrTrials))
                      : (Real)0;
    }
}

// start (i = 0): y_0 uniform on dOmega_h (plain) or on dOmega_h^{+/-} (VR), Q = beta(y_0) |part|
template <typename Real, int D, bool VR, bool STAR>
__device__ void chain_start(const SGeom<Real> &g, const DevGeom *gd, int h, int k, const StepWords &w,
                            const Rng &rng, Chain<Real, D> &ch)
{
    ch.T = 1;
    ch.alive = true;
    ch.s = h;
    ch.aj = 0;
    ch.ad = 0;
    Real u[D], nrm[D];
    double part_len = g.area[h];
    if constexpr (VR) {
        part_len = gd->part_len[h][k];
        if (!(part_len > 0.0) || gd->flux_basis[h] == kFluxZero) {
            ch.alive = false;
            ch.Q = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) ch.v[c] = 0;
            return;
        }
    }
    const bool is_star = STAR && g.type[h] == kStar;
    bool is_ell = false, is_mesh = false;
    if constexpr (STAR && D >= 3) is_ell = g.type[h] == kEllipsoid;
    if constexpr (STAR && D == 3) is_mesh = g.type[h] == kMesh;
    if (is_mesh) {
        if constexpr (STAR && D == 3) {
            mesh_uniform<Real>(gd, gd->mesh_slot[h], w, ch.v, nrm, &ch.aj);
#pragma unroll
            for (int c = 0; c < D; ++c) u[c] = nrm[c];
        }
    } else if (is_ell) {
        if constexpr (STAR && D >= 3) {
            const SEll<Real> &E = static_cast<const SGeomE<Real> &>(g).ell;
            ell_uniform<Real, D>(E, E.slot[h], rng, 0, k, w, ch.v, nrm);
#pragma unroll
            for (int c = 0; c < D; ++c) u[c] = nrm[c];
        }
    } else if (!VR && !is_star) {
        direction<Real, D>(w, u);
#pragma unroll
        for (int c = 0; c < D; ++c) {
            ch.v[c] = g.radius[h] * u[c];
            nrm[c] = u[c];
        }
    } else {
        if constexpr (D == 2 && (VR || STAR)) {   // (the plain walk on circles never gets here)
            // target position (FP64) along the surface, or along the concatenated
            // arcs of the requested sign (VR)
            const double s_target = (double)u01<Real>(w.a.y) * part_len;
            Real ct, st;
            int j_sel = 0;
            Real d_sel = 0;
            if constexpr (VR) {
                double s = s_target;
                const int want = k == 0 ? 1 : -1;
                int a_sel = -1;
                for (int a = gd->arc_off[h]; a < gd->arc_off[h] + gd->arc_n[h]; ++a) {
                    if (gd->arc_sign[a] != want) continue;
                    a_sel = a;
                    if (s < gd->arc_len[a]) break;
                    s -= gd->arc_len[a];
                }
                if (s > gd->arc_len[a_sel]) s = gd->arc_len[a_sel];
                if (is_star) {
                    if constexpr (STAR) {
                        star_at_arclen(star_geom(g), gd->arc_s0[a_sel] + s, &j_sel, &d_sel);
                        angle_cs(g, j_sel, d_sel, &ct, &st);
                    }
                } else {
                    // t = t0 + s / R, split into a node and an offset in FP64
                    const double t = gd->arc_t0[a_sel] + s / (double)gd->radius[h];
                    const double H = 2.0 * 3.14159265358979323846 / kNodes;
                    int j = (int)(t / H);
                    j = j < 0 ? 0 : (j >= kNodes ? kNodes - 1 : j);
                    angle_cs(g, j, (Real)(t - j * H), &ct, &st);
                }
            } else if constexpr (STAR) {   // (only a star reaches here in the plain walk)
                star_at_arclen(star_geom(g), s_target, &j_sel, &d_sel);
                angle_cs(g, j_sel, d_sel, &ct, &st);
            }
            if (is_star) {
                if constexpr (STAR) star_local(star_geom(g), ct, st, ch.v, nrm);
                ch.aj = j_sel;
                ch.ad = d_sel;
            } else {
                nrm[0] = ct;
                nrm[1] = st;
                ch.v[0] = g.radius[h] * ct;
                ch.v[1] = g.radius[h] * st;
            }
            u[0] = ct;
            u[1] = st;
        } else if constexpr (VR) {   // (in 3-6D only the variance-reduced walk reaches here)
            // VR on a d >= 3 sphere whose data is linear in u: the two parts are mirror-image
            // hemispheres, so a uniform direction that lands in the part of the wrong sign is
            // reflected, u -> -u, which leaves it uniform on the requested one
            direction<Real, D>(w, u);
            Real y0[D];
#pragma unroll
            for (int c = 0; c < D; ++c) {
                ch.v[c] = g.radius[h] * u[c];
                nrm[c] = u[c];
                y0[c] = (g.c_hi[h][c] + g.c_lo[h][c]) + ch.v[c];
            }
            const Real b = g.beta_scale[h] * flux_value<Real, D>(gd, h, y0, u, nrm);
            if (k != vr_part<Real, D>(gd, h, w, b)) {
#pragma unroll
                for (int c = 0; c < D; ++c) {
                    u[c] = -u[c];
                    nrm[c] = -nrm[c];
                    ch.v[c] = -ch.v[c];
                }
            }
        }
    }
    Real y[D];
#pragma unroll
    for (int c = 0; c < D; ++c) y[c] = (g.c_hi[h][c] + g.c_lo[h][c]) + ch.v[c];
    ch.Q = g.beta_scale[h] * flux_value<Real, D, STAR && !VR>(gd, h, y, u, nrm) * (Real)part_len;
}

// transition i >= 1 from an ellipsoid-bound state to ellipsoid h (relation rel); dy = y - c_h.
// Line (same surface): the other root t = -2 b / a of a t^2 + 2 b t + c = 0, Q *= 1/2, T *= q sign
// = +1 (a chord of a convex surface leaves it outward).  Ray (from a descendant): the positive
// root, Q and T unchanged.  Otherwise: uniform y' with Q *= K*(y', y) |dOmega_h|.
template <typename Real, int D>
__device__ void ell_step(const SGeomE<Real> &g, int h, int rel, const StepWords &w, const Rng &rng, int step,
                         int chain, const Real *dy, Chain<Real, D> &ch)
{
    using O = RealOps<Real>;
    constexpr double PI = 3.14159265358979323846;
    const SEll<Real> &E = g.ell;
    const int e = E.slot[h];
    if (rel == 2) {
        Real vn[D], nrm[D];
        ell_uniform<Real, D>(E, e, rng, step, chain, w, vn, nrm);
        Real r2 = 0, dot = 0;
#pragma unroll
        for (int c = 0; c < D; ++c) {
            const Real diff = vn[c] - dy[c];
            r2 += diff * diff;
            dot += diff * nrm[c];
            ch.v[c] = vn[c];
        }
        constexpr double omega = D == 3 ? 4.0 * PI : (D == 4 ? 2.0 * PI * PI : (D == 5 ? 8.0 * PI * PI / 3.0 : PI * PI * PI));
        const Real ir = O::rsqrt_(r2);
        Real inv_rd = ir;
#pragma unroll
        for (int k = 1; k < D; ++k) inv_rd *= ir;
        ch.Q *= dot * inv_rd * (Real)(1.0 / omega) * g.area[h];
    } else {
        Real z[D];
        direction<Real, D>(w, z);
        Real a2 = 0, b1 = 0, c0 = -1;
#pragma unroll
        for (int r = 0; r < D; ++r) {
            Real az = 0, ady = 0;
#pragma unroll
            for (int c = 0; c < D; ++c) {
                az += E.A[e][r][c] * z[c];
                ady += E.A[e][r][c] * dy[c];
            }
            a2 += z[r] * az;
            b1 += dy[r] * az;
            c0 += dy[r] * ady;
        }
        Real t;
        if (rel == 0) {
            t = (Real)-2 * b1 / a2;
            const Real tiny = sizeof(Real) == 4 ? (Real)1e-6 : (Real)1e-9;
            if (O::fabs_(t) * E.jmax[e] <= tiny) {   // tangent: only y itself, the walk ends
                ch.alive = false;
                ch.T = 0;
                return;
            }
            ch.Q *= (Real)0.5;
        } else {
            const Real disc = b1 * b1 - a2 * c0;
            const Real sq = O::sqrt_(disc > 0 ? disc : (Real)0);
            t = (b1 <= 0) ? (sq - b1) / a2 : -c0 / (b1 + sq);
        }
#pragma unroll
        for (int c = 0; c < D; ++c) ch.v[c] = dy[c] + t * z[c];
    }
    ch.s = h;
}

// transition i >= 1 from surface ch.s to h (relation rel)
template <typename Real, int D, bool STAR>
__device__ void chain_step(const SGeom<Real> &g, const DevGeom *gd, int h, int rel, const StepWords &w, const Rng &rng,
                           int step, int chain, Chain<Real, D> &ch)
{
    using O = RealOps<Real>;
    constexpr double PI = 3.14159265358979323846;
    // dy = y - c_h
    Real dy[D];
    if (rel == 0) {
#pragma unroll
        for (int c = 0; c < D; ++c) dy[c] = ch.v[c];
    } else {
        center_diff<Real, D>(g, ch.s, h, dy);
#pragma unroll
        for (int c = 0; c < D; ++c) dy[c] += ch.v[c];
    }
    if constexpr (STAR && D == 3) {
        if (g.type[h] == kMesh) {
            mesh_step<Real>(gd, g.area[h], h, rel, w, dy, ch);
            return;
        }
    }
    if constexpr (STAR && D >= 3) {
        if (g.type[h] == kEllipsoid) {
            ell_step<Real, D>(static_cast<const SGeomE<Real> &>(g), h, rel, w, rng, step, chain, dy, ch);
            return;
        }
    }
    if (STAR && g.type[h] == kStar) {
        if constexpr (STAR && D == 2) {
            const SGeomS<Real> &gs = star_geom(g);
            Real vn[2], nrm[2];
            if (rel == 2) {
                // uniform on the star by arc length; Q *= K*(y_i, y_{i-1}) |dOmega_h|
                int j;
                Real delta, ct, st;
                star_at_arclen(gs, (double)u01<Real>(w.a.y) * (double)gs.panel_s[kNodes], &j, &delta);
                angle_cs(g, j, delta, &ct, &st);
                star_local(gs, ct, st, vn, nrm);
                ch.aj = j;
                ch.ad = delta;
                const Real dx = vn[0] - dy[0], dyy = vn[1] - dy[1];
                const Real r2 = dx * dx + dyy * dyy;
                ch.Q *= (dx * nrm[0] + dyy * nrm[1]) * O::rcp(r2) * (Real)(1.0 / (2.0 * PI)) * g.area[h];
            } else {
                Real z[2];
                direction<Real, 2>(w, z);
                Real tt[kMaxRoots], dd[kMaxRoots];
                int jj[kMaxRoots];
                const int q = star_intersections(gs, dy, z, rel == 1, ch.aj, ch.ad, tt, jj, dd);
                if (q == 0) {
                    ch.alive = false;
                    ch.T = 0;
                    return;
                }
                const int pick = (int)(((uint64_t)w.get(choice_word<2>()) * (uint64_t)q) >> 32);
                // the pick-th smallest line parameter
                int sel = 0;
                for (int a = 0; a < q; ++a) {
                    int rank = 0;
                    for (int b = 0; b < q; ++b) rank += (tt[b] < tt[a]) || (tt[b] == tt[a] && b < a);
                    if (rank == pick) sel = a;
                }
                Real ct, st;
                angle_cs(g, jj[sel], dd[sel], &ct, &st);
                star_local(gs, ct, st, vn, nrm);
                ch.aj = jj[sel];
                ch.ad = dd[sel];
                const Real dot = (vn[0] - dy[0]) * nrm[0] + (vn[1] - dy[1]) * nrm[1];
                if (rel == 0) ch.Q *= (Real)0.5;
                ch.T *= (Real)q * (dot > 0 ? (Real)1 : (dot < 0 ? (Real)-1 : (Real)0));
            }
            ch.s = h;
            ch.v[0] = vn[0];
            ch.v[1] = vn[1];
            return;
        }
    }
    // circles / d-spheres: one isotropic unit vector z serves the three cases, evaluated
    // without branches (the lanes of a warp take different cases) and selected at the end
    Real z[D];
    direction<Real, D>(w, z);
    const Real R = g.radius[h];
    Real b = 0, c0 = -R * R, r2 = 0, dot = 0;
#pragma unroll
    for (int c = 0; c < D; ++c) {
        b += z[c] * dy[c];
        c0 += dy[c] * dy[c];
        const Real diff = R * z[c] - dy[c];
        r2 += diff * diff;
        dot += diff * z[c];
    }
    // same surface: line through a point of the sphere, the other intersection at t = -2 b;
    // Q *= 1/2, T *= q sign = +1.  A tangent line (|t| at rounding level) meets the sphere
    // only at y: q = 0 ends the walk.
    const Real tiny = sizeof(Real) == 4 ? (Real)1e-6 : (Real)1e-9;
    if (rel == 0 && O::fabs_((Real)2 * b) <= tiny * R) {
        ch.alive = false;
        ch.T = 0;
        return;
    }
    // descendant: ray from inside, t = -b + sqrt(b^2 - c0) > 0 in the stable form; Q, T unchanged
    const Real sq = O::sqrt_(b * b - c0 > 0 ? b * b - c0 : (Real)0);
    const Real t_ray = (b <= 0) ? (sq - b) : O::div_(-c0, b + sq);
    // otherwise: uniform y' = c_h + R z (normal z); Q *= K*(y', y) |dOmega_h| = (y'-y).z / (omega_d r^d) |dOmega_h|
    constexpr double omega = D == 2 ? 2.0 * PI : (D == 3 ? 4.0 * PI : (D == 4 ? 2.0 * PI * PI : (D == 5 ? 8.0 * PI * PI / 3.0 : PI * PI * PI)));
    Real inv_rd;
    if constexpr (D == 2) {
        inv_rd = O::rcp(r2);
    } else {
        const Real ir = O::rsqrt_(r2);
        inv_rd = ir;
#pragma unroll
        for (int k = 1; k < D; ++k) inv_rd *= ir;
    }
    const Real t = rel == 0 ? (Real)-2 * b : t_ray;
#pragma unroll
    for (int c = 0; c < D; ++c) ch.v[c] = rel == 2 ? R * z[c] : dy[c] + t * z[c];
    ch.Q *= rel == 0 ? (Real)0.5 : (rel == 1 ? (Real)1 : dot * inv_rd * (Real)(1.0 / omega) * g.area[h]);
    ch.s = h;
}

// ---------------------------------------------------------------------------
// one walk: returns the tally f[0] (u) and f[1..D] (grad u) of
// N sum_i w_i A^i prod_{m=1}^{i} sign(alpha_{H_m}) Q_i T_i Phi(x, Y_i), summed
// over the two chains for VR
// ---------------------------------------------------------------------------
// The steps of one walk (Algorithms 2-3), handing each state to `sink`:
// sink(i, k, chain, c) with c = N w_i ||alpha||_1^i prod_{m=1}^{i} sign(alpha_{H_m}) Q_i T_i
// the coefficient of Phi(x, y_i) (0 for a chain that has ended).
// The words of step i of one chain: one generator call per step, except on 2D instances of
// circles only (the sphere kernels of dimension 2), whose steps use two words (the schedule
// word and the angle or arc position): steps 2j and 2j + 1 share the call (j, chain, 0), step
// 2j taking its words x, y and step 2j + 1 its z, w, so that half the calls are made.  The
// call of the current pair is kept from one step to the next.
template <int D, bool STAR>
struct ChainWords {
    static constexpr bool kPair = D == 2 && !STAR;
    U4 c;
    int j = -1;
    __device__ __forceinline__ StepWords step(const Rng &rng, int i, int chain)
    {
        StepWords w;
        if constexpr (kPair) {
            if ((i >> 1) != j) {
                c = rng.words(i >> 1, chain, 0);
                j = i >> 1;
            }
            const bool odd = (i & 1) != 0;
            w.a.x = odd ? c.z : c.x;
            w.a.y = odd ? c.w : c.y;
            w.a.z = 0u;
            w.a.w = 0u;
        } else {
            w.a = rng.words(i, chain, 0);
            if constexpr (two_calls<D>()) w.b = rng.words(i, chain, 1);
        }
        return w;
    }
};

// the schedule word of step i of the walk `first` (a shared schedule's group leader), in the
// same layout
template <int D, bool STAR>
__device__ __forceinline__ uint32_t first_walk_schedule_word(const Rng &rng, uint64_t first, int i)
{
    if constexpr (ChainWords<D, STAR>::kPair) {
        const U4 c = philox10((uint32_t)first, (uint32_t)(first >> 32), (uint32_t)(i >> 1), 0u, rng.k0, rng.k1);
        return (i & 1) ? c.z : c.x;
    } else {
        return philox10((uint32_t)first, (uint32_t)(first >> 32), (uint32_t)i, 0u, rng.k0, rng.k1).x;
    }
}

// LANE0: the 32 lanes of the warp run the 32 walks of one schedule group together, lane 0
// the group's first, so a shared schedule word is lane 0's own (one shuffle per step).
// Otherwise the word is drawn from the first walk's stream here.
template <typename Real, int D, bool VR, bool STAR, bool LANE0 = false, typename Sink>
__device__ __forceinline__ void walk_steps(const SGeom<Real> &g, const DevGeom *gd, const Rng &rng, int sched_group,
                                           uint64_t group, Sink &sink)
{
    Chain<Real, D> ch[VR ? 2 : 1];
    ChainWords<D, STAR> cw[VR ? 2 : 1];
    Real S = 1;
    int hp = 0;
    for (int i = 0; i <= g.M; ++i) {
        const StepWords w0 = cw[0].step(rng, i, 0);
        uint32_t hw = w0.a.x;
        if (sched_group > 1) {
            if constexpr (LANE0) hw = __shfl_sync(0xFFFFFFFFu, hw, 0);
            else hw = first_walk_schedule_word<D, STAR>(rng, group * 32u, i);
        }
        const int h = schedule(g, i, hw);
        if (i > 0) S *= g.alpha_sign[h];
        const int rel = (i > 0) ? relation(g, hp, h) : 0;
        bool trials = false;
        if constexpr (VR) {
            if (i == 0 && gd->part_len[h][0] < 0.0) {
                vr_trials_start<Real, D, STAR>(g, gd, h, w0, rng, ch);
                trials = true;
            }
        }
        // with general surfaces, and on spheres in d >= 4, one copy of the transition code
        // serves both chains (the instruction footprint, not the work, bounds those kernels:
        // unrolled, the star's variance-reduced kernel is 1.6x and the 6D one 1.14x slower; on
        // spheres in d <= 3 the unrolled loop is 9 % faster)
#pragma unroll((STAR || D >= 4) ? 1 : 2)
        for (int k = 0; k < (VR ? 2 : 1); ++k) {
            StepWords w = w0;
            if constexpr (VR) {
                if (k == 1 && !trials) w = cw[1].step(rng, i, 1);
            }
            if (i == 0) {
                if (!trials) chain_start<Real, D, VR, STAR>(g, gd, h, k, w, rng, ch[k]);
            } else if (ch[k].alive) {
                chain_step<Real, D, STAR>(g, gd, h, rel, w, rng, i, k, ch[k]);
            }
            sink(i, k, ch[k], ch[k].alive ? g.coef[i] * S * ch[k].Q * ch[k].T : (Real)0);
        }
        hp = h;
    }
}

// sink that tallies Phi and grad Phi at one point (and optionally records the states)
template <typename Real, int D, bool TRACE>
struct TallySink {
    const SGeom<Real> &g;
    const Real (*xc)[kMaxDim];
    Real *f;
    double *trace;
    __device__ __forceinline__ void operator()(int i, int k, const Chain<Real, D> &ch, Real c)
    {
        if (ch.alive) tally<Real, D>(xc, ch.s, ch.v, c, f);
        if constexpr (TRACE) {
            if (trace) {
                double *t = trace + ((size_t)k * (g.M + 1) + i) * (D + 2);
                for (int q = 0; q < D; ++q)
                    t[q] = ((double)g.c_hi[ch.s][q] + (double)g.c_lo[ch.s][q]) + (double)ch.v[q];
                t[D] = (double)ch.Q;
                t[D + 1] = (double)ch.T;
            }
        }
    }
};

// one walk: returns the tally f[0] (u) and f[1..D] (grad u) of
// N sum_i w_i A^i prod_{m=1}^{i} sign(alpha_{H_m}) Q_i T_i Phi(x, Y_i), summed
// over the two chains for VR
template <typename Real, int D, bool VR, bool STAR, bool TRACE = false, bool LANE0 = false>
__device__ void walk(const SGeom<Real> &g, const DevGeom *gd, const Real (*xc)[kMaxDim], const Rng &rng,
                     int sched_group, uint64_t group, Real *f, double *trace = nullptr)
{
#pragma unroll
    for (int c = 0; c <= D; ++c) f[c] = 0;
    TallySink<Real, D, TRACE> sink{g, xc, f, trace};
    walk_steps<Real, D, VR, STAR, LANE0>(g, gd, rng, sched_group, group, sink);
}

// Two independent walks of one lane, advanced step by step in the same loop so that the
// scheduler can overlap their dependency chains (plain variant with per-walk schedules; each
// walk has its own stream, schedule and state, exactly as if walked alone): f[q] receives walk
// q's tally
template <typename Real, int D, bool STAR>
__device__ void walk_pair(const SGeom<Real> &g, const DevGeom *gd, const Real (*xc)[kMaxDim], const Rng *rng,
                          Real (*f)[D + 1])
{
    Chain<Real, D> ch[2];
    ChainWords<D, STAR> cw[2];
    Real S[2] = {1, 1};
    int hp[2] = {0, 0};
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int c = 0; c <= D; ++c) f[q][c] = 0;
    for (int i = 0; i <= g.M; ++i) {
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            const StepWords w = cw[q].step(rng[q], i, 0);
            const int h = schedule(g, i, w.a.x);
            if (i > 0) S[q] *= g.alpha_sign[h];
            const int rel = (i > 0) ? relation(g, hp[q], h) : 0;
            if (i == 0) chain_start<Real, D, false, STAR>(g, gd, h, 0, w, rng[q], ch[q]);
            else if (ch[q].alive) chain_step<Real, D, STAR>(g, gd, h, rel, w, rng[q], i, 0, ch[q]);
            if (ch[q].alive) tally<Real, D>(xc, ch[q].s, ch[q].v, g.coef[i] * S[q] * ch[q].Q * ch[q].T, f[q]);
            hp[q] = h;
        }
    }
}

}  // namespace woi
