/*
 * woi_oracle.c -- plain, slow FP64 CPU oracle of the Walk-on-Interfaces (WoI)
 * estimator (Ding & Stinchcombe, "Walk-on-Interfaces", arXiv 2508.16767).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file: only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, header, table or constant
 * generator with the CUDA library; the two agree only on the documented
 * random-number protocol (Philox4x32-10, written here from its published
 * definition) and on the input format.
 *
 * What it computes (section numbers are the paper's):
 *   - Sec. 3: unit-coefficient system gamma_i - alpha_i sum_j K*_ij gamma_j =
 *     beta_i and its truncated Neumann series with weights
 *     w_i = 1 - delta_{iM}/2.  alpha, beta scaling and the schedule
 *     thresholds are prepared by oracle.py and passed in.
 *   - Sec. 4.2.1, Eqs. naive_woi_p0 / naive_woi_p: the transition densities
 *     (uniform start; line-isotropic if h_{i-1} = h_i; ray-isotropic if
 *     h_{i-1} is a descendant of h_i; uniform otherwise).
 *   - Sec. 4.2.2, Eqs. naive_woi_Q / naive_woi_T: the Q and T factors.
 *   - Sec. 4.3.1, Thm 4.2 and Eq. woi_estimator: scheduled interfaces
 *     H_0 ~ U{1..N}, H_i ~ |alpha_n| / ||alpha||_1, the weight
 *     N ||alpha||_1^i prod_{m=1}^{i} sign(alpha_{H_m}).
 *   - Algorithms 1-2 (plain walk), Algorithm 3 and Eq.
 *     variance_reduced_woi_estimator (two chains from the beta >= 0 and
 *     beta < 0 parts of the first interface; in 2D the parts are arcs, in
 *     d >= 3 they are the hemispheres of data linear in the unit vector, and
 *     on other d >= 3 spheres the start is drawn from uniform trials).
 *   - Sec. 4.5, Eq. naive_woi_grad_estimator: the gradient tally uses
 *     grad_x Phi on the same trajectory.
 *   - Sec. 5, Example 2: ellipsoids (y - c)^T A (y - c) = 1 as surfaces, with
 *     the point-charge potential |x - x0|^{2-d} as manufactured solution.
 *     Uniform points by surface measure come from a uniform point u of the
 *     unit sphere mapped to y = c + A^{-1/2} u (the symmetric square root, so
 *     that the map does not depend on how an eigen-decomposition orders or
 *     signs its vectors), accepted with probability J(u) / max J, where
 *     J(u) = |A^{1/2} u| = sqrt(u^T A u) is the area ratio of the map (von
 *     Neumann rejection) and max J = sqrt(largest eigenvalue of A).
 *   - Closed triangle meshes (3D; the paper's primary surface representation,
 *     Sec. 5): uniform points by area (a triangle by the cumulative-area
 *     thresholds, then uniform barycentric coordinates), face normals, and
 *     line / ray intersections by testing every triangle (no acceleration
 *     structure); a line through a point of triangle j skips triangle j.
 *
 * Readings of the paper taken here, each with its reason:
 *   R1 the alpha-sign product runs over m = 1..i (Thm 4.2 and its proof), not
 *      m = 0..i as the algorithms print it: alpha_{h_0} never appears in the
 *      Neumann-series expansion of Sec. 3;
 *   R2 in the "otherwise" (uniform) transition T is left unchanged: the sign
 *      already lives in the signed K* inside Q (Thm 4.1 needs Q*T = prod K* / p);
 *   R3 K* is evaluated as K*(y_i, y_{i-1}) with the normal at the new point, as
 *      K*_ij is defined in Sec. 3 (Sec. 4.2.2 prints the arguments swapped);
 *   R4 "descendant" means strict descendant at any depth: a ray from inside
 *      any region nested in the target's meets the target from inside;
 *   R5 a line/ray that finds no admissible intersection (q = 0, a tangency of
 *      measure zero) ends the walk: T = 0 from then on, as T *= q gives.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_MAX_DIM 6
#define OR_MAX_STAR 16
#define OR_MAX_ROOTS 64
#define OR_STAR_SCAN 4096
#define OR_STAR_PANELS 256

#define OR_ELL_ATTEMPTS 64   /* rejection attempts for a uniform point on an ellipsoid; the last one is kept */
#define OR_VR_TRIALS 16      /* uniform trials of the VR start where |dOmega^+/-| has no closed form */

enum { OR_SPHERE = 0, OR_STAR = 1, OR_ELLIPSOID = 2, OR_MESH = 3 };
enum { OR_FLUX_ZERO = 0, OR_FLUX_FOURIER = 1, OR_FLUX_REAL_SH = 2, OR_FLUX_HARMONIC_POLY = 3,
       OR_FLUX_POINT_CHARGE = 4 };
enum { OR_REL_SAME = 0, OR_REL_DESC = 1, OR_REL_OTHER = 2 };

/* Planted-mistake switch.  Only the tests that show that the pins detect
 * plausible errors set it (on the CPU); it is 0 in every other use.
 *   1 uniform transition also multiplies T by the sign (|K*| instead of K*)
 *   2 alpha-sign product over m = 0..i          3 no half weight at i = M
 *   4 no factor N                               5 K* with the normal at the old point
 *   6 beta_i scaled by +2/(sigma_p + sigma_i)   7 line case keeps Q (no 1/2)
 *   8 gradient of Phi with the wrong sign       9 H_0 drawn like H_i (by |alpha|)
 *  10 d >= 3 part sampler without the reflection u -> -u
 *  11 VR start by trials weighs beta by |dOmega| / 2 instead of |dOmega| C_k / K */
static int or_mutant = 0;
void or_set_mutant(int m) { or_mutant = m; }

/* host threads of the estimator over points: n > 0 sets them; returns the count in use */
#ifdef _OPENMP
#include <omp.h>
int or_threads(int n)
{
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
}
#else
int or_threads(int n) { (void)n; return 1; }
#endif

/* Problem description.  All arrays are owned by the caller (oracle.py). */
typedef struct {
    int dim;
    int n_surf;
    const int *type;          /* [n_surf] OR_SPHERE or OR_STAR (star: dim 2 only) */
    const double *center;     /* [n_surf][OR_MAX_DIM] */
    const double *radius;     /* [n_surf] sphere radius, or star base radius R */
    const int *star_K;        /* [n_surf] star Fourier degree */
    const double *star_a;     /* [n_surf][OR_MAX_STAR+1] r = R(1 + sum a_k cos k t + b_k sin k t) */
    const double *star_b;
    const double *star_s;     /* [n_surf][OR_STAR_PANELS+1] arc length at t_j = 2 pi j / panels */
    const double *star_scan;  /* [n_surf][OR_STAR_SCAN+1][2] curve points at t_j = 2 pi j / OR_STAR_SCAN */
    const double *area;       /* [n_surf] |dOmega_i| */
    const int *is_desc;       /* [n_surf*n_surf] is_desc[a*n+b] = 1 iff a is a strict descendant of b */
    const double *alpha;      /* [n_surf] Sec. 3 */
    const double *beta_scale; /* [n_surf] beta_i = beta_scale_i * b_i */
    const uint64_t *thresh;   /* [n_surf] schedule thresholds, thresh[N-1] = 2^32 */
    double alpha_l1;          /* ||alpha||_1 */
    const int *flux_basis;    /* [n_surf] */
    const int *flux_off;      /* [n_surf] offset into flux_coef */
    const int *flux_n;        /* [n_surf] */
    const double *flux_coef;
    const int *arc_off;       /* [n_surf] first arc of the surface (2D variance reduction) */
    const int *arc_n;         /* [n_surf] number of arcs */
    const double *arc_t0;     /* parameter angle where the arc starts */
    const double *arc_t1;     /* parameter angle where the arc ends */
    const int *arc_sign;      /* +1: part of dOmega^+ (beta >= 0), -1: dOmega^- */
    const double *arc_len;
    const double *part_len;   /* [n_surf][2] |dOmega^+|, |dOmega^-| */
    const double *ell_A;      /* [n_surf][OR_MAX_DIM][OR_MAX_DIM] ellipsoid matrix A (row-major) */
    const double *ell_map;    /* [n_surf][OR_MAX_DIM][OR_MAX_DIM] A^{-1/2}: unit sphere -> ellipsoid */
    const double *ell_jmax;   /* [n_surf] sqrt of the largest eigenvalue of A */
    const int *mesh_off;      /* [n_surf] first triangle of a mesh surface */
    const int *mesh_n;        /* [n_surf] number of triangles */
    const double *tri;        /* [n_tri][4][3]: v0, e1 = v1 - v0, e2 = v2 - v0, unit normal (e1 x e2) */
    const uint64_t *tri_thresh; /* [n_tri] cumulative-area thresholds floor(2^32 C_j / A), last = 2^32 */
} or_problem;

typedef struct {
    int M;            /* truncation: steps 0..M */
    int variant;      /* 0 plain (Alg. 2), 1 variance reduced (Alg. 3) */
    int sched_group;  /* walkers per schedule (Alg. 1): 1 or 32 */
} or_opts;

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror, Shaw, "Parallel random numbers:  */
/* as easy as 1, 2, 3", SC'11: ten rounds of two 32x32->64 multiplies with   */
/* the round keys bumped by the Weyl constants between rounds.               */
/* ------------------------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4])
{
    uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
    uint32_t k0 = key_in[0], k1 = key_in[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        c0 = n0; c1 = lo1; c2 = n2; c3 = lo0;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Random-number protocol (the oracle and the library each implement it from this
 * definition; it is not in the paper, which draws its random numbers freely):
 *   key     = (seed_lo ^ point_id, seed_hi ^ instance)
 *   counter = (walk_lo, walk_hi, step, (chain << 4) | sub)      per-walk words
 * Word k of a (step, chain) stream is word k % 4 of sub-call k / 4, except on 2D instances
 * whose surfaces are all circles: a step there draws two words (the schedule word and the
 * angle or arc position), and steps 2j and 2j + 1 share one call, (step j, chain, sub 0),
 * step 2j taking its words 0 and 1 and step 2j + 1 its words 2 and 3.  With a shared
 * schedule (W_g walkers per schedule, Alg. 1) the schedule word of step i of every walk in
 * group g is the one the group's first walk, g W_g, draws for itself. */
typedef struct {
    uint32_t key[2];
    uint64_t walk;
    int cached_step, cached_chain, cached_sub;
    uint32_t words[4];
    int pair2;   /* 2D instance of circles only: two steps per call */
} or_rng;

/* word k of attempt `attempt` of a (step, chain) stream: counter word 3 is
 * (attempt << 9) | (chain << 4) | sub; attempt 0 is the stream itself, later
 * attempts serve rejection sampling */
static uint32_t or_word_at(or_rng *r, int step, int chain, int attempt, int k)
{
    if (r->pair2) {   /* words 0, 1 of step 2j + e are words 2e, 2e + 1 of call j */
        if (attempt != 0 || k > 1) {
            fprintf(stderr, "oracle: word %d (attempt %d) drawn on an instance of circles\n", k, attempt);
            abort();
        }
        k += 2 * (step & 1);
        step >>= 1;
    }
    int sub = (attempt << 5) | (k >> 2);
    if (r->cached_step != step || r->cached_chain != chain || r->cached_sub != sub) {
        uint32_t ctr[4] = {(uint32_t)r->walk, (uint32_t)(r->walk >> 32), (uint32_t)step,
                           ((uint32_t)attempt << 9) | (uint32_t)((chain << 4) | (k >> 2))};
        or_philox4x32_10(ctr, r->key, r->words);
        r->cached_step = step; r->cached_chain = chain; r->cached_sub = sub;
    }
    return r->words[k & 3];
}

static uint32_t or_word(or_rng *r, int step, int chain, int k) { return or_word_at(r, step, chain, 0, k); }

/* uniform on (0,1) from the top 23 bits: (2k+1) / 2^24 with k < 2^23, a value
 * that FP32 and FP64 both represent exactly */
static double or_u01(uint32_t w) { return ((double)(w >> 9) + 0.5) * (1.0 / 8388608.0); }

/* ------------------------------------------------------------------------ */
/* constants and Green's function (Sec. 2)                                   */
/* ------------------------------------------------------------------------ */
static double or_omega(int d) /* surface area of the unit sphere in R^d: d * alpha(d) */
{
    return 2.0 * pow(M_PI, 0.5 * d) / tgamma(0.5 * d);
}

static double or_dist(int d, const double *a, const double *b)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += (a[k] - b[k]) * (a[k] - b[k]);
    return sqrt(s);
}

/* Phi(x,y) = -ln|x-y| / (2 pi) in 2D, |x-y|^{2-d} / (d (d-2) alpha(d)) otherwise */
static double or_phi(int d, const double *x, const double *y)
{
    double r = or_dist(d, x, y);
    if (d == 2) return -log(r) / (2.0 * M_PI);
    return pow(r, 2.0 - d) / ((d - 2) * or_omega(d));
}

/* grad_x Phi(x,y) = -(x - y) / (d alpha(d) |x-y|^d)  (Sec. 4.5) */
static void or_grad_phi(int d, const double *x, const double *y, double *g)
{
    double r = or_dist(d, x, y);
    double c = (or_mutant == 8 ? 1.0 : -1.0) / (or_omega(d) * pow(r, (double)d));
    for (int k = 0; k < d; ++k) g[k] = c * (x[k] - y[k]);
}

/* ------------------------------------------------------------------------ */
/* geometry                                                                  */
/* ------------------------------------------------------------------------ */
static const double *or_center(const or_problem *P, int h) { return P->center + (size_t)h * OR_MAX_DIM; }

/* star radius r(t) and r'(t) */
static void or_star_r(const or_problem *P, int h, double t, double *r, double *dr)
{
    const double *a = P->star_a + (size_t)h * (OR_MAX_STAR + 1);
    const double *b = P->star_b + (size_t)h * (OR_MAX_STAR + 1);
    double R = P->radius[h], s = 1.0, ds = 0.0;
    for (int k = 1; k <= P->star_K[h]; ++k) {
        s += a[k] * cos(k * t) + b[k] * sin(k * t);
        ds += k * (-a[k] * sin(k * t) + b[k] * cos(k * t));
    }
    *r = R * s;
    *dr = R * ds;
}

static void or_star_point(const or_problem *P, int h, double t, double *y)
{
    double r, dr;
    or_star_r(P, h, t, &r, &dr);
    const double *c = or_center(P, h);
    y[0] = c[0] + r * cos(t);
    y[1] = c[1] + r * sin(t);
}

/* |gamma'(t)| and the outward unit normal of the counter-clockwise star */
static double or_star_speed_normal(const or_problem *P, int h, double t, double *n)
{
    double r, dr;
    or_star_r(P, h, t, &r, &dr);
    double tx = dr * cos(t) - r * sin(t);
    double ty = dr * sin(t) + r * cos(t);
    double sp = sqrt(tx * tx + ty * ty);
    if (n) { n[0] = ty / sp; n[1] = -tx / sp; }
    return sp;
}

/* arc length from 0 to t (t in [0, 2 pi]): stored panel sums + 16-point Gauss-Legendre */
static const double or_gl16_x[8] = {0.0950125098376374, 0.2816035507792589, 0.4580167776572274,
                                    0.6178762444026438, 0.7554044083550030, 0.8656312023878318,
                                    0.9445750230732326, 0.9894009349916499};
static const double or_gl16_w[8] = {0.1894506104550685, 0.1826034150449236, 0.1691565193950025,
                                    0.1495959888165767, 0.1246289712555339, 0.0951585116824928,
                                    0.0622535239386479, 0.0271524594117541};

static double or_star_arclen(const or_problem *P, int h, double t)
{
    const double H = 2.0 * M_PI / OR_STAR_PANELS;
    int j = (int)floor(t / H);
    if (j < 0) j = 0;
    if (j >= OR_STAR_PANELS) j = OR_STAR_PANELS - 1;
    double a = j * H, half = 0.5 * (t - a), mid = a + half, s = 0.0;
    for (int q = 0; q < 8; ++q) {
        s += or_gl16_w[q] * (or_star_speed_normal(P, h, mid - half * or_gl16_x[q], NULL) +
                             or_star_speed_normal(P, h, mid + half * or_gl16_x[q], NULL));
    }
    return P->star_s[(size_t)h * (OR_STAR_PANELS + 1) + j] + half * s;
}

/* parameter t in [t_lo, t_hi] with arclen(t) = s, by bisection */
static double or_star_invert(const or_problem *P, int h, double s, double t_lo, double t_hi)
{
    for (int it = 0; it < 200 && t_hi - t_lo > 1e-15; ++it) {
        double m = 0.5 * (t_lo + t_hi);
        if (or_star_arclen(P, h, m) < s) t_lo = m; else t_hi = m;
    }
    return 0.5 * (t_lo + t_hi);
}

static double or_param_angle(const or_problem *P, int h, const double *y)
{
    const double *c = or_center(P, h);
    double t = atan2(y[1] - c[1], y[0] - c[0]);
    if (t < 0) t += 2.0 * M_PI;
    return t;
}

/* outward unit normal at a point y of surface h (on a mesh: of triangle `tri`) */
static void or_normal(const or_problem *P, int h, int tri, const double *y, double *n)
{
    int d = P->dim;
    if (P->type[h] == OR_MESH) {
        const double *t = P->tri + (size_t)tri * 12;
        for (int k = 0; k < 3; ++k) n[k] = t[9 + k];
        return;
    }
    if (P->type[h] == OR_SPHERE) {
        const double *c = or_center(P, h);
        for (int k = 0; k < d; ++k) n[k] = (y[k] - c[k]) / P->radius[h];
    } else if (P->type[h] == OR_ELLIPSOID) {
        /* grad of (y - c)^T A (y - c) is 2 A (y - c) */
        const double *c = or_center(P, h), *A = P->ell_A + (size_t)h * OR_MAX_DIM * OR_MAX_DIM;
        double nn = 0.0;
        for (int k = 0; k < d; ++k) {
            n[k] = 0.0;
            for (int j = 0; j < d; ++j) n[k] += A[k * OR_MAX_DIM + j] * (y[j] - c[j]);
            nn += n[k] * n[k];
        }
        nn = sqrt(nn);
        for (int k = 0; k < d; ++k) n[k] /= nn;
    } else {
        or_star_speed_normal(P, h, or_param_angle(P, h, y), n);
    }
}

/* index of the word that picks one of q intersections (and, on an ellipsoid,
 * decides a rejection attempt: a uniform transition makes no pick) */
static int or_choice_word(int d) { return d == 2 ? 2 : (d == 3 ? 3 : (d == 4 ? 5 : 7)); }

/* isotropic unit direction from the words 1.. of attempt `a` of a (step, chain) stream */
static void or_direction_at(or_rng *r, int d, int step, int chain, int a, double *z)
{
    if (d == 2) {
        double phi = 2.0 * M_PI * or_u01(or_word_at(r, step, chain, a, 1));
        z[0] = cos(phi); z[1] = sin(phi);
        return;
    }
    if (d == 3) {
        double zz = 1.0 - 2.0 * or_u01(or_word_at(r, step, chain, a, 1));
        double phi = 2.0 * M_PI * or_u01(or_word_at(r, step, chain, a, 2));
        double rho = sqrt(1.0 - zz * zz);
        z[0] = rho * cos(phi); z[1] = rho * sin(phi); z[2] = zz;
        return;
    }
    /* d >= 4: Box-Muller on pairs of words (1,2), (3,4), (5,6), then normalise */
    double g[OR_MAX_DIM + 1], nrm = 0.0;
    for (int j = 0; 2 * j < d; ++j) {
        double ua = or_u01(or_word_at(r, step, chain, a, 1 + 2 * j));
        double ub = or_u01(or_word_at(r, step, chain, a, 2 + 2 * j));
        double rho = sqrt(-2.0 * log(ua));
        g[2 * j] = rho * cos(2.0 * M_PI * ub);
        g[2 * j + 1] = rho * sin(2.0 * M_PI * ub);
    }
    for (int k = 0; k < d; ++k) nrm += g[k] * g[k];
    nrm = sqrt(nrm);
    for (int k = 0; k < d; ++k) z[k] = g[k] / nrm;
}

static void or_direction(or_rng *r, int d, int step, int chain, double *z) { or_direction_at(r, d, step, chain, 0, z); }


/* uniform point on dOmega_h (Eq. naive_woi_p0; by surface measure); on a mesh
 * *tri receives the triangle (word 1 picks it by area, words 2 and 3 give
 * uniform barycentric coordinates (1 - s, s (1 - w), s w) with s = sqrt(u)) */
static void or_uniform_point(const or_problem *P, int h, or_rng *r, int step, int chain, double *y, int *tri)
{
    int d = P->dim;
    *tri = -1;
    if (P->type[h] == OR_MESH) {
        uint32_t w1 = or_word(r, step, chain, 1);
        int lo = P->mesh_off[h], hi = P->mesh_off[h] + P->mesh_n[h] - 1, j = hi;
        for (int k = lo; k <= hi; ++k)            /* first triangle whose threshold exceeds the word */
            if ((uint64_t)w1 < P->tri_thresh[k]) { j = k; break; }
        double u = or_u01(or_word(r, step, chain, 2)), w = or_u01(or_word(r, step, chain, 3));
        double sq = sqrt(u), b1 = sq * (1.0 - w), b2 = sq * w;
        const double *t = P->tri + (size_t)j * 12;
        for (int k = 0; k < 3; ++k) y[k] = t[k] + b1 * t[3 + k] + b2 * t[6 + k];
        *tri = j;
        return;
    }
    if (P->type[h] == OR_SPHERE) {
        double z[OR_MAX_DIM];
        or_direction(r, d, step, chain, z);
        const double *c = or_center(P, h);
        for (int k = 0; k < d; ++k) y[k] = c[k] + P->radius[h] * z[k];
    } else if (P->type[h] == OR_ELLIPSOID) {
        /* u uniform on the unit sphere, accepted when v^2 max J^2 <= J(u)^2 with v the
         * attempt's choice word and J(u)^2 = u^T A u */
        const double *c = or_center(P, h), *Mp = P->ell_map + (size_t)h * OR_MAX_DIM * OR_MAX_DIM;
        const double *A = P->ell_A + (size_t)h * OR_MAX_DIM * OR_MAX_DIM, jm = P->ell_jmax[h];
        double z[OR_MAX_DIM];
        for (int a = 0; a < OR_ELL_ATTEMPTS; ++a) {
            or_direction_at(r, d, step, chain, a, z);
            double J2 = 0.0;
            for (int k = 0; k < d; ++k)
                for (int j = 0; j < d; ++j) J2 += z[k] * A[k * OR_MAX_DIM + j] * z[j];
            double v = or_u01(or_word_at(r, step, chain, a, or_choice_word(d)));
            if (v * v * jm * jm <= J2) break;
        }
        for (int k = 0; k < d; ++k) {
            y[k] = c[k];
            for (int j = 0; j < d; ++j) y[k] += Mp[k * OR_MAX_DIM + j] * z[j];
        }
    } else {
        double s = or_u01(or_word(r, step, chain, 1)) * P->area[h];
        double t = or_star_invert(P, h, s, 0.0, 2.0 * M_PI);
        or_star_point(P, h, t, y);
    }
}

/* uniform point on dOmega_h^+ (part = 0) or dOmega_h^- (part = 1): the arcs of
 * the requested sign are concatenated in increasing parameter angle */
static double or_flux(const or_problem *P, int h, int tri, const double *y);

/* |grad_y b_h(y)| by central differences of the flux as it is evaluated off the surface too
 * (error bound of the tests only: how fast b_h changes when its point moves) */
static double or_flux_grad_mag(const or_problem *P, int h, int tri, const double *y)
{
    const int d = P->dim;
    const double *c = or_center(P, h);
    double r = 0.0;
    for (int k = 0; k < d; ++k) r += (y[k] - c[k]) * (y[k] - c[k]);
    const double step = 1e-6 * fmax(sqrt(r), 1e-3);
    double g2 = 0.0;
    for (int k = 0; k < d; ++k) {
        double yp[OR_MAX_DIM], ym[OR_MAX_DIM];
        for (int j = 0; j < d; ++j) yp[j] = ym[j] = y[j];
        yp[k] += step;
        ym[k] -= step;
        const double g = (or_flux(P, h, tri, yp) - or_flux(P, h, tri, ym)) / (2.0 * step);
        g2 += g * g;
    }
    return sqrt(g2);
}

static double or_beta(const or_problem *P, int h, int tri, const double *y);

static void or_uniform_part_point(const or_problem *P, int h, int part, or_rng *r, int step, int chain,
                                  double *y)
{
    if (P->dim >= 3) {
        /* a sphere whose data is linear in the unit vector u (degree-1 harmonics, linear
         * harmonic polynomials): the parts beta >= 0 and beta < 0 are the two hemispheres
         * {beta(u) >= 0} and its mirror image, so a uniform u that lands in the wrong one
         * is reflected, u -> -u, which keeps it uniform on the right one */
        double z[OR_MAX_DIM];
        const double *c = or_center(P, h);
        or_direction(r, P->dim, step, chain, z);
        for (int k = 0; k < P->dim; ++k) y[k] = c[k] + P->radius[h] * z[k];
        const double b = or_beta(P, h, -1, y);
        if ((part == 0) != (b >= 0.0) && or_mutant != 10)
            for (int k = 0; k < P->dim; ++k) y[k] = c[k] - P->radius[h] * z[k];
        return;
    }
    double s = or_u01(or_word(r, step, chain, 1)) * P->part_len[2 * h + part];
    int want = part == 0 ? 1 : -1, last = -1;
    for (int a = P->arc_off[h]; a < P->arc_off[h] + P->arc_n[h]; ++a) {
        if (P->arc_sign[a] != want) continue;
        last = a;
        if (s < P->arc_len[a]) break;
        s -= P->arc_len[a];
    }
    int a = last;
    if (s > P->arc_len[a]) s = P->arc_len[a];
    double t;
    if (P->type[h] == OR_SPHERE) {
        t = P->arc_t0[a] + s / P->radius[h];
        const double *c = or_center(P, h);
        y[0] = c[0] + P->radius[h] * cos(t);
        y[1] = c[1] + P->radius[h] * sin(t);
    } else {
        double s0 = or_star_arclen(P, h, P->arc_t0[a]);
        t = or_star_invert(P, h, s0 + s, P->arc_t0[a], P->arc_t1[a]);
        or_star_point(P, h, t, y);
    }
}

/* intersections y + t z of the line (ray = 0) or ray (ray = 1) with dOmega_h.
 * Line: t != 0 (the start point itself is excluded), ray: t > 0.  Returns q
 * and the parameters sorted increasingly. */
static int or_intersections(const or_problem *P, int h, const double *y, const double *z, int ray,
                            double *ts, int exclude, int *hit_tri)
{
    int d = P->dim, q = 0;
    const double tiny = 1e-9;
    if (P->type[h] == OR_MESH) {
        /* every triangle (Moller-Trumbore: y + t z = v0 + a e1 + b e2, a, b >= 0, a + b <= 1) */
        for (int j = P->mesh_off[h]; j < P->mesh_off[h] + P->mesh_n[h]; ++j) {
            if (j == exclude) continue;
            const double *T = P->tri + (size_t)j * 12, *e1 = T + 3, *e2 = T + 6;
            double p[3] = {z[1] * e2[2] - z[2] * e2[1], z[2] * e2[0] - z[0] * e2[2], z[0] * e2[1] - z[1] * e2[0]};
            double det = e1[0] * p[0] + e1[1] * p[1] + e1[2] * p[2];
            if (det == 0.0) continue;
            double sv[3] = {y[0] - T[0], y[1] - T[1], y[2] - T[2]};
            double a = (sv[0] * p[0] + sv[1] * p[1] + sv[2] * p[2]) / det;
            if (a < 0.0 || a > 1.0) continue;
            double qv[3] = {sv[1] * e1[2] - sv[2] * e1[1], sv[2] * e1[0] - sv[0] * e1[2], sv[0] * e1[1] - sv[1] * e1[0]};
            double b = (z[0] * qv[0] + z[1] * qv[1] + z[2] * qv[2]) / det;
            if (b < 0.0 || a + b > 1.0) continue;
            double t = (e2[0] * qv[0] + e2[1] * qv[1] + e2[2] * qv[2]) / det;
            if (ray && !(t > 0.0)) continue;
            if (q < OR_MAX_ROOTS) { ts[q] = t; hit_tri[q] = j; ++q; }
        }
        for (int a = 1; a < q; ++a) {            /* insertion sort by t, triangles alongside */
            double v = ts[a];
            int tv = hit_tri[a], b = a - 1;
            while (b >= 0 && ts[b] > v) { ts[b + 1] = ts[b]; hit_tri[b + 1] = hit_tri[b]; --b; }
            ts[b + 1] = v;
            hit_tri[b + 1] = tv;
        }
        return q;
    }
    if (P->type[h] == OR_SPHERE) {
        const double *c = or_center(P, h);
        double b = 0.0, c0 = 0.0, R = P->radius[h];
        for (int k = 0; k < d; ++k) {
            b += z[k] * (y[k] - c[k]);
            c0 += (y[k] - c[k]) * (y[k] - c[k]);
        }
        if (!ray) {
            /* a line through y on the sphere: |y + t z - c|^2 = R^2 with |y - c| = R leaves
             * t (t + 2 b) = 0, so the one intersection distinct from y is t = -2 b (the
             * reflection of y - c in the plane normal to z) */
            double t = -2.0 * b;
            if (fabs(t) > tiny * R) ts[q++] = t;
            return q;
        }
        c0 -= R * R;
        double disc = b * b - c0;
        if (disc < 0.0) return 0;
        double sq = sqrt(disc);
        double qq = -(b + (b >= 0 ? sq : -sq));     /* stable quadratic roots */
        double r1 = qq, r2 = (qq != 0.0) ? c0 / qq : 0.0;
        double cand[2] = {r1 < r2 ? r1 : r2, r1 < r2 ? r2 : r1};
        for (int j = 0; j < 2; ++j) {
            double t = cand[j];
            if (ray ? (t > tiny * R) : (fabs(t) > tiny * R)) ts[q++] = t;
        }
        return q;
    }
    if (P->type[h] == OR_ELLIPSOID) {
        /* (dy + t z)^T A (dy + t z) = 1: a2 t^2 + 2 b1 t + c0 = 0 */
        const double *c = or_center(P, h), *A = P->ell_A + (size_t)h * OR_MAX_DIM * OR_MAX_DIM;
        double dy[OR_MAX_DIM], a2 = 0.0, b1 = 0.0, c0 = -1.0;
        for (int k = 0; k < d; ++k) dy[k] = y[k] - c[k];
        for (int k = 0; k < d; ++k)
            for (int j = 0; j < d; ++j) {
                double Akj = A[k * OR_MAX_DIM + j];
                a2 += z[k] * Akj * z[j];
                b1 += z[k] * Akj * dy[j];
                c0 += dy[k] * Akj * dy[j];
            }
        if (!ray) {
            /* a line through y on the ellipsoid: c0 = 0 there, so a2 t^2 + 2 b1 t = 0 and the
             * intersection distinct from y is t = -2 b1 / a2 */
            double t = -2.0 * b1 / a2;
            if (fabs(t) > tiny / P->ell_jmax[h]) ts[q++] = t;
            return q;
        }
        double disc = b1 * b1 - a2 * c0;
        if (disc < 0.0) return 0;
        double sq = sqrt(disc);
        double qq = -(b1 + (b1 >= 0 ? sq : -sq));
        double r1 = qq / a2, r2 = (qq != 0.0) ? c0 / qq : 0.0;
        double cand[2] = {r1 < r2 ? r1 : r2, r1 < r2 ? r2 : r1};
        double scale = 1.0 / P->ell_jmax[h];      /* shortest semi-axis */
        for (int j = 0; j < 2; ++j) {
            double t = cand[j];
            if (ray ? (t > tiny * scale) : (fabs(t) > tiny * scale)) ts[q++] = t;
        }
        return q;
    }
    /* star: roots in the parameter angle of f(t) = cross(gamma(t) - y, z) = 0,
     * by a dense sign scan and bisection, then the line parameter of each root.
     * Ray from an interior point: scan f over [0, 2 pi].
     * Line through y = gamma(t_y) on the curve: f vanishes at t_y itself; scan
     * g(t) = f(t) / sin((t - t_y) / 2) over the open range (t_y, t_y + 2 pi),
     * where sin > 0, g has exactly the other roots of f, and g tends to
     * 2 f'(t_y) and -2 f'(t_y) at the two ends.  An intersection within one
     * scan step of y (a near-tangent line) is therefore not lost. */
    const double *scan = P->star_scan + (size_t)h * (OR_STAR_SCAN + 1) * 2;
    double pt[2];
    const double H = 2.0 * M_PI / OR_STAR_SCAN;
    if (ray) {
        double f_prev = 0.0, t_prev = 0.0;
        for (int j = 0; j <= OR_STAR_SCAN; ++j) {
            double th = H * j;
            double f = (scan[2 * j] - y[0]) * z[1] - (scan[2 * j + 1] - y[1]) * z[0];
            if (j > 0 && ((f_prev < 0.0) != (f < 0.0))) {
                double lo = t_prev, hi = th, flo = f_prev;
                for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
                    double m = 0.5 * (lo + hi);
                    or_star_point(P, h, m, pt);
                    double fm = (pt[0] - y[0]) * z[1] - (pt[1] - y[1]) * z[0];
                    if ((fm < 0.0) == (flo < 0.0)) { lo = m; flo = fm; } else hi = m;
                }
                or_star_point(P, h, 0.5 * (lo + hi), pt);
                double t = (pt[0] - y[0]) * z[0] + (pt[1] - y[1]) * z[1];
                if (t > tiny && q < OR_MAX_ROOTS) ts[q++] = t;
            }
            f_prev = f; t_prev = th;
        }
    } else {
        const double ty = or_param_angle(P, h, y);
        double r, dr;
        or_star_r(P, h, ty, &r, &dr);
        const double gx = dr * cos(ty) - r * sin(ty), gy = dr * sin(ty) + r * cos(ty);
        const double fpy = gx * z[1] - gy * z[0];      /* f'(t_y) */
        const int jy = (int)floor(ty / H);
        double g_prev = 2.0 * fpy, t_prev = ty;
        for (int k = 1; k <= OR_STAR_SCAN + 1; ++k) {
            double th, g;
            if (k <= OR_STAR_SCAN) {
                th = H * (jy + k);                      /* unwrapped angle in (t_y, t_y + 2 pi] */
                if (th >= ty + 2.0 * M_PI) continue;
                int j = (jy + k) % OR_STAR_SCAN;
                double f = (scan[2 * j] - y[0]) * z[1] - (scan[2 * j + 1] - y[1]) * z[0];
                g = f / sin(0.5 * (th - ty));
            } else {
                th = ty + 2.0 * M_PI;                   /* the limit at the far end */
                g = -2.0 * fpy;
            }
            if ((g_prev < 0.0) != (g < 0.0)) {
                double lo = t_prev, hi = th, glo = g_prev;
                for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
                    double m = 0.5 * (lo + hi);
                    or_star_point(P, h, m, pt);
                    double gm = ((pt[0] - y[0]) * z[1] - (pt[1] - y[1]) * z[0]) / sin(0.5 * (m - ty));
                    if ((gm < 0.0) == (glo < 0.0)) { lo = m; glo = gm; } else hi = m;
                }
                or_star_point(P, h, 0.5 * (lo + hi), pt);
                double t = (pt[0] - y[0]) * z[0] + (pt[1] - y[1]) * z[1];
                if (fabs(t) > tiny && q < OR_MAX_ROOTS) ts[q++] = t;
            }
            g_prev = g; t_prev = th;
        }
    }
    /* insertion sort by t */
    for (int a = 1; a < q; ++a) {
        double v = ts[a];
        int b = a - 1;
        while (b >= 0 && ts[b] > v) { ts[b + 1] = ts[b]; --b; }
        ts[b + 1] = v;
    }
    return q;
}

/* ------------------------------------------------------------------------ */
/* boundary data b_i and beta_i (Sec. 1, Sec. 3)                             */
/* ------------------------------------------------------------------------ */

/* orthonormal real spherical harmonic Y_l^m at a unit vector u (3D), with
 * the convention sin(phi) cos(theta) = sqrt(4 pi / 3) Y_1^1 (Example 3, 3D):
 * no Condon-Shortley phase, theta azimuth, phi polar. */
static double or_real_sh(int l, int m, const double *u)
{
    int am = m < 0 ? -m : m;
    double x = u[2];                       /* cos(phi) */
    double sx = sqrt(fmax(0.0, 1.0 - x * x));
    double pmm = 1.0;                      /* P_am^am without the (-1)^m phase */
    for (int k = 1; k <= am; ++k) pmm *= (2.0 * k - 1.0) * sx;
    double plm;
    if (l == am) {
        plm = pmm;
    } else {
        double p1 = x * (2.0 * am + 1.0) * pmm, p0 = pmm;
        plm = p1;
        for (int ll = am + 2; ll <= l; ++ll) {
            plm = ((2.0 * ll - 1.0) * x * p1 - (ll + am - 1.0) * p0) / (ll - am);
            p0 = p1; p1 = plm;
        }
    }
    double ratio = 1.0;                    /* (l-am)! / (l+am)! */
    for (int k = l - am + 1; k <= l + am; ++k) ratio /= k;
    double nlm = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * ratio);
    double az = atan2(u[1], u[0]);
    if (m == 0) return nlm * plm;
    if (m > 0) return sqrt(2.0) * nlm * plm * cos(am * az);
    return sqrt(2.0) * nlm * plm * sin(am * az);
}

/* flux datum b_h(y) at a point y of dOmega_h */
static double or_flux(const or_problem *P, int h, int tri, const double *y)
{
    int d = P->dim, n = P->flux_n[h];
    const double *c = P->flux_coef + P->flux_off[h];
    switch (P->flux_basis[h]) {
    case OR_FLUX_FOURIER: { /* [a0, a1, b1, ..., aK, bK] in the local parameter angle */
        double t = (P->type[h] == OR_SPHERE)
                       ? atan2(y[1] - or_center(P, h)[1], y[0] - or_center(P, h)[0])
                       : or_param_angle(P, h, y);
        double v = c[0];
        for (int k = 1; 2 * k <= n - 1; ++k) v += c[2 * k - 1] * cos(k * t) + c[2 * k] * sin(k * t);
        return v;
    }
    case OR_FLUX_REAL_SH: { /* coef[l*l + l + m] */
        double u[3];
        const double *cc = or_center(P, h);
        for (int k = 0; k < 3; ++k) u[k] = (y[k] - cc[k]) / P->radius[h];
        double nn = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int k = 0; k < 3; ++k) u[k] /= nn;
        double v = 0.0;
        for (int idx = 0; idx < n; ++idx) {
            if (c[idx] == 0.0) continue;
            int l = (int)floor(sqrt((double)idx) + 1e-9);
            int m = idx - l * l - l;
            v += c[idx] * or_real_sh(l, m, u);
        }
        return v;
    }
    case OR_FLUX_HARMONIC_POLY: { /* [s, T, (c, e_1..e_d) x T]: b = s n . grad P */
        double s = c[0];
        int T = (int)c[1];
        double nrm[OR_MAX_DIM], grad[OR_MAX_DIM] = {0};
        or_normal(P, h, tri, y, nrm);
        for (int t = 0; t < T; ++t) {
            const double *row = c + 2 + t * (d + 1);
            for (int k = 0; k < d; ++k) {
                int ek = (int)row[1 + k];
                if (ek == 0) continue;
                double term = row[0] * ek;
                for (int j = 0; j < d; ++j) {
                    int e = (int)row[1 + j] - (j == k ? 1 : 0);
                    for (int p = 0; p < e; ++p) term *= y[j];
                }
                grad[k] += term;
            }
        }
        double v = 0.0;
        for (int k = 0; k < d; ++k) v += nrm[k] * grad[k];
        return s * v;
    }
    case OR_FLUX_POINT_CHARGE: { /* [s, x0_1..x0_d]: b = s n . grad_y |y - x0|^{2-d} (d >= 3) */
        double nrm[OR_MAX_DIM], r2 = 0.0, dot = 0.0;
        or_normal(P, h, tri, y, nrm);
        for (int k = 0; k < d; ++k) {
            double e = y[k] - c[1 + k];
            r2 += e * e;
            dot += e * nrm[k];
        }
        return c[0] * (2.0 - d) * pow(r2, -0.5 * d) * dot;
    }
    default:
        return 0.0;
    }
}

/* sum of the magnitudes of the terms that make up b_h(y): the scale against
 * which the rounding error of evaluating b_h is measured in the tests */
static double or_flux_mag(const or_problem *P, int h, int tri, const double *y)
{
    int d = P->dim, n = P->flux_n[h];
    const double *c = P->flux_coef + P->flux_off[h];
    double m = 0.0;
    switch (P->flux_basis[h]) {
    case OR_FLUX_FOURIER:
        for (int k = 0; k < n; ++k) m += fabs(c[k]);
        return m;
    case OR_FLUX_REAL_SH: {
        double u[3];
        const double *cc = or_center(P, h);
        for (int k = 0; k < 3; ++k) u[k] = (y[k] - cc[k]) / P->radius[h];
        double nn = sqrt(u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
        for (int k = 0; k < 3; ++k) u[k] /= nn;
        for (int idx = 0; idx < n; ++idx) {
            if (c[idx] == 0.0) continue;
            int l = (int)floor(sqrt((double)idx) + 1e-9);
            m += fabs(c[idx] * or_real_sh(l, idx - l * l - l, u));
        }
        return m;
    }
    case OR_FLUX_HARMONIC_POLY: {
        int T = (int)c[1];
        double nrm[OR_MAX_DIM];
        or_normal(P, h, tri, y, nrm);
        for (int t = 0; t < T; ++t) {
            const double *row = c + 2 + t * (d + 1);
            for (int k = 0; k < d; ++k) {
                int ek = (int)row[1 + k];
                if (ek == 0) continue;
                double term = row[0] * ek;
                for (int j = 0; j < d; ++j) {
                    int e = (int)row[1 + j] - (j == k ? 1 : 0);
                    for (int p = 0; p < e; ++p) term *= fabs(y[j]);
                }
                m += fabs(term * nrm[k]);
            }
        }
        return fabs(c[0]) * m;
    }
    case OR_FLUX_POINT_CHARGE: {
        double nrm[OR_MAX_DIM], r2 = 0.0;
        or_normal(P, h, tri, y, nrm);
        for (int k = 0; k < d; ++k) r2 += (y[k] - c[1 + k]) * (y[k] - c[1 + k]);
        for (int k = 0; k < d; ++k) m += fabs((y[k] - c[1 + k]) * nrm[k]);
        return fabs(c[0] * (2.0 - d)) * pow(r2, -0.5 * d) * m;
    }
    default:
        return 0.0;
    }
}

static double or_beta(const or_problem *P, int h, int tri, const double *y)
{
    double sc = P->beta_scale[h];
    if (or_mutant == 6 && h > 0) sc = -sc;
    return sc * or_flux(P, h, tri, y);
}

/* ------------------------------------------------------------------------ */
/* one walk (Algorithm 2; Algorithm 3 when variant = 1)                      */
/* ------------------------------------------------------------------------ */
typedef struct {
    int *H;          /* [M+1] scheduled interfaces (0-based), or NULL */
    double *Y;       /* [2][M+1][dim] states of each chain, or NULL */
    double *scale;   /* [4], see the error bound below: B_u, B_g, the walk's conditioning
                        (largest running amplification of a state error by line / ray steps) and
                        the largest ratio (sum of the magnitudes of the start flux's terms) / |flux| */
    double *QT;      /* [2][M+1][2]: Q_i and T_i of each chain, or NULL */
    double *E;       /* [2][M+1][2]: the error bounds e_i of y_i and Qe_i of Q_i (units of u), or NULL */
} or_trace;

/* Per-walk first-order error bound (test tolerance, not part of the estimator).
 * A computation of the same walk whose every operation is rounded with unit
 * roundoff u differs from the exact one by at most about u B_u in the u tally and
 * u B_g in the gradient tally, where, summed over the tallied states of both chains,
 *   B_u = sum |C_i T_i| [ Qe_i (|Phi_i| + 1) + |Q_i| (|Phi_i| + 1 + |grad Phi_i| (e_i + r_x)) ]
 *   B_g = sum |C_i T_i| [ Qe_i |grad Phi_i| + |Q_i| (|grad Phi_i| + |D2 Phi_i| (e_i + r_x)) ]
 * with C_i = N w_i ||alpha||_1^i prod sign(alpha), |D2 Phi| = (d - 1) / (omega_d r^d) the norm of
 * the Hessian of Phi, r_x = |x - c_s| (x is rounded relative to the state's surface centre),
 * and, in units of u:
 *   e_i   a bound on the error of the state y_i: |y - c_s| for a fresh sample (start, uniform
 *         transition); a reflection chord (line on a sphere or ellipsoid, t = -2 b) adds
 *         |y' - c|; a line or ray whose intersection is found as a root multiplies the
 *         incoming error by 1 + 1 / |n(y') . z| (moving the line by delta moves a crossing
 *         at angle acos|n . z| to the normal by delta / |n . z| along it) and adds |y' - c|;
 *   Qe_i  a bound on the error of Q_i: the start flux contributes |beta scale| (sum of the
 *         magnitudes of its terms + |grad b| e_0) |part|, a uniform transition the first-order
 *         change of K*(y', y) under the errors of y, y' and of the normal at y', a line step
 *         halves it.
 * The walk's conditioning is the largest product of root-step amplifications since the
 * last fresh sample. */
static int or_mutant_bound = 0;  /* test hook: 1 drops the states' term from the bound */
void or_set_mutant_bound(int m) { or_mutant_bound = m; }

/* Test hook: every new walk state y on surface s is moved by or_perturb |y - c_s| and the
 * evaluation point by or_perturb |x - c_s| in each tally (a stand-in for rounding, in a
 * pseudo-random direction), so that a test can compare the change of the tallies with the
 * bound above.  0 (the default) leaves the walk exact. */
static double or_perturb = 0.0;
void or_set_perturb(double rel) { or_perturb = rel; }

static void or_perturb_vec(int d, uint64_t walk, int i, int k, int tag, double mag, double *v)
{
    uint64_t z = (walk + 1) * 0x9E3779B97F4A7C15ull + (uint64_t)(i * 64 + k * 8 + tag + 1) * 0xBF58476D1CE4E5B9ull;
    z ^= z >> 31;
    z *= 0x94D049BB133111EBull;
    z ^= z >> 29;
    const double s = mag / sqrt((double)d);
    for (int c = 0; c < d; ++c) v[c] += ((z >> (3 * c)) & 1) ? s : -s;
}

static double or_norm_rel(int d, const double *y, const double *c)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += (y[k] - c[k]) * (y[k] - c[k]);
    return sqrt(s);
}

/* H_i: 0-based index; i = 0 uniform over the N surfaces, i >= 1 by |alpha| */
static int or_schedule_from_word(const or_problem *P, int i, uint32_t w)
{
    if (i == 0 && or_mutant != 9) return (int)(((uint64_t)w * (uint64_t)P->n_surf) >> 32);
    for (int n = 0; n < P->n_surf; ++n)
        if ((uint64_t)w < P->thresh[n]) return n;
    return P->n_surf - 1;
}

static int or_relation(const or_problem *P, int prev, int cur)
{
    if (prev == cur) return OR_REL_SAME;
    if (P->is_desc[prev * P->n_surf + cur]) return OR_REL_DESC;
    return OR_REL_OTHER;
}

void or_walk(const or_problem *P, const or_opts *o, const double *x, uint32_t point_id, uint32_t instance,
             uint64_t walk, uint64_t seed, double *out_u, double *out_g, or_trace *tr)
{
    const int d = P->dim, M = o->M, N = P->n_surf;
    const int n_chain = o->variant == 1 ? 2 : 1;
    or_rng rng = {{(uint32_t)seed ^ point_id, (uint32_t)(seed >> 32) ^ instance}, walk, -1, -1, -1, {0}, 0};
    if (d == 2) {
        rng.pair2 = 1;
        for (int s = 0; s < N; ++s)
            if (P->type[s] != OR_SPHERE) rng.pair2 = 0;
    }
    uint64_t group = walk / (uint64_t)o->sched_group;
    double acc_u = 0.0, acc_g[OR_MAX_DIM] = {0};

    double y[2][OR_MAX_DIM], Q[2], T[2];
    double Qe[2] = {0.0, 0.0}, ey[2] = {0.0, 0.0}, amp[2] = {1.0, 1.0};   /* error bound, see above */
    double B_u = 0.0, B_g = 0.0, cond = 1.0, flux_ratio = 1.0;
    int alive[2] = {1, 1};
    int tri[2] = {-1, -1};   /* mesh triangle of each chain's state (-1 elsewhere) */
    int trial_n[2] = {0, 0}, trial_tri[2] = {-1, -1};   /* VR start by uniform trials */
    double trial_y[2][OR_MAX_DIM] = {{0}};
    double S = 1.0;          /* prod_{m=1}^{i} sign(alpha_{H_m}): alpha_{H_0} never enters the expansion */
    double Ai = 1.0;         /* ||alpha||_1^i */
    int h_prev = -1;
    const double omega = or_omega(d);

    for (int i = 0; i <= M; ++i) {
        const double weight = (i == M && or_mutant != 3) ? 0.5 : 1.0; /* w_i = 1 - delta_{iM}/2 */
        uint32_t hw;
        if (o->sched_group == 1) {
            hw = or_word(&rng, i, 0, 0);
        } else {   /* the group's first walk's own schedule word */
            or_rng first = rng;
            first.walk = group * (uint64_t)o->sched_group;
            first.cached_step = -1;
            hw = or_word(&first, i, 0, 0);
        }
        const int h = or_schedule_from_word(P, i, hw);
        if (tr && tr->H) tr->H[i] = h;
        const double *ch = or_center(P, h);

        if (i > 0 || or_mutant == 2) {
            if (i > 0) Ai *= P->alpha_l1;
            S *= (P->alpha[h] > 0.0) ? 1.0 : ((P->alpha[h] < 0.0) ? -1.0 : 0.0);
        }

        for (int k = 0; k < n_chain; ++k) {
            if (i == 0) {
                /* p0: uniform on dOmega_{h0} (plain) or on dOmega^{+/-} (Alg. 3) */
                T[k] = 1.0;
                double L = P->area[h];
                int start = 1;
                if (o->variant == 0) {
                    or_uniform_point(P, h, &rng, 0, k, y[k], &tri[k]);
                } else if (P->part_len[2 * h] < 0.0) {
                    /* parts of no closed form: K uniform trials on dOmega_h, shared by
                     * both chains (trial t draws the step-0 words of chain id t << 12).  Chain k starts
                     * at the first trial of its sign and weighs beta by |dOmega| C_k / K, C_k the
                     * trials of that sign: C_k / K is an unbiased estimate of |dOmega^+/-| / |dOmega|,
                     * independent of where the first trial of that sign lies */
                    if (k == 0) {
                        trial_n[0] = trial_n[1] = 0;
                        for (int t = 0; t < OR_VR_TRIALS; ++t) {
                            double yt[OR_MAX_DIM];
                            int tt;
                            or_uniform_point(P, h, &rng, 0, t << 12, yt, &tt);
                            const int part = or_beta(P, h, tt, yt) >= 0.0 ? 0 : 1;
                            if (trial_n[part]++ == 0) {
                                for (int c = 0; c < d; ++c) trial_y[part][c] = yt[c];
                                trial_tri[part] = tt;
                            }
                        }
                    }
                    if (trial_n[k] == 0 || P->flux_basis[h] == OR_FLUX_ZERO) {
                        alive[k] = 0; Q[k] = 0.0; start = 0;
                        for (int c = 0; c < d; ++c) y[k][c] = 0.0;
                    } else {
                        for (int c = 0; c < d; ++c) y[k][c] = trial_y[k][c];
                        tri[k] = trial_tri[k];
                        L *= or_mutant == 11 ? 0.5 : (double)trial_n[k] / OR_VR_TRIALS;
                    }
                } else {
                    L = P->part_len[2 * h + k];
                    if (L <= 0.0 || P->flux_basis[h] == OR_FLUX_ZERO) {
                        /* empty part, or beta = 0 on the whole surface: the chain carries no weight */
                        alive[k] = 0; Q[k] = 0.0; start = 0;
                        for (int c = 0; c < d; ++c) y[k][c] = 0.0;
                    } else {
                        or_uniform_part_point(P, h, k, &rng, 0, k, y[k]);
                        tri[k] = -1;
                    }
                }
                if (start) {
                    const double ry = or_norm_rel(d, y[k], ch);
                    if (or_perturb > 0.0) or_perturb_vec(d, walk, i, k, 0, or_perturb * ry, y[k]);
                    Q[k] = or_beta(P, h, tri[k], y[k]) * L;
                    const double b0 = fabs(or_flux(P, h, tri[k], y[k])), bm = or_flux_mag(P, h, tri[k], y[k]);
                    if (b0 > 0.0 && bm / b0 > flux_ratio) flux_ratio = bm / b0;
                    /* the flux's rounding (its terms' magnitudes) and its change under the
                     * start's own error |y - c_h| */
                    Qe[k] = fabs(P->beta_scale[h]) * (bm + or_flux_grad_mag(P, h, tri[k], y[k]) * ry) * L;
                    ey[k] = ry;
                    amp[k] = 1.0;
                }
            } else if (alive[k]) {
                const int rel = or_relation(P, h_prev, h);
                const double dc = or_dist(d, or_center(P, h_prev), ch);   /* centres: rounding of y - c_h */
                double ynew[OR_MAX_DIM];
                int tnew = -1;
                if (rel == OR_REL_OTHER) {
                    /* uniform on dOmega_h; Q *= K*(y_i, y_{i-1}) |dOmega_h| with the normal at the new
                     * point; T unchanged (the sign is already in K*) */
                    or_uniform_point(P, h, &rng, i, k, ynew, &tnew);
                    const double rn = or_norm_rel(d, ynew, ch);
                    if (or_perturb > 0.0) or_perturb_vec(d, walk, i, k, 0, or_perturb * rn, ynew);
                    double nrm[OR_MAX_DIM], dot = 0.0;
                    if (or_mutant == 5) {
                        or_normal(P, h_prev, tri[k], y[k], nrm);
                        for (int c = 0; c < d; ++c) dot += (y[k][c] - ynew[c]) * nrm[c];
                    } else {
                        or_normal(P, h, tnew, ynew, nrm);
                        for (int c = 0; c < d; ++c) dot += (ynew[c] - y[k][c]) * nrm[c];
                    }
                    double r = or_dist(d, ynew, y[k]);
                    double kstar = dot / (omega * pow(r, (double)d));
                    /* error bound: the difference y' - y carries the errors of both states and of
                     * the centres; the normal turns by (error of y') / |y' - c_h| = 1, which moves
                     * the dot product by r */
                    const double et = ey[k] + dc + rn;
                    const double dK = (et + r + d * fabs(dot) * et / r) / (omega * pow(r, (double)d)) + fabs(kstar);
                    Qe[k] = fabs(kstar * P->area[h]) * Qe[k] + fabs(Q[k]) * P->area[h] * dK;
                    Q[k] *= kstar * P->area[h];
                    if (or_mutant == 1) T[k] *= dot > 0.0 ? 1.0 : -1.0;
                    ey[k] = rn;
                    amp[k] = 1.0;
                } else {
                    /* isotropic line (same interface) or ray (from a descendant) */
                    double z[OR_MAX_DIM], ts[OR_MAX_ROOTS];
                    int hits[OR_MAX_ROOTS];
                    or_direction(&rng, d, i, k, z);
                    /* a line through a point of a mesh triangle skips that triangle */
                    int q = or_intersections(P, h, y[k], z, rel == OR_REL_DESC, ts,
                                             rel == OR_REL_SAME ? tri[k] : -1, hits);
                    if (q == 0) {            /* no admissible crossing (tangent line): the walk ends */
                        alive[k] = 0; T[k] = 0.0;
                        continue;
                    }
                    /* the pick among q crossings (a single crossing needs no word) */
                    int j = q == 1 ? 0 : (int)(((uint64_t)or_word(&rng, i, k, or_choice_word(d)) * (uint64_t)q) >> 32);
                    for (int c = 0; c < d; ++c) ynew[c] = y[k][c] + ts[j] * z[c];
                    tnew = P->type[h] == OR_MESH ? hits[j] : -1;
                    const double rn = or_norm_rel(d, ynew, ch);
                    double nrm[OR_MAX_DIM], dot = 0.0, nz = 0.0;
                    or_normal(P, h, tnew, ynew, nrm);
                    for (int c = 0; c < d; ++c) {
                        dot += (ynew[c] - y[k][c]) * nrm[c];
                        nz += z[c] * nrm[c];
                    }
                    double sg = dot > 0.0 ? 1.0 : (dot < 0.0 ? -1.0 : 0.0);
                    if (rel == OR_REL_SAME && or_mutant != 7) {
                        Q[k] *= 0.5;
                        Qe[k] *= 0.5;
                    }
                    T[k] *= (double)q * sg;
                    /* error bound: a chord of a sphere or ellipsoid is the reflection t = -2 b, which
                     * does not amplify an error of y; a crossing found as a root moves by the error
                     * over |n . z| */
                    const int reflect = rel == OR_REL_SAME && (P->type[h] == OR_SPHERE || P->type[h] == OR_ELLIPSOID);
                    if (reflect) {
                        ey[k] = ey[k] + rn;
                    } else {
                        const double a = 1.0 + 1.0 / fmax(fabs(nz), 1e-300);
                        ey[k] = (ey[k] + dc) * a + rn;
                        amp[k] *= a;
                        if (amp[k] > cond) cond = amp[k];
                    }
                    if (or_perturb > 0.0) or_perturb_vec(d, walk, i, k, 0, or_perturb * rn, ynew);
                }
                for (int c = 0; c < d; ++c) y[k][c] = ynew[c];
                tri[k] = tnew;
            }
            if (tr && tr->Y)
                for (int c = 0; c < d; ++c) tr->Y[((size_t)k * (M + 1) + i) * d + c] = y[k][c];
            if (tr && tr->QT) {
                tr->QT[((size_t)k * (M + 1) + i) * 2] = Q[k];
                tr->QT[((size_t)k * (M + 1) + i) * 2 + 1] = T[k];
            }
            if (tr && tr->E) {
                tr->E[((size_t)k * (M + 1) + i) * 2] = ey[k];
                tr->E[((size_t)k * (M + 1) + i) * 2 + 1] = Qe[k];
            }
            if (!alive[k]) continue;
            /* tally: N w_i ||alpha||^i prod sign(alpha) Q T Phi(x, y_i), and grad_x Phi */
            const double C = (or_mutant == 4 ? 1.0 : (double)N) * weight * Ai * S;
            double coef = C * Q[k] * T[k];
            const double rx = or_norm_rel(d, x, ch);
            double xp[OR_MAX_DIM];
            for (int c = 0; c < d; ++c) xp[c] = x[c];
            if (or_perturb > 0.0) or_perturb_vec(d, walk, i, k, 1, or_perturb * rx, xp);
            double phi = or_phi(d, xp, y[k]), g[OR_MAX_DIM];
            or_grad_phi(d, xp, y[k], g);
            acc_u += coef * phi;
            for (int c = 0; c < d; ++c) acc_g[c] += coef * g[c];
            double gn = 0.0;
            for (int c = 0; c < d; ++c) gn += g[c] * g[c];
            gn = sqrt(gn);
            const double r = or_dist(d, x, y[k]);
            const double hess = (d - 1) / (omega * pow(r, (double)d));
            const double near = or_mutant_bound == 1 ? 0.0 : ey[k] + rx;
            const double CT = fabs(C * T[k]);
            B_u += CT * (Qe[k] * (fabs(phi) + 1.0) + fabs(Q[k]) * (fabs(phi) + 1.0 + gn * near));
            B_g += CT * (Qe[k] * gn + fabs(Q[k]) * (gn + hess * near));
        }
        h_prev = h;
    }
    *out_u = acc_u;
    for (int c = 0; c < d; ++c) out_g[c] = acc_g[c];
    if (tr && tr->scale) { tr->scale[0] = B_u; tr->scale[1] = B_g; tr->scale[2] = cond; tr->scale[3] = flux_ratio; }
}

/* ------------------------------------------------------------------------ */
/* estimator over points (Algorithm 1): per point the walk sum and the       */
/* sums of the schedule-group means and of their squares                    */
/* ------------------------------------------------------------------------ */
int or_estimate(const or_problem *P, const or_opts *o, const double *points, int64_t n_pts, uint32_t point_offset,
                uint32_t instance, uint64_t walk_begin, uint64_t walk_end, uint64_t seed, double *sum_f /* [n_pts][d+1] */,
                double *sum_gm /* [n_pts][d+1] */, double *sum_gm2 /* [n_pts][d+1] */, int64_t *n_groups)
{
    const int d = P->dim, W_g = o->sched_group;
    if (W_g < 1 || walk_begin % (uint64_t)W_g != 0 || walk_end % (uint64_t)W_g != 0) return 1;
    int64_t G = (int64_t)((walk_end - walk_begin) / (uint64_t)W_g);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t p = 0; p < n_pts; ++p) {
        const double *x = points + (size_t)p * d;
        double sf[OR_MAX_DIM + 1] = {0}, sm[OR_MAX_DIM + 1] = {0}, sm2[OR_MAX_DIM + 1] = {0};
        for (uint64_t g0 = walk_begin; g0 < walk_end; g0 += (uint64_t)W_g) {
            double gs[OR_MAX_DIM + 1] = {0};
            for (int j = 0; j < W_g; ++j) {
                double fu, fg[OR_MAX_DIM];
                or_walk(P, o, x, point_offset + (uint32_t)p, instance, g0 + (uint64_t)j, seed, &fu, fg, NULL);
                gs[0] += fu;
                for (int c = 0; c < d; ++c) gs[1 + c] += fg[c];
            }
            for (int c = 0; c <= d; ++c) {
                double m = gs[c] / W_g;
                sf[c] += gs[c];
                sm[c] += m;
                sm2[c] += m * m;
            }
        }
        for (int c = 0; c <= d; ++c) {
            sum_f[p * (d + 1) + c] = sf[c];
            sum_gm[p * (d + 1) + c] = sm[c];
            sum_gm2[p * (d + 1) + c] = sm2[c];
        }
    }
    *n_groups = G;
    return 0;
}

/* per-walk values for pathwise replay: walks[w] for one point */
void or_walks(const or_problem *P, const or_opts *o, const double *x, uint32_t point_id, uint32_t instance,
              const uint64_t *walks, int64_t n_walks, uint64_t seed, double *out_u, double *out_g, int *out_H,
              double *out_Y, double *out_scale, double *out_QT, double *out_E)
{
    const int d = P->dim, M = o->M;
    /* walks are independent and write disjoint output slots */
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t w = 0; w < n_walks; ++w) {
        or_trace tr = {out_H ? out_H + w * (M + 1) : NULL, out_Y ? out_Y + (size_t)w * 2 * (M + 1) * d : NULL,
                       out_scale ? out_scale + 4 * w : NULL, out_QT ? out_QT + (size_t)w * 2 * (M + 1) * 2 : NULL,
                       out_E ? out_E + (size_t)w * 2 * (M + 1) * 2 : NULL};
        or_walk(P, o, x, point_id, instance, walks[w], seed, out_u + w, out_g + w * d, &tr);
    }
}

/* exposed for the tests of the building blocks */
double or_test_real_sh(int l, int m, const double *u) { return or_real_sh(l, m, u); }
double or_test_star_arclen(const or_problem *P, int h, double t) { return or_star_arclen(P, h, t); }
int or_test_intersections(const or_problem *P, int h, const double *y, const double *z, int ray, double *ts,
                          int exclude, int *hit_tri)
{
    int dummy[OR_MAX_ROOTS];
    return or_intersections(P, h, y, z, ray, ts, exclude, hit_tri ? hit_tri : dummy);
}
double or_test_flux(const or_problem *P, int h, int tri, const double *y) { return or_flux(P, h, tri, y); }
void or_test_uniform_point(const or_problem *P, int h, uint64_t seed, uint32_t point_id, uint64_t walk, int step,
                           double *y, int *tri)
{
    or_rng rng = {{(uint32_t)seed ^ point_id, (uint32_t)(seed >> 32)}, walk, -1, -1, -1, {0}};
    int t;
    or_uniform_point(P, h, &rng, step, 0, y, &t);
    if (tri) *tri = t;
}
void or_test_uniform_part_point(const or_problem *P, int h, int part, uint64_t seed, uint64_t walk, double *y)
{
    or_rng rng = {{(uint32_t)seed, (uint32_t)(seed >> 32)}, walk, -1, -1, -1, {0}};
    or_uniform_part_point(P, h, part, &rng, 0, part, y);
}
void or_test_direction(int d, uint64_t seed, uint64_t walk, int step, double *z)
{
    or_rng rng = {{(uint32_t)seed, (uint32_t)(seed >> 32)}, walk, -1, -1, -1, {0}};
    or_direction(&rng, d, step, 0, z);
}
