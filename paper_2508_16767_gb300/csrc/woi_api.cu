// woi_api.cu -- the C ABI of libwoi (include/woi.h): validation, the
// pre-processing of Sec. 3 (alpha, beta, schedule thresholds of Thm 4.2),
// geometry tables (areas, star arc lengths, beta-sign arcs of Sec. 4.4),
// device staging and kernel dispatch.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <cstdlib>
#include <map>
#include <string>
#include <vector>

#include "../../include/woi.h"
#include "woi_kernels.h"
#include "woi_layout.h"
#include "woi_mesh_host.h"

using namespace woi;

namespace {

thread_local std::string g_last_error;

woi_status fail(woi_status st, const char *fmt, ...)
{
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_last_error = buf;
    return st;
}

#define WOI_CUDA(call)                                                                               \
    do {                                                                                             \
        cudaError_t e_ = (call);                                                                     \
        if (e_ != cudaSuccess) return fail(WOI_E_CUDA, "%s: %s", #call, cudaGetErrorString(e_));    \
    } while (0)

constexpr double kPi = 3.14159265358979323846;

double omega_d(int d) { return 2.0 * std::pow(kPi, 0.5 * d) / std::tgamma(0.5 * d); }

// star curve r(t), r'(t)
struct StarCurve {
    double R = 1.0;
    int K = 0;
    double a[kMaxStar + 1] = {0}, b[kMaxStar + 1] = {0};
    double c[2] = {0, 0};
    void eval(double t, double *r, double *dr) const
    {
        double s = 1.0, ds = 0.0;
        for (int k = 1; k <= K; ++k) {
            s += a[k] * std::cos(k * t) + b[k] * std::sin(k * t);
            ds += k * (b[k] * std::cos(k * t) - a[k] * std::sin(k * t));
        }
        *r = R * s;
        *dr = R * ds;
    }
    double speed(double t) const
    {
        double r, dr;
        eval(t, &r, &dr);
        return std::sqrt(r * r + dr * dr);
    }
    void point(double t, double *p) const
    {
        double r, dr;
        eval(t, &r, &dr);
        p[0] = c[0] + r * std::cos(t);
        p[1] = c[1] + r * std::sin(t);
    }
};

// composite 8-point Gauss-Legendre of |gamma'| on [a, b] with m sub-panels
double star_length(const StarCurve &s, double a, double b, int m = 8)
{
    static const double x[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    static const double w[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    double tot = 0.0, h = (b - a) / m;
    for (int j = 0; j < m; ++j) {
        double mid = a + (j + 0.5) * h, half = 0.5 * h, acc = 0.0;
        for (int q = 0; q < 4; ++q) acc += w[q] * (s.speed(mid - half * x[q]) + s.speed(mid + half * x[q]));
        tot += half * acc;
    }
    return tot;
}

double fourier_eval(const std::vector<double> &c, double t)
{
    double v = c.empty() ? 0.0 : c[0];
    for (size_t k = 1; 2 * k <= c.size() - 1; ++k) v += c[2 * k - 1] * std::cos(k * t) + c[2 * k] * std::sin(k * t);
    return v;
}

bool pointer_on_device(const void *p)
{
    if (!p) return false;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace

// ---------------------------------------------------------------------------
// the geometry handle
// ---------------------------------------------------------------------------
struct woi_geometry {
    int dim = 0, n = 0;
    std::vector<woi_surface_desc> surf;
    std::vector<int> parent, tin, tout;
    std::vector<double> area;
    int star_idx = -1;
    StarCurve star;
    std::vector<double> star_panel_s;          // kNodes + 1
    std::vector<double> star_scan;             // kNodes * 2
    std::vector<double> star_scan_d;           // kNodes * 2: gamma'(t_j)
    double star_lmax = 0.0;
    double star_kpp = 0.0;                     // bound on |gamma''|
    double star_k3 = 0.0;                      // bound on |gamma'''|
    double star_rmin = 0.0, star_rmax = 0.0;
    struct Ellipsoid {
        double A[kMaxDim][kMaxDim];            // (y - c)^T A (y - c) = 1
        double map[kMaxDim][kMaxDim];          // A^{-1/2}: unit sphere -> surface (about c)
        double lam[kMaxDim];                   // eigenvalues of A
        double jmax;                           // sqrt(max eigenvalue)
    };
    std::vector<Ellipsoid> ell;
    std::vector<int> ell_slot;                 // per surface, -1 if not an ellipsoid
    std::vector<MeshHost> mesh;
    std::vector<int> mesh_slot;                // per surface, -1 if not a mesh

    bool data_ready = false;
    std::vector<double> sigma, alpha, beta_scale, flux_coef;
    std::vector<double> flux_dev;              // device format of flux_coef
    std::vector<float> flux_dev_f;
    std::vector<int> flux_basis_dev, flux_off_dev, flux_n_dev;   // device basis codes and layout
    std::vector<uint64_t> thresh;
    double alpha_l1 = 0.0;
    std::vector<int> flux_basis, flux_off, flux_n;
    bool vr_ok = false;
    std::vector<double> arc_t0, arc_t1, arc_len, arc_s0, part_len;
    std::vector<double> vr_tol;                                  // per surface, d >= 3 VR (FP64 sign check)
    std::vector<int> arc_sign, arc_off, arc_n;

    // device side
    int device = -1;
    bool dev_dirty = true;
    DevGeom blob{};
    DevGeom *d_blob = nullptr;
    float *d_flux_f = nullptr;
    double *d_flux = nullptr, *d_arc_t0 = nullptr, *d_arc_t1 = nullptr, *d_arc_len = nullptr, *d_arc_s0 = nullptr;
    int *d_arc_sign = nullptr;
    float *d_tri_f = nullptr;
    double *d_tri_d = nullptr;
    uint32_t *d_tri_tm1 = nullptr;
    int *d_tri_bucket = nullptr;
    BvhWide *d_bvh = nullptr;
    unsigned int *d_mesh_overflow = nullptr;
    int blob_M = -1;
    // grow-only scratch
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    int num_sms = 0;
    std::map<long long, int> occ_cache;        // (dim, vr, general surfaces, block) -> blocks per SM

    // kernels with non-sphere surfaces: the star (2D) or ellipsoids (d >= 3)
    bool general() const { return star_idx >= 0 || !ell.empty() || !mesh.empty(); }
    cudaEvent_t ev_start = nullptr, ev_stop = nullptr;
    bool timed = false;
    cudaEvent_t ev_done = nullptr;             // end of the last asynchronous estimate on a mesh geometry
    bool check_pending = false;                // its overflow counter has not been read yet

    ~woi_geometry() { release(); }
    void release()
    {
        if (device < 0) return;
        int cur = -1;
        cudaGetDevice(&cur);
        cudaSetDevice(device);
        cudaFree(d_blob);
        cudaFree(d_flux);
        cudaFree(d_flux_f);
        cudaFree(d_arc_t0);
        cudaFree(d_arc_t1);
        cudaFree(d_arc_len);
        cudaFree(d_arc_s0);
        cudaFree(d_arc_sign);
        cudaFree(d_tri_f);
        cudaFree(d_tri_d);
        cudaFree(d_tri_tm1);
        cudaFree(d_tri_bucket);
        cudaFree(d_bvh);
        cudaFree(d_mesh_overflow);
        cudaFree(d_scratch);
        if (ev_start) cudaEventDestroy(ev_start);
        if (ev_stop) cudaEventDestroy(ev_stop);
        if (ev_done) cudaEventDestroy(ev_done);
        ev_start = ev_stop = ev_done = nullptr;
        timed = false;
        check_pending = false;
        if (cur >= 0) cudaSetDevice(cur);
        d_blob = nullptr;
        d_flux = d_arc_t0 = d_arc_t1 = d_arc_len = d_arc_s0 = nullptr;
        d_flux_f = nullptr;
        d_arc_sign = nullptr;
        d_tri_f = nullptr;
        d_tri_d = nullptr;
        d_tri_tm1 = nullptr;
        d_tri_bucket = nullptr;
        d_bvh = nullptr;
        d_mesh_overflow = nullptr;
        d_scratch = nullptr;
        scratch_bytes = 0;
        device = -1;
    }
};

// ---------------------------------------------------------------------------
// geometry validation helpers
// ---------------------------------------------------------------------------
namespace {

double dist(int d, const double *a, const double *b)
{
    double s = 0.0;
    for (int k = 0; k < d; ++k) s += (a[k] - b[k]) * (a[k] - b[k]);
    return std::sqrt(s);
}

// symmetric eigen-decomposition A = V diag(lam) V^T by cyclic Jacobi rotations
// (each rotation in the (p, q) plane zeroes A_pq; converges quadratically)
void jacobi_eigen(int d, const double (*A_in)[kMaxDim], double *lam, double (*V)[kMaxDim])
{
    double A[kMaxDim][kMaxDim];
    double norm2 = 0.0;
    for (int i = 0; i < d; ++i)
        for (int j = 0; j < d; ++j) {
            A[i][j] = A_in[i][j];
            V[i][j] = i == j ? 1.0 : 0.0;
            norm2 += A[i][j] * A[i][j];
        }
    for (int sweep = 0; sweep < 64; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) off += A[p][q] * A[p][q];
        if (off <= 1e-32 * norm2) break;
        for (int p = 0; p < d; ++p)
            for (int q = p + 1; q < d; ++q) {
                if (A[p][q] == 0.0) continue;
                const double theta = (A[q][q] - A[p][p]) / (2.0 * A[p][q]);
                const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
                const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
                // A <- J^T A J, V <- V J with J the rotation by (c, sn) in the (p, q) plane
                for (int k = 0; k < d; ++k) {
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = c * akp - sn * akq;
                    A[k][q] = sn * akp + c * akq;
                }
                for (int k = 0; k < d; ++k) {
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = c * apk - sn * aqk;
                    A[q][k] = sn * apk + c * aqk;
                }
                for (int k = 0; k < d; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = c * vkp - sn * vkq;
                    V[k][q] = sn * vkp + c * vkq;
                }
            }
    }
    for (int k = 0; k < d; ++k) lam[k] = A[k][k];
}

// |dE| of {y : y^T A y = 1} from the eigenvalues lam of A.  The map u -> diag(a) u
// (a = lam^{-1/2}) takes the unit sphere onto the surface and scales area by
// prod(a) |diag(sqrt(lam)) u|, so |dE| = |S^{d-1}| prod(a) E_u |diag(sqrt(lam)) u|.
// For a standard normal g = |g| u, E_u[.] = E sqrt(S) / E|g| with S = sum lam_k g_k^2;
// sqrt(S) = pi^{-1/2} int_0^inf (1 - exp(-t^2 S)) t^{-2} dt turns E sqrt(S) into
// pi^{-1/2} int_0^inf (1 - prod_k (1 + 2 lam_k t^2)^{-1/2}) t^{-2} dt, integrated here
// over theta = atan(t / s) in [0, pi/2) by composite 8-point Gauss-Legendre.
double ellipsoid_area(int d, const double *lam)
{
    static const double x[4] = {0.1834346424956498, 0.5255324099163290, 0.7966664774136267, 0.9602898564975363};
    static const double w[4] = {0.3626837833783620, 0.3137066458778873, 0.2223810344533745, 0.1012285362903763};
    double lg = 0.0, prod_a = 1.0;
    for (int k = 0; k < d; ++k) {
        lg += std::log(lam[k]);
        prod_a /= std::sqrt(lam[k]);
    }
    const double sc = std::exp(-0.5 * lg / d);               // t = sc tan(theta)
    auto integrand = [&](double th) {
        const double t = sc * std::tan(th), t2 = t * t;
        double ls = 0.0;
        for (int k = 0; k < d; ++k) ls += std::log1p(2.0 * lam[k] * t2);
        const double sec = 1.0 / std::cos(th);
        return -std::expm1(-0.5 * ls) / t2 * sc * sec * sec;   // f(t) dt / dtheta
    };
    const int panels = 256;
    const double h = 0.5 * kPi / panels;
    double I = 0.0;
    for (int j = 0; j < panels; ++j) {
        const double mid = (j + 0.5) * h, half = 0.5 * h;
        double acc = 0.0;
        for (int q = 0; q < 4; ++q) acc += w[q] * (integrand(mid - half * x[q]) + integrand(mid + half * x[q]));
        I += half * acc;
    }
    const double e_sqrt_s = I / std::sqrt(kPi);
    const double e_norm = std::sqrt(2.0) * std::exp(std::lgamma(0.5 * (d + 1)) - std::lgamma(0.5 * d));
    return omega_d(d) * prod_a * e_sqrt_s / e_norm;
}

// deterministic points on surface i of a d >= 3 geometry (sphere or ellipsoid):
// unit vectors from SplitMix64 words by Box-Muller, mapped onto the surface
std::vector<double> sample_surface(const woi_geometry &g, int i, int m)
{
    const int d = g.dim;
    std::vector<double> p((size_t)m * d);
    uint64_t st = 0x9E3779B97F4A7C15ull * (uint64_t)(i + 1);
    auto next = [&]() {
        uint64_t z = (st += 0x9E3779B97F4A7C15ull);
        z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
        z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
        z ^= z >> 31;
        return ((double)(z >> 11) + 0.5) * (1.0 / 9007199254740992.0);
    };
    const woi_surface_desc &s = g.surf[i];
    if (s.type == WOI_MESH) {
        // the triangles' corners and centroids (local rows v0, e1, e2 back to global)
        const MeshHost &mh = g.mesh[g.mesh_slot[i]];
        p.assign((size_t)mh.ntri * 2 * 3, 0.0);
        for (int t = 0; t < mh.ntri; ++t) {
            const double *r = &mh.tri[(size_t)t * 12];
            for (int k = 0; k < 3; ++k) {
                p[(size_t)t * 6 + k] = mh.center[k] + r[k];
                p[(size_t)t * 6 + 3 + k] = mh.center[k] + r[k] + (r[3 + k] + r[6 + k]) / 3.0;
            }
        }
        return p;
    }
    for (int j = 0; j < m; ++j) {
        double u[kMaxDim + 1], nn = 0.0;
        for (int k = 0; k < d; k += 2) {
            const double r = std::sqrt(-2.0 * std::log(next())), a = 2.0 * kPi * next();
            u[k] = r * std::cos(a);
            u[k + 1] = r * std::sin(a);
        }
        for (int k = 0; k < d; ++k) nn += u[k] * u[k];
        nn = std::sqrt(nn);
        for (int k = 0; k < d; ++k) u[k] /= nn;
        for (int k = 0; k < d; ++k) {
            double v = s.center[k];
            if (s.type == WOI_ELLIPSOID) {
                const auto &e = g.ell[g.ell_slot[i]];
                for (int q = 0; q < d; ++q) v += e.map[k][q] * u[q];
            } else {
                v += s.radius * u[k];
            }
            p[(size_t)j * d + k] = v;
        }
    }
    return p;
}

// (x - c)^T A (x - c) of ellipsoid surface i
double ellipsoid_form(const woi_geometry &g, int i, const double *x)
{
    const auto &e = g.ell[g.ell_slot[i]];
    const double *c = g.surf[i].center;
    double q = 0.0;
    for (int a = 0; a < g.dim; ++a)
        for (int b = 0; b < g.dim; ++b) q += (x[a] - c[a]) * e.A[a][b] * (x[b] - c[b]);
    return q;
}

// a dense sample of surface i (2D only: circles and stars), used for star checks
std::vector<double> sample_curve(const woi_geometry &g, int i, int m)
{
    std::vector<double> p(2 * m);
    for (int j = 0; j < m; ++j) {
        double t = 2.0 * kPi * j / m;
        if (g.surf[i].type == WOI_STAR) {
            g.star.point(t, &p[2 * j]);
        } else {
            p[2 * j] = g.surf[i].center[0] + g.surf[i].radius * std::cos(t);
            p[2 * j + 1] = g.surf[i].center[1] + g.surf[i].radius * std::sin(t);
        }
    }
    return p;
}

// is point x strictly inside the region bounded by surface i?
bool inside_surface(const woi_geometry &g, int i, const double *x)
{
    const woi_surface_desc &s = g.surf[i];
    if (s.type == WOI_SPHERE) return dist(g.dim, x, s.center) < s.radius;
    if (s.type == WOI_ELLIPSOID) return ellipsoid_form(g, i, x) < 1.0;
    if (s.type == WOI_MESH) return mesh_inside(g.mesh[g.mesh_slot[i]], x);
    double t = std::atan2(x[1] - s.center[1], x[0] - s.center[0]);
    double r, dr;
    g.star.eval(t, &r, &dr);
    return std::hypot(x[0] - s.center[0], x[1] - s.center[1]) < r;
}

woi_status check_nesting(const woi_geometry &g)
{
    const int n = g.n, d = g.dim;
    const int M = 4096;
    for (int i = 1; i < n; ++i) {
        const int p = g.parent[i];
        const woi_surface_desc &si = g.surf[i], &sp = g.surf[p];
        // i strictly inside its parent
        if (si.type == WOI_SPHERE && sp.type == WOI_SPHERE) {
            if (!(dist(d, si.center, sp.center) + si.radius < sp.radius))
                return fail(WOI_E_GEOMETRY, "surface %d is not strictly inside its parent %d", i, p);
        } else if (d >= 3) {
            // convex surfaces: every point of surface i inside the parent (a dense sample)
            std::vector<double> pts = sample_surface(g, i, M * 4);
            for (size_t j = 0; j < pts.size() / d; ++j)
                if (!inside_surface(g, p, &pts[j * d]))
                    return fail(WOI_E_GEOMETRY, "surface %d is not strictly inside its parent %d", i, p);
        } else {
            std::vector<double> pts = sample_curve(g, i, M);
            for (int j = 0; j < M; ++j)
                if (!inside_surface(g, p, &pts[2 * j]))
                    return fail(WOI_E_GEOMETRY, "surface %d is not strictly inside its parent %d", i, p);
            if (sp.type == WOI_STAR) {
                std::vector<double> q = sample_curve(g, p, M);
                for (int j = 0; j < M; ++j)
                    if (inside_surface(g, i, &q[2 * j]))
                        return fail(WOI_E_GEOMETRY, "surface %d crosses its parent %d", i, p);
            }
        }
        // disjoint from its siblings
        for (int j = i + 1; j < n; ++j) {
            if (g.parent[j] != p) continue;
            const woi_surface_desc &sj = g.surf[j];
            if (si.type == WOI_SPHERE && sj.type == WOI_SPHERE) {
                if (!(dist(d, si.center, sj.center) > si.radius + sj.radius))
                    return fail(WOI_E_GEOMETRY, "surfaces %d and %d overlap", i, j);
            } else if (d >= 3) {
                std::vector<double> a = sample_surface(g, i, M * 4), b = sample_surface(g, j, M * 4);
                for (size_t k = 0; k < a.size() / d; ++k)
                    if (inside_surface(g, j, &a[k * d])) return fail(WOI_E_GEOMETRY, "surfaces %d and %d overlap", i, j);
                for (size_t k = 0; k < b.size() / d; ++k)
                    if (inside_surface(g, i, &b[k * d])) return fail(WOI_E_GEOMETRY, "surfaces %d and %d overlap", i, j);
            } else {
                std::vector<double> a = sample_curve(g, i, M), b = sample_curve(g, j, M);
                for (int k = 0; k < M; ++k)
                    if (inside_surface(g, j, &a[2 * k]) || inside_surface(g, i, &b[2 * k]))
                        return fail(WOI_E_GEOMETRY, "surfaces %d and %d overlap", i, j);
            }
        }
    }
    return WOI_OK;
}

// Laplacian of a monomial expansion is identically zero?
bool poly_is_harmonic(int d, int T, const double *rows, double *scale)
{
    std::map<std::vector<int>, double> lap;
    double tot = 0.0;
    for (int t = 0; t < T; ++t) {
        const double *row = rows + t * (d + 1);
        tot += std::fabs(row[0]);
        for (int k = 0; k < d; ++k) {
            int e = (int)row[1 + k];
            if (e < 2) continue;
            std::vector<int> key(d);
            for (int j = 0; j < d; ++j) key[j] = (int)row[1 + j];
            key[k] -= 2;
            lap[key] += row[0] * e * (e - 1);
        }
    }
    *scale = tot;
    for (auto &kv : lap)
        if (std::fabs(kv.second) > 1e-12 * std::max(tot, 1.0)) return false;
    return true;
}

}  // namespace

// ---------------------------------------------------------------------------
// C ABI
// ---------------------------------------------------------------------------
extern "C" {

const char *woi_version(void) { return "woi-gb300 1.0 (sm_103a)"; }

const char *woi_last_error(void) { return g_last_error.c_str(); }

void woi_default_opts(woi_opts *o)
{
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->M = 4;
    o->variant = WOI_PLAIN;
    o->precision = WOI_MIXED;
    o->sched_group = 1;
}

woi_status woi_create_geometry(int dim, int n_surf, const woi_surface_desc *surfaces, const int *parent,
                               woi_geometry **out)
{
    g_last_error.clear();
    if (!out || !surfaces || !parent) return fail(WOI_E_INVALID_ARG, "null argument");
    if (dim < 2 || dim > WOI_MAX_DIM) return fail(WOI_E_INVALID_ARG, "dim %d outside [2, %d]", dim, WOI_MAX_DIM);
    if (n_surf < 1 || n_surf > WOI_MAX_SURF)
        return fail(WOI_E_INVALID_ARG, "n_surf %d outside [1, %d]", n_surf, WOI_MAX_SURF);
    if (parent[0] != -1) return fail(WOI_E_INVALID_ARG, "parent[0] must be -1 (surface 0 is the outer boundary)");
    for (int i = 1; i < n_surf; ++i) {
        if (parent[i] < 0 || parent[i] >= n_surf || parent[i] == i)
            return fail(WOI_E_INVALID_ARG, "parent[%d] = %d is not a surface index", i, parent[i]);
        int p = parent[i], steps = 0;          // the chain of parents must reach 0 without a cycle
        while (p != 0 && steps <= n_surf) { p = parent[p]; ++steps; }
        if (p != 0) return fail(WOI_E_INVALID_ARG, "parent array has a cycle through surface %d", i);
    }
    auto *g = new (std::nothrow) woi_geometry();
    if (!g) return fail(WOI_E_OOM, "host allocation failed");
    g->dim = dim;
    g->n = n_surf;
    g->surf.assign(surfaces, surfaces + n_surf);
    g->parent.assign(parent, parent + n_surf);
    g->ell_slot.assign(n_surf, -1);
    g->mesh_slot.assign(n_surf, -1);
    size_t mesh_tris = 0;
    for (int i = 0; i < n_surf; ++i) {
        woi_surface_desc &s = g->surf[i];
        s.star_a = s.star_b = nullptr;         // deep copy below; no pointer retained
        s.matrix = nullptr;
        s.vertices = nullptr;
        s.triangles = nullptr;
        if (s.type == WOI_SPHERE) {
            if (!(s.radius > 0.0) || !std::isfinite(s.radius)) {
                delete g;
                return fail(WOI_E_INVALID_ARG, "surface %d: radius must be positive", i);
            }
        } else if (s.type == WOI_STAR) {
            if (dim != 2) { delete g; return fail(WOI_E_UNSUPPORTED, "star surfaces exist only in 2D"); }
            if (g->star_idx >= 0) { delete g; return fail(WOI_E_UNSUPPORTED, "at most one star surface per geometry"); }
            const int K = surfaces[i].star_degree;
            if (K < 0 || K > WOI_MAX_STAR_DEGREE || (K > 0 && (!surfaces[i].star_a || !surfaces[i].star_b))) {
                delete g;
                return fail(WOI_E_INVALID_ARG, "surface %d: bad star degree or coefficients", i);
            }
            if (!(s.radius > 0.0)) { delete g; return fail(WOI_E_INVALID_ARG, "surface %d: radius must be positive", i); }
            g->star_idx = i;
            g->star.R = s.radius;
            g->star.K = K;
            g->star.c[0] = s.center[0];
            g->star.c[1] = s.center[1];
            for (int k = 1; k <= K; ++k) {
                g->star.a[k] = surfaces[i].star_a[k];
                g->star.b[k] = surfaces[i].star_b[k];
            }
            for (int j = 0; j < 8192; ++j) {
                double r, dr;
                g->star.eval(2.0 * kPi * j / 8192, &r, &dr);
                if (!(r > 0.0)) { delete g; return fail(WOI_E_GEOMETRY, "surface %d: star radius not positive", i); }
            }
        } else if (s.type == WOI_ELLIPSOID) {
            if (dim < 3) { delete g; return fail(WOI_E_UNSUPPORTED, "ellipsoid surfaces need dim >= 3"); }
            if ((int)g->ell.size() >= kMaxEll) {
                delete g;
                return fail(WOI_E_UNSUPPORTED, "at most %d ellipsoids per geometry", kMaxEll);
            }
            const double *A = surfaces[i].matrix;
            if (!A) { delete g; return fail(WOI_E_INVALID_ARG, "surface %d: null ellipsoid matrix", i); }
            woi_geometry::Ellipsoid e{};
            double amax = 0.0;
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) {
                    e.A[a][b] = A[a * dim + b];
                    amax = std::max(amax, std::fabs(A[a * dim + b]));
                    if (!std::isfinite(A[a * dim + b])) { delete g; return fail(WOI_E_INVALID_ARG, "surface %d: matrix not finite", i); }
                }
            for (int a = 0; a < dim; ++a)
                for (int b = a + 1; b < dim; ++b)
                    if (std::fabs(e.A[a][b] - e.A[b][a]) > 1e-12 * amax) {
                        delete g;
                        return fail(WOI_E_INVALID_ARG, "surface %d: ellipsoid matrix is not symmetric", i);
                    }
            double lam[kMaxDim], V[kMaxDim][kMaxDim];
            jacobi_eigen(dim, e.A, lam, V);
            for (int k = 0; k < dim; ++k)
                if (!(lam[k] > 0.0)) {
                    delete g;
                    return fail(WOI_E_INVALID_ARG, "surface %d: ellipsoid matrix is not positive definite", i);
                }
            // the symmetric square root A^{-1/2} = V diag(lam^{-1/2}) V^T: unlike V diag(a) it does
            // not depend on the order or signs of the eigenvectors, so a uniform u on the unit
            // sphere gives the same surface point whatever routine decomposed A
            e.jmax = 0.0;
            for (int k = 0; k < dim; ++k) {
                e.lam[k] = lam[k];
                e.jmax = std::max(e.jmax, std::sqrt(lam[k]));
            }
            for (int a = 0; a < dim; ++a)
                for (int b = 0; b < dim; ++b) {
                    double m = 0.0;
                    for (int k = 0; k < dim; ++k) m += V[a][k] * V[b][k] / std::sqrt(lam[k]);
                    e.map[a][b] = m;
                }
            g->ell_slot[i] = (int)g->ell.size();
            g->ell.push_back(e);
        } else if (s.type == WOI_MESH) {
            if (dim != 3) { delete g; return fail(WOI_E_UNSUPPORTED, "mesh surfaces need dim = 3"); }
            if ((int)g->mesh.size() >= kMaxMesh) {
                delete g;
                return fail(WOI_E_UNSUPPORTED, "at most %d meshes per geometry", kMaxMesh);
            }
            const woi_surface_desc &in = surfaces[i];
            mesh_tris += (size_t)std::max(0, in.n_triangles);
            if (mesh_tris > (size_t)WOI_MAX_MESH_TRIANGLES) {
                delete g;
                return fail(WOI_E_UNSUPPORTED, "more than %d mesh triangles", WOI_MAX_MESH_TRIANGLES);
            }
            MeshHost mh;
            std::string why = mesh_prepare(in.vertices, in.n_vertices, in.triangles, in.n_triangles, in.center, mh);
            if (!why.empty()) {
                delete g;
                return fail(WOI_E_GEOMETRY, "surface %d: %s", i, why.c_str());
            }
            g->mesh_slot[i] = (int)g->mesh.size();
            g->mesh.push_back(std::move(mh));
        } else {
            delete g;
            return fail(WOI_E_INVALID_ARG, "surface %d: unknown type %d", i, s.type);
        }
    }
    woi_status st = check_nesting(*g);
    if (st != WOI_OK) { delete g; return st; }
    // Euler tour of the tree: a is a strict descendant of b iff tin[b] < tin[a] < tout[b]
    {
        std::vector<std::vector<int>> ch(n_surf);
        for (int i = 1; i < n_surf; ++i) ch[g->parent[i]].push_back(i);
        g->tin.assign(n_surf, 0);
        g->tout.assign(n_surf, 0);
        int clock = 0;
        std::vector<std::pair<int, size_t>> stack{{0, 0}};
        g->tin[0] = clock++;
        while (!stack.empty()) {
            auto &top = stack.back();
            if (top.second < ch[top.first].size()) {
                int c = ch[top.first][top.second++];
                g->tin[c] = clock++;
                stack.push_back({c, 0});
            } else {
                g->tout[top.first] = clock++;
                stack.pop_back();
            }
        }
    }
    // areas, star tables
    g->area.resize(n_surf);
    for (int i = 0; i < n_surf; ++i) {
        if (g->surf[i].type == WOI_SPHERE) {
            g->area[i] = omega_d(dim) * std::pow(g->surf[i].radius, dim - 1);
        } else if (g->surf[i].type == WOI_ELLIPSOID) {
            g->area[i] = ellipsoid_area(dim, g->ell[g->ell_slot[i]].lam);
        } else if (g->surf[i].type == WOI_MESH) {
            g->area[i] = g->mesh[g->mesh_slot[i]].area;
        }
    }
    if (g->star_idx >= 0) {
        g->star_panel_s.assign(kNodes + 1, 0.0);
        const double H = 2.0 * kPi / kNodes;
        for (int j = 0; j < kNodes; ++j)
            g->star_panel_s[j + 1] = g->star_panel_s[j] + star_length(g->star, j * H, (j + 1) * H, 4);
        g->area[g->star_idx] = g->star_panel_s[kNodes];
        g->star_scan.assign(2 * kNodes, 0.0);
        g->star_scan_d.assign(2 * kNodes, 0.0);
        for (int j = 0; j < kNodes; ++j) {
            double r, dr, t = 2.0 * kPi * j / kNodes;
            g->star.eval(t, &r, &dr);
            g->star_scan[2 * j] = r * std::cos(t);
            g->star_scan[2 * j + 1] = r * std::sin(t);
            g->star_scan_d[2 * j] = dr * std::cos(t) - r * std::sin(t);
            g->star_scan_d[2 * j + 1] = dr * std::sin(t) + r * std::cos(t);
        }
        double lm = 0.0, rmin = 1e300, rmax = 0.0, b1 = 0.0, b2 = 0.0;
        for (int k = 1; k <= g->star.K; ++k) {
            b1 += (double)k * (std::fabs(g->star.a[k]) + std::fabs(g->star.b[k]));
            b2 += (double)k * k * (std::fabs(g->star.a[k]) + std::fabs(g->star.b[k]));
        }
        b1 *= g->star.R;                                   // bound on |r'|
        b2 *= g->star.R;                                   // bound on |r''|
        const int ms = 16384;
        for (int j = 0; j < ms; ++j) {
            const double t = 2.0 * kPi * j / ms;
            double r, dr;
            g->star.eval(t, &r, &dr);
            lm = std::max(lm, std::sqrt(r * r + dr * dr));
            rmin = std::min(rmin, r);
            rmax = std::max(rmax, r);
        }
        const double h = 2.0 * kPi / ms, margin = b2 * h * h / 8.0 + 1e-9 * g->star.R;
        g->star_lmax = lm * 1.02 + 1e-12;
        g->star_rmin = std::max(0.0, rmin - margin);
        g->star_rmax = rmax + margin;
        // gamma'' = (r'' - r) e_r + 2 r' e_t, so |gamma''| <= |r''| + r + 2 |r'|
        g->star_kpp = b2 + g->star_rmax + 2.0 * b1;
        // gamma''' = (r''' - 3 r') e_r + (3 r'' - r) e_t
        double b3 = 0.0;
        for (int k = 1; k <= g->star.K; ++k)
            b3 += (double)k * k * k * (std::fabs(g->star.a[k]) + std::fabs(g->star.b[k]));
        g->star_k3 = b3 * g->star.R + 3.0 * b1 + 3.0 * b2 + g->star_rmax;
    }
    *out = g;
    return WOI_OK;
}

woi_status woi_surface_area(const woi_geometry *g, int i, double *area)
{
    g_last_error.clear();
    if (!g || !area) return fail(WOI_E_INVALID_ARG, "null argument");
    if (i < 0 || i >= g->n) return fail(WOI_E_INVALID_ARG, "surface %d out of range", i);
    *area = g->area[i];
    return WOI_OK;
}

woi_status woi_set_sigma_and_data(woi_geometry *g, const double *sigma, const woi_flux_desc *flux)
{
    g_last_error.clear();
    if (!g || !sigma || !flux) return fail(WOI_E_INVALID_ARG, "null argument");
    const int n = g->n, d = g->dim;
    if (!(sigma[0] > 0.0)) return fail(WOI_E_INVALID_ARG, "sigma_1 must be positive");
    for (int i = 0; i < n; ++i) {
        if (!(sigma[i] >= 0.0) || !std::isfinite(sigma[i])) return fail(WOI_E_INVALID_ARG, "sigma[%d] must be >= 0", i);
        if (i > 0 && !(sigma[i] + sigma[g->parent[i]] > 0.0))
            return fail(WOI_E_INVALID_ARG, "sigma[%d] + sigma[parent] must be positive", i);
    }
    // flux data: basis / surface fit and the compatibility condition (zero mean per surface)
    std::vector<int> basis(n), off(n), nc(n);
    std::vector<double> coef;
    for (int i = 0; i < n; ++i) {
        const woi_flux_desc &f = flux[i];
        if (f.n_coef < 0 || (f.n_coef > 0 && !f.coef)) return fail(WOI_E_INVALID_ARG, "flux[%d]: bad coefficients", i);
        std::vector<double> c(f.coef, f.coef + f.n_coef);
        basis[i] = f.basis;
        off[i] = (int)coef.size();
        nc[i] = f.n_coef;
        const woi_surface_desc &s = g->surf[i];
        switch (f.basis) {
        case WOI_FLUX_ZERO:
            break;
        case WOI_FLUX_FOURIER: {
            if (d != 2) return fail(WOI_E_UNSUPPORTED, "flux[%d]: Fourier data need a 2D surface", i);
            if (f.n_coef < 1 || f.n_coef % 2 == 0) return fail(WOI_E_INVALID_ARG, "flux[%d]: Fourier needs 2K+1 coefficients", i);
            // int b ds and int |b| ds by the trapezoidal rule in the parameter (spectrally accurate)
            const int m = 4096;
            double I = 0.0, I1 = 0.0;
            for (int j = 0; j < m; ++j) {
                double t = 2.0 * kPi * j / m;
                double ds = (s.type == WOI_STAR) ? g->star.speed(t) : s.radius;
                double b = fourier_eval(c, t);
                I += b * ds;
                I1 += std::fabs(b) * ds;
            }
            if (std::fabs(I) > 1e-10 * std::max(I1, 1e-300) && std::fabs(I) > 1e-300)
                return fail(WOI_E_COMPAT, "flux[%d]: int b dA = %.3e is not zero (|b|_1 = %.3e)", i, I, I1);
            break;
        }
        case WOI_FLUX_REAL_SH: {
            if (d != 3 || s.type != WOI_SPHERE) return fail(WOI_E_UNSUPPORTED, "flux[%d]: spherical harmonics need a 3D sphere", i);
            int L = (int)std::lround(std::sqrt((double)f.n_coef)) - 1;
            if (L < 0 || (L + 1) * (L + 1) != f.n_coef || L > 4)
                return fail(WOI_E_INVALID_ARG, "flux[%d]: need (L+1)^2 coefficients with L <= 4", i);
            double tot = 0.0;
            for (double v : c) tot += std::fabs(v);
            if (std::fabs(c[0]) > 1e-10 * tot) return fail(WOI_E_COMPAT, "flux[%d]: Y_0^0 coefficient must be zero", i);
            break;
        }
        case WOI_FLUX_HARMONIC_POLY: {
            if (f.n_coef < 2) return fail(WOI_E_INVALID_ARG, "flux[%d]: harmonic polynomial needs [s, T, ...]", i);
            int T = (int)c[1];
            if (T < 0 || (double)T != c[1] || f.n_coef != 2 + T * (d + 1))
                return fail(WOI_E_INVALID_ARG, "flux[%d]: harmonic polynomial layout [s, T, (c, e_1..e_d) x T]", i);
            for (int t = 0; t < T; ++t)
                for (int k = 0; k < d; ++k) {
                    double e = c[2 + t * (d + 1) + 1 + k];
                    if (e < 0 || e != std::floor(e) || e > 16) return fail(WOI_E_INVALID_ARG, "flux[%d]: bad exponent", i);
                }
            double sc;
            if (!poly_is_harmonic(d, T, c.data() + 2, &sc))
                return fail(WOI_E_COMPAT, "flux[%d]: the polynomial is not harmonic, its flux is not compatible", i);
            break;
        }
        case WOI_FLUX_POINT_CHARGE: {
            if (d < 3) return fail(WOI_E_UNSUPPORTED, "flux[%d]: the point-charge datum needs dim >= 3", i);
            if (f.n_coef != 1 + d) return fail(WOI_E_INVALID_ARG, "flux[%d]: point charge needs [s, x0_1..x0_d]", i);
            // the charge must lie outside the region the surface bounds: then d_n |y - x0|^{2-d}
            // integrates to zero over the surface (the potential is harmonic inside)
            const double *x0 = c.data() + 1;
            const bool outside = s.type == WOI_ELLIPSOID ? ellipsoid_form(*g, i, x0) > 1.0 + 1e-12
                                 : s.type == WOI_MESH   ? !inside_surface(*g, i, x0)
                                                        : dist(d, x0, s.center) > s.radius * (1.0 + 1e-12);
            if (!outside) return fail(WOI_E_COMPAT, "flux[%d]: the charge lies inside the surface, int b dA != 0", i);
            break;
        }
        default:
            return fail(WOI_E_INVALID_ARG, "flux[%d]: unknown basis %d", i, f.basis);
        }
        coef.insert(coef.end(), c.begin(), c.end());
    }
    // Sec. 3: alpha_1 = 2, alpha_i = 2 (sigma_i - sigma_p) / (sigma_p + sigma_i);
    //         beta_1 = (2 / sigma_1) b_1, beta_i = -2 b_i / (sigma_p + sigma_i)
    std::vector<double> alpha(n), bsc(n);
    for (int i = 0; i < n; ++i) {
        if (i == 0) {
            alpha[i] = 2.0;
            bsc[i] = 2.0 / sigma[0];
        } else {
            const double sp = sigma[g->parent[i]], si = sigma[i];
            alpha[i] = 2.0 * (si - sp) / (sp + si);
            bsc[i] = -2.0 / (sp + si);
        }
    }
    // Thm 4.2: P(H = n) = |alpha_n| / A; thresholds T_n = floor(2^32 C_n / A), T_N = 2^32
    double A = 0.0;
    for (int i = 0; i < n; ++i) A += std::fabs(alpha[i]);
    std::vector<uint64_t> th(n);
    double C = 0.0;
    for (int i = 0; i < n; ++i) {
        C += std::fabs(alpha[i]);
        th[i] = (uint64_t)std::floor(std::ldexp(C / A, 32));
    }
    th[n - 1] = 1ull << 32;
    // Sec. 4.4: arcs of dOmega^+ = {beta >= 0} and dOmega^- = {beta < 0} (2D Fourier data;
    // other 2D data is marked -1 and its start is drawn from uniform trials, as in d >= 3)
    bool vr_ok = (d == 2);
    std::vector<double> at0, at1, alen, as0, plen(2 * n, 0.0);
    std::vector<int> asg, aoff(n, 0), an(n, 0);
    for (int i = 0; i < n && vr_ok; ++i) {
        aoff[i] = (int)at0.size();
        const woi_surface_desc &s = g->surf[i];
        auto arc_length = [&](double t0, double t1) {
            if (s.type == WOI_SPHERE) return s.radius * (t1 - t0);
            return star_length(g->star, t0, t1, 64);
        };
        auto arc_start = [&](double t0) {
            if (s.type == WOI_SPHERE) return s.radius * t0;
            const double H = 2.0 * kPi / kNodes;
            int j = std::min(kNodes - 1, std::max(0, (int)(t0 / H)));
            return g->star_panel_s[j] + star_length(g->star, j * H, t0, 4);
        };
        if (basis[i] == WOI_FLUX_ZERO) {
            at0.push_back(0.0); at1.push_back(2.0 * kPi); asg.push_back(1);
            alen.push_back(g->area[i]);
            as0.push_back(0.0);
            plen[2 * i] += g->area[i];
            an[i] = 1;
            continue;
        }
        if (basis[i] != WOI_FLUX_FOURIER) {
            // other 2D data: parts of no closed form, the start is drawn from uniform trials
            plen[2 * i] = plen[2 * i + 1] = -1.0;
            continue;
        }
        std::vector<double> c(coef.begin() + off[i], coef.begin() + off[i] + nc[i]);
        auto beta = [&](double t) { return bsc[i] * fourier_eval(c, t); };
        const int m = 8192;
        std::vector<double> cuts{0.0};
        double tp = 0.0, fp = beta(0.0);
        for (int j = 1; j <= m; ++j) {
            double t = 2.0 * kPi * j / m, f = beta(t);
            if ((fp < 0) != (f < 0)) {
                double lo = tp, hi = t, flo = fp;
                for (int it = 0; it < 200 && hi - lo > 1e-16; ++it) {
                    double mid = 0.5 * (lo + hi), fm = beta(mid);
                    if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else hi = mid;
                }
                cuts.push_back(0.5 * (lo + hi));
            }
            tp = t;
            fp = f;
        }
        cuts.push_back(2.0 * kPi);
        for (size_t j = 0; j + 1 < cuts.size(); ++j) {
            const double a = cuts[j], b = cuts[j + 1];
            if (!(b > a)) continue;
            const int sg = beta(0.5 * (a + b)) >= 0 ? 1 : -1;
            const double L = arc_length(a, b);
            at0.push_back(a); at1.push_back(b); asg.push_back(sg); alen.push_back(L);
            as0.push_back(arc_start(a));
            plen[2 * i + (sg > 0 ? 0 : 1)] += L;
            an[i]++;
        }
    }
    g->sigma.assign(sigma, sigma + n);
    g->alpha = alpha;
    g->beta_scale = bsc;
    g->alpha_l1 = A;
    g->thresh = th;
    g->flux_basis = basis;
    g->flux_off = off;
    g->flux_n = nc;
    g->flux_coef = coef;
    // device format: real spherical harmonics carry N_lm = sqrt((2l+1)/(4 pi) (l-|m|)!/(l+|m|)!)
    // and the sqrt(2) of m != 0, so that the kernels evaluate only the Legendre recursion
    g->flux_dev = coef;
    for (int i = 0; i < n; ++i) {
        if (basis[i] != WOI_FLUX_REAL_SH) continue;
        for (int idx = 0; idx < nc[i]; ++idx) {
            int l = 0;
            while ((l + 1) * (l + 1) <= idx) ++l;
            const int m = idx - l * l - l, am = m < 0 ? -m : m;
            double ratio = 1.0;
            for (int k = l - am + 1; k <= l + am; ++k) ratio /= k;
            const double nlm = std::sqrt((2.0 * l + 1.0) / (4.0 * kPi) * ratio) * (m == 0 ? 1.0 : std::sqrt(2.0));
            g->flux_dev[off[i] + idx] *= nlm;
        }
    }
    // device format: a harmonic polynomial of degree <= 3 becomes the dense quadratic form of
    // its gradient, dP/dy_k = a_k + sum_j b_kj y_j + sum_{j<=l} c_kjl y_j y_l, so that the
    // kernels evaluate it with fused multiply-adds instead of decoding monomials
    {
        std::vector<double> dev;
        g->flux_basis_dev.assign(n, 0);
        g->flux_off_dev.assign(n, 0);
        g->flux_n_dev.assign(n, 0);
        const int nq = d * d * (d + 1) / 2 + d * d + d;    // per surface after the scale s
        for (int i = 0; i < n; ++i) {
            const double *c = g->flux_dev.data() + off[i];
            bool quad = basis[i] == WOI_FLUX_HARMONIC_POLY;
            if (quad) {
                const int T = (int)c[1];
                for (int t = 0; t < T && quad; ++t) {
                    int deg = 0;
                    for (int k = 0; k < d; ++k) deg += (int)c[2 + t * (d + 1) + 1 + k];
                    quad = deg <= 3;
                }
            }
            g->flux_off_dev[i] = (int)dev.size();
            if (basis[i] == WOI_FLUX_REAL_SH && nc[i] <= 9) {
                // degree <= 2 on a sphere: a quadratic polynomial of the unit vector u (coefficients
                // here already carry N_lm and sqrt 2); P_2^0 = (3z^2 - 1)/2, P_2^1 cos = 3zx,
                // P_2^1 sin = 3zy, P_2^2 cos = 3(x^2 - y^2), P_2^2 sin = 6xy (no Condon-Shortley phase)
                double cf[9] = {0};
                for (int idx = 0; idx < nc[i]; ++idx) cf[idx] = c[idx];
                // indices l*l + l + m: (0,0) 0; (1,-1) 1, (1,0) 2, (1,1) 3; (2,-2) 4 ... (2,2) 8
                double q[10] = {0};
                q[0] = cf[0] - 0.5 * cf[6];                  // constant
                q[1] = cf[3]; q[2] = cf[1]; q[3] = cf[2];    // x, y, z
                q[4] = 3.0 * cf[8];                          // xx
                q[5] = 6.0 * cf[4];                          // xy
                q[6] = 3.0 * cf[7];                          // xz
                q[7] = -3.0 * cf[8];                         // yy
                q[8] = 3.0 * cf[5];                          // yz
                q[9] = 1.5 * cf[6];                          // zz
                g->flux_basis_dev[i] = kFluxSphQuad;
                g->flux_n_dev[i] = 10;
                dev.insert(dev.end(), q, q + 10);
                continue;
            }
            if (!quad) {
                g->flux_basis_dev[i] = basis[i];
                g->flux_n_dev[i] = nc[i];
                dev.insert(dev.end(), c, c + nc[i]);
                continue;
            }
            g->flux_basis_dev[i] = kFluxHarmonicQuad;
            g->flux_n_dev[i] = 1 + nq;
            std::vector<double> q(1 + nq, 0.0);
            q[0] = c[0];
            const int T = (int)c[1];
            const int per_k = 1 + d + d * (d + 1) / 2;
            for (int t = 0; t < T; ++t) {
                const double *row = c + 2 + t * (d + 1);
                for (int k = 0; k < d; ++k) {
                    int e[kMaxDim];
                    for (int j = 0; j < d; ++j) e[j] = (int)row[1 + j];
                    if (e[k] == 0) continue;
                    const double coef = row[0] * e[k];
                    e[k] -= 1;                              // the monomial of dP/dy_k, degree <= 2
                    int vars[2], nv = 0;
                    for (int j = 0; j < d; ++j)
                        for (int r = 0; r < e[j]; ++r) vars[nv++] = j;
                    double *qk = &q[1 + k * per_k];
                    if (nv == 0) {
                        qk[0] += coef;
                    } else if (nv == 1) {
                        qk[1 + vars[0]] += coef;
                    } else {
                        const int a = std::min(vars[0], vars[1]), b2 = std::max(vars[0], vars[1]);
                        qk[1 + d + a * d - a * (a - 1) / 2 + (b2 - a)] += coef;
                    }
                }
            }
            dev.insert(dev.end(), q.begin(), q.end());
        }
        g->flux_dev = dev;
    }
    g->flux_dev_f.assign(g->flux_dev.begin(), g->flux_dev.end());
    // Sec. 4.4 in d >= 3 (and the sign tolerance of 2D trial starts).  On a sphere, data linear in the unit vector u (degree-1 real
    // harmonics, harmonic polynomials of degree <= 1) is negative exactly on the mirror image
    // of the half where it is positive: the parts are hemispheres of half the area.  Zero data
    // puts the whole surface in dOmega^+.  Other data, and every ellipsoid and mesh, has parts
    // of no closed form, marked -1: the start is drawn from uniform trials (the areas are
    // estimated by the trials themselves).  vr_tol[i] (spheres with data in the quadratic
    // device formats) bounds where an FP32 evaluation of beta may have the wrong sign: 1e-4
    // of a bound on the magnitude of its terms (the FP32 error is about 1e-6 of it); below it
    // the kernels decide the sign in FP64.  Elsewhere it is 0 and the kernels decide in their
    // own precision.
    std::vector<double> vtol(n, 0.0);
    auto sign_tolerance = [&](int i) {
        // |terms| <= sum |q| rho^deg with rho = max |y_k| on the sphere (rho = 1 for u)
        const int fb = g->flux_basis_dev[i];
        if (g->surf[i].type != WOI_SPHERE || (fb != kFluxSphQuad && fb != kFluxHarmonicQuad)) return 0.0;
        const double *q = g->flux_dev.data() + g->flux_off_dev[i];
        double bound = 0.0;
        if (fb == kFluxSphQuad) {
            for (int k = 0; k < 10; ++k) bound += std::fabs(q[k]);
        } else {
            double rho = 1.0;
            for (int k = 0; k < d; ++k) rho = std::max(rho, std::fabs(g->surf[i].center[k]) + g->surf[i].radius);
            for (int k = 1; k < g->flux_n_dev[i]; ++k) bound += std::fabs(q[k]);
            bound *= std::fabs(q[0]) * rho * rho;
        }
        return 1e-4 * std::fabs(bsc[i]) * bound;
    };
    if (d == 2)
        for (int i = 0; i < n; ++i)
            if (plen[2 * i] < 0.0) vtol[i] = sign_tolerance(i);
    if (d >= 3) {
        vr_ok = true;
        for (int i = 0; i < n; ++i) {
            if (basis[i] == WOI_FLUX_ZERO) { plen[2 * i] = g->area[i]; continue; }
            plen[2 * i] = plen[2 * i + 1] = -1.0;
            const int fb = g->flux_basis_dev[i];
            if (g->surf[i].type != WOI_SPHERE || (fb != kFluxSphQuad && fb != kFluxHarmonicQuad)) continue;
            const double *c = coef.data() + off[i];
            bool linear = true;
            if (basis[i] == WOI_FLUX_REAL_SH) {
                for (int idx = 0; idx < nc[i]; ++idx)
                    if ((idx < 1 || idx > 3) && c[idx] != 0.0) linear = false;
            } else {
                const int T = (int)c[1];
                for (int t = 0; t < T; ++t) {
                    double deg = 0.0;
                    for (int k = 0; k < d; ++k) deg += c[2 + t * (d + 1) + 1 + k];
                    if (deg > 1.0) linear = false;
                }
            }
            if (linear) plen[2 * i] = plen[2 * i + 1] = 0.5 * g->area[i];
            vtol[i] = sign_tolerance(i);
        }
    }
    g->vr_tol = vtol;
    g->vr_ok = vr_ok;
    g->arc_t0 = at0; g->arc_t1 = at1; g->arc_len = alen; g->arc_s0 = as0; g->arc_sign = asg;
    g->arc_off = aoff; g->arc_n = an; g->part_len = plen;
    g->data_ready = true;
    g->dev_dirty = true;
    g->blob_M = -1;
    return WOI_OK;
}

void woi_destroy_geometry(woi_geometry *g) { delete g; }

}  // extern "C"

// ---------------------------------------------------------------------------
// device staging and launches
// ---------------------------------------------------------------------------
namespace {

// ---------------------------------------------------------------------------
// autotuned launch shapes: (dim, star, variant, sched_group, M) -> (block, walks per lane)
// ---------------------------------------------------------------------------
std::map<uint64_t, std::pair<int, int>> g_tune;
bool g_tune_loaded = false;

uint64_t tune_key(int dim, bool star, int variant, int sched_group, int M)
{
    return ((uint64_t)dim << 40) | ((uint64_t)star << 32) | ((uint64_t)variant << 24) | ((uint64_t)sched_group << 8) |
           (uint64_t)M;
}

void tune_load()
{
    if (g_tune_loaded) return;
    g_tune_loaded = true;
    const char *path = std::getenv("WOI_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "r");
    if (!f) return;
    unsigned long long k;
    int b, l;
    // one entry per line: {"key": K, "block": B, "walks_per_lane": L}
    while (std::fscanf(f, " {\"key\": %llu, \"block\": %d, \"walks_per_lane\": %d}", &k, &b, &l) == 3)
        g_tune[(uint64_t)k] = {b, l};
    std::fclose(f);
}

void tune_save()
{
    const char *path = std::getenv("WOI_TUNE_CACHE");
    if (!path) return;
    FILE *f = std::fopen(path, "w");
    if (!f) return;
    for (auto &kv : g_tune)
        std::fprintf(f, "{\"key\": %llu, \"block\": %d, \"walks_per_lane\": %d}\n", (unsigned long long)kv.first,
                     kv.second.first, kv.second.second);
    std::fclose(f);
}

// launch shape of the FP32 walk kernel: explicit options, else the tuned table, else 256
// threads x default_L walks per lane
void launch_shape(const woi_opts *o, int dim, bool star, int *block, int *L, int default_L = 32)
{
    *block = o->block_size;
    *L = o->walks_per_lane;
    if (*block == 0 && *L == 0) {
        tune_load();
        auto it = g_tune.find(tune_key(dim, star, o->variant, o->sched_group, o->M));
        if (it != g_tune.end()) {
            *block = it->second.first;
            *L = it->second.second;
        }
    }
    if (*block == 0) *block = 256;
    if (*L == 0) *L = default_L;
}

woi_status ensure_device(woi_geometry *g)
{
    int count = 0;
    cudaError_t e = cudaGetDeviceCount(&count);
    if (e != cudaSuccess || count == 0) {
        cudaGetLastError();
        return fail(WOI_E_NO_DEVICE, "no CUDA device (%s)", cudaGetErrorString(e));
    }
    int dev = 0;
    WOI_CUDA(cudaGetDevice(&dev));
    if (g->device >= 0 && g->device != dev) g->release();
    if (g->device < 0) {
        g->device = dev;
        g->dev_dirty = true;
        WOI_CUDA(cudaDeviceGetAttribute(&g->num_sms, cudaDevAttrMultiProcessorCount, dev));
    }
    return WOI_OK;
}

template <typename T>
woi_status upload(T **dst, const std::vector<T> &src, cudaStream_t s)
{
    cudaFree(*dst);
    *dst = nullptr;
    size_t bytes = std::max<size_t>(1, src.size()) * sizeof(T);
    WOI_CUDA(cudaMalloc((void **)dst, bytes));
    if (!src.empty()) WOI_CUDA(cudaMemcpyAsync(*dst, src.data(), src.size() * sizeof(T), cudaMemcpyHostToDevice, s));
    return WOI_OK;
}

// the host image of the blob for truncation M (device pointers are set by the caller)
void fill_blob(const woi_geometry &g, int M, DevGeom &b)
{
    std::memset(&b, 0, sizeof(b));
    b.dim = g.dim;
    b.n = g.n;
    b.npad = 1;
    while (b.npad < g.n) b.npad <<= 1;
    b.M = M;
    b.star_idx = g.star_idx;
    b.star_K = g.star_idx >= 0 ? g.star.K : 0;
    b.star_lmax = g.star_lmax;
    b.star_kpp = g.star_kpp;
    b.star_k3 = g.star_k3;
    if (g.star_idx >= 0) {
        // r(t) (cos t, sin t) as a trigonometric polynomial of degree K + 1: cos kt cos t =
        // (cos (k+1)t + cos (k-1)t) / 2 and the like
        const double R = g.star.R;
        b.star_harm[1][0] += R;                            // R cos t
        b.star_harm[1][3] += R;                            // R sin t
        for (int k = 1; k <= g.star.K; ++k) {
            const double a = 0.5 * R * g.star.a[k], c = 0.5 * R * g.star.b[k];
            b.star_harm[k + 1][0] += a;  b.star_harm[k - 1][0] += a;    // a_k cos kt cos t
            b.star_harm[k + 1][1] += c;  b.star_harm[k - 1][1] += c;    // b_k sin kt cos t
            b.star_harm[k + 1][3] += a;  b.star_harm[k - 1][3] -= a;    // a_k cos kt sin t
            b.star_harm[k - 1][2] += c;  b.star_harm[k + 1][2] -= c;    // b_k sin kt sin t
        }
    }
    b.star_rmin = g.star_rmin;
    b.star_rmax = g.star_rmax;
    for (int i = 0; i < kMaxSurfPad; ++i) b.sched_tm1[i] = i < g.n ? (uint32_t)(g.thresh[i] - 1) : 0xFFFFFFFFu;
    {
        int n = 0;   // bucket k: the first surface whose threshold T_n - 1 reaches k 2^24
        for (int k = 0; k <= kSchedBuckets; ++k) {
            const uint64_t start = (uint64_t)k << 24;
            while (n < g.n - 1 && (uint64_t)b.sched_tm1[n] < start) ++n;
            b.sched_bucket[k] = n;
        }
    }
    for (int i = 0; i < g.n; ++i) {
        for (int k = 0; k < g.dim; ++k) b.center[i][k] = g.surf[i].center[k];
        b.radius[i] = g.surf[i].radius;
        b.area[i] = g.area[i];
        b.alpha_sign[i] = g.alpha[i] > 0 ? 1.0 : (g.alpha[i] < 0 ? -1.0 : 0.0);
        b.beta_scale[i] = g.beta_scale[i];
        b.tin[i] = g.tin[i];
        b.tout[i] = g.tout[i];
        b.type[i] = g.surf[i].type;
        b.flux_basis[i] = g.flux_basis_dev[i];
        b.flux_off[i] = g.flux_off_dev[i];
        b.flux_n[i] = g.flux_n_dev[i];
        b.part_len[i][0] = g.part_len.empty() ? 0.0 : g.part_len[2 * i];
        b.part_len[i][1] = g.part_len.empty() ? 0.0 : g.part_len[2 * i + 1];
        b.vr_tol[i] = g.vr_tol.empty() ? 0.0 : g.vr_tol[i];
        b.arc_off[i] = g.arc_off.empty() ? 0 : g.arc_off[i];
        b.arc_n[i] = g.arc_n.empty() ? 0 : g.arc_n[i];
        b.ell_slot[i] = g.ell_slot[i];
    }
    // N w_i ||alpha||_1^i (Eq. woi_estimator with w_i = 1 - delta_iM / 2)
    double Ai = 1.0;
    for (int i = 0; i <= M; ++i) {
        b.coef[i] = (double)g.n * (i == M ? 0.5 : 1.0) * Ai;
        Ai *= g.alpha_l1;
    }
    for (int j = 0; j < kNodes; ++j) {
        b.node_cs[j][0] = std::cos(2.0 * kPi * j / kNodes);
        b.node_cs[j][1] = std::sin(2.0 * kPi * j / kNodes);
    }
    if (g.star_idx >= 0) {
        for (int k = 1; k <= g.star.K; ++k) {
            b.star_a[k] = g.star.a[k];
            b.star_b[k] = g.star.b[k];
        }
        for (int j = 0; j < kNodes; ++j) {
            b.star_scan[j][0] = g.star_scan[2 * j];
            b.star_scan[j][1] = g.star_scan[2 * j + 1];
            b.star_scan_d[j][0] = g.star_scan_d[2 * j];
            b.star_scan_d[j][1] = g.star_scan_d[2 * j + 1];
        }
        for (int j = 0; j <= kNodes; ++j) b.star_panel_s[j] = g.star_panel_s[j];
    }
    b.n_mesh = (int)g.mesh.size();
    for (int i = 0; i < g.n; ++i) b.mesh_slot[i] = g.mesh_slot[i];
    {
        int tri_off = 0, node_off = 0;
        for (int m = 0; m < b.n_mesh; ++m) {
            b.mesh_tri_off[m] = tri_off;
            b.mesh_ntri[m] = g.mesh[m].ntri;
            b.mesh_node_off[m] = node_off;
            b.mesh_scale[m] = g.mesh[m].scale;
            tri_off += g.mesh[m].ntri;
            node_off += (int)g.mesh[m].wide.size();
        }
    }
    b.n_ell = (int)g.ell.size();
    for (int e = 0; e < b.n_ell; ++e) {
        for (int a = 0; a < kMaxDim; ++a)
            for (int c = 0; c < kMaxDim; ++c) {
                b.ell_A[e][a][c] = g.ell[e].A[a][c];
                b.ell_map[e][a][c] = g.ell[e].map[a][c];
            }
        b.ell_jmax[e] = g.ell[e].jmax;
    }
}

// build the blob (and per-M coefficients) and copy it to the device
woi_status stage_geometry(woi_geometry *g, int M, cudaStream_t s)
{
    if (!g->dev_dirty && g->blob_M == M) return WOI_OK;
    woi_status st;
    if (g->dev_dirty) {
        if ((st = upload(&g->d_flux, g->flux_dev, s)) != WOI_OK) return st;
        if ((st = upload(&g->d_flux_f, g->flux_dev_f, s)) != WOI_OK) return st;
        if ((st = upload(&g->d_arc_t0, g->arc_t0, s)) != WOI_OK) return st;
        if ((st = upload(&g->d_arc_t1, g->arc_t1, s)) != WOI_OK) return st;
        if ((st = upload(&g->d_arc_len, g->arc_len, s)) != WOI_OK) return st;
        if ((st = upload(&g->d_arc_s0, g->arc_s0, s)) != WOI_OK) return st;
        if ((st = upload(&g->d_arc_sign, g->arc_sign, s)) != WOI_OK) return st;
        if (!g->mesh.empty()) {
            // all meshes concatenated: triangle rows, thresholds and hierarchies (internal
            // children shifted by the mesh's entry offset, leaf triangles by its triangle offset)
            std::vector<double> tri_d;
            std::vector<uint32_t> tm1;
            std::vector<int> bucket;
            std::vector<BvhWide> nodes;
            for (const MeshHost &mh : g->mesh) {
                const int tri_off = (int)tm1.size(), node_off = (int)nodes.size();
                tri_d.insert(tri_d.end(), mh.tri.begin(), mh.tri.end());
                tm1.insert(tm1.end(), mh.tm1.begin(), mh.tm1.end());
                // bucket b: the first triangle whose threshold T_j - 1 reaches b 2^22
                int j = 0;
                for (int b = 0; b <= kTriBuckets; ++b) {
                    const uint64_t start = (uint64_t)b << 22;
                    while (j < mh.ntri && (uint64_t)mh.tm1[j] < start) ++j;
                    bucket.push_back(tri_off + std::min(j, mh.ntri - 1));
                }
                for (BvhWide nd : mh.wide) {
                    for (int c = 0; c < 2; ++c) {   // internal: entry + node_off; leaf: -(t + tri_off + 1)
                        const int ch = nd.child[c];
                        if (ch >= (int)mh.wide.size() || ch < -mh.ntri)
                            return fail(WOI_E_GEOMETRY, "mesh hierarchy reference %d out of range", ch);
                        nd.child[c] = ch >= 0 ? ch + node_off : ch - tri_off;
                    }
                    nodes.push_back(nd);
                }
            }
            std::vector<float> tri_f(tri_d.begin(), tri_d.end());
            if ((st = upload(&g->d_tri_d, tri_d, s)) != WOI_OK) return st;
            if ((st = upload(&g->d_tri_f, tri_f, s)) != WOI_OK) return st;
            if ((st = upload(&g->d_tri_tm1, tm1, s)) != WOI_OK) return st;
            if ((st = upload(&g->d_tri_bucket, bucket, s)) != WOI_OK) return st;
            if ((st = upload(&g->d_bvh, nodes, s)) != WOI_OK) return st;
            if (!g->d_mesh_overflow) WOI_CUDA(cudaMalloc((void **)&g->d_mesh_overflow, sizeof(unsigned int)));
            WOI_CUDA(cudaMemsetAsync(g->d_mesh_overflow, 0, sizeof(unsigned int), s));
            // the host vectors die at the end of this block: finish the pageable copies first
            WOI_CUDA(cudaStreamSynchronize(s));
        }
        if (!g->d_blob) WOI_CUDA(cudaMalloc((void **)&g->d_blob, sizeof(DevGeom)));
    }
    DevGeom &b = g->blob;
    fill_blob(*g, M, b);
    b.flux_coef = g->d_flux;
    b.flux_coef_f = g->d_flux_f;
    b.arc_t0 = g->d_arc_t0;
    b.arc_t1 = g->d_arc_t1;
    b.arc_len = g->d_arc_len;
    b.arc_s0 = g->d_arc_s0;
    b.arc_sign = g->d_arc_sign;
    b.tri_f = g->d_tri_f;
    b.tri_d = g->d_tri_d;
    b.tri_tm1 = g->d_tri_tm1;
    b.tri_bucket = g->d_tri_bucket;
    b.bvh = g->d_bvh;
    b.mesh_overflow = g->d_mesh_overflow;
    // pageable source: the copy is staged before cudaMemcpyAsync returns
    WOI_CUDA(cudaMemcpyAsync(g->d_blob, &b, sizeof(DevGeom), cudaMemcpyHostToDevice, s));
    g->dev_dirty = false;
    g->blob_M = M;
    return WOI_OK;
}

woi_status ensure_scratch(woi_geometry *g, size_t bytes)
{
    if (g->scratch_bytes >= bytes) return WOI_OK;
    cudaFree(g->d_scratch);
    g->d_scratch = nullptr;
    g->scratch_bytes = 0;
    size_t want = std::max(bytes, (size_t)1 << 20);
    if (cudaMalloc(&g->d_scratch, want) != cudaSuccess) {
        cudaGetLastError();
        return fail(WOI_E_OOM, "device scratch allocation of %zu bytes failed", want);
    }
    g->scratch_bytes = want;
    return WOI_OK;
}

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

woi_status check_opts(const woi_geometry *g, const woi_opts *o, int64_t n_pts, int64_t walk_begin, int64_t n_walks)
{
    if (!g->data_ready) return fail(WOI_E_STATE, "woi_set_sigma_and_data has not been called");
    if (!o) return fail(WOI_E_INVALID_ARG, "null options");
    if (o->M < 0 || o->M > WOI_MAX_M) return fail(WOI_E_INVALID_ARG, "M = %d outside [0, %d]", o->M, WOI_MAX_M);
    if (o->variant != WOI_PLAIN && o->variant != WOI_VR) return fail(WOI_E_INVALID_ARG, "unknown variant %d", o->variant);
    if (o->precision != WOI_MIXED && o->precision != WOI_FP64_PLAIN)
        return fail(WOI_E_INVALID_ARG, "unknown precision %d", o->precision);
    if (o->sched_group != 1 && o->sched_group != 32) return fail(WOI_E_INVALID_ARG, "sched_group must be 1 or 32");
    if (n_pts < 0 || n_walks < 1 || walk_begin < 0) return fail(WOI_E_INVALID_ARG, "need n_pts >= 0, n_walks >= 1");
    if (n_walks % o->sched_group || walk_begin % o->sched_group)
        return fail(WOI_E_INVALID_ARG, "walk range must be a multiple of sched_group");
    if (o->variant == WOI_VR && !g->vr_ok)
        return fail(WOI_E_UNSUPPORTED, "variance reduction is not available for this geometry");
    if (o->block_size != 0 && (o->block_size % 32 || o->block_size < 32 || o->block_size > kMixedMaxBlock))
        return fail(WOI_E_INVALID_ARG, "block_size must be a multiple of 32 in [32, %d]", kMixedMaxBlock);
    if (o->walks_per_lane < 0 || o->walks_per_lane > 4096) return fail(WOI_E_INVALID_ARG, "walks_per_lane out of range");
    if (o->tile_points != 0 && o->tile_points != kTile)
        return fail(WOI_E_INVALID_ARG, "tile_points must be 0 or %d", kTile);
    if (o->tile_points && o->precision != WOI_MIXED)
        return fail(WOI_E_UNSUPPORTED, "shared trajectories run in mixed precision only");
    return WOI_OK;
}

// points of the call on the device (staged copy for host input); host input is checked to lie inside
woi_status stage_points(woi_geometry *g, const double *points, int64_t n_pts, const double **d_points, void *staging,
                        cudaStream_t s)
{
    if (pointer_on_device(points)) {
        *d_points = points;
        return WOI_OK;
    }
    for (int64_t p = 0; p < n_pts; ++p)
        if (!inside_surface(*g, 0, points + p * g->dim))
            return fail(WOI_E_GEOMETRY, "point %lld lies outside the outer surface", (long long)p);
    WOI_CUDA(cudaMemcpyAsync(staging, points, (size_t)n_pts * g->dim * sizeof(double), cudaMemcpyHostToDevice, s));
    *d_points = (const double *)staging;
    return WOI_OK;
}

// lines of the last call that crossed a mesh more than kMaxHits times (the crossing lists were
// truncated): read after the call's work has finished, cleared, and reported as WOI_E_GEOMETRY
woi_status take_mesh_overflow(woi_geometry *g)
{
    g->check_pending = false;
    if (!g->d_mesh_overflow) return WOI_OK;
    unsigned int over = 0;
    WOI_CUDA(cudaMemcpy(&over, g->d_mesh_overflow, sizeof(over), cudaMemcpyDeviceToHost));
    if (!over) return WOI_OK;
    WOI_CUDA(cudaMemset(g->d_mesh_overflow, 0, sizeof(over)));
    return fail(WOI_E_GEOMETRY, "%u lines crossed a mesh more than %d times; estimates are invalid", over, kMaxHits);
}

struct OutBuf {
    double *user;
    bool on_dev;
    double *dev;
    size_t count;
};

woi_status run_estimate(woi_geometry *g, const woi_opts *o, const double *points, int64_t n_pts, int64_t walk_begin,
                        int64_t n_walks, uint64_t seed, double *u, double *grad, double *se_u, double *se_grad,
                        double *moments, uint32_t instance_id = 0)
{
    woi_status st;
    if ((st = check_opts(g, o, n_pts, walk_begin, n_walks)) != WOI_OK) return st;
    if (!points && n_pts > 0) return fail(WOI_E_INVALID_ARG, "null points");
    if ((st = ensure_device(g)) != WOI_OK) return st;
    if (n_pts == 0) return WOI_OK;
    cudaStream_t s = (cudaStream_t)o->cuda_stream;
    const int d = g->dim, C = d + 1;
    const bool vr = o->variant == WOI_VR, star = g->general(), fp64 = o->precision == WOI_FP64_PLAIN;
    if ((st = stage_geometry(g, o->M, s)) != WOI_OK) return st;
    // the mesh crossing-overflow counter counts this call's lines only
    if (g->d_mesh_overflow) WOI_CUDA(cudaMemsetAsync(g->d_mesh_overflow, 0, sizeof(unsigned int), s));

    int block, L;
    launch_shape(o, d, star, &block, &L);
    const bool tiled = o->tile_points != 0;
    if (tiled) {
        // per round a lane runs one walk and tallies 32: fewer walks per unit keep the queue balanced
        block = kSharedBlock;
        L = o->walks_per_lane > 0 ? o->walks_per_lane : 8;
    }
    const int64_t unit_walks = 32LL * L;       // warp-level work units
    const int64_t chunks = fp64 ? 1 : (n_walks + unit_walks - 1) / unit_walks;
    const int64_t n_tiles = (n_pts + kTile - 1) / kTile;
    const int64_t units = tiled ? n_tiles * chunks : n_pts * chunks;
    const int64_t rows = tiled ? units * kTile : units;

    // scratch layout: [inst desc][queue][partials][points][outputs]
    size_t off = 0;
    const size_t o_desc = off; off = align_up(off + sizeof(InstDesc), 256);
    const size_t o_queue = off; off = align_up(off + sizeof(unsigned long long), 256);
    const size_t o_part = off; off = align_up(off + (size_t)rows * 2 * C * sizeof(double), 256);
    const size_t o_pts = off; off = align_up(off + (size_t)n_pts * d * sizeof(double), 256);
    OutBuf outs[5] = {{u, false, nullptr, (size_t)n_pts}, {grad, false, nullptr, (size_t)n_pts * d},
                      {se_u, false, nullptr, (size_t)n_pts}, {se_grad, false, nullptr, (size_t)n_pts * d},
                      {moments, false, nullptr, (size_t)n_pts * 2 * C}};
    size_t o_out[5];
    for (int k = 0; k < 5; ++k) {
        outs[k].on_dev = pointer_on_device(outs[k].user);
        o_out[k] = off;
        if (outs[k].user && !outs[k].on_dev) off = align_up(off + outs[k].count * sizeof(double), 256);
    }
    if ((st = ensure_scratch(g, off)) != WOI_OK) return st;
    char *base = (char *)g->d_scratch;
    for (int k = 0; k < 5; ++k)
        outs[k].dev = !outs[k].user ? nullptr : (outs[k].on_dev ? outs[k].user : (double *)(base + o_out[k]));

    const double *d_points = nullptr;
    if ((st = stage_points(g, points, n_pts, &d_points, base + o_pts, s)) != WOI_OK) return st;
    if (o->timing && !g->ev_start) {
        WOI_CUDA(cudaEventCreate(&g->ev_start));
        WOI_CUDA(cudaEventCreate(&g->ev_stop));
    }
    g->timed = o->timing != 0;

    FinalizeParams fp{};
    fp.dim = d;
    fp.n_pts = n_pts;
    fp.n_walks = n_walks;
    fp.sched_group = o->sched_group;
    fp.unit_begin = 0;
    fp.chunks_per_point = chunks;
    fp.partials = (const double *)(base + o_part);
    fp.tile = tiled ? kTile : 0;
    fp.u = outs[0].dev;
    fp.grad = outs[1].dev;
    fp.se_u = outs[2].dev;
    fp.se_grad = outs[3].dev;
    fp.moments = outs[4].dev;

    if (!fp64) {
        InstDesc desc{};
        desc.geom = g->d_blob;
        desc.points = d_points;
        desc.n_pts = n_pts;
        desc.n_walks = n_walks;
        desc.walk_begin = walk_begin;
        desc.unit_begin = 0;
        desc.chunks_per_point = chunks;
        desc.instance_id = instance_id;
        desc.sched_group = o->sched_group;
        WOI_CUDA(cudaMemcpyAsync(base + o_desc, &desc, sizeof(desc), cudaMemcpyHostToDevice, s));
        WOI_CUDA(cudaMemsetAsync(base + o_queue, 0, sizeof(unsigned long long), s));
        const size_t smem = tiled ? (size_t)(kSharedBlock / 32) * (vr ? 2 : 1) * (o->M + 1) * 32 * shared_record_floats(d) *
                                        sizeof(float)
                                  : (size_t)(block / 32) * g->n * kMaxDim * sizeof(float);
        long long key = ((long long)tiled << 40) | ((long long)o->M << 32) | ((long long)d << 20) | ((long long)vr << 19) |
                        ((long long)star << 18) | ((long long)g->n << 10) | block;
        int per_sm = 0;
        auto it = g->occ_cache.find(key);
        if (it == g->occ_cache.end()) {
            if (tiled) WOI_CUDA(shared_occupancy(d, vr, star, smem, &per_sm));
            else WOI_CUDA(mixed_warp_occupancy(d, vr, star, block, smem, &per_sm));
            g->occ_cache[key] = per_sm;
        } else {
            per_sm = it->second;
        }
        if (per_sm < 1) return fail(WOI_E_UNSUPPORTED, "walk kernel does not fit on an SM (M = %d)", o->M);
        const int64_t warps = units;
        const int64_t grid = std::min<int64_t>((int64_t)g->num_sms * per_sm, (warps + block / 32 - 1) / (block / 32));
        MixedParams mp{};
        mp.inst = (const InstDesc *)(base + o_desc);
        mp.n_inst = 1;
        mp.total_units = units;
        mp.queue = (unsigned long long *)(base + o_queue);
        mp.partials = (double *)(base + o_part);
        mp.walks_per_lane = L;
        mp.seed = seed;
        if (o->timing) WOI_CUDA(cudaEventRecord(g->ev_start, s));
        if (tiled) WOI_CUDA(launch_shared(d, vr, star, mp, (int)grid, smem, s));
        else WOI_CUDA(launch_mixed_warp(d, vr, star, mp, (int)grid, block, smem, s));
        if (o->timing) WOI_CUDA(cudaEventRecord(g->ev_stop, s));
        WOI_CUDA(launch_finalize(fp, false, s));
    } else {
        // plain FP64 baseline: one launch per evaluation point into [n_pts][2C] accumulators
        double *acc = (double *)(base + o_part);
        WOI_CUDA(cudaMemsetAsync(acc, 0, (size_t)n_pts * 2 * C * sizeof(double), s));
        if (o->timing) WOI_CUDA(cudaEventRecord(g->ev_start, s));
        for (int64_t p = 0; p < n_pts; ++p) {
            Fp64PointParams pp{};
            pp.geom = g->d_blob;
            pp.x = d_points + p * d;
            pp.point_id = (uint32_t)p;
            pp.instance_id = instance_id;
            pp.walk_begin = walk_begin;
            pp.n_walks = n_walks;
            pp.sched_group = o->sched_group;
            pp.seed = seed;
            pp.acc = acc + p * 2 * C;
            WOI_CUDA(launch_fp64_point(d, vr, star, pp, s));
        }
        if (o->timing) WOI_CUDA(cudaEventRecord(g->ev_stop, s));
        WOI_CUDA(launch_finalize(fp, true, s));
    }
    bool any_host = false;
    for (int k = 0; k < 5; ++k) {
        if (outs[k].user && !outs[k].on_dev) {
            WOI_CUDA(cudaMemcpyAsync(outs[k].user, outs[k].dev, outs[k].count * sizeof(double), cudaMemcpyDeviceToHost, s));
            any_host = true;
        }
    }
    if (any_host || !pointer_on_device(points)) {
        WOI_CUDA(cudaStreamSynchronize(s));
        return take_mesh_overflow(g);
    }
    if (g->d_mesh_overflow) {
        // asynchronous call on a mesh geometry: woi_check_status waits for this event and reads the counter
        if (!g->ev_done) WOI_CUDA(cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming));
        WOI_CUDA(cudaEventRecord(g->ev_done, s));
        g->check_pending = true;
    }
    return WOI_OK;
}

// ---------------------------------------------------------------------------
// batched estimate: one persistent launch per (dimension, star) group over the
// (instance, point, chunk) units of all its instances, a batched finalize, and
// the launch sequence kept as a CUDA graph that is replayed for a repeated batch
// ---------------------------------------------------------------------------
struct BatchState {
    int device = -1;
    void *scratch = nullptr;
    size_t bytes = 0;
    cudaStream_t own_stream = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<uint64_t> key;                 // signature of the captured batch
};
BatchState g_batch;

woi_status batch_scratch(size_t bytes)
{
    int dev = 0;
    WOI_CUDA(cudaGetDevice(&dev));
    if (g_batch.device != dev) {
        if (g_batch.exec) cudaGraphExecDestroy(g_batch.exec);
        g_batch = BatchState{};
        g_batch.device = dev;
    }
    if (g_batch.bytes >= bytes) return WOI_OK;
    cudaFree(g_batch.scratch);
    g_batch.scratch = nullptr;
    g_batch.bytes = 0;
    if (g_batch.exec) {
        cudaGraphExecDestroy(g_batch.exec);
        g_batch.exec = nullptr;
        g_batch.key.clear();
    }
    const size_t want = std::max(bytes, (size_t)1 << 22);
    if (cudaMalloc(&g_batch.scratch, want) != cudaSuccess) {
        cudaGetLastError();
        return fail(WOI_E_OOM, "batch scratch allocation of %zu bytes failed", want);
    }
    g_batch.bytes = want;
    return WOI_OK;
}

woi_status run_batch(int n_inst, woi_geometry *const *geoms, const woi_opts *o, const int *m_per_inst,
                     const double *const *points, const int64_t *n_pts, const int64_t *n_walks, uint64_t seed,
                     double *const *u, double *const *grad, double *const *se_u, double *const *se_grad)
{
    if (n_inst < 1 || !geoms || !o || !points || !n_pts || !n_walks) return fail(WOI_E_INVALID_ARG, "null argument");
    woi_status st;
    // validation with each instance's truncation
    std::vector<woi_opts> oi(n_inst, *o);
    for (int k = 0; k < n_inst; ++k) {
        if (!geoms[k]) return fail(WOI_E_INVALID_ARG, "null geometry %d", k);
        if (m_per_inst) oi[k].M = m_per_inst[k];
        if ((st = check_opts(geoms[k], &oi[k], n_pts[k], 0, n_walks[k])) != WOI_OK) return st;
        if (n_pts[k] > 0 && !points[k]) return fail(WOI_E_INVALID_ARG, "null points of instance %d", k);
    }
    if (o->precision == WOI_FP64_PLAIN) {
        // the FP64 baseline: instance by instance, one launch per point
        for (int k = 0; k < n_inst; ++k)
            if ((st = run_estimate(geoms[k], &oi[k], points[k], n_pts[k], 0, n_walks[k], seed, u ? u[k] : nullptr,
                                   grad ? grad[k] : nullptr, se_u ? se_u[k] : nullptr, se_grad ? se_grad[k] : nullptr,
                                   nullptr, (uint32_t)k)) != WOI_OK)
                return st;
        return WOI_OK;
    }
    for (int k = 0; k < n_inst; ++k)
        if ((st = ensure_device(geoms[k])) != WOI_OK) return st;
    cudaStream_t s = (cudaStream_t)o->cuda_stream;
    if (!s) {
        if (!g_batch.own_stream) WOI_CUDA(cudaStreamCreateWithFlags(&g_batch.own_stream, cudaStreamNonBlocking));
        s = g_batch.own_stream;
    }
    for (int k = 0; k < n_inst; ++k)
        if ((st = stage_geometry(geoms[k], oi[k].M, s)) != WOI_OK) return st;
    const bool vr = o->variant == WOI_VR;
    const int block = o->block_size ? o->block_size : 256;
    const int L = o->walks_per_lane ? o->walks_per_lane : 32;
    const int64_t unit_walks = 32LL * L;        // warp-level work units

    // groups of instances that share a kernel: (dimension, star)
    std::map<int, std::vector<int>> groups;
    for (int k = 0; k < n_inst; ++k)
        if (n_pts[k] > 0) groups[geoms[k]->dim * 2 + (int)geoms[k]->general()].push_back(k);

    // scratch layout: per group [InstDesc x n][queue][partials]; then staged points and outputs
    struct Group {
        int dim;
        bool star;
        std::vector<int> members;
        std::vector<InstDesc> desc;
        size_t o_desc, o_queue, o_part;
        int64_t units, points;
        int max_surf;
    };
    std::vector<Group> gs;
    size_t off = 0;
    for (auto &kv : groups) {
        Group gr;
        gr.dim = kv.first / 2;
        gr.star = kv.first % 2;
        gr.members = kv.second;
        gr.units = gr.points = 0;
        gr.max_surf = 1;
        for (int k : gr.members) {
            gr.max_surf = std::max(gr.max_surf, geoms[k]->n);
            const int64_t chunks = (n_walks[k] + unit_walks - 1) / unit_walks;
            InstDesc d{};
            d.geom = geoms[k]->d_blob;
            d.n_pts = n_pts[k];
            d.n_walks = n_walks[k];
            d.walk_begin = 0;
            d.unit_begin = gr.units;
            d.chunks_per_point = chunks;
            d.instance_id = (uint32_t)k;
            d.sched_group = o->sched_group;
            d.point_begin = gr.points;
            gr.units += n_pts[k] * chunks;
            gr.points += n_pts[k];
            gr.desc.push_back(d);
        }
        gr.o_desc = off; off = align_up(off + gr.desc.size() * sizeof(InstDesc), 256);
        gr.o_queue = off; off = align_up(off + gr.desc.size() * sizeof(unsigned long long), 256);
        gr.o_part = off; off = align_up(off + (size_t)gr.units * 2 * (gr.dim + 1) * sizeof(double), 256);
        gs.push_back(std::move(gr));
    }
    // staged host inputs / outputs
    std::vector<size_t> o_pts(n_inst, 0), o_out(4 * (size_t)n_inst, 0);
    std::vector<char> pts_host(n_inst, 0), out_host(4 * (size_t)n_inst, 0);
    double *const *outs[4] = {u, grad, se_u, se_grad};
    for (int k = 0; k < n_inst; ++k) {
        const int d = geoms[k]->dim;
        if (n_pts[k] > 0 && !pointer_on_device(points[k])) {
            pts_host[k] = 1;
            o_pts[k] = off;
            off = align_up(off + (size_t)n_pts[k] * d * sizeof(double), 256);
        }
        const size_t cnt[4] = {(size_t)n_pts[k], (size_t)n_pts[k] * d, (size_t)n_pts[k], (size_t)n_pts[k] * d};
        for (int j = 0; j < 4; ++j) {
            double *p = outs[j] ? outs[j][k] : nullptr;
            if (p && !pointer_on_device(p)) {
                out_host[4 * k + j] = 1;
                o_out[4 * k + j] = off;
                off = align_up(off + cnt[j] * sizeof(double), 256);
            }
        }
    }
    if ((st = batch_scratch(off)) != WOI_OK) return st;
    char *base = (char *)g_batch.scratch;
    for (int k = 0; k < n_inst; ++k) {
        if (!pts_host[k]) continue;
        for (int64_t q = 0; q < n_pts[k]; ++q)
            if (!inside_surface(*geoms[k], 0, points[k] + q * geoms[k]->dim))
                return fail(WOI_E_GEOMETRY, "instance %d: point %lld lies outside the outer surface", k, (long long)q);
        WOI_CUDA(cudaMemcpyAsync(base + o_pts[k], points[k], (size_t)n_pts[k] * geoms[k]->dim * sizeof(double),
                                 cudaMemcpyHostToDevice, s));
    }
    // descriptors (host copies are staged before cudaMemcpyAsync returns)
    std::vector<uint64_t> key{(uint64_t)n_inst, seed, (uint64_t)o->variant, (uint64_t)o->sched_group, (uint64_t)block,
                              (uint64_t)L, (uint64_t)(uintptr_t)base};
    for (auto &gr : gs) {
        for (size_t i = 0; i < gr.members.size(); ++i) {
            const int k = gr.members[i];
            InstDesc &d = gr.desc[i];
            d.points = pts_host[k] ? (const double *)(base + o_pts[k]) : points[k];
            double *dv[4];
            for (int j = 0; j < 4; ++j) {
                double *p = outs[j] ? outs[j][k] : nullptr;
                dv[j] = !p ? nullptr : (out_host[4 * k + j] ? (double *)(base + o_out[4 * k + j]) : p);
            }
            d.u = dv[0];
            d.grad = dv[1];
            d.se_u = dv[2];
            d.se_grad = dv[3];
            key.insert(key.end(), {(uint64_t)(uintptr_t)d.geom, (uint64_t)(uintptr_t)d.points, (uint64_t)d.n_pts,
                                   (uint64_t)d.n_walks, (uint64_t)oi[k].M, (uint64_t)(uintptr_t)dv[0],
                                   (uint64_t)(uintptr_t)dv[1], (uint64_t)(uintptr_t)dv[2], (uint64_t)(uintptr_t)dv[3]});
        }
        WOI_CUDA(cudaMemcpyAsync(base + gr.o_desc, gr.desc.data(), gr.desc.size() * sizeof(InstDesc),
                                 cudaMemcpyHostToDevice, s));
    }
    // the launch sequence, captured once per batch signature and replayed
    if (!(g_batch.exec && g_batch.key == key)) {
        if (g_batch.exec) {
            cudaGraphExecDestroy(g_batch.exec);
            g_batch.exec = nullptr;
        }
        std::vector<int> grid(gs.size());
        std::vector<size_t> smem(gs.size());
        int num_sms = geoms[0]->num_sms;
        for (size_t i = 0; i < gs.size(); ++i) {
            int per_sm = 0;
            smem[i] = (size_t)(block / 32) * gs[i].max_surf * kMaxDim * sizeof(float);
            WOI_CUDA(mixed_occupancy(gs[i].dim, vr, gs[i].star, block, smem[i], &per_sm));
            if (per_sm < 1) return fail(WOI_E_UNSUPPORTED, "batched walk kernel does not fit on an SM");
            const int64_t warps = gs[i].units, per_block = block / 32;
            grid[i] = (int)std::min<int64_t>((int64_t)num_sms * per_sm, (warps + per_block - 1) / per_block);
        }
        cudaGraph_t graph = nullptr;
        WOI_CUDA(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
        cudaError_t ce = cudaSuccess;
        for (size_t i = 0; i < gs.size() && ce == cudaSuccess; ++i) {
            Group &gr = gs[i];
            ce = cudaMemsetAsync(base + gr.o_queue, 0, gr.desc.size() * sizeof(unsigned long long), s);
            if (ce != cudaSuccess) break;
            MixedParams mp{};
            mp.inst = (const InstDesc *)(base + gr.o_desc);
            mp.n_inst = (int)gr.desc.size();
            mp.total_units = gr.units;
            mp.queue = (unsigned long long *)(base + gr.o_queue);
            mp.partials = (double *)(base + gr.o_part);
            mp.walks_per_lane = L;
            mp.seed = seed;
            mp.max_surf = gr.max_surf;
            ce = launch_mixed(gr.dim, vr, gr.star, mp, grid[i], block, smem[i], s);
            if (ce != cudaSuccess) break;
            BatchFinalizeParams bp{};
            bp.inst = (const InstDesc *)(base + gr.o_desc);
            bp.n_inst = (int)gr.desc.size();
            bp.dim = gr.dim;
            bp.total_points = gr.points;
            bp.partials = (const double *)(base + gr.o_part);
            ce = launch_finalize_batch(bp, s);
        }
        cudaError_t ee = cudaStreamEndCapture(s, &graph);
        if (ce != cudaSuccess || ee != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            return fail(WOI_E_CUDA, "batch capture failed: %s", cudaGetErrorString(ce != cudaSuccess ? ce : ee));
        }
        ce = cudaGraphInstantiate(&g_batch.exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ce != cudaSuccess) {
            g_batch.exec = nullptr;
            return fail(WOI_E_CUDA, "batch graph instantiation failed: %s", cudaGetErrorString(ce));
        }
        g_batch.key = key;
    }
    for (int k = 0; k < n_inst; ++k)
        if (geoms[k]->d_mesh_overflow) WOI_CUDA(cudaMemsetAsync(geoms[k]->d_mesh_overflow, 0, sizeof(unsigned int), s));
    if (o->timing) {
        // events of the first geometry time the whole batch launch
        woi_geometry *g0 = geoms[0];
        if (!g0->ev_start) {
            WOI_CUDA(cudaEventCreate(&g0->ev_start));
            WOI_CUDA(cudaEventCreate(&g0->ev_stop));
        }
        g0->timed = true;
        WOI_CUDA(cudaEventRecord(g0->ev_start, s));
    }
    WOI_CUDA(cudaGraphLaunch(g_batch.exec, s));
    if (o->timing) WOI_CUDA(cudaEventRecord(geoms[0]->ev_stop, s));
    for (int k = 0; k < n_inst; ++k) {
        const size_t cnt[4] = {(size_t)n_pts[k], (size_t)n_pts[k] * geoms[k]->dim, (size_t)n_pts[k],
                               (size_t)n_pts[k] * geoms[k]->dim};
        for (int j = 0; j < 4; ++j)
            if (out_host[4 * k + j])
                WOI_CUDA(cudaMemcpyAsync(outs[j][k], base + o_out[4 * k + j], cnt[j] * sizeof(double),
                                         cudaMemcpyDeviceToHost, s));
    }
    // the batch scratch and the captured graph are shared by batch calls: finish before returning
    WOI_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < n_inst; ++k)
        if ((st = take_mesh_overflow(geoms[k])) != WOI_OK) return st;
    return WOI_OK;
}

}  // namespace

extern "C" {

woi_status woi_estimate(woi_geometry *g, const woi_opts *opts, const double *points, int64_t n_pts, int64_t n_walks,
                        uint64_t seed, double *u, double *grad, double *se_u, double *se_grad)
{
    g_last_error.clear();
    if (!g) return fail(WOI_E_INVALID_ARG, "null geometry");
    return run_estimate(g, opts, points, n_pts, 0, n_walks, seed, u, grad, se_u, se_grad, nullptr);
}

woi_status woi_estimate_range(woi_geometry *g, const woi_opts *opts, const double *points, int64_t n_pts,
                              int64_t walk_begin, int64_t n_walks, uint64_t seed, double *moments)
{
    g_last_error.clear();
    if (!g) return fail(WOI_E_INVALID_ARG, "null geometry");
    if (!moments) return fail(WOI_E_INVALID_ARG, "null moments");
    return run_estimate(g, opts, points, n_pts, walk_begin, n_walks, seed, nullptr, nullptr, nullptr, nullptr, moments);
}

static woi_status walk_values_impl(woi_geometry *g, const woi_opts *o, const double *x, uint32_t point_id,
                                   uint32_t instance_id, const uint64_t *walk_ids, int64_t n, uint64_t seed, double *f_u,
                                   double *f_grad, double *trace)
{
    g_last_error.clear();
    if (!g || !o || !x || (n > 0 && (!walk_ids || !f_u || !f_grad))) return fail(WOI_E_INVALID_ARG, "null argument");
    woi_status st;
    if ((st = check_opts(g, o, 1, 0, o->sched_group)) != WOI_OK) return st;
    if (n < 0) return fail(WOI_E_INVALID_ARG, "n < 0");
    if ((st = ensure_device(g)) != WOI_OK) return st;
    if (n == 0) return WOI_OK;
    cudaStream_t s = (cudaStream_t)o->cuda_stream;
    const int d = g->dim;
    const int chains = o->variant == WOI_VR ? 2 : 1;
    const size_t trace_count = (size_t)n * chains * (o->M + 1) * (d + 2);
    if ((st = stage_geometry(g, o->M, s)) != WOI_OK) return st;
    size_t off = 0;
    const size_t o_x = off; off = align_up(off + d * sizeof(double), 256);
    const size_t o_w = off; off = align_up(off + n * sizeof(uint64_t), 256);
    const size_t o_u = off; off = align_up(off + n * sizeof(double), 256);
    const size_t o_g = off; off = align_up(off + n * d * sizeof(double), 256);
    const size_t o_t = off; off = align_up(off + (trace ? trace_count : 0) * sizeof(double), 256);
    if ((st = ensure_scratch(g, off)) != WOI_OK) return st;
    char *base = (char *)g->d_scratch;
    WOI_CUDA(cudaMemcpyAsync(base + o_x, x, d * sizeof(double), cudaMemcpyHostToDevice, s));
    WOI_CUDA(cudaMemcpyAsync(base + o_w, walk_ids, n * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
    WalkValuesParams p{};
    p.geom = g->d_blob;
    p.x = (const double *)(base + o_x);
    p.point_id = point_id;
    p.instance_id = instance_id;
    p.walks = (const uint64_t *)(base + o_w);
    p.n = n;
    p.sched_group = o->sched_group;
    p.seed = seed;
    p.f_u = (double *)(base + o_u);
    p.f_grad = (double *)(base + o_g);
    p.trace = trace ? (double *)(base + o_t) : nullptr;
    if (trace) WOI_CUDA(cudaMemsetAsync(p.trace, 0, trace_count * sizeof(double), s));
    if (g->d_mesh_overflow) WOI_CUDA(cudaMemsetAsync(g->d_mesh_overflow, 0, sizeof(unsigned int), s));
    WOI_CUDA(launch_walk_values(d, o->variant == WOI_VR, g->general(), o->precision == WOI_FP64_PLAIN, p, s));
    WOI_CUDA(cudaMemcpyAsync(f_u, p.f_u, n * sizeof(double), cudaMemcpyDeviceToHost, s));
    WOI_CUDA(cudaMemcpyAsync(f_grad, p.f_grad, n * d * sizeof(double), cudaMemcpyDeviceToHost, s));
    if (trace) WOI_CUDA(cudaMemcpyAsync(trace, p.trace, trace_count * sizeof(double), cudaMemcpyDeviceToHost, s));
    WOI_CUDA(cudaStreamSynchronize(s));
    return take_mesh_overflow(g);
}

woi_status woi_walk_values(woi_geometry *g, const woi_opts *o, const double *x, uint32_t point_id,
                           uint32_t instance_id, const uint64_t *walk_ids, int64_t n, uint64_t seed, double *f_u,
                           double *f_grad)
{
    return walk_values_impl(g, o, x, point_id, instance_id, walk_ids, n, seed, f_u, f_grad, nullptr);
}

woi_status woi_walk_trace(woi_geometry *g, const woi_opts *o, const double *x, uint32_t point_id,
                          uint32_t instance_id, const uint64_t *walk_ids, int64_t n, uint64_t seed, double *f_u,
                          double *f_grad, double *trace)
{
    if (!trace) {
        g_last_error = "null trace";
        return WOI_E_INVALID_ARG;
    }
    return walk_values_impl(g, o, x, point_id, instance_id, walk_ids, n, seed, f_u, f_grad, trace);
}

woi_status woi_autotune(woi_geometry *g, const woi_opts *o, const double *points, int64_t n_pts, int64_t n_walks,
                        uint64_t seed, int *block_out, int *lpl_out)
{
    g_last_error.clear();
    if (!g) return fail(WOI_E_INVALID_ARG, "null geometry");
    woi_status st;
    if ((st = check_opts(g, o, n_pts, 0, n_walks)) != WOI_OK) return st;
    if (o->precision != WOI_MIXED) return fail(WOI_E_UNSUPPORTED, "the autotuner tunes the FP32 walk kernel");
    if (n_pts < 1) return fail(WOI_E_INVALID_ARG, "need at least one point");
    if ((st = ensure_device(g)) != WOI_OK) return st;
    tune_load();
    const int d = g->dim;
    const bool vr = o->variant == WOI_VR, star = g->general();
    const int blocks[2] = {128, 256}, lanes[4] = {8, 16, 32, 64};
    float best = 1e30f;
    int bb = 256, bl = 8;
    woi_opts t = *o;
    t.timing = 1;
    t.tile_points = 0;                 // the table holds shapes of the per-point kernel
    for (int bi = 0; bi < 2; ++bi)
        for (int li = 0; li < 4; ++li) {
            t.block_size = blocks[bi];
            t.walks_per_lane = lanes[li];
            // probe: enough points for about four waves of units of this shape
            int per_sm = 1;
            const size_t smem = (size_t)(blocks[bi] / 32) * g->n * kMaxDim * sizeof(float);
            if (mixed_warp_occupancy(d, vr, star, blocks[bi], smem, &per_sm) != cudaSuccess) {
                cudaGetLastError();
                continue;
            }
            const int64_t unit_walks = 32LL * lanes[li];
            const int64_t chunks = (n_walks + unit_walks - 1) / unit_walks;
            const int64_t want_units = 4LL * g->num_sms * std::max(per_sm, 1) * (blocks[bi] / 32);
            const int64_t probe_pts = std::max<int64_t>(1, std::min<int64_t>(n_pts, (want_units + chunks - 1) / chunks));
            // one untimed run (caches the geometry and scratch), one timed run
            if ((st = run_estimate(g, &t, points, probe_pts, 0, n_walks, seed, nullptr, nullptr, nullptr, nullptr,
                                   nullptr)) != WOI_OK)
                return st;
            if ((st = run_estimate(g, &t, points, probe_pts, 0, n_walks, seed, nullptr, nullptr, nullptr, nullptr,
                                   nullptr)) != WOI_OK)
                return st;
            float ms = 0.f;
            if ((st = woi_last_kernel_ms(g, &ms)) != WOI_OK) return st;
            const float per_walk = ms / (float)(probe_pts * n_walks);
            if (per_walk < best) {
                best = per_walk;
                bb = blocks[bi];
                bl = lanes[li];
            }
        }
    g_tune[tune_key(d, star, o->variant, o->sched_group, o->M)] = {bb, bl};
    tune_save();
    if (block_out) *block_out = bb;
    if (lpl_out) *lpl_out = bl;
    return WOI_OK;
}

woi_status woi_check_status(woi_geometry *g)
{
    g_last_error.clear();
    if (!g) return fail(WOI_E_INVALID_ARG, "null geometry");
    if (!g->check_pending) return WOI_OK;
    WOI_CUDA(cudaEventSynchronize(g->ev_done));
    return take_mesh_overflow(g);
}

woi_status woi_last_kernel_ms(woi_geometry *g, float *ms)
{
    g_last_error.clear();
    if (!g || !ms) return fail(WOI_E_INVALID_ARG, "null argument");
    if (!g->timed || !g->ev_stop) return fail(WOI_E_STATE, "no timed estimate on this handle");
    WOI_CUDA(cudaEventSynchronize(g->ev_stop));
    WOI_CUDA(cudaEventElapsedTime(ms, g->ev_start, g->ev_stop));
    return WOI_OK;
}

woi_status woi_finalize_moments(int dim, int64_t n_pts, int64_t n_walks, int sched_group, const double *moments,
                                void *cuda_stream, double *u, double *grad, double *se_u, double *se_grad)
{
    g_last_error.clear();
    if (dim < 2 || dim > WOI_MAX_DIM) return fail(WOI_E_INVALID_ARG, "dim = %d outside [2, %d]", dim, WOI_MAX_DIM);
    if (n_pts < 0 || n_walks < 1) return fail(WOI_E_INVALID_ARG, "need n_pts >= 0, n_walks >= 1");
    if (sched_group != 1 && sched_group != 32) return fail(WOI_E_INVALID_ARG, "sched_group must be 1 or 32");
    if (n_walks % sched_group) return fail(WOI_E_INVALID_ARG, "n_walks must be a multiple of sched_group");
    if (n_pts > 0 && !moments) return fail(WOI_E_INVALID_ARG, "null moments");
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return fail(WOI_E_NO_DEVICE, "no CUDA device");
    }
    if (n_pts == 0) return WOI_OK;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int C = dim + 1;
    // host arrays go through one temporary device buffer: [moments][u][grad][se_u][se_grad]
    double *user[5] = {const_cast<double *>(moments), u, grad, se_u, se_grad};
    const size_t count_of[5] = {(size_t)n_pts * 2 * C, (size_t)n_pts, (size_t)n_pts * dim, (size_t)n_pts,
                                (size_t)n_pts * dim};
    bool host[5];
    size_t off[5], bytes = 0;
    for (int k = 0; k < 5; ++k) {
        host[k] = user[k] && !pointer_on_device(user[k]);
        off[k] = bytes;
        if (host[k]) bytes = align_up(bytes + count_of[k] * sizeof(double), 256);
    }
    char *tmp = nullptr;
    if (bytes && cudaMalloc((void **)&tmp, bytes) != cudaSuccess) {
        cudaGetLastError();
        return fail(WOI_E_OOM, "device staging allocation of %zu bytes failed", bytes);
    }
    double *dev[5];
    for (int k = 0; k < 5; ++k) dev[k] = !user[k] ? nullptr : (host[k] ? (double *)(tmp + off[k]) : user[k]);
    woi_status st = WOI_OK;
    cudaError_t e = cudaSuccess;
    if (host[0]) e = cudaMemcpyAsync(dev[0], moments, count_of[0] * sizeof(double), cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) {
        FinalizeParams fp{};
        fp.dim = dim;
        fp.n_pts = n_pts;
        fp.n_walks = n_walks;
        fp.sched_group = sched_group;
        fp.partials = dev[0];
        fp.u = dev[1];
        fp.grad = dev[2];
        fp.se_u = dev[3];
        fp.se_grad = dev[4];
        fp.moments = nullptr;
        e = launch_finalize(fp, true, s);    // one row of accumulated moments per point
    }
    for (int k = 1; k < 5 && e == cudaSuccess; ++k)
        if (host[k]) e = cudaMemcpyAsync(user[k], dev[k], count_of[k] * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess && tmp) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) st = fail(WOI_E_CUDA, "woi_finalize_moments: %s", cudaGetErrorString(e));
    if (tmp) cudaFree(tmp);
    return st;
}

woi_status woi_estimate_batch(int n_inst, woi_geometry *const *geoms, const woi_opts *o, const int *m_per_inst,
                              const double *const *points, const int64_t *n_pts, const int64_t *n_walks, uint64_t seed,
                              double *const *u, double *const *grad, double *const *se_u, double *const *se_grad)
{
    g_last_error.clear();
    if (o && o->tile_points) return fail(WOI_E_UNSUPPORTED, "shared trajectories are not supported in a batch");
    return run_batch(n_inst, geoms, o, m_per_inst, points, n_pts, n_walks, seed, u, grad, se_u, se_grad);
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free estimate (no counterpart in the paper).
//
// For callers that may not allocate device memory while they run.  All scratch
// -- the geometry blob, flux and arc tables, the instance descriptor, the work
// queue head and the per-unit partials -- is carved out of one file-scope
// device array.  In host code the array's name is only a host-side stand-in,
// so its device address is looked up once per device with
// cudaGetSymbolAddress (that device current) and passed to the kernels.
// ---------------------------------------------------------------------------
static __device__ __align__(256) unsigned char g_noalloc_scratch[WOI_NOALLOC_SCRATCH_BYTES];

namespace {

constexpr int kNoallocMaxDevices = 64;
std::atomic<void *> g_noalloc_addr[kNoallocMaxDevices];   // zero-initialised (static storage)
thread_local DevGeom g_noalloc_blob;   // host image of the blob (no heap allocation)

// device address of the scratch array on device `dev` (current); looked up once per device.
// Two threads may look it up at the same time: both get the same address and store it.
woi_status noalloc_scratch_address(int dev, char **out)
{
    if (dev < 0 || dev >= kNoallocMaxDevices) return fail(WOI_E_UNSUPPORTED, "device ordinal %d too large", dev);
    void *p = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!p) {
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || !p)
            return fail(WOI_E_CUDA, "cudaGetSymbolAddress of the scratch array failed: %s", cudaGetErrorString(e));
        g_noalloc_addr[dev].store(p, std::memory_order_release);
    }
    *out = (char *)p;
    return WOI_OK;
}

}  // namespace

extern "C" woi_status woi_estimate_noalloc(woi_geometry *g, const woi_opts *o, const double *points, int64_t n_pts,
                                           int64_t n_walks, uint64_t seed, double *u, double *grad, double *se_u,
                                           double *se_grad)
{
    g_last_error.clear();
    if (!g) return fail(WOI_E_INVALID_ARG, "null geometry");
    woi_status st;
    if ((st = check_opts(g, o, n_pts, 0, n_walks)) != WOI_OK) return st;
    if (o->precision != WOI_MIXED) return fail(WOI_E_UNSUPPORTED, "the allocation-free estimate runs the mixed path only");
    if (o->tile_points) return fail(WOI_E_UNSUPPORTED, "the allocation-free estimate has no shared-trajectory mode");
    if (!g->mesh.empty()) return fail(WOI_E_UNSUPPORTED, "the allocation-free estimate does not take meshes");
    if (n_pts > 0 && !pointer_on_device(points)) return fail(WOI_E_INVALID_ARG, "points must be device memory");
    double *outs[4] = {u, grad, se_u, se_grad};
    for (double *p : outs)
        if (p && !pointer_on_device(p)) return fail(WOI_E_INVALID_ARG, "outputs must be device memory");
    int count = 0;
    if (cudaGetDeviceCount(&count) != cudaSuccess || count == 0) {
        cudaGetLastError();
        return fail(WOI_E_NO_DEVICE, "no CUDA device");
    }
    if (n_pts == 0) return WOI_OK;
    int dev = 0, num_sms = 0;
    WOI_CUDA(cudaGetDevice(&dev));
    WOI_CUDA(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    char *base = nullptr;
    if ((st = noalloc_scratch_address(dev, &base)) != WOI_OK) return st;

    cudaStream_t s = (cudaStream_t)o->cuda_stream;
    const int d = g->dim, C = d + 1, M = o->M;
    const bool vr = o->variant == WOI_VR, star = g->general();
    int block, L;
    launch_shape(o, d, star, &block, &L, 64);  // explicit options, else the tuned table, else 256 x 64
    const int64_t unit_walks = 32LL * L;       // warp-level work units
    const int64_t chunks = (n_walks + unit_walks - 1) / unit_walks;
    const int64_t units = n_pts * chunks;

    // layout inside the fixed array; reject what does not fit
    size_t off = 0;
    const size_t o_blob = off; off = align_up(off + sizeof(DevGeom), 256);
    const size_t o_flux = off; off = align_up(off + g->flux_dev.size() * sizeof(double), 256);
    const size_t o_flux_f = off; off = align_up(off + g->flux_dev_f.size() * sizeof(float), 256);
    const size_t o_t0 = off; off = align_up(off + g->arc_t0.size() * sizeof(double), 256);
    const size_t o_t1 = off; off = align_up(off + g->arc_t1.size() * sizeof(double), 256);
    const size_t o_len = off; off = align_up(off + g->arc_len.size() * sizeof(double), 256);
    const size_t o_s0 = off; off = align_up(off + g->arc_s0.size() * sizeof(double), 256);
    const size_t o_sign = off; off = align_up(off + g->arc_sign.size() * sizeof(int), 256);
    const size_t o_desc = off; off = align_up(off + sizeof(InstDesc), 256);
    const size_t o_queue = off; off = align_up(off + sizeof(unsigned long long), 256);
    const size_t o_part = off; off = align_up(off + (size_t)units * 2 * C * sizeof(double), 256);
    if (off > (size_t)WOI_NOALLOC_SCRATCH_BYTES)
        return fail(WOI_E_INVALID_ARG,
                    "%lld points x %lld walks need %zu bytes of scratch; the allocation-free estimate has %u",
                    (long long)n_pts, (long long)n_walks, off, (unsigned)WOI_NOALLOC_SCRATCH_BYTES);

    // tables of this geometry (pageable sources: staged before cudaMemcpyAsync returns)
    auto put = [&](size_t at, const void *src, size_t bytes) -> cudaError_t {
        return bytes ? cudaMemcpyAsync(base + at, src, bytes, cudaMemcpyHostToDevice, s) : cudaSuccess;
    };
    WOI_CUDA(put(o_flux, g->flux_dev.data(), g->flux_dev.size() * sizeof(double)));
    WOI_CUDA(put(o_flux_f, g->flux_dev_f.data(), g->flux_dev_f.size() * sizeof(float)));
    WOI_CUDA(put(o_t0, g->arc_t0.data(), g->arc_t0.size() * sizeof(double)));
    WOI_CUDA(put(o_t1, g->arc_t1.data(), g->arc_t1.size() * sizeof(double)));
    WOI_CUDA(put(o_len, g->arc_len.data(), g->arc_len.size() * sizeof(double)));
    WOI_CUDA(put(o_s0, g->arc_s0.data(), g->arc_s0.size() * sizeof(double)));
    WOI_CUDA(put(o_sign, g->arc_sign.data(), g->arc_sign.size() * sizeof(int)));

    DevGeom &b = g_noalloc_blob;
    fill_blob(*g, M, b);
    b.flux_coef = (const double *)(base + o_flux);
    b.flux_coef_f = (const float *)(base + o_flux_f);
    b.arc_t0 = (const double *)(base + o_t0);
    b.arc_t1 = (const double *)(base + o_t1);
    b.arc_len = (const double *)(base + o_len);
    b.arc_s0 = (const double *)(base + o_s0);
    b.arc_sign = (const int *)(base + o_sign);
    WOI_CUDA(put(o_blob, &b, sizeof(DevGeom)));

    InstDesc desc{};
    desc.geom = (const DevGeom *)(base + o_blob);
    desc.points = points;
    desc.n_pts = n_pts;
    desc.n_walks = n_walks;
    desc.walk_begin = 0;
    desc.unit_begin = 0;
    desc.chunks_per_point = chunks;
    desc.instance_id = 0;
    desc.sched_group = o->sched_group;
    WOI_CUDA(put(o_desc, &desc, sizeof(desc)));
    // the previous call's queue head is still in the array: restart it at zero
    WOI_CUDA(cudaMemsetAsync(base + o_queue, 0, sizeof(unsigned long long), s));

    int per_sm = 0;
    const size_t smem = (size_t)(block / 32) * g->n * kMaxDim * sizeof(float);
    WOI_CUDA(mixed_warp_occupancy(d, vr, star, block, smem, &per_sm));
    if (per_sm < 1) return fail(WOI_E_UNSUPPORTED, "walk kernel does not fit on an SM (M = %d)", M);
    const int64_t grid = std::min<int64_t>((int64_t)num_sms * per_sm, (units + block / 32 - 1) / (block / 32));
    MixedParams mp{};
    mp.inst = (const InstDesc *)(base + o_desc);
    mp.n_inst = 1;
    mp.total_units = units;
    mp.queue = (unsigned long long *)(base + o_queue);
    mp.partials = (double *)(base + o_part);   // every unit's row is written before it is read
    mp.walks_per_lane = L;
    mp.seed = seed;
    WOI_CUDA(launch_mixed_warp(d, vr, star, mp, (int)grid, block, smem, s));
    FinalizeParams fp{};
    fp.dim = d;
    fp.n_pts = n_pts;
    fp.n_walks = n_walks;
    fp.sched_group = o->sched_group;
    fp.unit_begin = 0;
    fp.chunks_per_point = chunks;
    fp.partials = (const double *)(base + o_part);
    fp.u = u;
    fp.grad = grad;
    fp.se_u = se_u;
    fp.se_grad = se_grad;
    fp.moments = nullptr;
    WOI_CUDA(launch_finalize(fp, false, s));
    return WOI_OK;
}
