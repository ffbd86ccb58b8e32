// woi_layout.h -- the device blob of one geometry instance, written by the
// host side of libwoi and read (then staged to shared memory) by its kernels.
#pragma once

#include <cstdint>

namespace woi {

constexpr int kMaxDim = 6;
constexpr int kMaxSurf = 128;          // surfaces per instance (WOI_MAX_SURF)
constexpr int kMaxSurfPad = 128;       // schedule thresholds padded to a power of two
constexpr int kSchedBuckets = 256;     // index of the schedule thresholds by the top 8 bits of the word
constexpr int kMaxM = 32;              // truncation (WOI_MAX_M)
constexpr int kMaxStar = 16;           // star Fourier degree (WOI_MAX_STAR_DEGREE)
constexpr int kNodes = 256;            // angle nodes t_j = 2 pi j / kNodes: star scan samples,
                                       // arc-length panels and the angle-addition table
constexpr int kMaxRoots = 2 * (kMaxStar + 1) + 2;
static_assert((kNodes & (kNodes - 1)) == 0, "node indices wrap with a mask");
constexpr int kMaxEll = 8;             // ellipsoids per instance (WOI_MAX_ELLIPSOIDS)
constexpr int kMaxMesh = 16;           // meshes per instance (WOI_MAX_MESHES)
constexpr int kMeshStack = 64;         // BVH traversal stack (the host caps the tree depth below it)
constexpr int kMaxHits = 32;           // intersections of one line with one mesh
constexpr int kTriBuckets = 1024;      // per mesh: the triangle range of each top-10-bit word bucket
constexpr int kEllAttempts = 64;       // rejection attempts for a uniform point on an ellipsoid
constexpr int kVrTrials = 16;          // uniform trials of the VR start where |dOmega^+/-| has no closed form

enum { kSphere = 0, kStar = 1, kEllipsoid = 2, kMesh = 3 };

// a node of a mesh's bounding-volume hierarchy as the host builds it (local coordinates of
// the surface, FP32 bounds rounded outward and padded): internal node a, b = children; leaf
// a = first entry of the leaf-triangle list, b = -(number of triangles)
struct BvhNode {
    float lo[3], hi[3];
    int a, b;
};
// the device form of the hierarchy: one entry per internal node, holding the boxes of both
// children (lo, hi of child 0, then of child 1) and their references: the entry index of an
// internal child, or -(triangle + 1) for a leaf (every leaf holds one triangle)
struct BvhWide {
    float box[2][6];
    int child[2];
    int pad[2];
};
static_assert(sizeof(BvhWide) == 64, "entries are read as four float4");
enum { kFluxZero = 0, kFluxFourier = 1, kFluxRealSH = 2, kFluxHarmonicPoly = 3, kFluxPointCharge = 4,
       kFluxHarmonicQuad = 16,     // device only: [s, (a_k, b_k[d], c_k[d(d+1)/2]) x d], grad P quadratic
       kFluxSphQuad = 17 };        // device only, 3D spheres: real harmonics of degree <= 2 as
                                   // [1, x, y, z, xx, xy, xz, yy, yz, zz] coefficients of the unit vector

struct DevGeom {
    int dim, n, npad, M;
    int star_idx, star_K;              // star_idx = -1: no star in this instance
    double star_lmax;                  // bound on |gamma'| of the star
    double star_kpp;                   // bound on |gamma''| of the star
    double star_k3;                    // bound on |gamma'''| of the star
    // gamma(t) - centre = sum_{m=0}^{K+1} (X_m cos mt + Y_m sin mt, U_m cos mt + V_m sin mt):
    // star_harm[m] = (X_m, Y_m, U_m, V_m)
    double star_harm[kMaxStar + 2][4];
    double star_rmin, star_rmax;       // bounds on r(t): every point of the star lies in this annulus
    uint32_t sched_tm1[kMaxSurfPad];   // T_n - 1, padded with 0xFFFFFFFF
    int sched_bucket[kSchedBuckets + 1]; // first n with T_n - 1 >= b 2^24 (N - 1 if none)
    double center[kMaxSurf][kMaxDim];
    double radius[kMaxSurf];
    double area[kMaxSurf];
    double alpha_sign[kMaxSurf];       // sign(alpha_n) in {-1, 0, 1}
    double beta_scale[kMaxSurf];       // beta_n / b_n (Sec. 3)
    int tin[kMaxSurf], tout[kMaxSurf]; // Euler-tour interval of each region in the tree
    int type[kMaxSurf];
    double coef[kMaxM + 1];            // N w_i ||alpha||_1^i for the current M
    double star_a[kMaxStar + 1], star_b[kMaxStar + 1];
    double node_cs[kNodes][2];         // cos t_j, sin t_j
    double star_scan[kNodes][2];       // gamma(t_j) - centre
    double star_scan_d[kNodes][2];     // gamma'(t_j)
    double star_panel_s[kNodes + 1];   // arc length at t_j
    int flux_basis[kMaxSurf], flux_off[kMaxSurf], flux_n[kMaxSurf];
    const double *flux_coef;           // device array, device format (real-SH entries carry their
                                       // normalisation); FP32 copy in flux_coef_f
    const float *flux_coef_f;
    double part_len[kMaxSurf][2];      // |dOmega^+|, |dOmega^-| (variance reduction); -1: by trials
    double vr_tol[kMaxSurf];           // d >= 3 VR: |beta| below which its sign is taken in FP64
    int arc_off[kMaxSurf], arc_n[kMaxSurf];
    const double *arc_t0;              // device arrays of the beta-sign arcs
    const double *arc_t1;
    const double *arc_len;
    const double *arc_s0;              // star: arc length at the arc's start angle
    const int *arc_sign;
    // ellipsoids (d >= 3): (y - c)^T A (y - c) = 1; map = A^{-1/2} (symmetric square root) takes
    // the unit sphere onto the surface with area ratio sqrt(u^T A u); jmax = sqrt(max eigenvalue)
    int n_ell;
    int ell_slot[kMaxSurf];            // slot of surface i, -1 if it is not an ellipsoid
    double ell_A[kMaxEll][kMaxDim][kMaxDim];
    double ell_map[kMaxEll][kMaxDim][kMaxDim];
    double ell_jmax[kMaxEll];
    // triangle meshes (d = 3), all meshes of the instance concatenated; triangle rows are
    // (v0, e1 = v1 - v0, e2 = v2 - v0, unit normal of e1 x e2) in the surface's local coordinates
    int n_mesh;
    int mesh_slot[kMaxSurf];           // slot of surface i, -1 if it is not a mesh
    int mesh_tri_off[kMaxMesh], mesh_ntri[kMaxMesh], mesh_node_off[kMaxMesh];
    double mesh_scale[kMaxMesh];       // largest |vertex - centre|
    const float *tri_f;                // [n_tri][12]
    const double *tri_d;               // [n_tri][12]
    const uint32_t *tri_tm1;           // [n_tri] T_j - 1 of the area-proportional triangle choice
    const int *tri_bucket;             // [n_mesh][kTriBuckets + 1]: first j with T_j - 1 >= b 2^22 (global j)
    const BvhWide *bvh;                // all meshes' hierarchies (mesh m's root at mesh_node_off[m])
    unsigned int *mesh_overflow;       // device counter of lines with more than kMaxHits crossings
};

// one instance of a (possibly batched) estimate
struct InstDesc {
    const DevGeom *geom;
    const double *points;              // device [n_pts][dim] FP64
    int64_t n_pts;
    int64_t n_walks;
    int64_t walk_begin;
    int64_t unit_begin;                // first work unit of this instance
    int64_t chunks_per_point;
    uint32_t instance_id;              // random-stream instance id
    int sched_group;
    int64_t point_begin;               // first point of this instance in a batch
    double *u, *grad, *se_u, *se_grad; // device outputs of a batch (each may be null)
};

}  // namespace woi
