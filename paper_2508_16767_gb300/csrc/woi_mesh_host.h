// woi_mesh_host.h -- host-side preparation of closed triangle meshes (d = 3):
// validation, triangle rows in local coordinates, the area-proportional
// triangle thresholds, a bounding-volume hierarchy, and an inside test.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "woi_layout.h"

namespace woi {

struct MeshHost {
    double center[3] = {0, 0, 0};
    int ntri = 0;
    std::vector<double> tri;        // [ntri][12]: v0 - center, e1, e2, unit normal (local coordinates)
    std::vector<double> tri_area;   // [ntri]
    double area = 0.0;              // sum of the triangle areas, in input order
    double scale = 0.0;             // largest |vertex - center|
    std::vector<uint32_t> tm1;      // [ntri] floor(2^32 C_j / A) - 1, the last 2^32 - 1
    std::vector<BvhNode> nodes;     // root first
    std::vector<int> leaf_tri;      // triangle indices (0..ntri-1) in leaf order
    std::vector<BvhWide> wide;      // the same hierarchy as the device reads it, root first
    int depth = 0;
};

// Checks that (V, T) is a closed, consistently oriented triangle mesh with positive
// enclosed volume and non-degenerate triangles, and builds everything above.  Returns
// an empty string on success, else the reason.
std::string mesh_prepare(const double *V, int nv, const int *T, int nt, const double *center, MeshHost &out);

// Is the global point x strictly inside the mesh?  Parity of the crossings of a ray
// in a fixed irrational direction (through the hierarchy).
bool mesh_inside(const MeshHost &m, const double *x);

}  // namespace woi
