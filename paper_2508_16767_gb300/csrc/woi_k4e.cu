// woi_k4e.cu -- walk kernels of dimension 4 with ellipsoid surfaces (instantiation unit).
#include "woi_kernels_impl.cuh"

namespace woi {
template struct DimLaunchers<4, true>;
}  // namespace woi
