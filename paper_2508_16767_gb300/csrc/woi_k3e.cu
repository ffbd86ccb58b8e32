// woi_k3e.cu -- walk kernels of dimension 3 with ellipsoid surfaces (instantiation unit).
#include "woi_kernels_impl.cuh"

namespace woi {
template struct DimLaunchers<3, true>;
}  // namespace woi
