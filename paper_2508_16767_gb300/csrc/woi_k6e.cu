// woi_k6e.cu -- walk kernels of dimension 6 with ellipsoid surfaces (instantiation unit).
#include "woi_kernels_impl.cuh"

namespace woi {
template struct DimLaunchers<6, true>;
}  // namespace woi
