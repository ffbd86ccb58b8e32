// woi_k5e.cu -- walk kernels of dimension 5 with ellipsoid surfaces (instantiation unit).
#include "woi_kernels_impl.cuh"

namespace woi {
template struct DimLaunchers<5, true>;
}  // namespace woi
