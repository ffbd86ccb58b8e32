// woi_k4.cu -- walk kernels of dimension 4 (instantiation unit).
#include "woi_kernels_impl.cuh"

namespace woi {
template struct DimLaunchers<4, false>;
}  // namespace woi
