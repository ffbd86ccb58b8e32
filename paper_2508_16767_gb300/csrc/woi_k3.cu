// woi_k3.cu -- walk kernels of dimension 3 (instantiation unit).
#include "woi_kernels_impl.cuh"

namespace woi {
template struct DimLaunchers<3, false>;
}  // namespace woi
