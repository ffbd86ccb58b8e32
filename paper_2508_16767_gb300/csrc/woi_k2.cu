// woi_k2.cu -- walk kernels of dimension 2 (instantiation unit).
#include "woi_kernels_impl.cuh"

namespace woi {
template struct DimLaunchers<2, false>;
}  // namespace woi
