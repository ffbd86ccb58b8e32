// woi_k5.cu -- walk kernels of dimension 5 (instantiation unit).
#include "woi_kernels_impl.cuh"

namespace woi {
template struct DimLaunchers<5, false>;
}  // namespace woi
