// woi_k6.cu -- walk kernels of dimension 6 (instantiation unit).
#include "woi_kernels_impl.cuh"

namespace woi {
template struct DimLaunchers<6, false>;
}  // namespace woi
