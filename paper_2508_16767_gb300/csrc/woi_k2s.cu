// woi_k2s.cu -- walk kernels of dimension 2 with a star surface (instantiation unit).
#include "woi_kernels_impl.cuh"

namespace woi {
template struct DimLaunchers<2, true>;
}  // namespace woi
