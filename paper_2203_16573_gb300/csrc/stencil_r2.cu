// stencil_r2.cu -- step and persistent-sweep kernels of spatial order 4
// for every tile configuration (see stencil_impl.cuh).
#include "stencil_impl.cuh"

namespace ssx {
#define SSX_R 2
SSX_DEFINE_DISPATCH(2)
#undef SSX_R
}  // namespace ssx
