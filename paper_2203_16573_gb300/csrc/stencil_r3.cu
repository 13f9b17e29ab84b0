// stencil_r3.cu -- step and persistent-sweep kernels of spatial order 6
// for every tile configuration (see stencil_impl.cuh).
#include "stencil_impl.cuh"

namespace ssx {
#define SSX_R 3
SSX_DEFINE_DISPATCH(3)
#undef SSX_R
}  // namespace ssx
