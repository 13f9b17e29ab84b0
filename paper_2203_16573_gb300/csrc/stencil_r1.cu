// stencil_r1.cu -- step and persistent-sweep kernels of spatial order 2
// for every tile configuration (see stencil_impl.cuh).
#include "stencil_impl.cuh"

namespace ssx {
#define SSX_R 1
SSX_DEFINE_DISPATCH(1)
#undef SSX_R
}  // namespace ssx
