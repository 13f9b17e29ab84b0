// stencil_r4.cu -- step and persistent-sweep kernels of spatial order 8
// for every tile configuration (see stencil_impl.cuh).
#include "stencil_impl.cuh"

namespace ssx {
#define SSX_R 4
SSX_DEFINE_DISPATCH(4)
#undef SSX_R
}  // namespace ssx
