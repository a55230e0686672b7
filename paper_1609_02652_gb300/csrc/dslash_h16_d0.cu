// Stencil instantiations for one (precision, adjoint) pair; see dslash_kernels.cuh.
#include "dslash_kernels.cuh"

namespace pfmp {
PFMP_DSLASH_INSTANTIATE(PFMP_H16, false)
}  // namespace pfmp
