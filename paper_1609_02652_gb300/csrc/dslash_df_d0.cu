// Stencil instantiations for one (precision, adjoint) pair; see dslash_kernels.cuh.
#include "dslash_kernels.cuh"

namespace pfmp {
PFMP_DSLASH_INSTANTIATE(PREC_DF, false)
}  // namespace pfmp
