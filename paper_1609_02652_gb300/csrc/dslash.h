// Stencil entry points exported by the dslash_<prec>_<dag>.cu translation units (one
// (precision, adjoint) pair each; definitions in dslash_kernels.cuh).  PREC is PFMP_F64,
// PFMP_F32, PFMP_H16 or PREC_DF (double-float); DAG selects the adjoint hop.
#pragma once
#include "context.h"
#include "dfloat.cuh"

namespace pfmp {

// out (parity p) = H in (the plain hop, restricted to one parity)
template <int PREC, bool DAG>
void hop_plain_t(pfmp_op* op, void* out, const void* in, int p);
// out (odd) = A_oo^{-1} H_oe in; every launch returns at once when scal->done is set
template <int PREC, bool DAG>
void hop_clov_odd_t(pfmp_op* op, void* out, const void* in, CGScalars* scal);
// out = M-hat in (DAG: M-hat^dag in) through the odd temporary t (caller-chosen buffer of
// one odd spinor field of this precision); ||out||^2 -> *norm_out (device) when not null,
// and with scal the CG step alpha = rr / ||out||^2
template <int PREC, bool DAG>
void mhat_t(pfmp_op* op, void* out, const void* in, double* norm_out, CGScalars* scal, void* t);

#define PFMP_DSLASH_DECLARE(PREC, DAG)                                                                  \
  extern template void hop_plain_t<PREC, DAG>(pfmp_op*, void*, const void*, int);                       \
  extern template void hop_clov_odd_t<PREC, DAG>(pfmp_op*, void*, const void*, CGScalars*);             \
  extern template void mhat_t<PREC, DAG>(pfmp_op*, void*, const void*, double*, CGScalars*, void*);

}  // namespace pfmp
