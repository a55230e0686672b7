// Host-side definitions of the library's opaque handles and of the internal entry
// points the C-ABI wrappers (capi.cu) call.
#pragma once
#include <cuda_runtime.h>

#include <complex>
#include <vector>

#include "pfmp_internal.cuh"
#include "reduce.cuh"

namespace pfmp {

// device scalars of one solver instance (written by reduction finishers)
struct CGScalars {
  double rr;        // current |r|^2
  double rr_new;
  double pAp;
  double alpha;
  double beta;
  double stop_rr;   // stop the device loop once rr < stop_rr
  int done;        // every CG kernel returns at once when set
  int done_next;   // raised by the x/r update, copied to done after the p update
  int iter;
};

}  // namespace pfmp

namespace pfmp {
struct MSWork;
// CUDA-event timing of the stencil kernels (off unless pfmp_profile_begin was called)
struct KernelProfile {
  bool on = false;
  std::vector<cudaEvent_t> pool;   // reusable events
  size_t used = 0;
  struct Rec {
    int cls;
    double bytes;
    cudaEvent_t a, b;
  };
  std::vector<Rec> recs;
};
}  // namespace pfmp

struct pfmp_ctx {
  pfmp::Geom g;
  pfmp::KernelProfile prof;
  cudaStream_t stream = nullptr;
  int device = 0;
  double2* U64 = nullptr;    // master [2][4][9][Vh]
  float4* U32 = nullptr;     // compressed [2][4][3][Vh]
  float4* Udf = nullptr;     // double-float full links [2][4][9][Vh] (complex as hi/lo pairs)
  uint4* U16 = nullptr;      // FP16 compressed, 24 bytes per link (planes: see link_plane)
  pfmp::ReduceBuf rb{};
  double* d_sums = nullptr;  // [64] results of generic reductions
  double* h_sums = nullptr;  // pinned mirror [64]
  double* canon = nullptr;   // canonical full-lattice scratch (V*24 doubles)
  long gauge_version = 0;
  double* fmunu = nullptr;   // clover field strength F_{mu nu}, [2][6][9][Vh] (built on demand)
  long fmunu_version = -1;   // gauge_version it was computed for
  int fmunu_prec = PFMP_F64; // arithmetic it was computed in
  float* hc32 = nullptr;     // FP32 copy of a clover insertion for the FP32 clover force (on demand)
};

struct pfmp_op {
  pfmp_ctx* ctx = nullptr;
  double kappa = 0, csw = 0;
  double2* clov64[2] = {nullptr, nullptr};  // [0]: A on even sites, [1]: A^{-1} on odd sites
  float4* clov32[2] = {nullptr, nullptr};
  float4* clovdf[2] = {nullptr, nullptr};   // double-float copy of clov64
  float4* tdf = nullptr;                    // odd / even double-float temporaries
  float4* edf = nullptr;
  float4* xdf = nullptr;
  float4* kdf = nullptr;
  double logdet_oo = 0;
  long built_version = -1;
  int built_prec = PFMP_F64;  // arithmetic of the field strength the clover blocks came from
  // workspace (odd temporaries and even scratch)
  double2* t64 = nullptr;
  float4* t32 = nullptr;
  double2* e64 = nullptr;
  float4* e32 = nullptr;
  uint4* clov16[2] = {nullptr, nullptr};    // FP16 copy of clov32: [9][Vh] per parity
  uint4* t16 = nullptr;                     // FP16 odd / even temporaries (with scales)
  uint4* e16 = nullptr;
  uint4* cg16[2] = {nullptr, nullptr};      // p and Ap of the FP16 CG
  double2* cg64[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // r p Ap | b x (host solve) | spare
  float4* cg32[4] = {nullptr, nullptr, nullptr, nullptr};
  pfmp::CGScalars* scal = nullptr;
  pfmp::CGScalars* h_scal = nullptr;
  // CUDA graph of one chunk of CG iterations per precision (captured on `cap`, replayed
  // on the context's stream); keyed by the buffers and the chunk length
  struct Graph {
    cudaGraphExec_t exec = nullptr;
    const void* key[4] = {nullptr, nullptr, nullptr, nullptr};
    int chunk = 0;
    long long kernels = 0;  // kernel nodes in the graph (for the launch counter)
  } graph[4];
  cudaStream_t cap = nullptr;
  pfmp::MSWork* ms = nullptr;  // multi-shift workspace (grown on demand)
  void* fgcr = nullptr;         // FGCR workspace (kept between solves), freed by fgcr_free
  void (*fgcr_free)(void*) = nullptr;
  long long kapply = 0;         // K applications done (CUDA-graph replays included)
  int nsplit[3] = {1, 1, 1};    // threads per site of the stencil kernels: FP64, FP32, double-float
  int hop_block = 128;          // threads per block of the stencil kernels (32..128)
};

namespace pfmp {

inline size_t spinor_bytes(const Geom& g, int prec) {
  if (prec == PFMP_H16) return (size_t)g.Vh * 52;  // 24 FP16 reals + one FP32 scale per site
  return (size_t)g.Vh * 24 * (prec == PFMP_F64 ? 8 : 4);
}
void* dev_alloc(size_t bytes);
void dev_free(void* p);

// core.cu
void gauge_refresh_compressed(pfmp_ctx* c);
void spinor_pack(pfmp_ctx* c, void* dst, int prec, const double* src_dev, int parity);
void spinor_unpack(pfmp_ctx* c, double* dst_dev, const void* src, int prec, int parity);

// clover.cu
// clover blocks from the field strength in FP64 (default) or FP32 arithmetic
void clover_build(pfmp_op* op, int fprec = PFMP_F64);
// the field strength F_{mu nu} of the current gauge field in c->fmunu (computed once per
// gauge-field version and precision, shared by every operator of the context)
void field_strength_update(pfmp_ctx* c, int prec = PFMP_F64);

// profiling (core.cu): bracket one launch with events when profiling is on
void prof_start(pfmp_ctx* c, cudaEvent_t* a);
void prof_stop(pfmp_ctx* c, int cls, double bytes, cudaEvent_t a);

// dslash.cu
void hop(pfmp_op* op, int prec, void* out, const void* in, int out_parity, bool dagger);
void clover_mul(pfmp_op* op, int prec, void* out, const void* in, int parity);
// out = M-hat in (or dagger); if pAp != nullptr the finisher of the second kernel
// stores ||out||^2 into *pAp (device scalar) and, when scal != nullptr, alpha = rr/pAp
void mhat(pfmp_op* op, int prec, void* out, const void* in, bool dagger, double* norm_out,
          CGScalars* scal);
void kop(pfmp_op* op, int prec, void* out, const void* in, double* pKp_dev, CGScalars* scal);

void hop_clov_odd(pfmp_op* op, int prec, void* out, const void* in, bool dagger);
void kop_df(pfmp_op* op, void* out, const void* in);
// r = b - K x with K applied in double-float; returns |r|^2 (synchronises)
double true_residual_df(pfmp_op* op, const void* x64, const void* b64, void* r64);
// the same with K in FP64 (x must not alias r)
double true_residual_f64(pfmp_op* op, const void* x64, const void* b64, void* r64);
// double-float, confirmed in FP64 once below target_rr; the FP64 value decides
double true_residual_mixed(pfmp_op* op, const void* x64, const void* b64, void* r64, double target_rr, long* kapply);

// cg_fused.cu: one FP32 CG iteration as four stencil kernels with the vector updates
// fused in (p = r + beta p formed by the next iteration; scalars in op->scal)
void cg_fused_iteration(pfmp_op* op, float4* x, float4* r, float4* p);

// force.cu
// One contraction Re a^dag dM-hat b: the even fields a and b, the odd fields
// y = A_oo^{-1} H_oe b and w = A_oo^{-1} H^dag_oe a (all of one precision), and the
// coefficients of its hop part (-kappa^2 coef), its clover part on the even sites
// (-kappa c_sw coef) and on the odd sites (kappa^2 kappa c_sw coef).
struct DerivSet {
  const void* a;
  const void* b;
  const void* y;
  const void* w;
  double c_hop, c_even, c_odd;
};
constexpr int kMaxDerivSets = 8;
struct DerivBatch {
  int n = 0;
  DerivSet s[kMaxDerivSets];
};
// F and Hc += every contraction of the batch, one launch per force kernel: the
// accumulators are read and written once per batch
void deriv_mhat_batch(pfmp_ctx* c, int prec, double* F, double* Hc, const DerivBatch& B);
void clover_insert_det(pfmp_op* op, double* Hc, double coef);
void clover_force(pfmp_ctx* c, int prec, double* F, const double* Hc);
void gauge_force(pfmp_ctx* c, int prec, double* F, double beta);

// blas.cu
void blas_zero(pfmp_ctx* c, int prec, void* x);
void blas_copy(pfmp_ctx* c, void* dst, int dprec, const void* src, int sprec);
void blas_axpy(pfmp_ctx* c, int prec, double are, double aim, const void* x, void* y);
void blas_norm2(pfmp_ctx* c, int prec, const void* x, double* out_dev);
void blas_cdot(pfmp_ctx* c, int prec, const void* x, const void* y, double* out_dev);
// r = b - Ax (F64), returns |r|^2 into out_dev
void blas_xmy_norm(pfmp_ctx* c, const void* b, const void* Ax, void* r, double* out_dev);
// CG steps (device scalars)
void cg_step_xr(pfmp_ctx* c, int prec, void* x, void* r, const void* p, const void* Ap, CGScalars* s);
void cg_step_p(pfmp_ctx* c, int prec, void* p, const void* r, CGScalars* s);
// x64 += x32 (accumulate the sloppy solution)
void blas_add_lo(pfmp_ctx* c, void* x64, const void* x32);

// multishift.cu
void caxpby(pfmp_ctx* c, std::complex<double> a, const void* x, std::complex<double> b, void* y);  // FP64
void caxpby(pfmp_ctx* c, int prec, std::complex<double> a, const void* x, std::complex<double> b, void* y);
int solve_multishift(pfmp_op* op, int prec, int ns, const std::complex<double>* sigma, void* const* x, const void* b,
                     double tol, int max_iter, int check, int* iters, double* max_true_res, long* kapply,
                     bool want_true_res);
// bit-reversed permutation of 0..n-1, and a root list in that order (stable products)
std::vector<int> stable_order(int n);
std::vector<std::complex<double>> stable_ordered(const std::vector<std::complex<double>>& z);
void ms_work_free(pfmp_op* op);
std::vector<std::complex<double>> cheb_roots(int n, double mu, double nu);
double cheb_norm(int n, double mu, double nu);
void poly_product(pfmp_op* op, const std::vector<std::complex<double>>& z, double scale, void* out, const void* in);

// probe.cu: measured FMA throughput (TFLOP/s) of the FP64 or FP32 pipe
double fma_rate(pfmp_ctx* c, int prec);

// solver.cu
int solve(pfmp_op* op, int method, double tol, int max_iter, double delta, int check_every, void* x,
          const void* b, int* iters, int* rel_updates, double* true_res, long* kapply);

}  // namespace pfmp
