// Gauge-covariant network (a learned flexible preconditioner) and FGCR.
//
// Layer (C_in -> C_out), for every site x and output channel o:
//   y_o(x) = sum_i [ W_0[o][i] a_i(x) + sum_mu ( W_{1+mu}[o][i] U_mu(x) a_i(x+mu)
//                                             + W_{5+mu}[o][i] U_mu(x-mu)^dag a_i(x-mu) ) ]
// W complex 4x4 on spin, U on colour, the fermion boundary factor on time hops.  The
// network is linear (a fixed operator, so FGCR sees one preconditioner), channels
// 1 -> C -> ... -> 1, input embedded on even sites, output read on even sites.
//
// Activations: complex [C][12][V] over the full lattice (lexicographic site index).
// Kernels: forward layer and its adjoint (thread per (site, channel); the adjoint of a
// forward hop is a backward transport with W^dag and vice versa), the weight gradient
// (per-site outer products summed over colour, warp shuffles, one atomic per warp),
// loss + its gradient, and Adam.  Templated on FP32 / FP64 (the FP64 instance is the
// one checked against the oracle's autograd gradients).
//
// FGCR (flexible GCR with restarts): FP32 inner iterations z_k = N(r), w_k = K z_k
// orthonormalised against earlier w_j (modified Gram-Schmidt, the same combination
// applied to z_k), e += <w_k, r> z_k, r -= <w_k, r> w_k; the FP64 outer loop adds e to x
// and recomputes b - K x in FP64, so the network can only change the path, never the
// answer.  Without progress the remaining correction is solved by the mixed CG.
#include <cmath>
#include <complex>
#include <vector>

#include "context.h"
#include "fields.cuh"

namespace pfmp {

template <typename T>
struct C2;
template <>
struct C2<double> {
  using t = double2;
};
template <>
struct C2<float> {
  using t = float2;
};

template <typename T>
__device__ __forceinline__ cplx<T> ld(const typename C2<T>::t* p, size_t i) {
  typename C2<T>::t v = p[i];
  return mk(v.x, v.y);
}
template <typename T>
__device__ __forceinline__ void st(typename C2<T>::t* p, size_t i, cplx<T> v) {
  typename C2<T>::t w;
  w.x = v.re;
  w.y = v.im;
  p[i] = w;
}

// link U_mu(y) from the master FP64 field, in precision T
template <typename T>
__device__ __forceinline__ Mat3<T> link_T(const double2* U, const Geom& g, const int y[4], int mu) {
  const int p = (y[0] + y[1] + y[2] + y[3]) & 1;
  Mat3<double> M;
  load_link18(M, U + (size_t)((p * 4 + mu) * 9) * g.Vh, cb_index(g, y), g.Vh);
  Mat3<T> R;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) R.m[i][j] = mk((T)M.m[i][j].re, (T)M.m[i][j].im);
  return R;
}

__device__ __forceinline__ void lex_coords(const Geom& g, int s, int x[4]) {
  x[0] = s % g.L[0];
  s /= g.L[0];
  x[1] = s % g.L[1];
  s /= g.L[1];
  x[2] = s % g.L[2];
  x[3] = s / g.L[2];
}

// transport of channel field a (at offset) to site x: kind 0 = site itself,
// 1 = forward U_mu(x) a(x+mu), 2 = backward U_mu(x-mu)^dag a(x-mu)
template <typename T>
__device__ __forceinline__ void transport(const typename C2<T>::t* a, const double2* U, const Geom& g, const int x[4],
                                          int kind, int mu, cplx<T> out[12]) {
  const size_t V = g.V;
  if (kind == 0) {
    const int s = lex_index(g, x);
    for (int k = 0; k < 12; ++k) out[k] = ld<T>(a, (size_t)k * V + s);
    return;
  }
  int y[4] = {x[0], x[1], x[2], x[3]};
  T bc = (T)1;
  if (kind == 1) {
    y[mu] = (y[mu] + 1) % g.L[mu];
    if (mu == 3 && x[3] == g.L[3] - 1) bc = (T)g.bc_t;
    const Mat3<T> Um = link_T<T>(U, g, x, mu);
    const int s = lex_index(g, y);
    for (int sp = 0; sp < 4; ++sp) {
      cplx<T> v[3];
      for (int c = 0; c < 3; ++c) v[c] = ld<T>(a, (size_t)(sp * 3 + c) * V + s);
      for (int i = 0; i < 3; ++i) out[sp * 3 + i] = bc * (Um.m[i][0] * v[0] + Um.m[i][1] * v[1] + Um.m[i][2] * v[2]);
    }
  } else {
    y[mu] = (y[mu] - 1 + g.L[mu]) % g.L[mu];
    if (mu == 3 && x[3] == 0) bc = (T)g.bc_t;
    const Mat3<T> Um = link_T<T>(U, g, y, mu);
    const int s = lex_index(g, y);
    for (int sp = 0; sp < 4; ++sp) {
      cplx<T> v[3];
      for (int c = 0; c < 3; ++c) v[c] = ld<T>(a, (size_t)(sp * 3 + c) * V + s);
      for (int i = 0; i < 3; ++i)
        out[sp * 3 + i] = bc * (cj_mul(Um.m[0][i], v[0]) + cj_mul(Um.m[1][i], v[1]) + cj_mul(Um.m[2][i], v[2]));
    }
  }
}

// W index helpers: W[d][o][i][s][s'] complex
__device__ __forceinline__ size_t widx(int d, int o, int i, int cout, int cin) {
  return ((((size_t)d * cout + o) * cin + i) * 16);
}

// forward layer (ADJ = false): out[o] = sum_d sum_i W_d[o][i] S_d in[i]
// adjoint (ADJ = true): out[i] = sum_d sum_o W_d[o][i]^dag S_d^dag in[o]
template <typename T, bool ADJ>
__global__ void k_nn_layer(Geom g, const double2* __restrict__ U, const typename C2<T>::t* __restrict__ W, int cin,
                           int cout, const typename C2<T>::t* __restrict__ in, typename C2<T>::t* __restrict__ out) {
  const int nout = ADJ ? cin : cout;
  const int nin = ADJ ? cout : cin;
  const long tid = blockIdx.x * (long)blockDim.x + threadIdx.x;
  if (tid >= (long)g.V * nout) return;
  const int s = (int)(tid % g.V);
  const int oc = (int)(tid / g.V);
  int x[4];
  lex_coords(g, s, x);
  cplx<T> acc[12];
  for (int k = 0; k < 12; ++k) acc[k] = mk<T>(0, 0);
  for (int d = 0; d < 9; ++d) {
    int kind = d == 0 ? 0 : (d <= 4 ? 1 : 2);
    const int mu = d == 0 ? 0 : (d - 1) % 4;
    if (ADJ && kind) kind = 3 - kind;  // adjoint of a forward hop is a backward transport
    for (int ic = 0; ic < nin; ++ic) {
      cplx<T> t[12];
      transport<T>(in + (size_t)ic * 12 * g.V, U, g, x, kind, mu, t);
      const size_t w0 = ADJ ? widx(d, ic, oc, cout, cin) : widx(d, oc, ic, cout, cin);
      for (int a = 0; a < 4; ++a)
        for (int b = 0; b < 4; ++b) {
          // forward: W[a][b] (row a, col b); adjoint: conj(W[b][a])
          cplx<T> w = ADJ ? conj(ld<T>(W, w0 + b * 4 + a)) : ld<T>(W, w0 + a * 4 + b);
          for (int c = 0; c < 3; ++c) acc[a * 3 + c] = acc[a * 3 + c] + w * t[b * 3 + c];
        }
    }
  }
  for (int k = 0; k < 12; ++k) st<T>(out, ((size_t)oc * 12 + k) * g.V + s, acc[k]);
}

// forward layer with every output channel of a site in one thread (COUT small): the
// parallel transports are computed once per (direction, input channel) and the layer's
// weights sit in shared memory
template <typename T, int COUT>
__global__ void __launch_bounds__(128) k_nn_layer_site(Geom g, const double2* __restrict__ U,
                                                       const typename C2<T>::t* __restrict__ W, int cin,
                                                       const typename C2<T>::t* __restrict__ in,
                                                       typename C2<T>::t* __restrict__ out) {
  extern __shared__ unsigned char smem_raw[];
  typename C2<T>::t* Ws = reinterpret_cast<typename C2<T>::t*>(smem_raw);
  const int nw = 9 * COUT * cin * 16;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) Ws[i] = W[i];
  __syncthreads();
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  lex_coords(g, s, x);
  cplx<T> acc[COUT][12];
#pragma unroll
  for (int o = 0; o < COUT; ++o)
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[o][k] = mk<T>(0, 0);
  for (int d = 0; d < 9; ++d) {
    const int kind = d == 0 ? 0 : (d <= 4 ? 1 : 2);
    const int mu = d == 0 ? 0 : (d - 1) % 4;
    for (int ic = 0; ic < cin; ++ic) {
      cplx<T> t[12];
      transport<T>(in + (size_t)ic * 12 * g.V, U, g, x, kind, mu, t);
#pragma unroll
      for (int o = 0; o < COUT; ++o) {
        const typename C2<T>::t* w0 = Ws + widx(d, o, ic, COUT, cin);
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) {
            const cplx<T> w = mk(w0[a * 4 + b].x, w0[a * 4 + b].y);
#pragma unroll
            for (int c = 0; c < 3; ++c) acc[o][a * 3 + c] = acc[o][a * 3 + c] + w * t[b * 3 + c];
          }
      }
    }
  }
#pragma unroll
  for (int o = 0; o < COUT; ++o)
#pragma unroll
    for (int k = 0; k < 12; ++k) st<T>(out, ((size_t)o * 12 + k) * g.V + s, acc[o][k]);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// gW_d[o][i] += sum_{x, colour} gout_o(x) (S_d in_i)(x)^dag (4x4 spin outer product)
template <typename T>
__global__ void k_nn_wgrad(Geom g, const double2* __restrict__ U, int cin, int cout,
                           const typename C2<T>::t* __restrict__ in, const typename C2<T>::t* __restrict__ gout,
                           T* __restrict__ gW) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const bool live = s < g.V;
  int x[4] = {0, 0, 0, 0};
  if (live) lex_coords(g, s, x);
  for (int d = 0; d < 9; ++d) {
    const int kind = d == 0 ? 0 : (d <= 4 ? 1 : 2);
    const int mu = d == 0 ? 0 : (d - 1) % 4;
    for (int ic = 0; ic < cin; ++ic) {
      cplx<T> t[12];
      if (live)
        transport<T>(in + (size_t)ic * 12 * g.V, U, g, x, kind, mu, t);
      else
        for (int k = 0; k < 12; ++k) t[k] = mk<T>(0, 0);
      for (int oc = 0; oc < cout; ++oc) {
        cplx<T> go[12];
        for (int k = 0; k < 12; ++k) go[k] = live ? ld<T>(gout, ((size_t)oc * 12 + k) * g.V + s) : mk<T>(0, 0);
        const size_t w0 = widx(d, oc, ic, cout, cin);
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b) {
            cplx<T> v = mk<T>(0, 0);
            for (int c = 0; c < 3; ++c) v = v + mul_cj(go[a * 3 + c], t[b * 3 + c]);
            T re = warp_sum(v.re), im = warp_sum(v.im);
            if ((threadIdx.x & 31) == 0) {
              atomicAdd(gW + 2 * (w0 + a * 4 + b), re);
              atomicAdd(gW + 2 * (w0 + a * 4 + b) + 1, im);
            }
          }
      }
    }
  }
}

// even device spinor (F32 [6][Vh] float4 or F64 [12][Vh] double2) <-> network channel 0
template <typename T, int PREC>
__global__ void k_nn_embed(Geom g, const typename Prec<PREC>::vec* __restrict__ src, typename C2<T>::t* __restrict__ dst) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  lex_coords(g, s, x);
  const bool even = ((x[0] + x[1] + x[2] + x[3]) & 1) == 0;
  Spinor<typename Prec<PREC>::real> v;
  if (even) load_spinor(v, src, s >> 1, g.Vh);
  for (int k = 0; k < 12; ++k) {
    cplx<T> c = even ? mk((T)v.s[k / 3][k % 3].re, (T)v.s[k / 3][k % 3].im) : mk<T>(0, 0);
    st<T>(dst, (size_t)k * g.V + s, c);
  }
}
template <typename T, int PREC>
__global__ void k_nn_extract(Geom g, const typename C2<T>::t* __restrict__ src, typename Prec<PREC>::vec* __restrict__ dst) {
  const int cb = blockIdx.x * blockDim.x + threadIdx.x;
  if (cb >= g.Vh) return;
  int x[4];
  cb_coords(g, cb, 0, x);
  const int s = lex_index(g, x);
  using R = typename Prec<PREC>::real;
  Spinor<R> v;
  for (int k = 0; k < 12; ++k) {
    cplx<T> c = ld<T>(src, (size_t)k * g.V + s);
    v.s[k / 3][k % 3] = mk((R)c.re, (R)c.im);
  }
  store_spinor(dst, v, cb, g.Vh);
}

// loss sum_even |y - x|^2 (and |x|^2), gradient g = 2 (y - x) / |x|^2 on even sites
template <typename T>
__global__ void k_nn_loss(Geom g, const typename C2<T>::t* __restrict__ y, const typename C2<T>::t* __restrict__ xt,
                          ReduceBuf rb, double* out) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  double v[2] = {0.0, 0.0};
  if (s < g.V) {
    int x[4];
    lex_coords(g, s, x);
    if (((x[0] + x[1] + x[2] + x[3]) & 1) == 0)
      for (int k = 0; k < 12; ++k) {
        cplx<T> a = ld<T>(y, (size_t)k * g.V + s), b = ld<T>(xt, (size_t)k * g.V + s);
        v[0] += (double)norm2(a - b);
        v[1] += (double)norm2(b);
      }
  }
  double t[2];
  if (grid_sum<2>(v, rb, t)) {
    out[0] = t[0];
    out[1] = t[1];
  }
}
template <typename T>
__global__ void k_nn_lossgrad(Geom g, const typename C2<T>::t* __restrict__ y, const typename C2<T>::t* __restrict__ xt,
                              const double* __restrict__ sums, T scale, typename C2<T>::t* __restrict__ gy) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int x[4];
  lex_coords(g, s, x);
  const bool even = ((x[0] + x[1] + x[2] + x[3]) & 1) == 0;
  const T f = (T)(2.0 / sums[1]) * scale;
  for (int k = 0; k < 12; ++k) {
    cplx<T> v = even ? f * (ld<T>(y, (size_t)k * g.V + s) - ld<T>(xt, (size_t)k * g.V + s)) : mk<T>(0, 0);
    st<T>(gy, (size_t)k * g.V + s, v);
  }
}

template <typename T>
__global__ void k_adam(T* __restrict__ w, const T* __restrict__ gw, T* __restrict__ m, T* __restrict__ v, long n, T lr,
                       T b1, T b2, T eps, T c1, T c2) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const T gr = gw[i];
    const T mi = b1 * m[i] + (1 - b1) * gr;
    const T vi = b2 * v[i] + (1 - b2) * gr * gr;
    m[i] = mi;
    v[i] = vi;
    w[i] -= lr * (mi / c1) / (sqrt(vi / c2) + eps);
  }
}

// ---- fused FGCR steps (FP32 fields, FP64 sums) --------------------------------------
struct CoefList {
  float2 h[32];
};

// runtime-length block sum of v[0..nv) (nv <= 34); returns true in thread 0 of the last
// block, whose out[0..nv) then holds the grid totals (deterministic order).  The last
// block adds the per-block partials with all its threads, one value at a time.
__device__ bool grid_sum_n(double* v, int nv, double* partials, unsigned* ticket, double* out) {
  __shared__ double sh[34][32];
  __shared__ bool last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int k = 0; k < nv; ++k) {
    double t = v[k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[k][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0;
    for (int w = 0; w < nw; ++w) t += sh[threadIdx.x][w];
    partials[(size_t)blockIdx.x * nv + threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (!last) return false;
  __threadfence();
  for (int k = 0; k < nv; ++k) {
    double t = 0;
    for (unsigned b = threadIdx.x; b < gridDim.x; b += blockDim.x) t += ((volatile double*)partials)[(size_t)b * nv + k];
    for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
    if (lane == 0) sh[k][warp] = t;
  }
  __syncthreads();
  if (threadIdx.x < nv) {
    double t = 0;
    for (int w = 0; w < nw; ++w) t += sh[threadIdx.x][w];
    out[threadIdx.x] = t;
  }
  if (threadIdx.x == 0) *ticket = 0u;
  return threadIdx.x == 0;
}

// The inner FGCR iteration runs without host round trips: the Gram-Schmidt coefficients,
// |w|^2, the step alpha and the residual norm stay in device memory, and the solver
// scalars' `done` flag (set by the step kernel's last block once |r| has fallen by delta)
// makes every later kernel of the cycle return at once.

// h_j = <W_j, w> (j < k) and <w, r>: out[2j], out[2j+1], out[2k], out[2k+1].  Block row
// y of the grid takes one product (y < k: <W_y, w>, y = k: <w, r>) and writes one partial
// per block; k_fgcr_dots_final adds each row's partials in a fixed order.
__global__ void k_fgcr_dots_part(float4* const* __restrict__ Wp, int k, const float4* __restrict__ w,
                                 const float4* __restrict__ r, long n, double* partials,
                                 const CGScalars* __restrict__ s) {
  if (s->done) return;
  const int y = blockIdx.y;
  const float4* __restrict__ q = y < k ? Wp[y] : r;
  // each thread's few products in FP32 (GB300's FP64 pipe is a small fraction of the FP32
  // one), the sums across threads and blocks in FP64
  float pr = 0.f, pi = 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    const float4 a = w[i], c = q[i];
    if (y < k) {  // conj(W_y) w
      pr += c.x * a.x + c.y * a.y + c.z * a.z + c.w * a.w;
      pi += c.x * a.y - c.y * a.x + c.z * a.w - c.w * a.z;
    } else {      // conj(w) r
      pr += a.x * c.x + a.y * c.y + a.z * c.z + a.w * c.w;
      pi += a.x * c.y - a.y * c.x + a.z * c.w - a.w * c.z;
    }
  }
  double v[2] = {(double)pr, (double)pi};
  __shared__ double sh[2 * 32];
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    partials[((size_t)y * gridDim.x + blockIdx.x) * 2] = v[0];
    partials[((size_t)y * gridDim.x + blockIdx.x) * 2 + 1] = v[1];
  }
}

__global__ void k_fgcr_dots_final(int nblk, const double* __restrict__ partials, double* __restrict__ out,
                                  const CGScalars* __restrict__ s) {
  if (s->done) return;
  const int y = blockIdx.x;
  double v[2] = {0.0, 0.0};
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) {
    v[0] += partials[((size_t)y * nblk + b) * 2];
    v[1] += partials[((size_t)y * nblk + b) * 2 + 1];
  }
  __shared__ double sh[2 * 32];
  block_sum<2>(v, sh);
  if (threadIdx.x == 0) {
    out[2 * y] = v[0];
    out[2 * y + 1] = v[1];
  }
}

// w -= sum_j h_j W_j, z -= sum_j h_j Z_j with h from the dots; *n2 = |w|^2
__global__ void k_fgcr_orth(float4* const* __restrict__ Wp, float4* const* __restrict__ Zp, int k,
                            const double* __restrict__ hd, float4* __restrict__ w, float4* __restrict__ z, long n,
                            double* partials, unsigned* ticket, double* n2, const CGScalars* __restrict__ s) {
  if (s->done) return;
  __shared__ float2 h[16];
  if (threadIdx.x < k) h[threadIdx.x] = make_float2((float)hd[2 * threadIdx.x], (float)hd[2 * threadIdx.x + 1]);
  __syncthreads();
  double v[1] = {0.0};
  float nt = 0.f;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float4 a = w[i], b = z[i];
    for (int j = 0; j < k; ++j) {
      const float2 c = h[j];
      const float4 q = Wp[j][i], p = Zp[j][i];
      a.x -= c.x * q.x - c.y * q.y;
      a.y -= c.x * q.y + c.y * q.x;
      a.z -= c.x * q.z - c.y * q.w;
      a.w -= c.x * q.w + c.y * q.z;
      b.x -= c.x * p.x - c.y * p.y;
      b.y -= c.x * p.y + c.y * p.x;
      b.z -= c.x * p.z - c.y * p.w;
      b.w -= c.x * p.w + c.y * p.z;
    }
    w[i] = a;
    z[i] = b;
    nt += a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;
  }
  v[0] = nt;  // per-thread sum in FP32, across threads in FP64
  grid_sum_n(v, 1, partials, ticket, n2);
}

// alpha = <w, r> / |w|^2: r -= alpha w, e += alpha z, then w, z scaled to unit |w|; the
// last block updates |r|^2 = |r|^2 - |<w, r>|^2 / |w|^2 (r is orthogonal to the earlier
// directions), counts the iteration and raises `done` below stop_rr (or when w vanished)
__global__ void k_fgcr_step(float4* __restrict__ w, float4* __restrict__ z, float4* __restrict__ r,
                            float4* __restrict__ e, const double* __restrict__ dots, int k,
                            const double* __restrict__ n2p, long n, CGScalars* s, unsigned* ticket) {
  if (s->done) return;
  const double n2 = *n2p;
  const double wr_re = dots[2 * k], wr_im = dots[2 * k + 1];
  const bool ok = n2 > 0;
  if (ok) {
    const float2 al = make_float2((float)(wr_re / n2), (float)(wr_im / n2));
    const float sc = (float)(1.0 / sqrt(n2));
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
      float4 a = w[i], b = z[i], rr = r[i], ee = e[i];
      rr.x -= al.x * a.x - al.y * a.y;
      rr.y -= al.x * a.y + al.y * a.x;
      rr.z -= al.x * a.z - al.y * a.w;
      rr.w -= al.x * a.w + al.y * a.z;
      ee.x += al.x * b.x - al.y * b.y;
      ee.y += al.x * b.y + al.y * b.x;
      ee.z += al.x * b.z - al.y * b.w;
      ee.w += al.x * b.w + al.y * b.z;
      r[i] = rr;
      e[i] = ee;
      w[i] = make_float4(sc * a.x, sc * a.y, sc * a.z, sc * a.w);
      z[i] = make_float4(sc * b.x, sc * b.y, sc * b.z, sc * b.w);
    }
  }
  __shared__ bool last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    last = atomicAdd(ticket, 1u) == gridDim.x - 1;
  }
  __syncthreads();
  if (last && threadIdx.x == 0) {
    *ticket = 0u;
    if (ok) {
      double rr = s->rr - (wr_re * wr_re + wr_im * wr_im) / n2;
      s->rr = rr > 0 ? rr : 0.0;
      s->iter += 1;
    }
    if (!ok || s->rr < s->stop_rr) s->done = 1;
  }
}

// z = r (GCR: no preconditioner) unless done
__global__ void k_fgcr_copy(float4* __restrict__ z, const float4* __restrict__ r, long n, const CGScalars* s) {
  if (s->done) return;
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) z[i] = r[i];
}

// start of a cycle: rr = |r|^2 (already in s->rr), stop = max(delta^2 rr, floor)
__global__ void k_fgcr_start(CGScalars* s, double delta2, double floor_rr) {
  const double st = delta2 * s->rr;
  s->stop_rr = st > floor_rr ? st : floor_rr;
  s->done = 0;
  s->iter = 0;
}

__global__ void k_scale32(float4* x, float a, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    float4 v = x[i];
    x[i] = make_float4(a * v.x, a * v.y, a * v.z, a * v.w);
  }
}

}  // namespace pfmp

using namespace pfmp;

struct pfmp_nn {
  pfmp_ctx* ctx = nullptr;
  int prec = PFMP_F32;
  std::vector<int> ch;             // channels, nlayers + 1
  std::vector<void*> W, gW, m, v;  // per layer (complex, elem = real pairs)
  std::vector<long> nw;            // complex weights per layer
  std::vector<void*> act;          // nlayers + 1 activations (max channels each)
  void* gbuf[2] = {nullptr, nullptr};
  void* target = nullptr;
  void* ev[3] = {nullptr, nullptr, nullptr};  // even fields for the residual loss
  double last_norm = 1;
  int maxc = 1;
  long step = 0;
  // tensor-core inference of the C -> C layers (nn_tc.cu)
  bool tc = false;               // use it in nn_apply
  bool packed = false;           // Bp holds the current weights
  std::vector<void*> Bp;         // packed FP16 operand per layer
  std::vector<void*> act16;      // FP16 scaled inputs of each layer
  void* z16 = nullptr;           // last layer: FP16 per-direction mixed outputs [9][12][V]
  float* sigma = nullptr;        // device scalar: 1 / rms of the network input
  int* err = nullptr;            // device error flag of the tensor-core kernel
  long long id = 0;              // unique per network (keys the FGCR cycle graphs)
};

namespace pfmp {

static size_t csz(const pfmp_nn* N) { return N->prec == PFMP_F64 ? sizeof(double2) : sizeof(float2); }

bool nn_tc_supported(int cin, int cout);
size_t nn_tc_packed_bytes(int cin, int cout);
void nn_tc_pack(pfmp_ctx* c, int cin, int cout, const void* W, void* Bp);
void nn_tc_scale(pfmp_ctx* c, const void* in_even_f32, float* sigma_dev, const int* skip);
void nn_tc_layer(pfmp_ctx* c, int cin, int cout, bool last, const void* Bp, const void* in, void* out,
                 const float* sigma, int* err, const int* skip);
void nn_tc_embed(pfmp_ctx* c, const void* in_even_f32, float* sigma, void* act16, const int* skip, const double* rr);
void nn_tc_last(pfmp_ctx* c, const void* Bp, const void* in, void* z16, void* out_even_f32, const float* sigma,
                int* err, const int* skip);
void nn_tc_init();

void nn_destroy(pfmp_nn* N) {
  if (!N) return;
  for (auto* vec : {&N->W, &N->gW, &N->m, &N->v, &N->act, &N->Bp, &N->act16})
    for (auto p : *vec) dev_free(p);
  dev_free(N->sigma);
  dev_free(N->err);
  dev_free(N->z16);
  dev_free(N->gbuf[0]);
  dev_free(N->gbuf[1]);
  dev_free(N->target);
  for (auto p : N->ev) dev_free(p);
  delete N;
}

pfmp_nn* nn_create(pfmp_ctx* c, int nl, const int* ch, int prec) {
  PFMP_REQUIRE(nl >= 1 && nl <= 16 && ch, PFMP_E_INVALID, "need 1..16 layers");
  PFMP_REQUIRE(ch[0] == 1 && ch[nl] == 1, PFMP_E_INVALID, "the network maps one spinor to one spinor");
  PFMP_REQUIRE(prec == PFMP_F32 || prec == PFMP_F64, PFMP_E_INVALID, "bad precision");
  static long long next_id = 0;
  pfmp_nn* N = new pfmp_nn();
  N->ctx = c;
  N->prec = prec;
  N->id = ++next_id;
  try {
    for (int l = 0; l <= nl; ++l) {
      PFMP_REQUIRE(ch[l] >= 1 && ch[l] <= 64, PFMP_E_INVALID, "channels must be in 1..64");
      N->ch.push_back(ch[l]);
      N->maxc = std::max(N->maxc, ch[l]);
    }
    for (int l = 0; l < nl; ++l) {
      const long n = 9L * ch[l] * ch[l + 1] * 16;
      N->nw.push_back(n);
      for (auto* vec : {&N->W, &N->gW, &N->m, &N->v}) {
        void* p = dev_alloc(n * csz(N));
        PFMP_CUDA(cudaMemset(p, 0, n * csz(N)));
        vec->push_back(p);
      }
    }
    for (int l = 0; l <= nl; ++l) N->act.push_back(dev_alloc((size_t)ch[l] * 12 * c->g.V * csz(N)));
    for (auto& p : N->gbuf) p = dev_alloc((size_t)N->maxc * 12 * c->g.V * csz(N));
    N->target = dev_alloc((size_t)12 * c->g.V * csz(N));
    for (auto& p : N->ev) p = dev_alloc(spinor_bytes(c->g, prec));
    bool all = prec == PFMP_F32 && nl >= 2;
    for (int l = 0; l < nl; ++l) all = all && nn_tc_supported(ch[l], ch[l + 1]);
    if (all) {  // every layer on the tensor cores (1 -> 8, 8 -> 8 ..., 8 -> 1)
      for (int l = 0; l < nl; ++l) {
        N->Bp.push_back(dev_alloc(nn_tc_packed_bytes(ch[l], ch[l + 1])));
        N->act16.push_back(dev_alloc((size_t)ch[l] * 12 * c->g.V * 4));
      }
      N->z16 = dev_alloc((size_t)9 * 12 * c->g.V * 4);
      N->tc = true;
      N->sigma = (float*)dev_alloc(sizeof(float));
      N->err = (int*)dev_alloc(sizeof(int));
      PFMP_CUDA(cudaMemset(N->err, 0, sizeof(int)));
    }
  } catch (...) {
    nn_destroy(N);
    throw;
  }
  return N;
}

long nn_num_weights(const pfmp_nn* N) {
  long t = 0;
  for (long n : N->nw) t += n;
  return t;
}

void nn_set_weights(pfmp_nn* N, const double* w) {
  long off = 0;
  for (size_t l = 0; l < N->W.size(); ++l) {
    const long n = N->nw[l];
    if (N->prec == PFMP_F64) {
      PFMP_CUDA(cudaMemcpy(N->W[l], w + 2 * off, n * sizeof(double2), cudaMemcpyHostToDevice));
    } else {
      std::vector<float> f(2 * n);
      for (long i = 0; i < 2 * n; ++i) f[i] = (float)w[2 * off + i];
      PFMP_CUDA(cudaMemcpy(N->W[l], f.data(), n * sizeof(float2), cudaMemcpyHostToDevice));
    }
    PFMP_CUDA(cudaMemset(N->m[l], 0, n * csz(N)));
    PFMP_CUDA(cudaMemset(N->v[l], 0, n * csz(N)));
    off += n;
  }
  N->step = 0;
  N->packed = false;
}

static void copy_out(pfmp_nn* N, const std::vector<void*>& src, double* w) {
  PFMP_CUDA(cudaStreamSynchronize(N->ctx->stream));
  long off = 0;
  for (size_t l = 0; l < src.size(); ++l) {
    const long n = N->nw[l];
    if (N->prec == PFMP_F64) {
      PFMP_CUDA(cudaMemcpy(w + 2 * off, src[l], n * sizeof(double2), cudaMemcpyDeviceToHost));
    } else {
      std::vector<float> f(2 * n);
      PFMP_CUDA(cudaMemcpy(f.data(), src[l], n * sizeof(float2), cudaMemcpyDeviceToHost));
      for (long i = 0; i < 2 * n; ++i) w[2 * off + i] = f[i];
    }
    off += n;
  }
}
void nn_get_weights(pfmp_nn* N, double* w) { copy_out(N, N->W, w); }

// tensor-core inference on / off (only FP32 networks with C -> C layers have it)
void nn_set_tc(pfmp_nn* N, bool on) {
  PFMP_REQUIRE(!on || !N->Bp.empty(), PFMP_E_UNSUPPORTED,
               "tensor-core inference needs an FP32 network 1 -> 8 -> ... -> 8 -> 1");
  N->tc = on;
}

// raises PFMP_E_TIMEOUT if a tensor-core kernel gave up waiting (synchronises)
void nn_check(pfmp_nn* N) {
  if (!N->err) return;
  int e = 0;
  PFMP_CUDA(cudaMemcpyAsync(&e, N->err, sizeof(int), cudaMemcpyDeviceToHost, N->ctx->stream));
  PFMP_CUDA(cudaStreamSynchronize(N->ctx->stream));
  if (e) {
    PFMP_CUDA(cudaMemsetAsync(N->err, 0, sizeof(int), N->ctx->stream));
    PFMP_REQUIRE(false, PFMP_E_TIMEOUT, "tensor-core network layer timed out waiting for its MMAs");
  }
}
void nn_get_grads(pfmp_nn* N, double* w) { copy_out(N, N->gW, w); }

template <typename T, int CO>
static bool layer_site(pfmp_ctx* c, const void* W, int cin, const void* in, void* out) {
  using C = typename C2<T>::t;
  const size_t sm = (size_t)9 * CO * cin * 16 * sizeof(C);
  if (sm > 48 * 1024) return false;
  k_nn_layer_site<T, CO><<<nblocks(c->g.V, 128), 128, sm, c->stream>>>(c->g, c->U64, (const C*)W, cin, (const C*)in,
                                                                      (C*)out);
  PFMP_CHECK_LAUNCH();
  return true;
}

// packed FP16 weights up to date and kernel attributes set (outside any stream capture)
static void tc_prepare(pfmp_nn* N) {
  if (!N->packed) {
    for (size_t l = 0; l < N->W.size(); ++l) nn_tc_pack(N->ctx, N->ch[l], N->ch[l + 1], N->W[l], N->Bp[l]);
    N->packed = true;
  }
  nn_tc_init();
}

// tensor-core forward pass: in (even FP32) -> out (even FP32) through FP16 activations;
// every kernel returns at once while *skip is set (FGCR after convergence)
// rr (optional): device |in|^2 known to the caller, used for the input scale
static void forward_tc(pfmp_nn* N, void* out, const void* in, const int* skip, const double* rr) {
  pfmp_ctx* c = N->ctx;
  const int L = (int)N->W.size();
  if (!rr) nn_tc_scale(c, in, N->sigma, skip);
  nn_tc_embed(c, in, N->sigma, N->act16[0], skip, rr);
  for (int l = 0; l < L - 1; ++l)
    nn_tc_layer(c, N->ch[l], N->ch[l + 1], false, N->Bp[l], N->act16[l], N->act16[l + 1], N->sigma, N->err, skip);
  // the last layer mixes channels at each site first and transports after (the colour
  // transport commutes with the spin/channel weights), on even sites only
  nn_tc_last(c, N->Bp[L - 1], N->act16[L - 1], N->z16, out, N->sigma, N->err, skip);
}

template <typename T>
static void forward_t(pfmp_nn* N) {
  pfmp_ctx* c = N->ctx;
  using C = typename C2<T>::t;
  for (size_t l = 0; l < N->W.size(); ++l) {
    const int cin = N->ch[l], cout = N->ch[l + 1];
    bool done = false;
    if (cout == 1) done = layer_site<T, 1>(c, N->W[l], cin, N->act[l], N->act[l + 1]);
    else if (cout == 2) done = layer_site<T, 2>(c, N->W[l], cin, N->act[l], N->act[l + 1]);
    else if (cout == 4) done = layer_site<T, 4>(c, N->W[l], cin, N->act[l], N->act[l + 1]);
    if (done) continue;
    const long n = (long)c->g.V * cout;
    k_nn_layer<T, false><<<nblocks(n, 128), 128, 0, c->stream>>>(c->g, c->U64, (const C*)N->W[l], cin, cout,
                                                                  (const C*)N->act[l], (C*)N->act[l + 1]);
    PFMP_CHECK_LAUNCH();
  }
}

// out_even = N(in_even); io precision prec_io (device layout of the library); skip: see
// forward_tc (tensor-core path only)
static void nn_apply_skip(pfmp_nn* N, void* out, const void* in, int prec_io, const int* skip,
                          const double* rr = nullptr) {
  pfmp_ctx* c = N->ctx;
  const Geom& g = c->g;
  const int L = (int)N->W.size();
  if (N->prec == PFMP_F64) {
    if (prec_io == PFMP_F64)
      k_nn_embed<double, PFMP_F64><<<nblocks(g.V), kBlock, 0, c->stream>>>(g, (const double2*)in, (double2*)N->act[0]);
    else
      k_nn_embed<double, PFMP_F32><<<nblocks(g.V), kBlock, 0, c->stream>>>(g, (const float4*)in, (double2*)N->act[0]);
    PFMP_CHECK_LAUNCH();
    forward_t<double>(N);
    if (prec_io == PFMP_F64)
      k_nn_extract<double, PFMP_F64><<<nblocks(g.Vh), kBlock, 0, c->stream>>>(g, (const double2*)N->act[L], (double2*)out);
    else
      k_nn_extract<double, PFMP_F32><<<nblocks(g.Vh), kBlock, 0, c->stream>>>(g, (const double2*)N->act[L], (float4*)out);
  } else {
    if (N->tc && prec_io == PFMP_F32) {
      tc_prepare(N);
      forward_tc(N, out, in, skip, rr);
      return;
    }
    if (prec_io == PFMP_F64)
      k_nn_embed<float, PFMP_F64><<<nblocks(g.V), kBlock, 0, c->stream>>>(g, (const double2*)in, (float2*)N->act[0]);
    else
      k_nn_embed<float, PFMP_F32><<<nblocks(g.V), kBlock, 0, c->stream>>>(g, (const float4*)in, (float2*)N->act[0]);
    PFMP_CHECK_LAUNCH();
    forward_t<float>(N);
    if (prec_io == PFMP_F64)
      k_nn_extract<float, PFMP_F64><<<nblocks(g.Vh), kBlock, 0, c->stream>>>(g, (const float2*)N->act[L], (double2*)out);
    else
      k_nn_extract<float, PFMP_F32><<<nblocks(g.Vh), kBlock, 0, c->stream>>>(g, (const float2*)N->act[L], (float4*)out);
  }
  PFMP_CHECK_LAUNCH();
}

void nn_apply(pfmp_nn* N, void* out, const void* in, int prec_io) { nn_apply_skip(N, out, in, prec_io, nullptr); }

// residual loss on even device fields of the network precision:
// r = K y - b, L = |r|^2 / |b|^2, dL/dy = 2 K r / |b|^2 (K Hermitian)
template <typename T>
static double residual_grad_t(pfmp_nn* N, pfmp_op* op, const void* b64) {
  pfmp_ctx* c = N->ctx;
  const Geom& g = c->g;
  using C = typename C2<T>::t;
  const int L = (int)N->W.size();
  const int pr = N->prec;
  void* y = N->ev[0];
  void* r = N->ev[1];
  void* bb = N->ev[2];
  if (pr == PFMP_F64) {
    k_nn_extract<double, PFMP_F64><<<nblocks(g.Vh), kBlock, 0, c->stream>>>(g, (const double2*)N->act[L], (double2*)y);
    PFMP_CUDA(cudaMemcpyAsync(bb, b64, spinor_bytes(g, PFMP_F64), cudaMemcpyDeviceToDevice, c->stream));
  } else {
    k_nn_extract<float, PFMP_F32><<<nblocks(g.Vh), kBlock, 0, c->stream>>>(g, (const float2*)N->act[L], (float4*)y);
    blas_copy(c, bb, PFMP_F32, b64, PFMP_F64);
  }
  PFMP_CHECK_LAUNCH();
  kop(op, pr, r, y, nullptr, nullptr);            // r = K y
  blas_axpy(c, pr, -1.0, 0.0, bb, r);             // r = K y - b
  double sums[2];
  blas_norm2(c, pr, r, c->d_sums);
  blas_norm2(c, pr, bb, c->d_sums + 1);
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  sums[0] = c->h_sums[0];
  sums[1] = c->h_sums[1];
  kop(op, pr, y, r, nullptr, nullptr);            // y = K r
  // gradient 2 K r / |b|^2 (times the caller's scale, applied below) into network layout
  if (pr == PFMP_F64)
    k_nn_embed<double, PFMP_F64><<<nblocks(g.V), kBlock, 0, c->stream>>>(g, (const double2*)y, (double2*)N->gbuf[L % 2]);
  else
    k_nn_embed<float, PFMP_F32><<<nblocks(g.V), kBlock, 0, c->stream>>>(g, (const float4*)y, (float2*)N->gbuf[L % 2]);
  PFMP_CHECK_LAUNCH();
  N->last_norm = sums[1];
  return sums[0] / sums[1];
}

template <typename T>
__global__ void k_scale_c(typename C2<T>::t* v, T a, long n) {
  for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n; i += (long)gridDim.x * blockDim.x) {
    typename C2<T>::t w = v[i];
    w.x *= a;
    w.y *= a;
    v[i] = w;
  }
}

// loss of one pair and accumulation of its weight gradient (scale multiplies the loss);
// kind 0: ||N(b) - x||^2 / ||x||^2, kind 1: ||K N(b) - b||^2 / ||b||^2
template <typename T>
static double loss_grad_t(pfmp_nn* N, pfmp_op* op, int kind, const void* b, const void* x, double scale) {
  pfmp_ctx* c = N->ctx;
  const Geom& g = c->g;
  using C = typename C2<T>::t;
  const int L = (int)N->W.size();
  // targets and input in network layout (both given as FP64 even device fields)
  k_nn_embed<T, PFMP_F64><<<nblocks(g.V), kBlock, 0, c->stream>>>(g, (const double2*)b, (C*)N->act[0]);
  PFMP_CHECK_LAUNCH();
  k_nn_embed<T, PFMP_F64><<<nblocks(g.V), kBlock, 0, c->stream>>>(g, (const double2*)x, (C*)N->target);
  PFMP_CHECK_LAUNCH();
  forward_t<T>(N);
  double loss = 0;
  if (kind == 0) {
    k_nn_loss<T><<<nblocks(g.V), kBlock, 0, c->stream>>>(g, (const C*)N->act[L], (const C*)N->target, c->rb, c->d_sums);
    PFMP_CHECK_LAUNCH();
    k_nn_lossgrad<T><<<nblocks(g.V), kBlock, 0, c->stream>>>(g, (const C*)N->act[L], (const C*)N->target, c->d_sums,
                                                             (T)scale, (C*)N->gbuf[L % 2]);
    PFMP_CHECK_LAUNCH();
  } else {
    loss = residual_grad_t<T>(N, op, b);
    const long n = 12L * g.V;
    k_scale_c<T><<<nblocks(n), kBlock, 0, c->stream>>>((C*)N->gbuf[L % 2], (T)(2.0 * scale / N->last_norm), n);
    PFMP_CHECK_LAUNCH();
  }
  for (int l = L - 1; l >= 0; --l) {
    const int cin = N->ch[l], cout = N->ch[l + 1];
    const C* gout = (const C*)N->gbuf[(l + 1) % 2];
    k_nn_wgrad<T><<<nblocks(g.V, 128), 128, 0, c->stream>>>(g, c->U64, cin, cout, (const C*)N->act[l], gout,
                                                            (T*)N->gW[l]);
    PFMP_CHECK_LAUNCH();
    if (l > 0) {
      const long n = (long)g.V * cin;
      k_nn_layer<T, true><<<nblocks(n, 128), 128, 0, c->stream>>>(g, c->U64, (const C*)N->W[l], cin, cout, gout,
                                                                   (C*)N->gbuf[l % 2]);
      PFMP_CHECK_LAUNCH();
    }
  }
  if (kind == 0) {
    PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
    loss = c->h_sums[0] / c->h_sums[1];
  }
  return loss;
}

void nn_zero_grad(pfmp_nn* N) {
  for (size_t l = 0; l < N->gW.size(); ++l)
    PFMP_CUDA(cudaMemsetAsync(N->gW[l], 0, N->nw[l] * csz(N), N->ctx->stream));
}

double nn_loss_grad(pfmp_nn* N, pfmp_op* op, int kind, const void* b, const void* x, double scale) {
  PFMP_REQUIRE(kind == 0 || kind == 1, PFMP_E_INVALID, "loss kind must be 0 (solution) or 1 (residual)");
  PFMP_REQUIRE(kind == 0 || (op && op->ctx == N->ctx), PFMP_E_INVALID, "the residual loss needs an operator on the network's context");
  return N->prec == PFMP_F64 ? loss_grad_t<double>(N, op, kind, b, x, scale) : loss_grad_t<float>(N, op, kind, b, x, scale);
}

void nn_adam(pfmp_nn* N, double lr) {
  pfmp_ctx* c = N->ctx;
  N->step += 1;
  N->packed = false;
  const double b1 = 0.9, b2 = 0.999, eps = 1e-8;
  const double c1 = 1 - std::pow(b1, (double)N->step), c2 = 1 - std::pow(b2, (double)N->step);
  for (size_t l = 0; l < N->W.size(); ++l) {
    const long n = 2 * N->nw[l];
    if (N->prec == PFMP_F64)
      k_adam<double><<<nblocks(n), kBlock, 0, c->stream>>>((double*)N->W[l], (const double*)N->gW[l],
                                                            (double*)N->m[l], (double*)N->v[l], n, lr, b1, b2, eps, c1, c2);
    else
      k_adam<float><<<nblocks(n), kBlock, 0, c->stream>>>((float*)N->W[l], (const float*)N->gW[l], (float*)N->m[l],
                                                           (float*)N->v[l], n, (float)lr, (float)b1, (float)b2,
                                                           (float)eps, (float)c1, (float)c2);
    PFMP_CHECK_LAUNCH();
  }
}

// minibatch Adam over the pairs: each step averages the loss gradient of `batch` pairs
double nn_train(pfmp_nn* N, pfmp_op* op, int kind, int npairs, const void* const* b, const void* const* x, int steps,
                int batch, double lr) {
  PFMP_REQUIRE(npairs >= 1 && steps >= 1 && batch >= 1, PFMP_E_INVALID, "bad training arguments");
  double last = 0;
  long k = 0;
  for (int s = 0; s < steps; ++s) {
    nn_zero_grad(N);
    double tot = 0;
    for (int j = 0; j < batch; ++j, ++k) {
      const int i = (int)(k % npairs);
      tot += nn_loss_grad(N, op, kind, b[i], x[i], 1.0 / batch);
    }
    nn_adam(N, lr);
    last = tot / batch;
  }
  return last;
}

// ------------------------------------------------------------------ FGCR
struct FgcrWork {
  int restart = 0, grid = 0;
  CGScalars* scal = nullptr;   // device: rr, stop_rr, done, iter of the current cycle
  CGScalars* h_scal = nullptr; // pinned host mirror
  cudaGraphExec_t exec = nullptr;  // one cycle of `glen` iterations, keyed by the network
  long long gkey = -1;
  int glen = 0;
  long long gkernels = 0;
  cudaStream_t cap = nullptr;
  std::vector<float4*> Z, W;
  float4 *r = nullptr, *e = nullptr, *z = nullptr, *w = nullptr;
  float4** dW = nullptr;
  float4** dZ = nullptr;
  double* part = nullptr;
  unsigned* ticket = nullptr;
  double* out = nullptr;
  ~FgcrWork() {
    if (exec) cudaGraphExecDestroy(exec);
    if (cap) cudaStreamDestroy(cap);
    dev_free(scal);
    if (h_scal) cudaFreeHost(h_scal);
    for (auto p : Z) dev_free(p);
    for (auto p : W) dev_free(p);
    dev_free(r);
    dev_free(e);
    dev_free(z);
    dev_free(w);
    dev_free(dW);
    dev_free(dZ);
    dev_free(part);
    dev_free(ticket);
    dev_free(out);
  }
};

int solve_fgcr(pfmp_op* op, pfmp_nn* nn, double tol, int max_iter, int restart, double delta, void* x, const void* b,
               int* iters, int* outer, double* true_res, long* kapply, int* fallback_iters) {
  pfmp_ctx* c = op->ctx;
  const Geom& g = c->g;
  PFMP_REQUIRE(!nn || nn->ctx == c, PFMP_E_INVALID, "the network must live on the operator's context");
  if (restart <= 0) restart = 16;
  PFMP_REQUIRE(restart <= 16, PFMP_E_INVALID, "FGCR restart length must be <= 16");
  if (!(delta > 0 && delta < 1)) delta = 1e-3;
  const size_t b32 = spinor_bytes(g, PFMP_F32), b64 = spinor_bytes(g, PFMP_F64);
  const long n32 = 6L * g.Vh;
  const int fgrid = (int)std::min<long>(nblocks(n32), 152 * 2);
  // workspace kept on the operator between solves (allocation is not per solve)
  FgcrWork* wp = (FgcrWork*)op->fgcr;
  if (!wp || wp->restart < restart) {
    if (wp) op->fgcr_free(wp);
    op->fgcr = nullptr;
    wp = new FgcrWork();
    try {
      for (int k = 0; k < restart; ++k) {
        wp->Z.push_back((float4*)dev_alloc(b32));
        wp->W.push_back((float4*)dev_alloc(b32));
      }
      wp->r = (float4*)dev_alloc(b32);
      wp->e = (float4*)dev_alloc(b32);
      wp->dW = (float4**)dev_alloc(restart * sizeof(float4*));
      wp->dZ = (float4**)dev_alloc(restart * sizeof(float4*));
      PFMP_CUDA(cudaMemcpy(wp->dW, wp->W.data(), restart * sizeof(float4*), cudaMemcpyHostToDevice));
      PFMP_CUDA(cudaMemcpy(wp->dZ, wp->Z.data(), restart * sizeof(float4*), cudaMemcpyHostToDevice));
      wp->part = (double*)dev_alloc((size_t)fgrid * 34 * sizeof(double));
      wp->ticket = (unsigned*)dev_alloc(sizeof(unsigned));
      PFMP_CUDA(cudaMemset(wp->ticket, 0, sizeof(unsigned)));
      wp->out = (double*)dev_alloc(40 * sizeof(double));
      wp->scal = (CGScalars*)dev_alloc(sizeof(CGScalars));
      PFMP_CUDA(cudaMallocHost(&wp->h_scal, sizeof(CGScalars)));
    } catch (...) {
      delete wp;
      throw;
    }
    wp->restart = restart;
    wp->grid = fgrid;
    op->fgcr = wp;
    op->fgcr_free = [](void* p) { delete (FgcrWork*)p; };
  }
  FgcrWork& wk = *wp;
  *iters = *outer = *fallback_iters = 0;
  *kapply = 0;
  blas_norm2(c, PFMP_F64, b, c->d_sums);
  PFMP_CUDA(cudaMemcpyAsync(c->h_sums, c->d_sums, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  PFMP_CUDA(cudaStreamSynchronize(c->stream));
  const double bb = c->h_sums[0];
  blas_zero(c, PFMP_F64, x);
  *true_res = 0;
  if (bb == 0) return PFMP_OK;
  void* r64 = op->cg64[0];
  PFMP_CUDA(cudaMemcpyAsync(r64, b, b64, cudaMemcpyDeviceToDevice, c->stream));
  double res = 1.0, prev = 1.0;
  int stall = 0;
  const bool use_graph = !c->prof.on;
  if (nn && nn->tc) tc_prepare(nn);
  while (*iters < max_iter) {
    // inner FGCR(restart) in FP32 on K e = r, one device-driven cycle: the launches of
    // `len` iterations go out without a host round trip (as one CUDA graph when the
    // cycle has the full length) and the host reads the scalars once at the end
    blas_copy(c, wk.r, PFMP_F32, r64, PFMP_F64);
    blas_zero(c, PFMP_F32, wk.e);
    blas_norm2(c, PFMP_F32, wk.r, &wk.scal->rr);
    k_fgcr_start<<<1, 1, 0, c->stream>>>(wk.scal, delta * delta, 0.25 * tol * tol * bb);
    PFMP_CHECK_LAUNCH();
    const int len = std::min(restart, max_iter - *iters);
    auto launch_cycle = [&](int n_it) {
      for (int k = 0; k < n_it; ++k) {
        float4* z = wk.Z[k];
        float4* w = wk.W[k];
        if (nn) {
          nn_apply_skip(nn, z, wk.r, PFMP_F32, &wk.scal->done, &wk.scal->rr);
        } else {
          k_fgcr_copy<<<fgrid, kBlock, 0, c->stream>>>(z, wk.r, n32, wk.scal);
          PFMP_CHECK_LAUNCH();
        }
        kop(op, PFMP_F32, w, z, nullptr, wk.scal);
        k_fgcr_dots_part<<<dim3(fgrid, k + 1), kBlock, 0, c->stream>>>(wk.dW, k, w, wk.r, n32, wk.part, wk.scal);
        PFMP_CHECK_LAUNCH();
        k_fgcr_dots_final<<<k + 1, kBlock, 0, c->stream>>>(fgrid, wk.part, wk.out, wk.scal);
        PFMP_CHECK_LAUNCH();
        k_fgcr_orth<<<fgrid, kBlock, 0, c->stream>>>(wk.dW, wk.dZ, k, wk.out, w, z, n32, wk.part, wk.ticket,
                                                     wk.out + 36, wk.scal);
        PFMP_CHECK_LAUNCH();
        k_fgcr_step<<<fgrid, kBlock, 0, c->stream>>>(w, z, wk.r, wk.e, wk.out, k, wk.out + 36, n32, wk.scal,
                                                     wk.ticket);
        PFMP_CHECK_LAUNCH();
      }
    };
    const long long key = nn ? nn->id * 2 + (nn->tc ? 1 : 0) : 0;
    const long long kap0 = op->kapply;
    if (use_graph && len == restart) {
      if (!wk.exec || wk.gkey != key || wk.glen != len) {
        if (wk.exec) {
          cudaGraphExecDestroy(wk.exec);
          wk.exec = nullptr;
        }
        if (!wk.cap) PFMP_CUDA(cudaStreamCreateWithFlags(&wk.cap, cudaStreamNonBlocking));
        cudaStream_t keep = c->stream;
        cudaGraph_t graph = nullptr;
        PFMP_CUDA(cudaStreamBeginCapture(wk.cap, cudaStreamCaptureModeThreadLocal));
        c->stream = wk.cap;
        const long long n0 = launch_count();
        try {
          launch_cycle(len);
        } catch (...) {
          c->stream = keep;
          cudaStreamEndCapture(wk.cap, &graph);
          if (graph) cudaGraphDestroy(graph);
          throw;
        }
        c->stream = keep;
        wk.gkernels = launch_count() - n0;
        count_launches(-wk.gkernels);  // captured, not launched
        PFMP_CUDA(cudaStreamEndCapture(wk.cap, &graph));
        cudaError_t e = cudaGraphInstantiate(&wk.exec, graph, 0);
        cudaGraphDestroy(graph);
        PFMP_CUDA(e);
        wk.gkey = key;
        wk.glen = len;
      }
      PFMP_CUDA(cudaGraphLaunch(wk.exec, c->stream));
      count_launches(wk.gkernels);
    } else {
      launch_cycle(len);
    }
    PFMP_CUDA(cudaMemcpyAsync(wk.h_scal, wk.scal, sizeof(CGScalars), cudaMemcpyDeviceToHost, c->stream));
    PFMP_CUDA(cudaStreamSynchronize(c->stream));
    PFMP_REQUIRE(std::isfinite(wk.h_scal->rr), PFMP_E_NAN, "FGCR residual is not finite");
    const int done_it = wk.h_scal->iter;
    op->kapply = kap0 + done_it;  // K applications the device actually did
    *iters += done_it;
    *kapply += done_it;
    // outer correction in FP64 storage, true residual in double-float
    blas_add_lo(c, x, wk.e);
    *outer += 1;
    res = std::sqrt(true_residual_mixed(op, x, b, r64, tol * tol * bb, kapply) / bb);
    PFMP_REQUIRE(std::isfinite(res), PFMP_E_NAN, "FGCR residual is not finite");
    if (res < tol) break;
    stall = res > 0.9 * prev ? stall + 1 : 0;
    prev = res;
    if (stall >= 2) {
      // fallback: the remaining correction by mixed CG
      void* ec = op->cg64[4];
      void* rc = op->cg64[3];  // the solver overwrites cg64[0..2]: hand it a copy of r
      PFMP_CUDA(cudaMemcpyAsync(rc, r64, b64, cudaMemcpyDeviceToDevice, c->stream));
      int it, rel;
      double r2;
      long kap;
      solve(op, PFMP_SOLVER_CG_MIXED, tol / res, max_iter, 1e-4, 8, ec, rc, &it, &rel, &r2, &kap);
      *fallback_iters = it;
      *kapply += kap;
      caxpby(c, 1.0, ec, 1.0, x);
      res = std::sqrt(true_residual_mixed(op, x, b, r64, tol * tol * bb, kapply) / bb);
      break;
    }
  }
  if (nn) nn_check(nn);
  *true_res = res;
  return res < tol ? PFMP_OK : PFMP_E_NOT_CONVERGED;
}

}  // namespace pfmp
