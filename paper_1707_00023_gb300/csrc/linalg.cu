// Bulk vector kernels of the Krylov path: Arnoldi pass B (Gram-Schmidt
// update and norm), the basis combination y = V_m u, the multi-shift update
// of the stationary parts, residual norms and the output-plane response.
// All reductions are deterministic: per-block partials in a fixed order,
// summed by the last block to finish.
#include <atomic>

#include "kx_eft.cuh"
#include "kx_internal.cuh"
#include "kx_reduce.cuh"

namespace kx {

#define warp_sum_l warp_sum

template <typename T> struct Vec;
template <> struct Vec<float> { using t = float4; static constexpr int w = 4; };
template <> struct Vec<double> { using t = double2; static constexpr int w = 2; };

template <typename T>
__device__ __forceinline__ void vfma(typename Vec<T>::t& x, T a, const typename Vec<T>::t& y);
template <>
__device__ __forceinline__ void vfma<float>(float4& x, float a, const float4& y) {
  x.x = fmaf(a, y.x, x.x); x.y = fmaf(a, y.y, x.y); x.z = fmaf(a, y.z, x.z); x.w = fmaf(a, y.w, x.w);
}
template <>
__device__ __forceinline__ void vfma<double>(double2& x, double a, const double2& y) {
  x.x = fma(a, y.x, x.x); x.y = fma(a, y.y, x.y);
}
__device__ __forceinline__ float vdot(const float4& a) { return a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w; }
__device__ __forceinline__ double vdot(const double2& a) { return a.x * a.x + a.y * a.y; }
__device__ __forceinline__ void vadd_f(float4& x, const float4& y) { x.x += y.x; x.y += y.y; x.z += y.z; x.w += y.w; }
__device__ __forceinline__ void vadd_f(double2& x, const double2& y) { x.x += y.x; x.y += y.y; }
template <typename T>
__device__ __forceinline__ void vadd(typename Vec<T>::t& x, const typename Vec<T>::t& y) { vadd_f(x, y); }
template <typename T> __device__ __forceinline__ typename Vec<T>::t vzero();
template <> __device__ __forceinline__ float4 vzero<float>() { return make_float4(0.f, 0.f, 0.f, 0.f); }
template <> __device__ __forceinline__ double2 vzero<double>() { return make_double2(0.0, 0.0); }

// ---------------------------------------------------------------------------
// Arnoldi pass B (step j): w <- w - sum_{i<=j} h_{ij} v_i (classical
// Gram-Schmidt), h_{j+1,j} = ||w||, scale[j+1] = 1/h_{j+1,j}.  The stored
// column stays unnormalised (delayed normalisation); a lucky breakdown
// h_{j+1,j} <= tol * max_i ||A v_i|| stops the process.  In FP32 the update
// is compensated (kx_eft.cuh) and rounded once when the column is stored.
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_pass_b(SlotSet<T> ss, int j, int64_t n, int64_t ld,
                                                    int ldh, int aug, double btol) {
  pdl_enter();
  using V4 = typename Vec<T>::t;
  constexpr int W = Vec<T>::w;
  const Slot<T> s = slot_at(ss, blockIdx.y);
  if (s.st->done || s.st->retired) return;
  __shared__ T coef[MMAX + 1];
  const int ncol = j + 1;
  for (int q = threadIdx.x; q < ncol; q += blockDim.x)
    coef[q] = (T)(s.H[q + (int64_t)j * ldh] * s.scale[q]);
  __syncthreads();
  T* __restrict__ w = s.V + (int64_t)(j + 1) * ld;
  double nrm = 0.0;
  const int64_t nv = n / W;
  const V4* __restrict__ Vv = reinterpret_cast<const V4*>(s.V);
  const int64_t ldv = ld / W;
  if constexpr (sizeof(T) == 4) {
    const float4* __restrict__ Vf = reinterpret_cast<const float4*>(s.V);
    float* __restrict__ wf = reinterpret_cast<float*>(w);
    for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
         q += (int64_t)gridDim.x * blockDim.x) {
      float4 x = reinterpret_cast<const float4*>(wf)[q];
      float4 lo = make_float4(0.f, 0.f, 0.f, 0.f);
      int col = 0;
      // eight independent column loads in flight per thread
      for (; col + 8 <= ncol; col += 8) {
        float4 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = Vf[(int64_t)(col + t) * ldv + q];
#pragma unroll
        for (int t = 0; t < 8; ++t) sub_fma4(x, lo, -(float)coef[col + t], v[t]);
      }
      for (; col < ncol; ++col) sub_fma4(x, lo, -(float)coef[col], Vf[(int64_t)col * ldv + q]);
      x = make_float4(x.x + lo.x, x.y + lo.y, x.z + lo.z, x.w + lo.w);
      reinterpret_cast<float4*>(wf)[q] = x;
      nrm += (double)vdot(x);
    }
    for (int64_t e = nv * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
         e += (int64_t)gridDim.x * blockDim.x) {
      float x = wf[e], lo = 0.f;
      for (int col = 0; col < ncol; ++col) sub_fma(x, lo, -(float)coef[col], (float)s.V[(int64_t)col * ld + e]);
      x += lo;
      wf[e] = x;
      nrm += (double)x * (double)x;
    }
    block_partial(nrm, s.part, s.ps, FINB_COL);
    return;
  }
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x) {
    V4 x = reinterpret_cast<const V4*>(w)[q];
    int col = 0;
    // eight independent column loads in flight per thread
    for (; col + 8 <= ncol; col += 8) {
      V4 v[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) v[t] = Vv[(int64_t)(col + t) * ldv + q];
#pragma unroll
      for (int t = 0; t < 8; ++t) vfma<T>(x, -coef[col + t], v[t]);
    }
    for (; col + 2 <= ncol; col += 2) {
      const V4 v0 = Vv[(int64_t)col * ldv + q];
      const V4 v1 = Vv[(int64_t)(col + 1) * ldv + q];
      vfma<T>(x, -coef[col], v0);
      vfma<T>(x, -coef[col + 1], v1);
    }
    for (; col < ncol; ++col) vfma<T>(x, -coef[col], Vv[(int64_t)col * ldv + q]);
    reinterpret_cast<V4*>(w)[q] = x;
    nrm += (double)vdot(x);
  }
  for (int64_t e = nv * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    T x = w[e];
    for (int col = 0; col < ncol; ++col) x -= coef[col] * s.V[(int64_t)col * ld + e];
    w[e] = x;
    nrm += (double)x * (double)x;
  }
  block_partial(nrm, s.part, s.ps, FINB_COL);
}

// Finalisation of pass B (one block): h_{j+1,j} = ||w||, scale, breakdown.
// The augmented entries of w (plain method only) get the same Gram-Schmidt
// update, their column sums spread over the block and reduced in a fixed
// order; slots without augmented entries skip it (the entries are zero).
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_fin_b(SlotSet<T> ss, int j, int ldh, int nb, int aug, double btol) {
  pdl_enter();
  const Slot<T> s = slot_at(ss, blockIdx.y);
  if (s.st->done || s.st->retired) return;
  const int ncol = j + 1;
  const bool augm = aug && s.st->aug;
  double x = 0.0, pa = 0.0, pb = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) x += __ldcg(s.part + (int64_t)FINB_COL * s.ps + b);
  if (augm) {
    for (int col = threadIdx.x; col < ncol; col += blockDim.x) {
      const double cc = s.H[col + (int64_t)j * ldh] * s.scale[col];
      pa += cc * s.aug[2 * col];
      pb += cc * s.aug[2 * col + 1];
    }
  }
  __shared__ double red[3][NWARPS];
  x = warp_sum(x);
  pa = warp_sum(pa);
  pb = warp_sum(pb);
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = x;
    red[1][threadIdx.x >> 5] = pa;
    red[2][threadIdx.x >> 5] = pb;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0, sa = 0.0, sb = 0.0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) {
      tot += red[0][w];
      sa += red[1][w];
      sb += red[2][w];
    }
    if (augm) {
      const double a = s.aug[2 * (j + 1)] - sa, b = s.aug[2 * (j + 1) + 1] - sb;
      s.aug[2 * (j + 1)] = a;
      s.aug[2 * (j + 1) + 1] = b;
      tot += a * a + b * b;
    }
    const double h = sqrt(tot);
    s.H[(j + 1) + (int64_t)j * ldh] = h;
    s.st->m_done = j + 1;
    if (abort_requested(s.st)) s.st->done = 1;
    if (!isfinite(h)) {
      s.st->status = KX_ENONFINITE;
      s.st->done = 1;
    } else if (h <= btol * s.st->wmax) {
      s.st->done = 1;            // invariant subspace: the projection is exact
      s.scale[j + 1] = 0.0;
    } else {
      s.scale[j + 1] = 1.0 / h;
    }
  }
}

// Grid of pass B: a persistent grid (shrunk for resident side CTAs); the
// next pass A needs it to finalise pass B itself.
int pass_b_grid(kx_ctx* c) {
  static std::atomic<int> grid[2];
  const int fp64 = c->d.precision == KX_FP64;
  if (!grid[fp64])
    grid[fp64] = persistent_grid(c, fp64 ? (const void*)k_pass_b<double> : (const void*)k_pass_b<float>,
                                 1 << 30, 0);
  const int64_t rounds = (c->n / (fp64 ? 2 : 4) + NTHREADS - 1) / NTHREADS;
  return reserve_grid(c, (int)std::max<int64_t>(1, std::min<int64_t>(std::min<int64_t>(rounds, grid[fp64].load()), c->ps)),
                      grid[fp64].load());
}

// Algorithmic bytes of pass B at step j: read w and V_0..V_j (j+2 vectors),
// write the updated column (1).
kx_status launch_pass_b(kx_ctx* c, int slot, int ns, int j, int finalize) {
  const int ldh = c->m + 1;
  const int aug = 1;  // augmented entries are zero when unused
  time_begin(c);
  struct End { kx_ctx* c; int j, ns; ~End() { time_end(c, KX_K_PASS_B, (j + 3.0) * c->n * c->esize * ns); } } end{c, j, ns};
  const int fp64 = c->d.precision == KX_FP64;
  const int nb = pass_b_grid(c);
  if (fp64) {
    launch_k(c, k_pass_b<double>, dim3(nb, ns), NTHREADS, 0, c->stream, make_slotset<double>(c, slot), j, c->n,
             c->ld, ldh, aug, 1e-12);
    KX_CHECK_LAUNCH(c);
    if (finalize)
      launch_k(c, k_fin_b<double>, dim3(1, ns), NTHREADS, 0, c->stream, make_slotset<double>(c, slot), j, ldh, nb,
               aug, 1e-12);
  } else {
    launch_k(c, k_pass_b<float>, dim3(nb, ns), NTHREADS, 0, c->stream, make_slotset<float>(c, slot), j, c->n, c->ld,
             ldh, aug, 1e-6);
    KX_CHECK_LAUNCH(c);
    if (finalize)
      launch_k(c, k_fin_b<float>, dim3(1, ns), NTHREADS, 0, c->stream, make_slotset<float>(c, slot), j, ldh, nb,
               aug, 1e-6);
  }
  if (finalize) KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// Start of a restart: beta = ||[V_0; aug_0]||, scale[0] = 1/beta, reset the
// Arnoldi state.  mode 0: V_0 as it is.  mode 1 (combine): V_0 <- sum_{i<m}
// u_i scale_i V_i first (the Krylov update y = V_m u, eq. (corr2) /
// (upd1)); in the augmented case the phase entries are then reset to their
// exact values eta (sin W t, cos W t).
// Error-free compensated combination (FP32 path): every coefficient is a
// float pair hi + lo of its FP64 value, each product's rounding error comes
// from an FMA and each sum's from Knuth's TwoSum, so the result is the
// correctly summed combination up to the final rounding.
__device__ __forceinline__ void acc_comp(float& s, float& c, float hi, float lo, float v) {
  const float p = hi * v;
  const float e = fmaf(hi, v, -p) + lo * v;
  const float t = s + p;
  const float z = t - s;
  c += ((s - (t - z)) + (p - z)) + e;
  s = t;
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_restart(SlotSet<T> ss, int64_t n, int64_t ld, int mode) {
  pdl_enter();
  using V4 = typename Vec<T>::t;
  constexpr int W = Vec<T>::w;
  const Slot<T> s = slot_at(ss, blockIdx.y);
  // retired, or (combination) a failed sub-step: nothing to combine
  if (s.st->retired || (mode == 1 && s.st->status)) return;
  __shared__ T coef[MMAX];
  __shared__ float coef_lo[MMAX];
  int m = 0;
  if (mode == 1) {
    m = s.st->m_done;
    for (int q = threadIdx.x; q < m; q += blockDim.x) {
      const double cf = s.u[q] * s.scale[q];
      coef[q] = (T)cf;
      coef_lo[q] = (float)(cf - (double)(T)cf);
    }
  }
  __syncthreads();
  T* __restrict__ y = s.V;
  double nrm = 0.0;
  const int64_t nv = n / W;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < nv;
       q += (int64_t)gridDim.x * blockDim.x) {
    V4 x;
    if (mode == 1 && sizeof(T) == 4) {
      const float4* __restrict__ Vf = reinterpret_cast<const float4*>(s.V);
      const int64_t ldv = ld / 4;
      float sx = 0.f, sy = 0.f, sz = 0.f, sw = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, cw = 0.f;
      int col = 0;
      for (; col + 4 <= m; col += 4) {
        float4 v[4];
#pragma unroll
        for (int t = 0; t < 4; ++t) v[t] = Vf[(int64_t)(col + t) * ldv + q];
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          const float hi = (float)coef[col + t], lo = coef_lo[col + t];
          acc_comp(sx, cx, hi, lo, v[t].x);
          acc_comp(sy, cy, hi, lo, v[t].y);
          acc_comp(sz, cz, hi, lo, v[t].z);
          acc_comp(sw, cw, hi, lo, v[t].w);
        }
      }
      for (; col < m; ++col) {
        const float4 v = Vf[(int64_t)col * ldv + q];
        const float hi = (float)coef[col], lo = coef_lo[col];
        acc_comp(sx, cx, hi, lo, v.x);
        acc_comp(sy, cy, hi, lo, v.y);
        acc_comp(sz, cz, hi, lo, v.z);
        acc_comp(sw, cw, hi, lo, v.w);
      }
      const float4 r = make_float4(sx + cx, sy + cy, sz + cz, sw + cw);
      x = *reinterpret_cast<const V4*>(&r);
      reinterpret_cast<V4*>(y)[q] = x;
    } else if (mode == 1) {
      const V4* __restrict__ Vv = reinterpret_cast<const V4*>(s.V);
      const int64_t ldv = ld / W;
      V4 x1 = vzero<T>();
      x = vzero<T>();
      int col = 0;
      for (; col + 8 <= m; col += 8) {
        V4 v[8];
#pragma unroll
        for (int t = 0; t < 8; ++t) v[t] = Vv[(int64_t)(col + t) * ldv + q];
#pragma unroll
        for (int t = 0; t < 8; t += 2) {
          vfma<T>(x, coef[col + t], v[t]);
          vfma<T>(x1, coef[col + t + 1], v[t + 1]);
        }
      }
      for (; col < m; ++col) vfma<T>(x, coef[col], Vv[(int64_t)col * ldv + q]);
      vadd<T>(x, x1);
      reinterpret_cast<V4*>(y)[q] = x;
    } else {
      x = reinterpret_cast<const V4*>(y)[q];
    }
    nrm += (double)vdot(x);
  }
  for (int64_t e = nv * W + blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    T x;
    if (mode == 1) {
      x = T(0);
      for (int col = 0; col < m; ++col) x += coef[col] * s.V[(int64_t)col * ld + e];
      y[e] = x;
    } else {
      x = y[e];
    }
    nrm += (double)x * (double)x;
  }
  block_partial(nrm, s.part, s.ps, 0);
  if (!last_block(s.counter)) return;
  double xs = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += blockDim.x) xs += __ldcg(s.part + b);
  __shared__ double red2[NWARPS];
  xs = warp_sum(xs);
  if ((threadIdx.x & 31) == 0) red2[threadIdx.x >> 5] = xs;
  __syncthreads();
  if (threadIdx.x == 0) {
    *s.counter = 0u;
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) tot += red2[w];
    if (s.st->aug) {
      const double t = s.st->t_now;
      s.aug[0] = s.st->eta * sin(s.st->omega * t);
      s.aug[1] = s.st->eta * cos(s.st->omega * t);
      tot += s.aug[0] * s.aug[0] + s.aug[1] * s.aug[1];
    } else {
      s.aug[0] = 0.0;
      s.aug[1] = 0.0;
    }
    const double b = sqrt(tot);
    s.st->beta = b;
    s.scale[0] = b > 0.0 ? 1.0 / b : 0.0;
    s.st->done = (b > 0.0 && isfinite(b)) ? 0 : 1;
    if (!isfinite(b)) s.st->status = KX_ENONFINITE;
    s.st->m_done = 0;
    s.st->wmax = 0.0;
    if (mode == 1 && s.st->finished) s.st->retired = 1;
  }
}

template <typename T>
static kx_status restart_t(kx_ctx* c, int slot, int ns, int mode) {
  // bytes: combine reads the m basis columns and writes one; norm reads one
  time_begin(c);
  launch_k(c, k_restart<T>, dim3(c->nblk, ns), NTHREADS, 0, c->stream, make_slotset<T>(c, slot), c->n, c->ld, mode);
  time_end(c, KX_K_RESTART, (mode == 1 ? c->m + 1.0 : 1.0) * c->n * c->esize * ns);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

kx_status launch_norm_init(kx_ctx* c, int slot, int ns) {
  return c->d.precision == KX_FP64 ? restart_t<double>(c, slot, ns, 0) : restart_t<float>(c, slot, ns, 0);
}

kx_status launch_combine(kx_ctx* c, int slot, int ns) {
  return c->d.precision == KX_FP64 ? restart_t<double>(c, slot, ns, 1) : restart_t<float>(c, slot, ns, 1);
}

// ---------------------------------------------------------------------------
// y += a x over n scalars (the periodic-source methods combine whole fields).
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_axpy(int64_t n, double a, const T* __restrict__ x, T* __restrict__ y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = (T)((double)y[e] + a * (double)x[e]);
}

kx_status launch_axpy(kx_ctx* c, double a, const void* x, void* y) {
  time_begin(c);
  if (c->d.precision == KX_FP64)
    k_axpy<double><<<c->nblk, NTHREADS, 0, c->stream>>>(c->n, a, (const double*)x, (double*)y);
  else
    k_axpy<float><<<c->nblk, NTHREADS, 0, c->stream>>>(c->n, a, (const float*)x, (float*)y);
  time_end(c, KX_K_RESTART, 3.0 * c->n * c->esize);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// Export the orthonormal basis: dV[:, i] = scale_i V_i (i <= m_done, and the
// column past a lucky breakdown is zero).
template <typename T>
__global__ void k_export(Slot<T> s, T* __restrict__ dV, int64_t n, int64_t ld, int m) {
  const int md = s.st->m_done;
  const int brk = s.st->done;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    for (int col = 0; col <= m; ++col) {
      T x = T(0);
      if (col < md || (col == md && !brk)) x = (T)(s.scale[col] * (double)s.V[(int64_t)col * ld + e]);
      dV[(int64_t)col * n + e] = x;
    }
  }
}

kx_status launch_basis_export(kx_ctx* c, int slot, void* dV, int m) {
  if (c->d.precision == KX_FP64)
    k_export<double><<<c->nblk, NTHREADS, 0, c->stream>>>(make_slot<double>(c, slot), (double*)dV, c->n, c->ld, m);
  else
    k_export<float><<<c->nblk, NTHREADS, 0, c->stream>>>(make_slot<float>(c, slot), (float*)dV, c->n, c->ld, m);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// Shifted FOM update of every stationary part on one basis:
//   z_j += V_m c_j,  c_j = rho_j (H_m + i W_j I)^{-1} e_1  (complex),
// the coefficients (already multiplied by the column scales) in coef:
//   coef[(2 f) * MMAX + i] real part, coef[(2 f + 1) * MMAX + i] imaginary.
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_zupdate(const T* __restrict__ V, int64_t ld, int m,
                                                     int64_t n, int nfreq, const T* __restrict__ coef,
                                                     T* __restrict__ zre, T* __restrict__ zim) {
  extern __shared__ unsigned char smem_raw[];
  T* cs = reinterpret_cast<T*>(smem_raw);
  for (int q = threadIdx.x; q < 2 * nfreq * MMAX; q += blockDim.x) cs[q] = coef[q];
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    T v[MMAX];
#pragma unroll
    for (int i = 0; i < MMAX; ++i) v[i] = (i < m) ? V[(int64_t)i * ld + e] : T(0);
    for (int f = 0; f < nfreq; ++f) {
      const T* cr = cs + (2 * f) * MMAX;
      const T* ci = cs + (2 * f + 1) * MMAX;
      T ar = T(0), ai = T(0);
#pragma unroll
      for (int i = 0; i < MMAX; ++i) {
        ar += cr[i] * v[i];
        ai += ci[i] * v[i];
      }
      zre[(int64_t)f * n + e] += ar;
      zim[(int64_t)f * n + e] += ai;
    }
  }
}

kx_status launch_zupdate(kx_ctx* c, int slot, int nfreq, void* zre, void* zim, int m) {
  const size_t sm = (size_t)2 * nfreq * MMAX * c->esize;
  static SmemOptIn attr_d{}, attr_f{};
  kx_status so = smem_opt_in(c, attr_d, (const void*)k_zupdate<double>, 2 * MAXF * MMAX * sizeof(double));
  if (so == KX_OK) so = smem_opt_in(c, attr_f, (const void*)k_zupdate<float>, 2 * MAXF * MMAX * sizeof(float));
  if (so != KX_OK) return so;
  // bytes: read m basis columns, read and write 2 nfreq stationary vectors
  time_begin(c);
  struct End { kx_ctx* c; int m, nf; ~End() { time_end(c, KX_K_ZUPDATE, (m + 4.0 * nf) * c->n * c->esize); } } end{c, m, nfreq};
  if (c->d.precision == KX_FP64) {
    Slot<double> s = make_slot<double>(c, slot);
    k_zupdate<double><<<c->nblk, NTHREADS, sm, c->stream>>>(s.V, c->ld, m, c->n, nfreq, c->d_coefd,
                                                            (double*)zre, (double*)zim);
  } else {
    Slot<float> s = make_slot<float>(c, slot);
    k_zupdate<float><<<c->nblk, NTHREADS, sm, c->stream>>>(s.V, c->ld, m, c->n, nfreq, c->d_coef,
                                                           (float*)zre, (float*)zim);
  }
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// ||g - (A + i W) z||^2 / ||g||^2 with Az_re, Az_im already applied:
//   r_re = g - A z_re + W z_im,   r_im = -(A z_im + W z_re).
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_resid(const T* __restrict__ g, const T* __restrict__ Azr,
                                                   const T* __restrict__ Azi, const T* __restrict__ zr,
                                                   const T* __restrict__ zi, double W, int64_t n,
                                                   double* part, int ps, unsigned* counter, double* out) {
  double rr = 0.0, gg = 0.0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    const double a = (double)g[e] - (double)Azr[e] + W * (double)zi[e];
    const double b = -((double)Azi[e] + W * (double)zr[e]);
    rr += a * a + b * b;
    gg += (double)g[e] * (double)g[e];
  }
  block_partial(rr, part, ps, 0);
  block_partial(gg, part, ps, 1);
  if (!last_block(counter)) return;
  __shared__ double tt[2];
  grid_columns(part, ps, 2, tt);
  if (threadIdx.x == 0) {
    *counter = 0u;
    const double R = tt[0], G = tt[1];
    *out = G > 0.0 ? sqrt(R / G) : 0.0;
  }
}

kx_status launch_true_residual(kx_ctx* c, const void* g, int nfreq, const double* h_om, void* zre,
                               void* zim, double* out_host) {
  for (int f = 0; f < nfreq; ++f) {
    const char* zr = (const char*)zre + (int64_t)f * c->n * c->esize;
    const char* zi = (const char*)zim + (int64_t)f * c->n * c->esize;
    kx_status st = launch_apply(c, zr, c->d_tmp, 0);
    if (st) return st;
    st = launch_apply(c, zi, c->d_tmp2, 0);
    if (st) return st;
    double* part = c->d_part;  // slot 0 partials (not in use during this call)
    if (c->d.precision == KX_FP64)
      k_resid<double><<<c->nblk, NTHREADS, 0, c->stream>>>(
          (const double*)g, (const double*)c->d_tmp, (const double*)c->d_tmp2, (const double*)zr,
          (const double*)zi, h_om[f], c->n, part, c->ps, c->d_counter, c->d_small + f);
    else
      k_resid<float><<<c->nblk, NTHREADS, 0, c->stream>>>(
          (const float*)g, (const float*)c->d_tmp, (const float*)c->d_tmp2, (const float*)zr,
          (const float*)zi, h_om[f], c->n, part, c->ps, c->d_counter, c->d_small + f);
    KX_CHECK_LAUNCH(c);
  }
  cudaError_t e = cudaMemcpyAsync(c->h_small, c->d_small, sizeof(double) * nfreq,
                                  cudaMemcpyDeviceToHost, c->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) {
    snprintf(c->err, sizeof(c->err), "residual read-back failed: %s", cudaGetErrorString(e));
    return KX_ECUDA;
  }
  for (int f = 0; f < nfreq; ++f) out_host[f] = c->h_small[f];
  return KX_OK;
}

// ---------------------------------------------------------------------------
// Response of one frequency (eq. (split1), final sign '-'):
//   split: y(T) = sin(W T) Re z + cos(W T) Im z - yhat(T) = Im(e^{iWT} z) - yhat
//   plain: y(T) = yt (already the full solution)
// Output plane values (E components) and the summed |E|^2; optionally the
// full field.
template <typename T>
__global__ void k_plane(Geo g, int split, double sW, double cW, const T* __restrict__ zr,
                        const T* __restrict__ zi, const T* __restrict__ yt, int axis, int idx,
                        T* __restrict__ E_plane, double* intensity) {
  const int nE = g.ne;
  int na, nb;
  plane_dims(g, axis, &na, &nb);
  const int64_t np = (int64_t)na * nb;
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < nE * np; t += blockDim.x) {
    const int64_t e = plane_node(g, axis, idx, t);
    double val = (double)yt[e];
    if (split) val = sW * (double)zr[e] + cW * (double)zi[e] - val;
    if (E_plane) E_plane[t] = (T)val;
    acc += val * val;
  }
  __shared__ double red[32];
  acc = warp_sum_l(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    *intensity = s;
  }
}

template <typename T>
__global__ void k_full(int64_t n, int split, double sW, double cW, const T* __restrict__ zr,
                       const T* __restrict__ zi, const T* __restrict__ yt, T* __restrict__ Y) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n;
       e += (int64_t)gridDim.x * blockDim.x) {
    double val = (double)yt[e];
    if (split) val = sW * (double)zr[e] + cW * (double)zi[e] - val;
    Y[e] = (T)val;
  }
}

kx_status launch_response(kx_ctx* c, int f, const double* h_om, double T, int split,
                          const void* zre, const void* zim, const void* yt, int plane_axis,
                          int plane_idx, void* E_plane, double* d_intensity, void* Yout) {
  const double W = h_om[f];
  const double sW = sin(W * T), cW = cos(W * T);
  if (c->d.precision == KX_FP64) {
    k_plane<double><<<1, 1024, 0, c->stream>>>(c->geo, split, sW, cW, (const double*)zre,
                                                (const double*)zim, (const double*)yt, plane_axis,
                                                plane_idx, (double*)E_plane, d_intensity);
    KX_CHECK_LAUNCH(c);
    if (Yout) {
      k_full<double><<<c->nblk, NTHREADS, 0, c->stream>>>(c->n, split, sW, cW, (const double*)zre,
                                                          (const double*)zim, (const double*)yt,
                                                          (double*)Yout);
      KX_CHECK_LAUNCH(c);
    }
  } else {
    k_plane<float><<<1, 1024, 0, c->stream>>>(c->geo, split, sW, cW, (const float*)zre,
                                               (const float*)zim, (const float*)yt, plane_axis,
                                               plane_idx, (float*)E_plane, d_intensity);
    KX_CHECK_LAUNCH(c);
    if (Yout) {
      k_full<float><<<c->nblk, NTHREADS, 0, c->stream>>>(c->n, split, sW, cW, (const float*)zre,
                                                         (const float*)zim, (const float*)yt,
                                                         (float*)Yout);
      KX_CHECK_LAUNCH(c);
    }
  }
  return KX_OK;
}

}  // namespace kx
