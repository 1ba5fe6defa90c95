// Residual-based restarting in Krylov dimension for many frequencies at
// once (Sect. 3.4, eq. (rst), Corollary 2, Fig. alg:rst; regular Krylov
// variant).  The Krylov basis of every restart comes from the Arnoldi
// passes (stencil.cu, linalg.cu) and serves all frequencies; this file holds
// the per-frequency projected work and the accumulation of the responses.
//
// Restart k, basis V_m, Hessenberg H_m, h = h_{m+1,m}:
//   u_j' = -H_m u_j + alpha_j(t) e_1,  u_j(0) = 0       (eq. (corr2))
//   y_j(T) += V_m u_j(T)                                (eq. (upd1))
//   alpha_j <- alphahat_j = -h e_m^T u_j(t)              (eqs. (resid), (rst))
// alpha_j is held on a uniform grid t_i = i d (i = 0..Nt, d = T / Nt) as
// the quintic Hermite interpolant of its value and first two derivatives
// at the grid points (Fig. alg:rst step 2(b) stores the samples), i.e. as
// six coefficients b_0..b_5 per interval, p(theta) = sum_j b_j theta^j,
// theta = (t - t_i) / d.  For that source the projected problem has the
// exact interval map
//   u(t_{i+1}) = E u(t_i) + sum_j b_j W_j,
//   E = exp(-d H_m),  W_j = d j! phi_{j+1}(-d H_m) e_1,
// and the derivatives of alphahat follow from the projected equation:
//   alphahat'  = -h e_m^T (-H_m u + alpha e_1),
//   alphahat'' = -h e_m^T (H_m^2 u - alpha H_m e_1 + alpha' e_1).
//
//   k_rst_source   restart 1's source ||g|| sin(W t) as interval coefficients.
//   k_rst_setup    one CTA: E and the W_j from one exponential of the
//                  (m+6)-square matrix [[-d H_m, e_1 e_1^T], [0, J]] (J the
//                  6x6 shift; its top right block holds phi_1..phi_6 (-d H_m) e_1).
//   k_rst_cascade  one CTA per frequency: the Nt interval maps, E held in
//                  registers; a fifth warp samples alphahat and its first two
//                  derivatives at every grid point.
//   k_rst_coef     the next restart's interval coefficients from those
//                  samples (all intervals in parallel).
//   k_rst_plane    y_j += V_m u_j(T) on the output plane, FP64 accumulators.
//   k_rst_full     the same on the full field (optional).
#include <atomic>
#include <cmath>

#include "kx_internal.cuh"
#include "kx_dense.cuh"
#include "kx_reduce.cuh"

namespace kx {

// Coefficients of p(theta) = sum_j b_j theta^j on an interval of length d
// with p, dp/dt, d2p/dt2 given at both ends (quintic Hermite interpolation).
__device__ __forceinline__ void hermite5(double a0, double da0, double dda0, double a1, double da1,
                                         double dda1, double d, double* b) {
  b[0] = a0;
  b[1] = d * da0;
  b[2] = 0.5 * d * d * dda0;
  const double R0 = a1 - (b[0] + b[1] + b[2]);
  const double R1 = d * da1 - (b[1] + 2.0 * b[2]);
  const double R2 = d * d * dda1 - 2.0 * b[2];
  b[3] = 10.0 * R0 - 4.0 * R1 + 0.5 * R2;
  b[4] = -15.0 * R0 + 7.0 * R1 - R2;
  b[5] = 6.0 * R0 - 3.0 * R1 + 0.5 * R2;
}

// ---------------------------------------------------------------------------
__global__ void k_rst_source(const double* __restrict__ om, double beta, int Nt, double d,
                             double* __restrict__ b) {
  const int f = blockIdx.y;
  const double W = om[f];
  double* bf = b + (int64_t)f * Nt * RST_P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Nt; i += gridDim.x * blockDim.x) {
    double s0, c0, s1, c1;
    sincos(W * (i * d), &s0, &c0);
    sincos(W * ((i + 1) * d), &s1, &c1);
    double bb[RST_P];
    hermite5(beta * s0, beta * W * c0, -beta * W * W * s0, beta * s1, beta * W * c1, -beta * W * W * s1, d, bb);
#pragma unroll
    for (int j = 0; j < RST_P; ++j) bf[(int64_t)i * RST_P + j] = bb[j];
  }
}

kx_status launch_rst_source(kx_ctx* c, cudaStream_t st, int nfreq, double beta, int Nt, double d, double* b) {
  const int gx = std::min((Nt + 255) / 256, 64);
  k_rst_source<<<dim3(gx, nfreq), 256, 0, st>>>(c->d_omegas, beta, Nt, d, b);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_rst_setup(const double* __restrict__ H, int ldh,
                                                   const SlotState* st, double d, double* mats,
                                                   double* gbuf, int* status) {
  __shared__ double red[32];
  __shared__ double lv[MMAX + RST_P + 2];
  __shared__ int piv;
  const int md = st->m_done;
  if (md < 1 || st->status) {
    // the Arnoldi process's own status (a non-finite value, a bounded wait
    // that ran out), else no step completed
    if (threadIdx.x == 0) *status = st->status ? st->status : KX_ENONFINITE;
    return;
  }
  // the six (m+6)-square work matrices live in global memory (L1/L2
  // resident): a large shared-memory request would keep this CTA off every
  // SM that runs the Arnoldi passes, which this kernel overlaps
  const int n = md + RST_P;
  double* buf[6];
  for (int q = 0; q < 6; ++q) buf[q] = gbuf + (size_t)q * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx - r * n;
    double v = 0.0;
    if (r < md && c < md) v = (r <= c + 1) ? -d * H[r + (int64_t)c * ldh] : 0.0;
    else if (r == 0 && c == md) v = 1.0;
    else if (r >= md && c == r + 1) v = 1.0;
    buf[0][idx] = v;
  }
  __syncthreads();
  double* X = cta_expm(buf, n, red, lv, &piv);
  if (!X) {
    if (threadIdx.x == 0) *status = KX_ENONFINITE;
    return;
  }
  for (int idx = threadIdx.x; idx < MMAX * MMAX; idx += blockDim.x) {
    const int r = idx / MMAX, c = idx - r * MMAX;
    mats[idx] = (r < md && c < md) ? X[r * n + c] : 0.0;
  }
  for (int idx = threadIdx.x; idx < RST_P * MMAX; idx += blockDim.x) {
    const int j = idx / MMAX, r = idx - j * MMAX;
    double fact = 1.0;
    for (int q = 2; q <= j; ++q) fact *= q;
    mats[RST_OFF_W + idx] = (r < md) ? d * fact * X[r * n + md + j] : 0.0;
  }
  // last rows of H_m and H_m^2 (row m-1 of H_m is nonzero in columns m-2, m-1)
  const int lr = md - 1;
  for (int c = threadIdx.x; c < MMAX; c += blockDim.x) {
    double r1 = 0.0, r2 = 0.0;
    if (c < md) {
      if (lr <= c + 1) r1 = H[lr + (int64_t)c * ldh];
      for (int k = max(0, lr - 1); k < md; ++k)
        if (k <= c + 1) r2 += H[lr + (int64_t)k * ldh] * H[k + (int64_t)c * ldh];
    }
    mats[RST_OFF_R1 + c] = r1;
    mats[RST_OFF_R2 + c] = r2;
  }
  if (threadIdx.x == 0) {
    mats[RST_OFF_SC + 0] = st->done ? 0.0 : H[md + (int64_t)(md - 1) * ldh];
    mats[RST_OFF_SC + 1] = (lr <= 1) ? H[lr] : 0.0;
    mats[RST_OFF_SC + 2] = (double)md;
  }
}

kx_status launch_rst_setup(kx_ctx* c, cudaStream_t st, int slot, double d) {
  Slot<float> s = make_slot<float>(c, slot);
  int* status = reinterpret_cast<int*>(c->d_small + 64);
  time_begin(c);
  k_rst_setup<<<1, 256, 0, st>>>(s.H, c->m + 1, s.st, d, c->d_rst_mats,
                                                            c->d_expm_ws, status);
  time_end(c, KX_K_PROJ, 0.0);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// One CTA per frequency.  Threads 0..127 apply the interval map, two per
// row r = tid / 2, columns q + 2k (q = tid % 2) with E's entries in
// registers; each adds half of the source responses b_j W_j[r] before the
// pair's sum.  Threads 128..159 (the sampling warp) read u_i meanwhile and
// write alphahat, d alphahat / dt and d2 alphahat / dt2 at t_i (lanes 0, 1,
// 2, each five FMAs: the last rows of H_m and H_m^2 touch only u's last
// three entries).  u is double-buffered in shared memory, one barrier per
// interval.  On this GPU a double-precision warp instruction costs the same
// issue time whatever its active lanes, so the interval's FP64 instruction
// count per warp is what the layout minimises.
constexpr int RST_MV = 2 * MMAX;
constexpr int RST_THREADS = RST_MV + 32;

__global__ void __launch_bounds__(RST_THREADS) k_rst_cascade(const double* __restrict__ mats,
                                                            const double* __restrict__ b,
                                                            double* __restrict__ smp, int Nt, double d,
                                                            double tol_abs, int* fstate, double* resid,
                                                            double* u_out) {
  const int f = blockIdx.x;
  const int tid = threadIdx.x;
  __shared__ int s_state;
  __shared__ double u[2][MMAX];
  if (tid == 0) s_state = fstate[f];
  for (int i = tid; i < 2 * MMAX; i += blockDim.x) (&u[0][0])[i] = 0.0;
  __syncthreads();
  if (s_state != 0) {
    if (tid == 0 && s_state == 1) fstate[f] = 2;
    return;
  }
  const int md = (int)mats[RST_OFF_SC + 2];
  const double h = mats[RST_OFF_SC + 0];
  const double hm0 = mats[RST_OFF_SC + 1];
  const double* bf = b + (int64_t)f * Nt * RST_P;
  double* sf = smp + (int64_t)f * (Nt + 1) * 3;
  const bool mv = tid < RST_MV;
  const int r = tid >> 1, q = tid & 1, lane = tid & 31;
  const bool samp = !mv && lane < 3;
  double Er[32], Wr[3];
  if (mv) {
#pragma unroll
    for (int k = 0; k < 32; ++k) {
      const int c = q + 2 * k;
      Er[k] = (r < md && c < md) ? mats[r * MMAX + c] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < 3; ++t) Wr[t] = r < md ? mats[RST_OFF_W + (q + 2 * t) * MMAX + r] : 0.0;
  }
  // sampler lane l: value = c0 u[i0] + c1 u[i1] + c2 u[i2] + c3 alpha + c4 (d alpha'),
  //   l = 0: alphahat = -h u_m
  //   l = 1: alphahat' = h (H_m u)_m - h [m = 1] alpha
  //   l = 2: alphahat'' = -h (H_m^2 u)_m + h (H_m)_{m,1} alpha - h [m = 1] alpha'
  int i0 = 0, i1 = 0, i2 = 0;
  double c0 = 0.0, c1 = 0.0, c2 = 0.0, c3 = 0.0, c4 = 0.0;
  if (samp) {
    const double* R1 = mats + RST_OFF_R1;
    const double* R2 = mats + RST_OFF_R2;
    const double del = md == 1 ? 1.0 : 0.0;
    i2 = md - 1;
    i1 = md >= 2 ? md - 2 : 0;
    i0 = md >= 3 ? md - 3 : 0;
    if (lane == 0) {
      c2 = -h;
    } else if (lane == 1) {
      c0 = md >= 3 ? h * R1[md - 3] : 0.0;
      c1 = md >= 2 ? h * R1[md - 2] : 0.0;
      c2 = h * R1[md - 1];
      c3 = -h * del;
    } else {
      c0 = md >= 3 ? -h * R2[md - 3] : 0.0;
      c1 = md >= 2 ? -h * R2[md - 2] : 0.0;
      c2 = -h * R2[md - 1];
      c3 = h * hm0;
      c4 = -h * del / d;
    }
  }
  // this thread's source coefficients of the current interval: b_q, b_{q+2},
  // b_{q+4} (map threads) or b_0, b_1 (sampler lanes)
  double bc[3] = {0.0, 0.0, 0.0};
  if (mv) {
#pragma unroll
    for (int t = 0; t < 3; ++t) bc[t] = bf[q + 2 * t];
  } else if (samp) {
    bc[0] = bf[0];
    bc[1] = bf[1];
  }
  double mx = 0.0;
  int cur = 0;
  for (int i = 0; i < Nt; ++i) {
    const bool pre = (i + 1 < Nt);
    double bn[3] = {0.0, 0.0, 0.0};
    if (pre) {
      const double* nx = bf + (int64_t)(i + 1) * RST_P;
      if (mv) {
#pragma unroll
        for (int t = 0; t < 3; ++t) bn[t] = nx[q + 2 * t];
      } else if (samp) {
        bn[0] = nx[0];
        bn[1] = nx[1];
      }
    }
    if (mv) {
      double s0 = 0.0, s1 = 0.0;
#pragma unroll
      for (int k = 0; k < 32; k += 2) {
        s0 = fma(Er[k], u[cur][q + 2 * k], s0);
        s1 = fma(Er[k + 1], u[cur][q + 2 * k + 2], s1);
      }
      s0 = fma(bc[0], Wr[0], s0);
      s1 = fma(bc[1], Wr[1], s1);
      s0 = fma(bc[2], Wr[2], s0);
      double sum = s0 + s1;
      sum += __shfl_xor_sync(0xffffffffu, sum, 1);
      if (q == 0 && r < md) u[cur ^ 1][r] = sum;
    } else if (samp) {
      double v = c0 * u[cur][i0];
      v = fma(c1, u[cur][i1], v);
      v = fma(c2, u[cur][i2], v);
      v = fma(c3, bc[0], v);
      v = fma(c4, bc[1], v);
      sf[(int64_t)i * 3 + lane] = v;
      if (lane == 0) mx = fmax(mx, fabs(v));
    }
    if (pre) {
#pragma unroll
      for (int t = 0; t < 3; ++t) bc[t] = bn[t];
    }
    __syncthreads();
    cur ^= 1;
  }
  // u[cur] = u(T): the last sample (source value and d-scaled slope from the
  // last interval's polynomial at theta = 1), the maximum, the stopping test
  if (samp) {
    const double* last = bf + (int64_t)(Nt - 1) * RST_P;
    double al = 0.0, dal = 0.0;
#pragma unroll
    for (int j = 0; j < RST_P; ++j) {
      al += last[j];
      dal += j * last[j];
    }
    double v = c0 * u[cur][i0];
    v = fma(c1, u[cur][i1], v);
    v = fma(c2, u[cur][i2], v);
    v = fma(c3, al, v);
    v = fma(c4, dal, v);
    sf[(int64_t)Nt * 3 + lane] = v;
    if (lane == 0) {
      mx = fmax(mx, fabs(v));
      resid[f] = mx;
      if (!isfinite(mx)) fstate[f] = 3;            // reported by the host
      else if (mx <= tol_abs) fstate[f] = 1;       // stops after this restart's combination
    }
  }
  for (int i = tid; i < MMAX; i += blockDim.x) u_out[(int64_t)f * MMAX + i] = i < md ? u[cur][i] : 0.0;
}

kx_status launch_rst_cascade(kx_ctx* c, cudaStream_t st, int nfreq, const double* b, int Nt, double d,
                             double tol_abs) {
  time_begin(c);
  k_rst_cascade<<<nfreq, RST_THREADS, 0, st>>>(c->d_rst_mats, b, c->d_rst_smp, Nt, d, tol_abs, c->d_rst_state,
                                               c->d_rst_res, c->d_rst_u);
  time_end(c, KX_K_CASCADE, 0.0);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// The next restart's interval coefficients from the samples (frequencies
// still running only).
__global__ void k_rst_coef(const double* __restrict__ smp, double* __restrict__ b, int Nt, double d,
                           const int* __restrict__ fstate) {
  const int f = blockIdx.y;
  if (fstate[f] != 0) return;
  const double* sf = smp + (int64_t)f * (Nt + 1) * 3;
  double* bf = b + (int64_t)f * Nt * RST_P;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < Nt; i += gridDim.x * blockDim.x) {
    double bb[RST_P];
    hermite5(sf[3 * i], sf[3 * i + 1], sf[3 * i + 2], sf[3 * i + 3], sf[3 * i + 4], sf[3 * i + 5], d, bb);
#pragma unroll
    for (int j = 0; j < RST_P; ++j) bf[(int64_t)i * RST_P + j] = bb[j];
  }
}

kx_status launch_rst_coef(kx_ctx* c, cudaStream_t st, int nfreq, double* b, int Nt, double d) {
  const int gx = std::min((Nt + 255) / 256, 64);
  k_rst_coef<<<dim3(gx, nfreq), 256, 0, st>>>(c->d_rst_smp, b, Nt, d, c->d_rst_state);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// v_{m+1} of one basis slot (stored unnormalised in column m_done) becomes
// column 0 of another; m_done is read on the device.
template <typename T>
__global__ void k_rst_nextvec(Slot<T> from, Slot<T> to, int64_t n, int64_t ld) {
  const int md = from.st->m_done;
  const T* __restrict__ src = from.V + (int64_t)md * ld;
  T* __restrict__ dst = to.V;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    dst[e] = src[e];
}

kx_status launch_rst_nextvec(kx_ctx* c, cudaStream_t st, int from, int to) {
  if (c->d.precision == KX_FP64)
    k_rst_nextvec<double><<<c->nblk, NTHREADS, 0, st>>>(make_slot<double>(c, from), make_slot<double>(c, to), c->n,
                                                        c->ld);
  else
    k_rst_nextvec<float><<<c->nblk, NTHREADS, 0, st>>>(make_slot<float>(c, from), make_slot<float>(c, to), c->n,
                                                       c->ld);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// y_j += V_m u_j(T) on the output plane (FP64), for frequencies not stopped
// before this restart.  Stored basis columns are unnormalised: v_i = scale_i V_i.
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_rst_plane(Slot<T> s, int64_t ld, Geo g, int axis, int idx,
                                                       int64_t P, const int* __restrict__ fstate,
                                                       const double* __restrict__ u, double* yp) {
  const int f = blockIdx.y;
  const int sf = fstate[f];
  if (sf == 2 || sf == 3) return;
  __shared__ double cf[MMAX];
  const int md = s.st->m_done;
  for (int q = threadIdx.x; q < md; q += blockDim.x) cf[q] = u[(int64_t)f * MMAX + q] * s.scale[q];
  __syncthreads();
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < P; t += (int64_t)gridDim.x * blockDim.x) {
    const int64_t e = plane_node(g, axis, idx, t);
    double acc = 0.0;
    for (int j = 0; j < md; ++j) acc = fma(cf[j], (double)s.V[(int64_t)j * ld + e], acc);
    yp[(int64_t)f * P + t] += acc;
  }
}

kx_status launch_rst_plane(kx_ctx* c, cudaStream_t st, int slot, int nfreq, int axis, int idx, int64_t P) {
  const int gx = (int)std::max<int64_t>(1, std::min<int64_t>((P + NTHREADS - 1) / NTHREADS, 64));
  time_begin(c);
  if (c->d.precision == KX_FP64)
    k_rst_plane<double><<<dim3(gx, nfreq), NTHREADS, 0, st>>>(make_slot<double>(c, slot), c->ld, c->geo,
                                                                   axis, idx, P, c->d_rst_state, c->d_rst_u,
                                                                   c->d_rst_yp);
  else
    k_rst_plane<float><<<dim3(gx, nfreq), NTHREADS, 0, st>>>(make_slot<float>(c, slot), c->ld, c->geo,
                                                                  axis, idx, P, c->d_rst_state, c->d_rst_u,
                                                                  c->d_rst_yp);
  time_end(c, KX_K_RESTART, 0.0);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// y_j += V_m u_j(T) on the full field.  FP64: plain accumulation into Y.
// FP32: every coefficient is split into a float pair hi + lo, the
// combination is summed error-free (two-product by FMA, Knuth's two-sum) and
// added to the float-pair accumulator (Y_j, lo_j) by a two-sum, so the
// accumulated response keeps about twice float precision over the restarts.
__device__ __forceinline__ void rst_acc(float& s, float& c, float hi, float lo, float v) {
  const float p = hi * v;
  const float e = fmaf(hi, v, -p) + lo * v;
  const float t = s + p;
  const float z = t - s;
  c += ((s - (t - z)) + (p - z)) + e;
  s = t;
}

template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_rst_full(Slot<T> s, int64_t ld, int64_t n, int nfreq,
                                                      const int* __restrict__ fstate,
                                                      const double* __restrict__ u, T* __restrict__ Y,
                                                      float* __restrict__ lo_acc) {
  __shared__ double cf[MAXF][MMAX];
  __shared__ int act[MAXF];
  const int md = s.st->m_done;
  for (int q = threadIdx.x; q < nfreq * MMAX; q += blockDim.x) {
    const int f = q / MMAX, j = q - f * MMAX;
    cf[f][j] = j < md ? u[(int64_t)f * MMAX + j] * s.scale[j] : 0.0;
  }
  for (int f = threadIdx.x; f < nfreq; f += blockDim.x) act[f] = !(fstate[f] == 2 || fstate[f] == 3);
  __syncthreads();
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    T v[MMAX];
#pragma unroll
    for (int j = 0; j < MMAX; ++j) v[j] = j < md ? s.V[(int64_t)j * ld + e] : T(0);
    for (int f = 0; f < nfreq; ++f) {
      if (!act[f]) continue;
      if constexpr (sizeof(T) == 8) {
        double acc = 0.0;
#pragma unroll
        for (int j = 0; j < MMAX; ++j) acc = fma(cf[f][j], (double)v[j], acc);
        Y[(int64_t)f * n + e] += (T)acc;
      } else {
        float sx = 0.f, cx = 0.f;
#pragma unroll
        for (int j = 0; j < MMAX; ++j) {
          const float hi = (float)cf[f][j];
          const float lo = (float)(cf[f][j] - (double)hi);
          rst_acc(sx, cx, hi, lo, (float)v[j]);
        }
        // (Y, lo) += sx + cx
        float& yh = reinterpret_cast<float*>(Y)[(int64_t)f * n + e];
        float& yl = lo_acc[(int64_t)f * n + e];
        const float t = yh + sx;
        const float z = t - yh;
        const float err = (yh - (t - z)) + (sx - z);
        yh = t;
        yl += err + cx;
      }
    }
  }
}

kx_status launch_rst_full(kx_ctx* c, cudaStream_t st, int slot, int nfreq, void* Y) {
  time_begin(c);
  if (c->d.precision == KX_FP64)
    k_rst_full<double><<<c->nblk, NTHREADS, 0, st>>>(make_slot<double>(c, slot), c->ld, c->n, nfreq,
                                                            c->d_rst_state, c->d_rst_u, (double*)Y, nullptr);
  else
    k_rst_full<float><<<c->nblk, NTHREADS, 0, st>>>(make_slot<float>(c, slot), c->ld, c->n, nfreq,
                                                           c->d_rst_state, c->d_rst_u, (float*)Y,
                                                           (float*)c->d_zre);
  time_end(c, KX_K_RESTART, (c->m + 3.0 * nfreq) * c->n * c->esize);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// Outputs: plane values in the context's precision and the summed |E|^2 per
// frequency (one CTA each); the full field's float pair folded to one float.
template <typename T>
__global__ void k_rst_out(const double* __restrict__ yp, int64_t P, T* __restrict__ E_plane, double* intensity) {
  const int f = blockIdx.x;
  double acc = 0.0;
  for (int64_t t = threadIdx.x; t < P; t += blockDim.x) {
    const double v = yp[(int64_t)f * P + t];
    if (E_plane) E_plane[(int64_t)f * P + t] = (T)v;
    acc += v * v;
  }
  __shared__ double red[32];
  acc = warp_sum(acc);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
    intensity[f] = s;
  }
}

__global__ void k_rst_fold(int64_t total, float* __restrict__ Y, const float* __restrict__ lo) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x)
    Y[e] += lo[e];
}

kx_status launch_rst_out(kx_ctx* c, cudaStream_t st, int nfreq, int64_t P, void* E_plane, double* d_intensity,
                         void* Y) {
  if (c->d.precision == KX_FP64)
    k_rst_out<double><<<nfreq, 1024, 0, st>>>(c->d_rst_yp, P, (double*)E_plane, d_intensity);
  else
    k_rst_out<float><<<nfreq, 1024, 0, st>>>(c->d_rst_yp, P, (float*)E_plane, d_intensity);
  KX_CHECK_LAUNCH(c);
  if (Y && c->d.precision == KX_FP32) {
    k_rst_fold<<<c->nblk, NTHREADS, 0, st>>>((int64_t)nfreq * c->n, (float*)Y, (const float*)c->d_zre);
    KX_CHECK_LAUNCH(c);
  }
  return KX_OK;
}

}  // namespace kx
