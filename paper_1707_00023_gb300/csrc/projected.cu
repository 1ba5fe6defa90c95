// FP64 projected (small, dense) work of the Krylov path, one CTA per matrix:
//  * matrix exponential by scaling and squaring with Pade approximants of
//    degree 3/5/7/9/13 (Higham 2005, "The scaling and squaring method for the
//    matrix exponential revisited", SIAM J. Matrix Anal. Appl. 26(4)),
//  * time sub-step control from Lemma 1's residual (eq. (resid)),
//  * projected solutions with a sine source (eq. (corr2), Corollary 1),
//  * shifted Hessenberg solves of the multi-shift FOM.
// Matrices live in shared memory, row-major, leading dimension = size.
#include <atomic>

#include "kx_internal.cuh"
#include "kx_dense.cuh"

namespace kx {

size_t expm_smem_bytes(int msz) { return (size_t)6 * msz * msz * sizeof(double); }

// ---------------------------------------------------------------------------
// Time sub-step control (restart in time, Sect. 3.3): with the Arnoldi
// decomposition of the current restart, u(t) = exp(-t H_m) beta e_1 is
// tabulated at t_k = k * tau / K, and Lemma 1 gives the residual norm
// ||r_m(t_k)|| = h_{m+1,m} |e_m^T u(t_k)| (||v_{m+1}|| = 1).  The largest t_k
// whose integrated residual (trapezoid rule, an error bound for a
// contractive exp(-tA)) stays below tol_rate * t_k is accepted; if none,
// tau shrinks 4x and the table is rebuilt.
__global__ void __launch_bounds__(256) k_substep(SlotSet<float> ss, int ldh, int K) {
  const Slot<float> sl = slot_at(ss, blockIdx.x);
  const double* H = sl.H;
  double* u_out = sl.u;
  SlotState* st = sl.st;
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double lv[72];
  __shared__ double uu[2][72];
  __shared__ int piv;
  __shared__ double s_err, s_tau;
  __shared__ int s_kacc, s_retry;
  if (st->finished || st->status || st->retired) return;
  const int m = st->m_done;
  if (m <= 0 || st->beta == 0.0) {
    if (threadIdx.x == 0) {
      st->t_now = st->T;
      st->finished = 1;
      for (int i = 0; i < ldh - 1; ++i) u_out[i] = 0.0;
    }
    return;
  }
  double* buf[6];
  for (int q = 0; q < 6; ++q) buf[q] = sm + (size_t)q * m * m;
  const double hnext = st->done ? 0.0 : H[m + (int64_t)(m - 1) * ldh];
  const double remaining = st->T - st->t_now;
  if (threadIdx.x == 0) {
    if (st->tol_mode == 0 && !(st->tol_abs > 0.0)) st->tol_abs = st->rtol * st->beta / st->T;
    double tau = st->tau_try;
    if (!(tau > 0.0)) {
      // first trial: Krylov dimension over the 1-norm of H_m
      double nrm = 0.0;
      for (int c = 0; c < m; ++c) {
        double s = 0.0;
        for (int r = 0; r <= min(c + 1, m - 1); ++r) s += fabs(H[r + (int64_t)c * ldh]);
        nrm = fmax(nrm, s);
      }
      tau = nrm > 0.0 ? 0.5 * m / nrm : remaining;
    }
    s_tau = fmin(tau, remaining);
  }
  __syncthreads();
  const double tol_rate = st->tol_mode ? st->rtol * st->beta / st->T : st->tol_abs;
  int evals = 0;
  for (int attempt = 0; attempt < 40; ++attempt) {
    const double tau = s_tau;
    const double dt = tau / K;
    for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
      const int r = idx / m, c = idx - r * m;
      // upper Hessenberg: the Arnoldi process writes nothing below the subdiagonal
      buf[0][idx] = (r <= c + 1) ? -dt * H[r + (int64_t)c * ldh] : 0.0;
    }
    __syncthreads();
    double* X = cta_expm(buf, m, red, lv, &piv);
    ++evals;
    if (!X) {
      // a failed slot stops: the later kernels of queued sub-steps skip it
      if (threadIdx.x == 0) {
        st->status = KX_ENONFINITE;
        st->done = 1;
      }
      return;
    }
    // tabulate u(t_k)
    for (int i = threadIdx.x; i < m; i += blockDim.x) uu[0][i] = (i == 0) ? st->beta : 0.0;
    if (threadIdx.x == 0) { s_err = 0.0; s_kacc = 0; s_retry = 0; }
    __syncthreads();
    double rho_prev = 0.0;
    int cur = 0;
    for (int k = 1; k <= K; ++k) {
      for (int r = threadIdx.x; r < m; r += blockDim.x) {
        double s = 0.0;
        for (int c = 0; c < m; ++c) s = fma(X[r * m + c], uu[cur][c], s);
        uu[cur ^ 1][r] = s;
      }
      __syncthreads();
      cur ^= 1;
      if (threadIdx.x == 0) {
        const double rho = fabs(hnext * uu[cur][m - 1]);
        const double e = s_err + 0.5 * dt * (rho_prev + rho);
        rho_prev = rho;
        if (isfinite(e) && e <= tol_rate * (k * dt)) {
          s_err = e;
          s_kacc = k;
          for (int i = 0; i < m; ++i) u_out[i] = uu[cur][i];
        } else {
          s_retry = 1;  // bound exceeded: stop the table here
        }
      }
      __syncthreads();
      if (s_retry) break;
    }
    if (s_kacc > 0) break;
    if (threadIdx.x == 0) s_tau = tau * 0.25;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    st->expm_evals += evals;
    if (s_kacc == 0) {
      st->status = KX_ENOCONV;
      st->done = 1;
      return;
    }
    const double tau = s_tau;
    const double dt = tau / K;
    const bool to_end = (tau >= remaining);
    const double tacc = (s_kacc == K && to_end) ? remaining : s_kacc * dt;
    st->t_now = (s_kacc == K && to_end) ? st->T : st->t_now + tacc;
    st->t_acc = tacc;
    st->err_acc += s_err;
    st->k_acc = s_kacc;
    st->substeps += 1;
    if (s_kacc == K) st->tau_try = to_end ? st->tau_try : tau * 1.5;
    else st->tau_try = tacc * 1.1;
    st->finished = (st->t_now >= st->T) ? 1 : 0;
  }
}

kx_status launch_substep_control(kx_ctx* c, int slot, int ns) {
  const int m = c->m;
  const size_t sm = expm_smem_bytes(m);
  static SmemOptIn attr{};
  const kx_status so = smem_opt_in(c, attr, (const void*)k_substep, expm_smem_bytes(MMAX + 2));
  if (so != KX_OK) return so;
  time_begin(c);
  k_substep<<<ns, 256, sm, c->stream>>>(make_slotset<float>(c, slot), m + 1, 32);
  time_end(c, KX_K_PROJ, 0.0);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// Projected solutions (one CTA per frequency):
//   nfreq == 0:  u = exp(-tau H_m) beta e_1
//   otherwise :  u_f = [exp(tau N_f)]_{0..m-1, m+1},
//                N_f = [[-H_m, beta e_1, 0], [0, 0, W_f], [0, -W_f, 0]],
// the exact solution of u' = -H_m u + sin(W_f t) beta e_1, u(0) = 0, whose
// two extra states carry sin and cos of W_f t (eq. (corr2)).
__global__ void __launch_bounds__(256) k_expm_project(const double* H, int ldh, int m, double beta,
                                                      double tau, const double* om, int nfreq,
                                                      double* u_out, int* status) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double lv[72];
  __shared__ int piv;
  const int f = blockIdx.x;
  const int n = nfreq > 0 ? m + 2 : m;
  double* buf[6];
  for (int q = 0; q < 6; ++q) buf[q] = sm + (size_t)q * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx - r * n;
    double v = 0.0;
    if (r < m && c < m) v = -H[r + (int64_t)c * ldh];
    if (nfreq > 0) {
      if (r == 0 && c == m) v = beta;
      if (r == m && c == m + 1) v = om[f];
      if (r == m + 1 && c == m) v = -om[f];
    }
    buf[0][idx] = tau * v;
  }
  __syncthreads();
  double* X = cta_expm(buf, n, red, lv, &piv);
  if (!X) {
    if (threadIdx.x == 0) *status = KX_ENONFINITE;
    return;
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x)
    u_out[(int64_t)f * m + i] = nfreq > 0 ? X[i * n + (m + 1)] : beta * X[i * n + 0];
}

kx_status launch_expm_project(kx_ctx* c, const double* dH, int ldh, int m, double beta, double tau,
                              const double* d_om, int nfreq, double* d_u) {
  const int n = nfreq > 0 ? m + 2 : m;
  static SmemOptIn attr{};
  const kx_status so = smem_opt_in(c, attr, (const void*)k_expm_project, expm_smem_bytes(MMAX + 2));
  if (so != KX_OK) return so;
  int* status = reinterpret_cast<int*>(c->d_small + 64);
  time_begin(c);
  k_expm_project<<<nfreq > 0 ? nfreq : 1, 256, expm_smem_bytes(n), c->stream>>>(
      dH, ldh, m, beta, tau, d_om, nfreq, d_u, status);
  time_end(c, KX_K_PROJ, 0.0);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// Shifted Hessenberg solves of the restarted multi-shift FOM (one warp per
// shift f):  (H_m + i W_f I) c_f = rho_f e_1,  then
//   coef_f = scale .* c_f  (real and imaginary parts, for z_f += V_m c_f),
//   rho_f <- -h_{m+1,m} e_m^T c_f   (the new residual is rho_f v_{m+1}).
// Gaussian elimination with partial pivoting between the two candidate
// rows of each column keeps the Hessenberg structure; the upper factor is
// kept in shared memory for the back substitution.
struct cplx { double r, i; };
__device__ __forceinline__ cplx cmul(cplx a, cplx b) { return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r}; }
__device__ __forceinline__ cplx csub(cplx a, cplx b) { return {a.r - b.r, a.i - b.i}; }
__device__ __forceinline__ cplx cdiv(cplx a, cplx b) {
  // Smith's algorithm
  if (fabs(b.r) >= fabs(b.i)) {
    const double q = b.i / b.r, d = b.r + b.i * q;
    return {(a.r + a.i * q) / d, (a.i - a.r * q) / d};
  }
  const double q = b.r / b.i, d = b.r * q + b.i;
  return {(a.r * q + a.i) / d, (a.i * q - a.r) / d};
}
__device__ __forceinline__ double cabs2(cplx a) { return hypot(a.r, a.i); }

template <typename T>
__global__ void k_shifted(const double* H, int ldh, int m, const double* scale, const double* om,
                          double* rho, T* coef, int* status) {
  extern __shared__ double smx[];
  cplx* U = reinterpret_cast<cplx*>(smx);          // m x m upper factor
  __shared__ cplx yv[MMAX];
  const int f = blockIdx.x;
  const int lane = threadIdx.x;
  const double W = om[f];
  auto Hc = [&](int r, int c) -> cplx {
    cplx v = {0.0, 0.0};
    if (r < m && c < m && r <= c + 1) v.r = H[r + (int64_t)c * ldh];
    if (r == c) v.i = W;
    return v;
  };
  // current pivot-candidate row (columns k..m-1) held across lanes
  cplx cur[2];
  for (int q = 0; q < 2; ++q) { const int c = lane + 32 * q; cur[q] = Hc(0, c); }
  cplx rcur = {rho[2 * f], rho[2 * f + 1]};
  bool ok = true;
  for (int k = 0; k < m; ++k) {
    cplx nxt[2];
    for (int q = 0; q < 2; ++q) { const int c = lane + 32 * q; nxt[q] = (k + 1 < m) ? Hc(k + 1, c) : cplx{0.0, 0.0}; }
    cplx rnxt = {0.0, 0.0};
    // diagonal entries at column k
    const int ql = k >> 5, ll = k & 31;
    cplx dk = {__shfl_sync(0xffffffffu, cur[ql].r, ll), __shfl_sync(0xffffffffu, cur[ql].i, ll)};
    cplx nk = {__shfl_sync(0xffffffffu, nxt[ql].r, ll), __shfl_sync(0xffffffffu, nxt[ql].i, ll)};
    const bool swap = (k + 1 < m) && (cabs2(nk) > cabs2(dk));
    if (swap) {
      for (int q = 0; q < 2; ++q) { const cplx t = cur[q]; cur[q] = nxt[q]; nxt[q] = t; }
      const cplx t = rcur; rcur = rnxt; rnxt = t;
      const cplx t2 = dk; dk = nk; nk = t2;
    }
    if (!(cabs2(dk) > 0.0)) ok = false;
    // pivot row is U's row k
    for (int q = 0; q < 2; ++q) { const int c = lane + 32 * q; if (c < m) U[k * m + c] = cur[q]; }
    if (lane == 0) yv[k] = rcur;
    if (k + 1 < m && ok) {
      const cplx l = cdiv(nk, dk);
      for (int q = 0; q < 2; ++q) { nxt[q] = csub(nxt[q], cmul(l, cur[q])); }
      rnxt = csub(rnxt, cmul(l, rcur));
      for (int q = 0; q < 2; ++q) cur[q] = nxt[q];
      rcur = rnxt;
    }
    __syncwarp();
  }
  __syncwarp();
  // back substitution
  __shared__ cplx cs[MMAX];
  for (int k = m - 1; k >= 0 && ok; --k) {
    cplx acc = {0.0, 0.0};
    for (int c = k + 1 + lane; c < m; c += 32) { const cplx p = cmul(U[k * m + c], cs[c]); acc.r += p.r; acc.i += p.i; }
    for (int o = 16; o > 0; o >>= 1) {
      acc.r += __shfl_xor_sync(0xffffffffu, acc.r, o);
      acc.i += __shfl_xor_sync(0xffffffffu, acc.i, o);
    }
    if (lane == 0) cs[k] = cdiv(csub(yv[k], acc), U[k * m + k]);
    __syncwarp();
  }
  if (!ok) {
    if (lane == 0) *status = KX_ENONFINITE;
    return;
  }
  for (int i = lane; i < MMAX; i += 32) {
    const double sc = (i < m) ? scale[i] : 0.0;
    coef[(2 * f) * MMAX + i] = (T)(i < m ? cs[i].r * sc : 0.0);
    coef[(2 * f + 1) * MMAX + i] = (T)(i < m ? cs[i].i * sc : 0.0);
  }
  if (lane == 0) {
    const double h = H[m + (int64_t)(m - 1) * ldh];
    rho[2 * f] = -h * cs[m - 1].r;
    rho[2 * f + 1] = -h * cs[m - 1].i;
  }
}

kx_status launch_shifted_solve(kx_ctx* c, int slot, int nfreq, int m) {
  Slot<double> s = make_slot<double>(c, slot);
  int* status = reinterpret_cast<int*>(c->d_small + 64);
  const size_t sm = (size_t)m * m * sizeof(cplx);
  static SmemOptIn attr_f{}, attr_d{};
  kx_status so = smem_opt_in(c, attr_f, (const void*)k_shifted<float>, MMAX * MMAX * sizeof(cplx));
  if (so == KX_OK) so = smem_opt_in(c, attr_d, (const void*)k_shifted<double>, MMAX * MMAX * sizeof(cplx));
  if (so != KX_OK) return so;
  time_begin(c);
  struct End { kx_ctx* c; ~End() { time_end(c, KX_K_PROJ, 0.0); } } end{c};
  if (c->d.precision == KX_FP64)
    k_shifted<double><<<nfreq, 32, sm, c->stream>>>(s.H, c->m + 1, m, s.scale, c->d_omegas, c->d_rho,
                                                     c->d_coefd, status);
  else
    k_shifted<float><<<nfreq, 32, sm, c->stream>>>(s.H, c->m + 1, m, s.scale, c->d_omegas, c->d_rho,
                                                    c->d_coef, status);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

}  // namespace kx
