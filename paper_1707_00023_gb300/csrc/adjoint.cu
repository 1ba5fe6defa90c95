// Adjoint of the frequency responses: gradient of the summed output-plane
// intensity L = sum_f sum_plane |E_f(T)|^2 with respect to the per-cell
// permittivity.  (The paper has no gradient; this follows from eq. (ode).)
//
//   dL/deps_c = -sum_f int_0^T lambda_f(t)^T (dA/deps_c) y_f(t) dt,
//   lambda_f(t) = exp(-(T - t) A^T) lambda_f(T),  lambda_f(T) = 2 P^T P y_f(T),
//   (dA/deps_c) y |_e = -(1 / (4 eps_e)) (A y)_e   for the E nodes e around c,
// so dL/deps_c = (1/4) sum_{e around c} Q_e with
//   Q_e = sum_f int_0^T lambda_e(t) (A y)_e(t) / eps_e dt.
//
// Per time sub-step [t_k, t_k + tau_k] of the forward solution (restarted
// in time), y(t_k + s) = V u(s) from the forward basis recomputed from the
// checkpoint y(t_k), (A y) = V_{m+1} H u + sin(W t) g from its Arnoldi
// relation, and lambda(t_k + s) = W w(tau_k - s) from an Arnoldi basis of A^T
// started at lambda(t_k + tau_k).  The integral over the sub-step is
// composite Gauss-Legendre quadrature; the projected coefficients u, w at the
// nodes are exact exponentials of the projected matrices.
#include <algorithm>
#include <cmath>
#include <vector>

#include "kx_dense.cuh"
#include <atomic>

#include "kx_internal.cuh"

namespace kx {

constexpr int GAUSS_P = 8;          // Gauss-Legendre nodes per sub-interval
constexpr double QUAD_DELTA = 0.4;  // longest sub-interval (time units)

// lambda(T) = 2 P^T P y: plane values of the E components, zero elsewhere.
template <typename T>
__global__ void k_adj_seed(Geo g, int axis, int idx, const T* __restrict__ y, T* __restrict__ lam) {
  const int nE = g.ne;
  int na, nb;
  if (g.dim == 2) {
    na = axis == 0 ? g.ny : g.nx;
    nb = 1;
  } else {
    na = axis == 0 ? g.ny : g.nx;
    nb = axis == 2 ? g.ny : g.nz;
  }
  const int64_t np = (int64_t)na * nb;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nE * np;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int q = (int)(t / np);
    const int64_t p = t % np;
    const int a = (int)(p % na), b = (int)(p / na);
    int i, j, k;
    if (g.dim == 2) {
      k = 0;
      if (axis == 0) { i = idx; j = a; } else { i = a; j = idx; }
    } else if (axis == 0) { i = idx; j = a; k = b; }
    else if (axis == 1) { i = a; j = idx; k = b; }
    else { i = a; j = b; k = idx; }
    const int64_t e = (int64_t)(g.nh + q) * g.ncell + ((int64_t)k * g.ny + j) * g.nx + i;
    lam[e] = (T)(2.0 * (double)y[e]);
  }
}

// y = M x for an m x m row-major matrix, four threads per row.
__device__ void cta_mv(const double* __restrict__ M, const double* x, double* y, int m) {
  const int r = threadIdx.x >> 2, part = threadIdx.x & 3;
  double s = 0.0;
  if (r < m)
    for (int c = part; c < m; c += 4) s = fma(M[r * m + c], x[c], s);
  s += __shfl_xor_sync(0xffffffffu, s, 1);
  s += __shfl_xor_sync(0xffffffffu, s, 2);
  __syncthreads();
  if (r < m && part == 0) y[r] = s;
  __syncthreads();
}

// Projected quadrature coefficients of one sub-step.  Block 0 works on the
// forward basis (slot 0), block 1 on the adjoint basis (slot 1).
//   nodes s_q = (i + x_j) delta, q = i * P + j, delta = tau / nsub
//   alpha[q][r] = scale_V[r] (H_V u(s_q))_r,  r <= m_V   (A y at s_q)
//   omg[q][r]   = scale_W[r] w(tau - s_q)_r,  r < m_W    (lambda at s_q)
//   cw[q] = delta * wg[j],  sn[q] = sin(W (t_k + s_q))
//   slot 1's u = w(tau)   (lambda at t_k, for the next sub-step)
__global__ void __launch_bounds__(256) k_adj_coeffs(SlotSet<float> ss, int ldh, double tau, int nsub,
                                                    const double* __restrict__ xg,
                                                    const double* __restrict__ wg, double omega,
                                                    double tk, double* __restrict__ Eg,
                                                    float* __restrict__ alpha, float* __restrict__ omg,
                                                    float* __restrict__ cw, float* __restrict__ sn,
                                                    int* status) {
  extern __shared__ double sm[];
  __shared__ double red[32];
  __shared__ double lv[72];
  __shared__ int piv;
  __shared__ double z[2][72], acc[72];
  const int which = blockIdx.x;
  const Slot<float> sl = slot_at(ss, which);
  const double* H = sl.H;
  const int m = sl.st->m_done;
  const double beta = sl.st->beta;
  const double delta = tau / nsub;
  double* E = Eg + (size_t)which * MMAX * MMAX;
  if (m <= 0 || beta == 0.0) {
    // zero state: every coefficient vanishes
    for (int q = threadIdx.x; q < nsub * GAUSS_P; q += blockDim.x) {
      for (int r = 0; r <= MMAX; ++r) {
        if (which == 0) alpha[(size_t)q * (MMAX + 1) + r] = 0.f;
        else if (r < MMAX) omg[(size_t)q * MMAX + r] = 0.f;
      }
      if (which == 0) {
        const int i = q / GAUSS_P, j = q % GAUSS_P;
        cw[q] = (float)(delta * wg[j]);
        sn[q] = (float)sin(omega * (tk + (i + xg[j]) * delta));
      }
    }
    if (which == 1 && threadIdx.x < ldh - 1) sl.u[threadIdx.x] = 0.0;
    return;
  }
  // E = exp(-delta H_m)
  double* buf[6];
  for (int q = 0; q < 6; ++q) buf[q] = sm + (size_t)q * m * m;
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    buf[0][idx] = (r <= c + 1) ? -delta * H[r + (int64_t)c * ldh] : 0.0;
  }
  __syncthreads();
  double* X = cta_expm(buf, m, red, lv, &piv);
  if (!X) {
    if (threadIdx.x == 0) *status = KX_ENONFINITE;
    return;
  }
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) E[idx] = X[idx];
  // H_m row-major in shared memory for the Taylor steps (buf[1] is free now)
  double* Hs = buf[0] == X ? buf[1] : buf[0];
  for (int idx = threadIdx.x; idx < m * m; idx += blockDim.x) {
    const int r = idx / m, c = idx - r * m;
    Hs[idx] = (r <= c + 1) ? H[r + (int64_t)c * ldh] : 0.0;
  }
  __syncthreads();
  const double hnext = H[m + (int64_t)(m - 1) * ldh];
  for (int j = 0; j < GAUSS_P; ++j) {
    // z = exp(-x_j delta H) beta e_1 by its Taylor series (|x_j delta H| small)
    const double h = -xg[j] * delta;
    for (int r = threadIdx.x; r < m; r += blockDim.x) {
      z[0][r] = r == 0 ? beta : 0.0;
      acc[r] = z[0][r];
    }
    __syncthreads();
    int cur = 0;
    for (int kk = 1; kk <= 60; ++kk) {
      cta_mv(Hs, z[cur], z[cur ^ 1], m);
      cur ^= 1;
      double nrm = 0.0, tot = 0.0;
      for (int r = threadIdx.x; r < m; r += blockDim.x) {
        z[cur][r] *= h / kk;
        acc[r] += z[cur][r];
      }
      __syncthreads();
      if (threadIdx.x < 32) {
        for (int r = threadIdx.x; r < m; r += 32) {
          nrm = fmax(nrm, fabs(z[cur][r]));
          tot = fmax(tot, fabs(acc[r]));
        }
        for (int o = 16; o > 0; o >>= 1) {
          nrm = fmax(nrm, __shfl_xor_sync(0xffffffffu, nrm, o));
          tot = fmax(tot, __shfl_xor_sync(0xffffffffu, tot, o));
        }
        if (threadIdx.x == 0) red[0] = (nrm <= 1e-18 * tot) ? 1.0 : 0.0;
      }
      __syncthreads();
      if (red[0] != 0.0) break;
      __syncthreads();
    }
    // march the sub-intervals: value at (i + x_j) delta is E^i z
    for (int r = threadIdx.x; r < m; r += blockDim.x) z[0][r] = acc[r];
    __syncthreads();
    cur = 0;
    for (int i = 0; i < nsub; ++i) {
      if (i > 0) {
        cta_mv(E, z[cur], z[cur ^ 1], m);
        cur ^= 1;
      }
      const double* u = z[cur];
      if (which == 0) {
        const int q = i * GAUSS_P + j;
        // alpha = scale .* (Hbar u), Hbar the (m+1) x m Hessenberg matrix
        for (int r = threadIdx.x; r <= m; r += blockDim.x) {
          double s = 0.0;
          if (r < m) {
            for (int c = max(r - 1, 0); c < m; ++c) s = fma(Hs[r * m + c], u[c], s);
          } else {
            s = hnext * u[m - 1];
          }
          alpha[(size_t)q * (MMAX + 1) + r] = (float)(sl.scale[r] * s);
        }
        for (int r = m + 1 + threadIdx.x; r <= MMAX; r += blockDim.x) alpha[(size_t)q * (MMAX + 1) + r] = 0.f;
        if (threadIdx.x == 0) {
          cw[q] = (float)(delta * wg[j]);
          sn[q] = (float)sin(omega * (tk + (i + xg[j]) * delta));
        }
      } else {
        // lambda at t_k + s_q needs w(tau - s_q): tau - s_q = (nsub-1-i + x_{P-1-j}) delta
        const int q = (nsub - 1 - i) * GAUSS_P + (GAUSS_P - 1 - j);
        for (int r = threadIdx.x; r < MMAX; r += blockDim.x)
          omg[(size_t)q * MMAX + r] = r < m ? (float)(sl.scale[r] * u[r]) : 0.f;
      }
      __syncthreads();
    }
  }
  if (which == 1) {
    // w(tau) = E^nsub beta e_1 for the update lambda(t_k) = W w(tau)
    for (int r = threadIdx.x; r < m; r += blockDim.x) z[0][r] = r == 0 ? beta : 0.0;
    __syncthreads();
    int cur = 0;
    for (int i = 0; i < nsub; ++i) {
      cta_mv(E, z[cur], z[cur ^ 1], m);
      cur ^= 1;
    }
    for (int r = threadIdx.x; r < m; r += blockDim.x) sl.u[r] = z[cur][r];
  }
}

// Q_e += sum_q cw_q (sum_i alpha_q,i V_i,e + sn_q g_e) (sum_i omg_q,i W_i,e) / eps_e
// over the E nodes e, in chunks of 32 quadrature nodes staged in shared memory.
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_adj_accum(Geo g, const T* __restrict__ V, const T* __restrict__ W,
                                                       int64_t ld, int mV, int mW, const T* __restrict__ gsrc,
                                                       const T* __restrict__ ie, int nq,
                                                       const float* __restrict__ alpha,
                                                       const float* __restrict__ omg,
                                                       const float* __restrict__ cw,
                                                       const float* __restrict__ sn, double* __restrict__ Q) {
  constexpr int CH = 32;
  __shared__ float sa[CH][MMAX + 1];
  __shared__ float so[CH][MMAX];
  __shared__ float scw[CH], ssn[CH];
  const int64_t nE = (int64_t)g.ne * g.ncell;
  const int64_t off = (int64_t)g.nh * g.ncell;
  const int64_t rounds = (nE + blockDim.x - 1) / blockDim.x;
  for (int64_t r0 = blockIdx.x; r0 < rounds; r0 += gridDim.x) {
    const int64_t e = r0 * blockDim.x + threadIdx.x;
    const bool act = e < nE;
    double qacc = 0.0;
    const T ge = act ? gsrc[off + e] : T(0);
    for (int q0 = 0; q0 < nq; q0 += CH) {
      const int nc = min(CH, nq - q0);
      __syncthreads();
      for (int t = threadIdx.x; t < nc * (MMAX + 1); t += blockDim.x)
        sa[t / (MMAX + 1)][t % (MMAX + 1)] = alpha[(size_t)(q0 + t / (MMAX + 1)) * (MMAX + 1) + t % (MMAX + 1)];
      for (int t = threadIdx.x; t < nc * MMAX; t += blockDim.x)
        so[t / MMAX][t % MMAX] = omg[(size_t)(q0 + t / MMAX) * MMAX + t % MMAX];
      for (int t = threadIdx.x; t < nc; t += blockDim.x) {
        scw[t] = cw[q0 + t];
        ssn[t] = sn[q0 + t];
      }
      __syncthreads();
      if (!act) continue;
      float a[CH], b[CH];
#pragma unroll
      for (int t = 0; t < CH; ++t) { a[t] = 0.f; b[t] = 0.f; }
      for (int i = 0; i <= mV; ++i) {
        const float v = (float)V[(int64_t)i * ld + off + e];
#pragma unroll
        for (int t = 0; t < CH; ++t) a[t] = fmaf(sa[t][i], v, a[t]);
      }
      for (int i = 0; i < mW; ++i) {
        const float w = (float)W[(int64_t)i * ld + off + e];
#pragma unroll
        for (int t = 0; t < CH; ++t) b[t] = fmaf(so[t][i], w, b[t]);
      }
      float part = 0.f;
#pragma unroll
      for (int t = 0; t < CH; ++t)
        if (t < nc) part = fmaf(scw[t] * fmaf(ssn[t], (float)ge, a[t]), b[t], part);
      qacc += (double)part;
    }
    if (act) Q[e] += qacc * (double)ie[e];
  }
}

// grad_c = (1/4) sum of Q over the E nodes whose closure holds cell c.
__global__ void k_adj_cells(Geo g, const double* __restrict__ Q, double* __restrict__ grad) {
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < g.ncell;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const int i = (int)(cell % g.nx);
    const int64_t r = cell / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    const int ip = i + 1 == g.nx ? 0 : i + 1, jp = j + 1 == g.ny ? 0 : j + 1;
    const int kp = (g.dim == 3 && k + 1 == g.nz) ? 0 : k + 1;
    const int64_t nx = g.nx, nxy = (int64_t)g.nx * g.ny, nc = g.ncell;
    double s = 0.0;
    if (g.dim == 2) {
      s = Q[j * nx + i] + Q[j * nx + ip] + Q[jp * nx + i] + Q[jp * nx + ip];
    } else {
      // Ex nodes (i, j or j+1, k or k+1); Ey (i or i+1, j, k or k+1); Ez (i or i+1, j or j+1, k)
      s += Q[k * nxy + j * nx + i] + Q[k * nxy + jp * nx + i] + Q[kp * nxy + j * nx + i] +
           Q[kp * nxy + jp * nx + i];
      s += Q[nc + k * nxy + j * nx + i] + Q[nc + k * nxy + j * nx + ip] + Q[nc + kp * nxy + j * nx + i] +
           Q[nc + kp * nxy + j * nx + ip];
      s += Q[2 * nc + k * nxy + j * nx + i] + Q[2 * nc + k * nxy + j * nx + ip] +
           Q[2 * nc + k * nxy + jp * nx + i] + Q[2 * nc + k * nxy + jp * nx + ip];
    }
    grad[cell] = 0.25 * s;
  }
}

// ---------------------------------------------------------------------------
kx_status launch_adj_seed(kx_ctx* c, const void* y, void* lam, int axis, int idx) {
  if (c->d.precision == KX_FP64)
    k_adj_seed<double><<<c->nblk, NTHREADS, 0, c->stream>>>(c->geo, axis, idx, (const double*)y, (double*)lam);
  else
    k_adj_seed<float><<<c->nblk, NTHREADS, 0, c->stream>>>(c->geo, axis, idx, (const float*)y, (float*)lam);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

kx_status launch_adj_substep(kx_ctx* c, double tau, double omega, double tk, const void* g) {
  const int nsub = std::max(1, (int)std::ceil(tau / QUAD_DELTA));
  if (nsub * GAUSS_P > c->adj_nq_max) {
    snprintf(c->err, sizeof(c->err), "adjoint: sub-step %.3g needs more than %d quadrature nodes", tau,
             c->adj_nq_max);
    return KX_EINVAL;
  }
  const int m = c->m;
  static SmemOptIn attr{};
  const kx_status so = smem_opt_in(c, attr, (const void*)k_adj_coeffs, expm_smem_bytes(MMAX + 2));
  if (so != KX_OK) return so;
  int* status = reinterpret_cast<int*>(c->d_small + 64);
  time_begin(c);
  k_adj_coeffs<<<2, 256, expm_smem_bytes(m), c->stream>>>(
      make_slotset<float>(c, 0), m + 1, tau, nsub, c->d_gauss, c->d_gauss + GAUSS_P, omega, tk,
      c->d_expm_ws, c->d_adj_alpha, c->d_adj_omg, c->d_adj_cw, c->d_adj_sn, status);
  time_end(c, KX_K_PROJ, 0.0);
  KX_CHECK_LAUNCH(c);
  const int nq = nsub * GAUSS_P;
  const int64_t nE = (int64_t)c->geo.ne * c->geo.ncell;
  const int blocks = (int)std::min<int64_t>((nE + NTHREADS - 1) / NTHREADS, (int64_t)c->nsm * 4);
  const int64_t sV = (int64_t)(m + 1) * c->ld;
  // the basis sizes are read back by the host after each Arnoldi run
  const int mV = c->h_state[0].m_done, mW = c->h_state[1].m_done;
  time_begin(c);
  if (c->d.precision == KX_FP64) {
    k_adj_accum<double><<<blocks, NTHREADS, 0, c->stream>>>(
        c->geo, (const double*)c->d_V, (const double*)c->d_V + sV, c->ld, mV, mW, (const double*)g,
        (const double*)c->d_inv_eps, nq, c->d_adj_alpha, c->d_adj_omg, c->d_adj_cw, c->d_adj_sn, c->d_adj_Q);
  } else {
    k_adj_accum<float><<<blocks, NTHREADS, 0, c->stream>>>(
        c->geo, (const float*)c->d_V, (const float*)c->d_V + sV, c->ld, mV, mW, (const float*)g,
        (const float*)c->d_inv_eps, nq, c->d_adj_alpha, c->d_adj_omg, c->d_adj_cw, c->d_adj_sn, c->d_adj_Q);
  }
  time_end(c, KX_K_ZUPDATE, (double)(mV + 1 + mW) * nE * c->esize);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

kx_status launch_adj_cells(kx_ctx* c, double* grad) {
  k_adj_cells<<<c->nblk, NTHREADS, 0, c->stream>>>(c->geo, c->d_adj_Q, grad);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// Gauss-Legendre nodes and weights on [0, 1] by Newton's method on P_n.
void gauss_legendre01(int n, double* x, double* w) {
  for (int i = 0; i < n; ++i) {
    double t = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = t;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      const double dp = n * (t * p1 - p0) / (t * t - 1.0);
      const double dt = p1 / dp;
      t -= dt;
      if (std::fabs(dt) < 1e-16) break;
    }
    double p0 = 1.0, p1 = t;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2 * k - 1) * t * p1 - (k - 1) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    const double dp = n * (t * p1 - p0) / (t * t - 1.0);
    // node on [-1, 1] -> [0, 1], ascending
    x[n - 1 - i] = 0.5 * (t + 1.0);
    w[n - 1 - i] = 1.0 / ((1.0 - t * t) * dp * dp);
  }
}

int gauss_points() { return GAUSS_P; }

}  // namespace kx
