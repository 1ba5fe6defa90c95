// Yee-grid operator A of eq. (ode) and the fused Arnoldi pass A.
//
// A = diag(M_mu, M_eps)^{-1} [[M_sigma, K], [-K^T, M_sigma]]   (Sect. 2.1)
//   H rows:  sigma H + curl E            (mu_r = 1)
//   E rows:  (sigma E - curl H) / eps
// K is the forward-difference curl of E on the H nodes and K^T the
// backward-difference curl of H on the E nodes.  One thread owns one cell
// (all 3 or 6 components of that cell), which keeps the neighbour planes of
// a block close in time and the reuse inside L1/L2.
#include "kx_internal.cuh"

namespace kx {

__device__ __forceinline__ bool is_wall(const Geo& g, int c, int i, int j, int k) {
  const unsigned mb = g.maskbits[c];
  return ((mb & 1u) && i == 0) || ((mb & 2u) && j == 0) || ((mb & 4u) && k == 0);
}

struct Cell {
  int i, j, k, ip, im, jp, jm, kp, km;
  int64_t c0, cip, cim, cjp, cjm, ckp, ckm;
};

__device__ __forceinline__ Cell make_cell(const Geo& g, int64_t cell) {
  Cell q;
  q.i = (int)(cell % g.nx);
  const int64_t r = cell / g.nx;
  q.j = (int)(r % g.ny);
  q.k = (int)(r / g.ny);
  q.ip = (q.i + 1 == g.nx) ? 0 : q.i + 1;
  q.im = (q.i == 0) ? g.nx - 1 : q.i - 1;
  q.jp = (q.j + 1 == g.ny) ? 0 : q.j + 1;
  q.jm = (q.j == 0) ? g.ny - 1 : q.j - 1;
  q.c0 = cell;
  q.cip = cell + (q.ip - q.i);
  q.cim = cell + (q.im - q.i);
  q.cjp = cell + (int64_t)(q.jp - q.j) * g.nx;
  q.cjm = cell + (int64_t)(q.jm - q.j) * g.nx;
  if (g.dim == 3) {
    const int64_t nxy = (int64_t)g.nx * g.ny;
    q.kp = (q.k + 1 == g.nz) ? 0 : q.k + 1;
    q.km = (q.k == 0) ? g.nz - 1 : q.k - 1;
    q.ckp = cell + (int64_t)(q.kp - q.k) * nxy;
    q.ckm = cell + (int64_t)(q.km - q.k) * nxy;
  } else {
    q.kp = q.km = 0;
    q.ckp = q.ckm = cell;
  }
  return q;
}

template <typename T>
__device__ __forceinline__ T ldv(const Geo& g, const T* __restrict__ v, int c, int64_t idx, int i,
                                 int j, int k) {
  return is_wall(g, c, i, j, k) ? T(0) : v[(int64_t)c * g.ncell + idx];
}

template <typename T>
__device__ __forceinline__ T sig_of(const Geo& g, const T* __restrict__ sig2, const Cell& q, int c) {
  const int li = g.la == 0 ? q.i : (g.la == 1 ? q.j : q.k);
  return sig2[2 * li + g.sighalf[c]];
}

// out = A v (TR = 0) or A^T v (TR = 1) at the components of one cell.
template <typename T, int DIM, int TR>
__device__ __forceinline__ void stencil(const Geo& g, const T* __restrict__ v,
                                        const T* __restrict__ ie, const T* __restrict__ sig2,
                                        const Cell& q, T* out) {
  const int64_t nc = g.ncell;
  const int i = q.i, j = q.j, k = q.k;
  if (DIM == 2) {
    // components 0 Hx (0,1/2), 1 Hy (1/2,0), 2 Ez (0,0)
    const T Hx = ldv(g, v, 0, q.c0, i, j, k), Hy = ldv(g, v, 1, q.c0, i, j, k);
    const T Hy_im = ldv(g, v, 1, q.cim, q.im, j, k), Hx_jm = ldv(g, v, 0, q.cjm, i, q.jm, k);
    T Ez = ldv(g, v, 2, q.c0, i, j, k);
    T Ez_jp = ldv(g, v, 2, q.cjp, i, q.jp, k), Ez_ip = ldv(g, v, 2, q.cip, q.ip, j, k);
    const T s0 = sig_of(g, sig2, q, 0), s1 = sig_of(g, sig2, q, 1), s2 = sig_of(g, sig2, q, 2);
    const T curlH = (Hy - Hy_im) - (Hx - Hx_jm);
    if (!TR) {
      out[0] = s0 * Hx + (Ez_jp - Ez);
      out[1] = s1 * Hy - (Ez_ip - Ez);
      out[2] = ie[q.c0] * (s2 * Ez - curlH);
    } else {
      Ez *= ie[q.c0];
      Ez_jp *= ie[q.cjp];
      Ez_ip *= ie[q.cip];
      out[0] = s0 * Hx - (Ez_jp - Ez);
      out[1] = s1 * Hy + (Ez_ip - Ez);
      out[2] = s2 * Ez + curlH;
    }
  } else {
    const int ip = q.ip, im = q.im, jp = q.jp, jm = q.jm, kp = q.kp, km = q.km;
    const T Hx = ldv(g, v, 0, q.c0, i, j, k), Hy = ldv(g, v, 1, q.c0, i, j, k);
    const T Hz = ldv(g, v, 2, q.c0, i, j, k);
    T Ex = ldv(g, v, 3, q.c0, i, j, k), Ey = ldv(g, v, 4, q.c0, i, j, k);
    T Ez = ldv(g, v, 5, q.c0, i, j, k);
    T Ez_jp = ldv(g, v, 5, q.cjp, i, jp, k), Ey_kp = ldv(g, v, 4, q.ckp, i, j, kp);
    T Ex_kp = ldv(g, v, 3, q.ckp, i, j, kp), Ez_ip = ldv(g, v, 5, q.cip, ip, j, k);
    T Ey_ip = ldv(g, v, 4, q.cip, ip, j, k), Ex_jp = ldv(g, v, 3, q.cjp, i, jp, k);
    const T Hz_jm = ldv(g, v, 2, q.cjm, i, jm, k), Hy_km = ldv(g, v, 1, q.ckm, i, j, km);
    const T Hx_km = ldv(g, v, 0, q.ckm, i, j, km), Hz_im = ldv(g, v, 2, q.cim, im, j, k);
    const T Hy_im = ldv(g, v, 1, q.cim, im, j, k), Hx_jm = ldv(g, v, 0, q.cjm, i, jm, k);
    T s[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) s[c] = sig_of(g, sig2, q, c);
    const T cHx = (Hz - Hz_jm) - (Hy - Hy_km);
    const T cHy = (Hx - Hx_km) - (Hz - Hz_im);
    const T cHz = (Hy - Hy_im) - (Hx - Hx_jm);
    if (!TR) {
      out[0] = s[0] * Hx + ((Ez_jp - Ez) - (Ey_kp - Ey));
      out[1] = s[1] * Hy + ((Ex_kp - Ex) - (Ez_ip - Ez));
      out[2] = s[2] * Hz + ((Ey_ip - Ey) - (Ex_jp - Ex));
      out[3] = ie[q.c0] * (s[3] * Ex - cHx);
      out[4] = ie[nc + q.c0] * (s[4] * Ey - cHy);
      out[5] = ie[2 * nc + q.c0] * (s[5] * Ez - cHz);
    } else {
      Ex *= ie[q.c0];
      Ey *= ie[nc + q.c0];
      Ez *= ie[2 * nc + q.c0];
      Ez_jp *= ie[2 * nc + q.cjp];
      Ey_kp *= ie[nc + q.ckp];
      Ex_kp *= ie[q.ckp];
      Ez_ip *= ie[2 * nc + q.cip];
      Ey_ip *= ie[nc + q.cip];
      Ex_jp *= ie[q.cjp];
      out[0] = s[0] * Hx - ((Ez_jp - Ez) - (Ey_kp - Ey));
      out[1] = s[1] * Hy - ((Ex_kp - Ex) - (Ez_ip - Ez));
      out[2] = s[2] * Hz - ((Ey_ip - Ey) - (Ex_jp - Ex));
      out[3] = s[3] * Ex + cHx;
      out[4] = s[4] * Ey + cHy;
      out[5] = s[5] * Ez + cHz;
    }
  }
  constexpr int NC = DIM == 2 ? 3 : 6;
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (is_wall(g, c, i, j, k)) out[c] = T(0);
}

// ---------------------------------------------------------------------------
// Material set-up: 1/eps on E nodes (mean over the cells whose closure holds
// the node) and the conductivity table sigma(2*index + half) on the layer axis.
template <typename T>
__global__ void k_setup_inv_eps(Geo g, const double* __restrict__ eps, T* __restrict__ ie) {
  const int64_t nc = g.ncell;
  const int nE = g.ncomp - g.nh;
  const int64_t nxy = (int64_t)g.nx * g.ny;
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nE * nc;
       t += (int64_t)gridDim.x * blockDim.x) {
    const int e = (int)(t / nc);
    const int64_t cell = t % nc;
    const Cell q = make_cell(g, cell);
    // E component e: half-integer along axis e (3D) / no axis (2D Ez); the
    // node touches cells index-1 and index along every integer axis.
    int half[3] = {0, 0, 0};
    if (g.dim == 3) half[e] = 1;
    double acc = 0.0;
    int cnt = 0;
    for (int dz = 0; dz <= ((g.dim == 3 && !half[2]) ? 1 : 0); ++dz)
      for (int dy = 0; dy <= (half[1] ? 0 : 1); ++dy)
        for (int dx = 0; dx <= (half[0] ? 0 : 1); ++dx) {
          const int ii = dx ? q.im : q.i;
          const int jj = dy ? q.jm : q.j;
          const int kk = dz ? q.km : q.k;
          acc += eps[((int64_t)kk * g.ny + jj) * g.nx + ii];
          ++cnt;
        }
    (void)nxy;
    ie[t] = (T)((double)cnt / acc);
  }
}

template <typename T>
__global__ void k_setup_sig(T* sig2, int n, int L, double smax) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * n) return;
  const double pos = 0.5 * t;
  double d = fmax(fmax((double)L - pos, pos - (double)(n - L)), 0.0);
  sig2[t] = (T)(smax * d / (double)L);
}

kx_status launch_setup_material(kx_ctx* c) {
  const Geo& g = c->geo;
  const int nE = g.ncomp - g.nh;
  const int64_t tot = nE * g.ncell;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 65535);
  const int nla = g.la == 0 ? g.nx : (g.la == 1 ? g.ny : g.nz);
  if (c->d.precision == KX_FP64) {
    k_setup_inv_eps<double><<<blocks, 256, 0, c->stream>>>(g, c->d_eps_cell, (double*)c->d_inv_eps);
    KX_CHECK_LAUNCH(c);
    k_setup_sig<double><<<(2 * nla + 255) / 256, 256, 0, c->stream>>>(
        (double*)c->d_sig2, nla, c->d.layer_cells, c->d.sigma_max);
  } else {
    k_setup_inv_eps<float><<<blocks, 256, 0, c->stream>>>(g, c->d_eps_cell, (float*)c->d_inv_eps);
    KX_CHECK_LAUNCH(c);
    k_setup_sig<float><<<(2 * nla + 255) / 256, 256, 0, c->stream>>>(
        (float*)c->d_sig2, nla, c->d.layer_cells, c->d.sigma_max);
  }
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// Plain operator application.
template <typename T, int DIM, int TR>
__global__ void __launch_bounds__(NTHREADS) k_apply(Geo g, const T* __restrict__ v, T* __restrict__ w,
                                                   const T* __restrict__ ie, const T* __restrict__ sig2) {
  constexpr int NC = DIM == 2 ? 3 : 6;
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < g.ncell;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const Cell q = make_cell(g, cell);
    T o[NC];
    stencil<T, DIM, TR>(g, v, ie, sig2, q, o);
#pragma unroll
    for (int c = 0; c < NC; ++c) w[(int64_t)c * g.ncell + cell] = o[c];
  }
}

template <typename T>
static kx_status apply_t(kx_ctx* c, const void* v, void* w, int tr) {
  const Geo& g = c->geo;
  const int blocks = (int)std::min<int64_t>((g.ncell + NTHREADS - 1) / NTHREADS, (int64_t)c->nblk * 4);
  const T* ie = (const T*)c->d_inv_eps;
  const T* sg = (const T*)c->d_sig2;
  if (g.dim == 2) {
    if (tr) k_apply<T, 2, 1><<<blocks, NTHREADS, 0, c->stream>>>(g, (const T*)v, (T*)w, ie, sg);
    else k_apply<T, 2, 0><<<blocks, NTHREADS, 0, c->stream>>>(g, (const T*)v, (T*)w, ie, sg);
  } else {
    if (tr) k_apply<T, 3, 1><<<blocks, NTHREADS, 0, c->stream>>>(g, (const T*)v, (T*)w, ie, sg);
    else k_apply<T, 3, 0><<<blocks, NTHREADS, 0, c->stream>>>(g, (const T*)v, (T*)w, ie, sg);
  }
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// Algorithmic bytes: read v, write w, read 1/eps on the E nodes.
kx_status launch_apply(kx_ctx* c, const void* v, void* w, int transpose) {
  const double bytes = 2.0 * c->n * c->esize + (double)(c->geo.ncomp - c->geo.nh) * c->geo.ncell * c->esize;
  time_begin(c);
  const kx_status st = c->d.precision == KX_FP64 ? apply_t<double>(c, v, w, transpose)
                                                 : apply_t<float>(c, v, w, transpose);
  time_end(c, KX_K_APPLY, bytes);
  return st;
}

// ---------------------------------------------------------------------------
// Deterministic grid reduction helpers.
template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Returns true in every thread of the last block to finish.
__device__ __forceinline__ bool last_block(unsigned* counter) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned t = atomicAdd(counter, 1u);
    am_last = (t == gridDim.x - 1);
  }
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// ---------------------------------------------------------------------------
// Arnoldi pass A (step j -> column j+1, Sect. 3.2 eq. (Arn)):
//   w = A v_j  (v_j = scale[j] * V_j)       [augmented: w = [A y - (a/eta) g; -W b; W a]]
//   d_i = V_i^T w for i <= j, and ||w||^2, fused in one sweep over the cells.
// The last block forms H[i, j] = scale[i] * d_i.
template <typename T, int DIM, int AUG>
__global__ void __launch_bounds__(NTHREADS) k_pass_a(Geo g, Slot<T> s, int j, int64_t ld, int ldh,
                                                    const T* __restrict__ ie,
                                                    const T* __restrict__ sig2,
                                                    const T* __restrict__ gsrc) {
  constexpr int NC = DIM == 2 ? 3 : 6;
  if (s.st->done) return;
  __shared__ double acc[NWARPS][MMAX + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < NWARPS * (MMAX + 2); q += blockDim.x) (&acc[0][0])[q] = 0.0;
  __syncthreads();
  const double sj = s.scale[j];
  const T tsj = (T)sj;
  const T* __restrict__ vin = s.V + (int64_t)j * ld;
  T* __restrict__ wout = s.V + (int64_t)(j + 1) * ld;
  T gco = T(0);
  if (AUG) gco = (T)(-(sj * s.aug[2 * j]) / s.st->eta);
  const int ncol = j + 1;
  const int64_t nc = g.ncell;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nc;
       base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = base + threadIdx.x;
    const bool act = cell < nc;
    T o[NC];
    if (act) {
      const Cell q = make_cell(g, cell);
      stencil<T, DIM, 0>(g, vin, ie, sig2, q, o);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        o[c] *= tsj;
        if (AUG) {
          if (!is_wall(g, c, q.i, q.j, q.k)) o[c] += gco * gsrc[(int64_t)c * nc + cell];
        }
        wout[(int64_t)c * nc + cell] = o[c];
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) o[c] = T(0);
    }
    T nrm = T(0);
#pragma unroll
    for (int c = 0; c < NC; ++c) nrm += o[c] * o[c];
    for (int c0 = 0; c0 < ncol; c0 += 8) {
      T p[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        p[t] = T(0);
        const int col = c0 + t;
        if (act && col < ncol) {
          const T* __restrict__ vc = s.V + (int64_t)col * ld + cell;
#pragma unroll
          for (int c = 0; c < NC; ++c) p[t] += vc[(int64_t)c * nc] * o[c];
        }
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) p[t] = warp_sum(p[t]);
      if (lane == 0) {
#pragma unroll
        for (int t = 0; t < 8; ++t)
          if (c0 + t < ncol) acc[warp][c0 + t] += (double)p[t];
      }
    }
    nrm = warp_sum(nrm);
    if (lane == 0) acc[warp][MMAX + 1] += (double)nrm;
  }
  __syncthreads();
  for (int col = threadIdx.x; col < MMAX + 2; col += blockDim.x) {
    if (col < ncol || col == MMAX + 1) {
      double t = 0.0;
#pragma unroll
      for (int w = 0; w < NWARPS; ++w) t += acc[w][col];
      s.part[(int64_t)blockIdx.x * PST + col] = t;
    }
  }
  if (!last_block(s.counter)) return;
  __shared__ double tot[MMAX + 2];
  for (int col = threadIdx.x; col < MMAX + 2; col += blockDim.x) {
    if (col < ncol || col == MMAX + 1) {
      double t = 0.0;
      for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(&s.part[(int64_t)b * PST + col]);
      tot[col] = t;
    }
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    *s.counter = 0u;
    double nrm2 = tot[MMAX + 1];
    if (AUG) {
      // augmented entries of w = scale_j * [-W b_j, W a_j]
      const double W = s.st->omega;
      const double wa = -W * sj * s.aug[2 * j + 1];
      const double wb = W * sj * s.aug[2 * j];
      s.aug[2 * (j + 1)] = wa;
      s.aug[2 * (j + 1) + 1] = wb;
      for (int col = 0; col < ncol; ++col)
        tot[col] += s.aug[2 * col] * wa + s.aug[2 * col + 1] * wb;
      nrm2 += wa * wa + wb * wb;
    }
    bool finite = isfinite(nrm2);
    for (int col = 0; col < ncol; ++col) {
      const double h = s.scale[col] * tot[col];
      finite = finite && isfinite(h);
      s.H[col + (int64_t)j * ldh] = h;
    }
    const double wn = sqrt(nrm2);
    if (wn > s.st->wmax) s.st->wmax = wn;
    s.part[(int64_t)gridDim.x * PST] = nrm2;  // ||w||^2 for pass B
    if (!finite) {
      s.st->status = KX_ENONFINITE;
      s.st->done = 1;
    }
  }
}

template <typename T>
static kx_status pass_a_t(kx_ctx* c, int slot, int j, const void* gaug) {
  const Geo& g = c->geo;
  const int m = c->m;
  Slot<T> s = make_slot<T>(c, slot);
  const T* ie = (const T*)c->d_inv_eps;
  const T* sg = (const T*)c->d_sig2;
  const T* gs = (const T*)gaug;
  const int ldh = m + 1;
  if (g.dim == 2) {
    if (gaug) k_pass_a<T, 2, 1><<<c->nblk, NTHREADS, 0, c->stream>>>(g, s, j, c->ld, ldh, ie, sg, gs);
    else k_pass_a<T, 2, 0><<<c->nblk, NTHREADS, 0, c->stream>>>(g, s, j, c->ld, ldh, ie, sg, gs);
  } else {
    if (gaug) k_pass_a<T, 3, 1><<<c->nblk, NTHREADS, 0, c->stream>>>(g, s, j, c->ld, ldh, ie, sg, gs);
    else k_pass_a<T, 3, 0><<<c->nblk, NTHREADS, 0, c->stream>>>(g, s, j, c->ld, ldh, ie, sg, gs);
  }
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// Algorithmic bytes of pass A at step j: read v_j and V_0..V_{j-1} (j+1
// vectors), write w (1), read 1/eps on the E nodes, and g when augmented.
kx_status launch_pass_a(kx_ctx* c, int slot, int j, const void* g_aug) {
  const double vb = (double)c->n * c->esize;
  const double bytes = (j + 2) * vb + (double)(c->geo.ncomp - c->geo.nh) * c->geo.ncell * c->esize +
                       (g_aug ? vb : 0.0);
  time_begin(c);
  const kx_status st = c->d.precision == KX_FP64 ? pass_a_t<double>(c, slot, j, g_aug)
                                                 : pass_a_t<float>(c, slot, j, g_aug);
  time_end(c, KX_K_PASS_A, bytes);
  return st;
}

}  // namespace kx
