// Yee-grid operator A of eq. (ode) and the fused Arnoldi pass A.
//
// A = diag(M_mu, M_eps)^{-1} [[M_sigma, K], [-K^T, M_sigma]]   (Sect. 2.1)
//   H rows:  sigma H + curl E            (mu_r = 1)
//   E rows:  (sigma E - curl H) / eps
// K is the forward-difference curl of E on the H nodes and K^T the
// backward-difference curl of H on the E nodes.  One thread owns one cell
// (all 3 or 6 components of that cell), which keeps the neighbour planes of
// a block close in time and the reuse inside L1/L2.
#include <atomic>

#include "kx_internal.cuh"
#include "kx_reduce.cuh"
#include "kx_stencil.cuh"

namespace kx {

// ---------------------------------------------------------------------------
// Material set-up: 1/eps on E nodes (mean over the cells whose closure holds
// the node) and the conductivity table sigma(2*index + half) on the layer axis.
template <typename T>
__global__ void k_setup_inv_eps(Geo g, const double* __restrict__ eps, T* __restrict__ ie) {
  const int64_t nc = g.ncell;
  const int nE = g.ne;
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

// Per-cell permittivity from a material id per cell and a table of the
// materials' permittivities.  An id outside the table flags *bad and leaves
// that cell at 1 (the caller then refuses the context).
__global__ void k_expand_materials(int64_t ncell, const uint8_t* __restrict__ id, const double* __restrict__ table,
                                   int n_mat, double* __restrict__ eps, int* bad) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < ncell; t += (int64_t)gridDim.x * blockDim.x) {
    const int k = id[t];
    if (k < n_mat) {
      eps[t] = table[k];
    } else {
      eps[t] = 1.0;
      *bad = 1;
    }
  }
}

kx_status launch_expand_materials(kx_ctx* c, const uint8_t* d_id, const double* d_table, int n_mat, int* d_bad) {
  const int64_t blocks = std::min<int64_t>((c->geo.ncell + 255) / 256, (int64_t)c->nsm * 16);
  k_expand_materials<<<(int)blocks, 256, 0, c->stream>>>(c->geo.ncell, d_id, d_table, n_mat, c->d_eps_cell, d_bad);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// Lossy layer: linear ramp sigma_max d / L; PML: quadratic sigma_max (d/L)^2
// (Sect. 4.1).
template <typename T>
__global__ void k_setup_sig(T* sig2, int n, int L, double smax, int quad) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 2 * n) return;
  const double pos = 0.5 * t;
  const double r = fmax(fmax((double)L - pos, pos - (double)(n - L)), 0.0) / (double)L;
  sig2[t] = (T)(smax * (quad ? r * r : r));
}

kx_status launch_setup_material(kx_ctx* c) {
  const Geo& g = c->geo;
  const int nE = g.ne;
  const int64_t tot = nE * g.ncell;
  const int blocks = (int)std::min<int64_t>((tot + 255) / 256, 65535);
  const int nla = g.la == 0 ? g.nx : (g.la == 1 ? g.ny : g.nz);
  if (c->d.precision == KX_FP64) {
    k_setup_inv_eps<double><<<blocks, 256, 0, c->stream>>>(g, c->d_eps_cell, (double*)c->d_inv_eps);
    KX_CHECK_LAUNCH(c);
    k_setup_sig<double><<<(2 * nla + 255) / 256, 256, 0, c->stream>>>(
        (double*)c->d_sig2, nla, c->d.layer_cells, c->d.sigma_max, g.pml);
  } else {
    k_setup_inv_eps<float><<<blocks, 256, 0, c->stream>>>(g, c->d_eps_cell, (float*)c->d_inv_eps);
    KX_CHECK_LAUNCH(c);
    k_setup_sig<float><<<(2 * nla + 255) / 256, 256, 0, c->stream>>>(
        (float*)c->d_sig2, nla, c->d.layer_cells, c->d.sigma_max, g.pml);
  }
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// ---------------------------------------------------------------------------
// Plain operator application.
template <typename T, int DIM, int TR>
__global__ void __launch_bounds__(NTHREADS) k_apply(Geo g, const T* __restrict__ v, T* __restrict__ w,
                                                   const T* __restrict__ ie, const T* __restrict__ sig2) {
  constexpr int NC = ncomp_of(DIM);
  for (int64_t cell = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; cell < g.ncell;
       cell += (int64_t)gridDim.x * blockDim.x) {
    const Cell q = make_cell(g, cell);
    T o[NC];
    stencil<T, DIM, TR>(g, v, TableMat<T>{ie, sig2}, q, o);
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
  if (g.dim == 2 && g.pml) {
    if (tr) k_apply<T, 4, 1><<<blocks, NTHREADS, 0, c->stream>>>(g, (const T*)v, (T*)w, ie, sg);
    else k_apply<T, 4, 0><<<blocks, NTHREADS, 0, c->stream>>>(g, (const T*)v, (T*)w, ie, sg);
  } else if (g.dim == 2) {
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
  const double bytes = 2.0 * c->n * c->esize + (double)c->geo.ne * c->geo.ncell * c->esize;
  time_begin(c);
  const kx_status st = c->d.precision == KX_FP64 ? apply_t<double>(c, v, w, transpose)
                                                 : apply_t<float>(c, v, w, transpose);
  time_end(c, KX_K_APPLY, bytes);
  return st;
}

// ---------------------------------------------------------------------------
// Arnoldi pass A (step j -> column j+1, Sect. 3.2 eq. (Arn)):
//   w = A v_j  (v_j = scale[j] * V_j)       [augmented: w = [A y - (a/eta) g; -W b; W a]]
//   d_i = V_i^T w for i <= j, and ||w||^2, fused in one sweep over the cells.
// The last block forms H[i, j] = scale[i] * d_i.
template <typename T, int DIM, int AUG, typename Mat, int TR = 0>
__global__ void __launch_bounds__(NTHREADS) k_pass_a(Geo g, SlotSet<T> ss, int j, int64_t ld, Mat mat,
                                                    const T* __restrict__ gsrc, int ldh, int nbb, double btol) {
  pdl_enter();
  constexpr int NC = ncomp_of(DIM);
  const Slot<T> s = slot_at(ss, blockIdx.y);
  if (s.st->done || s.st->retired) return;
  __shared__ double acc[NWARPS][MMAX + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < NWARPS * (MMAX + 2); q += blockDim.x) (&acc[0][0])[q] = 0.0;
  __syncthreads();
  // step j-1's pass B is finalised here when nbb > 0 (no separate kernel)
  double sj;
  if (nbb > 0) {
    if (!fin_prev_b(s, j, ldh, nbb, btol, &sj)) return;
  } else {
    sj = s.scale[j];
  }
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
      stencil<T, DIM, TR>(g, vin, mat, q, o);
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
  // block partials: columns 0..j are the dots, column j+1 is ||w||^2
  for (int col = threadIdx.x; col <= ncol; col += blockDim.x) {
    const int src = col < ncol ? col : MMAX + 1;
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) t += acc[w][src];
    s.part[(int64_t)col * s.ps + blockIdx.x] = t;
  }
}

// ---------------------------------------------------------------------------
// Pass A, 3D FP32, four consecutive x-cells per thread (nx % 4 == 0): every
// field, 1/eps and basis access is one 16-byte load (helpers in
// kx_stencil.cuh), and the dots of a chunk of 8 basis columns keep 48 such
// loads in flight per thread.  The stencil is written out here rather than
// through stencil_quad32: interleaved with the scaling it needs fewer
// registers.  Its index arithmetic is 32-bit (ncell < 2^31).

// The body of pass A in its quad form; two kernels below instantiate it.
template <int AUG>
__device__ __forceinline__ void pass_a4_body(Geo g, SlotSet<float> ss, int j, int64_t ld,
                                             const float* __restrict__ ie,
                                             const float* __restrict__ sig2,
                                             const float* __restrict__ gsrc, int ldh, int nbb,
                                             double btol) {
  pdl_enter();
  const Slot<float> s = slot_at(ss, blockIdx.y);
  if (s.st->done || s.st->retired) return;
  __shared__ double acc[NWARPS][MMAX + 2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < NWARPS * (MMAX + 2); q += blockDim.x) (&acc[0][0])[q] = 0.0;
  __syncthreads();
  double sj;
  if (nbb > 0) {
    if (!fin_prev_b(s, j, ldh, nbb, btol, &sj)) return;
  } else {
    sj = s.scale[j];
  }
  const float tsj = (float)sj;
  const float* __restrict__ v = s.V + (int64_t)j * ld;
  float* __restrict__ wout = s.V + (int64_t)(j + 1) * ld;
  float gco = 0.f;
  if (AUG) gco = (float)(-(sj * s.aug[2 * j]) / s.st->eta);
  const int ncol = j + 1;
  const int64_t nc = g.ncell;
  const int64_t nq = nc >> 2;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nq; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q4 = base + threadIdx.x;
    const bool act = q4 < nq;
    float4 o[6];
    if (act) {
      // 32-bit index arithmetic (ncell < 2^31) and the wall tests as
      // per-component bit masks, as in stencil_quad32
      const int c0 = (int)(q4 << 2);
      const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
      const unsigned r = (unsigned)c0 / (unsigned)nx;
      const int i0 = c0 - (int)r * nx;
      const unsigned kq = r / (unsigned)ny;
      const int jj = (int)r - (int)kq * ny, kk = (int)kq;
      const int jp = (jj + 1 == ny) ? 0 : jj + 1, jm = (jj == 0) ? ny - 1 : jj - 1;
      const int kp = (kk + 1 == nz) ? 0 : kk + 1, km = (kk == 0) ? nz - 1 : kk - 1;
      const int cjp = c0 + (jp - jj) * nx, cjm = c0 + (jm - jj) * nx;
      const int ckp = c0 + (kp - kk) * nxy, ckm = c0 + (km - kk) * nxy;
      const int ixp = (i0 + 4 == nx) ? 0 : i0 + 4;     // first element of the next quad
      const int ixm = (i0 == 0) ? nx - 1 : i0 - 1;     // element before the quad
      const int cxp = c0 - i0 + ixp, cxm = c0 - i0 + ixm;
      const unsigned xm = wall_bits(g, 0), ym = wall_bits(g, 1), zm = wall_bits(g, 2);
      const unsigned wx0 = i0 == 0 ? xm : 0u, wy = jj == 0 ? ym : 0u, wz = kk == 0 ? zm : 0u;
      const unsigned wyp = jp == 0 ? ym : 0u, wym = jm == 0 ? ym : 0u, wzp = kp == 0 ? zm : 0u;
      const unsigned wzm = km == 0 ? zm : 0u;
      const unsigned o0 = wx0 | wy | wz, o1 = wy | wz;   // the quad's first cell / the other three
      const float4 Hx = ldw4(v, c0, o0, o1, 0), Hy = ldw4(v + nc, c0, o0, o1, 1);
      const float4 Hz = ldw4(v + 2 * nc, c0, o0, o1, 2), Ex = ldw4(v + 3 * nc, c0, o0, o1, 3);
      const float4 Ey = ldw4(v + 4 * nc, c0, o0, o1, 4), Ez = ldw4(v + 5 * nc, c0, o0, o1, 5);
      const float4 Ez_jp = ldw4(v + 5 * nc, cjp, wx0 | wyp | wz, wyp | wz, 5);
      const float4 Ex_jp = ldw4(v + 3 * nc, cjp, wx0 | wyp | wz, wyp | wz, 3);
      const float4 Ey_kp = ldw4(v + 4 * nc, ckp, wx0 | wy | wzp, wy | wzp, 4);
      const float4 Ex_kp = ldw4(v + 3 * nc, ckp, wx0 | wy | wzp, wy | wzp, 3);
      const float4 Hz_jm = ldw4(v + 2 * nc, cjm, wx0 | wym | wz, wym | wz, 2);
      const float4 Hx_jm = ldw4(v, cjm, wx0 | wym | wz, wym | wz, 0);
      const float4 Hy_km = ldw4(v + nc, ckm, wx0 | wy | wzm, wy | wzm, 1);
      const float4 Hx_km = ldw4(v, ckm, wx0 | wy | wzm, wy | wzm, 0);
      const unsigned wxp = (ixp == 0 ? xm : 0u) | wy | wz, wxm = (ixm == 0 ? xm : 0u) | wy | wz;
      const float Ez_n = ldw(v + 5 * nc, cxp, wxp, 5), Ey_n = ldw(v + 4 * nc, cxp, wxp, 4);
      const float Hz_p = ldw(v + 2 * nc, cxm, wxm, 2), Hy_p = ldw(v + nc, cxm, wxm, 1);
      const float4 ie0 = ld4(ie + c0), ie1 = ld4(ie + nc + c0), ie2 = ld4(ie + 2 * nc + c0);
      float4 g4[6];
      if (AUG) {
#pragma unroll
        for (int c = 0; c < 6; ++c) g4[c] = ldw4(gsrc + c * nc, c0, o0, o1, c);
      }
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int li = g.la == 0 ? i0 + e : (g.la == 1 ? jj : kk);
        float sg[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) sg[c] = sig2[2 * li + g.sighalf[c]];
        const float ez = f4(Ez, e), ey = f4(Ey, e), ex = f4(Ex, e);
        const float hx = f4(Hx, e), hy = f4(Hy, e), hz = f4(Hz, e);
        const float ez_ip = e < 3 ? f4(Ez, e + 1) : Ez_n;
        const float ey_ip = e < 3 ? f4(Ey, e + 1) : Ey_n;
        const float hz_im = e > 0 ? f4(Hz, e - 1) : Hz_p;
        const float hy_im = e > 0 ? f4(Hy, e - 1) : Hy_p;
        const float cHx = (hz - f4(Hz_jm, e)) - (hy - f4(Hy_km, e));
        const float cHy = (hx - f4(Hx_km, e)) - (hz - hz_im);
        const float cHz = (hy - hy_im) - (hx - f4(Hx_jm, e));
        float out[6];
        out[0] = sg[0] * hx + ((f4(Ez_jp, e) - ez) - (f4(Ey_kp, e) - ey));
        out[1] = sg[1] * hy + ((f4(Ex_kp, e) - ex) - (ez_ip - ez));
        out[2] = sg[2] * hz + ((ey_ip - ey) - (f4(Ex_jp, e) - ex));
        out[3] = f4(ie0, e) * (sg[3] * ex - cHx);
        out[4] = f4(ie1, e) * (sg[4] * ey - cHy);
        out[5] = f4(ie2, e) * (sg[5] * ez - cHz);
        const unsigned me = e == 0 ? o0 : o1;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          float x = (me >> c) & 1u ? 0.f : out[c] * tsj;
          if (AUG) x += gco * f4(g4[c], e);
          set4(o[c], e, x);
        }
      }
#pragma unroll
      for (int c = 0; c < 6; ++c) *reinterpret_cast<float4*>(wout + c * nc + c0) = o[c];
    } else {
#pragma unroll
      for (int c = 0; c < 6; ++c) o[c] = make_float4(0.f, 0.f, 0.f, 0.f);
    }
    float nrm = 0.f;
#pragma unroll
    for (int c = 0; c < 6; ++c) nrm += dot4(o[c], o[c]);
    const int64_t cq = act ? (q4 << 2) : 0;
    for (int cb = 0; cb < ncol; cb += 8) {
      float p[8];
#pragma unroll
      for (int t = 0; t < 8; ++t) {
        p[t] = 0.f;
        const int col = cb + t;
        if (act && col < ncol) {
          const float* __restrict__ vc = s.V + (int64_t)col * ld + cq;
#pragma unroll
          for (int c = 0; c < 6; ++c) p[t] += dot4(ld4(vc + c * nc), o[c]);
        }
      }
#pragma unroll
      for (int t = 0; t < 8; ++t) p[t] = warp_sum(p[t]);
      if (lane < 8 && cb + lane < ncol) {
        float mine = p[0];
#pragma unroll
        for (int t = 1; t < 8; ++t) if (lane == t) mine = p[t];
        acc[warp][cb + lane] += (double)mine;
      }
    }
    nrm = warp_sum(nrm);
    if (lane == 0) acc[warp][MMAX + 1] += (double)nrm;
  }
  __syncthreads();
  for (int col = threadIdx.x; col <= ncol; col += blockDim.x) {
    const int src = col < ncol ? col : MMAX + 1;
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) t += acc[w][src];
    s.part[(int64_t)col * s.ps + blockIdx.x] = t;
  }
}

// Unconstrained registers (95, two resident blocks per SM), for grids the
// work limits: 64^3 has 256 blocks of work.
template <int AUG>
__global__ void __launch_bounds__(NTHREADS) k_pass_a4(Geo g, SlotSet<float> ss, int j, int64_t ld,
                                                     const float* __restrict__ ie, const float* __restrict__ sig2,
                                                     const float* __restrict__ gsrc, int ldh, int nbb, double btol) {
  pass_a4_body<AUG>(g, ss, j, ld, ie, sig2, gsrc, ldh, nbb, btol);
}

// Three resident blocks per SM (at most 85 registers a thread), for work
// that fills the GPU: at 128^3 the pass ran at 80 % of the measured copy
// bandwidth with two blocks and at 94 % with three.
template <int AUG>
__global__ void __launch_bounds__(NTHREADS, 3) k_pass_a4_dense(Geo g, SlotSet<float> ss, int j, int64_t ld,
                                                              const float* __restrict__ ie,
                                                              const float* __restrict__ sig2,
                                                              const float* __restrict__ gsrc, int ldh, int nbb,
                                                              double btol) {
  pass_a4_body<AUG>(g, ss, j, ld, ie, sig2, gsrc, ldh, nbb, btol);
}

// ---------------------------------------------------------------------------
// Finalisation of pass A, one block per column c <= j+1: sum the block
// partials of column c in a fixed order; columns c <= j give
// H[c, j] = scale[c] * d_c (plus the augmented entries' share), column j+1
// gives ||w|| (breakdown scale) and the augmented entries of w.
__global__ void __launch_bounds__(NTHREADS) k_fin_a(SlotSet<float> ss, int j, int ldh, int nb, int aug) {
  pdl_enter();
  const Slot<float> sl = slot_at(ss, blockIdx.y);
  double* part = sl.part;
  const int ps = sl.ps;
  double* H = sl.H;
  double* scale = sl.scale;
  double* augv = sl.aug;
  SlotState* st = sl.st;
  if (st->done || st->retired) return;
  const int col = blockIdx.x;
  const int ncol = j + 1;
  double x = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) x += __ldcg(part + (int64_t)col * ps + b);
  __shared__ double red[NWARPS];
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x != 0) return;
  double tot = 0.0;
#pragma unroll
  for (int w = 0; w < NWARPS; ++w) tot += red[w];
  const double sj = scale[j];
  double wa = 0.0, wb = 0.0;
  if (aug) {
    const double W = st->omega;
    wa = -W * sj * augv[2 * j + 1];
    wb = W * sj * augv[2 * j];
  }
  if (col < ncol) {
    if (aug) tot += augv[2 * col] * wa + augv[2 * col + 1] * wb;
    const double h = scale[col] * tot;
    H[col + (int64_t)j * ldh] = h;
    if (!isfinite(h)) { st->status = KX_ENONFINITE; st->done = 1; }
  } else {
    // the augmented entries of w (zero when the operator is not augmented,
    // so no stale entries of an earlier augmented run reach pass B)
    augv[2 * (j + 1)] = wa;
    augv[2 * (j + 1) + 1] = wb;
    if (aug) tot += wa * wa + wb * wb;
    const double wn = sqrt(tot);
    if (!isfinite(wn)) { st->status = KX_ENONFINITE; st->done = 1; }
    if (wn > st->wmax) st->wmax = wn;
  }
}

// Lucky-breakdown threshold relative to max ||A v_i||, by vector precision.
template <typename T>
constexpr double btol_of() { return sizeof(T) == 8 ? 1e-12 : 1e-6; }

template <typename T>
static kx_status pass_a_t(kx_ctx* c, int slot, int ns, int j, const void* gaug) {
  const Geo& g = c->geo;
  const int m = c->m;
  SlotSet<T> s = make_slotset<T>(c, slot);
  const T* ie = (const T*)c->d_inv_eps;
  const T* sg = (const T*)c->d_sig2;
  const T* gs = (const T*)gaug;
  const int ldh = m + 1;
  // the quad kernel needs 16-byte aligned rows of every array it reads
  const bool vec4 = sizeof(T) == 4 && g.dim == 3 && (g.nx % 4) == 0 &&
                    ((uintptr_t)gaug % 16) == 0 && g.ncell < ((int64_t)1 << 31);
  const int64_t items = vec4 ? g.ncell / 4 : g.ncell;
  const int64_t rounds = (items + NTHREADS - 1) / NTHREADS;
  // the quad kernel in its three-block form when the launch's work (all its
  // slots) exceeds what two resident blocks per SM cover
  const bool dense = vec4 && rounds * ns > 2 * (int64_t)c->nsm;
  static std::atomic<int> grid[5][2];
  const int kind = vec4 ? (dense ? 4 : 2) : (g.pml ? 3 : (g.dim == 3));
  std::atomic<int>& gr = grid[kind][gaug != nullptr];
  if (!gr) {
    const void* fn;
    if (vec4 && dense) fn = gaug ? (const void*)k_pass_a4_dense<1> : (const void*)k_pass_a4_dense<0>;
    else if (vec4) fn = gaug ? (const void*)k_pass_a4<1> : (const void*)k_pass_a4<0>;
    else if (g.dim == 2 && g.pml) fn = gaug ? (const void*)k_pass_a<T, 4, 1, TableMat<T>> : (const void*)k_pass_a<T, 4, 0, TableMat<T>>;
    else if (g.dim == 2) fn = gaug ? (const void*)k_pass_a<T, 2, 1, TableMat<T>> : (const void*)k_pass_a<T, 2, 0, TableMat<T>>;
    else fn = gaug ? (const void*)k_pass_a<T, 3, 1, TableMat<T>> : (const void*)k_pass_a<T, 3, 0, TableMat<T>>;
    gr = persistent_grid(c, fn, 1 << 30, 0);
  }
  const int nb = reserve_grid(c, (int)std::min<int64_t>(std::min<int64_t>(rounds, gr.load()), c->ps), gr.load());
  const dim3 grd(nb, ns);
  // a non-augmented process finalises step j-1's pass B here
  const int nbb = (j >= 1 && !gaug) ? pass_b_grid(c) : 0;
  const double bt = btol_of<T>();
  if (vec4) {
    SlotSet<float> sf = make_slotset<float>(c, slot);
    const float* ief = (const float*)c->d_inv_eps;
    const float* sgf = (const float*)c->d_sig2;
    const float* gf = (const float*)gaug;
    if (dense) {
      if (gaug) launch_k(c, k_pass_a4_dense<1>, grd, NTHREADS, 0, c->stream, g, sf, j, c->ld, ief, sgf, gf, ldh, nbb, bt);
      else launch_k(c, k_pass_a4_dense<0>, grd, NTHREADS, 0, c->stream, g, sf, j, c->ld, ief, sgf, gf, ldh, nbb, bt);
    } else {
      if (gaug) launch_k(c, k_pass_a4<1>, grd, NTHREADS, 0, c->stream, g, sf, j, c->ld, ief, sgf, gf, ldh, nbb, bt);
      else launch_k(c, k_pass_a4<0>, grd, NTHREADS, 0, c->stream, g, sf, j, c->ld, ief, sgf, gf, ldh, nbb, bt);
    }
  } else if (g.dim == 2 && g.pml) {
    if (gaug) launch_k(c, k_pass_a<T, 4, 1, TableMat<T>>, grd, NTHREADS, 0, c->stream, g, s, j, c->ld, TableMat<T>{ie, sg}, gs, ldh, nbb, bt);
    else launch_k(c, k_pass_a<T, 4, 0, TableMat<T>>, grd, NTHREADS, 0, c->stream, g, s, j, c->ld, TableMat<T>{ie, sg}, gs, ldh, nbb, bt);
  } else if (g.dim == 2) {
    if (gaug) launch_k(c, k_pass_a<T, 2, 1, TableMat<T>>, grd, NTHREADS, 0, c->stream, g, s, j, c->ld, TableMat<T>{ie, sg}, gs, ldh, nbb, bt);
    else launch_k(c, k_pass_a<T, 2, 0, TableMat<T>>, grd, NTHREADS, 0, c->stream, g, s, j, c->ld, TableMat<T>{ie, sg}, gs, ldh, nbb, bt);
  } else {
    if (gaug) launch_k(c, k_pass_a<T, 3, 1, TableMat<T>>, grd, NTHREADS, 0, c->stream, g, s, j, c->ld, TableMat<T>{ie, sg}, gs, ldh, nbb, bt);
    else launch_k(c, k_pass_a<T, 3, 0, TableMat<T>>, grd, NTHREADS, 0, c->stream, g, s, j, c->ld, TableMat<T>{ie, sg}, gs, ldh, nbb, bt);
  }
  KX_CHECK_LAUNCH(c);
  launch_k(c, k_fin_a, dim3(j + 2, ns), NTHREADS, 0, c->stream, make_slotset<float>(c, slot), j, ldh, nb,
           (int)(gaug != nullptr));
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// Pass A with the permittivity read per cell (CellMat): the variant used
// by the allocation-free entry point, which holds no 1/eps table.
template <typename T>
static kx_status pass_a_cells_t(kx_ctx* c, int slot, int j, const double* eps) {
  const Geo& g = c->geo;
  SlotSet<T> s = make_slotset<T>(c, slot);
  const CellMat<T> mat{eps, c->d.sigma_max, c->d.layer_cells};
  const int64_t rounds = (g.ncell + NTHREADS - 1) / NTHREADS;
  static std::atomic<int> grid[2];
  std::atomic<int>& gr = grid[g.dim == 3];
  if (!gr)
    gr = persistent_grid(c, g.dim == 2 ? (const void*)k_pass_a<T, 2, 0, CellMat<T>>
                                       : (const void*)k_pass_a<T, 3, 0, CellMat<T>>, 1 << 30, 0);
  const int nb = (int)std::min<int64_t>(std::min<int64_t>(rounds, gr.load()), c->ps);
  const int nbb = j >= 1 ? pass_b_grid(c) : 0;
  if (g.dim == 2)
    k_pass_a<T, 2, 0, CellMat<T>><<<nb, NTHREADS, 0, c->stream>>>(g, s, j, c->ld, mat, nullptr, c->m + 1, nbb,
                                                                  btol_of<T>());
  else
    k_pass_a<T, 3, 0, CellMat<T>><<<nb, NTHREADS, 0, c->stream>>>(g, s, j, c->ld, mat, nullptr, c->m + 1, nbb,
                                                                  btol_of<T>());
  KX_CHECK_LAUNCH(c);
  k_fin_a<<<j + 2, NTHREADS, 0, c->stream>>>(make_slotset<float>(c, slot), j, c->m + 1, nb, 0);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

// Pass A of the Arnoldi process for the transposed operator A^T (adjoint
// problem): same sweep with the transposed stencil.
template <typename T>
static kx_status pass_a_tr_t(kx_ctx* c, int slot, int ns, int j) {
  const Geo& g = c->geo;
  SlotSet<T> s = make_slotset<T>(c, slot);
  const TableMat<T> mat{(const T*)c->d_inv_eps, (const T*)c->d_sig2};
  const int64_t rounds = (g.ncell + NTHREADS - 1) / NTHREADS;
  static std::atomic<int> grid[2];
  std::atomic<int>& gr = grid[g.dim == 3];
  if (!gr)
    gr = persistent_grid(c, g.dim == 2 ? (const void*)k_pass_a<T, 2, 0, TableMat<T>, 1>
                                       : (const void*)k_pass_a<T, 3, 0, TableMat<T>, 1>, 1 << 30, 0);
  const int nb = (int)std::min<int64_t>(std::min<int64_t>(rounds, gr.load()), c->ps);
  const dim3 grd(nb, ns);
  const int nbb = j >= 1 ? pass_b_grid(c) : 0;
  if (g.dim == 2)
    k_pass_a<T, 2, 0, TableMat<T>, 1><<<grd, NTHREADS, 0, c->stream>>>(g, s, j, c->ld, mat, nullptr, c->m + 1, nbb,
                                                                       btol_of<T>());
  else
    k_pass_a<T, 3, 0, TableMat<T>, 1><<<grd, NTHREADS, 0, c->stream>>>(g, s, j, c->ld, mat, nullptr, c->m + 1, nbb,
                                                                       btol_of<T>());
  KX_CHECK_LAUNCH(c);
  k_fin_a<<<dim3(j + 2, ns), NTHREADS, 0, c->stream>>>(make_slotset<float>(c, slot), j, c->m + 1, nb, 0);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

kx_status launch_pass_a_tr(kx_ctx* c, int slot, int ns, int j) {
  const double vb = (double)c->n * c->esize;
  const double bytes = (j + 2) * vb + (double)c->geo.ne * c->geo.ncell * c->esize;
  time_begin(c);
  const kx_status st = c->d.precision == KX_FP64 ? pass_a_tr_t<double>(c, slot, ns, j)
                                                 : pass_a_tr_t<float>(c, slot, ns, j);
  time_end(c, KX_K_PASS_A, bytes * ns);
  return st;
}

kx_status launch_pass_a_cells(kx_ctx* c, int slot, int j, const double* d_eps_cell) {
  return c->d.precision == KX_FP64 ? pass_a_cells_t<double>(c, slot, j, d_eps_cell)
                                   : pass_a_cells_t<float>(c, slot, j, d_eps_cell);
}

// Algorithmic bytes of pass A at step j: read v_j and V_0..V_{j-1} (j+1
// vectors), write w (1), read 1/eps on the E nodes, and g when augmented.
kx_status launch_pass_a(kx_ctx* c, int slot, int ns, int j, const void* g_aug) {
  const double vb = (double)c->n * c->esize;
  const double bytes = (j + 2) * vb + (double)c->geo.ne * c->geo.ncell * c->esize +
                       (g_aug ? vb : 0.0);
  time_begin(c);
  const kx_status st = c->d.precision == KX_FP64 ? pass_a_t<double>(c, slot, ns, j, g_aug)
                                                 : pass_a_t<float>(c, slot, ns, j, g_aug);
  time_end(c, KX_K_PASS_A, bytes * ns);
  return st;
}

}  // namespace kx
