// Single-sweep Arnoldi process (Sect. 3.2, eqs. (Arn), (Arn1)): classical
// Gram-Schmidt arranged so that one pass over the stored basis per step
// both builds the new column and yields the dots of the next Hessenberg
// column.  The two-pass form (stencil.cu / linalg.cu) reads the basis twice
// per step, once for the dots and once for the update.
//
// Notation: stored columns V_i with scales s_i (v_i = s_i V_i, delayed
// normalisation as in the two-pass form); h_{i,j} the Hessenberg entries,
// beta_j = h_{j+1,j}.  Step j >= 1 takes two launches:
//   apply K_{j-1}: t = A V_{j-1}                       (one vector written)
//   sweep S_j    : t1 = s_{j-1} t = A v_{j-1},  t2 = A t1 = A^2 v_{j-1},
//                  x  = t1 - sum_{i<j} h_{i,j-1} v_i   (= beta_{j-1} v_j, stored as V_j)
//                  y  = A x = t2 - h_{j-1,j-1} t1 - sum_{k<j} c_k v_k,
// where the Arnoldi relation A v_i = sum_{k<=i+1} h_{k,i} v_k (i < j-1)
// gives c = H(0:j, 0:j-1) h(0:j-1, j-1).  The sweep removes the columns from
// x and y in the order i = 0 .. j-1 and, just before removing column i,
// takes the explicit dots b'_i = V_i . x^(i), a'_i = V_i . y^(i) with the
// partly reduced vectors x^(i) = t1 - sum_{k<i} h_{k,j-1} v_k (y^(i) alike);
// with the Gram matrix G_{i,k} = v_i . v_k these give
//   beta_{j-1} = ||x||,   v_j = x / beta_{j-1},
//   G_{i,j} = v_i . v_j   = (s_i b'_i - sum_{l=i}^{j-1} G_{i,l} h_{l,j-1}) / beta_{j-1},
//   h_{i,j} = v_i . A v_j = (s_i a'_i - sum_{k=i}^{j-1} G_{i,k} c_k) / beta_{j-1}   (i < j),
//   h_{j,j} = x.y / x.x,
// so Hessenberg column j is known when the sweep ends and only two vectors
// (x, y) stay live per cell.  Every vector that enters a column is an
// explicit product with the stored basis (A v_{j-1} is recomputed from
// V_{j-1}, never carried from step to step), so rounding does not
// accumulate through the relation; G carries the measured loss of
// orthogonality into the derived dots.  In exact arithmetic the process is
// classical Gram-Schmidt.
//
// Bytes per step (n unknowns, s bytes a scalar): the apply pass reads V_{j-1}
// and writes t (2 n s), the sweep reads t and V_0..V_{j-1} and writes V_j
// ((j + 2) n s), plus the 1/eps table in each: about (j + 5) n s against
// (2 j + 5) n s for the two-pass form.
#include <atomic>

#include "kx_eft.cuh"
#include "kx_internal.cuh"
#include "kx_reduce.cuh"
#include "kx_stencil.cuh"

namespace kx {

namespace {

constexpr int LG = MMAX + 1;   // leading dimension of the Gram matrix
static_assert(NTHREADS >= SWCOLS, "the finalisation stages one reduced column a thread");

// Sum over the four lanes of a row group (lanes 4r .. 4r+3) in a fixed order.
__device__ __forceinline__ double quad_sum(double x) {
  x += __shfl_xor_sync(0xffffffffu, x, 1);
  x += __shfl_xor_sync(0xffffffffu, x, 2);
  return x;
}

// Finalisation of step j, run by one whole block.
//   j == 0: tot = [V_0 . A V_0, ||A V_0||^2] (unscaled): h_{0,0}, ||A v_0||.
//   j >= 1: tot = sweep S_j's columns [a'_0..a'_{j-1}, b'_0..b'_{j-1}, x.x,
//           x.y, y.y] and uh, uc the row products of apply pass K_j:
//           beta_{j-1}, scale_j, m_done = j, the breakdown test, then
//           (unless final_step or the process stopped) G column j, H column
//           j and the coefficients of sweep S_{j+1}.
// Its inputs are first staged in shared memory in one parallel load phase
// (the step's latency is this block's chain of dependent loads); tot, uh and
// uc were written by other blocks of the same launch: read past L1.
template <typename T>
__device__ void sw_fin(const Slot<T>& s, SwCoef* co, double* G, int j, int ldh, double btol, int final_step) {
  __shared__ double sh_tot[SWCOLS], sh_u[2][MMAX], sh_sc[MMAX], sh_h[MMAX + 1];
  __shared__ double sh_H[LG * MMAX];   // the upper Hessenberg part of H(0:j, 0:j-1)
  __shared__ double sh_beta, sh_sig;
  __shared__ int sh_stop;
  SlotState* st = s.st;
  const int tid = threadIdx.x;
  if (j == 0) {
    if (tid == 0) {
      const double s0 = s.scale[0];
      const double h00 = s0 * s0 * __ldcg(&co->tot[0]);
      const double an = s0 * sqrt(__ldcg(&co->tot[1]));
      s.H[0] = h00;
      G[0] = 1.0;
      co->hc[0] = h00;
      co->cp[0] = 0.0;
      co->sprev = s0;
      co->hjj = h00;
      st->m_done = 0;
      if (!isfinite(h00) || !isfinite(an)) {
        st->status = KX_ENONFINITE;
        st->done = 1;
      } else if (an > st->wmax) {
        st->wmax = an;
      }
    }
    return;
  }
  // every load first (one L2 round trip), then the shared-memory stores;
  // blockDim.x == NTHREADS >= SWCOLS, so one reduced column a thread
  const bool full = !final_step;
  constexpr int HPER = (LG * MMAX + NTHREADS - 1) / NTHREADS;   // H entries a thread
  const int nh = full ? (j + 1) * j : 0;
  const double tv = tid < 2 * j + 3 ? __ldcg(&co->tot[tid]) : 0.0;
  double uv = 0.0, cv0 = 0.0, sv = 0.0, wm = 0.0;
  if (full && tid < j) {
    uv = __ldcg(&co->uh[tid]);
    cv0 = __ldcg(&co->uc[tid]);
    sv = s.scale[tid];
  }
  if (tid == 0) wm = st->wmax;
  // H(k, i), k <= j, i < j, nonzero for i >= k - 1 (H(j, j-1) is set below)
  double hv[HPER];
#pragma unroll
  for (int r = 0; r < HPER; ++r) {
    const int q = tid + r * NTHREADS;
    const int k = q % (j + 1), i = q / (j + 1);
    hv[r] = (q < nh && i >= k - 1 && k < j) ? s.H[k + (int64_t)i * ldh] : 0.0;
  }
  if (tid < 2 * j + 3) sh_tot[tid] = tv;
  if (full && tid < j) {
    sh_u[0][tid] = uv;
    sh_u[1][tid] = cv0;
    sh_sc[tid] = sv;
  }
#pragma unroll
  for (int r = 0; r < HPER; ++r) {
    const int q = tid + r * NTHREADS;
    if (q < nh) sh_H[(q % (j + 1)) + (q / (j + 1)) * LG] = hv[r];
  }
  __syncthreads();
  if (tid == 0) {
    const double b = sqrt(sh_tot[2 * j]);
    int stop = 0;
    double sig = 0.0;
    if (!isfinite(b)) stop = 2;
    else if (b <= btol * wm) stop = 1;   // invariant subspace: the projection is exact
    else sig = 1.0 / b;
    s.H[j + (int64_t)(j - 1) * ldh] = b;
    s.scale[j] = sig;
    st->m_done = j;
    if (stop == 2) st->status = KX_ENONFINITE;
    if (stop || abort_requested(st)) st->done = 1;
    sh_H[j + (j - 1) * LG] = b;
    sh_beta = b;
    sh_sig = sig;
    sh_stop = stop || final_step;
  }
  __syncthreads();
  if (sh_stop) return;
  const double beta = sh_beta, sig = sh_sig;
  for (int i = tid; i < j; i += blockDim.x) {
    const double gi = (sh_sc[i] * sh_tot[j + i] - sh_u[0][i]) / beta;
    const double hi = (sh_sc[i] * sh_tot[i] - sh_u[1][i]) / beta;
    G[i + (int64_t)j * LG] = gi;
    G[j + (int64_t)i * LG] = gi;
    sh_h[i] = hi;
  }
  if (tid == 0) {
    const double hjj = sig * sig * sh_tot[2 * j + 1];
    const double an = sig * sqrt(sh_tot[2 * j + 2]);
    sh_h[j] = hjj;
    G[j + (int64_t)j * LG] = 1.0;
    if (!isfinite(an)) {
      st->status = KX_ENONFINITE;
      st->done = 1;
    } else if (an > wm) {
      st->wmax = an;
    }
  }
  __syncthreads();
  for (int i = tid; i <= j; i += blockDim.x) {
    const double h = sh_h[i];
    if (!isfinite(h)) {
      st->status = KX_ENONFINITE;
      st->done = 1;
    }
    s.H[i + (int64_t)j * ldh] = h;
    co->hc[i] = h;
  }
  // c'_k = sum_{i<j} H(k, i) h_{i,j}, k <= j, four threads a row
  const int rstep = blockDim.x >> 2;
  for (int r0 = 0; r0 <= j; r0 += rstep) {
    const int row = r0 + (tid >> 2), part = tid & 3;
    double cv = 0.0;
    if (row <= j) {
      for (int i = max(row - 1, 0) + part; i < j; i += 4) cv += sh_H[row + i * LG] * sh_h[i];
    }
    cv = quad_sum(cv);
    if (row <= j && part == 0) co->cp[row] = cv;
  }
  if (tid == 0) {
    co->sprev = sig;
    co->hjj = sh_h[j];
  }
}

// Sum over b < nb of part[col * ps + b] in a fixed order, to every thread.
__device__ __forceinline__ double block_column_sum(const double* part, int ps, int col, int nb) {
  __shared__ double red[NWARPS];
  __shared__ double res;
  double x = 0.0;
  for (int b = threadIdx.x; b < nb; b += blockDim.x) x += __ldcg(part + (int64_t)col * ps + b);
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) t += red[w];
    res = t;
  }
  __syncthreads();
  return res;
}

// True in every thread of the last of `count` blocks to call it; that block
// then sees the global writes the others made before their call.
__device__ __forceinline__ bool last_of(unsigned* counter, unsigned count) {
  __shared__ bool am_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) am_last = atomicAdd(counter, 1u) == count - 1;
  __syncthreads();
  if (am_last) __threadfence();
  return am_last;
}

// Step j >= 1, in the SW_RED blocks at the front of apply pass K_j, which
// do no stencil work: sweep S_j's partial columns reduced (one warp a
// column, its lanes over the sweep's blocks in a fixed order) and the
// Gram-row products uh, uc of rows i < j (one warp a row); the last of these
// blocks finalises step j.  The stencil blocks behind them read none of it,
// so the finalisation runs beside the stencil instead of after it.
template <typename T>
__device__ __forceinline__ void sw_reduce_fin(const Slot<T>& s, const SwSlot& w, int j, int ldh, int nbs,
                                              double btol, int bid) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int gw = bid * NWARPS + warp;
  for (int col = gw; col < 2 * j + 3; col += SW_RED * NWARPS) {
    const double* p = w.part + (int64_t)col * w.ps;
    double x = 0.0;
#pragma unroll 4
    for (int b = lane; b < nbs; b += 32) x += __ldcg(p + b);
    x = warp_sum(x);
    if (lane == 0) w.co->tot[col] = x;
  }
  for (int row = gw; row < j; row += SW_RED * NWARPS) {
    double uh = 0.0, uc = 0.0;
    for (int l = row + lane; l < j; l += 32) {
      const double gil = w.G[row + (int64_t)l * LG];
      uh += gil * w.co->hc[l];
      uc += gil * w.co->cp[l];
    }
    uh = warp_sum(uh);
    uc = warp_sum(uc);
    if (lane == 0) {
      w.co->uh[row] = uh;
      w.co->uc[row] = uc;
    }
  }
  if (!last_of(&w.co->counter, (unsigned)SW_RED)) return;
  sw_fin<T>(s, w.co, w.G, j, ldh, btol, 0);
  if (threadIdx.x == 0) w.co->counter = 0u;
}

// Step 0, at the end of apply pass K_0: the block partials of its dots
// (d0 = V_0 . t, d1 = t . t); the last of the nblk blocks reduces them and
// finalises (bid: this block's index among them).
template <typename T>
__device__ __forceinline__ void sw_apply_tail0(const Slot<T>& s, const SwSlot& w, int ldh, double btol, double d0,
                                               double d1, int bid, int nblk) {
  block_partial_at(d0, w.part, w.ps, 0, bid);
  block_partial_at(d1, w.part, w.ps, 1, bid);
  if (!last_of(&w.co->counter, (unsigned)nblk)) return;
  for (int col = 0; col < 2; ++col) {
    const double x = block_column_sum(w.part, w.ps, col, nblk);
    if (threadIdx.x == 0) w.co->tot[col] = x;
  }
  __syncthreads();
  sw_fin<T>(s, w.co, w.G, 0, ldh, btol, 0);
  if (threadIdx.x == 0) w.co->counter = 0u;
}

// Apply pass K_j, any model and precision, one cell a thread: t = A V_j.
// Steps j >= 1 launch SW_RED more blocks in front, which finalise step j
// beside the stencil; step 0's finalisation follows its stencil.
template <typename T, int DIM, typename Mat>
__global__ void __launch_bounds__(NTHREADS) k_sw_apply(Geo g, Slot<T> s, SwSlot w, int j, int64_t ld, Mat mat,
                                                      int ldh, int nbs, double btol) {
  pdl_wait();
  if (s.st->done || s.st->retired) return;
  constexpr int NC = ncomp_of(DIM);
  const int R = j >= 1 ? SW_RED : 0;
  if ((int)blockIdx.x < R) {
    sw_reduce_fin<T>(s, w, j, ldh, nbs, btol, blockIdx.x);
    return;
  }
  const T* __restrict__ v = s.V + (int64_t)j * ld;
  T* __restrict__ t = (T*)w.t;
  const int64_t nc = g.ncell;
  double d0 = 0.0, d1 = 0.0;
  for (int64_t cell = (int64_t)(blockIdx.x - R) * blockDim.x + threadIdx.x; cell < nc;
       cell += (int64_t)(gridDim.x - R) * blockDim.x) {
    const Cell q = make_cell(g, cell);
    T o[NC];
    stencil<T, DIM, 0>(g, v, mat, q, o);
#pragma unroll
    for (int c = 0; c < NC; ++c) t[(int64_t)c * nc + cell] = o[c];
    if (j == 0) {
      T a = T(0), b = T(0);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        a += v[(int64_t)c * nc + cell] * o[c];
        b += o[c] * o[c];
      }
      d0 += (double)a;
      d1 += (double)b;
    }
  }
  pdl_trigger();
  if (j == 0) sw_apply_tail0<T>(s, w, ldh, btol, d0, d1, blockIdx.x, gridDim.x);
}

// Apply pass K_j, 3D FP32, one quad of x-cells a thread (nx % 4 == 0).
// Three resident blocks per SM (80 registers, a small spill): the stencil is
// latency-bound, and against two blocks (128 registers) the apply pass took
// 77 instead of 97 ms a step at 128^3 and 41.5 instead of 49 at 96^3.
// The body takes its block index among the launch's blocks for this slot
// (bid of nblk), so that one launch can serve several problems.
__device__ __forceinline__ void sw_apply4_body(const Geo& g, const Slot<float>& s, const SwSlot& w, int j, int64_t ld,
                                               const float* __restrict__ ie, const float* __restrict__ sig2, int ldh,
                                               int nbs, double btol, int bid, int nblk) {
  const int R = j >= 1 ? SW_RED : 0;
  if (bid < R) {
    sw_reduce_fin<float>(s, w, j, ldh, nbs, btol, bid);
    return;
  }
  const float* __restrict__ v = s.V + (int64_t)j * ld;
  float* __restrict__ t = (float*)w.t;
  const int64_t nc = g.ncell, nq = nc >> 2;
  double d0 = 0.0, d1 = 0.0;
  for (int64_t q4 = (int64_t)(bid - R) * blockDim.x + threadIdx.x; q4 < nq;
       q4 += (int64_t)(nblk - R) * blockDim.x) {
    const Quad qd = make_quad(g, q4);
    float4 o[6];
    stencil_quad(g, v, ie, sig2, qd, o);
#pragma unroll
    for (int c = 0; c < 6; ++c) *reinterpret_cast<float4*>(t + c * nc + qd.c0) = o[c];
    if (j == 0) {
      float a = 0.f, b = 0.f;
#pragma unroll
      for (int c = 0; c < 6; ++c) {
        a += dot4(ld4(v + c * nc + qd.c0), o[c]);
        b += dot4(o[c], o[c]);
      }
      d0 += (double)a;
      d1 += (double)b;
    }
  }
  pdl_trigger();
  if (j == 0) sw_apply_tail0<float>(s, w, ldh, btol, d0, d1, bid, nblk);
}

// Apply pass K_j for j >= 1, 3D FP32: SW_RED reducer blocks in front, then
// blocks of NTHREADS grid columns (quads of x-cells when QUAD, nx % 4 == 0),
// block b covering planes kz (b / ncb) .. kz (b / ncb + 1) - 1 of its
// columns, marching up in z (stencil_column_quad / stencil_column32: the
// index work once per column, four of the eighteen neighbour values a cell
// carried from the plane below).  Against one cell a thread with its
// per-cell index and wall arithmetic (ALU pipe at 70 % of peak), 128^3
// alone: 27-30 us (quads) and 32-35 us (cells) against 51-53 us.
template <bool QUAD>
__global__ void __launch_bounds__(NTHREADS, QUAD ? 2 : 3)
    k_sw_apply_col(Geo g, Slot<float> s, SwSlot w, int j, int64_t ld, const float* __restrict__ ie,
                   const float* __restrict__ sig2, int ldh, int nbs, double btol, int ncb, int kz) {
  pdl_wait();
  if (s.st->done || s.st->retired) return;
  if ((int)blockIdx.x < SW_RED) {
    sw_reduce_fin<float>(s, w, j, ldh, nbs, btol, blockIdx.x);
    return;
  }
  const int b = (int)blockIdx.x - SW_RED;
  const int zc = b / ncb;
  const int q = (b - zc * ncb) * NTHREADS + (int)threadIdx.x;
  const int ncol = QUAD ? (g.nx >> 2) * g.ny : g.nx * g.ny;
  const int k0 = zc * kz, k1 = min(g.nz, k0 + kz);
  if (q < ncol && k0 < k1) {
    const float* __restrict__ v = s.V + (int64_t)j * ld;
    float* __restrict__ t = (float*)w.t;
    if constexpr (QUAD)
      stencil_column_quad(g, v, ie, sig2, t, q, k0, k1);
    else
      stencil_column32(g, v, ie, sig2, t, q, k0, k1);
  }
  pdl_trigger();
}

__global__ void __launch_bounds__(NTHREADS, 3) k_sw_apply4(Geo g, Slot<float> s, SwSlot w, int j, int64_t ld,
                                                       const float* __restrict__ ie, const float* __restrict__ sig2,
                                                       int ldh, int nbs, double btol) {
  pdl_wait();
  if (s.st->done || s.st->retired) return;
  sw_apply4_body(g, s, w, j, ld, ie, sig2, ldh, nbs, btol, blockIdx.x, gridDim.x);
}

// Loads and arithmetic of CH basis columns cb .. cb+CH-1 for one cell: for
// each column the dots with the current y and x, then its removal from both.
// FULL: all CH columns exist (no per-column test).  An inactive thread
// (act false) removes nothing, so its x and y stay zero and so do its dots.
// In FP32 x is compensated (x + xl, kx_eft.cuh); in FP64 xl is unused.
template <typename T, int NC, int CH, bool FULL>
__device__ __forceinline__ void sw_columns(const T* __restrict__ V, int64_t ld, int64_t nc, int64_t cell, int cb,
                                           int j, const T* ch, const T* cc, bool act, T* x, T* xl, T* y, T* pa,
                                           T* pb) {
  T vv[CH][NC];
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    if (FULL || cb + k < j) {
      const T* __restrict__ vc = V + (int64_t)(cb + k) * ld + cell;
#pragma unroll
      for (int c = 0; c < NC; ++c) vv[k][c] = vc[(int64_t)c * nc];
    }
  }
#pragma unroll
  for (int k = 0; k < CH; ++k) {
    pa[k] = T(0);
    pb[k] = T(0);
    if (FULL || cb + k < j) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        pa[k] += vv[k][c] * y[c];
        pb[k] += vv[k][c] * x[c];
      }
      const T a = act ? ch[cb + k] : T(0), b = act ? cc[cb + k] : T(0);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        if constexpr (sizeof(T) == 4) {
          sub_fma(x[c], xl[c], -a, vv[k][c]);
        } else {
          (void)xl;
          x[c] -= a * vv[k][c];
        }
        y[c] -= b * vv[k][c];
      }
    }
  }
}

// Sweep S_j (j >= 1), any model and precision, one cell a thread.  Writes
// V_j = x and the block partials of [a'_0..a'_{j-1}, b'_0..b'_{j-1}, x.x, x.y, y.y].
template <typename T, int DIM, typename Mat>
__global__ void __launch_bounds__(NTHREADS) k_sw_pass(Geo g, Slot<T> s, SwSlot w, int j, int64_t ld, Mat mat) {
  pdl_wait();
  if (s.st->done || s.st->retired) return;
  constexpr int NC = ncomp_of(DIM);
  constexpr int CH = sizeof(T) == 4 ? 8 : 4;   // basis columns in flight per thread
  __shared__ T ch[MMAX], cc[MMAX];
  __shared__ double acc[NWARPS][SWCOLS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < NWARPS * SWCOLS; q += blockDim.x) (&acc[0][0])[q] = 0.0;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    const double sc = s.scale[i];
    ch[i] = (T)(w.co->hc[i] * sc);
    cc[i] = (T)(w.co->cp[i] * sc);
  }
  const T sp = (T)w.co->sprev, hjj = (T)w.co->hjj;
  const T spl = (T)(w.co->sprev - (double)sp);
  __syncthreads();
  const T* __restrict__ t = (const T*)w.t;
  T* __restrict__ xout = s.V + (int64_t)j * ld;
  const int64_t nc = g.ncell;
  for (int64_t base = (int64_t)blockIdx.x * blockDim.x; base < nc; base += (int64_t)gridDim.x * blockDim.x) {
    const int64_t cell = base + threadIdx.x;
    const bool act = cell < nc;
    T x[NC], xl[NC], y[NC];
    if (act) {
      const Cell q = make_cell(g, cell);
      T at[NC];
      stencil<T, DIM, 0>(g, t, mat, q, at);
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        const T tv = t[(int64_t)c * nc + cell];
        x[c] = sp * tv;
        xl[c] = sizeof(T) == 4 ? fma(spl, tv, fma(sp, tv, -x[c])) : T(0);
        y[c] = sp * at[c] - hjj * x[c];
      }
    } else {
#pragma unroll
      for (int c = 0; c < NC; ++c) x[c] = xl[c] = y[c] = T(0);
    }
    // an inactive thread reads cell 0 (in bounds), removes nothing and
    // contributes zero dots
    const int64_t cl = act ? cell : 0;
    for (int cb = 0; cb < j; cb += CH) {
      T pa[CH], pb[CH];
      if (cb + CH <= j) sw_columns<T, NC, CH, true>(s.V, ld, nc, cl, cb, j, ch, cc, act, x, xl, y, pa, pb);
      else sw_columns<T, NC, CH, false>(s.V, ld, nc, cl, cb, j, ch, cc, act, x, xl, y, pa, pb);
#pragma unroll
      for (int k = 0; k < CH; ++k) {
        pa[k] = warp_sum(pa[k]);
        pb[k] = warp_sum(pb[k]);
      }
      if (lane < CH && cb + lane < j) {
        T ma = pa[0], mb = pb[0];
#pragma unroll
        for (int k = 1; k < CH; ++k)
          if (lane == k) {
            ma = pa[k];
            mb = pb[k];
          }
        acc[warp][cb + lane] += (double)ma;
        acc[warp][j + cb + lane] += (double)mb;
      }
    }
    T xx = T(0), xy = T(0), yy = T(0);
    if (act) {
#pragma unroll
      for (int c = 0; c < NC; ++c) {
        x[c] += xl[c];   // the compensated column, rounded once (FP32; xl = 0 in FP64)
        xout[(int64_t)c * nc + cell] = x[c];
        xx += x[c] * x[c];
        xy += x[c] * y[c];
        yy += y[c] * y[c];
      }
    }
    xx = warp_sum(xx);
    xy = warp_sum(xy);
    yy = warp_sum(yy);
    if (lane == 0) {
      acc[warp][2 * j] += (double)xx;
      acc[warp][2 * j + 1] += (double)xy;
      acc[warp][2 * j + 2] += (double)yy;
    }
  }
  pdl_trigger();
  __syncthreads();
  for (int col = threadIdx.x; col < 2 * j + 3; col += blockDim.x) {
    double tsum = 0.0;
#pragma unroll
    for (int q = 0; q < NWARPS; ++q) tsum += acc[q][col];
    w.part[(int64_t)col * w.ps + blockIdx.x] = tsum;
  }
}

// ---------------------------------------------------------------------------
// Helpers of the quad sweep below: float4 halves for the packed two-lane
// FMAs, and a transposed warp reduction of two values.
__device__ __forceinline__ float2 lo2(const float4& v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(const float4& v) { return make_float2(v.z, v.w); }
__device__ __forceinline__ float4 join2(const float2& a, const float2& b) { return make_float4(a.x, a.y, b.x, b.y); }


// Warp sums of two values in a fixed order: lane l ends with the sum of
// value (l >> 4) & 1, so lanes 0 and 16 hold the sums of v0 and v1.
__device__ __forceinline__ float warp_sum2(float v0, float v1, int lane) {
  const bool b4 = (lane & 16) != 0;
  float r = (b4 ? v1 : v0) + __shfl_xor_sync(0xffffffffu, b4 ? v0 : v1, 16);
  r += __shfl_xor_sync(0xffffffffu, r, 8);
  r += __shfl_xor_sync(0xffffffffu, r, 4);
  r += __shfl_xor_sync(0xffffffffu, r, 2);
  r += __shfl_xor_sync(0xffffffffu, r, 1);
  return r;
}

// ---------------------------------------------------------------------------
// Sweep S_j, 3D FP32, with the basis staged through shared memory: a block
// owns tiles of SW_TILE cells (one quad a thread) and, for each tile,
// streams the columns V_0..V_{j-1} through a ring of SW_STAGES buffers that
// one thread fills with one-dimensional bulk copies (cp.async.bulk, their
// completion counted on an mbarrier per buffer).  The bytes in flight per SM
// then no longer depend on registers: a register-fed form, with the 128
// registers two blocks per SM allow, kept one column per warp in flight
// (measured at 128^3: 0.79 of the measured copy bandwidth, staged 0.84).
// Every wait is bounded: when one runs out the block records KX_ETIMEOUT,
// waits (bounded again) for its own copies and returns.
constexpr int SW_STAGES = 4;                                      // buffers in the ring (a power of 2)
constexpr size_t SW_STAGE_FLOATS = 6 * (size_t)SW_TILE;           // one column of a tile
constexpr size_t SW_SMEM = SW_STAGES * SW_STAGE_FLOATS * sizeof(float);
constexpr unsigned SW_WAIT_LIMIT = 1u << 22;                      // try_wait rounds of one wait
static_assert(SW_STAGES == 4, "the wait parity below is (e >> 2) & 1");
static_assert(SW_WAIT_LIMIT == KX_WAIT_SELFTEST_MAX_ROUNDS, "the self-test runs at most one wait's limit");

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t* b, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint64_t* b, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for the completion of phase `parity` of b: false when
// `limit` try_wait rounds pass without it.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, unsigned parity, unsigned limit = SW_WAIT_LIMIT) {
  for (unsigned k = 0; k < limit; ++k)
    if (mbar_test(b, parity)) return true;
  return false;
}

// The failure path of that wait, checked without a fault: one warp waits on
// an mbarrier that nothing completes (no copy is issued) and records
// KX_ETIMEOUT when the wait runs out, as the sweep does.
__global__ void k_wait_selftest(unsigned limit, int* status) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) {
    mbar_init(&bar, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncwarp();
  const bool ok = mbar_wait(&bar, 0u, limit);
  if (threadIdx.x == 0) *status = __all_sync(0xffffffffu, ok) ? KX_OK : KX_ETIMEOUT;
  else (void)__all_sync(0xffffffffu, ok);
}
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(b))
               : "memory");
}

// Element e of a block's stream: column `col` of tile `tile` (e = its
// index in the block's (tile, column) order), into buffer e % SW_STAGES
// (16-byte aligned: tiles start at multiples of 1024 cells, columns at
// multiples of 64 scalars, components at multiples of ncell with
// ncell % 4 == 0; each copy is a multiple of 16 bytes).
__device__ __forceinline__ void sw_issue(const Slot<float>& s, int64_t ld, int64_t nc, int64_t tile, int col, int b,
                                         float* ring, uint64_t* full) {
  const int64_t cell0 = tile * SW_TILE;
  const int64_t cells = nc - cell0 < SW_TILE ? nc - cell0 : SW_TILE;
  const unsigned bytes = (unsigned)(cells * (int64_t)sizeof(float));
  float* dst = ring + b * SW_STAGE_FLOATS;
  const float* src = s.V + (int64_t)col * ld + cell0;
  mbar_expect_tx(&full[b], 6u * bytes);
#pragma unroll
  for (int c = 0; c < 6; ++c) bulk_load(dst + c * SW_TILE, src + c * nc, bytes, &full[b]);
}

// The issue cursor of a block's stream (thread 0 only): advancing it by one
// element moves to the next column, or to the first column of the block's
// next tile (no division in the loop).
struct SwCursor {
  int64_t tile;
  int col;
  int stride;   // blocks of the block's problem: the tile stride
  __device__ __forceinline__ void next(int j) {
    if (++col == j) {
      col = 0;
      tile += stride;
    }
  }
};

// The body takes its block index among the launch's blocks for this slot
// (bid of nblk), so that one launch can serve several problems.
__device__ __forceinline__ void sw_pass4s_body(const Geo& g, const Slot<float>& s, const SwSlot& w, int j, int64_t ld,
                                               const float* __restrict__ ie, const float* __restrict__ sig2, int bid,
                                               int nblk) {
  extern __shared__ __align__(128) unsigned char sw_dyn[];
  float* ring = reinterpret_cast<float*>(sw_dyn);
  __shared__ __align__(8) uint64_t full[SW_STAGES];
  __shared__ float ch[MMAX], cc[MMAX];
  __shared__ double acc[NWARPS][SWCOLS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int q = threadIdx.x; q < NWARPS * SWCOLS; q += blockDim.x) (&acc[0][0])[q] = 0.0;
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    const double sc = s.scale[i];
    ch[i] = (float)(w.co->hc[i] * sc);
    cc[i] = (float)(w.co->cp[i] * sc);
  }
  const float sp = (float)w.co->sprev, spl = (float)(w.co->sprev - (double)sp);
  const float hjj = (float)w.co->hjj;
  const int64_t nc = g.ncell, nq = nc >> 2;
  const int64_t ntiles = (nc + SW_TILE - 1) / SW_TILE;
  const int64_t mine = (int64_t)bid < ntiles ? (ntiles - 1 - bid) / nblk + 1 : 0;
  const int64_t E = mine * j;
  if (threadIdx.x == 0) {
    for (int b = 0; b < SW_STAGES; ++b) mbar_init(&full[b], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  __syncthreads();
  SwCursor cur{(int64_t)bid, 0, nblk};   // the next element to issue (thread 0)
  if (threadIdx.x == 0)
    for (int64_t e = 0; e < E && e < SW_STAGES; ++e) {
      sw_issue(s, ld, nc, cur.tile, cur.col, (int)e, ring, full);
      cur.next(j);
    }
  const float* __restrict__ t = (const float*)w.t;
  float* __restrict__ xout = s.V + (int64_t)j * ld;
  // x = hi + lo (compensated, kx_eft.cuh); y plain FP32 (it enters only the dots)
  float4 x[6], xl[6], y[6];
  bool act = false, ok = true;
  int64_t c0 = 0, tile = bid;
  int col = 0;
  // Elements are consumed two at a time (two columns of the same tile, one
  // block barrier and two refills per pair), one at a time at a tile's odd
  // end; the arithmetic of every column is the same either way.
  for (int64_t e = 0; e < E;) {
    if (col == 0) {
      // a tile starts: x = A v_{j-1}, y = A^2 v_{j-1} - h_{j-1,j-1} A v_{j-1}
      const int64_t q4 = tile * NTHREADS + threadIdx.x;
      act = q4 < nq;
      c0 = 0;
      if (act) {
        c0 = q4 << 2;
        float4 at[6];
        stencil_quad32(g, t, ie, sig2, (int)c0, at);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          const float4 tv = ld4(t + c * nc + c0);
          // x = (sp + spl) t exactly up to the rounding of lo
          x[c] = make_float4(sp * tv.x, sp * tv.y, sp * tv.z, sp * tv.w);
          xl[c] = make_float4(fmaf(spl, tv.x, fmaf(sp, tv.x, -x[c].x)), fmaf(spl, tv.y, fmaf(sp, tv.y, -x[c].y)),
                              fmaf(spl, tv.z, fmaf(sp, tv.z, -x[c].z)), fmaf(spl, tv.w, fmaf(sp, tv.w, -x[c].w)));
          y[c] = make_float4(sp * at[c].x - hjj * x[c].x, sp * at[c].y - hjj * x[c].y, sp * at[c].z - hjj * x[c].z,
                             sp * at[c].w - hjj * x[c].w);
        }
      } else {
#pragma unroll
        for (int c = 0; c < 6; ++c) x[c] = xl[c] = y[c] = make_float4(0.f, 0.f, 0.f, 0.f);
      }
    }
    const int cnt = col + 1 < j ? 2 : 1;   // elements e .. e + cnt - 1: columns col .. col + cnt - 1
    const bool ends = col + cnt == j;      // the group holds the tile's last column
    if (ends) {
      // prefetch the next tile's stencil inputs
      const int64_t qn = (tile + nblk) * NTHREADS + threadIdx.x;
      if (qn < nq) prefetch_quad32(g, t, ie, (int)(qn << 2));
    }
#pragma unroll 1
    for (int q = 0; q < cnt; ++q) {
      const int64_t ee = e + q;
      const int cq = col + q;
      const int b = (int)(ee & (SW_STAGES - 1));
      if (ok) ok = mbar_wait(&full[b], (unsigned)((ee >> 2) & 1));
      float pa = 0.f, pb = 0.f;
      if (act) {
        // an inactive thread reads no buffer (the tile's tail is not copied)
        const float* sb = ring + b * SW_STAGE_FLOATS + 4 * threadIdx.x;
        float4 vv[6];
#pragma unroll
        for (int c = 0; c < 6; ++c) vv[c] = *reinterpret_cast<const float4*>(sb + c * SW_TILE);
        // two independent accumulator chains per dot (the quad's two halves)
        float2 sa = make_float2(0.f, 0.f), sa2 = sa, sx = sa, sx2 = sa;
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          sa = __ffma2_rn(lo2(vv[c]), lo2(y[c]), sa);
          sa2 = __ffma2_rn(hi2(vv[c]), hi2(y[c]), sa2);
          sx = __ffma2_rn(lo2(vv[c]), lo2(x[c]), sx);
          sx2 = __ffma2_rn(hi2(vv[c]), hi2(x[c]), sx2);
        }
        pa = (sa.x + sa2.x) + (sa.y + sa2.y);
        pb = (sx.x + sx2.x) + (sx.y + sx2.y);
        const float2 na = make_float2(-ch[cq], -ch[cq]), nb = make_float2(-cc[cq], -cc[cq]);
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          float2 h0 = lo2(x[c]), h1 = hi2(x[c]), l0 = lo2(xl[c]), l1 = hi2(xl[c]);
          sub_fma2(h0, l0, na, lo2(vv[c]));
          sub_fma2(h1, l1, na, hi2(vv[c]));
          x[c] = join2(h0, h1);
          xl[c] = join2(l0, l1);
          y[c] = join2(__ffma2_rn(nb, lo2(vv[c]), lo2(y[c])), __ffma2_rn(nb, hi2(vv[c]), hi2(y[c])));
        }
      }
      const float r = warp_sum2(pa, pb, lane);
      if ((lane & 15) == 0) acc[warp][(lane >> 4) * j + cq] += (double)r;
    }
    if (ends) {
      // the tile ends: store V_j = x (hi + lo rounded once), accumulate x.x, x.y, y.y
      float xx = 0.f, xy = 0.f, yy = 0.f;
      if (act) {
#pragma unroll
        for (int c = 0; c < 6; ++c) {
          x[c] = make_float4(x[c].x + xl[c].x, x[c].y + xl[c].y, x[c].z + xl[c].z, x[c].w + xl[c].w);
          *reinterpret_cast<float4*>(xout + c * nc + c0) = x[c];
          xx += dot4(x[c], x[c]);
          xy += dot4(x[c], y[c]);
          yy += dot4(y[c], y[c]);
        }
      }
      xx = warp_sum(xx);
      xy = warp_sum(xy);
      yy = warp_sum(yy);
      if (lane == 0) {
        acc[warp][2 * j] += (double)xx;
        acc[warp][2 * j + 1] += (double)xy;
        acc[warp][2 * j + 2] += (double)yy;
      }
    }
    // every thread is done with the group's buffers: refill them with
    // elements e + SW_STAGES ..
    if (!__syncthreads_and(ok)) {
      if (threadIdx.x == 0) {
        s.st->status = KX_ETIMEOUT;
        s.st->done = 1;
        for (int64_t f = e; f < E && f < e + SW_STAGES; ++f)
          mbar_wait(&full[f & (SW_STAGES - 1)], (unsigned)((f >> 2) & 1));
      }
      return;
    }
    if (threadIdx.x == 0) {
      for (int q = 0; q < cnt; ++q) {
        if (e + q + SW_STAGES >= E) break;
        if (q == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        sw_issue(s, ld, nc, cur.tile, cur.col, (int)((e + q) & (SW_STAGES - 1)), ring, full);
        cur.next(j);
      }
    }
    e += cnt;
    col += cnt;
    if (col == j) {
      col = 0;
      tile += nblk;
    }
  }
  pdl_trigger();
  __syncthreads();
  for (int c2 = threadIdx.x; c2 < 2 * j + 3; c2 += blockDim.x) {
    double tsum = 0.0;
#pragma unroll
    for (int q = 0; q < NWARPS; ++q) tsum += acc[q][c2];
    w.part[(int64_t)c2 * w.ps + bid] = tsum;
  }
}

__global__ void __launch_bounds__(NTHREADS, 2) k_sw_pass4s(Geo g, Slot<float> s, SwSlot w, int j, int64_t ld,
                                                          const float* __restrict__ ie,
                                                          const float* __restrict__ sig2) {
  pdl_wait();
  if (s.st->done || s.st->retired) return;
  sw_pass4s_body(g, s, w, j, ld, ie, sig2, blockIdx.x, gridDim.x);
}

// Finalisation after the last sweep S_m (one block): beta_{m-1}, scale_m,
// m_done = m and the breakdown test.
template <typename T>
__global__ void __launch_bounds__(NTHREADS) k_sw_last(Slot<T> s, SwSlot w, int m, int ldh, int nbs, double btol) {
  pdl_wait();
  if (s.st->done || s.st->retired) return;
  const double x = block_column_sum(w.part, w.ps, 2 * m, nbs);
  if (threadIdx.x == 0) w.co->tot[2 * m] = x;
  __syncthreads();
  sw_fin<T>(s, w.co, w.G, m, ldh, btol, 1);
}

// ---------------------------------------------------------------------------
// Batched forms: one launch serves every problem of a batch.  Block b of a
// launch belongs to problem i with off[i] <= b < off[i + 1] and runs that
// problem's body as its block b - off[i] of off[i + 1] - off[i]; the
// problem's record is copied to shared memory once per block.
__device__ __forceinline__ int inst_of(const int* __restrict__ off, int n, int b) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= b) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

__device__ __forceinline__ void load_inst(SwInst& dst, const SwInst* __restrict__ tab, int i) {
  static_assert(sizeof(SwInst) % 4 == 0, "copied as 32-bit words");
  const int* src = reinterpret_cast<const int*>(tab + i);
  int* d = reinterpret_cast<int*>(&dst);
  for (int k = threadIdx.x; k < (int)(sizeof(SwInst) / 4); k += blockDim.x) d[k] = __ldg(src + k);
  __syncthreads();
}

__global__ void __launch_bounds__(NTHREADS, 3) k_sw_apply4_batch(const SwInst* __restrict__ tab,
                                                             const int* __restrict__ off, int n, int slot, int j,
                                                             double btol) {
  __shared__ SwInst I;
  const int i = inst_of(off, n, blockIdx.x);
  load_inst(I, tab, i);
  pdl_wait();
  const Slot<float> s = I.s[slot];
  if (s.st->done || s.st->retired) return;
  sw_apply4_body(I.g, s, I.w[slot], j, I.ld, I.ie, I.sig2, I.ldh, I.ns, btol, (int)blockIdx.x - I.a0, I.na);
}

__global__ void __launch_bounds__(NTHREADS, 2) k_sw_pass4s_batch(const SwInst* __restrict__ tab,
                                                             const int* __restrict__ off, int n, int slot, int j) {
  __shared__ SwInst I;
  const int i = inst_of(off, n, blockIdx.x);
  load_inst(I, tab, i);
  pdl_wait();
  const Slot<float> s = I.s[slot];
  if (s.st->done || s.st->retired) return;
  sw_pass4s_body(I.g, s, I.w[slot], j, I.ld, I.ie, I.sig2, (int)blockIdx.x - I.s0, I.ns);
}

// Apply pass K_j (j >= 1) of every problem still running, the column march
// of k_sw_apply_col: the problem's SW_RED reducer blocks, then its column
// blocks, each over kz planes of NTHREADS quad columns.
__global__ void __launch_bounds__(NTHREADS, 2) k_sw_apply_col_batch(const SwInst* __restrict__ tab,
                                                                const int* __restrict__ off, int n, int slot,
                                                                int j, double btol) {
  __shared__ SwInst I;
  const int i = inst_of(off, n, blockIdx.x);
  load_inst(I, tab, i);
  pdl_wait();
  const Slot<float> s = I.s[slot];
  if (s.st->done || s.st->retired) return;
  const int bid = (int)blockIdx.x - I.c0;
  if (bid < SW_RED) {
    sw_reduce_fin<float>(s, I.w[slot], j, I.ldh, I.ns, btol, bid);
    return;
  }
  const int b = bid - SW_RED;
  const int zc = b / I.ncb;
  const int q = (b - zc * I.ncb) * NTHREADS + (int)threadIdx.x;
  const int k0 = zc * I.kz, k1 = min(I.g.nz, k0 + I.kz);
  if (q < (I.g.nx >> 2) * I.g.ny && k0 < k1)
    stencil_column_quad(I.g, s.V + (int64_t)j * I.ld, I.ie, I.sig2, (float*)I.w[slot].t, q, k0, k1);
  pdl_trigger();
}

// After the last sweep: one block per problem.
__global__ void __launch_bounds__(NTHREADS) k_sw_last_batch(const SwInst* __restrict__ tab, int slot, int m,
                                                            double btol) {
  __shared__ SwInst I;
  load_inst(I, tab, blockIdx.x);
  pdl_wait();
  const Slot<float> s = I.s[slot];
  if (s.st->done || s.st->retired) return;
  const SwSlot w = I.w[slot];
  const double x = block_column_sum(w.part, w.ps, 2 * m, I.ns);
  if (threadIdx.x == 0) w.co->tot[2 * m] = x;
  __syncthreads();
  sw_fin<float>(s, w.co, w.G, m, I.ldh, btol, 1);
}

}  // namespace

template <typename T>
constexpr double sw_btol() { return sizeof(T) == 8 ? 1e-12 : 1e-6; }

size_t sweep_smem_bytes() { return SW_SMEM; }
const void* sweep_batch_kernel() { return (const void*)k_sw_pass4s_batch; }

// Launch with programmatic dependent launch (the bodies wait for their
// predecessor before touching data and trigger their successor near the end).
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(void (*kern)(KArgs...), int grid, size_t smem, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(NTHREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, args...);
}

kx_status sweep_batch_prepare(kx_ctx* c0) {
  static SmemOptIn smem{};
  return smem_opt_in(c0, smem, (const void*)k_sw_pass4s_batch, SW_SMEM);
}

kx_status sweep_arnoldi_batch(kx_ctx* c0, cudaStream_t st, const SwInst* tab, const int* aoff, const int* soff,
                              const int* coff, int n, int na, int ns, int nc, int slot, int m, int64_t* launches,
                              std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* sweep_events) {
  const kx_status so = sweep_batch_prepare(c0);
  if (so != KX_OK) return so;
  const double bt = sw_btol<float>();
  for (int j = 0; j <= m; ++j) {
    cudaError_t e = cudaSuccess;
    if (j >= 1) {
      // optional event pair around the sweep launch (a measurement aid; the
      // events break the programmatic overlap with the neighbouring launches)
      cudaEvent_t ea = nullptr, eb = nullptr;
      if (sweep_events) {
        cudaEventCreate(&ea);
        cudaEventCreate(&eb);
        cudaEventRecord(ea, st);
      }
      e = launch_pdl(k_sw_pass4s_batch, ns, SW_SMEM, st, tab, soff, n, slot, j);
      if (e == cudaSuccess) ++*launches;
      if (sweep_events) {
        cudaEventRecord(eb, st);
        sweep_events->push_back({ea, eb});
      }
    }
    if (e == cudaSuccess) {
      // step 0's apply also takes the dots of its finalisation: the quad form
      e = j == m   ? launch_pdl(k_sw_last_batch, n, 0, st, tab, slot, m, bt)
          : j == 0 ? launch_pdl(k_sw_apply4_batch, na, 0, st, tab, aoff, n, slot, j, bt)
                   : launch_pdl(k_sw_apply_col_batch, nc, 0, st, tab, coff, n, slot, j, bt);
      if (e == cudaSuccess) ++*launches;
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      snprintf(c0->err, sizeof(c0->err), "batched Arnoldi launch failed: %s", cudaGetErrorString(e));
      return KX_ECUDA;
    }
  }
  return KX_OK;
}

static SwSlot sw_slot(kx_ctx* c, int slot) {
  SwSlot w;
  w.part = c->d_swpart + (int64_t)slot * SWCOLS * c->ps;
  w.ps = c->ps;
  w.G = c->d_swG + (int64_t)slot * LG * LG;
  w.co = c->d_swco + slot;
  w.t = c->d_swT;
  return w;
}

// Persistent grids (occupancy x SMs, capped by the work and the partial
// stride), shrunk for resident CTAs of kernels running beside the process.
// nb_sweep_late: the sweep grid of the steps past the side CTAs' window.
static void sw_grids(kx_ctx* c, const void* fa, const void* fs, size_t smem_s, int kind, int64_t items,
                     int* nb_apply, int* nb_sweep, int* nb_sweep_late) {
  static std::atomic<int> ga[8], gs[8];
  if (!ga[kind]) ga[kind] = persistent_grid(c, fa, 1 << 30, 0);
  if (!gs[kind]) gs[kind] = persistent_grid(c, fs, 1 << 30, smem_s);
  const int64_t rounds = (items + NTHREADS - 1) / NTHREADS;
  *nb_apply = reserve_grid(c, (int)std::min<int64_t>(rounds, ga[kind].load()), ga[kind].load());
  const int ns = (int)std::min<int64_t>(rounds, gs[kind].load());
  *nb_sweep = reserve_grid(c, ns, gs[kind].load());
  *nb_sweep_late = reserve_grid_at(c, ns, gs[kind].load(), c->side_steps);
}

// Grid of k_sw_apply_col for step j: SW_RED reducer blocks, then ncb column
// blocks on each of ceil(nz / kz) plane ranges, kz chosen so that every
// block finds a slot in the first wave beside the reducers (and, in the
// steps the side CTAs may overlap, beside them).
struct ColGrid {
  int blocks, ncb, kz;
};

static ColGrid col_grid(kx_ctx* c, const void* kernel, bool quad, int j) {
  static std::atomic<int> occ_cache[2];
  int occ = occ_cache[quad].load();
  if (!occ) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, NTHREADS, 0) != cudaSuccess || occ < 1) {
      cudaGetLastError();
      occ = 1;
    }
    occ_cache[quad] = occ;
  }
  const Geo& g = c->geo;
  const int full = c->nsm * occ;
  const int avail = std::max(1, reserve_grid_at(c, full, full, j) - SW_RED);
  const int64_t ncol = quad ? (int64_t)(g.nx / 4) * g.ny : (int64_t)g.nx * g.ny;
  ColGrid r;
  r.ncb = (int)((ncol + NTHREADS - 1) / NTHREADS);
  const int64_t kz = ((int64_t)g.nz * r.ncb + avail - 1) / avail;
  r.kz = (int)std::min<int64_t>(std::max<int64_t>(kz, 1), g.nz);
  r.blocks = SW_RED + r.ncb * ((g.nz + r.kz - 1) / r.kz);
  return r;
}

template <typename T, int DIM>
static kx_status sweep_t(kx_ctx* c, int slot, int m) {
  const Geo& g = c->geo;
  const Slot<T> s = make_slot<T>(c, slot);
  const SwSlot w = sw_slot(c, slot);
  const T* ie = (const T*)c->d_inv_eps;
  const T* sg = (const T*)c->d_sig2;
  const TableMat<T> mat{ie, sg};
  const int ldh = c->m + 1;
  const double bt = sw_btol<T>();
  // the quad kernels need 16-byte aligned rows of every array they read
  constexpr bool f3 = sizeof(T) == 4 && DIM == 3;
  const bool quad = f3 && (g.nx % 4) == 0 && g.ncell < ((int64_t)1 << 31);
  // steps j >= 1 apply A by the column march (32-bit cell offsets)
  const bool colm = f3 && g.ncell < ((int64_t)1 << 31);
  int nba = 0, nbs = 0, nbs_late = 0;
  if (quad) {
    // per device, and before any launch (contexts of the multi-problem
    // driver run on several host threads)
    static SmemOptIn smem{};
    const kx_status so = smem_opt_in(c, smem, (const void*)k_sw_pass4s, SW_SMEM);
    if (so != KX_OK) return so;
    sw_grids(c, (const void*)k_sw_apply4, (const void*)k_sw_pass4s, SW_SMEM, 7, g.ncell / 4, &nba, &nbs, &nbs_late);
  } else {
    sw_grids(c, (const void*)k_sw_apply<T, DIM, TableMat<T>>, (const void*)k_sw_pass<T, DIM, TableMat<T>>, 0,
             (sizeof(T) == 8 ? 3 : 0) + (DIM - 2), g.ncell, &nba, &nbs, &nbs_late);
  }
  const double vb = (double)c->n * c->esize;
  const double mb = (double)g.ne * g.ncell * c->esize;
  for (int j = 0; j <= m; ++j) {
    // sweep S_j's grid; apply pass K_j's reducers and k_sw_last take its partials
    const int nbs_j = j < c->side_steps ? nbs : nbs_late;
    if (j >= 1) {
      time_begin(c);
      if constexpr (f3) {
        if (quad)
          launch_k(c, k_sw_pass4s, dim3(nbs_j), dim3(NTHREADS), SW_SMEM, c->stream, g, (Slot<float>)s, w, j, c->ld,
                   (const float*)ie, (const float*)sg);
        else
          launch_k(c, k_sw_pass<T, DIM, TableMat<T>>, dim3(nbs_j), dim3(NTHREADS), 0, c->stream, g, s, w, j, c->ld,
                   mat);
      } else {
        launch_k(c, k_sw_pass<T, DIM, TableMat<T>>, dim3(nbs_j), dim3(NTHREADS), 0, c->stream, g, s, w, j, c->ld, mat);
      }
      time_end(c, KX_K_SWEEP, (j + 2.0) * vb + mb);
      KX_CHECK_LAUNCH(c);
    }
    // the apply grid: the stencil blocks (shrunk by the reducer blocks when
    // that keeps every block resident) and, from step 1, SW_RED in front
    const int ga = j == 0 ? nba : (nba > 2 * SW_RED ? nba - SW_RED : nba) + SW_RED;
    time_begin(c);
    if (j == m) {
      launch_k(c, k_sw_last<T>, dim3(1), dim3(NTHREADS), 0, c->stream, s, w, m, ldh, nbs_j, bt);
    } else if constexpr (f3) {
      if (j >= 1 && colm) {
        const void* kc = quad ? (const void*)k_sw_apply_col<true> : (const void*)k_sw_apply_col<false>;
        const ColGrid cg = col_grid(c, kc, quad, j);
        if (quad)
          launch_k(c, k_sw_apply_col<true>, dim3(cg.blocks), dim3(NTHREADS), 0, c->stream, g, (Slot<float>)s, w, j,
                   c->ld, (const float*)ie, (const float*)sg, ldh, nbs_j, bt, cg.ncb, cg.kz);
        else
          launch_k(c, k_sw_apply_col<false>, dim3(cg.blocks), dim3(NTHREADS), 0, c->stream, g, (Slot<float>)s, w,
                   j, c->ld, (const float*)ie, (const float*)sg, ldh, nbs_j, bt, cg.ncb, cg.kz);
      } else if (quad)
        launch_k(c, k_sw_apply4, dim3(ga), dim3(NTHREADS), 0, c->stream, g, (Slot<float>)s, w, j, c->ld,
                 (const float*)ie, (const float*)sg, ldh, nbs_j, bt);
      else
        launch_k(c, k_sw_apply<T, DIM, TableMat<T>>, dim3(ga), dim3(NTHREADS), 0, c->stream, g, s, w, j, c->ld, mat,
                 ldh, nbs_j, bt);
    } else {
      launch_k(c, k_sw_apply<T, DIM, TableMat<T>>, dim3(ga), dim3(NTHREADS), 0, c->stream, g, s, w, j, c->ld, mat,
               ldh, nbs_j, bt);
    }
    time_end(c, KX_K_SWAPPLY, j < m ? 2.0 * vb + mb : 0.0);
    KX_CHECK_LAUNCH(c);
  }
  c->stats.arnoldi_steps += m;
  c->stats.matvecs += 2 * (int64_t)m;
  return KX_OK;
}

kx_status launch_wait_selftest(kx_ctx* c, unsigned rounds, int* d_status) {
  k_wait_selftest<<<1, 32, 0, c->stream>>>(rounds, d_status);
  KX_CHECK_LAUNCH(c);
  return KX_OK;
}

kx_status sweep_arnoldi(kx_ctx* c, int slot, int m) {
  const Geo& g = c->geo;
  const bool fp64 = c->d.precision == KX_FP64;
  if (g.dim == 3) return fp64 ? sweep_t<double, 3>(c, slot, m) : sweep_t<float, 3>(c, slot, m);
  if (g.pml) return fp64 ? sweep_t<double, 4>(c, slot, m) : sweep_t<float, 4>(c, slot, m);
  return fp64 ? sweep_t<double, 2>(c, slot, m) : sweep_t<float, 2>(c, slot, m);
}

}  // namespace kx
