// Deterministic grid-wide reductions shared by the bulk kernels.
//
// Each block writes its partial sums into a column-major table
//   part[col * ps + block]            (ps >= gridDim.x)
// and the last block to finish (atomic ticket) sums every column with all
// its warps: lane l adds blocks l, l+32, ... and a fixed shuffle tree
// finishes, so the result does not depend on block scheduling.
#pragma once

#include "kx_internal.cuh"

namespace kx {

template <typename T>
__device__ __forceinline__ T warp_sum(T x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// True in every thread of the last block to finish; that block then sees
// every other block's partials.
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

// Block sum of one double per thread, written to part[col * ps + bid].
__device__ __forceinline__ void block_partial_at(double x, double* part, int ps, int col, int bid) {
  __shared__ double red[NWARPS];
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) t += red[w];
    part[(int64_t)col * ps + bid] = t;
  }
  __syncthreads();
}

// Block sum of one double per thread, written to part[col * ps + blockIdx.x].
__device__ __forceinline__ void block_partial(double x, double* part, int ps, int col) {
  __shared__ double red[NWARPS];
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) t += red[w];
    part[(int64_t)col * ps + blockIdx.x] = t;
  }
  __syncthreads();
}

// Finalisation of step j-1's pass B at the start of step j's pass A
// (non-augmented processes): every block sums the same nbb partials in the
// same order, so all reach the same h_{j,j-1} and the same breakdown
// decision; block 0 records them.  Returns false where the process stops
// (lucky breakdown or a non-finite norm); *sj receives scale_j = 1/h.
template <typename T>
__device__ __forceinline__ bool fin_prev_b(const Slot<T>& s, int j, int ldh, int nbb, double btol, double* sj) {
  double x = 0.0;
  for (int b = threadIdx.x; b < nbb; b += blockDim.x) x += __ldcg(s.part + (int64_t)FINB_COL * s.ps + b);
  __shared__ double red[NWARPS];
  __shared__ double res;
  __shared__ int stop;
  x = warp_sum(x);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = x;
  __syncthreads();
  if (threadIdx.x == 0) {
    double tot = 0.0;
#pragma unroll
    for (int w = 0; w < NWARPS; ++w) tot += red[w];
    const double h = sqrt(tot);
    int stp = 0;
    double scl = 0.0;
    if (!isfinite(h)) stp = 2;
    else if (h <= btol * s.st->wmax) stp = 1;   // invariant subspace: the projection is exact
    else scl = 1.0 / h;
    if (blockIdx.x == 0) {
      s.H[j + (int64_t)(j - 1) * ldh] = h;
      s.st->m_done = j;
      s.scale[j] = scl;
      if (stp == 2) s.st->status = KX_ENONFINITE;
      if (stp || abort_requested(s.st)) s.st->done = 1;
    }
    res = scl;
    stop = stp;
  }
  __syncthreads();
  *sj = res;
  return stop == 0;
}

// In the last block: tot[c] = sum over blocks of part[c * ps + b], c < ncols.
__device__ __forceinline__ void grid_columns(const double* part, int ps, int ncols, double* tot) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nb = gridDim.x;
  for (int col = warp; col < ncols; col += NWARPS) {
    const double* p = part + (int64_t)col * ps;
    double s0 = 0.0, s1 = 0.0;
    int b = lane;
    for (; b + 32 < nb; b += 64) {
      s0 += __ldcg(p + b);
      s1 += __ldcg(p + b + 32);
    }
    if (b < nb) s0 += __ldcg(p + b);
    s0 = warp_sum(s0 + s1);
    if (lane == 0) tot[col] = s0;
  }
  __syncthreads();
}

}  // namespace kx
