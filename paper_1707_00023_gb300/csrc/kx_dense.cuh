// Dense FP64 kernels-within-a-CTA for the projected (small) matrices:
// products, linear combinations, 1-norm, LU solve with partial pivoting and
// the scaling-and-squaring Pade exponential (Higham 2005, "The scaling and
// squaring method for the matrix exponential revisited").  All threads of
// the block take part; matrices are row-major in shared or global memory.
#pragma once

#include "kx_internal.cuh"

namespace kx {

// theta_m of Higham 2005, Table 2.3: largest 1-norm for which the degree-m
// diagonal Pade approximant meets double-precision backward error.
static __constant__ double c_theta[5] = {1.495585217958292e-2, 2.539398330063230e-1,
                                  9.504178996162932e-1, 2.097847961257068e0,
                                  5.371920351148152e0};

// Coefficient b_k of the degree-p diagonal Pade numerator of exp, normalised
// to b_0 = 1:  b_{k+1} = b_k (p - k) / ((2p - k)(k + 1)).
__device__ __forceinline__ double pade_b(int p, int k) {
  double b = 1.0;
  for (int q = 0; q < k; ++q) b *= (double)(p - q) / ((double)(2 * p - q) * (double)(q + 1));
  return b;
}

static __device__ void cta_mm(double* C, const double* A, const double* B, int n) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    const int r = idx / n, c = idx - r * n;
    double s = 0.0;
    for (int k = 0; k < n; ++k) s = fma(A[r * n + k], B[k * n + c], s);
    C[idx] = s;
  }
  __syncthreads();
}

// C = a1*M1 + a2*M2 + a3*M3 + a4*M4 + d*I (null matrices skipped).
static __device__ void cta_lin(double* C, double a1, const double* M1, double a2, const double* M2,
                        double a3, const double* M3, double a4, const double* M4, double d, int n) {
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
    double s = 0.0;
    if (M1) s += a1 * M1[idx];
    if (M2) s += a2 * M2[idx];
    if (M3) s += a3 * M3[idx];
    if (M4) s += a4 * M4[idx];
    const int r = idx / n;
    if (idx == r * n + r) s += d;
    C[idx] = s;
  }
  __syncthreads();
}

static __device__ double cta_norm1(const double* A, int n, double* red) {
  double mx = 0.0;
  for (int c = threadIdx.x; c < n; c += blockDim.x) {
    double s = 0.0;
    for (int r = 0; r < n; ++r) s += fabs(A[r * n + c]);
    mx = fmax(mx, s);
  }
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  double r = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) r = fmax(r, red[w]);
  __syncthreads();
  return r;
}

// Solve P X = Q in place (Gaussian elimination, partial pivoting); X -> Q.
// Returns false if a pivot is zero.
static __device__ bool cta_solve(double* P, double* Q, int n, double* lv, int* piv_sh) {
  __shared__ bool ok;
  if (threadIdx.x == 0) ok = true;
  __syncthreads();
  for (int k = 0; k < n; ++k) {
    if (threadIdx.x < 32) {
      double best = -1.0;
      int bi = k;
      for (int r = k + threadIdx.x; r < n; r += 32) {
        const double a = fabs(P[r * n + k]);
        if (a > best) { best = a; bi = r; }
      }
      for (int o = 16; o > 0; o >>= 1) {
        const double ob = __shfl_xor_sync(0xffffffffu, best, o);
        const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
        if (ob > best || (ob == best && oi < bi)) { best = ob; bi = oi; }
      }
      if (threadIdx.x == 0) {
        *piv_sh = bi;
        if (!(best > 0.0)) ok = false;
      }
    }
    __syncthreads();
    if (!ok) return false;
    const int p = *piv_sh;
    if (p != k) {
      for (int c = threadIdx.x; c < n; c += blockDim.x) {
        double t = P[k * n + c]; P[k * n + c] = P[p * n + c]; P[p * n + c] = t;
        t = Q[k * n + c]; Q[k * n + c] = Q[p * n + c]; Q[p * n + c] = t;
      }
    }
    __syncthreads();
    const double d = P[k * n + k];
    for (int r = k + 1 + threadIdx.x; r < n; r += blockDim.x) lv[r] = P[r * n + k] / d;
    __syncthreads();
    const int rows = n - k - 1;
    const int cols = (n - k - 1) + n;
    for (int idx = threadIdx.x; idx < rows * cols; idx += blockDim.x) {
      const int r = k + 1 + idx / cols;
      const int cc = idx % cols;
      if (cc < n - k - 1) {
        const int c = k + 1 + cc;
        P[r * n + c] = fma(-lv[r], P[k * n + c], P[r * n + c]);
      } else {
        const int c = cc - (n - k - 1);
        Q[r * n + c] = fma(-lv[r], Q[k * n + c], Q[r * n + c]);
      }
    }
    __syncthreads();
  }
  for (int k = n - 1; k >= 0; --k) {
    const double d = P[k * n + k];
    for (int c = threadIdx.x; c < n; c += blockDim.x) Q[k * n + c] /= d;
    __syncthreads();
    for (int idx = threadIdx.x; idx < k * n; idx += blockDim.x) {
      const int r = idx / n, c = idx - r * n;
      Q[r * n + c] = fma(-P[r * n + k], Q[k * n + c], Q[r * n + c]);
    }
    __syncthreads();
  }
  return true;
}

// exp(B) of the n x n matrix in buf[0]; returns the buffer holding the
// result (one of buf[0..5]), or nullptr on a singular Pade denominator.
static __device__ double* cta_expm(double* const* buf, int n, double* red, double* lv, int* piv) {
  double* A = buf[0];
  const double nrm = cta_norm1(A, n, red);
  int p = 13, s = 0;
  const int degs[4] = {3, 5, 7, 9};
  bool found = false;
  for (int q = 0; q < 4 && !found; ++q)
    if (nrm <= c_theta[q]) { p = degs[q]; found = true; }
  if (!found) {
    p = 13;
    if (nrm > c_theta[4]) s = max(0, (int)ceil(log2(nrm / c_theta[4])));
    if (s > 0) {
      const double f = ldexp(1.0, -s);
      for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) A[idx] *= f;
      __syncthreads();
    }
  }
  double b[14];
  for (int k = 0; k <= p; ++k) b[k] = pade_b(p, k);
  double *A2 = buf[1], *A4 = buf[2], *A6 = buf[3], *B4 = buf[4], *B5 = buf[5];
  double *U, *V;
  if (p == 13) {
    cta_mm(A2, A, A, n);
    cta_mm(A4, A2, A2, n);
    cta_mm(A6, A4, A2, n);
    cta_lin(B4, b[13], A6, b[11], A4, b[9], A2, 0.0, nullptr, 0.0, n);
    cta_mm(B5, A6, B4, n);
    cta_lin(B5, 1.0, B5, b[7], A6, b[5], A4, b[3], A2, b[1], n);
    cta_mm(B4, A, B5, n);                                   // U
    cta_lin(B5, b[12], A6, b[10], A4, b[8], A2, 0.0, nullptr, 0.0, n);
    cta_mm(A, A6, B5, n);
    cta_lin(A, 1.0, A, b[6], A6, b[4], A4, b[2], A2, b[0], n);  // V
    U = B4;
    V = A;
  } else {
    // powers A2, A4, A6, A8 as needed; V and the odd polynomial W, U = A W
    double* A8 = B4;
    cta_mm(A2, A, A, n);
    if (p >= 5) cta_mm(A4, A2, A2, n);
    if (p >= 7) cta_mm(A6, A4, A2, n);
    if (p >= 9) cta_mm(A8, A6, A2, n);
    const double* P4 = p >= 5 ? A4 : nullptr;
    const double* P6 = p >= 7 ? A6 : nullptr;
    const double* P8 = p >= 9 ? A8 : nullptr;
    // V into B5
    cta_lin(B5, b[2], A2, p >= 5 ? b[4] : 0.0, P4, p >= 7 ? b[6] : 0.0, P6,
            p >= 9 ? b[8] : 0.0, P8, b[0], n);
    // W into A8's buffer (A8 no longer needed afterwards)
    cta_lin(B4, b[3], A2, p >= 5 ? b[5] : 0.0, P4, p >= 7 ? b[7] : 0.0, P6,
            p >= 9 ? b[9] : 0.0, P8, b[1], n);
    cta_mm(A2, A, B4, n);  // U
    U = A2;
    V = B5;
  }
  // P = V - U, Q = V + U, solve P X = Q
  double* Pm = (U == A2) ? A4 : buf[1];
  double* Qm = (U == A2) ? A6 : buf[2];
  cta_lin(Pm, 1.0, V, -1.0, U, 0.0, nullptr, 0.0, nullptr, 0.0, n);
  cta_lin(Qm, 1.0, V, 1.0, U, 0.0, nullptr, 0.0, nullptr, 0.0, n);
  if (!cta_solve(Pm, Qm, n, lv, piv)) return nullptr;
  double* X = Qm;
  double* Y = (Qm == A6) ? buf[3 + 1] : buf[3];
  if (Y == X) Y = buf[5];
  for (int q = 0; q < s; ++q) {
    cta_mm(Y, X, X, n);
    double* t = X; X = Y; Y = t;
  }
  return X;
}


}  // namespace kx
