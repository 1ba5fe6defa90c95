// Yee-grid stencil of the operator A (eq. (ode)) shared by the kernels.
#pragma once

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

// Material accessors.  TableMat reads the 1/eps arrays and the sigma table
// built at context creation; CellMat derives both from the per-cell
// permittivity and the layer parameters on the fly (no precomputed arrays).
template <typename T>
struct TableMat {
  const T* __restrict__ ie;     // (ncomp - nh) x ncell
  const T* __restrict__ sig2;   // sigma at 2 * index + half along the layer axis
  __device__ __forceinline__ T inv_eps(const Geo& g, int e, int64_t idx) const {
    return ie[(int64_t)e * g.ncell + idx];
  }
  __device__ __forceinline__ T sigma(const Geo& g, const Cell& q, int c) const {
    const int li = g.la == 0 ? q.i : (g.la == 1 ? q.j : q.k);
    return sig2[2 * li + g.sighalf[c]];
  }
};

template <typename T>
struct CellMat {
  const double* __restrict__ eps;  // ncell, x fastest
  double smax;
  int L;
  // 1 / (mean permittivity of the cells whose closure holds E node e of cell idx)
  __device__ __forceinline__ T inv_eps(const Geo& g, int e, int64_t idx) const {
    const int i = (int)(idx % g.nx);
    const int64_t r = idx / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    const int im = i == 0 ? g.nx - 1 : i - 1, jm = j == 0 ? g.ny - 1 : j - 1;
    const int km = k == 0 ? g.nz - 1 : k - 1;
    const int64_t nx = g.nx, nxy = (int64_t)g.nx * g.ny;
    double s;
    if (g.dim == 2) {
      s = eps[j * nx + i] + eps[j * nx + im] + eps[jm * nx + i] + eps[jm * nx + im];
    } else if (e == 0) {   // Ex: half-integer along x
      s = eps[k * nxy + j * nx + i] + eps[k * nxy + jm * nx + i] + eps[km * nxy + j * nx + i] +
          eps[km * nxy + jm * nx + i];
    } else if (e == 1) {   // Ey: half-integer along y
      s = eps[k * nxy + j * nx + i] + eps[k * nxy + j * nx + im] + eps[km * nxy + j * nx + i] +
          eps[km * nxy + j * nx + im];
    } else {               // Ez: half-integer along z
      s = eps[k * nxy + j * nx + i] + eps[k * nxy + j * nx + im] + eps[k * nxy + jm * nx + i] +
          eps[k * nxy + jm * nx + im];
    }
    return (T)(4.0 / s);
  }
  __device__ __forceinline__ T sigma(const Geo& g, const Cell& q, int c) const {
    const int li = g.la == 0 ? q.i : (g.la == 1 ? q.j : q.k);
    const int na = g.la == 0 ? g.nx : (g.la == 1 ? g.ny : g.nz);
    const double pos = li + 0.5 * g.sighalf[c];
    const double d = fmax(fmax((double)L - pos, pos - (double)(na - L)), 0.0);
    return (T)(smax * d / (double)L);
  }
};


// Stored components per cell of a model: DIM = 2 (Hx, Hy, Ez), 3 (the six
// 3D fields), 4 (2D with the PML field P: Hx, Hy, Ez, P).
__host__ __device__ constexpr int ncomp_of(int DIM) { return DIM == 3 ? 6 : (DIM == 4 ? 4 : 3); }

// out = A v (TR = 0) or A^T v (TR = 1) at the components of one cell.
// DIM = 4 is the paper's 2D PML model (eq. (mxw)): sigma damps Hy and Ez at
// the same rate (not divided by eps), Ez' gains + P and
// P' = -(sigma / eps) dHx/dy, so the rows are
//   Hx: dEz/dy    Hy: sigma Hy - dEz/dx    Ez: sigma Ez - curl H / eps - P
//   P:  (sigma / eps) dHx/dy
// and A^T follows the blocks (with u = (w_Ez + sigma w_P) / eps on the Ez
// nodes): Hx: -du/dy, Hy: sigma w_Hy + d(w_Ez/eps)/dx, Ez: sigma w_Ez + curl
// w_H, P: -w_Ez.  sigma depends on x only.
template <typename T, int DIM, int TR, typename Mat>
__device__ __forceinline__ void stencil(const Geo& g, const T* __restrict__ v, const Mat& mat,
                                        const Cell& q, T* out) {
  const int64_t nc = g.ncell;
  const int i = q.i, j = q.j, k = q.k;
  if (DIM == 4) {
    (void)nc;
    const T Hx = ldv(g, v, 0, q.c0, i, j, k), Hy = ldv(g, v, 1, q.c0, i, j, k);
    const T Hy_im = ldv(g, v, 1, q.cim, q.im, j, k), Hx_jm = ldv(g, v, 0, q.cjm, i, q.jm, k);
    const T Ez = ldv(g, v, 2, q.c0, i, j, k), P = ldv(g, v, 3, q.c0, i, j, k);
    const T Ez_jp = ldv(g, v, 2, q.cjp, i, q.jp, k), Ez_ip = ldv(g, v, 2, q.cip, q.ip, j, k);
    const T sH = mat.sigma(g, q, 1), sE = mat.sigma(g, q, 2);
    const T ie0 = mat.inv_eps(g, 0, q.c0);
    const T curlH = (Hy - Hy_im) - (Hx - Hx_jm);
    if (!TR) {
      out[0] = Ez_jp - Ez;
      out[1] = sH * Hy - (Ez_ip - Ez);
      out[2] = sE * Ez - ie0 * curlH - P;
      out[3] = sE * ie0 * (Hx - Hx_jm);
    } else {
      const T P_jp = ldv(g, v, 3, q.cjp, i, q.jp, k);
      const T u = (Ez + sE * P) * ie0;
      const T u_jp = (Ez_jp + sE * P_jp) * mat.inv_eps(g, 0, q.cjp);
      out[0] = -(u_jp - u);
      out[1] = sH * Hy + (Ez_ip * mat.inv_eps(g, 0, q.cip) - Ez * ie0);
      out[2] = sE * Ez + curlH;
      out[3] = -Ez;
    }
  } else if (DIM == 2) {
    // components 0 Hx (0,1/2), 1 Hy (1/2,0), 2 Ez (0,0)
    const T Hx = ldv(g, v, 0, q.c0, i, j, k), Hy = ldv(g, v, 1, q.c0, i, j, k);
    const T Hy_im = ldv(g, v, 1, q.cim, q.im, j, k), Hx_jm = ldv(g, v, 0, q.cjm, i, q.jm, k);
    T Ez = ldv(g, v, 2, q.c0, i, j, k);
    T Ez_jp = ldv(g, v, 2, q.cjp, i, q.jp, k), Ez_ip = ldv(g, v, 2, q.cip, q.ip, j, k);
    const T s0 = mat.sigma(g, q, 0), s1 = mat.sigma(g, q, 1), s2 = mat.sigma(g, q, 2);
    const T curlH = (Hy - Hy_im) - (Hx - Hx_jm);
    if (!TR) {
      out[0] = s0 * Hx + (Ez_jp - Ez);
      out[1] = s1 * Hy - (Ez_ip - Ez);
      out[2] = mat.inv_eps(g, 0, q.c0) * (s2 * Ez - curlH);
    } else {
      Ez *= mat.inv_eps(g, 0, q.c0);
      Ez_jp *= mat.inv_eps(g, 0, q.cjp);
      Ez_ip *= mat.inv_eps(g, 0, q.cip);
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
    for (int c = 0; c < 6; ++c) s[c] = mat.sigma(g, q, c);
    const T cHx = (Hz - Hz_jm) - (Hy - Hy_km);
    const T cHy = (Hx - Hx_km) - (Hz - Hz_im);
    const T cHz = (Hy - Hy_im) - (Hx - Hx_jm);
    if (!TR) {
      out[0] = s[0] * Hx + ((Ez_jp - Ez) - (Ey_kp - Ey));
      out[1] = s[1] * Hy + ((Ex_kp - Ex) - (Ez_ip - Ez));
      out[2] = s[2] * Hz + ((Ey_ip - Ey) - (Ex_jp - Ex));
      out[3] = mat.inv_eps(g, 0, q.c0) * (s[3] * Ex - cHx);
      out[4] = mat.inv_eps(g, 1, q.c0) * (s[4] * Ey - cHy);
      out[5] = mat.inv_eps(g, 2, q.c0) * (s[5] * Ez - cHz);
    } else {
      Ex *= mat.inv_eps(g, 0, q.c0);
      Ey *= mat.inv_eps(g, 1, q.c0);
      Ez *= mat.inv_eps(g, 2, q.c0);
      Ez_jp *= mat.inv_eps(g, 2, q.cjp);
      Ey_kp *= mat.inv_eps(g, 1, q.ckp);
      Ex_kp *= mat.inv_eps(g, 0, q.ckp);
      Ez_ip *= mat.inv_eps(g, 2, q.cip);
      Ey_ip *= mat.inv_eps(g, 1, q.cip);
      Ex_jp *= mat.inv_eps(g, 0, q.cjp);
      out[0] = s[0] * Hx - ((Ez_jp - Ez) - (Ey_kp - Ey));
      out[1] = s[1] * Hy - ((Ex_kp - Ex) - (Ez_ip - Ez));
      out[2] = s[2] * Hz - ((Ey_ip - Ey) - (Ex_jp - Ex));
      out[3] = s[3] * Ex + cHx;
      out[4] = s[4] * Ey + cHy;
      out[5] = s[5] * Ez + cHz;
    }
  }
  constexpr int NC = ncomp_of(DIM);
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if (is_wall(g, c, i, j, k)) out[c] = T(0);
}


// ---------------------------------------------------------------------------
// The 3D lossy-layer model in FP32 on four consecutive x-cells (a quad;
// nx % 4 == 0): every field and 1/eps access is one 16-byte load, the
// x-neighbours of the quad's end cells are one scalar each.
__device__ __forceinline__ float4 ld4(const float* __restrict__ p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ float f4(const float4& v, int e) { return e == 0 ? v.x : (e == 1 ? v.y : (e == 2 ? v.z : v.w)); }
__device__ __forceinline__ void set4(float4& v, int e, float x) {
  if (e == 0) v.x = x; else if (e == 1) v.y = x; else if (e == 2) v.z = x; else v.w = x;
}
__device__ __forceinline__ float dot4(const float4& a, const float4& b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}
// zero the elements of a quad that lie on a wall of component c
__device__ __forceinline__ float4 wall4(const Geo& g, int c, float4 v, int i0, int j, int k) {
  const unsigned mb = g.maskbits[c];
  if (((mb & 2u) && j == 0) || ((mb & 4u) && k == 0)) return make_float4(0.f, 0.f, 0.f, 0.f);
  if ((mb & 1u) && i0 == 0) v.x = 0.f;
  return v;
}
__device__ __forceinline__ float wall1(const Geo& g, int c, float v, int i, int j, int k) {
  return is_wall(g, c, i, j, k) ? 0.f : v;
}

struct Quad {
  int64_t c0;      // first cell
  int i0, jj, kk;  // its indices
};

__device__ __forceinline__ Quad make_quad(const Geo& g, int64_t q4) {
  Quad q;
  q.c0 = q4 << 2;
  q.i0 = (int)(q.c0 % g.nx);
  const int64_t r = q.c0 / g.nx;
  q.jj = (int)(r % g.ny);
  q.kk = (int)(r / g.ny);
  return q;
}

// out[c] = component c of A v on the quad's four cells (wall nodes zero);
// the rows of eq. (ode) as in stencil<float, 3, 0, TableMat<float>>.
__device__ __forceinline__ void stencil_quad(const Geo& g, const float* __restrict__ v, const float* __restrict__ ie,
                                             const float* __restrict__ sig2, const Quad& q, float4 out[6]) {
  const int64_t nc = g.ncell;
  const int64_t nxy = (int64_t)g.nx * g.ny;
  const int64_t c0 = q.c0;
  const int i0 = q.i0, jj = q.jj, kk = q.kk;
  const int jp = (jj + 1 == g.ny) ? 0 : jj + 1, jm = (jj == 0) ? g.ny - 1 : jj - 1;
  const int kp = (kk + 1 == g.nz) ? 0 : kk + 1, km = (kk == 0) ? g.nz - 1 : kk - 1;
  const int64_t cjp = c0 + (int64_t)(jp - jj) * g.nx, cjm = c0 + (int64_t)(jm - jj) * g.nx;
  const int64_t ckp = c0 + (int64_t)(kp - kk) * nxy, ckm = c0 + (int64_t)(km - kk) * nxy;
  const int ixp = (i0 + 4 == g.nx) ? 0 : i0 + 4;     // first element of the next quad
  const int ixm = (i0 == 0) ? g.nx - 1 : i0 - 1;     // element before the quad
  const int64_t cxp = c0 - i0 + ixp, cxm = c0 - i0 + ixm;
  const float4 Hx = wall4(g, 0, ld4(v + c0), i0, jj, kk);
  const float4 Hy = wall4(g, 1, ld4(v + nc + c0), i0, jj, kk);
  const float4 Hz = wall4(g, 2, ld4(v + 2 * nc + c0), i0, jj, kk);
  const float4 Ex = wall4(g, 3, ld4(v + 3 * nc + c0), i0, jj, kk);
  const float4 Ey = wall4(g, 4, ld4(v + 4 * nc + c0), i0, jj, kk);
  const float4 Ez = wall4(g, 5, ld4(v + 5 * nc + c0), i0, jj, kk);
  const float4 Ez_jp = wall4(g, 5, ld4(v + 5 * nc + cjp), i0, jp, kk);
  const float4 Ex_jp = wall4(g, 3, ld4(v + 3 * nc + cjp), i0, jp, kk);
  const float4 Ey_kp = wall4(g, 4, ld4(v + 4 * nc + ckp), i0, jj, kp);
  const float4 Ex_kp = wall4(g, 3, ld4(v + 3 * nc + ckp), i0, jj, kp);
  const float4 Hz_jm = wall4(g, 2, ld4(v + 2 * nc + cjm), i0, jm, kk);
  const float4 Hx_jm = wall4(g, 0, ld4(v + cjm), i0, jm, kk);
  const float4 Hy_km = wall4(g, 1, ld4(v + nc + ckm), i0, jj, km);
  const float4 Hx_km = wall4(g, 0, ld4(v + ckm), i0, jj, km);
  const float Ez_n = wall1(g, 5, v[5 * nc + cxp], ixp, jj, kk);
  const float Ey_n = wall1(g, 4, v[4 * nc + cxp], ixp, jj, kk);
  const float Hz_p = wall1(g, 2, v[2 * nc + cxm], ixm, jj, kk);
  const float Hy_p = wall1(g, 1, v[nc + cxm], ixm, jj, kk);
  const float4 ie0 = ld4(ie + c0), ie1 = ld4(ie + nc + c0), ie2 = ld4(ie + 2 * nc + c0);
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    const int i = i0 + e;
    const int li = g.la == 0 ? i : (g.la == 1 ? jj : kk);
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
    float o[6];
    o[0] = sg[0] * hx + ((f4(Ez_jp, e) - ez) - (f4(Ey_kp, e) - ey));
    o[1] = sg[1] * hy + ((f4(Ex_kp, e) - ex) - (ez_ip - ez));
    o[2] = sg[2] * hz + ((ey_ip - ey) - (f4(Ex_jp, e) - ex));
    o[3] = f4(ie0, e) * (sg[3] * ex - cHx);
    o[4] = f4(ie1, e) * (sg[4] * ey - cHy);
    o[5] = f4(ie2, e) * (sg[5] * ez - cHz);
#pragma unroll
    for (int c = 0; c < 6; ++c) set4(out[c], e, is_wall(g, c, i, jj, kk) ? 0.f : o[c]);
  }
}

// Wall bits of the six components along one axis: bit c set when index 0
// along axis a is a wall node of component c.
__device__ __forceinline__ unsigned wall_bits(const Geo& g, int a) {
  unsigned m = 0u;
#pragma unroll
  for (int c = 0; c < 6; ++c) m |= ((g.maskbits[c] >> a) & 1u) << c;
  return m;
}

// Load of component c at offset idx, zero where bit c of the wall mask w is set.
__device__ __forceinline__ float ldw(const float* __restrict__ p, int idx, unsigned w, int c) {
  return (w >> c) & 1u ? 0.f : p[idx];
}

// t = A v, 3D FP32 lossy-layer model, for the cells of grid column col =
// i + nx j on planes k0 .. k1-1 (0 <= k0 < k1 <= nz): the rows of
// stencil_quad with the same operations in the same order (the same bits
// on every cell), the index and wall work done once per column and, marching
// up in z, E_x, E_y of plane k+1 and H_x, H_y of plane k kept in registers,
// where the next plane reads them as its own and its k-1 values (14 field
// loads a cell instead of 18).  32-bit cell offsets: ncell < 2^31.
__device__ __forceinline__ void stencil_column32(const Geo& g, const float* __restrict__ v,
                                                 const float* __restrict__ ie, const float* __restrict__ sig2,
                                                 float* __restrict__ t, int col, int k0, int k1) {
  const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny;
  const int nc = (int)g.ncell;
  const int i = col % nx, j = col / nx;
  const int ip = i + 1 == nx ? 0 : i + 1, im = i == 0 ? nx - 1 : i - 1;
  const int jp = j + 1 == ny ? 0 : j + 1, jm = j == 0 ? ny - 1 : j - 1;
  const int dip = ip - i, dim = im - i, djp = (jp - j) * nx, djm = (jm - j) * nx;
  const unsigned xm = wall_bits(g, 0), ym = wall_bits(g, 1), zm = wall_bits(g, 2);
  // wall masks of the columns read: (i, j), (ip, j), (im, j), (i, jp), (i, jm)
  const unsigned wc = (i == 0 ? xm : 0u) | (j == 0 ? ym : 0u);
  const unsigned wip = (ip == 0 ? xm : 0u) | (j == 0 ? ym : 0u);
  const unsigned wim = (im == 0 ? xm : 0u) | (j == 0 ? ym : 0u);
  const unsigned wjp = (i == 0 ? xm : 0u) | (jp == 0 ? ym : 0u);
  const unsigned wjm = (i == 0 ? xm : 0u) | (jm == 0 ? ym : 0u);
  const float* __restrict__ vHx = v;
  const float* __restrict__ vHy = v + nc;
  const float* __restrict__ vHz = v + 2 * (int64_t)nc;
  const float* __restrict__ vEx = v + 3 * (int64_t)nc;
  const float* __restrict__ vEy = v + 4 * (int64_t)nc;
  const float* __restrict__ vEz = v + 5 * (int64_t)nc;
  const int km0 = k0 == 0 ? nz - 1 : k0 - 1;
  unsigned zk = k0 == 0 ? zm : 0u;
  int cell = col + k0 * nxy;
  const int ckm0 = col + km0 * nxy;
  const unsigned wkm0 = wc | (km0 == 0 ? zm : 0u);
  float hx_km = ldw(vHx, ckm0, wkm0, 0), hy_km = ldw(vHy, ckm0, wkm0, 1);
  float ex = ldw(vEx, cell, wc | zk, 3), ey = ldw(vEy, cell, wc | zk, 4);
  for (int k = k0; k < k1; ++k, cell += nxy) {
    const int kp = k + 1 == nz ? 0 : k + 1;
    const unsigned zkp = kp == 0 ? zm : 0u;
    const int ckp = col + kp * nxy;
    const unsigned mk = wc | zk, mkp = wc | zkp;
    const float hx = ldw(vHx, cell, mk, 0), hy = ldw(vHy, cell, mk, 1);
    const float hz = ldw(vHz, cell, mk, 2), ez = ldw(vEz, cell, mk, 5);
    const float ex_kp = ldw(vEx, ckp, mkp, 3), ey_kp = ldw(vEy, ckp, mkp, 4);
    const float ez_jp = ldw(vEz, cell + djp, wjp | zk, 5), ex_jp = ldw(vEx, cell + djp, wjp | zk, 3);
    const float hz_jm = ldw(vHz, cell + djm, wjm | zk, 2), hx_jm = ldw(vHx, cell + djm, wjm | zk, 0);
    const float ez_ip = ldw(vEz, cell + dip, wip | zk, 5), ey_ip = ldw(vEy, cell + dip, wip | zk, 4);
    const float hz_im = ldw(vHz, cell + dim, wim | zk, 2), hy_im = ldw(vHy, cell + dim, wim | zk, 1);
    const int li = g.la == 0 ? i : (g.la == 1 ? j : k);
    float sg[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) sg[c] = sig2[2 * li + g.sighalf[c]];
    const float cHx = (hz - hz_jm) - (hy - hy_km);
    const float cHy = (hx - hx_km) - (hz - hz_im);
    const float cHz = (hy - hy_im) - (hx - hx_jm);
    float o[6];
    o[0] = sg[0] * hx + ((ez_jp - ez) - (ey_kp - ey));
    o[1] = sg[1] * hy + ((ex_kp - ex) - (ez_ip - ez));
    o[2] = sg[2] * hz + ((ey_ip - ey) - (ex_jp - ex));
    o[3] = ie[cell] * (sg[3] * ex - cHx);
    o[4] = ie[(int64_t)nc + cell] * (sg[4] * ey - cHy);
    o[5] = ie[2 * (int64_t)nc + cell] * (sg[5] * ez - cHz);
#pragma unroll
    for (int c = 0; c < 6; ++c) t[c * (int64_t)nc + cell] = (mk >> c) & 1u ? 0.f : o[c];
    hx_km = hx;
    hy_km = hy;
    ex = ex_kp;
    ey = ey_kp;
    zk = zkp;
  }
}

// Sixteen-byte load of four x-cells of component c at offset idx (a
// multiple of 4), zero where the wall mask says so: w0 for the first cell,
// w1 for the other three (only index 0 along x can be a wall).
__device__ __forceinline__ float4 ldw4(const float* __restrict__ p, int idx, unsigned w0, unsigned w1, int c) {
  float4 r = *reinterpret_cast<const float4*>(p + idx);
  if ((w0 >> c) & 1u) r.x = 0.f;
  if ((w1 >> c) & 1u) {
    r.y = 0.f;
    r.z = 0.f;
    r.w = 0.f;
  }
  return r;
}

// The column march of stencil_column32 on a quad of x-cells (nx % 4 == 0):
// quad column q = i0/4 + (nx/4) j, planes k0 .. k1-1; sixteen-byte loads
// and stores, the x neighbours outside the quad by one scalar load each
// side, the arithmetic of stencil_quad on every cell (the same bits).
__device__ __forceinline__ void stencil_column_quad(const Geo& g, const float* __restrict__ v,
                                                    const float* __restrict__ ie, const float* __restrict__ sig2,
                                                    float* __restrict__ t, int q, int k0, int k1) {
  const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny, nqx = nx >> 2;
  const int nc = (int)g.ncell;
  const int j = q / nqx, i0 = (q - j * nqx) << 2;
  const int col = i0 + j * nx;
  const int jp = j + 1 == ny ? 0 : j + 1, jm = j == 0 ? ny - 1 : j - 1;
  const int ixp = i0 + 4 == nx ? 0 : i0 + 4, ixm = i0 == 0 ? nx - 1 : i0 - 1;
  const int dxp = ixp - i0, dxm = ixm - i0, djp = (jp - j) * nx, djm = (jm - j) * nx;
  const unsigned xm = wall_bits(g, 0), ym = wall_bits(g, 1), zm = wall_bits(g, 2);
  const unsigned wy = j == 0 ? ym : 0u, wyp = jp == 0 ? ym : 0u, wym = jm == 0 ? ym : 0u;
  const unsigned wx0 = i0 == 0 ? xm : 0u;
  // first cell / other three cells of the quad columns read: (i0, j), (i0, jp), (i0, jm)
  const unsigned c0 = wx0 | wy, c1 = wy, p0 = wx0 | wyp, p1 = wyp, m0 = wx0 | wym, m1 = wym;
  const unsigned wxp = (ixp == 0 ? xm : 0u) | wy, wxm = (ixm == 0 ? xm : 0u) | wy;
  const float* __restrict__ vHx = v;
  const float* __restrict__ vHy = v + nc;
  const float* __restrict__ vHz = v + 2 * (int64_t)nc;
  const float* __restrict__ vEx = v + 3 * (int64_t)nc;
  const float* __restrict__ vEy = v + 4 * (int64_t)nc;
  const float* __restrict__ vEz = v + 5 * (int64_t)nc;
  const float* __restrict__ ie1 = ie + nc;
  const float* __restrict__ ie2 = ie + 2 * (int64_t)nc;
  const int km0 = k0 == 0 ? nz - 1 : k0 - 1;
  unsigned zk = k0 == 0 ? zm : 0u;
  int cell = col + k0 * nxy;
  const int ckm0 = col + km0 * nxy;
  const unsigned zkm0 = km0 == 0 ? zm : 0u;
  float4 Hx_km = ldw4(vHx, ckm0, c0 | zkm0, c1 | zkm0, 0), Hy_km = ldw4(vHy, ckm0, c0 | zkm0, c1 | zkm0, 1);
  float4 Ex = ldw4(vEx, cell, c0 | zk, c1 | zk, 3), Ey = ldw4(vEy, cell, c0 | zk, c1 | zk, 4);
  for (int k = k0; k < k1; ++k, cell += nxy) {
    const int kp = k + 1 == nz ? 0 : k + 1;
    const unsigned zkp = kp == 0 ? zm : 0u;
    const int ckp = col + kp * nxy;
    const float4 Hx = ldw4(vHx, cell, c0 | zk, c1 | zk, 0), Hy = ldw4(vHy, cell, c0 | zk, c1 | zk, 1);
    const float4 Hz = ldw4(vHz, cell, c0 | zk, c1 | zk, 2), Ez = ldw4(vEz, cell, c0 | zk, c1 | zk, 5);
    const float4 Ex_kp = ldw4(vEx, ckp, c0 | zkp, c1 | zkp, 3), Ey_kp = ldw4(vEy, ckp, c0 | zkp, c1 | zkp, 4);
    const float4 Ez_jp = ldw4(vEz, cell + djp, p0 | zk, p1 | zk, 5);
    const float4 Ex_jp = ldw4(vEx, cell + djp, p0 | zk, p1 | zk, 3);
    const float4 Hz_jm = ldw4(vHz, cell + djm, m0 | zk, m1 | zk, 2);
    const float4 Hx_jm = ldw4(vHx, cell + djm, m0 | zk, m1 | zk, 0);
    const float Ez_n = ldw(vEz, cell + dxp, wxp | zk, 5), Ey_n = ldw(vEy, cell + dxp, wxp | zk, 4);
    const float Hz_p = ldw(vHz, cell + dxm, wxm | zk, 2), Hy_p = ldw(vHy, cell + dxm, wxm | zk, 1);
    const float4 ie0q = ld4(ie + cell), ie1q = ld4(ie1 + cell), ie2q = ld4(ie2 + cell);
    float4 out[6];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int li = g.la == 0 ? i0 + e : (g.la == 1 ? j : k);
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
      float o[6];
      o[0] = sg[0] * hx + ((f4(Ez_jp, e) - ez) - (f4(Ey_kp, e) - ey));
      o[1] = sg[1] * hy + ((f4(Ex_kp, e) - ex) - (ez_ip - ez));
      o[2] = sg[2] * hz + ((ey_ip - ey) - (f4(Ex_jp, e) - ex));
      o[3] = f4(ie0q, e) * (sg[3] * ex - cHx);
      o[4] = f4(ie1q, e) * (sg[4] * ey - cHy);
      o[5] = f4(ie2q, e) * (sg[5] * ez - cHz);
      const unsigned me = (e == 0 ? c0 : c1) | zk;
#pragma unroll
      for (int c = 0; c < 6; ++c) set4(out[c], e, (me >> c) & 1u ? 0.f : o[c]);
    }
#pragma unroll
    for (int c = 0; c < 6; ++c) *reinterpret_cast<float4*>(t + c * (int64_t)nc + cell) = out[c];
    Hx_km = Hx;
    Hy_km = Hy;
    Ex = Ex_kp;
    Ey = Ey_kp;
    zk = zkp;
  }
}

// stencil_quad on the quad whose first cell is c0 (a multiple of 4, nx % 4
// == 0, ncell < 2^31), with 32-bit index arithmetic and the wall tests as
// per-component bit masks (the same operations on the field values, so the
// same bits); the sigma values are read once per quad unless the layer axis
// is x.  At the start of each tile of the single sweep this is the part that
// keeps the block from streaming; the 64-bit divisions and per-value wall
// tests of stencil_quad made it about twice as long.
__device__ __forceinline__ void stencil_quad32(const Geo& g, const float* __restrict__ v, const float* __restrict__ ie,
                                               const float* __restrict__ sig2, int c0, float4 out[6]) {
  const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny, nc = (int)g.ncell;
  const unsigned r = (unsigned)c0 / (unsigned)nx;
  const int i0 = c0 - (int)r * nx;
  const unsigned kq = r / (unsigned)ny;
  const int jj = (int)r - (int)kq * ny, kk = (int)kq;
  const int jp = (jj + 1 == ny) ? 0 : jj + 1, jm = (jj == 0) ? ny - 1 : jj - 1;
  const int kp = (kk + 1 == nz) ? 0 : kk + 1, km = (kk == 0) ? nz - 1 : kk - 1;
  const int cjp = c0 + (jp - jj) * nx, cjm = c0 + (jm - jj) * nx;
  const int ckp = c0 + (kp - kk) * nxy, ckm = c0 + (km - kk) * nxy;
  const int ixp = (i0 + 4 == nx) ? 0 : i0 + 4, ixm = (i0 == 0) ? nx - 1 : i0 - 1;
  const int cxp = c0 - i0 + ixp, cxm = c0 - i0 + ixm;
  const unsigned xm = wall_bits(g, 0), ym = wall_bits(g, 1), zm = wall_bits(g, 2);
  const unsigned wx0 = i0 == 0 ? xm : 0u, wy = jj == 0 ? ym : 0u, wz = kk == 0 ? zm : 0u;
  const unsigned wyp = jp == 0 ? ym : 0u, wym = jm == 0 ? ym : 0u, wzp = kp == 0 ? zm : 0u, wzm = km == 0 ? zm : 0u;
  const unsigned o0 = wx0 | wy | wz, o1 = wy | wz;   // the quad's first cell / the other three
  const float* __restrict__ vHx = v;
  const float* __restrict__ vHy = v + nc;
  const float* __restrict__ vHz = v + 2 * (int64_t)nc;
  const float* __restrict__ vEx = v + 3 * (int64_t)nc;
  const float* __restrict__ vEy = v + 4 * (int64_t)nc;
  const float* __restrict__ vEz = v + 5 * (int64_t)nc;
  const float4 Hx = ldw4(vHx, c0, o0, o1, 0), Hy = ldw4(vHy, c0, o0, o1, 1), Hz = ldw4(vHz, c0, o0, o1, 2);
  const float4 Ex = ldw4(vEx, c0, o0, o1, 3), Ey = ldw4(vEy, c0, o0, o1, 4), Ez = ldw4(vEz, c0, o0, o1, 5);
  const float4 Ez_jp = ldw4(vEz, cjp, wx0 | wyp | wz, wyp | wz, 5), Ex_jp = ldw4(vEx, cjp, wx0 | wyp | wz, wyp | wz, 3);
  const float4 Ey_kp = ldw4(vEy, ckp, wx0 | wy | wzp, wy | wzp, 4), Ex_kp = ldw4(vEx, ckp, wx0 | wy | wzp, wy | wzp, 3);
  const float4 Hz_jm = ldw4(vHz, cjm, wx0 | wym | wz, wym | wz, 2), Hx_jm = ldw4(vHx, cjm, wx0 | wym | wz, wym | wz, 0);
  const float4 Hy_km = ldw4(vHy, ckm, wx0 | wy | wzm, wy | wzm, 1), Hx_km = ldw4(vHx, ckm, wx0 | wy | wzm, wy | wzm, 0);
  const unsigned wxp = (ixp == 0 ? xm : 0u) | wy | wz, wxm = (ixm == 0 ? xm : 0u) | wy | wz;
  const float Ez_n = ldw(vEz, cxp, wxp, 5), Ey_n = ldw(vEy, cxp, wxp, 4);
  const float Hz_p = ldw(vHz, cxm, wxm, 2), Hy_p = ldw(vHy, cxm, wxm, 1);
  const float4 ie0 = ld4(ie + c0), ie1 = ld4(ie + nc + c0), ie2 = ld4(ie + 2 * (int64_t)nc + c0);
  float sgq[6];
  if (g.la != 0) {
    const int li = g.la == 1 ? jj : kk;
#pragma unroll
    for (int c = 0; c < 6; ++c) sgq[c] = sig2[2 * li + g.sighalf[c]];
  }
#pragma unroll
  for (int e = 0; e < 4; ++e) {
    float sg[6];
#pragma unroll
    for (int c = 0; c < 6; ++c) sg[c] = g.la == 0 ? sig2[2 * (i0 + e) + g.sighalf[c]] : sgq[c];
    const float ez = f4(Ez, e), ey = f4(Ey, e), ex = f4(Ex, e);
    const float hx = f4(Hx, e), hy = f4(Hy, e), hz = f4(Hz, e);
    const float ez_ip = e < 3 ? f4(Ez, e + 1) : Ez_n;
    const float ey_ip = e < 3 ? f4(Ey, e + 1) : Ey_n;
    const float hz_im = e > 0 ? f4(Hz, e - 1) : Hz_p;
    const float hy_im = e > 0 ? f4(Hy, e - 1) : Hy_p;
    const float cHx = (hz - f4(Hz_jm, e)) - (hy - f4(Hy_km, e));
    const float cHy = (hx - f4(Hx_km, e)) - (hz - hz_im);
    const float cHz = (hy - hy_im) - (hx - f4(Hx_jm, e));
    float o[6];
    o[0] = sg[0] * hx + ((f4(Ez_jp, e) - ez) - (f4(Ey_kp, e) - ey));
    o[1] = sg[1] * hy + ((f4(Ex_kp, e) - ex) - (ez_ip - ez));
    o[2] = sg[2] * hz + ((ey_ip - ey) - (f4(Ex_jp, e) - ex));
    o[3] = f4(ie0, e) * (sg[3] * ex - cHx);
    o[4] = f4(ie1, e) * (sg[4] * ey - cHy);
    o[5] = f4(ie2, e) * (sg[5] * ez - cHz);
    const unsigned me = e == 0 ? o0 : o1;
#pragma unroll
    for (int c = 0; c < 6; ++c) set4(out[c], e, (me >> c) & 1u ? 0.f : o[c]);
  }
}

__device__ __forceinline__ void prefetch_l2(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// L2 prefetch of the lines stencil_quad32 reads for the quad whose first
// cell is c0 (its own six components, the y and z neighbours it uses, the
// three 1/eps rows): issued a tile ahead, it lets the single sweep keep the
// next tile's stencil loads off DRAM.  32-bit index arithmetic (ncell < 2^31).
__device__ __forceinline__ void prefetch_quad32(const Geo& g, const float* v, const float* ie, int c0) {
  const int nx = g.nx, ny = g.ny, nz = g.nz, nxy = nx * ny, nc = (int)g.ncell;
  const unsigned r = (unsigned)c0 / (unsigned)nx;
  const unsigned kq = r / (unsigned)ny;
  const int jj = (int)r - (int)kq * ny, kk = (int)kq;
  const int jp = (jj + 1 == ny) ? 0 : jj + 1, jm = (jj == 0) ? ny - 1 : jj - 1;
  const int kp = (kk + 1 == nz) ? 0 : kk + 1, km = (kk == 0) ? nz - 1 : kk - 1;
  const int cjp = c0 + (jp - jj) * nx, cjm = c0 + (jm - jj) * nx;
  const int ckp = c0 + (kp - kk) * nxy, ckm = c0 + (km - kk) * nxy;
#pragma unroll
  for (int c = 0; c < 6; ++c) prefetch_l2(v + c * (int64_t)nc + c0);
  prefetch_l2(v + 5 * (int64_t)nc + cjp);
  prefetch_l2(v + 3 * (int64_t)nc + cjp);
  prefetch_l2(v + 4 * (int64_t)nc + ckp);
  prefetch_l2(v + 3 * (int64_t)nc + ckp);
  prefetch_l2(v + 2 * (int64_t)nc + cjm);
  prefetch_l2(v + cjm);
  prefetch_l2(v + nc + ckm);
  prefetch_l2(v + ckm);
#pragma unroll
  for (int e = 0; e < 3; ++e) prefetch_l2(ie + e * (int64_t)nc + c0);
}

}  // namespace kx
