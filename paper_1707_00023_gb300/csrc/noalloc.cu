// Allocation-free Arnoldi entry point (kx_arnoldi_noalloc, declared in
// include/kx.h).
//
// Some callers cannot allocate device memory: code running inside another
// runtime's memory pool, plug-ins handed a fixed arena, or hosts that forbid
// cudaMalloc/cudaFree after start-up.  This entry point needs no
// context and allocates nothing.  The caller passes every input and output
// (the permittivity per cell, the start vector, the basis and Hessenberg
// arrays); the basis array doubles as the Krylov workspace, and the remaining
// scratch (block partial sums, column scales, the step state and a
// completion counter) lives in one file-scope device array of fixed size.
//
// That array is shared by every call on a device and keeps the last call's
// contents; each call clears the parts that must start at zero.  Calls whose
// work overlaps on the GPU (different streams, or host threads without
// ordering) race on it.  Every GPU that loads the library holds the array
// until the process exits.
#include <atomic>
#include <cstring>

#include <cmath>

#include "kx_internal.cuh"

// The scratch array (file scope, internal linkage).
static __device__ __align__(256) unsigned char g_noalloc_scratch[KX_NOALLOC_SCRATCH_BYTES];

namespace {

using namespace kx;

// Partial-sum columns: PCOLS columns of up to PS_MAX blocks each.
constexpr int PS_MAX = 2432;
constexpr size_t PART_BYTES = (size_t)PCOLS * PS_MAX * sizeof(double);
constexpr size_t SCALE_OFF = PART_BYTES;
constexpr size_t AUG_OFF = SCALE_OFF + (MMAX + 2) * sizeof(double);
constexpr size_t U_OFF = AUG_OFF + (MMAX + 1) * 2 * sizeof(double);
constexpr size_t STATE_OFF = U_OFF + (MMAX + 2) * sizeof(double);
constexpr size_t COUNTER_OFF = (STATE_OFF + sizeof(SlotState) + 255) / 256 * 256;
constexpr size_t SCRATCH_USED = COUNTER_OFF + 8 * sizeof(unsigned);

static_assert(SCRATCH_USED <= KX_NOALLOC_SCRATCH_BYTES, "scratch layout exceeds the static array");

// Device address of the array, per device (host code cannot use the symbol
// itself: in host code it names a host-side stand-in).  Host threads may
// fill an entry at the same time; they store the same address.
constexpr int MAX_DEVICES = 64;
std::atomic<void*> g_scratch_addr[MAX_DEVICES];

thread_local char g_err[512] = {0};

kx_status err(kx_status code, const char* msg) {
  snprintf(g_err, sizeof(g_err), "%s", msg);
  return code;
}

kx_status cuda_err(cudaError_t e, const char* what) {
  snprintf(g_err, sizeof(g_err), "%s: %s", what, cudaGetErrorString(e));
  return KX_ECUDA;
}

// Set-up, once per device with that device current.
kx_status scratch_for_current_device(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return err(KX_EINVAL, "device index beyond 64");
  void* p = g_scratch_addr[dev].load(std::memory_order_acquire);
  if (!p) {
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_err(e, "cudaGetSymbolAddress of the scratch array");
    g_scratch_addr[dev].store(p, std::memory_order_release);
  }
  *out = p;
  return KX_OK;
}

}  // namespace

extern "C" kx_status kx_arnoldi_noalloc(const kx_desc* desc, const double* d_eps_cell, const void* d_v0,
                                        int m, void* d_V, double* d_H, double* beta, int* m_done,
                                        void* cuda_stream) {
  g_err[0] = 0;
  if (!desc || !d_eps_cell || !d_v0 || !d_V || !d_H || !beta || !m_done)
    return err(KX_EINVAL, "NULL argument");
  const kx_desc& d = *desc;
  if (m < 1 || m > MMAX) return err(KX_EINVAL, "m must be 1..64 (the scratch array holds 64 columns)");
  if (d.dim != 2 && d.dim != 3) return err(KX_EINVAL, "dim must be 2 or 3");
  for (int a = 0; a < d.dim; ++a) {
    if (d.n[a] < 3) return err(KX_EINVAL, "each n[a] must be >= 3");
    if (d.bc[a] != KX_PERIODIC && d.bc[a] != KX_PEC) return err(KX_EINVAL, "bad bc");
  }
  if (d.layer_axis < 0 || d.layer_axis >= d.dim || d.layer_cells < 1 ||
      2 * d.layer_cells > d.n[d.layer_axis] || !(d.sigma_max >= 0.0))
    return err(KX_EINVAL, "bad absorbing layer");
  if (d.precision != KX_FP64 && d.precision != KX_FP32) return err(KX_EINVAL, "bad precision");
  if (d.pml != 0) return err(KX_EINVAL, "the PML model is not available here (pml must be 0)");
  const int esize = d.precision == KX_FP64 ? 8 : 4;
  const int nz = d.dim == 3 ? d.n[2] : 1;
  const int64_t ncell = (int64_t)d.n[0] * d.n[1] * nz;
  const int ncomp = d.dim == 2 ? 3 : 6;
  const int64_t n = ncomp * ncell;
  if ((n * esize) % 16 != 0 || ((uintptr_t)d_V % 16) != 0)
    return err(KX_EINVAL, "the basis columns must be 16-byte aligned: n * sizeof(scalar) a multiple of 16 "
                          "and d_V 16-byte aligned");

  void* scratch = nullptr;
  kx_status st = scratch_for_current_device(&scratch);
  if (st != KX_OK) return st;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return cuda_err(e, "device query");

  // A context on the stack whose workspace points into the caller's arrays
  // and the static scratch: the shared launchers then allocate nothing.
  kx_ctx c{};
  c.d = d;
  if (d.dim == 2) c.d.n[2] = 1;
  c.stream = (cudaStream_t)cuda_stream;
  Geo& g = c.geo;
  g.dim = d.dim;
  g.nx = d.n[0];
  g.ny = d.n[1];
  g.nz = nz;
  g.ncell = ncell;
  g.ncomp = ncomp;
  g.nh = d.dim == 2 ? 2 : 3;
  g.ne = d.dim == 2 ? 1 : 3;
  g.la = d.layer_axis;
  static const int off2[3][3] = {{0, 1, 0}, {1, 0, 0}, {0, 0, 0}};
  static const int off3[6][3] = {{0, 1, 1}, {1, 0, 1}, {1, 1, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int comp = 0; comp < ncomp; ++comp) {
    const int* off = d.dim == 2 ? off2[comp] : off3[comp];
    unsigned mb = 0;
    for (int a = 0; a < d.dim; ++a)
      if (d.bc[a] == KX_PEC && off[a] == 0) mb |= 1u << a;
    g.maskbits[comp] = mb;
    g.sighalf[comp] = off[d.layer_axis];
  }
  c.n = n;
  c.esize = esize;
  c.ld = n;
  c.m = m;
  c.nsm = nsm;
  c.ps = nsm * 16 < PS_MAX ? nsm * 16 : PS_MAX;
  const int64_t want = (ncell + NTHREADS - 1) / NTHREADS;
  c.nblk = (int)(want < c.ps ? want : c.ps);
  unsigned char* base = (unsigned char*)scratch;
  c.d_V = d_V;
  c.d_H = d_H;
  c.d_part = (double*)base;
  c.d_scale = (double*)(base + SCALE_OFF);
  c.d_aug = (double*)(base + AUG_OFF);
  c.d_u = (double*)(base + U_OFF);
  c.d_state = (SlotState*)(base + STATE_OFF);
  c.d_counter = (unsigned*)(base + COUNTER_OFF);
  std::memset(&c.stats, 0, sizeof(c.stats));

  // clear what must start at zero: step state, counter, augmented entries, H
  e = cudaMemsetAsync(c.d_state, 0, sizeof(SlotState), c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.d_counter, 0, 8 * sizeof(unsigned), c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.d_aug, 0, (MMAX + 1) * 2 * sizeof(double), c.stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(d_H, 0, (size_t)(m + 1) * m * sizeof(double), c.stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_V, d_v0, (size_t)n * esize, cudaMemcpyDeviceToDevice, c.stream);
  if (e != cudaSuccess) return cuda_err(e, "scratch initialisation");

  if ((st = launch_norm_init(&c, 0, 1)) != KX_OK) return err(st, c.err);
  // refuse a zero or non-finite start vector before any step (as arnoldi() does)
  SlotState hs;
  e = cudaMemcpyAsync(&hs, c.d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_err(e, "start-vector norm read-back");
  if (!(hs.beta > 0.0) || !std::isfinite(hs.beta)) return err(KX_ENONFINITE, "v0 is zero or non-finite");
  for (int j = 0; j < m; ++j) {
    if ((st = launch_pass_a_cells(&c, 0, j, d_eps_cell)) != KX_OK) return err(st, c.err);
    if ((st = launch_pass_b(&c, 0, 1, j, j == m - 1)) != KX_OK) return err(st, c.err);
  }
  // normalise the basis in place (the stored columns carry their scales)
  if ((st = launch_basis_export(&c, 0, d_V, m)) != KX_OK) return err(st, c.err);
  e = cudaMemcpyAsync(&hs, c.d_state, sizeof(SlotState), cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return cuda_err(e, "result read-back");
  if (hs.status) return err((kx_status)hs.status, "non-finite value in the Arnoldi process");
  *beta = hs.beta;
  *m_done = hs.m_done;
  return KX_OK;
}

extern "C" const char* kx_noalloc_last_error(void) { return g_err; }
