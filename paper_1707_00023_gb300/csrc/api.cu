// C ABI of the library (declared in include/kx.h): context set-up and the
// host-side drivers of the Krylov methods.  Every numerical step runs in the
// library's kernels; the host only sequences launches on the context's
// stream and reads back small status records.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>
#include <vector>

#include "kx_internal.cuh"

using namespace kx;

namespace {

thread_local std::string g_create_err;

kx_status fail(kx_ctx* c, kx_status code, const std::string& msg) {
  if (c) snprintf(c->err, sizeof(c->err), "%s", msg.c_str());
  else g_create_err = msg;
  return code;
}

kx_status cuda_fail(kx_ctx* c, cudaError_t e, const char* what) {
  return fail(c, KX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

#define KX_TRY(expr)              \
  do {                            \
    kx_status s__ = (expr);       \
    if (s__ != KX_OK) return s__; \
  } while (0)

#define KX_CUDA(c, expr, what)                      \
  do {                                              \
    cudaError_t e__ = (expr);                       \
    if (e__ != cudaSuccess) return cuda_fail((c), e__, (what)); \
  } while (0)

void* vec_ptr(kx_ctx* c, void* base, int64_t col) {
  return (char*)base + col * c->n * c->esize;
}

void* slot_col(kx_ctx* c, int slot, int col) {
  return (char*)c->d_V + ((int64_t)slot * (c->m + 1) + col) * c->ld * c->esize;
}

kx_status sync(kx_ctx* c) {
  KX_CUDA(c, cudaStreamSynchronize(c->stream), "stream synchronise");
  return KX_OK;
}

kx_status upload_state(kx_ctx* c, int slot, const SlotState& s) {
  c->h_state[slot] = s;
  KX_CUDA(c, cudaMemcpyAsync(c->d_state + slot, c->h_state + slot, sizeof(SlotState),
                             cudaMemcpyHostToDevice, c->stream), "state upload");
  return sync(c);
}

kx_status read_state(kx_ctx* c, int slot, SlotState* out) {
  KX_CUDA(c, cudaMemcpyAsync(c->h_state + slot, c->d_state + slot, sizeof(SlotState),
                             cudaMemcpyDeviceToHost, c->stream), "state read");
  KX_TRY(sync(c));
  *out = c->h_state[slot];
  return KX_OK;
}

SlotState fresh_state() {
  SlotState s;
  std::memset(&s, 0, sizeof(s));
  return s;
}

// m Arnoldi steps on slots [slot0, slot0 + ns) from their (normalised)
// column 0, all slots in the same launches.
kx_status arnoldi_steps(kx_ctx* c, int slot0, int ns, int m, const void* g_aug) {
  for (int j = 0; j < m; ++j) {
    KX_TRY(launch_pass_a(c, slot0, ns, j, g_aug));
    // an augmented process finalises every pass B itself; otherwise the next
    // pass A does, and only the last step needs the finalisation kernel
    KX_TRY(launch_pass_b(c, slot0, ns, j, g_aug != nullptr || j == m - 1));
  }
  c->stats.arnoldi_steps += (int64_t)m * ns;
  c->stats.matvecs += (int64_t)m * ns;
  return KX_OK;
}

kx_status read_states(kx_ctx* c, int slot0, int ns) {
  KX_CUDA(c, cudaMemcpyAsync(c->h_state + slot0, c->d_state + slot0, sizeof(SlotState) * ns,
                             cudaMemcpyDeviceToHost, c->stream), "state read");
  return sync(c);
}

// Exponential Krylov restarted in time (Sect. 3.3): the states in column 0
// of slots [slot0, slot0 + ns) advance together to their final times by
// sub-steps x <- V_m exp(-t H_m) beta e_1; a slot that has arrived retires and
// every later kernel skips it.
// One sub-step's launches: m Arnoldi steps, the projected step control, the
// combination.
kx_status substep_launches(kx_ctx* c, int slot0, int ns, const void* g_aug) {
  KX_TRY(arnoldi_steps(c, slot0, ns, c->m, g_aug));
  KX_TRY(launch_substep_control(c, slot0, ns));
  return launch_combine(c, slot0, ns);
}

// A CUDA graph of one sub-step's launches (all parameters are fixed for the
// sub-steps of one time_loop; the changing state lives in device memory).
struct SubstepGraph {
  cudaGraphExec_t exec = nullptr;
  int64_t launches = 0;
  ~SubstepGraph() {
    if (exec) cudaGraphExecDestroy(exec);
  }
};

kx_status capture_substep(kx_ctx* c, int slot0, int ns, const void* g_aug, SubstepGraph* out) {
  const kx_stats saved = c->stats;   // capturing executes nothing: restore the counters
  const int64_t before = c->stats.kernel_launches;
  if (cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return KX_ECUDA;
  }
  const kx_status st = substep_launches(c, slot0, ns, g_aug);
  cudaGraph_t graph = nullptr;
  const cudaError_t e = cudaStreamEndCapture(c->stream, &graph);
  if (st != KX_OK || e != cudaSuccess || !graph) {
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    return KX_ECUDA;
  }
  const cudaError_t e2 = cudaGraphInstantiate(&out->exec, graph, 0);
  cudaGraphDestroy(graph);
  if (e2 != cudaSuccess) {
    cudaGetLastError();
    out->exec = nullptr;
    return KX_ECUDA;
  }
  out->launches = c->stats.kernel_launches - before;
  c->stats = saved;
  return KX_OK;
}

// Convergence is decided on the device: the step control retires a slot once
// it reaches its final time, and every kernel of a later sub-step returns at
// once for a retired slot (or one whose status records a failure).  The host
// therefore queues several sub-steps between two reads of the slot states --
// as many as the slowest slot is predicted to need, from its mean accepted
// sub-step so far, capped at SUBSTEP_BATCH -- instead of synchronising after
// every sub-step; queued sub-steps past the end cost only empty launches.
constexpr int SUBSTEP_BATCH = 8;

kx_status time_loop(kx_ctx* c, int slot0, int ns, const void* g_aug, double* err_est) {
  KX_TRY(launch_norm_init(c, slot0, ns));
  const int max_sub = 20000;
  bool all = false;
  // the first sub-step runs eagerly (one-time kernel set-up), the rest replay
  // a captured graph; capture is skipped on the legacy stream and while the
  // per-kernel timing is on
  bool use_graph = c->stream != nullptr && !c->timing;
  SubstepGraph graph;
  int queued = 0, batch = 1;
  while (queued < max_sub && !all) {
    for (int b = 0; b < batch && queued < max_sub; ++b, ++queued) {
      if (use_graph && queued >= 1 && !graph.exec && capture_substep(c, slot0, ns, g_aug, &graph) != KX_OK)
        use_graph = false;
      if (use_graph && graph.exec) {
        KX_CUDA(c, cudaGraphLaunch(graph.exec, c->stream), "sub-step graph launch");
        c->stats.kernel_launches += graph.launches;
      } else {
        const kx_stats before = c->stats;
        KX_TRY(substep_launches(c, slot0, ns, g_aug));
        // Arnoldi work is counted from the accepted sub-steps below
        c->stats.arnoldi_steps = before.arnoldi_steps;
        c->stats.matvecs = before.matvecs;
      }
    }
    KX_TRY(read_states(c, slot0, ns));
    all = true;
    double need = 1.0;
    for (int q = 0; q < ns; ++q) {
      const SlotState& st = c->h_state[slot0 + q];
      if (st.status)
        return fail(c, (kx_status)st.status,
                    st.status == KX_ENOCONV ? "time sub-step control: no step length met the tolerance"
                                            : "non-finite value in the Krylov process");
      all = all && st.retired;
      if (!st.retired && st.substeps > 0 && st.t_now > 0.0)
        need = std::max(need, std::ceil((st.T - st.t_now) * st.substeps / st.t_now));
    }
    batch = (int)std::min<double>(SUBSTEP_BATCH, need);
  }
  if (!all) return fail(c, KX_ENOCONV, "time stepping: sub-step cap reached");
  for (int q = 0; q < ns; ++q) {
    const SlotState& st = c->h_state[slot0 + q];
    c->stats.substeps += st.substeps;
    c->stats.expm_evals += st.expm_evals;
    // one m-step Arnoldi process per accepted sub-step
    c->stats.arnoldi_steps += (int64_t)c->m * st.substeps;
    c->stats.matvecs += (int64_t)c->m * st.substeps;
    if (err_est) err_est[q] = st.err_acc;
  }
  return KX_OK;
}

kx_status check_vec(kx_ctx* c, const void* p, const char* name) {
  if (!p) return fail(c, KX_EINVAL, std::string(name) + " is NULL");
  return KX_OK;
}

// Output plane {axis, index}: validated, and its node count (all E components).
kx_status check_plane(kx_ctx* c, const int* plane, int* axis, int* idx, int64_t* P) {
  if (!plane) return fail(c, KX_EINVAL, "plane is NULL");
  *axis = plane[0];
  *idx = plane[1];
  if (*axis < 0 || *axis >= c->d.dim) return fail(c, KX_EINVAL, "bad plane axis");
  const int na = *axis == 0 ? c->geo.nx : (*axis == 1 ? c->geo.ny : c->geo.nz);
  if (*idx < 0 || *idx >= na) return fail(c, KX_EINVAL, "bad plane index");
  int a = 0, b = 0;
  plane_dims(c->geo, *axis, &a, &b);
  *P = (int64_t)c->geo.ne * a * b;
  return KX_OK;
}

kx_status check_omegas(kx_ctx* c, const double* om, int nfreq) {
  if (nfreq < 1 || nfreq > c->d.max_freqs)
    return fail(c, KX_EINVAL, "nfreq out of range 1..max_freqs");
  if (!om) return fail(c, KX_EINVAL, "omegas is NULL");
  for (int f = 0; f < nfreq; ++f)
    if (!std::isfinite(om[f])) return fail(c, KX_ENONFINITE, "non-finite frequency");
  return KX_OK;
}

// Stationary parts into the buffers zre, zim (n x nfreq, leading dim n).
kx_status stationary_core(kx_ctx* c, const void* d_g, const double* omegas, int nfreq, double rtol,
                          int max_matvecs, void* zre, void* zim, double* rel_resid, int* matvecs_out) {
  const int slot = 0;
  KX_CUDA(c, cudaMemcpyAsync(slot_col(c, slot, 0), d_g, c->n * c->esize, cudaMemcpyDeviceToDevice,
                             c->stream), "copy g");
  KX_TRY(upload_state(c, slot, fresh_state()));
  KX_TRY(launch_norm_init(c, slot, 1));
  SlotState st;
  KX_TRY(read_state(c, slot, &st));
  const double beta = st.beta;
  if (!std::isfinite(beta)) return fail(c, KX_ENONFINITE, "non-finite source vector");
  KX_CUDA(c, cudaMemsetAsync(zre, 0, (size_t)nfreq * c->n * c->esize, c->stream), "zero z");
  KX_CUDA(c, cudaMemsetAsync(zim, 0, (size_t)nfreq * c->n * c->esize, c->stream), "zero z");
  if (beta == 0.0) {
    if (rel_resid) for (int f = 0; f < nfreq; ++f) rel_resid[f] = 0.0;
    if (matvecs_out) *matvecs_out = 0;
    return sync(c);
  }
  std::vector<double> rho(2 * nfreq);
  for (int f = 0; f < nfreq; ++f) { rho[2 * f] = beta; rho[2 * f + 1] = 0.0; }
  KX_CUDA(c, cudaMemcpyAsync(c->d_rho, rho.data(), sizeof(double) * 2 * nfreq, cudaMemcpyHostToDevice,
                             c->stream), "rho upload");
  KX_CUDA(c, cudaMemcpyAsync(c->d_omegas, omegas, sizeof(double) * nfreq, cudaMemcpyHostToDevice,
                             c->stream), "omega upload");
  KX_TRY(sync(c));
  int matvecs = 0;
  bool converged = false;
  double best = INFINITY;
  int since_best = 0;
  for (int cyc = 0; matvecs < max_matvecs; ++cyc) {
    KX_TRY(arnoldi_steps(c, slot, 1, c->m, nullptr));
    KX_TRY(read_state(c, slot, &st));
    if (st.status) return fail(c, (kx_status)st.status, "non-finite value in the Arnoldi process");
    const int md = st.m_done;
    KX_TRY(launch_shifted_solve(c, slot, nfreq, md));
    KX_TRY(launch_zupdate(c, slot, nfreq, zre, zim, md));
    matvecs += md;
    c->stats.fom_cycles++;
    KX_CUDA(c, cudaMemcpyAsync(c->h_small, c->d_rho, sizeof(double) * 2 * nfreq,
                               cudaMemcpyDeviceToHost, c->stream), "rho read");
    KX_TRY(sync(c));
    double worst = 0.0;
    for (int f = 0; f < nfreq; ++f) worst = std::max(worst, std::hypot(c->h_small[2 * f], c->h_small[2 * f + 1]));
    if (!std::isfinite(worst)) return fail(c, KX_ENONFINITE, "non-finite shifted-FOM residual");
    if (worst <= rtol * beta || st.done) { converged = true; break; }
    // stagnation (rounding floor of the working precision): stop early
    if (worst < 0.999 * best) { best = worst; since_best = 0; }
    else if (++since_best >= 20) break;
    // restart from v_{m+1}: copy column md to column 0 and renormalise
    KX_CUDA(c, cudaMemcpyAsync(slot_col(c, slot, 0), slot_col(c, slot, md), c->n * c->esize,
                               cudaMemcpyDeviceToDevice, c->stream), "restart copy");
    KX_TRY(launch_norm_init(c, slot, 1));
  }
  if (matvecs_out) *matvecs_out = matvecs;
  if (rel_resid) KX_TRY(launch_true_residual(c, d_g, nfreq, omegas, zre, zim, rel_resid));
  KX_TRY(sync(c));
  if (!converged) return fail(c, KX_ENOCONV, "shifted FOM: matvec cap reached before rtol");
  return KX_OK;
}

// One time loop over slots [0, ns): slot q (if on[q]) advances its column 0
// over Tq[q] -- by the augmented plain method (source phase from zero) when
// aug, else homogeneously; the other slots stay retired.  Error estimates are
// added to err[q].
kx_status slots_time_loop(kx_ctx* c, int ns, bool aug, const void* d_g, const double* omegas, int f0,
                          double rtol, double eta, const std::vector<double>& Tq, const std::vector<char>& on,
                          std::vector<double>& err) {
  bool any = false;
  for (int q = 0; q < ns; ++q) {
    SlotState s = fresh_state();
    if (!on[q]) {
      s.retired = 1;
    } else {
      any = true;
      s.T = Tq[q];
      s.rtol = rtol;
      if (aug) {
        s.aug = 1;
        s.omega = omegas[f0 + q];
        s.eta = eta;
        s.tol_mode = 1;
      }
    }
    c->h_state[q] = s;
  }
  if (!any) return KX_OK;
  KX_CUDA(c, cudaMemcpyAsync(c->d_state, c->h_state, sizeof(SlotState) * ns, cudaMemcpyHostToDevice, c->stream),
          "state upload");
  KX_TRY(sync(c));
  std::vector<double> e(ns, 0.0);
  KX_TRY(time_loop(c, 0, ns, aug ? d_g : nullptr, e.data()));
  for (int q = 0; q < ns; ++q)
    if (on[q]) err[q] += e[q];
  return KX_OK;
}

// Source splitting (eq. (split2)) for frequencies f0 .. f0+ns-1 in slots
// 0 .. ns-1, leaving y_f(T) in column 0 of slot q.  Subinterval dT = one
// source period (the source has the same phase at every subinterval start,
// so w2 is the same on all of them): w2(dT) is kept in d_zre[f], w2 over the
// remainder r = T - K dT in d_zim[f].
kx_status split2_wave(kx_ctx* c, const void* d_g, const double* omegas, int f0, int ns, double T, double rtol,
                      double eta, double* err_est) {
  const size_t vb = (size_t)c->n * c->esize;
  const double two_pi = 6.283185307179586476925286766559;
  std::vector<double> dT(ns), rem(ns), err(ns, 0.0);
  std::vector<int> K(ns);
  std::vector<char> all(ns, 1), has_r(ns, 0);
  int Kmax = 0;
  for (int q = 0; q < ns; ++q) {
    const double W = std::fabs(omegas[f0 + q]);
    dT[q] = W > 0.0 ? std::min(T, two_pi / W) : T;
    K[q] = std::max(1, (int)std::floor(T / dT[q] + 1e-12));
    rem[q] = T - K[q] * dT[q];
    if (rem[q] > 1e-12 * T) has_r[q] = 1;
    else rem[q] = 0.0;
    Kmax = std::max(Kmax, K[q]);
  }
  // w2 over one period, and over the remainder, from zero (plain method)
  for (int q = 0; q < ns; ++q)
    KX_CUDA(c, cudaMemsetAsync(slot_col(c, q, 0), 0, vb, c->stream), "zero w2");
  KX_TRY(slots_time_loop(c, ns, true, d_g, omegas, f0, rtol, eta, dT, all, err));
  for (int q = 0; q < ns; ++q) {
    KX_CUDA(c, cudaMemcpyAsync(vec_ptr(c, c->d_zre, f0 + q), slot_col(c, q, 0), vb, cudaMemcpyDeviceToDevice,
                               c->stream), "keep w2");
    KX_CUDA(c, cudaMemsetAsync(slot_col(c, q, 0), 0, vb, c->stream), "zero w2");
  }
  KX_TRY(slots_time_loop(c, ns, true, d_g, omegas, f0, rtol, eta, rem, has_r, err));
  for (int q = 0; q < ns; ++q)
    if (has_r[q])
      KX_CUDA(c, cudaMemcpyAsync(vec_ptr(c, c->d_zim, f0 + q), slot_col(c, q, 0), vb, cudaMemcpyDeviceToDevice,
                                 c->stream), "keep w2 of the remainder");
  // y(dT) = w2; y(k dT) = exp(-dT A) y((k-1) dT) + w2 for k = 2 .. K
  for (int q = 0; q < ns; ++q)
    KX_CUDA(c, cudaMemcpyAsync(slot_col(c, q, 0), vec_ptr(c, c->d_zre, f0 + q), vb, cudaMemcpyDeviceToDevice,
                               c->stream), "y = w2");
  for (int k = 2; k <= Kmax; ++k) {
    std::vector<char> on(ns);
    for (int q = 0; q < ns; ++q) on[q] = k <= K[q];
    KX_TRY(slots_time_loop(c, ns, false, nullptr, omegas, f0, rtol, eta, dT, on, err));
    for (int q = 0; q < ns; ++q)
      if (on[q]) KX_TRY(launch_axpy(c, 1.0, vec_ptr(c, c->d_zre, f0 + q), slot_col(c, q, 0)));
  }
  // the last, shorter subinterval
  KX_TRY(slots_time_loop(c, ns, false, nullptr, omegas, f0, rtol, eta, rem, has_r, err));
  for (int q = 0; q < ns; ++q)
    if (has_r[q]) KX_TRY(launch_axpy(c, 1.0, vec_ptr(c, c->d_zim, f0 + q), slot_col(c, q, 0)));
  if (err_est)
    for (int q = 0; q < ns; ++q) err_est[f0 + q] = err[q];
  return sync(c);
}

}  // namespace

// ===========================================================================
extern "C" {

}  // extern "C"

namespace {

// Context creation.  The permittivity comes either from a host array per
// cell (eps_cell) or from a device array of material ids per cell and a host
// table of their permittivities (d_mat_id, eps_table, n_mat).
kx_status create_impl(const kx_desc* desc, const double* eps_cell, const uint8_t* d_mat_id,
                      const double* eps_table, int n_mat, void* cuda_stream, kx_ctx** out) {
  if (!desc || !out || (!eps_cell && !(d_mat_id && eps_table))) return fail(nullptr, KX_EINVAL, "NULL argument");
  *out = nullptr;
  const kx_desc& d = *desc;
  if (d.dim != 2 && d.dim != 3) return fail(nullptr, KX_EINVAL, "dim must be 2 or 3");
  for (int a = 0; a < d.dim; ++a) {
    if (d.n[a] < 3) return fail(nullptr, KX_EINVAL, "each n[a] must be >= 3");
    if (d.bc[a] != KX_PERIODIC && d.bc[a] != KX_PEC) return fail(nullptr, KX_EINVAL, "bad bc");
  }
  if (d.layer_axis < 0 || d.layer_axis >= d.dim) return fail(nullptr, KX_EINVAL, "bad layer_axis");
  if (d.layer_cells < 1 || 2 * d.layer_cells > d.n[d.layer_axis])
    return fail(nullptr, KX_EINVAL, "bad layer_cells");
  if (!(d.sigma_max >= 0.0) || !std::isfinite(d.sigma_max)) return fail(nullptr, KX_EINVAL, "bad sigma_max");
  if (d.precision != KX_FP64 && d.precision != KX_FP32) return fail(nullptr, KX_EINVAL, "bad precision");
  if (d.krylov_dim < 2 || d.krylov_dim > MMAX) return fail(nullptr, KX_EINVAL, "krylov_dim must be 2..64");
  if (d.max_freqs < 1 || d.max_freqs > MAXF) return fail(nullptr, KX_EINVAL, "max_freqs must be 1..64");
  if (d.batch < 1 || d.batch > 64) return fail(nullptr, KX_EINVAL, "batch must be 1..64");
  if (d.max_checkpoints < 0 || (d.max_checkpoints > 0 && d.batch < 2))
    return fail(nullptr, KX_EINVAL, "max_checkpoints must be >= 0, and the adjoint needs batch >= 2");
  if (d.rst_samples < 0 || d.rst_samples > (1 << 24)) return fail(nullptr, KX_EINVAL, "rst_samples must be 0 .. 2^24");
  if (d.pml != 0 && d.pml != 1) return fail(nullptr, KX_EINVAL, "pml must be 0 or 1");
  if (d.pml && (d.dim != 2 || d.layer_axis != 0))
    return fail(nullptr, KX_EINVAL, "the PML model is 2D with the layer along x (layer_axis 0)");
  if (d.pml && d.max_checkpoints > 0) return fail(nullptr, KX_EINVAL, "the adjoint does not cover the PML model");
  if (d.arnoldi_form != KX_ARN_DEFAULT && d.arnoldi_form != KX_ARN_TWOPASS && d.arnoldi_form != KX_ARN_SWEEP)
    return fail(nullptr, KX_EINVAL, "arnoldi_form must be KX_ARN_DEFAULT, KX_ARN_TWOPASS or KX_ARN_SWEEP");
  const int nz = d.dim == 3 ? d.n[2] : 1;
  const int64_t ncell = (int64_t)d.n[0] * d.n[1] * nz;
  if (eps_cell) {
    for (int64_t i = 0; i < ncell; ++i)
      if (!(eps_cell[i] > 0.0) || !std::isfinite(eps_cell[i]))
        return fail(nullptr, KX_ENONFINITE, "eps_cell must be finite and > 0");
  } else {
    if (n_mat < 1 || n_mat > KX_MAX_MATERIALS) return fail(nullptr, KX_EINVAL, "n_mat must be 1 .. 64");
    for (int i = 0; i < n_mat; ++i)
      if (!(eps_table[i] > 0.0) || !std::isfinite(eps_table[i]))
        return fail(nullptr, KX_ENONFINITE, "eps_table entries must be finite and > 0");
  }

  kx_ctx* c = new (std::nothrow) kx_ctx();
  if (!c) return fail(nullptr, KX_ENOMEM, "host allocation failed");
  c->d = d;
  if (d.dim == 2) c->d.n[2] = 1;
  if (cuda_stream == KX_OWN_STREAM) {
    if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete c;
      return fail(nullptr, KX_ECUDA, "stream creation failed");
    }
    c->own_stream = true;
  } else {
    c->stream = (cudaStream_t)cuda_stream;
  }
  Geo& g = c->geo;
  g.dim = d.dim;
  g.nx = d.n[0];
  g.ny = d.n[1];
  g.nz = nz;
  g.ncell = ncell;
  g.pml = d.pml;
  g.ncomp = d.dim == 2 ? 3 + d.pml : 6;
  g.nh = d.dim == 2 ? 2 : 3;
  g.ne = d.dim == 2 ? 1 : 3;
  g.la = d.layer_axis;
  // staggered offsets: 1 = half-integer along the axis (P: on the Ez nodes)
  static const int off2[4][3] = {{0, 1, 0}, {1, 0, 0}, {0, 0, 0}, {0, 0, 0}};
  static const int off3[6][3] = {{0, 1, 1}, {1, 0, 1}, {1, 1, 0}, {1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
  for (int comp = 0; comp < g.ncomp; ++comp) {
    const int* off = d.dim == 2 ? off2[comp] : off3[comp];
    unsigned mb = 0;
    for (int a = 0; a < d.dim; ++a)
      if (d.bc[a] == KX_PEC && off[a] == 0) mb |= 1u << a;
    g.maskbits[comp] = mb;
    g.sighalf[comp] = off[d.layer_axis];
  }
  c->n = g.ncomp * ncell;
  c->esize = d.precision == KX_FP64 ? 8 : 4;
  c->ld = (c->n + 63) / 64 * 64;
  c->m = d.krylov_dim;
  int dev = 0, nsm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) {
    delete c;
    return fail(nullptr, KX_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  const int64_t want = (ncell + NTHREADS - 1) / NTHREADS;
  c->nsm = nsm;
  c->ps = nsm * 8;
  c->nblk = (int)std::max<int64_t>(1, std::min<int64_t>(want, (int64_t)nsm * 8));

  const int B = d.batch, m = c->m;
  const int nla = d.n[d.layer_axis];
  size_t bytes_V = (size_t)B * (m + 1) * c->ld * c->esize;
  struct Alloc { void** p; size_t bytes; } allocs[] = {
      {(void**)&c->d_inv_eps, (size_t)g.ne * ncell * c->esize},
      {(void**)&c->d_sig2, (size_t)2 * nla * c->esize},
      {(void**)&c->d_eps_cell, (size_t)ncell * sizeof(double)},
      {(void**)&c->d_V, bytes_V},
      {(void**)&c->d_aug, (size_t)B * (m + 1) * 2 * sizeof(double)},
      {(void**)&c->d_H, (size_t)B * (m + 1) * m * sizeof(double)},
      {(void**)&c->d_scale, (size_t)B * (m + 2) * sizeof(double)},
      {(void**)&c->d_part, (size_t)B * PCOLS * c->ps * sizeof(double)},
      {(void**)&c->d_counter, (size_t)B * 8 * sizeof(unsigned)},
      {(void**)&c->d_u, (size_t)B * (m + 2) * sizeof(double)},
      {(void**)&c->d_state, (size_t)B * sizeof(SlotState)},
      {(void**)&c->d_rho, (size_t)2 * MAXF * sizeof(double)},
      {(void**)&c->d_coef, (size_t)2 * MAXF * MMAX * sizeof(float)},
      {(void**)&c->d_coefd, (size_t)2 * MAXF * MMAX * sizeof(double)},
      {(void**)&c->d_omegas, (size_t)MAXF * sizeof(double)},
      {(void**)&c->d_small, (size_t)256 * sizeof(double)},
      {(void**)&c->d_tmp, (size_t)c->n * c->esize},
      {(void**)&c->d_tmp2, (size_t)c->n * c->esize},
      {(void**)&c->d_expm_ws, (size_t)(MMAX + 1) * MMAX * MAXF * sizeof(double)},
      {(void**)&c->d_zre, (size_t)d.max_freqs * c->n * c->esize},
      {(void**)&c->d_zim, (size_t)d.max_freqs * c->n * c->esize},
      {(void**)&c->d_swT, (size_t)c->n * c->esize},
      {(void**)&c->d_swpart, (size_t)B * SWCOLS * c->ps * sizeof(double)},
      {(void**)&c->d_swG, (size_t)B * (MMAX + 1) * (MMAX + 1) * sizeof(double)},
      {(void**)&c->d_swco, (size_t)B * sizeof(SwCoef)},
  };
  for (auto& a : allocs) {
    e = cudaMalloc(a.p, a.bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      krylov_expm_destroy(c);
      return fail(nullptr, KX_ENOMEM, std::string("device allocation failed: ") + cudaGetErrorString(e));
    }
  }
  if (d.max_checkpoints > 0) {
    const int P = gauss_points();
    c->adj_nq_max = 64 * P;
    const int64_t nE = (int64_t)g.ne * ncell;
    Alloc adj[] = {
        {(void**)&c->d_ckpt, (size_t)d.max_checkpoints * c->ld * c->esize},
        {(void**)&c->d_adj_Q, (size_t)nE * sizeof(double)},
        {(void**)&c->d_adj_alpha, (size_t)c->adj_nq_max * (MMAX + 1) * sizeof(float)},
        {(void**)&c->d_adj_omg, (size_t)c->adj_nq_max * MMAX * sizeof(float)},
        {(void**)&c->d_adj_cw, (size_t)c->adj_nq_max * sizeof(float)},
        {(void**)&c->d_adj_sn, (size_t)c->adj_nq_max * sizeof(float)},
        {(void**)&c->d_gauss, (size_t)2 * P * sizeof(double)},
    };
    for (auto& a : adj) {
      e = cudaMalloc(a.p, a.bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        krylov_expm_destroy(c);
        return fail(nullptr, KX_ENOMEM, std::string("adjoint allocation failed: ") + cudaGetErrorString(e));
      }
    }
    std::vector<double> gw(2 * P);
    gauss_legendre01(P, gw.data(), gw.data() + P);
    e = cudaMemcpy(c->d_gauss, gw.data(), sizeof(double) * 2 * P, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      krylov_expm_destroy(c);
      return fail(nullptr, KX_ECUDA, std::string("Gauss nodes upload failed: ") + cudaGetErrorString(e));
    }
  }
  if (d.rst_samples > 0) {
    int na = 0, nb = 0;
    int64_t pmax = 0;
    for (int a = 0; a < d.dim; ++a) {
      plane_dims(g, a, &na, &nb);
      pmax = std::max<int64_t>(pmax, (int64_t)na * nb);
    }
    c->rst_plane_max = (int64_t)g.ne * pmax;
    Alloc rst[] = {
        {(void**)&c->d_rst_b, (size_t)d.max_freqs * d.rst_samples * RST_P * sizeof(double)},
        {(void**)&c->d_rst_smp, (size_t)d.max_freqs * (d.rst_samples + 1) * 3 * sizeof(double)},
        {(void**)&c->d_rst_mats, (size_t)RST_MATS * sizeof(double)},
        {(void**)&c->d_rst_u, (size_t)MAXF * MMAX * sizeof(double)},
        {(void**)&c->d_rst_res, (size_t)MAXF * sizeof(double)},
        {(void**)&c->d_rst_state, (size_t)MAXF * sizeof(int)},
        {(void**)&c->d_rst_yp, (size_t)d.max_freqs * c->rst_plane_max * sizeof(double)},
    };
    for (auto& a : rst) {
      e = cudaMalloc(a.p, a.bytes);
      if (e != cudaSuccess) {
        cudaGetLastError();
        krylov_expm_destroy(c);
        return fail(nullptr, KX_ENOMEM, std::string("restart workspace allocation failed: ") + cudaGetErrorString(e));
      }
    }
    e = cudaStreamCreateWithFlags(&c->aux_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_arnoldi, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_proj[0], cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&c->ev_proj[1], cudaEventDisableTiming);
    if (e != cudaSuccess) {
      cudaGetLastError();
      krylov_expm_destroy(c);
      return fail(nullptr, KX_ECUDA, std::string("auxiliary stream creation failed: ") + cudaGetErrorString(e));
    }
  }
  e = cudaMallocHost((void**)&c->h_state, (size_t)B * sizeof(SlotState));
  if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_small, 256 * sizeof(double));
  if (e != cudaSuccess) {
    cudaGetLastError();
    krylov_expm_destroy(c);
    return fail(nullptr, KX_ENOMEM, "pinned host allocation failed");
  }
  e = cudaMemsetAsync(c->d_counter, 0, (size_t)B * 8 * sizeof(unsigned), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_swco, 0, (size_t)B * sizeof(SwCoef), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_state, 0, (size_t)B * sizeof(SlotState), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_V, 0, bytes_V, c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_aug, 0, (size_t)B * (m + 1) * 2 * sizeof(double), c->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(c->d_H, 0, (size_t)B * (m + 1) * m * sizeof(double), c->stream);
  int* d_bad = reinterpret_cast<int*>(c->d_small + KX_MAX_MATERIALS);
  if (e == cudaSuccess && eps_cell) {
    e = cudaMemcpyAsync(c->d_eps_cell, eps_cell, (size_t)ncell * sizeof(double), cudaMemcpyHostToDevice, c->stream);
  } else if (e == cudaSuccess) {
    // the table and the id check flag go through the small scratch buffer
    std::memcpy(c->h_small, eps_table, sizeof(double) * n_mat);
    e = cudaMemcpyAsync(c->d_small, c->h_small, sizeof(double) * n_mat, cudaMemcpyHostToDevice, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d_bad, 0, sizeof(int), c->stream);
  }
  if (e != cudaSuccess) {
    krylov_expm_destroy(c);
    return fail(nullptr, KX_ECUDA, std::string("initialisation failed: ") + cudaGetErrorString(e));
  }
  kx_status st = eps_cell ? KX_OK : launch_expand_materials(c, d_mat_id, c->d_small, n_mat, d_bad);
  if (st == KX_OK) st = launch_setup_material(c);
  if (st == KX_OK) {
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) st = KX_ECUDA, snprintf(c->err, sizeof(c->err), "%s", cudaGetErrorString(e));
  }
  if (st != KX_OK) {
    std::string msg = c->err;
    krylov_expm_destroy(c);
    return fail(nullptr, st, "material set-up failed: " + msg);
  }
  if (!eps_cell) {
    int bad = 0;
    e = cudaMemcpy(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess || bad) {
      krylov_expm_destroy(c);
      return fail(nullptr, e != cudaSuccess ? KX_ECUDA : KX_EINVAL,
                  e != cudaSuccess ? std::string("material check read-back: ") + cudaGetErrorString(e)
                                   : std::string("a material id is >= n_mat"));
    }
  }
  std::memset(&c->stats, 0, sizeof(c->stats));
  *out = c;
  return KX_OK;
}

}  // namespace

extern "C" {

kx_status krylov_expm_create(const kx_desc* desc, const double* eps_cell, void* cuda_stream, kx_ctx** out) {
  if (!eps_cell) return fail(nullptr, KX_EINVAL, "NULL argument");
  return create_impl(desc, eps_cell, nullptr, nullptr, 0, cuda_stream, out);
}

kx_status krylov_expm_create_mat(const kx_desc* desc, const uint8_t* d_mat_id, const double* eps_table, int n_mat,
                                 void* cuda_stream, kx_ctx** out) {
  if (!d_mat_id || !eps_table) return fail(nullptr, KX_EINVAL, "NULL argument");
  return create_impl(desc, nullptr, d_mat_id, eps_table, n_mat, cuda_stream, out);
}

kx_status krylov_expm_destroy(kx_ctx* c) {
  if (!c) return KX_OK;
  cudaStreamSynchronize(c->stream);
  void* ptrs[] = {c->d_inv_eps, c->d_sig2, c->d_eps_cell, c->d_V, c->d_aug, c->d_H, c->d_scale,
                  c->d_part, c->d_counter, c->d_u, c->d_state, c->d_rho, c->d_coef, c->d_coefd,
                  c->d_omegas, c->d_small, c->d_tmp, c->d_tmp2, c->d_expm_ws, c->d_zre, c->d_zim,
                  c->d_ckpt, c->d_adj_Q, c->d_adj_alpha, c->d_adj_omg, c->d_adj_cw, c->d_adj_sn,
                  c->d_gauss, c->d_rst_b, c->d_rst_smp, c->d_rst_mats, c->d_rst_u, c->d_rst_res,
                  c->d_rst_state, c->d_rst_yp, c->d_swT, c->d_swpart, c->d_swG, c->d_swco};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (c->h_state) cudaFreeHost(c->h_state);
  if (c->h_small) cudaFreeHost(c->h_small);
  if (c->aux_stream) {
    cudaStreamSynchronize(c->aux_stream);
    cudaStreamDestroy(c->aux_stream);
  }
  if (c->ev_arnoldi) cudaEventDestroy(c->ev_arnoldi);
  for (cudaEvent_t ev : c->ev_proj)
    if (ev) cudaEventDestroy(ev);
  if (c->own_stream) cudaStreamDestroy(c->stream);
  delete c;
  return KX_OK;
}

int64_t kx_num_unknowns(const kx_ctx* c) { return c ? c->n : 0; }

void* kx_stream(const kx_ctx* c) { return c ? (void*)c->stream : nullptr; }

kx_status apply_A(kx_ctx* c, const void* d_v, void* d_w, int transpose) {
  if (!c) return KX_EINVAL;
  KX_TRY(check_vec(c, d_v, "d_v"));
  KX_TRY(check_vec(c, d_w, "d_w"));
  if (d_v == d_w) return fail(c, KX_EINVAL, "d_v and d_w must not overlap");
  c->stats.matvecs++;
  return launch_apply(c, d_v, d_w, transpose ? 1 : 0);
}

kx_status arnoldi(kx_ctx* c, const void* d_v0, int m, void* d_V, double* H, double* beta,
                  int* m_done) {
  if (!c) return KX_EINVAL;
  KX_TRY(check_vec(c, d_v0, "d_v0"));
  if (m < 1 || m > c->m) return fail(c, KX_EINVAL, "m out of range 1..krylov_dim");
  if (!H || !beta || !m_done) return fail(c, KX_EINVAL, "NULL output");
  const int slot = 0;
  KX_CUDA(c, cudaMemcpyAsync(slot_col(c, slot, 0), d_v0, c->n * c->esize, cudaMemcpyDeviceToDevice,
                             c->stream), "copy v0");
  KX_CUDA(c, cudaMemsetAsync(c->d_H, 0, (size_t)(c->m + 1) * c->m * sizeof(double), c->stream), "zero H");
  KX_TRY(upload_state(c, slot, fresh_state()));
  KX_TRY(launch_norm_init(c, slot, 1));
  SlotState st;
  KX_TRY(read_state(c, slot, &st));
  if (!(st.beta > 0.0) || !std::isfinite(st.beta)) return fail(c, KX_ENONFINITE, "v0 is zero or non-finite");
  if (c->d.arnoldi_form == KX_ARN_SWEEP) KX_TRY(sweep_arnoldi(c, slot, m));
  else KX_TRY(arnoldi_steps(c, slot, 1, m, nullptr));
  KX_TRY(read_state(c, slot, &st));
  if (st.status) return fail(c, (kx_status)st.status, "non-finite value in the Arnoldi process");
  *beta = st.beta;
  *m_done = st.m_done;
  // H: context stride c->m + 1 -> caller stride m + 1
  const bool hdev = is_device_ptr(H);
  KX_CUDA(c, cudaMemcpy2DAsync(H, (size_t)(m + 1) * sizeof(double), c->d_H,
                               (size_t)(c->m + 1) * sizeof(double), (size_t)(m + 1) * sizeof(double), m,
                               hdev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->stream),
          "H copy");
  if (d_V) KX_TRY(launch_basis_export(c, slot, d_V, m));
  return sync(c);
}

kx_status expm_phi_project(kx_ctx* c, const double* H, int ldh, int m, double beta, double tau,
                           const double* omegas, int nfreq, double* u_out) {
  if (!c) return KX_EINVAL;
  if (!H || !u_out) return fail(c, KX_EINVAL, "NULL argument");
  if (m < 1 || m > c->m || ldh < m) return fail(c, KX_EINVAL, "bad m or ldh");
  if (nfreq < 0 || nfreq > c->d.max_freqs) return fail(c, KX_EINVAL, "bad nfreq");
  if (nfreq > 0) KX_TRY(check_omegas(c, omegas, nfreq));
  if (!std::isfinite(beta) || !std::isfinite(tau)) return fail(c, KX_ENONFINITE, "non-finite beta or tau");
  // H -> device workspace with leading dimension m+1 (column-major)
  double* dH = c->d_expm_ws;
  const bool hdev = is_device_ptr(H);
  KX_CUDA(c, cudaMemcpy2DAsync(dH, (size_t)(m + 1) * sizeof(double), H, (size_t)ldh * sizeof(double),
                               (size_t)m * sizeof(double), m,
                               hdev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->stream),
          "H upload");
  if (nfreq > 0)
    KX_CUDA(c, cudaMemcpyAsync(c->d_omegas, omegas, sizeof(double) * nfreq, cudaMemcpyHostToDevice,
                               c->stream), "omega upload");
  double* du = c->d_expm_ws + (size_t)(m + 1) * m;
  KX_CUDA(c, cudaMemsetAsync(c->d_small + 64, 0, sizeof(int), c->stream), "status reset");
  KX_TRY(launch_expm_project(c, dH, m + 1, m, beta, tau, c->d_omegas, nfreq, du));
  c->stats.expm_evals += nfreq > 0 ? nfreq : 1;
  const size_t ub = sizeof(double) * (size_t)m * std::max(1, nfreq);
  const bool udev = is_device_ptr(u_out);
  KX_CUDA(c, cudaMemcpyAsync(u_out, du, ub, udev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                             c->stream), "u copy");
  int status = 0;
  KX_CUDA(c, cudaMemcpyAsync(c->h_small, c->d_small + 64, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
          "status read");
  KX_TRY(sync(c));
  std::memcpy(&status, c->h_small, sizeof(int));
  if (status) return fail(c, KX_ENONFINITE, "singular Pade denominator");
  return KX_OK;
}

kx_status stationary_solve(kx_ctx* c, const void* d_g, const double* omegas, int nfreq, double rtol,
                           int max_matvecs, void* d_z_re, void* d_z_im, double* rel_resid, int* matvecs) {
  if (!c) return KX_EINVAL;
  KX_TRY(check_vec(c, d_g, "d_g"));
  KX_TRY(check_vec(c, d_z_re, "d_z_re"));
  KX_TRY(check_vec(c, d_z_im, "d_z_im"));
  KX_TRY(check_omegas(c, omegas, nfreq));
  if (!(rtol > 0.0) || max_matvecs < 1) return fail(c, KX_EINVAL, "rtol must be > 0, max_matvecs >= 1");
  return stationary_core(c, d_g, omegas, nfreq, rtol, max_matvecs, d_z_re, d_z_im, rel_resid, matvecs);
}

kx_status expm_action(kx_ctx* c, const void* d_y0, double T, double rtol, void* d_y, double* err_est) {
  if (!c) return KX_EINVAL;
  KX_TRY(check_vec(c, d_y0, "d_y0"));
  KX_TRY(check_vec(c, d_y, "d_y"));
  if (!(T >= 0.0) || !std::isfinite(T) || !(rtol > 0.0)) return fail(c, KX_EINVAL, "bad T or rtol");
  const int slot = 0;
  KX_CUDA(c, cudaMemcpyAsync(slot_col(c, slot, 0), d_y0, c->n * c->esize, cudaMemcpyDeviceToDevice,
                             c->stream), "copy y0");
  if (T == 0.0) {
    KX_CUDA(c, cudaMemcpyAsync(d_y, slot_col(c, slot, 0), c->n * c->esize, cudaMemcpyDeviceToDevice,
                               c->stream), "copy y");
    if (err_est) *err_est = 0.0;
    return sync(c);
  }
  SlotState s = fresh_state();
  s.T = T;
  s.rtol = rtol;
  s.tol_mode = 0;
  KX_TRY(upload_state(c, slot, s));
  KX_TRY(time_loop(c, slot, 1, nullptr, err_est));
  KX_CUDA(c, cudaMemcpyAsync(d_y, slot_col(c, slot, 0), c->n * c->esize, cudaMemcpyDeviceToDevice,
                             c->stream), "copy y");
  return sync(c);
}

kx_status response_at_freqs(kx_ctx* c, const void* d_g, const double* omegas, int nfreq, double T,
                            double rtol, int method, const int* plane, void* d_E_plane,
                            double* intensity, double* err_est, void* d_Y) {
  if (!c) return KX_EINVAL;
  KX_TRY(check_vec(c, d_g, "d_g"));
  KX_TRY(check_omegas(c, omegas, nfreq));
  if (!(T > 0.0) || !std::isfinite(T) || !(rtol > 0.0)) return fail(c, KX_EINVAL, "bad T or rtol");
  if (method == KX_RSTDIM)
    return response_restart_dim(c, d_g, omegas, nfreq, T, rtol, 0.0, 0, plane, d_E_plane, intensity, err_est,
                                nullptr, d_Y);
  if (method != KX_PLAIN && method != KX_SPLIT && method != KX_SPLIT2 && method != KX_SPLIT4D)
    return fail(c, KX_EINVAL, "bad method");
  const bool split = method == KX_SPLIT || method == KX_SPLIT4D;   // eq. (split1): stationary + transient
  if (!plane) return fail(c, KX_EINVAL, "plane is NULL");
  const int axis = plane[0], idx = plane[1];
  if (axis < 0 || axis >= c->d.dim) return fail(c, KX_EINVAL, "bad plane axis");
  const int na = axis == 0 ? c->geo.nx : (axis == 1 ? c->geo.ny : c->geo.nz);
  if (idx < 0 || idx >= na) return fail(c, KX_EINVAL, "bad plane index");
  int64_t np = 1;
  for (int a = 0; a < c->d.dim; ++a)
    if (a != axis) np *= c->d.n[a];
  const int nE = c->geo.ne;
  const int slot = 0;
  kx_status conv = KX_OK;
  double* d_int = c->d_small + 128;
  if (split) {
    // Fig. alg:spl1, steps 1-3 for every frequency, with all stationary
    // parts from one shifted solve (Corollary 1 applied to z_stat).
    kx_status st = stationary_core(c, d_g, omegas, nfreq, rtol * 0.1, 400 * c->m, c->d_zre,
                                   c->d_zim, nullptr, nullptr);
    if (st != KX_OK && st != KX_ENOCONV) return st;
    conv = st;
  } else {
    // eta = ||g|| balances the augmented phase entries against the field
    KX_CUDA(c, cudaMemcpyAsync(slot_col(c, slot, 0), d_g, c->n * c->esize, cudaMemcpyDeviceToDevice,
                               c->stream), "copy g");
    KX_TRY(upload_state(c, slot, fresh_state()));
    KX_TRY(launch_norm_init(c, slot, 1));
  }
  SlotState gst;
  KX_TRY(read_state(c, slot, &gst));
  const double gnorm = gst.beta;
  // frequencies advance in waves of up to `batch` slots sharing every launch
  const int B = c->d.batch;
  const size_t vb = (size_t)c->n * c->esize;
  for (int f0 = 0; f0 < nfreq; f0 += B) {
    const int ns = std::min(B, nfreq - f0);
    if (method == KX_SPLIT2) {
      KX_TRY(split2_wave(c, d_g, omegas, f0, ns, T, rtol, gnorm > 0.0 ? gnorm : 1.0, err_est));
      for (int q = 0; q < ns; ++q) {
        const int f = f0 + q;
        void* Ep = d_E_plane ? (char*)d_E_plane + (int64_t)f * nE * np * c->esize : nullptr;
        void* Yf = d_Y ? vec_ptr(c, d_Y, f) : nullptr;
        KX_TRY(launch_response(c, f, omegas, T, 0, nullptr, nullptr, slot_col(c, q, 0), axis, idx, Ep, d_int + f,
                               Yf));
      }
      continue;
    }
    if (method == KX_SPLIT4D) {
      // eq. (4diff): slot q carries Im z_f - Im z_{f-1} (f >= 1), solved to
      // a tolerance relative to Im z_f itself (its norm from a first pass)
      for (int q = 0; q < ns; ++q) {
        KX_CUDA(c, cudaMemcpyAsync(slot_col(c, q, 0), vec_ptr(c, c->d_zim, f0 + q), vb, cudaMemcpyDeviceToDevice,
                                   c->stream), "copy Im z");
        c->h_state[q] = fresh_state();
      }
      KX_CUDA(c, cudaMemcpyAsync(c->d_state, c->h_state, sizeof(SlotState) * ns, cudaMemcpyHostToDevice,
                                 c->stream), "state upload");
      KX_TRY(launch_norm_init(c, 0, ns));
      KX_TRY(read_states(c, 0, ns));
      std::vector<double> znorm(ns);
      for (int q = 0; q < ns; ++q) znorm[q] = c->h_state[q].beta;
      for (int q = 0; q < ns; ++q) {
        const int f = f0 + q;
        if (f >= 1) KX_TRY(launch_axpy(c, -1.0, vec_ptr(c, c->d_zim, f - 1), slot_col(c, q, 0)));
        SlotState s = fresh_state();
        s.T = T;
        s.rtol = rtol;
        s.tol_mode = 0;
        // frequency f sums the errors of the f differences before it: each
        // difference gets 1/nfreq of the budget rtol ||Im z_f||
        if (znorm[q] > 0.0) s.tol_abs = rtol * znorm[q] / (T * (f >= 1 ? nfreq : 1));
        c->h_state[q] = s;
      }
      KX_CUDA(c, cudaMemcpyAsync(c->d_state, c->h_state, sizeof(SlotState) * ns, cudaMemcpyHostToDevice,
                                 c->stream), "state upload");
      KX_TRY(sync(c));
      KX_TRY(time_loop(c, 0, ns, nullptr, err_est ? err_est + f0 : nullptr));
      // yhat_f(T) = yhat_{f-1}(T) + w_f(T)  (Fig. alg:spl1 steps 5-6); the
      // previous wave's last transient waits in d_tmp
      for (int q = 0; q < ns; ++q) {
        const int f = f0 + q;
        if (f >= 1) KX_TRY(launch_axpy(c, 1.0, q == 0 ? c->d_tmp : slot_col(c, q - 1, 0), slot_col(c, q, 0)));
      }
      KX_CUDA(c, cudaMemcpyAsync(c->d_tmp, slot_col(c, ns - 1, 0), vb, cudaMemcpyDeviceToDevice, c->stream),
              "keep the last transient");
      for (int q = 0; q < ns; ++q) {
        const int f = f0 + q;
        void* Ep = d_E_plane ? (char*)d_E_plane + (int64_t)f * nE * np * c->esize : nullptr;
        void* Yf = d_Y ? vec_ptr(c, d_Y, f) : nullptr;
        KX_TRY(launch_response(c, f, omegas, T, 1, vec_ptr(c, c->d_zre, f), vec_ptr(c, c->d_zim, f),
                               slot_col(c, q, 0), axis, idx, Ep, d_int + f, Yf));
      }
      continue;
    }
    for (int q = 0; q < ns; ++q) {
      const int f = f0 + q;
      SlotState s = fresh_state();
      s.T = T;
      s.rtol = rtol;
      if (method == KX_SPLIT) {
        // transient y^(T) = exp(-TA) Im z_f  (eq. (y_homo))
        KX_CUDA(c, cudaMemcpyAsync(slot_col(c, q, 0), vec_ptr(c, c->d_zim, f), c->n * c->esize,
                                   cudaMemcpyDeviceToDevice, c->stream), "copy Im z");
        s.tol_mode = 0;
      } else {
        // augmented system x' = -[[A, -g/eta, 0], [0, 0, -W], [0, W, 0]] x,
        // x(0) = [0; 0; eta]: the two extra entries are eta (sin Wt, cos Wt)
        KX_CUDA(c, cudaMemsetAsync(slot_col(c, q, 0), 0, c->n * c->esize, c->stream), "zero y");
        s.aug = 1;
        s.omega = omegas[f];
        s.eta = gnorm > 0.0 ? gnorm : 1.0;
        s.tol_mode = 1;
      }
      c->h_state[q] = s;
    }
    KX_CUDA(c, cudaMemcpyAsync(c->d_state, c->h_state, sizeof(SlotState) * ns, cudaMemcpyHostToDevice,
                               c->stream), "state upload");
    KX_TRY(sync(c));
    KX_TRY(time_loop(c, 0, ns, method == KX_SPLIT ? nullptr : d_g, err_est ? err_est + f0 : nullptr));
    for (int q = 0; q < ns; ++q) {
      const int f = f0 + q;
      void* Ep = d_E_plane ? (char*)d_E_plane + (int64_t)f * nE * np * c->esize : nullptr;
      void* Yf = d_Y ? vec_ptr(c, d_Y, f) : nullptr;
      KX_TRY(launch_response(c, f, omegas, T, method == KX_SPLIT, vec_ptr(c, c->d_zre, f),
                             vec_ptr(c, c->d_zim, f), slot_col(c, q, 0), axis, idx, Ep, d_int + f, Yf));
    }
  }
  if (intensity) {
    KX_CUDA(c, cudaMemcpyAsync(c->h_small, d_int, sizeof(double) * nfreq, cudaMemcpyDeviceToHost, c->stream),
            "intensity read");
    KX_TRY(sync(c));
    for (int f = 0; f < nfreq; ++f) intensity[f] = c->h_small[f];
  }
  KX_TRY(sync(c));
  if (conv != KX_OK) return fail(c, conv, "stationary solve did not reach its tolerance");
  return KX_OK;
}

// The Arnoldi process of one restart in Krylov dimension (basis slot
// `slot`, non-augmented).  By default the single-sweep form runs from
// SWEEP_MIN_UNKNOWNS unknowns up: its serial per-step finalisation (a few
// microseconds) hides behind the apply pass only on large grids (measured on
// GB300: at 64^3 the two-pass form is faster, from 96^3 up the single sweep).
constexpr int64_t SWEEP_MIN_UNKNOWNS = 3000000;

bool rst_uses_sweep(const kx_ctx* c) {
  if (c->d.arnoldi_form == KX_ARN_SWEEP) return true;
  if (c->d.arnoldi_form == KX_ARN_TWOPASS) return false;
  return c->n >= SWEEP_MIN_UNKNOWNS;
}

kx_status rst_arnoldi(kx_ctx* c, int slot) {
  if (rst_uses_sweep(c)) return sweep_arnoldi(c, slot, c->m);
  return arnoldi_steps(c, slot, 1, c->m, nullptr);
}

kx_status response_restart_dim(kx_ctx* c, const void* d_g, const double* omegas, int nfreq, double T,
                               double rtol, double dt_sample, int max_restarts, const int* plane,
                               void* d_E_plane, double* intensity, double* resid, int* restarts, void* d_Y) {
  if (!c) return KX_EINVAL;
  KX_TRY(check_vec(c, d_g, "d_g"));
  KX_TRY(check_omegas(c, omegas, nfreq));
  if (c->d.rst_samples <= 0) return fail(c, KX_EINVAL, "context created with rst_samples = 0");
  if (!(T > 0.0) || !std::isfinite(T)) return fail(c, KX_EINVAL, "T must be finite and > 0");
  if (!(rtol >= 0.0) || !std::isfinite(rtol)) return fail(c, KX_EINVAL, "rtol must be finite and >= 0");
  if (!(dt_sample >= 0.0) || !std::isfinite(dt_sample)) return fail(c, KX_EINVAL, "dt_sample must be finite and >= 0");
  if (max_restarts < 0) return fail(c, KX_EINVAL, "max_restarts must be >= 0");
  int axis = 0, idx = 0;
  int64_t P = 0;
  KX_TRY(check_plane(c, plane, &axis, &idx, &P));
  cudaStream_t A = c->stream;
  // with two basis slots the projected work of restart k (auxiliary stream)
  // overlaps the Arnoldi process of restart k + 1 (context stream); per-kernel
  // timing records on the context stream, so it runs everything there
  const bool ovl = c->d.batch >= 2 && !c->timing;
  cudaStream_t Bs = ovl ? c->aux_stream : A;
  // the cascade (one CTA per frequency) and the set-up CTA stay resident
  // beside the Arnoldi passes; their grids leave room for them (in both
  // modes: the grid fixes the order of the reductions, so the bits agree)
  struct SideCtas {
    kx_ctx* c;
    ~SideCtas() {
      c->side_ctas = 0;
      c->side_steps = 1 << 30;
      c->pdl = 0;
    }
  } side{c};
  c->side_ctas = nfreq + 1;
  // the projected work of a restart (set-up, cascade, ...) runs beside the
  // first steps of the next process; in the later steps the single-sweep
  // launches take every SM slot (half the steps covers it at 96^3 and
  // 128^3, where this runs 3-6 % faster than keeping the reservation
  // throughout).  The two-pass form, used on smaller grids whose processes
  // are shorter than the projected work, keeps it for every step.  A fixed
  // rule, so every mode has the same grids and bits.
  c->side_steps = (c->m + 1) / 2;
  // the Arnoldi chain of this method runs with programmatic dependent launch
  c->pdl = 1;
  const size_t vbytes = (size_t)c->n * c->esize;
  // restart 1 starts from v_1 = g / ||g|| in slot 0
  KX_CUDA(c, cudaMemcpyAsync(slot_col(c, 0, 0), d_g, vbytes, cudaMemcpyDeviceToDevice, A), "copy g");
  if (ovl) KX_TRY(upload_state(c, 1, fresh_state()));
  KX_TRY(upload_state(c, 0, fresh_state()));
  KX_TRY(launch_norm_init(c, 0, 1));
  SlotState st;
  KX_TRY(read_state(c, 0, &st));
  const double beta = st.beta;
  if (!std::isfinite(beta)) return fail(c, KX_ENONFINITE, "g is not finite");
  KX_CUDA(c, cudaMemsetAsync(c->d_rst_yp, 0, (size_t)nfreq * P * sizeof(double), A), "zero plane");
  KX_CUDA(c, cudaMemsetAsync(c->d_rst_state, 0, (size_t)nfreq * sizeof(int), A), "zero states");
  if (d_Y) {
    KX_CUDA(c, cudaMemsetAsync(d_Y, 0, (size_t)nfreq * vbytes, A), "zero Y");
    if (c->d.precision == KX_FP32)
      KX_CUDA(c, cudaMemsetAsync(c->d_zre, 0, (size_t)nfreq * vbytes, A), "zero Y low parts");
  }
  double* d_int = c->d_small + 128;
  std::vector<int> rcount(nfreq, 0);
  if (beta == 0.0) {
    // y = 0: every output is zero
    KX_TRY(launch_rst_out(c, A, nfreq, P, d_E_plane, d_int, nullptr));
    KX_TRY(sync(c));
    for (int f = 0; f < nfreq; ++f) {
      if (intensity) intensity[f] = 0.0;
      if (resid) resid[f] = 0.0;
      if (restarts) restarts[f] = 0;
    }
    return KX_OK;
  }
  KX_CUDA(c, cudaMemcpyAsync(c->d_omegas, omegas, sizeof(double) * nfreq, cudaMemcpyHostToDevice, A),
          "omega upload");
  KX_TRY(rst_arnoldi(c, 0));
  KX_TRY(read_state(c, 0, &st));
  if (st.status) return fail(c, (kx_status)st.status, "non-finite value in the Arnoldi process");
  // sample grid from ||H_m||_1 of the first restart
  const int ldh = c->m + 1;
  std::vector<double> Hh((size_t)ldh * c->m);
  KX_CUDA(c, cudaMemcpyAsync(Hh.data(), make_slot<double>(c, 0).H, Hh.size() * sizeof(double),
                             cudaMemcpyDeviceToHost, A), "H read");
  KX_TRY(sync(c));
  double nu = 0.0;
  for (int col = 0; col < st.m_done; ++col) {
    double sum = 0.0;
    for (int r = 0; r <= std::min(col + 1, st.m_done - 1); ++r) sum += std::fabs(Hh[r + (size_t)col * ldh]);
    nu = std::max(nu, sum);
  }
  if (!std::isfinite(nu)) return fail(c, KX_ENONFINITE, "non-finite Hessenberg matrix");
  const double per_unit = c->d.precision == KX_FP64 ? 0.3 : 1.0;
  double want = dt_sample > 0.0 ? T / dt_sample : T * nu / per_unit;
  want = std::max(1.0, std::ceil(want - 1e-9 * want));
  if (want > (double)c->d.rst_samples) {
    char msg[160];
    snprintf(msg, sizeof(msg), "T needs %.0f time samples; the context holds rst_samples = %d", want,
             c->d.rst_samples);
    return fail(c, KX_EINVAL, msg);
  }
  const int Nt = (int)want;
  const double d = T / Nt;
  const int kmax = max_restarts > 0 ? max_restarts
                                    : (int)std::min(100000.0, 3.0 * T * nu / c->m + 20.0);
  double* b = c->d_rst_b;
  KX_TRY(launch_rst_source(c, A, nfreq, beta, Nt, d, b));
  const double tol_abs = rtol * beta;
  bool all_stopped = false;
  int* h_states = reinterpret_cast<int*>(c->h_small);
  int* h_status = reinterpret_cast<int*>(c->h_small + 96);
  if (ovl) KX_CUDA(c, cudaEventRecord(c->ev_arnoldi, A), "event record");
  for (int k = 1;; ++k) {
    const int sl = ovl ? (k - 1) & 1 : 0;
    // projected work of restart k (Fig. alg:rst steps (2), (3))
    if (ovl) KX_CUDA(c, cudaStreamWaitEvent(Bs, c->ev_arnoldi, 0), "event wait");
    KX_CUDA(c, cudaMemsetAsync(c->d_small + 64, 0, sizeof(int), Bs), "status reset");
    KX_TRY(launch_rst_setup(c, Bs, sl, d));
    KX_TRY(launch_rst_cascade(c, Bs, nfreq, b, Nt, d, tol_abs));
    KX_TRY(launch_rst_plane(c, Bs, sl, nfreq, axis, idx, P));
    if (d_Y) KX_TRY(launch_rst_full(c, Bs, sl, nfreq, d_Y));
    KX_TRY(launch_rst_coef(c, Bs, nfreq, b, Nt, d));
    c->stats.expm_evals += 1;
    if (ovl) {
      KX_CUDA(c, cudaEventRecord(c->ev_proj[sl], Bs), "event record");
      // restart k + 1's Arnoldi process in the other slot, started before
      // restart k's stopping test is known (step (1) of the next pass)
      if (k < kmax) {
        const int nx = sl ^ 1;
        if (k >= 2) KX_CUDA(c, cudaStreamWaitEvent(A, c->ev_proj[nx], 0), "event wait");
        KX_TRY(launch_rst_nextvec(c, A, sl, nx));
        KX_TRY(launch_norm_init(c, nx, 1));
        KX_TRY(rst_arnoldi(c, nx));
        KX_CUDA(c, cudaEventRecord(c->ev_arnoldi, A), "event record");
      }
    }
    KX_CUDA(c, cudaMemcpyAsync(h_states, c->d_rst_state, sizeof(int) * nfreq, cudaMemcpyDeviceToHost, Bs),
            "state read");
    KX_CUDA(c, cudaMemcpyAsync(h_status, c->d_small + 64, sizeof(int), cudaMemcpyDeviceToHost, Bs),
            "status read");
    KX_CUDA(c, cudaStreamSynchronize(Bs), "stream synchronise");
    if (*h_status) {
      sync(c);
      if (*h_status == KX_ETIMEOUT)
        return fail(c, KX_ETIMEOUT, "Arnoldi process: a bounded wait for a basis copy ran out");
      return fail(c, KX_ENONFINITE, "restart set-up: non-finite Arnoldi process or projected exponential");
    }
    all_stopped = true;
    for (int f = 0; f < nfreq; ++f) {
      if (h_states[f] == 3) {
        sync(c);
        return fail(c, KX_ENONFINITE, "non-finite residual in the projected problem");
      }
      if (h_states[f] == 0 || h_states[f] == 1) rcount[f] = k;
      all_stopped = all_stopped && h_states[f] != 0;
    }
    if (all_stopped || k >= kmax) {
      if (ovl && k < kmax) {
        // restart k + 1's process runs speculatively in the other slot and is
        // not needed: its next step's finalisation stops it, and the launches
        // still queued return at entry; the request lands before the context
        // stream continues (it waits for the auxiliary stream below)
        int* one = reinterpret_cast<int*>(c->h_small + 255);
        *one = 1;
        SlotState* st_nx = c->d_state + (sl ^ 1);
        KX_CUDA(c, cudaMemcpyAsync(&st_nx->abort, one, sizeof(int), cudaMemcpyHostToDevice, Bs), "stop request");
        KX_CUDA(c, cudaEventRecord(c->ev_proj[sl], Bs), "event record");
      }
      break;
    }
    if (!ovl) {
      // the next basis starts from v_{m+1} (same slot, column m_done -> 0)
      KX_TRY(launch_rst_nextvec(c, A, 0, 0));
      KX_TRY(launch_norm_init(c, 0, 1));
      KX_TRY(rst_arnoldi(c, 0));
    }
  }
  if (ovl) KX_CUDA(c, cudaStreamWaitEvent(A, c->ev_proj[0], 0), "event wait");
  if (ovl) KX_CUDA(c, cudaStreamWaitEvent(A, c->ev_proj[1], 0), "event wait");
  KX_TRY(launch_rst_out(c, A, nfreq, P, d_E_plane, d_int, d_Y));
  KX_CUDA(c, cudaMemcpyAsync(c->h_small, d_int, sizeof(double) * nfreq, cudaMemcpyDeviceToHost, A),
          "intensity read");
  KX_CUDA(c, cudaMemcpyAsync(c->h_small + 64, c->d_rst_res, sizeof(double) * nfreq, cudaMemcpyDeviceToHost, A),
          "residual read");
  KX_TRY(sync(c));
  for (int f = 0; f < nfreq; ++f) {
    if (intensity) intensity[f] = c->h_small[f];
    if (resid) resid[f] = c->h_small[64 + f] / beta;
    if (restarts) restarts[f] = rcount[f];
  }
  if (!all_stopped) return fail(c, KX_ENOCONV, "restart in Krylov dimension: max_restarts reached");
  return KX_OK;
}

kx_status kx_set_permittivity(kx_ctx* c, const double* eps_cell) {
  if (!c || !eps_cell) return KX_EINVAL;
  const size_t bytes = (size_t)c->geo.ncell * sizeof(double);
  if (is_device_ptr(eps_cell)) {
    KX_CUDA(c, cudaMemcpyAsync(c->d_eps_cell, eps_cell, bytes, cudaMemcpyDeviceToDevice, c->stream), "eps copy");
  } else {
    for (int64_t i = 0; i < c->geo.ncell; ++i)
      if (!(eps_cell[i] > 0.0) || !std::isfinite(eps_cell[i]))
        return fail(c, KX_ENONFINITE, "eps_cell must be finite and > 0");
    KX_CUDA(c, cudaMemcpyAsync(c->d_eps_cell, eps_cell, bytes, cudaMemcpyHostToDevice, c->stream), "eps copy");
  }
  KX_TRY(launch_setup_material(c));
  return sync(c);
}

kx_status adjoint_response_grad(kx_ctx* c, const void* d_g, const double* omegas, int nfreq, double T,
                                double rtol, const int* plane, double* d_grad, double* loss) {
  if (!c) return KX_EINVAL;
  KX_TRY(check_vec(c, d_g, "d_g"));
  KX_TRY(check_omegas(c, omegas, nfreq));
  if (!d_grad || !loss || !plane) return fail(c, KX_EINVAL, "NULL argument");
  if (c->d.max_checkpoints <= 0) return fail(c, KX_EINVAL, "context created without checkpoint storage");
  if (!(T > 0.0) || !std::isfinite(T) || !(rtol > 0.0)) return fail(c, KX_EINVAL, "bad T or rtol");
  const int axis = plane[0], idx = plane[1];
  if (axis < 0 || axis >= c->d.dim) return fail(c, KX_EINVAL, "bad plane axis");
  const int na = axis == 0 ? c->geo.nx : (axis == 1 ? c->geo.ny : c->geo.nz);
  if (idx < 0 || idx >= na) return fail(c, KX_EINVAL, "bad plane index");
  const int64_t nE = (int64_t)c->geo.ne * c->geo.ncell;
  KX_CUDA(c, cudaMemsetAsync(c->d_adj_Q, 0, (size_t)nE * sizeof(double), c->stream), "zero Q");
  // ||g|| balances the augmented phase entries (as in response_at_freqs)
  KX_CUDA(c, cudaMemcpyAsync(slot_col(c, 0, 0), d_g, c->n * c->esize, cudaMemcpyDeviceToDevice, c->stream),
          "copy g");
  KX_TRY(upload_state(c, 0, fresh_state()));
  KX_TRY(launch_norm_init(c, 0, 1));
  SlotState gst;
  KX_TRY(read_state(c, 0, &gst));
  const double eta = gst.beta > 0.0 ? gst.beta : 1.0;
  double* d_int = c->d_small + 128;
  const size_t vbytes = (size_t)c->n * c->esize;
  for (int f = 0; f < nfreq; ++f) {
    const double W = omegas[f];
    // forward solution with a checkpoint at the start of every sub-step
    KX_CUDA(c, cudaMemsetAsync(slot_col(c, 0, 0), 0, vbytes, c->stream), "zero y");
    SlotState s = fresh_state();
    s.T = T;
    s.rtol = rtol;
    s.aug = 1;
    s.omega = W;
    s.eta = eta;
    s.tol_mode = 1;
    KX_TRY(upload_state(c, 0, s));
    KX_TRY(launch_norm_init(c, 0, 1));
    std::vector<double> tk, tauk;
    double tnow = 0.0;
    for (;;) {
      if ((int)tk.size() >= c->d.max_checkpoints)
        return fail(c, KX_ENOMEM, "adjoint: more time sub-steps than max_checkpoints");
      KX_CUDA(c, cudaMemcpyAsync((char*)c->d_ckpt + tk.size() * c->ld * c->esize, slot_col(c, 0, 0), vbytes,
                                 cudaMemcpyDeviceToDevice, c->stream), "checkpoint");
      tk.push_back(tnow);
      KX_TRY(arnoldi_steps(c, 0, 1, c->m, d_g));
      KX_TRY(launch_substep_control(c, 0, 1));
      KX_TRY(launch_combine(c, 0, 1));
      KX_TRY(read_states(c, 0, 1));
      const SlotState& st = c->h_state[0];
      if (st.status) return fail(c, (kx_status)st.status, "adjoint forward: Krylov process failed");
      tauk.push_back(st.t_acc);
      tnow = st.t_now;
      if (st.retired) break;
    }
    c->stats.substeps += (int64_t)tk.size();
    // loss and lambda(T) = 2 P^T P y(T) in slot 1
    KX_TRY(launch_response(c, f, omegas, T, 0, nullptr, nullptr, slot_col(c, 0, 0), axis, idx, nullptr,
                           d_int + f, nullptr));
    KX_CUDA(c, cudaMemsetAsync(slot_col(c, 1, 0), 0, vbytes, c->stream), "zero lambda");
    KX_TRY(launch_adj_seed(c, slot_col(c, 0, 0), slot_col(c, 1, 0), axis, idx));
    // backwards over the sub-steps
    for (int k = (int)tk.size() - 1; k >= 0; --k) {
      KX_CUDA(c, cudaMemcpyAsync(slot_col(c, 0, 0), (char*)c->d_ckpt + (size_t)k * c->ld * c->esize, vbytes,
                                 cudaMemcpyDeviceToDevice, c->stream), "restore checkpoint");
      SlotState s0 = fresh_state();
      s0.T = T;
      s0.aug = 1;
      s0.omega = W;
      s0.eta = eta;
      s0.t_now = tk[k];
      c->h_state[0] = s0;
      c->h_state[1] = fresh_state();
      KX_CUDA(c, cudaMemcpyAsync(c->d_state, c->h_state, 2 * sizeof(SlotState), cudaMemcpyHostToDevice,
                                 c->stream), "state upload");
      KX_TRY(sync(c));
      KX_TRY(launch_norm_init(c, 0, 2));
      for (int j = 0; j < c->m; ++j) {
        KX_TRY(launch_pass_a(c, 0, 1, j, d_g));
        KX_TRY(launch_pass_b(c, 0, 1, j, 1));
      }
      for (int j = 0; j < c->m; ++j) {
        KX_TRY(launch_pass_a_tr(c, 1, 1, j));
        KX_TRY(launch_pass_b(c, 1, 1, j, j == c->m - 1));
      }
      c->stats.arnoldi_steps += 2 * (int64_t)c->m;
      c->stats.matvecs += 2 * (int64_t)c->m;
      KX_TRY(read_states(c, 0, 2));
      if (c->h_state[0].status || c->h_state[1].status)
        return fail(c, KX_ENONFINITE, "adjoint backward: Krylov process failed");
      KX_CUDA(c, cudaMemsetAsync(c->d_small + 64, 0, sizeof(int), c->stream), "status reset");
      KX_TRY(launch_adj_substep(c, tauk[k], W, tk[k], d_g));
      KX_TRY(launch_combine(c, 1, 1));   // lambda(t_k) = W w(tau_k)
    }
  }
  KX_TRY(launch_adj_cells(c, d_grad));
  KX_CUDA(c, cudaMemcpyAsync(c->h_small, d_int, sizeof(double) * nfreq, cudaMemcpyDeviceToHost, c->stream),
          "loss read");
  KX_CUDA(c, cudaMemcpyAsync(c->h_small + 128, c->d_small + 64, sizeof(int), cudaMemcpyDeviceToHost, c->stream),
          "status read");
  KX_TRY(sync(c));
  int status = 0;
  std::memcpy(&status, c->h_small + 128, sizeof(int));
  if (status) return fail(c, KX_ENONFINITE, "adjoint: singular projected exponential");
  double L = 0.0;
  for (int f = 0; f < nfreq; ++f) L += c->h_small[f];
  *loss = L;
  return KX_OK;
}

// Independent problems solved concurrently: a pool of host threads takes
// the contexts largest-first from a shared counter; each context runs on its
// own stream, so the kernels of different problems overlap on the GPU.
kx_status response_at_freqs_multi(kx_ctx* const* ctxs, int nctx, const void* const* d_g,
                                  const double* omegas, int nfreq, double T, double rtol, int method,
                                  const int* planes, double* intensity, double* err_est, int nthreads) {
  if (!ctxs || nctx < 1 || !d_g || !omegas || !planes || nfreq < 1) {
    g_create_err = "response_at_freqs_multi: bad argument";
    return KX_EINVAL;
  }
  for (int i = 0; i < nctx; ++i)
    if (!ctxs[i]) {
      g_create_err = "response_at_freqs_multi: NULL context";
      return KX_EINVAL;
    }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    g_create_err = "response_at_freqs_multi: no CUDA device";
    return KX_ECUDA;
  }
  std::vector<int> order(nctx);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return ctxs[a]->n > ctxs[b]->n; });
  std::atomic<int> next{0};
  std::atomic<int> first_err{KX_OK};
  std::mutex mu;
  std::string err_text;
  auto worker = [&]() {
    cudaSetDevice(dev);
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= nctx || first_err.load() != KX_OK) return;
      const int i = order[k];
      const kx_status st = response_at_freqs(ctxs[i], d_g[i], omegas + (size_t)i * nfreq, nfreq, T, rtol, method,
                                             planes + 2 * i, nullptr, intensity ? intensity + (size_t)i * nfreq : nullptr,
                                             err_est ? err_est + (size_t)i * nfreq : nullptr, nullptr);
      if (st != KX_OK) {
        int expect = KX_OK;
        if (first_err.compare_exchange_strong(expect, st)) {
          std::lock_guard<std::mutex> lk(mu);
          err_text = std::string("problem ") + std::to_string(i) + ": " + ctxs[i]->err;
        }
        return;
      }
    }
  };
  const int nt = std::max(1, std::min(nthreads, nctx));
  std::vector<std::thread> pool;
  for (int t = 1; t < nt; ++t) pool.emplace_back(worker);
  worker();
  for (auto& th : pool) th.join();
  if (first_err.load() != KX_OK) {
    g_create_err = err_text;
    return (kx_status)first_err.load();
  }
  return KX_OK;
}

kx_status kx_get_stats(const kx_ctx* c, kx_stats* out) {
  if (!c || !out) return KX_EINVAL;
  *out = c->stats;
  return KX_OK;
}

kx_status kx_reset_stats(kx_ctx* c) {
  if (!c) return KX_EINVAL;
  std::memset(&c->stats, 0, sizeof(c->stats));
  return KX_OK;
}

const char* kx_last_error(const kx_ctx* c) {
  return c ? c->err : g_create_err.c_str();
}

}  // extern "C"

// ===========================================================================
// Per-kernel-class timing.
namespace kx {

void time_begin(kx_ctx* c) {
  if (!c->timing) return;
  cudaEventCreate(&c->pending_a);
  cudaEventRecord(c->pending_a, c->stream);
}

void time_end(kx_ctx* c, int cls, double bytes) {
  if (!c->timing || !c->pending_a) return;
  cudaEvent_t b;
  cudaEventCreate(&b);
  cudaEventRecord(b, c->stream);
  c->timed.push_back({cls, c->pending_a, b, bytes});
  c->pending_a = nullptr;
}

}  // namespace kx

extern "C" {

kx_status kx_wait_selftest(kx_ctx* c, unsigned rounds) {
  if (!c) return KX_EINVAL;
  if (rounds == 0 || rounds > KX_WAIT_SELFTEST_MAX_ROUNDS)
    return fail(c, KX_EINVAL, "rounds must be 1 .. KX_WAIT_SELFTEST_MAX_ROUNDS (4194304)");
  int* d_status = reinterpret_cast<int*>(c->d_small + 200);
  KX_CUDA(c, cudaMemsetAsync(d_status, 0xff, sizeof(int), c->stream), "status reset");
  KX_TRY(launch_wait_selftest(c, rounds, d_status));
  int h = -1;
  KX_CUDA(c, cudaMemcpyAsync(&h, d_status, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "status read");
  KX_TRY(sync(c));
  if (h == KX_ETIMEOUT) return fail(c, KX_ETIMEOUT, "bounded device wait ran out (self-test)");
  if (h != KX_OK) return fail(c, KX_ECUDA, "self-test kernel did not report");
  return KX_OK;
}

kx_status kx_set_timing(kx_ctx* c, int on) {
  if (!c) return KX_EINVAL;
  c->timing = on ? 1 : 0;
  return KX_OK;
}

kx_status kx_kernel_times(kx_ctx* c, kx_kernel_time out[KX_NKCLASS]) {
  if (!c || !out) return KX_EINVAL;
  for (int k = 0; k < KX_NKCLASS; ++k) out[k] = {0.0, 0.0, 0};
  cudaError_t e = cudaStreamSynchronize(c->stream);
  if (e != cudaSuccess) return cuda_fail(c, e, "stream synchronise");
  for (auto& t : c->timed) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, t.a, t.b);
    if (t.cls >= 0 && t.cls < KX_NKCLASS) {
      out[t.cls].ms += ms;
      out[t.cls].bytes += t.bytes;
      out[t.cls].launches += 1;
    }
    cudaEventDestroy(t.a);
    cudaEventDestroy(t.b);
  }
  c->timed.clear();
  return KX_OK;
}

}  // extern "C"

namespace kx {

int persistent_grid(kx_ctx* c, const void* kernel, int64_t rounds, size_t smem) {
  int occ = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, kernel, NTHREADS, smem) != cudaSuccess || occ < 1) {
    cudaGetLastError();
    occ = 1;
  }
  const int64_t cap = std::min<int64_t>((int64_t)c->nsm * occ, c->ps);
  return (int)std::max<int64_t>(1, std::min<int64_t>(rounds, cap));
}

kx_status smem_opt_in(kx_ctx* c, SmemOptIn& rec, const void* kernel, size_t bytes) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(c->err, sizeof(c->err), "cudaGetDevice: %s", cudaGetErrorString(e));
    return KX_ECUDA;
  }
  if (dev < 0 || dev >= SMEM_MAX_DEVICES) {
    snprintf(c->err, sizeof(c->err), "device index %d beyond %d", dev, SMEM_MAX_DEVICES);
    return KX_EINVAL;
  }
  if (__atomic_load_n(&rec.done[dev], __ATOMIC_ACQUIRE)) return KX_OK;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    snprintf(c->err, sizeof(c->err), "setting %zu bytes of dynamic shared memory: %s", bytes,
             cudaGetErrorString(e));
    return KX_ECUDA;
  }
  // stored after the attribute is in place: a thread that sees the flag may launch
  __atomic_store_n(&rec.done[dev], 1, __ATOMIC_RELEASE);
  return KX_OK;
}

}  // namespace kx
