// Internal declarations shared by the library's translation units.
#pragma once

#include <algorithm>
#include <cuda_runtime.h>
#include <stdint.h>
#include <cstdio>
#include <string>
#include <vector>

#include "../../include/kx.h"

namespace kx {

constexpr int MMAX = 64;            // largest Krylov dimension
constexpr int PCOLS = MMAX + 3;     // partial-sum columns per slot
constexpr int FINB_COL = PCOLS - 1; // pass B's norm partials (pass A writes columns <= MMAX)
constexpr int NTHREADS = 256;       // threads per block of the bulk kernels
constexpr int NWARPS = NTHREADS / 32;
constexpr int MAXF = 64;            // largest number of frequencies per call

// Geometry of one grid, passed by value to kernels.
struct Geo {
  int dim, nx, ny, nz;
  int64_t ncell;
  int ncomp, nh;
  int ne;                // E field components (1 in 2D, 3 in 3D)
  int pml;               // 1: 2D with the auxiliary PML field P as component 3
  unsigned maskbits[6];  // bit a set: node index 0 along axis a is a wall node
  int la;                // layer axis
  int sighalf[6];        // 1 if the component is half-integer along la
};

// Device-side state of one Krylov basis (one "slot").
struct SlotState {
  int done;          // Arnoldi stopped (lucky breakdown)
  int m_done;        // Arnoldi steps completed in this restart
  int finished;      // time stepping reached T
  int status;        // 0 ok, else a kx_status code raised on the device
  double wmax;       // max ||A v_j|| of this restart (breakdown scale)
  double beta;       // norm of the current starting vector
  double t_now;      // time reached
  double T;          // final time
  double tau_try;    // trial sub-step length
  double rtol;       // requested relative accuracy
  double tol_abs;    // allowed error per unit time (tol_mode 0, set at the first sub-step)
  double err_acc;    // accumulated error estimate
  double t_acc;      // last accepted sub-step
  double omega, eta; // augmented mode: angular frequency and phase scaling
  int aug;           // 1: state carries [eta sin, eta cos]
  int tol_mode;      // 0: tolerance from the initial norm; 1: from the current norm
  int k_acc;
  int substeps;
  int expm_evals;
  int retired;       // final combination done: every later kernel skips this slot
  int abort;         // set by the host while a process runs: the next step's
                     // finalisation stops it (done = 1), so the launches after
                     // it skip the slot (a speculative process found unneeded)
};

// The host's stop request of a running Arnoldi process, read by the block
// that finalises a step (it may land at any time: read past the caches).
__device__ __forceinline__ bool abort_requested(const SlotState* st) {
  return *reinterpret_cast<const volatile int*>(&st->abort) != 0;
}

// Pointers of one slot's workspace.
template <typename T>
struct Slot {
  T* V;              // (m+1) columns of ld scalars; stored columns are unnormalised
  double* aug;       // (m+1) x 2 augmented entries of each column (FP64)
  double* H;         // (m+1) x m, ldh = m+1, column-major
  double* scale;     // m+2 column scales: v_i = scale[i] * V_i
  double* part;      // PCOLS x ps partial sums, column-major by block
  int ps;            // partial-sum column stride (>= any grid size)
  unsigned* counter; // block-completion counter (8 slots)
  double* u;         // projected coefficients (m)
  SlotState* st;
};

// Consecutive slots: slot y's pointers are slot 0's plus y times the strides.
template <typename T>
struct SlotSet {
  Slot<T> s0;
  int64_t sV, saug, sH, sscale, spart, su;
};

template <typename T>
__host__ __device__ __forceinline__ Slot<T> slot_at(const SlotSet<T>& ss, int y) {
  Slot<T> s = ss.s0;
  s.V += y * ss.sV;
  s.aug += y * ss.saug;
  s.H += y * ss.sH;
  s.scale += y * ss.sscale;
  s.part += y * ss.spart;
  s.u += y * ss.su;
  s.counter += 8 * y;
  s.st += y;
  return s;
}

// Output plane perpendicular to `axis` at index `idx`: its nodes are
// t = q * (na * nb) + a + na * b, q the E component and (a, b) the two
// in-plane indices in increasing axis order.
__host__ __device__ __forceinline__ void plane_dims(const Geo& g, int axis, int* na, int* nb) {
  *na = axis == 0 ? g.ny : g.nx;
  *nb = g.dim == 2 ? 1 : (axis == 2 ? g.ny : g.nz);
}

__host__ __device__ __forceinline__ int64_t plane_node(const Geo& g, int axis, int idx, int64_t t) {
  int na, nb;
  plane_dims(g, axis, &na, &nb);
  const int64_t np = (int64_t)na * nb;
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
  return (int64_t)(g.nh + q) * g.ncell + ((int64_t)k * g.ny + j) * g.nx + i;
}

// Restart in Krylov dimension: polynomial degree + 1 of the interpolated
// source on one sample interval, and the layout (in doubles) of the per-
// restart set-up record: E = exp(-d H_m) (MMAX x MMAX, row-major), the
// interval responses W_j (RST_P x MMAX), the last rows of H_m and H_m^2, and
// the scalars h_{m+1,m}, (H_m)_{m,1}, m.
constexpr int RST_P = 6;
constexpr int RST_OFF_W = MMAX * MMAX;
constexpr int RST_OFF_R1 = RST_OFF_W + RST_P * MMAX;
constexpr int RST_OFF_R2 = RST_OFF_R1 + MMAX;
constexpr int RST_OFF_SC = RST_OFF_R2 + MMAX;
constexpr int RST_MATS = RST_OFF_SC + 8;

// Single-sweep Arnoldi (sweep.cu): reduced partial columns of the last
// pass, and the coefficients the next sweep applies.  One record per slot.
constexpr int SWCOLS = 2 * MMAX + 3;   // dots against t2 and t1 per column, x.x, x.y, y.y
constexpr int SW_RED = 16;             // blocks in front of an apply pass (from step 1) that finalise the step
constexpr int SW_TILE = 4 * NTHREADS;  // cells of one tile of the staged sweep (a quad a thread)
struct SwCoef {
  double tot[SWCOLS];   // reduced columns of the last sweep (step 0: v_0 . A v_0, ||A v_0||^2)
  double hc[MMAX + 1];  // h_{i,j-1}, i < j: the column the sweep S_j removes from A v_{j-1}
  double cp[MMAX + 1];  // c_k, k < j: sum_{i<j-1} h_{k,i} h_{i,j-1} (A v_i through the Arnoldi relation)
  double uh[MMAX + 1];  // sum_{l=i}^{j-1} G_{i,l} hc_l, row i < j (apply pass K_j)
  double uc[MMAX + 1];  // sum_{k=i}^{j-1} G_{i,k} c_k,  row i < j (apply pass K_j)
  double sprev;         // scale of column j-1
  double hjj;           // h_{j-1,j-1}
  unsigned counter;     // block-completion counter of the apply pass
};

// Pointers of the single-sweep workspace of one slot.
struct SwSlot {
  double* part;   // SWCOLS x ps block partials, column-major by block
  int ps;
  double* G;      // (MMAX+1) x (MMAX+1) Gram matrix v_i . v_k, column-major
  SwCoef* co;
  void* t;        // one vector: A V_{j-1} (shared by the slots: one process runs at a time)
};

// One problem of a batch (kx_batch): what its single-sweep Arnoldi kernels
// need, for both basis slots, and its block ranges in the batched launches
// (the apply launch's blocks [a0, a0 + na), the sweep launch's [s0, s0 + ns)).
struct SwInst {
  Geo g;
  Slot<float> s[2];
  SwSlot w[2];
  const float* ie;
  const float* sig2;
  int64_t ld;
  int ldh;
  int a0, na, s0, ns;
  // the column-march apply launch of steps j >= 1: blocks [c0, c0 + nc),
  // SW_RED reducers then ncb column blocks on each range of kz planes
  int c0, nc, ncb, kz;
};

struct Material {
  const void* inv_eps;   // (ncomp - nh) x ncell, 1 / mean eps on E nodes
  const void* sig2;      // sigma at 2*index + half along the layer axis
};

}  // namespace kx

struct kx_ctx {
  kx_desc d;
  cudaStream_t stream;
  bool own_stream = false;   // created by (and destroyed with) the context
  kx::Geo geo;
  int64_t n;        // unknowns
  int64_t ld;       // stride between stored basis columns
  int esize;        // bytes per scalar
  int m;            // krylov_dim
  int nblk;         // blocks of the light bulk kernels
  int nsm;          // streaming multiprocessors
  int ps;           // partial-sum column stride = nsm * 8
  void* d_inv_eps;
  void* d_sig2;
  double* d_eps_cell;
  // per-slot workspace
  void* d_V;
  double* d_aug;
  double* d_H;
  double* d_scale;
  double* d_part;
  unsigned* d_counter;
  double* d_u;
  kx::SlotState* d_state;
  kx::SlotState* h_state;   // pinned host mirror
  // stationary-solve workspace
  double* d_rho;            // 2 x MAXF complex residual coefficients
  float* d_coef;            // 2 x MAXF x MMAX update coefficients (FP32 path)
  double* d_coefd;          // 2 x MAXF x MMAX update coefficients (FP64 path)
  double* d_omegas;         // MAXF
  double* d_small;          // scratch for small host<->device transfers
  double* h_small;          // pinned
  void* d_tmp;              // one extra vector
  void* d_tmp2;             // one extra vector
  double* d_expm_ws;        // projected exponential workspace
  // adjoint workspace (max_checkpoints > 0)
  void* d_ckpt = nullptr;   // max_checkpoints states of the forward solution
  double* d_adj_Q = nullptr;      // per-E-node time integrals
  float* d_adj_alpha = nullptr;   // quadrature coefficients
  float* d_adj_omg = nullptr;
  float* d_adj_cw = nullptr;
  float* d_adj_sn = nullptr;
  double* d_gauss = nullptr;      // Gauss-Legendre nodes and weights on [0, 1]
  int adj_nq_max = 0;
  void* d_zre;              // stationary parts, max_freqs x n (real)
  void* d_zim;              // stationary parts, max_freqs x n (imaginary)
  // restart in Krylov dimension (rst_samples > 0)
  double* d_rst_b = nullptr;     // 2 x max_freqs x rst_samples x RST_P source coefficients
  double* d_rst_smp = nullptr;   // max_freqs x (rst_samples + 1) x 3 alphahat samples
  double* d_rst_mats = nullptr;  // set-up record of the current restart
  double* d_rst_u = nullptr;     // MAXF x MMAX projected solutions u(T)
  double* d_rst_res = nullptr;   // MAXF residual maxima
  int* d_rst_state = nullptr;    // MAXF: 0 active, 1 stops after this restart, 2 stopped
  double* d_rst_yp = nullptr;    // max_freqs x plane-node accumulators
  int64_t rst_plane_max = 0;     // plane nodes the accumulators hold per frequency
  cudaStream_t aux_stream = nullptr;   // projected work overlapping the next Arnoldi process
  int side_ctas = 0;        // long-lived CTAs of other kernels sharing the SMs meanwhile
  int side_steps = 1 << 30; // leading steps of each Arnoldi process that the side CTAs may overlap
  int pdl = 0;              // launch the Arnoldi chain with programmatic dependent launch
  // single-sweep Arnoldi workspace (per slot, and one shared vector)
  void* d_swT = nullptr;
  double* d_swpart = nullptr;
  double* d_swG = nullptr;
  kx::SwCoef* d_swco = nullptr;
  cudaEvent_t ev_arnoldi = nullptr;    // Arnoldi process of a restart complete
  cudaEvent_t ev_proj[2] = {nullptr, nullptr};  // projected work done with basis slot 0 / 1
  kx_stats stats;
  char err[512] = {0};   // fixed buffer: recording an error allocates nothing
  // per-kernel-class timing (kx_set_timing)
  int timing = 0;
  struct TimedLaunch { int cls; cudaEvent_t a, b; double bytes; };
  std::vector<TimedLaunch> timed;
  cudaEvent_t pending_a = nullptr;
};

// ---------------------------------------------------------------------------
// Launch helpers implemented in the .cu files.
namespace kx {

// stencil.cu  (slot0, ns: the consecutive slots [slot0, slot0 + ns) advance together)
kx_status launch_setup_material(kx_ctx* c);
// d_eps_cell[i] = d_table[d_id[i]]; *d_bad = 1 if an id is >= n_mat
kx_status launch_expand_materials(kx_ctx* c, const uint8_t* d_id, const double* d_table, int n_mat, int* d_bad);
kx_status launch_apply(kx_ctx* c, const void* v, void* w, int transpose);
kx_status launch_pass_a(kx_ctx* c, int slot0, int ns, int j, const void* g_aug);
// pass A with the transposed operator A^T
kx_status launch_pass_a_tr(kx_ctx* c, int slot0, int ns, int j);
// pass A reading the per-cell permittivity directly (no 1/eps table)
kx_status launch_pass_a_cells(kx_ctx* c, int slot, int j, const double* d_eps_cell);
// pass B of step j; finalize = 1 launches its finalisation kernel, otherwise
// the next step's pass A finalises it (non-augmented processes only)
kx_status launch_pass_b(kx_ctx* c, int slot0, int ns, int j, int finalize);
int pass_b_grid(kx_ctx* c);

// adjoint.cu
kx_status launch_adj_seed(kx_ctx* c, const void* y, void* lam, int axis, int idx);
kx_status launch_adj_substep(kx_ctx* c, double tau, double omega, double tk, const void* g);
kx_status launch_adj_cells(kx_ctx* c, double* grad);
void gauss_legendre01(int n, double* x, double* w);
int gauss_points();

// linalg.cu
kx_status launch_norm_init(kx_ctx* c, int slot0, int ns);
kx_status launch_combine(kx_ctx* c, int slot0, int ns);
kx_status launch_basis_export(kx_ctx* c, int slot, void* dV, int m);
// y += a x, n scalars of the context's precision
kx_status launch_axpy(kx_ctx* c, double a, const void* x, void* y);
kx_status launch_zupdate(kx_ctx* c, int slot, int nfreq, void* zre, void* zim, int m);
kx_status launch_true_residual(kx_ctx* c, const void* g, int nfreq, const double* d_om,
                               void* zre, void* zim, double* out_host);
kx_status launch_response(kx_ctx* c, int f, const double* h_om, double T, int split,
                          const void* zre, const void* zim, const void* Y, int plane_axis,
                          int plane_idx, void* E_plane, double* d_intensity, void* Yout);

// rstdim.cu
// (launches on stream st: the context's stream, or its auxiliary stream
// when the projected work overlaps the next restart's Arnoldi process)
kx_status launch_rst_source(kx_ctx* c, cudaStream_t st, int nfreq, double beta, int Nt, double d, double* b);
kx_status launch_rst_setup(kx_ctx* c, cudaStream_t st, int slot, double d);
kx_status launch_rst_cascade(kx_ctx* c, cudaStream_t st, int nfreq, const double* b, int Nt, double d,
                             double tol_abs);
kx_status launch_rst_coef(kx_ctx* c, cudaStream_t st, int nfreq, double* b, int Nt, double d);
kx_status launch_rst_plane(kx_ctx* c, cudaStream_t st, int slot, int nfreq, int axis, int idx, int64_t P);
kx_status launch_rst_full(kx_ctx* c, cudaStream_t st, int slot, int nfreq, void* Y);
kx_status launch_rst_out(kx_ctx* c, cudaStream_t st, int nfreq, int64_t P, void* E_plane, double* d_intensity,
                         void* Y);
// column m_done of basis slot `from` (the unnormalised v_{m+1}) -> column 0 of slot `to`
kx_status launch_rst_nextvec(kx_ctx* c, cudaStream_t st, int from, int to);

// sweep.cu: m steps of the single-sweep Arnoldi process on basis slot
// `slot`, from its column 0 as set by launch_norm_init (non-augmented)
kx_status sweep_arnoldi(kx_ctx* c, int slot, int m);
// the same for every problem of a batch at once (3D FP32, nx % 4 == 0): one
// launch per Arnoldi phase; tab/aoff/soff/coff device copies of the instance
// table and of the block offsets of the step-0 apply, sweep and column-march
// apply launches (n + 1 entries each), na/ns/nc the launch totals
// the per-device set-up of its launches (dynamic shared memory opt-in), done
// before a stream capture of them
kx_status sweep_batch_prepare(kx_ctx* c0);
kx_status sweep_arnoldi_batch(kx_ctx* c0, cudaStream_t st, const SwInst* tab, const int* aoff, const int* soff,
                              const int* coff, int n, int na, int ns, int nc, int slot, int m, int64_t* launches,
                              std::vector<std::pair<cudaEvent_t, cudaEvent_t>>* sweep_events);
size_t sweep_smem_bytes();
const void* sweep_batch_kernel();
// the bounded mbarrier wait of the sweep on a barrier nothing completes
kx_status launch_wait_selftest(kx_ctx* c, unsigned rounds, int* d_status);

// projected.cu
kx_status launch_substep_control(kx_ctx* c, int slot0, int ns);
kx_status launch_expm_project(kx_ctx* c, const double* dH, int ldh, int m, double beta,
                              double tau, const double* d_om, int nfreq, double* d_u);
kx_status launch_shifted_solve(kx_ctx* c, int slot, int nfreq, int m);

size_t expm_smem_bytes(int msz);

// Persistent grid for a kernel: resident blocks (occupancy) x SMs, capped
// by the work and by the partial-sum stride.
int persistent_grid(kx_ctx* c, const void* kernel, int64_t items_per_block_round, size_t smem);

// Opt-in of a kernel to more than 48 KB of dynamic shared memory.  The
// attribute belongs to the device that is current when it is set, so the
// record of which devices have it is kept per device; a set that fails is
// not recorded, and the caller gets KX_ECUDA (with the reason in c->err)
// instead of a launch that would fail later.
constexpr int SMEM_MAX_DEVICES = 64;
struct SmemOptIn {
  int done[SMEM_MAX_DEVICES];   // accessed atomically (1: set on that device)
};
kx_status smem_opt_in(kx_ctx* c, SmemOptIn& rec, const void* kernel, size_t bytes);

// Programmatic dependent launch.  A kernel of the Arnoldi chain may be
// launched while its predecessor in the stream is still running; it waits
// (griddepcontrol.wait: the predecessor grid has completed and its memory
// is visible) before touching any data, and lets its own successor start
// launching right away.  Without a programmatic predecessor the wait
// returns at once.
__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
}

// The two halves of pdl_enter, for kernels that let their successor launch
// only near their end: successor blocks launched early wait on the SMs and
// would hold the room that kernels of another stream, running beside the
// chain, need.  A block that exits counts as having triggered.
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" :::); }

template <typename... KArgs, typename... Args>
inline void launch_k(const kx_ctx* c, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem,
                     cudaStream_t st, Args... args) {
  if (c->pdl) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, kern, args...);
  } else {
    kern<<<grid, block, smem, st>>>(args...);
  }
}

// A persistent grid of gr blocks (full occupancy) shrunk by the CTAs that
// other, concurrently running kernels keep resident, so that every block
// still finds a slot in the first wave.
inline int reserve_grid(const kx_ctx* c, int nb, int gr) {
  if (c->side_ctas <= 0) return nb;
  return std::min(nb, std::max(c->nsm, gr - c->side_ctas));
}

// The same for the launches of Arnoldi step j: the side CTAs are only
// expected beside the first side_steps steps of a process.
inline int reserve_grid_at(const kx_ctx* c, int nb, int gr, int j) {
  return j < c->side_steps ? reserve_grid(c, nb, gr) : nb;
}

// Timing brackets around one launch (no-ops unless timing is on).
void time_begin(kx_ctx* c);
void time_end(kx_ctx* c, int cls, double bytes);

}  // namespace kx

namespace kx {
// Workspace pointers of basis slot `slot` of a context.
template <typename T>
inline Slot<T> make_slot(kx_ctx* c, int slot) {
  Slot<T> s;
  const int m = c->m;
  s.V = (T*)c->d_V + (int64_t)slot * (m + 1) * c->ld;
  s.aug = c->d_aug + (int64_t)slot * (m + 1) * 2;
  s.H = c->d_H + (int64_t)slot * (m + 1) * m;
  s.scale = c->d_scale + (int64_t)slot * (m + 2);
  s.part = c->d_part + (int64_t)slot * PCOLS * c->ps;
  s.ps = c->ps;
  s.counter = c->d_counter + slot * 8;
  s.u = c->d_u + (int64_t)slot * (m + 2);
  s.st = c->d_state + slot;
  return s;
}

template <typename T>
inline SlotSet<T> make_slotset(kx_ctx* c, int slot0) {
  SlotSet<T> ss;
  const int m = c->m;
  ss.s0 = make_slot<T>(c, slot0);
  ss.sV = (int64_t)(m + 1) * c->ld;
  ss.saug = (int64_t)(m + 1) * 2;
  ss.sH = (int64_t)(m + 1) * m;
  ss.sscale = m + 2;
  ss.spart = (int64_t)PCOLS * c->ps;
  ss.su = m + 2;
  return ss;
}
}  // namespace kx

#define KX_CHECK_LAUNCH(ctx)                                                        \
  do {                                                                              \
    cudaError_t e__ = cudaGetLastError();                                           \
    if (e__ != cudaSuccess) {                                                       \
      snprintf((ctx)->err, sizeof((ctx)->err), "kernel launch failed: %s at %s:%d", \
               cudaGetErrorString(e__), __FILE__, __LINE__);                        \
      return KX_ECUDA;                                                              \
    }                                                                               \
    (ctx)->stats.kernel_launches++;                                                 \
  } while (0)
