// Batched restart in Krylov dimension over many independent problems (the
// uneven batch: scatterer instances of different sizes, a few frequencies
// each; declared in include/kx.h as kx_batch_* and
// response_restart_dim_batch).
//
// Every problem keeps its own context (grid, medium, two basis slots,
// restart-in-dimension workspace, auxiliary stream).  The Arnoldi process of
// a restart (Sect. 3.2), which moves nearly all the bytes, runs for all
// problems together: one launch per phase (apply, sweep, last step) on the
// batch's stream, its blocks split between the problems by a table in
// device memory (SwInst, sweep.cu).  The per-frequency projected work of
// restart k (Fig. alg:rst steps (2), (3): set-up, cascade, plane, next
// coefficients; rstdim.cu) runs per problem on that problem's auxiliary
// stream, beside restart k + 1's batched Arnoldi process, as in the
// single-problem driver.
//
// The split of each launch between problems is chosen by an autotuner: for
// the batch's size class (the multiset of its grids) it times a short
// Arnoldi process of the whole batch under each candidate granularity --
// tiles of the staged sweep per block, stencil rounds per apply thread --
// keeps the fastest, and caches the choice for later batches of the same
// size class in this process.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "kx_internal.cuh"

using namespace kx;

struct kx_batch {
  std::vector<kx_ctx*> ctx;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::vector<SwInst> tab;
  std::vector<int> aoff, soff, coff;   // block offsets of the step-0 apply, sweep and column apply launches
  SwInst* d_tab = nullptr;
  int* d_off = nullptr;          // aoff, soff, coff (n + 1 each)
  int na = 0, ns = 0, nc = 0;    // launch totals
  int tpb = 0, rpt = 0;          // chosen granularity: sweep tiles per block, apply rounds per thread
  int from_cache = 0;
  double tune_ms = 0.0;
  cudaEvent_t ev_arn = nullptr;
  int* h_pin = nullptr;          // pinned host words: per problem MAXF states + a status; one word = 1
  int64_t launches = 0;
  // the batched Arnoldi process of each basis slot captured once as a CUDA
  // graph and replayed every restart (re-captured when the launch split or
  // the Krylov dimension changes; direct launches while tuning or timing)
  cudaGraphExec_t graph[2] = {nullptr, nullptr};
  int graph_m[2] = {0, 0};
  int64_t graph_count[2] = {0, 0};   // kernel launches one replay holds
  int64_t graph_replays = 0;
  bool tuning = false;
  bool graphs_off = false;           // a capture failed: direct launches from then on
  // per-launch event timing of the batched sweep launches (kx_batch_set_timing)
  int timing = 0;
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> sweep_events;
  std::vector<double> sweep_bytes;   // algorithmic bytes of each timed launch
  double sweep_ms = 0.0, sweep_bytes_sum = 0.0;
  int64_t sweep_timed = 0;
  char err[512] = {0};
};

namespace {

thread_local std::string g_batch_err;

kx_status bfail(kx_batch* b, kx_status code, const std::string& msg) {
  if (b) snprintf(b->err, sizeof(b->err), "%s", msg.c_str());
  else g_batch_err = msg;
  return code;
}

kx_status bcuda(kx_batch* b, cudaError_t e, const char* what) {
  cudaGetLastError();
  return bfail(b, KX_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

#define KB_CUDA(b, expr, what)                        \
  do {                                                \
    cudaError_t e__ = (expr);                         \
    if (e__ != cudaSuccess) return bcuda((b), e__, (what)); \
  } while (0)

// A launcher's status, with the context's own text carried over.
#define KB_TRY(b, c, expr)                                                 \
  do {                                                                     \
    kx_status s__ = (expr);                                                \
    if (s__ != KX_OK) return bfail((b), s__, std::string("problem: ") + (c)->err); \
  } while (0)

#define KB_OK(expr)               \
  do {                            \
    kx_status s__ = (expr);       \
    if (s__ != KX_OK) return s__; \
  } while (0)

constexpr int LGB = MMAX + 1;

SwSlot sw_slot_of(kx_ctx* c, int slot) {
  SwSlot w;
  w.part = c->d_swpart + (int64_t)slot * SWCOLS * c->ps;
  w.ps = c->ps;
  w.G = c->d_swG + (int64_t)slot * LGB * LGB;
  w.co = c->d_swco + slot;
  w.t = c->d_swT;
  return w;
}

void* col_ptr(kx_ctx* c, int slot, int col) {
  return (char*)c->d_V + ((int64_t)slot * (c->m + 1) + col) * c->ld * c->esize;
}

// The problems' own streams are swapped for the batch's during a call, so
// that their per-problem launches (normalisation, next start vector) order
// with the batched Arnoldi launches; restored on exit.
struct StreamSwap {
  std::vector<std::pair<kx_ctx*, cudaStream_t>> saved;
  explicit StreamSwap(kx_batch* b) {
    for (kx_ctx* c : b->ctx) {
      saved.push_back({c, c->stream});
      c->stream = b->stream;
      c->pdl = 0;
      c->side_ctas = 0;
    }
  }
  ~StreamSwap() {
    for (auto& p : saved) p.first->stream = p.second;
  }
};

void drop_graphs(kx_batch* b) {
  for (int s = 0; s < 2; ++s) {
    if (b->graph[s]) cudaGraphExecDestroy(b->graph[s]);
    b->graph[s] = nullptr;
    b->graph_m[s] = 0;
    b->graph_count[s] = 0;
  }
}

// Launch split for a granularity: problem i gets ns_i = ceil(tiles_i / tpb)
// sweep blocks, SW_RED + ceil(quads_i / (NTHREADS rpt)) step-0 apply blocks,
// each capped by its partial-sum stride, and SW_RED + ncb_i ceil(nz_i / kz)
// column-march apply blocks with kz = 2 rpt planes a block.
kx_status set_grids(kx_batch* b, int tpb, int rpt) {
  const int n = (int)b->ctx.size();
  drop_graphs(b);
  b->aoff.assign(n + 1, 0);
  b->soff.assign(n + 1, 0);
  b->coff.assign(n + 1, 0);
  for (int i = 0; i < n; ++i) {
    kx_ctx* c = b->ctx[i];
    const int64_t ntiles = (c->geo.ncell + SW_TILE - 1) / SW_TILE;
    const int64_t nquads = c->geo.ncell / 4;
    const int ns = (int)std::max<int64_t>(1, std::min<int64_t>((ntiles + tpb - 1) / tpb, c->ps));
    const int nst = (int)std::max<int64_t>(
        1, std::min<int64_t>((nquads + (int64_t)NTHREADS * rpt - 1) / ((int64_t)NTHREADS * rpt), c->ps - SW_RED));
    SwInst& I = b->tab[i];
    I.s0 = b->soff[i];
    I.ns = ns;
    I.a0 = b->aoff[i];
    I.na = SW_RED + nst;
    b->soff[i + 1] = b->soff[i] + ns;
    b->aoff[i + 1] = b->aoff[i] + I.na;
    const int64_t ncol = (int64_t)(c->geo.nx / 4) * c->geo.ny;
    I.ncb = (int)((ncol + NTHREADS - 1) / NTHREADS);
    I.kz = std::min(c->geo.nz, 2 * rpt);
    I.c0 = b->coff[i];
    I.nc = SW_RED + I.ncb * ((c->geo.nz + I.kz - 1) / I.kz);
    b->coff[i + 1] = b->coff[i] + I.nc;
  }
  b->na = b->aoff[n];
  b->ns = b->soff[n];
  b->nc = b->coff[n];
  b->tpb = tpb;
  b->rpt = rpt;
  KB_CUDA(b, cudaMemcpyAsync(b->d_tab, b->tab.data(), sizeof(SwInst) * n, cudaMemcpyHostToDevice, b->stream),
          "problem table upload");
  KB_CUDA(b, cudaMemcpyAsync(b->d_off, b->aoff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, b->stream),
          "offset upload");
  KB_CUDA(b, cudaMemcpyAsync(b->d_off + n + 1, b->soff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice,
                             b->stream),
          "offset upload");
  KB_CUDA(b, cudaMemcpyAsync(b->d_off + 2 * (n + 1), b->coff.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice,
                             b->stream),
          "offset upload");
  KB_CUDA(b, cudaStreamSynchronize(b->stream), "offset upload");
  return KX_OK;
}

// Algorithmic bytes of the batched sweep S_j over the problems still
// running: (j + 2) n_i s + 3 ncell_i s each (basis columns, t, the new
// column, 1/eps), the single-problem count summed.
double sweep_bytes_of(const kx_batch* b, int j, const std::vector<char>* active) {
  double sum = 0.0;
  for (size_t i = 0; i < b->ctx.size(); ++i) {
    if (active && !(*active)[i]) continue;
    const kx_ctx* c = b->ctx[i];
    sum += (j + 2.0) * (double)c->n * c->esize + 3.0 * (double)c->geo.ncell * c->esize;
  }
  return sum;
}

// Capture the batched Arnoldi process of a slot (no kernel runs during the
// capture); false if the capture or its instantiation fails.
bool capture_process(kx_batch* b, int slot) {
  const int n = (int)b->ctx.size();
  const int m = b->ctx[0]->m;
  if (sweep_batch_prepare(b->ctx[0]) != KX_OK) return false;
  if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  int64_t cnt = 0;
  const kx_status st = sweep_arnoldi_batch(b->ctx[0], b->stream, b->d_tab, b->d_off, b->d_off + n + 1,
                                           b->d_off + 2 * (n + 1), n, b->na, b->ns, b->nc, slot, m, &cnt, nullptr);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(b->stream, &g);
  bool ok = st == KX_OK && e == cudaSuccess && g != nullptr &&
            cudaGraphInstantiate(&b->graph[slot], g, 0) == cudaSuccess;
  if (g) cudaGraphDestroy(g);
  if (!ok) {
    cudaGetLastError();
    b->graph[slot] = nullptr;
    return false;
  }
  b->graph_m[slot] = m;
  b->graph_count[slot] = cnt;
  return true;
}

kx_status arnoldi_all(kx_batch* b, int slot, const std::vector<char>* active = nullptr) {
  const int n = (int)b->ctx.size();
  if (!b->timing && !b->tuning && !b->graphs_off) {
    if (b->graph[slot] && b->graph_m[slot] != b->ctx[0]->m) {
      cudaGraphExecDestroy(b->graph[slot]);
      b->graph[slot] = nullptr;
    }
    if (!b->graph[slot] && !capture_process(b, slot)) b->graphs_off = true;
    if (b->graph[slot]) {
      KB_CUDA(b, cudaGraphLaunch(b->graph[slot], b->stream), "graph launch");
      b->launches += b->graph_count[slot];
      b->graph_replays += 1;
      return KX_OK;
    }
  }
  const size_t before = b->sweep_events.size();
  const kx_status st = sweep_arnoldi_batch(b->ctx[0], b->stream, b->d_tab, b->d_off, b->d_off + n + 1,
                                           b->d_off + 2 * (n + 1), n, b->na, b->ns, b->nc, slot, b->ctx[0]->m,
                                           &b->launches,
                                           b->timing ? &b->sweep_events : nullptr);
  if (b->timing)
    for (size_t k = before; k < b->sweep_events.size(); ++k)
      b->sweep_bytes.push_back(sweep_bytes_of(b, (int)(k - before) + 1, active));
  if (st != KX_OK) return bfail(b, st, b->ctx[0]->err);
  return KX_OK;
}

// Fold the recorded sweep events into the totals (the stream is synchronised).
void collect_timing(kx_batch* b) {
  for (size_t k = 0; k < b->sweep_events.size(); ++k) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, b->sweep_events[k].first, b->sweep_events[k].second) == cudaSuccess) {
      b->sweep_ms += ms;
      b->sweep_bytes_sum += b->sweep_bytes[k];
      b->sweep_timed += 1;
    }
    cudaEventDestroy(b->sweep_events[k].first);
    cudaEventDestroy(b->sweep_events[k].second);
  }
  cudaGetLastError();
  b->sweep_events.clear();
  b->sweep_bytes.clear();
}

// A fixed pseudo-random start vector (the autotuner's timing input).
__global__ void k_fill_pattern(float* v, int64_t n, uint32_t salt) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)e * 2654435761u ^ salt;
    h ^= h >> 15;
    h *= 2246822519u;
    h ^= h >> 13;
    v[e] = (float)(h & 0xffffffu) * (1.0f / 16777216.0f) - 0.5f;
  }
}

kx_status fresh_slots(kx_batch* b, int slot) {
  for (kx_ctx* c : b->ctx) {
    std::memset(&c->h_state[slot], 0, sizeof(SlotState));
    KB_CUDA(b, cudaMemcpyAsync(c->d_state + slot, c->h_state + slot, sizeof(SlotState), cudaMemcpyHostToDevice,
                               b->stream),
            "state upload");
  }
  KB_CUDA(b, cudaStreamSynchronize(b->stream), "state upload");
  return KX_OK;
}

std::string size_class(const kx_batch* b) {
  std::vector<std::string> dims;
  for (const kx_ctx* c : b->ctx)
    dims.push_back(std::to_string(c->geo.nx) + "x" + std::to_string(c->geo.ny) + "x" + std::to_string(c->geo.nz));
  std::sort(dims.begin(), dims.end());
  std::string k = "m" + std::to_string(b->ctx[0]->m);
  for (auto& d : dims) k += "," + d;
  return k;
}

std::mutex g_tune_mu;
std::map<std::string, std::pair<int, int>> g_tune_cache;

// Time one short Arnoldi process (TUNE_STEPS steps, or krylov_dim if fewer;
// every problem) under each candidate granularity; keep the fastest.
constexpr int TUNE_STEPS = 12;

kx_status autotune(kx_batch* b) {
  const std::string key = size_class(b);
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(key);
    if (it != g_tune_cache.end()) {
      b->from_cache = 1;
      return set_grids(b, it->second.first, it->second.second);
    }
  }
  StreamSwap swap(b);
  // the timed candidates launch directly (their Krylov dimension is shortened)
  struct Tuning {
    kx_batch* b;
    ~Tuning() { b->tuning = false; }
  } tuning{b};
  b->tuning = true;
  for (kx_ctx* c : b->ctx) {
    k_fill_pattern<<<c->nblk, NTHREADS, 0, b->stream>>>((float*)col_ptr(c, 0, 0), c->n, 0x5bd1e995u);
    KB_CUDA(b, cudaGetLastError(), "start vector");
  }
  const int saved_m = b->ctx[0]->m;
  const int steps = std::min(TUNE_STEPS, saved_m);   // never past the slot's m + 1 columns
  static const int TPB[] = {1, 2, 4, 8, 16};
  static const int RPT[] = {1, 2, 4};
  cudaEvent_t e0, e1;
  KB_CUDA(b, cudaEventCreate(&e0), "event");
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return bcuda(b, cudaGetLastError(), "event");
  }
  struct Ev { cudaEvent_t a, b; ~Ev() { cudaEventDestroy(a); cudaEventDestroy(b); } } ev{e0, e1};
  float best = 1e30f;
  int bt = 4, br = 1;
  bool first = true;
  for (int tpb : TPB)
    for (int rpt : RPT) {
      KB_OK(set_grids(b, tpb, rpt));
      for (int rep = 0; rep < (first ? 2 : 1); ++rep) {   // the first candidate runs once untimed (warm-up)
        KB_OK(fresh_slots(b, 0));
        for (kx_ctx* c : b->ctx) KB_TRY(b, c, launch_norm_init(c, 0, 1));
        for (kx_ctx* c : b->ctx) c->m = steps;
        KB_CUDA(b, cudaEventRecord(e0, b->stream), "event");
        const kx_status st = arnoldi_all(b, 0);
        for (kx_ctx* c : b->ctx) c->m = saved_m;
        if (st != KX_OK) return st;
        KB_CUDA(b, cudaEventRecord(e1, b->stream), "event");
        KB_CUDA(b, cudaEventSynchronize(e1), "event");
      }
      first = false;
      float ms = 0.f;
      KB_CUDA(b, cudaEventElapsedTime(&ms, e0, e1), "event");
      b->tune_ms += ms;
      if (ms < best) {
        best = ms;
        bt = tpb;
        br = rpt;
      }
    }
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[key] = {bt, br};
  }
  return set_grids(b, bt, br);
}

kx_status read_slot_states(kx_batch* b, int slot) {
  for (kx_ctx* c : b->ctx)
    KB_CUDA(b, cudaMemcpyAsync(c->h_state + slot, c->d_state + slot, sizeof(SlotState), cudaMemcpyDeviceToHost,
                               b->stream),
            "state read");
  KB_CUDA(b, cudaStreamSynchronize(b->stream), "state read");
  return KX_OK;
}

}  // namespace

extern "C" {

kx_status kx_batch_create(kx_ctx* const* ctxs, int nctx, void* cuda_stream, kx_batch** out) {
  if (!ctxs || !out || nctx < 1) return bfail(nullptr, KX_EINVAL, "kx_batch_create: bad argument");
  *out = nullptr;
  for (int i = 0; i < nctx; ++i) {
    const kx_ctx* c = ctxs[i];
    if (!c) return bfail(nullptr, KX_EINVAL, "kx_batch_create: NULL context");
    for (int k = 0; k < i; ++k)
      if (ctxs[k] == c) return bfail(nullptr, KX_EINVAL, "kx_batch_create: a context appears twice");
    if (c->d.dim != 3 || c->d.precision != KX_FP32 || (c->geo.nx % 4) != 0 || c->d.pml)
      return bfail(nullptr, KX_EINVAL,
                   "kx_batch_create: every problem must be 3D, FP32, lossy layer, with n[0] a multiple of 4 "
                   "(problem " + std::to_string(i) + ")");
    if (c->d.batch < 2 || c->d.rst_samples <= 0)
      return bfail(nullptr, KX_EINVAL, "kx_batch_create: every context needs batch >= 2 and rst_samples > 0");
    if (c->m != ctxs[0]->m) return bfail(nullptr, KX_EINVAL, "kx_batch_create: krylov_dim must agree");
  }
  kx_batch* b = new (std::nothrow) kx_batch();
  if (!b) return bfail(nullptr, KX_ENOMEM, "host allocation failed");
  b->ctx.assign(ctxs, ctxs + nctx);
  struct Guard { kx_batch*& b; ~Guard() { if (b) kx_batch_destroy(b); } } guard{b};
  if (cuda_stream == KX_OWN_STREAM) {
    if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess)
      return bcuda(nullptr, cudaGetLastError(), "stream creation");
    b->own_stream = true;
  } else {
    b->stream = (cudaStream_t)cuda_stream;
  }
  if (cudaMalloc(&b->d_tab, sizeof(SwInst) * nctx) != cudaSuccess ||
      cudaMalloc(&b->d_off, sizeof(int) * 3 * (nctx + 1)) != cudaSuccess ||
      cudaMallocHost(&b->h_pin, sizeof(int) * (nctx * (MAXF + 1) + 1)) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_arn, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    return bfail(nullptr, KX_ENOMEM, "batch workspace allocation failed");
  }
  b->h_pin[nctx * (MAXF + 1)] = 1;
  b->tab.resize(nctx);
  for (int i = 0; i < nctx; ++i) {
    kx_ctx* c = b->ctx[i];
    SwInst& I = b->tab[i];
    std::memset(&I, 0, sizeof(I));
    I.g = c->geo;
    for (int sl = 0; sl < 2; ++sl) {
      I.s[sl] = make_slot<float>(c, sl);
      I.w[sl] = sw_slot_of(c, sl);
    }
    I.ie = (const float*)c->d_inv_eps;
    I.sig2 = (const float*)c->d_sig2;
    I.ld = c->ld;
    I.ldh = c->m + 1;
  }
  const kx_status st = autotune(b);
  if (st != KX_OK) {
    g_batch_err = b->err;
    return st;
  }
  *out = b;
  b = nullptr;   // owned by the caller now
  return KX_OK;
}

kx_status kx_batch_set_timing(kx_batch* b, int on) {
  if (!b) return KX_EINVAL;
  b->timing = on ? 1 : 0;
  if (!on) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    collect_timing(b);
  }
  return KX_OK;
}

kx_status kx_batch_destroy(kx_batch* b) {
  if (!b) return KX_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  collect_timing(b);
  drop_graphs(b);
  if (b->d_tab) cudaFree(b->d_tab);
  if (b->d_off) cudaFree(b->d_off);
  if (b->h_pin) cudaFreeHost(b->h_pin);
  if (b->ev_arn) cudaEventDestroy(b->ev_arn);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
  return KX_OK;
}

kx_status kx_batch_get_info(const kx_batch* b, kx_batch_info* out) {
  if (!b || !out) return KX_EINVAL;
  out->problems = (int)b->ctx.size();
  out->sweep_tiles_per_block = b->tpb;
  out->apply_rounds_per_thread = b->rpt;
  out->sweep_blocks = b->ns;
  out->apply_blocks = b->nc;
  out->from_cache = b->from_cache;
  out->tune_ms = b->tune_ms;
  out->batched_launches = b->launches;
  out->sweep_ms = b->sweep_ms;
  out->sweep_bytes = b->sweep_bytes_sum;
  out->sweep_timed_launches = b->sweep_timed;
  out->graph_replays = b->graph_replays;
  return KX_OK;
}

const char* kx_batch_last_error(const kx_batch* b) { return b ? b->err : g_batch_err.c_str(); }

kx_status response_restart_dim_batch(kx_batch* b, const void* const* d_g, const double* omegas, int nfreq, double T,
                                     double rtol, int max_restarts, const int* planes, double* intensity,
                                     double* resid, int* restarts) {
  if (!b) return KX_EINVAL;
  b->err[0] = 0;
  const int n = (int)b->ctx.size();
  if (!d_g || !omegas || !planes) return bfail(b, KX_EINVAL, "NULL argument");
  if (nfreq < 1 || nfreq > MAXF) return bfail(b, KX_EINVAL, "nfreq must be 1 .. 64");
  if (!(T > 0.0) || !std::isfinite(T)) return bfail(b, KX_EINVAL, "T must be finite and > 0");
  if (!(rtol >= 0.0) || !std::isfinite(rtol)) return bfail(b, KX_EINVAL, "rtol must be finite and >= 0");
  if (max_restarts < 0) return bfail(b, KX_EINVAL, "max_restarts must be >= 0");
  std::vector<int> axis(n), idx(n);
  std::vector<int64_t> P(n);
  for (int i = 0; i < n; ++i) {
    kx_ctx* c = b->ctx[i];
    if (!d_g[i]) return bfail(b, KX_EINVAL, "NULL source of problem " + std::to_string(i));
    if (nfreq > c->d.max_freqs) return bfail(b, KX_EINVAL, "nfreq exceeds max_freqs of problem " + std::to_string(i));
    for (int f = 0; f < nfreq; ++f)
      if (!std::isfinite(omegas[(size_t)i * nfreq + f])) return bfail(b, KX_ENONFINITE, "non-finite frequency");
    axis[i] = planes[2 * i];
    idx[i] = planes[2 * i + 1];
    if (axis[i] < 0 || axis[i] > 2) return bfail(b, KX_EINVAL, "bad plane axis");
    const int na = axis[i] == 0 ? c->geo.nx : (axis[i] == 1 ? c->geo.ny : c->geo.nz);
    if (idx[i] < 0 || idx[i] >= na) return bfail(b, KX_EINVAL, "bad plane index");
    int pa = 0, pb = 0;
    plane_dims(c->geo, axis[i], &pa, &pb);
    P[i] = (int64_t)c->geo.ne * pa * pb;
  }
  StreamSwap swap(b);
  const cudaStream_t S = b->stream;
  // restart 1 of every problem from v_1 = g / ||g|| in slot 0
  for (int i = 0; i < n; ++i) {
    kx_ctx* c = b->ctx[i];
    KB_CUDA(b, cudaMemcpyAsync(col_ptr(c, 0, 0), d_g[i], (size_t)c->n * c->esize, cudaMemcpyDeviceToDevice, S),
            "copy g");
  }
  KB_OK(fresh_slots(b, 0));
  KB_OK(fresh_slots(b, 1));
  for (kx_ctx* c : b->ctx) KB_TRY(b, c, launch_norm_init(c, 0, 1));
  KB_OK(read_slot_states(b, 0));
  std::vector<double> beta(n);
  std::vector<char> active(n, 1);
  for (int i = 0; i < n; ++i) {
    kx_ctx* c = b->ctx[i];
    beta[i] = c->h_state[0].beta;
    if (!std::isfinite(beta[i])) return bfail(b, KX_ENONFINITE, "source of problem " + std::to_string(i) + " is not finite");
    if (beta[i] == 0.0) active[i] = 0;   // y = 0; its slot is done, the batched kernels skip it
    KB_CUDA(b, cudaMemsetAsync(c->d_rst_yp, 0, (size_t)nfreq * P[i] * sizeof(double), S), "zero plane");
    KB_CUDA(b, cudaMemsetAsync(c->d_rst_state, 0, (size_t)nfreq * sizeof(int), S), "zero states");
    KB_CUDA(b, cudaMemcpyAsync(c->d_omegas, omegas + (size_t)i * nfreq, sizeof(double) * nfreq,
                               cudaMemcpyHostToDevice, S),
            "omega upload");
  }
  int* one = b->h_pin + n * (MAXF + 1);
  for (int i = 0; i < n; ++i)
    if (!active[i])
      for (int s2 = 0; s2 < 2; ++s2)
        KB_CUDA(b, cudaMemcpyAsync(&b->ctx[i]->d_state[s2].retired, one, sizeof(int), cudaMemcpyHostToDevice, S),
                "retire");
  KB_OK(arnoldi_all(b, 0, &active));
  KB_OK(read_slot_states(b, 0));
  // sample grid of each problem from ||H_m||_1 of its first restart
  std::vector<int> Nt(n, 0), kmax(n, 0), rcount((size_t)n * nfreq, 0);
  std::vector<double> dstep(n, 0.0);
  const int m = b->ctx[0]->m, ldh = m + 1;
  std::vector<double> Hh((size_t)ldh * m);
  for (int i = 0; i < n; ++i) {
    if (!active[i]) continue;
    kx_ctx* c = b->ctx[i];
    const SlotState& st = c->h_state[0];
    if (st.status)
      return bfail(b, (kx_status)st.status, "problem " + std::to_string(i) + ": Arnoldi process failed");
    KB_CUDA(b, cudaMemcpy(Hh.data(), make_slot<double>(c, 0).H, Hh.size() * sizeof(double), cudaMemcpyDeviceToHost),
            "H read");
    double nu = 0.0;
    for (int col = 0; col < st.m_done; ++col) {
      double sum = 0.0;
      for (int r = 0; r <= std::min(col + 1, st.m_done - 1); ++r) sum += std::fabs(Hh[r + (size_t)col * ldh]);
      nu = std::max(nu, sum);
    }
    if (!std::isfinite(nu)) return bfail(b, KX_ENONFINITE, "non-finite Hessenberg matrix");
    double want = std::max(1.0, std::ceil(T * nu - 1e-9 * T * nu));   // one sample per unit of T ||H_m||_1 (FP32)
    if (want > (double)c->d.rst_samples)
      return bfail(b, KX_EINVAL, "problem " + std::to_string(i) + " needs " + std::to_string((long long)want) +
                                     " time samples; its context holds rst_samples = " +
                                     std::to_string(c->d.rst_samples));
    Nt[i] = (int)want;
    dstep[i] = T / Nt[i];
    kmax[i] = max_restarts > 0 ? max_restarts : (int)std::min(100000.0, 3.0 * T * nu / m + 20.0);
    KB_TRY(b, c, launch_rst_source(c, S, nfreq, beta[i], Nt[i], dstep[i], c->d_rst_b));
  }
  KB_CUDA(b, cudaEventRecord(b->ev_arn, S), "event record");
  bool any = std::any_of(active.begin(), active.end(), [](char a) { return a != 0; });
  bool capped = false;
  for (int k = 1; any; ++k) {
    const int sl = (k - 1) & 1, nx = sl ^ 1;
    // projected work of restart k, per problem on its auxiliary stream
    for (int i = 0; i < n; ++i) {
      if (!active[i]) continue;
      kx_ctx* c = b->ctx[i];
      cudaStream_t X = c->aux_stream;
      int* hs = b->h_pin + i * (MAXF + 1);
      KB_CUDA(b, cudaStreamWaitEvent(X, b->ev_arn, 0), "event wait");
      KB_CUDA(b, cudaMemsetAsync(c->d_small + 64, 0, sizeof(int), X), "status reset");
      KB_TRY(b, c, launch_rst_setup(c, X, sl, dstep[i]));
      KB_TRY(b, c, launch_rst_cascade(c, X, nfreq, c->d_rst_b, Nt[i], dstep[i], rtol * beta[i]));
      KB_TRY(b, c, launch_rst_plane(c, X, sl, nfreq, axis[i], idx[i], P[i]));
      KB_TRY(b, c, launch_rst_coef(c, X, nfreq, c->d_rst_b, Nt[i], dstep[i]));
      KB_CUDA(b, cudaEventRecord(c->ev_proj[sl], X), "event record");
      KB_CUDA(b, cudaMemcpyAsync(hs, c->d_rst_state, sizeof(int) * nfreq, cudaMemcpyDeviceToHost, X), "state read");
      KB_CUDA(b, cudaMemcpyAsync(hs + MAXF, c->d_small + 64, sizeof(int), cudaMemcpyDeviceToHost, X), "status read");
    }
    // restart k + 1's batched Arnoldi process in the other slot, started
    // before restart k's stopping tests are known
    bool next = false;
    for (int i = 0; i < n; ++i) next = next || (active[i] && k < kmax[i]);
    if (next) {
      for (int i = 0; i < n; ++i) {
        if (!active[i]) continue;
        kx_ctx* c = b->ctx[i];
        if (k >= 2) KB_CUDA(b, cudaStreamWaitEvent(S, c->ev_proj[nx], 0), "event wait");
        if (k >= kmax[i]) {
          // capped: its next basis is not needed
          KB_CUDA(b, cudaMemcpyAsync(&c->d_state[nx].retired, one, sizeof(int), cudaMemcpyHostToDevice, S), "retire");
          continue;
        }
        KB_TRY(b, c, launch_rst_nextvec(c, S, sl, nx));
        KB_TRY(b, c, launch_norm_init(c, nx, 1));
      }
      KB_OK(arnoldi_all(b, nx, &active));
      KB_CUDA(b, cudaEventRecord(b->ev_arn, S), "event record");
    }
    // restart k's stopping tests (Fig. alg:rst step 2(c))
    any = false;
    for (int i = 0; i < n; ++i) {
      if (!active[i]) continue;
      kx_ctx* c = b->ctx[i];
      KB_CUDA(b, cudaStreamSynchronize(c->aux_stream), "stream synchronise");
      const int* hs = b->h_pin + i * (MAXF + 1);
      if (hs[MAXF]) {
        cudaStreamSynchronize(S);
        return bfail(b, hs[MAXF] == KX_ETIMEOUT ? KX_ETIMEOUT : KX_ENONFINITE,
                     "problem " + std::to_string(i) +
                         (hs[MAXF] == KX_ETIMEOUT ? ": a bounded wait for a basis copy ran out"
                                                  : ": non-finite Arnoldi process or projected exponential"));
      }
      bool all_stopped = true;
      for (int f = 0; f < nfreq; ++f) {
        if (hs[f] == 3) {
          cudaStreamSynchronize(S);
          return bfail(b, KX_ENONFINITE, "problem " + std::to_string(i) + ": non-finite residual");
        }
        if (hs[f] == 0 || hs[f] == 1) rcount[(size_t)i * nfreq + f] = k;
        all_stopped = all_stopped && hs[f] != 0;
      }
      if (all_stopped || k >= kmax[i]) {
        if (!all_stopped) capped = true;
        active[i] = 0;
        // its basis slots are skipped from now on by the batched kernels
        for (int s2 = 0; s2 < 2; ++s2)
          KB_CUDA(b, cudaMemcpyAsync(&c->d_state[s2].retired, one, sizeof(int), cudaMemcpyHostToDevice, S),
                  "retire");
      } else {
        any = true;
      }
    }
  }
  for (int i = 0; i < n; ++i) {
    kx_ctx* c = b->ctx[i];
    KB_CUDA(b, cudaStreamWaitEvent(S, c->ev_proj[0], 0), "event wait");
    KB_CUDA(b, cudaStreamWaitEvent(S, c->ev_proj[1], 0), "event wait");
  }
  for (int i = 0; i < n; ++i) {
    kx_ctx* c = b->ctx[i];
    KB_TRY(b, c, launch_rst_out(c, S, nfreq, P[i], nullptr, c->d_small + 128, nullptr));
    KB_CUDA(b, cudaMemcpyAsync(c->h_small, c->d_small + 128, sizeof(double) * nfreq, cudaMemcpyDeviceToHost, S),
            "intensity read");
    KB_CUDA(b, cudaMemcpyAsync(c->h_small + 64, c->d_rst_res, sizeof(double) * nfreq, cudaMemcpyDeviceToHost, S),
            "residual read");
  }
  KB_CUDA(b, cudaStreamSynchronize(S), "stream synchronise");
  if (b->timing) collect_timing(b);
  for (int i = 0; i < n; ++i) {
    kx_ctx* c = b->ctx[i];
    for (int f = 0; f < nfreq; ++f) {
      const size_t q = (size_t)i * nfreq + f;
      if (intensity) intensity[q] = beta[i] > 0.0 ? c->h_small[f] : 0.0;
      if (resid) resid[q] = beta[i] > 0.0 ? c->h_small[64 + f] / beta[i] : 0.0;
      if (restarts) restarts[q] = rcount[q];
    }
  }
  if (capped) return bfail(b, KX_ENOCONV, "restart in Krylov dimension: max_restarts reached for some problem");
  return KX_OK;
}

}  // extern "C"
