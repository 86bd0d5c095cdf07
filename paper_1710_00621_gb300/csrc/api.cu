// Error state, device buffers and the SHT entry points of the C ABI
// (synthesis Y, analysis Y^T W and adjoint synthesis Y^T; Sec. 2.1, Sec. 3.2).
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <mutex>
#include <string>
#include <unordered_set>
#include <vector>

#include "common.h"

namespace cmbws {

namespace {
std::mutex g_live_mu;
std::unordered_set<const void*> g_live[2];
}  // namespace

void handle_add(int kind, const void* p) {
  std::lock_guard<std::mutex> lk(g_live_mu);
  g_live[kind].insert(p);
}

bool handle_del(int kind, const void* p) {
  std::lock_guard<std::mutex> lk(g_live_mu);
  return p && g_live[kind].erase(p) == 1;
}

bool handle_live(int kind, const void* p) {
  if (!p) return false;
  std::lock_guard<std::mutex> lk(g_live_mu);
  return g_live[kind].count(p) != 0;
}

static thread_local std::string t_err;

void set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  t_err = buf;
}

void clear_error() { t_err.clear(); }

int DevMem::alloc(size_t n) {
  release();
  if (n == 0) n = 16;
  cudaError_t e = cudaMalloc(&p, n);
  if (e != cudaSuccess) {
    p = nullptr;
    cudaGetLastError();
    set_error("cudaMalloc(%zu) failed: %s", n, cudaGetErrorString(e));
    return CMBWS_ERR_NOMEM;
  }
  bytes = n;
  return CMBWS_OK;
}

int DevMem::ensure(size_t n) {
  if (p && bytes >= n) return CMBWS_OK;
  return alloc(n);
}

int DevMem::upload(const void* src, size_t n) {
  CMBWS_TRY(alloc(n));
  if (n) CMBWS_CUDA(cudaMemcpy(p, src, n, cudaMemcpyHostToDevice));
  return CMBWS_OK;
}

namespace {
struct ProfRec {
  int slot;
  ProfWork work;
  cudaEvent_t a, b;
};
std::mutex g_prof_mu;
std::atomic<bool> g_prof_on{false};
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_pool;

cudaEvent_t pool_get() {
  if (!g_pool.empty()) {
    cudaEvent_t e = g_pool.back();
    g_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}
}  // namespace

bool prof_enabled() { return g_prof_on.load(std::memory_order_relaxed); }

namespace {
std::atomic<int> g_tune_mode{0};
}

int autotune_mode() { return g_tune_mode.load(std::memory_order_relaxed); }

int autotune_pick(const Grid& g, int key, int nvar, int heuristic,
                  const std::function<int(int)>& launch, cudaStream_t s, int* chosen) {
  const int mode = autotune_mode();
  *chosen = mode == 1 ? heuristic : 0;
  if (mode != 2 || nvar < 2) return CMBWS_OK;
  std::lock_guard<std::mutex> lk(g.tune_mu);
  auto it = g.tuned.find(key);
  if (it != g.tuned.end()) {
    *chosen = it->second.variant;
    return CMBWS_OK;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    *chosen = heuristic;
    return CMBWS_OK;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  CMBWS_CUDA(cudaEventCreate(&a));
  if (cudaEventCreate(&b) != cudaSuccess) {
    cudaEventDestroy(a);
    CMBWS_CUDA(cudaGetLastError());
  }
  Grid::Tuned t;
  t.nvar = nvar < 8 ? nvar : 8;
  int st = CMBWS_OK;
  for (int v = 0; v < t.nvar && st == CMBWS_OK; ++v) {
    st = launch(v);  // warm-up
    if (st == CMBWS_OK) cudaEventRecord(a, s);
    for (int r = 0; r < 2 && st == CMBWS_OK; ++r) st = launch(v);
    if (st != CMBWS_OK) break;
    cudaEventRecord(b, s);
    if (cudaEventSynchronize(b) != cudaSuccess) {
      st = CMBWS_ERR_CUDA;
      break;
    }
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    t.ms[v] = 0.5f * ms;
    if (t.ms[v] < t.ms[t.variant]) t.variant = v;
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (st != CMBWS_OK) return st;
  g.tuned[key] = t;
  *chosen = t.variant;
  return CMBWS_OK;
}

ProfScope::ProfScope(int stage, cudaStream_t s_, int arith, ProfWork w)
    : slot(stage + PROF_N * arith), work(w), s(s_) {
  if (!g_prof_on.load(std::memory_order_relaxed)) return;  // no lock on the common path
  std::lock_guard<std::mutex> lk(g_prof_mu);
  if (!g_prof_on) return;
  a = pool_get();
  if (a) cudaEventRecord(a, s);
}

ProfScope::~ProfScope() {
  if (!a) return;
  std::lock_guard<std::mutex> lk(g_prof_mu);
  cudaEvent_t b = pool_get();
  if (!b) {
    g_pool.push_back(a);
    return;
  }
  cudaEventRecord(b, s);
  g_prof.push_back({slot, work, a, b});
}

int ensure_dyn_smem(const void* func, size_t bytes) {
  // fixed table (no host allocation): one slot per (kernel, device)
  struct Slot {
    const void* func;
    int dev;
    size_t bytes;
  };
  static std::mutex mu;
  static Slot lim[512];
  static int nlim = 0;
  int dev = 0;
  CMBWS_CUDA(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(mu);
  for (int i = 0; i < nlim; ++i)
    if (lim[i].func == func && lim[i].dev == dev) {
      if (lim[i].bytes >= bytes) return CMBWS_OK;
      CMBWS_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
      lim[i].bytes = bytes;
      return CMBWS_OK;
    }
  CMBWS_CUDA(cudaFuncSetAttribute(func, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  if (nlim < 512) lim[nlim++] = Slot{func, dev, bytes};
  return CMBWS_OK;
}

static int check_device(const Grid& g) {
  int dev = -1;
  CMBWS_CUDA(cudaGetDevice(&dev));
  if (dev != g.device) {
    set_error("grid was planned on device %d, current device is %d", g.device, dev);
    return CMBWS_ERR_ARG;
  }
  return CMBWS_OK;
}

}  // namespace cmbws

using namespace cmbws;

extern "C" const char* cmbws_last_error(void) { return t_err.c_str(); }

extern "C" const char* cmbws_version(void) { return "cmbws 0.1 (sm_103a)"; }

extern "C" int cmbws_set_autotune(int mode) {
  clear_error();
  if (mode < 0 || mode > 2) {
    set_error("cmbws_set_autotune: mode must be 0 (defaults), 1 (heuristic) or 2 (measured)");
    return CMBWS_ERR_ARG;
  }
  g_tune_mode = mode;
  return CMBWS_OK;
}

extern "C" int cmbws_grid_tuning(cmbws_grid gh, int prec, int nmaps, int* variant, float* ms,
                                 int* nvar) {
  clear_error();
  const Grid* g = as_grid(gh);
  if (!g || !variant || !nvar || nmaps < 1) {
    set_error("cmbws_grid_tuning: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g->tune_mu);
  auto it = g->tuned.find(synth_tune_key(prec, nmaps < 4 ? nmaps : 4));
  if (it == g->tuned.end()) {
    *variant = -1;
    *nvar = 0;
    return CMBWS_OK;
  }
  *variant = it->second.variant;
  *nvar = it->second.nvar;
  if (ms)
    for (int v = 0; v < it->second.nvar; ++v) ms[v] = it->second.ms[v];
  return CMBWS_OK;
}

extern "C" int cmbws_profile_enable(int on) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  g_prof_on = on != 0;
  return CMBWS_OK;
}

extern "C" int cmbws_profile_read(double* ms, int64_t* launches, double* flops, double* elems,
                                  double* map_elems, double* bytes, int reset) {
  clear_error();
  std::lock_guard<std::mutex> lk(g_prof_mu);
  constexpr int NS = PROF_ARITH * PROF_N;
  double t[NS] = {0}, f[NS] = {0}, e[NS] = {0}, me[NS] = {0}, by[NS] = {0};
  int64_t c[NS] = {0};
  for (const ProfRec& r : g_prof) {
    CMBWS_CUDA(cudaEventSynchronize(r.b));
    float dt = 0.f;
    CMBWS_CUDA(cudaEventElapsedTime(&dt, r.a, r.b));
    t[r.slot] += dt;
    f[r.slot] += r.work.flops;
    e[r.slot] += r.work.elems;
    me[r.slot] += r.work.melems;
    by[r.slot] += r.work.bytes;
    c[r.slot] += 1;
  }
  for (int i = 0; i < NS; ++i) {
    if (ms) ms[i] = t[i];
    if (launches) launches[i] = c[i];
    if (flops) flops[i] = f[i];
    if (elems) elems[i] = e[i];
    if (map_elems) map_elems[i] = me[i];
    if (bytes) bytes[i] = by[i];
  }
  if (reset) {
    for (const ProfRec& r : g_prof) {
      g_pool.push_back(r.a);
      g_pool.push_back(r.b);
    }
    g_prof.clear();
  }
  return CMBWS_OK;
}

extern "C" int cmbws_sht_synth(cmbws_grid gh, cmbws_prec prec, const double* alm, double* map,
                               int nmaps, void* stream) {
  clear_error();
  Grid* g = as_grid(gh);
  if (!g || !alm || !map || nmaps < 1 || !valid_prec(prec)) {
    set_error("cmbws_sht_synth: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  CMBWS_TRY(check_device(*g));
  if (!ringfft_smem_ok(*g, prec)) {
    set_error("cmbws_sht_synth: ring length %d too large for this precision", g->max_n);
    return CMBWS_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t es = prec_size(prec);
  const int64_t nlm = nlm_of(g->lmax);
  CMBWS_TRY(g->ws_alm.ensure((size_t)nmaps * nlm * 2 * es));
  CMBWS_TRY(g->ws_F.ensure((size_t)nmaps * g->nring * (g->lmax + 1) * 2 * es));
  CMBWS_TRY(pack_alm(*g, prec, nmaps, alm, g->ws_alm.p, s));
  CMBWS_TRY(legendre_synth(*g, prec, nmaps, g->ws_alm.p, g->ws_F.p, s));
  CMBWS_TRY(ringfft_synth(*g, prec, nmaps, g->ws_F.p, map, s));
  return CMBWS_OK;
}

extern "C" int cmbws_sht_analysis(cmbws_grid gh, cmbws_prec prec, const double* map, double* alm,
                                  int nmaps, int weighted, void* stream) {
  clear_error();
  Grid* g = as_grid(gh);
  if (!g || !alm || !map || nmaps < 1 || !valid_prec(prec)) {
    set_error("cmbws_sht_analysis: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  CMBWS_TRY(check_device(*g));
  if (!ringfft_smem_ok(*g, prec)) {
    set_error("cmbws_sht_analysis: ring length %d too large for this precision", g->max_n);
    return CMBWS_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const size_t es = prec_size(prec);
  const int64_t nlm = nlm_of(g->lmax);
  CMBWS_TRY(g->ws_F.ensure((size_t)nmaps * g->nring * (g->lmax + 1) * 2 * es));
  const size_t pb = legendre_adjoint_part_bytes(*g, prec, nmaps);
  CMBWS_TRY(g->ws_part.ensure(pb));
  CMBWS_TRY(g->ws_out.ensure((size_t)nmaps * nlm * 16));
  CMBWS_TRY(ringfft_analysis(*g, prec, nmaps, map, weighted, g->ws_F.p, g->ws_part.p, s));
  CMBWS_TRY(legendre_adjoint(*g, prec, nmaps, g->ws_F.p, g->ws_part.p, g->ws_part.bytes,
                             g->ws_out.as<double>(), s));
  CMBWS_TRY(unpack_alm(*g, nmaps, g->ws_out.as<double>(), alm, s));
  return CMBWS_OK;
}
