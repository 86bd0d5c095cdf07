// Preconditioned conjugate gradients for A x = b (Sec. 2.3) with M_PI (Sec. 3.3).
//
// Vectors are FP64 on the device.  Dot products are deterministic: a fixed
// grid writes per-block partial sums, one block adds them in a fixed order.
// The host reads one or two scalars per iteration (alpha and beta are
// computed on the host in FP64).
//
// FP64 models: plain PCG, then one FP64-accurate apply certifies ||b - A x|| / ||b||.
// FP32 models: iterative refinement.  Each pass solves A d = r by PCG with
// the FP32 transform chain (FP64 vectors and scalars) until the inner
// residual falls by inner_tol, then x += d and r = b - A x with an
// FP64-accurate chain (native FP64 or double-float, opts.cert_prec); the loop
// ends when that residual certifies tol.
#include <atomic>
#include <chrono>
#include <cmath>
#include <string>
#include <thread>
#include <vector>

#include "model.h"

namespace cmbws {

namespace {

constexpr int kRedBlocks = 1024;
constexpr int kRedThreads = 256;

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += sh[i];
  return t;
}

// partial[b] = sum_{i in block-stride range} a[i] * b[i]
__global__ void k_dot_partial(const double* __restrict__ a, const double* __restrict__ b, int64_t n,
                              double* __restrict__ partial) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    s += a[i] * b[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// x += alpha p; r -= alpha q; partial sums of r.r, with alpha = rz / pq read from the device
// (the PCG scalars stay on the device between the host's one read per iteration); alpha = 0
// when p.q is not a positive finite number or r.z is not finite, and the host then reports the
// breakdown with x, r unchanged.
__global__ void k_update_xr_dev(double* __restrict__ x, double* __restrict__ r,
                                const double* __restrict__ p, const double* __restrict__ q,
                                const double* __restrict__ rz, const double* __restrict__ pq,
                                int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  const double a = *rz, b = *pq;
  const double alpha = (b > 0.0 && isfinite(b) && isfinite(a)) ? a / b : 0.0;
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    x[i] += alpha * p[i];
    const double ri = r[i] - alpha * q[i];
    r[i] = ri;
    s += ri * ri;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// p = z + (rz_new / rz_old) p, the ratio read from the device
__global__ void k_xpby_dev(const double* __restrict__ z, double* __restrict__ p,
                           const double* __restrict__ rz_new, const double* __restrict__ rz_old,
                           int64_t n) {
  const double beta = *rz_new / *rz_old;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    p[i] = z[i] + beta * p[i];
}

// r = b - y; partial sums of r.r
__global__ void k_resid(const double* __restrict__ b, const double* __restrict__ y,
                        double* __restrict__ r, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double ri = b[i] - y[i];
    r[i] = ri;
    s += ri * ri;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

// y += x
__global__ void k_axpy1(const double* __restrict__ x, double* __restrict__ y, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x)
    y[i] += x[i];
}

// partial sums of |x + d - t|^2 (distance of the current iterate to a reference solution)
__global__ void k_err_partial(const double* __restrict__ x, const double* __restrict__ d,
                              const double* __restrict__ t, int64_t n, double* __restrict__ partial) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double e = x[i] + d[i] - t[i];
    s += e * e;
  }
  s = block_sum(s, sh);
  if (threadIdx.x == 0) partial[blockIdx.x] = s;
}

__global__ void k_finish(const double* __restrict__ partial, int nb, double* __restrict__ out) {
  __shared__ double sh[32];
  double s = 0.0;
  for (int i = threadIdx.x; i < nb; i += blockDim.x) s += partial[i];
  s = block_sum(s, sh);
  if (threadIdx.x == 0) *out = s;
}

struct Clock {
  std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
  double s() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

// The all-reduce of a band-sharded solve: called on each operator output so that every shard
// holds the full A p, M r and A x (cmbws_cg_solve_sharded).
struct Comm {
  cmbws_allreduce_fn fn;
  void* ctx;
};

// Device scalar slots after the reduction partials (red + kRedBlocks): 0 the last finished
// sum, 1 p.q, 2 r.r, 3 + (it & 1) r.z of iteration it.
constexpr int kScal = 8;
constexpr int kSlotPQ = 1, kSlotRR = 2, kSlotRZ = 3;

struct Solver {
  Model& M;
  cudaStream_t s;
  int64_t n;
  double* red;     // [kRedBlocks + kScal]
  double* hscal;   // pinned host copy of the kScal scalar slots
  const Comm* comm = nullptr;

  double* slot(int i) { return red + kRedBlocks + i; }
  // sum of a . b into a device slot (no host synchronisation)
  int dot_dev(const double* a, const double* b, double* out) {
    ProfScope ps_(PROF_CG, s);
    k_dot_partial<<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, red);
    CMBWS_LAUNCH_CHECK();
    k_finish<<<1, kRedThreads, 0, s>>>(red, kRedBlocks, out);
    CMBWS_LAUNCH_CHECK();
    return CMBWS_OK;
  }
  // the scalar slots, read back once (one host synchronisation)
  int read_slots() {
    CMBWS_CUDA(cudaMemcpyAsync(hscal, red + kRedBlocks, kScal * 8, cudaMemcpyDeviceToHost, s));
    CMBWS_CUDA(cudaStreamSynchronize(s));
    return CMBWS_OK;
  }

  // sum a device vector of n doubles over the shards (no-op for unsharded solves)
  int reduce(double* v) {
    if (!comm) return CMBWS_OK;
    const int rc = comm->fn(v, n, (void*)s, comm->ctx);
    if (rc != 0) {
      set_error("sharded solve: the all-reduce callback returned %d", rc);
      return CMBWS_ERR_COMM;
    }
    return CMBWS_OK;
  }

  int finish(double* out) {
    {
      ProfScope ps_(PROF_CG, s);
      k_finish<<<1, kRedThreads, 0, s>>>(red, kRedBlocks, red + kRedBlocks);
      CMBWS_LAUNCH_CHECK();
    }
    CMBWS_CUDA(cudaMemcpyAsync(hscal, red + kRedBlocks, 8, cudaMemcpyDeviceToHost, s));
    CMBWS_CUDA(cudaStreamSynchronize(s));
    *out = *hscal;
    return CMBWS_OK;
  }
  int dot(const double* a, const double* b, double* out) {
    {
      ProfScope ps_(PROF_CG, s);
      k_dot_partial<<<kRedBlocks, kRedThreads, 0, s>>>(a, b, n, red);
      CMBWS_LAUNCH_CHECK();
    }
    return finish(out);
  }
  int cert = CMBWS_FP64;  // arithmetic of the true-residual applies
  // r = b - A x (FP64-accurate chain), returns ||r||^2
  int true_residual(const double* b, const double* x, double* r, double* tmp, double* rr) {
    CMBWS_TRY(M.apply_A(x, tmp, cert, s));
    CMBWS_TRY(reduce(tmp));
    {
      ProfScope ps_(PROF_CG, s);
      k_resid<<<kRedBlocks, kRedThreads, 0, s>>>(b, tmp, r, n, red);
      CMBWS_LAUNCH_CHECK();
    }
    return finish(rr);
  }
};

}  // namespace

// z = M r: identity (use_M = 0), M_PI (1), M_add = M_PI + the model's mask preconditioners (2)
// or the block-diagonal M_diag (3)
static int precondition(Model& M, int use_M, int prec, const double* r, double* z, int64_t n,
                        cudaStream_t s) {
  if (!use_M) {
    CMBWS_CUDA(cudaMemcpyAsync(z, r, n * 8, cudaMemcpyDeviceToDevice, s));
    return CMBWS_OK;
  }
  if (use_M == 3) return M.apply_diag(r, z, s);
  CMBWS_TRY(M.apply_precond(r, z, M.prec_M >= 0 ? M.prec_M : prec, s));
  if (use_M == 2)
    for (MaskMG* mg : M.masks) CMBWS_TRY(mask_mg_apply(*mg, M, r, z, s));
  return CMBWS_OK;
}

void Model::drop_graphs() {
  for (OpGraph& g : graphs)
    if (g.exec) cudaGraphExecDestroy(g.exec);
  graphs.clear();
}

// One operator apply of PCG through a CUDA graph when the model asks for it: the launches of
// an apply (tens to hundreds of kernels for small problems) are replayed with one graph
// launch.  The first apply for a (operator, precision, in, out) runs eagerly (it performs any
// lazy allocation or table build), the second is captured and instantiated, later ones
// replay.  Capture is skipped while per-stage profiling is on (its events cannot be timed
// inside a graph) and falls back to the eager apply whenever capture or instantiation fails.
template <typename F>
static int run_op(Model& M, int op, int prec, const double* in, double* out, cudaStream_t s,
                  F&& eager) {
  if (!M.use_graphs || prof_enabled()) return eager();
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) {
    cudaGetLastError();
    return eager();
  }
  Model::OpGraph* g = nullptr;
  for (Model::OpGraph& e : M.graphs)
    if (e.op == op && e.prec == prec && e.in == in && e.out == out) g = &e;
  if (!g) {
    M.graphs.emplace_back();
    g = &M.graphs.back();
    g->op = op;
    g->prec = prec;
    g->in = in;
    g->out = out;
  }
  if (g->failed) return eager();
  if (g->exec) {
    CMBWS_CUDA(cudaGraphLaunch(g->exec, s));
    M.n_sht += g->nsht;
    return CMBWS_OK;
  }
  if (g->calls++ == 0) return eager();
  const long long n0 = M.n_sht;
  if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    g->failed = true;
    return eager();
  }
  const int st = eager();
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(s, &graph);
  const long long dn = M.n_sht - n0;
  M.n_sht = n0;  // the captured launches have not run
  cudaGraphExec_t ex = nullptr;
  if (st == CMBWS_OK && ce == cudaSuccess && graph) ce = cudaGraphInstantiate(&ex, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (st != CMBWS_OK || ce != cudaSuccess || !ex) {
    cudaGetLastError();
    clear_error();
    g->failed = true;
    return eager();
  }
  g->exec = ex;
  g->nsht = dn;
  CMBWS_CUDA(cudaGraphLaunch(ex, s));
  M.n_sht += dn;
  return CMBWS_OK;
}

enum { OP_APPLY_A = 0, OP_PRECOND = 1 };

// Where a PCG run starts: from d = 0 (a fresh pass), or from an exported state (the correction
// d, residual r and direction p already in the model's workspaces, with the iteration count
// and the scalars r.z and r.r of the next iteration).
struct PcgStart {
  bool resume = false;
  int it0 = 0;
  double rz = 0.0, rr = 0.0;
};

// Record of one iteration: ||r|| / ||b|| and, when tracked, ||x + d - x_true|| / ||x_true||.
struct PcgRecord {
  const double* x = nullptr;  // outer iterate (the current solution is x + d)
  double bnorm = 1.0, tnorm = 1.0;
};

static int record_iteration(Solver& S, const PcgRecord& rec, const double* d, double rr) {
  Model& M = S.M;
  M.hist_res.push_back(std::sqrt(rr) / rec.bnorm);
  if (!M.track_err) return CMBWS_OK;
  {
    ProfScope ps_(PROF_CG, S.s);
    k_err_partial<<<kRedBlocks, kRedThreads, 0, S.s>>>(rec.x, d, M.cg_xtrue.as<double>(), S.n, S.red);
    CMBWS_LAUNCH_CHECK();
  }
  double ee;
  CMBWS_TRY(S.finish(&ee));
  M.hist_err.push_back(std::sqrt(ee) / rec.tnorm);
  return CMBWS_OK;
}

// PCG on A d = r0 (d starts at zero unless resuming), operator precision `prec`; stops when
// ||r|| <= stop_abs or after maxit iterations in all (counting a resumed run's earlier ones).
// r0 is overwritten with the final residual; *rz_out is r.z of the next iteration.
static int pcg_core(Solver& S, int prec, int use_M, double* d, double* r, double stop_abs, int maxit,
                    int* iters, double* rr_out, const Clock& clk, double timeout,
                    const PcgStart& start, const PcgRecord& rec, double* rz_out) {
  Model& M = S.M;
  double* z = M.cg_z.as<double>();
  double* p = M.cg_p.as<double>();
  double* q = M.cg_q.as<double>();
  const int64_t n = S.n;
  auto precond = [&]() {
    if (!use_M) return precondition(M, use_M, prec, r, z, n, S.s);
    if (S.comm) {  // sharded: the partial M r, summed over the shards (no graphs)
      CMBWS_TRY(precondition(M, use_M, prec, r, z, n, S.s));
      return S.reduce(z);
    }
    return run_op(M, OP_PRECOND + 16 * use_M, M.prec_M >= 0 ? M.prec_M : prec, r, z, S.s,
                  [&]() { return precondition(M, use_M, prec, r, z, n, S.s); });
  };
  double rr, rz;
  if (start.resume) {
    rr = start.rr;
    rz = start.rz;
    *rr_out = rr;
    *rz_out = rz;
    *iters = start.it0;
    if (std::sqrt(rr) <= stop_abs) return CMBWS_OK;
  } else {
    CMBWS_CUDA(cudaMemsetAsync(d, 0, n * 8, S.s));
    CMBWS_TRY(S.dot(r, r, &rr));
    *rr_out = rr;
    *iters = 0;
    *rz_out = 0.0;
    if (std::sqrt(rr) <= stop_abs) return CMBWS_OK;
    CMBWS_TRY(precond());
    CMBWS_CUDA(cudaMemcpyAsync(p, z, n * 8, cudaMemcpyDeviceToDevice, S.s));
    CMBWS_TRY(S.dot(r, z, &rz));
    *rz_out = rz;
  }
  // the PCG scalars stay on the device: r.z of iteration it in slot kSlotRZ + (it & 1), p.q
  // and r.r in their slots; the host reads them once per iteration for the stopping test
  const int it0 = start.resume ? start.it0 : 0;
  S.hscal[kSlotRZ + (it0 & 1)] = rz;
  CMBWS_CUDA(cudaMemcpyAsync(S.slot(kSlotRZ + (it0 & 1)), &S.hscal[kSlotRZ + (it0 & 1)], 8,
                             cudaMemcpyHostToDevice, S.s));
  for (int it = it0; it < maxit; ++it) {
    if (S.comm) {  // sharded: the partial A p, summed over the shards (no graphs)
      CMBWS_TRY(M.apply_A(p, q, prec, S.s));
      CMBWS_TRY(S.reduce(q));
    } else {
      CMBWS_TRY(run_op(M, OP_APPLY_A, prec, p, q, S.s, [&]() { return M.apply_A(p, q, prec, S.s); }));
    }
    double* rz_cur = S.slot(kSlotRZ + (it & 1));
    double* rz_nxt = S.slot(kSlotRZ + ((it + 1) & 1));
    CMBWS_TRY(S.dot_dev(p, q, S.slot(kSlotPQ)));
    {
      ProfScope ps_(PROF_CG, S.s);
      k_update_xr_dev<<<kRedBlocks, kRedThreads, 0, S.s>>>(d, r, p, q, rz_cur, S.slot(kSlotPQ), n,
                                                           S.red);
      CMBWS_LAUNCH_CHECK();
      k_finish<<<1, kRedThreads, 0, S.s>>>(S.red, kRedBlocks, S.slot(kSlotRR));
      CMBWS_LAUNCH_CHECK();
    }
    CMBWS_TRY(S.read_slots());
    const double pq = S.hscal[kSlotPQ];
    rz = S.hscal[kSlotRZ + (it & 1)];
    *rz_out = rz;
    if (!(pq > 0.0) || !std::isfinite(pq) || !std::isfinite(rz)) {
      // a bounded device-side wait that ran out leaves NaN in the operator's output
      bool timed_out = false;
      if (tc_status_take(&timed_out) == CMBWS_OK && timed_out) {
        set_error("CG: a bounded device-side wait ran out in the operator apply (iteration %d)", it);
        return CMBWS_ERR_TIMEOUT;
      }
      set_error("CG breakdown: p.Ap = %g, r.z = %g at iteration %d", pq, rz, it);
      return CMBWS_ERR_BREAKDOWN;
    }
    rr = S.hscal[kSlotRR];
    *iters = it + 1;
    *rr_out = rr;
    if (!std::isfinite(rr)) {
      set_error("CG breakdown: non-finite residual at iteration %d", it);
      return CMBWS_ERR_BREAKDOWN;
    }
    CMBWS_TRY(record_iteration(S, rec, d, rr));
    if (std::sqrt(rr) <= stop_abs) return CMBWS_OK;
    if (timeout > 0 && clk.s() > timeout) {
      set_error("CG: wall-clock budget of %g s exhausted", timeout);
      return CMBWS_ERR_TIMEOUT;
    }
    CMBWS_TRY(precond());
    CMBWS_TRY(S.dot_dev(r, z, rz_nxt));
    {
      ProfScope ps_(PROF_CG, S.s);
      k_xpby_dev<<<kRedBlocks, kRedThreads, 0, S.s>>>(z, p, rz_nxt, rz_cur, n);
      CMBWS_LAUNCH_CHECK();
    }
  }
  // the state of a run stopped at its cap carries the last r.z
  CMBWS_TRY(S.read_slots());
  *rz_out = S.hscal[kSlotRZ + (maxit & 1)];
  return CMBWS_ERR_NOT_CONVERGED;
}

// One solve.  resume = nullptr: a fresh solve from the initial guess in x.  Otherwise (models
// without FP32 transforms) the run continues the exported PCG state that the caller placed in
// cg_d, cg_r and cg_p, with x holding the same initial guess as the interrupted solve.
static int cg_solve_impl(Model& M, const double* b, double* x, const cmbws_cg_opts& o,
                         cmbws_cg_report& rep, cudaStream_t s, const PcgStart* resume = nullptr,
                         const Comm* comm = nullptr) {
  const Clock clk;
  const int64_t n = M.nvec;
  CMBWS_TRY(M.cg_r.ensure(n * 8));
  CMBWS_TRY(M.cg_z.ensure(n * 8));
  CMBWS_TRY(M.cg_p.ensure(n * 8));
  CMBWS_TRY(M.cg_q.ensure(n * 8));
  CMBWS_TRY(M.cg_d.ensure(n * 8));
  CMBWS_TRY(M.cg_x.ensure(n * 8));
  CMBWS_TRY(M.cg_red.ensure((kRedBlocks + kScal) * 8));
  if (!M.cg_host) CMBWS_CUDA(cudaMallocHost(&M.cg_host, kScal * 8));
  Solver S{M, s, n, M.cg_red.as<double>(), M.cg_host};
  S.cert = o.cert_prec == CMBWS_FP32X2 ? CMBWS_FP32X2 : CMBWS_FP64;
  S.comm = comm;
  const long long sht0 = M.n_sht;
  M.hist_res.clear();
  M.hist_err.clear();
  if (!resume) M.ck_valid = false;

  double bb;
  CMBWS_TRY(S.dot(b, b, &bb));
  const double bnorm = std::sqrt(bb);
  double* r = M.cg_r.as<double>();
  double* tmp = M.cg_x.as<double>();
  double* d = M.cg_d.as<double>();
  if (bnorm == 0.0) {
    CMBWS_CUDA(cudaMemsetAsync(x, 0, n * 8, s));
    rep.rel_res = 0.0;
    return CMBWS_OK;
  }
  PcgRecord rec;
  rec.x = x;
  rec.bnorm = bnorm;
  if (M.track_err) {
    double tt;
    CMBWS_TRY(S.dot(M.cg_xtrue.as<double>(), M.cg_xtrue.as<double>(), &tt));
    rec.tnorm = tt > 0.0 ? std::sqrt(tt) : 1.0;
  }
  double rr;
  if (resume) {
    rr = resume->rr;
  } else {
    double xx;
    CMBWS_TRY(S.dot(x, x, &xx));
    if (xx == 0.0) {
      // x0 = 0: r = b without an apply of A
      CMBWS_CUDA(cudaMemcpyAsync(r, b, n * 8, cudaMemcpyDeviceToDevice, s));
      rr = bb;
    } else {
      CMBWS_TRY(S.true_residual(b, x, r, tmp, &rr));
    }
  }
  int status = CMBWS_ERR_NOT_CONVERGED;
  int total = resume ? resume->it0 : 0, outer = 0;
  const double target = o.tol * bnorm;
  PcgStart start;
  if (resume) start = *resume;
  while (true) {
    if (!start.resume && std::sqrt(rr) <= target) {
      status = CMBWS_OK;
      break;
    }
    if (total >= o.maxiter) {
      set_error("CG: %d iterations without reaching tol (rel. residual %g)", total,
                std::sqrt(rr) / bnorm);
      status = CMBWS_ERR_NOT_CONVERGED;
      break;
    }
    if (o.timeout_s > 0 && clk.s() > o.timeout_s) {
      set_error("CG: wall-clock budget of %g s exhausted", o.timeout_s);
      status = CMBWS_ERR_TIMEOUT;
      break;
    }
    if (M.prec != CMBWS_FP64 && outer >= o.max_outer) {
      set_error("CG: %d refinement passes without reaching tol", outer);
      status = CMBWS_ERR_NOT_CONVERGED;
      break;
    }
    // inner solve A d = r; FP64 models aim directly at the target (plus a small
    // margin for the gap between recursive and true residuals)
    const double stop = !is_f32(M.prec) ? 0.5 * target
                                             : std::max(o.inner_tol * std::sqrt(rr), 0.5 * target);
    int it = 0;
    double rr_in, rz = 0.0;
    // a resumed run counts its earlier iterations against the cap
    const int cap = start.resume ? o.maxiter : o.maxiter - total;
    const int st = pcg_core(S, M.prec, o.precond, d, r, stop, cap, &it, &rr_in, clk, o.timeout_s,
                            start, rec, &rz);
    total = (start.resume ? 0 : total) + it;
    start = PcgStart();
    ++outer;
    if (st != CMBWS_OK && st != CMBWS_ERR_NOT_CONVERGED) {
      status = st;
      break;
    }
    if (st == CMBWS_ERR_NOT_CONVERGED && M.ck_on && !is_f32(M.prec)) {
      // the state of the next iteration, before the certification overwrites r
      CMBWS_TRY(M.cg_ck.ensure(3 * n * 8));
      double* ck = M.cg_ck.as<double>();
      CMBWS_CUDA(cudaMemcpyAsync(ck, d, n * 8, cudaMemcpyDeviceToDevice, s));
      CMBWS_CUDA(cudaMemcpyAsync(ck + n, r, n * 8, cudaMemcpyDeviceToDevice, s));
      CMBWS_CUDA(cudaMemcpyAsync(ck + 2 * n, M.cg_p.p, n * 8, cudaMemcpyDeviceToDevice, s));
      M.ck_iters = total;
      M.ck_rz = rz;
      M.ck_rr = rr_in;
      M.ck_valid = true;
    }
    {
      ProfScope ps_(PROF_CG, s);
      k_axpy1<<<kRedBlocks, kRedThreads, 0, s>>>(d, x, n);
      CMBWS_LAUNCH_CHECK();
    }
    CMBWS_TRY(S.true_residual(b, x, r, tmp, &rr));
    if (st == CMBWS_ERR_NOT_CONVERGED && std::sqrt(rr) > target) {
      set_error("CG: iteration cap %d reached (rel. residual %g)", o.maxiter, std::sqrt(rr) / bnorm);
      status = CMBWS_ERR_NOT_CONVERGED;
      break;
    }
  }
  rep.iters = total;
  rep.outer = outer;
  rep.rel_res = std::sqrt(rr) / bnorm;
  rep.n_sht = (int)(M.n_sht - sht0);
  return status;
}

}  // namespace cmbws

using namespace cmbws;

extern "C" int cmbws_cg_solve(cmbws_model mh, const double* b, double* x, const cmbws_cg_opts* opts,
                              cmbws_cg_report* report, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (refuse_sharded(M, "cmbws_cg_solve")) return CMBWS_ERR_ARG;
  if (!M || !b || !x || !opts || b == x || !(opts->tol > 0.0) || opts->maxiter < 1 ||
      opts->precond < 0 || opts->precond > 3) {
    set_error("cmbws_cg_solve: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  cmbws_cg_opts o = *opts;
  if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0)) o.inner_tol = 1e-3;
  if (o.max_outer < 1) o.max_outer = 20;
  cmbws_cg_report rep{};
  const auto t0 = std::chrono::steady_clock::now();
  int st = cg_solve_impl(*M, b, x, o, rep, (cudaStream_t)stream);
  rep.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  rep.status = st;
  if (report) *report = rep;
  return st;
}

extern "C" int cmbws_model_set_graphs(cmbws_model mh, int on) {
  clear_error();
  Model* M = as_model(mh);
  if (!M) {
    set_error("cmbws_model_set_graphs: invalid model");
    return CMBWS_ERR_ARG;
  }
  if (!on) M->drop_graphs();
  M->use_graphs = on != 0;
  return CMBWS_OK;
}

extern "C" int cmbws_cg_solve_batched(const cmbws_model* models, int nprob, const double* const* b,
                                      double* const* x, const cmbws_cg_opts* opts,
                                      cmbws_cg_report* reports, int nworkers, void* stream) {
  clear_error();
  if (!models || nprob < 1 || !b || !x || !opts || !(opts->tol > 0.0) || opts->maxiter < 1 ||
      opts->precond < 0 || opts->precond > 3) {
    set_error("cmbws_cg_solve_batched: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  for (int i = 0; i < nprob; ++i) {
    if (!as_model(models[i]) || !b[i] || !x[i] || b[i] == x[i] ||
        refuse_sharded(as_model(models[i]), "cmbws_cg_solve_batched")) {
      set_error("cmbws_cg_solve_batched: invalid arguments for problem %d", i);
      return CMBWS_ERR_ARG;
    }
    for (int j = 0; j < i; ++j)
      if (models[j] == models[i]) {
        set_error("cmbws_cg_solve_batched: problems %d and %d share a model (workspace)", j, i);
        return CMBWS_ERR_ARG;
      }
  }
  cmbws_cg_opts o = *opts;
  if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0)) o.inner_tol = 1e-3;
  if (o.max_outer < 1) o.max_outer = 20;
  int dev = 0;
  CMBWS_CUDA(cudaGetDevice(&dev));
  // work queued on the caller's stream (the inputs) completes before the solves start
  CMBWS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  const int nw = std::max(1, std::min(nworkers > 0 ? nworkers : 8, nprob));
  std::vector<cudaStream_t> ws(nw, nullptr);
  for (int w = 0; w < nw; ++w)
    if (cudaStreamCreateWithFlags(&ws[w], cudaStreamNonBlocking) != cudaSuccess) {
      for (int v = 0; v < w; ++v) cudaStreamDestroy(ws[v]);
      set_error("cmbws_cg_solve_batched: stream creation failed");
      return CMBWS_ERR_CUDA;
    }
  std::vector<cmbws_cg_report> rep(nprob);
  std::vector<std::string> msg(nprob);
  std::atomic<int> next(0);
  auto worker = [&](int w) {
    cudaSetDevice(dev);
    for (int i = next.fetch_add(1); i < nprob; i = next.fetch_add(1)) {
      Model* M = reinterpret_cast<Model*>(models[i]);
      cmbws_cg_report r{};
      const auto t0 = std::chrono::steady_clock::now();
      clear_error();
      const int st = cg_solve_impl(*M, b[i], x[i], o, r, ws[w]);
      r.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
      r.status = st;
      if (st != CMBWS_OK) msg[i] = cmbws_last_error();
      rep[i] = r;
    }
  };
  std::vector<std::thread> th;
  for (int w = 1; w < nw; ++w) th.emplace_back(worker, w);
  worker(0);
  for (auto& t : th) t.join();
  for (int w = 0; w < nw; ++w) cudaStreamDestroy(ws[w]);
  int status = CMBWS_OK;
  for (int i = 0; i < nprob; ++i) {
    if (reports) reports[i] = rep[i];
    if (status == CMBWS_OK && rep[i].status != CMBWS_OK) {
      status = rep[i].status;
      set_error("cmbws_cg_solve_batched: problem %d: %s", i, msg[i].c_str());
    }
  }
  return status;
}

extern "C" int cmbws_cg_history(cmbws_model mh, double* rel_res, double* rel_err, int cap, int* n) {
  clear_error();
  Model* M = as_model(mh);
  if (!M || !n || cap < 0) {
    set_error("cmbws_cg_history: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  const int len = (int)M->hist_res.size();
  *n = len;
  for (int i = 0; i < len && i < cap; ++i) {
    if (rel_res) rel_res[i] = M->hist_res[i];
    if (rel_err) rel_err[i] = i < (int)M->hist_err.size() ? M->hist_err[i] : -1.0;
  }
  return CMBWS_OK;
}

extern "C" int cmbws_cg_track_error(cmbws_model mh, const double* x_true, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (!M) {
    set_error("cmbws_cg_track_error: invalid model");
    return CMBWS_ERR_ARG;
  }
  if (!x_true) {
    M->track_err = false;
    return CMBWS_OK;
  }
  CMBWS_TRY(M->cg_xtrue.ensure(M->nvec * 8));
  CMBWS_CUDA(cudaMemcpyAsync(M->cg_xtrue.p, x_true, M->nvec * 8, cudaMemcpyDeviceToDevice,
                             (cudaStream_t)stream));
  CMBWS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  M->track_err = true;
  return CMBWS_OK;
}

extern "C" int cmbws_cg_checkpointing(cmbws_model mh, int on) {
  clear_error();
  Model* M = as_model(mh);
  if (!M) {
    set_error("cmbws_cg_checkpointing: invalid model");
    return CMBWS_ERR_ARG;
  }
  if (on && is_f32(M->prec)) {
    set_error("cmbws_cg_checkpointing: models with FP32 transforms restart from x (refinement)");
    return CMBWS_ERR_ARG;
  }
  M->ck_on = on != 0;
  if (!on) M->ck_valid = false;
  return CMBWS_OK;
}

extern "C" int cmbws_cg_state_export(cmbws_model mh, double* d, double* r, double* p,
                                     double* scalars, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (!M || !d || !r || !p || !scalars) {
    set_error("cmbws_cg_state_export: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  if (!M->ck_valid) {
    set_error("cmbws_cg_state_export: no checkpoint (checkpointing off, or the last solve did "
              "not stop at its iteration cap)");
    return CMBWS_ERR_ARG;
  }
  const int64_t n = M->nvec;
  cudaStream_t s = (cudaStream_t)stream;
  const double* ck = M->cg_ck.as<double>();
  CMBWS_CUDA(cudaMemcpyAsync(d, ck, n * 8, cudaMemcpyDeviceToDevice, s));
  CMBWS_CUDA(cudaMemcpyAsync(r, ck + n, n * 8, cudaMemcpyDeviceToDevice, s));
  CMBWS_CUDA(cudaMemcpyAsync(p, ck + 2 * n, n * 8, cudaMemcpyDeviceToDevice, s));
  scalars[0] = M->ck_iters;
  scalars[1] = M->ck_rz;
  scalars[2] = M->ck_rr;
  return CMBWS_OK;
}

extern "C" int cmbws_cg_resume(cmbws_model mh, const double* b, double* x, const double* d,
                               const double* r, const double* p, const double* scalars,
                               const cmbws_cg_opts* opts, cmbws_cg_report* report, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (refuse_sharded(M, "cmbws_cg_resume")) return CMBWS_ERR_ARG;
  if (!M || !b || !x || !d || !r || !p || !scalars || !opts || b == x || !(opts->tol > 0.0) ||
      opts->maxiter < 1 || opts->precond < 0 || opts->precond > 3) {
    set_error("cmbws_cg_resume: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  if (is_f32(M->prec)) {
    set_error("cmbws_cg_resume: models with FP32 transforms restart from x (refinement)");
    return CMBWS_ERR_ARG;
  }
  const int it0 = (int)scalars[0];
  if (it0 < 0 || (double)it0 != scalars[0] || !std::isfinite(scalars[1]) || !std::isfinite(scalars[2])) {
    set_error("cmbws_cg_resume: invalid state scalars");
    return CMBWS_ERR_ARG;
  }
  cmbws_cg_opts o = *opts;
  if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0)) o.inner_tol = 1e-3;
  if (o.max_outer < 1) o.max_outer = 20;
  const int64_t n = M->nvec;
  cudaStream_t s = (cudaStream_t)stream;
  CMBWS_TRY(M->cg_d.ensure(n * 8));
  CMBWS_TRY(M->cg_r.ensure(n * 8));
  CMBWS_TRY(M->cg_p.ensure(n * 8));
  CMBWS_CUDA(cudaMemcpyAsync(M->cg_d.p, d, n * 8, cudaMemcpyDeviceToDevice, s));
  CMBWS_CUDA(cudaMemcpyAsync(M->cg_r.p, r, n * 8, cudaMemcpyDeviceToDevice, s));
  CMBWS_CUDA(cudaMemcpyAsync(M->cg_p.p, p, n * 8, cudaMemcpyDeviceToDevice, s));
  PcgStart st;
  st.resume = true;
  st.it0 = it0;
  st.rz = scalars[1];
  st.rr = scalars[2];
  cmbws_cg_report rep{};
  const auto t0 = std::chrono::steady_clock::now();
  const int code = cg_solve_impl(*M, b, x, o, rep, s, &st);
  rep.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  rep.status = code;
  if (report) *report = rep;
  return code;
}

extern "C" int cmbws_cg_solve_sharded(cmbws_model mh, const double* b, double* x,
                                      const cmbws_cg_opts* opts, cmbws_allreduce_fn allreduce,
                                      void* ctx, cmbws_cg_report* report, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (!M || !b || !x || !opts || !allreduce || b == x || !(opts->tol > 0.0) ||
      opts->maxiter < 1 || opts->precond < 0 || opts->precond > 1) {
    set_error("cmbws_cg_solve_sharded: invalid arguments (precond must be 0 or 1)");
    return CMBWS_ERR_ARG;
  }
  cmbws_cg_opts o = *opts;
  if (!(o.inner_tol > 0.0 && o.inner_tol < 1.0)) o.inner_tol = 1e-3;
  if (o.max_outer < 1) o.max_outer = 20;
  const Comm comm{allreduce, ctx};
  cmbws_cg_report rep{};
  const auto t0 = std::chrono::steady_clock::now();
  const int st = cg_solve_impl(*M, b, x, o, rep, (cudaStream_t)stream, nullptr, &comm);
  rep.ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  rep.status = st;
  if (report) *report = rep;
  return st;
}

extern "C" int cmbws_model_set_precond_prec(cmbws_model mh, int prec) {
  clear_error();
  Model* M = as_model(mh);
  if (!M || (prec != -1 && !valid_prec(prec))) {
    set_error("cmbws_model_set_precond_prec: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  M->prec_M = prec;
  M->drop_graphs();
  return CMBWS_OK;
}
