// Internal declarations shared by the translation units of libcmbws.
//
// Data layout in device memory
// ----------------------------
// * Internal harmonic layout ("lm"): for band-limit L, complex pairs
//   (cos part, sin part) of coefficient (l, m), m-major, l contiguous:
//   lm(m, l) = m (L+1) - m (m-1) / 2 + (l - m), nlm = (L+1)(L+2)/2.
//   The synthesis Legendre kernel consumes coefficients multiplied by the
//   recurrence normalisation c_lm (setup.cu); the adjoint returns final values.
// * Ring spectra F[map][ring][m] (complex, m = 0..L): output of the synthesis
//   Legendre stage / input of the adjoint Legendre stage; the ring FFT stage
//   reads and writes them.
// * Ring pairs: pair p joins ring p (north) and ring nring-1-p (south); an
//   equator ring (odd nring) is a pair with no south ring.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <functional>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/cmbws.h"

namespace cmbws {

void set_error(const char* fmt, ...);
void clear_error();

// Registry of live handles (api.cu): every grid and model the library hands out is recorded
// until it is destroyed, so calls with a destroyed, foreign or corrupted handle fail with
// CMBWS_ERR_ARG instead of dereferencing it.
enum { HANDLE_GRID = 0, HANDLE_MODEL = 1 };
void handle_add(int kind, const void* p);
bool handle_del(int kind, const void* p);  // false if p was not live
bool handle_live(int kind, const void* p);

#define CMBWS_CUDA(expr)                                                                     \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) {                                                                 \
      ::cmbws::set_error("%s failed: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__,   \
                         __LINE__);                                                          \
      return CMBWS_ERR_CUDA;                                                                 \
    }                                                                                        \
  } while (0)

#define CMBWS_LAUNCH_CHECK()                                                                 \
  do {                                                                                       \
    cudaError_t e_ = cudaGetLastError();                                                     \
    if (e_ != cudaSuccess) {                                                                 \
      ::cmbws::set_error("kernel launch failed: %s (%s:%d)", cudaGetErrorString(e_),         \
                         __FILE__, __LINE__);                                                \
      return CMBWS_ERR_CUDA;                                                                 \
    }                                                                                        \
  } while (0)

#define CMBWS_TRY(expr)            \
  do {                             \
    int s_ = (expr);               \
    if (s_ != CMBWS_OK) return s_; \
  } while (0)

// Owning device allocation.
struct DevMem {
  void* p = nullptr;
  size_t bytes = 0;
  DevMem() = default;
  DevMem(const DevMem&) = delete;
  DevMem& operator=(const DevMem&) = delete;
  DevMem(DevMem&& o) noexcept : p(o.p), bytes(o.bytes) {
    o.p = nullptr;
    o.bytes = 0;
  }
  DevMem& operator=(DevMem&& o) noexcept {
    if (this != &o) {
      release();
      p = o.p;
      bytes = o.bytes;
      o.p = nullptr;
      o.bytes = 0;
    }
    return *this;
  }
  ~DevMem() { release(); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  int alloc(size_t n);                  // exact size, contents undefined
  int ensure(size_t n);                 // grow if needed (contents lost on growth)
  int upload(const void* src, size_t n);
  template <typename T> T* as() const { return static_cast<T*>(p); }
};

// FP32 synthesis near the poles: the rescaled recurrence mu_l = A_l x mu_{l-1} - mu_{l-2}
// has an almost double characteristic root there (x -> 1, A_l alternating around 2 rho and
// 2 / rho), so FP32 rounding grows like l^2 eps.  Warps holding a ring pair with
// theta < kPolarTheta run the difference form e_l = mu_l - R_l mu_{l-1}, R_l = c_{l-1} / c_l:
//   e_l = ((B_l - A_l y) mu_{l-1} + S_l e_{l-1},  mu_l = R_l mu_{l-1} + e_l,
// B_l = A_l - R_l - 1 / R_{l-1}, S_l = 1 / R_{l-1}, whose increments stay small there.
constexpr double kPolarTheta = 0.2;
constexpr float kPolarY = 0.019933422f;  // 1 - cos(kPolarTheta): polar iff y < kPolarY
constexpr int kChunk = 8;    // l-chunk of the checkpointed FP32 adjoint (even)
constexpr int kChunkDf = 4;  // l-chunk of the checkpointed double-float adjoint (even)

inline __host__ __device__ int64_t lm_off(int L, int m) {
  return (int64_t)m * (L + 1) - (int64_t)m * (m - 1) / 2;
}

// Thread -> (m, l) of a kernel over the triangle 0 <= m <= l <= L: grid row y holds the rows
// m = y and m = L - y one after the other (L + 2 values of l together), so that no thread is
// launched for the empty part of the triangle; false for the padding of the last CTA of a row.
// Launch with tri_grid(L, threads per CTA).
__device__ __forceinline__ bool tri_lm(int L, int& m, int& l) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int y = blockIdx.y;
  const int n0 = L - y + 1;  // length of row y
  if (t < n0) {
    m = y;
    l = y + t;
    return true;
  }
  const int m2 = L - y, t2 = t - n0;  // row L - y has y + 1 values of l
  if (m2 == y || t2 > y) return false;
  m = m2;
  l = m2 + t2;
  return true;
}
inline dim3 tri_grid(int L, int nt) { return dim3((unsigned)((L + 2 + nt - 1) / nt), (unsigned)(L / 2 + 1)); }
inline __host__ __device__ int64_t nlm_of(int L) { return (int64_t)(L + 1) * (L + 2) / 2; }
// offset of the m block in the packed CMBWS_ALM layout
inline __host__ __device__ int64_t packed_off(int L, int m) {
  return m == 0 ? 0 : (int64_t)(L + 1) + (int64_t)(m - 1) * (2 * L + 2 - m);
}

// Per ring length: how the ring DFT is done.
struct FftPlan {
  int n;          // ring length
  int n2;         // power-of-two transform size (n itself, or the Bluestein size)
  int bluestein;  // 1 if n is not a power of two
  int pad;
  int64_t chirp;  // offset (complex entries) of b_t = exp(i pi t^2 / n), t < n
  int64_t filt;   // offset of the Bluestein filter spectrum (n2 entries, includes 1/n2,
                  // bit-reversed order)
  int64_t phase;  // offset of exp(i pi k / n), k < n (ring offset phi0 = pi / n)
};

constexpr int kTileMinPT = 16;  // ring pairs per tile of the FP32 checkpointed adjoint

struct Grid {
  int device = 0;
  int kind = 0, n = 0, lmax = 0, nring = 0, npair = 0;
  int64_t npix = 0;
  std::vector<double> theta, weight, phi0;
  std::vector<int> nphi;
  std::vector<int64_t> offset;

  // per ring pair (device)
  DevMem y64, y32;        // 1 - cos(theta) of the north ring [npair] (see setup.cu)
  DevMem pair_ring;       // int2 {north, south or -1} [npair]
  DevMem pair_plan;       // int plan index [npair]
  DevMem pair_phase;      // int: 1 if phi0 = pi / nphi, 0 if phi0 = 0 [npair]
  DevMem ring_off;        // int64 first pixel of each ring [nring + 1]
  DevMem ring_w64, ring_w32;  // per-pixel weight of each ring [nring]

  // Legendre recurrence tables (device), index lm(m, l)
  DevMem A64, A32;        // A_lm of the rescaled recurrence mu_l = A_l x mu_{l-1} - mu_{l-2}
  DevMem A2f;             // A_lm as a double-float pair (float2 hi, lo) for the FP32X2 kernels
  DevMem BRS32;           // {B, R, S}_lm (FP32) of the difference form used near the poles
  DevMem c64;             // lambda_lm = c_lm mu_lm
  DevMem ls;              // int [L+1][npair] first l (same parity as m) that is injected
  DevMem st64, st32;      // {mu_ls, mu_ls+1} [L+1][npair]
  DevMem ck32;            // FP32 {mu_l0, mu_l0+1} at every chunk start l0 = m + kChunk c
  DevMem ck_base;         // int64 [L+1]: offset of m's block [pair][chunk] in ck32
  DevMem ls_tmin;         // int [L+1][ceil(npair / kTileMinPT)]: smallest ls of each tile of pairs
  // warp tasks of the checkpointed adjoints: int2 {m, first chunk} per 32 consecutive
  // chunks of one m, m ascending (FP32 chunking; the double-float list is built with ck64)
  DevMem wt32;
  int nwt32 = 0;
  mutable DevMem wtdf;
  mutable int nwtdf = 0;
  mutable DevMem ck64;    // double-float {mu_l0, mu_l0+1} (float4) every kChunkDf; built on first use
  mutable DevMem ck64_base;  // int64 [L+1]: offset of m's block [pair][chunk] in ck64
  mutable DevMem y2f;     // y as a double-float pair (float2), built with ck64
  mutable std::mutex ck64_mu;
  std::vector<double> fmm_h;  // sqrt((2m+1)/(2m)) (host, for rebuilding seeds)

  // autotuner decisions for launches on this grid (legendre.cu), by kernel / precision / maps
  struct Tuned {
    int variant = 0, nvar = 0;
    float ms[8] = {0};
  };
  mutable std::map<int, Tuned> tuned;
  mutable std::mutex tune_mu;

  // ring FFT tables (device)
  std::vector<FftPlan> plans;
  DevMem plans_d;
  DevMem fft64, fft32;    // complex tables: chirps, filters, phases, twiddles
  DevMem fftdf;           // the same as double-float pairs (float4 per entry)
  int64_t tw_off = 0;     // offset of exp(-2 pi i k / nmax2), k < nmax2 / 2
  int nmax2 = 1;          // largest power-of-two transform size
  int max_n = 1;

  // workspace for cmbws_sht_* calls
  DevMem ws_alm, ws_F, ws_part, ws_out;
};

// the grid behind a handle, or nullptr if the handle is not a live grid
inline Grid* as_grid(const void* h) {
  return handle_live(HANDLE_GRID, h) ? const_cast<Grid*>(static_cast<const Grid*>(h)) : nullptr;
}

// ---- launchers (legendre.cu) ----
// alm: [nmaps][nlm] complex coefficients multiplied by c_lm; F: [nmaps][nring][L+1]
int legendre_synth(const Grid& g, int prec, int nmaps, const void* alm, void* F, cudaStream_t s);
// ring spectra -> out[nmaps][nlm] complex FP64 (final coefficients).  FP64 reads F (with
// per-CTA partial sums in part); the other precisions read the eo layout, which the forward
// ring FFT wrote into part.
int legendre_adjoint(const Grid& g, int prec, int nmaps, const void* F, void* part, size_t part_bytes,
                     double* out, cudaStream_t s);
size_t legendre_adjoint_part_bytes(const Grid& g, int prec, int nmaps);

// ---- launchers (ringfft.cu) ----
// Layout of the adjoint Legendre input ("eo") that the forward ring FFTs write for the
// checkpointed adjoints (every precision but FP64): maps in chunks of eo_maps(prec) (the
// adjoint's maps per launch); chunk c starts at scalar c * eo_maps * (L+1) * npair * 4 and,
// for its NMc maps, holds eo[(m * npair + p) * 4 NMc + q]: q < 2 NMc the even-l parts
// (north + south ring spectra, re / im per map), q >= 2 NMc the odd-l parts (north - south).
// Scalars are float (FP32 modes) or double-float pairs (FP32X2).
inline int eo_maps(int prec) { return prec == CMBWS_FP32X2 ? 3 : 4; }
// F (ring spectra) -> pixel maps map[nmaps][npix] (FP64 out)
int ringfft_synth(const Grid& g, int prec, int nmaps, const void* F, double* map, cudaStream_t s);
// map[nmaps][npix] (FP64 in) -> ring spectra: F (FP64) or the adjoint input eo (other
// precisions); weighted: multiply by quadrature weights
int ringfft_analysis(const Grid& g, int prec, int nmaps, const double* map, int weighted, void* F,
                     void* eo, cudaStream_t s);
// F -> pixels -> * pix[map] -> ring spectra, written to F in place (FP64) or to eo (other
// precisions).  pix: [nmaps] device pointers (prec type) of npix.
int ringfft_fused(const Grid& g, int prec, int nmaps, void* F, const void* const* pix, void* eo,
                  cudaStream_t s);
int ringfft_smem_ok(const Grid& g, int prec);

// warp-task list {m, first chunk} for chunks of `chunk` values of l (adjoint scheduling)
std::vector<int2> adjoint_warp_tasks(int L, int chunk);

// ---- grid setup (setup.cu) ----
int grid_build_tables(Grid& g);
// build the double-float chunk checkpoints of the FP32X2 adjoint if not yet built
int grid_ensure_ck64(const Grid& g);

// ---- pack / unpack (setup.cu) ----
// packed CMBWS_ALM FP64 [nmaps][(L+1)^2] -> internal lm complex (prec), multiplied by c_lm
int pack_alm(const Grid& g, int prec, int nmaps, const double* packed, void* alm, cudaStream_t s);
// internal lm complex FP64 [nmaps][nlm] -> packed FP64
int unpack_alm(const Grid& g, int nmaps, const double* lmc, double* packed, cudaStream_t s);

// FP32 transforms use float buffers; FP64 and FP32X2 use the FP64 layouts.
// FP32 buffers and CUDA-core FP32 stages (the TF32 modes differ in the Legendre synthesis only)
inline bool is_tc(int prec) {
  return prec == CMBWS_TF32 || prec == CMBWS_3XTF32 || prec == CMBWS_BF16 || prec == CMBWS_BF16X3;
}
inline bool is_f32(int prec) { return prec == CMBWS_FP32 || is_tc(prec); }
inline size_t prec_size(int prec) { return is_f32(prec) ? 4 : 8; }
inline bool valid_prec(int prec) {
  return prec == CMBWS_FP64 || prec == CMBWS_FP32 || prec == CMBWS_FP32X2 || is_tc(prec);
}

// ---- double-float Legendre stage (legendre_df.cu) ----
int legendre_synth_df(const Grid& g, int nmaps, const void* alm, void* F, cudaStream_t s);
// ---- tensor-core Legendre synthesis (legendre_tc.cu), prec TF32 / 3XTF32 / BF16 / BF16X3 ----
int legendre_synth_tc(const Grid& g, int prec, int nmaps, const void* alm, void* F, cudaStream_t s);
// adjoint synthesis on the tensor cores from the FP32 adjoint input (eo layout), prec BF16 / BF16X3
int legendre_adjoint_tc(const Grid& g, int prec, int nmaps, const float* eo, double* out,
                        cudaStream_t s);
// reads and clears the device-side status of the tensor-core kernels of the current device
// (synchronous): *timed_out is true if a bounded mbarrier wait ran out since the last read
int tc_status_take(bool* timed_out);
// double-float adjoint from chunk checkpoints: eo (double-float adjoint input of nm <= 3
// maps) -> out (FP64 coefficients)
int legendre_adj_df_ck(const Grid& g, int nm, const void* eo, double* out, cudaStream_t s);

// Raise a kernel's dynamic shared-memory limit to at least `bytes` on the current device.
// The limit only ever grows, so concurrent launches with different sizes (several host
// threads, cmbws_cg_solve_batched) never see it lowered under them.
int ensure_dyn_smem(const void* func, size_t bytes);
bool prof_enabled();  // per-stage CUDA-event profiling switched on (cmbws_profile_enable)

// Autotuner (api.cu): mode 0 = every launch uses its kernel's default tile, 1 = a heuristic by
// problem shape, 2 = the fastest tile measured with CUDA events on the first launch for a
// (grid, kernel, precision, maps) key.  autotune_pick returns the variant to launch; in mode 2
// it times launch(v) for every v (each launch writes the same output) unless the stream is
// being captured, and records the result in g.tuned[key].
int autotune_mode();
inline int synth_tune_key(int prec, int nmaps) { return 1000 + 10 * prec + nmaps; }
int autotune_pick(const Grid& g, int key, int nvar, int heuristic,
                  const std::function<int(int)>& launch, cudaStream_t s, int* chosen);

// ---- kernel timing (api.cu): CUDA events around launches while enabled ----
// Stages; a record's slot is stage + PROF_N * arith, arith 0 = FP32, 1 = FP64,
// 2 = double-float (FP32X2), 3 = TF32 tensor cores, 4 = split TF32, 5 = BF16 tensor cores,
// 6 = split BF16 (PROF_ARITH kinds).
// Each launch records its algorithmic work (ProfWork): Legendre stages their flops over the
// full (l, m) triangle (4 per (l, m, ring pair) for the recurrence plus 4 per map), the
// elements (l, m, ring pair) and elements x maps; ring FFTs the bytes they must move (ring
// spectra and pixel factors or maps, read and written once).  0 for stages without one.
enum {
  PROF_LEG_SYNTH = 0,
  PROF_LEG_ADJ = 1,
  PROF_LEG_RED = 2,
  PROF_FFT = 3,
  PROF_HARM = 4,
  PROF_CG = 5,
  PROF_N = 6,
  PROF_ARITH = 7
};
struct ProfWork {
  double flops = 0, elems = 0, melems = 0, bytes = 0;
};
// the work of one Legendre launch over every (l, m, ring pair) of grid g with nm maps
inline ProfWork leg_work(const Grid& g, int nm) {
  ProfWork w;
  w.elems = (double)g.npair * (double)nlm_of(g.lmax);
  w.melems = w.elems * nm;
  w.flops = 4.0 * (w.elems + w.melems);
  return w;
}
inline ProfWork byte_work(double bytes) {
  ProfWork w;
  w.bytes = bytes;
  return w;
}
struct ProfScope {
  int slot;
  ProfWork work;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(int stage, cudaStream_t s_, int arith = 1, ProfWork w = ProfWork());
  ~ProfScope();
};

// cp.async staging (global -> shared, asynchronous; 4/8-byte copies through L1,
// 16-byte copies bypassing it)
__device__ __forceinline__ void cp_async4(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N));
}

}  // namespace cmbws
