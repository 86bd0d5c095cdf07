// Adjoint synthesis / analysis without any device allocation.
//
// cmbws_sht_analysis keeps its workspace (ring spectra, the per-CTA partial
// sums of the adjoint Legendre kernel, the reduced coefficients) in buffers
// the grid allocates on first use.  Some callers cannot allocate device
// memory at that point: host runtimes that hand the library a fixed memory
// budget and forbid cudaMalloc after start-up, or real-time loops that must
// not block on the allocator (cudaMalloc can synchronise the device).
// cmbws_sht_analysis_noalloc serves them from one file-scope __device__ array
// of kScratchBytes (32 MiB), which every GPU that loads the library holds
// until the process exits.
//
// The host cannot use the array's name as a device address (in host code it
// names a host-side stand-in), so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on the device.  Make that first call before any stream
// capture begins.  The address belongs to the device's CUDA context at that
// time; after cudaDeviceReset the cached address is stale, so the library must
// not be used across a reset.  All calls share the one array and find the
// previous call's contents in it; the kernels overwrite every byte they read,
// so nothing needs clearing, but calls whose kernels overlap on the GPU (other
// streams, other host threads) race and must be serialised by the caller.
#include <mutex>

#include "common.h"

namespace cmbws {
namespace {

constexpr size_t kScratchBytes = size_t(32) << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

int scratch_address(void** out) {
  int dev = -1;
  CMBWS_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("cmbws_sht_analysis_noalloc: device index %d out of range", dev);
    return CMBWS_ERR_ARG;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess || !p) {
      set_error("cmbws_sht_analysis_noalloc: cudaGetSymbolAddress failed: %s",
                cudaGetErrorString(e));
      return CMBWS_ERR_CUDA;
    }
    g_addr[dev] = p;
  }
  *out = g_addr[dev];
  return CMBWS_OK;
}

size_t round256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace
}  // namespace cmbws

using namespace cmbws;

extern "C" int cmbws_sht_analysis_noalloc(cmbws_grid gh, cmbws_prec prec, const double* map,
                                          double* alm, int nmaps, int weighted, void* stream) {
  clear_error();
  Grid* g = as_grid(gh);
  if (!g || !alm || !map || nmaps < 1) {
    set_error("cmbws_sht_analysis_noalloc: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  if (prec != CMBWS_FP64 && prec != CMBWS_FP32) {
    set_error("cmbws_sht_analysis_noalloc: precision %d is not supported here (CMBWS_FP64 or "
              "CMBWS_FP32 only: the double-float and tensor-core modes build tables on first use)",
              (int)prec);
    return CMBWS_ERR_ARG;
  }
  int dev = -1;
  CMBWS_CUDA(cudaGetDevice(&dev));
  if (dev != g->device) {
    set_error("cmbws_sht_analysis_noalloc: grid was planned on device %d, current device is %d",
              g->device, dev);
    return CMBWS_ERR_ARG;
  }
  if (!ringfft_smem_ok(*g, prec)) {
    set_error("cmbws_sht_analysis_noalloc: ring length %d too large for this precision", g->max_n);
    return CMBWS_ERR_ARG;
  }
  const size_t es = prec_size(prec);
  const int64_t nlm = nlm_of(g->lmax);
  const size_t fb = round256((size_t)nmaps * g->nring * (g->lmax + 1) * 2 * es);
  const size_t pb = round256(legendre_adjoint_part_bytes(*g, prec, nmaps));
  const size_t ob = round256((size_t)nmaps * nlm * 16);
  if (fb + pb + ob > kScratchBytes) {
    set_error("cmbws_sht_analysis_noalloc: needs %zu bytes of scratch for nmaps=%d, lmax=%d, "
              "nring=%d; the static scratch holds %zu bytes (use cmbws_sht_analysis)",
              fb + pb + ob, nmaps, g->lmax, g->nring, kScratchBytes);
    return CMBWS_ERR_ARG;
  }
  void* base = nullptr;
  CMBWS_TRY(scratch_address(&base));
  unsigned char* p = static_cast<unsigned char*>(base);
  void* F = p;
  void* part = p + fb;
  double* out = reinterpret_cast<double*>(p + fb + pb);
  cudaStream_t s = (cudaStream_t)stream;
  CMBWS_TRY(ringfft_analysis(*g, prec, nmaps, map, weighted, F, part, s));
  CMBWS_TRY(legendre_adjoint(*g, prec, nmaps, F, part, pb, out, s));
  CMBWS_TRY(unpack_alm(*g, nmaps, out, alm, s));
  return CMBWS_OK;
}
