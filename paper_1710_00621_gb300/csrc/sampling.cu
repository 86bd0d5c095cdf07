// Constrained-realization draws on the device (Sec. 2.3): omega_1 (one standard normal per
// band pixel) and omega_2 (one per real harmonic coefficient) make the solution of A x = b a
// sample of p(s | d, S).  A Gibbs sampler repeats the draw and the solve many times, so the
// variates come from a counter-based generator: any variate is a pure function of
// (seed, sample, stream, index), generated where it is needed, with no generator state.
//
//   * Philox4x64-10 (Salmon, Moraes, Dror and Shaw, SC'11): counter (x0..x3), key (k0, k1);
//     a round maps x to (hi(M1 x2) ^ x1 ^ k0, lo(M1 x2), hi(M0 x0) ^ x3 ^ k1, lo(M0 x0)) and
//     the key is advanced by the Weyl constants (W0, W1) between rounds.
//   * Variate j of stream s: key (seed, sample), counter (j / 4, s, 0, 0), word j % 4; the
//     uniform u = ((w >> 12) + 1/2) 2^-52 (exact in FP64, inside (0, 1)); Box-Muller on the
//     pairs (u0, u1), (u2, u3): z = sqrt(-2 ln u_a) (cos 2 pi u_b, sin 2 pi u_b).
//   * omega_2: stream 0 over the stacked coefficient vector; omega_1 of band nu: stream
//     1 + nu over its pixels.
//
// One thread per counter (4 variates); the 10 rounds are 20 64-bit multiplies and the
// Box-Muller step one FP64 log, sqrt and sincospi per pair, so the draw of a full-size
// sample (~60 M variates) is a few milliseconds against a solve of ~0.4 s.
#include "model.h"

#include <cmath>

namespace cmbws {

namespace {

constexpr uint64_t kPhM0 = 0xD2E7470EE14C6C93ull;
constexpr uint64_t kPhM1 = 0xCA5A826395121157ull;
constexpr uint64_t kPhW0 = 0x9E3779B97F4A7C15ull;
constexpr uint64_t kPhW1 = 0xBB67AE8584CAA73Bull;
constexpr int kDrawNT = 256;

__device__ __forceinline__ void philox4x64_10(uint64_t& x0, uint64_t& x1, uint64_t& x2,
                                              uint64_t& x3, uint64_t k0, uint64_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kPhW0;
      k1 += kPhW1;
    }
    const uint64_t h0 = __umul64hi(kPhM0, x0), l0 = kPhM0 * x0;
    const uint64_t h1 = __umul64hi(kPhM1, x2), l1 = kPhM1 * x2;
    x0 = h1 ^ x1 ^ k0;
    x1 = l1;
    x2 = h0 ^ x3 ^ k1;
    x3 = l0;
  }
}

__device__ __forceinline__ double unit_open(uint64_t w) {
  return ((double)(w >> 12) + 0.5) * 0x1p-52;
}

// variates offset .. offset + n - 1 of stream `sid` -> out[0 .. n-1]; kind 0 normal, 1 uniform
__global__ void __launch_bounds__(kDrawNT)
k_draw(uint64_t seed, uint64_t sample, uint64_t sid, int64_t offset, int64_t n, int kind,
       double* __restrict__ out) {
  const int64_t first = offset >> 2;
  const int64_t ncnt = ((offset + n - 1) >> 2) - first + 1;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < ncnt; t += stride) {
    const int64_t i = first + t;
    uint64_t x0 = (uint64_t)i, x1 = sid, x2 = 0, x3 = 0;
    philox4x64_10(x0, x1, x2, x3, seed, sample);
    double v[4] = {unit_open(x0), unit_open(x1), unit_open(x2), unit_open(x3)};
    if (kind == 0) {
#pragma unroll
      for (int p = 0; p < 4; p += 2) {
        const double r = sqrt(-2.0 * log(v[p]));
        double sn, cs;
        sincospi(2.0 * v[p + 1], &sn, &cs);
        v[p] = r * cs;
        v[p + 1] = r * sn;
      }
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int64_t idx = 4 * i + j - offset;
      if (idx >= 0 && idx < n) out[idx] = v[j];
    }
  }
}

__global__ void k_powerlaw(double lnr, const double* __restrict__ beta,
                           const double* __restrict__ mask, int64_t n, double* __restrict__ q) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  q[i] = (mask && mask[i] == 0.0) ? 0.0 : exp(beta[i] * lnr);
}

}  // namespace

static int draw_variates(uint64_t seed, uint64_t sample, uint64_t sid, int64_t offset, int64_t n,
                  int kind, double* out, cudaStream_t s) {
  if (n <= 0) return CMBWS_OK;
  const int64_t ncnt = ((offset + n - 1) >> 2) - (offset >> 2) + 1;
  const int64_t blocks = std::min<int64_t>((ncnt + kDrawNT - 1) / kDrawNT, 152LL * 32);
  k_draw<<<(unsigned)blocks, kDrawNT, 0, s>>>(seed, sample, sid, offset, n, kind, out);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

int Model::cr_draw_rhs(const double* const* d, uint64_t seed, uint64_t sample, double* b,
                       cudaStream_t s) {
  int64_t tot = nvec;
  for (int nu = 0; nu < nobs; ++nu) tot += grids[nu]->npix;
  CMBWS_TRY(cr_w.ensure((size_t)tot * 8));
  double* w2 = cr_w.as<double>();
  std::vector<const double*> w1(nobs);
  int64_t off = nvec;
  {
    ProfScope ps(PROF_HARM, s, 1 + nobs);
    CMBWS_TRY(draw_variates(seed, sample, 0, 0, nvec, 0, w2, s));
    for (int nu = 0; nu < nobs; ++nu) {
      double* p = cr_w.as<double>() + off;
      CMBWS_TRY(draw_variates(seed, sample, 1 + (uint64_t)nu, 0, grids[nu]->npix, 0, p, s));
      w1[nu] = p;
      off += grids[nu]->npix;
    }
  }
  return rhs(d, w1.data(), w2, b, s);
}

}  // namespace cmbws

using namespace cmbws;

extern "C" int cmbws_draw(uint64_t seed, uint64_t sample, uint64_t stream_id, int64_t offset,
                          int64_t n, int kind, double* out, void* stream) {
  clear_error();
  if (offset < 0 || n < 0 || (n > 0 && !out) || (kind != 0 && kind != 1) ||
      offset > INT64_MAX / 2 - n) {
    set_error("cmbws_draw: invalid arguments (offset, n >= 0; kind 0 or 1; out for n > 0)");
    return CMBWS_ERR_ARG;
  }
  return draw_variates(seed, sample, stream_id, offset, n, kind, out, (cudaStream_t)stream);
}

extern "C" int cmbws_cr_sample(cmbws_model mh, const double* const* d, uint64_t seed,
                               uint64_t sample, double* x, const cmbws_cg_opts* opts,
                               cmbws_cg_report* report, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (refuse_sharded(M, "cmbws_cr_sample")) return CMBWS_ERR_ARG;
  if (!M || !d || !x || !opts) {
    set_error("cmbws_cr_sample: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  for (int nu = 0; nu < M->nobs; ++nu)
    if (!d[nu]) {
      set_error("cmbws_cr_sample: missing map for band %d", nu);
      return CMBWS_ERR_ARG;
    }
  const cudaStream_t s = (cudaStream_t)stream;
  CMBWS_TRY(M->cr_b.ensure((size_t)M->nvec * 8));
  CMBWS_TRY(M->cr_draw_rhs(d, seed, sample, M->cr_b.as<double>(), s));
  return cmbws_cg_solve(mh, M->cr_b.as<double>(), x, opts, report, stream);
}

extern "C" int cmbws_cr_rhs(cmbws_model mh, const double* const* d, uint64_t seed,
                            uint64_t sample, double* b, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (refuse_sharded(M, "cmbws_cr_rhs")) return CMBWS_ERR_ARG;
  if (!M || !d || !b) {
    set_error("cmbws_cr_rhs: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  for (int nu = 0; nu < M->nobs; ++nu)
    if (!d[nu]) {
      set_error("cmbws_cr_rhs: missing map for band %d", nu);
      return CMBWS_ERR_ARG;
    }
  return M->cr_draw_rhs(d, seed, sample, b, (cudaStream_t)stream);
}

extern "C" int cmbws_powerlaw_mixing(double nu_ratio, const double* beta, const double* mask,
                                     int64_t n, double* q, void* stream) {
  clear_error();
  if (!(nu_ratio > 0.0) || !std::isfinite(nu_ratio) || n < 0 || (n > 0 && (!beta || !q))) {
    set_error("cmbws_powerlaw_mixing: invalid arguments (nu_ratio > 0, n >= 0)");
    return CMBWS_ERR_ARG;
  }
  if (n == 0) return CMBWS_OK;
  k_powerlaw<<<(unsigned)((n + 255) / 256), 256, 0, (cudaStream_t)stream>>>(std::log(nu_ratio),
                                                                            beta, mask, n, q);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}
