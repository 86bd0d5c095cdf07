// Grid planning: ring geometry (Sec. 2.1-2.2 grids), Legendre recurrence
// tables with per-(m, ring) start values, ring-FFT tables, and the
// pack/unpack kernels between the boundary layout and the internal layout.
//
// Legendre recurrence (orthonormal lambda_lm, no Condon-Shortley phase):
//   lambda_mm = sqrt(1/4pi) prod_{j<=m} sqrt((2j+1)/(2j)) sin(theta)
//   lambda_{m+1,m} = sqrt(2m+3) cos(theta) lambda_mm
//   lambda_l = a_l x lambda_{l-1} - (a_l / a_{l-1}) lambda_{l-2},  a_l = sqrt((4l^2-1)/(l^2-m^2))
// The kernels run the rescaled form lambda_l = c_l mu_l with c_m = c_{m+1} = 1 and
// c_l = (a_l / a_{l-1}) c_{l-2}, for which
//   mu_l = A_l x mu_{l-1} - mu_{l-2},  A_l = a_l c_{l-1} / c_l,
// two operations per step (c stays within [0.17, 1.13] up to l = 4000).
// The kernels carry y = 1 - cos(theta) = 2 sin^2(theta/2) instead of x = cos(theta) and
// form A_l x = A_l - A_l y with one FMA: x rounded near the poles would shift theta by
// eps / sin(theta), a coherent phase error of l eps / sin(theta) in lambda_lm, whereas y
// keeps full relative precision there (still two operations per step).
// Near the poles lambda_mm underflows any floating-point range while
// lambda_lm at larger l is of order one, so the start of the recurrence is
// found once per grid in FP64 with an explicit exponent (values carried as
// v * 2^(-600 k)): for every (m, ring pair) the first l (same parity as m)
// at which |mu_l| or |mu_{l+1}| exceeds 1e-30 with k = 0, and the two values
// there.  Every skipped term is below 1e-30 in magnitude.
// The same FP64 pass stores, for the FP32 adjoint, the two recurrence values at the
// start of every chunk of kChunk = 8 values of l ([m][pair][chunk], FP32; about
// npair (L+1)^2 / 16 x 8 bytes: 9.7 GB at Nside 1024, L = 3071), so that the adjoint can
// restart the recurrence of any pair at any chunk without a serial walk along l.
#include <climits>
#include <cmath>
#include <complex>
#include <cstring>
#include <new>

#include "common.h"

namespace cmbws {

namespace {

constexpr double kStartThreshold = 1e-30;
constexpr double kShiftUp = 0x1p600;     // 2^600
constexpr double kShiftDown = 0x1p-600;  // 2^-600
constexpr double kGrow = 0x1p500;

// Gauss-Legendre nodes (descending cos theta) and weights by Newton iteration on P_n.
void gauss_legendre_nodes(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  const int half = (n + 1) / 2;
  for (int i = 0; i < half; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p1 = z; p0 = 1.0; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) {
        // one more evaluation of the derivative at the converged node
        p0 = 1.0; p1 = z;
        for (int k = 2; k <= n; ++k) {
          double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
          p0 = p1;
          p1 = p2;
        }
        if (n == 1) { p1 = z; p0 = 1.0; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    // at a root of P_n, P_n'(z) = n P_{n-1}(z) / (1 - z^2) exactly
    double q0 = 1.0, q1 = z;
    for (int k = 2; k <= n; ++k) {
      double q2 = ((2.0 * k - 1.0) * z * q1 - (k - 1.0) * q0) / k;
      q0 = q1;
      q1 = q2;
    }
    if (n == 1) q0 = 1.0;
    const double omz2 = (1.0 - z) * (1.0 + z);
    x[i] = z;
    x[n - 1 - i] = -z;
    w[i] = w[n - 1 - i] = 2.0 * omz2 / ((double)n * n * q0 * q0);
    (void)dp;
  }
  if (n % 2 == 1) x[n / 2] = 0.0;
}

void host_fft(std::vector<std::complex<double>>& a, int sign) {
  const int n = (int)a.size();
  for (int i = 1, j = 0; i < n; ++i) {
    int bit = n >> 1;
    for (; j & bit; bit >>= 1) j ^= bit;
    j ^= bit;
    if (i < j) std::swap(a[i], a[j]);
  }
  for (int len = 2; len <= n; len <<= 1) {
    for (int i = 0; i < n; i += len) {
      for (int k = 0; k < len / 2; ++k) {
        double ang = sign * 2.0 * M_PI * k / len;
        std::complex<double> w(std::cos(ang), std::sin(ang));
        std::complex<double> u = a[i + k], v = a[i + k + len / 2] * w;
        a[i + k] = u + v;
        a[i + k + len / 2] = u - v;
      }
    }
  }
}

bool is_pow2(int n) { return n > 0 && (n & (n - 1)) == 0; }
int next_pow2(int n) {
  int p = 1;
  while (p < n) p <<= 1;
  return p;
}

__global__ void k_seeds(const double* __restrict__ sinth, const double* __restrict__ fmm, int L,
                        int npair, double* __restrict__ sv, int* __restrict__ sk) {
  int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p >= npair) return;
  const double s = sinth[p];
  double v = 0.28209479177387814347;  // sqrt(1 / (4 pi))
  int k = 0;
  sv[p] = v;
  sk[p] = 0;
  for (int m = 1; m <= L; ++m) {
    v *= fmm[m] * s;
    if (v != 0.0 && fabs(v) < kShiftDown) {
      v *= kShiftUp;
      ++k;
    }
    sv[(int64_t)m * npair + p] = v;
    sk[(int64_t)m * npair + p] = k;
  }
}

__global__ void k_start(const double* __restrict__ y, const double* __restrict__ A, int L, int npair,
                        const double* __restrict__ sv, const int* __restrict__ sk,
                        int* __restrict__ ls, double2* __restrict__ st64, float2* __restrict__ st32,
                        const int64_t* __restrict__ ck_base, float2* __restrict__ ck,
                        const int64_t* __restrict__ ck64_base, float4* __restrict__ ck64) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (p >= npair) return;
  const int64_t idx = (int64_t)m * npair + p;
  const double yy = y[p];
  double v0 = sv[idx];
  int k = sk[idx];
  double v1 = sqrt(2.0 * m + 3.0) * (1.0 - yy) * v0;
  const double* Am = A + lm_off(L, m) - m;  // Am[l] = A_lm
  int l = m;
  int found = L + 1;
  double o0 = 0.0, o1 = 0.0;
  const int nck = (L - m + kChunk) / kChunk;
  const int nckd = (L - m + kChunkDf) / kChunkDf;
  float2* ckp = ck ? ck + ck_base[m] + (int64_t)p * nck : nullptr;
  float4* ckd = ck64 ? ck64 + ck64_base[m] + (int64_t)p * nckd : nullptr;
  while (l <= L) {
    if (found > L && k == 0 && (fabs(v0) > kStartThreshold || fabs(v1) > kStartThreshold)) {
      found = l;
      o0 = v0;
      o1 = (l + 1 <= L) ? v1 : 0.0;
      if (!ckp && !ckd) break;
    }
    // chunk checkpoints: the recurrence pair at the chunk's first l once the pair has
    // started there, zero before (a pair starting inside the chunk is injected at ls)
    const double w0 = found <= l ? v0 : 0.0;
    const double w1 = (found <= l && l + 1 <= L) ? v1 : 0.0;
    if (ckp && (l - m) % kChunk == 0) ckp[(l - m) / kChunk] = make_float2((float)w0, (float)w1);
    if (ckd && (l - m) % kChunkDf == 0) {
      const float h0 = (float)w0, h1 = (float)w1;
      ckd[(l - m) / kChunkDf] = make_float4(h0, (float)(w0 - (double)h0), h1, (float)(w1 - (double)h1));
    }
    if (l + 2 > L) break;
    const double n0 = fma(-Am[l + 2], yy, Am[l + 2]) * v1 - v0;
    const double n1 = (l + 3 <= L) ? fma(-Am[l + 3], yy, Am[l + 3]) * n0 - v1 : 0.0;
    v0 = n0;
    v1 = n1;
    if (k > 0 && fmax(fabs(v0), fabs(v1)) > kGrow) {
      v0 *= kShiftDown;
      v1 *= kShiftDown;
      --k;
    }
    l += 2;
  }
  ls[idx] = found;
  st64[idx] = make_double2(o0, o1);
  st32[idx] = make_float2((float)o0, (float)o1);
}

template <typename T2, typename T>
__global__ void k_pack(const double* __restrict__ packed, const double* __restrict__ c, int L,
                       T2* __restrict__ out) {
  const int m = blockIdx.y;
  const int map = blockIdx.z;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > L) return;
  const double* src = packed + (int64_t)map * (L + 1) * (L + 1) + packed_off(L, m);
  const int64_t i = lm_off(L, m) + (l - m);
  const double cc = c[i];
  const double re = src[l - m];
  const double im = m > 0 ? src[(L - m + 1) + (l - m)] : 0.0;
  T2 v;
  v.x = (T)(cc * re);
  v.y = (T)(cc * im);
  out[(int64_t)map * nlm_of(L) + i] = v;
}

__global__ void k_unpack(const double2* __restrict__ lmc, int L, double* __restrict__ packed) {
  const int m = blockIdx.y;
  const int map = blockIdx.z;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > L) return;
  const double2 v = lmc[(int64_t)map * nlm_of(L) + lm_off(L, m) + (l - m)];
  double* dst = packed + (int64_t)map * (L + 1) * (L + 1) + packed_off(L, m);
  dst[l - m] = v.x;
  if (m > 0) dst[(L - m + 1) + (l - m)] = v.y;
}

// tmin[m][t] = min over the pairs p of tile t (kTileMinPT consecutive pairs) of ls[m][p]
__global__ void k_tile_min(const int* __restrict__ ls, int npair, int ntile, int* __restrict__ tmin) {
  const int m = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntile) return;
  int v = INT_MAX;
  const int p1 = min(npair, (t + 1) * kTileMinPT);
  for (int p = t * kTileMinPT; p < p1; ++p) v = min(v, ls[(int64_t)m * npair + p]);
  tmin[(int64_t)m * ntile + t] = v;
}

}  // namespace

int pack_alm(const Grid& g, int prec, int nmaps, const double* packed, void* alm, cudaStream_t s) {
  const int L = g.lmax;
  dim3 blk(128), grd((L + 1 + 127) / 128, L + 1, nmaps);
  if (!is_f32(prec))
    k_pack<double2, double><<<grd, blk, 0, s>>>(packed, g.c64.as<double>(), L, (double2*)alm);
  else
    k_pack<float2, float><<<grd, blk, 0, s>>>(packed, g.c64.as<double>(), L, (float2*)alm);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

int unpack_alm(const Grid& g, int nmaps, const double* lmc, double* packed, cudaStream_t s) {
  const int L = g.lmax;
  dim3 blk(128), grd((L + 1 + 127) / 128, L + 1, nmaps);
  k_unpack<<<grd, blk, 0, s>>>((const double2*)lmc, L, packed);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

int grid_build_tables(Grid& g) {
  const int L = g.lmax;
  const int64_t nlm = nlm_of(L);

  // ---- ring pairs ----
  g.npair = (g.nring + 1) / 2;
  std::vector<double> yh(g.npair), sh(g.npair);
  std::vector<float> yf(g.npair);
  std::vector<int> pr(2 * g.npair), phase(g.npair);
  for (int p = 0; p < g.npair; ++p) {
    const int south = g.nring - 1 - p;
    pr[2 * p] = p;
    pr[2 * p + 1] = (south != p) ? south : -1;
    const double s2 = std::sin(0.5 * g.theta[p]);
    yh[p] = 2.0 * s2 * s2;
    sh[p] = std::sin(g.theta[p]);
    yf[p] = (float)yh[p];
    const double half = M_PI / g.nphi[p];
    if (g.phi0[p] == 0.0) phase[p] = 0;
    else if (std::fabs(g.phi0[p] - half) < 1e-15) phase[p] = 1;
    else {
      set_error("ring %d: unsupported azimuth offset", p);
      return CMBWS_ERR_ARG;
    }
  }
  CMBWS_TRY(g.y64.upload(yh.data(), yh.size() * 8));
  CMBWS_TRY(g.y32.upload(yf.data(), yf.size() * 4));
  CMBWS_TRY(g.pair_ring.upload(pr.data(), pr.size() * 4));
  CMBWS_TRY(g.pair_phase.upload(phase.data(), phase.size() * 4));
  CMBWS_TRY(g.ring_off.upload(g.offset.data(), (g.nring + 1) * 8));
  std::vector<float> wf(g.nring);
  for (int r = 0; r < g.nring; ++r) wf[r] = (float)g.weight[r];
  CMBWS_TRY(g.ring_w64.upload(g.weight.data(), g.nring * 8));
  CMBWS_TRY(g.ring_w32.upload(wf.data(), g.nring * 4));

  // ---- recurrence coefficients ----
  std::vector<double> A(nlm), c(nlm);
  std::vector<float> Af(nlm);
  for (int m = 0; m <= L; ++m) {
    const int64_t o = lm_off(L, m) - m;
    double a_prev = 0.0;  // a_{l-1}
    for (int l = m; l <= L; ++l) {
      double a = 0.0;
      if (l > m) a = std::sqrt((4.0 * l * l - 1.0) / ((double)l * l - (double)m * m));
      if (l <= m + 1) {
        c[o + l] = 1.0;
        A[o + l] = 0.0;
      } else {
        c[o + l] = (a / a_prev) * c[o + l - 2];
        A[o + l] = a * c[o + l - 1] / c[o + l];
      }
      Af[o + l] = (float)A[o + l];
      a_prev = a;
    }
  }
  CMBWS_TRY(g.A64.upload(A.data(), nlm * 8));
  CMBWS_TRY(g.A32.upload(Af.data(), nlm * 4));
  {
    // difference form of the recurrence near the poles (FP32 synthesis):
    // R_l = c_{l-1} / c_l, S_l = 1 / R_{l-1}, B_l = A_l - R_l - S_l
    std::vector<float> brs(3 * nlm, 0.f);
    for (int m = 0; m <= L; ++m) {
      const int64_t o = lm_off(L, m) - m;
      for (int l = m + 2; l <= L; ++l) {
        const double R = c[o + l - 1] / c[o + l], S = c[o + l - 1] / c[o + l - 2];
        brs[3 * (o + l)] = (float)(A[o + l] - R - S);
        brs[3 * (o + l) + 1] = (float)R;
        brs[3 * (o + l) + 2] = (float)S;
      }
      if (m + 1 <= L) brs[3 * (o + m + 1) + 1] = (float)(c[o + m] / c[o + m + 1]);
    }
    CMBWS_TRY(g.BRS32.upload(brs.data(), nlm * 12));
  }
  {
    std::vector<float> A2(2 * nlm);
    for (int64_t i = 0; i < nlm; ++i) {
      const float h = (float)A[i];
      A2[2 * i] = h;
      A2[2 * i + 1] = (float)(A[i] - (double)h);
    }
    CMBWS_TRY(g.A2f.upload(A2.data(), nlm * 8));
  }
  CMBWS_TRY(g.c64.upload(c.data(), nlm * 8));

  // ---- start values ----
  {
    std::vector<double> fmm(L + 1, 0.0);
    for (int m = 1; m <= L; ++m) fmm[m] = std::sqrt((2.0 * m + 1.0) / (2.0 * m));
    g.fmm_h = fmm;
    DevMem d_fmm, d_sin, d_sv, d_sk;
    CMBWS_TRY(d_fmm.upload(fmm.data(), fmm.size() * 8));
    CMBWS_TRY(d_sin.upload(sh.data(), sh.size() * 8));
    const int64_t nst = (int64_t)(L + 1) * g.npair;
    CMBWS_TRY(d_sv.alloc(nst * 8));
    CMBWS_TRY(d_sk.alloc(nst * 4));
    CMBWS_TRY(g.ls.alloc(nst * 4));
    CMBWS_TRY(g.st64.alloc(nst * 16));
    CMBWS_TRY(g.st32.alloc(nst * 8));
    k_seeds<<<(g.npair + 127) / 128, 128>>>(d_sin.as<double>(), d_fmm.as<double>(), L, g.npair,
                                            d_sv.as<double>(), d_sk.as<int>());
    CMBWS_LAUNCH_CHECK();
    dim3 grd((g.npair + 127) / 128, L + 1);
    // FP32 chunk checkpoints of the adjoint (legendre.cu): [m][pair][chunk]
    std::vector<int64_t> cb(L + 1, 0);
    int64_t tot = 0;
    for (int m = 0; m <= L; ++m) {
      cb[m] = tot;
      tot += (int64_t)g.npair * ((L - m + kChunk) / kChunk);
    }
    CMBWS_TRY(g.ck_base.upload(cb.data(), (L + 1) * 8));
    {
      const std::vector<int2> wt = adjoint_warp_tasks(L, kChunk);
      CMBWS_TRY(g.wt32.upload(wt.data(), wt.size() * sizeof(int2)));
      g.nwt32 = (int)wt.size();
    }
    CMBWS_TRY(g.ck32.alloc((size_t)tot * 8));
    k_start<<<grd, 128>>>(g.y64.as<double>(), g.A64.as<double>(), L, g.npair, d_sv.as<double>(),
                          d_sk.as<int>(), g.ls.as<int>(), g.st64.as<double2>(), g.st32.as<float2>(),
                          g.ck_base.as<int64_t>(), g.ck32.as<float2>(), nullptr, nullptr);
    CMBWS_LAUNCH_CHECK();
    const int ntile = (g.npair + kTileMinPT - 1) / kTileMinPT;
    CMBWS_TRY(g.ls_tmin.alloc((size_t)(L + 1) * ntile * 4));
    dim3 gt((ntile + 127) / 128, L + 1);
    k_tile_min<<<gt, 128>>>(g.ls.as<int>(), g.npair, ntile, g.ls_tmin.as<int>());
    CMBWS_LAUNCH_CHECK();
    CMBWS_CUDA(cudaDeviceSynchronize());
  }

  // ---- ring FFT plans ----
  {
    std::vector<int> plan_of_len;
    std::vector<int> pplan(g.npair);
    g.plans.clear();
    g.max_n = 1;
    g.nmax2 = 2;
    std::vector<std::complex<double>> tab;
    auto plan_for = [&](int n) -> int {
      for (size_t i = 0; i < g.plans.size(); ++i)
        if (g.plans[i].n == n) return (int)i;
      FftPlan P{};
      P.n = n;
      P.bluestein = is_pow2(n) ? 0 : 1;
      P.n2 = P.bluestein ? next_pow2(2 * n - 1) : n;
      P.chirp = (int64_t)tab.size();
      if (P.bluestein) {
        for (int t = 0; t < n; ++t) {
          const int64_t s = ((int64_t)t * t) % (2 * (int64_t)n);
          const double ang = M_PI * (double)s / n;
          tab.emplace_back(std::cos(ang), std::sin(ang));
        }
        std::vector<std::complex<double>> v(P.n2, 0.0);
        for (int t = 0; t < n; ++t) {
          v[t] = tab[P.chirp + t];
          if (t > 0) v[P.n2 - t] = tab[P.chirp + t];
        }
        host_fft(v, -1);
        // stored in bit-reversed order: the ring FFT multiplies it into a spectrum that its
        // decimation-in-frequency transform leaves bit-reversed
        P.filt = (int64_t)tab.size();
        int lg2 = 0;
        while ((1 << lg2) < P.n2) ++lg2;
        for (int q = 0; q < P.n2; ++q) {
          int j = 0;
          for (int b = 0; b < lg2; ++b) j |= ((q >> b) & 1) << (lg2 - 1 - b);
          tab.push_back(v[j] / (double)P.n2);
        }
      } else {
        P.filt = 0;
      }
      P.phase = (int64_t)tab.size();
      for (int k = 0; k < n; ++k) {
        const double ang = M_PI * (double)k / n;
        tab.emplace_back(std::cos(ang), std::sin(ang));
      }
      g.plans.push_back(P);
      if (P.n2 > g.nmax2) g.nmax2 = P.n2;
      if (n > g.max_n) g.max_n = n;
      return (int)g.plans.size() - 1;
    };
    for (int p = 0; p < g.npair; ++p) pplan[p] = plan_for(g.nphi[p]);
    g.tw_off = (int64_t)tab.size();
    for (int k = 0; k < g.nmax2 / 2; ++k) {
      const double ang = -2.0 * M_PI * k / g.nmax2;
      tab.emplace_back(std::cos(ang), std::sin(ang));
    }
    std::vector<float> tf(2 * tab.size());
    for (size_t i = 0; i < tab.size(); ++i) {
      tf[2 * i] = (float)tab[i].real();
      tf[2 * i + 1] = (float)tab[i].imag();
    }
    std::vector<float> td(4 * tab.size());  // (re hi, re lo, im hi, im lo)
    for (size_t i = 0; i < tab.size(); ++i) {
      const double re = tab[i].real(), im = tab[i].imag();
      td[4 * i] = (float)re;
      td[4 * i + 1] = (float)(re - (double)(float)re);
      td[4 * i + 2] = (float)im;
      td[4 * i + 3] = (float)(im - (double)(float)im);
    }
    CMBWS_TRY(g.fft64.upload(tab.data(), tab.size() * 16));
    CMBWS_TRY(g.fft32.upload(tf.data(), tf.size() * 4));
    CMBWS_TRY(g.fftdf.upload(td.data(), td.size() * 4));
    CMBWS_TRY(g.plans_d.upload(g.plans.data(), g.plans.size() * sizeof(FftPlan)));
    CMBWS_TRY(g.pair_plan.upload(pplan.data(), pplan.size() * 4));
  }
  return CMBWS_OK;
}

__global__ void k_to_df(const double* __restrict__ v, float2* __restrict__ o, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float h = (float)v[i];
  o[i] = make_float2(h, (float)(v[i] - (double)h));
}

std::vector<int2> adjoint_warp_tasks(int L, int chunk) {
  std::vector<int2> t;
  for (int m = 0; m <= L; ++m) {
    const int nck = (L - m + chunk) / chunk;
    for (int c = 0; c < nck; c += 32) t.push_back(make_int2(m, c));
  }
  return t;
}

int grid_ensure_ck64(const Grid& gc) {
  std::lock_guard<std::mutex> lk(gc.ck64_mu);
  if (gc.ck64.p) return CMBWS_OK;
  Grid& g = const_cast<Grid&>(gc);  // tables only; the geometry is not touched
  const int L = g.lmax;
  std::vector<int64_t> cb(L + 1, 0);
  int64_t tot = 0;
  for (int m = 0; m <= L; ++m) {
    cb[m] = tot;
    tot += (int64_t)g.npair * ((L - m + kChunkDf) / kChunkDf);
  }
  DevMem cbd;
  CMBWS_TRY(cbd.upload(cb.data(), (L + 1) * 8));
  DevMem d_fmm, d_sin, d_sv, d_sk, ls_t, st64_t, st32_t;
  std::vector<double> sh(g.npair);
  for (int p = 0; p < g.npair; ++p) sh[p] = std::sin(g.theta[p]);
  CMBWS_TRY(d_fmm.upload(g.fmm_h.data(), g.fmm_h.size() * 8));
  CMBWS_TRY(d_sin.upload(sh.data(), sh.size() * 8));
  const int64_t nst = (int64_t)(L + 1) * g.npair;
  CMBWS_TRY(d_sv.alloc(nst * 8));
  CMBWS_TRY(d_sk.alloc(nst * 4));
  CMBWS_TRY(ls_t.alloc(nst * 4));
  CMBWS_TRY(st64_t.alloc(nst * 16));
  CMBWS_TRY(st32_t.alloc(nst * 8));
  DevMem ck, y2;
  CMBWS_TRY(ck.alloc((size_t)tot * 16));
  CMBWS_TRY(y2.alloc((size_t)g.npair * 8));
  k_to_df<<<(g.npair + 127) / 128, 128>>>(g.y64.as<double>(), y2.as<float2>(), g.npair);
  CMBWS_LAUNCH_CHECK();
  k_seeds<<<(g.npair + 127) / 128, 128>>>(d_sin.as<double>(), d_fmm.as<double>(), L, g.npair,
                                          d_sv.as<double>(), d_sk.as<int>());
  CMBWS_LAUNCH_CHECK();
  dim3 grd((g.npair + 127) / 128, L + 1);
  k_start<<<grd, 128>>>(g.y64.as<double>(), g.A64.as<double>(), L, g.npair, d_sv.as<double>(),
                        d_sk.as<int>(), ls_t.as<int>(), st64_t.as<double2>(), st32_t.as<float2>(),
                        g.ck_base.as<int64_t>(), nullptr, cbd.as<int64_t>(), ck.as<float4>());
  CMBWS_LAUNCH_CHECK();
  CMBWS_CUDA(cudaDeviceSynchronize());
  {
    const std::vector<int2> wt = adjoint_warp_tasks(L, kChunkDf);
    DevMem w;
    CMBWS_TRY(w.upload(wt.data(), wt.size() * sizeof(int2)));
    g.wtdf = std::move(w);
    g.nwtdf = (int)wt.size();
  }
  g.y2f = std::move(y2);
  g.ck64_base = std::move(cbd);
  g.ck64 = std::move(ck);
  return CMBWS_OK;
}

// ---- grid geometry (host) and the public grid API ----

static int build_geometry(Grid& g, int kind, int n, int lmax) {
  g.kind = kind;
  g.n = n;
  g.lmax = lmax;
  if (kind == CMBWS_GRID_GL) {
    if (n < lmax + 1) {
      set_error("GL grid needs n >= lmax + 1 rings (n=%d, lmax=%d)", n, lmax);
      return CMBWS_ERR_ARG;
    }
    std::vector<double> x, w;
    gauss_legendre_nodes(n, x, w);
    const int nphi = 2 * lmax + 1;
    g.nring = n;
    for (int r = 0; r < n; ++r) {
      g.theta.push_back(std::acos(x[r]));
      g.nphi.push_back(nphi);
      g.phi0.push_back(0.0);
      g.weight.push_back(w[r] * 2.0 * M_PI / nphi);
    }
  } else if (kind == CMBWS_GRID_HEALPIX) {
    const int ns = n;
    g.nring = 4 * ns - 1;
    const double npix = 12.0 * ns * ns;
    for (int i = 1; i <= g.nring; ++i) {
      const int ip = i <= 2 * ns ? i : 4 * ns - i;
      double z;
      int np;
      double ph;
      if (ip < ns) {
        z = 1.0 - (double)ip * ip / (3.0 * ns * ns);
        np = 4 * ip;
        ph = M_PI / (4.0 * ip);
      } else {
        z = 4.0 / 3.0 - 2.0 * ip / (3.0 * ns);
        np = 4 * ns;
        ph = ((ip - ns) % 2 == 0) ? M_PI / (4.0 * ns) : 0.0;
      }
      if (i > 2 * ns) z = -z;
      g.theta.push_back(std::acos(z));
      g.nphi.push_back(np);
      g.phi0.push_back(ph);
      g.weight.push_back(4.0 * M_PI / npix);
    }
  } else {
    set_error("unknown grid kind %d", kind);
    return CMBWS_ERR_ARG;
  }
  g.offset.assign(g.nring + 1, 0);
  for (int r = 0; r < g.nring; ++r) g.offset[r + 1] = g.offset[r] + g.nphi[r];
  g.npix = g.offset[g.nring];
  return CMBWS_OK;
}

}  // namespace cmbws

using namespace cmbws;

extern "C" int cmbws_plan_grid(cmbws_grid_kind kind, int n, int lmax, cmbws_grid* out) {
  clear_error();
  if (!out || n < 1 || lmax < 0 || lmax > 8192) {
    set_error("cmbws_plan_grid: invalid arguments (n=%d, lmax=%d)", n, lmax);
    return CMBWS_ERR_ARG;
  }
  *out = nullptr;
  Grid* g = new (std::nothrow) Grid();
  if (!g) return CMBWS_ERR_NOMEM;
  cudaGetDevice(&g->device);
  int s = build_geometry(*g, (int)kind, n, lmax);
  if (s == CMBWS_OK) s = grid_build_tables(*g);
  if (s != CMBWS_OK) {
    delete g;
    return s;
  }
  handle_add(HANDLE_GRID, g);
  *out = reinterpret_cast<cmbws_grid>(g);
  return CMBWS_OK;
}

extern "C" int cmbws_grid_info(cmbws_grid gh, int64_t* npix, int* nring, const double** theta,
                               const double** weight) {
  clear_error();
  Grid* g = as_grid(gh);
  if (!g) {
    set_error("cmbws_grid_info: null grid");
    return CMBWS_ERR_ARG;
  }
  if (npix) *npix = g->npix;
  if (nring) *nring = g->nring;
  if (theta) *theta = g->theta.data();
  if (weight) *weight = g->weight.data();
  return CMBWS_OK;
}

extern "C" int cmbws_grid_rings(cmbws_grid gh, const double** phi0, const int** nphi,
                                const int64_t** offset, int* lmax) {
  clear_error();
  Grid* g = as_grid(gh);
  if (!g) {
    set_error("cmbws_grid_rings: null grid");
    return CMBWS_ERR_ARG;
  }
  if (phi0) *phi0 = g->phi0.data();
  if (nphi) *nphi = g->nphi.data();
  if (offset) *offset = g->offset.data();
  if (lmax) *lmax = g->lmax;
  return CMBWS_OK;
}

extern "C" int cmbws_grid_destroy(cmbws_grid gh) {
  clear_error();
  if (!gh) return CMBWS_OK;
  if (!handle_del(HANDLE_GRID, gh)) {
    set_error("cmbws_grid_destroy: not a live grid handle (destroyed twice?)");
    return CMBWS_ERR_ARG;
  }
  delete reinterpret_cast<Grid*>(gh);
  return CMBWS_OK;
}
