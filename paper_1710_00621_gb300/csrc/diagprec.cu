// Block-diagonal comparison preconditioner M_diag (Sec. 5 of the paper).
//
// The paper measures M_PI against the block-diagonal preconditioner of earlier Gibbs-sampling
// work, M_diag = (U^T diag(T) U)^-1: for every real coefficient (l, m, cos / sin) the
// Ncomp x Ncomp block
//   B_kk' = delta_kk' C_{k,l}^-1 + sum_nu b_{nu,l}^2 q_{nu,k} q_{nu,k'} D_nu(l, m, c/s)
// (q the preconditioner's scalars, Eq. optimal-q for variable maps) is inverted, with
// D_nu = diag(Y_nu^T N_nu^-1 Y_nu) from ring sums (Y_lm^c = sqrt(2) lambda cos(m phi), and
// 2 cos^2 = 1 + cos(2 m phi)):
//   D(l, 0) = sum_r lambda_l0^2 S_r,  D(l, m, c / s) = sum_r lambda_lm^2 (S_r +/- C_r(2m)),
// S_r = sum_j tau_rj, C_r(k) = sum_j tau_rj cos(k phi_rj).  North and south rings of a pair
// share lambda^2, so the ring quantities are added per pair.
//
// Built on the first solve that asks for it (precond = 3):
//   * k_ring_cos: FP64 ring sums by complex rotation, one CTA per ring, one thread per m;
//   * k_pair_g: the pair weights S_N + S_S +/- (C_N + C_S) (FP32);
//   * k_diag_l2: sum over pairs of lambda^2 g, one thread per chunk of 8 values of l from the
//     FP32 recurrence checkpoints of the adjoint (warp tasks of the grid), FP32 sums;
//   * k_diag_blocks: the blocks in FP64 and their inverses (Gauss-Jordan, SPD);
// and applied by k_diag_apply (one thread per (l, m), both parts).
#include "model.h"

namespace cmbws {

namespace {

constexpr int kMaxNc = kMaxComp;

// out[r * (L + 1) + m] = C_r(2m) (m >= 1) and out[r * (L + 1)] = S_r
__global__ void k_ring_cos(const double* __restrict__ tau, const int64_t* __restrict__ roff,
                           const double* __restrict__ phi0, int L, double* __restrict__ out) {
  const int r = blockIdx.x;
  const int64_t off = roff[r];
  const int n = (int)(roff[r + 1] - off);
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    const int64_t k = 2LL * m;
    const int kr = (int)(k % n);
    double sw, cw, s0, c0;
    sincospi(2.0 * kr / n, &sw, &cw);      // step exp(i 2 pi k / n)
    sincos((double)k * phi0[r], &s0, &c0);  // exp(i k phi0)
    double cr = c0, ci = s0, acc = 0.0;
    for (int j = 0; j < n; ++j) {
      acc = fma(tau[off + j], cr, acc);
      const double t = cr * cw - ci * sw;
      ci = cr * sw + ci * cw;
      cr = t;
    }
    out[(int64_t)r * (L + 1) + m] = acc;  // m = 0: S_r
  }
}

// g[m * npair + p] = (S_N + S_S + C_N(2m) + C_S(2m), S_N + S_S - C_N(2m) - C_S(2m)); m = 0: (S, 0)
__global__ void k_pair_g(const double* __restrict__ rc, const int2* __restrict__ pring, int L,
                         int npair, float2* __restrict__ g) {
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  const int m = blockIdx.y;
  if (p >= npair) return;
  const int2 rr = pring[p];
  double S = rc[(int64_t)rr.x * (L + 1)], C = rc[(int64_t)rr.x * (L + 1) + m];
  if (rr.y >= 0) {
    S += rc[(int64_t)rr.y * (L + 1)];
    C += rc[(int64_t)rr.y * (L + 1) + m];
  }
  g[(int64_t)m * npair + p] = m == 0 ? make_float2((float)S, 0.f) : make_float2((float)(S + C), (float)(S - C));
}

// D(l, m) = c_lm^2 sum_pairs mu_lm^2 g (cos, sin parts), one thread per chunk of kChunk l
__global__ void __launch_bounds__(128)
k_diag_l2(const float2* __restrict__ g, const float* __restrict__ Acoef, const int* __restrict__ ls_tab,
          const float2* __restrict__ st, const float* __restrict__ yr, const float2* __restrict__ ck,
          const int64_t* __restrict__ ck_base, const int2* __restrict__ tasks, int ntask,
          const double* __restrict__ c64, double2* __restrict__ out, int L, int npair) {
  constexpr int K = kChunk;
  const int lane = threadIdx.x & 31;
  const int task = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  if (task >= ntask) return;
  const int2 tk = tasks[task];
  const int m = tk.x;
  const int nck = (L - m + K) / K;
  const int c = tk.y + lane;
  if (c >= nck) return;
  const int l0 = m + K * c;
  const int64_t lmo = lm_off(L, m) - m;
  float Al[K], ac[K], as[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    Al[j] = (l0 + j <= L) ? Acoef[lmo + l0 + j] : 0.f;
    ac[j] = as[j] = 0.f;
  }
  const float2* ckc = ck + ck_base[m] + c;
  for (int p = 0; p < npair; ++p) {
    const int lsp = ls_tab[(int64_t)m * npair + p];
    if (lsp > l0 + K - 1) continue;
    const float2 cv = ckc[(int64_t)p * nck];
    const float2 gw = g[(int64_t)m * npair + p];
    const float2 sv = st[(int64_t)m * npair + p];
    const float yv = yr[p];
    float ma = cv.x, mb = cv.y;
    if (lsp == l0) {
      ma = sv.x;
      mb = sv.y;
    }
    ac[0] = fmaf(ma * ma, gw.x, ac[0]);
    as[0] = fmaf(ma * ma, gw.y, as[0]);
    ac[1] = fmaf(mb * mb, gw.x, ac[1]);
    as[1] = fmaf(mb * mb, gw.y, as[1]);
#pragma unroll
    for (int j = 2; j < K; j += 2) {
      float na = fmaf(-Al[j], yv, Al[j]) * mb - ma;
      float nb = fmaf(-Al[j + 1], yv, Al[j + 1]) * na - mb;
      if (l0 + j == lsp) {
        na = sv.x;
        nb = sv.y;
      }
      ma = na;
      mb = nb;
      ac[j] = fmaf(ma * ma, gw.x, ac[j]);
      as[j] = fmaf(ma * ma, gw.y, as[j]);
      ac[j + 1] = fmaf(mb * mb, gw.x, ac[j + 1]);
      as[j + 1] = fmaf(mb * mb, gw.y, as[j + 1]);
    }
  }
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int l = l0 + j;
    if (l > L) break;
    const double cc = c64[lmo + l];
    out[lmo + l] = make_double2(cc * cc * (double)ac[j], cc * cc * (double)as[j]);
  }
}

struct DiagArgs {
  int nc, nobs, Lmax;
  int L[kMaxBands];
  const double2* D[kMaxBands];  // band nu: (cos, sin) per (l, m), lm_off(L_nu) layout
};

// inverse blocks over the packed layout of Lmax (absent components: zero rows / columns)
__global__ void k_diag_blocks(HarmDev h, DiagArgs a, const double* __restrict__ qpre,
                              double* __restrict__ inv) {
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > a.Lmax) return;
  const int nc = a.nc;
  for (int cs = 0; cs < (m > 0 ? 2 : 1); ++cs) {
    double B[kMaxNc * kMaxNc], I[kMaxNc * kMaxNc];
    bool pres[kMaxNc];
    for (int k = 0; k < nc; ++k) pres[k] = l <= h.compL[k];
    for (int i = 0; i < nc * nc; ++i) B[i] = I[i] = 0.0;
    for (int nu = 0; nu < a.nobs; ++nu) {
      if (l > a.L[nu]) continue;
      const double2 d = a.D[nu][lm_off(a.L[nu], m) + (l - m)];
      const double b = h.beam[h.beamOff[nu] + l];
      const double w = b * b * (cs == 0 ? d.x : d.y);
      for (int k = 0; k < nc; ++k)
        for (int kk = 0; kk < nc; ++kk)
          B[k * nc + kk] += w * qpre[nu * nc + k] * qpre[nu * nc + kk];
    }
    for (int k = 0; k < nc; ++k) {
      B[k * nc + k] += pres[k] ? h.cinv[h.clOff[k] + l] : 0.0;
      for (int kk = 0; kk < nc; ++kk)
        if (!pres[k] || !pres[kk]) B[k * nc + kk] = (k == kk) ? 1.0 : 0.0;
      I[k * nc + k] = pres[k] ? 1.0 : 0.0;
    }
    // Gauss-Jordan on the symmetric positive definite block (absent rows are the identity)
    for (int col = 0; col < nc; ++col) {
      const double piv = B[col * nc + col];
      const double ip = piv != 0.0 ? 1.0 / piv : 0.0;
      for (int j = 0; j < nc; ++j) {
        B[col * nc + j] *= ip;
        I[col * nc + j] *= ip;
      }
      for (int r = 0; r < nc; ++r) {
        if (r == col) continue;
        const double f = B[r * nc + col];
        if (f == 0.0) continue;
        for (int j = 0; j < nc; ++j) {
          B[r * nc + j] -= f * B[col * nc + j];
          I[r * nc + j] -= f * I[col * nc + j];
        }
      }
    }
    const int64_t idx = packed_off(a.Lmax, m) + cs * (a.Lmax - m + 1) + (l - m);
    for (int i = 0; i < nc * nc; ++i) inv[idx * nc * nc + i] = I[i];
  }
}

__global__ void k_diag_apply(HarmDev h, int Lmax, const double* __restrict__ inv,
                             const double* __restrict__ r, double* __restrict__ z) {
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > Lmax) return;
  const int nc = h.ncomp;
  for (int cs = 0; cs < (m > 0 ? 2 : 1); ++cs) {
    double x[kMaxNc];
    int64_t pos[kMaxNc];
    for (int k = 0; k < nc; ++k) {
      const int Lk = h.compL[k];
      pos[k] = -1;
      x[k] = 0.0;
      if (l <= Lk) {
        pos[k] = h.compOff[k] + packed_off(Lk, m) + cs * (Lk - m + 1) + (l - m);
        x[k] = r[pos[k]];
      }
    }
    const int64_t idx = packed_off(Lmax, m) + cs * (Lmax - m + 1) + (l - m);
    const double* B = inv + idx * nc * nc;
    for (int k = 0; k < nc; ++k) {
      if (pos[k] < 0) continue;
      double s = 0.0;
      for (int kk = 0; kk < nc; ++kk) s += B[k * nc + kk] * x[kk];
      z[pos[k]] = s;
    }
  }
}

}  // namespace

int Model::build_diag(cudaStream_t s) {
  const HarmDev h = harm();
  DiagArgs a{};
  a.nc = ncomp;
  a.nobs = nobs;
  a.Lmax = Lcomp;
  int64_t tot = 0;
  std::vector<int64_t> off(nobs);
  for (int nu = 0; nu < nobs; ++nu) {
    off[nu] = tot;
    tot += nlm_of(Lnu[nu]);
  }
  CMBWS_TRY(dg_D.alloc((size_t)tot * 16));
  for (int nu = 0; nu < nobs; ++nu) {
    const Grid& g = *groups[band_group[nu]].grid;
    const int L = g.lmax;
    DevMem rc, gw, phi;
    CMBWS_TRY(rc.alloc((size_t)g.nring * (L + 1) * 8));
    CMBWS_TRY(gw.alloc((size_t)(L + 1) * g.npair * 8));
    CMBWS_TRY(phi.upload(g.phi0.data(), g.nring * 8));
    {
      ProfScope ps(PROF_HARM, s, 1);
      k_ring_cos<<<g.nring, 256, 0, s>>>(pixA64[nu].as<double>(), g.ring_off.as<int64_t>(),
                                        phi.as<double>(), L, rc.as<double>());
      dim3 gg((g.npair + 127) / 128, L + 1);
      k_pair_g<<<gg, 128, 0, s>>>(rc.as<double>(), g.pair_ring.as<int2>(), L, g.npair, gw.as<float2>());
      double2* D = dg_D.as<double2>() + off[nu];
      k_diag_l2<<<(g.nwt32 + 3) / 4, 128, 0, s>>>(gw.as<float2>(), g.A32.as<float>(), g.ls.as<int>(),
                                                  g.st32.as<float2>(), g.y32.as<float>(), g.ck32.as<float2>(),
                                                  g.ck_base.as<int64_t>(), g.wt32.as<int2>(), g.nwt32,
                                                  g.c64.as<double>(), D, L, g.npair);
      CMBWS_LAUNCH_CHECK();
    }
    CMBWS_CUDA(cudaStreamSynchronize(s));  // the temporaries are freed here
    a.L[nu] = L;
    a.D[nu] = dg_D.as<double2>() + off[nu];
  }
  CMBWS_TRY(dg_inv.alloc((size_t)(Lcomp + 1) * (Lcomp + 1) * ncomp * ncomp * 8));
  dim3 grd((Lcomp + 1 + 127) / 128, Lcomp + 1);
  k_diag_blocks<<<grd, 128, 0, s>>>(h, a, d_qpre.as<double>(), dg_inv.as<double>());
  CMBWS_LAUNCH_CHECK();
  CMBWS_CUDA(cudaStreamSynchronize(s));
  dg_ready = true;
  return CMBWS_OK;
}

int Model::apply_diag(const double* r, double* z, cudaStream_t s) {
  if (!dg_ready) CMBWS_TRY(build_diag(s));
  const HarmDev h = harm();
  dim3 grd((Lcomp + 1 + 127) / 128, Lcomp + 1);
  ProfScope ps(PROF_HARM, s, 1);
  k_diag_apply<<<grd, 128, 0, s>>>(h, Lcomp, dg_inv.as<double>(), r, z);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

}  // namespace cmbws

using namespace cmbws;

extern "C" int cmbws_apply_M_diag(cmbws_model mh, const double* r, double* z, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (refuse_sharded(M, "cmbws_apply_M_diag")) return CMBWS_ERR_ARG;
  if (!M || !r || !z || r == z) {
    set_error("cmbws_apply_M_diag: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  return M->apply_diag(r, z, (cudaStream_t)stream);
}
