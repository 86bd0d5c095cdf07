// Terms of the solution gradient: lambda^T (db/dtheta - dA/dtheta x) for the scalar
// mixing entries q_{nu,k} and a log-scale t_k of each prior spectrum.
//
// The paper solves A x = b (Eq. A) for fixed parameters; differentiating it gives
// A dx/dtheta = db/dtheta - (dA/dtheta) x, so a loss L(x) has
// dL/dtheta = lambda^T (db/dtheta - dA/dtheta x) with A lambda = dL/dx.  With
// P_{nu,k} = Y_nu B_nu q_{nu,k} (Eq. P, constant mixing) and the CR right-hand side
// b = P^T (N^-1 d + N^-1/2 w1) + S^-1/2 w2 (Sec. 2.3):
//
//   dq_{nu,k} = <B_nu lambda_k, Y_nu^T (N^-1 d + N^-1/2 w1 - N^-1 P_nu x)>
//             - <B_nu x_k, Y_nu^T N^-1 P_nu lambda>          (both over l <= min(L_nu, L_k))
//   dt_k = lambda_k^T S_k^-1 x_k - 1/2 lambda_k^T S_k^-1/2 w2_k
//
// Cost: two projections (Nobs syntheses each) and two adjoint passes (Nobs each), all
// FP64-accurate (FP64 transforms for FP64 models, double-float otherwise), plus
// harmonic-space dot products reduced in a fixed order.
//
// Spatially variable mixing (Eq. Q, Q~ = Y_nu^T W diag(q) Y_k on the pair's mixing grid):
// the derivative in the map value at pixel p is
//
//   dq_{nu,k}(p) = w_p [ (Y lambda_k)(p) (Y B_nu u_nu)(p) - (Y x_k)(p) (Y B_nu v_nu)(p) ]
//
// with u_nu, v_nu the band outputs of the two adjoint passes above, so each pass adds two
// syntheses per variable pair on its mixing grid and a pixel product.  The scalar entry of a
// variable pair is the derivative in a uniform offset of its map, the sum over its pixels.
#include "model.h"

namespace cmbws {

namespace {

constexpr int kDotNT = 128;

// map <- tau (d - map) + sqrt(tau) w1   (sign = -1), or map <- tau map   (sign = +1, d unused)
__global__ void k_grad_pixels(const double* __restrict__ d, const double* __restrict__ w1,
                              const double* __restrict__ tau, const double* __restrict__ tsq,
                              double* __restrict__ map, int64_t n, int resid) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double t = tau[i];
  if (!resid) {
    map[i] = t * map[i];
    return;
  }
  double v = t * (d[i] - map[i]);
  if (w1) v += tsq[i] * w1[i];
  map[i] = v;
}

__device__ __forceinline__ double block_sum(double v, double* sh) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  __syncthreads();
  if (lane == 0) sh[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += sh[i];
  return s;
}

// Per block (m, l-chunk): partial of sum_{l <= min(L_nu, L_k)} b_{nu,l} a_k(l, m) . u_nu(l, m)
// for every component k; u_nu is band nu's adjoint output (internal layout, (cos, sin) parts).
__global__ void __launch_bounds__(kDotNT)
k_grad_dot(HarmDev h, const double2* __restrict__ u, int Ln, const double* __restrict__ bnu,
           const double* __restrict__ a, double* __restrict__ part) {
  __shared__ double sh[kDotNT / 32];
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t blk = (int64_t)blockIdx.y * gridDim.x + blockIdx.x;
  double2 uv = make_double2(0.0, 0.0);
  double bl = 0.0;
  if (l <= Ln) {
    uv = u[lm_off(Ln, m) + (l - m)];
    bl = bnu[l];
  }
  for (int k = 0; k < h.ncomp; ++k) {
    const int Lk = h.compL[k];
    double v = 0.0;
    if (l <= Ln && l <= Lk) {
      const double* ak = a + h.compOff[k] + packed_off(Lk, m);
      v = ak[l - m] * uv.x;
      if (m > 0) v += ak[(Lk - m + 1) + (l - m)] * uv.y;
      v *= bl;
    }
    const double s = block_sum(v, sh);
    if (threadIdx.x == 0) part[blk * h.ncomp + k] = s;
  }
}

// Per block (m, l-chunk) of component k: partial of sum lambda_k (C^-1 x_k - 1/2 C^-1/2 w2_k)
__global__ void __launch_bounds__(kDotNT)
k_grad_prior(HarmDev h, int k, const double* __restrict__ lam, const double* __restrict__ x,
             const double* __restrict__ w2, double* __restrict__ part) {
  __shared__ double sh[kDotNT / 32];
  const int m = blockIdx.y;
  const int Lk = h.compL[k];
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  double v = 0.0;
  if (l <= Lk) {
    const double ci = h.cinv[h.clOff[k] + l], cs = h.cisq[h.clOff[k] + l];
    const int64_t base = h.compOff[k] + packed_off(Lk, m);
    for (int c = 0; c < (m > 0 ? 2 : 1); ++c) {
      const int64_t i = base + c * (Lk - m + 1) + (l - m);
      double t = ci * x[i];
      if (w2) t -= 0.5 * cs * w2[i];
      v += lam[i] * t;
    }
  }
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) part[(int64_t)blockIdx.y * gridDim.x + blockIdx.x] = s;
}

// Mixing-map gradient of group pair j: out[j][i] (+)= sign w_ring a[j][i] b[j][i] over the
// pixels of ring blockIdx.x, and the ring's partial sum of the result
__global__ void __launch_bounds__(256)
k_grad_mixmap(const double* __restrict__ a, const double* __restrict__ b,
              const int64_t* __restrict__ roff, const double* __restrict__ rw, int64_t npix,
              int nring, double sign, int accumulate, double* __restrict__ out,
              double* __restrict__ part) {
  __shared__ double sh[256 / 32];
  const int r = blockIdx.x, j = blockIdx.y;
  const double w = rw[r];
  double sum = 0.0;
  for (int64_t i = roff[r] + threadIdx.x; i < roff[r + 1]; i += blockDim.x) {
    const int64_t q = (int64_t)j * npix + i;
    double v = sign * w * a[q] * b[q];
    if (accumulate) v += out[q];
    out[q] = v;
    sum += v;
  }
  const double s = block_sum(sum, sh);
  if (threadIdx.x == 0) part[(int64_t)j * nring + r] = s;
}

struct MixOut {
  int idx[kMaxMaps];  // entry of the pair in the gradient terms (nu ncomp + k)
};

// terms[idx[j]] = sum over rings of part[j][r], in a fixed order
__global__ void k_grad_mixsum(const double* __restrict__ part, int nring, MixOut mo,
                              double* __restrict__ terms) {
  __shared__ double sh[256 / 32];
  const int j = blockIdx.x;
  double v = 0.0;
  for (int r = threadIdx.x; r < nring; r += blockDim.x) v += part[(int64_t)j * nring + r];
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) terms[mo.idx[j]] = s;
}

// out[k] (+)= sign * sum_b part[b * stride + k], k < nk, in a fixed order
__global__ void k_grad_finish(const double* __restrict__ part, int64_t nblk, int stride, int nk,
                              double sign, int accumulate, double* __restrict__ out) {
  __shared__ double sh[256 / 32];
  const int k = blockIdx.x;
  if (k >= nk) return;
  double v = 0.0;
  for (int64_t b = threadIdx.x; b < nblk; b += blockDim.x) v += part[b * stride + k];
  const double s = block_sum(v, sh);
  if (threadIdx.x == 0) out[k] = (accumulate ? out[k] : 0.0) + sign * s;
}

}  // namespace

// out: the gradient terms (nobs ncomp + ncomp) or nullptr; maps: per pair nu ncomp + k the
// mixing-map gradient of a variable pair (nullptr entries, or maps == nullptr, are skipped)
static int grad_run(Model& M, const double* x, const double* lam, const double* const* d,
                    const double* const* w1, const double* w2, double* out, double* const* maps,
                    cudaStream_t s) {
  const int ap = M.prec == CMBWS_FP64 ? CMBWS_FP64 : CMBWS_FP32X2;
  // mixing groups: two scratch map sets of the largest group, the accumulated gradient of
  // every variable pair and the per-ring partial sums
  std::vector<int64_t> moff(M.mgroups.size() + 1, 0);
  size_t scratch = 0, part_mix = 1;
  for (size_t gi = 0; gi < M.mgroups.size(); ++gi) {
    const Group& G = M.mgroups[gi];
    moff[gi + 1] = moff[gi] + (int64_t)G.nmaps * G.grid->npix;
    scratch = std::max(scratch, (size_t)G.nmaps * G.grid->npix);
    part_mix = std::max(part_mix, (size_t)G.nmaps * G.grid->nring);
  }
  if (M.nmix) {
    CMBWS_TRY(M.gradmix.ensure(2 * scratch * 8));
    CMBWS_TRY(M.gradmixout.ensure((size_t)moff.back() * 8));
    CMBWS_TRY(M.gradmixpart.ensure(part_mix * 8));
  }
  const HarmDev h = M.harm();
  // band maps, laid out group by group so that a group's maps are contiguous
  std::vector<double*> mp(M.nobs, nullptr);
  std::vector<int64_t> goff(M.groups.size() + 1, 0);
  for (size_t gi = 0; gi < M.groups.size(); ++gi)
    goff[gi + 1] = goff[gi] + (int64_t)M.groups[gi].nmaps * M.groups[gi].grid->npix;
  CMBWS_TRY(M.gradmaps.ensure((size_t)goff.back() * 8));
  int64_t nblk_max = 1;
  for (size_t gi = 0; gi < M.groups.size(); ++gi) {
    const Group& G = M.groups[gi];
    const int L = G.grid->lmax;
    nblk_max = std::max<int64_t>(nblk_max, (int64_t)((L + kDotNT) / kDotNT) * (L + 1));
    for (int j = 0; j < G.nmaps; ++j)
      mp[G.bands[j]] = M.gradmaps.as<double>() + goff[gi] + (int64_t)j * G.grid->npix;
  }
  for (int k = 0; k < M.ncomp; ++k)
    nblk_max = std::max<int64_t>(nblk_max, (int64_t)((M.Lk[k] + kDotNT) / kDotNT) * (M.Lk[k] + 1));
  CMBWS_TRY(M.gradpart.ensure((size_t)nblk_max * M.ncomp * 8));
  double* part = M.gradpart.as<double>();
  const BandDev bd = M.bands_dev(ap);

  for (int pass = 0; pass < 2; ++pass) {
    // pass 0: u = Y^T (N^-1 d + N^-1/2 w1 - N^-1 P x), dotted with lambda
    // pass 1: v = Y^T N^-1 P lambda, dotted with x (subtracted)
    const double* a = pass == 0 ? x : lam;
    CMBWS_TRY(M.project(a, mp.data(), ap, s));
    for (size_t gi = 0; gi < M.groups.size(); ++gi) {
      Group& G = M.groups[gi];
      const Grid& g = *G.grid;
      for (int j = 0; j < G.nmaps; ++j) {
        const int nu = G.bands[j];
        ProfScope ps(PROF_HARM, s, 1);
        k_grad_pixels<<<(unsigned)((g.npix + 255) / 256), 256, 0, s>>>(
            pass == 0 ? d[nu] : nullptr, pass == 0 && w1 ? w1[nu] : nullptr,
            M.pixA64[nu].as<double>(), M.tausq[nu].as<double>(), mp[nu], g.npix, pass == 0);
        CMBWS_LAUNCH_CHECK();
      }
      CMBWS_TRY(ringfft_analysis(g, ap, G.nmaps, M.gradmaps.as<double>() + goff[gi], 0, G.F.p,
                                 M.part.p, s));
      CMBWS_TRY(legendre_adjoint(g, ap, G.nmaps, G.F.p, M.part.p, M.part.bytes, G.out.as<double>(), s));
    }
    M.n_sht += M.nobs;
    const double* other = pass == 0 ? lam : x;
    if (out)
      for (int nu = 0; nu < M.nobs; ++nu) {
        const int Ln = bd.L[nu];
        dim3 grd((Ln + kDotNT) / kDotNT, Ln + 1);
        ProfScope ps(PROF_HARM, s, 1);
        k_grad_dot<<<grd, kDotNT, 0, s>>>(h, bd.out[nu], Ln, M.d_beam.as<double>() + M.beam_off_h[nu],
                                          other, part);
        CMBWS_LAUNCH_CHECK();
        k_grad_finish<<<M.ncomp, 256, 0, s>>>(part, (int64_t)grd.x * grd.y, M.ncomp, M.ncomp,
                                              pass == 0 ? 1.0 : -1.0, pass, out + nu * M.ncomp);
        CMBWS_LAUNCH_CHECK();
      }
    // variable pairs: w (Y other_k) (Y B_nu u_nu), added (pass 0) or subtracted (pass 1); after
    // the last pass each map is final, its sum replaces the scalar formula's entry
    for (size_t gi = 0; gi < M.mgroups.size(); ++gi) {
      Group& G = M.mgroups[gi];
      const Grid& g = *G.grid;
      double* ma = M.gradmix.as<double>();
      double* mb = ma + scratch;
      CMBWS_TRY(M.mixvar_maps_comp(G, ap, other, ma, s));
      CMBWS_TRY(M.mixvar_maps_band(G, ap, mb, s));
      ProfScope ps(PROF_HARM, s, 1);
      k_grad_mixmap<<<dim3(g.nring, G.nmaps), 256, 0, s>>>(
          ma, mb, g.ring_off.as<int64_t>(), g.ring_w64.as<double>(), g.npix, g.nring,
          pass == 0 ? 1.0 : -1.0, pass, M.gradmixout.as<double>() + moff[gi], M.gradmixpart.as<double>());
      CMBWS_LAUNCH_CHECK();
      if (pass == 0) continue;
      if (out) {
        MixOut mo{};
        for (int j = 0; j < G.nmaps; ++j) mo.idx[j] = G.bands[j];  // pair id nu ncomp + k
        k_grad_mixsum<<<G.nmaps, 256, 0, s>>>(M.gradmixpart.as<double>(), g.nring, mo, out);
        CMBWS_LAUNCH_CHECK();
      }
      if (maps)
        for (int j = 0; j < G.nmaps; ++j)
          if (maps[G.bands[j]])
            CMBWS_CUDA(cudaMemcpyAsync(maps[G.bands[j]],
                                       M.gradmixout.as<double>() + moff[gi] + (int64_t)j * g.npix,
                                       (size_t)g.npix * 8, cudaMemcpyDeviceToDevice, s));
    }
  }
  if (!out) return CMBWS_OK;
  for (int k = 0; k < M.ncomp; ++k) {
    dim3 grd((M.Lk[k] + kDotNT) / kDotNT, M.Lk[k] + 1);
    ProfScope ps(PROF_HARM, s, 1);
    k_grad_prior<<<grd, kDotNT, 0, s>>>(h, k, lam, x, w2, part);
    CMBWS_LAUNCH_CHECK();
    k_grad_finish<<<1, 256, 0, s>>>(part, (int64_t)grd.x * grd.y, 1, 1, 1.0, 0,
                                    out + M.nobs * M.ncomp + k);
    CMBWS_LAUNCH_CHECK();
  }
  return CMBWS_OK;
}

}  // namespace cmbws

using namespace cmbws;

extern "C" int cmbws_grad_terms(cmbws_model mh, const double* x, const double* lambda,
                                const double* const* d, const double* const* omega1,
                                const double* omega2, double* out, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (refuse_sharded(M, "cmbws_grad_terms")) return CMBWS_ERR_ARG;
  if (!M || !x || !lambda || !d || !out) {
    set_error("cmbws_grad_terms: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  for (int nu = 0; nu < M->nobs; ++nu)
    if (!d[nu] || (omega1 && !omega1[nu])) {
      set_error("cmbws_grad_terms: missing map for band %d", nu);
      return CMBWS_ERR_ARG;
    }
  return grad_run(*M, x, lambda, d, omega1, omega2, out, nullptr, (cudaStream_t)stream);
}

extern "C" int cmbws_grad_mix_maps(cmbws_model mh, const double* x, const double* lambda,
                                   const double* const* d, const double* const* omega1,
                                   double* const* out, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (refuse_sharded(M, "cmbws_grad_mix_maps")) return CMBWS_ERR_ARG;
  if (!M || !x || !lambda || !d || !out) {
    set_error("cmbws_grad_mix_maps: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  for (int nu = 0; nu < M->nobs; ++nu)
    if (!d[nu] || (omega1 && !omega1[nu])) {
      set_error("cmbws_grad_mix_maps: missing map for band %d", nu);
      return CMBWS_ERR_ARG;
    }
  if (!M->nmix) {
    set_error("cmbws_grad_mix_maps: the model has no spatially variable mixing");
    return CMBWS_ERR_ARG;
  }
  return grad_run(*M, x, lambda, d, omega1, nullptr, nullptr, out, (cudaStream_t)stream);
}
