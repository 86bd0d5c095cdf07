// The CR system A = S^-1 + P^T N^-1 P (Eq. A) and the pseudo-inverse
// preconditioner M_PI = U^+ T^+ (U^+)^T (Eq. fullmodel-preconditioner).
//
// apply_A, per grid group (the bands that share one grid handle, NM maps):
//   harmonic prologue   a_nu = B_nu sum_k q_{nu,k} x_k   (P = Y B Q~ with Q~ = q I, Eq. P)
//   Legendre synthesis  -> ring spectra
//   ring FFT, fused     synthesis, pixel multiply by tau_nu (N^-1), analysis transpose
//   Legendre adjoint    -> u_nu = Y^T N^-1 Y a_nu
// and one harmonic epilogue over all bands:  y_k = C_k^-1 x_k + sum_nu q_{nu,k} B_nu u_nu.
//
// apply_precond:
//   t = (U^+)^T r per (l, m)  -> band rows (fed to the SHT chain) and prior rows
//   band rows: T^+_nu = alpha_nu^2 Y^T W N W Y, the same chain with pixel factor
//   alpha^2 w^2 / tau (Sec. 3.3); prior rows: identity
//   z = U^+ t' per (l, m).
// U^+ is built on the host per l (one-sided Jacobi SVD of the (Nobs+Ncomp) x Ncomp
// block, Sec. 3.1; blocks do not depend on m, Eqs. U-data and U-prior).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>

#include "model.h"

namespace cmbws {

namespace {

template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };

// ---- harmonic prologue: a_nu = c_lm * b_{nu,l} * sum_k q_{nu,k} x_k(l, m) ----
template <typename T2>
__global__ void k_mix_forward(HarmDev h, GroupDev gd, const double* __restrict__ x) {
  const int L = gd.L;
  int m, l;
  if (!tri_lm(L, m, l)) return;
  const int64_t i = lm_off(L, m) + (l - m);
  const double cc = gd.c[i];
  // per-component values in registers: loops over kMaxComp unrolled (static indices), cut
  // at ncomp
  double xr[kMaxComp], xi[kMaxComp];
#pragma unroll
  for (int k = 0; k < kMaxComp; ++k) {
    xr[k] = xi[k] = 0.0;
    if (k >= h.ncomp) continue;
    const int Lk = h.compL[k];
    if (l <= Lk) {
      const double* xk = x + h.compOff[k] + packed_off(Lk, m);
      xr[k] = xk[l - m];
      xi[k] = m > 0 ? xk[(Lk - m + 1) + (l - m)] : 0.0;
    }
  }
  for (int j = 0; j < gd.nmaps; ++j) {
    const int nu = gd.bands[j];
    double ar = 0.0, ai = 0.0;
#pragma unroll
    for (int k = 0; k < kMaxComp; ++k) {
      if (k >= h.ncomp) break;
      const PairDev& pd = h.pairs[nu * h.ncomp + k];
      if (pd.var) {
        // Q~ x_k from the mixing chain (its output band-limit covers l <= L_nu)
        const double2 t = pd.out[lm_off(pd.L, m) + (l - m)];
        ar += t.x;
        ai += t.y;
        continue;
      }
      const double q = h.q[nu * h.ncomp + k];
      ar += q * xr[k];
      ai += q * xi[k];
    }
    const double b = h.beam[h.beamOff[nu] + l] * cc;
    T2 v;
    v.x = (decltype(v.x))(b * ar);
    v.y = (decltype(v.y))(b * ai);
    reinterpret_cast<T2*>(gd.alm)[(int64_t)j * gd.nlm + i] = v;
  }
}

// ---- harmonic epilogue: y_k = C_k^-1 x_k + sum_nu q_{nu,k} b_{nu,l} u_nu ----
__global__ void k_mix_adjoint(HarmDev h, BandDev bd, int k, const double* __restrict__ x,
                              double* __restrict__ y) {
  const int Lk = h.compL[k];
  int m, l;
  if (!tri_lm(Lk, m, l)) return;
  double yr = 0.0, yi = 0.0;
  for (int nu = 0; nu < h.nobs; ++nu) {
    if (!((h.own >> nu) & 1)) continue;  // another shard's band
    const PairDev& pd = h.pairs[nu * h.ncomp + k];
    if (pd.var) {
      // Q~^T B u_nu from the transposed mixing chain (covers l <= L_k)
      const double2 t = pd.out[lm_off(pd.L, m) + (l - m)];
      yr += t.x;
      yi += t.y;
      continue;
    }
    const int Ln = bd.L[nu];
    if (l > Ln) continue;
    const double2 u = bd.out[nu][lm_off(Ln, m) + (l - m)];
    const double w = h.q[nu * h.ncomp + k] * h.beam[h.beamOff[nu] + l];
    yr += w * u.x;
    yi += w * u.y;
  }
  const int64_t base = h.compOff[k] + packed_off(Lk, m);
  const bool pr = x && h.prior_on;
  const double ci = pr ? h.cinv[h.clOff[k] + l] : 0.0;
  y[base + (l - m)] = yr + (pr ? ci * x[base + (l - m)] : 0.0);
  if (m > 0) {
    const int64_t is = base + (Lk - m + 1) + (l - m);
    y[is] = yi + (pr ? ci * x[is] : 0.0);
  }
}

// ---- inputs of the variable-mixing chains (Eq. Q) ----
// forward: slot j of mixing group mg <- c_lm x_{k_j}(l, m), zero-padded above L_k
template <typename T2>
__global__ void k_mixvar_fwd_in(HarmDev h, MixGroupDev mg, const double* __restrict__ x) {
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  const int L = mg.L;
  if (l > L) return;
  const int64_t i = lm_off(L, m) + (l - m);
  const double cc = mg.c[i];
  for (int j = 0; j < mg.npairs; ++j) {
    const int k = mg.k[j];
    const int Lk = h.compL[k];
    double vr = 0.0, vi = 0.0;
    if (l <= Lk) {
      const double* xk = x + h.compOff[k] + packed_off(Lk, m);
      vr = xk[l - m];
      vi = m > 0 ? xk[(Lk - m + 1) + (l - m)] : 0.0;
    }
    T2 v;
    v.x = (decltype(v.x))(cc * vr);
    v.y = (decltype(v.y))(cc * vi);
    reinterpret_cast<T2*>(mg.alm)[(int64_t)j * mg.nlm + i] = v;
  }
}

// transposed: slot j <- c_lm b_{nu_j, l} u_{nu_j}(l, m), zero-padded above L_nu
template <typename T2>
__global__ void k_mixvar_adj_in(HarmDev h, BandDev bd, MixGroupDev mg) {
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  const int L = mg.L;
  if (l > L) return;
  const int64_t i = lm_off(L, m) + (l - m);
  const double cc = mg.c[i];
  for (int j = 0; j < mg.npairs; ++j) {
    const int nu = mg.nu[j];
    const int Ln = bd.L[nu];
    double vr = 0.0, vi = 0.0;
    if (l <= Ln) {
      const double2 u = bd.out[nu][lm_off(Ln, m) + (l - m)];
      const double b = h.beam[h.beamOff[nu] + l];
      vr = b * u.x;
      vi = b * u.y;
    }
    T2 v;
    v.x = (decltype(v.x))(cc * vr);
    v.y = (decltype(v.y))(cc * vi);
    reinterpret_cast<T2*>(mg.alm)[(int64_t)j * mg.nlm + i] = v;
  }
}

// per-ring sums of q and q^2 (unweighted, Eq. optimal-q) and the pixel factor q w
__global__ void k_mixq(const double* __restrict__ q, const int64_t* __restrict__ roff,
                       const double* __restrict__ rw, double* __restrict__ f64, float* __restrict__ f32,
                       double2* __restrict__ sums) {
  const int r = blockIdx.x;
  const int64_t b = roff[r], e = roff[r + 1];
  const double w = rw[r];
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
    const double v = q[i];
    s1 += v;
    s2 += v * v;
    f64[i] = v * w;
    f32[i] = (float)(v * w);
  }
  __shared__ double a1[256], a2[256];
  a1[threadIdx.x] = s1;
  a2[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      a1[threadIdx.x] += a1[threadIdx.x + o];
      a2[threadIdx.x] += a2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) sums[r] = make_double2(a1[0], a2[0]);
}

// ---- t = (U^+)^T r: band rows into the group inputs (times c_lm), prior rows into tp ----
template <typename T2>
__global__ void k_pinv_T(HarmDev h, BandDev bd, const double* __restrict__ r,
                         double* __restrict__ tp, int Ltop) {
  int m, l;
  if (!tri_lm(Ltop, m, l)) return;
  const int nc = h.ncomp, nr = h.nobs + h.ncomp;
  // per-component values in registers (unrolled over kMaxComp, cut at nc)
  double rr[kMaxComp], ri[kMaxComp];
#pragma unroll
  for (int k = 0; k < kMaxComp; ++k) {
    rr[k] = ri[k] = 0.0;
    if (k >= nc) continue;
    const int Lk = h.compL[k];
    if (l <= Lk) {
      const double* rk = r + h.compOff[k] + packed_off(Lk, m);
      rr[k] = rk[l - m];
      ri[k] = m > 0 ? rk[(Lk - m + 1) + (l - m)] : 0.0;
    }
  }
  const double* U = h.Up + (int64_t)min(l, h.Lup) * nc * nr;  // U^+[c][j]
  const bool inU = l <= h.Lup;
  for (int nu = 0; nu < h.nobs; ++nu) {
    const int Ln = bd.L[nu];
    if (l > Ln) continue;
    double tr = 0.0, ti = 0.0;
    if (inU) {
#pragma unroll
      for (int c = 0; c < kMaxComp; ++c) {
        if (c >= nc) break;
        const double u = U[c * nr + nu];
        tr += u * rr[c];
        ti += u * ri[c];
      }
    }
    const int64_t i = lm_off(Ln, m) + (l - m);
    const double cc = bd.c[nu][i];
    T2 v;
    v.x = (decltype(v.x))(cc * tr);
    v.y = (decltype(v.y))(cc * ti);
    reinterpret_cast<T2*>(bd.alm[nu])[i] = v;
  }
  for (int k = 0; k < nc; ++k) {
    const int Lk = h.compL[k];
    if (l > Lk) continue;
    double tr = 0.0, ti = 0.0;
    if (inU) {
#pragma unroll
      for (int c = 0; c < kMaxComp; ++c) {
        if (c >= nc) break;
        const double u = U[c * nr + h.nobs + k];
        tr += u * rr[c];
        ti += u * ri[c];
      }
    }
    const int64_t base = h.compOff[k] + packed_off(Lk, m);
    tp[base + (l - m)] = tr;
    if (m > 0) tp[base + (Lk - m + 1) + (l - m)] = ti;
  }
}

// ---- z = U^+ t' ----
__global__ void k_pinv(HarmDev h, BandDev bd, const double* __restrict__ tp, double* __restrict__ z,
                       int Lcomp) {
  int m, l;
  if (!tri_lm(Lcomp, m, l)) return;
  const int nc = h.ncomp, nr = h.nobs + h.ncomp;
  const double* U = h.Up + (int64_t)min(l, h.Lup) * nc * nr;
  // per-component sums in registers (unrolled over kMaxComp, cut at nc)
  double zr[kMaxComp], zi[kMaxComp];
#pragma unroll
  for (int c = 0; c < kMaxComp; ++c) zr[c] = zi[c] = 0.0;
  for (int nu = 0; nu < h.nobs; ++nu) {
    const int Ln = bd.L[nu];
    if (l > Ln || !((h.own >> nu) & 1)) continue;
    const double2 u = bd.out[nu][lm_off(Ln, m) + (l - m)];
#pragma unroll
    for (int c = 0; c < kMaxComp; ++c) {
      if (c >= nc) break;
      const double w = U[c * nr + nu];
      zr[c] += w * u.x;
      zi[c] += w * u.y;
    }
  }
  for (int k = 0; k < nc; ++k) {
    const int Lk = h.compL[k];
    if (l > Lk || !h.prior_on) continue;
    const int64_t base = h.compOff[k] + packed_off(Lk, m);
    const double tr = tp[base + (l - m)];
    const double ti = m > 0 ? tp[base + (Lk - m + 1) + (l - m)] : 0.0;
#pragma unroll
    for (int c = 0; c < kMaxComp; ++c) {
      if (c >= nc) break;
      const double w = U[c * nr + h.nobs + k];
      zr[c] += w * tr;
      zi[c] += w * ti;
    }
  }
#pragma unroll
  for (int c = 0; c < kMaxComp; ++c) {
    if (c >= nc) break;
    const int Lc = h.compL[c];
    if (l > Lc) continue;
    const int64_t base = h.compOff[c] + packed_off(Lc, m);
    z[base + (l - m)] = zr[c];
    if (m > 0) z[base + (Lc - m + 1) + (l - m)] = zi[c];
  }
}

// ---- pixel factors and alpha ----
__global__ void k_ring_sums(const double* __restrict__ tau, const int64_t* __restrict__ roff,
                            const double* __restrict__ rw, double2* __restrict__ out) {
  const int r = blockIdx.x;
  const int64_t b = roff[r], e = roff[r + 1];
  const double w = rw[r];
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
    const double v = tau[i] / w;
    s1 += v;
    s2 += v * v;
  }
  __shared__ double a1[256], a2[256];
  a1[threadIdx.x] = s1;
  a2[threadIdx.x] = s2;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if ((int)threadIdx.x < o) {
      a1[threadIdx.x] += a1[threadIdx.x + o];
      a2[threadIdx.x] += a2[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) out[r] = make_double2(a1[0], a2[0]);
}

__global__ void k_pixel_factors(const double* __restrict__ tau, const int64_t* __restrict__ roff,
                                const double* __restrict__ rw, double alpha2, double* pA64,
                                float* pA32, double* pM64, float* pM32, double* tau_sqrt) {
  const int r = blockIdx.x;
  const int64_t b = roff[r], e = roff[r + 1];
  const double w = rw[r];
  for (int64_t i = b + threadIdx.x; i < e; i += blockDim.x) {
    const double t = tau[i];
    const double f = alpha2 * w * w / t;
    pA64[i] = t;
    pA32[i] = (float)t;
    pM64[i] = f;
    pM32[i] = (float)f;
    tau_sqrt[i] = sqrt(t);
  }
}

// pixel maps for the RHS: d * tau + omega1 * sqrt(tau)
__global__ void k_rhs_pixels(const double* __restrict__ d, const double* __restrict__ w1,
                             const double* __restrict__ tau, const double* __restrict__ tsq,
                             double* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = d[i] * tau[i];
  if (w1) v += w1[i] * tsq[i];
  out[i] = v;
}

__global__ void k_add_scaled_prior(HarmDev h, const double* __restrict__ w2, double* __restrict__ b,
                                   int k) {
  const int Lk = h.compL[k];
  int m, l;
  if (!tri_lm(Lk, m, l) || !h.prior_on) return;  // the prior terms belong to one shard
  const int64_t base = h.compOff[k] + packed_off(Lk, m);
  const double s = h.cisq[h.clOff[k] + l];
  b[base + (l - m)] += s * w2[base + (l - m)];
  if (m > 0) b[base + (Lk - m + 1) + (l - m)] += s * w2[base + (Lk - m + 1) + (l - m)];
}


}  // namespace

// One-sided Jacobi SVD pseudo-inverse of an (nr x nc) matrix U (row-major), out (nc x nr).
// Returns false if a column of U is zero.
bool pinv_jacobi(const std::vector<double>& Uin, int nr, int nc, double rcond,
                 std::vector<double>& out) {
  std::vector<double> A(Uin), V(nc * nc, 0.0);
  for (int i = 0; i < nc; ++i) V[i * nc + i] = 1.0;
  for (int j = 0; j < nc; ++j) {
    double s = 0.0;
    for (int i = 0; i < nr; ++i) s += A[i * nc + j] * A[i * nc + j];
    if (s == 0.0) return false;
  }
  for (int sweep = 0; sweep < 60; ++sweep) {
    double off = 0.0;
    for (int p = 0; p < nc; ++p)
      for (int q = p + 1; q < nc; ++q) {
        double a = 0, b = 0, g = 0;
        for (int i = 0; i < nr; ++i) {
          a += A[i * nc + p] * A[i * nc + p];
          b += A[i * nc + q] * A[i * nc + q];
          g += A[i * nc + p] * A[i * nc + q];
        }
        if (g == 0.0) continue;
        const double rel = std::fabs(g) / std::sqrt(a * b);
        off = std::max(off, rel);
        if (rel < 1e-17) continue;
        const double zeta = (b - a) / (2.0 * g);
        const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
        for (int i = 0; i < nr; ++i) {
          const double ap = A[i * nc + p], aq = A[i * nc + q];
          A[i * nc + p] = c * ap - s * aq;
          A[i * nc + q] = s * ap + c * aq;
        }
        for (int i = 0; i < nc; ++i) {
          const double vp = V[i * nc + p], vq = V[i * nc + q];
          V[i * nc + p] = c * vp - s * vq;
          V[i * nc + q] = s * vp + c * vq;
        }
      }
    if (off < 1e-15) break;
  }
  std::vector<double> sig(nc);
  double smax = 0.0;
  for (int j = 0; j < nc; ++j) {
    double s = 0.0;
    for (int i = 0; i < nr; ++i) s += A[i * nc + j] * A[i * nc + j];
    sig[j] = std::sqrt(s);
    smax = std::max(smax, sig[j]);
  }
  out.assign((size_t)nc * nr, 0.0);
  for (int j = 0; j < nc; ++j) {
    if (sig[j] <= rcond * smax || sig[j] == 0.0) continue;
    const double inv2 = 1.0 / (sig[j] * sig[j]);  // W_j = A_j / sig_j, term V_j W_j^T / sig_j
    for (int c = 0; c < nc; ++c) {
      const double v = V[c * nc + j] * inv2;
      if (v == 0.0) continue;
      for (int i = 0; i < nr; ++i) out[(size_t)c * nr + i] += v * A[i * nc + j];
    }
  }
  return true;
}


// ---- the chain of one grid group: synthesis -> fused FFT/pixel multiply -> adjoint ----
int Model::group_chain(Group& G, int prec, int which, cudaStream_t s) {
  const Grid& g = *G.grid;
  const void* pix[kMaxMaps];
  for (int j = 0; j < G.nmaps; ++j) {
    const int nu = G.bands[j];
    pix[j] = which == 0 ? (!is_f32(prec) ? pixA64[nu].p : pixA32[nu].p)
                        : (!is_f32(prec) ? pixM64[nu].p : pixM32[nu].p);
  }
  CMBWS_TRY(legendre_synth(g, prec, G.nmaps, G.alm.p, G.F.p, s));
  CMBWS_TRY(ringfft_fused(g, prec, G.nmaps, G.F.p, pix, part.p, s));
  CMBWS_TRY(legendre_adjoint(g, prec, G.nmaps, G.F.p, part.p, part.bytes, G.out.as<double>(), s));
  return CMBWS_OK;
}

HarmDev Model::harm() const {
  HarmDev h{};
  h.ncomp = ncomp;
  h.nobs = nobs;
  h.compL = d_compL.as<int>();
  h.compOff = d_compOff.as<int64_t>();
  h.q = d_q.as<double>();
  h.beam = d_beam.as<double>();
  h.beamOff = d_beamOff.as<int64_t>();
  h.cinv = d_cinv.as<double>();
  h.cisq = d_cisq.as<double>();
  h.clOff = d_clOff.as<int64_t>();
  h.Up = d_Up.as<double>();
  h.Lup = Lup;
  h.pairs = d_pairs.as<PairDev>();
  h.own = shard_own;
  h.prior_on = shard_prior ? 1 : 0;
  return h;
}

BandDev Model::bands_dev(int prec) const {
  BandDev b{};
  for (int nu = 0; nu < nobs; ++nu) {
    const Group& G = groups[band_group[nu]];
    const int j = band_slot[nu];
    const int64_t nlm = nlm_of(G.grid->lmax);
    b.L[nu] = G.grid->lmax;
    b.out[nu] = G.out.as<double2>() + j * nlm;
    b.c[nu] = G.grid->c64.as<double>();
    b.alm[nu] = (char*)G.alm.p + (size_t)j * nlm * 2 * prec_size(prec);
  }
  return b;
}

int Model::mix_chain(Group& G, int prec, cudaStream_t s) {
  const Grid& g = *G.grid;
  const void* pix[kMaxMaps];
  for (int j = 0; j < G.nmaps; ++j) pix[j] = !is_f32(prec) ? pixQ64[G.bands[j]].p : pixQ32[G.bands[j]].p;
  CMBWS_TRY(legendre_synth(g, prec, G.nmaps, G.alm.p, G.F.p, s));
  CMBWS_TRY(ringfft_fused(g, prec, G.nmaps, G.F.p, pix, part.p, s));
  CMBWS_TRY(legendre_adjoint(g, prec, G.nmaps, G.F.p, part.p, part.bytes, G.out.as<double>(), s));
  return CMBWS_OK;
}

static MixGroupDev mix_dev(const Group& G, int ncomp) {
  MixGroupDev mg{};
  mg.L = G.grid->lmax;
  mg.npairs = G.nmaps;
  for (int j = 0; j < G.nmaps; ++j) {
    mg.nu[j] = G.bands[j] / ncomp;
    mg.k[j] = G.bands[j] % ncomp;
  }
  mg.c = G.grid->c64.as<double>();
  mg.alm = G.alm.p;
  mg.nlm = nlm_of(mg.L);
  return mg;
}

// t_{nu,k} = Q~_{nu,k} x_k for every variable pair
int Model::mixvar_forward(int prec, const double* x, cudaStream_t s) {
  const HarmDev h = harm();
  for (Group& G : mgroups) {
    const MixGroupDev mg = mix_dev(G, ncomp);
    dim3 grd((mg.L + 1 + 127) / 128, mg.L + 1);
    {
      ProfScope ps(PROF_HARM, s, is_f32(prec) ? 0 : 1);
      if (!is_f32(prec)) k_mixvar_fwd_in<double2><<<grd, 128, 0, s>>>(h, mg, x);
      else k_mixvar_fwd_in<float2><<<grd, 128, 0, s>>>(h, mg, x);
      CMBWS_LAUNCH_CHECK();
    }
    CMBWS_TRY(mix_chain(G, prec, s));
  }
  return CMBWS_OK;
}

// s_{nu,k} = Q~_{nu,k}^T B_nu u_nu for every variable pair (u_nu in the band outputs)
int Model::mixvar_adjoint(int prec, cudaStream_t s) {
  const HarmDev h = harm();
  const BandDev bd = bands_dev(prec);
  for (Group& G : mgroups) {
    const MixGroupDev mg = mix_dev(G, ncomp);
    dim3 grd((mg.L + 1 + 127) / 128, mg.L + 1);
    {
      ProfScope ps(PROF_HARM, s, is_f32(prec) ? 0 : 1);
      if (!is_f32(prec)) k_mixvar_adj_in<double2><<<grd, 128, 0, s>>>(h, bd, mg);
      else k_mixvar_adj_in<float2><<<grd, 128, 0, s>>>(h, bd, mg);
      CMBWS_LAUNCH_CHECK();
    }
    CMBWS_TRY(mix_chain(G, prec, s));
  }
  return CMBWS_OK;
}

int Model::mixvar_maps_comp(Group& G, int prec, const double* x, double* maps, cudaStream_t s) {
  const HarmDev h = harm();
  const MixGroupDev mg = mix_dev(G, ncomp);
  dim3 grd((mg.L + 1 + 127) / 128, mg.L + 1);
  {
    ProfScope ps(PROF_HARM, s, is_f32(prec) ? 0 : 1);
    if (!is_f32(prec)) k_mixvar_fwd_in<double2><<<grd, 128, 0, s>>>(h, mg, x);
    else k_mixvar_fwd_in<float2><<<grd, 128, 0, s>>>(h, mg, x);
    CMBWS_LAUNCH_CHECK();
  }
  CMBWS_TRY(legendre_synth(*G.grid, prec, G.nmaps, G.alm.p, G.F.p, s));
  CMBWS_TRY(ringfft_synth(*G.grid, prec, G.nmaps, G.F.p, maps, s));
  n_sht += G.nmaps;
  return CMBWS_OK;
}

int Model::mixvar_maps_band(Group& G, int prec, double* maps, cudaStream_t s) {
  const HarmDev h = harm();
  const BandDev bd = bands_dev(prec);
  const MixGroupDev mg = mix_dev(G, ncomp);
  dim3 grd((mg.L + 1 + 127) / 128, mg.L + 1);
  {
    ProfScope ps(PROF_HARM, s, is_f32(prec) ? 0 : 1);
    if (!is_f32(prec)) k_mixvar_adj_in<double2><<<grd, 128, 0, s>>>(h, bd, mg);
    else k_mixvar_adj_in<float2><<<grd, 128, 0, s>>>(h, bd, mg);
    CMBWS_LAUNCH_CHECK();
  }
  CMBWS_TRY(legendre_synth(*G.grid, prec, G.nmaps, G.alm.p, G.F.p, s));
  CMBWS_TRY(ringfft_synth(*G.grid, prec, G.nmaps, G.F.p, maps, s));
  n_sht += G.nmaps;
  return CMBWS_OK;
}

int Model::mix_forward(Group& G, int prec, const double* x, cudaStream_t s) {
  const HarmDev h = harm();
  GroupDev gd{};
  gd.L = G.grid->lmax;
  gd.nmaps = G.nmaps;
  for (int j = 0; j < G.nmaps; ++j) gd.bands[j] = G.bands[j];
  gd.c = G.grid->c64.as<double>();
  gd.alm = G.alm.p;
  gd.nlm = nlm_of(gd.L);
  const dim3 grd = tri_grid(gd.L, 128);
  ProfScope ps(PROF_HARM, s, is_f32(prec) ? 0 : 1);
  if (!is_f32(prec)) k_mix_forward<double2><<<grd, 128, 0, s>>>(h, gd, x);
  else k_mix_forward<float2><<<grd, 128, 0, s>>>(h, gd, x);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

int Model::project(const double* x, double* const* d, int prec, cudaStream_t s) {
  if (nmix) CMBWS_TRY(mixvar_forward(prec, x, s));
  for (Group& G : groups) {
    const Grid& g = *G.grid;
    CMBWS_TRY(pixtmp.ensure((size_t)G.nmaps * g.npix * 8));
    CMBWS_TRY(mix_forward(G, prec, x, s));
    CMBWS_TRY(legendre_synth(g, prec, G.nmaps, G.alm.p, G.F.p, s));
    CMBWS_TRY(ringfft_synth(g, prec, G.nmaps, G.F.p, pixtmp.as<double>(), s));
    for (int j = 0; j < G.nmaps; ++j)
      CMBWS_CUDA(cudaMemcpyAsync(d[G.bands[j]], pixtmp.as<double>() + (size_t)j * g.npix,
                                 (size_t)g.npix * 8, cudaMemcpyDeviceToDevice, s));
  }
  n_sht += nobs + 2 * nmix;
  return CMBWS_OK;
}

int Model::apply_A(const double* x, double* y, int prec, cudaStream_t s) {
  const HarmDev h = harm();
  if (nmix) CMBWS_TRY(mixvar_forward(prec, x, s));
  for (Group& G : groups) {
    if (!group_owned(G)) continue;  // another shard's bands
    CMBWS_TRY(mix_forward(G, prec, x, s));
    CMBWS_TRY(group_chain(G, prec, 0, s));
  }
  if (nmix) CMBWS_TRY(mixvar_adjoint(prec, s));
  const BandDev bd = bands_dev(prec);
  for (int k = 0; k < ncomp; ++k) {
    const dim3 grd = tri_grid(Lk[k], 128);
    ProfScope ps(PROF_HARM, s, is_f32(prec) ? 0 : 1);
    k_mix_adjoint<<<grd, 128, 0, s>>>(h, bd, k, x, y);
    CMBWS_LAUNCH_CHECK();
  }
  n_sht += nsht_A;
  return CMBWS_OK;
}

int Model::apply_precond_merged(const double* r, double* z, int prec, cudaStream_t s) {
  MergedPrec& P = *merged;
  HarmDev h = harm();
  h.nobs = P.nrow;  // rows of U' in place of the bands
  h.Up = P.d_Up.as<double>();
  BandDev bd{};
  for (int row = 0; row < P.nrow; ++row) {
    const Group& G = P.groups[P.row_group[row]];
    const int j = P.row_slot[row];
    const int64_t nlm = nlm_of(G.grid->lmax);
    bd.L[row] = G.grid->lmax;
    bd.out[row] = G.out.as<double2>() + j * nlm;
    bd.c[row] = G.grid->c64.as<double>();
    bd.alm[row] = (char*)G.alm.p + (size_t)j * nlm * 2 * prec_size(prec);
  }
  {
    const dim3 grd = tri_grid(Lall, 128);
    ProfScope ps(PROF_HARM, s, is_f32(prec) ? 0 : 1);
    if (!is_f32(prec)) k_pinv_T<double2><<<grd, 128, 0, s>>>(h, bd, r, tprior.as<double>(), Lall);
    else k_pinv_T<float2><<<grd, 128, 0, s>>>(h, bd, r, tprior.as<double>(), Lall);
    CMBWS_LAUNCH_CHECK();
  }
  for (Group& G : P.groups) {
    const Grid& g = *G.grid;
    const void* pix[kMaxMaps];
    for (int j = 0; j < G.nmaps; ++j)
      pix[j] = !is_f32(prec) ? P.pixM64[G.bands[j]].p : P.pixM32[G.bands[j]].p;
    CMBWS_TRY(legendre_synth(g, prec, G.nmaps, G.alm.p, G.F.p, s));
    CMBWS_TRY(ringfft_fused(g, prec, G.nmaps, G.F.p, pix, part.p, s));
    CMBWS_TRY(legendre_adjoint(g, prec, G.nmaps, G.F.p, part.p, part.bytes, G.out.as<double>(), s));
  }
  {
    const dim3 grd = tri_grid(Lcomp, 128);
    ProfScope ps(PROF_HARM, s, is_f32(prec) ? 0 : 1);
    k_pinv<<<grd, 128, 0, s>>>(h, bd, tprior.as<double>(), z, Lcomp);
    CMBWS_LAUNCH_CHECK();
  }
  n_sht += nsht_M;
  return CMBWS_OK;
}

int Model::apply_precond(const double* r, double* z, int prec, cudaStream_t s) {
  if (merged) return apply_precond_merged(r, z, prec, s);
  const HarmDev h = harm();
  const BandDev bd = bands_dev(prec);
  {
    const dim3 grd = tri_grid(Lall, 128);
    ProfScope ps(PROF_HARM, s, is_f32(prec) ? 0 : 1);
    if (!is_f32(prec)) k_pinv_T<double2><<<grd, 128, 0, s>>>(h, bd, r, tprior.as<double>(), Lall);
    else k_pinv_T<float2><<<grd, 128, 0, s>>>(h, bd, r, tprior.as<double>(), Lall);
    CMBWS_LAUNCH_CHECK();
  }
  for (Group& G : groups)
    if (group_owned(G)) CMBWS_TRY(group_chain(G, prec, 1, s));
  {
    const dim3 grd = tri_grid(Lcomp, 128);
    ProfScope ps(PROF_HARM, s, is_f32(prec) ? 0 : 1);
    k_pinv<<<grd, 128, 0, s>>>(h, bd, tprior.as<double>(), z, Lcomp);
    CMBWS_LAUNCH_CHECK();
  }
  n_sht += nsht_M;
  return CMBWS_OK;
}

int Model::rhs(const double* const* d, const double* const* w1, const double* w2, double* b,
               cudaStream_t s) {
  const HarmDev h = harm();
  const int ap = prec == CMBWS_FP64 ? CMBWS_FP64 : CMBWS_FP32X2;  // FP64-accurate either way
  // P^T applied to the pixel maps: per group, analysis FFT (unweighted) + Legendre adjoint
  for (Group& G : groups) {
    if (!group_owned(G)) continue;  // another shard's bands
    const Grid& g = *G.grid;
    CMBWS_TRY(pixtmp.ensure((size_t)G.nmaps * g.npix * 8));
    for (int j = 0; j < G.nmaps; ++j) {
      const int nu = G.bands[j];
      const int64_t n = g.npix;
      ProfScope ps(PROF_HARM, s, 1);
      k_rhs_pixels<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(
          d[nu], w1 ? w1[nu] : nullptr, pixA64[nu].as<double>(), tausq[nu].as<double>(),
          pixtmp.as<double>() + j * n, n);
      CMBWS_LAUNCH_CHECK();
    }
    CMBWS_TRY(ringfft_analysis(g, ap, G.nmaps, pixtmp.as<double>(), 0, G.F.p, part.p, s));
    CMBWS_TRY(legendre_adjoint(g, ap, G.nmaps, G.F.p, part.p, part.bytes, G.out.as<double>(), s));
  }
  // transposed variable mixing of B u_nu, then the epilogue without a prior term (x = NULL)
  if (nmix) CMBWS_TRY(mixvar_adjoint(ap, s));
  const BandDev bd = bands_dev(ap);
  for (int k = 0; k < ncomp; ++k) {
    const dim3 grd = tri_grid(Lk[k], 128);
    ProfScope ps(PROF_HARM, s, 1);
    k_mix_adjoint<<<grd, 128, 0, s>>>(h, bd, k, nullptr, b);
    CMBWS_LAUNCH_CHECK();
    if (w2) {
      ProfScope ps2(PROF_HARM, s, 1);
      k_add_scaled_prior<<<grd, 128, 0, s>>>(h, w2, b, k);
      CMBWS_LAUNCH_CHECK();
    }
  }
  n_sht += nobs + 2 * nmix;
  return CMBWS_OK;
}

int model_create(const cmbws_model_desc* desc, int prec, cudaStream_t s, Model** out) {
  const int nc = desc->ncomp, no = desc->nobs;
  if (nc < 1 || nc > kMaxComp || no < 1 || no > kMaxBands || !desc->lmax_comp || !desc->band_grid ||
      !desc->beam || !desc->cl || !desc->ninv || !desc->mix_scalar) {
    set_error("cmbws_model_create: invalid description (ncomp <= %d, nobs <= %d)", kMaxComp,
              kMaxBands);
    return CMBWS_ERR_ARG;
  }
  Model* M = new (std::nothrow) Model();
  if (!M) return CMBWS_ERR_NOMEM;
  std::unique_ptr<Model> guard(M);
  M->ncomp = nc;
  M->nobs = no;
  M->prec = prec;
  int dev = 0;
  CMBWS_CUDA(cudaGetDevice(&dev));
  M->Lk.assign(desc->lmax_comp, desc->lmax_comp + nc);
  M->compOff.assign(nc + 1, 0);
  for (int k = 0; k < nc; ++k) {
    if (M->Lk[k] < 0) {
      set_error("cmbws_model_create: negative L_k");
      return CMBWS_ERR_ARG;
    }
    M->compOff[k + 1] = M->compOff[k] + (int64_t)(M->Lk[k] + 1) * (M->Lk[k] + 1);
  }
  M->nvec = M->compOff[nc];
  M->Lcomp = *std::max_element(M->Lk.begin(), M->Lk.end());
  M->grids.resize(no);
  M->Lnu.resize(no);
  M->band_group.resize(no);
  M->band_slot.resize(no);
  for (int nu = 0; nu < no; ++nu) {
    Grid* g = as_grid(desc->band_grid[nu]);
    if (!g || g->device != dev) {
      set_error("cmbws_model_create: band %d has no grid on the current device", nu);
      return CMBWS_ERR_ARG;
    }
    if (!ringfft_smem_ok(*g, CMBWS_FP64)) {
      set_error("cmbws_model_create: band %d grid too large for FP64 ring transforms", nu);
      return CMBWS_ERR_ARG;
    }
    M->grids[nu] = g;
    M->Lnu[nu] = g->lmax;
    int gi = -1;
    for (size_t i = 0; i < M->groups.size(); ++i)
      if (M->groups[i].grid == g && M->groups[i].nmaps < kMaxMaps) gi = (int)i;
    if (gi < 0) {
      M->groups.emplace_back();
      M->groups.back().grid = g;
      gi = (int)M->groups.size() - 1;
    }
    Group& G = M->groups[gi];
    M->band_group[nu] = gi;
    M->band_slot[nu] = G.nmaps;
    G.bands[G.nmaps++] = nu;
  }
  M->Lall = std::max(M->Lcomp, *std::max_element(M->Lnu.begin(), M->Lnu.end()));

  // ---- host tables: beams, q, C^-1, C^-1/2 ----
  std::vector<double> beam, cinv, cisq, q(desc->mix_scalar, desc->mix_scalar + no * nc);
  std::vector<int64_t> beamOff(no), clOff(nc);
  for (int nu = 0; nu < no; ++nu) {
    if (!desc->beam[nu]) {
      set_error("cmbws_model_create: missing beam %d", nu);
      return CMBWS_ERR_ARG;
    }
    beamOff[nu] = (int64_t)beam.size();
    beam.insert(beam.end(), desc->beam[nu], desc->beam[nu] + M->Lnu[nu] + 1);
  }
  std::vector<std::vector<double>> cinv_k(nc);
  for (int k = 0; k < nc; ++k) {
    clOff[k] = (int64_t)cinv.size();
    cinv_k[k].assign(M->Lk[k] + 1, 0.0);
    for (int l = 0; l <= M->Lk[k]; ++l) {
      double ci = 0.0, cs = 0.0;
      if (desc->cl[k]) {
        const double c = desc->cl[k][l];
        if (std::isfinite(c) && c > 0.0) {
          ci = 1.0 / c;
          cs = 1.0 / std::sqrt(c);
        }
      }
      cinv.push_back(ci);
      cisq.push_back(cs);
      cinv_k[k][l] = cs;
    }
  }

  // ---- alpha_nu (Eq. optimal-alpha) and pixel factors ----
  M->alpha.resize(no);
  M->pixA64.resize(no);
  M->pixA32.resize(no);
  M->pixM64.resize(no);
  M->pixM32.resize(no);
  M->tausq.resize(no);
  for (int nu = 0; nu < no; ++nu) {
    const Grid& g = *M->grids[nu];
    if (!desc->ninv[nu]) {
      set_error("cmbws_model_create: missing inverse-noise map %d", nu);
      return CMBWS_ERR_ARG;
    }
    DevMem sums;
    CMBWS_TRY(sums.alloc((size_t)g.nring * 16));
    k_ring_sums<<<g.nring, 256, 0, s>>>(desc->ninv[nu], g.ring_off.as<int64_t>(),
                                        g.ring_w64.as<double>(), sums.as<double2>());
    CMBWS_LAUNCH_CHECK();
    std::vector<double> hs(2 * g.nring);
    CMBWS_CUDA(cudaMemcpyAsync(hs.data(), sums.p, hs.size() * 8, cudaMemcpyDeviceToHost, s));
    CMBWS_CUDA(cudaStreamSynchronize(s));
    double s1 = 0.0, s2 = 0.0;
    for (int r = 0; r < g.nring; ++r) {
      s1 += hs[2 * r];
      s2 += hs[2 * r + 1];
    }
    if (!(s1 > 0.0) || !std::isfinite(s2)) {
      set_error("cmbws_model_create: inverse-noise map %d is not positive and finite", nu);
      return CMBWS_ERR_ARG;
    }
    M->alpha[nu] = std::sqrt(s2 / s1);
    CMBWS_TRY(M->pixA64[nu].alloc(g.npix * 8));
    CMBWS_TRY(M->pixA32[nu].alloc(g.npix * 4));
    CMBWS_TRY(M->pixM64[nu].alloc(g.npix * 8));
    CMBWS_TRY(M->pixM32[nu].alloc(g.npix * 4));
    CMBWS_TRY(M->tausq[nu].alloc(g.npix * 8));
    k_pixel_factors<<<g.nring, 256, 0, s>>>(desc->ninv[nu], g.ring_off.as<int64_t>(),
                                            g.ring_w64.as<double>(), M->alpha[nu] * M->alpha[nu],
                                            M->pixA64[nu].as<double>(), M->pixA32[nu].as<float>(),
                                            M->pixM64[nu].as<double>(), M->pixM32[nu].as<float>(),
                                            M->tausq[nu].as<double>());
    CMBWS_LAUNCH_CHECK();
  }

  // ---- spatially variable mixing (Eq. Q) ----
  std::vector<double> qpre(q);  // scalars of the preconditioner (Eq. optimal-q for variable pairs)
  std::vector<PairDev> pairs((size_t)no * nc);
  for (auto& pd : pairs) pd = PairDev{nullptr, nullptr, nullptr, nullptr, 0, 0};
  M->pixQ64.resize((size_t)no * nc);
  M->pixQ32.resize((size_t)no * nc);
  if (desc->mix_grid && desc->mix_map) {
    for (int nu = 0; nu < no; ++nu)
      for (int k = 0; k < nc; ++k) {
        const int id = nu * nc + k;
        if (!desc->mix_map[id]) continue;
        Grid* g = as_grid(desc->mix_grid[id]);
        if (!g || g->device != dev) {
          set_error("cmbws_model_create: mixing pair (%d, %d) has no grid on this device", nu, k);
          return CMBWS_ERR_ARG;
        }
        if (g->lmax < std::max(M->Lk[k], M->Lnu[nu]) || !ringfft_smem_ok(*g, CMBWS_FP64)) {
          set_error("cmbws_model_create: mixing grid of pair (%d, %d) needs lmax >= %d", nu, k,
                    std::max(M->Lk[k], M->Lnu[nu]));
          return CMBWS_ERR_ARG;
        }
        int gi = -1;
        for (size_t i = 0; i < M->mgroups.size(); ++i)
          if (M->mgroups[i].grid == g && M->mgroups[i].nmaps < kMaxMaps) gi = (int)i;
        if (gi < 0) {
          M->mgroups.emplace_back();
          M->mgroups.back().grid = g;
          gi = (int)M->mgroups.size() - 1;
        }
        Group& G = M->mgroups[gi];
        G.bands[G.nmaps++] = id;
        CMBWS_TRY(M->pixQ64[id].alloc(g->npix * 8));
        CMBWS_TRY(M->pixQ32[id].alloc(g->npix * 4));
        DevMem sums;
        CMBWS_TRY(sums.alloc((size_t)g->nring * 16));
        k_mixq<<<g->nring, 256, 0, s>>>(desc->mix_map[id], g->ring_off.as<int64_t>(),
                                         g->ring_w64.as<double>(), M->pixQ64[id].as<double>(),
                                         M->pixQ32[id].as<float>(), sums.as<double2>());
        CMBWS_LAUNCH_CHECK();
        std::vector<double> hs(2 * g->nring);
        CMBWS_CUDA(cudaMemcpyAsync(hs.data(), sums.p, hs.size() * 8, cudaMemcpyDeviceToHost, s));
        CMBWS_CUDA(cudaStreamSynchronize(s));
        double s1 = 0.0, s2 = 0.0;
        for (int r = 0; r < g->nring; ++r) {
          s1 += hs[2 * r];
          s2 += hs[2 * r + 1];
        }
        if (!(s1 != 0.0) || !std::isfinite(s2)) {
          set_error("cmbws_model_create: mixing map of pair (%d, %d) sums to zero", nu, k);
          return CMBWS_ERR_ARG;
        }
        qpre[id] = s2 / s1;  // Eq. optimal-q
        M->nmix += 1;
      }
  }
  for (Group& G : M->mgroups) {
    const Grid& g = *G.grid;
    const int64_t nlm = nlm_of(g.lmax);
    CMBWS_TRY(G.alm.alloc((size_t)G.nmaps * nlm * 16));
    CMBWS_TRY(G.F.alloc((size_t)G.nmaps * g.nring * (g.lmax + 1) * 16));
    CMBWS_TRY(G.out.alloc((size_t)G.nmaps * nlm * 16));
    for (int j = 0; j < G.nmaps; ++j) {
      PairDev& pd = pairs[G.bands[j]];
      pd.out = G.out.as<double2>() + j * nlm;
      pd.alm64 = (char*)G.alm.p + (size_t)j * nlm * 16;
      pd.alm32 = (char*)G.alm.p + (size_t)j * nlm * 8;
      pd.c = g.c64.as<double>();
      pd.L = g.lmax;
      pd.var = 1;
    }
  }
  CMBWS_TRY(M->d_pairs.upload(pairs.data(), pairs.size() * sizeof(PairDev)));

  // ---- U blocks (Eqs. U-data, U-prior) and U^+ (Sec. 3.1) ----
  M->Lup = M->Lcomp;
  const int nr = no + nc;
  std::vector<double> Up((size_t)(M->Lup + 1) * nc * nr, 0.0);
  for (int l = 0; l <= M->Lup; ++l) {
    std::vector<int> act;
    for (int k = 0; k < nc; ++k)
      if (l <= M->Lk[k]) act.push_back(k);
    const int na = (int)act.size();
    std::vector<double> U((size_t)nr * na, 0.0), P;
    for (int a = 0; a < na; ++a) {
      const int k = act[a];
      for (int nu = 0; nu < no; ++nu)
        if (l <= M->Lnu[nu])
          U[(size_t)nu * na + a] = M->alpha[nu] * desc->beam[nu][l] * qpre[nu * nc + k];
      U[(size_t)(no + k) * na + a] = cinv_k[k][l];
    }
    if (!pinv_jacobi(U, nr, na, 1e-12, P)) {
      set_error("cmbws_model_create: at l = %d a component has neither data nor prior", l);
      return CMBWS_ERR_SINGULAR;
    }
    for (int a = 0; a < na; ++a)
      for (int j = 0; j < nr; ++j) Up[((size_t)l * nc + act[a]) * nr + j] = P[(size_t)a * nr + j];
  }

  // ---- upload ----
  std::vector<int> compL(M->Lk);
  CMBWS_TRY(M->d_compL.upload(compL.data(), nc * 4));
  CMBWS_TRY(M->d_compOff.upload(M->compOff.data(), nc * 8));
  CMBWS_TRY(M->d_q.upload(q.data(), q.size() * 8));
  CMBWS_TRY(M->d_beam.upload(beam.data(), beam.size() * 8));
  CMBWS_TRY(M->d_beamOff.upload(beamOff.data(), no * 8));
  M->beam_off_h = beamOff;
  CMBWS_TRY(M->d_cinv.upload(cinv.data(), cinv.size() * 8));
  CMBWS_TRY(M->d_cisq.upload(cisq.data(), cisq.size() * 8));
  CMBWS_TRY(M->d_clOff.upload(clOff.data(), nc * 8));
  CMBWS_TRY(M->d_Up.upload(Up.data(), Up.size() * 8));
  CMBWS_TRY(M->d_qpre.upload(qpre.data(), qpre.size() * 8));
  M->beam_h = beam;
  M->cisq_h = cisq;
  M->qpre_h = qpre;
  M->clOff_h = clOff;

  // ---- workspaces ----
  size_t part_bytes = 0;
  for (Group& G : M->groups) {
    const Grid& g = *G.grid;
    const int64_t nlm = nlm_of(g.lmax);
    CMBWS_TRY(G.alm.alloc((size_t)G.nmaps * nlm * 16));
    CMBWS_TRY(G.F.alloc((size_t)G.nmaps * g.nring * (g.lmax + 1) * 16));
    CMBWS_TRY(G.out.alloc((size_t)G.nmaps * nlm * 16));
    for (int pr : {CMBWS_FP64, CMBWS_FP32, CMBWS_FP32X2})
      part_bytes = std::max(part_bytes, legendre_adjoint_part_bytes(g, pr, G.nmaps));
  }
  for (Group& G : M->mgroups)
    for (int pr : {CMBWS_FP64, CMBWS_FP32, CMBWS_FP32X2})
      part_bytes = std::max(part_bytes, legendre_adjoint_part_bytes(*G.grid, pr, G.nmaps));
  CMBWS_TRY(M->part.alloc(part_bytes));
  CMBWS_TRY(M->tprior.alloc((size_t)M->nvec * 8));
  M->nsht_A = 2 * (2 * M->nmix + no);  // Sec. 3.3: 2 (2 Nmix + Nobs)
  M->nsht_M = 2 * no;
  CMBWS_CUDA(cudaStreamSynchronize(s));
  *out = guard.release();
  return CMBWS_OK;
}

}  // namespace cmbws

using namespace cmbws;

extern "C" int cmbws_model_create(const cmbws_model_desc* desc, cmbws_prec prec, void* stream,
                                  cmbws_model* out) {
  clear_error();
  if (!desc || !out || !valid_prec(prec)) {
    set_error("cmbws_model_create: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  *out = nullptr;
  Model* M = nullptr;
  int st = model_create(desc, (int)prec, (cudaStream_t)stream, &M);
  if (st != CMBWS_OK) return st;
  handle_add(HANDLE_MODEL, M);
  *out = reinterpret_cast<cmbws_model>(M);
  return CMBWS_OK;
}

extern "C" int cmbws_model_destroy(cmbws_model mh) {
  clear_error();
  if (!mh) return CMBWS_OK;
  if (!handle_del(HANDLE_MODEL, mh)) {
    set_error("cmbws_model_destroy: not a live model handle (destroyed twice?)");
    return CMBWS_ERR_ARG;
  }
  delete reinterpret_cast<Model*>(mh);
  return CMBWS_OK;
}

extern "C" int cmbws_model_info(cmbws_model mh, int64_t* nvec, int* nsht_A, int* nsht_M) {
  clear_error();
  Model* M = as_model(mh);
  if (!M) {
    set_error("cmbws_model_info: null model");
    return CMBWS_ERR_ARG;
  }
  if (nvec) *nvec = M->nvec;
  if (nsht_A) *nsht_A = M->nsht_A;
  if (nsht_M) *nsht_M = M->nsht_M;
  return CMBWS_OK;
}

extern "C" int cmbws_apply_A(cmbws_model mh, const double* x, double* y, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (!M || !x || !y || x == y) {
    set_error("cmbws_apply_A: invalid arguments (x and y must be distinct device buffers)");
    return CMBWS_ERR_ARG;
  }
  return M->apply_A(x, y, M->prec, (cudaStream_t)stream);
}

extern "C" int cmbws_apply_precond(cmbws_model mh, const double* r, double* z, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (!M || !r || !z || r == z) {
    set_error("cmbws_apply_precond: invalid arguments (r and z must be distinct device buffers)");
    return CMBWS_ERR_ARG;
  }
  return M->apply_precond(r, z, M->prec, (cudaStream_t)stream);
}

extern "C" int cmbws_project(cmbws_model mh, const double* x, double* const* d, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (!M || !x || !d) {
    set_error("cmbws_project: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  for (int nu = 0; nu < M->nobs; ++nu)
    if (!d[nu]) {
      set_error("cmbws_project: missing map for band %d", nu);
      return CMBWS_ERR_ARG;
    }
  return M->project(x, d, M->prec, (cudaStream_t)stream);
}

extern "C" int cmbws_rhs(cmbws_model mh, const double* const* d, const double* const* omega1,
                         const double* omega2, double* b, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (!M || !d || !b) {
    set_error("cmbws_rhs: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  for (int nu = 0; nu < M->nobs; ++nu)
    if (!d[nu] || (omega1 && !omega1[nu])) {
      set_error("cmbws_rhs: missing map for band %d", nu);
      return CMBWS_ERR_ARG;
    }
  return M->rhs(d, omega1, omega2, b, (cudaStream_t)stream);
}

extern "C" int cmbws_model_set_shard(cmbws_model mh, const int* owned, int prior) {
  clear_error();
  Model* M = as_model(mh);
  if (!M) {
    set_error("cmbws_model_set_shard: invalid model");
    return CMBWS_ERR_ARG;
  }
  if (!owned) {
    M->shard_on = false;
    M->shard_own = ~0ull;
    M->shard_prior = true;
    M->drop_graphs();
    return CMBWS_OK;
  }
  if (M->merged || !M->masks.empty()) {
    set_error("cmbws_model_set_shard: not available with merged rows or mask preconditioners");
    return CMBWS_ERR_ARG;
  }
  uint64_t own = 0;
  for (int nu = 0; nu < M->nobs; ++nu) {
    if (owned[nu] != 0 && owned[nu] != 1) {
      set_error("cmbws_model_set_shard: owned[%d] must be 0 or 1", nu);
      return CMBWS_ERR_ARG;
    }
    if (owned[nu]) own |= 1ull << nu;
  }
  M->shard_on = true;
  M->shard_own = own;
  M->shard_prior = prior != 0;
  M->drop_graphs();
  return CMBWS_OK;
}
