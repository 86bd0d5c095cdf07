// Mask-restricted preconditioner with a multigrid V-cycle (Sec. 4 of the paper).
//
// With the mask carried by the mixing maps, the CR system under the mask only sees the
// prior.  With Z = (pixels in the mask) Y R, R = diag(r_l) the low-pass filter of Eq. rl
// (r_l = exp(-beta l^2 (l+1)^2), beta such that r^2 = 0.05 at L/2),
//   M_mask = Z^T (Z S^-1 Z^T)^-1 Z   (Eq. M_mask),   M_add = M_PI + M_mask (Sec. 4.2),
// and G = Z S^-1 Z^T = Y D Y^T (Eq. W, d_l = r_l^2 / C_l) is inverted approximately by one
// basic V-cycle (Sec. 4.4):
//   * levels: HEALPix grids with Nside and band-limit halved per level; a coarse pixel is in
//     the mask when all four of its children are (parent = the coarse pixel containing the
//     child's centre);
//   * restriction Y_H R_H Y_h^T W_h (R_H the Eq. rl filter at L_H), interpolation its transpose;
//   * coarse operators d_H = r_H^2 d_h;
//   * smoother omega / diag(G_h), omega = 0.2, diag(G_h) = sum_l (2l+1) / (4 pi) d_{h,l}, with
//     omega capped so that omega lambda_max(G_h) / diag(G_h) <= 1 on oversampled grids;
//   * bottom: the SVD pseudo-inverse of the dense G on the mask pixels.
// Maps live full-sky on each level (zero outside the mask), as the paper's "zero padding".
// The transforms are the library's own (cmbws_sht_synth / cmbws_sht_analysis) on level grids
// owned by the preconditioner, in FP32 for FP32-family models and FP64 otherwise.
#include <cmath>

#include "model.h"

namespace cmbws {

namespace {

constexpr double kOmega = 0.2;
// Bottom pseudo-inverse cut-off, relative to the largest singular value.  The compounded
// Eq. rl filters make d_l span ~20 orders of magnitude, so G has eigenvalues far below the
// large scales the bottom solve is for (those stay within ~1e-3 of the largest); keeping
// eigenvalues down to 1e-10 would amplify the FP32 rounding of the right-hand side by up to
// 1e10 and make the preconditioner noisy (no longer a fixed symmetric operator).
constexpr double kBottomRcond = 1e-5;

// out[i] = mask[i] ? ca * a[i] + cb * b[i] : 0   (b may be null)
__global__ void k_map_lincomb(double* __restrict__ out, double ca, const double* a, double cb,
                              const double* b, const double* __restrict__ mask, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double v = ca * a[i];
  if (b) v += cb * b[i];
  out[i] = mask[i] != 0.0 ? v : 0.0;
}

// packed (CMBWS_ALM) coefficients: out (band-limit Lout) [+]= f_l * in (band-limit Lin, zero above)
__global__ void k_pk_xfer(const double* __restrict__ in, int Lin, double* __restrict__ out, int Lout,
                          const double* __restrict__ f, int accumulate) {
  const int m = blockIdx.y;
  const int l = m + blockIdx.x * blockDim.x + threadIdx.x;
  if (l > Lout) return;
  // f has min(Lin, Lout) + 1 entries: read it only where the input exists
  const double fl = l <= Lin ? f[l] : 0.0;
  const int64_t po = packed_off(Lout, m);
  for (int c = 0; c < (m > 0 ? 2 : 1); ++c) {
    double v = 0.0;
    if (l <= Lin) v = fl * in[packed_off(Lin, m) + c * (Lin - m + 1) + (l - m)];
    double* o = out + po + c * (Lout - m + 1) + (l - m);
    *o = accumulate ? *o + v : v;
  }
}

__global__ void k_gather(const double* __restrict__ in, const int* __restrict__ idx, int nb,
                         double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nb) out[i] = in[idx[i]];
}
__global__ void k_scatter(const double* __restrict__ in, const int* __restrict__ idx, int nb,
                          double* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < nb) out[idx[i]] = in[i];
}
// y = G x for a dense nb x nb matrix, one warp per row (fixed summation order)
__global__ void k_dense_mv(const double* __restrict__ G, int nb, const double* __restrict__ x,
                           double* __restrict__ y) {
  const int row = blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= nb) return;
  double s = 0.0;
  for (int j = lane; j < nb; j += 32) s += G[(int64_t)row * nb + j] * x[j];
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if (lane == 0) y[row] = s;
}

inline unsigned nblk(int64_t n, int t = 256) { return (unsigned)((n + t - 1) / t); }

// Eq. rl filter for l <= lfull, r^2 = 0.05 at L / 2
std::vector<double> rl_filter(int L, int lfull) {
  const double h = 0.5 * L;
  const double beta = L > 0 ? -std::log(0.05) / (2.0 * h * h * (h + 1.0) * (h + 1.0)) : 0.0;
  std::vector<double> r(lfull + 1);
  for (int l = 0; l <= lfull; ++l) r[l] = std::exp(-beta * (double)l * l * (l + 1.0) * (l + 1.0));
  return r;
}

// HEALPix ring-scheme pixel containing (theta, phi) (Gorski et al. 2005 geometry): in the
// equatorial zone |z| <= 2/3 the pixel boundaries are the lines t - 3z/4 = k / N and
// t + 3z/4 = k / N (t = 2 phi / pi - 1/2 ...), in the polar caps the lines
// t' N sqrt(3 (1 - |z|)) = k and (1 - t') N sqrt(3 (1 - |z|)) = k (t' the position in the
// face's quarter); the two integer line counts give the ring and the pixel in the ring.
int64_t ang2pix_ring(int N, double theta, double phi) {
  const double z = std::cos(theta);
  double t = std::fmod(phi, 2.0 * M_PI);
  if (t < 0) t += 2.0 * M_PI;
  t /= 0.5 * M_PI;  // [0, 4)
  const int64_t ncap = 2LL * N * (N - 1), npix = 12LL * N * N;
  if (std::fabs(z) <= 2.0 / 3.0) {
    const double a = N * (0.5 + t), b = N * 0.75 * z;
    const int64_t jp = (int64_t)std::floor(a - b), jm = (int64_t)std::floor(a + b);
    const int64_t ir = N + 1 + jp - jm;  // 1 .. 2N+1 within the belt
    const int64_t shifted = ((ir - 1) % 2 == 0) ? 1 : 0;
    int64_t j = (jp + jm + 1 - N - shifted) / 2;  // the numerator is always even
    j %= 4LL * N;
    if (j < 0) j += 4LL * N;
    return ncap + (ir - 1) * 4LL * N + j;
  }
  const double za = std::fabs(z);
  const int64_t face = (int64_t)std::floor(t);
  const double tp = t - face;
  const double tmp = N * std::sqrt(3.0 * (1.0 - za));
  const int64_t jp = (int64_t)std::floor(tp * tmp), jm = (int64_t)std::floor((1.0 - tp) * tmp);
  const int64_t ir = jp + jm + 1;  // ring counted from the nearer pole
  const int64_t ip = face * ir + std::min<int64_t>(jp, ir - 1);
  return z > 0 ? 2 * ir * (ir - 1) + ip : npix - 2 * ir * (ir + 1) + ip;
}

}  // namespace

struct MgLevel {
  Grid* g = nullptr;
  int nside = 0, L = 0;
  int64_t npix = 0;
  double w = 0.0, smooth = 0.0;
  int nb = 0;                       // bottom level: number of mask pixels
  std::vector<double> d_h, rH_h;    // host copies (d_l; restriction filter to the next level)
  std::vector<uint8_t> mask_h;
  DevMem mask, d, rH, idx, Gp, vb, vb2;
  DevMem b, x, t, y, a;             // maps (b, x, t, y) and packed coefficients a
  // optimized V-cycle (planned on first use): this level's grid at the next level's
  // band-limit L_H, packed coefficients at L_H, and the factors 1 and -d_l (l <= L_H)
  Grid* gH = nullptr;
  DevMem aH, ones, dneg;
};

struct MaskMG {
  int comp = 0, Lk = 0, L0 = 0, prec = CMBWS_FP64;
  std::vector<MgLevel> lv;
  DevMem r0;
  long long nsht = 0;  // SHTs of the applications (the paper's counting)
  ~MaskMG() {
    for (MgLevel& l : lv) {
      if (l.g) cmbws_grid_destroy(reinterpret_cast<cmbws_grid>(l.g));
      if (l.gH) cmbws_grid_destroy(reinterpret_cast<cmbws_grid>(l.gH));
    }
  }
};

void mask_mg_destroy(MaskMG* p) { delete p; }

Model::~Model() {
  drop_graphs();
  if (cg_host) cudaFreeHost(cg_host);
  for (MaskMG* p : masks) mask_mg_destroy(p);
}

namespace {

int synth_on(MaskMG& mg, Grid* g, const double* a, double* map, cudaStream_t s) {
  ++mg.nsht;
  return cmbws_sht_synth(reinterpret_cast<cmbws_grid>(g), (cmbws_prec)mg.prec, a, map, 1, s);
}
int adjoint_on(MaskMG& mg, Grid* g, const double* map, double* a, int weighted, cudaStream_t s) {
  ++mg.nsht;
  return cmbws_sht_analysis(reinterpret_cast<cmbws_grid>(g), (cmbws_prec)mg.prec, map, a, 1,
                            weighted, s);
}
int synth(MaskMG& mg, MgLevel& h, const double* a, double* map, cudaStream_t s) {
  return synth_on(mg, h.g, a, map, s);
}
int adjoint(MaskMG& mg, MgLevel& h, const double* map, double* a, int weighted, cudaStream_t s) {
  return adjoint_on(mg, h.g, map, a, weighted, s);
}

int lincomb(MgLevel& h, double* out, double ca, const double* a, double cb, const double* b,
            cudaStream_t s) {
  ProfScope ps(PROF_HARM, s, 1);
  k_map_lincomb<<<nblk(h.npix), 256, 0, s>>>(out, ca, a, cb, b, h.mask.as<double>(), h.npix);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

int xfer(const double* in, int Lin, double* out, int Lout, const double* f, int acc, cudaStream_t s) {
  ProfScope ps(PROF_HARM, s, 1);
  dim3 grd((Lout + 1 + 127) / 128, Lout + 1);
  k_pk_xfer<<<grd, 128, 0, s>>>(in, Lin, out, Lout, f, acc);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

// y = G_h x = P Y D Y^T x (x zero outside the mask)
int apply_G(MaskMG& mg, MgLevel& h, const double* x, double* y, cudaStream_t s) {
  CMBWS_TRY(adjoint(mg, h, x, h.a.as<double>(), 0, s));
  CMBWS_TRY(xfer(h.a.as<double>(), h.L, h.a.as<double>(), h.L, h.d.as<double>(), 0, s));
  CMBWS_TRY(synth(mg, h, h.a.as<double>(), y, s));
  return lincomb(h, y, 1.0, y, 0.0, nullptr, s);
}

// bottom level: x = G^+ b with the dense pseudo-inverse on the mask pixels
int bottom_solve(MgLevel& h, const double* b, double* x, cudaStream_t s) {
  ProfScope ps(PROF_HARM, s, 1);
  CMBWS_CUDA(cudaMemsetAsync(x, 0, h.npix * 8, s));
  k_gather<<<nblk(h.nb), 256, 0, s>>>(b, h.idx.as<int>(), h.nb, h.vb.as<double>());
  k_dense_mv<<<nblk(h.nb, 8), 256, 0, s>>>(h.Gp.as<double>(), h.nb, h.vb.as<double>(),
                                          h.vb2.as<double>());
  k_scatter<<<nblk(h.nb), 256, 0, s>>>(h.vb2.as<double>(), h.idx.as<int>(), h.nb, x);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

// x = V-cycle approximation of G_k^-1 b (basic V-cycle of Sec. 4.4)
int vcycle(MaskMG& mg, int k, const double* b, double* x, cudaStream_t s) {
  MgLevel& h = mg.lv[k];
  if (h.nb > 0) return bottom_solve(h, b, x, s);
  MgLevel& H = mg.lv[k + 1];
  double* t = h.t.as<double>();
  double* y = h.y.as<double>();
  CMBWS_TRY(lincomb(h, x, h.smooth, b, 0.0, nullptr, s));         // pre-smoothing
  CMBWS_TRY(apply_G(mg, h, x, y, s));
  CMBWS_TRY(lincomb(h, t, 1.0, b, -1.0, y, s));                   // residual
  // restriction: H.b = P_H Y_H R_H Y_h^T W_h t
  CMBWS_TRY(adjoint(mg, h, t, h.a.as<double>(), 1, s));
  CMBWS_TRY(xfer(h.a.as<double>(), h.L, H.a.as<double>(), H.L, h.rH.as<double>(), 0, s));
  CMBWS_TRY(synth(mg, H, H.a.as<double>(), H.b.as<double>(), s));
  CMBWS_TRY(lincomb(H, H.b.as<double>(), 1.0, H.b.as<double>(), 0.0, nullptr, s));
  CMBWS_TRY(vcycle(mg, k + 1, H.b.as<double>(), H.x.as<double>(), s));  // coarse correction
  // interpolation: x += P_h W_h Y_h R_H Y_H^T H.x
  CMBWS_TRY(adjoint(mg, H, H.x.as<double>(), H.a.as<double>(), 0, s));
  CMBWS_TRY(xfer(H.a.as<double>(), H.L, h.a.as<double>(), h.L, h.rH.as<double>(), 0, s));
  CMBWS_TRY(synth(mg, h, h.a.as<double>(), t, s));
  CMBWS_TRY(lincomb(h, x, 1.0, x, h.w, t, s));
  CMBWS_TRY(apply_G(mg, h, x, y, s));                             // post-smoothing
  CMBWS_TRY(lincomb(h, t, 1.0, b, -1.0, y, s));
  return lincomb(h, x, 1.0, x, h.smooth, t, s);
}

// The optimized V-cycle (Sec. 4.4, Fig. code:mg): I_h^H = Y_H R_H Y_h^T W_h and
// G_h = P Y_h D_h Y_h^T P inserted so that restriction and interpolation share transforms
// with G_h, and J = Y_h^T W_h P Y_h approximated by I as in the paper: 6 SHTs per level
// (Y_h^T at L_h, Y_h^T W_h at L_H, Y_H and Y_H^T, Y_h at L_H, Y_h at L_h).  b and x are
// zero outside the mask.
int vcycle_opt(MaskMG& mg, int k, const double* b, double* x, cudaStream_t s) {
  MgLevel& h = mg.lv[k];
  if (h.nb > 0) return bottom_solve(h, b, x, s);
  MgLevel& H = mg.lv[k + 1];
  double* t = h.t.as<double>();
  double* y = h.y.as<double>();
  double* u = h.a.as<double>();    // Y_h^T x, kept for the post-smoothing
  double* aH = h.aH.as<double>();
  CMBWS_TRY(lincomb(h, x, h.smooth, b, 0.0, nullptr, s));              // pre-smoothing
  CMBWS_TRY(adjoint(mg, h, x, u, 0, s));                                // u = Y_h^T x
  CMBWS_TRY(adjoint_on(mg, h.gH, b, aH, 1, s));                         // Y_h^T W_h b, l <= L_H
  CMBWS_TRY(xfer(u, h.L, aH, H.L, h.dneg.as<double>(), 1, s));          //   - D_h u
  CMBWS_TRY(xfer(aH, H.L, H.a.as<double>(), H.L, h.rH.as<double>(), 0, s));
  CMBWS_TRY(synth(mg, H, H.a.as<double>(), H.b.as<double>(), s));       // r_H = P Y_H R_H r~
  CMBWS_TRY(lincomb(H, H.b.as<double>(), 1.0, H.b.as<double>(), 0.0, nullptr, s));
  CMBWS_TRY(vcycle_opt(mg, k + 1, H.b.as<double>(), H.x.as<double>(), s));
  CMBWS_TRY(adjoint(mg, H, H.x.as<double>(), H.a.as<double>(), 0, s));  // c~ = R_H Y_H^T c_H
  CMBWS_TRY(xfer(H.a.as<double>(), H.L, aH, H.L, h.rH.as<double>(), 0, s));
  CMBWS_TRY(synth_on(mg, h.gH, aH, t, s));                              // x += P W_h Y_h c~
  CMBWS_TRY(lincomb(h, x, 1.0, x, h.w, t, s));
  CMBWS_TRY(xfer(aH, H.L, u, h.L, h.ones.as<double>(), 1, s));          // u + J c~, J ~ I
  CMBWS_TRY(xfer(u, h.L, u, h.L, h.d.as<double>(), 0, s));
  CMBWS_TRY(synth(mg, h, u, y, s));                                     // G_h x
  CMBWS_TRY(lincomb(h, t, 1.0, b, -1.0, y, s));                         // post-smoothing
  return lincomb(h, x, 1.0, x, h.smooth, t, s);
}

// plan the fine grids at the coarse band-limits and the factors of the optimized cycle
int prepare_opt(MaskMG& mg) {
  for (size_t k = 0; k + 1 < mg.lv.size(); ++k) {
    MgLevel& h = mg.lv[k];
    if (h.nb > 0 || h.gH) continue;
    const int LH = mg.lv[k + 1].L;
    cmbws_grid g = nullptr;
    CMBWS_TRY(cmbws_plan_grid(CMBWS_GRID_HEALPIX, h.nside, LH, &g));
    std::vector<double> ones(LH + 1, 1.0), dneg(LH + 1);
    for (int l = 0; l <= LH; ++l) dneg[l] = -h.d_h[l];
    CMBWS_TRY(h.ones.upload(ones.data(), ones.size() * 8));
    CMBWS_TRY(h.dneg.upload(dneg.data(), dneg.size() * 8));
    CMBWS_TRY(h.aH.alloc((size_t)(LH + 1) * (LH + 1) * 8));
    h.gH = reinterpret_cast<Grid*>(g);
  }
  return CMBWS_OK;
}

}  // namespace

// z += M_mask r on the preconditioner's component (stacked vectors)
int mask_mg_apply(MaskMG& mg, Model& M, const double* r, double* z, cudaStream_t s) {
  if (M.vcycle == 1) CMBWS_TRY(prepare_opt(mg));
  const long long n0 = mg.nsht;
  struct Count {
    MaskMG& mg;
    Model& M;
    long long n0;
    ~Count() { M.n_sht += mg.nsht - n0; }
  } count{mg, M, n0};
  MgLevel& h = mg.lv[0];
  const int64_t off = M.compOff[mg.comp];
  CMBWS_TRY(xfer(r + off, mg.Lk, h.a.as<double>(), mg.L0, mg.r0.as<double>(), 0, s));
  CMBWS_TRY(synth(mg, h, h.a.as<double>(), h.b.as<double>(), s));           // Z r
  CMBWS_TRY(lincomb(h, h.b.as<double>(), 1.0, h.b.as<double>(), 0.0, nullptr, s));
  if (M.vcycle == 1) CMBWS_TRY(vcycle_opt(mg, 0, h.b.as<double>(), h.x.as<double>(), s));
  else CMBWS_TRY(vcycle(mg, 0, h.b.as<double>(), h.x.as<double>(), s));
  CMBWS_TRY(adjoint(mg, h, h.x.as<double>(), h.a.as<double>(), 0, s));      // Z^T x
  return xfer(h.a.as<double>(), mg.L0, z + off, mg.Lk, mg.r0.as<double>(), 1, s);
}

namespace {

int add_level(MaskMG& mg, int nside, int L, const std::vector<uint8_t>& mask,
              const std::vector<double>& d) {
  mg.lv.emplace_back();
  MgLevel& h = mg.lv.back();
  cmbws_grid gh = nullptr;
  CMBWS_TRY(cmbws_plan_grid(CMBWS_GRID_HEALPIX, nside, L, &gh));
  h.g = reinterpret_cast<Grid*>(gh);
  h.nside = nside;
  h.L = L;
  h.npix = 12LL * nside * nside;
  h.w = 4.0 * M_PI / (double)h.npix;
  h.mask_h = mask;
  h.d_h = d;
  // damped smoother omega / diag(G): the paper's omega = 0.2 keeps omega M G below 2 on its
  // grids (L = 3 Nside); lambda_max(G) <= max_l d_l Npix / (4 pi), so on grids with more
  // pixels per harmonic mode omega is capped at diag(G) / (max_l d_l Npix / (4 pi)) (<= 1)
  double dg = 0.0, dmax = 0.0;
  for (int l = 0; l <= L; ++l) {
    dg += (2.0 * l + 1.0) / (4.0 * M_PI) * d[l];
    dmax = std::max(dmax, d[l]);
  }
  const double lmax_bound = dmax * (double)h.npix / (4.0 * M_PI);
  const double omega = lmax_bound > 0 ? std::min(kOmega, dg / lmax_bound) : kOmega;
  h.smooth = dg > 0 ? omega / dg : 0.0;
  std::vector<double> mk(h.npix);
  for (int64_t i = 0; i < h.npix; ++i) mk[i] = mask[i] ? 1.0 : 0.0;
  CMBWS_TRY(h.mask.upload(mk.data(), h.npix * 8));
  CMBWS_TRY(h.d.upload(d.data(), (L + 1) * 8));
  for (DevMem* m : {&h.b, &h.x, &h.t, &h.y}) CMBWS_TRY(m->alloc(h.npix * 8));
  CMBWS_TRY(h.a.alloc((size_t)(L + 1) * (L + 1) * 8));
  return CMBWS_OK;
}

// dense G on the mask pixels of the bottom level, its pseudo-inverse uploaded
int build_bottom(MaskMG& mg, MgLevel& h, cudaStream_t s) {
  std::vector<int> idx;
  for (int64_t i = 0; i < h.npix; ++i)
    if (h.mask_h[i]) idx.push_back((int)i);
  h.nb = (int)idx.size();
  if (h.nb == 0) return CMBWS_OK;
  CMBWS_TRY(h.idx.upload(idx.data(), idx.size() * 4));
  CMBWS_TRY(h.vb.alloc(h.nb * 8));
  CMBWS_TRY(h.vb2.alloc(h.nb * 8));
  const int saved = mg.prec;
  mg.prec = CMBWS_FP64;  // the dense matrix in FP64
  std::vector<double> G((size_t)h.nb * h.nb), col(h.npix);
  double* e = h.b.as<double>();
  double* ge = h.y.as<double>();
  for (int j = 0; j < h.nb; ++j) {
    CMBWS_CUDA(cudaMemsetAsync(e, 0, h.npix * 8, s));
    const double one = 1.0;
    CMBWS_CUDA(cudaMemcpyAsync(e + idx[j], &one, 8, cudaMemcpyHostToDevice, s));
    CMBWS_TRY(apply_G(mg, h, e, ge, s));
    CMBWS_CUDA(cudaMemcpyAsync(col.data(), ge, h.npix * 8, cudaMemcpyDeviceToHost, s));
    CMBWS_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < h.nb; ++i) G[(size_t)i * h.nb + j] = col[idx[i]];
  }
  mg.prec = saved;
  for (int i = 0; i < h.nb; ++i)  // symmetrise the FP64 rounding
    for (int j = i + 1; j < h.nb; ++j) {
      const double v = 0.5 * (G[(size_t)i * h.nb + j] + G[(size_t)j * h.nb + i]);
      G[(size_t)i * h.nb + j] = G[(size_t)j * h.nb + i] = v;
    }
  std::vector<double> P;
  if (!pinv_jacobi(G, h.nb, h.nb, kBottomRcond, P)) {
    set_error("mask preconditioner: singular bottom system (a pixel with zero coupling)");
    return CMBWS_ERR_SINGULAR;
  }
  CMBWS_TRY(h.Gp.upload(P.data(), P.size() * 8));
  return CMBWS_OK;
}

int mask_mg_build(Model& M, int comp, int nside, const double* mask_dev, int max_bottom,
                  cudaStream_t s, MaskMG** out) {
  const int Lk = M.Lk[comp];
  // the component's prior C^-1 (host copy)
  std::vector<int64_t> cloff(M.ncomp);
  CMBWS_CUDA(cudaMemcpy(cloff.data(), M.d_clOff.p, M.ncomp * 8, cudaMemcpyDeviceToHost));
  std::vector<double> cinv(Lk + 1);
  CMBWS_CUDA(cudaMemcpy(cinv.data(), M.d_cinv.as<double>() + cloff[comp], (Lk + 1) * 8,
                        cudaMemcpyDeviceToHost));
  bool any = false;
  for (double v : cinv) any |= v > 0;
  if (!any) {
    set_error("cmbws_model_add_mask_precond: component %d has no prior", comp);
    return CMBWS_ERR_ARG;
  }
  const int64_t npix0 = 12LL * nside * nside;
  std::vector<double> mk(npix0);
  CMBWS_CUDA(cudaMemcpy(mk.data(), mask_dev, npix0 * 8, cudaMemcpyDeviceToHost));
  std::vector<uint8_t> mask(npix0);
  for (int64_t i = 0; i < npix0; ++i) mask[i] = mk[i] != 0.0;

  MaskMG* mg = new MaskMG();
  std::unique_ptr<MaskMG> guard(mg);
  mg->comp = comp;
  mg->Lk = Lk;
  mg->L0 = std::min(3 * nside - 1, Lk);
  mg->prec = is_f32(M.prec) ? CMBWS_FP32 : CMBWS_FP64;
  const std::vector<double> r0 = rl_filter(mg->L0, mg->L0);
  CMBWS_TRY(mg->r0.upload(r0.data(), r0.size() * 8));
  std::vector<double> d(mg->L0 + 1);
  for (int l = 0; l <= mg->L0; ++l) d[l] = r0[l] * r0[l] * cinv[l];
  CMBWS_TRY(add_level(*mg, nside, mg->L0, mask, d));
  for (;;) {
    MgLevel& h = mg->lv.back();
    int64_t cnt = 0;
    for (uint8_t v : h.mask_h) cnt += v;
    if (cnt <= max_bottom || h.nside < 2 || h.L < 2) break;
    // coarse mask: parent of every fine pixel = the coarse pixel containing its centre
    const int NH = h.nside / 2;
    const int64_t npH = 12LL * NH * NH;
    std::vector<int> nchild(npH, 0), ninside(npH, 0);
    const Grid& g = *h.g;
    for (int r = 0; r < g.nring; ++r)
      for (int j = 0; j < g.nphi[r]; ++j) {
        const int64_t p = g.offset[r] + j;
        const double ph = g.phi0[r] + 2.0 * M_PI * j / g.nphi[r];
        const int64_t q = ang2pix_ring(NH, g.theta[r], ph);
        if (q < 0 || q >= npH) {
          set_error("mask preconditioner: pixel centre outside the coarse grid (Nside %d)", NH);
          return CMBWS_ERR_ARG;
        }
        nchild[q] += 1;
        ninside[q] += h.mask_h[p];
      }
    std::vector<uint8_t> mH(npH);
    bool anyH = false;
    for (int64_t q = 0; q < npH; ++q) {
      mH[q] = (nchild[q] == 4 && ninside[q] == 4);
      anyH |= mH[q] != 0;
    }
    if (!anyH) break;
    const int LH = h.L / 2;
    std::vector<double> rH = rl_filter(LH, LH), dH(LH + 1);
    for (int l = 0; l <= LH; ++l) dH[l] = rH[l] * rH[l] * h.d_h[l];
    h.rH_h = rH;
    CMBWS_TRY(h.rH.upload(rH.data(), rH.size() * 8));
    CMBWS_TRY(add_level(*mg, NH, LH, mH, dH));
  }
  CMBWS_TRY(build_bottom(*mg, mg->lv.back(), s));
  *out = guard.release();
  return CMBWS_OK;
}

}  // namespace

}  // namespace cmbws

using namespace cmbws;

extern "C" int cmbws_model_add_mask_precond(cmbws_model mh, int comp, int nside, const double* mask,
                                            int max_bottom, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (refuse_sharded(M, "cmbws_model_add_mask_precond")) return CMBWS_ERR_ARG;
  if (!M || !mask || comp < 0 || comp >= M->ncomp || nside < 1 || max_bottom < 1 ||
      max_bottom > 4096) {
    set_error("cmbws_model_add_mask_precond: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  MaskMG* mg = nullptr;
  const int st = mask_mg_build(*M, comp, nside, mask, max_bottom, (cudaStream_t)stream, &mg);
  if (st != CMBWS_OK) return st;
  M->drop_graphs();
  M->masks.push_back(mg);
  CMBWS_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  return CMBWS_OK;
}

extern "C" int cmbws_model_set_vcycle(cmbws_model mh, int kind) {
  clear_error();
  Model* M = as_model(mh);
  if (!M || (kind != 0 && kind != 1)) {
    set_error("cmbws_model_set_vcycle: invalid arguments (kind 0 = basic, 1 = optimized)");
    return CMBWS_ERR_ARG;
  }
  if (M->vcycle != kind) M->drop_graphs();
  M->vcycle = kind;
  return CMBWS_OK;
}

extern "C" int cmbws_apply_M_add(cmbws_model mh, const double* r, double* z, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (refuse_sharded(M, "cmbws_apply_M_add")) return CMBWS_ERR_ARG;
  if (!M || !r || !z || r == z) {
    set_error("cmbws_apply_M_add: invalid arguments");
    return CMBWS_ERR_ARG;
  }
  cudaStream_t s = (cudaStream_t)stream;
  CMBWS_TRY(M->apply_precond(r, z, M->prec, s));
  for (MaskMG* mg : M->masks) CMBWS_TRY(mask_mg_apply(*mg, *M, r, z, s));
  return CMBWS_OK;
}
