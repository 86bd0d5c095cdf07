// Observation merging in the pseudo-inverse preconditioner (App. A.3).
//
// Bands with identical normalised inverse noise and proportional rows of U (U_2 = gamma U_1,
// e.g. detector splits of one frequency channel) contribute (1 + gamma^2) U_1^T N~^-1 U_1 to
// U^T T U, so M_PI can use one row sqrt(1 + gamma^2) U_1 and one T^+ for all of them: one SHT
// pair per group instead of one per band.  For bands that are only similar, a group's row
// is, per l, the best rank-one fit of sum_{nu in G} U_nu^T U_nu (leading eigenpair; exact
// for proportional rows), and its T^+ uses the co-added inverse noise tau_G = sum tau_nu
// with alpha_G from Eq. optimal-alpha (for exact splits T_G^+ = T_nu^+).  Built once per
// call on the host (per l: an Ncomp x Ncomp symmetric eigenproblem by cyclic Jacobi, then the
// SVD pseudo-inverse of U' as for M_PI) and on the device (tau_G, ring sums, pixel factors);
// applied by Model::apply_precond_merged with the kernels of M_PI.
#include <cmath>

#include "model.h"

namespace cmbws {

namespace {

__global__ void k_tau_add(const double* __restrict__ t, double* __restrict__ acc, int64_t n,
                          int first) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  acc[i] = first ? t[i] : acc[i] + t[i];
}

// per ring: (sum tau / w, sum (tau / w)^2), the sums of Eq. optimal-alpha
__global__ void k_alpha_sums(const double* __restrict__ tau, const int64_t* __restrict__ roff,
                             const double* __restrict__ rw, double2* __restrict__ out) {
  __shared__ double a1[256], a2[256];
  const int r = blockIdx.x;
  const double w = rw[r];
  double s1 = 0.0, s2 = 0.0;
  for (int64_t i = roff[r] + threadIdx.x; i < roff[r + 1]; i += blockDim.x) {
    const double v = tau[i] / w;
    s1 += v;
    s2 += v * v;
  }
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

// T^+ pixel factor alpha^2 w^2 / tau (Sec. 3.3)
__global__ void k_tplus_factors(const double* __restrict__ tau, const int64_t* __restrict__ roff,
                                const double* __restrict__ rw, double alpha2,
                                double* __restrict__ f64, float* __restrict__ f32) {
  const int r = blockIdx.x;
  const double w = rw[r];
  for (int64_t i = roff[r] + threadIdx.x; i < roff[r + 1]; i += blockDim.x) {
    const double f = alpha2 * w * w / tau[i];
    f64[i] = f;
    f32[i] = (float)f;
  }
}

// Leading eigenpair of a symmetric n x n matrix (row-major) by cyclic Jacobi rotations.
void sym_top_eig(std::vector<double> S, int n, double* lam, std::vector<double>& v) {
  std::vector<double> V((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 64; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j) {
        const double a = S[(size_t)i * n + j] * S[(size_t)i * n + j];
        tot += a;
        if (i != j) off += a;
      }
    if (off <= 1e-32 * tot || tot == 0.0) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = S[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double theta = (S[(size_t)q * n + q] - S[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (theta >= 0 ? 1.0 : -1.0) / (std::fabs(theta) + std::sqrt(theta * theta + 1.0));
        const double c = 1.0 / std::sqrt(t * t + 1.0), sn = t * c;
        for (int k = 0; k < n; ++k) {  // columns p, q
          const double skp = S[(size_t)k * n + p], skq = S[(size_t)k * n + q];
          S[(size_t)k * n + p] = c * skp - sn * skq;
          S[(size_t)k * n + q] = sn * skp + c * skq;
        }
        for (int k = 0; k < n; ++k) {  // rows p, q
          const double spk = S[(size_t)p * n + k], sqk = S[(size_t)q * n + k];
          S[(size_t)p * n + k] = c * spk - sn * sqk;
          S[(size_t)q * n + k] = sn * spk + c * sqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - sn * vkq;
          V[(size_t)k * n + q] = sn * vkp + c * vkq;
        }
      }
  }
  int best = 0;
  for (int i = 1; i < n; ++i)
    if (S[(size_t)i * n + i] > S[(size_t)best * n + best]) best = i;
  *lam = S[(size_t)best * n + best];
  v.assign(n, 0.0);
  int big = 0;
  for (int i = 0; i < n; ++i) {
    v[i] = V[(size_t)i * n + best];
    if (std::fabs(v[i]) > std::fabs(v[big])) big = i;
  }
  if (v[big] < 0)
    for (double& x : v) x = -x;
}

}  // namespace

int Model::merge_precond(const int* group, cudaStream_t s) {
  drop_graphs();  // M_PI's launches (and possibly the partial-sum buffer) change
  if (!group) {
    merged.reset();
    nsht_M = 2 * nobs;
    return CMBWS_OK;
  }
  int nrow = 0;
  for (int nu = 0; nu < nobs; ++nu) {
    if (group[nu] < 0 || group[nu] >= nobs) {
      set_error("cmbws_model_merge_precond: group[%d] = %d outside 0..%d", nu, group[nu], nobs - 1);
      return CMBWS_ERR_ARG;
    }
    nrow = std::max(nrow, group[nu] + 1);
  }
  std::vector<std::vector<int>> members(nrow);
  for (int nu = 0; nu < nobs; ++nu) members[group[nu]].push_back(nu);
  for (int g = 0; g < nrow; ++g) {
    if (members[g].empty()) {
      set_error("cmbws_model_merge_precond: group %d has no band (ids must be 0..G-1)", g);
      return CMBWS_ERR_ARG;
    }
    for (int nu : members[g])
      if (grids[nu] != grids[members[g][0]]) {
        set_error("cmbws_model_merge_precond: bands %d and %d of group %d are on different grids",
                  members[g][0], nu, g);
        return CMBWS_ERR_ARG;
      }
  }
  auto P = std::make_unique<MergedPrec>();
  P->nrow = nrow;
  P->row_of_band.assign(group, group + nobs);
  P->pixM64.resize(nrow);
  P->pixM32.resize(nrow);
  P->alpha.resize(nrow);
  P->row_group.resize(nrow);
  P->row_slot.resize(nrow);

  // ---- T^+ of each row from the co-added inverse noise ----
  for (int g = 0; g < nrow; ++g) {
    const Grid& gr = *grids[members[g][0]];
    DevMem tau, sums;
    CMBWS_TRY(tau.alloc((size_t)gr.npix * 8));
    const unsigned nb = (unsigned)((gr.npix + 255) / 256);
    for (size_t j = 0; j < members[g].size(); ++j) {
      k_tau_add<<<nb, 256, 0, s>>>(pixA64[members[g][j]].as<double>(), tau.as<double>(), gr.npix,
                                   j == 0);
      CMBWS_LAUNCH_CHECK();
    }
    CMBWS_TRY(sums.alloc((size_t)gr.nring * 16));
    k_alpha_sums<<<gr.nring, 256, 0, s>>>(tau.as<double>(), gr.ring_off.as<int64_t>(),
                                          gr.ring_w64.as<double>(), sums.as<double2>());
    CMBWS_LAUNCH_CHECK();
    std::vector<double> hs(2 * (size_t)gr.nring);
    CMBWS_CUDA(cudaMemcpyAsync(hs.data(), sums.p, hs.size() * 8, cudaMemcpyDeviceToHost, s));
    CMBWS_CUDA(cudaStreamSynchronize(s));
    double s1 = 0.0, s2 = 0.0;
    for (int r = 0; r < gr.nring; ++r) {
      s1 += hs[2 * r];
      s2 += hs[2 * r + 1];
    }
    P->alpha[g] = std::sqrt(s2 / s1);
    CMBWS_TRY(P->pixM64[g].alloc((size_t)gr.npix * 8));
    CMBWS_TRY(P->pixM32[g].alloc((size_t)gr.npix * 4));
    k_tplus_factors<<<gr.nring, 256, 0, s>>>(tau.as<double>(), gr.ring_off.as<int64_t>(),
                                             gr.ring_w64.as<double>(), P->alpha[g] * P->alpha[g],
                                             P->pixM64[g].as<double>(), P->pixM32[g].as<float>());
    CMBWS_LAUNCH_CHECK();
    CMBWS_CUDA(cudaStreamSynchronize(s));  // tau is freed at the end of this iteration
  }

  // ---- rows sharing a grid are transformed together ----
  size_t part_bytes = part.bytes;
  for (int g = 0; g < nrow; ++g) {
    Grid* gr = grids[members[g][0]];
    int gi = -1;
    for (size_t i = 0; i < P->groups.size(); ++i)
      if (P->groups[i].grid == gr && P->groups[i].nmaps < kMaxMaps) gi = (int)i;
    if (gi < 0) {
      P->groups.emplace_back();
      P->groups.back().grid = gr;
      gi = (int)P->groups.size() - 1;
    }
    Group& G = P->groups[gi];
    P->row_group[g] = gi;
    P->row_slot[g] = G.nmaps;
    G.bands[G.nmaps++] = g;
  }
  for (Group& G : P->groups) {
    const Grid& gr = *G.grid;
    const int64_t nlm = nlm_of(gr.lmax);
    CMBWS_TRY(G.alm.alloc((size_t)G.nmaps * nlm * 16));
    CMBWS_TRY(G.F.alloc((size_t)G.nmaps * gr.nring * (gr.lmax + 1) * 16));
    CMBWS_TRY(G.out.alloc((size_t)G.nmaps * nlm * 16));
    for (int pr : {CMBWS_FP64, CMBWS_FP32, CMBWS_FP32X2})
      part_bytes = std::max(part_bytes, legendre_adjoint_part_bytes(gr, pr, G.nmaps));
  }
  if (part_bytes > part.bytes) CMBWS_TRY(part.ensure(part_bytes));

  // ---- U' per l: merged rows (rank-one fits) and the prior rows; U'^+ by SVD ----
  const int nc = ncomp, nr = nrow + nc;
  std::vector<double> Up((size_t)(Lup + 1) * nc * nr, 0.0);
  for (int l = 0; l <= Lup; ++l) {
    std::vector<int> act;
    for (int k = 0; k < nc; ++k)
      if (l <= Lk[k]) act.push_back(k);
    const int na = (int)act.size();
    if (!na) continue;
    std::vector<double> U((size_t)nr * na, 0.0), Pl, S((size_t)na * na), v;
    for (int g = 0; g < nrow; ++g) {
      std::fill(S.begin(), S.end(), 0.0);
      for (int nu : members[g]) {
        if (l > Lnu[nu]) continue;
        const double ab = alpha[nu] * beam_h[beam_off_h[nu] + l];
        for (int a = 0; a < na; ++a)
          for (int b = 0; b < na; ++b)
            S[(size_t)a * na + b] += ab * qpre_h[nu * nc + act[a]] * ab * qpre_h[nu * nc + act[b]];
      }
      double lam = 0.0;
      sym_top_eig(S, na, &lam, v);
      const double sc = std::sqrt(std::max(lam, 0.0));
      for (int a = 0; a < na; ++a) U[(size_t)g * na + a] = sc * v[a];
    }
    for (int a = 0; a < na; ++a) U[(size_t)(nrow + act[a]) * na + a] = cisq_h[clOff_h[act[a]] + l];
    if (!pinv_jacobi(U, nr, na, 1e-12, Pl)) {
      set_error("cmbws_model_merge_precond: at l = %d a component has neither data nor prior", l);
      return CMBWS_ERR_SINGULAR;
    }
    for (int a = 0; a < na; ++a)
      for (int j = 0; j < nr; ++j) Up[((size_t)l * nc + act[a]) * nr + j] = Pl[(size_t)a * nr + j];
  }
  CMBWS_TRY(P->d_Up.upload(Up.data(), Up.size() * 8));
  merged = std::move(P);
  nsht_M = 2 * nrow;
  return CMBWS_OK;
}

}  // namespace cmbws

using namespace cmbws;

extern "C" int cmbws_model_merge_precond(cmbws_model mh, const int* group, void* stream) {
  clear_error();
  Model* M = as_model(mh);
  if (refuse_sharded(M, "cmbws_model_merge_precond")) return CMBWS_ERR_ARG;
  if (!M) {
    set_error("cmbws_model_merge_precond: invalid model");
    return CMBWS_ERR_ARG;
  }
  return M->merge_precond(group, (cudaStream_t)stream);
}
