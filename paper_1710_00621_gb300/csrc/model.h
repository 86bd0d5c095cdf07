// Model object behind cmbws_model: the description of Sec. 2.2 resident on the
// device, the U^+ blocks of Sec. 3.3 and the workspaces of the apply chains.
#pragma once

#include <memory>

#include "common.h"

namespace cmbws {

constexpr int kMaxComp = 8;    // components
constexpr int kMaxBands = 64;  // observations (e.g. detector subsets of the frequency channels)
constexpr int kMaxMaps = 8;    // bands transformed together on one grid

struct MaskMG;  // mask-restricted multigrid preconditioner (maskmg.cu)

// Variable mixing pair (nu, k), device view (array of nobs * ncomp in device memory).
struct PairDev {
  const double2* out;  // chain output of the pair (internal layout of its mixing grid, FP64)
  void* alm64;         // chain input slot, FP64 / FP32X2 layout
  void* alm32;         // chain input slot, FP32 layout
  const double* c;     // c_lm of the mixing grid
  int L;               // mixing-grid band-limit
  int var;             // 1 if the pair is variable
};

// Device view of the harmonic-space model tables (kernel argument by value).
struct HarmDev {
  int ncomp, nobs, Lup;
  const int* compL;        // [ncomp] L_k
  const int64_t* compOff;  // [ncomp] offset of component k in a stacked vector
  const double* q;         // [nobs][ncomp]
  const double* beam;      // b_{nu,l} at beam[beamOff[nu] + l]
  const int64_t* beamOff;
  const double* cinv;      // C_{k,l}^-1 at cinv[clOff[k] + l] (0 = no prior)
  const double* cisq;      // C_{k,l}^-1/2
  const int64_t* clOff;
  const double* Up;        // U^+ [Lup+1][ncomp][nobs+ncomp]
  const PairDev* pairs;    // [nobs * ncomp] variable-mixing pairs (var = 0: scalar q)
  uint64_t own;            // bands whose terms this model adds (bit nu; all unless sharded)
  int prior_on;            // 1 if this model adds the prior terms (always unless sharded)
};

struct GroupDev {
  int L, nmaps;
  int bands[kMaxMaps];
  const double* c;         // c_lm of the group's grid
  void* alm;               // group input, internal layout (T2)
  int64_t nlm;
};

struct BandDev {
  int L[kMaxBands];
  const double2* out[kMaxBands];  // adjoint-chain result of band nu (internal layout, FP64)
  const double* c[kMaxBands];     // c_lm of band nu's grid
  void* alm[kMaxBands];           // chain input slot of band nu (T2)
};

struct MixGroupDev {
  int L, npairs;
  int nu[kMaxMaps], k[kMaxMaps];
  const double* c;
  void* alm;
  int64_t nlm;
};

struct Group {
  Grid* grid = nullptr;
  int nmaps = 0;
  int bands[kMaxMaps] = {0};
  DevMem alm;  // [nmaps][nlm] complex, sized for FP64
  DevMem F;    // [nmaps][nring][L+1] complex, sized for FP64
  DevMem out;  // [nmaps][nlm] complex FP64
};

// Observation merging in the preconditioner (App. A.3, merge.cu): M_PI over merged rows of U
// (groups of bands on one grid) instead of one row per band.
struct MergedPrec {
  int nrow = 0;
  std::vector<int> row_of_band;
  std::vector<Group> groups;              // rows sharing a grid; bands[] holds row ids
  std::vector<int> row_group, row_slot;
  std::vector<DevMem> pixM64, pixM32;     // T^+ pixel factors alpha_G^2 w^2 / tau_G per row
  std::vector<double> alpha;              // alpha_G (Eq. optimal-alpha of tau_G)
  DevMem d_Up;                            // U'^+ [Lup+1][ncomp][nrow + ncomp]
};

struct Model {
  int ncomp = 0, nobs = 0, prec = 0;
  std::vector<int> Lk, Lnu;
  std::vector<int64_t> compOff;
  int64_t nvec = 0;
  int Lcomp = 0, Lall = 0, Lup = 0;
  std::vector<Grid*> grids;
  std::vector<Group> groups;
  std::vector<int> band_group, band_slot;
  std::vector<double> alpha;
  std::vector<DevMem> pixA64, pixA32, pixM64, pixM32, tausq;
  DevMem d_compL, d_compOff, d_q, d_beam, d_beamOff, d_cinv, d_cisq, d_clOff, d_Up;
  std::vector<int64_t> beam_off_h;  // host copy of the beam offsets
  DevMem part, tprior, pixtmp;
  int nsht_A = 0, nsht_M = 0;
  long long n_sht = 0;  // SHTs executed since creation (paper's counting)

  // gradient-term workspace (grad.cu): band maps and per-block partial sums
  DevMem gradmaps, gradpart;
  DevMem gradmix, gradmixout, gradmixpart;  // mixing-map gradients (grad.cu)

  // CG workspace (cg.cu)
  DevMem cg_r, cg_z, cg_p, cg_q, cg_d, cg_x, cg_red;
  double* cg_host = nullptr;  // pinned: the PCG scalars read back once per iteration
  // per-iteration record of the last solve (cmbws_cg_history): ||r_i|| / ||b|| and, while a
  // reference solution is set (cmbws_cg_track_error), ||x_i - x_true|| / ||x_true||
  std::vector<double> hist_res, hist_err;
  DevMem cg_xtrue;
  bool track_err = false;
  // checkpoint of an FP64 solve stopped by its iteration cap (cmbws_cg_checkpointing):
  // the correction d, residual r and direction p, and the scalars of the next iteration
  bool ck_on = false, ck_valid = false;
  DevMem cg_ck;  // [3][nvec]
  int ck_iters = 0;
  double ck_rz = 0.0, ck_rr = 0.0;

  // spatially variable mixing (Eq. Q)
  int nmix = 0;
  std::vector<Group> mgroups;             // pairs sharing a mixing grid; bands[] holds pair ids
  std::vector<DevMem> pixQ64, pixQ32;     // q_{nu,k}(n) w(n) per pair id (empty if scalar)
  DevMem d_pairs;                         // PairDev [nobs * ncomp]

  // block-diagonal comparison preconditioner M_diag (diagprec.cu), built on first use:
  // per band diag(Y^T N^-1 Y) as (cos, sin) per (l, m), and the inverse blocks
  DevMem d_qpre;                 // [nobs][ncomp] scalars of the preconditioners (Eq. optimal-q)
  DevMem dg_D, dg_inv;
  bool dg_ready = false;
  int build_diag(cudaStream_t s);
  int apply_diag(const double* r, double* z, cudaStream_t s);

  // constrained-realization draws (sampling.cu): on-device omega_2 and omega_1 of every band,
  // and the right-hand side of the draw
  DevMem cr_w, cr_b;
  int cr_draw_rhs(const double* const* d, uint64_t seed, uint64_t sample, double* b,
                  cudaStream_t s);

  // observation merging (merge.cu): when set, apply_precond runs over the merged rows
  std::unique_ptr<MergedPrec> merged;
  std::vector<double> beam_h, cisq_h, qpre_h;  // host copies of b_{nu,l}, C^-1/2, q (U rows)
  std::vector<int64_t> clOff_h;
  int merge_precond(const int* group, cudaStream_t s);
  int apply_precond_merged(const double* r, double* z, int prec, cudaStream_t s);

  // CUDA graphs of the operator applies inside PCG (cg.cu), per (operator, precision,
  // input, output): the first apply runs eagerly, the second is captured, later ones replay.
  // Dropped whenever the model's internal buffers change.
  struct OpGraph {
    int op = 0, prec = 0;
    const double* in = nullptr;
    double* out = nullptr;
    int calls = 0;
    bool failed = false;
    cudaGraphExec_t exec = nullptr;
    long long nsht = 0;  // SHTs of one apply (the replay adds them to n_sht)
  };
  bool use_graphs = false;
  std::vector<OpGraph> graphs;
  void drop_graphs();

  // band sharding (cmbws_model_set_shard): the bands and the prior terms this model adds to
  // apply_A, apply_precond and rhs; the sum over the shards of all models is the full operator
  bool shard_on = false;
  uint64_t shard_own = ~0ull;
  bool shard_prior = true;
  bool group_owned(const Group& G) const {
    for (int j = 0; j < G.nmaps; ++j)
      if ((shard_own >> G.bands[j]) & 1) return true;
    return false;
  }

  // mask-restricted preconditioners (Sec. 4), applied with M_PI when precond = 2
  std::vector<MaskMG*> masks;
  int vcycle = 0;  // V-cycle of the mask preconditioners: 0 basic, 1 optimized (J ~ I)
  // arithmetic of the transforms of M_PI inside the solvers (-1: the model's own)
  int prec_M = -1;
  ~Model();

  HarmDev harm() const;
  BandDev bands_dev(int prec) const;
  int group_chain(Group& G, int prec, int which, cudaStream_t s);
  int mix_chain(Group& G, int prec, cudaStream_t s);
  int mixvar_forward(int prec, const double* x, cudaStream_t s);
  int mixvar_adjoint(int prec, cudaStream_t s);
  // pixel maps on mixing group G's grid ([pair][npix], FP64) of x_{k_j} (comp) or of the band
  // outputs times the beam, B_nu u_nu (band), synthesized in arithmetic prec
  int mixvar_maps_comp(Group& G, int prec, const double* x, double* maps, cudaStream_t s);
  int mixvar_maps_band(Group& G, int prec, double* maps, cudaStream_t s);
  int mix_forward(Group& G, int prec, const double* x, cudaStream_t s);
  int project(const double* x, double* const* d, int prec, cudaStream_t s);
  int apply_A(const double* x, double* y, int prec, cudaStream_t s);
  int apply_precond(const double* r, double* z, int prec, cudaStream_t s);
  int rhs(const double* const* d, const double* const* w1, const double* w2, double* b,
          cudaStream_t s);
};

int model_create(const cmbws_model_desc* desc, int prec, cudaStream_t s, Model** out);

// Calls other than cmbws_apply_A, cmbws_apply_precond, cmbws_rhs, cmbws_project and the
// sharded solve refuse a sharded model (their results would be one shard's partial terms).
inline bool refuse_sharded(const Model* M, const char* fn) {
  if (M && M->shard_on) {
    set_error("%s: the model is sharded (cmbws_model_set_shard); use cmbws_cg_solve_sharded", fn);
    return true;
  }
  return false;
}

// the model behind a handle, or nullptr if the handle is not a live model
inline Model* as_model(const void* h) {
  return handle_live(HANDLE_MODEL, h) ? const_cast<Model*>(static_cast<const Model*>(h)) : nullptr;
}

// One-sided Jacobi SVD pseudo-inverse of an (nr x nc) row-major matrix, out (nc x nr);
// singular values below rcond * max are dropped.  false if a column is zero.
bool pinv_jacobi(const std::vector<double>& Uin, int nr, int nc, double rcond,
                 std::vector<double>& out);

void mask_mg_destroy(MaskMG* p);
int mask_mg_apply(MaskMG& mg, Model& M, const double* r, double* z, cudaStream_t s);

}  // namespace cmbws
