// Legendre stage in double-float arithmetic (pairs of FP32 values, ~48-bit
// significand) for FP64-accurate transforms on the FP32 pipe.
//
// On GB300 the FP64 rate is 1/61 of the FP32 FMA rate, so the FP64 applies
// that certify the refined solution dominate a mixed-precision solve.  The
// same recurrence and contraction as legendre.cu run here with every value
// carried as hi + lo (Dekker / Knuth error-free transformations with FMA):
//   * recurrence  mu_l = (A_l - A_l y) mu_{l-1} - mu_{l-2}  in double-float;
//   * contraction per map part: the exact product (TwoProd plus the cross
//     terms) is added to a hi accumulator with TwoSum, and the rounding errors
//     of both go to a lo accumulator (the compensated dot product "Dot2" of
//     Ogita, Rump and Oishi 2005), renormalised once at the end.
// Coefficients and adjoint outputs keep the FP64 layout (double2); the ring spectra
// between this stage and the ring FFTs are double-float pairs (df2, 16 bytes like
// double2), which the double-float ring FFT (ringfft.cu) reads and writes directly,
// so no FP64 conversion sits between the two stages.
#include <climits>

#include "common.h"
#include "dfloat.h"

namespace cmbws {

namespace {

template <int NM, int R, int NT, int CH>
__global__ void __launch_bounds__(NT)
k_leg_synth_df(const double2* __restrict__ alm, int64_t alm_stride, const float2* __restrict__ Acoef,
               const int* __restrict__ ls_tab, const double2* __restrict__ st,
               const double* __restrict__ yr, const int2* __restrict__ pring,
               df2* __restrict__ F, int64_t F_stride, int L, int npair,
               const float4* __restrict__ ck, const int64_t* __restrict__ ck_base) {
  static_assert(R == 1, "one ring pair per thread (its checkpoint column)");
  __shared__ __align__(16) float2 sA[CH];
  __shared__ __align__(16) float4 sa[NM][CH];
  __shared__ int s_lo;
  const int m = blockIdx.y;
  const int64_t lmo = lm_off(L, m) - m;
  const int pbase = blockIdx.x * NT * R + threadIdx.x;

  int ls[R];
  df y[R], mu1[R], mu2[R], i0[R], i1[R];
  float eh[R][NM][2], el[R][NM][2], oh[R][NM][2], ol[R][NM][2];
  int mylo = INT_MAX;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int p = pbase + i * NT;
    if (p < npair) {
      ls[i] = ls_tab[(int64_t)m * npair + p];
      y[i] = df_from(yr[p]);
      const double2 s2 = st[(int64_t)m * npair + p];
      i0[i] = df_from(s2.x);
      i1[i] = df_from(s2.y);
    } else {
      ls[i] = INT_MAX;
      y[i] = {0.f, 0.f};
      i0[i] = i1[i] = {0.f, 0.f};
    }
    mylo = min(mylo, ls[i]);
    mu1[i] = mu2[i] = {0.f, 0.f};
#pragma unroll
    for (int k = 0; k < NM; ++k)
#pragma unroll
      for (int c = 0; c < 2; ++c) eh[i][k][c] = el[i][k][c] = oh[i][k][c] = ol[i][k][c] = 0.f;
  }
  if (threadIdx.x == 0) s_lo = INT_MAX;
  __syncthreads();
  atomicMin(&s_lo, mylo);
  __syncthreads();
  const int lo = s_lo;
  int nxt = mylo;
  const int wlo = __reduce_min_sync(0xffffffffu, mylo);  // first start of this warp's pairs
  // Checkpoints of the double-float adjoint: the FP64-computed pair (mu_l0, mu_l0+1) at every
  // l0 = m + kChunkDf c (zero before the pair's start).  At those l the recurrence values are
  // read instead of computed, so the recurrence runs for half of the steps; the column of the
  // next chunk is loaded one chunk ahead.
  const int nckd = (L - m + kChunkDf) / kChunkDf;
  const float4* ckc = (pbase < npair) ? ck + ck_base[m] + (int64_t)pbase * nckd : nullptr;
  static_assert(kChunkDf == 4, "one checkpoint every second step of two");
  float4 pre = make_float4(0.f, 0.f, 0.f, 0.f);
  int pre_l = -1;
  bool pre_ok = false;

  for (int c0 = lo; c0 <= L; c0 += CH) {
    __syncthreads();
    for (int j = threadIdx.x; j < CH; j += NT) {
      const int l = c0 + j;
      const bool ok = l <= L;
      sA[j] = ok ? Acoef[lmo + l] : make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        double2 v = make_double2(0.0, 0.0);
        if (ok) v = alm[k * alm_stride + lmo + l];
        const df re = df_from(v.x), im = df_from(v.y);
        sa[k][j] = make_float4(re.h, re.l, im.h, im.l);
      }
    }
    __syncthreads();
    // the last chunk stops at L (even count); warps whose pairs start later skip the chunk
    const int jn = min(CH, (L - c0 + 2) & ~1);
    if (c0 + jn <= wlo) continue;
    for (int j = 0; j < jn; j += 2) {
      const int l = c0 + j;
      const float2 a0 = sA[j], a1 = sA[j + 1];
      const df A0 = {a0.x, a0.y}, A1 = {a1.x, a1.y};
      df ma[R], mb[R];
      if (((l - m) & 3) == 0 && ckc) {  // a checkpoint at l (uniform but for the last pairs)
        const float4 cv = pre_ok && pre_l == l ? pre : ckc[(l - m) >> 2];
        ma[0] = {cv.x, cv.y};
        mb[0] = {cv.z, cv.w};
      } else {
        if (ckc && l + 2 <= L) {  // the next checkpoint, read while this step computes
          pre = ckc[(l + 2 - m) >> 2];
          pre_l = l + 2;
          pre_ok = true;
        }
#pragma unroll
        for (int i = 0; i < R; ++i) {
          ma[i] = df_recur(A0, y[i], mu1[i], mu2[i]);
          mb[i] = df_recur(A1, y[i], ma[i], mu1[i]);
        }
      }
      if (l == nxt) {
        int nn = INT_MAX;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (ls[i] == l) {
            ma[i] = i0[i];
            mb[i] = i1[i];
          }
          if (ls[i] > l) nn = min(nn, ls[i]);
        }
        nxt = nn;
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        mu2[i] = ma[i];
        mu1[i] = mb[i];
      }
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        const float4 v0 = sa[k][j], v1 = sa[k][j + 1];
        const df r0 = {v0.x, v0.y}, q0 = {v0.z, v0.w}, r1 = {v1.x, v1.y}, q1 = {v1.z, v1.w};
#pragma unroll
        for (int i = 0; i < R; ++i) {
          dot2_acc(eh[i][k][0], el[i][k][0], ma[i], r0);
          dot2_acc(eh[i][k][1], el[i][k][1], ma[i], q0);
          dot2_acc(oh[i][k][0], ol[i][k][0], mb[i], r1);
          dot2_acc(oh[i][k][1], ol[i][k][1], mb[i], q1);
        }
      }
    }
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int p = pbase + i * NT;
    if (p >= npair) continue;
    const int2 rr = pring[p];
#pragma unroll
    for (int k = 0; k < NM; ++k) {
      const df er{eh[i][k][0], el[i][k][0]}, ei{eh[i][k][1], el[i][k][1]};
      const df orr{oh[i][k][0], ol[i][k][0]}, oi{oh[i][k][1], ol[i][k][1]};
      F[k * F_stride + (int64_t)rr.x * (L + 1) + m] = df2{er + orr, ei + oi};
      if (rr.y >= 0) F[k * F_stride + (int64_t)rr.y * (L + 1) + m] = df2{er - orr, ei - oi};
    }
  }
}

template <int NM, int PT>
struct AdjCkDfWarp {  // one warp's double-buffered tile
  float2 eo[2][PT][4 * NM];
  float2 y[2][PT];
  int ls[2][PT];
  double2 st[2][PT];
  float4 ck[2][PT][32];
};

// Adjoint in double-float from chunk checkpoints (the FP32 kernel's scheme in
// legendre.cu with every value a hi + lo pair): one thread per chunk of kChunkDf values
// of l loops over all ring pairs, restarting the recurrence at its chunk from the
// double-float checkpoints, and accumulates each output (l, m, part) with the
// compensated dot product.  Each output has one owner and a fixed summation order, so
// no cross-thread reduction or partial-sum buffer is needed.
// four CTAs (16 warps) per SM: 128 registers per thread, measured 2.5 % faster than three
template <int NM, int NT, int PT>
__global__ void __launch_bounds__(NT, 4)
k_leg_adj_ck_df(const float2* __restrict__ eo, const float2* __restrict__ Acoef,
                const int* __restrict__ ls_tab, const double2* __restrict__ st,
                const float2* __restrict__ yr, const float4* __restrict__ ck,
                const int64_t* __restrict__ ck_base, const int2* __restrict__ tasks, int ntask,
                const int* __restrict__ tmin, const double* __restrict__ c64,
                double2* __restrict__ out, int64_t nlm, int L, int npair) {
  static_assert(kTileMinPT % PT == 0, "a tile must lie inside one entry of the tile-start table");
  constexpr int P = 2 * NM;
  constexpr int K = kChunkDf;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  AdjCkDfWarp<NM, PT>& S = reinterpret_cast<AdjCkDfWarp<NM, PT>*>(smem_raw)[warp];
  // every warp takes one task (32 consecutive chunks of one m); warps of a CTA are independent
  const int task = blockIdx.x * (NT / 32) + warp;
  if (task >= ntask) return;  // warp-uniform: no block barrier below
  const int2 tk = tasks[task];
  const int m = tk.x;
  const int nck = (L - m + K) / K;
  const int cw = tk.y;  // first chunk of this warp
  const int c = cw + lane;
  const bool valid = c < nck;
  const int l0 = m + K * c;
  const int64_t lmo = lm_off(L, m) - m;
  df Al[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const float2 a = (valid && l0 + j <= L) ? Acoef[lmo + l0 + j] : make_float2(0.f, 0.f);
    Al[j] = {a.x, a.y};
  }
  float ah[K][P], al[K][P];
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int q = 0; q < P; ++q) ah[j][q] = al[j][q] = 0.f;
  const float4* ckc = ck + ck_base[m] + c;  // + p * nck
  const float2* eom = eo + (int64_t)m * npair * 2 * P;
  const int ntile = (npair + PT - 1) / PT;
  // tiles whose pairs all start after the warp's last l add nothing and are not staged;
  // tmin holds the smallest start of each kTileMinPT pairs, a lower bound for this tile's
  const int llast = min(L, m + K * (cw + 32) - 1);
  const int* tm = tmin + (int64_t)m * ((npair + kTileMinPT - 1) / kTileMinPT);
  auto next_tile = [&](int t) {
    while (t < ntile && tm[t * PT / kTileMinPT] > llast) ++t;
    return t;
  };

  auto stage = [&](int t, int bf) {
    const int p0 = t * PT;
    const int np = min(PT, npair - p0);
    const float2* src = eom + (int64_t)p0 * 2 * P;
    for (int i = lane; i < np * P; i += 32) cp_async16(&S.eo[bf][0][0] + 2 * i, src + 2 * i);
    for (int i = lane; i < np; i += 32) {
      cp_async8(&S.y[bf][i], yr + p0 + i);
      cp_async4(&S.ls[bf][i], ls_tab + (int64_t)m * npair + p0 + i);
      cp_async16(&S.st[bf][i], st + (int64_t)m * npair + p0 + i);
    }
    if (valid)
      for (int i = 0; i < np; ++i) cp_async16(&S.ck[bf][i][lane], ckc + (int64_t)(p0 + i) * nck);
    cp_async_commit();
  };

  int t = next_tile(0);
  if (t < ntile) stage(t, 0);
  for (int k = 0; t < ntile; ++k) {
    const int tn = next_tile(t + 1);
    if (tn < ntile) {
      stage(tn, (k + 1) & 1);
      cp_async_wait<1>();
    } else {
      cp_async_wait<0>();
    }
    __syncwarp();
    if (valid) {
      const int bf = k & 1;
      const int np = min(PT, npair - t * PT);
      for (int i = 0; i < np; ++i) {
        const int jinj = S.ls[bf][i] - l0;  // where the pair starts, relative to the chunk
        if (jinj > K - 1) continue;         // the pair starts after this chunk
        const float4 cv = S.ck[bf][i][lane];
        df ma = {cv.x, cv.y}, mb = {cv.z, cv.w};
        const float2 yy = S.y[bf][i];
        const df yv = {yy.x, yy.y};
        const float2* e = S.eo[bf][i];
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const float2 ev = e[q], ov = e[P + q];
          dot2_acc(ah[0][q], al[0][q], ma, df{ev.x, ev.y});
          dot2_acc(ah[1][q], al[1][q], mb, df{ov.x, ov.y});
        }
#pragma unroll
        for (int j = 2; j < K; j += 2) {
          df na = df_recur(Al[j], yv, mb, ma);
          df nb = df_recur(Al[j + 1], yv, na, mb);
          if (j == jinj) {
            const double2 sv = S.st[bf][i];
            na = df_from(sv.x);
            nb = df_from(sv.y);
          }
          ma = na;
          mb = nb;
#pragma unroll
          for (int q = 0; q < P; ++q) {
            const float2 ev = e[q], ov = e[P + q];
            dot2_acc(ah[j][q], al[j][q], ma, df{ev.x, ev.y});
            dot2_acc(ah[j + 1][q], al[j + 1][q], mb, df{ov.x, ov.y});
          }
        }
      }
    }
    __syncwarp();  // buffer k & 1 is restaged two iterations later
    t = tn;
  }
  if (!valid) return;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int l = l0 + j;
    if (l > L) break;
    const int64_t i = lmo + l;
    const double cc = c64[i];
#pragma unroll
    for (int k = 0; k < NM; ++k)
      out[k * nlm + i] = make_double2(cc * ((double)ah[j][2 * k] + (double)al[j][2 * k]),
                                      cc * ((double)ah[j][2 * k + 1] + (double)al[j][2 * k + 1]));
  }
}

constexpr int kSR = 1, kSNT = 128, kSCH = 128;

template <int NM>
int launch_synth_df(const Grid& g, const void* alm, int64_t as, void* F, int64_t fs, cudaStream_t s) {
  const int L = g.lmax;
  dim3 grd((g.npair + kSNT * kSR - 1) / (kSNT * kSR), L + 1);
  ProfScope ps(PROF_LEG_SYNTH, s, 2, leg_work(g, NM));
  k_leg_synth_df<NM, kSR, kSNT, kSCH><<<grd, kSNT, 0, s>>>(
      (const double2*)alm, as, g.A2f.as<float2>(), g.ls.as<int>(), g.st64.as<double2>(),
      g.y64.as<double>(), g.pair_ring.as<int2>(), (df2*)F, fs, L, g.npair, g.ck64.as<float4>(),
      g.ck64_base.as<int64_t>());
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

constexpr int kANT = 128, kAPT = 8;

template <int NM>
int launch_adj_ck_df(const Grid& g, const float2* eo, double* out, cudaStream_t s) {
  const int L = g.lmax;
  const int64_t nlm = nlm_of(L);
  dim3 grd((g.nwtdf + kANT / 32 - 1) / (kANT / 32));
  constexpr size_t sm = sizeof(AdjCkDfWarp<NM, kAPT>) * (kANT / 32);
  auto kern = k_leg_adj_ck_df<NM, kANT, kAPT>;
  CMBWS_TRY(ensure_dyn_smem((const void*)kern, sm));
  ProfScope ps(PROF_LEG_ADJ, s, 2, leg_work(g, NM));
  kern<<<grd, kANT, sm, s>>>(eo, g.A2f.as<float2>(), g.ls.as<int>(), g.st64.as<double2>(),
                             g.y2f.as<float2>(), g.ck64.as<float4>(), g.ck64_base.as<int64_t>(),
                             g.wtdf.as<int2>(), g.nwtdf, g.ls_tmin.as<int>(), g.c64.as<double>(),
                             (double2*)out, nlm, L, g.npair);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

}  // namespace


int legendre_synth_df(const Grid& g, int nmaps, const void* alm, void* F, cudaStream_t s) {
  CMBWS_TRY(grid_ensure_ck64(g));
  const int64_t as = nlm_of(g.lmax), fs = (int64_t)g.nring * (g.lmax + 1);
  for (int k0 = 0; k0 < nmaps; k0 += 4) {
    const int nm = nmaps - k0 < 4 ? nmaps - k0 : 4;
    const void* a = (const double2*)alm + k0 * as;
    void* f = (double2*)F + k0 * fs;
    int st;
    switch (nm) {
      case 1: st = launch_synth_df<1>(g, a, as, f, fs, s); break;
      case 2: st = launch_synth_df<2>(g, a, as, f, fs, s); break;
      case 3: st = launch_synth_df<3>(g, a, as, f, fs, s); break;
      default: st = launch_synth_df<4>(g, a, as, f, fs, s); break;
    }
    if (st != CMBWS_OK) return st;
  }
  return CMBWS_OK;
}

int legendre_adj_df_ck(const Grid& g, int nm, const void* eo, double* out, cudaStream_t s) {
  CMBWS_TRY(grid_ensure_ck64(g));
  const float2* e = (const float2*)eo;
  switch (nm) {
    case 1: return launch_adj_ck_df<1>(g, e, out, s);
    case 2: return launch_adj_ck_df<2>(g, e, out, s);
    default: return launch_adj_ck_df<3>(g, e, out, s);
  }
}

}  // namespace cmbws
