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
// Inputs and outputs keep the FP64 layouts of the FP64 path (coefficients
// double2, ring spectra double2, partial sums double), so only this stage
// changes; the ring FFTs run in FP64.
#include <climits>

#include "common.h"

namespace cmbws {

namespace {

struct df {
  float h, l;
};

__device__ __forceinline__ df two_sum(float a, float b) {
  const float s = a + b;
  const float bb = s - a;
  const float e = (a - (s - bb)) + (b - bb);
  return {s, e};
}
__device__ __forceinline__ df quick_two_sum(float a, float b) {
  const float s = a + b;
  return {s, b - (s - a)};
}
__device__ __forceinline__ df df_from(double v) {
  const float h = (float)v;
  return {h, (float)(v - (double)h)};
}
__device__ __forceinline__ double df_to(df a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ df df_mul(df a, df b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  return quick_two_sum(p, e);
}
__device__ __forceinline__ df df_sub(df a, df b) {
  const df s = two_sum(a.h, -b.h);
  return quick_two_sum(s.h, s.l + (a.l - b.l));
}
// a * b - c
__device__ __forceinline__ df df_fms(df a, df b, df c) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const df s = two_sum(p, -c.h);
  return quick_two_sum(s.h, s.l + (e - c.l));
}
// compensated accumulation acc_h + acc_l += a * b
__device__ __forceinline__ void dot2_acc(float& acc_h, float& acc_l, df a, df b) {
  const float p = a.h * b.h;
  float e = fmaf(a.h, b.h, -p);
  e = fmaf(a.h, b.l, e);
  e = fmaf(a.l, b.h, e);
  const df s = two_sum(acc_h, p);
  acc_h = s.h;
  acc_l += s.l + e;
}

__device__ __forceinline__ df df_recur(df A, df y, df m1, df m2) {
  const df ax = df_sub(A, df_mul(A, y));
  return df_fms(ax, m1, m2);
}

template <int NM, int R, int NT, int CH>
__global__ void __launch_bounds__(NT)
k_leg_synth_df(const double2* __restrict__ alm, int64_t alm_stride, const double* __restrict__ Acoef,
               const int* __restrict__ ls_tab, const double2* __restrict__ st,
               const double* __restrict__ yr, const int2* __restrict__ pring,
               double2* __restrict__ F, int64_t F_stride, int L, int npair) {
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

  for (int c0 = lo; c0 <= L; c0 += CH) {
    __syncthreads();
    for (int j = threadIdx.x; j < CH; j += NT) {
      const int l = c0 + j;
      const bool ok = l <= L;
      const df a = df_from(ok ? Acoef[lmo + l] : 0.0);
      sA[j] = make_float2(a.h, a.l);
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        double2 v = make_double2(0.0, 0.0);
        if (ok) v = alm[k * alm_stride + lmo + l];
        const df re = df_from(v.x), im = df_from(v.y);
        sa[k][j] = make_float4(re.h, re.l, im.h, im.l);
      }
    }
    __syncthreads();
    for (int j = 0; j < CH; j += 2) {
      const int l = c0 + j;
      const float2 a0 = sA[j], a1 = sA[j + 1];
      const df A0 = {a0.x, a0.y}, A1 = {a1.x, a1.y};
      df ma[R], mb[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        ma[i] = df_recur(A0, y[i], mu1[i], mu2[i]);
        mb[i] = df_recur(A1, y[i], ma[i], mu1[i]);
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
      const double er = (double)eh[i][k][0] + (double)el[i][k][0];
      const double ei = (double)eh[i][k][1] + (double)el[i][k][1];
      const double orr = (double)oh[i][k][0] + (double)ol[i][k][0];
      const double oi = (double)oh[i][k][1] + (double)ol[i][k][1];
      F[k * F_stride + (int64_t)rr.x * (L + 1) + m] = make_double2(er + orr, ei + oi);
      if (rr.y >= 0) F[k * F_stride + (int64_t)rr.y * (L + 1) + m] = make_double2(er - orr, ei - oi);
    }
  }
}

__device__ __forceinline__ df df_add(df a, df b) {
  const df s = two_sum(a.h, b.h);
  return quick_two_sum(s.h, s.l + (a.l + b.l));
}

// Sum NV double-float values over the 32 lanes of a warp (reduce-scatter):
// afterwards lane q holds the sums of flat indices [q NV/32, (q+1) NV/32).
template <int NV>
__device__ __forceinline__ void warp_reduce_scatter_df(df (&v)[NV], int lane) {
  static_assert(NV % 32 == 0, "NV must be a multiple of 32");
#pragma unroll
  for (int s = 0; s < 5; ++s) {
    const int o = 16 >> s;
    const int h = (NV >> s) / 2;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const df send = up ? v[i] : v[i + h];
      const df keep = up ? v[i + h] : v[i];
      df recv;
      recv.h = __shfl_xor_sync(0xffffffffu, send.h, o);
      recv.l = __shfl_xor_sync(0xffffffffu, send.l, o);
      v[i] = df_add(keep, recv);
    }
  }
}

// Adjoint: per l-chunk each thread sums its R pairs' products in double-float
// (compensated), a double-float warp reduce-scatter adds the 32 lanes, and the
// warps of the CTA are added in FP64 in shared memory.
template <int NM, int R, int NT, int CH>
__global__ void __launch_bounds__(NT)
k_leg_adj_df(const double2* __restrict__ F, int64_t F_stride, const float2* __restrict__ Acoef,
             const int* __restrict__ ls_tab, const double2* __restrict__ st,
             const double* __restrict__ yr, const int2* __restrict__ pring, double* __restrict__ part,
             int64_t nlm, int L, int npair) {
  constexpr int P = 2 * NM;
  constexpr int NV0 = CH * P;
  constexpr int NV = (NV0 + 31) / 32 * 32;
  constexpr int PER = NV / 32;
  constexpr int NW = NT / 32;
  __shared__ double red[NW][NV];
  __shared__ int s_lo;
  const int m = blockIdx.y;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int64_t lmo = lm_off(L, m) - m;
  const float2* Am = Acoef + lmo;
  double* pout = part + (int64_t)blockIdx.x * P * nlm + lmo;
  const int pbase = blockIdx.x * NT * R + threadIdx.x;

  int ls[R];
  df y[R], mu1[R], mu2[R], i0[R], i1[R];
  df ev[R][P], ov[R][P];
  int mylo = INT_MAX;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int p = pbase + i * NT;
    mu1[i] = mu2[i] = {0.f, 0.f};
    if (p < npair) {
      ls[i] = ls_tab[(int64_t)m * npair + p];
      y[i] = df_from(yr[p]);
      const double2 s2 = st[(int64_t)m * npair + p];
      i0[i] = df_from(s2.x);
      i1[i] = df_from(s2.y);
      const int2 rr = pring[p];
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        const double2 gn = F[k * F_stride + (int64_t)rr.x * (L + 1) + m];
        const double2 gs = rr.y >= 0 ? F[k * F_stride + (int64_t)rr.y * (L + 1) + m]
                                     : make_double2(0.0, 0.0);
        ev[i][2 * k] = df_from(gn.x + gs.x);
        ev[i][2 * k + 1] = df_from(gn.y + gs.y);
        ov[i][2 * k] = df_from(rr.y >= 0 ? gn.x - gs.x : gn.x);
        ov[i][2 * k + 1] = df_from(rr.y >= 0 ? gn.y - gs.y : gn.y);
      }
    } else {
      ls[i] = INT_MAX;
      y[i] = {0.f, 0.f};
      i0[i] = i1[i] = {0.f, 0.f};
#pragma unroll
      for (int c = 0; c < P; ++c) ev[i][c] = ov[i][c] = {0.f, 0.f};
    }
    mylo = min(mylo, ls[i]);
  }
  if (threadIdx.x == 0) s_lo = INT_MAX;
  __syncthreads();
  atomicMin(&s_lo, mylo);
  __syncthreads();
  const int lo = s_lo;
  int nxt = mylo;
  {
    const int lend = min(lo, L + 1);
    for (int l = m + threadIdx.x; l < lend; l += NT)
#pragma unroll
      for (int pp = 0; pp < P; ++pp) pout[pp * nlm + l] = 0.0;
  }
  for (int c0 = lo; c0 <= L; c0 += CH) {
    df v[NV];
#pragma unroll
    for (int q = 0; q < NV; ++q) v[q] = {0.f, 0.f};
#pragma unroll
    for (int j = 0; j < CH; j += 2) {
      const int l = c0 + j;
      const float2 a0 = (l <= L) ? Am[l] : make_float2(0.f, 0.f);
      const float2 a1 = (l + 1 <= L) ? Am[l + 1] : make_float2(0.f, 0.f);
      const df A0 = {a0.x, a0.y}, A1 = {a1.x, a1.y};
      df ma[R], mb[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        ma[i] = df_recur(A0, y[i], mu1[i], mu2[i]);
        mb[i] = df_recur(A1, y[i], ma[i], mu1[i]);
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
#pragma unroll
        for (int c = 0; c < P; ++c) {
          dot2_acc(v[j * P + c].h, v[j * P + c].l, ma[i], ev[i][c]);
          dot2_acc(v[(j + 1) * P + c].h, v[(j + 1) * P + c].l, mb[i], ov[i][c]);
        }
      }
    }
    warp_reduce_scatter_df<NV>(v, lane);
#pragma unroll
    for (int q = 0; q < PER; ++q) red[warp][lane * PER + q] = (double)v[q].h + (double)v[q].l;
    __syncthreads();
    for (int f = threadIdx.x; f < NV0; f += NT) {
      double sum = 0.0;
#pragma unroll
      for (int w = 0; w < NW; ++w) sum += red[w][f];
      const int l = c0 + f / P;
      if (l <= L) pout[(f % P) * nlm + l] = sum;
    }
    __syncthreads();
  }
}

constexpr int kSR = 1, kSNT = 128, kSCH = 128;
constexpr int kAR = 2, kANT = 256, kACH = 4;

template <int NM>
int launch_synth_df(const Grid& g, const void* alm, int64_t as, void* F, int64_t fs, cudaStream_t s) {
  const int L = g.lmax;
  dim3 grd((g.npair + kSNT * kSR - 1) / (kSNT * kSR), L + 1);
  ProfScope ps(PROF_LEG_SYNTH, s, 2, 4.0 * g.npair * (double)nlm_of(L) * (NM + 1));
  k_leg_synth_df<NM, kSR, kSNT, kSCH><<<grd, kSNT, 0, s>>>(
      (const double2*)alm, as, g.A64.as<double>(), g.ls.as<int>(), g.st64.as<double2>(),
      g.y64.as<double>(), g.pair_ring.as<int2>(), (double2*)F, fs, L, g.npair);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

template <int NM>
int launch_adj_df(const Grid& g, const void* F, int64_t fs, double* part, cudaStream_t s) {
  const int L = g.lmax;
  const int64_t nlm = nlm_of(L);
  dim3 grd((g.npair + kANT * kAR - 1) / (kANT * kAR), L + 1);
  ProfScope ps(PROF_LEG_ADJ, s, 2, 4.0 * g.npair * (double)nlm * (NM + 1));
  k_leg_adj_df<NM, kAR, kANT, kACH><<<grd, kANT, 0, s>>>(
      (const double2*)F, fs, g.A2f.as<float2>(), g.ls.as<int>(), g.st64.as<double2>(),
      g.y64.as<double>(), g.pair_ring.as<int2>(), part, nlm, L, g.npair);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

}  // namespace

int legendre_df_adj_nblk(const Grid& g) { return (g.npair + kANT * kAR - 1) / (kANT * kAR); }

int legendre_synth_df(const Grid& g, int nmaps, const void* alm, void* F, cudaStream_t s) {
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

// F -> partial sums (FP64, [nblk][2 nm][nlm]) for maps k0 .. k0 + nm - 1
int legendre_adj_df_chunk(const Grid& g, int nm, const void* F, double* part, cudaStream_t s) {
  const int64_t fs = (int64_t)g.nring * (g.lmax + 1);
  switch (nm) {
    case 1: return launch_adj_df<1>(g, F, fs, part, s);
    case 2: return launch_adj_df<2>(g, F, fs, part, s);
    case 3: return launch_adj_df<3>(g, F, fs, part, s);
    default: return launch_adj_df<4>(g, F, fs, part, s);
  }
  (void)fs;
}

}  // namespace cmbws
