// Associated-Legendre stage of the spherical harmonic transform (Sec. 2.1),
// the dominant cost of every apply of A and M_PI (Sec. 3.3 counts SHTs).
//
// Synthesis, per m and ring pair (theta, pi - theta):
//   F_m(theta) = sum_l lambda_lm(theta) a_lm,  with lambda_lm(pi - theta) = (-1)^(l+m) lambda_lm(theta),
// so E = sum over l+m even and O = sum over l+m odd give F_north = E + O and
// F_south = E - O from one recurrence.  Adjoint synthesis is the transpose:
//   a_lm = sum_pairs lambda_lm(theta) (E-part or O-part of the ring spectra).
//
// Design (CUDA cores; the recurrence costs two operations per (l, m, pair),
// the contraction two FMAs per map):
// * one CTA per (m, block of ring pairs); each thread owns R pairs, walks l
//   upwards two steps at a time (even/odd partners) and starts each pair at
//   its precomputed first significant l (start values injected there);
// * synthesis: the coefficients of the current l-chunk are staged in shared
//   memory and read as broadcasts; every map of the grid group shares one
//   recurrence (NM maps per launch);
// * adjoint: for a chunk of CH values of l the recurrence values of the CTA's
//   pairs go to a shared-memory tile and the contraction over pairs runs as a
//   small GEMM from shared memory (register-blocked row pairs x pair slices),
//   the slices added in shared memory; each CTA writes its partial sums, which
//   a second kernel adds in a fixed order (deterministic) and scales by c_lm.
#include <climits>
#include <type_traits>

#include "common.h"

namespace cmbws {

namespace {

template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };

constexpr unsigned kFull = 0xffffffffu;

template <typename T, int NM, int R, int NT, int CH>
__global__ void __launch_bounds__(NT)
k_leg_synth(const typename V2<T>::t* __restrict__ alm, int64_t alm_stride,
            const T* __restrict__ Acoef, const float* __restrict__ brs,
            const int* __restrict__ ls_tab,
            const typename V2<T>::t* __restrict__ st, const T* __restrict__ yr,
            const int2* __restrict__ pring, typename V2<T>::t* __restrict__ F, int64_t F_stride,
            int L, int npair, int nring) {
  using T2 = typename V2<T>::t;
  constexpr bool kF32 = std::is_same<T, float>::value;
  __shared__ __align__(16) T sA[CH];
  __shared__ __align__(16) T2 sa[NM][CH];
  __shared__ __align__(16) float sBRS[kF32 ? 3 : 1][kF32 ? CH : 1];  // difference form (FP32)
  __shared__ int s_lo;

  const int m = blockIdx.y;
  const int64_t lmo = lm_off(L, m) - m;  // index of (m, l) is lmo + l
  const int pbase = blockIdx.x * NT * R + threadIdx.x;

  int ls[R];
  T y[R], mu1[R], mu2[R];
  T2 inj[R];
  T eR[R][NM], eI[R][NM], oR[R][NM], oI[R][NM];
  int mylo = INT_MAX;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int p = pbase + i * NT;
    if (p < npair) {
      ls[i] = ls_tab[(int64_t)m * npair + p];
      y[i] = yr[p];
      inj[i] = st[(int64_t)m * npair + p];
    } else {
      ls[i] = INT_MAX;
      y[i] = 0;
      inj[i].x = inj[i].y = 0;
    }
    mylo = min(mylo, ls[i]);
    mu1[i] = mu2[i] = 0;
#pragma unroll
    for (int k = 0; k < NM; ++k) eR[i][k] = eI[i][k] = oR[i][k] = oI[i][k] = 0;
  }
  if (threadIdx.x == 0) s_lo = INT_MAX;
  __syncthreads();
  atomicMin(&s_lo, mylo);
  __syncthreads();
  const int lo = s_lo;
  int nxt = mylo;  // next l at which one of this thread's pairs starts
  // first l at which a pair of this warp starts: the warp skips every chunk before it (its
  // recurrence values are zero there; warps without a valid pair skip all chunks)
  const int wlo = __reduce_min_sync(kFull, mylo);
  // warps holding a polar ring pair run the difference form (FP32 only; warp-uniform)
  bool polar = false;
  if constexpr (kF32) {
    bool mine = false;
#pragma unroll
    for (int i = 0; i < R; ++i) mine |= (pbase + i * NT < npair) && (float)y[i] < kPolarY;
    polar = __any_sync(kFull, mine);
  }

  for (int c0 = lo; c0 <= L; c0 += CH) {
    __syncthreads();
    for (int j = threadIdx.x; j < CH; j += NT) {
      const int l = c0 + j;
      const bool ok = l <= L;
      sA[j] = ok ? Acoef[lmo + l] : T(0);
      if constexpr (kF32) {
#pragma unroll
        for (int q = 0; q < 3; ++q) sBRS[q][j] = ok ? brs[3 * (lmo + l) + q] : 0.f;
      }
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        T2 v;
        v.x = v.y = 0;
        if (ok) v = alm[k * alm_stride + lmo + l];
        sa[k][j] = v;
      }
    }
    __syncthreads();
    // values of l in this chunk (the last chunk stops at L; an even count, the partner of
    // an odd tail reads the zeros staged beyond L)
    const int jn = min(CH, (L - c0 + 2) & ~1);
    if (c0 + jn <= wlo) continue;
    if constexpr (kF32) {
      if (polar) {
        // mu2 holds e_{l-1} = mu_{l-1} - R_{l-1} mu_{l-2} in this form
#pragma unroll 2
        for (int j = 0; j < jn; j += 2) {
          const int l = c0 + j;
          const T A0 = sA[j], A1 = sA[j + 1];
          const float B0 = sBRS[0][j], B1 = sBRS[0][j + 1], R0 = sBRS[1][j], R1 = sBRS[1][j + 1];
          const float S0 = sBRS[2][j], S1 = sBRS[2][j + 1];
          T ma[R], mb[R];
#pragma unroll
          for (int i = 0; i < R; ++i) {
            T e = fmaf(fmaf(-A0, y[i], B0), mu1[i], S0 * mu2[i]);
            ma[i] = fmaf(R0, mu1[i], e);
            e = fmaf(fmaf(-A1, y[i], B1), ma[i], S1 * e);
            mb[i] = fmaf(R1, ma[i], e);
            mu2[i] = e;
          }
          if (l == nxt) {
            int nn = INT_MAX;
#pragma unroll
            for (int i = 0; i < R; ++i) {
              if (ls[i] == l) {
                ma[i] = inj[i].x;
                mb[i] = inj[i].y;
                mu2[i] = fmaf(-R1, inj[i].x, inj[i].y);
              }
              if (ls[i] > l) nn = min(nn, ls[i]);
            }
            nxt = nn;
          }
#pragma unroll
          for (int i = 0; i < R; ++i) mu1[i] = mb[i];
#pragma unroll
          for (int k = 0; k < NM; ++k) {
            const T2 a0 = sa[k][j], a1 = sa[k][j + 1];
#pragma unroll
            for (int i = 0; i < R; ++i) {
              eR[i][k] += ma[i] * a0.x;
              eI[i][k] += ma[i] * a0.y;
              oR[i][k] += mb[i] * a1.x;
              oI[i][k] += mb[i] * a1.y;
            }
          }
        }
        continue;
      }
    }
#pragma unroll 2
    for (int j = 0; j < jn; j += 2) {
      const int l = c0 + j;
      const T A0 = sA[j], A1 = sA[j + 1];
      T ma[R], mb[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        ma[i] = fma(-A0, y[i], A0) * mu1[i] - mu2[i];
        mb[i] = fma(-A1, y[i], A1) * ma[i] - mu1[i];
      }
      if (l == nxt) {
        int nn = INT_MAX;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (ls[i] == l) {
            ma[i] = inj[i].x;
            mb[i] = inj[i].y;
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
        const T2 a0 = sa[k][j], a1 = sa[k][j + 1];
#pragma unroll
        for (int i = 0; i < R; ++i) {
          eR[i][k] += ma[i] * a0.x;
          eI[i][k] += ma[i] * a0.y;
          oR[i][k] += mb[i] * a1.x;
          oI[i][k] += mb[i] * a1.y;
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
      T2 fn, fs;
      fn.x = eR[i][k] + oR[i][k];
      fn.y = eI[i][k] + oI[i][k];
      F[k * F_stride + (int64_t)rr.x * (L + 1) + m] = fn;
      if (rr.y >= 0) {
        fs.x = eR[i][k] - oR[i][k];
        fs.y = eI[i][k] - oI[i][k];
        F[k * F_stride + (int64_t)rr.y * (L + 1) + m] = fs;
      }
    }
  }
}

// Adjoint as a per-chunk GEMM in shared memory.  For a chunk of CH values of l:
//   phase 1: thread i runs the recurrence of its R pairs and stores mu[pair][l] (tile muT);
//   phase 2: D[l][part] = sum_pairs mu[pair][l] * EO[pair][parity(l)][part], each thread
//            owning two rows (an even/odd l pair) and a slice of KS pairs, 2P accumulators;
//   phase 3: the NSLICE slice partials are added in shared memory and written out.
// Shared memory: muT [NR][CH+2], EO [NR][2P], red [NSLICE][CH/2][2P].
template <typename T, int NM, int R, int NT, int CH>
__global__ void __launch_bounds__(NT)
k_leg_adj2(const typename V2<T>::t* __restrict__ F, int64_t F_stride, const T* __restrict__ Acoef,
           const int* __restrict__ ls_tab, const typename V2<T>::t* __restrict__ st,
           const T* __restrict__ yr, const int2* __restrict__ pring, T* __restrict__ part,
           int64_t nlm, int L, int npair) {
  using T2 = typename V2<T>::t;
  constexpr int P = 2 * NM;
  constexpr int NR = NT * R;
  constexpr int CHP = CH + 2;
  constexpr int NJ = CH / 2;
  constexpr int NSLICE = NT / NJ;
  constexpr int KS = NR / NSLICE;
  static_assert(NT % NJ == 0 && NR % NSLICE == 0, "tile shape");
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* muT = reinterpret_cast<T*>(smem_raw);
  T* eo = muT + NR * CHP;
  T* red = eo + NR * 2 * P;
  __shared__ int s_lo;

  const int m = blockIdx.y;
  const int tid = threadIdx.x;
  const int64_t lmo = lm_off(L, m) - m;
  const T* Am = Acoef + lmo;
  T* pout = part + (int64_t)blockIdx.x * P * nlm + lmo;
  const int p0 = blockIdx.x * NR;

  // per-pair recurrence state (pairs tid + i NT of this block)
  int ls[R];
  T y[R], mu1[R], mu2[R];
  T2 inj[R];
  int mylo = INT_MAX;
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const int lp = tid + i * NT;
    const int p = p0 + lp;
    mu1[i] = mu2[i] = 0;
    T* e = eo + lp * 2 * P;
    if (p < npair) {
      ls[i] = ls_tab[(int64_t)m * npair + p];
      y[i] = yr[p];
      inj[i] = st[(int64_t)m * npair + p];
      const int2 rr = pring[p];
#pragma unroll
      for (int k = 0; k < NM; ++k) {
        const T2 gn = F[k * F_stride + (int64_t)rr.x * (L + 1) + m];
        T2 gs;
        gs.x = gs.y = 0;
        if (rr.y >= 0) gs = F[k * F_stride + (int64_t)rr.y * (L + 1) + m];
        e[2 * k] = gn.x + gs.x;
        e[2 * k + 1] = gn.y + gs.y;
        e[P + 2 * k] = rr.y >= 0 ? gn.x - gs.x : gn.x;
        e[P + 2 * k + 1] = rr.y >= 0 ? gn.y - gs.y : gn.y;
      }
    } else {
      ls[i] = INT_MAX;
      y[i] = 0;
      inj[i].x = inj[i].y = 0;
#pragma unroll
      for (int q = 0; q < 2 * P; ++q) e[q] = 0;
    }
    mylo = min(mylo, ls[i]);
  }
  if (tid == 0) s_lo = INT_MAX;
  __syncthreads();
  atomicMin(&s_lo, mylo);
  __syncthreads();
  const int lo = s_lo;
  int nxt = mylo;
  {
    const int lend = min(lo, L + 1);
    for (int l = m + tid; l < lend; l += NT)
#pragma unroll
      for (int pp = 0; pp < P; ++pp) pout[pp * nlm + l] = T(0);
  }
  const int jrow = tid % NJ, slice = tid / NJ;

  for (int c0 = lo; c0 <= L; c0 += CH) {
    // phase 1: recurrence into the tile
#pragma unroll 4
    for (int j = 0; j < CH; j += 2) {
      const int l = c0 + j;
      const T A0 = (l <= L) ? Am[l] : T(0);
      const T A1 = (l + 1 <= L) ? Am[l + 1] : T(0);
      T ma[R], mb[R];
#pragma unroll
      for (int i = 0; i < R; ++i) {
        ma[i] = fma(-A0, y[i], A0) * mu1[i] - mu2[i];
        mb[i] = fma(-A1, y[i], A1) * ma[i] - mu1[i];
      }
      if (l == nxt) {
        int nn = INT_MAX;
#pragma unroll
        for (int i = 0; i < R; ++i) {
          if (ls[i] == l) {
            ma[i] = inj[i].x;
            mb[i] = inj[i].y;
          }
          if (ls[i] > l) nn = min(nn, ls[i]);
        }
        nxt = nn;
      }
#pragma unroll
      for (int i = 0; i < R; ++i) {
        mu2[i] = ma[i];
        mu1[i] = mb[i];
        T2 v;
        v.x = ma[i];
        v.y = mb[i];
        *reinterpret_cast<T2*>(muT + (tid + i * NT) * CHP + j) = v;
      }
    }
    __syncthreads();
    // phase 2: rows (2 jrow, 2 jrow + 1) over the pairs of this slice
    T acc[2 * P];
#pragma unroll
    for (int q = 0; q < 2 * P; ++q) acc[q] = 0;
    const int pb = slice * KS;
#pragma unroll 4
    for (int pp = 0; pp < KS; ++pp) {
      const T2 mv = *reinterpret_cast<const T2*>(muT + (pb + pp) * CHP + 2 * jrow);
      const T* e = eo + (pb + pp) * 2 * P;
#pragma unroll
      for (int q = 0; q < P; ++q) {
        acc[q] += mv.x * e[q];
        acc[P + q] += mv.y * e[P + q];
      }
    }
    T* rs = red + (slice * NJ + jrow) * 2 * P;
#pragma unroll
    for (int q = 0; q < 2 * P; ++q) rs[q] = acc[q];
    __syncthreads();
    // phase 3: add the slices; output index f = row-pair j, q (q < P: even row, else odd)
    for (int f = tid; f < NJ * 2 * P; f += NT) {
      const int j = f / (2 * P), q = f % (2 * P);
      T sum = 0;
#pragma unroll 8
      for (int sl = 0; sl < NSLICE; ++sl) sum += red[(sl * NJ + j) * 2 * P + q];
      const int l = c0 + 2 * j + (q >= P ? 1 : 0);
      if (l <= L) pout[(q % P) * nlm + l] = sum;
    }
    __syncthreads();
  }
}


// FP32 adjoint from chunk checkpoints: one thread per chunk of kChunk values of l
// (a CTA covers NT consecutive chunks of one m) loops over every ring pair of the
// grid.  Each pair's recurrence restarts at the chunk from the stored FP64-computed
// values (setup.cu), so no thread needs another thread's sums: each output (l, m) is
// owned by one thread and summed over the pairs in a fixed order.
// Tiles of PT pairs are staged in shared memory with cp.async, double-buffered: the
// per-pair even/odd parts E, O (written by the forward ring FFT), y, the start index and values,
// and each thread's own column of checkpoints, so the HBM reads of the next tile
// overlap the arithmetic of the current one.
// E/O parts of every (pair, m): eo[(m * npair + p) * 2P + q], q < P even-l parts (north +
// south), q >= P odd-l parts (north - south), parts = (re, im) per map.
template <int NM, int PT>
struct AdjCkWarp {  // one warp's double-buffered tile
  float eo[2][PT][4 * NM];
  float y[2][PT];
  int ls[2][PT];
  float2 st[2][PT];
  float2 ck[2][PT][32];
};

template <int NM, int NT, int PT>
__global__ void __launch_bounds__(NT)
k_leg_adj_ck(const float* __restrict__ eo, const float* __restrict__ Acoef,
             const int* __restrict__ ls_tab, const float2* __restrict__ st,
             const float* __restrict__ yr, const float2* __restrict__ ck,
             const int64_t* __restrict__ ck_base, const int2* __restrict__ tasks, int ntask,
             const int* __restrict__ tmin, const double* __restrict__ c64,
             double2* __restrict__ out, int64_t nlm, int L, int npair) {
  static_assert(PT == kTileMinPT, "the tile-start table is built for kTileMinPT pairs per tile");
  constexpr int P = 2 * NM;
  constexpr int K = kChunk;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  AdjCkWarp<NM, PT>& S = reinterpret_cast<AdjCkWarp<NM, PT>*>(smem_raw)[warp];
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
  float Al[K];
#pragma unroll
  for (int j = 0; j < K; ++j) Al[j] = (valid && l0 + j <= L) ? Acoef[lmo + l0 + j] : 0.f;
  float acc[K][P];
#pragma unroll
  for (int j = 0; j < K; ++j)
#pragma unroll
    for (int q = 0; q < P; ++q) acc[j][q] = 0.f;
  const float2* ckc = ck + ck_base[m] + c;  // + p * nck
  const float* eom = eo + (int64_t)m * npair * 2 * P;
  const int ntile = (npair + PT - 1) / PT;
  // Pairs are not sorted by start; a tile whose pairs all start after the warp's last l
  // (tmin, the smallest start of the tile) adds nothing to this warp's outputs and is not
  // staged.  Pairs of a visited tile that have not started are skipped one by one.
  const int llast = min(L, m + K * (cw + 32) - 1);
  const int* tm = tmin + (int64_t)m * ntile;
  auto next_tile = [&](int t) {
    while (t < ntile && tm[t] > llast) ++t;
    return t;
  };

  auto stage = [&](int t, int bf) {
    const int p0 = t * PT;
    const int np = min(PT, npair - p0);
    const float* src = eom + (int64_t)p0 * 2 * P;
    for (int i = lane; i < np * NM; i += 32) cp_async16(&S.eo[bf][0][0] + 4 * i, src + 4 * i);
    for (int i = lane; i < np; i += 32) {
      cp_async4(&S.y[bf][i], yr + p0 + i);
      cp_async4(&S.ls[bf][i], ls_tab + (int64_t)m * npair + p0 + i);
      cp_async8(&S.st[bf][i], st + (int64_t)m * npair + p0 + i);
    }
    if (valid)
      for (int i = 0; i < np; ++i) cp_async8(&S.ck[bf][i][lane], ckc + (int64_t)(p0 + i) * nck);
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
        const int lsp = S.ls[bf][i];
        if (lsp > l0 + K - 1) continue;  // the pair starts after this chunk
        const float2 cv = S.ck[bf][i][lane];
        float ma = cv.x, mb = cv.y;
        if (lsp == l0) {
          ma = S.st[bf][i].x;
          mb = S.st[bf][i].y;
        }
        const float yv = S.y[bf][i];
        const float* e = S.eo[bf][i];
#pragma unroll
        for (int q = 0; q < P; ++q) {
          acc[0][q] += ma * e[q];
          acc[1][q] += mb * e[P + q];
        }
#pragma unroll
        for (int j = 2; j < K; j += 2) {
          float na = fmaf(-Al[j], yv, Al[j]) * mb - ma;
          float nb = fmaf(-Al[j + 1], yv, Al[j + 1]) * na - mb;
          if (l0 + j == lsp) {
            na = S.st[bf][i].x;
            nb = S.st[bf][i].y;
          }
          ma = na;
          mb = nb;
#pragma unroll
          for (int q = 0; q < P; ++q) {
            acc[j][q] += ma * e[q];
            acc[j + 1][q] += mb * e[P + q];
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
      out[k * nlm + i] = make_double2(cc * (double)acc[j][2 * k], cc * (double)acc[j][2 * k + 1]);
  }
}

template <typename T>
__global__ void k_adj_reduce(const T* __restrict__ part, int nblk, int64_t nlm, int nm,
                             const double* __restrict__ c, double2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int k = blockIdx.y;
  if (i >= nlm) return;
  double re = 0.0, im = 0.0;
  for (int b = 0; b < nblk; ++b) {
    const T* pb = part + ((int64_t)b * 2 * nm + 2 * k) * nlm;
    re += (double)pb[i];
    im += (double)pb[nlm + i];
  }
  const double cc = c[i];
  out[(int64_t)k * nlm + i] = make_double2(cc * re, cc * im);
}

// Launch configuration per precision.
template <typename T> struct Cfg;
template <> struct Cfg<float> {
  static constexpr int SR = 2, SNT = 128, SCH = 256;  // synthesis
  static constexpr int AR = 2, ANT = 256, ACH = 32;   // adjoint (shared-memory GEMM form)
};
template <> struct Cfg<double> {
  static constexpr int SR = 2, SNT = 128, SCH = 256;
  static constexpr int AR = 1, ANT = 256, ACH = 16;
};

template <typename T, int NM>
constexpr size_t adj2_smem() {
  using C = Cfg<T>;
  constexpr int P = 2 * NM, NR = C::ANT * C::AR, NJ = C::ACH / 2, NSLICE = C::ANT / NJ;
  return sizeof(T) * ((size_t)NR * (C::ACH + 2) + (size_t)NR * 2 * P + (size_t)NSLICE * NJ * 2 * P);
}

template <typename T, int NM, int R, int NT>
int launch_synth_rn(const Grid& g, const void* alm, int64_t alm_stride, void* F, int64_t F_stride,
                    cudaStream_t s) {
  using C = Cfg<T>;
  using T2 = typename V2<T>::t;
  const int L = g.lmax;
  dim3 grd((g.npair + NT * R - 1) / (NT * R), L + 1);
  const T* A = std::is_same<T, double>::value ? (const T*)g.A64.p : (const T*)g.A32.p;
  const T2* st = std::is_same<T, double>::value ? (const T2*)g.st64.p : (const T2*)g.st32.p;
  const T* yr = std::is_same<T, double>::value ? (const T*)g.y64.p : (const T*)g.y32.p;
  ProfScope ps(PROF_LEG_SYNTH, s, sizeof(T) == 8, leg_work(g, NM));
  k_leg_synth<T, NM, R, NT, C::SCH><<<grd, NT, 0, s>>>(
      (const T2*)alm, alm_stride, A, g.BRS32.as<float>(), g.ls.as<int>(), st, yr,
      g.pair_ring.as<int2>(), (T2*)F, F_stride, L, g.npair, g.nring);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

// Tile variants of the synthesis (ring pairs per thread R, threads per CTA NT): variant 0 is
// the default for large grids; the others trade pairs per CTA (fewer idle lanes on grids
// with few ring pairs) against coefficient reuse (R = 4: a shared-memory broadcast serves
// four recurrences).  The autotuner picks one per (grid, precision, maps).
constexpr int kSynthVariants = 4;

template <typename T, int NM>
int launch_synth_variant(int v, const Grid& g, const void* alm, int64_t as, void* F, int64_t fs,
                         cudaStream_t s) {
  switch (v) {
    case 1: return launch_synth_rn<T, NM, 1, 128>(g, alm, as, F, fs, s);
    case 2: return launch_synth_rn<T, NM, 1, 64>(g, alm, as, F, fs, s);
    case 3: return launch_synth_rn<T, NM, 4, 64>(g, alm, as, F, fs, s);
    default: return launch_synth_rn<T, NM, 2, 128>(g, alm, as, F, fs, s);
  }
}

// heuristic: the smallest CTA (in ring pairs) that holds all pairs of the grid
inline int synth_heuristic(const Grid& g) { return g.npair <= 64 ? 2 : g.npair <= 128 ? 1 : 0; }

template <typename T, int NM>
int launch_synth(const Grid& g, const void* alm, int64_t as, void* F, int64_t fs, cudaStream_t s) {
  int v = 0;
  const int prec = std::is_same<T, double>::value ? CMBWS_FP64 : CMBWS_FP32;
  CMBWS_TRY(autotune_pick(g, synth_tune_key(prec, NM), kSynthVariants, synth_heuristic(g),
                          [&](int vv) { return launch_synth_variant<T, NM>(vv, g, alm, as, F, fs, s); },
                          s, &v));
  return launch_synth_variant<T, NM>(v, g, alm, as, F, fs, s);
}

template <typename T>
int adj_nblk(const Grid& g) {
  using C = Cfg<T>;
  return (g.npair + C::ANT * C::AR - 1) / (C::ANT * C::AR);
}

template <int NM>
int launch_adj_ck(const Grid& g, const float* eo, double* out, cudaStream_t s) {
  // one warp per CTA: the warps are independent tasks (no CTA barrier), so an SM holds as
  // many as its registers allow (16 at 120 registers) instead of whole 4-warp CTAs (12 at 130):
  // 3.29 against 3.77 ms per Nside-1024 launch of 3 maps
  constexpr int NT = 32, PT = 16;
  const int L = g.lmax;
  const int64_t nlm = nlm_of(L);
  dim3 grd((g.nwt32 + NT / 32 - 1) / (NT / 32));
  constexpr size_t sm = sizeof(AdjCkWarp<NM, PT>) * (NT / 32);
  auto kern = k_leg_adj_ck<NM, NT, PT>;
  CMBWS_TRY(ensure_dyn_smem((const void*)kern, sm));
  ProfScope ps(PROF_LEG_ADJ, s, 0, leg_work(g, NM));
  kern<<<grd, NT, sm, s>>>(eo, g.A32.as<float>(), g.ls.as<int>(), g.st32.as<float2>(),
                           g.y32.as<float>(), g.ck32.as<float2>(), g.ck_base.as<int64_t>(),
                           g.wt32.as<int2>(), g.nwt32, g.ls_tmin.as<int>(), g.c64.as<double>(),
                           (double2*)out, nlm, L, g.npair);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

template <typename T, int NM>
int launch_adj(const Grid& g, const void* F, int64_t F_stride, T* part, double* out, cudaStream_t s) {
  using C = Cfg<T>;
  using T2 = typename V2<T>::t;
  const int L = g.lmax;
  const int64_t nlm = nlm_of(L);
  const int nblk = adj_nblk<T>(g);
  dim3 grd(nblk, L + 1);
  const T* A = std::is_same<T, double>::value ? (const T*)g.A64.p : (const T*)g.A32.p;
  const T2* st = std::is_same<T, double>::value ? (const T2*)g.st64.p : (const T2*)g.st32.p;
  const T* yr = std::is_same<T, double>::value ? (const T*)g.y64.p : (const T*)g.y32.p;
  {
    constexpr size_t sm = adj2_smem<T, NM>();
    auto kern = k_leg_adj2<T, NM, C::AR, C::ANT, C::ACH>;
    CMBWS_TRY(ensure_dyn_smem((const void*)kern, sm));
    ProfScope ps(PROF_LEG_ADJ, s, sizeof(T) == 8, leg_work(g, NM));
    kern<<<grd, C::ANT, sm, s>>>((const T2*)F, F_stride, A, g.ls.as<int>(), st, yr,
                                 g.pair_ring.as<int2>(), part, nlm, L, g.npair);
    CMBWS_LAUNCH_CHECK();
  }
  dim3 rg((unsigned)((nlm + 255) / 256), NM);
  ProfScope ps(PROF_LEG_RED, s, sizeof(T) == 8);
  k_adj_reduce<T><<<rg, 256, 0, s>>>(part, nblk, nlm, NM, g.c64.as<double>(), (double2*)out);
  CMBWS_LAUNCH_CHECK();
  return CMBWS_OK;
}

template <typename T>
int synth_dispatch(const Grid& g, int nmaps, const void* alm, void* F, cudaStream_t s) {
  using T2 = typename V2<T>::t;
  const int64_t as = nlm_of(g.lmax), fs = (int64_t)g.nring * (g.lmax + 1);
  for (int k0 = 0; k0 < nmaps; k0 += 4) {
    const int nm = nmaps - k0 < 4 ? nmaps - k0 : 4;
    const void* a = (const T2*)alm + k0 * as;
    void* f = (T2*)F + k0 * fs;
    int st = CMBWS_OK;
    switch (nm) {
      case 1: st = launch_synth<T, 1>(g, a, as, f, fs, s); break;
      case 2: st = launch_synth<T, 2>(g, a, as, f, fs, s); break;
      case 3: st = launch_synth<T, 3>(g, a, as, f, fs, s); break;
      default: st = launch_synth<T, 4>(g, a, as, f, fs, s); break;
    }
    if (st != CMBWS_OK) return st;
  }
  return CMBWS_OK;
}

template <typename T>
int adj_dispatch(const Grid& g, int nmaps, const void* F, void* part, double* out, cudaStream_t s) {
  using T2 = typename V2<T>::t;
  const int64_t nlm = nlm_of(g.lmax), fs = (int64_t)g.nring * (g.lmax + 1);
  for (int k0 = 0; k0 < nmaps; k0 += 4) {
    const int nm = nmaps - k0 < 4 ? nmaps - k0 : 4;
    const void* f = (const T2*)F + k0 * fs;
    double* o = out + 2 * k0 * nlm;
    int st = CMBWS_OK;
    switch (nm) {
      case 1: st = launch_adj<T, 1>(g, f, fs, (T*)part, o, s); break;
      case 2: st = launch_adj<T, 2>(g, f, fs, (T*)part, o, s); break;
      case 3: st = launch_adj<T, 3>(g, f, fs, (T*)part, o, s); break;
      default: st = launch_adj<T, 4>(g, f, fs, (T*)part, o, s); break;
    }
    if (st != CMBWS_OK) return st;
  }
  return CMBWS_OK;
}

// FP32 adjoints from the adjoint input (eo layout, chunks of 4 maps) that the ring FFT wrote
int adj_dispatch_ck(const Grid& g, int nmaps, const float* eo, double* out, cudaStream_t s) {
  const int64_t nlm = nlm_of(g.lmax), cs = (int64_t)(g.lmax + 1) * g.npair * 4;
  for (int k0 = 0; k0 < nmaps; k0 += 4) {
    const int nm = nmaps - k0 < 4 ? nmaps - k0 : 4;
    const float* e = eo + k0 * cs;
    double* o = out + 2 * k0 * nlm;
    int st = CMBWS_OK;
    switch (nm) {
      case 1: st = launch_adj_ck<1>(g, e, o, s); break;
      case 2: st = launch_adj_ck<2>(g, e, o, s); break;
      case 3: st = launch_adj_ck<3>(g, e, o, s); break;
      default: st = launch_adj_ck<4>(g, e, o, s); break;
    }
    if (st != CMBWS_OK) return st;
  }
  return CMBWS_OK;
}

}  // namespace

int legendre_synth(const Grid& g, int prec, int nmaps, const void* alm, void* F, cudaStream_t s) {
  if (prec == CMBWS_FP32X2) return legendre_synth_df(g, nmaps, alm, F, s);
  if (is_tc(prec)) return legendre_synth_tc(g, prec, nmaps, alm, F, s);
  if (prec == CMBWS_FP64) return synth_dispatch<double>(g, nmaps, alm, F, s);
  return synth_dispatch<float>(g, nmaps, alm, F, s);
}

size_t legendre_adjoint_part_bytes(const Grid& g, int prec, int nmaps) {
  // the adjoint input (eo layout) of every map: (L+1) npair 4 scalars per map
  const size_t eo = (size_t)nmaps * (g.lmax + 1) * g.npair * 4;
  if (is_f32(prec)) return eo * sizeof(float);
  if (prec == CMBWS_FP32X2) return eo * 2 * sizeof(float);
  const int nm = nmaps < 4 ? nmaps : 4;  // FP64: per-CTA partial sums of one launch
  return (size_t)adj_nblk<double>(g) * 2 * nm * nlm_of(g.lmax) * sizeof(double);
}

int legendre_adjoint(const Grid& g, int prec, int nmaps, const void* F, void* part,
                     size_t part_bytes, double* out, cudaStream_t s) {
  if (part_bytes < legendre_adjoint_part_bytes(g, prec, nmaps)) {
    set_error("legendre_adjoint: partial-sum buffer too small");
    return CMBWS_ERR_ARG;
  }
  if (prec == CMBWS_FP32X2) {
    const int64_t nlm = nlm_of(g.lmax), cs = (int64_t)(g.lmax + 1) * g.npair * 4;
    // at most 3 maps per launch: 4 maps' double-float accumulators exceed the register file
    for (int k0 = 0; k0 < nmaps; k0 += 3) {
      const int nm = nmaps - k0 < 3 ? nmaps - k0 : 3;
      CMBWS_TRY(legendre_adj_df_ck(g, nm, (const float2*)part + k0 * cs, out + 2 * k0 * nlm, s));
    }
    return CMBWS_OK;
  }
  if (prec == CMBWS_FP64) return adj_dispatch<double>(g, nmaps, F, part, out, s);
  if (prec == CMBWS_BF16 || prec == CMBWS_BF16X3)
    return legendre_adjoint_tc(g, prec, nmaps, (const float*)part, out, s);
  return adj_dispatch_ck(g, nmaps, (const float*)part, out, s);
}

}  // namespace cmbws
