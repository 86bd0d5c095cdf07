// Ring FFT stage of the SHT (Sec. 2.1) and the pixel-space multiplies of A
// (N^-1 = diag(tau), Eq. A) and of T^+ (alpha^2 W N W, Sec. 3.3).
//
// Synthesis of one ring with spectrum F_m = (Fc_m, Fs_m), m = 0..L:
//   f(phi_j) = Fc_0 + sqrt(2) sum_{m>=1} [Fc_m cos(m phi_j) + Fs_m sin(m phi_j)],
//   phi_j = phi0 + 2 pi j / n.
// Written as f_j = sum_k H_k exp(2 pi i k j / n) with the Hermitian spectrum
// H folded modulo n from frequencies -L..L (aliasing included), so f is the
// length-n inverse DFT of H.  The north and south rings of a pair share n
// and phi0 and are packed into one complex transform z = f_N + i f_S.  The
// adjoint (analysis, optionally quadrature-weighted) runs the forward DFT and
// unfolds Z back to m = 0..L with the exact transposes of these steps.
//
// One CTA per (ring pair, map); the DFT runs in shared memory: a power-of-two
// FFT for power-of-two n (equatorial HEALPix rings, polar rings 4i with i a power
// of two), Bluestein's chirp-z algorithm (a power-of-two convolution of size
// >= 2n - 1) for every other n (GL rings of 2L+1 pixels, most polar rings).  The
// power-of-two FFTs run radix-2 stages three at a time on 8-element register groups
// (decimation in time fed in bit-reversed order, decimation in frequency leaving its
// output bit-reversed), so no permutation pass is needed: the spectrum side of a
// power-of-two ring lives in bit-reversed order, its pixels in natural order.
// The fused mode goes synthesis -> pixel multiply -> analysis without the
// pixel map leaving shared memory.
//
// Arithmetic: FP32, FP64, or double-float (df, CMBWS_FP32X2: FP64-accurate on the
// FP32 pipe, whose rate is 61 times the FP64 one on GB300).  The double-float
// transform reads and writes double-float ring spectra (the layout of the
// double-float Legendre stage), so FP64 conversions happen only at the pixels.
#include <type_traits>

#include "common.h"
#include "dfloat.h"

namespace cmbws {

namespace {

template <typename T> struct V2;
template <> struct V2<double> { using t = double2; };
template <> struct V2<float> { using t = float2; };
template <> struct V2<df> { using t = df2; };
// storage type of pixel factors and ring weights
template <typename T> struct PixT { using t = T; };
template <> struct PixT<df> { using t = double; };

template <typename T2>
__device__ __forceinline__ T2 cmul(T2 a, T2 b) {
  T2 r;
  r.x = a.x * b.x - a.y * b.y;
  r.y = a.x * b.y + a.y * b.x;
  return r;
}
template <typename T2>
__device__ __forceinline__ T2 cconj(T2 a) {
  a.y = -a.y;
  return a;
}

template <typename T2>
__device__ __forceinline__ T2 cmul_conj_if(T2 a, T2 w, bool inv) {
  if (inv) w.y = -w.y;
  return cmul(a, w);
}

// The transform buffer in shared memory, addressed through a swizzle: element i lives at
// (i ^ ((i >> sh) & 15)) + i / 16.  The padding of one slot per 16 elements spreads the
// early butterfly passes (threads 8 or 64 elements apart) over distinct banks, and the XOR
// of the top four index bits (sh = log2(N) - 4) spreads the bit-reversed spectrum slots of
// consecutive frequencies; both are bijections, so any access pattern stays correct.
template <typename T2>
struct Sbuf {
  T2* p;
  int sh;
  __device__ __forceinline__ int idx(int i) const { return (i ^ ((i >> sh) & 15)) + (i >> 4); }
  __device__ __forceinline__ T2& operator[](int i) const { return p[idx(i)]; }
};

// Power-of-two FFTs of size N (2 <= N <= nmax) in shared memory, built from radix-2 stages
// that are grouped: a thread loads 2^S elements that stay closed under S consecutive stages,
// runs those S stages in registers and writes them back in place, so a transform of 2^n
// takes ceil(n / S) passes through shared memory (one barrier each).
// tw[k] = exp(-2 pi i k / nmax), k < nmax / 2; the inverse uses the conjugate twiddles
// (unnormalised).
//
// Decimation in time (fft_dit): input in bit-reversed order, output in natural order.  Stage
// s (1..n) joins j and j + 2^(s-1) inside blocks of 2^s with the twiddle
// exp(-2 pi i pos / 2^s), pos = j mod 2^(s-1), applied before the butterfly.
// Decimation in frequency (fft_dif): natural order in, bit-reversed order out; stages run
// from s = n down to 1 and the twiddle is applied after the butterfly, the exact transpose.
// Element hooks of a transform: the first pass can read its inputs through `ld(i)` (e.g.
// from the pixel maps, with a chirp applied) and the last pass can hand its outputs to
// `st(i, v)` (e.g. a filter multiply, or a write to the pixel maps), so that these
// element-wise steps cost no pass of their own through shared memory.
template <typename T2>
struct BufLoad {
  Sbuf<T2> b;
  __device__ __forceinline__ T2 operator()(int i) const { return b[i]; }
};
template <typename T2>
struct BufStore {
  Sbuf<T2> b;
  __device__ __forceinline__ void operator()(int i, const T2& v) const { b[i] = v; }
};

// exp(-2 pi i c / 2^e) for e <= 3 (a root of unity of order 2, 4 or 8) in the element type
template <typename T2>
__device__ __forceinline__ T2 unit_root(int c, int e) {
  constexpr double h = 0.70710678118654752440;  // sqrt(2) / 2
  const int q = (c << (3 - e)) & 7;              // angle in units of -2 pi / 8
  const double re[8] = {1.0, h, 0.0, -h, -1.0, -h, 0.0, h};
  const double im[8] = {0.0, -h, -1.0, -h, 0.0, h, 1.0, h};
  T2 r;
  r.x = decltype(r.x)(re[q]);
  r.y = decltype(r.y)(im[q]);
  return r;
}

// Twiddles of a group: at one stage they are w0 exp(-2 pi i c / 2^(t+1)), c < 2^t, with w0 the
// twiddle of the group's first butterfly.  In FP32 one table read per stage then serves the
// group (the other factors are compile-time roots of unity, one complex multiply each); FP64
// multiplies run at a 64th of that rate and a double-float complex multiply costs ~50 FP32
// operations, so those read every twiddle from the table.
template <typename T2>
__device__ __forceinline__ T2 group_twiddle(const T2* __restrict__ tw, int pos0, int step, int stride,
                                            const T2& w0, int c, int e) {
  if constexpr (std::is_same<T2, float2>::value) {
    return c == 0 ? w0 : cmul(w0, unit_root<T2>(c, e));
  } else {
    return tw[(pos0 + c * step) * stride];
  }
}
template <typename T2, int S, typename LD, typename ST>
__device__ __forceinline__ void dit_group(Sbuf<T2> buf, int g, int s0, const T2* __restrict__ tw,
                                          int nmax, bool inv, bool first, bool last, const LD& ld,
                                          const ST& st) {
  constexpr int E = 1 << S;
  const int half0 = 1 << (s0 - 1);
  const int pos0 = g & (half0 - 1);
  const int base = ((g >> (s0 - 1)) << (s0 - 1 + S)) + pos0;
  T2 x[E];
#pragma unroll
  for (int k = 0; k < E; ++k) x[k] = first ? ld(base + k * half0) : buf[base + k * half0];
#pragma unroll
  for (int t = 0; t < S; ++t) {
    const int stride = nmax >> (s0 + t);
    const T2 w0 = tw[pos0 * stride];
#pragma unroll
    for (int c = 0; c < (1 << t); ++c) {
      const T2 w = group_twiddle(tw, pos0, half0, stride, w0, c, t + 1);
#pragma unroll
      for (int k0 = 0; k0 < E; k0 += 2 << t) {
        const int k = k0 + c;
        const T2 v = cmul_conj_if(x[k + (1 << t)], w, inv);
        x[k + (1 << t)].x = x[k].x - v.x;
        x[k + (1 << t)].y = x[k].y - v.y;
        x[k].x = x[k].x + v.x;
        x[k].y = x[k].y + v.y;
      }
    }
  }
#pragma unroll
  for (int k = 0; k < E; ++k) {
    if (last) st(base + k * half0, x[k]);
    else buf[base + k * half0] = x[k];
  }
}

template <typename T2, int S, typename LD, typename ST>
__device__ __forceinline__ void dif_group(Sbuf<T2> buf, int g, int s1, const T2* __restrict__ tw,
                                          int nmax, bool inv, bool first, bool last, const LD& ld,
                                          const ST& st) {
  constexpr int E = 1 << S;
  const int h = 1 << (s1 - S);  // smallest half of the group's stages (stage s1 - S + 1)
  const int pos0 = g & (h - 1);
  const int base = ((g >> (s1 - S)) << s1) + pos0;
  T2 x[E];
#pragma unroll
  for (int k = 0; k < E; ++k) x[k] = first ? ld(base + k * h) : buf[base + k * h];
#pragma unroll
  for (int t = 0; t < S; ++t) {
    const int sh = S - 1 - t;  // partner distance 2^sh in the group at stage s1 - t
    const int stride = nmax >> (s1 - t);
    const T2 w0 = tw[pos0 * stride];
#pragma unroll
    for (int c = 0; c < (1 << sh); ++c) {
      const T2 w = group_twiddle(tw, pos0, h, stride, w0, c, sh + 1);
#pragma unroll
      for (int k0 = 0; k0 < E; k0 += 2 << sh) {
        const int k = k0 + c;
        const T2 a = x[k], bb = x[k + (1 << sh)];
        T2 d;
        d.x = a.x - bb.x;
        d.y = a.y - bb.y;
        x[k].x = a.x + bb.x;
        x[k].y = a.y + bb.y;
        x[k + (1 << sh)] = cmul_conj_if(d, w, inv);
      }
    }
  }
#pragma unroll
  for (int k = 0; k < E; ++k) {
    if (last) st(base + k * h, x[k]);
    else buf[base + k * h] = x[k];
  }
}

// Register groups of 8 elements (3 stages per pass) in every arithmetic (16-element FP32
// groups spilled under the register cap that keeps three CTAs resident per SM).  Transforms
// too small to give every thread a group of 8 use groups of 4 or 2, more passes over more
// threads: small rings are latency-bound (the two-component L = 63 solve: 6.1 -> 5.4 ms).
__device__ __forceinline__ int group_stages(int N) {
  const int nt = (int)blockDim.x;
  return (N >> 3) >= nt ? 3 : (N >> 2) >= nt ? 2 : 1;
}

// Decimation-in-time transform of size N (bit-reversed in, natural out); the first pass loads
// through ld, the last stores through st; ends with a barrier.
template <typename T2, typename LD, typename ST>
__device__ void fft_dit(Sbuf<T2> buf, int N, const T2* __restrict__ tw, int nmax, bool inv,
                        const LD& ld, const ST& st) {
  const int S = group_stages(N);
  const int n = 31 - __clz(N);
  if (n == 0) {
    if (threadIdx.x == 0) st(0, ld(0));
    __syncthreads();
    return;
  }
  const int r = n % S, np = n / S + (r ? 1 : 0);
  int s0 = 1;
  for (int pass = 0; pass < np; ++pass) {
    const bool first = pass == 0, last = pass == np - 1;
    const int st_ = (pass < n / S) ? S : r;
    if (st_ == 3) {
      for (int g = threadIdx.x; g < (N >> 3); g += blockDim.x)
        dit_group<T2, 3>(buf, g, s0, tw, nmax, inv, first, last, ld, st);
    } else if (st_ == 2) {
      for (int g = threadIdx.x; g < (N >> 2); g += blockDim.x)
        dit_group<T2, 2>(buf, g, s0, tw, nmax, inv, first, last, ld, st);
    } else {
      for (int g = threadIdx.x; g < (N >> 1); g += blockDim.x)
        dit_group<T2, 1>(buf, g, s0, tw, nmax, inv, first, last, ld, st);
    }
    s0 += st_;
    __syncthreads();
  }
}

// Decimation-in-frequency transform of size N (natural in, bit-reversed out); hooks as above.
template <typename T2, typename LD, typename ST>
__device__ void fft_dif(Sbuf<T2> buf, int N, const T2* __restrict__ tw, int nmax, bool inv,
                        const LD& ld, const ST& st) {
  const int S = group_stages(N);
  const int n = 31 - __clz(N);
  if (n == 0) {
    if (threadIdx.x == 0) st(0, ld(0));
    __syncthreads();
    return;
  }
  const int r = n % S, np = n / S + (r ? 1 : 0);
  int s1 = n;
  for (int pass = 0; pass < np; ++pass) {
    const bool first = pass == 0, last = pass == np - 1;
    const int st_ = (pass < n / S) ? S : r;
    if (st_ == 3) {
      for (int g = threadIdx.x; g < (N >> 3); g += blockDim.x)
        dif_group<T2, 3>(buf, g, s1, tw, nmax, inv, first, last, ld, st);
    } else if (st_ == 2) {
      for (int g = threadIdx.x; g < (N >> 2); g += blockDim.x)
        dif_group<T2, 2>(buf, g, s1, tw, nmax, inv, first, last, ld, st);
    } else {
      for (int g = threadIdx.x; g < (N >> 1); g += blockDim.x)
        dif_group<T2, 1>(buf, g, s1, tw, nmax, inv, first, last, ld, st);
    }
    s1 -= st_;
    __syncthreads();
  }
}

__device__ __forceinline__ int bitrev(int k, int logn) {
  return logn == 0 ? 0 : (int)(__brev((unsigned)k) >> (32 - logn));
}

enum { MODE_SYNTH = 0, MODE_ANALYSIS = 1, MODE_FUSED = 2 };
constexpr int kMaxPix = 8;

template <typename T>
struct PixPtrs {
  const T* p[kMaxPix];
};

// NT threads per CTA; the register cap keeps three CTAs of 256 threads (six of 128) resident
// per SM in FP32 and double-float, which is what the transform buffer of the largest rings
// allows (double-float and FP64 grids with 8192-entry buffers: one CTA of 512).
//
// Each ring pair's DFTs, in terms of the plan (n pixels; Bluestein plans convolve over n2):
// * power of two: the inverse DFT is a DIT transform whose input (the folded spectrum) is
//   written in bit-reversed order and whose last pass yields pixels in natural order; the
//   forward DFT is a DIF transform, natural in, spectrum left bit-reversed for the unfold;
// * Bluestein (chirp b_t = exp(i pi t^2 / n)): the forward DFT X = conj(b) (conv(z conj(b),
//   b)) runs as a DIF transform whose first pass applies the chirp and whose last pass
//   multiplies by the (bit-reversed) filter spectrum, then a DIT transform whose last pass
//   applies the final chirp; the inverse DFT is conj(forward(conj(Z))), with the conjugations
//   folded into the fold and into that last pass.
// In the fused mode the pixel multiply and the chirp of the next transform happen in the last
// pass of the inverse; in the synthesis mode that pass writes the pixel maps, and in the
// analysis mode the first pass of the forward DFT reads them.
// FP64 gets twice the register budget (two CTAs of 256 threads): under the FP32 cap its
// transform spilled.
template <typename T>
constexpr int fft_min_blocks(int nt) { return (std::is_same<T, double>::value ? 512 : 768) / nt; }

template <typename T, int MODE, int NT>
__global__ void __launch_bounds__(NT, fft_min_blocks<T>(NT))
k_ringfft(typename V2<T>::t* __restrict__ F, int64_t F_stride, double* __restrict__ map_out,
          const double* __restrict__ map_in, int64_t npix,
          const typename PixT<T>::t* __restrict__ ring_w, PixPtrs<typename PixT<T>::t> pix,
          const FftPlan* __restrict__ plans, const int* __restrict__ pair_plan,
          const int2* __restrict__ pring, const int* __restrict__ pphase,
          const int64_t* __restrict__ roff, const typename V2<T>::t* __restrict__ tab,
          int64_t tw_off, int nmax, int L, T* __restrict__ eo, int eo_nm, int k0, int nmaps,
          int npair) {
  using T2 = typename V2<T>::t;
  using TP = typename PixT<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];

  // maps vary fastest across the grid, so the CTAs that fill the adjoint input of one ring
  // pair (interleaved per m) run together
  const int k = blockIdx.x;
  const int p = blockIdx.y;
  const FftPlan P = plans[pair_plan[p]];
  const int lg = 31 - __clz(P.n2);
  const Sbuf<T2> buf{reinterpret_cast<T2*>(smem_raw), lg >= 8 ? lg - 4 : 31};
  const int n = P.n, n2 = P.n2;
  const bool blu = P.bluestein != 0;
  const int logn = 31 - __clz(n);
  const int2 rr = pring[p];
  const bool has_s = rr.y >= 0;
  const int ph = pphase[p];
  T2* FN = F + k * F_stride + (int64_t)rr.x * (L + 1);
  T2* FS = has_s ? F + k * F_stride + (int64_t)rr.y * (L + 1) : nullptr;
  const int64_t offN = roff[rr.x];
  const int64_t offS = has_s ? roff[rr.y] : 0;
  const T rs2 = T(0.70710678118654752440);  // 1/sqrt(2)
  const T sq2 = T(1.41421356237309504880);
  // Shifted rings (phi0 = pi / n): exp(i m phi0) = (-1)^(m div n) exp(i pi (m mod n) / n),
  // so the plan's table of n phases exp(i pi k / n) serves every alias of every frequency.
  const T2* __restrict__ ptab = tab + P.phase;
  const T2* __restrict__ tw = tab + tw_off;
  const T2* __restrict__ chirp = tab + P.chirp;
  const T2* __restrict__ filt = tab + P.filt;
  const BufLoad<T2> bload{buf};
  const BufStore<T2> bstore{buf};
  // filter multiply in the last pass of a Bluestein plan's DIF transform
  auto filt_store = [&](int q, const T2& v) { buf[q] = cmul(v, filt[q]); };

  if (MODE == MODE_SYNTH || MODE == MODE_FUSED) {
    // fold the two-sided spectrum modulo n:
    //   H_k = [k = 0] Fc_0 + P_k / sqrt(2) (sum_{m = k + jn} s_j (Fc - i Fs)_m
    //                                      + sum_{m = jn - k} s_j (Fc + i Fs)_m),
    // P_k = exp(i pi k / n), s_j = (-1)^j on shifted rings (P_k = s_j = 1 otherwise).
    // Power-of-two plans store H_k at bit-reversed k; Bluestein plans store the first input
    // of the chirp-z transform of conj(H), conj(H_k) conj(b_k), zero-padded to n2.
    // Alias sums of one frequency: +m frequencies m = kk + j n (j >= 1 at kk = 0), sum of
    // s_j (Fc, -Fs); -m frequencies m = j n - kk (j >= 1), sum of s_j (Fc, +Fs); the terms
    // j = j0 + part, j0 + part + tpk, ... of each series (all of them for tpk = 1).
    auto alias_sums = [&](int kk, int part, int tpk, T& anx, T& any, T& asx, T& asy) {
      anx = any = asx = asy = T(0);
      {
        int j = (kk == 0 ? 1 : 0) + part;
        for (int m = kk + j * n; m <= L; m += tpk * n, j += tpk) {
          const bool neg = ph && (j & 1);
          const T2 a = FN[m];
          anx += neg ? -a.x : a.x;
          any -= neg ? -a.y : a.y;
          if (has_s) {
            const T2 b = FS[m];
            asx += neg ? -b.x : b.x;
            asy -= neg ? -b.y : b.y;
          }
        }
      }
      {
        int j = 1 + part;
        for (int m = j * n - kk; m <= L; m += tpk * n, j += tpk) {
          const bool neg = ph && (j & 1);
          const T2 a = FN[m];
          anx += neg ? -a.x : a.x;
          any += neg ? -a.y : a.y;
          if (has_s) {
            const T2 b = FS[m];
            asx += neg ? -b.x : b.x;
            asy += neg ? -b.y : b.y;
          }
        }
      }
    };
    // H_k from the alias sums, stored where the inverse DFT reads it
    auto fold_store = [&](int kk, T anx, T any, T asx, T asy) {
      T cp = T(1), sp = T(0);
      if (ph) {
        const T2 e = ptab[kk];
        cp = e.x;
        sp = e.y;
      }
      // H = P (a) / sqrt(2) (+ Fc_0 at k = 0)
      T hnx = rs2 * (cp * anx - sp * any), hny = rs2 * (cp * any + sp * anx);
      T hsx = rs2 * (cp * asx - sp * asy), hsy = rs2 * (cp * asy + sp * asx);
      if (kk == 0) {
        hnx += FN[0].x;
        if (has_s) hsx += FS[0].x;
      }
      T2 z;
      z.x = hnx - hsy;
      z.y = hny + hsx;
      if (blu) buf[kk] = cmul(cconj(z), cconj(chirp[kk]));
      else buf[bitrev(kk, logn)] = z;
    };
    // Rings with fewer pixels than threads fold many aliases into each frequency: tpk threads
    // share a frequency, each summing every tpk-th alias, and the partial sums are added in a
    // fixed order (scratch: raw shared memory past this ring's buffer).
    const int scratch = n2 + n2 / 16 + 16;
    int tpk = n < NT / 2 ? NT / n : 1;
    if (scratch + 2 * NT > nmax + nmax / 16 + 16) tpk = 1;
    for (int kk = n + threadIdx.x; kk < n2; kk += blockDim.x) {
      T2 z;
      z.x = z.y = T(0);
      buf[kk] = z;
    }
    if (tpk == 1) {
      for (int kk = threadIdx.x; kk < n; kk += blockDim.x) {
        T anx, any, asx, asy;
        alias_sums(kk, 0, 1, anx, any, asx, asy);
        fold_store(kk, anx, any, asx, asy);
      }
    } else {
      T2* part = buf.p + scratch;
      const int t = threadIdx.x;
      if (t < n * tpk) {
        T anx, any, asx, asy;
        alias_sums(t % n, t / n, tpk, anx, any, asx, asy);
        part[2 * t].x = anx;
        part[2 * t].y = any;
        part[2 * t + 1].x = asx;
        part[2 * t + 1].y = asy;
      }
      __syncthreads();
      if (t < n) {
        T anx = T(0), any = T(0), asx = T(0), asy = T(0);
        for (int q = 0; q < tpk; ++q) {
          const T2 u = part[2 * (t + q * n)], v = part[2 * (t + q * n) + 1];
          anx += u.x;
          any += u.y;
          asx += v.x;
          asy += v.y;
        }
        fold_store(t, anx, any, asx, asy);
      }
    }
    __syncthreads();
    // the last pass of the inverse DFT: pixel values z_t (natural order) -> map or the
    // pixel multiply (and, for Bluestein plans, the first chirp of the forward DFT)
    const TP* pk = MODE == MODE_FUSED ? pix.p[k] : nullptr;
    double* mo = MODE == MODE_SYNTH ? map_out + k * npix : nullptr;
    auto pixel_store = [&](int t, T2 z) {
      if (blu) {
        if (t >= n) {
          if (MODE == MODE_FUSED) {
            T2 zz;
            zz.x = zz.y = T(0);
            buf[t] = zz;
          }
          return;
        }
        z = cconj(cmul(z, cconj(chirp[t])));
      }
      if (MODE == MODE_SYNTH) {
        mo[offN + t] = (double)z.x;
        if (has_s) mo[offS + t] = (double)z.y;
        return;
      }
      z.x = z.x * T(pk[offN + t]);
      z.y = has_s ? z.y * T(pk[offS + t]) : T(0);
      buf[t] = blu ? cmul(z, cconj(chirp[t])) : z;
    };
    if (!blu) {
      fft_dit(buf, n, tw, nmax, true, bload, pixel_store);
    } else {
      fft_dif(buf, n2, tw, nmax, false, bload, filt_store);
      fft_dit(buf, n2, tw, nmax, true, bload, pixel_store);
    }
    if (MODE == MODE_SYNTH) return;
    // forward DFT of the multiplied pixels (already chirped and padded for Bluestein plans)
    if (!blu) {
      fft_dif(buf, n, tw, nmax, false, bload, bstore);
    } else {
      fft_dif(buf, n2, tw, nmax, false, bload, filt_store);
      auto chirp_store = [&](int t, const T2& c) {
        if (t < n) buf[t] = cmul(c, cconj(chirp[t]));
      };
      fft_dit(buf, n2, tw, nmax, true, bload, chirp_store);
    }
  } else {
    // analysis: the first pass of the forward DFT reads the (optionally weighted) pixels
    const double* mi = map_in + k * npix;
    const T wN = ring_w ? T(ring_w[rr.x]) : T(1);
    const T wS = (ring_w && has_s) ? T(ring_w[rr.y]) : T(1);
    auto pixel_load = [&](int t) {
      T2 z;
      if (t >= n) {
        z.x = z.y = T(0);
        return z;
      }
      z.x = T(mi[offN + t]) * wN;
      z.y = has_s ? T(mi[offS + t]) * wS : T(0);
      return blu ? cmul(z, cconj(chirp[t])) : z;
    };
    if (!blu) {
      fft_dif(buf, n, tw, nmax, false, pixel_load, bstore);
    } else {
      fft_dif(buf, n2, tw, nmax, false, pixel_load, filt_store);
      auto chirp_store = [&](int t, const T2& c) {
        if (t < n) buf[t] = cmul(c, cconj(chirp[t]));
      };
      fft_dit(buf, n2, tw, nmax, true, bload, chirp_store);
    }
  }

  // unfold: G_m = exp(-i m phi0) X_{m mod n}; (Fc^T, Fs^T) = c_m (Re G, -Im G); the spectrum
  // X is bit-reversed for power-of-two plans, natural for Bluestein plans
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    const int kk = m % n;
    const int kc = (kk == 0) ? 0 : n - kk;
    const T2 zk = buf[blu ? kk : bitrev(kk, logn)];
    const T2 zc = cconj(buf[blu ? kc : bitrev(kc, logn)]);
    T xnx = T(0.5) * (zk.x + zc.x), xny = T(0.5) * (zk.y + zc.y);
    T xsx = T(0.5) * (zk.y - zc.y), xsy = T(-0.5) * (zk.x - zc.x);
    T c = T(1), s = T(0);
    if (ph) {
      const T2 e = ptab[kk];
      const bool neg = ((m / n) & 1) != 0;
      c = neg ? -e.x : e.x;
      s = neg ? -e.y : e.y;
    }
    const T cm = m == 0 ? T(1) : sq2;
    // G = (c - i s) X
    T gx = c * xnx + s * xny, gy = c * xny - s * xnx;
    T2 on, os;
    on.x = cm * gx;
    on.y = -cm * gy;
    if (m == 0) on.y = 0;
    if (has_s) {
      gx = c * xsx + s * xsy;
      gy = c * xsy - s * xsx;
      os.x = cm * gx;
      os.y = m == 0 ? T(0) : -cm * gy;
    }
    if (!eo) {
      FN[m] = on;
      if (has_s) FS[m] = os;
      continue;
    }
    // the adjoint input: even-l part north + south, odd-l part north - south (a ring pair
    // without a south ring counts its north ring in both)
    T2 ev = on, od = on;
    if (has_s) {
      ev.x = on.x + os.x;
      ev.y = on.y + os.y;
      od.x = on.x - os.x;
      od.y = on.y - os.y;
    }
    const int kg = k0 + k, ch = kg / eo_nm, j = kg - ch * eo_nm;
    const int nmc = min(eo_nm, nmaps - ch * eo_nm), P = 2 * nmc;
    T* e = eo + (int64_t)ch * eo_nm * (L + 1) * npair * 4 + ((int64_t)m * npair + p) * 2 * P;
    *reinterpret_cast<T2*>(e + 2 * j) = ev;
    *reinterpret_cast<T2*>(e + P + 2 * j) = od;
  }
}

template <typename T>
size_t smem_bytes(const Grid& g) {
  // the transform buffer with its swizzle padding (one slot per 16 elements)
  return (size_t)(g.nmax2 + g.nmax2 / 16 + 16) * sizeof(typename V2<T>::t);
}

// Threads per CTA: a grid with large transforms (>= 4096 entries, e.g. the Bluestein buffers
// of the polar rings from Nside 512 up) gets 256 threads, so that the butterfly passes of one
// ring have twice the warps to hide shared-memory latency with the same buffer per CTA; the
// others 128; 16-byte values with 8192-entry buffers (one CTA per SM) 512.
template <typename T, int MODE>
int launch(const Grid& g, int nmaps, void* F, double* map_out, const double* map_in, int weighted,
           const void* const* pix, void* eo, int eo_nm, cudaStream_t s);

template <typename T, int MODE, int NT>
int launch_nt(const Grid& g, int nmaps, void* F, double* map_out, const double* map_in,
              int weighted, const void* const* pix, void* eo, int eo_nm, cudaStream_t s) {
  using T2 = typename V2<T>::t;
  const size_t sm = smem_bytes<T>(g);
  if (sm > 227 * 1024) {
    set_error("ring FFT needs %zu bytes of shared memory (ring length %d) at this precision",
              sm, g.max_n);
    return CMBWS_ERR_ARG;
  }
  auto kern = k_ringfft<T, MODE, NT>;
  CMBWS_TRY(ensure_dyn_smem((const void*)kern, sm));
  using TP = typename PixT<T>::t;
  const int64_t fs = (int64_t)g.nring * (g.lmax + 1);
  constexpr bool f32 = std::is_same<T, float>::value, f64 = std::is_same<T, double>::value;
  const TP* rw = nullptr;
  if (MODE == MODE_ANALYSIS && weighted) rw = f32 ? (const TP*)g.ring_w32.p : (const TP*)g.ring_w64.p;
  const T2* tab = f32 ? (const T2*)g.fft32.p : f64 ? (const T2*)g.fft64.p : (const T2*)g.fftdf.p;
  for (int k0 = 0; k0 < nmaps; k0 += kMaxPix) {
    const int nm = nmaps - k0 < kMaxPix ? nmaps - k0 : kMaxPix;
    PixPtrs<TP> pp{};
    if (MODE == MODE_FUSED)
      for (int i = 0; i < nm; ++i) pp.p[i] = (const TP*)pix[k0 + i];
    dim3 grd(nm, g.npair);
    // algorithmic bytes: ring spectra read and/or written once, pixel factors (fused) or the
    // FP64 maps (synthesis output, analysis input) once
    const double fb = (double)g.nring * (g.lmax + 1) * sizeof(T2);
    const double pb = (double)g.npix * (MODE == MODE_FUSED ? sizeof(TP) : sizeof(double));
    ProfScope ps(PROF_FFT, s, f32 ? 0 : f64 ? 1 : 2,
                 byte_work(nm * ((MODE == MODE_FUSED ? 2.0 : 1.0) * fb + pb)));
    kern<<<grd, NT, sm, s>>>((T2*)F + k0 * fs, fs, map_out ? map_out + k0 * g.npix : nullptr,
                              map_in ? map_in + k0 * g.npix : nullptr, g.npix, rw, pp,
                              g.plans_d.as<FftPlan>(), g.pair_plan.as<int>(),
                              g.pair_ring.as<int2>(), g.pair_phase.as<int>(), g.ring_off.as<int64_t>(),
                              tab, g.tw_off, g.nmax2, g.lmax, (T*)eo, eo_nm, k0, nmaps, g.npair);
    CMBWS_LAUNCH_CHECK();
  }
  return CMBWS_OK;
}

template <typename T, int MODE>
int launch(const Grid& g, int nmaps, void* F, double* map_out, const double* map_in, int weighted,
           const void* const* pix, void* eo, int eo_nm, cudaStream_t s) {
  // 16-byte values (double-float, FP64) with 8192-entry buffers: about 140 KB per CTA, one CTA
  // per SM, so that CTA gets 512 threads (16 warps instead of 8)
  if constexpr (!std::is_same<T, float>::value)
    if (g.nmax2 >= 8192)
      return launch_nt<T, MODE, 512>(g, nmaps, F, map_out, map_in, weighted, pix, eo, eo_nm, s);
  if (g.nmax2 >= 4096)
    return launch_nt<T, MODE, 256>(g, nmaps, F, map_out, map_in, weighted, pix, eo, eo_nm, s);
  return launch_nt<T, MODE, 128>(g, nmaps, F, map_out, map_in, weighted, pix, eo, eo_nm, s);
}

}  // namespace

int ringfft_smem_ok(const Grid& g, int prec) {
  const size_t sm = !is_f32(prec) ? smem_bytes<double>(g) : smem_bytes<float>(g);
  return sm <= 227 * 1024;
}

// Spectra F: float2 (FP32 modes), double2 (FP64) or double-float pairs (FP32X2).
// Pixel factors: float (FP32 modes) or double.
int ringfft_synth(const Grid& g, int prec, int nmaps, const void* F, double* map, cudaStream_t s) {
  void* f = const_cast<void*>(F);
  if (prec == CMBWS_FP32X2)
    return launch<df, MODE_SYNTH>(g, nmaps, f, map, nullptr, 0, nullptr, nullptr, 0, s);
  if (!is_f32(prec))
    return launch<double, MODE_SYNTH>(g, nmaps, f, map, nullptr, 0, nullptr, nullptr, 0, s);
  return launch<float, MODE_SYNTH>(g, nmaps, f, map, nullptr, 0, nullptr, nullptr, 0, s);
}

int ringfft_analysis(const Grid& g, int prec, int nmaps, const double* map, int weighted, void* F,
                     void* eo, cudaStream_t s) {
  if (prec == CMBWS_FP32X2)
    return launch<df, MODE_ANALYSIS>(g, nmaps, F, nullptr, map, weighted, nullptr, eo,
                                     eo_maps(prec), s);
  if (!is_f32(prec))
    return launch<double, MODE_ANALYSIS>(g, nmaps, F, nullptr, map, weighted, nullptr, nullptr, 0, s);
  return launch<float, MODE_ANALYSIS>(g, nmaps, F, nullptr, map, weighted, nullptr, eo,
                                      eo_maps(prec), s);
}

int ringfft_fused(const Grid& g, int prec, int nmaps, void* F, const void* const* pix, void* eo,
                  cudaStream_t s) {
  if (prec == CMBWS_FP32X2)
    return launch<df, MODE_FUSED>(g, nmaps, F, nullptr, nullptr, 0, pix, eo, eo_maps(prec), s);
  if (!is_f32(prec))
    return launch<double, MODE_FUSED>(g, nmaps, F, nullptr, nullptr, 0, pix, nullptr, 0, s);
  return launch<float, MODE_FUSED>(g, nmaps, F, nullptr, nullptr, 0, pix, eo, eo_maps(prec), s);
}

}  // namespace cmbws
