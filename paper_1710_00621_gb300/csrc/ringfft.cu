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
// One CTA per (ring pair, map); the DFT runs in shared memory: radix-2 for
// power-of-two n (equatorial HEALPix rings, polar rings 4i with i a power of
// two), Bluestein's chirp-z algorithm (a power-of-two convolution of size
// >= 2n - 1) for every other n (GL rings of 2L+1 pixels, most polar rings).
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

// In-place power-of-two transform of size N (>= 1) in shared memory, decimation in
// time after a bit-reversal permutation; two radix-2 stages per pass (each thread owns
// a closed group of 4 elements i, i+h, i+2h, i+3h), so one barrier per two stages.
// tw[k] = exp(-2 pi i k / NMAX), k < NMAX/2.  inverse: exp(+2 pi i ...), unnormalised.
template <typename T2>
__device__ __forceinline__ void bfly(T2& a, T2& b, T2 w) {
  const T2 v = cmul(b, w);
  b.x = a.x - v.x;
  b.y = a.y - v.y;
  a.x += v.x;
  a.y += v.y;
}

template <typename T2>
__device__ void smem_fft(T2* buf, int N, const T2* __restrict__ tw, int nmax, bool inverse) {
  if (N < 2) return;
  const int logN = 31 - __clz(N);
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    const int j = (int)(__brev((unsigned)i) >> (32 - logN));
    if (i < j) {
      T2 t = buf[i];
      buf[i] = buf[j];
      buf[j] = t;
    }
  }
  __syncthreads();
  int lg = 1;
  for (; lg + 1 <= logN; lg += 2) {
    const int h = 1 << (lg - 1);  // stage lg pairs (i, i+h); stage lg+1 pairs (i, i+2h)
    const int s1 = nmax >> lg, s2 = nmax >> (lg + 1);
    for (int b = threadIdx.x; b < N / 4; b += blockDim.x) {
      const int pos = b & (h - 1);
      const int i = ((b >> (lg - 1)) << (lg + 1)) + pos;
      T2 w1 = tw[pos * s1], w2a = tw[pos * s2], w2b = tw[(pos + h) * s2];
      if (inverse) {
        w1.y = -w1.y;
        w2a.y = -w2a.y;
        w2b.y = -w2b.y;
      }
      T2 x0 = buf[i], x1 = buf[i + h], x2 = buf[i + 2 * h], x3 = buf[i + 3 * h];
      bfly(x0, x1, w1);
      bfly(x2, x3, w1);
      bfly(x0, x2, w2a);
      bfly(x1, x3, w2b);
      buf[i] = x0;
      buf[i + h] = x1;
      buf[i + 2 * h] = x2;
      buf[i + 3 * h] = x3;
    }
    __syncthreads();
  }
  if (lg == logN) {  // odd number of stages: one radix-2 stage left
    const int half = 1 << (lg - 1);
    const int tstride = nmax >> lg;
    for (int b = threadIdx.x; b < N / 2; b += blockDim.x) {
      const int pos = b & (half - 1);
      const int i = ((b >> (lg - 1)) << lg) + pos;
      T2 w = tw[pos * tstride];
      if (inverse) w.y = -w.y;
      T2 x0 = buf[i], x1 = buf[i + half];
      bfly(x0, x1, w);
      buf[i] = x0;
      buf[i + half] = x1;
    }
    __syncthreads();
  }
}

enum { MODE_SYNTH = 0, MODE_ANALYSIS = 1, MODE_FUSED = 2 };
constexpr int kMaxPix = 8;

template <typename T>
struct PixPtrs {
  const T* p[kMaxPix];
};

// Forward DFT of z[0..n) held in buf (Bluestein needs buf of n2); result Z[0..n) in buf.
template <typename T2>
__device__ void dft_forward(T2* buf, const FftPlan& P, const T2* __restrict__ tab, int64_t tw_off,
                            int nmax) {
  if (!P.bluestein) {
    smem_fft(buf, P.n, tab + tw_off, nmax, false);
    return;
  }
  const T2* b = tab + P.chirp;
  const T2* V = tab + P.filt;
  for (int t = threadIdx.x; t < P.n2; t += blockDim.x) {
    if (t < P.n) buf[t] = cmul(buf[t], cconj(b[t]));
    else buf[t].x = buf[t].y = 0;
  }
  __syncthreads();
  smem_fft(buf, P.n2, tab + tw_off, nmax, false);
  for (int t = threadIdx.x; t < P.n2; t += blockDim.x) buf[t] = cmul(buf[t], V[t]);
  __syncthreads();
  smem_fft(buf, P.n2, tab + tw_off, nmax, true);
  for (int t = threadIdx.x; t < P.n; t += blockDim.x) buf[t] = cmul(buf[t], cconj(b[t]));
  __syncthreads();
}

// Inverse (unnormalised) DFT of Z[0..n) in buf; result z[0..n) in buf.
template <typename T2>
__device__ void dft_inverse(T2* buf, const FftPlan& P, const T2* __restrict__ tab, int64_t tw_off,
                            int nmax) {
  if (!P.bluestein) {
    smem_fft(buf, P.n, tab + tw_off, nmax, true);
    return;
  }
  // z = conj(DFT(conj(Z)))
  for (int t = threadIdx.x; t < P.n; t += blockDim.x) buf[t] = cconj(buf[t]);
  __syncthreads();
  dft_forward(buf, P, tab, tw_off, nmax);
  for (int t = threadIdx.x; t < P.n; t += blockDim.x) buf[t] = cconj(buf[t]);
  __syncthreads();
}

template <typename T, int MODE, int NT>
__global__ void __launch_bounds__(NT)
k_ringfft(typename V2<T>::t* __restrict__ F, int64_t F_stride, double* __restrict__ map_out,
          const double* __restrict__ map_in, int64_t npix,
          const typename PixT<T>::t* __restrict__ ring_w, PixPtrs<typename PixT<T>::t> pix,
          const FftPlan* __restrict__ plans, const int* __restrict__ pair_plan,
          const int2* __restrict__ pring, const int* __restrict__ pphase,
          const int64_t* __restrict__ roff, const typename V2<T>::t* __restrict__ tab,
          int64_t tw_off, int nmax, int L) {
  using T2 = typename V2<T>::t;
  using TP = typename PixT<T>::t;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T2* buf = reinterpret_cast<T2*>(smem_raw);

  const int p = blockIdx.x;
  const int k = blockIdx.y;
  const FftPlan P = plans[pair_plan[p]];
  const int n = P.n;
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

  if (MODE == MODE_SYNTH || MODE == MODE_FUSED) {
    // fold the two-sided spectrum modulo n:
    //   H_k = [k = 0] Fc_0 + P_k / sqrt(2) (sum_{m = k + jn} s_j (Fc - i Fs)_m
    //                                      + sum_{m = jn - k} s_j (Fc + i Fs)_m),
    // P_k = exp(i pi k / n), s_j = (-1)^j on shifted rings (P_k = s_j = 1 otherwise)
    for (int kk = threadIdx.x; kk < n; kk += blockDim.x) {
      T anx = T(0), any = T(0), asx = T(0), asy = T(0);
      // +m frequencies, m = kk + j n >= 1: sum of s_j (Fc, -Fs)
      {
        int j = kk == 0 ? 1 : 0;
        for (int m = kk + j * n; m <= L; m += n, ++j) {
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
      // -m frequencies, m = j n - kk >= 1: sum of s_j (Fc, +Fs)
      {
        int j = 1;
        for (int m = n - kk; m <= L; m += n, ++j) {
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
      buf[kk] = z;
    }
    __syncthreads();
    dft_inverse(buf, P, tab, tw_off, nmax);
    if (MODE == MODE_SYNTH) {
      double* mo = map_out + k * npix;
      for (int j = threadIdx.x; j < n; j += blockDim.x) {
        const T2 z = buf[j];
        mo[offN + j] = (double)z.x;
        if (has_s) mo[offS + j] = (double)z.y;
      }
      return;
    }
    // pixel multiply in place
    const TP* pk = pix.p[k];
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      T2 z = buf[j];
      z.x *= T(pk[offN + j]);
      z.y = has_s ? z.y * T(pk[offS + j]) : T(0);
      buf[j] = z;
    }
    __syncthreads();
  } else {
    // analysis: load (optionally weighted) pixels
    const double* mi = map_in + k * npix;
    const T wN = ring_w ? T(ring_w[rr.x]) : T(1);
    const T wS = (ring_w && has_s) ? T(ring_w[rr.y]) : T(1);
    for (int j = threadIdx.x; j < n; j += blockDim.x) {
      T2 z;
      z.x = T(mi[offN + j]) * wN;
      z.y = has_s ? T(mi[offS + j]) * wS : T(0);
      buf[j] = z;
    }
    __syncthreads();
  }

  dft_forward(buf, P, tab, tw_off, nmax);

  // unfold: G_m = exp(-i m phi0) X_{m mod n}; (Fc^T, Fs^T) = c_m (Re G, -Im G)
  for (int m = threadIdx.x; m <= L; m += blockDim.x) {
    const int kk = m % n;
    const int kc = (kk == 0) ? 0 : n - kk;
    const T2 zk = buf[kk];
    const T2 zc = cconj(buf[kc]);
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
    T2 o;
    o.x = cm * gx;
    o.y = -cm * gy;
    if (m == 0) o.y = 0;
    FN[m] = o;
    if (has_s) {
      gx = c * xsx + s * xsy;
      gy = c * xsy - s * xsx;
      o.x = cm * gx;
      o.y = m == 0 ? T(0) : -cm * gy;
      FS[m] = o;
    }
  }
}

template <typename T>
size_t smem_bytes(const Grid& g) {
  return (size_t)g.nmax2 * sizeof(typename V2<T>::t);  // the transform buffer
}

// Threads per CTA: a grid with large transforms (>= 2048 entries, e.g. the 4 Nside-point
// equatorial rings from Nside 512 up) gets 512 threads, so that the butterfly passes of one
// ring have twice the warps to hide shared-memory latency with the same buffer per CTA.
template <typename T, int MODE>
int launch(const Grid& g, int nmaps, void* F, double* map_out, const double* map_in, int weighted,
           const void* const* pix, cudaStream_t s);

template <typename T, int MODE, int NT>
int launch_nt(const Grid& g, int nmaps, void* F, double* map_out, const double* map_in,
              int weighted, const void* const* pix, cudaStream_t s) {
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
    dim3 grd(g.npair, nm);
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
                              tab, g.tw_off, g.nmax2, g.lmax);
    CMBWS_LAUNCH_CHECK();
  }
  return CMBWS_OK;
}

template <typename T, int MODE>
int launch(const Grid& g, int nmaps, void* F, double* map_out, const double* map_in, int weighted,
           const void* const* pix, cudaStream_t s) {
  if (g.nmax2 >= 2048)
    return launch_nt<T, MODE, 512>(g, nmaps, F, map_out, map_in, weighted, pix, s);
  return launch_nt<T, MODE, 256>(g, nmaps, F, map_out, map_in, weighted, pix, s);
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
  if (prec == CMBWS_FP32X2) return launch<df, MODE_SYNTH>(g, nmaps, f, map, nullptr, 0, nullptr, s);
  if (!is_f32(prec)) return launch<double, MODE_SYNTH>(g, nmaps, f, map, nullptr, 0, nullptr, s);
  return launch<float, MODE_SYNTH>(g, nmaps, f, map, nullptr, 0, nullptr, s);
}

int ringfft_analysis(const Grid& g, int prec, int nmaps, const double* map, int weighted, void* F,
                     cudaStream_t s) {
  if (prec == CMBWS_FP32X2)
    return launch<df, MODE_ANALYSIS>(g, nmaps, F, nullptr, map, weighted, nullptr, s);
  if (!is_f32(prec))
    return launch<double, MODE_ANALYSIS>(g, nmaps, F, nullptr, map, weighted, nullptr, s);
  return launch<float, MODE_ANALYSIS>(g, nmaps, F, nullptr, map, weighted, nullptr, s);
}

int ringfft_fused(const Grid& g, int prec, int nmaps, void* F, const void* const* pix,
                  cudaStream_t s) {
  if (prec == CMBWS_FP32X2) return launch<df, MODE_FUSED>(g, nmaps, F, nullptr, nullptr, 0, pix, s);
  if (!is_f32(prec)) return launch<double, MODE_FUSED>(g, nmaps, F, nullptr, nullptr, 0, pix, s);
  return launch<float, MODE_FUSED>(g, nmaps, F, nullptr, nullptr, 0, pix, s);
}

}  // namespace cmbws
