// fft.cuh -- in-place mixed-radix FFT of one sequence held in shared memory.
//
// Stockham autosort: stage k with radix R and span Ns = R_0...R_{k-1} takes, for
// every butterfly j < n/R, the inputs x[j + r n/R] (r < R), multiplies input r
// by W_{Ns R}^{r (j mod Ns)} (W_q = e^{-2 pi i / q}), applies an R-point DFT and
// writes output k to position (j / Ns) Ns R + (j mod Ns) + k Ns; the result is in
// natural order after the last stage.
//
// Radices 2, 3, 4, 5, 7 and 8 (and 11, 13 in single precision) run as register butterflies: each thread loads
// the inputs of its butterflies, the block synchronises, and the outputs
// overwrite the inputs, so one shared buffer of n elements suffices.  Other odd
// primes (the 2L-1 lengths contain factors such as 13, 31, 73 or 127) use a
// dot-product stage in which each output is an R-term sum (compensated in
// FP32).  Where those sums would dominate (a prime 2L-1 such as 4093 makes the
// whole FFT one 4093-term stage), the plan runs the length 2L-1 by Bluestein's
// chirp-z convolution through a power-of-two length instead (fft_bluestein,
// at the end).  Twiddles come from one table of e^{-2 pi i k / n}, k < n.
#pragma once
#include <cuda_runtime.h>
#include "internal.h"

template <typename T> struct cplx;
template <> struct cplx<double> { typedef double2 t; };
template <> struct cplx<float> { typedef float2 t; };

template <typename T>
__device__ __forceinline__ typename cplx<T>::t mkc(T a, T b) {
  typename cplx<T>::t r; r.x = a; r.y = b; return r;
}

namespace fftk {

template <typename T> using C = typename cplx<T>::t;

template <typename T> __device__ __forceinline__ C<T> add(C<T> a, C<T> b) { return mkc<T>(a.x + b.x, a.y + b.y); }
template <typename T> __device__ __forceinline__ C<T> sub(C<T> a, C<T> b) { return mkc<T>(a.x - b.x, a.y - b.y); }
template <typename T> __device__ __forceinline__ C<T> mul(C<T> a, C<T> b) {
  return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T> __device__ __forceinline__ C<T> mulc(C<T> a, C<T> b) {  // a * conj(b)
  return mkc<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
// times -i (forward) or +i (inverse)
template <typename T> __device__ __forceinline__ C<T> rot(C<T> a, bool inv) {
  return inv ? mkc<T>(-a.y, a.x) : mkc<T>(a.y, -a.x);
}

// cos and sin of 2 pi k / R for the odd radices (k = 1 .. (R-1)/2)
__device__ __forceinline__ double cs3(int) { return -0.5; }
__device__ __forceinline__ double sn3(int) { return 0.86602540378443864676; }
__device__ __forceinline__ double cs5(int k) { return k == 1 ? 0.3090169943749474241 : -0.8090169943749474241; }
__device__ __forceinline__ double sn5(int k) { return k == 1 ? 0.95105651629515357212 : 0.58778525229247312917; }
__device__ __forceinline__ double cs7(int k) {
  return k == 1 ? 0.62348980185873353053 : (k == 2 ? -0.22252093395631440429 : -0.90096886790241912624);
}
__device__ __forceinline__ double sn7(int k) {
  return k == 1 ? 0.78183148246802980871 : (k == 2 ? 0.97492791218182360702 : 0.43388373911755812048);
}
__device__ __forceinline__ double cs11(int k) {
  constexpr double c[5] = {0.841253532831181168862, 0.415415013001886425529, -0.142314838273285140444,
                           -0.654860733945285064057, -0.95949297361449738989};
  return c[k - 1];
}
__device__ __forceinline__ double sn11(int k) {
  constexpr double c[5] = {0.540640817455597582108, 0.909631995354518371412, 0.989821441880932732376,
                           0.755749574354258283774, 0.281732556841429697711};
  return c[k - 1];
}
__device__ __forceinline__ double cs13(int k) {
  constexpr double c[6] = {0.8854560256532098959, 0.568064746731155802512, 0.120536680255323053349,
                           -0.35460488704253562597, -0.748510748171101098635, -0.970941817426052027157};
  return c[k - 1];
}
__device__ __forceinline__ double sn13(int k) {
  constexpr double c[6] = {0.464723172043768545656, 0.82298386589365639458, 0.992708874098053992801,
                           0.93501624268541482344, 0.663122658240795202377, 0.239315664287557767149};
  return c[k - 1];
}

// Odd R-point DFT by the symmetric pairing y_k = a_k +- i b_k with
// a_k = v_0 + sum_r (v_r + v_{R-r}) cos(2 pi r k/R), b_k = sum_r (v_r - v_{R-r}) sin(2 pi r k/R).
template <typename T, int R>
__device__ __forceinline__ void dft_odd(C<T>* v, bool inv) {
  constexpr int H = (R - 1) / 2;
  C<T> s[H], d[H];
#pragma unroll
  for (int r = 1; r <= H; ++r) { s[r - 1] = add<T>(v[r], v[R - r]); d[r - 1] = sub<T>(v[r], v[R - r]); }
  C<T> y0 = v[0];
#pragma unroll
  for (int r = 0; r < H; ++r) y0 = add<T>(y0, s[r]);
  C<T> out[R];
  out[0] = y0;
#pragma unroll
  for (int k = 1; k <= H; ++k) {
    C<T> a = v[0], b = mkc<T>(0, 0);
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      const int rk = (r * k) % R;
      const int q = rk <= H ? rk : R - rk;         // cos(2pi rk/R) = cos(2pi q/R)
      const T sg = rk <= H ? (T)1 : (T)-1;          // sin flips for rk > R/2
      const T c = (T)(R == 3 ? cs3(q) : (R == 5 ? cs5(q) : (R == 7 ? cs7(q) : (R == 11 ? cs11(q) : cs13(q)))));
      const T sn = sg * (T)(R == 3 ? sn3(q) : (R == 5 ? sn5(q) : (R == 7 ? sn7(q) : (R == 11 ? sn11(q) : sn13(q)))));
      a.x += s[r - 1].x * c; a.y += s[r - 1].y * c;
      b.x += d[r - 1].x * sn; b.y += d[r - 1].y * sn;
    }
    // forward: y_k = a - i b, y_{R-k} = a + i b (W = e^{-2 pi i/R}); inverse: swapped
    const C<T> ib = mkc<T>(-b.y, b.x);
    out[k] = inv ? add<T>(a, ib) : sub<T>(a, ib);
    out[R - k] = inv ? sub<T>(a, ib) : add<T>(a, ib);
  }
#pragma unroll
  for (int k = 0; k < R; ++k) v[k] = out[k];
}

template <typename T, int R>
__device__ __forceinline__ void dft_small(C<T>* v, bool inv) {
  if constexpr (R == 2) {
    const C<T> a = v[0], b = v[1];
    v[0] = add<T>(a, b);
    v[1] = sub<T>(a, b);
  } else if constexpr (R == 4) {
    const C<T> t0 = add<T>(v[0], v[2]), t1 = sub<T>(v[0], v[2]);
    const C<T> t2 = add<T>(v[1], v[3]), t3 = rot<T>(sub<T>(v[1], v[3]), inv);
    v[0] = add<T>(t0, t2);
    v[2] = sub<T>(t0, t2);
    v[1] = add<T>(t1, t3);
    v[3] = sub<T>(t1, t3);
  } else if constexpr (R == 8) {
    const T h = (T)0.707106781186547524401;
    C<T> a[4], b[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) { a[k] = add<T>(v[k], v[k + 4]); b[k] = sub<T>(v[k], v[k + 4]); }
    // b_r *= W_8^r
    b[1] = inv ? mkc<T>(h * (b[1].x - b[1].y), h * (b[1].x + b[1].y)) : mkc<T>(h * (b[1].x + b[1].y), h * (b[1].y - b[1].x));
    b[2] = rot<T>(b[2], inv);
    b[3] = inv ? mkc<T>(-h * (b[3].x + b[3].y), h * (b[3].x - b[3].y)) : mkc<T>(h * (b[3].y - b[3].x), -h * (b[3].x + b[3].y));
    dft_small<T, 4>(a, inv);
    dft_small<T, 4>(b, inv);
#pragma unroll
    for (int k = 0; k < 4; ++k) { v[2 * k] = a[k]; v[2 * k + 1] = b[k]; }
  } else {
    dft_odd<T, R>(v, inv);
  }
}

// One register-butterfly stage of radix R.
template <typename T, int R, int VPT>
__device__ __forceinline__ void stage_reg(C<T>* buf, int n, int Ns, const C<T>* __restrict__ tw, bool inv) {
  constexpr int BT = (VPT + R - 1) / R;
  const int nb = n / R, step = n / (Ns * R);
  C<T> v[BT][R];
#pragma unroll
  for (int q = 0; q < BT; ++q) {
    const int j = threadIdx.x + q * blockDim.x;
    if (j < nb) {
      const int jm = j % Ns;
#pragma unroll
      for (int r = 0; r < R; ++r) v[q][r] = buf[j + r * nb];
      if (Ns > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) {
          const C<T> w = tw[(r * jm) * step];
          v[q][r] = inv ? mulc<T>(v[q][r], w) : mul<T>(v[q][r], w);
        }
      }
      dft_small<T, R>(v[q], inv);
    }
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < BT; ++q) {
    const int j = threadIdx.x + q * blockDim.x;
    if (j < nb) {
      const int jm = j % Ns;
      const int base = (j - jm) * R + jm;
#pragma unroll
      for (int r = 0; r < R; ++r) buf[base + r * Ns] = v[q][r];
    }
  }
  __syncthreads();
}

// Running sum of a dot-product stage.  FP32: compensated (TwoSum of each
// addition, errors collected separately), so an R-term sum loses no more than
// its terms' own roundings -- a plain FP32 sum over a large prime radix (a
// prime 2L-1 such as 599 at L = 300 makes the whole FFT one R-term stage)
// grows its error with R and costs the mixed path's 1e-6.  FP64: plain sum.
template <typename T>
__device__ __forceinline__ void acc_add(T& s, T& c, T x) { s += x; }
template <>
__device__ __forceinline__ void acc_add<float>(float& s, float& c, float x) {
  const float t = __fadd_rn(s, x);
  const float v = __fsub_rn(t, s);
  c = __fadd_rn(c, __fadd_rn(__fsub_rn(s, __fsub_rn(t, v)), __fsub_rn(x, v)));
  s = t;
}

// Generic radix stage: every output an R-term dot product (odd primes > 7).
template <typename T, int VPT>
__device__ __forceinline__ void stage_dot(C<T>* buf, int n, int Ns, int R, const C<T>* __restrict__ tw, bool inv) {
  const int NsR = Ns * R, stride = n / R, step = n / NsR;
  C<T> val[VPT];
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const int o = threadIdx.x + v * blockDim.x;
    if (o < n) {
      const int om = o % NsR;
      const int j = (o / NsR) * Ns + (o % Ns);
      T ar = 0, ai = 0, cr = 0, ci = 0;
      int e = 0;
      for (int r = 0; r < R; ++r) {
        const C<T> x = buf[j + r * stride];
        const C<T> w = tw[e * step];
        const T wi = inv ? -w.y : w.y;
        acc_add<T>(ar, cr, x.x * w.x - x.y * wi);
        acc_add<T>(ai, ci, x.x * wi + x.y * w.x);
        e += om;
        if (e >= NsR) e -= NsR;
      }
      val[v] = mkc<T>(ar + cr, ai + ci);
    }
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < VPT; ++v) {
    const int o = threadIdx.x + v * blockDim.x;
    if (o < n) buf[o] = val[v];
  }
  __syncthreads();
}

}  // namespace fftk

// forward: e^{-}, unnormalised; inverse (inv = true): e^{+}, unnormalised.
// Requires blockDim.x * VPT >= d.n; all threads of the block must call it.
template <typename T, int VPT>
__device__ void fft_inplace(typename cplx<T>::t* buf, const FftDesc& d, const typename cplx<T>::t* __restrict__ tw,
                            bool inv) {
  int Ns = 1;
  for (int s = 0; s < d.nrad; ++s) {
    const int R = d.rad[s];
    switch (R) {
      case 2: fftk::stage_reg<T, 2, VPT>(buf, d.n, Ns, tw, inv); break;
      case 3: fftk::stage_reg<T, 3, VPT>(buf, d.n, Ns, tw, inv); break;
      case 4: fftk::stage_reg<T, 4, VPT>(buf, d.n, Ns, tw, inv); break;
      case 5: fftk::stage_reg<T, 5, VPT>(buf, d.n, Ns, tw, inv); break;
      case 7: fftk::stage_reg<T, 7, VPT>(buf, d.n, Ns, tw, inv); break;
      case 8: fftk::stage_reg<T, 8, VPT>(buf, d.n, Ns, tw, inv); break;
      // 11 and 13 in registers in single precision (two butterflies of 13 double
      // values per thread would not fit); double keeps the dot-product stage
      case 11:
        if constexpr (sizeof(T) == 4) fftk::stage_reg<T, 11, VPT>(buf, d.n, Ns, tw, inv);
        else fftk::stage_dot<T, VPT>(buf, d.n, Ns, R, tw, inv);
        break;
      case 13:
        if constexpr (sizeof(T) == 4) fftk::stage_reg<T, 13, VPT>(buf, d.n, Ns, tw, inv);
        else fftk::stage_dot<T, VPT>(buf, d.n, Ns, R, tw, inv);
        break;
      default: fftk::stage_dot<T, VPT>(buf, d.n, Ns, R, tw, inv); break;
    }
    Ns *= R;
  }
}

// Out-of-place variant: stages alternate between x and y (each n elements);
// a thread holds one butterfly at a time.  Returns the buffer holding the result.
namespace fftk {
template <typename T, int R>
__device__ __forceinline__ void stage_pp(const C<T>* __restrict__ in, C<T>* __restrict__ out, int n, int Ns,
                                         const C<T>* __restrict__ tw, bool inv) {
  const int nb = n / R, step = n / (Ns * R);
  for (int j = threadIdx.x; j < nb; j += blockDim.x) {
    C<T> v[R];
    const int jm = j % Ns;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = in[j + r * nb];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const C<T> w = tw[(r * jm) * step];
        v[r] = inv ? mulc<T>(v[r], w) : mul<T>(v[r], w);
      }
    }
    dft_small<T, R>(v, inv);
    const int base = (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) out[base + r * Ns] = v[r];
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void stage_dot_pp(const C<T>* __restrict__ in, C<T>* __restrict__ out, int n, int Ns,
                                             int R, const C<T>* __restrict__ tw, bool inv) {
  const int NsR = Ns * R, stride = n / R, step = n / NsR;
  for (int o = threadIdx.x; o < n; o += blockDim.x) {
    const int om = o % NsR;
    const int j = (o / NsR) * Ns + (o % Ns);
    T ar = 0, ai = 0, cr = 0, ci = 0;
    int e = 0;
    for (int r = 0; r < R; ++r) {
      const C<T> x = in[j + r * stride];
      const C<T> w = tw[e * step];
      const T wi = inv ? -w.y : w.y;
      acc_add<T>(ar, cr, x.x * w.x - x.y * wi);
      acc_add<T>(ai, ci, x.x * wi + x.y * w.x);
      e += om;
      if (e >= NsR) e -= NsR;
    }
    out[o] = mkc<T>(ar + cr, ai + ci);
  }
  __syncthreads();
}
}  // namespace fftk

template <typename T>
__device__ typename cplx<T>::t* fft_pp(typename cplx<T>::t* x, typename cplx<T>::t* y, const FftDesc& d,
                                       const typename cplx<T>::t* __restrict__ tw, bool inv) {
  int Ns = 1;
  for (int s = 0; s < d.nrad; ++s) {
    const int R = d.rad[s];
    switch (R) {
      case 2: fftk::stage_pp<T, 2>(x, y, d.n, Ns, tw, inv); break;
      case 3: fftk::stage_pp<T, 3>(x, y, d.n, Ns, tw, inv); break;
      case 4: fftk::stage_pp<T, 4>(x, y, d.n, Ns, tw, inv); break;
      case 5: fftk::stage_pp<T, 5>(x, y, d.n, Ns, tw, inv); break;
      case 7: fftk::stage_pp<T, 7>(x, y, d.n, Ns, tw, inv); break;
      case 8: fftk::stage_pp<T, 8>(x, y, d.n, Ns, tw, inv); break;
      case 11: fftk::stage_pp<T, 11>(x, y, d.n, Ns, tw, inv); break;
      case 13: fftk::stage_pp<T, 13>(x, y, d.n, Ns, tw, inv); break;
      default: fftk::stage_dot_pp<T>(x, y, d.n, Ns, R, tw, inv); break;
    }
    typename cplx<T>::t* t = x;
    x = y;
    y = t;
    Ns *= R;
  }
  return x;
}

// Two sequences of the same length at once: the second at x + off (its
// ping-pong partner at y + off).  Each stage runs the butterflies of both
// sequences between one pair of barriers.  Returns the buffer holding the
// first result (the second is at the same place + off).
namespace fftk {
template <typename T, int R>
__device__ __forceinline__ void stage_pp2(const C<T>* __restrict__ in, C<T>* __restrict__ out, int n, int off, int Ns,
                                          const C<T>* __restrict__ tw, bool inv) {
  const int nb = n / R, step = n / (Ns * R);
  for (int jj = threadIdx.x; jj < 2 * nb; jj += blockDim.x) {
    const int sq = jj >= nb ? 1 : 0, j = jj - sq * nb;
    const C<T>* src = in + sq * off;
    C<T> v[R];
    const int jm = j % Ns;
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = src[j + r * nb];
    if (Ns > 1) {
#pragma unroll
      for (int r = 1; r < R; ++r) {
        const C<T> w = tw[(r * jm) * step];
        v[r] = inv ? mulc<T>(v[r], w) : mul<T>(v[r], w);
      }
    }
    dft_small<T, R>(v, inv);
    C<T>* dst = out + sq * off + (j - jm) * R + jm;
#pragma unroll
    for (int r = 0; r < R; ++r) dst[r * Ns] = v[r];
  }
  __syncthreads();
}
}  // namespace fftk

template <typename T>
__device__ typename cplx<T>::t* fft_pp2(typename cplx<T>::t* x, typename cplx<T>::t* y, int off, const FftDesc& d,
                                        const typename cplx<T>::t* __restrict__ tw, bool inv) {
  int Ns = 1;
  for (int s = 0; s < d.nrad; ++s) {
    const int R = d.rad[s];
    switch (R) {
      case 2: fftk::stage_pp2<T, 2>(x, y, d.n, off, Ns, tw, inv); break;
      case 3: fftk::stage_pp2<T, 3>(x, y, d.n, off, Ns, tw, inv); break;
      case 4: fftk::stage_pp2<T, 4>(x, y, d.n, off, Ns, tw, inv); break;
      case 5: fftk::stage_pp2<T, 5>(x, y, d.n, off, Ns, tw, inv); break;
      case 7: fftk::stage_pp2<T, 7>(x, y, d.n, off, Ns, tw, inv); break;
      case 8: fftk::stage_pp2<T, 8>(x, y, d.n, off, Ns, tw, inv); break;
      default:  // other radices: one sequence after the other
        fftk::stage_dot_pp<T>(x, y, d.n, Ns, R, tw, inv);
        fftk::stage_dot_pp<T>(x + off, y + off, d.n, Ns, R, tw, inv);
        break;
    }
    typename cplx<T>::t* t = x;
    x = y;
    y = t;
    Ns *= R;
  }
  return x;
}

constexpr int kFftVPT = 16;          // outputs per thread per stage (in-place variant)
constexpr int kFftMaxThreads = 512;  // kFftVPT * kFftMaxThreads >= largest FFT (8192)

// In-place FFT of a power-of-two length (radices 8, 4 and 2 only: a short
// instantiation for the Bluestein convolution below); each thread holds VPT
// values per stage.  Needs blockDim.x * VPT >= d.n.
template <typename T, int VPT>
__device__ void fft_inplace_pow2(typename cplx<T>::t* buf, const FftDesc& d, const typename cplx<T>::t* __restrict__ tw,
                                 bool inv) {
  int Ns = 1;
  for (int s = 0; s < d.nrad; ++s) {
    const int R = d.rad[s];
    if (R == 8) fftk::stage_reg<T, 8, VPT>(buf, d.n, Ns, tw, inv);
    else if (R == 4) fftk::stage_reg<T, 4, VPT>(buf, d.n, Ns, tw, inv);
    else fftk::stage_reg<T, 2, VPT>(buf, d.n, Ns, tw, inv);
    Ns *= R;
  }
}

// Kernels whose only large FFT is a Bluestein one run 1024-thread blocks with
// 8 values per thread (the butterflies stay in 64 registers); kernels that
// also hold other FFTs keep 512 threads and 16 values.
constexpr int kBsVPT = 8;
constexpr int kBsMaxThreads = 1024;

// Bluestein's chirp-z form of a DFT of any length M.  With c_n = e^{-i pi n^2 / M},
// nk = (n^2 + k^2 - (k - n)^2) / 2 turns the DFT into
//   X_k = c_k sum_{n<M} (x_n c_n) conj(c_{k-n}),
// a convolution with lags in (-M, M), exact as a circular convolution of any
// length NB >= 2M - 1 (here a power of two).  It runs in place over
// buf[0, NB) (NB = fB.n): x_n c_n zero-padded to NB, FFT_NB, times chirpF (the
// DFT of conj(c) placed circularly, pre-scaled by 1/NB), inverse FFT_NB, times
// c_k.  Input and output in buf[0, M).  The inverse DFT (e^{+}) is the
// conjugate of the forward DFT of the conjugate.  Needs blockDim.x * VPT
// >= NB; every thread of the block calls it, after the input is in place and
// visible.
template <typename T, int VPT>
__device__ void fft_bluestein(typename cplx<T>::t* buf, int M, const FftDesc& fB,
                              const typename cplx<T>::t* __restrict__ twB,
                              const typename cplx<T>::t* __restrict__ chirp,
                              const typename cplx<T>::t* __restrict__ chirpF, bool inv) {
  using CT = typename cplx<T>::t;
  const int NB = fB.n;
  for (int n = threadIdx.x; n < NB; n += blockDim.x) {
    CT v = mkc<T>(0, 0);
    if (n < M) {
      v = buf[n];
      if (inv) v.y = -v.y;
      v = fftk::mul<T>(v, chirp[n]);
    }
    buf[n] = v;
  }
  __syncthreads();
  fft_inplace_pow2<T, VPT>(buf, fB, twB, false);
  for (int k = threadIdx.x; k < NB; k += blockDim.x) buf[k] = fftk::mul<T>(buf[k], chirpF[k]);
  __syncthreads();
  fft_inplace_pow2<T, VPT>(buf, fB, twB, true);
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    CT v = fftk::mul<T>(buf[k], chirp[k]);
    if (inv) v.y = -v.y;
    buf[k] = v;
  }
  __syncthreads();
}

// The length-M FFT of the MW stages (M = 2L - 1): tables of both routes.
template <typename T>
struct FftM {
  FftDesc d;                                 // mixed-radix factorisation of M
  const typename cplx<T>::t* tw;             // e^{-2 pi i k / M}, k < M
  FftDesc dB;                                // Bluestein: the power of two NB >= 2M - 1
  const typename cplx<T>::t* twB;            // e^{-2 pi i k / NB}, k < NB
  const typename cplx<T>::t* chirp;          // e^{-i pi n^2 / M}, n < M
  const typename cplx<T>::t* chirpF;         // DFT_NB of conj(chirp), circular, / NB
};

// DFT of length M of x[0, M): mixed radix with y[0, M) as the ping-pong
// partner (BS = false; returns x or y), or Bluestein in place over x[0, NB)
// with VPT values per thread (BS = true; returns x).
template <typename T, bool BS, int VPT = kBsVPT>
__device__ __forceinline__ typename cplx<T>::t* fft_m(typename cplx<T>::t* x, typename cplx<T>::t* y,
                                                      const FftM<T>& f, bool inv) {
  if constexpr (BS) {
    fft_bluestein<T, VPT>(x, f.d.n, f.dB, f.twB, f.chirp, f.chirpF, inv);
    return x;
  } else {
    return fft_pp<T>(x, y, f.d, f.tw, inv);
  }
}
