// fft.cuh -- in-place mixed-radix FFT of one sequence held in shared memory.
//
// Stockham formulation: stage k with radix R and span Ns = R_0...R_{k-1} writes
//   out[o] = sum_{r<R} in[j + r n/R] * W_{Ns R}^{r (o mod Ns R)},
//   j = (o / (Ns R)) Ns + (o mod Ns),   W_q = e^{-2 pi i / q},
// which leaves the DFT in natural order after the last stage.  Every output is
// an independent R-term dot product, so a thread computes its outputs into
// registers, the block synchronises, and the outputs overwrite the inputs (one
// shared buffer of n elements).  Odd prime radices (the 2L-1 lengths have
// factors such as 73 or 127) use the same dot product; no Bluestein step is
// needed.  Twiddles come from one table of e^{-2 pi i k / n}, k < n.
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

// forward: e^{-}, unnormalised; inverse (inv = true): e^{+}, unnormalised.
// Requires blockDim.x * VPT >= d.n; all threads of the block must call it.
template <typename T, int VPT>
__device__ void fft_inplace(typename cplx<T>::t* buf, const FftDesc& d,
                            const typename cplx<T>::t* __restrict__ tw, bool inv) {
  typedef typename cplx<T>::t C;
  const int n = d.n;
  int Ns = 1;
  for (int s = 0; s < d.nrad; ++s) {
    const int R = d.rad[s], NsR = Ns * R, stride = n / R, step = n / NsR;
    C val[VPT];
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int o = threadIdx.x + v * blockDim.x;
      if (o < n) {
        const int om = o % NsR;
        const int j = (o / NsR) * Ns + (o % Ns);
        T ar = 0, ai = 0;
        int e = 0;
        for (int r = 0; r < R; ++r) {
          const C x = buf[j + r * stride];
          const C w = tw[e * step];
          const T wi = inv ? -w.y : w.y;
          ar += x.x * w.x - x.y * wi;
          ai += x.x * wi + x.y * w.x;
          e += om;
          if (e >= NsR) e -= NsR;
        }
        val[v] = mkc<T>(ar, ai);
      }
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < VPT; ++v) {
      const int o = threadIdx.x + v * blockDim.x;
      if (o < n) buf[o] = val[v];
    }
    __syncthreads();
    Ns = NsR;
  }
}

constexpr int kFftVPT = 16;     // outputs per thread per stage
constexpr int kFftMaxThreads = 512;  // kFftVPT * kFftMaxThreads >= largest FFT (8192)
