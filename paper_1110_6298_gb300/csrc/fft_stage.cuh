// fft_stage.cuh -- helpers shared by the FFT-stage kernels (kernels_fft.cu:
// forward and inverse stages; kernels_fft_adj.cu: their adjoints): complex
// arithmetic in the stage precision T, the map and F+ layouts, and the launch
// geometry of one block per ring or per (m, map).
#pragma once
#include <cmath>

#include "fft.cuh"
#include "internal.h"

namespace {


template <typename T>
using C = typename cplx<T>::t;

template <typename T>
__device__ __forceinline__ C<T> cmul(C<T> a, C<T> b) {
  return mkc<T>(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
template <typename T>
__device__ __forceinline__ C<T> cmulc(C<T> a, C<T> b) {  // a * conj(b)
  return mkc<T>(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename T>
__device__ __forceinline__ C<T> cscale(C<T> a, T s) { return mkc<T>(a.x * s, a.y * s); }
template <typename T>
__device__ __forceinline__ C<T> from64(double2 v) { return mkc<T>((T)v.x, (T)v.y); }

// Element idx of the inverse contraction's F+ buffer: FP64 complex on the FP64
// path; on the mixed path float-float pairs (re_hi, re_lo, im_hi, im_lo) in the
// same 16 bytes, read as hi + lo in single precision.
template <typename T>
__device__ __forceinline__ C<T> load_fplus(const double2* __restrict__ Fp, long long idx) {
  if constexpr (sizeof(T) == 4) {
    const float4 v = reinterpret_cast<const float4*>(Fp)[idx];
    return mkc<T>(v.x + v.y, v.z + v.w);
  } else {
    return from64<T>(Fp[idx]);
  }
}
__device__ __forceinline__ double2 to64(double2 v) { return v; }
__device__ __forceinline__ double2 to64(float2 v) { return make_double2(v.x, v.y); }

// (-1)^k for any integer k
__device__ __forceinline__ int parity_sign(int k) { return (k & 1) ? -1 : 1; }

// i^k as (re, im)
__device__ __forceinline__ double2 ipow(int k) {
  const int r = k & 3;  // two's complement keeps k mod 4 for negative k
  return make_double2(r == 0 ? 1.0 : (r == 2 ? -1.0 : 0.0), r == 1 ? 1.0 : (r == 3 ? -1.0 : 0.0));
}

// x * i^k, exact (swaps and sign changes only)
template <typename T>
__device__ __forceinline__ C<T> mul_ipow(C<T> x, int k) {
  switch (k & 3) {
    case 0: return x;
    case 1: return mkc<T>(-x.y, x.x);
    case 2: return mkc<T>(-x.x, -x.y);
    default: return mkc<T>(x.y, -x.x);
  }
}

struct Dims {
  int L, M, N, B;
  long long nmw;  // samples per map
  int nreal;      // real-signal plans: real maps in the caller's buffer (map b packs maps 2b, 2b+1)
  int b0;         // first map of the launch (blockIdx.y counts from it)
};

// Sample i of map b.  Complex plans: the caller's complex map at moff[b].
// Real-signal plans: real maps 2b and 2b+1 (back to back, nmw doubles each) as
// the real and imaginary part; the second is zero past the last real map.
template <typename T, bool RealIo>
__device__ __forceinline__ C<T> load_sample(const void* __restrict__ map, const long long* __restrict__ moff,
                                            const Dims& d, int b, long long i) {
  if constexpr (RealIo) {
    const double* fr = static_cast<const double*>(map) + (long long)(2 * b) * d.nmw;
    const double im = (2 * b + 1 < d.nreal) ? fr[d.nmw + i] : 0.0;
    return mkc<T>((T)fr[i], (T)im);
  } else {
    return from64<T>(static_cast<const double2*>(map)[moff[b] + i]);
  }
}

// Store sample i of map b (the inverse of load_sample's layout; real-signal
// plans keep the real part in map 2b and the imaginary part in map 2b+1).
template <typename T, bool RealIo>
__device__ __forceinline__ void store_sample(void* __restrict__ map, const long long* __restrict__ moff, const Dims& d,
                                             int b, long long i, C<T> v) {
  if constexpr (RealIo) {
    double* fr = static_cast<double*>(map) + (long long)(2 * b) * d.nmw;
    fr[i] = (double)v.x;
    if (2 * b + 1 < d.nreal) fr[d.nmw + i] = (double)v.y;
  } else {
    static_cast<double2*>(map)[moff[b] + i] = make_double2((double)v.x, (double)v.y);
  }
}

__device__ __forceinline__ int spin_of(const int* spins, int b) { return spins[b]; }


template <typename K>
cudaError_t set_smem(K kernel, int bytes) {
  if (bytes > 48 * 1024) return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
  return cudaSuccess;
}

Dims dims_of(const mw_plan* p) {
  Dims d;
  d.L = p->L; d.M = p->M; d.N = p->N; d.B = p->B;
  d.nmw = (long long)(p->L - 1) * p->M + 1;
  d.nreal = p->real ? p->nreal : 0;
  d.b0 = 0;
  return d;
}

// block size of the ping-pong kernels (any size works; a multiple of 32 up to 512)
int threads_pp(int n) {
  int t = (n + 3) / 4;
  t = ((t + 31) / 32) * 32;
  return t < 32 ? 32 : (t > kFftMaxThreads ? kFftMaxThreads : t);
}
// block size of the in-place kernels: kFftVPT * threads >= n
int threads_inplace(int n) {
  int t = (n + kFftVPT - 1) / kFftVPT;
  t = ((t + 31) / 32) * 32;
  return t < 32 ? 32 : t;
}
constexpr int kSmemMax = 232448;

template <typename T> int pp_bytes(int n) { return 2 * n * (int)sizeof(C<T>); }

// Tables of the plan's length-M FFT (both routes; the Bluestein ones are null
// when the plan runs M by mixed radix).
template <typename T>
FftM<T> fft_m_of(const mw_plan* p) {
  FftM<T> f;
  f.d = p->fM;
  f.tw = (const C<T>*)p->d_twM;
  f.dB = p->fB;
  f.twB = (const C<T>*)p->d_twB;
  f.chirp = (const C<T>*)p->d_chirp;
  f.chirpF = (const C<T>*)p->d_chirpF;
  return f;
}
// shared memory (complex values) and block size of a kernel whose only FFT is
// the length-M one: a ping-pong pair of M, or the Bluestein length NB in place
int m_elems(const mw_plan* p) { return p->bluestein && p->fB.n > 2 * p->M ? p->fB.n : 2 * p->M; }
// (vpt: values per thread of the Bluestein FFTs, kBsVPT in the forward and
// inverse kernels, kFftVPT in the adjoints).  In single precision the
// mixed-radix route takes at most 256 threads: three 64 KB blocks per SM at
// 2L-1 = 4095 then overlap one another's ring loads and FFT stages (the phi
// stage measured 3.56 against 3.72 ms per round trip at L = 2048, B = 16 with
// 512 threads, 3.94 with 384); double precision, one 128 KB block per SM,
// keeps up to 512.
int m_threads(const mw_plan* p, int vpt = kBsVPT) {
  const int a = threads_pp(p->M);
  if (p->bluestein) {
    const int b = ((p->fB.n + vpt - 1) / vpt + 31) / 32 * 32;
    return a > b ? a : b;
  }
  return (p->prec != MW_PREC_FP64 && a > 256) ? 256 : a;
}

}  // namespace

#define DISPATCH(p, fn, ...) ((p)->prec == MW_PREC_FP64 ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

#define DISPATCH2(p, fn, R, ...) \
  ((p)->prec == MW_PREC_FP64 ? fn<double, R>(__VA_ARGS__) : fn<float, R>(__VA_ARGS__))
