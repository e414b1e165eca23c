// kernels_fft.cu -- the O(L^2 log L) stages of the MW transforms and their adjoints.
//
// Forward (Sec. IV-D):
//   phi_forward   : G_m(theta_t) = 2pi/M sum_p f(theta_t, phi_p) e^{-i m phi_p}, one
//                   block per ring; the pole ring f(pi,0) e^{i s phi} transforms in
//                   closed form to 2 pi f(pi,0) delta_{m,s}.
//   theta_forward : one block per (m, map): periodic extension with parity
//                   (-1)^(m+s), DFT over the 2L-1 extended nodes with the half-sample
//                   phase e^{-i m' pi/M} (F_mm'), the weight convolution of
//                   Eq. (Gmm_convolution) by its even lags (two circular
//                   convolutions of about 1.5 L points), then the +-m' fold
//                   G+_{m,m'} = G_mm' + (-1)^(m+s) G_{m,-m'} used by the Wigner stage.
// Inverse (Sec. IV-E):
//   theta_inverse : one block per (m, map): phase (-1)^s i^-(m+s) of Eq. (Fmm),
//                   unfold F_{m,-m'} = (-1)^(m+s) F_mm' (Eq. Fmm_sym1), inverse DFT over
//                   the extended nodes (Eq. Fmt), keep t < L.
//   phi_inverse   : one block per ring: inverse DFT in phi (Eq. f_pfft); the pole
//                   ring keeps its phi = 0 sample.
// Adjoints: each stage transposed and conjugated, run in reverse order.
//
// T is the arithmetic type of these stages (double for the FP64 path, float for
// the mixed path).  Map and f_lm buffers are always complex double.
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

// --------------------------------------------------------------------------
// forward
// --------------------------------------------------------------------------
template <typename T, bool RealIo>
__global__ void __launch_bounds__(kFftMaxThreads) k_phi_forward(Dims d, FftDesc fM, const C<T>* __restrict__ twM, const void* __restrict__ map,
                              const long long* __restrict__ moff,
                              C<T>* __restrict__ Gt /* [B][M][L] */, const int* __restrict__ spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int t = blockIdx.x, b = blockIdx.y;
  const int L = d.L, M = d.M;
  C<T>* out = Gt + (long long)b * M * L;
  if (t == L - 1) {  // pole ring: 2 pi f(pi,0) delta_{m,s}
    const int s = spin_of(spins, b);
    const C<T> fp = load_sample<T, RealIo>(map, moff, d, b, (long long)(L - 1) * M);
    const T tp = (T)(2.0 * M_PI);
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const int m = i - (L - 1);
      out[(long long)i * L + t] = (m == s) ? mkc<T>(fp.x * tp, fp.y * tp) : mkc<T>(0, 0);
    }
    return;
  }
  for (int p = threadIdx.x; p < M; p += blockDim.x) buf[p] = load_sample<T, RealIo>(map, moff, d, b, (long long)t * M + p);
  __syncthreads();
  const C<T>* res = fft_pp<T>(buf, buf + M, fM, twM, false);
  const T sc = (T)(2.0 * M_PI / M);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const int m = i - (L - 1);
    const int k = m < 0 ? m + M : m;
    out[(long long)i * L + t] = cscale<T>(res[k], sc);
  }
}

// Forward theta stage by even lags.  The weights w(k) vanish at odd k except
// k = +-1, and the w(+-1) terms drop out of every f_lm: the extended G~_m is
// reflection-symmetric about theta = pi (G~(2 pi - theta) = (-1)^(m+s) G~(theta)),
// so F_{m,-m''} = (-1)^(m+s) F_mm'', their contribution to G_mm' is odd under
// m' -> -m' and cancels in the fold G+ = G_mm' + (-1)^(m+s) G_{m,-m'} (at m' = 0
// it multiplies Delta_{0m} Delta_{0,-s}, which vanishes when m+s is odd).  With
// even lags only, Eq. (Gmm_convolution) splits into two convolutions with the
// kernel w(2d): even m'' = 2j into even m' = 2i, odd into odd, each a circular
// convolution of length NE (about 1.5 L) covering the lags that occur; and the
// even-lag G_mm' obeys the same symmetry, so G+_{m,m'} = 2 G_mm' for m' > 0 and
// only m' >= 0 is formed.  One block per (m, map): extension, FFT_M with the
// half-sample phase, the split into the two halves, inverse FFT_NE, product
// with the kernel's DFT, FFT_NE, every FFT in place (2 NE complex values of
// shared memory).
// Forward theta stage by even lags.  The weights w(k) vanish at odd k except
// k = +-1, and the w(+-1) terms drop out of every f_lm: the extended G~_m is
// reflection-symmetric about theta = pi (G~(2 pi - theta) = (-1)^(m+s) G~(theta)),
// so F_{m,-m''} = (-1)^(m+s) F_mm'', their contribution to G_mm' is odd under
// m' -> -m' and cancels in the fold G+ = G_mm' + (-1)^(m+s) G_{m,-m'} (at m' = 0
// it multiplies Delta_{0m} Delta_{0,-s}, which vanishes when m+s is odd).  With
// even lags only, Eq. (Gmm_convolution) splits into two convolutions with the
// kernel w(2d): even m'' = 2j into even m' = 2i, odd into odd, each a circular
// convolution of length NE (about 1.5 L) covering the lags that occur; and the
// even-lag G_mm' obeys the same symmetry, so G+_{m,m'} = 2 G_mm' for m' > 0 and
// only m' >= 0 is formed.  One block per (m, map): extension, FFT_M with the
// half-sample phase, the split into the two halves, inverse FFT_NE, product
// with the kernel's DFT, FFT_NE (ping-pong FFTs; max(2M, 4 NE) complex values of
// shared memory, against 2 N with N >= 4L-3 for the direct convolution).
constexpr int kEvenVPT = 8;  // values of F a thread carries through the split (512 threads up to M = 4095)

template <typename T>
__global__ void __launch_bounds__(kFftMaxThreads) k_theta_forward_even(
    Dims d, FftDesc fM, FftDesc fE, const C<T>* __restrict__ twM, const C<T>* __restrict__ twE,
    const C<T>* __restrict__ phase, const C<T>* __restrict__ Ue, const C<T>* __restrict__ Uo,
    const C<T>* __restrict__ Gt, C<T>* __restrict__ Gp, const int* __restrict__ spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int L = d.L, M = d.M, NE = fE.n;
  C<T>* X = buf;           // even half (ping-pong pair X, X + NE)
  C<T>* Y = buf + 2 * NE;  // odd half (Y, Y + NE)
  const int im = blockIdx.x, b = blockIdx.y;
  const int m = im - (L - 1);
  const int s = spin_of(spins, b);
  const T sg = (T)parity_sign(m + s);
  const C<T>* g = Gt + ((long long)b * M + im) * L;
  // periodic extension over the 2L-1 nodes, FFT_M
  for (int t = threadIdx.x; t < M; t += blockDim.x) buf[t] = (t < L) ? g[t] : cscale<T>(g[2 * L - 2 - t], sg);
  __syncthreads();
  const C<T>* F = fft_pp<T>(buf, buf + M, fM, twM, false);
  // F_mm'' times the half-sample phase, split by the parity of m'' into the
  // halves (m'' = 2j at X[j mod NE], m'' = 2j+1 at Y[j mod NE]), zero elsewhere
  C<T> v[kEvenVPT];
#pragma unroll
  for (int r = 0; r < kEvenVPT; ++r) {
    const int k = threadIdx.x + r * blockDim.x;
    if (k < M) {
      const int mp = (k <= L - 1) ? k : k - M;
      v[r] = cmul<T>(F[k], phase[mp + L - 1]);
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < NE; k += blockDim.x) X[k] = Y[k] = mkc<T>(0, 0);
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kEvenVPT; ++r) {
    const int k = threadIdx.x + r * blockDim.x;
    if (k < M) {
      const int mp = (k <= L - 1) ? k : k - M;
      const int j = (mp - (mp & 1)) / 2;  // floor(mp / 2)
      const int idx = j < 0 ? j + NE : j;
      if (mp & 1) Y[idx] = v[r];
      else X[idx] = v[r];
    }
  }
  __syncthreads();
  C<T>* xe = fft_pp<T>(X, X + NE, fE, twE, true);
  C<T>* xo = fft_pp<T>(Y, Y + NE, fE, twE, true);
  for (int k = threadIdx.x; k < NE; k += blockDim.x) {
    xe[k] = cmul<T>(xe[k], Ue[k]);
    xo[k] = cmul<T>(xo[k], Uo[k]);
  }
  __syncthreads();
  xe = fft_pp<T>(xe, xe == X ? X + NE : X, fE, twE, false);
  xo = fft_pp<T>(xo, xo == Y ? Y + NE : Y, fE, twE, false);
  // G+_{m,0} = G_m0, G+_{m,m'} = 2 G_mm' (m' > 0): m' = 2i from the even half, 2i+1 from the odd
  C<T>* out = Gp + ((long long)b * M + im) * L;
  for (int mp = threadIdx.x; mp < L; mp += blockDim.x) {
    const C<T> a = (mp & 1) ? xo[mp >> 1] : xe[mp >> 1];
    out[mp] = mp == 0 ? a : cscale<T>(a, (T)2);
  }
}

// --------------------------------------------------------------------------
// inverse
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kFftMaxThreads) k_theta_inverse(Dims d, FftDesc fM, const C<T>* __restrict__ twM, const C<T>* __restrict__ phase,
                                const double2* __restrict__ Gp, C<T>* __restrict__ Gt /* [B][L][M] */,
                                const int* __restrict__ spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int L = d.L, M = d.M;
  const int im = blockIdx.x, b = blockIdx.y;
  const int m = im - (L - 1);
  const int s = spin_of(spins, b);
  // (-1)^s i^-(m+s) and the unfold sign (-1)^(m+s) are applied exactly in T
  const int ph = -(m + s) + ((s & 1) ? 2 : 0);
  const double2* in = Gp + ((long long)b * M + im) * L;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const int mp = (k <= L - 1) ? k : k - M;  // slot of m' in the length-M DFT
    const int a = mp < 0 ? -mp : mp;
    const int q = ph + ((mp < 0 && ((m + s) & 1)) ? 2 : 0);
    const C<T> y = mul_ipow<T>(load_fplus<T>(in, a), q);
    // times e^{+i m' pi / M} = conj(phase)
    buf[k] = cmulc<T>(y, phase[mp + L - 1]);
  }
  __syncthreads();
  const C<T>* res = fft_pp<T>(buf, buf + M, fM, twM, true);
  C<T>* out = Gt + (long long)b * L * M;
  for (int t = threadIdx.x; t < L; t += blockDim.x) out[(long long)t * M + im] = res[t];
}

template <typename T, bool RealIo>
__global__ void __launch_bounds__(kFftMaxThreads) k_phi_inverse(Dims d, FftDesc fM, const C<T>* __restrict__ twM, const C<T>* __restrict__ Gt,
                              void* __restrict__ map, const long long* __restrict__ moff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int L = d.L, M = d.M;
  const int t = blockIdx.x, b = blockIdx.y;
  const C<T>* in = Gt + ((long long)b * L + t) * M;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const int m = (k <= L - 1) ? k : k - M;
    buf[k] = in[m + L - 1];
  }
  __syncthreads();
  const C<T>* res = fft_pp<T>(buf, buf + M, fM, twM, true);
  if (t < L - 1) {
    for (int p = threadIdx.x; p < M; p += blockDim.x) store_sample<T, RealIo>(map, moff, d, b, (long long)t * M + p, res[p]);
  } else if (threadIdx.x == 0) {
    store_sample<T, RealIo>(map, moff, d, b, (long long)(L - 1) * M, res[0]);
  }
}

// --------------------------------------------------------------------------
// adjoint of the forward: Wigner^H (run_wigner mode 1) -> theta_forward^H -> phi_forward^H
// --------------------------------------------------------------------------
template <typename T, bool PP>
__global__ void __launch_bounds__(kFftMaxThreads) k_theta_forward_adjoint(Dims d, FftDesc fM, FftDesc fN, const C<T>* __restrict__ twM,
                                        const C<T>* __restrict__ twN, const C<T>* __restrict__ phase,
                                        const C<T>* __restrict__ V, const double2* __restrict__ Gp,
                                        C<T>* __restrict__ Gt /* [B][L][M] */, const int* __restrict__ spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int L = d.L, M = d.M, N = d.N;
  const int im = blockIdx.x, b = blockIdx.y;
  const int m = im - (L - 1);
  const int s = spin_of(spins, b);
  const T sg = (T)parity_sign(m + s);
  const int ph = -(m + s) + ((s & 1) ? 2 : 0);  // conj of (-1)^s i^(m+s), exact
  const double2* in = Gp + ((long long)b * M + im) * L;
  // G^H_mm' for |m'| <= L-1, zero-padded to N
  for (int k = threadIdx.x; k < N; k += blockDim.x) {
    const int mp = (k <= L - 1) ? k : ((k >= N - (L - 1)) ? k - N : 0x7fffffff);
    if (mp == 0x7fffffff) { buf[k] = mkc<T>(0, 0); continue; }
    const int a = mp < 0 ? -mp : mp;
    const int q = ph + ((mp < 0 && ((m + s) & 1)) ? 2 : 0);
    buf[k] = mul_ipow<T>(load_fplus<T>(in, a), q);
  }
  __syncthreads();
  // convolution^H: zero-pad, inverse DFT, times conj(V), DFT; then the theta-DFT^H:
  // F^H_{m,m''} e^{+i m'' pi/M} placed on the length-M grid, inverse DFT
  C<T>* res;
  if constexpr (PP) {
    C<T>* y = fft_pp<T>(buf, buf + N, fN, twN, true);
    for (int k = threadIdx.x; k < N; k += blockDim.x) y[k] = cmulc<T>(y[k], V[k]);
    __syncthreads();
    C<T>* z = fft_pp<T>(y, (y == buf) ? buf + N : buf, fN, twN, false);
    C<T>* x = (z == buf) ? buf + N : buf;
    for (int k = threadIdx.x; k < M; k += blockDim.x) {
      const int mp = (k <= L - 1) ? k : k - M;
      x[k] = cmulc<T>(z[mp < 0 ? mp + N : mp], phase[mp + L - 1]);
    }
    __syncthreads();
    res = fft_pp<T>(x, z, fM, twM, true);
  } else {
    fft_inplace<T, kFftVPT>(buf, fN, twN, true);
    for (int k = threadIdx.x; k < N; k += blockDim.x) buf[k] = cmulc<T>(buf[k], V[k]);
    __syncthreads();
    fft_inplace<T, kFftVPT>(buf, fN, twN, false);
    C<T> v[kFftVPT];
#pragma unroll
    for (int r = 0; r < kFftVPT; ++r) {
      const int k = threadIdx.x + r * blockDim.x;
      if (k < M) {
        const int mp = (k <= L - 1) ? k : k - M;
        v[r] = cmulc<T>(buf[mp < 0 ? mp + N : mp], phase[mp + L - 1]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < kFftVPT; ++r) {
      const int k = threadIdx.x + r * blockDim.x;
      if (k < M) buf[k] = v[r];
    }
    __syncthreads();
    fft_inplace<T, kFftVPT>(buf, fM, twM, true);
    res = buf;
  }
  // extension^H: G^H(t) = G~^H(t) + (-1)^(m+s) G~^H(2L-2-t) for t <= L-2
  C<T>* out = Gt + (long long)b * L * M;
  for (int t = threadIdx.x; t < L; t += blockDim.x) {
    C<T> a = res[t];
    if (t <= L - 2) {
      const C<T> c = res[2 * L - 2 - t];
      a.x += (T)sg * c.x;
      a.y += (T)sg * c.y;
    }
    out[(long long)t * M + im] = a;
  }
}

template <typename T>
__global__ void __launch_bounds__(kFftMaxThreads) k_phi_forward_adjoint(Dims d, FftDesc fM, const C<T>* __restrict__ twM, const C<T>* __restrict__ Gt,
                                      double2* __restrict__ map, const long long* __restrict__ moff,
                                      const int* __restrict__ spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int L = d.L, M = d.M;
  const int t = blockIdx.x, b = blockIdx.y;
  const C<T>* in = Gt + ((long long)b * L + t) * M;
  double2* f = map + moff[b];
  if (t == L - 1) {  // pole: sum_p e^{-i s phi_p} (2pi/M) sum_m e^{i m phi_p} G^H = 2 pi G^H_s
    if (threadIdx.x == 0) {
      const int s = spin_of(spins, b);
      f[(long long)(L - 1) * M] = to64(cscale<T>(in[s + L - 1], (T)(2.0 * M_PI)));
    }
    return;
  }
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const int m = (k <= L - 1) ? k : k - M;
    buf[k] = in[m + L - 1];
  }
  __syncthreads();
  const C<T>* res = fft_pp<T>(buf, buf + M, fM, twM, true);
  const T sc = (T)(2.0 * M_PI / M);
  for (int p = threadIdx.x; p < M; p += blockDim.x) f[(long long)t * M + p] = to64(cscale<T>(res[p], sc));
}

// --------------------------------------------------------------------------
// adjoint of the inverse: phi_inverse^H -> theta_inverse^H -> Wigner^H (run_wigner mode 0)
// --------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kFftMaxThreads) k_phi_inverse_adjoint(Dims d, FftDesc fM, const C<T>* __restrict__ twM,
                                      const double2* __restrict__ map, const long long* __restrict__ moff,
                                      C<T>* __restrict__ Gt /* [B][M][L] */) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int L = d.L, M = d.M;
  const int t = blockIdx.x, b = blockIdx.y;
  const double2* f = map + moff[b];
  C<T>* out = Gt + (long long)b * M * L;
  if (t == L - 1) {  // only the phi = 0 sample of the pole ring is kept: F^H_m(pi) = x_pole
    const C<T> xp = from64<T>(f[(long long)(L - 1) * M]);
    for (int i = threadIdx.x; i < M; i += blockDim.x) out[(long long)i * L + t] = xp;
    return;
  }
  for (int p = threadIdx.x; p < M; p += blockDim.x) buf[p] = from64<T>(f[(long long)t * M + p]);
  __syncthreads();
  const C<T>* res = fft_pp<T>(buf, buf + M, fM, twM, false);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const int m = i - (L - 1);
    out[(long long)i * L + t] = res[m < 0 ? m + M : m];
  }
}

template <typename T>
__global__ void __launch_bounds__(kFftMaxThreads) k_theta_inverse_adjoint(Dims d, FftDesc fM, const C<T>* __restrict__ twM,
                                        const C<T>* __restrict__ phase, const C<T>* __restrict__ Gt,
                                        C<T>* __restrict__ Gp, const int* __restrict__ spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int L = d.L, M = d.M;
  const int im = blockIdx.x, b = blockIdx.y;
  const int m = im - (L - 1);
  const int s = spin_of(spins, b);
  const T sg = (T)parity_sign(m + s);
  const C<T>* g = Gt + ((long long)b * M + im) * L;
  for (int t = threadIdx.x; t < M; t += blockDim.x) buf[t] = (t < L) ? g[t] : mkc<T>(0, 0);
  __syncthreads();
  const C<T>* res = fft_pp<T>(buf, buf + M, fM, twM, false);
  // F^H_mm' = e^{-i m' pi/M} DFT[m'], folded for the Wigner stage
  C<T>* out = Gp + ((long long)b * M + im) * L;
  for (int mp = threadIdx.x; mp < L; mp += blockDim.x) {
    C<T> a = cmul<T>(res[mp], phase[mp + L - 1]);
    if (mp > 0) {
      const C<T> c = cmul<T>(res[M - mp], phase[-mp + L - 1]);
      a.x += sg * c.x;
      a.y += sg * c.y;
    }
    out[mp] = a;
  }
}

// Pole sample of the forward adjoint, in FP64 for both precisions.  At
// theta_{L-1} = pi the theta-DFT^H and convolution^H collapse to
//   pole = (2 pi / M) sum_{m'} G^H_{s,m'} u(m'),  u(m') = sum_{m''} (-1)^{m''} conj(w(m''-m')),
// and G^H_{s,-m'} = G^H_{s,m'} (the parity (-1)^(m+s) is +1 at m = s), so the sum
// runs over m' >= 0 against u(m') + u(-m').  Evaluated this way the value does not
// inherit the cancellation of the alternating sum over the FFT output.
__global__ void k_pole_forward_adjoint(Dims d, const double2* __restrict__ Gp, const double2* __restrict__ upole,
                                       double2* __restrict__ map, const long long* __restrict__ moff,
                                       const int* __restrict__ spins, int float_float) {
  __shared__ double2 red[256];
  const int b = blockIdx.x, L = d.L, M = d.M;
  const int s = spin_of(spins, b);
  const double2* w = Gp + ((long long)b * M + (s + L - 1)) * L;
  double sr = 0.0, si = 0.0;
  for (int mp = threadIdx.x; mp < L; mp += blockDim.x) {
    double2 x = w[mp];
    if (float_float) {  // mixed path: (re_hi, re_lo, im_hi, im_lo)
      const float4 v = reinterpret_cast<const float4*>(w)[mp];
      x = make_double2((double)v.x + (double)v.y, (double)v.z + (double)v.w);
    }
    const double2 u = upole[mp];
    sr += x.x * u.x - x.y * u.y;
    si += x.x * u.y + x.y * u.x;
  }
  red[threadIdx.x] = make_double2(sr, si);
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) {
      red[threadIdx.x].x += red[threadIdx.x + h].x;
      red[threadIdx.x].y += red[threadIdx.x + h].y;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double2 ph = ipow(-2 * s);  // (-1)^s i^-(m+s) at m = s
    if (s & 1) { ph.x = -ph.x; ph.y = -ph.y; }
    const double c = 2.0 * M_PI / M;
    const double2 v = red[0];
    map[moff[b] + (long long)(L - 1) * M] =
        make_double2(c * (ph.x * v.x - ph.y * v.y), c * (ph.x * v.y + ph.y * v.x));
  }
}

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

template <typename T, bool RealIo>
cudaError_t phi_forward_t(const mw_plan* p, const void* map, cudaStream_t st) {
  const int sm = pp_bytes<T>(p->M);
  cudaError_t e = set_smem(k_phi_forward<T, RealIo>, sm);
  if (e != cudaSuccess) return e;
  k_phi_forward<T, RealIo><<<dim3(p->L, p->B), threads_pp(p->M), sm, st>>>(
      dims_of(p), p->fM, (const C<T>*)p->d_twM, map, p->d_moff, (C<T>*)p->d_Gt, p->d_spins);
  return cudaGetLastError();
}
template <typename T>
cudaError_t theta_forward_t(const mw_plan* p, cudaStream_t st) {
  const int n = 2 * p->M > 4 * p->NE ? 2 * p->M : 4 * p->NE;
  const int sm = n * (int)sizeof(C<T>);
  cudaError_t e = set_smem(k_theta_forward_even<T>, sm);
  if (e != cudaSuccess) return e;
  int nt = ((p->M + kEvenVPT - 1) / kEvenVPT + 31) / 32 * 32;  // every thread carries <= kEvenVPT values of F
  const int pp = threads_pp(p->NE > p->M ? p->NE : p->M);
  if (nt < pp) nt = pp;
  k_theta_forward_even<T><<<dim3(p->M, p->B), nt, sm, st>>>(
      dims_of(p), p->fM, p->fE, (const C<T>*)p->d_twM, (const C<T>*)p->d_twE, (const C<T>*)p->d_phase,
      (const C<T>*)p->d_Ue, (const C<T>*)p->d_Uo, (const C<T>*)p->d_Gt, (C<T>*)p->d_Gp, p->d_spins);
  return cudaGetLastError();
}
template <typename T>
cudaError_t theta_inverse_t(const mw_plan* p, cudaStream_t st) {
  const int sm = pp_bytes<T>(p->M);
  cudaError_t e = set_smem(k_theta_inverse<T>, sm);
  if (e != cudaSuccess) return e;
  k_theta_inverse<T><<<dim3(p->M, p->B), threads_pp(p->M), sm, st>>>(
      dims_of(p), p->fM, (const C<T>*)p->d_twM, (const C<T>*)p->d_phase, p->d_Gp, (C<T>*)p->d_Gt, p->d_spins);
  return cudaGetLastError();
}
template <typename T, bool RealIo>
cudaError_t phi_inverse_t(const mw_plan* p, void* map, cudaStream_t st) {
  const int sm = pp_bytes<T>(p->M);
  cudaError_t e = set_smem(k_phi_inverse<T, RealIo>, sm);
  if (e != cudaSuccess) return e;
  k_phi_inverse<T, RealIo><<<dim3(p->L, p->B), threads_pp(p->M), sm, st>>>(
      dims_of(p), p->fM, (const C<T>*)p->d_twM, (const C<T>*)p->d_Gt, map, p->d_moff);
  return cudaGetLastError();
}
template <typename T>
cudaError_t theta_forward_adjoint_t(const mw_plan* p, cudaStream_t st) {
  cudaError_t e;
  if (pp_bytes<T>(p->N) <= kSmemMax) {
    const int sm = pp_bytes<T>(p->N);
    if ((e = set_smem(k_theta_forward_adjoint<T, true>, sm)) != cudaSuccess) return e;
    k_theta_forward_adjoint<T, true><<<dim3(p->M, p->B), threads_pp(p->N), sm, st>>>(
        dims_of(p), p->fM, p->fN, (const C<T>*)p->d_twM, (const C<T>*)p->d_twN, (const C<T>*)p->d_phase,
        (const C<T>*)p->d_V, p->d_Gp, (C<T>*)p->d_Gt, p->d_spins);
  } else {
    const int sm = p->N * (int)sizeof(C<T>);
    if ((e = set_smem(k_theta_forward_adjoint<T, false>, sm)) != cudaSuccess) return e;
    k_theta_forward_adjoint<T, false><<<dim3(p->M, p->B), threads_inplace(p->N), sm, st>>>(
        dims_of(p), p->fM, p->fN, (const C<T>*)p->d_twM, (const C<T>*)p->d_twN, (const C<T>*)p->d_phase,
        (const C<T>*)p->d_V, p->d_Gp, (C<T>*)p->d_Gt, p->d_spins);
  }
  return cudaGetLastError();
}
template <typename T>
cudaError_t phi_forward_adjoint_t(const mw_plan* p, double2* map, cudaStream_t st) {
  const int sm = pp_bytes<T>(p->M);
  cudaError_t e = set_smem(k_phi_forward_adjoint<T>, sm);
  if (e != cudaSuccess) return e;
  k_phi_forward_adjoint<T><<<dim3(p->L, p->B), threads_pp(p->M), sm, st>>>(
      dims_of(p), p->fM, (const C<T>*)p->d_twM, (const C<T>*)p->d_Gt, map, p->d_moff, p->d_spins);
  return cudaGetLastError();
}
template <typename T>
cudaError_t phi_inverse_adjoint_t(const mw_plan* p, const double2* map, cudaStream_t st) {
  const int sm = pp_bytes<T>(p->M);
  cudaError_t e = set_smem(k_phi_inverse_adjoint<T>, sm);
  if (e != cudaSuccess) return e;
  k_phi_inverse_adjoint<T><<<dim3(p->L, p->B), threads_pp(p->M), sm, st>>>(
      dims_of(p), p->fM, (const C<T>*)p->d_twM, map, p->d_moff, (C<T>*)p->d_Gt);
  return cudaGetLastError();
}
template <typename T>
cudaError_t theta_inverse_adjoint_t(const mw_plan* p, cudaStream_t st) {
  const int sm = pp_bytes<T>(p->M);
  cudaError_t e = set_smem(k_theta_inverse_adjoint<T>, sm);
  if (e != cudaSuccess) return e;
  k_theta_inverse_adjoint<T><<<dim3(p->M, p->B), threads_pp(p->M), sm, st>>>(
      dims_of(p), p->fM, (const C<T>*)p->d_twM, (const C<T>*)p->d_phase, (const C<T>*)p->d_Gt, (C<T>*)p->d_Gp,
      p->d_spins);
  return cudaGetLastError();
}

}  // namespace

#define DISPATCH(p, fn, ...) ((p)->prec == MW_PREC_FP64 ? fn<double>(__VA_ARGS__) : fn<float>(__VA_ARGS__))

#define DISPATCH2(p, fn, R, ...) \
  ((p)->prec == MW_PREC_FP64 ? fn<double, R>(__VA_ARGS__) : fn<float, R>(__VA_ARGS__))

cudaError_t launch_phi_forward(const mw_plan* p, const double2* map, cudaStream_t st) {
  return DISPATCH2(p, phi_forward_t, false, p, map, st);
}
cudaError_t launch_phi_forward_real(const mw_plan* p, const double* maps, cudaStream_t st) {
  return DISPATCH2(p, phi_forward_t, true, p, maps, st);
}
cudaError_t launch_phi_inverse_real(const mw_plan* p, double* maps, cudaStream_t st) {
  return DISPATCH2(p, phi_inverse_t, true, p, maps, st);
}
cudaError_t launch_theta_forward(const mw_plan* p, cudaStream_t st) { return DISPATCH(p, theta_forward_t, p, st); }
cudaError_t launch_theta_inverse(const mw_plan* p, cudaStream_t st) { return DISPATCH(p, theta_inverse_t, p, st); }
cudaError_t launch_phi_inverse(const mw_plan* p, double2* map, cudaStream_t st) {
  return DISPATCH2(p, phi_inverse_t, false, p, map, st);
}
cudaError_t launch_theta_forward_adjoint(const mw_plan* p, cudaStream_t st) {
  return DISPATCH(p, theta_forward_adjoint_t, p, st);
}
cudaError_t launch_phi_forward_adjoint(const mw_plan* p, double2* map, cudaStream_t st) {
  return DISPATCH(p, phi_forward_adjoint_t, p, map, st);
}
cudaError_t launch_phi_inverse_adjoint(const mw_plan* p, const double2* map, cudaStream_t st) {
  return DISPATCH(p, phi_inverse_adjoint_t, p, map, st);
}
cudaError_t launch_theta_inverse_adjoint(const mw_plan* p, cudaStream_t st) {
  return DISPATCH(p, theta_inverse_adjoint_t, p, st);
}
cudaError_t launch_pole_forward_adjoint(const mw_plan* p, double2* map, cudaStream_t st) {
  k_pole_forward_adjoint<<<p->B, 256, 0, st>>>(dims_of(p), p->d_Gp, p->d_upole, map, p->d_moff, p->d_spins,
                                                p->prec != MW_PREC_FP64 ? 1 : 0);
  return cudaGetLastError();
}
