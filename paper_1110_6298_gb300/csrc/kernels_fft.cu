// kernels_fft.cu -- the O(L^2 log L) stages of the MW transforms (their adjoints
// are in kernels_fft_adj.cu).
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
// T is the arithmetic type of these stages (double for the FP64 path, float for
// the mixed path).  Map and f_lm buffers are always complex double.  The
// length-(2L-1) DFTs run by mixed radix or, where the plan chose it, by
// Bluestein's convolution (template flag BS).
#include "fft_stage.cuh"

namespace {

// --------------------------------------------------------------------------
// forward
// --------------------------------------------------------------------------
template <typename T, bool RealIo, bool BS>
__device__ __forceinline__ void phi_forward_body(Dims d, FftM<T> fm, const void* __restrict__ map,
                              const long long* __restrict__ moff,
                              C<T>* __restrict__ Gt /* [B][M][L] */, const int* __restrict__ spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int t = blockIdx.x, b = d.b0 + blockIdx.y;
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
  const C<T>* res = fft_m<T, BS>(buf, buf + M, fm, false);
  const T sc = (T)(2.0 * M_PI / M);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const int m = i - (L - 1);
    const int k = m < 0 ? m + M : m;
    out[(long long)i * L + t] = cscale<T>(res[k], sc);
  }
}

template <typename T, bool RealIo>
__global__ void __launch_bounds__(kFftMaxThreads) k_phi_forward(Dims d, FftM<T> fm, const void* __restrict__ map,
                              const long long* __restrict__ moff,
                              C<T>* __restrict__ Gt /* [B][M][L] */, const int* __restrict__ spins) {
  phi_forward_body<T, RealIo, false>(d, fm, map, moff, Gt, spins);
}
// Bluestein variant: 1024-thread blocks, 8 values per thread in the in-place
// power-of-two FFTs (64 registers)
template <typename T, bool RealIo>
__global__ void __launch_bounds__(kBsMaxThreads, 1) k_phi_forward_bs(Dims d, FftM<T> fm, const void* __restrict__ map,
                              const long long* __restrict__ moff,
                              C<T>* __restrict__ Gt /* [B][M][L] */, const int* __restrict__ spins) {
  phi_forward_body<T, RealIo, true>(d, fm, map, moff, Gt, spins);
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
// with the kernel's DFT, FFT_NE (ping-pong FFTs; max(2M, 4 NE) complex values of
// shared memory, against 2 N with N >= 4L-3 for the direct convolution; at
// least N with a Bluestein FFT_M).
constexpr int kEvenVPT = 8;  // values of F a thread carries through the split (512 threads up to M = 4095)

template <typename T, bool BS>
__device__ __forceinline__ void theta_forward_even_body(
    Dims d, FftM<T> fm, FftDesc fE, const C<T>* __restrict__ twE,
    const C<T>* __restrict__ phase, const C<T>* __restrict__ Ue, const C<T>* __restrict__ Uo,
    const C<T>* __restrict__ Gt, C<T>* __restrict__ Gp, const int* __restrict__ spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int L = d.L, M = d.M, NE = fE.n;
  C<T>* X = buf;           // even half (ping-pong pair X, X + NE)
  C<T>* Y = buf + 2 * NE;  // odd half (Y, Y + NE)
  const int im = blockIdx.x, b = d.b0 + blockIdx.y;
  const int m = im - (L - 1);
  const int s = spin_of(spins, b);
  const T sg = (T)parity_sign(m + s);
  const C<T>* g = Gt + ((long long)b * M + im) * L;
  // periodic extension over the 2L-1 nodes, FFT_M
  for (int t = threadIdx.x; t < M; t += blockDim.x) buf[t] = (t < L) ? g[t] : cscale<T>(g[2 * L - 2 - t], sg);
  __syncthreads();
  const C<T>* F = fft_m<T, BS>(buf, buf + M, fm, false);
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
  // both halves in one pass per FFT stage (Y = X + 2 NE)
  C<T>* xe = fft_pp2<T>(X, X + NE, 2 * NE, fE, twE, true);
  C<T>* xo = xe + 2 * NE;
  for (int k = threadIdx.x; k < NE; k += blockDim.x) {
    xe[k] = cmul<T>(xe[k], Ue[k]);
    xo[k] = cmul<T>(xo[k], Uo[k]);
  }
  __syncthreads();
  xe = fft_pp2<T>(xe, xe == X ? X + NE : X, 2 * NE, fE, twE, false);
  xo = xe + 2 * NE;
  // G+_{m,0} = G_m0, G+_{m,m'} = 2 G_mm' (m' > 0): m' = 2i from the even half, 2i+1 from the odd
  C<T>* out = Gp + ((long long)b * M + im) * L;
  for (int mp = threadIdx.x; mp < L; mp += blockDim.x) {
    const C<T> a = (mp & 1) ? xo[mp >> 1] : xe[mp >> 1];
    out[mp] = mp == 0 ? a : cscale<T>(a, (T)2);
  }
}

template <typename T>
__global__ void __launch_bounds__(kFftMaxThreads) k_theta_forward_even(
    Dims d, FftM<T> fm, FftDesc fE, const C<T>* __restrict__ twE,
    const C<T>* __restrict__ phase, const C<T>* __restrict__ Ue, const C<T>* __restrict__ Uo,
    const C<T>* __restrict__ Gt, C<T>* __restrict__ Gp, const int* __restrict__ spins) {
  theta_forward_even_body<T, false>(d, fm, fE, twE, phase, Ue, Uo, Gt, Gp, spins);
}
// Bluestein variant: 1024-thread blocks, 8 values per thread in the in-place
// power-of-two FFTs (64 registers)
template <typename T>
__global__ void __launch_bounds__(kBsMaxThreads, 1) k_theta_forward_even_bs(
    Dims d, FftM<T> fm, FftDesc fE, const C<T>* __restrict__ twE,
    const C<T>* __restrict__ phase, const C<T>* __restrict__ Ue, const C<T>* __restrict__ Uo,
    const C<T>* __restrict__ Gt, C<T>* __restrict__ Gp, const int* __restrict__ spins) {
  theta_forward_even_body<T, true>(d, fm, fE, twE, phase, Ue, Uo, Gt, Gp, spins);
}

// --------------------------------------------------------------------------
// inverse
// --------------------------------------------------------------------------
template <typename T, bool BS>
__device__ __forceinline__ void theta_inverse_body(Dims d, FftM<T> fm, const C<T>* __restrict__ phase,
                                const double2* __restrict__ Gp, C<T>* __restrict__ Gt /* [B][L][M] */,
                                const int* __restrict__ spins) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int L = d.L, M = d.M;
  const int im = blockIdx.x, b = d.b0 + blockIdx.y;
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
  const C<T>* res = fft_m<T, BS>(buf, buf + M, fm, true);
  C<T>* out = Gt + (long long)b * L * M;
  for (int t = threadIdx.x; t < L; t += blockDim.x) out[(long long)t * M + im] = res[t];
}

template <typename T>
__global__ void __launch_bounds__(kFftMaxThreads) k_theta_inverse(Dims d, FftM<T> fm, const C<T>* __restrict__ phase,
                                const double2* __restrict__ Gp, C<T>* __restrict__ Gt /* [B][L][M] */,
                                const int* __restrict__ spins) {
  theta_inverse_body<T, false>(d, fm, phase, Gp, Gt, spins);
}
// Bluestein variant: 1024-thread blocks, 8 values per thread in the in-place
// power-of-two FFTs (64 registers)
template <typename T>
__global__ void __launch_bounds__(kBsMaxThreads, 1) k_theta_inverse_bs(Dims d, FftM<T> fm, const C<T>* __restrict__ phase,
                                const double2* __restrict__ Gp, C<T>* __restrict__ Gt /* [B][L][M] */,
                                const int* __restrict__ spins) {
  theta_inverse_body<T, true>(d, fm, phase, Gp, Gt, spins);
}

template <typename T, bool RealIo, bool BS>
__device__ __forceinline__ void phi_inverse_body(Dims d, FftM<T> fm, const C<T>* __restrict__ Gt,
                              void* __restrict__ map, const long long* __restrict__ moff) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C<T>* buf = reinterpret_cast<C<T>*>(smem_raw);
  const int L = d.L, M = d.M;
  const int t = blockIdx.x, b = d.b0 + blockIdx.y;
  const C<T>* in = Gt + ((long long)b * L + t) * M;
  for (int k = threadIdx.x; k < M; k += blockDim.x) {
    const int m = (k <= L - 1) ? k : k - M;
    buf[k] = in[m + L - 1];
  }
  __syncthreads();
  const C<T>* res = fft_m<T, BS>(buf, buf + M, fm, true);
  if (t < L - 1) {
    for (int p = threadIdx.x; p < M; p += blockDim.x) store_sample<T, RealIo>(map, moff, d, b, (long long)t * M + p, res[p]);
  } else if (threadIdx.x == 0) {
    store_sample<T, RealIo>(map, moff, d, b, (long long)(L - 1) * M, res[0]);
  }
}

template <typename T, bool RealIo>
__global__ void __launch_bounds__(kFftMaxThreads) k_phi_inverse(Dims d, FftM<T> fm, const C<T>* __restrict__ Gt,
                              void* __restrict__ map, const long long* __restrict__ moff) {
  phi_inverse_body<T, RealIo, false>(d, fm, Gt, map, moff);
}
// Bluestein variant: 1024-thread blocks, 8 values per thread in the in-place
// power-of-two FFTs (64 registers)
template <typename T, bool RealIo>
__global__ void __launch_bounds__(kBsMaxThreads, 1) k_phi_inverse_bs(Dims d, FftM<T> fm, const C<T>* __restrict__ Gt,
                              void* __restrict__ map, const long long* __restrict__ moff) {
  phi_inverse_body<T, RealIo, true>(d, fm, Gt, map, moff);
}

template <typename T, bool RealIo, bool BS>
cudaError_t phi_forward_b(const mw_plan* p, const void* map, cudaStream_t st, int b0, int nb) {
  const int sm = m_elems(p) * (int)sizeof(C<T>);
  auto kern = BS ? k_phi_forward_bs<T, RealIo> : k_phi_forward<T, RealIo>;
  cudaError_t e = set_smem(kern, sm);
  if (e != cudaSuccess) return e;
  Dims d = dims_of(p);
  d.b0 = b0;
  kern<<<dim3(p->L, nb), m_threads(p), sm, st>>>(d, fft_m_of<T>(p), map, p->d_moff, (C<T>*)p->d_Gt, p->d_spins);
  return cudaGetLastError();
}
template <typename T, bool RealIo>
cudaError_t phi_forward_t(const mw_plan* p, const void* map, cudaStream_t st, int b0, int nb) {
  return p->bluestein ? phi_forward_b<T, RealIo, true>(p, map, st, b0, nb)
                      : phi_forward_b<T, RealIo, false>(p, map, st, b0, nb);
}
template <typename T, bool BS>
cudaError_t theta_forward_b(const mw_plan* p, cudaStream_t st, int b0, int nb) {
  int n = 2 * p->M > 4 * p->NE ? 2 * p->M : 4 * p->NE;
  if (BS && p->fB.n > n) n = p->fB.n;
  const int sm = n * (int)sizeof(C<T>);
  auto kern = BS ? k_theta_forward_even_bs<T> : k_theta_forward_even<T>;
  cudaError_t e = set_smem(kern, sm);
  if (e != cudaSuccess) return e;
  int nt = ((p->M + kEvenVPT - 1) / kEvenVPT + 31) / 32 * 32;  // every thread carries <= kEvenVPT values of F
  const int pp = threads_pp(p->NE > p->M ? p->NE : p->M);
  if (nt < pp) nt = pp;
  const int nbs = BS ? ((p->fB.n + kBsVPT - 1) / kBsVPT + 31) / 32 * 32 : 0;  // Bluestein: kBsVPT values each
  if (nt < nbs) nt = nbs;
  Dims d = dims_of(p);
  d.b0 = b0;
  kern<<<dim3(p->M, nb), nt, sm, st>>>(
      d, fft_m_of<T>(p), p->fE, (const C<T>*)p->d_twE, (const C<T>*)p->d_phase,
      (const C<T>*)p->d_Ue, (const C<T>*)p->d_Uo, (const C<T>*)p->d_Gt, (C<T>*)p->d_Gp, p->d_spins);
  return cudaGetLastError();
}
template <typename T>
cudaError_t theta_forward_t(const mw_plan* p, cudaStream_t st, int b0, int nb) {
  return p->bluestein ? theta_forward_b<T, true>(p, st, b0, nb) : theta_forward_b<T, false>(p, st, b0, nb);
}
template <typename T, bool BS>
cudaError_t theta_inverse_b(const mw_plan* p, cudaStream_t st, int b0, int nb) {
  const int sm = m_elems(p) * (int)sizeof(C<T>);
  auto kern = BS ? k_theta_inverse_bs<T> : k_theta_inverse<T>;
  cudaError_t e = set_smem(kern, sm);
  if (e != cudaSuccess) return e;
  Dims d = dims_of(p);
  d.b0 = b0;
  kern<<<dim3(p->M, nb), m_threads(p), sm, st>>>(
      d, fft_m_of<T>(p), (const C<T>*)p->d_phase, p->d_Gp, (C<T>*)p->d_Gt, p->d_spins);
  return cudaGetLastError();
}
template <typename T>
cudaError_t theta_inverse_t(const mw_plan* p, cudaStream_t st, int b0, int nb) {
  return p->bluestein ? theta_inverse_b<T, true>(p, st, b0, nb) : theta_inverse_b<T, false>(p, st, b0, nb);
}
template <typename T, bool RealIo, bool BS>
cudaError_t phi_inverse_b(const mw_plan* p, void* map, cudaStream_t st, int b0, int nb) {
  const int sm = m_elems(p) * (int)sizeof(C<T>);
  auto kern = BS ? k_phi_inverse_bs<T, RealIo> : k_phi_inverse<T, RealIo>;
  cudaError_t e = set_smem(kern, sm);
  if (e != cudaSuccess) return e;
  Dims d = dims_of(p);
  d.b0 = b0;
  kern<<<dim3(p->L, nb), m_threads(p), sm, st>>>(d, fft_m_of<T>(p), (const C<T>*)p->d_Gt, map, p->d_moff);
  return cudaGetLastError();
}
template <typename T, bool RealIo>
cudaError_t phi_inverse_t(const mw_plan* p, void* map, cudaStream_t st, int b0, int nb) {
  return p->bluestein ? phi_inverse_b<T, RealIo, true>(p, map, st, b0, nb)
                      : phi_inverse_b<T, RealIo, false>(p, map, st, b0, nb);
}

}  // namespace

// b0, nb: the maps [b0, b0 + nb) of the plan (nb < 0: every map)
cudaError_t launch_phi_forward(const mw_plan* p, const double2* map, cudaStream_t st, int b0, int nb) {
  return DISPATCH2(p, phi_forward_t, false, p, map, st, b0, nb < 0 ? p->B : nb);
}
cudaError_t launch_phi_forward_real(const mw_plan* p, const double* maps, cudaStream_t st) {
  return DISPATCH2(p, phi_forward_t, true, p, maps, st, 0, p->B);
}
cudaError_t launch_phi_inverse_real(const mw_plan* p, double* maps, cudaStream_t st) {
  return DISPATCH2(p, phi_inverse_t, true, p, maps, st, 0, p->B);
}
cudaError_t launch_theta_forward(const mw_plan* p, cudaStream_t st, int b0, int nb) {
  return DISPATCH(p, theta_forward_t, p, st, b0, nb < 0 ? p->B : nb);
}
cudaError_t launch_theta_inverse(const mw_plan* p, cudaStream_t st, int b0, int nb) {
  return DISPATCH(p, theta_inverse_t, p, st, b0, nb < 0 ? p->B : nb);
}
cudaError_t launch_phi_inverse(const mw_plan* p, double2* map, cudaStream_t st, int b0, int nb) {
  return DISPATCH2(p, phi_inverse_t, false, p, map, st, b0, nb < 0 ? p->B : nb);
}
