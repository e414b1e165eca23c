// kernels_fft_adj.cu -- adjoints of the O(L^2 log L) stages of the MW
// transforms (no counterpart in the paper): each stage of kernels_fft.cu
// transposed and conjugated, run in reverse order, in the stage precision T
// (double for the FP64 path, float for the mixed path), map and f_lm buffers
// complex double.  The adjoint of the forward theta stage (weight convolution
// and theta DFT) is in kernels_fft_adj_theta.cu.
#include "fft_stage.cuh"

namespace {

// --------------------------------------------------------------------------
// adjoint of the forward: Wigner^H (run_wigner mode 1) -> theta_forward^H -> phi_forward^H
// --------------------------------------------------------------------------
template <typename T, bool BS>
__global__ void __launch_bounds__(kFftMaxThreads) k_phi_forward_adjoint(Dims d, FftM<T> fm, const C<T>* __restrict__ Gt,
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
  const C<T>* res = fft_m<T, BS, kFftVPT>(buf, buf + M, fm, true);
  const T sc = (T)(2.0 * M_PI / M);
  for (int p = threadIdx.x; p < M; p += blockDim.x) f[(long long)t * M + p] = to64(cscale<T>(res[p], sc));
}

// --------------------------------------------------------------------------
// adjoint of the inverse: phi_inverse^H -> theta_inverse^H -> Wigner^H (run_wigner mode 0)
// --------------------------------------------------------------------------
template <typename T, bool BS>
__global__ void __launch_bounds__(kFftMaxThreads) k_phi_inverse_adjoint(Dims d, FftM<T> fm,
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
  const C<T>* res = fft_m<T, BS, kFftVPT>(buf, buf + M, fm, false);
  for (int i = threadIdx.x; i < M; i += blockDim.x) {
    const int m = i - (L - 1);
    out[(long long)i * L + t] = res[m < 0 ? m + M : m];
  }
}

template <typename T, bool BS>
__global__ void __launch_bounds__(kFftMaxThreads) k_theta_inverse_adjoint(Dims d, FftM<T> fm,
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
  const C<T>* res = fft_m<T, BS, kFftVPT>(buf, buf + M, fm, false);
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

template <typename T, bool BS>
cudaError_t phi_forward_adjoint_b(const mw_plan* p, double2* map, cudaStream_t st) {
  const int sm = m_elems(p) * (int)sizeof(C<T>);
  cudaError_t e = set_smem(k_phi_forward_adjoint<T, BS>, sm);
  if (e != cudaSuccess) return e;
  k_phi_forward_adjoint<T, BS><<<dim3(p->L, p->B), m_threads(p, kFftVPT), sm, st>>>(
      dims_of(p), fft_m_of<T>(p), (const C<T>*)p->d_Gt, map, p->d_moff, p->d_spins);
  return cudaGetLastError();
}
template <typename T>
cudaError_t phi_forward_adjoint_t(const mw_plan* p, double2* map, cudaStream_t st) {
  return p->bluestein ? phi_forward_adjoint_b<T, true>(p, map, st) : phi_forward_adjoint_b<T, false>(p, map, st);
}
template <typename T, bool BS>
cudaError_t phi_inverse_adjoint_b(const mw_plan* p, const double2* map, cudaStream_t st) {
  const int sm = m_elems(p) * (int)sizeof(C<T>);
  cudaError_t e = set_smem(k_phi_inverse_adjoint<T, BS>, sm);
  if (e != cudaSuccess) return e;
  k_phi_inverse_adjoint<T, BS><<<dim3(p->L, p->B), m_threads(p, kFftVPT), sm, st>>>(
      dims_of(p), fft_m_of<T>(p), map, p->d_moff, (C<T>*)p->d_Gt);
  return cudaGetLastError();
}
template <typename T>
cudaError_t phi_inverse_adjoint_t(const mw_plan* p, const double2* map, cudaStream_t st) {
  return p->bluestein ? phi_inverse_adjoint_b<T, true>(p, map, st) : phi_inverse_adjoint_b<T, false>(p, map, st);
}
template <typename T, bool BS>
cudaError_t theta_inverse_adjoint_b(const mw_plan* p, cudaStream_t st) {
  const int sm = m_elems(p) * (int)sizeof(C<T>);
  cudaError_t e = set_smem(k_theta_inverse_adjoint<T, BS>, sm);
  if (e != cudaSuccess) return e;
  k_theta_inverse_adjoint<T, BS><<<dim3(p->M, p->B), m_threads(p, kFftVPT), sm, st>>>(
      dims_of(p), fft_m_of<T>(p), (const C<T>*)p->d_phase, (const C<T>*)p->d_Gt, (C<T>*)p->d_Gp, p->d_spins);
  return cudaGetLastError();
}
template <typename T>
cudaError_t theta_inverse_adjoint_t(const mw_plan* p, cudaStream_t st) {
  return p->bluestein ? theta_inverse_adjoint_b<T, true>(p, st) : theta_inverse_adjoint_b<T, false>(p, st);
}

}  // namespace

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
