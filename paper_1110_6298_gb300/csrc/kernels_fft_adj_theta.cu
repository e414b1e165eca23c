// kernels_fft_adj_theta.cu -- adjoint of the forward theta stage (no
// counterpart in the paper): the +-m' fold, the weight convolution of
// Eq. (Gmm_convolution) and the theta DFT over the 2L-1 extended nodes,
// transposed and conjugated, then the periodic extension's adjoint; one block
// per (m, map), in the stage precision T.
#include "fft_stage.cuh"

namespace {

template <typename T, bool PP, bool BS>
__global__ void __launch_bounds__(kFftMaxThreads) k_theta_forward_adjoint(Dims d, FftM<T> fm, FftDesc fN,
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
    res = fft_m<T, BS, kFftVPT>(x, z, fm, true);  // the launch leaves NB values of room from x
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
    if constexpr (BS) fft_bluestein<T, kFftVPT>(buf, M, fm.dB, fm.twB, fm.chirp, fm.chirpF, true);
    else fft_inplace<T, kFftVPT>(buf, fm.d, fm.tw, true);
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

template <typename T, bool BS>
cudaError_t theta_forward_adjoint_b(const mw_plan* p, cudaStream_t st) {
  // the length-M DFT runs in the half x (at buf or buf + N) of the ping-pong
  // pair, or in buf: a Bluestein one needs NB values from there
  const int NB = BS ? p->fB.n : 0;
  const int n_pp = 2 * p->N > p->N + NB ? 2 * p->N : p->N + NB;
  const int n_ip = p->N > NB ? p->N : NB;
  cudaError_t e;
  // single precision always fits the ping-pong pair (N, NB <= 8192: 128 KB), so
  // only double instantiates the in-place variant
  if (sizeof(T) == 4 || n_pp * (int)sizeof(C<T>) <= kSmemMax) {
    const int sm = n_pp * (int)sizeof(C<T>);
    if ((e = set_smem(k_theta_forward_adjoint<T, true, BS>, sm)) != cudaSuccess) return e;
    k_theta_forward_adjoint<T, true, BS><<<dim3(p->M, p->B), threads_pp(p->N), sm, st>>>(
        dims_of(p), fft_m_of<T>(p), p->fN, (const C<T>*)p->d_twN, (const C<T>*)p->d_phase, (const C<T>*)p->d_V,
        p->d_Gp, (C<T>*)p->d_Gt, p->d_spins);
  } else if constexpr (sizeof(T) == 8) {
    const int sm = n_ip * (int)sizeof(C<T>);
    if ((e = set_smem(k_theta_forward_adjoint<T, false, BS>, sm)) != cudaSuccess) return e;
    k_theta_forward_adjoint<T, false, BS><<<dim3(p->M, p->B), threads_inplace(p->N), sm, st>>>(
        dims_of(p), fft_m_of<T>(p), p->fN, (const C<T>*)p->d_twN, (const C<T>*)p->d_phase, (const C<T>*)p->d_V,
        p->d_Gp, (C<T>*)p->d_Gt, p->d_spins);
  }
  return cudaGetLastError();
}
template <typename T>
cudaError_t theta_forward_adjoint_t(const mw_plan* p, cudaStream_t st) {
  return p->bluestein ? theta_forward_adjoint_b<T, true>(p, st) : theta_forward_adjoint_b<T, false>(p, st);
}

}  // namespace

cudaError_t launch_theta_forward_adjoint(const mw_plan* p, cudaStream_t st) {
  return DISPATCH(p, theta_forward_adjoint_t, p, st);
}
