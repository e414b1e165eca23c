// kernels_quad.cu -- the MW quadrature rule (Sec. IV-F, Eq. quadrature).
//
//   I = sum_{t=0}^{L-1} sum_{p=0}^{L-1} f(theta_t, phi'_p) q(theta_t),   phi'_p = 2 pi p / L,
//   q(theta_t) = (2 pi / L) [ v(theta_t) + (1 - delta_{t,L-1}) (-1)^s v(theta_{2L-2-t}) ],
//   v(theta)   = 1/(2L-1) sum_{|m'| <= L-1} w(-m') e^{i m' theta}.
// With the weights w of Sec. IV-D (2/(1-k^2) for even k, +-i pi/2 at k = +-1,
// 0 for other odd k) the sum is real:
//   v(theta) = [ 2 + sum_{even m' = 2..L-1} 4/(1-m'^2) cos(m' theta) + pi sin(theta) [L >= 2] ] / (2L-1).
// Maps use the quadrature layout: rings t = 0..L-2 of L samples at phi'_p, then
// one pole sample f(pi, 0); the pole ring of a spin-s signal is
// f(pi, 0) e^{i s phi}, whose L samples sum to L f(pi, 0) for s = 0 and to 0
// for 0 < |s| < L.
#include <cmath>

#include "internal.h"

namespace {

constexpr int kQThreads = 256;

// fixed-order block reduction of a double (all threads get the result)
__device__ double block_sum(double v, double* red) {
  red[threadIdx.x] = v;
  __syncthreads();
  for (int h = blockDim.x / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  const double r = red[0];
  __syncthreads();
  return r;
}

// v(theta_u) for the extended node u (0 <= u <= 2L-2), theta_u = pi (2u+1) / M
__device__ double v_node(int L, int u, double* red) {
  const int M = 2 * L - 1;
  double acc = 0.0;
  // even m' = 2, 4, ..., L-1: cos(m' theta_u) = cos(pi k / M), k = m' (2u+1) mod 2M
  for (int h = 1 + (int)threadIdx.x; 2 * h <= L - 1; h += blockDim.x) {
    const int mp = 2 * h;
    const long long k = ((long long)mp * (2 * u + 1)) % (2 * M);
    acc += 4.0 / (1.0 - (double)mp * (double)mp) * cospi((double)k / (double)M);
  }
  const double s = block_sum(acc, red);
  const double odd = (L >= 2) ? 3.14159265358979323846 * sinpi((double)(2 * u + 1) / (double)M) : 0.0;
  return (2.0 + s + odd) / (double)M;
}

// q(theta_t) for t = blockIdx.x
__global__ void __launch_bounds__(kQThreads) k_quad_weights(int L, int s, double* __restrict__ q) {
  __shared__ double red[kQThreads];
  const int t = blockIdx.x;
  const double v1 = v_node(L, t, red);
  const double v2 = (t == L - 1) ? 0.0 : v_node(L, 2 * L - 2 - t, red);
  if (threadIdx.x == 0) {
    const double sg = (s & 1) ? -1.0 : 1.0;
    q[t] = 2.0 * 3.14159265358979323846 / (double)L * (v1 + sg * v2);
  }
}

// Partial sums over the rings [c R, (c+1) R) of map b: sum_t q_t sum_p f[t][p].
__global__ void __launch_bounds__(kQThreads) k_quad_partial(int L, int rings_per_chunk, const double2* __restrict__ maps,
                                                            const double* __restrict__ qw, int nq,
                                                            const int* __restrict__ spins, double2* __restrict__ part) {
  __shared__ double red[kQThreads];
  const int c = blockIdx.x, b = blockIdx.y, nc = gridDim.x;
  const long long n = (long long)L * (L - 1) + 1;
  const double2* f = maps + (long long)b * n;
  const double* q = qw + (size_t)((spins[b] & 1) ? 1 : 0) * nq;  // weights of even / odd spin
  const int t0 = c * rings_per_chunk, t1 = min(L - 1, t0 + rings_per_chunk);
  double re = 0.0, im = 0.0;
  for (int t = t0; t < t1; ++t) {
    double rr = 0.0, ri = 0.0;
    for (int p = threadIdx.x; p < L; p += blockDim.x) {
      const double2 v = f[(long long)t * L + p];
      rr += v.x;
      ri += v.y;
    }
    re += q[t] * rr;
    im += q[t] * ri;
  }
  re = block_sum(re, red);
  im = block_sum(im, red);
  if (threadIdx.x == 0) part[(size_t)b * nc + c] = make_double2(re, im);
}

// I_b = the chunk partials in order, plus the pole ring
__global__ void k_quad_final(int L, int nc, const double2* __restrict__ part, const double2* __restrict__ maps,
                             const double* __restrict__ qw, int nq, const int* __restrict__ spins,
                             double2* __restrict__ out) {
  const int b = blockIdx.x;
  if (threadIdx.x != 0) return;
  const long long n = (long long)L * (L - 1) + 1;
  double re = 0.0, im = 0.0;
  for (int c = 0; c < nc; ++c) {
    re += part[(size_t)b * nc + c].x;
    im += part[(size_t)b * nc + c].y;
  }
  if (spins[b] == 0) {
    const double* q = qw;
    const double2 fp = maps[(long long)b * n + n - 1];
    re += q[L - 1] * (double)L * fp.x;
    im += q[L - 1] * (double)L * fp.y;
  }
  out[b] = make_double2(re, im);
}

}  // namespace

// ring chunks per map: about four blocks per SM over the batch, at most one per ring
int quad_chunks(const mw_plan* p) {
  const int rings = p->L - 1 > 0 ? p->L - 1 : 1;
  int want = (p->risbo_grid + p->B - 1) / p->B;
  if (want < 1) want = 1;
  if (want > rings) want = rings;
  const int rpc = (rings + want - 1) / want;
  return (rings + rpc - 1) / rpc;
}

cudaError_t launch_quad_weights(int L, int s, double* q, cudaStream_t st) {
  k_quad_weights<<<L, kQThreads, 0, st>>>(L, s, q);
  return cudaGetLastError();
}

// Two stages: ring chunks (about 4 blocks per SM over the batch), then one
// thread per map sums its chunks in order.
cudaError_t launch_quadrature(const mw_plan* p, const double2* maps, double2* out, cudaStream_t st, int* launches) {
  const int L = p->L, B = p->B;
  const int nc = quad_chunks(p);
  const int rings = L - 1 > 0 ? L - 1 : 1;
  const int rpc = (rings + nc - 1) / nc;
  k_quad_partial<<<dim3(nc, B), kQThreads, 0, st>>>(L, rpc, maps, p->d_qw, L, p->d_spins, p->d_qpart);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_quad_final<<<B, 1, 0, st>>>(L, nc, p->d_qpart, maps, p->d_qw, L, p->d_spins, out);
  if (launches) *launches += 2;
  return cudaGetLastError();
}
