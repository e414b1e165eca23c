// kernels_dmma.cu -- the FP64 path's Delta contractions on the FP64 tensor
// instruction (mma.sync m8n8k4 .f64; tcgen05 has no FP64 kind).  On this part
// it issues to the same FP64 pipe as DFMA and runs at the same 1.05 TFLOP/s
// (measured), so its gain over FMA code is the operand reuse of the MMA tile:
// the kernels run with the FP64 pipe about 95% busy.
//
// Same GEMM structure as the split-precision kernels: for one chunk of planes
// and one |m| = am, the forward sum of Eq. (flm_wig) is
//   out[l, n] = sum_{m'} A[l, m'] B[n, m'],  A[l, m'] = Delta^l_{m',am} Delta^l_{m',-s},
// with n over (map, re/im) for m = +am and, multiplied by (-1)^{m'} in B and
// (-1)^l in the result, for m = -am (Delta_{m',-am} = (-1)^(l+m') Delta_{m',am}).
// The inverse sum of Eq. (Fmm) is the transposed GEMM with rows m' and K = l,
// accumulated over chunks in the FP64 buffer F+.  All arithmetic is FP64.
//
// Fragments of mma.m8n8k4.row.col.f64 (lane = 4 g + q): A holds A[g][q],
// B holds B[k = q][n = g], the accumulator holds D[g][2q], D[g][2q+1].
#include <cmath>

#include "internal.h"

namespace {

constexpr int kThreads = 256;  // 8 warps
constexpr int kRows = 64;      // tile rows (l for the forward, m' for the inverse)
constexpr int kN = 32;         // columns: 4 x 8 maps
constexpr int kKt = 32;        // K per shared-memory stage
constexpr int kAs = kKt + 2;   // padded row strides (doubles)

__device__ __forceinline__ void dmma(double& d0, double& d1, double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};"
               : "+d"(d0), "+d"(d1)
               : "d"(a), "d"(b));
}

__device__ __forceinline__ double kval(const double* __restrict__ P, int LD, int am, int as, int s, int l, int mp) {
  const double v = P[(size_t)am * LD + mp] * P[(size_t)as * LD + mp];
  return ((am + as + (s > 0 ? l + mp : 0)) & 1) ? -v : v;
}

// forward: one block per (am, spin group); rows l of the chunk
__global__ void __launch_bounds__(kThreads) k_dmma_forward(const double* __restrict__ S, int LD, int L, int M, int l0,
                                                           int l1, const SpinGroup* __restrict__ groups,
                                                           const double2* __restrict__ Gp,
                                                           const double* __restrict__ nltab,
                                                           double2* __restrict__ flm,
                                                           const long long* __restrict__ foff) {
  __shared__ double As[kRows][kAs];
  __shared__ double Bs[kN][kAs];
  const int am = blockIdx.x;
  const SpinGroup& g = groups[blockIdx.y];
  const int s = g.s, as = s < 0 ? -s : s, nb = g.nb;
  const int lstart = max(max(l0, am), as);
  if (lstart >= l1) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, q = lane & 3;
  const size_t plane = (size_t)LD * LD;
  double acc[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int mp0 = 0; mp0 < l1; mp0 += kKt) {
    for (int idx = tid; idx < kRows * kKt; idx += kThreads) {
      const int r = idx / kKt, k = idx % kKt;
      const int l = l0 + r, mp = mp0 + k;
      As[r][k] = (l >= lstart && l < l1 && mp <= l) ? kval(S + (size_t)(l % kChunk) * plane, LD, am, as, s, l, mp) : 0.0;
    }
    for (int idx = tid; idx < kN * kKt; idx += kThreads) {
      const int n = idx / kKt, k = idx % kKt;
      const int j = n >> 1, mp = mp0 + k;
      double x = 0.0;
      if (j < 2 * nb && mp < L) {
        const bool neg = j >= nb;
        if (!(neg && am == 0)) {
          const double2 v = Gp[((size_t)g.maps[neg ? j - nb : j] * M + (neg ? -am : am) + L - 1) * L + mp];
          x = (n & 1) ? v.y : v.x;
          if (neg && (mp & 1)) x = -x;
        }
      }
      Bs[n][k] = x;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kKt / 4; ++ks) {
      const double a = As[8 * warp + gq][4 * ks + q];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) dmma(acc[nt][0], acc[nt][1], a, Bs[8 * nt + gq][4 * ks + q]);
    }
    __syncthreads();
  }
  // epilogue: the thread holds map columns (re, im) of map j = 4 nt + q for row l
  const int l = l0 + 8 * warp + gq;
  if (l >= am && l >= l0 && l < l1) {
    const double nl = ((s & 1) ? -1.0 : 1.0) * nltab[l];
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int j = 4 * nt + q;
      if (j >= 2 * nb) continue;
      const bool neg = j >= nb;
      if (neg && am == 0) continue;
      const int m = neg ? -am : am;
      double2 o = make_double2(0.0, 0.0);
      if (l >= as) {
        const double sgn = (neg && (l & 1)) ? -nl : nl;
        const double ar = acc[nt][0] * sgn, ai = acc[nt][1] * sgn;
        switch ((m + s) & 3) {  // times i^(m+s)
          case 0: o = make_double2(ar, ai); break;
          case 1: o = make_double2(-ai, ar); break;
          case 2: o = make_double2(-ar, -ai); break;
          default: o = make_double2(ai, -ar); break;
        }
      }
      flm[foff[g.maps[neg ? j - nb : j]] + (size_t)l * l + l + m] = o;
    }
  }
}

// inverse: one block per (am, 64-row tile of m', spin group); F+ += chunk sum
__global__ void __launch_bounds__(kThreads) k_dmma_inverse(const double* __restrict__ S, int LD, int L, int M, int l0,
                                                           int l1, const SpinGroup* __restrict__ groups,
                                                           const double2* __restrict__ flm,
                                                           const long long* __restrict__ foff,
                                                           const double* __restrict__ nltab,
                                                           double2* __restrict__ Fp) {
  __shared__ double At[kKt][kRows + 1];  // [l][m'] as read from the planes; used transposed
  __shared__ double Bs[kN][kAs];
  const int am = blockIdx.x, mp0 = blockIdx.y * kRows;
  const SpinGroup& g = groups[blockIdx.z];
  const int s = g.s, as = s < 0 ? -s : s, nb = g.nb;
  const int lstart = max(max(l0, am), as);
  if (lstart >= l1 || mp0 >= l1) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31, gq = lane >> 2, q = lane & 3;
  const size_t plane = (size_t)LD * LD;
  double acc[4][2] = {{0, 0}, {0, 0}, {0, 0}, {0, 0}};
  for (int lb = l0; lb < l1; lb += kKt) {
    for (int idx = tid; idx < kKt * kRows; idx += kThreads) {
      const int k = idx / kRows, r = idx % kRows;
      const int l = lb + k, mp = mp0 + r;
      At[k][r] = (l >= lstart && l < l1 && mp <= l && mp < L)
                     ? kval(S + (size_t)(l % kChunk) * plane, LD, am, as, s, l, mp)
                     : 0.0;
    }
    for (int idx = tid; idx < kN * kKt; idx += kThreads) {
      const int n = idx / kKt, k = idx % kKt;
      const int j = n >> 1, l = lb + k;
      double x = 0.0;
      if (j < 2 * nb && l >= lstart && l < l1) {
        const bool neg = j >= nb;
        if (!(neg && am == 0)) {
          const double2 f = flm[foff[g.maps[neg ? j - nb : j]] + (size_t)l * l + l + (neg ? -am : am)];
          x = ((n & 1) ? f.y : f.x) * nltab[l];
          if (neg && (l & 1)) x = -x;
        }
      }
      Bs[n][k] = x;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kKt / 4; ++ks) {
      const double a = At[4 * ks + q][8 * warp + gq];
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) dmma(acc[nt][0], acc[nt][1], a, Bs[8 * nt + gq][4 * ks + q]);
    }
    __syncthreads();
  }
  const int mp = mp0 + 8 * warp + gq;
  if (mp < L && mp < l1) {
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const int j = 4 * nt + q;
      if (j >= 2 * nb) continue;
      const bool neg = j >= nb;
      if (neg && am == 0) continue;
      double re = acc[nt][0], im = acc[nt][1];
      if (neg && (mp & 1)) { re = -re; im = -im; }
      double2* dst = Fp + ((size_t)g.maps[neg ? j - nb : j] * M + (neg ? -am : am) + L - 1) * L + mp;
      double2 cur = *dst;
      cur.x += re;
      cur.y += im;
      *dst = cur;
    }
  }
}

}  // namespace

cudaError_t launch_dmma_forward(const mw_plan* p, int l0, int l1, double2* flm, cudaStream_t st) {
  k_dmma_forward<<<dim3(l1, (unsigned)p->groups.size()), kThreads, 0, st>>>(
      p->d_S, p->LD, p->L, p->M, l0, l1, p->d_groups, p->d_Gp, p->d_nl, flm, p->d_foff);
  return cudaGetLastError();
}

cudaError_t launch_dmma_inverse(const mw_plan* p, int l0, int l1, const double2* flm, cudaStream_t st) {
  const dim3 grid(l1, (l1 + kRows - 1) / kRows, (unsigned)p->groups.size());
  k_dmma_inverse<<<grid, kThreads, 0, st>>>(p->d_S, p->LD, p->L, p->M, l0, l1, p->d_groups, flm, p->d_foff, p->d_nl,
                                            p->d_Gp);
  return cudaGetLastError();
}
