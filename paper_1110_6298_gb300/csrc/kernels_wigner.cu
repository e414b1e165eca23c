// kernels_wigner.cu -- the O(L^3) Wigner stage: Delta^l_{mn} = d^l_{mn}(pi/2) by
// Risbo's recursion, and the contractions of Eq. (flm_wig) and Eq. (Fmm).
//
// Risbo's recursion couples d^j with the spin-1/2 matrix to get d^{j+1/2}; in
// gather form, for the new plane j' = j + 1/2 (p = q = cos(pi/4) at beta = pi/2):
//   e_{mu,nu} = 1/(2 sqrt2 j') [ sqrt(j'-nu) ( sqrt(j'-mu) d_{mu+1/2,nu+1/2}
//                                             - sqrt(j'+mu) d_{mu-1/2,nu+1/2} )
//                              + sqrt(j'+nu) ( sqrt(j'-mu) d_{mu+1/2,nu-1/2}
//                                             + sqrt(j'+mu) d_{mu-1/2,nu-1/2} ) ]
// (entries of d outside |index| <= j are zero).  Two half steps take Delta^{l-1}
// to Delta^l.  At beta = pi/2 the symmetries of Sec. III-C,
//   d_{-m,n} = (-1)^(j-n) d_{mn}   (Eq. wignerd_sym2 with beta = pi/2)
//   d_{m,-n} = (-1)^(j+m) d_{mn}   (with Eq. wignerd_sym1)
//   d_{nm}   = (-1)^(m-n) d_{mn}   (Eq. wignerd_sym3 and d(-b) = d(b)^T)
// let every plane be kept as its quarter mu, nu >= 0; the stencil reaches across
// the axes only at mu or nu = 0 of an integer plane, where it reflects.
//
// Plane storage: quarter plane with rows a = mu - off and columns b = nu - off
// (off = 0 for integer j, 1/2 for half-integer j), row stride LD = L + 1.
//
// The contraction uses the fold over +-m' (Delta_{-m',m} Delta_{-m',-s} =
// (-1)^(m+s) Delta_{m'm} Delta_{m',-s}) so that it runs over m' >= 0 only, and
// reads Delta_{m'm} from row |m| of the quarter plane through the transpose
// symmetry, so every access is a contiguous row segment.
#include <cmath>

#include "internal.h"

namespace {

__device__ __forceinline__ double sgn_pow(int k) { return (k & 1) ? -1.0 : 1.0; }

// new plane 2j' = two_jp from old plane (j = j' - 1/2)
__global__ void k_risbo_half(const double* __restrict__ d, double* __restrict__ e, int two_jp, int LD,
                             const double* __restrict__ sq, double scale, float* __restrict__ stage) {
  const int odd = two_jp & 1;                // j' half-integer
  const int nnew = odd ? (two_jp + 1) / 2 : two_jp / 2 + 1;
  const int nold = (two_jp + 1) / 2;
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  const int a = blockIdx.y * blockDim.y + threadIdx.y;
  if (a >= nnew || b >= nnew) return;
  const int mu2 = 2 * a + odd, nu2 = 2 * b + odd;  // twice mu, nu
  const int jo2 = two_jp - 1;                      // twice the old j
  const double cmm = sq[(two_jp - mu2) / 2], cpm = sq[(two_jp + mu2) / 2];
  const double cmn = sq[(two_jp - nu2) / 2], cpn = sq[(two_jp + nu2) / 2];
  // old indices of mu +- 1/2 and nu +- 1/2
  const int ip = a + odd, im = a - 1 + odd;
  const int jp = b + odd, jm = b - 1 + odd;
  auto at = [&](int i, int k) -> double {
    if (i >= nold || k >= nold) return 0.0;
    double sgn = 1.0;
    // only -1/2 can occur (integer new plane, old half-integer plane)
    if (i < 0) {  // d_{-1/2, n} = (-1)^(j - n) d_{1/2, n},  n = k + 1/2
      const int n2 = (k < 0) ? -1 : 2 * k + 1;
      sgn *= sgn_pow((jo2 - n2) / 2);
      i = 0;
    }
    if (k < 0) {  // d_{m, -1/2} = (-1)^(j + m) d_{m, 1/2},  m = i + 1/2 (after the row reflection)
      const int m2 = 2 * i + 1;
      sgn *= sgn_pow((jo2 + m2) / 2);
      k = 0;
    }
    return sgn * d[(size_t)i * LD + k];
  };
  const double dpp = at(ip, jp), dmp = at(im, jp), dpm = at(ip, jm), dmm = at(im, jm);
  const double v = cmn * (cmm * dpp - cpm * dmp) + cpn * (cmm * dpm + cpm * dmm);
  const double out = scale * v;
  e[(size_t)a * LD + b] = out;
  if (stage) stage[(size_t)a * LD + b] = (float)out;  // FP32 copy for the tensor-core contraction
}

__global__ void k_plane_init(double* S, float* S32) {
  S[0] = 1.0;
  if (S32) S32[0] = 1.0f;
}

// Forward contraction for planes l in [l0, l1) stored at slots l % kChunk:
//   f_lm = (-1)^s i^(m+s) N_l sum_{m'=0}^{l} K_m[l,m'] G+_{m,m'},
//   K_m[l,m'] = Delta^l_{m'm} Delta^l_{m',-s}.
// One block per (m, spin group); rows l of the chunk x maps of the group.
constexpr int kTileMp = 64;

__global__ void k_contract_forward(const double* __restrict__ S, int LD, int L, int M, int l0, int l1,
                                   const SpinGroup* __restrict__ groups, const double2* __restrict__ Gp,
                                   double2* __restrict__ flm) {
  __shared__ double Kt[kChunk][kTileMp + 1];
  __shared__ double2 Gs[kMaxGroupMaps][kTileMp];
  const int im = blockIdx.x, m = im - (L - 1), am = m < 0 ? -m : m;
  const SpinGroup& g = groups[blockIdx.y];
  const int s = g.s, as = s < 0 ? -s : s, nb = g.nb;
  const int lstart = max(l0, am);
  if (lstart >= l1) return;
  const int nl = l1 - l0;
  const int npairs = nl * nb;
  // per-thread accumulators over (l, map) pairs
  constexpr int kMaxPairsPerThread = (kChunk * kMaxGroupMaps + 255) / 256;
  double ar[kMaxPairsPerThread], ai[kMaxPairsPerThread];
#pragma unroll
  for (int q = 0; q < kMaxPairsPerThread; ++q) { ar[q] = 0.0; ai[q] = 0.0; }
  const int lmax = l1 - 1;
  for (int mp0 = 0; mp0 <= lmax; mp0 += kTileMp) {
    // K tile: rows l (chunk), columns m' in [mp0, mp0 + kTileMp)
    for (int idx = threadIdx.x; idx < nl * kTileMp; idx += blockDim.x) {
      const int r = idx / kTileMp, c = idx % kTileMp;
      const int l = l0 + r, mp = mp0 + c;
      double k = 0.0;
      if (l >= lstart && l >= as && mp <= l) {
        const double* P = S + (size_t)(l % kChunk) * LD * LD;
        // Delta_{m'|m|} = (-1)^(m'-|m|) P[|m|][m'], Delta_{m'|s|} likewise
        double v = P[(size_t)am * LD + mp] * P[(size_t)as * LD + mp];
        int ex = am + as;                      // (-1)^(m'-|m|) (-1)^(m'-|s|)
        if (m < 0) ex += l + mp;               // Delta_{m',-|m|} = (-1)^(l+m') Delta_{m',|m|}
        if (s > 0) ex += l + mp;               // Delta_{m',-s} for s > 0
        k = sgn_pow(ex) * v;
      }
      Kt[r][c] = k;
    }
    for (int idx = threadIdx.x; idx < nb * kTileMp; idx += blockDim.x) {
      const int bb = idx / kTileMp, c = idx % kTileMp;
      const int mp = mp0 + c;
      Gs[bb][c] = (mp < L) ? Gp[((size_t)g.maps[bb] * M + im) * L + mp] : make_double2(0.0, 0.0);
    }
    __syncthreads();
#pragma unroll
    for (int q = 0; q < kMaxPairsPerThread; ++q) {
      const int pidx = threadIdx.x + q * blockDim.x;
      if (pidx < npairs) {
        const int r = pidx / nb, bb = pidx % nb;
        double sr = ar[q], si = ai[q];
        for (int c = 0; c < kTileMp; ++c) {
          const double k = Kt[r][c];
          const double2 gv = Gs[bb][c];
          sr = fma(k, gv.x, sr);
          si = fma(k, gv.y, si);
        }
        ar[q] = sr; ai[q] = si;
      }
    }
    __syncthreads();
  }
  // epilogue: times (-1)^s i^(m+s) N_l, write f_lm (zero for l < |s|)
  const int r4 = (m + s) & 3;
  const double pr = (r4 == 0) ? 1.0 : (r4 == 2 ? -1.0 : 0.0);
  const double pi_ = (r4 == 1) ? 1.0 : (r4 == 3 ? -1.0 : 0.0);
  const double sgs = sgn_pow(s);
#pragma unroll
  for (int q = 0; q < kMaxPairsPerThread; ++q) {
    const int pidx = threadIdx.x + q * blockDim.x;
    if (pidx < npairs) {
      const int r = pidx / nb, bb = pidx % nb;
      const int l = l0 + r;
      if (l < lstart) continue;
      double2 o = make_double2(0.0, 0.0);
      if (l >= as) {
        const double nl_ = sgs * sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
        o.x = nl_ * (pr * ar[q] - pi_ * ai[q]);
        o.y = nl_ * (pr * ai[q] + pi_ * ar[q]);
      }
      flm[(size_t)g.maps[bb] * L * L + (size_t)l * l + l + m] = o;
    }
  }
}

// Inverse contraction, accumulated over chunks into F+ (m' >= 0):
//   F+_{m,m'} += sum_{l in chunk} N_l K_m[l,m'] f_lm
// (the phase (-1)^s i^-(m+s) is applied when F is unfolded).
// One block per (m, m'-tile, spin group).
__global__ void k_contract_inverse(const double* __restrict__ S, int LD, int L, int M, int l0, int l1,
                                   const SpinGroup* __restrict__ groups, const double2* __restrict__ flm,
                                   double2* __restrict__ Fp) {
  __shared__ double Kt[kChunk][kTileMp + 1];
  __shared__ double2 Fs[kMaxGroupMaps][kChunk];
  const int im = blockIdx.x, m = im - (L - 1), am = m < 0 ? -m : m;
  const int mp0 = blockIdx.y * kTileMp;
  const SpinGroup& g = groups[blockIdx.z];
  const int s = g.s, as = s < 0 ? -s : s, nb = g.nb;
  const int lstart = max(max(l0, am), as);
  if (lstart >= l1 || mp0 > l1 - 1) return;
  const int nl = l1 - l0;
  for (int idx = threadIdx.x; idx < nl * kTileMp; idx += blockDim.x) {
    const int r = idx / kTileMp, c = idx % kTileMp;
    const int l = l0 + r, mp = mp0 + c;
    double k = 0.0;
    if (l >= lstart && mp <= l) {
      const double* P = S + (size_t)(l % kChunk) * LD * LD;
      double v = P[(size_t)am * LD + mp] * P[(size_t)as * LD + mp];
      int ex = am + as;
      if (m < 0) ex += l + mp;
      if (s > 0) ex += l + mp;
      k = sgn_pow(ex) * v * sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
    }
    Kt[r][c] = k;
  }
  for (int idx = threadIdx.x; idx < nb * nl; idx += blockDim.x) {
    const int bb = idx / nl, r = idx % nl;
    const int l = l0 + r;
    Fs[bb][r] = (l >= lstart) ? flm[(size_t)g.maps[bb] * L * L + (size_t)l * l + l + m] : make_double2(0.0, 0.0);
  }
  __syncthreads();
  for (int pidx = threadIdx.x; pidx < kTileMp * nb; pidx += blockDim.x) {
    const int c = pidx % kTileMp, bb = pidx / kTileMp;
    const int mp = mp0 + c;
    if (mp >= L) continue;
    double2* dst = Fp + ((size_t)g.maps[bb] * M + im) * L + mp;
    double sr = dst->x, si = dst->y;
    for (int r = 0; r < nl; ++r) {
      const double k = Kt[r][c];
      const double2 f = Fs[bb][r];
      sr = fma(k, f.x, sr);
      si = fma(k, f.y, si);
    }
    *dst = make_double2(sr, si);
  }
}

}  // namespace

namespace {

cudaError_t run_wigner_fp64(mw_plan* p, int mode, const double2* flm_in, double2* flm_out, cudaStream_t st,
                            int* launches) {
  const int L = p->L, M = p->M, LD = p->LD;
  const int ng = (int)p->groups.size();
  int nl = 0;
  cudaError_t e;
  if (mode == 1) {
    e = cudaMemsetAsync(p->d_Gp, 0, sizeof(double2) * (size_t)p->B * M * L, st);
    if (e != cudaSuccess) return e;
  }
  k_plane_init<<<1, 1, 0, st>>>(p->d_S, nullptr);
  ++nl;
  for (int l0 = 0; l0 < L; l0 += kChunk) {
    const int l1 = (l0 + kChunk < L) ? l0 + kChunk : L;
    StageSpan span_d(p, MW_STAGE_DELTA, st);
    int nd = 0;
    for (int l = (l0 == 0 ? 1 : l0); l < l1; ++l) {
      const double* prev = p->d_S + (size_t)((l - 1) % kChunk) * LD * LD;
      double* cur = p->d_S + (size_t)(l % kChunk) * LD * LD;
      // half-integer plane j' = l - 1/2, then integer plane j' = l
      for (int h = 0; h < 2; ++h) {
        const int two_jp = 2 * l - 1 + h;
        const int nnew = (two_jp & 1) ? (two_jp + 1) / 2 : two_jp / 2 + 1;
        const dim3 blk(32, 8);
        const dim3 grd((nnew + 31) / 32, (nnew + 7) / 8);
        const double scale = 1.0 / (sqrt(2.0) * (double)two_jp);
        k_risbo_half<<<grd, blk, 0, st>>>(h == 0 ? prev : p->d_H, h == 0 ? p->d_H : cur, two_jp, LD, p->d_sqrt,
                                          scale, nullptr);
        ++nd;
      }
    }
    span_d.end(nd);
    nl += nd;
    StageSpan span_c(p, MW_STAGE_CONTRACT, st);
    if (mode == 0) {
      k_contract_forward<<<dim3(M, ng), 256, 0, st>>>(p->d_S, LD, L, M, l0, l1, p->d_groups, p->d_Gp, flm_out);
    } else {
      k_contract_inverse<<<dim3(M, (l1 + kTileMp - 1) / kTileMp, ng), 256, 0, st>>>(p->d_S, LD, L, M, l0, l1,
                                                                                     p->d_groups, flm_in, p->d_Gp);
    }
    span_c.end(1);
    ++nl;
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  if (launches) *launches += nl;
  return cudaGetLastError();
}

// Mixed path: FP64 recursion state in two ping-pong planes, FP32 copies of the
// integer planes of a 128-plane chunk for the tensor-core contraction.
cudaError_t run_wigner_mixed(mw_plan* p, int mode, const double2* flm_in, double2* flm_out, cudaStream_t st,
                             int* launches) {
  const int L = p->L, M = p->M, LD = p->LD;
  const size_t plane = (size_t)LD * LD;
  int nl = 0;
  cudaError_t e;
  if (mode == 1) {
    e = cudaMemsetAsync(p->d_Gp, 0, sizeof(double2) * (size_t)p->B * M * L, st);
    if (e != cudaSuccess) return e;
  }
  k_plane_init<<<1, 1, 0, st>>>(p->d_S, p->d_S32);
  ++nl;
  for (int l0 = 0; l0 < L; l0 += kTcChunk) {
    const int l1 = (l0 + kTcChunk < L) ? l0 + kTcChunk : L;
    StageSpan span_d(p, MW_STAGE_DELTA, st);
    int nd = 0;
    for (int l = (l0 == 0 ? 1 : l0); l < l1; ++l) {
      const double* prev = p->d_S + (size_t)((l - 1) & 1) * plane;
      double* cur = p->d_S + (size_t)(l & 1) * plane;
      for (int h = 0; h < 2; ++h) {
        const int two_jp = 2 * l - 1 + h;
        const int nnew = (two_jp & 1) ? (two_jp + 1) / 2 : two_jp / 2 + 1;
        const dim3 blk(32, 8);
        const dim3 grd((nnew + 31) / 32, (nnew + 7) / 8);
        const double scale = 1.0 / (sqrt(2.0) * (double)two_jp);
        k_risbo_half<<<grd, blk, 0, st>>>(h == 0 ? prev : p->d_H, h == 0 ? p->d_H : cur, two_jp, LD, p->d_sqrt,
                                          scale, h == 0 ? nullptr : p->d_S32 + (size_t)(l - l0) * plane);
        ++nd;
      }
    }
    span_d.end(nd);
    nl += nd;
    StageSpan span_c(p, MW_STAGE_CONTRACT, st);
    e = (mode == 0) ? launch_tc_forward(p, l0, l1, flm_out, st) : launch_tc_inverse(p, l0, l1, flm_in, st);
    span_c.end(1);
    ++nl;
    if (e != cudaSuccess) return e;
  }
  if (launches) *launches += nl;
  return cudaGetLastError();
}

}  // namespace

cudaError_t run_wigner(mw_plan* p, int mode, const double2* flm_in, double2* flm_out, cudaStream_t st,
                       int* launches) {
  return p->prec == MW_PREC_FP64 ? run_wigner_fp64(p, mode, flm_in, flm_out, st, launches)
                                 : run_wigner_mixed(p, mode, flm_in, flm_out, st, launches);
}
