// kernels_tn.cu -- Delta^l = d^l(pi/2) by the Trapani-Navaza recursion (cited
// in Sec. V-B as the alternative to Risbo's), for the mixed precisions.
//
// Column m of the quarter plane (m' = l .. 0, rows m', columns m) starts from
// the top row Delta^l_{l,m} = (-1)^(l-m) 2^-l sqrt(C(2l, l+m)) and recurses
// down the first index with the three-term relation of d^l at beta = pi/2,
//   sqrt((l+m')(l-m'+1)) Delta_{m'-1,m}
//     = 2 m Delta_{m',m} - sqrt((l-m')(l+m'+1)) Delta_{m'+1,m},
// stopping at m' = 0: every step then runs towards growing or oscillating
// values (the region of |m'| <= sqrt(l^2 - m^2) is where |Delta| is large), so
// the recursion is stable.  What limits the recursion in double precision is
// the start values, which fall to about exp(-0.28 l) at m = l / sqrt2 and to
// 2^-l at m = l and leave the double range near l = 2560.  Here each column
// carries its own power-of-two exponent: value = x 2^E with x a float-float
// pair, rescaled by 2^-64 whenever |x| exceeds 2^64 (tested every second
// step), and the start values come from a host table of (float-float
// mantissa, exponent) pairs.
//
// Planes are independent given their top rows, and so are the columns of a
// plane: one thread per column, one block per (plane, 128 or 256 columns), no waits
// between blocks.  A block first forms the plane's recursion coefficients
// 2/b(m') and a(m')/b(m') in shared memory (b = sqrt((l+m')(l-m'+1)),
// a = sqrt((l-m')(l+m'+1))); each step then costs an exact scaling of 2/b by
// the column index (3 FP32 instructions), one float-float product (7) and one
// multiply-add (15).  Every step writes one
// row of the FP32 staging plane, consecutive columns in consecutive threads,
// so the stores are coalesced and the full quarter is written without a
// transpose.
#include <cmath>

#include "ff.cuh"
#include "internal.h"

namespace {

constexpr int kTThreads = 256;  // largest block (columns per block: 128 or 256, chosen by the plan)
constexpr int kTMaxL = 2048;

struct TnArgs {
  float* S32;               // FP32 staging: plane l at slot l - l0
  int l0;
  int LD;
  const float2* sq;         // sqrt(k) as float-float
  const float2* rsq;        // 1/sqrt(k) as float-float
  const float2* top;        // top-row mantissas, plane l at l (l + 1) / 2
  const int* top_exp;       // top-row exponents
};

// 2^k as a float for -126 <= k <= 127 (exact, built from the exponent field)
__device__ __forceinline__ float exp2_int(int k) { return __int_as_float((k + 127) << 23); }

// The power of two 2^E of a column as two float factors f1 f2 (f1 = 2^max(E, -126),
// f2 = the rest, 0 below 2^-252), so that x 2^E = (x f1) f2: one rounding for
// every result in the normal range; below 2^-126 (irrelevant next to the
// 2^-24 staging precision) the result is a denormal or zero.
struct Scale2 {
  float f1, f2;
  __device__ __forceinline__ void set(int E) {
    const int e1 = E > -126 ? E : -126;
    f1 = exp2_int(e1);
    f2 = (E - e1 < -126) ? 0.0f : exp2_int(E - e1);
  }
  __device__ __forceinline__ float apply(float x) const { return __fmul_rn(__fmul_rn(x, f1), f2); }
};

__global__ void __launch_bounds__(kTThreads) k_tn_planes(TnArgs A, int lb) {
  __shared__ float4 cc[kTMaxL + 1];  // (2 / b(m'), a(m') / b(m')) as float-float pairs, one 16-byte load per step
  const int l = lb + (int)blockIdx.y;
  const int m0 = (int)(blockIdx.x * blockDim.x);
  if (m0 > l) return;  // whole block past the plane's last column (uniform)
  for (int mp = 1 + (int)threadIdx.x; mp <= l; mp += (int)blockDim.x) {
    const float2 ib = NumFF::mul(A.rsq[l + mp], A.rsq[l - mp + 1]);
    const float2 c2 = NumFF::mul(NumFF::mul(A.sq[l - mp], A.sq[l + mp + 1]), ib);
    cc[mp] = make_float4(2.0f * ib.x, 2.0f * ib.y, c2.x, c2.y);  // 2 ib exact
  }
  __syncthreads();
  const int m = m0 + (int)threadIdx.x;
  if (m > l) return;
  const int LD = A.LD;
  float* st = A.S32 + (size_t)(l - A.l0) * LD * LD + m;
  const size_t t0 = (size_t)l * (l + 1) / 2 + m;
  float2 cur = A.top[t0];
  float2 prev = make_float2(0.f, 0.f);
  int E = A.top_exp[t0];
  Scale2 sc;
  sc.set(E);
  st[(size_t)l * LD] = sc.apply(cur.x);
  const float mf = (float)m;  // exact (m <= 2047)
  // one step m' -> m' - 1: 2 m / b is the float-float 2 / b times the exact
  // integer m -- TwoProduct of the high part, the low part's product added to
  // its error, left unnormalised (the pair only feeds the fused multiply-add)
  auto step = [&](int mp) {
    const float4 c = cc[mp];
    const float tp = __fmul_rn(c.x, mf);
    const float2 t = make_float2(tp, __fmaf_rn(c.y, mf, __fmaf_rn(c.x, mf, -tp)));
    const float2 u = NumFF::mul(make_float2(c.z, c.w), prev);  // (a / b) Delta_{m'+1}
    const float2 nw = NumFF::fma(t, cur, make_float2(-u.x, -u.y));
    prev = cur;
    cur = nw;
    st[(size_t)(mp - 1) * LD] = sc.apply(cur.x);
  };
  // One step multiplies max(|cur|, |prev|) by at most 2m/b + a/b <=
  // sqrt(2l) + 1 < 2^7 (b >= sqrt(2l), a < b), so with both values below 2^64
  // two steps stay below 2^78: the rescale test runs once per pair of steps,
  // before the pair's stores take the scale.  Powers of two scale both parts
  // exactly.
  auto rescale = [&]() {
    if (fmaxf(fabsf(cur.x), fabsf(prev.x)) > 0x1p64f) {
      cur = make_float2(cur.x * 0x1p-64f, cur.y * 0x1p-64f);
      prev = make_float2(prev.x * 0x1p-64f, prev.y * 0x1p-64f);
      E += 64;
      sc.set(E);
    }
  };
  int mp = l;
  for (; mp >= 2; mp -= 2) {
    rescale();
    step(mp);
    step(mp - 1);
  }
  if (mp == 1) {
    rescale();
    step(1);
  }
}

}  // namespace

// Planes l in [lb, le) into the staging slots l - l0 of plan p's sweep state.
cudaError_t launch_tn(const mw_plan* p, int l0, int lb, int le, cudaStream_t st) {
  if (lb >= le) return cudaSuccess;
  if (le > kTMaxL) return cudaErrorInvalidValue;
  TnArgs a;
  a.S32 = p->d_S32;
  a.l0 = l0;
  a.LD = p->LD;
  a.sq = p->d_sqrt_ff;
  a.rsq = p->d_rsqrt_ff;
  a.top = p->d_tn_top;
  a.top_exp = p->d_tn_exp;
  const int nt = (p->tn_threads == 128 || p->tn_threads == 256) ? p->tn_threads : kTThreads;
  const dim3 grid((le - 1) / nt + 1, le - lb);
  k_tn_planes<<<grid, nt, 0, st>>>(a, lb);
  return cudaGetLastError();
}
