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
// The contractions (kernels_tc.cu, kernels_dmma.cu) use the fold over +-m'
// (Delta_{-m',m} Delta_{-m',-s} = (-1)^(m+s) Delta_{m'm} Delta_{m',-s}) so that
// they run over m' >= 0 only, and read Delta_{m'm} from row |m| of the quarter
// plane through the transpose symmetry, so every access is a contiguous row
// segment.
#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <utility>
#include <vector>

#include "ff.cuh"
#include "internal.h"

namespace {

__device__ __forceinline__ double sgn_pow(int k) { return (k & 1) ? -1.0 : 1.0; }

// v * (-1)^k by flipping the sign bit on the integer pipe (the FP64 pipe is the
// bottleneck of the recursion on this part)
__device__ __forceinline__ double flip_sign(double v, int k) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)(k & 1) << 63));
}

// double -> float, round to nearest (ties away), on the integer pipe; values
// below 2^-126 in magnitude (irrelevant for |Delta| <= 1 at the 1e-6 level)
// become signed zero.  |v| <= 1 here, so there is no overflow.
__device__ __forceinline__ float to_f32_int(double v) {
  const unsigned long long u = (unsigned long long)__double_as_longlong(v);
  const unsigned sign = (unsigned)(u >> 63) << 31;
  const int e = (int)((u >> 52) & 0x7FF);
  if (e <= 896) return __uint_as_float(sign);
  const unsigned long long m = u & 0xFFFFFFFFFFFFFull;
  const unsigned f = ((unsigned)(e - 896) << 23) + (unsigned)((m + (1ull << 28)) >> 29);
  return __uint_as_float(sign | f);
}

// ---------------------------------------------------------------------------
// Arithmetic of the recursion state.  The FP64 path recurses in double.  The
// mixed path recurses in float-float: a value is the unevaluated sum hi + lo of
// two floats with |lo| <= ulp(hi) / 2 (about 48 significant bits), built from
// the error-free transformations TwoSum (Knuth) and TwoProduct by FMA
// (Dekker's product with a fused multiply-add), so the stencil runs on the FP32
// pipe, which is about 68 times faster than the FP64 pipe on this part.  The
// planes feed an FP32 staging copy and a contraction designed for 1e-6, so 48
// bits leave a margin of about five orders of magnitude over the 2L half steps.
// The _rn intrinsics keep the compiler from contracting a product into the
// following sum, which would break the error terms.
// ---------------------------------------------------------------------------
struct NumF64 {
  using T = double;
  static __device__ __forceinline__ T zero() { return 0.0; }
  static __device__ __forceinline__ T mul(T a, T b) { return a * b; }
  static __device__ __forceinline__ T fma(T a, T b, T c) { return ::fma(a, b, c); }
  static __device__ __forceinline__ T fms(T a, T b, T c) { return ::fma(-a, b, c); }  // c - a b
  static __device__ __forceinline__ T flip(T v, int k) { return flip_sign(v, k); }
  static __device__ __forceinline__ float f32(T v) { return to_f32_int(v); }
};


// ---------------------------------------------------------------------------
// Persistent Risbo sweep over the planes l in [l_begin, l_end) of one chunk.
//
// One cooperative launch per chunk of planes.  Each l is one pass over 32 x 32
// tiles of the lower triangle
// b <= a of the new quarter plane (the transpose symmetry supplies the rest):
// a tile stages the previous integer plane Delta^{l-1} on rows/columns
// a0-1 .. a0+32 in shared memory, computes the half-integer plane d^{l-1/2} on
// rows/columns a0-1 .. a0+31 (including the index -1, i.e. m = -1/2, directly
// from the gather formula) and from it the integer plane Delta^l on the tile.
// Recomputing the 33 x 33 half plane per tile costs 6% more arithmetic than a
// global half step but saves a grid barrier and the half plane's memory
// traffic per l.  Per element the stencil costs 4 (half plane) or 5 (integer
// plane) multiply-adds: with the column factors cn = sqrt(j'-nu)/(2 sqrt2 j'),
// cp = sqrt(j'+nu)/(2 sqrt2 j') kept in shared memory,
//   e = cn (sqrt(j'-mu) d_{+,+} - sqrt(j'+mu) d_{-,+}) + cp (sqrt(j'-mu) d_{+,-} + sqrt(j'+mu) d_{-,-}).
// Integer planes are also written out as full quarters where a contraction
// reads them (FP32 staging copy on the mixed path; the FP64 plane itself on the
// FP64 path), the upper triangle through an in-shared-memory transpose.  The
// kernel is a template over the number type of the state (NumF64 on the FP64
// path, NumFF on the mixed paths); both take 8 bytes per element.
// ---------------------------------------------------------------------------
constexpr int kRT = 32;         // tile edge
constexpr int kRThreads = 256;  // 32 x 8 threads
constexpr unsigned kBarrierPolls = 1u << 24;

struct RisboArgs {
  void* S;            // integer planes (double or float-float); plane l at slot l % nslot
  int nslot;
  float* S32;         // FP32 staging of the integer planes (slot l - l0), or null
  int l0;
  int full64;         // write transposed tiles into the FP64 integer plane
  int LD;
  const void* sq;        // sqrt(k)               (tables in the recursion's number type)
  const void* rsq;       // 1/sqrt(k), k >= 1
  const void* rscale;    // 1 / (sqrt2 two_jp)
  int* prog;          // per-tile progress: last plane l published
  int* err;
  const int* perm;    // rank of each block in the tile assignment (null: blockIdx.x)
  int* smid_out;      // when set: record each block's SM id (placement probe)
  unsigned polls;     // poll limit of a neighbour wait
  int stall_l;        // debug: the block of rank stall_rank leaves before plane stall_l (-1: never)
  int stall_rank;
};

// Value of the integer plane Delta^{l-1} (j = l-1, quarter storage, lower
// triangle valid) at quarter indices (i, k), which may be -1 or above the
// diagonal: index -1 is m = -1 and reflects to +1 through
//   d_{-m,n} = (-1)^(j-n) d_{mn}, d_{m,-n} = (-1)^(j+m) d_{mn}  (Eq. wignerd_sym2 at pi/2, sym1),
// and the upper triangle is read through d_{mn} = (-1)^(m-n) d_{nm}.
template <class Nm>
__device__ __forceinline__ typename Nm::T prev_val(const typename Nm::T* __restrict__ d, int LD, int i, int k, int j) {
  int ex = 0;  // value = (-1)^ex d[i][k]
  if (i < 0) { ex += j - k; i = -i; }
  if (k < 0) { ex += j + i; k = -k; }
  if (i > j || k > j) return Nm::zero();
  if (k > i) { ex += i - k; const int t = i; i = k; k = t; }
  return Nm::flip(__ldcg(d + (size_t)i * LD + k), ex);  // L2: written by other blocks for the last l
}

// Tile (I, J), J <= I, of the lower triangle has linear index I (I+1)/2 + J.
__device__ __forceinline__ int tile_index(int I, int J) { return I * (I + 1) / 2 + J; }

// Wait until tile t has published step `step` (bounded by max_polls; returns
// false on timeout).  The first polls spin (a neighbour of the same wavefront
// is usually about to publish); later ones back off with a short sleep.
__device__ __forceinline__ bool wait_tile(const int* prog, int t, int step, unsigned max_polls) {
  for (unsigned polls = 0; polls < max_polls; ++polls) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(prog + t) : "memory");
    if (v >= step) return true;
    if (polls >= 256) __nanosleep(32);
  }
  return false;
}

__global__ void k_prog_init(int* prog, int n, int value) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) prog[i] = value;
}

// Dataflow scheduling: block c owns the tiles t = c, c + G, ... and processes
// (l, t) in increasing (l, t) order; before computing tile (I, J) of plane l it
// waits until the tiles of plane l-1 that its halo reads -- block rows I-1..I+1
// and columns J-1..J+1, mapped into the lower triangle -- have published l-1,
// then publishes l itself.  Every block follows the same global order and the
// launch is cooperative (all blocks co-resident), so every wait ends; a wait
// that exceeds its poll limit records the timeout and the block leaves.  A
// block that overwrites plane l-2 (two-plane ping-pong) does so only after all
// readers of that region -- its neighbours at step l-1 -- have finished.
// Shared memory of one block: kPair tiles of one step are processed together
// (tiles t and t + G are far apart, so neither waits for the other).  One tile
// per pass measured as fast as two, with half the shared memory.
constexpr int kPair = 1;
template <class V>
struct RisboSmem {
  V dh[kPair][kRT + 2][kRT + 3];  // Delta^{l-1} on rows/cols a0-1 .. a0+32
  V hh[kPair][kRT + 1][kRT + 1];  // d^{l-1/2} on rows/cols a0-1 .. a0+31
  V tr[kPair][kRT][kRT + 1];      // Delta^l on the tile
  V colf[kPair][4][kRT + 1];      // cn, cp of the half plane (33 cols) and of the integer plane (32)
  V rowf[kPair][4][kRT + 1];      // sqrt(j'-mu), sqrt(j'+mu) of the half-plane rows (33) and integer rows (32)
  int ok;
};
static_assert(sizeof(RisboSmem<double>) == sizeof(RisboSmem<float2>), "both number types take 8 bytes");
constexpr int kRisboSmem = (int)sizeof(RisboSmem<double>);

template <class Nm>
__global__ void __launch_bounds__(kRThreads, 5) k_risbo_sweep(RisboArgs A, int l_begin, int l_end) {
  using V = typename Nm::T;
  extern __shared__ __align__(16) unsigned char risbo_smem[];
  RisboSmem<V>& sm = *reinterpret_cast<RisboSmem<V>*>(risbo_smem);
  const V* sq = static_cast<const V*>(A.sq);
  const V* rsq = static_cast<const V*>(A.rsq);
  const V* rscale = static_cast<const V*>(A.rscale);
  const int tid = threadIdx.x, tx = tid & 31, ty = tid >> 5;
  const int LD = A.LD;
  const size_t plane = (size_t)LD * LD;
  const int G = gridDim.x;
  if (A.smid_out && tid == 0) {
    unsigned sid;
    asm volatile("mov.u32 %0, %%smid;" : "=r"(sid));
    A.smid_out[blockIdx.x] = (int)sid;
  }
  // Block ranks 0..#SM-1 are blocks on distinct SMs (see make_risbo_perm), so the
  // few tiles of the early planes spread over all SMs instead of sharing the
  // FP64 pipes of the SMs the first block indices land on.
  const int vrank = A.perm ? A.perm[blockIdx.x] : (int)blockIdx.x;
  for (int l = l_begin; l < l_end; ++l) {
    // debug fault injection on the host's request: this block leaves without
    // publishing, so its neighbours' bounded waits run out (no trap, no fault)
    if (l == A.stall_l && vrank == A.stall_rank) return;
    const int th = 2 * l - 1, ti = 2 * l;  // twice j' of the half and the integer plane
    const int nh = l, nnew = l + 1;        // sizes of the half plane and the new integer plane
    const V* d = static_cast<const V*>(A.S) + (size_t)((l - 1) % A.nslot) * plane;
    V* e = static_cast<V*>(A.S) + (size_t)(l % A.nslot) * plane;
    float* st = A.S32 ? A.S32 + (size_t)(l - A.l0) * plane : nullptr;
    const V sch = rscale[th], sci = rscale[ti];
    const int T = (nnew + kRT - 1) / kRT;       // tile rows of plane l
    const int Tp = (l + kRT - 1) / kRT;         // tile rows of plane l-1 (size l)
    const int ntiles = T * (T + 1) / 2;
    for (int tb = vrank; tb < ntiles; tb += kPair * G) {
      int tt[kPair], II[kPair], JJ[kPair];
      int np = 0;
#pragma unroll
      for (int k = 0; k < kPair; ++k) {
        const int t = tb + k * G;
        tt[k] = t;
        II[k] = JJ[k] = 0;
        if (t < ntiles) {
          int I = (int)((sqrtf(8.f * (float)t + 1.f) - 1.f) * 0.5f);
          while (I * (I + 1) / 2 > t) --I;
          while ((I + 1) * (I + 2) / 2 <= t) ++I;
          II[k] = I;
          JJ[k] = t - I * (I + 1) / 2;
          np = k + 1;
        }
      }
      if (tid < 32) {  // lanes 16k + q (q < 9) wait for neighbour q of tile k, concurrently
        int ok = 1;
        const int k = tx >> 4, q = tx & 15;
        if (l > l_begin && k < np && q < 9) {
          const int Ii = II[k] + q / 3 - 1, Jj = JJ[k] + q % 3 - 1;
          if (Ii >= 0 && Jj >= 0 && Ii < Tp && Jj < Tp) {  // part of plane l-1
            const int hi = Ii > Jj ? Ii : Jj, lo = Ii > Jj ? Jj : Ii;
            if (!wait_tile(A.prog, tile_index(hi, lo), l - 1, A.polls)) { ok = 0; atomicOr(A.err, 2); }
          }
        }
        ok = __all_sync(0xffffffffu, ok);
        if (tx == 0) sm.ok = ok && !*(volatile int*)A.err;
      } else {
        // meanwhile the other warps stage the row and column factors, which do
        // not depend on the neighbours, so that no FP64 phase starts with a
        // global load: per tile 33 + 32 rows and 33 + 32 columns
#pragma unroll
        for (int k = 0; k < kPair; ++k) {
          if (k >= np) continue;
          const int a0 = II[k] * kRT, b0 = JJ[k] * kRT;
          for (int y = tid - 32; y < 2 * (2 * kRT + 1); y += kRThreads - 32) {
            if (y <= kRT) {  // half-plane row i = a0-1+y (mu = i + 1/2)
              const int i = a0 - 1 + y, mu2 = 2 * i + 1;
              const bool in = i < nh;
              sm.rowf[k][0][y] = in ? sq[(th - mu2) / 2] : Nm::zero();
              sm.rowf[k][1][y] = in ? sq[(th + mu2) / 2] : Nm::zero();
            } else if (y < 2 * kRT + 1) {  // integer-plane row a = a0 + r
              const int r = y - (kRT + 1), a = a0 + r;
              const bool in = a < nnew;
              sm.rowf[k][2][r] = in ? sq[(ti - 2 * a) / 2] : Nm::zero();
              sm.rowf[k][3][r] = in ? sq[(ti + 2 * a) / 2] : Nm::zero();
            } else if (y < 3 * kRT + 2) {  // half-plane column k = b0-1+c (nu = k + 1/2)
              const int c = y - (2 * kRT + 1);
              const int nu2 = 2 * (b0 - 1 + c) + 1;
              const bool in = (b0 - 1 + c) < nh;
              if (l == 1) {  // cn, cp themselves
                sm.colf[k][0][c] = in ? Nm::mul(sch, sq[(th - nu2) / 2]) : Nm::zero();
                sm.colf[k][1][c] = in ? Nm::mul(sch, sq[(th + nu2) / 2]) : Nm::zero();
              } else {  // cn / cp (cp = sch sqrt(l + k) > 0 inside the plane)
                sm.colf[k][0][c] = in ? Nm::mul(sq[(th - nu2) / 2], rsq[(th + nu2) / 2]) : Nm::zero();
                sm.colf[k][1][c] = Nm::zero();
              }
            } else {  // integer-plane column b = b0 + c
              const int c = y - (3 * kRT + 2), bcol = b0 + c;
              const bool in = bcol < nnew;
              V f2 = in ? Nm::mul(sci, sq[(ti - 2 * bcol) / 2]) : Nm::zero();
              V f3 = in ? Nm::mul(sci, sq[(ti + 2 * bcol) / 2]) : Nm::zero();
              if (l > 1) {  // absorb the scales cp of half-plane columns c and c+1
                const int kc = b0 - 1 + c;    // half-plane column of hh column c
                f3 = Nm::mul(f3, (kc < nh) ? Nm::mul(sch, sq[l + kc]) : Nm::zero());
                f2 = Nm::mul(f2, (kc + 1 < nh) ? Nm::mul(sch, sq[l + kc + 1]) : Nm::zero());
              }
              sm.colf[k][2][c] = f2;
              sm.colf[k][3][c] = f3;
            }
          }
        }
      }
      __syncthreads();
      if (!sm.ok) return;
      {  // all of a thread's halo loads (both tiles) are issued before any is stored
        constexpr int kLoads = ((kRT + 2) * (kRT + 2) + kRThreads - 1) / kRThreads;  // 5
        V v[kPair][kLoads];
#pragma unroll
        for (int k = 0; k < kPair; ++k) {
          const int a0 = II[k] * kRT, b0 = JJ[k] * kRT;
#pragma unroll
          for (int q = 0; q < kLoads; ++q) {
            const int idx = tid + q * kRThreads;
            v[k][q] = Nm::zero();
            if (k < np && idx < (kRT + 2) * (kRT + 2)) {
              const int r = idx / (kRT + 2), c = idx % (kRT + 2);
              v[k][q] = prev_val<Nm>(d, LD, a0 - 1 + r, b0 - 1 + c, l - 1);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < kPair; ++k) {
#pragma unroll
          for (int q = 0; q < kLoads; ++q) {
            const int idx = tid + q * kRThreads;
            if (k < np && idx < (kRT + 2) * (kRT + 2)) sm.dh[k][idx / (kRT + 2)][idx % (kRT + 2)] = v[k][q];
          }
        }
      }
      __syncthreads();
      // half plane on (i, k) = (a0-1+r, b0-1+c), r, c < 33; old indices i+1 and i.
      // Row segments: the product sqrt(j'-mu) d_{+,jp} of column c is the
      // sqrt(j'-mu) d_{+,jm} of column c+1, so it is carried along (5 FP64
      // instructions per element).  Thread tid < 231 takes the same segment of
      // each tile of the pair.
      if (tid < (kRT + 1) * 7) {
        const int r = tid % (kRT + 1), seg = tid / (kRT + 1);
        const int c0 = seg * 5, c1 = min(c0 + 5, kRT + 1);  // six segments of 5 columns, one of 3
#pragma unroll
        for (int k = 0; k < kPair; ++k) {
          if (k >= np) continue;
          const int a0 = II[k] * kRT, b0 = JJ[k] * kRT;
          const int i = a0 - 1 + r;
          if (i >= nh) {
            for (int c = c0; c < c1; ++c) sm.hh[k][r][c] = Nm::zero();
            continue;
          }
          const V cmm = sm.rowf[k][0][r], cpm = sm.rowf[k][1][r];
          V pprev = Nm::mul(cmm, sm.dh[k][r + 1][c0]);
          if (l > 1) {
            // hh holds the half plane divided by its column factor cp (which the
            // integer step's column factors carry instead): 4 multiply-adds per
            // element.  Columns outside the plane have scale 0 there.
            for (int c = c0; c < c1; ++c) {
              const V p = Nm::mul(cmm, sm.dh[k][r + 1][c + 1]);
              const V t1 = Nm::fms(cpm, sm.dh[k][r][c + 1], p);
              const V t2 = Nm::fma(cpm, sm.dh[k][r][c], pprev);
              sm.hh[k][r][c] = Nm::fma(sm.colf[k][0][c], t1, t2);
              pprev = p;
            }
          } else {
            for (int c = c0; c < c1; ++c) {
              const V p = Nm::mul(cmm, sm.dh[k][r + 1][c + 1]);
              const V t1 = Nm::fms(cpm, sm.dh[k][r][c + 1], p);
              const V t2 = Nm::fma(cpm, sm.dh[k][r][c], pprev);
              sm.hh[k][r][c] =
                  (b0 - 1 + c < nh) ? Nm::fma(sm.colf[k][1][c], t2, Nm::mul(sm.colf[k][0][c], t1)) : Nm::zero();
              pprev = p;
            }
          }
        }
      }
      __syncthreads();
      // integer plane on each tile into shared memory (half-plane indices a and
      // a-1 -> hh rows r+1 and r; row segments of 4 columns carry the shared
      // product), then coalesced stores of the tile and, where needed, of its
      // transpose
      {
        const int r = tid & 31, seg = tid >> 5;  // 32 rows x 8 segments of 4 columns
        const int c0 = seg * 4;
#pragma unroll
        for (int k = 0; k < kPair; ++k) {
          if (k >= np) continue;
          const int a = II[k] * kRT + r;
          if (a < nnew) {
            const V cmm = sm.rowf[k][2][r], cpm = sm.rowf[k][3][r];
            V pprev = Nm::mul(cmm, sm.hh[k][r + 1][c0]);
#pragma unroll
            for (int c = c0; c < c0 + 4; ++c) {
              const V p = Nm::mul(cmm, sm.hh[k][r + 1][c + 1]);
              const V t1 = Nm::fms(cpm, sm.hh[k][r][c + 1], p);
              const V t2 = Nm::fma(cpm, sm.hh[k][r][c], pprev);
              pprev = p;
              sm.tr[k][r][c] = Nm::fma(sm.colf[k][3][c], t2, Nm::mul(sm.colf[k][2][c], t1));
            }
          } else {
#pragma unroll
            for (int c = c0; c < c0 + 4; ++c) sm.tr[k][r][c] = Nm::zero();
          }
        }
      }
      __syncthreads();
      // the FP64 state of the tiles (lower triangle), which the neighbours read
      // at the next step, is written and published first; the FP32 staging
      // copy and the transposed halves, read only by later kernels, follow
      // after the publication so that the fence does not wait for them
#pragma unroll
      for (int k = 0; k < kPair; ++k) {
        if (k >= np) continue;
        const int a0 = II[k] * kRT, b0 = JJ[k] * kRT;
#pragma unroll
        for (int q = 0; q < kRT / 8; ++q) {
          const int r = ty + 8 * q;
          const int a = a0 + r, bcol = b0 + tx;
          if (a < nnew && bcol < nnew) e[(size_t)a * LD + bcol] = sm.tr[k][r][tx];
        }
      }
      __syncthreads();  // all FP64 writes of the tiles issued
      if (tid == 0) {
        __threadfence();
#pragma unroll
        for (int k = 0; k < kPair; ++k)
          if (k < np) asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(A.prog + tt[k]), "r"(l) : "memory");
      }
#pragma unroll
      for (int k = 0; k < kPair; ++k) {
        if (k >= np) continue;
        const int a0 = II[k] * kRT, b0 = JJ[k] * kRT;
        if (st) {
#pragma unroll
          for (int q = 0; q < kRT / 8; ++q) {
            const int r = ty + 8 * q;
            const int a = a0 + r, bcol = b0 + tx;
            if (a < nnew && bcol < nnew) st[(size_t)a * LD + bcol] = Nm::f32(sm.tr[k][r][tx]);
          }
        }
        if ((JJ[k] < II[k]) && (st || A.full64)) {
#pragma unroll
          for (int q = 0; q < kRT / 8; ++q) {
            const int bb = b0 + ty + 8 * q, aa = a0 + tx;  // element (aa, bb) written at (bb, aa)
            if (aa < nnew && bb < nnew) {
              const V v = Nm::flip(sm.tr[k][tx][ty + 8 * q], aa - bb);
              if (A.full64) e[(size_t)bb * LD + aa] = v;
              if (st) st[(size_t)bb * LD + aa] = Nm::f32(v);
            }
          }
        }
      }
    }
  }
}

// Delta^0 = [1] (and its FP32 copy); the state is double or float-float (1, 0)
__global__ void k_plane_init(void* S, float* S32, int float_float) {
  if (float_float) static_cast<float2*>(S)[0] = make_float2(1.f, 0.f);
  else static_cast<double*>(S)[0] = 1.0;
  if (S32) S32[0] = 1.0f;
}

// the sweep kernel of a plan's precision: float-float on the mixed paths
const void* sweep_kernel(int prec) {
  return prec == MW_PREC_FP64 ? (const void*)k_risbo_sweep<NumF64> : (const void*)k_risbo_sweep<NumFF>;
}

}  // namespace

namespace {

cudaError_t launch_risbo(mw_plan* p, void* S, int nslot, float* S32, int l0, int full64, int lb, int le,
                         cudaStream_t st, int* nd) {
  if (lb >= le) return cudaSuccess;
  const int Tm = (le + kRT - 1) / kRT;
  k_prog_init<<<8, 256, 0, st>>>(p->d_prog, Tm * (Tm + 1) / 2, lb - 1);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  RisboArgs a;
  a.S = S; a.nslot = nslot; a.S32 = S32; a.l0 = l0; a.full64 = full64; a.LD = p->LD;
  const bool ff = p->prec != MW_PREC_FP64;
  a.sq = ff ? (const void*)p->d_sqrt_ff : (const void*)p->d_sqrt;
  a.rsq = ff ? (const void*)p->d_rsqrt_ff : (const void*)p->d_rsqrt;
  a.rscale = ff ? (const void*)p->d_rscale_ff : (const void*)p->d_rscale;
  a.prog = p->d_prog; a.err = p->d_err;
  a.perm = p->d_perm; a.smid_out = nullptr;
  // Debug knobs, read at every launch (never set in normal use):
  // MW_DEBUG_STALL_PLANE=<l> makes block rank 0 leave before plane l without
  // publishing it, MW_DEBUG_POLLS=<n> shortens every neighbour wait to n polls;
  // together they exercise the timeout path (MW_ETIMEOUT from mw_plan_sync).
  a.polls = kBarrierPolls;
  a.stall_l = -1;
  a.stall_rank = 0;
  if (const char* v = getenv("MW_DEBUG_STALL_PLANE")) a.stall_l = atoi(v);
  if (const char* v = getenv("MW_DEBUG_POLLS")) {
    const long n = atol(v);
    if (n >= 1 && n <= (long)kBarrierPolls) a.polls = (unsigned)n;
  }
  // every block of the persistent sweep must be resident at once (their waits
  // depend on one another): checked before the cooperative launch
  {
    int per_sm = 0, nsm = 0;
    const void* k = sweep_kernel(p->prec);
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kRThreads, (size_t)kRisboSmem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
    if (e != cudaSuccess) return e;
    if ((long)per_sm * nsm < (long)p->risbo_grid) return cudaErrorCooperativeLaunchTooLarge;
  }
  void* args[] = {&a, &lb, &le};
  e = cudaLaunchCooperativeKernel(sweep_kernel(p->prec), dim3(p->risbo_grid), dim3(kRThreads), args,
                                  (size_t)kRisboSmem, st);
  if (nd) *nd += 2;  // the progress reset and the sweep
  return e;
}

// One pass over the planes (Risbo's sweep, or the Trapani-Navaza planes when
// the owner's flags ask for them; recursion state and staging of the owner o)
// feeding the contractions of the jobs: for a regular plan one job on o itself; for a
// ragged plan one per band-limit sub-plan; for a fused forward+inverse call
// the forward jobs and the inverse jobs together.  Plane l serves every job
// with L > l: Delta^l depends on neither L nor s.
cudaError_t run_sweep(mw_plan* o, const WignerJob* jobs, int nj, cudaStream_t st, int* launches,
                      const ChunkHook* hook) {
  const bool fp64 = o->prec == MW_PREC_FP64;
  const int chunk = fp64 ? kChunk : o->chunk;
  for (int c = 0; c < nj; ++c) {  // work lists built for another chunk (after a tuning change)
    mw_plan* q = jobs[c].q;
    if (!fp64 && q->prec == MW_PREC_MIXED_BF16X3 && q->tc2_chunk != chunk) {
      cudaError_t ee = make_tc2_items(q, chunk);
      if (ee != cudaSuccess) return ee;
    }
  }
  int nl = 0;
  cudaError_t e;
  for (int c = 0; c < nj; ++c) {
    if (jobs[c].mode != 1) continue;
    mw_plan* q = jobs[c].q;
    e = cudaMemsetAsync(q->d_Gp, 0, sizeof(double2) * (size_t)q->B * q->M * q->L, st);
    if (e != cudaSuccess) return e;
    if (!fp64 && !jobs[c].chunked_flm) {
      e = (q->prec == MW_PREC_MIXED_BF16X3) ? launch_flm_transpose(q, jobs[c].flm_in, st)
                                            : launch_flm_to_f32(q, jobs[c].flm_in, st);
      if (e != cudaSuccess) return e;
      ++nl;
    }
  }
  k_plane_init<<<1, 1, 0, st>>>(o->d_S, fp64 ? nullptr : o->d_S32, fp64 ? 0 : 1);
  ++nl;
  for (int l0 = 0; l0 < o->L; l0 += chunk) {
    const int l1 = (l0 + chunk < o->L) ? l0 + chunk : o->L;
    StageSpan span_d(o, MW_STAGE_DELTA, st);
    int nd = 0;
    if (o->flags & MW_FLAG_DELTA_TN) {  // Trapani-Navaza: independent planes from their top rows
      e = launch_tn(o, l0, l0, l1, st);
      nd = 1;
    } else {
      e = launch_risbo(o, o->d_S, fp64 ? kChunk : 2, fp64 ? nullptr : o->d_S32, l0, fp64 ? 1 : 0,
                       (l0 == 0 ? 1 : l0), l1, st, &nd);
    }
    if (e != cudaSuccess) return e;
    span_d.end(nd);
    nl += nd;
    if (hook && hook->before) {
      e = hook->before(hook->ctx, l0, l1);
      if (e != cudaSuccess) return e;
    }
    StageSpan span_c(o, MW_STAGE_CONTRACT, st);
    int ncl = 0;
    for (int c = 0; c < nj; ++c) {
      mw_plan* q = jobs[c].q;
      if (q->L <= l0) continue;
      const int l1c = l1 < q->L ? l1 : q->L;
      if (fp64)
        e = (jobs[c].mode == 0) ? launch_dmma_forward(q, l0, l1c, jobs[c].flm_out, st)
                                : launch_dmma_inverse(q, l0, l1c, jobs[c].flm_in, st);
      else if (q->prec == MW_PREC_MIXED_BF16X3)
        e = launch_tc2(q, o, jobs[c].mode, l0, l1c, jobs[c].flm_out, st);
      else
        e = (jobs[c].mode == 0) ? launch_tc_forward(q, l0, l1c, jobs[c].flm_out, st)
                                : launch_tc_inverse(q, l0, l1c, q->d_flmf, st);
      ++ncl;
      if (e != cudaSuccess) return e;
    }
    span_c.end(ncl);
    nl += ncl;
    if (hook && hook->fn) {
      e = hook->fn(hook->ctx, l0, l1);
      if (e != cudaSuccess) return e;
    }
  }
  if (launches) *launches += nl;
  return cudaGetLastError();
}

}  // namespace

// Co-resident blocks per SM of the persistent recursion kernel: the occupancy
// limit, capped by MW_RISBO_BLOCKS_PER_SM (a tuning knob; default 5: with the
// float-float state the sweep is latency-bound, and 5 blocks of 48 registers
// measured 46.1 against 47.6 ms per round trip for 4 blocks of 64).
int risbo_blocks_per_sm(int prec) {
  int n = 0;
  const void* k = sweep_kernel(prec);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, kRisboSmem) != cudaSuccess ||
      cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, kRThreads, kRisboSmem) != cudaSuccess) {
    cudaGetLastError();
    return 1;
  }
  int cap = 5;
  if (const char* env = getenv("MW_RISBO_BLOCKS_PER_SM")) {
    const int v = atoi(env);
    if (v >= 1 && v <= 32) cap = v;
  }
  return n < 1 ? 1 : (n > cap ? cap : n);
}

// Placement-aware block ranks for the sweep of plan p: one empty launch of the
// sweep kernel records the SM of every block; ranks are then dealt round-robin
// over the SMs (rank r < #SM on distinct SMs, and so on).  Correctness does not
// depend on the placement, only the spread of the early, small planes does.
cudaError_t make_risbo_perm(mw_plan* p) {
  const int G = p->risbo_grid;
  int* d_smid = nullptr;
  cudaError_t e = cudaMalloc((void**)&d_smid, sizeof(int) * (size_t)G);
  if (e != cudaSuccess) return e;
  RisboArgs a{};
  a.LD = p->LD;
  a.smid_out = d_smid;
  a.polls = kBarrierPolls;
  a.stall_l = -1;
  int lb = 1, le = 1;  // no planes: the launch only records the placement
  void* args[] = {&a, &lb, &le};
  e = cudaLaunchCooperativeKernel(sweep_kernel(p->prec), dim3(G), dim3(kRThreads), args, (size_t)kRisboSmem, 0);
  std::vector<int> smid(G, 0);
  if (e == cudaSuccess) e = cudaMemcpy(smid.data(), d_smid, sizeof(int) * (size_t)G, cudaMemcpyDeviceToHost);
  cudaFree(d_smid);
  if (e != cudaSuccess) return e;
  // blocks grouped by SM (in order of SM id), dealt one per SM per round
  std::vector<std::pair<int, int>> bys(G);
  for (int b = 0; b < G; ++b) bys[b] = {smid[b], b};
  std::sort(bys.begin(), bys.end());
  std::vector<std::vector<int>> per_sm;
  for (int i = 0; i < G; ++i) {
    if (i == 0 || bys[i].first != bys[i - 1].first) per_sm.emplace_back();
    per_sm.back().push_back(bys[i].second);
  }
  std::vector<int> perm(G, -1);
  int r = 0;
  for (size_t round = 0; r < G; ++round)
    for (auto& v : per_sm)
      if (round < v.size()) perm[v[round]] = r++;
  e = cudaMalloc((void**)&p->d_perm, sizeof(int) * (size_t)G);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_perm, perm.data(), sizeof(int) * (size_t)G, cudaMemcpyHostToDevice);
  return e;
}

cudaError_t run_wigner(mw_plan* o, const WignerJob* jobs, int nj, cudaStream_t st, int* launches,
                       const ChunkHook* hook) {
  return run_sweep(o, jobs, nj, st, launches, hook);
}
