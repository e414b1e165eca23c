// kernels_tc.cu -- split-precision Delta contractions on the tensor cores (tcgen05).
//
// For one tile of 128 consecutive l and one |m| = am, the forward sum of
// Eq. (flm_wig) over m' >= 0 (the +-m' fold is already in G+) is a GEMM
//   out[l, n] = sum_{m'} A[l, m'] B[n, m'],   A[l, m'] = Delta^l_{m',am} Delta^l_{m',-s}
// with n running over (map, re/im) for m = +am and, for m = -am, over the same
// maps with B multiplied by (-1)^{m'} and the result by (-1)^l, because
// Delta_{m',-am} = (-1)^(l+m') Delta_{m',am} (Eq. wignerd_sym2 at pi/2).  So one
// A tile serves both signs of m and N = 4 x (maps of the spin group) <= 32.
// The inverse sum of Eq. (Fmm) is the transposed GEMM, rows m', K = l.
//
// Precision: A and B are formed in FP32 and split into three BF16 parts
// (x = hi + mid + lo); six products hi.hi, hi.mid, mid.hi, hi.lo, mid.mid,
// lo.hi are formed on the tensor cores.  A single K = 16 MMA into a fresh
// accumulator errs by about 2^-24 of the sum of its |products| (measured on
// this part), but every further MMA accumulated into the same FP32 accumulator
// adds an error of that size relative to the growing partial sum.  So the main
// hi.hi product of each K step goes to a fresh TMEM slot of its own, while the
// correction products (2^-8 and 2^-16 smaller) accumulate in two more slots;
// the six slots of a 64-wide K tile are then summed on the CUDA cores in
// float-float (TwoSum) accumulators, which also carry the sum across K tiles,
// and converted to FP64 at the end.
//
// Layout: operands in shared memory in the no-swizzle K-major core-matrix
// layout, written by all threads; thread 0 issues the MMAs and commits them to
// an mbarrier that every thread waits on (bounded; a timeout sets the plan's
// error word and skips the accumulator read); warp w then reads TMEM lanes
// 32w..32w+31 (= rows of the tile).
#include <cmath>

#include "internal.h"
#include "umma.cuh"

namespace {

constexpr int kKTile = 64;            // K per operand tile (4 MMAs of K = 16)
constexpr int kN = 4 * kTcGroupMaps;  // 32 accumulator columns
constexpr int kATile = 128 * kKTile * 2;  // bytes of one bf16 A split (16 KB)
constexpr int kBTile = kN * kKTile * 2;   // bytes of one bf16 B split (4 KB)
constexpr int kSmemUsed = 3 * kATile + 3 * kBTile + 64;
// Requested dynamic shared memory: at least 80 KB so that no more than two
// blocks share an SM, which keeps 2 x kTmemCols <= 512 TMEM columns.
constexpr int kSmem = kSmemUsed > 80 * 1024 ? kSmemUsed : 80 * 1024;
constexpr int kSlots = 4;               // TMEM accumulator slots of kN columns
constexpr uint32_t kTmemCols = 128;     // >= kSlots * kN, power of two
constexpr uint32_t kMaxPolls = 1u << 26;
// split pairs (A part, B part) of the six products, largest first, and the
// TMEM slot each goes to (slot ks/2 for hi.hi of K steps ks, 2 and 3 for the
// two correction classes)
__device__ __forceinline__ int split_a(int p) { return (0x210100 >> (4 * p)) & 0xF; }  // 0,0,1,0,1,2
__device__ __forceinline__ int split_b(int p) { return (0x012010 >> (4 * p)) & 0xF; }  // 0,1,0,2,1,0

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float b) {
  const float s = hi + b;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (b - bb);
  hi = s;
  lo += err;
}

// (h, l) += (bh, bl) in float-float: TwoSum of the high words, then the low
// words and the rounding error, renormalised (Fast2Sum).
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  const float s = h + bh;
  const float bb = s - h;
  const float e = (h - (s - bb)) + (bh - bb);
  const float t = l + bl + e;
  h = s + t;
  l = t - (h - s);
}

// Slot and accumulate flag of split product p in K step ks of a 64-wide K tile:
// the hi.hi products of K steps 2q and 2q+1 go to slot q (fresh at 2q), the
// correction products (2^-8 and 2^-16 smaller) accumulate in slots 2 and 3;
// every slot starts fresh in each tile.
__device__ __forceinline__ int slot_of(int p, int ks) { return (p == 0) ? (ks >> 1) : (p < 3 ? 2 : 3); }
__device__ __forceinline__ int acc_of(int p, int ks) {
  return (p == 0) ? (ks & 1) : ((ks == 0 && (p == 1 || p == 3)) ? 0 : 1);
}

// Issue the 4 K steps x 6 split products of one 64-wide K tile (K-major A).
__device__ __forceinline__ void issue_tile(uint32_t tmem, uint32_t sa, uint32_t sb, uint32_t idesc) {
#pragma unroll
  for (int ks = 0; ks < kKTile / 16; ++ks) {
#pragma unroll
    for (int p = 0; p < 6; ++p) {
      const uint64_t ad = umma::smem_desc(sa + split_a(p) * kATile + ks * 256, 128, (kKTile / 8) * 128);
      const uint64_t bd = umma::smem_desc(sb + split_b(p) * kBTile + ks * 256, 128, (kKTile / 8) * 128);
      umma::mma_bf16(tmem + (uint32_t)(slot_of(p, ks) * kN), ad, bd, idesc, acc_of(p, ks));
    }
  }
}

// Add the four slots into float-float accumulators: warp quadrant q owns TMEM
// lanes (tile rows) 32q..32q+31, half h owns columns 16h..16h+15 of each slot.
// The two hi.hi slots go through TwoSum; the two correction slots (at most
// 2^-8 of the sum) are added to the low word directly, where their own
// rounding is below 2^-32 of the result.  Loads are issued in pairs.
__device__ __forceinline__ void drain_half(uint32_t tmem, int quad, int half, float* hi, float* lo) {
  const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(16 * half);
  uint32_t a[16], b[16];
  umma::ld_32x32b_x16_async(base, a);
  umma::ld_32x32b_x16_async(base + (uint32_t)kN, b);
  umma::wait_ld();
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    two_sum_acc(hi[j], lo[j], __uint_as_float(a[j]));
    two_sum_acc(hi[j], lo[j], __uint_as_float(b[j]));
  }
  umma::ld_32x32b_x16_async(base + (uint32_t)(2 * kN), a);
  umma::ld_32x32b_x16_async(base + (uint32_t)(3 * kN), b);
  umma::wait_ld();
#pragma unroll
  for (int j = 0; j < 16; ++j) lo[j] += __uint_as_float(a[j]) + __uint_as_float(b[j]);
}

__device__ __forceinline__ void sync_all() {
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
}

// Every thread waits (bounded) for the committed MMAs; the result is made
// block-uniform so that the warp-collective TMEM loads are never divergent.
__device__ __forceinline__ bool wait_all(uint64_t* mbar, uint32_t phase) {
  const bool w = umma::mbar_wait(mbar, phase, kMaxPolls);
  umma::fence_before();
  const int all = __syncthreads_and(w ? 1 : 0);
  umma::fence_after();
  return all != 0;
}

constexpr int kThreads = 256;  // 8 warps: warp w drains TMEM lanes 32 (w % 4) .. + 31, columns 16 (w / 4) .. + 15

// 8 FP32 values -> three 16-byte rows of bf16 (hi, mid, lo) at byte offset off
// of each split tile; pairs are converted with one packed round-to-nearest
// conversion each (x ~= hi + mid + lo as in umma::split3, element 2i in the
// low half of word i)
__device__ __forceinline__ void store_split8(unsigned char* base, int tile_bytes, int off, const float* x) {
  uint32_t h[4], m[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 hp = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    const float2 hf = __bfloat1622float2(hp);
    const float r0 = x[2 * i] - hf.x, r1 = x[2 * i + 1] - hf.y;
    const __nv_bfloat162 mp = __floats2bfloat162_rn(r0, r1);
    const float2 mf = __bfloat1622float2(mp);
    const __nv_bfloat162 lp = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
    h[i] = *reinterpret_cast<const uint32_t*>(&hp);
    m[i] = *reinterpret_cast<const uint32_t*>(&mp);
    l[i] = *reinterpret_cast<const uint32_t*>(&lp);
  }
  *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(base + tile_bytes + off) = make_uint4(m[0], m[1], m[2], m[3]);
  *reinterpret_cast<uint4*>(base + 2 * tile_bytes + off) = make_uint4(l[0], l[1], l[2], l[3]);
}

// ---- TF32 x3 variant: x = hi + lo, each a TF32 value (11 significant bits);
// products hi.hi, hi.lo, lo.hi (K = 8 per MMA).  Tiles are K-major with 4
// values per 16-byte core-matrix row.
constexpr int kATile32 = 128 * kKTile * 4;  // bytes of one TF32 A split (32 KB)
constexpr int kBTile32 = kN * kKTile * 4;   // bytes of one TF32 B split (8 KB)
constexpr int kSmem32 = 2 * kATile32 + 2 * kBTile32 + 64;

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// byte offset of element (r, k) of a K-major TF32 tile of kKTile columns
__device__ __forceinline__ int tile_off32(int r, int k) {
  return (r >> 3) * ((kKTile / 4) * 128) + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4;
}
// 4 FP32 values (consecutive K of one row) -> the 16-byte rows of the hi and
// lo tiles at byte offset off
__device__ __forceinline__ void store_split4_tf32(unsigned char* base, int tile_bytes, int off, const float* x) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    h[i] = to_tf32(x[i]);
    l[i] = to_tf32(x[i] - __uint_as_float(h[i]));
  }
  *reinterpret_cast<uint4*>(base + off) = make_uint4(h[0], h[1], h[2], h[3]);
  *reinterpret_cast<uint4*>(base + tile_bytes + off) = make_uint4(l[0], l[1], l[2], l[3]);
}
// 8 consecutive K values of row r starting at k0 (a multiple of 8)
__device__ __forceinline__ void store_split8_tf32(unsigned char* base, int tile_bytes, int r, int k0, const float* x) {
  store_split4_tf32(base, tile_bytes, tile_off32(r, k0), x);
  store_split4_tf32(base, tile_bytes, tile_off32(r, k0 + 4), x + 4);
}
// The 8 K steps x 3 products of one 64-wide K tile: hi.hi of steps 4q..4q+3
// into slot q (fresh at 4q), hi.lo and lo.hi (2^-11 smaller) into slot 2.
__device__ __forceinline__ void issue_tile_tf32(uint32_t tmem, uint32_t sa, uint32_t sb, uint32_t idesc) {
#pragma unroll
  for (int ks = 0; ks < kKTile / 8; ++ks) {
#pragma unroll
    for (int p = 0; p < 3; ++p) {
      const int pa = (p == 2) ? 1 : 0, pb = (p == 1) ? 1 : 0;
      const uint64_t ad = umma::smem_desc(sa + pa * kATile32 + ks * 256, 128, (kKTile / 4) * 128);
      const uint64_t bd = umma::smem_desc(sb + pb * kBTile32 + ks * 256, 128, (kKTile / 4) * 128);
      const int slot = (p == 0) ? (ks >> 2) : 2;
      const int acc = (p == 0) ? ((ks & 3) != 0) : ((ks == 0 && p == 1) ? 0 : 1);
      umma::mma_tf32(tmem + (uint32_t)(slot * kN), ad, bd, idesc, acc);
    }
  }
}
// Drain of the three TF32 slots: two hi.hi slots through TwoSum, the
// correction slot added to the low word.
__device__ __forceinline__ void drain_tf32(uint32_t tmem, int quad, int half, float* hi, float* lo) {
  const uint32_t base = tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)(16 * half);
  uint32_t a[16], b[16], c[16];
  umma::ld_32x32b_x16_async(base, a);
  umma::ld_32x32b_x16_async(base + (uint32_t)kN, b);
  umma::ld_32x32b_x16_async(base + (uint32_t)(2 * kN), c);
  umma::wait_ld();
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    two_sum_acc(hi[j], lo[j], __uint_as_float(a[j]));
    two_sum_acc(hi[j], lo[j], __uint_as_float(b[j]));
    lo[j] += __uint_as_float(c[j]);
  }
}

// 8 consecutive floats from a 32-byte aligned address
__device__ __forceinline__ void load8(const float* __restrict__ p, float* v) {
  const float4 a = __ldg(reinterpret_cast<const float4*>(p));
  const float4 b = __ldg(reinterpret_cast<const float4*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w; v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
}

// Kernel values A = Delta_{m',am} Delta_{m',-s} (sign folded) for 8 consecutive m'
// of plane P; entries with m' > l are zero.
__device__ __forceinline__ void kernel8(const float* __restrict__ P, int LD, int am, int as, int s, int l, int mp,
                                        float* x) {
  float a[8], w[8];
  load8(P + (size_t)am * LD + mp, a);
  load8(P + (size_t)as * LD + mp, w);
  const int base = am + as + (s > 0 ? l + mp : 0);
  const bool alt = s > 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) {
    float v = a[i] * w[i];
    if ((base + (alt ? i : 0)) & 1) v = -v;
    x[i] = (mp + i <= l) ? v : 0.f;
  }
}

// ---------------------------------------------------------------------------
// forward: f_lm for l in [l0, l1), both signs of m = +-am, every spin group
// ---------------------------------------------------------------------------
template <bool TF>
__global__ void __launch_bounds__(kThreads, 2) k_tc_forward(const float* __restrict__ S, int LD, int L, int M, int l0,
                                                         int l1, const SpinGroup* __restrict__ groups, int ng,
                                                         const float2* __restrict__ Gp,
                                                         const double* __restrict__ nltab,
                                                         double2* __restrict__ flm, const long long* __restrict__ foff,
                                                         int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int aT = TF ? kATile32 : kATile, bT = TF ? kBTile32 : kBTile, np = TF ? 2 : 3;
  unsigned char* sA = smem;
  unsigned char* sB = smem + np * aT;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + np * aT + np * bT);
  uint32_t* slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int am = blockIdx.x;
  const int lt0 = l0 + 128 * blockIdx.y;           // rows l of this block: [lt0, lt1)
  const int lt1 = min(l1, lt0 + 128);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, half = warp >> 2;
  if (am >= lt1) return;  // block-uniform: no row l >= |m| here
  if (tid == 0) umma::mbar_init(mbar, 1);
  if (warp == 0) umma::tmem_alloc(slot, kTmemCols);
  sync_all();
  const uint32_t tmem = *slot;
  const uint32_t idesc = TF ? umma::idesc_tf32_f32(128, kN) : umma::idesc_bf16_f32(128, kN);
  const size_t plane = (size_t)LD * LD;
  uint32_t phase = 0;
  bool ok = true;
  const int row = quad * 32 + lane;  // TMEM lane = tile row = l - lt0
  for (int gi = 0; gi < ng; ++gi) {
    const SpinGroup& g = groups[gi];
    const int s = g.s, as = s < 0 ? -s : s, nb = g.nb;
    const int lstart = max(max(lt0, am), as);
    float ahi[16], alo[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) { ahi[j] = 0.f; alo[j] = 0.f; }
    if (lstart < lt1) {
      // Thread tid stages A rows r0 + 32k (k < 4) and B row r0 of 8-column chunk
      // cq: lanes 8q..8q+7 take the 8 rows of one core matrix (each 8-lane
      // phase of the 16-byte stores fills 128 contiguous bytes: no bank
      // conflicts) and the four lane octets of a warp take consecutive chunks
      // (128 contiguous bytes of each plane row).  The next tile's values are
      // gathered into registers while the current tile's MMAs and drain run.
      const int r0 = (tid & 7) + 8 * (tid >> 6), cq = (tid >> 3) & 7;
      float xa[4][8], xb[8];
      auto gather = [&](int mp0) {
        const int mp = mp0 + 8 * cq;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const int l = lt0 + r0 + 32 * k;
          if (l >= lstart && l < lt1 && mp <= l) {
            kernel8(S + (size_t)(l - l0) * plane, LD, am, as, s, l, mp, xa[k]);
          } else {
#pragma unroll
            for (int i = 0; i < 8; ++i) xa[k][i] = 0.f;
          }
        }
        // B row n = r0: (map, re/im) for +am, then the same maps for -am
        const int n = r0, j = n >> 1;
#pragma unroll
        for (int i = 0; i < 8; ++i) xb[i] = 0.f;
        if (j < 2 * nb) {
          const bool neg = j >= nb;
          if (!(neg && am == 0)) {
            const float2* src = Gp + ((size_t)g.maps[neg ? j - nb : j] * M + (neg ? -am : am) + L - 1) * L;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              if (mp + i < L) {
                const float2 v = src[mp + i];
                float y = (n & 1) ? v.y : v.x;
                if (neg && ((mp + i) & 1)) y = -y;
                xb[i] = y;
              }
            }
          }
        }
      };
      gather(0);
      for (int mp0 = 0; mp0 < lt1; mp0 += kKTile) {
        if constexpr (TF) {
#pragma unroll
          for (int k = 0; k < 4; ++k) store_split8_tf32(sA, kATile32, r0 + 32 * k, 8 * cq, xa[k]);
          store_split8_tf32(sB, kBTile32, r0, 8 * cq, xb);
        } else {
#pragma unroll
          for (int k = 0; k < 4; ++k) store_split8(sA, kATile, umma::tile_off(r0 + 32 * k, 8 * cq, kKTile / 8), xa[k]);
          store_split8(sB, kBTile, umma::tile_off(r0, 8 * cq, kKTile / 8), xb);
        }
        umma::fence_proxy_async();
        sync_all();
        if (tid == 0) {
          if constexpr (TF) issue_tile_tf32(tmem, umma::smem_u32(sA), umma::smem_u32(sB), idesc);
          else issue_tile(tmem, umma::smem_u32(sA), umma::smem_u32(sB), idesc);
          umma::commit(mbar);
        }
        if (mp0 + kKTile < lt1) gather(mp0 + kKTile);
        const bool w = wait_all(mbar, phase);
        phase ^= 1u;
        ok = ok && w;
        if (w) {
          if constexpr (TF) drain_tf32(tmem, quad, half, ahi, alo);
          else drain_half(tmem, quad, half, ahi, alo);
        }
        sync_all();
      }
    }
    // epilogue: columns 16*half .. +15 = (map j, re/im) for j = 8*half .. 8*half+7
    const int l = lt0 + row;
    if (l >= am && l < lt1) {
      const double nl = ((s & 1) ? -1.0 : 1.0) * nltab[l];
#pragma unroll
      for (int jj = 0; jj < 8; ++jj) {
        const int j = 8 * half + jj;
        if (j >= 2 * nb) continue;
        const bool neg = j >= nb;
        if (neg && am == 0) continue;
        const int m = neg ? -am : am;
        double2 o = make_double2(0.0, 0.0);
        if (l >= as) {
          double ar = (double)ahi[2 * jj] + (double)alo[2 * jj];
          double ai = (double)ahi[2 * jj + 1] + (double)alo[2 * jj + 1];
          const double sgn = (neg && (l & 1)) ? -nl : nl;
          ar *= sgn;
          ai *= sgn;
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
  if (!ok && tid == 0) atomicExch(err, 1);
  sync_all();
  if (warp == 0) umma::tmem_dealloc(tmem, kTmemCols);
}

// ---------------------------------------------------------------------------
// inverse: F+_{+-am, m'} += sum_{l in [l0,l1)} N_l Delta^l_{m',am} Delta^l_{m',-s} f_{l,+-am}
// one block per (am, 128-row tile of m', spin group).  F+ is kept across chunks
// as float-float pairs (about 48 significant bits): no FP64 arithmetic, which
// runs at 1/64 of the FP32 rate on this part.  The A operand (rows m',
// K = l) is stored MN-major: each 16-byte core-matrix row holds 8 consecutive m'
// of one l, exactly the layout of a plane row.
// ---------------------------------------------------------------------------
constexpr int kMnSbo = 128;                  // stride between 8-m' groups
constexpr int kMnLbo = (128 / 8) * 128;      // stride between 8-l groups (2048)

template <bool TF>
__global__ void __launch_bounds__(kThreads, 2) k_tc_inverse(const float* __restrict__ S, int LD, int L, int M, int l0,
                                                         int l1, const SpinGroup* __restrict__ groups,
                                                         const float2* __restrict__ flmf, double2* __restrict__ Fp,
                                                         int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  constexpr int aT = TF ? kATile32 : kATile, bT = TF ? kBTile32 : kBTile, np = TF ? 2 : 3;
  unsigned char* sA = smem;
  unsigned char* sB = smem + np * aT;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + np * aT + np * bT);
  uint32_t* slot = reinterpret_cast<uint32_t*>(mbar + 1);
  const int am = blockIdx.x, mp0 = blockIdx.y * 128;
  const SpinGroup& g = groups[blockIdx.z];
  const int s = g.s, as = s < 0 ? -s : s, nb = g.nb;
  const int lstart = max(max(l0, am), as);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int quad = warp & 3, half = warp >> 2;
  if (lstart >= l1 || mp0 >= l1) return;  // block-uniform: nothing to add
  if (tid == 0) umma::mbar_init(mbar, 1);
  if (warp == 0) umma::tmem_alloc(slot, kTmemCols);
  sync_all();
  const uint32_t tmem = *slot;
  // BF16: A MN-major (plane rows are contiguous in m'); TF32: A K-major
  const uint32_t idesc = TF ? umma::idesc_tf32_f32(128, kN) : (umma::idesc_bf16_f32(128, kN) | (1u << 15));
  const size_t plane = (size_t)LD * LD;
  uint32_t phase = 0;
  bool ok = true;
  float ahi[16], alo[16];
#pragma unroll
  for (int j = 0; j < 16; ++j) { ahi[j] = 0.f; alo[j] = 0.f; }
  // Thread tid stages A rows k0 + 16q (q < 4; rows are l, columns 8-wide
  // chunks cA of m') and B row n0 of chunk cB.  Lanes 8q..8q+7 take 8
  // consecutive l (one MN-major core matrix: conflict-free 16-byte stores), the
  // lane octets consecutive chunks.  The next tile is gathered into registers
  // while the current tile's MMAs and drain run.
  // (TF32: thread tid stages row m' = mp0 + (tid & 127) of A for the l groups
  // 4 ((tid >> 7) + 2q), q < 8 -- 8 lanes = 8 rows of one K-major core matrix.)
  const int k0 = (tid & 7) + 8 * (tid >> 7), cA = (tid >> 3) & 15;
  const int n0 = (tid & 7) + 8 * (tid >> 6), cB = (tid >> 3) & 7;
  const int mrow = tid & 127, g0 = tid >> 7;
  float xa[4][8], xb[8];
  auto gather = [&](int lb) {
    if constexpr (TF) {
      const int mp = mp0 + mrow;
#pragma unroll
      for (int q = 0; q < 8; ++q) {
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int l = lb + 4 * (g0 + 2 * q) + i;
          float v = 0.f;
          if (l >= lstart && l < l1 && mp <= l && mp < L) {
            const float* P = S + (size_t)(l - l0) * plane;
            v = __ldg(P + (size_t)am * LD + mp) * __ldg(P + (size_t)as * LD + mp);
            if ((am + as + (s > 0 ? l + mp : 0)) & 1) v = -v;
          }
          xa[q >> 1][4 * (q & 1) + i] = v;
        }
      }
    } else {
      const int mp = mp0 + 8 * cA;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int l = lb + k0 + 16 * q;
        if (l >= lstart && l < l1 && mp <= l && mp < L) {
          kernel8(S + (size_t)(l - l0) * plane, LD, am, as, s, l, mp, xa[q]);
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) xa[q][i] = 0.f;
        }
      }
    }
    const int j = n0 >> 1;
#pragma unroll
    for (int i = 0; i < 8; ++i) xb[i] = 0.f;
    if (j < 2 * nb) {
      const bool neg = j >= nb;
      if (!(neg && am == 0)) {
        const int b = g.maps[neg ? j - nb : j];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const int l = lb + 8 * cB + i;
          if (l >= lstart && l < l1) {
            const float2 f = flmf[(size_t)b * L * L + (size_t)l * l + l + (neg ? -am : am)];  // N_l f_lm
            float y = (n0 & 1) ? f.y : f.x;
            if (neg && (l & 1)) y = -y;
            xb[i] = y;
          }
        }
      }
    }
  };
  gather(l0);
  for (int kt = 0; kt * kKTile < l1 - l0; ++kt) {
    const int lb = l0 + kt * kKTile;
    if constexpr (TF) {
#pragma unroll
      for (int q = 0; q < 8; ++q)
        store_split4_tf32(sA, kATile32, tile_off32(mrow, 4 * (g0 + 2 * q)), &xa[q >> 1][4 * (q & 1)]);
      store_split8_tf32(sB, kBTile32, n0, 8 * cB, xb);
    } else {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int k = k0 + 16 * q;
        store_split8(sA, kATile, cA * kMnSbo + (k >> 3) * kMnLbo + (k & 7) * 16, xa[q]);
      }
      store_split8(sB, kBTile, umma::tile_off(n0, 8 * cB, kKTile / 8), xb);
    }
    umma::fence_proxy_async();
    sync_all();
    if (tid == 0 && TF) {
      issue_tile_tf32(tmem, umma::smem_u32(sA), umma::smem_u32(sB), idesc);
      umma::commit(mbar);
    } else if (tid == 0) {
#pragma unroll
      for (int ks = 0; ks < kKTile / 16; ++ks) {
#pragma unroll
        for (int p = 0; p < 6; ++p) {
          const uint64_t ad =
              umma::smem_desc(umma::smem_u32(sA) + split_a(p) * kATile + ks * 2 * kMnLbo, kMnLbo, kMnSbo);
          const uint64_t bd =
              umma::smem_desc(umma::smem_u32(sB) + split_b(p) * kBTile + ks * 256, 128, (kKTile / 8) * 128);
          umma::mma_bf16(tmem + (uint32_t)(slot_of(p, ks) * kN), ad, bd, idesc, acc_of(p, ks));
        }
      }
      umma::commit(mbar);
    }
    if ((kt + 1) * kKTile < l1 - l0) gather(lb + kKTile);
    const bool w = wait_all(mbar, phase);
    phase ^= 1u;
    ok = ok && w;
    if (!ok) break;
    if constexpr (TF) drain_tf32(tmem, quad, half, ahi, alo);
    else drain_half(tmem, quad, half, ahi, alo);
    sync_all();
  }
  // epilogue: add the chunk's sum into the FP64 accumulator F+
  const int mp = mp0 + quad * 32 + lane;
  if (ok && mp < L && mp < l1) {
#pragma unroll
    for (int jj = 0; jj < 8; ++jj) {
      const int j = 8 * half + jj;
      if (j >= 2 * nb) continue;
      const bool neg = j >= nb;
      if (neg && am == 0) continue;
      const int b = g.maps[neg ? j - nb : j];
      float4* dst = reinterpret_cast<float4*>(Fp) + ((size_t)b * M + (neg ? -am : am) + L - 1) * L + mp;
      float rh = ahi[2 * jj], rl = alo[2 * jj], ih = ahi[2 * jj + 1], il = alo[2 * jj + 1];
      if (neg && (mp & 1)) { rh = -rh; rl = -rl; ih = -ih; il = -il; }
      float4 cur = *dst;
      ff_add(cur.x, cur.y, rh, rl);
      ff_add(cur.z, cur.w, ih, il);
      *dst = cur;
    }
  }
  if (!ok && tid == 0) atomicExch(err, 1);
  sync_all();
  if (warp == 0) umma::tmem_dealloc(tmem, kTmemCols);
}

}  // namespace

// N_l f_lm in FP32 for the inverse contraction (one block per (l, map)).
__global__ void k_flm_to_f32(const double2* __restrict__ flm, const long long* __restrict__ foff,
                             float2* __restrict__ out, int L) {
  const int l = blockIdx.x, b = blockIdx.y;
  const float nl = sqrtf((2.f * l + 1.f) / (4.f * 3.14159265358979f));
  const size_t base = (size_t)b * L * L + (size_t)l * l;
  const double2* src = flm + foff[b] + (size_t)l * l;
  for (int i = threadIdx.x; i < 2 * l + 1; i += blockDim.x) {
    const double2 v = src[i];
    out[base + i] = make_float2((float)v.x * nl, (float)v.y * nl);
  }
}

cudaError_t launch_flm_to_f32(const mw_plan* p, const double2* flm, cudaStream_t st) {
  k_flm_to_f32<<<dim3(p->L, p->B), 128, 0, st>>>(flm, p->d_foff, p->d_flmf, p->L);
  return cudaGetLastError();
}

template <bool TF>
cudaError_t tc_forward_t(const mw_plan* p, int l0, int l1, double2* flm, cudaStream_t st) {
  const int sm = TF ? kSmem32 : kSmem;
  cudaError_t e = cudaFuncSetAttribute(k_tc_forward<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  const dim3 grid(l1, (l1 - l0 + 127) / 128);
  k_tc_forward<TF><<<grid, kThreads, sm, st>>>(p->d_S32, p->LD, p->L, p->M, l0, l1, p->d_groups,
                                               (int)p->groups.size(), reinterpret_cast<const float2*>(p->d_Gp),
                                               p->d_nl, flm, p->d_foff, p->d_err);
  return cudaGetLastError();
}

template <bool TF>
cudaError_t tc_inverse_t(const mw_plan* p, int l0, int l1, const float2* flm, cudaStream_t st) {
  const int sm = TF ? kSmem32 : kSmem;
  cudaError_t e = cudaFuncSetAttribute(k_tc_inverse<TF>, cudaFuncAttributeMaxDynamicSharedMemorySize, sm);
  if (e != cudaSuccess) return e;
  const dim3 grid(l1, (l1 + 127) / 128, (unsigned)p->groups.size());
  k_tc_inverse<TF><<<grid, kThreads, sm, st>>>(p->d_S32, p->LD, p->L, p->M, l0, l1, p->d_groups, flm,
                                               reinterpret_cast<double2*>(p->d_Gp), p->d_err);
  return cudaGetLastError();
}

cudaError_t launch_tc_forward(const mw_plan* p, int l0, int l1, double2* flm, cudaStream_t st) {
  return p->prec == MW_PREC_MIXED_TF32X3 ? tc_forward_t<true>(p, l0, l1, flm, st)
                                         : tc_forward_t<false>(p, l0, l1, flm, st);
}

cudaError_t launch_tc_inverse(const mw_plan* p, int l0, int l1, const float2* flm, cudaStream_t st) {
  return p->prec == MW_PREC_MIXED_TF32X3 ? tc_inverse_t<true>(p, l0, l1, flm, st)
                                         : tc_inverse_t<false>(p, l0, l1, flm, st);
}
