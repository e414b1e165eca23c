// kernels_tc2.cu -- the split-BF16 Delta contractions (Eq. flm_wig, Eq. Fmm)
// as a warp-specialised, persistent tcgen05 pipeline.
//
// The sums are the GEMMs of kernels_tc.cu: for one |m| = am and a tile of
// 128 rows (l for the forward, m' for the inverse) and each spin group of up to
// 8 maps, out[row, n] = sum_k A[row, k] B[n, k] with
//   A = Delta^l_{m',am} Delta^l_{m',-s} (sign folded; zero for m' > l),
//   B = G+_{+-am, m'} (forward) or N_l f_{l,+-am} (inverse),
// n = (map, +-m, re/im), N = 32, and one A tile serving both signs of m through
// Delta_{m',-am} = (-1)^(l+m') Delta_{m',am} (Eq. wignerd_sym2 at pi/2).
// Precision is that of kernels_tc.cu: A and B in FP32 split into three BF16
// parts, six products per K = 16 step, the hi.hi product of every 32-wide K
// tile in a fresh accumulator (summed across K tiles in float-float on the
// CUDA cores) and the five correction products in a second one that runs
// over the whole work item.
//
// What is new is the data flow.  Each CTA (one per SM; 16 warps, 17 with two
// groups per pass) walks a list of work items (am, row tile, spin-group slice
// of one or two groups); a work item is a run of 32-wide K tiles, and the K
// tiles of all the CTA's items form one pipelined sequence:
//   8 producer     form A for one row each (TMEM lane = row) from the plane
//   warps          tiles, split it, and store it straight into tensor memory
//                  (tcgen05.st), so the MMAs read only B from shared memory;
//                  they also split B into shared memory;
//   MMA lane       issues the six split products of each K = 16 step
//                  (tcgen05.mma, A from TMEM) and commits a stage's MMAs;
//   TMA lane       loads the FP32 plane tiles of a K tile -- row am and the
//                  spin row |s| of the 128 (forward) or 32 (inverse) planes --
//                  with plain per-CTA TMA (cp.async.bulk.tensor, this GPU's
//                  memory only, no multicast) up to four K tiles ahead;
//   drain warps    read the accumulators (tcgen05.ld), add them into
//                  float-float registers, release the accumulator, and write
//                  the item's outputs after its last K tile.
// With one group per pass the MMA and TMA lanes are lanes of their own (warps
// 8 and 9) and warps 12..15 drain.  With two groups per pass lane 0 of warp 8
// issues both, the MMAs of the next K tile before its warp drains the current
// one with warps 9..15.  A two-group slice whose groups have the same spin (a
// "twin": one batch of more than 8 maps of one spin) has one A for both: the
// producers form it once and each product is one N = 64 MMA over both groups'
// B rows, whose accumulator columns are adjacent; groups whose spins share
// |s| load one spin row.
// Operands and their accumulators run in kS stages (4 with one spin group per
// pass, 2 with two); stages are handed over with
// mbarriers: TMA bytes -> producers -> MMA -> (producers, drain) -> MMA.  A
// waiting thread is suspended in mbarrier.try_wait rather than spinning.
// Every wait is bounded (2 s of wall clock): a wait that gives up records the
// timeout in the plan's error word, raises the CTA's abort flag (which the
// other roles poll) and the CTA leaves after its MMAs and TMA loads have
// landed and the TMEM is released; the outputs of such a call are invalid.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <type_traits>
#include <vector>

#include "internal.h"
#include "umma.cuh"

namespace {

constexpr int kKT = 32;                    // K per tile (two K = 16 MMA steps)
constexpr int kRows = 128;                 // rows of a tile (TMEM lanes)
constexpr int kN = 32;                     // accumulator columns per spin group
constexpr int kTmaTile = 16384;            // one FP32 plane tile: 128 x 32 or 32 x 128 floats
constexpr int kBTile = kN * kKT * 2;       // one BF16 split of B (2 KB)
constexpr uint32_t kPolls = 1u << 24;
constexpr uint32_t kWaitNs = 2000000000u;  // 2 s: a healthy wait ends within microseconds

template <int NG>
struct Layout {
  // warps: 8 producers, then (NG = 1) the MMA and TMA lanes' warps, two idle
  // warps and 4 drain warps, or (NG = 2) 8 drain warps and one control warp
  static constexpr int kWarps = NG == 2 ? 17 : 16;
  static constexpr int kThreads = 32 * kWarps;
  static constexpr int kTS = NG == 2 ? 3 : 4;                        // TMA stages (plane tiles in flight)
  // operand + accumulator stages (A in TMEM, B in smem, the accumulators they
  // feed): with one spin group per pass, 4 fill the 512 TMEM columns (448 used)
  // and let the producers, the MMA lane and the drain run up to 4 K tiles apart
  // (27.1 ms per round trip at L = 2048, B = 16, against 28.8 with 2 stages and
  // 28.3 with 3); two groups per pass have room for 2
  static constexpr int kS = NG == 2 ? 2 : 4;
  static constexpr int kTmaStage = (1 + NG) * kTmaTile;             // row am + one spin row per group
  // B of a stage: split p of group g at (p * NG + g) * kBTile, so that the
  // groups' tiles of one split are consecutive 32-row blocks of one 64-row
  // operand (the twin pass below reads them with one N = 64 MMA)
  static constexpr int kBStage = NG * 3 * kBTile;
  static constexpr int kTmaOff = 0;                                  // 1024-aligned
  static constexpr int kBOff = kTS * kTmaStage;
  static constexpr int kEpiOff = kBOff + kS * kBStage;              // epilogue staging of one group
  static constexpr int kEpiBytes = 32 * 256 * 4;                     // 32 values x 256 drain threads
  static constexpr int kBarOff = kEpiOff + kEpiBytes;
  static constexpr int kBytes = kBarOff + 256;
  static constexpr int kSmem = kBytes + 1024;                        // slack for the manual alignment
  // TMEM columns: accumulators (hi, corr) per stage and group, then A per
  // stage, group, K step and split (8 columns = 16 bf16 of K each)
  // hi.hi accumulator per stage and group; correction accumulator per item
  // (kS of them in rotation) and group: it collects the five correction
  // products of every K tile of an item and is read once, at the item's last
  // K tile
  static constexpr int kAccCols = 2 * kS * NG * 32;
  static constexpr int kCols = kAccCols + kS * NG * 2 * 3 * 8;
  static constexpr uint32_t kAlloc = kCols <= 256 ? 256u : 512u;
  static_assert(kCols <= 512, "TMEM budget");
  static_assert(kSmem <= 227 * 1024, "shared memory budget");
  __device__ static uint32_t acc_hi(int a, int g) { return (uint32_t)((a * NG + g) * 32); }
  // the correction accumulator of item k is reused by item k + kS, whose
  // first MMAs wait (accempty) for the drain of a position at least kS
  // positions after item k's last one (every item has a K tile), which reads it
  __device__ static uint32_t acc_corr(int ic, int g) { return (uint32_t)((kS * NG + ic * NG + g) * 32); }
  __device__ static uint32_t a_col(int s, int g, int ks, int sp) {
    return (uint32_t)(kAccCols + ((s * NG + g) * 2 + ks) * 24 + sp * 8);
  }
};

struct Tc2Args {
  int L, M, l0, l1c, LD;
  const int4* items;  // (am, row-tile start, group slice, K tiles)
  int nitems;
  const SpinGroup* groups;
  int ng;
  const float2* bsrc;         // forward: G+ [B][M][L]; inverse: N_l f_lm transposed, [B][M][L]
  const double* nl;           // forward: sqrt((2l+1)/(4 pi))
  double2* flm;               // forward output
  const long long* foff;
  double2* Fp;                // inverse: float-float F+ accumulator
  int* err;
};

// ---- small PTX helpers --------------------------------------------------
// One test of an mbarrier phase; a thread whose phase is not complete is
// suspended (up to the hint, in ns) until it completes, so waiting warps do not
// take issue slots from the working ones.
__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(umma::smem_u32(bar)), "r"(parity), "r"(200000u)
      : "memory");
  return done != 0;
}
// Low 32 bits of the global nanosecond timer; differences are taken modulo
// 2^32, which is exact for waits shorter than 4.29 s.
__device__ __forceinline__ uint32_t now_ns() {
  uint32_t t;
  asm volatile("mov.u32 %0, %%globaltimer_lo;" : "=r"(t));
  return t;
}
// Bounded wait that ignores the abort flag (the abort path's own waits).
__device__ __forceinline__ bool wait_bar_all(uint64_t* bar, uint32_t parity) {
  const uint32_t t0 = now_ns();
  for (uint32_t it = 0; it < kPolls; ++it) {
    if (try_wait(bar, parity)) return true;
    if (now_ns() - t0 > kWaitNs) return false;
  }
  return false;
}
// Bounded wait (kWaitNs of wall clock, at most kPolls tests) that also gives up
// once another role has raised the abort flag.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  if (try_wait(bar, parity)) return true;
  const uint32_t t0 = now_ns();
  for (uint32_t it = 1; it < kPolls; ++it) {
    if (try_wait(bar, parity)) return true;
    if ((it & 63u) == 0u && (*abort_flag || now_ns() - t0 > kWaitNs)) return false;
  }
  return false;
}
__device__ __forceinline__ void arrive(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(umma::smem_u32(bar)) : "memory");
}
__device__ __forceinline__ void arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(umma::smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int x, int y, int z, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], "
      "[%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(z), "r"(umma::smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ void mma_ta(uint32_t d, uint32_t a_tmem, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\ntcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n}\n" ::"r"(d),
      "r"(a_tmem), "l"(bdesc), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void tmem_st8(uint32_t taddr, const uint32_t* r) {
  asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};" ::"r"(taddr), "r"(r[0]),
               "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
               : "memory");
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, uint32_t* r) {
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void two_sum_acc(float& hi, float& lo, float b) {
  const float s = __fadd_rn(hi, b);
  const float bb = __fsub_rn(s, hi);
  const float e = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bb)), __fsub_rn(b, bb));
  hi = s;
  lo = __fadd_rn(lo, e);
}
// (h, l) += (bh, bl) in float-float
__device__ __forceinline__ void ff_add(float& h, float& l, float bh, float bl) {
  const float s = __fadd_rn(h, bh);
  const float bb = __fsub_rn(s, h);
  const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(s, bb)), __fsub_rn(bh, bb));
  const float t = __fadd_rn(__fadd_rn(l, bl), e);
  h = __fadd_rn(s, t);
  l = __fsub_rn(t, __fsub_rn(h, s));
}

// x (two values) -> bf16 pairs hi, mid, lo with x = hi + mid + lo exactly.
// Each part is rounded to the nearest bf16 on the integer pipe -- half a bf16
// ulp added to the bit pattern, the low 16 bits cleared -- so that hi and mid
// are within half an ulp (ties away from zero), the remainders are exact and
// lo, at most 8 significant bits, is exact as a bf16; the pairs are packed
// (first value in the low half) by byte permutes.
__device__ __forceinline__ uint32_t bf16_bits_rn(float x) { return (__float_as_uint(x) + 0x8000u) & 0xffff0000u; }
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t& h, uint32_t& m, uint32_t& l) {
  const uint32_t h0 = bf16_bits_rn(x0), h1 = bf16_bits_rn(x1);
  const float r0 = __fsub_rn(x0, __uint_as_float(h0)), r1 = __fsub_rn(x1, __uint_as_float(h1));
  const uint32_t m0 = bf16_bits_rn(r0), m1 = bf16_bits_rn(r1);
  const float l0 = __fsub_rn(r0, __uint_as_float(m0)), l1 = __fsub_rn(r1, __uint_as_float(m1));
  h = __byte_perm(h0, h1, 0x7632);
  m = __byte_perm(m0, m1, 0x7632);
  l = __byte_perm(__float_as_uint(l0), __float_as_uint(l1), 0x7632);
}
// split parts p of the six products, largest first: (A part, B part)
__device__ __forceinline__ int split_a(int p) { return (0x210100 >> (4 * p)) & 0xF; }  // 0,0,1,0,1,2
__device__ __forceinline__ int split_b(int p) { return (0x012010 >> (4 * p)) & 0xF; }  // 0,1,0,2,1,0

// One work item of the sequence, decoded the same way by every role.
struct Item {
  int am, t0, gs, nk;   // |m|, first row (l or m'), group slice, K tiles
  int kstart;           // first K index (m' = 0 forward; first l inverse)
};
template <int DIR>
__device__ __forceinline__ Item item_of(const Tc2Args& A, int it) {
  const int4 v = A.items[it];
  Item x;
  x.am = v.x; x.t0 = v.y; x.gs = v.z; x.nk = v.w;
  x.kstart = DIR == 0 ? 0 : max(max(A.l0, x.am), x.t0);
  return x;
}

template <int DIR, int NG>
__global__ void __launch_bounds__(Layout<NG>::kThreads, 1) k_tc2(const __grid_constant__ CUtensorMap tmap, Tc2Args A) {
  using Ly = Layout<NG>;
  constexpr int kTS = Ly::kTS;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = umma::smem_u32(smem_raw);
  unsigned char* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Ly::kBarOff);
  constexpr int kS = Ly::kS;
  uint64_t* tma_full = bar;                  // [kTS] TMA bytes of a plane-tile stage arrived
  uint64_t* full = bar + kTS;                // [kS] producers wrote A (TMEM) and B (smem) of a stage
  uint64_t* done = bar + kTS + kS;           // [kS] the MMAs of a stage completed
  uint64_t* accempty = bar + kTS + 2 * kS;   // [kS] the drain read a stage's accumulators
  uint64_t* fin = bar + kTS + 3 * kS;        // final MMA completion on the abort path
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + kTS + 3 * kS + 1);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + kTS + 3 * kS + 2);
  uint64_t* tma_empty = bar + kTS + 3 * kS + 3;  // [kTS] producers read a plane-tile stage (split roles)
  static_assert((2 * kTS + 3 * kS + 3) * 8 <= 256, "barrier area");
  // Roles of the warps after the producers.  One spin group per pass
  // (NG = 1): lane 0 of warp 8 issues the MMAs, lane 0 of warp 9 the TMA
  // loads (refilling a stage once the producers report it read), and warps
  // 12..15 drain all 32 accumulator columns of their lane quarter.  Two groups
  // (NG = 2, whose float-float accumulators would not fit 4 drain warps'
  // registers): warps 8..15 drain, each 16 columns of each group in its lane
  // quarter, and lane 0 of warp 16 issues the MMAs and refills a TMA stage
  // once the MMAs of the position that read it have their operands.
  constexpr bool kSplit = NG == 1;
  constexpr int kCH = kSplit ? 4 : 2;        // 8-column accumulator chunks per drain thread
  constexpr int kDT = kSplit ? 128 : 256;    // drain threads
  constexpr int kPairs = 4 * kCH;            // (map, sign) columns per drain thread
  // the epilogue's output loops: fully unrolled with one group per pass; with
  // two, whose second group's sums are live during the first one's epilogue
  // (at 96 registers a thread), partly rolled, which spills less (24.5
  // against 25.3 ms per round trip at L = 2048, B = 16)
  constexpr int kUnrollFwd = NG == 2 ? 2 : kPairs;
  constexpr int kUnrollInv = NG == 2 ? 1 : kPairs / 4;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  if (tid == 0) {
    for (int t = 0; t < kTS; ++t) umma::mbar_init(&tma_full[t], 1);
    for (int t = 0; t < kTS; ++t) umma::mbar_init(&tma_empty[t], 8);
    for (int s = 0; s < kS; ++s) {
      umma::mbar_init(&full[s], 8);
      umma::mbar_init(&done[s], 1);
      umma::mbar_init(&accempty[s], kDT / 32);  // one arrival per drain warp
    }
    umma::mbar_init(fin, 1);
    *abort_flag = 0;
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(&tmap)) : "memory");
  }
  if (warp == 0) umma::tmem_alloc(tslot, Ly::kAlloc);
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t tma_base = umma::smem_u32(smem + Ly::kTmaOff);
  const uint32_t b_base = umma::smem_u32(smem + Ly::kBOff);
  auto fail = [&]() {
    *abort_flag = 1;
    atomicOr(A.err, 1);
  };

  if (warp < 8) {
    // ----------------------------------------------------------- producers
    const int ks = warp >> 2, qd = warp & 3;
    const int r = 32 * qd + lane;                       // tile row = TMEM lane
    const uint32_t lane_addr = (uint32_t)(32 * qd) << 16;
    // B unit of this thread: group bg, row n, kBV consecutive K of the 32-wide
    // tile (NG = 2: 8 K, 128 threads per group; NG = 1: 4 K, all 256 threads)
    constexpr int kBV = NG == 1 ? 4 : 8;
    const int pt = warp * 32 + lane;
    const int bg = NG == 1 ? 0 : pt >> 7;
    const int bn = NG == 1 ? (pt >> 3) & 31 : (pt >> 2) & 31;
    const int bk0 = NG == 1 ? 4 * (pt & 7) : 8 * (pt & 3);
    // B cursor, two positions ahead of the A position: kBV consecutive K of
    // row bn of group bg; the item's row pointer and signs are decoded once per item
    struct BPos {
      int it, kt, nk, k0;
      const float2* row;
      bool valid, neg;
    } P;
    const int kend = DIR == 0 ? A.L : A.l1c;
    auto load_bpos = [&](int it) {
      P.it = it;
      P.kt = 0;
      P.valid = false;
      if (it >= A.nitems) return;
      const Item x = item_of<DIR>(A, it);
      P.nk = x.nk;
      P.k0 = x.kstart + bk0;  // m' (forward) or l (inverse)
      const int gidx = x.gs * NG + bg;
      if (bg >= NG || gidx >= A.ng) return;
      const SpinGroup& g = A.groups[gidx];
      const int j = bn >> 1, nb = g.nb;
      if (j >= 2 * nb) return;
      P.neg = j >= nb;
      if (P.neg && x.am == 0) return;
      const int map = g.maps[P.neg ? j - nb : j];
      P.row = A.bsrc + ((size_t)map * A.M + (P.neg ? -x.am : x.am) + A.L - 1) * A.L;
      P.valid = true;
    };
    // The loads only: each value is the re or im word of a G+ / N_l f_lm
    // entry, read straight into the buffer (a predicated load leaves 0 past
    // the end), and the (-1)^k of the -am fold is recorded as a sign mask, so
    // no instruction waits for the data until the buffer is stored two
    // positions later.
    auto load_b = [&](float (&v)[kBV], uint32_t& sgn) {
#pragma unroll
      for (int i = 0; i < kBV; ++i) v[i] = 0.f;
      sgn = 0u;
      if (P.it >= A.nitems) return;
      if (P.valid) {
        const int k0 = P.k0 + kKT * P.kt;
        const float* src = reinterpret_cast<const float*>(P.row + k0) + (bn & 1);
#pragma unroll
        for (int i = 0; i < kBV; ++i)
          if (k0 + i < kend) v[i] = __ldg(src + 2 * i);
        // (-1)^m' (forward) or (-1)^l (inverse) of the -am fold: odd k negated
        if (P.neg) sgn = ((k0 & 1) ? 0x55u : 0xAAu) & ((1u << kBV) - 1u);  // bit i set: entry k0 + i is odd
      }
      if (++P.kt >= P.nk) load_bpos(P.it + G);
    };
    // the A position (item, K tile) and the item's spins
    int it = blockIdx.x, kt = 0, q = 0;
    Item x{};
    int ngl = 0, spin[NG];
    bool twin = false, row1 = true;  // (NG = 2) groups of one spin; one spin row in the stage
    auto load_item = [&]() {
      if (it >= A.nitems) return;
      x = item_of<DIR>(A, it);
      ngl = min(NG, A.ng - x.gs * NG);
#pragma unroll
      for (int g = 0; g < NG; ++g) spin[g] = g < ngl ? A.groups[x.gs * NG + g].s : 0;
      if constexpr (NG == 2) {
        twin = ngl == 2 && spin[0] == spin[1];
        row1 = ngl < 2 || abs(spin[0]) == abs(spin[1]);
      }
    };
    load_item();
    float b0[kBV], b1[kBV];
    uint32_t sg0, sg1;
    load_bpos(blockIdx.x);
    load_b(b0, sg0);
    load_b(b1, sg1);
    // One position: B of this position (loaded two positions ago) into
    // operand stage s, the B loads of the position two ahead, then A from the
    // plane tiles of TMA stage q % kTS into tensor memory.
    auto body = [&](float (&cur)[kBV], uint32_t& csg) -> bool {
      if (it >= A.nitems) return false;
      const int s = q % kS, ts = q % kTS;
      const uint32_t ph = (uint32_t)(q / kS) & 1u, tph = (uint32_t)(q / kTS) & 1u;
      // every lane waits; the outcome is made warp-uniform so that the
      // warp-collective TMEM stores and __syncwarp below never diverge
      const bool w = (q < kS || wait_bar(&done[s], ph ^ 1u, abort_flag)) && wait_bar(&tma_full[ts], tph, abort_flag);
      if (!__all_sync(0xffffffffu, w)) {
        if (lane == 0) fail();
        return false;
      }
      umma::fence_after();
      if (bg < NG) {
        uint32_t h[kBV / 2], m[kBV / 2], l[kBV / 2];
#pragma unroll
        for (int i = 0; i < kBV; ++i) cur[i] = __uint_as_float(__float_as_uint(cur[i]) ^ (((csg >> i) & 1u) << 31));
#pragma unroll
        for (int i = 0; i < kBV / 2; ++i) split_pair(cur[2 * i], cur[2 * i + 1], h[i], m[i], l[i]);
        unsigned char* sb = smem + Ly::kBOff + s * Ly::kBStage + bg * kBTile;
        constexpr int kSp = NG * kBTile;  // split stride
        const int off = umma::tile_off(bn, bk0, kKT / 8);
        if constexpr (kBV == 8) {
          *reinterpret_cast<uint4*>(sb + off) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>(sb + kSp + off) = make_uint4(m[0], m[1], m[2], m[3]);
          *reinterpret_cast<uint4*>(sb + 2 * kSp + off) = make_uint4(l[0], l[1], l[2], l[3]);
        } else {
          *reinterpret_cast<uint2*>(sb + off) = make_uint2(h[0], h[1]);
          *reinterpret_cast<uint2*>(sb + kSp + off) = make_uint2(m[0], m[1]);
          *reinterpret_cast<uint2*>(sb + 2 * kSp + off) = make_uint2(l[0], l[1]);
        }
      }
      load_b(cur, csg);
      const float* T = reinterpret_cast<const float*>(smem + Ly::kTmaOff + ts * Ly::kTmaStage);
      // row am of the planes (shared by the groups)
      float a[16];
      if (DIR == 0) {
        // forward: tile [128 planes][32 m'] with the 128-byte swizzle (16-byte
        // chunk c of row r stored at chunk c ^ (r & 7))
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const float4 v = *reinterpret_cast<const float4*>(T + r * 32 + (((4 * ks + c) ^ (r & 7)) << 2));
          a[4 * c] = v.x; a[4 * c + 1] = v.y; a[4 * c + 2] = v.z; a[4 * c + 3] = v.w;
        }
      } else {
        // inverse: tile [32 planes][128 m'], row-major
#pragma unroll
        for (int i = 0; i < 16; ++i) a[i] = T[(16 * ks + i) * 128 + r];
      }
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        if (g == 1 && twin) continue;  // the twin pass reads group 0's A for both groups
        const float* W = T + (1 + (row1 ? 0 : g)) * (kTmaTile / 4);
        uint32_t hp[8], mp[8], lp[8];
        if (g < ngl) {
          const int sv = spin[g], as = sv < 0 ? -sv : sv;
          if (DIR == 0) {
            const int l = x.t0 + r, mp0 = kKT * kt + 16 * ks;
            const bool row_ok = l >= x.am && l < A.l1c && l >= as;
            // sign (-1)^(am + as) (-1)^(l + m') [s > 0]; m' parity alternates along the row
            const float s0 = (((x.am + as + (sv > 0 ? l + mp0 : 0)) & 1) ? -1.f : 1.f);
            const float s1 = sv > 0 ? -s0 : s0;
            const int lim = row_ok ? l - mp0 : -1;  // entries i <= lim are inside the plane
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              const float4 v = *reinterpret_cast<const float4*>(W + r * 32 + (((4 * ks + c) ^ (r & 7)) << 2));
              float x0 = a[4 * c] * v.x * s0, x1 = a[4 * c + 1] * v.y * s1;
              float x2 = a[4 * c + 2] * v.z * s0, x3 = a[4 * c + 3] * v.w * s1;
              if (lim < 15) {  // the K step crosses the edge of the plane
                if (4 * c > lim) x0 = 0.f;
                if (4 * c + 1 > lim) x1 = 0.f;
                if (4 * c + 2 > lim) x2 = 0.f;
                if (4 * c + 3 > lim) x3 = 0.f;
              }
              split_pair(x0, x1, hp[2 * c], mp[2 * c], lp[2 * c]);
              split_pair(x2, x3, hp[2 * c + 1], mp[2 * c + 1], lp[2 * c + 1]);
            }
          } else {
            const int mpr = x.t0 + r, lb = x.kstart + kKT * kt + 16 * ks;
            const float s0 = (((x.am + as + (sv > 0 ? lb + mpr : 0)) & 1) ? -1.f : 1.f);
            const float s1 = sv > 0 ? -s0 : s0;
            const int lo_i = max(max(mpr, as) - lb, 0), hi_i = A.l1c - lb;  // valid i in [lo_i, hi_i)
#pragma unroll
            for (int i = 0; i < 8; ++i) {
              float x0 = a[2 * i] * W[(16 * ks + 2 * i) * 128 + r] * s0;
              float x1 = a[2 * i + 1] * W[(16 * ks + 2 * i + 1) * 128 + r] * s1;
              if (lo_i > 0 || hi_i < 16) {  // the K step crosses an edge
                if (2 * i < lo_i || 2 * i >= hi_i) x0 = 0.f;
                if (2 * i + 1 < lo_i || 2 * i + 1 >= hi_i) x1 = 0.f;
              }
              split_pair(x0, x1, hp[i], mp[i], lp[i]);
            }
          }
        } else {
#pragma unroll
          for (int i = 0; i < 8; ++i) hp[i] = mp[i] = lp[i] = 0u;
        }
        tmem_st8(tmem + lane_addr + Ly::a_col(s, g, ks, 0), hp);
        tmem_st8(tmem + lane_addr + Ly::a_col(s, g, ks, 1), mp);
        tmem_st8(tmem + lane_addr + Ly::a_col(s, g, ks, 2), lp);
      }
      tmem_wait_st();
      umma::fence_proxy_async();
      umma::fence_before();
      __syncwarp();
      if (lane == 0) {
        arrive(&full[s]);
        if (kSplit) arrive(&tma_empty[ts]);  // T and W of this stage are no longer read
      }
      ++q;
      if (++kt >= x.nk) {
        kt = 0;
        it += G;
        load_item();
      }
      return true;
    };
    // two copies of the body, so that the B buffers alternate without moves
    while (body(b0, sg0) && body(b1, sg1)) {
    }
  } else {
    // ------------------------------------------------- control and drain
    // The MMA lane and the TMA lane (one lane for both with NG = 2) never
    // wait for a drain other than through the accempty barriers.
    const int qd = warp & 3;
    const int half = kSplit ? 0 : (warp - 8) >> 2;
    const int dt = tid - (kSplit ? 12 : 8) * 32;  // drain thread index
    const bool drainer = kSplit ? warp >= 12 : warp < 16;
    const uint32_t lane_addr = (uint32_t)(32 * qd) << 16;
    const bool ctl = lane == 0 && warp == (kSplit ? 8 : 16);  // issues the MMAs (and, NG = 2, the TMA loads)
    const bool tma_thr = kSplit ? (warp == 9 && lane == 0) : ctl;
    struct TmaPos {
      int it, kt, nk, am, t0, kstart, nsr;
      int asr[NG];
    } P;  // TMA cursor (kTS positions ahead of the MMA cursor); nsr spin rows per stage
    struct MmaPos {
      int it, kt, nk, ngl, ip;
      bool twin;
    } Qm{};  // MMA cursor (ip: the item's correction accumulator, items in rotation)
    int n_tma = 0;  // TMA loads issued (stage t took those with index % kTS == t)
    int qm = 0;  // MMA position
    bool cok = true;
    auto load_pos = [&](int itp) {
      P.it = itp;
      P.kt = 0;
      if (itp >= A.nitems) return;
      const Item y = item_of<DIR>(A, itp);
      P.nk = y.nk; P.am = y.am; P.t0 = y.t0; P.kstart = y.kstart;
      const int ngl = min(NG, A.ng - y.gs * NG);
#pragma unroll
      for (int g = 0; g < NG; ++g) {
        const int sg = A.groups[y.gs * NG + min(g, ngl - 1)].s;
        P.asr[g] = sg < 0 ? -sg : sg;
      }
      // groups whose spins share |s| (and a slice of one group) read one spin row
      P.nsr = (NG == 2 && P.asr[0] == P.asr[NG - 1]) ? 1 : NG;
    };
    auto issue_tma = [&](int t) {
      arrive_expect_tx(&tma_full[t], (uint32_t)((1 + P.nsr) * kTmaTile));
      const uint32_t dst = tma_base + (uint32_t)(t * Ly::kTmaStage);
      int xx, zz;
      if (DIR == 0) { xx = kKT * P.kt; zz = P.t0 - A.l0; }               // 32 m' of 128 planes
      else { xx = P.t0; zz = P.kstart + kKT * P.kt - A.l0; }             // 128 m' of 32 planes
      tma_load_3d(dst, &tmap, xx, P.am, zz, &tma_full[t]);
#pragma unroll
      for (int g = 0; g < NG; ++g)
        if (g < P.nsr) tma_load_3d(dst + (uint32_t)((1 + g) * kTmaTile), &tmap, xx, P.asr[g], zz, &tma_full[t]);
      ++n_tma;
      if (++P.kt >= P.nk) load_pos(P.it + G);
    };
    auto load_mpos = [&](int itp) {
      Qm.ip = itp == (int)blockIdx.x ? 0 : (Qm.ip + 1 == kS ? 0 : Qm.ip + 1);
      Qm.it = itp;
      Qm.kt = 0;
      if (itp >= A.nitems) return;
      const int4 v = A.items[itp];
      Qm.nk = v.w;
      Qm.ngl = min(NG, A.ng - v.z * NG);
      Qm.twin = NG == 2 && Qm.ngl == 2 && A.groups[v.z * NG].s == A.groups[v.z * NG + NG - 1].s;
    };
    const uint32_t idesc = umma::idesc_bf16_f32(kRows, kN);
    const uint32_t idesc2 = umma::idesc_bf16_f32(kRows, 2 * kN);  // both groups of a twin pass
    const uint64_t bdesc0 = umma::smem_desc(b_base, 128, (kKT / 8) * 128);
    // MMAs of the MMA cursor's position, then the TMA kTS positions ahead
    auto mma_step = [&]() {
      if (!cok || Qm.it >= A.nitems) return;
      const int st = qm % kS;
      const uint32_t ph = (uint32_t)(qm / kS) & 1u;
      if (!wait_bar(&full[st], ph, abort_flag) || (qm >= kS && !wait_bar(&accempty[st], ph ^ 1u, abort_flag))) {
        fail();
        cok = false;
        return;
      }
      umma::fence_after();
      // descriptor start-address fields advance by offset / 16 (no carry below
      // 256 KB); TMEM addresses are constant offsets from the stage's bases.
      // Consecutive MMAs go to different accumulators (the groups' hi and
      // correction slots), so that accumulation chains overlap in the pipe.
      const uint64_t bd_s = bdesc0 + (uint64_t)((st * Ly::kBStage) >> 4);
      const uint32_t acc_s = tmem + Ly::acc_hi(st, 0), corr_s = tmem + Ly::acc_corr(Qm.ip, 0);
      const uint32_t a_s = tmem + Ly::a_col(st, 0, 0, 0);
      const bool first = Qm.kt == 0;  // the item's first K tile starts its correction accumulator
      // NGC groups of N = 32 with their own A; a twin pass (two groups of one
      // spin, so one A) as one N = 64 MMA per product over both groups' B
      // rows and accumulator columns, which are adjacent
      auto issue = [&](auto ngc, uint32_t id) {
        constexpr int NGC = decltype(ngc)::value;
#pragma unroll
        for (int k2 = 0; k2 < 2; ++k2)
#pragma unroll
          for (int p = 0; p < 6; ++p)
#pragma unroll
            for (int g = 0; g < NGC; ++g)
              mma_ta((p == 0 ? acc_s : corr_s) + (uint32_t)(g * 32),
                     a_s + (uint32_t)((g * 2 + k2) * 24 + split_a(p) * 8),
                     bd_s + (uint64_t)((((split_b(p) * NG + g) * kBTile) + k2 * 256) >> 4), id,
                     (p == 0) ? (k2 > 0) : !(first && k2 == 0 && p == 1));
      };
      if (NG == 2 && Qm.twin) issue(std::integral_constant<int, 1>{}, idesc2);
      else if (NG == 2 && Qm.ngl == 2) issue(std::integral_constant<int, NG>{}, idesc);
      else issue(std::integral_constant<int, 1>{}, idesc);
      umma::commit(&done[st]);
      // the plane tiles of this position were read (full was observed): refill
      if (!kSplit && P.it < A.nitems) issue_tma(qm % kTS);
      ++qm;
      if (++Qm.kt >= Qm.nk) load_mpos(Qm.it + G);
    };
    if (tma_thr) {
      load_pos(blockIdx.x);
      for (int t = 0; t < kTS && P.it < A.nitems; ++t) issue_tma(t);
    }
    if (ctl) {
      load_mpos(blockIdx.x);
      while (cok && Qm.it < A.nitems) mma_step();
    } else if (kSplit && tma_thr) {
      // refill the stage of position qt with position qt + kTS once the
      // producers have read it
      for (int qt = 0; P.it < A.nitems; ++qt) {
        const int t = qt % kTS;
        if (!wait_bar(&tma_empty[t], (uint32_t)(qt / kTS) & 1u, abort_flag)) {
          fail();
          break;
        }
        issue_tma(t);
      }
    }
    __syncwarp();
    float hi[NG][8 * kCH], lo[NG][8 * kCH];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int j = 0; j < 8 * kCH; ++j) hi[g][j] = lo[g][j] = 0.f;
    int q = 0, ipd = 0;  // ipd: correction accumulator of the drained item
    bool ok = drainer;
    for (int it = blockIdx.x; ok && it < A.nitems; it += G, ipd = (ipd + 1 == kS ? 0 : ipd + 1)) {
      const Item x = item_of<DIR>(A, it);
      const int ngl = min(NG, A.ng - x.gs * NG);
      for (int kt = 0; kt < x.nk; ++kt, ++q) {
        const int s = q % kS;
        const uint32_t ph = (uint32_t)(q / kS) & 1u;
        if (!__all_sync(0xffffffffu, wait_bar(&done[s], ph, abort_flag))) {
          if (lane == 0) fail();
          ok = false;
          break;
        }
        umma::fence_after();
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          if (g >= ngl) continue;
#pragma unroll
          for (int c = 0; c < kCH; ++c) {
            uint32_t vh[8];
            tmem_ld8(tmem + lane_addr + Ly::acc_hi(s, g) + 16 * half + 8 * c, vh);
            umma::wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j) two_sum_acc(hi[g][8 * c + j], lo[g][8 * c + j], __uint_as_float(vh[j]));
          }
          if (kt + 1 == x.nk) {  // the item's correction products, once
#pragma unroll
            for (int c = 0; c < kCH; ++c) {
              uint32_t vc[8];
              tmem_ld8(tmem + lane_addr + Ly::acc_corr(ipd, g) + 16 * half + 8 * c, vc);
              umma::wait_ld();
#pragma unroll
              for (int j = 0; j < 8; ++j) lo[g][8 * c + j] = __fadd_rn(lo[g][8 * c + j], __uint_as_float(vc[j]));
            }
          }
        }
        umma::fence_before();
        __syncwarp();
        if (lane == 0) arrive(&accempty[s]);
        if (kt + 1 < x.nk) continue;
        // ---- epilogue of the item, one group at a time: the group's
        // accumulators go through shared memory (slot k of drain thread t at
        // k * 256 + t, conflict-free) so that they are not live in registers
        // while its outputs are formed
        const int row = x.t0 + 32 * qd + lane;
        float* epi = reinterpret_cast<float*>(smem + Ly::kEpiOff) + dt;
        const volatile float* ep = epi;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          if (g >= ngl) continue;
#pragma unroll
          for (int j = 0; j < 8 * kCH; ++j) {
            epi[j * kDT] = hi[g][j];
            epi[(8 * kCH + j) * kDT] = lo[g][j];
            hi[g][j] = lo[g][j] = 0.f;
          }
          // the group's map indices for this thread's 8 (map, sign) columns,
          // loaded together, then the outputs' addresses, loaded together
          const SpinGroup* sgp = A.groups + (x.gs * NG + g);
          const int sv = sgp->s, as = sv < 0 ? -sv : sv, nb = sgp->nb;
          int mapj[kPairs];
#pragma unroll
          for (int jj = 0; jj < kPairs; ++jj) {
            const int j = kPairs * half + jj;
            const bool neg = j >= nb;
            mapj[jj] = (j < 2 * nb && !(neg && x.am == 0)) ? sgp->maps[neg ? j - nb : j] : -1;
          }
          if (DIR == 0) {
            const int l = row;
            if (l >= x.am && l < A.l1c) {
              long long base[kPairs];
#pragma unroll
              for (int jj = 0; jj < kPairs; ++jj) base[jj] = mapj[jj] >= 0 ? A.foff[mapj[jj]] : 0;
              const double nl = ((sv & 1) ? -1.0 : 1.0) * A.nl[l];
#pragma unroll kUnrollFwd
              for (int jj = 0; jj < kPairs; ++jj) {
                if (mapj[jj] < 0) continue;
                const bool neg = kPairs * half + jj >= nb;
                const int m = neg ? -x.am : x.am;
                double2 o = make_double2(0.0, 0.0);
                if (l >= as) {
                  double ar = (double)ep[(2 * jj) * kDT] + (double)ep[(8 * kCH + 2 * jj) * kDT];
                  double ai = (double)ep[(2 * jj + 1) * kDT] + (double)ep[(8 * kCH + 2 * jj + 1) * kDT];
                  const double sg2 = (neg && (l & 1)) ? -nl : nl;
                  ar *= sg2;
                  ai *= sg2;
                  switch ((m + sv) & 3) {  // times i^(m+s)
                    case 0: o = make_double2(ar, ai); break;
                    case 1: o = make_double2(-ai, ar); break;
                    case 2: o = make_double2(-ar, -ai); break;
                    default: o = make_double2(ai, -ar); break;
                  }
                }
                A.flm[base[jj] + (size_t)l * l + l + m] = o;
              }
            }
          } else {
            const int mpr = row;
            if (mpr < A.L && mpr < A.l1c) {
#pragma unroll kUnrollInv
              for (int j0 = 0; j0 < kPairs; j0 += 4) {  // four read-modify-writes in flight at a time
                float4* dst[4];
                float4 cur[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const int jj = j0 + u;
                  const bool neg = kPairs * half + jj >= nb;
                  dst[u] = reinterpret_cast<float4*>(A.Fp) +
                           ((size_t)(mapj[jj] < 0 ? 0 : mapj[jj]) * A.M + (neg ? -x.am : x.am) + A.L - 1) * A.L + mpr;
                  cur[u] = mapj[jj] >= 0 ? *dst[u] : make_float4(0.f, 0.f, 0.f, 0.f);
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                  const int jj = j0 + u;
                  if (mapj[jj] < 0) continue;
                  const bool neg = kPairs * half + jj >= nb;
                  float rh = ep[(2 * jj) * kDT], rl = ep[(8 * kCH + 2 * jj) * kDT];
                  float ih = ep[(2 * jj + 1) * kDT], il = ep[(8 * kCH + 2 * jj + 1) * kDT];
                  if (neg && (mpr & 1)) { rh = -rh; rl = -rl; ih = -ih; il = -il; }
                  ff_add(cur[u].x, cur[u].y, rh, rl);
                  ff_add(cur[u].z, cur[u].w, ih, il);
                  *dst[u] = cur[u];
                }
              }
            }
          }
        }
      }
    }
    if (ctl && *abort_flag) {
      // let the MMAs already issued finish before the TMEM is released
      umma::commit(fin);
      wait_bar_all(fin, 0);
    }
    if (tma_thr && *abort_flag) {
      // and the TMA loads already issued land before the CTA's shared memory goes
      for (int t = 0; t < kTS; ++t) {
        const int nt = n_tma > t ? (n_tma - t - 1) / kTS + 1 : 0;  // loads issued to stage t
        if (nt > 0) wait_bar_all(&tma_full[t], (uint32_t)(nt - 1) & 1u);
      }
    }
  }
  umma::fence_before();
  __syncthreads();
  umma::fence_after();
  if (warp == 0) umma::tmem_dealloc(tmem, Ly::kAlloc);
}

// ---- host side ------------------------------------------------------------

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  if (!fn) {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
    else
      cudaGetLastError();
  }
  return fn;
}

template <int DIR, int NG>
cudaError_t launch_t(const mw_plan* p, const mw_plan* o, int l0, int l1c, const int4* items, int nitems,
                     const float2* bsrc, double2* flm, cudaStream_t st) {
  if (nitems <= 0) return cudaSuccess;
  using Ly = Layout<NG>;
  cudaError_t e = cudaFuncSetAttribute(k_tc2<DIR, NG>, cudaFuncAttributeMaxDynamicSharedMemorySize, Ly::kSmem);
  if (e != cudaSuccess) return e;
  int nsm = 0;
  e = cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device);
  if (e != cudaSuccess) return e;
  Tc2Args a;
  a.L = p->L; a.M = p->M; a.l0 = l0; a.l1c = l1c; a.LD = o->LD;
  a.items = items; a.nitems = nitems;
  a.groups = p->d_groups; a.ng = (int)p->groups.size();
  a.bsrc = bsrc; a.nl = p->d_nl; a.flm = flm; a.foff = p->d_foff;
  a.Fp = p->d_Gp; a.err = p->d_err;
  const int grid = nitems < nsm ? nitems : nsm;
  k_tc2<DIR, NG><<<grid, Ly::kThreads, Ly::kSmem, st>>>(DIR == 0 ? o->tmap_fwd : o->tmap_inv, a);
  return cudaGetLastError();
}

}  // namespace

// Tensor maps of the owner's FP32 staging planes S32 [nslot][LD][LD]: the
// forward reads boxes of 32 m' x 1 row x 128 planes (128-byte swizzle), the
// inverse boxes of 128 m' x 1 row x 32 planes.  Out-of-range parts of a box
// read as zero.
cudaError_t make_tc2_tensor_maps(mw_plan* o) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return cudaErrorNotSupported;
  const int nslot = o->L < kTcChunk ? o->L : kTcChunk;
  const cuuint64_t dims[3] = {(cuuint64_t)o->LD, (cuuint64_t)o->LD, (cuuint64_t)nslot};
  const cuuint64_t strides[2] = {(cuuint64_t)o->LD * 4, (cuuint64_t)o->LD * o->LD * 4};
  const cuuint32_t es[3] = {1, 1, 1};
  const cuuint32_t box_f[3] = {32, 1, 128}, box_i[3] = {128, 1, 32};
  CUresult r = fn(&o->tmap_fwd, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, o->d_S32, dims, strides, box_f, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  r = fn(&o->tmap_inv, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, o->d_S32, dims, strides, box_i, es,
         CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
         CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) return cudaErrorInvalidValue;
  o->tc2_maps = true;
  return cudaSuccess;
}

// Work lists of plan p for every chunk [l0, l0 + kTcChunk) and both
// directions, as (am, first row, group slice, K tiles), each list ordered by
// |m| so that the items sharing one row of B run side by side (their B rows
// meet in L2), l tiles largest first.
cudaError_t make_tc2_items(mw_plan* p, int chunk) {
  const int L = p->L, ng = (int)p->groups.size();
  if (p->d_tc2_items) {
    cudaFree(p->d_tc2_items);
    p->d_tc2_items = nullptr;
  }
  const int ngs = (ng + p->tc2_ng - 1) / p->tc2_ng;
  std::vector<int4> all;
  p->tc2_off.clear();
  for (int dir = 0; dir < 2; ++dir) {
    for (int l0 = 0; l0 < L; l0 += chunk) {
      const int l1c = std::min(l0 + chunk, L);
      p->tc2_off.push_back((int)all.size());
      for (int am = 0; am < l1c; ++am) {
        if (dir == 0) {
          for (int lt0 = l0 + ((l1c - l0 - 1) / kRows) * kRows; lt0 >= l0; lt0 -= kRows) {
            const int lt1 = std::min(lt0 + kRows, l1c);
            if (lt1 <= am) continue;
            for (int gs = 0; gs < ngs; ++gs) all.push_back(make_int4(am, lt0, gs, (lt1 + kKT - 1) / kKT));
          }
        } else {
          for (int mp0 = 0; mp0 < l1c; mp0 += kRows) {
            const int kstart = std::max(std::max(l0, am), mp0);
            if (kstart >= l1c) continue;
            for (int gs = 0; gs < ngs; ++gs) all.push_back(make_int4(am, mp0, gs, (l1c - kstart + kKT - 1) / kKT));
          }
        }
      }
    }
  }
  p->tc2_off.push_back((int)all.size());
  p->tc2_chunk = chunk;
  if (all.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)&p->d_tc2_items, sizeof(int4) * all.size());
  if (e != cudaSuccess) return e;
  return cudaMemcpy(p->d_tc2_items, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice);
}

// N_l f_lm in FP32, transposed to [B][M][L] (row m + L - 1, l contiguous; zero
// for l < |m|): the inverse contraction reads 32 consecutive l of a row.  Rows
// l in [l0, l1) only (a chunk of planes whose f_lm rows have arrived).
__global__ void k_flm_transpose(const double2* __restrict__ flm, const long long* __restrict__ foff,
                                float2* __restrict__ out, int L, int l0, int l1) {
  const int mi = blockIdx.x, b = blockIdx.y;
  const int M = 2 * L - 1, m = mi - (L - 1), am = m < 0 ? -m : m;
  const double2* src = flm + foff[b];
  float2* dst = out + ((size_t)b * M + mi) * L;
  for (int l = l0 + threadIdx.x; l < l1; l += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (l >= am) {
      const double2 f = src[(size_t)l * l + l + m];
      const float nl = sqrtf((2.f * l + 1.f) / (4.f * 3.14159265358979f));
      v = make_float2((float)f.x * nl, (float)f.y * nl);
    }
    dst[l] = v;
  }
}

cudaError_t launch_flm_transpose(const mw_plan* p, const double2* flm, cudaStream_t st, int l0, int l1) {
  if (l1 < 0 || l1 > p->L) l1 = p->L;
  if (l0 >= l1) return cudaSuccess;
  k_flm_transpose<<<dim3(p->M, p->B), 256, 0, st>>>(flm, p->d_foff, p->d_flmT, p->L, l0, l1);
  return cudaGetLastError();
}

// Contraction of plan p (a consumer of owner o's staged planes) over the
// planes [l0, l1c) of the chunk that starts at l0.
cudaError_t launch_tc2(const mw_plan* p, const mw_plan* o, int dir, int l0, int l1c, double2* flm,
                       cudaStream_t st) {
  const int chunk = l0 / p->tc2_chunk;
  const int nch = (p->L + p->tc2_chunk - 1) / p->tc2_chunk;
  const int k = dir * nch + chunk;
  const int4* items = p->d_tc2_items + p->tc2_off[k];
  const int n = p->tc2_off[k + 1] - p->tc2_off[k];
  if (dir == 0) {
    return p->tc2_ng == 2 ? launch_t<0, 2>(p, o, l0, l1c, items, n, reinterpret_cast<const float2*>(p->d_Gp), flm, st)
                          : launch_t<0, 1>(p, o, l0, l1c, items, n, reinterpret_cast<const float2*>(p->d_Gp), flm, st);
  }
  return p->tc2_ng == 2 ? launch_t<1, 2>(p, o, l0, l1c, items, n, p->d_flmT, nullptr, st)
                        : launch_t<1, 1>(p, o, l0, l1c, items, n, p->d_flmT, nullptr, st);
}
