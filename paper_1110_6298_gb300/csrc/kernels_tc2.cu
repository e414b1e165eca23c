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
// tile in a fresh accumulator and the four correction products in a second
// one, both summed across K tiles in float-float on the CUDA cores.
//
// What is new is the data flow.  Each CTA (one per SM) walks a list of work
// items (am, row tile, spin-group slice); a work item is a run of 32-wide K
// tiles, and the K tiles of all the CTA's items form one pipelined sequence:
//   control warp   one thread loads the FP32 plane tiles of a K tile -- row am
//                  and the spin rows |s| of the 128 (forward) or 32
//                  (inverse) planes -- with plain per-CTA TMA
//                  (cp.async.bulk.tensor, this GPU's memory only, no
//                  multicast) two K tiles ahead, and issues the MMAs;
//   8 producer     form A for one row each (TMEM lane = row) for both spin
//   warps          groups from one plane tile, split it, and store it straight
//                  into tensor memory (tcgen05.st), so the MMAs read only B
//                  from shared memory; they also split B into shared memory;
//   8 drain warps  read the two accumulators per group (tcgen05.ld), add them
//                  into float-float registers, release the accumulator, and
//                  write the item's outputs after its last K tile.
// Operands and accumulators are double-buffered; stages are handed over with
// mbarriers: TMA bytes -> producers -> MMA -> (producers, drain) -> MMA.  Every
// wait is bounded: a wait that gives up records the timeout in the plan's error
// word, raises the CTA's abort flag (which the other roles poll) and the CTA
// leaves after the TMEM is released; the outputs of such a call are invalid.
#include <cuda.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "umma.cuh"

namespace {

constexpr int kKT = 32;                    // K per tile (two K = 16 MMA steps)
constexpr int kRows = 128;                 // rows of a tile (TMEM lanes)
constexpr int kN = 32;                     // accumulator columns per spin group
constexpr int kWarps = 17;                 // 1 control + 8 producer + 8 drain
constexpr int kThreads = 32 * kWarps;
constexpr int kTmaTile = 16384;            // one FP32 plane tile: 128 x 32 or 32 x 128 floats
constexpr int kBTile = kN * kKT * 2;       // one BF16 split of B (2 KB)
constexpr uint32_t kPolls = 1u << 24;

template <int NG>
struct Layout {
  static constexpr int kTmaStage = (1 + NG) * kTmaTile;             // row am + one spin row per group
  static constexpr int kBStage = NG * 3 * kBTile;
  static constexpr int kTmaOff = 0;                                  // 1024-aligned
  static constexpr int kBOff = 2 * kTmaStage;
  static constexpr int kEpiOff = kBOff + 2 * kBStage;                // drain epilogue staging
  static constexpr int kEpiBytes = 256 * NG * 32 * 4;                 // 256 drain threads x NG x 16 (hi, lo)
  static constexpr int kBarOff = kEpiOff + kEpiBytes;
  static constexpr int kBytes = kBarOff + 128;
  static constexpr int kSmem = kBytes + 1024;                        // slack for the manual alignment
  // TMEM columns: accumulators (hi, corr) per buffer and group, then A per
  // stage, group, K step and split (8 columns = 16 bf16 of K each)
  static constexpr int kAccCols = 2 * NG * 64;
  static constexpr int kCols = kAccCols + 2 * NG * 2 * 3 * 8;
  static constexpr uint32_t kAlloc = kCols <= 256 ? 256u : 512u;
  static_assert(kCols <= 512, "TMEM budget");
  static_assert(kSmem <= 227 * 1024, "shared memory budget");
  __device__ static uint32_t acc_hi(int a, int g) { return (uint32_t)((a * NG + g) * 64); }
  __device__ static uint32_t acc_corr(int a, int g) { return (uint32_t)((a * NG + g) * 64 + 32); }
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
__device__ __forceinline__ bool try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(umma::smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}
// Bounded wait that ignores the abort flag (the abort path's own waits).
__device__ __forceinline__ bool wait_bar_all(uint64_t* bar, uint32_t parity) {
  for (uint32_t it = 0; it < kPolls; ++it)
    if (try_wait(bar, parity)) return true;
  return false;
}
// Bounded wait that also gives up once another role has raised the abort flag.
__device__ __forceinline__ bool wait_bar(uint64_t* bar, uint32_t parity, volatile int* abort_flag) {
  for (uint32_t it = 0; it < kPolls; ++it) {
    if (try_wait(bar, parity)) return true;
    if ((it & 255u) == 255u && *abort_flag) return false;
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

// x (two values) -> bf16 pairs hi, mid, lo with x ~= hi + mid + lo
__device__ __forceinline__ void split_pair(float x0, float x1, uint32_t& h, uint32_t& m, uint32_t& l) {
  const __nv_bfloat162 hp = __floats2bfloat162_rn(x0, x1);
  const float2 hf = __bfloat1622float2(hp);
  const float r0 = x0 - hf.x, r1 = x1 - hf.y;
  const __nv_bfloat162 mp = __floats2bfloat162_rn(r0, r1);
  const float2 mf = __bfloat1622float2(mp);
  const __nv_bfloat162 lp = __floats2bfloat162_rn(r0 - mf.x, r1 - mf.y);
  h = *reinterpret_cast<const uint32_t*>(&hp);
  m = *reinterpret_cast<const uint32_t*>(&mp);
  l = *reinterpret_cast<const uint32_t*>(&lp);
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
__global__ void __launch_bounds__(kThreads, 1) k_tc2(const __grid_constant__ CUtensorMap tmap, Tc2Args A) {
  using Ly = Layout<NG>;
  extern __shared__ unsigned char smem_raw[];
  const uint32_t raw = umma::smem_u32(smem_raw);
  unsigned char* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
  uint64_t* bar = reinterpret_cast<uint64_t*>(smem + Ly::kBarOff);
  uint64_t* tma_full = bar;      // [2] TMA bytes of a stage arrived
  uint64_t* full = bar + 2;      // [2] producers wrote A (TMEM) and B (smem) of a stage
  uint64_t* done = bar + 4;      // [2] the MMAs of a stage completed
  uint64_t* accempty = bar + 6;  // [2] the drain read an accumulator buffer
  uint64_t* fin = bar + 8;       // final MMA completion on the abort path
  uint32_t* tslot = reinterpret_cast<uint32_t*>(bar + 9);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bar + 10);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int G = gridDim.x;
  if (tid == 0) {
    for (int s = 0; s < 2; ++s) {
      umma::mbar_init(&tma_full[s], 1);
      umma::mbar_init(&full[s], 8);
      umma::mbar_init(&done[s], 1);
      umma::mbar_init(&accempty[s], 8);
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

  if (warp == 0) {
    // ------------------------------------------------------------ control
    if (lane == 0) {
      const uint32_t idesc = umma::idesc_bf16_f32(kRows, kN);
      // TMA of sequence position (it, kt) into stage s
      auto issue_tma = [&](int it, int kt, int s) {
        const Item x = item_of<DIR>(A, it);
        const int ngl = min(NG, A.ng - x.gs * NG);
        arrive_expect_tx(&tma_full[s], (uint32_t)((1 + NG) * kTmaTile));
        const uint32_t dst = tma_base + (uint32_t)(s * Ly::kTmaStage);
        int xx, zz;
        if (DIR == 0) { xx = kKT * kt; zz = x.t0 - A.l0; }               // 32 m' of 128 planes
        else { xx = x.t0; zz = x.kstart + kKT * kt - A.l0; }             // 128 m' of 32 planes
        tma_load_3d(dst, &tmap, xx, x.am, zz, &tma_full[s]);
        for (int g = 0; g < NG; ++g) {
          // a slice with fewer groups loads its last spin row again (bytes must match)
          const int s_g = A.groups[x.gs * NG + min(g, ngl - 1)].s;
          tma_load_3d(dst + (uint32_t)((1 + g) * kTmaTile), &tmap, xx, s_g < 0 ? -s_g : s_g, zz, &tma_full[s]);
        }
      };
      // the sequence: items blockIdx.x, +G, ...; K tiles of each
      int it_n = blockIdx.x, kt_n = 0;  // position two ahead (TMA prefetch)
      int n_tma[2] = {0, 0};            // TMA loads issued per stage
      auto advance = [&](int& it, int& kt) {
        if (++kt >= A.items[it].w) { kt = 0; it += G; }
      };
      for (int s = 0; s < 2 && it_n < A.nitems; ++s) {
        issue_tma(it_n, kt_n, s);
        ++n_tma[s];
        advance(it_n, kt_n);
      }
      int q = 0;
      bool ok = true;
      for (int it = blockIdx.x; ok && it < A.nitems; it += G) {
        const Item x = item_of<DIR>(A, it);
        const int ngl = min(NG, A.ng - x.gs * NG);
        for (int kt = 0; kt < x.nk; ++kt, ++q) {
          const int s = q & 1;
          const uint32_t ph = (uint32_t)(q >> 1) & 1u;
          if (!wait_bar(&full[s], ph, abort_flag)) { fail(); ok = false; break; }
          if (q >= 2 && !wait_bar(&accempty[s], ph ^ 1u, abort_flag)) { fail(); ok = false; break; }
          umma::fence_after();
          for (int g = 0; g < ngl; ++g) {
#pragma unroll
            for (int ks = 0; ks < 2; ++ks) {
#pragma unroll
              for (int p = 0; p < 6; ++p) {
                const uint32_t bd_addr = b_base + (uint32_t)(s * Ly::kBStage + (g * 3 + split_b(p)) * kBTile + ks * 256);
                const uint64_t bd = umma::smem_desc(bd_addr, 128, (kKT / 8) * 128);
                const uint32_t d = tmem + (p == 0 ? Ly::acc_hi(s, g) : Ly::acc_corr(s, g));
                const int acc = (p == 0) ? (ks > 0) : !(ks == 0 && p == 1);
                mma_ta(d, tmem + Ly::a_col(s, g, ks, split_a(p)), bd, idesc, acc);
              }
            }
          }
          umma::commit(&done[s]);
          if (it_n < A.nitems) {  // the TMA tiles of stage s were read: refill two ahead
            issue_tma(it_n, kt_n, s);
            ++n_tma[s];
            advance(it_n, kt_n);
          }
        }
      }
      if (!ok) {
        // let the MMAs already issued finish before the TMEM is released, and
        // the TMA loads already issued land before the CTA's shared memory goes
        umma::commit(fin);
        wait_bar_all(fin, 0);
        for (int s = 0; s < 2; ++s)
          if (n_tma[s] > 0) wait_bar_all(&tma_full[s], (uint32_t)(n_tma[s] - 1) & 1u);
      }
    }
    __syncwarp();
  } else if (warp <= 8) {
    // ----------------------------------------------------------- producers
    const int pw = warp - 1, ks = pw >> 2, qd = warp & 3;
    const int r = 32 * qd + lane;                       // tile row = TMEM lane
    const uint32_t lane_addr = (uint32_t)(32 * qd) << 16;
    const int pt = pw * 32 + lane;                      // B unit: group pt / 128, row n, 8-wide K chunk
    const int bg = pt >> 7, bn = (pt >> 2) & 31, bkc = pt & 3;
    float bcur[8], bnext[8];
    // B values of sequence position (it, kt): 8 consecutive K of row bn of group bg
    auto load_b = [&](int it, int kt, float* v) {
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] = 0.f;
      if (it >= A.nitems) return;
      const Item x = item_of<DIR>(A, it);
      const int gidx = x.gs * NG + bg;
      if (bg >= NG || gidx >= A.ng) return;
      const SpinGroup& g = A.groups[gidx];
      const int j = bn >> 1, nb = g.nb;
      if (j >= 2 * nb) return;
      const bool neg = j >= nb;
      if (neg && x.am == 0) return;
      const int map = g.maps[neg ? j - nb : j];
      const int k0 = x.kstart + kKT * kt + 8 * bkc;  // m' (forward) or l (inverse)
      const float2* row = A.bsrc + ((size_t)map * A.M + (neg ? -x.am : x.am) + A.L - 1) * A.L;
      const int kend = DIR == 0 ? A.L : A.l1c;
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int k = k0 + i;
        if (k < kend) {
          const float2 f = __ldg(row + k);
          float y = (bn & 1) ? f.y : f.x;
          if (neg && (k & 1)) y = -y;  // (-1)^m' (forward) or (-1)^l (inverse) of the -am fold
          v[i] = y;
        }
      }
    };
    int it_b = blockIdx.x, kt_b = 0;  // position of bnext
    auto adv = [&](int& it, int& kt) {
      if (++kt >= A.items[it].w) { kt = 0; it += G; }
    };
    if (it_b < A.nitems) {
      load_b(it_b, kt_b, bcur);
      adv(it_b, kt_b);
    }
    int q = 0;
    bool ok = true;
    for (int it = blockIdx.x; ok && it < A.nitems; it += G) {
      const Item x = item_of<DIR>(A, it);
      const int ngl = min(NG, A.ng - x.gs * NG);
      for (int kt = 0; kt < x.nk; ++kt, ++q) {
        const int s = q & 1;
        const uint32_t ph = (uint32_t)(q >> 1) & 1u;
        load_b(it_b, kt_b, bnext);  // next position's B, in flight during this one
        // every lane waits; the outcome is made warp-uniform so that the
        // warp-collective TMEM stores and __syncwarp below never diverge
        bool w = (q < 2 || wait_bar(&done[s], ph ^ 1u, abort_flag)) && wait_bar(&tma_full[s], ph, abort_flag);
        if (!__all_sync(0xffffffffu, w)) { if (lane == 0) fail(); ok = false; break; }
        umma::fence_after();
        const float* T = reinterpret_cast<const float*>(smem + Ly::kTmaOff + s * Ly::kTmaStage);
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
          const float* W = T + (1 + g) * (kTmaTile / 4);
          uint32_t hp[8], mp[8], lp[8];
          if (g < ngl) {
            const SpinGroup& sg = A.groups[x.gs * NG + g];
            const int sv = sg.s, as = sv < 0 ? -sv : sv;
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
                if (4 * c > lim) x0 = 0.f;
                if (4 * c + 1 > lim) x1 = 0.f;
                if (4 * c + 2 > lim) x2 = 0.f;
                if (4 * c + 3 > lim) x3 = 0.f;
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
                if (2 * i < lo_i || 2 * i >= hi_i) x0 = 0.f;
                if (2 * i + 1 < lo_i || 2 * i + 1 >= hi_i) x1 = 0.f;
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
        // B: 8 K of row bn of group bg, split into the K-major core-matrix layout
        if (bg < NG) {
          uint32_t h[4], m[4], l[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) split_pair(bcur[2 * i], bcur[2 * i + 1], h[i], m[i], l[i]);
          unsigned char* sb = smem + Ly::kBOff + s * Ly::kBStage + bg * 3 * kBTile;
          const int off = umma::tile_off(bn, 8 * bkc, kKT / 8);
          *reinterpret_cast<uint4*>(sb + off) = make_uint4(h[0], h[1], h[2], h[3]);
          *reinterpret_cast<uint4*>(sb + kBTile + off) = make_uint4(m[0], m[1], m[2], m[3]);
          *reinterpret_cast<uint4*>(sb + 2 * kBTile + off) = make_uint4(l[0], l[1], l[2], l[3]);
        }
#pragma unroll
        for (int i = 0; i < 8; ++i) bcur[i] = bnext[i];
        if (it_b < A.nitems) adv(it_b, kt_b);
        tmem_wait_st();
        umma::fence_proxy_async();
        umma::fence_before();
        __syncwarp();
        if (lane == 0) arrive(&full[s]);
      }
    }
  } else {
    // --------------------------------------------------------------- drain
    const int dw = warp - 9, half = dw >> 2, qd = warp & 3;
    const uint32_t lane_addr = (uint32_t)(32 * qd) << 16;
    float hi[NG][16], lo[NG][16];
#pragma unroll
    for (int g = 0; g < NG; ++g)
#pragma unroll
      for (int j = 0; j < 16; ++j) hi[g][j] = lo[g][j] = 0.f;
    int q = 0;
    bool ok = true;
    for (int it = blockIdx.x; ok && it < A.nitems; it += G) {
      const Item x = item_of<DIR>(A, it);
      const int ngl = min(NG, A.ng - x.gs * NG);
      for (int kt = 0; kt < x.nk; ++kt, ++q) {
        const int s = q & 1;
        const uint32_t ph = (uint32_t)(q >> 1) & 1u;
        if (!__all_sync(0xffffffffu, wait_bar(&done[s], ph, abort_flag))) { if (lane == 0) fail(); ok = false; break; }
        umma::fence_after();
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          if (g >= ngl) continue;
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            uint32_t vh[8], vc[8];
            tmem_ld8(tmem + lane_addr + Ly::acc_hi(s, g) + 16 * half + 8 * c, vh);
            tmem_ld8(tmem + lane_addr + Ly::acc_corr(s, g) + 16 * half + 8 * c, vc);
            umma::wait_ld();
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              two_sum_acc(hi[g][8 * c + j], lo[g][8 * c + j], __uint_as_float(vh[j]));
              lo[g][8 * c + j] = __fadd_rn(lo[g][8 * c + j], __uint_as_float(vc[j]));
            }
          }
        }
        umma::fence_before();
        __syncwarp();
        if (lane == 0) arrive(&accempty[s]);
        if (kt + 1 < x.nk) continue;
        // ---- epilogue of the item: the accumulators go through shared memory
        // (this thread's own slots), so that they are not live in registers
        // while the outputs are formed
        float* epi = reinterpret_cast<float*>(smem + Ly::kEpiOff) + (size_t)(tid - 9 * 32) * NG * 32;
#pragma unroll
        for (int g = 0; g < NG; ++g)
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            epi[g * 32 + j] = hi[g][j];
            epi[g * 32 + 16 + j] = lo[g][j];
            hi[g][j] = lo[g][j] = 0.f;
          }
        const volatile float* ep = epi;  // read back at the point of use (keeps few values live)
        const int row = x.t0 + 32 * qd + lane;
#pragma unroll
        for (int g = 0; g < NG; ++g) {
          if (g >= ngl) continue;
          const SpinGroup& sg = A.groups[x.gs * NG + g];
          const int sv = sg.s, as = sv < 0 ? -sv : sv, nb = sg.nb;
          if (DIR == 0) {
            const int l = row;
            if (l >= x.am && l < A.l1c) {
              const double nl = ((sv & 1) ? -1.0 : 1.0) * A.nl[l];
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                const int j = 8 * half + jj;
                if (j >= 2 * nb) continue;
                const bool neg = j >= nb;
                if (neg && x.am == 0) continue;
                const int m = neg ? -x.am : x.am;
                double2 o = make_double2(0.0, 0.0);
                if (l >= as) {
                  double ar = (double)ep[g * 32 + 2 * jj] + (double)ep[g * 32 + 16 + 2 * jj];
                  double ai = (double)ep[g * 32 + 2 * jj + 1] + (double)ep[g * 32 + 16 + 2 * jj + 1];
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
                A.flm[A.foff[sg.maps[neg ? j - nb : j]] + (size_t)l * l + l + m] = o;
              }
            }
          } else {
            const int mpr = row;
            if (mpr < A.L && mpr < A.l1c) {
#pragma unroll
              for (int jj = 0; jj < 8; ++jj) {
                const int j = 8 * half + jj;
                if (j >= 2 * nb) continue;
                const bool neg = j >= nb;
                if (neg && x.am == 0) continue;
                const int b = sg.maps[neg ? j - nb : j];
                float4* dst = reinterpret_cast<float4*>(A.Fp) + ((size_t)b * A.M + (neg ? -x.am : x.am) + A.L - 1) * A.L + mpr;
                float rh = ep[g * 32 + 2 * jj], rl = ep[g * 32 + 16 + 2 * jj];
                float ih = ep[g * 32 + 2 * jj + 1], il = ep[g * 32 + 16 + 2 * jj + 1];
                if (neg && (mpr & 1)) { rh = -rh; rl = -rl; ih = -ih; il = -il; }
                float4 cur = *dst;
                ff_add(cur.x, cur.y, rh, rl);
                ff_add(cur.z, cur.w, ih, il);
                *dst = cur;
              }
            }
          }
        }
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
  k_tc2<DIR, NG><<<grid, kThreads, Ly::kSmem, st>>>(DIR == 0 ? o->tmap_fwd : o->tmap_inv, a);
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
cudaError_t make_tc2_items(mw_plan* p) {
  const int L = p->L, ng = (int)p->groups.size();
  const int ngs = (ng + p->tc2_ng - 1) / p->tc2_ng;
  std::vector<int4> all;
  p->tc2_off.clear();
  for (int dir = 0; dir < 2; ++dir) {
    for (int l0 = 0; l0 < L; l0 += kTcChunk) {
      const int l1c = std::min(l0 + kTcChunk, L);
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
  if (all.empty()) return cudaSuccess;
  cudaError_t e = cudaMalloc((void**)&p->d_tc2_items, sizeof(int4) * all.size());
  if (e != cudaSuccess) return e;
  p->ws_bytes += sizeof(int4) * all.size();
  return cudaMemcpy(p->d_tc2_items, all.data(), sizeof(int4) * all.size(), cudaMemcpyHostToDevice);
}

// N_l f_lm in FP32, transposed to [B][M][L] (row m + L - 1, l contiguous; zero
// for l < |m|): the inverse contraction reads 32 consecutive l of a row.
__global__ void k_flm_transpose(const double2* __restrict__ flm, const long long* __restrict__ foff,
                                float2* __restrict__ out, int L) {
  const int mi = blockIdx.x, b = blockIdx.y;
  const int M = 2 * L - 1, m = mi - (L - 1), am = m < 0 ? -m : m;
  const double2* src = flm + foff[b];
  float2* dst = out + ((size_t)b * M + mi) * L;
  for (int l = threadIdx.x; l < L; l += blockDim.x) {
    float2 v = make_float2(0.f, 0.f);
    if (l >= am) {
      const double2 f = src[(size_t)l * l + l + m];
      const float nl = sqrtf((2.f * l + 1.f) / (4.f * 3.14159265358979f));
      v = make_float2((float)f.x * nl, (float)f.y * nl);
    }
    dst[l] = v;
  }
}

cudaError_t launch_flm_transpose(const mw_plan* p, const double2* flm, cudaStream_t st) {
  k_flm_transpose<<<dim3(p->M, p->B), 256, 0, st>>>(flm, p->d_foff, p->d_flmT, p->L);
  return cudaGetLastError();
}

// Contraction of plan p (a consumer of owner o's staged planes) over the
// planes [l0, l1c) of the chunk that starts at l0.
cudaError_t launch_tc2(const mw_plan* p, const mw_plan* o, int dir, int l0, int l1c, double2* flm,
                       cudaStream_t st) {
  const int chunk = l0 / kTcChunk;
  const int nch = (p->L + kTcChunk - 1) / kTcChunk;
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
