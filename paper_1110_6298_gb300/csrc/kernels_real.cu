// kernels_real.cu -- real scalar signals (Sec. IV-G) on the complex transform.
//
// A real-signal plan transforms real maps two at a time: maps 2b and 2b+1 ride
// as the real and imaginary part of one complex spin-0 map g = f1 + i f2 (the
// phi kernels read and write the pairs directly).  Coefficients separate with
// the reality condition f_{l,-m} = (-1)^m conj(f_lm) of a real scalar signal:
//   (-1)^m conj(g_{l,-m}) = f1_lm - i f2_lm,
//   f1_lm = (g_lm + (-1)^m conj(g_{l,-m})) / 2,
//   f2_lm = (g_lm - (-1)^m conj(g_{l,-m})) / (2i).
// The inverse packs g_lm = h1_lm + i h2_lm, h the Hermitian part
// (f_lm + (-1)^m conj(f_{l,-m})) / 2 (the coefficients of Re f), so the real
// and imaginary parts of the synthesis of g are Re(f1) and Re(f2) synthesised.
// Every output pair (l, m), (l, -m) is formed by one thread from the pair it
// reads, so m < 0 is the exact mirror of m > 0.
#include "internal.h"

namespace {

constexpr int kRThreads = 128;

__device__ __forceinline__ double2 mirror(double2 v, int m) {  // (-1)^m conj(v)
  const double sg = (m & 1) ? -1.0 : 1.0;
  return make_double2(sg * v.x, -sg * v.y);
}

// g [Bc][L*L] -> flm [nreal][L*L]; block (l, b)
__global__ void __launch_bounds__(kRThreads) k_real_unpack(int L, int nreal, const double2* __restrict__ g,
                                                           double2* __restrict__ flm) {
  const int l = blockIdx.x, b = blockIdx.y;
  const size_t row = (size_t)l * l + l;
  const double2* gb = g + (size_t)b * L * L + row;
  double2* f1 = flm + (size_t)(2 * b) * L * L + row;
  double2* f2 = (2 * b + 1 < nreal) ? f1 + (size_t)L * L : nullptr;
  for (int m = threadIdx.x; m <= l; m += blockDim.x) {
    const double2 gp = gb[m];
    const double2 c = mirror(gb[-m], m);
    const double2 a = make_double2(0.5 * (gp.x + c.x), 0.5 * (gp.y + c.y));   // f1_lm
    const double2 d = make_double2(0.5 * (gp.y - c.y), -0.5 * (gp.x - c.x));  // f2_lm = -i (gp - c) / 2
    f1[m] = a;
    if (m) f1[-m] = mirror(a, m);
    if (f2) {
      f2[m] = d;
      if (m) f2[-m] = mirror(d, m);
    }
  }
}

// flm [nreal][L*L] -> g [Bc][L*L]; block (l, b)
__global__ void __launch_bounds__(kRThreads) k_real_pack(int L, int nreal, const double2* __restrict__ flm,
                                                         double2* __restrict__ g) {
  const int l = blockIdx.x, b = blockIdx.y;
  const size_t row = (size_t)l * l + l;
  const double2* f1 = flm + (size_t)(2 * b) * L * L + row;
  const double2* f2 = (2 * b + 1 < nreal) ? f1 + (size_t)L * L : nullptr;
  double2* gb = g + (size_t)b * L * L + row;
  for (int m = threadIdx.x; m <= l; m += blockDim.x) {
    double2 c1 = mirror(f1[-m], m), h1 = f1[m];
    h1 = make_double2(0.5 * (h1.x + c1.x), 0.5 * (h1.y + c1.y));
    double2 h2 = make_double2(0.0, 0.0);
    if (f2) {
      const double2 c2 = mirror(f2[-m], m), v = f2[m];
      h2 = make_double2(0.5 * (v.x + c2.x), 0.5 * (v.y + c2.y));
    }
    gb[m] = make_double2(h1.x - h2.y, h1.y + h2.x);  // h1 + i h2 at +m
    if (m) {
      const double2 n1 = mirror(h1, m), n2 = mirror(h2, m);
      gb[-m] = make_double2(n1.x - n2.y, n1.y + n2.x);
    }
  }
}

}  // namespace

cudaError_t launch_real_unpack(const mw_plan* p, const double2* g, double2* flm, cudaStream_t st) {
  k_real_unpack<<<dim3(p->L, p->B), kRThreads, 0, st>>>(p->L, p->nreal, g, flm);
  return cudaGetLastError();
}

cudaError_t launch_real_pack(const mw_plan* p, const double2* flm, double2* g, cudaStream_t st) {
  k_real_pack<<<dim3(p->L, p->B), kRThreads, 0, st>>>(p->L, p->nreal, flm, g);
  return cudaGetLastError();
}
