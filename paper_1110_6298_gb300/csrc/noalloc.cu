// noalloc.cu -- mw_inverse_noalloc: the FP64 inverse transform of one map with
// every intermediate in a static device array, for callers that cannot
// allocate device memory (inside a custom allocator's callbacks, hosts that
// forbid allocation after start-up, processes whose free device memory belongs
// to another pool).  Nothing here calls cudaMalloc, cudaFree or any other
// allocating routine; the plan-based entry points are untouched.
//
// What it computes is the inverse of Sec. IV-E for one map:
//   F_mm'     = (-1)^s i^-(m+s) sum_l sqrt((2l+1)/4pi) Delta^l_{m'm} Delta^l_{m',-s} f_lm   Eq. (Fmm)
//   F_m(th_t) = sum_m' F_mm' e^{i m' th_t}                                           Eq. (Fmt)
//   f(th_t, ph_p) = sum_m F_m(th_t) e^{i m ph_p}                                     Eq. (f_pfft)
// with Delta^l = d^l(pi/2) from Risbo's recursion (Sec. V-B) on full planes.
// It is sized for small band limits (L <= 128): one CTA runs the recursion and
// the Eq. (Fmm) sum, then one CTA per ring evaluates the two DFTs directly.
#include <mutex>

#include "../../include/mw.h"

#include <cuda_runtime.h>

namespace {

constexpr int kMaxL = MW_NOALLOC_MAX_L;
constexpr int kDim = 2 * kMaxL - 1;          // largest plane side (2l+1 for l = L-1) and M
constexpr int kPlaneStride = 65056;          // >= kDim^2, a multiple of 32 doubles (256 B)
constexpr int kScratchDoubles = 3 * kPlaneStride + 2 * kDim * kDim;
constexpr int kWignerThreads = 1024;
constexpr int kSynthThreads = 256;
constexpr int kMaxDevices = 64;
static_assert(kPlaneStride >= kDim * kDim, "plane stride too small");
static_assert(kScratchDoubles * 8 == MW_NOALLOC_SCRATCH_BYTES, "scratch size out of step with mw.h");

// The scratch array: three Delta planes (current, half step, next) followed by
// the M x M complex F_mm'.  In host code this name is only a stand-in for the
// symbol; its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_scratch[kScratchDoubles];

// One Risbo half step (Sec. V-B) at beta = pi/2 (p = q = 1/sqrt 2), in gather
// form: d is the P x P plane d^{(P-1)/2}, e the (P+1) x (P+1) plane d^{P/2}.
//   e[a][b] = (1/P) ( sq(P-a) sq(P-b) p d[a][b]   - sq(a) sq(P-b) q d[a-1][b]
//                   + sq(P-a) sq(b)   q d[a][b-1] + sq(a) sq(b)   p d[a-1][b-1] )
// with d = 0 outside [0, P) x [0, P) and sq(x) = sqrt(x).
__device__ void half_step(const double* d, double* e, int P, const double* sq, double c) {
  const int Q = P + 1;
  const double rP = 1.0 / (double)P;
  for (int idx = threadIdx.x; idx < Q * Q; idx += blockDim.x) {
    const int a = idx / Q, b = idx - a * Q;
    double v = 0.0;
    if (a < P && b < P) v += sq[P - a] * sq[P - b] * d[a * P + b];
    if (a > 0 && b < P) v -= sq[a] * sq[P - b] * d[(a - 1) * P + b];
    if (a < P && b > 0) v += sq[P - a] * sq[b] * d[a * P + b - 1];
    if (a > 0 && b > 0) v += sq[a] * sq[b] * d[(a - 1) * P + b - 1];
    e[idx] = v * c * rP;
  }
}

// Eq. (Fmm) for one map: the Risbo sweep l = 0..L-1 and the sum over l, by one
// CTA; planes and F_mm' in the scratch array.  F[(m+L-1) M + (m'+L-1)].
__global__ void __launch_bounds__(kWignerThreads) k_noalloc_wigner(int L, int s, const double2* __restrict__ flm,
                                                                   double* scratch) {
  __shared__ double sq[2 * kMaxL + 2];
  double* cur = scratch;
  double* half = scratch + kPlaneStride;
  double* next = scratch + 2 * kPlaneStride;
  double2* F = reinterpret_cast<double2*>(scratch + 3 * kPlaneStride);
  const int M = 2 * L - 1;
  const int as = s < 0 ? -s : s;
  const double c = sqrt(0.5);
  const double inv4pi = 0.25 / 3.14159265358979323846;
  // the previous call's F_mm' is still here: clear it
  for (int i = threadIdx.x; i < M * M; i += blockDim.x) F[i] = make_double2(0.0, 0.0);
  for (int x = threadIdx.x; x < 2 * L + 1; x += blockDim.x) sq[x] = sqrt((double)x);
  if (threadIdx.x == 0) cur[0] = 1.0;  // Delta^0 = [1]
  __syncthreads();
  for (int l = 0; l < L; ++l) {
    if (l > 0) {
      half_step(cur, half, 2 * l - 1, sq, c);  // d^{l-1} -> d^{l-1/2}
      __syncthreads();
      half_step(half, next, 2 * l, sq, c);     // d^{l-1/2} -> d^l
      __syncthreads();
      double* t = cur;
      cur = next;
      next = t;
    }
    if (l < as) continue;
    const int P = 2 * l + 1;
    const double Nl = sqrt((double)P * inv4pi);
    const int col_s = l - s;  // column of m = -s
    // thread order runs along m' so that the F_mm' updates are coalesced
    for (int idx = threadIdx.x; idx < P * P; idx += blockDim.x) {
      const int k = idx / P;        // m + l
      const int i = idx - k * P;    // m' + l
      const double w = Nl * cur[i * P + k] * cur[i * P + col_s];
      const double2 f = flm[l * l + k];
      double2* o = &F[(k - l + L - 1) * M + (i - l + L - 1)];
      o->x += w * f.x;
      o->y += w * f.y;
    }
    // every F entry is updated by a fixed thread within one l and the next
    // half steps hold barriers, so no two updates of one entry overlap
  }
  __syncthreads();
  // times (-1)^s i^-(m+s): a swap and sign changes, exact
  for (int idx = threadIdx.x; idx < M * M; idx += blockDim.x) {
    const int m = idx / M - (L - 1);
    const int r = (((-(m + s)) % 4) + 4) % 4;
    const double sg = (as & 1) ? -1.0 : 1.0;
    const double2 v = F[idx];
    double2 o;
    if (r == 0) o = make_double2(v.x, v.y);
    else if (r == 1) o = make_double2(-v.y, v.x);
    else if (r == 2) o = make_double2(-v.x, -v.y);
    else o = make_double2(v.y, -v.x);
    F[idx] = make_double2(sg * o.x, sg * o.y);
  }
}

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 warp_sum(double2 v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_xor_sync(0xffffffffu, v.x, o);
    v.y += __shfl_xor_sync(0xffffffffu, v.y, o);
  }
  return v;
}

// Eqs. (Fmt) and (f_pfft) for ring t = blockIdx.x, as direct sums over the
// 2L-1 Fourier modes (warp per output, fixed summation order).  The pole ring
// t = L-1 yields only its phi = 0 sample.
__global__ void __launch_bounds__(kSynthThreads) k_noalloc_synthesis(int L, const double* scratch,
                                                                    double2* __restrict__ f) {
  __shared__ double2 w[2 * kDim];  // e^{i pi k / M}, k = 0..2M-1
  __shared__ double2 Fm[kDim];
  const double2* F = reinterpret_cast<const double2*>(scratch + 3 * kPlaneStride);
  const int M = 2 * L - 1, t = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  for (int k = threadIdx.x; k < 2 * M; k += blockDim.x) {
    double sn, cs;
    sincospi((double)k / (double)M, &sn, &cs);
    w[k] = make_double2(cs, sn);
  }
  __syncthreads();
  // theta_t = pi (2t+1)/M: e^{i m' theta_t} = w[m' (2t+1) mod 2M]
  for (int mi = warp; mi < M; mi += nwarps) {
    double2 acc = make_double2(0.0, 0.0);
    for (int j = lane; j < M; j += 32) {
      int a = ((j - (L - 1)) * (2 * t + 1)) % (2 * M);
      if (a < 0) a += 2 * M;
      const double2 p = cmul(F[mi * M + j], w[a]);
      acc.x += p.x;
      acc.y += p.y;
    }
    acc = warp_sum(acc);
    if (lane == 0) Fm[mi] = acc;
  }
  __syncthreads();
  // phi_p = 2 pi p / M: e^{i m phi_p} = w[2 m p mod 2M]
  const int np = (t < L - 1) ? M : 1;
  for (int p = warp; p < np; p += nwarps) {
    double2 acc = make_double2(0.0, 0.0);
    for (int j = lane; j < M; j += 32) {
      int a = (2 * (j - (L - 1)) * p) % (2 * M);
      if (a < 0) a += 2 * M;
      const double2 q = cmul(Fm[j], w[a]);
      acc.x += q.x;
      acc.y += q.y;
    }
    acc = warp_sum(acc);
    if (lane == 0) f[(size_t)t * M + p] = acc;
  }
}

std::mutex g_setup_mutex;
double* g_scratch_ptr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  It is looked up again
// on every call made outside a stream capture (a context reset or a reloaded
// module may place the array elsewhere), and the last address seen is what a
// call made during a capture uses.
mw_status scratch_address(int dev, bool capturing, double** out) {
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!capturing || !g_scratch_ptr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || p == nullptr) {
      cudaGetLastError();
      return MW_ECUDA;
    }
    g_scratch_ptr[dev] = static_cast<double*>(p);
  }
  *out = g_scratch_ptr[dev];
  return MW_OK;
}

// True if ptr is device or managed memory usable on device dev.
bool device_reachable(const void* ptr, int dev) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

}  // namespace

extern "C" mw_status mw_inverse_noalloc(int L, int s, const void* flm_in, void* map_out, void* stream) {
  if (L < 1 || L > kMaxL || s <= -L || s >= L || !flm_in || !map_out) return MW_EINVAL;
  const size_t M = 2 * (size_t)L - 1;
  const size_t in_bytes = 16 * (size_t)L * L, out_bytes = 16 * ((size_t)(L - 1) * M + 1);
  const char* a = static_cast<const char*>(flm_in);
  const char* b = static_cast<const char*>(map_out);
  if (a < b + out_bytes && b < a + in_bytes) return MW_EINVAL;  // overlapping buffers
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return MW_ECUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) return MW_EUNSUPPORTED;
  if (!device_reachable(flm_in, dev) || !device_reachable(map_out, dev)) return MW_EINVAL;
  cudaStream_t cs = static_cast<cudaStream_t>(stream);
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(cs, &cap) != cudaSuccess) {
    cudaGetLastError();
    return MW_ECUDA;
  }
  double* scratch = nullptr;
  const mw_status st = scratch_address(dev, cap != cudaStreamCaptureStatusNone, &scratch);
  if (st != MW_OK) return st;
  k_noalloc_wigner<<<1, kWignerThreads, 0, cs>>>(L, s, static_cast<const double2*>(flm_in), scratch);
  k_noalloc_synthesis<<<L, kSynthThreads, 0, cs>>>(L, scratch, static_cast<double2*>(map_out));
  if (cudaGetLastError() != cudaSuccess) return MW_ECUDA;
  return MW_OK;
}
