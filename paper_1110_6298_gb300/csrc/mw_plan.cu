// mw_plan.cu -- plans, host-side tables and the C entry points of libmw.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "internal.h"

namespace {

// e^{-2 pi i x / n} for integer x, accurate to the last bit of double: the angle
// is formed in long double before rounding.
void unit_root(long long x, long long n, double* re, double* im) {
  x %= n;
  if (x < 0) x += n;
  const long double pi_l = 3.141592653589793238462643383279502884L;
  const long double a = 2.0L * pi_l * (long double)x / (long double)n;
  *re = (double)cosl(a);
  *im = (double)-sinl(a);
}

// Radix sequence of n: 8s, 4s, then 2, 3, 5, 7, then any remaining odd primes.
bool factorize(int n, FftDesc* d) {
  d->n = n;
  d->nrad = 0;
  int r = n;
  while (r % 8 == 0) { d->rad[d->nrad++] = 8; r /= 8; }
  while (r % 4 == 0) { d->rad[d->nrad++] = 4; r /= 4; }
  while (r % 2 == 0) { d->rad[d->nrad++] = 2; r /= 2; }
  for (int p = 3; r > 1; p += 2) {
    while (r % p == 0) {
      if (d->nrad >= 26) return false;
      d->rad[d->nrad++] = p;
      r /= p;
    }
  }
  return true;
}

bool smooth7(int n) {
  for (int p : {2, 3, 5, 7})
    while (n % p == 0) n /= p;
  return n == 1;
}

// Work of one length-n FFT by the stages of fft.cuh, in complex multiply-adds
// per element summed over the stages: about (R + 1) / 2 for a register
// butterfly of radix R; R for a dot-product stage, weighted by 2 in single
// precision (compensated sums) and 1.5 in double (two shared-memory loads per
// term against one per R terms).
double fft_work(const FftDesc& d, bool single) {
  double c = 0.0;
  for (int i = 0; i < d.nrad; ++i) {
    const int R = d.rad[i];
    const bool reg = R == 2 || R == 3 || R == 4 || R == 5 || R == 7 || R == 8 || (single && (R == 11 || R == 13));
    c += (double)d.n * (reg ? 0.5 * (R + 1) : (single ? 2.0 : 1.5) * R);
  }
  return c;
}

// Whether the plan runs its length-M FFTs by Bluestein's convolution through
// the power of two fB.n >= 2M - 1 (two FFTs of that length and three
// pointwise products) instead of M's own radices: the cheaper by fft_work.
// MW_FFT_BLUESTEIN=0 or =1 forces either route for every M.
bool choose_bluestein(const FftDesc& fM, const FftDesc& fB, bool single) {
  if (const char* v = getenv("MW_FFT_BLUESTEIN")) {
    if (v[0] == '0') return false;
    if (v[0] == '1') return true;
  }
  return 2.0 * fft_work(fB, single) + 3.0 * fB.n < fft_work(fM, single);
}

// weight w(k) of Sec. IV-D
void weight(int k, double* re, double* im) {
  *re = 0.0;
  *im = 0.0;
  if (k == 1) { *im = M_PI / 2; return; }
  if (k == -1) { *im = -M_PI / 2; return; }
  if ((k & 1) == 0) *re = 2.0 / (1.0 - (double)k * (double)k);
}

template <typename T>
cudaError_t upload_complex(const std::vector<double>& re, const std::vector<double>& im, void** dst) {
  const size_t n = re.size();
  std::vector<T> h(2 * n);
  for (size_t i = 0; i < n; ++i) { h[2 * i] = (T)re[i]; h[2 * i + 1] = (T)im[i]; }
  cudaError_t e = cudaMalloc(dst, sizeof(T) * 2 * n);
  if (e != cudaSuccess) return e;
  return cudaMemcpy(*dst, h.data(), sizeof(T) * 2 * n, cudaMemcpyHostToDevice);
}

void free_plan(mw_plan* p) {
  if (!p) return;
  for (mw_plan* c : p->subs) free_plan(c);
  for (mw_plan* c : p->twins) free_plan(c);
  if (p->shared_sweep) {
    p->d_S = nullptr; p->d_S32 = nullptr; p->d_err = nullptr; p->d_prog = nullptr; p->d_perm = nullptr;
    p->d_tn_top = nullptr; p->d_tn_exp = nullptr;
  }
  void* ptrs[] = {p->d_groups, p->d_spins, p->d_twM, p->d_twN, p->d_phase, p->d_V, p->d_sqrt, p->d_rsqrt, p->d_upole,
                  p->d_Gt,     p->d_Gp,    p->d_S,   p->d_H,   p->d_map_stage, p->d_flm_stage, p->d_S32, p->d_err,
                  p->d_map_stage2, p->d_flm_stage2,
                  p->d_prog,   p->d_rscale, p->d_nl, p->d_flmf, p->d_moff, p->d_foff, p->d_perm,
                  p->d_qw,     p->d_qpart, p->d_gpack, p->d_sqrt_ff, p->d_rsqrt_ff, p->d_rscale_ff,
                  p->d_tn_top, p->d_tn_exp, p->d_flmT, p->d_tc2_items, p->d_twE, p->d_Ue, p->d_Uo,
                  p->d_chirp, p->d_chirpF, p->d_twB};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
  if (p->cap_stream) cudaStreamDestroy(p->cap_stream);
  if (p->copy_stream) cudaStreamDestroy(p->copy_stream);
  for (auto ev : p->copy_ev) cudaEventDestroy(ev);
  for (auto& r : p->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto ev : p->pool) cudaEventDestroy(ev);
  delete p;
}

mw_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return MW_OK;
  if (e == cudaErrorMemoryAllocation) return MW_ENOMEM;
  return MW_ECUDA;
}

// Build a plan for B maps of band limit L.  moff / foff: caller-buffer offsets of
// each map / f_lm block (NULL: contiguous).  owner: a ragged parent whose sweep
// state (planes, staging, progress and error words) this plan borrows; its row
// stride LD is used.  sweep_only: allocate only the sweep state (ragged parent).
mw_status build_plan(mw_plan** out, int L, int B, const int* spins, unsigned flags, const long long* moff = nullptr,
                     const long long* foff = nullptr, mw_plan* owner = nullptr, bool sweep_only = false) {
  if (!out) return MW_EINVAL;
  *out = nullptr;
  if (L < 1 || L > 2048 || B < 1 || !spins) return MW_EINVAL;
  const int prec = (int)(flags & 0xffu);
  if (prec != MW_PREC_FP64 && prec != MW_PREC_MIXED && prec != MW_PREC_MIXED_TF32X3) return MW_EINVAL;
  if (flags & ~(0xffu | (unsigned)MW_FLAG_GRAPH | (unsigned)MW_FLAG_REAL | (unsigned)MW_FLAG_DELTA_TN |
                (unsigned)MW_FLAG_DELTA_RISBO | (unsigned)MW_FLAG_AUTOTUNE))
    return MW_EINVAL;
  if ((flags & MW_FLAG_DELTA_TN) && (flags & MW_FLAG_DELTA_RISBO)) return MW_EINVAL;
  if ((flags & MW_FLAG_DELTA_TN) && prec == MW_PREC_FP64) return MW_EUNSUPPORTED;
  // default recursion: Trapani-Navaza on the mixed precisions, Risbo on FP64
  if (!(flags & MW_FLAG_DELTA_RISBO) && prec != MW_PREC_FP64) flags |= MW_FLAG_DELTA_TN;
  for (int b = 0; b < B; ++b)
    if (spins[b] <= -L || spins[b] >= L) return MW_EINVAL;
  // real-signal plans: spin 0 only, caller-contiguous buffers, two real maps per complex map
  const bool real = (flags & MW_FLAG_REAL) != 0;
  const int nreal = B;
  std::vector<int> zeros;
  if (real) {
    if (moff || foff || sweep_only) return MW_EINVAL;
    for (int b = 0; b < B; ++b)
      if (spins[b] != 0) return MW_EINVAL;
    B = (B + 1) / 2;
    zeros.assign(B, 0);
    spins = zeros.data();
  }

  mw_plan* p = new (std::nothrow) mw_plan();
  if (!p) return MW_ENOMEM;
  p->L = L;
  p->B = B;
  p->M = 2 * L - 1;
  int N = 4 * L - 3;
  while (!smooth7(N)) ++N;
  p->N = N;
  p->flags = flags;
  p->prec = prec;
  p->LD = owner ? owner->LD : ((L + 1 + 7) / 8) * 8;  // 32-byte aligned plane rows
  cudaGetDevice(&p->device);
  p->spins.assign(spins, spins + B);
  const long long nmw = (long long)(L - 1) * (2 * L - 1) + 1;
  p->moff.resize(B);
  p->foff.resize(B);
  for (int b = 0; b < B; ++b) {
    p->moff[b] = moff ? moff[b] : (long long)b * nmw;
    p->foff[b] = foff ? foff[b] : (long long)b * L * L;
  }
  p->map_elems = (long long)B * nmw;
  p->flm_elems = (long long)B * L * L;
  if (real) {  // caller-facing sizes: nreal real maps and nreal f_lm blocks
    p->real = true;
    p->nreal = nreal;
    p->map_elems = (long long)nreal * nmw;
    p->flm_elems = (long long)nreal * L * L;
  }
  {
    const int nq = real ? nreal : B;
    p->q_L.assign(nq, L);
    p->q_s.resize(nq);
    p->q_moff.resize(nq);
    p->q_foff.resize(nq);
    for (int b = 0; b < nq; ++b) {
      p->q_s[b] = real ? 0 : spins[b];
      p->q_moff[b] = real ? (long long)b * nmw : p->moff[b];
      p->q_foff[b] = real ? (long long)b * L * L : p->foff[b];
    }
  }
  {
    // even-lag halves of the forward convolution: even m'' = 2j, |2j| <= L-1,
    // outputs m' = 2i in [0, L-1]; odd m'' = 2j+1, outputs m' = 2i+1; a
    // circular convolution of length NE is exact once NE covers every lag
    // j - i that occurs
    const int je = (L - 1) / 2;
    const int jo_min = -(L / 2), jo_max = (L - 2) / 2;
    const int span_e = 3 * je + 1;
    const int span_o = jo_max >= jo_min ? jo_max - (jo_min - jo_max) + 1 : 1;
    int NE = span_e > span_o ? span_e : span_o;
    while (!smooth7(NE)) ++NE;
    p->NE = NE;
  }
  if (!factorize(p->M, &p->fM) || !factorize(p->N, &p->fN) || !factorize(p->NE, &p->fE)) {
    free_plan(p);
    return MW_EUNSUPPORTED;
  }

  // spin groups (order of first appearance; at most kMaxGroupMaps maps each,
  // kTcGroupMaps on the tensor-core path)
  const int gmax = kTcGroupMaps;
  for (int b = 0; b < B; ++b) {
    SpinGroup* g = nullptr;
    for (auto& h : p->groups)
      if (h.s == spins[b] && h.nb < gmax) g = &h;
    if (!g) {
      SpinGroup ng{};
      ng.s = spins[b];
      ng.nb = 0;
      p->groups.push_back(ng);
      g = &p->groups.back();
    }
    g->maps[g->nb++] = b;
  }

  cudaError_t e = cudaSuccess;
  auto chk = [&](cudaError_t x) { if (e == cudaSuccess) e = x; };
  size_t ws = 0;
  auto alloc = [&](void** dst, size_t bytes) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(dst, bytes);
    ws += bytes;
  };

  // tables
  const int M = p->M;
  std::vector<double> re, im;
  auto twiddles = [&](int n) {
    re.assign(n, 0.0); im.assign(n, 0.0);
    for (int k = 0; k < n; ++k) unit_root(k, n, &re[k], &im[k]);
  };
  const bool dbl = prec == MW_PREC_FP64;
  if (!sweep_only) {
  twiddles(M);
  chk(dbl ? upload_complex<double>(re, im, &p->d_twM) : upload_complex<float>(re, im, &p->d_twM));
  twiddles(N);
  chk(dbl ? upload_complex<double>(re, im, &p->d_twN) : upload_complex<float>(re, im, &p->d_twN));
  // Bluestein tables: c_n = e^{-i pi n^2 / M} = e^{-2 pi i (n^2 mod 2M) / (2M)},
  // and the DFT of b_j = conj(c_|j|), |j| < M, placed circularly in length NB:
  // b is even in j, so DFT_NB(b)_k = b_0 + 2 sum_{j=1}^{M-1} b_j cos(2 pi j k / NB)
  {
    int NB = 1;
    while (NB < 2 * M - 1) NB *= 2;
    factorize(NB, &p->fB);
  }
  p->bluestein = choose_bluestein(p->fM, p->fB, !dbl);
  if (p->bluestein) {
    const int NB = p->fB.n;
    std::vector<double> cr(M), ci(M);
    for (int n = 0; n < M; ++n) unit_root(((long long)n * n) % (2LL * M), 2LL * M, &cr[n], &ci[n]);
    chk(dbl ? upload_complex<double>(cr, ci, &p->d_chirp) : upload_complex<float>(cr, ci, &p->d_chirp));
    twiddles(NB);
    chk(dbl ? upload_complex<double>(re, im, &p->d_twB) : upload_complex<float>(re, im, &p->d_twB));
    std::vector<double> cosB(re);  // cos(2 pi x / NB)
    re.assign(NB, 0.0); im.assign(NB, 0.0);
    for (int k = 0; k < NB; ++k) {
      double sr = cr[0], si = -ci[0];
      long long x = 0;
      for (int j = 1; j < M; ++j) {
        x += k;
        if (x >= NB) x -= NB;
        sr += 2.0 * cr[j] * cosB[x];
        si -= 2.0 * ci[j] * cosB[x];
      }
      re[k] = sr / NB;
      im[k] = si / NB;
    }
    chk(dbl ? upload_complex<double>(re, im, &p->d_chirpF) : upload_complex<float>(re, im, &p->d_chirpF));
  }
  // e^{-i pi m' / M} = e^{-2 pi i m' / (2M)}
  re.assign(M, 0.0); im.assign(M, 0.0);
  for (int i = 0; i < M; ++i) unit_root(i - (L - 1), 2LL * M, &re[i], &im[i]);
  chk(dbl ? upload_complex<double>(re, im, &p->d_phase) : upload_complex<float>(re, im, &p->d_phase));
  // V_j = sum_{|k| <= 2L-2} w(k) e^{-2 pi i j k / N} / (N M)
  {
    std::vector<double> cr(N), ci(N);
    for (int x = 0; x < N; ++x) unit_root(x, N, &cr[x], &ci[x]);
    re.assign(N, 0.0); im.assign(N, 0.0);
    for (int j = 0; j < N; ++j) {
      double sr = 0.0, si = 0.0;
      for (int k = -(2 * L - 2); k <= 2 * L - 2; ++k) {
        double wr, wi;
        weight(k, &wr, &wi);
        if (wr == 0.0 && wi == 0.0) continue;
        long long x = ((long long)j * k) % N;
        if (x < 0) x += N;
        sr += wr * cr[x] - wi * ci[x];
        si += wr * ci[x] + wi * cr[x];
      }
      re[j] = sr / ((double)N * M);
      im[j] = si / ((double)N * M);
    }
    chk(dbl ? upload_complex<double>(re, im, &p->d_V) : upload_complex<float>(re, im, &p->d_V));
  }
  {
    // U_k = sum_{d in [d0, d1]} w(2d) e^{-2 pi i k d / NE} / (NE M) for the even
    // half (d = j - i, j in [-je, je], i in [0, je]) and the odd half
    // (j in [jo_min, jo_max], i in [0, jo_max])
    const int NE = p->NE;
    twiddles(NE);
    chk(dbl ? upload_complex<double>(re, im, &p->d_twE) : upload_complex<float>(re, im, &p->d_twE));
    std::vector<double> cr(NE), ci(NE);
    for (int x = 0; x < NE; ++x) unit_root(x, NE, &cr[x], &ci[x]);
    const int je = (L - 1) / 2, jo_min = -(L / 2), jo_max = (L - 2) / 2;
    auto kernel_dft = [&](int d0, int d1, void** dst) {
      re.assign(NE, 0.0); im.assign(NE, 0.0);
      for (int k = 0; k < NE; ++k) {
        double sr = 0.0, si = 0.0;
        for (int d = d0; d <= d1; ++d) {
          double wr, wi;
          weight(2 * d, &wr, &wi);
          long long x = ((long long)k * d) % NE;
          if (x < 0) x += NE;
          sr += wr * cr[x];
          si += wr * ci[x];
        }
        re[k] = sr / ((double)NE * M);
        im[k] = si / ((double)NE * M);
      }
      chk(dbl ? upload_complex<double>(re, im, dst) : upload_complex<float>(re, im, dst));
    };
    kernel_dft(-2 * je, je, &p->d_Ue);
    if (jo_max >= jo_min) kernel_dft(jo_min - jo_max, jo_max, &p->d_Uo);
    else kernel_dft(0, 0, &p->d_Uo);
  }
  }  // !sweep_only
  {
    std::vector<double> sq(2 * L + 3);
    for (size_t k = 0; k < sq.size(); ++k) sq[k] = std::sqrt((double)k);
    alloc((void**)&p->d_sqrt, sizeof(double) * sq.size());
    if (e == cudaSuccess) chk(cudaMemcpy(p->d_sqrt, sq.data(), sizeof(double) * sq.size(), cudaMemcpyHostToDevice));
    std::vector<double> rq(sq.size(), 0.0);
    for (size_t k = 1; k < rq.size(); ++k) rq[k] = 1.0 / std::sqrt((double)k);
    alloc((void**)&p->d_rsqrt, sizeof(double) * rq.size());
    if (e == cudaSuccess) chk(cudaMemcpy(p->d_rsqrt, rq.data(), sizeof(double) * rq.size(), cudaMemcpyHostToDevice));
  }
  if (!sweep_only) {  // u(m') = sum_{|m''| <= L-1} (-1)^{m''} conj(w(m''-m')); folded u(m') + u(-m') for m' > 0
    auto u = [&](int mp, double* ur, double* ui) {
      double sr = 0.0, si = 0.0;
      for (int mpp = -(L - 1); mpp <= L - 1; ++mpp) {
        double wr, wi;
        weight(mpp - mp, &wr, &wi);
        const double sg = (mpp & 1) ? -1.0 : 1.0;
        sr += sg * wr;
        si -= sg * wi;
      }
      *ur = sr; *ui = si;
    };
    std::vector<double> up(2 * L);
    for (int mp = 0; mp < L; ++mp) {
      double ar, ai, br = 0.0, bi = 0.0;
      u(mp, &ar, &ai);
      if (mp > 0) u(-mp, &br, &bi);
      up[2 * mp] = ar + br;
      up[2 * mp + 1] = ai + bi;
    }
    alloc((void**)&p->d_upole, sizeof(double) * up.size());
    if (e == cudaSuccess) chk(cudaMemcpy(p->d_upole, up.data(), sizeof(double) * up.size(), cudaMemcpyHostToDevice));
  }
  {
    std::vector<double> rs(2 * L + 2, 0.0), nlv(L);
    for (int k = 1; k < (int)rs.size(); ++k) rs[k] = 1.0 / (std::sqrt(2.0) * (double)k);
    for (int l = 0; l < L; ++l) nlv[l] = std::sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
    alloc((void**)&p->d_rscale, sizeof(double) * rs.size());
    if (e == cudaSuccess) chk(cudaMemcpy(p->d_rscale, rs.data(), sizeof(double) * rs.size(), cudaMemcpyHostToDevice));
    alloc((void**)&p->d_nl, sizeof(double) * nlv.size());
    if (e == cudaSuccess) chk(cudaMemcpy(p->d_nl, nlv.data(), sizeof(double) * nlv.size(), cudaMemcpyHostToDevice));
  }
  if (!dbl) {  // float-float copies of the recursion's tables, split from long-double values
    auto ff_table = [&](float2** dst, size_t n, auto fn) {
      std::vector<float2> h(n);
      for (size_t k = 0; k < n; ++k) {
        const long double v = fn((long double)k);
        const float hi = (float)v;
        h[k] = make_float2(hi, (float)(v - (long double)hi));
      }
      alloc((void**)dst, sizeof(float2) * n);
      if (e == cudaSuccess) chk(cudaMemcpy(*dst, h.data(), sizeof(float2) * n, cudaMemcpyHostToDevice));
    };
    ff_table(&p->d_sqrt_ff, 2 * (size_t)L + 3, [](long double k) { return sqrtl(k); });
    ff_table(&p->d_rsqrt_ff, 2 * (size_t)L + 3, [](long double k) { return k > 0 ? 1.0L / sqrtl(k) : 0.0L; });
    ff_table(&p->d_rscale_ff, 2 * (size_t)L + 2,
             [](long double k) { return k > 0 ? 1.0L / (sqrtl(2.0L) * k) : 0.0L; });
  }
  alloc((void**)&p->d_spins, sizeof(int) * B);
  if (e == cudaSuccess) chk(cudaMemcpy(p->d_spins, spins, sizeof(int) * B, cudaMemcpyHostToDevice));
  alloc((void**)&p->d_moff, sizeof(long long) * B);
  if (e == cudaSuccess) chk(cudaMemcpy(p->d_moff, p->moff.data(), sizeof(long long) * B, cudaMemcpyHostToDevice));
  alloc((void**)&p->d_foff, sizeof(long long) * B);
  if (e == cudaSuccess) chk(cudaMemcpy(p->d_foff, p->foff.data(), sizeof(long long) * B, cudaMemcpyHostToDevice));
  alloc((void**)&p->d_groups, sizeof(SpinGroup) * p->groups.size());
  if (e == cudaSuccess)
    chk(cudaMemcpy(p->d_groups, p->groups.data(), sizeof(SpinGroup) * p->groups.size(), cudaMemcpyHostToDevice));

  // workspace
  const size_t fsz = dbl ? sizeof(double2) : sizeof(float2);
  if (!sweep_only) {
    alloc(&p->d_Gt, fsz * (size_t)B * M * L);
    alloc((void**)&p->d_Gp, sizeof(double2) * (size_t)B * M * L);
    if (prec == MW_PREC_MIXED_TF32X3) alloc((void**)&p->d_flmf, sizeof(float2) * (size_t)B * L * L);
    if (prec == MW_PREC_MIXED_BF16X3) alloc((void**)&p->d_flmT, sizeof(float2) * (size_t)B * p->M * L);
    if (real) alloc((void**)&p->d_gpack, sizeof(double2) * (size_t)B * L * L);
  }
  if (owner) {  // borrow the parent's sweep state
    p->shared_sweep = true;
    p->d_S = owner->d_S;
    p->d_S32 = owner->d_S32;
    p->d_err = owner->d_err;
    p->d_prog = owner->d_prog;
    p->d_perm = owner->d_perm;
    p->d_tn_top = owner->d_tn_top;
    p->d_tn_exp = owner->d_tn_exp;
    p->risbo_grid = owner->risbo_grid;
  } else {
    const size_t plane = (size_t)p->LD * p->LD;
    alloc((void**)&p->d_S, sizeof(double) * (dbl ? (size_t)kChunk : 2) * plane);
    if (!dbl) alloc((void**)&p->d_S32, sizeof(float) * (size_t)(L < kTcChunk ? L : kTcChunk) * plane);
    alloc((void**)&p->d_err, sizeof(int));
    if (e == cudaSuccess) chk(cudaMemset(p->d_err, 0, sizeof(int)));
    {
      const int Tm = (L + 1 + 31) / 32;
      alloc((void**)&p->d_prog, sizeof(int) * (size_t)(Tm * (Tm + 1) / 2 + 1));
    }
    if (flags & MW_FLAG_DELTA_TN) {
      // top rows Delta^l_{l,m} = (-1)^(l-m) 2^-l sqrt(C(2l, l+m)) as mantissa * 2^exponent:
      // Delta^l_{l,l} = 2^-l, and Delta^l_{l,m} = -(1/2) sqrt(2l (2l-1) / ((l+m)(l-m))) Delta^{l-1}_{l-1,m}
      // for m < l, in long double with the mantissa renormalised after every factor
      const size_t nt = (size_t)L * (L + 1) / 2;
      std::vector<float2> tm(nt);
      std::vector<int> te(nt);
      std::vector<long double> mt(L);
      std::vector<int> ex(L);
      for (int l = 0; l < L; ++l) {
        for (int m = 0; m < l; ++m) {
          const long double r2 = (long double)(2 * l) * (2 * l - 1) / ((long double)(l + m) * (l - m));
          int k = 0;
          mt[m] = frexpl(mt[m] * (-0.5L * sqrtl(r2)), &k);
          ex[m] += k;
        }
        mt[l] = 0.5L;
        ex[l] = 1 - l;
        const size_t t0 = (size_t)l * (l + 1) / 2;
        for (int m = 0; m <= l; ++m) {
          const float hi = (float)mt[m];
          tm[t0 + m] = make_float2(hi, (float)(mt[m] - (long double)hi));
          te[t0 + m] = ex[m];
        }
      }
      alloc((void**)&p->d_tn_top, sizeof(float2) * nt);
      if (e == cudaSuccess) chk(cudaMemcpy(p->d_tn_top, tm.data(), sizeof(float2) * nt, cudaMemcpyHostToDevice));
      alloc((void**)&p->d_tn_exp, sizeof(int) * nt);
      if (e == cudaSuccess) chk(cudaMemcpy(p->d_tn_exp, te.data(), sizeof(int) * nt, cudaMemcpyHostToDevice));
    }
    if (e == cudaSuccess && prec == MW_PREC_MIXED_BF16X3) chk(make_tc2_tensor_maps(p));
    if (e == cudaSuccess) {
      int nsm = 0;
      chk(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
      p->risbo_grid = nsm * risbo_blocks_per_sm(p->prec);
      if (e == cudaSuccess) chk(make_risbo_perm(p));
    }
  }
  if (e == cudaSuccess && !sweep_only && prec == MW_PREC_MIXED_BF16X3) {
    // spin groups per pass of the contraction pipeline: 2 (both groups of a
    // plane tile in one pass) unless MW_TC2_GROUPS=1; results do not depend on it
    if (const char* env = getenv("MW_TC2_GROUPS")) p->tc2_ng = (atoi(env) == 1) ? 1 : 2;
    p->chunk = owner ? owner->chunk : p->chunk;
    p->tn_threads = owner ? owner->tn_threads : p->tn_threads;
    chk(make_tc2_items(p, p->chunk));
  }
  if (e != cudaSuccess) {
    const mw_status st = from_cuda(e);
    cudaGetLastError();
    free_plan(p);
    return st;
  }
  p->ws_bytes = ws;
  *out = p;
  return MW_OK;
}

bool is_device_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// page-locked host memory (cudaMallocHost / cudaHostRegister): copies from and
// to it run asynchronously, so they can overlap kernels
bool is_pinned_host_ptr(const void* ptr) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, ptr) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeHost;
}

// FFT stages of every map of a plan (the launchers also take a map range)
cudaError_t phi_forward_all(const mw_plan* c, const double2* m, cudaStream_t st) { return launch_phi_forward(c, m, st); }
cudaError_t phi_inverse_all(const mw_plan* c, double2* m, cudaStream_t st) { return launch_phi_inverse(c, m, st); }
cudaError_t theta_forward_all(const mw_plan* c, cudaStream_t st) { return launch_theta_forward(c, st); }
cudaError_t theta_inverse_all(const mw_plan* c, cudaStream_t st) { return launch_theta_inverse(c, st); }

// Forward or inverse of a uniform complex plan with a pinned host input and/or
// output: the host copies run on the plan's copy stream in pieces that
// overlap the compute on st.
//   forward: the maps are copied in groups; the phi and theta stages of a
//            group start as soon as its copy has landed, while the next
//            group's copy runs; the f_lm rows of a chunk of planes are
//            copied back as soon as that chunk's contraction has written them.
//   inverse: f_lm is copied chunk of planes by chunk of planes (the rows
//            l0..l1-1 a chunk's contraction reads), all copies queued at the
//            start, each chunk's contraction waiting for its own; the theta
//            and phi stages run group by group and each group's maps are
//            copied back while the next group computes.
// Device-side inputs or outputs skip their copies.  Returns after the host
// output is written (st synchronised), as the staged path does.
struct PinnedCopies {
  mw_plan* p;
  cudaStream_t st, cp;
  double2* flm_host;   // forward: host f_lm (null: device output)
  const double2* flm_dev;
  int next_ev;
};

cudaError_t next_event(mw_plan* p, int* k, cudaEvent_t* ev) {
  if (*k >= (int)p->copy_ev.size()) {
    cudaEvent_t e;
    const cudaError_t r = cudaEventCreateWithFlags(&e, cudaEventDisableTiming);
    if (r != cudaSuccess) return r;
    p->copy_ev.push_back(e);
  }
  *ev = p->copy_ev[(*k)++];
  return cudaSuccess;
}

// st -> cp ordering: cp waits for the work enqueued on st so far
cudaError_t order(mw_plan* p, int* k, cudaStream_t from, cudaStream_t to) {
  cudaEvent_t ev;
  cudaError_t e = next_event(p, k, &ev);
  if (e == cudaSuccess) e = cudaEventRecord(ev, from);
  if (e == cudaSuccess) e = cudaStreamWaitEvent(to, ev, 0);
  return e;
}

cudaError_t copy_flm_rows(void* ctx, int l0, int l1) {
  PinnedCopies* c = static_cast<PinnedCopies*>(ctx);
  mw_plan* p = c->p;
  if (l1 > p->L) l1 = p->L;
  cudaError_t e = order(p, &c->next_ev, c->st, c->cp);
  if (e != cudaSuccess) return e;
  const size_t pitch = sizeof(double2) * (size_t)p->L * p->L;
  const size_t off = (size_t)l0 * l0, width = sizeof(double2) * ((size_t)l1 * l1 - off);
  return cudaMemcpy2DAsync(c->flm_host + off, pitch, c->flm_dev + off, pitch, width, p->B, cudaMemcpyDeviceToHost,
                           c->cp);
}

// Inverse from a pinned host f_lm: every chunk's rows [l0^2, l1^2) of every map
// are copied on the copy stream as soon as the call starts (one pitched copy
// per chunk, each followed by an event); just before a chunk's contraction the
// compute stream waits for that chunk's copy and, on the BF16x3 path,
// transposes those rows, so only the first chunk's copy is exposed.
struct PinnedUploads {
  mw_plan* p;
  cudaStream_t st;
  std::vector<cudaEvent_t> ev;  // per chunk
  int chunk;
  const double2* flm_dev;
  bool transpose;
  int launches;
};

cudaError_t upload_ready(void* ctx, int l0, int l1) {
  PinnedUploads* u = static_cast<PinnedUploads*>(ctx);
  cudaError_t e = cudaStreamWaitEvent(u->st, u->ev[l0 / u->chunk], 0);
  if (e == cudaSuccess && u->transpose) {
    e = launch_flm_transpose(u->p, u->flm_dev, u->st, l0, l1);
    ++u->launches;
  }
  return e;
}

cudaError_t run_pinned(mw_plan* p, bool forward, const void* in, void* out, bool in_dev, bool out_dev,
                       const double2* din, double2* dout, cudaStream_t st, int* nl) {
  cudaError_t e = cudaSuccess;
  if (!p->copy_stream) {
    e = cudaStreamCreateWithFlags(&p->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) return e;
  }
  cudaStream_t cp = p->copy_stream;
  int k = 0;
  const int B = p->B;
  const int gm = B <= 8 ? 1 : (B + 7) / 8;  // maps per group: at most 8 groups
  const size_t map_b = sizeof(double2) * (size_t)((long long)(p->L - 1) * p->M + 1);
  std::vector<mw_plan*> cs{p};
  if ((e = order(p, &k, st, cp)) != cudaSuccess) return e;  // the copies follow earlier work on st
  if (forward) {
    for (int b0 = 0; b0 < B && e == cudaSuccess; b0 += gm) {
      const int nb = b0 + gm <= B ? gm : B - b0;
      if (!in_dev) {
        e = cudaMemcpyAsync((double2*)din + p->moff[b0], (const double2*)in + p->moff[b0], map_b * nb,
                            cudaMemcpyHostToDevice, cp);
        if (e == cudaSuccess) e = order(p, &k, cp, st);
        if (e != cudaSuccess) break;
      }
      {
        StageSpan sp(p, MW_STAGE_PHI, st);
        e = launch_phi_forward(p, din, st, b0, nb);
        sp.end(1);
      }
      if (e == cudaSuccess) {
        StageSpan sp(p, MW_STAGE_THETA, st);
        e = launch_theta_forward(p, st, b0, nb);
        sp.end(1);
      }
      *nl += 2;
    }
    if (e != cudaSuccess) return e;
    WignerJob job{p, 0, nullptr, dout};
    PinnedCopies pc{p, st, cp, out_dev ? nullptr : (double2*)out, dout, k};
    ChunkHook hook{copy_flm_rows, &pc};
    e = run_wigner(p, &job, 1, st, nl, out_dev ? nullptr : &hook);
    k = pc.next_ev;
  } else {
    if (!in_dev && p->prec != MW_PREC_MIXED_TF32X3) {
      PinnedUploads up{p, st, {}, p->prec == MW_PREC_FP64 ? kChunk : p->chunk, din,
                       p->prec == MW_PREC_MIXED_BF16X3, 0};
      const size_t pitch = sizeof(double2) * (size_t)p->L * p->L;
      for (int l0 = 0; l0 < p->L && e == cudaSuccess; l0 += up.chunk) {
        const int l1 = l0 + up.chunk < p->L ? l0 + up.chunk : p->L;
        const size_t off = (size_t)l0 * l0, width = sizeof(double2) * ((size_t)l1 * l1 - off);
        e = cudaMemcpy2DAsync((double2*)din + off, pitch, (const double2*)in + off, pitch, width, (size_t)B,
                              cudaMemcpyHostToDevice, cp);
        cudaEvent_t ev = nullptr;
        if (e == cudaSuccess) e = next_event(p, &k, &ev);
        if (e == cudaSuccess) e = cudaEventRecord(ev, cp);
        up.ev.push_back(ev);
      }
      WignerJob job{p, 1, din, nullptr, up.transpose};
      ChunkHook hook{nullptr, &up, upload_ready};
      if (e == cudaSuccess) e = run_wigner(p, &job, 1, st, nl, &hook);
      *nl += up.launches;
    } else {
      if (!in_dev) e = cudaMemcpyAsync((double2*)din, in, sizeof(double2) * (size_t)p->flm_elems,
                                       cudaMemcpyHostToDevice, st);
      WignerJob job{p, 1, din, nullptr};
      if (e == cudaSuccess) e = run_wigner(p, &job, 1, st, nl);
    }
    for (int b0 = 0; b0 < B && e == cudaSuccess; b0 += gm) {
      const int nb = b0 + gm <= B ? gm : B - b0;
      {
        StageSpan sp(p, MW_STAGE_THETA, st);
        e = launch_theta_inverse(p, st, b0, nb);
        sp.end(1);
      }
      if (e == cudaSuccess) {
        StageSpan sp(p, MW_STAGE_PHI, st);
        e = launch_phi_inverse(p, dout, st, b0, nb);
        sp.end(1);
      }
      *nl += 2;
      if (e == cudaSuccess && !out_dev) {
        e = order(p, &k, st, cp);
        if (e == cudaSuccess)
          e = cudaMemcpyAsync((double2*)out + p->moff[b0], dout + p->moff[b0], map_b * nb, cudaMemcpyDeviceToHost,
                              cp);
      }
    }
  }
  if (e == cudaSuccess) e = order(p, &k, cp, st);  // st resumes after the last copy
  if (e == cudaSuccess && !out_dev) e = cudaStreamSynchronize(st);
  return e;
}

enum Direction { kForward, kInverse, kForwardAdjoint, kInverseAdjoint, kFused };

// Twins for fused forward+inverse calls: one per consumer plan (the plan
// itself, or each sub-plan of a ragged plan), borrowing p's sweep state.
mw_status ensure_twins(mw_plan* p) {
  if (!p->twins.empty()) return MW_OK;
  std::vector<mw_plan*> src;
  if (p->subs.empty()) src.push_back(p);
  else src = p->subs;
  for (mw_plan* q : src) {
    mw_plan* t = nullptr;
    const mw_status st =
        q->real ? build_plan(&t, q->L, q->nreal, std::vector<int>(q->nreal, 0).data(), q->flags, nullptr, nullptr, p)
                : build_plan(&t, q->L, q->B, q->spins.data(), q->flags, q->moff.data(), q->foff.data(), p, false);
    if (st != MW_OK) {
      for (mw_plan* u : p->twins) {
        p->ws_bytes -= u->ws_bytes;
        free_plan(u);
      }
      p->twins.clear();
      return st;
    }
    if (t->prec == MW_PREC_MIXED_BF16X3 && t->tc2_ng != q->tc2_ng) {  // the source plan's tuning
      t->tc2_ng = q->tc2_ng;
      const cudaError_t e = make_tc2_items(t, p->chunk);
      if (e != cudaSuccess) {
        cudaGetLastError();
        free_plan(t);
        return from_cuda(e);
      }
    }
    p->twins.push_back(t);
    p->ws_bytes += t->ws_bytes;
  }
  return MW_OK;
}

// One call.  For kFused, (in, out) = (map_in, flm_out) of the forward half and
// (in2, out2) = (flm_in, map_out) of the inverse half; otherwise in2/out2 are
// unused.
mw_status run(mw_plan* p, Direction dir, const void* in, void* out, void* stream, const void* in2 = nullptr,
              void* out2 = nullptr) {
  if (!p || !in || !out) return MW_EINVAL;
  const bool fused = dir == kFused;
  if (fused && (!in2 || !out2)) return MW_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  if (fused) {
    const mw_status ts = ensure_twins(p);
    if (ts != MW_OK) return ts;
  }
  // consumers: the plan itself, or the per-band-limit sub-plans of a ragged plan
  std::vector<mw_plan*> cs;
  if (p->subs.empty()) cs.push_back(p);
  else cs = p->subs;
  const bool real = p->real;
  if (real && (dir == kForwardAdjoint || dir == kInverseAdjoint)) return MW_EUNSUPPORTED;
  // buffer sizes in bytes: complex doubles, or real doubles for the maps of a real plan
  const size_t nmw = (size_t)p->map_elems * (real ? sizeof(double) : sizeof(double2));
  const size_t nlm = (size_t)p->flm_elems * sizeof(double2);
  const bool map_in = (dir == kForward || dir == kInverseAdjoint || fused);
  const size_t in_bytes = map_in ? nmw : nlm, out_bytes = map_in ? nlm : nmw;
  cudaError_t e = cudaSuccess;
  auto ensure = [&](double2** slot, size_t bytes) {
    if (e != cudaSuccess || *slot) return;
    e = cudaMalloc((void**)slot, bytes);
    if (e == cudaSuccess) p->ws_bytes += bytes;
  };
  // host buffers are staged through plan-owned device buffers (allocated on first use)
  const double2* din = (const double2*)in;
  double2* dout = (double2*)out;
  const double2* din2 = (const double2*)in2;
  double2* dout2 = (double2*)out2;
  double2** in_slot = map_in ? &p->d_map_stage : &p->d_flm_stage;
  double2** out_slot = map_in ? &p->d_flm_stage : &p->d_map_stage;
  const bool in_dev = is_device_ptr(in), out_dev = is_device_ptr(out);
  const bool in2_dev = !fused || is_device_ptr(in2), out2_dev = !fused || is_device_ptr(out2);
  if (!in_dev) ensure(in_slot, in_bytes);
  if (!out_dev) ensure(out_slot, out_bytes);
  if (!in2_dev) ensure(&p->d_flm_stage2, nlm);
  if (!out2_dev) ensure(&p->d_map_stage2, nmw);
  if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
  // pinned host buffers of a uniform complex plan: overlapped copies
  if (!fused && !real && p->subs.empty() && (dir == kForward || dir == kInverse) && (!in_dev || !out_dev) &&
      (in_dev || is_pinned_host_ptr(in)) && (out_dev || is_pinned_host_ptr(out))) {
    int nl = 0;
    e = run_pinned(p, dir == kForward, in, out, in_dev, out_dev, in_dev ? din : *in_slot, out_dev ? dout : *out_slot,
                   st, &nl);
    p->last_launches = nl;
    return from_cuda(e);
  }
  if (!in_dev) {
    e = cudaMemcpyAsync(*in_slot, in, in_bytes, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return from_cuda(e);
    din = *in_slot;
  }
  if (!in2_dev) {
    e = cudaMemcpyAsync(p->d_flm_stage2, in2, nlm, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return from_cuda(e);
    din2 = p->d_flm_stage2;
  }
  if (!out_dev) dout = *out_slot;
  if (!out2_dev) dout2 = p->d_map_stage2;

  int nl = 0;
  auto enqueue = [&](cudaStream_t st) -> cudaError_t {
  // one FFT stage for every consumer in cl, timed as one span on the plan
  auto stage = [&](const std::vector<mw_plan*>& cl, int stg, cudaError_t (*fn)(const mw_plan*, cudaStream_t)) {
    if (e != cudaSuccess) return;
    StageSpan sp(p, stg, st);
    for (mw_plan* c : cl) {
      if (e == cudaSuccess) e = fn(c, st);
      ++nl;
    }
    sp.end((int)cl.size());
  };
  auto phi = [&](const std::vector<mw_plan*>& cl, auto fn, auto ptr) {
    if (e != cudaSuccess) return;
    StageSpan sp(p, MW_STAGE_PHI, st);
    for (mw_plan* c : cl) {
      if (e == cudaSuccess) e = fn(c, ptr, st);
      ++nl;
    }
    sp.end((int)cl.size());
  };
  auto wigner = [&](const std::vector<mw_plan*>& fwd, double2* flm_out, const std::vector<mw_plan*>& inv,
                    const double2* flm_in) {
    if (e != cudaSuccess) return;
    std::vector<WignerJob> jobs;
    for (mw_plan* c : fwd) jobs.push_back({c, 0, nullptr, flm_out});
    for (mw_plan* c : inv) jobs.push_back({c, 1, flm_in, nullptr});
    e = run_wigner(p, jobs.data(), (int)jobs.size(), st, &nl);
  };
  const std::vector<mw_plan*> none;
  // real plans: f_lm pack (caller -> packed workspace) and unpack (packed -> caller)
  auto pack = [&](mw_plan* c, const double2* flm) {
    if (e != cudaSuccess) return;
    StageSpan sp(p, MW_STAGE_PHI, st);
    e = launch_real_pack(c, flm, c->d_gpack, st);
    ++nl;
    sp.end(1);
  };
  auto unpack = [&](mw_plan* c, double2* flm) {
    if (e != cudaSuccess) return;
    StageSpan sp(p, MW_STAGE_PHI, st);
    e = launch_real_unpack(c, c->d_gpack, flm, st);
    ++nl;
    sp.end(1);
  };
  if (real) {  // one consumer (no ragged real plans)
    mw_plan* c = cs[0];
    switch (dir) {
      case kForward:
        phi(cs, launch_phi_forward_real, (const double*)din);
        stage(cs, MW_STAGE_THETA, theta_forward_all);
        wigner(cs, c->d_gpack, none, nullptr);
        unpack(c, dout);
        break;
      case kInverse:
        pack(c, din);
        wigner(none, nullptr, cs, c->d_gpack);
        stage(cs, MW_STAGE_THETA, theta_inverse_all);
        phi(cs, launch_phi_inverse_real, (double*)dout);
        break;
      case kFused: {
        mw_plan* t = p->twins[0];
        phi(cs, launch_phi_forward_real, (const double*)din);
        stage(cs, MW_STAGE_THETA, theta_forward_all);
        pack(t, din2);
        wigner(cs, c->d_gpack, p->twins, t->d_gpack);
        unpack(c, dout);
        stage(p->twins, MW_STAGE_THETA, theta_inverse_all);
        phi(p->twins, launch_phi_inverse_real, (double*)dout2);
        break;
      }
      default:
        break;
    }
    return e;
  }
  switch (dir) {
    case kForward:
      phi(cs, phi_forward_all, din);
      stage(cs, MW_STAGE_THETA, theta_forward_all);
      wigner(cs, dout, none, nullptr);
      break;
    case kInverse:
      wigner(none, nullptr, cs, din);
      stage(cs, MW_STAGE_THETA, theta_inverse_all);
      phi(cs, phi_inverse_all, dout);
      break;
    case kForwardAdjoint:
      wigner(none, nullptr, cs, din);
      stage(cs, MW_STAGE_THETA, launch_theta_forward_adjoint);
      phi(cs, launch_phi_forward_adjoint, dout);
      phi(cs, launch_pole_forward_adjoint, dout);
      break;
    case kInverseAdjoint:
      phi(cs, launch_phi_inverse_adjoint, din);
      stage(cs, MW_STAGE_THETA, launch_theta_inverse_adjoint);
      wigner(cs, dout, none, nullptr);
      break;
    case kFused:  // forward half on cs, inverse half on the twins, one sweep for both
      phi(cs, phi_forward_all, din);
      stage(cs, MW_STAGE_THETA, theta_forward_all);
      wigner(cs, dout, p->twins, din2);
      stage(p->twins, MW_STAGE_THETA, theta_inverse_all);
      phi(p->twins, phi_inverse_all, dout2);
      break;
  }
  return e;
  };
  // CUDA graph: captured on the first call with these buffers, replayed after
  bool ran = false;
  const void* k_in2 = fused ? (const void*)din2 : nullptr;
  void* k_out2 = fused ? (void*)dout2 : nullptr;
  if ((p->flags & MW_FLAG_GRAPH) && !p->timing && !p->graph_failed) {
    for (auto& g : p->graphs)
      if (g.dir == (int)dir && g.in == (const void*)din && g.out == (void*)dout && g.in2 == k_in2 && g.out2 == k_out2) {
        e = cudaGraphLaunch(g.exec, st);
        p->last_launches = 1;
        ran = true;
        break;
      }
    if (!ran) {
      // capture on a plan-owned stream (the caller's may be the legacy default
      // stream, which cannot be captured); capturing runs nothing, and the
      // graph is then launched on the caller's stream
      cudaGraph_t graph = nullptr;
      cudaGraphExec_t exec = nullptr;
      cudaError_t ce = cudaSuccess;
      if (!p->cap_stream) ce = cudaStreamCreateWithFlags(&p->cap_stream, cudaStreamNonBlocking);
      if (ce == cudaSuccess) ce = cudaStreamBeginCapture(p->cap_stream, cudaStreamCaptureModeThreadLocal);
      if (ce == cudaSuccess) {
        cudaError_t ee = enqueue(p->cap_stream);
        ce = cudaStreamEndCapture(p->cap_stream, &graph);
        if (ee != cudaSuccess) ce = ee;
      }
      if (ce == cudaSuccess) ce = cudaGraphInstantiate(&exec, graph, 0);
      if (graph) cudaGraphDestroy(graph);
      if (ce == cudaSuccess) {
        if (p->graphs.size() >= 8) {
          cudaGraphExecDestroy(p->graphs.front().exec);
          p->graphs.erase(p->graphs.begin());
        }
        p->graphs.push_back({(int)dir, (const void*)din, (void*)dout, k_in2, k_out2, exec});
        e = cudaGraphLaunch(exec, st);
        p->last_launches = 1;
        ran = true;
      } else {
        cudaGetLastError();  // capture not possible here: fall back to direct launches
        if (getenv("MW_DEBUG")) fprintf(stderr, "libmw: graph capture failed (%s); running calls directly\n",
                                        cudaGetErrorString(ce));
        p->graph_failed = true;
        e = cudaSuccess;
        nl = 0;
      }
    }
  }
  if (!ran) {
    e = enqueue(st);
    p->last_launches = nl;
  }
  if (e != cudaSuccess) return from_cuda(e);
  if (!out_dev || !out2_dev) {
    if (!out_dev) e = cudaMemcpyAsync(out, dout, out_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && !out2_dev) e = cudaMemcpyAsync(out2, dout2, nmw, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
  }
  return MW_OK;
}

// ---- tuning ----------------------------------------------------------------

// Plans whose contraction work lists follow p's sweep: p itself (or its ragged
// sub-plans) and the twins of fused calls.
std::vector<mw_plan*> tuning_targets(mw_plan* p) {
  std::vector<mw_plan*> v;
  if (p->subs.empty()) v.push_back(p);
  for (mw_plan* c : p->subs) v.push_back(c);
  for (mw_plan* c : p->twins) v.push_back(c);
  return v;
}

bool tuning_valid(const mw_tuning& t) {
  return (t.chunk == 128 || t.chunk == 256 || t.chunk == 512) && (t.groups == 1 || t.groups == 2) &&
         (t.tn_threads == 128 || t.tn_threads == 256);
}

void drop_graphs(mw_plan* p) {
  for (auto& g : p->graphs) cudaGraphExecDestroy(g.exec);
  p->graphs.clear();
}

mw_status apply_tuning(mw_plan* p, const mw_tuning& t) {
  if (!tuning_valid(t)) return MW_EINVAL;
  p->chunk = t.chunk;
  p->tn_threads = t.tn_threads;
  p->tuned_ms = t.ms;
  for (mw_plan* q : tuning_targets(p)) {
    q->chunk = t.chunk;
    q->tn_threads = t.tn_threads;
    q->tc2_ng = t.groups;
    if (q->prec == MW_PREC_MIXED_BF16X3) {
      const cudaError_t e = make_tc2_items(q, t.chunk);
      if (e != cudaSuccess) {
        cudaGetLastError();
        return from_cuda(e);
      }
    }
  }
  drop_graphs(p);
  return MW_OK;
}

mw_tuning current_tuning(const mw_plan* p) {
  mw_tuning t;
  t.chunk = p->chunk;
  t.tn_threads = p->tn_threads;
  t.groups = p->subs.empty() ? p->tc2_ng : p->subs[0]->tc2_ng;
  t.ms = p->tuned_ms;
  return t;
}

// Time every candidate over one inverse + forward of the plan's batch on
// scratch buffers (one warm-up round trip, then two timed), keep the fastest.
mw_status autotune(mw_plan* p, cudaStream_t st) {
  const bool real = p->real;
  const size_t map_b = (size_t)p->map_elems * (real ? sizeof(double) : sizeof(double2));
  const size_t flm_b = (size_t)p->flm_elems * sizeof(double2);
  void *dmap = nullptr, *dflm = nullptr;
  cudaError_t e = cudaMalloc(&dmap, map_b);
  if (e == cudaSuccess) e = cudaMalloc(&dflm, flm_b);
  if (e == cudaSuccess) e = cudaMemsetAsync(dflm, 0, flm_b, st);
  cudaEvent_t a = nullptr, b = nullptr;
  if (e == cudaSuccess) e = cudaEventCreate(&a);
  if (e == cudaSuccess) e = cudaEventCreate(&b);
  std::vector<mw_tuning> cand;
  const mw_tuning base = current_tuning(p);
  const bool bf16 = p->prec == MW_PREC_MIXED_BF16X3, mixed = p->prec != MW_PREC_FP64;
  const bool tn = (p->flags & MW_FLAG_DELTA_TN) != 0;
  size_t maxg = 0;
  for (mw_plan* q : tuning_targets(p)) maxg = q->groups.size() > maxg ? q->groups.size() : maxg;
  cand.push_back(base);
  if (mixed) {
    for (int chunk : {512, 256, 128})
      for (int g : {2, 1})
        for (int t : {256, 128}) {
          if (chunk < 512 && chunk >= p->L) continue;        // one chunk either way
          if (g == 1 && (!bf16 || maxg < 2)) continue;       // one group per pass only matters with two
          if (t == 128 && !tn) continue;                     // the Risbo sweep has no such knob
          mw_tuning c{chunk, g, t, 0.0};
          if (c.chunk == base.chunk && c.groups == base.groups && c.tn_threads == base.tn_threads) continue;
          cand.push_back(c);
        }
  }
  const unsigned saved = p->flags;
  const bool saved_timing = p->timing;
  p->flags &= ~(unsigned)MW_FLAG_GRAPH;
  p->timing = false;
  int best = -1;
  float best_ms = 0.f;
  for (size_t i = 0; e == cudaSuccess && i < cand.size(); ++i) {
    if (apply_tuning(p, cand[i]) != MW_OK) { e = cudaErrorUnknown; break; }
    mw_status s1 = run(p, kInverse, dflm, dmap, st);
    if (s1 == MW_OK) s1 = run(p, kForward, dmap, dflm, st);
    if (s1 == MW_OK && cudaEventRecord(a, st) != cudaSuccess) s1 = MW_ECUDA;
    for (int r = 0; r < 2 && s1 == MW_OK; ++r) {
      s1 = run(p, kInverse, dflm, dmap, st);
      if (s1 == MW_OK) s1 = run(p, kForward, dmap, dflm, st);
    }
    float ms = 0.f;
    if (s1 == MW_OK) e = cudaEventRecord(b, st);
    if (s1 == MW_OK && e == cudaSuccess) e = cudaEventSynchronize(b);
    if (s1 == MW_OK && e == cudaSuccess) e = cudaEventElapsedTime(&ms, a, b);
    if (s1 != MW_OK) { e = cudaErrorUnknown; break; }
    cand[i].ms = ms / 2.0;
    if (best < 0 || ms < best_ms) { best = (int)i; best_ms = ms; }
  }
  p->flags = saved;
  p->timing = saved_timing;
  mw_status st_out = from_cuda(e);
  if (best >= 0) {
    const mw_status s2 = apply_tuning(p, cand[best]);
    if (st_out == MW_OK) st_out = s2;
  } else {
    apply_tuning(p, base);
  }
  if (a) cudaEventDestroy(a);
  if (b) cudaEventDestroy(b);
  if (dmap) cudaFree(dmap);
  if (dflm) cudaFree(dflm);
  if (st_out != MW_OK) cudaGetLastError();
  return st_out;
}

// The cache key of plan p (its maps, precision, recursion, real flag, device).
mw_status plan_key(const mw_plan* p, std::string* key) {
  std::vector<int> Ls, ss;
  if (!p->q_L.empty()) { Ls = p->q_L; ss = p->q_s; }
  if (Ls.empty()) return MW_EINVAL;
  cudaDeviceProp prop;
  const char* dev = "unknown";
  if (cudaGetDeviceProperties(&prop, p->device) == cudaSuccess) dev = prop.name;
  else cudaGetLastError();
  std::vector<char> buf(64 + 24 * Ls.size() + 256);
  const mw_status s = mw_tune_key((int)Ls.size(), Ls.data(), ss.data(), p->flags, dev, buf.data(), buf.size());
  if (s == MW_OK) *key = buf.data();
  return s;
}

// MW_FLAG_AUTOTUNE at creation: the cached tuning of the plan's key, or a
// search (recorded when MW_TUNE_CACHE is set).
mw_status tune_at_creation(mw_plan* p) {
  const char* path = getenv("MW_TUNE_CACHE");
  std::string key;
  if (plan_key(p, &key) != MW_OK) return MW_EINVAL;
  if (path && *path) {
    mw_tuning t;
    int found = 0;
    if (mw_tune_cache_lookup(path, key.c_str(), &t, &found) == MW_OK && found && tuning_valid(t))
      return apply_tuning(p, t);
  }
  mw_status s = autotune(p, 0);
  if (s == MW_OK && path && *path) {
    const mw_tuning t = current_tuning(p);
    mw_tune_cache_store(path, key.c_str(), &t);  // a cache that cannot be written only costs a later search
  }
  return s;
}

// Ragged plan: n maps with their own band limits and spins.  The parent owns
// the recursion state sized for max L; one sub-plan per distinct band limit
// owns that band limit's tables and buffers and reads/writes its maps at their
// offsets in the caller's buffers (maps and f_lm blocks back to back in the
// caller's order).
mw_status build_ragged(mw_plan** out, int n, const int* Ls, const int* spins, unsigned flags) {
  if (!out) return MW_EINVAL;
  *out = nullptr;
  if (n < 1 || n > (1 << 20) || !Ls || !spins || (flags & MW_FLAG_REAL)) return MW_EINVAL;
  int Lmax = 0;
  for (int b = 0; b < n; ++b) {
    if (Ls[b] < 1 || Ls[b] > 2048 || spins[b] <= -Ls[b] || spins[b] >= Ls[b]) return MW_EINVAL;
    Lmax = Ls[b] > Lmax ? Ls[b] : Lmax;
  }
  std::vector<long long> moff(n + 1), foff(n + 1);
  if (mw_layout_ragged(n, Ls, moff.data(), foff.data()) != MW_OK) return MW_EINVAL;
  const long long mo = moff[n], fo = foff[n];
  moff.pop_back();
  foff.pop_back();
  const int zero = 0;
  mw_plan* parent = nullptr;
  mw_status stt = build_plan(&parent, Lmax, 1, &zero, flags, nullptr, nullptr, nullptr, true);
  if (stt != MW_OK) return stt;
  parent->B = n;
  parent->spins.assign(spins, spins + n);
  parent->map_elems = mo;
  parent->flm_elems = fo;
  parent->q_L.assign(Ls, Ls + n);
  parent->q_s.assign(spins, spins + n);
  parent->q_moff = moff;
  parent->q_foff = foff;
  std::vector<int> done(n, 0);
  for (int b = 0; b < n; ++b) {
    if (done[b]) continue;
    const int L = Ls[b];
    std::vector<int> ss;
    std::vector<long long> mm, ff;
    for (int c = b; c < n; ++c)
      if (!done[c] && Ls[c] == L) {
        done[c] = 1;
        ss.push_back(spins[c]);
        mm.push_back(moff[c]);
        ff.push_back(foff[c]);
      }
    mw_plan* sub = nullptr;
    stt = build_plan(&sub, L, (int)ss.size(), ss.data(), flags, mm.data(), ff.data(), parent, false);
    if (stt != MW_OK) {
      free_plan(parent);
      return stt;
    }
    parent->ws_bytes += sub->ws_bytes;
    parent->subs.push_back(sub);
  }
  *out = parent;
  return MW_OK;
}

}  // namespace

StageSpan::StageSpan(mw_plan* p_, int stage_, cudaStream_t st_) : p(p_), stage(stage_), st(st_) {
  if (!p->timing) return;
  if (p->pool.empty()) {
    if (cudaEventCreate(&a) != cudaSuccess) { a = nullptr; cudaGetLastError(); return; }
  } else {
    a = p->pool.back();
    p->pool.pop_back();
  }
  cudaEventRecord(a, st);
}

void StageSpan::end(int launches) {
  if (!p->timing || !a) return;
  cudaEvent_t b;
  if (p->pool.empty()) {
    if (cudaEventCreate(&b) != cudaSuccess) { cudaGetLastError(); p->pool.push_back(a); return; }
  } else {
    b = p->pool.back();
    p->pool.pop_back();
  }
  cudaEventRecord(b, st);
  p->recs.push_back({stage, a, b});
  p->stage_launches[stage] += launches;
}

extern "C" {

mw_status mw_plan_sync(mw_plan* plan, void* stream) {
  if (!plan) return MW_EINVAL;
  cudaError_t e = cudaStreamSynchronize((cudaStream_t)stream);
  if (e != cudaSuccess) return from_cuda(e);
  int flag = 0;
  e = cudaMemcpy(&flag, plan->d_err, sizeof(int), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return from_cuda(e);
  if (flag) {
    cudaMemset(plan->d_err, 0, sizeof(int));
    return MW_ETIMEOUT;
  }
  return MW_OK;
}

mw_status mw_plan_set_timing(mw_plan* plan, int enable) {
  if (!plan) return MW_EINVAL;
  plan->timing = enable != 0;
  return MW_OK;
}

mw_status mw_plan_stage_times(mw_plan* plan, double* ms, long long* launches, int reset) {
  if (!plan) return MW_EINVAL;
  cudaError_t e = cudaSuccess;
  for (auto& r : plan->recs) {
    float t = 0.f;
    cudaError_t x = cudaEventSynchronize(r.b);
    if (x == cudaSuccess) x = cudaEventElapsedTime(&t, r.a, r.b);
    if (x != cudaSuccess && e == cudaSuccess) e = x;
    plan->stage_ms[r.stage] += t;
    plan->pool.push_back(r.a);
    plan->pool.push_back(r.b);
  }
  plan->recs.clear();
  for (int k = 0; k < MW_NUM_STAGES; ++k) {
    if (ms) ms[k] = plan->stage_ms[k];
    if (launches) launches[k] = plan->stage_launches[k];
    if (reset) { plan->stage_ms[k] = 0.0; plan->stage_launches[k] = 0; }
  }
  return from_cuda(e);
}

// A freshly built plan: with MW_FLAG_AUTOTUNE, its tuning from the cache or a search.
static mw_status finish_plan(mw_plan** out, mw_status st) {
  if (st != MW_OK || !(*out) || !((*out)->flags & MW_FLAG_AUTOTUNE)) return st;
  st = tune_at_creation(*out);
  if (st != MW_OK) {
    cudaDeviceSynchronize();
    free_plan(*out);
    *out = nullptr;
  }
  return st;
}

mw_status mw_plan_create(mw_plan** out, int L, int s, int batch, unsigned flags) {
  if (!out) return MW_EINVAL;
  *out = nullptr;
  if (batch < 1 || batch > (1 << 20)) return MW_EINVAL;
  std::vector<int> spins(batch, s);
  return finish_plan(out, build_plan(out, L, batch, spins.data(), flags));
}

mw_status mw_plan_create_ragged(mw_plan** out, int n, const int* L, const int* spins, unsigned flags) {
  return finish_plan(out, build_ragged(out, n, L, spins, flags));
}

mw_status mw_plan_create_spins(mw_plan** out, int L, int batch, const int* spins, unsigned flags) {
  if (!out) return MW_EINVAL;
  *out = nullptr;
  if (batch < 1 || batch > (1 << 20) || !spins) return MW_EINVAL;
  return finish_plan(out, build_plan(out, L, batch, spins, flags));
}

mw_status mw_plan_get_tuning(const mw_plan* plan, mw_tuning* out) {
  if (!plan || !out) return MW_EINVAL;
  *out = current_tuning(plan);
  return MW_OK;
}

mw_status mw_plan_set_tuning(mw_plan* plan, const mw_tuning* t) {
  if (!plan || !t || !tuning_valid(*t)) return MW_EINVAL;
  return apply_tuning(plan, *t);
}

mw_status mw_plan_autotune(mw_plan* plan, void* stream) {
  if (!plan) return MW_EINVAL;
  const mw_status st = autotune(plan, (cudaStream_t)stream);
  const char* path = getenv("MW_TUNE_CACHE");
  std::string key;
  if (st == MW_OK && path && *path && plan_key(plan, &key) == MW_OK) {
    const mw_tuning t = current_tuning(plan);
    mw_tune_cache_store(path, key.c_str(), &t);
  }
  return st;
}

mw_status mw_forward(mw_plan* plan, const void* map_in, void* flm_out, void* stream) {
  return run(plan, kForward, map_in, flm_out, stream);
}
mw_status mw_inverse(mw_plan* plan, const void* flm_in, void* map_out, void* stream) {
  return run(plan, kInverse, flm_in, map_out, stream);
}
mw_status mw_forward_adjoint(mw_plan* plan, const void* flm_in, void* map_out, void* stream) {
  return run(plan, kForwardAdjoint, flm_in, map_out, stream);
}
mw_status mw_forward_inverse(mw_plan* plan, const void* map_in, void* flm_out, const void* flm_in, void* map_out,
                             void* stream) {
  return run(plan, kFused, map_in, flm_out, stream, flm_in, map_out);
}
mw_status mw_inverse_adjoint(mw_plan* plan, const void* map_in, void* flm_out, void* stream) {
  return run(plan, kInverseAdjoint, map_in, flm_out, stream);
}

mw_status mw_quadrature_weights(int L, int s, double* q_out, void* stream) {
  if (L < 1 || L > 2048 || s <= -L || s >= L || !q_out || !is_device_ptr(q_out)) return MW_EINVAL;
  return from_cuda(launch_quad_weights(L, s, q_out, (cudaStream_t)stream));
}

mw_status mw_quadrature(mw_plan* plan, const void* maps_q, void* integrals, void* stream) {
  if (!plan || !maps_q || !integrals) return MW_EINVAL;
  if (!plan->subs.empty() || plan->real) return MW_EUNSUPPORTED;
  if (!is_device_ptr(maps_q) || !is_device_ptr(integrals)) return MW_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = cudaSuccess;
  if (!plan->d_qw) {  // weights of even and odd spin, computed once per plan
    e = cudaMalloc((void**)&plan->d_qw, sizeof(double) * 2 * (size_t)plan->L);
    if (e == cudaSuccess) e = launch_quad_weights(plan->L, 0, plan->d_qw, st);
    if (e == cudaSuccess) e = launch_quad_weights(plan->L, 1, plan->d_qw + plan->L, st);
    if (e == cudaSuccess) e = cudaMalloc((void**)&plan->d_qpart, sizeof(double2) * (size_t)plan->B * quad_chunks(plan));
    if (e == cudaSuccess) plan->ws_bytes += sizeof(double) * 2 * plan->L + sizeof(double2) * plan->B * quad_chunks(plan);
    if (e != cudaSuccess) {
      cudaGetLastError();
      cudaFree(plan->d_qw);
      plan->d_qw = nullptr;
      return from_cuda(e);
    }
  }
  int nl = 0;
  e = launch_quadrature(plan, (const double2*)maps_q, (double2*)integrals, st, &nl);
  plan->last_launches = nl;
  return from_cuda(e);
}

mw_status mw_plan_destroy(mw_plan* plan) {
  if (!plan) return MW_OK;
  cudaError_t e = cudaDeviceSynchronize();
  free_plan(plan);
  return from_cuda(e);
}

const char* mw_status_string(mw_status st) {
  switch (st) {
    case MW_OK: return "MW_OK: success";
    case MW_EINVAL: return "MW_EINVAL: invalid argument";
    case MW_ENOMEM: return "MW_ENOMEM: out of memory";
    case MW_ECUDA: return "MW_ECUDA: CUDA error";
    case MW_ETIMEOUT: return "MW_ETIMEOUT: device-side wait timed out";
    case MW_EUNSUPPORTED: return "MW_EUNSUPPORTED: unsupported request";
  }
  return "unknown status";
}

size_t mw_plan_map_elems(const mw_plan* plan) { return plan ? (size_t)plan->map_elems : 0; }
size_t mw_plan_flm_elems(const mw_plan* plan) { return plan ? (size_t)plan->flm_elems : 0; }

mw_status mw_layout_ragged(int n, const int* L, long long* map_offsets, long long* flm_offsets) {
  if (n < 1 || !L) return MW_EINVAL;
  for (int b = 0; b < n; ++b)
    if (L[b] < 1 || L[b] > 2048) return MW_EINVAL;
  long long mo = 0, fo = 0;
  for (int b = 0; b <= n; ++b) {
    if (map_offsets) map_offsets[b] = mo;
    if (flm_offsets) flm_offsets[b] = fo;
    if (b == n) break;
    mo += (long long)(L[b] - 1) * (2 * L[b] - 1) + 1;
    fo += (long long)L[b] * L[b];
  }
  return MW_OK;
}

int mw_plan_batch(const mw_plan* plan) { return plan ? (int)plan->q_L.size() : 0; }
static bool has_map(const mw_plan* plan, int b) { return plan && b >= 0 && b < (int)plan->q_L.size(); }
int mw_plan_band_limit(const mw_plan* plan, int b) { return has_map(plan, b) ? plan->q_L[b] : -1; }
int mw_plan_spin(const mw_plan* plan, int b) { return has_map(plan, b) ? plan->q_s[b] : -1; }
long long mw_plan_map_offset(const mw_plan* plan, int b) { return has_map(plan, b) ? plan->q_moff[b] : -1; }
long long mw_plan_flm_offset(const mw_plan* plan, int b) { return has_map(plan, b) ? plan->q_foff[b] : -1; }

size_t mw_map_size(int L) { return L < 1 ? 0 : (size_t)(L - 1) * (2 * (size_t)L - 1) + 1; }
size_t mw_flm_size(int L) { return L < 1 ? 0 : (size_t)L * (size_t)L; }
size_t mw_plan_workspace_bytes(const mw_plan* plan) { return plan ? plan->ws_bytes : 0; }
int mw_plan_last_launches(const mw_plan* plan) { return plan ? plan->last_launches : 0; }
int mw_plan_fft_bluestein(const mw_plan* plan) {
  if (!plan) return -1;
  if (plan->bluestein) return 1;
  for (const mw_plan* c : plan->subs)
    if (c->bluestein) return 1;
  return 0;
}

}  // extern "C"
