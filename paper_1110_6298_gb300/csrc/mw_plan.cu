// mw_plan.cu -- plans, host-side tables and the C entry points of libmw.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
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
  void* ptrs[] = {p->d_groups, p->d_spins, p->d_twM, p->d_twN, p->d_phase, p->d_V, p->d_sqrt, p->d_upole,
                  p->d_Gt,     p->d_Gp,    p->d_S,   p->d_H,   p->d_map_stage, p->d_flm_stage, p->d_S32, p->d_err, p->d_prog, p->d_rscale, p->d_nl, p->d_flmf};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  for (auto& r : p->recs) { cudaEventDestroy(r.a); cudaEventDestroy(r.b); }
  for (auto ev : p->pool) cudaEventDestroy(ev);
  delete p;
}

mw_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return MW_OK;
  if (e == cudaErrorMemoryAllocation) return MW_ENOMEM;
  return MW_ECUDA;
}

mw_status build_plan(mw_plan** out, int L, int B, const int* spins, unsigned flags) {
  if (!out) return MW_EINVAL;
  *out = nullptr;
  if (L < 1 || L > 2048 || B < 1 || !spins) return MW_EINVAL;
  const int prec = (int)(flags & 0xffu);
  if (prec != MW_PREC_FP64 && prec != MW_PREC_MIXED) return MW_EINVAL;
  for (int b = 0; b < B; ++b)
    if (spins[b] <= -L || spins[b] >= L) return MW_EINVAL;

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
  p->LD = ((L + 1 + 7) / 8) * 8;  // 32-byte aligned plane rows
  cudaGetDevice(&p->device);
  p->spins.assign(spins, spins + B);
  if (!factorize(p->M, &p->fM) || !factorize(p->N, &p->fN)) { free_plan(p); return MW_EUNSUPPORTED; }

  // spin groups (order of first appearance; at most kMaxGroupMaps maps each,
  // kTcGroupMaps on the tensor-core path)
  const int gmax = prec == MW_PREC_MIXED ? kTcGroupMaps : kMaxGroupMaps;
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
  twiddles(M);
  chk(dbl ? upload_complex<double>(re, im, &p->d_twM) : upload_complex<float>(re, im, &p->d_twM));
  twiddles(N);
  chk(dbl ? upload_complex<double>(re, im, &p->d_twN) : upload_complex<float>(re, im, &p->d_twN));
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
    std::vector<double> sq(2 * L + 3);
    for (size_t k = 0; k < sq.size(); ++k) sq[k] = std::sqrt((double)k);
    alloc((void**)&p->d_sqrt, sizeof(double) * sq.size());
    if (e == cudaSuccess) chk(cudaMemcpy(p->d_sqrt, sq.data(), sizeof(double) * sq.size(), cudaMemcpyHostToDevice));
  }
  {  // u(m') = sum_{|m''| <= L-1} (-1)^{m''} conj(w(m''-m')); folded u(m') + u(-m') for m' > 0
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
  alloc((void**)&p->d_spins, sizeof(int) * B);
  if (e == cudaSuccess) chk(cudaMemcpy(p->d_spins, spins, sizeof(int) * B, cudaMemcpyHostToDevice));
  alloc((void**)&p->d_groups, sizeof(SpinGroup) * p->groups.size());
  if (e == cudaSuccess)
    chk(cudaMemcpy(p->d_groups, p->groups.data(), sizeof(SpinGroup) * p->groups.size(), cudaMemcpyHostToDevice));

  // workspace
  const size_t fsz = dbl ? sizeof(double2) : sizeof(float2);
  alloc(&p->d_Gt, fsz * (size_t)B * M * L);
  alloc((void**)&p->d_Gp, sizeof(double2) * (size_t)B * M * L);
  const size_t plane = (size_t)p->LD * p->LD;
  alloc((void**)&p->d_S, sizeof(double) * (dbl ? (size_t)kChunk : 2) * plane);
  alloc((void**)&p->d_H, sizeof(double) * plane);
  if (!dbl) alloc((void**)&p->d_S32, sizeof(float) * (size_t)kTcChunk * plane);
  if (!dbl) alloc((void**)&p->d_flmf, sizeof(float2) * (size_t)B * L * L);
  alloc((void**)&p->d_err, sizeof(int));
  if (e == cudaSuccess) chk(cudaMemset(p->d_err, 0, sizeof(int)));
  {
    const int Tm = (L + 1 + 31) / 32;
    alloc((void**)&p->d_prog, sizeof(int) * (size_t)(Tm * (Tm + 1) / 2 + 1));
  }
  if (e == cudaSuccess) {
    int nsm = 0;
    chk(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, p->device));
    p->risbo_grid = nsm * risbo_blocks_per_sm();
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

enum Direction { kForward, kInverse, kForwardAdjoint, kInverseAdjoint };

mw_status run(mw_plan* p, Direction dir, const void* in, void* out, void* stream) {
  if (!p || !in || !out) return MW_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nmw = (size_t)(p->L - 1) * p->M + 1, nlm = (size_t)p->L * p->L;
  const bool map_in = (dir == kForward || dir == kInverseAdjoint);
  const size_t in_elems = (map_in ? nmw : nlm) * p->B, out_elems = (map_in ? nlm : nmw) * p->B;
  const bool in_dev = is_device_ptr(in), out_dev = is_device_ptr(out);
  cudaError_t e = cudaSuccess;
  // host staging buffers are allocated on first use
  if (!in_dev || !out_dev) {
    if (!p->d_map_stage) {
      e = cudaMalloc((void**)&p->d_map_stage, sizeof(double2) * nmw * p->B);
      if (e == cudaSuccess) p->ws_bytes += sizeof(double2) * nmw * p->B;
    }
    if (e == cudaSuccess && !p->d_flm_stage) {
      e = cudaMalloc((void**)&p->d_flm_stage, sizeof(double2) * nlm * p->B);
      if (e == cudaSuccess) p->ws_bytes += sizeof(double2) * nlm * p->B;
    }
    if (e != cudaSuccess) { cudaGetLastError(); return from_cuda(e); }
  }
  const double2* din = (const double2*)in;
  double2* dout = (double2*)out;
  if (!in_dev) {
    double2* stage = map_in ? p->d_map_stage : p->d_flm_stage;
    e = cudaMemcpyAsync(stage, in, sizeof(double2) * in_elems, cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) return from_cuda(e);
    din = stage;
  }
  if (!out_dev) dout = map_in ? p->d_flm_stage : p->d_map_stage;

  int nl = 0;
  auto stage = [&](int stg, cudaError_t (*fn)(const mw_plan*, cudaStream_t)) {
    if (e != cudaSuccess) return;
    StageSpan sp(p, stg, st);
    e = fn(p, st);
    sp.end(1);
    ++nl;
  };
  auto phi = [&](auto fn, auto ptr) {
    if (e != cudaSuccess) return;
    StageSpan sp(p, MW_STAGE_PHI, st);
    e = fn(p, ptr, st);
    sp.end(1);
    ++nl;
  };
  switch (dir) {
    case kForward:
      phi(launch_phi_forward, din);
      stage(MW_STAGE_THETA, launch_theta_forward);
      if (e == cudaSuccess) e = run_wigner(p, 0, nullptr, dout, st, &nl);
      break;
    case kInverse:
      if (e == cudaSuccess) e = run_wigner(p, 1, din, nullptr, st, &nl);
      stage(MW_STAGE_THETA, launch_theta_inverse);
      phi(launch_phi_inverse, dout);
      break;
    case kForwardAdjoint:
      if (e == cudaSuccess) e = run_wigner(p, 1, din, nullptr, st, &nl);
      stage(MW_STAGE_THETA, launch_theta_forward_adjoint);
      phi(launch_phi_forward_adjoint, dout);
      phi(launch_pole_forward_adjoint, dout);
      break;
    case kInverseAdjoint:
      phi(launch_phi_inverse_adjoint, din);
      stage(MW_STAGE_THETA, launch_theta_inverse_adjoint);
      if (e == cudaSuccess) e = run_wigner(p, 0, nullptr, dout, st, &nl);
      break;
  }
  p->last_launches = nl;
  if (e != cudaSuccess) return from_cuda(e);
  if (!out_dev) {
    e = cudaMemcpyAsync(out, dout, sizeof(double2) * out_elems, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return from_cuda(e);
  }
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

mw_status mw_plan_create(mw_plan** out, int L, int s, int batch, unsigned flags) {
  if (!out) return MW_EINVAL;
  *out = nullptr;
  if (batch < 1 || batch > (1 << 20)) return MW_EINVAL;
  std::vector<int> spins(batch, s);
  return build_plan(out, L, batch, spins.data(), flags);
}

mw_status mw_plan_create_spins(mw_plan** out, int L, int batch, const int* spins, unsigned flags) {
  if (!out) return MW_EINVAL;
  *out = nullptr;
  if (batch < 1 || batch > (1 << 20) || !spins) return MW_EINVAL;
  return build_plan(out, L, batch, spins, flags);
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
mw_status mw_inverse_adjoint(mw_plan* plan, const void* map_in, void* flm_out, void* stream) {
  return run(plan, kInverseAdjoint, map_in, flm_out, stream);
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

size_t mw_map_size(int L) { return L < 1 ? 0 : (size_t)(L - 1) * (2 * (size_t)L - 1) + 1; }
size_t mw_flm_size(int L) { return L < 1 ? 0 : (size_t)L * (size_t)L; }
size_t mw_plan_workspace_bytes(const mw_plan* plan) { return plan ? plan->ws_bytes : 0; }
int mw_plan_last_launches(const mw_plan* plan) { return plan ? plan->last_launches : 0; }

}  // extern "C"
