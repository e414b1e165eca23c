// internal.h -- plan layout and kernel entry points shared by the libmw sources.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>
#include <cstddef>
#include <cstdint>
#include <vector>

#include "../../include/mw.h"

// Radix sequence of one FFT length (passed by value to kernels).
struct FftDesc {
  int n;
  int nrad;
  int rad[26];
};

// Maps that share a spin are contracted together against one Delta plane.
// Each group holds at most kMaxGroupMaps maps (larger spin classes are split).
constexpr int kMaxGroupMaps = 32;
constexpr int kChunk = 64;         // Delta planes staged per FP64 contraction launch
constexpr int kTcChunk = 512;      // Delta planes staged per tensor-core contraction launch (8.7 GB at L=2048)
constexpr int kTcGroupMaps = 8;    // maps per spin group on both contraction paths (N = 4 x 8)

struct SpinGroup {
  int s;
  int nb;
  int maps[kMaxGroupMaps];
};

struct mw_plan {
  int L = 0, B = 0, M = 0, N = 0;
  unsigned flags = 0;
  int prec = MW_PREC_FP64;
  int device = 0;
  std::vector<int> spins;          // per map
  // real-signal plans (MW_FLAG_REAL): nreal real spin-0 maps packed two per
  // complex map, so B = (nreal + 1) / 2; d_gpack holds the packed f_lm [B][L*L]
  bool real = false;
  int nreal = 0;
  double2* d_gpack = nullptr;
  // caller-buffer offsets (complex elements) of each map and f_lm block
  std::vector<long long> moff, foff;
  long long* d_moff = nullptr;
  long long* d_foff = nullptr;
  long long map_elems = 0, flm_elems = 0;  // totals over the plan's maps
  // caller-facing layout, one entry per map of the caller's buffers (real maps
  // of a real plan, every map of a ragged plan): band limit, spin, offsets
  std::vector<int> q_L, q_s;
  std::vector<long long> q_moff, q_foff;
  // ragged plans: one sub-plan per band limit; the parent owns the sweep state
  std::vector<mw_plan*> subs;
  bool shared_sweep = false;       // sweep state borrowed from a parent (not freed here)
  std::vector<SpinGroup> groups;   // host copy
  SpinGroup* d_groups = nullptr;   // device copy
  int* d_spins = nullptr;

  FftDesc fM{}, fN{};
  // forward weight convolution by even lags (kernels_fft.cu): length NE of the
  // two half convolutions, its twiddles, and the DFTs of the even-lag kernel
  // w(2d) over the lags the even and the odd half use, pre-scaled by 1/(NE M)
  FftDesc fE{};
  int NE = 0;
  void* d_twE = nullptr;
  void* d_Ue = nullptr;
  void* d_Uo = nullptr;
  int fft_threads = 0;             // block size of the FFT kernels
  // tables, precision of the FFT stages (double2 or float2 per entry)
  void* d_twM = nullptr;           // e^{-2 pi i k / M}, k < M
  void* d_twN = nullptr;           // e^{-2 pi i k / N}, k < N
  void* d_phase = nullptr;         // e^{-i pi m' / M}, m' = -(L-1)..L-1 (index m'+L-1)
  void* d_V = nullptr;             // DFT_N of the reflected weights, pre-scaled by 1/(N M)
  // length-M FFTs by Bluestein's chirp-z convolution of power-of-two length
  // NB = fB.n >= 2M - 1 when M's prime factors would make the mixed-radix
  // dot-product stages dearer
  bool bluestein = false;
  FftDesc fB{};
  void* d_twB = nullptr;           // e^{-2 pi i k / NB}, k < NB
  void* d_chirp = nullptr;         // e^{-i pi n^2 / M}, n < M
  void* d_chirpF = nullptr;        // DFT_NB of conj(chirp) placed circularly, pre-scaled by 1/NB
  double* d_sqrt = nullptr;        // sqrt(k), k = 0..2L+2
  double* d_rsqrt = nullptr;       // 1/sqrt(k), k = 1..2L+2 (entry 0 unused, 0)
  double2* d_upole = nullptr;      // u(m') + u(-m') (m' > 0), u(0): pole row of the forward adjoint
  double* d_rscale = nullptr;      // 1 / (sqrt2 * two_jp) for the Risbo half step to plane two_jp / 2
  float2* d_sqrt_ff = nullptr;     // mixed paths: the three tables above as float-float (hi, lo)
  float2* d_rsqrt_ff = nullptr;
  float2* d_rscale_ff = nullptr;
  float2* d_tn_top = nullptr;      // MW_FLAG_DELTA_TN: top rows Delta^l_{l,m} as float-float mantissas
  int* d_tn_exp = nullptr;         // and their power-of-two exponents, plane l at l (l + 1) / 2
  double* d_nl = nullptr;          // sqrt((2l+1)/(4 pi)), l < L
  float2* d_flmf = nullptr;        // TF32x3 path: N_l f_lm in FP32 (input of the inverse contraction)
  float2* d_flmT = nullptr;        // BF16x3 path: N_l f_lm in FP32 transposed to [B][M][L] (zero for l < |m|)
  // BF16x3 contraction pipeline (kernels_tc2.cu): tensor maps of the staged
  // planes (owner only), work items of this plan per (direction, chunk), and
  // spin groups per pass (1 or 2)
  CUtensorMap tmap_fwd{}, tmap_inv{};
  bool tc2_maps = false;
  int tc2_ng = 2;
  int4* d_tc2_items = nullptr;
  std::vector<int> tc2_off;
  int tc2_chunk = 0;               // chunk the work lists were built for
  // tuning (mw_plan_set_tuning / mw_plan_autotune): planes per recursion +
  // contraction launch (the sweep owner's value governs), Trapani-Navaza
  // columns per block, and the measured round trip of the choice
  int chunk = kTcChunk;
  int tn_threads = 256;
  double tuned_ms = 0.0;

  // workspace
  void* d_Gt = nullptr;            // [B][M][L] G_m(theta_t) (forward) / [B][L][M] F_m(theta_t) (inverse)
  double2* d_Gp = nullptr;         // [B][M][L] folded G+_{m,m'} or F+_{m,m'}, m' >= 0; on the mixed path G+
                                   // as float2 and F+ as float-float (re_hi, re_lo, im_hi, im_lo)
  double* d_S = nullptr;           // FP64 path: [kChunk][LD][LD] staged integer Delta planes (quarter);
                                   // mixed path: [2][LD][LD] ping-pong recursion state (float-float pairs)
  float* d_S32 = nullptr;          // mixed path: [kTcChunk][LD][LD] FP32 copies of the integer planes
  int* d_err = nullptr;            // device error word (bit 0: tensor-core wait, bit 1: grid barrier)
  int* d_prog = nullptr;           // per-tile progress counters of the persistent Risbo kernel
  int risbo_grid = 0;              // co-resident blocks of the persistent Risbo kernel
  int* d_perm = nullptr;           // placement-aware rank of each Risbo block
  double* d_qw = nullptr;          // quadrature weights q(theta_t): [even spin][L], [odd spin][L]
  double2* d_qpart = nullptr;      // quadrature partial sums [B][chunks]
  double* d_H = nullptr;           // [LD][LD] half-integer plane
  int LD = 0;                      // plane row stride (L+1)
  double2* d_map_stage = nullptr;  // host-pointer staging
  double2* d_flm_stage = nullptr;
  double2* d_map_stage2 = nullptr;  // host-pointer staging of a fused call's inverse half
  double2* d_flm_stage2 = nullptr;
  // fused forward+inverse calls: plans of the same maps (one per sub-plan of a
  // ragged plan) that borrow this plan's sweep state and run the inverse half
  // with workspace of their own; built on the first fused call
  std::vector<mw_plan*> twins;

  size_t ws_bytes = 0;
  int last_launches = 0;

  // CUDA graphs of whole calls (MW_FLAG_GRAPH): one per (direction, input, output)
  struct GraphEntry { int dir; const void* in; void* out; const void* in2; void* out2; cudaGraphExec_t exec; };
  std::vector<GraphEntry> graphs;
  bool graph_failed = false;       // capture unsupported here: run calls directly
  cudaStream_t cap_stream = nullptr;  // stream the graphs are captured on
  // calls on pinned host buffers: the stream of the overlapped host copies
  // and the events that order them against the compute stream
  cudaStream_t copy_stream = nullptr;
  std::vector<cudaEvent_t> copy_ev;

  // optional per-stage timing (CUDA events on the call's stream)
  bool timing = false;
  struct Rec { int stage; cudaEvent_t a, b; };
  std::vector<Rec> recs;           // pending event pairs of recorded calls
  std::vector<cudaEvent_t> pool;   // free events
  double stage_ms[MW_NUM_STAGES] = {0};
  long long stage_launches[MW_NUM_STAGES] = {0};
};

// Event pair around a span of launches of one stage (no-op unless timing is on).
struct StageSpan {
  mw_plan* p;
  int stage;
  cudaStream_t st;
  cudaEvent_t a = nullptr;
  StageSpan(mw_plan* p_, int stage_, cudaStream_t st_);
  void end(int launches);
};

// ---- kernels (launch helpers return cudaGetLastError()) ----
// FFT stages of the maps [b0, b0 + nb) (nb < 0: every map of the plan)
cudaError_t launch_phi_forward(const mw_plan* p, const double2* map, cudaStream_t st, int b0 = 0, int nb = -1);
cudaError_t launch_theta_forward(const mw_plan* p, cudaStream_t st, int b0 = 0, int nb = -1);
cudaError_t launch_theta_inverse(const mw_plan* p, cudaStream_t st, int b0 = 0, int nb = -1);
cudaError_t launch_phi_inverse(const mw_plan* p, double2* map, cudaStream_t st, int b0 = 0, int nb = -1);
cudaError_t launch_phi_forward_adjoint(const mw_plan* p, double2* map, cudaStream_t st);
cudaError_t launch_theta_forward_adjoint(const mw_plan* p, cudaStream_t st);
cudaError_t launch_theta_inverse_adjoint(const mw_plan* p, cudaStream_t st);
cudaError_t launch_pole_forward_adjoint(const mw_plan* p, double2* map, cudaStream_t st);
cudaError_t launch_tc_forward(const mw_plan* p, int l0, int l1, double2* flm, cudaStream_t st);
cudaError_t launch_tc_inverse(const mw_plan* p, int l0, int l1, const float2* flmf, cudaStream_t st);
cudaError_t launch_flm_to_f32(const mw_plan* p, const double2* flm, cudaStream_t st);
cudaError_t launch_dmma_forward(const mw_plan* p, int l0, int l1, double2* flm, cudaStream_t st);
cudaError_t launch_dmma_inverse(const mw_plan* p, int l0, int l1, const double2* flm, cudaStream_t st);
cudaError_t launch_phi_inverse_adjoint(const mw_plan* p, const double2* map, cudaStream_t st);
// real-signal plans: phi stages on pairs of real maps, and the f_lm pack/unpack
cudaError_t launch_phi_forward_real(const mw_plan* p, const double* maps, cudaStream_t st);
cudaError_t launch_phi_inverse_real(const mw_plan* p, double* maps, cudaStream_t st);
cudaError_t launch_real_unpack(const mw_plan* p, const double2* g, double2* flm, cudaStream_t st);
cudaError_t launch_real_pack(const mw_plan* p, const double2* flm, double2* g, cudaStream_t st);
// BF16x3 contraction pipeline: tensor maps of owner o's staging planes, the
// work lists of plan p, the transposed N_l f_lm, and one chunk's contraction
// (dir 0: Eq. flm_wig into flm; dir 1: Eq. Fmm into F+)
cudaError_t make_tc2_tensor_maps(mw_plan* o);
cudaError_t make_tc2_items(mw_plan* p, int chunk);
// rows l in [l0, l1) (l1 < 0: every row)
cudaError_t launch_flm_transpose(const mw_plan* p, const double2* flm, cudaStream_t st, int l0 = 0, int l1 = -1);
cudaError_t launch_tc2(const mw_plan* p, const mw_plan* o, int dir, int l0, int l1c, double2* flm, cudaStream_t st);
// Trapani-Navaza planes l in [lb, le) into staging slots l - l0 (mixed paths)
cudaError_t launch_tn(const mw_plan* p, int l0, int lb, int le, cudaStream_t st);

// Wigner stage: one pass l = 0..o->L-1 over the planes of the owner o (Risbo's
// sweep or the Trapani-Navaza planes, by o's flags) and the contractions of
// the consumer plans.
// mode 0: f_lm from G+ (Eq. flm_wig); mode 1: F+ from f_lm (Eq. Fmm).
int risbo_blocks_per_sm(int prec);
int quad_chunks(const mw_plan* p);
cudaError_t launch_quad_weights(int L, int s, double* q, cudaStream_t st);
cudaError_t launch_quadrature(const mw_plan* p, const double2* maps, double2* out, cudaStream_t st, int* launches);
cudaError_t make_risbo_perm(mw_plan* p);

// One consumer of a Risbo sweep: plan q's forward contraction (mode 0, G+ in
// q's workspace -> flm_out) or inverse contraction (mode 1, flm_in -> F+ in q's
// workspace).  Plane l serves every consumer with L > l.
struct WignerJob {
  mw_plan* q;
  int mode;
  const double2* flm_in;
  double2* flm_out;
  // mode 1 on the BF16x3 path: flm_in's rows arrive chunk by chunk and the
  // hook's `before` transposes each chunk's rows (no transposition up front)
  bool chunked_flm = false;
};
// hook: if given, fn is called after the contraction launches of every chunk
// of planes [l0, l1) have been enqueued on st (the forward's f_lm rows
// l0..l1-1 are then final once st reaches that point), and before (if not
// null) just before them (after the chunk's recursion launch).
struct ChunkHook {
  cudaError_t (*fn)(void* ctx, int l0, int l1);
  void* ctx;
  cudaError_t (*before)(void* ctx, int l0, int l1) = nullptr;
};
cudaError_t run_wigner(mw_plan* o, const WignerJob* jobs, int nj, cudaStream_t st, int* launches,
                       const ChunkHook* hook = nullptr);
