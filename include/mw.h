/*
 * mw.h -- C ABI of libmw: GB300 (sm_103a) MW spin spherical harmonic transforms.
 *
 * The transforms are those of McEwen & Wiaux, "A novel sampling theorem on the
 * sphere", IEEE Trans. Signal Process. 59(12), 2011:
 *   inverse  f_lm -> f(theta_t, phi_p)   Sec. IV-E, Eqs. (Fmm), (Fmt), (f_pfft)
 *   forward  f(theta_t, phi_p) -> f_lm   Sec. IV-D, Eqs. (Gmt), (Gmm_convolution),
 *                                        (flm_wig)
 * for band limit L (f_lm = 0 for l >= L) and integer spin s with |s| < L, on the
 * equiangular grid of Sec. IV-C:
 *   theta_t = pi (2t+1) / (2L-1),  t = 0..L-1   (theta_{L-1} = pi, the south pole)
 *   phi_p   = 2 pi p / (2L-1),     p = 0..2L-2
 * which holds N_MW = (L-1)(2L-1) + 1 samples.
 *
 * Buffer layouts (all complex numbers are interleaved double pairs (re, im),
 * i.e. C99 double complex / numpy complex128):
 *   map : N_MW values per map: rings t = 0..L-2, each 2L-1 samples in phi_p
 *         order, then ONE pole sample f(pi, phi = 0).  A spin-s signal on the
 *         pole ring equals f(pi, 0) e^{i s phi}, because d^l_{m,-s}(pi) vanishes
 *         unless m = s (Eq. wignerd_sym2 at beta = 0), so the one sample fixes it.
 *   flm : L*L values per map, f_lm at index l*l + l + m.  Spin-s harmonics exist
 *         only for l >= |s| (Sec. III-B): such entries are written as 0 by the
 *         forward transform and ignored on input by the inverse.
 *   A batch of B maps is B such blocks back to back.
 *
 * Pointers may be device memory or host memory (pageable or pinned); host
 * buffers are staged through plan-owned device buffers with cudaMemcpyAsync on
 * the call's stream.  Inputs are never modified.  Outputs must not alias inputs.
 * All data pointers stay owned by the caller; the plan owns its workspace and
 * tables and frees them in mw_plan_destroy.
 *
 * Calls are enqueued on `stream` (a cudaStream_t; NULL means the legacy default
 * stream) and return before the GPU finishes; device memory results are valid
 * once the stream reaches them, host outputs once the call returns (the call
 * synchronises the stream when it has to copy results to host memory).  A plan
 * must not be used by two host threads at once, nor by two streams whose work
 * overlaps.  For a given plan and input the results are bitwise reproducible:
 * every reduction runs in a fixed order and no atomics touch the data.
 *
 * Errors: every function returns a status; MW_EINVAL for bad arguments (checked
 * before anything is enqueued), MW_ENOMEM when a device or host allocation
 * fails, MW_ECUDA when a CUDA call or launch fails (the plan stays usable if
 * the context does), MW_EUNSUPPORTED for valid but unimplemented requests.
 */
#ifndef MW_H
#define MW_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mw_plan mw_plan; /* opaque; created by mw_plan_create*, freed by mw_plan_destroy */

typedef enum {
  MW_OK = 0,
  MW_EINVAL = 1,
  MW_ENOMEM = 2,
  MW_ECUDA = 3,
  MW_ETIMEOUT = 4,
  MW_EUNSUPPORTED = 5
} mw_status;

/* Precision of a plan (flags & 0xff).
 * MW_PREC_FP64 : every stage in IEEE double.
 * MW_PREC_MIXED (= MW_PREC_MIXED_BF16X3): the Wigner-Delta recursion (Sec. V-B;
 *                Trapani-Navaza by default, Risbo's on request, see below) in
 *                float-float arithmetic (about 48 significant bits) on the FP32
 *                pipe; the Delta contraction on the tensor cores
 *                (tcgen05) with FP32 operands split into three BF16 parts (six
 *                products), FP32 accumulation and a float-float sum across
 *                K tiles and chunks; the FFT stages in single precision.
 * MW_PREC_MIXED_TF32X3: as MW_PREC_MIXED with the operands split into two TF32
 *                parts (three products: hi.hi, hi.lo, lo.hi).
 * Both mixed precisions are designed for a relative error below 1e-6 against
 * the FP64 path. */
enum { MW_PREC_FP64 = 0, MW_PREC_MIXED = 1, MW_PREC_MIXED_BF16X3 = 1, MW_PREC_MIXED_TF32X3 = 2 };

/* MW_FLAG_GRAPH (or-ed into flags): the first call with a given (direction,
 * input, output) captures the whole call into a CUDA graph, later calls with
 * the same buffers replay it as one launch.  Not used while per-stage timing is
 * on; if capture is not possible the plan runs its calls directly. */
enum { MW_FLAG_GRAPH = 1 << 8 };

/* MW_FLAG_REAL (or-ed into flags): real scalar signals (Sec. IV-G).  Every spin
 * must be 0 and `batch` counts real maps.  Map buffers hold real doubles,
 * [batch][N_MW]; f_lm buffers stay complex doubles [batch][L*L] with every m.
 *   mw_forward writes coefficients that satisfy the reality condition
 *     f_{l,-m} = (-1)^m conj(f_lm) exactly (m < 0 mirrors m > 0; f_l0 real).
 *   mw_inverse returns the real part of the synthesis of the given
 *     coefficients, which is the synthesis itself when they satisfy the
 *     reality condition.
 *   mw_forward_inverse: both, sharing the recursion as on complex plans.
 * The transforms pair the maps: maps 2b and 2b+1 travel as the real and
 * imaginary part of one complex spin-0 map and are separated with the reality
 * condition, so a real plan of `batch` maps costs a complex plan of
 * (batch + 1) / 2 maps plus one O(L^2) pass over the coefficients (the paper
 * halves the m range per map instead; the factor of two is the same).
 * Adjoints and mw_quadrature return MW_EUNSUPPORTED on real plans; ragged
 * plans reject the flag (MW_EINVAL). */
enum { MW_FLAG_REAL = 1 << 9 };

/* Recursion of the Wigner planes Delta^l (or-ed into flags; at most one):
 * MW_FLAG_DELTA_TN     the Trapani-Navaza recursion (cited in Sec. V-B as the
 *                      alternative to Risbo's).  Each column of each plane
 *                      recurses independently from the closed-form top row
 *                      Delta^l_{l,m} = (-1)^(l-m) 2^-l sqrt(C(2l, l+m)), so the
 *                      planes need no step-by-step synchronisation; each
 *                      column carries its own power-of-two exponent, which
 *                      removes the underflow of the start values that limits
 *                      the recursion in plain double precision (near
 *                      L = 2560).  Mixed precisions only (MW_EUNSUPPORTED with
 *                      MW_PREC_FP64).
 * MW_FLAG_DELTA_RISBO  Risbo's recursion (Sec. V-B), one synchronised sweep.
 * Neither: Trapani-Navaza on the mixed precisions, Risbo on MW_PREC_FP64.
 * Both agree to the FP32 staging precision the mixed contractions read. */
enum { MW_FLAG_DELTA_TN = 1 << 10, MW_FLAG_DELTA_RISBO = 1 << 11 };

/* MW_FLAG_AUTOTUNE (or-ed into flags): choose the plan's tuning (below) by
 * measurement.  At plan creation the tuning cache named by the environment
 * variable MW_TUNE_CACHE (a file of JSON lines, one per key) is consulted; if
 * it holds the plan's key the recorded tuning is applied, otherwise
 * mw_plan_autotune runs and, when MW_TUNE_CACHE is set, its choice is
 * recorded.  Without the flag a plan starts from the defaults (512, 2, 256). */
enum { MW_FLAG_AUTOTUNE = 1 << 12 };

/* Create a plan for `batch` maps of band limit L and spin s.
 * Requires 1 <= L <= 2048, |s| < L, batch >= 1, out != NULL.  Allocates the
 * device workspace on the current CUDA device; *out is NULL on failure. */
mw_status mw_plan_create(mw_plan **out, int L, int s, int batch, unsigned flags);

/* As mw_plan_create, with one spin per map: spins[b] is the spin of map b
 * (|spins[b]| < L).  Maps of different spin share each Wigner-Delta plane,
 * which depends on neither L nor s (Sec. V footnote on multiple spins). */
mw_status mw_plan_create_spins(mw_plan **out, int L, int batch, const int *spins, unsigned flags);

/* Ragged batch: n maps, map b of band limit L[b] (1 <= L[b] <= 2048) and spin
 * spins[b] (|spins[b]| < L[b]).  Buffers hold the maps (resp. f_lm blocks) back
 * to back in the given order, each of its own size; mw_plan_map_elems and
 * mw_plan_flm_elems give the totals.  One Wigner-Delta recursion to max L[b]
 * serves every map (Delta^l depends on neither L nor s). */
mw_status mw_plan_create_ragged(mw_plan **out, int n, const int *L, const int *spins, unsigned flags);

/* Total elements of the plan's map buffer and f_lm buffer (complex doubles;
 * the map buffer of a MW_FLAG_REAL plan counts real doubles). */
size_t mw_plan_map_elems(const mw_plan *plan);
size_t mw_plan_flm_elems(const mw_plan *plan);

/* Layout of a plan's buffers, as the plan computed it, so that callers need
 * not re-derive it:
 *   mw_plan_batch       number of maps b of the plan (real maps for a
 *                       MW_FLAG_REAL plan, n for a ragged plan); 0 for NULL.
 *   mw_plan_band_limit  L of map b (ragged plans: L[b]).
 *   mw_plan_spin        spin of map b.
 *   mw_plan_map_offset  element offset of map b in the map buffer (complex
 *                       doubles; real doubles on a MW_FLAG_REAL plan): the
 *                       prefix sum of (L-1)(2L-1)+1 over the maps before b.
 *   mw_plan_flm_offset  element offset of map b's f_lm block (complex
 *                       doubles): the prefix sum of L*L over the maps before b.
 * For uniform plans these are b*N_MW and b*L*L.  Each returns -1 for a NULL
 * plan or b outside [0, batch).  Host-only: no device work. */
int mw_plan_batch(const mw_plan *plan);
/* The same offsets without a plan (host-only, allocates nothing): for n maps of
 * band limits L[0..n-1] (1 <= L[b] <= 2048), map_offsets[b] and flm_offsets[b]
 * (either may be NULL) receive the prefix sums of (L-1)(2L-1)+1 and of L*L;
 * entry n of each (arrays of n + 1 elements) receives the total.  MW_EINVAL for
 * n < 1, a NULL L or a band limit out of range. */
mw_status mw_layout_ragged(int n, const int *L, long long *map_offsets, long long *flm_offsets);
int mw_plan_band_limit(const mw_plan *plan, int b);
int mw_plan_spin(const mw_plan *plan, int b);
long long mw_plan_map_offset(const mw_plan *plan, int b);
long long mw_plan_flm_offset(const mw_plan *plan, int b);

/* Forward transform (Sec. IV-D): map_in [batch][N_MW] -> flm_out [batch][L*L].
 * The result is that of the paper's algorithm: phi DFT of each ring (Eq. Gmt
 * discretised), periodic extension in theta with parity (-1)^(m+s), theta DFT
 * to F_mm', quadrature-weight convolution Eq. (Gmm_convolution), and the Wigner
 * sum Eq. (flm_wig).  It is exact for band-limited maps (forward(inverse(f)) = f)
 * and defined by those steps for any other map. */
mw_status mw_forward(mw_plan *plan, const void *map_in, void *flm_out, void *stream);

/* Inverse transform (Sec. IV-E): flm_in [batch][L*L] -> map_out [batch][N_MW]
 * through Eq. (Fmm) (with F_{m,-m'} = (-1)^(m+s) F_mm', Eq. Fmm_sym1),
 * Eq. (Fmt) and Eq. (f_pfft); it equals the synthesis sum_lm f_lm sY_lm on the
 * grid. */
mw_status mw_inverse(mw_plan *plan, const void *flm_in, void *map_out, void *stream);

/* Fused forward + inverse of independent inputs: the forward transform of
 * map_in [batch][N_MW] -> flm_out [batch][L*L] and the inverse transform of
 * flm_in [batch][L*L] -> map_out [batch][N_MW] in one call that runs the
 * Wigner-Delta recursion (Sec. V-B) once for both Wigner sums, Eq. (flm_wig)
 * and Eq. (Fmm): Delta^l depends on neither the direction nor the data, so each
 * plane l feeds both contractions while it is resident.  The results are
 * bitwise those of mw_forward(map_in) and mw_inverse(flm_in) on this plan.  The
 * four buffers must not overlap.  The first fused call on a plan allocates a
 * second set of workspace (the inverse half's), counted by
 * mw_plan_workspace_bytes; with MW_FLAG_GRAPH the whole call is one graph. */
mw_status mw_forward_inverse(mw_plan *plan, const void *map_in, void *flm_out, const void *flm_in, void *map_out,
                             void *stream);

/* Hermitian adjoints (not in the paper; used for gradients):
 * mw_forward_adjoint: flm_in [batch][L*L] -> map_out [batch][N_MW], = forward^H.
 * mw_inverse_adjoint: map_in [batch][N_MW] -> flm_out [batch][L*L], = inverse^H.
 * Each runs the stages of its transform in reverse order, conjugated; the
 * Wigner-Delta planes are recomputed, never stored. */
mw_status mw_forward_adjoint(mw_plan *plan, const void *flm_in, void *map_out, void *stream);
mw_status mw_inverse_adjoint(mw_plan *plan, const void *map_in, void *flm_out, void *stream);

/* MW quadrature rule (Sec. IV-F, Eq. quadrature): the integral over the sphere
 * of a map band-limited at L from L(L-1)+1 samples,
 *   I = sum_{t<L} sum_{p<L} f(theta_t, 2 pi p / L) q(theta_t),
 *   q(theta_t) = (2 pi / L) [ v(theta_t) + (1 - delta_{t,L-1}) (-1)^s v(theta_{2L-2-t}) ],
 *   v(theta_t) = 1/(2L-1) sum_{|m'| <= L-1} w(-m') e^{i m' theta_t}
 * (the Kronecker delta of the printed formula read as delta_{t,L-1}).
 * Quadrature layout of a map (complex doubles): rings t = 0..L-2, each with L
 * samples at phi'_p = 2 pi p / L, then ONE pole sample f(pi, 0) (its ring is
 * f(pi, 0) e^{i s phi}).
 * mw_quadrature_weights: q(theta_t), t = 0..L-1, into q_out (L doubles, device
 *   memory); 1 <= L <= 2048, |s| < L.  Allocates nothing.
 * mw_quadrature: for a uniform plan (not ragged), the integrals of its batch of
 *   maps in the quadrature layout, maps_q [batch][L(L-1)+1] -> integrals
 *   [batch] (complex doubles), both device memory; map b uses spin spins[b].
 *   The first call allocates the plan's weight table and partial sums.
 *   Results are bitwise reproducible (fixed-order reductions). */
mw_status mw_quadrature_weights(int L, int s, double *q_out, void *stream);
mw_status mw_quadrature(mw_plan *plan, const void *maps_q, void *integrals, void *stream);

/* Wait for the plan's work on `stream` and report device-side errors: returns
 * MW_ETIMEOUT (and clears the flag) if a bounded wait inside a kernel (a
 * tensor-core pipeline stage, or a neighbour's plane tile in Risbo's sweep)
 * gave up since the last check -- the affected outputs are then invalid and
 * the plan stays usable -- MW_ECUDA if the stream reports an error, MW_OK
 * otherwise.  Debug environment variables, read at every launch of Risbo's
 * sweep and never set in normal use: MW_DEBUG_STALL_PLANE=<l> makes one block
 * of the sweep leave before plane l without publishing it, and
 * MW_DEBUG_POLLS=<n> limits every neighbour wait to n polls, so that the
 * timeout path can be exercised without faulting or hanging the GPU. */
mw_status mw_plan_sync(mw_plan *plan, void *stream);

/* Free a plan and its workspace.  NULL-safe.  Synchronises the device. */
mw_status mw_plan_destroy(mw_plan *plan);

/* Static description of a status code. */
const char *mw_status_string(mw_status st);

/* Buffer sizes in complex elements per map: (L-1)(2L-1)+1 and L*L (0 for L < 1). */
size_t mw_map_size(int L);
size_t mw_flm_size(int L);

/* Plan introspection: bytes of device workspace held, and the number of
 * kernels the last call on this plan launched. */
size_t mw_plan_workspace_bytes(const mw_plan *plan);
int mw_plan_last_launches(const mw_plan *plan);

/* 1 if the plan's length-(2L-1) DFTs (the phi DFTs of Sec. IV-D / Eq. f_pfft
 * and the theta DFTs over the 2L-1 extended nodes, Sec. IV-C) run by
 * Bluestein's chirp-z convolution through the smooth convolution length
 * N >= 4L-3 (ragged plans: for at least one band limit), 0 if by the mixed-radix
 * factorisation of 2L-1, -1 for NULL.  The plan picks the cheaper route from
 * the factors of 2L-1 (a prime such as 4093 at L = 2047 takes Bluestein);
 * the environment variable MW_FFT_BLUESTEIN=0 or =1, read at plan creation,
 * forces either.  Both compute the same DFT; results differ by rounding. */
int mw_plan_fft_bluestein(const mw_plan *plan);

/* Per-stage timing (diagnostics, not in the paper).  With timing enabled, each
 * call records CUDA events on its stream around every stage:
 *   MW_STAGE_PHI     phi DFTs (and their adjoints); on real plans also the
 *                    f_lm pack / unpack of the map pairs
 *   MW_STAGE_THETA   theta extension / DFT / weight convolution (and adjoints)
 *   MW_STAGE_DELTA   recursion of the Wigner-Delta planes (Risbo or Trapani-Navaza)
 *   MW_STAGE_CONTRACT Delta contraction (forward or inverse sum)
 * mw_plan_stage_times waits for the recorded events, adds their durations to
 * running totals and returns them: ms[MW_NUM_STAGES] milliseconds and
 * launches[MW_NUM_STAGES] kernel launches since the last reset (either pointer
 * may be NULL); reset != 0 clears the totals afterwards. */
enum { MW_STAGE_PHI = 0, MW_STAGE_THETA = 1, MW_STAGE_DELTA = 2, MW_STAGE_CONTRACT = 3, MW_NUM_STAGES = 4 };
mw_status mw_plan_set_timing(mw_plan *plan, int enable);
mw_status mw_plan_stage_times(mw_plan *plan, double *ms, long long *launches, int reset);

/* Tuning (not in the paper): how the mixed-precision Wigner stage is cut into
 * launches and passes.  None of it changes what is computed; `groups` and
 * `tn_threads` leave results bitwise unchanged, `chunk` moves where the
 * inverse contraction's float-float partial sums are added (differences at
 * the 1e-7 level, inside the 1e-6 bar).
 *   chunk       Wigner planes per recursion + contraction launch: 128, 256 or
 *               512 (mixed precisions; the FP64 path stages 64 planes).
 *   groups      spin groups of up to 8 maps per pass of the BF16x3
 *               contraction pipeline: 1 or 2.
 *   tn_threads  columns per block of the Trapani-Navaza recursion: 128 or 256.
 *   ms          one inverse + forward of the plan's batch with these values, in
 *               milliseconds, as measured by mw_plan_autotune (0: not measured).
 * mw_plan_get_tuning  the plan's current values.
 * mw_plan_set_tuning  apply values (MW_EINVAL if one is out of range; ms is
 *                     kept as given).  Discards the plan's captured graphs.
 * mw_plan_autotune    time every candidate (chunk x groups x tn_threads, those
 *                     that apply to the plan's precision and recursion) with
 *                     CUDA events on `stream` over one inverse + forward of
 *                     the plan's batch on scratch buffers it allocates and
 *                     frees, apply the fastest and record it in MW_TUNE_CACHE
 *                     when that variable is set.  Synchronises `stream`.
 * Host-only helpers (no device work), for callers that manage caches:
 * mw_tune_key           the cache key of a plan of n maps (band limits L[b],
 *                       spins spins[b], the plan's flags) on a device of the
 *                       given name: the sorted multiset of (L, s), precision,
 *                       recursion, real-signal flag and device.  MW_EINVAL if
 *                       `len` is too small (the key is then not written).
 * mw_tune_cache_lookup  *found = 1 and *out filled if the file at `path` holds
 *                       `key`; *found = 0 if not, or if the file is absent.
 * mw_tune_cache_store   add `key` with *t to the file at `path`, replacing an
 *                       existing line of the same key (written to a temporary
 *                       file and renamed into place).  MW_EINVAL on I/O failure. */
typedef struct {
  int chunk;
  int groups;
  int tn_threads;
  double ms;
} mw_tuning;
mw_status mw_plan_get_tuning(const mw_plan *plan, mw_tuning *out);
mw_status mw_plan_set_tuning(mw_plan *plan, const mw_tuning *t);
mw_status mw_plan_autotune(mw_plan *plan, void *stream);
mw_status mw_tune_key(int n, const int *L, const int *spins, unsigned flags, const char *device, char *key,
                      size_t len);
mw_status mw_tune_cache_lookup(const char *path, const char *key, mw_tuning *out, int *found);
mw_status mw_tune_cache_store(const char *path, const char *key, const mw_tuning *t);

/* mw_inverse_noalloc: the inverse transform of ONE map of band limit L and spin
 * s, FP64 throughout, that allocates no memory at all -- no plan, no
 * cudaMalloc/cudaFree, no allocating library routine.  The paper has no
 * counterpart: it exists for callers that cannot allocate device memory --
 * code inside a custom allocator's own callbacks (which must not re-enter the
 * allocator), hosts that forbid allocation after start-up (real-time loops,
 * where cudaMalloc/cudaFree would also synchronise the device), or processes
 * that have handed all free device memory to another memory pool.
 *   flm_in  : L*L complex doubles (layout above), device or managed memory of
 *             the current device
 *   map_out : N_MW complex doubles (layout above), device or managed memory of
 *             the current device; must not overlap flm_in
 *   stream  : cudaStream_t of the current device (NULL: legacy default stream)
 * Limits: 1 <= L <= MW_NOALLOC_MAX_L and |s| < L; anything else, host
 * pointers included, returns MW_EINVAL before anything is enqueued.
 * Scratch: the Wigner-Delta planes and the F_mm' coefficients live in one
 * static device array of MW_NOALLOC_SCRATCH_BYTES (about 2.6 MB), which every
 * GPU that loads libmw holds until the process exits.  Every call made
 * outside a stream capture looks up that array's device address on the
 * current device (so a context reset does not leave a stale address behind);
 * a call made while its stream is being captured reuses the address the last
 * such lookup on that device found, so make one call on each device before
 * any stream capture begins.
 * Every call on a device uses the same array and finds the previous call's
 * contents there (the kernels clear what must start at zero), so calls whose
 * GPU work overlaps -- two streams, or two host threads -- race and give wrong
 * results: order them on one stream or with events.  Enqueues two kernels and
 * returns before the GPU finishes; MW_ECUDA if a CUDA call or launch fails. */
#define MW_NOALLOC_MAX_L 128
#define MW_NOALLOC_SCRATCH_BYTES 2601744u
mw_status mw_inverse_noalloc(int L, int s, const void *flm_in, void *map_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MW_H */
