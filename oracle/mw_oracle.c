/*
 * mw_oracle.c -- plain FP64 CPU oracle for the Wigner stages of the McEwen-Wiaux
 * (MW) spin spherical harmonic transforms (McEwen & Wiaux, IEEE TSP 2011).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or calls
 * this file; only tests/, the smoke check and the CPU-baseline leg of the
 * benchmark do.  It shares no code with the CUDA library.
 *
 * What it computes, in the paper's notation (Delta^l_{mn} = d^l_{mn}(pi/2)):
 *   - Wigner d planes d^j(beta) for j = 0, 1/2, 1, ..., by Risbo's recursion
 *     (the recursion the paper uses, Sec. V-B/V-C; its formula is not printed in
 *     the paper, so the scatter form below is the classical statement of the
 *     coupling with spin 1/2, and the tests pin it against Wigner's explicit
 *     d-function sum and against Eq. (wignerd_b)).
 *   - forward Wigner stage, Eq. (flm_wig):
 *       f_lm = (-1)^s i^(m+s) sqrt((2l+1)/4pi) sum_m' Delta^l_{m'm} Delta^l_{m',-s} G_mm'
 *   - inverse Wigner stage, Eq. (Fmm):
 *       F_mm' = (-1)^s i^-(m+s) sum_l sqrt((2l+1)/4pi) Delta^l_{m'm} Delta^l_{m',-s} f_lm
 *   - d^l_{m,-s}(theta) on chosen rings through the Fourier relation
 *     Eq. (wigner_sum_reln), and F_m(theta) = (-1)^s sum_l sqrt((2l+1)/4pi)
 *     d^l_{m,-s}(theta) f_lm (the representation printed in the footnote of
 *     Sec. IV-B), for spot checks of large inverse transforms one ring at a time.
 *
 * Conventions: complex numbers are interleaved (re, im) doubles.  A full plane of
 * d^j has size P = 2j+1 and is stored row-major with row i = m + j and column
 * k = n + j for d^j_{mn}.  Arrays over m in [-(L-1), L-1] are stored at index
 * m + L - 1.  f_lm is stored at index l*l + l + m.
 * Compile with -ffp-contract=off so that x86-64 and aarch64 round identically.
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* One half step of Risbo's recursion: plane d^j (size P = 2j+1) -> d^{j+1/2}
 * (size P+1), rotation angle beta through p = cos(beta/2), q = sin(beta/2).
 * Each entry d[i][k] of the old plane is coupled with the spin-1/2 matrix and
 * scattered onto four entries of the new plane:
 *   e[i][k]     += sqrt((P-i)(P-k))/P * p * d[i][k]
 *   e[i+1][k]   -= sqrt((i+1)(P-k))/P * q * d[i][k]
 *   e[i][k+1]   += sqrt((P-i)(k+1))/P * q * d[i][k]
 *   e[i+1][k+1] += sqrt((i+1)(k+1))/P * p * d[i][k]
 * Rows i of one parity write rows i and i+1 only, so each parity is a parallel
 * loop without races. */
static void risbo_half_step(int P, const double *d, double *e, double p, double q) {
  const int Q = P + 1;
  double *sq = (double *)malloc(sizeof(double) * (size_t)(P + 2));
  for (int x = 0; x <= P + 1; ++x) sq[x] = sqrt((double)x);
  memset(e, 0, sizeof(double) * (size_t)Q * Q);
  for (int parity = 0; parity < 2; ++parity) {
#pragma omp parallel for schedule(static)
    for (int i = parity; i < P; i += 2) {
      for (int k = 0; k < P; ++k) {
        const double v = d[(size_t)i * P + k] / P;
        e[(size_t)i * Q + k] += sq[P - i] * sq[P - k] * p * v;
        e[(size_t)(i + 1) * Q + k] -= sq[i + 1] * sq[P - k] * q * v;
        e[(size_t)i * Q + k + 1] += sq[P - i] * sq[k + 1] * q * v;
        e[(size_t)(i + 1) * Q + k + 1] += sq[i + 1] * sq[k + 1] * p * v;
      }
    }
  }
  free(sq);
}

/* Full plane d^j(beta) with two_j = 2j, written to out[(2j+1)^2].  Runs the
 * recursion from d^0 = [1].  Returns 0, or -1 on allocation failure. */
int orc_wigner_plane(int two_j, double beta, double *out) {
  if (two_j < 0) return -1;
  const double p = cos(0.5 * beta), q = sin(0.5 * beta);
  const size_t cap = (size_t)(two_j + 1) * (two_j + 1);
  double *a = (double *)malloc(sizeof(double) * cap);
  double *b = (double *)malloc(sizeof(double) * cap);
  if (!a || !b) { free(a); free(b); return -1; }
  a[0] = 1.0;
  for (int P = 1; P <= two_j; ++P) {
    risbo_half_step(P, a, b, p, q);
    double *t = a; a = b; b = t;
  }
  memcpy(out, a, sizeof(double) * cap);
  free(a); free(b);
  return 0;
}

/* i^k for integer k, as (re, im). */
static void ipow(int k, double *re, double *im) {
  int r = ((k % 4) + 4) % 4;
  *re = (r == 0) ? 1.0 : (r == 2) ? -1.0 : 0.0;
  *im = (r == 1) ? 1.0 : (r == 3) ? -1.0 : 0.0;
}

/* Sweep context: holds Delta^l for the current l as a full plane. */
typedef struct { double *cur, *half, *next; int l; } sweep_t;

static int sweep_init(sweep_t *sw, int L) {
  const size_t cap = (size_t)(2 * L + 1) * (2 * L + 1);
  sw->cur = (double *)malloc(sizeof(double) * cap);
  sw->half = (double *)malloc(sizeof(double) * cap);
  sw->next = (double *)malloc(sizeof(double) * cap);
  if (!sw->cur || !sw->half || !sw->next) return -1;
  sw->cur[0] = 1.0; sw->l = 0;
  return 0;
}
static void sweep_advance(sweep_t *sw) {  /* Delta^l -> Delta^{l+1}: two half steps */
  const double c = sqrt(0.5);
  const int P = 2 * sw->l + 1;
  risbo_half_step(P, sw->cur, sw->half, c, c);
  risbo_half_step(P + 1, sw->half, sw->next, c, c);
  double *t = sw->cur; sw->cur = sw->next; sw->next = t;
  sw->l += 1;
}
static void sweep_free(sweep_t *sw) { free(sw->cur); free(sw->half); free(sw->next); }

/* Forward Wigner stage, Eq. (flm_wig), for nmaps maps of spin s.
 *   G   : [nmaps][M][M] complex, G[b][m+L-1][m'+L-1] = G_mm'   (M = 2L-1)
 *   flm : [nmaps][L*L] complex output; entries with l < |s| are set to 0.
 *   m_list/nm: if m_list != NULL only those m are computed (others left as they
 *   are in flm), so that large transforms can be spot-checked column by column.
 * For each output the sum over m' runs in ascending order, m' = -l..l (Delta^l
 * vanishes for |m'| > l).  Returns 0, or -1 on bad arguments / allocation. */
int orc_forward_wigner(int L, int s, int nmaps, const double *G, const int *m_list, int nm,
                       double *flm) {
  if (L < 1 || abs(s) >= L || nmaps < 1) return -1;
  const int M = 2 * L - 1;
  int *ms = (int *)malloc(sizeof(int) * (m_list ? nm : M));
  if (!ms) return -1;
  int cnt = 0;
  if (m_list) { for (int a = 0; a < nm; ++a) { if (m_list[a] <= -L || m_list[a] >= L) { free(ms); return -1; } ms[cnt++] = m_list[a]; } }
  else { for (int m = -(L - 1); m <= L - 1; ++m) ms[cnt++] = m; }
  for (int b = 0; b < nmaps; ++b)
    for (int l = 0; l < L; ++l)
      for (int a = 0; a < cnt; ++a) {
        const int m = ms[a];
        if (abs(m) > l) continue;
        double *o = flm + 2 * ((size_t)b * L * L + (size_t)l * l + l + m);
        o[0] = 0.0; o[1] = 0.0;
      }
  sweep_t sw;
  if (sweep_init(&sw, L)) { free(ms); sweep_free(&sw); return -1; }
  for (int l = 0; l < L; ++l) {
    if (l > 0) sweep_advance(&sw);
    if (l < abs(s)) continue;
    const int P = 2 * l + 1;
    const double *D = sw.cur;  /* D[(m'+l)*P + (m+l)] = Delta^l_{m'm} */
    const double Nl = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
    double pr, pi_;
#pragma omp parallel for schedule(dynamic, 4) private(pr, pi_)
    for (int a = 0; a < cnt; ++a) {
      const int m = ms[a];
      if (abs(m) > l) continue;
      ipow(m + s, &pr, &pi_);
      const double sg = (s % 2 == 0) ? 1.0 : -1.0;
      for (int b = 0; b < nmaps; ++b) {
        const double *Gm = G + 2 * ((size_t)b * M * M + (size_t)(m + L - 1) * M);
        double accr = 0.0, acci = 0.0;
        for (int mp = -l; mp <= l; ++mp) {
          const double k = D[(size_t)(mp + l) * P + (m + l)] * D[(size_t)(mp + l) * P + (-s + l)];
          accr += k * Gm[2 * (mp + L - 1)];
          acci += k * Gm[2 * (mp + L - 1) + 1];
        }
        /* times (-1)^s i^(m+s) sqrt((2l+1)/4pi) */
        const double cr = sg * Nl * pr, ci = sg * Nl * pi_;
        double *o = flm + 2 * ((size_t)b * L * L + (size_t)l * l + l + m);
        o[0] = cr * accr - ci * acci;
        o[1] = cr * acci + ci * accr;
      }
    }
  }
  sweep_free(&sw);
  free(ms);
  return 0;
}

/* Inverse Wigner stage, Eq. (Fmm), for nmaps maps of spin s.
 *   flm : [nmaps][L*L] complex input (entries with l < |s| are ignored)
 *   F   : [nmaps][M][M] complex output, F[b][m+L-1][m'+L-1] = F_mm'
 * Every (m, m') is computed directly; for each output the sum over l runs in
 * ascending order.  Returns 0, or -1 on bad arguments / allocation. */
int orc_inverse_wigner(int L, int s, int nmaps, const double *flm, double *F) {
  if (L < 1 || abs(s) >= L || nmaps < 1) return -1;
  const int M = 2 * L - 1;
  memset(F, 0, sizeof(double) * 2 * (size_t)nmaps * M * M);
  sweep_t sw;
  if (sweep_init(&sw, L)) { sweep_free(&sw); return -1; }
  for (int l = 0; l < L; ++l) {
    if (l > 0) sweep_advance(&sw);
    if (l < abs(s)) continue;
    const int P = 2 * l + 1;
    const double *D = sw.cur;
    const double Nl = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
#pragma omp parallel for schedule(static)
    for (int m = -l; m <= l; ++m) {
      for (int b = 0; b < nmaps; ++b) {
        const double *f = flm + 2 * ((size_t)b * L * L + (size_t)l * l + l + m);
        double *Fm = F + 2 * ((size_t)b * M * M + (size_t)(m + L - 1) * M);
        for (int mp = -l; mp <= l; ++mp) {
          const double k = Nl * D[(size_t)(mp + l) * P + (m + l)] * D[(size_t)(mp + l) * P + (-s + l)];
          Fm[2 * (mp + L - 1)] += k * f[0];
          Fm[2 * (mp + L - 1) + 1] += k * f[1];
        }
      }
    }
  }
  sweep_free(&sw);
  /* times (-1)^s i^-(m+s) */
  for (int b = 0; b < nmaps; ++b)
    for (int m = -(L - 1); m <= L - 1; ++m) {
      double pr, pi_;
      ipow(-(m + s), &pr, &pi_);
      const double sg = (s % 2 == 0) ? 1.0 : -1.0;
      double *Fm = F + 2 * ((size_t)b * M * M + (size_t)(m + L - 1) * M);
      for (int j = 0; j < M; ++j) {
        const double re = Fm[2 * j], im = Fm[2 * j + 1];
        Fm[2 * j] = sg * (pr * re - pi_ * im);
        Fm[2 * j + 1] = sg * (pr * im + pi_ * re);
      }
    }
  return 0;
}

/* F_m(theta) on nth chosen colatitudes, for nmaps maps of spin s:
 *   d^l_{m,-s}(theta) = i^(-s-m) sum_m' Delta^l_{m'm} Delta^l_{m',-s} e^{i m' theta}
 *                                                          (Eq. wigner_sum_reln)
 *   F_m(theta)        = (-1)^s sum_l sqrt((2l+1)/4pi) d^l_{m,-s}(theta) f_lm
 *   out : [nmaps][nth][M] complex, out[b][r][m+L-1] = F_m(theta_r).
 * Returns 0, or -1 on bad arguments / allocation. */
int orc_inverse_rings(int L, int s, int nmaps, const double *flm, int nth, const double *theta,
                      double *out) {
  if (L < 1 || abs(s) >= L || nmaps < 1 || nth < 1) return -1;
  const int M = 2 * L - 1;
  memset(out, 0, sizeof(double) * 2 * (size_t)nmaps * nth * M);
  double *dth = (double *)malloc(sizeof(double) * 2 * (size_t)nth * M);
  double *ex = (double *)malloc(sizeof(double) * 2 * (size_t)nth * M); /* e^{i m' theta_r} */
  sweep_t sw;
  if (!dth || !ex || sweep_init(&sw, L)) { free(dth); free(ex); sweep_free(&sw); return -1; }
  for (int r = 0; r < nth; ++r)
    for (int mp = -(L - 1); mp <= L - 1; ++mp) {
      ex[2 * ((size_t)r * M + mp + L - 1)] = cos(mp * theta[r]);
      ex[2 * ((size_t)r * M + mp + L - 1) + 1] = sin(mp * theta[r]);
    }
  const double sg = (s % 2 == 0) ? 1.0 : -1.0;
  for (int l = 0; l < L; ++l) {
    if (l > 0) sweep_advance(&sw);
    if (l < abs(s)) continue;
    const int P = 2 * l + 1;
    const double *D = sw.cur;
    const double Nl = sqrt((2.0 * l + 1.0) / (4.0 * M_PI));
    /* sum over m' in ascending order for every (theta_r, m); the loop over m is
     * innermost so that plane rows are read contiguously; threads take (ring,
     * block of m) pairs */
    const int nblk = (P + 63) / 64;
#pragma omp parallel for schedule(dynamic, 1)
    for (int task = 0; task < nth * nblk; ++task) {
      const int r = task / nblk, m_lo = -l + (task % nblk) * 64;
      const int m_hi = (m_lo + 63 < l) ? m_lo + 63 : l;
      double *acc = dth + 2 * (size_t)r * M;
      for (int m = m_lo; m <= m_hi; ++m) { acc[2 * (m + L - 1)] = 0.0; acc[2 * (m + L - 1) + 1] = 0.0; }
      for (int mp = -l; mp <= l; ++mp) {
        const double w = D[(size_t)(mp + l) * P + (-s + l)];
        const double er = ex[2 * ((size_t)r * M + mp + L - 1)], ei = ex[2 * ((size_t)r * M + mp + L - 1) + 1];
        const double *row = D + (size_t)(mp + l) * P;
        for (int m = m_lo; m <= m_hi; ++m) {
          const double k = row[m + l] * w;
          acc[2 * (m + L - 1)] += k * er;
          acc[2 * (m + L - 1) + 1] += k * ei;
        }
      }
      for (int m = m_lo; m <= m_hi; ++m) {  /* times i^(-s-m) */
        double pr, pi_;
        ipow(-s - m, &pr, &pi_);
        const double ar = acc[2 * (m + L - 1)], ai = acc[2 * (m + L - 1) + 1];
        acc[2 * (m + L - 1)] = pr * ar - pi_ * ai;
        acc[2 * (m + L - 1) + 1] = pr * ai + pi_ * ar;
      }
    }
#pragma omp parallel for schedule(static) collapse(2)
    for (int b = 0; b < nmaps; ++b)
      for (int r = 0; r < nth; ++r)
        for (int m = -l; m <= l; ++m) {
          const double *f = flm + 2 * ((size_t)b * L * L + (size_t)l * l + l + m);
          const double dr = dth[2 * ((size_t)r * M + m + L - 1)], di = dth[2 * ((size_t)r * M + m + L - 1) + 1];
          double *o = out + 2 * (((size_t)b * nth + r) * M + m + L - 1);
          o[0] += sg * Nl * (dr * f[0] - di * f[1]);
          o[1] += sg * Nl * (dr * f[1] + di * f[0]);
        }
  }
  sweep_free(&sw);
  free(dth); free(ex);
  return 0;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
