/*
 * Seeded synthetic phase-space generator (input generator only).
 *
 * This header is the one module shared by the CUDA path and the CPU test
 * harness: it turns (seed, event index) into partonic momenta.  It holds none
 * of the matrix-element arithmetic.  It compiles as plain C99 on the host and,
 * under nvcc, as __host__ __device__ code.
 *
 * Pieces:
 *   - Philox4x32-10 counter-based generator (Salmon, Moraes, Dror, Shaw,
 *     "Parallel random numbers: as easy as 1, 2, 3", SC'11): 10 rounds of the
 *     4x32 Philox S-box with multipliers 0xD2511F53 / 0xCD9E8D57 and Weyl key
 *     increments 0x9E3779B9 / 0xBB67AE85.
 *   - RAMBO flat massless n-body phase space (Kleiss, Stirling, Ellis,
 *     Comput. Phys. Commun. 40 (1986) 359) in the partonic centre-of-mass frame
 *     (n = 2: a uniform direction, the same distribution drawn directly).
 *   - sqrt(s_hat) drawn log-uniform in [rs_lo, rs_hi]; incoming partons along
 *     +z / -z with energy sqrt(s_hat)/2 each.
 *   - Jet cuts pT > pt_min, |eta| < eta_max and, between every pair of
 *     final-state partons, Delta R > dr_min and (when ptij_min > 0) the
 *     relative transverse momentum min(pT_i, pT_j) Delta R_ij > ptij_min of
 *     the paper's Eq. (cuts-ptjj) -- Eq. (cuts) in the partonic frame.  A
 *     rejected point is redrawn completely with the next attempt counter.
 *
 * Momentum layout: mom[leg][4] = (E, px, py, pz) in GeV, legs ordered
 * (incoming a, incoming b, outgoing 1..n).
 */
#ifndef PS_PHASESPACE_H
#define PS_PHASESPACE_H

#include <stdint.h>
#include <math.h>

#ifdef __CUDACC__
#define PS_HD __host__ __device__ __forceinline__
#else
#define PS_HD static inline
#endif

#define PS_MAX_FINAL 8
#define PS_MAX_ATTEMPTS 4096

typedef struct {
  uint64_t seed;     /* Philox key */
  int n_final;       /* number of outgoing massless partons (2..PS_MAX_FINAL) */
  double rs_lo;      /* sqrt(s_hat) range, GeV */
  double rs_hi;
  double pt_min;     /* GeV */
  double eta_max;
  double dr_min;
  double ptij_min;   /* GeV, <= 0: no relative-pT cut */
} ps_config;

/* ---- Philox4x32-10 ---------------------------------------------------- */
PS_HD void ps_mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
  uint64_t p = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(p >> 32);
  *lo = (uint32_t)p;
}

PS_HD void ps_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2],
                            uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    ps_mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
    ps_mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0;
    uint32_t n1 = lo1;
    uint32_t n2 = hi0 ^ c3 ^ k1;
    uint32_t n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Uniform double in the open interval (0, 1) from two 32-bit words
 * (53 random bits, offset by half an ulp so that 0 never occurs). */
PS_HD double ps_u01(uint32_t a, uint32_t b) {
  uint64_t x = ((uint64_t)(a >> 5) << 26) | (uint64_t)(b >> 6);
  return ((double)x + 0.5) * (1.0 / 9007199254740992.0);
}

/* Stream of uniforms for one (event, attempt): call index j gives 2 doubles. */
typedef struct {
  uint32_t key[2];
  uint32_t ctr[4];
  double buf[2];
  int have;
} ps_stream;

PS_HD void ps_stream_init(ps_stream *s, uint64_t seed, uint64_t event,
                          uint32_t attempt) {
  s->key[0] = (uint32_t)seed;
  s->key[1] = (uint32_t)(seed >> 32);
  s->ctr[0] = 0u;
  s->ctr[1] = attempt;
  s->ctr[2] = (uint32_t)event;
  s->ctr[3] = (uint32_t)(event >> 32);
  s->have = 0;
}

PS_HD double ps_next(ps_stream *s) {
  if (s->have == 0) {
    uint32_t o[4];
    ps_philox4x32_10(s->ctr, s->key, o);
    s->ctr[0] += 1u;
    s->buf[0] = ps_u01(o[0], o[1]);
    s->buf[1] = ps_u01(o[2], o[3]);
    s->have = 2;
  }
  s->have -= 1;
  return s->buf[1 - s->have];
}

/* ---- RAMBO, massless ---------------------------------------------------- */
/* Uniforms RAMBO consumes for n partons: 2 for n = 2 (cos theta, phi), else 4
 * per parton (cos theta, phi, and two for the energy -log(r1 r2)). */
PS_HD int ps_rambo_dims(int n) { return n == 2 ? 2 : 4 * n; }

/* Writes n massless momenta with total momentum (rs, 0, 0, 0) into mom from
 * the ps_rambo_dims(n) uniforms u in (0, 1), in the order listed above. */
PS_HD void ps_rambo_massless_u(const double *u, int n, double rs, double (*mom)[4]) {
  const double twopi = 6.283185307179586476925286766559;
  if (n == 2) {
    /* Flat two-body massless phase space is a uniform direction in the
     * centre-of-mass frame; drawing it directly keeps both momenta exactly
     * back to back and on shell (RAMBO's conformal boost loses digits when
     * its two random vectors are nearly parallel). */
    double c = 2.0 * u[0] - 1.0;
    double sn = sqrt(1.0 - c * c);
    double f = twopi * u[1];
    double e = 0.5 * rs;
    mom[0][0] = e; mom[0][1] = e * sn * cos(f); mom[0][2] = e * sn * sin(f); mom[0][3] = e * c;
    mom[1][0] = e; mom[1][1] = -mom[0][1]; mom[1][2] = -mom[0][2]; mom[1][3] = -mom[0][3];
    return;
  }
  double q[PS_MAX_FINAL][4];
  double Q[4] = {0.0, 0.0, 0.0, 0.0};
  for (int i = 0; i < n; ++i) {
    double c = 2.0 * u[4 * i] - 1.0;
    double sn = sqrt(1.0 - c * c);
    double f = twopi * u[4 * i + 1];
    double r1 = u[4 * i + 2];
    double r2 = u[4 * i + 3];
    double e = -log(r1 * r2);
    q[i][0] = e;
    q[i][3] = e * c;
    q[i][2] = e * sn * sin(f);
    q[i][1] = e * sn * cos(f);
    for (int k = 0; k < 4; ++k) Q[k] += q[i][k];
  }
  double M = sqrt(Q[0] * Q[0] - Q[1] * Q[1] - Q[2] * Q[2] - Q[3] * Q[3]);
  double b[3] = {-Q[1] / M, -Q[2] / M, -Q[3] / M};
  double g = Q[0] / M;
  double a = 1.0 / (1.0 + g);
  double x = rs / M;
  for (int i = 0; i < n; ++i) {
    double bq = b[0] * q[i][1] + b[1] * q[i][2] + b[2] * q[i][3];
    mom[i][0] = x * (g * q[i][0] + bq);
    for (int k = 0; k < 3; ++k)
      mom[i][k + 1] = x * (q[i][k + 1] + b[k] * q[i][0] + a * bq * b[k]);
  }
  /* The boost above loses digits when Q is nearly light-like.  Remove the
   * residual total 3-momentum, put every parton back on shell (E = |p|) and
   * rescale to the exact total energy: a change at the 1e-13 level that
   * makes the point consistent to rounding. */
  double r[3] = {0.0, 0.0, 0.0};
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 3; ++k) r[k] += mom[i][k + 1];
  double esum = 0.0;
  for (int i = 0; i < n; ++i) {
    for (int k = 0; k < 3; ++k) mom[i][k + 1] -= r[k] / (double)n;
    mom[i][0] = sqrt(mom[i][1] * mom[i][1] + mom[i][2] * mom[i][2] + mom[i][3] * mom[i][3]);
    esum += mom[i][0];
  }
  double f = rs / esum;
  for (int i = 0; i < n; ++i)
    for (int k = 0; k < 4; ++k) mom[i][k] *= f;
}

/* RAMBO drawing its uniforms from the stream. */
PS_HD void ps_rambo_massless(ps_stream *s, int n, double rs, double (*mom)[4]) {
  double u[4 * PS_MAX_FINAL];
  const int d = ps_rambo_dims(n);
  for (int k = 0; k < d; ++k) u[k] = ps_next(s);
  ps_rambo_massless_u(u, n, rs, mom);
}

/* ---- cuts ---------------------------------------------------------------- */
PS_HD int ps_pass_cuts(const ps_config *cfg, int n, double (*p)[4]) {
  const double pi = 3.14159265358979323846264338328;
  double eta[PS_MAX_FINAL], phi[PS_MAX_FINAL], pts[PS_MAX_FINAL];
  for (int i = 0; i < n; ++i) {
    double pt = sqrt(p[i][1] * p[i][1] + p[i][2] * p[i][2]);
    if (!(pt > cfg->pt_min)) return 0;
    pts[i] = pt;
    eta[i] = asinh(p[i][3] / pt);
    if (!(fabs(eta[i]) < cfg->eta_max)) return 0;
    phi[i] = atan2(p[i][2], p[i][1]);
  }
  for (int i = 0; i < n; ++i)
    for (int j = i + 1; j < n; ++j) {
      double dphi = phi[i] - phi[j];
      while (dphi > pi) dphi -= 2.0 * pi;
      while (dphi <= -pi) dphi += 2.0 * pi;
      double deta = eta[i] - eta[j];
      double dr2 = deta * deta + dphi * dphi;
      if (!(dr2 > cfg->dr_min * cfg->dr_min)) return 0;
      if (cfg->ptij_min > 0.0 && !(fmin(pts[i], pts[j]) * sqrt(dr2) > cfg->ptij_min)) return 0;
    }
  return 1;
}

/* One accepted event: mom[(2 + n_final)][4].  Returns the attempt index that
 * was accepted, or -1 if PS_MAX_ATTEMPTS draws were all rejected (the last
 * draw is still written, so the output is always finite). */
PS_HD int ps_generate_event(const ps_config *cfg, uint64_t event,
                            double (*mom)[4]) {
  int n = cfg->n_final;
  int accepted = -1;
  for (uint32_t att = 0; att < PS_MAX_ATTEMPTS; ++att) {
    ps_stream s;
    ps_stream_init(&s, cfg->seed, event, att);
    double u = ps_next(&s);
    double rs = cfg->rs_lo * exp(u * log(cfg->rs_hi / cfg->rs_lo));
    double half = 0.5 * rs;
    mom[0][0] = half; mom[0][1] = 0.0; mom[0][2] = 0.0; mom[0][3] = half;
    mom[1][0] = half; mom[1][1] = 0.0; mom[1][2] = 0.0; mom[1][3] = -half;
    ps_rambo_massless(&s, n, rs, mom + 2);
    if (ps_pass_cuts(cfg, n, mom + 2)) { accepted = (int)att; break; }
  }
  return accepted;
}

/* ---- VEGAS points at fixed sqrt(s_hat) ------------------------------------ *
 * Adaptive importance sampling (G. P. Lepage, J. Comput. Phys. 27 (1978) 192)
 * over RAMBO's uniforms: dimension d has nb bins with edges
 * e[d][0] = 0 < e[d][1] < ... < e[d][nb] = 1; a uniform x lands in bin
 * i = floor(x nb) and maps linearly into [e[d][i], e[d][i+1]], with Jacobian
 * nb (e[d][i+1] - e[d][i]).  A point that fails the cuts has weight 0 (no
 * redraw).  The uniforms are those of attempt PS_VEGAS_ATTEMPT of the event,
 * a counter range the flat generator never reaches. */
#define PS_VEGAS_MAX_BINS 64
#define PS_VEGAS_ATTEMPT 0xFFFFFFFFu

/* mom[2 + n_final][4] <- the point of `event` (incoming legs along +-z at
 * sqrt(s_hat) = cfg->rs_lo); bins[d] <- its bin per dimension; returns the
 * weight (product of the Jacobians) or 0 when the cuts reject the point.
 * edges: [ps_rambo_dims(n_final)][nb + 1]. */
PS_HD double ps_vegas_event(const ps_config *cfg, const double *edges, int nb, uint64_t event,
                            double (*mom)[4], unsigned char *bins) {
  const int n = cfg->n_final;
  const int dims = ps_rambo_dims(n);
  ps_stream s;
  ps_stream_init(&s, cfg->seed, event, PS_VEGAS_ATTEMPT);
  double u[4 * PS_MAX_FINAL];
  double w = 1.0;
  for (int d = 0; d < dims; ++d) {
    const double x = ps_next(&s) * (double)nb;
    int b = (int)x;
    if (b > nb - 1) b = nb - 1;
    const double *e = edges + (size_t)d * (size_t)(nb + 1);
    const double width = e[b + 1] - e[b];
    double y = e[b] + (x - (double)b) * width;
    if (!(y > 0.0)) y = 0x1p-60;
    if (!(y < 1.0)) y = 1.0 - 0x1p-53;
    u[d] = y;
    w *= (double)nb * width;
    bins[d] = (unsigned char)b;
  }
  const double rs = cfg->rs_lo, half = 0.5 * rs;
  mom[0][0] = half; mom[0][1] = 0.0; mom[0][2] = 0.0; mom[0][3] = half;
  mom[1][0] = half; mom[1][1] = 0.0; mom[1][2] = 0.0; mom[1][3] = -half;
  ps_rambo_massless_u(u, n, rs, mom + 2);
  return ps_pass_cuts(cfg, n, mom + 2) ? w : 0.0;
}

#endif /* PS_PHASESPACE_H */
