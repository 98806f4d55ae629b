/*
 * Host entry points of the seeded phase-space generator (input generator
 * only; no matrix-element arithmetic).  Built as a small shared library so
 * that the CPU tests, the benchmark and the oracle harness can make the same
 * synthetic events that the CUDA generator makes on the device.
 */
#include <stddef.h>
#include "phasespace.h"

#ifdef _OPENMP
#include <omp.h>
#endif

/* out: [n_events][2 + n_final][4] doubles; attempts (nullable): [n_events]. */
int ps_generate_host(const ps_config *cfg, uint64_t first_event,
                     int64_t n_events, double *out, int32_t *attempts) {
  if (!cfg || !out || n_events < 0) return -1;
  if (cfg->n_final < 2 || cfg->n_final > PS_MAX_FINAL) return -1;
  const int n_ext = 2 + cfg->n_final;
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < n_events; ++e) {
    double (*mom)[4] = (double (*)[4])(out + (size_t)e * (size_t)n_ext * 4u);
    int a = ps_generate_event(cfg, first_event + (uint64_t)e, mom);
    if (attempts) attempts[e] = a;
  }
  return 0;
}

/* Raw Philox4x32-10 block, exposed for the known-answer test. */
void ps_philox_host(const uint32_t ctr[4], const uint32_t key[2],
                    uint32_t out[4]) {
  ps_philox4x32_10(ctr, key, out);
}

/* VEGAS points (ps_vegas_event) for events first_event .. first_event + n - 1:
 * out [n][2 + n_final][4], weight [n], bins [n][ps_rambo_dims(n_final)]. */
int ps_vegas_host(const ps_config *cfg, const double *edges, int nb, uint64_t first_event,
                  int64_t n_events, double *out, double *weight, unsigned char *bins) {
  if (!cfg || !edges || !out || !weight || !bins || n_events < 0) return -1;
  if (cfg->n_final < 2 || cfg->n_final > PS_MAX_FINAL || nb < 1 || nb > PS_VEGAS_MAX_BINS) return -1;
  const int n_ext = 2 + cfg->n_final;
  const int dims = ps_rambo_dims(cfg->n_final);
#pragma omp parallel for schedule(static)
  for (int64_t e = 0; e < n_events; ++e) {
    double (*mom)[4] = (double (*)[4])(out + (size_t)e * (size_t)n_ext * 4u);
    weight[e] = ps_vegas_event(cfg, edges, nb, first_event + (uint64_t)e, mom, bins + (size_t)e * (size_t)dims);
  }
  return 0;
}
