/* A plain C11 client of the C ABI in include/dies.h: one small externally
 * heated cloud (4 shells, 3 frequencies), every setter, then one run.  With a
 * GPU it prints the shell temperatures; without one the run must fail with a
 * status code and a message, not crash.  Exit code: 0 on the expected
 * outcome, 1 otherwise. */
#include <stdio.h>
#include <string.h>

#include "dies.h"

static int check(int rc, const char *what) {
  if (rc != DIES_OK) fprintf(stderr, "%s: status %d (%s)\n", what, rc, dies_last_error());
  return rc;
}

int main(int argc, char **argv) {
  const double radii[5] = {0.0, 0.25, 0.5, 0.75, 1.0};
  const double rho[4] = {4.0, 2.0, 1.0, 0.5};
  const double freq[3] = {3e12, 3e13, 3e14};
  const double kabs[3] = {0.1, 1.0, 10.0}, ksca[3] = {0.0, 0.5, 5.0}, g[3] = {0.0, 0.3, 0.6};
  const double J[3] = {1e-14, 1e-15, 1e-16};
  const int expect_gpu = (argc > 1 && strcmp(argv[1], "--gpu") == 0);
  dies_model *m = NULL;
  if (check(dies_create_model(radii, 5, rho, 4, 3.0857e17, &m), "create")) return 1;
  int bad = 0;
  bad |= check(dies_set_dust(m, freq, 3, kabs, ksca, g), "dust") != DIES_OK;
  bad |= check(dies_set_sources(m, J, 0.0, NULL), "sources") != DIES_OK;
  dies_weighting w;
  memset(&w, 0, sizeof w);
  w.k_bg = 1.0 / 3.0;
  w.forced_first_interaction = DIES_FFI_ABSORPTION;
  w.k_A = 1.0;
  w.k_S = 1.0;
  bad |= check(dies_set_weighting_ex(m, &w), "weighting") != DIES_OK;
  bad |= check(dies_set_precision(m, DIES_PREC_MIXED, 1, 0.0), "precision") != DIES_OK;
  if (dies_set_weighting(m, 0.5, 7) != DIES_EINVAL) bad = 1; /* unknown forcing mode */
  if (bad) {
    dies_destroy_model(m);
    return 1;
  }
  const int rc = dies_run(m, 100000, 1);
  int ok;
  if (expect_gpu) {
    double T[4];
    ok = (rc == DIES_OK) && dies_get_temperatures(m, T, 4) == DIES_OK;
    if (ok) printf("T = %.3f %.3f %.3f %.3f K\n", T[0], T[1], T[2], T[3]);
  } else {
    ok = (rc == DIES_ECUDA || rc == DIES_ENOMEM) && dies_last_error()[0] != '\0';
    if (ok) printf("no GPU: run refused with status %d (%s)\n", rc, dies_last_error());
  }
  dies_destroy_model(m);
  return ok ? 0 : 1;
}
