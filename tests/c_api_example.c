/*
 * The C ABI used from plain C, without Python or PyTorch: draw an ensemble,
 * take the Wilson-loop group sums of a flux tube on a small grid, and the
 * group statistics of the spinor loop.  Prints one line per point:
 *   p rho T mean(W_ferm - 1) sem  scal_sum(group 0)
 * with %.17g so a caller can compare the numbers bit for bit.
 *
 *   gcc -O2 -I include tests/c_api_example.c -L <dir of libwln.so> -lwln -o c_api_example
 *   ./c_api_example [device]
 * Exit status 0 on success, 1 with the library's message on failure.
 */
#include <stdio.h>
#include <stdlib.h>

#include "wln.h"

static int check(wln_ctx* ctx, wln_status st, const char* what) {
  if (st == WLN_OK) return 0;
  fprintf(stderr, "%s failed (%d): %s\n", what, (int)st, ctx ? wln_last_error(ctx) : "");
  return 1;
}

int main(int argc, char** argv) {
  const int device = argc > 1 ? atoi(argv[1]) : 0;
  const int32_t n_loops = 1024, ppl = 256, G = 8;
  wln_ctx* ctx = NULL;
  if (wln_create(&ctx, device, NULL) != WLN_OK) {
    fprintf(stderr, "wln_create failed\n");
    return 1;
  }
  wln_ensemble* ens = NULL;
  if (check(ctx, wln_gen_loops(ctx, 1, 0, n_loops, ppl, 0, &ens), "wln_gen_loops")) return 1;

  wln_profile tube = {WLN_PROFILE_FLUX_TUBE, 0, 10.0, 1.0, 0.0};
  const double rho[4] = {0.0, 1.0, 2.0, 3.0};
  const double T[3] = {0.1, 1.0, 10.0};
  const int32_t rho_off[2] = {0, 4}, T_off[2] = {0, 3};
  const int32_t n_points = 12;

  double* S = (double*)malloc(sizeof(double) * n_points * G * WLN_K);
  double mean[12], sem[12];
  int rc = check(ctx, wln_wilson_avg(ctx, ens, &tube, 1, rho, rho_off, T, T_off, G,
                                     WLN_PREC_FP32_COMP, S), "wln_wilson_avg");
  if (!rc)
    rc = check(ctx, wln_jackknife(ctx, S, n_points, G, n_loops / G, WLN_C_FERM, mean, sem,
                                  NULL, NULL), "wln_jackknife");
  if (!rc) {
    for (int p = 0; p < n_points; ++p)
      printf("%d %.17g %.17g %.17g %.17g %.17g\n", p, rho[p % 4], T[p / 4], mean[p], sem[p],
             S[(size_t)p * G * WLN_K + WLN_C_SCAL]);
  }
  /* an invalid call is refused with a message and leaves the context usable */
  if (!rc && wln_wilson_avg(ctx, ens, &tube, 1, rho, rho_off, T, T_off, 3, WLN_PREC_FP32_COMP, S) !=
                 WLN_EINVAL) {
    fprintf(stderr, "expected WLN_EINVAL for 3 groups of 1024 loops\n");
    rc = 1;
  }
  free(S);
  wln_free_ensemble(ctx, ens);
  wln_destroy(ctx);
  return rc;
}
