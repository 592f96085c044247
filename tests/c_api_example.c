/*
 * A plain C user of libatlasgb.so through include/atlas_gb.h only: build the
 * O<N> grid, its mesh and median dual, apply the gradient, divergence,
 * Laplacian and curl to device fields on the CUDA runtime's default stream,
 * and print one line of checks.  With no CUDA device the first operator
 * call must fail with ATLAS_ECUDA, which is what the CPU test checks.
 *
 * Checks on the device results (O<N>, nlev levels, F32):
 *   - the gradient of a constant field is exactly 0;
 *   - the divergence of the zonal flow (u, v) = (cos lat, 0) is exactly 0
 *     (its flux through every face cancels; see the oracle's pins);
 *   - sum_i V_i curl_i of random-like (u, v) vanishes to rounding.
 * Before the device part it exercises host-only calls: a regional grid with
 * its geometry check, and the geometry cache (argv[2] names the file).
 * Exit code 0 when every check passes, 2 when no device is present and the
 * library says so (ATLAS_ECUDA), 1 otherwise.
 */
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "atlas_gb.h"

#define CHECK(call)                                                                   \
  do {                                                                                \
    int rc_ = (call);                                                                 \
    if (rc_) {                                                                        \
      fprintf(stderr, "%s failed: %d (%s)\n", #call, rc_, atlas_last_error());        \
      return 1;                                                                       \
    }                                                                                 \
  } while (0)

int main(int argc, char** argv) {
  const int N = argc > 1 ? atoi(argv[1]) : 16;
  const int nlev = 4, ld = 4;
  atlas_grid_t g;
  atlas_mesh_t m;
  atlas_fvm_t f;
  CHECK(atlas_init());
  CHECK(atlas_grid_octahedral(N, &g));
  CHECK(atlas_mesh_build(g, &m));
  CHECK(atlas_fvm_build_dual(m, 6371220.0, &f));
  int64_t V;
  const double *lonlat, *vol;
  CHECK(atlas_grid_info(g, &V, NULL, NULL, &lonlat, NULL));
  CHECK(atlas_fvm_info(f, &vol, NULL, NULL, NULL));

  /* host-only calls (no device needed): a Lambert regional grid and its
   * geometry check, and the geometry cache round trip */
  {
    const double prm[8] = {-1.0e6, 1.0e6, -8.0e5, 9.0e5, 6371220.0, 5.0, 50.0, 0.0};
    atlas_grid_t rg;
    atlas_mesh_t rm;
    atlas_fvm_t rf, lf;
    atlas_grid_t lg;
    atlas_mesh_t lm;
    double worst = -1.0, R = 0.0;
    int64_t rV = 0, lV = 0;
    CHECK(atlas_grid_regional(ATLAS_PROJ_LAMBERT_CONFORMAL, 13, 9, prm, &rg));
    CHECK(atlas_mesh_build(rg, &rm));
    CHECK(atlas_fvm_build_dual(rm, 6371220.0, &rf));
    CHECK(atlas_fvm_check(rf, &worst));
    CHECK(atlas_grid_info(rg, &rV, NULL, NULL, NULL, NULL));
    const char* path = argc > 2 ? argv[2] : "c_api_example.geom";
    CHECK(atlas_fvm_save(rf, path));
    CHECK(atlas_fvm_load(path, &lg, &lm, &lf));
    CHECK(atlas_grid_info(lg, &lV, NULL, NULL, NULL, NULL));
    CHECK(atlas_fvm_radius(lf, &R));
    printf("regional 13 x 9: %lld nodes, closure %.1e; reloaded %lld nodes, R %.0f\n", (long long)rV, worst,
           (long long)lV, R);
    if (lV != rV || R != 6371220.0 || !(worst <= 1e-14)) return 1;
    atlas_fvm_destroy(lf);
    atlas_mesh_destroy(lm);
    atlas_grid_destroy(lg);
    atlas_fvm_destroy(rf);
    atlas_mesh_destroy(rm);
    atlas_grid_destroy(rg);
    remove(path);
  }

  const size_t bytes = (size_t)V * ld * sizeof(float);
  float* h = (float*)malloc(3 * bytes);
  float *hu = h, *hv = h + (size_t)V * ld, *hc = h + 2 * (size_t)V * ld;
  for (int64_t i = 0; i < V; ++i)
    for (int k = 0; k < ld; ++k) {
      hu[i * ld + k] = (float)cos(lonlat[2 * i + 1]);
      hv[i * ld + k] = 0.0f;
      hc[i * ld + k] = 2.5f;
    }
  float *du = NULL, *dv = NULL, *dc = NULL, *o0 = NULL, *o1 = NULL;
  if (cudaMalloc((void**)&du, bytes) != cudaSuccess || cudaMalloc((void**)&dv, bytes) != cudaSuccess ||
      cudaMalloc((void**)&dc, bytes) != cudaSuccess || cudaMalloc((void**)&o0, bytes) != cudaSuccess ||
      cudaMalloc((void**)&o1, bytes) != cudaSuccess) {
    /* no device: the library must refuse the operator call, not compute */
    int rc = atlas_nabla_gradient(f, hc, hu, hv, nlev, ld, ATLAS_F32, NULL);
    printf("no CUDA device: atlas_nabla_gradient returned %d (%s)\n", rc, atlas_last_error());
    return rc == ATLAS_ECUDA ? 2 : 1;
  }
  CHECK(atlas_field_sync(du, hu, bytes, 0, NULL));
  CHECK(atlas_field_sync(dv, hv, bytes, 0, NULL));
  CHECK(atlas_field_sync(dc, hc, bytes, 0, NULL));

  int ok = 1;
  float* r = (float*)malloc(2 * bytes);
  /* gradient of a constant: exactly zero */
  CHECK(atlas_nabla_gradient(f, dc, o0, o1, nlev, ld, ATLAS_F32, NULL));
  CHECK(atlas_field_sync(r, o0, bytes, 1, NULL));
  CHECK(atlas_field_sync(r + (size_t)V * ld, o1, bytes, 1, NULL));
  cudaDeviceSynchronize();
  for (int64_t q = 0; q < 2 * V * ld; ++q)
    if (r[q] != 0.0f) ok = 0;
  int grad_ok = ok;
  /* divergence of the zonal flow: zero to rounding */
  CHECK(atlas_nabla_divergence(f, du, dv, o0, nlev, ld, ATLAS_F32, NULL));
  CHECK(atlas_field_sync(r, o0, bytes, 1, NULL));
  cudaDeviceSynchronize();
  double dmax = 0;
  for (int64_t q = 0; q < V * ld; ++q) dmax = fmax(dmax, fabs((double)r[q]));
  int div_ok = dmax * 6371220.0 <= 1e-5;
  /* total circulation of (u, v) = (sin(3 lon) cos lat, cos(2 lon)): zero */
  for (int64_t i = 0; i < V; ++i)
    for (int k = 0; k < ld; ++k) {
      hu[i * ld + k] = (float)(sin(3 * lonlat[2 * i]) * cos(lonlat[2 * i + 1]));
      hv[i * ld + k] = (float)cos(2 * lonlat[2 * i]);
    }
  CHECK(atlas_field_sync(du, hu, bytes, 0, NULL));
  CHECK(atlas_field_sync(dv, hv, bytes, 0, NULL));
  CHECK(atlas_nabla_curl(f, du, dv, o0, nlev, ld, ATLAS_F32, NULL));
  CHECK(atlas_nabla_laplacian(f, du, o1, nlev, ld, ATLAS_F32, NULL));
  CHECK(atlas_field_sync(r, o0, bytes, 1, NULL));
  cudaDeviceSynchronize();
  double s = 0, a = 0;
  for (int64_t i = 0; i < V; ++i) {
    s += vol[i] * r[i * ld];
    a += fabs(vol[i] * r[i * ld]);
  }
  int curl_ok = fabs(s) <= 1e-5 * a;
  ok = grad_ok && div_ok && curl_ok;
  printf("O%d: nodes %lld, gradient of constant %s, zonal divergence max %.3e/R, total circulation %.3e of %.3e: %s\n",
         N, (long long)V, grad_ok ? "exactly 0" : "NOT 0", dmax * 6371220.0, s, a, ok ? "ok" : "FAILED");
  cudaFree(du); cudaFree(dv); cudaFree(dc); cudaFree(o0); cudaFree(o1);
  free(h); free(r);
  atlas_fvm_destroy(f);
  atlas_mesh_destroy(m);
  atlas_grid_destroy(g);
  CHECK(atlas_finalize());
  return ok ? 0 : 1;
}
