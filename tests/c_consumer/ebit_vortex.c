/* A plain C consumer of the library's ABI (include/ebit.h): no Python, no
 * binding.  Reads a case file, runs the steps through ebit_step, and writes
 * the final volume fractions and area.
 *
 * Case file (little-endian): int32 n, int32 prec (EBIT_FP64 / EBIT_FP32),
 * int32 steps, int32 ncircles; ncircles x (xc, yc, r) doubles; steps dt
 * doubles; then u and v, (n+1)*(n+1) elements each of the precision.
 * Output file: double area, then n*n fractions of the precision.
 * Exit status 0 on success; any failure prints the library's message. */
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime.h>

#include "ebit.h"

static int fail(const char* what) {
  fprintf(stderr, "%s: %s\n", what, ebit_last_error());
  return 1;
}

static int read_all(FILE* f, void* p, size_t bytes) { return fread(p, 1, bytes, f) == bytes; }

int main(int argc, char** argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s case.bin out.bin\n", argv[0]);
    return 2;
  }
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 2;
  int32_t hdr[4];
  if (!read_all(f, hdr, sizeof hdr)) return 2;
  const int n = hdr[0], prec = hdr[1], steps = hdr[2], nc = hdr[3];
  const size_t esz = prec == EBIT_FP32 ? 4 : 8;
  const size_t nv = (size_t)(n + 1) * (n + 1);
  ebit_circle* circles = (ebit_circle*)malloc(sizeof(ebit_circle) * (nc > 0 ? nc : 1));
  double* dts = (double*)malloc(sizeof(double) * (steps > 0 ? steps : 1));
  void* hu = malloc(nv * esz);
  void* hv = malloc(nv * esz);
  void* hc = malloc((size_t)n * n * esz);
  if (!circles || !dts || !hu || !hv || !hc) return 2;
  if (!read_all(f, circles, sizeof(ebit_circle) * nc) || !read_all(f, dts, sizeof(double) * steps) ||
      !read_all(f, hu, nv * esz) || !read_all(f, hv, nv * esz))
    return 2;
  fclose(f);

  void *du = NULL, *dv = NULL, *dc = NULL;
  if (cudaMalloc(&du, nv * esz) != cudaSuccess || cudaMalloc(&dv, nv * esz) != cudaSuccess ||
      cudaMalloc(&dc, (size_t)n * n * esz) != cudaSuccess)
    return 3;
  cudaMemcpy(du, hu, nv * esz, cudaMemcpyHostToDevice);
  cudaMemcpy(dv, hv, nv * esz, cudaMemcpyHostToDevice);

  ebit_grid grid = {n, n, 1.0 / n, prec, 0};
  ebit_scene scene = {0};
  scene.circles = circles;
  scene.ncircles = nc;
  ebit_ctx* ctx = NULL;
  if (ebit_init(&ctx, &grid, &scene, NULL) != EBIT_OK) return fail("ebit_init");
  for (int k = 0; k < steps; ++k)
    if (ebit_step(ctx, du, dv, dts[k]) != EBIT_OK) return fail("ebit_step");
  double area = 0.0;
  if (ebit_fraction(ctx, dc, &area) != EBIT_OK) return fail("ebit_fraction");
  if (cudaMemcpy(hc, dc, (size_t)n * n * esz, cudaMemcpyDeviceToHost) != cudaSuccess) return 3;
  if (ebit_sync(ctx) != EBIT_OK) return fail("ebit_sync");
  ebit_destroy(ctx);

  FILE* o = fopen(argv[2], "wb");
  if (!o) return 2;
  fwrite(&area, sizeof area, 1, o);
  fwrite(hc, esz, (size_t)n * n, o);
  fclose(o);
  printf("area %.17g\n", area);
  cudaFree(du);
  cudaFree(dv);
  cudaFree(dc);
  free(circles);
  free(dts);
  free(hu);
  free(hv);
  free(hc);
  return 0;
}
