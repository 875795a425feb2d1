/*
 * A plain C caller of libvndf: device buffers from the CUDA runtime, inputs
 * built on the host, vndf_sample with in-kernel Philox uniforms and its fused
 * density, vndf_pdf at the sampled normals, then everything written to a
 * binary file that the Python test compares with the FP64 oracle.  It also
 * exercises the documented argument errors from C.  Usage:
 *   vndf_c_caller <n> <output file>
 * Output: n, then wi_x, wi_y, wi_z, alpha_x, alpha_y, wm_x, wm_y, wm_z, pdf,
 * pdf_at_normals as n little-endian float32 each.  Exit status 0 on success.
 */
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "vndf.h"

#define CHECK_CUDA(x)                                                    \
  do {                                                                   \
    cudaError_t e_ = (x);                                                \
    if (e_ != cudaSuccess) {                                             \
      fprintf(stderr, "%s: %s\n", #x, cudaGetErrorString(e_));           \
      return 2;                                                          \
    }                                                                    \
  } while (0)

#define CHECK_VNDF(x)                                                    \
  do {                                                                   \
    int s_ = (x);                                                        \
    if (s_ != VNDF_OK) {                                                 \
      fprintf(stderr, "%s: %s (%d)\n", #x, vndf_status_string(s_), s_); \
      return 3;                                                          \
    }                                                                    \
  } while (0)

enum { IN_WX, IN_WY, IN_WZ, IN_AX, IN_AY, OUT_MX, OUT_MY, OUT_MZ, OUT_PDF, OUT_PDF2, N_ARRAYS };

int main(int argc, char **argv) {
  if (argc != 3) {
    fprintf(stderr, "usage: %s <n> <output file>\n", argv[0]);
    return 1;
  }
  const int64_t n = atoll(argv[1]);
  if (n <= 0) return 1;
  float *host[N_ARRAYS], *dev[N_ARRAYS];
  for (int k = 0; k < N_ARRAYS; ++k) {
    host[k] = (float *)malloc((size_t)n * sizeof(float));
    if (!host[k]) return 4;
    CHECK_CUDA(cudaMalloc((void **)&dev[k], (size_t)n * sizeof(float)));
  }
  /* incident directions over the upper hemisphere and roughness over [1e-3, 1] on a low-discrepancy lattice */
  for (int64_t i = 0; i < n; ++i) {
    const double a = fmod(0.6180339887498949 * (double)i, 1.0), b = fmod(0.7548776662466927 * (double)i, 1.0);
    const double ct = 1e-4 + (1.0 - 1e-4) * a, st = sqrt(1.0 - ct * ct), phi = 2.0 * 3.141592653589793 * b;
    host[IN_WX][i] = (float)(st * cos(phi));
    host[IN_WY][i] = (float)(st * sin(phi));
    host[IN_WZ][i] = (float)ct;
    host[IN_AX][i] = (float)pow(1e-3, fmod(0.5698402909980532 * (double)i, 1.0));
    host[IN_AY][i] = (float)pow(1e-3, fmod(0.8191725133961645 * (double)i, 1.0));
  }
  for (int k = IN_WX; k <= IN_AY; ++k)
    CHECK_CUDA(cudaMemcpy(dev[k], host[k], (size_t)n * sizeof(float), cudaMemcpyHostToDevice));

  /* documented host-side argument errors, returned before any work is enqueued */
  if (vndf_sample(-1, dev[IN_WX], dev[IN_WY], dev[IN_WZ], dev[IN_AX], dev[IN_AY], NULL, NULL, 0, 0, 0,
                  VNDF_METHOD_SPHERICAL_CAP, dev[OUT_MX], dev[OUT_MY], dev[OUT_MZ], NULL, NULL) != VNDF_ERR_SIZE ||
      vndf_sample(n, dev[IN_WX], dev[IN_WY], dev[IN_WZ], dev[IN_AX], dev[IN_AY], NULL, NULL, 0, 0, 0, 9,
                  dev[OUT_MX], dev[OUT_MY], dev[OUT_MZ], NULL, NULL) != VNDF_ERR_METHOD ||
      vndf_sample(n, dev[IN_WX], dev[IN_WY], dev[IN_WZ], dev[IN_AX], dev[IN_AY], NULL, NULL, 0, 0, 0,
                  VNDF_METHOD_SPHERICAL_CAP, dev[IN_WX], dev[OUT_MY], dev[OUT_MZ], NULL, NULL) != VNDF_ERR_ARG) {
    fprintf(stderr, "argument errors not reported as documented\n");
    return 5;
  }

  cudaStream_t s;
  CHECK_CUDA(cudaStreamCreate(&s));
  CHECK_VNDF(vndf_sample(n, dev[IN_WX], dev[IN_WY], dev[IN_WZ], dev[IN_AX], dev[IN_AY], NULL, NULL, 7, 3, 1,
                         VNDF_METHOD_SPHERICAL_CAP, dev[OUT_MX], dev[OUT_MY], dev[OUT_MZ], dev[OUT_PDF], s));
  CHECK_VNDF(vndf_pdf(n, dev[IN_WX], dev[IN_WY], dev[IN_WZ], dev[IN_AX], dev[IN_AY], dev[OUT_MX], dev[OUT_MY],
                      dev[OUT_MZ], dev[OUT_PDF2], s));
  CHECK_CUDA(cudaStreamSynchronize(s));
  for (int k = OUT_MX; k <= OUT_PDF2; ++k)
    CHECK_CUDA(cudaMemcpy(host[k], dev[k], (size_t)n * sizeof(float), cudaMemcpyDeviceToHost));

  FILE *f = fopen(argv[2], "wb");
  if (!f) return 6;
  fwrite(&n, sizeof(n), 1, f);
  for (int k = 0; k < N_ARRAYS; ++k) fwrite(host[k], sizeof(float), (size_t)n, f);
  fclose(f);
  for (int k = 0; k < N_ARRAYS; ++k) {
    free(host[k]);
    cudaFree(dev[k]);
  }
  cudaStreamDestroy(s);
  printf("vndf_c_caller: %lld samples, abi %d\n", (long long)n, vndf_abi_version());
  return 0;
}
