/*
 * part_client.c -- a plain C user of libpart.so: no Python, no torch.
 *
 *   part_client host          host-only calls (brick layout, workspace size,
 *                             argument errors); needs no GPU
 *   part_client step N SEED   one FP64 Boris + TSC + deposit step on a 16^3
 *                             periodic grid in a uniform field, with device
 *                             memory from cudaMalloc; prints the initial and
 *                             final state and the deposit as text, for a test
 *                             to compare with the oracle
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_runtime_api.h>

#include "part.h"

#define CHECK(call)                                                              \
  do {                                                                           \
    part_status s_ = (call);                                                     \
    if (s_ != PART_OK) {                                                         \
      fprintf(stderr, "%s -> %d: %s\n", #call, (int)s_, part_last_error(NULL));   \
      return 1;                                                                  \
    }                                                                            \
  } while (0)

#define CUDA(call)                                                               \
  do {                                                                           \
    cudaError_t e_ = (call);                                                     \
    if (e_ != cudaSuccess) {                                                     \
      fprintf(stderr, "%s -> %s\n", #call, cudaGetErrorString(e_));              \
      return 1;                                                                  \
    }                                                                            \
  } while (0)

static part_grid grid_of(int n) {
  part_grid g;
  memset(&g, 0, sizeof(g));
  g.dim = 3;
  for (int a = 0; a < 3; ++a) {
    g.n[a] = n;
    g.xmin[a] = -1.0;
    g.dx[a] = 2.0 / n;
    g.periodic[a] = 1;
  }
  return g;
}

static int host_checks(void) {
  part_grid g = grid_of(128);
  int b[3];
  int64_t nkeys = 0;
  size_t bytes = 0;
  CHECK(part_brick_dims(&g, b, &nkeys));
  printf("brick %d %d %d nkeys %lld\n", b[0], b[1], b[2], (long long)nkeys);
  CHECK(part_workspace_size(&g, PART_FP64, PART_BORIS, 1 << 20, 0, &bytes));
  printf("workspace %zu\n", bytes);
  g.dim = 4;
  part_status s = part_workspace_size(&g, PART_FP64, PART_BORIS, 10, 0, &bytes);
  printf("bad_dim %d %s\n", (int)s, part_last_error(NULL));
  return 0;
}

static int one_step(int64_t N, unsigned long long seed) {
  const int n = 16;
  const int64_t G = (int64_t)n * n * n;
  part_grid g = grid_of(n);
  size_t wsb = 0;
  CHECK(part_workspace_size(&g, PART_FP64, PART_BORIS, N, 0, &wsb));
  void *ws = NULL, *f = NULL, *x = NULL, *u = NULL, *out = NULL;
  CUDA(cudaMalloc(&ws, wsb));
  CUDA(cudaMalloc(&f, sizeof(double) * 6 * G));
  CUDA(cudaMalloc(&x, sizeof(double) * 3 * N));
  CUDA(cudaMalloc(&u, sizeof(double) * 3 * N));
  CUDA(cudaMalloc(&out, sizeof(double) * 3 * G));
  /* E = (0.01, 0, 0), B = (0, 0, 1) everywhere */
  double* fh = (double*)calloc((size_t)(6 * G), sizeof(double));
  for (int64_t c = 0; c < G; ++c) {
    fh[0 * G + c] = 0.01;
    fh[5 * G + c] = 1.0;
  }
  CUDA(cudaMemcpy(f, fh, sizeof(double) * 6 * G, cudaMemcpyHostToDevice));
  part_ctx* ctx = NULL;
  CHECK(part_init(&ctx, &g, PART_FP64, PART_TSC, PART_BORIS, N, 0, ws, wsb, NULL));
  CHECK(part_set_fields(ctx, f, 6, PART_FP64));
  CHECK(part_bind_particles(ctx, N, x, NULL, u, NULL, NULL, NULL, NULL, NULL));
  CHECK(part_init_particles(ctx, seed, 0.1, 0.0, 0.0, 0.0, 0.0));
  CHECK(part_sync(ctx));
  double* xh = (double*)malloc(sizeof(double) * 3 * N);
  double* uh = (double*)malloc(sizeof(double) * 3 * N);
  double* oh = (double*)malloc(sizeof(double) * 3 * G);
  CUDA(cudaMemcpy(xh, x, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(uh, u, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < 3 * N; ++i) printf("x0 %.17g\n", xh[i]);
  for (int64_t i = 0; i < 3 * N; ++i) printf("u0 %.17g\n", uh[i]);
  CHECK(part_enable_deposit(ctx, 1));
  CHECK(part_sort(ctx));
  CHECK(part_gather_push(ctx, 1.0, 0.05, 1));
  CHECK(part_deposit(ctx, (double*)out));
  CHECK(part_sync(ctx));
  CUDA(cudaMemcpy(xh, x, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(uh, u, sizeof(double) * 3 * N, cudaMemcpyDeviceToHost));
  CUDA(cudaMemcpy(oh, out, sizeof(double) * 3 * G, cudaMemcpyDeviceToHost));
  for (int64_t i = 0; i < 3 * N; ++i) printf("x1 %.17g\n", xh[i]);
  for (int64_t i = 0; i < 3 * N; ++i) printf("u1 %.17g\n", uh[i]);
  for (int64_t i = 0; i < 3 * G; ++i) printf("dep %.17g\n", oh[i]);
  printf("launches %lld\n", (long long)part_launch_count(ctx));
  CHECK(part_destroy(ctx));
  cudaFree(ws);
  cudaFree(f);
  cudaFree(x);
  cudaFree(u);
  cudaFree(out);
  free(fh);
  free(xh);
  free(uh);
  free(oh);
  return 0;
}

int main(int argc, char** argv) {
  if (argc >= 2 && strcmp(argv[1], "host") == 0) return host_checks();
  if (argc >= 4 && strcmp(argv[1], "step") == 0)
    return one_step(atoll(argv[2]), strtoull(argv[3], NULL, 10));
  fprintf(stderr, "usage: part_client host | part_client step N SEED\n");
  return 2;
}
