// probe.cu -- part_probe_fp64_fma: the device's FP64 fused multiply-add rate,
// measured, as the denominator of the FP64 kernels' arithmetic roofline.
//
// B300 has no published FP64 figure that matches its shipped clocks, and its
// FP64 (non-tensor) rate is so far below its FP32 rate that every FP64 kernel
// of this library that does real arithmetic per byte is bound by it, not by
// HBM.  The probe runs independent DFMA chains on every SM and times them with
// CUDA events on the caller's stream:
//   - grid: ctas_per_sm CTAs of 256 threads on every SM (the device's SM
//     count is queried), each thread kChains independent chains of `iters`
//     dependent fma(a, m, c) steps, so the FP64 pipe always has work ready;
//   - the chains' values stay bounded (m < 1, c > 0) and finite, and one
//     store to sink[0] that only happens if a value turned negative (never)
//     keeps the compiler from removing them;
//   - rate = 2 flop x threads x kChains x iters / (best of `reps` launches).
// Nothing is allocated: the caller passes an 8-byte device sink.
#include "part_internal.cuh"

namespace {

constexpr int kChains = 16;
constexpr int kProbeThreads = 256;

__global__ void __launch_bounds__(kProbeThreads)
    k_probe_dfma(double* __restrict__ sink, int iters, double m, double c) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; ++k) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < kChains; ++k) a[k] = fma(a[k], m, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; ++k) s += a[k];
  if (s < 0.0) sink[0] = s;  // never taken: the chains stay positive
}

}  // namespace

extern "C" part_status part_probe_fp64_fma(void* cuda_stream, double* sink, int ctas_per_sm,
                                           int iters, int reps, double* tflops,
                                           double* best_ms) {
  if (!sink || !tflops || ctas_per_sm < 1 || ctas_per_sm > 8 || iters < 1 ||
      iters > (1 << 20) || reps < 1 || reps > 100)
    return fail(nullptr, PART_EINVAL,
                "part_probe_fp64_fma: sink and tflops must be non-NULL, 1 <= ctas_per_sm <= 8, "
                "1 <= iters <= 2^20, 1 <= reps <= 100");
  if (reinterpret_cast<uintptr_t>(sink) % 8 != 0)
    return fail(nullptr, PART_EINVAL, "part_probe_fp64_fma: sink is not 8-byte aligned");
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1)
    return fail(nullptr, PART_ECUDA, "part_probe_fp64_fma: device query failed");
  if (!device_accessible(dev, sink))
    return fail(nullptr, PART_EINVAL, "part_probe_fp64_fma: sink is not device memory");
  cudaStream_t st = (cudaStream_t)cuda_stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaError_t e = cudaEventCreate(&e0);
  if (e == cudaSuccess) e = cudaEventCreate(&e1);
  const int grid = sms * ctas_per_sm;
  float best = 0.0f;
  // one untimed launch first (clocks up, module loaded), then `reps` timed ones
  for (int r = 0; r <= reps && e == cudaSuccess; ++r) {
    e = cudaEventRecord(e0, st);
    if (e == cudaSuccess) {
      k_probe_dfma<<<grid, kProbeThreads, 0, st>>>(sink, iters, 0.9999999, 1e-7);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaEventRecord(e1, st);
    if (e == cudaSuccess) e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess && r > 0 && (best == 0.0f || ms < best)) best = ms;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (e != cudaSuccess)
    return fail(nullptr, PART_ECUDA, std::string("part_probe_fp64_fma: ") + cudaGetErrorString(e));
  const double flop = 2.0 * grid * kProbeThreads * (double)kChains * iters;
  *tflops = flop / (best * 1e-3) / 1e12;
  if (best_ms) *best_ms = best;
  return PART_OK;
}
