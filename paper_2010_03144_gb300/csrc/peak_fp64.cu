// FP64 instruction-rate measurement (a measurement helper beside the compressor, built into its
// own libsdcsz_peak.so; not part of the compressor's C ABI).
//
// The float64 compressor evaluates every prediction, reconstruction and check with separately
// rounded IEEE additions and multiplications (no contraction), so the rate that bounds it is
// that of DADD / DMUL instructions, not the FMA-based FLOP/s figure vendors quote. Each thread
// runs kChains independent dependency chains x <- x * m + c, written as one multiplication and
// one addition, so the FP64 pipe is kept busy without waiting on a chain's latency. The FMA
// variant (one fused operation per step) gives the nominal FLOP/s figure for comparison.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kChains = 8;

template <bool FUSED>
__global__ void __launch_bounds__(256) k_fp64_rate(double* out, int iters, double m, double c) {
  double x[kChains];
#pragma unroll
  for (int q = 0; q < kChains; ++q) x[q] = 1.0 + 1e-3 * (threadIdx.x + q);
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int q = 0; q < kChains; ++q) {
      if (FUSED) x[q] = __fma_rn(x[q], m, c);
      else x[q] = __dadd_rn(__dmul_rn(x[q], m), c);
    }
  }
  double s = 0.0;
#pragma unroll
  for (int q = 0; q < kChains; ++q) s = __dadd_rn(s, x[q]);
  out[blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace

// Runs the separate (fused = 0) or fused (fused = 1) variant on `stream` with `blocks` CTAs of
// 256 threads and `iters` steps per chain; out needs blocks * 256 doubles of device memory.
// Writes the kernel's CUDA-event time in ms and the number of FP64 instructions it executed.
// Returns 0, or -1 on a CUDA error.
extern "C" int sdcsz_peak_fp64(double* out, int blocks, int iters, int fused, void* stream, float* ms,
                               unsigned long long* fp64_instructions) {
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return -1;
  const double m = 0.9999999, c = 1e-7;
  cudaEventRecord(e0, s);
  if (fused) k_fp64_rate<true><<<blocks, 256, 0, s>>>(out, iters, m, c);
  else k_fp64_rate<false><<<blocks, 256, 0, s>>>(out, iters, m, c);
  cudaEventRecord(e1, s);
  int rc = 0;
  if (cudaEventSynchronize(e1) != cudaSuccess || cudaGetLastError() != cudaSuccess) rc = -1;
  float t = 0.0f;
  if (!rc) cudaEventElapsedTime(&t, e0, e1);
  *ms = t;
  *fp64_instructions = (unsigned long long)blocks * 256ull * (unsigned long long)iters * kChains * (fused ? 1ull : 2ull);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return rc;
}
