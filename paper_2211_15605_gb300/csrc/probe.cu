// Measurement aid of the benchmark: the FP64 fused multiply-add rate of this GPU, the
// denominator of the FP64 form's roofline (the FP64 step is bound by FP64 arithmetic, not by
// HBM). Not part of the coupling-step library; built as its own small shared library.
#include <cuda_runtime.h>

namespace {

// Each thread runs 8 independent chains of `iters` FMAs (a = a * b + c) so that the FP64
// pipe, not the dependency latency, sets the rate; the sum is stored so nothing is removed.
__global__ void k_dfma(int iters, double b, double c, double* out) {
  double a[8];
#pragma unroll
  for (int k = 0; k < 8; ++k) a[k] = threadIdx.x * 1e-9 + k;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = fma(a[k], b, c);
  }
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 8; ++k) s += a[k];
  if (s == 12345.678) out[0] = s;            // never true for these inputs; keeps the chains
}

}  // namespace

extern "C" {

// Launches the probe on `stream` (a cudaStream_t; NULL = legacy default stream): blocks_per_sm
// blocks of 256 threads per SM, each thread 8 x iters FMAs. *flops receives the FP64
// operations of the launch (2 per FMA). Returns 0, or the CUDA error code of the launch.
int mppic_probe_dfma(int iters, int blocks_per_sm, void* stream, double* out, double* flops) {
  int dev = 0, nsm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int blocks = nsm * blocks_per_sm;
  k_dfma<<<blocks, 256, 0, static_cast<cudaStream_t>(stream)>>>(iters, 0.999999999, 1e-9, out);
  if (flops) *flops = 2.0 * 8.0 * (double)iters * (double)blocks * 256.0;
  return (int)cudaGetLastError();
}

}  // extern "C"
