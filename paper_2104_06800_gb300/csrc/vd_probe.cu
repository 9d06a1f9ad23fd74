// Throughput probes of the two pipes that bound the depth sampling and the
// pose scoring: the FP32 fused multiply-add pipe and the MUFU (transcendental)
// unit.  Timed by the caller with CUDA events around a launch, they measure
// the denominators of the roofline fractions on the running GPU; they
// compute nothing of the method.
#include "vd_internal.h"

#define VD_PROBE_CHAINS 8
#define VD_PROBE_UNROLL 16

// Written only when a chain's sum equals -1, which positive chains never
// reach: it keeps the compiler from removing the chains.
static __device__ float g_probe_sink;

// Eight independent FMA chains per thread, VD_PROBE_UNROLL x iters steps
// each: iters * 128 FFMA per thread.
__global__ void __launch_bounds__(256) k_probe_ffma(int iters) {
  float a[VD_PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < VD_PROBE_CHAINS; ++k) a[k] = 1e-3f * (float)(threadIdx.x + k);
  const float m = 0.9999f, c = 1e-4f;
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < VD_PROBE_UNROLL; ++r)
#pragma unroll
      for (int k = 0; k < VD_PROBE_CHAINS; ++k) a[k] = fmaf(a[k], m, c);
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < VD_PROBE_CHAINS; ++k) s += a[k];
  if (s == -1.0f) g_probe_sink = s;
}

// Eight independent MUFU log2 chains per thread (each step one MUFU.LG2 and
// one FP32 add): iters * 128 MUFU operations per thread.
__global__ void __launch_bounds__(256) k_probe_mufu(int iters) {
  float a[VD_PROBE_CHAINS];
#pragma unroll
  for (int k = 0; k < VD_PROBE_CHAINS; ++k) a[k] = 2.0f + 1e-3f * (float)(threadIdx.x + k);
  for (int i = 0; i < iters; ++i) {
#pragma unroll
    for (int r = 0; r < VD_PROBE_UNROLL; ++r)
#pragma unroll
      for (int k = 0; k < VD_PROBE_CHAINS; ++k) a[k] = __log2f(a[k]) + 1.5f;
  }
  float s = 0.0f;
#pragma unroll
  for (int k = 0; k < VD_PROBE_CHAINS; ++k) s += a[k];
  if (s == -1.0f) g_probe_sink = s;
}

extern "C" vd_status vd_probe_pipe(int kind, int blocks, int iters, double* ops_out,
                                   void* cuda_stream) {
  if ((kind != VD_PROBE_FP32 && kind != VD_PROBE_MUFU) || blocks < 1 || blocks > (1 << 20) ||
      iters < 1 || iters > (1 << 20) || !ops_out)
    return VD_ERR_ARG;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (kind == VD_PROBE_FP32) k_probe_ffma<<<blocks, 256, 0, s>>>(iters);
  else k_probe_mufu<<<blocks, 256, 0, s>>>(iters);
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) {
    vd_set_error(cudaGetErrorString(e));
    return VD_ERR_CUDA;
  }
  *ops_out = (double)blocks * 256.0 * (double)iters * VD_PROBE_CHAINS * VD_PROBE_UNROLL;
  return VD_OK;
}
