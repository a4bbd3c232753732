// dg_peak.cu -- arithmetic throughput probes that give the roofline denominators of the cost model
// (Sec. 3.6: the kernels are bound by the floating-point issue rate of the FP64, or FP32, pipes).
//
// Each probe keeps every warp of a full-occupancy grid busy with independent chains of one instruction:
//   DFMA  fma.rn.f64, eight independent chains per thread                 2 flops per lane and instruction
//   DMMA  mma.sync.aligned.m8n8k4 with f64 operands, four accumulators per warp   512 flops per warp and
//         instruction (an 8x8x4 product)
//   FFMA  fma.rn.f32, eight independent chains per thread                 2 flops per lane and instruction
// and writes its result only if it equals a value it cannot reach, so nothing is removed as dead code and
// no memory traffic is added.  The caller times the launch with events on the same stream.
#include <cstdint>

#include "dg_internal.h"

namespace {

constexpr int PROBE_THREADS = 256;
constexpr int PROBE_BLOCKS_PER_SM = 8;  // 2048 threads per SM: every warp slot filled
constexpr int CHAINS = 8;

__global__ void __launch_bounds__(PROBE_THREADS) probe_dfma(int64_t iters, double x, double y, double* sink) {
  double a[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) a[c] = (double)(threadIdx.x + c) * 1e-3;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = fma(a[c], x, y);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += a[c];
  if (s == -1.2345e300) sink[0] = s;
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_ffma(int64_t iters, float x, float y, double* sink) {
  float a[CHAINS];
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) a[c] = (float)(threadIdx.x + c) * 1e-3f;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < CHAINS; ++c) a[c] = fmaf(a[c], x, y);
  }
  float s = 0.f;
#pragma unroll
  for (int c = 0; c < CHAINS; ++c) s += a[c];
  if (s == -1.2345e30f) sink[0] = s;
}

constexpr int MMA_ACC = 4;

__device__ __forceinline__ void dmma_884(double (&d)[2], double a, double b) {
  asm volatile("mma.sync.aligned.m8n8k4.row.col.f64.f64.f64.f64 {%0,%1}, {%2}, {%3}, {%0,%1};\n"
               : "+d"(d[0]), "+d"(d[1])
               : "d"(a), "d"(b));
}

__global__ void __launch_bounds__(PROBE_THREADS) probe_dmma(int64_t iters, double x, double y, double* sink) {
  double acc[MMA_ACC][2];
#pragma unroll
  for (int c = 0; c < MMA_ACC; ++c) acc[c][0] = acc[c][1] = (double)(threadIdx.x + c) * 1e-3;
  const double a = x + (threadIdx.x & 31) * 1e-6, b = y - (threadIdx.x & 31) * 1e-6;
  for (int64_t i = 0; i < iters; ++i) {
#pragma unroll
    for (int c = 0; c < MMA_ACC; ++c) dmma_884(acc[c], a, b);
  }
  double s = 0.0;
#pragma unroll
  for (int c = 0; c < MMA_ACC; ++c) s += acc[c][0] + acc[c][1];
  if (s == -1.2345e300) sink[0] = s;
}

}  // namespace

extern "C" int dg_peak_probe(int32_t kind, int64_t iterations, double* sink_dev, double* flops, void* stream) {
  using namespace dgi;
  if (!sink_dev || !flops || iterations < 1 || kind < DG_PROBE_DFMA || kind > DG_PROBE_FFMA) {
    set_error("dg_peak_probe: bad kind, iterations < 1 or null pointer");
    return DG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int blocks = sm_count() * PROBE_BLOCKS_PER_SM;
  const double threads = (double)blocks * PROBE_THREADS;
  switch (kind) {
    case DG_PROBE_DFMA:
      probe_dfma<<<blocks, PROBE_THREADS, 0, s>>>(iterations, 0.999999, 1e-7, sink_dev);
      *flops = threads * (double)iterations * CHAINS * 2.0;
      break;
    case DG_PROBE_DMMA:
      probe_dmma<<<blocks, PROBE_THREADS, 0, s>>>(iterations, 0.999999, 1e-7, sink_dev);
      *flops = threads / 32.0 * (double)iterations * MMA_ACC * 512.0;
      break;
    default:
      probe_ffma<<<blocks, PROBE_THREADS, 0, s>>>(iterations, 0.999999f, 1e-7f, sink_dev);
      *flops = threads * (double)iterations * CHAINS * 2.0;
      break;
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : cuda_fail(e, "dg_peak_probe launch");
}
