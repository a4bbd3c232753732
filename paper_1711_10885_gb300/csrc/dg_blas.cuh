// dg_blas.cuh -- vector kernels of the Krylov solvers (deterministic fixed-order reductions).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dgb {

constexpr int RED_BLOCKS = 152 * 4;  // one wave of 4 CTAs per SM
constexpr int RED_THREADS = 256;
constexpr int MDOT_GROUP = 8;         // vectors reduced per pass over w

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// part[v * gridDim.x + block] = sum over this block's share of i of V[v*ld + i] * w[i]  (v < nv)
// Per-thread sums run in T; the block and final reductions in FP64.
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
mdot_partial(const T* __restrict__ V, size_t ld, int nv, const T* __restrict__ w, size_t n, double* __restrict__ part) {
  __shared__ double red[MDOT_GROUP][RED_THREADS / 32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (int v0 = 0; v0 < nv; v0 += MDOT_GROUP) {
    T acc[MDOT_GROUP];
#pragma unroll
    for (int q = 0; q < MDOT_GROUP; ++q) acc[q] = T(0);
    for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
      const T wi = w[i];
#pragma unroll
      for (int q = 0; q < MDOT_GROUP; ++q)
        if (v0 + q < nv) acc[q] = fma(V[(size_t)(v0 + q) * ld + i], wi, acc[q]);
    }
#pragma unroll
    for (int q = 0; q < MDOT_GROUP; ++q) {
      const double s = warp_sum((double)acc[q]);
      if (lane == 0) red[q][wid] = s;
    }
    __syncthreads();
    if (threadIdx.x < MDOT_GROUP && v0 + (int)threadIdx.x < nv) {
      double s = 0.0;
      for (int k = 0; k < RED_THREADS / 32; ++k) s += red[threadIdx.x][k];
      part[(size_t)(v0 + threadIdx.x) * gridDim.x + blockIdx.x] = s;
    }
    __syncthreads();
  }
}

// h[v] = sum_b part[v * nblk + b]; one CTA per v
__global__ void mdot_final(const double* __restrict__ part, int nblk, double* __restrict__ h) {
  __shared__ double red[RED_THREADS / 32];
  double s = 0.0;
  for (int b = threadIdx.x; b < nblk; b += blockDim.x) s += part[(size_t)blockIdx.x * nblk + b];
  s = warp_sum(s);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[k];
    h[blockIdx.x] = t;
  }
}

// w[i] -= sum_v V[v*ld + i] * h[v]   (nv <= 64)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
maxpy(const T* __restrict__ V, size_t ld, int nv, const double* __restrict__ h, T* __restrict__ w, size_t n) {
  __shared__ T hs[64];
  if (threadIdx.x < nv) hs[threadIdx.x] = (T)h[threadIdx.x];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    T acc = w[i];
    for (int v = 0; v < nv; ++v) acc = fma(-hs[v], V[(size_t)v * ld + i], acc);
    w[i] = acc;
  }
}

// x[i] += sum_v Z[v*ld + i] * y[v]  with x in FP64 (solution update of FGMRES), Z in T, y on the device
template <typename T, typename TX>
__global__ void __launch_bounds__(RED_THREADS)
lincomb_add(const T* __restrict__ Z, size_t ld, int nv, const double* __restrict__ y, TX* __restrict__ x, size_t n) {
  __shared__ double ys[64];
  if (threadIdx.x < nv) ys[threadIdx.x] = y[threadIdx.x];
  __syncthreads();
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    T acc = T(0);
    for (int v = 0; v < nv; ++v) acc = fma((T)ys[v], Z[(size_t)v * ld + i], acc);
    x[i] = (TX)((TX)acc + x[i]);
  }
}

// out[i] = alpha * in[i] (with a precision change)
template <typename TI, typename TO>
__global__ void __launch_bounds__(RED_THREADS)
scale_copy(const TI* __restrict__ in, TO* __restrict__ out, double alpha, size_t n) {
  const TI a = (TI)alpha;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (TO)(a * in[i]);
}

// out[i] = a[i] - b[i]
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
sub(const T* __restrict__ a, const T* __restrict__ b, T* __restrict__ out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

// counts non-finite entries (NaN/Inf) into *bad (one atomic per block that saw one)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS) count_nonfinite(const T* __restrict__ a, size_t n, int* bad) {
  int local = 0;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    local |= !isfinite((double)a[i]);
  if (__syncthreads_or(local) && threadIdx.x == 0) atomicAdd(bad, 1);
}

}  // namespace dgb
