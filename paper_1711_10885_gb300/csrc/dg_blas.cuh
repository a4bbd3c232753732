// dg_blas.cuh -- vector kernels of the Krylov solvers (deterministic fixed-order reductions).  The basis
// passes are bound by HBM bandwidth: they move 16 bytes per load and keep several rows in flight.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dgb {

constexpr int RED_BLOCKS = 152 * 4;   // rows of the partial-sum buffer hold up to this many block sums
constexpr int RED_THREADS = 256;
constexpr int PASS_MINB = 3;           // resident CTAs per SM of the basis passes (their launch bounds)
constexpr int PASS_BLOCKS = 152 * PASS_MINB;  // their grid: one wave
constexpr int PASS_LOADS = 8;          // rows loaded together by the dot and update passes (80 registers or fewer)
constexpr int FUSED_LOADS = 6;         // the same for the fused update-and-dots pass (no spills at 3 CTAs per SM)
constexpr int MAX_ROWS = 64;          // basis rows per pass (restart lengths up to 60, plus w . w)

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// W consecutive elements moved by one load or store (16 bytes when W = 16 / sizeof(T))
template <typename T, int W>
struct alignas(sizeof(T) * W) Pack {
  T v[W];
};

template <typename T, int W>
__device__ __forceinline__ Pack<T, W> ld_pack(const T* row, size_t p) {
  return reinterpret_cast<const Pack<T, W>*>(row)[p];
}

// The basis passes below read the rows V_q = V + q * ld (q < nv <= 60) in packs of W elements: thread t of
// block b takes packs p = b * RED_THREADS + t, p + gridDim.x * RED_THREADS, ...  Each thread keeps its partial
// dot products in its own column of shared memory (acc[q * RED_THREADS + t]), so w is loaded once per pack
// however many rows there are, and the block sums are taken in FP64 in a fixed order (deterministic).

// UPDATE = false: part[q * gridDim.x + b] = this block's share of V_q . w              (q < nv)
// UPDATE = true:  w <- w - sum_q h[q] V_q first (h on the device); then the same dots with the new w, and
//                 part[nv * gridDim.x + b] = its share of w . w
// Dynamic shared memory: (nv + UPDATE) * RED_THREADS * sizeof(T).  w is not a row of V[0 .. nv).
template <typename T, int W, bool UPDATE, int MINB = 2, int LOADS = 8>
__global__ void __launch_bounds__(RED_THREADS, MINB)
basis_dots(const T* __restrict__ V, size_t ld, int nv, const double* __restrict__ h, T* w, size_t npack,
           double* __restrict__ part) {
  extern __shared__ unsigned char basis_smem[];
  T* acc = reinterpret_cast<T*>(basis_smem);
  __shared__ T hs[MAX_ROWS];
  const int t = threadIdx.x;
  const int nrow = nv + (UPDATE ? 1 : 0);
  for (int q = 0; q < nrow; ++q) acc[q * RED_THREADS + t] = T(0);
  if (UPDATE && t < nv) hs[t] = (T)h[t];
  __syncthreads();
  for (size_t p = (size_t)blockIdx.x * RED_THREADS + t; p < npack; p += (size_t)gridDim.x * RED_THREADS) {
    Pack<T, W> wp = ld_pack<T, W>(w, p);
    if (UPDATE) {
      for (int v0 = 0; v0 < nv; v0 += LOADS) {
        Pack<T, W> a[LOADS];
#pragma unroll
        for (int q = 0; q < LOADS; ++q)
          if (v0 + q < nv) a[q] = ld_pack<T, W>(V + (size_t)(v0 + q) * ld, p);
#pragma unroll
        for (int q = 0; q < LOADS; ++q)
          if (v0 + q < nv) {
#pragma unroll
            for (int e = 0; e < W; ++e) wp.v[e] = fma(-hs[v0 + q], a[q].v[e], wp.v[e]);
          }
      }
      reinterpret_cast<Pack<T, W>*>(w)[p] = wp;
      T s = T(0);
#pragma unroll
      for (int e = 0; e < W; ++e) s = fma(wp.v[e], wp.v[e], s);
      acc[nv * RED_THREADS + t] += s;
    }
    // (with UPDATE the rows were just read: these loads are served by the caches)
    for (int v0 = 0; v0 < nv; v0 += LOADS) {
      Pack<T, W> a[LOADS];
#pragma unroll
      for (int q = 0; q < LOADS; ++q)
        if (v0 + q < nv) a[q] = ld_pack<T, W>(V + (size_t)(v0 + q) * ld, p);
#pragma unroll
      for (int q = 0; q < LOADS; ++q)
        if (v0 + q < nv) {
          T s = T(0);
#pragma unroll
          for (int e = 0; e < W; ++e) s = fma(a[q].v[e], wp.v[e], s);
          acc[(v0 + q) * RED_THREADS + t] += s;
        }
    }
  }
  __syncthreads();
  // warp k reduces rows k, k + 8, ... over the block's threads in FP64
  const int lane = t & 31, wid = t >> 5;
  for (int q = wid; q < nrow; q += RED_THREADS / 32) {
    double s = 0.0;
    for (int k = lane; k < RED_THREADS; k += 32) s += (double)acc[q * RED_THREADS + k];
    s = warp_sum(s);
    if (lane == 0) part[(size_t)q * gridDim.x + blockIdx.x] = s;
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

// w <- alpha (w - sum_{q < nv} h[q] V_q), h on the device.  alpha = 1, or with normalise
// alpha = 1 / sqrt(h[nv] - sum_q h[q]^2): when h[q] = V_q . w and h[nv] = w . w for orthonormal rows V_q, that
// is the inverse norm of the result (Pythagoras); alpha = 1 when the difference is not positive.
template <typename T, int W, int MINB = 2, int LOADS = 8>
__global__ void __launch_bounds__(RED_THREADS, MINB)
basis_update(const T* __restrict__ V, size_t ld, int nv, const double* __restrict__ h, int normalise, T* w,
             size_t npack) {
  __shared__ T hs[MAX_ROWS];
  __shared__ T alpha_s;
  const int t = threadIdx.x;
  if (t < nv) hs[t] = (T)h[t];
  if (t == 0) {
    double a = 1.0;
    if (normalise) {
      double s2 = h[nv];
      for (int q = 0; q < nv; ++q) s2 -= h[q] * h[q];
      if (s2 > 0.0) a = 1.0 / sqrt(s2);
    }
    alpha_s = (T)a;
  }
  __syncthreads();
  const T alpha = alpha_s;
  for (size_t p = (size_t)blockIdx.x * RED_THREADS + t; p < npack; p += (size_t)gridDim.x * RED_THREADS) {
    Pack<T, W> wp = ld_pack<T, W>(w, p);
    for (int v0 = 0; v0 < nv; v0 += LOADS) {
      Pack<T, W> a[LOADS];
#pragma unroll
      for (int q = 0; q < LOADS; ++q)
        if (v0 + q < nv) a[q] = ld_pack<T, W>(V + (size_t)(v0 + q) * ld, p);
#pragma unroll
      for (int q = 0; q < LOADS; ++q)
        if (v0 + q < nv) {
#pragma unroll
          for (int e = 0; e < W; ++e) wp.v[e] = fma(-hs[v0 + q], a[q].v[e], wp.v[e]);
        }
    }
    if (normalise) {
#pragma unroll
      for (int e = 0; e < W; ++e) wp.v[e] *= alpha;
    }
    reinterpret_cast<Pack<T, W>*>(w)[p] = wp;
  }
}

// x <- x + sum_{q < nv} y[q] Z_q  (the solution update of FGMRES; y on the device)
template <typename T, int W, int MINB = 2, int LOADS = 8>
__global__ void __launch_bounds__(RED_THREADS, MINB)
lincomb_add(const T* __restrict__ Z, size_t ld, int nv, const double* __restrict__ y, T* __restrict__ x,
            size_t npack) {
  __shared__ T ys[MAX_ROWS];
  if (threadIdx.x < nv) ys[threadIdx.x] = (T)y[threadIdx.x];
  __syncthreads();
  for (size_t p = (size_t)blockIdx.x * RED_THREADS + threadIdx.x; p < npack;
       p += (size_t)gridDim.x * RED_THREADS) {
    Pack<T, W> s;
#pragma unroll
    for (int e = 0; e < W; ++e) s.v[e] = T(0);
    for (int v0 = 0; v0 < nv; v0 += LOADS) {
      Pack<T, W> a[LOADS];
#pragma unroll
      for (int q = 0; q < LOADS; ++q)
        if (v0 + q < nv) a[q] = ld_pack<T, W>(Z + (size_t)(v0 + q) * ld, p);
#pragma unroll
      for (int q = 0; q < LOADS; ++q)
        if (v0 + q < nv) {
#pragma unroll
          for (int e = 0; e < W; ++e) s.v[e] = fma(ys[v0 + q], a[q].v[e], s.v[e]);
        }
    }
    Pack<T, W> xp = ld_pack<T, W>(x, p);
#pragma unroll
    for (int e = 0; e < W; ++e) xp.v[e] = s.v[e] + xp.v[e];
    reinterpret_cast<Pack<T, W>*>(x)[p] = xp;
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
