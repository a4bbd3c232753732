// dg_blas.cuh -- vector kernels of the Krylov solvers (deterministic fixed-order reductions).  The basis
// passes are bound by HBM bandwidth: they move 16 bytes per load and keep several rows in flight.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace dgb {

// grids are sized by the caller from the device's SM count: one wave of each kernel's resident CTAs
constexpr int RED_THREADS = 256;
constexpr int PASS_MINB = 3;           // resident CTAs per SM of the basis passes (their launch bounds)
constexpr int PASS_LOADS = 8;          // rows loaded together by the dot and update passes (80 registers or fewer)
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

// part[q * gridDim.x + b] = this block's share of V_q . w  (q < nv).  Dynamic shared memory:
// nv * RED_THREADS * sizeof(T).
template <typename T, int W, int MINB, int LOADS>
__global__ void __launch_bounds__(RED_THREADS, MINB)
basis_dots(const T* __restrict__ V, size_t ld, int nv, const T* __restrict__ w, size_t npack,
           double* __restrict__ part) {
  extern __shared__ unsigned char basis_smem[];
  T* acc = reinterpret_cast<T*>(basis_smem);
  const int t = threadIdx.x;
  for (int q = 0; q < nv; ++q) acc[q * RED_THREADS + t] = T(0);
  __syncthreads();
  for (size_t p = (size_t)blockIdx.x * RED_THREADS + t; p < npack; p += (size_t)gridDim.x * RED_THREADS) {
    const Pack<T, W> wp = ld_pack<T, W>(w, p);
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
  for (int q = wid; q < nv; q += RED_THREADS / 32) {
    double s = 0.0;
    for (int k = lane; k < RED_THREADS; k += 32) s += (double)acc[q * RED_THREADS + k];
    s = warp_sum(s);
    if (lane == 0) part[(size_t)q * gridDim.x + blockIdx.x] = s;
  }
}

// Arnoldi with the reorthogonalisation delayed by one step takes two passes per step over the basis.  Rows
// V_0 .. V_{nr-2} are final (orthonormal), the last row u = V_{nr-1} is provisional and w is the new vector.
constexpr int DOTS2_THREADS = 128;
constexpr int DOTS2_MINB = 6;
constexpr int PART_ROWS = 2 * MAX_ROWS + 1;  // rows of block sums a pass can produce
constexpr int DOTS2_LOADS = 6;

// pass 1, dots against u and w in one pass:
//   part row q       (q < nr): V_q . u   (q = nr - 1: u . u)
//   part row nr + q  (q < nr): V_q . w
//   part row 2 nr:             w . w
// Dynamic shared memory: (2 nr + 1) * DOTS2_THREADS * sizeof(T).
template <typename T, int W>
__global__ void __launch_bounds__(DOTS2_THREADS, DOTS2_MINB)
basis_dots2(const T* __restrict__ V, size_t ld, int nr, const T* __restrict__ w, size_t npack,
            double* __restrict__ part) {
  extern __shared__ unsigned char basis_smem[];
  T* acc = reinterpret_cast<T*>(basis_smem);
  const int t = threadIdx.x;
  const int nrow = 2 * nr + 1, nf = nr - 1;
  for (int q = 0; q < nrow; ++q) acc[q * DOTS2_THREADS + t] = T(0);
  __syncthreads();
  const T* u = V + (size_t)nf * ld;
  for (size_t p = (size_t)blockIdx.x * DOTS2_THREADS + t; p < npack; p += (size_t)gridDim.x * DOTS2_THREADS) {
    const Pack<T, W> wp = ld_pack<T, W>(w, p), up = ld_pack<T, W>(u, p);
    for (int v0 = 0; v0 < nf; v0 += DOTS2_LOADS) {
      Pack<T, W> a[DOTS2_LOADS];
#pragma unroll
      for (int q = 0; q < DOTS2_LOADS; ++q)
        if (v0 + q < nf) a[q] = ld_pack<T, W>(V + (size_t)(v0 + q) * ld, p);
#pragma unroll
      for (int q = 0; q < DOTS2_LOADS; ++q)
        if (v0 + q < nf) {
          T su = T(0), sw = T(0);
#pragma unroll
          for (int e = 0; e < W; ++e) {
            su = fma(a[q].v[e], up.v[e], su);
            sw = fma(a[q].v[e], wp.v[e], sw);
          }
          acc[(v0 + q) * DOTS2_THREADS + t] += su;
          acc[(nr + v0 + q) * DOTS2_THREADS + t] += sw;
        }
    }
    T uu = T(0), uw = T(0), ww = T(0);
#pragma unroll
    for (int e = 0; e < W; ++e) {
      uu = fma(up.v[e], up.v[e], uu);
      uw = fma(up.v[e], wp.v[e], uw);
      ww = fma(wp.v[e], wp.v[e], ww);
    }
    acc[nf * DOTS2_THREADS + t] += uu;
    acc[(nr + nf) * DOTS2_THREADS + t] += uw;
    acc[2 * nr * DOTS2_THREADS + t] += ww;
  }
  __syncthreads();
  const int lane = t & 31, wid = t >> 5;
  for (int q = wid; q < nrow; q += DOTS2_THREADS / 32) {
    double s = 0.0;
    for (int k = lane; k < DOTS2_THREADS; k += 32) s += (double)acc[q * DOTS2_THREADS + k];
    s = warp_sum(s);
    if (lane == 0) part[(size_t)q * gridDim.x + blockIdx.x] = s;
  }
}

// pass 2 (coef on the device: a[q] at coef[q], d[q] at coef[MAX_ROWS + q] for q < nr - 1, then 1/alpha, e, 1/beta
// at coef[2 MAX_ROWS + 0, 1, 2]):
//   u = V_{nr-1} <- (u - sum_q a[q] V_q) / alpha         (the reorthogonalised final row; only when write_u)
//   w            <- (w - sum_q d[q] V_q - e u_old) / beta  (the next provisional row)
template <typename T, int W>
__global__ void __launch_bounds__(RED_THREADS, PASS_MINB)
basis_update2(T* V, size_t ld, int nr, const double* __restrict__ coef, int write_u, T* w, size_t npack) {
  __shared__ T as[MAX_ROWS], ds[MAX_ROWS];
  __shared__ T sc[3];
  const int t = threadIdx.x, nf = nr - 1;
  if (t < nf) {
    as[t] = (T)coef[t];
    ds[t] = (T)coef[MAX_ROWS + t];
  }
  if (t < 3) sc[t] = (T)coef[2 * MAX_ROWS + t];
  __syncthreads();
  const T ia = sc[0], e = sc[1], ib = sc[2];
  T* u = V + (size_t)nf * ld;
  for (size_t p = (size_t)blockIdx.x * RED_THREADS + t; p < npack; p += (size_t)gridDim.x * RED_THREADS) {
    Pack<T, W> up = ld_pack<T, W>(u, p), wp = ld_pack<T, W>(w, p), tu, tw;
#pragma unroll
    for (int k = 0; k < W; ++k) {
      tu.v[k] = up.v[k];
      tw.v[k] = fma(-e, up.v[k], wp.v[k]);
    }
    for (int v0 = 0; v0 < nf; v0 += PASS_LOADS) {
      Pack<T, W> a[PASS_LOADS];
#pragma unroll
      for (int q = 0; q < PASS_LOADS; ++q)
        if (v0 + q < nf) a[q] = ld_pack<T, W>(V + (size_t)(v0 + q) * ld, p);
#pragma unroll
      for (int q = 0; q < PASS_LOADS; ++q)
        if (v0 + q < nf) {
#pragma unroll
          for (int k = 0; k < W; ++k) {
            tu.v[k] = fma(-as[v0 + q], a[q].v[k], tu.v[k]);
            tw.v[k] = fma(-ds[v0 + q], a[q].v[k], tw.v[k]);
          }
        }
    }
#pragma unroll
    for (int k = 0; k < W; ++k) {
      tu.v[k] *= ia;
      tw.v[k] *= ib;
    }
    if (write_u) reinterpret_cast<Pack<T, W>*>(u)[p] = tu;
    reinterpret_cast<Pack<T, W>*>(w)[p] = tw;
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

// out[i] = alpha * in[i] (with a precision change; out may be in)
template <typename TI, typename TO>
__global__ void __launch_bounds__(RED_THREADS)
scale_copy(const TI* in, TO* out, double alpha, size_t n) {
  const TI a = (TI)alpha;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = (TO)(a * in[i]);
}

// out[i] = a[i] - b[i]  (out may be b: each element is read before it is written by the same thread)
template <typename T>
__global__ void __launch_bounds__(RED_THREADS)
sub(const T* __restrict__ a, const T* b, T* out, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    out[i] = a[i] - b[i];
}

}  // namespace dgb
