// dg_blas.cuh -- vector kernels of the Krylov solvers (deterministic fixed-order reductions).  The basis
// passes are bound by HBM bandwidth: they move 16 bytes per load and keep several rows in flight.
#pragma once

#include <cuda_fp16.h>
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
// at coef[2 MAX_ROWS + 0, 1, 2]; nothing is done when *stop is set):
//   u = V_{nr-1} <- (u - sum_q a[q] V_q) / alpha         (the reorthogonalised final row; only when write_u)
//   w            <- (w - sum_q d[q] V_q - e u_old) / beta  (the next provisional row)
template <typename T, int W>
__global__ void __launch_bounds__(RED_THREADS, PASS_MINB)
basis_update2(T* V, size_t ld, int nr, const double* __restrict__ coef, int write_u, T* w, size_t npack,
              const int* __restrict__ stop) {
  if (stop && *stop) return;  // the device-side Arnoldi has ended this cycle: nothing to update
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

// ---------------------------------------------------------------------------------------------
// FP16 storage of the inner FP32 FGMRES basis.  The stored rows are unit vectors, or provisional rows of
// about unit length, so their entries are of magnitude 1 at most (typically n^-1/2, 3e-4 at n = 10^7).  They
// are stored times HB_SCALE = 2^8: the typical entry then sits in FP16's normal range (down to 2^-14), and a
// provisional row would have to exceed unit length 256-fold in one entry to overflow (which the Arnoldi step
// reports as a non-finite dot product).  Entries below 2^-22 become subnormal, an absolute error of 2^-33 at
// most.  All arithmetic is FP32; a row is read as (float)h * 2^-8 (exact) and written rounded to nearest.
// Packs of 8 elements: one 16-byte load of the FP16 row, two of an FP32 vector.
// ---------------------------------------------------------------------------------------------
constexpr float HB_SCALE = 256.f, HB_INV = 1.f / 256.f;

struct H8 {
  float v[8];
};
// raw 16-byte load of 8 FP16 entries (kept packed while in flight: 4 registers) and its conversion
__device__ __forceinline__ uint4 ld_raw(const __half* row, size_t p) { return reinterpret_cast<const uint4*>(row)[p]; }
__device__ __forceinline__ H8 unpack_h8(const uint4& q) {
  const __half2* h = reinterpret_cast<const __half2*>(&q);
  H8 r;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(h[i]);
    r.v[2 * i] = f.x * HB_INV;
    r.v[2 * i + 1] = f.y * HB_INV;
  }
  return r;
}
__device__ __forceinline__ H8 ld_h8(const __half* row, size_t p) {
  const uint4 q = reinterpret_cast<const uint4*>(row)[p];
  const __half2* h = reinterpret_cast<const __half2*>(&q);
  H8 r;
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 f = __half22float2(h[i]);
    r.v[2 * i] = f.x * HB_INV;
    r.v[2 * i + 1] = f.y * HB_INV;
  }
  return r;
}
__device__ __forceinline__ void st_h8(__half* row, size_t p, const H8& x) {
  uint4 q;
  __half2* h = reinterpret_cast<__half2*>(&q);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2half2_rn(x.v[2 * i] * HB_SCALE, x.v[2 * i + 1] * HB_SCALE);
  reinterpret_cast<uint4*>(row)[p] = q;
}
__device__ __forceinline__ H8 ld_f8(const float* row, size_t p) {
  const float4 a = reinterpret_cast<const float4*>(row)[2 * p], b = reinterpret_cast<const float4*>(row)[2 * p + 1];
  H8 r;
  r.v[0] = a.x, r.v[1] = a.y, r.v[2] = a.z, r.v[3] = a.w, r.v[4] = b.x, r.v[5] = b.y, r.v[6] = b.z, r.v[7] = b.w;
  return r;
}
__device__ __forceinline__ void st_f8(float* row, size_t p, const H8& x) {
  reinterpret_cast<float4*>(row)[2 * p] = make_float4(x.v[0], x.v[1], x.v[2], x.v[3]);
  reinterpret_cast<float4*>(row)[2 * p + 1] = make_float4(x.v[4], x.v[5], x.v[6], x.v[7]);
}

// row conversions: dst (FP16, scaled) = a * src (FP32); dst (FP32) = src (FP16, unscaled)
__global__ void __launch_bounds__(RED_THREADS) h_store_scaled(const float* __restrict__ src, float a,
                                                              __half* __restrict__ dst, size_t npack) {
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < npack; p += (size_t)gridDim.x * blockDim.x) {
    H8 x = ld_f8(src, p);
#pragma unroll
    for (int e = 0; e < 8; ++e) x.v[e] *= a;
    st_h8(dst, p, x);
  }
}
__global__ void __launch_bounds__(RED_THREADS) h_load(const __half* __restrict__ src, float* __restrict__ dst,
                                                      size_t npack) {
  for (size_t p = (size_t)blockIdx.x * blockDim.x + threadIdx.x; p < npack; p += (size_t)gridDim.x * blockDim.x)
    st_f8(dst, p, ld_h8(src, p));
}

// pass 1 with an FP16 basis (rows V_0 .. V_{nr-1}, u = V_{nr-1}) and an FP32 w; rows of `part` as basis_dots2
__global__ void __launch_bounds__(DOTS2_THREADS, DOTS2_MINB)
basis_dots2_h(const __half* __restrict__ V, size_t ld, int nr, const float* __restrict__ w, size_t npack,
              double* __restrict__ part) {
  extern __shared__ unsigned char basis_smem[];
  float* acc = reinterpret_cast<float*>(basis_smem);
  const int t = threadIdx.x;
  const int nrow = 2 * nr + 1, nf = nr - 1;
  for (int q = 0; q < nrow; ++q) acc[q * DOTS2_THREADS + t] = 0.f;
  __syncthreads();
  const __half* u = V + (size_t)nf * ld;
  for (size_t p = (size_t)blockIdx.x * DOTS2_THREADS + t; p < npack; p += (size_t)gridDim.x * DOTS2_THREADS) {
    const H8 wp = ld_f8(w, p), up = ld_h8(u, p);
    for (int v0 = 0; v0 < nf; v0 += DOTS2_LOADS) {
      uint4 a[DOTS2_LOADS];
#pragma unroll
      for (int q = 0; q < DOTS2_LOADS; ++q)
        if (v0 + q < nf) a[q] = ld_raw(V + (size_t)(v0 + q) * ld, p);
#pragma unroll
      for (int q = 0; q < DOTS2_LOADS; ++q)
        if (v0 + q < nf) {
          const H8 aq = unpack_h8(a[q]);
          float su = 0.f, sw = 0.f;
#pragma unroll
          for (int e = 0; e < 8; ++e) {
            su = fmaf(aq.v[e], up.v[e], su);
            sw = fmaf(aq.v[e], wp.v[e], sw);
          }
          acc[(v0 + q) * DOTS2_THREADS + t] += su;
          acc[(nr + v0 + q) * DOTS2_THREADS + t] += sw;
        }
    }
    float uu = 0.f, uw = 0.f, ww = 0.f;
#pragma unroll
    for (int e = 0; e < 8; ++e) {
      uu = fmaf(up.v[e], up.v[e], uu);
      uw = fmaf(up.v[e], wp.v[e], uw);
      ww = fmaf(wp.v[e], wp.v[e], ww);
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

// pass 2 with an FP16 basis: u = V_{nr-1} <- (u - V a) / alpha (when write_u), V_nr <- (w - V d - e u_old) / beta
// (w FP32, the new row written to the basis); nothing when *stop
__global__ void __launch_bounds__(RED_THREADS, PASS_MINB)
basis_update2_h(__half* V, size_t ld, int nr, const double* __restrict__ coef, int write_u, const float* w,
                size_t npack, const int* __restrict__ stop) {
  if (stop && *stop) return;
  __shared__ float as[MAX_ROWS], ds[MAX_ROWS];
  __shared__ float sc[3];
  const int t = threadIdx.x, nf = nr - 1;
  if (t < nf) {
    as[t] = (float)coef[t];
    ds[t] = (float)coef[MAX_ROWS + t];
  }
  if (t < 3) sc[t] = (float)coef[2 * MAX_ROWS + t];
  __syncthreads();
  const float ia = sc[0], e = sc[1], ib = sc[2];
  __half* u = V + (size_t)nf * ld;
  __half* out = V + (size_t)nr * ld;
  for (size_t p = (size_t)blockIdx.x * RED_THREADS + t; p < npack; p += (size_t)gridDim.x * RED_THREADS) {
    const H8 up = ld_h8(u, p), wp = ld_f8(w, p);
    H8 tu, tw;
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      tu.v[k] = up.v[k];
      tw.v[k] = fmaf(-e, up.v[k], wp.v[k]);
    }
    for (int v0 = 0; v0 < nf; v0 += PASS_LOADS) {
      uint4 a[PASS_LOADS];
#pragma unroll
      for (int q = 0; q < PASS_LOADS; ++q)
        if (v0 + q < nf) a[q] = ld_raw(V + (size_t)(v0 + q) * ld, p);
#pragma unroll
      for (int q = 0; q < PASS_LOADS; ++q)
        if (v0 + q < nf) {
          const H8 aq = unpack_h8(a[q]);
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            tu.v[k] = fmaf(-as[v0 + q], aq.v[k], tu.v[k]);
            tw.v[k] = fmaf(-ds[v0 + q], aq.v[k], tw.v[k]);
          }
        }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      tu.v[k] *= ia;
      tw.v[k] *= ib;
    }
    if (write_u) st_h8(u, p, tu);
    st_h8(out, p, tw);
  }
}

// part[q * gridDim.x + b] = this block's share of V_q . x (q < nv), FP16 rows and FP16 x
__global__ void __launch_bounds__(RED_THREADS, PASS_MINB)
basis_dots_h(const __half* __restrict__ V, size_t ld, int nv, const __half* __restrict__ x, size_t npack,
             double* __restrict__ part) {
  extern __shared__ unsigned char basis_smem[];
  float* acc = reinterpret_cast<float*>(basis_smem);
  const int t = threadIdx.x;
  for (int q = 0; q < nv; ++q) acc[q * RED_THREADS + t] = 0.f;
  __syncthreads();
  for (size_t p = (size_t)blockIdx.x * RED_THREADS + t; p < npack; p += (size_t)gridDim.x * RED_THREADS) {
    const H8 xp = ld_h8(x, p);
    for (int v0 = 0; v0 < nv; v0 += PASS_LOADS) {
      uint4 a[PASS_LOADS];
#pragma unroll
      for (int q = 0; q < PASS_LOADS; ++q)
        if (v0 + q < nv) a[q] = ld_raw(V + (size_t)(v0 + q) * ld, p);
#pragma unroll
      for (int q = 0; q < PASS_LOADS; ++q)
        if (v0 + q < nv) {
          const H8 aq = unpack_h8(a[q]);
          float s = 0.f;
#pragma unroll
          for (int e = 0; e < 8; ++e) s = fmaf(aq.v[e], xp.v[e], s);
          acc[(v0 + q) * RED_THREADS + t] += s;
        }
    }
  }
  __syncthreads();
  const int lane = t & 31, wid = t >> 5;
  for (int q = wid; q < nv; q += RED_THREADS / 32) {
    double s = 0.0;
    for (int k = lane; k < RED_THREADS; k += 32) s += (double)acc[q * RED_THREADS + k];
    s = warp_sum(s);
    if (lane == 0) part[(size_t)q * gridDim.x + blockIdx.x] = s;
  }
}

// ---------------------------------------------------------------------------------------------
// Device-side bookkeeping of the FGMRES cycle (one thread): the Hessenberg matrix, its Givens rotations, the
// rotated right-hand side g and the residual estimate |g[col + 1]| live in device memory, so a cycle runs
// without a host synchronisation per Arnoldi step.  The steps are those of the host loop they replace (see
// fgmres in dg_solve.cu): the reorthogonalisation of the provisional row u_j gives a and alpha and finalises
// Hessenberg column j - 1; the coefficients of w on the final rows give column j provisionally and the
// coefficients of pass 2.  A cycle ends (stop) on convergence, breakdown or a non-finite value; pass 2 and
// the later steps' bookkeeping then do nothing.
// ---------------------------------------------------------------------------------------------
struct ArnState {
  double res;   // current residual estimate |g[fin]|
  double btil;  // provisional norm of the last projection
  double tol;   // absolute stopping tolerance
  double prov;  // provisional estimate of the residual after the last step's column (H[j+1][j] ~ btil)
  int m;        // restart length (row length of H)
  int fin;      // columns 0 .. fin-1 of H are final and rotated into g
  int jend;     // columns of this cycle (Hessenberg columns computed)
  int stop;     // the cycle has ended
  int err;      // 1: a non-finite value was met
  int pad;
  double cs[MAX_ROWS], sn[MAX_ROWS], g[MAX_ROWS + 1], cprev[MAX_ROWS + 1], a[MAX_ROWS + 1];
  double H[(MAX_ROWS + 1) * MAX_ROWS];
};
constexpr int ARN_HEAD_BYTES = 56;  // res .. pad: what the host reads back

// The values a step works on, staged by the warp in shared memory before one thread does the scalar work (each
// global value is read once, in parallel, instead of by a chain of dependent loads).
struct ArnCache {
  double d[2 * MAX_ROWS + 1];  // the pass's dot products
  double cp[MAX_ROWS + 1];     // provisional column (cprev)
  double cs[MAX_ROWS], sn[MAX_ROWS], g[MAX_ROWS + 1];
  double h[MAX_ROWS + 1];      // the column being finalised
};

__device__ inline void arn_stage(ArnCache& k, const ArnState* st, const double* dots, int nd, int j) {
  for (int i = threadIdx.x; i < nd; i += blockDim.x) k.d[i] = dots[i];
  for (int i = threadIdx.x; i <= j; i += blockDim.x) k.cp[i] = st->cprev[i];
  for (int i = threadIdx.x; i < j; i += blockDim.x) {
    k.cs[i] = st->cs[i];
    k.sn[i] = st->sn[i];
  }
  for (int i = threadIdx.x; i <= j + 1 && i <= st->m; i += blockDim.x) k.g[i] = st->g[i];
  __syncthreads();
}

// column col of H from the provisional coefficients cp, btil and the next row's reorthogonalisation (ap, alpha),
// rotated by the previous rotations and a new one annihilating H[col+1][col]; g, fin and the residual estimate
// follow (thread 0; st in global memory, k the staged copies)
__device__ inline void arn_finalize(ArnState* st, ArnCache& k, int col, const double* ap, double alpha) {
  const int m = st->m;
  double* h = k.h;
  for (int i = 0; i <= col; ++i) h[i] = k.cp[i] + st->btil * ap[i];
  h[col + 1] = st->btil * alpha;
  for (int i = 0; i < col; ++i) {
    const double p = h[i], q = h[i + 1];
    h[i] = k.cs[i] * p + k.sn[i] * q;
    h[i + 1] = -k.sn[i] * p + k.cs[i] * q;
  }
  const double p = h[col], q = h[col + 1];
  const double rr = hypot(p, q);
  const double c = rr > 0 ? p / rr : 1.0, sn = rr > 0 ? q / rr : 0.0;
  k.cs[col] = st->cs[col] = c;
  k.sn[col] = st->sn[col] = sn;
  h[col] = rr;
  h[col + 1] = 0.0;
  for (int i = 0; i <= col + 1; ++i) st->H[i * m + col] = h[i];
  const double gc = k.g[col];
  k.g[col + 1] = st->g[col + 1] = -sn * gc;
  k.g[col] = st->g[col] = c * gc;
  st->fin = col + 1;
  st->res = fabs(k.g[col + 1]);
}

__global__ void arn_init(ArnState* st, int m, double tol, double beta) {
  st->res = beta;
  st->btil = 0.0;
  st->tol = tol;
  st->prov = beta;
  st->m = m;
  st->fin = st->jend = st->stop = st->err = 0;
  for (int i = 0; i <= m; ++i) st->g[i] = 0.0;
  st->g[0] = beta;
}

// step j (one warp): dots = (V_q . u_j, q <= j; V_q . w, q <= j; w . w) from pass 1; writes pass 2's coefficients
__global__ void arn_step(ArnState* st, const double* __restrict__ dots, int j, double* __restrict__ coef) {
  __shared__ ArnCache k;
  if (st->stop) return;  // uniform: every thread reads the same flag before any thread writes it
  arn_stage(k, st, dots, 2 * j + 3, j);
  if (threadIdx.x != 0) return;
  const double* pu = k.d;
  const double* qw = k.d + j + 1;
  const double ww = k.d[2 * j + 2];
  double* a = st->a;
  double alpha = 1.0;  // u_0 is final
  if (j > 0) {
    double s2 = pu[j];
    for (int i = 0; i < j; ++i) {
      a[i] = pu[i];
      s2 -= pu[i] * pu[i];
    }
    if (!isfinite(s2)) {
      st->err = 1;
      st->stop = 1;
      return;
    }
    alpha = sqrt(fmax(s2, 0.0));
    if (st->fin < j) arn_finalize(st, k, j - 1, pu, alpha);
    if (st->res <= st->tol || alpha == 0.0) {  // converged, or u_j in the span of the final rows (breakdown)
      st->jend = j;
      st->stop = 1;
      return;
    }
  }
  // coefficients of w on the final rows 0 .. j; they become the provisional column (cprev)
  double bt2 = ww, ca = 0.0;
  for (int i = 0; i < j; ++i) ca += pu[i] * qw[i];
  const double cj = (qw[j] - ca) / alpha;
  for (int i = 0; i < j; ++i) {
    k.cp[i] = st->cprev[i] = qw[i];
    bt2 -= qw[i] * qw[i];
  }
  k.cp[j] = st->cprev[j] = cj;
  bt2 -= cj * cj;
  if (!isfinite(bt2)) {
    st->err = 1;
    st->stop = 1;
    return;
  }
  st->jend = j + 1;
  if (bt2 <= 0.0) {  // w in the span of the basis: column j is final with a zero subdiagonal entry
    st->btil = 0.0;
    arn_finalize(st, k, j, pu, 0.0);
    st->stop = 1;
    return;
  }
  const double btil = sqrt(bt2);
  st->btil = btil;
  // provisional estimate of the residual after column j: the column rotated by the previous rotations, with
  // btil as its subdiagonal entry
  {
    double* col = k.h;
    for (int i = 0; i <= j; ++i) col[i] = k.cp[i];
    for (int i = 0; i < j; ++i) {
      const double p = col[i], q = col[i + 1];
      col[i] = k.cs[i] * p + k.sn[i] * q;
      col[i + 1] = -k.sn[i] * p + k.cs[i] * q;
    }
    st->prov = fabs(k.g[j]) * btil / fmax(hypot(col[j], btil), 1e-300);
  }
  // pass 2: v_j = (u_j - V_{<j} a) / alpha, u_{j+1} = (w - V_{<j} d - e u_j) / btil
  const double e = cj / alpha;
  for (int i = 0; i < j; ++i) {
    coef[i] = pu[i];
    coef[MAX_ROWS + i] = qw[i] - e * pu[i];
  }
  coef[2 * MAX_ROWS + 0] = 1.0 / alpha;
  coef[2 * MAX_ROWS + 1] = e;
  coef[2 * MAX_ROWS + 2] = 1.0 / btil;
}

// after the last step j of a cycle (one warp): dots = (V_q . u_{j+1}, q <= j + 1) finalise column j
__global__ void arn_final(ArnState* st, const double* __restrict__ dots, int j) {
  __shared__ ArnCache k;
  if (st->stop || st->fin >= st->jend) return;
  arn_stage(k, st, dots, j + 2, j);
  if (threadIdx.x != 0) return;
  double s2 = k.d[j + 1];
  for (int i = 0; i <= j; ++i) s2 -= k.d[i] * k.d[i];
  if (!isfinite(s2)) {
    st->err = 1;
    st->stop = 1;
    return;
  }
  arn_finalize(st, k, j, k.d, sqrt(fmax(s2, 0.0)));
}

// y = H^{-1} g over the cycle's jend columns (upper triangular after the rotations), zero beyond (one thread)
__global__ void arn_solve(const ArnState* st, double* __restrict__ y) {
  const int m = st->m, n = st->jend;
  for (int i = m - 1; i >= n; --i) y[i] = 0.0;
  for (int i = n - 1; i >= 0; --i) {
    double acc = st->g[i];
    for (int q = i + 1; q < n; ++q) acc -= st->H[i * m + q] * y[q];
    y[i] = st->H[i * m + i] != 0.0 ? acc / st->H[i * m + i] : 0.0;
  }
}

}  // namespace dgb
