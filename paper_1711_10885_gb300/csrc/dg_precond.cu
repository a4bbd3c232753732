// dg_precond.cu -- block-Jacobi preconditioner: per-cell diagonal blocks A_TT of the operator,
// inverted in a batch (Gauss-Jordan with partial pivoting), applied as a batched matrix-vector product.
#include <algorithm>
#include <cmath>
#include <string>

#include <cuda_fp16.h>

#include "dg_internal.h"

namespace dgi {

// In-place Gauss-Jordan inversion with partial (row) pivoting of one n x n row-major block per CTA.
// SMEM: the block is staged in shared memory; otherwise it is updated in global memory.
template <bool SMEM>
__global__ void __launch_bounds__(256) gj_invert(double* __restrict__ blocks, int n, int* __restrict__ status) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  double* sA = reinterpret_cast<double*>(smem_raw);
  __shared__ double fcol[512];
  __shared__ int perm[512];
  __shared__ double red_v[8];
  __shared__ int red_i[8];
  __shared__ int s_piv;
  __shared__ double s_d;
  double* g = blocks + (size_t)blockIdx.x * n * n;
  double* A = SMEM ? sA : g;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (SMEM) {
    for (int e = tid; e < n * n; e += nt) A[e] = g[e];
    __syncthreads();
  }
  for (int p = 0; p < n; ++p) {
    // pivot: argmax_{i >= p} |A[i][p]| (ties: smallest i)
    double bv = -1.0;
    int bi = p;
    for (int i = p + tid; i < n; i += nt) {
      const double v = fabs(A[(size_t)i * n + p]);
      if (v > bv) {
        bv = v;
        bi = i;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, bv, o);
      const int oi = __shfl_xor_sync(0xffffffffu, bi, o);
      if (ov > bv || (ov == bv && oi < bi)) {
        bv = ov;
        bi = oi;
      }
    }
    if ((tid & 31) == 0) {
      red_v[tid >> 5] = bv;
      red_i[tid >> 5] = bi;
    }
    __syncthreads();
    if (tid == 0) {
      double v = red_v[0];
      int i0 = red_i[0];
      for (int k = 1; k < (nt >> 5); ++k)
        if (red_v[k] > v || (red_v[k] == v && red_i[k] < i0)) {
          v = red_v[k];
          i0 = red_i[k];
        }
      s_piv = i0;
      perm[p] = i0;
    }
    __syncthreads();
    const int piv = s_piv;
    if (piv != p)
      for (int k = tid; k < n; k += nt) {
        const double t = A[(size_t)p * n + k];
        A[(size_t)p * n + k] = A[(size_t)piv * n + k];
        A[(size_t)piv * n + k] = t;
      }
    __syncthreads();
    if (tid == 0) {
      const double a = A[(size_t)p * n + p];
      if (a == 0.0 || !isfinite(a)) {
        atomicAdd(status, 1);
        s_d = 0.0;
      } else {
        s_d = 1.0 / a;
      }
    }
    __syncthreads();
    const double d = s_d;
    for (int k = tid; k < n; k += nt) A[(size_t)p * n + k] = (k == p ? 1.0 : A[(size_t)p * n + k]) * d;
    for (int i = tid; i < n; i += nt) fcol[i] = (i == p) ? 0.0 : A[(size_t)i * n + p];
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {
      const int i = e / n, k = e - i * n;
      if (i != p) A[e] = (k == p ? 0.0 : A[e]) - fcol[i] * A[(size_t)p * n + k];
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int p = n - 1; p >= 0; --p) {
    const int piv = perm[p];
    if (piv != p)
      for (int i = tid; i < n; i += nt) {
        const double t = A[(size_t)i * n + p];
        A[(size_t)i * n + p] = A[(size_t)i * n + piv];
        A[(size_t)i * n + piv] = t;
      }
    __syncthreads();
  }
  if (SMEM)
    for (int e = tid; e < n * n; e += nt) g[e] = A[e];
}

// z_T = A_TT^{-1} r_T with the stored (A_TT^{-1})^T: z_i = sum_j M[j][i] r_j  (one CTA per cell)
template <typename T>
__global__ void __launch_bounds__(256) bj_apply(const T* __restrict__ M, const T* __restrict__ r, T* __restrict__ z,
                                                int n) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* rs = reinterpret_cast<T*>(smem_raw);
  const size_t cell = blockIdx.x;
  const T* Mc = M + cell * n * n;
  for (int j = threadIdx.x; j < n; j += blockDim.x) rs[j] = r[cell * n + j];
  __syncthreads();
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    T acc = T(0);
    for (int j = 0; j < n; ++j) acc = fma(Mc[(size_t)j * n + i], rs[j], acc);
    z[cell * n + i] = acc;
  }
}

// FP32 copy of the inverse blocks with rows padded to np = n rounded up to 4 (16-byte rows)
__global__ void cast_blocks(const double* __restrict__ a, float* __restrict__ b, int64_t nblocks, int n, int np) {
  const size_t total = (size_t)nblocks * n * np;
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < total; i += (size_t)gridDim.x * blockDim.x) {
    const size_t blk = i / ((size_t)n * np);
    const int rem = (int)(i - blk * n * np), row = rem / np, col = rem - row * np;
    b[i] = col < n ? (float)a[(blk * n + row) * n + col] : 0.f;
  }
}

// FP32 block-Jacobi application: z_T = M_T^T r_T with M_T = (A_TT^{-1})^T stored row-padded to np.
// A cell is handled by wpc warps, thread t owning output columns 4t .. 4t+3 (float4 loads of the padded
// rows, several rows in flight); cpc cells share a CTA.
__global__ void __launch_bounds__(128) bj_apply_f32v(const float* __restrict__ M, const float* __restrict__ r,
                                                     float* __restrict__ z, int64_t ncell, int n, int np, int wpc,
                                                     int cpc) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* rs = reinterpret_cast<float*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lc = warp / wpc, wi = warp - lc * wpc;
  const int64_t cell = (int64_t)blockIdx.x * cpc + lc;
  const bool active = lc < cpc && cell < ncell;
  float* rc = rs + lc * np;
  if (active)
    for (int j = wi * 32 + lane; j < n; j += wpc * 32) rc[j] = r[cell * n + j];
  __syncthreads();
  if (!active) return;
  const int t = wi * 32 + lane;  // float4 column index
  if (4 * t >= n) return;
  const float4* Mc = reinterpret_cast<const float4*>(M + (size_t)cell * n * np) + t;
  const int q = np / 4;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  int j = 0;
  for (; j + 8 <= n; j += 8) {
    float4 m[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) m[u] = __ldg(Mc + (size_t)(j + u) * q);
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const float rv = rc[j + u];
      acc.x = fmaf(m[u].x, rv, acc.x);
      acc.y = fmaf(m[u].y, rv, acc.y);
      acc.z = fmaf(m[u].z, rv, acc.z);
      acc.w = fmaf(m[u].w, rv, acc.w);
    }
  }
  for (; j < n; ++j) {
    const float4 m = __ldg(Mc + (size_t)j * q);
    const float rv = rc[j];
    acc.x = fmaf(m.x, rv, acc.x);
    acc.y = fmaf(m.y, rv, acc.y);
    acc.z = fmaf(m.z, rv, acc.z);
    acc.w = fmaf(m.w, rv, acc.w);
  }
  float* zc = z + cell * n + 4 * t;
  const float v[4] = {acc.x, acc.y, acc.z, acc.w};
#pragma unroll
  for (int c = 0; c < 4; ++c)
    if (4 * t + c < n) zc[c] = v[c];
}

// FP16 copy of the inverse blocks for the FP32 inner solves of DG_SOLVE_MIXED: each block is divided by its
// largest |entry| (kept as an FP32 factor per cell), so FP16's range holds any diffusion contrast; rows padded
// to np8 = n rounded up to 8 (16-byte rows).  One CTA per block.
__global__ void __launch_bounds__(256) cast_blocks_f16(const double* __restrict__ a, __half* __restrict__ b,
                                                       float* __restrict__ scale, int n, int np8) {
  __shared__ double red[8];
  const size_t blk = blockIdx.x;
  const double* A = a + blk * n * n;
  double mx = 0.0;
  for (int e = threadIdx.x; e < n * n; e += blockDim.x) mx = fmax(mx, fabs(A[e]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x == 0) {
    double m = red[0];
    for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
    red[0] = m > 0.0 ? m : 1.0;
  }
  __syncthreads();
  const double sc = red[0], inv = 1.0 / sc;
  if (threadIdx.x == 0) scale[blk] = (float)sc;
  __half* B = b + blk * n * np8;
  for (int e = threadIdx.x; e < n * np8; e += blockDim.x) {
    const int row = e / np8, col = e - row * np8;
    B[e] = __double2half(col < n ? A[(size_t)row * n + col] * inv : 0.0);
  }
}

// FP32 block-Jacobi application from the FP16 blocks: z_T = s_T M16_T^T r_T.  Thread column group t owns output
// columns 8t .. 8t+7 (one 16-byte load per row); with at most 16 column groups a warp splits the rows between
// its two halves and adds the halves' sums at the end.  cpc cells share a CTA of 128 threads.
__global__ void __launch_bounds__(128) bj_apply_f16(const __half* __restrict__ M, const float* __restrict__ scale,
                                                    const float* __restrict__ r, float* __restrict__ z,
                                                    int64_t ncell, int n, int np8, int wpc, int cpc, int rsplit) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  float* rs = reinterpret_cast<float*>(smem_raw);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int lc = warp / wpc, wi = warp - lc * wpc;
  const int64_t cell = (int64_t)blockIdx.x * cpc + lc;
  const bool active = lc < cpc && cell < ncell;
  float* rc = rs + lc * np8;
  if (active)
    for (int j = wi * 32 + lane; j < n; j += wpc * 32) rc[j] = r[cell * n + j];
  __syncthreads();
  if (!active) return;
  const int ct = np8 / 8;
  const int t = rsplit == 2 ? (lane & 15) : wi * 32 + lane;  // column group
  const int part = rsplit == 2 ? (lane >> 4) : 0;           // rows part, part + rsplit, ...
  const bool cols = t < ct;
  const uint4* Mc = reinterpret_cast<const uint4*>(M + (size_t)cell * n * np8) + t;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (cols) {
    int j = part;
    for (; j + 3 * rsplit < n; j += 4 * rsplit) {
      uint4 m[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) m[u] = __ldg(Mc + (size_t)(j + u * rsplit) * ct);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const float rv = rc[j + u * rsplit];
        const __half2* h2 = reinterpret_cast<const __half2*>(&m[u]);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const float2 f = __half22float2(h2[q]);
          acc[2 * q] = fmaf(f.x, rv, acc[2 * q]);
          acc[2 * q + 1] = fmaf(f.y, rv, acc[2 * q + 1]);
        }
      }
    }
    for (; j < n; j += rsplit) {
      const uint4 m = __ldg(Mc + (size_t)j * ct);
      const float rv = rc[j];
      const __half2* h2 = reinterpret_cast<const __half2*>(&m);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const float2 f = __half22float2(h2[q]);
        acc[2 * q] = fmaf(f.x, rv, acc[2 * q]);
        acc[2 * q + 1] = fmaf(f.y, rv, acc[2 * q + 1]);
      }
    }
  }
  if (rsplit == 2) {
#pragma unroll
    for (int c = 0; c < 8; ++c) acc[c] += __shfl_xor_sync(0xffffffffu, acc[c], 16);
  }
  if (!cols || part != 0) return;
  const float sc = scale[cell];
  float* zc = z + cell * n + 8 * t;
#pragma unroll
  for (int c = 0; c < 8; ++c)
    if (8 * t + c < n) zc[c] = sc * acc[c];
}

int precond_bj_f16(const dg_handle* h, const float* r, float* z, cudaStream_t s) {
  const int n = h->N * h->N * h->N, np8 = (n + 7) / 8 * 8, ct = np8 / 8;
  const int rsplit = ct <= 16 ? 2 : 1;
  const int wpc = rsplit == 2 ? 1 : (ct + 31) / 32;
  const int cpc = wpc >= 4 ? 1 : 4 / wpc;
  const unsigned grid = (unsigned)((h->ncell + cpc - 1) / cpc);
  bj_apply_f16<<<grid, 32 * wpc * cpc, (size_t)cpc * np8 * sizeof(float), s>>>(
      static_cast<const __half*>(h->bj16), static_cast<const float*>(h->bj16s), r, z, h->ncell, n, np8, wpc, cpc,
      rsplit);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "block-Jacobi apply (FP16 blocks)");
}

int precond_bj_f64(const dg_handle* h, const double* r, double* z, cudaStream_t s) {
  const int n = h->N * h->N * h->N;
  const int threads = n >= 256 ? 256 : ((n + 31) / 32) * 32;
  bj_apply<double><<<(unsigned)h->ncell, threads, n * sizeof(double), s>>>(static_cast<const double*>(h->bj64), r, z, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "block-Jacobi apply");
}

int precond_bj_f32(const dg_handle* h, const float* r, float* z, cudaStream_t s) {
  const int n = h->N * h->N * h->N, np = (n + 3) / 4 * 4;
  const int wpc = (np / 4 + 31) / 32;            // warps per cell
  const int cpc = wpc >= 4 ? 1 : 4 / wpc;        // cells per CTA
  const int threads = 32 * wpc * cpc;
  const unsigned grid = (unsigned)((h->ncell + cpc - 1) / cpc);
  bj_apply_f32v<<<grid, threads, (size_t)cpc * np * sizeof(float), s>>>(static_cast<const float*>(h->bj32), r, z,
                                                                        h->ncell, n, np, wpc, cpc);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "block-Jacobi apply");
}

}  // namespace dgi

using namespace dgi;

extern "C" {

int dg_precond_setup(dg_handle* h, int32_t kind, void* stream) {
  if (!h || kind != 1) {
    set_error("dg_precond_setup: kind must be 1 (block-Jacobi)");
    return DG_ERR_INVALID_ARG;
  }
  if (h->vb || h->td) {
    set_error("dg_precond_setup: block-Jacobi needs a constant velocity, m = k+1 and scalar diffusion on the "
              "axis-parallel grid");
    return DG_ERR_INVALID_ARG;
  }
  for (int r = 0; r < 3; ++r)
    if (h->periodic[r] && h->n[r] == 1) {
      // the diagonal block would have to include the cell's coupling with itself across the wrap
      set_error("dg_precond_setup: a periodic axis needs at least 2 cells for block-Jacobi");
      return DG_ERR_INVALID_ARG;
    }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int N = h->N, n = N * N * N;
  if (n > 512) {
    set_error("dg_precond_setup: block-Jacobi supports (k+1)^3 <= 512");
    return DG_ERR_INVALID_ARG;
  }
  const size_t nblk = (size_t)h->ncell * n * n;
  const int np = (n + 3) / 4 * 4;
  cudaError_t e;
  if (!h->bj64) {
    e = cudaMalloc(&h->bj64, nblk * sizeof(double));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(block-Jacobi FP64)");
  }
  if (!h->bj32) {
    e = cudaMalloc(&h->bj32, (size_t)h->ncell * n * np * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(block-Jacobi FP32)");
  }
  const int np8 = (n + 7) / 8 * 8;
  if (!h->bj16) {
    e = cudaMalloc(&h->bj16, (size_t)h->ncell * n * np8 * sizeof(__half));
    if (e == cudaSuccess) e = cudaMalloc(&h->bj16s, (size_t)h->ncell * sizeof(float));
    if (e != cudaSuccess) return cuda_fail(e, "cudaMalloc(block-Jacobi FP16)");
  }
  // assemble in chunks of cells: each chunk needs (cells * n) virtual cells of work buffers
  int chunk = (int)std::max<int64_t>(1, std::min<int64_t>(h->ncell, h->ncell / n));
  double *V = nullptr, *tr = nullptr;
  const size_t nvirt = (size_t)chunk * n;
  e = cudaMalloc(&V, nvirt * n * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&tr, nvirt * 12 * N * N * sizeof(double));
  int* status = nullptr;
  if (e == cudaSuccess) e = cudaMalloc(&status, sizeof(int));
  if (e == cudaSuccess) e = cudaMemsetAsync(status, 0, sizeof(int), s);
  int rc = DG_OK;
  if (e != cudaSuccess) rc = cuda_fail(e, "block-Jacobi setup buffers");
  for (int64_t c0 = 0; rc == DG_OK && c0 < h->ncell; c0 += chunk) {
    const int nc = (int)std::min<int64_t>(chunk, h->ncell - c0);
    rc = launch_diag_blocks_f64(h, static_cast<double*>(h->bj64) + (size_t)c0 * n * n, (int)c0, nc, V, tr, s);
  }
  if (rc == DG_OK) {
    const size_t smem = (size_t)n * n * sizeof(double);
    if (smem <= 200 * 1024) {
      e = cudaFuncSetAttribute(gj_invert<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) {
        gj_invert<true><<<(unsigned)h->ncell, 256, smem, s>>>(static_cast<double*>(h->bj64), n, status);
        e = cudaGetLastError();
      }
    } else {
      gj_invert<false><<<(unsigned)h->ncell, 256, 0, s>>>(static_cast<double*>(h->bj64), n, status);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      cast_blocks<<<152 * 8, 256, 0, s>>>(static_cast<const double*>(h->bj64), static_cast<float*>(h->bj32), h->ncell,
                                         n, np);
      e = cudaGetLastError();
    }
    if (e == cudaSuccess) {
      cast_blocks_f16<<<(unsigned)h->ncell, 256, 0, s>>>(static_cast<const double*>(h->bj64),
                                                          static_cast<__half*>(h->bj16), static_cast<float*>(h->bj16s),
                                                          n, np8);
      e = cudaGetLastError();
    }
    if (e != cudaSuccess) rc = cuda_fail(e, "block inversion");
  }
  int bad = 0;
  if (rc == DG_OK) {
    e = cudaMemcpyAsync(&bad, status, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = cuda_fail(e, "block-Jacobi setup");
  } else {
    cudaStreamSynchronize(s);
  }
  cudaFree(V);
  cudaFree(tr);
  cudaFree(status);
  if (rc == DG_OK && bad) {
    set_error("dg_precond_setup: " + std::to_string(bad) + " singular diagonal block(s)");
    rc = DG_ERR_NAN;
  }
  return rc;
}

int dg_precond_apply(dg_handle* h, const void* r, void* z, int32_t precision, void* stream) {
  if (!h || !r || !z || r == z || (precision != DG_F64 && precision != DG_F32)) {
    set_error("dg_precond_apply: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  if (!h->bj64) {
    set_error("dg_precond_apply: call dg_precond_setup first");
    return DG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == DG_F64) return precond_bj_f64(h, static_cast<const double*>(r), static_cast<double*>(z), s);
  return precond_bj_f32(h, static_cast<const float*>(r), static_cast<float*>(z), s);
}

}  // extern "C"
