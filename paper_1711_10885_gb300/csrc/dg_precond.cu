// dg_precond.cu -- block-Jacobi preconditioner: per-cell diagonal blocks A_TT of the operator,
// inverted in a batch (Gauss-Jordan with partial pivoting), applied as a batched matrix-vector product.
#include <algorithm>
#include <cmath>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include <cuda_fp16.h>

#include "dg_eig.h"
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

// ---------------------------------------------------------------------------------------------
// Exact block inverse by fast diagonalisation.  On an axis-parallel cell with a per-cell scalar D and a constant
// velocity, every term of the diagonal block A_TT (the volume term and the self-coupling of the cell's faces,
// eq. blf) is a tensor product of a 1D matrix along one axis with identities (the basis is orthonormal), so
//   A_TT = I (x) I (x) A_x + I (x) A_y (x) I + A_z (x) I (x) I + c |T| I
// with per-cell 1D operators A_r = V_r diag(lambda_r) V_r^{-1}, and
//   A_TT^{-1} = (V_z (x) V_y (x) V_x) diag(1 / (lambda_x + lambda_y + lambda_z + c |T|)) (W_z (x) W_y (x) W_x),
// W_r = V_r^{-1}: six 1D complex contractions per cell instead of a dense n^3 x n^3 product, from 3 (2 n^2 + n)
// complex numbers per cell instead of n^6.
// Table per cell (float2 = complex FP32): for r = 0..2: W_r [n][n], V_r [n][n], lambda_r [n]; then c |T|.
// ---------------------------------------------------------------------------------------------
template <typename R>
struct Cx;
template <>
struct Cx<float> {
  using type = float2;
};
template <>
struct Cx<double> {
  using type = double2;
};

// cell indices of the group positions q0 .. q0 + here - 1 (cells null: position = cell), into shared memory
__device__ __forceinline__ void load_cells(int64_t* s_cell, const int64_t* __restrict__ cells, int64_t q0, int here) {
  for (int i = threadIdx.x; i < here; i += blockDim.x) s_cell[i] = cells ? cells[q0 + i] : q0 + i;
}

// kernels over one group of cells: positions 0 .. count - 1 of the group, tables in group order
template <int N, typename R>
__global__ void __launch_bounds__(256) fdm_apply(const typename Cx<R>::type* __restrict__ tab, const R* __restrict__ r,
                                                 R* __restrict__ z, int64_t count, const int64_t* __restrict__ cells,
                                                 int cpb) {
  using C = typename Cx<R>::type;
  constexpr int NN = N * N, N3 = NN * N, TS = 3 * (2 * NN + N) + 1;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t s_cell[64];
  C* U = reinterpret_cast<C*>(smem_raw);  // [cpb][N3]
  C* T = U + (size_t)cpb * N3;             // [cpb][TS]
  const int lc = threadIdx.x / NN, t = threadIdx.x - lc * NN;
  const int64_t q0 = (int64_t)blockIdx.x * cpb;
  const int here = (int)min((int64_t)cpb, count - q0);
  load_cells(s_cell, cells, q0, here);
  for (int e = threadIdx.x; e < here * TS; e += blockDim.x) T[e] = tab[q0 * TS + e];
  __syncthreads();
  for (int e = threadIdx.x; e < here * N3; e += blockDim.x) {
    const int l = e / N3;
    C v;
    v.x = r[s_cell[l] * N3 + (e - l * N3)];
    v.y = R(0);
    U[e] = v;
  }
  __syncthreads();
  const bool active = lc < here;
  C* u = U + lc * N3;
  const C* tb = T + lc * TS;
  // line of this thread along axis d: the N points with the other two indices (a, b) = (t % N, t / N)
  auto base = [&](int d) { return d == 0 ? N * t : (d == 1 ? (t % N) + NN * (t / N) : t); };
  auto stride = [](int d) { return d == 0 ? 1 : (d == 1 ? N : NN); };
  auto pass = [&](int d, const C* Mx) {  // u_line <- Mx u_line (complex N x N)
    if (active) {
      const int bs = base(d), st = stride(d);
      C x[N], y[N];
#pragma unroll
      for (int l = 0; l < N; ++l) x[l] = u[bs + l * st];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        R re = R(0), im = R(0);
#pragma unroll
        for (int l = 0; l < N; ++l) {
          const C m = Mx[i * N + l];
          re = fma(m.x, x[l].x, fma(-m.y, x[l].y, re));
          im = fma(m.x, x[l].y, fma(m.y, x[l].x, im));
        }
        y[i].x = re;
        y[i].y = im;
      }
#pragma unroll
      for (int i = 0; i < N; ++i) u[bs + i * st] = y[i];
    }
    __syncthreads();
  };
  for (int d = 0; d < 3; ++d) pass(d, tb + d * (2 * NN + N));  // W_d
  if (active) {
    // divide by lambda_x(a) + lambda_y(b) + lambda_z(c) + c |T| along this thread's z-line (a, b)
    const C* lx = tb + 0 * (2 * NN + N) + 2 * NN;
    const C* ly = tb + 1 * (2 * NN + N) + 2 * NN;
    const C* lz = tb + 2 * (2 * NN + N) + 2 * NN;
    const R cs = tb[TS - 1].x;
    const int a = t % N, b = t / N;
#pragma unroll
    for (int c = 0; c < N; ++c) {
      const R dr = lx[a].x + ly[b].x + lz[c].x + cs, di = lx[a].y + ly[b].y + lz[c].y;
      const R inv = R(1) / (dr * dr + di * di);
      C v = u[a + N * b + NN * c];
      const R vr = (v.x * dr + v.y * di) * inv, vi = (v.y * dr - v.x * di) * inv;
      v.x = vr;
      v.y = vi;
      u[a + N * b + NN * c] = v;
    }
  }
  __syncthreads();
  for (int d = 0; d < 3; ++d) pass(d, tb + d * (2 * NN + N) + NN);  // V_d
  for (int e = threadIdx.x; e < here * N3; e += blockDim.x) {
    const int l = e / N3;
    z[s_cell[l] * N3 + (e - l * N3)] = U[e].x;
  }
}

// FP32 variant for n <= 6 with fewer shared-memory transactions: n threads per cell.  Thread p owns the plane
// c = p for the x and y passes and the lines (a, b = p) for the z passes, so only two barriers separate the
// passes.  Each pass holds its n x n complex matrix in registers (one load per thread instead of one per line)
// and streams the thread's n lines through it; the first pass reads real data and the last keeps only the real
// part.  Plane and table pitches are odd (in 8-byte words), so lanes of neighbouring planes and cells fall on
// distinct shared-memory banks.
template <int N>
struct FdmPlanes {
  static constexpr int NN = N * N, N3 = NN * N;
  static constexpr int PP = NN | 1;                   // pitch of a plane c (complex words)
  static constexpr int CP = N * PP;                   // pitch of a cell's data
  static constexpr int TS = 3 * (2 * NN + N) + 1;     // table entries per cell
  static constexpr int TSP = TS | 1;                  // their pitch in shared memory
  static constexpr int CELL_BYTES = (CP + TSP) * 8;
  static constexpr int CB_SMEM = 56 * 1024 / CELL_BYTES;
  static constexpr int CB = CB_SMEM < 128 / N ? CB_SMEM : 128 / N;  // cells per CTA (4 CTAs per SM)
  static constexpr int SMEM = CB * CELL_BYTES;
};

// u[base + i * stride] <- sum_l m[i][l] u[base + l * stride] (complex); ROUT: only the real part of the output
// is formed
template <int N, bool ROUT>
__device__ __forceinline__ void fdm_line(const float2 (&m)[N][N], float2* u, int base, int stride) {
  float2 x[N], y[N];
#pragma unroll
  for (int l = 0; l < N; ++l) x[l] = u[base + l * stride];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float re = 0.f, im = 0.f;
#pragma unroll
    for (int l = 0; l < N; ++l) {
      re = fmaf(m[i][l].x, x[l].x, fmaf(-m[i][l].y, x[l].y, re));
      if (!ROUT) im = fmaf(m[i][l].x, x[l].y, fmaf(m[i][l].y, x[l].x, im));
    }
    y[i] = make_float2(re, im);
  }
#pragma unroll
  for (int i = 0; i < N; ++i) u[base + i * stride] = y[i];
}

template <int N>
__device__ __forceinline__ void fdm_matrix(float2 (&m)[N][N], const float2* M) {
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int l = 0; l < N; ++l) m[i][l] = M[i * N + l];
}

// asynchronous global -> shared copies (no registers held, so a thread keeps all its copies in flight)
__device__ __forceinline__ void cp_async(void* dst, const void* src, int bytes_is_8) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  if (bytes_is_8)
    asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(d), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

template <int N>
__global__ void __launch_bounds__(128, 4) fdm_apply_planes(const float2* __restrict__ tab, const float* __restrict__ r,
                                                          float* __restrict__ z, int64_t count,
                                                          const int64_t* __restrict__ cells) {
  using P = FdmPlanes<N>;
  constexpr int NN = P::NN, N3 = P::N3, PP = P::PP, CP = P::CP, TS = P::TS, TSP = P::TSP, AX = 2 * NN + N;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t s_cell[P::CB];
  float2* U = reinterpret_cast<float2*>(smem_raw);  // [CB][CP]: U[cell][c * PP + a + N b]
  float2* T = U + P::CB * CP;                        // [CB][TSP]
  const int64_t q0 = (int64_t)blockIdx.x * P::CB;
  const int here = (int)min((int64_t)P::CB, count - q0);
  load_cells(s_cell, cells, q0, here);
  for (int e = threadIdx.x; e < here * TS; e += blockDim.x) {
    const int l = e / TS;
    cp_async(T + l * TSP + (e - l * TS), tab + q0 * TS + e, 1);
  }
  __syncthreads();
  // the real input of plane c sits in the upper half of its complex slot: floats PP .. PP + NN - 1 of the plane
  for (int e = threadIdx.x; e < here * N3; e += blockDim.x) {
    const int l = e / N3, rem = e - l * N3, c = rem / NN;
    cp_async(reinterpret_cast<float*>(U + l * CP + c * PP) + PP + (rem - c * NN), r + s_cell[l] * N3 + rem, 0);
  }
  cp_async_wait_all();
  __syncthreads();
  const int lc = threadIdx.x / N, p = threadIdx.x - lc * N;
  const bool active = lc < here;
  float2* u = U + lc * CP;
  const float2* tb = T + lc * TSP;
  float2 m[N][N];
  if (active) {  // W_x on the x-lines (b, c = p) from the real input, W_y on the y-lines (a, c = p)
    fdm_matrix<N>(m, tb);
    const float* ur = reinterpret_cast<const float*>(u + p * PP) + PP;
    for (int b = 0; b < N; ++b) {
      // line b's complex output (floats 2 N b .. 2 N (b + 1) - 1 of the plane) stays below the real input of the
      // later lines (floats PP + N (b + 1) ...), since N (b + 1) <= N^2 < PP + 1
      float x[N];
#pragma unroll
      for (int l = 0; l < N; ++l) x[l] = ur[N * b + l];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        float re = 0.f, im = 0.f;
#pragma unroll
        for (int l = 0; l < N; ++l) {
          re = fmaf(m[i][l].x, x[l], re);
          im = fmaf(m[i][l].y, x[l], im);
        }
        u[p * PP + N * b + i] = make_float2(re, im);
      }
    }
    fdm_matrix<N>(m, tb + AX);
    for (int a = 0; a < N; ++a) fdm_line<N, false>(m, u, p * PP + a, N);
  }
  __syncthreads();
  if (active) {  // W_z on the z-lines (a, b = p); divide by lambda_x(a) + lambda_y(p) + lambda_z(c) + c |T|; V_z
    fdm_matrix<N>(m, tb + 2 * AX);
    for (int a = 0; a < N; ++a) fdm_line<N, false>(m, u, a + N * p, PP);
    const float2* lx = tb + 2 * NN;
    const float2 ly = tb[AX + 2 * NN + p];
    const float2* lz = tb + 2 * AX + 2 * NN;
    const float cs = tb[TS - 1].x;
    for (int a = 0; a < N; ++a) {
#pragma unroll
      for (int c = 0; c < N; ++c) {
        const float dr = lx[a].x + ly.x + lz[c].x + cs, di = lx[a].y + ly.y + lz[c].y;
        const float inv = 1.f / (dr * dr + di * di);
        float2 v = u[a + N * p + PP * c];
        u[a + N * p + PP * c] = make_float2((v.x * dr + v.y * di) * inv, (v.y * dr - v.x * di) * inv);
      }
    }
    fdm_matrix<N>(m, tb + 2 * AX + NN);
    for (int a = 0; a < N; ++a) fdm_line<N, false>(m, u, a + N * p, PP);
  }
  __syncthreads();
  if (active) {  // V_y on the y-lines, V_x on the x-lines (real part only)
    fdm_matrix<N>(m, tb + AX + NN);
    for (int a = 0; a < N; ++a) fdm_line<N, false>(m, u, p * PP + a, N);
    fdm_matrix<N>(m, tb + NN);
    for (int b = 0; b < N; ++b) fdm_line<N, true>(m, u, p * PP + N * b, 1);
  }
  __syncthreads();
  for (int e = threadIdx.x; e < here * N3; e += blockDim.x) {
    const int l = e / N3, rem = e - l * N3, c = rem / NN;
    z[s_cell[l] * N3 + rem] = U[l * CP + c * PP + (rem - c * NN)].x;
  }
}

// ---------------------------------------------------------------------------------------------
// The same inverse with real tables: when a cell's 1D operators have real eigenvalues (diffusion-dominated
// cells, the usual case: the convection term is a small skew perturbation of the symmetric stiffness and
// penalty terms) V_r, W_r and lambda_r are real, and each 1D contraction is a real n x n product (a quarter of
// the complex one's FMAs).  Table per cell (RealLay): for r = 0..2 at r * AXP: W_r [n][n], V_r [n][n],
// lambda_r [n], zero padding to a multiple of 4 entries; c |T| at 3 AXP; TP entries in all (a multiple of 4, so
// every cell's table, and for even n every matrix, starts on a 16-byte boundary in FP32).
// ---------------------------------------------------------------------------------------------
template <int N>
struct RealLay {
  static constexpr int NN = N * N;
  static constexpr int AXP = (2 * NN + N + 3) / 4 * 4;
  static constexpr int TP = 3 * AXP + 4;
};

__device__ __forceinline__ void cp_async16(void* dst, const void* src) {
  const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

// FP32, n <= 8: n threads per cell.  Thread p holds plane c = p in registers for the x and y passes and the
// z-lines (a, b = p) for the z pass, so the data crosses shared memory once per phase (three phases, two
// barriers), and each pass matrix is read once per thread (float4 rows for even n).  Cell data pitch UP and
// table pitch TP are multiples of 4 words: the 16-byte plane loads of the n threads of a cell and of
// neighbouring cells fall on distinct bank groups.
template <int N>
struct FdmPlanesR {
  static constexpr int NN = N * N, N3 = NN * N;
  static constexpr bool V4 = NN % 4 == 0;  // planes and matrices in 16-byte rows (even n)
  // cell pitch: a multiple of 4 words for the 16-byte rows, else odd (scalar accesses of neighbouring cells on
  // distinct banks)
  static constexpr int UP = V4 ? (N3 + 3) / 4 * 4 : (N3 | 1);
  static constexpr int TP = RealLay<N>::TP;
  static constexpr int CB = 128 / N;                  // cells per CTA
  static constexpr int TOFF = (CB * UP + 3) / 4 * 4;  // the tables start on a 16-byte boundary
  static constexpr int SMEM = (TOFF + CB * TP) * 4;
  static constexpr int SMEM_H = SMEM + CB * N3 * 2;    // plus the FP16 input staging
};

// n x n matrix (row-major) from shared memory into registers
template <int N, bool V4>
__device__ __forceinline__ void fdm_load_r(float* m, const float* M) {
  if constexpr (V4) {
#pragma unroll
    for (int q = 0; q < N * N / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(M)[q];
      m[4 * q] = v.x, m[4 * q + 1] = v.y, m[4 * q + 2] = v.z, m[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < N * N; ++q) m[q] = M[q];
  }
}

// v[o + s i] <- sum_l m[i][l] v[o + s l], i < n (registers: o and s are compile-time after unrolling)
template <int N>
__device__ __forceinline__ void fdm_reg_line(const float* m, float* v, int o, int s) {
  float x[N];
#pragma unroll
  for (int l = 0; l < N; ++l) x[l] = v[o + s * l];
#pragma unroll
  for (int i = 0; i < N; ++i) {
    float y = 0.f;
#pragma unroll
    for (int l = 0; l < N; ++l) y = fmaf(m[i * N + l], x[l], y);
    v[o + s * i] = y;
  }
}

// plane c of a cell (u[a + n b] at c n^2) into / out of registers pl[a + n b]
template <int N, bool V4>
__device__ __forceinline__ void plane_in(float* pl, const float* u) {
  if constexpr (V4) {
#pragma unroll
    for (int q = 0; q < N * N / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(u)[q];
      pl[4 * q] = v.x, pl[4 * q + 1] = v.y, pl[4 * q + 2] = v.z, pl[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < N * N; ++q) pl[q] = u[q];
  }
}
template <int N, bool V4>
__device__ __forceinline__ void plane_out(const float* pl, float* u) {
  if constexpr (V4) {
#pragma unroll
    for (int q = 0; q < N * N / 4; ++q)
      reinterpret_cast<float4*>(u)[q] = make_float4(pl[4 * q], pl[4 * q + 1], pl[4 * q + 2], pl[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < N * N; ++q) u[q] = pl[q];
  }
}

// TIn = __half (even n only): r is a scaled FP16 vector (r_i = in_scale * h_i), the FGMRES basis row of the FP32
// inner solve; its cells arrive by 16-byte cp.async in a staging area RH [CB][n^3] after the tables and are
// converted as the first phase loads its planes.
// sub (may be null): the input is r - sub (the defect of a Gauss-Seidel sweep), sub an FP32 vector read as the
// planes are loaded (even n: 16-byte loads).
template <int N, typename TIn>
__global__ void __launch_bounds__(FdmPlanesR<N>::CB * N) fdm_apply_planes_real(const float* __restrict__ tab,
                                                                               const TIn* __restrict__ r,
                                                                               float in_scale,
                                                                               float* __restrict__ z, int64_t count,
                                                                               const int64_t* __restrict__ cells,
                                                                               const float* __restrict__ sub) {
  using P = FdmPlanesR<N>;
  constexpr int NN = P::NN, N3 = P::N3, UP = P::UP, TP = P::TP, AXP = RealLay<N>::AXP;
  constexpr bool V4 = P::V4, HIN = std::is_same<TIn, __half>::value;
  constexpr bool HSTAGE = HIN && N3 % 8 == 0 && NN % 4 == 0;  // FP16 input staged by 16-byte copies (even n)
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t s_cell[P::CB];
  float* U = reinterpret_cast<float*>(smem_raw);  // [CB][UP]: U[cell][a + n b + n^2 c]
  float* T = U + P::TOFF;                          // [CB][TP]
  __half* RH = reinterpret_cast<__half*>(T + P::CB * TP);  // FP16 input: [CB][N3]
  const int64_t q0 = (int64_t)blockIdx.x * P::CB;
  const int here = (int)min((int64_t)P::CB, count - q0);
  load_cells(s_cell, cells, q0, here);
  for (int e = threadIdx.x; e < here * (TP / 4); e += blockDim.x)  // tables: contiguous in group order
    cp_async16(T + 4 * e, tab + q0 * TP + 4 * e);
  __syncthreads();
  if constexpr (HSTAGE) {
    for (int e = threadIdx.x; e < here * (N3 / 8); e += blockDim.x) {
      const int l = e / (N3 / 8), q = e - l * (N3 / 8);
      cp_async16(RH + l * N3 + 8 * q, r + s_cell[l] * N3 + 8 * q);
    }
  } else if constexpr (HIN) {
    // odd n: the planes are read straight from global memory in the first phase
  } else if constexpr (N3 % 4 == 0) {
    for (int e = threadIdx.x; e < here * (N3 / 4); e += blockDim.x) {
      const int l = e / (N3 / 4), q = e - l * (N3 / 4);
      cp_async16(U + l * UP + 4 * q, r + s_cell[l] * N3 + 4 * q);
    }
  } else {
    for (int e = threadIdx.x; e < here * N3; e += blockDim.x) {
      const int l = e / N3, q = e - l * N3;
      cp_async(U + l * UP + q, r + s_cell[l] * N3 + q, 0);
    }
  }
  cp_async_wait_all();
  __syncthreads();
  const int lc = threadIdx.x / N, p = threadIdx.x - lc * N;
  const bool active = lc < here;
  float* u = U + lc * UP;
  const float* tb = T + lc * TP;
  float m[NN], v[NN];
  if (active) {  // plane c = p: W_x on its x-lines, W_y on its y-lines
    if constexpr (HIN && !HSTAGE) {
      const TIn* src = r + s_cell[lc] * N3 + p * NN;
#pragma unroll
      for (int q = 0; q < NN; ++q) v[q] = __half2float(src[q]) * in_scale;
    } else if constexpr (HIN) {
      const uint2* src = reinterpret_cast<const uint2*>(RH + lc * N3 + p * NN);  // 4 halves per 8-byte load
#pragma unroll
      for (int q = 0; q < NN / 4; ++q) {
        const uint2 w = src[q];
        const float2 f0 = __half22float2(*reinterpret_cast<const __half2*>(&w.x));
        const float2 f1 = __half22float2(*reinterpret_cast<const __half2*>(&w.y));
        v[4 * q] = f0.x * in_scale, v[4 * q + 1] = f0.y * in_scale;
        v[4 * q + 2] = f1.x * in_scale, v[4 * q + 3] = f1.y * in_scale;
      }
    } else {
      plane_in<N, V4>(v, u + p * NN);
    }
    if (sub) {
      float w[NN];
      plane_in<N, V4>(w, sub + s_cell[lc] * N3 + p * NN);
#pragma unroll
      for (int q = 0; q < NN; ++q) v[q] -= w[q];
    }
    fdm_load_r<N, V4>(m, tb);
#pragma unroll
    for (int b = 0; b < N; ++b) fdm_reg_line<N>(m, v, N * b, 1);
    fdm_load_r<N, V4>(m, tb + AXP);
#pragma unroll
    for (int a = 0; a < N; ++a) fdm_reg_line<N>(m, v, a, N);
    plane_out<N, V4>(v, u + p * NN);
  }
  __syncthreads();
  if (active) {  // z-lines (a, b = p): W_z, divide by lambda_x(a) + lambda_y(p) + lambda_z(c) + c |T|, V_z
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
      for (int a = 0; a < N; ++a) v[a + N * c] = u[a + N * p + NN * c];
    fdm_load_r<N, V4>(m, tb + 2 * AXP);
#pragma unroll
    for (int a = 0; a < N; ++a) fdm_reg_line<N>(m, v, a, N);
    const float lyc = tb[AXP + 2 * NN + p] + tb[3 * AXP];
#pragma unroll
    for (int c = 0; c < N; ++c) {
      const float lzc = tb[2 * AXP + 2 * NN + c] + lyc;
#pragma unroll
      for (int a = 0; a < N; ++a) v[a + N * c] /= tb[2 * NN + a] + lzc;
    }
    fdm_load_r<N, V4>(m, tb + 2 * AXP + NN);
#pragma unroll
    for (int a = 0; a < N; ++a) fdm_reg_line<N>(m, v, a, N);
#pragma unroll
    for (int c = 0; c < N; ++c)
#pragma unroll
      for (int a = 0; a < N; ++a) u[a + N * p + NN * c] = v[a + N * c];
  }
  __syncthreads();
  if (active) {  // plane c = p: V_y, V_x
    plane_in<N, V4>(v, u + p * NN);
    fdm_load_r<N, V4>(m, tb + AXP + NN);
#pragma unroll
    for (int a = 0; a < N; ++a) fdm_reg_line<N>(m, v, a, N);
    fdm_load_r<N, V4>(m, tb + NN);
#pragma unroll
    for (int b = 0; b < N; ++b) fdm_reg_line<N>(m, v, N * b, 1);
    plane_out<N, V4>(v, u + p * NN);
  }
  __syncthreads();
  if constexpr (N3 % 4 == 0) {
    for (int e = threadIdx.x; e < here * (N3 / 4); e += blockDim.x) {
      const int l = e / (N3 / 4), q = e - l * (N3 / 4);
      reinterpret_cast<float4*>(z + s_cell[l] * N3)[q] = reinterpret_cast<const float4*>(U + l * UP)[q];
    }
  } else {
    for (int e = threadIdx.x; e < here * N3; e += blockDim.x) {
      const int l = e / N3, q = e - l * N3;
      z[s_cell[l] * N3 + q] = U[l * UP + q];
    }
  }
}

// any n and precision: one thread per line (n^2 threads per cell), the pass matrices read from shared memory
template <int N, typename R>
__global__ void __launch_bounds__(256) fdm_apply_real(const R* __restrict__ tab, const R* __restrict__ r,
                                                      R* __restrict__ z, int64_t count,
                                                      const int64_t* __restrict__ cells, int cpb) {
  constexpr int NN = N * N, N3 = NN * N, TS = RealLay<N>::TP, AX = RealLay<N>::AXP;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ int64_t s_cell[64];
  R* U = reinterpret_cast<R*>(smem_raw);  // [cpb][N3]
  R* T = U + (size_t)cpb * N3;             // [cpb][TS]
  const int lc = threadIdx.x / NN, t = threadIdx.x - lc * NN;
  const int64_t q0 = (int64_t)blockIdx.x * cpb;
  const int here = (int)min((int64_t)cpb, count - q0);
  load_cells(s_cell, cells, q0, here);
  for (int e = threadIdx.x; e < here * TS; e += blockDim.x) T[e] = tab[q0 * TS + e];
  __syncthreads();
  for (int e = threadIdx.x; e < here * N3; e += blockDim.x) {
    const int l = e / N3;
    U[e] = r[s_cell[l] * N3 + (e - l * N3)];
  }
  __syncthreads();
  const bool active = lc < here;
  R* u = U + lc * N3;
  const R* tb = T + lc * TS;
  auto base = [&](int d) { return d == 0 ? N * t : (d == 1 ? (t % N) + NN * (t / N) : t); };
  auto stride = [](int d) { return d == 0 ? 1 : (d == 1 ? N : NN); };
  auto pass = [&](int d, const R* Mx) {
    if (active) {
      const int bs = base(d), st = stride(d);
      R x[N];
#pragma unroll
      for (int l = 0; l < N; ++l) x[l] = u[bs + l * st];
#pragma unroll
      for (int i = 0; i < N; ++i) {
        R y = R(0);
#pragma unroll
        for (int l = 0; l < N; ++l) y = fma(Mx[i * N + l], x[l], y);
        u[bs + i * st] = y;
      }
    }
    __syncthreads();
  };
  for (int d = 0; d < 3; ++d) pass(d, tb + d * AX);  // W_d
  if (active) {
    const int a = t % N, b = t / N;
    const R lab = tb[2 * NN + a] + tb[AX + 2 * NN + b] + tb[3 * AX];
#pragma unroll
    for (int c = 0; c < N; ++c) u[a + N * b + NN * c] /= lab + tb[2 * AX + 2 * NN + c];
  }
  __syncthreads();
  for (int d = 0; d < 3; ++d) pass(d, tb + d * AX + NN);  // V_d
  for (int e = threadIdx.x; e < here * N3; e += blockDim.x) {
    const int l = e / N3;
    z[s_cell[l] * N3 + (e - l * N3)] = U[e];
  }
}

namespace {

// 1D cell operator of axis r for cell `cell` (row = test function, column = trial function), from the 1D
// tables: volume D |T| / h^2 S - b_r |T| / h C, plus the self-coupling of the two faces across r (interior
// faces with the neighbours' D, or the side's boundary type), each times |F| = |T| / h
void cell_operator_1d(const dg_handle* h, const std::vector<double>& D, int64_t cell, int r,
                      const std::vector<double>& S, const std::vector<double>& C, const double* e0, const double* e1,
                      const double* d0, const double* d1, double* A) {
  const int n = h->N;
  const int ic[3] = {(int)(cell % h->n[0]), (int)((cell / h->n[0]) % h->n[1]),
                     (int)(cell / ((int64_t)h->n[0] * h->n[1]))};
  const int64_t strides[3] = {1, h->n[0], (int64_t)h->n[0] * h->n[1]};
  const double hr = h->h[r], vol = h->h[0] * h->h[1] * h->h[2], area = vol / hr, b = h->b[r], Dt = D[cell];
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) A[i * n + j] = vol * (Dt / (hr * hr) * S[i * n + j] - b / hr * C[i * n + j]);
  for (int side = 0; side < 2; ++side) {
    const bool at_end = side ? ic[r] == h->n[r] - 1 : ic[r] == 0;
    const bool boundary = at_end && !h->periodic[r];
    const double* ev = side ? e1 : e0;
    const double* dv = side ? d1 : d0;
    const double sgn = side ? 1.0 : -1.0;  // outward normal along axis r
    double up, cons, pen;  // coefficients of ev ev^T (upwind), (ev dv^T + dv ev^T) / h (consistency), ev ev^T
    if (boundary) {
      const int bt = h->bc_type[2 * r + side];
      const double bnu = sgn * b;
      up = (bt != DG_BC_NEUMANN && bnu >= 0.0) ? bnu : 0.0;
      cons = bt == DG_BC_DIRICHLET ? -sgn * Dt : 0.0;
      pen = bt == DG_BC_DIRICHLET ? Dt * h->sigma / hr : 0.0;
    } else {
      const int64_t wrap = (int64_t)(h->n[r] - 1) * strides[r];
      const int64_t nbr = side ? (at_end ? cell - wrap : cell + strides[r]) : (at_end ? cell + wrap : cell - strides[r]);
      const double Dn = D[nbr], w = Dn / (Dt + Dn);  // weight of the own side's flux
      up = side ? (b >= 0.0 ? b : 0.0) : (b < 0.0 ? -b : 0.0);
      cons = -sgn * w * Dt;
      pen = 2.0 * Dt * Dn / (Dt + Dn) * h->sigma / hr;
    }
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        A[i * n + j] += area * ((up + pen) * ev[i] * ev[j] + cons / hr * (ev[i] * dv[j] + dv[i] * ev[j]));
  }
}

}  // namespace

// the fast-diagonalisation tables of every cell (host, threads over cells); false if a 1D operator could not be
// diagonalised (the preconditioner then keeps the dense blocks).  Cells whose three 1D operators have real
// eigenvalues and real eigenvectors get is_real = 1 and the same tables in real arithmetic in `real` (same
// layout, one double per entry).
bool build_fdm(const dg_handle* h, const std::vector<double>& D, std::vector<double2>& tab, std::vector<double>& real,
               std::vector<uint8_t>& is_real) {
  const int n = h->N, M = h->M, NN = n * n, TS = 3 * (2 * NN + n) + 1;
  const Tables1D& t = h->tab;
  // theta_j and theta_j' at the points and at the ends, from the Lagrange tables (exact: degree <= k < M)
  std::vector<double> th(M * n), dth(M * n), S(n * n, 0.0), C(n * n, 0.0);
  double e0[MAXN], e1[MAXN], d0[MAXN], d1[MAXN];
  for (int j = 0; j < n; ++j) {
    for (int i = 0; i < M; ++i) {
      th[i * n + j] = t.A[i][j];
      double acc = 0.0;
      for (int l = 0; l < M; ++l) acc += t.Dt[i][l] * t.A[l][j];
      dth[i * n + j] = acc;
    }
    double v0 = 0, v1 = 0, g0 = 0, g1 = 0;
    for (int l = 0; l < M; ++l) {
      v0 += t.L[0][l] * t.A[l][j];
      v1 += t.L[1][l] * t.A[l][j];
      g0 += t.P[0][l] * t.A[l][j];
      g1 += t.P[1][l] * t.A[l][j];
    }
    e0[j] = v0, e1[j] = v1, d0[j] = g0, d1[j] = g1;
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      for (int q = 0; q < M; ++q) {
        S[i * n + j] += t.w[q] * dth[q * n + i] * dth[q * n + j];
        C[i * n + j] += t.w[q] * dth[q * n + i] * th[q * n + j];
      }
  tab.assign((size_t)h->ncell * TS, make_double2(0.0, 0.0));
  real.assign((size_t)h->ncell * TS, 0.0);
  is_real.assign(h->ncell, 1);
  const double cvol = h->c * h->h[0] * h->h[1] * h->h[2];
  const int nth = (int)std::max(1u, std::min(32u, std::thread::hardware_concurrency()));
  std::vector<int> ok(nth, 1);
  auto work = [&](int w) {
    std::vector<double> A(NN);
    std::vector<dge::cd> V(NN), W(NN), lam(n);
    for (int64_t cell = w; cell < h->ncell && ok[w]; cell += nth) {
      double2* o = &tab[(size_t)cell * TS];
      double* orl = &real[(size_t)cell * TS];
      for (int r = 0; r < 3; ++r) {
        cell_operator_1d(h, D, cell, r, S, C, e0, e1, d0, d1, A.data());
        if (!dge::eig_general(n, A.data(), V.data(), W.data(), lam.data())) {
          ok[w] = 0;
          break;
        }
        double2* b = o + r * (2 * NN + n);
        for (int e = 0; e < NN; ++e) {
          b[e] = make_double2(W[e].real(), W[e].imag());
          b[NN + e] = make_double2(V[e].real(), V[e].imag());
        }
        for (int e = 0; e < n; ++e) b[2 * NN + e] = make_double2(lam[e].real(), lam[e].imag());
        double* br = orl + r * (2 * NN + n);
        if (is_real[cell] && !dge::real_decomposition(n, V.data(), lam.data(), br + NN, br, br + 2 * NN))
          is_real[cell] = 0;
      }
      o[TS - 1] = make_double2(cvol, 0.0);
      orl[TS - 1] = cvol;
    }
  };
  std::vector<std::thread> pool;
  for (int w = 1; w < nth; ++w) pool.emplace_back(work, w);
  work(0);
  for (auto& th_ : pool) th_.join();
  for (int w = 0; w < nth; ++w)
    if (!ok[w]) return false;
  return true;
}

// one group of cells with real tables: the plane kernel in FP32 up to n = 8, else one thread per line
// sub (FP32, may be null): the plane kernel takes r - sub as its input (the caller guarantees even n <= 8 and
// 16-byte aligned vectors when it passes one)
template <typename R>
int fdm_group_real(const dg_handle* h, const R* tab, const int64_t* cells, int64_t count, const R* r, R* z,
                   cudaStream_t s, const float* sub = nullptr) {
  const int N = h->N, NN = N * N, cpb = std::max(1, 256 / NN), TS = 3 * ((2 * NN + N + 3) / 4 * 4) + 4;
  // the plane kernel moves r and z in 16-byte pieces for even n: other vectors take the line kernel
  const bool aligned = N % 2 == 1 || (reinterpret_cast<uintptr_t>(r) % 16 == 0 && reinterpret_cast<uintptr_t>(z) % 16 == 0 &&
                                      reinterpret_cast<uintptr_t>(sub) % 16 == 0);
  if (sub && !(sizeof(R) == 4 && N <= 8 && aligned)) {
    set_error("fast diagonalisation: a subtracted input needs the FP32 plane kernel");
    return DG_ERR_INVALID_ARG;
  }
  if constexpr (sizeof(R) == 4) {
    if (N <= 8 && aligned) {
      switch (N) {
#define FDMR(NV)                                                                                          \
  case NV: {                                                                                              \
    using P = FdmPlanesR<NV>;                                                                             \
    static DeviceOnce attr;                                                                               \
    if (P::SMEM > 48 * 1024) {                                                                            \
      if (int rca = attr.run([] {                                                                         \
            cudaError_t ea = cudaFuncSetAttribute(fdm_apply_planes_real<NV, float>,                       \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM);  \
            return ea == cudaSuccess ? 0 : cuda_fail(ea, "cudaFuncSetAttribute(fdm_apply_planes_real)");  \
          }))                                                                                             \
        return rca;                                                                                       \
    }                                                                                                     \
    fdm_apply_planes_real<NV, float><<<(unsigned)((count + P::CB - 1) / P::CB), P::CB * NV, P::SMEM, s>>>( \
        tab, r, 1.f, z, count, cells, sub);                                                               \
    break;                                                                                                \
  }
        FDMR(2) FDMR(3) FDMR(4) FDMR(5) FDMR(6) FDMR(7) FDMR(8)
#undef FDMR
      }
      cudaError_t e = cudaGetLastError();
      return e == cudaSuccess ? 0 : cuda_fail(e, "block-Jacobi apply (fast diagonalisation, real)");
    }
  }
  const size_t smem = (size_t)cpb * (N * NN + TS) * sizeof(R);
  const unsigned grid = (unsigned)((count + cpb - 1) / cpb);
  switch (N) {
#define FDMG(NV)                                                                                          \
  case NV:                                                                                                \
    if (smem > 48 * 1024) {                                                                               \
      static DeviceOnce attr;                                                                             \
      if (int rca = attr.run([&] {                                                                        \
            cudaError_t ea = cudaFuncSetAttribute(fdm_apply_real<NV, R>,                                  \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            return ea == cudaSuccess ? 0 : cuda_fail(ea, "cudaFuncSetAttribute(fdm_apply_real)");         \
          }))                                                                                             \
        return rca;                                                                                       \
    }                                                                                                     \
    fdm_apply_real<NV, R><<<grid, cpb * NN, smem, s>>>(tab, r, z, count, cells, cpb);                     \
    break;
    FDMG(2) FDMG(3) FDMG(4) FDMG(5) FDMG(6) FDMG(7) FDMG(8) FDMG(9) FDMG(10) FDMG(11)
#undef FDMG
    default:
      set_error("fast diagonalisation: unsupported degree");
      return DG_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "block-Jacobi apply (fast diagonalisation, real)");
}

// one group of cells with complex tables: the plane kernel in FP32 up to n = 6, else one thread per line
template <typename R>
int fdm_group_complex(const dg_handle* h, const typename Cx<R>::type* tab, const int64_t* cells, int64_t count,
                      const R* r, R* z, cudaStream_t s) {
  using C = typename Cx<R>::type;
  const int N = h->N, NN = N * N, cpb = std::max(1, 256 / NN), TS = 3 * (2 * NN + N) + 1;
  if constexpr (sizeof(R) == 4) {
    if (N <= 6) {
      switch (N) {
#define FDMP(NV)                                                                                          \
  case NV: {                                                                                              \
    using P = FdmPlanes<NV>;                                                                              \
    static DeviceOnce attr;                                                                               \
    if (P::SMEM > 48 * 1024) {                                                                            \
      if (int rca = attr.run([] {                                                                         \
            cudaError_t ea = cudaFuncSetAttribute(fdm_apply_planes<NV>,                                   \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM);  \
            return ea == cudaSuccess ? 0 : cuda_fail(ea, "cudaFuncSetAttribute(fdm_apply_planes)");       \
          }))                                                                                             \
        return rca;                                                                                       \
    }                                                                                                     \
    fdm_apply_planes<NV><<<(unsigned)((count + P::CB - 1) / P::CB), P::CB * NV, P::SMEM, s>>>(tab, r, z,  \
                                                                                           count, cells); \
    break;                                                                                                \
  }
        FDMP(2) FDMP(3) FDMP(4) FDMP(5) FDMP(6)
#undef FDMP
      }
      cudaError_t e = cudaGetLastError();
      return e == cudaSuccess ? 0 : cuda_fail(e, "block-Jacobi apply (fast diagonalisation)");
    }
  }
  const size_t smem = (size_t)cpb * (N * NN + TS) * sizeof(C);
  const unsigned grid = (unsigned)((count + cpb - 1) / cpb);
  switch (N) {
#define FDM(NV)                                                                                           \
  case NV:                                                                                                \
    if (smem > 48 * 1024) {                                                                               \
      static DeviceOnce attr;                                                                             \
      if (int rca = attr.run([&] {                                                                        \
            cudaError_t ea = cudaFuncSetAttribute(fdm_apply<NV, R>,                                       \
                                                  cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem); \
            return ea == cudaSuccess ? 0 : cuda_fail(ea, "cudaFuncSetAttribute(fdm_apply)");              \
          }))                                                                                             \
        return rca;                                                                                       \
    }                                                                                                     \
    fdm_apply<NV, R><<<grid, cpb * NN, smem, s>>>(tab, r, z, count, cells, cpb);                          \
    break;
    FDM(2) FDM(3) FDM(4) FDM(5) FDM(6) FDM(7) FDM(8) FDM(9) FDM(10) FDM(11)
#undef FDM
    default:
      set_error("fast diagonalisation: unsupported degree");
      return DG_ERR_INVALID_ARG;
  }
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "block-Jacobi apply (fast diagonalisation)");
}

// positions [lo, hi) of a group's cells for a colour (-1: all, 0: red, 1: black)
inline void color_range(int64_t n, int64_t nred, int color, int64_t* lo, int64_t* hi) {
  *lo = color == 1 ? nred : 0;
  *hi = color == 0 ? nred : n;
}

// z = A_TT^{-1} r on every cell of a colour (-1: every cell): the real group, then the complex group (disjoint
// cells); z is not written on the other cells
template <typename R>
int precond_fdm(const dg_handle* h, const R* r, R* z, cudaStream_t s, int color = -1) {
  using C = typename Cx<R>::type;
  const FdmTables& f = h->fdm;
  if (!f.built) {
    set_error("block-Jacobi: the fast diagonalisation was not set up");
    return DG_ERR_INVALID_ARG;
  }
  const int N = h->N, NN = N * N;
  const int64_t TPR = 3 * ((2 * NN + N + 3) / 4 * 4) + 4, TS = 3 * (2 * NN + N) + 1;
  int64_t lo, hi;
  color_range(f.nre, f.nre_red, color, &lo, &hi);
  if (hi > lo)
    if (int rc = fdm_group_real<R>(h, static_cast<const R*>(sizeof(R) == 4 ? f.re32 : f.re64) + lo * TPR,
                                   f.re_cells + lo, hi - lo, r, z, s))
      return rc;
  color_range(f.ncx, f.ncx_red, color, &lo, &hi);
  if (hi > lo)
    if (int rc = fdm_group_complex<R>(h, static_cast<const C*>(sizeof(R) == 4 ? f.cx32 : f.cx64) + lo * TS,
                                      f.cx_cells + lo, hi - lo, r, z, s))
      return rc;
  return 0;
}

int precond_fdm_f32(const dg_handle* h, const float* r, float* z, cudaStream_t s) { return precond_fdm(h, r, z, s); }


namespace {
// dst[c n^3 + i] = scale * src[c n^3 + i] for the listed cells (FP16 -> FP32)
__global__ void half_cells_to_float(const __half* __restrict__ src, float scale, const int64_t* __restrict__ cells,
                                    int64_t count, int n3, float* __restrict__ dst) {
  const int64_t total = count * n3;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / n3, i = e - q * n3, c = cells ? cells[q] : q;
    dst[c * n3 + i] = __half2float(src[c * n3 + i]) * scale;
  }
}

template <int N>
int fdm_real_half(const dg_handle* h, const float* tab, const int64_t* cells, int64_t count, const __half* r,
                  float scale, float* z, cudaStream_t s, const float* sub = nullptr) {
  using P = FdmPlanesR<N>;
  static DeviceOnce attr;
  if (P::SMEM_H > 48 * 1024)
    if (int rca = attr.run([] {
          cudaError_t ea = cudaFuncSetAttribute(fdm_apply_planes_real<N, __half>,
                                                cudaFuncAttributeMaxDynamicSharedMemorySize, P::SMEM_H);
          return ea == cudaSuccess ? 0 : cuda_fail(ea, "cudaFuncSetAttribute(fdm_apply_planes_real, FP16 input)");
        }))
      return rca;
  fdm_apply_planes_real<N, __half><<<(unsigned)((count + P::CB - 1) / P::CB), P::CB * N, P::SMEM_H, s>>>(
      tab, r, scale, z, count, cells, sub);
  return 0;
}
}  // namespace

// z = A_TT^{-1} (scale * r) for a scaled FP16 vector r (the FP16 basis rows of the inner solve).  The real group
// reads r directly (even n <= 8, 16-byte aligned r and z); the complex group and every other case first convert
// their entries into tmp (n FP32 values, 16-byte aligned) and take the FP32 path.
int precond_fdm_f32_half(const dg_handle* h, const __half* r, float scale, float* z, float* tmp, cudaStream_t s,
                         int color) {
  const FdmTables& f = h->fdm;
  if (!f.built) {
    set_error("block-Jacobi: the fast diagonalisation was not set up");
    return DG_ERR_INVALID_ARG;
  }
  const int N = h->N, N3 = N * N * N, NN = N * N;
  const int64_t TPR = 3 * ((2 * NN + N + 3) / 4 * 4) + 4, TS = 3 * (2 * NN + N) + 1;
  const bool direct = N <= 8 && (N % 2 == 1 || (reinterpret_cast<uintptr_t>(r) % 16 == 0 &&
                                                reinterpret_cast<uintptr_t>(z) % 16 == 0));
  if (!direct) {
    half_cells_to_float<<<sm_count() * 4, 256, 0, s>>>(r, scale, nullptr, h->ncell, N3, tmp);
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_fail(e, "FP16 row conversion");
    return precond_fdm(h, static_cast<const float*>(tmp), z, s, color);
  }
  int64_t lo, hi;
  color_range(f.nre, f.nre_red, color, &lo, &hi);
  if (hi > lo) {
    const float* tab = static_cast<const float*>(f.re32) + lo * TPR;
    const int64_t* cells = f.re_cells + lo;
    int rc = 0;
    switch (N) {
      case 2: rc = fdm_real_half<2>(h, tab, cells, hi - lo, r, scale, z, s); break;
      case 3: rc = fdm_real_half<3>(h, tab, cells, hi - lo, r, scale, z, s); break;
      case 4: rc = fdm_real_half<4>(h, tab, cells, hi - lo, r, scale, z, s); break;
      case 5: rc = fdm_real_half<5>(h, tab, cells, hi - lo, r, scale, z, s); break;
      case 6: rc = fdm_real_half<6>(h, tab, cells, hi - lo, r, scale, z, s); break;
      case 7: rc = fdm_real_half<7>(h, tab, cells, hi - lo, r, scale, z, s); break;
      default: rc = fdm_real_half<8>(h, tab, cells, hi - lo, r, scale, z, s); break;
    }
    if (rc) return rc;
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess)
      return cuda_fail(e, "block-Jacobi apply (fast diagonalisation, FP16 input)");
  }
  color_range(f.ncx, f.ncx_red, color, &lo, &hi);
  if (hi > lo) {
    half_cells_to_float<<<sm_count() * 4, 256, 0, s>>>(r, scale, f.cx_cells + lo, hi - lo, N3, tmp);
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_fail(e, "FP16 row conversion");
    if (int rc = fdm_group_complex<float>(h, static_cast<const float2*>(f.cx32) + lo * TS, f.cx_cells + lo, hi - lo,
                                          tmp, z, s))
      return rc;
  }
  return 0;
}

// ---------------------------------------------------------------------------------------------
// Red-black block Gauss-Seidel: with the cells coloured by the parity of ix + iy + iz, the face neighbours of a
// red cell are black and vice versa (on a periodic axis with an odd cell count the two cells across the wrap
// share a colour, and their coupling is then treated as in block-Jacobi).  One application is the exact solve
// with the block lower-triangular part of A in red-before-black order:
//   z_red = A_rr^{-1} r_red,   z_black = A_bb^{-1} (r - A z_red)_black,
// with the diagonal blocks inverted by fast diagonalisation and A z_red the operator itself applied to z (zero on
// the black cells).  t: scratch vector of n values.  In FP32 with even n <= 8 and 16-byte aligned vectors the
// black cells' defect r - A z_red is formed inside the block-inverse kernel as it loads its planes (real cells)
// or for the listed cells only (complex cells); otherwise by a separate pass over the vector.
// ---------------------------------------------------------------------------------------------
namespace {
template <typename R>
__global__ void __launch_bounds__(256) rbgs_defect(const R* __restrict__ r, R* __restrict__ t, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    t[i] = r[i] - t[i];
}
__global__ void __launch_bounds__(256) rbgs_defect_half(const __half* __restrict__ r, float scale,
                                                        float* __restrict__ t, size_t n) {
  for (size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    t[i] = __half2float(r[i]) * scale - t[i];
}
// t = scale * r - t on the listed cells only
template <typename TIn>
__global__ void __launch_bounds__(256) rbgs_defect_cells(const TIn* __restrict__ r, float scale,
                                                         const int64_t* __restrict__ cells, int64_t count, int n3,
                                                         float* __restrict__ t) {
  const int64_t total = count * n3;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t q = e / n3, i = cells[q] * n3 + (e - q * n3);
    t[i] = (float)r[i] * scale - t[i];
  }
}

template <typename R>
int rbgs_apply_A(const dg_handle* h, const R* z, R* t, cudaStream_t s) {
  if constexpr (sizeof(R) == 4)
    return launch_apply_f32(h, z, t, 0, 3, s);
  else
    return launch_apply_f64(h, z, t, 0, 3, s);
}

inline bool al16(const void* p) { return reinterpret_cast<uintptr_t>(p) % 16 == 0; }

// black cells from r - t (t = A z_red on entry; overwritten) with the defect fused (FP32, even n <= 8, aligned;
// r FP32 or scaled FP16)
template <typename TIn>
int rbgs_black_fused(const dg_handle* h, const TIn* r, float scale, float* z, float* t, cudaStream_t s) {
  const FdmTables& f = h->fdm;
  const int N = h->N, NN = N * N, N3 = NN * N;
  const int64_t TPR = 3 * ((2 * NN + N + 3) / 4 * 4) + 4, TS = 3 * (2 * NN + N) + 1;
  if (f.nre > f.nre_red) {
    const float* tab = static_cast<const float*>(f.re32) + f.nre_red * TPR;
    const int64_t* cells = f.re_cells + f.nre_red;
    const int64_t cnt = f.nre - f.nre_red;
    int rc = 0;
    if constexpr (std::is_same<TIn, __half>::value) {
      switch (N) {
        case 2: rc = fdm_real_half<2>(h, tab, cells, cnt, r, scale, z, s, t); break;
        case 3: rc = fdm_real_half<3>(h, tab, cells, cnt, r, scale, z, s, t); break;
        case 4: rc = fdm_real_half<4>(h, tab, cells, cnt, r, scale, z, s, t); break;
        case 5: rc = fdm_real_half<5>(h, tab, cells, cnt, r, scale, z, s, t); break;
        case 6: rc = fdm_real_half<6>(h, tab, cells, cnt, r, scale, z, s, t); break;
        case 7: rc = fdm_real_half<7>(h, tab, cells, cnt, r, scale, z, s, t); break;
        default: rc = fdm_real_half<8>(h, tab, cells, cnt, r, scale, z, s, t); break;
      }
      if (!rc)
        if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) rc = cuda_fail(e, "red-black Gauss-Seidel (black)");
    } else {
      rc = fdm_group_real<float>(h, tab, cells, cnt, r, z, s, t);
    }
    if (rc) return rc;
  }
  if (f.ncx > f.ncx_red) {
    const int64_t* cells = f.cx_cells + f.ncx_red;
    const int64_t cnt = f.ncx - f.ncx_red;
    rbgs_defect_cells<TIn><<<sm_count() * 4, 256, 0, s>>>(r, scale, cells, cnt, N3, t);
    if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_fail(e, "red-black Gauss-Seidel (defect)");
    if (int rc = fdm_group_complex<float>(h, static_cast<const float2*>(f.cx32) + f.ncx_red * TS, cells, cnt, t, z, s))
      return rc;
  }
  return 0;
}

// In FP32 at degree 5 the operator runs on the red cells and writes the black ones only (launch_offdiag_f32), so
// z needs no clearing; otherwise z is cleared and the whole operator applied.
template <typename R, typename First, typename Defect>
int rbgs_sweep(const dg_handle* h, R* z, R* t, cudaStream_t s, First first, Defect defect_then_black) {
  const FdmTables& f = h->fdm;
  if (!f.built) {
    set_error("red-black Gauss-Seidel: dg_precond_setup was not called");
    return DG_ERR_INVALID_ARG;
  }
  const size_t n = (size_t)h->ncell * h->N * h->N * h->N;
  const bool offdiag = sizeof(R) == 4 && has_offdiag_f32(h);
  if (!offdiag) {
    cudaError_t e = cudaMemsetAsync(z, 0, n * sizeof(R), s);
    if (e != cudaSuccess) return cuda_fail(e, "red-black Gauss-Seidel: clear z");
  }
  if (int rc = first()) return rc;
  if constexpr (sizeof(R) == 4) {
    if (offdiag) {
      if (int rc = launch_offdiag_f32(h, z, t, f.red32, f.nred, f.black32, f.nblack, s)) return rc;
      return defect_then_black(n);
    }
  }
  if (int rc = rbgs_apply_A<R>(h, z, t, s)) return rc;
  return defect_then_black(n);
}
}  // namespace

int precond_rbgs_f32(const dg_handle* h, const float* r, float* z, float* t, cudaStream_t s) {
  const int N = h->N;
  const bool fused = N <= 8 && (N % 2 == 1 || (al16(r) && al16(z) && al16(t)));
  return rbgs_sweep<float>(
      h, z, t, s, [&] { return precond_fdm<float>(h, r, z, s, 0); },
      [&](size_t n) -> int {
        if (fused) return rbgs_black_fused<float>(h, r, 1.f, z, t, s);
        rbgs_defect<float><<<sm_count() * 4, 256, 0, s>>>(r, t, n);
        if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_fail(e, "red-black Gauss-Seidel");
        return precond_fdm<float>(h, t, z, s, 1);
      });
}
int precond_rbgs_f64(const dg_handle* h, const double* r, double* z, double* t, cudaStream_t s) {
  return rbgs_sweep<double>(
      h, z, t, s, [&] { return precond_fdm<double>(h, r, z, s, 0); },
      [&](size_t n) -> int {
        rbgs_defect<double><<<sm_count() * 4, 256, 0, s>>>(r, t, n);
        if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_fail(e, "red-black Gauss-Seidel");
        return precond_fdm<double>(h, t, z, s, 1);
      });
}
int precond_rbgs_f32_half(const dg_handle* h, const __half* r, float scale, float* z, float* t, float* tmp,
                          cudaStream_t s) {
  const int N = h->N;
  const bool fused = N <= 8 && (N % 2 == 1 || (al16(r) && al16(z) && al16(t)));
  return rbgs_sweep<float>(
      h, z, t, s, [&] { return precond_fdm_f32_half(h, r, scale, z, tmp, s, 0); },
      [&](size_t n) -> int {
        if (fused) return rbgs_black_fused<__half>(h, r, scale, z, t, s);
        rbgs_defect_half<<<sm_count() * 4, 256, 0, s>>>(r, scale, t, n);
        if (cudaError_t e = cudaGetLastError(); e != cudaSuccess) return cuda_fail(e, "red-black Gauss-Seidel");
        return precond_fdm<float>(h, t, z, s, 1);
      });
}

// ---------------------------------------------------------------------------------------------
// Gauss-Seidel sweep and operator together (Eisenstat's form).  With the blocks ordered red before black and a
// two-cyclic colouring, A = D + L + U where D is block diagonal, L = A_br (black rows, red columns) and U = A_rb;
// the sweep is M = D + L, so for z = M^{-1} u:
//   A z = (M + U) z = u + U z,
// and U z is the operator restricted to the red rows and the black columns (launch_offdiag_f32 from the black
// cells to the red ones).  So the Krylov step's operator application costs half an operator.  The block
// inverses are exact up to FP32 rounding, so the identity holds to that level; the flexible outer method
// absorbs it like any other inexactness of the inner solve.
// ---------------------------------------------------------------------------------------------
namespace {
// w = scale * u + (red cell ? w : 0), w holding (U z) on the red cells on entry.  One warp per cell (its colour
// computed once), packs of 4 values (n^3 a multiple of 4, 16-byte aligned vectors)
template <typename TU, bool VEC>
__global__ void __launch_bounds__(256) eisenstat_combine(const TU* __restrict__ u, float scale, float* __restrict__ w,
                                                         int64_t ncell, int n3, int nx, int ny) {
  const int lane = threadIdx.x & 31, np = n3 >> 2;
  for (int64_t c = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; c < ncell;
       c += ((int64_t)gridDim.x * blockDim.x) >> 5) {
    const int64_t ix = c % nx, iy = (c / nx) % ny, iz = c / ((int64_t)nx * ny);
    const bool red = ((ix + iy + iz) & 1) == 0;
    if constexpr (!VEC) {  // n^3 not a multiple of 4: one value per lane and step
      for (int q = lane; q < n3; q += 32) {
        const int64_t i = c * n3 + q;
        w[i] = fmaf((float)u[i], scale, red ? w[i] : 0.f);
      }
      continue;
    }
    float4* wc = reinterpret_cast<float4*>(w + c * n3);
    for (int q = lane; q < np; q += 32) {
      float4 uv;
      if constexpr (std::is_same<TU, __half>::value) {
        const uint2 raw = reinterpret_cast<const uint2*>(u + c * n3)[q];
        const float2 a = __half22float2(*reinterpret_cast<const __half2*>(&raw.x));
        const float2 b = __half22float2(*reinterpret_cast<const __half2*>(&raw.y));
        uv = make_float4(a.x, a.y, b.x, b.y);
      } else {
        uv = reinterpret_cast<const float4*>(u + c * n3)[q];
      }
      float4 r = red ? wc[q] : make_float4(0.f, 0.f, 0.f, 0.f);
      r.x = fmaf(uv.x, scale, r.x);
      r.y = fmaf(uv.y, scale, r.y);
      r.z = fmaf(uv.z, scale, r.z);
      r.w = fmaf(uv.w, scale, r.w);
      wc[q] = r;
    }
  }
}
}  // namespace

// degree 5 only: there the plane kernels are the faster FP32 operator, so half of one beats a whole apply; at
// degree 4 a one-colour plane apply plus the addition pass cost as much as the whole line-kernel apply (measured:
// the 64^3 Q4 solve with the FP32 basis took 1.91 s with it, 1.85 s without)
bool has_rbgs_eisenstat(const dg_handle* h) { return h->fdm.built && h->fdm.two_cyclic && h->N == 6 && has_offdiag_f32(h); }

int precond_rbgs_eisenstat_f32(const dg_handle* h, const float* u, float* z, float* w, float* t, cudaStream_t s) {
  if (int rc = precond_rbgs_f32(h, u, z, t, s)) return rc;
  const FdmTables& f = h->fdm;
  if (int rc = launch_offdiag_f32(h, z, w, f.black32, f.nblack, f.red32, f.nred, s)) return rc;
  const size_t n = (size_t)h->ncell * h->N * h->N * h->N;
  const int n3 = (int)(n / h->ncell);
  if (n3 % 4 == 0 && al16(u) && al16(w))
    eisenstat_combine<float, true><<<sm_count() * 8, 256, 0, s>>>(u, 1.f, w, h->ncell, n3, h->n[0], h->n[1]);
  else
    eisenstat_combine<float, false><<<sm_count() * 8, 256, 0, s>>>(u, 1.f, w, h->ncell, n3, h->n[0], h->n[1]);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "Gauss-Seidel operator combination");
}

int precond_rbgs_eisenstat_f32_half(const dg_handle* h, const __half* u, float scale, float* z, float* w, float* t,
                                    float* tmp, cudaStream_t s) {
  if (int rc = precond_rbgs_f32_half(h, u, scale, z, t, tmp, s)) return rc;
  const FdmTables& f = h->fdm;
  if (int rc = launch_offdiag_f32(h, z, w, f.black32, f.nblack, f.red32, f.nred, s)) return rc;
  const size_t n = (size_t)h->ncell * h->N * h->N * h->N;
  const int n3 = (int)(n / h->ncell);
  if (n3 % 4 == 0 && reinterpret_cast<uintptr_t>(u) % 8 == 0 && al16(w))
    eisenstat_combine<__half, true><<<sm_count() * 8, 256, 0, s>>>(u, scale, w, h->ncell, n3, h->n[0], h->n[1]);
  else
    eisenstat_combine<__half, false><<<sm_count() * 8, 256, 0, s>>>(u, scale, w, h->ncell, n3, h->n[0], h->n[1]);
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "Gauss-Seidel operator combination");
}

int precond_bj_f16(const dg_handle* h, const float* r, float* z, cudaStream_t s) {
  if (!h->bj16) return precond_fdm(h, r, z, s);
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
  if (!h->bj64) return precond_fdm(h, r, z, s);  // set up with the fast diagonalisation only
  const int n = h->N * h->N * h->N;
  const int threads = n >= 256 ? 256 : ((n + 31) / 32) * 32;
  bj_apply<double><<<(unsigned)h->ncell, threads, n * sizeof(double), s>>>(static_cast<const double*>(h->bj64), r, z, n);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "block-Jacobi apply");
}

int precond_bj_f32(const dg_handle* h, const float* r, float* z, cudaStream_t s) {
  if (!h->bj32) return precond_fdm(h, r, z, s);
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

namespace {
// the fast-diagonalisation tables of every cell (FP32 and FP64; real for the cells that allow it, complex for the
// others, each group with its list of cells); DG_ERR_NAN if a 1D cell operator could not be diagonalised
int setup_fdm(dg_handle* h) {
  if (h->fdm.built) return DG_OK;
  std::vector<double> Dh(h->ncell);
  cudaError_t e = cudaMemcpy(Dh.data(), h->p64.D, h->ncell * sizeof(double), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_fail(e, "fast diagonalisation: D");
  std::vector<double2> tab;
  std::vector<double> real;
  std::vector<uint8_t> is_real;
  if (!build_fdm(h, Dh, tab, real, is_real)) {
    set_error("dg_precond_setup: a 1D cell operator could not be diagonalised");
    return DG_ERR_NAN;
  }
  const int N = h->N, NN = N * N, AX = 2 * NN + N, TS = 3 * AX + 1;
  const int AXP = (AX + 3) / 4 * 4, TP = 3 * AXP + 4;  // the padded layout of the real kernels
  // groups: real / complex cells, each red (ix + iy + iz even) first, then black, ascending within a colour
  std::vector<int64_t> re_cells, cx_cells;
  int64_t nre_red = 0, ncx_red = 0;
  for (int color = 0; color < 2; ++color) {
    for (int64_t c = 0; c < h->ncell; ++c) {
      const int64_t ix = c % h->n[0], iy = (c / h->n[0]) % h->n[1], iz = c / ((int64_t)h->n[0] * h->n[1]);
      if ((int)((ix + iy + iz) & 1) != color) continue;
      (is_real[c] ? re_cells : cx_cells).push_back(c);
    }
    if (color == 0) {
      nre_red = (int64_t)re_cells.size();
      ncx_red = (int64_t)cx_cells.size();
    }
  }
  const int64_t nre = (int64_t)re_cells.size(), ncx = (int64_t)cx_cells.size();
  // group tables in group order; real ones with each axis block (W, V, lambda) padded to AXP entries
  std::vector<double> re64((size_t)nre * TP, 0.0);
  std::vector<float> re32((size_t)nre * TP, 0.f);
  for (int64_t q = 0; q < nre; ++q) {
    const double* src = &real[(size_t)re_cells[q] * TS];
    double* dst = &re64[(size_t)q * TP];
    for (int ax = 0; ax < 3; ++ax)
      for (int i = 0; i < AX; ++i) dst[ax * AXP + i] = src[ax * AX + i];
    dst[3 * AXP] = src[TS - 1];
    for (int i = 0; i < TP; ++i) re32[(size_t)q * TP + i] = (float)dst[i];
  }
  std::vector<double2> cx64((size_t)ncx * TS);
  std::vector<float2> cx32((size_t)ncx * TS);
  for (int64_t q = 0; q < ncx; ++q)
    for (int i = 0; i < TS; ++i) {
      const double2 v = tab[(size_t)cx_cells[q] * TS + i];
      cx64[(size_t)q * TS + i] = v;
      cx32[(size_t)q * TS + i] = make_float2((float)v.x, (float)v.y);
    }
  FdmTables f;
  f.nre = nre;
  f.ncx = ncx;
  f.nre_red = nre_red;
  f.ncx_red = ncx_red;
  auto up = [&](void** dst, const void* src, size_t bytes) {
    if (e != cudaSuccess || bytes == 0) return;
    e = cudaMalloc(dst, bytes);
    if (e == cudaSuccess) e = cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice);
  };
  up(&f.re32, re32.data(), re32.size() * sizeof(float));
  up(&f.re64, re64.data(), re64.size() * sizeof(double));
  up(&f.cx32, cx32.data(), cx32.size() * sizeof(float2));
  up(&f.cx64, cx64.data(), cx64.size() * sizeof(double2));
  up(reinterpret_cast<void**>(&f.re_cells), re_cells.data(), re_cells.size() * sizeof(int64_t));
  up(reinterpret_cast<void**>(&f.cx_cells), cx_cells.data(), cx_cells.size() * sizeof(int64_t));
  std::vector<int> reds, blacks;
  for (int64_t c = 0; c < h->ncell; ++c) {
    const int64_t ix = c % h->n[0], iy = (c / h->n[0]) % h->n[1], iz = c / ((int64_t)h->n[0] * h->n[1]);
    ((ix + iy + iz) & 1 ? blacks : reds).push_back((int)c);
  }
  f.nred = (int64_t)reds.size();
  f.nblack = (int64_t)blacks.size();
  f.two_cyclic = true;
  for (int r = 0; r < 3; ++r)
    if (h->periodic[r] && (h->n[r] & 1)) f.two_cyclic = false;
  up(reinterpret_cast<void**>(&f.red32), reds.data(), reds.size() * sizeof(int));
  up(reinterpret_cast<void**>(&f.black32), blacks.data(), blacks.size() * sizeof(int));
  if (e != cudaSuccess) {
    for (void* q : {f.re32, f.re64, f.cx32, f.cx64, (void*)f.re_cells, (void*)f.cx_cells, (void*)f.red32,
                    (void*)f.black32})
      cudaFree(q);
    return cuda_fail(e, "fast diagonalisation tables");
  }
  f.built = true;
  h->fdm = f;
  return DG_OK;
}
}  // namespace

int dg_precond_setup(dg_handle* h, int32_t kind, void* stream) {
  if (!h || (kind != DG_BJ_DENSE && kind != DG_BJ_FAST_DIAG)) {
    set_error("dg_precond_setup: kind must be DG_BJ_DENSE (1) or DG_BJ_FAST_DIAG (2)");
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
  if (kind == DG_BJ_FAST_DIAG) {
    const cudaError_t e0 = cudaStreamSynchronize(s);
    if (e0 != cudaSuccess) return cuda_fail(e0, "dg_precond_setup synchronize");
    return setup_fdm(h);
  }
  if (n > 512) {
    set_error("dg_precond_setup: dense block-Jacobi supports (k+1)^3 <= 512");
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
      cast_blocks<<<sm_count() * 8, 256, 0, s>>>(static_cast<const double*>(h->bj64), static_cast<float*>(h->bj32), h->ncell,
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
  if (rc == DG_OK && !bad) {
    // also the exact block inverse by fast diagonalisation for FP32 applies (kept only if every cell's 1D
    // operators could be diagonalised; otherwise the FP32 applies use the dense blocks)
    const int frc = setup_fdm(h);
    if (frc == DG_ERR_CUDA || frc == DG_ERR_OOM) rc = frc;
  }
  if (rc == DG_OK && bad) {
    set_error("dg_precond_setup: " + std::to_string(bad) + " singular diagonal block(s)");
    rc = DG_ERR_NAN;
  }
  return rc;
}

int dg_precond_info(const dg_handle* h, int32_t* info, int64_t* complex_cells) {
  if (!h || !info) {
    set_error("dg_precond_info: null handle or output");
    return DG_ERR_INVALID_ARG;
  }
  *info = (h->bj64 ? DG_PRECOND_HAS_DENSE : 0) | (h->fdm.built ? DG_PRECOND_HAS_FAST_DIAG : 0) |
          (h->fdm.built && h->fdm.ncx == 0 ? DG_PRECOND_FAST_DIAG_REAL : 0);
  if (complex_cells) *complex_cells = h->fdm.built ? h->fdm.ncx : 0;
  return DG_OK;
}

int dg_precond_apply_rbgs(dg_handle* h, const void* r, void* z, void* work, int32_t precision, void* stream) {
  if (!h || !r || !z || !work || r == z || r == work || z == work || (precision != DG_F64 && precision != DG_F32)) {
    set_error("dg_precond_apply_rbgs: bad arguments (r, z, work distinct device vectors; DG_F64 or DG_F32)");
    return DG_ERR_INVALID_ARG;
  }
  if (!h->fdm.built) {
    set_error("dg_precond_apply_rbgs: call dg_precond_setup first");
    return DG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == DG_F64)
    return precond_rbgs_f64(h, static_cast<const double*>(r), static_cast<double*>(z), static_cast<double*>(work), s);
  return precond_rbgs_f32(h, static_cast<const float*>(r), static_cast<float*>(z), static_cast<float*>(work), s);
}

int dg_precond_apply(dg_handle* h, const void* r, void* z, int32_t precision, void* stream) {
  if (!h || !r || !z || r == z || (precision != DG_F64 && precision != DG_F32)) {
    set_error("dg_precond_apply: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  if (!h->bj64 && !h->fdm.built) {
    set_error("dg_precond_apply: call dg_precond_setup first");
    return DG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (precision == DG_F64) return precond_bj_f64(h, static_cast<const double*>(r), static_cast<double*>(z), s);
  // FP32: the exact block inverse by fast diagonalisation when it was built, else the FP32 dense blocks
  if (h->fdm.built) return precond_fdm_f32(h, static_cast<const float*>(r), static_cast<float*>(z), s);
  return precond_bj_f32(h, static_cast<const float*>(r), static_cast<float*>(z), s);
}

}  // extern "C"
