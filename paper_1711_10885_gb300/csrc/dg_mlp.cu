// dg_mlp.cu -- per-element MLP preconditioner: feature gather, fused BF16 tensor-core forward pass,
// backward pass on the tensor cores (BF16 operands, FP32 accumulation), Adam, and the preconditioner
// application z = M(r) used inside FGMRES.
//
// Network (per cell T): x = [r_T / s, log D_T, log D of the 6 face neighbours (own value where there is
// no neighbour)], s = ||r_T||_2;  h1 = relu(W1 x + b1), h2 = relu(W2 h1 + b2), y = W3 h2 + b3 (256 hidden
// units each); the correction is z_T = s * t_scale * y.  Weights are kept in FP32 (master copy, Adam
// moments) and rounded to BF16 for the forward GEMMs; accumulation is FP32.
#include <cmath>
#include <cstdlib>
#include <cstdio>
#include <cstring>
#include <random>
#include <string>
#include <vector>

#include <cuda_bf16.h>

#include "dg_internal.h"

namespace dgm {

constexpr int HID = 256;
constexpr int ROWS = 64;      // rows (cells) per CTA in the forward kernel
constexpr int FWD_THREADS = 256;

struct Dims {
  int nb;    // (k+1)^3
  int kin;   // nb + 7
  int kinp;  // kin rounded up to 16
  int outp;  // nb rounded up to 16
};

inline Dims dims_for(int k) {
  Dims d;
  d.nb = (k + 1) * (k + 1) * (k + 1);
  d.kin = d.nb + 7;
  d.kinp = (d.kin + 15) / 16 * 16;
  d.outp = (d.nb + 15) / 16 * 16;
  return d;
}

__device__ __forceinline__ void mma_bf16(float (&c)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
  return *reinterpret_cast<uint32_t*>(&v);
}

// One warp computes a 16 x (8 * NT) block of C = A(16 x K, shared memory, row stride lda elements)
// times W^T (W: row-major [n][K] in global memory, rows n0 .. n0 + 8 NT - 1).
template <int NT>
__device__ __forceinline__ void warp_gemm(const __nv_bfloat16* As, int lda, const __nv_bfloat16* __restrict__ W,
                                          int ldw, int n0, int K, float (&acc)[NT][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
#pragma unroll
  for (int j = 0; j < NT; ++j) acc[j][0] = acc[j][1] = acc[j][2] = acc[j][3] = 0.f;
  for (int k0 = 0; k0 < K; k0 += 16) {
    uint32_t a[4];
    a[0] = *reinterpret_cast<const uint32_t*>(As + g * lda + k0 + tig * 2);
    a[1] = *reinterpret_cast<const uint32_t*>(As + (g + 8) * lda + k0 + tig * 2);
    a[2] = *reinterpret_cast<const uint32_t*>(As + g * lda + k0 + 8 + tig * 2);
    a[3] = *reinterpret_cast<const uint32_t*>(As + (g + 8) * lda + k0 + 8 + tig * 2);
#pragma unroll
    for (int j = 0; j < NT; ++j) {
      const __nv_bfloat16* wr = W + (size_t)(n0 + 8 * j + g) * ldw + k0 + tig * 2;
      const uint32_t b0 = __ldg(reinterpret_cast<const unsigned int*>(wr));
      const uint32_t b1 = __ldg(reinterpret_cast<const unsigned int*>(wr + 8));
      mma_bf16(acc[j], a, b0, b1);
    }
  }
}

struct FwdArgs {
  const __nv_bfloat16* X;  // [rows][kinp]
  const __nv_bfloat16* W1; // [HID][kinp]
  const float* b1;
  const __nv_bfloat16* W2; // [HID][HID]
  const float* b2;
  const __nv_bfloat16* W3; // [outp][HID]
  const float* b3;
  __nv_bfloat16* H1;       // optional [rows][HID] (training)
  __nv_bfloat16* H2;       // optional [rows][HID]
  float* Y;                // optional [rows][outp]
  // preconditioner output (optional): z[cell * nb + j] = scale[row] * y[row][j]
  const float* scale;
  void* z;
  int z_is_f64;
  int z_accumulate;  // z += ... instead of z = ...
  int64_t rows;
  int kinp, outp, nb;
  // tcgen05 kernel: W1, W2, W3 pre-packed in the canonical shared-memory layout (see pack_canonical)
  const __nv_bfloat16* W1p;
  const __nv_bfloat16* W2p;
  const __nv_bfloat16* W3p;
  uint32_t w_wait_tries;  // tcgen05 kernel: polls of the weight-arrival wait before it counts as timed out
};

// Output layer on 8 NT columns starting at c0 for this warp's 16 rows, with the bias and either the
// raw output Y or the scaled preconditioner output z.
template <int NT>
__device__ __forceinline__ void layer3_chunk(const FwdArgs& a, const __nv_bfloat16* As, int lda, int c0, int rA,
                                             int rB, int64_t row0, int here) {
  const int tig = (threadIdx.x & 31) & 3;
  float acc[NT][4];
  warp_gemm<NT>(As, lda, a.W3, HID, c0, HID, acc);
#pragma unroll
  for (int j = 0; j < NT; ++j) {
    const int col = c0 + 8 * j + 2 * tig;
    const float y0 = acc[j][0] + a.b3[col], y1 = acc[j][1] + a.b3[col + 1];
    const float y2 = acc[j][2] + a.b3[col], y3 = acc[j][3] + a.b3[col + 1];
    if (a.Y) {
      if (rA < here) {
        a.Y[(row0 + rA) * a.outp + col] = y0;
        a.Y[(row0 + rA) * a.outp + col + 1] = y1;
      }
      if (rB < here) {
        a.Y[(row0 + rB) * a.outp + col] = y2;
        a.Y[(row0 + rB) * a.outp + col + 1] = y3;
      }
    }
    if (a.z) {
      const float vals[4] = {y0, y1, y2, y3};
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = q < 2 ? rA : rB, cc = col + (q & 1);
        if (r < here && cc < a.nb) {
          const float v = a.scale[row0 + r] * vals[q];
          const size_t zi = (size_t)(row0 + r) * a.nb + cc;
          if (a.z_is_f64) {
            double* zp = static_cast<double*>(a.z) + zi;
            *zp = a.z_accumulate ? *zp + (double)v : (double)v;
          } else {
            float* zp = static_cast<float*>(a.z) + zi;
            *zp = a.z_accumulate ? *zp + v : v;
          }
        }
      }
    }
  }
}

// Fused 3-layer forward pass for 64 rows per CTA: 8 warps = 4 row tiles x 2 column halves.
__global__ void __launch_bounds__(FWD_THREADS) mlp_forward(const FwdArgs a) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int ldx = a.kinp + 8, ldh = HID + 8;
  __nv_bfloat16* Xs = reinterpret_cast<__nv_bfloat16*>(smem_raw);
  __nv_bfloat16* H1s = Xs + ROWS * ldx;
  __nv_bfloat16* H2s = H1s + ROWS * ldh;
  const int64_t row0 = (int64_t)blockIdx.x * ROWS;
  const int here = (int)min((int64_t)ROWS, a.rows - row0);
  // stage X (rows beyond `here` are zero)
  for (int e = threadIdx.x; e < ROWS * a.kinp / 2; e += blockDim.x) {
    const int r = e / (a.kinp / 2), c2 = e - r * (a.kinp / 2);
    uint32_t v = 0;
    if (r < here) v = *reinterpret_cast<const uint32_t*>(a.X + (row0 + r) * a.kinp + 2 * c2);
    *reinterpret_cast<uint32_t*>(Xs + r * ldx + 2 * c2) = v;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  const int mt = warp & 3, nh = warp >> 2;
  const int rA = 16 * mt + g, rB = rA + 8;
  // layer 1 and 2: 16 x 128 per warp
#pragma unroll 1
  for (int layer = 0; layer < 2; ++layer) {
    const __nv_bfloat16* As = layer == 0 ? Xs : H1s;
    const int lda = layer == 0 ? ldx : ldh;
    const int K = layer == 0 ? a.kinp : HID;
    const __nv_bfloat16* W = layer == 0 ? a.W1 : a.W2;
    const float* bias = layer == 0 ? a.b1 : a.b2;
    __nv_bfloat16* Hs = layer == 0 ? H1s : H2s;
    __nv_bfloat16* Hg = layer == 0 ? a.H1 : a.H2;
    float acc[16][4];
    warp_gemm<16>(As + 16 * mt * lda, lda, W, K, 128 * nh, K, acc);
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int col = 128 * nh + 8 * j + 2 * tig;
      const float bb0 = bias[col], bb1 = bias[col + 1];
      const uint32_t lo = pack_bf16(fmaxf(acc[j][0] + bb0, 0.f), fmaxf(acc[j][1] + bb1, 0.f));
      const uint32_t hi = pack_bf16(fmaxf(acc[j][2] + bb0, 0.f), fmaxf(acc[j][3] + bb1, 0.f));
      *reinterpret_cast<uint32_t*>(Hs + rA * ldh + col) = lo;
      *reinterpret_cast<uint32_t*>(Hs + rB * ldh + col) = hi;
      if (Hg) {
        if (rA < here) *reinterpret_cast<uint32_t*>(Hg + (row0 + rA) * HID + col) = lo;
        if (rB < here) *reinterpret_cast<uint32_t*>(Hg + (row0 + rB) * HID + col) = hi;
      }
    }
    __syncthreads();
  }
  // layer 3: outp columns, split in halves between the two warp columns, up to 128 columns at a time
  const int half = a.outp / 2;
  for (int c0 = nh * half; c0 < (nh + 1) * half; c0 += 128) {
    const int ntiles = min(128, (nh + 1) * half - c0) / 8;  // outp is a multiple of 16
    switch (ntiles) {
#define L3(NT) \
  case NT:     \
    layer3_chunk<NT>(a, H2s + 16 * mt * ldh, ldh, c0, rA, rB, row0, here); \
    break;
      L3(1) L3(2) L3(3) L3(4) L3(5) L3(6) L3(7) L3(8) L3(9) L3(10) L3(11) L3(12) L3(13) L3(14) L3(15) L3(16)
#undef L3
      default:
        break;
    }
  }
}

// ---------------------------------------------------------------------------------------------
// The same fused forward pass on the 5th-generation tensor cores (tcgen05): one CTA per 128 rows.  For
// each layer the A operand (the X tile, then H1, then H2, BF16) and the layer's weights are staged in
// shared memory in the no-swizzle K-major canonical layout (8-row x 16-byte core matrices, consecutive
// along K at LBO = 128 B, 8-row groups at SBO = K/8 x 128 B); one thread issues the K/16 MMAs
// (M = 128, N = layer width, FP32 accumulator in tensor memory) and commits them to an mbarrier; the four
// warps then read their 32 accumulator rows back with tcgen05.ld for the bias / ReLU / BF16 epilogue,
// which writes the next layer's A operand in place.  Inference only (kinp <= 256, outp <= 256).
// ---------------------------------------------------------------------------------------------
constexpr int TC_ROWS = 128;
constexpr int TC_THREADS = 256;  // 8 warps: warp w reads TMEM lanes 32 (w % 4) .. (its rows), columns half w / 4
constexpr int TC_KMAX = 256;
constexpr uint32_t TC_TMEM_COLS = 256;
constexpr size_t TC_ABYTES = (size_t)TC_ROWS * TC_KMAX * 2;  // 64 KB
constexpr size_t TC_WBYTES = (size_t)HID * TC_KMAX * 2;      // 128 KB
constexpr size_t TC_BBYTES = 3 * HID * 4;                    // the three bias vectors (FP32)
constexpr size_t TC_SMEM = TC_ABYTES + TC_WBYTES + TC_BBYTES + 64;  // + mbarriers and the tensor-memory address
constexpr uint32_t TC_WAIT_ITERS = 1u << 21;                 // bounded mbarrier wait (about a second)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// byte offset of the 16-byte chunk (row r, elements 8c..8c+7) in the canonical layout of a K-wide operand
__device__ __forceinline__ uint32_t core_chunk(int r, int c, int K) {
  return (uint32_t)((r >> 3) * (K >> 3) * 128 + c * 128 + (r & 7) * 16);
}
// shared memory matrix descriptor: start address, LBO, SBO (all >> 4), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}
// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both K-major, M x N
__device__ __forceinline__ uint32_t tc_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void tc_mma(uint32_t tmem_d, uint64_t ad, uint64_t bd, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem_d),
      "l"(ad), "l"(bd), "r"(idesc), "r"(acc)
      : "memory");
}
__device__ __forceinline__ void tc_commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t mbar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}\n"
      : "=r"(ok)
      : "r"(mbar), "r"(parity)
      : "memory");
  return ok != 0;
}
// wait for the mbarrier phase with the given parity; false after `tries` unsuccessful tries
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, uint32_t tries = TC_WAIT_ITERS) {
  for (uint32_t it = 0; it < tries; ++it) {
    if (mbar_try_wait(mbar, parity)) return true;
    __nanosleep(128);
  }
  return false;
}
// 32 (or 8) consecutive accumulator columns of this thread's TMEM lane
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,"
      "%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
        "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
        "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float (&v)[8]) {
  uint32_t r[8];
  asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
               : "r"(taddr)
               : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// a row-major [128][K] BF16 tile into the canonical layout at dst (zero rows from `valid` on): thread t takes row
// t % 128 and half t / 128 of its 16-byte chunks, eight loads in flight
__device__ __forceinline__ void tc_stage_rows(unsigned char* dst, const __nv_bfloat16* __restrict__ src, int valid,
                                              int K) {
  const int n = threadIdx.x & (TC_ROWS - 1), nc = K >> 3, hc = (nc + 1) >> 1;
  const int cbeg = (threadIdx.x >> 7) * hc, cend = min(nc, cbeg + hc);
  const uint4* row = reinterpret_cast<const uint4*>(src + (size_t)n * K);
  for (int c0 = cbeg; c0 < cend; c0 += 8) {
    uint4 v[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) v[j] = (n < valid && c0 + j < cend) ? __ldg(row + c0 + j) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int j = 0; j < 8; ++j)
      if (c0 + j < cend) *reinterpret_cast<uint4*>(dst + core_chunk(n, c0 + j, K)) = v[j];
  }
}

// bulk asynchronous copy of `bytes` (a multiple of 16) from global memory into shared memory, completing as
// transaction bytes on the mbarrier; issued in pieces of at most 32 KB by one thread, after it announced the
// total with expect_tx
__device__ __forceinline__ void tc_bulk_load(uint32_t dst, const void* src, uint32_t bytes, uint32_t mbar) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(mbar), "r"(bytes) : "memory");
  const char* g = static_cast<const char*>(src);
  for (uint32_t o = 0; o < bytes; o += 32768u) {
    const uint32_t n = bytes - o < 32768u ? bytes - o : 32768u;
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     dst + o),
                 "l"(g + o), "r"(n), "r"(mbar)
                 : "memory");
  }
}

// one layer: D (tensor memory) = A (128 x K) W^T (W: N x K), issued by one thread and committed to the mbarrier
// mbar
__device__ __forceinline__ void tc_layer(uint32_t tmem, uint32_t a_s, uint32_t w_s, int K, int N, uint32_t mbar) {
  const uint32_t idesc = tc_idesc(TC_ROWS, N), sbo = (uint32_t)(K >> 3) * 128;
  for (int kk = 0; kk < (K >> 4); ++kk)
    tc_mma(tmem, tc_sdesc(a_s + kk * 256, 128, sbo), tc_sdesc(w_s + kk * 256, 128, sbo), idesc, kk > 0 ? 1u : 0u);
  tc_commit(mbar);
}

// bias + ReLU of this thread's accumulator row (columns of its half), as BF16, into the next layer's A operand
// (K = HID); bias in shared memory.  Hrow (training): the same BF16 values also go to this row of the hidden
// layer in global memory (row-major [rows][HID]), or nullptr.
__device__ __forceinline__ void tc_hidden_epilogue(uint32_t trow, int row, int c_lo, const float* bias,
                                                   unsigned char* As, __nv_bfloat16* Hrow) {
  for (int cb = c_lo; cb < c_lo + HID / 2; cb += 32) {
    float v[32];
    tmem_ld32(trow + cb, v);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      uint32_t p[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int j = 8 * q + 2 * i;
        const float x0 = fmaxf(v[j] + bias[cb + j], 0.f);
        const float x1 = fmaxf(v[j + 1] + bias[cb + j + 1], 0.f);
        p[i] = pack_bf16(x0, x1);
      }
      const uint4 v4 = make_uint4(p[0], p[1], p[2], p[3]);
      *reinterpret_cast<uint4*>(As + core_chunk(row, (cb >> 3) + q, HID)) = v4;
      if (Hrow) *reinterpret_cast<uint4*>(Hrow + cb + 8 * q) = v4;
    }
  }
}

// Bounded waits: thread 0 alone waits for the weights and keeps count of the asynchronous work in flight (the
// weight copy into Ws, the committed MMAs); every thread waits for MMA completion before it reads the accumulator.
// A timed-out wait clears the CTA's status flag (shared memory); from then on no MMA and no copy is issued, the
// epilogues are skipped, thread 0 waits again (bounded, the full limit) for whatever is still in flight, the rows
// of this tile are written as NaN straight to global memory, and the tensor memory is freed before returning.
__global__ void __launch_bounds__(TC_THREADS, 1) mlp_forward_tc(const FwdArgs a) {
  extern __shared__ __align__(1024) unsigned char tc_smem[];
  unsigned char* As = tc_smem;
  unsigned char* Ws = tc_smem + TC_ABYTES;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(tc_smem + TC_ABYTES + TC_WBYTES);  // MMA completion
  uint64_t* wbar = mbar + 1;                                                      // weight arrival
  uint32_t* tslot = reinterpret_cast<uint32_t*>(tc_smem + TC_ABYTES + TC_WBYTES + 16);
  volatile uint32_t* status = tslot + 1;  // 1 while every wait has succeeded
  float* bs = reinterpret_cast<float*>(tc_smem + TC_ABYTES + TC_WBYTES + 64);  // b1, b2, b3
  const int tid = threadIdx.x, warp = tid >> 5;
  const int row = 32 * (warp & 3) + (tid & 31), half = warp >> 2;  // TMEM lane = row; column half
  const int64_t row0 = (int64_t)blockIdx.x * TC_ROWS;
  const int here = (int)min((int64_t)TC_ROWS, a.rows - row0);
  const uint32_t a_s = smem_u32(As), w_s = smem_u32(Ws), mb = smem_u32(mbar), wb = smem_u32(wbar);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)),
                 "r"(TC_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  // thread 0's record of asynchronous work in flight, with the phase parities of the two mbarriers
  bool w_pending = false, m_pending = false;
  uint32_t wpar = 0, mpar = 0;
  if (tid == 0) {
    *status = 1u;
    mbar_init(mb, 1);
    mbar_init(wb, 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    fence_async_smem();
    tc_bulk_load(w_s, a.W1p, (uint32_t)(HID * a.kinp * 2), wb);  // W1 streams in while the X tile is staged
    w_pending = true;
  }
  tc_stage_rows(As, a.X + row0 * a.kinp, here, a.kinp);
  for (int i = tid; i < 3 * HID; i += TC_THREADS) {
    const int l = i / HID, j = i - l * HID;
    bs[i] = l == 0 ? __ldg(a.b1 + j) : (l == 1 ? __ldg(a.b2 + j) : (j < a.outp ? __ldg(a.b3 + j) : 0.f));
  }
  fence_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);  // this warp's 32 lanes = its 32 rows
#pragma unroll 1
  for (int layer = 0; layer < 3; ++layer) {
    // thread 0: weights arrived -> the layer's MMAs, committed to mb
    if (tid == 0 && *status == 1u) {
      if (mbar_wait(wb, wpar, a.w_wait_tries)) {
        w_pending = false;
        wpar ^= 1u;
        tc_layer(tmem, a_s, w_s, layer == 0 ? a.kinp : HID, layer == 2 ? a.outp : HID, mb);
        m_pending = true;
      } else {
        *status = 0u;
      }
    }
    __syncthreads();
    // every thread: the MMAs have completed (their accumulator is readable, A and W are free again)
    bool saw = false;
    if (*status == 1u) {
      saw = mbar_wait(mb, mpar);
      if (!saw) *status = 0u;
    }
    tc_fence_after();
    __syncthreads();
    const bool ok = *status == 1u;
    if (tid == 0 && saw) {
      m_pending = false;
      mpar ^= 1u;
      // the next layer's weights stream in during the epilogue, which overwrites A with the hidden layer
      if (ok && layer < 2) {
        tc_bulk_load(w_s, layer == 0 ? a.W2p : a.W3p, (uint32_t)((layer == 0 ? HID : a.outp) * HID * 2), wb);
        w_pending = true;
      }
    }
    if (layer == 2 || !ok) break;
    __nv_bfloat16* Hg = layer == 0 ? a.H1 : a.H2;
    tc_hidden_epilogue(trow, row, half * (HID / 2), bs + layer * HID, As,
                       (Hg && row < here) ? Hg + (row0 + row) * HID : nullptr);
    fence_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  }
  // after a timeout: wait (bounded) for the copy or MMAs still in flight before shared or tensor memory is reused
  if (tid == 0) {
    if (m_pending && mbar_wait(mb, mpar)) m_pending = false;
    if (w_pending && mbar_wait(wb, wpar)) w_pending = false;
  }
  __syncthreads();
  if (*status == 1u) {
    // output layer: the accumulator rows plus bias go through shared memory (A and W are free now; rows padded
    // by four floats), then the tile's block of Y (rows x outp) or z (cells x nb, scaled) is written
    // contiguously
    float* Ys = reinterpret_cast<float*>(tc_smem);
    const int ys = a.outp + 4;
    const int ohalf = a.outp >> 1;  // a multiple of 8
    for (int cb = half * ohalf; cb < (half + 1) * ohalf; cb += 8) {
      float v[8];
      tmem_ld8(trow + cb, v);
#pragma unroll
      for (int i = 0; i < 8; ++i) v[i] += bs[2 * HID + cb + i];
      *reinterpret_cast<float4*>(Ys + row * ys + cb) = make_float4(v[0], v[1], v[2], v[3]);
      *reinterpret_cast<float4*>(Ys + row * ys + cb + 4) = make_float4(v[4], v[5], v[6], v[7]);
    }
    __syncthreads();
    if (a.Y) {
      float* dst = a.Y + row0 * a.outp;
      for (int e = tid; e < here * a.outp; e += TC_THREADS) {
        const int r = e / a.outp, c = e - r * a.outp;
        dst[e] = Ys[r * ys + c];
      }
    }
    if (a.z) {
      for (int e = tid; e < here * a.nb; e += TC_THREADS) {
        const int r = e / a.nb, c = e - r * a.nb;
        const float zv = a.scale[row0 + r] * Ys[r * ys + c];
        const size_t zi = (size_t)row0 * a.nb + e;
        if (a.z_is_f64) {
          double* zp = static_cast<double*>(a.z) + zi;
          *zp = a.z_accumulate ? *zp + (double)zv : (double)zv;
        } else {
          float* zp = static_cast<float*>(a.z) + zi;
          *zp = a.z_accumulate ? *zp + zv : zv;
        }
      }
    }
  } else {
    // a wait timed out: NaN rows (a solve that uses them reports a non-finite residual)
    const float nan = __int_as_float(0x7fc00000);
    if (a.Y)
      for (int e = tid; e < here * a.outp; e += TC_THREADS) a.Y[row0 * a.outp + e] = nan;
    if (a.z)
      for (int e = tid; e < here * a.nb; e += TC_THREADS) {
        const size_t zi = (size_t)row0 * a.nb + e;
        if (a.z_is_f64)
          static_cast<double*>(a.z)[zi] = (double)nan;
        else
          static_cast<float*>(a.z)[zi] = nan;
      }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(TC_TMEM_COLS) : "memory");
  }
}

// One warp writes the feature row of `cell` into xr: [sign r_T / s, log D (own, x-, x+, y-, y+, z-, z+), 0 ...] in
// BF16, s = ||r_T||_2 (a zero residual gives a zero row); returns s on every lane.
template <typename T>
__device__ __forceinline__ float feature_row(const T* __restrict__ rc, float sign, const double* __restrict__ D, int nx,
                                             int ny, int nz, int64_t cell, int nb, int kinp, __nv_bfloat16* xr) {
  const int lane = threadIdx.x & 31;
  float ss = 0.f;
  for (int j = lane; j < nb; j += 32) {
    const float v = (float)rc[j];
    ss = fmaf(v, v, ss);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  const float s = sqrtf(ss);
  const float inv = s > 0.f ? sign / s : 0.f;
  for (int j = lane; j < nb; j += 32) xr[j] = __float2bfloat16_rn((float)rc[j] * inv);
  if (lane < 7) {
    const int ic[3] = {(int)(cell % nx), (int)((cell / nx) % ny), (int)(cell / ((int64_t)nx * ny))};
    int64_t c = cell;
    if (lane > 0) {
      const int dir = (lane - 1) / 2, up = (lane - 1) & 1;
      const int n[3] = {nx, ny, nz};
      const int64_t st[3] = {1, nx, (int64_t)nx * ny};
      const bool inside = up ? ic[dir] + 1 < n[dir] : ic[dir] > 0;
      if (inside) c = up ? cell + st[dir] : cell - st[dir];
    }
    xr[nb + lane] = __float2bfloat16_rn((float)log(D[c]));
  }
  for (int j = nb + 7 + lane; j < kinp; j += 32) xr[j] = __float2bfloat16_rn(0.f);
  return s;
}

// Feature rows for cells: X[row] = feature_row(r on cell), scale[row] = s * t_scale.
template <typename T>
__global__ void mlp_features(const T* __restrict__ r, const double* __restrict__ D, int nx, int ny, int nz,
                             const int* __restrict__ cells, int64_t nrows, int nb, int kinp, float t_scale,
                             __nv_bfloat16* __restrict__ X, float* __restrict__ scale) {
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t row = warp0; row < nrows; row += nwarps) {
    const int64_t cell = cells ? cells[row] : row;
    const float s = feature_row<T>(r + cell * nb, 1.f, D, nx, ny, nz, cell, nb, kinp, X + row * kinp);
    if ((threadIdx.x & 31) == 0) scale[row] = s * t_scale;
  }
}

// Training pairs from a solver state: y = A x - F is the negated residual r = F - A x; for sample i (cell cells[i],
// output row rows[i]) X[row] = feature_row(r), E[row][j] = (xstar - x - BJ(r))_j / ||r_cell|| on the cell, where
// bjy = BJ(y) = -BJ(r) is the block-Jacobi correction of y (or null: no subtraction); zero where r_cell = 0.
__global__ void mlp_pairs(const double* __restrict__ y, const double* __restrict__ x, const double* __restrict__ xstar,
                          const double* __restrict__ bjy, const double* __restrict__ D, int nx, int ny, int nz,
                          const int* __restrict__ cells, const int* __restrict__ rows, int64_t count, int nb, int kinp,
                          __nv_bfloat16* __restrict__ X, float* __restrict__ E) {
  const int lane = threadIdx.x & 31;
  const int64_t warp0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t i = warp0; i < count; i += nwarps) {
    const int64_t cell = cells[i], row = rows[i];
    const float s = feature_row<double>(y + cell * nb, -1.f, D, nx, ny, nz, cell, nb, kinp, X + row * kinp);
    const double inv = s > 0.f ? 1.0 / (double)s : 0.0;
    const int64_t b = cell * nb;
    for (int j = lane; j < nb; j += 32) {
      double e = xstar[b + j] - x[b + j];
      if (bjy) e += bjy[b + j];
      E[row * nb + j] = (float)(e * inv);
    }
  }
}

// sum of squares of E in FP64: per-block partial sums
__global__ void sum_squares(const float* __restrict__ E, int64_t n, double* __restrict__ part) {
  __shared__ double red[8];
  double acc = 0.0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    acc += (double)E[i] * E[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    part[blockIdx.x] = t;
  }
}

__global__ void scale_in_place(float* __restrict__ E, int64_t n, float a) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    E[i] *= a;
}

// ---- backward pass: BF16 tensor-core GEMMs with FP32 accumulation ----

// C[M x N] = sum_k A(m,k) B(k,n) with A(m,k) = A[m*sam + k*sak] and B(k,n) = B[k*sbk + n] (n contiguous), both
// rounded to BF16 on the way into shared memory; mma.sync m16n8k16 (BF16 in, FP32 accumulate).  CTA tile 64 x 64,
// K step 32, four warps of 32 x 32 (2 x 4 MMA tiles).  Shared tiles: As[m][k], Bs[n][k] (B transposed, so that
// both fragments are 32-bit loads of consecutive k), rows padded to 40 halves.
constexpr int GB_M = 64, GB_N = 64, GB_K = 32, GB_KP = GB_K + 8, GB_THREADS = 128;

template <typename TA, typename TB>
__global__ void __launch_bounds__(GB_THREADS) gemm_bf16_tc(int M, int N, int K, const TA* __restrict__ A, int64_t sam,
                                                           int64_t sak, const TB* __restrict__ B, int64_t sbk,
                                                           float* __restrict__ C, int ldc) {
  __shared__ __align__(16) __nv_bfloat16 As[GB_M * GB_KP];
  __shared__ __align__(16) __nv_bfloat16 Bs[GB_N * GB_KP];
  const int m0 = blockIdx.y * GB_M, n0 = blockIdx.x * GB_N;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, tig = lane & 3;
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  const bool a_m_fast = sam == 1;  // consecutive threads read consecutive m (else consecutive k)
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
  for (int k0 = 0; k0 < K; k0 += GB_K) {
    for (int e = threadIdx.x; e < GB_M * GB_K; e += GB_THREADS) {
      const int mm = a_m_fast ? e % GB_M : e / GB_K, kk = a_m_fast ? e / GB_M : e % GB_K;
      const int gm = m0 + mm, gk = k0 + kk;
      const float v = (gm < M && gk < K) ? (float)A[gm * sam + gk * sak] : 0.f;
      As[mm * GB_KP + kk] = __float2bfloat16_rn(v);
    }
    for (int e = threadIdx.x; e < GB_N * GB_K; e += GB_THREADS) {
      const int nn = e % GB_N, kk = e / GB_N;
      const int gn = n0 + nn, gk = k0 + kk;
      const float v = (gn < N && gk < K) ? (float)B[gk * sbk + gn] : 0.f;
      Bs[nn * GB_KP + kk] = __float2bfloat16_rn(v);
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < GB_K; ks += 16) {
      uint32_t a[2][4];
#pragma unroll
      for (int i = 0; i < 2; ++i) {
        const __nv_bfloat16* ap = As + (wm + 16 * i + g) * GB_KP + ks + 2 * tig;
        a[i][0] = *reinterpret_cast<const uint32_t*>(ap);
        a[i][1] = *reinterpret_cast<const uint32_t*>(ap + 8 * GB_KP);
        a[i][2] = *reinterpret_cast<const uint32_t*>(ap + 8);
        a[i][3] = *reinterpret_cast<const uint32_t*>(ap + 8 * GB_KP + 8);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const __nv_bfloat16* bp = Bs + (wn + 8 * j + g) * GB_KP + ks + 2 * tig;
        const uint32_t b0 = *reinterpret_cast<const uint32_t*>(bp);
        const uint32_t b1 = *reinterpret_cast<const uint32_t*>(bp + 8);
#pragma unroll
        for (int i = 0; i < 2; ++i) mma_bf16(acc[i][j], a[i], b0, b1);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int gm = m0 + wm + 16 * i + g + (q >= 2 ? 8 : 0), gn = n0 + wn + 8 * j + 2 * tig + (q & 1);
        if (gm < M && gn < N) C[(size_t)gm * ldc + gn] = acc[i][j][q];
      }
}

// dY = 2 (Y - T) / (rows * nb) on the nb real outputs (zero on the padding); loss partials per block
__global__ void loss_grad(const float* __restrict__ Y, const float* __restrict__ T, int64_t rows, int nb, int outp,
                          float* __restrict__ dY, double* __restrict__ loss_part) {
  __shared__ double red[8];
  double acc = 0.0;
  const float inv = 2.f / (float)((double)rows * nb);
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < rows * outp; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / outp;
    const int c = (int)(e - r * outp);
    float d = 0.f;
    if (c < nb) {
      d = Y[e] - T[r * nb + c];
      acc += (double)d * d;
    }
    dY[e] = d * inv;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += red[w];
    loss_part[blockIdx.x] = t;
  }
}

// dZ = dH * (H > 0)
__global__ void relu_back(float* __restrict__ dH, const __nv_bfloat16* __restrict__ H, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    if (!(__bfloat162float(H[i]) > 0.f)) dH[i] = 0.f;
}

// db[c] = sum_r dZ[r][c]  (one thread per column, fixed order)
__global__ void col_sum(const float* __restrict__ dZ, int64_t rows, int cols, float* __restrict__ db) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= cols) return;
  float acc = 0.f;
  for (int64_t r = 0; r < rows; ++r) acc += dZ[r * cols + c];
  db[c] = acc;
}

// W (row-major [N][K] BF16) into the canonical no-swizzle K-major layout of the tcgen05 forward pass: the
// 16-byte chunk (n, c) at byte (n / 8) (K / 8) 128 + 128 c + 16 (n % 8)
__global__ void pack_canonical(const __nv_bfloat16* __restrict__ W, int N, int K, __nv_bfloat16* __restrict__ P) {
  const int nc = K >> 3;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < N * nc; e += gridDim.x * blockDim.x) {
    const int n = e / nc, c = e - n * nc;
    const size_t dst = ((size_t)(n >> 3) * nc * 128 + (size_t)c * 128 + (n & 7) * 16) / 2;
    *reinterpret_cast<uint4*>(P + dst) = *reinterpret_cast<const uint4*>(W + (size_t)n * K + 8 * c);
  }
}

__global__ void adam_step(float* __restrict__ w, const float* __restrict__ g, float* __restrict__ m,
                          float* __restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float c1,
                          float c2, __nv_bfloat16* __restrict__ wh) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    const float wi = w[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    w[i] = wi;
    if (wh) wh[i] = __float2bfloat16_rn(wi);
  }
}

__global__ void to_bf16(const float* __restrict__ a, __nv_bfloat16* __restrict__ b, int64_t n) {
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    b[i] = __float2bfloat16_rn(a[i]);
}

}  // namespace dgm

// Parameters: one FP32 master block [W1 | b1 | W2 | b2 | W3 | b3] with its Adam moments, and BF16
// copies of W1, W2, W3 (biases stay FP32 in the forward pass).
struct dg_mlp {
  int k = 0;
  dgm::Dims d;
  float t_scale = 1.f;
  int64_t nparam = 0;
  int64_t off[6] = {};   // offsets of W1, b1, W2, b2, W3, b3 in the FP32 block
  float* w = nullptr;    // FP32 master
  float* g = nullptr;    // gradient
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* wh = nullptr;  // BF16 copy of the whole block (only W1, W2, W3 are read)
  // W1, W2, W3 of wh packed for the tcgen05 forward pass (refreshed when wh_version moves on)
  mutable __nv_bfloat16* whp = nullptr;
  mutable int64_t packed_version = -1;
  int64_t wh_version = 0;
  int64_t adam_t = 0;
  // training / inference scratch (grown on demand)
  void* ws = nullptr;
  size_t ws_bytes = 0;
};

namespace dgi {
bool mlp_matches(const dg_mlp* m, const dg_handle* h) { return m && h && m->d.nb == h->N * h->N * h->N; }
}  // namespace dgi

namespace {

using namespace dgi;

int cfail(cudaError_t e, const char* what) { return e == cudaSuccess ? 0 : cuda_fail(e, what); }

size_t fwd_smem(const dgm::Dims& d) {
  return ((size_t)dgm::ROWS * (d.kinp + 8) + 2 * (size_t)dgm::ROWS * (dgm::HID + 8)) * sizeof(__nv_bfloat16);
}

int ensure_ws(dg_mlp* m, size_t bytes) {
  if (m->ws_bytes >= bytes) return 0;
  cudaFree(m->ws);
  m->ws = nullptr;
  m->ws_bytes = 0;
  if (int rc = cfail(cudaMalloc(&m->ws, bytes), "cudaMalloc(MLP workspace)")) return rc;
  m->ws_bytes = bytes;
  return 0;
}

// Polls of the tcgen05 kernel's weight-arrival wait (about a second at the default).  DG_MLP_WEIGHT_WAIT_TRIES
// lowers it to exercise the timeout path: with 0 the wait gives up at once, the kernel issues nothing more,
// waits (with the full limit) for the copy still in flight and writes NaN rows.
uint32_t weight_wait_tries() {
  const char* v = std::getenv("DG_MLP_WEIGHT_WAIT_TRIES");
  if (!v || !*v) return dgm::TC_WAIT_ITERS;
  char* end = nullptr;
  const unsigned long t = std::strtoul(v, &end, 10);
  return (end && *end == 0 && t < dgm::TC_WAIT_ITERS) ? (uint32_t)t : dgm::TC_WAIT_ITERS;
}

dgm::FwdArgs fwd_args(const dg_mlp* m, const __nv_bfloat16* X, int64_t rows) {
  dgm::FwdArgs a{};
  a.X = X;
  a.W1 = m->wh + m->off[0];
  a.b1 = m->w + m->off[1];
  a.W2 = m->wh + m->off[2];
  a.b2 = m->w + m->off[3];
  a.W3 = m->wh + m->off[4];
  a.b3 = m->w + m->off[5];
  a.rows = rows;
  a.kinp = m->d.kinp;
  a.outp = m->d.outp;
  a.nb = m->d.nb;
  a.w_wait_tries = weight_wait_tries();
  return a;
}

// the tensor-memory (tcgen05) forward pass serves networks with kinp, outp <= 256 (degrees 1..5), for inference
// and for training (where it also stores the hidden layers); larger networks use the mma.sync kernel
bool use_tc_forward(const dg_mlp* m, const dgm::FwdArgs&) {
  return m->d.kinp <= dgm::TC_KMAX && m->d.outp <= dgm::HID && !std::getenv("DG_MLP_NO_TCGEN05");
}

// the weights of the tcgen05 kernel in its shared-memory layout, repacked on the stream after every change of
// the BF16 copy
int packed_weights(const dg_mlp* m, cudaStream_t s, dgm::FwdArgs& a) {
  const int H = dgm::HID;
  const int64_t n1 = (int64_t)H * m->d.kinp, n2 = (int64_t)H * H, n3 = (int64_t)m->d.outp * H;
  if (!m->whp) {
    if (int rc = cfail(cudaMalloc(&m->whp, (n1 + n2 + n3) * sizeof(__nv_bfloat16)), "cudaMalloc(MLP packed)"))
      return rc;
  }
  if (m->packed_version != m->wh_version) {
    dgm::pack_canonical<<<64, 256, 0, s>>>(m->wh + m->off[0], H, m->d.kinp, m->whp);
    dgm::pack_canonical<<<64, 256, 0, s>>>(m->wh + m->off[2], H, H, m->whp + n1);
    dgm::pack_canonical<<<64, 256, 0, s>>>(m->wh + m->off[4], m->d.outp, H, m->whp + n1 + n2);
    if (int rc = cfail(cudaGetLastError(), "MLP weight packing")) return rc;
    m->packed_version = m->wh_version;
  }
  a.W1p = m->whp;
  a.W2p = m->whp + n1;
  a.W3p = m->whp + n1 + n2;
  return 0;
}

int launch_forward(const dg_mlp* m, const dgm::FwdArgs& a_in, cudaStream_t s) {
  dgm::FwdArgs a = a_in;
  if (use_tc_forward(m, a)) {
    if (int rc = packed_weights(m, s, a)) return rc;
    static DeviceOnce tc_attr;
    if (int rc = tc_attr.run([] {
          return cfail(cudaFuncSetAttribute(dgm::mlp_forward_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)dgm::TC_SMEM),
                       "MLP tcgen05 forward smem");
        }))
      return rc;
    const unsigned grid = (unsigned)((a.rows + dgm::TC_ROWS - 1) / dgm::TC_ROWS);
    if (grid == 0) return 0;
    dgm::mlp_forward_tc<<<grid, dgm::TC_THREADS, dgm::TC_SMEM, s>>>(a);
    return cfail(cudaGetLastError(), "MLP tcgen05 forward");
  }
  const size_t smem = fwd_smem(m->d);
  if (smem > 48 * 1024) {  // set on every launch above the default: the size depends on the network
    if (int rc = cfail(cudaFuncSetAttribute(dgm::mlp_forward, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)smem),
                       "MLP forward smem"))
      return rc;
  }
  const unsigned grid = (unsigned)((a.rows + dgm::ROWS - 1) / dgm::ROWS);
  if (grid == 0) return 0;
  dgm::mlp_forward<<<grid, dgm::FWD_THREADS, smem, s>>>(a);
  return cfail(cudaGetLastError(), "MLP forward");
}

// C = A B on the tensor cores (BF16 operands, FP32 accumulation); B's n index is contiguous (sbn = 1)
template <typename TA, typename TB>
int gemm(int M, int N, int K, const TA* A, int64_t sam, int64_t sak, const TB* B, int64_t sbk, int64_t sbn, float* C,
         int ldc, cudaStream_t s) {
  if (sbn != 1) {
    set_error("MLP backward GEMM: B must have its n index contiguous");
    return DG_ERR_INVALID_ARG;
  }
  dim3 grid((N + dgm::GB_N - 1) / dgm::GB_N, (M + dgm::GB_M - 1) / dgm::GB_M);
  dgm::gemm_bf16_tc<TA, TB><<<grid, dgm::GB_THREADS, 0, s>>>(M, N, K, A, sam, sak, B, sbk, C, ldc);
  return cfail(cudaGetLastError(), "MLP backward GEMM");
}

// loss and gradient (into m->g) of one batch: X bf16 [rows][kinp], T fp32 [rows][nb]
int loss_and_grad(dg_mlp* m, const __nv_bfloat16* X, const float* T, int64_t rows, double* loss, cudaStream_t s) {
  const dgm::Dims& d = m->d;
  const int H = dgm::HID;
  // scratch: H1, H2 (bf16), Y, dY (f32 rows x outp), dH (f32 rows x H), loss partials
  const size_t nbh = (size_t)rows * H * sizeof(__nv_bfloat16);
  const size_t nY = (size_t)rows * d.outp * sizeof(float);
  const size_t ndH = (size_t)rows * H * sizeof(float);
  const int lblocks = 256;
  const size_t bytes = 2 * nbh + 2 * nY + 2 * ndH + lblocks * sizeof(double) + 1024;
  if (int rc = ensure_ws(m, bytes)) return rc;
  unsigned char* p = static_cast<unsigned char*>(m->ws);
  auto* H1 = reinterpret_cast<__nv_bfloat16*>(p);
  auto* H2 = reinterpret_cast<__nv_bfloat16*>(p + nbh);
  auto* Y = reinterpret_cast<float*>(p + 2 * nbh);
  auto* dY = reinterpret_cast<float*>(p + 2 * nbh + nY);
  auto* dH = reinterpret_cast<float*>(p + 2 * nbh + 2 * nY);
  auto* dH1 = reinterpret_cast<float*>(p + 2 * nbh + 2 * nY + ndH);
  auto* lp = reinterpret_cast<double*>(p + 2 * nbh + 2 * nY + 2 * ndH);
  dgm::FwdArgs a = fwd_args(m, X, rows);
  a.H1 = H1;
  a.H2 = H2;
  a.Y = Y;
  if (int rc = launch_forward(m, a, s)) return rc;
  dgm::loss_grad<<<lblocks, 256, 0, s>>>(Y, T, rows, d.nb, d.outp, dY, lp);
  float* g = m->g;
  const __nv_bfloat16* W2 = m->wh + m->off[2];
  const __nv_bfloat16* W3 = m->wh + m->off[4];
  int rc = 0;
  // layer 3: dW3[o][h] = sum_r dY[r][o] H2[r][h]; db3; dH2 = dY W3
  rc = gemm<float, __nv_bfloat16>(d.outp, H, (int)rows, dY, 1, d.outp, H2, H, 1, g + m->off[4], H, s);
  if (!rc) {
    dgm::col_sum<<<(d.outp + 127) / 128, 128, 0, s>>>(dY, rows, d.outp, g + m->off[5]);
    rc = gemm<float, __nv_bfloat16>((int)rows, H, d.outp, dY, d.outp, 1, W3, H, 1, dH, H, s);
  }
  // layer 2
  if (!rc) {
    dgm::relu_back<<<1024, 256, 0, s>>>(dH, H2, (int64_t)rows * H);
    rc = gemm<float, __nv_bfloat16>(H, H, (int)rows, dH, 1, H, H1, H, 1, g + m->off[2], H, s);
  }
  if (!rc) {
    dgm::col_sum<<<(H + 127) / 128, 128, 0, s>>>(dH, rows, H, g + m->off[3]);
    rc = gemm<float, __nv_bfloat16>((int)rows, H, H, dH, H, 1, W2, H, 1, dH1, H, s);  // dH1 = dZ2 W2
  }
  // layer 1
  if (!rc) {
    dgm::relu_back<<<1024, 256, 0, s>>>(dH1, H1, (int64_t)rows * H);
    rc = gemm<float, __nv_bfloat16>(H, d.kinp, (int)rows, dH1, 1, H, X, d.kinp, 1, g + m->off[0], d.kinp, s);
  }
  if (!rc) {
    dgm::col_sum<<<(H + 127) / 128, 128, 0, s>>>(dH1, rows, H, g + m->off[1]);
    rc = cfail(cudaGetLastError(), "MLP backward");
  }
  if (!rc && loss) {
    std::vector<double> h(lblocks);
    rc = cfail(cudaMemcpyAsync(h.data(), lp, lblocks * sizeof(double), cudaMemcpyDeviceToHost, s), "loss copy");
    if (!rc) rc = cfail(cudaStreamSynchronize(s), "loss sync");
    double t = 0;
    for (double x : h) t += x;
    *loss = t / ((double)rows * d.nb);
  }
  return rc;
}

void free_mlp(dg_mlp* m) {
  if (!m) return;
  cudaFree(m->w);
  cudaFree(m->g);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->wh);
  cudaFree(m->whp);
  cudaFree(m->ws);
  delete m;
}

}  // namespace

extern "C" {

int dg_mlp_create(int32_t k, uint64_t seed, dg_mlp** out) {
  if (!out || k < 1 || k > 7) {
    set_error("dg_mlp_create: degree must be in [1, 7]");
    return DG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  dg_mlp* m = new dg_mlp();
  m->k = k;
  m->d = dgm::dims_for(k);
  const int H = dgm::HID;
  // layer 3 keeps a full HID x HID-sized backing so the backward pass can reuse its buffers
  const int64_t sizes[6] = {(int64_t)H * m->d.kinp, H, (int64_t)H * H, H, (int64_t)m->d.outp * H, m->d.outp};
  int64_t o = 0;
  for (int i = 0; i < 6; ++i) {
    m->off[i] = o;
    o += (sizes[i] + 63) / 64 * 64;
  }
  m->nparam = o;
  // He-uniform initialisation on the real fan-in; padding rows/columns start at zero
  std::vector<float> w(o, 0.f);
  std::mt19937_64 rng(seed);
  auto init = [&](int64_t off, int rows, int cols, int fan_in, int real_rows, int real_cols) {
    const float lim = std::sqrt(6.f / (float)fan_in);
    std::uniform_real_distribution<float> u(-lim, lim);
    for (int r = 0; r < rows; ++r)
      for (int c = 0; c < cols; ++c) w[off + (int64_t)r * cols + c] = (r < real_rows && c < real_cols) ? u(rng) : 0.f;
  };
  init(m->off[0], H, m->d.kinp, m->d.kin, H, m->d.kin);
  init(m->off[2], H, H, H, H, H);
  init(m->off[4], m->d.outp, H, H, m->d.nb, H);
  int rc = cfail(cudaMalloc(&m->w, o * sizeof(float)), "cudaMalloc(MLP)");
  if (!rc) rc = cfail(cudaMalloc(&m->g, o * sizeof(float)), "cudaMalloc(MLP grad)");
  if (!rc) rc = cfail(cudaMalloc(&m->m, o * sizeof(float)), "cudaMalloc(MLP m)");
  if (!rc) rc = cfail(cudaMalloc(&m->v, o * sizeof(float)), "cudaMalloc(MLP v)");
  if (!rc) rc = cfail(cudaMalloc(&m->wh, o * sizeof(__nv_bfloat16)), "cudaMalloc(MLP bf16)");
  if (!rc) rc = cfail(cudaMemcpy(m->w, w.data(), o * sizeof(float), cudaMemcpyHostToDevice), "MLP upload");
  if (!rc) rc = cfail(cudaMemset(m->m, 0, o * sizeof(float)), "MLP memset");
  if (!rc) rc = cfail(cudaMemset(m->v, 0, o * sizeof(float)), "MLP memset");
  if (!rc) rc = cfail(cudaMemset(m->g, 0, o * sizeof(float)), "MLP memset");
  if (!rc) {
    dgm::to_bf16<<<256, 256>>>(m->w, m->wh, o);
    ++m->wh_version;
    rc = cfail(cudaDeviceSynchronize(), "MLP init");
  }
  if (rc) {
    free_mlp(m);
    return rc;
  }
  *out = m;
  return DG_OK;
}

int dg_mlp_destroy(dg_mlp* m) {
  free_mlp(m);
  return DG_OK;
}

int dg_mlp_dims(const dg_mlp* m, int32_t* k, int32_t* kin, int32_t* kin_padded, int32_t* out_padded,
                int64_t* nparam) {
  if (!m) {
    set_error("dg_mlp_dims: null");
    return DG_ERR_INVALID_ARG;
  }
  if (k) *k = m->k;
  if (kin) *kin = m->d.kin;
  if (kin_padded) *kin_padded = m->d.kinp;
  if (out_padded) *out_padded = m->d.outp;
  if (nparam) *nparam = m->nparam;
  return DG_OK;
}

int dg_mlp_params(dg_mlp* m, float* host, int32_t direction, float* t_scale) {
  // direction 0: device -> host (weights), 1: host -> device (weights, BF16 copy refreshed),
  // 2: device -> host (last gradient)
  if (!m || !host || direction < 0 || direction > 2) {
    set_error("dg_mlp_params: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  const size_t bytes = m->nparam * sizeof(float);
  int rc = 0;
  if (direction == 0) rc = cfail(cudaMemcpy(host, m->w, bytes, cudaMemcpyDeviceToHost), "MLP download");
  if (direction == 2) rc = cfail(cudaMemcpy(host, m->g, bytes, cudaMemcpyDeviceToHost), "MLP grad download");
  if (direction == 1) {
    rc = cfail(cudaMemcpy(m->w, host, bytes, cudaMemcpyHostToDevice), "MLP upload");
    if (!rc) {
      dgm::to_bf16<<<256, 256>>>(m->w, m->wh, m->nparam);
      ++m->wh_version;
      rc = cfail(cudaDeviceSynchronize(), "MLP bf16 refresh");
    }
    if (!rc && t_scale) m->t_scale = *t_scale;
  } else if (t_scale) {
    *t_scale = m->t_scale;
  }
  return rc;
}

int dg_mlp_param_offsets(const dg_mlp* m, int64_t* offsets6) {
  if (!m || !offsets6) {
    set_error("dg_mlp_param_offsets: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  for (int i = 0; i < 6; ++i) offsets6[i] = m->off[i];
  return DG_OK;
}

int dg_mlp_features(const dg_mlp* m, const dg_handle* h, const void* r, int32_t precision, const int32_t* cells,
                    int64_t rows, void* X, float* scale, void* stream) {
  if (!m || !h || !r || !X || !scale || (precision != DG_F64 && precision != DG_F32) ||
      h->N * h->N * h->N != m->d.nb || h->td) {
    set_error("dg_mlp_features: bad arguments, degree mismatch, or a tensor-diffusion handle (the features use "
              "the scalar log D of each cell)");
    return DG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t n = cells ? rows : h->ncell;
  auto* Xb = static_cast<__nv_bfloat16*>(X);
  if (precision == DG_F64)
    dgm::mlp_features<double><<<sm_count() * 8, 256, 0, s>>>(static_cast<const double*>(r), static_cast<const double*>(h->p64.D),
                                                      h->n[0], h->n[1], h->n[2], cells, n, m->d.nb, m->d.kinp,
                                                      m->t_scale, Xb, scale);
  else
    dgm::mlp_features<float><<<sm_count() * 8, 256, 0, s>>>(static_cast<const float*>(r), static_cast<const double*>(h->p64.D),
                                                     h->n[0], h->n[1], h->n[2], cells, n, m->d.nb, m->d.kinp,
                                                     m->t_scale, Xb, scale);
  return cfail(cudaGetLastError(), "MLP features");
}

int dg_mlp_pairs(dg_mlp* m, dg_handle* h, const double* x, const double* xstar, const int32_t* cells,
                 const int32_t* rows, int64_t count, int32_t subtract_block_jacobi, void* X, float* E, void* stream) {
  if (!m || !h || !x || !xstar || !cells || !rows || !X || !E || count < 0 || h->N * h->N * h->N != m->d.nb ||
      h->td) {
    set_error("dg_mlp_pairs: bad arguments, degree mismatch, or a tensor-diffusion handle");
    return DG_ERR_INVALID_ARG;
  }
  if (subtract_block_jacobi && !h->bj64 && !h->fdm.built) {
    set_error("dg_mlp_pairs: subtract_block_jacobi needs dg_precond_setup first");
    return DG_ERR_INVALID_ARG;
  }
  if (count == 0) return DG_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const size_t ndof = (size_t)h->ncell * m->d.nb;
  if (int rc = ensure_ws(m, (subtract_block_jacobi ? 2 : 1) * ndof * sizeof(double))) return rc;
  double* y = static_cast<double*>(m->ws);
  double* bjy = subtract_block_jacobi ? y + ndof : nullptr;
  if (int rc = launch_apply_f64(h, x, y, 1, 3, s)) return rc;  // y = A x - F
  if (bjy)
    if (int rc = precond_bj_f64(h, y, bjy, s)) return rc;
  dgm::mlp_pairs<<<sm_count() * 8, 256, 0, s>>>(y, x, xstar, bjy, static_cast<const double*>(h->p64.D), h->n[0],
                                                 h->n[1], h->n[2], cells, rows, count, m->d.nb, m->d.kinp,
                                                 static_cast<__nv_bfloat16*>(X), E);
  return cfail(cudaGetLastError(), "MLP training pairs");
}

int dg_mlp_normalize_targets(dg_mlp* m, float* E, int64_t rows, float* t_scale, void* stream) {
  if (!m || !E || rows < 1) {
    set_error("dg_mlp_normalize_targets: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  constexpr int B = 256;
  if (int rc = ensure_ws(m, B * sizeof(double))) return rc;
  double* part = static_cast<double*>(m->ws);
  const int64_t n = rows * m->d.nb;
  dgm::sum_squares<<<B, 256, 0, s>>>(E, n, part);
  std::vector<double> h(B);
  if (int rc = cfail(cudaMemcpyAsync(h.data(), part, B * sizeof(double), cudaMemcpyDeviceToHost, s), "RMS copy"))
    return rc;
  if (int rc = cfail(cudaStreamSynchronize(s), "RMS sync")) return rc;
  double tot = 0.0;
  for (double v : h) tot += v;
  const double rms = std::sqrt(tot / (double)n);
  if (!std::isfinite(rms)) {
    set_error("dg_mlp_normalize_targets: non-finite targets");
    return DG_ERR_NAN;
  }
  if (rms > 0) {
    dgm::scale_in_place<<<sm_count() * 8, 256, 0, s>>>(E, n, (float)(1.0 / rms));
    if (int rc = cfail(cudaGetLastError(), "target scaling")) return rc;
    m->t_scale = (float)rms;
  }
  if (t_scale) *t_scale = m->t_scale;
  return DG_OK;
}

int dg_mlp_forward(const dg_mlp* m, const void* X, int64_t rows, float* Y, void* stream) {
  if (!m || !X || !Y || rows < 0) {
    set_error("dg_mlp_forward: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  dgm::FwdArgs a = fwd_args(m, static_cast<const __nv_bfloat16*>(X), rows);
  a.Y = Y;
  return launch_forward(m, a, static_cast<cudaStream_t>(stream));
}

int dg_mlp_loss_grad(dg_mlp* m, const void* X, const float* T, int64_t rows, double* loss, void* stream) {
  if (!m || !X || !T || rows < 1) {
    set_error("dg_mlp_loss_grad: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  return loss_and_grad(m, static_cast<const __nv_bfloat16*>(X), T, rows, loss, static_cast<cudaStream_t>(stream));
}

int dg_mlp_train(dg_mlp* m, const void* X, const float* T, int64_t rows, const dg_mlp_train_opts* o,
                 dg_mlp_train_stats* st, void* stream) {
  if (!m || !X || !T || !o || rows < 1 || o->batch < 1 || o->epochs < 1 || !(o->lr > 0)) {
    set_error("dg_mlp_train: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const auto* Xb = static_cast<const __nv_bfloat16*>(X);
  const int64_t nbatch = rows / o->batch;
  if (nbatch < 1) {
    set_error("dg_mlp_train: fewer rows than one batch");
    return DG_ERR_INVALID_ARG;
  }
  double first = -1, last = 0;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < o->epochs; ++ep) {
    double sum = 0;
    for (int64_t bi = 0; bi < nbatch; ++bi) {
      double loss = 0;
      const int64_t r0 = bi * o->batch;
      int rc = loss_and_grad(m, Xb + r0 * m->d.kinp, T + r0 * m->d.nb, o->batch, &loss, s);
      if (rc) return rc;
      if (!std::isfinite(loss)) {
        set_error("dg_mlp_train: non-finite loss");
        return DG_ERR_NAN;
      }
      sum += loss;
      ++m->adam_t;
      const float c1 = 1.f - std::pow(b1, (float)m->adam_t), c2 = 1.f - std::pow(b2, (float)m->adam_t);
      dgm::adam_step<<<512, 256, 0, s>>>(m->w, m->g, m->m, m->v, m->nparam, (float)o->lr, b1, b2, eps, c1, c2, m->wh);
      ++m->wh_version;
      if ((rc = cfail(cudaGetLastError(), "Adam step"))) return rc;
    }
    const double mean = sum / nbatch;
    if (ep == 0) first = mean;
    last = mean;
  }
  if (st) {
    st->first_epoch_loss = first;
    st->last_epoch_loss = last;
    st->steps = m->adam_t;
  }
  return cfail(cudaStreamSynchronize(s), "dg_mlp_train sync");
}

int dg_mlp_set_target_scale(dg_mlp* m, float t_scale) {
  if (!m || !(t_scale > 0) || !std::isfinite(t_scale)) {
    set_error("dg_mlp_set_target_scale: scale must be finite and > 0");
    return DG_ERR_INVALID_ARG;
  }
  m->t_scale = t_scale;
  return DG_OK;
}

}  // extern "C"

namespace dgi {
int mlp_apply_impl(dg_mlp* m, const dg_handle* h, const void* r, void* z, int32_t precision, int accumulate,
                   cudaStream_t s);
}

extern "C" {

int dg_mlp_apply(dg_mlp* m, const dg_handle* h, const void* r, void* z, int32_t precision, void* stream) {
  return dgi::mlp_apply_impl(m, h, r, z, precision, 0, static_cast<cudaStream_t>(stream));
}

int dg_mlp_apply_add(dg_mlp* m, const dg_handle* h, const void* r, void* z, int32_t precision, void* stream) {
  return dgi::mlp_apply_impl(m, h, r, z, precision, 1, static_cast<cudaStream_t>(stream));
}

}  // extern "C"

int dgi::mlp_apply_impl(dg_mlp* m, const dg_handle* h, const void* r, void* z, int32_t precision, int accumulate,
                        cudaStream_t s) {
  void* stream = s;
  if (!m || !h || !r || !z || r == z || (precision != DG_F64 && precision != DG_F32) ||
      h->N * h->N * h->N != m->d.nb || h->td) {
    set_error("dg_mlp_apply: bad arguments, degree mismatch, or a tensor-diffusion handle");
    return DG_ERR_INVALID_ARG;
  }
  const int64_t rows = h->ncell;
  const size_t bx = (size_t)rows * m->d.kinp * sizeof(__nv_bfloat16);
  const size_t bytes = (bx + 255) / 256 * 256 + rows * sizeof(float);
  // the preconditioner keeps its own buffer (not the training workspace, which may be larger)
  if (int rc = ensure_ws(m, bytes)) return rc;
  auto* X = static_cast<__nv_bfloat16*>(m->ws);
  auto* scale = reinterpret_cast<float*>(static_cast<unsigned char*>(m->ws) + (bx + 255) / 256 * 256);
  if (int rc = dg_mlp_features(m, h, r, precision, nullptr, rows, X, scale, stream)) return rc;
  dgm::FwdArgs a = fwd_args(m, X, rows);
  a.scale = scale;
  a.z = z;
  a.z_is_f64 = precision == DG_F64;
  a.z_accumulate = accumulate;
  return launch_forward(m, a, s);
}

extern "C" {

int dg_mlp_save(const dg_mlp* m, const char* path) {
  if (!m || !path) {
    set_error("dg_mlp_save: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  std::vector<float> w(m->nparam), mm(m->nparam), vv(m->nparam);
  int rc = cfail(cudaMemcpy(w.data(), m->w, m->nparam * sizeof(float), cudaMemcpyDeviceToHost), "save");
  if (!rc) rc = cfail(cudaMemcpy(mm.data(), m->m, m->nparam * sizeof(float), cudaMemcpyDeviceToHost), "save");
  if (!rc) rc = cfail(cudaMemcpy(vv.data(), m->v, m->nparam * sizeof(float), cudaMemcpyDeviceToHost), "save");
  if (rc) return rc;
  FILE* f = std::fopen(path, "wb");
  if (!f) {
    set_error(std::string("dg_mlp_save: cannot open ") + path);
    return DG_ERR_INVALID_ARG;
  }
  const char magic[8] = {'D', 'G', 'M', 'L', 'P', '0', '1', 0};
  int64_t hdr[3] = {m->k, m->nparam, m->adam_t};
  bool ok = std::fwrite(magic, 1, 8, f) == 8 && std::fwrite(hdr, sizeof(int64_t), 3, f) == 3 &&
            std::fwrite(&m->t_scale, sizeof(float), 1, f) == 1 &&
            std::fwrite(w.data(), sizeof(float), m->nparam, f) == (size_t)m->nparam &&
            std::fwrite(mm.data(), sizeof(float), m->nparam, f) == (size_t)m->nparam &&
            std::fwrite(vv.data(), sizeof(float), m->nparam, f) == (size_t)m->nparam;
  ok = (std::fclose(f) == 0) && ok;
  if (!ok) {
    set_error("dg_mlp_save: write failed");
    return DG_ERR_INVALID_ARG;
  }
  return DG_OK;
}

int dg_mlp_load(const char* path, dg_mlp** out) {
  if (!path || !out) {
    set_error("dg_mlp_load: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  FILE* f = std::fopen(path, "rb");
  if (!f) {
    set_error(std::string("dg_mlp_load: cannot open ") + path);
    return DG_ERR_INVALID_ARG;
  }
  char magic[8];
  int64_t hdr[3];
  float ts = 1.f;
  bool ok = std::fread(magic, 1, 8, f) == 8 && std::memcmp(magic, "DGMLP01", 8) == 0 &&
            std::fread(hdr, sizeof(int64_t), 3, f) == 3 && std::fread(&ts, sizeof(float), 1, f) == 1;
  dg_mlp* m = nullptr;
  if (ok && dg_mlp_create((int32_t)hdr[0], 0, &m) == DG_OK && m->nparam == hdr[1]) {
    std::vector<float> w(m->nparam), mm(m->nparam), vv(m->nparam);
    ok = std::fread(w.data(), sizeof(float), m->nparam, f) == (size_t)m->nparam &&
         std::fread(mm.data(), sizeof(float), m->nparam, f) == (size_t)m->nparam &&
         std::fread(vv.data(), sizeof(float), m->nparam, f) == (size_t)m->nparam;
    if (ok) {
      ok = cudaMemcpy(m->w, w.data(), m->nparam * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(m->m, mm.data(), m->nparam * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess &&
           cudaMemcpy(m->v, vv.data(), m->nparam * sizeof(float), cudaMemcpyHostToDevice) == cudaSuccess;
      if (ok) {
        dgm::to_bf16<<<256, 256>>>(m->w, m->wh, m->nparam);
        ++m->wh_version;
        ok = cudaDeviceSynchronize() == cudaSuccess;
      }
      m->t_scale = ts;
      m->adam_t = hdr[2];
    }
  } else {
    ok = false;
  }
  std::fclose(f);
  if (!ok) {
    free_mlp(m);
    set_error("dg_mlp_load: bad or truncated file");
    return DG_ERR_INVALID_ARG;
  }
  *out = m;
  return DG_OK;
}

}  // extern "C"
