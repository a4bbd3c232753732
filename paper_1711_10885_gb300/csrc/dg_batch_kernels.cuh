// dg_batch_kernels.cuh -- the persistent kernels of the batched apply (dg_batch.cu), one pair per degree and
// launch variant.
//
// Each kernel takes tiles of its own degree from a work queue (a global counter, no waiting) and runs the
// cell or face code of dg_kernels.cuh on them.  A variant fixes the CTA's thread layout: cells per CTA and
// lines per thread (LPT; the threads of a cell take the lines t0, t0 + ceil(N^2 / LPT), ...).  Kernels of
// one degree carry that degree's register allocation and launch bounds only.
#pragma once

#include "dg_launch.cuh"

namespace dgbt {

constexpr int NMIN = 2, NMAX = 9;  // degrees 1..8
constexpr int NVAR = 4;            // launch variants per degree (see Variant)

struct Tabs {
  dgk::Tab<2, double> t2;
  dgk::Tab<3, double> t3;
  dgk::Tab<4, double> t4;
  dgk::Tab<5, double> t5;
  dgk::Tab<6, double> t6;
  dgk::Tab<7, double> t7;
  dgk::Tab<8, double> t8;
  dgk::Tab<9, double> t9;
};

template <int N>
__device__ __forceinline__ const dgk::Tab<N, double>& tab_of(const Tabs& t) {
  if constexpr (N == 2) return t.t2;
  else if constexpr (N == 3) return t.t3;
  else if constexpr (N == 4) return t.t4;
  else if constexpr (N == 5) return t.t5;
  else if constexpr (N == 6) return t.t6;
  else if constexpr (N == 7) return t.t7;
  else if constexpr (N == 8) return t.t8;
  else return t.t9;
}

struct Problem {
  const double* z;
  double* y;
  const double* D;
  const double* fc;
  const double* F;
  double* V;
  double* tr;
  dgk::Geo<double> geo;
  int N;
  int mode;  // 0 Jacobian, 1 residual
};

struct Tile {
  int problem, cell0, here;
};

// Variant v of degree N: (cells per CTA, lines per thread).  F = the standalone kernels' cells per CTA
// (floor(256 / N^2)): v0 (F, 1), v1 (F / 2, 1), v2 (F, 2), v3 (2 F, 2).
template <int N>
struct Variant {
  static constexpr int F = dgk::Launch<N>::CPB;
  template <int V>
  static constexpr int cpb() {
    return V == 0 ? F : V == 1 ? (F / 2 > 0 ? F / 2 : 1) : V == 2 ? F : 2 * F;
  }
  template <int V>
  static constexpr int lpt() {
    return V < 2 ? 1 : 2;
  }
  template <int V>
  static constexpr int threads() {
    return cpb<V>() * ((N * N + lpt<V>() - 1) / lpt<V>());
  }
};

__device__ __forceinline__ dgk::FaceArgs<double> face_args(const Problem& p) {
  dgk::FaceArgs<double> fa;
  fa.V = p.V;
  fa.traces = p.tr;
  fa.fc = p.fc;
  fa.F = p.F;
  for (int i = 0; i < 6; ++i) fa.g[i] = nullptr;
  fa.y = p.y;
  fa.mode = p.mode;
  fa.u = nullptr;
  fa.z0 = nullptr;
  fa.cz = fa.cu = fa.cr = 0.0;
  return fa;
}

// next tile index of this CTA from the queue counter (one atomic per tile, broadcast through shared memory)
__device__ __forceinline__ int next_tile(int* counter, int* s_tile) {
  if (threadIdx.x == 0) *s_tile = atomicAdd(counter, 1);
  __syncthreads();
  const int ti = *s_tile;
  __syncthreads();
  return ti;
}

template <int N, int V>
__global__ void __launch_bounds__(Variant<N>::template threads<V>())
batch_cell_kernel(const __grid_constant__ Tabs tabs, const Problem* __restrict__ probs,
                  const Tile* __restrict__ tiles, int ntiles, int* __restrict__ counter) {
  constexpr int CPB = Variant<N>::template cpb<V>(), LPT = Variant<N>::template lpt<V>();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_tile;
  for (;;) {
    const int ti = next_tile(counter, &s_tile);
    if (ti >= ntiles) return;
    const Tile tl = tiles[ti];
    const Problem& p = probs[tl.problem];
    dgk::cell_tile<N, double, false, CPB, double, N, false, LPT>(tab_of<N>(tabs), p.geo, p.z, p.D, p.V, p.tr, tl.cell0,
                                                                 tl.here, 0, smem);
    __syncthreads();
  }
}

template <int N, int V>
__global__ void __launch_bounds__(Variant<N>::template threads<V>())
batch_face_kernel(const __grid_constant__ Tabs tabs, const Problem* __restrict__ probs,
                  const Tile* __restrict__ tiles, int ntiles, int* __restrict__ counter) {
  constexpr int CPB = Variant<N>::template cpb<V>(), LPT = Variant<N>::template lpt<V>();
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_tile;
  for (;;) {
    const int ti = next_tile(counter, &s_tile);
    if (ti >= ntiles) return;
    const Tile tl = tiles[ti];
    const Problem& p = probs[tl.problem];
    const dgk::FaceArgs<double> fa = face_args(p);
    dgk::face_tile<N, double, false, CPB, double, N, false, true, false, false, LPT>(tab_of<N>(tabs), p.geo, fa,
                                                                                     tl.cell0, tl.here, 0, smem);
    __syncthreads();
  }
}

using KernelFn = void (*)(Tabs, const Problem*, const Tile*, int, int*);

// launch shape of one variant
struct VariantInfo {
  KernelFn cell, face;
  int cpb, lpt, threads;
  size_t smem_cell, smem_face;
};

template <int N, int V>
VariantInfo variant_info() {
  VariantInfo v;
  v.cell = &batch_cell_kernel<N, V>;
  v.face = &batch_face_kernel<N, V>;
  v.cpb = Variant<N>::template cpb<V>();
  v.lpt = Variant<N>::template lpt<V>();
  v.threads = Variant<N>::template threads<V>();
  v.smem_cell = dgi::cell_smem<N, double, Variant<N>::template cpb<V>()>();
  v.smem_face = dgi::face_smem<N, double, Variant<N>::template cpb<V>()>();
  return v;
}

template <int N>
VariantInfo variant_info_n(int v) {
  switch (v) {
    case 0: return variant_info<N, 0>();
    case 1: return variant_info<N, 1>();
    case 2: return variant_info<N, 2>();
    default: return variant_info<N, 3>();
  }
}

// degrees 1..4 (N <= 5) and 5..8 are instantiated in two translation units
VariantInfo variant_info_lo(int N, int v);
VariantInfo variant_info_hi(int N, int v);
inline VariantInfo variant_info(int N, int v) { return N <= 5 ? variant_info_lo(N, v) : variant_info_hi(N, v); }

}  // namespace dgbt
