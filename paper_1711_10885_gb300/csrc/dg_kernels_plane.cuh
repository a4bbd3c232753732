// dg_kernels_plane.cuh -- FP32 operator kernels with one thread per PLANE of a cell (the FP32 operator of the
// inner solve, Problem A: per-cell scalar D, constant b, axis-parallel cells, M = N Gauss points).  The launcher
// (dg_launch.cuh) uses them where they beat the line kernels on GB300, which is degree 5 (N = 6).
//
// The line kernels of dg_kernels.cuh give each thread one line of the cell tensor, so every 1D pass (eq.
// sum_fact_kernel) loads and stores the whole tensor through shared memory.  On the FP64 pipe that is hidden;
// the FP32 pipes issue 64x more FMAs per clock, and there the address and shared-memory instructions take most
// of the issue slots.  Here each of the N threads of a cell holds a whole plane (N^2 values) in registers:
//
//   cell kernel   plane j3 = p   : A x A along x and y (modal -> points), in registers
//                 transpose 1    -> plane i2 = p : A along z; the z and x derivative passes (pointwise flux,
//                                   transposed derivative into V), z- and x-face traces, all in registers
//                 transpose 2    -> plane i3 = p : the y derivative pass and the y-face traces
//                 transpose 3    -> plane i2 = p : the y part added to V, which is stored as planes i2
//   face kernel   plane i2 = p of V : fluxes of the x and z faces lifted onto their normal lines; the y-face
//                                   weights of the points (i1, i3 = p), contracted along x; A^T along z and x
//                 transpose      -> plane j3 = p : the y-face weights contracted along z and lifted onto the y
//                                   lines (a lift commutes with the tangential contractions), A^T along y,
//                                   minus F, stored as modal plane j3 = p
//
// Every transpose writes N-float chunks and reads whole planes as float4 rows (strides below).  The face traces
// are stored with the plane index fastest, traces[((cell * 6 + face) * 2 + {u, du}) * N^2 + p + N k] for the
// point (plane p, line k) of the face, so that the N threads of a cell touch N consecutive floats in each load
// and store.  The arithmetic is that of the line kernels (the same even-odd 1D operators, the same pointwise
// flux and face terms), so the results agree to FP32 rounding.
#pragma once

#include "dg_kernels.cuh"

namespace dgk {

// Shared-memory strides (floats), chosen by an exhaustive search over the two access patterns of a transpose
// (float4 rows read by eight consecutive threads; float2 or float chunks written by a half warp or warp) and over
// the broadcast reads of the face kernel's y-face buffer, for the fewest bank conflicts: PS between the rows of a
// cell, CS between cells (>= N * PS), GS between the y-face buffers of two cells.
constexpr int plane_ps(int N) { return N == 2 ? 16 : N == 3 ? 12 : N == 4 ? 20 : N == 5 ? 28 : N == 6 ? 40 : 52; }
constexpr int plane_cs(int N) { return N == 2 ? 36 : N == 3 ? 36 : N == 4 ? 80 : N == 5 ? 140 : N == 6 ? 260 : 364; }
constexpr int plane_gs(int N) { return N == 2 ? 18 : N == 3 ? 37 : N == 4 ? 66 : N == 5 ? 100 : N == 6 ? 146 : 196; }

template <int N>
struct PlaneCfg {
  static_assert(N >= 2 && N <= 7, "plane kernels: degrees 1..6");
  static constexpr int CPB = 128 / N;         // cells per CTA: about 128 threads, so that several CTAs (each
                                              // loading, computing or storing) share an SM
  static constexpr int THREADS = CPB * N;
  static constexpr int NN = N * N;
  static constexpr int PS = plane_ps(N);
  static constexpr int CS = plane_cs(N);
  static constexpr int GS = plane_gs(N);
  static_assert(PS >= NN && PS % 4 == 0 && CS >= N * PS && CS % 4 == 0 && GS >= 4 * NN, "plane strides");
  static constexpr bool VEC = (NN % 4) == 0;  // modal planes in global memory are float4-aligned
};

// The basis at the points in full, A[i][j] = theta_j(xi_i) (the face kernel indexes one column of it by thread).
template <int N>
struct PlaneTab {
  float A[N][N];
};

// ---- register-plane helpers (all indices compile-time after unrolling) ----

template <int N>
__device__ __forceinline__ void rowvec_load(const float* __restrict__ src, float (&x)[N * N]) {
  if constexpr (PlaneCfg<N>::VEC) {
#pragma unroll
    for (int q = 0; q < N * N / 4; ++q) {
      const float4 v = reinterpret_cast<const float4*>(src)[q];
      x[4 * q] = v.x;
      x[4 * q + 1] = v.y;
      x[4 * q + 2] = v.z;
      x[4 * q + 3] = v.w;
    }
  } else {
#pragma unroll
    for (int q = 0; q < N * N; ++q) x[q] = src[q];
  }
}
template <int N>
__device__ __forceinline__ void rowvec_store(float* __restrict__ dst, const float (&x)[N * N]) {
  if constexpr (PlaneCfg<N>::VEC) {
#pragma unroll
    for (int q = 0; q < N * N / 4; ++q)
      reinterpret_cast<float4*>(dst)[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
  } else {
#pragma unroll
    for (int q = 0; q < N * N; ++q) dst[q] = x[q];
  }
}
// shared-memory row of PS floats (always float4-aligned, PS a multiple of 4)
template <int N>
__device__ __forceinline__ void srow_load(const float* src, float (&x)[N * N]) {
  constexpr int NN = N * N;
#pragma unroll
  for (int q = 0; q < NN / 4; ++q) {
    const float4 v = reinterpret_cast<const float4*>(src)[q];
    x[4 * q] = v.x;
    x[4 * q + 1] = v.y;
    x[4 * q + 2] = v.z;
    x[4 * q + 3] = v.w;
  }
#pragma unroll
  for (int q = NN / 4 * 4; q < NN; ++q) x[q] = src[q];
}
// chunk of N floats at dst (8-byte aligned when N is even)
template <int N>
__device__ __forceinline__ void chunk_store(float* dst, const float* x) {
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int q = 0; q < N / 2; ++q) reinterpret_cast<float2*>(dst)[q] = make_float2(x[2 * q], x[2 * q + 1]);
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) dst[q] = x[q];
  }
}
template <int N>
__device__ __forceinline__ void chunk_load(const float* src, float* x) {
  if constexpr (N % 2 == 0) {
#pragma unroll
    for (int q = 0; q < N / 2; ++q) {
      const float2 v = reinterpret_cast<const float2*>(src)[q];
      x[2 * q] = v.x;
      x[2 * q + 1] = v.y;
    }
  } else {
#pragma unroll
    for (int q = 0; q < N; ++q) x[q] = src[q];
  }
}

// line helpers on a plane stored row-major as P[b * N + a]: "rows" are the lines along a (fixed b), "columns"
// the lines along b (fixed a)
template <int N>
__device__ __forceinline__ void get_row(const float (&P)[N * N], int b, float (&x)[N]) {
#pragma unroll
  for (int a = 0; a < N; ++a) x[a] = P[b * N + a];
}
template <int N>
__device__ __forceinline__ void put_row(float (&P)[N * N], int b, const float (&x)[N]) {
#pragma unroll
  for (int a = 0; a < N; ++a) P[b * N + a] = x[a];
}
template <int N>
__device__ __forceinline__ void get_col(const float (&P)[N * N], int a, float (&x)[N]) {
#pragma unroll
  for (int b = 0; b < N; ++b) x[b] = P[b * N + a];
}
template <int N>
__device__ __forceinline__ void put_col(float (&P)[N * N], int a, const float (&x)[N]) {
#pragma unroll
  for (int b = 0; b < N; ++b) P[b * N + a] = x[b];
}

// One derivative pass on a point line u (eq. gauss_points / evalblf): c = B [w_perp (sa d_r u + sb u)] added to v
// (FIRST: v = sc w u + c, the reaction), and the face traces of the line: t[0] = u(0), t[1] = du/dxi(0),
// t[2] = u(1), t[3] = du/dxi(1).  Same operations as deriv_line.
template <int N, bool FIRST>
__device__ __forceinline__ void deriv_pl(const TabNM<N, N, float>& tb, const float (&u)[N], float (&v)[N], float sa,
                                         float sb, float sc, float (&t)[4]) {
  constexpr int H = N / 2, C = (N + 1) / 2;
  float s[C], d[H > 0 ? H : 1], gr[N], X[N];
  split_sd<N, float>(u, s, d);
  eo_anti<N, float>(tb.DHm, tb.DHp, s, d, gr);
#pragma unroll
  for (int i = 0; i < N; ++i) X[i] = fmaf(sa, gr[i], sb * u[i]);
  float xs[C], xd[H > 0 ? H : 1], c[N];
  split_sd<N, float>(X, xs, xd);
  eo_anti<N, float>(tb.BHm, tb.BHp, xs, xd, c);
  if (FIRST) {
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] = fmaf(sc * tb.w[l], u[l], c[l]);
  } else {
#pragma unroll
    for (int l = 0; l < N; ++l) v[l] += c[l];
  }
  float t1 = 0.f, t2 = 0.f, q1 = 0.f, q2 = 0.f;
#pragma unroll
  for (int l = 0; l < C; ++l) {
    t1 = fmaf(tb.LS[l], s[l], t1);
    q1 = fmaf(tb.PS[l], s[l], q1);
  }
#pragma unroll
  for (int l = 0; l < H; ++l) {
    t2 = fmaf(tb.LD[l], d[l], t2);
    q2 = fmaf(tb.PD[l], d[l], q2);
  }
  t[0] = t1 - t2;
  t[1] = q2 - q1;
  t[2] = t1 + t2;
  t[3] = q1 + q2;
}

// ---------------------------------------------------------------------------------------------
// Cell kernel (plane form).  Outputs: V as planes i2, Vout[(cell * N + i2) * N^2 + i1 + N i3], and the traces with
// the plane index fastest: x faces (i2, i3) at i2 + N i3, y faces (i1, i3) at i3 + N i1, z faces (i1, i2) at
// i2 + N i1.
// ---------------------------------------------------------------------------------------------
template <int N>
__global__ void __launch_bounds__(PlaneCfg<N>::THREADS)
dg_cell_kernel_pl(const __grid_constant__ TabNM<N, N, float> tb, const __grid_constant__ Geo<float> g,
                  const float* __restrict__ z, const float* __restrict__ Dcell, float* __restrict__ Vout,
                  float* __restrict__ traces, const int* __restrict__ cells, int count) {
  using C = PlaneCfg<N>;
  constexpr int NN = N * N, PS = C::PS;
  extern __shared__ __align__(16) float smp[];
  const int lc = threadIdx.x / N, p = threadIdx.x - lc * N;
  // the cells of this CTA: positions blockIdx.x * CPB + lc of the list `cells` (null: every cell, count = ncell)
  const int pos = blockIdx.x * C::CPB + lc;
  const bool active = pos < count;
  const int cell = cells ? (active ? cells[pos] : 0) : pos;
  float* rows = smp + lc * C::CS;  // this cell's N rows of PS floats
  float U[NN], V[NN];

  // modal plane j3 = p: U[j2 * N + j1]; modal -> points along x (rows) and y (columns)
  if (active) {
    rowvec_load<N>(z + ((size_t)cell * N + p) * NN, U);
  } else {
#pragma unroll
    for (int q = 0; q < NN; ++q) U[q] = 0.f;
  }
#pragma unroll
  for (int b = 0; b < N; ++b) {
    float x[N], y[N];
    get_row<N>(U, b, x);
    eo_fwd<N, N, float>(tb, x, y);
    put_row<N>(U, b, y);
  }
#pragma unroll
  for (int a = 0; a < N; ++a) {
    float x[N], y[N];
    get_col<N>(U, a, x);
    eo_fwd<N, N, float>(tb, x, y);
    put_col<N>(U, a, y);
  }
  // transpose 1: row i2 holds (i1, j3) at i1 + N j3; this thread writes the chunk j3 = p of every row
#pragma unroll
  for (int b = 0; b < N; ++b) chunk_store<N>(rows + b * PS + N * p, U + b * N);
  __syncthreads();
  // plane i2 = p: U[j3 * N + i1]; modal -> points along z (columns) gives U[i3 * N + i1]
  srow_load<N>(rows + p * PS, U);
#pragma unroll
  for (int a = 0; a < N; ++a) {
    float x[N], y[N];
    get_col<N>(U, a, x);
    eo_fwd<N, N, float>(tb, x, y);
    put_col<N>(U, a, y);
  }
  const float DT = active ? Dcell[cell] : 0.f;
  float* trc = traces + (size_t)(active ? cell : 0) * 12 * NN;
  // z derivative pass on the z-lines (columns a = i1) with the reaction: face points (a, p)
  // (faces 4 (z-) and 5 (z+): (u, du) of face 4 at slots 0, 1, of face 5 at slots 2, 3)
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const float wperp = tb.w[a] * tb.w[p];
    float u[N], v[N], t[4];
    get_col<N>(U, a, u);
    deriv_pl<N, true>(tb, u, v, wperp * (DT * g.alpha[2]), wperp * g.beta[2], wperp * g.creact, t);
    put_col<N>(V, a, v);
    if (active) {
#pragma unroll
      for (int q = 0; q < 4; ++q) trc[(8 + q) * NN + p + N * a] = t[q];
    }
  }
  // x derivative pass on the x-lines (rows b = i3): face points (p, b)
#pragma unroll
  for (int b = 0; b < N; ++b) {
    const float wperp = tb.w[p] * tb.w[b];
    float u[N], v[N], t[4];
    get_row<N>(U, b, u);
    get_row<N>(V, b, v);
    deriv_pl<N, false>(tb, u, v, wperp * (DT * g.alpha[0]), wperp * g.beta[0], 0.f, t);
    put_row<N>(V, b, v);
    if (active) {
#pragma unroll
      for (int q = 0; q < 4; ++q) trc[q * NN + p + N * b] = t[q];
    }
  }
  __syncthreads();  // every row of transpose 1 has been read
  // transpose 2: row i3 holds (i1, i2) at i1 + N i2; this thread writes the chunk i2 = p of every row
#pragma unroll
  for (int b = 0; b < N; ++b) chunk_store<N>(rows + b * PS + N * p, U + b * N);
  __syncthreads();
  // plane i3 = p: U[i2 * N + i1]; y derivative pass on the y-lines (columns a = i1): face points (a, p)
  srow_load<N>(rows + p * PS, U);
#pragma unroll
  for (int a = 0; a < N; ++a) {
    const float wperp = tb.w[a] * tb.w[p];
    float u[N], c[N], t[4];
    get_col<N>(U, a, u);
#pragma unroll
    for (int l = 0; l < N; ++l) c[l] = 0.f;
    deriv_pl<N, false>(tb, u, c, wperp * (DT * g.alpha[1]), wperp * g.beta[1], 0.f, t);
    put_col<N>(U, a, c);  // U now holds the y contribution to V
    if (active) {
#pragma unroll
      for (int q = 0; q < 4; ++q) trc[(4 + q) * NN + p + N * a] = t[q];
    }
  }
  __syncthreads();  // every row of transpose 2 has been read
  // transpose 3: row i2 holds (i1, i3) at i1 + N i3; this thread (i3 = p) writes the chunk i3 = p of every row
#pragma unroll
  for (int b = 0; b < N; ++b) chunk_store<N>(rows + b * PS + N * p, U + b * N);
  __syncthreads();
  srow_load<N>(rows + p * PS, U);  // plane i2 = p of the y contribution, U[i3 * N + i1]
#pragma unroll
  for (int q = 0; q < NN; ++q) V[q] += U[q];
  if (active) rowvec_store<N>(Vout + ((size_t)cell * N + p) * NN, V);
}

// Face terms of one face point (eq. blf), the interior and boundary branches of face_weights for a constant
// velocity and scalar D: own trace (uo, dO), neighbour trace (un, dn), coefficients c3 of the face, normal
// velocity bq; returns the value weight Vf and the normal-derivative weight Wf of the test functions.
__device__ __forceinline__ void face_point_pl(const float* __restrict__ c3, bool boundary, int s, float bq,
                                              float wf, float uo, float dO, float un, float dn, float& Vf,
                                              float& Wf) {
  const float a0 = c3[0], a1 = c3[1], gam = c3[2];
  if (!boundary) {
    const float um = s ? uo : un, up = s ? un : uo;
    const float jump = um - up;
    const float avg = fmaf(a0, dO, a1 * dn);         // nu . {D grad u}_w
    const float phi = bq * (bq >= 0.f ? um : up);    // upwind flux
    const float H = fmaf(gam, jump, phi - avg);
    Vf = s ? wf * H : -wf * H;
    Wf = -wf * a0 * jump;
  } else {
    // the side's type is in the coefficients (a1 weights the upwind flux; Neumann / outflow: a0 = gam = 0)
    const float sgn = s ? 1.f : -1.f;
    const float bnu = sgn * bq;
    const float phi = bnu >= 0.f ? bnu * uo : 0.f;
    Vf = wf * (a1 * phi - sgn * a0 * dO + gam * uo);
    Wf = -wf * sgn * a0 * uo;
  }
}

// the neighbour across face (dir, s) of a cell at grid position ic (with PER, a periodic axis wraps around)
template <bool PER>
__device__ __forceinline__ int neighbour_pl(const Geo<float>& g, int cell, const int (&ic)[3], int dir, int s,
                                            bool at_end) {
  const int nstride = dir == 0 ? 1 : (dir == 1 ? g.n[0] : g.n[0] * g.n[1]);
  if (!PER) return s ? cell + nstride : cell - nstride;
  const int nwrap = (g.n[dir] - 1) * nstride;
  return s ? (at_end ? cell - nwrap : cell + nstride) : (at_end ? cell + nwrap : cell - nstride);
}

// Face weights of the N points (plane p, line k = 0 .. N-1) of face (dir, s) that this thread handles, stored at
// p + N k, with wf_k = area * w * w of the point given by the caller in wf[].
//
// own_zero: the cell's own traces are taken as zero (the operator applied to a vector that vanishes on this cell's
// colour); so is a neighbour across a periodic wrap of odd length, which has the cell's own colour.
template <int N, bool PER>
__device__ __forceinline__ void face_row_pl(const Geo<float>& g, const FaceArgs<float, float>& fa, int cell,
                                            const int (&ic)[3], int dir, int s, int p, const float (&wf)[N],
                                            float (&Vf)[N], float (&Wf)[N], bool own_zero = false) {
  constexpr int NN = N * N;
  const int face = 2 * dir + s;
  const bool at_end = s ? (ic[dir] == g.n[dir] - 1) : (ic[dir] == 0);
  const bool boundary = at_end && !(PER && g.periodic[dir]);
  const bool nb_zero = own_zero && at_end && (g.n[dir] & 1);
  const float* c3 = fa.fc + ((size_t)cell * 6 + face) * 3;
  const float* tro = fa.traces + ((size_t)cell * 6 + face) * 2 * NN + p;
  float uo[N], dO[N], un[N], dn[N];
#pragma unroll
  for (int k = 0; k < N; ++k) {
    uo[k] = own_zero ? 0.f : tro[N * k];
    dO[k] = own_zero ? 0.f : tro[NN + N * k];
  }
  if (!boundary && !nb_zero) {
    const int nb = neighbour_pl<PER>(g, cell, ic, dir, s, at_end);
    const float* trn = fa.traces + ((size_t)nb * 6 + (2 * dir + 1 - s)) * 2 * NN + p;
#pragma unroll
    for (int k = 0; k < N; ++k) {
      un[k] = trn[N * k];
      dn[k] = trn[NN + N * k];
    }
  } else {
#pragma unroll
    for (int k = 0; k < N; ++k) un[k] = dn[k] = 0.f;
  }
  const float bq = g.b[dir];
#pragma unroll
  for (int k = 0; k < N; ++k) face_point_pl(c3, boundary, s, bq, wf[k], uo[k], dO[k], un[k], dn[k], Vf[k], Wf[k]);
}

// ---------------------------------------------------------------------------------------------
// Face kernel (plane form): reads V as planes i2 (dg_cell_kernel_pl) and the traces; y = A z (mode 0) or A z - F
// (mode 1) as modal planes j3.
// ---------------------------------------------------------------------------------------------
template <int N, bool PER>
__global__ void __launch_bounds__(PlaneCfg<N>::THREADS)
dg_face_kernel_pl(const __grid_constant__ TabNM<N, N, float> tb, const __grid_constant__ PlaneTab<N> pt,
                  const __grid_constant__ Geo<float> g, const __grid_constant__ FaceArgs<float, float> fa,
                  const int* __restrict__ cells, int count, int own_zero) {
  using C = PlaneCfg<N>;
  constexpr int NN = N * N, PS = C::PS;
  extern __shared__ __align__(16) float smp[];
  const int lc = threadIdx.x / N, p = threadIdx.x - lc * N;
  // positions of the list `cells` (null: every cell); own_zero (mode 0 only): the cell's own V and traces are
  // taken as zero, so y on the listed cells is the coupling to the other colour (the off-diagonal blocks)
  const int pos = blockIdx.x * C::CPB + lc;
  const bool active = pos < count;
  const int cell = active ? (cells ? cells[pos] : pos) : 0;  // inactive threads work on cell 0 and store nothing
  float* rows = smp + lc * C::CS;
  float* Gs = smp + C::CPB * C::CS + lc * C::GS;  // y-face weights [s * 2 + {V, W}][i3][j1]
  int ic[3];
  ic[0] = cell % g.n[0];
  ic[1] = (cell / g.n[0]) % g.n[1];
  ic[2] = cell / (g.n[0] * g.n[1]);
  float X[NN];
  // plane i2 = p of V: X[i3 * N + i1]
  if (own_zero) {
#pragma unroll
    for (int q = 0; q < NN; ++q) X[q] = 0.f;
  } else {
    rowvec_load<N>(fa.V + ((size_t)cell * N + p) * NN, X);
  }
  // x faces (points (i2, i3) = (p, b)) lifted onto the x-lines (rows b = i3)
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    float wf[N], Vf[N], Wf[N];
#pragma unroll
    for (int b = 0; b < N; ++b) wf[b] = g.area[0] * tb.w[p] * tb.w[b];
    face_row_pl<N, PER>(g, fa, cell, ic, 0, s, p, wf, Vf, Wf, own_zero);
#pragma unroll
    for (int b = 0; b < N; ++b)
#pragma unroll
      for (int l = 0; l < N; ++l) X[b * N + l] = fmaf(tb.L[s][l], Vf[b], fmaf(tb.P[s][l], Wf[b], X[b * N + l]));
  }
  // z faces (points (i1, i2) = (a, p)) lifted onto the z-lines (columns a = i1)
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    float wf[N], Vf[N], Wf[N];
#pragma unroll
    for (int a = 0; a < N; ++a) wf[a] = g.area[2] * tb.w[a] * tb.w[p];
    face_row_pl<N, PER>(g, fa, cell, ic, 2, s, p, wf, Vf, Wf, own_zero);
#pragma unroll
    for (int a = 0; a < N; ++a)
#pragma unroll
      for (int l = 0; l < N; ++l) X[l * N + a] = fmaf(tb.L[s][l], Vf[a], fmaf(tb.P[s][l], Wf[a], X[l * N + a]));
  }
  // y faces: weights of the points (i1, i3) = (a, p), contracted along x (points -> modes j1)
#pragma unroll
  for (int s = 0; s < 2; ++s) {
    float wf[N], Vf[N], Wf[N], gv[N], gw[N];
#pragma unroll
    for (int a = 0; a < N; ++a) wf[a] = g.area[1] * tb.w[a] * tb.w[p];
    face_row_pl<N, PER>(g, fa, cell, ic, 1, s, p, wf, Vf, Wf, own_zero);
    eo_bwd<N, N, float>(tb, Vf, gv);
    eo_bwd<N, N, float>(tb, Wf, gw);
    chunk_store<N>(Gs + ((2 * s) * N + p) * N, gv);
    chunk_store<N>(Gs + ((2 * s + 1) * N + p) * N, gw);
  }
  // points -> modes along z (columns) and x (rows): X[j3 * N + j1]
#pragma unroll
  for (int a = 0; a < N; ++a) {
    float x[N], y[N];
    get_col<N>(X, a, x);
    eo_bwd<N, N, float>(tb, x, y);
    put_col<N>(X, a, y);
  }
#pragma unroll
  for (int b = 0; b < N; ++b) {
    float x[N], y[N];
    get_row<N>(X, b, x);
    eo_bwd<N, N, float>(tb, x, y);
    put_row<N>(X, b, y);
  }
  // transpose: row j3 holds (j1, i2) at j1 + N i2; this thread writes the chunk i2 = p of every row
#pragma unroll
  for (int b = 0; b < N; ++b) chunk_store<N>(rows + b * PS + N * p, X + b * N);
  __syncthreads();
  // plane j3 = p: X[i2 * N + j1]
  srow_load<N>(rows + p * PS, X);
  // the y-face weights contracted along z for j3 = p: G[k][j1] = sum_i3 theta_p(xi_i3) Gs[k][i3][j1]
  float G[4][N];
#pragma unroll
  for (int k = 0; k < 4; ++k)
#pragma unroll
    for (int a = 0; a < N; ++a) G[k][a] = 0.f;
#pragma unroll
  for (int i3 = 0; i3 < N; ++i3) {
    const float th = pt.A[i3][p];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      float row[N];
      chunk_load<N>(Gs + (k * N + i3) * N, row);
#pragma unroll
      for (int a = 0; a < N; ++a) G[k][a] = fmaf(th, row[a], G[k][a]);
    }
  }
  // lift onto the y-lines (columns a = j1) and points -> modes along y
#pragma unroll
  for (int a = 0; a < N; ++a) {
    float x[N], y[N];
    get_col<N>(X, a, x);
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
      for (int l = 0; l < N; ++l) x[l] = fmaf(tb.L[s][l], G[2 * s][a], fmaf(tb.P[s][l], G[2 * s + 1][a], x[l]));
    eo_bwd<N, N, float>(tb, x, y);
    put_col<N>(X, a, y);
  }
  // modal plane j3 = p: X[j2 * N + j1]
  if (active) {
    const size_t off = ((size_t)cell * N + p) * NN;
    if (fa.mode == 1) {
      float F[NN];
      rowvec_load<N>(fa.F + off, F);
#pragma unroll
      for (int q = 0; q < NN; ++q) X[q] -= F[q];
    }
    rowvec_store<N>(fa.y + off, X);
  }
}

}  // namespace dgk
