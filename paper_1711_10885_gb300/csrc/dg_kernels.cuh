// dg_kernels.cuh -- sm_103a kernels of the matrix-free WSIPG operator (arXiv 1711.10885).
//
// The operator application of Algorithm 1 (Sec. 3.6) is split into two kernels
// that each own whole cells, so no output is written by two CTAs:
//
//   dg_cell_kernel  (Algorithm 1 steps 1-3 and the "evaluate" halves of 4/8)
//     z (modal)  --A x A x A-->  U  (values at the m^3 Gauss points, Sec. 3.3)
//     for every axis r:  grad_r U by the collocation derivative along r,
//       pointwise flux  x^(r) = w * (D/h_r^2 d_r u - b_r/h_r u)     (eq. gauss_points)
//       and its transposed derivative, summed into the point-space residual V
//       (eq. evalblf), plus the reaction c u
//     traces of u and of the reference normal derivative at all 6 faces,
//       extrapolated along the normal lines from U (Sec. 3.4)
//     writes V (m^3 per cell) and the traces (6 x 2 x m^2 per cell)
//
//   dg_face_kernel  (Algorithm 1 steps 4-10 "integrate" halves, and step 3's last contraction)
//     reads V and, for each of its 6 faces, its own and its neighbour's traces,
//     evaluates the interior upwind / consistency / symmetry / penalty flux or the
//     Dirichlet flux at the m^2 face points, lifts the face test weights onto the
//     normal lines of V, then contracts V back to the modal test functions with
//     A^T x A^T x A^T and optionally subtracts F (residual).
//
// Each 1D contraction (eq. sum_fact_kernel) is done by one thread on one line of
// the cell tensor held in shared memory, with the 1D matrices as kernel
// parameters (constant bank, broadcast to the warp).  The rotation between
// directions is implicit: the next pass reads lines along the next axis.
//
// Every 1D operator is applied in even-odd form: the Gauss points are symmetric
// about 1/2 and theta_j(1-x) = (-1)^j theta_j(x), so each N x N matrix splits into
// two half-size blocks acting on the symmetric and antisymmetric parts of the
// line.  That is the same product with about 40 % fewer FP64 operations, which
// is what bounds these kernels on GB300 (FP64 issue rate, not memory).
//
// N = k+1 basis functions and M Gauss points per direction.  M = N is the rule
// of the benchmark problems (q = 2p); M = N+2 is the q = 2p+4 rule of the
// transport example (Sec. 5.3).  With M > N the first passes map N modal
// values to M points and the last ones map M points back to N test functions;
// everything in between (collocation derivative, face extrapolation, lifting)
// works on M-point lines, which is exact because a degree-k polynomial is its
// own interpolant on M > k points.  VB = true reads the velocity at every
// quadrature point (a flow field b(x), Sec. 5.3) instead of one constant b.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "dg_dfloat.cuh"

namespace dgk {

// 1D tables for N = k+1 modes and M Gauss points (Sec. 3.1), in even-odd form.  HN = floor(N/2),
// CN = ceil(N/2), and HM, CM likewise for the M points (point pairs i, M-1-i, and the middle point).
template <int N, int M, typename T>
struct TabNM {
  static constexpr int HN = N / 2, CN = (N + 1) / 2, HM = M / 2, CM = (M + 1) / 2;
  // basis at the points A[i][j] = theta_j(xi_i): AE[i][e] = A[i][2e] (i < CM), AO[i][o] = A[i][2o+1] (i < HM)
  T AE[CM][CN];
  T AO[HM][HN];
  // collocation derivative X[i][l] = l_l'(xi_i) (Lagrange basis on the M Gauss points) and the weighted
  // transpose B[l][i] = w_i X[i][l]; both satisfy X[M-1-i][M-1-l] = -X[i][l].  Half blocks:
  //   XHm[i][l] = (X[i][l] - X[i][M-1-l]) / 2  (i < CM, l < HM),  XHp[i][l] = (X[i][l] + X[i][M-1-l]) / 2  (i < HM, l < CM)
  T DHm[CM][HM];
  T DHp[HM][CM];
  T BHm[CM][HM];
  T BHp[HM][CM];
  // face extrapolation from a point line: value/derivative at xi = 1 are LS.s + LD.d and PS.s + PD.d,
  // at xi = 0 they are LS.s - LD.d and -PS.s + PD.d (s, d: symmetric / antisymmetric parts)
  T LS[CM], LD[HM], PS[CM], PD[HM];
  T w[M];     // Gauss weights on [0,1]
  T L[2][M];  // L[s][l] = l_l(s): lift of a face value onto the normal line
  T P[2][M];  // P[s][l] = l_l'(s): lift of a face normal-derivative weight
  T Dc[M][M]; // the collocation derivative itself, Dc[i][l] = l_l'(xi_i) (tangential derivatives on faces)
};
template <int N, typename T>
using Tab = TabNM<N, N, T>;

template <typename T>
struct Geo {
  int n[3];
  int ncell;
  T vol;       // |T| = h_x h_y h_z
  T area[3];   // |F| of a face normal to axis r
  T inv_area[3];  // 1 / |F| (conormal traces of the tensor-diffusion kernels)
  T alpha[3];  // |T| / h_r^2       (times D_T: diffusion weight of d_r u)
  T beta[3];   // -b_r |T| / h_r    (convection weight of u)
  T b[3];      // velocity
  T creact;    // c |T|
  int periodic[3];  // 1: the two end faces along this axis are one interior face (Sec. 5.3)
  int bc[6];        // boundary side 2*dir+side: 0 Dirichlet, 1 Neumann, 2 outflow (eq. modelproblem)
  // velocity field (VB kernels only, else null):
  //   bsc[((cell*3 + r)*M + l)*M^2 + t] = -b_r(x) |T| / h_r * w_a w_b at the point l of x-line/y-line/z-line t
  //     (t = a + M b over the two other point indices in increasing axis order)
  //   bface[(cell*6 + face)*M^2 + t] = b(x) . e_dir at the face points; an interior face takes the value that
  //     its lower cell (T-) holds for its upper face, so both cells see one flux
  const T* bsc;
  const T* bface;
};

// shared-memory tensor of one cell: element (i1,i2,i3) at i1 + (N+1)*(i2 + N*i3)
// (the x-lines are padded by one element so that thread-per-x-line access is conflict-free)
template <int N>
struct Lay {
  static constexpr int LS = N + 1;
  static constexpr int CS = (N + 1) * N * N;  // elements per cell buffer
  __device__ static __forceinline__ int base(int dir, int t) {
    const int a = t % N, b = t / N;
    return dir == 0 ? LS * t : (dir == 1 ? a + LS * N * b : a + LS * b);
  }
  __device__ static __forceinline__ int stride(int dir) { return dir == 0 ? 1 : (dir == 1 ? LS : LS * N); }
  __device__ static __forceinline__ int idx(int i1, int i2, int i3) { return i1 + LS * (i2 + N * i3); }
};

// Lines of the modal (N-long) passes in the M-point cell buffer: the x pass runs over (j2, j3) < N, the y
// pass over (i1 < M, j3 < N) and the z pass over (i1, i2) < M; with M = N these are the point lines.
template <int N, int M>
struct ModalLines {
  __device__ static __forceinline__ int count(int dir) { return dir == 0 ? N * N : (dir == 1 ? M * N : M * M); }
  __device__ static __forceinline__ int base(int dir, int t) {
    if constexpr (M == N) {
      return Lay<M>::base(dir, t);
    } else {
      if (dir == 0) return Lay<M>::idx(0, t % N, t / N);
      if (dir == 1) return Lay<M>::idx(t % M, 0, t / M);
      return Lay<M>::base(2, t);
    }
  }
};

// Dot products sum_i a_i b_i: plain FMA chains for float / double; the pair type has its own lazily
// normalised accumulator (dot_begin / dot_add / dot_end in dg_dfloat.cuh).
template <typename T>
struct DotAcc {
  using type = T;
};
template <>
struct DotAcc<dfl> {
  using type = dacc;
};
template <typename T>
__device__ __forceinline__ T dot_begin(T a, T b) {
  return a * b;
}
template <typename T>
__device__ __forceinline__ void dot_add(T& c, T a, T b) {
  c = fma(a, b, c);
}
template <typename T>
__device__ __forceinline__ T dot_end(const T& c) {
  return c;
}

// conversions between the vector element type TV and the compute type T
template <typename T, typename TV>
__device__ __forceinline__ T to_compute(TV v) {
  return T(v);
}
template <>
__device__ __forceinline__ dfl to_compute<dfl, double>(double v) {
  return dfl_from_double(v);
}
template <typename TV, typename T>
__device__ __forceinline__ TV from_compute(T v) {
  return static_cast<TV>(v);
}
template <>
__device__ __forceinline__ double from_compute<double, dfl>(dfl v) {
  return dfl_to_double(v);
}

template <int N, typename T>
__device__ __forceinline__ void load_line(const T* s, int base, int st, T (&x)[N]) {
#pragma unroll
  for (int l = 0; l < N; ++l) x[l] = s[base + l * st];
}
template <int N, typename T>
__device__ __forceinline__ void store_line(T* s, int base, int st, const T (&x)[N]) {
#pragma unroll
  for (int l = 0; l < N; ++l) s[base + l * st] = x[l];
}

// symmetric / antisymmetric parts of a point line: s[i] = x[i] + x[N-1-i], d[i] = x[i] - x[N-1-i]
// (i < H); for odd N the middle point goes to s[H] = x[H] unchanged.
template <int N, typename T>
__device__ __forceinline__ void split_sd(const T (&x)[N], T (&s)[(N + 1) / 2], T (&d)[N / 2 > 0 ? N / 2 : 1]) {
  constexpr int H = N / 2;
#pragma unroll
  for (int i = 0; i < H; ++i) {
    s[i] = x[i] + x[N - 1 - i];
    d[i] = x[i] - x[N - 1 - i];
  }
  if (N & 1) s[H] = x[H];
}

// modal -> points along one line: y[i] = sum_j theta_j(xi_i) x[j]   (eq. evalfe, one direction)
template <int N, int M, typename T>
__device__ __forceinline__ void eo_fwd(const TabNM<N, M, T>& tb, const T (&x)[N], T (&y)[M]) {
  constexpr int HN = N / 2, CN = (N + 1) / 2, HM = M / 2, CM = (M + 1) / 2;
  T e[CM], o[HM];
#pragma unroll
  for (int i = 0; i < CM; ++i) {
    typename DotAcc<T>::type acc = dot_begin(tb.AE[i][0], x[0]);
#pragma unroll
    for (int k = 1; k < CN; ++k) dot_add(acc, tb.AE[i][k], x[2 * k]);
    e[i] = dot_end(acc);
  }
#pragma unroll
  for (int i = 0; i < HM; ++i) {
    typename DotAcc<T>::type acc = dot_begin(tb.AO[i][0], x[1]);
#pragma unroll
    for (int k = 1; k < HN; ++k) dot_add(acc, tb.AO[i][k], x[2 * k + 1]);
    o[i] = dot_end(acc);
  }
#pragma unroll
  for (int i = 0; i < HM; ++i) {
    y[i] = e[i] + o[i];
    y[M - 1 - i] = e[i] - o[i];
  }
  if (M & 1) y[HM] = e[HM];
}

// points -> modal along one line: y[j] = sum_i theta_j(xi_i) x[i]   (test functions, eq. evalblf)
template <int N, int M, typename T>
__device__ __forceinline__ void eo_bwd(const TabNM<N, M, T>& tb, const T (&x)[M], T (&y)[N]) {
  constexpr int HN = N / 2, CN = (N + 1) / 2, HM = M / 2, CM = (M + 1) / 2;
  T s[CM], d[HM];
  split_sd<M, T>(x, s, d);
#pragma unroll
  for (int k = 0; k < CN; ++k) {
    typename DotAcc<T>::type acc = dot_begin(tb.AE[0][k], s[0]);
#pragma unroll
    for (int i = 1; i < CM; ++i) dot_add(acc, tb.AE[i][k], s[i]);
    y[2 * k] = dot_end(acc);
  }
#pragma unroll
  for (int k = 0; k < HN; ++k) {
    typename DotAcc<T>::type acc = dot_begin(tb.AO[0][k], d[0]);
#pragma unroll
    for (int i = 1; i < HM; ++i) dot_add(acc, tb.AO[i][k], d[i]);
    y[2 * k + 1] = dot_end(acc);
  }
}

// points -> points with a centro-antisymmetric matrix X given by its half blocks (Hm, Hp), from the
// split parts (s, d) of the input line: out[i] = Gp[i] + Gm[i], out[N-1-i] = Gp[i] - Gm[i].
template <int N, typename T>
__device__ __forceinline__ void eo_anti(const T (&Hm)[(N + 1) / 2][N / 2], const T (&Hp)[N / 2][(N + 1) / 2],
                                        const T (&s)[(N + 1) / 2], const T (&d)[N / 2], T (&out)[N]) {
  constexpr int H = N / 2, C = (N + 1) / 2;
  T gp[C], gm[H];
#pragma unroll
  for (int i = 0; i < C; ++i) {
    typename DotAcc<T>::type acc = dot_begin(Hm[i][0], d[0]);
#pragma unroll
    for (int l = 1; l < H; ++l) dot_add(acc, Hm[i][l], d[l]);
    gp[i] = dot_end(acc);
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    typename DotAcc<T>::type acc = dot_begin(Hp[i][0], s[0]);
#pragma unroll
    for (int l = 1; l < C; ++l) dot_add(acc, Hp[i][l], s[l]);
    gm[i] = dot_end(acc);
  }
#pragma unroll
  for (int i = 0; i < H; ++i) {
    out[i] = gp[i] + gm[i];
    out[N - 1 - i] = gp[i] - gm[i];
  }
  if (N & 1) out[H] = gp[H];
}

template <int N>
struct Launch {
  static constexpr int NN = N * N;
  static constexpr int CPB = (256 / NN) > 0 ? (256 / NN) : 1;  // cells per CTA
  static constexpr int THREADS = CPB * NN;
};

// copy cpb cells (contiguous in global memory, N^3 each) into padded shared buffers laid out for M points
// per direction (the N^3 values take the corner j1, j2, j3 < N)
// (TV: element type of the vector in global memory, converted to the compute type T on load)
template <int N, typename T, typename TV, int M = N>
__device__ __forceinline__ void gload_cells(T* sbuf, const TV* __restrict__ g, int cell0, int ncells_here) {
  constexpr int N3 = N * N * N;
  const int total = ncells_here * N3;
  const TV* src = g + (size_t)cell0 * N3;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int c = e / N3, r = e - c * N3;
    const int i1 = r % N, i23 = r / N;
    if constexpr (M == N) {
      sbuf[c * Lay<M>::CS + i1 + Lay<M>::LS * i23] = to_compute<T, TV>(src[e]);
    } else {
      sbuf[c * Lay<M>::CS + Lay<M>::idx(i1, i23 % N, i23 / N)] = to_compute<T, TV>(src[e]);
    }
  }
}
template <int N, typename T>
__device__ __forceinline__ void gstore_cells(T* __restrict__ g, const T* sbuf, int cell0, int ncells_here) {
  constexpr int N3 = N * N * N;
  const int total = ncells_here * N3;
  T* dst = g + (size_t)cell0 * N3;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int c = e / N3, r = e - c * N3;
    const int i1 = r % N, i23 = r / N;
    dst[e] = sbuf[c * Lay<N>::CS + i1 + Lay<N>::LS * i23];
  }
}

// One derivative pass along axis `dir` for the line u (values at the M points) owned by this thread:
// v (+)= B [ w_perp (sa d_r u + sb u) ] and the two face traces of this line.  With VB the convection
// weight is the point-wise bl[i * M^2] (pre-scaled velocity, see Geo::bsc) instead of the constant sb.
template <int N, int M, typename T, bool FIRST, bool VB = false>
__device__ __forceinline__ void deriv_line(const TabNM<N, M, T>& tb, const T (&u)[M], T (&v)[M], T sa, T sb, T sc,
                                           const T* __restrict__ bl, T* __restrict__ tr, int NN, int t) {
  constexpr int H = M / 2, C = (M + 1) / 2;
  T bv[VB ? M : 1];
  if constexpr (VB) {
#pragma unroll
    for (int i = 0; i < M; ++i) bv[i] = bl[i * M * M];
  }
  T s[C], d[H > 0 ? H : 1], gr[M], X[M];
  split_sd<M, T>(u, s, d);
  eo_anti<M, T>(tb.DHm, tb.DHp, s, d, gr);  // d u / d xi_r at the points (reference derivative)
  if constexpr (VB) {
#pragma unroll
    for (int i = 0; i < M; ++i) X[i] = fma(sa, gr[i], bv[i] * u[i]);  // eq. gauss_points, b = b(x_i)
  } else {
#pragma unroll
    for (int i = 0; i < M; ++i) X[i] = fma(sa, gr[i], sb * u[i]);  // eq. gauss_points, times w_perp
  }
  T xs[C], xd[H > 0 ? H : 1], c[M];
  split_sd<M, T>(X, xs, xd);
  eo_anti<M, T>(tb.BHm, tb.BHp, xs, xd, c);  // sum_i w_i l_l'(xi_i) X[i]
  if (FIRST) {
#pragma unroll
    for (int l = 0; l < M; ++l) v[l] = fma(sc * tb.w[l], u[l], c[l]);  // + c |T| w u (reaction)
  } else {
#pragma unroll
    for (int l = 0; l < M; ++l) v[l] += c[l];
  }
  // traces at xi_r = 1 and 0 (value, reference normal derivative), Sec. 3.4
  T t1 = T(0), t2 = T(0), q1 = T(0), q2 = T(0);
#pragma unroll
  for (int l = 0; l < C; ++l) {
    t1 = fma(tb.LS[l], s[l], t1);
    q1 = fma(tb.PS[l], s[l], q1);
  }
#pragma unroll
  for (int l = 0; l < H; ++l) {
    t2 = fma(tb.LD[l], d[l], t2);
    q2 = fma(tb.PD[l], d[l], q2);
  }
  tr[0 * NN + t] = t1 - t2;   // face xi = 0: u
  tr[1 * NN + t] = q2 - q1;   // face xi = 0: du/dxi
  tr[2 * NN + t] = t1 + t2;   // face xi = 1: u
  tr[3 * NN + t] = q1 + q2;   // face xi = 1: du/dxi
}

// ---------------------------------------------------------------------------------------------
// Kernel 1: modal -> points, volume integrand, point-space residual V, face traces
// ---------------------------------------------------------------------------------------------
// Diagonal-block mode (SELF = true): "virtual cell" vc = (cell - cell_base) * N^3 + j stands for the unit
// vector e_j supported on one real cell, with every neighbour's contribution zero; the outputs are indexed
// by vc.  This assembles the cell's diagonal block A_TT column by column with the operator's own code.
struct SelfArgs {
  int nvirt;      // number of virtual cells in this launch
  int cell_base;  // first real cell of the chunk
};

// Cell-kernel work on one tile of `here` consecutive cells starting at cell0 (virtual cells in SELF mode),
// run by all threads of the CTA (blockDim.x >= CPB * ceil(M^2 / LPT); threads beyond that only help with copies).
// LPT lines per thread: the ceil(M^2 / LPT) threads of a cell take the lines t0, t0 + ceil(M^2 / LPT), ...
template <int N, typename T, bool SELF, int CPB, typename TV = T, int M = N, bool VB = false, int LPT = 1>
__device__ __forceinline__ void cell_tile(const TabNM<N, M, T>& tb, const Geo<T>& g, const TV* __restrict__ z,
                                          const T* __restrict__ Dcell, T* __restrict__ Vout, T* __restrict__ traces,
                                          int cell0, int here, int cell_base, unsigned char* smem_raw) {
  constexpr int NN = M * M, N3 = N * N * N, CS = Lay<M>::CS, TPC = (NN + LPT - 1) / LPT;
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sV = sU + CPB * CS;
  const int lc = threadIdx.x / TPC, t0 = threadIdx.x - lc * TPC;
  const bool active = lc < here;
  const int cell = cell0 + lc;                                 // output index (virtual in SELF mode)
  const int rcell = SELF ? cell_base + cell / N3 : cell;       // real cell (coefficients)
  T* U = sU + lc * CS;
  T* V = sV + lc * CS;

  if (SELF) {
    for (int e = threadIdx.x; e < here * N3; e += blockDim.x) {
      const int c = e / N3, r = e - c * N3;
      const int j1 = r % N, j23 = r / N;
      const int pos = M == N ? j1 + Lay<M>::LS * j23 : Lay<M>::idx(j1, j23 % N, j23 / N);
      sU[c * CS + pos] = (r == (cell0 + c) % N3) ? T(1) : T(0);
    }
  } else {
    gload_cells<N, T, TV, M>(sU, z, cell0, here);
  }
  __syncthreads();

  // Sec. 3.3, eq. evalfe: u at the Gauss points, axis x then y ...
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
      const int t = t0 + l * TPC;
      if (active && t < NN && (M == N || t < ModalLines<N, M>::count(dir))) {
        T x[N], y[M];
        const int bs = ModalLines<N, M>::base(dir, t), st = Lay<M>::stride(dir);
        load_line<N>(U, bs, st, x);
        eo_fwd<N, M, T>(tb, x, y);
        store_line<M>(U, bs, st, y);
      }
    }
    __syncthreads();
  }

  const T DT = active ? Dcell[rcell] : T(0);
  T* trc = traces + (size_t)cell * 12 * NN;
  // ... then z, kept in registers for the z derivative pass (Sec. 3.2, eqs. evalblf / gauss_points):
  // V = c|T| w u + B_z [w (alpha_z D d_z u + beta_z u)], traces on the two z faces
#pragma unroll
  for (int l = 0; l < LPT; ++l) {
    const int t = t0 + l * TPC;
    if (active && t < NN) {
      const int a = t % M, b = t / M;
      const T wperp = tb.w[a] * tb.w[b];
      const T* bl = VB ? g.bsc + (size_t)rcell * 3 * M * NN + t : nullptr;
      T x[N], u[M], v[M];
      const int bs = Lay<M>::base(2, t), st = Lay<M>::stride(2);
      load_line<N>(U, bs, st, x);
      eo_fwd<N, M, T>(tb, x, u);
      store_line<M>(U, bs, st, u);
      deriv_line<N, M, T, true, VB>(tb, u, v, wperp * (DT * g.alpha[2]), wperp * g.beta[2], wperp * g.creact,
                                    VB ? bl + 2 * M * NN : nullptr, trc + 8 * NN, NN, t);
      store_line<M>(V, bs, st, v);
    }
  }
  __syncthreads();
  // x and y derivative passes accumulate into V
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
      const int t = t0 + l * TPC;
      if (active && t < NN) {
        const int a = t % M, b = t / M;
        const T wperp = tb.w[a] * tb.w[b];
        const T* bl = VB ? g.bsc + (size_t)rcell * 3 * M * NN + t : nullptr;
        T u[M], v[M];
        const int bs = Lay<M>::base(dir, t), st = Lay<M>::stride(dir);
        load_line<M>(U, bs, st, u);
        load_line<M>(V, bs, st, v);
        deriv_line<N, M, T, false, VB>(tb, u, v, wperp * (DT * g.alpha[dir]), wperp * g.beta[dir], T(0),
                                       VB ? bl + dir * M * NN : nullptr, trc + 4 * dir * NN, NN, t);
        store_line<M>(V, bs, st, v);
      }
    }
    __syncthreads();
  }
  gstore_cells<M>(Vout, sV, cell0, here);
}

// Cell-kernel work with a full diffusion metric (TD: a per-cell tensor D_T and/or an affine geometry).
// Reference coordinates: with the cell Jacobian J, K = |det J| J^{-1} D_T J^{-T} (Kc[cell][6] = K00, K11,
// K22, K01, K02, K12) and the convection vector g.beta = -|det J| J^{-1} b, the volume term of eq. blf is
//   sum_points w (K grad u + beta u) . grad v + c |det J| w u v        (gradients in reference coordinates).
// Every flux component needs all three reference derivatives, so the derivative and the transposed
// derivative passes are split: (1) three derivative passes store grad u; (2) a pointwise pass forms
// X_r = (K grad u)_r + beta_r u and the reaction; (3) three transposed passes sum B_r (w_perp X_r) into V.
// The second trace slot of each face holds the physical conormal flux nu . D grad u = (K grad u)_r / |F_r|
// (nu along +reference axis r), extrapolated from X_r.
//
// PW (coefficients given at the quadrature points, Problem B of Sec. 5.1): K, beta and c vary from point to
// point.  Kc is then the point table [cell][10][M^3] of (K00, K11, K22, K01, K02, K12, beta_0, beta_1, beta_2,
// c |det J| w) with the point index q = i1 + M (i2 + M i3) fastest, and Kf [cell][face][3][M^2] holds row r of
// K at each face point divided by |F_r| (K from the tensor at the face point itself).  The conormal traces are
// then sum_c Kf_c (grad u)_c with grad u extrapolated to the face along the normal lines; extrapolating X_r
// instead would only be exact when K grad u is a polynomial of degree < M along the line.
template <int N, typename T, int CPB, typename TV = T, int M = N, bool PW = false>
__device__ __forceinline__ void cell_tile_td(const TabNM<N, M, T>& tb, const Geo<T>& g, const TV* __restrict__ z,
                                             const T* __restrict__ Kc, const T* __restrict__ Kf,
                                             T* __restrict__ Vout, T* __restrict__ traces, int cell0, int here,
                                             unsigned char* smem_raw) {
  constexpr int NN = M * M, CS = Lay<M>::CS, H = M / 2, C = (M + 1) / 2;
  T* sU = reinterpret_cast<T*>(smem_raw);  // u, then V
  T* sG = sU + CPB * CS;                    // [3][CPB][CS]: grad u, then X
  const int lc = threadIdx.x / NN, t = threadIdx.x - lc * NN;
  const bool active = lc < here;
  const int cell = cell0 + lc;
  T* U = sU + lc * CS;
  T* G[3] = {sG + lc * CS, sG + (CPB + lc) * CS, sG + (2 * CPB + lc) * CS};

  gload_cells<N, T, TV, M>(sU, z, cell0, here);
  __syncthreads();
#pragma unroll
  for (int dir = 0; dir < 2; ++dir) {
    if (active && (M == N || t < ModalLines<N, M>::count(dir))) {
      T x[N], y[M];
      const int bs = ModalLines<N, M>::base(dir, t), st = Lay<M>::stride(dir);
      load_line<N>(U, bs, st, x);
      eo_fwd<N, M, T>(tb, x, y);
      store_line<M>(U, bs, st, y);
    }
    __syncthreads();
  }
  T* trc = traces + (size_t)cell * 12 * NN;
  T ut[3][2];  // value traces of this thread's lines, kept for the conormal traces
  // (1) z values (last modal pass), then the three derivative passes
  if (active) {
    T x[N], u[M];
    const int bs = Lay<M>::base(2, t), st = Lay<M>::stride(2);
    load_line<N>(U, bs, st, x);
    eo_fwd<N, M, T>(tb, x, u);
    store_line<M>(U, bs, st, u);
  }
  __syncthreads();
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    if (active) {
      T u[M], s[C], d[H > 0 ? H : 1], gr[M];
      const int bs = Lay<M>::base(dir, t), st = Lay<M>::stride(dir);
      load_line<M>(U, bs, st, u);
      split_sd<M, T>(u, s, d);
      eo_anti<M, T>(tb.DHm, tb.DHp, s, d, gr);
      store_line<M>(G[dir], bs, st, gr);
      T t1 = T(0), t2 = T(0);
#pragma unroll
      for (int l = 0; l < C; ++l) t1 = fma(tb.LS[l], s[l], t1);
#pragma unroll
      for (int l = 0; l < H; ++l) t2 = fma(tb.LD[l], d[l], t2);
      ut[dir][0] = t1 - t2;
      ut[dir][1] = t1 + t2;
      trc[(4 * dir + 0) * NN + t] = ut[dir][0];
      trc[(4 * dir + 2) * NN + t] = ut[dir][1];
    }
  }
  __syncthreads();
  if constexpr (PW) {
    // (1b) conormal traces nu . D grad u = sum_c Kf_c (grad u)_c at both faces of each normal line
    if (active) {
      const T* kf = Kf + (size_t)cell * 18 * NN + t;
#pragma unroll
      for (int dir = 0; dir < 3; ++dir) {
        const int bs = Lay<M>::base(dir, t), st = Lay<M>::stride(dir);
        T f0 = T(0), f1 = T(0);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          T x[M], s[C], d[H > 0 ? H : 1];
          load_line<M>(G[c], bs, st, x);
          split_sd<M, T>(x, s, d);
          T t1 = T(0), t2 = T(0);
#pragma unroll
          for (int l = 0; l < C; ++l) t1 = fma(tb.LS[l], s[l], t1);
#pragma unroll
          for (int l = 0; l < H; ++l) t2 = fma(tb.LD[l], d[l], t2);
          f0 = fma(kf[((2 * dir) * 3 + c) * NN], t1 - t2, f0);
          f1 = fma(kf[((2 * dir + 1) * 3 + c) * NN], t1 + t2, f1);
        }
        trc[(4 * dir + 1) * NN + t] = f0;
        trc[(4 * dir + 3) * NN + t] = f1;
      }
    }
    __syncthreads();
    // (2) pointwise with the coefficients of each point (coalesced: consecutive t, consecutive points)
    if (active) {
      const int a = t % M, b = t / M;
      const T* kq = Kc + (size_t)cell * 10 * M * NN + t;
      constexpr int FS = M * NN;  // stride between the ten fields
#pragma unroll 2
      for (int l = 0; l < M; ++l) {
        const int p = Lay<M>::idx(a, b, l);
        const T* q = kq + l * NN;
        const T u = U[p], g0 = G[0][p], g1 = G[1][p], g2 = G[2][p];
        const T k0 = q[0], k1 = q[FS], k2 = q[2 * FS], k3 = q[3 * FS], k4 = q[4 * FS], k5 = q[5 * FS];
        G[0][p] = fma(k0, g0, fma(k3, g1, fma(k4, g2, q[6 * FS] * u)));
        G[1][p] = fma(k3, g0, fma(k1, g1, fma(k5, g2, q[7 * FS] * u)));
        G[2][p] = fma(k4, g0, fma(k5, g1, fma(k2, g2, q[8 * FS] * u)));
        U[p] = q[9 * FS] * u;
      }
    }
  } else if (active) {
    // (2) pointwise: X_r = (K grad u)_r + beta_r u in place of grad u; V = c |det J| w u in place of u.
    // Thread t handles the points of its z-line (a, b).
    T k6[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) k6[q] = Kc[(size_t)cell * 6 + q];
    const int a = t % M, b = t / M;
    const T wab = tb.w[a] * tb.w[b];
#pragma unroll
    for (int l = 0; l < M; ++l) {
      const int p = Lay<M>::idx(a, b, l);
      const T u = U[p], g0 = G[0][p], g1 = G[1][p], g2 = G[2][p];
      G[0][p] = fma(k6[0], g0, fma(k6[3], g1, fma(k6[4], g2, g.beta[0] * u)));
      G[1][p] = fma(k6[3], g0, fma(k6[1], g1, fma(k6[5], g2, g.beta[1] * u)));
      G[2][p] = fma(k6[4], g0, fma(k6[5], g1, fma(k6[2], g2, g.beta[2] * u)));
      U[p] = g.creact * wab * tb.w[l] * u;
    }
  }
  __syncthreads();
  // (3) transposed passes V += B_r (w_perp X_r); conormal traces (X_face - beta_r u_face) / |F_r|
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    if (active) {
      T X[M], v[M], xs[C], xd[H > 0 ? H : 1], c[M];
      const int bs = Lay<M>::base(dir, t), st = Lay<M>::stride(dir);
      const int a = t % M, b = t / M;
      const T wperp = tb.w[a] * tb.w[b];
      load_line<M>(G[dir], bs, st, X);
      load_line<M>(U, bs, st, v);
      split_sd<M, T>(X, xs, xd);
      if constexpr (!PW) {
        T t1 = T(0), t2 = T(0);
#pragma unroll
        for (int l = 0; l < C; ++l) t1 = fma(tb.LS[l], xs[l], t1);
#pragma unroll
        for (int l = 0; l < H; ++l) t2 = fma(tb.LD[l], xd[l], t2);
        trc[(4 * dir + 1) * NN + t] = (t1 - t2 - g.beta[dir] * ut[dir][0]) * g.inv_area[dir];
        trc[(4 * dir + 3) * NN + t] = (t1 + t2 - g.beta[dir] * ut[dir][1]) * g.inv_area[dir];
      }
#pragma unroll
      for (int i = 0; i < C; ++i) xs[i] = wperp * xs[i];
#pragma unroll
      for (int i = 0; i < (H > 0 ? H : 1); ++i) xd[i] = wperp * xd[i];
      eo_anti<M, T>(tb.BHm, tb.BHp, xs, xd, c);
#pragma unroll
      for (int l = 0; l < M; ++l) v[l] += c[l];
      store_line<M>(U, bs, st, v);
    }
    __syncthreads();
  }
  gstore_cells<M>(Vout, sU, cell0, here);
}

template <int N, typename T, int CPB, typename TV = T, int M = N, bool PW = false>
__global__ void __launch_bounds__(CPB * M * M)
dg_cell_kernel_td(const __grid_constant__ TabNM<N, M, T> tb, const __grid_constant__ Geo<T> g,
                  const TV* __restrict__ z, const T* __restrict__ Kc, const T* __restrict__ Kf,
                  T* __restrict__ Vout, T* __restrict__ traces) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cell0 = blockIdx.x * CPB;
  const int here = min(CPB, g.ncell - cell0);
  cell_tile_td<N, T, CPB, TV, M, PW>(tb, g, z, Kc, Kf, Vout, traces, cell0, here, smem_raw);
}

template <int N, typename T, bool SELF = false, int CPB = Launch<N>::CPB, typename TV = T, int M = N, bool VB = false>
__global__ void __launch_bounds__(CPB * M * M, (N == 8 && M == 8 && sizeof(T) == 8 && !VB) ? 4 : 1)
dg_cell_kernel(const __grid_constant__ TabNM<N, M, T> tb, const __grid_constant__ Geo<T> g, const TV* __restrict__ z,
               const T* __restrict__ Dcell, T* __restrict__ Vout, T* __restrict__ traces, SelfArgs sa_) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cell0 = blockIdx.x * CPB;
  const int here = min(CPB, (SELF ? sa_.nvirt : g.ncell) - cell0);
  cell_tile<N, T, SELF, CPB, TV, M, VB>(tb, g, z, Dcell, Vout, traces, cell0, here, sa_.cell_base, smem_raw);
}

// ---------------------------------------------------------------------------------------------
// Kernel 2: face fluxes + lift + backward contraction (+ residual)
// fc[(cell*6 + face)*3 + {0,1,2}]: interior: (w_own D_own / h, w_nbr D_nbr / h, gamma_F);
//                                   boundary: (D_own / h, 0, gamma_F)
// mode 0: y = A z;  mode 1: y = A z - F;  mode 2 (right hand side): V from f, faces from g;
// mode 3 (explicit Runge-Kutta stage, Sec. 2 "ODE"): y = c_z z0 + c_u u - c_r (A u - F), u the stage input
// ---------------------------------------------------------------------------------------------
template <typename T, typename TV = T>
struct FaceArgs {
  const T* V;       // point-space residual from dg_cell_kernel (mode 0/1/3), or f at points (mode 2)
  const T* traces;  // traces from dg_cell_kernel (mode 0/1/3)
  const T* fc;      // face coefficients
  const T* F;       // right hand side (mode 1/3), in the compute type
  const T* g[6];    // Dirichlet data per boundary side (mode 2), may be null
  TV* y;            // output vector (element type TV)
  int mode;
  const TV* u;      // mode 3: the stage input (the vector the cell kernel read)
  const TV* z0;     // mode 3: the step's initial value (may be y: each element is read before it is written)
  double cz, cu, cr;  // mode 3 coefficients (the stage update runs in FP64)
};

// face test weights of this thread's face point on face (dir, s): value weight Vf and normal-derivative
// weight Wf (eq. blf: interior upwind, consistency, symmetry and penalty terms, or the Dirichlet terms;
// mode 2: the Dirichlet terms of l_h).  With PER, an axis flagged periodic has interior end faces whose
// neighbour is the cell at the other end (PER = false compiles the plain mesh only, which keeps the
// register count of the FP32 and double-float kernels down).
//
// TD (tensor diffusion / affine geometry): the face coefficients are (w_own, w_nbr, gamma, kn, kt1, kt2) with
// kn, kt = w_own (K_rr, K_r,ta, K_r,tb) / |F_r| (boundary: w_own = 1, w_nbr = 0), the second trace is the
// conormal flux nu . D grad u, and the test-function side -nu.{D grad v}_w also has tangential parts: Wt1,
// Wt2 weight the reference derivatives of v along the lower and upper tangential axes at the face point.
// PW (coefficients at the quadrature points): the six coefficients vary over the face points, stored as
// fc[((cell*6 + face)*6 + q)*M^2 + t] (the weights and the penalty from both cells' tensors at the point).
template <int N, typename T, bool SELF, typename TV, int M = N, bool VB = false, bool PER = false, bool TD = false,
          bool PW = false>
__device__ __forceinline__ void face_weights(const Geo<T>& g, const FaceArgs<T, TV>& fa, int cell, int tcell,
                                             const int (&ic)[3], int dir, int s, int t, T wf, T& Vf, T& Wf,
                                             T& Wt1, T& Wt2) {
  constexpr int NN = M * M;
  const int face = 2 * dir + s;
  const bool at_end = s ? (ic[dir] == g.n[dir] - 1) : (ic[dir] == 0);
  const bool boundary = at_end && !(PER && g.periodic[dir]);
  const int btype = boundary ? g.bc[face] : 0;  // F^D, F^N or F^O of eq. blf
  const T* c3 = PW ? fa.fc + ((size_t)cell * 6 + face) * 6 * NN + t : fa.fc + ((size_t)cell * 6 + face) * (TD ? 6 : 3);
  constexpr int CST = PW ? NN : 1;  // stride between the coefficients of one face point
  const T kn = TD ? c3[3 * CST] : c3[0];  // coefficient of the normal reference derivative of v
  // the neighbour across this face (on a periodic axis the end faces wrap around to the other end)
  auto neighbour = [&]() {
    const int nstride = dir == 0 ? 1 : (dir == 1 ? g.n[0] : g.n[0] * g.n[1]);
    const int nwrap = (g.n[dir] - 1) * nstride;
    if (!PER) return s ? cell + nstride : cell - nstride;
    return s ? (at_end ? cell - nwrap : cell + nstride) : (at_end ? cell + nwrap : cell - nstride);
  };
  // normal velocity b . e_dir at this face point (interior faces: the lower cell's upper-face value)
  T bq;
  if constexpr (VB) {
    const int owner = (boundary || s) ? cell : neighbour();
    const int oface = boundary ? face : 2 * dir + 1;
    bq = g.bface[((size_t)owner * 6 + oface) * NN + t];
  } else {
    bq = g.b[dir];
  }
  Vf = T(0);
  Wf = T(0);
  Wt1 = T(0);
  Wt2 = T(0);
  if (fa.mode == 2) {
    // Dirichlet: -(Phi(0,g,b_nu), v) - (nu.D grad v, g) + gamma (g, v); Neumann: -(j, v); outflow: nothing
    const T* gs = fa.g[face];
    if (boundary && gs != nullptr && btype != 2) {
      const int ta = dir == 0 ? 1 : 0, tbx = dir == 2 ? 1 : 2;
      const int fidx = ic[ta] + g.n[ta] * ic[tbx];
      const T gv = gs[(size_t)fidx * NN + t];
      if (btype == 1) {
        Vf = -wf * gv;
        return;
      }
      const T sgn = s ? T(1) : T(-1);
      const T bnu = sgn * bq;
      const T phi = bnu >= T(0) ? T(0) : bnu * gv;
      Vf = wf * (c3[2 * CST] * gv - phi);
      Wf = -wf * sgn * kn * gv;
      if (TD) {
        Wt1 = -wf * sgn * c3[4 * CST] * gv;
        Wt2 = -wf * sgn * c3[5 * CST] * gv;
      }
    }
    return;
  }
  const T* tro = fa.traces + ((size_t)tcell * 6 + face) * 2 * NN;
  const T uo = tro[t], dO = tro[NN + t];
  if (!boundary) {
    T un = T(0), dn = T(0);  // the neighbour contributes nothing to a diagonal block
    if (!SELF) {
      const int nb = neighbour();
      const T* trn = fa.traces + ((size_t)nb * 6 + (2 * dir + 1 - s)) * 2 * NN;
      un = trn[t];
      dn = trn[NN + t];
    }
    const T ao = c3[0], an = c3[1 * CST], gam = c3[2 * CST];
    // the own cell is T- for s = 1 and T+ for s = 0; nu = +e_dir
    const T um = s ? uo : un, up = s ? un : uo;
    const T jump = um - up;
    const T avg = fma(ao, dO, an * dn);          // nu . {D grad u}_w
    const T phi = bq * (bq >= T(0) ? um : up);   // upwind flux Phi(u-, u+, b_nu)
    const T H = fma(gam, jump, phi - avg);        // Phi - nu.{D grad u}_w + gamma [[u]]
    Vf = s ? wf * H : -wf * H;                    // times [[v]] = +v (T-) or -v (T+)
    Wf = -wf * kn * jump;                         // -nu.{D grad v}_w [[u]]
    if (TD) {
      Wt1 = -wf * c3[4 * CST] * jump;
      Wt2 = -wf * c3[5 * CST] * jump;
    }
  } else {
    // Phi(u,0,b_nu) v - (nu.D grad u) v - (nu.D grad v) u + gamma u v, nu = outward normal.  The set-up encodes
    // the side's type in the coefficients: the second one multiplies the upwind flux (1 on Dirichlet and
    // outflow faces, 0 on Neumann faces); an outflow or Neumann face has zero diffusion and penalty ones.
    const T sgn = s ? T(1) : T(-1);
    const T bnu = sgn * bq;
    const T phi = bnu >= T(0) ? bnu * uo : T(0);
    const T aD = c3[0];
    Vf = wf * (c3[1 * CST] * phi - sgn * aD * dO + c3[2 * CST] * uo);
    Wf = -wf * sgn * kn * uo;
    if (TD) {
      Wt1 = -wf * sgn * c3[4 * CST] * uo;
      Wt2 = -wf * sgn * c3[5 * CST] * uo;
    }
  }
}

// Face-kernel work on one tile of `here` consecutive cells starting at cell0 (see cell_tile; LPT lines per thread,
// 1 for the tensor-diffusion path, whose tangential weights pass through shared memory between two barriers).
template <int N, typename T, bool SELF, int CPB, typename TV = T, int M = N, bool VB = false, bool PER = false,
          bool TD = false, bool PW = false, int LPT = 1>
__device__ __forceinline__ void face_tile(const TabNM<N, M, T>& tb, const Geo<T>& g, const FaceArgs<T, TV>& fa,
                                          int cell0, int here, int cell_base, unsigned char* smem_raw) {
  static_assert(LPT == 1 || !TD, "several lines per thread: scalar diffusion only");
  constexpr int NN = M * M, N3 = N * N * N, CS = Lay<M>::CS, TPC = (NN + LPT - 1) / LPT;
  T* sV = reinterpret_cast<T*>(smem_raw);
  T* sW = sV + CPB * CS;  // TD: tangential weights [CPB][side][2][M^2]
  const int lc = threadIdx.x / TPC, t0 = threadIdx.x - lc * TPC;
  const bool active = lc < here;
  const int vcell = cell0 + lc;                                // output / trace index
  const int cell = SELF ? cell_base + vcell / N3 : vcell;      // real cell
  T* V = sV + lc * CS;

  gload_cells<M>(sV, fa.V, cell0, here);
  __syncthreads();
  if (fa.mode == 2 && active) {
    // (f, v)_T: scale f by the quadrature weight Delta_T w_i (Sec. 3.1)
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
      const int t = t0 + l * TPC;
      if (t < NN) {
        const int a = t % M, b = t / M;
        const T wz = g.vol * tb.w[a] * tb.w[b];
#pragma unroll
        for (int q = 0; q < M; ++q) V[Lay<M>::idx(q, a, b)] *= wz * tb.w[q];
      }
    }
  }
  __syncthreads();

  int ic[3];
  ic[0] = cell % g.n[0];
  ic[1] = (cell / g.n[0]) % g.n[1];
  ic[2] = cell / (g.n[0] * g.n[1]);
  // lift the face weights onto the normal lines, x then y then z (Sec. 3.4, normal direction last):
  // v_l += l_l(s) Vf + l_l'(s) Wf; the z pass continues with the first transposed contraction
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
      const int t = t0 + l * TPC;
      const bool line = active && t < NN;
      const int a = line ? t % M : 0, b = line ? t / M : 0;  // t < NN keeps a, b < M
      const T wab = tb.w[a] * tb.w[b];
      T Vf[2], Wf[2];
      if (line) {
        const T wf = g.area[dir] * wab;
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          T Wt1, Wt2;
          face_weights<N, T, SELF, TV, M, VB, PER, TD, PW>(g, fa, cell, vcell, ic, dir, s, t, wf, Vf[s], Wf[s], Wt1,
                                                           Wt2);
          if (TD) {
            sW[((lc * 2 + s) * 2 + 0) * NN + t] = Wt1;
            sW[((lc * 2 + s) * 2 + 1) * NN + t] = Wt2;
          }
        }
      }
      if (TD) {
        // tangential derivatives of v at the face points, transposed: the weight Wt at (a2, b) reaches the
        // value of v at (a, b) through Dc[a2][a] (and likewise along b)  (LPT == 1 here)
        __syncthreads();
        if (line) {
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            const T* W1 = sW + ((lc * 2 + s) * 2 + 0) * NN;
            const T* W2 = sW + ((lc * 2 + s) * 2 + 1) * NN;
            T e = Vf[s];
#pragma unroll
            for (int q = 0; q < M; ++q) e = fma(tb.Dc[q][a], W1[q + M * b], fma(tb.Dc[q][b], W2[a + M * q], e));
            Vf[s] = e;
          }
        }
      }
      if (line) {
        const int bs = Lay<M>::base(dir, t), st = Lay<M>::stride(dir);
        T v[M];
        load_line<M>(V, bs, st, v);
#pragma unroll
        for (int s = 0; s < 2; ++s) {
#pragma unroll
          for (int q = 0; q < M; ++q) v[q] = fma(tb.L[s][q], Vf[s], fma(tb.P[s][q], Wf[s], v[q]));
        }
        if (dir == 2) {
          T y[N];
          eo_bwd<N, M, T>(tb, v, y);
          store_line<N>(V, bs, st, y);
        } else {
          store_line<M>(V, bs, st, v);
        }
      }
    }
    __syncthreads();
  }

  // Sec. 3.2: test functions, A^T along y and x (M -> N on the modal lines)
#pragma unroll
  for (int dd = 0; dd < 2; ++dd) {
    const int dir = 1 - dd;
#pragma unroll
    for (int l = 0; l < LPT; ++l) {
      const int t = t0 + l * TPC;
      if (active && t < NN && (M == N || t < ModalLines<N, M>::count(dir))) {
        T x[M], y[N];
        const int bs = ModalLines<N, M>::base(dir, t), st = Lay<M>::stride(dir);
        load_line<M>(V, bs, st, x);
        eo_bwd<N, M, T>(tb, x, y);
        store_line<N>(V, bs, st, y);
      }
    }
    __syncthreads();
  }
  // write out (minus F for the residual, or the Runge-Kutta stage combination)
  const int total = here * N3;
  TV* dst = fa.y + (size_t)cell0 * N3;
  const T* Fs = fa.F ? fa.F + (size_t)cell0 * N3 : nullptr;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int c = e / N3, r = e - c * N3;
    const int i1 = r % N, i23 = r / N;
    T val;
    if constexpr (M == N) {
      val = sV[c * CS + i1 + Lay<M>::LS * i23];
    } else {
      val = sV[c * CS + Lay<M>::idx(i1, i23 % N, i23 / N)];
    }
    if (fa.mode == 1) val = val - Fs[e];
    TV out = from_compute<TV, T>(val);
    if constexpr (!std::is_same<T, float>::value) {
      // Runge-Kutta stage (FP64 vectors): the update itself is done in FP64 also when the operator ran in
      // double-float, so the state keeps full FP64 precision from step to step
      if (fa.mode == 3) {
        const size_t ge = (size_t)cell0 * N3 + e;
        const double rd = Fs ? out - from_compute<double, T>(Fs[e]) : out;
        out = fma(fa.cz, (double)fa.z0[ge], fma(fa.cu, (double)fa.u[ge], -fa.cr * rd));
      }
    }
    dst[e] = out;
  }
}

template <int N, typename T, bool SELF = false, int CPB = Launch<N>::CPB, typename TV = T, int M = N, bool VB = false,
          bool PER = false, bool TD = false, bool PW = false>
__global__ void __launch_bounds__(CPB * M * M)
dg_face_kernel(const __grid_constant__ TabNM<N, M, T> tb, const __grid_constant__ Geo<T> g,
               const __grid_constant__ FaceArgs<T, TV> fa, SelfArgs sa_) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cell0 = blockIdx.x * CPB;
  const int here = min(CPB, (SELF ? sa_.nvirt : g.ncell) - cell0);
  face_tile<N, T, SELF, CPB, TV, M, VB, PER, TD, PW>(tb, g, fa, cell0, here, sa_.cell_base, smem_raw);
}

// The same kernel with 8 resident CTAs of 256 threads requested: used for FP32 when a CTA has 256 threads
// (k = 1, 3, 7), where the compiler otherwise settles on more than the 32 registers per thread that allow it.
template <int N, typename T, int CPB, typename TV, int M, bool PER>
__global__ void __launch_bounds__(CPB * M * M, 8)
dg_face_kernel_occ8(const __grid_constant__ TabNM<N, M, T> tb, const __grid_constant__ Geo<T> g,
                    const __grid_constant__ FaceArgs<T, TV> fa, SelfArgs sa_) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int cell0 = blockIdx.x * CPB;
  const int here = min(CPB, g.ncell - cell0);
  face_tile<N, T, false, CPB, TV, M, false, PER>(tb, g, fa, cell0, here, sa_.cell_base, smem_raw);
}

// the face kernel of a launch configuration (the FP32 256-thread variant above, or the general one)
template <int N, typename T, int CPB, typename TV, int M, bool VB, bool PER, bool TD = false, bool PW = false>
constexpr auto face_kernel_for() {
  if constexpr (std::is_same<T, float>::value && !VB && !TD && CPB * M * M == 256) {
    return &dg_face_kernel_occ8<N, T, CPB, TV, M, PER>;
  } else {
    return &dg_face_kernel<N, T, false, CPB, TV, M, VB, PER, TD, PW>;
  }
}

}  // namespace dgk
