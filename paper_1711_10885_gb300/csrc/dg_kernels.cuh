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
#pragma once

#include <cuda_runtime.h>

namespace dgk {

// 1D tables for n = m = N: basis at the Gauss points, collocation derivative, face extrapolation.
template <int N, typename T>
struct Tab {
  T A[N][N];    // A[i][j] = theta_j(xi_i)
  T Dt[N][N];   // Dt[i][l] = l_l'(xi_i)   (Lagrange basis on the Gauss points)
  T DtW[N][N];  // DtW[i][l] = w_i * Dt[i][l]
  T w[N];       // Gauss weights on [0,1]
  T L[2][N];    // L[s][l] = l_l(s),  s = 0, 1 (face at xi = s)
  T P[2][N];    // P[s][l] = l_l'(s)
};

template <typename T>
struct Geo {
  int n[3];
  int ncell;
  T vol;      // |T| = h_x h_y h_z
  T area[3];  // |F| of a face normal to axis r
  T alpha[3]; // |T| / h_r^2       (times D_T: diffusion weight of d_r u)
  T beta[3];  // -b_r |T| / h_r    (convection weight of u)
  T b[3];     // velocity
  T creact;   // c |T|
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

// y[i] = sum_j M[i][j] x[j]
template <int N, typename T>
__device__ __forceinline__ void mv(const T (&M)[N][N], const T (&x)[N], T (&y)[N]) {
#pragma unroll
  for (int i = 0; i < N; ++i) {
    T acc = M[i][0] * x[0];
#pragma unroll
    for (int j = 1; j < N; ++j) acc = fma(M[i][j], x[j], acc);
    y[i] = acc;
  }
}
// y[j] = y0[j] + sum_i M[i][j] x[i]
template <int N, typename T>
__device__ __forceinline__ void mvt_acc(const T (&M)[N][N], const T (&x)[N], T (&y)[N]) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T acc = y[j];
#pragma unroll
    for (int i = 0; i < N; ++i) acc = fma(M[i][j], x[i], acc);
    y[j] = acc;
  }
}
// y[j] = sum_i M[i][j] x[i]
template <int N, typename T>
__device__ __forceinline__ void mvt(const T (&M)[N][N], const T (&x)[N], T (&y)[N]) {
#pragma unroll
  for (int j = 0; j < N; ++j) {
    T acc = M[0][j] * x[0];
#pragma unroll
    for (int i = 1; i < N; ++i) acc = fma(M[i][j], x[i], acc);
    y[j] = acc;
  }
}

template <int N>
struct Launch {
  static constexpr int NN = N * N;
  static constexpr int CPB = (256 / NN) > 0 ? (256 / NN) : 1;  // cells per CTA
  static constexpr int THREADS = CPB * NN;
};

// copy cpb cells (contiguous in global memory, N^3 each) into padded shared buffers
template <int N, typename T>
__device__ __forceinline__ void gload_cells(T* sbuf, const T* __restrict__ g, int cell0, int ncells_here) {
  constexpr int N3 = N * N * N;
  const int total = ncells_here * N3;
  const T* src = g + (size_t)cell0 * N3;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int c = e / N3, r = e - c * N3;
    const int i1 = r % N, i23 = r / N;
    sbuf[c * Lay<N>::CS + i1 + Lay<N>::LS * i23] = src[e];
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

// ---------------------------------------------------------------------------------------------
// Kernel 1: modal -> points, volume integrand, point-space residual V, face traces
// ---------------------------------------------------------------------------------------------
template <int N, typename T>
__global__ void __launch_bounds__(Launch<N>::THREADS)
dg_cell_kernel(const __grid_constant__ Tab<N, T> tb, const __grid_constant__ Geo<T> g, const T* __restrict__ z,
               const T* __restrict__ Dcell, T* __restrict__ Vout, T* __restrict__ traces) {
  constexpr int NN = N * N, CPB = Launch<N>::CPB, CS = Lay<N>::CS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sU = reinterpret_cast<T*>(smem_raw);
  T* sV = sU + CPB * CS;
  const int cell0 = blockIdx.x * CPB;
  const int here = min(CPB, g.ncell - cell0);
  const int lc = threadIdx.x / NN, t = threadIdx.x - lc * NN;
  const bool active = lc < here;
  const int cell = cell0 + lc;
  T* U = sU + lc * CS;
  T* V = sV + lc * CS;

  gload_cells<N>(sU, z, cell0, here);
  __syncthreads();

  // Sec. 3.3, eq. evalfe: u at the Gauss points, one axis at a time (x, then y, then z)
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    if (active) {
      T x[N], y[N];
      const int bs = Lay<N>::base(dir, t), st = Lay<N>::stride(dir);
      load_line<N>(U, bs, st, x);
      mv<N>(tb.A, x, y);
      store_line<N>(U, bs, st, y);
    }
    __syncthreads();
  }

  // Sec. 3.2, eqs. evalblf / gauss_points: per axis r, V += Dt_r^T [w (alpha_r D d_r u + beta_r u)]
  // and the six face traces (value and reference normal derivative) from the same lines.
  const T DT = active ? Dcell[cell] : T(0);
  const int a = t % N, b = t / N;
  const T wperp = tb.w[a] * tb.w[b];
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    if (active) {
      T u[N], gr[N], X[N], v[N];
      const int bs = Lay<N>::base(dir, t), st = Lay<N>::stride(dir);
      load_line<N>(U, bs, st, u);
      mv<N>(tb.Dt, u, gr);
      const T sa = wperp * (DT * g.alpha[dir]);
      const T sb = wperp * g.beta[dir];
#pragma unroll
      for (int i = 0; i < N; ++i) X[i] = fma(sa, gr[i], sb * u[i]);
      if (dir == 0) {
        const T sc = wperp * g.creact;
#pragma unroll
        for (int l = 0; l < N; ++l) v[l] = (sc * tb.w[l]) * u[l];
      } else {
        load_line<N>(V, bs, st, v);
      }
      mvt_acc<N>(tb.DtW, X, v);
      store_line<N>(V, bs, st, v);
      // traces at xi_dir = 0 and 1: field 0 = u, field 1 = d u / d xi_dir (reference)
      T* tr = traces + ((size_t)cell * 6 + 2 * dir) * 2 * NN;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        T tv = T(0), td = T(0);
#pragma unroll
        for (int l = 0; l < N; ++l) {
          tv = fma(tb.L[s][l], u[l], tv);
          td = fma(tb.P[s][l], u[l], td);
        }
        tr[(2 * s + 0) * NN + t] = tv;
        tr[(2 * s + 1) * NN + t] = td;
      }
    }
    __syncthreads();
  }
  gstore_cells<N>(Vout, sV, cell0, here);
}

// ---------------------------------------------------------------------------------------------
// Kernel 2: face fluxes + lift + backward contraction (+ residual)
// fc[(cell*6 + face)*3 + {0,1,2}]: interior: (w_own D_own / h, w_nbr D_nbr / h, gamma_F);
//                                   boundary: (D_own / h, 0, gamma_F)
// mode 0: y = A z;  mode 1: y = A z - F;  mode 2 (right hand side): V from f, faces from g
// ---------------------------------------------------------------------------------------------
template <typename T>
struct FaceArgs {
  const T* V;       // point-space residual from dg_cell_kernel (mode 0/1), or f at points (mode 2)
  const T* traces;  // traces from dg_cell_kernel (mode 0/1)
  const T* fc;      // face coefficients
  const T* F;       // right hand side (mode 1)
  const T* g[6];    // Dirichlet data per boundary side (mode 2), may be null
  T* y;
  int mode;
};

template <int N, typename T>
__global__ void __launch_bounds__(Launch<N>::THREADS)
dg_face_kernel(const __grid_constant__ Tab<N, T> tb, const __grid_constant__ Geo<T> g,
               const __grid_constant__ FaceArgs<T> fa) {
  constexpr int NN = N * N, CPB = Launch<N>::CPB, CS = Lay<N>::CS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sV = reinterpret_cast<T*>(smem_raw);
  const int cell0 = blockIdx.x * CPB;
  const int here = min(CPB, g.ncell - cell0);
  const int lc = threadIdx.x / NN, t = threadIdx.x - lc * NN;
  const bool active = lc < here;
  const int cell = cell0 + lc;
  T* V = sV + lc * CS;

  gload_cells<N>(sV, fa.V, cell0, here);
  __syncthreads();
  if (fa.mode == 2 && active) {
    // (f, v)_T: scale f by the quadrature weight Delta_T w_i (Sec. 3.1)
    const int a = t % N, b = t / N;
    const T wz = g.vol * tb.w[a] * tb.w[b];
#pragma unroll
    for (int l = 0; l < N; ++l) {
      const int e = Lay<N>::idx(l, a, b);
      V[e] *= wz * tb.w[l];
    }
  }
  __syncthreads();

  int ic[3];
  ic[0] = cell % g.n[0];
  ic[1] = (cell / g.n[0]) % g.n[1];
  ic[2] = cell / (g.n[0] * g.n[1]);
  const int a = t % N, b = t / N;
#pragma unroll
  for (int dir = 0; dir < 3; ++dir) {
    if (active) {
      const int bs = Lay<N>::base(dir, t), st = Lay<N>::stride(dir);
      T v[N];
      load_line<N>(V, bs, st, v);
      const T wf = g.area[dir] * tb.w[a] * tb.w[b];
      const int nstride = dir == 0 ? 1 : (dir == 1 ? g.n[0] : g.n[0] * g.n[1]);
      const T bq = g.b[dir];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int face = 2 * dir + s;
        const bool boundary = s ? (ic[dir] == g.n[dir] - 1) : (ic[dir] == 0);
        const T* c3 = fa.fc + ((size_t)cell * 6 + face) * 3;
        T Vf = T(0), Wf = T(0);
        if (fa.mode == 2) {
          // Dirichlet terms of l_h: -(Phi(0,g,b_nu), v) - (nu.D grad v, g) + gamma (g, v)
          const T* gs = fa.g[face];
          if (boundary && gs != nullptr) {
            const int ta = dir == 0 ? 1 : 0, tbx = dir == 2 ? 1 : 2;
            const int fidx = ic[ta] + g.n[ta] * ic[tbx];
            const T gv = gs[(size_t)fidx * NN + t];
            const T sgn = s ? T(1) : T(-1);
            const T bnu = sgn * bq;
            const T phi = bnu >= T(0) ? T(0) : bnu * gv;
            Vf = wf * (c3[2] * gv - phi);
            Wf = -wf * sgn * c3[0] * gv;
          }
        } else {
          const T* tro = fa.traces + ((size_t)cell * 6 + face) * 2 * NN;
          const T uo = tro[t], dO = tro[NN + t];
          if (!boundary) {
            const int nb = s ? cell + nstride : cell - nstride;
            const T* trn = fa.traces + ((size_t)nb * 6 + (2 * dir + 1 - s)) * 2 * NN;
            const T un = trn[t], dn = trn[NN + t];
            const T ao = c3[0], an = c3[1], gam = c3[2];
            // eq. blf on an interior face; the own cell is T- for s = 1 and T+ for s = 0
            const T um = s ? uo : un, up = s ? un : uo;
            const T jump = um - up;
            const T avg = fma(ao, dO, an * dn);            // nu . {D grad u}_w
            const T phi = bq * (bq >= T(0) ? um : up);     // upwind flux
            const T H = fma(gam, jump, phi - avg);          // Phi - avg + gamma [[u]]
            Vf = s ? wf * H : -wf * H;                     // times [[v]] = +-v
            Wf = -wf * ao * jump;                          // -nu.{D grad v}_w [[u]]
          } else {
            // Dirichlet face: Phi(u,0,b_nu) v - (nu.D grad u) v - (nu.D grad v) u + gamma u v
            const T sgn = s ? T(1) : T(-1);
            const T bnu = sgn * bq;
            const T phi = bnu >= T(0) ? bnu * uo : T(0);
            const T aD = c3[0];
            Vf = wf * (phi - sgn * aD * dO + c3[2] * uo);
            Wf = -wf * sgn * aD * uo;
          }
        }
        // lift onto the normal line: v_l += l_l(s) Vf + l_l'(s) Wf  (Sec. 3.4, normal direction last)
#pragma unroll
        for (int l = 0; l < N; ++l) v[l] = fma(tb.L[s][l], Vf, fma(tb.P[s][l], Wf, v[l]));
      }
      store_line<N>(V, bs, st, v);
    }
    __syncthreads();
  }

  // Sec. 3.2: test functions, A^T along z, y, x
#pragma unroll
  for (int dd = 0; dd < 3; ++dd) {
    const int dir = 2 - dd;
    if (active) {
      T x[N], y[N];
      const int bs = Lay<N>::base(dir, t), st = Lay<N>::stride(dir);
      load_line<N>(V, bs, st, x);
      mvt<N>(tb.A, x, y);
      store_line<N>(V, bs, st, y);
    }
    __syncthreads();
  }
  // write out (minus F for the residual)
  constexpr int N3 = N * N * N;
  const int total = here * N3;
  T* dst = fa.y + (size_t)cell0 * N3;
  const T* Fs = fa.F ? fa.F + (size_t)cell0 * N3 : nullptr;
  for (int e = threadIdx.x; e < total; e += blockDim.x) {
    const int c = e / N3, r = e - c * N3;
    const int i1 = r % N, i23 = r / N;
    T val = sV[c * CS + i1 + Lay<N>::LS * i23];
    if (fa.mode == 1) val -= Fs[e];
    dst[e] = val;
  }
}

}  // namespace dgk
