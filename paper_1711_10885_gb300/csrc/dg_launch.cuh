// dg_launch.cuh -- template launchers shared by the per-precision translation units.
#pragma once

#include "dg_internal.h"
#include "dg_kernels.cuh"

namespace dgi {

template <int N, typename T>
dgk::Tab<N, T> make_tab(const Tables1D& t) {
  constexpr int H = N / 2, C = (N + 1) / 2;
  dgk::Tab<N, T> r;
  // B[o][i] = w_i Dt[i][o]: the weighted transposed collocation derivative
  double B[MAXN][MAXN];
  for (int o = 0; o < N; ++o)
    for (int i = 0; i < N; ++i) B[o][i] = t.w[i] * t.Dt[i][o];
  for (int i = 0; i < C; ++i) {
    for (int k = 0; k < C; ++k) r.AE[i][k] = (T)t.A[i][2 * k];
    for (int k = 0; k < H; ++k) r.AO[i][k] = (T)t.A[i][2 * k + 1];
    for (int l = 0; l < H; ++l) {
      r.DHm[i][l] = (T)(0.5 * (t.Dt[i][l] - t.Dt[i][N - 1 - l]));
      r.BHm[i][l] = (T)(0.5 * (B[i][l] - B[i][N - 1 - l]));
    }
  }
  for (int i = 0; i < H; ++i)
    for (int l = 0; l < C; ++l) {
      r.DHp[i][l] = (T)(0.5 * (t.Dt[i][l] + t.Dt[i][N - 1 - l]));
      r.BHp[i][l] = (T)(0.5 * (B[i][l] + B[i][N - 1 - l]));
    }
  for (int l = 0; l < C; ++l) {
    r.LS[l] = (T)(0.5 * (t.L[1][l] + t.L[1][N - 1 - l]));
    r.PS[l] = (T)(0.5 * (t.P[1][l] + t.P[1][N - 1 - l]));
  }
  for (int l = 0; l < H; ++l) {
    r.LD[l] = (T)(0.5 * (t.L[1][l] - t.L[1][N - 1 - l]));
    r.PD[l] = (T)(0.5 * (t.P[1][l] - t.P[1][N - 1 - l]));
  }
  for (int i = 0; i < N; ++i) {
    r.w[i] = (T)t.w[i];
    for (int s = 0; s < 2; ++s) {
      r.L[s][i] = (T)t.L[s][i];
      r.P[s][i] = (T)t.P[s][i];
    }
  }
  return r;
}

template <typename T>
dgk::Geo<T> make_geo(const dg_handle* h) {
  dgk::Geo<T> g;
  const double vol = h->h[0] * h->h[1] * h->h[2];
  for (int r = 0; r < 3; ++r) {
    g.n[r] = h->n[r];
    g.area[r] = (T)(vol / h->h[r]);
    g.alpha[r] = (T)(vol / (h->h[r] * h->h[r]));
    g.beta[r] = (T)(-h->b[r] * vol / h->h[r]);
    g.b[r] = (T)h->b[r];
  }
  g.ncell = (int)h->ncell;
  g.vol = (T)vol;
  g.creact = (T)(h->c * vol);
  return g;
}

template <int N, typename T>
size_t cell_smem() {
  return 2 * (size_t)dgk::Launch<N>::CPB * dgk::Lay<N>::CS * sizeof(T);
}
template <int N, typename T>
size_t face_smem() {
  return (size_t)dgk::Launch<N>::CPB * dgk::Lay<N>::CS * sizeof(T);
}

template <int N, typename T, typename TV = T>
int set_smem_attrs() {
  static bool done = false;  // per instantiation; attributes are per function
  if (done) return 0;
  cudaError_t e = cudaFuncSetAttribute(dgk::dg_cell_kernel<N, T, false, dgk::Launch<N>::CPB, TV>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cell_smem<N, T>());
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_cell_kernel)");
  e = cudaFuncSetAttribute(dgk::dg_face_kernel<N, T, false, dgk::Launch<N>::CPB, TV>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, (int)face_smem<N, T>());
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_face_kernel)");
  done = true;
  return 0;
}

// coefficient copies in the compute precision
template <typename T>
const Buffers& buffers_for(const dg_handle* h);
template <>
inline const Buffers& buffers_for<double>(const dg_handle* h) { return h->p64; }
template <>
inline const Buffers& buffers_for<float>(const dg_handle* h) { return h->p32; }
template <>
inline const Buffers& buffers_for<dgk::dfl>(const dg_handle* h) { return h->pX; }

template <int N>
int set_self_smem_attrs() {
  static bool done = false;
  if (done) return 0;
  cudaError_t e = cudaFuncSetAttribute(dgk::dg_cell_kernel<N, double, true>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cell_smem<N, double>());
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_cell_kernel self)");
  e = cudaFuncSetAttribute(dgk::dg_face_kernel<N, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           (int)face_smem<N, double>());
  if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_face_kernel self)");
  done = true;
  return 0;
}

template <int N, typename T, typename TV = T>
int apply_n(const dg_handle* h, const TV* z, TV* y, int mode, int stages, cudaStream_t s) {
  if (int rc = set_smem_attrs<N, T, TV>()) return rc;
  const Buffers& bf = buffers_for<T>(h);
  const auto tb = make_tab<N, T>(h->tab);
  const auto geo = make_geo<T>(h);
  const int cpb = dgk::Launch<N>::CPB;
  const unsigned grid = (unsigned)((h->ncell + cpb - 1) / cpb);
  T* V = static_cast<T*>(h->work_V);
  T* tr = static_cast<T*>(h->work_tr);
  if (stages & 1)
    dgk::dg_cell_kernel<N, T, false, dgk::Launch<N>::CPB, TV><<<grid, dgk::Launch<N>::THREADS, cell_smem<N, T>(), s>>>(
        tb, geo, z, static_cast<const T*>(bf.D), V, tr, dgk::SelfArgs{0, 0});
  dgk::FaceArgs<T, TV> fa;
  fa.V = V;
  fa.traces = tr;
  fa.fc = static_cast<const T*>(bf.fc);
  fa.F = mode == 1 ? static_cast<const T*>(bf.F) : nullptr;
  for (int i = 0; i < 6; ++i) fa.g[i] = nullptr;
  fa.y = y;
  fa.mode = mode;
  if (stages & 2)
    dgk::dg_face_kernel<N, T, false, dgk::Launch<N>::CPB, TV>
        <<<grid, dgk::Launch<N>::THREADS, face_smem<N, T>(), s>>>(tb, geo, fa, dgk::SelfArgs{0, 0});
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "operator kernel launch");
  return 0;
}

template <int N, typename T>
int rhs_n(const dg_handle* h, const T* f, const T* const g[6], T* F, cudaStream_t s) {
  if (int rc = set_smem_attrs<N, T>()) return rc;
  const Buffers& bf = sizeof(T) == 8 ? h->p64 : h->p32;
  const auto tb = make_tab<N, T>(h->tab);
  const auto geo = make_geo<T>(h);
  const int cpb = dgk::Launch<N>::CPB;
  const unsigned grid = (unsigned)((h->ncell + cpb - 1) / cpb);
  dgk::FaceArgs<T> fa;
  fa.V = f;
  fa.traces = nullptr;
  fa.fc = static_cast<const T*>(bf.fc);
  fa.F = nullptr;
  for (int i = 0; i < 6; ++i) fa.g[i] = g[i];
  fa.y = F;
  fa.mode = 2;
  dgk::dg_face_kernel<N, T><<<grid, dgk::Launch<N>::THREADS, face_smem<N, T>(), s>>>(tb, geo, fa,
                                                                                    dgk::SelfArgs{0, 0});
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rhs kernel launch");
  return 0;
}

// Diagonal blocks of cells [cell_base, cell_base + ncells): column j of block c is written to
// out[(c * N^3 + j) * N^3 + i], i.e. each block is stored as A_TT^T in row-major order.
template <int N>
int diag_blocks_n(const dg_handle* h, double* out, int cell_base, int ncells, double* V, double* tr, cudaStream_t s) {
  if (int rc = set_smem_attrs<N, double>()) return rc;
  if (int rc = set_self_smem_attrs<N>()) return rc;
  constexpr int N3 = N * N * N;
  const auto tb = make_tab<N, double>(h->tab);
  const auto geo = make_geo<double>(h);
  const int cpb = dgk::Launch<N>::CPB;
  const int nvirt = ncells * N3;
  const unsigned grid = (unsigned)((nvirt + cpb - 1) / cpb);
  const dgk::SelfArgs sa{nvirt, cell_base};
  dgk::dg_cell_kernel<N, double, true><<<grid, dgk::Launch<N>::THREADS, cell_smem<N, double>(), s>>>(
      tb, geo, static_cast<const double*>(nullptr), static_cast<const double*>(h->p64.D), V, tr, sa);
  dgk::FaceArgs<double> fa;
  fa.V = V;
  fa.traces = tr;
  fa.fc = static_cast<const double*>(h->p64.fc);
  fa.F = nullptr;
  for (int i = 0; i < 6; ++i) fa.g[i] = nullptr;
  fa.y = out;
  fa.mode = 0;
  dgk::dg_face_kernel<N, double, true><<<grid, dgk::Launch<N>::THREADS, face_smem<N, double>(), s>>>(tb, geo, fa,
                                                                                                    sa);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "diagonal block kernel launch");
  return 0;
}

inline int diag_blocks_dispatch(const dg_handle* h, double* out, int cell_base, int ncells, double* V, double* tr,
                                cudaStream_t s) {
  switch (h->N) {
    case 2: return diag_blocks_n<2>(h, out, cell_base, ncells, V, tr, s);
    case 3: return diag_blocks_n<3>(h, out, cell_base, ncells, V, tr, s);
    case 4: return diag_blocks_n<4>(h, out, cell_base, ncells, V, tr, s);
    case 5: return diag_blocks_n<5>(h, out, cell_base, ncells, V, tr, s);
    case 6: return diag_blocks_n<6>(h, out, cell_base, ncells, V, tr, s);
    case 7: return diag_blocks_n<7>(h, out, cell_base, ncells, V, tr, s);
    case 8: return diag_blocks_n<8>(h, out, cell_base, ncells, V, tr, s);
    case 9: return diag_blocks_n<9>(h, out, cell_base, ncells, V, tr, s);
    case 10: return diag_blocks_n<10>(h, out, cell_base, ncells, V, tr, s);
    case 11: return diag_blocks_n<11>(h, out, cell_base, ncells, V, tr, s);
    default: set_error("unsupported degree"); return DG_ERR_INVALID_ARG;
  }
}

template <typename T, typename TV = T>
int apply_dispatch(const dg_handle* h, const TV* z, TV* y, int mode, int stages, cudaStream_t s) {
  switch (h->N) {
    case 2: return apply_n<2, T, TV>(h, z, y, mode, stages, s);
    case 3: return apply_n<3, T, TV>(h, z, y, mode, stages, s);
    case 4: return apply_n<4, T, TV>(h, z, y, mode, stages, s);
    case 5: return apply_n<5, T, TV>(h, z, y, mode, stages, s);
    case 6: return apply_n<6, T, TV>(h, z, y, mode, stages, s);
    case 7: return apply_n<7, T, TV>(h, z, y, mode, stages, s);
    case 8: return apply_n<8, T, TV>(h, z, y, mode, stages, s);
    case 9: return apply_n<9, T, TV>(h, z, y, mode, stages, s);
    case 10: return apply_n<10, T, TV>(h, z, y, mode, stages, s);
    case 11: return apply_n<11, T, TV>(h, z, y, mode, stages, s);
    default: set_error("unsupported degree"); return DG_ERR_INVALID_ARG;
  }
}

template <typename T>
int rhs_dispatch(const dg_handle* h, const T* f, const T* const g[6], T* F, cudaStream_t s) {
  switch (h->N) {
    case 2: return rhs_n<2, T>(h, f, g, F, s);
    case 3: return rhs_n<3, T>(h, f, g, F, s);
    case 4: return rhs_n<4, T>(h, f, g, F, s);
    case 5: return rhs_n<5, T>(h, f, g, F, s);
    case 6: return rhs_n<6, T>(h, f, g, F, s);
    case 7: return rhs_n<7, T>(h, f, g, F, s);
    case 8: return rhs_n<8, T>(h, f, g, F, s);
    case 9: return rhs_n<9, T>(h, f, g, F, s);
    case 10: return rhs_n<10, T>(h, f, g, F, s);
    case 11: return rhs_n<11, T>(h, f, g, F, s);
    default: set_error("unsupported degree"); return DG_ERR_INVALID_ARG;
  }
}

}  // namespace dgi
