// dg_launch.cuh -- template launchers shared by the per-precision translation units.
#pragma once

#include "dg_internal.h"
#include "dg_kernels.cuh"
#include "dg_kernels_plane.cuh"

namespace dgi {

template <int N, typename T, int M = N>
dgk::TabNM<N, M, T> make_tab(const Tables1D& t) {
  constexpr int HN = N / 2, CN = (N + 1) / 2, HM = M / 2, CM = (M + 1) / 2;
  dgk::TabNM<N, M, T> r;
  // B[o][i] = w_i Dt[i][o]: the weighted transposed collocation derivative
  double B[MAXM][MAXM];
  for (int o = 0; o < M; ++o)
    for (int i = 0; i < M; ++i) B[o][i] = t.w[i] * t.Dt[i][o];
  for (int i = 0; i < CM; ++i) {
    for (int k = 0; k < CN; ++k) r.AE[i][k] = (T)t.A[i][2 * k];
    for (int l = 0; l < HM; ++l) {
      r.DHm[i][l] = (T)(0.5 * (t.Dt[i][l] - t.Dt[i][M - 1 - l]));
      r.BHm[i][l] = (T)(0.5 * (B[i][l] - B[i][M - 1 - l]));
    }
  }
  for (int i = 0; i < HM; ++i) {
    for (int k = 0; k < HN; ++k) r.AO[i][k] = (T)t.A[i][2 * k + 1];
    for (int l = 0; l < CM; ++l) {
      r.DHp[i][l] = (T)(0.5 * (t.Dt[i][l] + t.Dt[i][M - 1 - l]));
      r.BHp[i][l] = (T)(0.5 * (B[i][l] + B[i][M - 1 - l]));
    }
  }
  for (int l = 0; l < CM; ++l) {
    r.LS[l] = (T)(0.5 * (t.L[1][l] + t.L[1][M - 1 - l]));
    r.PS[l] = (T)(0.5 * (t.P[1][l] + t.P[1][M - 1 - l]));
  }
  for (int l = 0; l < HM; ++l) {
    r.LD[l] = (T)(0.5 * (t.L[1][l] - t.L[1][M - 1 - l]));
    r.PD[l] = (T)(0.5 * (t.P[1][l] - t.P[1][M - 1 - l]));
  }
  for (int i = 0; i < M; ++i) {
    r.w[i] = (T)t.w[i];
    for (int s = 0; s < 2; ++s) {
      r.L[s][i] = (T)t.L[s][i];
      r.P[s][i] = (T)t.P[s][i];
    }
    for (int l = 0; l < M; ++l) r.Dc[i][l] = (T)t.Dt[i][l];
  }
  return r;
}

template <typename T>
dgk::Geo<T> make_geo(const dg_handle* h) {
  dgk::Geo<T> g;
  if (!h->affine) {
    const double vol = h->h[0] * h->h[1] * h->h[2];
    for (int r = 0; r < 3; ++r) {
      g.n[r] = h->n[r];
      g.area[r] = (T)(vol / h->h[r]);
      g.inv_area[r] = (T)(h->h[r] / vol);
      g.alpha[r] = (T)(vol / (h->h[r] * h->h[r]));
      g.beta[r] = (T)(-h->b[r] * vol / h->h[r]);
      g.b[r] = (T)h->b[r];
    }
    g.vol = (T)vol;
    g.creact = (T)(h->c * vol);
  } else {
    // affine cells: |F_r| = |det J| |J^{-T} e_r|, b . nu_r = (J^{-1} b)_r / |J^{-T} e_r|,
    // convection weight -|det J| (J^{-1} b)_r
    for (int r = 0; r < 3; ++r) {
      const double jb = h->Jinv[r][0] * h->b[0] + h->Jinv[r][1] * h->b[1] + h->Jinv[r][2] * h->b[2];
      g.n[r] = h->n[r];
      g.area[r] = (T)(h->detJ * h->fscale[r]);
      g.inv_area[r] = (T)(1.0 / (h->detJ * h->fscale[r]));
      g.alpha[r] = T(0);
      g.beta[r] = (T)(-h->detJ * jb);
      g.b[r] = (T)(jb / h->fscale[r]);
    }
    g.vol = (T)h->detJ;
    g.creact = (T)(h->c * h->detJ);
  }
  if (h->ml) {
    // multilinear cells: the volume and area elements vary over a cell and are folded into the point tables,
    // the face coefficients and the right hand side data, so the kernels see |T| = 1 and |F| = 1
    for (int r = 0; r < 3; ++r) g.area[r] = T(1);
    g.vol = T(1);
  }
  g.ncell = (int)h->ncell;
  for (int r = 0; r < 3; ++r) g.periodic[r] = h->periodic[r];
  for (int f = 0; f < 6; ++f) g.bc[f] = h->bc_type[f];
  g.bsc = nullptr;
  g.bface = nullptr;
  return g;
}

// shared memory of the two kernels for M points per direction and CPB cells per CTA
template <int M, typename T, int CPB = dgk::Launch<M>::CPB>
size_t cell_smem() {
  return 2 * (size_t)CPB * dgk::Lay<M>::CS * sizeof(T);
}
template <int M, typename T, int CPB = dgk::Launch<M>::CPB>
size_t face_smem() {
  return (size_t)CPB * dgk::Lay<M>::CS * sizeof(T);
}

// cells per CTA of the small-mesh variant of the FP64 kernels: a quarter of the full tile, so that meshes of
// fewer full tiles than SMs still spread over all SMs (each SM issues only two FP64 FMAs per clock)
template <int M>
constexpr int small_cpb() {
  return dgk::Launch<M>::CPB / 4 > 0 ? dgk::Launch<M>::CPB / 4 : 1;
}

template <int N, typename T, typename TV = T, int M = N, bool VB = false, int CPB = dgk::Launch<M>::CPB>
int set_smem_attrs() {
  static DeviceOnce once;  // per instantiation and device; attributes are per function
  return once.run([]() -> int {
    cudaError_t e = cudaFuncSetAttribute(dgk::dg_cell_kernel<N, T, false, CPB, TV, M, VB>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cell_smem<M, T, CPB>());
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_cell_kernel)");
    e = cudaFuncSetAttribute(dgk::face_kernel_for<N, T, CPB, TV, M, VB, true>(),
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)face_smem<M, T, CPB>());
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_face_kernel)");
    if constexpr (!VB) {
      e = cudaFuncSetAttribute(dgk::face_kernel_for<N, T, CPB, TV, M, VB, false>(),
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)face_smem<M, T, CPB>());
      if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_face_kernel)");
    }
    return 0;
  });
}

// face kernel launch: the periodic-aware variant when the mesh has a periodic axis (always for the
// velocity field kernels)
template <int N, typename T, typename TV, int M, bool VB, int CPB = dgk::Launch<M>::CPB>
void launch_face(const dg_handle* h, const dgk::TabNM<N, M, T>& tb, const dgk::Geo<T>& geo,
                 const dgk::FaceArgs<T, TV>& fa, unsigned grid, cudaStream_t s) {
  const bool per = h->periodic[0] || h->periodic[1] || h->periodic[2];
  if (VB || per) {
    dgk::face_kernel_for<N, T, CPB, TV, M, VB, true>()
        <<<grid, CPB * M * M, face_smem<M, T, CPB>(), s>>>(tb, geo, fa, dgk::SelfArgs{0, 0});
  } else if constexpr (!VB) {
    dgk::face_kernel_for<N, T, CPB, TV, M, VB, false>()
        <<<grid, CPB * M * M, face_smem<M, T, CPB>(), s>>>(tb, geo, fa, dgk::SelfArgs{0, 0});
  }
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
  static DeviceOnce once;
  return once.run([&]() -> int {
    cudaError_t e = cudaFuncSetAttribute(dgk::dg_cell_kernel<N, double, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)cell_smem<N, double>());
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_cell_kernel self)");
    e = cudaFuncSetAttribute(dgk::dg_face_kernel<N, double, true, dgk::Launch<N>::CPB, double, N, false, true>,
                             cudaFuncAttributeMaxDynamicSharedMemorySize, (int)face_smem<N, double>());
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_face_kernel self)");
    return 0;
  });
}

// geometry of the handle with the velocity field tables of the VB kernels (FP64, or the double-float copies)
template <typename T, bool VB>
dgk::Geo<T> geo_for(const dg_handle* h) {
  dgk::Geo<T> geo = make_geo<T>(h);
  if (VB) {
    const bool pair = std::is_same<T, dgk::dfl>::value;
    geo.bsc = static_cast<const T*>(pair ? h->bscX : h->bsc);
    geo.bface = static_cast<const T*>(pair ? h->bfaceX : h->bface);
  }
  return geo;
}

template <int N, typename T, typename TV = T, int M = N, bool VB = false, int CPB = dgk::Launch<M>::CPB>
int apply_n(const dg_handle* h, const TV* z, TV* y, int mode, int stages, cudaStream_t s,
            const StageArgs* st = nullptr) {
  if (int rc = set_smem_attrs<N, T, TV, M, VB, CPB>()) return rc;
  const Buffers& bf = buffers_for<T>(h);
  const auto tb = make_tab<N, T, M>(h->tab);
  const auto geo = geo_for<T, VB>(h);
  const unsigned grid = (unsigned)((h->ncell + CPB - 1) / CPB);
  T* V = static_cast<T*>(h->work_V);
  T* tr = static_cast<T*>(h->work_tr);
  if (stages & 1)
    dgk::dg_cell_kernel<N, T, false, CPB, TV, M, VB><<<grid, CPB * M * M, cell_smem<M, T, CPB>(), s>>>(
        tb, geo, z, static_cast<const T*>(bf.D), V, tr, dgk::SelfArgs{0, 0});
  dgk::FaceArgs<T, TV> fa;
  fa.V = V;
  fa.traces = tr;
  fa.fc = static_cast<const T*>(bf.fc);
  fa.F = (mode == 1 || mode == 3) ? static_cast<const T*>(bf.F) : nullptr;
  for (int i = 0; i < 6; ++i) fa.g[i] = nullptr;
  fa.y = y;
  fa.mode = mode;
  fa.u = z;
  fa.z0 = nullptr;
  fa.cz = fa.cu = fa.cr = 0.0;
  if (mode == 3) {
    if (!st || !std::is_same<TV, double>::value || std::is_same<T, float>::value) {
      set_error("Runge-Kutta stages need FP64 vectors and the FP64 or double-float operator");
      return DG_ERR_INVALID_ARG;
    }
    fa.z0 = reinterpret_cast<const TV*>(st->z0);
    fa.cz = st->cz;
    fa.cu = st->cu;
    fa.cr = st->cr;
  }
  if (stages & 2) launch_face<N, T, TV, M, VB, CPB>(h, tb, geo, fa, grid, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "operator kernel launch");
  return 0;
}

// FP32 operator with one thread per plane of a cell (dg_kernels_plane.cuh), modes 0 and 1.  V is kept in the plane
// layout between its two kernels.  Measured on GB300 at about 24 M DOF (FP32 Jacobian applies), against the line
// kernels: k = 5 222 us vs 252 us; k = 1, 2, 3, 4, 6: 731, 464, 329, 400, 414 us vs 468, 385, 256, 273, 274 us
// (odd N and N = 2 leave the plane transposes scalar and short).  So only k = 5 takes it.
template <int N>
int apply_plane(const dg_handle* h, const float* z, float* y, int mode, int stages, cudaStream_t s) {
  using C = dgk::PlaneCfg<N>;
  const size_t smem_cell = (size_t)C::CPB * C::CS * sizeof(float);
  const size_t smem_face = (size_t)C::CPB * (C::CS + C::GS) * sizeof(float);
  static DeviceOnce once;
  if (int rc = once.run([&]() -> int {
        cudaError_t e = cudaFuncSetAttribute(dgk::dg_cell_kernel_pl<N>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)smem_cell);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(dgk::dg_face_kernel_pl<N, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_face);
        if (e == cudaSuccess)
          e = cudaFuncSetAttribute(dgk::dg_face_kernel_pl<N, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)smem_face);
        return e == cudaSuccess ? 0 : cuda_fail(e, "cudaFuncSetAttribute(plane kernels)");
      }))
    return rc;
  const auto tb = make_tab<N, float>(h->tab);
  dgk::PlaneTab<N> pt;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) pt.A[i][j] = (float)h->tab.A[i][j];
  const auto geo = make_geo<float>(h);
  const unsigned grid = (unsigned)((h->ncell + C::CPB - 1) / C::CPB);
  float* V = static_cast<float*>(h->work_V);
  float* tr = static_cast<float*>(h->work_tr);
  const int ncell = (int)h->ncell;
  if (stages & 1)
    dgk::dg_cell_kernel_pl<N><<<grid, C::THREADS, smem_cell, s>>>(tb, geo, z, static_cast<const float*>(h->p32.D),
                                                                   V, tr, nullptr, ncell);
  if (stages & 2) {
    dgk::FaceArgs<float, float> fa;
    fa.V = V;
    fa.traces = tr;
    fa.fc = static_cast<const float*>(h->p32.fc);
    fa.F = mode == 1 ? static_cast<const float*>(h->p32.F) : nullptr;
    for (int i = 0; i < 6; ++i) fa.g[i] = nullptr;
    fa.y = y;
    fa.mode = mode;
    fa.u = z;
    fa.z0 = nullptr;
    fa.cz = fa.cu = fa.cr = 0.0;
    if (h->periodic[0] || h->periodic[1] || h->periodic[2])
      dgk::dg_face_kernel_pl<N, true><<<grid, C::THREADS, smem_face, s>>>(tb, pt, geo, fa, nullptr, ncell, 0);
    else
      dgk::dg_face_kernel_pl<N, false><<<grid, C::THREADS, smem_face, s>>>(tb, pt, geo, fa, nullptr, ncell, 0);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "FP32 operator kernel launch");
}

// t = (A z)_to for a z that vanishes outside the cells `from` (the plane kernels: the cell kernel on `from` only,
// the face kernel on `to` only with the listed cells' own volume and traces taken as zero), i.e. the coupling of
// the cells `to` to the cells `from`; `from` and `to` are two colours of a red-black colouring.  t is written on
// the cells `to` only; z is read on the cells `from` only.
template <int N>
int apply_plane_offdiag(const dg_handle* h, const float* z, float* t, const int* from, int nfrom, const int* to,
                        int nto, cudaStream_t s) {
  using C = dgk::PlaneCfg<N>;
  if (int rc = apply_plane<N>(h, z, t, 0, 0, s)) return rc;  // the shared-memory attributes (no launch)
  const size_t smem_cell = (size_t)C::CPB * C::CS * sizeof(float);
  const size_t smem_face = (size_t)C::CPB * (C::CS + C::GS) * sizeof(float);
  const auto tb = make_tab<N, float>(h->tab);
  dgk::PlaneTab<N> pt;
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) pt.A[i][j] = (float)h->tab.A[i][j];
  const auto geo = make_geo<float>(h);
  float* V = static_cast<float*>(h->work_V);
  float* tr = static_cast<float*>(h->work_tr);
  if (nfrom > 0)
    dgk::dg_cell_kernel_pl<N><<<(unsigned)((nfrom + C::CPB - 1) / C::CPB), C::THREADS, smem_cell, s>>>(
        tb, geo, z, static_cast<const float*>(h->p32.D), V, tr, from, nfrom);
  if (nto > 0) {
    dgk::FaceArgs<float, float> fa;
    fa.V = V;
    fa.traces = tr;
    fa.fc = static_cast<const float*>(h->p32.fc);
    fa.F = nullptr;
    for (int i = 0; i < 6; ++i) fa.g[i] = nullptr;
    fa.y = t;
    fa.mode = 0;
    fa.u = z;
    fa.z0 = nullptr;
    fa.cz = fa.cu = fa.cr = 0.0;
    const unsigned grid = (unsigned)((nto + C::CPB - 1) / C::CPB);
    if (h->periodic[0] || h->periodic[1] || h->periodic[2])
      dgk::dg_face_kernel_pl<N, true><<<grid, C::THREADS, smem_face, s>>>(tb, pt, geo, fa, to, nto, 1);
    else
      dgk::dg_face_kernel_pl<N, false><<<grid, C::THREADS, smem_face, s>>>(tb, pt, geo, fa, to, nto, 1);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? 0 : cuda_fail(e, "FP32 off-diagonal operator launch");
}

// FP64 applies: meshes with fewer full tiles than SMs take the small-tile variant; FP32 applies of degree 5
// (modes 0, 1) take the plane kernels
template <int N, typename T, typename TV>
int apply_sized(const dg_handle* h, const TV* z, TV* y, int mode, int stages, cudaStream_t s, const StageArgs* st) {
  if constexpr (std::is_same<T, float>::value && std::is_same<TV, float>::value && N == 6) {
    if (mode == 0 || mode == 1) return apply_plane<N>(h, z, y, mode, stages, s);
  }
  if constexpr (std::is_same<T, double>::value && std::is_same<TV, double>::value &&
                small_cpb<N>() < dgk::Launch<N>::CPB) {
    if (h->ncell < (int64_t)sm_count() * dgk::Launch<N>::CPB)
      return apply_n<N, T, TV, N, false, small_cpb<N>()>(h, z, y, mode, stages, s, st);
  }
  return apply_n<N, T, TV>(h, z, y, mode, stages, s, st);
}

template <int N, typename T, int M = N, bool VB = false>
int rhs_n(const dg_handle* h, const T* f, const T* const g[6], T* F, cudaStream_t s, bool project = false) {
  if (int rc = set_smem_attrs<N, T, T, M, VB>()) return rc;
  constexpr int CPB = dgk::Launch<M>::CPB;
  const Buffers& bf = sizeof(T) == 8 ? h->p64 : h->p32;
  const auto tb = make_tab<N, T, M>(h->tab);
  auto geo = geo_for<T, VB>(h);
  if (project) geo.vol = T(1);  // (f, phi_i)_T / |T|: the mass matrix is |T| I
  const unsigned grid = (unsigned)((h->ncell + CPB - 1) / CPB);
  dgk::FaceArgs<T> fa;
  fa.V = f;
  fa.traces = nullptr;
  fa.fc = static_cast<const T*>(bf.fc);
  fa.F = nullptr;
  for (int i = 0; i < 6; ++i) fa.g[i] = project ? nullptr : g[i];
  fa.y = F;
  fa.mode = 2;
  fa.u = nullptr;
  fa.z0 = nullptr;
  fa.cz = fa.cu = fa.cr = 0.0;
  launch_face<N, T, T, M, VB>(h, tb, geo, fa, grid, s);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "rhs kernel launch");
  return 0;
}

// Diagonal blocks of cells [cell_base, cell_base + ncells): column j of block c is written to
// out[(c * N^3 + j) * N^3 + i], i.e. each block is stored as A_TT^T in row-major order.
template <int N>
int diag_blocks_n(const dg_handle* h, double* out, int cell_base, int ncells, double* V, double* tr, cudaStream_t s) {
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
  fa.u = nullptr;
  fa.z0 = nullptr;
  fa.cz = fa.cu = fa.cr = 0.0;
  dgk::dg_face_kernel<N, double, true, dgk::Launch<N>::CPB, double, N, false, true>
      <<<grid, dgk::Launch<N>::THREADS, face_smem<N, double>(), s>>>(tb, geo, fa, sa);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "diagonal block kernel launch");
  return 0;
}

template <typename T, typename TV = T>
int apply_dispatch(const dg_handle* h, const TV* z, TV* y, int mode, int stages, cudaStream_t s,
                   const StageArgs* st = nullptr) {
  switch (h->N) {
    case 2: return apply_sized<2, T, TV>(h, z, y, mode, stages, s, st);
    case 3: return apply_sized<3, T, TV>(h, z, y, mode, stages, s, st);
    case 4: return apply_sized<4, T, TV>(h, z, y, mode, stages, s, st);
    case 5: return apply_sized<5, T, TV>(h, z, y, mode, stages, s, st);
    case 6: return apply_sized<6, T, TV>(h, z, y, mode, stages, s, st);
    case 7: return apply_sized<7, T, TV>(h, z, y, mode, stages, s, st);
    case 8: return apply_sized<8, T, TV>(h, z, y, mode, stages, s, st);
    case 9: return apply_sized<9, T, TV>(h, z, y, mode, stages, s, st);
    case 10: return apply_sized<10, T, TV>(h, z, y, mode, stages, s, st);
    case 11: return apply_sized<11, T, TV>(h, z, y, mode, stages, s, st);
    default: set_error("unsupported degree"); return DG_ERR_INVALID_ARG;
  }
}

template <typename T>
int rhs_dispatch(const dg_handle* h, const T* f, const T* const g[6], T* F, cudaStream_t s, bool project = false) {
  switch (h->N) {
    case 2: return rhs_n<2, T>(h, f, g, F, s, project);
    case 3: return rhs_n<3, T>(h, f, g, F, s, project);
    case 4: return rhs_n<4, T>(h, f, g, F, s, project);
    case 5: return rhs_n<5, T>(h, f, g, F, s, project);
    case 6: return rhs_n<6, T>(h, f, g, F, s, project);
    case 7: return rhs_n<7, T>(h, f, g, F, s, project);
    case 8: return rhs_n<8, T>(h, f, g, F, s, project);
    case 9: return rhs_n<9, T>(h, f, g, F, s, project);
    case 10: return rhs_n<10, T>(h, f, g, F, s, project);
    case 11: return rhs_n<11, T>(h, f, g, F, s, project);
    default: set_error("unsupported degree"); return DG_ERR_INVALID_ARG;
  }
}

}  // namespace dgi

namespace dgi {

// The velocity field kernels: M = N (q = 2p) or M = N + 2 (q = 2p+4), degrees 1..8, FP64 vectors, operator
// in FP64 (T = double) or double-float (T = dfl).
template <int N, typename T = double>
int apply_vb_n(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
               cudaStream_t s) {
  if (h->M == N) return apply_n<N, T, double, N, true>(h, z, y, mode, stages, s, st);
  if (h->M == N + 2) return apply_n<N, T, double, N + 2, true>(h, z, y, mode, stages, s, st);
  set_error("unsupported number of quadrature points");
  return DG_ERR_INVALID_ARG;
}
template <int N>
int rhs_vb_n(const dg_handle* h, const double* f, const double* const g[6], double* F, cudaStream_t s,
             bool project) {
  if (h->M == N) return rhs_n<N, double, N, true>(h, f, g, F, s, project);
  if (h->M == N + 2) return rhs_n<N, double, N + 2, true>(h, f, g, F, s, project);
  set_error("unsupported number of quadrature points");
  return DG_ERR_INVALID_ARG;
}

}  // namespace dgi

namespace dgi {

// Tensor diffusion / affine geometry kernels (M = N), FP64 (T = double) or double-float (T = dfl) operator.
template <int N, typename T>
int set_td_smem_attrs() {
  static DeviceOnce once;
  return once.run([&]() -> int {
    constexpr int CPB = dgk::Launch<N>::CPB;
    cudaError_t e = cudaFuncSetAttribute(dgk::dg_cell_kernel_td<N, T, CPB, double, N>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * cell_smem<N, T>()));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_cell_kernel_td)");
    e = cudaFuncSetAttribute(dgk::face_kernel_for<N, T, CPB, double, N, false, true, true>(),
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(face_smem<N, T>() + (size_t)CPB * 4 * N * N * sizeof(T)));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_face_kernel td)");
    return 0;
  });
}

template <int N, typename T>
int apply_td_n(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
               const double* const g6[6], cudaStream_t s, bool project) {
  if (int rc = set_td_smem_attrs<N, T>()) return rc;
  constexpr int CPB = dgk::Launch<N>::CPB;
  const Buffers& bf = buffers_for<T>(h);
  const auto tb = make_tab<N, T>(h->tab);
  auto geo = make_geo<T>(h);
  const unsigned grid = (unsigned)((h->ncell + CPB - 1) / CPB);
  T* V = static_cast<T*>(h->work_V);
  T* tr = static_cast<T*>(h->work_tr);
  if (mode != 2 && (stages & 1))
    dgk::dg_cell_kernel_td<N, T, CPB, double, N><<<grid, dgk::Launch<N>::THREADS, 2 * cell_smem<N, T>(), s>>>(
        tb, geo, z, static_cast<const T*>(bf.D), nullptr, V, tr);
  dgk::FaceArgs<T, double> fa;
  fa.V = mode == 2 ? reinterpret_cast<const T*>(z) : V;
  fa.traces = mode == 2 ? nullptr : tr;
  fa.fc = static_cast<const T*>(bf.fc);
  fa.F = (mode == 1 || mode == 3) ? static_cast<const T*>(bf.F) : nullptr;
  for (int i = 0; i < 6; ++i) fa.g[i] = (mode == 2 && !project && g6) ? reinterpret_cast<const T*>(g6[i]) : nullptr;
  fa.y = y;
  fa.mode = mode;
  fa.u = z;
  fa.z0 = nullptr;
  fa.cz = fa.cu = fa.cr = 0.0;
  if (mode == 2 && project) geo.vol = T(1);
  if (mode == 3) {
    if (!st) {
      set_error("Runge-Kutta stage without coefficients");
      return DG_ERR_INVALID_ARG;
    }
    fa.z0 = st->z0;
    fa.cz = st->cz;
    fa.cu = st->cu;
    fa.cr = st->cr;
  }
  if (stages & 2)
    dgk::face_kernel_for<N, T, CPB, double, N, false, true, true>()
        <<<grid, dgk::Launch<N>::THREADS, face_smem<N, T>() + (size_t)CPB * 4 * N * N * sizeof(T), s>>>(
            tb, geo, fa, dgk::SelfArgs{0, 0});
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "tensor-diffusion kernel launch");
  return 0;
}

}  // namespace dgi

namespace dgi {

// Point-wise coefficient kernels (Problem B of Sec. 5.1): the tensor-diffusion kernels with K, beta and c read
// at every volume point and the face coefficients at every face point; M = N (q = 2p) or M = N + 2
// (q = 2p+4); FP64 (T = double) or double-float (T = dfl) operator, FP64 vectors.
template <int N, typename T, int M>
int set_pw_smem_attrs() {
  static DeviceOnce once;
  return once.run([&]() -> int {
    constexpr int CPB = dgk::Launch<M>::CPB;
    cudaError_t e = cudaFuncSetAttribute(dgk::dg_cell_kernel_td<N, T, CPB, double, M, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(2 * cell_smem<M, T>()));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_cell_kernel_td pw)");
    e = cudaFuncSetAttribute(dgk::face_kernel_for<N, T, CPB, double, M, true, true, true, true>(),
                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(face_smem<M, T>() + (size_t)CPB * 4 * M * M * sizeof(T)));
    if (e != cudaSuccess) return cuda_fail(e, "cudaFuncSetAttribute(dg_face_kernel pw)");
    return 0;
  });
}

template <int N, typename T, int M>
int apply_pw_nm(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                const double* const g6[6], cudaStream_t s, bool project) {
  if (int rc = set_pw_smem_attrs<N, T, M>()) return rc;
  constexpr int CPB = dgk::Launch<M>::CPB;
  const bool pair = std::is_same<T, dgk::dfl>::value;
  const Buffers& bf = buffers_for<T>(h);
  const auto tb = make_tab<N, T, M>(h->tab);
  auto geo = geo_for<T, true>(h);  // normal velocity at the face points
  const unsigned grid = (unsigned)((h->ncell + CPB - 1) / CPB);
  T* V = static_cast<T*>(h->work_V);
  T* tr = static_cast<T*>(h->work_tr);
  if (mode != 2 && (stages & 1))
    dgk::dg_cell_kernel_td<N, T, CPB, double, M, true><<<grid, dgk::Launch<M>::THREADS, 2 * cell_smem<M, T>(), s>>>(
        tb, geo, z, static_cast<const T*>(pair ? h->kqX : h->kq64), static_cast<const T*>(pair ? h->kfX : h->kf64),
        V, tr);
  dgk::FaceArgs<T, double> fa;
  fa.V = mode == 2 ? reinterpret_cast<const T*>(z) : V;
  fa.traces = mode == 2 ? nullptr : tr;
  fa.fc = static_cast<const T*>(bf.fc);
  fa.F = (mode == 1 || mode == 3) ? static_cast<const T*>(bf.F) : nullptr;
  for (int i = 0; i < 6; ++i) fa.g[i] = (mode == 2 && !project && g6) ? reinterpret_cast<const T*>(g6[i]) : nullptr;
  fa.y = y;
  fa.mode = mode;
  fa.u = z;
  fa.z0 = nullptr;
  fa.cz = fa.cu = fa.cr = 0.0;
  if (mode == 2 && project) geo.vol = T(1);
  if (mode == 3) {
    if (!st) {
      set_error("Runge-Kutta stage without coefficients");
      return DG_ERR_INVALID_ARG;
    }
    fa.z0 = st->z0;
    fa.cz = st->cz;
    fa.cu = st->cu;
    fa.cr = st->cr;
  }
  if (stages & 2)
    dgk::face_kernel_for<N, T, CPB, double, M, true, true, true, true>()
        <<<grid, dgk::Launch<M>::THREADS, face_smem<M, T>() + (size_t)CPB * 4 * M * M * sizeof(T), s>>>(
            tb, geo, fa, dgk::SelfArgs{0, 0});
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(e, "point-wise coefficient kernel launch");
  return 0;
}

template <int N, typename T>
int apply_pw_n(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
               const double* const g6[6], cudaStream_t s, bool project) {
  if (h->M == N) return apply_pw_nm<N, T, N>(h, z, y, mode, stages, st, g6, s, project);
  if (h->M == N + 2) return apply_pw_nm<N, T, N + 2>(h, z, y, mode, stages, st, g6, s, project);
  set_error("unsupported number of quadrature points");
  return DG_ERR_INVALID_ARG;
}

template <typename T>
int pw_dispatch(const dg_handle* h, const double* z, double* y, int mode, int stages, const StageArgs* st,
                const double* const g6[6], cudaStream_t s, bool project) {
  switch (h->N) {
    case 2: return apply_pw_n<2, T>(h, z, y, mode, stages, st, g6, s, project);
    case 3: return apply_pw_n<3, T>(h, z, y, mode, stages, st, g6, s, project);
    case 4: return apply_pw_n<4, T>(h, z, y, mode, stages, st, g6, s, project);
    case 5: return apply_pw_n<5, T>(h, z, y, mode, stages, st, g6, s, project);
    case 6: return apply_pw_n<6, T>(h, z, y, mode, stages, st, g6, s, project);
    case 7: return apply_pw_n<7, T>(h, z, y, mode, stages, st, g6, s, project);
    case 8: return apply_pw_n<8, T>(h, z, y, mode, stages, st, g6, s, project);
    case 9: return apply_pw_n<9, T>(h, z, y, mode, stages, st, g6, s, project);
    default: set_error("point-wise coefficient kernels support degrees 1..8"); return DG_ERR_INVALID_ARG;
  }
}

}  // namespace dgi
