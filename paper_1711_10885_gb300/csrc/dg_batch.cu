// dg_batch.cu -- many uneven problems (different meshes and degrees) applied in one CUDA graph launch.
//
// The two operator phases (cell kernel, face kernel) each run as ONE persistent kernel over the tiles of
// all problems: a CTA takes the next tile from a global counter (a work queue without waiting) and runs
// the tile with the degree's cell or face code, then takes the next one.  The graph holds the two
// counter resets and the two persistent kernels.  Cells per CTA (and so the CTA's thread layout) is
// chosen per degree by timing the candidates at batch creation (autotuner).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dg_internal.h"
#include "dg_launch.cuh"

namespace dgbt {

constexpr int NMIN = 2, NMAX = 9;  // degrees 1..8
constexpr int THREADS = 256;

template <int N>
struct Cpb {
  static constexpr int FULL = dgk::Launch<N>::CPB;
  static constexpr int HALF = FULL / 2 > 0 ? FULL / 2 : 1;
};

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
  int problem, cell0, here, variant;
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

#define DG_BATCH_CASES(X) X(2, t2) X(3, t3) X(4, t4) X(5, t5) X(6, t6) X(7, t7) X(8, t8) X(9, t9)

__global__ void __launch_bounds__(THREADS)
dg_batch_cell_kernel(const __grid_constant__ Tabs tabs, const Problem* __restrict__ probs,
                     const Tile* __restrict__ tiles, int ntiles, int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int ti = s_tile;
    __syncthreads();
    if (ti >= ntiles) return;
    const Tile tl = tiles[ti];
    const Problem& p = probs[tl.problem];
    switch (p.N * 2 + tl.variant) {
#define X(NV, TB)                                                                                                  \
  case 2 * NV:                                                                                                     \
    dgk::cell_tile<NV, double, false, Cpb<NV>::FULL>(tabs.TB, p.geo, p.z, p.D, p.V, p.tr, tl.cell0, tl.here, 0,   \
                                                     smem);                                                        \
    break;                                                                                                         \
  case 2 * NV + 1:                                                                                                 \
    dgk::cell_tile<NV, double, false, Cpb<NV>::HALF>(tabs.TB, p.geo, p.z, p.D, p.V, p.tr, tl.cell0, tl.here, 0,   \
                                                     smem);                                                        \
    break;
      DG_BATCH_CASES(X)
#undef X
      default:
        break;
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(THREADS)
dg_batch_face_kernel(const __grid_constant__ Tabs tabs, const Problem* __restrict__ probs,
                     const Tile* __restrict__ tiles, int ntiles, int* __restrict__ counter) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_tile;
  for (;;) {
    if (threadIdx.x == 0) s_tile = atomicAdd(counter, 1);
    __syncthreads();
    const int ti = s_tile;
    __syncthreads();
    if (ti >= ntiles) return;
    const Tile tl = tiles[ti];
    const Problem& p = probs[tl.problem];
    const dgk::FaceArgs<double> fa = face_args(p);
    switch (p.N * 2 + tl.variant) {
#define X(NV, TB)                                                                                        \
  case 2 * NV:                                                                                           \
    dgk::face_tile<NV, double, false, Cpb<NV>::FULL, double, NV, false, true>(tabs.TB, p.geo, fa, tl.cell0,  \
                                                                              tl.here, 0, smem);         \
    break;                                                                                               \
  case 2 * NV + 1:                                                                                       \
    dgk::face_tile<NV, double, false, Cpb<NV>::HALF, double, NV, false, true>(tabs.TB, p.geo, fa, tl.cell0,  \
                                                                              tl.here, 0, smem);         \
    break;
      DG_BATCH_CASES(X)
#undef X
      default:
        break;
    }
    __syncthreads();
  }
}

int cpb_of(int N, int variant) {
  switch (N) {
#define X(NV, TB) \
  case NV:        \
    return variant ? Cpb<NV>::HALF : Cpb<NV>::FULL;
    DG_BATCH_CASES(X)
#undef X
    default:
      return 1;
  }
}

size_t smem_bytes() {
  size_t m = 0;
  for (int N = NMIN; N <= NMAX; ++N) m = std::max(m, 2 * (size_t)cpb_of(N, 0) * (N + 1) * N * N * sizeof(double));
  return m;
}

}  // namespace dgbt

struct dg_batch {
  std::vector<dg_handle*> hs;
  std::vector<dgbt::Problem> probs;
  dgbt::Problem* d_probs = nullptr;
  dgbt::Problem* h_probs_pinned = nullptr;
  dgbt::Tile* d_tiles = nullptr;
  int ntiles = 0;
  int* d_counters = nullptr;
  dgbt::Tabs tabs;
  int variant[dgbt::NMAX + 1] = {};
  float tune_ms[dgbt::NMAX + 1][2] = {};
  int grid = 0;
  size_t smem = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool uploaded = false;  // device descriptors match probs
};

namespace {

using namespace dgi;

int cfail(cudaError_t e, const char* what) { return e == cudaSuccess ? 0 : cuda_fail(e, what); }

std::vector<dgbt::Tile> make_tiles(const dg_batch* b, int onlyN, const int* variant_of) {
  std::vector<dgbt::Tile> t;
  for (int p = 0; p < (int)b->hs.size(); ++p) {
    const int N = b->hs[p]->N;
    if (onlyN && N != onlyN) continue;
    const int v = variant_of[N];
    const int cpb = dgbt::cpb_of(N, v);
    for (int64_t c0 = 0; c0 < b->hs[p]->ncell; c0 += cpb)
      t.push_back({p, (int)c0, (int)std::min<int64_t>(cpb, b->hs[p]->ncell - c0), v});
  }
  // heaviest first (FP64 work per cell grows like N^4), so the queue ends on light tiles
  std::stable_sort(t.begin(), t.end(), [&](const dgbt::Tile& a, const dgbt::Tile& c) {
    const double wa = std::pow((double)b->hs[a.problem]->N, 4) * a.here;
    const double wc = std::pow((double)b->hs[c.problem]->N, 4) * c.here;
    return wa > wc;
  });
  return t;
}

int enqueue(dg_batch* b, int ntiles, cudaStream_t s) {
  if (int rc = cfail(cudaMemsetAsync(b->d_counters, 0, 2 * sizeof(int), s), "batch counter reset")) return rc;
  dgbt::dg_batch_cell_kernel<<<b->grid, dgbt::THREADS, b->smem, s>>>(b->tabs, b->d_probs, b->d_tiles, ntiles,
                                                                     b->d_counters);
  dgbt::dg_batch_face_kernel<<<b->grid, dgbt::THREADS, b->smem / 2, s>>>(b->tabs, b->d_probs, b->d_tiles, ntiles,
                                                                         b->d_counters + 1);
  return cfail(cudaGetLastError(), "batch kernels");
}

int upload_probs(dg_batch* b, cudaStream_t s) {
  std::memcpy(b->h_probs_pinned, b->probs.data(), b->probs.size() * sizeof(dgbt::Problem));
  if (int rc = cfail(cudaMemcpyAsync(b->d_probs, b->h_probs_pinned, b->probs.size() * sizeof(dgbt::Problem),
                                     cudaMemcpyHostToDevice, s),
                     "batch descriptor upload"))
    return rc;
  return 0;
}

void destroy(dg_batch* b) {
  if (!b) return;
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  cudaFree(b->d_probs);
  cudaFree(b->d_tiles);
  cudaFree(b->d_counters);
  if (b->h_probs_pinned) cudaFreeHost(b->h_probs_pinned);
  delete b;
}

}  // namespace

extern "C" {

int dg_batch_destroy(dg_batch* b) {
  destroy(b);
  return DG_OK;
}

int dg_batch_create(dg_handle* const* hs, int32_t count, void* stream, dg_batch** out) {
  if (!out || !hs || count < 1) {
    set_error("dg_batch_create: need count >= 1 handles and an output pointer");
    return DG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  int dev = -1;
  cudaGetDevice(&dev);
  for (int i = 0; i < count; ++i)
    if (!hs[i] || hs[i]->N < dgbt::NMIN || hs[i]->N > dgbt::NMAX || hs[i]->device != dev || hs[i]->vb || hs[i]->td) {
      set_error("dg_batch_create: every handle must exist, live on the current device, have 1 <= k <= 8, a "
                "constant velocity, m = k+1 and scalar diffusion on the axis-parallel grid");
      return DG_ERR_INVALID_ARG;
    }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  dg_batch* b = new dg_batch();
  b->hs.assign(hs, hs + count);
  // 1D tables of every degree (the same as a standalone handle of that degree builds)
  {
    dgi::Tables1D t;
#define X(NV, TB)                              \
  dgi::build_tables(NV, NV, &t);                 \
  b->tabs.TB = dgi::make_tab<NV, double>(t);
    DG_BATCH_CASES(X)
#undef X
  }
  b->probs.resize(count);
  size_t max_ndof = 0;
  for (int i = 0; i < count; ++i) {
    const dg_handle* h = hs[i];
    dgbt::Problem& p = b->probs[i];
    p.z = nullptr;
    p.y = nullptr;
    p.D = static_cast<const double*>(h->p64.D);
    p.fc = static_cast<const double*>(h->p64.fc);
    p.F = static_cast<const double*>(h->p64.F);
    p.V = static_cast<double*>(h->work_V);
    p.tr = static_cast<double*>(h->work_tr);
    p.geo = dgi::make_geo<double>(h);
    p.N = h->N;
    p.mode = 0;
    max_ndof = std::max(max_ndof, (size_t)h->ncell * h->N * h->N * h->N);
  }
  int rc = 0;
  size_t max_tiles = 0;
  for (int i = 0; i < count; ++i) max_tiles += (size_t)hs[i]->ncell;  // at least one cell per tile
  rc = cfail(cudaMalloc(&b->d_probs, count * sizeof(dgbt::Problem)), "cudaMalloc(batch descriptors)");
  if (!rc) rc = cfail(cudaMallocHost(&b->h_probs_pinned, count * sizeof(dgbt::Problem)), "cudaMallocHost(batch)");
  if (!rc) rc = cfail(cudaMalloc(&b->d_tiles, max_tiles * sizeof(dgbt::Tile)), "cudaMalloc(batch tiles)");
  if (!rc) rc = cfail(cudaMalloc(&b->d_counters, 2 * sizeof(int)), "cudaMalloc(batch counters)");
  b->smem = dgbt::smem_bytes();
  if (!rc)
    rc = cfail(cudaFuncSetAttribute(dgbt::dg_batch_cell_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                    (int)b->smem),
               "batch smem attribute");
  int occ = 0, sms = 0;
  if (!rc)
    rc = cfail(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, dgbt::dg_batch_cell_kernel, dgbt::THREADS,
                                                             b->smem),
               "batch occupancy");
  if (!rc) rc = cfail(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev), "SM count");
  b->grid = std::max(1, occ) * sms;

  // autotune cells per CTA per degree: time both candidates on that degree's problems alone
  double* tz = nullptr;
  double* ty = nullptr;
  size_t tot = 0;
  for (int i = 0; i < count; ++i) tot += (size_t)hs[i]->ncell * hs[i]->N * hs[i]->N * hs[i]->N;
  if (!rc) rc = cfail(cudaMalloc(&tz, tot * sizeof(double)), "cudaMalloc(tuning input)");
  if (!rc) rc = cfail(cudaMalloc(&ty, tot * sizeof(double)), "cudaMalloc(tuning output)");
  if (!rc) rc = cfail(cudaMemsetAsync(tz, 0, tot * sizeof(double), s), "tuning memset");
  if (!rc) {
    size_t off = 0;
    for (int i = 0; i < count; ++i) {
      b->probs[i].z = tz + off;
      b->probs[i].y = ty + off;
      off += (size_t)hs[i]->ncell * hs[i]->N * hs[i]->N * hs[i]->N;
    }
    rc = upload_probs(b, s);
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (!rc) rc = cfail(cudaEventCreate(&e0), "event");
  if (!rc) rc = cfail(cudaEventCreate(&e1), "event");
  for (int N = dgbt::NMIN; !rc && N <= dgbt::NMAX; ++N) {
    bool present = false;
    for (int i = 0; i < count; ++i) present |= hs[i]->N == N;
    if (!present) continue;
    for (int v = 0; v < 2 && !rc; ++v) {
      int var[dgbt::NMAX + 1];
      for (int q = 0; q <= dgbt::NMAX; ++q) var[q] = v;
      std::vector<dgbt::Tile> t = make_tiles(b, N, var);
      rc = cfail(cudaMemcpyAsync(b->d_tiles, t.data(), t.size() * sizeof(dgbt::Tile), cudaMemcpyHostToDevice, s),
                 "tile upload");
      float best = 1e30f;
      for (int rep = 0; rep < 4 && !rc; ++rep) {
        rc = cfail(cudaEventRecord(e0, s), "event");
        if (!rc) rc = enqueue(b, (int)t.size(), s);
        if (!rc) rc = cfail(cudaEventRecord(e1, s), "event");
        if (!rc) rc = cfail(cudaEventSynchronize(e1), "tuning sync");
        float ms = 0;
        if (!rc) cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0) best = std::min(best, ms);  // first run warms up
      }
      b->tune_ms[N][v] = best;
    }
    b->variant[N] = b->tune_ms[N][1] < b->tune_ms[N][0] ? 1 : 0;
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(tz);
  cudaFree(ty);
  if (!rc) {
    std::vector<dgbt::Tile> t = make_tiles(b, 0, b->variant);
    b->ntiles = (int)t.size();
    rc = cfail(cudaMemcpyAsync(b->d_tiles, t.data(), t.size() * sizeof(dgbt::Tile), cudaMemcpyHostToDevice, s),
               "tile upload");
    if (!rc) rc = cfail(cudaStreamSynchronize(s), "batch setup sync");
  }
  for (auto& p : b->probs) p.z = nullptr, p.y = nullptr;
  if (rc) {
    destroy(b);
    return rc;
  }
  *out = b;
  return DG_OK;
}

int dg_batch_tuning(const dg_batch* b, int32_t k, int32_t* cells_per_cta, float* ms_candidates) {
  if (!b || k < 1 || k > 8) {
    set_error("dg_batch_tuning: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  const int N = k + 1;
  if (cells_per_cta) *cells_per_cta = dgbt::cpb_of(N, b->variant[N]);
  if (ms_candidates) {
    ms_candidates[0] = b->tune_ms[N][0];
    ms_candidates[1] = b->tune_ms[N][1];
  }
  return DG_OK;
}

int dg_batch_apply(dg_batch* b, const double* const* in_dev, double* const* out_dev, int32_t residual, void* stream) {
  if (!b || !in_dev || !out_dev) {
    set_error("dg_batch_apply: null arguments");
    return DG_ERR_INVALID_ARG;
  }
  const int count = (int)b->probs.size();
  bool changed = !b->uploaded;
  for (int i = 0; i < count; ++i) {
    if (!in_dev[i] || !out_dev[i] || in_dev[i] == out_dev[i]) {
      set_error("dg_batch_apply: problem " + std::to_string(i) + " has a null or aliased vector");
      return DG_ERR_INVALID_ARG;
    }
    changed |= b->probs[i].z != in_dev[i] || b->probs[i].y != out_dev[i] || b->probs[i].mode != (residual ? 1 : 0);
    b->probs[i].z = in_dev[i];
    b->probs[i].y = out_dev[i];
    b->probs[i].mode = residual ? 1 : 0;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  // the descriptors are read by the kernels at run time, so one captured graph serves every call;
  // they are re-uploaded only when a vector or the mode changed since the last call
  if (changed) {
    cudaError_t e = cudaStreamSynchronize(s);  // the pinned staging copy must not be overwritten in flight
    if (e != cudaSuccess) return cuda_fail(e, "dg_batch_apply sync");
    if (int rc = upload_probs(b, s)) return rc;
    b->uploaded = true;
  }
  if (!b->exec) {
    cudaStream_t cap;
    if (int rc = cfail(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "capture stream")) return rc;
    int rc = cfail(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "begin capture");
    if (!rc) rc = enqueue(b, b->ntiles, cap);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cap, &g);
    if (!rc) rc = cfail(ee, "end capture");
    if (!rc) rc = cfail(cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
    b->graph = g;
    cudaStreamDestroy(cap);
    if (rc) return rc;
  }
  return cfail(cudaGraphLaunch(b->exec, s), "graph launch");
}

}  // extern "C"
