// dg_batch.cu -- many uneven problems (different meshes and degrees) applied in one CUDA graph launch.
//
// For every degree present the two operator phases (cell kernel, face kernel) run as persistent kernels over
// that degree's tiles: a CTA takes the next tile from a global counter (a work queue without waiting), runs
// it with the degree's cell or face code, and takes the next one.  The graph forks one branch per degree
// (counter reset, cell kernel, face kernel), so the branches of different degrees overlap on the GPU, and
// joins them.  Each degree has its own kernels, so its register allocation and launch bounds are its own.
// The thread layout of every degree (cells per CTA x lines per thread, four candidates) is chosen at batch
// creation by timing each candidate on that degree's problems alone (autotuner); all timings are kept.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "dg_batch_kernels.cuh"
#include "dg_internal.h"

struct dg_batch {
  std::vector<dg_handle*> hs;
  std::vector<dgbt::Problem> probs;
  dgbt::Problem* d_probs = nullptr;
  dgbt::Problem* h_probs_pinned = nullptr;
  dgbt::Tile* d_tiles = nullptr;      // the tiles of every degree, degree by degree
  int* d_counters = nullptr;          // two queue counters per degree
  dgbt::Tabs tabs;
  bool present[dgbt::NMAX + 1] = {};
  int variant[dgbt::NMAX + 1] = {};
  int tile_off[dgbt::NMAX + 1] = {};  // first tile of a degree in d_tiles
  int ntiles[dgbt::NMAX + 1] = {};
  int grid_cell[dgbt::NMAX + 1] = {}, grid_face[dgbt::NMAX + 1] = {};
  float tune_ms[dgbt::NMAX + 1][dgbt::NVAR] = {};
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  bool uploaded = false;  // device descriptors match probs
};

namespace {

using namespace dgi;

int cfail(cudaError_t e, const char* what) { return e == cudaSuccess ? 0 : cuda_fail(e, what); }

// the tiles of degree N for cells-per-CTA cpb, heaviest problems first (the queue ends on light tiles)
std::vector<dgbt::Tile> make_tiles(const dg_batch* b, int N, int cpb) {
  std::vector<dgbt::Tile> t;
  for (int p = 0; p < (int)b->hs.size(); ++p) {
    if (b->hs[p]->N != N) continue;
    for (int64_t c0 = 0; c0 < b->hs[p]->ncell; c0 += cpb)
      t.push_back({p, (int)c0, (int)std::min<int64_t>(cpb, b->hs[p]->ncell - c0)});
  }
  std::stable_sort(t.begin(), t.end(), [](const dgbt::Tile& a, const dgbt::Tile& c) { return a.here > c.here; });
  return t;
}

// opt-in shared memory and persistent grid sizes (one wave of resident CTAs) of a variant
int prepare_variant(const dgbt::VariantInfo& v, int* grid_cell, int* grid_face) {
  int occ_c = 0, occ_f = 0;
  cudaError_t e = cudaFuncSetAttribute(v.cell, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem_cell);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(v.face, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)v.smem_face);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_c, v.cell, v.threads, v.smem_cell);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ_f, v.face, v.threads, v.smem_face);
  if (e != cudaSuccess) return cuda_fail(e, "batch kernel attributes");
  *grid_cell = std::max(1, occ_c) * sm_count();
  *grid_face = std::max(1, occ_f) * sm_count();
  return 0;
}

// one degree's branch: counter reset, cell kernel, face kernel (tiles at `tiles`, counters at `counters`)
int enqueue_degree(dg_batch* b, const dgbt::VariantInfo& v, int gc, int gf, const dgbt::Tile* tiles, int ntiles,
                   int* counters, cudaStream_t s) {
  if (int rc = cfail(cudaMemsetAsync(counters, 0, 2 * sizeof(int), s), "batch counter reset")) return rc;
  const int gcell = std::min(gc, std::max(1, ntiles)), gface = std::min(gf, std::max(1, ntiles));
  v.cell<<<gcell, v.threads, v.smem_cell, s>>>(b->tabs, b->d_probs, tiles, ntiles, counters);
  v.face<<<gface, v.threads, v.smem_face, s>>>(b->tabs, b->d_probs, tiles, ntiles, counters + 1);
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

// capture the graph: fork one branch per degree from s, join them back into s.  The branch streams and the
// events are returned in br / ev and destroyed by the caller after the capture has ended.
int capture(dg_batch* b, cudaStream_t s, std::vector<cudaStream_t>& br, std::vector<cudaEvent_t>& ev) {
  cudaEvent_t fork = nullptr;
  int rc = cfail(cudaEventCreateWithFlags(&fork, cudaEventDisableTiming), "fork event");
  if (!rc) ev.push_back(fork);
  if (!rc) rc = cfail(cudaEventRecord(fork, s), "fork");
  for (int N = dgbt::NMIN; !rc && N <= dgbt::NMAX; ++N) {
    if (!b->present[N]) continue;
    cudaStream_t st = nullptr;
    cudaEvent_t done = nullptr;
    rc = cfail(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking), "branch stream");
    if (!rc) br.push_back(st);
    if (!rc) rc = cfail(cudaEventCreateWithFlags(&done, cudaEventDisableTiming), "join event");
    if (!rc) ev.push_back(done);
    if (!rc) rc = cfail(cudaStreamWaitEvent(st, fork, 0), "branch wait");
    if (!rc)
      rc = enqueue_degree(b, dgbt::variant_info(N, b->variant[N]), b->grid_cell[N], b->grid_face[N],
                          b->d_tiles + b->tile_off[N], b->ntiles[N], b->d_counters + 2 * N, st);
    if (!rc) rc = cfail(cudaEventRecord(done, st), "branch done");
    if (!rc) rc = cfail(cudaStreamWaitEvent(s, done, 0), "join");
  }
  return rc;
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
  if (int rc = cfail(cudaGetDevice(&dev), "cudaGetDevice")) return rc;
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
#define X(NV, TB)                \
  dgi::build_tables(NV, NV, &t); \
  b->tabs.TB = dgi::make_tab<NV, double>(t);
    X(2, t2) X(3, t3) X(4, t4) X(5, t5) X(6, t6) X(7, t7) X(8, t8) X(9, t9)
#undef X
  }
  b->probs.resize(count);
  size_t tot = 0, max_tiles = 0;
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
    b->present[h->N] = true;
    tot += (size_t)h->ncell * h->N * h->N * h->N;
    max_tiles += (size_t)h->ncell;  // at least one cell per tile
  }
  int rc = cfail(cudaMalloc(&b->d_probs, count * sizeof(dgbt::Problem)), "cudaMalloc(batch descriptors)");
  if (!rc) rc = cfail(cudaMallocHost(&b->h_probs_pinned, count * sizeof(dgbt::Problem)), "cudaMallocHost(batch)");
  if (!rc) rc = cfail(cudaMalloc(&b->d_tiles, max_tiles * sizeof(dgbt::Tile)), "cudaMalloc(batch tiles)");
  if (!rc) rc = cfail(cudaMalloc(&b->d_counters, 2 * (dgbt::NMAX + 1) * sizeof(int)), "cudaMalloc(batch counters)");

  // autotune the thread layout of every degree: time each candidate on that degree's problems alone
  double* tz = nullptr;
  double* ty = nullptr;
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
    if (!b->present[N]) continue;
    float best_ms = 1e30f;
    for (int v = 0; v < dgbt::NVAR && !rc; ++v) {
      const dgbt::VariantInfo vi = dgbt::variant_info(N, v);
      int gc = 0, gf = 0;
      rc = prepare_variant(vi, &gc, &gf);
      std::vector<dgbt::Tile> t = make_tiles(b, N, vi.cpb);
      if (!rc)
        rc = cfail(cudaMemcpyAsync(b->d_tiles, t.data(), t.size() * sizeof(dgbt::Tile), cudaMemcpyHostToDevice, s),
                   "tile upload");
      float best = 1e30f;
      for (int rep = 0; rep < 4 && !rc; ++rep) {
        rc = cfail(cudaEventRecord(e0, s), "event");
        if (!rc) rc = enqueue_degree(b, vi, gc, gf, b->d_tiles, (int)t.size(), b->d_counters, s);
        if (!rc) rc = cfail(cudaEventRecord(e1, s), "event");
        if (!rc) rc = cfail(cudaEventSynchronize(e1), "tuning sync");
        float ms = 0;
        if (!rc) rc = cfail(cudaEventElapsedTime(&ms, e0, e1), "tuning time");
        if (rep > 0) best = std::min(best, ms);  // the first run warms up
      }
      b->tune_ms[N][v] = best;
      if (best < best_ms) {
        best_ms = best;
        b->variant[N] = v;
      }
    }
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(s);
  cudaFree(tz);
  cudaFree(ty);
  // the chosen variants' tiles, degree after degree
  if (!rc) {
    std::vector<dgbt::Tile> all;
    for (int N = dgbt::NMIN; N <= dgbt::NMAX && !rc; ++N) {
      if (!b->present[N]) continue;
      const dgbt::VariantInfo vi = dgbt::variant_info(N, b->variant[N]);
      rc = prepare_variant(vi, &b->grid_cell[N], &b->grid_face[N]);
      std::vector<dgbt::Tile> t = make_tiles(b, N, vi.cpb);
      b->tile_off[N] = (int)all.size();
      b->ntiles[N] = (int)t.size();
      all.insert(all.end(), t.begin(), t.end());
    }
    if (!rc)
      rc = cfail(cudaMemcpyAsync(b->d_tiles, all.data(), all.size() * sizeof(dgbt::Tile), cudaMemcpyHostToDevice, s),
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

int dg_batch_tuning(const dg_batch* b, int32_t k, int32_t* cells_per_cta, int32_t* lines_per_thread,
                    float* ms_candidates) {
  if (!b || k < 1 || k > 8) {
    set_error("dg_batch_tuning: bad arguments");
    return DG_ERR_INVALID_ARG;
  }
  const int N = k + 1;
  const dgbt::VariantInfo vi = dgbt::variant_info(N, b->variant[N]);
  if (cells_per_cta) *cells_per_cta = b->present[N] ? vi.cpb : 0;
  if (lines_per_thread) *lines_per_thread = b->present[N] ? vi.lpt : 0;
  if (ms_candidates)
    for (int v = 0; v < dgbt::NVAR; ++v) ms_candidates[v] = b->present[N] ? b->tune_ms[N][v] : 0.f;
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
    std::vector<cudaStream_t> br;
    std::vector<cudaEvent_t> ev;
    if (!rc) rc = capture(b, cap, br, ev);
    cudaGraph_t g = nullptr;
    cudaError_t ee = cudaStreamEndCapture(cap, &g);
    for (auto e : ev) cudaEventDestroy(e);
    for (auto st : br) cudaStreamDestroy(st);
    if (!rc) rc = cfail(ee, "end capture");
    if (!rc) rc = cfail(cudaGraphInstantiate(&b->exec, g, 0), "graph instantiate");
    b->graph = g;
    cudaStreamDestroy(cap);
    if (rc) return rc;
  }
  return cfail(cudaGraphLaunch(b->exec, s), "graph launch");
}

}  // extern "C"
