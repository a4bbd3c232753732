// dg_matrix.cu -- the matrix-based comparison of Sec. 5.2 (table "Matrix-based" / "Matrix Assembly"):
// the operator's matrix in block compressed row storage (one (k+1)^3 x (k+1)^3 block per coupled cell
// pair), assembled with the operator's own kernels, and its matrix-vector product.
//
// Assembly probes the matrix-free operator.  Cells are coloured by (ix mod cx, iy mod cy, iz mod cz) so
// that two cells of one colour never share a face neighbour (cx = 3 per axis, or a divisor of n >= 3 on a
// periodic axis, or n itself for n <= 2).  For each colour and each local basis index j, the vector that is
// 1 at DOF j of every cell of the colour is applied; the result restricted to cell T, for T a cell of the
// colour or one of its face neighbours, is column j of the block A_{T,S}.  That is colours * (k+1)^3
// applications, each of the whole mesh.
//
// Blocks are stored column-major with the columns padded to an even length ld (entry (i, j) at j*ld + i):
// a probe writes one contiguous column, and in the product each thread owns two consecutive rows and
// reads each column of a block with one 16-byte load, so a block row's threads read every column as one
// contiguous segment.  Measured on GB300 at 70-74 % of the copy bandwidth; a row-major layout with a
// lane group per row (35-60 %), one row per thread (58-70 %) and four rows per thread (64-69 %) were
// slower.
#include <algorithm>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "dg_internal.h"

struct dg_matrix {
  int device = 0;
  int nb = 0;          // block size (k+1)^3
  int ld = 0;          // column stride of a block: nb rounded up to even
  int64_t nrows = 0;   // block rows = cells
  int64_t nnzb = 0;    // stored blocks
  int* rowptr = nullptr;   // device [nrows + 1]
  int* colidx = nullptr;   // device [nnzb]
  double* vals = nullptr;  // device [nnzb][nb][ld], column-major blocks with padded columns
  std::vector<int> h_rowptr, h_colidx;
  double assemble_seconds = 0.0;
  int probes = 0;
};

namespace {

using dgi::cuda_fail;
using dgi::set_error;

// for each listed cell S of the colour: set (value = 1) or clear (value = 0) DOF j of S
__global__ void probe_set(double* __restrict__ x, const int* __restrict__ cells, int ncells, int nb, int j,
                          double value) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < ncells; i += gridDim.x * blockDim.x)
    x[(size_t)cells[i] * nb + j] = value;
}

// column j of A_{T,S} for every listed S and every T coupled to S (the blocks of column S): y restricted to T
__global__ void probe_scatter(const double* __restrict__ y, const int* __restrict__ cells, int ncells,
                              const int* __restrict__ rowptr, const int* __restrict__ colidx,
                              const int* __restrict__ tslots, const int* __restrict__ tcells, int nb, int ld,
                              int j, double* __restrict__ vals) {
  // tcells[(c * 7 + q)]: the q-th distinct cell coupled to cells[c] (-1: none); tslots: its slot in T's row
  const int c = blockIdx.x;
  if (c >= ncells) return;
  for (int q = 0; q < 7; ++q) {
    const int T = tcells[c * 7 + q];
    if (T < 0) continue;
    const int slot = tslots[c * 7 + q];
    double* col = vals + ((size_t)slot * nb + j) * ld;
    const double* src = y + (size_t)T * nb;
    for (int i = threadIdx.x; i < nb; i += blockDim.x) col[i] = src[i];
  }
}

// y_T = sum_S A_{T,S} x_S.  Each thread owns rows 2t and 2t+1 of a block row (tpr = ceil(nb/2) threads per
// block row, rpc block rows per CTA, at most 256 threads).  The x blocks the CTA's rows need are staged in
// shared memory first; the matrix then streams through once with 16-byte loads, four in flight per thread.
__global__ void __launch_bounds__(256) bcsr_spmv(const int* __restrict__ rowptr, const int* __restrict__ colidx,
                                                 const double* __restrict__ vals, const double* __restrict__ x,
                                                 double* __restrict__ y, int64_t nrows, int nb, int ld, int rpc) {
  extern __shared__ double xs[];  // [rpc][7][nb]
  const int tpr = (nb + 1) / 2;
  const int r = threadIdx.x / tpr, t = threadIdx.x - r * tpr;
  const int64_t Tbase = (int64_t)blockIdx.x * rpc;
  for (int e = threadIdx.x; e < rpc * 7 * nb; e += blockDim.x) {
    const int rr = e / (7 * nb), rem = e - rr * 7 * nb, q = rem / nb, jj = rem - q * nb;
    const int64_t TT = Tbase + rr;
    double v = 0.0;
    if (TT < nrows) {
      const int b0 = rowptr[TT], b1 = rowptr[TT + 1];
      if (q < b1 - b0) v = x[(size_t)colidx[b0 + q] * nb + jj];
    }
    xs[e] = v;
  }
  __syncthreads();
  const int64_t T = Tbase + r;
  if (r >= rpc || T >= nrows) return;
  const int b0 = rowptr[T], b1 = rowptr[T + 1];
  const int ld2 = ld / 2;
  double2 acc0 = make_double2(0.0, 0.0), acc1 = acc0, acc2 = acc0, acc3 = acc0;
  for (int b = b0; b < b1; ++b) {
    const double2* A = reinterpret_cast<const double2*>(vals + (size_t)b * nb * ld) + t;
    const double* xb = xs + ((size_t)r * 7 + (b - b0)) * nb;
    int j = 0;
    for (; j + 3 < nb; j += 4) {
      const double2 a0 = __ldcs(A + (size_t)j * ld2), a1 = __ldcs(A + (size_t)(j + 1) * ld2);
      const double2 a2 = __ldcs(A + (size_t)(j + 2) * ld2), a3 = __ldcs(A + (size_t)(j + 3) * ld2);
      const double x0 = xb[j], x1 = xb[j + 1], x2 = xb[j + 2], x3 = xb[j + 3];
      acc0.x = fma(a0.x, x0, acc0.x);
      acc0.y = fma(a0.y, x0, acc0.y);
      acc1.x = fma(a1.x, x1, acc1.x);
      acc1.y = fma(a1.y, x1, acc1.y);
      acc2.x = fma(a2.x, x2, acc2.x);
      acc2.y = fma(a2.y, x2, acc2.y);
      acc3.x = fma(a3.x, x3, acc3.x);
      acc3.y = fma(a3.y, x3, acc3.y);
    }
    for (; j < nb; ++j) {
      const double2 a0 = __ldcs(A + (size_t)j * ld2);
      acc0.x = fma(a0.x, xb[j], acc0.x);
      acc0.y = fma(a0.y, xb[j], acc0.y);
    }
  }
  double* yT = y + (size_t)T * nb;
  yT[2 * t] = (acc0.x + acc1.x) + (acc2.x + acc3.x);
  if (2 * t + 1 < nb) yT[2 * t + 1] = (acc0.y + acc1.y) + (acc2.y + acc3.y);
}

int colours_along(int n, bool periodic) {
  if (!periodic || n % 3 == 0) return std::min(n, 3);
  if (n <= 2) return n;
  for (int d = 3; d <= n; ++d)
    if (n % d == 0) return d;
  return n;
}

void destroy(dg_matrix* m) {
  if (!m) return;
  cudaFree(m->rowptr);
  cudaFree(m->colidx);
  cudaFree(m->vals);
  delete m;
}

}  // namespace

extern "C" {

int dg_assemble(dg_handle* h, void* stream, dg_matrix** out) {
  if (!h || !out) {
    set_error("dg_assemble: null argument");
    return DG_ERR_INVALID_ARG;
  }
  *out = nullptr;
  const int N = h->N, nb = N * N * N;
  if (nb > 512) {
    set_error("dg_assemble: block size (k+1)^3 must be <= 512 (k <= 7)");
    return DG_ERR_INVALID_ARG;
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int64_t ncell = h->ncell;
  const int nx = h->n[0], ny = h->n[1], nz = h->n[2];
  auto cell_of = [&](int ix, int iy, int iz) { return ix + nx * (iy + ny * iz); };
  // coupled cells of each cell: itself and its face neighbours (periodic wrap, duplicates merged), sorted
  std::vector<std::vector<int>> nbrs(ncell);
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) {
        const int ic[3] = {ix, iy, iz};
        std::vector<int>& v = nbrs[cell_of(ix, iy, iz)];
        v.push_back(cell_of(ix, iy, iz));
        for (int dir = 0; dir < 3; ++dir)
          for (int sd = -1; sd <= 1; sd += 2) {
            int jc[3] = {ic[0], ic[1], ic[2]};
            jc[dir] += sd;
            if (jc[dir] < 0 || jc[dir] >= h->n[dir]) {
              if (!h->periodic[dir]) continue;
              jc[dir] = (jc[dir] + h->n[dir]) % h->n[dir];
            }
            v.push_back(cell_of(jc[0], jc[1], jc[2]));
          }
        std::sort(v.begin(), v.end());
        v.erase(std::unique(v.begin(), v.end()), v.end());
      }
  dg_matrix* m = new (std::nothrow) dg_matrix();
  if (!m) {
    set_error("dg_assemble: host allocation failed");
    return DG_ERR_OOM;
  }
  cudaGetDevice(&m->device);
  m->nb = nb;
  m->ld = nb + (nb & 1);
  m->nrows = ncell;
  m->h_rowptr.resize(ncell + 1);
  m->h_rowptr[0] = 0;
  for (int64_t t = 0; t < ncell; ++t) m->h_rowptr[t + 1] = m->h_rowptr[t] + (int)nbrs[t].size();
  m->nnzb = m->h_rowptr[ncell];
  m->h_colidx.reserve(m->nnzb);
  for (int64_t t = 0; t < ncell; ++t) m->h_colidx.insert(m->h_colidx.end(), nbrs[t].begin(), nbrs[t].end());
  // colour classes and, per cell S, its coupled cells T with the slot of block (T, S) in T's row (the
  // structure is symmetric, so the coupled cells of S are the block columns of row S)
  const int cx = colours_along(nx, h->periodic[0]), cy = colours_along(ny, h->periodic[1]),
            cz = colours_along(nz, h->periodic[2]);
  const int ncol = cx * cy * cz;
  std::vector<std::vector<int>> members(ncol);
  for (int iz = 0; iz < nz; ++iz)
    for (int iy = 0; iy < ny; ++iy)
      for (int ix = 0; ix < nx; ++ix) members[(ix % cx) + cx * ((iy % cy) + cy * (iz % cz))].push_back(cell_of(ix, iy, iz));
  auto slot_of = [&](int T, int S) {
    const int* b = m->h_colidx.data() + m->h_rowptr[T];
    const int* e = m->h_colidx.data() + m->h_rowptr[T + 1];
    return (int)(std::lower_bound(b, e, S) - m->h_colidx.data());
  };
  int rc = DG_OK;
  cudaError_t e = cudaSuccess;
  double *x = nullptr, *y = nullptr;
  int *d_cells = nullptr, *d_tc = nullptr, *d_ts = nullptr;
  const size_t ndof = (size_t)ncell * nb;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
#define DG_TRY(call, what)        \
  do {                            \
    e = (call);                   \
    if (e != cudaSuccess) {       \
      rc = cuda_fail(e, what);    \
      goto fail;                  \
    }                             \
  } while (0)
  {
    DG_TRY(cudaMalloc(&m->rowptr, (ncell + 1) * sizeof(int)), "dg_assemble: cudaMalloc(rowptr)");
    DG_TRY(cudaMalloc(&m->colidx, m->nnzb * sizeof(int)), "dg_assemble: cudaMalloc(colidx)");
    DG_TRY(cudaMalloc(&m->vals, (size_t)m->nnzb * nb * m->ld * sizeof(double)), "dg_assemble: cudaMalloc(values)");
    DG_TRY(cudaMemsetAsync(m->vals, 0, (size_t)m->nnzb * nb * m->ld * sizeof(double), s), "dg_assemble: clear values");
    DG_TRY(cudaMalloc(&x, ndof * sizeof(double)), "dg_assemble: cudaMalloc(probe)");
    DG_TRY(cudaMalloc(&y, ndof * sizeof(double)), "dg_assemble: cudaMalloc(response)");
    DG_TRY(cudaMemcpyAsync(m->rowptr, m->h_rowptr.data(), (ncell + 1) * sizeof(int), cudaMemcpyHostToDevice, s),
           "dg_assemble: copy rowptr");
    DG_TRY(cudaMemcpyAsync(m->colidx, m->h_colidx.data(), m->nnzb * sizeof(int), cudaMemcpyHostToDevice, s),
           "dg_assemble: copy colidx");
    DG_TRY(cudaMemsetAsync(x, 0, ndof * sizeof(double), s), "dg_assemble: clear probe");
    size_t maxmem = 0;
    for (auto& mm : members) maxmem = std::max(maxmem, mm.size());
    DG_TRY(cudaMalloc(&d_cells, maxmem * sizeof(int)), "dg_assemble: cudaMalloc(cells)");
    DG_TRY(cudaMalloc(&d_tc, maxmem * 7 * sizeof(int)), "dg_assemble: cudaMalloc(targets)");
    DG_TRY(cudaMalloc(&d_ts, maxmem * 7 * sizeof(int)), "dg_assemble: cudaMalloc(slots)");
    DG_TRY(cudaEventCreate(&ev0), "dg_assemble: event");
    DG_TRY(cudaEventCreate(&ev1), "dg_assemble: event");
    DG_TRY(cudaEventRecord(ev0, s), "dg_assemble: event");
    for (int col = 0; col < ncol; ++col) {
      const std::vector<int>& cs = members[col];
      if (cs.empty()) continue;
      std::vector<int> tc(cs.size() * 7, -1), ts(cs.size() * 7, -1);
      for (size_t c = 0; c < cs.size(); ++c) {
        const std::vector<int>& v = nbrs[cs[c]];
        for (size_t q = 0; q < v.size(); ++q) {
          tc[c * 7 + q] = v[q];
          ts[c * 7 + q] = slot_of(v[q], cs[c]);
        }
      }
      // synchronous copies: the host vectors are rebuilt for the next colour
      DG_TRY(cudaMemcpyAsync(d_cells, cs.data(), cs.size() * sizeof(int), cudaMemcpyHostToDevice, s), "copy cells");
      DG_TRY(cudaMemcpyAsync(d_tc, tc.data(), tc.size() * sizeof(int), cudaMemcpyHostToDevice, s), "copy targets");
      DG_TRY(cudaMemcpyAsync(d_ts, ts.data(), ts.size() * sizeof(int), cudaMemcpyHostToDevice, s), "copy slots");
      const int nc = (int)cs.size();
      const unsigned g1 = (unsigned)std::min(dgi::sm_count() * 8, (nc + 255) / 256);
      for (int j = 0; j < nb; ++j) {
        probe_set<<<g1, 256, 0, s>>>(x, d_cells, nc, nb, j, 1.0);
        rc = dgi::launch_apply_f64(h, x, y, 0, 3, s);
        if (rc != DG_OK) goto fail;
        probe_scatter<<<nc, 128, 0, s>>>(y, d_cells, nc, m->rowptr, m->colidx, d_ts, d_tc, nb, m->ld, j, m->vals);
        probe_set<<<g1, 256, 0, s>>>(x, d_cells, nc, nb, j, 0.0);
        ++m->probes;
      }
      DG_TRY(cudaGetLastError(), "dg_assemble: probe kernels");
      DG_TRY(cudaStreamSynchronize(s), "dg_assemble: synchronize");
    }
    DG_TRY(cudaEventRecord(ev1, s), "dg_assemble: event");
    DG_TRY(cudaEventSynchronize(ev1), "dg_assemble: synchronize");
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ev0, ev1);
    m->assemble_seconds = ms * 1e-3;
  }
#undef DG_TRY
  cudaFree(x);
  cudaFree(y);
  cudaFree(d_cells);
  cudaFree(d_tc);
  cudaFree(d_ts);
  cudaEventDestroy(ev0);
  cudaEventDestroy(ev1);
  *out = m;
  return DG_OK;
fail:
  cudaStreamSynchronize(s);
  cudaFree(x);
  cudaFree(y);
  cudaFree(d_cells);
  cudaFree(d_tc);
  cudaFree(d_ts);
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  destroy(m);
  return rc;
}

int dg_matrix_info(const dg_matrix* m, int64_t* nrows, int64_t* nnzb, int32_t* block, double* assemble_seconds) {
  if (!m) {
    set_error("dg_matrix_info: null matrix");
    return DG_ERR_INVALID_ARG;
  }
  if (nrows) *nrows = m->nrows;
  if (nnzb) *nnzb = m->nnzb;
  if (block) *block = m->nb;
  if (assemble_seconds) *assemble_seconds = m->assemble_seconds;
  return DG_OK;
}

int dg_matrix_export(const dg_matrix* m, int32_t* rowptr, int32_t* colidx, double* vals) {
  if (!m) {
    set_error("dg_matrix_export: null matrix");
    return DG_ERR_INVALID_ARG;
  }
  if (rowptr) std::memcpy(rowptr, m->h_rowptr.data(), (m->nrows + 1) * sizeof(int));
  if (colidx) std::memcpy(colidx, m->h_colidx.data(), m->nnzb * sizeof(int));
  if (vals) {
    const size_t per = (size_t)m->nb * m->ld;
    std::vector<double> tmp(per * m->nnzb);
    cudaError_t e = cudaMemcpy(tmp.data(), m->vals, tmp.size() * sizeof(double), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "dg_matrix_export: copy values");
    for (int64_t c = 0; c < m->nnzb * m->nb; ++c)  // drop the column padding
      std::memcpy(vals + c * m->nb, tmp.data() + c * m->ld, m->nb * sizeof(double));
  }
  return DG_OK;
}

int dg_spmv(const dg_matrix* m, const double* x, double* y, void* stream) {
  if (!m || !x || !y || x == y) {
    set_error("dg_spmv: null matrix or vector, or x == y");
    return DG_ERR_INVALID_ARG;
  }
  const int nb = m->nb, tpr = (nb + 1) / 2;
  // block rows per CTA: up to 256 threads, and the staged x blocks within the default 48 KB of shared memory
  const int rpc = std::max(1, std::min(256 / tpr, (48 * 1024) / (7 * nb * (int)sizeof(double))));
  const size_t smem = (size_t)rpc * 7 * nb * sizeof(double);
  const unsigned grid = (unsigned)((m->nrows + rpc - 1) / rpc);
  bcsr_spmv<<<grid, rpc * tpr, smem, static_cast<cudaStream_t>(stream)>>>(m->rowptr, m->colidx, m->vals, x, y,
                                                                            m->nrows, nb, m->ld, rpc);
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? DG_OK : cuda_fail(e, "dg_spmv launch");
}

int dg_matrix_destroy(dg_matrix* m) {
  destroy(m);
  return DG_OK;
}

}  // extern "C"
