// Host runtime for block matrices: validation of the caller's BSR, the
// conversion to the ELL-7 + tail layout, the synthetic-assembly bookkeeping
// and the matrix entry points of the C ABI.
#include <algorithm>
#include <numeric>

#include "trs_api_common.cuh"

namespace trs {

namespace {

// slot of column j in cell row i of an nx*ny*nz grid, or -1
int ell_slot(const Geom &g, int64_t i, int64_t j) {
  const int64_t x = i % g.nx, y = (i / g.nx) % g.ny, z = i / ((int64_t)g.nx * g.ny);
  const int64_t d = j - i;
  if (d == 0) return kSelf;
  if (d == -1 && x > 0) return 2;
  if (d == 1 && x + 1 < g.nx) return 4;
  if (d == -(int64_t)g.nx && y > 0) return 1;
  if (d == (int64_t)g.nx && y + 1 < g.ny) return 5;
  if (d == -(int64_t)g.nx * g.ny && z > 0) return 0;
  if (d == (int64_t)g.nx * g.ny && z + 1 < g.nz) return 6;
  return -1;
}

int64_t find_sorted(const std::vector<int32_t> &col, int64_t lo, int64_t hi, int64_t j) {
  auto b = col.begin() + lo, e = col.begin() + hi;
  auto it = std::lower_bound(b, e, (int32_t)j);
  return (it != e && *it == j) ? (int64_t)(it - col.begin()) : -1;
}

}  // namespace

void validate_pattern(int64_t n, int b, const int64_t *rp, const int32_t *col) {
  TRS_REQUIRE(n > 0, TRS_ERR_INVALID, "n_block_rows must be positive");
  TRS_REQUIRE(n < ((int64_t)1 << 31), TRS_ERR_UNSUPPORTED, "at most 2^31-1 block rows");
  TRS_REQUIRE(b >= 1 && b <= kMaxB, TRS_ERR_UNSUPPORTED, "block size must be 1..5");
  TRS_REQUIRE(rp && col, TRS_ERR_INVALID, "row_ptr and col_idx are required");
  TRS_REQUIRE(rp[0] == 0, TRS_ERR_INVALID, "row_ptr[0] must be 0");
  for (int64_t i = 0; i < n; i++) {
    TRS_REQUIRE(rp[i + 1] >= rp[i], TRS_ERR_INVALID, "row_ptr must be non-decreasing");
    bool diag = false;
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      TRS_REQUIRE(col[p] >= 0 && col[p] < n, TRS_ERR_INVALID, "column index out of range");
      if (p > rp[i]) TRS_REQUIRE(col[p] > col[p - 1], TRS_ERR_INVALID, "columns must be sorted and unique");
      diag |= col[p] == i;
    }
    TRS_REQUIRE(diag, TRS_ERR_INVALID, "every row must hold its diagonal block");
  }
  std::vector<int32_t> cv(col, col + rp[n]);
  for (int64_t i = 0; i < n; i++)
    for (int64_t p = rp[i]; p < rp[i + 1]; p++)
      TRS_REQUIRE(find_sorted(cv, rp[col[p]], rp[col[p] + 1], i) >= 0, TRS_ERR_INVALID,
                  "the block pattern must be structurally symmetric");
}

// Builds the device layout of a (validated) canonical pattern.
void build_layout(trs_bsr *A, int64_t n, int b, const int64_t *rp, const int32_t *col, const int32_t *grid,
                  cudaStream_t s) {
  A->b = b;
  A->n = n;
  A->nnzb = rp[n];
  A->h_rp.assign(rp, rp + n + 1);
  A->h_col.assign(col, col + rp[n]);
  if (grid) {
    TRS_REQUIRE(grid[0] > 0 && grid[1] > 0 && grid[2] > 0, TRS_ERR_INVALID, "grid dimensions must be positive");
    TRS_REQUIRE((int64_t)grid[0] * grid[1] * grid[2] <= n, TRS_ERR_INVALID, "grid has more cells than rows");
    A->g = make_geom(grid[0], grid[1], grid[2], n);
    A->structured = true;
  } else {
    A->g = make_geom(1, 1, 1, n);
    A->g.nc = 0;
    A->g.nx = A->g.ny = A->g.nz = 0;
    A->structured = false;
  }
  const Geom &g = A->g;
  const int64_t nc = g.nc, nnzb = A->nnzb;
  std::vector<uint8_t> emask(nc, 0);
  std::vector<int64_t> map(nnzb), tptr(n + 1, 0);
  std::vector<int32_t> urow(nnzb), ucol(nnzb);
  std::vector<int> slot(nnzb, -1);
  for (int64_t i = 0; i < n; i++)
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      urow[p] = (int32_t)i;
      ucol[p] = col[p];
      if (i < nc && col[p] < nc) slot[p] = ell_slot(g, i, col[p]);
      if (slot[p] < 0) tptr[i + 1]++;
    }
  for (int64_t i = 0; i < n; i++) tptr[i + 1] += tptr[i];
  const int64_t ntail = tptr[n];
  A->ntail = ntail;
  std::vector<int32_t> tcol(std::max<int64_t>(ntail, 1));
  std::vector<int64_t> tdiag(std::max<int64_t>(n - nc, 1), -1);
  for (int64_t i = 0; i < n; i++) {
    int64_t t = tptr[i];
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      if (slot[p] >= 0) {
        emask[i] |= (uint8_t)(1u << slot[p]);
        map[p] = (int64_t)slot[p] * nc + i;
      } else {
        tcol[t] = col[p];
        map[p] = (int64_t)kSlots * nc + t;
        if (col[p] == i && i >= nc) tdiag[i - nc] = t;
        t++;
      }
    }
  }
  for (int64_t i = 0; i < nc; i++)
    if (tptr[i + 1] > tptr[i]) emask[i] |= (uint8_t)kTailBit;
  // tail entries grouped by column, rows ascending
  std::vector<int64_t> tc_ptr(n + 1, 0), tc_src(std::max<int64_t>(ntail, 1));
  std::vector<int32_t> tc_row(std::max<int64_t>(ntail, 1));
  for (int64_t t = 0; t < ntail; t++) tc_ptr[tcol[t] + 1]++;
  for (int64_t i = 0; i < n; i++) tc_ptr[i + 1] += tc_ptr[i];
  std::vector<int64_t> fill(tc_ptr.begin(), tc_ptr.end() - 1);
  for (int64_t i = 0; i < n; i++)
    for (int64_t t = tptr[i]; t < tptr[i + 1]; t++) {
      const int64_t q = fill[tcol[t]]++;
      tc_src[q] = t;
      tc_row[q] = (int32_t)i;
    }
  const int bb = b * b;
  A->emask.alloc(std::max<int64_t>(nc, 1));
  A->emask.upload(emask.data(), nc, s);
  A->tptr.alloc(n + 1);
  A->tptr.upload(tptr.data(), n + 1, s);
  A->tcol.alloc(std::max<int64_t>(ntail, 1));
  A->tcol.upload(tcol.data(), ntail, s);
  A->tdiag.alloc(std::max<int64_t>(n - nc, 1));
  A->tdiag.upload(tdiag.data(), n - nc, s);
  A->map.alloc(std::max<int64_t>(nnzb, 1));
  A->map.upload(map.data(), nnzb, s);
  A->urow.alloc(std::max<int64_t>(nnzb, 1));
  A->urow.upload(urow.data(), nnzb, s);
  A->ucol.alloc(std::max<int64_t>(nnzb, 1));
  A->ucol.upload(ucol.data(), nnzb, s);
  A->tc_ptr.alloc(n + 1);
  A->tc_ptr.upload(tc_ptr.data(), n + 1, s);
  A->tc_src.alloc(std::max<int64_t>(ntail, 1));
  A->tc_src.upload(tc_src.data(), ntail, s);
  A->tc_row.alloc(std::max<int64_t>(ntail, 1));
  A->tc_row.upload(tc_row.data(), ntail, s);
  A->ell.alloc(std::max<int64_t>((int64_t)kSlots * bb * nc, 1));
  A->ell.zero(s);
  A->tval.alloc(std::max<int64_t>(ntail * bb, 1));
  A->tval.zero(s);
  TRS_CUDA(cudaStreamSynchronize(s));  // host staging vectors go out of scope
}

void upload_values(trs_bsr *A, const double *values, bool on_device, cudaStream_t s) {
  const int bb = A->b * A->b;
  const int64_t cnt = A->nnzb * bb;
  if (on_device) {
    launch_scatter_values(A->nnzb, bb, A->map.p, values, A->g.nc, A->ell.p, A->tval.p, s);
  } else {
    DBuf<double> stage(std::max<int64_t>(cnt, 1));
    TRS_CUDA(cudaMemcpyAsync(stage.p, values, cnt * sizeof(double), cudaMemcpyHostToDevice, s));
    launch_scatter_values(A->nnzb, bb, A->map.p, stage.p, A->g.nc, A->ell.p, A->tval.p, s);
    TRS_CUDA(cudaStreamSynchronize(s));
  }
}

}  // namespace trs

using namespace trs;

extern "C" {

trs_status trs_bsr_create(int64_t n, int32_t b, const int64_t *row_ptr, const int32_t *col_idx,
                          const double *values, const int32_t *grid_dims, void *stream, trs_bsr **out) {
  return guarded([&] {
    TRS_REQUIRE(out, TRS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    validate_pattern(n, b, row_ptr, col_idx);
    cudaStream_t s = (cudaStream_t)stream;
    auto A = std::make_unique<trs_bsr>();
    build_layout(A.get(), n, b, row_ptr, col_idx, grid_dims, s);
    if (values) upload_values(A.get(), values, false, s);
    *out = A.release();
  });
}

trs_status trs_bsr_create_synthetic(int32_t nx, int32_t ny, int32_t nz, int32_t b, int32_t n_wells,
                                    int64_t n_perf, const int32_t *perf_well, const int32_t *perf_cell,
                                    void *stream, trs_bsr **out) {
  return guarded([&] {
    TRS_REQUIRE(out, TRS_ERR_INVALID, "out is NULL");
    *out = nullptr;
    TRS_REQUIRE(nx > 0 && ny > 0 && nz > 0, TRS_ERR_INVALID, "grid dimensions must be positive");
    TRS_REQUIRE(n_wells >= 0 && n_perf >= 0, TRS_ERR_INVALID, "negative well or perforation count");
    TRS_REQUIRE(n_perf == 0 || (perf_well && perf_cell), TRS_ERR_INVALID, "perforation arrays are NULL");
    TRS_REQUIRE(b >= 1 && b <= kMaxB, TRS_ERR_UNSUPPORTED, "block size must be 1..5");
    const Geom g = make_geom(nx, ny, nz, (int64_t)nx * ny * nz + n_wells);
    const int64_t nc = g.nc, n = g.n_rows;
    // perforation lists by cell and by well, ascending perforation index
    std::vector<int64_t> cptr(nc + 1, 0), wptr(n_wells + 1, 0);
    for (int64_t m = 0; m < n_perf; m++) {
      TRS_REQUIRE(perf_cell[m] >= 0 && perf_cell[m] < nc, TRS_ERR_INVALID, "perforated cell out of range");
      TRS_REQUIRE(perf_well[m] >= 0 && perf_well[m] < n_wells, TRS_ERR_INVALID, "well index out of range");
      cptr[perf_cell[m] + 1]++;
      wptr[perf_well[m] + 1]++;
    }
    for (int64_t c = 0; c < nc; c++) cptr[c + 1] += cptr[c];
    for (int w = 0; w < n_wells; w++) wptr[w + 1] += wptr[w];
    std::vector<int64_t> cidx(std::max<int64_t>(n_perf, 1)), widx(std::max<int64_t>(n_perf, 1));
    {
      std::vector<int64_t> fc(cptr.begin(), cptr.end() - 1), fw(wptr.begin(), wptr.end() - 1);
      for (int64_t m = 0; m < n_perf; m++) {
        cidx[fc[perf_cell[m]]++] = m;
        widx[fw[perf_well[m]]++] = m;
      }
    }
    // canonical pattern: cell rows (7-point neighbours, self, wells), well rows
    std::vector<int64_t> rp(n + 1, 0);
    std::vector<int32_t> col;
    col.reserve(7 * nc + 2 * n_perf + n_wells);
    std::vector<int32_t> tmp;
    for (int64_t c = 0; c < nc; c++) {
      for (int s = 0; s < kSlots; s++)
        if (s == kSelf || ell_slot(g, c, c + g.off[s]) == s) col.push_back((int32_t)(c + g.off[s]));
      tmp.clear();
      for (int64_t t = cptr[c]; t < cptr[c + 1]; t++) tmp.push_back((int32_t)(nc + perf_well[cidx[t]]));
      std::sort(tmp.begin(), tmp.end());
      TRS_REQUIRE(std::adjacent_find(tmp.begin(), tmp.end()) == tmp.end(), TRS_ERR_INVALID,
                  "a well perforates a cell twice");
      col.insert(col.end(), tmp.begin(), tmp.end());
      rp[c + 1] = (int64_t)col.size();
    }
    for (int w = 0; w < n_wells; w++) {
      tmp.clear();
      for (int64_t t = wptr[w]; t < wptr[w + 1]; t++) tmp.push_back(perf_cell[widx[t]]);
      tmp.push_back((int32_t)(nc + w));
      std::sort(tmp.begin(), tmp.end());
      col.insert(col.end(), tmp.begin(), tmp.end());
      rp[nc + w + 1] = (int64_t)col.size();
    }
    cudaStream_t s = (cudaStream_t)stream;
    auto A = std::make_unique<trs_bsr>();
    const int32_t grid[3] = {nx, ny, nz};
    build_layout(A.get(), n, b, rp.data(), col.data(), grid, s);
    // tail slots of (c, w), (w, c) and (w, w)
    std::vector<int64_t> tptr = download(A->tptr.p, n + 1, s);
    std::vector<int32_t> tcol = download(A->tcol.p, std::max<int64_t>(A->ntail, 1), s);
    std::vector<int64_t> pcw(std::max<int64_t>(n_perf, 1)), pwc(std::max<int64_t>(n_perf, 1));
    std::vector<int64_t> wdiag(std::max(n_wells, 1));
    for (int64_t m = 0; m < n_perf; m++) {
      const int64_t c = perf_cell[m], w = nc + perf_well[m];
      pcw[m] = find_sorted(tcol, tptr[c], tptr[c + 1], w);
      pwc[m] = find_sorted(tcol, tptr[w], tptr[w + 1], c);
    }
    for (int w = 0; w < n_wells; w++) wdiag[w] = find_sorted(tcol, tptr[nc + w], tptr[nc + w + 1], nc + w);
    A->synthetic = true;
    A->n_wells = n_wells;
    A->n_perf = n_perf;
    A->cperf_ptr.alloc(nc + 1);
    A->cperf_ptr.upload(cptr.data(), nc + 1, s);
    A->cperf_idx.alloc(cidx.size());
    A->cperf_idx.upload(cidx.data(), n_perf, s);
    A->wperf_ptr.alloc(n_wells + 1);
    A->wperf_ptr.upload(wptr.data(), n_wells + 1, s);
    A->wperf_idx.alloc(widx.size());
    A->wperf_idx.upload(widx.data(), n_perf, s);
    A->perf_cw.alloc(pcw.size());
    A->perf_cw.upload(pcw.data(), n_perf, s);
    A->perf_wc.alloc(pwc.size());
    A->perf_wc.upload(pwc.data(), n_perf, s);
    A->wdiag.alloc(wdiag.size());
    A->wdiag.upload(wdiag.data(), n_wells, s);
    A->perf_cell.alloc(std::max<int64_t>(n_perf, 1));
    A->perf_well.alloc(std::max<int64_t>(n_perf, 1));
    if (n_perf) {
      A->perf_cell.upload(perf_cell, n_perf, s);
      A->perf_well.upload(perf_well, n_perf, s);
    }
    TRS_CUDA(cudaStreamSynchronize(s));
    *out = A.release();
  });
}

trs_status trs_bsr_assemble(trs_bsr *A, const double *perm, int32_t perm_is_log, double kvkh, double c_t,
                            const double *M, const double *acc, const double *wi, const double *lam,
                            void *stream) {
  return guarded([&] {
    TRS_REQUIRE(A && A->synthetic, TRS_ERR_INVALID, "matrix was not made by trs_bsr_create_synthetic");
    TRS_REQUIRE(perm && M && acc, TRS_ERR_INVALID, "NULL input array");
    TRS_REQUIRE(A->n_perf == 0 || (wi && lam), TRS_ERR_INVALID, "NULL perforation array");
    launch_assemble(A->b, A, perm, perm_is_log, kvkh, c_t, M, acc, wi, lam, (cudaStream_t)stream);
  });
}

trs_status trs_bsr_assemble_host(trs_bsr *A, const double *perm, int32_t perm_is_log, double kvkh, double c_t,
                                 const double *M, const double *acc, const double *wi, const double *lam,
                                 void *stream) {
  return guarded([&] {
    TRS_REQUIRE(A && A->synthetic, TRS_ERR_INVALID, "matrix was not made by trs_bsr_create_synthetic");
    TRS_REQUIRE(perm && M && acc, TRS_ERR_INVALID, "NULL input array");
    TRS_REQUIRE(A->n_perf == 0 || (wi && lam), TRS_ERR_INVALID, "NULL perforation array");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t nc = A->g.nc, bb = (int64_t)A->b * A->b, np = A->n_perf;
    // one staging area, each input at a 256-byte aligned offset
    auto up = [](int64_t c) { return (c + 31) / 32 * 32; };
    const int64_t o_perm = 0, o_M = up(nc), o_acc = o_M + up(6 * bb * nc), o_wi = o_acc + up(bb * nc),
                  o_lam = o_wi + up(np), total = o_lam + up(np * A->b);
    if ((int64_t)A->host_stage.n < total) A->host_stage.alloc(total);
    double *d = A->host_stage.p;
    auto copy = [&](int64_t at, const double *h, int64_t cnt) {
      if (cnt) TRS_CUDA(cudaMemcpyAsync(d + at, h, cnt * sizeof(double), cudaMemcpyHostToDevice, s));
    };
    copy(o_perm, perm, nc);
    copy(o_M, M, 6 * bb * nc);
    copy(o_acc, acc, bb * nc);
    if (np) {
      copy(o_wi, wi, np);
      copy(o_lam, lam, np * A->b);
    }
    launch_assemble(A->b, A, d + o_perm, perm_is_log, kvkh, c_t, d + o_M, d + o_acc, np ? d + o_wi : nullptr,
                    np ? d + o_lam : nullptr, s);
  });
}

trs_status trs_bsr_update_values(trs_bsr *A, const double *values, int32_t on_device, void *stream) {
  return guarded([&] {
    TRS_REQUIRE(A && values, TRS_ERR_INVALID, "NULL argument");
    upload_values(A, values, on_device != 0, (cudaStream_t)stream);
  });
}

trs_status trs_bsr_get_values(const trs_bsr *A, double *values, int32_t on_device, void *stream) {
  return guarded([&] {
    TRS_REQUIRE(A && values, TRS_ERR_INVALID, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const int bb = A->b * A->b;
    const int64_t cnt = A->nnzb * bb;
    if (on_device) {
      launch_gather_values(A->nnzb, bb, A->map.p, A->ell.p, A->tval.p, A->g.nc, values, s);
    } else {
      DBuf<double> stage(std::max<int64_t>(cnt, 1));
      launch_gather_values(A->nnzb, bb, A->map.p, A->ell.p, A->tval.p, A->g.nc, stage.p, s);
      TRS_CUDA(cudaMemcpyAsync(values, stage.p, cnt * sizeof(double), cudaMemcpyDeviceToHost, s));
      TRS_CUDA(cudaStreamSynchronize(s));
    }
  });
}

trs_status trs_bsr_scale_diagonal(trs_bsr *A, const double *sc, void *stream) {
  return guarded([&] {
    TRS_REQUIRE(A && sc, TRS_ERR_INVALID, "NULL argument");
    launch_scale_diagonal(A->b, A, sc, (cudaStream_t)stream);
  });
}

trs_status trs_bsr_pattern(const trs_bsr *A, int64_t *row_ptr, int32_t *col_idx) {
  return guarded([&] {
    TRS_REQUIRE(A && row_ptr && col_idx, TRS_ERR_INVALID, "NULL argument");
    std::copy(A->h_rp.begin(), A->h_rp.end(), row_ptr);
    std::copy(A->h_col.begin(), A->h_col.end(), col_idx);
  });
}

trs_status trs_bsr_get_info(const trs_bsr *A, trs_bsr_info *info) {
  return guarded([&] {
    TRS_REQUIRE(A && info, TRS_ERR_INVALID, "NULL argument");
    info->n_block_rows = A->n;
    info->b = A->b;
    info->nnzb = A->nnzb;
    info->n_cells = A->g.nc;
    info->grid[0] = A->g.nx;
    info->grid[1] = A->g.ny;
    info->grid[2] = A->g.nz;
  });
}

trs_status trs_bsr_spmv(const trs_bsr *A, double alpha, const double *x, double beta, double *y,
                        int32_t transpose, void *stream) {
  return guarded([&] {
    TRS_REQUIRE(A && x && y, TRS_ERR_INVALID, "NULL argument");
    TRS_REQUIRE(x != y, TRS_ERR_INVALID, "x and y must not alias");
    require_aligned(x, "x");
    require_aligned(y, "y");
    if (transpose) launch_spmv_t(A->b, *A, x, y, alpha, beta, (cudaStream_t)stream);
    else launch_spmv<double, double>(A->b, A->view(), x, y, alpha, beta, (cudaStream_t)stream);
  });
}

trs_status trs_bsr_transpose(const trs_bsr *A, void *stream, trs_bsr **out) {
  return guarded([&] {
    TRS_REQUIRE(A && out, TRS_ERR_INVALID, "NULL argument");
    *out = nullptr;
    const int64_t n = A->n, nnzb = A->nnzb;
    std::vector<int64_t> rp(n + 1, 0), src(std::max<int64_t>(nnzb, 1));
    std::vector<int32_t> col(std::max<int64_t>(nnzb, 1));
    for (int64_t p = 0; p < nnzb; p++) rp[A->h_col[p] + 1]++;
    for (int64_t i = 0; i < n; i++) rp[i + 1] += rp[i];
    std::vector<int64_t> fill(rp.begin(), rp.end() - 1);
    for (int64_t i = 0; i < n; i++)
      for (int64_t p = A->h_rp[i]; p < A->h_rp[i + 1]; p++) {
        const int64_t q = fill[A->h_col[p]]++;
        col[q] = (int32_t)i;
        src[q] = p;
      }
    cudaStream_t s = (cudaStream_t)stream;
    auto T = std::make_unique<trs_bsr>();
    const int32_t grid[3] = {A->g.nx, A->g.ny, A->g.nz};
    build_layout(T.get(), n, A->b, rp.data(), col.data(), A->structured ? grid : nullptr, s);
    T->tsrc.alloc(src.size());
    T->tsrc.upload(src.data(), nnzb, s);
    // the tail entries of T in tail order (build_layout fills the tail in
    // canonical order with the blocks that have no geometric slot)
    std::vector<int64_t> tq;
    tq.reserve(std::max<int64_t>(T->ntail, 1));
    const int64_t tnc = T->g.nc;
    for (int64_t i = 0; i < n; i++)
      for (int64_t q = rp[i]; q < rp[i + 1]; q++)
        if (!(i < tnc && col[q] < tnc && ell_slot(T->g, i, col[q]) >= 0)) tq.push_back(q);
    TRS_REQUIRE((int64_t)tq.size() == T->ntail, TRS_ERR_INVALID, "tail count of the transpose");
    T->ttail.alloc(std::max<int64_t>(T->ntail, 1));
    T->ttail.upload(tq.data(), T->ntail, s);
    launch_transpose_values(*A, *T, s);
    TRS_CUDA(cudaStreamSynchronize(s));
    *out = T.release();
  });
}

trs_status trs_bsr_transpose_values(const trs_bsr *A, trs_bsr *AT, void *stream) {
  return guarded([&] {
    TRS_REQUIRE(A && AT, TRS_ERR_INVALID, "NULL argument");
    TRS_REQUIRE(AT->tsrc.p && AT->ttail.p && AT->n == A->n && AT->b == A->b && AT->nnzb == A->nnzb &&
                    AT->g.nc == A->g.nc && AT->g.nx == A->g.nx && AT->g.ny == A->g.ny,
                TRS_ERR_INVALID, "AT was not made by trs_bsr_transpose of a matrix with A's pattern");
    launch_transpose_values(*A, *AT, (cudaStream_t)stream);
  });
}

void trs_bsr_destroy(trs_bsr *A) { delete A; }

}  // extern "C"
