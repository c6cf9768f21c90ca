// Internal declarations of libtrs (not part of the C ABI).
//
// Block matrices live in an "ELL-7 + tail" layout:
//   * the first nc rows are cells of an nx*ny*nz grid; their couplings to the
//     six 7-point neighbours and to themselves sit in seven slots ordered by
//     ascending column (-z, -y, -x, self, +x, +y, +z), stored structure-of-
//     arrays: ell[(slot * bb + e) * nc + row], e = r*b + c of the b x b block.
//     Columns are implicit (row + kSlotOff[slot]); emask[row] bit s says
//     whether slot s is stored (the caller's pattern), so coalesced
//     row-parallel loads need no column indices.
//   * every other block (well columns of perforated cells, all blocks of the
//     well rows, everything for unstructured matrices) is in a block-CSR tail
//     over all rows: tptr[n_rows+1], tcol[ntail], tval[t * bb + e].
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <cstring>
#include <stdexcept>
#include <string>
#include <utility>
#include <vector>

#include "../../include/trs.h"

namespace trs {

constexpr int kMaxB = 5;
constexpr int kSlots = 7;
constexpr int kSelf = 3;
// Bit 7 of a cell's slot mask (emask) and of a position's lower mask
// (lmask): the row also has entries in the tail, so that rows without any
// (almost all cells) never read their tail pointers.
constexpr unsigned kTailBit = 0x80u;
// Block ILU(1) keeps the level-1 fill of a cell row that falls on one of the
// 18 cells two 7-point steps away in fill slots next to the 7 stencil slots:
// (dx, dy, dz) of fill slot s, ordered by (dz, dy, dx).
constexpr int kFill = 18;
constexpr int kFillD[kFill][3] = {{0, 0, -2}, {0, -1, -1}, {-1, 0, -1}, {1, 0, -1}, {0, 1, -1}, {0, -2, 0},
                                  {-1, -1, 0}, {1, -1, 0}, {-2, 0, 0}, {2, 0, 0}, {-1, 1, 0}, {1, 1, 0},
                                  {0, 2, 0}, {0, -1, 1}, {-1, 0, 1}, {1, 0, 1}, {0, 1, 1}, {0, 0, 2}};
constexpr int kMaxLevels = 16;
constexpr int kDenseMax = 4096;
constexpr int kMaxColours = 64;
constexpr int kMaxRestart = 64;

struct Error : std::runtime_error {
  trs_status code;
  Error(trs_status c, const std::string &m) : std::runtime_error(m), code(c) {}
};

#define TRS_CUDA(call)                                                                         \
  do {                                                                                         \
    cudaError_t e_ = (call);                                                                   \
    if (e_ != cudaSuccess)                                                                     \
      throw ::trs::Error(e_ == cudaErrorMemoryAllocation ? TRS_ERR_OOM : TRS_ERR_CUDA,         \
                         std::string(#call) + ": " + cudaGetErrorString(e_));                  \
  } while (0)
// Every kernel launch is followed by TRS_LAUNCHED(), which checks the launch
// and counts it (trs_kernel_launches()).
void note_launch();
#define TRS_LAUNCHED()                                                                         \
  do {                                                                                         \
    ::trs::note_launch();                                                                      \
    TRS_CUDA(cudaGetLastError());                                                              \
  } while (0)
#define TRS_REQUIRE(cond, code, msg)                                                           \
  do {                                                                                         \
    if (!(cond)) throw ::trs::Error((code), (msg));                                            \
  } while (0)

// Owning device buffer (move-only).
template <class T>
struct DBuf {
  T *p = nullptr;
  size_t n = 0;
  DBuf() = default;
  explicit DBuf(size_t count) { alloc(count); }
  DBuf(const DBuf &) = delete;
  DBuf &operator=(const DBuf &) = delete;
  DBuf(DBuf &&o) noexcept : p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf &operator=(DBuf &&o) noexcept {
    if (this != &o) { release(); p = o.p; n = o.n; o.p = nullptr; o.n = 0; }
    return *this;
  }
  ~DBuf() { release(); }
  void alloc(size_t count) {
    release();
    n = count;
    if (count) TRS_CUDA(cudaMalloc(reinterpret_cast<void **>(&p), count * sizeof(T)));
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
  void upload(const T *h, size_t count, cudaStream_t s) {
    if (count) TRS_CUDA(cudaMemcpyAsync(p, h, count * sizeof(T), cudaMemcpyHostToDevice, s));
  }
  void zero(cudaStream_t s) {
    if (n) TRS_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
  T *get() const { return p; }
};

// Stream-ordered temporary device buffer (cudaMallocAsync / cudaFreeAsync on
// the stream that uses it): no device-wide synchronisation on free.
template <class T>
struct TBuf {
  T *p = nullptr;
  size_t n = 0;
  cudaStream_t s = nullptr;
  TBuf(size_t count, cudaStream_t st) : n(count), s(st) {
    if (count) TRS_CUDA(cudaMallocAsync(reinterpret_cast<void **>(&p), count * sizeof(T), s));
  }
  TBuf(const TBuf &) = delete;
  TBuf &operator=(const TBuf &) = delete;
  ~TBuf() {
    if (p) cudaFreeAsync(p, s);
  }
  void zero() {
    if (n) TRS_CUDA(cudaMemsetAsync(p, 0, n * sizeof(T), s));
  }
};

// Keeps freed stream-ordered memory in the current device's pool.
void keep_pool_memory();

template <class T>
std::vector<T> download(const T *d, size_t count, cudaStream_t s) {
  std::vector<T> h(count);
  if (count) {
    TRS_CUDA(cudaMemcpyAsync(h.data(), d, count * sizeof(T), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaStreamSynchronize(s));
  }
  return h;
}

// Geometry of the structured part.
// Programmatic dependent launch (sm_90 and later): every kernel of the library
// is launched with programmatic stream serialisation, so that the next kernel
// in the stream is scheduled while this one drains instead of after it; each
// kernel waits (griddepcontrol.wait: the previous grid complete and its
// memory visible) before it touches memory, and lets its successor launch
// once all of its own blocks run.  Stream order is kept: nothing is read
// before the producer has finished.
template <class... KArgs, class... Args>
void launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s, Args &&...args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TRS_CUDA(cudaLaunchKernelEx(&cfg, kernel, static_cast<KArgs>(std::forward<Args>(args))...));
}

__device__ __forceinline__ void pdl_enter() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" :::);
}

// Relative-permeability tables of the thermal model, passed by value.
constexpr int kThermalTableMax = 32;
struct ThermalTables {
  int nswt, nslt;
  double swt[3 * kThermalTableMax];   // S_w, k_rw, k_row
  double slt[3 * kThermalTableMax];   // S_l, k_rg, k_rog
  // per segment i, the slopes (y_{i+1} - y_i) / (x_{i+1} - x_i) of columns 1, 2
  double swt_slope[2 * kThermalTableMax];
  double slt_slope[2 * kThermalTableMax];
};

struct Geom {
  int64_t nc;       // cells
  int64_t n_rows;   // cells + other rows
  int64_t off[kSlots];
  int64_t off2[kFill];   // index offsets of the fill slots
  int nx, ny, nz;
};

inline Geom make_geom(int nx, int ny, int nz, int64_t n_rows) {
  Geom g;
  g.nx = nx; g.ny = ny; g.nz = nz;
  g.nc = (int64_t)nx * ny * nz;
  g.n_rows = n_rows;
  const int64_t sxy = (int64_t)nx * ny;
  int64_t o[kSlots] = {-sxy, -(int64_t)nx, -1, 0, 1, nx, sxy};
  for (int s = 0; s < kSlots; s++) g.off[s] = o[s];
  for (int s = 0; s < kFill; s++) g.off2[s] = kFillD[s][0] + kFillD[s][1] * (int64_t)nx + kFillD[s][2] * sxy;
  return g;
}

// Device view of a block (or scalar, bb = 1) matrix in ELL-7 + tail form.
template <class T>
struct MatView {
  Geom g;
  const uint8_t *emask;   // [nc]
  const int64_t *tptr;    // [n_rows + 1]
  const int32_t *tcol;    // [ntail]
  const T *ell;           // [7][bb][nc] (the decoupled matrix Ã: [7][nc][bb], blocks contiguous)
  const T *tval;          // [ntail][bb]
};

}  // namespace trs

// The handles of the C ABI.
struct trs_bsr {
  int b = 0;
  int64_t n = 0, nnzb = 0, ntail = 0;
  trs::Geom g{};
  bool structured = false;
  trs::DBuf<uint8_t> emask;
  trs::DBuf<int64_t> tptr;
  trs::DBuf<int32_t> tcol;
  trs::DBuf<double> ell, tval;
  trs::DBuf<int64_t> tdiag;   // [n - nc] tail index of the diagonal block of each non-cell row
  // canonical BSR order: internal location of each block, row and column
  trs::DBuf<int64_t> map;
  trs::DBuf<int32_t> urow, ucol;
  std::vector<int64_t> h_rp;
  std::vector<int32_t> h_col;
  // for a matrix made by trs_bsr_transpose: canonical index in the source of
  // each canonical block (refresh with trs_bsr_transpose_values)
  trs::DBuf<int64_t> tsrc;
  trs::DBuf<int64_t> ttail;   // canonical index of each tail entry, in tail order
  // tail entries grouped by column (for the transposed product)
  trs::DBuf<int64_t> tc_ptr, tc_src;
  trs::DBuf<int32_t> tc_row;
  // synthetic assembly bookkeeping
  bool synthetic = false;
  int n_wells = 0;
  int64_t n_perf = 0;
  trs::DBuf<int64_t> cperf_ptr, cperf_idx, wperf_ptr, wperf_idx;   // perforations by cell / well
  trs::DBuf<int32_t> perf_cell, perf_well;
  trs::DBuf<int64_t> perf_cw, perf_wc, wdiag;                      // tail slots of (c,w), (w,c), (w,w)
  trs::DBuf<double> host_stage;   // device copy of host assembly inputs (trs_bsr_assemble_host)
  trs::DBuf<double> thermal_props;  // per-cell thermal properties with derivatives (trs_thermal_assemble)

  template <class T = double>
  trs::MatView<T> view() const {
    return trs::MatView<T>{g, emask.p, tptr.p, tcol.p, ell.p, tval.p};
  }
};
