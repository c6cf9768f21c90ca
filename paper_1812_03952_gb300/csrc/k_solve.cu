// Solve-phase kernels: block SpMV, multicolour ILU(0) sweeps, CPR residuals,
// AMG V-cycle pieces and the FGMRES / CGS2 reductions.
//
// All reductions are deterministic: a fixed grid, warp shuffles in a fixed
// pattern, per-block partial sums, and the last block to finish summing the
// partials in block order.
#include <atomic>
#include <mutex>

#include "trs_api_common.cuh"

namespace trs {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kRedStride = kMaxRestart + 16;  // room for the last 16-wide chunk

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Warp sums of KM per-lane values by reduce-scatter: at each of the first
// log2(KM) levels a lane keeps one half of its values, adds the partner's
// copy of that half and hands over the other half, then the last 5 -
// log2(KM) levels add one value.  KM - 1 + 5 - log2(KM) FP64 additions per
// lane instead of 5 KM (on GB300 the additions of a shuffle reduction share
// the FP64 pipe with the dot products themselves).  Returns the warp total of
// value v(lane) = (lane >> (5 - log2 KM)) & (KM - 1); the lanes with
// lane % (32 / KM) == 0 hold the KM totals once each.
template <int KM>
__device__ __forceinline__ double warp_reduce_scatter(double (&a)[KM], int lane) {
  static_assert(KM >= 1 && KM <= 32 && (KM & (KM - 1)) == 0, "KM must be a power of two up to 32");
  int o = 16;
#pragma unroll
  for (int h = KM / 2; h >= 1; h /= 2) {
    const bool upper = (lane & o) != 0;
#pragma unroll
    for (int i = 0; i < h; i++) {
      const double keep = upper ? a[i + h] : a[i];
      const double send = upper ? a[i] : a[i + h];
      a[i] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
    o >>= 1;
  }
  double v = a[0];
#pragma unroll
  for (; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <class T>
__device__ __forceinline__ double to_d(T v) { return static_cast<double>(v); }



// b consecutive entries of a block vector (16-byte aligned for b = 2, 4:
// the base pointers come from cudaMalloc-class allocations and block starts
// are multiples of b entries), with 128-bit accesses where they fit.
template <int B, class T>
__device__ __forceinline__ void load_blk(const T *p, T (&v)[B]) {
  if constexpr (B == 4 && sizeof(T) == 4) {
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
  } else if constexpr (B == 4 && sizeof(T) == 8) {
    const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  } else if constexpr (B == 2 && sizeof(T) == 8) {
    const double2 a = *reinterpret_cast<const double2 *>(p);
    v[0] = a.x; v[1] = a.y;
  } else {
#pragma unroll
    for (int c = 0; c < B; c++) v[c] = p[c];
  }
}

template <int B, class T>
__device__ __forceinline__ void store_blk(T *p, const T (&v)[B]) {
  if constexpr (B == 4 && sizeof(T) == 4) {
    *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
  } else if constexpr (B == 4 && sizeof(T) == 8) {
    reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
    reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
  } else {
#pragma unroll
    for (int c = 0; c < B; c++) p[c] = v[c];
  }
}

// One b x b block stored contiguously (the per-slot layout [7][rows][bb] of
// the decoupled matrix and of the ILU factors), with 128-bit loads where the
// block size allows (block starts are multiples of bb elements from a
// cudaMalloc base, so 16-byte aligned when bb * sizeof(T) is).
template <int B, class T>
__device__ __forceinline__ void load_block(const T *__restrict__ p, T (&v)[B * B]) {
  constexpr int BB = B * B;
  if constexpr (sizeof(T) == 4 && BB % 4 == 0) {
#pragma unroll
    for (int k = 0; k < BB / 4; k++) {
      const float4 t = reinterpret_cast<const float4 *>(p)[k];
      v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
    }
  } else if constexpr (sizeof(T) == 8 && BB % 2 == 0) {
#pragma unroll
    for (int k = 0; k < BB / 2; k++) {
      const double2 t = reinterpret_cast<const double2 *>(p)[k];
      v[2 * k] = t.x; v[2 * k + 1] = t.y;
    }
  } else {
#pragma unroll
    for (int e = 0; e < BB; e++) v[e] = p[e];
  }
}

// y2_j = y1_j + Pi_p e0_j (y1 = NULL: zero)
template <int B, class T>
__device__ __forceinline__ void load_y2(const T *__restrict__ y1, const T *__restrict__ e0, int64_t j, T (&v)[B]) {
  if (y1) {
    load_blk<B>(y1 + j * B, v);
  } else {
#pragma unroll
    for (int c = 0; c < B; c++) v[c] = T(0);
  }
  v[0] = v[0] + e0[j];
}

// ------------------------------------------------------------ block SpMV
template <int B, class TA, class TX>
__device__ __forceinline__ void cell_row_apply(const MatView<TA> &A, int64_t i, const TX *__restrict__ x,
                                               double (&acc)[B]) {
  constexpr int BB = B * B;
  const int64_t nc = A.g.nc;
  const unsigned m = A.emask[i];
#pragma unroll
  for (int s = 0; s < kSlots; s++) {
    if (!((m >> s) & 1u)) continue;
    const int64_t j = i + A.g.off[s];
    TX xv[B];
    load_blk<B>(x + j * B, xv);
    double xj[B];
#pragma unroll
    for (int c = 0; c < B; c++) xj[c] = to_d(xv[c]);
    const TA *blk = A.ell + (int64_t)s * BB * nc + i;
#pragma unroll
    for (int r = 0; r < B; r++)
#pragma unroll
      for (int c = 0; c < B; c++) acc[r] = fma(to_d(blk[(int64_t)(r * B + c) * nc]), xj[c], acc[r]);
  }
  if (!(m & kTailBit)) return;
  for (int64_t t = A.tptr[i]; t < A.tptr[i + 1]; t++) {
    const int64_t j = A.tcol[t];
    const TA *blk = A.tval + t * BB;
#pragma unroll
    for (int r = 0; r < B; r++)
#pragma unroll
      for (int c = 0; c < B; c++) acc[r] = fma(to_d(blk[r * B + c]), to_d(x[j * B + c]), acc[r]);
  }
}

// one warp, one long row (all entries in the tail); result valid on every lane
template <int B, class TA, class TX>
__device__ __forceinline__ void long_row_apply(const MatView<TA> &A, int64_t i, const TX *__restrict__ x,
                                               double (&acc)[B], int lane) {
  constexpr int BB = B * B;
  for (int64_t t = A.tptr[i] + lane; t < A.tptr[i + 1]; t += 32) {
    const int64_t j = A.tcol[t];
    const TA *blk = A.tval + t * BB;
#pragma unroll
    for (int r = 0; r < B; r++)
#pragma unroll
      for (int c = 0; c < B; c++) acc[r] = fma(to_d(blk[r * B + c]), to_d(x[j * B + c]), acc[r]);
  }
#pragma unroll
  for (int r = 0; r < B; r++) acc[r] = warp_sum(acc[r]);
}

template <int B, class TA, class TX>
__global__ void __launch_bounds__(kThreads) k_spmv(MatView<TA> A, const TX *__restrict__ x,
                                                   double *__restrict__ y, double alpha, double beta,
                                                   int64_t cell_blocks) {
  pdl_enter();
  if (blockIdx.x < cell_blocks) {
    const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (i >= A.g.nc) return;
    double acc[B] = {};
    cell_row_apply<B>(A, i, x, acc);
    if (alpha == 1.0 && beta == 0.0) {   // y = A x: no scaling on the FP64 unit (1.0 * v is v exactly)
      store_blk<B>(y + i * B, acc);
      return;
    }
#pragma unroll
    for (int r = 0; r < B; r++)
      y[i * B + r] = (beta == 0.0) ? alpha * acc[r] : fma(alpha, acc[r], beta * y[i * B + r]);
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t i = A.g.nc + (blockIdx.x - cell_blocks) * (int64_t)kWarps + (threadIdx.x >> 5);
    if (i >= A.g.n_rows) return;
    double acc[B] = {};
    long_row_apply<B>(A, i, x, acc, lane);
    if (lane == 0)
#pragma unroll
      for (int r = 0; r < B; r++)
        y[i * B + r] = (beta == 0.0) ? alpha * acc[r] : fma(alpha, acc[r], beta * y[i * B + r]);
  }
}

inline int64_t cell_blocks_of(int64_t nc) { return (nc + kThreads - 1) / kThreads; }
inline int64_t long_blocks_of(int64_t nl) { return (nl + kWarps - 1) / kWarps; }

// Sum of B values over a block (warp butterflies, then the warps in index
// order: a fixed order); the result is valid in thread 0.
template <int B>
__device__ __forceinline__ void block_sum(double (&acc)[B]) {
  __shared__ double part[kWarps][B];
#pragma unroll
  for (int r = 0; r < B; r++) acc[r] = warp_sum(acc[r]);
  if ((threadIdx.x & 31) == 0)
#pragma unroll
    for (int r = 0; r < B; r++) part[threadIdx.x >> 5][r] = acc[r];
  __syncthreads();
  if (threadIdx.x == 0)
#pragma unroll
    for (int r = 0; r < B; r++) {
      double t = part[0][r];
      for (int w = 1; w < kWarps; w++) t = t + part[w][r];
      acc[r] = t;
    }
}

// ----------------------------------------------------- reduction helpers
template <int KC>
__device__ void block_partial(double (&acc)[KC], double *__restrict__ dst) {
  __shared__ double sm[kWarps][KC];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kSpan = 32 / KC;
  const double v = warp_reduce_scatter<KC>(acc, lane);
  if ((lane & (kSpan - 1)) == 0) sm[warp][lane / kSpan] = v;
  __syncthreads();
  if (threadIdx.x < KC) {
    double s = 0.0;
    for (int w = 0; w < kWarps; w++) s += sm[w][threadIdx.x];
    dst[threadIdx.x] = s;
  }
  __syncthreads();
}

// Called by every block after its partials are stored.  The last block sums
// the partials of all blocks in block order into out[0..K-1]; if sqrt_out,
// out[K] also receives sqrt(out[K-1]).
__device__ void last_block_finish(const double *partial, unsigned int *counter, int K, double *out,
                                  int sqrt_out) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  __shared__ double sm[kWarps];
  for (int k = 0; k < K; k++) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) s += __ldcg(partial + (int64_t)b * kRedStride + k);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
      double t = 0.0;
      for (int w = 0; w < kWarps; w++) t += sm[w];
      out[k] = t;
      if (sqrt_out && k == K - 1) out[K] = sqrt(t);
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) *counter = 0u;
}

// r = rhs - A x and ||r||^2 (out[0]), sqrt in out[1]
template <int B>
__global__ void __launch_bounds__(kThreads) k_true_residual(MatView<double> A, const double *__restrict__ x,
                                                            const double *__restrict__ rhs,
                                                            double *__restrict__ r, int64_t cell_blocks,
                                                            int64_t rows_per_block_long, double *partial,
                                                            unsigned int *counter, double *out) {
  pdl_enter();
  // grid-stride over cell rows and long rows so that the grid stays fixed
  double acc2[1] = {0.0};
  const int64_t nc = A.g.nc, nl = A.g.n_rows - nc;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < nc; i += (int64_t)gridDim.x * kThreads) {
    double acc[B] = {};
    cell_row_apply<B>(A, i, x, acc);
#pragma unroll
    for (int rr = 0; rr < B; rr++) {
      const double v = rhs[i * B + rr] - acc[rr];
      r[i * B + rr] = v;
      acc2[0] = fma(v, v, acc2[0]);
    }
  }
  const int lane = threadIdx.x & 31;
  for (int64_t w = blockIdx.x * (int64_t)kWarps + (threadIdx.x >> 5); w < nl; w += (int64_t)gridDim.x * kWarps) {
    const int64_t i = nc + w;
    double acc[B] = {};
    long_row_apply<B>(A, i, x, acc, lane);
    if (lane == 0)
#pragma unroll
      for (int rr = 0; rr < B; rr++) {
        const double v = rhs[i * B + rr] - acc[rr];
        r[i * B + rr] = v;
        acc2[0] = fma(v, v, acc2[0]);
      }
  }
  (void)cell_blocks; (void)rows_per_block_long;
  block_partial<1>(acc2, partial + (int64_t)blockIdx.x * kRedStride);
  last_block_finish(partial, counter, 1, out, 1);
}

__global__ void __launch_bounds__(kThreads) k_norm2(const double *__restrict__ x, int64_t n, double *partial,
                                                    unsigned int *counter, double *out) {
  pdl_enter();
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    acc[0] = fma(x[i], x[i], acc[0]);
  block_partial<1>(acc, partial + (int64_t)blockIdx.x * kRedStride);
  last_block_finish(partial, counter, 1, out, 1);
}

// ----------------------------------------------------------- D^-1 scale
// f = D^-1 (w / *div) (and vout = w / *div); rows of colour 0, which have no
// earlier-ordered neighbour, also get y0 = f: the first forward ILU(0) sweep
// of f, done here (seed.colour == nullptr: no seeding).
template <class T>
struct Seed {
  const int32_t *colour;
  T *y0;
};

template <int B, class T>
__device__ __forceinline__ void seed_row(const Seed<T> &sd, int64_t i, const T *row) {
  if (sd.colour && sd.colour[i] == 0) {
#pragma unroll
    for (int c = 0; c < B; c++) sd.y0[i * B + c] = row[c];
  }
}

template <int B, class T>
__global__ void __launch_bounds__(kThreads) k_dscale(int64_t n, const double *__restrict__ w,
                                                     const double *__restrict__ div, double *__restrict__ vout,
                                                     const T *__restrict__ dinv, T *__restrict__ f, Seed<T> sd) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  double v[B];
  load_blk<B>(w + i * B, v);
  if (div) {
    const double rd = 1.0 / *div;
#pragma unroll
    for (int c = 0; c < B; c++) v[c] = v[c] * rd;
  }
  if (vout) store_blk<B>(vout + i * B, v);
  T fr[B];
#pragma unroll
  for (int r = 0; r < B; r++) {
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < B; c++) acc = fma(dinv[(int64_t)(r * B + c) * n + i], static_cast<T>(v[c]), acc);
    f[i * B + r] = acc;
    fr[r] = acc;
  }
  seed_row<B>(sd, i, fr);
}

// ------------------------------------------------------------ ILU sweeps
// The cell rows of a colour are swept by B lanes per block row: lane r of a
// group computes row r of every block-vector product (t_r -= sum_c F_rc
// y_j,c), so that a group reads each b x b block as one contiguous span and a
// warp keeps 32 / B rows in flight.  The sums run in the same order as a
// whole-row product would (slots, fill slots, tail; c ascending).
template <int B>
struct RowLanes {
  static constexpr int kRowsPerWarp = 32 / B;
  int r;            // block row of this lane
  int base;         // first lane of the group
  unsigned mask;    // the group's lanes
  int64_t q;        // position of the row, or -1 for an idle lane
  __device__ __forceinline__ RowLanes(int64_t q0, int64_t q1) {
    const int lane = threadIdx.x & 31, g = lane / B;
    r = lane - g * B;
    base = g * B;
    mask = ((1u << B) - 1u) << base;
    const int64_t w = blockIdx.x * (int64_t)kWarps + (threadIdx.x >> 5);
    q = q0 + w * kRowsPerWarp + g;
    if (g >= kRowsPerWarp || q >= q1) q = -1;
  }
};

inline int64_t row_lane_blocks_of(int64_t rows, int b) {
  const int64_t per_block = (int64_t)kWarps * (32 / b);
  return (rows + per_block - 1) / per_block;
}

// Blocks of a multiple of 16 bytes (b = 1, 2, 4) are swept a thread per row
// with 128-bit loads, which measured faster at b = 4; the others (b = 3, 5),
// whose blocks take no vector loads, by B lanes per row.
template <int B, class T>
constexpr bool kRowLanes = B > 1 && (B * B * sizeof(T)) % 16 != 0;

// t -= sum over the ILU(1) fill slots f in fm of F_f y_(i + off2[f]) (whole rows)
template <int B, class T>
__device__ __forceinline__ void fill_slots_apply(const IluView<T> &F, unsigned fm, int64_t i, int64_t q,
                                                 const T *y, T (&t)[B]) {
  constexpr int BB = B * B;
  if (!fm) return;
  const int64_t np = F.g.n_rows;
#pragma unroll
  for (int f = 0; f < kFill; f++) {
    if (!((fm >> f) & 1u)) continue;
    const int64_t j = i + F.g.off2[f];
    T yj[B];
    load_blk<B>(y + j * B, yj);
    T bv[BB];
    load_block<B>(F.fell + ((int64_t)(kSlots + f) * np + q) * BB, bv);
#pragma unroll
    for (int r = 0; r < B; r++)
#pragma unroll
      for (int c = 0; c < B; c++) t[r] = fma(-bv[r * B + c], yj[c], t[r]);
  }
}

// t -= the slots in sm, the fill slots in fm and the lower (lower == true) or
// upper tail entries of row i, a thread per whole row
template <int B, class T>
__device__ __forceinline__ void whole_row_sweep(const IluView<T> &F, int64_t i, int64_t q, unsigned sm, unsigned fm,
                                                bool tail, bool lower, const T *y, T (&t)[B]) {
  constexpr int BB = B * B;
  const int64_t np = F.g.n_rows;
#pragma unroll
  for (int s = 0; s < kSlots; s++) {
    if (!((sm >> s) & 1u)) continue;
    const int64_t j = i + F.g.off[s];
    T yj[B];
    load_blk<B>(y + j * B, yj);
    T bv[BB];
    load_block<B>(F.fell + ((int64_t)s * np + q) * BB, bv);
#pragma unroll
    for (int r = 0; r < B; r++)
#pragma unroll
      for (int c = 0; c < B; c++) t[r] = fma(-bv[r * B + c], yj[c], t[r]);
  }
  fill_slots_apply<B>(F, fm, i, q, y, t);
  if (tail)
    for (int64_t u = F.ftptr[q]; u < F.ftptr[q + 1]; u++) {
      const int64_t j = F.ftcol[u];
      if (lower ? !F.ftlow[u] : (F.ftlow[u] || j == i)) continue;
      const T *blk = F.ftval + u * BB;
#pragma unroll
      for (int r = 0; r < B; r++)
#pragma unroll
        for (int c = 0; c < B; c++) t[r] = fma(-blk[r * B + c], y[j * B + c], t[r]);
    }
}

// t_r -= sum over c of F_rc y_j,c for one b x b block F (row r at p)
template <int B, class T>
__device__ __forceinline__ void row_update(const T *__restrict__ p, const T *y, int64_t j, T &t) {
  T row[B], yj[B];
  load_blk<B>(p, row);
  load_blk<B>(y + j * B, yj);
#pragma unroll
  for (int c = 0; c < B; c++) t = fma(-row[c], yj[c], t);
}

// lane r of row i's group: t_r -= the slots in sm, the fill slots in fm, and
// the tail entries that are lower (lower == true) or upper (j != i)
template <int B, class T>
__device__ __forceinline__ void row_sweep(const IluView<T> &F, int64_t i, int64_t q, int r, unsigned sm, unsigned fm,
                                          bool tail, bool lower, const T *y, T &t) {
  constexpr int BB = B * B;
  const int64_t np = F.g.n_rows;
#pragma unroll
  for (int s = 0; s < kSlots; s++)
    if ((sm >> s) & 1u) row_update<B>(F.fell + ((int64_t)s * np + q) * BB + r * B, y, i + F.g.off[s], t);
  if (fm)
#pragma unroll
    for (int f = 0; f < kFill; f++)
      if ((fm >> f) & 1u) row_update<B>(F.fell + ((int64_t)(kSlots + f) * np + q) * BB + r * B, y, i + F.g.off2[f], t);
  if (tail)
    for (int64_t u = F.ftptr[q]; u < F.ftptr[q + 1]; u++) {
      const int64_t j = F.ftcol[u];
      if (lower ? !F.ftlow[u] : (F.ftlow[u] || j == i)) continue;
      row_update<B>(F.ftval + u * BB + r * B, y, j, t);
    }
}

// x_i = U_ii^-1 t written over y_i, and z_i = y1_i + Pi e0_i + x_i to zout
template <int B, class T, class TZ>
__device__ __forceinline__ void ilu_bwd_finish(const IluView<T> &F, int64_t q, int64_t i, const T (&t)[B], T *y,
                                               const T *__restrict__ y1, const T *__restrict__ e0,
                                               TZ *__restrict__ zout) {
  constexpr int BB = B * B;
  T dg[BB];
  load_block<B>(F.fell + ((int64_t)kSelf * F.g.n_rows + q) * BB, dg);
  T xv[B];
#pragma unroll
  for (int r = 0; r < B; r++) {
    T a = T(0);
#pragma unroll
    for (int c = 0; c < B; c++) a = fma(dg[r * B + c], t[c], a);
    xv[r] = a;
  }
  store_blk<B>(y + i * B, xv);
  if (zout) {
    T zb[B];
    load_y2<B>(y1, e0, i, zb);
    TZ zo[B];
#pragma unroll
    for (int r = 0; r < B; r++) zo[r] = static_cast<TZ>(zb[r] + xv[r]);
    store_blk<B>(zout + i * B, zo);
  }
}

template <int B, class T>
__global__ void __launch_bounds__(kThreads) k_ilu_fwd(IluView<T> F, const T *__restrict__ rhs, T *y, int64_t q0,
                                                      int64_t q1, int64_t q2, int64_t cell_blocks) {
  pdl_enter();
  constexpr int BB = B * B;
  if (blockIdx.x < cell_blocks) {
    if constexpr (kRowLanes<B, T>) {
      const RowLanes<B> L(q0, q1);
      if (L.q < 0) return;
      const int64_t q = L.q, i = F.crow[q];
      T t = rhs[i * B + L.r];
      const unsigned lm = F.lmask[q];
      row_sweep<B>(F, i, q, L.r, lm, F.flmask ? F.flmask[q] : 0u, lm & kTailBit, true, y, t);
      y[i * B + L.r] = t;
    } else {
      const int64_t q = q0 + blockIdx.x * (int64_t)kThreads + threadIdx.x;
      if (q >= q1) return;
      const int64_t i = F.crow[q];
      T t[B];
      load_blk<B>(rhs + i * B, t);
      const unsigned lm = F.lmask[q];
      whole_row_sweep<B>(F, i, q, lm, F.flmask ? F.flmask[q] : 0u, lm & kTailBit, true, y, t);
      store_blk<B>(y + i * B, t);
    }
  } else {
    // a long row (a well), one block per row
    const int64_t q = q1 + (blockIdx.x - cell_blocks);
    if (q >= q2) return;
    const int64_t i = F.crow[q];
    double acc[B] = {};
    for (int64_t u = F.ftptr[q] + threadIdx.x; u < F.ftptr[q + 1]; u += kThreads) {
      if (!F.ftlow[u]) continue;
      const int64_t j = F.ftcol[u];
      const T *blk = F.ftval + u * BB;
#pragma unroll
      for (int r = 0; r < B; r++)
#pragma unroll
        for (int c = 0; c < B; c++) acc[r] = fma(to_d(blk[r * B + c]), to_d(y[j * B + c]), acc[r]);
    }
    block_sum<B>(acc);
    if (threadIdx.x == 0)
#pragma unroll
      for (int r = 0; r < B; r++) y[i * B + r] = static_cast<T>(to_d(rhs[i * B + r]) - acc[r]);
  }
}

// Backward sweep of one colour: x_i = U_ii^-1 (y_i - sum over upper j of
// U_ij x_j), written over y (and z = y1 + Pi e0 + x to zout when given).
// With rhs given (the last colour, whose rows have no upper neighbour), the
// forward sweep of the colour is done in the same pass: t = rhs_i - sum over
// lower j of L_ij y_j, the same operations as k_ilu_fwd, then x_i = U_ii^-1 t.
template <int B, class T, class TZ>
__global__ void __launch_bounds__(kThreads) k_ilu_bwd(IluView<T> F, T *y, int64_t q0, int64_t q1, int64_t q2,
                                                      int64_t cell_blocks, const T *__restrict__ y1,
                                                      const T *__restrict__ e0, TZ *__restrict__ zout,
                                                      const T *__restrict__ rhs) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t np = F.g.n_rows;
  if (blockIdx.x < cell_blocks && !kRowLanes<B, T>) {
    const int64_t q = q0 + blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (q >= q1) return;
    const int64_t i = F.crow[q];
    T t[B];
    load_blk<B>((rhs ? rhs : y) + i * B, t);
    const unsigned lmq = F.lmask[q];
    const unsigned um = rhs ? lmq : F.emask[i] & ~lmq & ~(1u << kSelf);
    const unsigned fm = F.fmask ? (rhs ? F.flmask[q] : F.fmask[q] & ~F.flmask[q]) : 0u;
    whole_row_sweep<B>(F, i, q, um, fm, lmq & kTailBit, rhs != nullptr, y, t);
    ilu_bwd_finish<B, T, TZ>(F, q, i, t, y, y1, e0, zout);
    return;
  }
  if (blockIdx.x < cell_blocks) {
    const RowLanes<B> L(q0, q1);
    if (L.q < 0) return;   // whole groups leave together
    const int64_t q = L.q, i = F.crow[q];
    const int r = L.r;
    T t = (rhs ? rhs : y)[i * B + r];
    const unsigned lmq = F.lmask[q];
    const unsigned um = rhs ? lmq : F.emask[i] & ~lmq & ~(1u << kSelf);
    const unsigned fm = F.fmask ? (rhs ? F.flmask[q] : F.fmask[q] & ~F.flmask[q]) : 0u;
    row_sweep<B>(F, i, q, r, um, fm, lmq & kTailBit, rhs != nullptr, y, t);
    // x_r = sum_c (U_ii^-1)_rc t_c, t_c from lane c of the group
    T dg[B];
    load_blk<B>(F.fell + ((int64_t)kSelf * np + q) * BB + r * B, dg);
    T x = T(0);
#pragma unroll
    for (int c = 0; c < B; c++) x = fma(dg[c], __shfl_sync(L.mask, t, L.base + c), x);
    y[i * B + r] = x;
    if (zout) {
      T zb = y1 ? y1[i * B + r] : T(0);
      if (r == 0) zb = zb + e0[i];
      zout[i * B + r] = static_cast<TZ>(zb + x);
    }
    return;
  }
  // a long row (a well), one block per row
  const int64_t q = q1 + (blockIdx.x - cell_blocks);
  if (q >= q2) return;
  const int64_t i = F.crow[q];
  double acc[B] = {};
  for (int64_t u = F.ftptr[q] + threadIdx.x; u < F.ftptr[q + 1]; u += kThreads) {
    const int64_t j = F.ftcol[u];
    if (rhs ? !F.ftlow[u] : (F.ftlow[u] || j == i)) continue;
    const T *blk = F.ftval + u * BB;
#pragma unroll
    for (int r = 0; r < B; r++)
#pragma unroll
      for (int c = 0; c < B; c++) acc[r] = fma(to_d(blk[r * B + c]), to_d(y[j * B + c]), acc[r]);
  }
  block_sum<B>(acc);
  if (threadIdx.x != 0) return;
  const T *src = rhs ? rhs : y;
  T t[B];
#pragma unroll
  for (int r = 0; r < B; r++) t[r] = static_cast<T>(to_d(src[i * B + r]) - acc[r]);
  ilu_bwd_finish<B, T, TZ>(F, q, i, t, y, y1, e0, zout);
}

// --------------------------------------------------- CPR residuals on Ã
// rp_i = f_i0 - (Ã y)_i0, Ã_ii = I
template <int B, class T>
__global__ void __launch_bounds__(kThreads) k_resid_p(MatView<T> At, const T *__restrict__ atp,
                                                      const T *__restrict__ f, const T *__restrict__ y,
                                                      T *__restrict__ rp, int64_t cell_blocks, int unit) {
  pdl_enter();
  constexpr int BB = B * B;
  if (blockIdx.x < cell_blocks) {
    const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (i >= At.g.nc) return;
    const int64_t nc = At.g.nc;
    T acc = unit ? y[i * B] : T(0);
    const unsigned m = At.emask[i] & (unit ? ~(1u << kSelf) : ~0u);
    // all slots' loads at once; an absent slot reads row i and adds zero terms
#pragma unroll
    for (int s = 0; s < kSlots; s++) {
      const bool on = (m >> s) & 1u;
      const int64_t j = on ? i + At.g.off[s] : i;
#pragma unroll
      for (int c = 0; c < B; c++)
        acc = fma(on ? atp[((int64_t)s * B + c) * nc + i] : T(0), y[j * B + c], acc);
    }
    if (m & kTailBit)
    for (int64_t t = At.tptr[i]; t < At.tptr[i + 1]; t++) {
      const int64_t j = At.tcol[t];
      if (unit && j == i) continue;
      const T *blk = At.tval + t * BB;
#pragma unroll
      for (int c = 0; c < B; c++) acc = fma(blk[c], y[j * B + c], acc);
    }
    rp[i] = f[i * B] - acc;
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t i = At.g.nc + (blockIdx.x - cell_blocks) * (int64_t)kWarps + (threadIdx.x >> 5);
    if (i >= At.g.n_rows) return;
    double acc = 0.0;
    for (int64_t t = At.tptr[i] + lane; t < At.tptr[i + 1]; t += 32) {
      const int64_t j = At.tcol[t];
      if (unit && j == i) continue;
      const T *blk = At.tval + t * BB;
#pragma unroll
      for (int c = 0; c < B; c++) acc = fma(to_d(blk[c]), to_d(y[j * B + c]), acc);
    }
    acc = warp_sum(acc);
    if (lane == 0) rp[i] = static_cast<T>(to_d(f[i * B]) - ((unit ? to_d(y[i * B]) : 0.0) + acc));
  }
}

// r = f - Ã y2 with y2 = y1 + e0 in entry 0 of every block
template <int B, class T>
__global__ void __launch_bounds__(kThreads) k_resid_full(MatView<T> At, const T *__restrict__ f,
                                                         const T *__restrict__ y1, const T *__restrict__ e0,
                                                         T *__restrict__ r, int64_t cell_blocks, int unit,
                                                         Seed<T> sd) {
  pdl_enter();
  constexpr int BB = B * B;
  if (blockIdx.x < cell_blocks) {
    const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (i >= At.g.nc) return;
    const int64_t nc = At.g.nc;
    T acc[B];
    if (unit) {
      load_y2<B>(y1, e0, i, acc);
    } else {
#pragma unroll
      for (int c = 0; c < B; c++) acc[c] = T(0);
    }
    const unsigned m = At.emask[i] & (unit ? ~(1u << kSelf) : ~0u);
#pragma unroll
    for (int s = 0; s < kSlots; s++) {
      if (!((m >> s) & 1u)) continue;
      const int64_t j = i + At.g.off[s];
      T yj[B];
      load_y2<B>(y1, e0, j, yj);
      T bv[BB];
      load_block<B>(At.ell + ((int64_t)s * nc + i) * BB, bv);
#pragma unroll
      for (int rr = 0; rr < B; rr++)
#pragma unroll
        for (int c = 0; c < B; c++) acc[rr] = fma(bv[rr * B + c], yj[c], acc[rr]);
    }
    if (m & kTailBit)
    for (int64_t t = At.tptr[i]; t < At.tptr[i + 1]; t++) {
      const int64_t j = At.tcol[t];
      if (unit && j == i) continue;
      T yj[B];
#pragma unroll
      for (int c = 0; c < B; c++) yj[c] = y1 ? y1[j * B + c] : T(0);
      yj[0] = yj[0] + e0[j];
      const T *blk = At.tval + t * BB;
#pragma unroll
      for (int rr = 0; rr < B; rr++)
#pragma unroll
        for (int c = 0; c < B; c++) acc[rr] = fma(blk[rr * B + c], yj[c], acc[rr]);
    }
    T fv[B];
    load_blk<B>(f + i * B, fv);
#pragma unroll
    for (int rr = 0; rr < B; rr++) fv[rr] = fv[rr] - acc[rr];
    store_blk<B>(r + i * B, fv);
    seed_row<B>(sd, i, fv);
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t i = At.g.nc + (blockIdx.x - cell_blocks) * (int64_t)kWarps + (threadIdx.x >> 5);
    if (i >= At.g.n_rows) return;
    double acc[B] = {};
    for (int64_t t = At.tptr[i] + lane; t < At.tptr[i + 1]; t += 32) {
      const int64_t j = At.tcol[t];
      if (unit && j == i) continue;
      const T *blk = At.tval + t * BB;
#pragma unroll
      for (int c = 0; c < B; c++) {
        double yj = y1 ? to_d(y1[j * B + c]) : 0.0;
        if (c == 0) yj += to_d(e0[j]);
#pragma unroll
        for (int rr = 0; rr < B; rr++) acc[rr] = fma(to_d(blk[rr * B + c]), yj, acc[rr]);
      }
    }
#pragma unroll
    for (int rr = 0; rr < B; rr++) acc[rr] = warp_sum(acc[rr]);
    if (lane == 0)
#pragma unroll
      for (int rr = 0; rr < B; rr++) {
        double own = 0.0;
        if (unit) {
          own = y1 ? to_d(y1[i * B + rr]) : 0.0;
          if (rr == 0) own += to_d(e0[i]);
        }
        const T rv = static_cast<T>(to_d(f[i * B + rr]) - (own + acc[rr]));
        r[i * B + rr] = rv;
        if (sd.colour && sd.colour[i] == 0) sd.y0[i * B + rr] = rv;
      }
  }
}

// ------------------------------------------------------------- AMG pieces
// (A x)_i of a scalar level, with x_j = xv(j) (an array read, or a value
// formed on the fly from the inputs of a fused step)
template <class T, class XV>
__device__ __forceinline__ T scalar_rowdot_fn(const ScalarOp<T> &op, int64_t i, XV xv) {
  T acc = T(0);
  if (op.is_ell) {
    if (i < op.g.nc) {
      // every slot's loads are issued at once, an absent slot reading row i
      // and contributing a zero term, so a row costs one memory round trip
      const unsigned m = op.emask[i];
      T a[kSlots], x[kSlots];
#pragma unroll
      for (int s = 0; s < kSlots; s++) {
        const bool on = (m >> s) & 1u;
        a[s] = on ? op.ell[(int64_t)s * op.g.nc + i] : T(0);
        x[s] = xv(on ? i + op.g.off[s] : i);
      }
#pragma unroll
      for (int s = 0; s < kSlots; s++) acc = fma(a[s], x[s], acc);
      if (!(m & kTailBit)) return acc;
    }
    for (int64_t t = op.tptr[i]; t < op.tptr[i + 1]; t++) acc = fma(op.tval[t], xv((int64_t)op.tcol[t]), acc);
  } else {
#pragma unroll 4
    for (int64_t p = op.rp[i]; p < op.rp[i + 1]; p++) acc = fma(op.val[p], xv((int64_t)op.col[p]), acc);
  }
  return acc;
}

template <class T>
__device__ __forceinline__ T scalar_rowdot(const ScalarOp<T> &op, int64_t i, const T *__restrict__ x) {
  return scalar_rowdot_fn(op, i, [x](int64_t j) { return x[j]; });
}

template <class T>
__global__ void k_cheb_resid_init(ScalarOp<T> op, const T *__restrict__ r, const T *__restrict__ e,
                                  const T *__restrict__ dinv, T inv_theta, T *__restrict__ res,
                                  T *__restrict__ d) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= op.n) return;
  const T v = r[i] - scalar_rowdot(op, i, e);
  res[i] = v;
  d[i] = (dinv[i] * v) * inv_theta;
}

// res -= A d; dn = c1 d + c2 D^-1 res; e = (e + d) [+ dn if last]
template <class T>
__global__ void k_cheb_step(ScalarOp<T> op, const T *res_in, T *res_out, const T *__restrict__ d,
                            const T *__restrict__ dinv, T c1, T c2, T *__restrict__ dn, T *e, int last) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= op.n) return;
  const T rv = res_in[i] - scalar_rowdot(op, i, d);
  res_out[i] = rv;
  const T di = d[i];
  const T nv = fma(c1, di, c2 * (dinv[i] * rv));
  const T ev = e[i] + di;
  if (last) {
    e[i] = ev + nv;
  } else {
    e[i] = ev;
    dn[i] = nv;
  }
}

// The first Chebyshev step from e = 0 fused with its initialisation: with
// d = D^-1 r / theta formed on the fly for the neighbours, res = r - A d,
// dn = c1 d + c2 D^-1 res, e = d (+ dn on the last step): the same
// operations as setting d = D^-1 r / theta, e = 0 and then k_cheb_step.
template <class T>
__global__ void k_cheb_first(ScalarOp<T> op, const T *__restrict__ r, const T *__restrict__ dinv, T inv_theta,
                             T c1, T c2, T *__restrict__ res_out, T *__restrict__ d_out, T *__restrict__ dn,
                             T *__restrict__ e, int last) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= op.n) return;
  auto dval = [&](int64_t j) { return (dinv[j] * r[j]) * inv_theta; };
  const T rv = r[i] - scalar_rowdot_fn(op, i, dval);
  const T di = dval(i);
  const T nv = fma(c1, di, c2 * (dinv[i] * rv));
  const T ev = T(0) + di;
  if (last) {
    e[i] = ev + nv;
  } else {
    e[i] = ev;
    dn[i] = nv;
    res_out[i] = rv;
    d_out[i] = di;
  }
}

// Restriction fused with the fine residual: rc_I = sum over the members i of
// I, ascending, of (r_i - (A e)_i).  A group of kGroup lanes serves one
// aggregate: lane k forms the residual of members k, k + kGroup, ...; the
// group then adds them in member order, so the sum is the sequential one.
constexpr int kGroup = 8;

template <class T>
__global__ void k_restrict_resid(ScalarOp<T> op, int64_t nc, const int64_t *__restrict__ mptr,
                                 const int32_t *__restrict__ midx, const T *__restrict__ r,
                                 const T *__restrict__ e, T *__restrict__ rc) {
  pdl_enter();
  const int64_t I = (blockIdx.x * (int64_t)kThreads + threadIdx.x) / kGroup;
  if (I >= nc) return;  // the whole group leaves together
  const int k = threadIdx.x & (kGroup - 1);
  const unsigned gmask = ((1u << kGroup) - 1u) << ((threadIdx.x & 31) & ~(kGroup - 1));
  const int64_t t1 = mptr[I + 1];
  T s = T(0);
  for (int64_t t0 = mptr[I]; t0 < t1; t0 += kGroup) {
    T v = T(0);
    if (t0 + k < t1) {
      const int64_t i = midx[t0 + k];
      v = r[i] - scalar_rowdot(op, i, e);
    }
#pragma unroll
    for (int q = 0; q < kGroup; q++) {
      const T vq = __shfl_sync(gmask, v, q, kGroup);
      if (t0 + q < t1) s = s + vq;
    }
  }
  if (k == 0) rc[I] = s;
}

template <class T>
__global__ void k_prolong(int64_t n, const int32_t *__restrict__ agg, const T *__restrict__ ec,
                          T *__restrict__ e) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  const int32_t a = agg[i];
  if (a >= 0) e[i] = e[i] + ec[a];
}

template <class T>
__global__ void k_dense_gemv(int64_t n, const double *__restrict__ Minv, const T *__restrict__ r,
                             T *__restrict__ e) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int64_t i = blockIdx.x * (int64_t)kWarps + (threadIdx.x >> 5);
  if (i >= n) return;
  double acc = 0.0;
  for (int64_t j = lane; j < n; j += 32) acc = fma(Minv[i * n + j], to_d(r[j]), acc);
  acc = warp_sum(acc);
  if (lane == 0) e[i] = static_cast<T>(acc);
}

// The V-cycle from level h.l0 down, by one block of 1024 threads: the same
// Chebyshev, residual, restriction, coarsest solve and prolongation steps as
// the per-level kernels above (identical arithmetic), separated by block
// barriers instead of launches.
template <class T>
__device__ __forceinline__ T csr_rowdot(const CoarseLevel<T> &L, int64_t i, const T *x) {
  T acc = T(0);
  for (int64_t p = L.rp[i]; p < L.rp[i + 1]; p++) acc = fma(L.val[p], x[L.col[p]], acc);
  return acc;
}

template <class T>
__device__ void coarse_cheb(const CoarseLevel<T> &L, int deg, bool zero_init) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const T *r = L.r;
  T *e = L.e, *res = L.res, *d = L.d, *dn = L.dn;
  if (zero_init) {
    for (int64_t i = tid; i < L.n; i += nt) {
      d[i] = (L.dinv[i] * r[i]) * L.inv_theta;
      e[i] = T(0);
    }
  } else {
    for (int64_t i = tid; i < L.n; i += nt) {
      const T v = r[i] - csr_rowdot(L, i, e);
      res[i] = v;
      d[i] = (L.dinv[i] * v) * L.inv_theta;
    }
  }
  __syncthreads();
  const T *res_in = zero_init ? r : res;
  for (int k = 1; k < deg; k++) {
    const int last = (k == deg - 1);
    for (int64_t i = tid; i < L.n; i += nt) {
      const T rv = res_in[i] - csr_rowdot(L, i, d);
      res[i] = rv;
      const T di = d[i];
      const T nv = fma(L.c1[k], di, L.c2[k] * (L.dinv[i] * rv));
      const T ev = e[i] + di;
      if (last) e[i] = ev + nv;
      else { e[i] = ev; dn[i] = nv; }
    }
    __syncthreads();
    res_in = res;
    T *t = d; d = dn; dn = t;
  }
}

template <class T>
__global__ void __launch_bounds__(1024) k_vcycle_coarse(CoarseHierarchy<T> h) {
  pdl_enter();
  const int tid = threadIdx.x, nt = blockDim.x;
  const int last = h.nlev - 1;
  for (int l = h.l0; l < last; l++) {
    const CoarseLevel<T> &L = h.lv[l];
    coarse_cheb(L, h.deg, true);
    for (int64_t i = tid; i < L.n; i += nt) L.res[i] = L.r[i] - csr_rowdot(L, i, L.e);
    __syncthreads();
    const CoarseLevel<T> &C = h.lv[l + 1];
    for (int64_t I = tid; I < C.n; I += nt) {
      T acc = T(0);
      for (int64_t t = L.mptr[I]; t < L.mptr[I + 1]; t++) acc = acc + L.res[L.midx[t]];
      C.r[I] = acc;
    }
    __syncthreads();
  }
  {
    const CoarseLevel<T> &C = h.lv[last];
    for (int64_t i = tid; i < C.n; i += nt) {
      double acc = 0.0;
      for (int64_t j = 0; j < C.n; j++) acc = fma(h.cinv[i * C.n + j], to_d(C.r[j]), acc);
      C.e[i] = static_cast<T>(acc);
    }
    __syncthreads();
  }
  for (int l = last - 1; l >= h.l0; l--) {
    const CoarseLevel<T> &L = h.lv[l];
    const CoarseLevel<T> &C = h.lv[l + 1];
    for (int64_t i = tid; i < L.n; i += nt) {
      const int32_t a = L.agg[i];
      if (a >= 0) L.e[i] = L.e[i] + C.e[a];
    }
    __syncthreads();
    coarse_cheb(L, h.deg, false);
  }
}

// ------------------------------------------------------- FGMRES / CGS2
// w -= sum_k h_k V_k; if want_norm: out[0] = ||w||^2
__global__ void __launch_bounds__(kThreads) k_cgs_update(const double *__restrict__ V, int64_t N, int K,
                                                         const double *__restrict__ h, double *__restrict__ w,
                                                         int want_norm, double *partial, unsigned int *counter,
                                                         double *out) {
  pdl_enter();
  __shared__ double sh[kMaxRestart + 1];
  for (int k = threadIdx.x; k < K; k += kThreads) sh[k] = h[k];
  __syncthreads();
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < N; i += (int64_t)gridDim.x * kThreads) {
    double v = w[i];
    // unrolled so that several basis loads are in flight ahead of the FMA chain
#pragma unroll 8
    for (int k = 0; k < K; k++) v = fma(-sh[k], V[(int64_t)k * N + i], v);
    w[i] = v;
    acc[0] = fma(v, v, acc[0]);
  }
  if (!want_norm) return;
  block_partial<1>(acc, partial + (int64_t)blockIdx.x * kRedStride);
  last_block_finish(partial, counter, 1, out, 0);
}

// ---- CGS2 in three passes over V (K + 1 <= KM outputs per reduction) ----
// Partial sums are stored [k][block] so that the last block reduces each k
// with one warp and coalesced loads, in block order.
__device__ void last_block_finish_kb(const double *partial, unsigned int *counter, int K, double *out) {
  __shared__ bool is_last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int k = warp; k < K; k += kWarps) {
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(partial + (int64_t)k * gridDim.x + b);
    s = warp_sum(s);
    if (lane == 0) out[k] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) *counter = 0u;
}

template <int KM>
__device__ void block_partial_kb(double (&acc)[KM], int K, double *partial, const double *extra = nullptr) {
  // partial[k][block] for k < K from acc, and for k = K from *extra if given
  __shared__ double sm[kWarps][KM + 1];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  constexpr int kSpan = 32 / KM;
  const double v = warp_reduce_scatter<KM>(acc, lane);
  if ((lane & (kSpan - 1)) == 0) sm[warp][lane / kSpan] = v;
  if (extra) {
    const double e = warp_sum(*extra);
    if (lane == 0) sm[warp][KM] = e;
  }
  __syncthreads();
  const int Kt = K + (extra ? 1 : 0);
  for (int k = threadIdx.x; k < Kt; k += kThreads) {
    const int src = k < K ? k : KM;
    double t = 0.0;
    for (int w = 0; w < kWarps; w++) t += sm[w][src];
    partial[(int64_t)k * gridDim.x + blockIdx.x] = t;
  }
  __syncthreads();
}

// out[k] = <V_k, w> for k < K, out[K] = <w, w>, for any K up to the
// largest restart: chunks of KC vectors, one pass over each chunk, partial
// sums stored [k][block] and finished a warp per k.
template <int KC>
__global__ void __launch_bounds__(kThreads) k_multidot(const double *__restrict__ V, int64_t N, int K,
                                                       const double *__restrict__ w, double *partial,
                                                       unsigned int *counter, double *out) {
  pdl_enter();
  for (int k0 = 0; k0 < K; k0 += KC) {
    const int Kc = min(KC, K - k0);
    const bool last = k0 + KC >= K;
    const double *Vc = V + (int64_t)k0 * N;
    double acc[KC] = {};
    double ww = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < N; i += (int64_t)gridDim.x * kThreads) {
      const double wi = w[i];
      if (last) ww = fma(wi, wi, ww);
#pragma unroll
      for (int g = 0; g < KC; g += 8) {
        if (g < Kc) {
#pragma unroll
          for (int u = g; u < g + 8; u++)
            if (u < Kc) acc[u] = fma(Vc[(int64_t)u * N + i], wi, acc[u]);
        }
      }
    }
    block_partial_kb<KC>(acc, Kc, partial + (int64_t)k0 * gridDim.x, last ? &ww : nullptr);
  }
  last_block_finish_kb(partial, counter, K + 1, out);
}

// out[k] = <V_k, w> for k < K, out[K] = <w, w>
template <int KM>
__global__ void __launch_bounds__(kThreads) k_cgs_dots(const double *__restrict__ V, int64_t N, int K,
                                                       const double *__restrict__ w, double *partial,
                                                       unsigned int *counter, double *out) {
  pdl_enter();
  double acc[KM] = {};
  double ww = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < N; i += (int64_t)gridDim.x * kThreads) {
    const double wi = w[i];
    ww = fma(wi, wi, ww);
    // groups of eight: K is the same for every thread, so a group past K is
    // branched over rather than issued with its lanes masked off, and the
    // eight loads of a group are in flight together
#pragma unroll
    for (int g = 0; g < KM; g += 8) {
      if (g < K) {
#pragma unroll
        for (int u = g; u < g + 8; u++)
          if (u < K) acc[u] = fma(V[(int64_t)u * N + i], wi, acc[u]);
      }
    }
  }
  block_partial_kb<KM>(acc, K, partial, &ww);
  last_block_finish_kb(partial, counter, K + 1, out);
}

// w -= sum_k h_k V_k; out[k] = <V_k, w> with the updated w
template <int KM>
__global__ void __launch_bounds__(kThreads) k_cgs_update_dots(const double *__restrict__ V, int64_t N, int K,
                                                              const double *__restrict__ h, double *__restrict__ w,
                                                              double *partial, unsigned int *counter, double *out) {
  pdl_enter();
  __shared__ double sh[KM];
  for (int k = threadIdx.x; k < K; k += kThreads) sh[k] = h[k];
  __syncthreads();
  double acc[KM] = {};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < N; i += (int64_t)gridDim.x * kThreads) {
    double t = w[i];
    double vv[KM];
#pragma unroll
    for (int g = 0; g < KM; g += 4) {
      if (g < K) {
#pragma unroll
        for (int u = g; u < g + 4; u++)
          if (u < K) {
            vv[u] = V[(int64_t)u * N + i];
            t = fma(-sh[u], vv[u], t);
          }
      }
    }
    w[i] = t;
#pragma unroll
    for (int g = 0; g < KM; g += 4) {
      if (g < K) {
#pragma unroll
        for (int u = g; u < g + 4; u++)
          if (u < K) acc[u] = fma(vv[u], t, acc[u]);
      }
    }
  }
  block_partial_kb<KM>(acc, K, partial);
  last_block_finish_kb(partial, counter, K, out);
}

// ------------------------------------------- bulk-copy staged Gram-Schmidt
// The basis tile of a block (kTE consecutive elements of each of the K
// vectors, and of w) is brought into shared memory by one-dimensional bulk
// copies (cp.async.bulk, completed on an mbarrier), double-buffered, so that
// the next tile is in flight while the FP64 pipe works on this one.  Every
// wait is bounded: past kMbarSpin polls the block marks its sums NaN (the
// solve then stops with TRS_ERR_NAN), waits (bounded) for its copies still
// in flight and finishes.  Needs N even (16-byte aligned vector rows).
constexpr int kTE = kThreads;   // elements per tile, one per thread
constexpr int kMbarSpin = 1 << 20;      // polls of a tile's barrier
constexpr int kMbarDrain = 1 << 16;     // polls for copies still in flight after a failure

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint64_t *bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\tselp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0u;
}
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int polls) {
  for (int it = 0; it < polls; it++)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

// UPD = false: out[k] = <V_k, w> (k < K), out[K] = <w, w>.
// UPD = true:  w -= sum_k h_k V_k, then out[k] = <V_k, w> with the new w.
template <int KM, bool UPD>
__global__ void __launch_bounds__(kThreads, 1) k_cgs_staged(const double *__restrict__ V, int64_t N, int K,
                                                            const double *__restrict__ h, double *__restrict__ w,
                                                            double *partial, unsigned int *counter, double *out,
                                                            uint32_t tx_extra) {
  extern __shared__ __align__(128) double tile[];   // [2][KM + 1][kTE]: K vectors, then w
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ double sh[KM];
  const int tid = threadIdx.x;
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  pdl_enter();
  if (UPD)
    for (int k = tid; k < K; k += kThreads) sh[k] = h[k];
  __syncthreads();
  const int64_t ntiles = (N + kTE - 1) / kTE;
  // thread 0: the copies of tile t into buffer b
  auto issue = [&](int64_t t, int b) {
    const int64_t e0 = t * kTE;
    const uint32_t bytes = (uint32_t)min((int64_t)kTE, N - e0) * 8u;
    double *dst = tile + (size_t)b * (KM + 1) * kTE;
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    mbar_expect_tx(&bar[b], bytes * (uint32_t)(K + 1) + tx_extra);
    for (int u = 0; u < K; u++) bulk_g2s(dst + (size_t)u * kTE, V + (int64_t)u * N + e0, bytes, &bar[b]);
    bulk_g2s(dst + (size_t)KM * kTE, w + e0, bytes, &bar[b]);
  };
  double acc[KM] = {};
  double ww = 0.0;
  // bit b: the phase parity of bar[b]; a copy into buffer b not yet waited for
  uint32_t parity = 0u, pending = 0u;
  bool failed = false;
  int64_t t = blockIdx.x;
  if (tid == 0 && t < ntiles) issue(t, 0);
  if (t < ntiles) pending |= 1u;
  for (int b = 0; t < ntiles; t += gridDim.x, b ^= 1) {
    const int64_t tn = t + gridDim.x;
    if (tid == 0 && tn < ntiles) issue(tn, b ^ 1);
    if (tn < ntiles) pending |= 1u << (b ^ 1);
    const bool ok = mbar_wait_bounded(&bar[b], (parity >> b) & 1u, kMbarSpin);
    if (__syncthreads_or(!ok)) {
      failed = true;
      break;
    }
    parity ^= 1u << b;
    pending &= ~(1u << b);
    const int64_t i = t * kTE + tid;
    if (i < N) {
      const double *tv = tile + (size_t)b * (KM + 1) * kTE + tid;
      const double wi = tv[(size_t)KM * kTE];
      if (!UPD) {
        ww = fma(wi, wi, ww);
#pragma unroll
        for (int g = 0; g < KM; g += 4) {
          if (g < K) {
#pragma unroll
            for (int u = g; u < g + 4; u++)
              if (u < K) acc[u] = fma(tv[(size_t)u * kTE], wi, acc[u]);
          }
        }
      } else {
        double tt = wi;
#pragma unroll
        for (int g = 0; g < KM; g += 4) {
          if (g < K) {
#pragma unroll
            for (int u = g; u < g + 4; u++)
              if (u < K) tt = fma(-sh[u], tv[(size_t)u * kTE], tt);
          }
        }
        w[i] = tt;
#pragma unroll
        for (int g = 0; g < KM; g += 4) {
          if (g < K) {
#pragma unroll
            for (int u = g; u < g + 4; u++)
              if (u < K) acc[u] = fma(tv[(size_t)u * kTE], tt, acc[u]);
          }
        }
      }
    }
    __syncthreads();   // buffer b is read before it is refilled
  }
  if (failed) {
    // copies still in flight land before the block leaves (bounded)
    for (int b = 0; b < 2; b++)
      if ((pending >> b) & 1u) mbar_wait_bounded(&bar[b], (parity >> b) & 1u, kMbarDrain);
#pragma unroll
    for (int u = 0; u < KM; u++) acc[u] = __longlong_as_double(0x7ff8000000000000ll);
    ww = __longlong_as_double(0x7ff8000000000000ll);
  }
  block_partial_kb<KM>(acc, K, partial, UPD ? nullptr : &ww);
  last_block_finish_kb(partial, counter, UPD ? K : K + 1, out);
}

// Arnoldi column j of H (row-major, m columns): h1 + h2, norm; Givens.
// status[0] = |g_{j+1}| / ||b||, status[1] = breakdown flag, hnorm[0] = h_{j+1,j}
__global__ void k_givens(int j, int m, double *H, const double *h1, const double *h2, const double *hn2,
                         const double *wn2, double *cs, double *sn, double *g, double *hnorm,
                         double *status, double inv_bnorm) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int k = 0; k <= j; k++) H[k * m + j] = h1[k] + h2[k];
  const double hn = sqrt(hn2[0]);
  H[(j + 1) * m + j] = hn;
  for (int k = 0; k < j; k++) {
    const double a = H[k * m + j], c = H[(k + 1) * m + j];
    H[k * m + j] = cs[k] * a + sn[k] * c;
    H[(k + 1) * m + j] = -sn[k] * a + cs[k] * c;
  }
  const double a = H[j * m + j], c = H[(j + 1) * m + j];
  const double d = sqrt(a * a + c * c);
  cs[j] = a / d;
  sn[j] = c / d;
  H[j * m + j] = d;
  H[(j + 1) * m + j] = 0.0;
  g[j + 1] = -sn[j] * g[j];
  g[j] = cs[j] * g[j];
  hnorm[0] = hn;
  status[0] = fabs(g[j + 1]) * inv_bnorm;
  status[1] = (hn <= 1e-14 * sqrt(wn2[0])) ? 1.0 : 0.0;
}

__global__ void k_lsq(int jdone, int m, const double *H, const double *g, double *y) {
  pdl_enter();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  for (int i = jdone - 1; i >= 0; i--) {
    double s = g[i];
    for (int k = i + 1; k < jdone; k++) s = s - H[i * m + k] * y[k];
    y[i] = s / H[i * m + i];
  }
}

template <class TZ>
__global__ void __launch_bounds__(kThreads) k_xupdate(const TZ *__restrict__ Z, int64_t N, int K,
                                                      const double *__restrict__ y, double *__restrict__ x) {
  pdl_enter();
  __shared__ double sy[kMaxRestart];
  for (int k = threadIdx.x; k < K; k += kThreads) sy[k] = y[k];
  __syncthreads();
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < N; i += (int64_t)gridDim.x * kThreads) {
    double v = x[i];
#pragma unroll 8
    for (int k = 0; k < K; k++) v = fma(sy[k], to_d(Z[(int64_t)k * N + i]), v);
    x[i] = v;
  }
}

template <class TS, class TD>
__global__ void k_cast(const TS *__restrict__ a, TD *__restrict__ b, int64_t n) {
  pdl_enter();
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    b[i] = static_cast<TD>(a[i]);
}

// ----------------------------------------- CPR-FP / CPR-PF pieces
// z = y1 + Pi_p e0 in FP64 (the last step of CPR-FP)
template <int B, class T>
__global__ void __launch_bounds__(kThreads) k_cpr_combine(int64_t n, const T *__restrict__ y1,
                                                          const T *__restrict__ e0, double *__restrict__ z) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  T v[B];
  load_y2<B>(y1, e0, i, v);
  double o[B];
#pragma unroll
  for (int c = 0; c < B; c++) o[c] = to_d(v[c]);
  store_blk<B>(z + i * B, o);
}

// rp = Pi_r f, the pressure entries (the first step of CPR-PF)
template <class T>
__global__ void k_pressure_of(int64_t n, int b, const T *__restrict__ f, T *__restrict__ rp) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i < n) rp[i] = f[i * b];
}

// ------------------------------------------------------------- BiCGSTAB
// The recurrences of van der Vorst's BiCGSTAB, right-preconditioned: the
// scalars (rho, alpha, omega, ...) stay in device memory, written by the
// last block of each reduction and read by the next kernel, so an iteration
// synchronises with the host once.

// Sums K partials per block in block order; true in the last block to
// arrive, where every thread holds the K sums.
template <int K>
__device__ __forceinline__ bool last_block_sums(const double *partial, unsigned int *counter, double (&sum)[K]) {
  __shared__ bool is_last;
  __shared__ double sm[kWarps];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return false;
  __threadfence();
  for (int k = 0; k < K; k++) {
    double s = 0.0;
    for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) s += __ldcg(partial + (int64_t)b * kRedStride + k);
    s = warp_sum(s);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    double t = 0.0;
    for (int w = 0; w < kWarps; w++) t += sm[w];
    sum[k] = t;
    __syncthreads();
  }
  if (threadIdx.x == 0) *counter = 0u;
  return true;
}

// (Re)start from the true residual r (r^ = r): rho = <r^, r> = ||r||^2.
__global__ void k_bicg_start(BicgScalars *sc, const double *rr, double bnorm, double rtol) {
  pdl_enter();
  sc->rho = rr[0];
  sc->rho_old = 1.0;
  sc->alpha = 1.0;
  sc->omega = 1.0;
  sc->rr = rr[0];
  sc->half = 0.0;
  sc->bnorm = bnorm;
  sc->rtol = rtol;
}

// p = r + beta (p - omega v), beta = (rho / rho_old)(alpha / omega), or p = r
// on the first step of a cycle; then f = D^-1 p, the input of CPR.
template <int B, class T>
__global__ void __launch_bounds__(kThreads) k_bicg_dir(int64_t n, const double *__restrict__ r,
                                                       const double *__restrict__ v, double *__restrict__ p,
                                                       const BicgScalars *__restrict__ sc, int first,
                                                       const T *__restrict__ dinv, T *__restrict__ f,
                                                       Seed<T> sd) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  double rv[B], pv[B];
  load_blk<B>(r + i * B, rv);
  if (first) {
#pragma unroll
    for (int c = 0; c < B; c++) pv[c] = rv[c];
  } else {
    const double beta = (sc->rho / sc->rho_old) * (sc->alpha / sc->omega), om = sc->omega;
    double vv[B];
    load_blk<B>(v + i * B, vv);
    load_blk<B>(p + i * B, pv);
#pragma unroll
    for (int c = 0; c < B; c++) pv[c] = rv[c] + beta * (pv[c] - om * vv[c]);
  }
  store_blk<B>(p + i * B, pv);
  T fr[B];
#pragma unroll
  for (int rr = 0; rr < B; rr++) {
    T acc = T(0);
#pragma unroll
    for (int c = 0; c < B; c++) acc = fma(dinv[(int64_t)(rr * B + c) * n + i], static_cast<T>(pv[c]), acc);
    f[i * B + rr] = acc;
    fr[rr] = acc;
  }
  seed_row<B>(sd, i, fr);
}

// y = A x with <w, y> (ND = 1) or <w, y>, <y, y> (ND = 2), one thread per
// cell row (blocks [0, cell_blocks)) and one warp per long row (the rest),
// as k_spmv.  Each block stores its ND partial sums at part[block * ND]; the
// last block sums them in block order and sets alpha = rho / <r^, v> (ND = 1:
// x = p^, y = v, w = r^) or omega = <t, s> / <t, t> (ND = 2: x = s^, y = t,
// w = s).
template <int B, int ND>
__global__ void __launch_bounds__(kThreads) k_bicg_spmv(MatView<double> A, const double *__restrict__ x,
                                                        double *__restrict__ y, const double *__restrict__ w,
                                                        int64_t cell_blocks, double *part, unsigned int *counter,
                                                        BicgScalars *sc) {
  pdl_enter();
  double acc2[ND] = {};
  if (blockIdx.x < cell_blocks) {
    const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (i < A.g.nc) {
      double acc[B] = {};
      cell_row_apply<B>(A, i, x, acc);
      store_blk<B>(y + i * B, acc);
      double wv[B];
      load_blk<B>(w + i * B, wv);
#pragma unroll
      for (int r = 0; r < B; r++) {
        acc2[0] = fma(wv[r], acc[r], acc2[0]);
        if constexpr (ND == 2) acc2[1] = fma(acc[r], acc[r], acc2[1]);
      }
    }
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t i = A.g.nc + (blockIdx.x - cell_blocks) * (int64_t)kWarps + (threadIdx.x >> 5);
    if (i < A.g.n_rows) {
      double acc[B] = {};
      long_row_apply<B>(A, i, x, acc, lane);
      if (lane == 0)
#pragma unroll
        for (int r = 0; r < B; r++) {
          y[i * B + r] = acc[r];
          acc2[0] = fma(w[i * B + r], acc[r], acc2[0]);
          if constexpr (ND == 2) acc2[1] = fma(acc[r], acc[r], acc2[1]);
        }
    }
  }
  // block sums (fixed shuffle pattern, warps in order)
  __shared__ double sm[kWarps][ND];
  __shared__ bool is_last;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < ND; k++) {
    const double v = warp_sum(acc2[k]);
    if (lane == 0) sm[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x < ND) {
    double t = 0.0;
    for (int q = 0; q < kWarps; q++) t += sm[q][threadIdx.x];
    part[(int64_t)blockIdx.x * ND + threadIdx.x] = t;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) is_last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!is_last) return;
  __threadfence();
  __shared__ double tot[kWarps][ND];
  double t[ND] = {};
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads)
#pragma unroll
    for (int k = 0; k < ND; k++) t[k] += __ldcg(part + (int64_t)b * ND + k);
#pragma unroll
  for (int k = 0; k < ND; k++) {
    const double v = warp_sum(t[k]);
    if (lane == 0) tot[warp][k] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double sum[ND];
#pragma unroll
    for (int k = 0; k < ND; k++) {
      sum[k] = 0.0;
      for (int q = 0; q < kWarps; q++) sum[k] += tot[q][k];
    }
    if constexpr (ND == 1) {
      sc->rv = sum[0];
      sc->alpha = sc->rho / sum[0];
    } else {
      sc->ts = sum[0];
      sc->tt = sum[1];
      sc->omega = sum[1] > 0.0 ? sum[0] / sum[1] : 0.0;
    }
    *counter = 0u;
  }
}

// s = r - alpha v and ||s||^2; the last block flags ||s|| <= rtol ||b||.
__global__ void __launch_bounds__(kThreads) k_bicg_s(int64_t N, const double *__restrict__ r,
                                                     const double *__restrict__ v, double *__restrict__ s,
                                                     double *partial, unsigned int *counter, BicgScalars *sc) {
  pdl_enter();
  const double alpha = sc->alpha;
  double acc[1] = {0.0};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < N; i += (int64_t)gridDim.x * kThreads) {
    const double si = r[i] - alpha * v[i];
    s[i] = si;
    acc[0] = fma(si, si, acc[0]);
  }
  block_partial<1>(acc, partial + (int64_t)blockIdx.x * kRedStride);
  double sum[1];
  if (!last_block_sums<1>(partial, counter, sum)) return;
  if (threadIdx.x == 0) {
    sc->ss = sum[0];
    sc->half = (sqrt(sum[0]) / sc->bnorm <= sc->rtol) ? 1.0 : 0.0;
  }
}

// x += alpha p^ + omega s^, r = s - omega t (omega taken as 0 when ||s|| met
// the tolerance); ||r||^2 and the next rho = <r^, r>.
__global__ void __launch_bounds__(kThreads) k_bicg_xr(int64_t N, const double *__restrict__ ph,
                                                      const double *__restrict__ sh, const double *__restrict__ s,
                                                      const double *__restrict__ t, const double *__restrict__ rh,
                                                      double *__restrict__ x, double *__restrict__ r,
                                                      double *partial, unsigned int *counter, BicgScalars *sc) {
  pdl_enter();
  const double alpha = sc->alpha, omega = sc->half != 0.0 ? 0.0 : sc->omega;
  double acc[2] = {0.0, 0.0};
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < N; i += (int64_t)gridDim.x * kThreads) {
    x[i] = x[i] + alpha * ph[i] + omega * sh[i];
    const double ri = s[i] - omega * t[i];
    r[i] = ri;
    acc[0] = fma(ri, ri, acc[0]);
    acc[1] = fma(rh[i], ri, acc[1]);
  }
  block_partial<2>(acc, partial + (int64_t)blockIdx.x * kRedStride);
  double sum[2];
  if (!last_block_sums<2>(partial, counter, sum)) return;
  if (threadIdx.x == 0) {
    sc->rr = sum[0];
    sc->rho_old = sc->rho;
    sc->rho = sum[1];
  }
}

inline unsigned grid_of(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }



}  // namespace

// ================================================================ launchers
template <class TA, class TX>
void launch_spmv(int b, const MatView<TA> &A, const TX *x, double *y, double alpha, double beta,
                 cudaStream_t s) {
  const int64_t cb = cell_blocks_of(A.g.nc), lb = long_blocks_of(A.g.n_rows - A.g.nc);
  if (cb + lb == 0) return;
  TRS_DISPATCH_B(b, launch_pdl(k_spmv<B, TA, TX>, (unsigned)(cb + lb), kThreads, 0, s, A, x, y, alpha, beta, cb));
  TRS_LAUNCHED();
}
template void launch_spmv<double, double>(int, const MatView<double> &, const double *, double *, double,
                                          double, cudaStream_t);
template void launch_spmv<double, float>(int, const MatView<double> &, const float *, double *, double,
                                         double, cudaStream_t);

void launch_true_residual(int b, const MatView<double> &A, const double *x, const double *rhs, double *r,
                          const RedScratch &red, double *out_norm2, cudaStream_t s) {
  TRS_DISPATCH_B(b, launch_pdl(k_true_residual<B>, red.grid, kThreads, 0, s, A, x, rhs, r, 0, 0, red.partial,
                                                                      red.counter, out_norm2));
  TRS_LAUNCHED();
}

void launch_norm2(const double *x, int64_t n, const RedScratch &red, double *out, cudaStream_t s) {
  launch_pdl(k_norm2, red.grid, kThreads, 0, s, x, n, red.partial, red.counter, out);
  TRS_LAUNCHED();
}

template <class T>
void launch_dscale(int b, int64_t n_rows, const double *w, const double *div, double *vout, const T *dinv, T *f,
                   const int32_t *colour, T *y0, cudaStream_t s) {
  if (!n_rows) return;
  const Seed<T> sd{colour, y0};
  TRS_DISPATCH_B(b, launch_pdl(k_dscale<B, T>, grid_of(n_rows), kThreads, 0, s, n_rows, w, div, vout, dinv, f, sd));
  TRS_LAUNCHED();
}

template <class T>
void launch_ilu_fwd(int b, const IluView<T> &F, const T *rhs, T *y, int64_t q0, int64_t q1, int64_t q2,
                    cudaStream_t s) {
  TRS_DISPATCH_B(b, {
    // cell rows: a thread or B lanes per row; long rows: one block per row
    const int64_t cb = kRowLanes<B, T> ? row_lane_blocks_of(q1 - q0, B) : cell_blocks_of(q1 - q0), lb = q2 - q1;
    if (cb + lb == 0) return;
    launch_pdl(k_ilu_fwd<B, T>, (unsigned)(cb + lb), kThreads, 0, s, F, rhs, y, q0, q1, q2, cb);
  });
  TRS_LAUNCHED();
}

template <class T, class TZ>
void launch_ilu_bwd(int b, const IluView<T> &F, T *y, int64_t q0, int64_t q1, int64_t q2, const T *y1,
                    const T *e0, TZ *zout, const T *rhs, cudaStream_t s) {
  TRS_DISPATCH_B(b, {
    const int64_t cb = kRowLanes<B, T> ? row_lane_blocks_of(q1 - q0, B) : cell_blocks_of(q1 - q0), lb = q2 - q1;
    if (cb + lb == 0) return;
    launch_pdl(k_ilu_bwd<B, T, TZ>, (unsigned)(cb + lb), kThreads, 0, s, F, y, q0, q1, q2, cb, y1, e0, zout, rhs);
  });
  TRS_LAUNCHED();
}

template <class T>
void launch_resid_p(int b, const MatView<T> &At, const T *atp, const T *f, const T *y, T *rp, int unit,
                    cudaStream_t s) {
  const int64_t cb = cell_blocks_of(At.g.nc), lb = long_blocks_of(At.g.n_rows - At.g.nc);
  if (cb + lb == 0) return;
  TRS_DISPATCH_B(b, launch_pdl(k_resid_p<B, T>, (unsigned)(cb + lb), kThreads, 0, s, At, atp, f, y, rp, cb, unit));
  TRS_LAUNCHED();
}

template <class T>
void launch_resid_full(int b, const MatView<T> &At, const T *f, const T *y1, const T *e0, T *r, int unit,
                       const int32_t *colour, T *x0, cudaStream_t s) {
  const int64_t cb = cell_blocks_of(At.g.nc), lb = long_blocks_of(At.g.n_rows - At.g.nc);
  if (cb + lb == 0) return;
  const Seed<T> sd{colour, x0};
  TRS_DISPATCH_B(b, launch_pdl(k_resid_full<B, T>, (unsigned)(cb + lb), kThreads, 0, s, At, f, y1, e0, r, cb, unit, sd));
  TRS_LAUNCHED();
}

template <class T>
void launch_cpr_combine(int b, int64_t n, const T *y1, const T *e0, double *z, cudaStream_t s) {
  if (!n) return;
  TRS_DISPATCH_B(b, launch_pdl(k_cpr_combine<B, T>, grid_of(n), kThreads, 0, s, n, y1, e0, z));
  TRS_LAUNCHED();
}

template <class T>
void launch_pressure_of(int b, int64_t n, const T *f, T *rp, cudaStream_t s) {
  if (!n) return;
  launch_pdl(k_pressure_of<T>, grid_of(n), kThreads, 0, s, n, b, f, rp);
  TRS_LAUNCHED();
}

template <class T>
void launch_cheb_resid_init(const ScalarOp<T> &op, const T *r, const T *e, const T *dinv, double inv_theta,
                            T *res, T *d, cudaStream_t s) {
  if (!op.n) return;
  launch_pdl(k_cheb_resid_init<T>, grid_of(op.n), kThreads, 0, s, op, r, e, dinv, static_cast<T>(inv_theta), res, d);
  TRS_LAUNCHED();
}
template <class T>
void launch_cheb_step(const ScalarOp<T> &op, const T *res_in, T *res_out, const T *d, const T *dinv, double c1,
                      double c2, T *dn, T *e, int last, cudaStream_t s) {
  if (!op.n) return;
  launch_pdl(k_cheb_step<T>, grid_of(op.n), kThreads, 0, s, op, res_in, res_out, d, dinv, static_cast<T>(c1),
                                                    static_cast<T>(c2), dn, e, last);
  TRS_LAUNCHED();
}
template <class T>
void launch_cheb_first(const ScalarOp<T> &op, const T *r, const T *dinv, double inv_theta, double c1, double c2,
                       T *res_out, T *d_out, T *dn, T *e, int last, cudaStream_t s) {
  if (!op.n) return;
  launch_pdl(k_cheb_first<T>, grid_of(op.n), kThreads, 0, s, op, r, dinv, static_cast<T>(inv_theta), static_cast<T>(c1),
                                                     static_cast<T>(c2), res_out, d_out, dn, e, last);
  TRS_LAUNCHED();
}
template <class T>
void launch_restrict_resid(const ScalarOp<T> &op, int64_t nc, const int64_t *mptr, const int32_t *midx, const T *r,
                           const T *e, T *rc, cudaStream_t s) {
  if (!nc) return;
  launch_pdl(k_restrict_resid<T>, grid_of(nc * kGroup), kThreads, 0, s, op, nc, mptr, midx, r, e, rc);
  TRS_LAUNCHED();
}
template <class T>
void launch_prolong(int64_t n, const int32_t *agg, const T *ec, T *e, cudaStream_t s) {
  if (!n) return;
  launch_pdl(k_prolong<T>, grid_of(n), kThreads, 0, s, n, agg, ec, e);
  TRS_LAUNCHED();
}
template <class T>
void launch_dense_gemv(int64_t n, const double *Minv, const T *r, T *e, cudaStream_t s) {
  if (!n) return;
  launch_pdl(k_dense_gemv<T>, (unsigned)((n + kWarps - 1) / kWarps), kThreads, 0, s, n, Minv, r, e);
  TRS_LAUNCHED();
}

// Grid of one wave: the blocks of `kernel` that fit on the device at once
// (at most cap).  The FP64-bound Gram-Schmidt kernels stride over the vector,
// so one resident wave avoids a tail wave and keeps the number of partial
// sums (and their reduction) small.  Looked up once per kernel and device.
template <class... KArgs>
unsigned resident_grid(void (*kernel)(KArgs...), unsigned cap) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void *, int>, unsigned>> cache;
  int dev = 0;
  TRS_CUDA(cudaGetDevice(&dev));
  const void *key = reinterpret_cast<const void *>(kernel);
  std::lock_guard<std::mutex> lock(mu);
  for (auto &e : cache)
    if (e.first.first == key && e.first.second == dev) return std::min(cap, e.second);
  int per_sm = 0, sms = 0;
  TRS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, 0));
  TRS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned g = (unsigned)std::max(1, per_sm * sms);
  cache.push_back({{key, dev}, g});
  return std::min(cap, g);
}

// Blocks of a staged Gram-Schmidt kernel resident per GB300 SM times the SM
// count (its shared-memory opt-in set on first use), capped at cap.
template <class... KArgs>
unsigned staged_grid(void (*kernel)(KArgs...), size_t smem, unsigned cap) {
  static std::mutex mu;
  static std::vector<std::pair<std::pair<const void *, int>, unsigned>> cache;
  int dev = 0;
  TRS_CUDA(cudaGetDevice(&dev));
  const void *key = reinterpret_cast<const void *>(kernel);
  std::lock_guard<std::mutex> lock(mu);
  for (auto &e : cache)
    if (e.first.first == key && e.first.second == dev) return std::min(cap, e.second);
  TRS_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, sms = 0;
  TRS_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, kThreads, smem));
  TRS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const unsigned g = (unsigned)std::max(1, per_sm * sms);
  cache.push_back({{key, dev}, g});
  return std::min(cap, g);
}

// The staged kernels copy whole 16-byte units: N even, V and w 16-byte aligned.
inline bool stageable(const double *V, int64_t N, const double *w) {
  return N % 2 == 0 && ((uintptr_t)V & 15u) == 0 && ((uintptr_t)w & 15u) == 0;
}

// bytes each stage expects beyond its copies (trs_test_stall_staged_copies)
std::atomic<uint32_t> g_stage_stall{0u};

template <int KM, bool UPD>
void launch_staged(const double *V, int64_t N, int K, const double *h, double *w, const RedScratch &red,
                   double *out, cudaStream_t s) {
  const size_t smem = (size_t)2 * (KM + 1) * kTE * sizeof(double);
  launch_pdl(k_cgs_staged<KM, UPD>, staged_grid(k_cgs_staged<KM, UPD>, smem, (unsigned)red.grid), kThreads, smem,
             s, V, N, K, h, w, red.partial, red.counter, out, g_stage_stall.load(std::memory_order_relaxed));
}

void launch_multidot(const double *V, int64_t N, int K, const double *w, const RedScratch &red, double *out,
                     cudaStream_t s) {
  launch_pdl(k_multidot<32>, resident_grid(k_multidot<32>, (unsigned)red.grid), kThreads, 0, s, V, N, K, w,
             red.partial, red.counter, out);
  TRS_LAUNCHED();
}
void launch_cgs_update(const double *V, int64_t N, int K, const double *h, double *w, int want_norm,
                       const RedScratch &red, double *out, cudaStream_t s) {
  launch_pdl(k_cgs_update, red.grid, kThreads, 0, s, V, N, K, h, w, want_norm, red.partial, red.counter, out);
  TRS_LAUNCHED();
}
void launch_cgs_dots(const double *V, int64_t N, int K, const double *w, const RedScratch &red, double *out,
                     cudaStream_t s) {
  const unsigned cap = (unsigned)red.grid;
  // staged up to 16 vectors; at 32 one 135 KB block per SM keeps too few
  // tiles in flight for a pass of one FMA per element (measured slower than
  // the register kernel there)
  if (stageable(V, N, w) && K + 1 <= 16) {
    double *wm = const_cast<double *>(w);   // read only (UPD = false)
    if (K + 1 <= 8) launch_staged<8, false>(V, N, K, nullptr, wm, red, out, s);
    else launch_staged<16, false>(V, N, K, nullptr, wm, red, out, s);
  } else if (K + 1 <= 8)
    launch_pdl(k_cgs_dots<8>, resident_grid(k_cgs_dots<8>, cap), kThreads, 0, s, V, N, K, w, red.partial,
               red.counter, out);
  else if (K + 1 <= 16)
    launch_pdl(k_cgs_dots<16>, resident_grid(k_cgs_dots<16>, cap), kThreads, 0, s, V, N, K, w, red.partial,
               red.counter, out);
  else if (K + 1 <= 32)
    launch_pdl(k_cgs_dots<32>, resident_grid(k_cgs_dots<32>, cap), kThreads, 0, s, V, N, K, w, red.partial,
               red.counter, out);
  else throw Error(TRS_ERR_UNSUPPORTED, "fused CGS2 supports at most 31 basis vectors");
  TRS_LAUNCHED();
}
void launch_cgs_update_dots(const double *V, int64_t N, int K, const double *h, double *w, const RedScratch &red,
                            double *out, cudaStream_t s) {
  const unsigned cap = (unsigned)red.grid;
  if (stageable(V, N, w) && K <= 32) {
    if (K <= 8) launch_staged<8, true>(V, N, K, h, w, red, out, s);
    else if (K <= 16) launch_staged<16, true>(V, N, K, h, w, red, out, s);
    else launch_staged<32, true>(V, N, K, h, w, red, out, s);
  } else if (K <= 8)
    launch_pdl(k_cgs_update_dots<8>, resident_grid(k_cgs_update_dots<8>, cap), kThreads, 0, s, V, N, K, h, w,
               red.partial, red.counter, out);
  else if (K <= 16)
    launch_pdl(k_cgs_update_dots<16>, resident_grid(k_cgs_update_dots<16>, cap), kThreads, 0, s, V, N, K, h, w,
               red.partial, red.counter, out);
  else if (K <= 32)
    launch_pdl(k_cgs_update_dots<32>, resident_grid(k_cgs_update_dots<32>, cap), kThreads, 0, s, V, N, K, h, w,
               red.partial, red.counter, out);
  else throw Error(TRS_ERR_UNSUPPORTED, "fused CGS2 supports at most 31 basis vectors");
  TRS_LAUNCHED();
}
void launch_givens(int j, int m, double *H, const double *h1, const double *h2, const double *hn2,
                   const double *wn2, double *cs, double *sn, double *g, double *hnorm_out, double *status,
                   double inv_bnorm, cudaStream_t s) {
  launch_pdl(k_givens, 1, 32, 0, s, j, m, H, h1, h2, hn2, wn2, cs, sn, g, hnorm_out, status, inv_bnorm);
  TRS_LAUNCHED();
}
void launch_lsq(int jdone, int m, const double *H, const double *g, double *y, cudaStream_t s) {
  launch_pdl(k_lsq, 1, 32, 0, s, jdone, m, H, g, y);
  TRS_LAUNCHED();
}
template <class TZ>
void launch_xupdate(const TZ *Z, int64_t N, int K, const double *y, double *x, cudaStream_t s) {
  if (!N || !K) return;
  unsigned grid = grid_of(N);
  if (grid > 152u * 16u) grid = 152u * 16u;
  launch_pdl(k_xupdate<TZ>, grid, kThreads, 0, s, Z, N, K, y, x);
  TRS_LAUNCHED();
}
template <class T>
void launch_vcycle_coarse(const CoarseHierarchy<T> &h, cudaStream_t s) {
  launch_pdl(k_vcycle_coarse<T>, 1, 1024, 0, s, h);
  TRS_LAUNCHED();
}
template void launch_vcycle_coarse<float>(const CoarseHierarchy<float> &, cudaStream_t);
template void launch_vcycle_coarse<double>(const CoarseHierarchy<double> &, cudaStream_t);


template <class TS, class TD>
void launch_cast(const TS *src, TD *dst, int64_t n, cudaStream_t s) {
  if (!n) return;
  unsigned grid = grid_of(n);
  if (grid > 152u * 16u) grid = 152u * 16u;
  launch_pdl(k_cast<TS, TD>, grid, kThreads, 0, s, src, dst, n);
  TRS_LAUNCHED();
}

void launch_bicg_start(BicgScalars *sc, const double *rr, double bnorm, double rtol, cudaStream_t s) {
  launch_pdl(k_bicg_start, 1, 1, 0, s, sc, rr, bnorm, rtol);
  TRS_LAUNCHED();
}

template <class T>
void launch_bicg_dir(int b, int64_t n, const double *r, const double *v, double *p, const BicgScalars *sc,
                     int first, const T *dinv, T *f, const int32_t *colour, T *y0, cudaStream_t s) {
  if (!n) return;
  const Seed<T> sd{colour, y0};
  TRS_DISPATCH_B(b, launch_pdl(k_bicg_dir<B, T>, grid_of(n), kThreads, 0, s, n, r, v, p, sc, first, dinv, f, sd));
  TRS_LAUNCHED();
}
template void launch_bicg_dir<double>(int, int64_t, const double *, const double *, double *, const BicgScalars *,
                                      int, const double *, double *, const int32_t *, double *, cudaStream_t);
template void launch_bicg_dir<float>(int, int64_t, const double *, const double *, double *, const BicgScalars *,
                                     int, const float *, float *, const int32_t *, float *, cudaStream_t);

int64_t bicg_spmv_blocks(const Geom &g) { return cell_blocks_of(g.nc) + long_blocks_of(g.n_rows - g.nc); }

void launch_bicg_spmv(int b, const MatView<double> &A, const double *x, double *y, const double *w, int nd,
                      double *part, unsigned int *counter, BicgScalars *sc, cudaStream_t s) {
  const int64_t cb = cell_blocks_of(A.g.nc), nb = bicg_spmv_blocks(A.g);
  if (nd == 1) {
    TRS_DISPATCH_B(b, launch_pdl(k_bicg_spmv<B, 1>, (unsigned)nb, kThreads, 0, s, A, x, y, w, cb, part, counter, sc));
  } else {
    TRS_DISPATCH_B(b, launch_pdl(k_bicg_spmv<B, 2>, (unsigned)nb, kThreads, 0, s, A, x, y, w, cb, part, counter, sc));
  }
  TRS_LAUNCHED();
}

void launch_bicg_s(int64_t N, const double *r, const double *v, double *sv, const RedScratch &red,
                   BicgScalars *sc, cudaStream_t s) {
  launch_pdl(k_bicg_s, red.grid, kThreads, 0, s, N, r, v, sv, red.partial, red.counter, sc);
  TRS_LAUNCHED();
}

void launch_bicg_xr(int64_t N, const double *ph, const double *sh, const double *sv, const double *t,
                    const double *rh, double *x, double *r, const RedScratch &red, BicgScalars *sc,
                    cudaStream_t s) {
  launch_pdl(k_bicg_xr, red.grid, kThreads, 0, s, N, ph, sh, sv, t, rh, x, r, red.partial, red.counter, sc);
  TRS_LAUNCHED();
}

#define TRS_INST_T(T)                                                                                       \
  template void launch_dscale<T>(int, int64_t, const double *, const double *, double *, const T *, T *,     \
                                 const int32_t *, T *, cudaStream_t);                                       \
  template void launch_ilu_fwd<T>(int, const IluView<T> &, const T *, T *, int64_t, int64_t, int64_t,        \
                                  cudaStream_t);                                                            \
  template void launch_ilu_bwd<T, double>(int, const IluView<T> &, T *, int64_t, int64_t, int64_t, const T *,\
                                          const T *, double *, const T *, cudaStream_t);                    \
  template void launch_resid_p<T>(int, const MatView<T> &, const T *, const T *, const T *, T *, int,      \
                                  cudaStream_t);                                                            \
  template void launch_resid_full<T>(int, const MatView<T> &, const T *, const T *, const T *, T *, int,    \
                                     const int32_t *, T *, cudaStream_t);                                   \
  template void launch_cpr_combine<T>(int, int64_t, const T *, const T *, double *, cudaStream_t);          \
  template void launch_pressure_of<T>(int, int64_t, const T *, T *, cudaStream_t);                          \
  template void launch_cheb_resid_init<T>(const ScalarOp<T> &, const T *, const T *, const T *, double, T *, \
                                          T *, cudaStream_t);                                               \
  template void launch_cheb_step<T>(const ScalarOp<T> &, const T *, T *, const T *, const T *, double,      \
                                    double, T *, T *, int, cudaStream_t);                                   \
  template void launch_cheb_first<T>(const ScalarOp<T> &, const T *, const T *, double, double, double, T *, \
                                     T *, T *, T *, int, cudaStream_t);                                     \
  template void launch_restrict_resid<T>(const ScalarOp<T> &, int64_t, const int64_t *, const int32_t *,     \
                                         const T *, const T *, T *, cudaStream_t);                          \
  template void launch_prolong<T>(int64_t, const int32_t *, const T *, T *, cudaStream_t);                  \
  template void launch_dense_gemv<T>(int64_t, const double *, const T *, T *, cudaStream_t);                \
  template void launch_xupdate<T>(const T *, int64_t, int, const double *, double *, cudaStream_t);

TRS_INST_T(double)
TRS_INST_T(float)
template void launch_ilu_bwd<float, float>(int, const IluView<float> &, float *, int64_t, int64_t, int64_t,
                                           const float *, const float *, float *, const float *, cudaStream_t);
template void launch_cast<double, float>(const double *, float *, int64_t, cudaStream_t);
template void launch_cast<float, double>(const float *, double *, int64_t, cudaStream_t);
template void launch_cast<double, double>(const double *, double *, int64_t, cudaStream_t);

}  // namespace trs

// ============================================ allocation-free residual norm
// Some callers cannot allocate device memory while they run: loops where
// cudaMalloc's implicit device-wide synchronisation is unacceptable, or
// processes whose device memory is entirely handed to their own pool
// allocator.  For them the residual and its norm run on a reduction scratch
// that lives in this file-scope array, loaded with the library and kept by
// every GPU that loads it until the process exits.  Size: the partial sums of
// at most kStaticGrid blocks (the same grid the solver uses, so results are
// identical) plus a ticket counter and the output, 778,752 bytes in all.  The
// call copies the norm to the caller's host pointer and synchronises its
// stream before returning.
namespace trs {
namespace {

constexpr int kStaticGrid = 152 * 8;
constexpr size_t kStaticCounterAt = (size_t)kStaticGrid * kRedStride;  // 256-byte aligned slot
constexpr size_t kStaticOutAt = kStaticCounterAt + 32;
constexpr size_t kStaticDoubles = kStaticOutAt + 32;

static __device__ __align__(256) double g_static_scratch[kStaticDoubles];

constexpr int kMaxDevices = 64;
std::mutex g_static_mutex;
double *g_static_addr[kMaxDevices] = {};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
double *static_scratch() {
  int dev = 0;
  TRS_CUDA(cudaGetDevice(&dev));
  TRS_REQUIRE(dev >= 0 && dev < kMaxDevices, TRS_ERR_UNSUPPORTED, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_static_mutex);
  if (!g_static_addr[dev]) {
    void *p = nullptr;
    TRS_CUDA(cudaGetSymbolAddress(&p, g_static_scratch));
    g_static_addr[dev] = static_cast<double *>(p);
  }
  return g_static_addr[dev];
}

}  // namespace

}  // namespace trs

extern "C" trs_status trs_residual_norm_noalloc(const trs_bsr *A, const double *x, const double *b, double *r,
                                                double *norm, void *stream) {
  using namespace trs;
  return guarded([&] {
    TRS_REQUIRE(A && x && b && r && norm, TRS_ERR_INVALID, "NULL argument");
    TRS_REQUIRE(x != r && b != r, TRS_ERR_INVALID, "r must not alias x or b");
    require_aligned(x, "x");
    require_aligned(b, "b");
    require_aligned(r, "r");
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = A->n * A->b;
    const int64_t grid = std::min<int64_t>(kStaticGrid, std::max<int64_t>(1, (N + kThreads - 1) / kThreads));
    TRS_REQUIRE(grid <= kStaticGrid, TRS_ERR_UNSUPPORTED, "reduction grid larger than the static scratch");
    double *base = static_scratch();
    unsigned int *counter = reinterpret_cast<unsigned int *>(base + kStaticCounterAt);
    double *out = base + kStaticOutAt;
    TRS_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned int), s));
    const MatView<double> Av = A->view();
    TRS_DISPATCH_B(A->b, k_true_residual<B><<<(unsigned)grid, kThreads, 0, s>>>(Av, x, b, r, 0, 0, base, counter,
                                                                                out));
    TRS_LAUNCHED();
    TRS_CUDA(cudaMemcpyAsync(norm, out + 1, sizeof(double), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaStreamSynchronize(s));
  });
}

extern "C" trs_status trs_test_stall_staged_copies(int32_t extra_bytes) {
  using namespace trs;
  return guarded([&] {
    TRS_REQUIRE(extra_bytes >= 0 && extra_bytes <= 65536 && extra_bytes % 16 == 0, TRS_ERR_INVALID,
                "extra_bytes must be 0..65536 and a multiple of 16");
    g_stage_stall.store((uint32_t)extra_bytes, std::memory_order_relaxed);
  });
}
