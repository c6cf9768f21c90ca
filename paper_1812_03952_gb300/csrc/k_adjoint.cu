// Adjoint kernels: transposed block SpMV (a gather, no explicit transpose),
// block transposition of values, the pattern-restricted outer product
// -lambda_i x_j^T and its chain through the harmonic transmissibility to
// theta = ln k.
#include "trs_kernels.cuh"

namespace trs {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

inline unsigned grid_of(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// y_i = alpha * sum_j (A_ji)^T x_j + beta * y_i.  For a cell row the blocks
// A_ji of its 7-point neighbours sit in the neighbour's opposite slot; blocks
// of the tail are found through the column lists tc_*.
template <int B>
__global__ void __launch_bounds__(kThreads) k_spmv_t(MatView<double> A, const int64_t *tc_ptr, const int64_t *tc_src,
                                                     const int32_t *tc_row, const double *x, double *y, double alpha,
                                                     double beta, int64_t cell_blocks) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t nc = A.g.nc;
  if (blockIdx.x < cell_blocks) {
    const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
    if (i >= nc) return;
    double acc[B] = {};
    const unsigned m = A.emask[i];
#pragma unroll
    for (int s = 0; s < kSlots; s++) {
      if (!((m >> s) & 1u)) continue;
      const int64_t j = i + A.g.off[s];
      const int so = kSlots - 1 - s;
      const double *blk = A.ell + (int64_t)so * BB * nc + j;
#pragma unroll
      for (int r = 0; r < B; r++) {
        const double xr = x[j * B + r];
#pragma unroll
        for (int c = 0; c < B; c++) acc[c] = fma(blk[(int64_t)(r * B + c) * nc], xr, acc[c]);
      }
    }
    for (int64_t t = tc_ptr[i]; t < tc_ptr[i + 1]; t++) {
      const int64_t j = tc_row[t];
      const double *blk = A.tval + tc_src[t] * BB;
#pragma unroll
      for (int r = 0; r < B; r++)
#pragma unroll
        for (int c = 0; c < B; c++) acc[c] = fma(blk[r * B + c], x[j * B + r], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < B; c++)
      y[i * B + c] = (beta == 0.0) ? alpha * acc[c] : fma(alpha, acc[c], beta * y[i * B + c]);
  } else {
    const int lane = threadIdx.x & 31;
    const int64_t i = nc + (blockIdx.x - cell_blocks) * (int64_t)kWarps + (threadIdx.x >> 5);
    if (i >= A.g.n_rows) return;
    double acc[B] = {};
    for (int64_t t = tc_ptr[i] + lane; t < tc_ptr[i + 1]; t += 32) {
      const int64_t j = tc_row[t];
      const double *blk = A.tval + tc_src[t] * BB;
#pragma unroll
      for (int r = 0; r < B; r++)
#pragma unroll
        for (int c = 0; c < B; c++) acc[c] = fma(blk[r * B + c], x[j * B + r], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < B; c++) acc[c] = warp_sum(acc[c]);
    if (lane == 0)
#pragma unroll
      for (int c = 0; c < B; c++)
        y[i * B + c] = (beta == 0.0) ? alpha * acc[c] : fma(alpha, acc[c], beta * y[i * B + c]);
  }
}

// Cell part of A^T: the block in slot s of cell i is the transpose of the
// block in the opposite slot of cell j = i + off[s] (the slots are geometric,
// so that block is always in A's ELL part).  One thread per (slot, cell):
// for a fixed element the reads and the writes are both unit-stride in i.
template <int B>
__global__ void __launch_bounds__(kThreads) k_transpose_ell(Geom g, const uint8_t *__restrict__ emask_dst,
                                                            const double *__restrict__ ell_src,
                                                            double *__restrict__ ell_dst) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t nc = g.nc;
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= nc) return;
  const int s = blockIdx.y;
  double *dst = ell_dst + (int64_t)s * BB * nc + i;
  if ((emask_dst[i] >> s) & 1u) {
    const double *src = ell_src + (int64_t)(kSlots - 1 - s) * BB * nc + (i + g.off[s]);
#pragma unroll
    for (int r = 0; r < B; r++)
#pragma unroll
      for (int c = 0; c < B; c++) dst[(int64_t)(r * B + c) * nc] = src[(int64_t)(c * B + r) * nc];
  } else {
#pragma unroll
    for (int e = 0; e < BB; e++) dst[(int64_t)e * nc] = 0.0;
  }
}

// Tail part of A^T: entry t of the tail is canonical block tq[t]; its source
// is canonical block src_canon[tq[t]] of A, wherever A keeps it.
__global__ void __launch_bounds__(kThreads) k_transpose_tail(int b, int64_t ntail, const int64_t *__restrict__ tq,
                                                             const int64_t *__restrict__ src_canon,
                                                             const int64_t *__restrict__ map_src,
                                                             const double *__restrict__ ell_src,
                                                             const double *__restrict__ tval_src, int64_t nc,
                                                             double *__restrict__ tval_dst) {
  pdl_enter();
  const int bb = b * b;
  const int64_t idx = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (idx >= ntail * bb) return;
  const int64_t t = idx / bb;
  const int e = (int)(idx % bb), r = e / b, c = e % b;
  const int64_t ls = map_src[src_canon[tq[t]]];
  const int es = c * b + r;  // transposed element
  tval_dst[idx] = ls < kSlots * nc ? ell_src[((ls / nc) * bb + es) * nc + ls % nc]
                                   : tval_src[(ls - kSlots * nc) * bb + es];
}

template <int B>
__global__ void k_outer_product(int64_t nnzb, const int32_t *urow, const int32_t *ucol, const double *lambda,
                                const double *x, double *dA) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t idx = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (idx >= nnzb * BB) return;
  const int64_t p = idx / BB;
  const int e = (int)(idx % BB), r = e / B, c = e % B;
  dA[idx] = -(lambda[(int64_t)urow[p] * B + r] * x[(int64_t)ucol[p] * B + c]);
}

__device__ __forceinline__ double chain_face_T(double ki, double kj, int vertical, double kvkh, double c_t) {
  if (vertical) { ki = kvkh * ki; kj = kvkh * kj; }
  const double den = ki + kj;
  if (den == 0.0) return 0.0;
  return c_t * (((2.0 * ki) * kj) / den);
}

// dL/dtheta_i = sum over the faces f of i of dL/dT_f * T_f * k_j / (k_i + k_j),
// dL/dT_f = lambda_i^T M_if (x_j - x_i) + lambda_j^T M_jf' (x_i - x_j): the
// contraction of -lambda x^T with dA/dT_f (A_ij = -T M_if, A_ii += T M_if,
// and the same from cell j), computed from both sides without atomics.
template <int B>
__global__ void k_chain_theta(Geom g, const uint8_t *emask, const double *perm, int is_log, double kvkh,
                              double c_t, const double *M, const double *lambda, const double *x,
                              double *dtheta) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= g.nc) return;
  const double ki = is_log ? exp(perm[i]) : perm[i];
  const unsigned m = emask[i];
  double li[B], xi[B];
#pragma unroll
  for (int r = 0; r < B; r++) { li[r] = lambda[i * B + r]; xi[r] = x[i * B + r]; }
  double acc = 0.0;
  for (int d = 0; d < 6; d++) {
    const int s = d < 3 ? d : d + 1;
    if (!((m >> s) & 1u)) continue;
    const int64_t j = i + g.off[s];
    const double kj = is_log ? exp(perm[j]) : perm[j];
    if (ki + kj == 0.0) continue;
    const double T = chain_face_T(ki, kj, d == 0 || d == 5, kvkh, c_t);
    const double *Mi = M + (i * 6 + d) * BB;
    const double *Mj = M + (j * 6 + (5 - d)) * BB;
    double dLdT = 0.0;
#pragma unroll
    for (int r = 0; r < B; r++) {
      const double lj = lambda[j * B + r];
#pragma unroll
      for (int c = 0; c < B; c++) {
        const double dx = x[j * B + c] - xi[c];
        dLdT = fma(li[r] * Mi[r * B + c], dx, dLdT);
        dLdT = fma(-lj * Mj[r * B + c], dx, dLdT);
      }
    }
    acc = fma(dLdT, T * (kj / (ki + kj)), acc);
  }
  dtheta[i] = acc;
}

}  // namespace

void launch_spmv_t(int b, const trs_bsr &A, const double *x, double *y, double alpha, double beta,
                   cudaStream_t s) {
  const int64_t cb = (A.g.nc + kThreads - 1) / kThreads;
  const int64_t lb = (A.g.n_rows - A.g.nc + kWarps - 1) / kWarps;
  if (cb + lb == 0) return;
  TRS_DISPATCH_B(b, launch_pdl(k_spmv_t<B>, (unsigned)(cb + lb), kThreads, 0, s, A.view(), A.tc_ptr.p, A.tc_src.p,
                                                                         A.tc_row.p, x, y, alpha, beta, cb));
  TRS_LAUNCHED();
}

void launch_transpose_values(const trs_bsr &A, trs_bsr &AT, cudaStream_t s) {
  const int64_t nc = AT.g.nc;
  if (nc) {
    TRS_DISPATCH_B(A.b, launch_pdl(k_transpose_ell<B>, dim3(grid_of(nc), kSlots), dim3(kThreads), 0, s, AT.g,
                                   (const uint8_t *)AT.emask.p, (const double *)A.ell.p, AT.ell.p));
  }
  if (AT.ntail) {
    const int bb = A.b * A.b;
    launch_pdl(k_transpose_tail, grid_of(AT.ntail * bb), kThreads, 0, s, A.b, AT.ntail, (const int64_t *)AT.ttail.p,
               (const int64_t *)AT.tsrc.p, (const int64_t *)A.map.p, (const double *)A.ell.p,
               (const double *)A.tval.p, A.g.nc, AT.tval.p);
  }
  TRS_LAUNCHED();
}

void launch_outer_product(int b, const trs_bsr &A, const double *lambda, const double *x, double *dA,
                          cudaStream_t s) {
  if (!A.nnzb) return;
  TRS_DISPATCH_B(b, launch_pdl(k_outer_product<B>, grid_of(A.nnzb * B * B), kThreads, 0, s, A.nnzb, A.urow.p, A.ucol.p,
                                                                                    lambda, x, dA));
  TRS_LAUNCHED();
}

void launch_chain_theta(int b, const trs_bsr &A, const double *perm, int perm_is_log, double kvkh, double c_t,
                        const double *M, const double *lambda, const double *x, double *dtheta, cudaStream_t s) {
  if (!A.g.nc) return;
  TRS_DISPATCH_B(b, launch_pdl(k_chain_theta<B>, grid_of(A.g.nc), kThreads, 0, s, A.g, A.emask.p, perm, perm_is_log,
                                                                          kvkh, c_t, M, lambda, x, dtheta));
  TRS_LAUNCHED();
}

}  // namespace trs
