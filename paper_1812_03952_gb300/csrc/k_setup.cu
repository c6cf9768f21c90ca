// Setup-phase kernels: value layout, synthetic assembly, ABF/GJE decoupling,
// pressure extraction, aggregation AMG setup, multicolouring and block ILU(0)
// factorisation.
//
// This translation unit is compiled with -fmad=false: every a*b+c is a
// rounded product followed by a rounded sum, divisions and square roots are
// IEEE, and every sum runs in the order stated next to it, so the integer
// decisions taken from these values (strong connections, MIS-2, aggregates,
// colours) are reproducible bit for bit by any implementation of the same
// definitions.
#include <algorithm>

#include "trs_kernels.cuh"

namespace trs {

namespace {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;

inline unsigned grid_of(int64_t n) { return (unsigned)((n + kThreads - 1) / kThreads); }

// murmur3 32-bit finaliser (Appleby, MurmurHash3 "fmix32"): a reproducible
// pseudo-random priority for every node.
__device__ __forceinline__ uint32_t fmix32(uint32_t h) {
  h ^= h >> 16;
  h *= 0x85ebca6bu;
  h ^= h >> 13;
  h *= 0xc2b2ae35u;
  h ^= h >> 16;
  return h;
}
__device__ __forceinline__ uint64_t node_key(int64_t i, uint32_t seed) {
  return ((uint64_t)fmix32((uint32_t)i ^ seed) << 32) | (uint64_t)(uint32_t)i;
}

// ------------------------------------------------------------------ scan
constexpr int kScanItems = 16;
constexpr int kScanChunk = kThreads * kScanItems;

__global__ void k_scan_reduce(const int64_t *in, int64_t n, int64_t *bsum) {
  pdl_enter();
  __shared__ int64_t sm[kWarps];
  int64_t base = (int64_t)blockIdx.x * kScanChunk, s = 0;
  for (int k = threadIdx.x; k < kScanChunk; k += kThreads) {
    int64_t i = base + k;
    if (i < n) s += in[i];
  }
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    int64_t t = 0;
    for (int w = 0; w < kWarps; w++) t += sm[w];
    bsum[blockIdx.x] = t;
  }
}

__global__ void k_scan_bsums(int64_t *bsum, int64_t nb, int64_t *total) {
  pdl_enter();
  if (threadIdx.x != 0) return;
  int64_t run = 0;
  for (int64_t b = 0; b < nb; b++) {
    int64_t v = bsum[b];
    bsum[b] = run;
    run += v;
  }
  if (total) *total = run;
}

__global__ void k_scan_apply(const int64_t *in, int64_t *out, int64_t n, const int64_t *bsum) {
  pdl_enter();
  __shared__ int64_t wsum[kWarps];
  const int64_t base = (int64_t)blockIdx.x * kScanChunk + (int64_t)threadIdx.x * kScanItems;
  int64_t v[kScanItems];
  int64_t s = 0;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + k;
    v[k] = i < n ? in[i] : 0;
    s += v[k];
  }
  // exclusive scan of per-thread sums
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int64_t incl = s;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t t = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += t;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int64_t woff = 0;
  for (int w = 0; w < warp; w++) woff += wsum[w];
  int64_t run = bsum[blockIdx.x] + woff + incl - s;
#pragma unroll
  for (int k = 0; k < kScanItems; k++) {
    int64_t i = base + k;
    if (i < n) out[i] = run;
    run += v[k];
  }
}

// ------------------------------------------------------- value layout
__global__ void k_scatter_values(int64_t nnzb, int bb, const int64_t *map, const double *uval, int64_t nc,
                                 double *ell, double *tval) {
  pdl_enter();
  const int64_t idx = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (idx >= nnzb * bb) return;
  const int64_t p = idx / bb, e = idx % bb, loc = map[p];
  if (loc < kSlots * nc) {
    const int64_t s = loc / nc, row = loc % nc;
    ell[(s * bb + e) * nc + row] = uval[idx];
  } else {
    tval[(loc - kSlots * nc) * bb + e] = uval[idx];
  }
}

__global__ void k_gather_values(int64_t nnzb, int bb, const int64_t *map, const double *ell,
                                const double *tval, int64_t nc, int aos, double *uval) {
  pdl_enter();
  const int64_t idx = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (idx >= nnzb * bb) return;
  const int64_t p = idx / bb, e = idx % bb, loc = map[p];
  if (loc < kSlots * nc) {
    const int64_t s = loc / nc, row = loc % nc;
    uval[idx] = aos ? ell[(s * nc + row) * bb + e] : ell[(s * bb + e) * nc + row];
  } else {
    uval[idx] = tval[(loc - kSlots * nc) * bb + e];
  }
}

// Reference to one stored block of the factor: base pointer and stride.
template <class T>
struct BRef {
  T *p;
  int64_t stride;
};

// Blocks with unit stride start at multiples of bb elements of a cudaMalloc
// allocation, so they take 128-bit accesses when bb * sizeof(T) allows.
template <int B, class T>
__device__ __forceinline__ void bload(BRef<T> r, T (&v)[B * B]) {
  constexpr int BB = B * B;
  if constexpr (sizeof(T) == 4 && BB % 4 == 0) {
    if (r.stride == 1) {
#pragma unroll
      for (int k = 0; k < BB / 4; k++) {
        const float4 t = reinterpret_cast<const float4 *>(r.p)[k];
        v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
      }
      return;
    }
  } else if constexpr (sizeof(T) == 8 && BB % 2 == 0) {
    if (r.stride == 1) {
#pragma unroll
      for (int k = 0; k < BB / 2; k++) {
        const double2 t = reinterpret_cast<const double2 *>(r.p)[k];
        v[2 * k] = t.x; v[2 * k + 1] = t.y;
      }
      return;
    }
  }
#pragma unroll
  for (int e = 0; e < BB; e++) v[e] = r.p[e * r.stride];
}
template <int B, class T>
__device__ __forceinline__ void bstore(BRef<T> r, const T (&v)[B * B]) {
  constexpr int BB = B * B;
  if constexpr (sizeof(T) == 4 && BB % 4 == 0) {
    if (r.stride == 1) {
#pragma unroll
      for (int k = 0; k < BB / 4; k++)
        reinterpret_cast<float4 *>(r.p)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
      return;
    }
  } else if constexpr (sizeof(T) == 8 && BB % 2 == 0) {
    if (r.stride == 1) {
#pragma unroll
      for (int k = 0; k < BB / 2; k++) reinterpret_cast<double2 *>(r.p)[k] = make_double2(v[2 * k], v[2 * k + 1]);
      return;
    }
  }
#pragma unroll
  for (int e = 0; e < BB; e++) r.p[e * r.stride] = v[e];
}

// ------------------------------------------------------------ assembly
// Harmonic-mean geometric transmissibility of one face (unit cell, unit
// face), zero when both permeabilities vanish.
__device__ __forceinline__ double face_T(double ki, double kj, int vertical, double kvkh, double c_t) {
  if (vertical) { ki = kvkh * ki; kj = kvkh * kj; }
  const double den = ki + kj;
  if (den == 0.0) return 0.0;
  const double num = (2.0 * ki) * kj;
  return c_t * (num / den);
}

__device__ __forceinline__ double perm_of(const double *perm, int is_log, int64_t i) {
  return is_log ? exp(perm[i]) : perm[i];
}

template <int B>
__global__ void k_assemble_cells(Geom g, const uint8_t *emask, double *ell, double *tval, const double *perm,
                                 int is_log, double kvkh, double c_t, const double *M, const double *acc,
                                 const int64_t *cperf_ptr, const int64_t *cperf_idx, const int64_t *perf_cw,
                                 const double *wi, const double *lam) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t c = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (c >= g.nc) return;
  const int64_t nc = g.nc;
  double dg[BB];
  bload<B, double>(BRef<double>{const_cast<double *>(acc) + c * BB, 1}, dg);
  const double kc = perm_of(perm, is_log, c);
  const unsigned m = emask[c];
  for (int d = 0; d < 6; d++) {
    const int s = d < 3 ? d : d + 1;
    if (!((m >> s) & 1u)) continue;
    const int64_t j = c + g.off[s];
    const double T = face_T(kc, perm_of(perm, is_log, j), d == 0 || d == 5, kvkh, c_t);
    double Mij[BB];
    bload<B, double>(BRef<double>{const_cast<double *>(M) + (c * 6 + d) * BB, 1}, Mij);
#pragma unroll
    for (int e = 0; e < BB; e++) {
      const double flux = T * Mij[e];
      ell[((int64_t)s * BB + e) * nc + c] = -flux;
      dg[e] = dg[e] + flux;
    }
  }
  for (int64_t t = cperf_ptr[c]; t < cperf_ptr[c + 1]; t++) {
    const int64_t mm = cperf_idx[t];
    double *blk = tval + perf_cw[mm] * BB;
#pragma unroll
    for (int r = 0; r < B; r++) {
      const double q = wi[mm] * lam[mm * B + r];
      dg[r * B] = dg[r * B] + q;
      blk[r * B] = -q;
    }
  }
#pragma unroll
  for (int e = 0; e < BB; e++) ell[((int64_t)kSelf * BB + e) * nc + c] = dg[e];
}

template <int B>
__global__ void k_assemble_wells(int nw, double *tval, const int64_t *wperf_ptr, const int64_t *wperf_idx,
                                 const int64_t *perf_wc, const int64_t *wdiag, const double *wi,
                                 const double *lam) {
  pdl_enter();
  constexpr int BB = B * B;
  const int w = blockIdx.x * kThreads + threadIdx.x;
  if (w >= nw) return;
  double sum = 0.0;
  for (int64_t t = wperf_ptr[w]; t < wperf_ptr[w + 1]; t++) {
    const int64_t mm = wperf_idx[t];
    double Lam = 0.0;
#pragma unroll
    for (int r = 0; r < B; r++) Lam = Lam + lam[mm * B + r];
    const double q = wi[mm] * Lam;
    sum = sum + q;
    tval[perf_wc[mm] * BB] = -q;
  }
  double *dgb = tval + wdiag[w] * BB;
  dgb[0] = sum;
#pragma unroll
  for (int s = 1; s < B; s++) dgb[s * B + s] = 1.0;
}

template <int B>
__global__ void k_scale_diag(Geom g, double *ell, double *tval, const int64_t *tdiag, const double *sc) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= g.n_rows) return;
  const double f = sc[i];
  if (i < g.nc) {
#pragma unroll
    for (int e = 0; e < BB; e++) {
      double *p = ell + ((int64_t)kSelf * BB + e) * g.nc + i;
      *p = *p * f;
    }
  } else {
    double *p = tval + tdiag[i - g.nc] * BB;
#pragma unroll
    for (int e = 0; e < BB; e++) p[e] = p[e] * f;
  }
}

// ------------------------------------------------------------ decoupling
// Gauss-Jordan inversion with row pivoting (GJE of Sec. "Decoupling
// Methods"): pivot = first row of largest |a| in the column at or below the
// diagonal; pivot row scaled by the reciprocal of the pivot (one division
// per column); its multiple a(r,c) subtracted from every other row.
template <int B, class T = double>
__device__ bool gj_inverse(const T (&D)[B * B], T (&inv)[B * B]) {
  T a[B * B];
#pragma unroll
  for (int e = 0; e < B * B; e++) { a[e] = D[e]; inv[e] = T(0); }
#pragma unroll
  for (int r = 0; r < B; r++) inv[r * B + r] = T(1);
#pragma unroll
  for (int c = 0; c < B; c++) {
    int p = c;
    T best = fabs(a[c * B + c]);
#pragma unroll
    for (int r = c + 1; r < B; r++) {
      const T v = fabs(a[r * B + c]);
      if (v > best) { best = v; p = r; }
    }
    if (best == 0.0 || !isfinite(best)) return false;
#pragma unroll
    for (int r = c + 1; r < B; r++) {
      if (r == p) {
#pragma unroll
        for (int s = 0; s < B; s++) {
          T t = a[c * B + s]; a[c * B + s] = a[r * B + s]; a[r * B + s] = t;
          t = inv[c * B + s]; inv[c * B + s] = inv[r * B + s]; inv[r * B + s] = t;
        }
      }
    }
    const T rpiv = T(1) / a[c * B + c];
#pragma unroll
    for (int s = 0; s < B; s++) {
      a[c * B + s] = a[c * B + s] * rpiv;
      inv[c * B + s] = inv[c * B + s] * rpiv;
    }
#pragma unroll
    for (int r = 0; r < B; r++) {
      if (r == c) continue;
      const T f = a[r * B + c];
#pragma unroll
      for (int s = 0; s < B; s++) {
        a[r * B + s] = a[r * B + s] - f * a[c * B + s];
        inv[r * B + s] = inv[r * B + s] - f * inv[c * B + s];
      }
    }
  }
  return true;
}

// C = A * Bm (b x b), inner index ascending, first product then running sums
template <int B, class T = double>
__device__ __forceinline__ void bmul(const T (&A)[B * B], const T (&Bm)[B * B], T (&C)[B * B]) {
#pragma unroll
  for (int r = 0; r < B; r++)
#pragma unroll
    for (int s = 0; s < B; s++) {
      T acc = A[r * B] * Bm[s];
#pragma unroll
      for (int t = 1; t < B; t++) acc = acc + A[r * B + t] * Bm[t * B + s];
      C[r * B + s] = acc;
    }
}

// Left factor D_i^-1 of block row i (Sec. "Decoupling Methods"), by mode:
// ABF: A_ii^-1 (Gauss-Jordan with partial pivoting); NONE: I; FRS: R (ones
// in the first row and on the diagonal, adding every row into the pressure
// row); FRS+ABF: (R A_ii)^-1 R, with Ai = (R A_ii)^-1 kept for the blocks.
template <int B>
__device__ __forceinline__ void frs_matrix(double (&R)[B * B]) {
#pragma unroll
  for (int r = 0; r < B; r++)
#pragma unroll
    for (int c = 0; c < B; c++) R[r * B + c] = (r == 0 || r == c) ? 1.0 : 0.0;
}

// The factor applied to the blocks of the row, Ai (ABF: A_ii^-1; FRS+ABF:
// (R A_ii)^-1, the blocks then pre-multiplied by R; NONE: I; FRS: R), and the
// stored D_i^-1 (Ai, or Ai R for FRS+ABF).  D is replaced by R D for FRS+ABF.
template <int B>
__device__ bool decoupling_factor(int mode, double (&D)[B * B], double (&Ai)[B * B], double (&Dm)[B * B]) {
  constexpr int BB = B * B;
  if (mode == TRS_DEC_NONE) {
#pragma unroll
    for (int e = 0; e < BB; e++) Ai[e] = Dm[e] = (e % (B + 1) == 0) ? 1.0 : 0.0;
    return true;
  }
  if (mode == TRS_DEC_FRS) {
    frs_matrix<B>(Ai);
#pragma unroll
    for (int e = 0; e < BB; e++) Dm[e] = Ai[e];
    return true;
  }
  double R[BB];
  if (mode == TRS_DEC_FRS_ABF) {
    double T[BB];
    frs_matrix<B>(R);
    bmul<B>(R, D, T);
#pragma unroll
    for (int e = 0; e < BB; e++) D[e] = T[e];
  }
  if (!gj_inverse<B>(D, Ai)) return false;
  if (mode == TRS_DEC_FRS_ABF) {
    bmul<B>(Ai, R, Dm);
  } else {
#pragma unroll
    for (int e = 0; e < BB; e++) Dm[e] = Ai[e];
  }
  return true;
}

// Ã_ij = D_i^-1 A_ij; for FRS+ABF in the order of the two stages, Ai (R A_ij).
template <int B>
__device__ __forceinline__ void decouple_block(int mode, const double (&Ai)[B * B], double (&blk)[B * B],
                                               double (&out)[B * B]) {
  if (mode == TRS_DEC_FRS_ABF) {
    double R[B * B], Rb[B * B];
    frs_matrix<B>(R);
    bmul<B>(R, blk, Rb);
#pragma unroll
    for (int e = 0; e < B * B; e++) blk[e] = Rb[e];
  }
  bmul<B>(Ai, blk, out);
}

__device__ __forceinline__ bool unit_diagonal(int mode) { return mode == TRS_DEC_ABF || mode == TRS_DEC_FRS_ABF; }

// Decoupling of one block row per thread: D_i^-1 ([bb][n]), Ã = D^-1 A in
// the ELL/tail layout of A (diagonal exactly I for ABF and FRS+ABF), and
// the pressure entries (Ã_ij)_00.
template <int B>
__global__ void k_decouple(MatView<double> A, const int64_t *tdiag, int mode, double *at_ell, double *at_p,
                           double *at_tval, double *dinv, double *ap_ell, double *ap_tval, int *err) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t nc = A.g.nc, n = A.g.n_rows;
  if (i >= n) return;
  double D[BB], Dm[BB], Ai[BB], blk[BB], out[BB];
  const bool cell = i < nc;
  const bool unit = unit_diagonal(mode);
  const int64_t dtail = cell ? -1 : tdiag[i - nc];
  if (cell) {
#pragma unroll
    for (int e = 0; e < BB; e++) D[e] = A.ell[((int64_t)kSelf * BB + e) * nc + i];
  } else {
#pragma unroll
    for (int e = 0; e < BB; e++) D[e] = A.tval[dtail * BB + e];
  }
  if (!decoupling_factor<B>(mode, D, Ai, Dm)) {
    atomicExch(err, 1);
    return;
  }
#pragma unroll
  for (int e = 0; e < BB; e++) dinv[(int64_t)e * n + i] = Dm[e];
  if (cell) {
    const unsigned m = A.emask[i];
    for (int s = 0; s < kSlots; s++) {
      if (!((m >> s) & 1u)) continue;
      if (s == kSelf && unit) {
#pragma unroll
        for (int e = 0; e < BB; e++) at_ell[((int64_t)s * nc + i) * BB + e] = (e % (B + 1) == 0) ? 1.0 : 0.0;
#pragma unroll
        for (int c = 0; c < B; c++) at_p[((int64_t)s * B + c) * nc + i] = c == 0 ? 1.0 : 0.0;
        ap_ell[(int64_t)s * nc + i] = 1.0;
        continue;
      }
#pragma unroll
      for (int e = 0; e < BB; e++) blk[e] = A.ell[((int64_t)s * BB + e) * nc + i];
      decouple_block<B>(mode, Ai, blk, out);
      bstore<B, double>(BRef<double>{at_ell + ((int64_t)s * nc + i) * BB, 1}, out);
#pragma unroll
      for (int c = 0; c < B; c++) at_p[((int64_t)s * B + c) * nc + i] = out[c];
      ap_ell[(int64_t)s * nc + i] = out[0];
    }
  }
  for (int64_t t = A.tptr[i]; t < A.tptr[i + 1]; t++) {
    if (t == dtail && unit) {
#pragma unroll
      for (int e = 0; e < BB; e++) at_tval[t * BB + e] = (e % (B + 1) == 0) ? 1.0 : 0.0;
      ap_tval[t] = 1.0;
      continue;
    }
#pragma unroll
    for (int e = 0; e < BB; e++) blk[e] = A.tval[t * BB + e];
    decouple_block<B>(mode, Ai, blk, out);
#pragma unroll
    for (int e = 0; e < BB; e++) at_tval[t * BB + e] = out[e];
    ap_tval[t] = out[0];
  }
}

// The same decoupling for the FP32 preconditioner: D_i^-1 and the pressure
// entries (Ã_ij)_00 are formed in FP64 exactly as above (they decide the
// aggregates); the blocks Ã_ij and D_i^-1 are stored in FP32, the product
// taken in FP32 (for FRS+ABF: Ai in FP32 times R A_ij formed in FP64).
template <int B>
__global__ void k_decouple_mixed(MatView<double> A, const int64_t *tdiag, int mode, float *at_ell, float *at_p,
                                 float *at_tval, float *dinv, double *ap_ell, double *ap_tval, int *err) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t nc = A.g.nc, n = A.g.n_rows;
  if (i >= n) return;
  double D[BB], Dm[BB], Ai[BB], L[BB], blk[BB];
  float Lf[BB], bf[BB], of[BB];
  const bool cell = i < nc;
  const bool unit = unit_diagonal(mode);
  const bool two_stage = mode == TRS_DEC_FRS_ABF;
  const int64_t dtail = cell ? -1 : tdiag[i - nc];
  if (cell) {
#pragma unroll
    for (int e = 0; e < BB; e++) D[e] = A.ell[((int64_t)kSelf * BB + e) * nc + i];
  } else {
#pragma unroll
    for (int e = 0; e < BB; e++) D[e] = A.tval[dtail * BB + e];
  }
  if (!decoupling_factor<B>(mode, D, Ai, Dm)) {
    atomicExch(err, 1);
    return;
  }
#pragma unroll
  for (int e = 0; e < BB; e++) {
    dinv[(int64_t)e * n + i] = (float)Dm[e];
    L[e] = Ai[e];
    Lf[e] = (float)L[e];
  }
  // (Ã_ij)_00 in FP64 (first product, then a running sum over the inner
  // index) and the FP32 block
  auto one = [&](float *dst, int64_t dstride, double *pdst) {
    double src[BB];
    if (two_stage) {
      double R[BB];
      frs_matrix<B>(R);
      bmul<B>(R, blk, src);
    } else {
#pragma unroll
      for (int e = 0; e < BB; e++) src[e] = blk[e];
    }
    double acc = L[0] * src[0];
#pragma unroll
    for (int t = 1; t < B; t++) acc = acc + L[t] * src[t * B];
    *pdst = acc;
#pragma unroll
    for (int e = 0; e < BB; e++) bf[e] = (float)src[e];
    bmul<B, float>(Lf, bf, of);
    bstore<B, float>(BRef<float>{dst, dstride}, of);
  };
  if (cell) {
    const unsigned m = A.emask[i];
    for (int s = 0; s < kSlots; s++) {
      if (!((m >> s) & 1u)) continue;
      if (s == kSelf && unit) {
#pragma unroll
        for (int e = 0; e < BB; e++) at_ell[((int64_t)s * nc + i) * BB + e] = (e % (B + 1) == 0) ? 1.f : 0.f;
#pragma unroll
        for (int c = 0; c < B; c++) at_p[((int64_t)s * B + c) * nc + i] = c == 0 ? 1.f : 0.f;
        ap_ell[(int64_t)s * nc + i] = 1.0;
        continue;
      }
#pragma unroll
      for (int e = 0; e < BB; e++) blk[e] = A.ell[((int64_t)s * BB + e) * nc + i];
      one(at_ell + ((int64_t)s * nc + i) * BB, 1, ap_ell + (int64_t)s * nc + i);
#pragma unroll
      for (int c = 0; c < B; c++) at_p[((int64_t)s * B + c) * nc + i] = of[c];
    }
  }
  for (int64_t t = A.tptr[i]; t < A.tptr[i + 1]; t++) {
    if (t == dtail && unit) {
#pragma unroll
      for (int e = 0; e < BB; e++) at_tval[t * BB + e] = (e % (B + 1) == 0) ? 1.f : 0.f;
      ap_tval[t] = 1.0;
      continue;
    }
#pragma unroll
    for (int e = 0; e < BB; e++) blk[e] = A.tval[t * BB + e];
    one(at_tval + t * BB, 1, ap_tval + t);
  }
}

// ------------------------------------------------------- pressure CSR
__global__ void k_ap_rowlen(Geom g, const uint8_t *emask, const int64_t *tptr, int64_t *len) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= g.n_rows) return;
  int64_t l = tptr[i + 1] - tptr[i];
  if (i < g.nc) l += __popc((unsigned)emask[i] & ~kTailBit);
  len[i] = l;
}

// merge of the implicit ELL columns and the (sorted) tail columns
__global__ void k_ap_fill(Geom g, const uint8_t *emask, const int64_t *tptr, const int32_t *tcol,
                          const double *ap_ell, const double *ap_tval, const int64_t *rp, int32_t *col,
                          double *val) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= g.n_rows) return;
  int64_t q = rp[i], t = tptr[i];
  const int64_t te = tptr[i + 1];
  if (i < g.nc) {
    const unsigned m = emask[i];
    for (int s = 0; s < kSlots; s++) {
      if (!((m >> s) & 1u)) continue;
      const int64_t j = i + g.off[s];
      while (t < te && tcol[t] < j) { col[q] = tcol[t]; val[q] = ap_tval[t]; q++; t++; }
      col[q] = (int32_t)j;
      val[q] = ap_ell[(int64_t)s * g.nc + i];
      q++;
    }
  }
  while (t < te) { col[q] = tcol[t]; val[q] = ap_tval[t]; q++; t++; }
}

__device__ __forceinline__ int64_t bsearch_col(const int64_t *rp, const int32_t *col, int64_t i, int64_t j) {
  int64_t lo = rp[i], hi = rp[i + 1] - 1;
  while (lo <= hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    const int64_t c = col[mid];
    if (c == j) return mid;
    if (c < j) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

__global__ void k_diag_pos(int64_t n, const int64_t *rp, const int32_t *col, const double *val, int64_t *dpos,
                           double *dval) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  const int64_t d = bsearch_col(rp, col, i, i);
  dpos[i] = d;
  dval[i] = d < 0 ? 0.0 : val[d];
}

// ------------------------------------------------------------- strength
// j != i is strong if s = max(|a_ij|, |a_ji|) > 0 and s >= theta*sqrt(|a_ii a_jj|).
// Eight lanes per row, each lane a share of the row's entries, so that the
// searches for a_ji of one row are in flight together; dval holds a_ii.
constexpr int kStrengthLanes = 8;

__global__ void k_strength(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                           const double *dval, double theta, uint8_t *sflag, int32_t *sdeg) {
  pdl_enter();
  const int64_t gid = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  const int64_t i = gid / kStrengthLanes;
  const int sub = (int)(gid % kStrengthLanes);
  int32_t deg = 0;
  if (i < n) {
    const double aii = dval[i];
    const int64_t e = rp[i + 1];
    for (int64_t p = rp[i] + sub; p < e; p += kStrengthLanes) {
      const int64_t j = col[p];
      uint8_t f = 0;
      if (j != i) {
        const double ajj = dval[j];
        const int64_t pt = bsearch_col(rp, col, j, i);
        const double aij = fabs(val[p]), aji = pt < 0 ? 0.0 : fabs(val[pt]);
        const double sv = aij > aji ? aij : aji;
        const double thr = theta * sqrt(fabs(aii * ajj));
        f = (sv > 0.0 && sv >= thr) ? 1 : 0;
      }
      sflag[p] = f;
      deg += f;
    }
  }
#pragma unroll
  for (int o = kStrengthLanes / 2; o > 0; o >>= 1) deg += __shfl_xor_sync(0xffffffffu, deg, o);
  if (i < n && sub == 0) sdeg[i] = deg;
}

// ----------------------------------------------------------------- MIS-2
enum : int8_t { kOut = 0, kUndecided = 1, kIn = 2 };

__global__ void k_mis2_init(int64_t n, const int32_t *sdeg, int8_t *state) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  state[i] = sdeg[i] > 0 ? kUndecided : kOut;
}

// The tuple (state, key) with key = fmix32(i ^ seed) << 32 | i, packed into
// one word as state << 62 | fmix32(i ^ seed) << 30 | i (i < 2^30): word order
// is the tuple order, so one 64-bit maximum replaces the tuple comparison.
__device__ __forceinline__ uint64_t mis2_word(int8_t state, int64_t i, uint32_t seed) {
  return ((uint64_t)(uint8_t)state << 62) | ((uint64_t)fmix32((uint32_t)i ^ seed) << 30) | (uint64_t)i;
}

// The two max-propagation sweeps of a round: the first forms
// out_i = max over {i} U strong(i) of the packed tuples of the states, the
// second (mis2_sweep_row_w) the same maximum over the first sweep's words.
// Entries are read eight at a time so that their gathers are in flight
// together (the maximum does not depend on order).
__device__ __forceinline__ uint64_t mis2_sweep_row_w(int64_t i, const int64_t *rp, const int32_t *col,
                                                     const uint8_t *sflag, const uint64_t *w1) {
  uint64_t best = w1[i];
  const int64_t e = rp[i + 1];
  for (int64_t p0 = rp[i]; p0 < e; p0 += 8) {
    int32_t jj[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const int64_t p = p0 + u;
      jj[u] = (p < e && sflag[p]) ? col[p] : -1;
    }
#pragma unroll
    for (int u = 0; u < 8; u++) {
      if (jj[u] < 0) continue;
      const uint64_t w = w1[jj[u]];
      best = w > best ? w : best;
    }
  }
  return best;
}

__global__ void k_mis2_sweep(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *sflag,
                             const int8_t *state, uint32_t seed, uint64_t *out_w) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  uint64_t best = mis2_word(state[i], i, seed);
  const int64_t e = rp[i + 1];
  for (int64_t p0 = rp[i]; p0 < e; p0 += 8) {
    int32_t jj[8];
#pragma unroll
    for (int u = 0; u < 8; u++) {
      const int64_t p = p0 + u;
      jj[u] = (p < e && sflag[p]) ? col[p] : -1;
    }
#pragma unroll
    for (int u = 0; u < 8; u++) {
      if (jj[u] < 0) continue;
      const uint64_t w = mis2_word(state[jj[u]], jj[u], seed);
      best = w > best ? w : best;
    }
  }
  out_w[i] = best;
}

// The second sweep fused with the decision: row i's distance-2 maximum is
// formed from the first sweep's words (which no state write of this kernel
// touches) and decides row i at once; the undecided rows are counted.
__global__ void k_mis2_sweep_decide(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *sflag,
                                    int8_t *state, const uint64_t *w1, uint32_t seed,
                                    unsigned long long *undecided) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  if (state[i] != kUndecided) return;
  const uint64_t w = mis2_sweep_row_w(i, rp, col, sflag, w1);
  if (w == mis2_word(kUndecided, i, seed)) {
    state[i] = kIn;
  } else if ((int8_t)(w >> 62) == kIn) {
    state[i] = kOut;
  } else {
    atomicAdd(undecided, 1ull);
  }
}

__global__ void k_in_flag(int64_t n, const int8_t *state, int64_t *flag) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  flag[i] = state[i] == kIn ? 1 : 0;
}

// roots get their rank; strong neighbours of a root take the first root met
// in column order
__global__ void k_agg_pass1(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *sflag,
                            const int32_t *sdeg, const int8_t *state, const int64_t *rootid, int32_t *first) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  int32_t a = -1;
  if (state[i] == kIn) {
    a = (int32_t)rootid[i];
  } else if (sdeg[i] > 0) {
    for (int64_t p = rp[i]; p < rp[i + 1]; p++)
      if (sflag[p] && state[col[p]] == kIn) { a = (int32_t)rootid[col[p]]; break; }
  }
  first[i] = a;
}

// the rest join the first-pass neighbour of largest |a_ij|, smaller id on ties
__global__ void k_agg_pass2(int64_t n, const int64_t *rp, const int32_t *col, const double *val,
                            const uint8_t *sflag, const int32_t *sdeg, const int32_t *first, int32_t *agg) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  int32_t a = first[i];
  if (a < 0 && sdeg[i] > 0) {
    double best = -1.0;
    int32_t pick = -1;
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      if (!sflag[p]) continue;
      const int32_t fj = first[col[p]];
      if (fj < 0) continue;
      const double v = fabs(val[p]);
      if (v > best || (v == best && fj < pick)) { best = v; pick = fj; }
    }
    a = pick;
  }
  agg[i] = a;
}

__global__ void k_member_count(int64_t n, const int32_t *agg, int64_t *cnt) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  if (agg[i] >= 0) atomicAdd((unsigned long long *)&cnt[agg[i]], 1ull);
}

__global__ void k_member_fill(int64_t n, const int32_t *agg, const int64_t *mptr, int64_t *cursor,
                              int32_t *midx) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  const int32_t a = agg[i];
  if (a < 0) return;
  const int64_t at = (int64_t)atomicAdd((unsigned long long *)&cursor[a], 1ull);
  midx[mptr[a] + at] = (int32_t)i;
}

__global__ void k_member_sort(int64_t na, const int64_t *mptr, int32_t *midx) {
  pdl_enter();
  const int64_t a = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (a >= na) return;
  for (int64_t t = mptr[a] + 1; t < mptr[a + 1]; t++) {
    const int32_t v = midx[t];
    int64_t u = t - 1;
    while (u >= mptr[a] && midx[u] > v) { midx[u + 1] = midx[u]; u--; }
    midx[u + 1] = v;
  }
}

// ------------------------------------------------------------- Galerkin
// One warp per coarse row I.  The (J, a) pairs of the members of I (members
// ascending, entries in column order) are staged in shared memory in that
// order, with keys J << 32 | staging index; a warp bitonic sort of the keys
// puts equal J together in staging order, and the first lane of each run
// sums its run's values from 0.0 in that order (the definition's order).
// Rows with more pairs than the staging area go to k_galerkin_long (their
// count is marked -1).  The distinct J of a row are counted and written, with
// their sums, at I * kGalCap of pcol/pval: a padded area that k_gal_compact
// packs once the counts are scanned, so that the staging and the sort run
// once.
constexpr int kGalCap = 256;

__global__ void __launch_bounds__(kThreads) k_galerkin(int64_t na, const int64_t *rp, const int32_t *col,
                                                       const double *val, const int32_t *agg, const int64_t *mptr,
                                                       const int32_t *midx, int64_t *pcount, int32_t *pcol,
                                                       double *pval, int32_t *long_rows, int *n_long) {
  pdl_enter();
  __shared__ uint64_t sK[kWarps][kGalCap];
  __shared__ double sV[kWarps][kGalCap];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int64_t I = blockIdx.x * (int64_t)kWarps + wid;
  if (I >= na) return;
  const int64_t m0 = mptr[I], m1 = mptr[I + 1];
  // stage, 32 members at a time: the lanes read the members' row extents
  // together, a warp scan gives each member's offset, and every lane then
  // fills the pairs q = lane, lane + 32, ... of the flattened (member,
  // entry) order, so the loads of all members are in flight at once
  int total = 0;
  bool staged = true;
  for (int64_t t0 = m0; t0 < m1; t0 += 32) {
    const int nm = (int)(m1 - t0 < 32 ? m1 - t0 : 32);
    int64_t p0 = 0;
    int len = 0;
    if (lane < nm) {
      const int64_t i = midx[t0 + lane];
      p0 = rp[i];
      len = (int)(rp[i + 1] - p0);
    }
    int inc = len;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, inc, o);
      if (lane >= o) inc += v;
    }
    const int ctot = __shfl_sync(0xffffffffu, inc, 31);
    if (total + ctot > kGalCap) { staged = false; break; }
    const int excl = inc - len;
    for (int q0 = 0; q0 < ctot; q0 += 32) {
      const int q = q0 + lane;
      int m = 0;
      for (int mm = 1; mm < nm; mm++)
        if (__shfl_sync(0xffffffffu, excl, mm) <= q) m = mm;
      const int64_t pm = __shfl_sync(0xffffffffu, p0, m);
      const int em = __shfl_sync(0xffffffffu, excl, m);
      if (q < ctot) {
        const int64_t p = pm + (q - em);
        // columns outside the coarse space (agg < 0, a zero row of P) take the
        // largest key: they sort last and start no run
        const int32_t a = agg[col[p]];
        sK[wid][total + q] = a < 0 ? ~0ull : (((uint64_t)(uint32_t)a << 32) | (uint64_t)(total + q));
        sV[wid][total + q] = val[p];
      }
    }
    total += ctot;
  }
  if (!staged) {
    if (lane == 0) {
      long_rows[atomicAdd(n_long, 1)] = (int32_t)I;
      pcount[I] = -1;   // counted and written by k_galerkin_long
    }
    return;
  }
  // bitonic sort of the keys, padded with the largest key to a power of two
  int P = 1;
  while (P < total) P <<= 1;
  for (int t = total + lane; t < P; t += 32) sK[wid][t] = ~0ull;
  __syncwarp();
  for (int k2 = 2; k2 <= P; k2 <<= 1)
    for (int j = k2 >> 1; j > 0; j >>= 1) {
      for (int t = lane; t < P; t += 32) {
        const int u = t ^ j;
        if (u > t) {
          const uint64_t a = sK[wid][t], b = sK[wid][u];
          if ((a > b) == ((t & k2) == 0)) {
            sK[wid][t] = b;
            sK[wid][u] = a;
          }
        }
      }
      __syncwarp();
    }
  // runs of equal J: count them, or write each with its sum
  int64_t count = 0;
  for (int t0 = 0; t0 < total; t0 += 32) {
    const int t = t0 + lane;
    bool head = false;
    uint32_t J = 0;
    if (t < total) {
      J = (uint32_t)(sK[wid][t] >> 32);
      head = J != 0xffffffffu && (t == 0 || (uint32_t)(sK[wid][t - 1] >> 32) != J);
    }
    const unsigned hm = __ballot_sync(0xffffffffu, head);
    if (head) {
      double sum = 0.0;
      for (int u = t; u < total && (uint32_t)(sK[wid][u] >> 32) == J; u++)
        sum = sum + sV[wid][(int)(sK[wid][u] & 0xffffffffu)];
      const int64_t at = I * kGalCap + count + __popc(hm & ((1u << lane) - 1u));
      pcol[at] = (int32_t)J;
      pval[at] = sum;
    }
    count += __popc(hm);
  }
  if (lane == 0) pcount[I] = count;
}

// Counts of the warp rows for the scan; long rows (-1) are counted by
// k_galerkin_long into the zeroed entries.
__global__ void k_gal_count_merge(int64_t na, const int64_t *pcount, int64_t *count) {
  pdl_enter();
  const int64_t I = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (I >= na) return;
  const int64_t c = pcount[I];
  count[I] = c < 0 ? 0 : c;
}

// Packs the rows written by k_galerkin from their padded area
// into the scanned CSR: a warp per coarse row (rows marked -1 are long rows,
// written by k_galerkin_long).
__global__ void __launch_bounds__(kThreads) k_gal_compact(int64_t na, const int64_t *pcount, const int32_t *pcol,
                                                          const double *pval, const int64_t *crp, int32_t *ccol,
                                                          double *cval) {
  pdl_enter();
  const int lane = threadIdx.x & 31;
  const int64_t I = blockIdx.x * (int64_t)kWarps + (threadIdx.x >> 5);
  if (I >= na) return;
  const int64_t c = pcount[I];
  if (c < 0) return;
  const int64_t src = I * kGalCap, dst = crp[I];
  for (int64_t t = lane; t < c; t += 32) {
    ccol[dst + t] = pcol[src + t];
    cval[dst + t] = pval[src + t];
  }
}

// Long coarse rows: one block per row.  The (J, a) pairs are staged in
// shared memory under the key (J << 32 | sequence number), bitonic-sorted,
// and each run of equal J is summed by one thread in sequence order (the
// same order as the warp path and the definition above).
constexpr int kGalLongMax = 8192;

// exclusive scan of one int per thread over the block; returns the total
__device__ int block_exclusive_scan(int v, int &excl) {
  __shared__ int ws[kWarps];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += t;
  }
  if (lane == 31) ws[warp] = inc;
  __syncthreads();
  int woff = 0, total = 0;
  for (int w = 0; w < kWarps; w++) {
    if (w < warp) woff += ws[w];
    total += ws[w];
  }
  excl = woff + inc - v;
  __syncthreads();
  return total;
}

__global__ void __launch_bounds__(kThreads) k_galerkin_long(const int64_t *rp, const int32_t *col, const double *val,
                                                            const int32_t *agg, const int64_t *mptr,
                                                            const int32_t *midx, const int32_t *long_rows,
                                                            const int *n_long, int fill, int64_t *ccount,
                                                            const int64_t *crp, int32_t *ccol, double *cval,
                                                            int *err) {
  pdl_enter();
  extern __shared__ unsigned long long gsm[];
  unsigned long long *key = gsm;                                     // [kGalLongMax]
  double *sv = reinterpret_cast<double *>(gsm + kGalLongMax);        // [kGalLongMax]
  const uint64_t kPad = ~0ull;
  for (int r = blockIdx.x; r < *n_long; r += gridDim.x) {
    const int64_t I = long_rows[r];
    const int64_t m0 = mptr[I], m1 = mptr[I + 1];
    // stage: member offsets by a block scan over chunks of members
    int64_t base = 0;
    bool overflow = false;
    for (int64_t c0 = m0; c0 < m1; c0 += kThreads) {
      const int64_t t = c0 + threadIdx.x;
      int64_t i = -1, len = 0;
      if (t < m1) {
        i = midx[t];
        len = rp[i + 1] - rp[i];
      }
      int off = 0;
      const int tot = block_exclusive_scan((int)len, off);
      if (base + tot > kGalLongMax) { overflow = true; break; }
      for (int64_t k = 0; k < len; k++) {
        const int64_t p = rp[i] + k, q = base + off + k;
        const int32_t J = agg[col[p]];
        key[q] = J >= 0 ? (((unsigned long long)(uint32_t)J << 32) | (unsigned long long)q) : kPad;
        sv[q] = val[p];
      }
      base += tot;
    }
    if (overflow) {
      if (threadIdx.x == 0) atomicExch(err, 1);
      __syncthreads();
      continue;
    }
    int P = 1;
    while (P < base) P <<= 1;
    for (int q = (int)base + threadIdx.x; q < P; q += kThreads) key[q] = kPad;
    __syncthreads();
    for (int k = 2; k <= P; k <<= 1)
      for (int j = k >> 1; j > 0; j >>= 1) {
        for (int q = threadIdx.x; q < P; q += kThreads) {
          const int x = q ^ j;
          if (x > q) {
            const unsigned long long a = key[q], b = key[x];
            const bool up = (q & k) == 0;
            if ((a > b) == up) { key[q] = b; key[x] = a; }
          }
        }
        __syncthreads();
      }
    // runs of equal J
    int64_t seg_base = 0;
    for (int c0 = 0; c0 < P; c0 += kThreads) {
      const int q = c0 + threadIdx.x;
      int start = 0;
      if (q < P && key[q] != kPad) start = (q == 0 || (key[q] >> 32) != (key[q - 1] >> 32)) ? 1 : 0;
      int before = 0;
      const int tot = block_exclusive_scan(start, before);
      if (fill && start) {
        const unsigned long long J = key[q] >> 32;
        double sum = 0.0;
        for (int m = q; m < P && key[m] != kPad && (key[m] >> 32) == J; m++) sum = sum + sv[key[m] & 0xffffffffull];
        ccol[crp[I] + seg_base + before] = (int32_t)J;
        cval[crp[I] + seg_base + before] = sum;
      }
      seg_base += tot;
    }
    if (!fill && threadIdx.x == 0) ccount[I] = seg_base;
    __syncthreads();
  }
}

// ----------------------------------------------------- smoother set-up
// The maximum is taken on the bit patterns of the non-negative q_i (the
// same order as their values), first within the block, then with one
// atomic per block.
__global__ void k_gershgorin(int64_t n, const int64_t *rp, const double *val, const int64_t *dpos,
                             double *dinv, unsigned long long *lam_bits) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  unsigned long long qb = 0ull;
  if (i < n) {
    double s = 0.0;
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) s = s + fabs(val[p]);
    const double d = dpos[i] < 0 ? 0.0 : val[dpos[i]];
    const double q = s / fabs(d);
    dinv[i] = 1.0 / d;
    qb = (unsigned long long)__double_as_longlong(q);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long other = __shfl_xor_sync(0xffffffffu, qb, o);
    qb = other > qb ? other : qb;
  }
  __shared__ unsigned long long sm[kThreads / 32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = qb;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long m = sm[0];
    for (int w = 1; w < kThreads / 32; w++) m = sm[w] > m ? sm[w] : m;
    atomicMax(lam_bits, m);
  }
}

// ------------------------------------------------- coarsest dense solve
// Inverse of the coarsest operator by Gauss-Jordan elimination on the
// augmented matrix [A | I] (n x 2n, row-major) with partial pivoting (first
// row of largest |a| in the column on ties).  One launch per pivot step k:
// every block eliminates column k from its rows and reports the candidate
// pivot of column k+1 among them; the last block to finish swaps and scales
// the next pivot row.  The right half ends as A^-1.
__global__ void k_csr_to_aug(int64_t n, const int64_t *rp, const int32_t *col, const double *val, double *aug) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  for (int64_t p = rp[i]; p < rp[i + 1]; p++) aug[i * 2 * n + col[p]] = val[p];
  aug[i * 2 * n + n + i] = 1.0;
}

// block-wide argmax of (value, row) with ties to the smaller row
__device__ void block_argmax(double &v, int &r) {
  __shared__ double sv[kWarps];
  __shared__ int sr[kWarps];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double ov = __shfl_xor_sync(0xffffffffu, v, o);
    const int orr = __shfl_xor_sync(0xffffffffu, r, o);
    if (ov > v || (ov == v && orr < r)) { v = ov; r = orr; }
  }
  if ((threadIdx.x & 31) == 0) { sv[threadIdx.x >> 5] = v; sr[threadIdx.x >> 5] = r; }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kWarps; w++)
      if (sv[w] > sv[0] || (sv[w] == sv[0] && sr[w] < sr[0])) { sv[0] = sv[w]; sr[0] = sr[w]; }
  }
  __syncthreads();
  v = sv[0];
  r = sr[0];
  __syncthreads();
}

// swap row k with the pivot row p and divide it by the pivot (one block)
__device__ void gj_pivot_row(int n, int k, int p, double *aug, int *err) {
  const int64_t w = 2 * (int64_t)n;
  // rows updated by other blocks are read around L1 (__ldcg)
  if (p != k) {
    for (int64_t j = threadIdx.x; j < w; j += kThreads) {
      const double t = __ldcg(aug + k * w + j);
      aug[k * w + j] = __ldcg(aug + p * w + j);
      aug[p * w + j] = t;
    }
  } else {
    for (int64_t j = threadIdx.x; j < w; j += kThreads) aug[k * w + j] = __ldcg(aug + k * w + j);
  }
  __syncthreads();
  const double piv = aug[k * w + k];
  if (!(fabs(piv) > 0.0) || !isfinite(piv)) {
    if (threadIdx.x == 0) *err = 1;
    return;
  }
  __syncthreads();
  for (int64_t j = threadIdx.x; j < w; j += kThreads) aug[k * w + j] = aug[k * w + j] / piv;
}

__global__ void __launch_bounds__(kThreads) k_gj_first(int n, double *aug, int *err) {
  pdl_enter();
  const int64_t w = 2 * (int64_t)n;
  double v = -1.0;
  int r = n;
  for (int i = threadIdx.x; i < n; i += kThreads) {
    const double a = fabs(aug[i * w]);
    if (a > v || (a == v && i < r)) { v = a; r = i; }
  }
  block_argmax(v, r);
  gj_pivot_row(n, 0, r, aug, err);
}

__global__ void __launch_bounds__(kThreads) k_gj_step(int n, int k, double *aug, double *pv, int *pr,
                                                     unsigned int *counter, int *err) {
  pdl_enter();
  const int64_t w = 2 * (int64_t)n;
  if (*err) return;
  double v = -1.0;
  int r = n;
  // rows of this block: blockIdx.x, blockIdx.x + gridDim.x, ...
  for (int i = blockIdx.x; i < n; i += gridDim.x) {
    if (i == k) continue;
    const double f = aug[i * w + k];
    __syncthreads();  // every thread holds the multiplier before column k is overwritten
    if (f != 0.0)
      for (int64_t j = k + threadIdx.x; j < w; j += kThreads) aug[i * w + j] = aug[i * w + j] - f * aug[k * w + j];
    __syncthreads();
    if (threadIdx.x == 0 && i > k && k + 1 < n) {
      const double a = fabs(aug[i * w + k + 1]);
      if (a > v || (a == v && i < r)) { v = a; r = i; }
    }
  }
  if (threadIdx.x == 0) {
    pv[blockIdx.x] = v;
    pr[blockIdx.x] = r;
  }
  __shared__ bool last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x == 0) *counter = 0u;
  if (k + 1 >= n) return;
  v = -1.0;
  r = n;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kThreads) {
    const double bv = __ldcg(pv + b);
    const int br = __ldcg(pr + b);
    if (bv > v || (bv == v && br < r)) { v = bv; r = br; }
  }
  block_argmax(v, r);
  gj_pivot_row(n, k + 1, r, aug, err);
}

// The same Gauss-Jordan inverse for n <= kDenseSmall, in shared memory by one
// block of 1024 threads.
constexpr int kDenseSmall = 64;

__global__ void __launch_bounds__(1024) k_gj_small(int n, const int64_t *rp, const int32_t *col,
                                                   const double *val, double *inv, int *err) {
  pdl_enter();
  __shared__ double a[kDenseSmall][2 * kDenseSmall];
  __shared__ double fk[kDenseSmall];
  __shared__ double bv[32];
  __shared__ int br[32];
  __shared__ int piv_row;
  const int w = 2 * n, tid = threadIdx.x, nt = blockDim.x;
  for (int e = tid; e < n * w; e += nt) a[e / w][e % w] = 0.0;
  __syncthreads();
  for (int i = tid; i < n; i += nt) {
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) a[i][col[p]] = val[p];
    a[i][n + i] = 1.0;
  }
  __syncthreads();
  for (int k = 0; k < n; k++) {
    double v = -1.0;
    int r = n;
    for (int i = k + tid; i < n; i += nt) {
      const double x = fabs(a[i][k]);
      if (x > v || (x == v && i < r)) { v = x; r = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ov = __shfl_xor_sync(0xffffffffu, v, o);
      const int orr = __shfl_xor_sync(0xffffffffu, r, o);
      if (ov > v || (ov == v && orr < r)) { v = ov; r = orr; }
    }
    if ((tid & 31) == 0) { bv[tid >> 5] = v; br[tid >> 5] = r; }
    __syncthreads();
    if (tid == 0) {
      double b0 = -1.0;
      int r0 = n;
      for (int x = 0; x < nt / 32; x++)
        if (bv[x] > b0 || (bv[x] == b0 && br[x] < r0)) { b0 = bv[x]; r0 = br[x]; }
      if (!(b0 > 0.0) || !isfinite(b0)) *err = 1;
      piv_row = r0;
    }
    __syncthreads();
    if (*err) return;
    const int p = piv_row;
    if (p != k)
      for (int j = tid; j < w; j += nt) {
        const double t = a[k][j];
        a[k][j] = a[p][j];
        a[p][j] = t;
      }
    __syncthreads();
    const double pv = a[k][k];
    __syncthreads();
    for (int j = tid; j < w; j += nt) a[k][j] = a[k][j] / pv;
    for (int i = tid; i < n; i += nt) fk[i] = a[i][k];   // multipliers, before column k changes
    __syncthreads();
    for (int e = tid; e < n * (w - k); e += nt) {
      const int i = e / (w - k), j = k + e % (w - k);
      if (i != k) a[i][j] = a[i][j] - fk[i] * a[k][j];
    }
    __syncthreads();
  }
  for (int e = tid; e < n * n; e += nt) inv[e] = a[e / n][n + e % n];
}

__global__ void k_aug_to_inv(int64_t n, const double *aug, double *inv) {
  pdl_enter();
  const int64_t idx = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (idx >= n * n) return;
  const int64_t i = idx / n, j = idx % n;
  inv[idx] = aug[i * 2 * n + n + j];
}

// ------------------------------------------------------------ colouring
// Jones-Plassmann round with first-fit colours; reads the colours of the
// previous round only (double buffer), so the result does not depend on
// thread timing.
__global__ void k_colour_round(Geom g, const uint8_t *emask, const int64_t *tptr, const int32_t *tcol,
                               uint32_t seed, const int32_t *cin, int32_t *cout, unsigned long long *coloured,
                               int *overflow) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= g.n_rows) return;
  const int32_t ci = cin[i];
  cout[i] = ci;
  if (ci >= 0) return;
  const uint64_t ki = node_key(i, seed);
  uint64_t used = 0;
  bool ready = true;
  if (i < g.nc) {
    const unsigned m = emask[i];
    for (int s = 0; s < kSlots; s++) {
      if (s == kSelf || !((m >> s) & 1u)) continue;
      const int64_t j = i + g.off[s];
      const int32_t cj = cin[j];
      if (cj < 0) {
        if (node_key(j, seed) > ki) ready = false;
      } else {
        used |= 1ull << cj;
      }
    }
  }
  for (int64_t t = tptr[i]; t < tptr[i + 1]; t++) {
    const int64_t j = tcol[t];
    if (j == i) continue;
    const int32_t cj = cin[j];
    if (cj < 0) {
      if (node_key(j, seed) > ki) ready = false;
    } else {
      used |= 1ull << cj;
    }
  }
  if (!ready) return;
  if (used == ~0ull) {
    atomicExch(overflow, 1);
    return;
  }
  cout[i] = __ffsll((long long)~used) - 1;
  atomicAdd(coloured, 1ull);
}

__global__ void k_colour_count(Geom g, const int32_t *colour, unsigned long long *cnt, unsigned long long *cnt_cells) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= g.n_rows) return;
  atomicAdd(&cnt[colour[i]], 1ull);
  if (i < g.nc) atomicAdd(&cnt_cells[colour[i]], 1ull);
}

__global__ void k_colour_flag(int64_t n, const int32_t *colour, int c, int64_t *flag) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n) return;
  flag[i] = colour[i] == c ? 1 : 0;
}

__global__ void k_colour_place(int64_t n, const int32_t *colour, int c, const int64_t *rank, int64_t base,
                               int32_t *crow, int64_t *pos) {
  pdl_enter();
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i >= n || colour[i] != c) return;
  const int64_t q = base + rank[i];
  crow[q] = (int32_t)i;
  pos[i] = q;
}

// ------------------------------------------------------------------ ILU(0)
__global__ void k_ilu_lmask_len(Geom g, const uint8_t *emask, const int64_t *tptr, const int32_t *crow,
                                const int64_t *pos, uint8_t *lmask, int64_t *len) {
  pdl_enter();
  const int64_t q = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (q >= g.n_rows) return;
  const int64_t i = crow[q];
  unsigned lm = 0;
  if (i < g.nc) {
    const unsigned m = emask[i];
    for (int s = 0; s < kSlots; s++)
      if (s != kSelf && ((m >> s) & 1u) && pos[i + g.off[s]] < q) lm |= 1u << s;
  }
  len[q] = tptr[i + 1] - tptr[i];
  if (len[q] > 0) lm |= kTailBit;
  lmask[q] = (uint8_t)lm;
}

__global__ void k_ilu_tail_fill(Geom g, const int64_t *tptr, const int32_t *tcol, const int32_t *crow,
                                const int64_t *pos, const int64_t *ftptr, int32_t *ftcol, uint8_t *ftlow,
                                int64_t *ftsrc) {
  pdl_enter();
  const int64_t q = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (q >= g.n_rows) return;
  const int64_t i = crow[q];
  int64_t u = ftptr[q];
  for (int64_t t = tptr[i]; t < tptr[i + 1]; t++, u++) {
    ftcol[u] = tcol[t];
    ftlow[u] = pos[tcol[t]] < q ? 1 : 0;
    ftsrc[u] = t;
  }
}

// Factor storage from Ã: the 7 stencil slots of every position, gathered
// from natural to colour-major order, then the tail entries (a thread per
// entry; fill entries of ILU(1) have no source block and start from zero).
// Blocks of a multiple of 16 bytes are copied a thread per position with
// 128-bit accesses; other sizes (b = 3, 5) a warp per 32 consecutive blocks
// of one slot, lane by lane over their elements, so that the stores stay
// contiguous.
template <int B, class T>
__global__ void k_ilu_init(Geom g, const uint8_t *emask, const int32_t *crow, const T *at_ell,
                           const T *at_tval, const int64_t *ftsrc, int64_t nft, int64_t slot_warps, T *fell,
                           T *ftval) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t np = g.n_rows;
  const int64_t w = (blockIdx.x * (int64_t)kThreads + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (w < slot_warps) {
    if constexpr (BB * sizeof(T) % 16 == 0) {
      const int64_t q = w * 32 + lane;   // slot_warps covers the positions once
      if (q >= np) return;
      const int64_t i = crow[q];
      const unsigned m = i < g.nc ? emask[i] : 0u;
#pragma unroll
      for (int s = 0; s < kSlots; s++) {
        T v[BB];
        if ((m >> s) & 1u) {
          bload<B, T>(BRef<T>{const_cast<T *>(at_ell) + ((int64_t)s * g.nc + i) * BB, 1}, v);
        } else {
#pragma unroll
          for (int e = 0; e < BB; e++) v[e] = T(0);
        }
        bstore<B, T>(BRef<T>{fell + ((int64_t)s * np + q) * BB, 1}, v);
      }
    } else {
      const int64_t chunks = (np + 31) / 32;
      const int s = (int)(w / chunks);
      const int64_t q0 = (w % chunks) * 32;
      const int64_t nq = np - q0 < 32 ? np - q0 : 32;
      T *dst = fell + ((int64_t)s * np + q0) * BB;
      for (int64_t e = lane; e < nq * BB; e += 32) {
        const int64_t i = crow[q0 + e / BB];
        T v = T(0);
        if (i < g.nc && ((emask[i] >> s) & 1u)) v = at_ell[((int64_t)s * g.nc + i) * BB + e % BB];
        dst[e] = v;
      }
    }
    return;
  }
  const int64_t idx = (w - slot_warps) * 32 + lane;
  if (idx >= nft) return;
  const int64_t src = ftsrc[idx];
#pragma unroll
  for (int e = 0; e < BB; e++) ftval[idx * BB + e] = src >= 0 ? at_tval[src * BB + e] : T(0);
}

// IKJ ILU(0) of the rows at positions [q0, q1) (one colour): for every
// earlier-ordered k of row i in ascending order, L_ik = W_ik U_kk^-1 and
// W_ij -= L_ik U_kj for later-ordered j of row i with (k, j) stored; then
// U_ii^-1 replaces W_ii in slot 3.  The pairs (k, j) are found by walking
// row k (its slots, then its tail) and locating each j in row i: by offset
// for a slot neighbour, directly for j = i, by a search of row i's (short)
// tail otherwise; the positions of row i's slot neighbours stay in
// registers.  With ILU(1) (fmask given) the fill slots (fell slots 7 + f,
// neighbour at off2[f]) are one more set of slots of every cell row: the
// same IKJ steps on the level-1 pattern.  The FP32 form is held to two
// resident blocks per SM (b = 5 otherwise takes 207 registers and one).
template <int B, class T>
__global__ void __launch_bounds__(kThreads, sizeof(T) == 4 ? 2 : 1) k_ilu_factor(Geom g, const uint8_t *emask, const int32_t *crow, const int64_t *pos,
                             const int64_t *ftptr, const int32_t *ftcol, const uint8_t *ftlow,
                             const uint32_t *fmask, T *fell, T *ftval, int64_t q0, int64_t q1, int *err) {
  pdl_enter();
  constexpr int BB = B * B;
  const int64_t q = q0 + blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (q >= q1) return;
  const int64_t np = g.n_rows, i = crow[q];
  const bool cell = i < g.nc;
  const unsigned m = cell ? emask[i] : 0u;
  const unsigned fm = (cell && fmask) ? fmask[q] : 0u;
  const int64_t u0 = ftptr[q], u1 = ftptr[q + 1];
  int64_t spos[kSlots];
#pragma unroll
  for (int s = 0; s < kSlots; s++) spos[s] = (s != kSelf && ((m >> s) & 1u)) ? pos[i + g.off[s]] : -1;
  auto fslot = [&](int f) -> T * { return fell + ((int64_t)(kSlots + f) * np + q) * BB; };
  // reference to the entry of row i in column j with its position, or p = nullptr
  auto target = [&](int64_t j, int64_t &pj) -> BRef<T> {
    if (j == i) {
      pj = q;
      if (cell) return BRef<T>{fell + ((int64_t)kSelf * np + q) * BB, 1};
    } else if (cell && j < g.nc) {
      const int64_t d = j - i;
#pragma unroll
      for (int s = 0; s < kSlots; s++)
        if (s != kSelf && ((m >> s) & 1u) && g.off[s] == d) {
          pj = spos[s];
          return BRef<T>{fell + ((int64_t)s * np + q) * BB, 1};
        }
      if (fm)
        for (int f = 0; f < kFill; f++)
          if (((fm >> f) & 1u) && g.off2[f] == d) {
            pj = pos[j];
            return BRef<T>{fslot(f), 1};
          }
    }
    for (int64_t u = u0; u < u1; u++)
      if (ftcol[u] == j) {
        pj = j == i ? q : pos[j];
        return BRef<T>{ftval + u * BB, 1};
      }
    return BRef<T>{nullptr, 0};
  };
  int64_t cur = -1;
  for (;;) {
    // next lower entry in ascending position
    int64_t pbest = q, kr = -1;
    BRef<T> wref{nullptr, 0};
#pragma unroll
    for (int s = 0; s < kSlots; s++) {
      const int64_t pc = spos[s];
      if (pc > cur && pc < pbest) {
        pbest = pc;
        kr = i + g.off[s];
        wref = BRef<T>{fell + ((int64_t)s * np + q) * BB, 1};
      }
    }
    if (fm)
      for (int f = 0; f < kFill; f++) {
        if (!((fm >> f) & 1u)) continue;
        const int64_t pc = pos[i + g.off2[f]];
        if (pc > cur && pc < pbest) {
          pbest = pc;
          kr = i + g.off2[f];
          wref = BRef<T>{fslot(f), 1};
        }
      }
    for (int64_t u = u0; u < u1; u++) {
      const int64_t c = ftcol[u];
      if (c == i) continue;
      const int64_t pc = pos[c];
      if (pc > cur && pc < pbest) {
        pbest = pc;
        kr = c;
        wref = BRef<T>{ftval + u * BB, 1};
      }
    }
    if (kr < 0) break;
    cur = pbest;
    T W[BB], Uinv[BB], L[BB];
    bload<B, T>(wref, W);
    bload<B, T>(BRef<T>{fell + ((int64_t)kSelf * np + pbest) * BB, 1}, Uinv);
    bmul<B, T>(W, Uinv, L);
    bstore<B, T>(wref, L);
    // W_ij -= L_ik U_kj for the entry (k, j) of row k kept in `ub`
    auto update = [&](int64_t j, const T *ub) {
      int64_t pj = -1;
      const BRef<T> wr = target(j, pj);
      if (!wr.p || pj <= pbest) return;
      T U[BB], P[BB], Wij[BB];
      bload<B, T>(BRef<T>{const_cast<T *>(ub), 1}, U);
      bmul<B, T>(L, U, P);
      bload<B, T>(wr, Wij);
#pragma unroll
      for (int e = 0; e < BB; e++) Wij[e] = Wij[e] - P[e];
      bstore<B, T>(wr, Wij);
    };
    // row k: its slots, its fill slots, then its tail
    const bool kcell = kr < g.nc;
    const unsigned mk = kcell ? emask[kr] : 0u;
    for (int s2 = 0; s2 < kSlots; s2++) {
      if (s2 == kSelf || !((mk >> s2) & 1u)) continue;
      update(kr + g.off[s2], fell + ((int64_t)s2 * np + pbest) * BB);
    }
    const unsigned fk = (kcell && fmask) ? fmask[pbest] : 0u;
    if (fk)
      for (int f = 0; f < kFill; f++) {
        if (!((fk >> f) & 1u)) continue;
        update(kr + g.off2[f], fell + ((int64_t)(kSlots + f) * np + pbest) * BB);
      }
    const int64_t k0 = ftptr[pbest], k1 = ftptr[pbest + 1];
    for (int64_t uk = k0; uk < k1; uk++) {
      const int64_t j = ftcol[uk];
      if (j == kr) continue;
      update(j, ftval + uk * BB);
    }
  }
  // diagonal: slot 3 for cells, the tail entry for other rows
  T Wd[BB], inv[BB];
  BRef<T> dref{fell + ((int64_t)kSelf * np + q) * BB, 1};
  if (!cell) {
    for (int64_t u = u0; u < u1; u++)
      if (ftcol[u] == i) { dref = BRef<T>{ftval + u * BB, 1}; break; }
  }
  bload<B, T>(dref, Wd);
  if (!gj_inverse<B, T>(Wd, inv)) {
    atomicExch(err, 1);
    return;
  }
  bstore<B, T>(BRef<T>{fell + ((int64_t)kSelf * np + q) * BB, 1}, inv);
  (void)ftlow;
}

// The same factorisation for rows held entirely in the tail (wells, general
// rows), one warp per row: the next earlier-ordered k is found by a warp
// minimum over the row's entries, L_ik = W_ik U_kk^-1 is formed, and the
// entries (k, j) of row k, later-ordered than k, are matched by binary
// search in row i and update W_ij, each lane one entry of row k.
template <int B, class T>
__global__ void __launch_bounds__(kThreads) k_ilu_factor_long(Geom g, const uint8_t *emask, const int32_t *crow,
                                                              const int64_t *pos, const int64_t *ftptr,
                                                              const int32_t *ftcol, const uint32_t *fmask,
                                                              T *fell, T *ftval, int64_t q1, int64_t q2, int *err) {
  pdl_enter();
  constexpr int BB = B * B;
  const int lane = threadIdx.x & 31;
  const int64_t q = q1 + blockIdx.x * (int64_t)kWarps + (threadIdx.x >> 5);
  if (q >= q2) return;
  const int64_t np = g.n_rows, i = crow[q];
  const int64_t u0 = ftptr[q], u1 = ftptr[q + 1];
  // the row's columns and their positions, cached per warp when short enough
  constexpr int kCache = 384;
  __shared__ int32_t s_col[kWarps][kCache];
  __shared__ int64_t s_pos[kWarps][kCache];
  const int wid = threadIdx.x >> 5;
  const bool cached = (u1 - u0) <= kCache;
  if (cached)
    for (int64_t u = u0 + lane; u < u1; u += 32) {
      s_col[wid][u - u0] = ftcol[u];
      s_pos[wid][u - u0] = pos[ftcol[u]];
    }
  __syncwarp();
  auto col_at = [&](int64_t u) -> int64_t { return cached ? s_col[wid][u - u0] : ftcol[u]; };
  auto pos_at = [&](int64_t u) -> int64_t { return cached ? s_pos[wid][u - u0] : pos[ftcol[u]]; };
  int64_t cur = -1;
  for (;;) {
    long long pb = q, ub = -1;
    for (int64_t u = u0 + lane; u < u1; u += 32) {
      const int64_t c = col_at(u);
      if (c == i) continue;
      const int64_t pc = pos_at(u);
      if (pc > cur && pc < pb) { pb = pc; ub = u; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const long long opb = __shfl_xor_sync(0xffffffffu, pb, o);
      const long long oub = __shfl_xor_sync(0xffffffffu, ub, o);
      if (opb < pb) { pb = opb; ub = oub; }
    }
    if (ub < 0) break;
    cur = pb;
    const int64_t kr = col_at(ub);
    // L = W_ik U_kk^-1, one entry per lane (first product, then running sum)
    __shared__ T s_L[kWarps][BB];
    __shared__ int64_t s_dst[kWarps][32];
    __shared__ int64_t s_src[kWarps][32];
    __shared__ int64_t s_srcs[kWarps][32];
    const int64_t ku0 = ftptr[pb], ku1 = ftptr[pb + 1];
    if (lane < BB) {
      const int r = lane / B, c = lane % B;
      const T *W = ftval + ub * BB;
      const T *U = fell + ((int64_t)kSelf * np + pb) * BB;
      T acc = W[r * B] * U[c];
#pragma unroll
      for (int t = 1; t < B; t++) acc = acc + W[r * B + t] * U[t * B + c];
      s_L[wid][lane] = acc;
    }
    __syncwarp();
    if (lane < BB) ftval[ub * BB + lane] = s_L[wid][lane];
    // entries (k, j) of row k later than k with j stored in row i: lane e
    // resolves entry e of row k (slots first, then the ILU(1) fill slots,
    // then the tail)
    const int nks = fmask ? kSlots + kFill : kSlots;
    const int nk = nks + (int)(ku1 - ku0);
    const unsigned mk = kr < g.nc ? emask[kr] : 0u;
    const unsigned fk = (kr < g.nc && fmask) ? fmask[pb] : 0u;
    for (int e0 = 0; e0 < nk; e0 += 32) {
      const int e = e0 + lane;
      int64_t dst = -1, src = 0, srcs = 1;
      if (e < nk) {
        int64_t j = -1;
        if (e < kSlots) {
          if (e != kSelf && ((mk >> e) & 1u)) {
            j = kr + g.off[e];
            src = ((int64_t)e * np + pb) * BB;  // into fell
            srcs = -1;                          // negative marks fell
          }
        } else if (e < nks) {
          if ((fk >> (e - kSlots)) & 1u) {
            j = kr + g.off2[e - kSlots];
            src = ((int64_t)e * np + pb) * BB;
            srcs = -1;
          }
        } else {
          const int64_t uk = ku0 + (e - nks);
          j = ftcol[uk];
          if (j == kr) j = -1;
          src = uk * BB;
        }
        if (j >= 0 && pos[j] > pb) {
          int64_t lo = u0, hi = u1 - 1;
          while (lo <= hi) {
            const int64_t mid = lo + (hi - lo) / 2;
            const int64_t c = col_at(mid);
            if (c == j) { dst = mid; break; }
            if (c < j) lo = mid + 1; else hi = mid - 1;
          }
        }
      }
      s_dst[wid][lane] = dst;
      s_src[wid][lane] = src;
      s_srcs[wid][lane] = srcs;
      __syncwarp();
      const int cnt = min(32, nk - e0);
      // W_ij -= L U_kj, one (entry, element) pair per lane
      for (int task = lane; task < cnt * BB; task += 32) {
        const int ent = task / BB, el = task % BB;
        const int64_t d = s_dst[wid][ent];
        if (d < 0) continue;
        const int r = el / B, c = el % B;
        const int64_t sb = s_src[wid][ent], ss = s_srcs[wid][ent];
        const T *U = ss < 0 ? fell + sb : ftval + sb;
        const int64_t st = 1;
        T acc = s_L[wid][r * B] * U[(int64_t)c * st];
#pragma unroll
        for (int t = 1; t < B; t++) acc = acc + s_L[wid][r * B + t] * U[(int64_t)(t * B + c) * st];
        T *Wp = ftval + d * BB + el;
        *Wp = *Wp - acc;
      }
      __syncwarp();
    }
  }
  if (lane != 0) return;
  int64_t lo = u0, hi = u1 - 1, dg = -1;
  while (lo <= hi) {
    const int64_t mid = lo + (hi - lo) / 2;
    const int64_t c = col_at(mid);
    if (c == i) { dg = mid; break; }
    if (c < i) lo = mid + 1; else hi = mid - 1;
  }
  T Wd[BB], inv[BB];
  if (dg < 0) { atomicExch(err, 1); return; }
  bload<B, T>(BRef<T>{ftval + dg * BB, 1}, Wd);
  if (!gj_inverse<B, T>(Wd, inv)) {
    atomicExch(err, 1);
    return;
  }
  bstore<B, T>(BRef<T>{fell + ((int64_t)kSelf * np + q) * BB, 1}, inv);
}

// Long rows with a precomputed plan, one block per row: the row's blocks,
// the U_kk^-1 of its earlier-ordered entries and (when they fit) the U_kj
// blocks of the plan's pairs are staged in shared memory; the IKJ steps run
// in ascending position of k, each step forming L_ik = W_ik U_kk^-1 with
// BB threads and then W_ij -= L_ik U_kj with one thread per (pair,
// element), the same products in the same order as the other kernels.
template <int B, class T>
__global__ void __launch_bounds__(kThreads) k_ilu_factor_planned(
    int64_t np, const int64_t *ftptr, LongRowPlan plan, int64_t first, int64_t q1, int ub_in_smem, T *fell,
    T *ftval, int *err) {
  pdl_enter();
  constexpr int BB = B * B;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const int64_t r = first + blockIdx.x, q = q1 + blockIdx.x;
  const int64_t u0 = ftptr[q], ne = ftptr[q + 1] - u0;
  const int64_t l0 = plan.Lptr[r], nl = plan.Lptr[r + 1] - l0;
  const int64_t p0 = plan.Pptr[l0], npair = plan.Pptr[l0 + nl] - p0;
  T *W = reinterpret_cast<T *>(smem_raw);
  T *Ui = W + ne * BB;
  T *Ub = Ui + nl * BB;
  __shared__ T Lsh[BB];
  for (int64_t x = threadIdx.x; x < ne * BB; x += kThreads) W[x] = ftval[u0 * BB + x];
  for (int64_t x = threadIdx.x; x < nl * BB; x += kThreads) {
    const int64_t t = x / BB, e = x % BB;
    Ui[x] = fell[((int64_t)kSelf * np + plan.Lpk[l0 + t]) * BB + e];
  }
  auto ublk = [&](int64_t pidx, int e) -> T {
    const int64_t src = plan.Psrc[pidx];
    return src >= 0 ? ftval[src + e] : fell[~src + e];
  };
  if (ub_in_smem)
    for (int64_t x = threadIdx.x; x < npair * BB; x += kThreads) Ub[x] = ublk(p0 + x / BB, (int)(x % BB));
  __syncthreads();
  for (int64_t t = 0; t < nl; t++) {
    const int64_t ut = plan.Lu[l0 + t];
    if (threadIdx.x < BB) {
      const int rr = threadIdx.x / B, c = threadIdx.x % B;
      const T *Wt = W + ut * BB, *U = Ui + t * BB;
      T acc = Wt[rr * B] * U[c];
#pragma unroll
      for (int tt = 1; tt < B; tt++) acc = acc + Wt[rr * B + tt] * U[tt * B + c];
      Lsh[threadIdx.x] = acc;
    }
    __syncthreads();
    if (threadIdx.x < BB) W[ut * BB + threadIdx.x] = Lsh[threadIdx.x];
    const int64_t pa = plan.Pptr[l0 + t], pb = plan.Pptr[l0 + t + 1];
    for (int64_t task = threadIdx.x; task < (pb - pa) * BB; task += kThreads) {
      const int64_t pidx = pa + task / BB;
      const int el = (int)(task % BB), rr = el / B, c = el % B;
      T acc;
      if (ub_in_smem) {
        const T *U = Ub + (pidx - p0) * BB;
        acc = Lsh[rr * B] * U[c];
#pragma unroll
        for (int tt = 1; tt < B; tt++) acc = acc + Lsh[rr * B + tt] * U[tt * B + c];
      } else {
        acc = Lsh[rr * B] * ublk(pidx, c);
#pragma unroll
        for (int tt = 1; tt < B; tt++) acc = acc + Lsh[rr * B + tt] * ublk(pidx, tt * B + c);
      }
      T *Wd = W + (int64_t)plan.Pdst[pidx] * BB + el;
      *Wd = *Wd - acc;
    }
    __syncthreads();
  }
  for (int64_t x = threadIdx.x; x < ne * BB; x += kThreads) ftval[u0 * BB + x] = W[x];
  if (threadIdx.x != 0) return;
  const int32_t dg = plan.diag[r];
  T Wd[BB], inv[BB];
  if (dg < 0) { atomicExch(err, 1); return; }
#pragma unroll
  for (int e = 0; e < BB; e++) Wd[e] = W[(int64_t)dg * BB + e];
  if (!gj_inverse<B, T>(Wd, inv)) {
    atomicExch(err, 1);
    return;
  }
  bstore<B, T>(BRef<T>{fell + ((int64_t)kSelf * np + q) * BB, 1}, inv);
}

}  // namespace

// =============================================================== launchers
void keep_pool_memory() {
  int dev = 0;
  TRS_CUDA(cudaGetDevice(&dev));
  cudaMemPool_t pool;
  TRS_CUDA(cudaDeviceGetDefaultMemPool(&pool, dev));
  uint64_t thr = UINT64_MAX;
  TRS_CUDA(cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr));
}

void exclusive_scan(const int64_t *in, int64_t *out, int64_t n, int64_t *total, cudaStream_t s) {
  if (n <= 0) {
    if (total) TRS_CUDA(cudaMemsetAsync(total, 0, sizeof(int64_t), s));
    return;
  }
  const int64_t nb = (n + kScanChunk - 1) / kScanChunk;
  TBuf<int64_t> bsum(nb, s);
  launch_pdl(k_scan_reduce, (unsigned)nb, kThreads, 0, s, in, n, bsum.p);
  TRS_LAUNCHED();
  launch_pdl(k_scan_bsums, 1, 32, 0, s, bsum.p, nb, total);
  TRS_LAUNCHED();
  launch_pdl(k_scan_apply, (unsigned)nb, kThreads, 0, s, in, out, n, bsum.p);
  TRS_LAUNCHED();
}

void launch_scatter_values(int64_t nnzb, int bb, const int64_t *map, const double *uval, int64_t nc, double *ell,
                           double *tval, cudaStream_t s) {
  if (!nnzb) return;
  launch_pdl(k_scatter_values, grid_of(nnzb * bb), kThreads, 0, s, nnzb, bb, map, uval, nc, ell, tval);
  TRS_LAUNCHED();
}

void launch_gather_values(int64_t nnzb, int bb, const int64_t *map, const double *ell, const double *tval,
                          int64_t nc, double *uval, cudaStream_t s, int aos) {
  if (!nnzb) return;
  launch_pdl(k_gather_values, grid_of(nnzb * bb), kThreads, 0, s, nnzb, bb, map, ell, tval, nc, aos, uval);
  TRS_LAUNCHED();
}

void launch_assemble(int b, trs_bsr *A, const double *perm, int perm_is_log, double kvkh, double c_t,
                     const double *M, const double *acc, const double *wi, const double *lam, cudaStream_t s) {
  A->tval.zero(s);
  TRS_DISPATCH_B(b, {
    if (A->g.nc) {
      launch_pdl(k_assemble_cells<B>, grid_of(A->g.nc), kThreads, 0, s, 
          A->g, A->emask.p, A->ell.p, A->tval.p, perm, perm_is_log, kvkh, c_t, M, acc, A->cperf_ptr.p,
          A->cperf_idx.p, A->perf_cw.p, wi, lam);
      TRS_LAUNCHED();
    }
    if (A->n_wells)
      launch_pdl(k_assemble_wells<B>, grid_of(A->n_wells), kThreads, 0, s, A->n_wells, A->tval.p, A->wperf_ptr.p,
                                                                   A->wperf_idx.p, A->perf_wc.p, A->wdiag.p,
                                                                   wi, lam);
  });
  TRS_LAUNCHED();
}

void launch_decouple(int b, const MatView<double> &A, const int64_t *tdiag, int mode, double *at_ell,
                     double *at_p, double *at_tval, double *dinv, double *ap_ell, double *ap_tval, int *err,
                     cudaStream_t s) {
  if (!A.g.n_rows) return;
  TRS_DISPATCH_B(b, launch_pdl(k_decouple<B>, grid_of(A.g.n_rows), kThreads, 0, s, A, tdiag, mode, at_ell, at_p, at_tval,
                                                                           dinv, ap_ell, ap_tval, err));
  TRS_LAUNCHED();
}

void launch_decouple_mixed(int b, const MatView<double> &A, const int64_t *tdiag, int mode, float *at_ell,
                           float *at_p, float *at_tval, float *dinv, double *ap_ell, double *ap_tval, int *err,
                           cudaStream_t s) {
  if (!A.g.n_rows) return;
  TRS_DISPATCH_B(b, launch_pdl(k_decouple_mixed<B>, grid_of(A.g.n_rows), kThreads, 0, s, A, tdiag, mode, at_ell, at_p,
                                                                                 at_tval, dinv, ap_ell, ap_tval,
                                                                                 err));
  TRS_LAUNCHED();
}

void launch_ap_csr_rowlen(const Geom &g, const uint8_t *emask, const int64_t *tptr, int64_t *len, cudaStream_t s) {
  launch_pdl(k_ap_rowlen, grid_of(g.n_rows), kThreads, 0, s, g, emask, tptr, len);
  TRS_LAUNCHED();
}

void launch_ap_csr_fill(const Geom &g, const uint8_t *emask, const int64_t *tptr, const int32_t *tcol,
                        const double *ap_ell, const double *ap_tval, const int64_t *rp, int32_t *col, double *val,
                        cudaStream_t s) {
  launch_pdl(k_ap_fill, grid_of(g.n_rows), kThreads, 0, s, g, emask, tptr, tcol, ap_ell, ap_tval, rp, col, val);
  TRS_LAUNCHED();
}

void launch_diag_pos(int64_t n, const int64_t *rp, const int32_t *col, const double *val, int64_t *dpos,
                     double *dval, cudaStream_t s) {
  if (!n) return;
  launch_pdl(k_diag_pos, grid_of(n), kThreads, 0, s, n, rp, col, val, dpos, dval);
  TRS_LAUNCHED();
}

void launch_strength(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const double *dval,
                     double theta, uint8_t *sflag, int32_t *sdeg, cudaStream_t s) {
  if (!n) return;
  launch_pdl(k_strength, grid_of(n * kStrengthLanes), kThreads, 0, s, n, rp, col, val, dval, theta, sflag, sdeg);
  TRS_LAUNCHED();
}

void launch_mis2_init(int64_t n, const int32_t *sdeg, int8_t *state, cudaStream_t s) {
  launch_pdl(k_mis2_init, grid_of(n), kThreads, 0, s, n, sdeg, state);
  TRS_LAUNCHED();
}

void launch_mis2_sweep(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *sflag, const int8_t *state,
                       uint32_t seed, uint64_t *out_w, cudaStream_t s) {
  if (n >= (int64_t(1) << 30)) throw Error(TRS_ERR_UNSUPPORTED, "AMG levels are limited to 2^30 rows");
  launch_pdl(k_mis2_sweep, grid_of(n), kThreads, 0, s, n, rp, col, sflag, state, seed, out_w);
  TRS_LAUNCHED();
}

void launch_mis2_sweep_decide(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *sflag, int8_t *state,
                              const uint64_t *w1, uint32_t seed, unsigned long long *undecided, cudaStream_t s) {
  launch_pdl(k_mis2_sweep_decide, grid_of(n), kThreads, 0, s, n, rp, col, sflag, state, w1, seed, undecided);
  TRS_LAUNCHED();
}

void launch_in_flag(int64_t n, const int8_t *state, int64_t *flag, cudaStream_t s) {
  launch_pdl(k_in_flag, grid_of(n), kThreads, 0, s, n, state, flag);
  TRS_LAUNCHED();
}

void launch_agg_pass1(int64_t n, const int64_t *rp, const int32_t *col, const uint8_t *sflag, const int32_t *sdeg,
                      const int8_t *state, const int64_t *rootid, int32_t *first, cudaStream_t s) {
  launch_pdl(k_agg_pass1, grid_of(n), kThreads, 0, s, n, rp, col, sflag, sdeg, state, rootid, first);
  TRS_LAUNCHED();
}

void launch_agg_pass2(int64_t n, const int64_t *rp, const int32_t *col, const double *val, const uint8_t *sflag,
                      const int32_t *sdeg, const int32_t *first, int32_t *agg, cudaStream_t s) {
  launch_pdl(k_agg_pass2, grid_of(n), kThreads, 0, s, n, rp, col, val, sflag, sdeg, first, agg);
  TRS_LAUNCHED();
}

void launch_members(int64_t n, const int32_t *agg, int64_t n_agg, DBuf<int64_t> &mptr, DBuf<int32_t> &midx,
                    cudaStream_t s) {
  TBuf<int64_t> cnt(n_agg + 1, s), cursor(n_agg + 1, s);
  cnt.zero();
  cursor.zero();
  if (mptr.n < (size_t)(n_agg + 1)) mptr.alloc(n_agg + 1);
  launch_pdl(k_member_count, grid_of(n), kThreads, 0, s, n, agg, cnt.p);
  TRS_LAUNCHED();
  exclusive_scan(cnt.p, mptr.p, n_agg + 1, nullptr, s);
  if (midx.n < (size_t)std::max<int64_t>(n, 1)) midx.alloc(std::max<int64_t>(n, 1));  // members <= n
  launch_pdl(k_member_fill, grid_of(n), kThreads, 0, s, n, agg, mptr.p, cursor.p, midx.p);
  TRS_LAUNCHED();
  launch_pdl(k_member_sort, grid_of(n_agg), kThreads, 0, s, n_agg, mptr.p, midx.p);
  TRS_LAUNCHED();
}

void launch_galerkin(const Csr &F, const int32_t *agg, int64_t n_agg, const int64_t *mptr, const int32_t *midx,
                     Csr &C, cudaStream_t s) {
  static bool attr_set = false;
  const size_t long_smem = (size_t)kGalLongMax * (sizeof(unsigned long long) + sizeof(double));
  if (!attr_set) {
    TRS_CUDA(cudaFuncSetAttribute(k_galerkin_long, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)long_smem));
    attr_set = true;
  }
  TBuf<int64_t> cnt(n_agg + 1, s), pcnt(std::max<int64_t>(n_agg, 1), s);
  TBuf<int32_t> long_rows(std::max<int64_t>(n_agg, 1), s), pcol(std::max<int64_t>(n_agg, 1) * kGalCap, s);
  TBuf<double> pval(std::max<int64_t>(n_agg, 1) * kGalCap, s);
  TBuf<int> n_long(1, s), err(1, s);
  cnt.zero();
  n_long.zero();
  err.zero();
  const unsigned grid = (unsigned)((n_agg + kWarps - 1) / kWarps);
  const unsigned long_grid = 152;
  // warp rows: counted and written to their padded area in one pass
  launch_pdl(k_galerkin, grid, kThreads, 0, s, n_agg, F.rp.p, F.col.p, F.val.p, agg, mptr, midx, pcnt.p, pcol.p,
             pval.p, long_rows.p, n_long.p);
  TRS_LAUNCHED();
  launch_pdl(k_gal_count_merge, grid_of(n_agg), kThreads, 0, s, n_agg, (const int64_t *)pcnt.p, cnt.p);
  TRS_LAUNCHED();
  launch_pdl(k_galerkin_long, long_grid, kThreads, long_smem, s, F.rp.p, F.col.p, F.val.p, agg, mptr, midx, long_rows.p,
                                                         n_long.p, 0, cnt.p, nullptr, nullptr, nullptr, err.p);
  TRS_LAUNCHED();
  C.n = n_agg;
  if (C.rp.n < (size_t)(n_agg + 1)) C.rp.alloc(n_agg + 1);
  exclusive_scan(cnt.p, C.rp.p, n_agg + 1, nullptr, s);
  int herr = 0, hlong = 0;
  TRS_CUDA(cudaMemcpyAsync(&C.nnz, C.rp.p + n_agg, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaMemcpyAsync(&hlong, n_long.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaStreamSynchronize(s));
  TRS_REQUIRE(!herr, TRS_ERR_UNSUPPORTED, "a coarse AMG row has more than 8192 Galerkin contributions");
  if (C.col.n < (size_t)std::max<int64_t>(C.nnz, 1)) C.col.alloc(std::max<int64_t>(C.nnz, 1));
  if (C.val.n < (size_t)std::max<int64_t>(C.nnz, 1)) C.val.alloc(std::max<int64_t>(C.nnz, 1));
  launch_pdl(k_gal_compact, grid, kThreads, 0, s, n_agg, (const int64_t *)pcnt.p, (const int32_t *)pcol.p,
             (const double *)pval.p, (const int64_t *)C.rp.p, C.col.p, C.val.p);
  TRS_LAUNCHED();
  if (hlong) {
    launch_pdl(k_galerkin_long, long_grid, kThreads, long_smem, s, F.rp.p, F.col.p, F.val.p, agg, mptr, midx,
               long_rows.p, n_long.p, 1, nullptr, C.rp.p, C.col.p, C.val.p, err.p);
    TRS_LAUNCHED();
  }
}

void launch_gershgorin_dinv(const Csr &A, const int64_t *dpos, double *dinv, unsigned long long *lam_bits,
                            cudaStream_t s) {
  TRS_CUDA(cudaMemsetAsync(lam_bits, 0, sizeof(unsigned long long), s));
  launch_pdl(k_gershgorin, grid_of(A.n), kThreads, 0, s, A.n, A.rp.p, A.val.p, dpos, dinv, lam_bits);
  TRS_LAUNCHED();
}

int launch_dense_inverse(const Csr &A, DBuf<double> &inv, cudaStream_t s) {
  const int n = (int)A.n;
  if (n <= kDenseSmall) {
    TBuf<int> err(1, s);
    err.zero();
    if (inv.n < (size_t)std::max(n * n, 1)) inv.alloc((size_t)std::max(n * n, 1));
    launch_pdl(k_gj_small, 1, 1024, 0, s, n, A.rp.p, A.col.p, A.val.p, inv.p, err.p);
    TRS_LAUNCHED();
    int herr = 0;
    TRS_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaStreamSynchronize(s));
    return herr ? 1 : 0;
  }
  TBuf<double> aug((size_t)2 * n * n, s);
  const int grid = std::max(1, std::min(n, 152 * 4));
  TBuf<double> pv(grid, s);
  TBuf<int> pr(grid, s), err(1, s);
  TBuf<unsigned int> counter(1, s);
  aug.zero();
  err.zero();
  counter.zero();
  launch_pdl(k_csr_to_aug, grid_of(n), kThreads, 0, s, n, A.rp.p, A.col.p, A.val.p, aug.p);
  TRS_LAUNCHED();
  launch_pdl(k_gj_first, 1, kThreads, 0, s, n, aug.p, err.p);
  TRS_LAUNCHED();
  for (int k = 0; k < n; k++) {
    launch_pdl(k_gj_step, grid, kThreads, 0, s, n, k, aug.p, pv.p, pr.p, counter.p, err.p);
    TRS_LAUNCHED();
  }
  int herr = 0;
  TRS_CUDA(cudaMemcpyAsync(&herr, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaStreamSynchronize(s));
  if (herr) return 1;
  if (inv.n < (size_t)n * n) inv.alloc((size_t)n * n);
  launch_pdl(k_aug_to_inv, grid_of((int64_t)n * n), kThreads, 0, s, n, aug.p, inv.p);
  TRS_LAUNCHED();
  return 0;
}

int launch_colour(const Geom &g, const uint8_t *emask, const int64_t *tptr, const int32_t *tcol, uint32_t seed,
                  int32_t *colour, cudaStream_t s) {
  const int64_t n = g.n_rows;
  TBuf<int32_t> other(n, s);
  TBuf<unsigned long long> cnt(1, s);
  TBuf<int> overflow(1, s);
  cnt.zero();
  overflow.zero();
  TRS_CUDA(cudaMemsetAsync(colour, 0xff, n * sizeof(int32_t), s));
  int32_t *a = colour, *bbuf = other.p;
  unsigned long long done = 0;
  int rounds = 0;
  while (done < (unsigned long long)n) {
    launch_pdl(k_colour_round, grid_of(n), kThreads, 0, s, g, emask, tptr, tcol, seed, a, bbuf, cnt.p, overflow.p);
    TRS_LAUNCHED();
    std::swap(a, bbuf);
    int ov = 0;
    TRS_CUDA(cudaMemcpyAsync(&done, cnt.p, sizeof(done), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaMemcpyAsync(&ov, overflow.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaStreamSynchronize(s));
    if (ov) return -1;
    if (++rounds > 100000) return -1;
  }
  if (a != colour) TRS_CUDA(cudaMemcpyAsync(colour, a, n * sizeof(int32_t), cudaMemcpyDeviceToDevice, s));
  TRS_CUDA(cudaStreamSynchronize(s));
  return rounds;
}

void launch_colour_order(const Geom &g, const int32_t *colour, int ncol, std::vector<int64_t> &cptr,
                         std::vector<int64_t> &cmid, int32_t *crow, int64_t *pos, cudaStream_t s) {
  const int64_t n = g.n_rows;
  TBuf<unsigned long long> cnt(kMaxColours, s), cntc(kMaxColours, s);
  cnt.zero();
  cntc.zero();
  launch_pdl(k_colour_count, grid_of(n), kThreads, 0, s, g, colour, cnt.p, cntc.p);
  TRS_LAUNCHED();
  auto hc = download(cnt.p, kMaxColours, s);
  auto hcc = download(cntc.p, kMaxColours, s);
  cptr.assign(ncol + 1, 0);
  cmid.assign(ncol, 0);
  for (int c = 0; c < ncol; c++) {
    cptr[c + 1] = cptr[c] + (int64_t)hc[c];
    cmid[c] = cptr[c] + (int64_t)hcc[c];
  }
  TBuf<int64_t> flag(n, s), rank(n, s);
  for (int c = 0; c < ncol; c++) {
    launch_pdl(k_colour_flag, grid_of(n), kThreads, 0, s, n, colour, c, flag.p);
    TRS_LAUNCHED();
    exclusive_scan(flag.p, rank.p, n, nullptr, s);
    launch_pdl(k_colour_place, grid_of(n), kThreads, 0, s, n, colour, c, rank.p, cptr[c], crow, pos);
    TRS_LAUNCHED();
  }
  TRS_CUDA(cudaStreamSynchronize(s));
}

void launch_ilu_structure(const Geom &g, const uint8_t *emask, const int64_t *tptr, const int32_t *tcol,
                          const int32_t *crow, const int64_t *pos, uint8_t *lmask, DBuf<int64_t> &ftptr,
                          DBuf<int32_t> &ftcol, DBuf<uint8_t> &ftlow, DBuf<int64_t> &ftsrc, cudaStream_t s) {
  const int64_t n = g.n_rows;
  TBuf<int64_t> len(n + 1, s);
  len.zero();
  launch_pdl(k_ilu_lmask_len, grid_of(n), kThreads, 0, s, g, emask, tptr, crow, pos, lmask, len.p);
  TRS_LAUNCHED();
  ftptr.alloc(n + 1);
  exclusive_scan(len.p, ftptr.p, n + 1, nullptr, s);
  int64_t nft = 0;
  TRS_CUDA(cudaMemcpyAsync(&nft, ftptr.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaStreamSynchronize(s));
  ftcol.alloc(std::max<int64_t>(nft, 1));
  ftlow.alloc(std::max<int64_t>(nft, 1));
  ftsrc.alloc(std::max<int64_t>(nft, 1));
  launch_pdl(k_ilu_tail_fill, grid_of(n), kThreads, 0, s, g, tptr, tcol, crow, pos, ftptr.p, ftcol.p, ftlow.p, ftsrc.p);
  TRS_LAUNCHED();
}

template <class T>
void launch_ilu_init(int b, const Geom &g, const uint8_t *emask, const int32_t *crow, const T *at_ell,
                     const T *at_tval, const int64_t *ftsrc, int64_t nft, int nslots, T *fell, T *ftval,
                     cudaStream_t s) {
  const int64_t np = g.n_rows, bb = (int64_t)b * b;
  // ILU(1) fill slots (7 .. nslots - 1) start from zero
  if (nslots > kSlots)
    TRS_CUDA(cudaMemsetAsync(fell + (int64_t)kSlots * np * bb, 0, (size_t)(nslots - kSlots) * np * bb * sizeof(T), s));
  const bool aligned = (bb * (int64_t)sizeof(T)) % 16 == 0;
  const int64_t slot_warps = (aligned ? 1 : kSlots) * ((np + 31) / 32);
  const int64_t threads = slot_warps * 32 + nft;
  if (!threads) return;
  TRS_DISPATCH_B(b, launch_pdl(k_ilu_init<B, T>, grid_of(threads), kThreads, 0, s, g, emask, crow, at_ell, at_tval, ftsrc,
                                                                           nft, slot_warps, fell, ftval));
  TRS_LAUNCHED();
}
template void launch_ilu_init<double>(int, const Geom &, const uint8_t *, const int32_t *, const double *,
                                      const double *, const int64_t *, int64_t, int, double *, double *,
                                      cudaStream_t);
template void launch_ilu_init<float>(int, const Geom &, const uint8_t *, const int32_t *, const float *,
                                     const float *, const int64_t *, int64_t, int, float *, float *, cudaStream_t);

template <class T>
void launch_ilu_factor_colour(int b, const Geom &g, const uint8_t *emask, const int32_t *crow, const int64_t *pos,
                              const int64_t *ftptr, const int32_t *ftcol, const uint8_t *ftlow,
                              const uint32_t *fmask, T *fell, T *ftval, int64_t q0, int64_t q1, int64_t q2,
                              const LongRowPlan *plan, const LongRowColour *pc, int *err, cudaStream_t s) {
  if (q1 > q0) {
    TRS_DISPATCH_B(b, launch_pdl(k_ilu_factor<B, T>, grid_of(q1 - q0), kThreads, 0, s, g, emask, crow, pos, ftptr, ftcol,
                                                                               ftlow, fmask, fell, ftval, q0, q1,
                                                                               err));
    TRS_LAUNCHED();
  }
  if (q2 > q1 && plan && pc) {
    // shared memory: the rows' blocks, the U_kk^-1 and, if they fit, the U_kj
    const size_t bbs = (size_t)b * b * sizeof(T);
    const size_t base = (size_t)(pc->max_ne + pc->max_nl) * bbs, full = base + (size_t)pc->max_np * bbs;
    constexpr size_t kSmemMax = 200 * 1024;
    if (base <= kSmemMax) {
      const int ub = full <= kSmemMax;
      const size_t bytes = ub ? full : base;
      TRS_DISPATCH_B(b, {
        auto kfn = k_ilu_factor_planned<B, T>;
        TRS_CUDA(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
        launch_pdl(kfn, (unsigned)(q2 - q1), kThreads, bytes, s, g.n_rows, ftptr, *plan, pc->first, q1, ub, fell, ftval,
                                                         err);
      });
      TRS_LAUNCHED();
      return;
    }
  }
  if (q2 > q1) {
    const unsigned grid = (unsigned)((q2 - q1 + kWarps - 1) / kWarps);
    TRS_DISPATCH_B(b, launch_pdl(k_ilu_factor_long<B, T>, grid, kThreads, 0, s, g, emask, crow, pos, ftptr, ftcol, fmask,
                                                                        fell, ftval, q1, q2, err));
    TRS_LAUNCHED();
  }
}
template void launch_ilu_factor_colour<double>(int, const Geom &, const uint8_t *, const int32_t *, const int64_t *,
                                               const int64_t *, const int32_t *, const uint8_t *, const uint32_t *,
                                               double *, double *, int64_t, int64_t, int64_t, const LongRowPlan *,
                                               const LongRowColour *, int *, cudaStream_t);
template void launch_ilu_factor_colour<float>(int, const Geom &, const uint8_t *, const int32_t *, const int64_t *,
                                              const int64_t *, const int32_t *, const uint8_t *, const uint32_t *,
                                              float *, float *, int64_t, int64_t, int64_t, const LongRowPlan *,
                                              const LongRowColour *, int *, cudaStream_t);

void launch_scale_diagonal(int b, trs_bsr *A, const double *sc, cudaStream_t s) {
  if (!A->n) return;
  TRS_DISPATCH_B(b, launch_pdl(k_scale_diag<B>, grid_of(A->n), kThreads, 0, s, A->g, A->ell.p, A->tval.p, A->tdiag.p, sc));
  TRS_LAUNCHED();
}

}  // namespace trs
