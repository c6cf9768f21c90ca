// Host runtime for the CPR-FPF preconditioner and the FGMRES solve.
//
// Setup (Sec. "Decoupling Methods", Sec. "Preconditioners"):
//   ABF/GJE decoupling -> pressure matrix -> aggregation AMG hierarchy ->
//   multicolouring -> block ILU(0) -> optional FP32 copies.
// Application, with f = D^-1 v (Algorithm pc-fpf read from its prose):
//   y1 = F^-1 f; r1_p = (f - Ã y1)_0; e = V-cycle(r1_p);
//   r2 = f - Ã (y1 + Pi_p e); z = y1 + Pi_p e + F^-1 r2.
#include <algorithm>
#include <atomic>
#include <mutex>
#include <chrono>
#include <cmath>

#include "trs_api_common.cuh"

namespace trs {

namespace {
thread_local std::string g_last_error;

constexpr uint32_t kLevelSeedMul = 0x9E3779B9u;
constexpr uint32_t kColourSeedXor = 0x85EBCA77u;
constexpr int kRedGridMax = 152 * 8;

template <class T>
T *tp(const DBuf<char> &b) { return reinterpret_cast<T *>(b.p); }

void alloc_vec(DBuf<char> &b, int64_t n, size_t elem) { b.alloc(std::max<int64_t>(n, 1) * elem); }

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    TRS_CUDA(cudaEventCreate(&a));
    TRS_CUDA(cudaEventCreate(&b));
    TRS_CUDA(cudaEventRecord(a, s));
  }
  double stop() {
    TRS_CUDA(cudaEventRecord(b, s));
    TRS_CUDA(cudaEventSynchronize(b));
    float ms = 0.f;
    TRS_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

// ------------------------------------------------------------ AMG setup
template <class T>
void reserve(DBuf<T> &b, int64_t n) {
  if (b.n < (size_t)std::max<int64_t>(n, 1)) b.alloc(std::max<int64_t>(n, 1));
}

void build_hierarchy(trs_cpr *M, cudaStream_t s) {
  const trs_cpr_opts &o = M->opts;
  auto &lev = M->lev;
  reserve(M->lam_bits, kMaxLevels);
  int nlev = 1;
  for (int l = 0;; l++) {
    Level &F = lev[l];
    const int64_t n = F.A.n;
    reserve(F.dpos, n);
    reserve(F.dval, n);
    launch_diag_pos(n, F.A.rp.p, F.A.col.p, F.A.val.p, F.dpos.p, F.dval.p, s);
    reserve(F.dinv64, n);
    launch_gershgorin_dinv(F.A, F.dpos.p, F.dinv64.p, M->lam_bits.p + l, s);
    if (n <= o.coarse_max || l + 1 >= o.max_levels) break;
    const int64_t nnz = F.A.nnz;
    TBuf<uint8_t> sflag(std::max<int64_t>(nnz, 1), s);
    TBuf<int32_t> sdeg(n, s);
    launch_strength(n, F.A.rp.p, F.A.col.p, F.A.val.p, F.dval.p, o.theta, sflag.p, sdeg.p, s);
    // MIS-2 rounds (first sweep; second sweep with the decision), each
    // counting its undecided rows in its own counter; the count is read
    // every second round (an extra round after completion changes nothing)
    const uint32_t seed = o.seed ^ (kLevelSeedMul * (uint32_t)(l + 1));
    constexpr int kMaxRounds = 10000;
    TBuf<int8_t> state(n, s);
    TBuf<uint64_t> w1(n, s);
    TBuf<unsigned long long> und(kMaxRounds, s);
    und.zero();
    launch_mis2_init(n, sdeg.p, state.p, s);
    for (int round = 0;; round++) {
      TRS_REQUIRE(round < kMaxRounds, TRS_ERR_COARSENING, "MIS-2 did not terminate");
      launch_mis2_sweep(n, F.A.rp.p, F.A.col.p, sflag.p, state.p, seed, w1.p, s);
      launch_mis2_sweep_decide(n, F.A.rp.p, F.A.col.p, sflag.p, state.p, w1.p, seed, und.p + round, s);
      if (round % 2 == 0) continue;
      unsigned long long left = 0;
      TRS_CUDA(cudaMemcpyAsync(&left, und.p + round, sizeof(left), cudaMemcpyDeviceToHost, s));
      TRS_CUDA(cudaStreamSynchronize(s));
      if (!left) break;
    }
    // aggregates
    TBuf<int64_t> flag(n + 1, s), rootid(n + 1, s);
    flag.zero();
    launch_in_flag(n, state.p, flag.p, s);
    exclusive_scan(flag.p, rootid.p, n + 1, nullptr, s);
    int64_t n_agg = 0;
    TRS_CUDA(cudaMemcpyAsync(&n_agg, rootid.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaStreamSynchronize(s));
    if (n_agg == 0 || 10 * n_agg >= 9 * n) break;
    TBuf<int32_t> first(n, s);
    reserve(F.agg, n);
    launch_agg_pass1(n, F.A.rp.p, F.A.col.p, sflag.p, sdeg.p, state.p, rootid.p, first.p, s);
    launch_agg_pass2(n, F.A.rp.p, F.A.col.p, F.A.val.p, sflag.p, sdeg.p, first.p, F.agg.p, s);
    F.n_agg = n_agg;
    launch_members(n, F.agg.p, n_agg, F.mptr, F.midx, s);
    if ((int)lev.size() < l + 2) lev.emplace_back();
    launch_galerkin(lev[l].A, lev[l].agg.p, n_agg, lev[l].mptr.p, lev[l].midx.p, lev[l + 1].A, s);
    nlev = l + 2;
  }
  M->nlev = nlev;
  Level &C = lev[nlev - 1];
  C.n_agg = 0;
  TRS_REQUIRE(C.A.n <= kDenseMax, TRS_ERR_COARSENING, "AMG coarsening stalled above the dense-solve limit");
  TRS_REQUIRE(launch_dense_inverse(C.A, M->cinv, s) == 0, TRS_ERR_SINGULAR_BLOCK, "coarsest AMG matrix is singular");
  unsigned long long bits[kMaxLevels];
  TRS_CUDA(cudaMemcpyAsync(bits, M->lam_bits.p, nlev * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaStreamSynchronize(s));
  for (int l = 0; l < nlev; l++) std::memcpy(&lev[l].lam, &bits[l], sizeof(double));
}

// Values only, for a matrix with the same pattern: the aggregates (and so P
// and every coarse pattern) are kept; the level-0 pressure matrix, every
// Galerkin product, the Gershgorin bounds and D^-1 of every level and the
// coarsest inverse are recomputed from the new values.
void refresh_hierarchy(trs_cpr *M, cudaStream_t s) {
  auto &lev = M->lev;
  Csr &C0 = lev[0].A;
  launch_ap_csr_fill(M->g, M->emask.p, M->tptr.p, M->tcol.p, M->ap_ell64.p, M->ap_tval64.p, C0.rp.p, C0.col.p,
                     C0.val.p, s);
  for (int l = 0; l < M->nlev; l++) {
    Level &F = lev[l];
    launch_gershgorin_dinv(F.A, F.dpos.p, F.dinv64.p, M->lam_bits.p + l, s);
    if (l + 1 < M->nlev)
      launch_galerkin(F.A, F.agg.p, F.n_agg, F.mptr.p, F.midx.p, lev[l + 1].A, s);
  }
  Level &C = lev[M->nlev - 1];
  TRS_REQUIRE(launch_dense_inverse(C.A, M->cinv, s) == 0, TRS_ERR_SINGULAR_BLOCK, "coarsest AMG matrix is singular");
  unsigned long long bits[kMaxLevels];
  TRS_CUDA(cudaMemcpyAsync(bits, M->lam_bits.p, M->nlev * sizeof(unsigned long long), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaStreamSynchronize(s));
  for (int l = 0; l < M->nlev; l++) std::memcpy(&lev[l].lam, &bits[l], sizeof(double));
}

void alloc_level_vectors(trs_cpr *M) {
  const size_t es = M->prec == TRS_FP32_PREC ? sizeof(float) : sizeof(double);
  for (int l = 0; l < M->nlev; l++) {
    Level &L = M->lev[l];
    const int64_t bytes = std::max<int64_t>(L.A.n, 1) * (int64_t)es;
    reserve(L.r, bytes);
    reserve(L.e, bytes);
    reserve(L.res, bytes);
    reserve(L.d, bytes);
    reserve(L.dn, bytes);
  }
}

// ------------------------------------------------------ block ILU(1)
// Distance-2 colours of a grid matrix: cell (x, y, z) takes (x + 2y + 3z)
// mod 7, which differs between any two cells one or two 7-point steps apart
// (the offsets are +-1, +-2, +-3 mod 7 and their pairwise sums, never 0 mod
// 7 for |sum| <= 6); the other rows, in index order, take the first colour
// from 7 on not taken by an earlier such row that is adjacent to them or
// shares a neighbour with them.
std::vector<int32_t> distance2_colours(const trs_bsr *A) {
  const int64_t n = A->n, nc = A->g.nc;
  const int64_t nx = A->g.nx, nxy = (int64_t)A->g.nx * A->g.ny;
  const auto &rp = A->h_rp;
  const auto &col = A->h_col;
  std::vector<int32_t> c(n);
  for (int64_t i = 0; i < nc; i++) c[i] = (int32_t)((i % nx + 2 * ((i / nx) % A->g.ny) + 3 * (i / nxy)) % 7);
  for (int64_t w = nc; w < n; w++) {
    uint64_t used = 0;
    for (int64_t p = rp[w]; p < rp[w + 1]; p++) {
      const int64_t k = col[p];
      if (k == w) continue;
      if (k >= nc && k < w) used |= 1ull << (c[k] - 7);
      for (int64_t q = rp[k]; q < rp[k + 1]; q++) {
        const int64_t j = col[q];
        if (j >= nc && j < w) used |= 1ull << (c[j] - 7);
      }
    }
    int f = 0;
    while (f < kMaxColours - 7 && ((used >> f) & 1ull)) f++;
    TRS_REQUIRE(f < kMaxColours - 7, TRS_ERR_UNSUPPORTED, "more than 64 colours needed");
    c[w] = 7 + f;
  }
  return c;
}

// The factor structure of block ILU(1), once per pattern, on the host: the
// level-1 fill of row i is every j, not already in row i, with a neighbour
// k of i ordered before both i and j ((i, k), (k, j) stored).  Fill blocks
// go to the fill slots of their row when they join two cells two 7-point
// steps apart, and otherwise to the tail of their row (sorted by column, no
// source block); all start from zero.  The parallel sweeps need the rows of
// one colour uncoupled in the resulting pattern, which is checked here.
void build_ilu1_structure(trs_cpr *M, const trs_bsr *A, const std::vector<int32_t> &colour, cudaStream_t s) {
  const int64_t n = M->n, nc = M->g.nc;
  const auto &rp = A->h_rp;
  const auto &col = A->h_col;
  const auto hpos = download(M->pos.p, n, s);
  const auto hcrow = download(M->crow.p, n, s);
  const auto htptr = download(M->tptr.p, n + 1, s);
  const auto htcol = download(M->tcol.p, M->ntail, s);
  const auto hem = download(M->emask.p, nc, s);
  std::vector<int64_t> fptr(n + 1, 0), stamp(n, -1);
  std::vector<int32_t> fcol;
  fcol.reserve((size_t)rp[n]);
  for (int64_t i = 0; i < n; i++) {
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      stamp[col[p]] = i;
      TRS_REQUIRE(col[p] == i || colour[col[p]] != colour[i], TRS_ERR_UNSUPPORTED,
                  "block ILU(1): two coupled rows share a colour (the order needs a 7-point grid)");
    }
    for (int64_t p = rp[i]; p < rp[i + 1]; p++) {
      const int64_t k = col[p];
      if (hpos[k] >= hpos[i]) continue;
      for (int64_t q = rp[k]; q < rp[k + 1]; q++) {
        const int64_t j = col[q];
        if (hpos[j] <= hpos[k] || stamp[j] == i) continue;
        stamp[j] = i;
        TRS_REQUIRE(colour[j] != colour[i], TRS_ERR_UNSUPPORTED,
                    "block ILU(1): level-1 fill couples two rows of one colour (the order needs a 7-point grid)");
        fcol.push_back((int32_t)j);
      }
    }
    fptr[i + 1] = (int64_t)fcol.size();
  }
  // fill slot of a cell-to-cell fill block (i, j), or -1: by the cells' grid displacement
  const int64_t nx = M->g.nx, ny = M->g.ny, nxy = nx * ny;
  auto fill_slot = [&](int64_t i, int64_t j) -> int {
    if (i >= nc || j >= nc) return -1;
    const int64_t dx = j % nx - i % nx, dy = (j / nx) % ny - (i / nx) % ny, dz = j / nxy - i / nxy;
    for (int f = 0; f < kFill; f++)
      if (kFillD[f][0] == dx && kFillD[f][1] == dy && kFillD[f][2] == dz) return f;
    return -1;
  };
  std::vector<int64_t> ftptr(n + 1, 0), ftsrc;
  std::vector<int32_t> ftcol;
  std::vector<uint8_t> ftlow, lmask(n);
  std::vector<uint32_t> fmask(n, 0u), flmask(n, 0u);
  const size_t total = (size_t)(M->ntail + fptr[n]);
  ftsrc.reserve(total);
  ftcol.reserve(total);
  ftlow.reserve(total);
  std::vector<std::pair<int32_t, int64_t>> row;
  for (int64_t q = 0; q < n; q++) {
    const int64_t i = hcrow[q];
    row.clear();
    for (int64_t t = htptr[i]; t < htptr[i + 1]; t++) row.push_back({htcol[t], t});
    for (int64_t u = fptr[i]; u < fptr[i + 1]; u++) {
      const int f = fill_slot(i, fcol[u]);
      if (f >= 0) {
        fmask[q] |= 1u << f;
        if (hpos[fcol[u]] < q) flmask[q] |= 1u << f;
      } else {
        row.push_back({fcol[u], -1});
      }
    }
    std::sort(row.begin(), row.end());
    for (const auto &e : row) {
      ftcol.push_back(e.first);
      ftsrc.push_back(e.second);
      ftlow.push_back(hpos[e.first] < q ? 1 : 0);
    }
    ftptr[q + 1] = (int64_t)ftcol.size();
    unsigned lm = 0;
    if (i < nc)
      for (int sl = 0; sl < kSlots; sl++)
        if (sl != kSelf && ((hem[i] >> sl) & 1u) && hpos[i + M->g.off[sl]] < q) lm |= 1u << sl;
    if (!row.empty()) lm |= kTailBit;
    lmask[q] = (uint8_t)lm;
  }
  M->nft = (int64_t)ftcol.size();
  M->ftptr.alloc(n + 1);
  M->ftptr.upload(ftptr.data(), n + 1, s);
  M->ftcol.alloc(std::max<size_t>(ftcol.size(), 1));
  M->ftcol.upload(ftcol.data(), ftcol.size(), s);
  M->ftlow.alloc(std::max<size_t>(ftlow.size(), 1));
  M->ftlow.upload(ftlow.data(), ftlow.size(), s);
  M->ftsrc.alloc(std::max<size_t>(ftsrc.size(), 1));
  M->ftsrc.upload(ftsrc.data(), ftsrc.size(), s);
  M->lmask.upload(lmask.data(), n, s);
  M->fmask.alloc(n);
  M->fmask.upload(fmask.data(), n, s);
  M->flmask.alloc(n);
  M->flmask.upload(flmask.data(), n, s);
  M->nfslots = kSlots + kFill;
  TRS_CUDA(cudaStreamSynchronize(s));
}

// ------------------------------------------------- long-row ILU plan
// Built once per pattern on the host from the colour-major structure: for
// every long row, its earlier-ordered entries in ascending position and the
// (k, j) pairs that update it (the same sets the IKJ factorisation visits).
void build_long_row_plan(trs_cpr *M, cudaStream_t s) {
  const int64_t n = M->n, nc = M->g.nc;
  const int bb = M->b * M->b;
  M->lr_col.assign(M->ncol, LongRowColour{});
  int64_t nlong = 0;
  for (int c = 0; c < M->ncol; c++) nlong += M->cptr[c + 1] - M->cmid[c];
  if (!nlong) return;
  const auto hpos = download(M->pos.p, n, s);
  const auto hft = download(M->ftptr.p, n + 1, s);
  const auto hcol = download(M->ftcol.p, M->nft, s);
  const auto hem = download(M->emask.p, nc, s);
  const auto hcrow = download(M->crow.p, n, s);
  const bool fill = M->nfslots > kSlots;
  const auto hfm = fill ? download(M->fmask.p, n, s) : std::vector<uint32_t>();
  std::vector<int64_t> Lptr{0}, Lpk, Pptr{0}, Psrc;
  std::vector<int32_t> diag, Lu, Pdst;
  std::vector<std::pair<int64_t, int32_t>> Ls;
  for (int c = 0; c < M->ncol; c++) {
    LongRowColour &pc = M->lr_col[c];
    pc.first = (int64_t)diag.size();
    for (int64_t q = M->cmid[c]; q < M->cptr[c + 1]; q++) {
      const int64_t i = hcrow[q], u0 = hft[q], u1 = hft[q + 1];
      auto local = [&](int64_t j) -> int32_t {
        const auto b0 = hcol.begin() + u0, b1 = hcol.begin() + u1;
        const auto it = std::lower_bound(b0, b1, (int32_t)j);
        return (it != b1 && *it == j) ? (int32_t)(it - b0) : -1;
      };
      diag.push_back(local(i));
      Ls.clear();
      for (int64_t u = u0; u < u1; u++) {
        const int64_t cj = hcol[u];
        if (cj != i && hpos[cj] < q) Ls.push_back({hpos[cj], (int32_t)(u - u0)});
      }
      std::sort(Ls.begin(), Ls.end());
      const int64_t pairs0 = (int64_t)Pdst.size();
      for (const auto &L : Ls) {
        const int64_t pk = L.first, kr = hcol[u0 + L.second];
        Lu.push_back(L.second);
        Lpk.push_back(pk);
        if (kr < nc) {
          const unsigned m = hem[kr];
          for (int s2 = 0; s2 < kSlots; s2++) {
            if (s2 == kSelf || !((m >> s2) & 1u)) continue;
            const int64_t j = kr + M->g.off[s2];
            if (hpos[j] <= pk) continue;
            const int32_t d = local(j);
            if (d < 0) continue;
            Pdst.push_back(d);
            Psrc.push_back(~(((int64_t)s2 * n + pk) * bb));
          }
          for (int f = 0; fill && f < kFill; f++) {
            if (!((hfm[pk] >> f) & 1u)) continue;
            const int64_t j = kr + M->g.off2[f];
            if (hpos[j] <= pk) continue;
            const int32_t d = local(j);
            if (d < 0) continue;
            Pdst.push_back(d);
            Psrc.push_back(~(((int64_t)(kSlots + f) * n + pk) * bb));
          }
        }
        for (int64_t uk = hft[pk]; uk < hft[pk + 1]; uk++) {
          const int64_t j = hcol[uk];
          if (j == kr || hpos[j] <= pk) continue;
          const int32_t d = local(j);
          if (d < 0) continue;
          Pdst.push_back(d);
          Psrc.push_back(uk * bb);
        }
        Pptr.push_back((int64_t)Pdst.size());
      }
      Lptr.push_back((int64_t)Lu.size());
      pc.max_ne = std::max<int64_t>(pc.max_ne, u1 - u0);
      pc.max_nl = std::max<int64_t>(pc.max_nl, (int64_t)Ls.size());
      pc.max_np = std::max<int64_t>(pc.max_np, (int64_t)Pdst.size() - pairs0);
    }
  }
  auto up = [&](auto &dst, const auto &src) {
    dst.alloc(std::max<size_t>(src.size(), 1));
    dst.upload(src.data(), src.size(), s);
  };
  up(M->lr_Lptr, Lptr);
  up(M->lr_diag, diag);
  up(M->lr_Lu, Lu);
  up(M->lr_Lpk, Lpk);
  up(M->lr_Pptr, Pptr);
  up(M->lr_Pdst, Pdst);
  up(M->lr_Psrc, Psrc);
  TRS_CUDA(cudaStreamSynchronize(s));
}

LongRowPlan long_row_plan(const trs_cpr *M) {
  LongRowPlan p;
  p.Lptr = M->lr_Lptr.p;
  p.diag = M->lr_diag.p;
  p.Lu = M->lr_Lu.p;
  p.Lpk = M->lr_Lpk.p;
  p.Pptr = M->lr_Pptr.p;
  p.Pdst = M->lr_Pdst.p;
  p.Psrc = M->lr_Psrc.p;
  return p;
}

// --------------------------------------------------- decoupling + ILU
void build_values(trs_cpr *M, const trs_bsr *A, bool rebuild_amg, cudaStream_t s) {
  const int b = M->b, bb = b * b;
  const int64_t n = M->n, nc = M->g.nc;
  TBuf<int> err(1, s);
  err.zero();
  const bool mixed = M->prec == TRS_FP32_PREC;
  const int mode = M->opts.decoupling;
  if (mixed)
    launch_decouple_mixed(b, A->view(), A->tdiag.p, mode, M->at_ell32.p, M->at_p32.p, M->at_tval32.p, M->dinv32.p,
                          M->ap_ell64.p, M->ap_tval64.p, err.p, s);
  else
    launch_decouple(b, A->view(), A->tdiag.p, mode, M->at_ell64.p, M->at_p64.p, M->at_tval64.p, M->dinv64.p,
                    M->ap_ell64.p, M->ap_tval64.p, err.p, s);
  // The block ILU factorisation (of Ã) and the AMG hierarchy (of A_p) are
  // independent once the decoupling is done: the factorisation runs on the
  // side stream while the hierarchy, latency-bound and synchronised with the
  // host level by level, is built on s; s waits for both at the end.
  if (!M->side) {
    TRS_CUDA(cudaStreamCreateWithFlags(&M->side, cudaStreamNonBlocking));
    TRS_CUDA(cudaEventCreateWithFlags(&M->ev_fork, cudaEventDisableTiming));
    TRS_CUDA(cudaEventCreateWithFlags(&M->ev_join, cudaEventDisableTiming));
  }
  cudaStream_t s2 = M->side;
  TRS_CUDA(cudaEventRecord(M->ev_fork, s));
  TRS_CUDA(cudaStreamWaitEvent(s2, M->ev_fork, 0));
  // On an error exit (a throw between the fork and the join) the side stream
  // may still read Ã and write the factors; it is drained before the caller
  // can queue new work that rewrites them.
  struct SideJoin {
    cudaStream_t st;
    bool armed;
    ~SideJoin() {
      if (armed) cudaStreamSynchronize(st);
    }
  } side_join{s2, true};
  TBuf<int> err2(1, s2);
  err2.zero();
  {
    const LongRowPlan plan = long_row_plan(M);
    const uint32_t *fm = M->nfslots > kSlots ? M->fmask.p : nullptr;
    if (mixed) {
      launch_ilu_init<float>(b, M->g, M->emask.p, M->crow.p, M->at_ell32.p, M->at_tval32.p, M->ftsrc.p, M->nft,
                             M->nfslots, M->fell32.p, M->ftval32.p, s2);
      for (int c = 0; c < M->ncol; c++)
        launch_ilu_factor_colour<float>(b, M->g, M->emask.p, M->crow.p, M->pos.p, M->ftptr.p, M->ftcol.p,
                                        M->ftlow.p, fm, M->fell32.p, M->ftval32.p, M->cptr[c], M->cmid[c],
                                        M->cptr[c + 1], &plan, M->lr_col.empty() ? nullptr : &M->lr_col[c],
                                        err2.p, s2);
    } else {
      launch_ilu_init<double>(b, M->g, M->emask.p, M->crow.p, M->at_ell64.p, M->at_tval64.p, M->ftsrc.p, M->nft,
                              M->nfslots, M->fell64.p, M->ftval64.p, s2);
      for (int c = 0; c < M->ncol; c++)
        launch_ilu_factor_colour<double>(b, M->g, M->emask.p, M->crow.p, M->pos.p, M->ftptr.p, M->ftcol.p,
                                         M->ftlow.p, fm, M->fell64.p, M->ftval64.p, M->cptr[c], M->cmid[c],
                                         M->cptr[c + 1], &plan, M->lr_col.empty() ? nullptr : &M->lr_col[c],
                                         err2.p, s2);
    }
  }
  TRS_CUDA(cudaEventRecord(M->ev_join, s2));
  if (rebuild_amg) {
    if (M->lev.empty()) M->lev.emplace_back();
    Csr &C0 = M->lev[0].A;
    C0.n = n;
    reserve(C0.rp, n + 1);
    TBuf<int64_t> len(n + 1, s);
    len.zero();
    launch_ap_csr_rowlen(M->g, M->emask.p, M->tptr.p, len.p, s);
    exclusive_scan(len.p, C0.rp.p, n + 1, nullptr, s);
    int herr0 = 0;
    TRS_CUDA(cudaMemcpyAsync(&C0.nnz, C0.rp.p + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaMemcpyAsync(&herr0, err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaStreamSynchronize(s));
    TRS_REQUIRE(!herr0, TRS_ERR_SINGULAR_BLOCK, "a diagonal block is singular");
    reserve(C0.col, C0.nnz);
    reserve(C0.val, C0.nnz);
    launch_ap_csr_fill(M->g, M->emask.p, M->tptr.p, M->tcol.p, M->ap_ell64.p, M->ap_tval64.p, C0.rp.p, C0.col.p,
                       C0.val.p, s);
    build_hierarchy(M, s);
    alloc_level_vectors(M);
  } else {
    refresh_hierarchy(M, s);
  }
  if (mixed) {
    auto cast = [&](DBuf<double> &src, DBuf<float> &dst, int64_t cnt) {
      reserve(dst, cnt);
      launch_cast<double, float>(src.p, dst.p, cnt, s);
    };
    cast(M->ap_ell64, M->ap_ell32, (int64_t)kSlots * nc);
    cast(M->ap_tval64, M->ap_tval32, M->ntail);
    for (int l = 0; l < M->nlev; l++) {
      Level &L = M->lev[l];
      cast(L.dinv64, L.dinv32, L.A.n);
      if (l > 0) cast(L.A.val, L.val32, L.A.nnz);
    }
  }
  TRS_CUDA(cudaStreamWaitEvent(s, M->ev_join, 0));
  side_join.armed = false;
  int herr[2] = {0, 0};
  TRS_CUDA(cudaMemcpyAsync(&herr[0], err.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaMemcpyAsync(&herr[1], err2.p, sizeof(int), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaStreamSynchronize(s));
  TRS_REQUIRE(!herr[0] && !herr[1], TRS_ERR_SINGULAR_BLOCK, "a singular diagonal or block ILU pivot block");
}

void setup_all(trs_cpr *M, const trs_bsr *A, cudaStream_t s) {
  const int b = A->b, bb = b * b;
  const int64_t n = A->n, nc = A->g.nc;
  M->b = b;
  M->n = n;
  M->N = n * b;
  M->g = A->g;
  M->ntail = A->ntail;
  M->nnzb = A->nnzb;
  keep_pool_memory();
  auto copy_d2d = [&](auto &dst, const auto &src, int64_t cnt) {
    using E = std::remove_reference_t<decltype(*src.p)>;
    dst.alloc(std::max<int64_t>(cnt, 1));
    if (cnt) TRS_CUDA(cudaMemcpyAsync(dst.p, src.p, cnt * sizeof(E), cudaMemcpyDeviceToDevice, s));
  };
  copy_d2d(M->emask, A->emask, nc);
  copy_d2d(M->tptr, A->tptr, n + 1);
  copy_d2d(M->tcol, A->tcol, A->ntail);
  copy_d2d(M->tdiag, A->tdiag, n - nc);
  copy_d2d(M->map, A->map, A->nnzb);
  if (M->prec == TRS_FP32_PREC) {
    M->at_ell32.alloc(std::max<int64_t>((int64_t)kSlots * bb * nc, 1));
    M->at_ell32.zero(s);
    M->at_p32.alloc(std::max<int64_t>((int64_t)kSlots * b * nc, 1));
    M->at_p32.zero(s);
    M->at_tval32.alloc(std::max<int64_t>(A->ntail * bb, 1));
    M->dinv32.alloc((size_t)bb * n);
  } else {
    M->at_ell64.alloc(std::max<int64_t>((int64_t)kSlots * bb * nc, 1));
    M->at_ell64.zero(s);
    M->at_p64.alloc(std::max<int64_t>((int64_t)kSlots * b * nc, 1));
    M->at_p64.zero(s);
    M->at_tval64.alloc(std::max<int64_t>(A->ntail * bb, 1));
    M->dinv64.alloc((size_t)bb * n);
  }
  M->ap_ell64.alloc(std::max<int64_t>((int64_t)kSlots * nc, 1));
  M->ap_ell64.zero(s);
  M->ap_tval64.alloc(std::max<int64_t>(A->ntail, 1));
  // colouring of the block pattern and the colour-major order
  M->colour.alloc(n);
  std::vector<int32_t> hcolour;
  if (M->opts.ilu_fill == TRS_ILU1) {
    hcolour = distance2_colours(A);
    M->colour.upload(hcolour.data(), n, s);
  } else {
    const int rounds = launch_colour(M->g, M->emask.p, M->tptr.p, M->tcol.p, M->opts.seed ^ kColourSeedXor,
                                     M->colour.p, s);
    TRS_REQUIRE(rounds >= 0, TRS_ERR_UNSUPPORTED, "more than 64 colours needed");
    hcolour = download(M->colour.p, n, s);
  }
  {
    int mx = 0;
    for (auto c : hcolour) mx = std::max(mx, c + 1);
    M->ncol = mx;
  }
  M->crow.alloc(n);
  M->pos.alloc(n);
  launch_colour_order(M->g, M->colour.p, M->ncol, M->cptr, M->cmid, M->crow.p, M->pos.p, s);
  M->lmask.alloc(n);
  if (M->opts.ilu_fill == TRS_ILU1) {
    build_ilu1_structure(M, A, hcolour, s);
  } else {
    launch_ilu_structure(M->g, M->emask.p, M->tptr.p, M->tcol.p, M->crow.p, M->pos.p, M->lmask.p, M->ftptr,
                         M->ftcol, M->ftlow, M->ftsrc, s);
    M->nft = M->ntail;
  }
  build_long_row_plan(M, s);
  if (M->prec == TRS_FP32_PREC) {
    M->fell32.alloc((size_t)M->nfslots * bb * n);
    M->ftval32.alloc(std::max<int64_t>(M->nft * bb, 1));
  } else {
    M->fell64.alloc((size_t)M->nfslots * bb * n);
    M->ftval64.alloc(std::max<int64_t>(M->nft * bb, 1));
  }
  build_values(M, A, true, s);
  // work vectors
  const size_t es = M->prec == TRS_FP32_PREC ? sizeof(float) : sizeof(double);
  alloc_vec(M->wf, M->N, es);
  alloc_vec(M->wy, M->N, es);
  alloc_vec(M->wr, M->N, es);
  alloc_vec(M->wx, M->N, es);
  alloc_vec(M->wz, M->N, es);
}

// ------------------------------------------------------------ application
template <class T>
struct Prec {
  static const T *dinv(const trs_cpr *M);
};

template <class T>
const T *atp_of(const trs_cpr *M) {
  if constexpr (std::is_same<T, float>::value) return M->at_p32.p;
  else return M->at_p64.p;
}

template <class T>
MatView<T> at_view(const trs_cpr *M) {
  MatView<T> v{M->g, M->emask.p, M->tptr.p, M->tcol.p, nullptr, nullptr};
  if constexpr (std::is_same<T, float>::value) { v.ell = M->at_ell32.p; v.tval = M->at_tval32.p; }
  else { v.ell = M->at_ell64.p; v.tval = M->at_tval64.p; }
  return v;
}

template <class T>
IluView<T> ilu_view(const trs_cpr *M) {
  IluView<T> v{M->g,    M->crow.p, M->emask.p, M->lmask.p, M->ftptr.p, M->ftcol.p, M->ftlow.p, nullptr, nullptr,
               M->nfslots > kSlots ? M->fmask.p : nullptr, M->nfslots > kSlots ? M->flmask.p : nullptr};
  if constexpr (std::is_same<T, float>::value) { v.fell = M->fell32.p; v.ftval = M->ftval32.p; }
  else { v.fell = M->fell64.p; v.ftval = M->ftval64.p; }
  return v;
}

template <class T>
const T *dinv_of(const trs_cpr *M) {
  if constexpr (std::is_same<T, float>::value) return M->dinv32.p;
  else return M->dinv64.p;
}

template <class T>
ScalarOp<T> level_op(const trs_cpr *M, int l) {
  ScalarOp<T> op{};
  const Level &L = M->lev[l];
  op.n = L.A.n;
  if (l == 0) {
    op.is_ell = 1;
    op.g = M->g;
    op.emask = M->emask.p;
    op.tptr = M->tptr.p;
    op.tcol = M->tcol.p;
    if constexpr (std::is_same<T, float>::value) { op.ell = M->ap_ell32.p; op.tval = M->ap_tval32.p; }
    else { op.ell = M->ap_ell64.p; op.tval = M->ap_tval64.p; }
  } else {
    op.is_ell = 0;
    op.rp = L.A.rp.p;
    op.col = L.A.col.p;
    if constexpr (std::is_same<T, float>::value) op.val = L.val32.p;
    else op.val = L.A.val.p;
  }
  return op;
}

template <class T>
const T *level_dinv(const Level &L) {
  if constexpr (std::is_same<T, float>::value) return L.dinv32.p;
  else return L.dinv64.p;
}

// Chebyshev smoothing of degree >= 2 (Saad, Alg. 12.1 on D^-1 A over
// [0.3 lam, lam]); zero_init starts from e = 0, with the first step fused
// into its initialisation.
template <class T>
void chebyshev(const trs_cpr *M, int l, const T *r, T *e, bool zero_init, cudaStream_t s) {
  const Level &L = M->lev[l];
  const ScalarOp<T> op = level_op<T>(M, l);
  const double alpha = 0.3 * L.lam, beta = L.lam;
  const double theta = (beta + alpha) / 2.0, delta = (beta - alpha) / 2.0;
  const double sigma = theta / delta;
  double rho = 1.0 / sigma;
  T *res = tp<T>(L.res), *d = tp<T>(L.d), *dn = tp<T>(L.dn);
  const T *dinv = level_dinv<T>(L);
  const int deg = M->opts.cheb_degree;
  int k = 1;
  if (zero_init) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const double c1 = rho_new * rho, c2 = (2.0 * rho_new) / delta;
    launch_cheb_first<T>(op, r, dinv, 1.0 / theta, c1, c2, res, d, dn, e, deg == 2, s);
    std::swap(d, dn);
    rho = rho_new;
    k = 2;
  } else {
    launch_cheb_resid_init<T>(op, r, e, dinv, 1.0 / theta, res, d, s);
  }
  for (; k < deg; k++) {
    const double rho_new = 1.0 / (2.0 * sigma - rho);
    const double c1 = rho_new * rho, c2 = (2.0 * rho_new) / delta;
    const int last = (k == deg - 1);
    launch_cheb_step<T>(op, res, res, d, dinv, c1, c2, dn, e, last, s);
    std::swap(d, dn);
    rho = rho_new;
  }
}

// First level handled by the single-block coarse kernel (rows <= 4096 on it
// and below), or nlev if none.
int coarse_fuse_level(const trs_cpr *M) {
  int l0 = M->nlev;
  while (l0 > 1 && M->lev[l0 - 1].A.n <= kCoarseFuseRows) l0--;
  return l0;
}

template <class T>
CoarseHierarchy<T> coarse_hierarchy(const trs_cpr *M, int l0) {
  CoarseHierarchy<T> h{};
  h.l0 = l0;
  h.nlev = M->nlev;
  h.deg = M->opts.cheb_degree;
  h.cinv = M->cinv.p;
  for (int l = l0; l < M->nlev; l++) {
    const Level &L = M->lev[l];
    CoarseLevel<T> &c = h.lv[l];
    c.n = L.A.n;
    c.rp = L.A.rp.p;
    c.col = L.A.col.p;
    if constexpr (std::is_same<T, float>::value) c.val = L.val32.p;
    else c.val = L.A.val.p;
    c.dinv = level_dinv<T>(L);
    c.agg = L.agg.p;
    c.mptr = L.mptr.p;
    c.midx = L.midx.p;
    const double alpha = 0.3 * L.lam, beta = L.lam;
    const double theta = (beta + alpha) / 2.0, delta = (beta - alpha) / 2.0;
    const double sigma = theta / delta;
    double rho = 1.0 / sigma;
    c.inv_theta = static_cast<T>(1.0 / theta);
    for (int k = 1; k < h.deg && k < kMaxCheb; k++) {
      const double rho_new = 1.0 / (2.0 * sigma - rho);
      c.c1[k] = static_cast<T>(rho_new * rho);
      c.c2[k] = static_cast<T>((2.0 * rho_new) / delta);
      rho = rho_new;
    }
    c.r = tp<T>(L.r);
    c.e = tp<T>(L.e);
    c.res = tp<T>(L.res);
    c.d = tp<T>(L.d);
    c.dn = tp<T>(L.dn);
  }
  return h;
}

template <class T>
void vcycle(const trs_cpr *M, int l, const T *r, T *e, cudaStream_t s) {
  const int L = M->nlev;
  const Level &Lv = M->lev[l];
  if (l == L - 1 && l == 0) {
    launch_dense_gemv<T>(Lv.A.n, M->cinv.p, r, e, s);
    return;
  }
  if (l > 0 && l == coarse_fuse_level(M)) {
    // r and e are this level's own buffers (written by the restriction above)
    launch_vcycle_coarse<T>(coarse_hierarchy<T>(M, l), s);
    return;
  }
  if (l == L - 1) {
    launch_dense_gemv<T>(Lv.A.n, M->cinv.p, r, e, s);
    return;
  }
  chebyshev<T>(M, l, r, e, true, s);
  const Level &C = M->lev[l + 1];
  launch_restrict_resid<T>(level_op<T>(M, l), C.A.n, Lv.mptr.p, Lv.midx.p, r, e, tp<T>(C.r), s);
  vcycle<T>(M, l + 1, tp<T>(C.r), tp<T>(C.e), s);
  launch_prolong<T>(Lv.A.n, Lv.agg.p, tp<T>(C.e), e, s);
  chebyshev<T>(M, l, r, e, false, s);
}

// The forward sweep starts at colour 1: the kernel that produced rhs also
// wrote y = rhs on the rows of colour 0, which have no earlier-ordered
// neighbour (the sweep of colour 0).  The rows of the last colour have no
// later-ordered neighbour, so their forward and backward sweeps are one pass.
template <class T, class TZ>
void ilu_solve(const trs_cpr *M, const T *rhs, T *y, const T *y1, const T *e0, TZ *zout, cudaStream_t s) {
  const IluView<T> F = ilu_view<T>(M);
  const int last = M->ncol - 1;
  for (int c = 1; c < last; c++) launch_ilu_fwd<T>(M->b, F, rhs, y, M->cptr[c], M->cmid[c], M->cptr[c + 1], s);
  for (int c = last; c >= 0; c--)
    launch_ilu_bwd<T, TZ>(M->b, F, y, M->cptr[c], M->cmid[c], M->cptr[c + 1], y1, e0, zout,
                          c == last ? rhs : nullptr, s);
}

// z = CPR(Ã)^-1 f (f already scaled by D^-1), written to z in FP64.  With F
// the block ILU(0) of Ã and P one AMG V-cycle on the pressure entries:
//   FPF: y = F^-1 f; e = P (f - Ã y)_p; z = y + Pi e + F^-1 (f - Ã (y + Pi e));
//   FP:  z = y + Pi e (the first two stages);
//   PF:  e = P f_p; z = Pi e + F^-1 (f - Ã Pi e).
template <class T>
void cpr_apply_scaled(const trs_cpr *M, double *z, cudaStream_t s) {
  T *f = tp<T>(M->wf), *y = tp<T>(M->wy), *r = tp<T>(M->wr), *x = tp<T>(M->wx);
  const Level &L0 = M->lev[0];
  const int unit = M->opts.decoupling == TRS_DEC_ABF || M->opts.decoupling == TRS_DEC_FRS_ABF;
  if (M->opts.stages == TRS_CPR_PF) {
    launch_pressure_of<T>(M->b, M->n, f, tp<T>(L0.r), s);
    vcycle<T>(M, 0, tp<T>(L0.r), tp<T>(L0.e), s);
    launch_resid_full<T>(M->b, at_view<T>(M), f, nullptr, tp<T>(L0.e), r, unit, M->colour.p, x, s);
    ilu_solve<T, double>(M, r, x, nullptr, tp<T>(L0.e), z, s);
    return;
  }
  ilu_solve<T, T>(M, f, y, nullptr, nullptr, (T *)nullptr, s);
  launch_resid_p<T>(M->b, at_view<T>(M), atp_of<T>(M), f, y, tp<T>(L0.r), unit, s);
  vcycle<T>(M, 0, tp<T>(L0.r), tp<T>(L0.e), s);
  if (M->opts.stages == TRS_CPR_FP) {
    launch_cpr_combine<T>(M->b, M->n, y, tp<T>(L0.e), z, s);
    return;
  }
  launch_resid_full<T>(M->b, at_view<T>(M), f, y, tp<T>(L0.e), r, unit, M->colour.p, x, s);
  ilu_solve<T, double>(M, r, x, y, tp<T>(L0.e), z, s);
}

template <class T>
void cpr_apply_full(const trs_cpr *M, const double *v, const double *div, double *vout, double *z, cudaStream_t s) {
  launch_dscale<T>(M->b, M->n, v, div, vout, dinv_of<T>(M), tp<T>(M->wf), M->colour.p, tp<T>(M->wy), s);
  cpr_apply_scaled<T>(M, z, s);
}

// Reduction scratch and norms shared by the Krylov solvers.
void ensure_reduction(trs_cpr *M) {
  if (M->red_grid > 0) return;
  const int64_t N = M->N;
  M->r.alloc(N);
  M->norms.alloc(4);
  M->status.alloc(2);
  M->red_grid = (int)std::min<int64_t>(kRedGridMax, std::max<int64_t>(1, (N + 255) / 256));
  M->partial.alloc((size_t)M->red_grid * (kMaxRestart + 16));
  M->counter.alloc(1);
  M->counter.zero(0);
  TRS_CUDA(cudaDeviceSynchronize());
}

// -------------------------------------------------------------- FGMRES
void ensure_workspace(trs_cpr *M, int m) {
  ensure_reduction(M);
  if (M->ws_m >= m) return;
  const int64_t N = M->N;
  M->V.alloc((size_t)(m + 1) * N);
  M->Z.alloc((size_t)m * N * sizeof(double));
  M->w.alloc(N);
  M->H.alloc((size_t)(m + 1) * m);
  M->cs.alloc(m);
  M->sn.alloc(m);
  M->gv.alloc(m + 1);
  M->h1.alloc(m + 2);
  M->h2.alloc(m + 2);
  M->hn2.alloc(2);
  M->hnorm.alloc(2);
  M->yv.alloc(m);
  TRS_CUDA(cudaDeviceSynchronize());
  M->ws_m = m;
}

// Optional device timing of the operator SpMV launches inside the Krylov
// solves, process-wide (trs_profile_spmv); the totals are taken from the
// phase events below.
struct SpmvProfile {
  bool on = false;
  double ms = 0.0;
  int64_t launches = 0;
};
SpmvProfile g_spmv_prof;
std::mutex g_prof_mutex;

// Phase timing of one solve (opts.time_phases or trs_profile_spmv): events
// recorded on the solve's stream between the phases of an iteration and read
// after the iteration's host synchronisation.  Phases: 0 preconditioner,
// 1 operator SpMV, 2 orthogonalisation / vector updates.
struct PhaseTimer {
  static constexpr int kEvents = 7;
  bool on = false;
  cudaEvent_t ev[kEvents] = {};
  double ms[3] = {0.0, 0.0, 0.0};
  int64_t spmv = 0;
  explicit PhaseTimer(bool enable) : on(enable) {
    if (on)
      for (auto &e : ev) TRS_CUDA(cudaEventCreate(&e));
  }
  PhaseTimer(const PhaseTimer &) = delete;
  PhaseTimer &operator=(const PhaseTimer &) = delete;
  ~PhaseTimer() {
    for (auto e : ev)
      if (e) cudaEventDestroy(e);
  }
  void mark(int k, cudaStream_t s) {
    if (on) TRS_CUDA(cudaEventRecord(ev[k], s));
  }
  void add(int phase, int from, int to) {
    if (!on) return;
    float t = 0.f;
    TRS_CUDA(cudaEventElapsedTime(&t, ev[from], ev[to]));
    ms[phase] += t;
  }
  void finish(trs_solve_stats &st) {
    if (!on) return;
    st.ms_precond = ms[0];
    st.ms_spmv = ms[1];
    st.ms_orth = ms[2];
    st.spmv_launches = spmv;
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    if (g_spmv_prof.on) {
      g_spmv_prof.ms += ms[1];
      g_spmv_prof.launches += spmv;
    }
  }
};

template <class T>
trs_status fgmres(const trs_bsr *A, trs_cpr *M, const double *b, double *x, const trs_solve_opts &o,
                  cudaStream_t s, trs_solve_stats *st) {
  const int m = o.restart;
  const int64_t N = M->N;
  ensure_workspace(M, m);
  const RedScratch red{M->partial.p, M->counter.p, M->red_grid};
  const MatView<double> Av = A->view();
  double *Z = tp<double>(M->Z);
  double *V = M->V.p;
  trs_solve_stats local{};
  PhaseTimer pt(o.time_phases != 0 || g_spmv_prof.on);
  Timer timer(s);
  launch_norm2(b, N, red, M->norms.p + 2, s);
  double hb[2];
  TRS_CUDA(cudaMemcpyAsync(hb, M->norms.p + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaStreamSynchronize(s));
  const double bnorm = hb[1];
  TRS_REQUIRE(std::isfinite(bnorm), TRS_ERR_NAN, "the right-hand side holds NaN or Inf");
  if (!o.use_x0) TRS_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
  trs_status result = TRS_ERR_NOT_CONVERGED;
  if (bnorm == 0.0) {
    TRS_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
    local.converged = 1;
    result = TRS_OK;
  }
  int iters = 0, cycles = 0;
  double relres = 0.0;
  bool x_zero = !o.use_x0;
  while (result != TRS_OK) {
    if (x_zero) {   // from x = 0 the residual is b itself: no SpMV
      TRS_CUDA(cudaMemcpyAsync(M->r.p, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      TRS_CUDA(cudaMemcpyAsync(M->norms.p, M->norms.p + 2, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
      x_zero = false;
    } else {
      launch_true_residual(M->b, Av, x, b, M->r.p, red, M->norms.p, s);
    }
    double hn[2];
    TRS_CUDA(cudaMemcpyAsync(hn, M->norms.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaStreamSynchronize(s));
    relres = hn[1] / bnorm;
    local.true_relres = relres;
    if (!std::isfinite(relres)) { result = TRS_ERR_NAN; break; }
    if (relres <= o.rtol) { result = TRS_OK; local.converged = 1; break; }
    if (iters >= o.maxit) break;
    TRS_CUDA(cudaMemsetAsync(M->gv.p, 0, (m + 1) * sizeof(double), s));
    TRS_CUDA(cudaMemcpyAsync(M->gv.p, M->norms.p + 1, sizeof(double), cudaMemcpyDeviceToDevice, s));
    int jdone = 0;
    bool breakdown = false;
    for (int j = 0; j < m; j++) {
      double *vj = V + (int64_t)j * N;
      double *zj = Z + (int64_t)j * N;
      pt.mark(0, s);
      if (j == 0) cpr_apply_full<T>(M, M->r.p, M->norms.p + 1, vj, zj, s);
      else cpr_apply_full<T>(M, M->w.p, M->hnorm.p, vj, zj, s);
      pt.mark(1, s);
      launch_spmv<double, double>(M->b, Av, zj, M->w.p, 1.0, 0.0, s);
      pt.mark(2, s);
      // CGS2: h1 = V^T w (and ||w||^2); w -= V h1 with h2 = V^T w fused; w -= V h2 with ||w||^2
      if (j + 2 <= 32) {
        launch_cgs_dots(V, N, j + 1, M->w.p, red, M->h1.p, s);
        launch_cgs_update_dots(V, N, j + 1, M->h1.p, M->w.p, red, M->h2.p, s);
      } else {
        launch_multidot(V, N, j + 1, M->w.p, red, M->h1.p, s);
        launch_cgs_update(V, N, j + 1, M->h1.p, M->w.p, 0, red, nullptr, s);
        launch_multidot(V, N, j + 1, M->w.p, red, M->h2.p, s);
      }
      launch_cgs_update(V, N, j + 1, M->h2.p, M->w.p, 1, red, M->hn2.p, s);
      launch_givens(j, m, M->H.p, M->h1.p, M->h2.p, M->hn2.p, M->h1.p + j + 1, M->cs.p, M->sn.p, M->gv.p,
                    M->hnorm.p, M->status.p, 1.0 / bnorm, s);
      pt.mark(3, s);
      iters++;
      double hs[2];
      TRS_CUDA(cudaMemcpyAsync(hs, M->status.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
      TRS_CUDA(cudaStreamSynchronize(s));
      pt.add(0, 0, 1);
      pt.add(1, 1, 2);
      pt.add(2, 2, 3);
      pt.spmv += pt.on;
      local.est_relres = hs[0];
      if (!std::isfinite(hs[0])) { result = TRS_ERR_NAN; break; }
      breakdown = hs[1] != 0.0;
      if (hs[0] <= o.rtol || iters >= o.maxit || breakdown) { jdone = j + 1; break; }
      jdone = j + 1;
    }
    if (result == TRS_ERR_NAN) break;
    launch_lsq(jdone, m, M->H.p, M->gv.p, M->yv.p, s);
    launch_xupdate<double>(Z, N, jdone, M->yv.p, x, s);
    cycles++;
    if (breakdown && local.est_relres > o.rtol) {
      // x is exact in the Krylov space; a last true-residual check follows
    }
  }
  local.iters = iters;
  local.restarts = cycles > 0 ? cycles - 1 : 0;
  local.amg_levels = M->nlev;
  local.n_colours = M->ncol;
  local.ms_setup = M->ms_setup;
  local.ms_solve = timer.stop();
  pt.finish(local);
  if (st) *st = local;
  return result;
}

// ------------------------------------------------------------ BiCGSTAB
// Right-preconditioned BiCGSTAB (van der Vorst), the Krylov method of the
// paper's runs, with M^-1 = CPR(Ã)^-1 D^-1:
//   p = r + beta (p - omega v);  p^ = M^-1 p;  v = A p^;  alpha = rho / <r^, v>;
//   s = r - alpha v;  s^ = M^-1 s;  t = A s^;  omega = <t, s> / <t, t>;
//   x += alpha p^ + omega s^;  r = s - omega t;  rho' = <r^, r>.
// When ||s|| already meets the tolerance the step ends with x += alpha p^.
// A cycle ends when the recurrence residual meets the tolerance or on
// breakdown (rho = 0 or omega = 0); the next cycle starts from the true FP64
// residual, with r^ = r, and the solve stops only when that meets rtol.
void ensure_bicg(trs_cpr *M) {
  ensure_reduction(M);
  if (M->bw.n) return;
  M->bw.alloc((size_t)7 * M->N);
  M->bsc.alloc(sizeof(BicgScalars) / sizeof(double));
  M->bpart.alloc((size_t)2 * std::max<int64_t>(1, bicg_spmv_blocks(M->g)));
  TRS_CUDA(cudaDeviceSynchronize());
}

template <class T>
trs_status bicgstab(const trs_bsr *A, trs_cpr *M, const double *b, double *x, const trs_solve_opts &o,
                    cudaStream_t s, trs_solve_stats *st) {
  const int64_t N = M->N;
  ensure_bicg(M);
  const RedScratch red{M->partial.p, M->counter.p, M->red_grid};
  const MatView<double> Av = A->view();
  double *r = M->r.p, *rh = M->bw.p, *p = rh + N, *v = p + N, *ph = v + N, *sv = ph + N, *sh = sv + N,
         *t = sh + N;
  BicgScalars *sc = reinterpret_cast<BicgScalars *>(M->bsc.p);
  trs_solve_stats local{};
  PhaseTimer pt(o.time_phases != 0 || g_spmv_prof.on);
  Timer timer(s);
  launch_norm2(b, N, red, M->norms.p + 2, s);
  double hb[2];
  TRS_CUDA(cudaMemcpyAsync(hb, M->norms.p + 2, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
  TRS_CUDA(cudaStreamSynchronize(s));
  const double bnorm = hb[1];
  TRS_REQUIRE(std::isfinite(bnorm), TRS_ERR_NAN, "the right-hand side holds NaN or Inf");
  if (!o.use_x0 || bnorm == 0.0) TRS_CUDA(cudaMemsetAsync(x, 0, N * sizeof(double), s));
  trs_status result = TRS_ERR_NOT_CONVERGED;
  int iters = 0, cycles = 0;
  bool breakdown = false;
  if (bnorm == 0.0) {
    local.converged = 1;
    result = TRS_OK;
  }
  bool x_zero = !o.use_x0;
  while (result != TRS_OK) {
    if (x_zero) {   // from x = 0 the residual is b itself: no SpMV
      TRS_CUDA(cudaMemcpyAsync(r, b, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
      TRS_CUDA(cudaMemcpyAsync(M->norms.p, M->norms.p + 2, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
      x_zero = false;
    } else {
      launch_true_residual(M->b, Av, x, b, r, red, M->norms.p, s);
    }
    double hn[2];
    TRS_CUDA(cudaMemcpyAsync(hn, M->norms.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaStreamSynchronize(s));
    const double relres = hn[1] / bnorm;
    local.true_relres = relres;
    if (!std::isfinite(relres)) { result = TRS_ERR_NAN; break; }
    if (relres <= o.rtol) { result = TRS_OK; local.converged = 1; break; }
    if (iters >= o.maxit) break;
    TRS_CUDA(cudaMemcpyAsync(rh, r, N * sizeof(double), cudaMemcpyDeviceToDevice, s));
    launch_bicg_start(sc, M->norms.p, bnorm, o.rtol, s);
    cycles++;
    breakdown = false;
    for (int k = 0; iters < o.maxit; k++) {
      pt.mark(0, s);
      launch_bicg_dir<T>(M->b, M->n, r, v, p, sc, k == 0, dinv_of<T>(M), tp<T>(M->wf), M->colour.p, tp<T>(M->wy), s);
      cpr_apply_scaled<T>(M, ph, s);
      pt.mark(1, s);
      launch_bicg_spmv(M->b, Av, ph, v, rh, 1, M->bpart.p, M->counter.p, sc, s);
      pt.mark(2, s);
      launch_bicg_s(N, r, v, sv, red, sc, s);
      pt.mark(3, s);
      launch_dscale<T>(M->b, M->n, sv, nullptr, nullptr, dinv_of<T>(M), tp<T>(M->wf), M->colour.p, tp<T>(M->wy), s);
      cpr_apply_scaled<T>(M, sh, s);
      pt.mark(4, s);
      launch_bicg_spmv(M->b, Av, sh, t, sv, 2, M->bpart.p, M->counter.p, sc, s);
      pt.mark(5, s);
      launch_bicg_xr(N, ph, sh, sv, t, rh, x, r, red, sc, s);
      pt.mark(6, s);
      iters++;
      BicgScalars h;
      TRS_CUDA(cudaMemcpyAsync(&h, sc, sizeof(h), cudaMemcpyDeviceToHost, s));
      TRS_CUDA(cudaStreamSynchronize(s));
      pt.add(0, 0, 1);
      pt.add(0, 3, 4);
      pt.add(1, 1, 2);
      pt.add(1, 4, 5);
      pt.add(2, 2, 3);
      pt.add(2, 5, 6);
      pt.spmv += 2 * pt.on;
      const double est = std::sqrt(h.rr) / bnorm;
      local.est_relres = est;
      if (!std::isfinite(est) || !std::isfinite(h.rho)) { breakdown = true; break; }
      if (est <= o.rtol) break;
      if (h.omega == 0.0 || h.rho == 0.0) { breakdown = true; break; }
    }
  }
  local.iters = iters;
  local.restarts = cycles > 0 ? cycles - 1 : 0;
  local.amg_levels = M->nlev;
  local.n_colours = M->ncol;
  local.ms_setup = M->ms_setup;
  local.ms_solve = timer.stop();
  pt.finish(local);
  if (st) *st = local;
  return result;
}

trs_status run_solve(const trs_bsr *A, trs_cpr *M, const double *b, double *x, const trs_solve_opts *opts,
                     cudaStream_t s, trs_solve_stats *st) {
  trs_solve_opts o;
  trs_solve_default_opts(&o);
  if (opts) o = *opts;
  TRS_REQUIRE(A && M && b && x, TRS_ERR_INVALID, "NULL argument");
  TRS_REQUIRE(A->n == M->n && A->b == M->b, TRS_ERR_INVALID, "matrix and preconditioner sizes differ");
  require_aligned(b, "b");
  require_aligned(x, "x");
  TRS_REQUIRE(o.restart >= 1 && o.restart <= kMaxRestart, TRS_ERR_INVALID, "restart must be 1..64");
  TRS_REQUIRE(o.maxit >= 1 && o.rtol > 0.0, TRS_ERR_INVALID, "maxit must be >= 1 and rtol > 0");
  TRS_REQUIRE(o.method == TRS_FGMRES || o.method == TRS_BICGSTAB, TRS_ERR_INVALID,
              "method must be TRS_FGMRES or TRS_BICGSTAB");
  if (o.method == TRS_BICGSTAB) {
    if (M->prec == TRS_FP32_PREC) return bicgstab<float>(A, M, b, x, o, s, st);
    return bicgstab<double>(A, M, b, x, o, s, st);
  }
  if (M->prec == TRS_FP32_PREC) return fgmres<float>(A, M, b, x, o, s, st);
  return fgmres<double>(A, M, b, x, o, s, st);
}

trs_status solve_entry(const trs_bsr *A, const trs_cpr *M, const double *b, double *x, const trs_solve_opts *opts,
                       int method, cudaStream_t s, trs_solve_stats *stats) {
  trs_status st = TRS_OK;
  trs_status g = guarded([&] {
    trs_solve_opts o;
    trs_solve_default_opts(&o);
    if (opts) o = *opts;
    if (method >= 0) o.method = method;
    st = run_solve(A, const_cast<trs_cpr *>(M), b, x, &o, s, stats);
  });
  if (g != TRS_OK) return g;
  if (st == TRS_ERR_NOT_CONVERGED) set_last_error("iteration limit reached before the tolerance");
  if (st == TRS_ERR_NAN) set_last_error("NaN or Inf in a residual norm");
  return st;
}

trs_status solve_host_entry(const trs_bsr *A, const trs_cpr *M, const double *b_host, double *x_host,
                            const trs_solve_opts *opts, int method, cudaStream_t s, trs_solve_stats *stats) {
  trs_status st = TRS_OK;
  trs_status g = guarded([&] {
    TRS_REQUIRE(A && M && b_host && x_host, TRS_ERR_INVALID, "NULL argument");
    // device copies of b and x, kept by the handle after the first call
    trs_cpr *Mw = const_cast<trs_cpr *>(M);
    if ((int64_t)Mw->host_bx.n < 2 * M->N) Mw->host_bx.alloc((size_t)2 * M->N);
    double *db = Mw->host_bx.p, *dx = db + M->N;
    TRS_CUDA(cudaMemcpyAsync(db, b_host, M->N * sizeof(double), cudaMemcpyHostToDevice, s));
    trs_solve_opts o;
    trs_solve_default_opts(&o);
    if (opts) o = *opts;
    if (method >= 0) o.method = method;
    if (o.use_x0) TRS_CUDA(cudaMemcpyAsync(dx, x_host, M->N * sizeof(double), cudaMemcpyHostToDevice, s));
    st = run_solve(A, Mw, db, dx, &o, s, stats);
    TRS_CUDA(cudaMemcpyAsync(x_host, dx, M->N * sizeof(double), cudaMemcpyDeviceToHost, s));
    TRS_CUDA(cudaStreamSynchronize(s));
  });
  return g != TRS_OK ? g : st;
}

}  // namespace

void set_last_error(const std::string &msg) { g_last_error = msg; }

namespace {
std::atomic<uint64_t> g_launches{0};
}
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

}  // namespace trs

using namespace trs;

extern "C" {

void trs_cpr_default_opts(trs_cpr_opts *o) {
  if (!o) return;
  o->precision = TRS_FP64;
  o->theta = 0.08;
  o->coarse_max = 64;
  o->max_levels = 12;
  o->cheb_degree = 2;
  o->seed = 0x5EED1812u;
  o->stages = TRS_CPR_FPF;
  o->decoupling = TRS_DEC_ABF;
  o->ilu_fill = TRS_ILU0;
}

void trs_solve_default_opts(trs_solve_opts *o) {
  if (!o) return;
  o->rtol = 1e-6;
  o->restart = 30;
  o->maxit = 1000;
  o->use_x0 = 0;
  o->method = TRS_FGMRES;
  o->time_phases = 0;
}

trs_status trs_cpr_setup(const trs_bsr *A, const trs_cpr_opts *opts, void *stream, trs_cpr **out) {
  return guarded([&] {
    TRS_REQUIRE(A && out, TRS_ERR_INVALID, "NULL argument");
    *out = nullptr;
    trs_cpr_opts o;
    trs_cpr_default_opts(&o);
    if (opts) o = *opts;
    TRS_REQUIRE(o.precision == TRS_FP64 || o.precision == TRS_FP32_PREC, TRS_ERR_INVALID, "unknown precision");
    TRS_REQUIRE(o.cheb_degree >= 2 && o.cheb_degree <= 8, TRS_ERR_UNSUPPORTED, "Chebyshev degree must be 2..8");
    TRS_REQUIRE(o.max_levels >= 1 && o.max_levels <= kMaxLevels, TRS_ERR_INVALID, "max_levels must be 1..16");
    TRS_REQUIRE(o.coarse_max >= 1 && o.coarse_max <= kDenseMax, TRS_ERR_INVALID, "coarse_max must be 1..4096");
    TRS_REQUIRE(o.stages >= TRS_CPR_FPF && o.stages <= TRS_CPR_PF, TRS_ERR_INVALID,
                "stages must be TRS_CPR_FPF, TRS_CPR_FP or TRS_CPR_PF");
    TRS_REQUIRE(o.decoupling >= TRS_DEC_ABF && o.decoupling <= TRS_DEC_FRS_ABF, TRS_ERR_INVALID,
                "decoupling must be TRS_DEC_ABF, TRS_DEC_NONE, TRS_DEC_FRS or TRS_DEC_FRS_ABF");
    TRS_REQUIRE(o.ilu_fill == TRS_ILU0 || o.ilu_fill == TRS_ILU1, TRS_ERR_INVALID,
                "ilu_fill must be TRS_ILU0 or TRS_ILU1");
    TRS_REQUIRE(o.ilu_fill == TRS_ILU0 || A->structured, TRS_ERR_UNSUPPORTED,
                "block ILU(1) needs a matrix created with grid dimensions");
    cudaStream_t s = (cudaStream_t)stream;
    auto M = std::make_unique<trs_cpr>();
    M->opts = o;
    M->prec = o.precision;
    Timer t(s);
    setup_all(M.get(), A, s);
    M->ms_setup = t.stop();
    *out = M.release();
  });
}

trs_status trs_cpr_update(trs_cpr *M, const trs_bsr *A, int32_t reuse_amg, void *stream) {
  return guarded([&] {
    TRS_REQUIRE(M && A, TRS_ERR_INVALID, "NULL argument");
    TRS_REQUIRE(A->n == M->n && A->b == M->b && A->nnzb == M->nnzb, TRS_ERR_INVALID, "pattern differs");
    cudaStream_t s = (cudaStream_t)stream;
    Timer t(s);
    build_values(M, A, reuse_amg == 0, s);
    M->ms_setup = t.stop();
  });
}

trs_status trs_cpr_apply(const trs_cpr *M, const double *v, double *z, void *stream) {
  return guarded([&] {
    TRS_REQUIRE(M && v && z, TRS_ERR_INVALID, "NULL argument");
    require_aligned(v, "v");
    require_aligned(z, "z");
    cudaStream_t s = (cudaStream_t)stream;
    if (M->prec == TRS_FP32_PREC) {
      cpr_apply_full<float>(M, v, nullptr, nullptr, z, s);
    } else {
      cpr_apply_full<double>(M, v, nullptr, nullptr, z, s);
    }
  });
}

trs_status trs_cpr_vcycle(const trs_cpr *M, const double *r, double *e, void *stream) {
  return guarded([&] {
    TRS_REQUIRE(M && r && e, TRS_ERR_INVALID, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const Level &L0 = M->lev[0];
    if (M->prec == TRS_FP32_PREC) {
      launch_cast<double, float>(r, tp<float>(L0.r), L0.A.n, s);
      vcycle<float>(M, 0, tp<float>(L0.r), tp<float>(L0.e), s);
      launch_cast<float, double>(tp<float>(L0.e), e, L0.A.n, s);
    } else {
      vcycle<double>(M, 0, r, e, s);
    }
  });
}

trs_status trs_cpr_get_info(const trs_cpr *M, trs_cpr_info *info) {
  return guarded([&] {
    TRS_REQUIRE(M && info, TRS_ERR_INVALID, "NULL argument");
    std::memset(info, 0, sizeof(*info));
    info->n_levels = M->nlev;
    info->n_colours = M->ncol;
    info->precision = M->prec;
    for (int l = 0; l < M->nlev && l < 16; l++) {
      info->level_rows[l] = M->lev[l].A.n;
      info->level_nnz[l] = M->lev[l].A.nnz;
      info->level_lambda[l] = M->lev[l].lam;
    }
  });
}

trs_status trs_cpr_get_aggregates(const trs_cpr *M, int32_t level, int32_t *agg) {
  return guarded([&] {
    TRS_REQUIRE(M && agg, TRS_ERR_INVALID, "NULL argument");
    TRS_REQUIRE(level >= 0 && level < M->nlev, TRS_ERR_INVALID, "level out of range");
    const Level &L = M->lev[level];
    if (level < M->nlev - 1) {
      auto h = download(L.agg.p, L.A.n, 0);
      std::copy(h.begin(), h.end(), agg);
    } else {
      std::fill(agg, agg + L.A.n, -1);
    }
  });
}

trs_status trs_cpr_get_colours(const trs_cpr *M, int32_t *colour) {
  return guarded([&] {
    TRS_REQUIRE(M && colour, TRS_ERR_INVALID, "NULL argument");
    auto h = download(M->colour.p, M->n, 0);
    std::copy(h.begin(), h.end(), colour);
  });
}

trs_status trs_cpr_get_decoupled(const trs_cpr *M, double *vt, double *dinv) {
  return guarded([&] {
    TRS_REQUIRE(M, TRS_ERR_INVALID, "NULL argument");
    const int bb = M->b * M->b;
    const bool mixed = M->prec == TRS_FP32_PREC;
    DBuf<double> ell64, tval64, dinv64;
    const double *ellp = M->at_ell64.p, *tvalp = M->at_tval64.p, *dinvp = M->dinv64.p;
    if (mixed) {  // FP32 copies, widened
      ell64.alloc(M->at_ell32.n);
      tval64.alloc(M->at_tval32.n);
      dinv64.alloc(M->dinv32.n);
      launch_cast<float, double>(M->at_ell32.p, ell64.p, M->at_ell32.n, 0);
      launch_cast<float, double>(M->at_tval32.p, tval64.p, M->at_tval32.n, 0);
      launch_cast<float, double>(M->dinv32.p, dinv64.p, M->dinv32.n, 0);
      ellp = ell64.p;
      tvalp = tval64.p;
      dinvp = dinv64.p;
    }
    if (vt) {
      DBuf<double> stage(std::max<int64_t>(M->nnzb * bb, 1));
      launch_gather_values(M->nnzb, bb, M->map.p, ellp, tvalp, M->g.nc, stage.p, 0, /*aos=*/1);
      auto h = download(stage.p, M->nnzb * bb, 0);
      std::copy(h.begin(), h.end(), vt);
    }
    if (dinv) {
      auto h = download(dinvp, (size_t)bb * M->n, 0);
      for (int64_t i = 0; i < M->n; i++)
        for (int e = 0; e < bb; e++) dinv[i * bb + e] = h[(size_t)e * M->n + i];
    }
  });
}

trs_status trs_cpr_get_level(const trs_cpr *M, int32_t level, int64_t *row_ptr, int32_t *col, double *val) {
  return guarded([&] {
    TRS_REQUIRE(M && row_ptr && col && val, TRS_ERR_INVALID, "NULL argument");
    TRS_REQUIRE(level >= 0 && level < M->nlev, TRS_ERR_INVALID, "level out of range");
    const Csr &C = M->lev[level].A;
    auto a = download(C.rp.p, C.n + 1, 0);
    auto b = download(C.col.p, C.nnz, 0);
    auto c = download(C.val.p, C.nnz, 0);
    std::copy(a.begin(), a.end(), row_ptr);
    std::copy(b.begin(), b.end(), col);
    std::copy(c.begin(), c.end(), val);
  });
}

void trs_cpr_destroy(trs_cpr *M) { delete M; }

trs_status trs_fgmres_solve(const trs_bsr *A, const trs_cpr *M, const double *b, double *x,
                            const trs_solve_opts *opts, void *stream, trs_solve_stats *stats) {
  return solve_entry(A, M, b, x, opts, TRS_FGMRES, (cudaStream_t)stream, stats);
}

trs_status trs_fgmres_solve_host(const trs_bsr *A, const trs_cpr *M, const double *b_host, double *x_host,
                                 const trs_solve_opts *opts, void *stream, trs_solve_stats *stats) {
  return solve_host_entry(A, M, b_host, x_host, opts, TRS_FGMRES, (cudaStream_t)stream, stats);
}

trs_status trs_bicgstab_solve(const trs_bsr *A, const trs_cpr *M, const double *b, double *x,
                              const trs_solve_opts *opts, void *stream, trs_solve_stats *stats) {
  return solve_entry(A, M, b, x, opts, TRS_BICGSTAB, (cudaStream_t)stream, stats);
}

trs_status trs_bicgstab_solve_host(const trs_bsr *A, const trs_cpr *M, const double *b_host, double *x_host,
                                   const trs_solve_opts *opts, void *stream, trs_solve_stats *stats) {
  return solve_host_entry(A, M, b_host, x_host, opts, TRS_BICGSTAB, (cudaStream_t)stream, stats);
}

trs_status trs_solve_adjoint(const trs_bsr *A, const trs_bsr *AT, const trs_cpr *M_T, const double *g,
                             const double *x, double *lambda, double *dA, const trs_solve_opts *opts, void *stream,
                             trs_solve_stats *stats) {
  trs_status st = TRS_OK;
  trs_status gs = guarded([&] {
    TRS_REQUIRE(A && AT && M_T && g && lambda, TRS_ERR_INVALID, "NULL argument");
    TRS_REQUIRE(AT->n == A->n && AT->b == A->b && AT->nnzb == A->nnzb, TRS_ERR_INVALID, "AT is not A^T-shaped");
    cudaStream_t s = (cudaStream_t)stream;
    st = run_solve(AT, const_cast<trs_cpr *>(M_T), g, lambda, opts, s, stats);
    if (dA) {
      TRS_REQUIRE(x, TRS_ERR_INVALID, "x is required for dA");
      launch_outer_product(A->b, *A, lambda, x, dA, s);
    }
  });
  return gs != TRS_OK ? gs : st;
}

trs_status trs_outer_product(const trs_bsr *A, const double *lambda, const double *x, double *dA, void *stream) {
  return guarded([&] {
    TRS_REQUIRE(A && lambda && x && dA, TRS_ERR_INVALID, "NULL argument");
    launch_outer_product(A->b, *A, lambda, x, dA, (cudaStream_t)stream);
  });
}

trs_status trs_chain_theta(const trs_bsr *A, const double *perm, int32_t perm_is_log, double kvkh, double c_t,
                           const double *M, const double *lambda, const double *x, double *dtheta, void *stream) {
  return guarded([&] {
    TRS_REQUIRE(A && perm && M && lambda && x && dtheta, TRS_ERR_INVALID, "NULL argument");
    TRS_REQUIRE(A->structured, TRS_ERR_INVALID, "the chain needs a structured (grid) matrix");
    launch_chain_theta(A->b, *A, perm, perm_is_log, kvkh, c_t, M, lambda, x, dtheta, (cudaStream_t)stream);
  });
}

const char *trs_last_error(void) { return g_last_error.c_str(); }

const char *trs_version(void) { return "trs 0.1 (sm_103a)"; }

uint64_t trs_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

trs_status trs_profile_spmv(int32_t enable, double *total_ms, int64_t *launches) {
  return guarded([&] {
    std::lock_guard<std::mutex> lock(g_prof_mutex);
    if (total_ms) *total_ms = g_spmv_prof.ms;
    if (launches) *launches = g_spmv_prof.launches;
    if (enable) {
      g_spmv_prof.ms = 0.0;
      g_spmv_prof.launches = 0;
    }
    g_spmv_prof.on = enable != 0;
  });
}

}  // extern "C"
