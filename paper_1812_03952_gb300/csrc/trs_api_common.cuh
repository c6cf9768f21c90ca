// Shared host-side pieces of the C ABI implementation: error capture and
// the preconditioner handle.
#pragma once

#include <memory>

#include "trs_kernels.cuh"

namespace trs {

void set_last_error(const std::string &msg);

// Runs f, converting any exception into a status code and a thread-local
// message; no exception crosses the C boundary.
template <class F>
trs_status guarded(F &&f) {
  try {
    f();
    return TRS_OK;
  } catch (const Error &e) {
    set_last_error(e.what());
    return e.code;
  } catch (const std::bad_alloc &) {
    set_last_error("host allocation failed");
    return TRS_ERR_OOM;
  } catch (const std::exception &e) {
    set_last_error(e.what());
    return TRS_ERR_INVALID;
  }
}

void validate_pattern(int64_t n, int b, const int64_t *rp, const int32_t *col);

// Device vectors are read and written with 128-bit accesses.
inline void require_aligned(const void *p, const char *what) {
  TRS_REQUIRE(((uintptr_t)p & 15u) == 0, TRS_ERR_INVALID, std::string(what) + " must be 16-byte aligned");
}
void build_layout(trs_bsr *A, int64_t n, int b, const int64_t *rp, const int32_t *col, const int32_t *grid,
                  cudaStream_t s);
void upload_values(trs_bsr *A, const double *values, bool on_device, cudaStream_t s);

// One level of the pressure hierarchy.
struct Level {
  Csr A;                       // FP64 operator (level 0: CSR copy used by the setup only)
  DBuf<float> val32;           // FP32 values of A (levels >= 1, mixed precision)
  DBuf<int64_t> dpos;
  DBuf<double> dval;           // diagonal values (for the strength test)
  DBuf<int32_t> agg;           // aggregate of each row in the next level (not on the coarsest)
  int64_t n_agg = 0;
  DBuf<int64_t> mptr;          // members of each next-level aggregate, ascending
  DBuf<int32_t> midx;
  DBuf<double> dinv64;
  DBuf<float> dinv32;
  double lam = 0.0;
  // work vectors in the preconditioner precision
  DBuf<char> r, e, res, d, dn;
};

}  // namespace trs

struct trs_cpr {
  int prec = TRS_FP64;
  int b = 0;
  int64_t n = 0, N = 0, ntail = 0, nnzb = 0;
  trs::Geom g{};
  trs_cpr_opts opts{};
  // copy of the matrix pattern
  trs::DBuf<uint8_t> emask;
  trs::DBuf<int64_t> tptr, tdiag, map;
  trs::DBuf<int32_t> tcol;
  // decoupled matrix (ELL part [7][nc][bb], blocks contiguous), D^-1 ([bb][n]) and the
  // level-0 pressure matrix
  trs::DBuf<double> at_ell64, at_tval64, dinv64, ap_ell64, ap_tval64;
  trs::DBuf<float> at_ell32, at_tval32, dinv32, ap_ell32, ap_tval32;
  trs::DBuf<double> at_p64;    // pressure rows of Ã's ELL part, [7][b][nc] (the first-stage residual)
  trs::DBuf<float> at_p32;
  // pressure AMG
  std::vector<trs::Level> lev;   // lev[0 .. nlev-1] active; extra entries keep their buffers
  int nlev = 0;
  trs::DBuf<unsigned long long> lam_bits;
  trs::DBuf<double> cinv;      // inverse of the coarsest operator
  // multicolour block ILU(0)
  int ncol = 0;
  std::vector<int64_t> cptr, cmid;
  trs::DBuf<int32_t> colour, crow;
  trs::DBuf<int64_t> pos, ftptr, ftsrc;
  trs::DBuf<int32_t> ftcol;
  trs::DBuf<uint8_t> lmask, ftlow;
  trs::DBuf<uint32_t> fmask, flmask;   // ILU(1) fill slots by position
  int nfslots = trs::kSlots;           // factor slots per position: 7, or 7 + 18 with ILU(1)
  int64_t nft = 0;
  trs::DBuf<double> fell64, ftval64;
  trs::DBuf<float> fell32, ftval32;
  // symbolic IKJ plan of the long rows (see trs::LongRowPlan)
  trs::DBuf<int64_t> lr_Lptr, lr_Lpk, lr_Pptr, lr_Psrc;
  trs::DBuf<int32_t> lr_diag, lr_Lu, lr_Pdst;
  std::vector<trs::LongRowColour> lr_col;
  // preconditioner work vectors (precision of the preconditioner)
  trs::DBuf<char> wf, wy, wr, wx, wz;
  // Krylov workspace, sized on first use
  int ws_m = 0;
  trs::DBuf<double> V, w, r, H, cs, sn, gv, h1, h2, hn2, hnorm, status, yv, norms;
  trs::DBuf<char> Z;
  trs::DBuf<double> bw, bsc, bpart;   // BiCGSTAB vectors (r^, p, v, p^, s, s^, t), scalars, SpMV partials
  trs::DBuf<double> host_bx;          // device copies of b and x for the host-buffer solves (2 N)
  trs::DBuf<double> partial;
  trs::DBuf<unsigned int> counter;
  int red_grid = 0;
  double ms_setup = 0.0;
  // side stream of the setup: the block ILU factorisation runs on it while
  // the AMG hierarchy is built on the caller's stream
  cudaStream_t side = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
  trs_cpr() = default;
  trs_cpr(const trs_cpr &) = delete;
  trs_cpr &operator=(const trs_cpr &) = delete;
  ~trs_cpr() {
    if (ev_fork) cudaEventDestroy(ev_fork);
    if (ev_join) cudaEventDestroy(ev_join);
    if (side) cudaStreamDestroy(side);
  }
};
