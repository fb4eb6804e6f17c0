// Host-side CSR utilities of the C ABI: validation, canonicalisation (sorted
// rows, duplicates summed), a stable transpose (qp_csr_transpose and the
// symmetry check of Q; qp_create builds A' on the device) and the symmetry
// check itself.  Plain C++, no CUDA.
#pragma once

#include <algorithm>
#include <cstdint>
#include <string>
#include <thread>
#include <vector>

namespace pdhcg {

struct HostCsr {
  int32_t rows = 0, cols = 0;
  std::vector<int32_t> rowptr, col;
  std::vector<double> val;
  int64_t nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
};

// Non-owning view of a CSR matrix (the caller's arrays or a HostCsr).
struct CsrView {
  int32_t rows = 0, cols = 0;
  const int32_t* rowptr = nullptr;
  const int32_t* col = nullptr;
  const double* val = nullptr;
  int64_t nnz() const { return rowptr ? rowptr[rows] : 0; }
};

inline CsrView view_of(const HostCsr& H) {
  return CsrView{H.rows, H.cols, H.rowptr.data(), H.col.data(), H.val.data()};
}

// Checks rowptr[0] = 0, monotone rowptr, nnz < 2^31, columns in range and
// finite values.  On failure returns false and fills *why.
bool csr_validate(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
                  const double* val, std::string* why);

// csr_validate and, on the same multi-threaded pass over the entries,
// *canonical = every row's columns strictly increasing (when canonical is
// not NULL and the matrix is valid).
bool csr_check(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
               const double* val, std::string* why, bool* canonical);

// True when every row's columns are strictly increasing (sorted, no duplicates).
bool csr_is_canonical(int32_t rows, const int32_t* rowptr, const int32_t* col);

// Copy of a valid CSR with every row sorted by column and duplicate entries
// summed (the order of summation is the input order).
HostCsr csr_canonical(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
                      const double* val);

// Stable counting-sort transpose: output row j lists the entries of input
// column j in increasing input-row order (multi-threaded; same output for
// any thread count).
void csr_transpose(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
                   const double* val, int32_t* t_rowptr, int32_t* t_col, double* t_val);

// True when the canonical square matrix M satisfies |M_ij - M_ji| <= rtol * max|M|.
bool csr_is_symmetric(const HostCsr& M, double rtol);

// Section 4 augmented penalty on the equality rows G (the first m_eq rows of
// the canonical A): rho = 0.1 ||Q||_2 / ||G'G||_2, each norm from `iters`
// power iterations started at ones/sqrt(n) (||Q v|| for the symmetric Q,
// ||G'G v|| for G'G), and rho = 0 when ||G'G||_2 <= eps_zero.  Then
// Qp = Q + rho G'G (canonical: every entry Q_jk + rho sum_r g_rj g_rk) and
// cp = c - rho G'q with q the first m_eq entries of b.  Returns false with
// *why when G'G would take more than max_products products (sum over the
// equality rows of their length squared: a dense row makes G'G dense).
bool csr_penalize(const CsrView& Q, const CsrView& A, int32_t m_eq, const double* c,
                  const double* b, int iters, double eps_zero, int64_t max_products,
                  HostCsr* Qp, std::vector<double>* cp, double* rho, std::string* why);

// The host's hardware threads, asked once per process: the standard call
// reads the system's CPU lists on every use (tens of microseconds), which
// adds up where thousands of small instances are checked one by one.
inline int hw_threads() {
  static const int n = int(std::max(1u, std::thread::hardware_concurrency()));
  return n;
}

// f(t, lo, hi) for T contiguous ranges [lo, hi) covering [0, n), range t on
// host thread t (t = 0 on the caller's), T = min(max_threads, the hardware
// threads, n / min_per_thread), at least 1.  Returns T.
template <class F>
int parallel_ranges(int64_t n, int max_threads, int64_t min_per_thread, F&& f) {
  const int64_t hw = hw_threads();
  const int T = int(std::max<int64_t>(
      1, std::min<int64_t>({int64_t(max_threads), hw, n / std::max<int64_t>(1, min_per_thread)})));
  auto run = [&](int t) { f(t, n * t / T, n * (t + 1) / T); };
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(run, t);
  run(0);
  for (auto& x : th) x.join();
  return T;
}

}  // namespace pdhcg
