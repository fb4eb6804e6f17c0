// Host-side CSR utilities of the C ABI: validation, canonicalisation (sorted
// rows, duplicates summed), the stable transpose that builds A' once at
// create time, and the symmetry check of Q.  Plain C++, no CUDA.
#pragma once

#include <cstdint>
#include <string>
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

// Diagonal preconditioning of K = [[Q, A'], [A, 0]]: `ruiz_iters` Ruiz steps
// (each row of the current D K D divided on both sides by the square root of
// its infinity norm), then one Pock-Chambolle step (the same with the 1-norm).
// At is A' (rows = columns of A).  Rows that are entirely zero keep scale 1.
void diagonal_scaling(const CsrView& Q, const CsrView& A, const CsrView& At, int ruiz_iters,
                      std::vector<double>* d1, std::vector<double>* d2);

// Copy of M with entry (i, j) multiplied by (dr[i] * M_ij) * dc[j].
HostCsr scaled_copy(const CsrView& M, const double* dr, const double* dc);

// True when the canonical square matrix M satisfies |M_ij - M_ji| <= rtol * max|M|.
bool csr_is_symmetric(const HostCsr& M, double rtol);

}  // namespace pdhcg
