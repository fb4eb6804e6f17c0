// Host-side CSR utilities of the C ABI: validation, canonicalisation (sorted
// rows, duplicates summed), a stable transpose (qp_csr_transpose and the
// symmetry check of Q; qp_create builds A' on the device) and the symmetry
// check itself.  Plain C++, no CUDA.
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

// True when the canonical square matrix M satisfies |M_ij - M_ji| <= rtol * max|M|.
bool csr_is_symmetric(const HostCsr& M, double rtol);

}  // namespace pdhcg
