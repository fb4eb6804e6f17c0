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

// Checks rowptr[0] = 0, monotone rowptr, nnz < 2^31, columns in range and
// finite values.  On failure returns false and fills *why.
bool csr_validate(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
                  const double* val, std::string* why);

// Copy of a valid CSR with every row sorted by column and duplicate entries
// summed (the order of summation is the input order).
HostCsr csr_canonical(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
                      const double* val);

// Stable counting-sort transpose: output row j lists the entries of input
// column j in increasing input-row order.
void csr_transpose(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
                   const double* val, int32_t* t_rowptr, int32_t* t_col, double* t_val);

// True when the canonical square matrix M satisfies |M_ij - M_ji| <= rtol * max|M|.
bool csr_is_symmetric(const HostCsr& M, double rtol);

}  // namespace pdhcg
