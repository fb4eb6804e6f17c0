#include "host_csr.h"

#include <algorithm>
#include <cmath>
#include <numeric>

namespace pdhcg {

bool csr_validate(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
                  const double* val, std::string* why) {
  auto fail = [&](const std::string& s) {
    if (why) *why = s;
    return false;
  };
  if (rows < 0 || cols < 0) return fail("negative dimension");
  if (!rowptr) return fail("rowptr is NULL");
  if (rowptr[0] != 0) return fail("rowptr[0] != 0");
  for (int32_t i = 0; i < rows; ++i)
    if (rowptr[i + 1] < rowptr[i]) return fail("rowptr is not monotone at row " + std::to_string(i));
  const int64_t nnz = rowptr[rows];
  if (nnz < 0 || nnz >= (int64_t(1) << 31)) return fail("nnz out of int32 range");
  if (nnz > 0 && (!col || !val)) return fail("col or val is NULL");
  for (int64_t k = 0; k < nnz; ++k) {
    if (col[k] < 0 || col[k] >= cols)
      return fail("column index out of range at entry " + std::to_string(k));
    if (!std::isfinite(val[k])) return fail("non-finite value at entry " + std::to_string(k));
  }
  return true;
}

HostCsr csr_canonical(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
                      const double* val) {
  HostCsr out;
  out.rows = rows;
  out.cols = cols;
  out.rowptr.assign(size_t(rows) + 1, 0);
  const int64_t nnz = rowptr[rows];
  out.col.reserve(size_t(nnz));
  out.val.reserve(size_t(nnz));
  std::vector<int64_t> idx;
  for (int32_t i = 0; i < rows; ++i) {
    const int64_t s = rowptr[i], e = rowptr[i + 1];
    bool sorted = true;
    for (int64_t k = s + 1; k < e; ++k)
      if (col[k] <= col[k - 1]) { sorted = false; break; }
    if (sorted) {
      out.col.insert(out.col.end(), col + s, col + e);
      out.val.insert(out.val.end(), val + s, val + e);
    } else {
      idx.resize(size_t(e - s));
      std::iota(idx.begin(), idx.end(), s);
      std::stable_sort(idx.begin(), idx.end(), [&](int64_t a, int64_t b) { return col[a] < col[b]; });
      for (size_t t = 0; t < idx.size(); ++t) {
        const int32_t cj = col[idx[t]];
        if (!out.col.empty() && int64_t(out.col.size()) > out.rowptr[i] && out.col.back() == cj)
          out.val.back() += val[idx[t]];
        else {
          out.col.push_back(cj);
          out.val.push_back(val[idx[t]]);
        }
      }
    }
    out.rowptr[size_t(i) + 1] = int32_t(out.col.size());
  }
  return out;
}

void csr_transpose(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
                   const double* val, int32_t* t_rowptr, int32_t* t_col, double* t_val) {
  const int64_t nnz = rowptr[rows];
  std::fill(t_rowptr, t_rowptr + cols + 1, 0);
  for (int64_t k = 0; k < nnz; ++k) t_rowptr[col[k] + 1]++;
  for (int32_t j = 0; j < cols; ++j) t_rowptr[j + 1] += t_rowptr[j];
  std::vector<int32_t> next(t_rowptr, t_rowptr + cols);
  for (int32_t i = 0; i < rows; ++i)
    for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
      const int32_t dst = next[col[k]]++;
      t_col[dst] = i;
      t_val[dst] = val[k];
    }
}

bool csr_is_symmetric(const HostCsr& M, double rtol) {
  if (M.rows != M.cols) return false;
  const int64_t nnz = M.nnz();
  std::vector<int32_t> tr(static_cast<size_t>(M.cols) + 1);
  std::vector<int32_t> tc(static_cast<size_t>(nnz));
  std::vector<double> tv(static_cast<size_t>(nnz));
  csr_transpose(M.rows, M.cols, M.rowptr.data(), M.col.data(), M.val.data(), tr.data(), tc.data(),
                tv.data());
  double amax = 0.0;
  for (double v : M.val) amax = std::max(amax, std::fabs(v));
  const double tol = rtol * amax;
  // Both are canonical (sorted, no duplicates): merge row by row.
  for (int32_t i = 0; i < M.rows; ++i) {
    int64_t a = M.rowptr[i], ae = M.rowptr[i + 1], b = tr[i], be = tr[i + 1];
    while (a < ae || b < be) {
      if (b >= be || (a < ae && M.col[a] < tc[b])) {
        if (std::fabs(M.val[a]) > tol) return false;
        ++a;
      } else if (a >= ae || tc[b] < M.col[a]) {
        if (std::fabs(tv[b]) > tol) return false;
        ++b;
      } else {
        if (std::fabs(M.val[a] - tv[b]) > tol) return false;
        ++a;
        ++b;
      }
    }
  }
  return true;
}

}  // namespace pdhcg
