#include "host_csr.h"

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstring>
#include <numeric>
#include <thread>

namespace pdhcg {

namespace {

// Worker threads for `work` items: at most the hardware threads (<= 32) and
// at least ~256K items each.
int worker_count(int64_t work) {
  const unsigned hc = unsigned(std::min(hw_threads(), 32));
  return int(std::max<int64_t>(1, std::min<int64_t>(hc, work / (int64_t(1) << 18))));
}

template <class F>
void parallel_for(int T, F&& f) {
  std::vector<std::thread> th;
  for (int t = 1; t < T; ++t) th.emplace_back(f, t);
  f(0);
  for (auto& x : th) x.join();
}

// Row ranges [b[t], b[t+1]) holding about nnz/T entries each.
std::vector<int32_t> split_rows(const int32_t* rowptr, int32_t rows, int T) {
  std::vector<int32_t> b(size_t(T) + 1, rows);
  b[0] = 0;
  const int64_t nnz = rowptr[rows];
  for (int t = 1; t < T; ++t) {
    const int64_t target = nnz * t / T;
    b[size_t(t)] = int32_t(std::lower_bound(rowptr, rowptr + rows + 1, target) - rowptr);
    b[size_t(t)] = std::min(std::max(b[size_t(t)], b[size_t(t) - 1]), rows);
  }
  return b;
}

}  // namespace

bool csr_check(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
               const double* val, std::string* why, bool* canonical) {
  auto fail = [&](const std::string& s) {
    if (why) *why = s;
    return false;
  };
  if (rows < 0 || cols < 0) return fail("negative dimension");
  if (!rowptr) return fail("rowptr is NULL");
  if (rowptr[0] != 0) return fail("rowptr[0] != 0");
  // rowptr monotone, in parallel chunks of rows; the first bad row is reported
  const int Tr = worker_count(rows);
  std::atomic<int64_t> bad_row(rows);
  parallel_for(Tr, [&](int t) {
    const int64_t lo = int64_t(rows) * t / Tr, hi = int64_t(rows) * (t + 1) / Tr;
    for (int64_t i = lo; i < hi; ++i)
      if (rowptr[i + 1] < rowptr[i]) {
        int64_t cur = bad_row.load();
        while (i < cur && !bad_row.compare_exchange_weak(cur, i)) {
        }
        break;
      }
  });
  if (bad_row.load() < rows)
    return fail("rowptr is not monotone at row " + std::to_string(bad_row.load()));
  const int64_t nnz = rowptr[rows];
  if (nnz < 0 || nnz >= (int64_t(1) << 31)) return fail("nnz out of int32 range");
  if (nnz > 0 && (!col || !val)) return fail("col or val is NULL");
  // Entries, in parallel row ranges of about equal entry counts, in one
  // branch-free pass: columns in range and finite values (on a failure the
  // range is scanned again for its first bad entry, and the lowest over the
  // ranges is reported) and strictly increasing columns in every row.
  const int T = worker_count(nnz);
  const std::vector<int32_t> b = split_rows(rowptr, rows, T);
  std::atomic<int64_t> first_bad(nnz);
  std::atomic<bool> sorted(true);
  const uint64_t exp_mask = 0x7ff0000000000000ull;
  parallel_for(T, [&](int t) {
    bool bad = false, unsorted = false;
    for (int32_t i = b[size_t(t)]; i < b[size_t(t) + 1]; ++i) {
      int32_t prev = -1;
      for (int64_t k = rowptr[i], e = rowptr[i + 1]; k < e; ++k) {
        const int32_t j = col[k];
        uint64_t bits;
        std::memcpy(&bits, val + k, sizeof bits);
        bad |= (uint32_t(j) >= uint32_t(cols)) | ((bits & exp_mask) == exp_mask);
        unsorted |= j <= prev;
        prev = j;
      }
    }
    if (bad) {
      for (int64_t k = rowptr[b[size_t(t)]]; k < rowptr[b[size_t(t) + 1]]; ++k)
        if (col[k] < 0 || col[k] >= cols || !std::isfinite(val[k])) {
          int64_t cur = first_bad.load();
          while (k < cur && !first_bad.compare_exchange_weak(cur, k)) {
          }
          break;
        }
    }
    if (unsorted) sorted = false;
  });
  const int64_t k = first_bad.load();
  if (k < nnz) {
    if (col[k] < 0 || col[k] >= cols)
      return fail("column index out of range at entry " + std::to_string(k));
    return fail("non-finite value at entry " + std::to_string(k));
  }
  if (canonical) *canonical = sorted.load();
  return true;
}

bool csr_validate(int32_t rows, int32_t cols, const int32_t* rowptr, const int32_t* col,
                  const double* val, std::string* why) {
  return csr_check(rows, cols, rowptr, col, val, why, nullptr);
}

bool csr_is_canonical(int32_t rows, const int32_t* rowptr, const int32_t* col) {
  const int T = worker_count(rowptr[rows]);
  const std::vector<int32_t> b = split_rows(rowptr, rows, T);
  std::atomic<bool> ok(true);
  parallel_for(T, [&](int t) {
    for (int32_t i = b[size_t(t)]; i < b[size_t(t) + 1] && ok.load(std::memory_order_relaxed); ++i)
      for (int64_t k = int64_t(rowptr[i]) + 1; k < rowptr[i + 1]; ++k)
        if (col[k] <= col[k - 1]) {
          ok = false;
          break;
        }
  });
  return ok.load();
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
  // Threads own row ranges; each keeps a column histogram of its range, so
  // its entries land after those of every earlier range: the output is the
  // stable (row-ordered) transpose for any thread count.
  int T = worker_count(nnz);
  T = int(std::max<int64_t>(1, std::min<int64_t>(T, (int64_t(1) << 26) / std::max(cols, 1))));
  const std::vector<int32_t> b = split_rows(rowptr, rows, T);
  std::vector<int32_t> cnt(size_t(T) * size_t(cols));
  parallel_for(T, [&](int t) {
    int32_t* c = cnt.data() + size_t(t) * cols;
    std::fill(c, c + cols, 0);
    for (int64_t k = rowptr[b[size_t(t)]]; k < rowptr[b[size_t(t) + 1]]; ++k) c[col[k]]++;
  });
  // Column totals and their exclusive scan, then per-thread start offsets.
  t_rowptr[0] = 0;
  {
    const int TC = worker_count(int64_t(cols) * T);
    std::vector<int64_t> block_sum(size_t(TC) + 1, 0);
    parallel_for(TC, [&](int u) {
      const int64_t lo = int64_t(cols) * u / TC, hi = int64_t(cols) * (u + 1) / TC;
      int64_t s = 0;
      for (int64_t j = lo; j < hi; ++j) {
        int32_t tot = 0;
        for (int t = 0; t < T; ++t) tot += cnt[size_t(t) * cols + j];
        t_rowptr[j + 1] = tot;
        s += tot;
      }
      block_sum[size_t(u) + 1] = s;
    });
    for (int u = 0; u < TC; ++u) block_sum[size_t(u) + 1] += block_sum[size_t(u)];
    parallel_for(TC, [&](int u) {
      const int64_t lo = int64_t(cols) * u / TC, hi = int64_t(cols) * (u + 1) / TC;
      int64_t s = block_sum[size_t(u)];
      for (int64_t j = lo; j < hi; ++j) {
        int64_t start = s;
        s += t_rowptr[j + 1];
        t_rowptr[j + 1] = int32_t(s);
        for (int t = 0; t < T; ++t) {
          int32_t& c = cnt[size_t(t) * cols + j];
          const int32_t here = c;
          c = int32_t(start);
          start += here;
        }
      }
    });
  }
  parallel_for(T, [&](int t) {
    int32_t* next = cnt.data() + size_t(t) * cols;
    for (int32_t i = b[size_t(t)]; i < b[size_t(t) + 1]; ++i)
      for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
        const int32_t dst = next[col[k]]++;
        t_col[dst] = i;
        t_val[dst] = val[k];
      }
  });
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

namespace {

double norm2(const std::vector<double>& v) {
  double s = 0.0;
  for (double x : v) s += x * x;
  return std::sqrt(s);
}

// y = M v over rows [0, rows) of a canonical CSR view.
void spmv(const CsrView& M, int32_t rows, const std::vector<double>& v, std::vector<double>* y) {
  for (int32_t i = 0; i < rows; ++i) {
    double s = 0.0;
    for (int32_t k = M.rowptr[i]; k < M.rowptr[i + 1]; ++k) s += M.val[k] * v[size_t(M.col[k])];
    (*y)[size_t(i)] = s;
  }
}

}  // namespace

bool csr_penalize(const CsrView& Q, const CsrView& A, int32_t m_eq, const double* c,
                  const double* b, int iters, double eps_zero, int64_t max_products,
                  HostCsr* Qp, std::vector<double>* cp, double* rho, std::string* why) {
  const int32_t n = Q.rows;
  *rho = 0.0;
  cp->assign(c, c + n);
  if (m_eq <= 0 || n == 0) return true;
  int64_t products = 0;
  for (int32_t r = 0; r < m_eq; ++r) {
    const int64_t len = A.rowptr[r + 1] - A.rowptr[r];
    products += len * len;
  }
  if (products > max_products) {
    *why = "the augmented penalty would make Q dense: G'G needs " + std::to_string(products) +
           " products (limit " + std::to_string(max_products) + ")";
    return false;
  }
  // ||Q||_2 and ||G'G||_2 by power iteration from ones/sqrt(n)
  const double v0 = 1.0 / std::sqrt(double(n));
  std::vector<double> v(static_cast<size_t>(n), v0);
  std::vector<double> w(static_cast<size_t>(n), 0.0);
  std::vector<double> u(static_cast<size_t>(m_eq), 0.0);
  double lam_q = 0.0;
  for (int t = 0; t < iters; ++t) {
    spmv(Q, n, v, &w);
    lam_q = norm2(w);
    if (lam_q == 0.0) break;
    for (int32_t j = 0; j < n; ++j) v[size_t(j)] = w[size_t(j)] / lam_q;
  }
  std::fill(v.begin(), v.end(), v0);
  double lam_g = 0.0;
  for (int t = 0; t < iters; ++t) {
    spmv(A, m_eq, v, &u);  // u = G v
    std::fill(w.begin(), w.end(), 0.0);
    for (int32_t r = 0; r < m_eq; ++r)  // w = G'u
      for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k)
        w[size_t(A.col[k])] += A.val[k] * u[size_t(r)];
    lam_g = norm2(w);
    if (lam_g == 0.0) break;
    for (int32_t j = 0; j < n; ++j) v[size_t(j)] = w[size_t(j)] / lam_g;
  }
  if (!(lam_g > eps_zero)) return true;
  *rho = 0.1 * lam_q / lam_g;
  // G' (rows of G by column), then Qp row j = Q row j + rho sum_r g_rj G_r
  std::vector<int32_t> tp(size_t(n) + 1, 0);
  for (int32_t k = 0; k < A.rowptr[m_eq]; ++k) ++tp[size_t(A.col[k]) + 1];
  for (int32_t j = 0; j < n; ++j) tp[size_t(j) + 1] += tp[size_t(j)];
  std::vector<int32_t> trow(size_t(A.rowptr[m_eq])), fill(tp.begin(), tp.end() - 1);
  std::vector<double> tval(trow.size());
  for (int32_t r = 0; r < m_eq; ++r)
    for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
      const int32_t e = fill[size_t(A.col[k])]++;
      trow[size_t(e)] = r;
      tval[size_t(e)] = A.val[k];
    }
  for (int32_t j = 0; j < n; ++j) {  // c - rho G'q
    double s = 0.0;
    for (int32_t e = tp[size_t(j)]; e < tp[size_t(j) + 1]; ++e)
      s += tval[size_t(e)] * b[size_t(trow[size_t(e)])];
    (*cp)[size_t(j)] = c[j] - *rho * s;
  }
  Qp->rows = Qp->cols = n;
  Qp->rowptr.assign(size_t(n) + 1, 0);
  Qp->col.clear();
  Qp->val.clear();
  std::vector<double> gg(size_t(n), 0.0), qv(size_t(n), 0.0);
  std::vector<int32_t> mark(size_t(n), -1), touched;
  for (int32_t j = 0; j < n; ++j) {
    touched.clear();
    for (int32_t k = Q.rowptr[j]; k < Q.rowptr[j + 1]; ++k) {
      const int32_t col = Q.col[k];
      mark[size_t(col)] = j;
      touched.push_back(col);
      qv[size_t(col)] = Q.val[k];
      gg[size_t(col)] = 0.0;
    }
    for (int32_t e = tp[size_t(j)]; e < tp[size_t(j) + 1]; ++e) {
      const int32_t r = trow[size_t(e)];
      const double g = tval[size_t(e)];
      for (int32_t k = A.rowptr[r]; k < A.rowptr[r + 1]; ++k) {
        const int32_t col = A.col[k];
        if (mark[size_t(col)] != j) {
          mark[size_t(col)] = j;
          touched.push_back(col);
          qv[size_t(col)] = 0.0;
          gg[size_t(col)] = 0.0;
        }
        gg[size_t(col)] += g * A.val[k];
      }
    }
    std::sort(touched.begin(), touched.end());
    for (int32_t col : touched) {
      Qp->col.push_back(col);
      Qp->val.push_back(qv[size_t(col)] + *rho * gg[size_t(col)]);
    }
    Qp->rowptr[size_t(j) + 1] = int32_t(Qp->col.size());
  }
  return true;
}

}  // namespace pdhcg
