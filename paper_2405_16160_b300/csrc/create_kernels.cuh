// Create-time device kernels of the B300 restarted-PDHCG solver: the
// explicit transpose A' (built once per qp_create) and the Section 4
// diagonal scaling of K = [[Q, A'], [A, 0]].  None of them runs inside a
// solve.
#pragma once

#include "kernels.cuh"

namespace pdhcg {

// ------------------------------------------------------ row tables
// Row census of a CSR matrix for the row kernels' tables: out[0] = the rows
// of at most kRuleRowMax entries, out[1] = their entries (the inputs of the
// lanes-per-row rule), out[2] = the rows of more than kCandidateMin entries
// (every medium or long row at any lanes per row is among them).  Integer
// atomics, one per warp: the totals do not depend on the order.
constexpr int kRuleRowMax = 64;
constexpr int kCandidateMin = 16;

__global__ void __launch_bounds__(kBlock) k_row_census(const int32_t* __restrict__ rowptr,
                                                       int rows, unsigned long long* out) {
  unsigned long long r = 0, z = 0, c = 0;
  for (long long i = grid_tid(); i < rows; i += grid_threads()) {
    const int len = __ldg(rowptr + i + 1) - __ldg(rowptr + i);
    if (len <= kRuleRowMax) {
      ++r;
      z += (unsigned long long)len;
    }
    c += len > kCandidateMin;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    r += __shfl_xor_sync(0xffffffffu, r, o);
    z += __shfl_xor_sync(0xffffffffu, z, o);
    c += __shfl_xor_sync(0xffffffffu, c, o);
  }
  if ((threadIdx.x & 31) == 0 && (r | z | c) != 0) {
    atomicAdd(out, r);
    atomicAdd(out + 1, z);
    atomicAdd(out + 2, c);
  }
}

// The rows of more than min_len entries (a stream-compaction predicate
// over row indices).
struct RowLongerThan {
  const int32_t* rowptr;
  int32_t min_len;
  __host__ __device__ __forceinline__ bool operator()(const int32_t& i) const {
    return rowptr[i + 1] - rowptr[i] > min_len;
  }
};

// The first and one-past-last entry of each listed row.
__global__ void k_row_bounds(const int32_t* __restrict__ rowptr, const int32_t* __restrict__ list,
                             int count, int32_t* b, int32_t* e) {
  for (long long k = grid_tid(); k < count; k += grid_threads()) {
    const int32_t i = list[k];
    b[k] = rowptr[i];
    e[k] = rowptr[i + 1];
  }
}

// The transpose kernels take one warp per row, so a row of any length is
// read with coalesced loads.

// row_of[k] = i for every entry k of row i.
__global__ void __launch_bounds__(kBlock) k_row_of_entry(const int32_t* __restrict__ rowptr,
                                                         int rows, int32_t* row_of) {
  const int lane = threadIdx.x & 31;
  for (long long i = grid_tid() >> 5; i < rows; i += grid_threads() >> 5)
    for (int k = __ldg(rowptr + i) + lane; k < __ldg(rowptr + i + 1); k += 32) row_of[k] = int(i);
}

__global__ void k_iota(int32_t* v, long long n) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) v[i] = int32_t(i);
}

// Entries per column (integer atomics: the totals do not depend on order).
__global__ void k_count_columns(const int32_t* __restrict__ col, long long nnz, int32_t* count) {
  for (long long k = grid_tid(); k < nnz; k += grid_threads()) atomicAdd(count + col[k], 1);
}

// A' entries from the entries of A sorted stably by column: entry k of A'
// is entry perm[k] of A (so each row of A' lists increasing rows of A).
__global__ void k_gather_transpose(const int32_t* __restrict__ perm,
                                   const int32_t* __restrict__ row_of,
                                   const double* __restrict__ val, long long nnz, int32_t* t_col,
                                   double* t_val) {
  for (long long k = grid_tid(); k < nnz; k += grid_threads()) {
    const int32_t e = perm[k];
    t_col[k] = row_of[e];
    t_val[k] = val[e];
  }
}

__device__ __forceinline__ double warp_max_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, shfl_xor(v, o));
  return v;
}

// Rows of the scaling kernels go to warps eight at a time: row base + lane/4
// to a group of four lanes when it has at most kShortRow entries, and every
// longer row of the eight to the whole warp afterwards, in row order.  Short
// rows (the common case) keep all lanes busy; a row of any length is still
// read with coalesced loads.  A group's four partial values are combined
// with xor shuffles, so a row's norm does not depend on the launch.
constexpr int kScaleGroup = 4;
constexpr int kScaleRowsPerWarp = 32 / kScaleGroup;
constexpr int kShortRow = 64;

// Row-norm accumulators of the scaling.  The inf-norm keeps the bit pattern
// of its largest term: non-negative doubles order as their bit patterns, so
// the maximum is an integer one and stays off the FP64 pipe (a small fraction
// of the FP32 rate on this GPU); the 1-norm is a plain FP64 sum of fused
// products.  Either way a stored entry costs one FP64 instruction.
template <bool kInf>
struct NormAcc;

template <>
struct NormAcc<true> {
  long long v = 0;  // +0.0
  __device__ __forceinline__ void add_prod(double a, double b) {
    v = max(v, __double_as_longlong(a * b));
  }
  __device__ __forceinline__ void add(double t) { v = max(v, __double_as_longlong(t)); }
  __device__ __forceinline__ void merge_shfl(int o) {
    v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  }
  __device__ __forceinline__ void merge(const NormAcc& o) { v = max(v, o.v); }
  __device__ __forceinline__ double value() const { return __longlong_as_double(v); }
};

template <>
struct NormAcc<false> {
  double v = 0.0;
  __device__ __forceinline__ void add_prod(double a, double b) { v = fma(a, b, v); }
  __device__ __forceinline__ void add(double t) { v += t; }
  __device__ __forceinline__ void merge_shfl(int o) {
    v += __shfl_xor_sync(0xffffffffu, v, o);
  }
  __device__ __forceinline__ void merge(const NormAcc& o) { v += o.v; }
  __device__ __forceinline__ double value() const { return v; }
};

// A lane's share of a short row's norm of |M_ik| d_k (the row's own factor is
// applied once to the row's total): entries b + sub, b + sub + G, ... of the
// row, four per trip (the column and value loads issued first, then the four
// gathers of the scaling factor, then the four terms in entry order).
template <bool kInf>
__device__ __forceinline__ NormAcc<kInf> scale_row_part(const CsrT<double>& M, const double* d,
                                                        int b, int e, int sub) {
  NormAcc<kInf> r;
  for (int k = b + sub; k < e; k += 4 * kScaleGroup) {
    int c[4];
    double a[4], dc[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int kk = k + u * kScaleGroup;
      c[u] = kk < e ? __ldg(M.col + kk) : -1;
      a[u] = kk < e ? __ldg(M.val + kk) : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u) dc[u] = c[u] >= 0 ? d[c[u]] : 0.0;
#pragma unroll
    for (int u = 0; u < 4; ++u)
      if (c[u] >= 0) r.add_prod(fabs(a[u]), dc[u]);
  }
  return r;
}

template <bool kInf>
__device__ __forceinline__ NormAcc<kInf> group_combine(NormAcc<kInf> v) {
#pragma unroll
  for (int o = kScaleGroup / 2; o > 0; o >>= 1) v.merge_shfl(o);
  return v;
}

template <bool kInf>
__device__ __forceinline__ NormAcc<kInf> warp_combine(NormAcc<kInf> v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v.merge_shfl(o);
  return v;
}

// A row of more than kShortRow entries by a whole warp: the norm of
// |M_ik| d_k over the row (from the segment pre-pass for rows longer than
// kLongRow), on every lane.
template <bool kInf>
__device__ __forceinline__ NormAcc<kInf> scale_warp_row(const CsrT<double>& M, const double* d,
                                                        int row, int lane) {
  const int b = __ldg(M.rowptr + row), e = __ldg(M.rowptr + row + 1);
  NormAcc<kInf> s;
  if (e - b > kLongRow) {  // from the segment pre-pass (k_scale_long_parts)
    if (lane == 0) s.add(M.long_val[long_slot(M, row)]);
  } else {
    for (int k = b + lane; k < e; k += 32) s.add_prod(fabs(M.val[k]), d[M.col[k]]);
  }
  return warp_combine(s);
}

// Section 4 scaling of K = [[Q, A'], [A, 0]] under the current D = diag(D2,
// D1): the norm of each row of D K D, the inf-norm for a Ruiz step (kInf) or
// the 1-norm for the Pock-Chambolle step.  Variable rows j read row j of Q
// and row j of A'; constraint rows i read row i of A.  Row j's norm is
// D2_j times the norm of |K_jk| D_k (the row factor is common to its terms).
template <bool kInf>
__global__ void __launch_bounds__(kBlock) k_scale_norms_n(CsrT<double> Q, CsrT<double> At,
                                                          const double* __restrict__ d1,
                                                          const double* __restrict__ d2,
                                                          double* rn) {
  const int lane = threadIdx.x & 31, sub = lane & (kScaleGroup - 1);
  const long long nw = grid_threads() >> 5;
  for (long long base = (grid_tid() >> 5) * kScaleRowsPerWarp; base < Q.rows;
       base += nw * kScaleRowsPerWarp) {
    const int j = int(base) + lane / kScaleGroup;
    bool long_row = false;
    NormAcc<kInf> r, ra;
    if (j < Q.rows) {
      const int qb = __ldg(Q.rowptr + j), qe = __ldg(Q.rowptr + j + 1);
      const int ab = __ldg(At.rowptr + j), ae = __ldg(At.rowptr + j + 1);
      long_row = (qe - qb) + (ae - ab) > kShortRow;
      if (!long_row) {
        r = scale_row_part<kInf>(Q, d2, qb, qe, sub);
        ra = scale_row_part<kInf>(At, d1, ab, ae, sub);
      }
    }
    r = group_combine(r);
    ra = group_combine(ra);
    if (j < Q.rows && !long_row && sub == 0) {
      r.merge(ra);
      rn[j] = d2[j] * r.value();
    }
    unsigned lm = __ballot_sync(0xffffffffu, long_row && sub == 0);
    while (lm) {
      const int jj = int(base) + (__ffs(lm) - 1) / kScaleGroup;
      lm &= lm - 1;
      NormAcc<kInf> s = scale_warp_row<kInf>(Q, d2, jj, lane);
      s.merge(scale_warp_row<kInf>(At, d1, jj, lane));
      if (lane == 0) rn[jj] = d2[jj] * s.value();
    }
  }
}

template <bool kInf>
__global__ void __launch_bounds__(kBlock) k_scale_norms_m(CsrT<double> A,
                                                          const double* __restrict__ d1,
                                                          const double* __restrict__ d2,
                                                          double* rm) {
  const int lane = threadIdx.x & 31, sub = lane & (kScaleGroup - 1);
  const long long nw = grid_threads() >> 5;
  for (long long base = (grid_tid() >> 5) * kScaleRowsPerWarp; base < A.rows;
       base += nw * kScaleRowsPerWarp) {
    const int i = int(base) + lane / kScaleGroup;
    bool long_row = false;
    NormAcc<kInf> r;
    if (i < A.rows) {
      const int b = __ldg(A.rowptr + i), e = __ldg(A.rowptr + i + 1);
      long_row = e - b > kShortRow;
      if (!long_row) r = scale_row_part<kInf>(A, d2, b, e, sub);
    }
    r = group_combine(r);
    if (i < A.rows && !long_row && sub == 0) rm[i] = d1[i] * r.value();
    unsigned lm = __ballot_sync(0xffffffffu, long_row && sub == 0);
    while (lm) {
      const int ii = int(base) + (__ffs(lm) - 1) / kScaleGroup;
      lm &= lm - 1;
      const NormAcc<kInf> s = scale_warp_row<kInf>(A, d2, ii, lane);
      if (lane == 0) rm[ii] = d1[ii] * s.value();
    }
  }
}

// D <- D / sqrt(row norm), as D times the reciprocal square root (one
// library call instead of a square root and a division, both long FP64
// sequences on this GPU); an all-zero row keeps its scale.
__global__ void k_scale_apply(double* d2, const double* __restrict__ rn, int n, double* d1,
                              const double* __restrict__ rm, int m) {
  for (long long j = grid_tid(); j < n; j += grid_threads())
    d2[j] *= rsqrt(rn[j] > 0.0 ? rn[j] : 1.0);
  for (long long i = grid_tid(); i < m; i += grid_threads())
    d1[i] *= rsqrt(rm[i] > 0.0 ? rm[i] : 1.0);
}

// M_ik <- (dr_i M_ik) dc_k in place (rows split as in the norm kernels).
__global__ void __launch_bounds__(kBlock) k_scale_matrix(CsrT<double> M,
                                                         const double* __restrict__ dr,
                                                         const double* __restrict__ dc,
                                                         double* val) {
  const int lane = threadIdx.x & 31, sub = lane & (kScaleGroup - 1);
  const long long nw = grid_threads() >> 5;
  for (long long base = (grid_tid() >> 5) * kScaleRowsPerWarp; base < M.rows;
       base += nw * kScaleRowsPerWarp) {
    const int i = int(base) + lane / kScaleGroup;
    bool long_row = false;
    if (i < M.rows) {
      const int b = __ldg(M.rowptr + i), e = __ldg(M.rowptr + i + 1);
      long_row = e - b > kShortRow;
      if (!long_row) {
        const double di = dr[i];
        for (int k = b + sub; k < e; k += kScaleGroup) val[k] = (di * val[k]) * dc[M.col[k]];
      }
    }
    unsigned lm = __ballot_sync(0xffffffffu, long_row && sub == 0);
    while (lm) {
      const int ii = int(base) + (__ffs(lm) - 1) / kScaleGroup;
      lm &= lm - 1;
      const int b = __ldg(M.rowptr + ii), e = __ldg(M.rowptr + ii + 1);
      if (e - b > kLongRow) continue;  // k_scale_long_matrix
      const double di = dr[ii];
      for (int k = b + lane; k < e; k += 32) val[k] = (di * val[k]) * dc[M.col[k]];
    }
  }
}

// Rows longer than kLongRow in the scaling: one warp per kSegLen-entry segment
// (the long-row table of the products), so that a row of millions of entries
// spreads over the whole GPU instead of one warp.
//
// Norm pass, phase 1: seg[s] = the segment's inf- or 1-norm of |M_ik| dc_k
// (the row's own factor is applied by the row kernels).
template <bool kInf>
__global__ void __launch_bounds__(kBlock) k_scale_long_parts(CsrT<double> M, LongRows L,
                                                             const double* __restrict__ dc,
                                                             double* seg) {
  const int lane = threadIdx.x & 31;
  for (long long sg = grid_tid() >> 5; sg < L.nseg; sg += grid_threads() >> 5) {
    NormAcc<kInf> v;
    for (int k = __ldg(L.seg_begin + sg) + lane; k < __ldg(L.seg_end + sg); k += 32)
      v.add_prod(fabs(M.val[k]), dc[M.col[k]]);
    v = warp_combine(v);
    if (lane == 0) seg[sg] = v.value();
  }
}

// Phase 2: each long row's segments in order.
template <bool kInf>
__global__ void k_scale_long_totals(LongRows L, const double* __restrict__ seg, double* total) {
  for (long long r = grid_tid(); r < L.nlong; r += grid_threads()) {
    NormAcc<kInf> v;
    for (int s = __ldg(L.seg_ptr + r); s < __ldg(L.seg_ptr + r + 1); ++s) v.add(seg[s]);
    total[r] = v.value();
  }
}

// The scaled values of the long rows: one warp per segment; a segment's row
// is found in the row table by binary search.
__global__ void __launch_bounds__(kBlock) k_scale_long_matrix(CsrT<double> M, LongRows L,
                                                              const double* __restrict__ dr,
                                                              const double* __restrict__ dc,
                                                              double* val) {
  const int lane = threadIdx.x & 31;
  for (long long sg = grid_tid() >> 5; sg < L.nseg; sg += grid_threads() >> 5) {
    int lo = 0, hi = L.nlong - 1;  // the last row r with seg_ptr[r] <= sg
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(L.seg_ptr + mid) <= sg)
        lo = mid;
      else
        hi = mid - 1;
    }
    const double di = dr[__ldg(M.long_rows + lo)];
    for (int k = __ldg(L.seg_begin + sg) + lane; k < __ldg(L.seg_end + sg); k += 32)
      val[k] = (di * val[k]) * dc[M.col[k]];
  }
}

// v <- d v and inv = 1/d.
// ---- qp_create's checks of the problem as given, on the device copies.
// Row pointers: the lowest row whose pointer decreases to *bad_row, and a
// mark at the first entry of every non-empty row (marks only at offsets in
// [0, nnz), so the entry pass stays in bounds whatever the pointers hold).
__global__ void k_check_rows(const int32_t* __restrict__ rowptr, int rows, long long nnz,
                             uint8_t* first, unsigned long long* bad_row) {
  for (long long i = grid_tid(); i < rows; i += grid_threads()) {
    const int32_t a = rowptr[i], e = rowptr[i + 1];
    if (e < a) atomicMin(bad_row, (unsigned long long)i);
    if (a < e && a >= 0 && a < nnz) first[a] = 1;
  }
}

// Entries: the lowest one with a column outside [0, cols) or a non-finite
// value to *bad_entry; *unsorted = 1 if a column does not exceed its
// predecessor within a row.
__global__ void k_check_entries(const int32_t* __restrict__ col, const double* __restrict__ val,
                                long long nnz, int cols, const uint8_t* __restrict__ first,
                                unsigned long long* bad_entry, int* unsorted) {
  bool uns = false;
  for (long long k = grid_tid(); k < nnz; k += grid_threads()) {
    const int32_t j = col[k];
    if (uint32_t(j) >= uint32_t(cols) || !isfinite(val[k]))
      atomicMin(bad_entry, (unsigned long long)k);
    uns |= k > 0 && !first[k] && j <= col[k - 1];
  }
  if (uns) *unsorted = 1;
}

// The lowest index of a non-finite value to *bad.
__global__ void k_check_finite(const double* __restrict__ v, long long n,
                               unsigned long long* bad) {
  for (long long i = grid_tid(); i < n; i += grid_threads())
    if (!isfinite(v[i])) atomicMin(bad, (unsigned long long)i);
}

__global__ void k_fill(double* v, double a, int n) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) v[i] = a;
}

// out = v * d elementwise: a solution back in the caller's variables.
__global__ void k_unscale(double* out, const double* __restrict__ v, const double* __restrict__ d,
                          int n) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) out[i] = v[i] * d[i];
}

__global__ void k_scale_vector(double* v, const double* __restrict__ d, double* inv, int n) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    v[i] *= d[i];
    inv[i] = 1.0 / d[i];
  }
}

}  // namespace pdhcg
