// Create-time device kernels of the B300 restarted-PDHCG solver: the
// explicit transpose A' (built once per qp_create) and the Section 4
// diagonal scaling of K = [[Q, A'], [A, 0]].  None of them runs inside a
// solve.
#pragma once

#include "kernels.cuh"

namespace pdhcg {

// One warp per row throughout, so a row of any length is read with coalesced
// loads.

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

// Section 4 scaling of K = [[Q, A'], [A, 0]] under the current D = diag(D2,
// D1): the norm of each row of D K D, the inf-norm for a Ruiz step (inf = 1)
// or the 1-norm for the Pock-Chambolle step.  Variable rows j read row j of
// Q and row j of A'; constraint rows i read row i of A.
__global__ void __launch_bounds__(kBlock) k_scale_norms_n(CsrT<double> Q, CsrT<double> At,
                                                          const double* __restrict__ d1,
                                                          const double* __restrict__ d2,
                                                          double* rn, int inf) {
  const int lane = threadIdx.x & 31;
  for (long long j = grid_tid() >> 5; j < Q.rows; j += grid_threads() >> 5) {
    const double dj = d2[j];
    double r = 0.0, ra = 0.0;
    for (int k = __ldg(Q.rowptr + j) + lane; k < __ldg(Q.rowptr + j + 1); k += 32) {
      const double v = (dj * fabs(Q.val[k])) * d2[Q.col[k]];
      r = inf ? fmax(r, v) : r + v;
    }
    for (int k = __ldg(At.rowptr + j) + lane; k < __ldg(At.rowptr + j + 1); k += 32) {
      const double v = (d1[At.col[k]] * fabs(At.val[k])) * dj;
      ra = inf ? fmax(ra, v) : ra + v;
    }
    r = inf ? warp_max_d(r) : warp_sum(r);
    ra = inf ? warp_max_d(ra) : warp_sum(ra);
    if (lane == 0) rn[j] = inf ? fmax(r, ra) : r + ra;
  }
}

__global__ void __launch_bounds__(kBlock) k_scale_norms_m(CsrT<double> A,
                                                          const double* __restrict__ d1,
                                                          const double* __restrict__ d2,
                                                          double* rm, int inf) {
  const int lane = threadIdx.x & 31;
  for (long long i = grid_tid() >> 5; i < A.rows; i += grid_threads() >> 5) {
    const double di = d1[i];
    double r = 0.0;
    for (int k = __ldg(A.rowptr + i) + lane; k < __ldg(A.rowptr + i + 1); k += 32) {
      const double v = (di * fabs(A.val[k])) * d2[A.col[k]];
      r = inf ? fmax(r, v) : r + v;
    }
    r = inf ? warp_max_d(r) : warp_sum(r);
    if (lane == 0) rm[i] = r;
  }
}

// D <- D / sqrt(row norm); an all-zero row keeps its scale.
__global__ void k_scale_apply(double* d2, const double* __restrict__ rn, int n, double* d1,
                              const double* __restrict__ rm, int m) {
  for (long long j = grid_tid(); j < n; j += grid_threads())
    d2[j] /= sqrt(rn[j] > 0.0 ? rn[j] : 1.0);
  for (long long i = grid_tid(); i < m; i += grid_threads())
    d1[i] /= sqrt(rm[i] > 0.0 ? rm[i] : 1.0);
}

// M_ik <- (dr_i M_ik) dc_k in place.
__global__ void __launch_bounds__(kBlock) k_scale_matrix(CsrT<double> M,
                                                         const double* __restrict__ dr,
                                                         const double* __restrict__ dc,
                                                         double* val) {
  const int lane = threadIdx.x & 31;
  for (long long i = grid_tid() >> 5; i < M.rows; i += grid_threads() >> 5) {
    const double di = dr[i];
    for (int k = __ldg(M.rowptr + i) + lane; k < __ldg(M.rowptr + i + 1); k += 32)
      val[k] = (di * val[k]) * dc[M.col[k]];
  }
}

// v <- d v and inv = 1/d.
__global__ void k_scale_vector(double* v, const double* __restrict__ d, double* inv, int n) {
  for (long long i = grid_tid(); i < n; i += grid_threads()) {
    v[i] *= d[i];
    inv[i] = 1.0 / d[i];
  }
}

}  // namespace pdhcg
