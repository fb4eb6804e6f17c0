// qp_gather_rate: the random-gather ceiling that bounds the solver's SpMVs
// on this GPU, measured live.
//
// Every SpMV of the method reads a vector at the column indices of a sparse
// matrix.  With uniformly random columns each 4-byte read costs its own
// 32-byte sector, and the rate at which an SM's L1TEX unit takes distinct
// sectors, not DRAM bandwidth, caps the product.  This entry point times a
// kernel that does nothing but such reads (a sum of v[idx[k]] over `count`
// pseudo-random indices into an n-float vector that stays in L2), so that a
// benchmark can report its SpMV kernels against the ceiling they actually
// face, next to their fraction of HBM bandwidth.  Not part of a solve.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdint>

#include "../../include/pdhcg.h"

void pdhcg_set_last_error(const char* msg);

namespace {

// idx[k] = a 64-bit mix of (seed, k) reduced into [0, n): uniform enough for a
// gather probe, and independent of the launch configuration.
__global__ void k_fill_indices(int32_t* idx, long long count, int32_t n, unsigned long long seed) {
  for (long long k = (long long)blockIdx.x * blockDim.x + threadIdx.x; k < count;
       k += (long long)gridDim.x * blockDim.x) {
    unsigned long long z = seed + 0x9E3779B97F4A7C15ull * (unsigned long long)(k + 1);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    z ^= z >> 31;
    idx[k] = int32_t(z % (unsigned long long)n);
  }
}

__global__ void k_fill_vector(float* v, int32_t n) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    v[i] = 1.0f + float(i & 7) * 0.125f;
}

// Four independent gathers in flight per thread, like the SpMV row loop.
__global__ void __launch_bounds__(256) k_gather(const int32_t* __restrict__ idx, long long count,
                                                const float* __restrict__ v, float* out) {
  const long long t0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long nt = (long long)gridDim.x * blockDim.x;
  float s = 0.f;
  for (long long k = t0; k < count; k += 4 * nt) {
    int32_t c[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) c[j] = k + j * nt < count ? __ldg(idx + k + j * nt) : 0;
#pragma unroll
    for (int j = 0; j < 4; ++j) s += v[c[j]];
  }
  out[t0] = s;
}

}  // namespace

extern "C" qp_status qp_gather_rate(int64_t count, int32_t n, int32_t reps, uint64_t seed,
                                    double* gathers_per_s) {
  if (count < 1 || n < 1 || reps < 1 || !gathers_per_s) {
    pdhcg_set_last_error("qp_gather_rate: count, n and reps must be positive");
    return QP_ERR_INVALID_ARG;
  }
  int sms = 0, dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    pdhcg_set_last_error("qp_gather_rate: no CUDA device");
    return QP_ERR_NO_DEVICE;
  }
  const int grid = sms * 8, block = 256;
  int32_t* idx = nullptr;
  float *v = nullptr, *out = nullptr;
  cudaStream_t s = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  qp_status st = QP_OK;
  if (cudaMalloc(&idx, size_t(count) * sizeof(int32_t)) != cudaSuccess ||
      cudaMalloc(&v, size_t(n) * sizeof(float)) != cudaSuccess ||
      cudaMalloc(&out, size_t(grid) * block * sizeof(float)) != cudaSuccess) {
    pdhcg_set_last_error("qp_gather_rate: cudaMalloc failed");
    st = QP_ERR_OOM;
  }
  if (st == QP_OK && (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess ||
                      cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)) {
    pdhcg_set_last_error("qp_gather_rate: stream/event creation failed");
    st = QP_ERR_CUDA;
  }
  if (st == QP_OK) {
    k_fill_indices<<<grid, block, 0, s>>>(idx, count, n, seed);
    k_fill_vector<<<grid, block, 0, s>>>(v, n);
    k_gather<<<grid, block, 0, s>>>(idx, count, v, out);  // warm-up: v into L2
    float best = 0.f;
    for (int r = 0; r < reps && st == QP_OK; ++r) {
      cudaEventRecord(e0, s);
      k_gather<<<grid, block, 0, s>>>(idx, count, v, out);
      cudaEventRecord(e1, s);
      if (cudaEventSynchronize(e1) != cudaSuccess) {
        st = QP_ERR_CUDA;
        break;
      }
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      if (ms > 0.f && (best == 0.f || ms < best)) best = ms;
    }
    if (st == QP_OK && cudaGetLastError() != cudaSuccess) st = QP_ERR_CUDA;
    if (st == QP_OK) *gathers_per_s = best > 0.f ? double(count) / (double(best) * 1e-3) : 0.0;
    if (st != QP_OK) pdhcg_set_last_error("qp_gather_rate: kernel failed");
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  if (s) {
    cudaStreamSynchronize(s);
    cudaStreamDestroy(s);
  }
  cudaFree(idx);
  cudaFree(v);
  cudaFree(out);
  cudaGetLastError();
  return st;
}
