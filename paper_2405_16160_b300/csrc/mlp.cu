// The learned warm start's network (qp_mlp_* in include/pdhcg.h): a
// multilayer perceptron with ReLU after every layer but the last, its
// weighted squared-error loss, backpropagation and the Adam update, all in
// FP32 kernels written here.  Activations are row-major (a row per sample);
// layer l maps width[l-1] -> width[l] as z = a W + b with W row-major
// (width[l-1] x width[l]); parameters are packed in layer order, W then b.
//
// The products are three shapes of one tiled GEMM (C = op(A) op(B) with an
// optional bias, ReLU or ReLU-mask epilogue): a W (forward), a' dZ (weight
// gradient) and dZ W' (back through a layer).  Every output element is
// summed by one thread in a fixed order, so results do not depend on the
// launch; the bias gradient and the loss are reduced in a fixed order too.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <vector>

#include "../../include/pdhcg.h"

void pdhcg_set_last_error(const char* msg);

namespace {

void merror(const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  pdhcg_set_last_error(buf);
}

#define MCUDA(call)                                                                       \
  do {                                                                                    \
    cudaError_t e_ = (call);                                                              \
    if (e_ != cudaSuccess) {                                                              \
      merror("%s failed: %s (%s:%d)", #call, cudaGetErrorString(e_), __FILE__, __LINE__); \
      return QP_ERR_CUDA;                                                                 \
    }                                                                                     \
  } while (0)

#define MTRY(call)              \
  do {                          \
    qp_status s_ = (call);      \
    if (s_ != QP_OK) return s_; \
  } while (0)

constexpr int kBM = 64, kBN = 64, kBK = 16;  // GEMM tile
constexpr int kEpiNone = 0, kEpiRelu = 1, kEpiMask = 2;

// C (M x N, row-major, ldc = N) = op(A) op(B) (+ bias) with the epilogue:
//   kEpiRelu  max(., 0)
//   kEpiMask  . * (mask > 0), mask M x N like C (ReLU backward)
// op(A) is M x K: A row-major M x K (TA = false) or K x M (TA = true).
// op(B) is K x N: B row-major K x N (TB = false) or N x K (TB = true).
// 256 threads, each a 4 x 4 block of C at rows ty + 16 i, columns tx + 16 j.
template <bool TA, bool TB, int EPI>
__global__ void __launch_bounds__(256) k_gemm(int M, int N, int K, const float* __restrict__ A,
                                              const float* __restrict__ B,
                                              const float* __restrict__ bias,
                                              const float* __restrict__ mask, float* C) {
  __shared__ float As[kBK][kBM + 4];
  __shared__ float Bs[kBK][kBN + 4];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int m0 = blockIdx.y * kBM, n0 = blockIdx.x * kBN;
  float acc[4][4] = {};
  for (int k0 = 0; k0 < K; k0 += kBK) {
    // 1024 elements of each tile, 4 per thread
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      const int idx = tid + 256 * e;
      int mm, kk;
      if (TA) {  // coalesced along m
        kk = idx / kBM;
        mm = idx % kBM;
      } else {  // coalesced along k
        mm = idx / kBK;
        kk = idx % kBK;
      }
      const int gm = m0 + mm, gk = k0 + kk;
      float v = 0.f;
      if (gm < M && gk < K) v = TA ? A[size_t(gk) * M + gm] : A[size_t(gm) * K + gk];
      As[kk][mm] = v;
      int nn;
      if (TB) {  // coalesced along k
        nn = idx / kBK;
        kk = idx % kBK;
      } else {  // coalesced along n
        kk = idx / kBN;
        nn = idx % kBN;
      }
      const int gn = n0 + nn, gk2 = k0 + kk;
      float u = 0.f;
      if (gn < N && gk2 < K) u = TB ? B[size_t(gn) * K + gk2] : B[size_t(gk2) * N + gn];
      Bs[kk][nn] = u;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kBK; ++kk) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const int gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      float v = acc[i][j];
      if (bias) v += bias[gn];
      if (EPI == kEpiRelu) v = fmaxf(v, 0.f);
      if (EPI == kEpiMask) v = mask[size_t(gm) * N + gn] > 0.f ? v : 0.f;
      C[size_t(gm) * N + gn] = v;
    }
  }
}

// d loss / d out = (2/B) w_j (out - target), and per-block partial sums of
// w_j (out - target)^2 (the loss before the division by B).
__global__ void __launch_bounds__(256) k_mse_grad(int B, int N, const float* __restrict__ out,
                                                  const float* __restrict__ target,
                                                  const float* __restrict__ w, float* grad,
                                                  double* part) {
  __shared__ double red[256];
  const long long total = (long long)B * N;
  const float scale = 2.f / float(B);
  double s = 0.0;
  for (long long i = (long long)blockIdx.x * 256 + threadIdx.x; i < total;
       i += (long long)gridDim.x * 256) {
    const int j = int(i % N);
    const float wj = w ? w[j] : 1.f;
    const float d = out[i] - target[i];
    grad[i] = scale * wj * d;
    s += double(wj) * double(d) * double(d);
  }
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_loss_finish(const double* part, int n, int B, double* loss) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += part[i];
  *loss = s / double(B);
}

// db_j = sum_r dZ_rj, rows in order.
__global__ void k_colsum(int B, int N, const float* __restrict__ g, float* out) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= N) return;
  float s = 0.f;
  for (int r = 0; r < B; ++r) s += g[size_t(r) * N + j];
  out[j] = s;
}

// Adam with the bias corrections c1 = 1/(1 - beta1^t), c2 = 1/(1 - beta2^t).
__global__ void k_adam(long long n, float* p, const float* __restrict__ g, float* m, float* v,
                       float lr, float b1, float b2, float eps, float c1, float c2) {
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = b1 * m[i] + (1.f - b1) * gi;
    const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi * c1) / (sqrtf(vi * c2) + eps);
  }
}

}  // namespace

struct qp_mlp {
  int device = 0;
  cudaStream_t stream = nullptr, user_stream = nullptr;
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  qp_device_ctx ctx{};
  bool has_alloc = false;
  std::vector<std::pair<void*, size_t>> allocs;
  std::vector<int32_t> widths;
  int max_batch = 0;
  int64_t nparam = 0;
  std::vector<int64_t> w_off, b_off;  // per layer, into the packed vectors
  float *params = nullptr, *grad = nullptr, *m = nullptr, *v = nullptr;
  std::vector<float*> act;  // hidden activations a_1..a_{L-1} (max_batch x width)
  float *out = nullptr, *gout = nullptr, *gtmp = nullptr;
  double *part = nullptr, *loss = nullptr;
  int nparts = 0;
  long long step = 0;
};

namespace {

qp_status malloc_dev(qp_mlp* h, void** out, size_t bytes) {
  bytes = (std::max<size_t>(bytes, 256) + 255) & ~size_t(255);
  void* ptr = nullptr;
  if (h->has_alloc) {
    ptr = h->ctx.alloc(bytes, h->ctx.user, h->ctx.stream);
    if (!ptr) {
      merror("device allocator callback returned NULL for %zu bytes", bytes);
      return QP_ERR_OOM;
    }
  } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
    cudaGetLastError();
    merror("cudaMalloc(%zu) failed", bytes);
    return QP_ERR_OOM;
  }
  h->allocs.emplace_back(ptr, bytes);
  *out = ptr;
  return QP_OK;
}

template <class T>
qp_status falloc(qp_mlp* h, T** out, size_t count) {
  return malloc_dev(h, reinterpret_cast<void**>(out), count * sizeof(T));
}

qp_status mbegin(qp_mlp* h) {
  MCUDA(cudaSetDevice(h->device));
  // the caller's stream; 0 is the legacy default stream (PyTorch's default)
  MCUDA(cudaEventRecord(h->ev_a, h->user_stream));
  MCUDA(cudaStreamWaitEvent(h->stream, h->ev_a, 0));
  return QP_OK;
}

qp_status mend(qp_mlp* h) {
  MCUDA(cudaEventRecord(h->ev_b, h->stream));
  MCUDA(cudaStreamWaitEvent(h->user_stream, h->ev_b, 0));
  return QP_OK;
}

template <bool TA, bool TB, int EPI>
void gemm(qp_mlp* h, int M, int N, int K, const float* A, const float* B, const float* bias,
          const float* mask, float* C) {
  const dim3 grid((N + kBN - 1) / kBN, (M + kBM - 1) / kBM);
  k_gemm<TA, TB, EPI><<<grid, 256, 0, h->stream>>>(M, N, K, A, B, bias, mask, C);
}

// Forward pass of `batch` rows; the output lands in h->out.
qp_status run_forward(qp_mlp* h, int batch, const float* in) {
  const int L = int(h->widths.size()) - 1;
  const float* a = in;
  for (int l = 0; l < L; ++l) {
    const int K = h->widths[size_t(l)], N = h->widths[size_t(l) + 1];
    const float* W = h->params + h->w_off[size_t(l)];
    const float* b = h->params + h->b_off[size_t(l)];
    if (l + 1 < L) {
      gemm<false, false, kEpiRelu>(h, batch, N, K, a, W, b, nullptr, h->act[size_t(l)]);
      a = h->act[size_t(l)];
    } else {
      gemm<false, false, kEpiNone>(h, batch, N, K, a, W, b, nullptr, h->out);
    }
  }
  MCUDA(cudaGetLastError());
  return QP_OK;
}

}  // namespace

extern "C" {

qp_status qp_mlp_create(qp_mlp** out, int32_t n_layers, const int32_t* widths, int32_t max_batch,
                        const qp_device_ctx* ctx) {
  if (!out) return QP_ERR_INVALID_ARG;
  *out = nullptr;
  if (n_layers < 1 || n_layers > 16 || !widths || max_batch < 1) {
    merror("bad network: %d layers, max batch %d", n_layers, max_batch);
    return QP_ERR_INVALID_ARG;
  }
  for (int l = 0; l <= n_layers; ++l)
    if (widths[l] < 1 || widths[l] > (1 << 20)) {
      merror("bad width %d at %d", widths[l], l);
      return QP_ERR_INVALID_ARG;
    }
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    merror("no CUDA device visible");
    return QP_ERR_NO_DEVICE;
  }
  qp_mlp* h = new qp_mlp();
  cudaGetDevice(&h->device);
  if (ctx) {
    h->ctx = *ctx;
    h->has_alloc = ctx->alloc && ctx->free;
    h->user_stream = static_cast<cudaStream_t>(ctx->stream);
  }
  h->widths.assign(widths, widths + n_layers + 1);
  h->max_batch = max_batch;
  int64_t o = 0;
  for (int l = 0; l < n_layers; ++l) {
    h->w_off.push_back(o);
    o += int64_t(widths[l]) * widths[l + 1];
    h->b_off.push_back(o);
    o += widths[l + 1];
  }
  h->nparam = o;
  qp_status s = QP_OK;
  if (cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_a, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreateWithFlags(&h->ev_b, cudaEventDisableTiming) != cudaSuccess) {
    cudaGetLastError();
    merror("stream/event creation failed");
    s = QP_ERR_CUDA;
  }
  auto step = [&](qp_status s2) {
    if (s == QP_OK) s = s2;
  };
  step(falloc(h, &h->params, size_t(o)));
  step(falloc(h, &h->grad, size_t(o)));
  step(falloc(h, &h->m, size_t(o)));
  step(falloc(h, &h->v, size_t(o)));
  int wmax = 0;
  for (int l = 0; l <= n_layers; ++l) wmax = std::max(wmax, widths[l]);
  for (int l = 1; l < n_layers; ++l) {
    float* a = nullptr;
    step(falloc(h, &a, size_t(max_batch) * widths[l]));
    h->act.push_back(a);
  }
  step(falloc(h, &h->out, size_t(max_batch) * widths[n_layers]));
  step(falloc(h, &h->gout, size_t(max_batch) * wmax));
  step(falloc(h, &h->gtmp, size_t(max_batch) * wmax));
  h->nparts = 296;
  step(falloc(h, &h->part, size_t(h->nparts)));
  step(falloc(h, &h->loss, 1));
  if (s == QP_OK) {
    s = mbegin(h);
    if (s == QP_OK && cudaMemsetAsync(h->params, 0, size_t(o) * sizeof(float), h->stream) != 0)
      s = QP_ERR_CUDA;
    if (s == QP_OK) s = mend(h);
  }
  if (s != QP_OK) {
    qp_mlp_destroy(h);
    return s;
  }
  *out = h;
  return QP_OK;
}

void qp_mlp_destroy(qp_mlp* h) {
  if (!h) return;
  cudaSetDevice(h->device);
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& a : h->allocs) {
    if (h->has_alloc)
      h->ctx.free(a.first, a.second, h->ctx.user, h->ctx.stream);
    else
      cudaFree(a.first);
  }
  if (h->ev_a) cudaEventDestroy(h->ev_a);
  if (h->ev_b) cudaEventDestroy(h->ev_b);
  if (h->stream) cudaStreamDestroy(h->stream);
  delete h;
}

int64_t qp_mlp_param_count(const qp_mlp* h) { return h ? h->nparam : 0; }

qp_status qp_mlp_set_params(qp_mlp* h, const float* params) {
  if (!h || !params) return QP_ERR_INVALID_ARG;
  MTRY(mbegin(h));
  const size_t bytes = size_t(h->nparam) * sizeof(float);
  MCUDA(cudaMemcpyAsync(h->params, params, bytes, cudaMemcpyHostToDevice, h->stream));
  MCUDA(cudaMemsetAsync(h->m, 0, bytes, h->stream));
  MCUDA(cudaMemsetAsync(h->v, 0, bytes, h->stream));
  MCUDA(cudaStreamSynchronize(h->stream));
  h->step = 0;
  return mend(h);
}

qp_status qp_mlp_get_params(const qp_mlp* hc, float* params) {
  if (!hc || !params) return QP_ERR_INVALID_ARG;
  qp_mlp* h = const_cast<qp_mlp*>(hc);
  MTRY(mbegin(h));
  MCUDA(cudaMemcpyAsync(params, h->params, size_t(h->nparam) * sizeof(float),
                        cudaMemcpyDeviceToHost, h->stream));
  MCUDA(cudaStreamSynchronize(h->stream));
  return mend(h);
}

qp_status qp_mlp_forward(qp_mlp* h, int32_t batch, const float* in, float* out) {
  if (!h || !in || !out || batch < 1 || batch > h->max_batch) return QP_ERR_INVALID_ARG;
  MTRY(mbegin(h));
  MTRY(run_forward(h, batch, in));
  MCUDA(cudaMemcpyAsync(out, h->out, size_t(batch) * h->widths.back() * sizeof(float),
                        cudaMemcpyDeviceToDevice, h->stream));
  return mend(h);
}

qp_status qp_mlp_loss_grad(qp_mlp* h, int32_t batch, const float* in, const float* target,
                           const float* w, float* grad, double* loss) {
  if (!h || !in || !target || batch < 1 || batch > h->max_batch) return QP_ERR_INVALID_ARG;
  MTRY(mbegin(h));
  MTRY(run_forward(h, batch, in));
  const int L = int(h->widths.size()) - 1;
  const int nout = h->widths.back();
  k_mse_grad<<<h->nparts, 256, 0, h->stream>>>(batch, nout, h->out, target, w, h->gout, h->part);
  k_loss_finish<<<1, 32, 0, h->stream>>>(h->part, h->nparts, batch, h->loss);
  // backward: g holds d loss / d z_l (batch x width[l+1])
  float* g = h->gout;
  float* other = h->gtmp;
  for (int l = L - 1; l >= 0; --l) {
    const int K = h->widths[size_t(l)], N = h->widths[size_t(l) + 1];
    const float* a_prev = l == 0 ? in : h->act[size_t(l) - 1];
    gemm<true, false, kEpiNone>(h, K, N, batch, a_prev, g, nullptr, nullptr,
                                h->grad + h->w_off[size_t(l)]);
    k_colsum<<<(N + 255) / 256, 256, 0, h->stream>>>(batch, N, g, h->grad + h->b_off[size_t(l)]);
    if (l > 0) {
      // d loss / d z_{l-1} = (g W') * (a_{l-1} > 0)
      gemm<false, true, kEpiMask>(h, batch, K, N, g, h->params + h->w_off[size_t(l)], nullptr,
                                  a_prev, other);
      std::swap(g, other);
    }
  }
  MCUDA(cudaGetLastError());
  if (grad)
    MCUDA(cudaMemcpyAsync(grad, h->grad, size_t(h->nparam) * sizeof(float),
                          cudaMemcpyDeviceToDevice, h->stream));
  if (loss) {
    MCUDA(cudaMemcpyAsync(loss, h->loss, sizeof(double), cudaMemcpyDeviceToHost, h->stream));
    MCUDA(cudaStreamSynchronize(h->stream));
  }
  return mend(h);
}

qp_status qp_mlp_adam_step(qp_mlp* h, float lr) {
  if (!h || !(lr > 0.f)) return QP_ERR_INVALID_ARG;
  MTRY(mbegin(h));
  h->step += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = float(1.0 / (1.0 - std::pow(b1, double(h->step))));
  const float c2 = float(1.0 / (1.0 - std::pow(b2, double(h->step))));
  const int grid = int(std::min<int64_t>((h->nparam + 255) / 256, 1184));
  k_adam<<<grid, 256, 0, h->stream>>>(h->nparam, h->params, h->grad, h->m, h->v, lr, float(b1),
                                      float(b2), 1e-8f, c1, c2);
  MCUDA(cudaGetLastError());
  return mend(h);
}

}  // extern "C"
