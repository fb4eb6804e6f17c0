// One instantiation of the batched solver's kernel, k_batch<BATCH_V,
// BATCH_NT>, with its host entry points (BatchLaunch, batch_kernels.cuh).
// The build compiles this file once per value type (float, double) and block
// size (64, 128, 256, 512).
#include "batch_kernels.cuh"

#if !defined(BATCH_V) || !defined(BATCH_NT)
#error "compile with -DBATCH_V=<float|double> -DBATCH_NT=<64|128|256|512>"
#endif

namespace pdhcg {

template <class V, int NT>
cudaError_t BatchLaunch<V, NT>::prepare(size_t smem, int* occupancy) {
  const cudaError_t e =
      cudaFuncSetAttribute(k_batch<V, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, int(smem));
  if (e != cudaSuccess) return e;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occupancy, k_batch<V, NT>, NT, smem);
}

template <class V, int NT>
cudaError_t BatchLaunch<V, NT>::launch(int grid, size_t smem, cudaStream_t stream,
                                       const BatchData<V>& B) {
  k_batch<V, NT><<<grid, NT, smem, stream>>>(B);
  return cudaGetLastError();
}

template struct BatchLaunch<BATCH_V, BATCH_NT>;

}  // namespace pdhcg
