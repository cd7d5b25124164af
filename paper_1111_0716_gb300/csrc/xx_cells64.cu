// Batched band-pair passes over several cells, FP64 (see xx_cells.cuh).
#include "xx_cells.cuh"

namespace xx {

constexpr int kCellThreads64[4] = {480, 256, 480, 480};   // A, B, C, CT: largest body

cudaError_t launch_cell_pass64(int pass, const CellItems& items, long long ctas, int threads,
                               size_t smem, cudaStream_t s) {
  if (threads > kCellThreads64[pass]) return cudaErrorInvalidValue;
  switch (pass) {
    case kCellPassA:
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_cells<double, kCellPassA, 480, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_cells<double, kCellPassA, 480, 1><<<(unsigned)ctas, threads, smem, s>>>(items);
      break;
    case kCellPassB:
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_cells<double, kCellPassB, 256, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_cells<double, kCellPassB, 256, 1><<<(unsigned)ctas, threads, smem, s>>>(items);
      break;
    case kCellPassC:
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_cells<double, kCellPassC, 480, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_cells<double, kCellPassC, 480, 1><<<(unsigned)ctas, threads, smem, s>>>(items);
      break;
    default:
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_cells<double, kCellPassCT, 480, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_cells<double, kCellPassCT, 480, 1><<<(unsigned)ctas, threads, smem, s>>>(items);
      break;
  }
  return cudaGetLastError();
}

}  // namespace xx
