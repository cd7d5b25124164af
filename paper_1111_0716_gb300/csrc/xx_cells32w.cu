// Batched passes C and role-swapped C over several cells, FP32, for launches
// whose largest body has at most 640 threads (grid lengths up to 80): the
// 640-thread bound leaves each thread 96 registers, which the 80-point body
// needs without spilling (the 768-thread kernel, which also serves length 96,
// has 80).  See xx_cells.cuh.
#include "xx_cells.cuh"

namespace xx {

cudaError_t launch_cell_pass32_640(int pass, const CellItems& items, long long ctas, int threads,
                                   size_t smem, cudaStream_t s) {
  if (threads > 640 || (pass != kCellPassC && pass != kCellPassCT)) return cudaErrorInvalidValue;
  if (pass == kCellPassC) {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_cells<float, kCellPassC, 640, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cells<float, kCellPassC, 640, 1><<<(unsigned)ctas, threads, smem, s>>>(items);
  } else {
    if (smem > 48 * 1024)
      cudaFuncSetAttribute(k_cells<float, kCellPassCT, 640, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_cells<float, kCellPassCT, 640, 1><<<(unsigned)ctas, threads, smem, s>>>(items);
  }
  return cudaGetLastError();
}

}  // namespace xx
