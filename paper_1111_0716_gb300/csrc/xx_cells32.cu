// Batched band-pair passes over several cells, FP32, and the host helpers of
// both precisions (see xx_cells.cuh).
#include "xx_cells.cuh"

namespace xx {

cudaError_t launch_cell_pass64(int pass, const CellItems& items, long long ctas, int threads,
                               size_t smem, cudaStream_t s);
cudaError_t launch_cell_pass32_640(int pass, const CellItems& items, long long ctas, int threads,
                                   size_t smem, cudaStream_t s);

namespace {

constexpr int kCellThreads32[4] = {384, 256, 768, 768};   // A, B, C, CT: largest body

template <int N>
int body_threads(int pass, bool fp64) {
  if (pass == kCellPassB) return 256;
  if (pass == kCellPassA)
    return fp64 ? PlaneCfg<N, double, cell_pass_a_db<N, double>()>::NT
                : PlaneCfg<N, float, cell_pass_a_db<N, float>()>::NT;
  return fp64 ? PlaneCfg<N, double>::NT : PlaneCfg<N, float>::NT;
}

template <int N>
size_t body_smem(int pass, bool fp64, int P1, int P3) {
  if (pass == kCellPassB) return fp64 ? smem_pencil<N, double>(P1, P3) : smem_pencil<N, float>(P1, P3);
  // the same sizes as the single-cell launchers
  if (pass == kCellPassA)
    return fp64 ? PlaneCfg<N, double, cell_pass_a_db<N, double>()>::smem()
                : PlaneCfg<N, float, cell_pass_a_db<N, float>()>::smem();
  return fp64 ? PlaneCfg<N, double>::smem() : PlaneCfg<N, float>::smem();
}

}  // namespace

bool cell_length_supported(int n) {
  switch (n) {
    case 24: case 32: case 36: case 40: case 48: case 54: case 60: case 64: case 72: case 80: case 96:
      return true;
    default:
      return false;
  }
}

int cell_body_threads(int pass, bool fp64, int n) {
  switch (n) {
    case 24: return body_threads<24>(pass, fp64);
    case 32: return body_threads<32>(pass, fp64);
    case 36: return body_threads<36>(pass, fp64);
    case 40: return body_threads<40>(pass, fp64);
    case 48: return body_threads<48>(pass, fp64);
    case 54: return body_threads<54>(pass, fp64);
    case 60: return body_threads<60>(pass, fp64);
    case 64: return body_threads<64>(pass, fp64);
    case 72: return body_threads<72>(pass, fp64);
    case 80: return body_threads<80>(pass, fp64);
    case 96: return body_threads<96>(pass, fp64);
    default: return 0;
  }
}

size_t cell_body_smem(int pass, bool fp64, int n, int P1, int P3) {
  switch (n) {
    case 24: return body_smem<24>(pass, fp64, P1, P3);
    case 32: return body_smem<32>(pass, fp64, P1, P3);
    case 36: return body_smem<36>(pass, fp64, P1, P3);
    case 40: return body_smem<40>(pass, fp64, P1, P3);
    case 48: return body_smem<48>(pass, fp64, P1, P3);
    case 54: return body_smem<54>(pass, fp64, P1, P3);
    case 60: return body_smem<60>(pass, fp64, P1, P3);
    case 64: return body_smem<64>(pass, fp64, P1, P3);
    case 72: return body_smem<72>(pass, fp64, P1, P3);
    case 80: return body_smem<80>(pass, fp64, P1, P3);
    case 96: return body_smem<96>(pass, fp64, P1, P3);
    default: return 0;
  }
}

cudaError_t launch_cell_pass(int pass, bool fp64, const CellItems& items, long long ctas,
                             int threads, size_t smem, cudaStream_t s) {
  if (pass < 0 || pass > 3 || ctas <= 0 || ctas > 0x7fffffffLL) return cudaErrorInvalidValue;
  if (fp64) return launch_cell_pass64(pass, items, ctas, threads, smem, s);
  if (threads > kCellThreads32[pass]) return cudaErrorInvalidValue;
  if ((pass == kCellPassC || pass == kCellPassCT) && threads <= 640)
    return launch_cell_pass32_640(pass, items, ctas, threads, smem, s);
  switch (pass) {
    case kCellPassA:
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_cells<float, kCellPassA, 384, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_cells<float, kCellPassA, 384, 2><<<(unsigned)ctas, threads, smem, s>>>(items);
      break;
    case kCellPassB:
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_cells<float, kCellPassB, 256, 3>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_cells<float, kCellPassB, 256, 3><<<(unsigned)ctas, threads, smem, s>>>(items);
      break;
    case kCellPassC:
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_cells<float, kCellPassC, 768, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_cells<float, kCellPassC, 768, 1><<<(unsigned)ctas, threads, smem, s>>>(items);
      break;
    default:
      if (smem > 48 * 1024)
        cudaFuncSetAttribute(k_cells<float, kCellPassCT, 768, 1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      k_cells<float, kCellPassCT, 768, 1><<<(unsigned)ctas, threads, smem, s>>>(items);
      break;
  }
  return cudaGetLastError();
}

}  // namespace xx
