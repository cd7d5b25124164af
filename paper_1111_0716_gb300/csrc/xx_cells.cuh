// xx_cells.cuh -- batched launches of the band-pair passes over several cells
// with different FFT grid lengths: one launch per pass covers every band-pair
// batch ("item") of every cell.  Each CTA finds its item in a table passed as
// a kernel parameter and runs the pass body of that item's grid length; the
// block is as large as the largest body needs, and the threads beyond the
// body's own count leave at once (the bodies synchronise on counted barriers).
#pragma once

#include "xx_kernels.cuh"

namespace xx {

// One band-pair batch of one cell.
struct CellItem {
  PairArgs a;             // the batch, exactly as the single-cell passes take it
  long long cta0;         // first CTA of this item in the launch
  int n;                  // length of the pass's transforms: x, y (passes A, C and the
                          // role-swapped C) or z (pass B) of the cell's grid
};

// Items of one launch; passed by value (kernel parameter space, < 32 KB).
constexpr int kMaxCellItems = 96;
struct CellItems {
  int n_items;
  CellItem item[kMaxCellItems];
};
static_assert(sizeof(CellItems) <= 32000, "kernel parameter space");

enum CellPass { kCellPassA = 0, kCellPassB = 1, kCellPassC = 2, kCellPassCT = 3 };

// CTAs of one item in a launch of the given pass.
inline long long cell_item_ctas(int pass, const PairArgs& a) {
  switch (pass) {
    case kCellPassA:
    case kCellPassC:
      return (long long)a.TA * a.nz;
    case kCellPassB:
      return (long long)a.P2 * a.TA * a.TJ;
    default:
      return (long long)a.TJ * a.nz;
  }
}

// Host side (xx_cells32.cu / xx_cells64.cu).  Length 108 has no batched body: its
// planes need more threads than the batched blocks hold.
// Threads and dynamic shared memory of the body of `pass` for grid length n
// (0 when n has no body); block size of a launch is the largest over its items.
bool cell_length_supported(int n);
int cell_body_threads(int pass, bool fp64, int n);
size_t cell_body_smem(int pass, bool fp64, int n, int P1, int P3);
// Launch one batched pass over the items (their cta0 already set); returns the
// CUDA launch error.
cudaError_t launch_cell_pass(int pass, bool fp64, const CellItems& items, long long total_ctas,
                             int threads, size_t smem, cudaStream_t s);

// ------------------------------------------------------------- device side --

// Pass A plane of the batched launch: one buffer as in the single-cell pass A,
// except FP32 at N = 60 (A = 6, B = 10), whose one-buffer plane needs 480
// threads; its two-buffer plane needs 384, which keeps the batched pass A at
// 384 threads, two CTAs per SM.
template <int N, typename T> __host__ __device__ constexpr bool cell_pass_a_db() {
  return sizeof(T) == 4 && N == 60;
}

// The item a CTA belongs to (items sorted by cta0; a handful per launch).
__device__ __forceinline__ int cell_item_of(const CellItems& it, long long b) {
  int i = 0;
  while (i + 1 < it.n_items && it.item[i + 1].cta0 <= b) ++i;
  return i;
}

template <int N, typename T, int PASS>
__device__ __forceinline__ void cell_body(const PairArgs& a, long long l, unsigned char* smem) {
  if constexpr (PASS == kCellPassA) {
    constexpr bool DB = cell_pass_a_db<N, T>();
    if (threadIdx.x < PlaneCfg<N, T, DB>::NT) pass_a_body<N, T, DB>(a, (int)(l % a.TA), (int)(l / a.TA), smem);
  } else if constexpr (PASS == kCellPassB) {
    // consecutive CTAs take consecutive f_y rows of one pair, as the single-cell
    // launch does (its grid is (P2, pairs)), so neighbouring CTAs read neighbouring rows
    constexpr int NTB = 256;
    if (threadIdx.x < NTB) pass_b_body<N, NTB, T>(a, (int)(l % a.P2), (int)(l / a.P2), smem);
  } else if constexpr (PASS == kCellPassC) {
    if (threadIdx.x < PlaneCfg<N, T>::NT) pass_c_body<N, T, false>(a, (int)(l % a.TA), (int)(l / a.TA), smem);
  } else {
    if (threadIdx.x < PlaneCfg<N, T>::NT) pass_ct_body<N, T>(a, (int)(l % a.TJ), (int)(l / a.TJ), smem);
  }
}

// Threads of a body (what cell_body_threads reports on the host).
template <int N, typename T, int PASS> __host__ __device__ constexpr int cell_body_nt() {
  if constexpr (PASS == kCellPassB) return 256;
  else if constexpr (PASS == kCellPassA) return PlaneCfg<N, T, cell_pass_a_db<N, T>()>::NT;
  else return PlaneCfg<N, T>::NT;
}

// A body is compiled into a kernel only when its threads fit the kernel's
// block bound; the host picks a kernel whose bound covers every item's body.
template <int N, typename T, int PASS, int NTMAX>
__device__ __forceinline__ void cell_body_fit(const PairArgs& a, long long l, unsigned char* smem) {
  if constexpr (cell_body_nt<N, T, PASS>() <= NTMAX) cell_body<N, T, PASS>(a, l, smem);
}

template <typename T, int PASS, int NTMAX, int MINB>
__global__ void __launch_bounds__(NTMAX, MINB) k_cells(const __grid_constant__ CellItems items) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  const long long b = blockIdx.x;
  const int i = cell_item_of(items, b);
  const CellItem& it = items.item[i];
  const long long l = b - it.cta0;
  switch (it.n) {
    case 24: cell_body_fit<24, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    case 32: cell_body_fit<32, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    case 36: cell_body_fit<36, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    case 40: cell_body_fit<40, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    case 48: cell_body_fit<48, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    case 54: cell_body_fit<54, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    case 60: cell_body_fit<60, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    case 64: cell_body_fit<64, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    case 72: cell_body_fit<72, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    case 80: cell_body_fit<80, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    case 96: cell_body_fit<96, T, PASS, NTMAX>(it.a, l, smem_raw); break;
    default: break;
  }
}

}  // namespace xx
