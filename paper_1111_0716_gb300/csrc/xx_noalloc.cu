// xx_noalloc.cu -- the E_x reduction for callers that cannot allocate device
// memory.
//
// xx_energy_from_vx keeps its per-target partial sums in workspace that the
// plan allocates with cudaMalloc.  Some callers cannot do that: applications
// whose memory manager has already reserved the device memory (a framework's
// caching allocator, a fixed per-process budget), and callers that must not
// hit the device-wide synchronisation that cudaFree implies.  This file gives
// them xx_energy_from_vx_noalloc: the same fixed-order FP64 reduction, needing
// no plan, with its partial sums in a fixed-size array that lives in the
// library's device image.  The caller still passes every input and output.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/xx.h"

namespace {

constexpr int kThreads = 256;
constexpr double kSpin = 2.0;   // spin-paired: s = 2
constexpr int kMaxDevices = 64;

// Per-target partial sums <c_ka|vx_ka> (re, im).  Every GPU that loads the
// library holds this array until the process exits; all calls on a device
// share it.
static __device__ __align__(256) double2 xx_noalloc_dots[XX_NOALLOC_MAX_ROWS];

// Device address of xx_noalloc_dots for each device, looked up once per device.
double2* g_dots_addr[kMaxDevices] = {nullptr};
std::mutex g_setup_mutex;

// dots[row] = sum_g conj(c[row][g]) vx[row][g]; one CTA per row, fixed-order tree.
// The basis size comes from device memory the host cannot check, so it is
// clamped to [0, npw_max]: a bad npw never reads past a row.
__global__ void __launch_bounds__(kThreads) k_noalloc_dots(const double2* c, const double2* vx,
                                                           const int* npw, int n_tgt, int npw_max,
                                                           double2* dots) {
  __shared__ double re_s[kThreads], im_s[kThreads];
  const int row = blockIdx.x;
  const int n = min(max(npw[row / n_tgt], 0), npw_max);
  const double2* a = c + (long long)row * npw_max;
  const double2* b = vx + (long long)row * npw_max;
  double re = 0.0, im = 0.0;
  for (int g = threadIdx.x; g < n; g += kThreads) {
    const double2 x = a[g], y = b[g];
    re += x.x * y.x + x.y * y.y;
    im += x.x * y.y - x.y * y.x;
  }
  re_s[threadIdx.x] = re;
  im_s[threadIdx.x] = im;
  __syncthreads();
  for (int off = kThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      re_s[threadIdx.x] += re_s[threadIdx.x + off];
      im_s[threadIdx.x] += im_s[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) dots[row] = make_double2(re_s[0], im_s[0]);
}

// ex[0..1] = scale * sum_row w[row] dots[row]; one CTA, fixed order
__global__ void __launch_bounds__(kThreads) k_noalloc_energy(const double2* dots, const double* w,
                                                             int nrows, double scale, double* ex) {
  __shared__ double re_s[kThreads], im_s[kThreads];
  double re = 0.0, im = 0.0;
  for (int r = threadIdx.x; r < nrows; r += kThreads) {
    re += w[r] * dots[r].x;
    im += w[r] * dots[r].y;
  }
  re_s[threadIdx.x] = re;
  im_s[threadIdx.x] = im;
  __syncthreads();
  for (int off = kThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      re_s[threadIdx.x] += re_s[threadIdx.x + off];
      im_s[threadIdx.x] += im_s[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    ex[0] = scale * re_s[0];
    ex[1] = scale * im_s[0];
  }
}

int status_of(cudaError_t e) {
  if (e == cudaSuccess) return XX_OK;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return XX_ERR_NO_DEVICE;
  return XX_ERR_CUDA;
}

// The host-side name xx_noalloc_dots is only a stand-in for the device array:
// kernels get its device address, looked up here once per device with that
// device current.
int dots_address(double2** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return status_of(e);
  }
  if (dev < 0 || dev >= kMaxDevices) return XX_ERR_NO_DEVICE;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_dots_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, xx_noalloc_dots);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return status_of(e == cudaSuccess ? cudaErrorInvalidSymbol : e);
    }
    g_dots_addr[dev] = static_cast<double2*>(p);
  }
  *out = g_dots_addr[dev];
  return XX_OK;
}

}  // namespace

extern "C" int xx_energy_from_vx_noalloc(int nk, int n_tgt, int npw_max, const int* npw,
                                         const void* c_tgt, const double* w_tgt, const void* vx,
                                         double* ex_out, void* stream) {
  if (nk < 1 || n_tgt < 0 || npw_max < 1 || !npw || !ex_out) return XX_ERR_INVALID_ARGUMENT;
  if ((long long)nk * n_tgt > XX_NOALLOC_MAX_ROWS) return XX_ERR_SIZE_LIMIT;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (n_tgt == 0) return status_of(cudaMemsetAsync(ex_out, 0, 2 * sizeof(double), s));
  if (!c_tgt || !w_tgt || !vx) return XX_ERR_INVALID_ARGUMENT;
  double2* dots = nullptr;
  const int st = dots_address(&dots);
  if (st != XX_OK) return st;
  const int rows = nk * n_tgt;
  // every row of dots is written before it is read: nothing needs clearing
  k_noalloc_dots<<<rows, kThreads, 0, s>>>(static_cast<const double2*>(c_tgt),
                                           static_cast<const double2*>(vx), npw, n_tgt, npw_max,
                                           dots);
  k_noalloc_energy<<<1, kThreads, 0, s>>>(dots, w_tgt, rows, 0.5 * kSpin / nk, ex_out);
  return status_of(cudaGetLastError());
}
