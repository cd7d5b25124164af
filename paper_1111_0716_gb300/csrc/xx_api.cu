// xx_api.cu -- C ABI of the Fock-exchange library: plan creation, workspace,
// the host loops over k, q and band-pair batches, and the FP64 reductions.
//
// Host loop structure (Hutchinson & Widom, Sec. "Our Implementation": outer
// loops over two k-points on the host, inner band loops on the GPU, the
// innermost band loop multiplexed into batches whose size bounds GPU memory):
//   sphere -> grid for every target and occupied orbital (once each)
//   for k: zero the FP64 accumulators of the targets of k
//     for q: kernel table v(k - q + G)
//       for each (target batch, occupied batch): pass A, pass B, pass C
//     grid -> sphere of the accumulators into V_x c
// (with the pair symmetry, blocks q > k also feed the targets of q, and the
// accumulators of every k-point are zeroed once up front)
#include <cudaTypedefs.h>
#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <ctime>
#include <new>
#include <vector>

#include "../../include/xx.h"
#include "xx_cells.cuh"
#include "xx_launch.cuh"

namespace xx {
const KernelTable* kernel_table_24();
const KernelTable* kernel_table_32();
const KernelTable* kernel_table_36();
const KernelTable* kernel_table_40();
const KernelTable* kernel_table_48();
const KernelTable* kernel_table_54();
const KernelTable* kernel_table_60();
const KernelTable* kernel_table_64();
const KernelTable* kernel_table_72();
const KernelTable* kernel_table_80();
const KernelTable* kernel_table_96();
const KernelTable* kernel_table_108();

const KernelTable* kernel_table(int n) {
  switch (n) {
    case 24: return kernel_table_24();
    case 32: return kernel_table_32();
    case 36: return kernel_table_36();
    case 40: return kernel_table_40();
    case 48: return kernel_table_48();
    case 54: return kernel_table_54();
    case 60: return kernel_table_60();
    case 64: return kernel_table_64();
    case 72: return kernel_table_72();
    case 80: return kernel_table_80();
    case 96: return kernel_table_96();
    case 108: return kernel_table_108();
    default: return nullptr;
  }
}

constexpr int kRedThreads = 256;
constexpr double kSpin = 2.0;   // spin-paired: s = 2

// out[b][g] = scale * box[b][m3][m2][m1] for g < npw, zero padding up to npw_max
__global__ void k_g2s_gather(GridArgs g) {
  const long long total = (long long)g.nb * g.npw_max;
  const double2* box = reinterpret_cast<const double2*>(g.box);
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / g.npw_max), ig = (int)(i % g.npw_max);
    double2 v = make_double2(0.0, 0.0);
    if (ig < g.npw) {
      const int* m = g.miller + 3 * ig;
      const int x = m[0] + g.n1, y = m[1] + g.n2, z = m[2] + g.n3;
      if (x < 0 || x >= g.Q1 || y < 0 || y >= g.Q2 || z < 0 || z >= g.Q3) {
        atomicOr(g.err, 2);
      } else {
        const double2 s = box[(((long long)b * g.Q3 + z) * g.Q2 + y) * g.Q1 + x];
        v = make_double2(g.scale * s.x, g.scale * s.y);
      }
    }
    g.out[i] = v;
  }
}

// dots[row] = sum_g conj(c[row][g]) vx[row][g], fixed-order block reduction
__global__ void __launch_bounds__(kRedThreads) k_dot_rows(const double2* c, const double2* vx,
                                                          const int* npw, int n_per_k, int npw_max,
                                                          double2* dots) {
  __shared__ double re_s[kRedThreads], im_s[kRedThreads];
  const int row = blockIdx.x;
  const int n = npw[row / n_per_k];
  const double2* a = c + (long long)row * npw_max;
  const double2* b = vx + (long long)row * npw_max;
  double re = 0.0, im = 0.0;
  for (int g = threadIdx.x; g < n; g += kRedThreads) {
    const double2 x = a[g], y = b[g];
    re += x.x * y.x + x.y * y.y;
    im += x.x * y.y - x.y * y.x;
  }
  re_s[threadIdx.x] = re;
  im_s[threadIdx.x] = im;
  __syncthreads();
  for (int off = kRedThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) {
      re_s[threadIdx.x] += re_s[threadIdx.x + off];
      im_s[threadIdx.x] += im_s[threadIdx.x + off];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) dots[row] = make_double2(re_s[0], im_s[0]);
}

// ex[0..1] = scale * sum_row w[row] dots[row], one CTA, fixed order
__global__ void __launch_bounds__(kRedThreads) k_energy(const double2* dots, const double* w,
                                                        int nrows, double scale, double* ex) {
  __shared__ double re_s[kRedThreads], im_s[kRedThreads];
  double re = 0.0, im = 0.0;
  for (int r = threadIdx.x; r < nrows; r += kRedThreads) {
    re += w[r] * dots[r].x;
    im += w[r] * dots[r].y;
  }
  re_s[threadIdx.x] = re;
  im_s[threadIdx.x] = im;
  __syncthreads();
  for (int off = kRedThreads / 2; off > 0; off >>= 1) {
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

// acc[0] += scale * sum over the batch's pairs of w_a w_j sum_kyb partial, one CTA, fixed order
__global__ void __launch_bounds__(kRedThreads) k_dmu_batch(const double* partial, int P2, int TA,
                                                           int TJ, const double* w_tgt,
                                                           const double* w_occ, double scale,
                                                           double* acc) {
  __shared__ double s_s[kRedThreads];
  double s = 0.0;
  for (int p = threadIdx.x; p < TA * TJ; p += kRedThreads) {
    double t = 0.0;
    for (int r = 0; r < P2; ++r) t += partial[(long long)p * P2 + r];
    s += w_tgt[p / TJ] * (w_occ ? w_occ[p % TJ] : 1.0) * t;
  }
  s_s[threadIdx.x] = s;
  __syncthreads();
  for (int off = kRedThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) s_s[threadIdx.x] += s_s[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) acc[0] += scale * s_s[0];
}

// acc[c] += scale * sum over the batch's pairs of w_a w_j sum_kyb partial[.][c], c < 7
__global__ void __launch_bounds__(kRedThreads) k_strain_batch(const double* partial, int P2, int TA,
                                                              int TJ, const double* w_tgt,
                                                              const double* w_occ, double scale,
                                                              double* acc) {
  __shared__ double s_s[7][kRedThreads];
  double s[7] = {0, 0, 0, 0, 0, 0, 0};
  for (int p = threadIdx.x; p < TA * TJ; p += kRedThreads) {
    const double w = w_tgt[p / TJ] * (w_occ ? w_occ[p % TJ] : 1.0);
    for (int r = 0; r < P2; ++r)
      for (int c = 0; c < 7; ++c) s[c] += w * partial[((long long)p * P2 + r) * 7 + c];
  }
  for (int c = 0; c < 7; ++c) s_s[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int off = kRedThreads / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
      for (int c = 0; c < 7; ++c) s_s[c][threadIdx.x] += s_s[c][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x < 7) acc[threadIdx.x] += scale * s_s[threadIdx.x][0];
}

// out[3a+b] = -delta_ab E_x + (s Omega / N_k^2) acc[comp(a,b)], E_x = -(s/2)(Omega/N_k^2) acc[0]
__global__ void k_strain_final(const double* acc, double omega, int nk, double* out, double* ex) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double f = omega / ((double)nk * (double)nk);
  const double e = -0.5 * kSpin * f * acc[0];
  const int comp[9] = {1, 6, 5, 6, 2, 4, 5, 4, 3};
  for (int i = 0; i < 9; ++i) out[i] = (i % 4 == 0 ? -e : 0.0) + kSpin * f * acc[comp[i]];
  if (ex) ex[0] = e;
}

__global__ void k_scale_scalar(const double* in, double factor, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) out[0] = factor * in[0];
}

// dc[row][g] = factor * w[row] * vx[row][g]
__global__ void k_scale_rows(const double2* vx, const double* w, long long nrows, int npw_max,
                             double factor, double2* dc) {
  const long long total = nrows * npw_max;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const double f = factor * w[i / npw_max];
    const double2 v = vx[i];
    dc[i] = make_double2(f * v.x, f * v.y);
  }
}

// Real orbitals at Gamma: occupied slot p packs bands 2p and 2p+1 as
//   cp[p] = s_2p c[2p] - i s_2p+1 c[2p+1]   (the second term absent past n_occ)
// with s = sqrt(w) when fold (negative w sets the error flag and counts as 0),
// else s = 1 and wp[p] = (w_2p, w_2p+1).
__global__ void k_pack_real(const double2* c, const double* w, int n_occ, int npw_max, bool fold,
                            double2* cp, double2* wp, int* err) {
  const int n_slot = (n_occ + 1) / 2;
  const long long total = (long long)n_slot * npw_max;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int slot = (int)(i / npw_max), g = (int)(i % npw_max);
    const int b1 = 2 * slot, b2 = b1 + 1;
    const bool has2 = b2 < n_occ;
    const double w1 = w[b1], w2 = has2 ? w[b2] : 0.0;
    double s1 = 1.0, s2 = has2 ? 1.0 : 0.0;
    if (fold) {
      if (w1 < 0.0 || w2 < 0.0) atomicOr(err, 2);
      s1 = w1 > 0.0 ? sqrt(w1) : 0.0;
      s2 = w2 > 0.0 ? sqrt(w2) : 0.0;
    }
    const double2 x = c[(long long)b1 * npw_max + g];
    const double2 y = has2 ? c[(long long)b2 * npw_max + g] : make_double2(0.0, 0.0);
    // s1 x - i s2 y
    cp[i] = make_double2(s1 * x.x + s2 * y.y, s1 * x.y - s2 * y.x);
    if (g == 0 && wp) wp[slot] = make_double2(w1, w2);
  }
}

// Real part of V_x u: acc[a].y = 0 for every target a, and, when packed slot
// accumulators are given, acc[b].x += slot[b/2].x (b even) or -slot[b/2].y (b odd)
// for b < n_occ (the contributions that the k = q pair symmetry routes to band b).
__global__ void k_real_combine(double2* acc, int n_tgt, const double2* slot, int n_occ, long long n3) {
  const long long total = (long long)n_tgt * n3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / n3);
    const long long r = i % n3;
    double x = acc[i].x;
    if (slot && b < n_occ) {
      const double2 v = slot[(long long)(b / 2) * n3 + r];
      x += (b % 2 == 0) ? v.x : -v.y;
    }
    acc[i] = make_double2(x, 0.0);
  }
}

}  // namespace xx

using namespace xx;

// ------------------------------------------------------------------ plan --

namespace {

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct xx_plan_s {
  int device = 0;
  int N = 0;              // x and y length of the FFT grid (after the axis permutation)
  int NZ = 0;             // z length
  int perm[3] = {0, 1, 2};   // plan axis i is the caller's axis perm[i]
  int grid[3] = {0, 0, 0};
  int nk = 0;
  int npw_max = 0;
  double lattice[9];
  double B[9];            // reciprocal rows
  double M[9];            // reciprocal metric
  double omega = 0.0;
  std::vector<double> kfrac;
  std::vector<int> npw;
  int nmax[3] = {0, 0, 0};
  int h[3] = {0, 0, 0};   // pruned half-widths 2 n_max
  int kernel = 0;
  double mu = 0.0;
  int prec = 0;
  size_t cap = 0;
  int ta_user = 0, tj_user = 0;
  bool pair_symmetry = true;
  int tma_pass_b = 1;          // XX_OPT_TMA_PASS_B: 0 off, 1 for z length >= 80 with <= 3/4 of a row kept, 2 always
  int stage_pass_a = 1;        // XX_OPT_STAGE_PASS_A: 0 off, 1 for N <= 48, 2 always
  bool test_wait_expiry = false;   // XX_OPT_TEST_WAIT_EXPIRY
  bool fused_vjp = true;           // XX_OPT_FUSED_VJP
  // XX_OPT_ACC_LIMIT_MB: MiB of FP64 accumulators held for every k-point at once
  // (the k != q pair symmetry of xx_apply, the fused VJP); 64 GiB by default
  long long acc_limit_mb = 64 << 10;
  int sm_count = 0;
  int tma_per_sm = -1;         // resident tensor-copy pass B CTAs per SM (-1: not queried)
  bool real_gamma = false;     // XX_OPT_REAL_GAMMA
  bool gamma_closed = false;   // one k-point at Gamma whose basis holds -G for every G
  int ta_last = 0, tj_last = 0, g_last = 1;
  // xx_set_shard: this plan computes the contributions of the (k, q) blocks that
  // the block assignment gives to shard `shard` of `n_shards` (1: every block)
  int shard = 0, n_shards = 1;
  // Layout of the shared orbital grids (occupied = leading target bands): the
  // occupied bands of every k-point first ([nk][split]), then the remaining
  // targets ([nk][n_tgt - split]), so the occupied grids of consecutive
  // k-points are contiguous; split = 0: plain [k][n_tgt]
  int split = 0, split_nk = 0, split_ntgt = 0;
  const KernelTable* kt = nullptr;   // = &kx
  KernelTable kx;                    // plane kernels of length N, pencil kernels of length NZ
  int* d_miller = nullptr;   // [nk][npw_max][3]
  int* d_npw = nullptr;      // [nk]
  void* d_tw32 = nullptr;
  void* d_tw64 = nullptr;
  void* d_twz32 = nullptr;   // z twiddles (length NZ)
  void* d_twz64 = nullptr;
  int* d_err = nullptr;
  DevBuf u_tgt, u_occ, inter, acc, vt, dvt, box, stage, dots, partial, dmu_acc, vx_tmp, u_bar,
      stab, cpack, wpair, acc2, cells_tab, vt_all, kf_dev;
  // Kernel tables of every (k, q), built once (they depend only on the plan's
  // cell, k-points and kernel) when they fit: vt_all_state 0 not built, 1 built
  // (event vt_all_ev marks the end of the build), 2 built and known complete,
  // -1 not used (too large).  vt_sel: the table segment the next band-pair batch
  // reads (nullptr: the per-batch buffer vt).
  int vt_all_state = 0;
  cudaEvent_t vt_all_ev = nullptr;
  const void* vt_sel = nullptr;
  size_t ws_bytes = 0, peak_bytes = 0;
  long long launches = 0;
  long long pairs = 0;          // band pairs (or packed slots) through pass A so far
  // optional per-kernel-class timing with events on the launch stream
  bool profiling = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Rec { int cls; int e0, e1; };
  std::vector<Rec> recs;
  size_t ev_next = 0;
  // own stream and join events for xx_run_many
  cudaStream_t own_stream = nullptr;
  cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
};

namespace {

const size_t kDefaultCap = (size_t)16 << 30;
const int kDefaultTA = 64, kDefaultTJ = 80;   // band-pair batch (targets x occupied)
// widest occupied batch when whole occupied sets of several q-points share one
// (measured on GB300, alpha-boron cell, 18 occupied bands: 8 q-points per batch
// 1.5 % faster than 4, 2 q-points 2.7 % slower)
const int kDefaultTJMulti = 160;

// NVTX range for timeline tools (nsys, ncu --nvtx); free when no tool is attached
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};
const int kGridChunk = 32;   // orbitals per sphere<->grid launch

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return XX_OK;
  if (e == cudaErrorMemoryAllocation) return XX_ERR_OUT_OF_MEMORY;
  if (e == cudaErrorNoDevice || e == cudaErrorInsufficientDriver) return XX_ERR_NO_DEVICE;
  return XX_ERR_CUDA;
}

int ensure(xx_plan p, DevBuf& b, size_t bytes) {
  if (b.bytes >= bytes) return XX_OK;
  if (b.p) {
    cudaFree(b.p);   // synchronises with prior work that may still use it
    p->ws_bytes -= b.bytes;
    b.p = nullptr;
    b.bytes = 0;
  }
  cudaError_t e = cudaMalloc(&b.p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    b.p = nullptr;
    return cuda_status(e);
  }
  b.bytes = bytes;
  p->ws_bytes += bytes;
  if (p->ws_bytes > p->peak_bytes) p->peak_bytes = p->ws_bytes;
  return XX_OK;
}

void release(DevBuf& b) {
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

// release a workspace buffer while the plan lives on (counted in ws_bytes)
void release_counted(xx_plan p, DevBuf& b) {
  p->ws_bytes -= b.bytes;
  release(b);
}

bool supported_n(int n) { return kernel_table(n) != nullptr; }

size_t elem_bytes(const xx_plan p) { return p->prec == XX_FP64 ? 16 : 8; }

long long n3(const xx_plan p) { return (long long)p->N * p->N * p->NZ; }

int P(const xx_plan p, int ax) { return 2 * p->h[ax] + 1; }
int Q(const xx_plan p, int ax) { return 2 * p->nmax[ax] + 1; }

// Row pitch of the pair intermediates: the P1 kept f_x, rounded up to an even
// count in FP32 so that every row is a whole number of 16-byte units (the
// tensor-copy rule of pass B).
int LX(const xx_plan p) { return p->prec == XX_FP64 ? P(p, 0) : (P(p, 0) + 1) & ~1; }

// bytes of one band pair's intermediate, [N][P2][LX]
size_t inter_pair_bytes(const xx_plan p) {
  return (size_t)p->NZ * P(p, 1) * LX(p) * (p->prec == XX_FP64 ? 16 : 8);
}

const KernelSet& kset(const xx_plan p) { return p->prec == XX_FP64 ? p->kt->f64 : p->kt->f32; }

int launched(xx_plan p, int count) {
  p->launches += count;
  return cuda_status(cudaGetLastError());
}

// Profiling brackets: record an event before and after the launches of one
// kernel class on stream s (no-ops unless profiling is enabled).
int prof_event(xx_plan p) {
  if (p->ev_next == p->ev_pool.size()) {
    cudaEvent_t e;
    if (cudaEventCreate(&e) != cudaSuccess) return -1;
    p->ev_pool.push_back(e);
  }
  return (int)p->ev_next++;
}

int prof_begin(xx_plan p, cudaStream_t s) {
  if (!p->profiling) return -1;
  const int e = prof_event(p);
  if (e >= 0) cudaEventRecord(p->ev_pool[e], s);
  return e;
}

void prof_end(xx_plan p, int cls, int e0, cudaStream_t s) {
  if (!p->profiling || e0 < 0) return;
  const int e1 = prof_event(p);
  if (e1 < 0) return;
  cudaEventRecord(p->ev_pool[e1], s);
  p->recs.push_back({cls, e0, e1});
}

// sphere -> grid for nb orbitals of k-point k: c[b][npw_max] -> u[b][N^3]
int sphere_to_grid(xx_plan p, int k, const double2* c, int nb, void* u, cudaStream_t s) {
  Range r("xx sphere->grid");
  const size_t eb = elem_bytes(p);
  const int Q1 = Q(p, 0), Q2 = Q(p, 1), Q3 = Q(p, 2);
  const int chunk = nb < kGridChunk ? nb : kGridChunk;
  int st = ensure(p, p->box, (size_t)chunk * Q1 * Q2 * Q3 * eb);
  if (st) return st;
  st = ensure(p, p->stage, (size_t)chunk * p->NZ * Q1 * Q2 * eb);
  if (st) return st;
  for (int b0 = 0; b0 < nb; b0 += chunk) {
    const int cb = (nb - b0) < chunk ? (nb - b0) : chunk;
    GridArgs g{};
    g.c = c + (long long)b0 * p->npw_max;
    g.miller = p->d_miller + (long long)k * p->npw_max * 3;
    g.npw = p->npw[k];
    g.npw_max = p->npw_max;
    g.nb = cb;
    g.box = p->box.p;
    g.stage = p->stage.p;
    g.u = (char*)u + (size_t)b0 * n3(p) * eb;
    g.tw = p->prec == XX_FP64 ? p->d_tw64 : p->d_tw32;
    g.twz = p->prec == XX_FP64 ? p->d_twz64 : p->d_twz32;
    g.nz = p->NZ;
    g.n1 = p->nmax[0];
    g.n2 = p->nmax[1];
    g.n3 = p->nmax[2];
    g.Q1 = Q1;
    g.Q2 = Q2;
    g.Q3 = Q3;
    g.scale = 1.0 / std::sqrt(p->omega);
    g.err = p->d_err;
    const int e = prof_begin(p, s);
    cudaMemsetAsync(p->box.p, 0, (size_t)cb * Q1 * Q2 * Q3 * eb, s);
    const int blocks = (int)(((long long)cb * g.npw + 255) / 256);
    if (p->prec == XX_FP64)
      k_s2g_scatter<double><<<blocks, 256, 0, s>>>(g);
    else
      k_s2g_scatter<float><<<blocks, 256, 0, s>>>(g);
    kset(p).s2g_z(g, s);
    kset(p).s2g_xy(g, s);
    prof_end(p, XX_PROF_SPHERE_TO_GRID, e, s);
    if ((st = launched(p, 3))) return st;
  }
  return XX_OK;
}

// grid -> sphere for nb FP64 grids f[b][N^3] of k-point k into out[b][npw_max]
int grid_to_sphere(xx_plan p, int k, const double2* f, int nb, double2* out, cudaStream_t s) {
  Range r("xx grid->sphere");
  const int Q1 = Q(p, 0), Q2 = Q(p, 1), Q3 = Q(p, 2);
  const int chunk = nb < kGridChunk ? nb : kGridChunk;
  int st = ensure(p, p->box, (size_t)chunk * Q1 * Q2 * Q3 * 16);
  if (st) return st;
  st = ensure(p, p->stage, (size_t)chunk * p->NZ * Q1 * Q2 * 16);
  if (st) return st;
  for (int b0 = 0; b0 < nb; b0 += chunk) {
    const int cb = (nb - b0) < chunk ? (nb - b0) : chunk;
    GridArgs g{};
    g.out = out + (long long)b0 * p->npw_max;
    g.miller = p->d_miller + (long long)k * p->npw_max * 3;
    g.npw = p->npw[k];
    g.npw_max = p->npw_max;
    g.nb = cb;
    g.box = p->box.p;
    g.stage = p->stage.p;
    g.f = f + (long long)b0 * n3(p);
    g.tw = p->d_tw64;
    g.twz = p->d_twz64;
    g.nz = p->NZ;
    g.n1 = p->nmax[0];
    g.n2 = p->nmax[1];
    g.n3 = p->nmax[2];
    g.Q1 = Q1;
    g.Q2 = Q2;
    g.Q3 = Q3;
    g.scale = std::sqrt(p->omega) / (double)n3(p);
    g.err = p->d_err;
    const int e = prof_begin(p, s);
    p->kt->g2s_xy(g, s);
    p->kt->g2s_z(g, s);
    const int blocks = (int)(((long long)cb * p->npw_max + 255) / 256);
    k_g2s_gather<<<blocks, 256, 0, s>>>(g);
    prof_end(p, XX_PROF_GRID_TO_SPHERE, e, s);
    if ((st = launched(p, 3))) return st;
  }
  return XX_OK;
}

// The kernel tables of every (k, q) in one launch, when nk^2 tables fit in
// min(1 GiB, workspace cap / 8) and nk^2 <= 65535 (the grid's y extent); the
// values are those of the per-(k, q) launches (same device function).  A later
// call on another stream waits for the build's event until it has completed.
int build_all_tables(xx_plan p, cudaStream_t s) {
  if (p->vt_all_state < 0) return XX_OK;
  if (p->vt_all_state == 2) return XX_OK;
  if (p->vt_all_state == 1) {
    const cudaError_t q = cudaEventQuery(p->vt_all_ev);
    if (q == cudaSuccess) {
      p->vt_all_state = 2;
      return XX_OK;
    }
    if (q != cudaErrorNotReady) return cuda_status(q);
    cudaError_t e = cudaStreamWaitEvent(s, p->vt_all_ev, 0);
    return e == cudaSuccess ? XX_OK : cuda_status(e);
  }
  const size_t eb = p->prec == XX_FP64 ? 8 : 4;
  const long long nbox = (long long)P(p, 0) * P(p, 1) * P(p, 2);
  const long long pairs = (long long)p->nk * p->nk;
  const size_t bytes = (size_t)pairs * (size_t)nbox * eb;
  const size_t limit = std::min((size_t)1 << 30, p->cap / 8);
  if (pairs > 65535 || bytes > limit) {
    p->vt_all_state = -1;
    return XX_OK;
  }
  int st = ensure(p, p->kf_dev, (size_t)3 * p->nk * sizeof(double));
  if (st) return st;
  if ((st = ensure(p, p->vt_all, bytes))) return st;
  cudaError_t e = cudaMemcpyAsync(p->kf_dev.p, p->kfrac.data(), (size_t)3 * p->nk * sizeof(double),
                                  cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) return cuda_status(e);
  if (!p->vt_all_ev && (e = cudaEventCreateWithFlags(&p->vt_all_ev, cudaEventDisableTiming)) != cudaSuccess)
    return cuda_status(e);
  VtabArgs a{};
  std::memcpy(a.M, p->M, sizeof(a.M));
  a.h1 = p->h[0];
  a.h2 = p->h[1];
  a.h3 = p->h[2];
  a.P1 = P(p, 0);
  a.P2 = P(p, 1);
  a.P3 = P(p, 2);
  a.kernel = p->kernel;
  a.mu = p->mu;
  a.inv_n = 1.0 / (double)n3(p);
  a.inv_n2 = a.inv_n * a.inv_n;
  const dim3 grid((unsigned)((nbox + 255) / 256), (unsigned)pairs);
  const int ev = prof_begin(p, s);
  if (p->prec == XX_FP64)
    k_vtab_all<double><<<grid, 256, 0, s>>>((double*)p->vt_all.p, (const double*)p->kf_dev.p, p->nk, a);
  else
    k_vtab_all<float><<<grid, 256, 0, s>>>((float*)p->vt_all.p, (const double*)p->kf_dev.p, p->nk, a);
  prof_end(p, XX_PROF_KERNEL_TABLE, ev, s);
  if ((st = launched(p, 1))) return st;
  if ((e = cudaEventRecord(p->vt_all_ev, s)) != cudaSuccess) return cuda_status(e);
  p->vt_all_state = 1;
  return XX_OK;
}

// v(k - q + G)/N (and dv/dmu/N^2) over the pruned box into table slot `slot` of
// `slots` (each P1 P2 P3 values); the buffers are sized for every slot first
int kernel_table_for(xx_plan p, int k, int q, bool with_dmu, cudaStream_t s, int slot = 0, int slots = 1) {
  const size_t eb = p->prec == XX_FP64 ? 8 : 4;
  const long long nbox = (long long)P(p, 0) * P(p, 1) * P(p, 2);
  p->vt_sel = nullptr;
  if (!with_dmu) {
    const int st = build_all_tables(p, s);
    if (st) return st;
    if (p->vt_all_state > 0) {
      // consecutive q of one segment are consecutive tables
      p->vt_sel = (const char*)p->vt_all.p + ((long long)k * p->nk + q - slot) * nbox * (long long)eb;
      return XX_OK;
    }
  }
  int st = ensure(p, p->vt, (size_t)slots * nbox * eb);
  if (st) return st;
  if (with_dmu && (st = ensure(p, p->dvt, (size_t)slots * nbox * eb))) return st;
  VtabArgs a{};
  std::memcpy(a.M, p->M, sizeof(a.M));
  for (int i = 0; i < 3; ++i) a.d[i] = p->kfrac[3 * k + i] - p->kfrac[3 * q + i];
  a.h1 = p->h[0];
  a.h2 = p->h[1];
  a.h3 = p->h[2];
  a.P1 = P(p, 0);
  a.P2 = P(p, 1);
  a.P3 = P(p, 2);
  a.kernel = p->kernel;
  a.mu = p->mu;
  a.inv_n = 1.0 / (double)n3(p);
  a.inv_n2 = a.inv_n * a.inv_n;
  const int blocks = (int)((nbox + 255) / 256);
  const int e = prof_begin(p, s);
  if (p->prec == XX_FP64)
    k_vtab<double><<<blocks, 256, 0, s>>>((double*)p->vt.p + slot * nbox,
                                          with_dmu ? (double*)p->dvt.p + slot * nbox : nullptr, a);
  else
    k_vtab<float><<<blocks, 256, 0, s>>>((float*)p->vt.p + slot * nbox,
                                         with_dmu ? (float*)p->dvt.p + slot * nbox : nullptr, a);
  prof_end(p, XX_PROF_KERNEL_TABLE, e, s);
  return launched(p, 1);
}

void batch_shape(xx_plan p, int n_tgt, int n_occ, int* TA, int* TJ) {
  const size_t per_pair = inter_pair_bytes(p);
  // 64 x 80 measured best on the 96^3 workload: a long occupied loop amortises
  // pass C's prologue and FP64 accumulator update, and 6144 CTAs per launch
  // keep the last wave short
  int ta = p->ta_user > 0 ? p->ta_user : kDefaultTA;
  int tj = p->tj_user > 0 ? p->tj_user : kDefaultTJ;
  if (ta > n_tgt) ta = n_tgt;
  if (tj > n_occ) tj = n_occ;
  while ((size_t)ta * tj * per_pair > p->cap && tj > 1) tj = (tj + 1) / 2;
  while ((size_t)ta * tj * per_pair > p->cap && ta > 1) ta = (ta + 1) / 2;
  *TA = ta < 1 ? 1 : ta;
  *TJ = tj < 1 ? 1 : tj;
}

PairArgs pair_args(xx_plan p, int TA, int TJ) {
  PairArgs a{};
  a.inter = p->inter.p;
  a.vt = p->vt_sel ? p->vt_sel : p->vt.p;
  a.dvt = p->dvt.p;
  a.partial = (double*)p->partial.p;
  a.tw = p->prec == XX_FP64 ? p->d_tw64 : p->d_tw32;
  a.twz = p->prec == XX_FP64 ? p->d_twz64 : p->d_twz32;
  a.nz = p->NZ;
  a.u_tgt_stride = n3(p);
  a.u_occ_stride = n3(p);
  a.TA = TA;
  a.TJ = TJ;
  a.h1 = p->h[0];
  a.h2 = p->h[1];
  a.h3 = p->h[2];
  a.P1 = P(p, 0);
  a.P2 = P(p, 1);
  a.P3 = P(p, 2);
  a.LX = LX(p);
  a.coef = -1.0 / (double)p->nk;
  a.err = p->d_err;
  a.test_wait_expiry = p->test_wait_expiry ? 1 : 0;
  a.nj = TJ;   // one q-point per occupied batch unless the caller sets segments
  // measured on GB300 against the unstaged pass A with its L1 prefetch of the next
  // occupied plane: the beta step on its 60^3 grid 3.5 % slower staged, the alpha step
  // (48^3) the same either way, the 96^3 pass A 13 % slower staged (one CTA of 768
  // threads per SM against two of 384)
  a.stage_a = p->prec == XX_FP32_MIXED && (p->stage_pass_a == 2 || (p->stage_pass_a == 1 && p->N <= 48)) ? 1 : 0;
  return a;
}

bool bad_ptr(const void* a) { return a == nullptr; }

// Index of band b of k-point k in a split layout of nk k-points: the first
// `split` bands of every k-point, then the other n_b - split (split = 0: plain).
long long split_index(int split, int nk, int n_b, int k, int b) {
  if (split <= 0) return (long long)k * n_b + b;
  if (b < split) return (long long)k * split + b;
  return (long long)nk * split + (long long)k * (n_b - split) + (b - split);
}

// Grids of targets (and occupied, unless shared) for every k.
// Targets of k-points k0..k0+kn-1 (c_tgt holds only those), occupied of every q.
// Shared grids use the split layout (occupied bands of every k-point first).
int build_grids(xx_plan p, int k0, int kn, const void* c_occ, int ld_occ, int n_occ,
                const void* c_tgt, int n_tgt, bool shared, cudaStream_t s) {
  const size_t eb = elem_bytes(p);
  int st = ensure(p, p->u_tgt, (size_t)kn * n_tgt * n3(p) * eb);
  if (st) return st;
  p->split = shared && n_occ < n_tgt ? n_occ : 0;
  p->split_nk = kn;
  p->split_ntgt = n_tgt;
  for (int kk = 0; kk < kn; ++kk) {
    const double2* ck = (const double2*)c_tgt + (long long)kk * n_tgt * p->npw_max;
    const int parts = p->split > 0 ? 2 : 1;
    for (int part = 0; part < parts; ++part) {
      const int b0 = part == 0 ? 0 : p->split;
      const int nb = parts == 1 ? n_tgt : (part == 0 ? p->split : n_tgt - p->split);
      const long long idx = split_index(p->split, kn, n_tgt, kk, b0);
      st = sphere_to_grid(p, k0 + kk, ck + (long long)b0 * p->npw_max, nb,
                          (char*)p->u_tgt.p + (size_t)idx * n3(p) * eb, s);
      if (st) return st;
    }
  }
  if (!shared) {
    if ((st = ensure(p, p->u_occ, (size_t)p->nk * n_occ * n3(p) * eb))) return st;
    for (int q = 0; q < p->nk; ++q) {
      st = sphere_to_grid(p, q, (const double2*)c_occ + (long long)q * ld_occ * p->npw_max, n_occ,
                          (char*)p->u_occ.p + (size_t)q * n_occ * n3(p) * eb, s);
      if (st) return st;
    }
  }
  return XX_OK;
}

// grid of band j of k-point q: shared = in the target grids (split layout),
// else in the separate occupied grids [nk][n_occ]
const char* grid_ptr(xx_plan p, bool shared, int q, int j, int n_occ, int n_tgt) {
  const size_t eb = elem_bytes(p);
  if (shared)
    return (const char*)p->u_tgt.p + (size_t)split_index(p->split, p->split_nk, n_tgt, q, j) * n3(p) * eb;
  return (const char*)p->u_occ.p + ((size_t)q * n_occ + j) * n3(p) * eb;
}

int run_apply_real(xx_plan p, const void* c_occ, int ld_occ, const double* w_occ, int n_occ,
                   const void* c_tgt, int n_tgt, void* vx_out, cudaStream_t s);

// Index of the unordered k-point block {k, q}, k <= q, in the upper triangle
// (row-major): 0 .. nk (nk + 1) / 2 - 1.
int block_index(int nk, int k, int q) {
  if (k > q) std::swap(k, q);
  return k * nk - k * (k - 1) / 2 + (q - k);
}

// Owner shard of every block {k, q}: longest-processing-time greedy on the
// band-pair transforms of a block (the k = q square counted once per pair; a
// k != q block's occupied square once, its targets past the occupied set
// against both k-points), blocks taken in decreasing cost, ties by index, each
// to the least-loaded shard (ties: lowest shard).  Deterministic.
void assign_blocks(int nk, int n_occ, int n_tgt, int n_shards, std::vector<int>& owner) {
  const int nb = nk * (nk + 1) / 2;
  owner.assign(nb, 0);
  if (n_shards <= 1) return;
  const long long rest = (long long)(n_tgt > n_occ ? n_tgt - n_occ : 0) * n_occ;
  std::vector<std::pair<long long, int>> order;
  for (int k = 0; k < nk; ++k)
    for (int q = k; q < nk; ++q) {
      const long long cost = k == q ? (long long)n_occ * (n_occ + 1) / 2 + rest
                                    : (long long)n_occ * n_occ + 2 * rest;
      order.push_back({cost, block_index(nk, k, q)});
    }
  std::stable_sort(order.begin(), order.end(), [](const std::pair<long long, int>& a,
                                                  const std::pair<long long, int>& b) {
    return a.first != b.first ? a.first > b.first : a.second < b.second;
  });
  std::vector<long long> load(n_shards, 0);
  for (const auto& b : order) {
    int best = 0;
    for (int r = 1; r < n_shards; ++r)
      if (load[r] < load[best]) best = r;
    owner[b.second] = best;
    load[best] += b.first;
  }
}

// The band-pair passes of one batch, each bracketed for per-class timing;
// pass A counts the batch's pairs.
void run_pass_a(xx_plan p, const PairArgs& a, cudaStream_t s) {
  const int e = prof_begin(p, s);
  kset(p).pass_a(a, s);
  prof_end(p, XX_PROF_PASS_A, e, s);
  p->pairs += (long long)a.TA * a.TJ;
}

// cuTensorMapEncodeTiled from the driver, resolved once (nullptr if unavailable)
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = [] {
    void* f = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &f, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      f = nullptr;
    }
    return reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(f);
  }();
  return fn;
}

// Pass B of one batch.  In FP32, when the kept f_x are at most 3/4 of a row (or
// when forced), it takes the tensor-copy staged kernel: the intermediates viewed
// as floats [N * pairs][P2][2 LX], one box of 2 LX x 1 x N (a row's N z-planes)
// per item; a row is 8 LX bytes (a multiple of 16, LX even).
void run_pass_b(xx_plan p, const PairArgs& a, cudaStream_t s) {
  const int e = prof_begin(p, s);
  bool done = false;
  // measured on GB300 (beta cell, 64 targets x 160 occupied x 8 q): P1 = 57 of N = 96,
  // tensor-copy kernel 6.7 % faster than the row kernel (243.9 vs 261.3 ms); P1 = 57
  // of N = 60, 14 % slower
  // measured on GB300 (cubic cells, 2x2x2 k-mesh, 32 x 32 bands; the beta cell): the
  // tensor-copy kernel gains 6-7 % of pass B at N = 80 and 96 with P1 = 57 and is
  // within 4 % either way at N = 96 otherwise, but loses 3-28 % at N <= 72
  const bool want = p->tma_pass_b == 2 || (p->tma_pass_b == 1 && p->NZ >= 80 && 4 * a.P1 <= 3 * p->N);
  PFN_cuTensorMapEncodeTiled_v12000 enc = p->prec == XX_FP32_MIXED && want ? tensor_map_encoder() : nullptr;
  if (enc && 2 * a.LX <= 256 && p->NZ <= 256) {
    if (p->tma_per_sm < 0) {
      p->tma_per_sm = p->kt->pass_b_tma_per_sm(a.LX, a.P1, a.P3);
      if (cudaDeviceGetAttribute(&p->sm_count, cudaDevAttrMultiProcessorCount, p->device) != cudaSuccess) {
        cudaGetLastError();
        p->tma_per_sm = 0;
      }
    }
    if (p->tma_per_sm > 0) {
      const cuuint64_t dims[3] = {(cuuint64_t)(2 * a.LX), (cuuint64_t)a.P2, (cuuint64_t)p->NZ * a.TA * a.TJ};
      const cuuint64_t strides[2] = {(cuuint64_t)a.LX * 8, (cuuint64_t)a.P2 * a.LX * 8};
      const cuuint32_t box[3] = {(cuuint32_t)(2 * a.LX), 1, (cuuint32_t)p->NZ};
      const cuuint32_t estr[3] = {1, 1, 1};
      CUtensorMap tm;
      if (enc(&tm, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, a.inter, dims, strides, box, estr,
              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
              CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS) {
        const long long items = (long long)a.P2 * a.TA * a.TJ;
        const long long slots = (long long)p->sm_count * p->tma_per_sm;
        p->kt->pass_b_tma(a, tm, (int)(items < slots ? items : slots), s);
        done = true;
      }
    }
  }
  if (!done) kset(p).pass_b(a, s);
  prof_end(p, XX_PROF_PASS_B, e, s);
}

void run_pass_c(xx_plan p, const PairArgs& a, cudaStream_t s) {
  const int e = prof_begin(p, s);
  kset(p).pass_c(a, s);
  prof_end(p, XX_PROF_PASS_C, e, s);
}

// role-swapped pass C (profiled with pass C)
void run_pass_ct(xx_plan p, const PairArgs& a, cudaStream_t s) {
  const int e = prof_begin(p, s);
  kset(p).pass_ct(a, s);
  prof_end(p, XX_PROF_PASS_C, e, s);
}

// One band-pair batch: targets a0.. (ta of them, grids u_tgt consecutive) of
// k-point k against an occupied batch of G segments, one per k-point q0, q0+1,
// .., of nj bands each (G > 1 only with whole occupied sets), whose grids
// (u_occ), occupations (w_occ) and role-swapped accumulators (acc_j) are
// consecutive across the segments; kernel tables of the G q-points in slots
// 0..G-1.  Pass C adds -(w_qj/N_k) u_qj W_aj into the accumulators acc_a of the
// targets; with acc_j set, the role-swapped pass C adds -(w_ka/N_k) u_ka
// conj(W_aj) into them (W_qj,ka = conj(W_ka,qj)).
struct SegBatch {
  const char* u_tgt = nullptr;
  int ta = 0;
  const char* u_occ = nullptr;
  int G = 1, nj = 0;
  const double* w_occ = nullptr;
  double2* acc_a = nullptr;
  double2* acc_j = nullptr;
  const double* w_tgt = nullptr;   // occupations of the targets (role-swapped pass C)
};

int seg_batch(xx_plan p, const SegBatch& b, cudaStream_t s) {
  PairArgs a = pair_args(p, b.ta, b.G * b.nj);
  a.u_tgt = b.u_tgt;
  a.u_occ = b.u_occ;
  a.nj = b.nj;
  a.vt_seg = (long long)P(p, 0) * P(p, 1) * P(p, 2);
  a.acc = b.acc_a;
  a.w_occ = b.w_occ;
  run_pass_a(p, a, s);
  run_pass_b(p, a, s);
  run_pass_c(p, a, s);
  int nl = 3;
  if (b.acc_j) {
    PairArgs c = a;
    c.w_tgt = b.w_tgt;
    c.w_occ = nullptr;
    c.acc = b.acc_j;
    run_pass_ct(p, c, s);
    ++nl;
  }
  return launched(p, nl);
}

// real: take the real-orbital Gamma path (plan option XX_OPT_REAL_GAMMA)
int run_apply(xx_plan p, int k0, int kn, const void* c_occ, int ld_occ, const double* w_occ,
              int n_occ, const void* c_tgt, int n_tgt, void* vx_out, bool real, cudaStream_t s) {
  if (real) {
    // one k-point: its single block {0, 0} belongs to shard 0
    if (p->n_shards > 1 && p->shard != 0)
      return cuda_status(cudaMemsetAsync(vx_out, 0, (size_t)kn * n_tgt * p->npw_max * 16, s));
    return run_apply_real(p, c_occ, ld_occ, w_occ, n_occ, c_tgt, n_tgt, vx_out, s);
  }
  const bool shared = (c_occ == c_tgt && ld_occ == n_tgt && k0 == 0 && kn == p->nk);
  int st = build_grids(p, k0, kn, c_occ, ld_occ, n_occ, c_tgt, n_tgt, shared, s);
  if (st) return st;
  int TA, TJ;
  batch_shape(p, n_tgt, n_occ, &TA, &TJ);
  // An occupied batch spans G_max consecutive q-points when a q-point's whole
  // occupied set fits the batch width at least twice (few bands, many k-points):
  // fewer, wider launches.
  const int tj_cap = p->tj_user > 0 ? p->tj_user : kDefaultTJMulti;
  int G_max = 1;
  if (n_occ > 0 && 2 * n_occ <= tj_cap) {
    G_max = tj_cap / n_occ < p->nk ? tj_cap / n_occ : p->nk;
    while (G_max > 1 && (size_t)TA * G_max * n_occ * inter_pair_bytes(p) > p->cap) --G_max;
  }
  p->ta_last = TA;
  p->tj_last = TJ;
  p->g_last = G_max;
  const long long nn = n3(p);
  const int TJb = G_max > 1 ? G_max * n_occ : TJ;   // occupied columns of the widest batch
  if ((st = ensure(p, p->inter, (size_t)TA * TJb * inter_pair_bytes(p)))) return st;
  // Pair symmetry: with the occupied grids shared with the leading targets,
  // W_qj,ka = conj(W_ka,qj) (v(q - k + G) = v(k - q - G)).  On k = q blocks the
  // occupied square is tiled and only tiles I <= J are transformed; across
  // k-points (cross) only blocks q > k are, which needs the accumulators of
  // every k-point at once (in the split layout of the grids).
  const bool sym = shared && p->pair_symmetry && n_occ > 1;
  const size_t acc_k_bytes = (size_t)n_tgt * nn * 16;
  bool cross = sym && p->nk > 1 && (size_t)p->nk * acc_k_bytes <= ((size_t)p->acc_limit_mb << 20);
  if (cross) {
    st = ensure(p, p->acc, (size_t)p->nk * acc_k_bytes);
    if (st == XX_ERR_OUT_OF_MEMORY)
      cross = false;
    else if (st)
      return st;
  }
  if (!cross && (st = ensure(p, p->acc, acc_k_bytes))) return st;
  if (cross) cudaMemsetAsync(p->acc.p, 0, (size_t)p->nk * acc_k_bytes, s);
  const int split = cross ? p->split : 0;
  // accumulator of band b of k-point k (targets of one k when not cross)
  auto acc_ptr = [&](int k, int b) -> double2* {
    if (!cross) return (double2*)p->acc.p + (long long)b * nn;
    return (double2*)p->acc.p + split_index(split, p->nk, n_tgt, k, b) * nn;
  };
  const int T = TJ < TA ? TJ : TA;
  // sharded plan: only the blocks {k, q} this shard owns
  std::vector<int> owner;
  assign_blocks(p->nk, n_occ, n_tgt, p->n_shards, owner);
  auto owned = [&](int k, int q) { return owner[block_index(p->nk, k, q)] == p->shard; };
  for (int kk = 0; kk < kn; ++kk) {
    const int k = k0 + kk;
    char name[40];
    std::snprintf(name, sizeof(name), "xx target k-point %d", k);
    Range r(name);
    if (!cross) cudaMemsetAsync(p->acc.p, 0, acc_k_bytes, s);
    // targets [a_lo, a_hi) of k (cut at n_occ, where the split layout jumps)
    // against the occupied sets of the q-points [q_lo, q_hi), in segments of up
    // to G_max q-points; mirrored: the role-swapped pass C too (blocks q > k)
    auto run_q = [&](int q_lo, int q_hi, int a_lo, int a_hi, bool mirrored) -> int {
      if (a_lo >= a_hi) return XX_OK;
      for (int q0 = q_lo; q0 < q_hi;) {
        const int G = (q_hi - q0) < G_max ? (q_hi - q0) : G_max;
        for (int g = 0; g < G; ++g) {
          const int e = kernel_table_for(p, k, q0 + g, false, s, g, G);
          if (e) return e;
        }
        const int cut = a_lo < n_occ && n_occ < a_hi ? n_occ : a_hi;
        for (int part = 0; part < 2; ++part) {
          const int lo = part == 0 ? a_lo : cut, hi = part == 0 ? cut : a_hi;
          for (int a0 = lo; a0 < hi; a0 += TA) {
            const int ta = (hi - a0) < TA ? (hi - a0) : TA;
            const int jstep = G > 1 ? n_occ : TJ;
            for (int j0 = 0; j0 < n_occ; j0 += jstep) {
              SegBatch b;
              b.u_tgt = grid_ptr(p, true, kk, a0, n_occ, n_tgt);
              b.ta = ta;
              b.u_occ = grid_ptr(p, shared, q0, j0, n_occ, n_tgt);
              b.G = G;
              b.nj = (n_occ - j0) < jstep ? (n_occ - j0) : jstep;
              b.w_occ = w_occ + (long long)q0 * n_occ + j0;
              b.acc_a = acc_ptr(k, a0);
              if (mirrored) {
                b.acc_j = acc_ptr(q0, j0);
                b.w_tgt = w_occ + (long long)k * n_occ + a0;
              }
              const int e = seg_batch(p, b, s);
              if (e) return e;
            }
          }
        }
        q0 += G;
      }
      return XX_OK;
    };
    // run_q over the maximal runs of q in [q_lo, q_hi) whose block {k, q} this shard owns
    auto run_owned = [&](int q_lo, int q_hi, int a_lo, int a_hi, bool mirrored) -> int {
      for (int q = q_lo; q < q_hi;) {
        if (!owned(k, q)) {
          ++q;
          continue;
        }
        int q_end = q + 1;
        while (q_end < q_hi && owned(k, q_end)) ++q_end;
        const int e = run_q(q, q_end, a_lo, a_hi, mirrored);
        if (e) return e;
        q = q_end;
      }
      return XX_OK;
    };
    if (!sym) {
      if ((st = run_owned(0, p->nk, 0, n_tgt, false))) return st;
    } else if (owned(k, k)) {
      // k = q: tiles I <= J of the occupied square (tiles J > I receive
      // -(w_a/N_k) u_a conj(W_aj) through the role-swapped pass C), then the
      // targets past the occupied set
      if ((st = kernel_table_for(p, k, k, false, s))) return st;
      for (int i0 = 0; i0 < n_occ; i0 += T) {
        const int ti = (n_occ - i0) < T ? (n_occ - i0) : T;
        for (int j0 = i0; j0 < n_occ; j0 += T) {
          SegBatch b;
          b.u_tgt = grid_ptr(p, true, k, i0, n_occ, n_tgt);
          b.ta = ti;
          b.u_occ = grid_ptr(p, true, k, j0, n_occ, n_tgt);
          b.nj = (n_occ - j0) < T ? (n_occ - j0) : T;
          b.w_occ = w_occ + (long long)k * n_occ + j0;
          b.acc_a = acc_ptr(k, i0);
          if (j0 > i0) {
            b.acc_j = acc_ptr(k, j0);
            b.w_tgt = w_occ + (long long)k * n_occ + i0;
          }
          if ((st = seg_batch(p, b, s))) return st;
        }
      }
      if ((st = run_q(k, k + 1, n_occ, n_tgt, false))) return st;
    }
    if (sym) {
      if (cross) {
        // blocks q < k: their occupied squares ran with block (q, k)
        if ((st = run_owned(0, k, n_occ, n_tgt, false))) return st;
        if ((st = run_owned(k + 1, p->nk, 0, n_occ, true))) return st;
        if ((st = run_owned(k + 1, p->nk, n_occ, n_tgt, false))) return st;
      } else {
        if ((st = run_owned(0, k, 0, n_tgt, false))) return st;
        if ((st = run_owned(k + 1, p->nk, 0, n_tgt, false))) return st;
      }
    }
    // every contribution to the targets of k is in (blocks (k', k) with k' < k
    // ran in earlier iterations); the split layout keeps them in two runs
    double2* out = (double2*)vx_out + (long long)kk * n_tgt * p->npw_max;
    if (split > 0) {
      if ((st = grid_to_sphere(p, k, acc_ptr(k, 0), split, out, s))) return st;
      st = grid_to_sphere(p, k, acc_ptr(k, split), n_tgt - split, out + (long long)split * p->npw_max, s);
    } else {
      st = grid_to_sphere(p, k, acc_ptr(k, 0), n_tgt, out, s);
    }
    if (st) return st;
  }
  return XX_OK;
}

// ---------------------------------------------- real orbitals at Gamma --
// Every codensity conj(u_j) u_a is real and v(G) = v(-G) is real, so every W_aj
// is real: occupied bands 2p and 2p+1 share one transform as the slot
// u_2p - i u_2p+1 (codensity rho_a,2p + i rho_a,2p+1, potential W_a,2p + i W_a,2p+1).

// Packed occupied grids of the n_occ occupied bands (k = 0) into p->u_occ, slot
// weights into p->wpair; fold puts sqrt(w) into the slots instead.
int build_packed(xx_plan p, const void* c_occ, const double* w_occ, int n_occ, bool fold,
                 cudaStream_t s) {
  const int n_slot = (n_occ + 1) / 2;
  int st = ensure(p, p->cpack, (size_t)n_slot * p->npw_max * 16);
  if (st) return st;
  if ((st = ensure(p, p->wpair, (size_t)n_slot * 16))) return st;
  if ((st = ensure(p, p->u_occ, (size_t)n_slot * n3(p) * elem_bytes(p)))) return st;
  const long long total = (long long)n_slot * p->npw_max;
  const long long want = (total + 255) / 256;
  k_pack_real<<<(int)(want < 4096 ? want : 4096), 256, 0, s>>>(
      (const double2*)c_occ, w_occ, n_occ, p->npw_max, fold, (double2*)p->cpack.p,
      (double2*)p->wpair.p, p->d_err);
  if ((st = launched(p, 1))) return st;
  return sphere_to_grid(p, 0, (const double2*)p->cpack.p, n_slot, p->u_occ.p, s);
}

// Band tile of the pair-symmetric real path: even, at most TA targets and TJ slots.
int real_tile(int TA, int TJ) {
  int t = TA < 2 * TJ ? TA : 2 * TJ;
  t &= ~1;
  return t < 2 ? 2 : t;
}

// Visits the (target range, slot range) batches of the real path:
// f(a0, ta, s0, ns, mirrored).  With sym, the occupied bands (the leading
// targets) are cut into band tiles of T and only tile pairs J >= I are visited,
// mirrored = J > I (the pair (J, I) is implied by symmetry); targets past
// n_occ then meet every slot.  Without sym, every target batch meets every slot
// batch.
template <typename F>
int for_real_tiles(int n_tgt, int n_occ, int TA, int TJ, bool sym, int T, F&& f) {
  const int n_slot = (n_occ + 1) / 2;
  int st;
  int a_first = 0;
  if (sym) {
    for (int i0 = 0; i0 < n_occ; i0 += T) {
      const int ti = (n_occ - i0) < T ? (n_occ - i0) : T;
      for (int j0 = i0; j0 < n_occ; j0 += T) {
        const int tj = (n_occ - j0) < T ? (n_occ - j0) : T;
        if ((st = f(i0, ti, j0 / 2, (tj + 1) / 2, j0 > i0))) return st;
      }
    }
    a_first = n_occ;
  }
  for (int a0 = a_first; a0 < n_tgt; a0 += TA) {
    const int ta = (n_tgt - a0) < TA ? (n_tgt - a0) : TA;
    for (int s0 = 0; s0 < n_slot; s0 += TJ) {
      const int ns = (n_slot - s0) < TJ ? (n_slot - s0) : TJ;
      if ((st = f(a0, ta, s0, ns, false))) return st;
    }
  }
  return XX_OK;
}

int run_apply_real(xx_plan p, const void* c_occ, int ld_occ, const double* w_occ, int n_occ,
                   const void* c_tgt, int n_tgt, void* vx_out, cudaStream_t s) {
  const bool shared = (c_occ == c_tgt && ld_occ == n_tgt);
  const size_t eb = elem_bytes(p);
  const long long nn = n3(p);
  int st = ensure(p, p->u_tgt, (size_t)n_tgt * nn * eb);
  if (st) return st;
  if ((st = sphere_to_grid(p, 0, (const double2*)c_tgt, n_tgt, p->u_tgt.p, s))) return st;
  if ((st = build_packed(p, c_occ, w_occ, n_occ, false, s))) return st;
  const int n_slot = (n_occ + 1) / 2;
  int TA, TJ;
  batch_shape(p, n_tgt, n_slot, &TA, &TJ);
  p->ta_last = TA;
  p->tj_last = TJ;
  const bool sym = shared && p->pair_symmetry && n_occ > 1;
  const int T = real_tile(TA, TJ);
  long long npair = (long long)TA * TJ;
  if (sym && (long long)T * (T / 2) > npair) npair = (long long)T * (T / 2);
  if ((st = ensure(p, p->inter, (size_t)npair * inter_pair_bytes(p)))) return st;
  if ((st = ensure(p, p->acc, (size_t)n_tgt * nn * 16))) return st;
  cudaMemsetAsync(p->acc.p, 0, (size_t)n_tgt * nn * 16, s);
  if (sym) {
    if ((st = ensure(p, p->acc2, (size_t)n_slot * nn * 16))) return st;
    cudaMemsetAsync(p->acc2.p, 0, (size_t)n_slot * nn * 16, s);
  }
  if ((st = kernel_table_for(p, 0, 0, false, s))) return st;
  const KernelSet& ks = kset(p);
  st = for_real_tiles(n_tgt, n_occ, TA, TJ, sym, T, [&](int a0, int ta, int s0, int ns, bool mirrored) {
    PairArgs a = pair_args(p, ta, ns);
    a.u_tgt = (const char*)p->u_tgt.p + (size_t)a0 * nn * eb;
    a.u_occ = (const char*)p->u_occ.p + (size_t)s0 * nn * eb;
    a.acc = (double2*)p->acc.p + (long long)a0 * nn;
    a.w_pair = (const double2*)p->wpair.p + s0;
    run_pass_a(p, a, s);
    run_pass_b(p, a, s);
    int e = prof_begin(p, s);
    ks.pass_c_packed(a, s);
    prof_end(p, XX_PROF_PASS_C, e, s);
    if (!mirrored) return launched(p, 3);
    // the slots of tile J receive -(w_a/N_k) u_a conj(W_a,slot) from the targets of
    // tile I: real part for band 2p, minus the imaginary part for band 2p+1
    PairArgs c = a;
    c.w_tgt = w_occ + a0;
    c.w_occ = nullptr;
    c.acc = (double2*)p->acc2.p + (long long)s0 * nn;
    run_pass_ct(p, c, s);
    return launched(p, 4);
  });
  if (st) return st;
  const long long want = ((long long)n_tgt * nn + 255) / 256;
  k_real_combine<<<(int)(want < 4096 ? want : 4096), 256, 0, s>>>(
      (double2*)p->acc.p, n_tgt, sym ? (const double2*)p->acc2.p : nullptr, n_occ, nn);
  if ((st = launched(p, 1))) return st;
  return grid_to_sphere(p, 0, (const double2*)p->acc.p, n_tgt, (double2*)vx_out, s);
}

// Band-pair sums of the real path for dE/dmu (nsum = 1) and the strain
// derivative (nsum = 7): sqrt(w) is folded into the slots, so a (target, slot)
// pair carries w_2p S_a,2p + w_2p+1 S_a,2p+1 (the cross term sums to zero over
// +-G for real codensities and an even table); reduced with w_a.
int run_pair_sums_real(xx_plan p, const void* c, const double* w, int n_b, bool strain,
                       cudaStream_t s) {
  const size_t eb = elem_bytes(p);
  const long long nn = n3(p);
  int st = ensure(p, p->u_tgt, (size_t)n_b * nn * eb);
  if (st) return st;
  if ((st = sphere_to_grid(p, 0, (const double2*)c, n_b, p->u_tgt.p, s))) return st;
  if ((st = build_packed(p, c, w, n_b, true, s))) return st;
  const int n_slot = (n_b + 1) / 2;
  int TA, TJ;
  batch_shape(p, n_b, n_slot, &TA, &TJ);
  const bool sym = p->pair_symmetry && n_b > 1;
  const int T = real_tile(TA, TJ);
  long long npair = (long long)TA * TJ;
  if (sym && (long long)T * (T / 2) > npair) npair = (long long)T * (T / 2);
  const int nsum = strain ? 7 : 1;
  if ((st = ensure(p, p->inter, (size_t)npair * inter_pair_bytes(p)))) return st;
  if ((st = ensure(p, p->partial, (size_t)npair * P(p, 1) * nsum * 8))) return st;
  const KernelSet& ks = kset(p);
  return for_real_tiles(n_b, n_b, TA, TJ, sym, T, [&](int a0, int ta, int s0, int ns, bool mirrored) {
    PairArgs a = pair_args(p, ta, ns);
    a.u_tgt = (const char*)p->u_tgt.p + (size_t)a0 * nn * eb;
    a.u_occ = (const char*)p->u_occ.p + (size_t)s0 * nn * eb;
    const double scale = mirrored ? 2.0 : 1.0;
    run_pass_a(p, a, s);
    if (strain) {
      a.dvt = p->stab.p;
      ks.pass_b_strain(a, s);
      k_strain_batch<<<1, kRedThreads, 0, s>>>((const double*)p->partial.p, P(p, 1), ta, ns, w + a0,
                                               nullptr, scale, (double*)p->dmu_acc.p);
    } else {
      ks.pass_b_dmu(a, s);
      k_dmu_batch<<<1, kRedThreads, 0, s>>>((const double*)p->partial.p, P(p, 1), ta, ns, w + a0,
                                            nullptr, scale, (double*)p->dmu_acc.p);
    }
    return launched(p, 3);
  });
}

int run_energy_reduce(xx_plan p, int k0, int kn, const void* c_tgt, const double* w_tgt, int n_tgt,
                      const void* vx, double* ex_out, cudaStream_t s) {
  Range r("xx E_x reduction");
  const int rows = kn * n_tgt;
  int st = ensure(p, p->dots, (size_t)rows * 16);
  if (st) return st;
  const int e = prof_begin(p, s);
  k_dot_rows<<<rows, kRedThreads, 0, s>>>((const double2*)c_tgt, (const double2*)vx, p->d_npw + k0,
                                           n_tgt, p->npw_max, (double2*)p->dots.p);
  k_energy<<<1, kRedThreads, 0, s>>>((const double2*)p->dots.p, w_tgt, rows, 0.5 * kSpin / p->nk, ex_out);
  prof_end(p, XX_PROF_REDUCE, e, s);
  return launched(p, 2);
}

// dE/dmu accumulation: codensities recomputed (pass A) + forward z with dv/dmu (pass B')
int run_dmu(xx_plan p, const void* c, const double* w, int n_b, double grad, double* dmu_out,
            cudaStream_t s) {
  Range r("xx dE/dmu");
  const double factor = -0.5 * kSpin * p->omega / ((double)p->nk * (double)p->nk) * grad;
  int st;
  if (p->real_gamma) {
    if ((st = ensure(p, p->dmu_acc, 8))) return st;
    cudaMemsetAsync(p->dmu_acc.p, 0, 8, s);
    if ((st = kernel_table_for(p, 0, 0, true, s))) return st;
    if ((st = run_pair_sums_real(p, c, w, n_b, false, s))) return st;
    k_scale_scalar<<<1, 32, 0, s>>>((const double*)p->dmu_acc.p, factor, dmu_out);
    return launched(p, 1);
  }
  st = build_grids(p, 0, p->nk, c, n_b, n_b, c, n_b, true, s);
  if (st) return st;
  int TA, TJ;
  batch_shape(p, n_b, n_b, &TA, &TJ);
  const size_t eb = elem_bytes(p);
  if ((st = ensure(p, p->inter, (size_t)TA * TJ * inter_pair_bytes(p)))) return st;
  if ((st = ensure(p, p->partial, (size_t)TA * TJ * P(p, 1) * 8))) return st;
  if ((st = ensure(p, p->dmu_acc, 8))) return st;
  cudaMemsetAsync(p->dmu_acc.p, 0, 8, s);
  const KernelSet& ks = kset(p);
  // pair symmetry (option XX_OPT_PAIR_SYMMETRY): the pair sum of (qj, ka) equals
  // that of (ka, qj) (|rhohat_qj,ka(G)| = |rhohat_ka,qj(-G)|, v'(q - k + G) =
  // v'(k - q - G)), so blocks q < k are skipped and blocks q > k count twice; on
  // k = q blocks tiles I < J count twice and tiles J < I are skipped
  const int T = TJ < TA ? TJ : TA;
  for (int k = 0; k < p->nk; ++k)
    for (int q = 0; q < p->nk; ++q) {
      if (p->pair_symmetry && q < k) continue;
      if ((st = kernel_table_for(p, k, q, true, s))) return st;
      const bool diag = p->pair_symmetry && q == k && n_b > 1;
      const double block_scale = (p->pair_symmetry && q > k) ? 2.0 : 1.0;
      const int SA = diag ? T : TA, SJ = diag ? T : TJ;
      for (int a0 = 0; a0 < n_b; a0 += SA) {
        const int ta = (n_b - a0) < SA ? (n_b - a0) : SA;
        for (int j0 = diag ? a0 : 0; j0 < n_b; j0 += SJ) {
          const int tj = (n_b - j0) < SJ ? (n_b - j0) : SJ;
          const double scale = (diag && j0 > a0) ? 2.0 : block_scale;
          PairArgs a = pair_args(p, ta, tj);
          a.u_tgt = grid_ptr(p, true, k, a0, n_b, n_b);
          a.u_occ = grid_ptr(p, true, q, j0, n_b, n_b);
          run_pass_a(p, a, s);
          int e = prof_begin(p, s);
          ks.pass_b_dmu(a, s);
          prof_end(p, XX_PROF_PASS_B_DMU, e, s);
          k_dmu_batch<<<1, kRedThreads, 0, s>>>((const double*)p->partial.p, P(p, 1), ta, tj,
                                                w + (long long)k * n_b + a0,
                                                w + (long long)q * n_b + j0, scale,
                                                (double*)p->dmu_acc.p);
          if ((st = launched(p, 3))) return st;
        }
      }
    }
  k_scale_scalar<<<1, 32, 0, s>>>((const double*)p->dmu_acc.p, factor, dmu_out);
  return launched(p, 1);
}

// Strain derivative of E_x[c] at fixed coefficients: pass A + forward z with the
// seven tables of k_strain_tab, reduced with w_a w_j (pair symmetry on k = q).
// the seven strain tables of k - q into p->stab
int strain_tables(xx_plan p, int k, int q, cudaStream_t s) {
  const long long nbox = (long long)P(p, 0) * P(p, 1) * P(p, 2);
  int st = ensure(p, p->stab, (size_t)7 * nbox * (p->prec == XX_FP64 ? 8 : 4));
  if (st) return st;
  VtabArgs va{};
  std::memcpy(va.Bm, p->B, sizeof(va.Bm));
  std::memcpy(va.M, p->M, sizeof(va.M));
  for (int i = 0; i < 3; ++i) va.d[i] = p->kfrac[3 * k + i] - p->kfrac[3 * q + i];
  va.h1 = p->h[0];
  va.h2 = p->h[1];
  va.h3 = p->h[2];
  va.P1 = P(p, 0);
  va.P2 = P(p, 1);
  va.P3 = P(p, 2);
  va.kernel = p->kernel;
  va.mu = p->mu;
  va.inv_n = 1.0 / (double)n3(p);
  va.inv_n2 = va.inv_n * va.inv_n;
  const int blocks = (int)((nbox + 255) / 256);
  if (p->prec == XX_FP64)
    k_strain_tab<double><<<blocks, 256, 0, s>>>((double*)p->stab.p, va);
  else
    k_strain_tab<float><<<blocks, 256, 0, s>>>((float*)p->stab.p, va);
  return launched(p, 1);
}

int run_strain(xx_plan p, const void* c, const double* w, int n_b, double* out9, double* ex_out,
               cudaStream_t s) {
  Range r("xx strain derivative");
  int st = ensure(p, p->dmu_acc, 7 * 8);
  if (st) return st;
  cudaMemsetAsync(p->dmu_acc.p, 0, 7 * 8, s);
  if (p->real_gamma) {
    if ((st = strain_tables(p, 0, 0, s))) return st;
    if ((st = run_pair_sums_real(p, c, w, n_b, true, s))) return st;
    k_strain_final<<<1, 32, 0, s>>>((const double*)p->dmu_acc.p, p->omega, p->nk, out9, ex_out);
    return launched(p, 1);
  }
  st = build_grids(p, 0, p->nk, c, n_b, n_b, c, n_b, true, s);
  if (st) return st;
  int TA, TJ;
  batch_shape(p, n_b, n_b, &TA, &TJ);
  const size_t eb = elem_bytes(p);
  if ((st = ensure(p, p->inter, (size_t)TA * TJ * inter_pair_bytes(p)))) return st;
  if ((st = ensure(p, p->partial, (size_t)TA * TJ * P(p, 1) * 7 * 8))) return st;
  const KernelSet& ks = kset(p);
  const int T = TJ < TA ? TJ : TA;
  // pair symmetry as in the dE/dmu sums (g_a g_b is even in g)
  for (int k = 0; k < p->nk; ++k)
    for (int q = 0; q < p->nk; ++q) {
      if (p->pair_symmetry && q < k) continue;
      if ((st = strain_tables(p, k, q, s))) return st;
      const bool diag = p->pair_symmetry && q == k && n_b > 1;
      const double block_scale = (p->pair_symmetry && q > k) ? 2.0 : 1.0;
      const int SA = diag ? T : TA, SJ = diag ? T : TJ;
      for (int a0 = 0; a0 < n_b; a0 += SA) {
        const int ta = (n_b - a0) < SA ? (n_b - a0) : SA;
        for (int j0 = diag ? a0 : 0; j0 < n_b; j0 += SJ) {
          const int tj = (n_b - j0) < SJ ? (n_b - j0) : SJ;
          const double scale = (diag && j0 > a0) ? 2.0 : block_scale;
          PairArgs a = pair_args(p, ta, tj);
          a.u_tgt = grid_ptr(p, true, k, a0, n_b, n_b);
          a.u_occ = grid_ptr(p, true, q, j0, n_b, n_b);
          a.dvt = p->stab.p;
          run_pass_a(p, a, s);
          ks.pass_b_strain(a, s);
          k_strain_batch<<<1, kRedThreads, 0, s>>>((const double*)p->partial.p, P(p, 1), ta, tj,
                                                   w + (long long)k * n_b + a0,
                                                   w + (long long)q * n_b + j0, scale,
                                                   (double*)p->dmu_acc.p);
          if ((st = launched(p, 3))) return st;
        }
      }
    }
  k_strain_final<<<1, 32, 0, s>>>((const double*)p->dmu_acc.p, p->omega, p->nk, out9, ex_out);
  return launched(p, 1);
}

// Occupied-orbital part of the vector-Jacobian product of y = V_x[c_occ] c_tgt
// for a cotangent ybar = dL/dy* (Wirtinger):
//   dL/dc_qj* = P_q[ -(w_qj/N_k) sum_{k,a} ( ubar_ka conj(W_aj) + u_ka conj(Wbar_aj) ) ]
// with W_aj = K(conj(u_qj) u_ka), Wbar_aj = K(conj(u_qj) ubar_ka), ubar the
// grids of ybar and P_q the grid->sphere projection of q.
int run_vjp_occ(xx_plan p, const void* c_occ, int ld_occ, const double* w_occ, int n_occ,
                const void* c_tgt, int n_tgt, const void* ybar, void* grad_occ, cudaStream_t s) {
  const bool shared = (c_occ == c_tgt && ld_occ == n_tgt);
  int st = build_grids(p, 0, p->nk, c_occ, ld_occ, n_occ, c_tgt, n_tgt, shared, s);
  if (st) return st;
  const size_t eb = elem_bytes(p);
  if ((st = ensure(p, p->u_bar, (size_t)p->nk * n_tgt * n3(p) * eb))) return st;
  for (int k = 0; k < p->nk; ++k) {
    st = sphere_to_grid(p, k, (const double2*)ybar + (long long)k * n_tgt * p->npw_max, n_tgt,
                        (char*)p->u_bar.p + (size_t)k * n_tgt * n3(p) * eb, s);
    if (st) return st;
  }
  int TA, TJ;
  batch_shape(p, n_tgt, n_occ, &TA, &TJ);
  if ((st = ensure(p, p->inter, (size_t)TA * TJ * inter_pair_bytes(p)))) return st;
  if ((st = ensure(p, p->acc, (size_t)n_occ * n3(p) * 16))) return st;
  const KernelSet& ks = kset(p);
  for (int q = 0; q < p->nk; ++q) {
    cudaMemsetAsync(p->acc.p, 0, (size_t)n_occ * n3(p) * 16, s);
    for (int k = 0; k < p->nk; ++k) {
      if ((st = kernel_table_for(p, k, q, false, s))) return st;
      // target batches never cross the split of the shared grids' layout
      for (int a0 = 0, ta = 0; a0 < n_tgt; a0 += ta) {
        const int a_end = p->split > 0 && a0 < p->split ? p->split : n_tgt;
        ta = (a_end - a0) < TA ? (a_end - a0) : TA;
        for (int j0 = 0; j0 < n_occ; j0 += TJ) {
          const int tj = (n_occ - j0) < TJ ? (n_occ - j0) : TJ;
          const char* ut = grid_ptr(p, true, k, a0, n_occ, n_tgt);
          const char* ub = (const char*)p->u_bar.p + ((size_t)k * n_tgt + a0) * n3(p) * eb;
          PairArgs a = pair_args(p, ta, tj);
          a.u_occ = grid_ptr(p, shared, q, j0, n_occ, n_tgt);
          a.acc = (double2*)p->acc.p + (long long)j0 * n3(p);
          a.w_occ = w_occ + (long long)q * n_occ + j0;
          // term 1: W_aj from (u_a, u_j), multiplied by ubar_a
          a.u_tgt = ut;
          run_pass_a(p, a, s);
          run_pass_b(p, a, s);
          a.u_tgt = ub;
          ks.pass_ct(a, s);
          // term 2: Wbar_aj from (ubar_a, u_j), multiplied by u_a
          run_pass_a(p, a, s);
          run_pass_b(p, a, s);
          a.u_tgt = ut;
          ks.pass_ct(a, s);
          if ((st = launched(p, 6))) return st;
        }
      }
    }
    st = grid_to_sphere(p, q, (const double2*)p->acc.p, n_occ,
                        (double2*)grad_occ + (long long)q * n_occ * p->npw_max, s);
    if (st) return st;
  }
  return XX_OK;
}

// Both parts of the vector-Jacobian product from two transforms per band pair:
// Wbar_aj = K(conj(u_qj) ubar_ka) feeds dL/dc_tgt* = V_x ybar (pass C into the
// accumulators of the targets of k) and the u_ka conj(Wbar_aj) term of
// dL/dc_qj* (role-swapped pass C); W_aj = K(conj(u_qj) u_ka) feeds the
// ubar_ka conj(W_aj) term.  The occupied accumulators of every q are held at
// once (nk * n_occ * N^3 * 16 bytes).  Returns XX_ERR_OUT_OF_MEMORY (nothing
// launched beyond the grids) when they do not fit, so the caller can run the
// two parts separately.
int run_vjp_fused(xx_plan p, const void* c_occ, int ld_occ, const double* w_occ, int n_occ,
                  const void* c_tgt, int n_tgt, const void* ybar, void* grad_tgt, void* grad_occ,
                  cudaStream_t s) {
  const long long nn = n3(p);
  const size_t occ_bytes = (size_t)p->nk * n_occ * nn * 16;
  if (occ_bytes > ((size_t)p->acc_limit_mb << 20)) return XX_ERR_OUT_OF_MEMORY;
  const bool shared = (c_occ == c_tgt && ld_occ == n_tgt);
  int st = build_grids(p, 0, p->nk, c_occ, ld_occ, n_occ, c_tgt, n_tgt, shared, s);
  if (st) return st;
  const size_t eb = elem_bytes(p);
  if ((st = ensure(p, p->u_bar, (size_t)p->nk * n_tgt * nn * eb))) return st;
  for (int k = 0; k < p->nk; ++k) {
    st = sphere_to_grid(p, k, (const double2*)ybar + (long long)k * n_tgt * p->npw_max, n_tgt,
                        (char*)p->u_bar.p + (size_t)k * n_tgt * nn * eb, s);
    if (st) return st;
  }
  int TA, TJ;
  batch_shape(p, n_tgt, n_occ, &TA, &TJ);
  if ((st = ensure(p, p->inter, (size_t)TA * TJ * inter_pair_bytes(p)))) return st;
  if ((st = ensure(p, p->acc2, occ_bytes))) return st;
  if ((st = ensure(p, p->acc, (size_t)n_tgt * nn * 16))) return st;
  cudaMemsetAsync(p->acc2.p, 0, occ_bytes, s);
  for (int k = 0; k < p->nk; ++k) {
    cudaMemsetAsync(p->acc.p, 0, (size_t)n_tgt * nn * 16, s);
    for (int q = 0; q < p->nk; ++q) {
      if ((st = kernel_table_for(p, k, q, false, s))) return st;
      double2* acc_q = (double2*)p->acc2.p + (long long)q * n_occ * nn;
      // target batches never cross the split of the shared grids' layout
      for (int a0 = 0, ta = 0; a0 < n_tgt; a0 += ta) {
        const int a_end = p->split > 0 && a0 < p->split ? p->split : n_tgt;
        ta = (a_end - a0) < TA ? (a_end - a0) : TA;
        for (int j0 = 0; j0 < n_occ; j0 += TJ) {
          const int tj = (n_occ - j0) < TJ ? (n_occ - j0) : TJ;
          const char* ut = grid_ptr(p, true, k, a0, n_occ, n_tgt);
          const char* ub = (const char*)p->u_bar.p + ((size_t)k * n_tgt + a0) * nn * eb;
          PairArgs a = pair_args(p, ta, tj);
          a.u_occ = grid_ptr(p, shared, q, j0, n_occ, n_tgt);
          a.w_occ = w_occ + (long long)q * n_occ + j0;
          // Wbar: V_x ybar for the targets of k, and u_a conj(Wbar) for j
          a.u_tgt = ub;
          run_pass_a(p, a, s);
          run_pass_b(p, a, s);
          a.acc = (double2*)p->acc.p + (long long)a0 * nn;
          run_pass_c(p, a, s);
          a.u_tgt = ut;
          a.acc = acc_q + (long long)j0 * nn;
          run_pass_ct(p, a, s);
          // W: ubar_a conj(W) for j
          run_pass_a(p, a, s);
          run_pass_b(p, a, s);
          a.u_tgt = ub;
          run_pass_ct(p, a, s);
          if ((st = launched(p, 7))) return st;
        }
      }
    }
    st = grid_to_sphere(p, k, (const double2*)p->acc.p, n_tgt,
                        (double2*)grad_tgt + (long long)k * n_tgt * p->npw_max, s);
    if (st) return st;
  }
  for (int q = 0; q < p->nk; ++q) {
    st = grid_to_sphere(p, q, (const double2*)p->acc2.p + (long long)q * n_occ * nn, n_occ,
                        (double2*)grad_occ + (long long)q * n_occ * p->npw_max, s);
    if (st) return st;
  }
  return XX_OK;
}

// Two equal axis lengths, each length built in; perm puts the equal pair first
// (plan axes x, y), the third length on z.  Three different lengths are raised to
// two equal ones in xx_create before this is asked.
bool supported_grid(const int* g, int perm[3]) {
  if (!supported_n(g[0]) || !supported_n(g[1]) || !supported_n(g[2])) return false;
  if (g[0] == g[1]) {
    perm[0] = 0, perm[1] = 1, perm[2] = 2;
  } else if (g[0] == g[2]) {
    perm[0] = 0, perm[1] = 2, perm[2] = 1;
  } else if (g[1] == g[2]) {
    perm[0] = 1, perm[1] = 2, perm[2] = 0;
  } else {
    return false;
  }
  return true;
}

}  // namespace

// ------------------------------------------------------------------ C ABI --

extern "C" {

const char* xx_status_string(int status) {
  switch (status) {
    case XX_OK: return "ok";
    case XX_ERR_INVALID_ARGUMENT: return "invalid argument";
    case XX_ERR_UNSUPPORTED_GRID: return "unsupported FFT grid (axis lengths 24, 32, 36, 40, 48, 54, 60, 64, 72, 80, 96 or 108; a z-pencil row within shared memory)";
    case XX_ERR_GRID_ALIASING: return "FFT grid too small: an axis has N < 4 n_max + 1 (codensity wrap-around)";
    case XX_ERR_OUT_OF_MEMORY: return "out of device memory";
    case XX_ERR_CUDA: return "CUDA error";
    case XX_ERR_DEVICE_FLAG: return "device-side check failed (inconsistent basis data or a negative occupation)";
    case XX_ERR_TIMEOUT: return "timed out waiting for the stream";
    case XX_ERR_NO_DEVICE: return "no usable CUDA device";
    case XX_ERR_SIZE_LIMIT: return "size exceeds the fixed scratch of the no-allocation entry point (XX_NOALLOC_MAX_ROWS)";
    default: return "unknown status";
  }
}

int xx_create(xx_plan* out, const double* lattice, const int* grid, int nk, const double* kfrac,
              const int* npw, int npw_max, const int* miller, int kernel_type, double mu,
              int precision, size_t workspace_cap) {
  if (!out) return XX_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (!lattice || !grid || !kfrac || !npw || !miller || nk < 1 || npw_max < 1)
    return XX_ERR_INVALID_ARGUMENT;
  if (kernel_type != XX_KERNEL_HSE && kernel_type != XX_KERNEL_COULOMB_G0_DROPPED)
    return XX_ERR_INVALID_ARGUMENT;
  if (kernel_type == XX_KERNEL_HSE && !(mu > 0.0 && std::isfinite(mu))) return XX_ERR_INVALID_ARGUMENT;
  if (precision != XX_FP32_MIXED && precision != XX_FP64) return XX_ERR_INVALID_ARGUMENT;
  for (int i = 0; i < 9; ++i)
    if (!std::isfinite(lattice[i])) return XX_ERR_INVALID_ARGUMENT;
  for (int i = 0; i < 3 * nk; ++i)
    if (!std::isfinite(kfrac[i])) return XX_ERR_INVALID_ARGUMENT;
  for (int k = 0; k < nk; ++k)
    if (npw[k] < 1 || npw[k] > npw_max) return XX_ERR_INVALID_ARGUMENT;
  for (int ax = 0; ax < 3; ++ax)
    if (!supported_n(grid[ax])) return XX_ERR_UNSUPPORTED_GRID;
  // largest |Miller index| per axis of the caller's basis; the caller's grid must be
  // free of wrap-around on every axis
  int nmax[3] = {0, 0, 0};
  for (int k = 0; k < nk; ++k)
    for (int g = 0; g < npw[k]; ++g)
      for (int ax = 0; ax < 3; ++ax) {
        const int m = miller[((long long)k * npw_max + g) * 3 + ax];
        const int am = m < 0 ? -m : m;
        if (am > 4096) return XX_ERR_INVALID_ARGUMENT;
        if (am > nmax[ax]) nmax[ax] = am;
      }
  for (int ax = 0; ax < 3; ++ax)
    if (grid[ax] < 4 * nmax[ax] + 1) return XX_ERR_GRID_ALIASING;
  // Three different lengths: compute on the grid that raises the shorter of two axes
  // to the longer, the pair giving the fewest points.  The caller's grid is free of
  // wrap-around (checked above), so the raised one is too, and both give the same
  // V_x c, E_x and derivatives up to rounding.
  int raised[3] = {grid[0], grid[1], grid[2]};
  if (grid[0] != grid[1] && grid[0] != grid[2] && grid[1] != grid[2]) {
    const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
    long long best = -1;
    for (const auto& pr : pairs) {
      int g[3] = {grid[0], grid[1], grid[2]};
      g[pr[0]] = g[pr[1]] = std::max(grid[pr[0]], grid[pr[1]]);
      const long long pts = (long long)g[0] * g[1] * g[2];
      if (best < 0 || pts < best) {
        best = pts;
        std::copy(g, g + 3, raised);
      }
    }
  }
  grid = raised;
  int perm[3];
  if (!supported_grid(grid, perm)) return XX_ERR_UNSUPPORTED_GRID;
  // Relabel the axes so that the two equal grid lengths are x and y: lattice
  // rows, fractional k components and Miller components follow the grid.  The
  // operator does not depend on the labelling; V_x c keeps the caller's basis
  // order, and E_x and the Cartesian strain derivative are unchanged.
  double lat[9];
  int gridp[3], nmaxp[3];
  for (int i = 0; i < 3; ++i) {
    gridp[i] = grid[perm[i]];
    nmaxp[i] = nmax[perm[i]];
    for (int c = 0; c < 3; ++c) lat[3 * i + c] = lattice[3 * perm[i] + c];
  }
  std::vector<double> kfp(3 * (size_t)nk);
  for (int k = 0; k < nk; ++k)
    for (int i = 0; i < 3; ++i) kfp[3 * k + i] = kfrac[3 * k + perm[i]];
  std::vector<int> milp(3 * (size_t)nk * npw_max);
  for (size_t g = 0; g < (size_t)nk * npw_max; ++g)
    for (int i = 0; i < 3; ++i) milp[3 * g + i] = miller[3 * g + perm[i]];
  kfrac = kfp.data();
  miller = milp.data();
  grid = gridp;
  lattice = lat;
  std::copy(nmaxp, nmaxp + 3, nmax);

  // cell volume and reciprocal metric (b_i = 2 pi inverse-transpose rows)
  const double* a = lattice;
  const double c23[3] = {a[4] * a[8] - a[5] * a[7], a[5] * a[6] - a[3] * a[8], a[3] * a[7] - a[4] * a[6]};
  const double c31[3] = {a[7] * a[2] - a[8] * a[1], a[8] * a[0] - a[6] * a[2], a[6] * a[1] - a[7] * a[0]};
  const double c12[3] = {a[1] * a[5] - a[2] * a[4], a[2] * a[3] - a[0] * a[5], a[0] * a[4] - a[1] * a[3]};
  const double vol = a[0] * c23[0] + a[1] * c23[1] + a[2] * c23[2];
  if (!(std::fabs(vol) > 1e-12)) return XX_ERR_INVALID_ARGUMENT;

  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev < 1) {
    cudaGetLastError();
    return XX_ERR_NO_DEVICE;
  }
  {
    // the z pencils of pass B hold a row of z-planes (grid[2] x P1) and its kept
    // frequencies (P3 x P1) in shared memory; the plane kernels fit by construction
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
      cudaGetLastError();
      return XX_ERR_NO_DEVICE;
    }
    const long long P1 = 4 * nmax[0] + 1, P3 = 4 * nmax[2] + 1;
    const long long pencil = (grid[2] + grid[2] * P1 + P3 * P1) * (precision == XX_FP64 ? 16 : 8);
    if (pencil > optin) return XX_ERR_UNSUPPORTED_GRID;
  }

  xx_plan p = new (std::nothrow) xx_plan_s();
  if (!p) return XX_ERR_OUT_OF_MEMORY;
  cudaGetDevice(&p->device);
  p->N = grid[0];
  p->NZ = grid[2];
  for (int i = 0; i < 3; ++i) {
    p->grid[i] = grid[i];
    p->perm[i] = perm[i];
  }
  p->nk = nk;
  p->npw_max = npw_max;
  std::memcpy(p->lattice, lattice, sizeof(p->lattice));
  p->omega = std::fabs(vol);
  double B[9];
  const double tp = 2.0 * 3.14159265358979323846 / vol;
  for (int i = 0; i < 3; ++i) {
    B[0 + i] = tp * c23[i];
    B[3 + i] = tp * c31[i];
    B[6 + i] = tp * c12[i];
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      p->M[3 * i + j] = B[3 * i] * B[3 * j] + B[3 * i + 1] * B[3 * j + 1] + B[3 * i + 2] * B[3 * j + 2];
  std::memcpy(p->B, B, sizeof(p->B));
  p->kfrac.assign(kfrac, kfrac + 3 * nk);
  p->npw.assign(npw, npw + nk);
  for (int ax = 0; ax < 3; ++ax) {
    p->nmax[ax] = nmax[ax];
    p->h[ax] = 2 * nmax[ax];
  }
  // real orbitals need a single k-point at Gamma whose basis is closed under G -> -G
  if (nk == 1 && kfrac[0] == 0.0 && kfrac[1] == 0.0 && kfrac[2] == 0.0) {
    std::vector<long long> keys(npw[0]);
    auto key = [](long long a, long long b, long long c) { return ((a + 8192) * 16384 + (b + 8192)) * 16384 + (c + 8192); };
    for (int g = 0; g < npw[0]; ++g)
      keys[g] = key(miller[3 * g], miller[3 * g + 1], miller[3 * g + 2]);
    std::sort(keys.begin(), keys.end());
    bool closed = std::adjacent_find(keys.begin(), keys.end()) == keys.end();
    for (int g = 0; g < npw[0] && closed; ++g)
      closed = std::binary_search(keys.begin(), keys.end(),
                                  key(-miller[3 * g], -miller[3 * g + 1], -miller[3 * g + 2]));
    p->gamma_closed = closed;
  }
  p->kernel = kernel_type;
  p->mu = mu;
  p->prec = precision;
  p->cap = workspace_cap ? workspace_cap : kDefaultCap;
  // plane kernels (x, y) of length N, pencil kernels (z) of length NZ
  p->kx = *kernel_table(p->N);
  const KernelTable* tz = kernel_table(p->NZ);
  for (KernelSet* ks : {&p->kx.f32, &p->kx.f64}) {
    const KernelSet& zs = ks == &p->kx.f32 ? tz->f32 : tz->f64;
    ks->pass_b = zs.pass_b;
    ks->pass_b_dmu = zs.pass_b_dmu;
    ks->pass_b_strain = zs.pass_b_strain;
    ks->s2g_z = zs.s2g_z;
  }
  p->kx.pass_b_tma = tz->pass_b_tma;
  p->kx.pass_b_tma_per_sm = tz->pass_b_tma_per_sm;
  p->kx.g2s_z = tz->g2s_z;
  p->kt = &p->kx;

  // twiddles exp(-2 pi i e / L) for L = N and NZ, evaluated in long double on the host
  auto twiddles = [](int L, std::vector<double2>& t64, std::vector<float2>& t32) {
    t64.resize(L);
    t32.resize(L);
    for (int e = 0; e < L; ++e) {
      const long double ang = -2.0L * 3.141592653589793238462643383279502884L * e / L;
      t64[e] = make_double2((double)cosl(ang), (double)sinl(ang));
      t32[e] = make_float2((float)t64[e].x, (float)t64[e].y);
    }
  };
  std::vector<double2> t64, tz64;
  std::vector<float2> t32, tz32;
  twiddles(p->N, t64, t32);
  twiddles(p->NZ, tz64, tz32);
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = cudaMalloc(&p->d_miller, sizeof(int) * 3 * (size_t)nk * npw_max);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_npw, sizeof(int) * nk);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_tw64, sizeof(double2) * p->N);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_tw32, sizeof(float2) * p->N);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_twz64, sizeof(double2) * p->NZ);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_twz32, sizeof(float2) * p->NZ);
  if (e == cudaSuccess) e = cudaMalloc(&p->d_err, sizeof(int));
  if (e == cudaSuccess)
    e = cudaMemcpy(p->d_miller, miller, sizeof(int) * 3 * (size_t)nk * npw_max, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_npw, npw, sizeof(int) * nk, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_tw64, t64.data(), sizeof(double2) * p->N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_tw32, t32.data(), sizeof(float2) * p->N, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_twz64, tz64.data(), sizeof(double2) * p->NZ, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(p->d_twz32, tz32.data(), sizeof(float2) * p->NZ, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(p->d_err, 0, sizeof(int));
  if (e != cudaSuccess) {
    cudaGetLastError();
    xx_destroy(p);
    return cuda_status(e);
  }
  *out = p;
  return XX_OK;
}

int xx_destroy(xx_plan p) {
  if (!p) return XX_OK;
  cudaDeviceSynchronize();
  DevBuf* bufs[] = {&p->u_tgt, &p->u_occ, &p->inter, &p->acc, &p->vt, &p->dvt, &p->box,
                    &p->stage, &p->dots, &p->partial, &p->dmu_acc, &p->vx_tmp, &p->u_bar,
                    &p->stab, &p->cpack, &p->wpair, &p->acc2, &p->cells_tab, &p->vt_all, &p->kf_dev};
  for (DevBuf* b : bufs) release(*b);
  if (p->vt_all_ev) cudaEventDestroy(p->vt_all_ev);
  if (p->d_miller) cudaFree(p->d_miller);
  if (p->d_npw) cudaFree(p->d_npw);
  if (p->d_tw32) cudaFree(p->d_tw32);
  if (p->d_tw64) cudaFree(p->d_tw64);
  if (p->d_twz32) cudaFree(p->d_twz32);
  if (p->d_twz64) cudaFree(p->d_twz64);
  if (p->d_err) cudaFree(p->d_err);
  for (cudaEvent_t e : p->ev_pool) cudaEventDestroy(e);
  if (p->ev_fork) cudaEventDestroy(p->ev_fork);
  if (p->ev_join) cudaEventDestroy(p->ev_join);
  if (p->own_stream) cudaStreamDestroy(p->own_stream);
  delete p;
  return XX_OK;
}

}  // extern "C"

namespace {

int apply_range(xx_plan p, int k_first, int k_count, const void* c_occ, int ld_occ,
                const double* w_occ, int n_occ, const void* c_tgt, int n_tgt, void* vx_out,
                bool real, void* stream) {
  Range r("xx apply");
  if (!p || n_occ < 0 || n_tgt < 0 || k_first < 0 || k_count < 0 || k_first + k_count > p->nk)
    return XX_ERR_INVALID_ARGUMENT;
  if (ld_occ == 0) ld_occ = n_occ;
  if (ld_occ < n_occ) return XX_ERR_INVALID_ARGUMENT;
  if (n_tgt == 0 || k_count == 0) return XX_OK;
  if (bad_ptr(c_tgt) || bad_ptr(vx_out) || vx_out == c_tgt || vx_out == c_occ) return XX_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_occ == 0) {
    const cudaError_t e = cudaMemsetAsync(vx_out, 0, (size_t)k_count * n_tgt * p->npw_max * 16, s);
    return cuda_status(e);
  }
  if (bad_ptr(c_occ) || bad_ptr(w_occ)) return XX_ERR_INVALID_ARGUMENT;
  return run_apply(p, k_first, k_count, c_occ, ld_occ, w_occ, n_occ, c_tgt, n_tgt, vx_out, real, s);
}

}  // namespace

extern "C" {

int xx_apply_range(xx_plan p, int k_first, int k_count, const void* c_occ, int ld_occ,
                   const double* w_occ, int n_occ, const void* c_tgt, int n_tgt, void* vx_out,
                   void* stream) {
  if (!p) return XX_ERR_INVALID_ARGUMENT;
  return apply_range(p, k_first, k_count, c_occ, ld_occ, w_occ, n_occ, c_tgt, n_tgt, vx_out,
                     p->real_gamma, stream);
}

int xx_apply(xx_plan p, const void* c_occ, int ld_occ, const double* w_occ, int n_occ,
             const void* c_tgt, int n_tgt, void* vx_out, void* stream) {
  if (!p) return XX_ERR_INVALID_ARGUMENT;
  return xx_apply_range(p, 0, p->nk, c_occ, ld_occ, w_occ, n_occ, c_tgt, n_tgt, vx_out, stream);
}

int xx_energy_from_vx_range(xx_plan p, int k_first, int k_count, const void* c_tgt,
                            const double* w_tgt, int n_tgt, const void* vx, double* ex_out,
                            void* stream) {
  if (!p || n_tgt < 0 || bad_ptr(ex_out) || k_first < 0 || k_count < 0 || k_first + k_count > p->nk)
    return XX_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_tgt == 0 || k_count == 0) return cuda_status(cudaMemsetAsync(ex_out, 0, 2 * sizeof(double), s));
  if (bad_ptr(c_tgt) || bad_ptr(w_tgt) || bad_ptr(vx)) return XX_ERR_INVALID_ARGUMENT;
  return run_energy_reduce(p, k_first, k_count, c_tgt, w_tgt, n_tgt, vx, ex_out, s);
}

int xx_energy_from_vx(xx_plan p, const void* c_tgt, const double* w_tgt, int n_tgt, const void* vx,
                      double* ex_out, void* stream) {
  if (!p) return XX_ERR_INVALID_ARGUMENT;
  return xx_energy_from_vx_range(p, 0, p->nk, c_tgt, w_tgt, n_tgt, vx, ex_out, stream);
}

int xx_energy_range(xx_plan p, int k_first, int k_count, const void* c_occ, int ld_occ,
                    const double* w_occ, int n_occ, const void* c_tgt, const double* w_tgt,
                    int n_tgt, void* vx_out, double* ex_out, void* stream) {
  if (!p || bad_ptr(ex_out)) return XX_ERR_INVALID_ARGUMENT;
  if (n_tgt > 0 && k_count > 0 && bad_ptr(vx_out)) return XX_ERR_INVALID_ARGUMENT;
  int st = xx_apply_range(p, k_first, k_count, c_occ, ld_occ, w_occ, n_occ, c_tgt, n_tgt, vx_out,
                          stream);
  if (st) return st;
  return xx_energy_from_vx_range(p, k_first, k_count, c_tgt, w_tgt, n_tgt, vx_out, ex_out, stream);
}

int xx_energy(xx_plan p, const void* c_occ, int ld_occ, const double* w_occ, int n_occ,
              const void* c_tgt, const double* w_tgt, int n_tgt, void* vx_out, double* ex_out,
              void* stream) {
  if (!p) return XX_ERR_INVALID_ARGUMENT;
  return xx_energy_range(p, 0, p->nk, c_occ, ld_occ, w_occ, n_occ, c_tgt, w_tgt, n_tgt, vx_out,
                         ex_out, stream);
}

int xx_apply_backward(xx_plan p, const void* c, const double* w, int n_b, const void* vx,
                      double grad_ex, void* dc_out, double* dmu_out, void* stream) {
  if (!p || n_b < 0 || !std::isfinite(grad_ex)) return XX_ERR_INVALID_ARGUMENT;
  if (dmu_out && p->kernel != XX_KERNEL_HSE) return XX_ERR_INVALID_ARGUMENT;
  if (dmu_out && p->n_shards > 1) return XX_ERR_INVALID_ARGUMENT;   // dE/dmu is not sharded
  cudaStream_t s = (cudaStream_t)stream;
  if (n_b == 0) {
    if (dmu_out) return cuda_status(cudaMemsetAsync(dmu_out, 0, sizeof(double), s));
    return XX_OK;
  }
  if (bad_ptr(c) || bad_ptr(w)) return XX_ERR_INVALID_ARGUMENT;
  int st;
  if (dc_out) {
    if (dc_out == c) return XX_ERR_INVALID_ARGUMENT;
    const void* v = vx;
    if (!v) {
      if ((st = ensure(p, p->vx_tmp, (size_t)p->nk * n_b * p->npw_max * 16))) return st;
      if ((st = run_apply(p, 0, p->nk, c, n_b, w, n_b, c, n_b, p->vx_tmp.p, p->real_gamma, s)))
        return st;
      v = p->vx_tmp.p;
    }
    const long long rows = (long long)p->nk * n_b;
    const int blocks = (int)((rows * p->npw_max + 255) / 256);
    k_scale_rows<<<blocks < 65535 ? blocks : 65535, 256, 0, s>>>(
        (const double2*)v, w, rows, p->npw_max, grad_ex * kSpin / p->nk, (double2*)dc_out);
    if ((st = launched(p, 1))) return st;
  }
  if (dmu_out) return run_dmu(p, c, w, n_b, grad_ex, dmu_out, s);
  return XX_OK;
}

int xx_strain_derivative(xx_plan p, const void* c, const double* w, int n_b, double* dex_deps,
                         double* ex_out, void* stream) {
  if (!p || n_b < 0 || bad_ptr(dex_deps) || p->n_shards > 1) return XX_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_b == 0) {
    cudaError_t e = cudaMemsetAsync(dex_deps, 0, 9 * sizeof(double), s);
    if (e == cudaSuccess && ex_out) e = cudaMemsetAsync(ex_out, 0, sizeof(double), s);
    return cuda_status(e);
  }
  if (bad_ptr(c) || bad_ptr(w)) return XX_ERR_INVALID_ARGUMENT;
  return run_strain(p, c, w, n_b, dex_deps, ex_out, s);
}

int xx_run_many(int n_jobs, const xx_job* jobs, void* stream) {
  if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return XX_ERR_INVALID_ARGUMENT;
  for (int i = 0; i < n_jobs; ++i) {
    if (!jobs[i].plan) return XX_ERR_INVALID_ARGUMENT;
    for (int j = 0; j < i; ++j)
      if (jobs[j].plan == jobs[i].plan) return XX_ERR_INVALID_ARGUMENT;
  }
  cudaStream_t caller = (cudaStream_t)stream;
  // fork: every job's stream waits for the caller's queued work
  for (int i = 0; i < n_jobs; ++i) {
    xx_plan p = jobs[i].plan;
    cudaError_t e = cudaSuccess;
    if (!p->own_stream) e = cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !p->ev_fork) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !p->ev_join) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_fork, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->own_stream, p->ev_fork, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
  }
  int status = XX_OK;
  for (int i = 0; i < n_jobs; ++i) {
    const xx_job& j = jobs[i];
    xx_plan p = j.plan;
    int st;
    if (j.ex_out)
      st = xx_energy(p, j.c_occ, j.ld_occ, j.w_occ, j.n_occ, j.c_tgt, j.w_tgt, j.n_tgt, j.vx_out,
                     j.ex_out, p->own_stream);
    else
      st = xx_apply(p, j.c_occ, j.ld_occ, j.w_occ, j.n_occ, j.c_tgt, j.n_tgt, j.vx_out, p->own_stream);
    if (st != XX_OK && status == XX_OK) status = st;
  }
  // join: the caller's stream waits for every job
  for (int i = 0; i < n_jobs; ++i) {
    xx_plan p = jobs[i].plan;
    cudaError_t e = cudaEventRecord(p->ev_join, p->own_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, p->ev_join, 0);
    if (e != cudaSuccess && status == XX_OK) status = cuda_status(e);
  }
  return status;
}

}  // extern "C"

namespace {

// One band-pair batch of one job in the batched path: its pair arguments
// (inter set per round) and whether its role-swapped pass C runs too.  One
// launch holds batches that add into the same targets, so every batch adds
// into private accumulator planes of its own (a0, ta: its pass C targets; j0,
// tj and ct_plane0: its role-swapped targets), summed per target afterwards in
// batch order.
struct BatchedItem {
  PairArgs a;
  PairArgs ct;       // role-swapped arguments (mirrored items)
  bool mirrored = false;
  size_t pairs = 0;
  int a0 = 0, ta = 0, j0 = 0, tj = 0;
  long long c_plane0 = 0, ct_plane0 = 0;   // first private plane of each side
};

// acc[row] = sum over the row's private planes in table order; grid (chunks, rows)
__global__ void k_sum_planes(const double2* priv, const int* row_ptr, const int* planes, long long nn,
                             double2* acc) {
  const int row = blockIdx.y;
  const int b = row_ptr[row], e = row_ptr[row + 1];
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nn;
       i += (long long)gridDim.x * blockDim.x) {
    double2 sum = make_double2(0.0, 0.0);
    for (int k = b; k < e; ++k) {
      const double2 v = priv[(long long)planes[k] * nn + i];
      sum.x += v.x;
      sum.y += v.y;
    }
    acc[(long long)row * nn + i] = sum;
  }
}

// The batches of one Gamma-only job, as run_apply forms them: k = q tiles I <= J
// of the occupied square with the pair symmetry (tiles J > I mirrored), then the
// targets past the occupied set; without it, every target batch against every
// occupied batch.
void batched_items(xx_plan p, const xx_job& j, bool shared, std::vector<BatchedItem>& out) {
  int TA, TJ;
  batch_shape(p, j.n_tgt, j.n_occ, &TA, &TJ);
  long long planes = 0;
  auto add = [&](int a0, int ta, int j0, int tj, bool mirrored) {
    BatchedItem it;
    it.a = pair_args(p, ta, tj);
    it.a.u_tgt = grid_ptr(p, true, 0, a0, j.n_occ, j.n_tgt);
    it.a.u_occ = grid_ptr(p, shared, 0, j0, j.n_occ, j.n_tgt);
    it.a.w_occ = j.w_occ + j0;
    it.mirrored = mirrored;
    it.a0 = a0;
    it.ta = ta;
    it.j0 = j0;
    it.tj = tj;
    it.c_plane0 = planes;
    planes += ta;
    if (mirrored) {
      it.ct = it.a;
      it.ct.w_tgt = j.w_occ + a0;
      it.ct.w_occ = nullptr;
      it.ct_plane0 = planes;
      planes += tj;
    }
    it.pairs = (size_t)ta * tj;
    out.push_back(it);
  };
  const int n_occ = j.n_occ, n_tgt = j.n_tgt;
  if (shared && p->pair_symmetry && n_occ > 1) {
    const int T = TJ < TA ? TJ : TA;
    for (int i0 = 0; i0 < n_occ; i0 += T)
      for (int j0 = i0; j0 < n_occ; j0 += T)
        add(i0, std::min(T, n_occ - i0), j0, std::min(T, n_occ - j0), j0 > i0);
    for (int a0 = n_occ; a0 < n_tgt; a0 += TA)
      for (int j0 = 0; j0 < n_occ; j0 += TJ) add(a0, std::min(TA, n_tgt - a0), j0, std::min(TJ, n_occ - j0), false);
  } else {
    for (int a0 = 0; a0 < n_tgt; a0 += TA)
      for (int j0 = 0; j0 < n_occ; j0 += TJ) add(a0, std::min(TA, n_tgt - a0), j0, std::min(TJ, n_occ - j0), false);
  }
}

// Fork: each job's own stream waits for the work queued on `caller`.
int fork_streams(int n_jobs, const xx_job* jobs, cudaStream_t caller) {
  for (int i = 0; i < n_jobs; ++i) {
    xx_plan p = jobs[i].plan;
    cudaError_t e = cudaSuccess;
    if (!p->own_stream) e = cudaStreamCreateWithFlags(&p->own_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess && !p->ev_fork) e = cudaEventCreateWithFlags(&p->ev_fork, cudaEventDisableTiming);
    if (e == cudaSuccess && !p->ev_join) e = cudaEventCreateWithFlags(&p->ev_join, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventRecord(p->ev_fork, caller);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(p->own_stream, p->ev_fork, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
  }
  return XX_OK;
}

// Join: `caller` waits for the work queued on every job's own stream.
int join_streams(int n_jobs, const xx_job* jobs, cudaStream_t caller) {
  for (int i = 0; i < n_jobs; ++i) {
    xx_plan p = jobs[i].plan;
    cudaError_t e = cudaEventRecord(p->ev_join, p->own_stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(caller, p->ev_join, 0);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return cuda_status(e);
    }
  }
  return XX_OK;
}

// One batched launch of `pass` over the given items (each with its plan's grid
// length); splits into several launches past kMaxCellItems items.
int launch_batched(int pass, bool fp64, const std::vector<std::pair<const PairArgs*, int>>& items,
                   cudaStream_t s) {
  for (size_t first = 0; first < items.size(); first += kMaxCellItems) {
    const size_t count = std::min(items.size() - first, (size_t)kMaxCellItems);
    CellItems ci{};
    ci.n_items = (int)count;
    long long ctas = 0;
    int threads = 32;
    size_t smem = 0;
    for (size_t i = 0; i < count; ++i) {
      const PairArgs& a = *items[first + i].first;
      const int n = pass == kCellPassB ? a.nz : items[first + i].second;
      ci.item[i].a = a;
      ci.item[i].n = n;
      ci.item[i].cta0 = ctas;
      ctas += cell_item_ctas(pass, a);
      threads = std::max(threads, cell_body_threads(pass, fp64, n));
      smem = std::max(smem, cell_body_smem(pass, fp64, n, a.P1, a.P3));
    }
    const cudaError_t e = launch_cell_pass(pass, fp64, ci, ctas, threads, smem, s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  return XX_OK;
}

}  // namespace

extern "C" {

int xx_run_batched(int n_jobs, const xx_job* jobs, void* stream) {
  Range r("xx run batched");
  if (n_jobs < 0 || (n_jobs > 0 && !jobs)) return XX_ERR_INVALID_ARGUMENT;
  if (n_jobs == 0) return XX_OK;
  const int prec = jobs[0].plan ? jobs[0].plan->prec : -1;
  for (int i = 0; i < n_jobs; ++i) {
    const xx_job& j = jobs[i];
    xx_plan p = j.plan;
    if (!p || p->prec != prec || p->nk != 1 || p->n_shards > 1 || !cell_length_supported(p->N) ||
        !cell_length_supported(p->NZ))
      return XX_ERR_INVALID_ARGUMENT;
    for (int k = 0; k < i; ++k)
      if (jobs[k].plan == p) return XX_ERR_INVALID_ARGUMENT;
    if (j.n_occ < 0 || j.n_tgt < 0 || j.ld_occ < 0 || (j.ld_occ > 0 && j.ld_occ < j.n_occ))
      return XX_ERR_INVALID_ARGUMENT;
    if (j.n_tgt > 0 && (bad_ptr(j.c_tgt) || bad_ptr(j.vx_out))) return XX_ERR_INVALID_ARGUMENT;
    if (j.n_tgt > 0 && j.n_occ > 0 && (bad_ptr(j.c_occ) || bad_ptr(j.w_occ))) return XX_ERR_INVALID_ARGUMENT;
    if (j.ex_out && j.n_tgt > 0 && bad_ptr(j.w_tgt)) return XX_ERR_INVALID_ARGUMENT;
  }
  cudaStream_t caller = (cudaStream_t)stream;
  const bool fp64 = prec == XX_FP64;
  int st;
  // per job, on its own stream: orbital grids, kernel table, zeroed accumulators
  // and band-pair batches
  if ((st = fork_streams(n_jobs, jobs, caller))) return st;
  std::vector<std::vector<BatchedItem>> items(n_jobs);
  for (int i = 0; i < n_jobs; ++i) {
    const xx_job& j = jobs[i];
    xx_plan p = j.plan;
    cudaStream_t s = p->own_stream;
    if (j.n_tgt == 0 || j.n_occ == 0) continue;
    const int ld = j.ld_occ > 0 ? j.ld_occ : j.n_occ;
    const bool shared = j.c_occ == j.c_tgt && ld == j.n_tgt;
    if ((st = build_grids(p, 0, 1, j.c_occ, ld, j.n_occ, j.c_tgt, j.n_tgt, shared, s))) return st;
    if ((st = kernel_table_for(p, 0, 0, false, s))) return st;
    if ((st = ensure(p, p->acc, (size_t)j.n_tgt * n3(p) * 16))) return st;
    batched_items(p, j, shared, items[i]);
    // private accumulator planes of the batches (zeroed), and the table of the
    // planes that add up to each target, in batch order
    const BatchedItem& last = items[i].back();
    const long long planes = last.mirrored ? last.ct_plane0 + last.tj : last.c_plane0 + last.ta;
    const size_t priv_bytes = (size_t)planes * n3(p) * 16;
    if ((st = ensure(p, p->acc2, priv_bytes))) return st;
    if ((st = cuda_status(cudaMemsetAsync(p->acc2.p, 0, priv_bytes, s)))) return st;
    std::vector<std::vector<int>> rows(j.n_tgt);
    for (BatchedItem& it : items[i]) {
      it.a.acc = (double2*)p->acc2.p + it.c_plane0 * n3(p);
      for (int a = 0; a < it.ta; ++a) rows[it.a0 + a].push_back((int)(it.c_plane0 + a));
      if (it.mirrored) {
        it.ct.acc = (double2*)p->acc2.p + it.ct_plane0 * n3(p);
        for (int b = 0; b < it.tj; ++b) rows[it.j0 + b].push_back((int)(it.ct_plane0 + b));
      }
    }
    std::vector<int> tab(1, 0);
    for (const auto& row : rows) tab.push_back(tab.back() + (int)row.size());
    for (const auto& row : rows) tab.insert(tab.end(), row.begin(), row.end());
    if ((st = ensure(p, p->cells_tab, tab.size() * sizeof(int)))) return st;
    // pageable source: the copy has taken the data when the call returns
    if ((st = cuda_status(cudaMemcpyAsync(p->cells_tab.p, tab.data(), tab.size() * sizeof(int),
                                          cudaMemcpyHostToDevice, s))))
      return st;
  }
  if ((st = join_streams(n_jobs, jobs, caller))) return st;
  // rounds: each job's batches in order, as many per round as its workspace cap
  // holds (one round when every job's batches fit at once); in a launch the
  // batches run largest first (grid points x pairs), which shortens its tail
  std::vector<size_t> next(n_jobs, 0);
  cudaStream_t s = caller;
  for (;;) {
    std::vector<std::pair<const PairArgs*, int>> all, mirrored;
    for (int i = 0; i < n_jobs; ++i) {
      xx_plan p = jobs[i].plan;
      const size_t per_pair = inter_pair_bytes(p);
      size_t used = 0, first = next[i], end = next[i];
      while (end < items[i].size() && (end == first || (used + items[i][end].pairs) * per_pair <= p->cap))
        used += items[i][end++].pairs;
      if (end == first) continue;
      if ((st = ensure(p, p->inter, used * per_pair))) return st;
      size_t off = 0;
      for (size_t k = first; k < end; ++k) {
        BatchedItem& it = items[i][k];
        it.a.inter = (char*)p->inter.p + off * per_pair;
        it.ct.inter = it.a.inter;
        off += it.pairs;
        all.push_back({&it.a, p->N});
        if (it.mirrored) mirrored.push_back({&it.ct, p->N});
        p->pairs += (long long)it.pairs;
      }
      next[i] = end;
    }
    if (all.empty()) break;
    auto larger = [](const std::pair<const PairArgs*, int>& x, const std::pair<const PairArgs*, int>& y) {
      const double wx = (double)x.second * x.second * x.first->nz * x.first->TA * x.first->TJ;
      const double wy = (double)y.second * y.second * y.first->nz * y.first->TA * y.first->TJ;
      return wx > wy;
    };
    std::stable_sort(all.begin(), all.end(), larger);
    std::stable_sort(mirrored.begin(), mirrored.end(), larger);
    if ((st = launch_batched(kCellPassA, fp64, all, s))) return st;
    if ((st = launch_batched(kCellPassB, fp64, all, s))) return st;
    if ((st = launch_batched(kCellPassC, fp64, all, s))) return st;
    if (!mirrored.empty() && (st = launch_batched(kCellPassCT, fp64, mirrored, s))) return st;
    jobs[0].plan->launches += mirrored.empty() ? 3 : 4;
  }
  // per job, on its own stream: the sums of the private planes, grid -> sphere and E_x
  if ((st = fork_streams(n_jobs, jobs, caller))) return st;
  for (int i = 0; i < n_jobs; ++i) {
    const xx_job& j = jobs[i];
    xx_plan p = j.plan;
    cudaStream_t s = p->own_stream;
    if (j.n_tgt == 0) {
      if (j.ex_out && (st = cuda_status(cudaMemsetAsync(j.ex_out, 0, 2 * sizeof(double), s)))) return st;
      continue;
    }
    if (j.n_occ == 0) {
      if ((st = cuda_status(cudaMemsetAsync(j.vx_out, 0, (size_t)j.n_tgt * p->npw_max * 16, s)))) return st;
    } else {
      const int* tab = (const int*)p->cells_tab.p;
      const long long nn = n3(p);
      const int chunks = (int)std::min<long long>((nn + 255) / 256, 1024);
      k_sum_planes<<<dim3(chunks, j.n_tgt), 256, 0, s>>>((const double2*)p->acc2.p, tab, tab + j.n_tgt + 1,
                                                         nn, (double2*)p->acc.p);
      if ((st = launched(p, 1))) return st;
      if ((st = grid_to_sphere(p, 0, (double2*)p->acc.p, j.n_tgt, (double2*)j.vx_out, s))) return st;
    }
    if (j.ex_out && (st = run_energy_reduce(p, 0, 1, j.c_tgt, j.w_tgt, j.n_tgt, j.vx_out, j.ex_out, s)))
      return st;
  }
  return join_streams(n_jobs, jobs, caller);
}

int xx_apply_vjp(xx_plan p, const void* c_occ, int ld_occ, const double* w_occ, int n_occ,
                 const void* c_tgt, int n_tgt, const void* ybar, void* grad_tgt_out,
                 void* grad_occ_out, void* stream) {
  Range r("xx vjp");
  if (!p || n_occ < 0 || n_tgt < 0 || p->n_shards > 1) return XX_ERR_INVALID_ARGUMENT;
  if (ld_occ == 0) ld_occ = n_occ;
  if (ld_occ < n_occ) return XX_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  if (n_tgt > 0 && bad_ptr(ybar)) return XX_ERR_INVALID_ARGUMENT;
  const void* outs[2] = {grad_tgt_out, grad_occ_out};
  for (const void* o : outs)
    if (o && (o == c_occ || o == c_tgt || o == ybar)) return XX_ERR_INVALID_ARGUMENT;
  int st;
  if (grad_tgt_out && n_tgt > 0 && grad_occ_out && n_occ > 0 && p->fused_vjp) {
    if (bad_ptr(c_occ) || bad_ptr(w_occ) || bad_ptr(c_tgt)) return XX_ERR_INVALID_ARGUMENT;
    st = run_vjp_fused(p, c_occ, ld_occ, w_occ, n_occ, c_tgt, n_tgt, ybar, grad_tgt_out,
                       grad_occ_out, s);
    if (st != XX_ERR_OUT_OF_MEMORY) return st;
    // the occupied accumulators of every q do not fit: the two parts one after the other
  }
  if (grad_tgt_out && n_tgt > 0) {
    // V_x is Hermitian: dL/dc_tgt* = V_x ybar (a complex cotangent: general path)
    if ((st = apply_range(p, 0, p->nk, c_occ, ld_occ, w_occ, n_occ, ybar, n_tgt, grad_tgt_out,
                          false, stream)))
      return st;
  }
  if (grad_occ_out && n_occ > 0) {
    if (n_tgt == 0)
      return cuda_status(cudaMemsetAsync(grad_occ_out, 0, (size_t)p->nk * n_occ * p->npw_max * 16, s));
    if (bad_ptr(c_occ) || bad_ptr(w_occ) || bad_ptr(c_tgt)) return XX_ERR_INVALID_ARGUMENT;
    if ((st = run_vjp_occ(p, c_occ, ld_occ, w_occ, n_occ, c_tgt, n_tgt, ybar, grad_occ_out, s)))
      return st;
  }
  return XX_OK;
}

int xx_sync(xx_plan p, void* stream, double timeout_s) {
  if (!p) return XX_ERR_INVALID_ARGUMENT;
  cudaStream_t s = (cudaStream_t)stream;
  if (timeout_s > 0.0) {
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return XX_ERR_CUDA;
    cudaEventRecord(ev, s);
    struct timespec ts0, ts1;
    clock_gettime(CLOCK_MONOTONIC, &ts0);
    for (;;) {
      const cudaError_t q = cudaEventQuery(ev);
      if (q == cudaSuccess) break;
      if (q != cudaErrorNotReady) {
        cudaEventDestroy(ev);
        return cuda_status(q);
      }
      clock_gettime(CLOCK_MONOTONIC, &ts1);
      const double el = (ts1.tv_sec - ts0.tv_sec) + 1e-9 * (ts1.tv_nsec - ts0.tv_nsec);
      if (el > timeout_s) {
        cudaEventDestroy(ev);
        return XX_ERR_TIMEOUT;
      }
      struct timespec nap = {0, 200000};
      nanosleep(&nap, nullptr);
    }
    cudaEventDestroy(ev);
  } else {
    const cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_status(e);
  }
  int flag = 0;
  if (cudaMemcpy(&flag, p->d_err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return XX_ERR_CUDA;
  if (flag) {
    cudaMemset(p->d_err, 0, sizeof(int));
    return XX_ERR_DEVICE_FLAG;
  }
  return XX_OK;
}

int xx_set_option(xx_plan p, int option, long long value) {
  if (!p) return XX_ERR_INVALID_ARGUMENT;
  switch (option) {
    case XX_OPT_PAIR_SYMMETRY:
      p->pair_symmetry = value != 0;
      return XX_OK;
    case XX_OPT_REAL_GAMMA:
      if (value != 0 && !p->gamma_closed) return XX_ERR_INVALID_ARGUMENT;
      p->real_gamma = value != 0;
      return XX_OK;
    case XX_OPT_ACC_LIMIT_MB:
      if (value < 0) return XX_ERR_INVALID_ARGUMENT;
      p->acc_limit_mb = value;
      return XX_OK;
    case XX_OPT_FUSED_VJP:
      p->fused_vjp = value != 0;
      return XX_OK;
    case XX_OPT_TEST_WAIT_EXPIRY:
      p->test_wait_expiry = value != 0;
      return XX_OK;
    case XX_OPT_STAGE_PASS_A:
      if (value < 0 || value > 2) return XX_ERR_INVALID_ARGUMENT;
      p->stage_pass_a = (int)value;
      return XX_OK;
    case XX_OPT_TMA_PASS_B:
      if (value < 0 || value > 2) return XX_ERR_INVALID_ARGUMENT;
      p->tma_pass_b = (int)value;
      return XX_OK;
    case XX_OPT_TABLE_CACHE:
      if (value == 0) {
        release_counted(p, p->vt_all);
        p->vt_all_state = -1;
      } else if (p->vt_all_state < 0) {
        p->vt_all_state = 0;
      }
      p->vt_sel = nullptr;
      return XX_OK;
    default:
      return XX_ERR_INVALID_ARGUMENT;
  }
}

int xx_set_shard(xx_plan p, int shard, int n_shards) {
  if (!p || n_shards < 1 || shard < 0 || shard >= n_shards) return XX_ERR_INVALID_ARGUMENT;
  p->shard = shard;
  p->n_shards = n_shards;
  return XX_OK;
}

int xx_shard_blocks(int nk, int n_occ, int n_tgt, int n_shards, int* owner_out) {
  if (nk < 1 || n_occ < 0 || n_tgt < 0 || n_shards < 1 || !owner_out) return XX_ERR_INVALID_ARGUMENT;
  std::vector<int> owner;
  assign_blocks(nk, n_occ, n_tgt, n_shards, owner);
  std::copy(owner.begin(), owner.end(), owner_out);
  return XX_OK;
}

int xx_set_batch(xx_plan p, int targets_per_batch, int occupied_per_batch) {
  if (!p || targets_per_batch < 0 || occupied_per_batch < 0) return XX_ERR_INVALID_ARGUMENT;
  p->ta_user = targets_per_batch;
  p->tj_user = occupied_per_batch;
  return XX_OK;
}

int xx_profile_enable(xx_plan p, int enable) {
  if (!p) return XX_ERR_INVALID_ARGUMENT;
  p->profiling = enable != 0;
  return XX_OK;
}

int xx_profile_read(xx_plan p, double* ms, long long* launches, int n_classes, int reset) {
  if (!p || n_classes < 0 || (n_classes > 0 && (!ms || !launches))) return XX_ERR_INVALID_ARGUMENT;
  for (int c = 0; c < n_classes; ++c) {
    ms[c] = 0.0;
    launches[c] = 0;
  }
  for (const auto& r : p->recs) {
    float t = 0.0f;
    cudaError_t e = cudaEventSynchronize(p->ev_pool[r.e1]);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, p->ev_pool[r.e0], p->ev_pool[r.e1]);
    if (e != cudaSuccess) return cuda_status(e);
    if (r.cls < n_classes) {
      ms[r.cls] += t;
      launches[r.cls] += 1;
    }
  }
  if (reset) {
    p->recs.clear();
    p->ev_next = 0;
  }
  return XX_OK;
}

int xx_exact_grid(const int* n_max, int* n_out) {
  if (!n_max || !n_out) return XX_ERR_INVALID_ARGUMENT;
  int need = 0;
  for (int ax = 0; ax < 3; ++ax) {
    if (n_max[ax] < 0 || n_max[ax] > 4096) return XX_ERR_INVALID_ARGUMENT;
    const int m = 4 * n_max[ax] + 1;
    if (m > need) need = m;
  }
  for (int n = need; n <= 108; ++n)
    if (supported_n(n)) {
      *n_out = n;
      return XX_OK;
    }
  return XX_ERR_UNSUPPORTED_GRID;
}

int xx_exact_grid3(const int* n_max, int* grid_out) {
  if (!n_max || !grid_out) return XX_ERR_INVALID_ARGUMENT;
  int m[3];
  for (int ax = 0; ax < 3; ++ax) {
    if (n_max[ax] < 0 || n_max[ax] > 4096) return XX_ERR_INVALID_ARGUMENT;
    const int nm1[3] = {n_max[ax], 0, 0};
    const int st = xx_exact_grid(nm1, &m[ax]);
    if (st != XX_OK) return st;
  }
  // the two axes made equal take the longer of their lengths
  const int pairs[3][2] = {{0, 1}, {0, 2}, {1, 2}};
  long long best = -1;
  for (const auto& pr : pairs) {
    int g[3] = {m[0], m[1], m[2]};
    const int L = std::max(m[pr[0]], m[pr[1]]);
    g[pr[0]] = g[pr[1]] = L;
    const long long pts = (long long)g[0] * g[1] * g[2];
    if (best < 0 || pts < best) {
      best = pts;
      std::copy(g, g + 3, grid_out);
    }
  }
  return XX_OK;
}

int xx_plan_info(xx_plan p, xx_info* info) {
  if (!p || !info) return XX_ERR_INVALID_ARGUMENT;
  std::memset(info, 0, sizeof(*info));
  for (int i = 0; i < 3; ++i) {   // in the caller's axis order
    info->grid[p->perm[i]] = p->grid[i];
    info->n_max[p->perm[i]] = p->nmax[i];
    info->pruned[p->perm[i]] = 2 * p->h[i] + 1;
  }
  info->nk = p->nk;
  info->npw_max = p->npw_max;
  info->precision = p->prec;
  info->targets_per_batch = p->ta_last;
  info->occupied_per_batch = p->tj_last;
  info->omega = p->omega;
  info->workspace_bytes = p->ws_bytes;
  info->peak_workspace_bytes = p->peak_bytes;
  info->kernel_launches = p->launches;
  info->pairs_transformed = p->pairs;
  info->q_per_batch = p->g_last;
  return XX_OK;
}

}  // extern "C"
