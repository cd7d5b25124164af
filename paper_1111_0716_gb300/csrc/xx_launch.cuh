// xx_launch.cuh -- host launchers of the templated kernels and the per-grid-
// length kernel table.  Each supported FFT length N is instantiated in its own
// translation unit (xx_n<N>.cu) so that the builds run in parallel.
#pragma once

#include "xx_kernels.cuh"

namespace xx {

constexpr int kThreads = 256;

struct KernelSet {
  void (*pass_a)(const PairArgs&, cudaStream_t);
  void (*pass_b)(const PairArgs&, cudaStream_t);
  void (*pass_b_dmu)(const PairArgs&, cudaStream_t);
  void (*pass_b_strain)(const PairArgs&, cudaStream_t);
  void (*pass_c)(const PairArgs&, cudaStream_t);
  void (*pass_c_packed)(const PairArgs&, cudaStream_t);
  void (*pass_ct)(const PairArgs&, cudaStream_t);
  void (*s2g_z)(const GridArgs&, cudaStream_t);
  void (*s2g_xy)(const GridArgs&, cudaStream_t);
};

struct KernelTable {
  int n;
  KernelSet f32, f64;
  // FP32 pass B staged by tensor copies (persistent grid of `grid` CTAs), and
  // its resident CTAs per SM for a given intermediate shape
  void (*pass_b_tma)(const PairArgs&, const CUtensorMap&, int grid, cudaStream_t);
  int (*pass_b_tma_per_sm)(int LX, int P1, int P3);
  void (*g2s_xy)(const GridArgs&, cudaStream_t);
  void (*g2s_z)(const GridArgs&, cudaStream_t);
};

// Returns the table for FFT length n, or nullptr when n is not built in.
const KernelTable* kernel_table(int n);

template <typename K> inline void allow_smem(K kernel, size_t bytes) {
  if (bytes > 48 * 1024) cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

template <int N, typename T> void launch_pass_a(const PairArgs& p, cudaStream_t s) {
  if (sizeof(T) == 4 && p.stage_a) {
    const size_t sm = smem_pass_a_staged<N>();
    allow_smem(k_pass_a_staged<N>, sm);
    k_pass_a_staged<N><<<dim3(p.TA, p.nz), PassASCfg<N>::NT, sm, s>>>(p);
    return;
  }
  using G = PassACfg<N, T>;
  const size_t sm = G::smem();
  allow_smem(k_pass_a<N, T>, sm);
  k_pass_a<N, T><<<dim3(p.TA, p.nz), G::NT, sm, s>>>(p);
}
template <int N, typename T> void launch_pass_b(const PairArgs& p, cudaStream_t s) {
  const size_t sm = smem_pencil<N, T>(p.P1, p.P3);
  allow_smem(k_pass_b<N, kThreads, T>, sm);
  k_pass_b<N, kThreads, T><<<dim3(p.P2, p.TA * p.TJ), kThreads, sm, s>>>(p);
}
template <int N> void launch_pass_b_tma(const PairArgs& p, const CUtensorMap& tm, int grid, cudaStream_t s) {
  const size_t sm = smem_pass_b_tma<N>(p.LX, p.P1, p.P3);
  allow_smem(k_pass_b_tma<N, kThreads>, sm);
  k_pass_b_tma<N, kThreads><<<grid, kThreads, sm, s>>>(tm, p, p.P2 * p.TA * p.TJ);
}
template <int N> int pass_b_tma_per_sm(int LX, int P1, int P3) {
  const size_t sm = smem_pass_b_tma<N>(LX, P1, P3);
  allow_smem(k_pass_b_tma<N, kThreads>, sm);
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k_pass_b_tma<N, kThreads>, kThreads, sm) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}
template <int N, typename T> void launch_pass_b_dmu(const PairArgs& p, cudaStream_t s) {
  const size_t sm = smem_pencil<N, T>(p.P1, 0);
  allow_smem(k_pass_b_dmu<N, kThreads, T>, sm);
  k_pass_b_dmu<N, kThreads, T><<<dim3(p.P2, p.TA * p.TJ), kThreads, sm, s>>>(p);
}
template <int N, typename T> void launch_pass_b_strain(const PairArgs& p, cudaStream_t s) {
  const size_t sm = smem_pencil<N, T>(p.P1, 0);
  allow_smem(k_pass_b_strain<N, kThreads, T>, sm);
  k_pass_b_strain<N, kThreads, T><<<dim3(p.P2, p.TA * p.TJ), kThreads, sm, s>>>(p);
}
template <int N, typename T, bool PACKED> void launch_pass_c(const PairArgs& p, cudaStream_t s) {
  using G = PlaneCfg<N, T>;
  const size_t sm = G::smem();
  allow_smem(k_pass_c<N, T, PACKED>, sm);
  k_pass_c<N, T, PACKED><<<dim3(p.TA, p.nz), G::NT, sm, s>>>(p);
}
template <int N, typename T> void launch_pass_ct(const PairArgs& p, cudaStream_t s) {
  using G = PlaneCfg<N, T>;
  const size_t sm = G::smem();
  allow_smem(k_pass_ct<N, T>, sm);
  k_pass_ct<N, T><<<dim3(p.TJ, p.nz), G::NT, sm, s>>>(p);
}
template <int N, typename T> void launch_s2g_z(const GridArgs& g, cudaStream_t s) {
  const size_t sm = smem_pencil<N, T>(g.Q1, 0);
  allow_smem(k_s2g_z<N, kThreads, T>, sm);
  k_s2g_z<N, kThreads, T><<<dim3(g.Q2, g.nb), kThreads, sm, s>>>(g);
}
template <int N, typename T> void launch_s2g_xy(const GridArgs& g, cudaStream_t s) {
  using G = PlaneCfg<N, T>;
  const size_t sm = G::smem();
  allow_smem(k_s2g_xy<N, T>, sm);
  k_s2g_xy<N, T><<<dim3(g.nb, g.nz), G::NT, sm, s>>>(g);
}
template <int N> void launch_g2s_xy(const GridArgs& g, cudaStream_t s) {
  using G = PlaneCfg<N, double>;
  const size_t sm = G::smem();
  allow_smem(k_g2s_xy<N>, sm);
  k_g2s_xy<N><<<dim3(g.nb, g.nz), G::NT, sm, s>>>(g);
}
template <int N> void launch_g2s_z(const GridArgs& g, cudaStream_t s) {
  const size_t sm = smem_pencil<N, double>(g.Q1, 0);
  allow_smem(k_g2s_z<N, kThreads>, sm);
  k_g2s_z<N, kThreads><<<dim3(g.Q2, g.nb), kThreads, sm, s>>>(g);
}

template <int N> const KernelTable* make_table() {
  static const KernelTable t = {
      N,
      {launch_pass_a<N, float>, launch_pass_b<N, float>, launch_pass_b_dmu<N, float>,
       launch_pass_b_strain<N, float>, launch_pass_c<N, float, false>, launch_pass_c<N, float, true>,
       launch_pass_ct<N, float>, launch_s2g_z<N, float>,
       launch_s2g_xy<N, float>},
      {launch_pass_a<N, double>, launch_pass_b<N, double>, launch_pass_b_dmu<N, double>,
       launch_pass_b_strain<N, double>, launch_pass_c<N, double, false>, launch_pass_c<N, double, true>,
       launch_pass_ct<N, double>, launch_s2g_z<N, double>,
       launch_s2g_xy<N, double>},
      launch_pass_b_tma<N>,
      pass_b_tma_per_sm<N>,
      launch_g2s_xy<N>,
      launch_g2s_z<N>};
  return &t;
}

}  // namespace xx

#define XX_INSTANTIATE(N) \
  namespace xx {          \
  const KernelTable* kernel_table_##N() { return make_table<N>(); } \
  }
