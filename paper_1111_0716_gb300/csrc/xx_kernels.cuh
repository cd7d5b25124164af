// xx_kernels.cuh -- CUDA kernels of the Fock-exchange pipeline (sm_103a).
//
// The exchange loops of Hutchinson & Widom (Sec. "Our Implementation", Eq. 2):
// for every k, q and target band a, occupied band j,
//   rho = conj(u_qj) u_ka;  rhohat = FFT(rho)/N;  What = v(k-q+G) rhohat;
//   W = IFFT(What);  acc_ka += -(w_qj/N_q) u_qj W,
// are run as three fused passes over a batch of band pairs (the NSIM-style
// multiplexing of the paper's innermost loop):
//   pass A  one z-plane per CTA: codensity + forward x and y FFTs, output
//           pruned to |f_x|,|f_y| <= 2 n_max (the codensity's exact support);
//   pass B  one (pair, f_y) row per CTA: forward z FFT, multiply by the kernel
//           table, inverse z FFT, in place;
//   pass C  one z-plane per CTA: inverse y and x FFTs, multiply by u_qj and
//           accumulate over the occupied batch in registers, then add into the
//           FP64 accumulator of the target.
// Around them: sphere->grid (scatter + inverse FFT) once per orbital, the
// kernel table once per (k, q), grid->sphere (FFT + gather) once per target,
// and fixed-order reductions for E_x and dE_x/dmu.
#pragma once

#include "xx_fft.cuh"

namespace xx {

// ------------------------------------------------------------- arguments --

struct PairArgs {
  const void* u_tgt;     // [TA][N^3] grids of the target batch (at k)
  const void* u_occ;     // [TJ][N^3] grids of the occupied batch (at q)
  void* inter;           // [TA*TJ][N][P2][P1] pair intermediates
  const void* vt;        // [P3][P2][P1] v(k-q+G)/N   (pass B)
  const void* dvt;       // [P3][P2][P1] dv/dmu/N^2   (pass B, mu-gradient)
  double2* acc;          // [TA][N^3] FP64 accumulators of the target batch
  const double* w_occ;   // [TJ] occupations of the occupied batch
  const double* w_tgt;   // [TA] occupations of the target batch
  double* partial;       // [TA*TJ][P2] mu-gradient partial sums
  const void* tw;        // [N] exp(-2 pi i e / N) in the pass precision
  long long u_tgt_stride;  // elements between consecutive target grids
  long long u_occ_stride;  // elements between consecutive occupied grids
  int TA, TJ;
  int h1, h2, h3, P1, P2, P3;
  double coef;           // -1 / N_q
};

struct GridArgs {        // sphere <-> grid
  const double2* c;      // [nb][npw_max] sphere coefficients (FP64)
  double2* out;          // [nb][npw_max] sphere output (grid -> sphere)
  const int* miller;     // [npw_max][3] of this k-point
  int npw, npw_max, nb;
  void* box;             // [nb][Q3][Q2][Q1]
  void* stage;           // [nb][N][Q2][Q1]
  void* u;               // [nb][N^3] grids (sphere -> grid output)
  const double2* f;      // [nb][N^3] FP64 grids (grid -> sphere input)
  const void* tw;
  int n1, n2, n3, Q1, Q2, Q3;
  double scale;
  int* err;
};

struct VtabArgs {
  double M[9];           // reciprocal metric b_i . b_j
  double d[3];           // k - q (fractional)
  int h1, h2, h3, P1, P2, P3;
  int kernel;            // 0 screened, 1 Coulomb (g = 0 dropped)
  double mu;
  double inv_n, inv_n2;  // 1/N, 1/N^2
};

// ---------------------------------------------------- CTA building blocks --

// Forward x then y transform of one real-space plane held in sA (N rows of
// N + 1), in place; outputs only the kept frequencies |f_x| <= h1, |f_y| <= h2
// through store(kyb, kxb, value).  After the x transform, frequency
// f_x = k1 + A*k2 sits in column k1*B + k2 (the second step's natural order).
template <int N, int NT, typename T, typename Load, typename Store>
__device__ __forceinline__ void plane_forward(const cplx<T>* tw, cplx<T>* sA, int h1, int P1,
                                              int h2, Load load, Store store) {
  using C = cplx<T>;
  constexpr int A = Fac<N>::A, B = Fac<N>::B, LD = N + 1;
#pragma unroll 1
  for (int it = threadIdx.x; it < N * B; it += NT) {
    const int n2 = it % B, y = it / B;
    C r[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) r[n1] = load(y, B * n1 + n2);
    dft<A, false>(r);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) sA[y * LD + k1 * B + n2] = tw_mul<false>(r[k1], tw[n2 * k1]);
  }
  __syncthreads();
#pragma unroll 1
  for (int it = threadIdx.x; it < N * A; it += NT) {
    const int k1 = it % A, y = it / A;
    C r[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) r[n2] = sA[y * LD + k1 * B + n2];
    dft<B, false>(r);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) sA[y * LD + k1 * B + k2] = r[k2];
  }
  __syncthreads();
#pragma unroll 1
  for (int it = threadIdx.x; it < P1 * B; it += NT) {
    const int kxb = it % P1, n2 = it / P1;
    const int fx = idx_of_box(kxb, N, h1);
    const int col = (fx % A) * B + fx / A;
    C r[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) r[n1] = sA[(B * n1 + n2) * LD + col];
    dft<A, false>(r);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) sA[(k1 * B + n2) * LD + col] = tw_mul<false>(r[k1], tw[n2 * k1]);
  }
  __syncthreads();
#pragma unroll 1
  for (int it = threadIdx.x; it < P1 * A; it += NT) {
    const int kxb = it % P1, k1 = it / P1;
    const int fx = idx_of_box(kxb, N, h1);
    const int col = (fx % A) * B + fx / A;
    C r[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) r[n2] = sA[(k1 * B + n2) * LD + col];
    dft<B, false>(r);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) {
      const int k = k1 + A * k2;
      if (kept(k, N, h2)) store(box_of(k, N, h2), kxb, r[k2]);
    }
  }
  __syncthreads();
}

// Inverse y then x transform of one plane from kept frequencies
// (load(kyb, kxb)) to the full real-space plane, in place in sA.  Every output
// goes to consume(i, k2, y, x, value), where (i, k2) is a compile-time
// register slot of the calling thread (fixed across calls).  After the y
// transform, row y = k1 + A*k2 sits in sA row k1*B + k2.
template <int N, int NT, typename T, typename Load, typename Consume>
__device__ __forceinline__ void plane_inverse(const cplx<T>* tw, cplx<T>* sA, int h1, int P1,
                                              int h2, Load load, Consume consume) {
  using C = cplx<T>;
  constexpr int A = Fac<N>::A, B = Fac<N>::B, LD = N + 1;
  constexpr int IPT = (N * A + NT - 1) / NT;
#pragma unroll 1
  for (int it = threadIdx.x; it < P1 * B; it += NT) {
    const int kxb = it % P1, n2 = it / P1;
    const int xm = idx_of_box(kxb, N, h1);
    C r[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) {
      const int m = B * n1 + n2;
      r[n1] = kept(m, N, h2) ? load(box_of(m, N, h2), kxb) : czero<C>();
    }
    dft<A, true>(r);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) sA[(k1 * B + n2) * LD + xm] = tw_mul<true>(r[k1], tw[n2 * k1]);
  }
  __syncthreads();
#pragma unroll 1
  for (int it = threadIdx.x; it < P1 * A; it += NT) {
    const int kxb = it % P1, k1 = it / P1;
    const int xm = idx_of_box(kxb, N, h1);
    C r[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) r[n2] = sA[(k1 * B + n2) * LD + xm];
    dft<B, true>(r);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) sA[(k1 * B + k2) * LD + xm] = r[k2];
  }
  __syncthreads();
#pragma unroll 1
  for (int it = threadIdx.x; it < N * B; it += NT) {
    const int n2 = it % B, row = it / B;
    C r[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) {
      const int m = B * n1 + n2;
      r[n1] = kept(m, N, h1) ? sA[row * LD + m] : czero<C>();
    }
    dft<A, true>(r);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) sA[row * LD + k1 * B + n2] = tw_mul<true>(r[k1], tw[n2 * k1]);
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const int it = threadIdx.x + i * NT;
    if (it < N * A) {
      const int k1 = it % A, row = it / A;
      const int y = row / B + A * (row % B);
      C r[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) r[n2] = sA[row * LD + k1 * B + n2];
      dft<B, true>(r);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) consume(i, k2, y, k1 + A * k2, r[k2]);
    }
  }
  __syncthreads();
}

// Forward z transform of a row of width W (pencils indexed by c < W);
// load(z, c) real space, out(kzb, c, value) for kept |f_z| <= h3.
template <int N, int NT, typename T, typename Load, typename Out>
__device__ __forceinline__ void pencil_forward(const cplx<T>* tw, cplx<T>* sZ, int W, int h3,
                                              Load load, Out out) {
  using C = cplx<T>;
  constexpr int A = Fac<N>::A, B = Fac<N>::B;
#pragma unroll 1
  for (int it = threadIdx.x; it < W * B; it += NT) {
    const int c = it % W, n2 = it / W;
    C r[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) r[n1] = load(B * n1 + n2, c);
    dft<A, false>(r);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) sZ[(k1 * B + n2) * W + c] = tw_mul<false>(r[k1], tw[n2 * k1]);
  }
  __syncthreads();
#pragma unroll 1
  for (int it = threadIdx.x; it < W * A; it += NT) {
    const int c = it % W, k1 = it / W;
    C r[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) r[n2] = sZ[(k1 * B + n2) * W + c];
    dft<B, false>(r);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) {
      const int k = k1 + A * k2;
      if (kept(k, N, h3)) out(box_of(k, N, h3), c, r[k2]);
    }
  }
}

// Inverse z transform of a row of width W from kept frequencies load(kzb, c)
// to real space store(z, c, value).
template <int N, int NT, typename T, typename Load, typename Store>
__device__ __forceinline__ void pencil_inverse(const cplx<T>* tw, cplx<T>* sZ, int W, int h3,
                                              Load load, Store store) {
  using C = cplx<T>;
  constexpr int A = Fac<N>::A, B = Fac<N>::B;
#pragma unroll 1
  for (int it = threadIdx.x; it < W * B; it += NT) {
    const int c = it % W, n2 = it / W;
    C r[A];
#pragma unroll
    for (int n1 = 0; n1 < A; ++n1) {
      const int m = B * n1 + n2;
      r[n1] = kept(m, N, h3) ? load(box_of(m, N, h3), c) : czero<C>();
    }
    dft<A, true>(r);
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) sZ[(k1 * B + n2) * W + c] = tw_mul<true>(r[k1], tw[n2 * k1]);
  }
  __syncthreads();
#pragma unroll 1
  for (int it = threadIdx.x; it < W * A; it += NT) {
    const int c = it % W, k1 = it / W;
    C r[B];
#pragma unroll
    for (int n2 = 0; n2 < B; ++n2) r[n2] = sZ[(k1 * B + n2) * W + c];
    dft<B, true>(r);
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) store(k1 + A * k2, c, r[k2]);
  }
}

template <int N, typename T> __device__ __forceinline__ void load_twiddles(cplx<T>* dst, const void* src) {
  for (int i = threadIdx.x; i < N; i += blockDim.x) dst[i] = ((const cplx<T>*)src)[i];
}

// Shared-memory sizes (bytes) of each kernel.
template <int N, typename T> constexpr size_t smem_plane() {
  return sizeof(cplx<T>) * ((size_t)N + (size_t)N * (N + 1));
}
template <int N, typename T> constexpr size_t smem_pencil(int W, int P3) {
  return sizeof(cplx<T>) * ((size_t)N + (size_t)N * W + (size_t)P3 * W);
}

// ------------------------------------------------------------- the passes --

// Pass A: grid (TA, N); CTA (ta, z) loops over the TJ occupied bands.
template <int N, int NT, typename T>
__global__ void __launch_bounds__(NT) k_pass_a(PairArgs p) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sA = tw + N;
  load_twiddles<N, T>(tw, p.tw);
  __syncthreads();
  const int ta = blockIdx.x, z = blockIdx.y;
  constexpr long long plane = (long long)N * N;
  const C* ua = reinterpret_cast<const C*>(p.u_tgt) + ta * p.u_tgt_stride + z * plane;
#pragma unroll 1
  for (int tj = 0; tj < p.TJ; ++tj) {
    const C* uj = reinterpret_cast<const C*>(p.u_occ) + tj * p.u_occ_stride + z * plane;
    C* out = reinterpret_cast<C*>(p.inter) +
             ((long long)(ta * p.TJ + tj) * N + z) * (long long)p.P2 * p.P1;
    const int P1 = p.P1;
    plane_forward<N, NT, T>(
        tw, sA, p.h1, p.P1, p.h2,
        [&](int y, int x) { return cmulc(uj[y * N + x], ua[y * N + x]); },
        [&](int kyb, int kxb, C v) { out[kyb * P1 + kxb] = v; });
    __syncthreads();
  }
}

// Pass B: grid (P2, TA*TJ); CTA (kyb, pair) transforms its row along z,
// multiplies by v(k - q + G)/N and transforms back, in place.
template <int N, int NT, typename T>
__global__ void __launch_bounds__(NT) k_pass_b(PairArgs p) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sZ = tw + N;
  C* sK = sZ + N * p.P1;
  load_twiddles<N, T>(tw, p.tw);
  __syncthreads();
  const int kyb = blockIdx.x, pair = blockIdx.y;
  const int P1 = p.P1, P2 = p.P2;
  const long long zstride = (long long)P2 * P1;
  C* row = reinterpret_cast<C*>(p.inter) + (long long)pair * N * zstride + (long long)kyb * P1;
  const T* vt = reinterpret_cast<const T*>(p.vt);
  pencil_forward<N, NT, T>(
      tw, sZ, P1, p.h3, [&](int z, int c) { return row[z * zstride + c]; },
      [&](int kzb, int c, C v) {
        const T s = vt[((long long)kzb * P2 + kyb) * P1 + c];
        sK[kzb * P1 + c] = s * v;
      });
  __syncthreads();
  pencil_inverse<N, NT, T>(
      tw, sZ, P1, p.h3, [&](int kzb, int c) { return sK[kzb * P1 + c]; },
      [&](int z, int c, C v) { row[z * zstride + c] = v; });
}

// Pass B for dE/dmu: forward z only, partial[pair][kyb] = sum dv/dmu/N^2 |rho|^2.
template <int N, int NT, typename T>
__global__ void __launch_bounds__(NT) k_pass_b_dmu(PairArgs p) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sZ = tw + N;
  __shared__ double red[NT];
  load_twiddles<N, T>(tw, p.tw);
  __syncthreads();
  const int kyb = blockIdx.x, pair = blockIdx.y;
  const int P1 = p.P1, P2 = p.P2;
  const long long zstride = (long long)P2 * P1;
  const C* row = reinterpret_cast<const C*>(p.inter) + (long long)pair * N * zstride + (long long)kyb * P1;
  const T* dvt = reinterpret_cast<const T*>(p.dvt);
  double s = 0.0;
  pencil_forward<N, NT, T>(
      tw, sZ, P1, p.h3, [&](int z, int c) { return row[z * zstride + c]; },
      [&](int kzb, int c, C v) {
        const double w = (double)dvt[((long long)kzb * P2 + kyb) * P1 + c];
        s += w * ((double)v.x * (double)v.x + (double)v.y * (double)v.y);
      });
  red[threadIdx.x] = s;
  __syncthreads();
  for (int off = NT / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off) red[threadIdx.x] += red[threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x == 0) p.partial[(long long)pair * P2 + kyb] = red[0];
}

// Pass C: grid (TA, N); CTA (ta, z) accumulates -(w_j/N_q) u_j W over the
// occupied batch in registers and adds the plane into the FP64 accumulator.
template <int N, int NT, typename T>
__global__ void __launch_bounds__(NT) k_pass_c(PairArgs p) {
  using C = cplx<T>;
  constexpr int A = Fac<N>::A, B = Fac<N>::B;
  constexpr int IPT = (N * A + NT - 1) / NT;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sA = tw + N;
  load_twiddles<N, T>(tw, p.tw);
  __syncthreads();
  const int ta = blockIdx.x, z = blockIdx.y;
  constexpr long long plane = (long long)N * N;
  const int P1 = p.P1;
  C acc[IPT][B];
#pragma unroll
  for (int i = 0; i < IPT; ++i)
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) acc[i][k2] = czero<C>();
#pragma unroll 1
  for (int tj = 0; tj < p.TJ; ++tj) {
    const C* in = reinterpret_cast<const C*>(p.inter) +
                  ((long long)(ta * p.TJ + tj) * N + z) * (long long)p.P2 * p.P1;
    const C* uj = reinterpret_cast<const C*>(p.u_occ) + tj * p.u_occ_stride + z * plane;
    const T cf = (T)(p.coef * p.w_occ[tj]);
    plane_inverse<N, NT, T>(
        tw, sA, p.h1, p.P1, p.h2, [&](int kyb, int kxb) { return in[kyb * P1 + kxb]; },
        [&](int i, int k2, int y, int x, C v) {
          const C t = cmul(uj[y * N + x], v);
          acc[i][k2].x += cf * t.x;
          acc[i][k2].y += cf * t.y;
        });
  }
  double2* dst = p.acc + ta * plane * N + z * plane;
#pragma unroll
  for (int i = 0; i < IPT; ++i) {
    const int it = threadIdx.x + i * NT;
    if (it < N * A) {
      // same slot -> (y, x) map as plane_inverse's last step
      const int k1 = it % A, row = it / A;
      const int y = row / B + A * (row % B);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) {
        double2* o = dst + y * N + k1 + A * k2;
        double2 cur = *o;
        cur.x += (double)acc[i][k2].x;
        cur.y += (double)acc[i][k2].y;
        *o = cur;
      }
    }
  }
}

// ------------------------------------------------------ kernel table (a2) --

// v(k - q + G)/N and dv/dmu/N^2 over the pruned box, evaluated in FP64.
template <typename T>
__global__ void k_vtab(T* vt, T* dvt, VtabArgs a) {
  const long long n = (long long)a.P1 * a.P2 * a.P3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % a.P1), ky = (int)((i / a.P1) % a.P2), kz = (int)(i / ((long long)a.P1 * a.P2));
    const double m0 = (double)(kx - a.h1) + a.d[0];
    const double m1 = (double)(ky - a.h2) + a.d[1];
    const double m2 = (double)(kz - a.h3) + a.d[2];
    const bool zero = (m0 == 0.0 && m1 == 0.0 && m2 == 0.0);
    const double g2 = m0 * (a.M[0] * m0 + a.M[1] * m1 + a.M[2] * m2) +
                      m1 * (a.M[3] * m0 + a.M[4] * m1 + a.M[5] * m2) +
                      m2 * (a.M[6] * m0 + a.M[7] * m1 + a.M[8] * m2);
    const double pi = 3.14159265358979323846;
    double v, dv;
    if (a.kernel == 0) {
      const double x = g2 / (4.0 * a.mu * a.mu);
      v = zero ? pi / (a.mu * a.mu) : 4.0 * pi / g2 * (-expm1(-x));
      dv = -2.0 * pi / (a.mu * a.mu * a.mu) * exp(-x);
    } else {
      v = zero ? 0.0 : 4.0 * pi / g2;
      dv = 0.0;
    }
    vt[i] = (T)(v * a.inv_n);
    if (dvt) dvt[i] = (T)(dv * a.inv_n2);
  }
}

// ---------------------------------------------------- sphere <-> grid (a1, a8) --

template <typename T>
__global__ void k_s2g_scatter(GridArgs g) {
  using C = cplx<T>;
  const long long total = (long long)g.nb * g.npw;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const int b = (int)(i / g.npw), ig = (int)(i % g.npw);
    const int* m = g.miller + 3 * ig;
    const int x = m[0] + g.n1, y = m[1] + g.n2, z = m[2] + g.n3;
    if (x < 0 || x >= g.Q1 || y < 0 || y >= g.Q2 || z < 0 || z >= g.Q3) {
      atomicOr(g.err, 1);
      continue;
    }
    const double2 c = g.c[(long long)b * g.npw_max + ig];
    reinterpret_cast<C*>(g.box)[(((long long)b * g.Q3 + z) * g.Q2 + y) * g.Q1 + x] = C{(T)c.x, (T)c.y};
  }
}

// grid (Q2, nb): inverse z transform of box row (b, kyb) into stage[b][z][kyb][:]
template <int N, int NT, typename T>
__global__ void __launch_bounds__(NT) k_s2g_z(GridArgs g) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sZ = tw + N;
  load_twiddles<N, T>(tw, g.tw);
  __syncthreads();
  const int kyb = blockIdx.x, b = blockIdx.y;
  const int Q1 = g.Q1, Q2 = g.Q2, Q3 = g.Q3;
  const C* box = reinterpret_cast<const C*>(g.box) + (long long)b * Q3 * Q2 * Q1 + (long long)kyb * Q1;
  C* st = reinterpret_cast<C*>(g.stage) + (long long)b * N * Q2 * Q1 + (long long)kyb * Q1;
  pencil_inverse<N, NT, T>(
      tw, sZ, Q1, g.n3, [&](int kzb, int c) { return box[(long long)kzb * Q2 * Q1 + c]; },
      [&](int z, int c, C v) { st[(long long)z * Q2 * Q1 + c] = v; });
}

// grid (nb, N): inverse y and x transforms of stage plane (b, z) into u[b][z]
template <int N, int NT, typename T>
__global__ void __launch_bounds__(NT) k_s2g_xy(GridArgs g) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sA = tw + N;
  load_twiddles<N, T>(tw, g.tw);
  __syncthreads();
  const int b = blockIdx.x, z = blockIdx.y;
  const int Q1 = g.Q1, Q2 = g.Q2;
  const C* st = reinterpret_cast<const C*>(g.stage) + ((long long)b * N + z) * Q2 * Q1;
  C* u = reinterpret_cast<C*>(g.u) + (long long)b * N * N * N + (long long)z * N * N;
  const T sc = (T)g.scale;
  plane_inverse<N, NT, T>(
      tw, sA, g.n1, Q1, g.n2, [&](int kyb, int kxb) { return st[kyb * Q1 + kxb]; },
      [&](int, int, int y, int x, C v) { u[y * N + x] = sc * v; });
}

// grid (nb, N): forward x and y transforms of FP64 grid plane (b, z) into stage
template <int N, int NT>
__global__ void __launch_bounds__(NT) k_g2s_xy(GridArgs g) {
  using C = double2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sA = tw + N;
  load_twiddles<N, double>(tw, g.tw);
  __syncthreads();
  const int b = blockIdx.x, z = blockIdx.y;
  const int Q1 = g.Q1;
  const C* f = g.f + (long long)b * N * N * N + (long long)z * N * N;
  C* st = reinterpret_cast<C*>(g.stage) + ((long long)b * N + z) * g.Q2 * Q1;
  plane_forward<N, NT, double>(
      tw, sA, g.n1, Q1, g.n2, [&](int y, int x) { return f[y * N + x]; },
      [&](int kyb, int kxb, C v) { st[kyb * Q1 + kxb] = v; });
}

// grid (Q2, nb): forward z transform of stage row (b, kyb) into box
template <int N, int NT>
__global__ void __launch_bounds__(NT) k_g2s_z(GridArgs g) {
  using C = double2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sZ = tw + N;
  load_twiddles<N, double>(tw, g.tw);
  __syncthreads();
  const int kyb = blockIdx.x, b = blockIdx.y;
  const int Q1 = g.Q1, Q2 = g.Q2, Q3 = g.Q3;
  const C* st = reinterpret_cast<const C*>(g.stage) + (long long)b * N * Q2 * Q1 + (long long)kyb * Q1;
  C* box = reinterpret_cast<C*>(g.box) + (long long)b * Q3 * Q2 * Q1 + (long long)kyb * Q1;
  pencil_forward<N, NT, double>(
      tw, sZ, Q1, g.n3, [&](int z, int c) { return st[(long long)z * Q2 * Q1 + c]; },
      [&](int kzb, int c, C v) { box[(long long)kzb * Q2 * Q1 + c] = v; });
}

// out[b][g] = scale * box[b][m3][m2][m1] on the sphere, zero padding beyond npw
__global__ void k_g2s_gather(GridArgs g);

}  // namespace xx
