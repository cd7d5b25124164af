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
//   pass B  one (pair, f_y) row per CTA, or per item of a persistent CTA whose
//           rows arrive by tensor copies: forward z FFT, multiply by the
//           kernel table, inverse z FFT, in place;
//   pass C  one z-plane per CTA: inverse y and x FFTs, multiply by u_qj and
//           accumulate over the occupied batch in registers, then add into the
//           FP64 accumulator of the target.
// Around them: sphere->grid (scatter + inverse FFT) once per orbital, the
// kernel table once per (k, q), grid->sphere (FFT + gather) once per target,
// and fixed-order reductions for E_x and dE_x/dmu.
#pragma once

#include <cuda.h>   // CUtensorMap (the tensor map itself is encoded on the host)

#include "xx_fft.cuh"

namespace xx {

// ------------------------------------------------------------- arguments --

struct PairArgs {
  const void* u_tgt;     // [TA][N^3] grids of the target batch (at k)
  const void* u_occ;     // [TJ][N^3] grids of the occupied batch (at q)
  void* inter;           // [TA*TJ][N][P2][LX] pair intermediates (kept f_x < P1 of each row)
  const void* vt;        // [P3][P2][P1] v(k-q+G)/N   (pass B)
  const void* dvt;       // [P3][P2][P1] dv/dmu/N^2   (pass B, mu-gradient)
  double2* acc;          // [TA][N^3] FP64 accumulators of the target batch
  const double* w_occ;   // [TJ] occupations of the occupied batch
  const double* w_tgt;   // [TA] occupations of the target batch
  const double2* w_pair; // [TJ] (w_2p, w_2p+1) of packed occupied slots (real orbitals)
  double* partial;       // [TA*TJ][P2] mu-gradient partial sums
  const void* tw;        // [N] exp(-2 pi i e / N) in the pass precision (x, y: plane passes)
  const void* twz;       // [nz] exp(-2 pi i e / nz) (z: pencil passes)
  int nz;                // z-planes of a grid (N3); the grid is N x N x nz
  long long u_tgt_stride;  // elements between consecutive target grids
  long long u_occ_stride;  // elements between consecutive occupied grids
  int TA, TJ;
  int h1, h2, h3, P1, P2, P3;
  int LX;                // row pitch of the intermediates (>= P1; even in FP32, so a row
                         // is a whole number of 16-byte units)
  double coef;           // -1 / N_q
  int* err;              // device error flag (bit 2: a tensor-copy wait ran out)
  int stage_a;           // FP32 pass A: occupied planes by bulk copies into shared memory
  int test_wait_expiry;  // tests only: announce the first pass-B copy of each CTA 16
                         // bytes longer than it is, so its bounded wait runs out
  // The occupied batch may span several q-points (their grids, occupations and
  // accumulators laid out contiguously by the caller): column tj belongs to
  // q-point segment tj / nj, whose kernel table starts vt_seg values after the
  // previous one (one segment when nj >= TJ).
  int nj;
  long long vt_seg;
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
  const void* tw;        // x, y twiddles (plane kernels)
  const void* twz;       // z twiddles (pencil kernels)
  int nz;                // z-planes of a grid (N3)
  int n1, n2, n3, Q1, Q2, Q3;
  double scale;
  int* err;
};

struct VtabArgs {
  double Bm[9];          // reciprocal rows b_i (Cartesian), for the strain tables
  double M[9];           // reciprocal metric b_i . b_j
  double d[3];           // k - q (fractional)
  int h1, h2, h3, P1, P2, P3;
  int kernel;            // 0 screened, 1 Coulomb (g = 0 dropped)
  double mu;
  double inv_n, inv_n2;  // 1/N, 1/N^2
};

// ---------------------------------------------------- CTA building blocks --
//
// Shared-memory layout of a plane (N rows of LD complex values): between the
// two steps of the x transform, row y holds slot k1*S + n2 (S >= B); the x
// transform's output and the y transform's data sit at natural positions
// (row y, column x or f_x).  S and LD are chosen per N by csrc/bank_layout.py,
// which counts the wavefronts of 8-byte accesses in half-warp phases over every
// S in [B, B + 16] and LD in [N, N + 40]: the x steps replay 1.0x at N = 32, 36, 96,
// at most 1.2x at N = 24, 60, 72, 1.34x at N = 108 and 1.5x at N = 40, 48, 54, 64, 80.
// The y steps
// (lanes over kept columns) are conflict-free when 16 divides N; otherwise the
// wrap from column N - 1 to column 0 replays up to 2x in one half-warp.
// FP32 planes use two buffers (the x-step exchange goes from one to the
// other); FP64 planes use one buffer and hold a step's outputs in registers
// across a barrier.

template <int N> struct Lay;
template <> struct Lay<24> { static constexpr int A = 8, B = 3, S = 4, LD = 35; };
template <> struct Lay<32> { static constexpr int A = 8, B = 4, S = 5, LD = 44; };
template <> struct Lay<36> { static constexpr int A = 6, B = 6, S = 9, LD = 54; };
template <> struct Lay<40> { static constexpr int A = 8, B = 5, S = 5, LD = 44; };
template <> struct Lay<48> { static constexpr int A = 8, B = 6, S = 7, LD = 60; };
template <> struct Lay<54> { static constexpr int A = 6, B = 9, S = 9, LD = 54; };
template <> struct Lay<60> { static constexpr int A = 6, B = 10, S = 15, LD = 90; };
template <> struct Lay<64> { static constexpr int A = 8, B = 8, S = 9, LD = 76; };
template <> struct Lay<72> { static constexpr int A = 8, B = 9, S = 12, LD = 105; };
template <> struct Lay<80> { static constexpr int A = 8, B = 10, S = 11, LD = 92; };
template <> struct Lay<96> { static constexpr int A = 8, B = 12, S = 13, LD = 108; };
template <> struct Lay<108> { static constexpr int A = 6, B = 18, S = 19, LD = 114; };

constexpr int gcd_c(int a, int b) { return b == 0 ? a : gcd_c(b, a % b); }
constexpr int lcm_c(int a, int b) { return a / gcd_c(a, b) * b; }
constexpr int round_up(int x, int m) { return (x + m - 1) / m * m; }

// DB: two plane buffers and one second-step item per thread; otherwise one
// buffer, half as many threads (a multiple of B, and of A when A != 8, so every
// iteration covers whole rows) and register holds across barriers.  The
// default is two buffers for FP32 (pass C keeps its accumulator in registers)
// and one for FP64 (two FP64 buffers exceed shared memory).
// NT_ > 0 overrides the thread count (the one-buffer variant then needs it to be a
// multiple of 32, of B and, when A != 8, of A).
template <int N, typename T, bool DB_ = (sizeof(T) == 4), int NT_ = 0> struct PlaneCfg {
  static constexpr int A = Lay<N>::A, B = Lay<N>::B, S = Lay<N>::S, LD = Lay<N>::LD;
  static constexpr bool DB = DB_;
  static constexpr int NT = NT_ > 0 ? NT_
                            : DB ? round_up(N * A, 32)
                                 : round_up(N * A / 2, lcm_c(lcm_c(32, B), A == 8 ? 1 : A));
  static constexpr int NW = NT / 32;
  static constexpr bool REG_TW = (NT % B) == 0;                    // thread's x-step n2 fixed
  static constexpr int X1_IT = (N * B + NT - 1) / NT;
  static constexpr int X2_IT = (N * A + NT - 1) / NT;
  static constexpr int BUF = N * LD;                               // elements per buffer
  // the one-buffer variant holds one iteration's outputs across a barrier,
  // which is only safe when every iteration covers whole rows
  static_assert(DB || (NT % B == 0 && NT % 32 == 0 && (A == 8 || NT % A == 0)),
                "register hold needs whole rows per iteration");
  static_assert(NT <= 1024, "too many threads");
  // twiddles (N) + [k1][n2] twiddle table (N) + plane buffer(s)
  static constexpr size_t smem() { return sizeof(cplx<T>) * ((size_t)2 * N + (size_t)BUF * (DB ? 2 : 1)); }
};

struct NoHook {
  __device__ __forceinline__ void operator()() const {}
};

// Barrier among the first NT threads of the CTA (barrier 0 with a thread
// count).  Every building block below synchronises with it, so a transform of
// NT threads can run inside a larger CTA whose other threads have left (the
// batched launches over cells of different grid lengths); with NT equal to the
// block size it is the ordinary CTA barrier.
template <int NT> __device__ __forceinline__ void bsync() {
  static_assert(NT % 32 == 0, "barriers count whole warps");
  asm volatile("bar.sync 0, %0;" ::"n"(NT) : "memory");
}

// Cooperative L1 prefetch of [p, p + bytes): one 128-byte line per thread.
__device__ __forceinline__ void prefetch_l1(const void* p, long long bytes) {
  const long long line = (long long)threadIdx.x * 128;
  if (line < bytes) asm volatile("prefetch.global.L1 [%0];" ::"l"((const char*)p + line));
}

// The same over the first NT threads, each taking every NT-th line.
template <int NT> __device__ __forceinline__ void prefetch_l1_all(const void* p, long long bytes) {
  for (long long line = (long long)threadIdx.x * 128; line < bytes; line += (long long)NT * 128)
    asm volatile("prefetch.global.L1 [%0];" ::"l"((const char*)p + line));
}

// Second x step item -> (k1, row).  For A = 8 each half-warp covers four k1
// values of four consecutive rows (the conflict-free pattern for slot stride S).
template <int A> __device__ __forceinline__ void x2_item(int it, int& k1, int& row) {
  if constexpr (A == 8) {
    const int l = it & 31, w = it >> 5;
    k1 = (l & 3) | ((l >> 4) << 2);
    row = 4 * w + ((l >> 2) & 3);
  } else {
    k1 = it % A;
    row = it / A;
  }
}

// Forward x then y transform of one real-space plane; outputs only the kept
// frequencies |f_x| <= h1, |f_y| <= h2 through store(kyb, kxb, value).
// s0 (and s1 when double-buffered) are the plane buffers.
// after_x1() runs on every thread right after the barrier that ends the first x
// step (the last use of load); before_end() right before the final barrier.
// NTO overrides the thread count of PlaneCfg (0: its default).
template <int N, typename T, bool DB, int NTO = 0, typename Load, typename Store, typename AfterX1 = NoHook,
          typename BeforeEnd = NoHook>
__device__ __forceinline__ void plane_forward(const cplx<T>* tw, cplx<T>* s0, cplx<T>* s1, int h1,
                                              int P1, int h2, Load load, Store store,
                                              AfterX1 after_x1 = AfterX1(), BeforeEnd before_end = BeforeEnd()) {
  using C = cplx<T>;
  using G = PlaneCfg<N, T, DB, NTO>;
  constexpr int A = G::A, B = G::B, S = G::S, LD = G::LD, NT = G::NT, NW = G::NW;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  C* sy = G::DB ? s1 : s0;   // buffer of the natural-order plane
  C twr[A];
  if constexpr (G::REG_TW) {
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) twr[k1] = tw[(t % B) * k1];
  }
  // x, step 1: codensity in, length-A DFTs over stride-B subsequences
#pragma unroll
  for (int i = 0; i < G::X1_IT; ++i) {
    const int it = t + i * NT;
    if (it < N * B) {
      const int n2 = it % B, y = it / B;
      C r[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) r[n1] = load(y, B * n1 + n2);
      dft<A, false>(r);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1)
        s0[y * LD + k1 * S + n2] = tw_mul<false>(r[k1], G::REG_TW ? twr[k1] : tw[n2 * k1], k1);
    }
  }
  bsync<NT>();
  after_x1();
  // x, step 2: length-B DFTs, output at natural f_x positions
  if constexpr (G::DB) {
#pragma unroll
    for (int i = 0; i < G::X2_IT; ++i) {
      const int it = t + i * NT;
      if (it < N * A) {
        int k1, row;
        x2_item<A>(it, k1, row);
        C r[B];
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) r[n2] = s0[row * LD + k1 * S + n2];
        dft<B, false>(r);
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) sy[row * LD + k1 + A * k2] = r[k2];
      }
    }
  } else {
    // one buffer: each iteration covers whole rows (NT is a multiple of 4 rows
    // of A items), so its outputs are held in registers across one barrier
#pragma unroll
    for (int i = 0; i < G::X2_IT; ++i) {
      const int it = t + i * NT;
      int k1 = 0, row = 0;
      C hold[B];
      if (it < N * A) {
        x2_item<A>(it, k1, row);
#pragma unroll
        for (int n2 = 0; n2 < B; ++n2) hold[n2] = s0[row * LD + k1 * S + n2];
        dft<B, false>(hold);
      }
      bsync<NT>();
      if (it < N * A) {
#pragma unroll
        for (int k2 = 0; k2 < B; ++k2) sy[row * LD + k1 + A * k2] = hold[k2];
      }
    }
  }
  bsync<NT>();
  // y, step 1: warp-uniform n2, lanes over kept f_x columns; in place
  const int nkb = (P1 + 31) >> 5;
#pragma unroll 1
  for (int u = warp; u < B * nkb; u += NW) {
    const int n2 = u % B, kxb = lane + 32 * (u / B);
    if (kxb < P1) {
      const int fx = idx_of_box(kxb, N, h1);
      C r[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) r[n1] = sy[(B * n1 + n2) * LD + fx];
      dft<A, false>(r);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) sy[(k1 * B + n2) * LD + fx] = tw_mul<false>(r[k1], tw[n2 * k1], k1);
    }
  }
  bsync<NT>();
  // y, step 2: warp-uniform k1; kept f_y go to store
#pragma unroll 1
  for (int u = warp; u < A * nkb; u += NW) {
    const int k1 = u % A, kxb = lane + 32 * (u / A);
    if (kxb < P1) {
      const int fx = idx_of_box(kxb, N, h1);
      C r[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) r[n2] = sy[(k1 * B + n2) * LD + fx];
      dft<B, false>(r);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) {
        const int k = k1 + A * k2;
        if (kept(k, N, h2)) store(box_of(k, N, h2), kxb, r[k2]);
      }
    }
  }
  before_end();
  bsync<NT>();
}

// Inverse y then x transform from kept frequencies (load(kyb, kxb)) to the
// full real-space plane.  Every output goes to consume(i, k2, y, x, value),
// where (i, k2) is a compile-time register slot of the calling thread (fixed
// across calls).  After the y transform, row y = k1 + A*k2 sits in row
// k1*B + k2 of the natural-order buffer.
// tw2 is the [k1][n2] table of W_N^(n2*k1) (make_twiddles2), read by the x
// step whenever its twiddles are not kept in registers; callers always pass it.
template <int N, typename T, bool TWREG, typename Load, typename Consume>
__device__ __forceinline__ void plane_inverse(const cplx<T>* tw, const cplx<T>* tw2, cplx<T>* s0,
                                              cplx<T>* s1, int h1, int P1, int h2, Load load,
                                              Consume consume, const void* pf_x = nullptr,
                                              long long pf_x_bytes = 0, const void* pf_next = nullptr,
                                              long long pf_next_bytes = 0) {
  using C = cplx<T>;
  using G = PlaneCfg<N, T>;
  constexpr int A = G::A, B = G::B, S = G::S, LD = G::LD, NT = G::NT, NW = G::NW;
  constexpr bool REG = TWREG && G::REG_TW;
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  C* sx = G::DB ? s1 : s0;   // buffer of the slot-order x exchange
  C twr[REG ? A : 1];
  if constexpr (REG) {
#pragma unroll
    for (int k1 = 0; k1 < A; ++k1) twr[k1] = tw[(t % B) * k1];
  }
  const int nkb = (P1 + 31) >> 5;
  // y, step 1: kept f_y in, warp-uniform n2, lanes over kept f_x
#pragma unroll 1
  for (int u = warp; u < B * nkb; u += NW) {
    const int n2 = u % B, kxb = lane + 32 * (u / B);
    if (kxb < P1) {
      const int xm = idx_of_box(kxb, N, h1);
      C r[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) {
        const int m = B * n1 + n2;
        r[n1] = kept(m, N, h2) ? load(box_of(m, N, h2), kxb) : czero<C>();
      }
      dft<A, true>(r);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) s0[(k1 * B + n2) * LD + xm] = tw_mul<true>(r[k1], tw[n2 * k1], k1);
    }
  }
  bsync<NT>();
  // y, step 2: warp-uniform k1, in place (row y = k1 + A*k2 lands in row k1*B + k2)
#pragma unroll 1
  for (int u = warp; u < A * nkb; u += NW) {
    const int k1 = u % A, kxb = lane + 32 * (u / A);
    if (kxb < P1) {
      const int xm = idx_of_box(kxb, N, h1);
      C r[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) r[n2] = s0[(k1 * B + n2) * LD + xm];
      dft<B, true>(r);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) s0[(k1 * B + k2) * LD + xm] = r[k2];
    }
  }
  bsync<NT>();
  // optional L1 prefetch of what the last step reads (pass C: the u_j plane)
  if (pf_x) prefetch_l1(pf_x, pf_x_bytes);
  // x, step 1: kept f_x of every row in, slot-order out
  if constexpr (G::DB) {
#pragma unroll
    for (int i = 0; i < G::X1_IT; ++i) {
      const int it = t + i * NT;
      if (it < N * B) {
        const int n2 = it % B, row = it / B;
        C r[A];
#pragma unroll
        for (int n1 = 0; n1 < A; ++n1) {
          const int m = B * n1 + n2;
          r[n1] = kept(m, N, h1) ? s0[row * LD + m] : czero<C>();
        }
        dft<A, true>(r);
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
          C w;
          if constexpr (REG) w = twr[k1]; else w = tw2[k1 * B + n2];
          sx[row * LD + k1 * S + n2] = tw_mul<true>(r[k1], w, k1);
        }
      }
    }
  } else {
    // one buffer: each iteration covers whole rows (NT is a multiple of B), so
    // its outputs are held in registers across one barrier
#pragma unroll
    for (int i = 0; i < G::X1_IT; ++i) {
      const int it = t + i * NT;
      const int n2 = it % B, row = it / B;
      C hold[A];
      if (it < N * B) {
#pragma unroll
        for (int n1 = 0; n1 < A; ++n1) {
          const int m = B * n1 + n2;
          hold[n1] = kept(m, N, h1) ? s0[row * LD + m] : czero<C>();
        }
        dft<A, true>(hold);
      }
      bsync<NT>();
      if (it < N * B) {
#pragma unroll
        for (int k1 = 0; k1 < A; ++k1) {
          C w;
          if constexpr (REG) w = twr[k1]; else w = tw2[k1 * B + n2];
          sx[row * LD + k1 * S + n2] = tw_mul<true>(hold[k1], w, k1);
        }
      }
    }
  }
  bsync<NT>();
  // optional L1 prefetch of the next call's input (pass C: the next plane)
  if (pf_next) prefetch_l1(pf_next, pf_next_bytes);
  // x, step 2: every output to consume
#pragma unroll
  for (int i = 0; i < G::X2_IT; ++i) {
    const int it = t + i * NT;
    if (it < N * A) {
      int k1, row;
      x2_item<A>(it, k1, row);
      const int y = row / B + A * (row % B);
      C r[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) r[n2] = sx[row * LD + k1 * S + n2];
      dft<B, true>(r);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) consume(i, k2, y, k1 + A * k2, r[k2]);
    }
  }
  bsync<NT>();
}

// Forward z transform of a row of W pencils: load(z, c) real space,
// out(kzb, c, value) for the kept |f_z| <= h3.  Warp-uniform n2 / k1, lanes
// over c, so shared accesses are bank-conflict free and twiddles broadcast.
// sZ holds N rows of pitch ld (0: W).  Step 1 reads and writes the same rows
// of a column, so load may read sZ itself (an in-place transform).
template <int N, int NT, typename T, typename Load, typename Out>
__device__ __forceinline__ void pencil_forward(const cplx<T>* tw, cplx<T>* sZ, int W, int h3,
                                              Load load, Out out, int ld = 0) {
  using C = cplx<T>;
  constexpr int A = Lay<N>::A, B = Lay<N>::B, NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncb = (W + 31) >> 5;
  if (ld <= 0) ld = W;
#pragma unroll 1
  for (int u = warp; u < B * ncb; u += NW) {
    const int n2 = u % B, c = lane + 32 * (u / B);
    if (c < W) {
      C r[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) r[n1] = load(B * n1 + n2, c);
      dft<A, false>(r);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) sZ[(k1 * B + n2) * ld + c] = tw_mul<false>(r[k1], tw[n2 * k1], k1);
    }
  }
  bsync<NT>();
#pragma unroll 1
  for (int u = warp; u < A * ncb; u += NW) {
    const int k1 = u % A, c = lane + 32 * (u / A);
    if (c < W) {
      C r[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) r[n2] = sZ[(k1 * B + n2) * ld + c];
      dft<B, false>(r);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) {
        const int k = k1 + A * k2;
        if (kept(k, N, h3)) out(box_of(k, N, h3), c, r[k2]);
      }
    }
  }
}

// Inverse z transform of a row of W pencils from kept frequencies
// load(kzb, c) to real space store(z, c, value); sZ rows of pitch ld (0: W).
template <int N, int NT, typename T, typename Load, typename Store>
__device__ __forceinline__ void pencil_inverse(const cplx<T>* tw, cplx<T>* sZ, int W, int h3,
                                              Load load, Store store, int ld = 0) {
  using C = cplx<T>;
  constexpr int A = Lay<N>::A, B = Lay<N>::B, NW = NT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int ncb = (W + 31) >> 5;
  if (ld <= 0) ld = W;
#pragma unroll 1
  for (int u = warp; u < B * ncb; u += NW) {
    const int n2 = u % B, c = lane + 32 * (u / B);
    if (c < W) {
      C r[A];
#pragma unroll
      for (int n1 = 0; n1 < A; ++n1) {
        const int m = B * n1 + n2;
        r[n1] = kept(m, N, h3) ? load(box_of(m, N, h3), c) : czero<C>();
      }
      dft<A, true>(r);
#pragma unroll
      for (int k1 = 0; k1 < A; ++k1) sZ[(k1 * B + n2) * ld + c] = tw_mul<true>(r[k1], tw[n2 * k1], k1);
    }
  }
  bsync<NT>();
#pragma unroll 1
  for (int u = warp; u < A * ncb; u += NW) {
    const int k1 = u % A, c = lane + 32 * (u / A);
    if (c < W) {
      C r[B];
#pragma unroll
      for (int n2 = 0; n2 < B; ++n2) r[n2] = sZ[(k1 * B + n2) * ld + c];
      dft<B, true>(r);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) store(k1 + A * k2, c, r[k2]);
    }
  }
}

// NT > 0: only the first NT threads take part (stride NT); 0: the whole block
template <int N, typename T, int NT = 0>
__device__ __forceinline__ void load_twiddles(cplx<T>* dst, const void* src) {
  const int stride = NT > 0 ? NT : (int)blockDim.x;
  for (int i = threadIdx.x; i < N; i += stride) dst[i] = ((const cplx<T>*)src)[i];
}

// tw2[k1 * B + n2] = tw[n2 * k1] (call after load_twiddles and a barrier)
template <int N, typename T, int NT = 0>
__device__ __forceinline__ void make_twiddles2(cplx<T>* tw2, const cplx<T>* tw) {
  constexpr int A = Lay<N>::A, B = Lay<N>::B;
  const int stride = NT > 0 ? NT : (int)blockDim.x;
  for (int i = threadIdx.x; i < A * B; i += stride) tw2[i] = tw[(i % B) * (i / B)];
}

template <int N, typename T> constexpr size_t smem_pencil(int W, int P3) {
  return sizeof(cplx<T>) * ((size_t)N + (size_t)N * W + (size_t)P3 * W);
}

// ------------------------------------------------------------- the passes --

// Pass A: grid (TA, N); CTA (ta, z) loops over the TJ occupied bands.  One
// plane buffer, so two CTAs share an SM and overlap each other's barriers.
// The body takes its CTA's (ta, z) and its shared memory from the caller, so
// the batched launch over several cells (k_pass_a_cells) runs the same code.
// DB = true: the two-buffer plane (more threads per plane, no register holds;
// the batched launches use it at N = 60, whose one-buffer plane needs 480 threads).
template <int N, typename T> using PassACfg = PlaneCfg<N, T, false>;
template <int N, typename T, bool DB = false>
__device__ __forceinline__ void pass_a_body(const PairArgs& p, int ta, int z, unsigned char* smem_raw) {
  using C = cplx<T>;
  using G = PlaneCfg<N, T, DB>;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s0 = tw + N;
  C* s1 = s0 + G::BUF;
  load_twiddles<N, T, G::NT>(tw, p.tw);
  bsync<G::NT>();
  constexpr long long plane = (long long)N * N;
  const C* ua = reinterpret_cast<const C*>(p.u_tgt) + ta * p.u_tgt_stride + z * plane;
  const int LX = p.LX;
#pragma unroll 1
  for (int tj = 0; tj < p.TJ; ++tj) {
    const C* uj = reinterpret_cast<const C*>(p.u_occ) + tj * p.u_occ_stride + z * plane;
    const C* uj_next = tj + 1 < p.TJ ? uj + p.u_occ_stride : nullptr;
    C* out = reinterpret_cast<C*>(p.inter) +
             ((long long)(ta * p.TJ + tj) * p.nz + z) * (long long)p.P2 * LX;
    // once the first x step has read this band's plane, the next band's plane is
    // prefetched into L1 (measured on GB300 at 96^3: pass A 15.2 -> 13.4 ms per
    // 64 x 80 launch)
    plane_forward<N, T, DB>(
        tw, s0, s1, p.h1, p.P1, p.h2,
        [&](int y, int x) { return cmulc(uj[y * N + x], ua[y * N + x]); },
        [&](int kyb, int kxb, C v) { out[kyb * LX + kxb] = v; },
        [&] { if (uj_next) prefetch_l1_all<G::NT>(uj_next, plane * (long long)sizeof(C)); });
  }
}
template <int N, typename T>
__global__ void __launch_bounds__(PassACfg<N, T>::NT, sizeof(T) == 4 ? 2 : 1) k_pass_a(PairArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_a_body<N, T>(p, blockIdx.x, blockIdx.y, smem_raw);
}

// Pass B: grid (P2, TA*TJ); CTA (kyb, pair) transforms its row along z,
// multiplies by v(k - q + G)/N and transforms back, in place.
template <int N, int NT, typename T>
__device__ __forceinline__ void pass_b_body(const PairArgs& p, int kyb, int pair, unsigned char* smem_raw) {
  using C = cplx<T>;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sZ = tw + N;
  C* sK = sZ + N * p.P1;
  load_twiddles<N, T, NT>(tw, p.twz);
  bsync<NT>();
  const int P1 = p.P1, P2 = p.P2;
  const int zstride = P2 * p.LX;               // a pair's planes stay within 32-bit offsets
  C* row = reinterpret_cast<C*>(p.inter) + (long long)pair * N * zstride + kyb * p.LX;
  const T* vt = reinterpret_cast<const T*>(p.vt) + (long long)((pair % p.TJ) / p.nj) * p.vt_seg + kyb * P1;
  pencil_forward<N, NT, T>(
      tw, sZ, P1, p.h3, [&](int z, int c) { return row[z * zstride + c]; },
      [&](int kzb, int c, C v) {
        const T s = vt[kzb * (P2 * P1) + c];
        sK[kzb * P1 + c] = s * v;
      });
  bsync<NT>();
  pencil_inverse<N, NT, T>(
      tw, sZ, P1, p.h3, [&](int kzb, int c) { return sK[kzb * P1 + c]; },
      [&](int z, int c, C v) { row[z * zstride + c] = v; });
}
template <int N, int NT, typename T>
__global__ void __launch_bounds__(NT, sizeof(T) == 4 ? 3 : 1) k_pass_b(PairArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_b_body<N, NT, T>(p, blockIdx.x, blockIdx.y, smem_raw);
}
// --------------------------------------------- tensor-copy staged pass B --
//
// Bulk tensor copies (TMA) with mbarrier completion.  Every wait on an mbarrier
// is bounded: after kMbarLimitNs of unsuccessful polls (global timer) the caller
// sets an error flag and leaves instead of spinning forever.

constexpr unsigned long long kMbarLimitNs = 2000000000ull;   // 2 s

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned smem_addr(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// makes the initialised barriers visible to the tensor-copy unit
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
               : "memory");
}

// true once the phase with the given parity has completed; false when it has
// not completed kMbarLimitNs after the first unsuccessful poll
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, unsigned parity) {
  const unsigned a = smem_addr(bar);
  unsigned long long t0 = 0;
  for (;;) {
    unsigned done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
    const unsigned long long now = global_ns();
    if (t0 == 0)
      t0 = now;
    else if (now - t0 > kMbarLimitNs)
      return false;
  }
}

// orders this thread's earlier shared-memory accesses before later tensor copies
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 3-D tile load global -> shared, completion counted in bytes on bar
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* tm, int c0, int c1, int c2,
                                            uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_addr(dst)),
      "l"(tm), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
      : "memory");
}

// contiguous global -> shared bulk copy (16-byte aligned ends), completion on bar
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_addr(dst)),
      "l"(src), "r"(bytes), "r"(smem_addr(bar))
      : "memory");
}

// Shared staging of one contiguous plane per loop step (pass A: the occupied
// orbital's plane z): the plane of step s + 1 is copied in by one bulk copy
// issued as soon as step s has read its plane, and waited for before step s
// ends.  All waits are bounded; a wait that runs out makes every thread leave
// (ok == 0).
struct PlaneStage {
  uint64_t* bar;
  int* ok;
  void* buf;
  unsigned bytes;
  __device__ __forceinline__ void start(const void* first) {
    if (threadIdx.x == 0) {
      mbar_init(bar, 1);
      mbar_init_fence();
      mbar_arrive_expect_tx(bar, bytes);
      bulk_load(buf, first, bytes, bar);
      *ok = mbar_wait(bar, 0) ? 1 : 0;
    }
    __syncthreads();
  }
  // start of step s: false (on every thread) when the copy never completed
  __device__ __forceinline__ bool ready(int s) {
    if (!*ok) {
      if (threadIdx.x == 0) atomicOr(err_flag, 2);
      return false;
    }
    mbar_wait(bar, (unsigned)(s & 1));   // completes at once; publishes the bytes
    return true;
  }
  __device__ __forceinline__ void issue(const void* next) {
    if (threadIdx.x == 0 && next) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(bar, bytes);
      bulk_load(buf, next, bytes, bar);
    }
  }
  __device__ __forceinline__ void wait_next(int s, bool has_next) {
    if (threadIdx.x == 0 && has_next) *ok = mbar_wait(bar, (unsigned)((s + 1) & 1)) ? 1 : 0;
  }
  int* err_flag;
};

// Pass B, FP32, persistent and tensor-copy staged: item i = (pair i / P2, row
// kyb = i % P2).  The row's N z-planes x LX values arrive by one 3-D tensor copy
// (tm views the intermediates as [N * pairs][P2][2 LX] floats) into one of two
// shared buffers, issued two items ahead, so the copy of the next row overlaps
// this row's transforms.  The forward z step 1 runs in place in the buffer,
// step 2 writes the kept f_z times v(k - q + G)/N to sK, the inverse step 1
// writes back into the buffer and step 2 stores the row to global memory.
// Tensor-copy destinations must be 128-byte aligned: the buffers start at the
// first 128-byte boundary of the dynamic shared memory (the launch adds 128
// bytes of slack) and each spans a multiple of 128 bytes.
template <int N> __host__ __device__ constexpr int pass_b_tma_buf_elems(int LX) {
  return (N * LX + 15) / 16 * 16;   // float2 elements, a multiple of 128 bytes
}

template <int N, int NT>
__global__ void __launch_bounds__(NT, 2) k_pass_b_tma(const __grid_constant__ CUtensorMap tm, PairArgs p,
                                                      int n_items) {
  using C = float2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar[2];
  __shared__ int ok;
  const int LX = p.LX, P1 = p.P1, P2 = p.P2;
  const unsigned pad = (128u - (smem_addr(smem_raw) & 127u)) & 127u;
  C* buf0 = reinterpret_cast<C*>(smem_raw + pad);
  const int BUF = pass_b_tma_buf_elems<N>(LX);
  C* sK = buf0 + 2 * BUF;
  const C* tw = reinterpret_cast<const C*>(p.twz);
  const unsigned bytes = (unsigned)(N * LX * sizeof(C));
  const int G = gridDim.x;
  const int zstride = P2 * LX;
  // uniform across the block: never issue a copy to a misaligned buffer
  if ((smem_addr(buf0) & 127u) != 0u || ((BUF * sizeof(C)) & 127u) != 0u) {
    if (threadIdx.x == 0) atomicOr(p.err, 2);
    return;
  }
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init_fence();
    for (int b = 0; b < 2; ++b) {
      const int item = blockIdx.x + b * G;
      if (item < n_items) {
        mbar_arrive_expect_tx(&bar[b], bytes + (b == 0 && p.test_wait_expiry ? 16u : 0u));
        tma_load_3d(buf0 + b * BUF, &tm, 0, item % P2, (item / P2) * N, &bar[b]);
      }
    }
    // one thread decides whether each row arrived, before the barrier that
    // starts the row, so the whole block takes the same branch
    ok = mbar_wait(&bar[0], 0) ? 1 : 0;
  }
  __syncthreads();
  int it = 0;
  for (int item = blockIdx.x; item < n_items; item += G, ++it) {
    const int b = it & 1;
    C* X = buf0 + b * BUF;
    if (!ok) {
      // the copy never completed: flag it, give the other buffer's copy (if
      // any) its bounded wait, and leave
      if (threadIdx.x == 0) {
        atomicOr(p.err, 2);
        if (item + G < n_items) mbar_wait(&bar[b ^ 1], ((it + 1) >> 1) & 1);
      }
      return;
    }
    // completes at once: makes the copied bytes visible to every thread
    mbar_wait(&bar[b], (it >> 1) & 1);
    const int kyb = item % P2, pair = item / P2;
    const float* vt =
        reinterpret_cast<const float*>(p.vt) + (long long)((pair % p.TJ) / p.nj) * p.vt_seg + kyb * P1;
    pencil_forward<N, NT, float>(
        tw, X, P1, p.h3, [&](int z, int c) { return X[z * LX + c]; },
        [&](int kzb, int c, C v) { sK[kzb * P1 + c] = vt[kzb * (P2 * P1) + c] * v; }, LX);
    __syncthreads();
    C* row = reinterpret_cast<C*>(p.inter) + (long long)pair * N * zstride + kyb * LX;
    pencil_inverse<N, NT, float>(
        tw, X, P1, p.h3, [&](int kzb, int c) { return sK[kzb * P1 + c]; },
        [&](int z, int c, C v) { row[z * zstride + c] = v; }, LX);
    // the next row's copy was issued two rows ago: wait for it before the
    // barrier (bounded), so the barrier both frees X and publishes the decision
    if (threadIdx.x == 0 && item + G < n_items) ok = mbar_wait(&bar[b ^ 1], ((it + 1) >> 1) & 1) ? 1 : 0;
    __syncthreads();   // every read of X and sK is done
    const int next = item + 2 * G;
    if (threadIdx.x == 0 && next < n_items) {
      fence_proxy_async_smem();
      mbar_arrive_expect_tx(&bar[b], bytes);
      tma_load_3d(X, &tm, 0, next % P2, (next / P2) * N, &bar[b]);
    }
  }
}

// dynamic shared memory of k_pass_b_tma: 128 bytes of alignment slack, two
// row buffers, the kept-f_z block
template <int N> constexpr size_t smem_pass_b_tma(int LX, int P1, int P3) {
  return 128 + sizeof(float2) * ((size_t)2 * pass_b_tma_buf_elems<N>(LX) + (size_t)P3 * P1);
}

// Pass A, FP32, with the u_j planes staged: one CTA per SM of
// PassASCfg::NT threads (one x-step item each) and one plane buffer; each
// occupied band's plane z arrives in shared memory by one bulk copy, issued as
// soon as the previous band's plane has been read (after the first x step), so
// only u_a (the same plane for the whole loop, kept in L1) is read from global
// memory.
template <int N> using PassASCfg =
    PlaneCfg<N, float, false, round_up(N * Lay<N>::A, lcm_c(lcm_c(32, Lay<N>::B), Lay<N>::A == 8 ? 1 : Lay<N>::A))>;
template <int N>
__global__ void __launch_bounds__(PassASCfg<N>::NT, 1) k_pass_a_staged(PairArgs p) {
  using C = float2;
  using G = PassASCfg<N>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t bar;
  __shared__ int ok;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s0 = tw + N;
  C* stage = s0 + G::BUF;
  load_twiddles<N, float>(tw, p.tw);
  __syncthreads();
  const int ta = blockIdx.x, z = blockIdx.y;
  constexpr long long plane = (long long)N * N;
  const C* ua = reinterpret_cast<const C*>(p.u_tgt) + ta * p.u_tgt_stride + z * plane;
  const C* uj0 = reinterpret_cast<const C*>(p.u_occ) + z * plane;
  const int LX = p.LX;
  PlaneStage st{&bar, &ok, stage, (unsigned)(plane * sizeof(C)), p.err};
  st.start(uj0);
#pragma unroll 1
  for (int tj = 0; tj < p.TJ; ++tj) {
    C* out = reinterpret_cast<C*>(p.inter) + ((long long)(ta * p.TJ + tj) * p.nz + z) * (long long)p.P2 * LX;
    const bool has_next = tj + 1 < p.TJ;
    const C* next = has_next ? uj0 + (tj + 1) * p.u_occ_stride : nullptr;
    if (!st.ready(tj)) return;
    plane_forward<N, float, false, G::NT>(
        tw, s0, s0, p.h1, p.P1, p.h2, [&](int y, int x) { return cmulc(stage[y * N + x], ua[y * N + x]); },
        [&](int kyb, int kxb, C v) { out[kyb * LX + kxb] = v; }, [&] { st.issue(next); },
        [&] { st.wait_next(tj, has_next); });
  }
}

template <int N> constexpr size_t smem_pass_a_staged() {
  return sizeof(float2) * ((size_t)N + (size_t)PassASCfg<N>::BUF + (size_t)N * N);
}

// Pass B for dE/dmu: forward z only, partial[pair][kyb] = sum dv/dmu/N^2 |rho|^2.
template <int N, int NT, typename T>
__global__ void __launch_bounds__(NT) k_pass_b_dmu(PairArgs p) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sZ = tw + N;
  __shared__ double red[NT];
  load_twiddles<N, T>(tw, p.twz);
  __syncthreads();
  const int kyb = blockIdx.x, pair = blockIdx.y;
  const int P1 = p.P1, P2 = p.P2;
  const long long zstride = (long long)P2 * p.LX;
  const C* row = reinterpret_cast<const C*>(p.inter) + (long long)pair * N * zstride + (long long)kyb * p.LX;
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
// PACKED (real orbitals at Gamma): occupied slot p holds u_2p - i u_2p+1, so W
// holds W_a,2p + i W_a,2p+1 and only the real part is accumulated,
//   acc_a.x += -(1/N_q) (w_2p u_2p W_a,2p + w_2p+1 u_2p+1 W_a,2p+1)
//            = -(1/N_q) (w_2p Re(u) Re(W) - w_2p+1 Im(u) Im(W)).
template <int N, typename T, bool PACKED>
__device__ __forceinline__ void pass_c_body(const PairArgs& p, int ta, int z, unsigned char* smem_raw) {
  using C = cplx<T>;
  using G = PlaneCfg<N, T>;
  constexpr int A = G::A, B = G::B, NT = G::NT;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* tw2 = tw + N;
  C* s0 = tw2 + N;
  C* s1 = s0 + G::BUF;
  load_twiddles<N, T, NT>(tw, p.tw);
  bsync<NT>();
  make_twiddles2<N, T, NT>(tw2, tw);
  bsync<NT>();
  constexpr long long plane = (long long)N * N;
  const int LX = p.LX;
  C acc[G::X2_IT][B];
#pragma unroll
  for (int i = 0; i < G::X2_IT; ++i)
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) acc[i][k2] = czero<C>();
#pragma unroll 1
  for (int tj = 0; tj < p.TJ; ++tj) {
    const C* in = reinterpret_cast<const C*>(p.inter) +
                  ((long long)(ta * p.TJ + tj) * p.nz + z) * (long long)p.P2 * LX;
    const C* uj = reinterpret_cast<const C*>(p.u_occ) + tj * p.u_occ_stride + z * plane;
    T cf, cf2;
    if (PACKED) {
      const double2 w = p.w_pair[tj];
      cf = (T)(p.coef * w.x);
      cf2 = (T)(-p.coef * w.y);
    } else {
      cf = (T)(p.coef * p.w_occ[tj]);
      cf2 = (T)0;
    }
    const long long pbytes = (long long)p.P2 * LX * (long long)sizeof(C);
    const C* next = tj + 1 < p.TJ ? in + (long long)p.nz * p.P2 * LX : nullptr;
    plane_inverse<N, T, false>(
        tw, tw2, s0, s1, p.h1, p.P1, p.h2, [&](int kyb, int kxb) { return in[kyb * LX + kxb]; },
        [&](int i, int k2, int y, int x, C v) {
          const C u = uj[y * N + x];
          if (PACKED) {
            acc[i][k2].x += cf * (u.x * v.x) + cf2 * (u.y * v.y);
          } else {
            const C t = cmul(u, v);
            acc[i][k2].x += cf * t.x;
            acc[i][k2].y += cf * t.y;
          }
        },
        uj, plane * (long long)sizeof(C), next, pbytes);
  }
  double2* dst = p.acc + ta * plane * p.nz + z * plane;
#pragma unroll
  for (int i = 0; i < G::X2_IT; ++i) {
    const int it = threadIdx.x + i * NT;
    if (it < N * A) {
      // same slot -> (y, x) map as plane_inverse's last step
      int k1, row;
      x2_item<A>(it, k1, row);
      const int y = row / B + A * (row % B);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) {
        double2* o = dst + y * N + k1 + A * k2;
        if (PACKED) {
          o->x += (double)acc[i][k2].x;
        } else {
          double2 cur = *o;
          cur.x += (double)acc[i][k2].x;
          cur.y += (double)acc[i][k2].y;
          *o = cur;
        }
      }
    }
  }
}
template <int N, typename T, bool PACKED>
__global__ void __launch_bounds__(PlaneCfg<N, T>::NT) k_pass_c(PairArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_c_body<N, T, PACKED>(p, blockIdx.x, blockIdx.y, smem_raw);
}

// Pass C with the roles swapped: grid (TJ, N); CTA (tj, z) owns band j of the
// batch's second index and loops over the TA bands a of its first index,
// accumulating w_a conj(W_aj) f_a in registers (f = u_tgt grids; w_a = w_tgt[a],
// or 1 when w_tgt is null), then adds coef * w_occ[j] (or coef) times the plane
// into the FP64 accumulator of j.  Uses: the vector-Jacobian product with
// respect to the occupied orbitals (f = cotangent or target grids, weight
// w_j), and the pair symmetry W_qj,ka = conj(W_ka,qj) (f_a = u_a, weight w_a)
// on k = q tiles and k != q blocks.
template <int N, typename T>
__device__ __forceinline__ void pass_ct_body(const PairArgs& p, int tj, int z, unsigned char* smem_raw) {
  using C = cplx<T>;
  using G = PlaneCfg<N, T>;
  constexpr int A = G::A, B = G::B, NT = G::NT;
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* tw2 = tw + N;
  C* s0 = tw2 + N;
  C* s1 = s0 + G::BUF;
  load_twiddles<N, T, NT>(tw, p.tw);
  bsync<NT>();
  make_twiddles2<N, T, NT>(tw2, tw);
  bsync<NT>();
  constexpr long long plane = (long long)N * N;
  const int LX = p.LX;
  const long long pstride = (long long)p.P2 * LX;
  C acc[G::X2_IT][B];
#pragma unroll
  for (int i = 0; i < G::X2_IT; ++i)
#pragma unroll
    for (int k2 = 0; k2 < B; ++k2) acc[i][k2] = czero<C>();
#pragma unroll 1
  for (int ta = 0; ta < p.TA; ++ta) {
    const C* in = reinterpret_cast<const C*>(p.inter) + ((long long)(ta * p.TJ + tj) * p.nz + z) * pstride;
    const C* fa = reinterpret_cast<const C*>(p.u_tgt) + ta * p.u_tgt_stride + z * plane;
    const C* next = ta + 1 < p.TA ? in + (long long)p.TJ * p.nz * pstride : nullptr;
    const T wa = p.w_tgt ? (T)p.w_tgt[ta] : (T)1;
    plane_inverse<N, T, false>(
        tw, tw2, s0, s1, p.h1, p.P1, p.h2, [&](int kyb, int kxb) { return in[kyb * LX + kxb]; },
        [&](int i, int k2, int y, int x, C v) {
          const C t = cmulc(v, fa[y * N + x]);   // conj(W) * f_a
          acc[i][k2].x += wa * t.x;
          acc[i][k2].y += wa * t.y;
        },
        fa, plane * (long long)sizeof(C), next, pstride * (long long)sizeof(C));
  }
  const double cf = p.coef * (p.w_occ ? p.w_occ[tj] : 1.0);
  double2* dst = p.acc + tj * plane * p.nz + z * plane;
#pragma unroll
  for (int i = 0; i < G::X2_IT; ++i) {
    const int it = threadIdx.x + i * NT;
    if (it < N * A) {
      int k1, row;
      x2_item<A>(it, k1, row);
      const int y = row / B + A * (row % B);
#pragma unroll
      for (int k2 = 0; k2 < B; ++k2) {
        double2* o = dst + y * N + k1 + A * k2;
        double2 cur = *o;
        cur.x += cf * (double)acc[i][k2].x;
        cur.y += cf * (double)acc[i][k2].y;
        *o = cur;
      }
    }
  }
}
template <int N, typename T>
__global__ void __launch_bounds__(PlaneCfg<N, T>::NT) k_pass_ct(PairArgs p) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  pass_ct_body<N, T>(p, blockIdx.x, blockIdx.y, smem_raw);
}

// ------------------------------------------------------ kernel table (a2) --

// v(k - q + G)/N and dv/dmu/N^2 over the pruned box, evaluated in FP64.
// v(g)/N (and dv/dmu/N^2) at box index i of the pruned box, g = k - q + G with
// d = k - q (fractional)
__device__ __forceinline__ void vtab_value(const VtabArgs& a, const double d[3], long long i, double& v,
                                           double& dv) {
  const int kx = (int)(i % a.P1), ky = (int)((i / a.P1) % a.P2), kz = (int)(i / ((long long)a.P1 * a.P2));
  const double m0 = (double)(kx - a.h1) + d[0];
  const double m1 = (double)(ky - a.h2) + d[1];
  const double m2 = (double)(kz - a.h3) + d[2];
  const bool zero = (m0 == 0.0 && m1 == 0.0 && m2 == 0.0);
  const double g2 = m0 * (a.M[0] * m0 + a.M[1] * m1 + a.M[2] * m2) +
                    m1 * (a.M[3] * m0 + a.M[4] * m1 + a.M[5] * m2) +
                    m2 * (a.M[6] * m0 + a.M[7] * m1 + a.M[8] * m2);
  const double pi = 3.14159265358979323846;
  if (a.kernel == 0) {
    const double x = g2 / (4.0 * a.mu * a.mu);
    v = zero ? pi / (a.mu * a.mu) : 4.0 * pi / g2 * (-expm1(-x));
    dv = -2.0 * pi / (a.mu * a.mu * a.mu) * exp(-x);
  } else {
    v = zero ? 0.0 : 4.0 * pi / g2;
    dv = 0.0;
  }
  v *= a.inv_n;
  dv *= a.inv_n2;
}

template <typename T>
__global__ void k_vtab(T* vt, T* dvt, VtabArgs a) {
  const long long n = (long long)a.P1 * a.P2 * a.P3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double v, dv;
    vtab_value(a, a.d, i, v, dv);
    vt[i] = (T)v;
    if (dvt) dvt[i] = (T)dv;
  }
}

// Every (k, q) table at once: blockIdx.y = k * nk + q, table (k, q) at
// vt + (k * nk + q) * box (kfrac: [nk][3] fractional k-points).
template <typename T>
__global__ void k_vtab_all(T* vt, const double* kfrac, int nk, VtabArgs a) {
  const long long n = (long long)a.P1 * a.P2 * a.P3;
  const int k = blockIdx.y / nk, q = blockIdx.y % nk;
  const double d[3] = {kfrac[3 * k] - kfrac[3 * q], kfrac[3 * k + 1] - kfrac[3 * q + 1],
                       kfrac[3 * k + 2] - kfrac[3 * q + 2]};
  T* out = vt + (long long)blockIdx.y * n;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    double v, dv;
    vtab_value(a, d, i, v, dv);
    out[i] = (T)v;
  }
}

// dv/dx for x = |g|^2: screened t = x/(4 mu^2), v'(x) = (4 pi/x^2)(t e^-t + expm1(-t)),
// with the series sum_{m>=2} (-1)^(m-1) (m-1) t^m / m! for small t (the two
// terms cancel there); Coulomb -4 pi/x^2.  The g = 0 point never contributes
// (it is multiplied by g_a g_b = 0), so it returns 0.
__device__ __forceinline__ double dv_dx(int kernel, double mu, double x, bool zero) {
  const double pi = 3.14159265358979323846;
  if (zero) return 0.0;
  if (kernel != 0) return -4.0 * pi / (x * x);
  const double t = x / (4.0 * mu * mu);
  double f;
  if (t < 0.05) {
    double term = t;            // t^m / m! built up from m = 1
    f = 0.0;
    for (int m = 2; m <= 14; ++m) {
      term *= t / m;
      f += ((m & 1) ? 1.0 : -1.0) * (m - 1) * term;
    }
  } else {
    f = t * exp(-t) + expm1(-t);
  }
  return 4.0 * pi / (x * x) * f;
}

// Seven tables over the pruned box for the strain derivative, FP64-evaluated:
// tab[0] = v/N^2, tab[1..6] = v'(|g|^2) g_a g_b / N^2 for ab = xx, yy, zz, yz, xz, xy.
template <typename T>
__global__ void k_strain_tab(T* tab, VtabArgs a) {
  const long long n = (long long)a.P1 * a.P2 * a.P3;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const int kx = (int)(i % a.P1), ky = (int)((i / a.P1) % a.P2), kz = (int)(i / ((long long)a.P1 * a.P2));
    const double m0 = (double)(kx - a.h1) + a.d[0];
    const double m1 = (double)(ky - a.h2) + a.d[1];
    const double m2 = (double)(kz - a.h3) + a.d[2];
    const bool zero = (m0 == 0.0 && m1 == 0.0 && m2 == 0.0);
    double g[3];
    for (int c = 0; c < 3; ++c) g[c] = m0 * a.Bm[c] + m1 * a.Bm[3 + c] + m2 * a.Bm[6 + c];
    const double x = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    const double pi = 3.14159265358979323846;
    double v;
    if (a.kernel == 0)
      v = zero ? pi / (a.mu * a.mu) : 4.0 * pi / x * (-expm1(-x / (4.0 * a.mu * a.mu)));
    else
      v = zero ? 0.0 : 4.0 * pi / x;
    const double dv = dv_dx(a.kernel, a.mu, x, zero) * a.inv_n2;
    tab[i] = (T)(v * a.inv_n2);
    tab[n + i] = (T)(dv * g[0] * g[0]);
    tab[2 * n + i] = (T)(dv * g[1] * g[1]);
    tab[3 * n + i] = (T)(dv * g[2] * g[2]);
    tab[4 * n + i] = (T)(dv * g[1] * g[2]);
    tab[5 * n + i] = (T)(dv * g[0] * g[2]);
    tab[6 * n + i] = (T)(dv * g[0] * g[1]);
  }
}

// Pass B for the strain derivative: forward z only, partial[pair][kyb][c] =
// sum tab_c |rho|^2 for the seven tables (p.dvt holds them, P3*P2*P1 apart).
template <int N, int NT, typename T>
__global__ void __launch_bounds__(NT) k_pass_b_strain(PairArgs p) {
  using C = cplx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sZ = tw + N;
  __shared__ double red[7][NT];
  load_twiddles<N, T>(tw, p.twz);
  __syncthreads();
  const int kyb = blockIdx.x, pair = blockIdx.y;
  const int P1 = p.P1, P2 = p.P2;
  const long long zstride = (long long)P2 * p.LX;
  const long long nbox = (long long)P2 * P1 * p.P3;
  const C* row = reinterpret_cast<const C*>(p.inter) + (long long)pair * N * zstride + (long long)kyb * p.LX;
  const T* tab = reinterpret_cast<const T*>(p.dvt);
  double acc[7] = {0, 0, 0, 0, 0, 0, 0};
  pencil_forward<N, NT, T>(
      tw, sZ, P1, p.h3, [&](int z, int c) { return row[z * zstride + c]; },
      [&](int kzb, int c, C v) {
        const long long i = ((long long)kzb * P2 + kyb) * P1 + c;
        const double r2 = (double)v.x * (double)v.x + (double)v.y * (double)v.y;
#pragma unroll
        for (int t = 0; t < 7; ++t) acc[t] += (double)tab[t * nbox + i] * r2;
      });
#pragma unroll
  for (int t = 0; t < 7; ++t) red[t][threadIdx.x] = acc[t];
  __syncthreads();
  for (int off = NT / 2; off > 0; off >>= 1) {
    if (threadIdx.x < off)
#pragma unroll
      for (int t = 0; t < 7; ++t) red[t][threadIdx.x] += red[t][threadIdx.x + off];
    __syncthreads();
  }
  if (threadIdx.x < 7) p.partial[((long long)pair * P2 + kyb) * 7 + threadIdx.x] = red[threadIdx.x][0];
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
  load_twiddles<N, T>(tw, g.twz);
  __syncthreads();
  const int kyb = blockIdx.x, b = blockIdx.y;
  const int Q1 = g.Q1, Q2 = g.Q2, Q3 = g.Q3;
  const C* box = reinterpret_cast<const C*>(g.box) + (long long)b * Q3 * Q2 * Q1 + (long long)kyb * Q1;
  C* st = reinterpret_cast<C*>(g.stage) + (long long)b * N * Q2 * Q1 + (long long)kyb * Q1;
  pencil_inverse<N, NT, T>(
      tw, sZ, Q1, g.n3, [&](int kzb, int c) { return box[(long long)kzb * Q2 * Q1 + c]; },
      [&](int z, int c, C v) { st[(long long)z * Q2 * Q1 + c] = v; });
}

// grid (nb, nz): inverse y and x transforms of stage plane (b, z) into u[b][z]
template <int N, typename T>
__global__ void __launch_bounds__(PlaneCfg<N, T>::NT) k_s2g_xy(GridArgs g) {
  using C = cplx<T>;
  using G = PlaneCfg<N, T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* tw2 = tw + N;
  C* s0 = tw2 + N;
  C* s1 = s0 + G::BUF;
  load_twiddles<N, T>(tw, g.tw);
  __syncthreads();
  make_twiddles2<N, T>(tw2, tw);
  __syncthreads();
  const int b = blockIdx.x, z = blockIdx.y;
  const int Q1 = g.Q1, Q2 = g.Q2;
  const C* st = reinterpret_cast<const C*>(g.stage) + ((long long)b * g.nz + z) * Q2 * Q1;
  C* u = reinterpret_cast<C*>(g.u) + (long long)b * N * N * g.nz + (long long)z * N * N;
  const T sc = (T)g.scale;
  plane_inverse<N, T, true>(
      tw, tw2, s0, s1, g.n1, Q1, g.n2, [&](int kyb, int kxb) { return st[kyb * Q1 + kxb]; },
      [&](int, int, int y, int x, C v) { u[y * N + x] = sc * v; });
}

// grid (nb, nz): forward x and y transforms of FP64 grid plane (b, z) into stage
template <int N>
__global__ void __launch_bounds__(PlaneCfg<N, double>::NT) k_g2s_xy(GridArgs g) {
  using C = double2;
  using G = PlaneCfg<N, double>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* s0 = tw + N;
  C* s1 = s0 + G::BUF;
  load_twiddles<N, double>(tw, g.tw);
  __syncthreads();
  const int b = blockIdx.x, z = blockIdx.y;
  const int Q1 = g.Q1;
  const C* f = g.f + (long long)b * N * N * g.nz + (long long)z * N * N;
  C* st = reinterpret_cast<C*>(g.stage) + ((long long)b * g.nz + z) * g.Q2 * Q1;
  plane_forward<N, double, PlaneCfg<N, double>::DB>(
      tw, s0, s1, g.n1, Q1, g.n2, [&](int y, int x) { return f[y * N + x]; },
      [&](int kyb, int kxb, C v) { st[kyb * Q1 + kxb] = v; });
}

// grid (Q2, nb): forward z transform of stage row (b, kyb) into box
template <int N, int NT>
__global__ void __launch_bounds__(NT) k_g2s_z(GridArgs g) {
  using C = double2;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* tw = reinterpret_cast<C*>(smem_raw);
  C* sZ = tw + N;
  load_twiddles<N, double>(tw, g.twz);
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
