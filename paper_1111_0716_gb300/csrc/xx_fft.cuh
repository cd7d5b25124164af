// xx_fft.cuh -- complex arithmetic, in-register small DFTs and the two-step
// line-FFT factorisation used by every pass of the exchange pipeline.
//
// Transform convention (same as the method's codensity transforms):
//   forward  X[k] = sum_n x[n] exp(-2 pi i n k / L)
//   inverse  x[n] = sum_k X[k] exp(+2 pi i n k / L)      (no 1/L)
// A length-N line is split as N = A * B (Cooley-Tukey, decimation in time):
//   step 1: for each n2 < B, a length-A DFT of x[B*n1 + n2] over n1, then the
//           inter-step twiddle W_N^(n2*k1);
//   step 2: for each k1 < A, a length-B DFT over n2, giving X[k1 + A*k2].
// Both small DFTs run in registers; only the exchange between the steps goes
// through shared memory.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "xx_roots.cuh"

namespace xx {

template <typename T> struct cvec;
template <> struct cvec<float> { using type = float2; };
template <> struct cvec<double> { using type = double2; };
template <typename T> using cplx = typename cvec<T>::type;

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 operator*(float s, float2 a) { return make_float2(s * a.x, s * a.y); }
__device__ __forceinline__ double2 operator+(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 operator-(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 operator*(double s, double2 a) { return make_double2(s * a.x, s * a.y); }

template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return C{a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
// conj(a) * b
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return C{a.x * b.x + a.y * b.y, a.x * b.y - a.y * b.x};
}
template <typename C> __device__ __forceinline__ C czero() { return C{0, 0}; }

// z * (-i) for the forward sign, z * (+i) for the inverse sign
template <bool INV, typename C> __device__ __forceinline__ C rotq(C z) {
  if (INV) return C{-z.y, z.x};
  return C{z.y, -z.x};
}

// z * exp(-+ 2 pi i m / R) with compile-time-foldable constants (m, R known after unrolling);
// the quarter turns are exact rotations and sign changes
template <int R, bool INV, typename C> __device__ __forceinline__ C root_mul(C z, int m) {
  m %= R;
  if (m == 0) return z;
  if (2 * m == R) return C{-z.x, -z.y};
  if (4 * m == R) return rotq<INV>(z);
  if (4 * m == 3 * R) return rotq<!INV>(z);
  using T = decltype(z.x);
  const T c = (T)xx_root_cos(R, m);
  const T s = INV ? (T)xx_root_sin(R, m) : -(T)xx_root_sin(R, m);
  return C{z.x * c - z.y * s, z.x * s + z.y * c};
}

// ------------------------------------------------------------ small DFTs --

template <bool INV, typename C> __device__ __forceinline__ void dft2(C* x) {
  C t = x[0];
  x[0] = t + x[1];
  x[1] = t - x[1];
}

template <bool INV, typename C> __device__ __forceinline__ void dft3(C* x) {
  using T = decltype(x[0].x);
  const T s3 = (T)0.86602540378443864676;          // sin(2 pi / 3)
  C t1 = x[1] + x[2];
  C t2 = x[0] - (T)0.5 * t1;
  C t3 = s3 * rotq<INV>(x[1] - x[2]);
  x[0] = x[0] + t1;
  x[1] = t2 + t3;
  x[2] = t2 - t3;
}

template <bool INV, typename C> __device__ __forceinline__ void dft4(C* x) {
  C a = x[0] + x[2], b = x[0] - x[2], c = x[1] + x[3];
  C d = rotq<INV>(x[1] - x[3]);
  x[0] = a + c;
  x[2] = a - c;
  x[1] = b + d;
  x[3] = b - d;
}

template <bool INV, typename C> __device__ __forceinline__ void dft5(C* x) {
  using T = decltype(x[0].x);
  const T c1 = (T)0.30901699437494742410, c2 = (T)-0.80901699437494742410;   // cos(2pi/5), cos(4pi/5)
  const T s1 = (T)0.95105651629515357212, s2 = (T)0.58778525229247312917;    // sin(2pi/5), sin(4pi/5)
  C A1 = x[1] + x[4], A2 = x[2] + x[3], B1 = x[1] - x[4], B2 = x[2] - x[3];
  C p1 = x[0] + c1 * A1 + c2 * A2;
  C p2 = x[0] + c2 * A1 + c1 * A2;
  C q1 = rotq<INV>(s1 * B1 + s2 * B2);
  C q2 = rotq<INV>(s2 * B1 - s1 * B2);
  x[0] = x[0] + A1 + A2;
  x[1] = p1 + q1;
  x[4] = p1 - q1;
  x[2] = p2 + q2;
  x[3] = p2 - q2;
}

template <bool INV, typename C> __device__ __forceinline__ void dft8(C* x) {
  using T = decltype(x[0].x);
  const T r = (T)0.70710678118654752440;           // sqrt(2) / 2
  C e[4] = {x[0], x[2], x[4], x[6]};
  C o[4] = {x[1], x[3], x[5], x[7]};
  dft4<INV>(e);
  dft4<INV>(o);
  // o[k] *= exp(-+ 2 pi i k / 8)
  if (INV) {
    o[1] = C{r * (o[1].x - o[1].y), r * (o[1].x + o[1].y)};
    o[3] = C{-r * (o[3].x + o[3].y), r * (o[3].x - o[3].y)};
  } else {
    o[1] = C{r * (o[1].x + o[1].y), r * (o[1].y - o[1].x)};
    o[3] = C{r * (o[3].y - o[3].x), -r * (o[3].x + o[3].y)};
  }
  o[2] = rotq<INV>(o[2]);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    x[k] = e[k] + o[k];
    x[k + 4] = e[k] - o[k];
  }
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dft(C* x);

constexpr int gcd_i(int a, int b) { return b == 0 ? a : gcd_i(b, a % b); }
// inverse of a modulo m (a, m coprime), by search (m is a small radix)
constexpr int modinv_i(int a, int m) {
  int r = 1;
  while ((a * r) % m != 1) ++r;
  return r;
}

// Composite length R = P * Q with P, Q coprime, in registers, by the prime-factor
// (Good-Thomas) mapping: input n = (Q n1 + P n2) mod R, output
// k = (Q (Q^-1 mod P) k1 + P (P^-1 mod Q) k2) mod R turn the length-R DFT into a
// P x Q two-dimensional DFT with no twiddle factors between the steps.
template <int P, int Q, bool INV, typename C> __device__ __forceinline__ void dft_pfa(C* x) {
  constexpr int R = P * Q;
  static_assert(gcd_i(P, Q) == 1, "prime-factor mapping needs coprime factors");
  constexpr int a = modinv_i(Q % P, P), b = modinv_i(P % Q, Q);
  C y[R];
#pragma unroll
  for (int n2 = 0; n2 < Q; ++n2) {
    C s[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) s[n1] = x[(Q * n1 + P * n2) % R];
    dft<P, INV>(s);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) y[k1 * Q + n2] = s[k1];
  }
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) {
    C s[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) s[n2] = y[k1 * Q + n2];
    dft<Q, INV>(s);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) x[(Q * a * k1 + P * b * k2) % R] = s[k2];
  }
}

// Composite length R = P * Q in registers (same two-step split as the lines).
template <int P, int Q, bool INV, typename C> __device__ __forceinline__ void dft_ct(C* x) {
  constexpr int R = P * Q;
  C y[R];
#pragma unroll
  for (int n2 = 0; n2 < Q; ++n2) {
    C s[P];
#pragma unroll
    for (int n1 = 0; n1 < P; ++n1) s[n1] = x[Q * n1 + n2];
    dft<P, INV>(s);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) y[n2 * P + k1] = root_mul<R, INV>(s[k1], n2 * k1);
  }
#pragma unroll
  for (int k1 = 0; k1 < P; ++k1) {
    C s[Q];
#pragma unroll
    for (int n2 = 0; n2 < Q; ++n2) s[n2] = y[n2 * P + k1];
    dft<Q, INV>(s);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) x[k1 + P * k2] = s[k2];
  }
}

template <int R, bool INV, typename C> __device__ __forceinline__ void dft(C* x) {
  if constexpr (R == 1) {
  } else if constexpr (R == 2) {
    dft2<INV>(x);
  } else if constexpr (R == 3) {
    dft3<INV>(x);
  } else if constexpr (R == 4) {
    dft4<INV>(x);
  } else if constexpr (R == 5) {
    dft5<INV>(x);
  } else if constexpr (R == 8) {
    dft8<INV>(x);
  } else if constexpr (R == 6) {
    dft_pfa<2, 3, INV>(x);
  } else if constexpr (R == 9) {
    dft_ct<3, 3, INV>(x);
  } else if constexpr (R == 10) {
    dft_pfa<2, 5, INV>(x);
  } else if constexpr (R == 12) {
    dft_pfa<4, 3, INV>(x);
  } else if constexpr (R == 16) {
    dft_ct<4, 4, INV>(x);
  } else if constexpr (R == 18) {
    dft_pfa<2, 9, INV>(x);
  } else {
    static_assert(R == 0, "unsupported in-register DFT length");
  }
}

// ------------------------------------------------------ line factorisation --

template <int N> struct Fac;
template <> struct Fac<24> { static constexpr int A = 8, B = 3; };
template <> struct Fac<32> { static constexpr int A = 8, B = 4; };
template <> struct Fac<36> { static constexpr int A = 6, B = 6; };
template <> struct Fac<40> { static constexpr int A = 8, B = 5; };
template <> struct Fac<48> { static constexpr int A = 8, B = 6; };
template <> struct Fac<54> { static constexpr int A = 6, B = 9; };
template <> struct Fac<60> { static constexpr int A = 6, B = 10; };
template <> struct Fac<64> { static constexpr int A = 8, B = 8; };
template <> struct Fac<72> { static constexpr int A = 8, B = 9; };
template <> struct Fac<80> { static constexpr int A = 8, B = 10; };
template <> struct Fac<96> { static constexpr int A = 8, B = 12; };
template <> struct Fac<108> { static constexpr int A = 6, B = 18; };

// inter-step twiddle: z * conj?(tw[(n2*k1) mod N]), tw[e] = exp(-2 pi i e / N)
template <bool INV, typename C> __device__ __forceinline__ C tw_mul(C z, C w) {
  if (INV) return cmulc(w, z);
  return cmul(z, w);
}
// the same for output k1 of a first-step DFT: the twiddle of k1 = 0 is exactly 1
// (k1 is a compile-time value after unrolling, so the multiply and the load fold away)
template <bool INV, typename C> __device__ __forceinline__ C tw_mul(C z, C w, int k1) {
  if (k1 == 0) return z;
  return tw_mul<INV>(z, w);
}

// ----------------------------------------------------- frequency pruning --
// A pruned axis keeps the frequencies f in [-h, h] (FFT index f mod N); the
// kept set is stored densely as "box" index b = f + h in [0, 2h].
__device__ __forceinline__ bool kept(int m, int N, int h) { return m <= h || m >= N - h; }
__device__ __forceinline__ int box_of(int m, int N, int h) { return m <= h ? m + h : m - N + h; }
__device__ __forceinline__ int idx_of_box(int b, int N, int h) { return b >= h ? b - h : b - h + N; }

}  // namespace xx
