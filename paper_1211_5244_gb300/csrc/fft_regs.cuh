// Compile-time DFTs held entirely in registers (FP32 complex), for the
// specialised pass kernels.
//
// rdft<N, DIR, HZ>(x): in-place N-point DFT (N a power of two, N <= 64, or
// three times one), natural order in and out, DIR = -1 forward
// (W = exp(-2 pi i / N)), +1 inverse (unnormalised). Recursive decimation in
// time with radix 3 first where N has the factor, then radix 4 (radix 2 at the
// bottom when N is 2 * 4^k). HZ = true declares that the
// upper half of the input is zero (the zero padding of §3), which removes
// the additions of the leaf butterflies. Outputs that the caller never reads
// are removed by the compiler, which is how the truncated inverse transforms
// of §3 ("compactification") cost less.
#pragma once

#include <utility>

#include "common.cuh"

namespace ps {
namespace regs {

// cos(2 pi m / 64), m = 0..16
constexpr double kCos64[17] = {
    1.0, 0.99518472667219688624, 0.98078528040323044913, 0.95694033573220886494,
    0.92387953251128675613, 0.88192126434835502971, 0.83146961230254523708, 0.77301045336273696081,
    0.7071067811865475244, 0.63439328416364549822, 0.55557023301960222474, 0.47139673682599764856,
    0.38268343236508977173, 0.29028467725446236764, 0.19509032201612826785, 0.098017140329560601994,
    0.0};

constexpr double cos64(int m) {
  return (m & 63) < 16   ? kCos64[m & 15]
         : (m & 63) < 32 ? -kCos64[16 - ((m & 63) - 16)]
         : (m & 63) < 48 ? -kCos64[(m & 63) - 32]
                         : kCos64[16 - ((m & 63) - 48)];
}
constexpr double sin64(int m) { return cos64(m - 16); }

// cos(2 pi m / 96), m = 0..24 (a quarter wave): the constant twiddles of
// lengths with a factor 3 (any N dividing 96)
constexpr double kCos96[25] = {
    1.0, 0.99785892323860350674, 0.99144486137381041114, 0.98078528040323044913,
    0.96592582628906828675, 0.94693012949510566426, 0.92387953251128675613, 0.89687274153268830389,
    0.86602540378443864676, 0.83146961230254523708, 0.79335334029123516458, 0.75183980747897739641,
    0.70710678118654752440, 0.65934581510006886843, 0.60876142900872063942, 0.55557023301960222474,
    0.5, 0.44228869021900128200, 0.38268343236508977173, 0.32143946530316158070,
    0.25881904510252076235, 0.19509032201612826785, 0.13052619222005159155, 0.06540312923014306682,
    0.0};

constexpr double cos96(int m) {
  return (m % 96 + 96) % 96 <= 24   ? kCos96[(m % 96 + 96) % 96]
         : (m % 96 + 96) % 96 <= 48 ? -kCos96[48 - (m % 96 + 96) % 96]
         : (m % 96 + 96) % 96 <= 72 ? -kCos96[(m % 96 + 96) % 96 - 48]
                                    : kCos96[96 - (m % 96 + 96) % 96];
}
constexpr double sin96(int m) { return cos96(m - 24); }

__device__ __forceinline__ float2 operator+(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 operator-(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }

// v * W_N^K (DIR = -1) or v * conj(W_N^K) (DIR = +1), constants folded
template <int N, int K, int DIR>
__device__ __forceinline__ float2 twc(float2 v) {
  static_assert(64 % N == 0, "N must divide 64");
  constexpr int m = (K * (64 / N)) & 63;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 32) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (m == 16) {  // forward: -i, inverse: +i
    return DIR < 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
  } else if constexpr (m == 48) {  // forward: +i, inverse: -i
    return DIR < 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  } else if constexpr (m == 8 || m == 24 || m == 40 || m == 56) {
    constexpr float s = 0.70710678118654752440f;
    // (cos, sin) = (+-s, +-s)
    constexpr float c = (float)cos64(m), sn = (float)sin64(m);
    if constexpr (DIR < 0) {
      // (a + ib)(c - i sn) = (a c + b sn) + i (b c - a sn)
      if constexpr (c > 0 && sn > 0) return make_float2(s * (v.x + v.y), s * (v.y - v.x));
      else if constexpr (c < 0 && sn > 0) return make_float2(s * (v.y - v.x), -s * (v.x + v.y));
      else if constexpr (c < 0 && sn < 0) return make_float2(-s * (v.x + v.y), s * (v.x - v.y));
      else return make_float2(s * (v.x - v.y), s * (v.x + v.y));
    } else {
      // (a + ib)(c + i sn) = (a c - b sn) + i (b c + a sn)
      if constexpr (c > 0 && sn > 0) return make_float2(s * (v.x - v.y), s * (v.x + v.y));
      else if constexpr (c < 0 && sn > 0) return make_float2(-s * (v.x + v.y), s * (v.x - v.y));
      else if constexpr (c < 0 && sn < 0) return make_float2(s * (v.y - v.x), -s * (v.x + v.y));
      else return make_float2(s * (v.x + v.y), s * (v.y - v.x));
    }
  } else {
    constexpr float c = (float)cos64(m), sn = (float)sin64(m);
    if constexpr (DIR < 0) return make_float2(v.x * c + v.y * sn, v.y * c - v.x * sn);
    else return make_float2(v.x * c - v.y * sn, v.y * c + v.x * sn);
  }
}

// multiply by DIR * i
template <int DIR>
__device__ __forceinline__ float2 mul_i(float2 v) {
  return DIR < 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
}

// v * W_N^K (DIR = -1) or v * conj(W_N^K) (DIR = +1) for N dividing 96 (the
// radix-3 combinations), constants folded
template <int N, int K, int DIR>
__device__ __forceinline__ float2 twk(float2 v) {
  static_assert(96 % N == 0 && K >= 0, "N must divide 96");
  constexpr int m = (K * (96 / N)) % 96;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 48) {
    return make_float2(-v.x, -v.y);
  } else if constexpr (m == 24) {  // forward: -i, inverse: +i
    return DIR < 0 ? make_float2(v.y, -v.x) : make_float2(-v.y, v.x);
  } else if constexpr (m == 72) {
    return DIR < 0 ? make_float2(-v.y, v.x) : make_float2(v.y, -v.x);
  } else {
    constexpr float c = (float)cos96(m), sn = (float)sin96(m);
    if constexpr (DIR < 0) return make_float2(v.x * c + v.y * sn, v.y * c - v.x * sn);
    else return make_float2(v.x * c - v.y * sn, v.y * c + v.x * sn);
  }
}

// 3-point DFT in place: y0 = a + s, y1,2 = (a - s/2) +- DIR i (sqrt(3)/2)(b - c), s = b + c
template <int DIR>
__device__ __forceinline__ void bfly3(float2& a, float2& b, float2& c) {
  constexpr float h = 0.86602540378443864676f;
  const float2 s = b + c, d = b - c;
  const float2 m = make_float2(a.x - 0.5f * s.x, a.y - 0.5f * s.y);
  const float2 u = mul_i<DIR>(make_float2(h * d.x, h * d.y));
  a = a + s;
  b = m + u;
  c = m - u;
}

template <int N, int DIR, bool HZ>
__device__ __forceinline__ void rdft(float2 (&x)[N]);

// radix-4 combination for output index K of an N-point DIT step
template <int N, int K, int DIR>
__device__ __forceinline__ void bfly4(float2 (&x)[N], const float2 (&s0)[N / 4], const float2 (&s1)[N / 4],
                                      const float2 (&s2)[N / 4], const float2 (&s3)[N / 4]) {
  const float2 t0 = s0[K];
  const float2 t1 = twc<N, K, DIR>(s1[K]);
  const float2 t2 = twc<N, 2 * K, DIR>(s2[K]);
  const float2 t3 = twc<N, 3 * K, DIR>(s3[K]);
  const float2 a = t0 + t2, b = t0 - t2, c = t1 + t3, d = mul_i<DIR>(t1 - t3);
  x[K] = a + c;
  x[K + N / 4] = b + d;
  x[K + N / 2] = a - c;
  x[K + 3 * N / 4] = b - d;
}

// radix-3 combination for output index K of an N-point DIT step (N = 3 M):
// X[K + M q] = sum_r W_3^{rq} W_N^{rK} S_r[K]
template <int N, int K, int DIR>
__device__ __forceinline__ void bfly3k(float2 (&x)[N], const float2 (&s0)[N / 3], const float2 (&s1)[N / 3],
                                       const float2 (&s2)[N / 3]) {
  float2 t0 = s0[K], t1 = twk<N, K, DIR>(s1[K]), t2 = twk<N, 2 * K, DIR>(s2[K]);
  bfly3<DIR>(t0, t1, t2);
  x[K] = t0;
  x[K + N / 3] = t1;
  x[K + 2 * N / 3] = t2;
}

template <int N, int DIR, int... K>
__device__ __forceinline__ void combine3(float2 (&x)[N], const float2 (&s0)[N / 3], const float2 (&s1)[N / 3],
                                         const float2 (&s2)[N / 3], std::integer_sequence<int, K...>) {
  (bfly3k<N, K, DIR>(x, s0, s1, s2), ...);
}

template <int N, int DIR, int... K>
__device__ __forceinline__ void combine4(float2 (&x)[N], const float2 (&s0)[N / 4], const float2 (&s1)[N / 4],
                                         const float2 (&s2)[N / 4], const float2 (&s3)[N / 4],
                                         std::integer_sequence<int, K...>) {
  (bfly4<N, K, DIR>(x, s0, s1, s2, s3), ...);
}

template <int N, int DIR, bool HZ>
__device__ __forceinline__ void rdft(float2 (&x)[N]) {
  if constexpr (N == 1) {
  } else if constexpr (N == 2) {
    if constexpr (HZ) {
      x[1] = x[0];
    } else {
      const float2 a = x[0];
      x[0] = a + x[1];
      x[1] = a - x[1];
    }
  } else if constexpr (N == 4 && HZ) {
    const float2 a = x[0], d = mul_i<DIR>(x[1]);
    x[2] = a - x[1];
    x[0] = a + x[1];
    x[1] = a + d;
    x[3] = a - d;
  } else if constexpr (N % 3 == 0) {
    // radix 3 first (N = 3 * 2^k): three interleaved sub-DFTs; the zero upper
    // half of the input is the zero upper half of each of them
    constexpr int M = N / 3;
    static_assert(!HZ || M % 2 == 0, "HZ needs an even sub-length");
    float2 s0[M], s1[M], s2[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      s0[i] = x[3 * i];
      s1[i] = x[3 * i + 1];
      s2[i] = x[3 * i + 2];
    }
    rdft<M, DIR, HZ>(s0);
    rdft<M, DIR, HZ>(s1);
    rdft<M, DIR, HZ>(s2);
    combine3<N, DIR>(x, s0, s1, s2, std::make_integer_sequence<int, M>{});
  } else {
    constexpr int M = N / 4;
    float2 s0[M], s1[M], s2[M], s3[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      s0[i] = x[4 * i];
      s1[i] = x[4 * i + 1];
      s2[i] = x[4 * i + 2];
      s3[i] = x[4 * i + 3];
    }
    rdft<M, DIR, HZ>(s0);
    rdft<M, DIR, HZ>(s1);
    rdft<M, DIR, HZ>(s2);
    rdft<M, DIR, HZ>(s3);
    combine4<N, DIR>(x, s0, s1, s2, s3, std::make_integer_sequence<int, M>{});
  }
}

}  // namespace regs
}  // namespace ps
