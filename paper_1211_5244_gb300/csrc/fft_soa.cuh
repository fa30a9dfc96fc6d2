// Pairs of register DFTs in structure-of-arrays form, on the packed FP32x2
// arithmetic of sm_100-class GPUs.
//
// A c2 holds two complex numbers: re = (re_0, re_1), im = (im_0, im_1). Two
// transforms with the same shape (the same constants) are carried out at once:
// every complex addition is two FP32x2 additions instead of four FP32
// additions. Multiplications by the constant twiddles use scalar FMAs with
// immediates (as many instructions as before); those by +-i are free (a swap of
// re and im folded into the following additions).
#pragma once

#include <utility>

#include "fft_regs.cuh"

namespace ps {
namespace soa {

struct c2 {
  float2 re, im;
};

__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
// a - b as one packed subtraction (no separate negation of b)
__device__ __forceinline__ float2 sub2(float2 a, float2 b) {
  unsigned long long ra, rb, rd;
  asm("mov.b64 %0, {%1, %2};" : "=l"(ra) : "f"(a.x), "f"(a.y));
  asm("mov.b64 %0, {%1, %2};" : "=l"(rb) : "f"(b.x), "f"(b.y));
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(rd) : "l"(ra), "l"(rb));
  float2 d;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(d.x), "=f"(d.y) : "l"(rd));
  return d;
}
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }

__device__ __forceinline__ c2 operator+(c2 a, c2 b) { return {add2(a.re, b.re), add2(a.im, b.im)}; }
__device__ __forceinline__ c2 operator-(c2 a, c2 b) { return {sub2(a.re, b.re), sub2(a.im, b.im)}; }

// a pair as one 16-byte word (re_0, re_1, im_0, im_1) and back
__device__ __forceinline__ c2 unpack(float4 v) { return {make_float2(v.x, v.y), make_float2(v.z, v.w)}; }
__device__ __forceinline__ float4 pack(c2 v) { return make_float4(v.re.x, v.re.y, v.im.x, v.im.y); }

// v * w (DIR = -1) or v * conj(w) (DIR = +1), lane by lane, w a pair of
// complex factors as (re_0, re_1, im_0, im_1)
template <int DIR>
__device__ __forceinline__ c2 cmul_pair(c2 v, float4 w) {
  const float2 wr = make_float2(w.x, w.y), wi = make_float2(w.z, w.w);
  if (DIR < 0) return {sub2(mul2(v.re, wr), mul2(v.im, wi)), fma2(v.re, wi, mul2(v.im, wr))};
  return {fma2(v.im, wi, mul2(v.re, wr)), sub2(mul2(v.im, wr), mul2(v.re, wi))};
}

// a + DIR i b and a - DIR i b, with the multiplication by i folded in
template <int DIR>
__device__ __forceinline__ c2 add_i(c2 a, c2 b) {  // a + (DIR i) b
  return DIR < 0 ? c2{add2(a.re, b.im), sub2(a.im, b.re)} : c2{sub2(a.re, b.im), add2(a.im, b.re)};
}
template <int DIR>
__device__ __forceinline__ c2 sub_i(c2 a, c2 b) {  // a - (DIR i) b
  return DIR < 0 ? c2{sub2(a.re, b.im), add2(a.im, b.re)} : c2{add2(a.re, b.im), sub2(a.im, b.re)};
}

// v * W_N^K (DIR = -1) or v * conj(W_N^K) (DIR = +1), both lanes, constants folded.
template <int N, int K, int DIR>
__device__ __forceinline__ c2 twc2(c2 v) {
  static_assert(64 % N == 0, "N must divide 64");
  constexpr int m = (K * (64 / N)) & 63;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 32) {
    return {make_float2(-v.re.x, -v.re.y), make_float2(-v.im.x, -v.im.y)};
  } else if constexpr (m == 16 || m == 48) {
    // forward m = 16 and inverse m = 48 multiply by -i: (re, im) -> (im, -re)
    constexpr bool minus_i = (m == 16) == (DIR < 0);
    return minus_i ? c2{v.im, make_float2(-v.re.x, -v.re.y)} : c2{make_float2(-v.im.x, -v.im.y), v.re};
  } else if constexpr (m == 8 || m == 24 || m == 40 || m == 56) {
    // (cos, sin) = (+-s, +-s): sums and differences of the pair times s
    constexpr float s = 0.70710678118654752440f;
    constexpr float c = (float)regs::cos64(m), sn = (float)regs::sin64(m);
    const float2 S = make_float2(s, s), NS = make_float2(-s, -s);
    const float2 apb = add2(v.re, v.im), amb = sub2(v.re, v.im), bma = sub2(v.im, v.re);
    if constexpr (DIR < 0) {  // (a + ib)(c - i sn)
      if constexpr (c > 0 && sn > 0) return {mul2(apb, S), mul2(bma, S)};
      else if constexpr (c < 0 && sn > 0) return {mul2(bma, S), mul2(apb, NS)};
      else if constexpr (c < 0 && sn < 0) return {mul2(apb, NS), mul2(amb, S)};
      else return {mul2(amb, S), mul2(apb, S)};
    } else {  // (a + ib)(c + i sn)
      if constexpr (c > 0 && sn > 0) return {mul2(amb, S), mul2(apb, S)};
      else if constexpr (c < 0 && sn > 0) return {mul2(apb, NS), mul2(amb, S)};
      else if constexpr (c < 0 && sn < 0) return {mul2(bma, S), mul2(apb, NS)};
      else return {mul2(apb, S), mul2(bma, S)};
    }
  } else {
    // both lanes at once: (a + ib)(c -+ i sn) as packed products with the
    // constants in register pairs
    constexpr float c = (float)regs::cos64(m), sn = (float)regs::sin64(m);
    const float2 C = make_float2(c, c), SN = make_float2(sn, sn), NSN = make_float2(-sn, -sn);
    if constexpr (DIR < 0) return {fma2(v.im, SN, mul2(v.re, C)), fma2(v.re, NSN, mul2(v.im, C))};
    else return {fma2(v.im, NSN, mul2(v.re, C)), fma2(v.re, SN, mul2(v.im, C))};
  }
}

// v * W_N^K (DIR = -1) or v * conj(W_N^K) (DIR = +1), both lanes, for N
// dividing 96 (the radix-3 combinations), constants folded
template <int N, int K, int DIR>
__device__ __forceinline__ c2 twk2(c2 v) {
  static_assert(96 % N == 0 && K >= 0, "N must divide 96");
  constexpr int m = (K * (96 / N)) % 96;
  if constexpr (m == 0) {
    return v;
  } else if constexpr (m == 48) {
    return {make_float2(-v.re.x, -v.re.y), make_float2(-v.im.x, -v.im.y)};
  } else if constexpr (m == 24 || m == 72) {
    constexpr bool minus_i = (m == 24) == (DIR < 0);
    return minus_i ? c2{v.im, make_float2(-v.re.x, -v.re.y)} : c2{make_float2(-v.im.x, -v.im.y), v.re};
  } else {
    constexpr float c = (float)regs::cos96(m), sn = (float)regs::sin96(m);
    const float2 C = make_float2(c, c), SN = make_float2(sn, sn), NSN = make_float2(-sn, -sn);
    if constexpr (DIR < 0) return {fma2(v.im, SN, mul2(v.re, C)), fma2(v.re, NSN, mul2(v.im, C))};
    else return {fma2(v.im, NSN, mul2(v.re, C)), fma2(v.re, SN, mul2(v.im, C))};
  }
}

// 3-point DFT of both lanes in place: y0 = a + s, y1,2 = (a - s/2) +- DIR i
// (sqrt(3)/2)(b - c), s = b + c
template <int DIR>
__device__ __forceinline__ void bfly3(c2& a, c2& b, c2& c) {
  const float2 H = make_float2(0.86602540378443864676f, 0.86602540378443864676f);
  const float2 NHALF = make_float2(-0.5f, -0.5f);
  const c2 s = b + c, d = b - c;
  const c2 m = {fma2(s.re, NHALF, a.re), fma2(s.im, NHALF, a.im)};
  const c2 hd = {mul2(d.re, H), mul2(d.im, H)};
  a = a + s;
  b = add_i<DIR>(m, hd);
  c = sub_i<DIR>(m, hd);
}

template <int N, int DIR, bool HZ, bool HO = false>
__device__ __forceinline__ void dft2(c2 (&x)[N]);

// radix-3 combination for output index K of an N-point DIT step (N = 3 M)
template <int N, int K, int DIR>
__device__ __forceinline__ void bfly3k(c2 (&x)[N], const c2 (&s0)[N / 3], const c2 (&s1)[N / 3],
                                       const c2 (&s2)[N / 3]) {
  c2 t0 = s0[K], t1 = twk2<N, K, DIR>(s1[K]), t2 = twk2<N, 2 * K, DIR>(s2[K]);
  bfly3<DIR>(t0, t1, t2);
  x[K] = t0;
  x[K + N / 3] = t1;
  x[K + 2 * N / 3] = t2;
}
template <int N, int DIR, int... K>
__device__ __forceinline__ void combine3(c2 (&x)[N], const c2 (&s0)[N / 3], const c2 (&s1)[N / 3],
                                         const c2 (&s2)[N / 3], std::integer_sequence<int, K...>) {
  (bfly3k<N, K, DIR>(x, s0, s1, s2), ...);
}

// HO: only the outputs below N/2 are formed
template <int N, int K, int DIR, bool HO>
__device__ __forceinline__ void bfly4(c2 (&x)[N], const c2 (&s0)[N / 4], const c2 (&s1)[N / 4],
                                      const c2 (&s2)[N / 4], const c2 (&s3)[N / 4]) {
  constexpr int m2 = (2 * K * (64 / N)) & 63;
  const c2 t0 = s0[K];
  const c2 t1 = twc2<N, K, DIR>(s1[K]);
  const c2 t3 = twc2<N, 3 * K, DIR>(s3[K]);
  c2 a, b;
  if constexpr (m2 == 16) {
    // t2 = (DIR i) s2: fold the factor into the additions
    a = add_i<DIR>(t0, s2[K]);
    b = sub_i<DIR>(t0, s2[K]);
  } else {
    const c2 t2 = twc2<N, 2 * K, DIR>(s2[K]);
    a = t0 + t2;
    b = t0 - t2;
  }
  const c2 c = t1 + t3, d = t1 - t3;
  x[K] = a + c;
  x[K + N / 4] = add_i<DIR>(b, d);
  if constexpr (!HO) {
    x[K + N / 2] = a - c;
    x[K + 3 * N / 4] = sub_i<DIR>(b, d);
  }
}

template <int N, int DIR, bool HO, int... K>
__device__ __forceinline__ void combine4(c2 (&x)[N], const c2 (&s0)[N / 4], const c2 (&s1)[N / 4],
                                         const c2 (&s2)[N / 4], const c2 (&s3)[N / 4],
                                         std::integer_sequence<int, K...>) {
  (bfly4<N, K, DIR, HO>(x, s0, s1, s2, s3), ...);
}

// In-place N-point DFTs of both lanes (N a power of two <= 64, or three
// times one), natural order. HZ: the upper half of the input is zero. HO:
// only the lower half of the output is needed (N >= 8; the upper half is left
// undefined; with the factor 3 the caller's unread outputs are simply not
// formed by the compiler).
template <int N, int DIR, bool HZ, bool HO>
__device__ __forceinline__ void dft2(c2 (&x)[N]) {
  static_assert(!HO || N >= 8, "output pruning needs the radix-4 combine");
  if constexpr (N % 3 == 0) {
    constexpr int M = N / 3;
    static_assert(!HZ || M % 2 == 0, "HZ needs an even sub-length");
    c2 s0[M], s1[M], s2[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      s0[i] = x[3 * i];
      s1[i] = x[3 * i + 1];
      s2[i] = x[3 * i + 2];
    }
    dft2<M, DIR, HZ>(s0);
    dft2<M, DIR, HZ>(s1);
    dft2<M, DIR, HZ>(s2);
    combine3<N, DIR>(x, s0, s1, s2, std::make_integer_sequence<int, M>{});
  } else if constexpr (N == 1) {
  } else if constexpr (N == 2) {
    if constexpr (HZ) {
      x[1] = x[0];
    } else {
      const c2 a = x[0];
      x[0] = a + x[1];
      x[1] = a - x[1];
    }
  } else if constexpr (N == 4 && HZ) {
    const c2 a = x[0], b = x[1];
    x[0] = a + b;
    x[2] = a - b;
    x[1] = add_i<DIR>(a, b);
    x[3] = sub_i<DIR>(a, b);
  } else {
    constexpr int M = N / 4;
    c2 s0[M], s1[M], s2[M], s3[M];
#pragma unroll
    for (int i = 0; i < M; ++i) {
      s0[i] = x[4 * i];
      s1[i] = x[4 * i + 1];
      s2[i] = x[4 * i + 2];
      s3[i] = x[4 * i + 3];
    }
    dft2<M, DIR, HZ>(s0);
    dft2<M, DIR, HZ>(s1);
    dft2<M, DIR, HZ>(s2);
    dft2<M, DIR, HZ>(s3);
    combine4<N, DIR, HO>(x, s0, s1, s2, s3, std::make_integer_sequence<int, M>{});
  }
}

}  // namespace soa
}  // namespace ps
