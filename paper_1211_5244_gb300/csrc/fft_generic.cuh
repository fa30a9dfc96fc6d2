// Generic tile transform: Stockham autosort FFT of any length N <= 4096 on a
// shared-memory tile of `tk` independent lines, laid out [N][ldt] (element m
// of line t at m * ldt + t), run by the whole CTA.
//
// Each stage of radix R (current sub-length Ns) takes butterfly b from the
// inputs b + r * N / R, multiplies input r by W_N^{r * (b mod Ns) * N/(Ns R)},
// does an R-point DFT and writes output q to ((b / Ns) * Ns * R + b mod Ns +
// q * Ns): after the last stage the result is in natural order. Radices 2, 3,
// 4, 5, 7 and 8 have closed-form butterflies; any other factor (a prime from
// 11 up to 4096) uses the direct R-point sum. Lanes of a warp take
// consecutive lines t, so every shared-memory access of a warp is contiguous.
#pragma once

#include "common.cuh"
#include "fft_regs.cuh"

namespace ps {

// multiply by W^idx (DIR = -1) or its conjugate (DIR = +1); the table holds
// W_L^k = exp(-2 pi i k / L) and is read with stride `tws` (= L / N)
template <int DIR, typename C>
__device__ __forceinline__ C twid(C v, const C* __restrict__ tw, int idx, int tws) {
  C w = tw[idx * tws];
  return DIR < 0 ? cmul(v, w) : cmulc(v, w);
}

template <int DIR, typename C>
__device__ __forceinline__ void dft2(C& v0, C& v1) {
  C t = v0;
  v0 = cadd(t, v1);
  v1 = csub(t, v1);
}

template <int DIR, typename C>
__device__ __forceinline__ void dft4(C& v0, C& v1, C& v2, C& v3) {
  C s02 = cadd(v0, v2), d02 = csub(v0, v2);
  C s13 = cadd(v1, v3), d13 = csub(v1, v3);
  C r = cmul_i<DIR>(d13);  // DIR * i * (v1 - v3)
  v0 = cadd(s02, s13);
  v2 = csub(s02, s13);
  v1 = cadd(d02, r);
  v3 = csub(d02, r);
}

// 3-point DFT: y0 = a + s, y1,2 = (a - s/2) +- DIR i (sqrt3/2)(b - c), s = b + c.
template <int DIR, typename C>
__device__ __forceinline__ void dft3(C& v0, C& v1, C& v2) {
  using R = decltype(v0.x);
  const R h = R(0.86602540378443864676);  // sqrt(3)/2
  const C s = cadd(v1, v2), d = csub(v1, v2);
  const C t = mk(v0.x - R(0.5) * s.x, v0.y - R(0.5) * s.y);
  const C u = cmul_i<DIR>(cscale(d, h));
  v0 = cadd(v0, s);
  v1 = cadd(t, u);
  v2 = csub(t, u);
}

// 5-point DFT with cos(2 pi / 5), cos(4 pi / 5), sin(2 pi / 5), sin(4 pi / 5):
// y1,4 = t1 +- DIR i u1, y2,3 = t2 +- DIR i u2 with
// t1 = x0 + c1 a1 + c2 a2, t2 = x0 + c2 a1 + c1 a2, u1 = s1 b1 + s2 b2,
// u2 = s2 b1 - s1 b2, a1,b1 = x1 +- x4, a2,b2 = x2 +- x3.
template <int DIR, typename C>
__device__ __forceinline__ void dft5(C* v) {
  using R = decltype(v[0].x);
  const R c1 = R(0.30901699437494742410), c2 = R(-0.80901699437494742410);
  const R s1 = R(0.95105651629515357212), s2 = R(0.58778525229247312917);
  const C a1 = cadd(v[1], v[4]), b1 = csub(v[1], v[4]);
  const C a2 = cadd(v[2], v[3]), b2 = csub(v[2], v[3]);
  const C t1 = mk(v[0].x + c1 * a1.x + c2 * a2.x, v[0].y + c1 * a1.y + c2 * a2.y);
  const C t2 = mk(v[0].x + c2 * a1.x + c1 * a2.x, v[0].y + c2 * a1.y + c1 * a2.y);
  const C u1 = cmul_i<DIR>(mk(s1 * b1.x + s2 * b2.x, s1 * b1.y + s2 * b2.y));
  const C u2 = cmul_i<DIR>(mk(s2 * b1.x - s1 * b2.x, s2 * b1.y - s1 * b2.y));
  v[0] = cadd(v[0], cadd(a1, a2));
  v[1] = cadd(t1, u1);
  v[4] = csub(t1, u1);
  v[2] = cadd(t2, u2);
  v[3] = csub(t2, u2);
}

// 7-point DFT, the same symmetric form as dft5 with c_k = cos(2 pi k / 7),
// s_k = sin(2 pi k / 7), a_k, b_k = x_k +- x_{7-k} (k = 1, 2, 3):
// y_m, y_{7-m} = t_m +- DIR i u_m, t_m = x0 + sum_k cos(2 pi m k / 7) a_k,
// u_m = sum_k sin(2 pi m k / 7) b_k, the angles reduced to k = 1, 2, 3.
template <int DIR, typename C>
__device__ __forceinline__ void dft7(C* v) {
  using R = decltype(v[0].x);
  const R c1 = R(0.62348980185873353053), c2 = R(-0.22252093395631440429), c3 = R(-0.90096886790241912624);
  const R s1 = R(0.78183148246802980871), s2 = R(0.97492791218182360702), s3 = R(0.43388373911755812048);
  const C a1 = cadd(v[1], v[6]), b1 = csub(v[1], v[6]);
  const C a2 = cadd(v[2], v[5]), b2 = csub(v[2], v[5]);
  const C a3 = cadd(v[3], v[4]), b3 = csub(v[3], v[4]);
  const C x0 = v[0];
  const C t1 = mk(x0.x + c1 * a1.x + c2 * a2.x + c3 * a3.x, x0.y + c1 * a1.y + c2 * a2.y + c3 * a3.y);
  const C t2 = mk(x0.x + c2 * a1.x + c3 * a2.x + c1 * a3.x, x0.y + c2 * a1.y + c3 * a2.y + c1 * a3.y);
  const C t3 = mk(x0.x + c3 * a1.x + c1 * a2.x + c2 * a3.x, x0.y + c3 * a1.y + c1 * a2.y + c2 * a3.y);
  const C u1 = cmul_i<DIR>(mk(s1 * b1.x + s2 * b2.x + s3 * b3.x, s1 * b1.y + s2 * b2.y + s3 * b3.y));
  const C u2 = cmul_i<DIR>(mk(s2 * b1.x - s3 * b2.x - s1 * b3.x, s2 * b1.y - s3 * b2.y - s1 * b3.y));
  const C u3 = cmul_i<DIR>(mk(s3 * b1.x - s1 * b2.x + s2 * b3.x, s3 * b1.y - s1 * b2.y + s2 * b3.y));
  v[0] = cadd(x0, cadd(a1, cadd(a2, a3)));
  v[1] = cadd(t1, u1);
  v[6] = csub(t1, u1);
  v[2] = cadd(t2, u2);
  v[5] = csub(t2, u2);
  v[3] = cadd(t3, u3);
  v[4] = csub(t3, u3);
}

// 8-point DFT: two 4-point DFTs (even / odd inputs) joined by W_8^k.
template <int DIR, typename C>
__device__ __forceinline__ void dft8(C* v) {
  using R = decltype(v[0].x);
  const R s = R(0.70710678118654752440);  // sqrt(1/2)
  C a0 = v[0], a1 = v[2], a2 = v[4], a3 = v[6];
  C b0 = v[1], b1 = v[3], b2 = v[5], b3 = v[7];
  dft4<DIR>(a0, a1, a2, a3);
  dft4<DIR>(b0, b1, b2, b3);
  // W^1 = s (1 + DIR i), W^2 = DIR i, W^3 = s (-1 + DIR i)
  C w1 = mk(s * (b1.x - DIR * b1.y), s * (b1.y + DIR * b1.x));
  C w2 = cmul_i<DIR>(b2);
  C w3 = mk(s * (-b3.x - DIR * b3.y), s * (-b3.y + DIR * b3.x));
  v[0] = cadd(a0, b0); v[4] = csub(a0, b0);
  v[1] = cadd(a1, w1); v[5] = csub(a1, w1);
  v[2] = cadd(a2, w2); v[6] = csub(a2, w2);
  v[3] = cadd(a3, w3); v[7] = csub(a3, w3);
}

// Runs all stages; `a` holds the input and is clobbered. Returns the buffer
// (a or b) that holds the result. Ends with __syncthreads().
template <int DIR, typename T>
__device__ cpx<T>* stockham(cpx<T>* a, cpx<T>* b, int N, int tk, int ldt, const Stages& st,
                            const cpx<T>* __restrict__ tw, int tws) {
  using C = cpx<T>;
  // tk is a power of two dividing blockDim.x: each thread keeps one line t and
  // takes every (blockDim.x / tk)-th butterfly of it
  const int ltk = __ffs(tk) - 1;
  const int t = threadIdx.x & (tk - 1);
  const int bstep = blockDim.x >> ltk;
  int Ns = 1;
  for (int s = 0; s < st.n; ++s) {
    const int R = st.R[s];
    const int NR = N / R;
    const int estep = N / (Ns * R);
    const unsigned mg = st.mg[s];
    for (int bf = threadIdx.x >> ltk; bf < NR; bf += bstep) {
      const int q = div_by(bf, mg);  // bf / Ns
      const int k = bf - q * Ns;
      const int e = k * estep;  // r * e < N for every r < R
      const int ob = q * Ns * R + k;
      const C* in = a + bf * ldt + t;
      C* out = b + ob * ldt + t;
      if (R == 2) {
        C v0 = in[0], v1 = in[NR * ldt];
        if (e) v1 = twid<DIR>(v1, tw, e, tws);
        dft2<DIR>(v0, v1);
        out[0] = v0;
        out[Ns * ldt] = v1;
      } else if (R == 4) {
        C v0 = in[0], v1 = in[NR * ldt], v2 = in[2 * NR * ldt], v3 = in[3 * NR * ldt];
        if (e) {
          v1 = twid<DIR>(v1, tw, e, tws);
          v2 = twid<DIR>(v2, tw, 2 * e, tws);
          v3 = twid<DIR>(v3, tw, 3 * e, tws);
        }
        dft4<DIR>(v0, v1, v2, v3);
        out[0] = v0;
        out[Ns * ldt] = v1;
        out[2 * Ns * ldt] = v2;
        out[3 * Ns * ldt] = v3;
      } else if (R == 3) {
        C v0 = in[0], v1 = in[NR * ldt], v2 = in[2 * NR * ldt];
        if (e) {
          v1 = twid<DIR>(v1, tw, e, tws);
          v2 = twid<DIR>(v2, tw, 2 * e, tws);
        }
        dft3<DIR>(v0, v1, v2);
        out[0] = v0;
        out[Ns * ldt] = v1;
        out[2 * Ns * ldt] = v2;
      } else if (R == 5) {
        C v[5];
#pragma unroll
        for (int r = 0; r < 5; ++r) v[r] = in[r * NR * ldt];
        if (e) {
#pragma unroll
          for (int r = 1; r < 5; ++r) v[r] = twid<DIR>(v[r], tw, r * e, tws);
        }
        dft5<DIR>(v);
#pragma unroll
        for (int r = 0; r < 5; ++r) out[r * Ns * ldt] = v[r];
      } else if (R == 7) {
        C v[7];
#pragma unroll
        for (int r = 0; r < 7; ++r) v[r] = in[r * NR * ldt];
        if (e) {
#pragma unroll
          for (int r = 1; r < 7; ++r) v[r] = twid<DIR>(v[r], tw, r * e, tws);
        }
        dft7<DIR>(v);
#pragma unroll
        for (int r = 0; r < 7; ++r) out[r * Ns * ldt] = v[r];
      } else if (R == 8) {
        C v[8];
#pragma unroll
        for (int r = 0; r < 8; ++r) v[r] = in[r * NR * ldt];
        if (e) {
#pragma unroll
          for (int r = 1; r < 8; ++r) v[r] = twid<DIR>(v[r], tw, r * e, tws);
        }
        dft8<DIR>(v);
#pragma unroll
        for (int r = 0; r < 8; ++r) out[r * Ns * ldt] = v[r];
      } else {
        // direct R-point sum: output q = sum_r in_r W_N^{r (e + q N/R)}
        for (int q = 0; q < R; ++q) {
          const int step = e + q * NR;  // < N
          int idx = 0;
          C acc = mk(T(0), T(0));
          for (int r = 0; r < R; ++r) {
            C v = twid<DIR>(in[r * NR * ldt], tw, idx, tws);
            acc = cadd(acc, v);
            idx += step;
            if (idx >= N) idx -= N;
          }
          out[q * Ns * ldt] = acc;
        }
      }
    }
    __syncthreads();
    C* tmp = a;
    a = b;
    b = tmp;
    Ns *= R;
  }
  return a;
}

// Copies the twiddles a tile transform reads into shared memory: W_N^j for
// j < N (from the length-L table, stride tws), or W_M^j for j < M in
// Bluestein form. No barrier: the caller's next __syncthreads covers it.
// Lengths whose table does not fit beside the tile read the global table.
// Returns the table and stride the transform reads: tsm when `in_smem`, else
// the global table itself.
template <typename T>
__device__ const cpx<T>* load_twiddles(cpx<T>* tsm, const cpx<T>* __restrict__ tw, int N, int tws,
                                       const BlueArgs& bl, bool in_smem, int* tstr) {
  if (!in_smem) {
    *tstr = bl.M ? 1 : tws;
    return bl.M ? static_cast<const cpx<T>*>(bl.twM) : tw;
  }
  *tstr = 1;
  if (bl.M) {
    const cpx<T>* __restrict__ tm = static_cast<const cpx<T>*>(bl.twM);
    for (int j = threadIdx.x; j < bl.M; j += blockDim.x) tsm[j] = tm[j];
  } else {
    for (int j = threadIdx.x; j < N; j += blockDim.x) tsm[j] = tw[(size_t)j * tws];
  }
  return tsm;
}

// The transform of a tile (as stockham), in Bluestein form when bl.M > 0:
// with the stored chirp c[m] = exp(-i pi m^2 / N) (its conjugate for the
// inverse, DIR = +1), X[k] = c[k] sum_m (x[m] c[m]) conj(c[k - m]) since
// m k = (m^2 + k^2 - (k - m)^2) / 2. The sum is a cyclic convolution of
// length M >= 2N - 1, done with length-M Stockham transforms and bl.Bf, the
// transform of the conjugate chirp divided by M. Both buffers hold M rows.
// `ttab` with stride `tstr` holds W_N^j (W_M^j in Bluestein form): the
// shared-memory table of load_twiddles (stride 1), or a global table.
template <int DIR, typename T>
__device__ cpx<T>* line_transform(cpx<T>* a, cpx<T>* b, int N, int tk, int ldt, const Stages& st,
                                  const cpx<T>* ttab, int tstr, const BlueArgs& bl) {
  using C = cpx<T>;
  if (bl.M == 0) return stockham<DIR, T>(a, b, N, tk, ldt, st, ttab, tstr);
  const int M = bl.M;
  const C* ch = static_cast<const C*>(bl.chirp);  // shared or global memory
  const C* Bf = static_cast<const C*>(bl.Bf);
  const int ltk = __ffs(tk) - 1;
  const int t = threadIdx.x & (tk - 1);  // blockDim.x is a multiple of tk
  const int mstep = blockDim.x >> ltk;
  for (int m = threadIdx.x >> ltk; m < M; m += mstep) {
    C v = mk(T(0), T(0));
    if (m < N) v = DIR < 0 ? cmul(a[m * ldt + t], ch[m]) : cmulc(a[m * ldt + t], ch[m]);
    a[m * ldt + t] = v;
  }
  __syncthreads();
  C* r = stockham<-1, T>(a, b, M, tk, ldt, bl.st, ttab, tstr);
  C* o = (r == a) ? b : a;
  for (int m = threadIdx.x >> ltk; m < M; m += mstep)
    r[m * ldt + t] = DIR < 0 ? cmul(r[m * ldt + t], Bf[m]) : cmulc(r[m * ldt + t], Bf[m]);
  __syncthreads();
  r = stockham<1, T>(r, o, M, tk, ldt, bl.st, ttab, tstr);
  for (int k = threadIdx.x >> ltk; k < N; k += mstep)
    r[k * ldt + t] = DIR < 0 ? cmul(r[k * ldt + t], ch[k]) : cmulc(r[k * ldt + t], ch[k]);
  __syncthreads();
  return r;
}

// The Bluestein form of line_transform for FP32 lines whose convolution length
// M = P * Q is a power of two with M >= 2N: the length-M transforms as
// four-step transforms on compile-time register DFTs instead of Stockham
// stages. With m = b + Q a and k = k1 + P k2 (a, k1 < P; b, k2 < Q):
//   step 1, column b of a line: y[k1] = sum_a u[b + Q a] W_P^{a k1}, with
//     u[m] = x[m] c[m] for m < N (zero above; a >= P/2 is past M/2 >= N),
//     times W_M^{b k1}, to row k1 Q + b of `b`;
//   steps 2-3, row k1: the Q-point DFT over b gives U[k1 + P k2]; times Bf
//     (the transform of the conjugate chirp over M); the inverse Q-point DFT
//     over k2 and conj W_M^{b k1} give column b of the inverse's second
//     step, to row b P + k1 of `a`;
//   step 4, column b: the inverse P-point DFT over k1 gives v[b + Q a], kept
//     for m < N, times c[m], to row m of `b`.
// Three barriers instead of two per Stockham stage and one per multiply.
// DIR = +1 conjugates the chirp and Bf as line_transform does. Returns b.
template <int P, int Q, int DIR>
__device__ float2* blue_regs(float2* a, float2* b, int N, int tk, int ldt, const float2* ttab, int tstr,
                             const BlueArgs& bl) {
  const float2* ch = static_cast<const float2*>(bl.chirp);  // shared or global memory
  const float2* Bf = static_cast<const float2*>(bl.Bf);
  const int ltk = __ffs(tk) - 1;
  for (int i = threadIdx.x; i < (Q << ltk); i += blockDim.x) {
    const int t = i & (tk - 1), col = i >> ltk;
    float2 y[P];
#pragma unroll
    for (int r = 0; r < P; ++r) {
      const int m = col + Q * r;
      y[r] = make_float2(0.f, 0.f);
      if (r < P / 2 && m < N) {
        const float2 x = a[m * ldt + t], c = ch[m];
        y[r] = DIR < 0 ? cmul(x, c) : cmulc(x, c);
      }
    }
    regs::rdft<P, -1, true>(y);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) b[(k1 * Q + col) * ldt + t] = k1 ? cmul(y[k1], ttab[col * k1 * tstr]) : y[k1];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (P << ltk); i += blockDim.x) {
    const int t = i & (tk - 1), k1 = i >> ltk;
    float2 z[Q];
#pragma unroll
    for (int c2 = 0; c2 < Q; ++c2) z[c2] = b[(k1 * Q + c2) * ldt + t];
    regs::rdft<Q, -1, false>(z);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      const float2 f = Bf[k1 + P * k2];
      z[k2] = DIR < 0 ? cmul(z[k2], f) : cmulc(z[k2], f);
    }
    regs::rdft<Q, 1, false>(z);
#pragma unroll
    for (int c2 = 0; c2 < Q; ++c2) a[(c2 * P + k1) * ldt + t] = c2 ? cmulc(z[c2], ttab[c2 * k1 * tstr]) : z[c2];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < (Q << ltk); i += blockDim.x) {
    const int t = i & (tk - 1), col = i >> ltk;
    float2 y[P];
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) y[k1] = a[(col * P + k1) * ldt + t];
    regs::rdft<P, 1, false>(y);
#pragma unroll
    for (int r = 0; r < P / 2; ++r) {
      const int m = col + Q * r;
      if (m < N) {
        const float2 c = ch[m];
        b[m * ldt + t] = DIR < 0 ? cmul(y[r], c) : cmulc(y[r], c);
      }
    }
  }
  __syncthreads();
  return b;
}

// The Bluestein tables in shared memory, after the W_M table of
// load_twiddles, when the table has room for them (in_smem: 2M + N
// entries): the transformed chirp Bf at tsm + M and the chirp at tsm + 2M.
// Returns the BlueArgs the transform reads. No barrier: the caller's next
// __syncthreads covers it.
template <typename T>
__device__ __forceinline__ BlueArgs blue_tables(cpx<T>* tsm, const BlueArgs& bl, int N, bool in_smem) {
  BlueArgs b = bl;
  const int M = bl.M;
  if (M > 0 && in_smem) {
    const cpx<T>* __restrict__ bf = static_cast<const cpx<T>*>(bl.Bf);
    const cpx<T>* __restrict__ ch = static_cast<const cpx<T>*>(bl.chirp);
    for (int j = threadIdx.x; j < M; j += blockDim.x) tsm[M + j] = bf[j];
    for (int j = threadIdx.x; j < N; j += blockDim.x) tsm[2 * M + j] = ch[j];
    b.Bf = tsm + M;
    b.chirp = tsm + 2 * M;
  }
  return b;
}

// P of the four-step split M = P * Q of blue_regs (Q = M / P)
constexpr int blue_p(int M) { return M <= 32 ? 4 : M <= 128 ? 8 : M <= 512 ? 16 : 32; }

// The line transform of a generic pass: blue_regs when BM (a power-of-two
// Bluestein length, FP32) is set, else line_transform.
template <int DIR, typename T, int BM>
__device__ __forceinline__ cpx<T>* gen_transform(cpx<T>* a, cpx<T>* b, int N, int tk, int ldt, const Stages& st,
                                                 const cpx<T>* ttab, int tstr, const BlueArgs& bl) {
  if constexpr (BM > 0) {
    static_assert(sizeof(T) == 4, "register Bluestein form is FP32");
    return blue_regs<blue_p(BM), BM / blue_p(BM), DIR>(a, b, N, tk, ldt, ttab, tstr, bl);
  } else {
    return line_transform<DIR, T>(a, b, N, tk, ldt, st, ttab, tstr, bl);
  }
}

}  // namespace ps
