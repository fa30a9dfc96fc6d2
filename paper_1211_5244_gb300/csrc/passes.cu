// The five passes of one solve (generic kernels for any transform length).
//
//   P1  forward x: zero-padded real-to-complex transform of length L1 of every
//       x row (n2 * n3 rows; §3: no transform of all-zero rows), keeping
//       c = L1/2 + 1 outputs                          rho -> A[z][y][kx]
//   P2  forward y: length-L2 transform of the c * n3 lines whose n2 nonzero
//       inputs are the physical y range               A -> B[z][ky][kx]
//   P3  z: forward length-L3 transform of the c * L2 lines (n3 nonzeros),
//       multiplication by K^F (Eq. 3), inverse transform, and only the n3
//       physical outputs are kept (compaction, §3); also the energy
//       E = 1/2 h^3 sum rho V as the Parseval sum 1/2 h^3 sum_k K^F |rho^F|^2
//       over the padded spectrum                      B -> B (in place)
//   P4  inverse y: length-L2 inverse of the c * n3 lines, n2 outputs kept
//                                                     B -> A
//   P5  inverse x: complex-to-real length-L1 inverse of the n2 * n3 rows,
//       n1 outputs kept                               A -> V
//
// The spread and compaction of §3 never touch memory: a pass loads only the
// nonzero part of a line into its shared-memory tile (the rest is zero) and
// stores only the part that a later pass reads. The transposes of §3 are
// replaced by tiles of `tk` lines that are adjacent in kx, the contiguous
// axis of A and B, so every global access is a run of tk consecutive complex
// numbers. K^F is stored once, scaled by 1/(L1 L2 L3), as its even octant in
// the [kz][ky][kx] layout the z pass reads (§3: the transposed kernel).
#include <algorithm>
#include <cstdio>
#include <cstdlib>

#include "common.cuh"
#include "fft_fast.cuh"
#include "fft_generic.cuh"
#include "reduce.cuh"

namespace ps {

constexpr int kU = 4;  // global loads each thread keeps in flight in the tile loops

struct GenArgs {
  int n1, n2, n3;
  int L1, L2, L3;
  int c, H2, H3;
  int ldc, ldk;
  int tk, ldt;
  int N;    // transform length of this pass
  int tws;  // twiddle-table stride (table length / N)
  int rows; // rows of each shared-memory buffer (>= N, and >= M in Bluestein form)
  int ltk;  // log2 tk (tk is a power of two)
  int twn;  // entries of the shared-memory twiddle table (N, or M in Bluestein form, 2M + N with
            // the Bluestein tables); 0: global
  unsigned mn1, mc, mN1;  // div_magic of n1, c and N + 1
  Stages st;
  BlueArgs bl;
};

// ---------------------------------------------------------------- P1

template <typename T, int BM = 0>
__global__ void __launch_bounds__(256) p1_generic(const T* __restrict__ rho, cpx<T>* __restrict__ A,
                                                  const cpx<T>* __restrict__ tw, GenArgs a) {
  using C = cpx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + a.rows * a.ldt;
  int tstr;  // the twiddles of the transform: in shared memory after the buffers when a.twn > 0
  const C* ttab = load_twiddles<T>(buf1 + a.rows * a.ldt, tw, a.N, a.tws, a.bl, a.twn > 0, &tstr);
  const BlueArgs bl = blue_tables<T>(buf1 + a.rows * a.ldt, a.bl, a.N, a.bl.M && a.twn >= 2 * a.bl.M + a.N);
  const int nrows = a.n2 * a.n3;
  const bool even = (a.L1 % 2) == 0;
  // even L1: row t is the complex line z[m] = x[2m] + i x[2m+1] of length N;
  // odd L1: rows 2t and 2t+1 are the real and imaginary parts of line t
  const int rpc = even ? a.tk : 2 * a.tk;  // rows per CTA
  const int row0 = blockIdx.x * rpc;
  for (int w = threadIdx.x; w < a.N * a.ldt; w += blockDim.x) buf0[w] = mk(T(0), T(0));
  __syncthreads();
  // the tile's rows are consecutive rows of rho: kU loads in flight per thread
  const int nin = rpc * a.n1;
  const long long base = (long long)row0 * a.n1, lim = (long long)nrows * a.n1;
  for (int w0 = threadIdx.x; w0 < nin; w0 += kU * blockDim.x) {
    T v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int w = w0 + u * blockDim.x;
      v[u] = (w < nin && base + w < lim) ? rho[base + w] : T(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int w = w0 + u * blockDim.x;
      const int t = div_by(w, a.mn1), i = w - t * a.n1;
      if (w < nin && row0 + t < nrows) {
        if (even) {
          T* f = reinterpret_cast<T*>(&buf0[(i >> 1) * a.ldt + t]);
          f[i & 1] = v[u];
        } else {
          T* f = reinterpret_cast<T*>(&buf0[i * a.ldt + (t >> 1)]);
          f[t & 1] = v[u];
        }
      }
    }
  }
  __syncthreads();
  C* out = gen_transform<-1, T, BM>(buf0, buf1, a.N, a.tk, a.ldt, a.st, ttab, tstr, bl);
  if (even) {
    // X[k] = E[k] + W_L^k O[k],  E = (Z[k] + conj Z[N-k]) / 2,  O = -i (Z[k] - conj Z[N-k]) / 2
    const int N = a.N;
    for (int w = threadIdx.x; w < a.tk * (N + 1); w += blockDim.x) {
      const int t = div_by(w, a.mN1), k = w - t * (N + 1);
      const int row = row0 + t;
      if (row >= nrows) continue;
      const C zk = out[(k == N ? 0 : k) * a.ldt + t];
      const C zm = out[(k == 0 ? 0 : N - k) * a.ldt + t];
      const C e = mk(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
      const C o = mk(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x));
      A[(size_t)row * a.ldc + k] = cadd(e, cmul(o, tw[k]));
    }
  } else {
    // two real rows from one complex line: Xa[k] = (Z[k] + conj Z[N-k]) / 2,
    // Xb[k] = (Z[k] - conj Z[N-k]) / (2i)
    const int N = a.N;
    for (int w = threadIdx.x; w < rpc * a.c; w += blockDim.x) {
      const int r = div_by(w, a.mc), k = w - r * a.c;
      const int row = row0 + r;
      if (row >= nrows) continue;
      const C zk = out[k * a.ldt + (r >> 1)];
      const C zm = out[(k == 0 ? 0 : N - k) * a.ldt + (r >> 1)];
      A[(size_t)row * a.ldc + k] = (r & 1) ? mk(T(0.5) * (zk.y + zm.y), T(-0.5) * (zk.x - zm.x))
                                           : mk(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
    }
  }
}

// ---------------------------------------------------------------- P2 / P4

// Transform along y of the tile kx0 .. kx0 + tk - 1 at one z:
//   DIR = -1: n2 inputs from A (rest zero), L2 outputs to B
//   DIR = +1: L2 inputs from B, n2 outputs to A
template <int DIR, typename T, int BM = 0>
__global__ void __launch_bounds__(256) py_generic(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst,
                                                  const cpx<T>* __restrict__ tw, GenArgs a) {
  using C = cpx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + a.rows * a.ldt;
  int tstr;  // the twiddles of the transform: in shared memory after the buffers when a.twn > 0
  const C* ttab = load_twiddles<T>(buf1 + a.rows * a.ldt, tw, a.N, a.tws, a.bl, a.twn > 0, &tstr);
  const BlueArgs bl = blue_tables<T>(buf1 + a.rows * a.ldt, a.bl, a.N, a.bl.M && a.twn >= 2 * a.bl.M + a.N);
  const int kx0 = blockIdx.x * a.tk;
  const int z = blockIdx.y;
  const int nin = DIR < 0 ? a.n2 : a.L2;
  const int nout = DIR < 0 ? a.L2 : a.n2;
  const int rows_in = DIR < 0 ? a.n2 : a.L2;   // row count of the source plane
  const int rows_out = DIR < 0 ? a.L2 : a.n2;
  const C* s = src + (size_t)z * rows_in * a.ldc + kx0;
  C* d = dst + (size_t)z * rows_out * a.ldc + kx0;
  const int ntot = a.tk * a.N;
  for (int w0 = threadIdx.x; w0 < ntot; w0 += kU * blockDim.x) {  // kU loads in flight per thread
    C v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int w = w0 + u * blockDim.x;
      const int t = w & (a.tk - 1), y = w >> a.ltk;
      v[u] = mk(T(0), T(0));
      if (w < ntot && y < nin && kx0 + t < a.c) v[u] = s[(size_t)y * a.ldc + t];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int w = w0 + u * blockDim.x;
      if (w < ntot) buf0[(w >> a.ltk) * a.ldt + (w & (a.tk - 1))] = v[u];
    }
  }
  __syncthreads();
  C* out = gen_transform<DIR, T, BM>(buf0, buf1, a.N, a.tk, a.ldt, a.st, ttab, tstr, bl);
  for (int w = threadIdx.x; w < a.tk * nout; w += blockDim.x) {
    const int t = w & (a.tk - 1), y = w >> a.ltk;
    if (kx0 + t < a.c) d[(size_t)y * a.ldc + t] = out[y * a.ldt + t];
  }
}

// ---------------------------------------------------------------- P3

template <typename T, int BM = 0>
__global__ void __launch_bounds__(256) pz_generic(cpx<T>* __restrict__ Bw, const T* __restrict__ K,
                                                  const cpx<T>* __restrict__ tw, GenArgs a,
                                                  double* partials, unsigned* counter,
                                                  double escale, double* E) {
  using C = cpx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + a.rows * a.ldt;
  int tstr;  // the twiddles of the transform: in shared memory after the buffers when a.twn > 0
  const C* ttab = load_twiddles<T>(buf1 + a.rows * a.ldt, tw, a.N, a.tws, a.bl, a.twn > 0, &tstr);
  const BlueArgs bl = blue_tables<T>(buf1 + a.rows * a.ldt, a.bl, a.N, a.bl.M && a.twn >= 2 * a.bl.M + a.N);
  const int kx0 = blockIdx.x * a.tk;
  const int ky = blockIdx.y;
  const size_t zstride = (size_t)a.L2 * a.ldc;
  C* line = Bw + (size_t)ky * a.ldc + kx0;
  const int ntot = a.tk * a.N;
  for (int w0 = threadIdx.x; w0 < ntot; w0 += kU * blockDim.x) {  // kU loads in flight per thread
    C v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int w = w0 + u * blockDim.x;
      const int t = w & (a.tk - 1), z = w >> a.ltk;
      v[u] = mk(T(0), T(0));
      if (w < ntot && z < a.n3 && kx0 + t < a.c) v[u] = line[z * zstride + t];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int w = w0 + u * blockDim.x;
      if (w < ntot) buf0[(w >> a.ltk) * a.ldt + (w & (a.tk - 1))] = v[u];
    }
  }
  __syncthreads();
  C* spec = gen_transform<-1, T, BM>(buf0, buf1, a.N, a.tk, a.ldt, a.st, ttab, tstr, bl);
  C* other = (spec == buf0) ? buf1 : buf0;
  // multiply by the octant of K^F; accumulate w(kx) K |rho^F|^2 for the energy
  const int kyo = min(ky, a.L2 - ky);
  const T* Krow = K + (size_t)kyo * a.ldk + kx0;
  const size_t kzstride = (size_t)(a.H2 + 1) * a.ldk;
  T eacc = T(0);
  for (int w0 = threadIdx.x; w0 < ntot; w0 += kU * blockDim.x) {  // kU K^F loads in flight per thread
    T kk[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int w = w0 + u * blockDim.x;
      const int t = w & (a.tk - 1), kz = w >> a.ltk;
      kk[u] = T(0);
      if (w < ntot && kx0 + t < a.c) kk[u] = Krow[min(kz, a.L3 - kz) * kzstride + t];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int w = w0 + u * blockDim.x;
      if (w >= ntot) continue;
      const int t = w & (a.tk - 1), kz = w >> a.ltk;
      const int kx = kx0 + t;
      C v = spec[kz * a.ldt + t];
      const T wgt = (kx == 0 || 2 * kx == a.L1) ? T(1) : T(2);  // kk = 0 past the last column
      eacc += wgt * kk[u] * (v.x * v.x + v.y * v.y);
      spec[kz * a.ldt + t] = cscale(v, kk[u]);
    }
  }
  __syncthreads();
  C* res = gen_transform<1, T, BM>(spec, other, a.N, a.tk, a.ldt, a.st, ttab, tstr, bl);
  for (int w = threadIdx.x; w < a.tk * a.n3; w += blockDim.x) {
    const int t = w & (a.tk - 1), z = w >> a.ltk;
    if (kx0 + t < a.c) line[z * zstride + t] = res[z * a.ldt + t];
  }
  if (E != nullptr) energy_finish((double)eacc, partials, counter, escale, E);
}

// ---------------------------------------------------------------- P5

template <typename T, int BM = 0>
__global__ void __launch_bounds__(256) p5_generic(const cpx<T>* __restrict__ A, T* __restrict__ V,
                                                  const cpx<T>* __restrict__ tw, GenArgs a) {
  using C = cpx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + a.rows * a.ldt;
  int tstr;  // the twiddles of the transform: in shared memory after the buffers when a.twn > 0
  const C* ttab = load_twiddles<T>(buf1 + a.rows * a.ldt, tw, a.N, a.tws, a.bl, a.twn > 0, &tstr);
  const BlueArgs bl = blue_tables<T>(buf1 + a.rows * a.ldt, a.bl, a.N, a.bl.M && a.twn >= 2 * a.bl.M + a.N);
  const int nrows = a.n2 * a.n3;
  const bool even = (a.L1 % 2) == 0;
  // even L1: row t's spectrum gives the complex line of length N; odd L1:
  // rows 2t and 2t+1 become the real and imaginary parts of line t (their
  // half spectra sit at buffer rows [0, c) and [c, 2c); the buffers hold
  // N + 1 = 2c rows)
  const int rpc = even ? a.tk : 2 * a.tk;  // rows per CTA
  const int row0 = blockIdx.x * rpc;
  const int ntot = rpc * a.c;
  for (int w0 = threadIdx.x; w0 < ntot; w0 += kU * blockDim.x) {  // kU loads in flight per thread
    C v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int w = w0 + u * blockDim.x;
      const int t = div_by(w, a.mc), k = w - t * a.c;
      v[u] = mk(T(0), T(0));
      if (w < ntot && row0 + t < nrows) v[u] = A[(size_t)(row0 + t) * a.ldc + k];
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int w = w0 + u * blockDim.x;
      const int t = div_by(w, a.mc), k = w - t * a.c;
      if (w < ntot) {
        if (even)
          buf0[k * a.ldt + t] = v[u];
        else
          buf0[(k + (t & 1) * a.c) * a.ldt + (t >> 1)] = v[u];
      }
    }
  }
  __syncthreads();
  const int N = a.N;
  if (even) {
    // Z[k] = E' + i O',  E' = X[k] + conj X[N-k],  O' = (X[k] - conj X[N-k]) conj(W_L^k)
    for (int w = threadIdx.x; w < a.tk * N; w += blockDim.x) {
      const int t = w & (a.tk - 1), k = w >> a.ltk;
      const C xk = buf0[k * a.ldt + t];
      const C xm = buf0[(N - k) * a.ldt + t];
      const C e = mk(xk.x + xm.x, xk.y - xm.y);
      const C o = cmulc(mk(xk.x - xm.x, xk.y + xm.y), tw[k]);
      buf1[k * a.ldt + t] = mk(e.x - o.y, e.y + o.x);
    }
  } else {
    // Z[k] = A[k] + i B[k] over the Hermitian extensions of the two half
    // spectra; X[0] of a real row is real, so its (rounding-level) imaginary
    // part is dropped instead of leaking into the other row
    for (int w = threadIdx.x; w < a.tk * N; w += blockDim.x) {
      const int t = w & (a.tk - 1), k = w >> a.ltk;
      C xa = k < a.c ? buf0[k * a.ldt + t] : cconj(buf0[(N - k) * a.ldt + t]);
      C xb = k < a.c ? buf0[(a.c + k) * a.ldt + t] : cconj(buf0[(a.c + N - k) * a.ldt + t]);
      if (k == 0) {
        xa.y = T(0);
        xb.y = T(0);
      }
      buf1[k * a.ldt + t] = mk(xa.x - xb.y, xa.y + xb.x);
    }
  }
  __syncthreads();
  C* out = gen_transform<1, T, BM>(buf1, buf0, N, a.tk, a.ldt, a.st, ttab, tstr, bl);
  for (int w = threadIdx.x; w < rpc * a.n1; w += blockDim.x) {
    const int t = div_by(w, a.mn1), i = w - t * a.n1;
    const int row = row0 + t;
    if (row >= nrows) continue;
    T v;
    if (even) {
      const C zz = out[(i >> 1) * a.ldt + t];
      v = (i & 1) ? zz.y : zz.x;
    } else {
      const C zz = out[i * a.ldt + (t >> 1)];
      v = (t & 1) ? zz.y : zz.x;
    }
    V[(size_t)row * a.n1 + i] = v;
  }
}

// ---------------------------------------------------------------- kernel table

// The five generic kernels of one Bluestein form: BM = 0 runs the Stockham
// stages (any length), BM > 0 the register four-step convolution of length
// BM (FP32; 32, 64, 96, 128, 192, 256 or 384).
template <typename T>
struct GenKernels {
  void (*p1)(const T*, cpx<T>*, const cpx<T>*, GenArgs);
  void (*pyf)(const cpx<T>*, cpx<T>*, const cpx<T>*, GenArgs);
  void (*pyi)(const cpx<T>*, cpx<T>*, const cpx<T>*, GenArgs);
  void (*pz)(cpx<T>*, const T*, const cpx<T>*, GenArgs, double*, unsigned*, double, double*);
  void (*p5)(const cpx<T>*, T*, const cpx<T>*, GenArgs);
};

template <typename T, int BM>
static GenKernels<T> gen_kernels_of() {
  return {p1_generic<T, BM>, py_generic<-1, T, BM>, py_generic<1, T, BM>, pz_generic<T, BM>, p5_generic<T, BM>};
}

template <typename T>
static GenKernels<T> gen_kernels(int bm) {
  if constexpr (sizeof(T) == 4) {
    switch (bm) {
      case 32: return gen_kernels_of<T, 32>();
      case 64: return gen_kernels_of<T, 64>();
      case 96: return gen_kernels_of<T, 96>();
      case 128: return gen_kernels_of<T, 128>();
      case 192: return gen_kernels_of<T, 192>();
      case 256: return gen_kernels_of<T, 256>();
      case 384: return gen_kernels_of<T, 384>();
      default: break;
    }
  }
  return gen_kernels_of<T, 0>();
}

// ---------------------------------------------------------------- energy

// E = 1/2 h^3 sum_r rho(r) V(r) in real space with FP64 accumulation: the
// energy of the tensor-core mode, whose Parseval sum over the spectrum of the
// TF32 split products would carry that spectrum's error twice
template <typename T>
__global__ void __launch_bounds__(256)
    energy_real_kernel(const T* __restrict__ rho, const T* __restrict__ V, long long n, double* partials,
                       unsigned* counter, double scale, double* E) {
  double acc = 0.0;
  const long long step = (long long)gridDim.x * blockDim.x;
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if constexpr (sizeof(T) == 4) {
    // FP32 products summed in groups of eight, each group added in FP64 (a
    // conversion per element would run at the FP64 rate)
    while (i < n) {
      float f = 0.f;
#pragma unroll
      for (int k = 0; k < 8; ++k, i += step)
        if (i < n) f = fmaf(rho[i], V[i], f);
      acc += (double)f;
    }
  } else {
    for (; i < n; i += step) acc += rho[i] * V[i];
  }
  energy_finish(acc, partials, counter, scale, E);
}

// ---------------------------------------------------------------- VJP term

// out = (accumulate ? out : 0) + h^3 * gE * V   (the dE/drho = h^3 V term of the VJP)
template <typename T>
__global__ void vjp_axpy_kernel(T* __restrict__ out, const T* __restrict__ V, const double* __restrict__ gE,
                                double h3, long long n, int accumulate) {
  const T a = (T)(h3 * __ldg(gE));
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x) {
    const T v = a * V[i];
    out[i] = accumulate ? out[i] + v : v;
  }
}

template <typename T>
cudaError_t launch_vjp_axpy(ps_plan_s* p, T* out, const T* V, const double* gE, bool accumulate,
                            cudaStream_t s) {
  const long long n = (long long)p->n[0] * p->n[1] * p->n[2];
  long long blocks = (n + 255) / 256;
  if (blocks > 152 * 16) blocks = 152 * 16;
  vjp_axpy_kernel<T><<<(int)blocks, 256, 0, s>>>(out, V, gE, p->h * p->h * p->h, n, accumulate ? 1 : 0);
  return cudaGetLastError();
}

template cudaError_t launch_vjp_axpy<float>(ps_plan_s*, float*, const float*, const double*, bool, cudaStream_t);
template cudaError_t launch_vjp_axpy<double>(ps_plan_s*, double*, const double*, const double*, bool,
                                             cudaStream_t);

// ---------------------------------------------------------------- host side

Stages factorize(int N, int pref) {
  Stages s;
  s.n = 0;
  int m = N;
  int twos = 0;
  while (m % 2 == 0) { m /= 2; ++twos; }
  if (pref == 1) {
    // radix 4 (and one radix 2 for an odd power): more, cheaper stages
    for (int i = 0; i < twos / 2; ++i) s.R[s.n++] = 4;
    if (twos % 2) s.R[s.n++] = 2;
  } else {
    // powers of two: as many radix-8 stages as possible, the rest as 4 or 2
    int eights = twos / 3, rest = twos % 3;
    if (rest == 1 && eights > 0) { --eights; s.R[s.n++] = 4; s.R[s.n++] = 4; rest = 0; }
    for (int i = 0; i < eights; ++i) s.R[s.n++] = 8;
    if (rest == 1) s.R[s.n++] = 2;
    if (rest == 2) s.R[s.n++] = 4;
  }
  for (int p = 3; m > 1; p += 2) {
    while (m % p == 0) { s.R[s.n++] = p; m /= p; }
    if (p * p > m && m > 1) { s.R[s.n++] = m; m = 1; }
  }
  int Ns = 1;
  for (int i = 0; i < s.n; ++i) {
    s.mg[i] = div_magic((unsigned)Ns);
    Ns *= s.R[i];
  }
  return s;
}

// Tile width (lines per CTA, a power of two <= tk0) of a generic pass and
// whether its twiddle table sits in shared memory: the widest tile whose two
// buffers and table leave room for three CTAs per SM (72 KB each), else the
// widest within the 200 KB a CTA may take, else without the table. Narrow
// tiles of long lines keep the SM busy: with two resident CTAs and global
// twiddles the generic kernels waited on their loads most of the time.
static int pick_tk(int rows, int twn, size_t csz, int tk0, int pad, int* ldt, size_t* smem, int* twn_out) {
  const size_t budgets[3] = {(size_t)72 * 1024, (size_t)200 * 1024, (size_t)200 * 1024};
  for (int pass = 0; pass < 3; ++pass) {
    const int tw = pass < 2 ? twn : 0;
    for (int tk = tk0; tk >= 1; tk /= 2) {
      const int l = tk + pad;
      const size_t b = (size_t)2 * rows * l * csz + (size_t)tw * csz;
      if (b <= budgets[pass]) {
        *ldt = l;
        *smem = b;
        *twn_out = tw;
        return tk;
      }
    }
  }
  return 0;
}

// rows of each shared-memory buffer of a generic pass: the transform length,
// the Bluestein length, and for the real-to-complex passes room for the half
// spectra (x first: N + 1 = L1/2 + 1 rows, or two of c rows for an odd L1;
// another first axis: two of c rows of the paired lines)
int gen_rows(const ps_plan_s* p, int pass) {
  const int axis = pass_axis(p, pass);
  const int N = xform_len(p, axis);
  int r = N;
  if (pass == P1 || pass == P5) r = axis == 0 ? N + 1 : 2 * p->c;
  if (p->blue[axis].M > r) r = p->blue[axis].M;
  return r;
}

template <typename T>
static GenArgs gen_args(const ps_plan_s* p, int pass) {
  GenArgs a;
  a.n1 = p->n[0]; a.n2 = p->n[1]; a.n3 = p->n[2];
  a.L1 = p->L[0]; a.L2 = p->L[1]; a.L3 = p->L[2];
  a.c = p->c; a.H2 = p->H[1]; a.H3 = p->H[2];
  a.ldc = (int)p->ldc;
  a.ldk = (int)p->ldk;
  a.tk = p->cfg[pass].tk; a.ldt = p->cfg[pass].ldt;
  const int axis = pass_axis(p, pass);
  a.N = xform_len(p, axis);
  a.tws = p->L[axis] / a.N;
  a.st = p->st[axis];
  a.bl = p->blue[axis];
  a.rows = gen_rows(p, pass);
  a.ltk = 0;
  while ((1 << a.ltk) < a.tk) ++a.ltk;
  a.twn = p->cfg[pass].twn;
  a.mn1 = div_magic((unsigned)a.n1);
  a.mc = div_magic((unsigned)a.c);
  a.mN1 = div_magic((unsigned)(a.N + 1));
  return a;
}

template <typename T>
cudaError_t configure_passes(ps_plan_s* p) {
  using C = cpx<T>;
  const size_t budget = 200 * 1024;
  // most lines per generic tile: the plan's schedule for the pass's axis
  // (ps_plan_set_axis_schedule, else ps_plan_set_schedule, or the autotuner),
  // else 16 (FP32) / 8 (FP64)
  const int tk_def = sizeof(T) == 4 ? 16 : 8;
  const int rows[5] = {gen_rows(p, P1), gen_rows(p, P2), gen_rows(p, P3), gen_rows(p, P4), gen_rows(p, P5)};
  for (int k = 0; k < 5; ++k) {
    PassCfg& cf = p->cfg[k];
    cf.threads = 256;
    cf.fast = 0;
    const int axis = pass_axis(p, k);
    const int Nk = xform_len(p, axis);
    const int tk0 = axis_tile(p, axis) > 0 ? axis_tile(p, axis) : tk_def;
    const int bm = sizeof(T) == 4 ? blue_regs_length(p->blue[axis].M, Nk) : 0;
    const int twn = p->blue[axis].M ? p->blue[axis].M : Nk;  // W_N, or W_M in Bluestein form
    // row pitch: tk + 1 for passes along x, whose tile loops transpose rows (a
    // pitch of tk would put a row's consecutive elements on one bank); tk
    // for passes along y and z, whose tile rows are contiguous runs
    cf.tk = pick_tk(rows[k], twn, sizeof(C), tk0, axis == 0 ? 1 : 0, &cf.ldt, &cf.gsmem, &cf.twn);
    cf.smem = cf.gsmem;
    cf.bm = bm;
    // Bluestein form: the transformed chirp and the chirp join the
    // shared-memory table when they fit within the same budget at this tile width
    const int M = p->blue[axis].M;
    if (M && cf.twn > 0) {
      const size_t ext = cf.gsmem + (size_t)(M + Nk) * sizeof(C);
      if (ext <= (cf.gsmem <= (size_t)72 * 1024 ? (size_t)72 * 1024 : budget)) {
        cf.gsmem = ext;
        cf.smem = ext;
        cf.twn = 2 * M + Nk;
      }
    }
    if (cf.tk == 0) {
      set_error("transform length %d needs more shared memory than a CTA has", rows[k]);
      return cudaErrorInvalidConfiguration;
    }
    // register-form Bluestein: as many threads as the widest step has tasks
    // (max(P, Q) x tk lines), so that no thread idles through steps 1 and 3
    if (bm > 0 && canonical_order(p)) {
      const int bp = blue_p(bm), tasks = std::max(bp, bm / bp) * cf.tk;
      if (tasks < 256) cf.threads = (tasks + 31) / 32 * 32;
    }
  }
  cudaError_t e;
  for (int k = -1; k < 5; ++k) {  // the Stockham kernels and those of each pass's Bluestein form
    const GenKernels<T> g = gen_kernels<T>(k < 0 ? 0 : p->cfg[k].bm);
    for (const void* f : {(const void*)g.p1, (const void*)g.pyf, (const void*)g.pyi, (const void*)g.pz,
                          (const void*)g.p5})
      if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)budget)) != cudaSuccess)
        return e;
  }
  p->fastord = 0;
  if (!canonical_order(p)) {
    // the generic kernels along strided axes (passes_ord.cu); energy
    // partials: one per CTA of the fused pass
    p->npart = ord_conv_ctas(p);
    if ((e = configure_ord<T>(p)) != cudaSuccess) return e;
    if constexpr (sizeof(T) == 4) {
      // x first (x, z, y): the specialised x kernels, and the y- and z-pass
      // kernels along z and y through strides, when all three middle passes have them
      if (p->ord[0] == 0) {
        if ((e = configure_fast_f32(p)) != cudaSuccess) return e;
        p->fastord = p->cfg[P2].fast && p->cfg[P3].fast && p->cfg[P4].fast;
        if (p->fastord) {
          const int ntk = (p->c + p->cfg[P3].tk - 1) / p->cfg[P3].tk;
          p->npart = std::max(p->npart, ntk * p->L[p->ord[1]]);
        }
      }
    }
    return cudaSuccess;
  }
  if constexpr (sizeof(T) == 4) {
    e = configure_fast_f32(p);
    if (e != cudaSuccess) return e;
  }
  // energy partials: one per CTA of the z pass
  const int ntk = (p->c + p->cfg[P3].tk - 1) / p->cfg[P3].tk;
  p->npart = ntk * p->L[1];
  return cudaSuccess;
}

template <typename T>
cudaError_t launch_solve(ps_plan_s* p, const T* rho, T* V, double* E, cudaStream_t s,
                         cudaEvent_t* ev) {
  using C = cpx<T>;
  if (!canonical_order(p) && !p->fastord) return launch_solve_ord<T>(p, rho, V, E, s, ev);
  C* A = static_cast<C*>(p->A);
  C* B = static_cast<C*>(p->B);
  const C* tw0 = static_cast<const C*>(p->tw[0]);
  const C* tw1 = static_cast<const C*>(p->tw[1]);
  const C* tw2 = static_cast<const C*>(p->tw[2]);
  const int nrows = p->n[1] * p->n[2];
  const double escale = 0.5 * p->h * p->h * p->h;

  // the x-pass kernels read and write 8-byte pairs of reals
  const bool a8 = ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(V)) & 7) == 0;
  // fused x/y passes: one kernel for P1 + P2 and one for P4 + P5 (A unused);
  // the forward one copies rows of rho in 16-byte pieces
  const bool xyf = p->xyfuse && ((reinterpret_cast<uintptr_t>(rho) | reinterpret_cast<uintptr_t>(V)) & 15) == 0;
  cudaError_t e;
  // the tensor-core z pass leaves the energy to a real-space sum after P5
  double* const Ez = p->tctab ? nullptr : E;
  auto energy_after = [&]() -> cudaError_t {
    if (!p->tctab || E == nullptr) return cudaSuccess;
    const long long npts = (long long)p->n[0] * p->n[1] * p->n[2];
    const long long want = (npts + 255) / 256;
    const int grid = (int)std::min<long long>(std::min<long long>(want, 1216), p->npart);
    energy_real_kernel<T><<<grid, 256, 0, s>>>(rho, V, npts, p->partials, p->counter, escale, E);
    return cudaGetLastError();
  };
  auto pass3 = [&]() -> cudaError_t {
    if (p->cfg[P3].fast) return launch_fast(p, P3, B, B, Ez, escale, s);
    GenArgs a = gen_args<T>(p, P3);
    dim3 g((p->c + a.tk - 1) / a.tk, p->L[1]);
    gen_kernels<T>(p->cfg[P3].bm).pz<<<g, p->cfg[P3].threads, p->cfg[P3].gsmem, s>>>(
        B, static_cast<const T*>(p->K), tw2, a, p->partials, p->counter, escale, E);
    return cudaGetLastError();
  };
  if (!xyf && a8 && p->chunks > 1) {
    // x and y passes chunk by chunk of z planes through the first chunk of A
    const int n3 = p->n[2];
    const int nz = (n3 + p->chunks - 1) / p->chunks;
    if (ev) cudaEventRecord(ev[0], s);
    for (int z0 = 0; z0 < n3; z0 += nz) {
      const int cz = std::min(nz, n3 - z0);
      if ((e = launch_fast_chunk(p, P1, rho, B, A, z0, cz, s)) != cudaSuccess) return e;
      if ((e = launch_fast_chunk(p, P2, rho, B, A, z0, cz, s)) != cudaSuccess) return e;
    }
    if (ev) cudaEventRecord(ev[1], s);
    if (ev) cudaEventRecord(ev[2], s);
    if ((e = pass3()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[3], s);
    for (int z0 = 0; z0 < n3; z0 += nz) {
      const int cz = std::min(nz, n3 - z0);
      if ((e = launch_fast_chunk(p, P4, V, B, A, z0, cz, s)) != cudaSuccess) return e;
      if ((e = launch_fast_chunk(p, P5, V, B, A, z0, cz, s)) != cudaSuccess) return e;
    }
    if ((e = energy_after()) != cudaSuccess) return e;
    if (ev) cudaEventRecord(ev[4], s);
    if (ev) cudaEventRecord(ev[5], s);
    return cudaGetLastError();
  }
  if (ev) cudaEventRecord(ev[0], s);
  // P1
  if (xyf) {
    if ((e = launch_xy(p, 0, rho, B, s)) != cudaSuccess) return e;
  } else if (p->cfg[P1].fast && a8) {
    if ((e = launch_fast(p, P1, rho, A, nullptr, 0.0, s)) != cudaSuccess) return e;
  } else {
    GenArgs a = gen_args<T>(p, P1);
    const int rpc = (p->L[0] % 2 == 0) ? a.tk : 2 * a.tk;  // odd L1: two real rows per line
    gen_kernels<T>(p->cfg[P1].bm).p1<<<(nrows + rpc - 1) / rpc, p->cfg[P1].threads, p->cfg[P1].gsmem, s>>>(
        rho, A, tw0, a);
  }
  if (ev) cudaEventRecord(ev[1], s);
  // P2
  if (xyf) {
    // done by the fused kernel above
  } else if (p->cfg[P2].fast) {
    if ((e = launch_fast(p, P2, A, B, nullptr, 0.0, s)) != cudaSuccess) return e;
  } else {
    GenArgs a = gen_args<T>(p, P2);
    dim3 g((p->c + a.tk - 1) / a.tk, p->n[2]);
    gen_kernels<T>(p->cfg[P2].bm).pyf<<<g, p->cfg[P2].threads, p->cfg[P2].gsmem, s>>>(A, B, tw1, a);
  }
  if (ev) cudaEventRecord(ev[2], s);
  // P3
  if ((e = pass3()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[3], s);
  // P4
  if (xyf) {
    if ((e = launch_xy(p, 1, B, V, s)) != cudaSuccess) return e;
  } else if (p->cfg[P4].fast) {
    if ((e = launch_fast(p, P4, B, A, nullptr, 0.0, s)) != cudaSuccess) return e;
  } else {
    GenArgs a = gen_args<T>(p, P4);
    dim3 g((p->c + a.tk - 1) / a.tk, p->n[2]);
    gen_kernels<T>(p->cfg[P4].bm).pyi<<<g, p->cfg[P4].threads, p->cfg[P4].gsmem, s>>>(B, A, tw1, a);
  }
  if (ev) cudaEventRecord(ev[4], s);
  // P5
  if (xyf) {
    // done by the fused kernel above
  } else if (p->cfg[P5].fast && a8) {
    if ((e = launch_fast(p, P5, A, V, nullptr, 0.0, s)) != cudaSuccess) return e;
  } else {
    GenArgs a = gen_args<T>(p, P5);
    const int rpc = (p->L[0] % 2 == 0) ? a.tk : 2 * a.tk;  // odd L1: two real rows per line
    gen_kernels<T>(p->cfg[P5].bm).p5<<<(nrows + rpc - 1) / rpc, p->cfg[P5].threads, p->cfg[P5].gsmem, s>>>(
        A, V, tw0, a);
  }
  if ((e = energy_after()) != cudaSuccess) return e;
  if (ev) cudaEventRecord(ev[5], s);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_x_pass(ps_plan_s* p, int pass, const void* src, void* dst, cudaStream_t s) {
  using C = cpx<T>;
  GenArgs a = gen_args<T>(p, pass);
  const int nrows = p->n[1] * p->n[2];
  const int rpc = (p->L[0] % 2 == 0) ? a.tk : 2 * a.tk;  // odd L1: two real rows per line
  const C* tw0 = static_cast<const C*>(p->tw[0]);
  if (pass == P1)
    gen_kernels<T>(p->cfg[P1].bm).p1<<<(nrows + rpc - 1) / rpc, p->cfg[P1].threads, p->cfg[P1].gsmem, s>>>(
        static_cast<const T*>(src), static_cast<C*>(dst), tw0, a);
  else
    gen_kernels<T>(p->cfg[P5].bm).p5<<<(nrows + rpc - 1) / rpc, p->cfg[P5].threads, p->cfg[P5].gsmem, s>>>(
        static_cast<const C*>(src), static_cast<T*>(dst), tw0, a);
  return cudaGetLastError();
}

template cudaError_t launch_x_pass<float>(ps_plan_s*, int, const void*, void*, cudaStream_t);
template cudaError_t launch_x_pass<double>(ps_plan_s*, int, const void*, void*, cudaStream_t);
template cudaError_t configure_passes<float>(ps_plan_s*);
template cudaError_t configure_passes<double>(ps_plan_s*);
template cudaError_t launch_solve<float>(ps_plan_s*, const float*, float*, double*, cudaStream_t,
                                         cudaEvent_t*);
template cudaError_t launch_solve<double>(ps_plan_s*, const double*, double*, double*, cudaStream_t,
                                          cudaEvent_t*);

}  // namespace ps
