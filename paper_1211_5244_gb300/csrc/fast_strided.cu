// Specialised FP32 kernels for the y and z passes, power-of-two lengths.
//
// A CTA owns 16 lines adjacent in kx (the contiguous axis of A and B), so a
// warp reads or writes two runs of 16 consecutive complex numbers (2 x 128 B)
// per instruction. Each line of length L = P * Q is transformed by T = min(P, Q)
// threads with the four-step factorisation
//     X[k1 + P k2] = sum_b W_Q^{b k2} W_L^{b k1} sum_a x[b + Q a] W_P^{a k1},
// step 1 (P-point DFTs over a) and step 3 (Q-point DFTs over b) in registers,
// one exchange through shared memory between them. With zero padding (§3)
// the inputs x[b + Q a] with a >= P/2 are zero and are never loaded; on the
// inverse, outputs with a >= P/2 are never formed. The z pass runs the
// forward transform, the K^F multiplication (Eq. 3) and the inverse in one
// kernel: the inverse's first step needs exactly the k1 values the forward's
// last step left in each thread, so the spectrum never leaves registers.
#include "fft_fast.cuh"
#include "fft_regs.cuh"
#include "reduce.cuh"

namespace ps {

using regs::rdft;

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 cmulcf(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

constexpr int kTK = 16;  // lines per CTA

// z pass: rows ky and L2 - ky read the same row of the K^F octant; launch
// them from adjacent CTA rows (y = 0 -> ky = 0, y = 1 -> ky = L2/2, then
// pairs p, L2 - p) so the second read hits L2.
template <int P, int Q, int KIND, bool HALF>
__global__ void __launch_bounds__(kTK*(P < Q ? P : Q),
                                  kTK * (P < Q ? P : Q) <= 256 ? (KIND == 2 ? 2 : 3) : 1)
    k_strided(const void* src_v, void* dst_v, const float* __restrict__ K, const float2* __restrict__ tw,
              FastArgs a, double* partials, unsigned* counter, double escale, double* E) {
  pdl_wait();
  constexpr int L = P * Q;
  constexpr int T = P < Q ? P : Q;
  constexpr int NB = Q / T;            // step-1 transforms per thread
  constexpr int NK = P / T;            // step-3 transforms per thread
  constexpr int NA = HALF ? P / 2 : P; // a-range of the nonzero inputs / kept outputs
  extern __shared__ float2 sh[];       // [L][kTK]: element e of line t at e * kTK + t
  const float2* src = static_cast<const float2*>(src_v);
  float2* dst = static_cast<float2*>(dst_v);
  const int t = threadIdx.x % kTK;
  const int j = threadIdx.x / kTK;
  const int kx = blockIdx.x * kTK + t;
  const bool valid = kx < a.c;
  const int yblk = KIND == 2 ? paired_ky(blockIdx.y, a.L2)
                             : (a.rev ? (int)(gridDim.y - 1 - blockIdx.y) : (int)blockIdx.y);
  const float2* s = src + yblk * a.src_plane + kx;
  float2* d = dst + yblk * a.dst_plane + kx;
  float2 X[NK][Q];  // X[v][k2] = spectrum at k1 + P k2, k1 = j + T v

  if constexpr (KIND == 0 || KIND == 2) {
    float2 y[NB][P];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int b = j + T * u;
#pragma unroll
      for (int aa = 0; aa < P; ++aa) {
        y[u][aa] = make_float2(0.f, 0.f);
        if (aa < NA && valid && b + Q * aa < a.nl) y[u][aa] = s[(long long)(b + Q * aa) * a.src_elem];
      }
    }
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int b = j + T * u;
      rdft<P, -1, HALF>(y[u]);
#pragma unroll
      for (int k1 = 1; k1 < P; ++k1) y[u][k1] = cmulf(y[u][k1], __ldg(&tw[b * k1]));
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) sh[(b * P + k1) * kTK + t] = y[u][k1];
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < NK; ++v) {
      const int k1 = j + T * v;
#pragma unroll
      for (int b = 0; b < Q; ++b) X[v][b] = sh[(b * P + k1) * kTK + t];
      rdft<Q, -1, false>(X[v]);
    }
  } else {
#pragma unroll
    for (int v = 0; v < NK; ++v) {
      const int k1 = j + T * v;
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2)
        X[v][k2] = valid ? s[(long long)(k1 + P * k2) * a.src_elem] : make_float2(0.f, 0.f);
    }
  }

  if constexpr (KIND == 0) {
    if (valid) {
#pragma unroll
      for (int v = 0; v < NK; ++v) {
        const int k1 = j + T * v;
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) d[(long long)(k1 + P * k2) * a.dst_elem] = X[v][k2];
      }
    }
    return;
  } else {
    float eacc = 0.f;
    if constexpr (KIND == 2) {
      // V^F = K^F rho^F on the even octant of K^F; energy sum w(kx) K |rho^F|^2
      const int ky = yblk;
      const int kyo = min(ky, a.L2 - ky);
      const float* Kp = K + (long long)kyo * a.ldk + kx;
#pragma unroll
      for (int v = 0; v < NK; ++v) {
        const int k1 = j + T * v;
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2) {
          const int kz = k1 + P * k2;
          const int kzo = kz <= L / 2 ? kz : L - kz;
          const float kk = valid ? __ldg(&Kp[(long long)kzo * a.kz_stride]) : 0.f;
          const float2 x = X[v][k2];
          eacc = fmaf(kk, x.x * x.x + x.y * x.y, eacc);
          X[v][k2] = make_float2(kk * x.x, kk * x.y);
        }
      }
      eacc *= (kx == 0 || 2 * kx == a.L1) ? 1.f : 2.f;
    }
    // inverse: Q-point transforms over k2, conjugate twiddles, exchange,
    // P-point transforms over k1
#pragma unroll
    for (int v = 0; v < NK; ++v) {
      const int k1 = j + T * v;
      rdft<Q, 1, false>(X[v]);
#pragma unroll
      for (int b = 1; b < Q; ++b) X[v][b] = cmulcf(X[v][b], __ldg(&tw[b * k1]));
    }
    if constexpr (KIND == 2) __syncthreads();  // the forward exchange has been read
#pragma unroll
    for (int v = 0; v < NK; ++v) {
      const int k1 = j + T * v;
#pragma unroll
      for (int b = 0; b < Q; ++b) sh[(b * P + k1) * kTK + t] = X[v][b];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int b = j + T * u;
      float2 y[P];
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) y[k1] = sh[(b * P + k1) * kTK + t];
      rdft<P, 1, false>(y);
      if (valid) {
#pragma unroll
        for (int aa = 0; aa < NA; ++aa)
          if (b + Q * aa < a.nl) d[(long long)(b + Q * aa) * a.dst_elem] = y[aa];
      }
    }
    if constexpr (KIND == 2) {
      if (E != nullptr) energy_finish_f32(eacc, partials, counter, escale, E);
    }
  }
}

template <int P, int Q>
static const void* pick_strided(int kind, bool half) {
  if (kind == 0) return half ? (const void*)k_strided<P, Q, 0, true> : (const void*)k_strided<P, Q, 0, false>;
  if (kind == 1) return half ? (const void*)k_strided<P, Q, 1, true> : (const void*)k_strided<P, Q, 1, false>;
  return half ? (const void*)k_strided<P, Q, 2, true> : (const void*)k_strided<P, Q, 2, false>;
}

const void* strided_kernel(int L, int kind, bool half, int* threads, size_t* smem) {
  const void* fn = nullptr;
  int T = 0;
  switch (L) {
    case 64: fn = pick_strided<8, 8>(kind, half); T = 8; break;
    case 128: fn = pick_strided<16, 8>(kind, half); T = 8; break;
    case 256: fn = pick_strided<16, 16>(kind, half); T = 16; break;
    case 512: fn = pick_strided<16, 32>(kind, half); T = 16; break;
    case 1024: fn = pick_strided<32, 32>(kind, half); T = 32; break;
    default: return nullptr;
  }
  *threads = kTK * T;
  *smem = (size_t)L * kTK * sizeof(float2);
  return fn;
}

// ---------------------------------------------------------------- pipelined y

// Persistent y pass (KIND 0 forward, 1 inverse), 16 lines per tile, tiles =
// (kx tile, z plane) with kx fastest. The shared-memory tile serves twice: as
// the landing area of the tile's input rows (copied with cp.async) and as the
// exchange of the four-step transform. Once a tile's exchange has been read,
// the next tile's rows are copied in while the last transform step and the
// stores of the current tile run.
template <int P, int Q, int KIND, bool HALF>
__global__ void __launch_bounds__(kTK*(P < Q ? P : Q), P * Q >= 512 ? 2 : 3)
    k_ypipe(const void* src_v, void* dst_v, const float*, const float2* __restrict__ tw, FastArgs a, double*,
            unsigned*, double, double*) {
  pdl_wait();
  constexpr int L = P * Q;
  constexpr int T = P < Q ? P : Q;
  constexpr int NB = Q / T;
  constexpr int NK = P / T;
  constexpr int NA = HALF ? P / 2 : P;
  constexpr int ROWS = KIND == 0 ? NA * Q : L;  // input rows of a line
  extern __shared__ float2 sh[];               // [L][kTK]
  const float2* src = static_cast<const float2*>(src_v);
  float2* dst = static_cast<float2*>(dst_v);
  const int t = threadIdx.x % kTK;
  const int j = threadIdx.x / kTK;
  const int ntk = a.ntk_loc;  // kx tiles a.kt0 .. a.kt0 + ntk - 1
  const int ntiles = ntk * (int)a.nrows;  // nrows = number of z planes here

  auto prefetch = [&](int tile) {
    const int kx0 = (a.kt0 + tile % ntk) * kTK;
    const int zp = a.rev ? (int)a.nrows - 1 - tile / ntk : tile / ntk;
    const float2* sp = src + (long long)zp * a.src_plane + kx0;
    for (int q = threadIdx.x; q < ROWS * (kTK / 2); q += blockDim.x) {
      const int row = q / (kTK / 2), part = q % (kTK / 2);
      if (KIND == 1 || row < a.nl)
        cp_async16(sh + row * kTK + 2 * part, sp + (long long)row * a.src_elem + 2 * part);
      else  // beyond the physical rows of the plane: zeros
        cp_async16_zero(sh + row * kTK + 2 * part, sp);
    }
  };

  int tile = blockIdx.x;
  if (tile < ntiles) prefetch(tile);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    const int kx = (a.kt0 + tile % ntk) * kTK + t;
    const bool valid = kx < a.c;
    const int zp = a.rev ? (int)a.nrows - 1 - tile / ntk : tile / ntk;
    float2* d = dst + (long long)zp * a.dst_plane + kx;
    cp_async_wait_all();
    __syncthreads();  // the tile's rows have landed
    float2 X[NK][Q];
    if constexpr (KIND == 0) {
      float2 y[NB][P];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int b = j + T * u;
#pragma unroll
        for (int aa = 0; aa < P; ++aa) {
          y[u][aa] = make_float2(0.f, 0.f);
          if (aa < NA && valid) y[u][aa] = sh[(b + Q * aa) * kTK + t];
        }
      }
      __syncthreads();  // inputs read: the tile becomes the exchange
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int b = j + T * u;
        rdft<P, -1, HALF>(y[u]);
#pragma unroll
        for (int k1 = 1; k1 < P; ++k1) y[u][k1] = cmulf(y[u][k1], __ldg(&tw[b * k1]));
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) sh[(b * P + k1) * kTK + t] = y[u][k1];
      }
      __syncthreads();
#pragma unroll
      for (int v = 0; v < NK; ++v) {
        const int k1 = j + T * v;
#pragma unroll
        for (int b = 0; b < Q; ++b) X[v][b] = sh[(b * P + k1) * kTK + t];
      }
      __syncthreads();  // exchange read: the next tile's rows may land
      if (next < ntiles) prefetch(next);
      cp_async_commit();
#pragma unroll
      for (int v = 0; v < NK; ++v) {
        const int k1 = j + T * v;
        rdft<Q, -1, false>(X[v]);
        if (valid) {
#pragma unroll
          for (int k2 = 0; k2 < Q; ++k2) d[(long long)(k1 + P * k2) * a.dst_elem] = X[v][k2];
        }
      }
    } else {
#pragma unroll
      for (int v = 0; v < NK; ++v) {
        const int k1 = j + T * v;
#pragma unroll
        for (int k2 = 0; k2 < Q; ++k2)
          X[v][k2] = valid ? sh[(k1 + P * k2) * kTK + t] : make_float2(0.f, 0.f);
      }
      __syncthreads();  // inputs read: the tile becomes the exchange
#pragma unroll
      for (int v = 0; v < NK; ++v) {
        const int k1 = j + T * v;
        rdft<Q, 1, false>(X[v]);
#pragma unroll
        for (int b = 1; b < Q; ++b) X[v][b] = cmulcf(X[v][b], __ldg(&tw[b * k1]));
#pragma unroll
        for (int b = 0; b < Q; ++b) sh[(b * P + k1) * kTK + t] = X[v][b];
      }
      __syncthreads();
      float2 y[NB][P];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int b = j + T * u;
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) y[u][k1] = sh[(b * P + k1) * kTK + t];
      }
      __syncthreads();  // exchange read: the next tile's rows may land
      if (next < ntiles) prefetch(next);
      cp_async_commit();
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int b = j + T * u;
        rdft<P, 1, false>(y[u]);
        if (valid) {
#pragma unroll
          for (int aa = 0; aa < NA; ++aa)
            if (b + Q * aa < a.nl) d[(long long)(b + Q * aa) * a.dst_elem] = y[u][aa];
        }
      }
    }
  }
  cp_async_wait_all();
}

template <int P, int Q>
static const void* pick_ypipe(int kind, bool half) {
  if (kind == 0) return half ? (const void*)k_ypipe<P, Q, 0, true> : (const void*)k_ypipe<P, Q, 0, false>;
  return half ? (const void*)k_ypipe<P, Q, 1, true> : (const void*)k_ypipe<P, Q, 1, false>;
}

const void* ypipe_kernel(int L, int kind, bool half, int* threads, size_t* smem) {
  const void* fn = nullptr;
  int T = 0;
  switch (L) {
    case 256: fn = pick_ypipe<16, 16>(kind, half); T = 16; break;
    case 512: fn = pick_ypipe<16, 32>(kind, half); T = 16; break;
    default: return nullptr;
  }
  *threads = kTK * T;
  *smem = (size_t)L * kTK * sizeof(float2);
  return fn;
}

}  // namespace ps
