// Specialised FP32 kernels for the y and z passes, power-of-two lengths and
// 96 = 24 x 4, 192 = 24 x 8 (radix-3 register DFTs).
//
// A CTA owns 16 lines adjacent in kx (the contiguous axis of A and B), so a
// warp reads or writes two runs of 16 consecutive complex numbers (2 x 128 B)
// per instruction; at L = 1024, 8 lines (64-byte runs), which keeps a CTA at
// 256 threads and 64 KB of shared memory. Each line of length L = P * Q is transformed by T = min(P, Q)
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
template <int P, int Q, int KIND, bool HALF, int TK>
__global__ void __launch_bounds__(TK*(P < Q ? P : Q),
                                  TK * (P < Q ? P : Q) <= 256 ? (KIND == 2 ? 2 : 3) : 1)
    k_strided(const void* src_v, void* dst_v, const float* __restrict__ K, const float2* __restrict__ tw,
              FastArgs a, double* partials, unsigned* counter, double escale, double* E) {
  pdl_wait();
  constexpr int L = P * Q;
  constexpr int T = P < Q ? P : Q;
  constexpr int NB = Q / T;            // step-1 transforms per thread
  constexpr int NK = P / T;            // step-3 transforms per thread
  constexpr int NA = HALF ? P / 2 : P; // a-range of the nonzero inputs / kept outputs
  extern __shared__ float2 sh[];       // [L][TK]: element e of line t at e * TK + t
  const float2* src = static_cast<const float2*>(src_v);
  float2* dst = static_cast<float2*>(dst_v);
  const int t = threadIdx.x % TK;
  const int j = threadIdx.x / TK;
  const int kx = blockIdx.x * TK + t;
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
      for (int k1 = 0; k1 < P; ++k1) sh[(b * P + k1) * TK + t] = y[u][k1];
    }
    __syncthreads();
#pragma unroll
    for (int v = 0; v < NK; ++v) {
      const int k1 = j + T * v;
#pragma unroll
      for (int b = 0; b < Q; ++b) X[v][b] = sh[(b * P + k1) * TK + t];
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
      for (int b = 0; b < Q; ++b) sh[(b * P + k1) * TK + t] = X[v][b];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int b = j + T * u;
      float2 y[P];
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) y[k1] = sh[(b * P + k1) * TK + t];
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

template <int P, int Q, int TK = kTK>
static const void* pick_strided(int kind, bool half) {
  if (kind == 0) return half ? (const void*)k_strided<P, Q, 0, true, TK> : (const void*)k_strided<P, Q, 0, false, TK>;
  if (kind == 1) return half ? (const void*)k_strided<P, Q, 1, true, TK> : (const void*)k_strided<P, Q, 1, false, TK>;
  return half ? (const void*)k_strided<P, Q, 2, true, TK> : (const void*)k_strided<P, Q, 2, false, TK>;
}

// L = 1024 takes 8 lines per CTA (256 threads, 64 KB of shared memory); the
// shorter lengths 16
const void* strided_kernel(int L, int kind, bool half, int* threads, size_t* smem, int* tk) {
  const void* fn = nullptr;
  int T = 0, TK = kTK;
  switch (L) {
    case 64: fn = pick_strided<8, 8>(kind, half); T = 8; break;
    case 128: fn = pick_strided<16, 8>(kind, half); T = 8; break;
    case 256: fn = pick_strided<16, 16>(kind, half); T = 16; break;
    case 512: fn = pick_strided<16, 32>(kind, half); T = 16; break;
    case 1024: fn = pick_strided<32, 32, 8>(kind, half); T = 32; TK = 8; break;
    default: return nullptr;
  }
  *threads = TK * T;
  *smem = (size_t)L * TK * sizeof(float2);
  *tk = TK;
  return fn;
}

// ---------------------------------------------------------------- pipelined z

// Persistent z pass on unpacked lines (L3 = 256, and 1024, where a packed pair
// of 32-point transforms would not fit in registers): TK lines per tile, tiles
// = (kx tile, ky row in the paired order) with kx fastest. The tile's n3 input
// rows land in the exchange (cp.async), the K^F octant slice in a stage of its
// own; the next tile's K^F slice is copied once the current one has been
// used, its input rows once the exchange has been read for the last time.
// With 8 lines per tile (64-byte exchange rows) the exchange has one padding
// row after every 32: the four line positions j of a warp then write rows 33
// apart, on alternate halves of the banks, instead of 32 apart on the same
// 16 banks (a 4-way conflict in the forward write and the inverse read).
template <int P, int Q, bool HALF, int TK>
__global__ void __launch_bounds__(TK*(P < Q ? P : Q), P > Q ? 512 / (TK * Q) : (P * Q >= 1024 ? 2 : 3))
    k_zpipe_u(const void*, void* line_v, const float* __restrict__ K, const float2* __restrict__ tw, FastArgs a,
              double* partials, unsigned* counter, double escale, double* E) {
  constexpr int L = P * Q;
  constexpr int T = P < Q ? P : Q;
  constexpr int NB = Q / T;
  constexpr int NK = P / T;
  constexpr int NA = HALF ? P / 2 : P;
  constexpr int ROWS = NA * Q;      // input rows of a line
  constexpr int KROWS = L / 2 + 1;  // rows of the K^F octant
  constexpr int RG = TK * 8 < 128 ? P : 0;  // exchange rows per padded group (0: no padding)
  static_assert(RG == 0 || (P == RG && Q == RG), "padded exchange: P = Q = rows per group");
  constexpr int PP = RG ? P + 1 : P;         // row pitch of b in the exchange (rows b * PP + k1)
  constexpr int QQ = RG ? Q + 1 : Q;         // row pitch of aa for the input rows b + Q aa
  constexpr int LP = RG ? L + L / RG : L;    // exchange rows including the padding
  extern __shared__ float2 sh[];    // exchange [LP][TK]; the K^F slice [KROWS][TK] floats; W_L^i, i < L
  float* const kstage = reinterpret_cast<float*>(sh + LP * TK);
  float2* const tws = reinterpret_cast<float2*>(kstage + ((KROWS * TK + 1) & ~1));
  for (int i = threadIdx.x; i < L; i += blockDim.x) tws[i] = __ldg(&tw[i]);  // before the first barrier
  float2* const base = static_cast<float2*>(line_v);
  const int t = threadIdx.x % TK;
  const int j = threadIdx.x / TK;
  const int ntk = a.ntk_loc;
  const int ntiles = ntk * a.L2;
  const long long es = a.src_elem;

  constexpr int NT = TK * T;
  constexpr int IPR = TK / 2;  // 16-byte pieces per input row
  constexpr int ISTEP = NT / IPR;
  static_assert(NT % IPR == 0 && ROWS % ISTEP == 0, "input copy shape");
  static_assert(RG == 0 || ISTEP % RG == 0, "padded input copy shape");
  constexpr int ISTEPP = RG ? ISTEP + ISTEP / RG : ISTEP;  // exchange rows per sweep, padding included
  const int irow0 = threadIdx.x / IPR;
  const long long igoff = (long long)irow0 * es + 2 * (threadIdx.x % IPR);
  const long long igstep = (long long)ISTEP * es;
  float2* const is0 = sh + (RG ? irow0 + irow0 / RG : irow0) * TK + 2 * (threadIdx.x % IPR);
  const int ivalid = a.nl - irow0;
  constexpr int KPR = TK / 4;  // 16-byte pieces per K^F row
  constexpr int KSTEP = NT / KPR;
  constexpr int KIT = (KROWS + KSTEP - 1) / KSTEP;
  const int krow0 = threadIdx.x / KPR;
  const long long kgoff = (long long)krow0 * a.kz_stride + 4 * (threadIdx.x % KPR);
  const long long kgstep = (long long)KSTEP * a.kz_stride;
  float* const ks0 = kstage + krow0 * TK + 4 * (threadIdx.x % KPR);

  const int dkt = gridDim.x % ntk, dyi = gridDim.x / ntk;
  auto step_tile = [&](int& kt, int& yi) {
    kt += dkt;
    yi += dyi;
    if (kt >= ntk) {
      kt -= ntk;
      ++yi;
    }
  };
  auto issue_input = [&](int kt, int yi) {
    const float2* src0 = base + paired_ky(yi, a.L2) * a.src_plane + (a.kt0 + kt) * TK;
    const float2* src = src0 + igoff;
#pragma unroll
    for (int i = 0; i < ROWS / ISTEP; ++i) {
      if (ISTEP * i < ivalid)
        cp_async16(is0 + i * ISTEPP * TK, src);
      else  // beyond the physical z rows: zeros (nothing is read)
        cp_async16_zero(is0 + i * ISTEPP * TK, src0);
      src += igstep;
    }
  };
  auto issue_k = [&](int kt, int yi) {
    const int ky = paired_ky(yi, a.L2);
    const int kyo = min(ky, a.L2 - ky);
    const float* src = K + (long long)kyo * a.ldk + (a.kt0 + kt) * TK + kgoff;
#pragma unroll
    for (int i = 0; i < KIT; ++i) {
      if ((i + 1) * KSTEP <= KROWS || krow0 + i * KSTEP < KROWS) cp_async16(ks0 + i * KSTEP * TK, src);
      src += kgstep;
    }
  };

  float eacc = 0.f;
  int tile = blockIdx.x;
  int kt = tile % ntk, yi = tile / ntk;
  int nkt = kt, nyi = yi;
  step_tile(nkt, nyi);
  if (tile < ntiles) issue_k(kt, yi);  // K^F is not written by any pass
  pdl_wait();
  if (tile < ntiles) issue_input(kt, yi);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    const int kx = (a.kt0 + kt) * TK + t;
    const bool valid = kx < a.c;
    const int ky = paired_ky(yi, a.L2);
    float2* line = base + ky * a.src_plane + kx;
    cp_async_wait_all();
    __syncthreads();  // this tile's input rows and K^F slice have landed

    float2 y[NB][P];
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int b = j + T * u;
#pragma unroll
      for (int aa = 0; aa < P; ++aa) {
        y[u][aa] = make_float2(0.f, 0.f);
        if (aa < NA && valid) y[u][aa] = sh[(b + QQ * aa) * TK + t];
      }
    }
    __syncthreads();  // inputs read: the space becomes the exchange
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int b = j + T * u;
      rdft<P, -1, HALF>(y[u]);
#pragma unroll
      for (int k1 = 1; k1 < P; ++k1) y[u][k1] = cmulf(y[u][k1], tws[b * k1]);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) sh[(b * PP + k1) * TK + t] = y[u][k1];
    }
    __syncthreads();
    float2 X[NK][Q];
    float e1 = 0.f;
#pragma unroll
    for (int v = 0; v < NK; ++v) {
      const int k1 = j + T * v;
#pragma unroll
      for (int b = 0; b < Q; ++b) X[v][b] = sh[(b * PP + k1) * TK + t];
      rdft<Q, -1, false>(X[v]);
      // V^F = K^F rho^F on the even octant of K^F; energy sum K |rho^F|^2
#pragma unroll
      for (int k2 = 0; k2 < Q; ++k2) {
        const int kz = k1 + P * k2;
        const int kzo = kz <= L / 2 ? kz : L - kz;
        const float kk = valid ? kstage[kzo * TK + t] : 0.f;
        const float2 x = X[v][k2];
        e1 = fmaf(kk, x.x * x.x + x.y * x.y, e1);
        X[v][k2] = make_float2(kk * x.x, kk * x.y);
      }
      rdft<Q, 1, false>(X[v]);
#pragma unroll
      for (int b = 1; b < Q; ++b) X[v][b] = cmulcf(X[v][b], tws[b * k1]);
    }
    eacc += e1 * ((kx == 0 || 2 * kx == a.L1) ? 1.f : 2.f);
    __syncthreads();  // the forward exchange and the K^F slice have been read
    if (next < ntiles) issue_k(nkt, nyi);
    cp_async_commit();
#pragma unroll
    for (int v = 0; v < NK; ++v) {
      const int k1 = j + T * v;
#pragma unroll
      for (int b = 0; b < Q; ++b) sh[(b * PP + k1) * TK + t] = X[v][b];
    }
    __syncthreads();
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int b = j + T * u;
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) y[u][k1] = sh[(b * PP + k1) * TK + t];
    }
    __syncthreads();  // the exchange has been read: the next tile's rows may land in it
    if (next < ntiles) issue_input(nkt, nyi);
    cp_async_commit();
#pragma unroll
    for (int u = 0; u < NB; ++u) {
      const int b = j + T * u;
      rdft<P, 1, false>(y[u]);
      if (valid) {
#pragma unroll
        for (int aa = 0; aa < NA; ++aa)
          if (b + Q * aa < a.nl) line[(long long)(b + Q * aa) * es] = y[u][aa];
      }
    }
    kt = nkt;
    yi = nyi;
    step_tile(nkt, nyi);
  }
  cp_async_wait_all();
  if (E != nullptr) energy_finish_f32(eacc, partials, counter, escale, E);
}

const void* zpipe_u_kernel(int L, bool half, int* threads, size_t* smem, int* tk) {
  const void* fn = nullptr;
  int T = 0, TK = 8;
  switch (L) {
    case 96:  // 24 x 4 and 24 x 8 (radix-3 register DFTs), 16 lines per tile
      fn = half ? (const void*)k_zpipe_u<24, 4, true, 16> : (const void*)k_zpipe_u<24, 4, false, 16>;
      T = 4;
      TK = 16;
      break;
    case 192:
      fn = half ? (const void*)k_zpipe_u<24, 8, true, 16> : (const void*)k_zpipe_u<24, 8, false, 16>;
      T = 8;
      TK = 16;
      break;
    case 1024: fn = half ? (const void*)k_zpipe_u<32, 32, true, 8> : (const void*)k_zpipe_u<32, 32, false, 8>; T = 32;
      break;
    default: return nullptr;
  }
  *threads = TK * T;
  const int LP = TK * 8 < 128 ? L + L / T : L;  // exchange rows, with the kernel's padding rows
  *smem = (size_t)LP * TK * sizeof(float2) + (size_t)(((L / 2 + 1) * TK + 1) & ~1) * sizeof(float) +
          (size_t)L * sizeof(float2);
  *tk = TK;
  return fn;
}

// ---------------------------------------------------------------- pipelined y

// Persistent y pass (KIND 0 forward, 1 inverse), 16 lines per tile, tiles =
// (kx tile, z plane) with kx fastest. The shared-memory tile serves twice: as
// the landing area of the tile's input rows (copied with cp.async) and as the
// exchange of the four-step transform. Once a tile's exchange has been read,
// the next tile's rows are copied in while the last transform step and the
// stores of the current tile run. With 8 lines per tile (64-byte rows) the
// exchange has one padding row after every 32, as in the L = 1024 z kernel:
// the forward write and the inverse read of a warp then fall on alternate
// bank halves instead of 4-way on the same 16 banks. The input rows keep the
// unpadded layout (they are read before the exchange is written).
template <int P, int Q, int KIND, bool HALF, int TK>
__global__ void __launch_bounds__(TK*(P < Q ? P : Q), P > Q ? 512 / (TK * Q) : (P * Q >= 512 ? 2 : 3))
    k_ypipe(const void* src_v, void* dst_v, const float*, const float2* __restrict__ tw, FastArgs a, double*,
            unsigned*, double, double*) {
  pdl_wait();
  constexpr int L = P * Q;
  constexpr int T = P < Q ? P : Q;
  constexpr int NB = Q / T;
  constexpr int NK = P / T;
  constexpr int NA = HALF ? P / 2 : P;
  constexpr int ROWS = KIND == 0 ? NA * Q : L;  // input rows of a line
  constexpr int RG = TK * 8 < 128 ? P : 0;      // exchange rows per padded group (0: no padding)
  static_assert(RG == 0 || (P == RG && Q == RG), "padded exchange: P = Q = rows per group");
  constexpr int PP = RG ? P + 1 : P;             // row pitch of b in the exchange (rows b * PP + k1)
  extern __shared__ float2 sh[];               // inputs [ROWS][TK]; later, in the same space, the exchange [L + L / RG][TK]
  const float2* src = static_cast<const float2*>(src_v);
  float2* dst = static_cast<float2*>(dst_v);
  const int t = threadIdx.x % TK;
  const int j = threadIdx.x / TK;
  const int ntk = a.ntk_loc;  // kx tiles a.kt0 .. a.kt0 + ntk - 1
  const int ntiles = ntk * (int)a.nrows;  // nrows = number of z planes here

  // the input copy: ROWS rows of TK float2 in 16-byte pieces, a fixed number
  // of sweeps of the CTA, per-thread offsets computed once
  constexpr int NT = TK * T;
  constexpr int IPR = TK / 2;
  constexpr int ISTEP = NT / IPR;
  static_assert(NT % IPR == 0 && ROWS % ISTEP == 0, "input copy shape");
  const int irow0 = threadIdx.x / IPR;
  const long long igoff = (long long)irow0 * a.src_elem + 2 * (threadIdx.x % IPR);
  const long long igstep = (long long)ISTEP * a.src_elem;
  float2* const is0 = sh + irow0 * TK + 2 * (threadIdx.x % IPR);
  const int ivalid = a.nl - irow0;  // sweep i copies a physical row iff ISTEP * i < ivalid
  auto plane = [&](int zi) { return a.rev ? (int)a.nrows - 1 - zi : zi; };
  auto prefetch = [&](int kt, int zi) {
    const float2* sp0 = src + (long long)plane(zi) * a.src_plane + (a.kt0 + kt) * TK;
    const float2* sp = sp0 + igoff;
#pragma unroll
    for (int i = 0; i < ROWS / ISTEP; ++i) {
      if (KIND == 1 || ISTEP * i < ivalid)
        cp_async16(is0 + i * ISTEP * TK, sp);
      else  // beyond the physical rows of the plane: zeros
        cp_async16_zero(is0 + i * ISTEP * TK, sp0);
      sp += igstep;
    }
  };
  // tile = kt + ntk * zi (kx tile fastest); the CTA steps by gridDim.x tiles
  const int dkt = gridDim.x % ntk, dzi = gridDim.x / ntk;
  auto step_tile = [&](int& kt, int& zi) {
    kt += dkt;
    zi += dzi;
    if (kt >= ntk) {
      kt -= ntk;
      ++zi;
    }
  };

  int tile = blockIdx.x;
  int kt = tile % ntk, zi = tile / ntk;
  int nkt = kt, nzi = zi;
  step_tile(nkt, nzi);
  if (tile < ntiles) prefetch(kt, zi);
  cp_async_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    const int kx = (a.kt0 + kt) * TK + t;
    const bool valid = kx < a.c;
    float2* d = dst + (long long)plane(zi) * a.dst_plane + kx;
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
          if (aa < NA && valid) y[u][aa] = sh[(b + Q * aa) * TK + t];
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
        for (int k1 = 0; k1 < P; ++k1) sh[(b * PP + k1) * TK + t] = y[u][k1];
      }
      __syncthreads();
#pragma unroll
      for (int v = 0; v < NK; ++v) {
        const int k1 = j + T * v;
#pragma unroll
        for (int b = 0; b < Q; ++b) X[v][b] = sh[(b * PP + k1) * TK + t];
      }
      __syncthreads();  // exchange read: the next tile's rows may land
      if (next < ntiles) prefetch(nkt, nzi);
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
          X[v][k2] = valid ? sh[(k1 + P * k2) * TK + t] : make_float2(0.f, 0.f);
      }
      __syncthreads();  // inputs read: the tile becomes the exchange
#pragma unroll
      for (int v = 0; v < NK; ++v) {
        const int k1 = j + T * v;
        rdft<Q, 1, false>(X[v]);
#pragma unroll
        for (int b = 1; b < Q; ++b) X[v][b] = cmulcf(X[v][b], __ldg(&tw[b * k1]));
#pragma unroll
        for (int b = 0; b < Q; ++b) sh[(b * PP + k1) * TK + t] = X[v][b];
      }
      __syncthreads();
      float2 y[NB][P];
#pragma unroll
      for (int u = 0; u < NB; ++u) {
        const int b = j + T * u;
#pragma unroll
        for (int k1 = 0; k1 < P; ++k1) y[u][k1] = sh[(b * PP + k1) * TK + t];
      }
      __syncthreads();  // exchange read: the next tile's rows may land
      if (next < ntiles) prefetch(nkt, nzi);
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
    kt = nkt;
    zi = nzi;
    step_tile(nkt, nzi);
  }
  cp_async_wait_all();
}

template <int P, int Q, int TK = kTK>
static const void* pick_ypipe(int kind, bool half) {
  if (kind == 0) return half ? (const void*)k_ypipe<P, Q, 0, true, TK> : (const void*)k_ypipe<P, Q, 0, false, TK>;
  return half ? (const void*)k_ypipe<P, Q, 1, true, TK> : (const void*)k_ypipe<P, Q, 1, false, TK>;
}

const void* ypipe_kernel(int L, int kind, bool half, int* threads, size_t* smem, int* tk) {
  const void* fn = nullptr;
  int T = 0, TK = kTK;
  switch (L) {
    case 96: fn = pick_ypipe<24, 4>(kind, half); T = 4; break;    // 24 x 4 (radix-3 register DFTs)
    case 192: fn = pick_ypipe<24, 8>(kind, half); T = 8; break;   // 24 x 8
    case 256: fn = pick_ypipe<16, 16>(kind, half); T = 16; break;
    case 512: fn = pick_ypipe<16, 32>(kind, half); T = 16; break;
    case 1024: fn = pick_ypipe<32, 32, 8>(kind, half); T = 32; TK = 8; break;
    default: return nullptr;
  }
  *threads = TK * T;
  const int LP = TK * 8 < 128 ? L + L / T : L;  // exchange rows, with the kernel's padding rows
  *smem = (size_t)LP * TK * sizeof(float2);
  *tk = TK;
  return fn;
}

}  // namespace ps
