// z pass (forward transform, K^F multiply, inverse transform) for L3 = P * 2T
// (P = T = 8: 128, P = T = 16: 512; P = 12, T = 16: 384) on packed FP32x2 pairs.
//
// Same four-step factorisation as fast_strided.cu with P rows, Q = 2T columns
// and T threads per line, but every thread carries its two step-1 transforms
// (b = j and b = j + T) as one structure-of-arrays pair, so their additions
// run as FP32x2 instructions. With P < T (L = 384) the threads j >= P hold no
// row in steps 2 and 3 and wait at the barriers. The exchange stores each pair as one 16-byte
// word. The Q-point step splits into a radix-2 stage across the pair
// (lanes b and b + T) and two T-point transforms that again form a pair
// (even and odd outputs). The same pairing returns in the inverse. The
// twiddles W_L^{b k1} of both lanes come from one float4 table,
// tw4[r * P + c] = (Re W^{rc}, Re W^{(r+T)c}, Im W^{rc}, Im W^{(r+T)c}), r < T, c < P,
// used as (r, c) = (j, k1) by the forward and (b, j) by the inverse step.
#include "fft_fast.cuh"
#include "fft_soa.cuh"
#include "reduce.cuh"

namespace ps {

using soa::c2;
using soa::cmul_pair;
using soa::pack;
using soa::unpack;

namespace {


// radix-2 DIF stage of a 2T-point forward DFT across the lanes of z[b]
// (lanes x_b, x_{b+T}): z[b] <- (x_b + x_{b+T}, (x_b - x_{b+T}) W_{2T}^b)
template <int T, int B>
__device__ __forceinline__ void dif_lanes(c2 (&z)[T]) {
  const float2 x0 = make_float2(z[B].re.x, z[B].im.x), x1 = make_float2(z[B].re.y, z[B].im.y);
  const float2 s = make_float2(x0.x + x1.x, x0.y + x1.y);
  const float2 d = regs::twc<2 * T, B, -1>(make_float2(x0.x - x1.x, x0.y - x1.y));
  z[B] = {make_float2(s.x, d.x), make_float2(s.y, d.y)};
}
template <int T, int... B>
__device__ __forceinline__ void dif_all(c2 (&z)[T], std::integer_sequence<int, B...>) {
  (dif_lanes<T, B>(z), ...);
}

// radix-2 DIT stage of a 2T-point inverse DFT across the lanes of z[b]
// (lanes E_b, O_b): z[b] <- (E_b + W_{2T}^{-b} O_b, E_b - W_{2T}^{-b} O_b)
template <int T, int B>
__device__ __forceinline__ void dit_lanes(c2 (&z)[T]) {
  const float2 e = make_float2(z[B].re.x, z[B].im.x);
  const float2 o = regs::twc<2 * T, B, 1>(make_float2(z[B].re.y, z[B].im.y));
  z[B] = {make_float2(e.x + o.x, e.x - o.x), make_float2(e.y + o.y, e.y - o.y)};
}
template <int T, int... B>
__device__ __forceinline__ void dit_all(c2 (&z)[T], std::integer_sequence<int, B...>) {
  (dit_lanes<T, B>(z), ...);
}

}  // namespace

// ---------------------------------------------------------------- pipelined

// Persistent z pass with TK lines per tile (8 by default, 16 as a schedule
// choice of the autotuner): each CTA walks tiles (kx tile fastest, then the paired ky
// rows) and copies the next tile's n3 input rows and its K^F octant slice into
// shared memory with cp.async while it computes the current tile, so the
// global-load latency of one tile overlaps the arithmetic of the previous one.
template <int T, int P, bool HALF, int TK>
__global__ void __launch_bounds__(TK * T, 512 / (TK * T))
    k_zconv_pipe(const void*, void* line_v, const float* __restrict__ K, const float4* __restrict__ tw4,
                 FastArgs a, double* partials, unsigned* counter, double escale, double* E) {
  constexpr int Q = 2 * T, L = P * Q;
  static_assert(P <= T, "a thread holds at most one row of steps 2 and 3");
  constexpr int NA = HALF ? P / 2 : P;
  constexpr int ROWS = NA * Q;          // input rows per line (n3)
  constexpr int KROWS = L / 2 + 1;      // rows of the K^F octant
  // 16 lines per tile: the next tile's input rows land in a stage of their own
  // as soon as the current ones are in registers. 8 lines per tile: they land
  // in the exchange buffer once its last use in the tile has been read, which
  // keeps a CTA at 42 KB of shared memory (four CTAs per SM).
  constexpr bool SEP = TK == 16;
  extern __shared__ float4 smem4[];
  float4* sh4 = smem4;                                              // exchange [T * P][TK]
  float2* stage = SEP ? reinterpret_cast<float2*>(smem4 + T * P * TK)  // inputs [ROWS][TK]
                      : reinterpret_cast<float2*>(smem4);
  float* kstage = SEP ? reinterpret_cast<float*>(stage + ROWS * TK)    // K^F [KROWS][TK]
                      : reinterpret_cast<float*>(smem4 + T * P * TK);
  // 8 lines per tile: the paired twiddle table also sits in shared memory,
  // rows padded to P + 1 so that the 4 rows a warp reads at once fall on
  // different banks (16 lines per tile read it through L1)
  float4* tws = reinterpret_cast<float4*>(kstage + KROWS * TK);
  if constexpr (!SEP) {
    for (int i = threadIdx.x; i < T * P; i += blockDim.x) tws[(i / P) * (P + 1) + i % P] = __ldg(&tw4[i]);
  }
  auto twid = [&](int r, int c) { return SEP ? __ldg(&tw4[r * P + c]) : tws[r * (P + 1) + c]; };
  const int t = threadIdx.x % TK;
  const int j = threadIdx.x / TK;
  auto xi = [](int r, int c) { return (r * P + c) * TK; };  // exchange slot (r, c) of line t: xi(r, c) + t
  const int ntk = a.ntk_loc;  // kx tiles a.kt0 .. a.kt0 + ntk - 1
  const int ntiles = ntk * a.L2;
  float2* const base = static_cast<float2*>(line_v);
  const long long es = a.src_elem;

  // Copies of a tile's rows, with trip counts fixed at compile time and the
  // per-thread offsets computed once: the input rows (n3 rows of TK float2,
  // 16-byte pieces) and the K^F slice (KROWS rows of TK floats).
  constexpr int NT = TK * T;            // threads per CTA
  constexpr int IPR = TK / 2;           // 16-byte pieces per input row
  constexpr int ISTEP = NT / IPR;       // rows per sweep of the CTA
  static_assert(NT % IPR == 0 && ROWS % ISTEP == 0, "input copy shape");
  constexpr int IIT = ROWS / ISTEP;
  const int irow0 = threadIdx.x / IPR;
  const long long igoff = (long long)irow0 * es + 2 * (threadIdx.x % IPR);
  const long long igstep = (long long)ISTEP * es;
  float2* const is0 = stage + irow0 * TK + 2 * (threadIdx.x % IPR);
  const int ivalid = a.nl - irow0;      // sweep i copies a physical row iff ISTEP * i < ivalid
  constexpr int KPR = TK / 4;           // 16-byte pieces per K^F row
  constexpr int KSTEP = NT / KPR;
  static_assert(NT % KPR == 0, "K copy shape");
  constexpr int KIT = (KROWS + KSTEP - 1) / KSTEP;
  const int krow0 = threadIdx.x / KPR;
  const long long kgoff = (long long)krow0 * a.kz_stride + 4 * (threadIdx.x % KPR);
  const long long kgstep = (long long)KSTEP * a.kz_stride;
  float* const ks0 = kstage + krow0 * TK + 4 * (threadIdx.x % KPR);

  // tile = kt + ntk * yi (kx tile fastest); the CTA steps by gridDim.x tiles
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
    for (int i = 0; i < IIT; ++i) {
      if (ISTEP * i < ivalid)
        cp_async16(is0 + i * ISTEP * TK, src);
      else  // beyond the physical z rows: zeros (nothing is read)
        cp_async16_zero(is0 + i * ISTEP * TK, src0);
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
  int kt = tile % ntk, yi = tile / ntk;  // this tile
  int nkt = kt, nyi = yi;                // the next one
  step_tile(nkt, nyi);
  // the first K^F slice does not depend on the previous pass: its copy starts
  // before the wait for that pass (programmatic dependent launch)
  if (tile < ntiles) issue_k(kt, yi);
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
    __syncthreads();  // this tile's inputs and K^F slice have landed

    c2 y[P];
#pragma unroll
    for (int aa = 0; aa < P; ++aa) {
      y[aa] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
      if (aa < NA && valid) {
        const float2 u0 = stage[(j + Q * aa) * TK + t];
        const float2 u1 = stage[(j + T + Q * aa) * TK + t];
        y[aa] = {make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
      }
    }
    __syncthreads();  // the input stage is free
    if constexpr (SEP) {
      if (next < ntiles) issue_input(nkt, nyi);
      cp_async_commit();
    }

    soa::dft2<P, -1, HALF>(y);
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) y[k1] = cmul_pair<-1>(y[k1], twid(j, k1));
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) sh4[xi(j, k1) + t] = pack(y[k1]);
    __syncthreads();

    // steps 2 and 3 on row k1 = j (rows exist for j < P only)
    const bool has_row = P == T || j < P;
    c2 z[T];
    if (has_row) {
#pragma unroll
      for (int b = 0; b < T; ++b) z[b] = unpack(sh4[xi(b, j) + t]);
      dif_all<T>(z, std::make_integer_sequence<int, T>{});
      soa::dft2<T, -1, false>(z);

      float2 e2 = make_float2(0.f, 0.f);
#pragma unroll
      for (int m = 0; m < T; ++m) {
        // kz0 = j + 2 P m and kz1 = kz0 + P (j < P) are both below L/2 = P T
        // exactly when m < T/2; above, the even octant is read at L - kz
        const int kz0 = j + P * 2 * m, kz1 = kz0 + P;
        const int o0 = m < T / 2 ? kz0 : L - kz0, o1 = m < T / 2 ? kz1 : L - kz1;
        const float2 kk = valid ? make_float2(kstage[o0 * TK + t], kstage[o1 * TK + t]) : make_float2(0.f, 0.f);
        const float2 p2 = soa::fma2(z[m].re, z[m].re, soa::mul2(z[m].im, z[m].im));
        e2 = soa::fma2(kk, p2, e2);
        z[m] = {soa::mul2(z[m].re, kk), soa::mul2(z[m].im, kk)};
      }
      eacc += (e2.x + e2.y) * ((kx == 0 || 2 * kx == a.L1) ? 1.f : 2.f);

      soa::dft2<T, 1, false>(z);
      dit_all<T>(z, std::make_integer_sequence<int, T>{});
#pragma unroll
      for (int b = 0; b < T; ++b) z[b] = cmul_pair<1>(z[b], twid(b, j));
    }
    __syncthreads();  // the forward exchange and the K^F stage have been read
    if (next < ntiles) issue_k(nkt, nyi);
    cp_async_commit();
    if (has_row) {
#pragma unroll
      for (int b = 0; b < T; ++b) sh4[xi(b, j) + t] = pack(z[b]);
    }
    __syncthreads();

#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) y[k1] = unpack(sh4[xi(j, k1) + t]);
    if constexpr (!SEP) {
      __syncthreads();  // the exchange has been read: the next tile's rows may land in it
      if (next < ntiles) issue_input(nkt, nyi);
      cp_async_commit();
    }
    soa::dft2<P, 1, false, HALF>(y);  // only the NA stored outputs when HALF
    if (valid) {
      float2* p0 = line + (long long)j * es;
      float2* p1 = p0 + (long long)T * es;
      const long long step = (long long)Q * es;
      if (a.nl >= ROWS) {  // every output row is physical
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
          *p0 = make_float2(y[aa].re.x, y[aa].im.x);
          *p1 = make_float2(y[aa].re.y, y[aa].im.y);
          p0 += step;
          p1 += step;
        }
      } else {
#pragma unroll
        for (int aa = 0; aa < NA; ++aa) {
          if (j + Q * aa < a.nl) *p0 = make_float2(y[aa].re.x, y[aa].im.x);
          if (j + T + Q * aa < a.nl) *p1 = make_float2(y[aa].re.y, y[aa].im.y);
          p0 += step;
          p1 += step;
        }
      }
    }
    kt = nkt;
    yi = nyi;
    step_tile(nkt, nyi);
  }
  cp_async_wait_all();
  if (E != nullptr) energy_finish_f32(eacc, partials, counter, escale, E);
}

const void* zpipe_kernel(int L, bool half, int* tk_io, int* threads, size_t* smem, int* P_out) {
  const void* fn = nullptr;
  int T = 0;
  int tk = *tk_io;
  if (tk != 8 && tk != 16) return nullptr;
  int P = 0;
  switch (L) {
    case 128:  // 16 lines per tile (8 would leave a CTA at two warps)
      fn = half ? (const void*)k_zconv_pipe<8, 8, true, 16> : (const void*)k_zconv_pipe<8, 8, false, 16>;
      T = P = 8;
      tk = 16;
      break;
    case 384:  // 12 x 32, 8 lines per tile
      fn = half ? (const void*)k_zconv_pipe<16, 12, true, 8> : (const void*)k_zconv_pipe<16, 12, false, 8>;
      T = 16;
      P = 12;
      tk = 8;
      break;
    case 512:
      if (tk == 16)
        fn = half ? (const void*)k_zconv_pipe<16, 16, true, 16> : (const void*)k_zconv_pipe<16, 16, false, 16>;
      else
        fn = half ? (const void*)k_zconv_pipe<16, 16, true, 8> : (const void*)k_zconv_pipe<16, 16, false, 8>;
      T = P = 16;
      break;
    default: return nullptr;
  }
  const int NA = half ? P / 2 : P;
  *tk_io = tk;
  *threads = tk * T;
  *P_out = P;
  // exchange, input stage (16 lines only; 8 lines reuse the exchange), K^F
  // slice, twiddle table (8 lines only)
  *smem = (size_t)T * P * tk * sizeof(float4) + (tk == 16 ? (size_t)NA * 2 * T * tk * sizeof(float2) : 0) +
          (size_t)(P * T + 1) * tk * sizeof(float) + (tk == 8 ? (size_t)T * (P + 1) * sizeof(float4) : 0);
  return fn;
}

// ---------------------------------------------------------------- packed, L = 256

// Persistent z pass for L3 = 256 = 16 * 16 on packed FP32x2 pairs: 8 threads
// per line, each carrying two columns of step 1 (b = j, j + 8) and then two
// rows of step 2 (k1 = j, j + 8) as one pair, so that every DFT of the line is
// a 16-point DFT of a pair and no stage crosses the lanes. The exchange holds
// slot (r, c) = the pair (column r, column r + 8) at row c, one 16-byte word;
// step 2 forms its row pairs from two slots, step 3 returns them the same way.
// The twiddles W_256^{b k1} of both lanes come from a paired table built in
// shared memory from W_256^i: tp[r][c] = (W^{r c}, W^{(r + 8) c}), r < 8, c < 16,
// used as (j, k1) by step 1 and (j, b) by step 3. TK lines per tile; the next
// tile's input rows land in the exchange once step 4 has read it, the next
// K^F slice once step 2 has used the current one.
template <bool HALF, int TK>
__global__ void __launch_bounds__(TK * 8, 4)
    k_zpipe_q(const void*, void* line_v, const float* __restrict__ K, const float2* __restrict__ tw, FastArgs a,
              double* partials, unsigned* counter, double escale, double* E) {
  constexpr int T = 8, P = 16, Q = 16, L = P * Q;
  constexpr int NA = HALF ? P / 2 : P;  // nonzero inputs / kept outputs per column
  constexpr int ROWS = NA * Q;          // input rows per line (n3)
  constexpr int KROWS = L / 2 + 1;      // rows of the K^F octant
  constexpr int TP = P + 1;             // paired twiddle table row pitch
  extern __shared__ float4 smem4[];
  float4* sh4 = smem4;                                          // exchange [T * P][TK]
  float2* stage = reinterpret_cast<float2*>(smem4);             // input rows [ROWS][TK] (same space)
  float* kstage = reinterpret_cast<float*>(smem4 + T * P * TK);  // K^F [KROWS][TK]
  float4* tp = reinterpret_cast<float4*>(kstage + KROWS * TK);  // [T][TP]
  static_assert((KROWS * TK) % 4 == 0, "paired table alignment");
  for (int i = threadIdx.x; i < T * P; i += blockDim.x) {  // before the first barrier
    const int r = i / P, c = i % P;
    const float2 w0 = __ldg(&tw[r * c]), w1 = __ldg(&tw[(r + T) * c]);
    tp[r * TP + c] = make_float4(w0.x, w1.x, w0.y, w1.y);
  }
  const int t = threadIdx.x % TK;
  const int j = threadIdx.x / TK;
  auto xi = [](int r, int c) { return (r * P + c) * TK; };  // exchange slot (r, c) of line t: xi(r, c) + t
  const int ntk = a.ntk_loc;
  const int ntiles = ntk * a.L2;
  float2* const base = static_cast<float2*>(line_v);
  const long long es = a.src_elem;

  constexpr int NT = TK * T;
  constexpr int IPR = TK / 2;  // 16-byte pieces per input row
  constexpr int ISTEP = NT / IPR;
  static_assert(NT % IPR == 0 && ROWS % ISTEP == 0, "input copy shape");
  constexpr int IIT = ROWS / ISTEP;
  const int irow0 = threadIdx.x / IPR;
  const long long igoff = (long long)irow0 * es + 2 * (threadIdx.x % IPR);
  const long long igstep = (long long)ISTEP * es;
  float2* const is0 = stage + irow0 * TK + 2 * (threadIdx.x % IPR);
  const int ivalid = a.nl - irow0;
  constexpr int KPR = TK / 4;  // 16-byte pieces per K^F row
  constexpr int KSTEP = NT / KPR;
  static_assert(NT % KPR == 0, "K copy shape");
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
    for (int i = 0; i < IIT; ++i) {
      if (ISTEP * i < ivalid)
        cp_async16(is0 + i * ISTEP * TK, src);
      else  // beyond the physical z rows: zeros (nothing is read)
        cp_async16_zero(is0 + i * ISTEP * TK, src0);
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
  const float2 zero = make_float2(0.f, 0.f);
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    const int kx = (a.kt0 + kt) * TK + t;
    const bool valid = kx < a.c;
    const int ky = paired_ky(yi, a.L2);
    float2* line = base + ky * a.src_plane + kx;
    cp_async_wait_all();
    __syncthreads();  // this tile's input rows and K^F slice have landed

    // step 1, columns j and j + 8: DFT over aa of x[b + Q aa]
    c2 y[P];
#pragma unroll
    for (int aa = 0; aa < P; ++aa) {
      y[aa] = {zero, zero};
      if (aa < NA && valid) {
        const float2 u0 = stage[(j + Q * aa) * TK + t];
        const float2 u1 = stage[(j + T + Q * aa) * TK + t];
        y[aa] = {make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
      }
    }
    __syncthreads();  // the input rows are in registers: the space becomes the exchange
    soa::dft2<P, -1, HALF>(y);
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) y[k1] = cmul_pair<-1>(y[k1], tp[j * TP + k1]);
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) sh4[xi(j, k1) + t] = pack(y[k1]);
    __syncthreads();

    // steps 2 and 3, rows j and j + 8: DFT over b, K^F, inverse DFT
    c2 z[Q];
#pragma unroll
    for (int b = 0; b < T; ++b) {
      const c2 s0 = unpack(sh4[xi(b, j) + t]), s1 = unpack(sh4[xi(b, j + T) + t]);
      z[b] = {make_float2(s0.re.x, s1.re.x), make_float2(s0.im.x, s1.im.x)};
      z[b + T] = {make_float2(s0.re.y, s1.re.y), make_float2(s0.im.y, s1.im.y)};
    }
    soa::dft2<Q, -1, false>(z);
    float2 e2 = zero;
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      // lanes k1 = j and j + 8: kz = k1 + P k2, the even octant at min(kz, L - kz)
      const int kz0 = j + P * k2, kz1 = kz0 + T;
      const int o0 = kz0 <= L / 2 ? kz0 : L - kz0, o1 = kz1 <= L / 2 ? kz1 : L - kz1;
      const float2 kk = valid ? make_float2(kstage[o0 * TK + t], kstage[o1 * TK + t]) : zero;
      const float2 p2 = soa::fma2(z[k2].re, z[k2].re, soa::mul2(z[k2].im, z[k2].im));
      e2 = soa::fma2(kk, p2, e2);
      z[k2] = {soa::mul2(z[k2].re, kk), soa::mul2(z[k2].im, kk)};
    }
    eacc += (e2.x + e2.y) * ((kx == 0 || 2 * kx == a.L1) ? 1.f : 2.f);
    soa::dft2<Q, 1, false>(z);
#pragma unroll
    for (int b = 1; b < Q; ++b) z[b] = cmul_pair<1>(z[b], tp[j * TP + b]);
    __syncthreads();  // the forward exchange and the K^F slice have been read
    if (next < ntiles) issue_k(nkt, nyi);
    cp_async_commit();
#pragma unroll
    for (int b = 0; b < T; ++b) {
      sh4[xi(b, j) + t] = make_float4(z[b].re.x, z[b + T].re.x, z[b].im.x, z[b + T].im.x);
      sh4[xi(b, j + T) + t] = make_float4(z[b].re.y, z[b + T].re.y, z[b].im.y, z[b + T].im.y);
    }
    __syncthreads();

    // step 4, columns j and j + 8: inverse DFT over k1, outputs aa < NA
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) y[k1] = unpack(sh4[xi(j, k1) + t]);
    __syncthreads();  // the exchange has been read: the next tile's rows may land in it
    if (next < ntiles) issue_input(nkt, nyi);
    cp_async_commit();
    soa::dft2<P, 1, false, HALF>(y);  // only the NA stored outputs when HALF
    if (valid) {
      float2* p0 = line + (long long)j * es;
      float2* p1 = p0 + (long long)T * es;
      const long long step = (long long)Q * es;
#pragma unroll
      for (int aa = 0; aa < NA; ++aa) {
        if (j + Q * aa < a.nl) *p0 = make_float2(y[aa].re.x, y[aa].im.x);
        if (j + T + Q * aa < a.nl) *p1 = make_float2(y[aa].re.y, y[aa].im.y);
        p0 += step;
        p1 += step;
      }
    }
    kt = nkt;
    yi = nyi;
    step_tile(nkt, nyi);
  }
  cp_async_wait_all();
  if (E != nullptr) energy_finish_f32(eacc, partials, counter, escale, E);
}

const void* zpipe_q_kernel(int L, bool half, int* threads, size_t* smem, int* tk) {
  if (L != 256) return nullptr;
  constexpr int TK = 16;
  *threads = TK * 8;
  // exchange (also the input rows), K^F slice, paired twiddle table
  *smem = (size_t)8 * 16 * TK * sizeof(float4) + (size_t)129 * TK * sizeof(float) + (size_t)8 * 17 * sizeof(float4);
  *tk = TK;
  return half ? (const void*)k_zpipe_q<true, TK> : (const void*)k_zpipe_q<false, TK>;
}
// ---------------------------------------------------------------- packed y passes

// Persistent packed y pass for L2 = P * 32 (T = 16; P = 16: 512, P = 12:
// 384): KIND 0 forward (n2 inputs, L2 outputs), KIND 1 inverse (L2 inputs, n2
// outputs). Same pairs as the z kernel (with P < T the threads j >= P hold no
// row of the 2T-point step); the next tile's rows land (cp.async) in the
// exchange buffer once the current tile's exchange has been read. Rows beyond
// a.nl (a count below L2/2) are zero on input and not stored on output.
template <int KIND, int P, bool HALF, int TK = 16>
__global__ void __launch_bounds__(TK * 16, 512 / (TK * 16))
    k_ysoa_pipe(const void* src_v, void* dst_v, const float*, const float4* __restrict__ tw4, FastArgs a,
                double*, unsigned*, double, double*) {
  constexpr int T = 16, Q = 2 * T, L = P * Q;
  static_assert(P <= T, "a thread holds at most one row of the 2T-point step");
  constexpr int NA = HALF ? P / 2 : P;
  constexpr int ROWS = KIND == 0 ? NA * Q : L;
  extern __shared__ float4 smem4[];
  float4* sh4 = smem4;                                  // exchange [T * P][TK] float4
  float2* stage = reinterpret_cast<float2*>(smem4);     // input rows [ROWS][TK] float2 (same space)
  // the paired twiddle table in shared memory, rows padded to P + 1 (the two
  // rows a warp reads at once fall on different banks)
  float4* tws = smem4 + T * P * TK;
  for (int i = threadIdx.x; i < T * P; i += blockDim.x) tws[(i / P) * (P + 1) + i % P] = __ldg(&tw4[i]);
  pdl_wait();
  const float2* src = static_cast<const float2*>(src_v);
  float2* dst = static_cast<float2*>(dst_v);
  const int t = threadIdx.x % TK;
  const int j = threadIdx.x / TK;
  const int ntk = a.ntk_loc;  // kx tiles a.kt0 .. a.kt0 + ntk - 1
  const int ntiles = ntk * a.nrows;  // nrows = z planes

  // the input copy: ROWS rows of TK float2 in 16-byte pieces, a fixed number
  // of sweeps of the CTA, per-thread offsets computed once
  constexpr int NT = TK * T;
  constexpr int IPR = TK / 2;
  constexpr int ISTEP = NT / IPR;
  static_assert(NT % IPR == 0 && ROWS % ISTEP == 0, "input copy shape");
  const int irow0 = threadIdx.x / IPR;
  const long long igoff = (long long)irow0 * a.src_elem + 2 * (threadIdx.x % IPR);
  const long long igstep = (long long)ISTEP * a.src_elem;
  float2* const is0 = stage + irow0 * TK + 2 * (threadIdx.x % IPR);
  auto plane = [&](int zi) { return a.rev ? (int)a.nrows - 1 - zi : zi; };
  const int ivalid = KIND == 0 ? a.nl - irow0 : ROWS;  // sweep i copies a physical row iff ISTEP * i < ivalid
  auto prefetch = [&](int kt, int zi) {
    const float2* sp0 = src + (long long)plane(zi) * a.src_plane + (a.kt0 + kt) * TK;
    const float2* sp = sp0 + igoff;
#pragma unroll
    for (int i = 0; i < ROWS / ISTEP; ++i) {
      if (ISTEP * i < ivalid)
        cp_async16(is0 + i * ISTEP * TK, sp);
      else  // beyond the physical rows: zeros (nothing is read)
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
    const long long de = a.dst_elem;
    cp_async_wait_all();
    __syncthreads();
    if constexpr (KIND == 0) {
      c2 y[P];
#pragma unroll
      for (int aa = 0; aa < P; ++aa) {
        y[aa] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
        if (aa < NA && valid) {
          const float2 u0 = stage[(j + Q * aa) * TK + t];
          const float2 u1 = stage[(j + T + Q * aa) * TK + t];
          y[aa] = {make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
        }
      }
      __syncthreads();  // inputs read: the space becomes the exchange
      soa::dft2<P, -1, HALF>(y);
#pragma unroll
      for (int k1 = 1; k1 < P; ++k1) y[k1] = cmul_pair<-1>(y[k1], tws[j * (P + 1) + k1]);
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) sh4[(j * P + k1) * TK + t] = pack(y[k1]);
      __syncthreads();
      const bool has_row = P == T || j < P;
      c2 z[T];
      if (has_row) {
#pragma unroll
        for (int b = 0; b < T; ++b) z[b] = unpack(sh4[(b * P + j) * TK + t]);
      }
      __syncthreads();  // exchange read: the next tile's rows may land
      if (next < ntiles) prefetch(nkt, nzi);
      cp_async_commit();
      if (has_row) {
      dif_all<T>(z, std::make_integer_sequence<int, T>{});
      soa::dft2<T, -1, false>(z);
      if (valid) {
        // z[m] = (X[j + 2P m], X[j + P + 2P m])
        float2* p0 = d + (long long)j * de;
        float2* p1 = p0 + (long long)P * de;
        const long long step = (long long)(2 * P) * de;
#pragma unroll
        for (int m = 0; m < T; ++m) {
          *p0 = make_float2(z[m].re.x, z[m].im.x);
          *p1 = make_float2(z[m].re.y, z[m].im.y);
          p0 += step;
          p1 += step;
        }
      }
      }
    } else {
      const bool has_row = P == T || j < P;
      c2 z[T];
      if (has_row) {
#pragma unroll
        for (int m = 0; m < T; ++m) {
          const float2 u0 = valid ? stage[(j + 2 * P * m) * TK + t] : make_float2(0.f, 0.f);
          const float2 u1 = valid ? stage[(j + P + 2 * P * m) * TK + t] : make_float2(0.f, 0.f);
          z[m] = {make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
        }
      }
      __syncthreads();  // inputs read: the space becomes the exchange
      if (has_row) {
        soa::dft2<T, 1, false>(z);
        dit_all<T>(z, std::make_integer_sequence<int, T>{});
#pragma unroll
        for (int b = 0; b < T; ++b) z[b] = cmul_pair<1>(z[b], tws[b * (P + 1) + j]);
#pragma unroll
        for (int b = 0; b < T; ++b) sh4[(b * P + j) * TK + t] = pack(z[b]);
      }
      __syncthreads();
      c2 y[P];
#pragma unroll
      for (int k1 = 0; k1 < P; ++k1) y[k1] = unpack(sh4[(j * P + k1) * TK + t]);
      __syncthreads();  // exchange read: the next tile's rows may land
      if (next < ntiles) prefetch(nkt, nzi);
      cp_async_commit();
      soa::dft2<P, 1, false, HALF>(y);  // only the NA stored outputs when HALF
      if (valid) {
        float2* p0 = d + (long long)j * de;
        float2* p1 = p0 + (long long)T * de;
        const long long step = (long long)Q * de;
        if (a.nl >= NA * Q) {  // every output row is physical
#pragma unroll
          for (int aa = 0; aa < NA; ++aa) {
            *p0 = make_float2(y[aa].re.x, y[aa].im.x);
            *p1 = make_float2(y[aa].re.y, y[aa].im.y);
            p0 += step;
            p1 += step;
          }
        } else {
#pragma unroll
          for (int aa = 0; aa < NA; ++aa) {
            if (j + Q * aa < a.nl) *p0 = make_float2(y[aa].re.x, y[aa].im.x);
            if (j + T + Q * aa < a.nl) *p1 = make_float2(y[aa].re.y, y[aa].im.y);
            p0 += step;
            p1 += step;
          }
        }
      }
    }
    kt = nkt;
    zi = nzi;
    step_tile(nkt, nzi);
  }
  cp_async_wait_all();
}

const void* ysoa_kernel(int L, int kind, bool half, int* threads, size_t* smem, int* tk) {
  const void* fn = nullptr;
  int P = 0, TK = 16;
  if (L == 512) {
    P = 16;
    fn = kind == 0 ? (half ? (const void*)k_ysoa_pipe<0, 16, true> : (const void*)k_ysoa_pipe<0, 16, false>)
                   : (half ? (const void*)k_ysoa_pipe<1, 16, true> : (const void*)k_ysoa_pipe<1, 16, false>);
  } else if (L == 384) {
    P = 12;
    TK = 8;
    fn = kind == 0 ? (half ? (const void*)k_ysoa_pipe<0, 12, true, 8> : (const void*)k_ysoa_pipe<0, 12, false, 8>)
                   : (half ? (const void*)k_ysoa_pipe<1, 12, true, 8> : (const void*)k_ysoa_pipe<1, 12, false, 8>);
  } else {
    return nullptr;
  }
  *threads = 16 * TK;
  *tk = TK;
  // exchange (the input rows share it), twiddles
  *smem = (size_t)16 * P * TK * sizeof(float4) + (size_t)16 * (P + 1) * sizeof(float4);
  return fn;
}

}  // namespace ps
