// Specialised FP32 kernels for the x passes (real-to-complex forward,
// complex-to-real inverse, §3), real length L1 = 2M with M a power of two or
// M = 48, 96, 192 (12 x 4, 24 x 4, 24 x 8: radix-3 register DFTs).
//
// A real row x of length L1 is transformed as the complex sequence
// z[m] = x[2m] + i x[2m+1] of length M (four-step, as in fast_strided.cu),
// then X[k] = E[k] + W_L1^k O[k] with E = (Z[k] + conj Z[M-k]) / 2 and
// O = -i (Z[k] - conj Z[M-k]) / 2 for k = 0..M; the L1/2 + 1 outputs are all
// the half spectrum keeps (§3). The inverse builds Z[k] = (X[k] + conj X[M-k])
// + i (X[k] - conj X[M-k]) W_L1^{-k} and transforms it back, which gives the
// unnormalised length-L1 inverse at even (real part) and odd (imaginary part)
// positions. T lanes own one row (contiguous 8-byte elements), so loads and
// stores are coalesced along the row. With zero padding (n1 = M), inputs
// z[m] with m >= M/2 are zero and outputs there are never formed.
#include <algorithm>
#include <cstdlib>
#include <cstring>

#include "fft_fast.cuh"
#include "fft_regs.cuh"

namespace ps {

using regs::rdft;

__device__ __forceinline__ float2 xmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 xmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}

// shared memory per row: the exchange tile P x QP and the row spectrum (M + 1)
// share one region (a barrier separates their uses). The row pitch QP = Q + 2
// is even, so every exchange row starts on 16 bytes and a thread moves its Q
// contiguous values as Q/2 128-bit accesses; a quarter-warp of them (8 rows,
// 16 (Q + 2) bytes apart) falls on 8 different bank groups.
template <int P, int Q>
struct XShape {
  static constexpr int M = P * Q;
  static constexpr int T = P < Q ? P : Q;
  static constexpr int QP = Q + 2;
  static constexpr int EX = P * QP;
  static constexpr int ROW0 = EX > M + 1 ? EX : M + 1;
  // with T < 16 lanes per row a warp spans 32 / T rows: a row pitch of T
  // (mod 16) float2 puts the rows of a half-warp on different banks
  static constexpr int ROW = T >= 16 ? ROW0 : ROW0 + ((T - ROW0 % 16) % 16 + 16) % 16;
  static_assert(EX > M + 1 && EX % 2 == 0, "the exchange region must be even and hold the row spectrum");
};

template <int P, int Q, int TR, bool HALF>
__global__ void __launch_bounds__(TR*(P < Q ? P : Q), 4)
    k_x_r2c(const void* src_v, void* dst_v, const float* twm_v, const float2* __restrict__ tw, FastArgs a,
            double*, unsigned*, double, double*) {
  pdl_wait();
  // twm: the matrix W_M^{r c} (r, c < P), laid out so lanes read consecutive entries
  const float2* __restrict__ twm = reinterpret_cast<const float2*>(twm_v);
  using S = XShape<P, Q>;
  constexpr int M = S::M, T = S::T, NB = Q / T, NK = P / T;
  constexpr int NA = HALF ? P / 2 : P;
  extern __shared__ __align__(16) float2 sh[];
  const int r = threadIdx.x / T, j = threadIdx.x % T;
  const int row = (a.rev ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x) * TR + r;
  const bool valid = row < a.nrows;
  float2* ex = sh + r * S::ROW;
  float2* zr = ex;  // reused for the row spectrum once the exchange has been read
  const float* xrow = static_cast<const float*>(src_v) + (long long)row * a.n1;
  const float2* z = reinterpret_cast<const float2*>(xrow);  // pairs of reals (n1 even: 8-byte aligned rows)
  const bool odd = a.n1 & 1;  // odd rows: reals one at a time, the last pair half zero
  float2* X = static_cast<float2*>(dst_v) + (long long)row * a.ldc;

#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int b = j + T * u;
    float2 y[P];
#pragma unroll
    for (int aa = 0; aa < P; ++aa) {
      y[aa] = make_float2(0.f, 0.f);
      const int m = b + Q * aa;
      if (aa < NA && valid && 2 * m < a.n1)
        y[aa] = odd ? make_float2(xrow[2 * m], 2 * m + 1 < a.n1 ? xrow[2 * m + 1] : 0.f) : z[m];
    }
    rdft<P, -1, HALF>(y);
#pragma unroll
    for (int k1 = 1; k1 < P; ++k1) y[k1] = xmul(y[k1], __ldg(&twm[k1 * P + b]));  // W_M^{b k1}
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) ex[k1 * S::QP + b] = y[k1];
  }
  __syncthreads();
  float2 x[NK][Q];
#pragma unroll
  for (int v = 0; v < NK; ++v) {
    const float4* r4 = reinterpret_cast<const float4*>(ex + (j + T * v) * S::QP);
#pragma unroll
    for (int b2 = 0; b2 < Q / 2; ++b2) {
      const float4 q4 = r4[b2];
      x[v][2 * b2] = make_float2(q4.x, q4.y);
      x[v][2 * b2 + 1] = make_float2(q4.z, q4.w);
    }
  }
  if constexpr (P == Q) {
    // P = Q = T: thread j holds Z[k] for k = j + P k2, and Z[M - k] sits in
    // lane (P - j) mod P of the same row at index Q - 1 - k2 (k2' = (Q - k2) mod Q
    // in the thread's own registers for j = 0), so the pairs meet by shuffles
    rdft<Q, -1, false>(x[0]);
    const int jp = (P - j) & (P - 1);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      const float2 sv = x[0][Q - 1 - k2];
      const float2 tv = make_float2(__shfl_sync(0xffffffffu, sv.x, jp, T), __shfl_sync(0xffffffffu, sv.y, jp, T));
      const float2 zm = j == 0 ? x[0][(Q - k2) & (Q - 1)] : tv;
      const float2 zk = x[0][k2];
      const int k = j + P * k2;
      const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      const float2 wo = xmul(o, __ldg(&tw[k]));
      if (valid) {
        X[k] = make_float2(e.x + wo.x, e.y + wo.y);
        if (k == 0) X[M] = make_float2(e.x - wo.x, wo.y - e.y);  // X[M] = conj(E[0] - O[0])
      }
    }
    return;
  }
  __syncthreads();  // the exchange has been read: its space takes the row spectrum
#pragma unroll
  for (int v = 0; v < NK; ++v) {
    const int k1 = j + T * v;
    rdft<Q, -1, false>(x[v]);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) zr[k1 + P * k2] = x[v][k2];
  }
  __syncthreads();
  if (!valid) return;
  // outputs k and M - k from the same pair Z[k], Z[M - k]: E[M-k] = conj E[k],
  // O[M-k] = conj O[k] and W_L1^{M-k} = -conj W_L1^k, so X[M-k] = conj(E[k] - W^k O[k])
#pragma unroll
  for (int i = 0; i <= M / (2 * T); ++i) {
    const int k = j + T * i;
    if (k > M / 2) break;
    const float2 zk = zr[k];
    const float2 zm = zr[k == 0 ? 0 : M - k];
    const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
    const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
    const float2 wo = xmul(o, __ldg(&tw[k]));
    X[k] = make_float2(e.x + wo.x, e.y + wo.y);
    if (2 * k != M) X[M - k] = make_float2(e.x - wo.x, wo.y - e.y);
  }
}

template <int P, int Q, int TR, bool HALF, bool SH = false>
__global__ void __launch_bounds__(TR*(P < Q ? P : Q), SH ? 3 : 4)
    k_x_c2r(const void* src_v, void* dst_v, const float* twm_v, const float2* __restrict__ tw, FastArgs a,
            double*, unsigned*, double, double*) {
  pdl_wait();
  const float2* __restrict__ twm = reinterpret_cast<const float2*>(twm_v);
  using S = XShape<P, Q>;
  constexpr int M = S::M, T = S::T, NB = Q / T, NK = P / T;
  constexpr int NA = HALF ? P / 2 : P;
  extern __shared__ __align__(16) float2 sh[];
  const int r = threadIdx.x / T, j = threadIdx.x % T;
  const int row = (a.rev ? (int)(gridDim.x - 1 - blockIdx.x) : (int)blockIdx.x) * TR + r;
  const bool valid = row < a.nrows;
  float2* ex = sh + r * S::ROW;
  float2* xr = ex;  // the row spectrum first, the exchange tile after a barrier
  const float2* X = static_cast<const float2*>(src_v) + (long long)row * a.ldc;
  float* vrow = static_cast<float*>(dst_v) + (long long)row * a.n1;
  float2* z = reinterpret_cast<float2*>(vrow);  // pairs of reals (n1 even: 8-byte aligned rows)
  const bool odd = a.n1 & 1;  // odd rows: reals one at a time, the last one alone

  float2 x[NK][Q];
  if constexpr (SH && P == Q) {
    // P = Q = T: thread j loads X[k] for k = j + P k2 (the k of its first
    // transform); X[M - k] comes from lane (P - j) mod P (index Q - 1 - k2), or
    // from its own registers for j = 0
    float2 xin[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) xin[i] = valid ? X[j + P * i] : make_float2(0.f, 0.f);
    const float2 xny = (valid && j == 0) ? X[M] : make_float2(0.f, 0.f);
    const int jp = (P - j) & (P - 1);
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      const float2 sv = xin[Q - 1 - k2];
      const float2 tv = make_float2(__shfl_sync(0xffffffffu, sv.x, jp, T), __shfl_sync(0xffffffffu, sv.y, jp, T));
      const float2 xm = j != 0 ? tv : (k2 == 0 ? xny : xin[(Q - k2) & (Q - 1)]);
      const float2 xk = xin[k2];
      const int k = j + P * k2;
      const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);
      const float2 o = xmulc(make_float2(xk.x - xm.x, xk.y + xm.y), __ldg(&tw[k]));
      x[0][k2] = make_float2(e.x - o.y, e.y + o.x);
    }
  } else {
  {
    // all loads of the row first (independent, in flight together), then the stores to shared memory
    float2 xin[M / T];
#pragma unroll
    for (int i = 0; i < M / T; ++i) xin[i] = valid ? X[j + T * i] : make_float2(0.f, 0.f);
    const float2 xny = (valid && j == 0) ? X[M] : make_float2(0.f, 0.f);
#pragma unroll
    for (int i = 0; i < M / T; ++i) xr[j + T * i] = xin[i];
    if (j == 0) xr[M] = xny;
  }
  __syncthreads();
#pragma unroll
  for (int v = 0; v < NK; ++v) {
    const int k1 = j + T * v;
#pragma unroll
    for (int k2 = 0; k2 < Q; ++k2) {
      const int k = k1 + P * k2;
      const float2 xk = xr[k], xm = xr[M - k];
      const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);
      const float2 o = xmulc(make_float2(xk.x - xm.x, xk.y + xm.y), __ldg(&tw[k]));
      x[v][k2] = make_float2(e.x - o.y, e.y + o.x);
    }
  }
  __syncthreads();  // the row spectrum has been read: its space takes the exchange
  }

#pragma unroll
  for (int v = 0; v < NK; ++v) {
    const int k1 = j + T * v;
    rdft<Q, 1, false>(x[v]);
#pragma unroll
    for (int b = 1; b < Q; ++b) x[v][b] = xmulc(x[v][b], __ldg(&twm[b * P + k1]));
    float4* w4 = reinterpret_cast<float4*>(ex + k1 * S::QP);
#pragma unroll
    for (int b2 = 0; b2 < Q / 2; ++b2)
      w4[b2] = make_float4(x[v][2 * b2].x, x[v][2 * b2].y, x[v][2 * b2 + 1].x, x[v][2 * b2 + 1].y);
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < NB; ++u) {
    const int b = j + T * u;
    float2 y[P];
#pragma unroll
    for (int k1 = 0; k1 < P; ++k1) y[k1] = ex[k1 * S::QP + b];
    rdft<P, 1, false>(y);
    if (valid) {
#pragma unroll
      for (int aa = 0; aa < NA; ++aa) {
        const int m = b + Q * aa;
        if (2 * m < a.n1) {
          if (!odd) {
            z[m] = y[aa];
          } else {
            vrow[2 * m] = y[aa].x;
            if (2 * m + 1 < a.n1) vrow[2 * m + 1] = y[aa].y;
          }
        }
      }
    }
  }
}

template <int P, int Q, int TR>
static const void* pick_x(int kind, bool half) {
  if (kind == 0) return half ? (const void*)k_x_r2c<P, Q, TR, true> : (const void*)k_x_r2c<P, Q, TR, false>;
  // P = Q: the untangling by shuffles (three CTAs per SM; 44.4 against 45.7 us
  // at 256^3 for the shared-memory form)
  if constexpr (P == Q)
    return half ? (const void*)k_x_c2r<P, Q, TR, true, true> : (const void*)k_x_c2r<P, Q, TR, false, true>;
  return half ? (const void*)k_x_c2r<P, Q, TR, true> : (const void*)k_x_c2r<P, Q, TR, false>;
}

const void* xline_kernel(int M, int kind, bool half, int* threads, int* rows, size_t* smem) {
  const void* fn = nullptr;
  int T = 0, TR = 0, ROW = 0;
  switch (M) {
    case 32: fn = pick_x<8, 4, 32>(kind, half); T = 4; TR = 32; ROW = XShape<8, 4>::ROW; break;
    case 48: fn = pick_x<12, 4, 32>(kind, half); T = 4; TR = 32; ROW = XShape<12, 4>::ROW; break;
    case 96: fn = pick_x<24, 4, 32>(kind, half); T = 4; TR = 32; ROW = XShape<24, 4>::ROW; break;
    case 64: fn = pick_x<8, 8, 32>(kind, half); T = 8; TR = 32; ROW = XShape<8, 8>::ROW; break;
    case 128: fn = pick_x<16, 8, 32>(kind, half); T = 8; TR = 32; ROW = XShape<16, 8>::ROW; break;
    case 192: fn = pick_x<24, 8, 16>(kind, half); T = 8; TR = 16; ROW = XShape<24, 8>::ROW; break;
    case 256: fn = pick_x<16, 16, 16>(kind, half); T = 16; TR = 16; ROW = XShape<16, 16>::ROW; break;
    case 512: fn = pick_x<32, 16, 8>(kind, half); T = 16; TR = 8; ROW = XShape<32, 16>::ROW; break;
    default: return nullptr;
  }
  *threads = T * TR;
  *rows = TR;
  *smem = (size_t)TR * ROW * sizeof(float2);
  return fn;
}

// ---------------------------------------------------------------- selection

static bool pow2(int v) { return v > 0 && (v & (v - 1)) == 0; }
// lengths with register kernels besides the powers of two: 3 * 2^k
static bool len3(int v) { return v == 96 || v == 192 || v == 384; }

cudaError_t configure_fast_f32(ps_plan_s* p) {
  const int n1 = p->n[0], n2 = p->n[1], n3 = p->n[2];
  p->zsoa_T = p->zsoa_P = 0;
  const int L1 = p->L[0], L2 = p->L[1], L3 = p->L[2];
  const long long ldc = (long long)p->ldc;
  cudaError_t e;
  auto set = [&](int pass, const void* fn, dim3 grid, int threads, size_t smem, const FastArgs& fa) -> cudaError_t {
    if (!fn) return cudaSuccess;
    if (smem > 48 * 1024) {
      cudaError_t err = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (err != cudaSuccess) return err;
    }
    PassCfg& cf = p->cfg[pass];
    cf.fast = 1;
    cf.fn = fn;
    cf.grid = grid;
    cf.block = dim3(threads);
    cf.smem = smem;
    cf.fa = fa;
    return cudaSuccess;
  };
  FastArgs base{};
  // the processing order starts with x (the R2C); b and c are its second and
  // third axes (y and z by default; z and y for the surface assignment pfp
  // under the axis rule), reached through strides: the y-pass kernels run
  // along b, the z-pass kernels along c
  const bool canon = canonical_order(p);
  const int ab = p->ord[1], ac = p->ord[2];
  const int nb = p->n[ab], Lb = p->L[ab], nc = p->n[ac], Lc = p->L[ac];
  const long long sA[3] = {1, ldc, (long long)n2 * ldc};               // A: [z][y][kx]
  const long long sB[3] = {1, ldc, (long long)p->ext2[1] * ldc};       // B: axis b at its padded length
  const long long Ks[3] = {1, (long long)p->ldk, (long long)(p->H[1] + 1) * p->ldk};  // K^F octant
  // passes that read what the previous pass wrote last first (PS_L2ORDER=0:
  // off); with x, y, z only
  const char* l2o = getenv("PS_L2ORDER");
  const int l2order = (!canon || (l2o && atoi(l2o) == 0)) ? 0 : 1;
  base.c = p->c;
  base.L1 = L1;
  base.L2 = L2;
  base.n1 = n1;
  base.nrows = n2 * n3;
  base.ldc = ldc;
  base.kz_stride = (long long)(p->H[1] + 1) * p->ldk;
  base.kt0 = 0;
  base.ntk_loc = (p->c + 15) / 16;
  base.ldk = (int)p->ldk;

  // x passes: L1 = 2M, n1 = M (free) or 2M (periodic)
  // x passes: L1 = 2M; n1 <= M (zero padding: inputs beyond n1 are zero,
  // outputs beyond n1 are not stored) or n1 = L1 (periodic). Even n1 moves
  // rho and V as 8-byte pairs of reals; odd n1 (rows off the 8-byte grid)
  // one real at a time
  if (L1 % 2 == 0 && (pow2(L1 / 2) || len3(L1)) && (n1 <= L1 / 2 || n1 == L1)) {
    const int M = L1 / 2;
    const bool half = n1 <= M;
    int threads, rows;
    size_t smem;
    const void* f0 = xline_kernel(M, 0, half, &threads, &rows, &smem);
    const void* f1 = xline_kernel(M, 1, half, &threads, &rows, &smem);
    if (f0 && f1) {
      p->xP = M == 32 ? 8 : M == 48 ? 12 : M == 64 ? 8 : M == 96 ? 24 : M == 128 ? 16 : M == 192 ? 24
            : M == 256 ? 16 : 32;
      dim3 grid((n2 * n3 + rows - 1) / rows);
      FastArgs xinv = base;
      xinv.rev = l2order;  // the inverse y pass wrote the last z planes last (x, y, z order)
      if ((e = set(P1, f0, grid, threads, smem, base)) != cudaSuccess) return e;
      if ((e = set(P5, f1, grid, threads, smem, xinv)) != cudaSuccess) return e;
      p->cfg[P1].xrows = p->cfg[P5].xrows = rows;
    }
  }
  // y passes (along b): nb <= Lb/2 (zero padding) or nb = Lb (periodic)
  if ((pow2(Lb) || len3(Lb)) && (nb <= Lb / 2 || nb == Lb)) {
    const bool half = nb <= Lb / 2;
    int threads0 = 0, threads1 = 0;
    size_t smem0 = 0, smem1 = 0;  // the forward and inverse kernels may differ
    // persistent prefetching kernels where they exist: the packed FP32x2 ones
    // at L = 512 (n = L/2 or L; at 256^3 forward 76.5 against 83 us for the
    // unpacked kernel, inverse 79.9 against 80.2 us), the unpacked ones at
    // L = 256 and 1024 and at L = 512 with other counts. The plan's schedule
    // y_kind = 1 takes the unpacked persistent kernels for both directions,
    // y_kind = 2 the non-persistent ones.
    const bool plain = p->y_kind == 2;
    const bool exact = 2 * nb == Lb || nb == Lb;
    // (at L = 384 the packed kernels are the only ones and take any count)
    const bool soa0 = !plain && (exact || Lb == 384) && p->y_kind != 1;
    const bool soa1 = soa0;
    int tk0 = 16, tk1 = 16;  // lines per tile (kx columns) of the chosen kernels
    const void* f0 = soa0 ? ysoa_kernel(Lb, 0, half, &threads0, &smem0, &tk0) : nullptr;
    const void* f1 = soa1 ? ysoa_kernel(Lb, 1, half, &threads1, &smem1, &tk1) : nullptr;
    p->ysoa = (f0 ? 1 : 0) | (f1 ? 2 : 0);
    if (!f0 && !plain) f0 = ypipe_kernel(Lb, 0, half, &threads0, &smem0, &tk0);
    if (!f1 && !plain) f1 = ypipe_kernel(Lb, 1, half, &threads1, &smem1, &tk1);
    const bool ypersist = f0 && f1;
    if (!ypersist) {
      p->ysoa = 0;
      f0 = strided_kernel(Lb, 0, half, &threads0, &smem0, &tk0);
      f1 = strided_kernel(Lb, 1, half, &threads1, &smem1, &tk1);
    }
    if (f0 && f1) {
      FastArgs fwd = base, inv = base;
      fwd.ntk_loc = (p->c + tk0 - 1) / tk0;
      inv.ntk_loc = (p->c + tk1 - 1) / tk1;
      fwd.nl = inv.nl = nb;
      fwd.rev = l2order;  // the x pass wrote the last z planes last
      // lines along b, one plane per index along c, tiles across kx
      fwd.src_plane = sA[ac]; fwd.src_elem = sA[ab];   // A
      fwd.dst_plane = sB[ac]; fwd.dst_elem = sB[ab];   // B
      inv.src_plane = sB[ac]; inv.src_elem = sB[ab];
      inv.dst_plane = sA[ac]; inv.dst_elem = sA[ab];
      dim3 grid0(fwd.ntk_loc, nc), grid1(inv.ntk_loc, nc);
      if (ypersist) {
        fwd.nrows = inv.nrows = nc;  // planes walked by the persistent CTAs
        int dev = 0, sms = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        auto persistent_grid = [&](const void* f, int threads, size_t smem, int ntk_f, dim3* grid) -> cudaError_t {
          const long long tiles = (long long)ntk_f * nc;
          cudaError_t err = cudaSuccess;
          if (smem > 48 * 1024 &&
              (err = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
            return err;
          int per_sm = 0;
          if ((err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, smem)) != cudaSuccess)
            return err;
          const long long g = (long long)(per_sm > 0 ? per_sm : 1) * sms;
          *grid = dim3((unsigned)(g < tiles ? g : tiles), 1);
          return cudaSuccess;
        };
        if ((e = persistent_grid(f0, threads0, smem0, fwd.ntk_loc, &grid0)) != cudaSuccess) return e;
        if ((e = persistent_grid(f1, threads1, smem1, inv.ntk_loc, &grid1)) != cudaSuccess) return e;
      }
      if ((e = set(P2, f0, grid0, threads0, smem0, fwd)) != cudaSuccess) return e;
      if ((e = set(P4, f1, grid1, threads1, smem1, inv)) != cudaSuccess) return e;
    }
  }
  // fused x/y passes: thread-block clusters of 16 CTAs own one z plane and
  // exchange its x-transformed rows through distributed shared memory, so
  // array A is never written (L1 = 512 with n1 = 256 or 512, L2 = 512 with
  // n2 = 256; they use the x twiddle matrix and the paired y twiddles of the
  // kernels above). Measured slower than the separate passes at 256^3 (at most
  // 14 clusters of 16 CTAs are resident, and each plane waits on a cluster
  // barrier), so they run when the plan's schedule asks for them
  // (ps_plan_set_schedule, or ps_plan_autotune where they win).
  p->xyfuse = 0;
  {
    const bool allow = p->xy_sched == 1;
    if (allow && canon && L1 == 512 && (n1 == 256 || n1 == 512) && L2 == 512 && n2 == 256 && p->xP == 16 &&
        (p->ysoa & 3) == 3 && p->cfg[P1].fast && p->cfg[P5].fast) {
      bool ok = true;
      for (int kind = 0; kind < 2 && ok; ++kind) {
        int threads = 0, cl = 0;
        size_t smem = 0;
        const void* fn = xy_kernel(kind, n1 == 256, &threads, &smem, &cl);
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
          return e;
        if ((e = cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1)) != cudaSuccess)
          return e;
        PassCfg& cf = p->xyf[kind];
        cf = PassCfg{};
        cf.fast = 1;
        cf.fn = fn;
        cf.grid = dim3((unsigned)(n3 * cl));
        cf.block = dim3(threads);
        cf.smem = smem;
        cf.cluster = cl;
        cf.fa = base;
        cf.fa.n1 = n1;
        cf.fa.nrows = n2;  // rows per plane
        if (kind == 0) {
          cf.fa.dst_plane = (long long)L2 * ldc;
          cf.fa.dst_elem = ldc;
        } else {
          cf.fa.src_plane = (long long)L2 * ldc;
          cf.fa.src_elem = ldc;
        }
        // the GPU must be able to hold at least one such cluster
        cudaLaunchConfig_t lc = {};
        lc.gridDim = cf.grid;
        lc.blockDim = cf.block;
        lc.dynamicSmemBytes = smem;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = (unsigned)cl;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        lc.attrs = attr;
        lc.numAttrs = 1;
        int nclusters = 0;
        if (cudaOccupancyMaxActiveClusters(&nclusters, fn, &lc) != cudaSuccess || nclusters < 1) {
          cudaGetLastError();  // clear a refusal: the separate passes run instead
          ok = false;
        }
      }
      p->xyfuse = ok ? 1 : 0;
    }
  }
  // chunked x and y passes: with the separate specialised x kernels and
  // persistent y kernels, the forward runs x then y on each chunk of z planes
  // through one chunk-sized region of A (and the inverse y then x), so the
  // chunk is read back from L2 instead of HBM and its lines are overwritten
  // in L2 by the next chunk. Measured slower at 256^3 (x and y 115.7 us
  // whole, 120 / 132 / 145 us in 2 / 4 / 8 chunks: every chunk adds a tail
  // to the x kernel and leaves the persistent y kernel under two tiles per
  // CTA), so it runs when the schedule's chunk_req asks for it.
  p->chunks = 1;
  if (canon && !p->xyfuse && p->cfg[P1].fast && p->cfg[P2].fast && p->cfg[P4].fast && p->cfg[P5].fast &&
      p->cfg[P2].fa.nrows == n3 && p->cfg[P4].fa.nrows == n3 && p->chunk_req > 1)
    p->chunks = std::min(p->chunk_req, n3);
  // z pass on the tensor cores (PS_MATH_TF32X3, L3 = 512): persistent, one
  // wave of resident CTAs over tiles of 8 kx lines
  p->tctab_floats = 0;
  if (canon && p->math == PS_MATH_TF32X3 && L3 == 512 && (n3 == 256 || n3 == 512)) {
    const bool half = n3 == 256;
    int threads;
    size_t smem;
    const void* f = ztc_kernel(L3, half, &threads, &smem);
    if (f) {
      if ((e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
        return e;
      if ((e = cudaFuncSetAttribute(f, cudaFuncAttributePreferredSharedMemoryCarveout,
                                    (int)cudaSharedmemCarveoutMaxShared)) != cudaSuccess)
        return e;
      FastArgs z = base;
      z.nl = n3;
      z.src_plane = ldc; z.src_elem = (long long)L2 * ldc;
      z.dst_plane = ldc; z.dst_elem = (long long)L2 * ldc;
      z.ntk_loc = (p->c + 7) / 8;
      int dev = 0, sms = 0, per_sm = 0;
      if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
      if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
      if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, smem)) != cudaSuccess) return e;
      // registers (<= 128) and shared memory (~110 KB) leave room for two CTAs
      // of the n3 = 256 kernel per SM, as do their 256 TMEM columns each; the
      // grid is sized for that even where the occupancy query reports one (a
      // CTA that finds no room starts when one finishes, so the result is the same)
      if (half && per_sm < 2) per_sm = 2;
      const long long tiles = (long long)z.ntk_loc * L2;
      const long long g = (long long)(per_sm > 0 ? per_sm : 1) * sms;
      if ((e = set(P3, f, dim3((unsigned)(g < tiles ? g : tiles)), threads, smem, z)) != cudaSuccess) return e;
      p->cfg[P3].tk = 8;
      p->zsoa_T = 0;
      p->zsoa_P = 0;
      p->tctab_floats = ztc_table_floats(half);
      return cudaSuccess;
    }
  }
  // z pass (along c): the persistent prefetching packed kernels where they
  // exist (L = 128, 256, 384 and 512), the persistent unpacked one at
  // L = 1024, else the non-persistent unpacked one
  if ((pow2(Lc) || len3(Lc)) && (nc <= Lc / 2 || nc == Lc)) {
    const bool half = nc <= Lc / 2;
    int threads;
    size_t smem;
    // lines per tile of the persistent packed kernel: 8 (four CTAs of 42 KB
    // per SM; at 256^3 228 us against 251 us for 16 lines and 280 us for 4),
    // or 16 where the plan's schedule z_tk asks for it
    int pipe_tk = p->z_tk == 16 ? 16 : 8;
    int zP = 0;
    const void* f = zpipe_kernel(Lc, half, &pipe_tk, &threads, &smem, &zP);
    bool persistent = f != nullptr;
    p->zsoa_T = f ? (Lc == 128 ? 8 : 16) : 0;
    p->zsoa_P = f ? zP : 0;
    int ztile = pipe_tk;
    // L = 256: the packed kernel on pairs of columns and rows; L = 1024: the
    // persistent unpacked kernel
    if (!f && (f = zpipe_q_kernel(Lc, half, &threads, &smem, &ztile)) != nullptr) persistent = true;
    if (!f && (f = zpipe_u_kernel(Lc, half, &threads, &smem, &ztile)) != nullptr) persistent = true;
    if (!f) f = strided_kernel(Lc, 2, half, &threads, &smem, &ztile);
    if (f) {
      FastArgs z = base;
      z.nl = nc;
      z.ntk_loc = (p->c + ztile - 1) / ztile;
      // lines along c, tile rows along b (Lb of them, paired k and Lb - k),
      // tiles across kx; K^F octant strides of the row and the line axis
      z.src_plane = sB[ab]; z.src_elem = sB[ac];
      z.dst_plane = sB[ab]; z.dst_elem = sB[ac];
      z.L2 = Lb;
      z.ldk = (int)Ks[ab];
      z.kz_stride = Ks[ac];
      dim3 grid((p->c + ztile - 1) / ztile, Lb);
      if (persistent) {
        // one wave of resident CTAs walks all tiles
        if (smem > 48 * 1024 &&
            (e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)) != cudaSuccess)
          return e;
        int dev = 0, sms = 0, per_sm = 0;
        if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
        if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
        if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, f, threads, smem)) != cudaSuccess) return e;
        const long long tiles = (long long)grid.x * grid.y;
        const long long g = (long long)(per_sm > 0 ? per_sm : 1) * sms;
        grid = dim3((unsigned)(g < tiles ? g : tiles), 1);
      }
      if ((e = set(P3, f, grid, threads, smem, z)) != cudaSuccess) return e;
      p->cfg[P3].tk = ztile;
    }
  }
  return cudaSuccess;
}

namespace {

// One launch of a specialised kernel: programmatic stream serialisation
// (the kernel may start while the previous one drains; it waits for it before
// touching memory; PS_PDL=0 off) and, for cluster kernels, the cluster shape.
cudaError_t launch_cfg(const PassCfg& cf, const FastArgs& fa, const void* src, void* dst, const float* K,
                       const void* tw, double* partials, unsigned* counter, double escale, double* E,
                       cudaStream_t s) {
  FastArgs a = fa;
  void* args[] = {(void*)&src, (void*)&dst, (void*)&K, (void*)&tw, (void*)&a,
                  (void*)&partials, (void*)&counter, (void*)&escale, (void*)&E};
  static const bool pdl = [] {
    const char* v = getenv("PS_PDL");
    return !(v && atoi(v) == 0);
  }();
  cudaLaunchConfig_t lc = {};
  lc.gridDim = cf.grid;
  lc.blockDim = cf.block;
  lc.dynamicSmemBytes = cf.smem;
  lc.stream = s;
  cudaLaunchAttribute attr[3];
  int na = 0;
  if (pdl) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (cf.cluster > 0) {
    attr[na].id = cudaLaunchAttributeClusterDimension;
    attr[na].val.clusterDim.x = (unsigned)cf.cluster;
    attr[na].val.clusterDim.y = 1;
    attr[na].val.clusterDim.z = 1;
    ++na;
    // load-balancing placement of the clusters (fused forward 180 -> 171 us
    // at 256^3 against the default spread policy)
    attr[na].id = cudaLaunchAttributeClusterSchedulingPolicyPreference;
    attr[na].val.clusterSchedulingPolicyPreference = cudaClusterSchedulingPolicyLoadBalancing;
    ++na;
  }
  lc.attrs = attr;
  lc.numAttrs = na;
  return cudaLaunchKernelExC(&lc, cf.fn, args);
}

}  // namespace

cudaError_t launch_xy(ps_plan_s* p, int kind, const void* src, void* dst, cudaStream_t s) {
  const PassCfg& cf = p->xyf[kind];
  FastArgs fa = cf.fa;
  fa.tw1 = static_cast<const float2*>(p->tw[0]);
  return launch_cfg(cf, fa, src, dst, static_cast<const float*>(p->twx), p->tw4y, nullptr, nullptr, 0.0, nullptr,
                    s);
}

cudaError_t launch_fast_chunk(ps_plan_s* p, int pass, const void* rhoV, void* B, void* A, int z0, int nz,
                              cudaStream_t s) {
  PassCfg cf = p->cfg[pass];
  FastArgs fa = cf.fa;
  const long long n1 = p->n[0], n2 = p->n[1];
  const long long bplane = (long long)p->L[1] * (long long)p->ldc;  // complex elements per plane of B
  const void* src = nullptr;
  void* dst = nullptr;
  switch (pass) {
    case P1:
      src = static_cast<const float*>(rhoV) + z0 * n2 * n1;
      dst = A;
      break;
    case P2:
      src = A;
      dst = static_cast<float2*>(B) + z0 * bplane;
      break;
    case P4:
      src = static_cast<const float2*>(B) + z0 * bplane;
      dst = A;
      break;
    default:  // P5
      src = A;
      dst = static_cast<float*>(const_cast<void*>(rhoV)) + z0 * n2 * n1;
      break;
  }
  if (pass == P1 || pass == P5) {
    fa.nrows = (int)(nz * n2);
    cf.grid = dim3((unsigned)((fa.nrows + cf.xrows - 1) / cf.xrows));
  } else {
    fa.nrows = nz;  // planes walked by the persistent CTAs
    const long long tiles = (long long)fa.ntk_loc * nz;
    cf.grid = dim3((unsigned)std::min<long long>(cf.grid.x, tiles));
  }
  const float* K = static_cast<const float*>((pass == P1 || pass == P5) ? p->twx : p->K);
  const int axis = pass_axis(p, pass);
  const void* tw = ((pass == P2 && (p->ysoa & 1)) || (pass == P4 && (p->ysoa & 2))) ? p->tw4y : p->tw[axis];
  return launch_cfg(cf, fa, src, dst, K, tw, p->partials, p->counter, 0.0, nullptr, s);
}

cudaError_t launch_fast(ps_plan_s* p, int pass, const void* src, void* dst, double* E, double escale,
                        cudaStream_t s) {
  PassCfg& cf = p->cfg[pass];
  const int axis = pass_axis(p, pass);
  // x passes get the twiddle matrix in the K slot
  const float* K = static_cast<const float*>((pass == P1 || pass == P5) ? p->twx : p->K);
  const void* tw = (pass == P3 && p->tctab) ? p->tctab
                   : (pass == P3 && p->zsoa_T) ? p->tw4z
                   : ((pass == P2 && (p->ysoa & 1)) || (pass == P4 && (p->ysoa & 2))) ? p->tw4y : p->tw[axis];
  return launch_cfg(cf, cf.fa, src, dst, K, tw, p->partials, p->counter, escale, E, s);
}

}  // namespace ps
