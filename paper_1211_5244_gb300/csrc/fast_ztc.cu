// z pass (forward transform, K^F multiply, inverse transform, Eq. 3) for
// L3 = 512 with its 32-point stages on the tensor cores (tcgen05, TF32 with
// split operands).
//
// A z line x[n] (n < n3; n3 = 256 for a free axis, 512 for a periodic one) is
// transformed with 512 = 16 * 32: writing n = n1 + 32 n2 and k = k2 + 16 k1,
//   Y[n1][k2] = sum_n2 x[n1 + 32 n2] W_16^{n2 k2}                  (stage 1)
//   X[k2 + 16 k1] = sum_n1 (Y[n1][k2] W_512^{n1 k2}) W_32^{n1 k1}  (stage 2)
// then V^F = K^F X, and back with the conjugate steps (stage 3: 32-point,
// stage 4: 16-point, keeping n < n3). Stages 1 and 4 are register DFTs on
// the CUDA cores (one (n1, line) row per thread). Stages 2 and 3 are dense
// products on the tensor cores: rows (k2, line) of the data, real-ified as
// (re, im) pairs along K, times the 64 x 64 real form of the 32-point DFT
// matrix ([[cos, -sin], [sin, cos]] blocks). Stage 3 uses the same forward
// matrix on conjugated data (conj(F^H z) = F conj(z)).
//
// Precision: operands are split into a TF32 part and an FP32 remainder,
// x = hi + lo (hi = x rounded to TF32, lo = x - hi exactly), for the data
// and for the matrix. The matrix is stored as [F_hi | F_lo] along N (N =
// 128), so the two products X_hi [F_hi | F_lo] and X_lo [F_hi | F_lo],
// accumulated in FP32, give all four partial products in two column halves,
// summed on the CUDA cores. The tensor cores read only the TF32 bits of an
// operand, so hi is passed as is and lo loses at most 2^-11 of itself.
//
// Layout per CTA (256 threads, 8 lines per tile, persistent):
//   TMEM (256 columns): [0, 128) the A operand (hi, lo), [128, 256) the
//   product (F_hi half, F_lo half). Rows are (k2, line), k2 < 16.
//   Shared memory: the matrix in the canonical K-major no-swizzle layout,
//   the tile's n3 input rows and K^F slice (prefetched with cp.async during
//   the previous tile), a padded transpose buffer, and the output rows.
// One thread issues the MMAs, commits them to an mbarrier and polls it, the
// other threads wait at a barrier. The poll is bounded (about a second),
// after which the kernel records an error in counter[1], finishes without
// further tiles and releases its TMEM.
#include <cstdint>
#include <cstring>

#include "fft_fast.cuh"
#include "fft_regs.cuh"
#include "reduce.cuh"

namespace ps {
namespace tc {

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

// shared-memory matrix descriptor: K-major, no swizzle; lbo = byte stride
// between core matrices along K, sbo = byte stride between 8-row groups
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// instruction descriptor: kind::tf32, FP32 accumulator, A and B K-major, M = 128
template <int N>
__host__ __device__ constexpr uint32_t idesc() {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
}

__device__ __forceinline__ void mma(uint32_t d, uint32_t a, uint64_t b, uint32_t id, uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], [%1], %2, %3, p;\n}" ::"r"(d),
      "r"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(uint32_t mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(mbar)
               : "memory");
}
__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// bounded wait for the mbarrier phase `parity`; false after ~2^31 cycles
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}"
        : "=r"(done)
        : "r"(mbar), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > (1ll << 31)) return false;
  }
}

__device__ __forceinline__ uint32_t tf32_hi(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}
// x -> (hi, lo) with hi the TF32 rounding of x and lo = x - hi
__device__ __forceinline__ void split(float x, uint32_t& hi, uint32_t& lo) {
  hi = tf32_hi(x);
  lo = __float_as_uint(x - __uint_as_float(hi));
}

// tcgen05.ld / st of 16 or 32 consecutive columns of the warp's 32 lanes;
// the loads wait for completion inside the same asm statement
__device__ __forceinline__ void ld16(uint32_t ta, uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
      : "r"(ta)
      : "memory");
}
__device__ __forceinline__ void ld32(uint32_t ta, uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
      "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
      "tcgen05.wait::ld.sync.aligned;"
      : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
        "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
        "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
        "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
      : "r"(ta)
      : "memory");
}
__device__ __forceinline__ void st16(uint32_t ta, const uint32_t (&v)[16]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};" ::"r"(
          ta),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
      : "memory");
}
__device__ __forceinline__ void st32(uint32_t ta, const uint32_t (&v)[32]) {
  asm volatile(
      "tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
      "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};" ::"r"(ta),
      "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]), "r"(v[9]),
      "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]), "r"(v[16]), "r"(v[17]), "r"(v[18]),
      "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]), "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]),
      "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
      : "memory");
}
__device__ __forceinline__ void wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem, int bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(su32(smem)), "l"(gmem), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ void cp_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

}  // namespace tc

namespace {

constexpr int kTcLines = 8;      // lines (kx columns) per tile
constexpr int kTpitch = 264;     // transpose buffer: 32 n1 x 8 lines + 8 padding, per k2
constexpr int kKRows = 257;      // rows of the K^F octant for L3 = 512

// byte offsets inside the dynamic shared memory
template <int NZ>
struct TcLayout {
  static constexpr int MATS = 64 * 128;    // [F_hi | F_lo], K = 64, N = 128 (floats)
  static constexpr int ROWS = 32 * NZ;     // n3
  static constexpr int S_OFF = MATS * 4;
  static constexpr int K_OFF = S_OFF + ROWS * kTcLines * 8;
  static constexpr int T_OFF = K_OFF + 8448;  // 257 x 8 floats, rounded up
  static constexpr int O_OFF = T_OFF + 16 * kTpitch * 8;
  static constexpr int BAR_OFF = O_OFF + ROWS * kTcLines * 8;
  static constexpr int SMEM = BAR_OFF + 16;
};

// one 32-point stage: D = A_hi [F_hi | F_lo] + A_lo [F_hi | F_lo]
// (A in TMEM columns [0, 64) and [64, 128), D in [128, 256))
__device__ __forceinline__ void stage32_mma(uint32_t tb, uint32_t mats) {
  constexpr uint32_t id = tc::idesc<128>();
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) tc::mma(tb + 128, tb + 8 * ks, tc::sdesc(mats + 256 * ks, 128, 2048), id, ks > 0);
#pragma unroll
  for (int ks = 0; ks < 8; ++ks) tc::mma(tb + 128, tb + 64 + 8 * ks, tc::sdesc(mats + 256 * ks, 128, 2048), id, 1);
}

__device__ __forceinline__ float2 cmulf(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

}  // namespace

template <int NZ>
__global__ void __launch_bounds__(256, NZ == 8 ? 2 : 1)
    k_ztc(const void*, void* line_v, const float* __restrict__ K, const float2* __restrict__ tab, FastArgs a,
          double* partials, unsigned* counter, double escale, double* E) {
  pdl_wait();
  using Lay = TcLayout<NZ>;
  constexpr int TK = kTcLines, ROWS = Lay::ROWS;
  extern __shared__ __align__(1024) unsigned char smem[];
  float* mats = reinterpret_cast<float*>(smem);
  float2* S = reinterpret_cast<float2*>(smem + Lay::S_OFF);   // [ROWS][8] input rows
  float* Ks = reinterpret_cast<float*>(smem + Lay::K_OFF);    // [257][8] K^F slice
  float2* T = reinterpret_cast<float2*>(smem + Lay::T_OFF);   // [16][264] transpose
  float2* O = reinterpret_cast<float2*>(smem + Lay::O_OFF);   // [ROWS][8] output rows
  uint64_t* mbar = reinterpret_cast<uint64_t*>(smem + Lay::BAR_OFF);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(smem + Lay::BAR_OFF + 8);
  __shared__ int s_abort;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp >> 2, q = warp & 3;
  const uint32_t lane_base = (uint32_t)(32 * q) << 16;
  // roles: row (n1, t) of stages 1 and 4; row (k2, t) and column half g of stages 2 and 3
  const int t = lane & 7;
  const int n1 = 16 * g + 4 * q + (lane >> 3);
  const int k2r = 4 * q + (lane >> 3);

  {
    const float4* src = reinterpret_cast<const float4*>(tab);
    float4* dst = reinterpret_cast<float4*>(mats);
    for (int i = tid; i < Lay::MATS / 4; i += 256) dst[i] = __ldg(src + i);
  }
  const float2* twt = tab + Lay::MATS / 2;
  float2 tw[16];  // W_512^{n1 k2}
#pragma unroll
  for (int k = 0; k < 16; ++k) tw[k] = __ldg(twt + n1 * 16 + k);
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;" ::"r"(tc::su32(tslot)));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::su32(mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
    s_abort = 0;
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tb = *tslot;
  const uint32_t mb = tc::su32(mbar);
  const uint32_t mats_a = tc::su32(mats);
  uint32_t phase = 0;

  const int ntk = a.ntk_loc;  // kx tiles of 8 lines
  const int ntiles = ntk * a.L2;
  float2* const base = static_cast<float2*>(line_v);
  const long long es = a.src_elem;

  auto issue_input = [&](int tile) {
    const int kx0 = (a.kt0 + tile % ntk) * TK;
    const int ky = paired_ky(tile / ntk, a.L2);
    const float2* src = base + ky * a.src_plane + kx0;
    for (int i = tid; i < ROWS * (TK / 2); i += 256) {
      const int row = i >> 2, part = i & 3;
      const int valid = a.c - (kx0 + 2 * part);
      const int bytes = valid >= 2 ? 16 : (valid == 1 ? 8 : 0);
      const float2* gp = src + (long long)row * es + (bytes ? 2 * part : 0);
      tc::cp_async16(S + row * TK + 2 * part, gp, bytes);
    }
  };
  auto issue_k = [&](int tile) {
    const int kx0 = (a.kt0 + tile % ntk) * TK;
    const int ky = paired_ky(tile / ntk, a.L2);
    const int kyo = min(ky, a.L2 - ky);
    const float* src = K + (long long)kyo * a.ldk + kx0;
    for (int i = tid; i < kKRows * (TK / 4); i += 256) {
      const int row = i >> 1, part = i & 1;
      tc::cp_async16(Ks + row * TK + 4 * part, src + (long long)row * a.kz_stride + 4 * part, 16);
    }
  };
  // thread 0 polls the MMA completion, the others wait at the barrier
  auto wait_mma = [&]() {
    if (tid == 0) {
      if (!tc::mbar_wait(mb, phase)) s_abort = 1;
      tc::fence_before();
    }
    phase ^= 1u;
    __syncthreads();
    tc::fence_after();
  };
  // the two column halves of the product, summed: 16 complex values
  auto load_product = [&](float2 (&v)[16]) {
    uint32_t dh[32], dl[32];
    tc::ld32(tb + lane_base + 128 + 32 * g, dh);
    tc::ld32(tb + lane_base + 192 + 32 * g, dl);
#pragma unroll
    for (int i = 0; i < 16; ++i)
      v[i] = make_float2(__uint_as_float(dh[2 * i]) + __uint_as_float(dl[2 * i]),
                         __uint_as_float(dh[2 * i + 1]) + __uint_as_float(dl[2 * i + 1]));
  };
  // 16 complex values as this warpgroup's half of an A operand row (hi, lo)
  auto store_operand = [&](const float2 (&v)[16]) {
    uint32_t hi[32], lo[32];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      tc::split(v[i].x, hi[2 * i], lo[2 * i]);
      tc::split(v[i].y, hi[2 * i + 1], lo[2 * i + 1]);
    }
    tc::st32(tb + lane_base + 32 * g, hi);
    tc::st32(tb + lane_base + 64 + 32 * g, lo);
    tc::wait_st();
  };

  float eacc = 0.f;
  int tile = blockIdx.x;
  if (tile < ntiles) {
    issue_input(tile);
    issue_k(tile);
  }
  tc::cp_commit();
  for (; tile < ntiles; tile += gridDim.x) {
    const int next = tile + gridDim.x;
    const int kx0 = (a.kt0 + tile % ntk) * TK;
    const int ky = paired_ky(tile / ntk, a.L2);
    tc::cp_wait_all();
    __syncthreads();  // this tile's rows and K^F slice have landed
    if (s_abort) break;

    // ---- stage 1 on the CUDA cores: row (n1, t), 16-point DFT over n2,
    // twiddle W_512^{n1 k2}, transpose through T
    {
      float2 y[16];
#pragma unroll
      for (int n2 = 0; n2 < 16; ++n2) y[n2] = n2 < NZ ? S[(n1 + 32 * n2) * TK + t] : make_float2(0.f, 0.f);
      regs::rdft<16, -1, NZ == 8>(y);
#pragma unroll
      for (int k = 0; k < 16; ++k) T[k * kTpitch + n1 * TK + t] = k ? cmulf(y[k], tw[k]) : y[k];
    }
    __syncthreads();
    if (next < ntiles) issue_input(next);  // the input rows have been read
    tc::cp_commit();
    // ---- stage 2 operand: row (k2, t), K = (n1, re/im), this warpgroup's n1 half
    {
      float2 v[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) v[i] = T[k2r * kTpitch + (16 * g + i) * TK + t];
      store_operand(v);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
      stage32_mma(tb, mats_a);
      tc::commit(mb);
    }
    wait_mma();
    if (s_abort) break;  // no further MMA or TMEM access: one commit stays outstanding

    // ---- stage 2 result X[k2 + 16 k1]: V^F = K^F X on the even octant,
    // energy, and the conjugate as the stage 3 operand (K = (k1, re/im))
    {
      float2 v[16];
      load_product(v);
      float e = 0.f;
#pragma unroll
      for (int i = 0; i < 16; ++i) {
        const int kz = k2r + 16 * (16 * g + i);
        const int o = kz <= 256 ? kz : 512 - kz;
        const float kk = Ks[o * TK + t];
        e = fmaf(kk, fmaf(v[i].x, v[i].x, v[i].y * v[i].y), e);
        v[i] = make_float2(v[i].x * kk, -v[i].y * kk);
      }
      const int kx = kx0 + t;
      eacc = fmaf(e, (kx == 0 || 2 * kx == a.L1) ? 1.f : 2.f, eacc);
      store_operand(v);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (tid == 0) {
      stage32_mma(tb, mats_a);
      tc::commit(mb);
    }
    if (next < ntiles) issue_k(next);  // the K^F slice has been read
    tc::cp_commit();
    wait_mma();
    if (s_abort) break;

    // ---- stage 3 result conj(U[n1][k2]): transpose through T
    {
      float2 v[16];
      load_product(v);
#pragma unroll
      for (int i = 0; i < 16; ++i) T[k2r * kTpitch + (16 * g + i) * TK + t] = v[i];
    }
    __syncthreads();
    // ---- stage 4 on the CUDA cores: row (n1, t); conj(U W_512^{-n1 k2}) =
    // conj(U) W_512^{n1 k2}, forward 16-point DFT over k2, conjugate: v[n1 + 32 n2]
    {
      float2 w[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        const float2 u = T[k * kTpitch + n1 * TK + t];
        w[k] = k ? cmulf(u, tw[k]) : u;
      }
      regs::rdft<16, -1, false>(w);
#pragma unroll
      for (int n2 = 0; n2 < NZ; ++n2) O[(n1 + 32 * n2) * TK + t] = make_float2(w[n2].x, -w[n2].y);
    }
    __syncthreads();
    {
      const float4* O4 = reinterpret_cast<const float4*>(O);
      float2* dst = base + ky * a.src_plane + kx0;
      for (int i = tid; i < ROWS * (TK / 2); i += 256) {
        const int row = i >> 2, part = i & 3;
        const int valid = a.c - (kx0 + 2 * part);
        if (valid <= 0) continue;
        const float4 v = O4[i];
        float2* p = dst + (long long)row * es + 2 * part;
        if (valid >= 2)
          *reinterpret_cast<float4*>(p) = v;
        else
          *p = make_float2(v.x, v.y);
      }
    }
  }
  tc::cp_wait_all();
  // An expired wait (wait_mma above) leaves the commit of its MMAs
  // outstanding: the MMAs may still write this CTA's TMEM, and the commit
  // arrives on an mbarrier in this CTA's shared memory. Before the TMEM is
  // freed and the CTA exits, thread 0 waits for that commit once more, with
  // the same bound (the phase it gave up on is the one before the last flip).
  // A slow MMA then completes before its TMEM and mbarrier go away. If it
  // does not complete even then, the tensor pipe has stopped and no order of
  // teardown makes its TMEM safe; the status word tells the host that the
  // results are invalid (ps_plan_device_status returns PS_ERR_TIMEOUT).
  if (tid == 0 && s_abort) tc::mbar_wait(mb, phase ^ 1u);
  if (tid == 0 && s_abort) atomicExch(counter + 1, 1u);
  tc::fence_before();
  __syncthreads();
  if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" ::"r"(tb));
  if (E != nullptr) energy_finish_f32(eacc, partials, counter, escale, E);
}

const void* ztc_kernel(int L, bool half, int* threads, size_t* smem) {
  if (L != 512) return nullptr;
  *threads = 256;
  if (half) {
    *smem = TcLayout<8>::SMEM;
    return (const void*)k_ztc<8>;
  }
  *smem = TcLayout<16>::SMEM;
  return (const void*)k_ztc<16>;
}

// The 32-point DFT matrix as [F_hi | F_lo] (K = 64, N = 128) in the
// canonical K-major layout, then the twiddles W_512^{n1 k2} (n1 < 32,
// k2 < 16), computed in double precision.
size_t ztc_table_floats(bool) { return (size_t)64 * 128 + 32 * 16 * 2; }

namespace {

float tf32_round(double v) {
  float f = (float)v;
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7F800000u) != 0x7F800000u) u = (u + 0x1000u) & 0xFFFFE000u;  // nearest, ties away
  memcpy(&f, &u, 4);
  return f;
}

// element (k, n) of a K x N matrix in the canonical layout, in floats
inline size_t canon(int k, int n, int Kd) { return (size_t)(n / 8) * (Kd / 4) * 32 + (k / 4) * 32 + (n % 8) * 4 + (k % 4); }

}  // namespace

void ztc_fill_table(bool, float* out) {
  const double pi = 3.14159265358979323846;
  for (int j = 0; j < 32; ++j)
    for (int k = 0; k < 32; ++k) {
      const double th = 2.0 * pi * (double)(j * k % 32) / 32.0;
      const double c = cos(th), s = sin(th);
      const double v[2][2] = {{c, -s}, {s, c}};  // [re/im of the input][re/im of the output]
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          const float h = tf32_round(v[a][b]);
          out[canon(2 * j + a, 2 * k + b, 64)] = h;                             // F_hi: columns 0..63
          out[canon(2 * j + a, 64 + 2 * k + b, 64)] = (float)(v[a][b] - (double)h);  // F_lo: 64..127
        }
    }
  float* tw = out + 64 * 128;
  for (int a = 0; a < 32; ++a)
    for (int k = 0; k < 16; ++k) {
      const double th = -2.0 * pi * (double)(a * k) / 512.0;
      tw[2 * (a * 16 + k)] = (float)cos(th);
      tw[2 * (a * 16 + k) + 1] = (float)sin(th);
    }
}

}  // namespace ps
