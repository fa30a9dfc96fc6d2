// Fused x/y passes in thread-block clusters (FP32): the forward x transform
// (R2C) and the forward y transform of one z plane in one kernel, and the
// inverse y transform and the inverse x transform (C2R) of one plane in
// another, so the x-transformed plane (array A of the five-pass form) never
// leaves the chip.
//
// §3 runs the x step, a transpose, and the y step as separate kernels with
// the plane in global memory between them. Here a cluster of CS = 16 CTAs
// owns one plane (L1 = 512, real rows of n1 = 256 or 512 points; L2 = 512
// with n2 = 256 physical rows):
//   forward   CTA r transforms the x rows y = 16 r .. 16 r + 15 (four-step
//             register FFT of the complex row z[m] = x[2m] + i x[2m+1] and
//             the R2C untangling, as in fast_x.cu) and stores each output
//             straight into the shared memory of the CTA that owns its kx
//             column (distributed shared memory, plain stores: CTA q owns kx
//             columns 16 q .. 16 q + 15); after one cluster barrier every CTA
//             holds its 16 columns of all 256 rows locally and runs the
//             length-512 y transform of these 16 lines (packed FP32x2 pairs,
//             as in fast_zsoa.cu), writing B[z][ky][kx] directly.
//   inverse   CTA r runs the inverse y transform of kx columns 16 r ..
//             16 r + 15 (all 512 ky rows read from B, the 256 physical rows
//             kept) and stores each output row segment into the shared memory
//             of the CTA that owns the row (CTA q owns rows 16 q .. 16 q + 15);
//             after one cluster barrier every CTA runs the C2R of its 16 rows
//             from local shared memory, writing V.
// The R2C of a real row keeps L1/2 + 1 = 257 outputs, of which X[0] and
// X[256] are real. They travel as one complex column X[0] + i X[256] in slot
// 0, so 256 columns split evenly over the 16 CTAs. Forward, the y transform of
// that column is the transform of two real sequences, separated by Hermitian
// symmetry, Y0[k] = (Z[k] + conj Z[-k]) / 2 and YM[k] = (Z[k] - conj Z[-k]) / 2i.
// Inverse, the inverse y transforms of the kx = 0 and kx = 256 columns are
// real (V is real), so the packed inverse gives them as the real and
// imaginary parts.
//
// The data move by remote stores, which the writer does not wait for, and
// one cluster barrier per plane (release / acquire: the stores are visible
// after it). Each CTA arrives at a relaxed cluster barrier when it starts and
// waits on it just before its first remote store, so every CTA of the cluster
// is running (its shared memory exists) before any is written to; no CTA
// touches remote shared memory after the second barrier.
//
// Shared memory per CTA: the 32 KB stage the other CTAs store into, a region
// for the local exchange of the four-step transform (the x exchange, or the
// y exchange, which may also take the stage once it has been read), the
// paired y twiddles and a 4 KB line for the packed column.
#include <cooperative_groups.h>

#include "fft_fast.cuh"
#include "fft_regs.cuh"
#include "fft_soa.cuh"

namespace ps {

namespace cg = cooperative_groups;
using regs::rdft;
using soa::c2;

namespace {

constexpr int kCS = 16;       // CTAs per cluster
constexpr int kNT = 256;      // threads per CTA
constexpr int kXP = 16;       // x: M = 256 = P x Q, T = 16 threads per row
constexpr int kXQ = 16;
constexpr int kM = kXP * kXQ;
constexpr int kXQP = kXQ + 2;         // x exchange row pitch (float2), even: 128-bit accesses
constexpr int kXROW = kXP * kXQP;     // x exchange floats2 per row (288)
constexpr int kRows = 16;             // x rows per CTA (n2 / kCS)
constexpr int kYT = 16;               // y: L2 = 512 = 16 x 32, packed pairs, T = 16 threads per line
constexpr int kYL = 2 * kYT * kYT;
constexpr int kTK = 16;               // y lines (kx columns) per CTA
constexpr int kYEx = kYT * kYT * kTK;      // float4 of the 64 KB y exchange
constexpr int kStage = 256 * 16 / 2;       // float4 of the 32 KB stage (256 x 16 float2)
constexpr int kXEx = kRows * kXROW / 2;    // float4 of the x exchange (36 KB)
constexpr int kRegion = (kStage + kXEx > kYEx) ? kStage + kXEx : kYEx;  // stage | x exchange, or y exchange
static_assert(kRows * kXROW % 2 == 0, "x exchange in float4");

__device__ __forceinline__ void cluster_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.aligned;" ::: "memory"); }

__device__ __forceinline__ float2 xmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 xmulc(float2 a, float2 b) {
  return make_float2(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
using soa::cmul_pair;
using soa::pack;
using soa::unpack;

// radix-2 stages across the two lanes of a pair (as in fast_zsoa.cu)
template <int B>
__device__ __forceinline__ void dif_lanes(c2 (&z)[kYT]) {
  const float2 x0 = make_float2(z[B].re.x, z[B].im.x), x1 = make_float2(z[B].re.y, z[B].im.y);
  const float2 s = make_float2(x0.x + x1.x, x0.y + x1.y);
  const float2 d = regs::twc<2 * kYT, B, -1>(make_float2(x0.x - x1.x, x0.y - x1.y));
  z[B] = {make_float2(s.x, d.x), make_float2(s.y, d.y)};
}
template <int... B>
__device__ __forceinline__ void dif_all(c2 (&z)[kYT], std::integer_sequence<int, B...>) {
  (dif_lanes<B>(z), ...);
}
template <int B>
__device__ __forceinline__ void dit_lanes(c2 (&z)[kYT]) {
  const float2 e = make_float2(z[B].re.x, z[B].im.x);
  const float2 o = regs::twc<2 * kYT, B, 1>(make_float2(z[B].re.y, z[B].im.y));
  z[B] = {make_float2(e.x + o.x, e.x - o.x), make_float2(e.y + o.y, e.y - o.y)};
}
template <int... B>
__device__ __forceinline__ void dit_all(c2 (&z)[kYT], std::integer_sequence<int, B...>) {
  (dit_lanes<B>(z), ...);
}

// the paired y twiddle table into shared memory, rows padded to 17
__device__ __forceinline__ void load_y_twiddles(float4* tws, const float4* __restrict__ tw4) {
  for (int i = threadIdx.x; i < kYT * kYT; i += blockDim.x) tws[(i / kYT) * (kYT + 1) + i % kYT] = __ldg(&tw4[i]);
}

}  // namespace

// Forward: rho plane z -> B[z][ky][kx]. HX: n1 = 256 (the upper half of each
// complex row z[m] is zero padding), else n1 = 512. Grid: n3 clusters of kCS CTAs.
template <bool HX>
__global__ void __launch_bounds__(kNT, 2)
    k_xy_fwd(const void* src_v, void* dst_v, const float* twm_v, const float4* __restrict__ tw4, FastArgs a,
             double*, unsigned*, double, double*) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int z = blockIdx.x / kCS;
  const float2* __restrict__ twm = reinterpret_cast<const float2*>(twm_v);  // W_M^{r c}, r, c < 16
  const float2* __restrict__ tw1 = a.tw1;                                   // W_L1^k, k <= M
  extern __shared__ __align__(16) float4 smem4[];
  float2* const stage = reinterpret_cast<float2*>(smem4);            // [256 rows][16 columns], filled remotely
  float2* const ex = reinterpret_cast<float2*>(smem4 + kStage);      // x exchange [kRows][kXROW]
  float4* const sh4 = smem4;                                          // y exchange [kYT * kYT][kTK]
  float4* const tws = smem4 + kRegion;                                // paired y twiddles [16][17]
  float2* const lin = reinterpret_cast<float2*>(tws + kYT * (kYT + 1));  // the packed column [512]
  cluster_arrive_relaxed();  // this CTA is running
  load_y_twiddles(tws, tw4);
  pdl_wait();

  // ---- x: rows y = 16 rank + r, thread j of the row (T = P = Q = 16)
  {
    constexpr int NA = HX ? kXP / 2 : kXP;
    const int r = threadIdx.x / kXP, j = threadIdx.x % kXP;
    const int row = rank * kRows + r;
    const float2* zr = reinterpret_cast<const float2*>(static_cast<const float*>(src_v) +
                                                       ((long long)z * a.nrows + row) * a.n1);
    float2* exr = ex + r * kXROW;
    float2 y[kXP];
#pragma unroll
    for (int aa = 0; aa < kXP; ++aa) y[aa] = aa < NA ? zr[j + kXQ * aa] : make_float2(0.f, 0.f);
    rdft<kXP, -1, HX>(y);
#pragma unroll
    for (int k1 = 1; k1 < kXP; ++k1) y[k1] = xmul(y[k1], __ldg(&twm[k1 * kXP + j]));  // W_M^{j k1}
#pragma unroll
    for (int k1 = 0; k1 < kXP; ++k1) exr[k1 * kXQP + j] = y[k1];
    __syncthreads();
    float2 x[kXQ];
    const float4* r4 = reinterpret_cast<const float4*>(exr + j * kXQP);
#pragma unroll
    for (int b2 = 0; b2 < kXQ / 2; ++b2) {
      const float4 q4 = r4[b2];
      x[2 * b2] = make_float2(q4.x, q4.y);
      x[2 * b2 + 1] = make_float2(q4.z, q4.w);
    }
    rdft<kXQ, -1, false>(x);
    cluster_wait();  // every CTA of the cluster is running: remote stores may start
    // thread j holds Z[k], k = j + 16 k2; Z[M - k] is in lane (16 - j) mod 16
    // of the row at index 15 - k2 (own registers for j = 0). Column k belongs
    // to CTA k2, where it is column j of row `row`.
    const int jp = (kXP - j) & (kXP - 1);
#pragma unroll
    for (int k2 = 0; k2 < kXQ; ++k2) {
      const float2 sv = x[kXQ - 1 - k2];
      const float2 tv = make_float2(__shfl_sync(0xffffffffu, sv.x, jp, kXP), __shfl_sync(0xffffffffu, sv.y, jp, kXP));
      const float2 zm = j == 0 ? x[(kXQ - k2) & (kXQ - 1)] : tv;
      const float2 zk = x[k2];
      const int k = j + kXP * k2;
      const float2 e = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      const float2 o = make_float2(0.5f * (zk.y + zm.y), -0.5f * (zk.x - zm.x));
      const float2 wo = xmul(o, __ldg(&tw1[k]));
      // X[k] = E + W^k O; slot 0 carries the real X[0] = E + O and X[M] = E - O as one complex number
      const float2 X = k == 0 ? make_float2(e.x + wo.x, e.x - wo.x) : make_float2(e.x + wo.x, e.y + wo.y);
      *(cluster.map_shared_rank(stage, k2) + row * kTK + j) = X;
    }
  }
  cluster.sync();  // every CTA's stage holds its 16 columns of all 256 rows

  // ---- y: lines kx = 16 rank + t (packed slot numbering), thread jj of the line
  const int t = threadIdx.x % kTK, jj = threadIdx.x / kTK;
  const int col = rank * kTK + t;
  c2 v[kYT];
#pragma unroll
  for (int aa = 0; aa < kYT / 2; ++aa) {  // rows jj + 32 aa and jj + 16 + 32 aa; n2 = 256
    const float2 u0 = stage[(jj + 2 * kYT * aa) * kTK + t];
    const float2 u1 = stage[(jj + kYT + 2 * kYT * aa) * kTK + t];
    v[aa] = {make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
  }
#pragma unroll
  for (int aa = kYT / 2; aa < kYT; ++aa) v[aa] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
  __syncthreads();  // the stage has been read: the region takes the y exchange
  soa::dft2<kYT, -1, true>(v);
#pragma unroll
  for (int k1 = 1; k1 < kYT; ++k1) v[k1] = cmul_pair<-1>(v[k1], tws[jj * (kYT + 1) + k1]);
#pragma unroll
  for (int k1 = 0; k1 < kYT; ++k1) sh4[(jj * kYT + k1) * kTK + t] = pack(v[k1]);
  __syncthreads();
  c2 w[kYT];
#pragma unroll
  for (int b = 0; b < kYT; ++b) w[b] = unpack(sh4[(b * kYT + jj) * kTK + t]);
  dif_all(w, std::make_integer_sequence<int, kYT>{});
  soa::dft2<kYT, -1, false>(w);
  // w[m] = (Y[jj + 32 m], Y[jj + 16 + 32 m]) of column col
  float2* const bz = static_cast<float2*>(dst_v) + (long long)z * a.dst_plane;
  const long long de = a.dst_elem;
  if (col != 0) {
    float2* p0 = bz + (long long)jj * de + col;
    float2* p1 = p0 + (long long)kYT * de;
#pragma unroll
    for (int m = 0; m < kYT; ++m) {
      *p0 = make_float2(w[m].re.x, w[m].im.x);
      *p1 = make_float2(w[m].re.y, w[m].im.y);
      p0 += 2 * kYT * de;
      p1 += 2 * kYT * de;
    }
  }
  if (rank == 0) {
    // the packed column Z = Y0 + i YM of the two real columns kx = 0 and kx = M
    if (t == 0) {
#pragma unroll
      for (int m = 0; m < kYT; ++m) {
        lin[jj + 2 * kYT * m] = make_float2(w[m].re.x, w[m].im.x);
        lin[jj + kYT + 2 * kYT * m] = make_float2(w[m].re.y, w[m].im.y);
      }
    }
    __syncthreads();
    for (int k = threadIdx.x; k < kYL; k += blockDim.x) {
      const float2 zk = lin[k], zm = lin[(kYL - k) & (kYL - 1)];
      bz[(long long)k * de] = make_float2(0.5f * (zk.x + zm.x), 0.5f * (zk.y - zm.y));
      bz[(long long)k * de + kM] = make_float2(0.5f * (zk.y + zm.y), 0.5f * (zm.x - zk.x));
    }
  }
}

// Inverse: B[z][ky][kx] -> V plane z (n2 = 256 rows kept; n1 = 256 (HX) or
// 512 reals kept of each C2R row). Grid: n3 clusters of kCS CTAs.
template <bool HX>
__global__ void __launch_bounds__(kNT, 2)
    k_xy_inv(const void* src_v, void* dst_v, const float* twm_v, const float4* __restrict__ tw4, FastArgs a,
             double*, unsigned*, double, double*) {
  cg::cluster_group cluster = cg::this_cluster();
  const int rank = (int)cluster.block_rank();
  const int z = blockIdx.x / kCS;
  const float2* __restrict__ twm = reinterpret_cast<const float2*>(twm_v);
  const float2* __restrict__ tw1 = a.tw1;
  extern __shared__ __align__(16) float4 smem4[];
  float2* const stage = reinterpret_cast<float2*>(smem4);    // [16 rows][256 columns], filled remotely
  float4* const sh4 = smem4 + kStage;                         // y exchange [kYT * kYT][kTK]
  float2* const ex = reinterpret_cast<float2*>(smem4 + kStage);  // x exchange [kRows][kXROW] (after the y one)
  float4* const tws = smem4 + kStage + kYEx;
  cluster_arrive_relaxed();  // this CTA is running
  load_y_twiddles(tws, tw4);
  pdl_wait();

  // ---- inverse y: lines kx = 16 rank + t (packed slot 0 = kx 0 + i kx M)
  {
    const int t = threadIdx.x % kTK, jj = threadIdx.x / kTK;
    const int col = rank * kTK + t;
    const float2* bz = static_cast<const float2*>(src_v) + (long long)z * a.src_plane + col;
    const long long se = a.src_elem;
    c2 w[kYT];
#pragma unroll
    for (int m = 0; m < kYT; ++m) {
      float2 u0 = bz[(long long)(jj + 2 * kYT * m) * se];
      float2 u1 = bz[(long long)(jj + kYT + 2 * kYT * m) * se];
      if (col == 0) {  // + i times the kx = M column
        const float2 q0 = bz[(long long)(jj + 2 * kYT * m) * se + kM];
        const float2 q1 = bz[(long long)(jj + kYT + 2 * kYT * m) * se + kM];
        u0 = make_float2(u0.x - q0.y, u0.y + q0.x);
        u1 = make_float2(u1.x - q1.y, u1.y + q1.x);
      }
      w[m] = {make_float2(u0.x, u1.x), make_float2(u0.y, u1.y)};
    }
    soa::dft2<kYT, 1, false>(w);
    dit_all(w, std::make_integer_sequence<int, kYT>{});
#pragma unroll
    for (int b = 0; b < kYT; ++b) w[b] = cmul_pair<1>(w[b], tws[b * (kYT + 1) + jj]);
#pragma unroll
    for (int b = 0; b < kYT; ++b) sh4[(b * kYT + jj) * kTK + t] = pack(w[b]);
    __syncthreads();
    c2 v[kYT];
#pragma unroll
    for (int k1 = 0; k1 < kYT; ++k1) v[k1] = unpack(sh4[(jj * kYT + k1) * kTK + t]);
    soa::dft2<kYT, 1, false, true>(v);  // rows jj + 32 aa and jj + 16 + 32 aa, aa < 8 (n2 = 256)
    cluster_wait();  // every CTA of the cluster is running: remote stores may start
    // row y belongs to CTA y / 16, where it is row y % 16 (= jj): column col
#pragma unroll
    for (int aa = 0; aa < kYT / 2; ++aa) {
      *(cluster.map_shared_rank(stage, 2 * aa) + jj * kM + col) = make_float2(v[aa].re.x, v[aa].im.x);
      *(cluster.map_shared_rank(stage, 2 * aa + 1) + jj * kM + col) = make_float2(v[aa].re.y, v[aa].im.y);
    }
  }
  cluster.sync();  // every CTA's stage holds its 16 rows of all 256 columns

  // ---- inverse x (C2R): rows y = 16 rank + r, thread j; X[k], k = j + 16 i
  constexpr int NA = HX ? kXP / 2 : kXP;
  const int r = threadIdx.x / kXP, j = threadIdx.x % kXP;
  const int row = rank * kRows + r;
  float2 xin[kXQ];
#pragma unroll
  for (int i = 0; i < kXQ; ++i) xin[i] = stage[r * kM + j + kXP * i];
  // slot 0 of the row: X[0] + i X[M], both real
  const float2 xny = make_float2(xin[0].y, 0.f);
  if (j == 0) xin[0] = make_float2(xin[0].x, 0.f);
  float2 x[kXQ];
  {
    const int jp = (kXP - j) & (kXP - 1);
#pragma unroll
    for (int k2 = 0; k2 < kXQ; ++k2) {
      const float2 sv = xin[kXQ - 1 - k2];
      const float2 tv = make_float2(__shfl_sync(0xffffffffu, sv.x, jp, kXP), __shfl_sync(0xffffffffu, sv.y, jp, kXP));
      const float2 xm = j != 0 ? tv : (k2 == 0 ? xny : xin[(kXQ - k2) & (kXQ - 1)]);
      const float2 xk = xin[k2];
      const int k = j + kXP * k2;
      const float2 e = make_float2(xk.x + xm.x, xk.y - xm.y);
      const float2 o = xmulc(make_float2(xk.x - xm.x, xk.y + xm.y), __ldg(&tw1[k]));
      x[k2] = make_float2(e.x - o.y, e.y + o.x);
    }
  }
  rdft<kXQ, 1, false>(x);
#pragma unroll
  for (int b = 1; b < kXQ; ++b) x[b] = xmulc(x[b], __ldg(&twm[b * kXP + j]));
  float2* exr = ex + r * kXROW;
  {
    float4* w4 = reinterpret_cast<float4*>(exr + j * kXQP);
#pragma unroll
    for (int b2 = 0; b2 < kXQ / 2; ++b2)
      w4[b2] = make_float4(x[2 * b2].x, x[2 * b2].y, x[2 * b2 + 1].x, x[2 * b2 + 1].y);
  }
  __syncthreads();
  float2 y[kXP];
#pragma unroll
  for (int k1 = 0; k1 < kXP; ++k1) y[k1] = exr[k1 * kXQP + j];
  rdft<kXP, 1, false>(y);
  float2* vz = reinterpret_cast<float2*>(static_cast<float*>(dst_v) + ((long long)z * a.nrows + row) * a.n1);
#pragma unroll
  for (int aa = 0; aa < NA; ++aa) vz[j + kXQ * aa] = y[aa];
}

const void* xy_kernel(int kind, bool half, int* threads, size_t* smem, int* cluster) {
  *threads = kNT;
  *cluster = kCS;
  // forward: stage and x exchange (the y exchange overlays them), the paired
  // y twiddles, the packed column's line; inverse: stage, y exchange (the x
  // exchange overlays it), the paired y twiddles
  *smem = kind == 0 ? (size_t)kRegion * sizeof(float4) + (size_t)kYT * (kYT + 1) * sizeof(float4) +
                          (size_t)kYL * sizeof(float2)
                    : (size_t)(kStage + kYEx) * sizeof(float4) + (size_t)kYT * (kYT + 1) * sizeof(float4);
  if (kind == 0) return half ? (const void*)k_xy_fwd<true> : (const void*)k_xy_fwd<false>;
  return half ? (const void*)k_xy_inv<true> : (const void*)k_xy_inv<false>;
}

}  // namespace ps
