// Internal definitions shared by the CUDA translation units of libpsolver.
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <vector>

#include "psolver.h"

namespace ps {

// ---------------------------------------------------------------- complex

template <typename T> struct CT;
template <> struct CT<float> { using type = float2; };
template <> struct CT<double> { using type = double2; };
template <typename T> using cpx = typename CT<T>::type;

__host__ __device__ __forceinline__ float2 mk(float a, float b) { return make_float2(a, b); }
__host__ __device__ __forceinline__ double2 mk(double a, double b) { return make_double2(a, b); }

template <typename C> __device__ __forceinline__ C cadd(C a, C b) { return mk(a.x + b.x, a.y + b.y); }
template <typename C> __device__ __forceinline__ C csub(C a, C b) { return mk(a.x - b.x, a.y - b.y); }
template <typename C> __device__ __forceinline__ C cmul(C a, C b) {
  return mk(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
// a * conj(b)
template <typename C> __device__ __forceinline__ C cmulc(C a, C b) {
  return mk(a.x * b.x + a.y * b.y, a.y * b.x - a.x * b.y);
}
template <typename C> __device__ __forceinline__ C cconj(C a) { return mk(a.x, -a.y); }
// multiply by +i (s = +1) or -i (s = -1)
template <int S, typename C> __device__ __forceinline__ C cmul_i(C a) {
  return S > 0 ? mk(-a.y, a.x) : mk(a.y, -a.x);
}
template <typename C, typename R> __device__ __forceinline__ C cscale(C a, R s) {
  return mk(a.x * s, a.y * s);
}

// ---------------------------------------------------------------- radix plans

constexpr int kMaxStages = 16;
constexpr int kMaxLen = 4096;

// x / d for an invariant divisor d >= 1 as one multiply-high by m = ceil(2^32 / d)
// (m = 0 stands for d = 1). With m d = 2^32 + e, 0 <= e < d, the quotient
// x m / 2^32 = x / d + x e / (d 2^32) is exact whenever x d < 2^32, which the
// tile and stage indices (x < 2^20, d <= 4097) satisfy.
inline unsigned div_magic(unsigned d) { return d <= 1 ? 0u : (unsigned)(((1ull << 32) + d - 1) / d); }
__device__ __forceinline__ int div_by(int x, unsigned m) { return m ? (int)__umulhi((unsigned)x, m) : x; }

// Factorisation of a transform length into Stockham stages (radix per stage).
struct Stages {
  int n;                 // number of stages (0 for length 1)
  int R[kMaxStages];
  unsigned mg[kMaxStages];  // div_magic of the sub-length Ns entering each stage
};

// ---------------------------------------------------------------- plan

enum Pass { P1 = 0, P2 = 1, P3 = 2, P4 = 3, P5 = 4 };

// Bluestein (chirp-z) form of a transform of length N with a large prime
// factor: a cyclic convolution of length M >= 2N - 1 (factors 2, 3, 5).
struct BlueArgs {
  int M;              // 0: the transform runs as plain Stockham stages
  Stages st;          // stages of the length-M transforms
  const void* twM;    // W_M^k, k < M
  const void* chirp;  // c[m] = exp(-i pi m^2 / N), m < N
  const void* Bf;     // DFT_M of the conjugate chirp, divided by M
};

// Arguments of the specialised FP32 pass kernels (strides in complex elements).
struct FastArgs {
  int c;                  // valid kx columns (L1/2 + 1)
  int L1, L2;
  int n1, nrows;          // x passes: row length (reals) and row count
  long long ldc;          // row pitch of A / B
  int ldk;                // kx pitch of the K^F octant
  long long src_plane, src_elem;
  long long dst_plane, dst_elem;
  long long kz_stride;    // z pass: (L2/2 + 1) * ldk, the kz stride of the K^F octant
  int kt0, ntk_loc;       // persistent y/z kernels: first kx tile and number of kx tiles walked
  int nl;                 // y/z passes: physical points along the line (n2 or n3); rows at and
                          // beyond nl are zero on input and not stored on output
  int rev;                // walk the z planes (y passes) or rows (x passes) from the last one:
                          // the previous pass wrote them last, so they are still in L2
  const float2* tw1;      // fused x/y kernels: W_L1^k, k < L1 (set at launch)
};

struct PassCfg {
  int tk;       // lines (tile width) per CTA
  int ldt;      // shared-memory row stride in complex elements
  int threads;  // threads per CTA
  size_t smem;  // dynamic shared memory bytes (of the specialised kernel when `fast`)
  size_t gsmem; // dynamic shared memory bytes of the generic kernel of the pass (the x passes
                // fall back to it when rho or V is not 8-byte aligned)
  int twn;      // generic passes: twiddle entries kept in shared memory (0: read from global memory)
  int bm;       // generic FP32 passes in Bluestein form: the power-of-two M of the register
                // four-step convolution (0: Stockham stages)
  int fast;     // 1 if a compile-time specialised kernel runs this pass
  const void* fn;  // the specialised kernel
  dim3 grid, block;
  int cluster;  // CTAs per thread-block cluster (0: launched without clusters)
  int xrows;    // specialised x passes: rows per CTA
  FastArgs fa;
};

}  // namespace ps

struct ps_plan_s {
  int n[3];
  int bc[3];
  int L[3];
  // physical axes (0 x, 1 y, 2 z) in forward processing order (§3: periodic
  // axes first, free axes last): ord[0] takes the real-to-complex transform
  // and keeps L/2 + 1 outputs, ord[2] the K^F multiply; the inverse runs in
  // the reverse order
  int ord[3];
  int ext1[3], ext2[3];  // extents (x, y, z) of the arrays after the first and second forward passes
  int fastord;           // an order other than x, y, z that starts with x runs the specialised kernels
  size_t ld1, ld2;       // their x pitch in complex elements
  int H[3];      // L/2 (floor): last index of the even octant per axis
  int c;         // L1/2 + 1
  double h;
  int dtype;
  int math;
  int gen_tk_max;  // most lines per tile of the generic passes (0: 16 for FP32, 8 for FP64)
  bool built;
  int device;
  size_t esz;    // bytes per real element
  size_t ldc;    // row pitch of the spectral work arrays, complex elements
  size_t ldk;    // kx pitch of the stored K^F octant (c rounded up to 16), real elements
  // device memory owned by the plan
  void* A;       // [n3][n2][ldc] complex: x-transformed rows (passes 1/2 and 4/5)
  void* B;       // [n3][L2][ldc] complex: y-transformed planes (passes 2..4)
  void* K;       // [H3+1][H2+1][ldk] real: K^F / (L1 L2 L3), even octant (kx < c used)
  void* tw[3];   // W_{L_j}^k, k < L_j, complex, per axis
  void* tw4z;    // paired z twiddles of the packed z kernel (T*T float4), or NULL
  void* tw4y;    // paired y twiddles of the packed y kernels (16*16 float4), or NULL
  void* twx;     // x passes: W_M^{r c}, r, c < xP (float2, M = L1/2), or NULL
  int xP;        // size of twx (the larger step of the x-pass factorisation)
  int ysoa;      // packed y kernels (L2 = 512): bit 0 forward, bit 1 inverse
  int zsoa_T;    // T of the packed z kernel (L3 = P * 2T), 0 if not used
  int zsoa_P;    // P of the packed z kernel (T, or 12 at L3 = 384)
  void* tctab;   // tensor-core z pass: DFT matrices (hi, lo) and twiddles, or NULL
  size_t tctab_floats;
  double* partials;     // per-CTA energy partials of the z pass
  unsigned* counter;    // [0] arrival counter of the last-CTA energy reduction,
                        // [1] device status: nonzero once a bounded wait gave up
  int npart;
  void* d_rho;   // staging for ps_solve_host (and slot 0 of ps_solve_host_stream)
  void* d_V;
  double* d_E;   // two doubles: one per ps_solve_host_stream slot
  void* d_rho2;  // slot 1 of ps_solve_host_stream
  void* d_V2;
  double* d_Eb;           // energies of a ps_solve_host_stream batch (grown as needed)
  int d_Eb_cap;
  cudaStream_t hs[3];     // upload, compute, download streams of ps_solve_host_stream
  cudaEvent_t hev[7];     // per-slot upload / compute / download events, and a start event
  size_t ws_bytes;
  ps::Stages st[3];     // stages of the 1D transform per axis (x: length L1/2 if L1 even)
  ps::BlueArgs blue[3]; // Bluestein descriptors per axis (M = 0: off); device pointers owned
  ps::PassCfg cfg[5];
  // fused x/y passes (thread-block clusters): xyf[0] runs passes 1 and 2,
  // xyf[1] passes 4 and 5, when xyfuse is set and rho and V are 16-byte aligned
  int xyfuse;
  ps::PassCfg xyf[2];
  // kernel schedule (chosen by ps_plan_autotune; 0 = the default choice):
  int xy_sched;    // 1: fused x/y passes where they apply
  int z_tk;        // lines per tile of the persistent packed z kernel (8 or 16)
  int y_kind;      // y passes: 1 unpacked persistent kernels, 2 non-persistent ones
  int radix_pref;  // generic Stockham stages: 0 radix 8 first, 1 radix 4 and 2 only
  int tile_ax[3];  // per physical axis: most lines per generic tile of its passes (0: gen_tk_max)
  int radix_ax[3]; // per physical axis: radix split of its Stockham stages (-1: radix_pref)
  int chunk_req;   // chunks of z planes for the x and y passes (0: chosen by size, 1: none)
  // the x and y passes run chunk by chunk of z planes (x then y for each
  // chunk forward, y then x inverse) through the first chunk's rows of A, which
  // stay in L2 between the two passes; 1: whole passes
  int chunks;
  // per-pass timing (ps_plan_set_profiling): 6 events per recorded solve
  bool profiling;
  std::vector<cudaEvent_t> events;
  size_t events_used;
};

namespace ps {
// the generic tile width limit and radix split of the passes along physical axis j
inline int axis_tile(const ps_plan_s* p, int j) { return p->tile_ax[j] ? p->tile_ax[j] : p->gen_tk_max; }
inline int axis_radix(const ps_plan_s* p, int j) { return p->radix_ax[j] >= 0 ? p->radix_ax[j] : p->radix_pref; }
}  // namespace ps

namespace ps {

// The plan processes x first and y second (the specialised kernels' layout).
inline bool canonical_order(const ps_plan_s* p) { return p->ord[0] == 0 && p->ord[1] == 1 && p->ord[2] == 2; }

// Length of the complex 1D transforms along physical axis j: an even-length x
// axis that takes the real-to-complex transform runs it as a complex
// transform of half the length; every other axis at its full length (a
// real-to-complex transform along y or z pairs two real lines).
inline int xform_len(const ps_plan_s* p, int j) {
  return (j == 0 && p->ord[0] == 0 && p->L[0] % 2 == 0) ? p->L[0] / 2 : p->L[j];
}

// Physical axis transformed by pass k (0 fwd first axis .. 4 inv first axis).
inline int pass_axis(const ps_plan_s* p, int k) {
  static const int slot[5] = {0, 1, 2, 1, 0};
  return p->ord[slot[k]];
}

// Error reporting (thread-local message), defined in api.cu.
void set_error(const char* fmt, ...);

// Radix factorisation used by the generic kernels (pref 1: no radix-8 stages).
Stages factorize(int N, int pref = 0);
// M if a Bluestein convolution of length M for a transform of length N runs
// in the register four-step form (M a power of two, 32 <= M <= 1024, M >= 2N), else 0
int blue_regs_length(int M, int N);

// Launchers (defined in passes.cu / kernel_build.cu). They only enqueue.
template <typename T>
cudaError_t configure_passes(ps_plan_s* p);
template <typename T>
cudaError_t launch_solve(ps_plan_s* p, const T* rho, T* V, double* E, cudaStream_t s,
                         cudaEvent_t* ev);
template <typename T>
cudaError_t launch_vjp_axpy(ps_plan_s* p, T* out, const T* V, const double* gE, bool accumulate,
                            cudaStream_t s);
// passes_ord.cu: the solve for a processing order other than x, y, z
template <typename T>
cudaError_t launch_solve_ord(ps_plan_s* p, const T* rho, T* V, double* E, cudaStream_t s, cudaEvent_t* ev);
// energy partials (CTAs of the fused pass) of a plan in another order, and
// the launch attributes of its kernels
int ord_conv_ctas(const ps_plan_s* p);
template <typename T>
cudaError_t configure_ord(const ps_plan_s* p);
// rows of each shared-memory buffer of a generic pass (passes.cu)
int gen_rows(const ps_plan_s* p, int pass);
// passes.cu: the generic x pass (P1 forward R2C, P5 inverse C2R) of a plan
// that processes x first, on A with pitch ld1
template <typename T>
cudaError_t launch_x_pass(ps_plan_s* p, int pass, const void* src, void* dst, cudaStream_t s);
cudaError_t build_twiddles(ps_plan_s* p, cudaStream_t s);
// batch.cu: the batch as one cached CUDA graph of concurrent per-problem chains
cudaError_t batch_solve_graph(int count, ps_plan_s* const* plans, const void* const* rho, void* const* V,
                              double* E, int device, cudaStream_t s);
void batch_forget_plan(const ps_plan_s* p);
cudaError_t build_kernel(ps_plan_s* p, cudaStream_t s);
// K^F from a caller's real-space kernel on its even octant (host, FP64)
cudaError_t build_kernel_from_real(ps_plan_s* p, const double* host_octant, cudaStream_t s);

}  // namespace ps
