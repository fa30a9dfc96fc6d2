// Specialised FP32 pass kernels: register-resident four-step transforms for
// power-of-two lengths, selected per pass by configure_fast_f32.
#pragma once

#include "common.cuh"

namespace ps {

// z-pass tile row y -> ky, a bijection of [0, L2) that puts the rows ky and
// L2 - ky, which read the same K^F octant row, next to each other (the
// second read hits L2): 0, then L2/2 when L2 is even, then the pairs
// (p, L2 - p) for p = 1, 2, ...
__device__ __forceinline__ int paired_ky(int y, int L2) {
  if (y == 0) return 0;
  if ((L2 & 1) == 0) {
    if (y == 1) return L2 / 2;
    const int p = (y - 2) / 2 + 1;
    return (y & 1) ? L2 - p : p;
  }
  const int p = (y - 1) / 2 + 1;
  return (y & 1) ? p : L2 - p;
}

// Every specialised kernel starts with this wait: it is launched with
// programmatic stream serialisation, so its CTAs may start while the previous
// kernel of the stream finishes; the wait returns once that kernel has
// completed and its writes are visible (immediately for an ordinary launch).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Asynchronous global -> shared copies (cp.async): 16 bytes (L2 only), 16
// bytes of zeros (nothing is read), 8 bytes; commit and wait for all groups.
__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async16_zero(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, 0;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async8(void* smem, const void* gmem) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;\n" ::: "memory"); }

// Kernel signature shared by every specialised pass kernel.
//   src, dst   pass input / output (A, B, rho or V)
//   K          K^F octant (z pass only)
//   tw         twiddle table W_L^k of the pass's axis
using FastKernel = void (*)(const void*, void*, const float*, const float2*, FastArgs, double*,
                            unsigned*, double, double*);

// Returns the kernel for a y/z pass of length L, or nullptr.
//   kind 0: forward (n nonzero inputs, L outputs), 1: inverse (L inputs,
//   n outputs), 2: forward, K^F multiply, inverse; half: n = L/2 (else n = L)
const void* strided_kernel(int L, int kind, bool half, int* threads, size_t* smem, int* tk);
// Returns the kernel for an x pass (real length 2M): kind 0 R2C, 1 C2R.
const void* xline_kernel(int M, int kind, bool half, int* threads, int* rows, size_t* smem);

// The persistent packed y-pass kernels (L2 = 512), or nullptr.
const void* ysoa_kernel(int L, int kind, bool half, int* threads, size_t* smem, int* tk);

// The persistent, prefetching y-pass kernels (L2 = 256, 512), or nullptr.
const void* ypipe_kernel(int L, int kind, bool half, int* threads, size_t* smem, int* tk);
// persistent unpacked z kernel (L = 1024) and its lines per tile
const void* zpipe_u_kernel(int L, bool half, int* threads, size_t* smem, int* tk);
// persistent packed z kernel for L = 256 (pairs of columns, then of rows)
const void* zpipe_q_kernel(int L, bool half, int* threads, size_t* smem, int* tk);

// The persistent, prefetching packed z-pass kernel (L3 = 512), or nullptr.
// tk lines per tile (8 or 16).
// *tk: requested in, used out; *P: rows of the four-step factorisation L = P * 2T
const void* zpipe_kernel(int L, bool half, int* tk, int* threads, size_t* smem, int* P);

// The tensor-core z-pass kernel (L3 = 512; half: n3 = 256, else n3 = 512),
// its table size in floats and the host fill of that table.
const void* ztc_kernel(int L, bool half, int* threads, size_t* smem);
size_t ztc_table_floats(bool half);
void ztc_fill_table(bool half, float* out);

// The fused x/y kernels (fast_xy.cu; kind 0 forward, 1 inverse) for L1 = 512
// (half: n1 = 256, else 512) and L2 = 512 with n2 = 256, and their launch shape.
const void* xy_kernel(int kind, bool half, int* threads, size_t* smem, int* cluster);

// Fills p->cfg[k].fast / fn / grid / block / smem / fa for the passes covered.
cudaError_t configure_fast_f32(ps_plan_s* p);

// Launches pass `pass` with its specialised kernel.
cudaError_t launch_fast(ps_plan_s* p, int pass, const void* src, void* dst, double* E, double escale,
                        cudaStream_t s);
// Launches the fused forward (kind 0: rho -> B) or inverse (kind 1: B -> V) x/y kernel.
cudaError_t launch_xy(ps_plan_s* p, int kind, const void* src, void* dst, cudaStream_t s);
// Launches x pass P1 / P5 or y pass P2 / P4 on the z planes z0 .. z0 + nz - 1:
// rho, V and B at those planes, A (src or dst) at its first plane.
cudaError_t launch_fast_chunk(ps_plan_s* p, int pass, const void* rhoV, void* B, void* A, int z0, int nz,
                              cudaStream_t s);

}  // namespace ps
