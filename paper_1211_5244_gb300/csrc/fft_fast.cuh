// Specialised FP32 pass kernels: register-resident four-step transforms for
// power-of-two lengths, selected per pass by configure_fast_f32.
#pragma once

#include "common.cuh"

namespace ps {

// Kernel signature shared by every specialised pass kernel.
//   src, dst   pass input / output (A, B, rho or V)
//   K          K^F octant (z pass only)
//   tw         twiddle table W_L^k of the pass's axis
using FastKernel = void (*)(const void*, void*, const float*, const float2*, FastArgs, double*,
                            unsigned*, double, double*);

// Returns the kernel for a y/z pass of length L, or nullptr.
//   kind 0: forward (n nonzero inputs, L outputs), 1: inverse (L inputs,
//   n outputs), 2: forward, K^F multiply, inverse; half: n = L/2 (else n = L)
const void* strided_kernel(int L, int kind, bool half, int* threads, size_t* smem);
// Returns the kernel for an x pass (real length 2M): kind 0 R2C, 1 C2R.
const void* xline_kernel(int M, int kind, bool half, int* threads, int* rows, size_t* smem);

// The packed FP32x2 z-pass kernel for L3 = 2 T^2 (T = 8, 16) with tk lines
// per CTA (8 or 16), or nullptr.
const void* zsoa_kernel(int L, bool half, int tk, int* threads, size_t* smem);

// The persistent packed y-pass kernels (L2 = 512), or nullptr.
const void* ysoa_kernel(int L, int kind, bool half, int* threads, size_t* smem);

// The persistent, prefetching y-pass kernels (L2 = 256, 512), or nullptr.
const void* ypipe_kernel(int L, int kind, bool half, int* threads, size_t* smem);

// The persistent, prefetching packed z-pass kernel (L3 = 512), or nullptr.
const void* zpipe_kernel(int L, bool half, int* threads, size_t* smem);

// Fills p->cfg[k].fast / fn / grid / block / smem / fa for the passes covered.
cudaError_t configure_fast_f32(ps_plan_s* p);

// Launches pass `pass` with its specialised kernel.
cudaError_t launch_fast(ps_plan_s* p, int pass, const void* src, void* dst, double* E, double escale,
                        cudaStream_t s);

}  // namespace ps
