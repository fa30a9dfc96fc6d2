/*
 * psolver.h -- C ABI of the GB300 free/mixed-boundary FFT Poisson solver.
 *
 * Method (Dugan, Genovese, Goedecker, "A Customized 3D GPU Poisson Solver for
 * Free Boundary Conditions"):
 *   Eq. 1   laplacian(V) = rho            (sign as printed, no -4 pi)
 *   Eq. 2   V(r) = sum_r' K(r - r') rho(r')
 *   Eq. 3   V^F(k) = K^F(k) rho^F(k)
 *   §2      free axes are zero padded to twice their length (any padded length
 *           L >= 2n - 1 gives the same physical result); periodic axes are
 *           transformed at their own length n
 *   §3      the 3D FFT skips every 1D transform of an all-zero line on the
 *           forward pass, computes only the physical n-wide output on the
 *           inverse pass, uses a real-to-complex transform on the first axis
 *           and keeps L1/2 + 1 of its outputs, and stores K^F in the layout of
 *           the last forward axis so that no final transpose is needed.
 *
 * Conventions shared by every entry point
 *   - Grids are real arrays of n1*n2*n3 elements, x fastest:
 *       rho[i + n1*(j + n2*k)],  i < n1 (x), j < n2 (y), k < n3 (z).
 *     In PyTorch this is a contiguous (n3, n2, n1) tensor.
 *   - The element type is the plan's dtype: float (PS_F32) or double (PS_F64).
 *   - "device pointer" means memory of the device the plan was built on;
 *     "host pointer" means ordinary or pinned host memory.
 *   - Every call returns a status (enum ps_status). PS_OK is 0. On error
 *     nothing has been launched unless the status is PS_ERR_CUDA (a launch or
 *     runtime call failed); ps_last_error() then holds a message for the
 *     calling thread.
 *   - Calls that take a stream enqueue their work on it (NULL = the legacy
 *     default stream) and return without waiting, except where noted.
 *   - A plan owns its workspace and K^F. One plan must not be used by two
 *     solves that may run at the same time (two streams); give each stream
 *     its own plan.
 */
#ifndef PSOLVER_H
#define PSOLVER_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ps_plan_s* ps_plan;

/* Boundary condition per axis. The paper's B_j = 1 (periodic) / 2 (free), §3. */
enum ps_bc { PS_BC_PERIODIC = 0, PS_BC_FREE = 1 };

/* Element type of rho and V, and of the arithmetic of the solve. */
enum ps_dtype { PS_F32 = 0, PS_F64 = 1 };

/* Arithmetic of the 1D transforms.
 * PS_MATH_CUDACORE: register FFTs on the CUDA cores (every plan).
 * PS_MATH_TF32X3:   FP32 plans only. Where a tensor-core kernel exists (today
 *   the z pass of L3 = 512 with n3 = 256 or 512) its DFT stages run as
 *   dense products with small DFT matrices on the tensor cores (tcgen05),
 *   each operand split into a TF32 part and a remainder, the partial
 *   products accumulated in FP32 in two halves (those with the matrix's TF32
 *   part, those with its remainder) that the CUDA cores add (about FP32
 *   accuracy); the other passes stay on the CUDA cores, and the energy is
 *   the real-space sum 1/2 h^3 sum rho V accumulated in FP64 after the last
 *   pass. ps_plan_query's tensor_passes tells which passes use the tensor cores.
 * PS_MATH_BF16X3:   split-BF16 tensor-core stages. Not built: this build's
 *   ps_plan_set_math returns PS_ERR_UNSUPPORTED for it. FP32-level accuracy
 *   from BF16 needs every operand split into three BF16 terms and six of the
 *   nine partial products, about 1.5 times the MMA columns of the TF32 form
 *   and twice its operand splitting on the CUDA cores, and the TF32 form is
 *   already slower than the CUDA-core stages on this GPU. */
enum ps_math { PS_MATH_CUDACORE = 0, PS_MATH_TF32X3 = 1, PS_MATH_BF16X3 = 2 };

enum ps_status {
  PS_OK = 0,
  PS_ERR_ARG = 1,          /* invalid argument (sizes, enums, null pointers) */
  PS_ERR_UNSUPPORTED = 2,  /* valid but outside what this build handles      */
  PS_ERR_NOT_BUILT = 3,    /* ps_kernel_build has not run on this plan       */
  PS_ERR_CUDA = 4,         /* a CUDA runtime call or launch failed           */
  PS_ERR_OOM = 5,          /* device allocation failed                       */
  PS_ERR_TIMEOUT = 6       /* reserved: a bounded device wait gave up        */
};

/* Host-side description of a plan (ps_plan_query). */
typedef struct {
  int n[3];                 /* physical grid n1, n2, n3                           */
  int bc[3];                /* enum ps_bc per axis x, y, z                        */
  int L[3];                 /* FFT length per axis (§3: S_j = N_j B_j by default) */
  int c;                    /* L/2 + 1 of the first axis of the processing order:
                               the spectrum kept after the R2C (§3)             */
  int dtype;                /* enum ps_dtype                                      */
  int math;                 /* enum ps_math                                       */
  long long lines[5];       /* 1D transforms per pass, in processing order
                               (order[] below; x, y, z by default): fwd first
                               axis, fwd second axis, last axis (each of its
                               lines is transformed forward and back), inv
                               second axis, inv first axis                      */
  long long line_len[5];    /* their lengths                                      */
  double fft_points;        /* sum over the passes above of lines * length (the
                               last axis's lines counted twice)                  */
  double paper_points;      /* §3 count for one forward 3D transform: rows times
                               length per step with complex rows, in processing
                               order a, b, c: N_b N_c S_a + S_a N_c S_b +
                               S_a S_b S_c                                       */
  double paper_full_points; /* the same count for an unpruned padded 3D FFT,
                               3 S_x S_y S_z (paper_points / paper_full_points is
                               7/12 for free and wire, 2/3 for surface BCs, with
                               the paper's axis order)                           */
  double alg_bytes;         /* HBM bytes one solve must move in this design:
                               rho in, V out, the intermediate write+read pairs
                               (four; two where the x and y passes are fused),
                               and one read of the stored K^F octant            */
  size_t workspace_bytes;   /* device bytes the plan allocates at build          */
  int launches;             /* kernels one ps_solve launches (0 before build)    */
  int tensor_passes;        /* bit k set: pass k (0 fwd x .. 4 inv x) runs on the
                               tensor cores (0 before build)                     */
  int blocks[5];            /* CTAs launched per pass by its specialised kernel
                               (0 before build and where the generic kernel runs;
                               a fused pass reports the CTAs of its kernel)      */
  int fused;                /* bit 1: the forward y pass runs inside the forward x
                               kernel, bit 4: the inverse x pass inside the
                               inverse y kernel (thread-block clusters exchange
                               each z plane through distributed shared memory;
                               used when rho and V are 16-byte aligned)         */
  int order[3];             /* physical axes (0 x, 1 y, 2 z) in forward
                               processing order (ps_plan_set_order)             */
  int schedule[6];          /* kernel schedule requested (0 = default): generic
                               lines per tile, generic radix split (1: radix 4
                               only), lines per tile of the persistent packed z
                               kernel, y kernel form (1 unpacked persistent, 2
                               non-persistent), fused x/y passes (1), chunks   */
  int chunks;               /* chunks of z planes in which the x and y passes
                               run (forward x then y per chunk, inverse y then
                               x), through one chunk of the x-transformed array
                               that stays in L2 (1: whole passes; 0 before the
                               build; used when rho and V are 8-byte aligned)  */
  int axis_schedule[3][2];  /* per physical axis (x, y, z): generic lines per
                               tile and radix split of the passes along it, as
                               set by ps_plan_set_axis_schedule (0 and -1: the
                               plan-wide schedule[0] and schedule[1])          */
} ps_plan_info;

/*
 * ps_plan_create -- describe a solve; allocates host memory only.
 *   n1, n2, n3 >= 1      physical grid (x, y, z)
 *   h > 0                grid spacing (isotropic), in the length unit of V
 *   bc_x, bc_y, bc_z     enum ps_bc
 *   dtype                enum ps_dtype
 *   out                  receives the plan (caller frees with ps_plan_destroy)
 * Free axes get the paper's padded length L = 2n; periodic axes L = n.
 * Errors: PS_ERR_ARG for n < 1, h <= 0 or NaN, a bad enum or out == NULL;
 * PS_ERR_UNSUPPORTED if a length exceeds this build's maximum (4096).
 */
int ps_plan_create(int n1, int n2, int n3, double h, int bc_x, int bc_y, int bc_z,
                   int dtype, ps_plan* out);

/*
 * ps_plan_set_lengths -- override the padded length of free axes before the
 * build. Any L >= 2n - 1 gives the same physical result (§2); a smooth length
 * (factors 2, 3, 5, 7) is cheaper than 2n when 2n has a large prime factor.
 * Pass 0 to keep an axis's current length. Periodic axes must keep L = n.
 * Errors: PS_ERR_ARG (plan NULL, L too small, periodic L != n, plan built).
 */
int ps_plan_set_lengths(ps_plan plan, int L1, int L2, int L3);

/*
 * ps_plan_set_order -- the processing order of the axes (0 x, 1 y, 2 z):
 * axis a0 takes the forward real-to-complex transform (keeping L/2 + 1
 * outputs), a1 the second forward transform, a2 the last one with the K^F
 * multiply; the inverse runs in the reverse order. ps_plan_create sets §3's
 * rule: periodic axes first (their transforms run before any zero padding
 * exists), free axes last, so that wire BCs do 7/12 and surface BCs 2/3 of a
 * full padded 3D FFT's 1D transforms for any assignment of the axes. Orders
 * other than x, y, z run the generic kernels along strided axes (the
 * specialised FP32 kernels, the fused x/y passes and the tensor-core z pass
 * need x first); every order gives the same result up to rounding. No
 * transpose: the passes index the x-fastest arrays through strides.
 * Errors: PS_ERR_ARG (plan NULL or built, not a permutation of 0, 1, 2).
 */
int ps_plan_set_order(ps_plan plan, int a0, int a1, int a2);

/*
 * ps_plan_autotune -- choose the padded lengths of the free axes and the
 * kernel schedule by timing. Any L >= 2n - 1 gives the same physical result
 * (§2); the candidates are the paper's 2n, the smallest lengths >= 2n - 1
 * made of the factors {2}, {2, 3} and {2, 3, 5, 7}, and the smallest length
 * >= 2n - 1 with register-resident FP32 kernels (a power of two, 96, 192 or
 * 384). Then, at the fastest lengths, each schedule
 * choice that applies to the plan is timed in turn and kept if faster: the
 * lines per tile of the generic passes, their radix split (radix 8 first or
 * radix 4 only), both again per physical axis, the lines per tile of the persistent packed z kernel, the y
 * kernel form (packed persistent, unpacked persistent, non-persistent), the
 * fused x/y passes (see ps_plan_info.fused), the chunks of the x and y passes
 * and, for a plan whose order is not x first, the x-first order. One trial plan per candidate
 * is built on the current device and `reps` solves of it are timed on
 * `stream` (reps < 1 means 5); the choice is set on `plan` (not built; see
 * ps_plan_info.schedule). Results are cached per geometry and device in
 * memory and, when the environment variable PS_TUNE_CACHE names a file, in
 * that file. Must precede ps_kernel_build; synchronises `stream`.
 * Errors: PS_ERR_ARG (plan NULL or built), PS_ERR_OOM, PS_ERR_CUDA.
 */
int ps_plan_autotune(ps_plan plan, int reps, void* stream);

/* ps_plan_set_math -- enum ps_math; must precede the build (PS_ERR_ARG
 * otherwise, and for an unknown mode). PS_MATH_TF32X3 on an FP64 plan, and
 * PS_MATH_BF16X3 on any plan: PS_ERR_UNSUPPORTED. */
int ps_plan_set_math(ps_plan plan, int math_mode);

/*
 * ps_plan_set_schedule -- choose the kernel schedule by hand before the build
 * (ps_plan_autotune chooses it by timing). Every choice gives the same result
 * up to rounding; a choice that does not apply to the plan's shapes is
 * ignored. 0 keeps a field's default.
 *   tile    most lines per tile of the generic passes: 0, 1, 2, 4, 8, 16 or 32
 *   radix   generic Stockham stages: 0 radix 8 first, 1 radix 4 and 2 only
 *   ztk     lines per tile of the persistent packed z kernel: 0, 8 or 16
 *   ykind   y kernels: 0 default, 1 unpacked persistent, 2 non-persistent
 *   xy      1: fused x/y passes where the shapes have them (ps_plan_info.fused)
 *   chunks  the x and y passes chunk by chunk of z planes (2 .. 64), or whole
 *           (0 or 1; see ps_plan_info.chunks)
 * Errors: PS_ERR_ARG (plan NULL or built, a value out of range).
 */
int ps_plan_set_schedule(ps_plan plan, int tile, int radix, int ztk, int ykind, int xy, int chunks);

/*
 * ps_plan_set_axis_schedule -- the generic-kernel choices of ps_plan_set_schedule
 * for the passes along one physical axis (0 x, 1 y, 2 z) only, before the
 * build; they take precedence over the plan-wide ones (ps_plan_autotune tunes
 * them axis by axis). Same results up to rounding.
 *   tile    most lines per tile of the generic passes along the axis: 0 (the
 *           plan-wide tile), 1, 2, 4, 8, 16 or 32
 *   radix   their Stockham stages: -1 (the plan-wide radix), 0 radix 8 first,
 *           1 radix 4 and 2 only
 * Errors: PS_ERR_ARG (plan NULL or built, axis or a value out of range).
 */
int ps_plan_set_axis_schedule(ps_plan plan, int axis, int tile, int radix);

/* ps_plan_query -- fill *info (host only; valid before and after the build). */
int ps_plan_query(ps_plan plan, ps_plan_info* info);

/*
 * ps_kernel_build -- allocate the workspace on the current device and build
 * K^F there in FP64 (the Green's function of the plan's boundary conditions,
 * transformed along the free axes; §2, §3 "transposed kernel"), then store it
 * in the solve dtype, scaled by 1/(L1 L2 L3), as its even octant in the layout
 * the z pass reads. Idempotent. Synchronises `stream` once to report errors.
 * Errors: PS_ERR_OOM, PS_ERR_CUDA, PS_ERR_ARG (plan NULL).
 */
int ps_kernel_build(ps_plan plan, void* stream);

/*
 * ps_kernel_get -- copy the stored K^F octant to device memory `dst`
 * (dtype elements, layout [kz][ky][kx] with kx < L1/2+1, ky <= L2/2,
 * kz <= L3/2, kx fastest), scaled by 1/(L1 L2 L3) as stored.
 * Errors: PS_ERR_NOT_BUILT, PS_ERR_ARG (dst NULL), PS_ERR_CUDA.
 */
int ps_kernel_get(ps_plan plan, void* dst, void* stream);

/*
 * ps_kernel_set_real -- replace the plan's kernel by a caller's convolution
 * kernel given in real space, so that ps_solve and the other solve calls
 * compute V(r) = sum_r' K(r - r') rho(r') with it (§5: the same zero-padded
 * convolution serves other kernels, e.g. a local potential applied to many
 * wave functions; a complex field is two real solves). No h^3 factor is
 * added; the energy output is still 1/2 h^3 sum rho V.
 *   kernel  host pointer, FP64, the kernel's even octant of offsets,
 *           kernel[d1 + D1*(d2 + D2*d3)], d_j = 0 .. L_j/2 (floor), D_j = L_j/2 + 1;
 *           the kernel must be even in every offset (K(-d) = K(d)), which is
 *           what makes K^F real. Along a free axis |d_j| <= n_j - 1 couple
 *           physical points (larger offsets are never used); along a periodic
 *           axis the kernel has period n_j.
 * K^F is formed on the device in FP64 (even-cosine transforms along all three
 * axes), scaled by 1/(L1 L2 L3) and stored in the plan's dtype. The plan must
 * be built; synchronises `stream`. The previous kernel is overwritten.
 * Errors: PS_ERR_ARG (NULL), PS_ERR_NOT_BUILT, PS_ERR_CUDA.
 */
int ps_kernel_set_real(ps_plan plan, const double* kernel, void* stream);

/*
 * ps_solve -- V = K * rho (Eq. 2 via Eq. 3 on the padded grid), and
 * optionally the Hartree energy E = 1/2 h^3 sum rho V.
 *   rho           device pointer, n1*n2*n3 dtype elements (read only)
 *   V             device pointer, n1*n2*n3 dtype elements (written); must not
 *                 overlap rho
 *   ehartree_dev  device pointer to one double, or NULL to skip the energy
 * Five kernel launches on `stream`. For periodic axes the mean of rho is
 * dropped (K^F(0) = 0).
 * Errors: PS_ERR_ARG (NULL or aliasing pointers), PS_ERR_NOT_BUILT, PS_ERR_CUDA.
 */
int ps_solve(ps_plan plan, const void* rho, void* V, double* ehartree_dev, void* stream);

/*
 * ps_solve_adjoint -- rhobar = K^T vbar. K is even (K(d) = K(-d)), so the
 * operator is symmetric and this is the same convolution; it is the
 * vector-Jacobian product of V with respect to rho. Same pointers and errors
 * as ps_solve, without the energy.
 */
int ps_solve_adjoint(ps_plan plan, const void* vbar, void* rhobar, void* stream);

/*
 * ps_solve_vjp -- vector-Jacobian product of the solve's two outputs,
 *   rhobar = K^T vbar + h^3 gE V,
 * the gradient with respect to rho of <vbar, V> + gE * E, since V = K rho,
 * E = 1/2 h^3 <rho, K rho> and K is symmetric (dE/drho = h^3 V).
 *   vbar    device pointer (n1*n2*n3 dtype) or NULL (term omitted)
 *   V       device pointer to the forward result, or NULL (term omitted)
 *   gE_dev  device pointer to one double, or NULL (term omitted); V and
 *           gE_dev are both given or both NULL
 *   rhobar  device pointer (written); must not overlap vbar or V
 * Errors as ps_solve; PS_ERR_ARG if every term is omitted.
 */
int ps_solve_vjp(ps_plan plan, const void* vbar, const void* V, const double* gE_dev, void* rhobar,
                 void* stream);

/*
 * ps_solve_batched -- count independent solves, each with its own built plan
 * (shapes, boundary conditions and dtypes may differ), enqueued on one stream.
 *   plans[i], rho[i], V[i]   as in ps_solve
 *   ehartree_dev             NULL or device array of count doubles
 * Each plan may appear at most once. Errors as ps_solve, with the index of
 * the failing item in ps_last_error().
 * The launches of every problem are captured once into a CUDA graph in
 * which different problems' chains run concurrently (up to 16 at a time);
 * the instantiated graph is cached for the exact set of plans and pointers
 * and replayed by later calls with the same arguments (destroying a plan drops
 * the graphs that use it). The first call with a new argument set therefore
 * costs a capture. When the caller's stream is itself being captured, or the
 * plans live on different devices, the solves are launched in order instead.
 * Per-pass profiling events are not recorded for batched solves.
 */
int ps_solve_batched(int count, const ps_plan* plans, const void* const* rho,
                     void* const* V, double* ehartree_dev, void* stream);

/*
 * ps_solve_host -- ps_solve on host buffers: copies rho host->device, solves,
 * copies V and E device->host, and waits for `stream` before returning.
 *   rho_host, V_host   host pointers, n1*n2*n3 dtype elements (pinned memory
 *                      gives asynchronous, faster copies)
 *   ehartree_host      host pointer to one double, or NULL
 * The plan holds the device copies of rho and V (allocated on first use).
 * Errors as ps_solve, plus PS_ERR_OOM.
 */
int ps_solve_host(ps_plan plan, const void* rho_host, void* V_host, double* ehartree_host,
                  void* stream);

/*
 * ps_plan_set_profiling -- when enable != 0, every later solve on this plan
 * records a CUDA event on its stream before the first pass and after each of
 * the five passes (the per-step timers of the paper's §4 measurements, at
 * pass granularity). Recording adds no device work and no host wait.
 * Errors: PS_ERR_ARG (plan NULL).
 */
int ps_plan_set_profiling(ps_plan plan, int enable);

/*
 * ps_plan_pass_times -- waits for the events of every solve recorded since the
 * last call, writes the summed device time of each pass in milliseconds to
 * ms[0..4] (forward x, forward y, z, inverse y, inverse x) and the number of
 * recorded solves to *count, then forgets them. Host pointers.
 * Errors: PS_ERR_ARG (NULL pointer), PS_ERR_CUDA.
 */
int ps_plan_pass_times(ps_plan plan, double* ms, int* count);

/*
 * ps_plan_device_status -- synchronise `stream`, then report whether a
 * bounded device-side wait in this plan's kernels (the tensor-core z pass
 * waits on its own MMA completions, about one second at most) gave up since
 * the last call: PS_ERR_TIMEOUT (the flag is then cleared; results of the
 * solves since the last call are not valid) or PS_OK.
 * Errors: PS_ERR_ARG (plan NULL), PS_ERR_NOT_BUILT, PS_ERR_CUDA.
 */
int ps_plan_device_status(ps_plan plan, void* stream);

/*
 * ps_solve_host_stream -- ps_solve_host for `count` densities with the
 * transfers overlapped: while density i is solved, density i+1 is copied to
 * the device and the potential of density i-1 is copied back (the pipelining
 * of successive densities proposed in the paper's conclusions, §5).
 *   count >= 0              number of densities
 *   rho_host[i], V_host[i]  host pointers, n1*n2*n3 dtype elements each; use
 *                           pinned memory, or the copies cannot overlap
 *   ehartree_host           NULL or host array of count doubles
 * The plan holds two device buffer sets and three streams of its own
 * (allocated on first use). The batch starts after the work already queued on
 * `stream`, and the call waits for the whole batch before returning.
 * Errors as ps_solve_host.
 */
int ps_solve_host_stream(ps_plan plan, int count, const void* const* rho_host, void* const* V_host,
                         double* ehartree_host, void* stream);

/* ps_plan_destroy -- free the plan and its device memory. NULL is a no-op. */
int ps_plan_destroy(ps_plan plan);

/*
 * ps_hartree_energy_noalloc -- E = 1/2 h^3 sum_r rho(r) V(r) without allocating
 * any device memory. The paper has no counterpart: this entry point exists for
 * callers that must not call cudaMalloc or cudaFree on their compute path --
 * a host application whose device memory is owned by its own arena or by a
 * framework's allocator, or code that cannot risk an allocation failing, or
 * the device-wide synchronisation cudaFree implies, in the middle of a run.
 *   dtype          enum ps_dtype of rho and V
 *   npoints        number of grid points, 1 .. 536870912 (= 65536 * 8192);
 *                  larger grids return PS_ERR_UNSUPPORTED before any launch
 *   h > 0          grid spacing
 *   rho, V         device pointers, npoints elements each (read only)
 *   ehartree_dev   device pointer to one double (written)
 * The grid reduction's scratch (65536 partial sums and a counter, 512 KiB) is
 * a static device array inside the library, held by every GPU that loads the
 * library until the process exits. The first call on a device looks up the
 * array's device address (cudaGetSymbolAddress, with that device current), so
 * make that first call before any stream capture. The address is kept for the
 * life of the library: after a cudaDeviceReset of that device, unload and
 * reload the library before calling again. Every call shares the one
 * array: calls whose work may overlap on the GPU (two streams, or two host
 * threads) race and give wrong energies; serialise them. The counter is
 * cleared at the start of every call; the partial sums are overwritten.
 * Errors: PS_ERR_ARG (dtype, npoints < 1, h, NULL or misaligned pointers),
 * PS_ERR_UNSUPPORTED (npoints too large, or a device ordinal of 64 or more),
 * PS_ERR_CUDA.
 */
int ps_hartree_energy_noalloc(int dtype, long long npoints, double h, const void* rho,
                              const void* V, double* ehartree_dev, void* stream);

/* ps_strerror -- static description of a status code. */
const char* ps_strerror(int status);

/* ps_last_error -- detail of the last error on the calling thread ("" if none). */
const char* ps_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* PSOLVER_H */
