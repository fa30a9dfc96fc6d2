// C ABI of libpsolver: argument checking, plan bookkeeping, device memory, and
// the sequence of launches of one solve. All arithmetic runs in the kernels of
// passes.cu and kernel_build.cu.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <initializer_list>
#include <new>

#include "common.cuh"
#include "fft_fast.cuh"

namespace ps {

static thread_local char g_err[512];

void set_error(const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
}

// lengths of the register four-step Bluestein convolution (FP32): powers of
// two and 3 * 2^k from 32 to 384, at least 2N (the N inputs fill the lower
// half of each column of its first step)
int blue_regs_length(int M, int N) {
  for (const int v : {32, 64, 96, 128, 192, 256, 384})
    if (v == M) return M >= 2 * N ? M : 0;
  return 0;
}

}  // namespace ps

using namespace ps;

namespace {

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  set_error("%s", buf);
  return code;
}

int cuda_fail(cudaError_t e, const char* what) {
  if (e == cudaErrorMemoryAllocation) return fail(PS_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
  return fail(PS_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

// Makes the plan's device current for the duration of a call.
struct DeviceGuard {
  int prev = -1;
  bool changed = false;
  explicit DeviceGuard(int dev) {
    if (dev < 0) return;
    if (cudaGetDevice(&prev) == cudaSuccess && prev != dev) {
      changed = cudaSetDevice(dev) == cudaSuccess;
    }
  }
  ~DeviceGuard() {
    if (changed) cudaSetDevice(prev);
  }
};

size_t round_up(size_t v, size_t m) { return (v + m - 1) / m * m; }

void free_device(ps_plan_s* p) {
  void** bufs[] = {&p->tctab, &p->A, &p->B, &p->K, &p->tw[0], &p->tw[1], &p->tw[2], &p->tw4z, &p->tw4y, &p->twx,
                   reinterpret_cast<void**>(&p->partials), reinterpret_cast<void**>(&p->counter),
                   &p->d_rho, &p->d_V, reinterpret_cast<void**>(&p->d_E), &p->d_rho2, &p->d_V2,
                   reinterpret_cast<void**>(&p->d_Eb)};
  for (void** b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  for (int j = 0; j < 3; ++j) {
    for (const void** b : {&p->blue[j].twM, &p->blue[j].chirp, &p->blue[j].Bf}) {
      if (*b) cudaFree(const_cast<void*>(*b));
      *b = nullptr;
    }
  }
  p->built = false;
  p->ws_bytes = 0;
}

size_t grid_points(const ps_plan_s* p) { return (size_t)p->n[0] * p->n[1] * p->n[2]; }

bool overlap(const void* a, const void* b, size_t bytes) {
  const char* x = static_cast<const char*>(a);
  const char* y = static_cast<const char*>(b);
  return x < y + bytes && y < x + bytes;
}

// Estimated instructions of one length-M Stockham transform in the generic
// kernels: per stage of radix R and per point, the shared-memory load and
// store, the twiddle products of the R - 1 non-trivial inputs (5 each), the
// R-point butterfly's own operations, about 15 index and loop operations per
// butterfly, and 4 for the stage's barrier. The generic kernels are bound by
// instruction issue, so fewer stages can beat a shorter length.
double stockham_cost(int M) {
  const Stages s = factorize(M);
  double c = 0.0;
  for (int i = 0; i < s.n; ++i) {
    const int R = s.R[i];
    double f;
    switch (R) {
      case 2: f = 4; break;
      case 3: f = 12; break;
      case 4: f = 16; break;
      case 5: f = 34; break;
      case 7: f = 66; break;
      case 8: f = 52; break;
      default: f = 8.0 * R * R; break;  // direct sum with table twiddles
    }
    c += (2.0 * R + 5.0 * (R - 1) + f + 15.0) / R + 4.0;
  }
  return c * M;
}

bool smooth(int m, std::initializer_list<int> primes) {
  for (int q : primes)
    while (m % q == 0) m /= q;
  return m == 1;
}

// Convolution length M >= 2N - 1 of the Bluestein form of a length-N
// transform: among the 2,3,5,7-smooth lengths up to the next power of two and
// at most max_M, the one with the least stockham_cost (PS_BLUE_M=min, or no
// candidate within max_M: the smallest 5-smooth length, which the caller
// checks against max_M).
int bluestein_length(int N, int max_M) {
  const int lo = 2 * N - 1;
  int first = lo;
  while (!smooth(first, {2, 3, 5})) ++first;
  const char* v = getenv("PS_BLUE_M");
  if (v && strcmp(v, "min") == 0) return first;
  int hi = 1;
  while (hi < lo) hi *= 2;
  int best = 0;
  double best_cost = 0.0;
  for (int M = lo; M <= hi && M <= max_M; ++M) {
    if (!smooth(M, {2, 3, 5, 7})) continue;
    const double c = stockham_cost(M);
    if (best == 0 || c < best_cost) {
      best = M;
      best_cost = c;
    }
  }
  return best ? best : first;
}

int check_solve_args(ps_plan p, const void* in, const void* out) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (!in || !out) return fail(PS_ERR_ARG, "input or output pointer is NULL");
  if (!p->built) return fail(PS_ERR_NOT_BUILT, "ps_kernel_build has not run on this plan");
  const size_t bytes = grid_points(p) * p->esz;
  if (overlap(in, out, bytes)) return fail(PS_ERR_ARG, "input and output overlap");
  if ((reinterpret_cast<uintptr_t>(in) | reinterpret_cast<uintptr_t>(out)) % p->esz)
    return fail(PS_ERR_ARG, "pointers must be aligned to the element size");
  return PS_OK;
}

int run_solve(ps_plan p, const void* rho, void* V, double* E, cudaStream_t s) {
  cudaError_t e;
  cudaEvent_t* ev = nullptr;
  if (p->profiling) {
    while (p->events.size() < p->events_used + 6) {
      cudaEvent_t x;
      if ((e = cudaEventCreate(&x)) != cudaSuccess) return cuda_fail(e, "profiling event");
      p->events.push_back(x);
    }
    ev = p->events.data() + p->events_used;
    p->events_used += 6;
  }
  if (p->dtype == PS_F32)
    e = launch_solve<float>(p, static_cast<const float*>(rho), static_cast<float*>(V), E, s, ev);
  else
    e = launch_solve<double>(p, static_cast<const double*>(rho), static_cast<double*>(V), E, s, ev);
  if (e != cudaSuccess) return cuda_fail(e, "solve launch");
  return PS_OK;
}

}  // namespace

extern "C" {

int ps_plan_create(int n1, int n2, int n3, double h, int bc_x, int bc_y, int bc_z, int dtype,
                   ps_plan* out) {
  set_error("%s", "");
  if (!out) return fail(PS_ERR_ARG, "out is NULL");
  *out = nullptr;
  const int n[3] = {n1, n2, n3};
  const int bc[3] = {bc_x, bc_y, bc_z};
  for (int j = 0; j < 3; ++j) {
    if (n[j] < 1) return fail(PS_ERR_ARG, "n%d = %d must be >= 1", j + 1, n[j]);
    if (bc[j] != PS_BC_PERIODIC && bc[j] != PS_BC_FREE) return fail(PS_ERR_ARG, "bad bc on axis %d", j);
  }
  if (!(h > 0.0) || !std::isfinite(h)) return fail(PS_ERR_ARG, "h must be finite and > 0");
  if (dtype != PS_F32 && dtype != PS_F64) return fail(PS_ERR_ARG, "bad dtype %d", dtype);
  ps_plan_s* p = new (std::nothrow) ps_plan_s();
  if (!p) return fail(PS_ERR_OOM, "host allocation failed");
  for (int j = 0; j < 3; ++j) {
    p->n[j] = n[j];
    p->bc[j] = bc[j];
    p->L[j] = bc[j] == PS_BC_FREE ? 2 * n[j] : n[j];  // §3: S_j = N_j B_j
  }
  // §3's axis rule: periodic axes first on the forward transform (no zero
  // padding to carry through the first steps), free axes last; in x, y, z
  // order among axes of the same kind
  {
    int k = 0;
    for (int pass = 0; pass < 2; ++pass)
      for (int j = 0; j < 3; ++j)
        if ((bc[j] == PS_BC_PERIODIC) == (pass == 0)) p->ord[k++] = j;
  }
  p->h = h;
  p->dtype = dtype;
  p->math = PS_MATH_CUDACORE;
  p->esz = dtype == PS_F32 ? 4 : 8;
  p->device = -1;
  for (int j = 0; j < 3; ++j) p->radix_ax[j] = -1;
  const int rc = ps_plan_set_lengths(p, 0, 0, 0);  // validates lengths, derives c, H, stages
  if (rc != PS_OK) {
    delete p;
    return rc;
  }
  *out = p;
  return PS_OK;
}

int ps_plan_set_lengths(ps_plan p, int L1, int L2, int L3) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (p->built) return fail(PS_ERR_ARG, "lengths must be set before ps_kernel_build");
  const int Lr[3] = {L1, L2, L3};
  int L[3];
  for (int j = 0; j < 3; ++j) {
    L[j] = Lr[j] > 0 ? Lr[j] : p->L[j];
    if (p->bc[j] == PS_BC_PERIODIC && L[j] != p->n[j])
      return fail(PS_ERR_ARG, "periodic axis %d must keep L = n", j);
    if (p->bc[j] == PS_BC_FREE && L[j] < 2 * p->n[j] - 1)
      return fail(PS_ERR_ARG, "free axis %d needs L >= 2n - 1", j);
    if (L[j] > kMaxLen) return fail(PS_ERR_UNSUPPORTED, "length %d exceeds %d", L[j], kMaxLen);
  }
  for (int j = 0; j < 3; ++j) {
    p->L[j] = L[j];
    p->H[j] = L[j] / 2;
  }
  const int a0 = p->ord[0], a1 = p->ord[1];
  p->c = p->L[a0] / 2 + 1;  // outputs kept by the real-to-complex transform (§3)
  for (int j = 0; j < 3; ++j) p->st[j] = factorize(xform_len(p, j));
  // Bluestein for transform lengths with a prime factor >= 11 (a direct sum
  // over that factor would cost N * p per line), if M fits the tile
  for (int j = 0; j < 3; ++j) {
    const int N = xform_len(p, j);
    int big = 1;
    for (int r = 0; r < p->st[j].n; ++r) big = p->st[j].R[r] > big ? p->st[j].R[r] : big;
    p->blue[j] = BlueArgs{};
    if (big >= 11) {
      // two buffers of M rows for a one-line tile (ldt = 2) must fit the
      // 200 KiB shared-memory budget of the generic kernels
      const size_t csz = 2 * (p->dtype == PS_F32 ? 4 : 8);
      const int max_M = (int)std::min<size_t>(kMaxLen, 200 * 1024 / (2 * 2 * csz));
      int M = bluestein_length(N, max_M);
      // FP32: the shortest length >= 2N where the register four-step form
      // exists (a power of two or 3 * 2^k up to 384: up to twice the points of
      // the smooth length, at a fraction of the cost per point of the
      // Stockham stages); PS_BLUE_REGS=0 (or PS_BLUE_M=min) keeps the smooth length
      const char* rv = getenv("PS_BLUE_REGS");
      const char* mv = getenv("PS_BLUE_M");
      const bool regs = !(rv && atoi(rv) == 0) && !(mv && strcmp(mv, "min") == 0);
      int m2 = 0;
      for (const int v : {32, 64, 96, 128, 192, 256, 384})
        if (m2 == 0 && v >= 2 * N) m2 = v;
      if (p->dtype == PS_F32 && regs && m2 && blue_regs_length(m2, N)) M = m2;
      if (M <= max_M) {
        p->blue[j].M = M;
        p->blue[j].st = factorize(M);
      }
    }
  }
  // the arrays after the first forward pass (extent c along the first axis)
  // and after the second (the second axis at its padded length), x fastest
  // with a pitch of 128 bytes
  for (int j = 0; j < 3; ++j) p->ext1[j] = p->n[j];
  p->ext1[a0] = p->c;
  for (int j = 0; j < 3; ++j) p->ext2[j] = p->ext1[j];
  p->ext2[a1] = p->L[a1];
  const size_t pitch = p->dtype == PS_F32 ? 16 : 8;
  p->ld1 = round_up((size_t)p->ext1[0], pitch);
  p->ld2 = round_up((size_t)p->ext2[0], pitch);
  p->ldc = p->ld1;  // x first: both arrays keep the c columns of the x spectrum
  p->ldk = round_up((size_t)p->H[0] + 1, 16);  // the K^F octant: kx <= L1/2
  return PS_OK;
}

int ps_plan_set_order(ps_plan p, int a0, int a1, int a2) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (p->built) return fail(PS_ERR_ARG, "the order must be set before ps_kernel_build");
  const int a[3] = {a0, a1, a2};
  int seen = 0;
  for (int k = 0; k < 3; ++k) {
    if (a[k] < 0 || a[k] > 2 || (seen & (1 << a[k]))) return fail(PS_ERR_ARG, "(%d, %d, %d) is not a permutation of the axes 0, 1, 2", a0, a1, a2);
    seen |= 1 << a[k];
  }
  int old[3];
  for (int k = 0; k < 3; ++k) {
    old[k] = p->ord[k];
    p->ord[k] = a[k];
  }
  const int rc = ps_plan_set_lengths(p, 0, 0, 0);  // c, stages and array shapes of the new order
  if (rc != PS_OK)
    for (int k = 0; k < 3; ++k) p->ord[k] = old[k];
  return rc;
}

int ps_plan_set_math(ps_plan p, int math_mode) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (p->built) return fail(PS_ERR_ARG, "math mode must be set before ps_kernel_build");
  if (math_mode != PS_MATH_CUDACORE && math_mode != PS_MATH_TF32X3 && math_mode != PS_MATH_BF16X3)
    return fail(PS_ERR_ARG, "unknown math mode %d", math_mode);
  if (math_mode == PS_MATH_BF16X3)
    return fail(PS_ERR_UNSUPPORTED,
                "split-BF16 tensor-core stages are not built (three-term splits and six partial products "
                "per stage cost more than the TF32x3 form, itself slower than the CUDA cores here)");
  if (math_mode == PS_MATH_TF32X3 && p->dtype != PS_F32)
    return fail(PS_ERR_UNSUPPORTED, "tensor-core math needs an FP32 plan");
  p->math = math_mode;
  return PS_OK;
}

int ps_plan_set_schedule(ps_plan p, int tile, int radix, int ztk, int ykind, int xy, int chunks) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (p->built) return fail(PS_ERR_ARG, "the schedule must be set before ps_kernel_build");
  if (tile < 0 || tile > 32 || (tile & (tile - 1)) != 0)
    return fail(PS_ERR_ARG, "tile = %d: 0 or a power of two up to 32", tile);
  if (radix != 0 && radix != 1) return fail(PS_ERR_ARG, "radix = %d: 0 or 1", radix);
  if (ztk != 0 && ztk != 8 && ztk != 16) return fail(PS_ERR_ARG, "ztk = %d: 0, 8 or 16", ztk);
  if (ykind < 0 || ykind > 2) return fail(PS_ERR_ARG, "ykind = %d: 0, 1 or 2", ykind);
  if (xy != 0 && xy != 1) return fail(PS_ERR_ARG, "xy = %d: 0 or 1", xy);
  if (chunks < 0 || chunks > 64) return fail(PS_ERR_ARG, "chunks = %d: 0 .. 64", chunks);
  p->gen_tk_max = tile;
  p->radix_pref = radix;
  p->z_tk = ztk;
  p->y_kind = ykind;
  p->xy_sched = xy;
  p->chunk_req = chunks;
  return PS_OK;
}

int ps_plan_set_axis_schedule(ps_plan p, int axis, int tile, int radix) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (p->built) return fail(PS_ERR_ARG, "the schedule must be set before ps_kernel_build");
  if (axis < 0 || axis > 2) return fail(PS_ERR_ARG, "axis = %d: 0, 1 or 2", axis);
  if (tile < 0 || tile > 32 || (tile & (tile - 1)) != 0)
    return fail(PS_ERR_ARG, "tile = %d: 0 or a power of two up to 32", tile);
  if (radix < -1 || radix > 1) return fail(PS_ERR_ARG, "radix = %d: -1, 0 or 1", radix);
  p->tile_ax[axis] = tile;
  p->radix_ax[axis] = radix;
  return PS_OK;
}

int ps_plan_query(ps_plan p, ps_plan_info* info) {
  if (!p || !info) return fail(PS_ERR_ARG, "plan or info is NULL");
  memset(info, 0, sizeof *info);
  for (int j = 0; j < 3; ++j) {
    info->n[j] = p->n[j];
    info->bc[j] = p->bc[j];
    info->L[j] = p->L[j];
  }
  info->c = p->c;
  info->dtype = p->dtype;
  info->math = p->math;
  const int a0 = p->ord[0], a1 = p->ord[1], a2 = p->ord[2];
  const long long n1 = p->n[0], n2 = p->n[1], n3 = p->n[2];
  const long long L1 = p->L[0], L2 = p->L[1], L3 = p->L[2], c = p->c;
  // in processing order: S = padded lengths, N = physical counts
  const long long Sa = p->L[a0], Sb = p->L[a1], Sc = p->L[a2], Nb = p->n[a1], Nc = p->n[a2];
  info->lines[0] = Nb * Nc;  info->line_len[0] = Sa;
  info->lines[1] = c * Nc;   info->line_len[1] = Sb;
  info->lines[2] = c * Sb;   info->line_len[2] = Sc;
  info->lines[3] = c * Nc;   info->line_len[3] = Sb;
  info->lines[4] = Nb * Nc;  info->line_len[4] = Sa;
  for (int k = 0; k < 3; ++k) info->order[k] = p->ord[k];
  double pts = 0.0;
  for (int k = 0; k < 5; ++k) pts += (double)info->lines[k] * (double)info->line_len[k];
  pts += (double)info->lines[2] * (double)info->line_len[2];  // last axis: forward and inverse
  info->fft_points = pts;
  // §3 count of one forward 3D transform: rows x length per step, complex rows
  info->paper_points = (double)(Nb * Nc * Sa) + (double)(Sa * Nc * Sb) + (double)(Sa * Sb * Sc);
  info->paper_full_points = 3.0 * (double)(L1 * L2 * L3);
  const double b = (double)p->esz;
  const bool xyf = p->built && p->xyfuse;
  // the fused x/y kernels never write or read A: the intermediate pairs of
  // the x-transformed array drop out
  info->alg_bytes = 2.0 * (double)(n1 * n2 * n3) * b + 8.0 * b * (double)(c * Nc * ((xyf ? 0 : Nb) + Sb)) +
                    b * (double)(p->H[0] + 1) * (double)(p->H[1] + 1) * (double)(p->H[2] + 1);
  info->workspace_bytes = p->ws_bytes;
  info->launches = p->built ? (xyf ? 3 : 5) : 0;
  info->tensor_passes = (p->built && p->tctab) ? (1 << 2) : 0;
  info->fused = xyf ? ((1 << 1) | (1 << 4)) : 0;
  info->schedule[0] = p->gen_tk_max;
  info->schedule[1] = p->radix_pref;
  info->schedule[2] = p->z_tk;
  info->schedule[3] = p->y_kind;
  info->schedule[4] = p->xy_sched;
  info->schedule[5] = p->chunk_req;
  info->chunks = p->built ? p->chunks : 0;
  for (int j = 0; j < 3; ++j) {
    info->axis_schedule[j][0] = p->tile_ax[j];
    info->axis_schedule[j][1] = p->radix_ax[j];
  }
  for (int k = 0; k < 5; ++k)
    info->blocks[k] = (p->built && p->cfg[k].fast) ? (int)(p->cfg[k].grid.x * p->cfg[k].grid.y) : 0;
  if (xyf) {
    info->blocks[0] = info->blocks[1] = (int)p->xyf[0].grid.x;
    info->blocks[3] = info->blocks[4] = (int)p->xyf[1].grid.x;
  }
  return PS_OK;
}

int ps_kernel_build(ps_plan p, void* stream) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (p->built) return PS_OK;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(e, "cudaGetDevice");
  p->device = dev;
  for (int j = 0; j < 3; ++j) {  // the schedule's radix split of the generic stages, per axis
    const int r = axis_radix(p, j);
    if (!r) continue;
    p->st[j] = factorize(xform_len(p, j), r);
    if (p->blue[j].M) p->blue[j].st = factorize(p->blue[j].M, r);
  }
  e = p->dtype == PS_F32 ? configure_passes<float>(p) : configure_passes<double>(p);
  if (e != cudaSuccess) return cuda_fail(e, "configure passes");
  const size_t csz = 2 * p->esz;
  // A: the array after the first forward pass, B: after the second
  const size_t szA = p->ld1 * (size_t)p->ext1[1] * p->ext1[2] * csz;
  const size_t szB = p->ld2 * (size_t)p->ext2[1] * p->ext2[2] * csz;
  const size_t szK = p->ldk * (p->H[1] + 1) * (p->H[2] + 1) * p->esz;
  struct { void** ptr; size_t bytes; const char* what; } allocs[] = {
      {&p->A, szA, "workspace A"},
      {&p->B, szB, "workspace B"},
      {&p->K, szK, "K^F"},
      {&p->tw[0], (size_t)p->L[0] * csz, "twiddles x"},
      {&p->tw[1], (size_t)p->L[1] * csz, "twiddles y"},
      {&p->tw[2], (size_t)p->L[2] * csz, "twiddles z"},
      {reinterpret_cast<void**>(&p->partials), (size_t)p->npart * sizeof(double), "energy partials"},
      {reinterpret_cast<void**>(&p->counter), 2 * sizeof(unsigned), "energy counter and status"},
      {&p->tctab, p->tctab_floats * sizeof(float), "tensor-core z tables"},
      {&p->tw4z, p->zsoa_T ? (size_t)p->zsoa_T * p->zsoa_P * 16 : 0, "paired z twiddles"},
      {&p->twx, p->xP ? (size_t)p->xP * p->xP * 8 : 0, "x twiddle matrix"},
      {&p->tw4y, p->ysoa ? (size_t)16 * 16 * 16 : 0, "paired y twiddles"},
  };
  size_t total = 0;
  for (auto& a : allocs) {
    if (a.bytes == 0) continue;
    e = cudaMalloc(a.ptr, a.bytes);
    if (e != cudaSuccess) {
      free_device(p);
      return cuda_fail(e, a.what);
    }
    total += a.bytes;
  }
  for (int j = 0; j < 3 && e == cudaSuccess; ++j) {
    if (!p->blue[j].M) continue;
    const int N = xform_len(p, j);
    void *twM = nullptr, *ch = nullptr, *bf = nullptr;
    e = cudaMalloc(&twM, (size_t)p->blue[j].M * csz);
    if (e == cudaSuccess) e = cudaMalloc(&ch, (size_t)N * csz);
    if (e == cudaSuccess) e = cudaMalloc(&bf, (size_t)p->blue[j].M * csz);
    p->blue[j].twM = twM;
    p->blue[j].chirp = ch;
    p->blue[j].Bf = bf;
    total += (size_t)(2 * p->blue[j].M + N) * csz;
  }
  if (e != cudaSuccess) {
    free_device(p);
    return cuda_fail(e, "Bluestein tables");
  }
  p->ws_bytes = total;
  e = cudaMemsetAsync(p->counter, 0, 2 * sizeof(unsigned), s);
  // the row padding of the work arrays (kx from c to the pitch) is read by the
  // tile copies of the y and z passes but never written: zero it once, so that
  // it holds finite values (the z pass multiplies it by K^F = 0 in the energy)
  if (e == cudaSuccess) e = cudaMemsetAsync(p->A, 0, szA, s);
  if (e == cudaSuccess) e = cudaMemsetAsync(p->B, 0, szB, s);
  std::vector<float> tctab_host;
  if (e == cudaSuccess && p->tctab) {
    tctab_host.resize(p->tctab_floats);
    ztc_fill_table(p->n[2] * 2 == p->L[2], tctab_host.data());
    e = cudaMemcpyAsync(p->tctab, tctab_host.data(), p->tctab_floats * sizeof(float), cudaMemcpyHostToDevice, s);
  }
  if (e == cudaSuccess) e = build_twiddles(p, s);
  if (e == cudaSuccess) e = build_kernel(p, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_device(p);
    return cuda_fail(e, "kernel build");
  }
  p->built = true;
  return PS_OK;
}

int ps_kernel_set_real(ps_plan p, const double* kernel, void* stream) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (!p->built) return fail(PS_ERR_NOT_BUILT, "ps_kernel_build has not run on this plan");
  if (!kernel) return fail(PS_ERR_ARG, "kernel is NULL");
  DeviceGuard g(p->device);
  cudaError_t e = build_kernel_from_real(p, kernel, static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "kernel from real space");
  return PS_OK;
}

int ps_kernel_get(ps_plan p, void* dst, void* stream) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (!p->built) return fail(PS_ERR_NOT_BUILT, "ps_kernel_build has not run on this plan");
  if (!dst) return fail(PS_ERR_ARG, "dst is NULL");
  DeviceGuard g(p->device);
  const size_t D0 = (size_t)p->H[0] + 1;  // kx <= L1/2
  cudaError_t e = cudaMemcpy2DAsync(dst, D0 * p->esz, p->K, p->ldk * p->esz, D0 * p->esz,
                                    (size_t)(p->H[1] + 1) * (p->H[2] + 1), cudaMemcpyDeviceToDevice,
                                    static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(e, "copy K^F");
  return PS_OK;
}

int ps_solve(ps_plan p, const void* rho, void* V, double* ehartree_dev, void* stream) {
  int rc = check_solve_args(p, rho, V);
  if (rc != PS_OK) return rc;
  DeviceGuard g(p->device);
  return run_solve(p, rho, V, ehartree_dev, static_cast<cudaStream_t>(stream));
}

int ps_solve_adjoint(ps_plan p, const void* vbar, void* rhobar, void* stream) {
  int rc = check_solve_args(p, vbar, rhobar);
  if (rc != PS_OK) return rc;
  DeviceGuard g(p->device);
  return run_solve(p, vbar, rhobar, nullptr, static_cast<cudaStream_t>(stream));
}

int ps_solve_vjp(ps_plan p, const void* vbar, const void* V, const double* gE_dev, void* rhobar,
                 void* stream) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (!rhobar) return fail(PS_ERR_ARG, "rhobar is NULL");
  if (!vbar && !V) return fail(PS_ERR_ARG, "every term of the VJP is omitted");
  if ((V == nullptr) != (gE_dev == nullptr)) return fail(PS_ERR_ARG, "V and gE_dev must be given together");
  if (!p->built) return fail(PS_ERR_NOT_BUILT, "ps_kernel_build has not run on this plan");
  const size_t bytes = grid_points(p) * p->esz;
  if ((vbar && overlap(vbar, rhobar, bytes)) || (V && overlap(V, rhobar, bytes)))
    return fail(PS_ERR_ARG, "rhobar overlaps an input");
  if ((reinterpret_cast<uintptr_t>(vbar) | reinterpret_cast<uintptr_t>(V) |
       reinterpret_cast<uintptr_t>(rhobar)) % p->esz)
    return fail(PS_ERR_ARG, "pointers must be aligned to the element size");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if (vbar) {
    int rc = run_solve(p, vbar, rhobar, nullptr, s);
    if (rc != PS_OK) return rc;
  }
  if (V) {
    cudaError_t e = p->dtype == PS_F32
        ? launch_vjp_axpy<float>(p, static_cast<float*>(rhobar), static_cast<const float*>(V), gE_dev,
                                 vbar != nullptr, s)
        : launch_vjp_axpy<double>(p, static_cast<double*>(rhobar), static_cast<const double*>(V), gE_dev,
                                  vbar != nullptr, s);
    if (e != cudaSuccess) return cuda_fail(e, "vjp energy term");
  }
  return PS_OK;
}

int ps_solve_batched(int count, const ps_plan* plans, const void* const* rho, void* const* V,
                     double* ehartree_dev, void* stream) {
  if (count < 0) return fail(PS_ERR_ARG, "count < 0");
  if (count == 0) return PS_OK;
  if (!plans || !rho || !V) return fail(PS_ERR_ARG, "NULL array argument");
  for (int i = 0; i < count; ++i) {
    int rc = check_solve_args(plans[i], rho[i], V[i]);
    if (rc != PS_OK) return fail(rc, "item %d: %s", i, ps_last_error());
    for (int j = 0; j < i; ++j)
      if (plans[j] == plans[i]) return fail(PS_ERR_ARG, "item %d: plan repeated (item %d)", i, j);
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  bool one_device = true;
  for (int i = 1; i < count; ++i) one_device &= plans[i]->device == plans[0]->device;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (count >= 2 && one_device && cudaStreamIsCapturing(s, &cap) == cudaSuccess &&
      cap == cudaStreamCaptureStatusNone) {
    DeviceGuard g(plans[0]->device);
    cudaError_t e = batch_solve_graph(count, plans, rho, V, ehartree_dev, plans[0]->device, s);
    if (e != cudaSuccess) return cuda_fail(e, "batched graph");
    return PS_OK;
  }
  // one problem, several devices, or a stream that is itself being captured:
  // plain launches in order on the caller's stream
  for (int i = 0; i < count; ++i) {
    DeviceGuard g(plans[i]->device);
    int rc = run_solve(plans[i], rho[i], V[i], ehartree_dev ? ehartree_dev + i : nullptr, s);
    if (rc != PS_OK) return fail(rc, "item %d: %s", i, ps_last_error());
  }
  return PS_OK;
}

int ps_solve_host(ps_plan p, const void* rho_host, void* V_host, double* ehartree_host, void* stream) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (!rho_host || !V_host) return fail(PS_ERR_ARG, "host pointer is NULL");
  if (!p->built) return fail(PS_ERR_NOT_BUILT, "ps_kernel_build has not run on this plan");
  DeviceGuard g(p->device);
  const size_t bytes = grid_points(p) * p->esz;
  cudaError_t e;
  if (!p->d_rho) {
    if ((e = cudaMalloc(&p->d_rho, bytes)) != cudaSuccess) return cuda_fail(e, "staging rho");
    if ((e = cudaMalloc(&p->d_V, bytes)) != cudaSuccess) return cuda_fail(e, "staging V");
    if ((e = cudaMalloc(&p->d_E, 2 * sizeof(double))) != cudaSuccess) return cuda_fail(e, "staging E");
  }
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((e = cudaMemcpyAsync(p->d_rho, rho_host, bytes, cudaMemcpyHostToDevice, s)) != cudaSuccess)
    return cuda_fail(e, "copy rho to device");
  int rc = run_solve(p, p->d_rho, p->d_V, ehartree_host ? p->d_E : nullptr, s);
  if (rc != PS_OK) return rc;
  if ((e = cudaMemcpyAsync(V_host, p->d_V, bytes, cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "copy V to host");
  if (ehartree_host &&
      (e = cudaMemcpyAsync(ehartree_host, p->d_E, sizeof(double), cudaMemcpyDeviceToHost, s)) != cudaSuccess)
    return cuda_fail(e, "copy E to host");
  if ((e = cudaStreamSynchronize(s)) != cudaSuccess) return cuda_fail(e, "solve");
  return PS_OK;
}

int ps_plan_set_profiling(ps_plan p, int enable) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  p->profiling = enable != 0;
  return PS_OK;
}

int ps_plan_device_status(ps_plan p, void* stream) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (!p->built) return fail(PS_ERR_NOT_BUILT, "ps_kernel_build has not run on this plan");
  DeviceGuard g(p->device);
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  unsigned flag = 0;
  cudaError_t e = cudaMemcpyAsync(&flag, p->counter + 1, sizeof(unsigned), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess && flag) e = cudaMemsetAsync(p->counter + 1, 0, sizeof(unsigned), s);
  if (e == cudaSuccess && flag) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return cuda_fail(e, "device status");
  if (flag) return fail(PS_ERR_TIMEOUT, "a bounded device wait gave up");
  return PS_OK;
}

int ps_plan_pass_times(ps_plan p, double* ms, int* count) {
  if (!p || !ms || !count) return fail(PS_ERR_ARG, "NULL argument");
  for (int k = 0; k < 5; ++k) ms[k] = 0.0;
  *count = (int)(p->events_used / 6);
  if (p->events_used == 0) return PS_OK;
  DeviceGuard g(p->device);
  cudaError_t e = cudaEventSynchronize(p->events[p->events_used - 1]);
  if (e != cudaSuccess) return cuda_fail(e, "profiling wait");
  for (size_t i = 0; i + 6 <= p->events_used; i += 6) {
    for (int k = 0; k < 5; ++k) {
      float t = 0.f;
      e = cudaEventElapsedTime(&t, p->events[i + k], p->events[i + k + 1]);
      if (e != cudaSuccess) return cuda_fail(e, "profiling elapsed time");
      ms[k] += t;
    }
  }
  p->events_used = 0;
  return PS_OK;
}

int ps_solve_host_stream(ps_plan p, int count, const void* const* rho_host, void* const* V_host,
                         double* ehartree_host, void* stream) {
  if (!p) return fail(PS_ERR_ARG, "plan is NULL");
  if (count < 0) return fail(PS_ERR_ARG, "count < 0");
  if (count == 0) return PS_OK;
  if (!rho_host || !V_host) return fail(PS_ERR_ARG, "NULL array argument");
  for (int i = 0; i < count; ++i)
    if (!rho_host[i] || !V_host[i]) return fail(PS_ERR_ARG, "item %d: host pointer is NULL", i);
  if (!p->built) return fail(PS_ERR_NOT_BUILT, "ps_kernel_build has not run on this plan");
  DeviceGuard g(p->device);
  const size_t bytes = grid_points(p) * p->esz;
  cudaError_t e;
  if (!p->d_rho) {
    if ((e = cudaMalloc(&p->d_rho, bytes)) != cudaSuccess) return cuda_fail(e, "staging rho");
    if ((e = cudaMalloc(&p->d_V, bytes)) != cudaSuccess) return cuda_fail(e, "staging V");
    if ((e = cudaMalloc(&p->d_E, 2 * sizeof(double))) != cudaSuccess) return cuda_fail(e, "staging E");
  }
  if (!p->d_rho2) {
    if ((e = cudaMalloc(&p->d_rho2, bytes)) != cudaSuccess) return cuda_fail(e, "staging rho");
    if ((e = cudaMalloc(&p->d_V2, bytes)) != cudaSuccess) return cuda_fail(e, "staging V");
  }
  if (ehartree_host && p->d_Eb_cap < count) {
    // the energies stay on the device until the batch ends: a copy of 8 bytes
    // to pageable host memory would block the host and serialise the pipeline
    if (p->d_Eb) cudaFree(p->d_Eb);
    p->d_Eb = nullptr;
    p->d_Eb_cap = 0;
    if ((e = cudaMalloc(&p->d_Eb, (size_t)count * sizeof(double))) != cudaSuccess) return cuda_fail(e, "energies");
    p->d_Eb_cap = count;
  }
  if (!p->hs[0]) {
    for (int k = 0; k < 3; ++k)
      if ((e = cudaStreamCreateWithFlags(&p->hs[k], cudaStreamNonBlocking)) != cudaSuccess)
        return cuda_fail(e, "transfer streams");
    for (int k = 0; k < 7; ++k)
      if ((e = cudaEventCreateWithFlags(&p->hev[k], cudaEventDisableTiming)) != cudaSuccess)
        return cuda_fail(e, "transfer events");
  }
  cudaStream_t up = p->hs[0], comp = p->hs[1], down = p->hs[2];
  cudaEvent_t* ev_in = p->hev;        // [2] upload of slot done
  cudaEvent_t* ev_comp = p->hev + 2;  // [2] solve of slot done (its rho buffer is free)
  cudaEvent_t* ev_out = p->hev + 4;   // [2] download of slot done (its V buffer is free)
  cudaEvent_t start = p->hev[6];
  void* drho[2] = {p->d_rho, p->d_rho2};
  void* dV[2] = {p->d_V, p->d_V2};
  cudaStream_t s = static_cast<cudaStream_t>(stream);
#define PS_TRY(call, what)                          \
  do {                                              \
    if ((e = (call)) != cudaSuccess) return cuda_fail(e, what); \
  } while (0)
  PS_TRY(cudaEventRecord(start, s), "ordering");
  for (int k = 0; k < 3; ++k) PS_TRY(cudaStreamWaitEvent(p->hs[k], start, 0), "ordering");
  for (int i = 0; i < count; ++i) {
    const int b = i & 1;
    if (i >= 2) PS_TRY(cudaStreamWaitEvent(up, ev_comp[b], 0), "ordering");
    PS_TRY(cudaMemcpyAsync(drho[b], rho_host[i], bytes, cudaMemcpyHostToDevice, up), "copy rho to device");
    PS_TRY(cudaEventRecord(ev_in[b], up), "ordering");
    PS_TRY(cudaStreamWaitEvent(comp, ev_in[b], 0), "ordering");
    if (i >= 2) PS_TRY(cudaStreamWaitEvent(comp, ev_out[b], 0), "ordering");
    int rc = run_solve(p, drho[b], dV[b], ehartree_host ? p->d_Eb + i : nullptr, comp);
    if (rc != PS_OK) return fail(rc, "item %d: %s", i, ps_last_error());
    PS_TRY(cudaEventRecord(ev_comp[b], comp), "ordering");
    PS_TRY(cudaStreamWaitEvent(down, ev_comp[b], 0), "ordering");
    PS_TRY(cudaMemcpyAsync(V_host[i], dV[b], bytes, cudaMemcpyDeviceToHost, down), "copy V to host");
    PS_TRY(cudaEventRecord(ev_out[b], down), "ordering");
  }
  if (ehartree_host) {
    PS_TRY(cudaStreamWaitEvent(down, ev_comp[(count - 1) & 1], 0), "ordering");
    PS_TRY(cudaMemcpyAsync(ehartree_host, p->d_Eb, (size_t)count * sizeof(double), cudaMemcpyDeviceToHost, down),
           "copy energies to host");
  }
  PS_TRY(cudaStreamSynchronize(down), "transfer pipeline");
  PS_TRY(cudaStreamSynchronize(comp), "transfer pipeline");
#undef PS_TRY
  return PS_OK;
}

int ps_plan_destroy(ps_plan p) {
  if (!p) return PS_OK;
  batch_forget_plan(p);
  {
    DeviceGuard g(p->device);
    for (int k = 0; k < 3; ++k)
      if (p->hs[k]) cudaStreamDestroy(p->hs[k]);
    for (int k = 0; k < 7; ++k)
      if (p->hev[k]) cudaEventDestroy(p->hev[k]);
    for (cudaEvent_t e : p->events) cudaEventDestroy(e);
    p->events.clear();
    free_device(p);
  }
  delete p;
  return PS_OK;
}

const char* ps_strerror(int status) {
  switch (status) {
    case PS_OK: return "success";
    case PS_ERR_ARG: return "invalid argument";
    case PS_ERR_UNSUPPORTED: return "unsupported configuration";
    case PS_ERR_NOT_BUILT: return "kernel not built (call ps_kernel_build)";
    case PS_ERR_CUDA: return "CUDA error";
    case PS_ERR_OOM: return "out of device memory";
    case PS_ERR_TIMEOUT: return "device wait timed out";
    default: return "unknown status";
  }
}

const char* ps_last_error(void) { return ps::g_err; }

}  // extern "C"
