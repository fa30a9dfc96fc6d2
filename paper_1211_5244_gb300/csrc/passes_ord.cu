// The five passes for a processing order other than x, y, z (§3's axis rule:
// periodic axes first on the forward transform, free axes last), on the
// generic shared-memory Stockham kernels, with every array kept x fastest and
// each pass reaching its axis through strides (no transposes):
//
//   P1  real-to-complex transform along the first axis a0 of the order. When
//       a0 is x this is the x pass of passes.cu; along y or z the real columns
//       x = 2i and 2i + 1 form one complex line a + ib, its transform
//       Z = A + iB is separated by Hermitian symmetry,
//         A[k] = (Z[k] + conj Z[N-k]) / 2,   B[k] = (Z[k] - conj Z[N-k]) / 2i,
//       and the c = L/2 + 1 outputs k = 0 .. L/2 of both columns are kept
//                                                       rho -> A (a0 extent c)
//   P2  forward transform along a1, n inputs, L outputs  A -> B (a1 extent L)
//   P3  forward transform along a2 (n inputs), multiplication by the K^F
//       octant (Eq. 3) at the folded wavenumbers of all three axes, inverse,
//       n outputs kept; the Hartree energy as the Parseval sum with weight 1
//       on the k = 0 and k = L/2 planes of a0 and 2 elsewhere   B -> B
//   P4  inverse transform along a1, n outputs kept        B -> A
//   P5  complex-to-real inverse along a0: the half spectra of the two columns
//       are extended by Hermitian symmetry, Z = A + iB is transformed back,
//       and its real and imaginary parts are the two real columns   A -> V
//
// A tile is `tk` lines adjacent along the tile axis: x for lines along y or
// z (every access a run of consecutive elements), y for lines along x (the
// loads then run along the lines). Zero inputs of the padding are not
// loaded, unneeded outputs are not stored, as in passes.cu.
#include "common.cuh"
#include "fft_generic.cuh"
#include "reduce.cuh"

namespace ps {

namespace {

struct OrdArgs {
  // transform of length N on a tile of tk lines, shared-memory rows `rows`
  int N, tk, ldt, ltk, rows, twn, tws;
  Stages st;
  BlueArgs bl;
  // element e of line t0 + t of plane pl at pl * sp + (t0 + t) * st + e * se
  long long sp_in, st_in, se_in, sp_out, st_out, se_out;
  int ntl;       // lines along the tile axis (P1 / P5: pairs of real columns)
  int nin, nout;  // elements loaded (the rest zero) / stored per line
  int lcont;     // the line axis is the contiguous one
  unsigned mnin, mnout;  // div_magic of nin and nout
  int nreal;     // P1 / P5: real columns along x (n1)
  // P3: physical axes of the line, tile and plane indices, folding lengths
  // and K^F octant strides per physical axis, the first axis and its length
  int ax_e, ax_t, ax_p;
  int Lax[3];
  long long Ks[3];
  int a0, La0;
};

// loads nin elements of each of the tile's lines into rows [0, nin) of buf
// (rows [nin, N) zero); lines beyond ntl are zero
template <typename T>
__device__ void load_tile(cpx<T>* buf, const cpx<T>* __restrict__ src, const OrdArgs& a, int t0) {
  using C = cpx<T>;
  const int tot = a.tk * a.nin;
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    int t, e;
    if (a.lcont) {  // consecutive threads along a line
      t = div_by(w, a.mnin);
      e = w - t * a.nin;
    } else {        // consecutive threads across the lines
      t = w & (a.tk - 1);
      e = w >> a.ltk;
    }
    buf[e * a.ldt + t] = (t0 + t < a.ntl) ? src[(long long)t * a.st_in + (long long)e * a.se_in] : mk(T(0), T(0));
  }
  for (int w = threadIdx.x; w < a.tk * (a.N - a.nin); w += blockDim.x)
    buf[(a.nin + (w >> a.ltk)) * a.ldt + (w & (a.tk - 1))] = mk(T(0), T(0));
}

template <typename T>
__device__ void store_tile(cpx<T>* __restrict__ dst, const cpx<T>* buf, const OrdArgs& a, int t0) {
  const int tot = a.tk * a.nout;
  for (int w = threadIdx.x; w < tot; w += blockDim.x) {
    int t, e;
    if (a.lcont) {
      t = div_by(w, a.mnout);
      e = w - t * a.nout;
    } else {
      t = w & (a.tk - 1);
      e = w >> a.ltk;
    }
    if (t0 + t < a.ntl) dst[(long long)t * a.st_out + (long long)e * a.se_out] = buf[e * a.ldt + t];
  }
}

// P2 / P4: transform along a strided (or the contiguous) axis
template <int DIR, typename T>
__global__ void __launch_bounds__(256) ord_line(const cpx<T>* __restrict__ src, cpx<T>* __restrict__ dst,
                                                const cpx<T>* __restrict__ tw, OrdArgs a) {
  using C = cpx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + a.rows * a.ldt;
  int tstr;
  const C* ttab = load_twiddles<T>(buf1 + a.rows * a.ldt, tw, a.N, a.tws, a.bl, a.twn > 0, &tstr);
  const int t0 = blockIdx.x * a.tk;
  const long long pl = blockIdx.y;
  load_tile<T>(buf0, src + pl * a.sp_in + (long long)t0 * a.st_in, a, t0);
  __syncthreads();
  C* out = line_transform<DIR, T>(buf0, buf1, a.N, a.tk, a.ldt, a.st, ttab, tstr, a.bl);
  store_tile<T>(dst + pl * a.sp_out + (long long)t0 * a.st_out, out, a, t0);
}

// P3: forward transform, K^F multiply (and the energy), inverse, in place
template <typename T>
__global__ void __launch_bounds__(256) ord_conv(cpx<T>* __restrict__ X, const T* __restrict__ K,
                                                const cpx<T>* __restrict__ tw, OrdArgs a, double* partials,
                                                unsigned* counter, double escale, double* E) {
  using C = cpx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + a.rows * a.ldt;
  int tstr;
  const C* ttab = load_twiddles<T>(buf1 + a.rows * a.ldt, tw, a.N, a.tws, a.bl, a.twn > 0, &tstr);
  const int t0 = blockIdx.x * a.tk;
  const int pl = blockIdx.y;
  C* line = X + (long long)pl * a.sp_in + (long long)t0 * a.st_in;
  load_tile<T>(buf0, line, a, t0);
  __syncthreads();
  C* spec = line_transform<-1, T>(buf0, buf1, a.N, a.tk, a.ldt, a.st, ttab, tstr, a.bl);
  C* other = (spec == buf0) ? buf1 : buf0;
  // wavenumbers: e along the line axis, t0 + t along the tile axis, pl along
  // the plane axis, each folded into the even octant min(k, L - k)
  auto fold = [](int k, int L) { return k <= L - k ? k : L - k; };
  const long long kp = (long long)fold(pl, a.Lax[a.ax_p]) * a.Ks[a.ax_p];
  T eacc = T(0);
  for (int w = threadIdx.x; w < a.tk * a.N; w += blockDim.x) {
    const int t = w & (a.tk - 1), e = w >> a.ltk;
    const int kt = t0 + t;
    T kk = T(0);
    if (kt < a.ntl)
      kk = K[kp + (long long)fold(kt, a.Lax[a.ax_t]) * a.Ks[a.ax_t] + (long long)fold(e, a.Lax[a.ax_e]) * a.Ks[a.ax_e]];
    const int k0 = a.a0 == a.ax_t ? kt : pl;  // wavenumber along the real-to-complex axis
    const T wgt = (k0 == 0 || 2 * k0 == a.La0) ? T(1) : T(2);
    const C v = spec[e * a.ldt + t];
    eacc += wgt * kk * (v.x * v.x + v.y * v.y);
    spec[e * a.ldt + t] = cscale(v, kk);
  }
  __syncthreads();
  C* res = line_transform<1, T>(spec, other, a.N, a.tk, a.ldt, a.st, ttab, tstr, a.bl);
  store_tile<T>(line, res, a, t0);
  if (E != nullptr) energy_finish((double)eacc, partials, counter, escale, E);
}

// P1 along y or z: real columns x = 2 (t0 + t) and x + 1 as one complex line
template <typename T>
__global__ void __launch_bounds__(256) ord_r2c(const T* __restrict__ rho, cpx<T>* __restrict__ A,
                                               const cpx<T>* __restrict__ tw, OrdArgs a) {
  using C = cpx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + a.rows * a.ldt;
  int tstr;
  const C* ttab = load_twiddles<T>(buf1 + a.rows * a.ldt, tw, a.N, a.tws, a.bl, a.twn > 0, &tstr);
  const int t0 = blockIdx.x * a.tk;
  const long long pl = blockIdx.y;
  const T* src = rho + pl * a.sp_in + 2LL * t0;
  const int w2 = 2 * a.tk;  // real columns per tile
  for (int w = threadIdx.x; w < w2 * a.nin; w += blockDim.x) {
    const int xl = w & (w2 - 1), e = w >> (a.ltk + 1);
    const T v = (2 * t0 + xl < a.nreal) ? src[(long long)e * a.se_in + xl] : T(0);
    reinterpret_cast<T*>(&buf0[e * a.ldt + (xl >> 1)])[xl & 1] = v;
  }
  for (int w = threadIdx.x; w < a.tk * (a.N - a.nin); w += blockDim.x)
    buf0[(a.nin + (w >> a.ltk)) * a.ldt + (w & (a.tk - 1))] = mk(T(0), T(0));
  __syncthreads();
  C* Z = line_transform<-1, T>(buf0, buf1, a.N, a.tk, a.ldt, a.st, ttab, tstr, a.bl);
  C* dst = A + pl * a.sp_out + 2LL * t0;
  for (int w = threadIdx.x; w < a.tk * a.nout; w += blockDim.x) {
    const int t = w & (a.tk - 1), k = w >> a.ltk;
    const int x = 2 * (t0 + t);
    if (x >= a.nreal) continue;
    const C zk = Z[k * a.ldt + t];
    const C zm = Z[(k == 0 ? 0 : a.N - k) * a.ldt + t];
    C* o = dst + (long long)k * a.se_out + 2 * t;
    o[0] = mk(T(0.5) * (zk.x + zm.x), T(0.5) * (zk.y - zm.y));
    if (x + 1 < a.nreal) o[1] = mk(T(0.5) * (zk.y + zm.y), T(0.5) * (zm.x - zk.x));
  }
}

// P5 along y or z: the inverse of ord_r2c
template <typename T>
__global__ void __launch_bounds__(256) ord_c2r(const cpx<T>* __restrict__ A, T* __restrict__ V,
                                               const cpx<T>* __restrict__ tw, OrdArgs a) {
  using C = cpx<T>;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  C* buf0 = reinterpret_cast<C*>(smem_raw);
  C* buf1 = buf0 + a.rows * a.ldt;
  int tstr;
  const C* ttab = load_twiddles<T>(buf1 + a.rows * a.ldt, tw, a.N, a.tws, a.bl, a.twn > 0, &tstr);
  const int t0 = blockIdx.x * a.tk;
  const long long pl = blockIdx.y;
  const int c = a.nin;
  // the half spectra of columns 2 (t0 + t) (rows [0, c)) and 2 (t0 + t) + 1
  // (rows [c, 2c)) of buf1
  const C* src = A + pl * a.sp_in + 2LL * t0;
  const int w2 = 2 * a.tk;
  for (int w = threadIdx.x; w < w2 * c; w += blockDim.x) {
    const int xl = w & (w2 - 1), k = w >> (a.ltk + 1);
    const C v = (2 * t0 + xl < a.nreal) ? src[(long long)k * a.se_in + xl] : mk(T(0), T(0));
    buf1[(k + (xl & 1) * c) * a.ldt + (xl >> 1)] = v;
  }
  __syncthreads();
  // Z[k] = A[k] + i B[k] over the Hermitian extensions; A[0], B[0] (and
  // A[N/2], B[N/2]) of real columns are real, so their (rounding-level)
  // imaginary parts are dropped instead of leaking into the other column
  for (int w = threadIdx.x; w < a.tk * a.N; w += blockDim.x) {
    const int t = w & (a.tk - 1), k = w >> a.ltk;
    C xa = k < c ? buf1[k * a.ldt + t] : cconj(buf1[(a.N - k) * a.ldt + t]);
    C xb = k < c ? buf1[(c + k) * a.ldt + t] : cconj(buf1[(c + a.N - k) * a.ldt + t]);
    if (k == 0 || 2 * k == a.N) {
      xa.y = T(0);
      xb.y = T(0);
    }
    buf0[k * a.ldt + t] = mk(xa.x - xb.y, xa.y + xb.x);
  }
  __syncthreads();
  C* z = line_transform<1, T>(buf0, buf1, a.N, a.tk, a.ldt, a.st, ttab, tstr, a.bl);
  T* dst = V + pl * a.sp_out + 2LL * t0;
  for (int w = threadIdx.x; w < w2 * a.nout; w += blockDim.x) {
    const int xl = w & (w2 - 1), e = w >> (a.ltk + 1);
    if (2 * t0 + xl >= a.nreal) continue;
    const C v = z[e * a.ldt + (xl >> 1)];
    dst[(long long)e * a.se_out + xl] = (xl & 1) ? v.y : v.x;
  }
}

// strides (x, y, z) of an x-fastest array with extents e and x pitch ld
void strides(long long* s, const int* e, long long ld) {
  s[0] = 1;
  s[1] = ld;
  s[2] = (long long)e[1] * ld;
}

// tile and plane axes of a pass along `al`: across x for y and z lines, across
// y for x lines
void tile_axes(int al, int* at, int* ap) {
  if (al == 0) {
    *at = 1;
    *ap = 2;
  } else {
    *at = 0;
    *ap = 3 - al;
  }
}

template <typename T>
OrdArgs ord_args(const ps_plan_s* p, int pass, dim3* grid) {
  OrdArgs a{};
  const PassCfg& cf = p->cfg[pass];
  const int al = pass_axis(p, pass);
  a.N = xform_len(p, al);
  a.tk = cf.tk;
  a.ldt = cf.ldt;
  a.ltk = 0;
  while ((1 << a.ltk) < a.tk) ++a.ltk;
  a.rows = gen_rows(p, pass);
  a.twn = cf.twn;
  a.tws = p->L[al] / a.N;
  a.st = p->st[al];
  a.bl = p->blue[al];
  a.nreal = p->n[0];
  const int a0 = p->ord[0];
  a.a0 = a0;
  a.La0 = p->L[a0];
  long long sr[3], s1[3], s2[3];
  const int er[3] = {p->n[0], p->n[1], p->n[2]};
  strides(sr, er, p->n[0]);
  strides(s1, p->ext1, (long long)p->ld1);
  strides(s2, p->ext2, (long long)p->ld2);
  const long long *si = s1, *so = s1;
  const int* ext = p->ext1;
  int at, ap;
  tile_axes(al, &at, &ap);
  switch (pass) {
    case P1:  // rho -> A along a0 (y or z): pairs of real columns across x
      si = sr;
      so = s1;
      a.nin = p->n[al];
      a.nout = p->c;
      break;
    case P2:
      si = s1;
      so = s2;
      a.nin = p->n[al];
      a.nout = p->L[al];
      break;
    case P3:
      si = so = s2;
      ext = p->ext2;
      a.nin = a.nout = p->n[al];
      break;
    case P4:
      si = s2;
      so = s1;
      ext = p->ext2;
      a.nin = p->L[al];
      a.nout = p->n[al];
      break;
    default:  // P5: A -> V along a0
      si = s1;
      so = sr;
      a.nin = p->c;
      a.nout = p->n[al];
      break;
  }
  a.lcont = al == 0;
  a.se_in = si[al];
  a.st_in = si[at];
  a.sp_in = si[ap];
  a.se_out = so[al];
  a.st_out = so[at];
  a.sp_out = so[ap];
  a.ntl = (pass == P1 || pass == P5) ? (p->n[0] + 1) / 2 : ext[at];
  a.mnin = div_magic((unsigned)a.nin);
  a.mnout = div_magic((unsigned)a.nout);
  a.ax_e = al;
  a.ax_t = at;
  a.ax_p = ap;
  for (int j = 0; j < 3; ++j) a.Lax[j] = p->L[j];
  a.Ks[0] = 1;
  a.Ks[1] = (long long)p->ldk;
  a.Ks[2] = (long long)(p->H[1] + 1) * (long long)p->ldk;
  const int nplanes = (pass == P1 || pass == P5) ? p->n[ap] : ext[ap];
  *grid = dim3((unsigned)((a.ntl + a.tk - 1) / a.tk), (unsigned)nplanes);
  return a;
}

}  // namespace

int ord_conv_ctas(const ps_plan_s* p) {
  int at, ap;
  const int al = p->ord[2];
  tile_axes(al, &at, &ap);
  const int tk = p->cfg[P3].tk;
  return ((p->ext2[at] + tk - 1) / tk) * p->ext2[ap];
}

template <typename T>
cudaError_t launch_solve_ord(ps_plan_s* p, const T* rho, T* V, double* E, cudaStream_t s, cudaEvent_t* ev) {
  using C = cpx<T>;
  C* A = static_cast<C*>(p->A);
  C* B = static_cast<C*>(p->B);
  auto tw = [&](int pass) { return static_cast<const C*>(p->tw[pass_axis(p, pass)]); };
  const bool xfirst = p->ord[0] == 0;
  cudaError_t e;
  dim3 g;
  if (ev) cudaEventRecord(ev[0], s);
  if (xfirst) {
    if ((e = launch_x_pass<T>(p, P1, rho, A, s)) != cudaSuccess) return e;
  } else {
    OrdArgs a = ord_args<T>(p, P1, &g);
    ord_r2c<T><<<g, p->cfg[P1].threads, p->cfg[P1].gsmem, s>>>(rho, A, tw(P1), a);
  }
  if (ev) cudaEventRecord(ev[1], s);
  {
    OrdArgs a = ord_args<T>(p, P2, &g);
    ord_line<-1, T><<<g, p->cfg[P2].threads, p->cfg[P2].gsmem, s>>>(A, B, tw(P2), a);
  }
  if (ev) cudaEventRecord(ev[2], s);
  {
    OrdArgs a = ord_args<T>(p, P3, &g);
    ord_conv<T><<<g, p->cfg[P3].threads, p->cfg[P3].gsmem, s>>>(B, static_cast<const T*>(p->K), tw(P3), a,
                                                                p->partials, p->counter,
                                                                0.5 * p->h * p->h * p->h, E);
  }
  if (ev) cudaEventRecord(ev[3], s);
  {
    OrdArgs a = ord_args<T>(p, P4, &g);
    ord_line<1, T><<<g, p->cfg[P4].threads, p->cfg[P4].gsmem, s>>>(B, A, tw(P4), a);
  }
  if (ev) cudaEventRecord(ev[4], s);
  if (xfirst) {
    if ((e = launch_x_pass<T>(p, P5, A, V, s)) != cudaSuccess) return e;
  } else {
    OrdArgs a = ord_args<T>(p, P5, &g);
    ord_c2r<T><<<g, p->cfg[P5].threads, p->cfg[P5].gsmem, s>>>(A, V, tw(P5), a);
  }
  if (ev) cudaEventRecord(ev[5], s);
  return cudaGetLastError();
}

// the dynamic shared memory of every generic kernel of these passes
template <typename T>
cudaError_t configure_ord(const ps_plan_s*) {
  cudaError_t e;
  const int budget = 200 * 1024;
  if ((e = cudaFuncSetAttribute(ord_line<-1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(ord_line<1, T>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(ord_conv<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget)) != cudaSuccess)
    return e;
  if ((e = cudaFuncSetAttribute(ord_r2c<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget)) != cudaSuccess)
    return e;
  return cudaFuncSetAttribute(ord_c2r<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, budget);
}

template cudaError_t launch_solve_ord<float>(ps_plan_s*, const float*, float*, double*, cudaStream_t, cudaEvent_t*);
template cudaError_t launch_solve_ord<double>(ps_plan_s*, const double*, double*, double*, cudaStream_t,
                                              cudaEvent_t*);
template cudaError_t configure_ord<float>(const ps_plan_s*);
template cudaError_t configure_ord<double>(const ps_plan_s*);

}  // namespace ps
