// K^F construction, in FP64 on the device (once per plan; not on the timed path).
//
// The convolution kernel (Eq. 2) for each boundary-condition class, written
// spectrally along the periodic axes (wavenumber k) and in real space along
// the free axes (offset d, in grid units), with the grid weights included:
//
//   0 periodic axes (free, §2):   K(d) = -h^2 / (4 pi |d|),    K(0) = -h^2 C3 / (4 pi)
//   1 periodic axis (wire):       K    = h^2 G_k(r),  r = h |d|
//        G_0(r) = ln(r) / (2 pi),  G_k(r) = -K0(k r) / (2 pi),
//        r = 0: the average of G_k over the h x h cell
//   2 periodic axes (surface):    K    = h G_k(z),   z = h |d|
//        G_0(z) = z / 2,  G_k(z) = -exp(-k z) / (2 k)
//   3 periodic axes:              K^F  = -1 / k^2,  K^F(0) = 0
//
// The paper (§2) only cites the mixed-BC Green's functions; these are the
// Green's functions of the Laplacian restricted to the free axes, consistent
// with Eq. 1 as printed (no -4 pi). K is even in every axis, so K^F is real
// and even: it is sampled on the octant 0..L_j/2 of every axis and the DFT
// along a free axis of length L is the even cosine sum
//   K^F(k) = sum_{i=0}^{L/2} w_i M(i) cos(2 pi k i / L),
//   w_0 = 1, w_{L/2} = 1 for even L, w_i = 2 otherwise.
// The result is scaled by 1/(L1 L2 L3) (the inverse-transform normalisation)
// and stored in the solve dtype in the [kz][ky][kx] layout of the z pass (§3:
// the transposed kernel, built once and reused by every solve).
#include <cmath>

#include "common.cuh"

namespace ps {

// cell average of 1/|u| over the unit cube:  3 ln(2 + sqrt 3) - pi / 2
__device__ __constant__ double kC3 = 2.3800773639795529;
// cell average of ln|u| over the unit square: -3/2 + pi/4 - ln(2)/2
__device__ __constant__ double kC2 = -1.0611754268825244;
__device__ __constant__ double kEulerGamma = 0.57721566490153286061;
__device__ __constant__ double kPi = 3.14159265358979323846;

// ---------------------------------------------------------------- K0

// K0(x) = int_0^inf exp(-x cosh t) dt = e^{-x} int_0^inf exp(-2 x sinh^2(t/2)) dt,
// by the trapezoidal rule, which converges exponentially fast for this
// integrand (analytic in the strip |Im t| < pi/2 and decaying double
// exponentially; Trefethen & Weideman, "The exponentially convergent
// trapezoidal rule", SIAM Review 56 (2014)). The step keeps both error terms
// below 1e-16: tau <= 0.2 for the strip, tau <= 0.6 / sqrt(x) for the width
// ~1/sqrt(x) of the peak at t = 0 when x is large.
__device__ double bessel_k0(double x) {
  const double tau = fmin(0.2, 0.6 / sqrt(x));
  double sum = 0.5;
  for (int j = 1; j < 20000; ++j) {
    const double sh = sinh(0.5 * tau * j);
    const double term = exp(-2.0 * x * sh * sh);
    sum += term;
    if (term < 1e-18 * sum) break;
  }
  return tau * exp(-x) * sum;
}

// F(R) = int_0^R [K0(k r) + ln r] r dr, from the power series of K0
// (K0(x) = -(ln(x/2) + gamma) I0(x) + sum_{m>=1} (x/2)^{2m} H_m / (m!)^2,
// Abramowitz & Stegun 9.6.13) integrated term by term:
//   F(R) = -(ln(k/2) + gamma) R^2 / 2
//        + sum_{m>=1} a_m R^{2m+2} / (2m+2) [H_m - ln(k/2) - gamma - ln R + 1/(2m+2)],
//   a_m = (k/2)^{2m} / (m!)^2.
__device__ double wire_F(double k, double R) {
  const double lk = log(0.5 * k) + kEulerGamma;
  const double lR = log(R);
  const double R2 = R * R;
  const double q = 0.25 * k * k * R2;
  double F = -0.5 * lk * R2;
  double am = 1.0;  // (kR/2)^{2m} / (m!)^2
  double Hm = 0.0;
  for (int m = 1; m < 200; ++m) {
    am *= q / ((double)m * (double)m);
    Hm += 1.0 / m;
    const double inv = 1.0 / (2.0 * m + 2.0);
    const double term = am * R2 * inv * (Hm - lk - lR + inv);
    F += term;
    if (fabs(term) <= 1e-18 * R2 && m > 2) break;
  }
  return F;
}

// I(k) = int over the h x h cell of [K0(k|u|) + ln|u|] = 8 int_0^{pi/4} F(h / (2 cos t)) dt
// (eight triangles with the apex at the origin), by Gauss-Legendre in t.
__device__ double wire_cell(double k, double h, const double* glx, const double* glw, int ngl) {
  const double half = 0.125 * kPi;  // (pi/4) / 2
  double acc = 0.0;
  for (int q = 0; q < ngl; ++q) {
    const double t = half * (1.0 + glx[q]);
    acc += glw[q] * wire_F(k, 0.5 * h / cos(t));
  }
  return 8.0 * half * acc;
}

// Gauss-Legendre nodes/weights on [-1, 1]: Newton on the three-term recurrence
// of the Legendre polynomials, one thread per node.
__global__ void gauss_legendre_kernel(int n, double* x, double* w) {
  const int i = threadIdx.x;
  if (i >= n) return;
  double z = cos(kPi * (i + 0.75) / (n + 0.5));
  double dp = 1.0;
  for (int it = 0; it < 100; ++it) {
    double p0 = 1.0, p1 = z;
    for (int j = 2; j <= n; ++j) {
      const double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    const double dz = p1 / dp;
    z -= dz;
    if (fabs(dz) < 1e-16) break;
  }
  x[i] = z;
  w[i] = 2.0 / ((1.0 - z * z) * dp * dp);
}

// ---------------------------------------------------------------- sampling

struct KArgs {
  int n[3], L[3], H[3], per[3];
  int nper;
  double h;
  const double* glx;
  const double* glw;
  int ngl;
};

__device__ double green_mixed(const KArgs& a, double kp, double d) {
  const double h = a.h;
  switch (a.nper) {
    case 0:
      return d == 0.0 ? -h * h * kC3 / (4.0 * kPi) : -h * h / (4.0 * kPi * d);
    case 1: {
      if (d == 0.0) {
        double v = (log(h) + kC2) / (2.0 * kPi);
        if (kp > 0.0) v -= wire_cell(kp, h, a.glx, a.glw, a.ngl) / (2.0 * kPi * h * h);
        return h * h * v;
      }
      const double r = h * d;
      if (kp == 0.0) return h * h * log(r) / (2.0 * kPi);
      return -h * h * bessel_k0(kp * r) / (2.0 * kPi);
    }
    case 2: {
      const double z = h * d;
      if (kp == 0.0) return h * 0.5 * z;
      return -h * exp(-kp * z) / (2.0 * kp);
    }
    default:
      return kp == 0.0 ? 0.0 : -1.0 / (kp * kp);
  }
}

// octant index (i1 fastest): i_j <= H_j; along a periodic axis i_j is the
// wavenumber index m (k = 2 pi m / (n h)), along a free axis the offset d
__global__ void fill_octant_kernel(double* M, KArgs a) {
  const size_t D0 = a.H[0] + 1, D1 = a.H[1] + 1, D2 = a.H[2] + 1;
  const size_t total = D0 * D1 * D2;
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i[3] = {(int)(idx % D0), (int)((idx / D0) % D1), (int)(idx / (D0 * D1))};
    double kp2 = 0.0, d2 = 0.0;
    for (int j = 0; j < 3; ++j) {
      if (a.per[j]) {
        const double k = 2.0 * kPi * i[j] / (a.n[j] * a.h);
        kp2 += k * k;
      } else {
        d2 += (double)i[j] * (double)i[j];
      }
    }
    M[idx] = green_mixed(a, sqrt(kp2), sqrt(d2));
  }
}

__global__ void cos_table_kernel(double* tab, int L) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < L; m += gridDim.x * blockDim.x)
    tab[m] = cospi(2.0 * m / L);
}

// out(k along `axis`) = sum_{i=0}^{H} w_i in(i along `axis`) cos(2 pi k i / L)
__global__ void cos_transform_kernel(const double* __restrict__ in, double* __restrict__ out,
                                     int D0, int D1, int D2, int axis, int L,
                                     const double* __restrict__ tab) {
  const size_t total = (size_t)D0 * D1 * D2;
  const int H = L / 2;
  const size_t stride = axis == 0 ? 1 : (axis == 1 ? (size_t)D0 : (size_t)D0 * D1);
  for (size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x; idx < total;
       idx += (size_t)gridDim.x * blockDim.x) {
    const int i0 = (int)(idx % D0), i1 = (int)((idx / D0) % D1), i2 = (int)(idx / ((size_t)D0 * D1));
    const int k = axis == 0 ? i0 : (axis == 1 ? i1 : i2);
    const size_t base = idx - (size_t)k * stride;
    double acc = 0.0;
    int ci = 0;  // (k * i) mod L
    for (int i = 0; i <= H; ++i) {
      const double wgt = (i == 0 || 2 * i == L) ? 1.0 : 2.0;
      acc += wgt * in[base + (size_t)i * stride] * tab[ci];
      ci += k;
      if (ci >= L) ci -= L;
    }
    out[idx] = acc;
  }
}

// dense octant (kx fastest, D0 = c columns) -> K with row pitch ldk
template <typename T>
__global__ void store_kernel(const double* __restrict__ M, T* __restrict__ K, size_t n, int D0, size_t ldk,
                             double scale) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x)
    K[(i / D0) * ldk + i % D0] = (T)(M[i] * scale);
}

template <typename T>
__global__ void twiddle_kernel(cpx<T>* tw, int L) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < L; k += gridDim.x * blockDim.x) {
    double s, c;
    sincospi(2.0 * k / L, &s, &c);
    tw[k] = mk((T)c, (T)(-s));
  }
}

// twiddle matrix of the x passes: twx[r P + c] = W_M^{r c} = W_L1^{2 r c}, r, c < P
__global__ void twiddle_matrix_kernel(float2* twx, int L1, int P) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < P * P; idx += gridDim.x * blockDim.x) {
    const int r = idx / P, c = idx % P;
    double s, co;
    sincospi(2.0 * ((2 * r * c) % L1) / L1, &s, &co);
    twx[idx] = make_float2((float)co, (float)(-s));
  }
}

// paired twiddles of the packed z kernel: tw4[r T + c] = (Re W^{rc}, Re W^{(r+T)c},
// Im W^{rc}, Im W^{(r+T)c}), W = exp(-2 pi i / L), r, c < T
__global__ void twiddle_pairs_kernel(float4* tw4, int L, int T, int P) {
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < T * P; idx += gridDim.x * blockDim.x) {
    const int r = idx / P, c = idx % P;
    double s0, c0, s1, c1;
    sincospi(2.0 * ((r * c) % L) / L, &s0, &c0);
    sincospi(2.0 * (((r + T) * c) % L) / L, &s1, &c1);
    tw4[idx] = make_float4((float)c0, (float)c1, (float)(-s0), (float)(-s1));
  }
}

// Bluestein tables for a transform of length N, convolution length M:
//   chirp[m] = exp(-i pi m^2 / N), m < N
//   Bf[k] = (1/M) sum_j b[j] W_M^{jk}, b[j] = conj(chirp[|j|]) for |j| < N (j taken mod M)
// Phases are reduced exactly in integers (m^2 mod 2N, j k mod M) before sincospi.
template <typename T>
__global__ void chirp_kernel(cpx<T>* ch, int N) {
  for (int m = blockIdx.x * blockDim.x + threadIdx.x; m < N; m += gridDim.x * blockDim.x) {
    const long long q = ((long long)m * m) % (2LL * N);
    double s, c;
    sincospi((double)q / N, &s, &c);
    ch[m] = mk((T)c, (T)(-s));
  }
}

template <typename T>
__global__ void bluestein_bf_kernel(cpx<T>* Bf, int N, int M) {
  for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < M; k += gridDim.x * blockDim.x) {
    double re = 0.0, im = 0.0;
    for (int j = 0; j < N; ++j) {
      const double a = (double)(((long long)j * j) % (2LL * N)) / N;  // exp(+i pi j^2 / N)
      const double w = 2.0 * (double)(((long long)j * k) % M) / M;   // W_M^{jk}:  exp(-i pi w)
      double s, c;
      sincospi(a - w, &s, &c);
      re += c;
      im += s;
      if (j > 0) {  // the mirrored sample at M - j: exp(+i pi j^2 / N) W_M^{(M - j) k}
        sincospi(a + w, &s, &c);
        re += c;
        im += s;
      }
    }
    Bf[k] = mk((T)(re / M), (T)(im / M));
  }
}

// ---------------------------------------------------------------- host

static int grid_for(size_t n) {
  size_t g = (n + 255) / 256;
  if (g > 152 * 64) g = 152 * 64;
  return (int)(g < 1 ? 1 : g);
}

cudaError_t build_twiddles(ps_plan_s* p, cudaStream_t s) {
  for (int j = 0; j < 3; ++j) {
    const int L = p->L[j];
    if (p->dtype == PS_F32)
      twiddle_kernel<float><<<grid_for(L), 256, 0, s>>>(static_cast<float2*>(p->tw[j]), L);
    else
      twiddle_kernel<double><<<grid_for(L), 256, 0, s>>>(static_cast<double2*>(p->tw[j]), L);
  }
  for (int j = 0; j < 3; ++j) {
    const BlueArgs& b = p->blue[j];
    if (!b.M) continue;
    const int N = xform_len(p, j);
    if (p->dtype == PS_F32) {
      twiddle_kernel<float><<<grid_for(b.M), 256, 0, s>>>((float2*)b.twM, b.M);
      chirp_kernel<float><<<grid_for(N), 256, 0, s>>>((float2*)b.chirp, N);
      bluestein_bf_kernel<float><<<grid_for(b.M), 256, 0, s>>>((float2*)b.Bf, N, b.M);
    } else {
      twiddle_kernel<double><<<grid_for(b.M), 256, 0, s>>>((double2*)b.twM, b.M);
      chirp_kernel<double><<<grid_for(N), 256, 0, s>>>((double2*)b.chirp, N);
      bluestein_bf_kernel<double><<<grid_for(b.M), 256, 0, s>>>((double2*)b.Bf, N, b.M);
    }
  }
  if (p->xP)
    twiddle_matrix_kernel<<<grid_for(p->xP * p->xP), 256, 0, s>>>(static_cast<float2*>(p->twx), p->L[0], p->xP);
  // the packed y and z kernels run along the second and third axes of the order
  if (p->ysoa)
    twiddle_pairs_kernel<<<grid_for(256), 256, 0, s>>>(static_cast<float4*>(p->tw4y), p->L[p->ord[1]], 16,
                                                       p->L[p->ord[1]] / 32);  // L2 = P * 32
  if (p->zsoa_T)
    twiddle_pairs_kernel<<<grid_for(p->zsoa_T * p->zsoa_P), 256, 0, s>>>(
        static_cast<float4*>(p->tw4z), p->L[p->ord[2]], p->zsoa_T, p->zsoa_P);
  return cudaGetLastError();
}

cudaError_t build_kernel(ps_plan_s* p, cudaStream_t s) {
  const int D0 = p->H[0] + 1, D1 = p->H[1] + 1, D2 = p->H[2] + 1;
  const size_t total = (size_t)D0 * D1 * D2;
  double *M0 = nullptr, *M1 = nullptr, *gl = nullptr, *tab = nullptr;
  cudaError_t e = cudaSuccess;
  KArgs a;
  for (int j = 0; j < 3; ++j) {
    a.n[j] = p->n[j]; a.L[j] = p->L[j]; a.H[j] = p->H[j];
    a.per[j] = p->bc[j] == PS_BC_PERIODIC;
  }
  a.nper = a.per[0] + a.per[1] + a.per[2];
  a.h = p->h;
  a.ngl = 32;
  int maxL = 0;
  for (int j = 0; j < 3; ++j) maxL = p->L[j] > maxL ? p->L[j] : maxL;

  if ((e = cudaMalloc(&M0, total * sizeof(double))) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&M1, total * sizeof(double))) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&gl, 2 * a.ngl * sizeof(double))) != cudaSuccess) goto done;
  if ((e = cudaMalloc(&tab, (size_t)maxL * sizeof(double))) != cudaSuccess) goto done;
  a.glx = gl;
  a.glw = gl + a.ngl;
  gauss_legendre_kernel<<<1, 64, 0, s>>>(a.ngl, gl, gl + a.ngl);
  fill_octant_kernel<<<grid_for(total), 256, 0, s>>>(M0, a);
  for (int j = 0; j < 3; ++j) {
    if (a.per[j]) continue;
    cos_table_kernel<<<grid_for(p->L[j]), 256, 0, s>>>(tab, p->L[j]);
    cos_transform_kernel<<<grid_for(total), 256, 0, s>>>(M0, M1, D0, D1, D2, j, p->L[j], tab);
    double* t = M0; M0 = M1; M1 = t;
  }
  {
    const double scale = 1.0 / ((double)p->L[0] * (double)p->L[1] * (double)p->L[2]);
    // the pitch padding stays zero
    e = cudaMemsetAsync(p->K, 0, p->ldk * (size_t)D1 * D2 * p->esz, s);
    if (e != cudaSuccess) goto done;
    if (p->dtype == PS_F32)
      store_kernel<float><<<grid_for(total), 256, 0, s>>>(M0, static_cast<float*>(p->K), total, D0, p->ldk, scale);
    else
      store_kernel<double><<<grid_for(total), 256, 0, s>>>(M0, static_cast<double*>(p->K), total, D0, p->ldk,
                                                            scale);
  }
  if ((e = cudaGetLastError()) != cudaSuccess) goto done;
  e = cudaStreamSynchronize(s);
done:
  // temporaries are released only after the stream has drained (or failed)
  cudaStreamSynchronize(s);
  if (M0) cudaFree(M0);
  if (M1) cudaFree(M1);
  if (gl) cudaFree(gl);
  if (tab) cudaFree(tab);
  return e;
}

// A caller's kernel given in real space on its even octant, octant[d1 + D0 (d2
// + D1 d3)] = K(d1, d2, d3), d_j <= L_j / 2: the even-cosine transform along
// every axis (free and periodic alike: an even sequence of period L_j) gives
// K^F on the octant of wavenumber indices, stored like build_kernel's.
cudaError_t build_kernel_from_real(ps_plan_s* p, const double* host_octant, cudaStream_t s) {
  const int D0 = p->H[0] + 1, D1 = p->H[1] + 1, D2 = p->H[2] + 1;
  const size_t total = (size_t)D0 * D1 * D2;
  double *M0 = nullptr, *M1 = nullptr, *tab = nullptr;
  int maxL = 0;
  for (int j = 0; j < 3; ++j) maxL = p->L[j] > maxL ? p->L[j] : maxL;
  cudaError_t e = cudaMalloc(&M0, total * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&M1, total * sizeof(double));
  if (e == cudaSuccess) e = cudaMalloc(&tab, (size_t)maxL * sizeof(double));
  if (e == cudaSuccess) e = cudaMemcpyAsync(M0, host_octant, total * sizeof(double), cudaMemcpyHostToDevice, s);
  for (int j = 0; j < 3 && e == cudaSuccess; ++j) {
    cos_table_kernel<<<grid_for(p->L[j]), 256, 0, s>>>(tab, p->L[j]);
    cos_transform_kernel<<<grid_for(total), 256, 0, s>>>(M0, M1, D0, D1, D2, j, p->L[j], tab);
    double* t = M0; M0 = M1; M1 = t;
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) {
    const double scale = 1.0 / ((double)p->L[0] * (double)p->L[1] * (double)p->L[2]);
    e = cudaMemsetAsync(p->K, 0, p->ldk * (size_t)D1 * D2 * p->esz, s);
    if (e == cudaSuccess) {
      if (p->dtype == PS_F32)
        store_kernel<float><<<grid_for(total), 256, 0, s>>>(M0, static_cast<float*>(p->K), total, D0, p->ldk, scale);
      else
        store_kernel<double><<<grid_for(total), 256, 0, s>>>(M0, static_cast<double*>(p->K), total, D0, p->ldk,
                                                              scale);
      e = cudaGetLastError();
    }
  }
  cudaError_t e2 = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = e2;
  if (M0) cudaFree(M0);
  if (M1) cudaFree(M1);
  if (tab) cudaFree(tab);
  return e;
}

}  // namespace ps
