// Imaginary-time grid and tau <-> Matsubara transform matrices, built on the
// device (Sec. "Self-consistent finite-temperature GW", Eqs. tau_to_iw and
// iw_to_tau; Sec. "Representation on the imaginary axes").
//
// tau_j = beta sin^2(pi (2j+1) / (4 ntau)) (first-kind Chebyshev roots,
// ascending).  L_j(x) = sum_k C[k][j] T_k(x), C[k][j] = (2 - delta_k0)/ntau
// T_k(x_j).  TF[n][j] = (beta/2) e^{i a_n} sum_k I_k(a_n) C[k][j] with the
// Chebyshev moments I_k(a) = int_{-1}^{1} T_k(x) e^{i a x} dx summed from the
// Jacobi-Anger series (Bessel J_m(a) by Miller's backward recurrence).
// a = (2n+1) pi/2 (fermions) or m pi (bosons): e^{i a} is exact.
// TB = TF^{-1} by Gauss-Jordan with partial pivoting (one thread block).
#include <math.h>
#include "gw_internal.cuh"
#include "gj.cuh"

namespace gwk {

__device__ __forceinline__ double half_angle(int f, int ntau, const int* fn, const int* bm) {
  return f < ntau ? (2.0 * fn[f] + 1.0) * (M_PI / 2.0) : (double)bm[f - ntau] * M_PI;
}
__host__ __device__ inline int bessel_mmax(double a, int ntau) {
  double aa = fabs(a);
  return (int)(aa + 25.0 * cbrt(aa + 1.0) + 50.0) + ntau;
}

// J[f][m] = J_m(a_f), m <= mmax(f), by backward recurrence normalised with
// J_0 + 2 sum_{k>=1} J_{2k} = 1.  One thread per frequency.
__global__ void bessel_kernel(int ntau, const int* fn, const int* bm, double* J, int ld) {
  int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= 2 * ntau) return;
  double a = half_angle(f, ntau, fn, bm);
  int mmax = bessel_mmax(a, ntau);
  double* Jf = J + (int64_t)f * ld;
  double aa = fabs(a);
  if (aa == 0.0) {
    Jf[0] = 1.0;
    for (int m = 1; m <= mmax; ++m) Jf[m] = 0.0;
    return;
  }
  int M = mmax + 40 + (int)(10.0 * cbrt(aa));
  M += (M & 1);
  double jp = 0.0, jc = 1e-280, S = 0.0;
  for (int m = M; m >= 1; --m) {
    // jc = j_m, jp = j_{m+1}
    if (m <= mmax) Jf[m] = jc;
    if ((m & 1) == 0) S += 2.0 * jc;
    double jm = (2.0 * m / aa) * jc - jp;
    jp = jc; jc = jm;
    if (fabs(jc) > 1e250) {
      const double sc = 1e-250;
      jc *= sc; jp *= sc; S *= sc;
      for (int t = m; t <= mmax; ++t) Jf[t] *= sc;
    }
  }
  Jf[0] = jc;
  S += jc;
  double inv = 1.0 / S;
  double sgn = a < 0 ? -1.0 : 1.0;  // J_m(-a) = (-1)^m J_m(a)
  for (int m = 0; m <= mmax; ++m) Jf[m] *= ((m & 1) && sgn < 0) ? -inv : inv;
}

// I[f][k] = sum_m c_m W_km,  c_m = eps_m i^m J_m(a_f),  W_km = int T_k T_m.
__global__ void moments_kernel(int ntau, const int* fn, const int* bm, const double* J, int ld, double2* I) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * ntau * ntau) return;
  int f = e / ntau, k = e - f * ntau;
  double a = half_angle(f, ntau, fn, bm);
  int mmax = bessel_mmax(a, ntau);
  const double* Jf = J + (int64_t)f * ld;
  double sr = 0, si = 0, cr = 0, ci = 0;  // Kahan compensation
  for (int m = (k & 1); m <= mmax; m += 2) {
    double kp = (double)(k + m), km = (double)(k - m);
    double w = 1.0 / (1.0 - kp * kp) + 1.0 / (1.0 - km * km);
    double v = (m == 0 ? 1.0 : 2.0) * Jf[m] * w;
    // i^m
    double re = 0, im = 0;
    switch (m & 3) { case 0: re = v; break; case 1: im = v; break; case 2: re = -v; break; default: im = -v; }
    double y = re - cr, t = sr + y; cr = (t - sr) - y; sr = t;
    y = im - ci; t = si + y; ci = (t - si) - y; si = t;
  }
  I[e] = make_double2(sr, si);
}

// C[k][j] = (2 - delta_k0)/ntau T_k(x_j),  T_k(x_j) = cos(pi k (2 ntau - 2j - 1) / (2 ntau))
__device__ __forceinline__ double cheb_c(int k, int j, int ntau) {
  long long r = ((long long)k * (2 * ntau - 2 * j - 1)) % (4LL * ntau);
  double t = cospi((double)r / (2.0 * ntau));
  return (k == 0 ? 1.0 : 2.0) / ntau * t;
}

__global__ void tf_kernel(int ntau, double beta, const int* fn, const int* bm, const double2* I,
                          double2* TFf, double2* TFb) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 2 * ntau * ntau) return;
  int f = e / ntau, j = e - f * ntau;
  double sr = 0, si = 0;
  for (int k = 0; k < ntau; ++k) {
    double c = cheb_c(k, j, ntau);
    double2 v = I[(int64_t)f * ntau + k];
    sr += v.x * c; si += v.y * c;
  }
  // e^{i a}: fermions i^{2n+1}, bosons (-1)^m
  int q = f < ntau ? (((2 * fn[f] + 1) % 4) + 4) % 4 : ((((bm[f - ntau]) % 2) + 2) % 2) * 2;
  double re = 0, im = 0;
  switch (q) { case 0: re = sr; im = si; break; case 1: re = -si; im = sr; break;
               case 2: re = -sr; im = -si; break; default: re = si; im = -sr; }
  double h = 0.5 * beta;
  if (f < ntau) TFf[(int64_t)f * ntau + j] = make_double2(h * re, h * im);
  else TFb[(int64_t)(f - ntau) * ntau + j] = make_double2(h * re, h * im);
}

__global__ void nodes_kernel(int ntau, double beta, double* tau, double* lb, double* l0) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= ntau) return;
  double s = sinpi((2.0 * j + 1.0) / (4.0 * ntau));
  tau[j] = beta * s * s;
  double b = 0, z = 0;
  for (int k = 0; k < ntau; ++k) {
    double c = cheb_c(k, j, ntau);
    b += c;                         // T_k(1) = 1
    z += (k & 1) ? -c : c;          // T_k(-1) = (-1)^k
  }
  lb[j] = b; l0[j] = z;
}

size_t grid_ws_bytes(int ntau, const int* fn_host, const int* bm_host, int* ld_out) {
  int ld = 0;
  for (int f = 0; f < ntau; ++f) {
    int m1 = bessel_mmax((2.0 * fn_host[f] + 1.0) * (M_PI / 2.0), ntau) + 1;
    int m2 = bessel_mmax((double)bm_host[f] * M_PI, ntau) + 1;
    ld = ld > m1 ? ld : m1;
    ld = ld > m2 ? ld : m2;
  }
  *ld_out = ld;
  return (size_t)2 * ntau * ld * sizeof(double) + (size_t)2 * ntau * ntau * sizeof(double2);
}

cudaError_t grid_build_ws(int ntau, double beta, const int* d_fn, const int* d_bm, int ld, void* ws,
                          double* tau, double2* TFf, double2* TFb, double* lb, double* l0, cudaStream_t st) {
  double* J = (double*)ws;
  double2* I = (double2*)(J + (size_t)2 * ntau * ld);
  bessel_kernel<<<(2 * ntau + 63) / 64, 64, 0, st>>>(ntau, d_fn, d_bm, J, ld);
  int ne = 2 * ntau * ntau;
  moments_kernel<<<(ne + 127) / 128, 128, 0, st>>>(ntau, d_fn, d_bm, J, ld, I);
  tf_kernel<<<(ne + 127) / 128, 128, 0, st>>>(ntau, beta, d_fn, d_bm, I, TFf, TFb);
  nodes_kernel<<<(ntau + 63) / 64, 64, 0, st>>>(ntau, beta, tau, lb, l0);
  return cudaGetLastError();
}

// In-place inversion of one n x n matrix in global memory by a single block.
__global__ void __launch_bounds__(1024) gj_global_kernel(double2* A, int n, int* info) {
  extern __shared__ unsigned char smem[];
  double2* f = (double2*)smem;
  int* perm = (int*)(f + n);
  double* rv = (double*)(perm + n + (n & 1));
  int* ri = (int*)(rv + blockDim.x);
  int bad = gj_invert_smem(A, n, n, f, perm, rv, ri);  // A in global memory, same algorithm
  if (threadIdx.x == 0 && bad) atomicOr(info, 1);
}
cudaError_t invert_small_gj(double2* A, int n, int* d_info, cudaStream_t st) {
  int nt = 256;
  size_t sm = (size_t)n * sizeof(double2) + (size_t)(n + 1) * sizeof(int) + 8 + nt * (sizeof(double) + sizeof(int));
  gj_global_kernel<<<1, nt, sm, st>>>(A, n, d_info);
  return cudaGetLastError();
}

// r[n] = sum_j lb[j] TBf[j][n], TBf [ntau][nwf]  (weights of the density: gamma = -sum_n r_n G(i w_n))
__global__ void rweights_kernel(int ntau, int nwf, const double* lb, const double2* TBf, double2* r) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= nwf) return;
  double re = 0, im = 0;
  for (int j = 0; j < ntau; ++j) { double2 t = TBf[(int64_t)j * nwf + n]; re += lb[j] * t.x; im += lb[j] * t.y; }
  r[n] = make_double2(re, im);
}
cudaError_t density_weights(int ntau, int nwf, const double* lb, const double2* TBf, double2* r, cudaStream_t st) {
  rweights_kernel<<<(nwf + 63) / 64, 64, 0, st>>>(ntau, nwf, lb, TBf, r);
  return cudaGetLastError();
}

// frequencies w_n = (2n+1) pi / beta
__global__ void freq_kernel(int nwf, double beta, const int* fn, double* wn) {
  int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n < nwf) wn[n] = (2.0 * fn[n] + 1.0) * M_PI / beta;
}
cudaError_t fermi_freqs(int nwf, double beta, const int* fn, double* wn, cudaStream_t st) {
  freq_kernel<<<(nwf + 63) / 64, 64, 0, st>>>(nwf, beta, fn, wn);
  return cudaGetLastError();
}

}  // namespace gwk
