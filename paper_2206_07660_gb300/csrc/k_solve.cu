// Screened interaction in the auxiliary basis (Eq. tilde_P_omega):
// P~ = [I - P~0]^{-1} P~0 = [I - P~0]^{-1} - I, for every (q, Omega_m).
//
// The identity [I - P~0]^{-1} P~0 = [I - P~0]^{-1} - I turns the solve into one
// in-place inversion per system (n^3 complex MACs instead of 4n^3/3 for an LU
// solve with n right-hand sides).  The inversion is a blocked Gauss-Jordan
// sweep without pivoting across blocks (I - P~0 has a positive-definite
// Hermitian part because P~0(i Omega) has a negative-semidefinite one), with
// partial pivoting inside each nb x nb diagonal block.  Per block step:
//   Dinv = A[b,b]^{-1};  Rn = Dinv A[b,:] (with Rn[:,b] = Dinv);
//   A[i,:] -= A[i,b] Rn for i not in b (A[:,b] zeroed first);  A[b,:] = Rn.
// The rank-nb update is the generic contraction kernel, batched over systems.
//
// With the tensor cores available the inversion runs in complex64 and two Newton
// steps with FP64-accurate residuals bring it to FP64 accuracy (screened_refine).
#include "gw_internal.cuh"
#include "gj.cuh"

namespace gwk {

template <typename T> struct TyOf;
template <> struct TyOf<double2> { static constexpr Ty v = Ty::C128; };
template <> struct TyOf<float2> { static constexpr Ty v = Ty::C64; };

template <typename T>
__global__ void extract_kernel(const T* __restrict__ X, int64_t n, int nb, int64_t kb, int64_t count, T* Cp, T* Rp) {
  const int64_t per = 2 * n * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * count; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t z = e / per, r = e - z * per;
    const T* Xz = X + z * n * n;
    if (r < n * nb) {          // column panel Cp[i][c] (rows of block b zeroed)
      int64_t i = r / nb, c = r - i * nb;
      T v = Xz[i * n + kb + c];
      if (i >= kb && i < kb + nb) { v.x = 0; v.y = 0; }
      Cp[z * n * nb + r] = v;
    } else {                   // row panel Rp[c][j]
      r -= n * nb;
      int64_t c = r / n, j = r - c * n;
      Rp[z * n * nb + r] = Xz[(kb + c) * n + j];
    }
  }
}

template <typename T>
__global__ void zero_cols_kernel(T* X, int64_t n, int nb, int64_t kb, int64_t count) {
  const int64_t per = n * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * count; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t z = e / per, r = e - z * per, i = r / nb, c = r - i * nb;
    T v; v.x = 0; v.y = 0;
    X[z * n * n + i * n + kb + c] = v;
  }
}

// Dinv[z] = (Rp[z][:, kb:kb+nb])^{-1}, one block per system, in shared memory, in
// T's precision.
template <typename T>
__global__ void __launch_bounds__(256) block_inv_kernel(const T* __restrict__ Rp, int64_t n, int nb, int64_t kb,
                                                        int64_t count, T* Dinv, int* info) {
  using R = typename gj_real<T>::t;
  extern __shared__ __align__(16) unsigned char smem[];
  T* A = (T*)smem;
  T* f = A + nb * nb;
  int* perm = (int*)(f + nb);
  R* rv = (R*)(perm + nb + (nb & 1));
  int* ri = (int*)(rv + blockDim.x);
  for (int64_t z = blockIdx.x; z < count; z += gridDim.x) {
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) {
      int r = e / nb, c = e - r * nb;
      A[e] = Rp[z * n * nb + (int64_t)r * n + kb + c];
    }
    __syncthreads();
    int bad = gj_invert_smem(A, nb, nb, f, perm, rv, ri);
    if (bad && threadIdx.x == 0) atomicOr(info, 1);
    for (int e = threadIdx.x; e < nb * nb; e += blockDim.x) Dinv[z * nb * nb + e] = A[e];
    __syncthreads();
  }
}

// Rn[z][r][kb + c] = Dinv[z][r][c]
template <typename T>
__global__ void put_dinv_kernel(T* Rn, const T* __restrict__ Dinv, int64_t n, int nb, int64_t kb, int64_t count) {
  const int64_t per = (int64_t)nb * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * count; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t z = e / per, r = (e - z * per) / nb, c = (e - z * per) % nb;
    Rn[z * n * nb + r * n + kb + c] = Dinv[e];
  }
}

template <typename T>
static size_t block_inv_smem(int64_t nb, int nt) {
  using R = typename gj_real<T>::t;
  return (size_t)nb * nb * sizeof(T) + (size_t)nb * sizeof(T) + (size_t)(nb + 1) * sizeof(int) + 8 +
         (size_t)nt * (sizeof(R) + sizeof(int));
}

// X[z][kb + r][j] = Rn[z][r][j]
template <typename T>
__global__ void put_rows_kernel(T* X, const T* __restrict__ Rn, int64_t n, int nb, int64_t kb, int64_t count) {
  const int64_t per = n * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * count; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t z = e / per, r = e - z * per;
    X[z * n * n + kb * n + r] = Rn[e];
  }
}

static const int NB = 64;

template <typename T>
static size_t gj_bytes_per_sys(int64_t n) {
  const int64_t nb = n < NB ? n : NB;
  return (size_t)(3 * n * nb + nb * nb) * sizeof(T);
}

// workspace of gj_blocked for `count` systems at once (the block inverses start on a
// 256-byte boundary after the three panels)
template <typename T>
static size_t gj_work_bytes(int64_t n, int64_t count) { return (size_t)count * gj_bytes_per_sys<T>(n) + 256; }

size_t screened_work_bytes(int64_t n, int64_t count) { return gj_work_bytes<double2>(n, count); }

static inline int grid1(int64_t work) {
  int64_t b = (work + 255) / 256;
  return (int)(b < 152 * 32 ? b : 152 * 32);
}

// In-place blocked Gauss-Jordan inversion of count n x n systems (contiguous) stored
// as T, in T's precision (the SIMT contraction kernel for the rank-nb updates).
// Returns the number of kernels launched in *nlaunch (when not null).
template <typename T>
static cudaError_t gj_blocked(T* X, int64_t n, int64_t count, void* work, size_t work_bytes, int* d_info,
                              cudaStream_t st, int64_t* nlaunch) {
  const int64_t nbmax = n < NB ? n : NB;
  const size_t per_sys = gj_bytes_per_sys<T>(n);
  int64_t chunk = work_bytes > 256 ? (int64_t)((work_bytes - 256) / per_sys) : 0;
  if (chunk <= 0) return cudaErrorMemoryAllocation;
  if (chunk > 65535) chunk = 65535;
  const int nt = 256;
  const size_t sm = block_inv_smem<T>(nbmax, nt);
  cudaError_t e;
  if (sm > 48 * 1024) {
    e = cudaFuncSetAttribute(block_inv_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  const Ty ty = TyOf<T>::v;
  int64_t launches = 0;
  for (int64_t z0 = 0; z0 < count; z0 += chunk) {
    const int64_t cz = (count - z0) < chunk ? (count - z0) : chunk;
    T* Xc = X + z0 * n * n;
    T* Cp = (T*)work;
    T* Rp = Cp + cz * n * nbmax;
    T* Rn = Rp + cz * n * nbmax;
    T* Di = (T*)((char*)work + (((size_t)3 * cz * n * nbmax * sizeof(T) + 255) & ~(size_t)255));
    for (int64_t kb = 0; kb < n; kb += nbmax) {
      const int nb = (int)((n - kb) < nbmax ? (n - kb) : nbmax);
      extract_kernel<T><<<grid1(2 * n * nb * cz), 256, 0, st>>>(Xc, n, nb, kb, cz, Cp, Rp);
      zero_cols_kernel<T><<<grid1(n * nb * cz), 256, 0, st>>>(Xc, n, nb, kb, cz);
      block_inv_kernel<T><<<(int)(cz < 152 * 8 ? cz : 152 * 8), nt, sm, st>>>(Rp, n, nb, kb, cz, Di, d_info);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      // Rn[z] = Dinv[z] (nb x nb) * Rp[z] (nb x n)
      GettDesc g{};
      g.M = nb; g.N = n; g.K = nb; g.Z = cz;
      g.am = I1(nb); g.ak = I1(1); g.az = I1((int64_t)nb * nb);
      g.bk = I1(n); g.bn = I1(1); g.bz = I1(n * nb);
      g.cm = I1(n); g.cn = I1(1); g.cz = I1(n * nb);
      g.alpha = make_double2(1, 0); g.beta = make_double2(0, 0); g.ksplit = 1;
      if ((e = gett(g, Di, ty, Rp, ty, Rn, ty, ty, nullptr, 0, st)) != cudaSuccess) return e;
      put_dinv_kernel<T><<<grid1((int64_t)nb * nb * cz), 256, 0, st>>>(Rn, Di, n, nb, kb, cz);
      // X[z] -= Cp[z] (n x nb) * Rn[z] (nb x n)
      GettDesc u{};
      u.M = n; u.N = n; u.K = nb; u.Z = cz;
      u.am = I1(nb); u.ak = I1(1); u.az = I1(n * nb);
      u.bk = I1(n); u.bn = I1(1); u.bz = I1(n * nb);
      u.cm = I1(n); u.cn = I1(1); u.cz = I1(n * n);
      u.alpha = make_double2(-1, 0); u.beta = make_double2(1, 0); u.ksplit = 1;
      if ((e = gett(u, Cp, ty, Rn, ty, Xc, ty, ty, nullptr, 0, st)) != cudaSuccess) return e;
      put_rows_kernel<T><<<grid1(n * nb * cz), 256, 0, st>>>(Xc, Rn, n, nb, kb, cz);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      launches += 7;
    }
  }
  if (nlaunch) *nlaunch += launches;
  return cudaSuccess;
}

static inline int64_t pad32(int64_t x) { return (x + 31) / 32 * 32; }

// split planes of one block step of gj_blocked_tc, per system
static size_t gj_tc_plane_bytes(int64_t n) {
  const int64_t nb = n < NB ? n : NB, Kb = pad32(2 * nb);
  return (size_t)8 * Kb * (5 * n + nb);   // hi/lo of Cp (n rows), Dinv (nb), Rp^T and Rn^T (2n each)
}

// gj_blocked for complex64 storage with both products of a block step on the
// tensor cores (split TF32, three products): Rn = Dinv Rp and X -= Cp Rn; block
// inverses in complex64.  planes: gj_tc_plane_bytes(n) per system.
static cudaError_t gj_blocked_tc(float2* X, int64_t n, int64_t cz, void* pan, float* planes, int* d_info, int* d_err,
                                 cudaStream_t st, int64_t* nlaunch) {
  const int64_t nbmax = n < NB ? n : NB, Kb = pad32(2 * nbmax);
  const int nt = 256;
  const size_t sm = block_inv_smem<float2>(nbmax, nt);
  cudaError_t e;
  if (sm > 48 * 1024) {
    e = cudaFuncSetAttribute(block_inv_kernel<float2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  float2* Cp = (float2*)pan;
  float2* Rp = Cp + cz * n * nbmax;
  float2* Rn = Rp + cz * n * nbmax;
  float2* Di = (float2*)((char*)pan + (((size_t)3 * cz * n * nbmax * sizeof(float2) + 255) & ~(size_t)255));
  float* Ch = planes;
  float* Cl = Ch + cz * n * Kb;
  float* Dh = Cl + cz * n * Kb;
  float* Dl = Dh + cz * nbmax * Kb;
  float* Rh = Dl + cz * nbmax * Kb;
  float* Rl = Rh + cz * 2 * n * Kb;
  float* Nh = Rl + cz * 2 * n * Kb;
  float* Nl = Nh + cz * 2 * n * Kb;
  int64_t launches = 0;
  for (int64_t kb = 0; kb < n; kb += nbmax) {
    const int nb = (int)((n - kb) < nbmax ? (n - kb) : nbmax);
    const int64_t Kp = pad32(2 * nb);
    extract_kernel<float2><<<grid1(2 * n * nb * cz), 256, 0, st>>>(X, n, nb, kb, cz, Cp, Rp);
    zero_cols_kernel<float2><<<grid1(n * nb * cz), 256, 0, st>>>(X, n, nb, kb, cz);
    block_inv_kernel<float2><<<(int)(cz < 152 * 8 ? cz : 152 * 8), nt, sm, st>>>(Rp, n, nb, kb, cz, Di, d_info);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    // Rn[z] = Dinv[z] (nb x nb) Rp[z] (nb x n)
    if ((e = split_rows(Di, false, cz * nb, nb, nb, false, Dh, Dl, Kp, st)) != cudaSuccess) return e;
    if ((e = embed_t_batched(Rp, false, cz, nb, n, n, n * nb, Rh, Rl, Kp, 2 * n * Kp, st)) != cudaSuccess) return e;
    {
      UmmaOperand a{Dh, Dl, nb, cz, Kp, nb * Kp}, b{Rh, Rl, 2 * n, cz, Kp, 2 * n * Kp};
      if ((e = umma_gemm(a, b, nb, (int)(2 * n), Kp, (int)cz, Rn, false, 1.0, false, 2 * n, 2 * n * nb, 3, d_err, st,
                         1, 0, 0, 0, 0, nullptr, nullptr, 2 * nb)) != cudaSuccess)
        return e;
    }
    put_dinv_kernel<float2><<<grid1((int64_t)nb * nb * cz), 256, 0, st>>>(Rn, Di, n, nb, kb, cz);
    // X[z] -= Cp[z] (n x nb) Rn[z] (nb x n)
    if ((e = split_rows(Cp, false, cz * n, nb, nb, false, Ch, Cl, Kp, st)) != cudaSuccess) return e;
    if ((e = embed_t_batched(Rn, false, cz, nb, n, n, n * nb, Nh, Nl, Kp, 2 * n * Kp, st)) != cudaSuccess) return e;
    {
      UmmaOperand a{Ch, Cl, n, cz, Kp, n * Kp}, b{Nh, Nl, 2 * n, cz, Kp, 2 * n * Kp};
      if ((e = umma_gemm(a, b, (int)n, (int)(2 * n), Kp, (int)cz, X, false, -1.0, true, 2 * n, 2 * n * n, 3, d_err,
                         st, 1, 0, 0, 0, 0, nullptr, nullptr, 2 * nb)) != cudaSuccess)
        return e;
    }
    put_rows_kernel<float2><<<grid1(n * nb * cz), 256, 0, st>>>(X, Rn, n, nb, kb, cz);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    launches += 11;
  }
  if (nlaunch) *nlaunch += launches;
  return cudaSuccess;
}

// In-place: X (count systems of n x n, contiguous) holds P~0 on entry and P~ on exit.
cudaError_t screened_inplace(double2* X, int64_t n, int64_t count, double2* work, size_t work_bytes,
                             int* d_info, cudaStream_t st) {
  cudaError_t e = identity_minus(X, n, count, -1.0, st);        // X <- I - P~0
  if (e != cudaSuccess) return e;
  if ((e = gj_blocked<double2>(X, n, count, work, work_bytes, d_info, st, nullptr)) != cudaSuccess) return e;
  return identity_minus(X, n, count, +1.0, st);                 // X <- (I - P~0)^{-1} - I
}

// ------------------------------------------------------------------ mixed-precision refinement
// Y = (I - P~0)^{-1} from a complex64 inversion, refined by Newton steps
//   E = I - (I - P~0) Y = I - Y + P~0 Y,   Y <- Y + Y E,
// with P~0 Y from digit-split products on the tensor cores and Y E in split TF32
// (its size is that of E, ~1e-7 after the first inversion, so FP32-class relative
// accuracy suffices).  A step with a residual computed to an absolute error delta
// leaves ||E'|| ~ ||E||^2 + delta: the first step takes the leading 5 digits of the
// product (delta ~ sqrt(2n) 9e-11, squared below FP64 rounding by the next step),
// the last one all 8 (FP64-exact).  Relative error: 1e-7 -> 1e-14 -> FP64 rounding.

__global__ void f_from_iminus_kernel(const double2* __restrict__ X, float2* __restrict__ F, int64_t n, int64_t tot) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % (n * n);
    const double d = (r / n == r % n) ? 1.0 : 0.0;
    const double2 v = X[e];
    F[e] = make_float2((float)(d - v.x), (float)(-v.y));
  }
}
__global__ void x_from_f_kernel(const float2* __restrict__ F, double2* __restrict__ X, int64_t tot) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const float2 v = F[e];
    X[e] = make_double2((double)v.x, (double)v.y);
  }
}
// T <- I - Y + T
__global__ void resid_kernel(const double2* __restrict__ Y, double2* __restrict__ T, int64_t n, int64_t tot) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % (n * n);
    const double d = (r / n == r % n) ? 1.0 : 0.0;
    const double2 y = Y[e], t = T[e];
    T[e] = make_double2(d - y.x + t.x, -y.y + t.y);
  }
}
// Y <- Y + F  (last: minus I as well)
__global__ void y_update_kernel(double2* __restrict__ Y, const float2* __restrict__ F, int64_t n, int64_t tot,
                                int last) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e % (n * n);
    const double d = (last && r / n == r % n) ? 1.0 : 0.0;
    const double2 y = Y[e];
    const float2 f = F[e];
    Y[e] = make_double2(y.x + (double)f.x - d, y.y + (double)f.y);
  }
}

static size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }

// split planes of the correction product Y E, per system
static size_t corr_plane_bytes(int64_t n) { return (size_t)24 * n * emul_kpad(n); }

// the region that holds the digits of Y during the residual, the split planes of the
// inversion before and those of the correction after it
static size_t shared_plane_bytes(int64_t n) {
  size_t b = emul_digit_bytes(2 * n, n);
  if (gj_tc_plane_bytes(n) > b) b = gj_tc_plane_bytes(n);
  if (corr_plane_bytes(n) > b) b = corr_plane_bytes(n);
  return b;
}

size_t screened_refine_bytes(int64_t n, int64_t chunk) {
  const int64_t n2 = n * n;
  return al256((size_t)chunk * n2 * sizeof(float2)) +            // F: complex64 matrix / correction
         al256(gj_work_bytes<float2>(n, chunk)) +                 // panels of the complex64 inversion
         al256((size_t)chunk * n2 * sizeof(double2)) +           // T: P~0 Y, then E
         al256((size_t)chunk * emul_digit_bytes(n, n)) +          // digits of P~0 (rows)
         al256((size_t)chunk * shared_plane_bytes(n)) +           // digits of Y / split planes
         2 * al256((size_t)chunk * n * sizeof(int));              // exponents
}

bool screened_refine_ok(int64_t n) { return n >= 1 && emul_launches(n) > 0; }

cudaError_t screened_refine(double2* X, int64_t n, int64_t count, void* work, size_t work_bytes, int nsteps,
                            int* d_info, int* d_err, cudaStream_t st, int64_t* nlaunch) {
  if (!screened_refine_ok(n)) return cudaErrorInvalidValue;
  // largest batch that fits, then balanced over the batches
  if (count <= 0) return cudaSuccess;
  if (screened_refine_bytes(n, 1) > work_bytes) return cudaErrorMemoryAllocation;
  int64_t lo = 1, hi = count < 65535 ? count : 65535;
  while (lo < hi) {
    const int64_t mid = (lo + hi + 1) / 2;
    if (screened_refine_bytes(n, mid) <= work_bytes) lo = mid; else hi = mid - 1;
  }
  const int64_t nchunks = (count + lo - 1) / lo;
  const int64_t chunk = (count + nchunks - 1) / nchunks;
  const int64_t n2 = n * n;
  constexpr int kLeadDigits = 5;   // digits of the product in every step but the last
  cudaError_t e;
  int64_t launches = 0;
  for (int64_t z0 = 0; z0 < count; z0 += chunk) {
    const int64_t cz = (count - z0) < chunk ? (count - z0) : chunk;
    const int64_t tot = cz * n2;
    double2* Xc = X + z0 * n2;
    char* p = (char*)work;
    float2* F = (float2*)p;  p += al256((size_t)chunk * n2 * sizeof(float2));
    void* pan = p;           p += al256(gj_work_bytes<float2>(n, chunk));
    double2* T = (double2*)p; p += al256((size_t)chunk * n2 * sizeof(double2));
    float* Ad = (float*)p;   p += al256((size_t)chunk * emul_digit_bytes(n, n));
    float* Bd = (float*)p;   p += al256((size_t)chunk * shared_plane_bytes(n));
    int* Ae = (int*)p;       p += al256((size_t)chunk * n * sizeof(int));
    int* Be = (int*)p;
    // digits of P~0 (kept for every step), then Y0 = complex64 inverse of I - P~0
    if ((e = emul_split_rows(Xc, cz, n, n, n, n2, Ad, Ae, st)) != cudaSuccess) return e;
    f_from_iminus_kernel<<<grid1(tot), 256, 0, st>>>(Xc, F, n, tot);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = gj_blocked_tc(F, n, cz, pan, Bd, d_info, d_err, st, &launches)) != cudaSuccess) return e;
    x_from_f_kernel<<<grid1(tot), 256, 0, st>>>(F, Xc, tot);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    launches += 3;
    for (int s = 0; s < nsteps; ++s) {
      if ((e = emul_split_cols(Xc, cz, n, n, n, n2, Bd, Be, st)) != cudaSuccess) return e;
      const int nd = s == nsteps - 1 ? 8 : kLeadDigits;
      if ((e = emul_cgemm_batched(Ad, Ae, Bd, Be, cz, n, n, n, T, d_err, st, nd)) != cudaSuccess) return e;
      resid_kernel<<<grid1(tot), 256, 0, st>>>(Xc, T, n, tot);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      // F = Y E  (split TF32 on the tensor cores, FP32 output: E is small)
      {
        const int64_t Kp = emul_kpad(n);
        float* Yh = Bd;
        float* Yl = Yh + cz * n * Kp;
        float* Eh = Yl + cz * n * Kp;
        float* El = Eh + cz * 2 * n * Kp;
        if ((e = split_rows(Xc, true, cz * n, n, n, false, Yh, Yl, Kp, st)) != cudaSuccess) return e;
        if ((e = embed_t_batched(T, true, cz, n, n, n, n2, Eh, El, Kp, 2 * n * Kp, st)) != cudaSuccess) return e;
        UmmaOperand a{Yh, Yl, n, cz, Kp, n * Kp}, b{Eh, El, 2 * n, cz, Kp, 2 * n * Kp};
        if ((e = umma_gemm(a, b, (int)n, (int)(2 * n), Kp, (int)cz, F, false, 1.0, false, 2 * n, 2 * n2, 3, d_err, st,
                           1, 0, 0, 0, 0, nullptr, nullptr, 2 * n)) != cudaSuccess)
          return e;
      }
      y_update_kernel<<<grid1(tot), 256, 0, st>>>(Xc, F, n, tot, s == nsteps - 1 ? 1 : 0);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      launches += 6 + emul_launches(n, nd);
    }
    if (nsteps == 0) {
      if ((e = identity_minus(Xc, n, cz, +1.0, st)) != cudaSuccess) return e;
      launches += 1;
    }
  }
  if (nlaunch) *nlaunch += launches;
  return cudaSuccess;
}
}  // namespace gwk

// ------------------------------------------------------------------ test hook
// X (count x n x n complex128, device, in place): P~0 -> P~ through the refined
// inversion with nsteps Newton steps and a workspace of work_bytes (so that tests can
// force several batches).  Returns 0, a CUDA error code, 1000 for a zero pivot, or
// 100 + role when a tensor-core wait gave up.
extern "C" int gwdbg_screened_refine(double2* X, int64_t n, int64_t count, int64_t work_bytes, int nsteps) {
  using namespace gwk;
  void* work = nullptr;
  int* flags = nullptr;
  if (cudaMalloc(&work, (size_t)work_bytes) || cudaMalloc(&flags, 8)) return -1;
  cudaMemset(flags, 0, 8);
  cudaError_t e = screened_refine(X, n, count, work, (size_t)work_bytes, nsteps, flags, flags + 1, 0, nullptr);
  if (!e) e = cudaDeviceSynchronize();
  int h[2] = {0, 0};
  cudaMemcpy(h, flags, 8, cudaMemcpyDeviceToHost);
  cudaFree(work); cudaFree(flags);
  return e ? (int)e : h[1] ? h[1] : h[0] ? 1000 : 0;
}
extern "C" int64_t gwdbg_screened_refine_bytes(int64_t n, int64_t chunk) { return (int64_t)gwk::screened_refine_bytes(n, chunk); }
