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
#include "gw_internal.cuh"
#include "gj.cuh"

namespace gwk {

__global__ void extract_kernel(const double2* __restrict__ X, int64_t n, int nb, int64_t kb, int64_t count,
                               double2* Cp, double2* Rp) {
  const int64_t per = 2 * n * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * count; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t z = e / per, r = e - z * per;
    const double2* Xz = X + z * n * n;
    if (r < n * nb) {          // column panel Cp[i][c] (rows of block b zeroed)
      int64_t i = r / nb, c = r - i * nb;
      Cp[z * n * nb + r] = (i >= kb && i < kb + nb) ? make_double2(0, 0) : Xz[i * n + kb + c];
    } else {                   // row panel Rp[c][j]
      r -= n * nb;
      int64_t c = r / n, j = r - c * n;
      Rp[z * n * nb + r] = Xz[(kb + c) * n + j];
    }
  }
}

__global__ void zero_cols_kernel(double2* X, int64_t n, int nb, int64_t kb, int64_t count) {
  const int64_t per = n * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * count; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t z = e / per, r = e - z * per, i = r / nb, c = r - i * nb;
    X[z * n * n + i * n + kb + c] = make_double2(0, 0);
  }
}

// Dinv[z] = (Rp[z][:, kb:kb+nb])^{-1}, one block per system, in shared memory.
__global__ void __launch_bounds__(256) block_inv_kernel(const double2* __restrict__ Rp, int64_t n, int nb, int64_t kb,
                                                        int64_t count, double2* Dinv, int* info) {
  extern __shared__ unsigned char smem[];
  double2* A = (double2*)smem;
  double2* f = A + nb * nb;
  int* perm = (int*)(f + nb);
  double* rv = (double*)(perm + nb + (nb & 1));
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
__global__ void put_dinv_kernel(double2* Rn, const double2* __restrict__ Dinv, int64_t n, int nb, int64_t kb, int64_t count) {
  const int64_t per = (int64_t)nb * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * count; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t z = e / per, r = (e - z * per) / nb, c = (e - z * per) % nb;
    Rn[z * n * nb + r * n + kb + c] = Dinv[e];
  }
}

// X[z][kb + r][j] = Rn[z][r][j]
__global__ void put_rows_kernel(double2* X, const double2* __restrict__ Rn, int64_t n, int nb, int64_t kb, int64_t count) {
  const int64_t per = n * nb;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < per * count; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t z = e / per, r = e - z * per;
    X[z * n * n + kb * n + r] = Rn[e];
  }
}

static const int NB = 64;

size_t screened_work_bytes(int64_t n, int64_t count) {
  int64_t nb = n < NB ? n : NB;
  return (size_t)count * (size_t)(3 * n * nb + nb * nb) * sizeof(double2);
}

static inline int grid1(int64_t work) {
  int64_t b = (work + 255) / 256;
  return (int)(b < 152 * 32 ? b : 152 * 32);
}

// In-place: X (count systems of n x n, contiguous) holds P~0 on entry and P~ on exit.
cudaError_t screened_inplace(double2* X, int64_t n, int64_t count, double2* work, size_t work_bytes,
                             int* d_info, cudaStream_t st) {
  cudaError_t e = identity_minus(X, n, count, -1.0, st);        // X <- I - P~0
  if (e != cudaSuccess) return e;
  const int64_t nbmax = n < NB ? n : NB;
  const size_t per_sys = (size_t)(3 * n * nbmax + nbmax * nbmax) * sizeof(double2);
  int64_t chunk = (int64_t)(work_bytes / per_sys);
  if (chunk <= 0) return cudaErrorMemoryAllocation;
  if (chunk > 65535) chunk = 65535;
  const int nt = 256;
  size_t sm = (size_t)nbmax * nbmax * sizeof(double2) + (size_t)nbmax * sizeof(double2) +
              (size_t)(nbmax + 1) * sizeof(int) + 8 + nt * (sizeof(double) + sizeof(int));
  if (sm > 48 * 1024) {
    e = cudaFuncSetAttribute(block_inv_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  for (int64_t z0 = 0; z0 < count; z0 += chunk) {
    const int64_t cz = (count - z0) < chunk ? (count - z0) : chunk;
    double2* Xc = X + z0 * n * n;
    double2* Cp = work;
    double2* Rp = Cp + cz * n * nbmax;
    double2* Rn = Rp + cz * n * nbmax;
    double2* Di = Rn + cz * n * nbmax;
    for (int64_t kb = 0; kb < n; kb += nbmax) {
      const int nb = (int)((n - kb) < nbmax ? (n - kb) : nbmax);
      extract_kernel<<<grid1(2 * n * nb * cz), 256, 0, st>>>(Xc, n, nb, kb, cz, Cp, Rp);
      zero_cols_kernel<<<grid1(n * nb * cz), 256, 0, st>>>(Xc, n, nb, kb, cz);
      block_inv_kernel<<<(int)(cz < 152 * 8 ? cz : 152 * 8), nt, sm, st>>>(Rp, n, nb, kb, cz, Di, d_info);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
      // Rn[z] = Dinv[z] (nb x nb) * Rp[z] (nb x n)
      GettDesc g{};
      g.M = nb; g.N = n; g.K = nb; g.Z = cz;
      g.am = I1(nb); g.ak = I1(1); g.az = I1((int64_t)nb * nb);
      g.bk = I1(n); g.bn = I1(1); g.bz = I1(n * nb);
      g.cm = I1(n); g.cn = I1(1); g.cz = I1(n * nb);
      g.alpha = make_double2(1, 0); g.beta = make_double2(0, 0); g.ksplit = 1;
      if ((e = gett(g, Di, Ty::C128, Rp, Ty::C128, Rn, Ty::C128, Ty::C128, nullptr, 0, st)) != cudaSuccess) return e;
      put_dinv_kernel<<<grid1((int64_t)nb * nb * cz), 256, 0, st>>>(Rn, Di, n, nb, kb, cz);
      // X[z] -= Cp[z] (n x nb) * Rn[z] (nb x n)
      GettDesc u{};
      u.M = n; u.N = n; u.K = nb; u.Z = cz;
      u.am = I1(nb); u.ak = I1(1); u.az = I1(n * nb);
      u.bk = I1(n); u.bn = I1(1); u.bz = I1(n * nb);
      u.cm = I1(n); u.cn = I1(1); u.cz = I1(n * n);
      u.alpha = make_double2(-1, 0); u.beta = make_double2(1, 0); u.ksplit = 1;
      if ((e = gett(u, Cp, Ty::C128, Rn, Ty::C128, Xc, Ty::C128, Ty::C128, nullptr, 0, st)) != cudaSuccess) return e;
      put_rows_kernel<<<grid1(n * nb * cz), 256, 0, st>>>(Xc, Rn, n, nb, kb, cz);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  return identity_minus(X, n, count, +1.0, st);                 // X <- (I - P~0)^{-1} - I
}

}  // namespace gwk
