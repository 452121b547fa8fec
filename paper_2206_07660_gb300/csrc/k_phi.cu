// Trace-log of I - P~0(i Omega) for the dynamical part of the GW Luttinger-Ward
// functional (Eq. tilde_Phi_GW): for each matrix A = P~0^q(i Omega_m),
//
//   f = tr ln(I - A) + tr A = sum_j ln u_jj + tr A,
//
// with u_jj the pivots of an LU factorisation of I - A without row exchanges.
// A polarization whose Hermitian part is negative semidefinite makes the
// Hermitian part of I - A positive definite; then elimination without pivoting
// is stable, every pivot lies in the right half-plane, and the sum of the
// principal logarithms of the pivots is the branch of ln det(I - A) that is
// continuous from A = 0 (the sum of the principal logarithms of the
// eigenvalues).  A pivot with non-positive real part is reported instead.
//
// One block per matrix, FP64 throughout.  Blocked right-looking elimination:
// a panel of PB columns (rows r0..n-1) and the PB x (n - r0 - PB) block row to
// its right are staged in shared memory, factored there, and the trailing
// matrix receives one rank-PB update in global memory (each element read and
// written once per panel).  Only the pivots are kept: L and U are not stored.
#include "gw_internal.cuh"

namespace gwk {

constexpr int PHI_THREADS = 256;
constexpr size_t PHI_SMEM_CAP = 200 * 1024;

__device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

__device__ __forceinline__ double2 cdiv(double2 a, double2 b) {
  const double s = 1.0 / (b.x * b.x + b.y * b.y);
  return make_double2((a.x * b.x + a.y * b.y) * s, (a.y * b.x - a.x * b.y) * s);
}

// A[mat] (n x n, row stride n, matrices `stride` apart) holds P~0(i Omega) on entry and
// is overwritten.  out[mat] = tr ln(I - A) + tr A.  flag: |= 1 for a zero or non-finite
// pivot, |= 2 for a pivot with non-positive real part.
__global__ void __launch_bounds__(PHI_THREADS) lu_tracelog_kernel(double2* A, int n, int64_t stride, int64_t count,
                                                                  int pb, double2* out, int* flag) {
  extern __shared__ double2 sh[];
  double2* P = sh;                         // panel: (n - r0) rows x pb, row-major
  double2* U = sh + (size_t)n * pb;        // block row: pb rows x (n - r0 - pb)
  __shared__ double red_re[PHI_THREADS / 32], red_im[PHI_THREADS / 32];
  __shared__ int s_bad;
  const int tid = threadIdx.x;
  for (int64_t mat = blockIdx.x; mat < count; mat += gridDim.x) {
    double2* M = A + mat * stride;
    // I - A in place, and tr A
    double tre = 0.0, tim = 0.0;
    for (int64_t e = tid; e < (int64_t)n * n; e += PHI_THREADS) {
      const int i = (int)(e / n), j = (int)(e - (int64_t)i * n);
      double2 v = M[e];
      if (i == j) { tre += v.x; tim += v.y; v = make_double2(1.0 - v.x, -v.y); }
      else v = make_double2(-v.x, -v.y);
      M[e] = v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      tre += __shfl_xor_sync(0xffffffffu, tre, o);
      tim += __shfl_xor_sync(0xffffffffu, tim, o);
    }
    if ((tid & 31) == 0) { red_re[tid >> 5] = tre; red_im[tid >> 5] = tim; }
    if (tid == 0) s_bad = 0;
    __syncthreads();
    double lre = 0.0, lim = 0.0;          // sum of ln u_jj (thread 0)
    for (int r0 = 0; r0 < n; r0 += pb) {
      const int w = min(pb, n - r0);      // panel width
      const int r1 = r0 + w, nr = n - r0, nc = n - r1;
      for (int e = tid; e < nr * w; e += PHI_THREADS) {
        const int i = e / w, k = e - i * w;
        P[i * pb + k] = M[(int64_t)(r0 + i) * n + r0 + k];
      }
      for (int e = tid; e < w * nc; e += PHI_THREADS) {
        const int k = e / nc, cc = e - k * nc;
        U[k * nc + cc] = M[(int64_t)(r0 + k) * n + r1 + cc];
      }
      __syncthreads();
      for (int j = 0; j < w; ++j) {
        const double2 piv = P[j * pb + j];
        const double mag = hypot(piv.x, piv.y);
        if (tid == 0) {
          if (!(mag > 0.0) || !isfinite(mag)) s_bad |= 1;
          else if (!(piv.x > 0.0)) s_bad |= 2;
          lre += log(mag);
          lim += atan2(piv.y, piv.x);
        }
        // rows below the pivot: multipliers and the panel's remaining columns
        if (mag > 0.0) {
          for (int i = j + 1 + tid; i < nr; i += PHI_THREADS) {
            const double2 l = cdiv(P[i * pb + j], piv);
            P[i * pb + j] = l;
            for (int k = j + 1; k < w; ++k) {
              const double2 t = cmul(l, P[j * pb + k]);
              P[i * pb + k] = make_double2(P[i * pb + k].x - t.x, P[i * pb + k].y - t.y);
            }
          }
        }
        __syncthreads();
        // forward substitution of the block row with the unit lower triangle
        for (int e = tid; e < (w - j - 1) * nc; e += PHI_THREADS) {
          const int k = j + 1 + e / nc, cc = e - (k - j - 1) * nc;
          const double2 t = cmul(P[k * pb + j], U[j * nc + cc]);
          U[k * nc + cc] = make_double2(U[k * nc + cc].x - t.x, U[k * nc + cc].y - t.y);
        }
        __syncthreads();
      }
      // trailing update: M[i][c] -= sum_k L21[i][k] U12[k][c] for i, c >= r1
      for (int64_t e = tid; e < (int64_t)nc * nc; e += PHI_THREADS) {
        const int i = (int)(e / nc), cc = (int)(e - (int64_t)i * nc);
        const double2* li = P + (size_t)(i + w) * pb;
        double2 s = M[(int64_t)(r1 + i) * n + r1 + cc];
        for (int k = 0; k < w; ++k) {
          const double2 t = cmul(li[k], U[k * nc + cc]);
          s.x -= t.x; s.y -= t.y;
        }
        M[(int64_t)(r1 + i) * n + r1 + cc] = s;
      }
      __syncthreads();
    }
    if (tid == 0) {
      double sre = 0.0, sim = 0.0;
      for (int wv = 0; wv < PHI_THREADS / 32; ++wv) { sre += red_re[wv]; sim += red_im[wv]; }
      out[mat] = make_double2(lre + sre, lim + sim);
      if (s_bad) atomicOr(flag, s_bad);
    }
    __syncthreads();
  }
}

int tracelog_panel(int n) {
  int pb = 16;
  while (pb > 1 && (size_t)2 * n * pb * sizeof(double2) > PHI_SMEM_CAP) pb >>= 1;
  return (size_t)2 * n * pb * sizeof(double2) <= PHI_SMEM_CAP ? pb : 0;
}

cudaError_t lu_tracelog(double2* A, int n, int64_t count, int64_t stride, double2* out, int* flag, cudaStream_t st) {
  if (n <= 0 || count <= 0) return cudaSuccess;
  const int pb = tracelog_panel(n);
  if (pb == 0) return cudaErrorInvalidValue;
  const size_t smem = (size_t)2 * n * pb * sizeof(double2);
  cudaError_t e = cudaFuncSetAttribute(lu_tracelog_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int64_t blocks = count < 152 * 8 ? count : 152 * 8;
  lu_tracelog_kernel<<<(unsigned)blocks, PHI_THREADS, smem, st>>>(A, n, stride, count, pb, out, flag);
  return cudaGetLastError();
}

}  // namespace gwk
