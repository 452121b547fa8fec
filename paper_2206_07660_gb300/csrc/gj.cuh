// In-place Gauss-Jordan inversion with partial pivoting of one n x n complex
// matrix held in shared memory, executed by a whole thread block.
#pragma once
#include <cuda_runtime.h>

namespace gwk {

static __device__ __forceinline__ double2 cmul(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
static __device__ __forceinline__ double2 cinv(double2 a) {
  double d = a.x * a.x + a.y * a.y;
  return make_double2(a.x / d, -a.y / d);
}

// A: n x n row-major with leading dimension lda (shared memory).
// f: n complex scratch, perm: n ints, red_v/red_i: blockDim.x scratch.
// Returns (in every thread) 1 if a zero pivot was met, else 0.
static __device__ int gj_invert_smem(double2* A, int n, int lda, double2* f, int* perm, double* red_v, int* red_i) {
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    // pivot: argmax_{r >= c} |A[r][c]| (ties -> smallest r)
    double bv = -1.0; int bi = c;
    for (int r = c + tid; r < n; r += nt) {
      double2 v = A[r * lda + c];
      double m = v.x * v.x + v.y * v.y;
      if (m > bv) { bv = m; bi = r; }
    }
    red_v[tid] = bv; red_i[tid] = bi;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
      if (tid < s) {
        double ov = red_v[tid + s]; int oi = red_i[tid + s];
        if (ov > red_v[tid] || (ov == red_v[tid] && oi < red_i[tid])) { red_v[tid] = ov; red_i[tid] = oi; }
      }
      __syncthreads();
    }
    const int p = red_i[0];
    const bool zero = !(red_v[0] > 0.0);
    __syncthreads();
    if (tid == 0) { perm[c] = p; if (zero) s_bad = 1; }
    if (p != c)
      for (int j = tid; j < n; j += nt) {
        double2 t = A[p * lda + j]; A[p * lda + j] = A[c * lda + j]; A[c * lda + j] = t;
      }
    __syncthreads();
    double2 piv = A[c * lda + c];
    double2 ip = zero ? make_double2(0.0, 0.0) : cinv(piv);
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      double2 v = (j == c) ? make_double2(1.0, 0.0) : A[c * lda + j];
      A[c * lda + j] = cmul(v, ip);
    }
    for (int r = tid; r < n; r += nt) {
      f[r] = (r == c) ? make_double2(0.0, 0.0) : A[r * lda + c];
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {
      int r = e / n, j = e - r * n;
      if (r == c) continue;
      double2 fr = f[r];
      double2 cj = A[c * lda + j];
      double2 v = (j == c) ? make_double2(0.0, 0.0) : A[r * lda + j];
      v.x -= fr.x * cj.x - fr.y * cj.y;
      v.y -= fr.x * cj.y + fr.y * cj.x;
      A[r * lda + j] = v;
    }
    __syncthreads();
  }
  // undo the row interchanges as column interchanges, last first
  for (int c = n - 1; c >= 0; --c) {
    int p = perm[c];
    if (p != c)
      for (int r = tid; r < n; r += nt) {
        double2 t = A[r * lda + p]; A[r * lda + p] = A[r * lda + c]; A[r * lda + c] = t;
      }
    __syncthreads();
  }
  int bad = s_bad;
  __syncthreads();
  return bad;
}

}  // namespace gwk
