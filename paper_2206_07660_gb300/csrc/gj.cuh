// In-place Gauss-Jordan inversion with partial pivoting of one n x n complex
// matrix held in shared memory, executed by a whole thread block.
#pragma once
#include <cuda_runtime.h>

namespace gwk {

template <typename T> struct gj_real;
template <> struct gj_real<double2> { using t = double; };
template <> struct gj_real<float2> { using t = float; };

template <typename T>
static __device__ __forceinline__ T cmul(T a, T b) {
  T r; r.x = a.x * b.x - a.y * b.y; r.y = a.x * b.y + a.y * b.x; return r;
}
template <typename T>
static __device__ __forceinline__ T cinv(T a) {
  const auto d = a.x * a.x + a.y * a.y;
  T r; r.x = a.x / d; r.y = -a.y / d; return r;
}
template <typename T>
static __device__ __forceinline__ T cval(double re, double im) {
  T r; r.x = (decltype(r.x))re; r.y = (decltype(r.y))im; return r;
}

// A: n x n row-major with leading dimension lda (shared memory), complex T
// (double2 or float2, arithmetic in T's precision).
// f: n complex scratch, perm: n ints, red_v/red_i: blockDim.x scratch.
// Returns (in every thread) 1 if a zero pivot was met, else 0.
template <typename T>
static __device__ int gj_invert_smem(T* A, int n, int lda, T* f, int* perm, typename gj_real<T>::t* red_v,
                                     int* red_i) {
  using R = typename gj_real<T>::t;
  const int tid = threadIdx.x, nt = blockDim.x;
  __shared__ int s_bad;
  if (tid == 0) s_bad = 0;
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    // pivot: argmax_{r >= c} |A[r][c]| (ties -> smallest r)
    R bv = -1; int bi = c;
    for (int r = c + tid; r < n; r += nt) {
      T v = A[r * lda + c];
      R m = v.x * v.x + v.y * v.y;
      if (m > bv) { bv = m; bi = r; }
    }
    red_v[tid] = bv; red_i[tid] = bi;
    __syncthreads();
    for (int s = nt / 2; s > 0; s >>= 1) {
      if (tid < s) {
        R ov = red_v[tid + s]; int oi = red_i[tid + s];
        if (ov > red_v[tid] || (ov == red_v[tid] && oi < red_i[tid])) { red_v[tid] = ov; red_i[tid] = oi; }
      }
      __syncthreads();
    }
    const int p = red_i[0];
    const bool zero = !(red_v[0] > (R)0);
    __syncthreads();
    if (tid == 0) { perm[c] = p; if (zero) s_bad = 1; }
    if (p != c)
      for (int j = tid; j < n; j += nt) {
        T t = A[p * lda + j]; A[p * lda + j] = A[c * lda + j]; A[c * lda + j] = t;
      }
    __syncthreads();
    T piv = A[c * lda + c];
    T ip = zero ? cval<T>(0.0, 0.0) : cinv(piv);
    __syncthreads();
    for (int j = tid; j < n; j += nt) {
      T v = (j == c) ? cval<T>(1.0, 0.0) : A[c * lda + j];
      A[c * lda + j] = cmul(v, ip);
    }
    for (int r = tid; r < n; r += nt) {
      f[r] = (r == c) ? cval<T>(0.0, 0.0) : A[r * lda + c];
    }
    __syncthreads();
    for (int e = tid; e < n * n; e += nt) {
      int r = e / n, j = e - r * n;
      if (r == c) continue;
      T fr = f[r];
      T cj = A[c * lda + j];
      T v = (j == c) ? cval<T>(0.0, 0.0) : A[r * lda + j];
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
        T t = A[r * lda + p]; A[r * lda + p] = A[r * lda + c]; A[r * lda + c] = t;
      }
    __syncthreads();
  }
  int bad = s_bad;
  __syncthreads();
  return bad;
}

}  // namespace gwk
