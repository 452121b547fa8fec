// Operand preparation for the split-TF32 tensor-core GEMM (k_umma.cu): complex
// matrices become real K-major rows (the complex product as a real GEMM on
// embedded operands) split into TF32 high and low planes, hi = rna(x) and
// lo = rna(x - hi), zero-padded to a multiple of 32 floats.
#include "gw_internal.cuh"

namespace gwk {

__device__ __forceinline__ float tf32_rna(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}
__device__ __forceinline__ void split2(double x, float& hi, float& lo) {
  hi = tf32_rna((float)x);
  lo = tf32_rna((float)(x - (double)hi));
}

// Rows of a complex matrix (element (r, k) at src + r*ld + k, complex units) into
// real hi/lo rows of length Kpad (zero padded): out[r][2k + s] = (re, +-im).
template <typename T>
__global__ void split_rows_kernel(const T* __restrict__ src, int64_t rows, int64_t K, int64_t ld, int conj,
                                  float* hi, float* lo, int64_t Kpad) {
  const int64_t tot = rows * Kpad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r = e / Kpad, c = e - r * Kpad;
    double v = 0.0;
    if (c < 2 * K) {
      const T x = src[r * ld + (c >> 1)];
      v = (c & 1) ? (conj ? -(double)x.y : (double)x.y) : (double)x.x;
    }
    float h, l;
    split2(v, h, l);
    hi[e] = h;
    if (lo) lo[e] = l;
  }
}

// Doubled operand of C = A conj(B)^T from B (rows n, complex K): rows 2n = (re, im),
// rows 2n+1 = (-im, re).
template <typename T>
__global__ void embed_conj_kernel(const T* __restrict__ src, int64_t rows, int64_t K, float* hi, float* lo,
                                  int64_t Kpad) {
  const int64_t tot = 2 * rows * Kpad;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t r2 = e / Kpad, c = e - r2 * Kpad, n = r2 >> 1;
    double v = 0.0;
    if (c < 2 * K) {
      const T x = src[n * K + (c >> 1)];
      if ((r2 & 1) == 0) v = (c & 1) ? (double)x.y : (double)x.x;
      else v = (c & 1) ? (double)x.x : -(double)x.y;
    }
    float h, l;
    split2(v, h, l);
    hi[e] = h;
    if (lo) lo[e] = l;
  }
}

// Batched embed_conj: `count` matrices of `rows` x K complex (src stride `ss` complex
// elements) into `count` doubled operands of 2*rows x Kpad floats (dst stride `ds`).
__global__ void embed_conj_batched_kernel(const double2* __restrict__ src, int64_t count, int64_t ss, int64_t rows,
                                          int64_t K, float* hi, float* lo, int64_t Kpad, int64_t ds) {
  const int64_t per = 2 * rows * Kpad, tot = per * count;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = e / per, r = e - z * per, r2 = r / Kpad, c = r - r2 * Kpad, n = r2 >> 1;
    double v = 0.0;
    if (c < 2 * K) {
      const double2 x = src[z * ss + n * K + (c >> 1)];
      if ((r2 & 1) == 0) v = (c & 1) ? x.y : x.x;
      else v = (c & 1) ? x.x : -x.y;
    }
    float h, l;
    split2(v, h, l);
    hi[z * ds + r] = h;
    lo[z * ds + r] = l;
  }
}

// Batched doubled operand of C = A B^T with B[n][k] = src[z][n][k] taken as is:
// rows 2n = (re, -im), rows 2n+1 = (im, re).  Matrix z is read at src + z*ss
// (complex elements; ss may be negative to walk a tau axis backwards).
__global__ void embed_plain_batched_kernel(const double2* __restrict__ src, int64_t count, int64_t ss, int64_t rows,
                                           int64_t K, float* hi, float* lo, int64_t Kpad, int64_t ds) {
  const int64_t per = 2 * rows * Kpad, tot = per * count;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t z = e / per, r = e - z * per, r2 = r / Kpad, c = r - r2 * Kpad, n = r2 >> 1;
    double v = 0.0;
    if (c < 2 * K) {
      const double2 x = src[z * ss + n * K + (c >> 1)];
      if ((r2 & 1) == 0) v = (c & 1) ? -x.y : x.x;
      else v = (c & 1) ? x.x : x.y;
    }
    float h, l;
    split2(v, h, l);
    hi[z * ds + r] = h;
    lo[z * ds + r] = l;
  }
}

// Doubled operand of C = A B^T where B[n][k] = src[z][k][n] (src: count matrices of
// K rows of N complex, row stride ld, matrix stride zs): rows 2n = (re, -im), rows
// 2n+1 = (im, re) of Kpad floats (operand stride ds per matrix), transposed through
// shared memory.  Grid: (N/32, K/32, count).
template <typename T>
__global__ void embed_t_kernel(const T* __restrict__ src, int64_t K, int64_t N, int64_t ld, int64_t zs, float* hi,
                               float* lo, int64_t Kpad, int64_t ds) {
  __shared__ double2 tile[32][33];
  const int64_t k0 = blockIdx.y * 32, nb = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  src += (int64_t)blockIdx.z * zs;
  hi += (int64_t)blockIdx.z * ds;
  if (lo) lo += (int64_t)blockIdx.z * ds;
  for (int r = ty; r < 32; r += 8) {
    const int64_t k = k0 + r, n = nb + tx;
    double2 v = make_double2(0, 0);
    if (k < K && n < N) { T x = src[k * ld + n]; v = make_double2((double)x.x, (double)x.y); }
    tile[r][tx] = v;
  }
  __syncthreads();
  // write rows 2n, 2n+1 for n in block, columns 2k, 2k+1 for k in block
  for (int r = ty; r < 32; r += 8) {
    const int64_t n = nb + r;
    if (n >= N) continue;
    const int64_t k = k0 + tx;
    const double2 v = tile[tx][r];
    float h, l;
    if (k < K) {
      float* h0 = hi + (2 * n) * Kpad + 2 * k;
      float* h1 = hi + (2 * n + 1) * Kpad + 2 * k;
      split2(v.x, h, l); h0[0] = h; if (lo) lo[(2 * n) * Kpad + 2 * k] = l;
      split2(-v.y, h, l); h0[1] = h; if (lo) lo[(2 * n) * Kpad + 2 * k + 1] = l;
      split2(v.y, h, l); h1[0] = h; if (lo) lo[(2 * n + 1) * Kpad + 2 * k] = l;
      split2(v.x, h, l); h1[1] = h; if (lo) lo[(2 * n + 1) * Kpad + 2 * k + 1] = l;
    }
  }
  // zero padding columns [2K, Kpad) once, by the first column of blocks
  if (blockIdx.y == 0) {
    for (int r = ty; r < 32; r += 8) {
      const int64_t n = nb + r;
      if (n >= N) continue;
      for (int64_t c = 2 * K + tx; c < Kpad; c += 32) {
        hi[(2 * n) * Kpad + c] = 0.f; hi[(2 * n + 1) * Kpad + c] = 0.f;
        if (lo) { lo[(2 * n) * Kpad + c] = 0.f; lo[(2 * n + 1) * Kpad + c] = 0.f; }
      }
    }
  }
}

static inline int nb_(int64_t n) { int64_t b = (n + 255) / 256; return (int)(b < 152 * 16 ? b : 152 * 16); }

cudaError_t split_rows(const void* src, bool src_c128, int64_t rows, int64_t K, int64_t ld, bool conj, float* hi,
                       float* lo, int64_t Kpad, cudaStream_t st) {
  if (src_c128) split_rows_kernel<double2><<<nb_(rows * Kpad), 256, 0, st>>>((const double2*)src, rows, K, ld, conj, hi, lo, Kpad);
  else split_rows_kernel<float2><<<nb_(rows * Kpad), 256, 0, st>>>((const float2*)src, rows, K, ld, conj, hi, lo, Kpad);
  return cudaGetLastError();
}
cudaError_t embed_conj(const void* src, bool src_c128, int64_t rows, int64_t K, float* hi, float* lo, int64_t Kpad,
                       cudaStream_t st) {
  if (src_c128) embed_conj_kernel<double2><<<nb_(2 * rows * Kpad), 256, 0, st>>>((const double2*)src, rows, K, hi, lo, Kpad);
  else embed_conj_kernel<float2><<<nb_(2 * rows * Kpad), 256, 0, st>>>((const float2*)src, rows, K, hi, lo, Kpad);
  return cudaGetLastError();
}
cudaError_t embed_conj_batched(const double2* src, int64_t count, int64_t ss, int64_t rows, int64_t K, float* hi,
                               float* lo, int64_t Kpad, int64_t ds, cudaStream_t st) {
  embed_conj_batched_kernel<<<nb_(2 * rows * Kpad * count), 256, 0, st>>>(src, count, ss, rows, K, hi, lo, Kpad, ds);
  return cudaGetLastError();
}

cudaError_t embed_plain_batched(const double2* src, int64_t count, int64_t ss, int64_t rows, int64_t K, float* hi,
                                float* lo, int64_t Kpad, int64_t ds, cudaStream_t st) {
  embed_plain_batched_kernel<<<nb_(2 * rows * Kpad * count), 256, 0, st>>>(src, count, ss, rows, K, hi, lo, Kpad, ds);
  return cudaGetLastError();
}

cudaError_t embed_t(const void* src, bool src_c128, int64_t K, int64_t N, float* hi, float* lo, int64_t Kpad,
                    cudaStream_t st) {
  return embed_t_batched(src, src_c128, 1, K, N, N, 0, hi, lo, Kpad, 0, st);
}

cudaError_t embed_t_batched(const void* src, bool src_c128, int64_t count, int64_t K, int64_t N, int64_t ld,
                            int64_t zs, float* hi, float* lo, int64_t Kpad, int64_t ds, cudaStream_t st) {
  if (count < 1 || count > 65535) return cudaErrorInvalidValue;
  dim3 grid((unsigned)((N + 31) / 32), (unsigned)((K + 31) / 32), (unsigned)count);
  if (src_c128) embed_t_kernel<double2><<<grid, 256, 0, st>>>((const double2*)src, K, N, ld, zs, hi, lo, Kpad, ds);
  else embed_t_kernel<float2><<<grid, 256, 0, st>>>((const float2*)src, K, N, ld, zs, hi, lo, Kpad, ds);
  return cudaGetLastError();
}

}  // namespace gwk
