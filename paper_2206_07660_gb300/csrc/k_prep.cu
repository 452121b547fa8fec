// Operand preparation for the split tensor-core GEMM (k_umma.cu): complex matrices
// become real K-major rows (the complex product as a real GEMM on embedded
// operands) split into high and low planes, zero-padded to whole 128-byte k-blocks.
// TF32 pieces: hi = rna(x), lo = rna(x - hi).  fp16 pieces: each row is stored with
// a power-of-two scale 2^e (max |x| 2^-e < 2^15), hi = rn16(x 2^-e), lo =
// rn16(x 2^-e - hi), and e goes into the row's exponent entry; the GEMM's epilogue
// multiplies by 2^(eA + eB).
#include <cuda_fp16.h>
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
// real hi/lo rows of length Kpad (zero padded) at row stride ldo: out[r][2k + s] =
// (re, +-im).
template <typename T>
__global__ void split_rows_kernel(const T* __restrict__ src, int64_t rows, int64_t K, int64_t ld, int conj,
                                  float* hi, float* lo, int64_t Kpad, int64_t ldo) {
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
    hi[r * ldo + c] = h;
    if (lo) lo[r * ldo + c] = l;
  }
}

// Doubled operand of C = A conj(B)^T from B (rows n, complex K): rows 2n = (re, im),
// rows 2n+1 = (-im, re), Kpad floats each at row stride ldo.
template <typename T>
__global__ void embed_conj_kernel(const T* __restrict__ src, int64_t rows, int64_t K, float* hi, float* lo,
                                  int64_t Kpad, int64_t ldo) {
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
    hi[r2 * ldo + c] = h;
    if (lo) lo[r2 * ldo + c] = l;
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
                       float* lo, int64_t Kpad, cudaStream_t st, int64_t ldo) {
  if (ldo <= 0) ldo = Kpad;
  if (src_c128)
    split_rows_kernel<double2><<<nb_(rows * Kpad), 256, 0, st>>>((const double2*)src, rows, K, ld, conj, hi, lo, Kpad, ldo);
  else
    split_rows_kernel<float2><<<nb_(rows * Kpad), 256, 0, st>>>((const float2*)src, rows, K, ld, conj, hi, lo, Kpad, ldo);
  return cudaGetLastError();
}
cudaError_t embed_conj(const void* src, bool src_c128, int64_t rows, int64_t K, float* hi, float* lo, int64_t Kpad,
                       cudaStream_t st, int64_t ldo) {
  if (ldo <= 0) ldo = Kpad;
  if (src_c128)
    embed_conj_kernel<double2><<<nb_(2 * rows * Kpad), 256, 0, st>>>((const double2*)src, rows, K, hi, lo, Kpad, ldo);
  else
    embed_conj_kernel<float2><<<nb_(2 * rows * Kpad), 256, 0, st>>>((const float2*)src, rows, K, hi, lo, Kpad, ldo);
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

// ------------------------------------------------------------------ fp16 pieces

// exponent e of a row with max |x| = m: m 2^-e < 2^15 (m = f 2^E, f in [0.5, 1))
__device__ __forceinline__ int f16_row_exp(double m) {
  int E = 0;
  if (m > 0.0) frexp(m, &E);
  return E - 15;
}
__device__ __forceinline__ void f16split(double x, int e, __half& h, __half& l) {
  const double d = ldexp(x, -e);
  h = __double2half(d);
  l = __double2half(d - (double)__half2float(h));
}
__device__ __forceinline__ double warp_max(double m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}

// Rows of a complex matrix (element (r, k) at src + r*ld + k) as real rows
// (re, +-im) of Kpad fp16 pieces with one exponent per row; one warp per row.
template <typename T>
__global__ void __launch_bounds__(256) split_rows_f16_kernel(const T* __restrict__ src, int64_t rows, int64_t K,
                                                             int64_t ld, int conj, __half* hi, __half* lo,
                                                             int64_t Kpad, int* ex) {
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= rows) return;
  const T* x = src + r * ld;
  double m = 0.0;
  for (int64_t k = lane; k < K; k += 32) {
    const T v = x[k];
    m = fmax(m, fmax(fabs((double)v.x), fabs((double)v.y)));
  }
  const int e = f16_row_exp(warp_max(m));
  if (lane == 0) ex[r] = e;
  __half2* h2 = (__half2*)(hi + r * Kpad);
  __half2* l2 = (__half2*)(lo + r * Kpad);
  for (int64_t c = lane; 2 * c < Kpad; c += 32) {
    double re = 0.0, im = 0.0;
    if (c < K) {
      const T v = x[c];
      re = (double)v.x;
      im = conj ? -(double)v.y : (double)v.y;
    }
    __half hr, lr, hm, lm;
    f16split(re, e, hr, lr);
    f16split(im, e, hm, lm);
    h2[c] = __halves2half2(hr, hm);
    l2[c] = __halves2half2(lr, lm);
  }
}

// Doubled operand of C = A conj(B)^T from complex rows n of B (K entries): real rows
// 2n = (re, im), 2n+1 = (-im, re) of fp16 pieces, one exponent per complex row n;
// one warp per complex row.
template <typename T>
__global__ void __launch_bounds__(256) embed_conj_f16_kernel(const T* __restrict__ src, int64_t rows, int64_t K,
                                                             __half* hi, __half* lo, int64_t Kpad, int* ex) {
  const int lane = threadIdx.x & 31;
  const int64_t n = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (n >= rows) return;
  const T* x = src + n * K;
  double m = 0.0;
  for (int64_t k = lane; k < K; k += 32) {
    const T v = x[k];
    m = fmax(m, fmax(fabs((double)v.x), fabs((double)v.y)));
  }
  const int e = f16_row_exp(warp_max(m));
  if (lane == 0) ex[n] = e;
  __half2* h0 = (__half2*)(hi + 2 * n * Kpad);
  __half2* l0 = (__half2*)(lo + 2 * n * Kpad);
  __half2* h1 = (__half2*)(hi + (2 * n + 1) * Kpad);
  __half2* l1 = (__half2*)(lo + (2 * n + 1) * Kpad);
  for (int64_t c = lane; 2 * c < Kpad; c += 32) {
    double re = 0.0, im = 0.0;
    if (c < K) {
      const T v = x[c];
      re = (double)v.x;
      im = (double)v.y;
    }
    __half hr, lr, hi_, li, hn, ln;
    f16split(re, e, hr, lr);
    f16split(im, e, hi_, li);
    f16split(-im, e, hn, ln);
    h0[c] = __halves2half2(hr, hi_);
    l0[c] = __halves2half2(lr, li);
    h1[c] = __halves2half2(hn, hr);
    l1[c] = __halves2half2(ln, lr);
  }
}

cudaError_t split_rows_f16(const void* src, bool src_c128, int64_t rows, int64_t K, int64_t ld, bool conj, void* hi,
                           void* lo, int64_t Kpad, int* ex, cudaStream_t st) {
  const int64_t nb = (rows + 7) / 8;
  if (Kpad % 64 || nb > INT32_MAX) return cudaErrorInvalidValue;
  if (src_c128)
    split_rows_f16_kernel<double2><<<(unsigned)nb, 256, 0, st>>>((const double2*)src, rows, K, ld, conj ? 1 : 0,
                                                                 (__half*)hi, (__half*)lo, Kpad, ex);
  else
    split_rows_f16_kernel<float2><<<(unsigned)nb, 256, 0, st>>>((const float2*)src, rows, K, ld, conj ? 1 : 0,
                                                                (__half*)hi, (__half*)lo, Kpad, ex);
  return cudaGetLastError();
}

cudaError_t embed_conj_f16(const void* src, bool src_c128, int64_t rows, int64_t K, void* hi, void* lo, int64_t Kpad,
                           int* ex, cudaStream_t st) {
  const int64_t nb = (rows + 7) / 8;
  if (Kpad % 64 || nb > INT32_MAX) return cudaErrorInvalidValue;
  if (src_c128)
    embed_conj_f16_kernel<double2><<<(unsigned)nb, 256, 0, st>>>((const double2*)src, rows, K, (__half*)hi,
                                                                 (__half*)lo, Kpad, ex);
  else
    embed_conj_f16_kernel<float2><<<(unsigned)nb, 256, 0, st>>>((const float2*)src, rows, K, (__half*)hi,
                                                                (__half*)lo, Kpad, ex);
  return cudaGetLastError();
}

}  // namespace gwk

// ------------------------------------------------------------------ test hooks
// C (M x N complex128, row-major) = A (M x K) conj(B)^T (B: N x K), complex128 device
// pointers, through fp16 pieces with row scales (three products).  Allocates its
// scratch; returns 0, a CUDA error code or 100 + role (a tensor-core wait gave up).
extern "C" int gwdbg_umma_cgemm_f16(const double2* A, const double2* B, int M, int N, int K, double* C) {
  using namespace gwk;
  const int64_t Kpad = (2 * (int64_t)K + 63) / 64 * 64;
  void *ah, *al, *bh, *bl;
  int *ea, *eb, *err;
  const size_t asz = (size_t)M * Kpad * 2, bsz = (size_t)2 * N * Kpad * 2;
  if (cudaMalloc(&ah, asz) || cudaMalloc(&al, asz) || cudaMalloc(&bh, bsz) || cudaMalloc(&bl, bsz) ||
      cudaMalloc(&ea, (size_t)M * 4) || cudaMalloc(&eb, (size_t)N * 4) || cudaMalloc(&err, 4))
    return -1;
  cudaMemset(err, 0, 4);
  cudaError_t e = split_rows_f16(A, true, M, K, K, false, ah, al, Kpad, ea, 0);
  if (!e) e = embed_conj_f16(B, true, N, K, bh, bl, Kpad, eb, 0);
  UmmaOperand oa{(const float*)ah, (const float*)al, M, 1, Kpad, 0, 1};
  UmmaOperand ob{(const float*)bh, (const float*)bl, 2 * (int64_t)N, 1, Kpad, 0, 1};
  UmmaScale sc{ea, eb, 0, 0, 0};
  if (!e) e = umma_gemm(oa, ob, M, 2 * N, Kpad, 1, C, true, 1.0, false, 2 * N, 0, 3, err, 0, 1, 0, 0, 0, 0, nullptr,
                        &sc, 2 * (int64_t)K);
  int herr = 0;
  if (!e) e = cudaDeviceSynchronize();
  cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
  cudaFree(ah); cudaFree(al); cudaFree(bh); cudaFree(bl); cudaFree(ea); cudaFree(eb); cudaFree(err);
  return e ? (int)e : herr;
}

__global__ void gwdbg_fill_half_kernel(__half* x, int64_t n, uint32_t seed) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    uint32_t h = (uint32_t)e * 2654435761u ^ seed;
    h ^= h >> 15; h *= 2246822519u; h ^= h >> 13; h *= 3266489917u; h ^= h >> 16;
    x[e] = __float2half((float)(h >> 8) * (1.0f / 8388608.0f) - 1.0f);
  }
}

// Timing of the fp16-piece GEMM on pseudo-random operands (zero row exponents):
// C[z] (M x N real) (+)= A[z] (M x Kpad) B (N x Kpad)^T, three products; fp64 output
// accumulates, fp32 output is stored.  *ms: mean device milliseconds per launch.
extern "C" int gwdbg_umma_bench_f16(int M, int N, int Kpad, int batch, int c_fp64, int iters, double* ms) {
  using namespace gwk;
  void *ah, *bh, *C;
  int *ez, *err;
  const size_t asz = (size_t)M * Kpad * 2 * batch, bsz = (size_t)N * Kpad * 2;
  const int emax = M > N ? M : N;
  if (cudaMalloc(&ah, asz) || cudaMalloc(&bh, bsz) || cudaMalloc(&C, (size_t)M * N * 8 * batch) ||
      cudaMalloc(&ez, (size_t)emax * 4) || cudaMalloc(&err, 4))
    return -1;
  gwdbg_fill_half_kernel<<<1216, 256>>>((__half*)ah, (int64_t)(asz / 2), 12345u);
  gwdbg_fill_half_kernel<<<1216, 256>>>((__half*)bh, (int64_t)(bsz / 2), 67890u);
  cudaMemset(C, 0, (size_t)M * N * 8 * batch); cudaMemset(ez, 0, (size_t)emax * 4); cudaMemset(err, 0, 4);
  UmmaOperand oa{(const float*)ah, (const float*)ah, M, batch, Kpad, (int64_t)M * Kpad, 1};
  UmmaOperand ob{(const float*)bh, (const float*)bh, N, 1, Kpad, 0, 1};
  UmmaScale sc{ez, ez, 0, 0, 0};
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  const bool acc = c_fp64 != 0;
  cudaError_t e = umma_gemm(oa, ob, M, N, Kpad, batch, C, c_fp64, 1.0, acc, N, (int64_t)M * N, 3, err, 0, 1, 0, 0, 0, 0,
                            nullptr, &sc, 0);
  cudaEventRecord(e0, 0);
  for (int i = 0; i < iters && !e; ++i)
    e = umma_gemm(oa, ob, M, N, Kpad, batch, C, c_fp64, 1.0, acc, N, (int64_t)M * N, 3, err, 0, 1, 0, 0, 0, 0,
                  nullptr, &sc, 0);
  cudaEventRecord(e1, 0);
  if (!e) e = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  *ms = t / iters;
  int herr = 0;
  cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
  cudaFree(ah); cudaFree(bh); cudaFree(C); cudaFree(ez); cudaFree(err);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  return e ? (int)e : herr;
}
