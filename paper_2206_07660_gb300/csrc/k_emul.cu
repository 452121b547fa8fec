// FP64 complex GEMMs on the TF32 tensor cores by exact digit splitting.
//
// Each real value x of an operand row is written x = 2^e sum_{i=1..S} d_i 2^(-7 i)
// with one exponent e per row (max |x| <= 2^e) and integer digits d_i
// (|d_1| <= 128, |d_i| <= 64 for i > 1, balanced rounding), i.e. 56 bits.
// Every digit is an integer that TF32 holds exactly, every digit product has at
// most 14 bits (|d_1 d_1| <= 2^14, |d_1 d_j| <= 2^13, |d_i d_j| <= 2^12 for i, j > 1),
// and the pairs of one launch are chosen so that the sum over its pairs of K times
// that bound stays <= 2^24: every partial sum is an integer below 2^24 and the
// tensor pipe's FP32 accumulation of a launch is exact.  The product
//   x_A x_B = 2^(eA + eB) sum_{i,j} d_i d_j 2^(-7 (i + j))
// keeps the pairs with i + j <= S + 1 (36 of them); each launch covers pairs of
// one i + j and is added into the FP64 output with the exact scale
// 2^(eA + eB - 7 (i + j)) (the tensor-core GEMM's scaled FP64 epilogue).  The
// dropped pairs and the truncated digits leave an error below ~2^-54 relative to
// K max|A_row| max|B_col|, at the level of an FP64 GEMM.
//
// Operand layout: digit planes of a row are stored one after another,
// [row][S][Kp] (Kp = padded real K), so the K range of a launch is contiguous.
// The digits are stored as fp16 (exact for |d| <= 2048) and multiplied with
// tcgen05 kind::f16 (FP32 accumulation): half the bytes of TF32 storage and twice
// the tensor rate, with the same exact sums.
// B's planes are stored in reverse digit order so that the B slices that pair
// with A slices i0..i1 of a launch are contiguous as well.
//
// Used for the tau <-> i nu transforms Y[z] = T X[z]: A = X[z]^T (rows = columns
// of X, complex K = ntau), B = T (rows 2m, 2m+1 = the real 2x2 blocks of T[m][j]),
// output written transposed into Y (lane-per-row FP64 stores); and for the batched
// square products C[z] = A[z] B[z] of the screened solve's refinement (A split from
// its rows, B from its columns, output row-major).
#include <cuda_fp16.h>
#include "gw_internal.cuh"

namespace gwk {

using dig_t = __half;   // storage of one digit

constexpr int EM_BETA = 7;
constexpr int EM_S = 8;
static_assert(EM_BETA == 7, "the balanced digit masks below are for 7-bit digits");

// digits of x / 2^e (|x| <= 2^e): d[0..S-1].  x is rounded once to a multiple of
// 2^(e - 7S) (an exact integer v with |v| <= 2^(7S) = 2^56), whose balanced base-128
// digits d_S .. d_2 in [-64, 63] are peeled off with integer shifts; the rest is
// d_1 (|d_1| <= 128).
__device__ __forceinline__ void em_digits(double x, int e, float* d) {
  long long v = __double2ll_rn(ldexp(x, EM_BETA * EM_S - e));
#pragma unroll
  for (int i = EM_S - 1; i >= 1; --i) {
    const long long di = ((v + 64) & 127) - 64;
    d[i] = (float)di;
    v = (v - di) >> EM_BETA;
  }
  d[0] = (float)v;
}

__device__ __forceinline__ int em_exponent(double m) {
  if (!(m > 0.0)) return 0;
  int e;
  frexp(m, &e);   // m = f 2^e, f in [0.5, 1): m < 2^e
  return e;
}

// A-operand digits from a transposed source: row n of the operand is column n of a
// K x ncol complex matrix (element (n, k) at src[z*zs + k*ld + n]), real K index
// 2k + c (re, im).  Padding columns [2K, Kp) are written as zeros.  Block: 32 rows x
// all K; the source tile goes through shared memory so both the reads (along n)
// and the digit writes (along k) are coalesced.
__global__ void __launch_bounds__(256) em_split_t_kernel(const double2* __restrict__ src, int64_t K, int64_t ncol,
                                                         int64_t ld, int64_t zs, dig_t* __restrict__ dig,
                                                         int* __restrict__ ex, int64_t Kp) {
  __shared__ double2 tile[32][33];
  __shared__ double red[8][32];
  __shared__ int es[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t z = blockIdx.y;
  const double2* X = src + z * zs;
  dig_t* D = dig + z * ncol * (int64_t)EM_S * Kp;
  int* E = ex + z * ncol;
  const int64_t n0 = (int64_t)blockIdx.x * 32;
  const int64_t n = n0 + tx;
  double m = 0.0;
  if (n < ncol)
    for (int64_t j = ty; j < K; j += 8) {
      const double2 v = X[j * ld + n];
      m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
    }
  red[ty][tx] = m;
  __syncthreads();
  if (ty == 0) {
    double mm = red[0][tx];
    for (int r = 1; r < 8; ++r) mm = fmax(mm, red[r][tx]);
    const int e = em_exponent(mm);
    es[tx] = e;
    if (n < ncol) E[n] = e;
  }
  __syncthreads();
  const int64_t rowlen = (int64_t)EM_S * Kp;
  const int64_t kc = (Kp + 1) / 2;   // complex columns incl. padding
  for (int64_t j0 = 0; j0 < kc; j0 += 32) {
    for (int jj = ty; jj < 32; jj += 8) {
      const int64_t j = j0 + jj;
      tile[jj][tx] = (j < K && n < ncol) ? X[j * ld + n] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {
      const int64_t row = n0 + rr, j = j0 + tx;
      if (row < ncol && 2 * j < Kp) {
        const double2 v = tile[tx][rr];
        float dr[EM_S], di[EM_S];
        em_digits(v.x, es[rr], dr);
        em_digits(v.y, es[rr], di);
        dig_t* o = D + row * rowlen + 2 * j;
#pragma unroll
        for (int i = 0; i < EM_S; ++i) *(__half2*)(o + (int64_t)i * Kp) = __floats2half2_rn(dr[i], di[i]);
      }
    }
    __syncthreads();
  }
}

// B operand of C = A B^T from a small complex matrix B[m][j] (rows x K, row stride
// ldb): rows 2m = (Br, -Bi), 2m+1 = (Bi, Br) along the real K index 2j + c;
// digit planes in reverse order; one exponent per complex row m.
__global__ void em_split_b_kernel(const double2* __restrict__ B, int64_t rows, int64_t K, int64_t ldb,
                                  dig_t* __restrict__ dig, int* __restrict__ ex, int64_t Kp) {
  const int64_t m = blockIdx.x;
  __shared__ double red[256];
  double mx = 0.0;
  for (int64_t j = threadIdx.x; j < K; j += blockDim.x) {
    const double2 v = B[m * ldb + j];
    mx = fmax(mx, fmax(fabs(v.x), fabs(v.y)));
  }
  red[threadIdx.x] = mx;
  __syncthreads();
  for (int s = blockDim.x / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
    __syncthreads();
  }
  const int e = em_exponent(red[0]);
  if (threadIdx.x == 0) ex[m] = e;
  const int64_t rowlen = (int64_t)EM_S * Kp;
  for (int64_t j = threadIdx.x; j < K; j += blockDim.x) {
    const double2 v = B[m * ldb + j];
    float dr[EM_S], di[EM_S];
    em_digits(v.x, e, dr);
    em_digits(v.y, e, di);
    dig_t* r0 = dig + (2 * m) * rowlen + 2 * j;
    dig_t* r1 = dig + (2 * m + 1) * rowlen + 2 * j;
#pragma unroll
    for (int i = 0; i < EM_S; ++i) {
      const int64_t p = (int64_t)(EM_S - 1 - i) * Kp;   // reverse digit order
      *(__half2*)(r0 + p) = __floats2half2_rn(dr[i], -di[i]);
      *(__half2*)(r1 + p) = __floats2half2_rn(di[i], dr[i]);
    }
  }
}

// A-operand digits from complex rows: row r of batch z is src[z*zs + r*ld + k],
// k < K, real K index 2k + c.  One warp per row; padding columns [2K, Kp) are
// written as zeros.
__global__ void __launch_bounds__(256) em_split_r_kernel(const double2* __restrict__ src, int64_t rows, int64_t K,
                                                         int64_t ld, int64_t zs, int64_t count,
                                                         dig_t* __restrict__ dig, int* __restrict__ ex, int64_t Kp) {
  const int lane = threadIdx.x & 31;
  const int64_t gr = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (gr >= rows * count) return;
  const int64_t z = gr / rows, r = gr - z * rows;
  const double2* x = src + z * zs + r * ld;
  double m = 0.0;
  for (int64_t k = lane; k < K; k += 32) {
    const double2 v = x[k];
    m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  const int e = em_exponent(m);
  if (lane == 0) ex[gr] = e;
  dig_t* o = dig + gr * (int64_t)EM_S * Kp;
  for (int64_t k = lane; 2 * k < Kp; k += 32) {
    float dr[EM_S], di[EM_S];
    if (k < K) {
      const double2 v = x[k];
      em_digits(v.x, e, dr);
      em_digits(v.y, e, di);
    } else {
#pragma unroll
      for (int i = 0; i < EM_S; ++i) dr[i] = di[i] = 0.f;
    }
#pragma unroll
    for (int i = 0; i < EM_S; ++i) *(__half2*)(o + (int64_t)i * Kp + 2 * k) = __floats2half2_rn(dr[i], di[i]);
  }
}

// B-operand digits of C = A B from the columns of a complex K x ncol matrix B[z]
// (element (k, j) at src[z*zs + k*ld + j]): rows 2j = (Br, -Bi), 2j+1 = (Bi, Br)
// along the real K index 2k + c, digit planes in reverse order, one exponent per
// column j.  Block: 32 columns x all K through a shared-memory tile (reads along j,
// digit writes along k); padding columns [2K, Kp) are written as zeros.
__global__ void __launch_bounds__(256) em_split_bt_kernel(const double2* __restrict__ src, int64_t K, int64_t ncol,
                                                          int64_t ld, int64_t zs, dig_t* __restrict__ dig,
                                                          int* __restrict__ ex, int64_t Kp) {
  __shared__ double2 tile[32][33];
  __shared__ double red[8][32];
  __shared__ int es[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t z = blockIdx.y;
  const double2* X = src + z * zs;
  const int64_t rowlen = (int64_t)EM_S * Kp;
  dig_t* D = dig + z * 2 * ncol * rowlen;
  int* E = ex + z * ncol;
  const int64_t n0 = (int64_t)blockIdx.x * 32;
  const int64_t n = n0 + tx;
  double m = 0.0;
  if (n < ncol)
    for (int64_t j = ty; j < K; j += 8) {
      const double2 v = X[j * ld + n];
      m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
    }
  red[ty][tx] = m;
  __syncthreads();
  if (ty == 0) {
    double mm = red[0][tx];
    for (int r = 1; r < 8; ++r) mm = fmax(mm, red[r][tx]);
    const int e = em_exponent(mm);
    es[tx] = e;
    if (n < ncol) E[n] = e;
  }
  __syncthreads();
  const int64_t kc = Kp / 2;   // complex columns incl. padding
  for (int64_t j0 = 0; j0 < kc; j0 += 32) {
    for (int jj = ty; jj < 32; jj += 8) {
      const int64_t j = j0 + jj;
      tile[jj][tx] = (j < K && n < ncol) ? X[j * ld + n] : make_double2(0.0, 0.0);
    }
    __syncthreads();
    for (int rr = ty; rr < 32; rr += 8) {
      const int64_t col = n0 + rr, j = j0 + tx;
      if (col < ncol && j < kc) {
        const double2 v = tile[tx][rr];
        float dr[EM_S], di[EM_S];
        em_digits(v.x, es[rr], dr);
        em_digits(v.y, es[rr], di);
        dig_t* r0 = D + (2 * col) * rowlen + 2 * j;
        dig_t* r1 = r0 + rowlen;
#pragma unroll
        for (int i = 0; i < EM_S; ++i) {
          const int64_t p = (int64_t)(EM_S - 1 - i) * Kp;
          *(__half2*)(r0 + p) = __floats2half2_rn(dr[i], -di[i]);
          *(__half2*)(r1 + p) = __floats2half2_rn(di[i], dr[i]);
        }
      }
    }
    __syncthreads();
  }
}

// Launch plan of the digit-pair products for a real K extent kreal, keeping the
// pairs with i + j <= nd + 1 of the first nd digits: launches of pairs (i, g - i),
// i = i0..i1 (1-based digits), one significance g each, smallest contributions
// first, each summing at most 2^24 in magnitude (exact in FP32).  Returns the number
// of launches, or -1 when one pair alone could round (kreal > 1024).
struct EmLaunch { int g, i0, i1; };
static int em_plan(int64_t kreal, EmLaunch* out, int nd = EM_S) {
  if (kreal * (int64_t)(1 << 14) > ((int64_t)1 << 24) || nd < 1 || nd > EM_S) return -1;
  int n = 0;
  for (int g = nd + 1; g >= 2; --g) {
    const int lo = g - nd > 1 ? g - nd : 1, hi = g - 1 < nd ? g - 1 : nd;
    int i0 = lo;
    int64_t acc = 0;
    for (int i = lo; i <= hi; ++i) {
      const int j = g - i;
      const int64_t b = kreal * (int64_t)((i == 1 && j == 1) ? 1 << 14 : (i == 1 || j == 1) ? 1 << 13 : 1 << 12);
      if (i > i0 && acc + b > ((int64_t)1 << 24)) {
        out[n++] = EmLaunch{g, i0, i - 1};
        i0 = i;
        acc = 0;
      }
      acc += b;
    }
    out[n++] = EmLaunch{g, i0, hi};
  }
  return n;
}
constexpr int EM_MAXL = EM_S * EM_S;

int emul_launches(int64_t K, int nd) {
  EmLaunch pl[EM_MAXL];
  return em_plan(2 * K, pl, nd);
}

// real K padded to whole 128-byte k-blocks of fp16
int64_t emul_kpad(int64_t K) { return (2 * K + 63) / 64 * 64; }
size_t emul_digit_bytes(int64_t rows, int64_t K) { return (size_t)rows * EM_S * emul_kpad(K) * sizeof(dig_t); }

cudaError_t emul_split_b(const double2* B, int64_t rows, int64_t K, int64_t ldb, void* dig, int* ex,
                         cudaStream_t st) {
  const int64_t Kp = emul_kpad(K);
  cudaError_t e = cudaMemsetAsync(dig, 0, emul_digit_bytes(2 * rows, K), st);
  if (e != cudaSuccess) return e;
  em_split_b_kernel<<<(unsigned)rows, 256, 0, st>>>(B, rows, K, ldb, (dig_t*)dig, ex, Kp);
  return cudaGetLastError();
}

// Y (nrow x ncol complex, row stride ldy) (+)= T_digits (nrow x K) * X (K x ncol, row
// stride ldx), FP64-exact up to ~2^-54 relative.  Bd/Be: digits and exponents of T
// from emul_split_b (2*nrow rows).  Ad/Ae: workspace of emul_digit_bytes(ncol, K)
// bytes (zeroed once by the caller: the padding columns must stay zero) and ncol ints.
cudaError_t emul_transform(const void* Bdv, const int* Be, int64_t nrow, const double2* X, int64_t K, int64_t ncol,
                           int64_t ldx, double2* Y, int64_t ldy, void* Adv, int* Ae, int* err, cudaStream_t st) {
  if (ldy != ncol) return cudaErrorInvalidValue;   // transposed lane-per-row stores assume packed rows
  const dig_t* Bd = (const dig_t*)Bdv;
  dig_t* Ad = (dig_t*)Adv;
  const int64_t Kp = emul_kpad(K);
  em_split_t_kernel<<<dim3((unsigned)((ncol + 31) / 32), 1), 256, 0, st>>>(X, K, ncol, ldx, 0, Ad, Ae, Kp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t ld = (int64_t)EM_S * Kp;
  EmLaunch pl[EM_MAXL];
  const int nl = em_plan(2 * K, pl);
  if (nl < 0) return cudaErrorInvalidValue;
  for (int l = 0; l < nl; ++l) {
    const int g = pl[l].g, i0 = pl[l].i0, np = pl[l].i1 - pl[l].i0 + 1;
    UmmaOperand oa{(const float*)(Ad + (int64_t)(i0 - 1) * Kp), nullptr, ncol, 1, ld, 0, 1};
    UmmaOperand ob{(const float*)(Bd + (int64_t)(EM_S - g + i0) * Kp), nullptr, 2 * nrow, 1, ld, 0, 1};
    UmmaScale sc{Ae, Be, 0, 0, -EM_BETA * g};
    e = umma_gemm(oa, ob, (int)ncol, (int)(2 * nrow), (int64_t)np * Kp, 1, (void*)Y, true, 1.0, l > 0, 2, 0, 1,
                  err, st, 1, 0, 0, 2, 2 * ldy, nullptr, &sc, (int64_t)(np - 1) * Kp + 2 * K);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

// Digits of the batched operands of C[z] = A[z] B[z] (A: count x M x K complex, row
// stride lda, batch stride sa; B: count x K x N, row stride ldb, batch stride sb).
// Ad/Ae: emul_digit_bytes(M, K) and M ints per batch; Bd/Be: emul_digit_bytes(2N, K)
// and N ints per batch.
cudaError_t emul_split_rows(const double2* A, int64_t count, int64_t M, int64_t K, int64_t lda, int64_t sa,
                            void* Ad, int* Ae, cudaStream_t st) {
  const int64_t Kp = emul_kpad(K);
  const int64_t nb = (M * count + 7) / 8;
  if (nb > INT32_MAX) return cudaErrorInvalidValue;
  em_split_r_kernel<<<(unsigned)nb, 256, 0, st>>>(A, M, K, lda, sa, count, (dig_t*)Ad, Ae, Kp);
  return cudaGetLastError();
}
cudaError_t emul_split_cols(const double2* B, int64_t count, int64_t K, int64_t N, int64_t ldb, int64_t sb,
                            void* Bd, int* Be, cudaStream_t st) {
  const int64_t Kp = emul_kpad(K);
  if (count > 65535) return cudaErrorInvalidValue;
  em_split_bt_kernel<<<dim3((unsigned)((N + 31) / 32), (unsigned)count), 256, 0, st>>>(B, K, N, ldb, sb, (dig_t*)Bd,
                                                                                        Be, Kp);
  return cudaGetLastError();
}

// C[z] (M x N complex, row-major, row stride N, batch stride M N) = A[z] B[z] from the
// digits of emul_split_rows / emul_split_cols, FP64-exact up to ~2^-54 relative with
// nd = 8 digits; nd < 8 keeps the pairs with i + j <= nd + 1 of the leading nd
// digits: each real product then errs by up to ~(nd + 1) 2^(13 - 7 (nd + 2)) of
// max|A_row| max|B_col| (9e-11 for nd = 5).
cudaError_t emul_cgemm_batched(const void* Adv, const int* Ae, const void* Bdv, const int* Be, int64_t count,
                               int64_t M, int64_t N, int64_t K, double2* C, int* err, cudaStream_t st, int nd) {
  const dig_t* Ad = (const dig_t*)Adv;
  const dig_t* Bd = (const dig_t*)Bdv;
  const int64_t Kp = emul_kpad(K), ld = (int64_t)EM_S * Kp;
  EmLaunch pl[EM_MAXL];
  const int nl = em_plan(2 * K, pl, nd);
  if (nl < 0 || count > 65535) return cudaErrorInvalidValue;
  for (int l = 0; l < nl; ++l) {
    const int g = pl[l].g, i0 = pl[l].i0, np = pl[l].i1 - pl[l].i0 + 1;
    UmmaOperand oa{(const float*)(Ad + (int64_t)(i0 - 1) * Kp), nullptr, M, count, ld, M * ld, 1};
    UmmaOperand ob{(const float*)(Bd + (int64_t)(EM_S - g + i0) * Kp), nullptr, 2 * N, count, ld, 2 * N * ld, 1};
    UmmaScale sc{Ae, Be, M, N, -EM_BETA * g};
    cudaError_t e = umma_gemm(oa, ob, (int)M, (int)(2 * N), (int64_t)np * Kp, (int)count, (void*)C, true, 1.0, l > 0,
                              2 * N, 2 * M * N, 1, err, st, 1, 0, 0, 0, 0, nullptr, &sc,
                              (int64_t)(np - 1) * Kp + 2 * K);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace gwk

// ------------------------------------------------------------------ test hook
// Y (nrow x ncol) = T (nrow x K) X (K x ncol), complex128 device pointers, through
// the digit-split tensor-core path.  Allocates its scratch; returns 0 or an error code.
extern "C" int gwdbg_emul_transform(const double2* T, const double2* X, double2* Y, int nrow, int K, int ncol,
                                    double* ms) {
  using namespace gwk;
  const int64_t Kp = emul_kpad(K);
  float *Bd = nullptr, *Ad = nullptr;
  int *Be = nullptr, *Ae = nullptr, *err = nullptr;
  if (cudaMalloc(&Bd, emul_digit_bytes(2 * (int64_t)nrow, K)) || cudaMalloc(&Be, (size_t)nrow * 4) ||
      cudaMalloc(&Ad, emul_digit_bytes(ncol, K)) || cudaMalloc(&Ae, (size_t)ncol * 4) || cudaMalloc(&err, 4))
    return -1;
  cudaMemset(Ad, 0, emul_digit_bytes(ncol, K));
  cudaMemset(err, 0, 4);
  cudaError_t e = emul_split_b(T, nrow, K, K, Bd, Be, 0);
  if (!e) e = emul_transform(Bd, Be, nrow, X, K, ncol, ncol, Y, ncol, Ad, Ae, err, 0);   // warm-up / tuning
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0); cudaEventCreate(&e1);
  cudaEventRecord(e0, 0);
  if (!e) e = emul_transform(Bd, Be, nrow, X, K, ncol, ncol, Y, ncol, Ad, Ae, err, 0);
  cudaEventRecord(e1, 0);
  if (!e) e = cudaEventSynchronize(e1);
  float t = 0.f;
  cudaEventElapsedTime(&t, e0, e1);
  if (ms) *ms = t;
  int herr = 0;
  cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
  cudaFree(Bd); cudaFree(Be); cudaFree(Ad); cudaFree(Ae); cudaFree(err);
  cudaEventDestroy(e0); cudaEventDestroy(e1);
  return e ? (int)e : herr;
}

// C[z] (M x N) = A[z] (M x K) B[z] (K x N), complex128 device pointers, row-major and
// contiguous per batch, through the digit-split tensor-core path with nd digits.
// Allocates its scratch; returns 0 or an error code (100 + role: a tensor-core wait
// gave up).
extern "C" int gwdbg_emul_cgemm(const double2* A, const double2* B, double2* C, int count, int M, int N, int K,
                                int nd) {
  using namespace gwk;
  float *Ad = nullptr, *Bd = nullptr;
  int *Ae = nullptr, *Be = nullptr, *err = nullptr;
  if (cudaMalloc(&Ad, (size_t)count * emul_digit_bytes(M, K)) || cudaMalloc(&Bd, (size_t)count * emul_digit_bytes(2 * N, K)) ||
      cudaMalloc(&Ae, (size_t)count * M * 4) || cudaMalloc(&Be, (size_t)count * N * 4) || cudaMalloc(&err, 4))
    return -1;
  cudaMemset(err, 0, 4);
  cudaError_t e = emul_split_rows(A, count, M, K, K, (int64_t)M * K, Ad, Ae, 0);
  if (!e) e = emul_split_cols(B, count, K, N, N, (int64_t)K * N, Bd, Be, 0);
  if (!e) e = emul_cgemm_batched(Ad, Ae, Bd, Be, count, M, N, K, C, err, 0, nd);
  if (!e) e = cudaDeviceSynchronize();
  int herr = 0;
  cudaMemcpy(&herr, err, 4, cudaMemcpyDeviceToHost);
  cudaFree(Ad); cudaFree(Bd); cudaFree(Ae); cudaFree(Be); cudaFree(err);
  return e ? (int)e : herr;
}

// Host-only view of the launch plan of a digit-split product (no GPU needed): writes
// up to cap launches as (g, i0, i1) triples into out and returns their number (-1
// when kreal is too large for exact sums).
extern "C" int gwdbg_emul_plan(int64_t kreal, int nd, int* out, int cap) {
  using namespace gwk;
  EmLaunch pl[EM_MAXL];
  const int n = em_plan(kreal, pl, nd);
  for (int l = 0; l < n && l < cap; ++l) {
    out[3 * l] = pl[l].g;
    out[3 * l + 1] = pl[l].i0;
    out[3 * l + 2] = pl[l].i1;
  }
  return n;
}
