// FP64 complex GEMMs on the TF32 tensor cores by exact digit splitting.
//
// Each real value x of an operand row is written x = 2^e sum_{i=1..S} d_i 2^(-7 i)
// with one exponent e per row (max |x| <= 2^e) and integer digits d_i
// (|d_1| <= 128, |d_i| <= 64 for i > 1, balanced rounding), i.e. 56 bits.
// Every digit is an integer that TF32 holds exactly, every digit product has at
// most 14 bits, and a launch sums at most 1024 products per output (pairs x K),
// so the tensor pipe's FP32 accumulation of a launch is exact.  The product
//   x_A x_B = 2^(eA + eB) sum_{i,j} d_i d_j 2^(-7 (i + j))
// keeps the pairs with i + j <= S + 1 (36 of them); each launch covers pairs of
// one i + j and is added into the FP64 output with the exact scale
// 2^(eA + eB - 7 (i + j)) (the tensor-core GEMM's scaled FP64 epilogue).  The
// dropped pairs and the truncated digits leave an error below ~2^-54 relative to
// K max|A_row| max|B_col|, at the level of an FP64 GEMM.
//
// Operand layout: digit planes of a row are stored one after another,
// [row][S][Kp] (Kp = padded real K), so the K range of a launch is contiguous.
// B's planes are stored in reverse digit order so that the B slices that pair
// with A slices i0..i1 of a launch are contiguous as well.
//
// Used for the tau <-> i nu transforms Y[z] = T X[z]: A = X[z]^T (rows = columns
// of X, complex K = ntau), B = T (rows 2m, 2m+1 = the real 2x2 blocks of T[m][j]),
// output written transposed into Y (lane-per-row FP64 stores).
#include "gw_internal.cuh"

namespace gwk {

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
                                                         int64_t ld, int64_t zs, float* __restrict__ dig,
                                                         int* __restrict__ ex, int64_t Kp) {
  __shared__ double2 tile[32][33];
  __shared__ double red[8][32];
  __shared__ int es[32];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  const int64_t z = blockIdx.y;
  const double2* X = src + z * zs;
  float* D = dig + z * ncol * (int64_t)EM_S * Kp;
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
        float* o = D + row * rowlen + 2 * j;
#pragma unroll
        for (int i = 0; i < EM_S; ++i) *(float2*)(o + (int64_t)i * Kp) = make_float2(dr[i], di[i]);
      }
    }
    __syncthreads();
  }
}

// B operand of C = A B^T from a small complex matrix B[m][j] (rows x K, row stride
// ldb): rows 2m = (Br, -Bi), 2m+1 = (Bi, Br) along the real K index 2j + c;
// digit planes in reverse order; one exponent per complex row m.
__global__ void em_split_b_kernel(const double2* __restrict__ B, int64_t rows, int64_t K, int64_t ldb,
                                  float* __restrict__ dig, int* __restrict__ ex, int64_t Kp) {
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
    float* r0 = dig + (2 * m) * rowlen + 2 * j;
    float* r1 = dig + (2 * m + 1) * rowlen + 2 * j;
#pragma unroll
    for (int i = 0; i < EM_S; ++i) {
      const int64_t p = (int64_t)(EM_S - 1 - i) * Kp;   // reverse digit order
      *(float2*)(r0 + p) = make_float2(dr[i], -di[i]);
      *(float2*)(r1 + p) = make_float2(di[i], dr[i]);
    }
  }
}

int64_t emul_kpad(int64_t K) { return (2 * K + 31) / 32 * 32; }
size_t emul_digit_bytes(int64_t rows, int64_t K) { return (size_t)rows * EM_S * emul_kpad(K) * 4; }

cudaError_t emul_split_b(const double2* B, int64_t rows, int64_t K, int64_t ldb, float* dig, int* ex,
                         cudaStream_t st) {
  const int64_t Kp = emul_kpad(K);
  cudaError_t e = cudaMemsetAsync(dig, 0, (size_t)2 * rows * EM_S * Kp * 4, st);
  if (e != cudaSuccess) return e;
  em_split_b_kernel<<<(unsigned)rows, 256, 0, st>>>(B, rows, K, ldb, dig, ex, Kp);
  return cudaGetLastError();
}

// Y (nrow x ncol complex, row stride ldy) (+)= T_digits (nrow x K) * X (K x ncol, row
// stride ldx), FP64-exact up to ~2^-54 relative.  Bd/Be: digits and exponents of T
// from emul_split_b (2*nrow rows).  Ad/Ae: workspace of emul_digit_bytes(ncol, K)
// bytes (zeroed once by the caller: the padding columns must stay zero) and ncol ints.
cudaError_t emul_transform(const float* Bd, const int* Be, int64_t nrow, const double2* X, int64_t K, int64_t ncol,
                           int64_t ldx, double2* Y, int64_t ldy, float* Ad, int* Ae, int* err, cudaStream_t st) {
  if (ldy != ncol) return cudaErrorInvalidValue;   // transposed lane-per-row stores assume packed rows
  const int64_t Kp = emul_kpad(K);
  em_split_t_kernel<<<dim3((unsigned)((ncol + 31) / 32), 1), 256, 0, st>>>(X, K, ncol, ldx, 0, Ad, Ae, Kp);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const int64_t ld = (int64_t)EM_S * Kp;
  const int pmax = (int)(1024 / Kp) < 1 ? 1 : (int)(1024 / Kp);
  bool first = true;
  for (int g = EM_S + 1; g >= 2; --g) {   // smallest contributions first
    const int lo = g - EM_S > 1 ? g - EM_S : 1, hi = g - 1 < EM_S ? g - 1 : EM_S;
    for (int i0 = lo; i0 <= hi; i0 += pmax) {
      const int i1 = i0 + pmax - 1 < hi ? i0 + pmax - 1 : hi;
      const int np = i1 - i0 + 1;
      UmmaOperand oa{Ad + (int64_t)(i0 - 1) * Kp, nullptr, ncol, 1, ld, 0};
      UmmaOperand ob{const_cast<float*>(Bd) + (int64_t)(EM_S - g + i0) * Kp, nullptr, 2 * nrow, 1, ld, 0};
      UmmaScale sc{Ae, Be, 0, 0, -EM_BETA * g};
      e = umma_gemm(oa, ob, (int)ncol, (int)(2 * nrow), (int64_t)np * Kp, 1, (void*)Y, true, 1.0, !first, 2, 0, 1,
                    err, st, 1, 0, 0, 2, 2 * ldy, nullptr, &sc, (int64_t)(np - 1) * Kp + 2 * K);
      if (e != cudaSuccess) return e;
      first = false;
    }
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
  if (cudaMalloc(&Bd, (size_t)2 * nrow * EM_S * Kp * 4) || cudaMalloc(&Be, (size_t)nrow * 4) ||
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
