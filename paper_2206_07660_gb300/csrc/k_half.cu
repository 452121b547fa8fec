// Operands of the tensor-core contraction chains as 16-bit pieces (fp16 or bf16)
// with power-of-two scales, and the a-priori bounds that fix those scales.
//
// A value x of a row with scale exponent e is stored as hi = rn(x 2^-e),
// lo = rn(x 2^-e - hi) in the 16-bit format; hi + lo carries 22 significant bits
// (fp16) or 16 (bf16).  The GEMM's epilogue multiplies its fp32 sums by
// 2^(eA + eB) and, when it writes the next GEMM's operand, by 2^-eO of that
// operand's row.  With fp16 the scaled values must stay below 2^15 in magnitude;
// every exponent here is taken from an upper bound of the row's values (a row
// maximum, or a product of norms that bounds a matrix product), so nothing
// overflows.  Values far below the bound keep an absolute error of 2^-24 of it.
//
// Exponent rule: for a bound b = f 2^E (f in [0.5, 1)), e = E - 15 when b is the
// exact row maximum, E - 14 (one bit of margin) when it bounds a sum computed in
// fp32 by the tensor cores.
//
// The per-pair operand kernels take a list of source slabs (one output block each), so
// that one launch prepares the operands of several k-points, and they are launched as
// programmatic dependents of the previous kernel on the stream.
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include "gw_internal.cuh"

namespace gwk {

__device__ __forceinline__ int bound_exp(double b, int margin) {
  int E = 0;
  if (b > 0.0) frexp(b, &E);
  // kept inside [-100, 100] so that 2^-e and every product of scales stays a normal
  // float (rows below 2^-115 are zero to working accuracy)
  const int e = E - 15 + margin;
  return e < -100 ? -100 : (e > 100 ? 100 : e);
}

// 2^e as a float (e within the normal range; clamped)
__device__ __forceinline__ float pow2f(int e) {
  e = e < -126 ? -126 : (e > 127 ? 127 : e);
  return __int_as_float((e + 127) << 23);
}

// pieces of x 2^-e, x rounded to fp32 first (24 bits, more than the 22 the two
// pieces keep); the scaling by a power of two is exact; fp32 arithmetic only (the
// FP64 pipe is a small fraction of the SM's throughput)
__device__ __forceinline__ void pieces(int fmt, double x, int e, uint16_t& h, uint16_t& l) {
  const float d = (float)x * pow2f(-e);
  if (fmt == 2) {
    const __nv_bfloat16 hb = __float2bfloat16_rn(d);
    const __nv_bfloat16 lb = __float2bfloat16_rn(d - __bfloat162float(hb));
    h = __bfloat16_as_ushort(hb);
    l = __bfloat16_as_ushort(lb);
  } else {
    const __half hh = __float2half_rn(d);
    const __half lh = __float2half_rn(d - __half2float(hh));
    h = __half_as_ushort(hh);
    l = __half_as_ushort(lh);
  }
}

__device__ __forceinline__ double wmax(double m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  return m;
}
__device__ __forceinline__ double wsum(double m) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
  return m;
}
__device__ __forceinline__ double cabs2(double2 v) { return sqrt(v.x * v.x + v.y * v.y); }

// Rows r of a complex matrix (element (r, k) at src + r*ld + k) as real rows
// (re, +-im) of Kpad 16-bit pieces at row stride ldo, one exponent per row from the
// row's max |re|, |im| (ex[r]); exs (optional) receives the exponent of the row's
// sum of moduli (a bound of any product of the row with a vector of modulus <= 1).
// One warp per row.
// Kernels launched as programmatic dependents of the stream's previous kernel start
// while it finishes and wait here for it to complete before touching memory.
__device__ __forceinline__ void dep_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
static cudaError_t launch_dep(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t st, Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = 0;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, (KArgs)args...);
}

__global__ void __launch_bounds__(256) half_rows_kernel(const double2* __restrict__ src, int64_t rows, int64_t K,
                                                        int64_t ld, int conj, uint16_t* hi, uint16_t* lo,
                                                        int64_t Kpad, int64_t ldo, int fmt, int* ex, int* exs,
                                                        const __grid_constant__ SrcList list, int64_t dstride, int64_t estride) {
  dep_wait();
  // matrix blockIdx.y of the list: its source offset, its output and exponent blocks
  src += list.off[blockIdx.y];
  hi += blockIdx.y * dstride;
  lo += blockIdx.y * dstride;
  ex += blockIdx.y * estride;
  if (exs) exs += blockIdx.y * estride;
  const int lane = threadIdx.x & 31;
  const int64_t r = (int64_t)blockIdx.x * 8 + (threadIdx.x >> 5);
  if (r >= rows) return;
  const double2* x = src + r * ld;
  // fp32 is enough for the bounds: a rounded maximum only moves the exponent up, and
  // the row sum is enlarged by far more than its rounding error
  float m = 0.f, sm = 0.f;
  for (int64_t k = lane; k < K; k += 32) {
    const double2 v = x[k];
    const float a = (float)v.x, b = (float)v.y;
    m = fmaxf(m, fmaxf(fabsf(a), fabsf(b)));
    sm += sqrtf(a * a + b * b);
  }
  const int e = bound_exp((double)wmax((double)m), 0);
  sm = (float)wsum((double)sm);
  if (lane == 0) {
    ex[r] = e;
    if (exs) exs[r] = bound_exp((double)sm * (1.0 + 1e-4), 0);
  }
  uint32_t* h2 = (uint32_t*)(hi + r * ldo);
  uint32_t* l2 = (uint32_t*)(lo + r * ldo);
  for (int64_t c = lane; 2 * c < Kpad; c += 32) {
    double re = 0.0, im = 0.0;
    if (c < K) {
      const double2 v = x[c];
      re = v.x;
      im = conj ? -v.y : v.y;
    }
    uint16_t hr, lr, hm, lm;
    pieces(fmt, re, e, hr, lr);
    pieces(fmt, im, e, hm, lm);
    h2[c] = (uint32_t)hr | ((uint32_t)hm << 16);
    l2[c] = (uint32_t)lr | ((uint32_t)lm << 16);
  }
}

// Doubled operand of C = A conj(B)^T from complex rows n of B (K entries): real rows
// 2n = (re, im), 2n+1 = (-im, re) of 16-bit pieces at row stride ldo, with the given
// exponent ex[n] of each complex row.  Grid (column blocks of 256 complex entries, rows).
__global__ void __launch_bounds__(256) half_embed_conj_kernel(const double2* __restrict__ src, int64_t rows,
                                                              int64_t K, uint16_t* hi, uint16_t* lo, int64_t Kpad,
                                                              int64_t ldo, int fmt, const int* ex,
                                                              const __grid_constant__ SrcList list, int64_t dstride) {
  dep_wait();
  src += list.off[blockIdx.z];
  hi += blockIdx.z * dstride;
  lo += blockIdx.z * dstride;
  const int64_t n = blockIdx.y;
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= rows || 2 * c >= Kpad) return;
  const double2* x = src + n * K;
  const int e = ex[n];
  uint32_t* h0 = (uint32_t*)(hi + 2 * n * ldo);
  uint32_t* l0 = (uint32_t*)(lo + 2 * n * ldo);
  uint32_t* h1 = (uint32_t*)(hi + (2 * n + 1) * ldo);
  uint32_t* l1 = (uint32_t*)(lo + (2 * n + 1) * ldo);
  {
    double re = 0.0, im = 0.0;
    if (c < K) {
      const double2 v = x[c];
      re = v.x;
      im = v.y;
    }
    uint16_t hr, lr, hi_, li, hn, ln;
    pieces(fmt, re, e, hr, lr);
    pieces(fmt, im, e, hi_, li);
    pieces(fmt, -im, e, hn, ln);
    h0[c] = (uint32_t)hr | ((uint32_t)hi_ << 16);
    l0[c] = (uint32_t)lr | ((uint32_t)li << 16);
    h1[c] = (uint32_t)hn | ((uint32_t)hr << 16);
    l1[c] = (uint32_t)ln | ((uint32_t)lr << 16);
  }
}

// Doubled operand of C = A B^T where B[n][k] = src[k][n] (K rows of N complex, row
// stride N): rows 2n = (re, -im), 2n+1 = (im, re) of 16-bit pieces with one exponent
// e for the whole operand, transposed through shared memory.  Grid (N/32, K/32).
__global__ void half_embed_t_kernel(const double2* __restrict__ src, int64_t K, int64_t N, uint16_t* hi, uint16_t* lo,
                                    int64_t Kpad, int fmt, int e, int64_t kin, int64_t kout, const __grid_constant__ SrcList list,
                                    int64_t dstride) {
  dep_wait();
  src += list.off[blockIdx.z];
  hi += blockIdx.z * dstride;
  lo += blockIdx.z * dstride;
  __shared__ double2 tile[32][33];
  const int64_t k0 = blockIdx.y * 32, nb = blockIdx.x * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  for (int r = ty; r < 32; r += 8) {
    const int64_t k = k0 + r, n = nb + tx;
    tile[r][tx] = (k < K && n < N) ? src[k * N + n] : make_double2(0, 0);
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int64_t n = nb + r, k = k0 + tx;
    if (n >= N || k >= K) continue;
    const double2 v = tile[tx][r];
    const int64_t kd = kin > 0 ? (k % kin) * kout + k / kin : k;   // K index in the operand
    uint16_t a, b, c, a2, b2, c2;
    pieces(fmt, v.x, e, a, a2);
    pieces(fmt, -v.y, e, b, b2);
    pieces(fmt, v.y, e, c, c2);
    *(uint32_t*)(hi + (2 * n) * Kpad + 2 * kd) = (uint32_t)a | ((uint32_t)b << 16);
    *(uint32_t*)(lo + (2 * n) * Kpad + 2 * kd) = (uint32_t)a2 | ((uint32_t)b2 << 16);
    *(uint32_t*)(hi + (2 * n + 1) * Kpad + 2 * kd) = (uint32_t)c | ((uint32_t)a << 16);
    *(uint32_t*)(lo + (2 * n + 1) * Kpad + 2 * kd) = (uint32_t)c2 | ((uint32_t)a2 << 16);
  }
  // zero padding columns [2K, Kpad), by the first column of blocks
  if (blockIdx.y == 0) {
    for (int r = ty; r < 32; r += 8) {
      const int64_t n = nb + r;
      if (n >= N) continue;
      for (int64_t cc = 2 * K + tx; cc < Kpad; cc += 32) {
        hi[(2 * n) * Kpad + cc] = 0; hi[(2 * n + 1) * Kpad + cc] = 0;
        lo[(2 * n) * Kpad + cc] = 0; lo[(2 * n + 1) * Kpad + cc] = 0;
      }
    }
  }
}

// Batched doubled operands of the nao x nao matrices src[z] (z < count, at src + z*ss
// complex elements; ss may be negative): plain = 0 gives the operand of C = A conj(B)^T
// (rows 2n = (re, im), 2n+1 = (-im, re)), plain = 1 that of C = A B^T (rows 2n =
// (re, -im), 2n+1 = (im, re)).  One exponent per matrix from its max |re|, |im|
// (ex[z]).  One block per matrix.
__global__ void __launch_bounds__(256) half_embed_mats_kernel(const double2* __restrict__ src, int64_t ss, int64_t rows,
                                                              int64_t K, uint16_t* hi, uint16_t* lo, int64_t Kpad,
                                                              int64_t ds, int fmt, int plain, int* ex) {
  dep_wait();
  __shared__ double red[8];
  const int64_t z = blockIdx.x;
  const double2* x = src + z * ss;
  float mf = 0.f;
  for (int64_t i = threadIdx.x; i < rows * K; i += blockDim.x)
    mf = fmaxf(mf, fmaxf(fabsf((float)x[i].x), fabsf((float)x[i].y)));
  double m = wmax((double)mf);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < 8 ? red[threadIdx.x] : 0.0;
    v = wmax(v);
    if (threadIdx.x == 0) red[0] = v;
  }
  __syncthreads();
  const int e = bound_exp(red[0], 0);
  if (threadIdx.x == 0) ex[z] = e;
  uint16_t* H = hi + z * ds;
  uint16_t* L = lo + z * ds;
  const int64_t half = Kpad / 2;
  for (int64_t i = threadIdx.x; i < rows * half; i += blockDim.x) {
    const int64_t n = i / half, c = i - n * half;
    double re = 0.0, im = 0.0;
    if (c < K) {
      const double2 v = x[n * K + c];
      re = v.x;
      im = v.y;
    }
    uint16_t hr, lr, hi_, li, hn, ln;
    pieces(fmt, re, e, hr, lr);
    pieces(fmt, im, e, hi_, li);
    pieces(fmt, -im, e, hn, ln);
    uint32_t* h0 = (uint32_t*)(H + 2 * n * Kpad);
    uint32_t* l0 = (uint32_t*)(L + 2 * n * Kpad);
    uint32_t* h1 = (uint32_t*)(H + (2 * n + 1) * Kpad);
    uint32_t* l1 = (uint32_t*)(L + (2 * n + 1) * Kpad);
    if (plain) {
      h0[c] = (uint32_t)hr | ((uint32_t)hn << 16);
      l0[c] = (uint32_t)lr | ((uint32_t)ln << 16);
      h1[c] = (uint32_t)hi_ | ((uint32_t)hr << 16);
      l1[c] = (uint32_t)li | ((uint32_t)lr << 16);
    } else {
      h0[c] = (uint32_t)hr | ((uint32_t)hi_ << 16);
      l0[c] = (uint32_t)lr | ((uint32_t)li << 16);
      h1[c] = (uint32_t)hn | ((uint32_t)hr << 16);
      l1[c] = (uint32_t)ln | ((uint32_t)lr << 16);
    }
  }
}

// ------------------------------------------------------------------ norms and bounds

// atomic max of non-negative floats through their (order-preserving) bit patterns
__device__ __forceinline__ void atomic_fmax_pos(float* p, float v) { atomicMax((int*)p, __float_as_int(v)); }

// Per auxiliary index Q over every (k, k') slab of V [nk*nk][naux][nao][nao]:
// vmax[Q] = max |V_da(Q)| and vrs[Q] = max_d sum_a |V_da(Q)| (moduli).  Rounded up
// by a relative 1e-6 so that the float results bound the double values.
__global__ void v_norms_kernel(const double2* __restrict__ V, int64_t nslab, int naux, int nao, float* vmax,
                               float* vrs) {
  const int64_t rowsall = nslab * naux * nao;
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  for (int64_t r = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); r < rowsall; r += (int64_t)gridDim.x * warps) {
    const int Q = (int)((r / nao) % naux);
    const double2* x = V + r * nao;
    double m = 0.0, s = 0.0;
    for (int a = lane; a < nao; a += 32) {
      const double v = cabs2(x[a]);
      m = fmax(m, v);
      s += v;
    }
    m = wmax(m);
    s = wsum(s);
    if (lane == 0) {
      atomic_fmax_pos(vmax + Q, (float)(m * (1 + 1e-6)));
      atomic_fmax_pos(vrs + Q, (float)(s * (1 + 1e-6)));
    }
  }
}

// Per tau over every k of G [ntau][nk][nao][nao]: gmax[t] = max |G_ab(t)|,
// grs[t] = max_c sum_d |G_cd(t)| (moduli), rounded up as above.  Grid (blocks, ntau).
__global__ void g_norms_kernel(const double2* __restrict__ G, int nk, int nao, float* gmax, float* grs) {
  const int t = blockIdx.y;
  const int64_t rows = (int64_t)nk * nao;
  const int warps = blockDim.x >> 5, lane = threadIdx.x & 31;
  const double2* Gt = G + (int64_t)t * rows * nao;
  for (int64_t r = (int64_t)blockIdx.x * warps + (threadIdx.x >> 5); r < rows; r += (int64_t)gridDim.x * warps) {
    const double2* x = Gt + r * nao;
    double m = 0.0, s = 0.0;
    for (int a = lane; a < nao; a += 32) {
      const double v = cabs2(x[a]);
      m = fmax(m, v);
      s += v;
    }
    m = wmax(m);
    s = wsum(s);
    if (lane == 0) {
      atomic_fmax_pos(gmax + t, (float)(m * (1 + 1e-6)));
      atomic_fmax_pos(grs + t, (float)(s * (1 + 1e-6)));
    }
  }
}

// Row exponents of the P~0 chain intermediates (one per (tau, Q)):
//   Y[t][Q] = V(Q) G(t):          |Y_db| <= vrs[Q] gmax_p[t]                  -> eY
//   Z[t][Q] = G(-t) V(Q) G(t):    |Z_cb| <= grs_m[ntau-1-t] vrs[Q] gmax_p[t]  -> eZ
// (gmax_p from the G(t) factor, grs_m from the G(-t) factor; G(-t_j) = -G(t_{ntau-1-j})).
__global__ void polar_exps_kernel(const float* vrs, const float* gmax_p, const float* grs_m, int ntau, int naux,
                                  int* eY, int* eZ) {
  const int64_t n = (int64_t)ntau * naux;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const int t = (int)(i / naux), Q = (int)(i - (int64_t)t * naux);
    const double y = (double)vrs[Q] * (double)gmax_p[t];
    eY[i] = bound_exp(y, 1);
    eZ[i] = bound_exp(y * (double)grs_m[ntau - 1 - t], 1);
  }
}

// Row exponent of the Sigma~ chain's Y[t][i][(Q', b)] (uniform over Q'):
// |Y| <= max_Q' 2^(eX[t][Q'] + 15) grs[t], with eX the exponents of X's rows.
__global__ void sigma_exps_kernel(const int* eX, int shift, const float* grs, int ntau, int naux, int* eY3) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ntau) return;
  int m = -100000;
  for (int q = 0; q < naux; ++q) m = max(m, eX[(int64_t)t * naux + q]);
  int E = 0;
  if (grs[t] > 0.f) frexpf(grs[t], &E);
  eY3[t] = m + shift + E + 1;
}

__global__ void max_exp_kernel(const float* v, int n, int* out) {
  float m = 0.f;
  for (int i = 0; i < n; ++i) m = fmaxf(m, v[i]);
  int E = 0;
  if (m > 0.f) frexpf(m, &E);
  out[0] = E;
}

__global__ void row_exps_kernel(const float* v, int n, int* out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = bound_exp((double)v[i], 0);
}

static inline unsigned nblk(int64_t rows, int per) {
  const int64_t b = (rows + per - 1) / per;
  return (unsigned)(b < 1 ? 1 : b);
}

// Gathers n blocks of 16-bit pieces (hi and lo planes, `words` 16-byte words each) and
// their exponents (ecount each) from block indices list.off[i] into consecutive blocks.
__global__ void __launch_bounds__(256) gather_blocks_kernel(const uint4* __restrict__ shi, const uint4* __restrict__ slo,
                                                            const int* __restrict__ se, uint4* dhi, uint4* dlo, int* de,
                                                            int64_t words, int64_t ecount, const __grid_constant__ SrcList list) {
  dep_wait();
  const int64_t i = blockIdx.y, src = list.off[i];
  for (int64_t w = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; w < words; w += (int64_t)gridDim.x * blockDim.x) {
    dhi[i * words + w] = shi[src * words + w];
    dlo[i * words + w] = slo[src * words + w];
  }
  if (blockIdx.x == 0)
    for (int64_t e = threadIdx.x; e < ecount; e += blockDim.x) de[i * ecount + e] = se[src * ecount + e];
}

// ------------------------------------------------------------------ launch wrappers

static SrcList one_src() {
  SrcList l{};
  l.n = 1;
  return l;
}

cudaError_t half_rows_multi(const double2* src, const int64_t* offs, int n, int64_t rows, int64_t K, int64_t ld,
                            bool conj, void* hi, void* lo, int64_t Kpad, int64_t ldo, int64_t dstride, int fmt,
                            int* ex, int* exs, int64_t estride, cudaStream_t st) {
  if (Kpad % 64 || rows <= 0 || n < 1 || n > kSrcListMax) return cudaErrorInvalidValue;
  SrcList l{};
  l.n = n;
  for (int i = 0; i < n; ++i) l.off[i] = offs ? offs[i] : 0;
  return launch_dep(half_rows_kernel, dim3(nblk(rows, 8), (unsigned)n), dim3(256), st, src, rows, K, ld,
                    conj ? 1 : 0, (uint16_t*)hi, (uint16_t*)lo, Kpad, ldo > 0 ? ldo : Kpad, fmt, ex, exs, l, dstride,
                    estride);
}

cudaError_t half_rows(const double2* src, int64_t rows, int64_t K, int64_t ld, bool conj, void* hi, void* lo,
                      int64_t Kpad, int64_t ldo, int fmt, int* ex, int* exs, cudaStream_t st) {
  if (Kpad % 64 || rows <= 0) return cudaErrorInvalidValue;
  return launch_dep(half_rows_kernel, dim3(nblk(rows, 8)), dim3(256), st, src, rows, K, ld, conj ? 1 : 0, (uint16_t*)hi,
                    (uint16_t*)lo, Kpad, ldo > 0 ? ldo : Kpad, fmt, ex, exs, one_src(), (int64_t)0, (int64_t)0);
}

cudaError_t half_embed_conj_multi(const double2* src, const int64_t* offs, int n, int64_t rows, int64_t K, void* hi,
                                  void* lo, int64_t Kpad, int64_t ldo, int64_t dstride, int fmt, const int* ex,
                                  cudaStream_t st) {
  if (Kpad % 64 || rows <= 0 || rows > 65535 || n < 1 || n > kSrcListMax) return cudaErrorInvalidValue;
  SrcList l{};
  l.n = n;
  for (int i = 0; i < n; ++i) l.off[i] = offs ? offs[i] : 0;
  dim3 grid(nblk(Kpad / 2, 256), (unsigned)rows, (unsigned)n);
  return launch_dep(half_embed_conj_kernel, grid, dim3(256), st, src, rows, K, (uint16_t*)hi, (uint16_t*)lo, Kpad,
                    ldo > 0 ? ldo : Kpad, fmt, ex, l, dstride);
}

cudaError_t half_embed_conj(const double2* src, int64_t rows, int64_t K, void* hi, void* lo, int64_t Kpad,
                            int64_t ldo, int fmt, const int* ex, cudaStream_t st) {
  if (Kpad % 64 || rows <= 0 || rows > 65535) return cudaErrorInvalidValue;
  dim3 grid(nblk(Kpad / 2, 256), (unsigned)rows);
  return launch_dep(half_embed_conj_kernel, grid, dim3(256), st, src, rows, K, (uint16_t*)hi, (uint16_t*)lo, Kpad,
                    ldo > 0 ? ldo : Kpad, fmt, ex, one_src(), (int64_t)0);
}

cudaError_t half_embed_t_multi(const double2* src, const int64_t* offs, int n, int64_t K, int64_t N, void* hi,
                               void* lo, int64_t Kpad, int64_t dstride, int fmt, int e, cudaStream_t st, int64_t kin,
                               int64_t kout) {
  if (Kpad % 64 || K <= 0 || N <= 0 || n < 1 || n > kSrcListMax) return cudaErrorInvalidValue;
  if (kin > 0 && (K % kin || kout * kin != K)) return cudaErrorInvalidValue;   // a permutation of [0, K)
  SrcList l{};
  l.n = n;
  for (int i = 0; i < n; ++i) l.off[i] = offs ? offs[i] : 0;
  dim3 grid((unsigned)((N + 31) / 32), (unsigned)((K + 31) / 32), (unsigned)n);
  return launch_dep(half_embed_t_kernel, grid, dim3(256), st, src, K, N, (uint16_t*)hi, (uint16_t*)lo, Kpad, fmt, e,
                    kin, kout, l, dstride);
}

cudaError_t half_embed_t(const double2* src, int64_t K, int64_t N, void* hi, void* lo, int64_t Kpad, int fmt, int e,
                         cudaStream_t st, int64_t kin, int64_t kout) {
  if (Kpad % 64 || K <= 0 || N <= 0) return cudaErrorInvalidValue;
  if (kin > 0 && (K % kin || kout * kin != K)) return cudaErrorInvalidValue;   // a permutation of [0, K)
  dim3 grid((unsigned)((N + 31) / 32), (unsigned)((K + 31) / 32), 1);
  return launch_dep(half_embed_t_kernel, grid, dim3(256), st, src, K, N, (uint16_t*)hi, (uint16_t*)lo, Kpad, fmt, e,
                    kin, kout, one_src(), (int64_t)0);
}

cudaError_t half_embed_mats(const double2* src, int64_t count, int64_t ss, int64_t rows, int64_t K, void* hi,
                            void* lo, int64_t Kpad, int64_t ds, int fmt, bool plain, int* ex, cudaStream_t st) {
  if (Kpad % 64 || count <= 0 || count > INT32_MAX) return cudaErrorInvalidValue;
  return launch_dep(half_embed_mats_kernel, dim3((unsigned)count), dim3(256), st, src, ss, rows, K, (uint16_t*)hi,
                    (uint16_t*)lo, Kpad, ds, fmt, plain ? 1 : 0, ex);
}

cudaError_t v_norms(const double2* V, int64_t nslab, int naux, int nao, float* vmax, float* vrs, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(vmax, 0, (size_t)naux * 4, st);
  if (!e) e = cudaMemsetAsync(vrs, 0, (size_t)naux * 4, st);
  if (e) return e;
  v_norms_kernel<<<152 * 8, 256, 0, st>>>(V, nslab, naux, nao, vmax, vrs);
  return cudaGetLastError();
}

cudaError_t g_norms(const double2* G, int ntau, int nk, int nao, float* gmax, float* grs, cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(gmax, 0, (size_t)ntau * 4, st);
  if (!e) e = cudaMemsetAsync(grs, 0, (size_t)ntau * 4, st);
  if (e) return e;
  const int64_t rows = (int64_t)nk * nao;
  dim3 grid(nblk(rows, 8 * 4) > 64 ? 64 : nblk(rows, 8 * 4), (unsigned)ntau);
  g_norms_kernel<<<grid, 256, 0, st>>>(G, nk, nao, gmax, grs);
  return cudaGetLastError();
}

cudaError_t polar_exps(const float* vrs, const float* gmax_p, const float* grs_m, int ntau, int naux, int* eY, int* eZ,
                       cudaStream_t st) {
  polar_exps_kernel<<<nblk((int64_t)ntau * naux, 256), 256, 0, st>>>(vrs, gmax_p, grs_m, ntau, naux, eY, eZ);
  return cudaGetLastError();
}

cudaError_t sigma_exps(const int* eX, int shift, const float* grs, int ntau, int naux, int* eY3, cudaStream_t st) {
  sigma_exps_kernel<<<nblk(ntau, 128), 128, 0, st>>>(eX, shift, grs, ntau, naux, eY3);
  return cudaGetLastError();
}

cudaError_t max_exp(const float* v, int n, int* out, cudaStream_t st) {
  max_exp_kernel<<<1, 1, 0, st>>>(v, n, out);
  return cudaGetLastError();
}

cudaError_t row_exps(const float* v, int n, int* out, cudaStream_t st) {
  row_exps_kernel<<<nblk(n, 256), 256, 0, st>>>(v, n, out);
  return cudaGetLastError();
}

}  // namespace gwk

namespace gwk {
cudaError_t gather_blocks(const void* shi, const void* slo, const int* se, void* dhi, void* dlo, int* de,
                          int64_t block_bytes, int64_t ecount, const int* idx, int n, cudaStream_t st) {
  if (block_bytes % 16 || n < 1 || n > kSrcListMax) return cudaErrorInvalidValue;
  SrcList l{};
  l.n = n;
  for (int i = 0; i < n; ++i) l.off[i] = idx[i];
  const int64_t words = block_bytes / 16;
  const unsigned gx = (unsigned)std::min<int64_t>((words + 255) / 256, 152);
  return launch_dep(gather_blocks_kernel, dim3(gx, (unsigned)n), dim3(256), st, (const uint4*)shi, (const uint4*)slo,
                    se, (uint4*)dhi, (uint4*)dlo, de, words, ecount, l);
}
}  // namespace gwk
