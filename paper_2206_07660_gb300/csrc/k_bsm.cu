// Batched small complex products with one operand shared across a group:
//   C[g][e] = alpha * opA(A[g][e]) * opB(B[g][e]),  M, N, K <= 64,
// where A or B does not depend on e (it is loaded into shared memory once per
// block and reused for every e the block owns).  These are the nao x nao x nao
// steps of the GEMM chains of Eqs. tilde_P0_tau and tilde_sigma2 (e.g.
// G^k(-tau) Y_Q for all Q at one tau) and of Eq. HF_K.
//
// Each thread owns a 4 x 4 micro-tile of one product; a block of 256 threads
// works on EP = 256 / (ceil(M/4) ceil(N/4)) products at a time, so small
// orders (nao 8..26) still keep every thread busy.  fp32 FMA on complex64
// data; the output is complex64, or TF32 hi/lo float planes (x = hi + lo)
// that feed the tensor-core GEMM directly.
#include "gw_internal.cuh"

namespace gwk {

__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

constexpr int BSM_MAX = 64;

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

// Copies `ne` row-major operands (R rows, Cc columns; element (r, c) at
// src + e*es + r*rs + c*cs) into shared memory [e][r][LD]: one warp per row,
// lanes along the columns.  Conjugation is applied later, at use.
__device__ __forceinline__ void load_rows_async(float2* dst, int dst_stride, const float2* src, int64_t es,
                                                int64_t rs, int64_t cs, int ne, int R, int Cc, int LD) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int row = warp; row < ne * R; row += 8) {
    const int e = row / R, r = row - e * R;
    const float2* s = src + e * es + (int64_t)r * rs;
    float2* d = dst + e * dst_stride + r * LD;
    for (int c = lane; c < Cc; c += 32) cp_async8(d + c, s + (int64_t)c * cs);
  }
}

template <bool CA, bool CB>
__device__ __forceinline__ void bsm_compute(const float2* As, int LDA, const float2* Bs, int LDB, int K, int M, int N,
                                            int m0, int n0, float2 (&acc)[4][4]) {
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
  const int mi = M - m0 < 4 ? M - m0 : 4, nj = N - n0 < 4 ? N - n0 : 4;
  for (int k = 0; k < K; ++k) {
    float2 a[4], b[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      a[i] = i < mi ? As[(m0 + i) * LDA + k] : make_float2(0.f, 0.f);
      if (CA) a[i].y = -a[i].y;
    }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      b[j] = j < nj ? Bs[k * LDB + n0 + j] : make_float2(0.f, 0.f);
      if (CB) b[j].y = -b[j].y;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        acc[i][j].x = fmaf(a[i].x, b[j].x, acc[i][j].x);
        acc[i][j].x = fmaf(-a[i].y, b[j].y, acc[i][j].x);
        acc[i][j].y = fmaf(a[i].x, b[j].y, acc[i][j].y);
        acc[i][j].y = fmaf(a[i].y, b[j].x, acc[i][j].y);
      }
  }
}

template <bool CA, bool CB>
__global__ void __launch_bounds__(256, 2) bsm_kernel(BsmDesc d) {
  extern __shared__ float2 sm[];
  const int tid = threadIdx.x;
  const int tm = (d.M + 3) / 4, tn = (d.N + 3) / 4, T = tm * tn;
  const int EP = 256 / T < 1 ? 1 : 256 / T;
  // layout: shared operand, then two buffers of EP varying operands (double buffering)
  const int LDA = d.K + 1, LDB = d.N + 1;
  const int shared_sz = d.a_shared ? d.M * LDA : d.K * LDB;
  const int vary_sz = d.a_shared ? d.K * LDB : d.M * LDA;
  float2* S = sm;
  float2* const Vb0 = sm + shared_sz;
  const int vbuf_sz = EP * vary_sz;
  const int el = tid / T, ti = (tid % T) / tn, tj = (tid % T) % tn;
  const bool active = el < EP;
  // varying-operand geometry
  const int vR = d.a_shared ? d.K : d.M, vC = d.a_shared ? d.N : d.K, vLD = d.a_shared ? LDB : LDA;
  const int64_t vrs = d.a_shared ? d.b_rs : d.a_rs, vcs = d.a_shared ? d.b_cs : d.a_cs;
  const int64_t ves = d.a_shared ? d.b_es : d.a_es;
  const int per = d.per_block;
  const int64_t blocks_per_group = (d.E + per - 1) / per;
  for (int64_t blk = blockIdx.x; blk < d.G * blocks_per_group; blk += gridDim.x) {
    const int64_t g = blk / blocks_per_group;
    const int64_t e0 = (blk - g * blocks_per_group) * per;
    const int64_t e1 = e0 + per < d.E ? e0 + per : d.E;
    const float2* vbase = d.a_shared ? d.B + g * d.b_gs : d.A + g * d.a_gs;
    __syncthreads();
    // shared operand of the group, and the first pass of varying operands
    if (d.a_shared) load_rows_async(S, 0, d.A + g * d.a_gs, 0, d.a_rs, d.a_cs, 1, d.M, d.K, LDA);
    else load_rows_async(S, 0, d.B + g * d.b_gs, 0, d.b_rs, d.b_cs, 1, d.K, d.N, LDB);
    {
      const int ne0 = (int)((e1 - e0) < EP ? (e1 - e0) : EP);
      load_rows_async(Vb0, vary_sz, vbase + e0 * ves, ves, vrs, vcs, ne0, vR, vC, vLD);
    }
    cp_async_commit();
    int buf = 0;
    for (int64_t eb = e0; eb < e1; eb += EP) {
      const int ne = (int)((e1 - eb) < EP ? (e1 - eb) : EP);
      cp_async_wait_all();
      __syncthreads();   // pass eb resident; the other buffer is free
      const int64_t en = eb + EP;
      if (en < e1) {
        const int nn = (int)((e1 - en) < EP ? (e1 - en) : EP);
        load_rows_async(Vb0 + (buf ^ 1) * vbuf_sz, vary_sz, vbase + en * ves, ves, vrs, vcs, nn, vR, vC, vLD);
      }
      cp_async_commit();
      if (active && el < ne) {
        const float2* Vcur = Vb0 + buf * vbuf_sz + el * vary_sz;
        const float2* As = d.a_shared ? S : Vcur;
        const float2* Bs = d.a_shared ? Vcur : S;
        const int m0 = ti * 4, n0 = tj * 4;
        float2 acc[4][4];
        bsm_compute<CA, CB>(As, LDA, Bs, LDB, d.K, d.M, d.N, m0, n0, acc);
        const int64_t cbase = g * d.c_gs + (eb + el) * d.c_es;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int m = m0 + i;
          if (m >= d.M) continue;
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int n = n0 + j;
            if (n >= d.N) continue;
            const float re = d.alpha * acc[i][j].x, im = d.alpha * acc[i][j].y;
            const int64_t o = cbase + (int64_t)m * d.c_rs + (int64_t)n;   // complex index
            if (d.C) {
              d.C[o] = make_float2(re, im);
            } else {
              const float h0 = tf32r(re), h1 = tf32r(im);
              *(float2*)(d.Chi + 2 * o) = make_float2(h0, h1);
              *(float2*)(d.Clo + 2 * o) = make_float2(tf32r(re - h0), tf32r(im - h1));
            }
          }
        }
      }
      buf ^= 1;
    }
    cp_async_wait_all();
  }
}

cudaError_t bsm(const BsmDesc& d, cudaStream_t st) {
  if (d.M > BSM_MAX || d.N > BSM_MAX || d.K > BSM_MAX || d.M <= 0 || d.N <= 0 || d.K <= 0)
    return cudaErrorInvalidValue;
  if (!!d.a_shared == !!d.b_shared) return cudaErrorInvalidValue;   // exactly one operand is shared
  const int T = ((d.M + 3) / 4) * ((d.N + 3) / 4);
  const int EP = 256 / T < 1 ? 1 : 256 / T;
  const int shared_sz = d.a_shared ? d.M * (d.K + 1) : d.K * (d.N + 1);
  const int vary_sz = d.a_shared ? d.K * (d.N + 1) : d.M * (d.K + 1);
  const size_t sm = (size_t)(shared_sz + 2 * EP * vary_sz) * sizeof(float2);
  if (sm > 110 * 1024) return cudaErrorInvalidValue;
  const int64_t nblk = d.G * ((d.E + d.per_block - 1) / d.per_block);
  const int grid = (int)(nblk < 152 * 2 * 8 ? nblk : 152 * 2 * 8);
  auto k = d.conjA ? (d.conjB ? bsm_kernel<true, true> : bsm_kernel<true, false>)
                   : (d.conjB ? bsm_kernel<false, true> : bsm_kernel<false, false>);
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, 110 * 1024);
  if (e != cudaSuccess) return e;
  k<<<grid, 256, sm, st>>>(d);
  return cudaGetLastError();
}

}  // namespace gwk
