// Batched small complex products with one operand shared across a group:
//   C[g][e] = alpha * opA(A[g][e]) * opB(B[g][e]),  M, N, K <= 64,
// where A or B does not depend on e (it is loaded into shared memory once per
// block and reused for every e the block owns).  These are the nao x nao x nao
// steps of the GEMM chains of Eqs. tilde_P0_tau and tilde_sigma2 (e.g.
// G^k(-tau) Y_Q for all Q at one tau) and of Eq. HF_K; with K and N at most 64
// each block does a whole product per batch element instead of one small
// tile per block.  fp32 FMA on complex64 data; the output is complex64, or
// TF32 hi/lo planes (x = hi + lo) that feed the tensor-core GEMM directly.
#include "gw_internal.cuh"

namespace gwk {

__device__ __forceinline__ float tf32r(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// smem tiles: [64][65] complex (padding against bank conflicts on column reads)
constexpr int BS = 64, BSP = 65;

__global__ void __launch_bounds__(256, 2) bsm_kernel(BsmDesc d) {
  extern __shared__ float2 sm[];
  float2* As = sm;                 // A tile: [m][k]
  float2* Bs = sm + BS * BSP;      // B tile: [k][n]
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int per = d.per_block;
  const int64_t blocks_per_group = (d.E + per - 1) / per;
  for (int64_t blk = blockIdx.x; blk < d.G * blocks_per_group; blk += gridDim.x) {
    const int64_t g = blk / blocks_per_group;
    const int64_t e0 = (blk - g * blocks_per_group) * per;
    const int64_t e1 = e0 + per < d.E ? e0 + per : d.E;
    bool first = true;
    for (int64_t e = e0; e < e1; ++e) {
      // load A (if varying or first) and B (if varying or first)
      const bool loadA = first || !d.a_shared, loadB = first || !d.b_shared;
      __syncthreads();
      if (loadA) {
        const float2* A = d.A + g * d.a_gs + (d.a_shared ? 0 : e * d.a_es);
        for (int t = tid; t < d.M * d.K; t += 256) {
          int m = t / d.K, k = t - m * d.K;
          float2 v = A[(int64_t)m * d.a_rs + (int64_t)k * d.a_cs];
          if (d.conjA) v.y = -v.y;
          As[m * BSP + k] = v;
        }
      }
      if (loadB) {
        const float2* B = d.B + g * d.b_gs + (d.b_shared ? 0 : e * d.b_es);
        for (int t = tid; t < d.K * d.N; t += 256) {
          int k = t / d.N, n = t - k * d.N;
          float2 v = B[(int64_t)k * d.b_rs + (int64_t)n * d.b_cs];
          if (d.conjB) v.y = -v.y;
          Bs[k * BSP + n] = v;
        }
      }
      first = false;
      __syncthreads();
      float2 acc[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = make_float2(0.f, 0.f);
      for (int k = 0; k < d.K; ++k) {
        float2 a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[(ty + 16 * i) * BSP + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[k * BSP + tx + 16 * j];
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
      // epilogue
      const int64_t cbase = g * d.c_gs + e * d.c_es;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int m = ty + 16 * i;
        if (m >= d.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int n = tx + 16 * j;
          if (n >= d.N) continue;
          const float re = d.alpha * acc[i][j].x, im = d.alpha * acc[i][j].y;
          const int64_t o = cbase + (int64_t)m * d.c_rs + (int64_t)n;   // complex index
          if (d.C) {
            d.C[o] = make_float2(re, im);
          } else {
            float h0 = tf32r(re), h1 = tf32r(im);
            d.Chi[2 * o] = h0; d.Chi[2 * o + 1] = h1;
            d.Clo[2 * o] = tf32r(re - h0); d.Clo[2 * o + 1] = tf32r(im - h1);
          }
        }
      }
    }
  }
}

cudaError_t bsm(const BsmDesc& d, cudaStream_t st) {
  if (d.M > BS || d.N > BS || d.K > BS || d.M <= 0 || d.N <= 0 || d.K <= 0) return cudaErrorInvalidValue;
  const size_t sm = 2 * (size_t)BS * BSP * sizeof(float2);
  cudaError_t e = cudaFuncSetAttribute(bsm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
  if (e != cudaSuccess) return e;
  const int64_t nblk = d.G * ((d.E + d.per_block - 1) / d.per_block);
  const int grid = (int)(nblk < 152 * 2 * 8 ? nblk : 152 * 2 * 8);
  bsm_kernel<<<grid, 256, sm, st>>>(d);
  return cudaGetLastError();
}

}  // namespace gwk
