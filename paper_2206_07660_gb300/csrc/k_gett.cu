// Generic batched strided complex contraction (SIMT, fp64 or fp32 FMA).
//
// Every contraction of the method -- the two GEMM chains of P~0 (Eq.
// tilde_P0_tau) and Sigma~ (Eq. tilde_sigma2), the exchange term (Eq. HF_K),
// the tau <-> Matsubara transforms and the rank-nb updates of the screened
// solve -- is a product of two tensor slices whose row, column and reduction
// indices are each made of at most two strided parts.  One tiled kernel reads
// all of them in place (no transposition copies).  On GB300 the fp64 pipe is
// the bound for the fp64 instantiation, so the tile is sized for register
// reuse (4x4 complex outputs per thread), not for bandwidth.
#include "gw_internal.cuh"

namespace gwk {

template <typename S> struct C2;
template <> struct C2<double> { using t = double2; };
template <> struct C2<float>  { using t = float2; };

template <typename S, typename T>
__device__ __forceinline__ typename C2<S>::t cvt(T v) {
  typename C2<S>::t r; r.x = (S)v.x; r.y = (S)v.y; return r;
}
template <typename T, typename S>
__device__ __forceinline__ T cvt_out(S re, S im) { T r; r.x = (decltype(r.x))re; r.y = (decltype(r.y))im; return r; }

__device__ __forceinline__ int64_t off2(int64_t i, const Idx2& d) {
  if (i < d.inner) return i * d.s0;
  int64_t o = i / d.inner;
  return o * d.s1 + (i - o * d.inner) * d.s0;
}

constexpr int BM = 64, BN = 64, BK = 16, NT = 256;

template <typename TA, typename TB, typename TC, typename S>
__global__ void __launch_bounds__(NT) gett_kernel(GettDesc d, const TA* __restrict__ A,
                                                  const TB* __restrict__ B, TC* C,
                                                  typename C2<S>::t* ws) {
  using CS = typename C2<S>::t;
  __shared__ CS As[BK][BM];
  __shared__ CS Bs[BK][BN];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.y * BM, n0 = (int64_t)blockIdx.x * BN;
  const int ks = d.ksplit > 1 ? d.ksplit : 1;
  // loader geometry: which of (m,k) / (k,n) is the contiguous index
  const bool a_kfast = (d.ak.s0 == 1);
  const bool b_nfast = (d.bn.s0 == 1);
  const S sa = d.conjA ? (S)-1 : (S)1, sb = d.conjB ? (S)-1 : (S)1;

  for (int64_t zz = blockIdx.z; zz < d.Z * ks; zz += gridDim.z) {
    const int64_t z = zz / ks;
    const int split = (int)(zz - z * ks);
    const TA* Az = A + off2(z, d.az);
    const TB* Bz = B + off2(z, d.bz);
    int64_t kbeg = 0, kend = d.K;
    if (ks > 1) {
      int64_t kc = (d.K + ks - 1) / ks;
      kc = (kc + BK - 1) / BK * BK;
      kbeg = split * kc;
      kend = min(d.K, kbeg + kc);
    }
    // per-thread load coordinates
    int am[4], ak[4], bkk[4], bnn[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      if (a_kfast) { ak[r] = tid % BK; am[r] = tid / BK + 16 * r; }
      else         { am[r] = tid % BM; ak[r] = tid / BM + 4 * r; }
      if (b_nfast) { bnn[r] = tid % BN; bkk[r] = tid / BN + 4 * r; }
      else         { bkk[r] = tid % BK; bnn[r] = tid / BK + 16 * r; }
    }
    int64_t aoff_m[4], boff_n[4];
    bool aok_m[4], bok_n[4];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int64_t m = m0 + am[r];
      aok_m[r] = m < d.M;
      aoff_m[r] = aok_m[r] ? off2(m, d.am) : 0;
      int64_t n = n0 + bnn[r];
      bok_n[r] = n < d.N;
      boff_n[r] = bok_n[r] ? off2(n, d.bn) : 0;
    }
    CS acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) { acc[i][j].x = 0; acc[i][j].y = 0; }

    CS ra[4], rb[4];
    auto gload = [&](int64_t kt) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        int64_t k = kt + ak[r];
        CS v; v.x = 0; v.y = 0;
        if (aok_m[r] && k < kend) { v = cvt<S>(__ldg(Az + aoff_m[r] + off2(k, d.ak))); v.y *= sa; }
        ra[r] = v;
        int64_t kb = kt + bkk[r];
        CS w; w.x = 0; w.y = 0;
        if (bok_n[r] && kb < kend) { w = cvt<S>(__ldg(Bz + boff_n[r] + off2(kb, d.bk))); w.y *= sb; }
        rb[r] = w;
      }
    };
    if (kbeg < kend) gload(kbeg);
    for (int64_t kt = kbeg; kt < kend; kt += BK) {
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        As[ak[r]][am[r]] = ra[r];
        Bs[bkk[r]][bnn[r]] = rb[r];
      }
      __syncthreads();
      if (kt + BK < kend) gload(kt + BK);
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        CS a[4], b[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            acc[i][j].x = fma(a[i].x, b[j].x, acc[i][j].x);
            acc[i][j].x = fma(-a[i].y, b[j].y, acc[i][j].x);
            acc[i][j].y = fma(a[i].x, b[j].y, acc[i][j].y);
            acc[i][j].y = fma(a[i].y, b[j].x, acc[i][j].y);
          }
      }
      __syncthreads();
    }
    // epilogue
    if (ks > 1) {
      CS* W = ws + ((int64_t)split * d.Z + z) * d.M * d.N;
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int64_t m = m0 + ty + 16 * i;
        if (m >= d.M) continue;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int64_t n = n0 + tx + 16 * j;
          if (n < d.N) W[m * d.N + n] = acc[i][j];
        }
      }
    } else {
      TC* Cz = C + off2(z, d.cz);
      const bool rd = (d.beta.x != 0.0 || d.beta.y != 0.0);
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        int64_t m = m0 + ty + 16 * i;
        if (m >= d.M) continue;
        int64_t cmo = off2(m, d.cm);
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          int64_t n = n0 + tx + 16 * j;
          if (n >= d.N) continue;
          TC* p = Cz + cmo + off2(n, d.cn);
          // epilogue in double: a fp32 product slab is added to an fp64 C exactly
          double ax = (double)acc[i][j].x, ay = (double)acc[i][j].y;
          double re = d.alpha.x * ax - d.alpha.y * ay;
          double im = d.alpha.x * ay + d.alpha.y * ax;
          if (rd) {
            double cx = (double)p->x, cy = (double)p->y;
            re += d.beta.x * cx - d.beta.y * cy;
            im += d.beta.x * cy + d.beta.y * cx;
          }
          *p = cvt_out<TC, double>(re, im);
        }
      }
    }
  }
}

// C(m,n) = alpha * sum_s W[s][z][m][n] + beta * C(m,n), summed in split order.
template <typename TC, typename S>
__global__ void splitk_reduce(GettDesc d, const typename C2<S>::t* __restrict__ ws, TC* C) {
  using CS = typename C2<S>::t;
  const int64_t MN = d.M * d.N;
  const int64_t total = MN * d.Z;
  const bool rd = (d.beta.x != 0.0 || d.beta.y != 0.0);
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < total;
       t += (int64_t)gridDim.x * blockDim.x) {
    int64_t z = t / MN, mn = t - z * MN, m = mn / d.N, n = mn - m * d.N;
    double re = 0, im = 0;
    for (int s = 0; s < d.ksplit; ++s) {
      CS v = ws[((int64_t)s * d.Z + z) * MN + mn];
      re += (double)v.x; im += (double)v.y;
    }
    TC* p = C + off2(z, d.cz) + off2(m, d.cm) + off2(n, d.cn);
    double orr = d.alpha.x * re - d.alpha.y * im;
    double oi = d.alpha.x * im + d.alpha.y * re;
    if (rd) {
      double cr = (double)p->x, ci = (double)p->y;
      orr += d.beta.x * cr - d.beta.y * ci;
      oi += d.beta.x * ci + d.beta.y * cr;
    }
    p->x = (decltype(p->x))orr; p->y = (decltype(p->y))oi;
  }
}

size_t gett_ws_bytes(const GettDesc& d, Ty acc) {
  if (d.ksplit <= 1) return 0;
  return (size_t)d.ksplit * d.Z * d.M * d.N * (acc == Ty::C128 ? 16 : 8);
}

template <typename TA, typename TB, typename TC, typename S>
static cudaError_t launch(const GettDesc& d, const void* A, const void* B, void* C, void* ws,
                          cudaStream_t st) {
  if (d.M <= 0 || d.N <= 0 || d.Z <= 0) return cudaSuccess;
  int ks = d.ksplit > 1 ? d.ksplit : 1;
  dim3 grid((unsigned)((d.N + BN - 1) / BN), (unsigned)((d.M + BM - 1) / BM),
            (unsigned)(d.Z * ks < 65535 ? d.Z * ks : 65535));
  if (grid.y > 65535) return cudaErrorInvalidConfiguration;
  gett_kernel<TA, TB, TC, S><<<grid, NT, 0, st>>>(d, (const TA*)A, (const TB*)B, (TC*)C,
                                                  (typename C2<S>::t*)ws);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || ks == 1) return e;
  int64_t total = d.M * d.N * d.Z;
  int64_t nb = (total + 255) / 256; int blocks = (int)(nb < 152 * 16 ? nb : 152 * 16);
  splitk_reduce<TC, S><<<blocks, 256, 0, st>>>(d, (const typename C2<S>::t*)ws, (TC*)C);
  return cudaGetLastError();
}

template <typename TA, typename TB, typename TC>
static cudaError_t disp_acc(const GettDesc& d, const void* A, const void* B, void* C, Ty acc, void* ws,
                            cudaStream_t st) {
  return acc == Ty::C128 ? launch<TA, TB, TC, double>(d, A, B, C, ws, st)
                         : launch<TA, TB, TC, float>(d, A, B, C, ws, st);
}
template <typename TA, typename TB>
static cudaError_t disp_c(const GettDesc& d, const void* A, const void* B, void* C, Ty tc, Ty acc,
                          void* ws, cudaStream_t st) {
  return tc == Ty::C128 ? disp_acc<TA, TB, double2>(d, A, B, C, acc, ws, st)
                        : disp_acc<TA, TB, float2>(d, A, B, C, acc, ws, st);
}
template <typename TA>
static cudaError_t disp_b(const GettDesc& d, const void* A, const void* B, Ty tb, void* C, Ty tc, Ty acc,
                          void* ws, cudaStream_t st) {
  return tb == Ty::C128 ? disp_c<TA, double2>(d, A, B, C, tc, acc, ws, st)
                        : disp_c<TA, float2>(d, A, B, C, tc, acc, ws, st);
}

cudaError_t gett(const GettDesc& d, const void* A, Ty ta, const void* B, Ty tb, void* C, Ty tc, Ty acc,
                 void* ws, size_t ws_bytes, cudaStream_t st) {
  if (d.ksplit > 1 && (ws == nullptr || ws_bytes < gett_ws_bytes(d, acc)))
    return cudaErrorInvalidValue;
  return ta == Ty::C128 ? disp_b<double2>(d, A, B, tb, C, tc, acc, ws, st)
                        : disp_b<float2>(d, A, B, tb, C, tc, acc, ws, st);
}

}  // namespace gwk
