// Bandwidth-bound helper kernels: Hermitian symmetrisation, density matrix,
// Hartree term, mixing, identity shifts, input checks, conversions.
#include "gw_internal.cuh"

namespace gwk {

static inline int nblk(int64_t n, int t = 256, int cap = 152 * 32) {
  int64_t b = (n + t - 1) / t;
  return (int)(b < cap ? b : cap);
}

// X <- (X + X^H)/2 for `count` n x n matrices spaced `stride` apart.  Each
// block owns a tile pair (I <= J) so that both mirror tiles are read once and
// written once through shared memory (coalesced in both directions).
__global__ void __launch_bounds__(256) herm_kernel(double2* X, int n, int nt, int64_t count,
                                                   int64_t stride) {
  __shared__ double2 a[32][33];
  __shared__ double2 b[32][33];
  int p = blockIdx.x, I = 0;
  while (p >= nt - I) { p -= nt - I; ++I; }
  const int J = I + p;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
  for (int64_t mat = blockIdx.y; mat < count; mat += gridDim.y) {
    double2* M = X + mat * stride;
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int rr = ty + 8 * r;
      int i = I * 32 + rr, j = J * 32 + tx;
      if (i < n && j < n) a[rr][tx] = M[(int64_t)i * n + j];
      i = J * 32 + rr; j = I * 32 + tx;
      if (i < n && j < n) b[rr][tx] = M[(int64_t)i * n + j];
    }
    __syncthreads();
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      int rr = ty + 8 * r;
      int i = I * 32 + rr, j = J * 32 + tx;
      if (i < n && j < n) {
        double2 u = a[rr][tx], v = b[tx][rr];
        M[(int64_t)i * n + j] = make_double2(0.5 * (u.x + v.x), 0.5 * (u.y - v.y));
      }
      if (I != J) {
        i = J * 32 + rr; j = I * 32 + tx;
        if (i < n && j < n) {
          double2 u = b[rr][tx], v = a[tx][rr];
          M[(int64_t)i * n + j] = make_double2(0.5 * (u.x + v.x), 0.5 * (u.y - v.y));
        }
      }
    }
    __syncthreads();
  }
}

cudaError_t herm_batched(double2* X, int64_t n, int64_t count, int64_t stride, cudaStream_t st) {
  if (n <= 0 || count <= 0) return cudaSuccess;
  int nt = (int)((n + 31) / 32);
  int pairs = nt * (nt + 1) / 2;
  dim3 grid(pairs, (unsigned)(count < 65535 ? count : 65535));
  herm_kernel<<<grid, 256, 0, st>>>(X, (int)n, nt, count, stride);
  return cudaGetLastError();
}

// gamma[e] = -sum_j lb_j G[j][e]  (density matrix from the beta^- endpoint row)
__global__ void gamma_kernel(const double2* __restrict__ G, const double* __restrict__ lb, double2* gam,
                             int ntau, int64_t ne) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < ne; e += (int64_t)gridDim.x * blockDim.x) {
    double re = 0, im = 0;
    for (int j = 0; j < ntau; ++j) {
      double2 g = G[(int64_t)j * ne + e];
      re += lb[j] * g.x; im += lb[j] * g.y;
    }
    gam[e] = make_double2(-re, -im);
  }
}
cudaError_t density_gamma(const double2* G, const double* lb, double2* gam, int ntau, int64_t ne, cudaStream_t st) {
  gamma_kernel<<<nblk(ne), 256, 0, st>>>(G, lb, gam, ntau, ne);
  return cudaGetLastError();
}

// t[Q] = sum_k sum_ab gamma^k_ab V^{kk}_ba(Q)   (inner trace of Eq. HF_J)
__global__ void __launch_bounds__(256) hartree_t_kernel(const double2* __restrict__ V, const double2* __restrict__ gam,
                                                        double2* t, int nk, int naux, int nao) {
  const int Q = blockIdx.x;
  const int64_t n2 = (int64_t)nao * nao;
  double re = 0, im = 0;
  for (int64_t e = threadIdx.x; e < (int64_t)nk * n2; e += blockDim.x) {
    int k = (int)(e / n2);
    int64_t ab = e - k * n2;
    int a = (int)(ab / nao), b = (int)(ab - (int64_t)a * nao);
    double2 g = gam[e];
    double2 v = V[(((int64_t)k * nk + k) * naux + Q) * n2 + (int64_t)b * nao + a];
    re += g.x * v.x - g.y * v.y;
    im += g.x * v.y + g.y * v.x;
  }
  __shared__ double sr[256], si[256];
  sr[threadIdx.x] = re; si[threadIdx.x] = im;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if (threadIdx.x < s) { sr[threadIdx.x] += sr[threadIdx.x + s]; si[threadIdx.x] += si[threadIdx.x + s]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) t[Q] = make_double2(sr[0], si[0]);
}
cudaError_t hartree_t(const double2* V, const double2* gam, double2* t, int nk, int naux, int nao, cudaStream_t st) {
  hartree_t_kernel<<<naux, 256, 0, st>>>(V, gam, t, nk, naux, nao);
  return cudaGetLastError();
}

// J^k_ij = fac * sum_Q V^{kk}_ij(Q) t(Q)
__global__ void hartree_j_kernel(const double2* __restrict__ V, const double2* __restrict__ t, double2* J,
                                 int nk, int naux, int nao, double fac) {
  const int64_t n2 = (int64_t)nao * nao;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < nk * n2; e += (int64_t)gridDim.x * blockDim.x) {
    int k = (int)(e / n2);
    int64_t ij = e - k * n2;
    double re = 0, im = 0;
    const double2* Vk = V + ((int64_t)k * nk + k) * naux * n2 + ij;
    for (int Q = 0; Q < naux; ++Q) {
      double2 v = Vk[(int64_t)Q * n2], tq = t[Q];
      re += v.x * tq.x - v.y * tq.y;
      im += v.x * tq.y + v.y * tq.x;
    }
    J[e] = make_double2(fac * re, fac * im);
  }
}
cudaError_t hartree_j(const double2* V, const double2* t, double2* J, int nk, int naux, int nao, double fac,
                      cudaStream_t st) {
  hartree_j_kernel<<<nblk((int64_t)nk * nao * nao), 256, 0, st>>>(V, t, J, nk, naux, nao, fac);
  return cudaGetLastError();
}

// y <- a x + b y
__global__ void axpby_kernel(double2* y, const double2* x, double a, double b, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double2 u = x[e], v = y[e];
    y[e] = make_double2(a * u.x + b * v.x, a * u.y + b * v.y);
  }
}
cudaError_t axpby(double2* y, const double2* x, double a, double b, int64_t n, cudaStream_t st) {
  axpby_kernel<<<nblk(n), 256, 0, st>>>(y, x, a, b, n);
  return cudaGetLastError();
}

// X <- sign * X + I  (sign = -1: I - X;  sign = +1 with the identity subtracted: X - I)
__global__ void idshift_kernel(double2* X, int64_t n, int64_t count, double sign, double diag) {
  const int64_t n2 = n * n, tot = n2 * count;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t r = e % n2;
    double2 v = X[e];
    v.x *= sign; v.y *= sign;
    if (r / n == r % n) v.x += diag;
    X[e] = v;
  }
}
cudaError_t identity_minus(double2* X, int64_t n, int64_t count, double sign, cudaStream_t st) {
  // sign < 0: X <- I - X;  sign > 0: X <- X - I
  idshift_kernel<<<nblk(n * n * count), 256, 0, st>>>(X, n, count, sign, sign < 0 ? 1.0 : -1.0);
  return cudaGetLastError();
}

__device__ __forceinline__ void atomic_max_nonneg(double* p, double v) {
  atomicMax((unsigned long long*)p, (unsigned long long)__double_as_longlong(v));
}

// out[0] = max |V^{kk'}_ij(Q) - conj V^{k'k}_ji(Q)|, out[1] = max |V|
__global__ void vpair_kernel(const double2* __restrict__ V, int nk, int naux, int nao, double* out) {
  const int64_t n2 = (int64_t)nao * nao, tot = (int64_t)nk * nk * naux * n2;
  double dev = 0, mx = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t ij = e % n2, rest = e / n2;
    int Q = (int)(rest % naux); rest /= naux;
    int k2 = (int)(rest % nk), k = (int)(rest / nk);
    int i = (int)(ij / nao), j = (int)(ij % nao);
    double2 a = V[e];
    double2 b = V[(((int64_t)k2 * nk + k) * naux + Q) * n2 + (int64_t)j * nao + i];
    dev = fmax(dev, hypot(a.x - b.x, a.y + b.y));
    // a non-finite entry makes the magnitude +inf (fmax alone would skip a NaN)
    mx = (isfinite(a.x) && isfinite(a.y)) ? fmax(mx, hypot(a.x, a.y)) : INFINITY;
  }
  atomic_max_nonneg(out, dev);
  atomic_max_nonneg(out + 1, mx);
}
cudaError_t check_v_pairing(const double2* V, int nk, int naux, int nao, double* d_out, cudaStream_t st) {
  vpair_kernel<<<152 * 8, 256, 0, st>>>(V, nk, naux, nao, d_out);
  return cudaGetLastError();
}

// out[0] = max |X_ij - conj X_ji|, out[1] = max |X|
__global__ void herm_check_kernel(const double2* __restrict__ X, int64_t n, int64_t count, double* out) {
  const int64_t n2 = n * n, tot = n2 * count;
  double dev = 0, mx = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    int64_t m = e / n2, r = e - m * n2, i = r / n, j = r - i * n;
    double2 a = X[e], b = X[m * n2 + j * n + i];
    dev = fmax(dev, hypot(a.x - b.x, a.y + b.y));
    mx = (isfinite(a.x) && isfinite(a.y)) ? fmax(mx, hypot(a.x, a.y)) : INFINITY;
  }
  atomic_max_nonneg(out, dev);
  atomic_max_nonneg(out + 1, mx);
}
cudaError_t check_herm(const double2* X, int64_t n, int64_t count, double* d_out, cudaStream_t st) {
  herm_check_kernel<<<nblk(n * n * count), 256, 0, st>>>(X, n, count, d_out);
  return cudaGetLastError();
}

__global__ void maxdiff_kernel(const double2* __restrict__ a, const double2* __restrict__ b, int64_t n, double* out) {
  double m = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
    double2 u = a[e], v = b[e];
    m = fmax(m, hypot(u.x - v.x, u.y - v.y));
  }
  atomic_max_nonneg(out, m);
}
cudaError_t maxabs_diff(const double2* a, const double2* b, int64_t n, double* d_out, cudaStream_t st) {
  maxdiff_kernel<<<nblk(n), 256, 0, st>>>(a, b, n, d_out);
  return cudaGetLastError();
}

__global__ void c64_kernel(const double2* __restrict__ x, float2* y, int64_t n) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    y[e] = make_float2((float)x[e].x, (float)x[e].y);
}
cudaError_t to_c64(const double2* x, float2* y, int64_t n, cudaStream_t st) {
  c64_kernel<<<nblk(n), 256, 0, st>>>(x, y, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------ time-reversal symmetry

// out[0] = max |X[s] - conj X[partner[s]]| over slabs s of `len` complex entries,
// out[1] = max |X| (+inf when an entry is not finite)
__global__ void trs_check_kernel(const double2* __restrict__ X, int64_t nslab, int64_t len,
                                 const int* __restrict__ partner, double* out) {
  const int64_t tot = nslab * len;
  double dev = 0, mx = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = e / len, i = e - s * len;
    const double2 a = X[e], b = X[(int64_t)partner[s] * len + i];
    dev = fmax(dev, hypot(a.x - b.x, a.y + b.y));
    mx = (isfinite(a.x) && isfinite(a.y)) ? fmax(mx, hypot(a.x, a.y)) : INFINITY;
  }
  atomic_max_nonneg(out, dev);
  atomic_max_nonneg(out + 1, mx);
}
cudaError_t check_trs(const double2* X, int64_t nslab, int64_t len, const int* partner, double* d_out,
                      cudaStream_t st) {
  trs_check_kernel<<<nblk(nslab * len), 256, 0, st>>>(X, nslab, len, partner, d_out);
  return cudaGetLastError();
}

// X[o][k][:] = conj X[o][src[k]][:] for every k with need[k] (layout [outer][nk][inner])
__global__ void conj_fill_kernel(double2* X, int64_t outer, int nk, int64_t inner, const int* __restrict__ src,
                                 const int* __restrict__ need) {
  const int64_t tot = outer * nk * inner;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < tot; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t o = e / ((int64_t)nk * inner), r = e - o * nk * inner;
    const int k = (int)(r / inner);
    if (!need[k]) continue;
    const int64_t i = r - (int64_t)k * inner;
    const double2 v = X[(o * nk + src[k]) * inner + i];
    X[e] = make_double2(v.x, -v.y);
  }
}
cudaError_t conj_fill(double2* X, int64_t outer, int nk, int64_t inner, const int* src, const int* need,
                      cudaStream_t st) {
  conj_fill_kernel<<<nblk(outer * nk * inner), 256, 0, st>>>(X, outer, nk, inner, src, need);
  return cudaGetLastError();
}

}  // namespace gwk
