// Dyson equation on the sampled Matsubara points and the chemical-potential
// search (Eq. Dyson; Sec. "scGW workflow": mu adjusted to charge neutrality).
//
// One thread block per (n, k): A = (i w_n + mu) S - H0 - Sigma_inf - Sigma~(i w_n)
// is built in shared memory and inverted in place (Gauss-Jordan, partial
// pivoting).  For the electron count the block returns Re[r_n tr(A^{-1} S)];
// a single-block kernel reduces those in a fixed order (deterministic) and
// advances a bracketing/bisection state machine held in device memory, so the
// whole search runs without host round trips except a periodic "done" read.
#include "gw_internal.cuh"
#include "gj.cuh"

namespace gwk {

__global__ void __launch_bounds__(256) dyson_kernel(DysonArgs a, const double* mu_ptr, double2* G_out,
                                                    double* partial, const int* done_flag, int* info) {
  if (done_flag && *(volatile const int*)done_flag) return;
  extern __shared__ unsigned char smem[];
  const int n = a.nao, lda = n;
  double2* A = (double2*)smem;
  double2* f = A + n * lda;
  int* perm = (int*)(f + n);
  double* rv = (double*)(perm + n + (n & 1));
  int* ri = (int*)(rv + blockDim.x);
  const double mu = *mu_ptr;
  const int64_t n2 = (int64_t)n * n;
  const int64_t nsys = (int64_t)a.nw * a.nk;
  for (int64_t sys = blockIdx.x; sys < nsys; sys += gridDim.x) {
    const int w = (int)(sys / a.nk), k = (int)(sys - (int64_t)w * a.nk);
    const double wn = a.wn[w];
    const double2* S = a.S + k * n2;
    const double2* H = a.H0 + k * n2;
    const double2* Si = a.Sinf + k * n2;
    const double2* Sw = a.Siw + sys * n2;
    for (int e = threadIdx.x; e < n2; e += blockDim.x) {
      double2 s = S[e], h = H[e], x = Si[e], y = Sw[e];
      // (i wn + mu) s
      double re = mu * s.x - wn * s.y, im = mu * s.y + wn * s.x;
      A[e] = make_double2(re - h.x - x.x - y.x, im - h.y - x.y - y.y);
    }
    __syncthreads();
    int bad = gj_invert_smem(A, n, lda, f, perm, rv, ri);
    if (bad && threadIdx.x == 0) atomicOr(info, 1);
    if (G_out) {
      double2* Gd = G_out + sys * n2;
      for (int e = threadIdx.x; e < n2; e += blockDim.x) Gd[e] = A[e];
    }
    if (partial) {
      // tr(A^{-1} S) = sum_ij Ainv_ij S_ji
      double tr = 0, ti = 0;
      for (int e = threadIdx.x; e < n2; e += blockDim.x) {
        int i = e / n, j = e - i * n;
        double2 g = A[e], s = S[(int64_t)j * n + i];
        tr += g.x * s.x - g.y * s.y;
        ti += g.x * s.y + g.y * s.x;
      }
      rv[threadIdx.x] = tr;
      __syncthreads();
      for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) rv[threadIdx.x] += rv[threadIdx.x + s];
        __syncthreads();
      }
      double trr = rv[0];
      __syncthreads();
      rv[threadIdx.x] = ti;
      __syncthreads();
      for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) rv[threadIdx.x] += rv[threadIdx.x + s];
        __syncthreads();
      }
      if (threadIdx.x == 0) {
        double2 r = a.r[w];
        partial[sys] = r.x * trr - r.y * rv[0];   // Re(r_n tr)
      }
    }
    __syncthreads();
  }
}

size_t dyson_smem(int nao, int nt) {
  return (size_t)nao * nao * sizeof(double2) + (size_t)nao * sizeof(double2) + (size_t)(nao + 1) * sizeof(int) + 8 +
         (size_t)nt * (sizeof(double) + sizeof(int));
}

cudaError_t dyson_eval(const DysonArgs& a, const double* mu_ptr, double2* G_out, double* partial,
                       const int* done_flag, int* info, cudaStream_t st) {
  const int nt = 256;
  size_t sm = dyson_smem(a.nao, nt);
  if (sm > 48 * 1024) {
    cudaError_t e = cudaFuncSetAttribute(dyson_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
  }
  int64_t nsys = (int64_t)a.nw * a.nk;
  int blocks = (int)(nsys < 152 * 8 ? nsys : 152 * 8);
  dyson_kernel<<<blocks, nt, sm, st>>>(a, mu_ptr, G_out, partial, done_flag, info);
  return cudaGetLastError();
}

// One step of the bracketing search (expand until N(lo) <= target <= N(hi), then
// Illinois steps with a bisection every fourth step, until |N - target| <= tol and
// hi - lo <= width).  state->x is the point evaluated by the preceding
// dyson_kernel; `scale` turns the summed partials into N(x).
__global__ void __launch_bounds__(1024) mu_step_kernel(MuState* s, const double* partial, int64_t count,
                                                       double scale) {
  if (*(volatile int*)&s->done) return;
  __shared__ double red[1024];
  double acc = 0;
  for (int64_t i = threadIdx.x; i < count; i += blockDim.x) acc += partial[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int t = blockDim.x / 2; t > 0; t >>= 1) {
    if (threadIdx.x < t) red[threadIdx.x] += red[threadIdx.x + t];
    __syncthreads();
  }
  if (threadIdx.x != 0) return;
  const double N = scale * red[0];
  s->iter += 1;
  if (s->phase == 0) {            // N at lo: must be <= target
    s->Nlo = N;
    if (N > s->target) { double w = s->hi - s->lo; s->lo -= 2.0 * w; s->x = s->lo; }
    else { s->phase = 1; s->x = s->hi; }
  } else if (s->phase == 1) {     // N at hi: must be >= target
    s->Nhi = N;
    if (N < s->target) { double w = s->hi - s->lo; s->hi += 2.0 * w; s->x = s->hi; }
    else {
      s->phase = 2;
      s->flo = s->Nlo - s->target; s->fhi = N - s->target; s->side = 0;
      const double d = s->fhi - s->flo;
      const double xs = d > 0 ? s->lo - s->flo * (s->hi - s->lo) / d : 0.5 * (s->lo + s->hi);
      s->x = (xs > s->lo && xs < s->hi) ? xs : 0.5 * (s->lo + s->hi);
    }
  } else {                        // Illinois (regula falsi with halved stale end), bisection every 4th step
    s->Nx = N;
    const double F = N - s->target;
    if (fabs(F) <= s->tol && (s->hi - s->lo) <= s->width) {
      s->done = 1; s->status = 0;
    } else {
      if (F < 0) {
        s->lo = s->x; s->flo = F;
        if (s->side == -1) s->fhi *= 0.5;
        s->side = -1;
      } else {
        s->hi = s->x; s->fhi = F;
        if (s->side == 1) s->flo *= 0.5;
        s->side = 1;
      }
      const double mid = 0.5 * (s->lo + s->hi), d = s->fhi - s->flo;
      double xs = d > 0 ? s->lo - s->flo * (s->hi - s->lo) / d : mid;
      if (!(xs > s->lo && xs < s->hi) || (s->iter & 3) == 0) xs = mid;
      s->x = xs;
    }
  }
  if (!s->done && s->iter >= s->maxit) { s->done = 1; s->status = 1; }
}

// Re-arms the search around the previous converged x (device-side, for captured graphs).
__global__ void mu_init_kernel(MuState* s, double target, double tol, double width, int maxit) {
  const double center = s->x;
  s->lo = center - 1.0; s->hi = center + 1.0; s->x = s->lo;
  s->Nlo = s->Nhi = s->Nx = 0.0;
  s->target = target; s->tol = tol; s->width = width;
  s->phase = 0; s->iter = 0; s->maxit = maxit; s->done = 0; s->status = 0;
  s->flo = s->fhi = 0.0; s->side = 0;
}
cudaError_t mu_init_device(MuState* s, double target, double tol, double width, int maxit, cudaStream_t st) {
  mu_init_kernel<<<1, 1, 0, st>>>(s, target, tol, width, maxit);
  return cudaGetLastError();
}

cudaError_t mu_step(MuState* s, const double* partial, int64_t count, double scale, cudaStream_t st) {
  mu_step_kernel<<<1, 1024, 0, st>>>(s, partial, count, scale);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- Dyson tangent
// G = [(i w + mu) S - H0 - Sigma_inf - Sigma(i w)]^-1 at the electron count N(mu) = N_e:
//   dG = G (dSigma_inf + dSigma(i w)) G - dmu G S G,
//   dmu = Re sum r_n tr[G D G S] / Re sum r_n tr[G S G S]   (so that dN = 0).
// The products run on the contraction kernel; these kernels form D, the weighted
// traces, dmu and the combination.

// D[w][k] = dSinf[k] + dSiw[w][k]
__global__ void dyson_tangent_rhs_kernel(const double2* __restrict__ dSinf, const double2* __restrict__ dSiw,
                                         double2* __restrict__ D, int64_t nk, int64_t n2, int64_t total) {
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const int64_t k = (e / n2) % nk, i = e % n2;
    const double2 a = dSinf[k * n2 + i], b = dSiw[e];
    D[e] = make_double2(a.x + b.x, a.y + b.y);
  }
}

// part[sys] = Re(r_w tr(X_sys S_k)), part[nsys + sys] = Re(r_w tr(Y_sys S_k)); one block per system
__global__ void __launch_bounds__(256) dyson_tangent_trace_kernel(const double2* __restrict__ X,
                                                                  const double2* __restrict__ Y,
                                                                  const double2* __restrict__ S,
                                                                  const double2* __restrict__ r, int nao, int nk,
                                                                  int64_t nsys, double* part) {
  __shared__ double red[4][256];
  const int64_t n2 = (int64_t)nao * nao;
  for (int64_t sys = blockIdx.x; sys < nsys; sys += gridDim.x) {
    const int w = (int)(sys / nk), k = (int)(sys - (int64_t)w * nk);
    const double2* x = X + sys * n2;
    const double2* y = Y + sys * n2;
    const double2* s = S + (int64_t)k * n2;
    double xr = 0, xi = 0, yr = 0, yi = 0;
    for (int64_t e = threadIdx.x; e < n2; e += blockDim.x) {
      const int64_t i = e / nao, j = e - i * nao;
      const double2 sv = s[j * nao + i], a = x[e], b = y[e];
      xr += a.x * sv.x - a.y * sv.y; xi += a.x * sv.y + a.y * sv.x;
      yr += b.x * sv.x - b.y * sv.y; yi += b.x * sv.y + b.y * sv.x;
    }
    red[0][threadIdx.x] = xr; red[1][threadIdx.x] = xi; red[2][threadIdx.x] = yr; red[3][threadIdx.x] = yi;
    __syncthreads();
    for (int t = blockDim.x / 2; t > 0; t >>= 1) {
      if ((int)threadIdx.x < t)
        for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + t];
      __syncthreads();
    }
    if (threadIdx.x == 0) {
      const double2 rw = r[w];
      part[sys] = rw.x * red[0][0] - rw.y * red[1][0];
      part[nsys + sys] = rw.x * red[2][0] - rw.y * red[3][0];
    }
    __syncthreads();
  }
}

// dmu = sum part[0:nsys] / sum part[nsys:2 nsys], in a fixed order
__global__ void __launch_bounds__(1024) dyson_tangent_dmu_kernel(const double* part, int64_t nsys, double* dmu) {
  __shared__ double ra[1024], rb[1024];
  double a = 0, b = 0;
  for (int64_t i = threadIdx.x; i < nsys; i += blockDim.x) { a += part[i]; b += part[nsys + i]; }
  ra[threadIdx.x] = a; rb[threadIdx.x] = b;
  __syncthreads();
  for (int t = blockDim.x / 2; t > 0; t >>= 1) {
    if ((int)threadIdx.x < t) { ra[threadIdx.x] += ra[threadIdx.x + t]; rb[threadIdx.x] += rb[threadIdx.x + t]; }
    __syncthreads();
  }
  if (threadIdx.x == 0) *dmu = rb[0] != 0.0 ? ra[0] / rb[0] : 0.0;
}

// dG = X - dmu Y
__global__ void dyson_tangent_combine_kernel(const double2* __restrict__ X, const double2* __restrict__ Y,
                                             const double* dmu, double2* __restrict__ dG, int64_t total) {
  const double m = *dmu;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
    const double2 x = X[e], y = Y[e];
    dG[e] = make_double2(x.x - m * y.x, x.y - m * y.y);
  }
}

static inline int nblk_(int64_t n) { int64_t b = (n + 255) / 256; return (int)(b < 152 * 16 ? b : 152 * 16); }

cudaError_t dyson_tangent_rhs(const double2* dSinf, const double2* dSiw, double2* D, int64_t nk, int64_t n2,
                              int64_t nw, cudaStream_t st) {
  const int64_t total = nw * nk * n2;
  dyson_tangent_rhs_kernel<<<nblk_(total), 256, 0, st>>>(dSinf, dSiw, D, nk, n2, total);
  return cudaGetLastError();
}

cudaError_t dyson_tangent_finish(const double2* X, const double2* Y, const double2* S, const double2* r, int nao,
                                 int nk, int nw, double* part, double* dmu, double2* dG, cudaStream_t st) {
  const int64_t nsys = (int64_t)nw * nk, total = nsys * nao * nao;
  dyson_tangent_trace_kernel<<<(int)(nsys < 152 * 8 ? nsys : 152 * 8), 256, 0, st>>>(X, Y, S, r, nao, nk, nsys, part);
  dyson_tangent_dmu_kernel<<<1, 1024, 0, st>>>(part, nsys, dmu);
  dyson_tangent_combine_kernel<<<nblk_(total), 256, 0, st>>>(X, Y, dmu, dG, total);
  return cudaGetLastError();
}

// Real inner product sum_e (a_e.x b_e.x + a_e.y b_e.y) as per-block partials (count
// <= 1216 blocks); the host adds them in order.
__global__ void __launch_bounds__(256) rdot_kernel(const double2* __restrict__ a, const double2* __restrict__ b,
                                                   int64_t n, double* part) {
  __shared__ double red[256];
  double s = 0;
  for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
    s += a[e].x * b[e].x + a[e].y * b[e].y;
  red[threadIdx.x] = s;
  __syncthreads();
  for (int t = blockDim.x / 2; t > 0; t >>= 1) {
    if ((int)threadIdx.x < t) red[threadIdx.x] += red[threadIdx.x + t];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

int rdot_blocks(int64_t n) { int64_t b = (n + 255) / 256; return (int)(b < 1216 ? b : 1216); }

cudaError_t rdot_partials(const double2* a, const double2* b, int64_t n, double* part, cudaStream_t st) {
  rdot_kernel<<<rdot_blocks(n), 256, 0, st>>>(a, b, n, part);
  return cudaGetLastError();
}

}  // namespace gwk
