// Adjoints (vector-Jacobian products) of the two contractions, for a real
// loss L and PyTorch's conjugate-Wirtinger convention: for a map y = f(x)
// that is complex-linear in each factor, xbar = sum conj(dy/dx) * ybar.
// (X + X^H)/2 is self-adjoint under Re<a, b>, so the symmetrisation steps
// pass their cotangent through (Xbar + Xbar^H)/2.
//
// P~0 (Eq. tilde_P0_tau): P_QQ' = (s/Nk) sum_k sum V1_da(Q) G'_ab V2_bc(Q') Gm_cd,
//   V1 = V^{k,k+q}, V2 = V^{k+q,k}, G' = G^{k+q}(t), Gm = G^k(-t) = -G^k(t_{n-1-j}):
//   G'bar_ab  += (s/Nk) sum conj(V1_da(Q) V2_bc(Q') Gm_cd) Pbar_QQ'
//   Gm bar_cd += (s/Nk) sum conj(V1_da(Q) G'_ab V2_bc(Q')) Pbar_QQ'
// Sigma~ (Eq. tilde_sigma2): S_ij = -(1/Nk) sum V1_ia(Q) G_ab P_QQ' V2_bj(Q'),
//   V1 = V^{k,k-q}, V2 = V^{k-q,k}, G = G^{k-q}(t), P = P~^q(t):
//   Gbar_ab  += -(1/Nk) sum conj(V1_ia(Q) P_QQ' V2_bj(Q')) Sbar_ij
//   Pbar_QQ' += -(1/Nk) sum conj(V1_ia(Q) G_ab V2_bj(Q')) Sbar_ij
// Every chain runs on the strided contraction kernel: in complex128, or with
// complex64 operands (V, G, P~ and the cotangent rounded to complex64) and fp32
// accumulation within each launch, the outputs still accumulated in fp64 across
// the (q, k) slabs.
#include <string>
#include "gw_internal.cuh"

using namespace gwk;

namespace gwadj {
struct View {   // the context's tensors seen by the adjoint chains (same layout in gw_api.cu)
  int nao, naux, nk, ntau;
  double spin;
  const double2* V;
  const double2* G_tau;
  const double2* P_tau;
  const int* kplus;
  const int* kminus;
  void* ws;
  size_t ws_bytes;
  double2 *bufA, *bufB, *bufC;   // three fp64 chain buffers of ntau*naux*nao^2
  cudaStream_t st;
  bool c64;                       // complex64 arithmetic: the operands below
  const float2* V32;
  const float2* G32;
  const float2* P32;
  float2* bar32;                  // complex64 copy of the symmetrised cotangent
};
}  // namespace gwadj

static GettDesc desc(int64_t M, int64_t N, int64_t K, int64_t Z) {
  GettDesc d{};
  d.M = M; d.N = N; d.K = K; d.Z = Z;
  d.az = d.bz = d.cz = I1(0);
  d.alpha = make_double2(1, 0); d.beta = make_double2(0, 0);
  d.ksplit = 1;
  return d;
}
// operands in the View's arithmetic type; C is an intermediate of that type, or (out)
// one of the fp64 cotangent outputs
static cudaError_t run(const gwadj::View& v, const GettDesc& d, const void* A, const void* B, void* C, bool out = false) {
  const Ty t = v.c64 ? Ty::C64 : Ty::C128;
  return gett(d, A, t, B, t, C, out ? Ty::C128 : t, t, v.ws, v.ws_bytes, v.st);
}
// element e of an operand array in the View's arithmetic type
static const void* at(const gwadj::View& v, const double2* p64, const float2* p32, int64_t e) {
  return v.c64 ? (const void*)(p32 + e) : (const void*)(p64 + e);
}

namespace gwadj {

// Gbar (ntau,nk,nao,nao) += VJP of the symmetrised P~0(tau) w.r.t. G(tau); Pbar is
// herm-projected into bufC first.
cudaError_t polarization_vjp(const View& v, const double2* Pbar, double2* Gbar, int64_t* launches) {
  const int nk = v.nk, nao = v.nao, naux = v.naux, ntau = v.ntau;
  const int64_t n2 = (int64_t)nao * nao, na2 = (int64_t)naux * naux, slab = (int64_t)naux * n2,
                gstep = (int64_t)nk * n2;
  const double f = v.spin / nk;
  cudaError_t e;
  double2* Pr = v.bufC;   // herm(Pbar) for one q at a time
  for (int q = 0; q < nk; ++q) {
    if ((e = cudaMemcpyAsync(Pr, Pbar + (size_t)q * ntau * na2, (size_t)ntau * na2 * 16, cudaMemcpyDeviceToDevice,
                             v.st)))
      return e;
    if ((e = herm_batched(Pr, naux, ntau, na2, v.st))) return e;
    *launches += 1;
    const void* Pa = Pr;
    if (v.c64) {
      if ((e = to_c64(Pr, v.bar32, (int64_t)ntau * na2, v.st))) return e;
      Pa = v.bar32;
      *launches += 1;
    }
    for (int k = 0; k < nk; ++k) {
      const int kq = v.kplus[(size_t)q * nk + k];
      const void* V1 = at(v, v.V, v.V32, ((int64_t)k * nk + kq) * slab);
      const void* V2 = at(v, v.V, v.V32, ((int64_t)kq * nk + k) * slab);
      // X[t][Q'][(d,a)] = sum_Q Pr[t][Q][Q'] conj(V1[Q][(d,a)])
      GettDesc d1 = desc(naux, n2, naux, ntau);
      d1.am = I1(1); d1.ak = I1(naux); d1.az = I1(na2);
      d1.bk = I1(n2); d1.bn = I1(1); d1.conjB = true;
      d1.cm = I1(n2); d1.cn = I1(1); d1.cz = I1(slab);
      if ((e = run(v, d1, Pa, V1, v.bufA))) return e;
      // Y[t][Q'][c][a] = sum_d conj(Gm[t][c][d]) X[t][Q'][d][a],  Gm(t) = -G^k(t_{n-1-j})
      GettDesc d2 = desc(nao, (int64_t)naux * nao, nao, ntau);
      d2.am = I1(nao); d2.ak = I1(1); d2.az = I1(-gstep); d2.conjA = true;
      d2.bk = I1(nao); d2.bn = I2(nao, n2, 1); d2.bz = I1(slab);
      d2.cm = I1(nao); d2.cn = I2(nao, n2, 1); d2.cz = I1(slab);
      d2.alpha = make_double2(-1, 0);
      const void* Gm = at(v, v.G_tau, v.G32, (int64_t)(ntau - 1) * gstep + (int64_t)k * n2);
      if ((e = run(v, d2, Gm, v.bufA, v.bufB))) return e;
      // G'bar[t][a][b] += f sum_{Q',c} Y[t][Q'][c][a] conj(V2[Q'][b][c])
      GettDesc d3 = desc(nao, nao, (int64_t)naux * nao, ntau);
      d3.am = I1(1); d3.ak = I2(nao, n2, nao); d3.az = I1(slab);
      d3.bk = I2(nao, n2, 1); d3.bn = I1(nao); d3.conjB = true;
      d3.cm = I1(nao); d3.cn = I1(1); d3.cz = I1(gstep);
      d3.alpha = make_double2(f, 0); d3.beta = make_double2(1, 0);
      if ((e = run(v, d3, v.bufB, V2, Gbar + (size_t)kq * n2, true))) return e;
      // T[t][Q'][d][b] = sum_a X[t][Q'][d][a] conj(G'[t][a][b])
      GettDesc d4 = desc((int64_t)naux * nao, nao, nao, ntau);
      d4.am = I1(nao); d4.ak = I1(1); d4.az = I1(slab);
      d4.bk = I1(nao); d4.bn = I1(1); d4.bz = I1(gstep); d4.conjB = true;
      d4.cm = I1(nao); d4.cn = I1(1); d4.cz = I1(slab);
      if ((e = run(v, d4, v.bufA, at(v, v.G_tau, v.G32, (int64_t)kq * n2), v.bufB))) return e;
      // Gm bar[t][c][d] = f sum_{Q',b} conj(V2[Q'][b][c]) T[t][Q'][d][b];  G^k(t_{n-1-j}) gets -Gm bar(t_j)
      GettDesc d5 = desc(nao, nao, (int64_t)naux * nao, ntau);
      d5.am = I1(1); d5.ak = I2(nao, n2, nao); d5.conjA = true;
      d5.bk = I2(nao, n2, 1); d5.bn = I1(nao); d5.bz = I1(slab);
      d5.cm = I1(nao); d5.cn = I1(1); d5.cz = I1(-gstep);
      d5.alpha = make_double2(-f, 0); d5.beta = make_double2(1, 0);
      if ((e = run(v, d5, V2, v.bufB, Gbar + (size_t)(ntau - 1) * gstep + (size_t)k * n2, true))) return e;
      *launches += 5;
    }
  }
  return cudaSuccess;
}

// Gbar (ntau,nk,nao,nao) += and Pbar (nq,ntau,naux,naux) += VJP of the symmetrised
// Sigma~(tau) w.r.t. G(tau) and P~(tau); Sbar is herm-projected into bufC first.
cudaError_t selfenergy_vjp(const View& v, const double2* Sbar, double2* Gbar, double2* Pbar, int64_t* launches) {
  const int nk = v.nk, nao = v.nao, naux = v.naux, ntau = v.ntau;
  const int64_t n2 = (int64_t)nao * nao, na2 = (int64_t)naux * naux, slab = (int64_t)naux * n2,
                gstep = (int64_t)nk * n2;
  const double f = -1.0 / nk;
  cudaError_t e;
  double2* Sr = v.bufC;
  if ((e = cudaMemcpyAsync(Sr, Sbar, (size_t)ntau * gstep * 16, cudaMemcpyDeviceToDevice, v.st))) return e;
  if ((e = herm_batched(Sr, nao, (int64_t)ntau * nk, n2, v.st))) return e;
  *launches += 1;
  if (v.c64) {
    if ((e = to_c64(Sr, v.bar32, (int64_t)ntau * gstep, v.st))) return e;
    *launches += 1;
  }
  for (int q = 0; q < nk; ++q) {
    const void* Pq = at(v, v.P_tau, v.P32, (int64_t)q * ntau * na2);
    for (int k = 0; k < nk; ++k) {
      const int kmq = v.kminus[(size_t)q * nk + k];
      const void* V1 = at(v, v.V, v.V32, ((int64_t)k * nk + kmq) * slab);
      const void* V2 = at(v, v.V, v.V32, ((int64_t)kmq * nk + k) * slab);
      const void* Sk = at(v, Sr, v.bar32, (int64_t)k * n2);
      // E[t][Q'][(i,a)] = sum_Q conj(P[t][Q][Q']) conj(V1[Q][(i,a)])
      GettDesc d1 = desc(naux, n2, naux, ntau);
      d1.am = I1(1); d1.ak = I1(naux); d1.az = I1(na2); d1.conjA = true;
      d1.bk = I1(n2); d1.bn = I1(1); d1.conjB = true;
      d1.cm = I1(n2); d1.cn = I1(1); d1.cz = I1(slab);
      if ((e = run(v, d1, Pq, V1, v.bufA))) return e;
      // F[t][Q'][a][j] = sum_i E[t][Q'][i][a] Sr[t][k][i][j]
      GettDesc d2 = desc((int64_t)naux * nao, nao, nao, ntau);
      d2.am = I2(nao, n2, 1); d2.ak = I1(nao); d2.az = I1(slab);
      d2.bk = I1(nao); d2.bn = I1(1); d2.bz = I1(gstep);
      d2.cm = I2(nao, n2, nao); d2.cn = I1(1); d2.cz = I1(slab);
      if ((e = run(v, d2, v.bufA, Sk, v.bufB))) return e;
      // Gbar^{k-q}[t][a][b] += f sum_{Q',j} F[t][Q'][a][j] conj(V2[Q'][b][j])
      GettDesc d3 = desc(nao, nao, (int64_t)naux * nao, ntau);
      d3.am = I1(nao); d3.ak = I2(nao, n2, 1); d3.az = I1(slab);
      d3.bk = I2(nao, n2, 1); d3.bn = I1(nao); d3.conjB = true;
      d3.cm = I1(nao); d3.cn = I1(1); d3.cz = I1(gstep);
      d3.alpha = make_double2(f, 0); d3.beta = make_double2(1, 0);
      if ((e = run(v, d3, v.bufB, V2, Gbar + (size_t)kmq * n2, true))) return e;
      // H[t][Q][j][a] = sum_i Sr[t][k][i][j] conj(V1[Q][i][a])
      GettDesc d4 = desc(nao, (int64_t)naux * nao, nao, ntau);
      d4.am = I1(1); d4.ak = I1(nao); d4.az = I1(gstep);
      d4.bk = I1(nao); d4.bn = I2(nao, n2, 1); d4.conjB = true;
      d4.cm = I1(nao); d4.cn = I2(nao, n2, 1); d4.cz = I1(slab);
      if ((e = run(v, d4, Sk, V1, v.bufA))) return e;
      // W[t][Q][j][b] = sum_a H[t][Q][j][a] conj(G^{k-q}[t][a][b])
      GettDesc d5 = desc((int64_t)naux * nao, nao, nao, ntau);
      d5.am = I1(nao); d5.ak = I1(1); d5.az = I1(slab);
      d5.bk = I1(nao); d5.bn = I1(1); d5.bz = I1(gstep); d5.conjB = true;
      d5.cm = I1(nao); d5.cn = I1(1); d5.cz = I1(slab);
      if ((e = run(v, d5, v.bufA, at(v, v.G_tau, v.G32, (int64_t)kmq * n2), v.bufB))) return e;
      // Pbar^q[t][Q][Q'] += f sum_{(j,b)} W[t][Q][(j,b)] conj(V2[Q'][b][j])
      GettDesc d6 = desc((int64_t)ntau * naux, naux, n2, 1);
      d6.am = I1(n2); d6.ak = I1(1);
      d6.bk = I2(nao, 1, nao); d6.bn = I1(n2); d6.conjB = true;
      d6.cm = I1(naux); d6.cn = I1(1);
      d6.alpha = make_double2(f, 0); d6.beta = make_double2(1, 0);
      if ((e = run(v, d6, v.bufB, V2, Pbar + (size_t)q * ntau * na2, true))) return e;
      *launches += 6;
    }
  }
  return cudaSuccess;
}

}  // namespace gwadj
