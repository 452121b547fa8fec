// C ABI of the library (declared in include/gwgb.h): context, buffers and
// the stage drivers of one self-consistent GW iteration.  Every arithmetic
// step runs in the kernels of this directory; the host only sequences
// launches on the caller's stream.
#include <stdio.h>
#include <string.h>
#include <math.h>
#include <cmath>
#include <new>
#include <string>
#include <vector>
#include <atomic>
#include <nvtx3/nvToolsExt.h>
#include "gw_internal.cuh"

using namespace gwk;

namespace gwk { std::atomic<long long> g_launches{0}; }

struct gw_ctx {
  gw_config cfg{};
  int nao = 0, naux = 0, nk = 0, ntau = 0, nw = 0;   // nw: fermionic Matsubara points (= nwf)
  int nwf = 0, nwb = 0;                              // fermionic / bosonic Matsubara points
  int q0 = 0, q1 = 0;   // q-points [q0, q1) of the P~0, screened and Sigma~ contractions (all by default)
  // time-reversal symmetry (GW_TRS): kneg[k] = index of -k; the forward P~0, screened solve and
  // Sigma~ skip every q (k) with kneg < q (k) and take its result as the conjugate of its partner's
  bool trs = false, reduce = false;
  std::vector<int> kneg;
  int *d_kneg = nullptr, *d_kneed = nullptr, *d_vpart = nullptr;
  int64_t n2 = 0, na2 = 0;
  double spin = 2.0;
  cudaStream_t st = nullptr;
  std::string err;
  std::vector<int> kplus, kminus;  // [q * nk + k]
  std::vector<void*> owned;
  // inputs
  double2 *H0 = nullptr, *S = nullptr, *V = nullptr;
  float2* V32 = nullptr;
  // grid
  double *tau = nullptr, *lb = nullptr, *l0 = nullptr, *wn = nullptr;
  double2 *TFf = nullptr, *TBf = nullptr, *TFb = nullptr, *TBb = nullptr, *r = nullptr;
  // transforms on tensor cores by exact digit splitting: digits/exponents of TFf, TBf,
  // TFb, TBb and the workspace for the transposed data operand
  bool emul = false;
  float* Tdig[4] = {nullptr, nullptr, nullptr, nullptr};
  int* Texp[4] = {nullptr, nullptr, nullptr, nullptr};
  float* emA = nullptr;
  int* emAe = nullptr;
  size_t emA_bytes = 0;
  // screened solve as a complex64 inversion refined to FP64 accuracy (with emul)
  void* irws = nullptr;
  size_t irws_bytes = 0;
  int *d_fn = nullptr, *d_bm = nullptr;
  // state
  double2 *G_tau = nullptr, *G_iw = nullptr, *G_prev = nullptr, *gamma = nullptr, *tQ = nullptr;
  double2 *Sinf = nullptr, *Sinf_new = nullptr, *Siw = nullptr, *Siw_new = nullptr, *Stau = nullptr;
  double2 *P0_tau = nullptr, *P_iw = nullptr, *P_tau = nullptr;
  // chain intermediates and workspaces
  void *chA = nullptr, *chB = nullptr;
  size_t ch_bytes = 0;
  float2 *G32 = nullptr, *P32 = nullptr, *gam32 = nullptr;
  float2* G32m = nullptr;   // c64 copy of the G(-tau) factor when it differs from G(tau) (tangents)
  // tangent of the self-consistency map: dG(i w), dG(tau), dSigma~(tau), dgamma, dP~, reductions
  double2 *tGiw = nullptr, *tGtau = nullptr, *tS = nullptr, *tgam = nullptr, *tP = nullptr;
  double* tpart = nullptr;
  std::vector<double2*> kry;   // Newton-Krylov basis (owned through `owned`)
  std::vector<double2*> dx, dr;   // DIIS history: inputs and residuals (owned through `owned`)
  double2* dnext = nullptr;
  int nvec = 0;
  // split-TF32 tensor-core operands (hi / lo planes, rows padded to 32 fp32)
  float *Zhi = nullptr, *Zlo = nullptr, *Vhi = nullptr, *Vlo = nullptr;
  float *Pchi = nullptr, *Pclo = nullptr, *VThi = nullptr, *VTlo = nullptr;
  float *Y3hi = nullptr, *Y3lo = nullptr, *W3hi = nullptr, *W3lo = nullptr;   // last Sigma step
  int64_t kpadP = 0, kpadS = 0, kpad3 = 0;
  int pgroup = 1;   // k-points whose last P~0 step runs as one GEMM (K concatenated over k)
  size_t y3bytes = 0;
  double2 *adjA = nullptr, *adjB = nullptr, *adjC = nullptr;   // fp64 chains of the adjoints (lazy)
  float2 *adjG32 = nullptr, *adjP32 = nullptr, *adjBar32 = nullptr;   // complex64 adjoint operands (lazy)
  // captured iteration (gw_iterate_graph): status checks are deferred while capturing
  bool deferred = false;
  cudaStream_t gst = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  int64_t graph_kernels = 0;   // kernel nodes of the captured iteration (counted per replay)
  cudaEvent_t gev[3]{};
  // nao-sized steps on tensor cores: V slab split, doubled G(tau) per k, X hi/lo
  float *Vs_hi = nullptr, *Vs_lo = nullptr, *Ge_hi = nullptr, *Ge_lo = nullptr, *Xs_hi = nullptr, *Xs_lo = nullptr;
  float *Gp_hi = nullptr, *Gp_lo = nullptr;
  // k-points per launch of the 16-bit chains (their per-k operands side by side) and the
  // G blocks of k+q (or k-q) gathered in k order for such a launch
  int pbatch = 1;
  float *Gq_hi = nullptr, *Gq_lo = nullptr;
  int* eGq = nullptr;
  int64_t kpadA = 0;
  size_t zbytes = 0;
  // 16-bit pieces (GW_SPLIT_F16 / GW_SPLIT_BF16): format (1 fp16, 2 bf16; 0 none), norms of V per Q
  // (max, max row sum of moduli), their exponents, and the row exponents of every chain operand
  int hfmt = 0;
  float *vQmax = nullptr, *vQrs = nullptr, *gn = nullptr;   // gn: gmax, grs of G(t) and of G(-t) factor
  int *eVQ = nullptr, *eVall = nullptr, *eV1 = nullptr, *eY = nullptr, *eZ = nullptr, *eGe = nullptr,
      *eGp = nullptr, *ePc = nullptr, *ePs = nullptr, *eY3 = nullptr;
  int h_Evmax = 0;   // exponent of max_Q vQmax (host copy)
  void* ws = nullptr;
  size_t ws_bytes = 0;
  double* partial = nullptr;
  MuState* mus = nullptr;
  MuState* h_mus = nullptr;  // pinned
  int* info = nullptr;
  double* dscr = nullptr;    // small device scratch (max reductions)
  double* h_scr = nullptr;   // pinned
  double mu = 0.0, n_at_mu = 0.0;
  int mu_steps = 0;
  bool have_G = false, have_mu = false, have_sigma = false, have_P0 = false, have_P = false;
  // one bit per gw_quantity whose buffer holds a result (set by gw_set or by the call
  // that computes it); gw_get refuses the others with GW_ERR_STATE
  uint32_t valid = 0;
  cudaEvent_t ev[8]{};
  // optional per-launch timing of the contraction kernel (gw_profile)
  bool prof = false;
  std::vector<cudaEvent_t> pev;
  size_t pused = 0;
  double pflops = 0.0;
  int64_t plaunch = 0;
  std::vector<cudaEvent_t> uev;   // same for the tensor-core kernel
  size_t uused = 0;
  double uflops = 0.0;
  int64_t ulaunch = 0;
};

static thread_local std::string g_init_err;

static inline uint32_t qbit(gw_quantity q) { return 1u << (unsigned)q; }
static inline void mark(gw_ctx* c, gw_quantity q) { c->valid |= qbit(q); }
static inline void unmark(gw_ctx* c, gw_quantity q) { c->valid &= ~qbit(q); }

// The nao-sized chain steps (K = 2 nao) run on the tensor-core GEMM by default:
// with the persistent kernel and lane-per-row stores of the transposed outputs they
// beat the FP32 SIMT small-product kernel (C3 shapes with a 2x2x2 k-mesh: P~0 stage
// 327 ms against 530 ms, Sigma~ 244 ms against 331 ms per iteration).
static constexpr bool kTensorSmallSteps = true;   // GW_SMALL_TENSOR / GW_SMALL_SIMT override

// Screened solve with the tensor cores: complex64 inversion of I - P~0 and two Newton
// steps with FP64-accurate residuals (relative error ~1e-7 -> ~1e-14 -> FP64
// rounding); the systems are processed in batches whose workspace (digit planes of
// P~0 and of the iterate, residual, complex64 panels) stays below kRefineBytes.
static constexpr int kRefineSteps = 2;
static constexpr size_t kZGroupBytes = (size_t)8 << 30;
static int g_pgroup_cap = 0;   // test hook: upper bound on the k-points per group (0: none)
static int g_pbatch_cap = 0;   // test hook: upper bound on the k-points per chain launch (0: none)

// k-points per launch of the 16-bit chains: enough output tiles of a nao-sized step
// (naux nao rows in 128-row tiles, one per tau) for ~16 rounds of the 152 SMs, at most
// the operand lists' length and nk
static int chain_pbatch(int nao, int naux, int nk, int ntau) {
  const int64_t tiles1 = ((int64_t)naux * nao + 127) / 128 * ntau;
  int64_t kb = tiles1 > 0 ? (16 * 152 + tiles1 - 1) / tiles1 : 1;
  if (kb > kSrcListMax) kb = kSrcListMax;
  if (kb > nk) kb = nk;
  if (g_pbatch_cap > 0 && kb > g_pbatch_cap) kb = g_pbatch_cap;
  return kb < 1 ? 1 : (int)kb;
}
static constexpr size_t kRefineBytes = (size_t)6 << 30;

#define CK(x)                                                                        \
  do {                                                                               \
    cudaError_t e_ = (x);                                                            \
    if (e_ != cudaSuccess) return fail(c, GW_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

static gw_status fail(gw_ctx* c, gw_status s, const std::string& m) {
  if (c) c->err = m; else g_init_err = m;
  return s;
}

static void* dalloc(gw_ctx* c, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void* p = nullptr;
  if (c->cfg.dev_alloc) p = c->cfg.dev_alloc(c->cfg.alloc_user, bytes);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  if (p) c->owned.push_back(p);
  return p;
}

// gives back one allocation made with dalloc (optional workspaces that did not fit)
static void dfree(gw_ctx* c, void* p) {
  if (!p) return;
  for (size_t i = 0; i < c->owned.size(); ++i)
    if (c->owned[i] == p) { c->owned.erase(c->owned.begin() + (long)i); break; }
  if (c->cfg.dev_free) c->cfg.dev_free(c->cfg.alloc_user, p); else cudaFree(p);
}

// budget of one optional workspace: its cap, and at most 1/32 of the device memory
// free when the context is created (several contexts share the device)
static size_t opt_budget(size_t cap) {
  size_t fr = 0, tot = 0;
  if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return cap;
  return fr / 32 < cap ? fr / 32 : cap;
}

static void free_all(gw_ctx* c) {
  if (c->st) cudaStreamSynchronize(c->st); else cudaDeviceSynchronize();
  for (void* p : c->owned) {
    if (c->cfg.dev_free) c->cfg.dev_free(c->cfg.alloc_user, p); else cudaFree(p);
  }
  c->owned.clear();
  if (c->h_mus) cudaFreeHost(c->h_mus);
  if (c->h_scr) cudaFreeHost(c->h_scr);
  c->h_mus = nullptr; c->h_scr = nullptr;
  for (auto& e : c->ev) if (e) { cudaEventDestroy(e); e = nullptr; }
  for (auto& e : c->pev) cudaEventDestroy(e);
  c->pev.clear();
  for (auto& e : c->uev) cudaEventDestroy(e);
  c->uev.clear();
  if (c->gexec) cudaGraphExecDestroy(c->gexec);
  if (c->graph) cudaGraphDestroy(c->graph);
  if (c->gst) cudaStreamDestroy(c->gst);
  for (auto& e : c->gev) if (e) { cudaEventDestroy(e); e = nullptr; }
  c->gexec = nullptr; c->graph = nullptr; c->gst = nullptr;
}

static inline void count(int n) { g_launches += n; }

// contractions on the tensor cores (the wait-timeout flag is then meaningful)
static inline bool uses_tc(const gw_ctx* c) {
  return c->cfg.contract_prec == GW_SPLIT_TF32 || c->hfmt != 0;
}
// the time-reversal reduction applies to forward stages over the full q range
static inline bool trs_reduce(const gw_ctx* c) { return c->trs && c->q0 == 0 && c->q1 == c->nk; }
// pointer to 16-bit element `e` of a buffer typed as float*
static inline float* hofs(float* p, int64_t e) { return (float*)((uint16_t*)p + e); }

static cudaError_t run_gett(const GettDesc& d, const void* A, Ty ta, const void* B, Ty tb, void* C, Ty tc, Ty acc,
                            gw_ctx* c) {
  count(d.ksplit > 1 ? 2 : 1);
  if (!c->prof) return gett(d, A, ta, B, tb, C, tc, acc, c->ws, c->ws_bytes, c->st);
  while (c->pev.size() < c->pused + 2) {
    cudaEvent_t e;
    cudaError_t r = cudaEventCreate(&e);
    if (r != cudaSuccess) return r;
    c->pev.push_back(e);
  }
  cudaEventRecord(c->pev[c->pused], c->st);
  cudaError_t r = gett(d, A, ta, B, tb, C, tc, acc, c->ws, c->ws_bytes, c->st);
  cudaEventRecord(c->pev[c->pused + 1], c->st);
  c->pused += 2;
  c->pflops += 8.0 * (double)d.M * (double)d.N * (double)d.K * (double)d.Z;
  c->plaunch += 1;
  return r;
}

// tensor-core launch with optional event timing; flops = useful complex-MAC flops
static cudaError_t run_umma(gw_ctx* c, double flops, const UmmaOperand& A, const UmmaOperand& B, int M, int N,
                            int64_t Kpad, int batch, void* C, bool c_fp64, double alpha, bool accumulate, int64_t c_ld,
                            int64_t c_zs, int ksplit = 1, int64_t row_inner = 0, int64_t row_s1 = 0,
                            int64_t col_inner = 0, int64_t col_s1 = 0, float* C_lo = nullptr,
                            int64_t kvalid = 0, const UmmaScale* scale = nullptr, const UmmaOut* out = nullptr,
                            const UmmaZ* zz = nullptr) {
  count(1);
  if (c->prof) {
    while (c->uev.size() < c->uused + 2) {
      cudaEvent_t e;
      cudaError_t r = cudaEventCreate(&e);
      if (r != cudaSuccess) return r;
      c->uev.push_back(e);
    }
    cudaEventRecord(c->uev[c->uused], c->st);
  }
  // named range around the contraction GEMMs of the P~0 / Sigma~ chains, so that a
  // profiler can select exactly these launches
  nvtxRangePushA("contraction");
  cudaError_t r = umma_gemm(A, B, M, N, Kpad, batch, C, c_fp64, alpha, accumulate, c_ld, c_zs, 3, c->info + 1, c->st,
                            ksplit, row_inner, row_s1, col_inner, col_s1, C_lo, scale, kvalid, out, zz);
  nvtxRangePop();
  if (c->prof) {
    cudaEventRecord(c->uev[c->uused + 1], c->st);
    c->uused += 2; c->uflops += flops; c->ulaunch += 1;
  }
  return r;
}

static cudaError_t run_bsm(gw_ctx* c, BsmDesc d) {
  // elements per block: a few waves of 2 blocks per SM, and a multiple of the
  // products one block computes at a time
  const int T = ((d.M + 3) / 4) * ((d.N + 3) / 4);
  const int ep = 256 / T < 1 ? 1 : 256 / T;
  const int64_t tot = d.G * d.E;
  const int64_t target = 152 * 2 * 4;
  int64_t per = (tot + target - 1) / target;
  per = (per + ep - 1) / ep * ep;
  d.per_block = (int)(per < 1 ? 1 : per);
  count(1);
  return bsm(d, c->st);
}

// Ge[k][t] = doubled operand of conj(G^k(t)) for C = A conj(Ge)^T (TF32 hi/lo); with a
// Hermitian G(t) that product is A G(t).  Gp (polarization only) holds the reversed
// plain operands G^k(t_{ntau-1-j}).
static cudaError_t build_gemb(gw_ctx* c, const double2* Gplus, const double2* Gminus) {
  const int64_t n2 = c->n2, gstep = (int64_t)c->nk * n2, per = 2 * (int64_t)c->nao * c->kpadA;
  cudaError_t e = cudaSuccess;
  for (int k = 0; k < c->nk && !e; ++k)
    e = embed_conj_batched(Gplus + (size_t)k * n2, c->ntau, gstep, c->nao, c->nao, c->Ge_hi + (size_t)k * c->ntau * per,
                           c->Ge_lo + (size_t)k * c->ntau * per, c->kpadA, per, c->st);
  count(c->nk);
  if (!c->Gp_hi || !Gminus) return e;
  // Gp[k][j] = doubled operand of G^k(t_{ntau-1-j}) for C = A Gp^T (the G(-t) factor up to its sign)
  for (int k = 0; k < c->nk && !e; ++k)
    e = embed_plain_batched(Gminus + (size_t)(c->ntau - 1) * gstep + (size_t)k * n2, c->ntau, -gstep, c->nao, c->nao,
                            c->Gp_hi + (size_t)k * c->ntau * per, c->Gp_lo + (size_t)k * c->ntau * per, c->kpadA, per,
                            c->st);
  count(c->nk);
  return e;
}

static GettDesc base_desc(int64_t M, int64_t N, int64_t K, int64_t Z) {
  GettDesc d{};
  d.M = M; d.N = N; d.K = K; d.Z = Z;
  d.az = d.bz = d.cz = I1(0);
  d.alpha = make_double2(1, 0); d.beta = make_double2(0, 0);
  d.ksplit = 1;
  return d;
}

// Y[z] = T (nrow x ntau) * X[z] (ntau x ncol): transforms along the tau axis, FP64 either
// way: digit-split products on the tensor cores (k_emul.cu) or the FP64 contraction kernel.
static cudaError_t transform(gw_ctx* c, const double2* T, const double2* X, double2* Y, int64_t nrow, int64_t ncol,
                             int64_t batch, int64_t xstride, int64_t ystride) {
  // K of each transform: TFf, TFb take tau values; TBf takes nwf, TBb nwb Matsubara values
  const double2* Ts[4] = {c->TFf, c->TBf, c->TFb, c->TBb};
  const int64_t Ks[4] = {c->ntau, c->nwf, c->ntau, c->nwb};
  int idx = -1;
  for (int i = 0; i < 4; ++i) if (Ts[i] == T) idx = i;
  if (idx < 0) return cudaErrorInvalidValue;
  const int64_t K = Ks[idx];
  if (c->emul && emul_digit_bytes(ncol, K) <= c->emA_bytes) {
    for (int64_t z = 0; z < batch; ++z) {
      cudaError_t e = emul_transform(c->Tdig[idx], c->Texp[idx], nrow, X + z * xstride, K, ncol, ncol,
                                     Y + z * ystride, ncol, c->emA, c->emAe, c->info + 1, c->st);
      if (e != cudaSuccess) return e;
    }
    count((int)(batch * (1 + emul_launches(K))));
    return cudaSuccess;
  }
  GettDesc d = base_desc(nrow, ncol, K, batch);
  d.am = I1(K); d.ak = I1(1);
  d.bk = I1(ncol); d.bn = I1(1); d.bz = I1(xstride);
  d.cm = I1(ncol); d.cn = I1(1); d.cz = I1(ystride);
  return run_gett(d, T, Ty::C128, X, Ty::C128, Y, Ty::C128, Ty::C128, c);
}

static int kidx(const int* m, int a, int b, int cc) {
  return ((a % m[0] + m[0]) % m[0] * m[1] + (b % m[1] + m[1]) % m[1]) * m[2] + (cc % m[2] + m[2]) % m[2];
}

// ------------------------------------------------------------------ init / destroy

static gw_status init_impl(const gw_config* cfg, const gw_grid* grid, const double* H0, const double* S,
                           const double* V, gw_ctx** out);

extern "C" gw_status gw_init(const gw_config* cfg, const double* H0, const double* S, const double* V,
                             gw_ctx** out) {
  return init_impl(cfg, nullptr, H0, S, V, out);
}

extern "C" gw_status gw_init_grid(const gw_config* cfg, const gw_grid* grid, const double* H0, const double* S,
                                  const double* V, gw_ctx** out) {
  if (out) *out = nullptr;
  if (!grid) return fail(nullptr, GW_ERR_ARG, "null grid");
  return init_impl(cfg, grid, H0, S, V, out);
}

static gw_status init_impl(const gw_config* cfg, const gw_grid* grid, const double* H0, const double* S,
                           const double* V, gw_ctx** out) {
  if (!out) return fail(nullptr, GW_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg || !H0 || !S || !V) return fail(nullptr, GW_ERR_ARG, "null config or input pointer");
  if (cfg->nao <= 0 || cfg->naux <= 0 || cfg->ntau <= 0 || cfg->kmesh[0] <= 0 || cfg->kmesh[1] <= 0 ||
      cfg->kmesh[2] <= 0)
    return fail(nullptr, GW_ERR_ARG, "sizes must be positive");
  if (cfg->nao > 96) return fail(nullptr, GW_ERR_ARG, "nao > 96 is not supported by the Dyson kernel");
  if (grid) {
    if (grid->ntau != cfg->ntau || grid->nwf <= 0 || grid->nwb <= 0)
      return fail(nullptr, GW_ERR_ARG, "grid: ntau must equal cfg->ntau and nwf, nwb be positive");
    if (!grid->tau || !grid->fermi_n || !grid->bose_m || !grid->TFf || !grid->TBf || !grid->TFb || !grid->TBb ||
        !grid->lb)
      return fail(nullptr, GW_ERR_ARG, "grid: null array");
  }
  if (!(cfg->beta > 0) || (!grid && (!cfg->fermi_n || !cfg->bose_m)))
    return fail(nullptr, GW_ERR_ARG, "bad beta or index sets");
  if (cfg->contract_prec != GW_FP64 && cfg->contract_prec != GW_FP32 && cfg->contract_prec != GW_SPLIT_TF32 &&
      cfg->contract_prec != GW_SPLIT_F16 && cfg->contract_prec != GW_SPLIT_BF16)
    return fail(nullptr, GW_ERR_ARG, "contract_prec not available");
  if ((cfg->flags & GW_BORROW_V) && !(cfg->flags & GW_INPUT_DEVICE))
    return fail(nullptr, GW_ERR_ARG, "GW_BORROW_V needs GW_INPUT_DEVICE");
  const int nwf_ = grid ? grid->nwf : cfg->ntau, nwb_ = grid ? grid->nwb : cfg->ntau;
  const int32_t* fn_h = grid ? grid->fermi_n : cfg->fermi_n;
  const int32_t* bm_h = grid ? grid->bose_m : cfg->bose_m;
  for (int i = 0; i < nwf_; ++i)
    for (int j = i + 1; j < nwf_; ++j)
      if (fn_h[i] == fn_h[j]) return fail(nullptr, GW_ERR_ARG, "repeated Matsubara index");
  for (int i = 0; i < nwb_; ++i)
    for (int j = i + 1; j < nwb_; ++j)
      if (bm_h[i] == bm_h[j]) return fail(nullptr, GW_ERR_ARG, "repeated Matsubara index");
  gw_ctx* c = new (std::nothrow) gw_ctx();
  if (!c) return fail(nullptr, GW_ERR_OOM, "host allocation failed");
  c->cfg = *cfg;
  c->nao = cfg->nao; c->naux = cfg->naux; c->ntau = cfg->ntau;
  c->nwf = c->nw = nwf_; c->nwb = nwb_;
  c->nk = cfg->kmesh[0] * cfg->kmesh[1] * cfg->kmesh[2];
  c->q0 = 0; c->q1 = c->nk;
  c->n2 = (int64_t)c->nao * c->nao; c->na2 = (int64_t)c->naux * c->naux;
  c->spin = cfg->spin_factor > 0 ? cfg->spin_factor : 2;
  c->st = (cudaStream_t)cfg->stream;
  if (c->cfg.mu_tol <= 0) c->cfg.mu_tol = 1e-9;
  if (c->cfg.mu_maxit <= 0) c->cfg.mu_maxit = 400;
  const int nk = c->nk, nao = c->nao, naux = c->naux, ntau = c->ntau;
  const int64_t n2 = c->n2, na2 = c->na2;
  // k-mesh tables: k + q and k - q componentwise modulo the mesh
  c->kplus.resize((size_t)nk * nk); c->kminus.resize((size_t)nk * nk);
  const int* m = cfg->kmesh;
  for (int q = 0; q < nk; ++q) {
    int q1 = q / (m[1] * m[2]), q2 = (q / m[2]) % m[1], q3 = q % m[2];
    for (int k = 0; k < nk; ++k) {
      int k1 = k / (m[1] * m[2]), k2 = (k / m[2]) % m[1], k3 = k % m[2];
      c->kplus[(size_t)q * nk + k] = kidx(m, k1 + q1, k2 + q2, k3 + q3);
      c->kminus[(size_t)q * nk + k] = kidx(m, k1 - q1, k2 - q2, k3 - q3);
    }
  }
  c->trs = (cfg->flags & GW_TRS) != 0;
  c->kneg.resize((size_t)nk);
  for (int k = 0; k < nk; ++k) {
    const int k1 = k / (m[1] * m[2]), k2 = (k / m[2]) % m[1], k3 = k % m[2];
    c->kneg[(size_t)k] = kidx(m, -k1, -k2, -k3);
  }
  auto A = [&](size_t bytes) { return dalloc(c, bytes); };
  const size_t cb = sizeof(double2);
  const size_t vbytes = (size_t)nk * nk * naux * n2 * cb;
  bool ok = true;
  auto need = [&](void* p) { ok = ok && p != nullptr; return p; };
  c->H0 = (double2*)need(A(nk * n2 * cb));
  c->S = (double2*)need(A(nk * n2 * cb));
  if (cfg->flags & GW_BORROW_V) c->V = (double2*)V;
  else c->V = (double2*)need(A(vbytes));
  const bool lowp = cfg->contract_prec != GW_FP64;
  if (lowp) c->V32 = (float2*)need(A(vbytes / 2));
  const int nwf = c->nwf, nwb = c->nwb;
  const int kmax = ntau > nwf ? (ntau > nwb ? ntau : nwb) : (nwf > nwb ? nwf : nwb);
  c->tau = (double*)need(A(ntau * 8)); c->lb = (double*)need(A(ntau * 8)); c->l0 = (double*)need(A(ntau * 8));
  c->wn = (double*)need(A(nwf * 8));
  // transforms: TFf [nwf][ntau], TBf [ntau][nwf], TFb [nwb][ntau], TBb [ntau][nwb]
  c->TFf = (double2*)need(A((size_t)nwf * ntau * cb)); c->TBf = (double2*)need(A((size_t)ntau * nwf * cb));
  c->TFb = (double2*)need(A((size_t)nwb * ntau * cb)); c->TBb = (double2*)need(A((size_t)ntau * nwb * cb));
  c->emul = !(cfg->flags & GW_FP64_NATIVE);
  if (c->emul) {
    const int64_t ncmax = (int64_t)na2 > (int64_t)nk * n2 ? (int64_t)na2 : (int64_t)nk * n2;
    c->emA_bytes = emul_digit_bytes(ncmax, kmax);
    c->emA = (float*)need(A(c->emA_bytes));
    c->emAe = (int*)need(A((size_t)ncmax * 4));
    const int rows[4] = {nwf, ntau, nwb, ntau}, kk[4] = {ntau, nwf, ntau, nwb};
    for (int i = 0; i < 4; ++i) {
      c->Tdig[i] = (float*)need(A(emul_digit_bytes(2 * (int64_t)rows[i], kk[i])));
      c->Texp[i] = (int*)need(A((size_t)rows[i] * 4));
    }
  }
  c->r = (double2*)need(A(nwf * cb));
  c->d_fn = (int*)need(A(nwf * 4)); c->d_bm = (int*)need(A(nwb * 4));
  const size_t gsz = (size_t)ntau * nk * n2 * cb, gszw = (size_t)nwf * nk * n2 * cb;
  c->G_tau = (double2*)need(A(gsz)); c->G_iw = (double2*)need(A(gszw)); c->G_prev = (double2*)need(A(gsz));
  c->Stau = (double2*)need(A(gsz)); c->Siw = (double2*)need(A(gszw)); c->Siw_new = (double2*)need(A(gszw));
  c->gamma = (double2*)need(A(nk * n2 * cb)); c->tQ = (double2*)need(A(naux * cb));
  c->Sinf = (double2*)need(A(nk * n2 * cb)); c->Sinf_new = (double2*)need(A(nk * n2 * cb));
  const size_t psz = (size_t)nk * ntau * na2 * cb, pszw = (size_t)nk * nwb * na2 * cb;
  c->P0_tau = (double2*)need(A(psz)); c->P_iw = (double2*)need(A(pszw)); c->P_tau = (double2*)need(A(psz));
  // chain intermediates: max(ntau * naux * n2, nk * naux * n2) complex of the contraction type
  size_t chn = (size_t)(ntau > nk ? ntau : nk) * naux * n2;
  c->ch_bytes = chn * (lowp ? 8 : 16);
  c->chA = need(A(c->ch_bytes)); c->chB = need(A(c->ch_bytes));
  if (lowp) {
    c->G32 = (float2*)need(A(gsz / 2)); c->P32 = (float2*)need(A(psz / 2));
    c->gam32 = (float2*)need(A(nk * n2 * 8));
  }
  if (cfg->contract_prec == GW_SPLIT_TF32) {
    c->kpadP = (2 * n2 + 31) / 32 * 32;
    c->kpadS = (2 * (int64_t)naux + 31) / 32 * 32;
    // the last P~0 step of pgroup k-points is one GEMM with their K ranges side by
    // side (one FP64 read-modify-write of P~0^q per group, long K loops); the group
    // is as large as kZGroupBytes of Z hi/lo planes allow
    const size_t zk = (size_t)ntau * naux * c->kpadP * 4, vk = (size_t)2 * naux * c->kpadP * 4;
    c->pgroup = (int)(opt_budget(kZGroupBytes) / (2 * zk));
    if (c->pgroup > nk) c->pgroup = nk;
    if (g_pgroup_cap > 0 && c->pgroup > g_pgroup_cap) c->pgroup = g_pgroup_cap;
    if (c->pgroup < 1) c->pgroup = 1;
    size_t zb = 0;
    for (;;) {   // a smaller group when the planes do not fit (one k-point at least)
      zb = zk * c->pgroup;
      const size_t vb = vk * c->pgroup;
      c->Zhi = (float*)A(zb); c->Zlo = (float*)A(zb); c->Vhi = (float*)A(vb); c->Vlo = (float*)A(vb);
      if ((c->Zhi && c->Zlo && c->Vhi && c->Vlo) || c->pgroup == 1) break;
      dfree(c, c->Zhi); dfree(c, c->Zlo); dfree(c, c->Vhi); dfree(c, c->Vlo);
      c->pgroup /= 2;
    }
    need(c->Zhi); need(c->Zlo); need(c->Vhi); need(c->Vlo);
    const size_t pb = (size_t)ntau * naux * c->kpadS * 4, tb = (size_t)2 * n2 * c->kpadS * 4;
    c->Pchi = (float*)need(A(pb)); c->Pclo = (float*)need(A(pb));
    c->zbytes = zb;
    if (nao <= 64) {
      const bool small_tc = (cfg->flags & GW_SMALL_TENSOR) ? true : (cfg->flags & GW_SMALL_SIMT) ? false
                                                                                                 : kTensorSmallSteps;
      if (small_tc) {   // nao-sized steps on tensor cores
        c->kpadA = (2 * (int64_t)nao + 31) / 32 * 32;
        const size_t vs = (size_t)naux * nao * c->kpadA * 4, ge = (size_t)nk * ntau * 2 * nao * c->kpadA * 4;
        const size_t xs = (size_t)ntau * naux * nao * c->kpadA * 4;
        c->Vs_hi = (float*)need(A(vs)); c->Vs_lo = (float*)need(A(vs));
        c->Ge_hi = (float*)need(A(ge)); c->Ge_lo = (float*)need(A(ge));
        c->Gp_hi = (float*)need(A(ge)); c->Gp_lo = (float*)need(A(ge));
        c->Xs_hi = (float*)need(A(xs)); c->Xs_lo = (float*)need(A(xs));
      }
      c->kpad3 = (2 * (int64_t)naux * nao + 31) / 32 * 32;
      c->y3bytes = (size_t)ntau * nao * c->kpad3 * 4;
      c->Y3hi = (float*)need(A(c->y3bytes)); c->Y3lo = (float*)need(A(c->y3bytes));
      c->W3hi = (float*)need(A((size_t)2 * nao * c->kpad3 * 4)); c->W3lo = (float*)need(A((size_t)2 * nao * c->kpad3 * 4));
    }
    c->VThi = (float*)need(A(tb)); c->VTlo = (float*)need(A(tb));
  }
  if (cfg->contract_prec == GW_SPLIT_F16 || cfg->contract_prec == GW_SPLIT_BF16) {
    // every contraction GEMM on the tensor cores with 16-bit pieces: operand rows padded to
    // 64 elements (128 bytes), two bytes per element, one exponent per operand row
    c->hfmt = cfg->contract_prec == GW_SPLIT_F16 ? 1 : 2;
    auto r64 = [](int64_t x) { return (x + 63) / 64 * 64; };
    c->kpadA = r64(2 * (int64_t)nao);
    c->kpadP = r64(2 * n2);
    c->kpadS = r64(2 * (int64_t)naux);
    c->kpad3 = r64(2 * (int64_t)naux * nao);
    const size_t zk = (size_t)ntau * naux * c->kpadP * 2, vk = (size_t)2 * naux * c->kpadP * 2;
    c->pgroup = (int)(opt_budget(kZGroupBytes) / (2 * zk));
    if (c->pgroup > nk) c->pgroup = nk;
    if (g_pgroup_cap > 0 && c->pgroup > g_pgroup_cap) c->pgroup = g_pgroup_cap;
    if (c->pgroup < 1) c->pgroup = 1;
    size_t zb = 0;
    for (;;) {
      zb = zk * c->pgroup;
      const size_t vb = vk * c->pgroup;
      c->Zhi = (float*)A(zb); c->Zlo = (float*)A(zb); c->Vhi = (float*)A(vb); c->Vlo = (float*)A(vb);
      if ((c->Zhi && c->Zlo && c->Vhi && c->Vlo) || c->pgroup == 1) break;
      dfree(c, c->Zhi); dfree(c, c->Zlo); dfree(c, c->Vhi); dfree(c, c->Vlo);
      c->pgroup /= 2;
    }
    need(c->Zhi); need(c->Zlo); need(c->Vhi); need(c->Vlo);
    c->zbytes = zb;
    // k-points per launch of the chains: enough output tiles for ~16 rounds of the SMs in the
    // nao-sized steps (small systems put several (k, k+q) pairs into each GEMM); the per-k
    // operand buffers below hold that many blocks
    c->pbatch = chain_pbatch(nao, naux, nk, ntau);
    const size_t kb = (size_t)c->pbatch;
    const size_t pb = (size_t)ntau * naux * c->kpadS * 2, tb = (size_t)2 * n2 * c->kpadS * 2;
    c->Pchi = (float*)need(A(pb)); c->Pclo = (float*)need(A(pb));
    c->VThi = (float*)need(A(kb * tb)); c->VTlo = (float*)need(A(kb * tb));
    const size_t vs = (size_t)naux * nao * c->kpadA * 2, ge = (size_t)nk * ntau * 2 * nao * c->kpadA * 2;
    const size_t xs = (size_t)ntau * naux * nao * c->kpadA * 2;
    c->Vs_hi = (float*)need(A(kb * vs)); c->Vs_lo = (float*)need(A(kb * vs));
    c->Ge_hi = (float*)need(A(ge)); c->Ge_lo = (float*)need(A(ge));
    c->Gp_hi = (float*)need(A(ge)); c->Gp_lo = (float*)need(A(ge));
    if (kb > 1) {
      const size_t gq = kb * ntau * 2 * nao * c->kpadA * 2;
      c->Gq_hi = (float*)need(A(gq)); c->Gq_lo = (float*)need(A(gq));
      c->eGq = (int*)need(A(kb * ntau * 4));
    }
    c->Xs_hi = (float*)need(A(kb * xs)); c->Xs_lo = (float*)need(A(kb * xs));
    c->y3bytes = (size_t)ntau * nao * c->kpad3 * 2;
    c->Y3hi = (float*)need(A(kb * c->y3bytes)); c->Y3lo = (float*)need(A(kb * c->y3bytes));
    c->W3hi = (float*)need(A(kb * 2 * nao * c->kpad3 * 2)); c->W3lo = (float*)need(A(kb * 2 * nao * c->kpad3 * 2));
    c->vQmax = (float*)need(A((size_t)naux * 4)); c->vQrs = (float*)need(A((size_t)naux * 4));
    c->gn = (float*)need(A((size_t)4 * ntau * 4));
    c->eVQ = (int*)need(A((size_t)naux * 4)); c->eVall = (int*)need(A(16));
    c->eV1 = (int*)need(A(kb * naux * nao * 4));
    c->eY = (int*)need(A((size_t)ntau * naux * 4)); c->eZ = (int*)need(A((size_t)ntau * naux * 4));
    c->eGe = (int*)need(A((size_t)nk * ntau * 4)); c->eGp = (int*)need(A((size_t)nk * ntau * 4));
    c->ePc = (int*)need(A((size_t)ntau * naux * 4)); c->ePs = (int*)need(A((size_t)ntau * naux * 4));
    c->eY3 = (int*)need(A((size_t)ntau * 4));
  }
  // workspace: split-K partials and the screened-solve panels
  size_t ws = screened_work_bytes(naux, (int64_t)nk * nwb);
  const size_t ws_cap = (size_t)4 << 30;
  size_t ws_min = screened_work_bytes(naux, 1) * 8;
  if (ws > ws_cap) ws = ws_cap;
  if (ws < ws_min) ws = ws_min;
  size_t splitk = (size_t)64 * ntau * n2 * cb;          // Sigma last contraction, ksplit <= 64
  size_t splitk2 = (size_t)64 * nk * n2 * cb;           // exchange
  if (ws < splitk) ws = splitk;
  if (ws < splitk2) ws = splitk2;
  int ld = 0;
  if (!grid) {
    size_t gws = grid_ws_bytes(ntau, cfg->fermi_n, cfg->bose_m, &ld);
    if (ws < gws) ws = gws;
  }
  c->ws_bytes = ws;
  c->ws = need(A(ws));
  c->partial = (double*)need(A((size_t)(ntau > nwf ? ntau : nwf) * nk * 8));
  if (c->trs) {
    c->d_kneg = (int*)need(A((size_t)nk * 4));
    c->d_kneed = (int*)need(A((size_t)nk * 4));
    c->d_vpart = (int*)need(A((size_t)nk * nk * 4));
  }
  c->mus = (MuState*)need(A(sizeof(MuState)));
  c->info = (int*)need(A(64));
  c->dscr = (double*)need(A(64 * 8));
  if (ok && c->emul && screened_refine_ok(naux)) {
    // refined screened solve: as many (q, Omega) systems per batch as the budget
    // allows; without room for one system the FP64 Gauss-Jordan solve is used
    const int64_t cnt = (int64_t)nk * nwb;
    const size_t per = screened_refine_bytes(naux, 1);
    int64_t chunk = (int64_t)(opt_budget(kRefineBytes) / per);
    if (chunk < 1) chunk = 1;
    if (chunk > cnt) chunk = cnt;
    for (; chunk >= 1; chunk /= 2) {
      c->irws_bytes = screened_refine_bytes(naux, chunk);
      c->irws = A(c->irws_bytes);
      if (c->irws) break;
    }
    if (!c->irws) c->irws_bytes = 0;
  }
  if (!ok) { free_all(c); delete c; return fail(nullptr, GW_ERR_OOM, "device allocation failed"); }
  if (cudaMallocHost(&c->h_mus, sizeof(MuState)) != cudaSuccess ||
      cudaMallocHost(&c->h_scr, 64 * 8) != cudaSuccess) {
    free_all(c); delete c; return fail(nullptr, GW_ERR_OOM, "pinned allocation failed");
  }
  for (auto& e : c->ev) cudaEventCreate(&e);
  cudaStream_t st = c->st;
  cudaMemcpyKind kind = (cfg->flags & GW_INPUT_DEVICE) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
  gw_status s = GW_OK;
  auto chk = [&](cudaError_t e, const char* what) {
    if (e != cudaSuccess && s == GW_OK) { s = GW_ERR_CUDA; c->err = std::string(what) + ": " + cudaGetErrorString(e); }
  };
  chk(cudaMemcpyAsync(c->H0, H0, nk * n2 * cb, kind, st), "H0 copy");
  chk(cudaMemcpyAsync(c->S, S, nk * n2 * cb, kind, st), "S copy");
  if (!(cfg->flags & GW_BORROW_V)) chk(cudaMemcpyAsync(c->V, V, vbytes, kind, st), "V copy");
  chk(cudaMemcpyAsync(c->d_fn, fn_h, nwf * 4, cudaMemcpyHostToDevice, st), "index copy");
  chk(cudaMemcpyAsync(c->d_bm, bm_h, nwb * 4, cudaMemcpyHostToDevice, st), "index copy");
  chk(cudaMemsetAsync(c->info, 0, 64, st), "memset");
  chk(cudaMemsetAsync(c->Sinf, 0, nk * n2 * cb, st), "memset");
  chk(cudaMemsetAsync(c->Siw, 0, gszw, st), "memset");
  if (c->Zhi && !c->hfmt) {
    chk(cudaMemsetAsync(c->Zhi, 0, c->zbytes, st), "memset");
    chk(cudaMemsetAsync(c->Zlo, 0, c->zbytes, st), "memset");
  }
  if (c->Y3hi && !c->hfmt) {
    chk(cudaMemsetAsync(c->Y3hi, 0, c->y3bytes, st), "memset");
    chk(cudaMemsetAsync(c->Y3lo, 0, c->y3bytes, st), "memset");
    if (c->Xs_hi) {
      const size_t xs = (size_t)ntau * naux * nao * c->kpadA * 4;
      chk(cudaMemsetAsync(c->Xs_hi, 0, xs, st), "memset");
      chk(cudaMemsetAsync(c->Xs_lo, 0, xs, st), "memset");
    }
  }
  // grid and transforms: the Chebyshev grid built here, or the caller's sampling grid
  if (!grid) {
    chk(grid_build_ws(ntau, cfg->beta, c->d_fn, c->d_bm, ld, c->ws, c->tau, c->TFf, c->TFb, c->lb, c->l0, st),
        "grid");
    count(4);
    chk(cudaMemcpyAsync(c->TBf, c->TFf, (size_t)ntau * ntau * cb, cudaMemcpyDeviceToDevice, st), "copy");
    chk(cudaMemcpyAsync(c->TBb, c->TFb, (size_t)ntau * ntau * cb, cudaMemcpyDeviceToDevice, st), "copy");
    chk(invert_small_gj(c->TBf, ntau, c->info, st), "TBf");
    chk(invert_small_gj(c->TBb, ntau, c->info, st), "TBb");
  } else {
    chk(cudaMemcpyAsync(c->tau, grid->tau, ntau * 8, cudaMemcpyHostToDevice, st), "grid copy");
    chk(cudaMemcpyAsync(c->lb, grid->lb, ntau * 8, cudaMemcpyHostToDevice, st), "grid copy");
    chk(cudaMemsetAsync(c->l0, 0, ntau * 8, st), "memset");
    chk(cudaMemcpyAsync(c->TFf, grid->TFf, (size_t)nwf * ntau * cb, cudaMemcpyHostToDevice, st), "grid copy");
    chk(cudaMemcpyAsync(c->TBf, grid->TBf, (size_t)ntau * nwf * cb, cudaMemcpyHostToDevice, st), "grid copy");
    chk(cudaMemcpyAsync(c->TFb, grid->TFb, (size_t)nwb * ntau * cb, cudaMemcpyHostToDevice, st), "grid copy");
    chk(cudaMemcpyAsync(c->TBb, grid->TBb, (size_t)ntau * nwb * cb, cudaMemcpyHostToDevice, st), "grid copy");
  }
  chk(density_weights(ntau, nwf, c->lb, c->TBf, c->r, st), "weights");
  if (c->emul) {
    chk(cudaMemsetAsync(c->emA, 0, c->emA_bytes, st), "memset");
    const double2* Ts[4] = {c->TFf, c->TBf, c->TFb, c->TBb};
    const int rows[4] = {nwf, ntau, nwb, ntau}, kk[4] = {ntau, nwf, ntau, nwb};
    for (int i = 0; i < 4; ++i)
      chk(emul_split_b(Ts[i], rows[i], kk[i], kk[i], c->Tdig[i], c->Texp[i], st), "digits");
  }
  chk(fermi_freqs(nwf, cfg->beta, c->d_fn, c->wn, st), "freqs");
  count(4);
  if (lowp) { chk(to_c64(c->V, c->V32, vbytes / cb, st), "V32"); count(1); }
  if (c->hfmt) {
    // V's norms per Q over every slab fix the exponents of the V operands (uniform over the
    // (k, k') pairs, so that the operands of one grouped GEMM share them)
    chk(v_norms(c->V, (int64_t)nk * nk, naux, nao, c->vQmax, c->vQrs, st), "V norms");
    chk(row_exps(c->vQmax, naux, c->eVQ, st), "V exponents");
    chk(max_exp(c->vQmax, naux, c->eVall + 1, st), "V exponent");
    count(3);
    chk(cudaMemsetAsync(c->Zhi, 0, c->zbytes, st), "memset");
    chk(cudaMemsetAsync(c->Zlo, 0, c->zbytes, st), "memset");
    // the padding columns of the chain intermediates stay zero (every k block)
    chk(cudaMemsetAsync(c->Y3hi, 0, (size_t)c->pbatch * c->y3bytes, st), "memset");
    chk(cudaMemsetAsync(c->Y3lo, 0, (size_t)c->pbatch * c->y3bytes, st), "memset");
    const size_t xs = (size_t)c->pbatch * ntau * naux * nao * c->kpadA * 2;
    chk(cudaMemsetAsync(c->Xs_hi, 0, xs, st), "memset");
    chk(cudaMemsetAsync(c->Xs_lo, 0, xs, st), "memset");
  }
  // input checks
  chk(cudaMemsetAsync(c->dscr, 0, 64 * 8, st), "memset");
  std::vector<int> kneed((size_t)nk), vpart((size_t)nk * nk);
  if (c->trs) {
    for (int k = 0; k < nk; ++k) {
      kneed[(size_t)k] = c->kneg[(size_t)k] < k ? 1 : 0;
      for (int k2 = 0; k2 < nk; ++k2) vpart[(size_t)k * nk + k2] = c->kneg[(size_t)k] * nk + c->kneg[(size_t)k2];
    }
    chk(cudaMemcpyAsync(c->d_kneg, c->kneg.data(), (size_t)nk * 4, cudaMemcpyHostToDevice, st), "copy");
    chk(cudaMemcpyAsync(c->d_kneed, kneed.data(), (size_t)nk * 4, cudaMemcpyHostToDevice, st), "copy");
    chk(cudaMemcpyAsync(c->d_vpart, vpart.data(), (size_t)nk * nk * 4, cudaMemcpyHostToDevice, st), "copy");
  }
  if (!(cfg->flags & GW_SKIP_CHECKS)) {
    if (c->trs) {   // H0(-k) = conj H0(k), S(-k) = conj S(k), V^{-k,-k'} = conj V^{kk'}
      chk(check_trs(c->H0, nk, n2, c->d_kneg, c->dscr + 10, st), "check");
      chk(check_trs(c->S, nk, n2, c->d_kneg, c->dscr + 12, st), "check");
      chk(check_trs(c->V, (int64_t)nk * nk, (int64_t)naux * n2, c->d_vpart, c->dscr + 14, st), "check");
      count(3);
    }
    chk(check_herm(c->H0, nao, nk, c->dscr, st), "check");
    chk(check_herm(c->S, nao, nk, c->dscr + 2, st), "check");
    chk(check_v_pairing(c->V, nk, naux, nao, c->dscr + 4, st), "check");
    count(3);
  }
  chk(cudaMemcpyAsync(c->h_scr, c->dscr, 64 * 8, cudaMemcpyDeviceToHost, st), "copy");
  int h_info = 0;
  chk(cudaMemcpyAsync(&h_info, c->info, 4, cudaMemcpyDeviceToHost, st), "copy");
  int h_ev = 0;
  if (c->hfmt) chk(cudaMemcpyAsync(&h_ev, c->eVall + 1, 4, cudaMemcpyDeviceToHost, st), "copy");
  chk(cudaStreamSynchronize(st), "sync");
  if (c->hfmt) {
    // uniform exponent of the transposed V operands: max |V| 2^-e < 2^15
    c->h_Evmax = h_ev;
    const int ev = h_ev - 15;
    chk(cudaMemcpy(c->eVall, &ev, 4, cudaMemcpyHostToDevice), "copy");
  }
  if (s == GW_OK && h_info) { s = GW_ERR_SINGULAR; c->err = "transform matrix is singular"; }
  if (s == GW_OK && !(cfg->flags & GW_SKIP_CHECKS)) {
    const double* h = c->h_scr;
    if (!std::isfinite(h[1]) || !std::isfinite(h[3]) || !std::isfinite(h[5])) {
      s = GW_ERR_ARG;
      c->err = std::string("non-finite value in ") + (!std::isfinite(h[1]) ? "H0" : !std::isfinite(h[3]) ? "S" : "V");
    } else if (h[0] > 1e-10 * (h[1] > 1 ? h[1] : 1)) { s = GW_ERR_ARG; c->err = "H0 is not Hermitian"; }
    else if (h[2] > 1e-10 * (h[3] > 1 ? h[3] : 1)) { s = GW_ERR_ARG; c->err = "S is not Hermitian"; }
    else if (h[4] > 1e-10 * (h[5] > 1e-300 ? h[5] : 1)) { s = GW_ERR_ARG; c->err = "V^{k'k}(Q) != V^{kk'}(Q)^H"; }
    else if (c->trs && (h[10] > 1e-10 * (h[11] > 1 ? h[11] : 1) || h[12] > 1e-10 * (h[13] > 1 ? h[13] : 1) ||
                        h[14] > 1e-10 * (h[15] > 1e-300 ? h[15] : 1))) {
      s = GW_ERR_ARG;
      c->err = "GW_TRS: inputs are not time-reversal symmetric (H0(-k) = conj H0(k), S(-k) = conj S(k), "
               "V^{-k,-k'} = conj V^{kk'} within 1e-10)";
    }
  }
  if (s != GW_OK) { g_init_err = c->err; free_all(c); delete c; return s; }
  // zero self-energy and the grid are defined from the start
  for (gw_quantity q : {GW_Q_SIGMA_INF, GW_Q_SIGMA_IW, GW_Q_TFF, GW_Q_TBF, GW_Q_TFB, GW_Q_TBB, GW_Q_LB, GW_Q_TAU})
    mark(c, q);
  *out = c;
  return GW_OK;
}

extern "C" gw_status gw_destroy(gw_ctx* c) {
  if (!c) return GW_ERR_ARG;
  free_all(c);
  delete c;
  return GW_OK;
}

extern "C" const char* gw_last_error(const gw_ctx* c) { return c ? c->err.c_str() : g_init_err.c_str(); }
extern "C" int64_t gw_kernel_launches(const gw_ctx*) { return (int64_t)g_launches.load(); }

// ------------------------------------------------------------------ get / set

static bool qinfo(gw_ctx* c, gw_quantity q, void** p, size_t* bytes, bool* settable) {
  const size_t cb = 16;
  const size_t gsz = (size_t)c->ntau * c->nk * c->n2 * cb, ksz = (size_t)c->nk * c->n2 * cb;
  const size_t gszw = (size_t)c->nwf * c->nk * c->n2 * cb;
  const size_t psz = (size_t)c->nk * c->ntau * c->na2 * cb, pszw = (size_t)c->nk * c->nwb * c->na2 * cb;
  const size_t tszf = (size_t)c->ntau * c->nwf * cb, tszb = (size_t)c->ntau * c->nwb * cb;
  *settable = false;
  switch (q) {
    case GW_Q_G_TAU: *p = c->G_tau; *bytes = gsz; *settable = true; return true;
    case GW_Q_G_IW: *p = c->G_iw; *bytes = gszw; return true;
    case GW_Q_SIGMA_INF: *p = c->Sinf; *bytes = ksz; *settable = true; return true;
    case GW_Q_SIGMA_INF_NEW: *p = c->Sinf_new; *bytes = ksz; return true;
    case GW_Q_SIGMA_TAU: *p = c->Stau; *bytes = gsz; *settable = true; return true;
    case GW_Q_SIGMA_IW: *p = c->Siw; *bytes = gszw; *settable = true; return true;
    case GW_Q_P0_TAU: *p = c->P0_tau; *bytes = psz; *settable = true; return true;
    case GW_Q_P0_IW: *p = c->P_iw; *bytes = pszw; *settable = true; return true;
    case GW_Q_P_IW: *p = c->P_iw; *bytes = pszw; return true;
    case GW_Q_P_TAU: *p = c->P_tau; *bytes = psz; *settable = true; return true;
    case GW_Q_GAMMA: *p = c->gamma; *bytes = ksz; return true;
    case GW_Q_TFF: *p = c->TFf; *bytes = tszf; return true;
    case GW_Q_TBF: *p = c->TBf; *bytes = tszf; return true;
    case GW_Q_TFB: *p = c->TFb; *bytes = tszb; return true;
    case GW_Q_TBB: *p = c->TBb; *bytes = tszb; return true;
    case GW_Q_LB: *p = c->lb; *bytes = (size_t)c->ntau * 8; return true;
    case GW_Q_TAU: *p = c->tau; *bytes = (size_t)c->ntau * 8; return true;
    default: return false;
  }
}

extern "C" gw_status gw_set(gw_ctx* c, gw_quantity q, const void* src, size_t bytes, int on_device) {
  if (!c || !src) return fail(c, GW_ERR_ARG, "null argument");
  if (q == GW_Q_MU) {
    if (bytes != 8 || on_device) return fail(c, GW_ERR_ARG, "mu is one host double");
    c->mu = *(const double*)src; c->have_mu = true;
    mark(c, GW_Q_MU);
    return GW_OK;
  }
  void* p; size_t nb; bool settable;
  if (!qinfo(c, q, &p, &nb, &settable) || !settable) return fail(c, GW_ERR_ARG, "quantity is not settable");
  if (bytes != nb) return fail(c, GW_ERR_ARG, "byte count does not match the quantity");
  CK(cudaMemcpyAsync(p, src, nb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c->st));
  if (!on_device) CK(cudaStreamSynchronize(c->st));
  mark(c, q);
  if (q == GW_Q_G_TAU) c->have_G = true;
  if (q == GW_Q_P0_IW) { c->have_P0 = true; unmark(c, GW_Q_P_IW); }
  if (q == GW_Q_P_TAU) c->have_P = true;
  if (q == GW_Q_SIGMA_INF || q == GW_Q_SIGMA_IW) c->have_sigma = true;
  return GW_OK;
}

extern "C" gw_status gw_get(gw_ctx* c, gw_quantity q, void* dst, size_t bytes, int on_device) {
  if (!c || !dst) return fail(c, GW_ERR_ARG, "null argument");
  if (q == GW_Q_MU || q == GW_Q_N_ELEC) {
    if (bytes != 8 || on_device) return fail(c, GW_ERR_ARG, "scalar is one host double");
    if (!(c->valid & qbit(q))) return fail(c, GW_ERR_STATE, "no chemical potential yet");
    *(double*)dst = q == GW_Q_MU ? c->mu : c->n_at_mu;
    return GW_OK;
  }
  void* p; size_t nb; bool settable;
  if (!qinfo(c, q, &p, &nb, &settable)) return fail(c, GW_ERR_ARG, "unknown quantity");
  if (bytes != nb) return fail(c, GW_ERR_ARG, "byte count does not match the quantity");
  if (!(c->valid & qbit(q)))
    return fail(c, GW_ERR_STATE, "quantity " + std::to_string((int)q) + " has not been computed or set yet");
  CK(cudaMemcpyAsync(dst, p, nb, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c->st));
  if (!on_device) CK(cudaStreamSynchronize(c->st));
  return GW_OK;
}

extern "C" gw_status gw_reset_sigma(gw_ctx* c) {
  if (!c) return GW_ERR_ARG;
  c->have_sigma = false;
  CK(cudaMemsetAsync(c->Sinf, 0, (size_t)c->nk * c->n2 * 16, c->st));
  CK(cudaMemsetAsync(c->Siw, 0, (size_t)c->nwf * c->nk * c->n2 * 16, c->st));
  return GW_OK;
}

// ------------------------------------------------------------------ A1: gamma, J, K

static gw_status exchange(gw_ctx* c, const double2* gamma, double2* out) {
  // K^k_ij = -(1/Nk) sum_{k',Q,a,b} V^{kk'}_ia(Q) gamma^{k'}_ab V^{k'k}_bj(Q)    (Eq. HF_K)
  const int nk = c->nk, nao = c->nao, naux = c->naux;
  const int64_t n2 = c->n2, slab = (int64_t)naux * n2;
  const bool f32 = c->cfg.contract_prec != GW_FP64;
  const Ty tv = f32 ? Ty::C64 : Ty::C128, acc = f32 ? Ty::C64 : Ty::C128;
  const void* Vp = f32 ? (const void*)c->V32 : (const void*)c->V;
  const void* gp = gamma;
  Ty tg = Ty::C128;
  if (f32) { CK(to_c64(gamma, c->gam32, nk * n2, c->st)); count(1); gp = c->gam32; tg = Ty::C64; }
  const size_t es = f32 ? 8 : 16;
  for (int kp = 0; kp < nk; ++kp) {
    // Y[k][i][Q][b] = sum_a V^{k k'}[Q][i][a] gamma^{k'}[a][b]    (batch over k)
    GettDesc d = base_desc((int64_t)naux * nao, nao, nao, nk);
    d.am = I1(nao); d.ak = I1(1); d.az = I1((int64_t)nk * slab);
    d.bk = I1(nao); d.bn = I1(1); d.bz = I1(0);
    d.cm = I2(nao, nao, (int64_t)naux * nao); d.cn = I1(1); d.cz = I1(slab);
    const char* Vb = (const char*)Vp + (size_t)kp * slab * es;
    const char* gb = (const char*)gp + (size_t)kp * n2 * es;
    if (f32 && nao <= 64) {
      BsmDesc b{};
      b.M = b.N = b.K = nao; b.G = nk; b.E = naux; b.alpha = 1.f;
      b.A = (const float2*)Vb; b.a_gs = (int64_t)nk * slab; b.a_es = n2; b.a_rs = nao; b.a_cs = 1;
      b.B = (const float2*)gb; b.b_gs = 0; b.b_rs = nao; b.b_cs = 1; b.b_shared = 1;
      b.C = (float2*)c->chA; b.c_gs = slab; b.c_es = nao; b.c_rs = (int64_t)naux * nao;
      CK(run_bsm(c, b));
    } else {
      CK(run_gett(d, Vb, tv, gb, tg, c->chA, tv, acc, c));
    }
    // K[k][i][j] += -(1/Nk) sum_{(Q,b)} Y[k][i][(Q,b)] V^{k' k}[Q][b][j]
    GettDesc e = base_desc(nao, nao, (int64_t)naux * nao, nk);
    e.am = I1((int64_t)naux * nao); e.ak = I1(1); e.az = I1(slab);
    e.bk = I1(nao); e.bn = I1(1); e.bz = I1(slab);
    e.cm = I1(nao); e.cn = I1(1); e.cz = I1(n2);
    e.alpha = make_double2(-1.0 / nk, 0); e.beta = make_double2(1, 0);
    e.ksplit = 16;
    const char* Vk = (const char*)Vp + (size_t)kp * nk * slab * es;
    CK(run_gett(e, c->chA, tv, Vk, tv, out, Ty::C128, acc, c));
  }
  return GW_OK;
}

// Sigma_inf = J[gamma] + K[gamma] with gamma = -G(beta^-) from Gsrc (linear in G, so the
// same routine gives the tangent from a tangent of G).
static gw_status hf_core(gw_ctx* c, const double2* Gsrc, double2* gamma, double2* out) {
  const int nk = c->nk, nao = c->nao, naux = c->naux;
  CK(density_gamma(Gsrc, c->lb, gamma, c->ntau, (int64_t)nk * c->n2, c->st));
  CK(hartree_t(c->V, gamma, c->tQ, nk, naux, nao, c->st));
  CK(hartree_j(c->V, c->tQ, out, nk, naux, nao, c->spin / nk, c->st));   // Eq. HF_J
  count(3);
  return exchange(c, gamma, out);
}

extern "C" gw_status gw_hf(gw_ctx* c) {
  if (!c) return GW_ERR_ARG;
  if (!c->have_G) return fail(c, GW_ERR_STATE, "no Green's function yet");
  gw_status s = hf_core(c, c->G_tau, c->gamma, c->Sinf_new);
  if (s == GW_OK) { mark(c, GW_Q_GAMMA); mark(c, GW_Q_SIGMA_INF_NEW); }
  return s;
}

// ------------------------------------------------------------------ A2/A3: polarization

// The P~0 chain of Eq. tilde_P0_tau with its two G factors taken from separate
// tensors: Gplus supplies G^{k+q}(t), Gminus supplies G^k(-t) (= -Gminus^k(t_{ntau-1-j})).
// out (nq, ntau, naux, naux) receives the unsymmetrised sum, added to its contents
// when accumulate.  The forward map uses G_tau for both; its tangent runs the chain
// twice with the tangent in one slot.
static gw_status polar_chain_half(gw_ctx* c, const double2* Gplus, const double2* Gminus, double2* out,
                                  bool accumulate);
static gw_status sigma_chain_half(gw_ctx* c, const double2* Gsrc, const double2* Psrc, double2* out, bool accumulate);

static gw_status polar_chain(gw_ctx* c, const double2* Gplus, const double2* Gminus, double2* out, bool accumulate) {
  if (c->hfmt) return polar_chain_half(c, Gplus, Gminus, out, accumulate);
  const int nk = c->nk, nao = c->nao, naux = c->naux, ntau = c->ntau;
  const int64_t n2 = c->n2, na2 = c->na2, slab = (int64_t)naux * n2, gstep = (int64_t)nk * n2;
  const bool f32 = c->cfg.contract_prec != GW_FP64;
  const bool tc = c->cfg.contract_prec == GW_SPLIT_TF32;
  const Ty tv = f32 ? Ty::C64 : Ty::C128, acc = tv;
  const void* Vp = f32 ? (const void*)c->V32 : (const void*)c->V;
  const void* Gp = Gplus;
  const void* Gmp = Gminus;
  const size_t es = f32 ? 8 : 16;
  if (f32) {
    CK(to_c64(Gplus, c->G32, (int64_t)ntau * gstep, c->st)); count(1); Gp = c->G32; Gmp = c->G32;
    if (Gminus != Gplus) {
      if (!c->G32m) {
        c->G32m = (float2*)dalloc(c, (size_t)ntau * gstep * 8);
        if (!c->G32m) return fail(c, GW_ERR_OOM, "tangent buffer");
      }
      CK(to_c64(Gminus, c->G32m, (int64_t)ntau * gstep, c->st)); count(1); Gmp = c->G32m;
    }
  }
  if (!c->deferred) CK(cudaMemsetAsync(c->info + 1, 0, 4, c->st));
  const bool tca = tc && c->Vs_hi != nullptr;   // nao-sized steps on tensor cores
  if (tca) CK(build_gemb(c, Gplus, Gminus));
  // tensor cores: the last step of G k-points at a time as one GEMM; Z and the
  // embedded V of k-point j of a group sit at column block j of rows of length G kp
  const int G = tc ? c->pgroup : 1;
  const int64_t zld = tc ? G * c->kpadP : 0;
  for (int q = c->q0; q < c->q1; ++q) {
    if (c->reduce && c->kneg[(size_t)q] < q) continue;   // the conjugate of P~0^{-q}
    double2* Pq = out + (size_t)q * ntau * na2;
    for (int k = 0; k < nk; ++k) {
      const int kq = c->kplus[(size_t)q * nk + k];
      const int j = k % G;                      // column block of this k in its group
      float* Zh = tc ? c->Zhi + j * c->kpadP : nullptr;
      float* Zl = tc ? c->Zlo + j * c->kpadP : nullptr;
      const char* Vkq = (const char*)Vp + ((size_t)k * nk + kq) * slab * es;
      const char* Gm = (const char*)Gmp + ((size_t)(ntau - 1) * gstep + (size_t)k * n2) * es;
      if (tca) {
        // Y[t][Q][d][b] = sum_a V^{k,k+q}[Q][d][a] G^{k+q}[t][a][b] on tensor cores (G Hermitian), written
        // transposed per Q as TF32 hi/lo rows (t, Q, b) of (d, re/im): the A operand of the next step
        const int64_t ka = c->kpadA, per = 2 * (int64_t)nao * ka;
        CK(split_rows((const char*)c->V + ((size_t)k * nk + kq) * slab * 16, true, (int64_t)naux * nao, nao, nao, false,
                      c->Vs_hi, c->Vs_lo, ka, c->st));
        count(1);
        UmmaOperand oa{c->Vs_hi, c->Vs_lo, (int64_t)naux * nao, 1, ka, 0};
        UmmaOperand ob{c->Ge_hi + (size_t)kq * ntau * per, c->Ge_lo + (size_t)kq * ntau * per, 2 * (int64_t)nao, ntau, ka,
                       per};
        CK(run_umma(c, 8.0 * ntau * naux * (double)nao * n2, oa, ob, naux * nao, 2 * nao, ka, ntau, c->Xs_hi, false, 1.0,
                    false, 2, (int64_t)naux * nao * ka, 1, nao, (int64_t)nao * ka, 2, ka, c->Xs_lo, 2 * (int64_t)nao));
        // Z[t][Q][c][b] = -sum_d G^k(t_{ntau-1-j})[c][d] Y[t][Q][d][b] as rows (t, Q, b) of (c, re/im),
        // written into the (c, b) layout of the last step's A operand
        UmmaOperand ya{c->Xs_hi, c->Xs_lo, (int64_t)naux * nao, ntau, ka, (int64_t)naux * nao * ka};
        UmmaOperand gb{c->Gp_hi + (size_t)k * ntau * per, c->Gp_lo + (size_t)k * ntau * per, 2 * (int64_t)nao, ntau, ka,
                       per};
        CK(run_umma(c, 8.0 * ntau * naux * (double)nao * n2, ya, gb, naux * nao, 2 * nao, ka, ntau, Zh, false, -1.0,
                    false, 2, (int64_t)naux * zld, 1, nao, zld, 2, 2 * (int64_t)nao, Zl, 2 * (int64_t)nao));
      } else if (f32 && nao <= 64) {
        // Y[t][Q][d][b] = sum_a V^{k,k+q}[Q][d][a] G^{k+q}[t][a][b]   (G shared per t)
        BsmDesc b1{};
        b1.M = b1.N = b1.K = nao; b1.G = ntau; b1.E = naux; b1.alpha = 1.f;
        b1.A = (const float2*)Vkq; b1.a_gs = 0; b1.a_es = n2; b1.a_rs = nao; b1.a_cs = 1;
        b1.B = (const float2*)Gp + (size_t)kq * n2; b1.b_gs = gstep; b1.b_rs = nao; b1.b_cs = 1; b1.b_shared = 1;
        b1.C = (float2*)c->chA; b1.c_gs = slab; b1.c_es = n2; b1.c_rs = nao;
        CK(run_bsm(c, b1));
        // Z[t][Q][c][b] = -sum_d G^k(t_{ntau-1-j})[c][d] Y[t][Q][d][b]   (G^k(-t) shared per t)
        BsmDesc b2{};
        b2.M = b2.N = b2.K = nao; b2.G = ntau; b2.E = naux; b2.alpha = -1.f;
        b2.A = (const float2*)Gm; b2.a_gs = -gstep; b2.a_rs = nao; b2.a_cs = 1; b2.a_shared = 1;
        b2.B = (const float2*)c->chA; b2.b_gs = slab; b2.b_es = n2; b2.b_rs = nao; b2.b_cs = 1;
        if (tc) {   // straight into the TF32 hi/lo operand of the tensor-core GEMM
          const int64_t hk = zld / 2;
          b2.Chi = Zh; b2.Clo = Zl; b2.c_gs = (int64_t)naux * hk; b2.c_es = hk; b2.c_rs = nao;
        } else {
          b2.C = (float2*)c->chB; b2.c_gs = slab; b2.c_es = n2; b2.c_rs = nao;
        }
        CK(run_bsm(c, b2));
      } else {
      // Y[t][(Q,d)][b] = sum_a V^{k,k+q}[Q][d][a] G^{k+q}[t][a][b]
      GettDesc d1 = base_desc((int64_t)naux * nao, nao, nao, ntau);
      d1.am = I1(nao); d1.ak = I1(1); d1.az = I1(0);
      d1.bk = I1(nao); d1.bn = I1(1); d1.bz = I1(gstep);
      d1.cm = I1(nao); d1.cn = I1(1); d1.cz = I1(slab);
      CK(run_gett(d1, Vkq, tv, (const char*)Gp + (size_t)kq * n2 * es, tv, c->chA, tv, acc, c));
      // Z[t][Q][c][b] = sum_d G^k_cd(-t) Y[t][Q][d][b],  G(-t_j) = -G(t_{ntau-1-j})
      GettDesc d2 = base_desc(nao, (int64_t)naux * nao, nao, ntau);
      d2.am = I1(nao); d2.ak = I1(1); d2.az = I1(-gstep);
      d2.bk = I1(nao); d2.bn = I2(nao, n2, 1); d2.bz = I1(slab);
      d2.cm = I1(nao); d2.cn = I2(nao, n2, 1); d2.cz = I1(slab);
      d2.alpha = make_double2(-1, 0);
      CK(run_gett(d2, Gm, tv, c->chA, tv, c->chB, tv, acc, c));
      }
      // P[t][Q][Q'] += (s/Nk) sum_{(c,b)} Z[t][Q][(c,b)] V^{k+q,k}_{bc}(Q'),
      // with V^{k+q,k}_{bc}(Q') = conj V^{k,k+q}_{cb}(Q') (pairing checked at init)
      if (tc) {
        // tensor cores: split-TF32 real GEMM on the embedded operands, once per group
        // of G k-points (K = their column blocks side by side)
        const int64_t kp = c->kpadP;
        if (nao > 64) {
          CK(split_rows(c->chB, false, (int64_t)ntau * naux, n2, n2, false, Zh, Zl, kp, c->st, zld));
          count(1);
        }
        CK(embed_conj((const char*)c->V + ((size_t)k * nk + kq) * slab * 16, true, naux, n2, c->Vhi + j * kp,
                      c->Vlo + j * kp, kp, c->st, zld));
        count(1);
        if (j == G - 1 || k == nk - 1) {
          const int g = j + 1, k0 = k - j;
          UmmaOperand oa{c->Zhi, c->Zlo, (int64_t)ntau * naux, 1, zld, 0};
          UmmaOperand ob{c->Vhi, c->Vlo, 2 * (int64_t)naux, 1, zld, 0};
          CK(run_umma(c, 8.0 * g * ntau * naux * (double)naux * n2, oa, ob, ntau * naux, 2 * naux, g * kp, 1, Pq,
                      true, c->spin / nk, accumulate || k0 > 0, 2 * (int64_t)naux, 0, 1, 0, 0, 0, 0, nullptr,
                      (g - 1) * kp + 2 * n2));
        }
        continue;
      }
      GettDesc d3 = base_desc((int64_t)ntau * naux, naux, n2, 1);
      d3.am = I1(n2); d3.ak = I1(1);
      d3.bk = I1(1); d3.bn = I1(n2); d3.conjB = true;
      d3.cm = I1(naux); d3.cn = I1(1);
      d3.alpha = make_double2(c->spin / nk, 0);
      d3.beta = make_double2(accumulate || k > 0 ? 1.0 : 0.0, 0);
      CK(run_gett(d3, c->chB, tv, Vkq, tv, Pq, Ty::C128, acc, c));
    }
  }
  return GW_OK;
}

// ------------------------------------------------------------------ chains with 16-bit pieces

// The P~0 chain of Eq. tilde_P0_tau with every GEMM on the tensor cores in 16-bit pieces
// (same steps and layouts as the split-TF32 chain above):
//   Y[t][Q][d][b] = sum_a V^{k,k+q}_da(Q) G^{k+q}_ab(t)              (rows (Q, d), batch t)
//   Z[t][Q][c][b] = -sum_d G^k_cd(t_{ntau-1-j}) Y[t][Q][d][b]         (rows (Q, b), batch t)
//   P[t][Q][Q'] += (s/Nk) sum_(c,b) Z[t][Q][(c,b)] conj V^{k,k+q}_cb(Q')   (group of k-points)
// Y and Z are written by the GEMM epilogues directly as the next GEMM's 16-bit operand,
// scaled by 2^-e with e from the bounds |Y| <= vrs(Q) max|G(t)| and |Z| <= rowsum|G(-t)| |Y|.
static gw_status polar_chain_half(gw_ctx* c, const double2* Gplus, const double2* Gminus, double2* out,
                                  bool accumulate) {
  const int nk = c->nk, nao = c->nao, naux = c->naux, ntau = c->ntau, fmt = c->hfmt;
  const int64_t n2 = c->n2, slab = (int64_t)naux * n2, gstep = (int64_t)nk * n2;
  const int64_t ka = c->kpadA, per = 2 * (int64_t)nao * ka, kp = c->kpadP;
  const int G = c->pgroup;
  const int64_t zld = G * kp;
  const int64_t kAll = (int64_t)1 << 40;   // exponent index divisor: one exponent per batch entry
  cudaStream_t st = c->st;
  if (!c->deferred) CK(cudaMemsetAsync(c->info + 1, 0, 4, st));
  // norms of the two G factors, then the row exponents of Y and Z per (t, Q)
  CK(g_norms(Gplus, ntau, nk, c->nao, c->gn, c->gn + ntau, st));
  const float* grs_m = c->gn + ntau;
  if (Gminus != Gplus) {
    CK(g_norms(Gminus, ntau, nk, nao, c->gn + 2 * ntau, c->gn + 3 * ntau, st));
    grs_m = c->gn + 3 * ntau;
    count(1);
  }
  CK(polar_exps(c->vQrs, c->gn, grs_m, ntau, naux, c->eY, c->eZ, st));
  count(2);
  // G operands per k: Ge[k][t] from G^k(t) (C = A conj(Ge)^T = A G for Hermitian G),
  // Gp[k][j] from G^k(t_{ntau-1-j}) (C = A Gp^T), one exponent per matrix
  for (int k = 0; k < nk; ++k) {
    CK(half_embed_mats(Gplus + (size_t)k * n2, ntau, gstep, nao, nao, hofs(c->Ge_hi, (int64_t)k * ntau * per),
                       hofs(c->Ge_lo, (int64_t)k * ntau * per), ka, per, fmt, false, c->eGe + (size_t)k * ntau, st));
    CK(half_embed_mats(Gminus + (size_t)(ntau - 1) * gstep + (size_t)k * n2, ntau, -gstep, nao, nao,
                       hofs(c->Gp_hi, (int64_t)k * ntau * per), hofs(c->Gp_lo, (int64_t)k * ntau * per), ka, per, fmt,
                       true, c->eGp + (size_t)k * ntau, st));
  }
  count(2 * nk);
  const double fl12 = 8.0 * ntau * naux * (double)nao * n2;
  // k-points per launch: several (k, k+q) pairs of small systems share each GEMM
  // (batch entry z = (k, t)), whole groups of the last step at most
  const int KB = c->pbatch < G ? c->pbatch : G;
  const int64_t vs_blk = (int64_t)naux * nao * ka, xs_blk = (int64_t)ntau * naux * nao * ka;
  for (int q = c->q0; q < c->q1; ++q) {
    if (c->reduce && c->kneg[(size_t)q] < q) continue;   // the conjugate of P~0^{-q}
    double2* Pq = out + (size_t)q * ntau * c->na2;
    for (int g0 = 0; g0 < nk; g0 += G) {
      const int gn = nk - g0 < G ? nk - g0 : G;
      for (int b0 = 0; b0 < gn; b0 += KB) {
        const int kn = gn - b0 < KB ? gn - b0 : KB, k0 = g0 + b0;
        int64_t voff[kSrcListMax];
        int kq[kSrcListMax];
        for (int l = 0; l < kn; ++l) {
          kq[l] = c->kplus[(size_t)q * nk + k0 + l];
          voff[l] = ((int64_t)(k0 + l) * nk + kq[l]) * slab;
        }
        // Y: A = V^{k,k+q} rows (Q, d) with exact row exponents, B = Ge[k+q][t]
        CK(half_rows_multi(c->V, voff, kn, (int64_t)naux * nao, nao, nao, false, c->Vs_hi, c->Vs_lo, ka, ka, vs_blk,
                           fmt, c->eV1, nullptr, (int64_t)naux * nao, st));
        count(1);
        const void *gbh = hofs(c->Ge_hi, (int64_t)kq[0] * ntau * per), *gbl = hofs(c->Ge_lo, (int64_t)kq[0] * ntau * per);
        const int* gbe = c->eGe + (size_t)kq[0] * ntau;
        if (kn > 1) {   // the blocks of G^{k+q} in k order
          CK(gather_blocks(c->Ge_hi, c->Ge_lo, c->eGe, c->Gq_hi, c->Gq_lo, c->eGq, (int64_t)ntau * per * 2, ntau, kq, kn,
                           st));
          count(1);
          gbh = c->Gq_hi; gbl = c->Gq_lo; gbe = c->eGq;
        }
        {
          UmmaOperand oa{c->Vs_hi, c->Vs_lo, (int64_t)naux * nao, kn, ka, vs_blk, fmt};
          UmmaOperand ob{(const float*)gbh, (const float*)gbl, 2 * (int64_t)nao, (int64_t)kn * ntau, ka, per, fmt};
          UmmaScale sc{c->eV1, gbe, 0, 1, 0, 1, kAll};
          UmmaOut o{fmt, c->eY, naux, nao, 0};
          // z = (k, t): A and the row exponents per k, B and its exponents per (k, t), Y blocks per (k, t)
          UmmaZ zz{ntau, 1, 0, ntau, 1, (int64_t)naux * nao, ntau, 0, xs_blk};
          CK(run_umma(c, fl12 * kn, oa, ob, naux * nao, 2 * nao, ka, kn * ntau, c->Xs_hi, false, 1.0, false, 2,
                      (int64_t)naux * nao * ka, 1, nao, (int64_t)nao * ka, 2, ka, c->Xs_lo, 2 * (int64_t)nao, &sc, &o,
                      kn > 1 ? &zz : nullptr));
        }
        // Z: A = Y^T rows (Q, b) per (k, t) (exponent per (t, Q)), B = Gp[k][t]; written into
        // the (c, b) columns of blocks b0.. of the grouped last step's A operand
        {
          UmmaOperand ya{c->Xs_hi, c->Xs_lo, (int64_t)naux * nao, (int64_t)kn * ntau, ka, (int64_t)naux * nao * ka, fmt};
          UmmaOperand gb{hofs(c->Gp_hi, (int64_t)k0 * ntau * per), hofs(c->Gp_lo, (int64_t)k0 * ntau * per),
                         2 * (int64_t)nao, (int64_t)kn * ntau, ka, per, fmt};
          UmmaScale sc{c->eY, c->eGp + (size_t)k0 * ntau, naux, 1, 0, nao, kAll};
          UmmaOut o{fmt, c->eZ, naux, nao, 0};
          UmmaZ zz{ntau, ntau, 1, ntau, 1, 0, ntau, 0, kp};
          CK(run_umma(c, fl12 * kn, ya, gb, naux * nao, 2 * nao, ka, kn * ntau, hofs(c->Zhi, b0 * kp), false, -1.0, false,
                      2, (int64_t)naux * zld, 1, nao, zld, 2, 2 * (int64_t)nao, hofs(c->Zlo, b0 * kp),
                      2 * (int64_t)nao, &sc, &o, kn > 1 ? &zz : nullptr));
        }
        // embedded conj V^{k,k+q}(Q') rows with the per-Q exponents shared by the group
        CK(half_embed_conj_multi(c->V, voff, kn, naux, n2, hofs(c->Vhi, b0 * kp), hofs(c->Vlo, b0 * kp), kp, zld, kp,
                                 fmt, c->eVQ, st));
        count(1);
      }
      const int g = gn;
      UmmaOperand oa{c->Zhi, c->Zlo, (int64_t)ntau * naux, 1, zld, 0, fmt};
      UmmaOperand ob{c->Vhi, c->Vlo, 2 * (int64_t)naux, 1, zld, 0, fmt};
      UmmaScale sc{c->eZ, c->eVQ, 0, 0, 0, 1, 1};
      CK(run_umma(c, 8.0 * g * ntau * naux * (double)naux * n2, oa, ob, ntau * naux, 2 * naux, g * kp, 1, Pq, true,
                  c->spin / nk, accumulate || g0 > 0, 2 * (int64_t)naux, 0, 1, 0, 0, 0, 0, nullptr,
                  (g - 1) * kp + 2 * n2, &sc, nullptr));
    }
  }
  return GW_OK;
}

// The Sigma~ chain of Eq. tilde_sigma2 with 16-bit pieces:
//   X[t][Q'][(i,a)] = sum_Q conj P~^q_Q'Q(t) V^{k,k-q}_ia(Q)         (rows (t, Q'))
//   Y[t][i][(b,Q')] = sum_a X[t][Q'][i][a] G^{k-q}_ab(t)             (rows (i, Q'), batch t)
//   Sigma~[t][k][i][j] += -(1/Nk) sum_(b,Q') Y[t][i][(b,Q')] V^{k-q,k}_bj(Q')
// X is written as rows (t, i, Q') and the last step's K runs over (b, Q'), so that the
// middle step's consecutive rows Q' are adjacent complex entries of its output (the
// coalesced lane-per-row write-out).
// X's rows are scaled from P~'s row sums of moduli times max |V|; Y's from max_Q' of X's
// bounds times the row sums of G(t).
static gw_status sigma_chain_half(gw_ctx* c, const double2* Gsrc, const double2* Psrc, double2* out, bool accumulate) {
  const int nk = c->nk, nao = c->nao, naux = c->naux, ntau = c->ntau, fmt = c->hfmt;
  const int64_t n2 = c->n2, na2 = c->na2, slab = (int64_t)naux * n2, gstep = (int64_t)nk * n2;
  const int64_t ka = c->kpadA, per = 2 * (int64_t)nao * ka, kps = c->kpadS, kp3 = c->kpad3;
  const int64_t kAll = (int64_t)1 << 40;
  const int shift = c->h_Evmax + 1;   // X rows: 2^(ePs + shift) bounds |X|
  cudaStream_t st = c->st;
  if (!c->deferred) CK(cudaMemsetAsync(c->info + 1, 0, 4, st));
  if (!accumulate) CK(cudaMemsetAsync(out, 0, (size_t)ntau * gstep * 16, st));
  CK(g_norms(Gsrc, ntau, nk, nao, c->gn, c->gn + ntau, st));
  count(1);
  for (int k = 0; k < nk; ++k)
    CK(half_embed_mats(Gsrc + (size_t)k * n2, ntau, gstep, nao, nao, hofs(c->Ge_hi, (int64_t)k * ntau * per),
                       hofs(c->Ge_lo, (int64_t)k * ntau * per), ka, per, fmt, false, c->eGe + (size_t)k * ntau, st));
  count(nk);
  const double fl1 = 8.0 * ntau * naux * (double)naux * n2, fl2 = 8.0 * ntau * naux * (double)nao * n2;
  const int64_t mt = ((int64_t)ntau * nao + 127) / 128, nt = (2 * (int64_t)nao + 159) / 160;
  const int KB = c->pbatch;
  const int64_t xs_blk = (int64_t)ntau * naux * nao * ka, y3_blk = (int64_t)ntau * nao * kp3;
  const int64_t vt_blk = 2 * n2 * kps, w3_blk = 2 * (int64_t)nao * kp3;
  std::vector<int> act;
  act.reserve((size_t)nk);
  for (int q = c->q0; q < c->q1; ++q) {
    // A operand of the first step: conj P~^q(t) rows (t, Q') with exact row exponents and
    // the exponents of their sums of moduli; then Y's exponent per t
    CK(half_rows(Psrc + (size_t)q * ntau * na2, (int64_t)ntau * naux, naux, naux, true, c->Pchi, c->Pclo, kps, kps, fmt,
                 c->ePc, c->ePs, st));
    CK(sigma_exps(c->ePs, shift, c->gn + ntau, ntau, naux, c->eY3, st));
    count(2);
    act.clear();
    for (int k = 0; k < nk; ++k)
      if (!(c->reduce && c->kneg[(size_t)k] < k)) act.push_back(k);   // else the conjugate of Sigma~^{-k}
    for (size_t b0 = 0; b0 < act.size();) {
      // a run of consecutive k (their Sigma~^k blocks are equally spaced), KB at most
      int kn = 1;
      while (kn < KB && b0 + kn < act.size() && act[b0 + kn] == act[b0] + kn) ++kn;
      const int k0 = act[b0];
      b0 += kn;
      int64_t voffX[kSrcListMax], voffW[kSrcListMax];
      int kmq[kSrcListMax];
      for (int l = 0; l < kn; ++l) {
        kmq[l] = c->kminus[(size_t)q * nk + k0 + l];
        voffX[l] = ((int64_t)(k0 + l) * nk + kmq[l]) * slab;
        voffW[l] = ((int64_t)kmq[l] * nk + k0 + l) * slab;
      }
      // X = conj(P~) V: B = V^{k,k-q} transposed, rows (i, a), K = Q, one exponent
      CK(half_embed_t_multi(c->V, voffX, kn, naux, n2, c->VThi, c->VTlo, kps, vt_blk, fmt, c->h_Evmax - 15, st));
      count(1);
      {
        UmmaOperand oa{c->Pchi, c->Pclo, (int64_t)ntau * naux, 1, kps, 0, fmt};
        UmmaOperand ob{c->VThi, c->VTlo, 2 * n2, kn, kps, vt_blk, fmt};
        UmmaScale sc{c->ePc, c->eVall, 0, 0, 0, 1, kAll};
        UmmaOut o{fmt, c->ePs, 0, 1, shift};
        // output row (t, Q'), column (i, a re/im) -> X row (t, i, Q'), entry (a re/im); one X block per k
        CK(run_umma(c, fl1 * kn, oa, ob, ntau * naux, (int)(2 * n2), kps, kn, c->Xs_hi, false, 1.0, false, ka,
                    kn > 1 ? xs_blk : 0, 1, naux, (int64_t)nao * naux * ka, 2 * (int64_t)nao, (int64_t)naux * ka,
                    c->Xs_lo, 2 * (int64_t)naux, &sc, &o));
      }
      // Y = X G^{k-q}(t): A rows (i, Q') per (k, t) (exponent of row Q'), B = Ge[k-q][t]; row (i, Q'),
      // column (b re/im) lands at row (t, i), K entry (b, Q') of the last step's operand
      {
        const void *gbh = hofs(c->Ge_hi, (int64_t)kmq[0] * ntau * per), *gbl = hofs(c->Ge_lo, (int64_t)kmq[0] * ntau * per);
        const int* gbe = c->eGe + (size_t)kmq[0] * ntau;
        if (kn > 1) {
          CK(gather_blocks(c->Ge_hi, c->Ge_lo, c->eGe, c->Gq_hi, c->Gq_lo, c->eGq, (int64_t)ntau * per * 2, ntau, kmq,
                           kn, st));
          count(1);
          gbh = c->Gq_hi; gbl = c->Gq_lo; gbe = c->eGq;
        }
        UmmaOperand xa{c->Xs_hi, c->Xs_lo, (int64_t)naux * nao, (int64_t)kn * ntau, ka, (int64_t)naux * nao * ka, fmt};
        UmmaOperand gb{(const float*)gbh, (const float*)gbl, 2 * (int64_t)nao, (int64_t)kn * ntau, ka, per, fmt};
        UmmaScale sc{c->ePs, gbe, naux, 1, shift, 1, kAll};
        sc.ea_mod = naux;
        UmmaOut o{fmt, c->eY3, 1, kAll, 0};
        UmmaZ zz{ntau, ntau, 1, ntau, 1, 0, ntau, 0, y3_blk};
        CK(run_umma(c, fl2 * kn, xa, gb, naux * nao, 2 * nao, ka, kn * ntau, c->Y3hi, false, 1.0, false, 2,
                    (int64_t)nao * kp3, 1, naux, kp3, 2, 2 * (int64_t)naux, c->Y3lo, 2 * (int64_t)nao, &sc, &o,
                    kn > 1 ? &zz : nullptr));
      }
      // Sigma~ += -(1/Nk) Y V^{k-q,k}: B = V^{k-q,k} transposed, rows j, K = (b, Q') (source rows (Q', b))
      CK(half_embed_t_multi(c->V, voffW, kn, (int64_t)naux * nao, nao, c->W3hi, c->W3lo, kp3, w3_blk, fmt,
                            c->h_Evmax - 15, st, nao, naux));
      count(1);
      {
        int64_t ks = (304 + mt * nt * kn - 1) / (mt * nt * kn);
        if (ks > kp3 / 64) ks = kp3 / 64;
        if (ks < 1) ks = 1;
        UmmaOperand ya{c->Y3hi, c->Y3lo, (int64_t)ntau * nao, kn, kp3, y3_blk, fmt};
        UmmaOperand wb{c->W3hi, c->W3lo, 2 * (int64_t)nao, kn, kp3, w3_blk, fmt};
        UmmaScale sc{c->eY3, c->eVall, 0, 0, 0, nao, kAll};
        CK(run_umma(c, fl2 * kn, ya, wb, ntau * nao, 2 * nao, kp3, kn, (double*)(out + (size_t)k0 * n2), true,
                    -1.0 / nk, true, 2 * (int64_t)nao, 2 * n2, (int)ks, nao, 2 * gstep, 0, 0, nullptr,
                    2 * (int64_t)naux * nao, &sc, nullptr));
      }
    }
  }
  return GW_OK;
}

extern "C" gw_status gw_polarization(gw_ctx* c) {
  if (!c) return GW_ERR_ARG;
  if (!c->have_G) return fail(c, GW_ERR_STATE, "no Green's function yet");
  const int nk = c->nk, naux = c->naux, ntau = c->ntau;
  const int64_t na2 = c->na2;
  const bool tc = uses_tc(c);
  const bool red = trs_reduce(c);
  c->reduce = red;
  gw_status s = polar_chain(c, c->G_tau, c->G_tau, c->P0_tau, false);
  c->reduce = false;
  if (s != GW_OK) return s;
  if (red) {   // P~0^{-q}(tau) = conj P~0^q(tau) (time-reversal symmetry)
    CK(conj_fill(c->P0_tau, 1, nk, (int64_t)ntau * na2, c->d_kneg, c->d_kneed, c->st));
    count(1);
  }
  if (tc && !c->deferred) {
    int h = 0;
    CK(cudaMemcpyAsync(c->h_scr, c->info + 1, 4, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    memcpy(&h, c->h_scr, 4);
    if (h) return fail(c, GW_ERR_TIMEOUT, "tensor-core contraction gave up waiting (code " + std::to_string(h) + ")");
  }
  const int nq = c->q1 - c->q0;
  double2* P0q = c->P0_tau + (size_t)c->q0 * ntau * na2;
  CK(herm_batched(P0q, naux, (int64_t)nq * ntau, na2, c->st));
  count(1);
  // P~0(i Omega_m) = sum_j TFb[m][j] P~0(tau_j)   (Eq. P0t_to_P0w)
  CK(transform(c, c->TFb, P0q, c->P_iw + (size_t)c->q0 * c->nwb * na2, c->nwb, na2, nq, (int64_t)ntau * na2,
               (int64_t)c->nwb * na2));
  c->have_P0 = true;
  c->have_P = false;
  mark(c, GW_Q_P0_TAU); mark(c, GW_Q_P0_IW); unmark(c, GW_Q_P_IW);
  return GW_OK;
}

// ------------------------------------------------------------------ A4/A5: screened solve

// Screened solve and backward transform of the q-points [qa, qb)
static gw_status screened_block(gw_ctx* c, int qa, int qb) {
  const int naux = c->naux, ntau = c->ntau, nq = qb - qa;
  const int64_t na2 = c->na2;
  double2* Pw = c->P_iw + (size_t)qa * c->nwb * na2;
  double2* Pt = c->P_tau + (size_t)qa * ntau * na2;
  if (c->irws) {
    // complex64 inversion refined to FP64 accuracy (P~0 Y on the tensor cores)
    int64_t nl = 0;
    CK(screened_refine(Pw, naux, (int64_t)nq * c->nwb, c->irws, c->irws_bytes, kRefineSteps, c->info + 2,
                       c->info + 1, c->st, &nl));
    count((int)nl);
  } else {
    CK(screened_inplace(Pw, naux, (int64_t)nq * c->nwb, (double2*)c->ws, c->ws_bytes, c->info + 2, c->st));
    int64_t nbk = (naux + 63) / 64;
    count((int)(2 + nbk * 7));
  }
  // P~(tau_j) = sum_m TBb[j][m] P~(i Omega_m)   (Eq. Piw_to_Pt), symmetrised
  CK(transform(c, c->TBb, Pw, Pt, ntau, na2, nq, (int64_t)c->nwb * na2, (int64_t)ntau * na2));
  CK(herm_batched(Pt, naux, (int64_t)nq * ntau, na2, c->st));
  count(1);
  return GW_OK;
}

extern "C" gw_status gw_screened(gw_ctx* c) {
  if (!c) return GW_ERR_ARG;
  if (!c->have_P0) return fail(c, GW_ERR_STATE, "no polarization yet");
  if (!c->deferred) {
    CK(cudaMemsetAsync(c->info + 1, 0, 8, c->st));
  }
  gw_status s = GW_OK;
  if (trs_reduce(c)) {
    // time-reversal symmetry: solve the runs of irreducible q, then P~^{-q} = conj P~^q
    for (int qa = 0; qa < c->nk && s == GW_OK;) {
      if (c->kneg[(size_t)qa] < qa) { ++qa; continue; }
      int qb = qa + 1;
      while (qb < c->nk && c->kneg[(size_t)qb] >= qb) ++qb;
      s = screened_block(c, qa, qb);
      qa = qb;
    }
    if (s != GW_OK) return s;
    CK(conj_fill(c->P_iw, 1, c->nk, (int64_t)c->nwb * c->na2, c->d_kneg, c->d_kneed, c->st));
    CK(conj_fill(c->P_tau, 1, c->nk, (int64_t)c->ntau * c->na2, c->d_kneg, c->d_kneed, c->st));
    count(2);
  } else {
    s = screened_block(c, c->q0, c->q1);
    if (s != GW_OK) return s;
  }
  c->have_P0 = false;   // P~0(i Omega) was overwritten
  if (!c->deferred) {
    int h[2] = {0, 0};
    CK(cudaMemcpyAsync(c->h_scr, c->info + 1, 8, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    memcpy(h, c->h_scr, 8);
    if (h[0]) return fail(c, GW_ERR_TIMEOUT, "tensor-core product gave up waiting (code " + std::to_string(h[0]) + ")");
    if (h[1]) return fail(c, GW_ERR_SINGULAR, "zero pivot in the screened solve");
  }
  c->have_P = true;
  mark(c, GW_Q_P_IW); mark(c, GW_Q_P_TAU); unmark(c, GW_Q_P0_IW);
  return GW_OK;
}

// ------------------------------------------------------------------ A6: self-energy

// The Sigma~ chain of Eq. tilde_sigma2 with G^{k-q}(t) from Gsrc and P~^q(t) from
// Psrc; out (ntau, nk, nao, nao) receives the unsymmetrised sum (added to its
// contents when accumulate).  The forward map uses G_tau and P_tau; the tangent runs
// it with the tangent in either slot.
static gw_status sigma_chain(gw_ctx* c, const double2* Gsrc, const double2* Psrc, double2* out, bool accumulate) {
  if (c->hfmt) return sigma_chain_half(c, Gsrc, Psrc, out, accumulate);
  const int nk = c->nk, nao = c->nao, naux = c->naux, ntau = c->ntau;
  const int64_t n2 = c->n2, na2 = c->na2, slab = (int64_t)naux * n2, gstep = (int64_t)nk * n2;
  const bool f32 = c->cfg.contract_prec != GW_FP64;
  const bool tc = c->cfg.contract_prec == GW_SPLIT_TF32;
  const Ty tv = f32 ? Ty::C64 : Ty::C128, acc = tv;
  const void* Vp = f32 ? (const void*)c->V32 : (const void*)c->V;
  const void* Gp = Gsrc;
  const void* Pp = Psrc;
  if (!c->deferred) CK(cudaMemsetAsync(c->info + 1, 0, 4, c->st));
  const bool tc3 = tc && c->Y3hi != nullptr;   // last step on tensor cores (atomic fp64 accumulation)
  if (tc3 && !accumulate) CK(cudaMemsetAsync(out, 0, (size_t)ntau * gstep * 16, c->st));
  const bool tc2 = tc3 && c->Xs_hi != nullptr;   // middle step on tensor cores too
  if (tc2) CK(build_gemb(c, Gsrc, nullptr));
  const size_t es = f32 ? 8 : 16;
  if (f32) {
    CK(to_c64(Gsrc, c->G32, (int64_t)ntau * gstep, c->st));
    CK(to_c64(Psrc, c->P32, (int64_t)nk * ntau * na2, c->st));
    count(2);
    Gp = c->G32; Pp = c->P32;
  }
  for (int q = c->q0; q < c->q1; ++q) {
    const char* Pq = (const char*)Pp + (size_t)q * ntau * na2 * es;
    if (tc) {
      // A operand of the tensor-core stage: conj P~^q(t) = P~^q(t)^T (Hermitian), split hi/lo
      CK(split_rows(Psrc + (size_t)q * ntau * na2, true, (int64_t)ntau * naux, naux, naux, true, c->Pchi,
                    c->Pclo, c->kpadS, c->st));
      count(1);
    }
    for (int k = 0; k < nk; ++k) {
      if (c->reduce && c->kneg[(size_t)k] < k) continue;   // the conjugate of Sigma~^{-k}
      const int kmq = c->kminus[(size_t)q * nk + k];
      if (tc) {
        // X[t][Q'][(i,a)] = sum_Q conj(P~[t][Q'][Q]) V^{k,k-q}[Q][(i,a)] on tensor cores
        const int64_t kp = c->kpadS;
        CK(embed_t((const char*)c->V + ((size_t)k * nk + kmq) * slab * 16, true, naux, n2, c->VThi, c->VTlo, kp,
                   c->st));
        // V is shared by all t: the rows (t, Q') of every t form one M = ntau naux
        UmmaOperand oa{c->Pchi, c->Pclo, (int64_t)ntau * naux, 1, kp, 0};
        UmmaOperand ob{c->VThi, c->VTlo, 2 * n2, 1, kp, 0};
        if (tc2) {
          // X written as TF32 hi/lo rows (t, Q', i) of length kpadA: the A operand of the next step
          const int64_t ka = c->kpadA;
          CK(run_umma(c, 8.0 * ntau * naux * (double)naux * n2, oa, ob, ntau * naux, (int)(2 * n2), kp, 1, c->Xs_hi,
                      false, 1.0, false, (int64_t)nao * ka, 0, 1, 0, 0, 2 * (int64_t)nao, ka, c->Xs_lo,
                      2 * (int64_t)naux));
        } else {
          CK(run_umma(c, 8.0 * ntau * naux * (double)naux * n2, oa, ob, ntau * naux, (int)(2 * n2), kp, 1, c->chA,
                      false, 1.0, false, 2 * n2, 0, 1, 0, 0, 0, 0, nullptr, 2 * (int64_t)naux));
        }
        count(1);
      } else {
      // X[t][Q'][(i,a)] = sum_Q P~^q[t][Q][Q'] V^{k,k-q}[Q][(i,a)]
      GettDesc d1 = base_desc(naux, n2, naux, ntau);
      d1.am = I1(1); d1.ak = I1(naux); d1.az = I1(na2);
      d1.bk = I1(n2); d1.bn = I1(1); d1.bz = I1(0);
      d1.cm = I1(n2); d1.cn = I1(1); d1.cz = I1(slab);
      const char* Vkk = (const char*)Vp + ((size_t)k * nk + kmq) * slab * es;
      CK(run_gett(d1, Pq, tv, Vkk, tv, c->chA, tv, acc, c));
      }
      // Y[t][i][Q'][b] = sum_a X[t][Q'][i][a] G^{k-q}[t][a][b]
      if (tc2) {
        // on tensor cores: rows (Q', i) per t, written as hi/lo rows (t, i) at column block Q'
        const int64_t ka = c->kpadA, per = 2 * (int64_t)nao * ka;
        UmmaOperand oa{c->Xs_hi, c->Xs_lo, (int64_t)naux * nao, ntau, ka, (int64_t)naux * nao * ka};
        UmmaOperand ob{c->Ge_hi + (size_t)kmq * ntau * per, c->Ge_lo + (size_t)kmq * ntau * per, 2 * (int64_t)nao, ntau,
                       ka, per};
        CK(run_umma(c, 8.0 * ntau * naux * (double)nao * n2, oa, ob, naux * nao, 2 * nao, ka, ntau, c->Y3hi, false, 1.0,
                    false, c->kpad3, (int64_t)nao * c->kpad3, 1, nao, 2 * (int64_t)nao, 0, 0, c->Y3lo,
                    2 * (int64_t)nao));
        count(1);
      } else if (f32 && nao <= 64) {
        BsmDesc b{};
        b.M = b.N = b.K = nao; b.G = ntau; b.E = naux; b.alpha = 1.f;
        b.A = (const float2*)c->chA; b.a_gs = slab; b.a_es = n2; b.a_rs = nao; b.a_cs = 1;
        b.B = (const float2*)Gp + (size_t)kmq * n2; b.b_gs = gstep; b.b_rs = nao; b.b_cs = 1; b.b_shared = 1;
        if (tc3) {  // TF32 hi/lo rows (t, i), columns (Q', b): the A operand of the last step
          const int64_t hk = c->kpad3 / 2;
          b.Chi = c->Y3hi; b.Clo = c->Y3lo; b.c_gs = nao * hk; b.c_es = nao; b.c_rs = hk;
        } else {
          b.C = (float2*)c->chB; b.c_gs = slab; b.c_es = nao; b.c_rs = (int64_t)naux * nao;
        }
        CK(run_bsm(c, b));
      } else {
      GettDesc d2 = base_desc((int64_t)naux * nao, nao, nao, ntau);
      d2.am = I1(nao); d2.ak = I1(1); d2.az = I1(slab);
      d2.bk = I1(nao); d2.bn = I1(1); d2.bz = I1(gstep);
      d2.cm = I2(nao, nao, (int64_t)naux * nao); d2.cn = I1(1); d2.cz = I1(slab);
      CK(run_gett(d2, c->chA, tv, (const char*)Gp + (size_t)kmq * n2 * es, tv, c->chB, tv, acc, c));
      }
      // Sigma~[t][k][i][j] += -(1/Nk) sum_{(Q',b)} Y[t][i][(Q',b)] V^{k-q,k}[Q'][b][j]
      if (tc3) {
        // one GEMM over all (t, i) rows on tensor cores, K split over blocks
        const int64_t kp = c->kpad3;
        CK(embed_t((const char*)c->V + ((size_t)kmq * nk + k) * slab * 16, true, (int64_t)naux * nao, nao, c->W3hi,
                   c->W3lo, kp, c->st));
        UmmaOperand oa{c->Y3hi, c->Y3lo, (int64_t)ntau * nao, 1, kp, 0};
        UmmaOperand ob{c->W3hi, c->W3lo, 2 * (int64_t)nao, 1, kp, 0};
        const int64_t mt = ((int64_t)ntau * nao + 127) / 128, nt = (2 * (int64_t)nao + 159) / 160;
        int64_t ks = (304 + mt * nt - 1) / (mt * nt);
        if (ks > kp / 32) ks = kp / 32;
        if (ks < 1) ks = 1;
        CK(run_umma(c, 8.0 * ntau * nao * (double)nao * naux * nao, oa, ob, ntau * nao, 2 * nao, kp, 1,
                    (double*)(out + (size_t)k * n2), true, -1.0 / nk, true, 2 * (int64_t)nao, 0, (int)ks, nao,
                    2 * gstep, 0, 0, nullptr, 2 * (int64_t)naux * nao));
        count(1);
        continue;
      }
      GettDesc d3 = base_desc(nao, nao, (int64_t)naux * nao, ntau);
      d3.am = I1((int64_t)naux * nao); d3.ak = I1(1); d3.az = I1(slab);
      d3.bk = I1(nao); d3.bn = I1(1); d3.bz = I1(0);
      d3.cm = I1(nao); d3.cn = I1(1); d3.cz = I1(gstep);
      d3.alpha = make_double2(-1.0 / nk, 0);
      d3.beta = make_double2(accumulate || q > c->q0 ? 1.0 : 0.0, 0);
      d3.ksplit = 8;
      const char* Vk2 = (const char*)Vp + ((size_t)kmq * nk + k) * slab * es;
      CK(run_gett(d3, c->chB, tv, Vk2, tv, out + (size_t)k * n2, Ty::C128, acc, c));
    }
  }
  return GW_OK;
}

// Sigma~(tau) over the context's q range (Eq. tilde_sigma2), symmetrised, into Stau
static gw_status sigma_tau_part(gw_ctx* c) {
  const int nk = c->nk, nao = c->nao, ntau = c->ntau;
  const int64_t n2 = c->n2;
  const bool tc = uses_tc(c);
  const bool red = trs_reduce(c);
  c->reduce = red;
  gw_status s = sigma_chain(c, c->G_tau, c->P_tau, c->Stau, false);
  c->reduce = false;
  if (s != GW_OK) return s;
  if (red) {   // Sigma~^{-k}(tau) = conj Sigma~^k(tau)
    CK(conj_fill(c->Stau, ntau, nk, n2, c->d_kneg, c->d_kneed, c->st));
    count(1);
  }
  if (tc && !c->deferred) {
    int h = 0;
    CK(cudaMemcpyAsync(c->h_scr, c->info + 1, 4, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    memcpy(&h, c->h_scr, 4);
    if (h) return fail(c, GW_ERR_TIMEOUT, "tensor-core contraction gave up waiting (code " + std::to_string(h) + ")");
  }
  CK(herm_batched(c->Stau, nao, (int64_t)ntau * nk, n2, c->st));
  count(1);
  mark(c, GW_Q_SIGMA_TAU);
  return GW_OK;
}

// Sigma~(i w_n) = sum_j TFf[n][j] Sigma~(tau_j)   (Eq. tau_to_iw) into Siw_new
static gw_status sigma_iw_new(gw_ctx* c) {
  CK(transform(c, c->TFf, c->Stau, c->Siw_new, c->nw, (int64_t)c->nk * c->n2, 1, 0, 0));
  return GW_OK;
}

static gw_status sigma_dynamic(gw_ctx* c) {
  gw_status s = sigma_tau_part(c);
  return s != GW_OK ? s : sigma_iw_new(c);
}

extern "C" gw_status gw_selfenergy_partial(gw_ctx* c) {
  if (!c) return GW_ERR_ARG;
  if (!c->have_G) return fail(c, GW_ERR_STATE, "no Green's function yet");
  if (!c->have_P) return fail(c, GW_ERR_STATE, "no screened interaction yet");
  return sigma_tau_part(c);
}

extern "C" gw_status gw_selfenergy_finish(gw_ctx* c) {
  if (!c) return GW_ERR_ARG;
  if (!c->have_G) return fail(c, GW_ERR_STATE, "no Green's function yet");
  if (!(c->valid & qbit(GW_Q_SIGMA_TAU))) return fail(c, GW_ERR_STATE, "no Sigma~(tau) yet");
  gw_status s = gw_hf(c);
  if (s != GW_OK) return s;
  s = sigma_iw_new(c);
  if (s != GW_OK) return s;
  const int64_t ksz = (int64_t)c->nk * c->n2, gsz = (int64_t)c->nwf * ksz;
  CK(cudaMemsetAsync(c->dscr + 8, 0, 8, c->st));
  CK(maxabs_diff(c->Siw_new, c->Siw, gsz, c->dscr + 8, c->st));
  count(1);
  const double a = c->have_sigma ? c->cfg.damping : 1.0;
  CK(axpby(c->Sinf, c->Sinf_new, a, 1.0 - a, ksz, c->st));
  CK(axpby(c->Siw, c->Siw_new, a, 1.0 - a, gsz, c->st));
  count(2);
  c->have_sigma = true;
  return GW_OK;
}

extern "C" gw_status gw_selfenergy(gw_ctx* c) {
  gw_status s = gw_selfenergy_partial(c);
  return s != GW_OK ? s : gw_selfenergy_finish(c);
}

extern "C" gw_status gw_set_q_range(gw_ctx* c, int32_t q0, int32_t q1) {
  if (!c) return GW_ERR_ARG;
  if (q0 < 0 || q1 > c->nk || q0 >= q1) return fail(c, GW_ERR_ARG, "q range must satisfy 0 <= q0 < q1 <= nk");
  c->q0 = q0; c->q1 = q1;
  // results of another range are not those of this one
  c->have_P0 = c->have_P = false;
  for (gw_quantity q : {GW_Q_P0_TAU, GW_Q_P0_IW, GW_Q_P_IW, GW_Q_P_TAU, GW_Q_SIGMA_TAU}) unmark(c, q);
  return GW_OK;
}

// ------------------------------------------------------------------ A7: Dyson + mu

static DysonArgs dyson_args(gw_ctx* c) {
  DysonArgs a{};
  a.nao = c->nao; a.nk = c->nk; a.nw = c->nw;
  a.H0 = c->H0; a.S = c->S; a.Sinf = c->Sinf; a.Siw = c->Siw;
  a.wn = c->wn; a.r = c->r; a.spin = c->spin;
  return a;
}

extern "C" gw_status gw_dyson(gw_ctx* c, double* mu_out) {
  if (!c) return GW_ERR_ARG;
  DysonArgs a = dyson_args(c);
  const int64_t nsys = (int64_t)c->nw * c->nk;
  const double scale = -c->spin / c->nk;
  MuState* h = c->h_mus;
  memset(h, 0, sizeof(MuState));
  const double center = c->have_mu ? c->mu : 0.0;
  h->lo = center - 1.0; h->hi = center + 1.0; h->x = h->lo;
  h->target = c->cfg.n_elec; h->tol = c->cfg.mu_tol; h->width = 1e-13; h->maxit = c->cfg.mu_maxit;
  CK(cudaMemcpyAsync(c->mus, h, sizeof(MuState), cudaMemcpyHostToDevice, c->st));
  CK(cudaMemsetAsync(c->info, 0, 4, c->st));
  const int chunk = 8;
  for (int it = 0; it < c->cfg.mu_maxit + chunk; it += chunk) {
    for (int j = 0; j < chunk; ++j) {
      CK(dyson_eval(a, &c->mus->x, nullptr, c->partial, &c->mus->done, c->info, c->st));
      CK(mu_step(c->mus, c->partial, nsys, scale, c->st));
      count(2);
    }
    CK(cudaMemcpyAsync(h, c->mus, sizeof(MuState), cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (h->done) break;
  }
  c->mu_steps = h->iter;
  if (!h->done || h->status != 0) {
    char msg[320];
    snprintf(msg, sizeof msg,
             "chemical-potential search hit its cap: steps %d phase %d bracket [%.17g, %.17g] N(lo)=%.12g "
             "N(hi)=%.12g last x=%.17g N(x)=%.12g target %.12g",
             h->iter, h->phase, h->lo, h->hi, h->Nlo, h->Nhi, h->x, h->Nx, h->target);
    return fail(c, GW_ERR_NOT_CONVERGED, msg);
  }
  c->mu = h->x; c->have_mu = true; c->n_at_mu = h->Nx;
  // G(i w) at the final mu, then G(tau) = TBf G(i w), symmetrised
  CK(dyson_eval(a, &c->mus->x, c->G_iw, nullptr, nullptr, c->info, c->st));
  count(1);
  const int64_t gstep = (int64_t)c->nk * c->n2;
  CK(transform(c, c->TBf, c->G_iw, c->G_tau, c->ntau, gstep, 1, 0, 0));
  CK(herm_batched(c->G_tau, c->nao, (int64_t)c->ntau * c->nk, c->n2, c->st));
  count(1);
  int bad = 0;
  CK(cudaMemcpyAsync(c->h_scr, c->info, 4, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  memcpy(&bad, c->h_scr, 4);
  if (bad) return fail(c, GW_ERR_SINGULAR, "zero pivot in the Dyson inversion");
  c->have_G = true;
  mark(c, GW_Q_G_TAU); mark(c, GW_Q_G_IW); mark(c, GW_Q_MU); mark(c, GW_Q_N_ELEC);
  if (mu_out) *mu_out = c->mu;
  return GW_OK;
}

// mu search and Dyson with every step on the device (no host reads): the form
// captured into a graph.  The search restarts around the previous mu and runs a
// fixed number of (evaluate, step) pairs; converged pairs exit at once.
static gw_status dyson_device(gw_ctx* c) {
  DysonArgs a = dyson_args(c);
  const int64_t nsys = (int64_t)c->nw * c->nk;
  const double scale = -c->spin / c->nk;
  const int steps = c->cfg.mu_maxit < 96 ? c->cfg.mu_maxit : 96;
  CK(mu_init_device(c->mus, c->cfg.n_elec, c->cfg.mu_tol, 1e-13, steps, c->st));
  count(1);
  for (int j = 0; j < steps; ++j) {
    CK(dyson_eval(a, &c->mus->x, nullptr, c->partial, &c->mus->done, c->info, c->st));
    CK(mu_step(c->mus, c->partial, nsys, scale, c->st));
    count(2);
  }
  CK(dyson_eval(a, &c->mus->x, c->G_iw, nullptr, nullptr, c->info, c->st));
  const int64_t gstep = (int64_t)c->nk * c->n2;
  CK(transform(c, c->TBf, c->G_iw, c->G_tau, c->ntau, gstep, 1, 0, 0));
  CK(herm_batched(c->G_tau, c->nao, (int64_t)c->ntau * c->nk, c->n2, c->st));
  count(2);
  mark(c, GW_Q_G_TAU); mark(c, GW_Q_G_IW);
  return GW_OK;
}

// ------------------------------------------------------------------ iteration

extern "C" gw_status gw_iterate(gw_ctx* c, int32_t n_iter, gw_iter_stats* stats) {
  if (!c || n_iter < 0) return GW_ERR_ARG;
  gw_status s;
  if (!c->have_G) { if ((s = gw_dyson(c, nullptr)) != GW_OK) return s; }
  const int64_t gsz = (int64_t)c->ntau * c->nk * c->n2;
  for (int it = 0; it < n_iter; ++it) {
    CK(cudaEventRecord(c->ev[0], c->st));
    CK(cudaMemcpyAsync(c->G_prev, c->G_tau, gsz * 16, cudaMemcpyDeviceToDevice, c->st));
    if ((s = gw_polarization(c)) != GW_OK) return s;
    CK(cudaEventRecord(c->ev[1], c->st));
    if ((s = gw_screened(c)) != GW_OK) return s;
    CK(cudaEventRecord(c->ev[2], c->st));
    if ((s = gw_selfenergy(c)) != GW_OK) return s;
    CK(cudaEventRecord(c->ev[3], c->st));
    if ((s = gw_dyson(c, nullptr)) != GW_OK) return s;
    CK(cudaEventRecord(c->ev[4], c->st));
    CK(cudaMemsetAsync(c->dscr + 9, 0, 8, c->st));
    CK(maxabs_diff(c->G_tau, c->G_prev, gsz, c->dscr + 9, c->st));
    count(1);
    CK(cudaMemcpyAsync(c->h_scr, c->dscr, 16 * 8, cudaMemcpyDeviceToHost, c->st));
    CK(cudaStreamSynchronize(c->st));
    if (stats) {
      memset(stats, 0, sizeof(*stats));
      stats->mu = c->mu; stats->n_elec = c->n_at_mu; stats->mu_steps = c->mu_steps;
      stats->max_dSigma = c->h_scr[8]; stats->max_dG = c->h_scr[9];
      cudaEventElapsedTime(&stats->ms_total, c->ev[0], c->ev[4]);
      cudaEventElapsedTime(&stats->ms_polarization, c->ev[0], c->ev[1]);
      cudaEventElapsedTime(&stats->ms_screened, c->ev[1], c->ev[2]);
      cudaEventElapsedTime(&stats->ms_selfenergy, c->ev[2], c->ev[3]);
      cudaEventElapsedTime(&stats->ms_dyson, c->ev[3], c->ev[4]);
    }
  }
  return GW_OK;
}

// ------------------------------------------------------------------ profiling

extern "C" gw_status gw_profile(gw_ctx* c, int enable) {
  if (!c) return GW_ERR_ARG;
  CK(cudaStreamSynchronize(c->st));
  c->prof = enable != 0;
  c->pused = 0; c->pflops = 0.0; c->plaunch = 0;
  c->uused = 0; c->uflops = 0.0; c->ulaunch = 0;
  return GW_OK;
}

extern "C" gw_status gw_profile_read(gw_ctx* c, double* out6) {
  if (!c || !out6) return GW_ERR_ARG;
  CK(cudaStreamSynchronize(c->st));
  double ms = 0.0, ums = 0.0;
  for (size_t i = 0; i + 1 < c->pused; i += 2) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->pev[i], c->pev[i + 1]));
    ms += t;
  }
  for (size_t i = 0; i + 1 < c->uused; i += 2) {
    float t = 0.f;
    CK(cudaEventElapsedTime(&t, c->uev[i], c->uev[i + 1]));
    ums += t;
  }
  out6[0] = ms; out6[1] = c->pflops; out6[2] = (double)c->plaunch;
  out6[3] = ums; out6[4] = c->uflops; out6[5] = (double)c->ulaunch;
  c->pused = 0; c->pflops = 0.0; c->plaunch = 0;
  c->uused = 0; c->uflops = 0.0; c->ulaunch = 0;
  return GW_OK;
}

// ------------------------------------------------------------------ adjoints (A10)

namespace gwadj {
struct View {
  int nao, naux, nk, ntau;
  double spin;
  const double2* V;
  const double2* G_tau;
  const double2* P_tau;
  const int* kplus;
  const int* kminus;
  void* ws;
  size_t ws_bytes;
  double2 *bufA, *bufB, *bufC;
  cudaStream_t st;
  bool c64;
  const float2* V32;
  const float2* G32;
  const float2* P32;
  float2* bar32;
};
cudaError_t polarization_vjp(const View& v, const double2* Pbar, double2* Gbar, int64_t* launches);
cudaError_t selfenergy_vjp(const View& v, const double2* Sbar, double2* Gbar, double2* Pbar, int64_t* launches);

}  // namespace gwadj

// complex64 operands of the adjoint chains: V (the context's copy when it has one), G(tau),
// P~(tau) and the cotangent, converted on each call
static gw_status adj_c64(gw_ctx* c, gwadj::View* v) {
  const size_t gsz = (size_t)c->ntau * c->nk * c->n2, psz = (size_t)c->nk * c->ntau * c->na2;
  const size_t vsz = (size_t)c->nk * c->nk * c->naux * c->n2;
  if (!c->V32) {
    c->V32 = (float2*)dalloc(c, vsz * 8);
    if (!c->V32) return fail(c, GW_ERR_OOM, "complex64 copy of V");
    CK(to_c64(c->V, c->V32, (int64_t)vsz, c->st));
    count(1);
  }
  if (!c->adjG32) {
    c->adjG32 = (float2*)dalloc(c, gsz * 8);
    c->adjP32 = (float2*)dalloc(c, psz * 8);
    c->adjBar32 = (float2*)dalloc(c, (gsz > (size_t)c->ntau * c->na2 ? gsz : (size_t)c->ntau * c->na2) * 8);
    if (!c->adjG32 || !c->adjP32 || !c->adjBar32) return fail(c, GW_ERR_OOM, "complex64 adjoint buffers");
  }
  CK(to_c64(c->G_tau, c->adjG32, (int64_t)gsz, c->st));
  count(1);
  if (c->have_P) { CK(to_c64(c->P_tau, c->adjP32, (int64_t)psz, c->st)); count(1); }
  v->c64 = true; v->V32 = c->V32; v->G32 = c->adjG32; v->P32 = c->adjP32; v->bar32 = c->adjBar32;
  return GW_OK;
}

static gw_status adj_view(gw_ctx* c, gwadj::View* v) {
  const int64_t n2 = c->n2;
  const size_t tw = (size_t)(c->ntau > c->nwf ? (c->ntau > c->nwb ? c->ntau : c->nwb) : (c->nwf > c->nwb ? c->nwf : c->nwb));
  size_t need = (size_t)c->ntau * c->naux * n2;
  if (tw * c->na2 > need) need = tw * c->na2;
  if (tw * c->nk * n2 > need) need = tw * c->nk * n2;
  if (!c->adjA) {
    c->adjA = (double2*)dalloc(c, need * 16);
    c->adjB = (double2*)dalloc(c, need * 16);
    c->adjC = (double2*)dalloc(c, need * 16);
    if (!c->adjA || !c->adjB || !c->adjC) return fail(c, GW_ERR_OOM, "adjoint buffers");
  }
  v->nao = c->nao; v->naux = c->naux; v->nk = c->nk; v->ntau = c->ntau; v->spin = c->spin;
  v->V = c->V; v->G_tau = c->G_tau; v->P_tau = c->P_tau;
  v->kplus = c->kplus.data(); v->kminus = c->kminus.data();
  v->ws = c->ws; v->ws_bytes = c->ws_bytes;
  v->bufA = c->adjA; v->bufB = c->adjB; v->bufC = c->adjC;
  v->st = c->st;
  v->c64 = false; v->V32 = nullptr; v->G32 = nullptr; v->P32 = nullptr; v->bar32 = nullptr;
  return GW_OK;
}

static gw_status polarization_vjp_impl(gw_ctx* c, const double* Pbar, double* Gbar, bool c64) {
  if (!c || !Pbar || !Gbar) return fail(c, GW_ERR_ARG, "null argument");
  if (!c->have_G) return fail(c, GW_ERR_STATE, "no Green's function yet");
  gwadj::View v;
  gw_status s = adj_view(c, &v);
  if (s == GW_OK && c64) s = adj_c64(c, &v);
  if (s != GW_OK) return s;
  CK(cudaMemsetAsync(Gbar, 0, (size_t)c->ntau * c->nk * c->n2 * 16, c->st));
  int64_t l = 0;
  CK(gwadj::polarization_vjp(v, (const double2*)Pbar, (double2*)Gbar, &l));
  count((int)l);
  return GW_OK;
}

extern "C" gw_status gw_polarization_vjp(gw_ctx* c, const double* Pbar, double* Gbar) {
  return polarization_vjp_impl(c, Pbar, Gbar, false);
}
extern "C" gw_status gw_polarization_vjp_c64(gw_ctx* c, const double* Pbar, double* Gbar) {
  return polarization_vjp_impl(c, Pbar, Gbar, true);
}

static gw_status selfenergy_vjp_impl(gw_ctx* c, const double* Sbar, double* Gbar, double* Pbar, bool c64) {
  if (!c || !Sbar || !Gbar || !Pbar) return fail(c, GW_ERR_ARG, "null argument");
  if (!c->have_G) return fail(c, GW_ERR_STATE, "no Green's function yet");
  if (!c->have_P) return fail(c, GW_ERR_STATE, "no screened interaction yet");
  gwadj::View v;
  gw_status s = adj_view(c, &v);
  if (s == GW_OK && c64) s = adj_c64(c, &v);
  if (s != GW_OK) return s;
  CK(cudaMemsetAsync(Gbar, 0, (size_t)c->ntau * c->nk * c->n2 * 16, c->st));
  CK(cudaMemsetAsync(Pbar, 0, (size_t)c->nk * c->ntau * c->na2 * 16, c->st));
  int64_t l = 0;
  CK(gwadj::selfenergy_vjp(v, (const double2*)Sbar, (double2*)Gbar, (double2*)Pbar, &l));
  count((int)l);
  return GW_OK;
}

extern "C" gw_status gw_selfenergy_vjp(gw_ctx* c, const double* Sbar, double* Gbar, double* Pbar) {
  return selfenergy_vjp_impl(c, Sbar, Gbar, Pbar, false);
}
extern "C" gw_status gw_selfenergy_vjp_c64(gw_ctx* c, const double* Sbar, double* Gbar, double* Pbar) {
  return selfenergy_vjp_impl(c, Sbar, Gbar, Pbar, true);
}

// ------------------------------------------------------------------ tangents (A10)

// Tangents of the contraction chains at the context's precision: the forward chains
// with the tangent in one G (or P~) slot at a time (P~0 is quadratic in G, Sigma~
// bilinear in (G, P~)), then the symmetrisation.
static gw_status tc_check(gw_ctx* c) {
  if (!uses_tc(c) || c->deferred) return GW_OK;
  int h = 0;
  CK(cudaMemcpyAsync(c->h_scr, c->info + 1, 4, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  memcpy(&h, c->h_scr, 4);
  if (h) return fail(c, GW_ERR_TIMEOUT, "tensor-core contraction gave up waiting (code " + std::to_string(h) + ")");
  return GW_OK;
}

extern "C" gw_status gw_polarization_jvp(gw_ctx* c, const double* dG, double* dP0) {
  if (!c || !dG || !dP0) return fail(c, GW_ERR_ARG, "null argument");
  if (!c->have_G) return fail(c, GW_ERR_STATE, "no Green's function yet");
  const double2* g = (const double2*)dG;
  double2* out = (double2*)dP0;
  gw_status s = polar_chain(c, g, c->G_tau, out, false);
  if (s == GW_OK) s = polar_chain(c, c->G_tau, g, out, true);
  if (s == GW_OK) s = tc_check(c);
  if (s != GW_OK) return s;
  CK(herm_batched(out, c->naux, (int64_t)c->nk * c->ntau, c->na2, c->st));
  count(1);
  return GW_OK;
}

// dP~(tau) from dP~0(tau) through Eqs. P0t_to_P0w, tilde_P_omega and Piw_to_Pt:
// with X = (I - P~0(i Omega))^-1 = I + P~(i Omega), dP~(i Omega) = X dP~0(i Omega) X.
extern "C" gw_status gw_screened_jvp(gw_ctx* c, const double* dP0_tau, double* dP_tau) {
  if (!c || !dP0_tau || !dP_tau) return fail(c, GW_ERR_ARG, "null argument");
  if (!c->have_P) return fail(c, GW_ERR_STATE, "no screened interaction yet");
  gwadj::View v;
  gw_status s = adj_view(c, &v);
  if (s != GW_OK) return s;
  const int naux = c->naux, ntau = c->ntau, nw = c->nwb;
  const int64_t na2 = c->na2;
  for (int q = 0; q < c->nk; ++q) {
    const double2* x = (const double2*)dP0_tau + (size_t)q * ntau * na2;
    const double2* Pw = c->P_iw + (size_t)q * nw * na2;
    // T1 = TFb dP~0(tau)
    CK(transform(c, c->TFb, x, v.bufA, nw, na2, 1, 0, 0));
    // T2 = T1 + P~ T1   (per Omega)
    CK(cudaMemcpyAsync(v.bufB, v.bufA, (size_t)nw * na2 * 16, cudaMemcpyDeviceToDevice, c->st));
    GettDesc d = base_desc(naux, naux, naux, nw);
    d.am = I1(naux); d.ak = I1(1); d.az = I1(na2);
    d.bk = I1(naux); d.bn = I1(1); d.bz = I1(na2);
    d.cm = I1(naux); d.cn = I1(1); d.cz = I1(na2);
    d.beta = make_double2(1, 0);
    CK(run_gett(d, Pw, Ty::C128, v.bufA, Ty::C128, v.bufB, Ty::C128, Ty::C128, c));
    // T3 = T2 + T2 P~
    CK(cudaMemcpyAsync(v.bufA, v.bufB, (size_t)nw * na2 * 16, cudaMemcpyDeviceToDevice, c->st));
    CK(run_gett(d, v.bufB, Ty::C128, Pw, Ty::C128, v.bufA, Ty::C128, Ty::C128, c));
    // dP~(tau) = TBb T3
    CK(transform(c, c->TBb, v.bufA, (double2*)dP_tau + (size_t)q * ntau * na2, ntau, na2, 1, 0, 0));
  }
  CK(herm_batched((double2*)dP_tau, naux, (int64_t)c->nk * ntau, na2, c->st));
  count(1);
  return GW_OK;
}

extern "C" gw_status gw_selfenergy_jvp(gw_ctx* c, const double* dG, const double* dP_tau, double* dS_tau) {
  if (!c || !dG || !dP_tau || !dS_tau) return fail(c, GW_ERR_ARG, "null argument");
  if (!c->have_G) return fail(c, GW_ERR_STATE, "no Green's function yet");
  if (!c->have_P) return fail(c, GW_ERR_STATE, "no screened interaction yet");
  double2* out = (double2*)dS_tau;
  gw_status s = sigma_chain(c, (const double2*)dG, c->P_tau, out, false);
  if (s == GW_OK) s = sigma_chain(c, c->G_tau, (const double2*)dP_tau, out, true);
  if (s == GW_OK) s = tc_check(c);
  if (s != GW_OK) return s;
  CK(herm_batched(out, c->nao, (int64_t)c->ntau * c->nk, c->n2, c->st));
  count(1);
  return GW_OK;
}

// ------------------------------------------------------------------ tangent of the SC map (A10)

static gw_status sc_tangent_buffers(gw_ctx* c) {
  if (c->tGiw) return GW_OK;
  const size_t gsz = (size_t)c->ntau * c->nk * c->n2 * 16, psz = (size_t)c->nk * c->ntau * c->na2 * 16;
  c->tGiw = (double2*)dalloc(c, (size_t)c->nwf * c->nk * c->n2 * 16);
  c->tGtau = (double2*)dalloc(c, gsz);
  c->tS = (double2*)dalloc(c, gsz);
  c->tgam = (double2*)dalloc(c, (size_t)c->nk * c->n2 * 16);
  c->tP = (double2*)dalloc(c, psz);
  const size_t np = (size_t)2 * c->nw * c->nk + 8;
  c->tpart = (double*)dalloc(c, (np > 1224 ? np : 1224) * 8);   // Dyson-tangent traces / inner-product partials
  if (!c->tGiw || !c->tGtau || !c->tS || !c->tgam || !c->tP || !c->tpart) return fail(c, GW_ERR_OOM, "tangent buffers");
  return GW_OK;
}

// One tangent of the self-consistency map F: (Sigma_inf, Sigma(i w)) -> (Sigma_inf', Sigma'(i w))
// at the context's state (G from gw_dyson at this Sigma, P~ from gw_screened at this G).
static gw_status sc_jvp(gw_ctx* c, const double2* dSinf, const double2* dSiw, double2* oSinf, double2* oSiw) {
  gwadj::View v;
  gw_status s = adj_view(c, &v);
  if (s == GW_OK) s = sc_tangent_buffers(c);
  if (s != GW_OK) return s;
  const int nao = c->nao, nk = c->nk, nw = c->nw;
  const int64_t n2 = c->n2, nsys = (int64_t)nw * nk, gstep = (int64_t)nk * n2;
  // Dyson: dG(i w) = G D G - dmu G S G, D = dSigma_inf + dSigma(i w)
  CK(dyson_tangent_rhs(dSinf, dSiw, v.bufA, nk, n2, nw, c->st));
  GettDesc d = base_desc(nao, nao, nao, nsys);
  d.am = I1(nao); d.ak = I1(1); d.az = I1(n2);
  d.bk = I1(nao); d.bn = I1(1); d.bz = I1(n2);
  d.cm = I1(nao); d.cn = I1(1); d.cz = I1(n2);
  CK(run_gett(d, c->G_iw, Ty::C128, v.bufA, Ty::C128, v.bufB, Ty::C128, Ty::C128, c));   // G D
  CK(run_gett(d, v.bufB, Ty::C128, c->G_iw, Ty::C128, v.bufA, Ty::C128, Ty::C128, c));   // (G D) G
  GettDesc ds = d;
  ds.bz = I2(nk, 0, n2);   // S^k for system (w, k)
  CK(run_gett(ds, c->G_iw, Ty::C128, c->S, Ty::C128, v.bufB, Ty::C128, Ty::C128, c));    // G S
  CK(run_gett(d, v.bufB, Ty::C128, c->G_iw, Ty::C128, v.bufC, Ty::C128, Ty::C128, c));   // (G S) G
  CK(dyson_tangent_finish(v.bufA, v.bufC, c->S, c->r, nao, nk, nw, c->tpart, c->tpart + 2 * nsys, c->tGiw, c->st));
  count(4);
  // dG(tau) = TBf dG(i w), symmetrised
  CK(transform(c, c->TBf, c->tGiw, c->tGtau, c->ntau, gstep, 1, 0, 0));
  CK(herm_batched(c->tGtau, nao, (int64_t)c->ntau * nk, n2, c->st));
  count(1);
  // dSigma_inf' = J[dgamma] + K[dgamma]
  if ((s = hf_core(c, c->tGtau, c->tgam, oSinf)) != GW_OK) return s;
  // dP~0, then dP~ through the screened block (in place), then dSigma~
  if ((s = polar_chain(c, c->tGtau, c->G_tau, c->tP, false)) != GW_OK) return s;
  if ((s = polar_chain(c, c->G_tau, c->tGtau, c->tP, true)) != GW_OK) return s;
  CK(herm_batched(c->tP, c->naux, (int64_t)nk * c->ntau, c->na2, c->st));
  count(1);
  if ((s = gw_screened_jvp(c, (const double*)c->tP, (double*)c->tP)) != GW_OK) return s;
  if ((s = sigma_chain(c, c->tGtau, c->P_tau, c->tS, false)) != GW_OK) return s;
  if ((s = sigma_chain(c, c->G_tau, c->tP, c->tS, true)) != GW_OK) return s;
  if ((s = tc_check(c)) != GW_OK) return s;
  CK(herm_batched(c->tS, nao, (int64_t)c->ntau * nk, n2, c->st));
  count(1);
  // dSigma'(i w) = TFf dSigma~(tau)
  CK(transform(c, c->TFf, c->tS, oSiw, nw, gstep, 1, 0, 0));
  return GW_OK;
}

extern "C" gw_status gw_sc_jvp(gw_ctx* c, const double* dSinf, const double* dSiw, double* oSinf, double* oSiw) {
  if (!c || !dSinf || !dSiw || !oSinf || !oSiw) return fail(c, GW_ERR_ARG, "null argument");
  if (!c->have_G || !c->have_mu) return fail(c, GW_ERR_STATE, "no Dyson solution yet");
  if (!c->have_P) return fail(c, GW_ERR_STATE, "no screened interaction yet");
  return sc_jvp(c, (const double2*)dSinf, (const double2*)dSiw, (double2*)oSinf, (double2*)oSiw);
}

// ------------------------------------------------------------------ Newton-Krylov iterations (A10)

static gw_status rdot(gw_ctx* c, const double2* a, const double2* b, int64_t n, double* out) {
  const int nb = rdot_blocks(n);
  CK(rdot_partials(a, b, n, c->tpart, c->st));
  double acc = 0;
  std::vector<double> h((size_t)nb);
  CK(cudaMemcpyAsync(h.data(), c->tpart, (size_t)nb * 8, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  for (int i = 0; i < nb; ++i) acc += h[(size_t)i];
  *out = acc;
  count(1);
  return GW_OK;
}

// The forward map at the current Sigma: Dyson (mu search), P~0, screened, Sigma_inf'
// and Sigma'(i w) (unmixed) into Sinf_new / Siw_new.
static gw_status sc_forward(gw_ctx* c) {
  gw_status s;
  if ((s = gw_dyson(c, nullptr)) != GW_OK) return s;
  if ((s = gw_polarization(c)) != GW_OK) return s;
  if ((s = gw_screened(c)) != GW_OK) return s;
  if ((s = hf_core(c, c->G_tau, c->gamma, c->Sinf_new)) != GW_OK) return s;
  mark(c, GW_Q_GAMMA); mark(c, GW_Q_SIGMA_INF_NEW);
  return sigma_dynamic(c);
}

extern "C" gw_status gw_iterate_newton(gw_ctx* c, int32_t n_outer, int32_t m, double tol, double* res_out) {
  if (!c || n_outer < 0 || m < 1 || m > 64) return fail(c, GW_ERR_ARG, "bad Newton-Krylov arguments");
  gw_status s = sc_tangent_buffers(c);
  if (s != GW_OK) return s;
  gwadj::View v;
  if ((s = adj_view(c, &v)) != GW_OK) return s;
  const int64_t ki = (int64_t)c->nk * c->n2, nx = ki + (int64_t)c->nw * ki;
  if (c->nvec < m + 2) {
    c->kry.clear();
    for (int i = 0; i < m + 2; ++i) {
      double2* p = (double2*)dalloc(c, (size_t)nx * 16);
      if (!p) return fail(c, GW_ERR_OOM, "Krylov basis");
      c->kry.push_back(p);
    }
    c->nvec = m + 2;
  }
  double2* R = c->kry[(size_t)m + 1];   // residual F(x) - x
  for (int it = 0; it < n_outer; ++it) {
    if ((s = sc_forward(c)) != GW_OK) return s;
    // R = F(x) - x
    CK(cudaMemcpyAsync(R, c->Sinf_new, (size_t)ki * 16, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(R + ki, c->Siw_new, (size_t)(nx - ki) * 16, cudaMemcpyDeviceToDevice, c->st));
    CK(axpby(R, c->Sinf, -1.0, 1.0, ki, c->st));
    CK(axpby(R + ki, c->Siw, -1.0, 1.0, nx - ki, c->st));
    count(2);
    double rr = 0;
    if ((s = rdot(c, R, R, nx, &rr)) != GW_OK) return s;
    const double beta = std::sqrt(rr);
    if (res_out) res_out[it] = beta;
    if (beta <= tol) { for (int j = it + 1; j < n_outer; ++j) if (res_out) res_out[j] = beta; break; }
    // GMRES on (J - I) delta = -R: v0 = -R / beta
    std::vector<double> H((size_t)(m + 1) * m, 0.0);
    CK(cudaMemsetAsync(c->kry[0], 0, (size_t)nx * 16, c->st));
    CK(axpby(c->kry[0], R, -1.0 / beta, 0.0, nx, c->st));
    int used = 0;
    for (int j = 0; j < m; ++j) {
      double2* w = c->kry[(size_t)j + 1];
      if ((s = sc_jvp(c, c->kry[(size_t)j], c->kry[(size_t)j] + ki, w, w + ki)) != GW_OK) return s;
      CK(axpby(w, c->kry[(size_t)j], -1.0, 1.0, nx, c->st));   // (J - I) v_j
      for (int i = 0; i <= j; ++i) {   // modified Gram-Schmidt
        double h = 0;
        if ((s = rdot(c, w, c->kry[(size_t)i], nx, &h)) != GW_OK) return s;
        H[(size_t)i * m + j] = h;
        CK(axpby(w, c->kry[(size_t)i], -h, 1.0, nx, c->st));
      }
      double hn = 0;
      if ((s = rdot(c, w, w, nx, &hn)) != GW_OK) return s;
      hn = std::sqrt(hn);
      H[(size_t)(j + 1) * m + j] = hn;
      used = j + 1;
      if (hn <= 1e-14 * beta) break;
      CK(axpby(w, w, 0.0, 1.0 / hn, nx, c->st));
    }
    // least squares min || beta e1 - H y || by Givens rotations (host, used <= 64)
    std::vector<double> g((size_t)used + 1, 0.0), y((size_t)used, 0.0);
    g[0] = beta;
    std::vector<double> Hc = H;
    for (int j = 0; j < used; ++j) {
      const double a = Hc[(size_t)j * m + j], b = Hc[(size_t)(j + 1) * m + j];
      const double rho = std::sqrt(a * a + b * b);
      const double cs = rho > 0 ? a / rho : 1.0, sn = rho > 0 ? b / rho : 0.0;
      for (int k = j; k < used; ++k) {
        const double u = Hc[(size_t)j * m + k], t = Hc[(size_t)(j + 1) * m + k];
        Hc[(size_t)j * m + k] = cs * u + sn * t;
        Hc[(size_t)(j + 1) * m + k] = -sn * u + cs * t;
      }
      const double gj = g[(size_t)j];
      g[(size_t)j] = cs * gj;
      g[(size_t)j + 1] = -sn * gj;
    }
    for (int j = used - 1; j >= 0; --j) {
      double t = g[(size_t)j];
      for (int k = j + 1; k < used; ++k) t -= Hc[(size_t)j * m + k] * y[(size_t)k];
      const double dgl = Hc[(size_t)j * m + j];
      y[(size_t)j] = dgl != 0.0 ? t / dgl : 0.0;
    }
    // x <- x + sum y_j v_j  (x lives in Sinf / Siw)
    for (int j = 0; j < used; ++j) {
      CK(axpby(c->Sinf, c->kry[(size_t)j], y[(size_t)j], 1.0, ki, c->st));
      CK(axpby(c->Siw, c->kry[(size_t)j] + ki, y[(size_t)j], 1.0, nx - ki, c->st));
    }
    count(2 * used);
    c->have_sigma = true;
  }
  // leave the context at a consistent state: G from the final Sigma
  if ((s = gw_dyson(c, nullptr)) != GW_OK) return s;
  c->have_P0 = false;
  c->have_P = false;
  return GW_OK;
}

// ------------------------------------------------------------------ DIIS self-consistency (F4)

// Least-squares solution of the (n x n) system A c = rhs by Householder QR (row-major,
// A overwritten); columns whose pivot is negligible get a zero coefficient.
static void small_lstsq(std::vector<double>& A, std::vector<double>& rhs, int n, std::vector<double>& c) {
  for (int j = 0; j < n; ++j) {
    double nrm = 0;
    for (int i = j; i < n; ++i) nrm += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    nrm = std::sqrt(nrm);
    if (nrm == 0.0) continue;
    const double a0 = A[(size_t)j * n + j];
    const double alpha = a0 > 0 ? -nrm : nrm;
    std::vector<double> v((size_t)n, 0.0);
    for (int i = j; i < n; ++i) v[(size_t)i] = A[(size_t)i * n + j];
    v[(size_t)j] -= alpha;
    double vv = 0;
    for (int i = j; i < n; ++i) vv += v[(size_t)i] * v[(size_t)i];
    if (vv == 0.0) continue;
    for (int k = j; k < n; ++k) {
      double d = 0;
      for (int i = j; i < n; ++i) d += v[(size_t)i] * A[(size_t)i * n + k];
      d = 2.0 * d / vv;
      for (int i = j; i < n; ++i) A[(size_t)i * n + k] -= d * v[(size_t)i];
    }
    double d = 0;
    for (int i = j; i < n; ++i) d += v[(size_t)i] * rhs[(size_t)i];
    d = 2.0 * d / vv;
    for (int i = j; i < n; ++i) rhs[(size_t)i] -= d * v[(size_t)i];
  }
  double rmax = 0;
  for (int j = 0; j < n; ++j) rmax = std::fmax(rmax, std::fabs(A[(size_t)j * n + j]));
  c.assign((size_t)n, 0.0);
  for (int j = n - 1; j >= 0; --j) {
    const double r = A[(size_t)j * n + j];
    if (std::fabs(r) <= 1e-14 * rmax) continue;
    double t = rhs[(size_t)j];
    for (int k = j + 1; k < n; ++k) t -= A[(size_t)j * n + k] * c[(size_t)k];
    c[(size_t)j] = t / r;
  }
}

extern "C" gw_status gw_iterate_diis(gw_ctx* c, int32_t n_iter, int32_t m, double mix, double tol, double* res_out) {
  if (!c || n_iter < 0 || m < 1 || m > 32) return fail(c, GW_ERR_ARG, "bad DIIS arguments");
  gw_status s = sc_tangent_buffers(c);   // inner-product partials
  if (s != GW_OK) return s;
  const int64_t ki = (int64_t)c->nk * c->n2, nx = ki + (int64_t)c->nw * ki;
  if ((int)c->dx.size() < m) {
    for (int i = (int)c->dx.size(); i < m; ++i) {
      double2* px = (double2*)dalloc(c, (size_t)nx * 16);
      double2* pr = (double2*)dalloc(c, (size_t)nx * 16);
      if (!px || !pr) return fail(c, GW_ERR_OOM, "DIIS history");
      c->dx.push_back(px);
      c->dr.push_back(pr);
    }
  }
  if (!c->dnext) {
    c->dnext = (double2*)dalloc(c, (size_t)nx * 16);
    if (!c->dnext) return fail(c, GW_ERR_OOM, "DIIS buffer");
  }
  // history of this call: slot h % m holds step h; B[i][j] = Re <r_i, r_j>
  std::vector<double> B((size_t)m * m, 0.0);
  int nh = 0;
  for (int it = 0; it < n_iter; ++it) {
    if ((s = sc_forward(c)) != GW_OK) return s;
    const int slot = nh % m;
    double2* X = c->dx[(size_t)slot];
    double2* R = c->dr[(size_t)slot];
    // x = current input, r = F(x) - x
    CK(cudaMemcpyAsync(X, c->Sinf, (size_t)ki * 16, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(X + ki, c->Siw, (size_t)(nx - ki) * 16, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(R, c->Sinf_new, (size_t)ki * 16, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(R + ki, c->Siw_new, (size_t)(nx - ki) * 16, cudaMemcpyDeviceToDevice, c->st));
    CK(axpby(R, X, -1.0, 1.0, nx, c->st));
    count(1);
    ++nh;
    const int n = nh < m ? nh : m;
    // new row / column of B (oldest entry replaced in the ring)
    for (int j = 0; j < n; ++j) {
      const int sj = (nh - n + j) % m;
      double b = 0;
      if ((s = rdot(c, R, c->dr[(size_t)sj], nx, &b)) != GW_OK) return s;
      B[(size_t)slot * m + sj] = B[(size_t)sj * m + slot] = b;
    }
    const double rn = std::sqrt(B[(size_t)slot * m + slot]);
    if (res_out) res_out[it] = rn;
    if (rn <= tol) { for (int j = it + 1; j < n_iter; ++j) if (res_out) res_out[j] = rn; break; }
    // min || sum c_i r_i ||^2 with sum c_i = 1: bordered system, scaled by max B_ii
    double scale = 0;
    for (int j = 0; j < n; ++j) {
      const int sj = (nh - n + j) % m;
      scale = std::fmax(scale, B[(size_t)sj * m + sj]);
    }
    if (scale <= 0) scale = 1.0;
    const int N = n + 1;
    std::vector<double> A((size_t)N * N, 0.0), rhs((size_t)N, 0.0), coef;
    for (int i = 0; i < n; ++i) {
      const int si = (nh - n + i) % m;
      for (int j = 0; j < n; ++j) A[(size_t)i * N + j] = B[(size_t)si * m + (nh - n + j) % m] / scale;
      A[(size_t)i * N + n] = A[(size_t)n * N + i] = 1.0;
    }
    rhs[(size_t)n] = 1.0;
    small_lstsq(A, rhs, N, coef);
    // x_next = sum c_i (x_i + mix r_i)
    CK(cudaMemsetAsync(c->dnext, 0, (size_t)nx * 16, c->st));
    for (int i = 0; i < n; ++i) {
      const int si = (nh - n + i) % m;
      CK(axpby(c->dnext, c->dx[(size_t)si], coef[(size_t)i], 1.0, nx, c->st));
      CK(axpby(c->dnext, c->dr[(size_t)si], coef[(size_t)i] * mix, 1.0, nx, c->st));
    }
    count(2 * n);
    CK(cudaMemcpyAsync(c->Sinf, c->dnext, (size_t)ki * 16, cudaMemcpyDeviceToDevice, c->st));
    CK(cudaMemcpyAsync(c->Siw, c->dnext + ki, (size_t)(nx - ki) * 16, cudaMemcpyDeviceToDevice, c->st));
    c->have_sigma = true;
  }
  // leave the context at a consistent state: G from the final Sigma
  if ((s = gw_dyson(c, nullptr)) != GW_OK) return s;
  c->have_P0 = false;
  c->have_P = false;
  return GW_OK;
}

// ------------------------------------------------------------------ captured iterations (A9)

static gw_status capture_iteration(gw_ctx* c) {
  if (c->gexec) return GW_OK;
  if (!c->gst) {
    CK(cudaStreamCreateWithFlags(&c->gst, cudaStreamNonBlocking));
    for (auto& e : c->gev) CK(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  }
  const int64_t gsz = (int64_t)c->ntau * c->nk * c->n2;
  cudaStream_t keep = c->st;
  c->st = c->gst;
  c->deferred = true;
  gw_status s = GW_OK;
  cudaError_t e = cudaStreamBeginCapture(c->gst, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaMemsetAsync(c->info, 0, 16, c->gst);
    cudaMemcpyAsync(c->G_prev, c->G_tau, gsz * 16, cudaMemcpyDeviceToDevice, c->gst);
    if (s == GW_OK) s = gw_polarization(c);
    if (s == GW_OK) s = gw_screened(c);
    if (s == GW_OK) s = gw_selfenergy(c);
    if (s == GW_OK) s = dyson_device(c);
    cudaGraph_t g = nullptr;
    cudaError_t e2 = cudaStreamEndCapture(c->gst, &g);
    if (s == GW_OK && e2 != cudaSuccess) s = fail(c, GW_ERR_CUDA, std::string("capture: ") + cudaGetErrorString(e2));
    if (s == GW_OK) {
      c->graph = g;
      e2 = cudaGraphInstantiate(&c->gexec, g, 0);
      if (e2 != cudaSuccess) s = fail(c, GW_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e2));
      size_t nn = 0;
      if (s == GW_OK && cudaGraphGetNodes(g, nullptr, &nn) == cudaSuccess && nn > 0) {
        std::vector<cudaGraphNode_t> nodes(nn);
        if (cudaGraphGetNodes(g, nodes.data(), &nn) == cudaSuccess) {
          c->graph_kernels = 0;
          for (size_t i = 0; i < nn; ++i) {
            cudaGraphNodeType t;
            if (cudaGraphNodeGetType(nodes[i], &t) == cudaSuccess && t == cudaGraphNodeTypeKernel) ++c->graph_kernels;
          }
        }
      }
    } else if (g) {
      cudaGraphDestroy(g);
    }
  } else {
    s = fail(c, GW_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
  }
  c->deferred = false;
  c->st = keep;
  return s;
}

static gw_status launch_graph(gw_ctx* c) {
  CK(cudaEventRecord(c->gev[0], c->st));
  CK(cudaStreamWaitEvent(c->gst, c->gev[0], 0));
  CK(cudaGraphLaunch(c->gexec, c->gst));
  g_launches += c->graph_kernels;
  CK(cudaEventRecord(c->gev[1], c->gst));
  CK(cudaStreamWaitEvent(c->st, c->gev[1], 0));
  return GW_OK;
}

static gw_status finish_graph(gw_ctx* c, gw_iter_stats* stats) {
  CK(cudaMemcpyAsync(c->h_mus, c->mus, sizeof(MuState), cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(c->h_scr + 20, c->info, 16, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  int flags[4];
  memcpy(flags, c->h_scr + 20, 16);
  const MuState* h = c->h_mus;
  c->mu_steps = h->iter;
  if (flags[1]) return fail(c, GW_ERR_TIMEOUT, "tensor-core contraction gave up waiting");
  if (flags[2]) return fail(c, GW_ERR_SINGULAR, "zero pivot in the screened solve");
  if (flags[0]) return fail(c, GW_ERR_SINGULAR, "zero pivot in the Dyson inversion");
  if (!h->done || h->status != 0) return fail(c, GW_ERR_NOT_CONVERGED, "chemical-potential search hit its cap");
  c->mu = h->x; c->have_mu = true; c->n_at_mu = h->Nx;
  mark(c, GW_Q_MU); mark(c, GW_Q_N_ELEC);
  if (stats) {
    memset(stats, 0, sizeof(*stats));
    stats->mu = c->mu; stats->n_elec = c->n_at_mu; stats->mu_steps = c->mu_steps;
  }
  return GW_OK;
}

static gw_status graph_prologue(gw_ctx* c, int32_t* n_iter) {
  gw_status s;
  if (!c->have_G) { if ((s = gw_dyson(c, nullptr)) != GW_OK) return s; }
  if (!c->have_sigma && *n_iter > 0) {   // the first GW iteration is not mixed: run it uncaptured
    if ((s = gw_iterate(c, 1, nullptr)) != GW_OK) return s;
    *n_iter -= 1;
  }
  return capture_iteration(c);
}

extern "C" gw_status gw_iterate_graph(gw_ctx* c, int32_t n_iter, gw_iter_stats* stats) {
  if (!c || n_iter < 0) return GW_ERR_ARG;
  gw_status s = graph_prologue(c, &n_iter);
  if (s != GW_OK) return s;
  CK(cudaEventRecord(c->ev[0], c->st));
  for (int it = 0; it < n_iter; ++it)
    if ((s = launch_graph(c)) != GW_OK) return s;
  CK(cudaEventRecord(c->ev[4], c->st));
  s = finish_graph(c, stats);
  if (s == GW_OK && stats && n_iter > 0) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c->ev[0], c->ev[4]);
    stats->ms_total = ms / n_iter;
  }
  return s;
}

extern "C" gw_status gw_batch_iterate(gw_ctx* const* ctxs, int32_t n, int32_t n_iter) {
  if (!ctxs || n <= 0 || n_iter < 0) return fail(nullptr, GW_ERR_ARG, "bad batch");
  std::vector<int32_t> left(n, n_iter);
  for (int i = 0; i < n; ++i) {
    if (!ctxs[i]) return fail(nullptr, GW_ERR_ARG, "null context in batch");
    gw_status s = graph_prologue(ctxs[i], &left[i]);
    if (s != GW_OK) { g_init_err = "system " + std::to_string(i) + ": " + ctxs[i]->err; return s; }
  }
  // round-robin launches: each system's graph runs on its own stream, so the
  // GPU overlaps the systems
  int32_t maxleft = 0;
  for (int i = 0; i < n; ++i) maxleft = left[i] > maxleft ? left[i] : maxleft;
  for (int it = 0; it < maxleft; ++it)
    for (int i = 0; i < n; ++i)
      if (it < left[i]) {
        gw_status s = launch_graph(ctxs[i]);
        if (s != GW_OK) { g_init_err = "system " + std::to_string(i) + ": " + ctxs[i]->err; return s; }
      }
  for (int i = 0; i < n; ++i) {
    gw_status s = finish_graph(ctxs[i], nullptr);
    if (s != GW_OK) { g_init_err = "system " + std::to_string(i) + ": " + ctxs[i]->err; return s; }
  }
  return GW_OK;
}

// ------------------------------------------------------------------ checkpoint / resume

// File layout: a fixed header (magic, version, sizes, beta, mu, state flags), then G(tau),
// Sigma_inf and Sigma~(i w) as complex128 arrays, then an FNV-1a hash of everything before it.
namespace {
struct StateHeader {
  char magic[8];
  int32_t version, nao, naux, ntau, kmesh[3], flags, nwf, nwb;
  double beta, mu, n_at_mu;
};
constexpr char kStateMagic[8] = {'G', 'W', 'G', 'B', 'S', 'T', 'A', '1'};
uint64_t fnv1a(const void* p, size_t n, uint64_t h) {
  const unsigned char* b = (const unsigned char*)p;
  for (size_t i = 0; i < n; ++i) { h ^= b[i]; h *= 1099511628211ull; }
  return h;
}
}  // namespace

extern "C" gw_status gw_save_state(gw_ctx* c, const char* path) {
  if (!c || !path) return fail(c, GW_ERR_ARG, "null argument");
  if (!c->have_G) return fail(c, GW_ERR_STATE, "no Green's function to save");
  const size_t gsz = (size_t)c->ntau * c->nk * c->n2, ksz = (size_t)c->nk * c->n2, wsz = (size_t)c->nwf * ksz;
  std::vector<double2> G(gsz), Si(ksz), Sw(wsz);
  CK(cudaMemcpyAsync(G.data(), c->G_tau, gsz * 16, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(Si.data(), c->Sinf, ksz * 16, cudaMemcpyDeviceToHost, c->st));
  CK(cudaMemcpyAsync(Sw.data(), c->Siw, wsz * 16, cudaMemcpyDeviceToHost, c->st));
  CK(cudaStreamSynchronize(c->st));
  StateHeader h{};
  memcpy(h.magic, kStateMagic, 8);
  h.version = 1; h.nao = c->nao; h.naux = c->naux; h.ntau = c->ntau; h.nwf = c->nwf; h.nwb = c->nwb;
  for (int i = 0; i < 3; ++i) h.kmesh[i] = c->cfg.kmesh[i];
  h.flags = (c->have_sigma ? 1 : 0) | (c->have_mu ? 2 : 0);
  h.beta = c->cfg.beta; h.mu = c->mu; h.n_at_mu = c->n_at_mu;
  FILE* f = fopen(path, "wb");
  if (!f) return fail(c, GW_ERR_ARG, std::string("cannot open ") + path + " for writing");
  uint64_t hash = 1469598103934665603ull;
  bool ok = fwrite(&h, sizeof h, 1, f) == 1;
  hash = fnv1a(&h, sizeof h, hash);
  for (const std::vector<double2>* v : {&G, &Si, &Sw}) {
    ok = ok && fwrite(v->data(), 16, v->size(), f) == v->size();
    hash = fnv1a(v->data(), v->size() * 16, hash);
  }
  ok = ok && fwrite(&hash, 8, 1, f) == 1;
  ok = (fclose(f) == 0) && ok;
  if (!ok) return fail(c, GW_ERR_INTERNAL, std::string("write failed: ") + path);
  return GW_OK;
}

extern "C" gw_status gw_load_state(gw_ctx* c, const char* path) {
  if (!c || !path) return fail(c, GW_ERR_ARG, "null argument");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(c, GW_ERR_ARG, std::string("cannot open ") + path);
  StateHeader h{};
  const size_t gsz = (size_t)c->ntau * c->nk * c->n2, ksz = (size_t)c->nk * c->n2, wsz = (size_t)c->nwf * ksz;
  std::vector<double2> G(gsz), Si(ksz), Sw(wsz);
  uint64_t hash = 1469598103934665603ull, stored = 0;
  bool ok = fread(&h, sizeof h, 1, f) == 1;
  const bool same = ok && memcmp(h.magic, kStateMagic, 8) == 0 && h.version == 1 && h.nao == c->nao &&
                    h.naux == c->naux && h.ntau == c->ntau && h.nwf == c->nwf && h.nwb == c->nwb &&
                    h.kmesh[0] == c->cfg.kmesh[0] &&
                    h.kmesh[1] == c->cfg.kmesh[1] && h.kmesh[2] == c->cfg.kmesh[2] && h.beta == c->cfg.beta;
  if (!same) { fclose(f); return fail(c, GW_ERR_ARG, "state file does not match this context's sizes"); }
  hash = fnv1a(&h, sizeof h, hash);
  for (std::vector<double2>* v : {&G, &Si, &Sw}) {
    ok = ok && fread(v->data(), 16, v->size(), f) == v->size();
    if (ok) hash = fnv1a(v->data(), v->size() * 16, hash);
  }
  ok = ok && fread(&stored, 8, 1, f) == 1;
  char extra;
  ok = ok && fread(&extra, 1, 1, f) == 0;
  fclose(f);
  if (!ok || stored != hash) return fail(c, GW_ERR_ARG, "state file is truncated or corrupt");
  CK(cudaMemcpyAsync(c->G_tau, G.data(), gsz * 16, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->Sinf, Si.data(), ksz * 16, cudaMemcpyHostToDevice, c->st));
  CK(cudaMemcpyAsync(c->Siw, Sw.data(), wsz * 16, cudaMemcpyHostToDevice, c->st));
  CK(cudaStreamSynchronize(c->st));
  c->have_G = true;
  c->have_sigma = (h.flags & 1) != 0;
  c->have_mu = (h.flags & 2) != 0;
  c->mu = h.mu; c->n_at_mu = h.n_at_mu;
  c->have_P0 = c->have_P = false;
  for (gw_quantity q : {GW_Q_P0_TAU, GW_Q_P0_IW, GW_Q_P_IW, GW_Q_P_TAU, GW_Q_SIGMA_TAU, GW_Q_G_IW, GW_Q_GAMMA,
                        GW_Q_SIGMA_INF_NEW})
    unmark(c, q);
  mark(c, GW_Q_G_TAU);
  if (c->have_mu) { mark(c, GW_Q_MU); mark(c, GW_Q_N_ELEC); }
  return GW_OK;
}

// ------------------------------------------------------------------ F4: Phi~ (Eq. tilde_Phi_GW)

extern "C" gw_status gw_grand_potential(gw_ctx* c, double* phi) {
  if (!c || !phi) return fail(c, GW_ERR_ARG, "null argument");
  if (c->deferred) return fail(c, GW_ERR_STATE, "not available inside a captured iteration");
  if (!(c->valid & qbit(GW_Q_P0_TAU))) return fail(c, GW_ERR_STATE, "no polarization P~0(tau) yet");
  const int ntau = c->ntau, nwb = c->nwb, naux = c->naux;
  const int64_t na2 = c->na2;
  if (tracelog_panel(naux) == 0) return fail(c, GW_ERR_ARG, "naux too large for the trace-log kernel");
  cudaStream_t st = c->st;
  // Matsubara-sum weights w_m = sum_j lb_j TBb[j][m]
  std::vector<double> lb((size_t)ntau);
  std::vector<double2> TB((size_t)ntau * nwb);
  CK(cudaMemcpyAsync(lb.data(), c->lb, (size_t)ntau * 8, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(TB.data(), c->TBb, TB.size() * 16, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  std::vector<double2> w((size_t)nwb, make_double2(0, 0));
  for (int j = 0; j < ntau; ++j)
    for (int m = 0; m < nwb; ++m) {
      w[(size_t)m].x += lb[(size_t)j] * TB[(size_t)j * nwb + m].x;
      w[(size_t)m].y += lb[(size_t)j] * TB[(size_t)j * nwb + m].y;
    }
  // P~0(i Omega) of a block of q per pass, factored in place
  const int nq = c->q1 - c->q0;
  const size_t per_q = (size_t)nwb * na2 * 16;
  int64_t qb = (int64_t)(opt_budget((size_t)4 << 30) / per_q);
  if (qb > nq) qb = nq;
  if (qb < 1) qb = 1;
  double2* ws = nullptr;
  while (!(ws = (double2*)dalloc(c, (size_t)qb * per_q)) && qb > 1) qb /= 2;
  double2* f = (double2*)dalloc(c, (size_t)nq * nwb * 16 + 16);
  if (!ws || !f) {
    dfree(c, ws); dfree(c, f);
    return fail(c, GW_ERR_OOM, "no room for the trace-log workspace");
  }
  int* flag = (int*)(f + (size_t)nq * nwb);
  gw_status s = GW_OK;
  cudaError_t e = cudaMemsetAsync(flag, 0, 4, st);
  for (int qa = c->q0; qa < c->q1 && e == cudaSuccess; qa += (int)qb) {
    const int64_t nb = std::min<int64_t>(qb, c->q1 - qa);
    e = transform(c, c->TFb, c->P0_tau + (size_t)qa * ntau * na2, ws, nwb, na2, nb, (int64_t)ntau * na2,
                  (int64_t)nwb * na2);
    if (e == cudaSuccess) {
      e = lu_tracelog(ws, naux, nb * nwb, na2, f + (size_t)(qa - c->q0) * nwb, flag, st);
      count(1);
    }
  }
  std::vector<double2> fh((size_t)nq * nwb);
  int hflag = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(fh.data(), f, fh.size() * 16, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaMemcpyAsync(c->h_scr, flag, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e == cudaSuccess) memcpy(&hflag, c->h_scr, 4);
  dfree(c, ws);
  dfree(c, f);
  if (e != cudaSuccess) return fail(c, GW_ERR_CUDA, cudaGetErrorString(e));
  if (hflag & 1) return fail(c, GW_ERR_SINGULAR, "zero pivot in the trace-log of I - P~0");
  if (hflag & 2)
    return fail(c, GW_ERR_SINGULAR, "pivot with non-positive real part: I - P~0 is not positive definite");
  double re = 0.0;
  for (int q = 0; q < nq; ++q)
    for (int m = 0; m < nwb; ++m) {
      const double2 v = fh[(size_t)q * nwb + m], ww = w[(size_t)m];
      re += ww.x * v.x - ww.y * v.y;
    }
  *phi = re / (2.0 * c->nk);
  return s;
}

// The k-points per launch that a 16-bit context of these sizes uses (host only).
extern "C" int gwdbg_chain_pbatch(int nao, int naux, int nk, int ntau) {
  return chain_pbatch(nao, naux, nk, ntau);
}

// Caps the number of k-points per launch of the 16-bit chains in contexts created
// afterwards (0: no cap); returns the old cap.
extern "C" int gwdbg_set_pbatch_cap(int cap) {
  const int old = g_pbatch_cap;
  g_pbatch_cap = cap < 0 ? 0 : cap;
  return old;
}

// Caps the number of k-points whose last P~0 step runs as one GEMM in contexts created
// afterwards (0: no cap); returns the old cap.
extern "C" int gwdbg_set_pgroup_cap(int cap) {
  const int old = g_pgroup_cap;
  g_pgroup_cap = cap < 0 ? 0 : cap;
  return old;
}
