// Internal declarations shared by the library's translation units.
// Complex numbers are interleaved (re, im) pairs: double2 / float2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>
#include <string>
#include <vector>
#include "../../include/gwgb.h"

namespace gwk {

// ------------------------------------------------------------------ complex helpers
template <typename T> struct cplx;
template <> struct cplx<double> { using t = double2; };
template <> struct cplx<float>  { using t = float2; };

__host__ __device__ inline double2 mk(double r, double i) { return make_double2(r, i); }
__host__ __device__ inline float2  mkf(float r, float i) { return make_float2(r, i); }

// ------------------------------------------------------------------ generic strided contraction
// C(m,n) = alpha * sum_k opA(A(m,k)) * opB(B(k,n)) + beta * C(m,n), batched.
// Each of m, n, k (and the batch index z) is split into an outer and an inner
// part, idx = outer * inner_extent + inner, and the address of an element is
// outer * stride1 + inner * stride0.  This lets one kernel read every tensor
// slice of the method (transposed blocks, (Q,i) row pairs, ...) in place.
struct Idx2 {
  int64_t inner;   // inner extent (>= 1)
  int64_t s1, s0;  // strides of outer and inner part, in complex elements
};
struct GettDesc {
  int64_t M, N, K, Z;       // Z = batch count
  Idx2 am, ak, az;          // A(m, k) in batch z
  Idx2 bk, bn, bz;          // B(k, n)
  Idx2 cm, cn, cz;          // C(m, n)
  bool conjA, conjB;
  double2 alpha, beta;      // beta == 0 -> C is not read
  int ksplit;               // > 1: deterministic split-K through a workspace
};

// element type tags for the contraction kernels
enum class Ty : int { C64 = 0, C128 = 1 };

// Launch a contraction.  ta/tb/tc: storage types of A, B, C.  acc: accumulate
// in double (C128) or float (C64).  ws: workspace for split-K (may be null
// when ksplit == 1); returns cudaError_t.
cudaError_t gett(const GettDesc& d, const void* A, Ty ta, const void* B, Ty tb, void* C, Ty tc,
                 Ty acc, void* ws, size_t ws_bytes, cudaStream_t st);
size_t gett_ws_bytes(const GettDesc& d, Ty acc);

inline Idx2 I1(int64_t s0) { return Idx2{INT64_MAX / 4, 0, s0}; }          // plain index
inline Idx2 I2(int64_t inner, int64_t s1, int64_t s0) { return Idx2{inner, s1, s0}; }

// ------------------------------------------------------------------ other kernels
cudaError_t herm_batched(double2* X, int64_t n, int64_t count, int64_t stride, cudaStream_t st);
// out[m] = tr ln(I - A_m) + tr A_m for `count` n x n matrices A_m spaced `stride` apart
// (overwritten), by FP64 LU without row exchanges; flag |= 1 (zero pivot), 2 (pivot with
// non-positive real part).  tracelog_panel(n) == 0: n too large for the shared-memory panel.
int tracelog_panel(int n);
cudaError_t lu_tracelog(double2* A, int n, int64_t count, int64_t stride, double2* out, int* flag, cudaStream_t st);
size_t grid_ws_bytes(int ntau, const int* fn_host, const int* bm_host, int* ld_out);
cudaError_t grid_build_ws(int ntau, double beta, const int* d_fn, const int* d_bm, int ld, void* ws,
                          double* tau, double2* TFf, double2* TFb, double* lb, double* l0, cudaStream_t st);
cudaError_t density_weights(int ntau, int nwf, const double* lb, const double2* TBf, double2* r, cudaStream_t st);
cudaError_t fermi_freqs(int nwf, double beta, const int* fn, double* wn, cudaStream_t st);
cudaError_t invert_small_gj(double2* A, int n, int* d_info, cudaStream_t st);
cudaError_t screened_inplace(double2* P, int64_t n, int64_t count, double2* work, size_t work_bytes,
                             int* d_info, cudaStream_t st);
size_t screened_work_bytes(int64_t n, int64_t count);
// complex64 inversion + nsteps Newton steps with FP64-accurate residuals (k_solve.cu)
size_t screened_refine_bytes(int64_t n, int64_t chunk);
bool screened_refine_ok(int64_t n);
cudaError_t screened_refine(double2* X, int64_t n, int64_t count, void* work, size_t work_bytes, int nsteps,
                            int* d_info, int* d_err, cudaStream_t st, int64_t* nlaunch);

struct DysonArgs {
  int nao, nk, nw;
  const double2* H0; const double2* S; const double2* Sinf; const double2* Siw; // Siw [nw][nk][nao2]
  const double* wn;      // fermionic frequencies [nw]
  const double2* r;      // density weights [nw] (complex)
  double spin;
};
cudaError_t dyson_eval(const DysonArgs& a, const double* mu_ptr, double2* G_out, double* partial,
                       const int* done_flag, int* d_info, cudaStream_t st);
struct MuState {
  double lo, hi, Nlo, Nhi, x, Nx, target, tol, width;
  int phase, iter, maxit, done, status;
  double flo, fhi;   // Illinois-weighted N - target at the bracket ends
  int side;          // which end moved last (-1 lo, +1 hi, 0 none)
};
cudaError_t mu_step(MuState* s, const double* partial, int64_t count, double scale, cudaStream_t st);
cudaError_t dyson_tangent_rhs(const double2* dSinf, const double2* dSiw, double2* D, int64_t nk, int64_t n2,
                              int64_t nw, cudaStream_t st);
cudaError_t dyson_tangent_finish(const double2* X, const double2* Y, const double2* S, const double2* r, int nao,
                                 int nk, int nw, double* part, double* dmu, double2* dG, cudaStream_t st);
int rdot_blocks(int64_t n);
cudaError_t rdot_partials(const double2* a, const double2* b, int64_t n, double* part, cudaStream_t st);
size_t dyson_smem(int nao, int nt);
cudaError_t mu_init_device(MuState* s, double target, double tol, double width, int maxit, cudaStream_t st);

cudaError_t density_gamma(const double2* G_tau, const double* lb, double2* gamma, int ntau, int64_t nelem,
                          cudaStream_t st);
cudaError_t hartree_t(const double2* V, const double2* gamma, double2* t, int nk, int naux, int nao,
                      cudaStream_t st);
cudaError_t hartree_j(const double2* V, const double2* t, double2* J, int nk, int naux, int nao, double fac,
                      cudaStream_t st);
cudaError_t axpby(double2* y, const double2* x, double a, double b, int64_t n, cudaStream_t st);
cudaError_t identity_minus(double2* X, int64_t n, int64_t count, double sign, cudaStream_t st);
cudaError_t check_v_pairing(const double2* V, int nk, int naux, int nao, double* d_maxdev, cudaStream_t st);
cudaError_t check_herm(const double2* X, int64_t n, int64_t count, double* d_maxdev, cudaStream_t st);
cudaError_t maxabs_diff(const double2* a, const double2* b, int64_t n, double* d_out, cudaStream_t st);
cudaError_t to_c64(const double2* x, float2* y, int64_t n, cudaStream_t st);
cudaError_t check_trs(const double2* X, int64_t nslab, int64_t len, const int* partner, double* d_out,
                      cudaStream_t st);
cudaError_t conj_fill(double2* X, int64_t outer, int nk, int64_t inner, const int* src, const int* need,
                      cudaStream_t st);

// ------------------------------------------------------------------ batched small products (k_bsm.cu)
// C[g][e] = alpha * A[g][e] * B[g][e] (complex64), M, N, K <= 64; element (r, c) of
// an operand at base + r*rs + c*cs (complex units); A or B may be shared by all e.
// Output: complex64 C (C != null) or TF32 hi/lo float planes Chi/Clo (complex index o
// -> floats 2o, 2o+1); C element (m, n) at g*c_gs + e*c_es + m*c_rs + n.
struct BsmDesc {
  int M, N, K;
  int64_t G, E;
  int per_block;
  const float2* A; int64_t a_gs, a_es, a_rs, a_cs; int a_shared, conjA;
  const float2* B; int64_t b_gs, b_es, b_rs, b_cs; int b_shared, conjB;
  float2* C; float* Chi; float* Clo; int64_t c_gs, c_es, c_rs;
  float alpha;
};
cudaError_t bsm(const BsmDesc& d, cudaStream_t st);

// ------------------------------------------------------------------ tensor-core split-TF32 GEMM
// Source matrices of one batched operand-preparation launch: entry i reads at src + off[i]
// (complex elements) and writes its output block i (up to kSrcListMax entries).
constexpr int kSrcListMax = 32;
struct SrcList {
  int n;
  int64_t off[kSrcListMax];
};
// copies n blocks (block_bytes of hi and of lo pieces, ecount exponents each) from block
// indices idx[i] of the sources into consecutive blocks of the destinations
cudaError_t gather_blocks(const void* shi, const void* slo, const int* se, void* dhi, void* dlo, int* de,
                          int64_t block_bytes, int64_t ecount, const int* idx, int n, cudaStream_t st);
cudaError_t half_rows_multi(const double2* src, const int64_t* offs, int n, int64_t rows, int64_t K, int64_t ld,
                            bool conj, void* hi, void* lo, int64_t Kpad, int64_t ldo, int64_t dstride, int fmt,
                            int* ex, int* exs, int64_t estride, cudaStream_t st);
cudaError_t half_embed_conj_multi(const double2* src, const int64_t* offs, int n, int64_t rows, int64_t K, void* hi,
                                  void* lo, int64_t Kpad, int64_t ldo, int64_t dstride, int fmt, const int* ex,
                                  cudaStream_t st);
cudaError_t half_embed_t_multi(const double2* src, const int64_t* offs, int n, int64_t K, int64_t N, void* hi,
                               void* lo, int64_t Kpad, int64_t dstride, int fmt, int e, cudaStream_t st,
                               int64_t kin = 0, int64_t kout = 0);
struct UmmaOperand {
  const float* hi;
  const float* lo;
  int64_t rows, batch;   // rows per batch, batch count (1 = shared by all z)
  int64_t ld, bs;        // row stride and batch stride in elements
  int f16 = 0;           // 1: hi/lo hold fp16 pieces, 2: bf16 pieces (cast pointers), K and strides in
                         // 16-bit elements
};
// ksplit > 1: the K range is split over blocks and partial results are added to
// an fp64 C with atomics (requires accumulate).  row_inner > 0: output row m =
// o * row_inner + i is written at o * row_s1 + i * c_ld (real elements); col_inner
// > 0: column n = o * col_inner + i at o * col_s1 + i.  C_lo != null: fp32 output
// written as TF32 hi (C) / lo (C_lo) planes.
// kvalid > 0: real K extent holding data (the rest of Kpad is zero padding in both
// operands); the persistent kernel skips whole K = 8 steps of that padding.
// scale != null (persistent kernel only): D[m][n] is multiplied by
// 2^(eA[z*ea_zs + m] + eB[z*eb_zs + n/2] + eshift) before it is added or stored; fp16
// operands require it (their rows are stored with power-of-two scales).
struct UmmaScale {
  const int* eA;
  const int* eB;
  int64_t ea_zs, eb_zs;
  int eshift;
  int64_t ea_div = 1, eb_div = 1;   // row m uses eA[z*ea_zs + m/ea_div], column n eB[z*eb_zs + (n/2)/eb_div]
  int64_t ea_mod = 0;               // > 0: row m uses eA[z*ea_zs + (m/ea_div) % ea_mod]
};
// 16-bit pieces as the output of a GEMM (C: hi, C_lo: lo, fp32-class layout in 16-bit
// elements): D * 2^-(eO[z*eo_zs + m/eo_div] + eo_shift) in fp16 (half = 1) or bf16 (2)
struct UmmaOut {
  int half;
  const int* eO;
  int64_t eo_zs, eo_div;
  int eo_shift;
};
// Two-level batches (several k-points of a chain step in one launch): batch entry
// z = zo * zin + zi; the TMA batch coordinate of A is zo * za_o + zi * za_i (B likewise),
// and the exponent and output strides of the other arguments (ea_zs, eb_zs, eo_zs, c_zs)
// apply to zi while ea_zso, eb_zso, eo_zso, c_zso apply to zo.
struct UmmaZ {
  int zin;
  int za_o, za_i, zb_o, zb_i;
  int64_t ea_zso, eb_zso, eo_zso, c_zso;
};
cudaError_t umma_gemm(const UmmaOperand& A, const UmmaOperand& B, int M, int N, int64_t Kpad, int batch, void* C,
                      bool c_fp64, double alpha, bool accumulate, int64_t c_ld, int64_t c_zs, int nseg, int* err,
                      cudaStream_t st, int ksplit = 1, int64_t row_inner = 0, int64_t row_s1 = 0,
                      int64_t col_inner = 0, int64_t col_s1 = 0, float* C_lo = nullptr,
                      const UmmaScale* scale = nullptr, int64_t kvalid = 0, const UmmaOut* out = nullptr,
                      const UmmaZ* zz = nullptr);
// FP64 complex products on tensor cores by exact digit splitting (k_emul.cu)
int64_t emul_kpad(int64_t K);
size_t emul_digit_bytes(int64_t rows, int64_t K);
// digit planes are fp16 arrays (emul_digit_bytes), passed as untyped pointers
cudaError_t emul_split_b(const double2* B, int64_t rows, int64_t K, int64_t ldb, void* dig, int* ex, cudaStream_t st);
cudaError_t emul_transform(const void* Bd, const int* Be, int64_t nrow, const double2* X, int64_t K, int64_t ncol,
                           int64_t ldx, double2* Y, int64_t ldy, void* Ad, int* Ae, int* err, cudaStream_t st);
// tensor-core launches of one product with complex K and nd digits (-1: K too large)
int emul_launches(int64_t K, int nd = 8);
cudaError_t emul_split_rows(const double2* A, int64_t count, int64_t M, int64_t K, int64_t lda, int64_t sa,
                            void* Ad, int* Ae, cudaStream_t st);
cudaError_t emul_split_cols(const double2* B, int64_t count, int64_t K, int64_t N, int64_t ldb, int64_t sb,
                            void* Bd, int* Be, cudaStream_t st);
cudaError_t emul_cgemm_batched(const void* Ad, const int* Ae, const void* Bd, const int* Be, int64_t count,
                               int64_t M, int64_t N, int64_t K, double2* C, int* err, cudaStream_t st, int nd = 8);

// ldo: row stride of the output planes (0: Kpad)
cudaError_t split_rows(const void* src, bool src_c128, int64_t rows, int64_t K, int64_t ld, bool conj, float* hi,
                       float* lo, int64_t Kpad, cudaStream_t st, int64_t ldo = 0);
cudaError_t embed_conj(const void* src, bool src_c128, int64_t rows, int64_t K, float* hi, float* lo, int64_t Kpad,
                       cudaStream_t st, int64_t ldo = 0);
cudaError_t embed_t(const void* src, bool src_c128, int64_t K, int64_t N, float* hi, float* lo, int64_t Kpad,
                    cudaStream_t st);
// fp16 pieces with one power-of-two exponent per (complex) row; Kpad a multiple of 64
cudaError_t split_rows_f16(const void* src, bool src_c128, int64_t rows, int64_t K, int64_t ld, bool conj, void* hi,
                           void* lo, int64_t Kpad, int* ex, cudaStream_t st);
cudaError_t embed_conj_f16(const void* src, bool src_c128, int64_t rows, int64_t K, void* hi, void* lo, int64_t Kpad,
                           int* ex, cudaStream_t st);
cudaError_t embed_t_batched(const void* src, bool src_c128, int64_t count, int64_t K, int64_t N, int64_t ld,
                            int64_t zs, float* hi, float* lo, int64_t Kpad, int64_t ds, cudaStream_t st);
cudaError_t embed_conj_batched(const double2* src, int64_t count, int64_t ss, int64_t rows, int64_t K, float* hi,
                               float* lo, int64_t Kpad, int64_t ds, cudaStream_t st);
cudaError_t embed_plain_batched(const double2* src, int64_t count, int64_t ss, int64_t rows, int64_t K, float* hi,
                                float* lo, int64_t Kpad, int64_t ds, cudaStream_t st);

// ------------------------------------------------------------------ 16-bit operand pieces (k_half.cu)
// fmt: 1 fp16, 2 bf16.  Element offsets and Kpad / ldo / ds in 16-bit elements (Kpad a multiple of 64).
cudaError_t half_rows(const double2* src, int64_t rows, int64_t K, int64_t ld, bool conj, void* hi, void* lo,
                      int64_t Kpad, int64_t ldo, int fmt, int* ex, int* exs, cudaStream_t st);
cudaError_t half_embed_conj(const double2* src, int64_t rows, int64_t K, void* hi, void* lo, int64_t Kpad,
                            int64_t ldo, int fmt, const int* ex, cudaStream_t st);
// kin > 0: source row k lands at K index (k % kin) * kout + k / kin (a K order permuted from
// (outer, inner) to (inner, outer))
cudaError_t half_embed_t(const double2* src, int64_t K, int64_t N, void* hi, void* lo, int64_t Kpad, int fmt, int e,
                         cudaStream_t st, int64_t kin = 0, int64_t kout = 0);
cudaError_t half_embed_mats(const double2* src, int64_t count, int64_t ss, int64_t rows, int64_t K, void* hi,
                            void* lo, int64_t Kpad, int64_t ds, int fmt, bool plain, int* ex, cudaStream_t st);
cudaError_t v_norms(const double2* V, int64_t nslab, int naux, int nao, float* vmax, float* vrs, cudaStream_t st);
cudaError_t g_norms(const double2* G, int ntau, int nk, int nao, float* gmax, float* grs, cudaStream_t st);
cudaError_t polar_exps(const float* vrs, const float* gmax_p, const float* grs_m, int ntau, int naux, int* eY, int* eZ,
                       cudaStream_t st);
cudaError_t sigma_exps(const int* eX, int shift, const float* grs, int ntau, int naux, int* eY3, cudaStream_t st);
cudaError_t max_exp(const float* v, int n, int* out, cudaStream_t st);
cudaError_t row_exps(const float* v, int n, int* out, cudaStream_t st);

}  // namespace gwk
