/*
 * gwgb.h -- C ABI of a single-GPU (GB300, sm_103a) library for fully
 * self-consistent finite-temperature GW in Gaussian Bloch orbitals with
 * density-fitted Coulomb integrals (Yeh, Iskakov, Zgid, Gull, "Fully
 * Self-Consistent Finite-Temperature GW in Gaussian Bloch Orbitals for
 * Solids").
 *
 * Data conventions
 *   - Complex arrays are interleaved (re, im) IEEE doubles, row-major.
 *   - nk = kmesh[0]*kmesh[1]*kmesh[2]; k = (i1*kmesh[1] + i2)*kmesh[2] + i3
 *     (Gamma-centred mesh); k+q and k-q are taken componentwise modulo the mesh.
 *   - nwf, nwb: sampled fermionic / bosonic Matsubara points.  With gw_init both
 *     equal ntau; with gw_init_grid they are the caller's grid's.
 *   - Layouts:  H0, S, Sigma_inf, gamma          [nk][nao][nao]
 *               V^{k k'}_{ij}(Q)                 [nk][nk][naux][nao][nao]
 *               G, Sigma~ (tau)                  [ntau][nk][nao][nao]
 *               G, Sigma~ (i w)                  [nwf][nk][nao][nao]
 *               P~0, P~ (tau)                    [nq = nk][ntau][naux][naux]
 *               P~0, P~ (i Omega)                [nq][nwb][naux][naux]
 *   - gw_init's tau grid is the first-kind Chebyshev roots on [0, beta]; a
 *     function of tau is represented by the interpolating polynomial through its
 *     node values.  The forward transform is the exact Fourier integral of that
 *     interpolant at the sampled frequencies (Eq. tau_to_iw); the backward
 *     transform is its exact inverse (stand-in for Eq. iw_to_tau).  gw_init_grid
 *     takes any sparse-sampling grid instead (the paper's IR basis, Sec.
 *     "Representation on the imaginary axes").
 *
 * Ownership and errors
 *   - Inputs are copied during gw_init (device pointers with GW_INPUT_DEVICE;
 *     with GW_BORROW_V the V tensor is referenced, not copied, and must
 *     outlive the context).  The caller keeps ownership of its buffers.
 *   - Device memory comes from cfg->dev_alloc / dev_free when given (for
 *     instance PyTorch's caching allocator), else from cudaMalloc / cudaFree.
 *   - All work is enqueued on cfg->stream.  Calls that return a status which
 *     depends on device results (gw_init's input checks, gw_dyson,
 *     gw_screened, gw_iterate) synchronise that stream.
 *   - No call aborts, traps or throws across the ABI.  On failure a call
 *     returns a non-zero gw_status and gw_last_error() gives a message.
 *   - A context is used by one host thread at a time.
 */
#ifndef GWGB_H
#define GWGB_H
#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct gw_ctx gw_ctx;

typedef enum {
  GW_OK = 0,
  GW_ERR_ARG = 1,            /* bad size, null pointer, input fails a check     */
  GW_ERR_CUDA = 2,           /* a CUDA runtime call failed                      */
  GW_ERR_OOM = 3,            /* device allocation failed                        */
  GW_ERR_NOT_CONVERGED = 4,  /* chemical-potential search hit its step cap      */
  GW_ERR_SINGULAR = 5,       /* zero pivot in a Dyson or screened-solve inverse */
  GW_ERR_TIMEOUT = 6,        /* a bounded device wait gave up                   */
  GW_ERR_STATE = 7,          /* call out of order (e.g. no G yet)               */
  GW_ERR_INTERNAL = 8
} gw_status;

/* Number format of the two dominant contractions (P~0 and Sigma~). */
typedef enum {
  GW_FP64 = 0,        /* complex128 throughout                                  */
  GW_FP32 = 1,        /* complex64 products, fp32 accumulation per k-slab,
                         fp64 accumulation across slabs                         */
  GW_SPLIT_BF16 = 2,  /* every GEMM of both chains on tcgen05 tensor cores (kind::f16) with
                         x = hi + lo bf16 pieces (16 significant bits; hi*hi + hi*lo + lo*hi,
                         fp32 accumulation, fp64 accumulation across (q, k) slabs); chain
                         intermediates are written by the GEMMs as bf16 pieces             */
  GW_SPLIT_TF32 = 3,  /* the dominant GEMM of each contraction on tcgen05 tensor cores with
                         x = hi + lo TF32 splits (hi*hi + hi*lo + lo*hi, fp32 accumulation,
                         fp64 accumulation across (q, k) slabs); other steps as GW_FP32 */
  GW_SPLIT_F16 = 4    /* as GW_SPLIT_BF16 with fp16 pieces (22 significant bits, the accuracy
                         of the TF32 split at twice its tensor rate and half its operand
                         bytes); every operand row carries a power-of-two scale taken from
                         an upper bound of its values (norms of V per auxiliary index and
                         of G per tau), applied exactly in the GEMM epilogues            */
} gw_precision;

enum {
  GW_INPUT_DEVICE = 1u << 0, /* H0, S, V passed to gw_init are device pointers   */
  GW_BORROW_V     = 1u << 1, /* with GW_INPUT_DEVICE: use V in place, no copy     */
  GW_SKIP_CHECKS  = 1u << 2, /* skip the Hermiticity / pairing checks of gw_init  */
  GW_SMALL_TENSOR = 1u << 3, /* GW_SPLIT_TF32, nao <= 64: the nao-sized steps of the
                                P~0 / Sigma~ chains also on tensor cores (split TF32)  */
  GW_SMALL_SIMT   = 1u << 4, /* GW_SPLIT_TF32, nao <= 64: those steps on the FP32
                                SIMT small-product kernel.  Neither flag: library default */
  GW_FP64_NATIVE  = 1u << 5, /* FP64 SIMT arithmetic for the tau <-> i nu transforms
                                and the screened solve, instead of the defaults:
                                FP64-accurate digit-split products on the tensor cores
                                and a complex64 inversion refined to FP64 accuracy    */
  GW_TRS          = 1u << 6  /* the system is time-reversal symmetric: H0(-k) =
                                conj H0(k), S(-k) = conj S(k), V^{-k,-k'}(Q) =
                                conj V^{kk'}(Q) (checked by gw_init unless
                                GW_SKIP_CHECKS; GW_ERR_ARG otherwise).  Then
                                G^{-k} = conj G^k, P~0^{-q} = conj P~0^q, P~^{-q} =
                                conj P~^q and Sigma~^{-k} = conj Sigma~^k hold
                                exactly on the discrete grid, and gw_polarization,
                                gw_screened and gw_selfenergy compute only the q (k)
                                with index(-q) >= q (the inversion-symmetry reduction
                                of the q-points, Sec. "GPU performance") and fill the
                                others by conjugation.  Not applied while a q range
                                is set, nor to the tangents and adjoints.         */
};

typedef void* (*gw_alloc_fn)(void* user, size_t bytes);
typedef void (*gw_free_fn)(void* user, void* ptr);

typedef struct {
  int32_t nao;            /* orbitals per cell                                    */
  int32_t naux;           /* auxiliary (density-fitting) functions, Eq. U_decompose */
  int32_t kmesh[3];       /* Gamma-centred k-mesh                                 */
  int32_t ntau;           /* tau nodes = sampled Matsubara points                 */
  double beta;            /* inverse temperature (1/Ha)                           */
  double n_elec;          /* electrons per cell (half filling: nao)               */
  double mu_tol;          /* |N(mu) - n_elec| threshold; the paper uses 1e-9      */
  int32_t mu_maxit;       /* cap on N(mu) evaluations -> GW_ERR_NOT_CONVERGED     */
  double damping;         /* alpha of Sigma <- (1-alpha) Sigma_old + alpha Sigma_new */
  int32_t contract_prec;  /* gw_precision of the P~0 and Sigma~ contractions       */
  int32_t spin_factor;    /* s = 2 for a spin-restricted closed shell             */
  const int32_t* fermi_n; /* [ntau] host: sampled fermionic n, w_n = (2n+1) pi/beta */
  const int32_t* bose_m;  /* [ntau] host: sampled bosonic m, Omega_m = 2 m pi/beta  */
  void* stream;           /* cudaStream_t; NULL = legacy default stream           */
  gw_alloc_fn dev_alloc;  /* optional device allocator                            */
  gw_free_fn dev_free;
  void* alloc_user;
  uint64_t flags;         /* GW_INPUT_DEVICE | GW_BORROW_V | GW_SKIP_CHECKS |
                             GW_SMALL_TENSOR | GW_SMALL_SIMT | GW_FP64_NATIVE |
                             GW_TRS                                                 */
} gw_config;

/* Quantities readable with gw_get / writable with gw_set.  Sizes in bytes. */
typedef enum {
  GW_Q_G_TAU = 0,      /* [ntau][nk][nao][nao] c128  (get, set)                 */
  GW_Q_G_IW = 1,       /* [nwf][nk][nao][nao]  c128  (get)                      */
  GW_Q_SIGMA_INF = 2,  /* [nk][nao][nao]       c128  (get, set) static part      */
  GW_Q_SIGMA_TAU = 3,  /* [ntau][nk][nao][nao] c128  (get, set)                 */
  GW_Q_SIGMA_IW = 4,   /* [nwf][nk][nao][nao]  c128  (get, set) dynamic part     */
  GW_Q_P0_TAU = 5,     /* [nq][ntau][naux][naux] c128 (get, set)                */
  GW_Q_P0_IW = 6,      /* [nq][nwb][naux][naux] c128 (get, set); overwritten by
                          gw_screened, which leaves P~(i Omega) in its place    */
  GW_Q_P_IW = 7,       /* same buffer as GW_Q_P0_IW after gw_screened (get)     */
  GW_Q_P_TAU = 8,      /* [nq][ntau][naux][naux] c128 (get, set)                */
  GW_Q_GAMMA = 9,      /* [nk][nao][nao] c128 density matrix (get)              */
  GW_Q_MU = 10,        /* double (get, set)                                     */
  GW_Q_TFF = 11,       /* [nwf][ntau] c128 fermionic tau -> i w   (get)         */
  GW_Q_TBF = 12,       /* [ntau][nwf] c128 fermionic i w -> tau   (get)         */
  GW_Q_TFB = 13,       /* [nwb][ntau] c128 bosonic tau -> i Omega (get)         */
  GW_Q_TBB = 14,       /* [ntau][nwb] c128 bosonic i Omega -> tau (get)         */
  GW_Q_LB = 15,        /* [ntau] double  L_j(beta^-)             (get)          */
  GW_Q_TAU = 16,       /* [ntau] double  tau nodes               (get)          */
  GW_Q_N_ELEC = 17,    /* double electron count at the last mu   (get)          */
  GW_Q_SIGMA_INF_NEW = 18 /* [nk][nao][nao] c128 last HF result before mixing (get) */
} gw_quantity;

typedef struct {
  double mu;          /* chemical potential after the iteration               */
  double n_elec;      /* N(mu) reached                                        */
  int32_t mu_steps;   /* N(mu) evaluations of the search                      */
  double max_dG;      /* max |G_new(tau) - G_old(tau)|                        */
  double max_dSigma;  /* max |Sigma~_new(i w) - Sigma~_old(i w)| before mixing */
  float ms_total;     /* device time of the iteration                         */
  float ms_polarization, ms_screened, ms_selfenergy, ms_dyson, ms_hf;
} gw_iter_stats;

/* A sparse-sampling grid supplied by the caller (host arrays, read during
 * gw_init_grid only): the paper represents functions of tau and i w on the IR
 * basis and samples them at points of that basis (Sec. "Representation on the
 * imaginary axes"); any grid with the same structure works.  A function X of tau
 * is given by its values at the ntau points; X(i w_n) = sum_j TFf[n][j] X(tau_j)
 * at the nwf fermionic points, X(tau_j) = sum_n TBf[j][n] X(i w_n) back (and TFb,
 * TBb at the nwb bosonic points); X(beta^-) = sum_j lb[j] X(tau_j) gives the
 * density matrix.  Complex matrices are interleaved (re, im) doubles, row-major. */
typedef struct {
  int32_t ntau;            /* tau points (must equal the config's ntau)            */
  int32_t nwf, nwb;        /* fermionic / bosonic Matsubara points                  */
  const double* tau;       /* [ntau] in [0, beta]                                   */
  const int32_t* fermi_n;  /* [nwf] w_n = (2n+1) pi / beta (distinct)               */
  const int32_t* bose_m;   /* [nwb] Omega_m = 2 m pi / beta (distinct)              */
  const double* TFf;       /* [nwf][ntau] complex                                   */
  const double* TBf;       /* [ntau][nwf] complex                                   */
  const double* TFb;       /* [nwb][ntau] complex                                   */
  const double* TBb;       /* [ntau][nwb] complex                                   */
  const double* lb;        /* [ntau] real                                           */
} gw_grid;

/* Create a context: validates sizes (nao <= 96, the Dyson kernel's bound; GW_ERR_ARG
 * otherwise), copies H0, S (Eq. scalar_S) and V (Eq. U_decompose), builds the tau
 * grid, the transform matrices and the density weights on the device.  Unless
 * GW_SKIP_CHECKS, rejects with GW_ERR_ARG inputs where H0 or S is not Hermitian or
 * V^{k'k}(Q) != V^{kk'}(Q)^H beyond 1e-10 relative.  Synchronises cfg->stream.
 * *out is NULL on failure. */
gw_status gw_init(const gw_config* cfg, const double* H0, const double* S, const double* V,
                  gw_ctx** out);

/* gw_init on the caller's sampling grid instead of the Chebyshev grid (the
 * config's fermi_n / bose_m are then ignored).  GW_ERR_ARG for a null array, a
 * grid whose ntau differs from the config's, or repeated Matsubara indices. */
gw_status gw_init_grid(const gw_config* cfg, const gw_grid* grid, const double* H0, const double* S,
                       const double* V, gw_ctx** out);

/* Free every device buffer of the context (borrowed V excepted). */
gw_status gw_destroy(gw_ctx* ctx);

/* Copy a quantity in (gw_set) or out (gw_get).  `bytes` must equal the size
 * listed for it in gw_quantity.  on_device != 0: src/dst is a device pointer.
 * gw_get synchronises the stream when dst is a host pointer.  gw_get returns
 * GW_ERR_STATE for a quantity that neither gw_set nor the call computing it
 * has written yet (Sigma_inf, Sigma(i w), the grid and the transforms are
 * defined from gw_init on; P~0(i Omega) stops being readable once gw_screened
 * has replaced it by P~(i Omega)). */
gw_status gw_set(gw_ctx* ctx, gw_quantity which, const void* src, size_t bytes, int on_device);
gw_status gw_get(gw_ctx* ctx, gw_quantity which, void* dst, size_t bytes, int on_device);

/* Static self-energy (Sec. "Hartree-Fock self-energy"): gamma^k = -G^k(beta^-)
 * from the current G(tau), then Sigma_inf = J + K (Eqs. HF_J, HF_K), stored as
 * GW_Q_SIGMA_INF_NEW.  Requires G. */
gw_status gw_hf(gw_ctx* ctx);

/* P~0^q(tau) for all q (Eq. tilde_P0_tau; P~0 = (s/Nk) sum V G^{k+q}(tau) V
 * G^k(-tau), G(-tau) = -G(beta - tau)), Hermitian-symmetrised, then its bosonic
 * transform P~0^q(i Omega_m) (Eq. P0t_to_P0w).  Requires G. */
gw_status gw_polarization(gw_ctx* ctx);

/* Screened solve P~ = [I - P~0(i Omega)]^{-1} P~0(i Omega) for every (q, m)
 * (Eq. tilde_P_omega), then P~^q(tau) (Eq. Piw_to_Pt), Hermitian-symmetrised.
 * FP64-accurate either way: by default Y = (I - P~0)^{-1} is inverted in complex64
 * on the tensor cores and refined by two Newton steps Y <- Y + Y (I - (I - P~0) Y)
 * whose residual products are exact digit-split GEMMs; GW_FP64_NATIVE (or naux >
 * 512, or no room for the refinement workspace) inverts in FP64 arithmetic.
 * Returns GW_ERR_SINGULAR on a zero pivot, GW_ERR_TIMEOUT when a tensor-core wait
 * gave up.  Synchronises. */
gw_status gw_screened(gw_ctx* ctx);

/* Sigma~^k(tau) = -(1/Nk) sum_q sum V^{k,k-q} G^{k-q}(tau) P~^q(tau) V^{k-q,k}
 * (Eq. tilde_sigma2), symmetrised, its fermionic transform Sigma~(i w), and the
 * static part of gw_hf.  The self-energy used by the next gw_dyson becomes
 * (1-damping) Sigma_old + damping Sigma_new when an earlier self-energy exists
 * (else Sigma_new).  Requires G and P~(tau). */
gw_status gw_selfenergy(gw_ctx* ctx);

/* The two halves of gw_selfenergy, for a q range split over several contexts
 * (one per GPU, Sec. "GPU acceleration": the q-points are distributed and the
 * self-energy is reduced over them).  gw_selfenergy_partial computes
 * Sigma~^k(tau) summed over the context's q range only (Eq. tilde_sigma2),
 * symmetrised, into GW_Q_SIGMA_TAU; the caller adds the partial sums of all
 * contexts (Sigma~ is a sum over q) and writes the total back with gw_set.
 * gw_selfenergy_finish then computes the static part (as gw_hf), Sigma~(i w)
 * from GW_Q_SIGMA_TAU (Eq. tau_to_iw) and the damped update.  Requires G and
 * P~(tau) (partial) or Sigma~(tau) (finish); GW_ERR_STATE otherwise. */
gw_status gw_selfenergy_partial(gw_ctx* ctx);
gw_status gw_selfenergy_finish(gw_ctx* ctx);

/* Restrict the q-points of gw_polarization, gw_screened and the Sigma~
 * contraction (and of the tangents built on them) to [q0, q1), 0 <= q0 < q1 <=
 * nk; the default is every q.  P~0 and P~ of the other q are neither computed
 * nor read, and Sigma~(tau) becomes the partial sum over [q0, q1).  The
 * adjoints always run over every q.  Forgets the P~0 / P~ / Sigma~(tau) of
 * the previous range (GW_ERR_ARG for a bad range). */
gw_status gw_set_q_range(gw_ctx* ctx, int32_t q0, int32_t q1);

/* Dyson equation (Eq. Dyson) with chemical-potential search: a bracketing
 * search on N(mu) = (s/Nk) sum_k tr[gamma^k S^k] (the bracket [mu_prev - 1,
 * mu_prev + 1] widened until N - n_elec changes sign, then Illinois
 * regula-falsi steps with a plain bisection every fourth step) until
 * |N - n_elec| <= mu_tol and the bracket is below 1e-13, then G(i w) = [(i w + mu) S - H0 - Sigma_inf -
 * Sigma~(i w)]^{-1} and G(tau) (symmetrised).  With no self-energy set this is
 * the non-interacting G0.  Synchronises.  mu_out may be NULL. */
gw_status gw_dyson(gw_ctx* ctx, double* mu_out);

/* n_iter full GW iterations from the current G (computing G0 first when no G
 * exists): gw_hf, gw_polarization, gw_screened, gw_selfenergy, gw_dyson.
 * stats_out (may be NULL) receives the record of the last iteration. */
gw_status gw_iterate(gw_ctx* ctx, int32_t n_iter, gw_iter_stats* stats_out);

/* n_iter GW iterations replayed from a CUDA graph: the first call captures one
 * iteration (gw_polarization, gw_screened, gw_selfenergy and a device-side mu
 * search of min(mu_maxit, 96) bisection steps plus Dyson) on a private stream
 * of the context and later calls replay it, ordered after cfg->stream by
 * events.  Status checks are deferred to the end of the call (one
 * synchronisation).  A first, unmixed GW iteration is run uncaptured when no
 * self-energy exists yet.  stats_out (may be NULL) gets mu, n_elec, mu_steps
 * and the mean device time per replay in ms_total. */
gw_status gw_iterate_graph(gw_ctx* ctx, int32_t n_iter, gw_iter_stats* stats_out);

/* n_iter captured iterations of each of n independent systems (contexts of any
 * sizes): the systems' graphs are launched round-robin on their own streams so
 * the GPU overlaps them (the batching pattern of many uneven systems).
 * Synchronises every context at the end; on failure gw_last_error(NULL) names
 * the system. */
gw_status gw_batch_iterate(gw_ctx* const* ctxs, int32_t n, int32_t n_iter);

/* Drop the stored self-energy so that the next gw_selfenergy is not mixed. */
gw_status gw_reset_sigma(gw_ctx* ctx);

/* Checkpoint / resume of a self-consistent run.  gw_save_state writes the state
 * the next iteration starts from -- G(tau), Sigma_inf, Sigma~(i w), mu and whether
 * a self-energy exists (so damping resumes as it would have) -- to `path` (host
 * file, complex128 arrays after a fixed header, then a 64-bit FNV-1a hash of the
 * file's contents).  gw_load_state reads it into a context of the same sizes and
 * beta (GW_ERR_ARG on a mismatch, a missing, truncated or corrupt file); the next
 * gw_iterate continues exactly as the saved run would have.  P~0 and P~ are not
 * saved (they are recomputed from G).  Both synchronise the context's stream. */
gw_status gw_save_state(gw_ctx* ctx, const char* path);
gw_status gw_load_state(gw_ctx* ctx, const char* path);

/* Message of the last failure of this context (or of gw_init when ctx is NULL). */
const char* gw_last_error(const gw_ctx* ctx);

/* Number of kernels the library has launched so far (all contexts). */
int64_t gw_kernel_launches(const gw_ctx* ctx);

/* Per-launch timing of the two contraction kernels that carry Eqs.
 * tilde_P0_tau, tilde_sigma2 and HF_K (the SIMT strided contraction and the
 * tensor-core split-TF32 GEMM): with enable != 0 every launch is bracketed by
 * CUDA events on cfg->stream (a few microseconds of overhead per launch).
 * Synchronises and resets the accumulators. */
gw_status gw_profile(gw_ctx* ctx, int enable);

/* Reads and resets the accumulators of gw_profile.  out6[0..2]: SIMT
 * contraction kernel -- summed device milliseconds, useful flops (8 per
 * complex multiply-add), launches; out6[3..5]: the same for the tensor-core
 * kernel.  Synchronises. */
gw_status gw_profile_read(gw_ctx* ctx, double* out6);

/* Adjoint of gw_polarization's P~0(tau) (Eq. tilde_P0_tau, symmetrised) with
 * respect to G(tau), at the context's current G: Gbar = sum conj(dP~0/dG) Pbar
 * for a real loss (PyTorch's conjugate-Wirtinger convention).  Pbar
 * [nq][ntau][naux][naux] and Gbar [ntau][nk][nao][nao] are device pointers;
 * Gbar is overwritten.  Runs in fp64 whatever contract_prec is; allocates
 * three chain buffers of ntau*naux*nao^2 complex on first use. */
gw_status gw_polarization_vjp(gw_ctx* ctx, const double* Pbar, double* Gbar);

/* Adjoint of gw_selfenergy's Sigma~(tau) (Eq. tilde_sigma2, symmetrised) with
 * respect to G(tau) and P~(tau), at the context's current G and P~(tau).
 * Sbar [ntau][nk][nao][nao]; outputs Gbar [ntau][nk][nao][nao] and Pbar
 * [nq][ntau][naux][naux] are overwritten.  Device pointers; fp64. */
gw_status gw_selfenergy_vjp(gw_ctx* ctx, const double* Sbar, double* Gbar, double* Pbar);

/* The two adjoints above in complex64 arithmetic: V, G(tau), P~(tau) and the
 * (symmetrised) cotangent are rounded to complex64, every chain step runs with
 * fp32 accumulation within a launch, and the cotangent outputs accumulate in
 * fp64 across the (q, k) slabs.  Same arguments, layouts and fp64 storage as
 * gw_polarization_vjp / gw_selfenergy_vjp.  The first call of an FP64 context
 * allocates a complex64 copy of V (half of V's size); complex64 copies of G,
 * P~ and the cotangent are allocated on first use. */
gw_status gw_polarization_vjp_c64(gw_ctx* ctx, const double* Pbar, double* Gbar);
gw_status gw_selfenergy_vjp_c64(gw_ctx* ctx, const double* Sbar, double* Gbar, double* Pbar);

/* Tangent (Jacobian-vector product) of gw_polarization's P~0(tau) (Eq.
 * tilde_P0_tau, symmetrised) along dG at the context's current G.  P~0 is a
 * quadratic form in G, so dP~0 = P(dG(tau), G(-tau)) + P(G(tau), dG(-tau)).
 * dG [ntau][nk][nao][nao] in, dP0 [nq][ntau][naux][naux] out (overwritten);
 * device pointers.  Runs the forward chain of contract_prec (FP64, complex64
 * SIMT or split-TF32 tensor cores) twice; with complex64 contractions a second
 * c64 copy of G is allocated on first use. */
gw_status gw_polarization_jvp(gw_ctx* ctx, const double* dG, double* dP0);

/* Tangent of the screened block (Eqs. P0t_to_P0w, tilde_P_omega, Piw_to_Pt)
 * along dP~0(tau): with X = (I - P~0(i Omega))^-1 = I + P~(i Omega) from the
 * last gw_screened, dP~(i Omega) = X dP~0(i Omega) X, transformed back and
 * symmetrised.  dP0_tau in, dP_tau out, both [nq][ntau][naux][naux] device
 * pointers; fp64.  GW_ERR_STATE before gw_screened. */
gw_status gw_screened_jvp(gw_ctx* ctx, const double* dP0_tau, double* dP_tau);

/* Tangent of gw_selfenergy's Sigma~(tau) (Eq. tilde_sigma2, symmetrised) along
 * (dG, dP~(tau)) at the context's current G and P~(tau): Sigma~ is bilinear,
 * dSigma~ = S(dG, P~) + S(G, dP~).  dG [ntau][nk][nao][nao], dP_tau
 * [nq][ntau][naux][naux] in; dS_tau [ntau][nk][nao][nao] out (overwritten);
 * device pointers; runs the forward chain of contract_prec twice. */
gw_status gw_selfenergy_jvp(gw_ctx* ctx, const double* dG, const double* dP_tau, double* dS_tau);

/* Tangent of the self-consistency map F: (Sigma_inf, Sigma(i w)) -> (Sigma_inf',
 * Sigma'(i w)) (one pass of Eqs. Dyson, iw_to_tau, HF_J/HF_K, tilde_P0_tau,
 * tilde_P_omega, tilde_sigma2, tau_to_iw, with mu held at N(mu) = n_elec) along
 * (dSinf [nk][nao][nao], dSiw [nwf][nk][nao][nao]), at the context's state: G
 * from gw_dyson at the current Sigma and P~ from gw_polarization + gw_screened
 * at that G (GW_ERR_STATE otherwise).  Outputs oSinf, oSiw (same shapes) are
 * overwritten; all device pointers.  The Dyson and mu tangents
 * (dG = G D G - dmu G S G, dmu from dN = 0) and the transforms run in FP64, the
 * contraction tangents at contract_prec.  Allocates its buffers on first use. */
gw_status gw_sc_jvp(gw_ctx* ctx, const double* dSinf, const double* dSiw, double* oSinf, double* oSiw);

/* Newton-Krylov self-consistency: n_outer steps x <- x + delta on x =
 * (Sigma_inf, Sigma(i w)), with (J - I) delta = -(F(x) - x) solved by GMRES(m)
 * (1 <= m <= 64) whose products J v are gw_sc_jvp calls.  Stops early when
 * ||F(x) - x||_2 <= tol; res_out (host, n_outer doubles, may be NULL) receives
 * the residual norm of each step.  The context ends with G from gw_dyson at the
 * final Sigma (no damping is applied). */
gw_status gw_iterate_newton(gw_ctx* ctx, int32_t n_outer, int32_t m, double tol, double* res_out);

/* DIIS self-consistency (Sec. "Self-consistent finite-temperature GW": the loop is
 * converged with a DIIS scheme): the fixed-point problem x = F(x), x = (Sigma_inf,
 * Sigma~(i w)), F = one GW step (gw_dyson with the mu search at x, then P~0, the
 * screened solve and the new Sigma_inf, Sigma~(i w)).  Each step records x_i and
 * r_i = F(x_i) - x_i (the last m, 1 <= m <= 32), takes the affine combination of
 * least residual, min || sum c_i r_i ||^2 subject to sum c_i = 1 (inner product
 * Re <a, b> over all entries; the bordered normal equations scaled by max
 * ||r_i||^2, solved by QR on the host), and continues from x = sum c_i (x_i + mix
 * r_i).  Stops early when ||r||_2 <= tol; res_out (host, n_iter doubles, may be
 * NULL) receives ||r||_2 of each step.  The context ends with G from gw_dyson at
 * the final x.  Allocates 2m + 1 vectors of x's size on first use. */
gw_status gw_iterate_diis(gw_ctx* ctx, int32_t n_iter, int32_t m, double mix, double tol, double* res_out);

/* Dynamical part of the GW Luttinger-Ward functional (Sec. "Thermodynamics",
 * Eq. tilde_Phi_GW):
 *   Phi~ = 1/(2 Nk) sum_q (1/beta) sum_n tr{ln[I - P~0^q(i Omega_n)] + P~0^q(i Omega_n)},
 * from the context's P~0(tau) (gw_polarization or gw_set of GW_Q_P0_TAU; GW_ERR_STATE
 * otherwise), summed over the context's q range (gw_set_q_range: the ranks' values
 * add up to Phi~).  The bosonic Matsubara sum is the grid's own: (1/beta) sum_n F =
 * F(tau = beta^-) of the interpolant fitted at the sampled frequencies, i.e.
 * sum_m w_m F(i Omega_m) with w = lb TBb (the construction of gamma = -G(beta^-));
 * the real part is returned in *phi (host double).  P~0(i Omega_m) comes from
 * P~0(tau) by the FP64 transform; tr ln(I - P~0) is the sum of the logarithms of
 * the pivots of an FP64 LU factorisation without row exchanges, the continuous
 * branch when the Hermitian part of I - P~0 is positive definite (a negative
 * semidefinite polarization).  GW_ERR_SINGULAR for a zero pivot or one with
 * non-positive real part.  naux <= 6400 (GW_ERR_ARG otherwise).  Synchronises the
 * context's stream; allocates a workspace of up to nq nwb naux^2 complex doubles
 * for the duration of the call (GW_ERR_OOM when even one q does not fit). */
gw_status gw_grand_potential(gw_ctx* ctx, double* phi);

/* Allocation-free screened solve: P = [I - P0]^{-1} P0 for `count` complex
 * n x n matrices (interleaved (re, im) doubles, row-major, contiguous), the
 * operation of gw_screened without a context.  The paper has no counterpart;
 * it exists for callers that cannot allocate device memory when they need the
 * solve (memory owned by an arena or pool they do not control, hosts that
 * forbid cudaMalloc after start-up, code that must not hit an allocator's
 * implicit synchronisation).  P0 and P are device pointers owned by the caller
 * (P == P0 solves in place; otherwise the two ranges must not overlap, else
 * GW_ERR_ARG).  Scratch is one fixed array of 64 MiB inside the
 * library (GW_NOALLOC_SCRATCH_BYTES), resident on every device that loads the
 * library until the process exits; n is limited to orders whose per-matrix
 * workspace fits it (GW_ERR_ARG otherwise; n = 20000 fits).  The first call on
 * a device looks up the array's device address; make that first call before
 * any stream capture.  All calls share the array, so calls that overlap on the
 * GPU (different streams or threads) race and must be serialised by the
 * caller.  Work runs on `stream` (cudaStream_t, NULL = legacy default) and the
 * call synchronises it to read the pivot status: GW_ERR_SINGULAR on a zero
 * pivot.  No cudaMalloc, cudaFree or allocating library routine is called. */
#define GW_NOALLOC_SCRATCH_BYTES (64u << 20)
gw_status gw_screened_solve_noalloc(const double* P0, double* P, int64_t n, int64_t count, void* stream);

/* Message of the last failure of gw_screened_solve_noalloc in the calling thread
 * (empty after a successful call). */
const char* gw_noalloc_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* GWGB_H */
