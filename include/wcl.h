/*
 * wcl.h -- C ABI of libwcl, a GB300 (sm_103a) Wilson-clover propagator solver.
 *
 * The calls follow the statement of the problem in arXiv:2411.08461:
 * load a gauge field with kappa and c_sw and build the clover field
 * (Sec. III.B, "loadGauge ... the clover field is then created"), apply the
 * fermion matrix (Sec. II.E), and invert it for one or twelve spin-colour
 * sources, returning the solution, the true residual and the iteration count
 * (Sec. III.B: 12 inversions per propagator, invertMultiSrcQuda as the
 * batched form).
 *
 * Conventions (Sec. II.A):
 *   - lattice [Lx, Ly, Lz, Lt], Lx even, every extent >= 2;
 *   - QDP checkerboard ("cb2") order: parity p = (x+y+z+t) mod 2 first, then
 *     cb = ((t*Lz + z)*Ly + y)*(Lx/2) + x/2;
 *   - gauge   [4][2][Lt][Lz][Ly][Lx/2][3][3] complex128 (interleaved re, im),
 *             U[mu] is the link from s to s + mu_hat, mu = 0..3 <-> x, y, z, t,
 *             row-column colour order;
 *   - fermion [2][Lt][Lz][Ly][Lx/2][4][3] complex128, spin then colour;
 *     several right-hand sides are stored back to back, [nrhs][fermion];
 *   - DeGrand-Rossi gamma matrices (Chroma convention).
 *
 * Operator (Eq. 5, isotropic, multiplied by 2*kappa):
 *   M = A - kappa * H,
 *   H psi(s) = sum_mu eta (1 - gamma_mu) U_mu(s) psi(s+mu)
 *                   + eta (1 + gamma_mu) U_mu(s-mu)^+ psi(s-mu),
 *   A = 1 - kappa c_sw sum_{mu<nu} sigma_{mu nu} F_{mu nu},
 *   sigma_{mu nu} = [gamma_mu, gamma_nu]/2, F the traceless anti-Hermitian
 *   clover-leaf field strength; eta = t_boundary on hops across the time
 *   boundary (Sec. III.B: t_boundary = -1, antiperiodic), periodic in space.
 *   The solution of the mass-normalised operator a_t*M of the paper is 2*kappa*x.
 *
 * Even-odd (Schur) form used by the solvers and by wcl_apply_Mpc:
 *   M_hat = A_ee - kappa^2 D_eo A_oo^-1 D_oe.
 *
 * Ownership and execution:
 *   - every d_* pointer is caller-owned, contiguous device memory (e.g. a
 *     torch tensor's data_ptr()) -- fermion buffers may also be page-locked host
 *     memory, see wcl_apply_D -- and must stay valid for the duration of the
 *     call; the library never frees it;
 *   - the library owns its internal copies (reordered links, clover, solver
 *     workspace) and frees them in wcl_destroy;
 *   - all device work is issued on the stream given to wcl_create; every call
 *     returns only after its work is complete, so results and info structs are
 *     valid on return;
 *   - a context must not be used from two host threads at once.
 *
 * Errors: every call returns a wcl_status and never aborts the process.  A
 * CUDA error is reported as WCL_ERR_CUDA; wcl_last_error() gives the text of
 * the most recent failure on the calling thread.
 */
#ifndef WCL_H
#define WCL_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct wcl_ctx wcl_ctx; /* opaque, owned by the library */

typedef enum {
  WCL_OK = 0,
  WCL_ERR_INVALID_ARG = 1,  /* bad dims, null pointer, unsupported option */
  WCL_ERR_CUDA = 2,         /* a CUDA runtime call failed */
  WCL_ERR_OOM = 3,          /* device allocation failed */
  WCL_ERR_NOT_CONVERGED = 4,/* maxiter reached; x and info hold the best iterate */
  WCL_ERR_BREAKDOWN = 5,    /* Krylov breakdown persisted after restarts */
  WCL_ERR_NONFINITE = 6,    /* NaN or Inf in an input or in a residual */
  WCL_ERR_RECONSTRUCT = 7,  /* a link is not SU(3) to 1e-12: 12-real storage impossible */
  WCL_ERR_TIMEOUT = 8,      /* a bounded device wait expired */
  WCL_ERR_NO_GAUGE = 9,     /* wcl_load_gauge has not been called */
  WCL_ERR_NO_PRECOND = 10   /* learned solver requested without weights */
} wcl_status;

typedef enum {
  WCL_F64 = 0,
  WCL_F32 = 1,
  WCL_F16 = 2,   /* FP16 storage with per-site norms, FP32 arithmetic */
  WCL_BF16 = 3,  /* BF16 storage with per-site norms, FP32 arithmetic */
  WCL_DF64 = 4   /* double-float: every FP64 value stored as an FP32 pair (hi, lo), ~48-bit
                    significand, arithmetic on the FP32 pipes; for wcl_apply_D /
                    wcl_apply_Mpc, and as wcl_solve_params.outer for the residual
                    replacements in the middle of a solve (every reported residual is FP64). */
} wcl_prec;

typedef enum {
  WCL_BICGSTAB = 0,      /* BiCGStab on M_hat (Sec. II.E: default for clover) */
  WCL_CGNR = 1,          /* CG on M_hat^+ M_hat (Sec. II.E: CG) */
  WCL_FGCR_LEARNED = 2,  /* flexible GCR on M_hat with the learned preconditioner */
  WCL_GCR = 3,           /* the same GCR without a preconditioner (the comparison method) */
  WCL_FGCR_MG = 4,       /* flexible GCR on the whole-lattice M preconditioned by the two-level
                            multigrid K-cycle of wcl_mg_setup (Sec. II.E: QUDA's multigrid), FP32
                            between IEEE FP64 true-residual restarts; right-hand sides one after
                            another, wcl_invert only.  Uses tol, maxiter and gcr_nkrylov. */
  WCL_FGCR_MG_BATCHED = 5 /* every right-hand side at once: flexible GCR on M_hat (as WCL_GCR, with
                            its FP64 residual replacements) preconditioned by the batched K-cycle
                            (wcl_mg_cycle_batched) applied to the even residual with zero odd sites;
                            sloppy must be WCL_F32; wcl_invert only. */
} wcl_solver;

typedef struct {
  wcl_solver solver;
  wcl_prec outer;        /* residual replacements of a mixed-precision solve: WCL_DF64 (default)
                            runs the intermediate ones with the double-float operator and the
                            final ones in IEEE FP64; WCL_F64 runs all of them in FP64.  The
                            solution, the reductions and every reported residual are FP64. */
  wcl_prec sloppy;       /* precision of the inner Krylov vectors, links and clover */
  double tol;            /* target relative true residual ||b - M x|| / ||b|| */
  int maxiter;           /* total inner iterations per right-hand side */
  double delta_reliable; /* reliable update when ||r|| < delta * max||r|| since the last one */
  int restart_on_update; /* 1: restart the Krylov space at every update (defect correction) */
  int gcr_nkrylov;       /* FGCR restart length */
  int use_graphs;        /* capture check_every iterations in a CUDA graph */
  int check_every;       /* iterations between host convergence checks */
} wcl_solve_params;

typedef struct {
  int iters;             /* inner iterations */
  double true_residual;  /* ||b - M x|| / ||b|| in FP64 over the whole lattice */
  int reliable_updates;  /* residual replacements (double-float or FP64) */
  int status;            /* wcl_status of this right-hand side */
  double seconds;        /* wall time of the whole call */
} wcl_solve_info;

/* Fill *p with defaults: BiCGStab, outer DF64, sloppy F32, tol 1e-10,
 * maxiter 20000, delta 0.1, no restarts, nkrylov 20, graphs on, check_every 8. */
void wcl_default_params(wcl_solve_params* p);

/* Human-readable name of a status code (static storage). */
const char* wcl_status_string(wcl_status s);

/* Text of the most recent error on the calling thread ("" if none). */
const char* wcl_last_error(void);

/* Create a context for one lattice.
 *   dims       : {Lx, Ly, Lz, Lt}; Lx even, all >= 2, volume < 2^31 sites.
 *   t_boundary : +1 periodic or -1 antiperiodic fermion time boundary.
 *   device     : CUDA device ordinal; made current for every call on ctx.
 *   cuda_stream: cudaStream_t (NULL = legacy default stream).
 * The caller owns *out and releases it with wcl_destroy. */
wcl_status wcl_create(wcl_ctx** out, const int dims[4], int t_boundary, int device, void* cuda_stream);

/* Load a gauge field and build the clover term and its inverse (Sec. III.B).
 *   d_gauge: device, complex128, QDP layout above; read only.
 *   kappa  : hopping parameter, csw: clover coefficient (isotropic).
 * The links are checked to be SU(3) (|U U^+ - 1|, |det U - 1| < 1e-12);
 * otherwise WCL_ERR_RECONSTRUCT.  Non-finite entries give WCL_ERR_NONFINITE.
 * The clover field is built from the bare links in FP64, inverted per chiral
 * 6x6 block in FP64 and stored in every precision. */
wcl_status wcl_load_gauge(wcl_ctx* ctx, const void* d_gauge, double kappa, double csw);

/* Anisotropic form of Eq. 5 (Sec. III.B):
 *   2 kappa a_t M = 1 - kappa [ W_4 + (nu/xi0) sum_i W_i
 *                               + c_sw^t sum_i sigma_i4 F_i4 + (c_sw^r/xi0) sum_{i<j} sigma_ij F_ij ]
 * (W_mu the Wilson hops of the isotropic operator above).  Everything else is as for
 * wcl_load_gauge; wcl_load_gauge(kappa, csw) is the case xi0 = nu = 1,
 * c_sw^t = c_sw^r = csw.  Internally the hopping parameter is kappa nu/xi0 with the
 * t hops weighted by xi0/nu, so solutions and residuals are those of the operator
 * above.  WCL_ERR_INVALID_ARG unless all values are finite and xi0, nu > 0. */
wcl_status wcl_load_gauge_aniso(wcl_ctx* ctx, const void* d_gauge, double kappa, double xi0, double nu,
                                double csw_t, double csw_r);

/* Fermion buffers (d_in, d_out, d_x, d_b below) are device memory of the
 * context's GPU, or page-locked host memory (cudaHostAlloc / cudaHostRegister),
 * which the import and export kernels read and write in place through its device
 * alias over the host link; anything else gives WCL_ERR_INVALID_ARG.  As for
 * device buffers, the results are complete when the call returns.
 *
 * d_out = M d_in on the whole lattice for nrhs fields (QDP layout, complex128),
 * computed in precision prec (links, clover and spinors stored in prec). */
wcl_status wcl_apply_D(wcl_ctx* ctx, void* d_out, const void* d_in, wcl_prec prec, int nrhs);

/* d_out_e = M_hat d_in_e (dagger = 0) or M_hat^+ d_in_e (dagger = 1) on the even
 * half-lattice: each field is [Lt][Lz][Ly][Lx/2][4][3] complex128 (the first
 * half of a QDP fermion), nrhs of them back to back. */
wcl_status wcl_apply_Mpc(wcl_ctx* ctx, void* d_out_e, const void* d_in_e, wcl_prec prec, int nrhs, int dagger);

/* Solve M x = b for nrhs right-hand sides (1..12) through the Schur complement.
 *   d_x, d_b: [nrhs][QDP fermion] complex128 (device or page-locked host);
 *             d_x is written.
 *   info    : host array of nrhs entries, filled on return.
 * Returns WCL_OK when every right-hand side reached params->tol, otherwise the
 * first failing status (x still holds the best iterate). */
wcl_status wcl_invert(wcl_ctx* ctx, void* d_x, const void* d_b, int nrhs,
                      const wcl_solve_params* params, wcl_solve_info* info);

/* Solve on several lattices of different sizes at once: one launch per solver
 * step covers every lattice and right-hand side (nctx <= 8, same nrhs on each).
 *   ctxs[i], d_x[i], d_b[i]: the context and the fields of lattice i;
 *   info: host array of nctx * nrhs entries, lattice-major. */
wcl_status wcl_invert_batch(wcl_ctx* const* ctxs, int nctx, void* const* d_x, const void* const* d_b, int nrhs,
                            const wcl_solve_params* params, wcl_solve_info* info);

/* ---- learned preconditioner ------------------------------------------------
 * Not part of the paper: a gauge-covariant parallel-transport network N used as
 * the preconditioner of flexible GCR (WCL_FGCR_LEARNED).  Four linear layers with
 * channels 1 -> 4 -> 4 -> 4 -> 1,
 *   out_{c'}(x) = sum_{c,s} W[c',c,s] (T_s in_c)(x),  s in {0, +x, -x, +y, -y, +z, -z, +t, -t},
 *   T_0 = 1, T_{+mu} psi(x) = eta U_mu(x) psi(x+mu), T_{-mu} psi(x) = eta U_mu(x-mu)^+ psi(x-mu),
 * W[c',c,s] a complex 4x4 spin matrix.  It acts on even-parity fields (the odd
 * sites of its input are zero; the even part of its output approximates
 * M_hat^-1 r), so the weights do not depend on the gauge field or the volume.
 * Weights: WCL_PTC_NWEIGHTS complex numbers, layer by layer, each layer indexed
 * ((c_out * c_in + c_in_index) * 9 + s) * 16 + 4 * row + col, shifts ordered
 * 0, +x, -x, +y, -y, +z, -z, +t, -t.  Host arrays are interleaved (re, im) doubles. */
#define WCL_PTC_NWEIGHTS 5760

typedef struct {
  int epochs;   /* passes over the pairs */
  int batch;    /* pairs per Adam step */
  double lr, beta1, beta2, eps; /* Adam on real and imaginary parts */
} wcl_train_params;

/* Defaults: 4 epochs, batch 8, Adam lr 1e-3, betas 0.9 / 0.999, eps 1e-8. */
void wcl_default_train_params(wcl_train_params* p);

/* Copy WCL_PTC_NWEIGHTS complex weights (host, interleaved doubles) to ctx; resets Adam. */
wcl_status wcl_precond_load(wcl_ctx* ctx, const double* h_weights);

/* Copy the current FP32 master weights of ctx back to the host. */
wcl_status wcl_precond_get(wcl_ctx* ctx, double* h_weights);

/* d_out_e = N(d_in_e) for nrhs even half-fields (QDP even half, complex128);
 * bf16 != 0 uses the BF16 copy of the weights (FP32 accumulation either way). */
wcl_status wcl_precond_apply(wcl_ctx* ctx, void* d_out_e, const void* d_in_e, int nrhs, int bf16);

/* Loss L = (1/n) sum_b ||N(r_b)_e - e_b||^2 / ||e_b||^2 over n pairs of even
 * half-fields (device, [n][even half] complex128) and its gradient with respect
 * to every weight, G = dL/dRe W + i dL/dIm W (host array, interleaved doubles,
 * may be NULL), using the FP32 weights. */
wcl_status wcl_precond_loss_grad(wcl_ctx* ctx, const void* d_r_e, const void* d_e_e, int npairs, double* loss,
                                 double* h_grad);

/* Train the weights of ctx with Adam on n pairs (r, e), r = M_hat e (device,
 * [n][even half] complex128).  Forward, backward and update run on the GPU with
 * this library's kernels.  h_loss_per_epoch (host, epochs entries, may be NULL)
 * receives the mean batch loss of every epoch. */
wcl_status wcl_precond_train(wcl_ctx* ctx, const void* d_r_e, const void* d_e_e, int npairs,
                             const wcl_train_params* params, double* h_loss_per_epoch);

/* Propagator layout (Sec. II.A): [2][Lt][Lz][Ly][Lx/2][Ns][Ns][Nc][Nc] complex128
 * with sink-source spin and sink-source colour order.  The twelve solutions of
 * wcl_invert for the spin-colour sources k = 3 * spin + colour ([12][fermion]) are
 * its source columns: prop[..., s, s0, c, c0] = x[3 s0 + c0][..., s, c].
 *   d_prop, d_x12: device or page-locked host memory (as the fermion buffers of
 *   wcl_apply_D), caller-owned, not overlapping.  Pure data movement (bit exact). */
wcl_status wcl_fermions_to_propagator(wcl_ctx* ctx, void* d_prop, const void* d_x12);
wcl_status wcl_propagator_to_fermions(wcl_ctx* ctx, void* d_x12, const void* d_prop);

/* ---- Propagator workflow around the solve (Sec. III.A, III.B) ----------------
 * Momentum modes n = mom[0..2] (x, y, z; NULL = zero momentum) give
 * p_k = 2 pi n_k / L_k.  A momentum source carries exp(+i p.x) and the sink of a
 * contraction or a sequential source exp(-i p.x), the source and sink phases of
 * Eq. 1 and Eq. 2.  Gamma arguments are host arrays of 16 complex entries (32
 * doubles, row-major, re then im) with exactly one nonzero entry per row equal to
 * 1, i, -1 or -i (within 1e-12): every product of DeGrand-Rossi gamma matrices,
 * see wcl_gamma; anything else is WCL_ERR_INVALID_ARG.  Buffers are caller-owned
 * device or page-locked host memory, complex128, QDP layout. */

/* Gamma(n) = gamma_1^b0 gamma_2^b1 gamma_3^b2 gamma_4^b3 (b_k the bits of n, 0..15)
 * in the DeGrand-Rossi basis (Sec. II.A; Gamma(15) = gamma_5, Gamma(4) = gamma_3,
 * so Eq. 7's insertion is Gamma(15) Gamma(4)).  h_out: 32 doubles.  Host only: needs
 * no context and no GPU. */
wcl_status wcl_gamma(int n, double* h_out);

/* kappa = 1 / (2 (m0 + 4)): the relation under Eq. 5 with xi_0 = nu = 1 (isotropic).
 * Host only; WCL_ERR_INVALID_ARG unless m0 is finite and m0 > -4. */
wcl_status wcl_kappa_from_mass(double m0, double* kappa);

/* kappa = 1 / (2 (m0 + 1 + 3 nu/xi0)), the relation under Eq. 5.  Host only;
 * WCL_ERR_INVALID_ARG unless the values are finite, xi0, nu > 0 and the bracket > 0. */
wcl_status wcl_kappa_from_mass_aniso(double m0, double xi0, double nu, double* kappa);

/* The twelve spin-colour wall sources on timeslice t0 (Sec. III.B): d_b12 is
 * [12][fermion]; fermion k = 3 s + c is exp(+i p.x) (1 at zero momentum) in spin s,
 * colour c on timeslice t0 and zero elsewhere -- the input of wcl_invert with
 * nrhs = 12 for the propagator S_{p, t0} of Eq. 2. */
wcl_status wcl_wall_source(wcl_ctx* ctx, void* d_b12, int t0, const int* mom);

/* Sequential source (Eq. 4 and the sequential-source equation of Sec. III.B):
 * X[site][i][k][a][b] = exp(-i p.x) sum_j Gamma[i][j] S[site][j][k][a][b] on timeslice
 * t and zero elsewhere; d_X and d_S are propagators (distinct buffers), h_gamma NULL
 * means gamma_5.  Invert its twelve source columns (wcl_propagator_to_fermions,
 * wcl_invert) for the sequential propagator. */
wcl_status wcl_sequential_source(wcl_ctx* ctx, void* d_X, const void* d_S, int t, const int* mom,
                                 const double* h_gamma);

/* Meson contraction (Eq. 6, Eq. 7): for every timeslice t,
 *   out[t] = sum_{x in t} exp(-i p.x) sum_{i,j,k,a,b} conj(A[x][j][i][b][a]) Gamma[j][k] B[x][k][i][b][a]
 * with A, B propagators and h_gamma NULL meaning the identity.  Eq. 6 is
 * (A, B, Gamma, p) = (S_0, S_p, 1, p); Eq. 7 is (S_seq, S_p, gamma_5 gamma_3, 0).
 * d_A, d_B: device memory (read with asynchronous shared-memory copies); d_out: Lt
 * complex128, device or page-locked host.  Sums are FP64, added in a fixed order
 * (deterministic). */
wcl_status wcl_contract(wcl_ctx* ctx, void* d_out, const void* d_A, const void* d_B, const double* h_gamma,
                        const int* mom);

/* Options of a context (wcl_set_option). */
typedef enum {
  WCL_OPT_TENSOR_CORES = 1 /* 1: 16-bit multi-RHS dslash (4..16 RHS) with the link and clover
                              multiplies on the tensor cores (mma.sync, FP32 accumulation);
                              0 (default): the per-thread kernel, faster with this field layout */
  ,
  WCL_OPT_SHARED_LINKS = 2 /* 1 (default) or 8, 16, 32: the multi-RHS dslash (4..16 RHS, Schur
                              operator) may stage the links and clover of a tile of sites in shared
                              memory once for all RHS; the value is the tile (1 = 16 sites) used
                              when the autotuner is off (FP64 always uses 16).
                              0: one thread per (site, RHS) reading its own links and clover */
  ,
  WCL_OPT_AUTOTUNE = 3 /* 1 (default): the first launch of each dslash configuration (precision,
                          operator form, RHS count, lattice shapes) outside graph capture times
                          every eligible kernel variant and launch shape and keeps the fastest
                          for the process; the environment variable WCL_TUNE_CACHE=<file>
                          makes the choices persist (text, appended).  0: fixed defaults */
  ,
  WCL_OPT_PTC_TENSOR_CORES = 4 /* how the learned preconditioner's BF16 layers do the channel
                                  and spin mixing (BF16 weights, FP32 accumulation): 2 (default)
                                  on the fifth-generation tensor cores (tcgen05: one CTA per 128
                                  sites, operands in shared memory, accumulators in tensor memory;
                                  inputs as WCL_OPT_PTC_SPLIT BF16 terms; a bounded wait that
                                  expires makes the call return WCL_ERR_TIMEOUT); 1: mma.sync,
                                  inputs split into three BF16 terms; 0: FP32 SIMT mixing.  Other
                                  values: WCL_ERR_INVALID_ARG */
  ,
  WCL_OPT_STAGED_SPINORS = 5 /* 1: when the tuner is off, the multi-RHS dslash (16-site tiles)
                                also stages each thread's neighbour spinors in shared memory with
                                asynchronous copies (cp.async, two hops in flight); 0 (default):
                                direct loads.  With the tuner on, both are candidates. */
  ,
  WCL_OPT_BLOCKED_TILES = 6 /* 1: when the tuner is off, the multi-RHS dslash walks its tiles in
                               blocks of z planes on lattices with more than 512 tiles per time
                               slice, so that the t neighbours of a site are still in L2 (DRAM
                               traffic 1.07x instead of 1.25x the algorithmic bytes at 32^3x64);
                               0 (default): site order.  With the tuner on, both are candidates. */
  ,
  WCL_OPT_PAIRED_RHS = 7 /* 1: when the tuner is off, the multi-RHS FP32 / 16-bit dslash (4..16 RHS)
                            runs the packed-pair kernel: each thread owns one site and two
                            right-hand sides held in float2 registers, so that one packed FP32
                            instruction (FFMA2 / FADD2) serves both; the tile is that of
                            WCL_OPT_SHARED_LINKS (or 16 with WCL_OPT_BLOCKED_TILES).  0 (default):
                            one right-hand side per thread.  With the tuner on, both are candidates. */
  ,
  WCL_OPT_PREFETCH_SPINORS = 8 /* 1: when the tuner is off, the multi-RHS FP32 / 16-bit dslash (16-site
                                  tiles, one right-hand side per thread) loads the neighbour spinor
                                  of the next hop into registers before computing the current one,
                                  so that one hop's gathers are always in flight; 0 (default): each
                                  hop loads and then computes.  With the tuner on, both are candidates. */
  ,
  WCL_OPT_TMA_STAGING = 9 /* 1: when the tuner is off, the multi-RHS FP32 dslash on a lattice with Lx = 32
                             runs the persistent kernel whose tiles are whole x-rows and whose links and
                             clover reach shared memory by tensor copies (TMA, cp.async.bulk.tensor),
                             double buffered under the previous tile's compute; 2: the same kernel with
                             one CTA per tile (copies issued at its start); 0 (default): ordinary loads.
                             With the tuner on, all are candidates where the kernel applies. */
  ,
  WCL_OPT_PTC_SPLIT = 10 /* BF16 terms each transported input is split into on the tcgen05 network
                            layers (WCL_OPT_PTC_TENSOR_CORES = 2): 1 (default, plain BF16 inputs),
                            2 (16 significant bits) or 3 (24 bits: the FP32 layer to FP32 rounding);
                            fewer terms need less shared memory per CTA and fewer MMAs.  The
                            network is a preconditioner of flexible GCR, whose true residual does
                            not depend on it. */
  ,
  WCL_OPT_SLOPPY_UPDATES = 11 /* k in 1..8: in a solve with an FP16 or BF16 inner solver and
                                 double-float intermediate updates (outer WCL_DF64), a reliable
                                 update made while the iterated residual is above 10^-k ||b||
                                 evaluates b - M x with the FP32 operator, whose rounding is far
                                 below the 16-bit recurrence's; later updates stay double-float
                                 and the final ones IEEE FP64, so every reported residual is FP64.
                                 0 (default): every intermediate update double-float. */
} wcl_option;

/* Set an option of ctx; unknown options give WCL_ERR_INVALID_ARG. */
wcl_status wcl_set_option(wcl_ctx* ctx, int option, int value);

/* Counters for measurement. */
typedef struct {
  long long kernel_launches; /* every kernel of this library launched on ctx (graph replays included) */
  long long dslash_launches; /* fused dslash + clover launches among them */
  double dslash_ms;          /* summed device time of the timed dslash launches (profiling on) */
  long long dslash_timed;    /* how many dslash launches were timed */
  double dslash_bytes;       /* algorithmic bytes of the timed launches */
  double dslash_flops;       /* algorithmic flops of the timed launches (1320 + 504 per clover site) */
  /* the timed launches split by arithmetic precision, indexed by wcl_prec (F64, F32, F16, BF16, DF64) */
  double prec_ms[5];
  long long prec_timed[5];
  double prec_bytes[5];
  double prec_flops[5];
} wcl_stats;

/* When enabled, every fused dslash launch on ctx is bracketed by CUDA events on
 * the stream it runs on (also inside captured graphs) and its device time is
 * accumulated into wcl_stats. */
wcl_status wcl_set_profiling(wcl_ctx* ctx, int enable);

/* Read (and with reset != 0, afterwards zero) the counters of ctx. */
wcl_status wcl_get_stats(wcl_ctx* ctx, wcl_stats* out, int reset);

/* Largest number of sites per parity (Vh rounded up to a multiple of 64) that
 * wcl_apply_Mpc_noalloc accepts; e.g. 8^3x32, 16^3x8, 16x16x8x16. */
#define WCL_NOALLOC_MAX_VH 16384

/* d_out_e = M_hat d_in_e (dagger = 0) or M_hat^+ d_in_e (dagger = 1) in FP64 for
 * one even half-field, exactly as wcl_apply_Mpc(ctx, d_out_e, d_in_e, WCL_F64, 1,
 * dagger), but without allocating any memory in the call.
 *
 * The paper has no counterpart: this entry point exists for callers that cannot
 * let a library allocate device memory while they run -- for instance a program
 * whose own pool allocator owns all device memory, or a time-critical loop that
 * cannot accept cudaMalloc's implicit device synchronisation or its failure
 * part-way through a run.  The context (links, clover) must be prepared
 * beforehand with wcl_create / wcl_load_gauge.
 *
 * Scratch: the input copy, the odd-parity intermediate and the output live in
 * one fixed device array of 3 x 192 x WCL_NOALLOC_MAX_VH bytes (9 MiB).  It is
 * set up -- its device address looked up, which loads the library module that
 * holds it -- by wcl_create, so every GPU on which a context has been created
 * holds it until the process exits, and the call itself allocates nothing, also
 * the first time and on a lattice shape it has not seen (the autotuner is not
 * consulted beyond its cache: an untuned configuration runs its default kernel).
 * A cudaDeviceReset invalidates it together with every context of that device.
 * Lattices with more than WCL_NOALLOC_MAX_VH padded sites per parity are rejected
 * with WCL_ERR_INVALID_ARG.  Every call shares the array and leaves its contents
 * behind (each call writes everything it reads, so nothing is cleared); calls
 * whose GPU work overlaps -- from different streams, threads or contexts on the
 * same device -- race on it and must be serialised by the caller.
 *   d_in_e, d_out_e: device memory of the context's GPU, [Lt][Lz][Ly][Lx/2][4][3]
 *   complex128, caller-owned; anything else (page-locked or pageable host memory,
 *   another GPU's memory) is WCL_ERR_INVALID_ARG. */
wcl_status wcl_apply_Mpc_noalloc(wcl_ctx* ctx, void* d_out_e, const void* d_in_e, int dagger);

/* ---- adaptive aggregation multigrid (Sec. II.E; Sec. III.B passes one block size per level) ----
 * Two levels on the whole-lattice operator M.  The paper names the method without its
 * steps; the library takes the standard aggregation ones:
 *   null space : nvec start vectors relaxed towards M x = 0 by relax_steps minimal-residual
 *                steps (r = -M x; alpha = <M r, r> / |M r|^2; x += alpha r; r -= alpha M r),
 *                then normalised;
 *   P          : per block of block[0] x block[1] x block[2] x block[3] sites and per
 *                chirality (spins {0,1} and {2,3}) the restrictions of the null vectors,
 *                made orthonormal (modified Gram-Schmidt, twice): P^+ P = 1;
 *   coarse op  : A_c = P^+ M P as the nine-point stencil
 *                (A_c c)(x) = X(x) c(x) + sum_mu [Yf_mu(x) c(x + mu) + Yb_mu(x) c(x - mu)]
 *                of (2 nvec) x (2 nvec) blocks, built from the links, the clover term and P;
 *   K-cycle    : pre minimal-residual steps from zero, e += P A_c^-1 P^+ (r - M e) with
 *                the coarse system solved by GCR(coarse_nkrylov) to coarse_tol (at most
 *                coarse_maxiter steps), post minimal-residual steps.
 * Arithmetic is FP32 (FP64 sums).  Coarse vectors are [Ct][Cz][Cy][Cx][2][nvec] complex128,
 * C_mu = L_mu / block[mu], chirality before vector index. */
typedef struct {
  int block[4];        /* block extents (x, y, z, t); each divides the lattice extent */
  int nvec;            /* null vectors, 1..32 and at most 6 x block sites */
  int relax_steps;     /* minimal-residual steps per null vector (0: the starts as given) */
  int pre, post;       /* smoothing steps of the K-cycle */
  double coarse_tol;   /* relative residual of the coarse GCR */
  int coarse_maxiter;  /* coarse GCR steps at most */
  int coarse_nkrylov;  /* coarse GCR restart length (1..64) */
} wcl_mg_params;

/* Defaults: blocks 4^4, 24 vectors, 20 relaxation steps, 2 + 2 smoothing steps,
 * coarse GCR(8) to 0.1 in at most 50 steps. */
void wcl_default_mg_params(wcl_mg_params* p);

/* Build the hierarchy of ctx's operator (after wcl_load_gauge) from nvec start vectors
 * d_starts: [nvec][QDP fermion] complex128, device or page-locked host (random numbers
 * are the caller's).  WCL_ERR_BREAKDOWN if a vector vanishes or the vectors are linearly
 * dependent on a block. */
wcl_status wcl_mg_setup(wcl_ctx* ctx, const void* d_starts, const wcl_mg_params* params);

/* d_out = K-cycle(d_in): one application of the preconditioner to a whole-lattice field
 * (QDP fermion, complex128); coarse_iters (may be NULL) receives the coarse GCR steps. */
wcl_status wcl_mg_cycle(wcl_ctx* ctx, void* d_out, const void* d_in, int* coarse_iters);

/* d_out[r] = K-cycle(d_in[r]) for nrhs whole-lattice QDP fermions (complex128, device or
 * page-locked host) at once: the steps of wcl_mg_cycle with every minimal-residual and
 * Gram-Schmidt coefficient computed on the device per right-hand side, the coarse stencil
 * read once for up to six right-hand sides, and exactly coarse_maxiter coarse GCR steps
 * (restarted every coarse_nkrylov; coarse_tol is not consulted), so no step waits on the
 * host.  Allocates its work space on first use.  1 <= nrhs <= 12. */
wcl_status wcl_mg_cycle_batched(wcl_ctx* ctx, void* d_out, const void* d_in, int nrhs);

/* Restriction P^+ (QDP fermion -> coarse vector) and prolongation P (coarse -> QDP
 * fermion, overwritten); coarse vectors are complex128, device or host memory. */
wcl_status wcl_mg_restrict(wcl_ctx* ctx, void* d_coarse, const void* d_fine);
wcl_status wcl_mg_prolong(wcl_ctx* ctx, void* d_fine, const void* d_coarse);

/* d_out = A_c d_in on coarse vectors (complex128, device or host). */
wcl_status wcl_mg_coarse_apply(wcl_ctx* ctx, void* d_out, const void* d_in);

/* Copy P to the host: [2][Lt][Lz][Ly][Lx/2] sites (QDP order) x [12] rows (3 spin + colour)
 * x [2 nvec] columns (chirality nvec + vector), complex128 interleaved; entries whose row
 * and column chiralities differ are zero. */
wcl_status wcl_mg_get_prolongator(wcl_ctx* ctx, double* h_P);

/* Copy the stencil to the host: [9][coarse site][2 nvec][2 nvec] complex128 (row, column),
 * block 0 = X, 1 + 2 mu = Yf_mu, 2 + 2 mu = Yb_mu. */
wcl_status wcl_mg_get_stencil(wcl_ctx* ctx, double* h_Y);

/* ---- staggered operator of the HISQ action on given smeared links (Sec. II.A, II.E) ----
 *   M chi = 2 m chi + D chi,
 *   D chi(x) = sum_mu eta_mu(x) [ V_mu(x) chi(x+mu) - V_mu(x-mu)^+ chi(x-mu)
 *                               + W_mu(x) chi(x+3mu) - W_mu(x-3mu)^+ chi(x-3mu) ]
 * with V the fat (one-hop) and W the long (three-hop, Naik coefficient included) links of
 * the HISQ smearing, the MILC phases eta_x = 1, eta_y = (-1)^x, eta_z = (-1)^(x+y),
 * eta_t = (-1)^(x+y+z), and t_boundary (wcl_create) on every hop across t = Lt-1 -> 0.
 * wcl_hisq_smear makes V and W from thin links.  Staggered fields are
 * [2][Lt][Lz][Ly][Lx/2][3] complex128 (QDP order, colour only), nrhs back to back. */

/* HISQ link smearing in FP64 (Sec. II.A: the HISQ process of Follana et al. in the MILC
 * convention, with a U(3) projection of the first fattened links; the paper gives no
 * coefficients, these are the fat7 / asqtad ones).  With staple(+-rho, F) the mu-directed
 * object F carried one step along +-rho and back, a smearing (c1, c3, c5, c7, cL) replaces
 * each link by c1 U_mu + c3 sum of 3-link staples + c5 sum of 5-link staples (all ordered
 * pairs of signed directions) + c7 sum of 7-link staples (ordered triples) + cL sum of the
 * straight 5-link (Lepage) staples:
 *   V = smear(U; 1/8, 1/16, 1/64, 1/384, 0),   W = V (V^+ V)^(-1/2),
 *   fat = smear(W; 5/8, 1/16, 1/64, 1/384, -1/16) + eps/8 W,
 *   long_mu(x) = -(1 + eps)/24 W_mu(x) W_mu(x+mu) W_mu(x+2mu),
 * ready for wcl_load_staggered.  d_gauge: thin links U, QDP gauge layout [4][2][Lt][Lz][Ly]
 * [Lx/2][3][3] complex128 (device or page-locked host, read only, periodic: no boundary
 * sign); d_fat, d_long: caller-owned outputs in the same layout, written entirely (not
 * valid after an error).  eps_naik: the Naik epsilon (0 for light quarks).  Uses ctx's
 * lattice shape, device and stream, not its gauge field; allocates and frees about
 * 15 x 144 bytes per site of work space during the call.  Errors: WCL_ERR_INVALID_ARG,
 * WCL_ERR_NONFINITE (a non-finite thin link), WCL_ERR_RECONSTRUCT (a first-level link V
 * with V^+ V not positive definite), WCL_ERR_OOM, WCL_ERR_CUDA. */
wcl_status wcl_hisq_smear(wcl_ctx* ctx, void* d_fat, void* d_long, const void* d_gauge, double eps_naik);

/* Load V and W (QDP gauge layout, complex128, device or page-locked host; any complex
 * 3x3 matrices) and the mass m (> 0: the solve is even-odd).  Kept in FP64 and FP32. */
wcl_status wcl_load_staggered(wcl_ctx* ctx, const void* d_fat, const void* d_long, double mass);

/* d_out = M d_in on the whole lattice for nrhs fields, prec WCL_F64 or WCL_F32. */
wcl_status wcl_apply_staggered(wcl_ctx* ctx, void* d_out, const void* d_in, wcl_prec prec, int nrhs);

/* Solve M x = b for nrhs staggered right-hand sides (one after another) by CG on the even
 * sites, (4 m^2 - D_eo D_oe) x_e = 2 m b_e - D_eo b_o, x_o = (b_o - D_oe x_e)/(2 m) (Sec. II.E:
 * CG is the HISQ default), in params->sloppy (WCL_F32: FP32 CG between IEEE FP64 restarts
 * from the true residual; WCL_F64: FP64 CG), to ||b - M x|| / ||b|| <= params->tol computed
 * in FP64; uses tol and maxiter.  info: host array of nrhs entries. */
wcl_status wcl_invert_staggered(wcl_ctx* ctx, void* d_x, const void* d_b, int nrhs, const wcl_solve_params* params,
                                wcl_solve_info* info);

/* ---- clover fermion force (Sec. IV: the paper's HMC uses the clover and HISQ forces) ----
 * F = the force of the two-flavour even-odd clover action of ctx's (isotropic) operator,
 *   S(U) = phi^+ (M_hat^+ M_hat)^-1 phi - 2 sum_{x odd} log det A(x),
 * the second term (the clover determinant of the odd sites) only with include_logdet != 0.
 * d_x_e: X = (M_hat^+ M_hat)^-1 phi on the even sites ([Lt][Lz][Ly][Lx/2][4][3]
 * complex128, the caller's solve; the force is evaluated for whatever X is given).
 * d_force: [4][2][Lt][Lz][Ly][Lx/2][3][3] complex128 (the QDP gauge layout), receives
 * F_mu(x), traceless anti-Hermitian, defined by dS/d eps = -Tr(Q F_mu(x)) for the left
 * variation U_mu(x) -> exp(eps Q) U_mu(x) (Q traceless anti-Hermitian); an HMC step then
 * moves the momenta by -dt F.  Both buffers device memory of ctx's GPU or page-locked host
 * memory, caller-owned.  FP64 throughout (links, clover inverse and operator of ctx).
 * Errors: WCL_ERR_NO_GAUGE; WCL_ERR_INVALID_ARG (null or foreign pointer, or a context
 * loaded with wcl_load_gauge_aniso); WCL_ERR_NONFINITE (non-finite X); WCL_ERR_CUDA. */
wcl_status wcl_clover_force(wcl_ctx* ctx, void* d_force, const void* d_x_e, int include_logdet);

/* Release every library-owned resource of ctx (cf. dirac.destroy, Sec. III.B). */
wcl_status wcl_destroy(wcl_ctx* ctx);

#ifdef __cplusplus
}
#endif

#endif /* WCL_H */
