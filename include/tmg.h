/*
 * tmg.h -- C ABI of the GB300 twisted-mass DD-alpha-AMG library (libtmg.so).
 *
 * Operators and method follow arXiv:1710.06198 ("Multigrid accelerated simulations for Twisted
 * Mass fermions"):
 *   - Sec. 1.1: clover-improved Wilson operator D, twisted mass D(+-mu) = D +- i mu G5,
 *     error propagation of the DD-alpha-AMG preconditioner (Eq. 1): SAP smoother M, aggregation
 *     prolongation P (G5 P = P G5_c), coarse operator D_c = P^dag D P, D_c(+-mu) = D_c +- i mu G5_c,
 *     flexible Krylov outer solver.
 *   - Eq. 2: non-degenerate doublet D_ND(mubar, epsbar) = D x I2 + i mubar G5 x tau3 - epsbar I x tau1.
 *   - Sec. 1.1: D^dag(mu) D(mu) solved in two steps, D(-mu) x = G5 b then D(mu) y = G5 x.
 *
 * Conventions (readings of what the paper leaves open):
 *   - lattice dims {Lx, Ly, Lz, T}; lexicographic site index x + Lx*(y + Ly*(z + Lz*t));
 *   - D_W psi(x) = (4 + m0) psi(x) - 1/2 sum_mu [(1 - g_mu) U_mu(x) psi(x+mu)
 *                  + (1 + g_mu) U_mu(x-mu)^dag psi(x-mu)] + (i c_sw/32) sum_{mu!=nu} sigma_mu_nu
 *                  (Q_mu_nu - Q_nu_mu) psi(x), with m0 = 1/(2 kappa) - 4 and a Euclidean chiral
 *                  gamma basis in which g5 = diag(1, 1, -1, -1);
 *   - periodic in space; the time boundary sign t_bc multiplies every hop across t = T-1 <-> 0;
 *   - host/device vectors exchanged through this ABI are FP64 complex, interleaved (re, im), in
 *     lexicographic site order: a fine spinor is [V][4 spins][3 colours], a gauge field is
 *     [V][4 directions][3][3] (row-major), a coarse vector is [V_c][2 N_v] with the coarse sites in
 *     lexicographic order of the aggregate coordinates and dofs ordered [+: 0..N_v-1, -: 0..N_v-1].
 *
 * Ownership and errors: the library copies what it keeps (gauge field, test vectors).  Caller
 * buffers are only read or written during a call.  `where` selects host (TMG_HOST, pageable or
 * pinned memory; the call copies and synchronises) or device pointers (TMG_DEVICE, memory on the
 * context's device; the call is stream-ordered on the context stream and returns without a
 * host synchronisation unless it has to read a scalar back).  Every call returns a tmg_status;
 * no call aborts, traps or prints.  tmg_last_error() gives the text of the last failure.  A
 * context is not thread-safe.
 */
#ifndef TMG_H
#define TMG_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct tmg_ctx tmg_ctx;

typedef enum {
  TMG_OK = 0,
  TMG_ERR_ARG = -1,       /* invalid argument, unsupported geometry or size */
  TMG_ERR_CUDA = -2,      /* a CUDA runtime call failed (text in tmg_last_error) */
  TMG_ERR_OOM = -3,       /* device allocation failed */
  TMG_ERR_NOCONV = -4,    /* solver hit its iteration cap; x holds the last iterate */
  TMG_ERR_BREAKDOWN = -5, /* NaN/Inf or Krylov breakdown detected */
  TMG_ERR_TIMEOUT = -6,   /* a bounded device-side wait gave up */
  TMG_ERR_STATE = -7      /* call out of order (e.g. solve before setup) */
} tmg_status;

enum { TMG_PREC_F64 = 0, TMG_PREC_F32 = 1, TMG_PREC_F16 = 2 };
enum { TMG_HOST = 0, TMG_DEVICE = 1 };

/* operators for tmg_apply */
enum {
  TMG_OP_D = 0,      /* y = D(mu) x                          (Sec. 1.1)            */
  TMG_OP_DDAG = 1,   /* y = D(mu)^dag x = G5 D(-mu) G5 x     (Sec. 1.1)            */
  TMG_OP_DND = 2,    /* y = D_ND(mubar, epsbar) x, x = [2 flavours][V][4][3] (Eq. 2) */
  TMG_OP_HOP = 3,    /* y = hopping term only (for tests and bandwidth runs)        */
  TMG_OP_DHAT = 4,   /* y_o = Dhat(mu) x_o, the even-odd reduced operator on the odd
                        sites, Dhat = M_o - H_oe M_e^-1 H_eo with M = A + i mu g5 the
                        site-local part and H the hopping part of D (Sec. 1.2 runs on the
                        even-odd reduced operator); x, y full-lattice fields of which the
                        odd sites (x + y + z + t odd) are read / written, y zero on the
                        even sites; F64 (12-real links) or F32 (8-real links) only; Lx even */
  TMG_OP_DHAT_DAG = 5 /* y_o = Dhat(mu)^dag x_o = g5 Dhat(-mu) g5 x_o, same conventions */
};

/* Create a context for a Lx x Ly x Lz x T lattice on `device`.  `block` is the SAP block, which is
 * also the fine-level aggregate: every dim must divide the lattice, the number of blocks along
 * every direction must be even and >= 2, and the block volume must be a multiple of 32 and
 * <= 256 (one CTA of one thread per site works on a block).  `stream` is a cudaStream_t (NULL: the legacy default stream).  Section 1.1 of the
 * paper uses lattice blocks both as SAP domains and as aggregates. */
int tmg_create(tmg_ctx **ctx, const int dims[4], const int block[4], int device, void *stream);
int tmg_destroy(tmg_ctx *ctx);
const char *tmg_last_error(const tmg_ctx *ctx);
/* Library version string; needs no context. */
const char *tmg_version(void);

/* Load the gauge field U (FP64, [V][4][3][3] complex) and set the time boundary sign t_bc
 * (+1 periodic, -1 antiperiodic).  Rebuilds the clover field on the device (Sec. 1.1: the
 * clover-improved operator) and the FP32 / FP16 copies of links and clover.  Every link must be
 * in SU(3) (the compressed formats rebuild the third row from the first two): a link with
 * max(|U U^dag - 1|, |det U - 1|) > TMG_SU3_TOL, or a non-finite entry, returns TMG_ERR_ARG
 * (the message names the site and direction) and leaves the loaded field unchanged. */
#define TMG_SU3_TOL 1e-8
int tmg_load_gauge(tmg_ctx *ctx, const double *U, int where, int t_bc);

/* Host-only SU(3) check (needs no context and no GPU): the largest defect
 * max(|U U^dag - 1|_max, |det U - 1|) over n_links FP64 links ([n_links][3][3] complex, host
 * memory) into *worst and the index of that link into *worst_index (either may be NULL).
 * TMG_OK if it is <= TMG_SU3_TOL, TMG_ERR_ARG otherwise or for a NULL U / negative count. */
int tmg_check_links(const double *U, long long n_links, double *worst, long long *worst_index);

/* Operator parameters: kappa (m0 = 1/(2 kappa) - 4), c_sw, the twist mu (Sec. 1.1) and the
 * non-degenerate doublet's mubar, epsbar (Eq. 2).  Must precede tmg_load_gauge's clover build or
 * be followed by it: changing kappa or c_sw rebuilds the clover field if a gauge field is loaded. */
int tmg_set_params(tmg_ctx *ctx, double kappa, double csw, double mu, double mubar, double epsbar);

/* Shifted doublet (Sec. 3): every doublet operator of the context (TMG_OP_DND, the doublet SAP,
 * coarse operators and solves) becomes D_ND + i delta (G5 x tau1), so that (G5 x tau1) times it is
 * Q_ND + i delta and the shifted systems Q_ND^2 + delta^2 = (Q_ND - i delta)(Q_ND + i delta) of the
 * rational approximation are two such solves.  delta = 0 (the default) is Eq. 2 itself. */
int tmg_set_ndshift(tmg_ctx *ctx, double delta);

/* y = op x for n_rhs fine spinors ([n_rhs][V][4][3], or [n_rhs][2][V][4][3] for TMG_OP_DND) in
 * the storage precision `prec` (inputs rounded to it; FP16 storage computes in FP32).  With
 * TMG_PREC_F16, D, D^dag and the hopping term keep every field in 16-bit fixed point: spinors with
 * one FP32 norm per site (the site's largest |component|; value = q / 32767 * norm, rounded to
 * nearest), links as two rows at scale 1, the clover field with a per-site scale (348 bytes per
 * site and application); the doublet operator in F16 keeps FP32 spinors.
 * mu_per_col (n_rhs values) overrides the twist per column; NULL uses the context's mu. */
int tmg_apply(tmg_ctx *ctx, int op, const double *x, double *y, int n_rhs,
              const double *mu_per_col, int prec, int where);

/* ---- multigrid (Eq. 1) ---- */
typedef struct tmg_mg_params {
  int nv;              /* test vectors N_v (coarse dofs per site = 2 N_v); 2..32 */
  int sap_sweeps;      /* k of Eq. 1 */
  int sap_mr;          /* MR steps per SAP block solve */
  int coarse_m;        /* max GMRES steps of the coarse solve (<= 64) */
  double coarse_rtol;  /* relative residual target of the coarse solve */
  int n_init;          /* initial SAP inverse-iteration passes of the setup */
  int n_iter;          /* adaptive setup iterations (cycle-based) */
  int restart;         /* outer FGMRES restart length (<= 64) */
  int prec_fine;       /* TMG_PREC_F64 / F32 / F16 for SAP, P, P^dag inside the cycle */
  int prec_coarse;     /* TMG_PREC_F64 / F32 for D_c and the coarse solve */
} tmg_mg_params;

/* Fill p with the defaults (nv 8, k 3, MR 4, coarse GMRES 30 / 5e-2, setup 5 + 3, restart 10,
 * fine F32, coarse F32). */
int tmg_mg_defaults(tmg_mg_params *p);

/* Adaptive setup (Sec. 1.1 and Sec. 2): start from the caller's N_v vectors v0 ([nv][V][4][3],
 * host or device per `where`), run n_init SAP inverse-iteration passes, build P and D_c, then
 * n_iter cycle-based setup iterations.  With n_init = n_iter = 0 the vectors only get
 * orthonormalised, which lets a caller impose a given P. */
int tmg_setup(tmg_ctx *ctx, const tmg_mg_params *p, const double *v0, int where);

/* Copy out the orthonormalised test vectors W ([nv][V][4][3] FP64) that define P. */
int tmg_get_vectors(tmg_ctx *ctx, double *W, int where);

/* Pieces of the cycle, each in precision `prec` (fine) or the coarse precision:
 *   tmg_sap:      x <- k SAP sweeps on D x = b starting from the given x (Eq. 1: M);
 *   tmg_restrict: c = P^dag r;  tmg_prolong: e = P c;
 *   tmg_coarse_apply: y = D_c(mu) x on coarse vectors ([V_c][2 N_v]);
 *   tmg_cycle:    z = one application of the preconditioner of Eq. 1 to r (zero start). */
int tmg_sap(tmg_ctx *ctx, const double *b, double *x, int prec, int where);
int tmg_restrict(tmg_ctx *ctx, const double *r, double *c, int prec, int where);
int tmg_prolong(tmg_ctx *ctx, const double *c, double *e, int prec, int where);
int tmg_coarse_apply(tmg_ctx *ctx, const double *x, double *y, double mu, int prec, int where);
int tmg_cycle(tmg_ctx *ctx, const double *r, double *z, int where);
/* Multi-RHS coarse operator Y = D_c(mu_n) X (Eq. 1's D_c, twist per column, Sec. 1.1) for
 * n_rhs (1..32) coarse vectors ([n_rhs][V_c][2 N_v]) on the tensor cores (tcgen05, split TF32,
 * FP32-level accuracy), N_v one of 4, 8, 12, 16, 24, 32 (compiled tile shapes; TMG_ERR_ARG
 * otherwise).  TMG_ERR_TIMEOUT if a bounded device-side wait gave up. */
int tmg_coarse_apply_multi(tmg_ctx *ctx, const double *x, double *y, int n_rhs, const double *mu_per_col, int where);
/* x ~= D_c(mu)^-1 b (Eq. 1's coarse solve): GMRES from zero with at most coarse_m steps, stopping
 * at relative residual coarse_rtol; coarse vectors [V_c][2 N_v], computed in precision prec. */
int tmg_coarse_solve(tmg_ctx *ctx, const double *b, double *x, double mu, int prec, int where);
/* X[n] ~= D_c(mu_n)^-1 B[n] for n_rhs (1..32) coarse right-hand sides [n_rhs][V_c][2 N_v] in
 * lock-step (the coarse solve of the batched cycle, Sec. 1.2's multiple right-hand sides): GMRES
 * from zero per column with its own Givens rotations and stopping test (coarse_m, coarse_rtol),
 * FP32 vectors and FP64 reductions.  With "batched_coarse_tc" on (the default) and N_v one of 4,
 * 8, 12, 16, 24, 32, D_c is applied to all columns at once on the tensor cores (as
 * tmg_coarse_apply_multi); otherwise by one persistent CUDA-core kernel.  mu_per_col may be NULL
 * (every column takes the context's mu).  Synchronises.  TMG_ERR_STATE before tmg_setup,
 * TMG_ERR_ARG for a bad count or pointer, TMG_ERR_TIMEOUT if a tensor-core completion wait gave
 * up. */
int tmg_coarse_solve_multi(tmg_ctx *ctx, const double *b, double *x, int n_rhs, const double *mu_per_col, int where);

/* ---- third level (Sec. 1.2 runs the method with three levels) ----
 * The level-1 operator D_c is aggregated again: level-2 aggregates are agg[0..3] blocks of
 * level-1 sites (x, y, z, t; each must divide the level-1 lattice), the level-2 basis P2 holds nv
 * level-1 vectors split by level-1 chirality (G5_c-compatible like P, so the twist stays
 * i mu G5 on level 2), orthonormalised per (aggregate, chirality) by modified Gram-Schmidt twice
 * in FP64.  D_cc = P2^dag D_c P2 is a 9-point stencil of [2 nv]^2 blocks (twist excluded).
 * Once built, the coarse solve of every cycle (tmg_cycle, tmg_solve, tmg_force) becomes the
 * level-1 K-cycle: FGMRES on D_c (at most k_restart steps, stop at k_rtol) preconditioned by the
 * level-1 cycle z = P2 D_cc^-1 P2^dag r (level-2 GMRES, coarse_m / coarse_rtol) followed by
 * smooth_m GMRES steps on D_c(mu) e = r - D_c z.  The whole K-cycle runs as one persistent kernel
 * in the multigrid's coarse precision. */
typedef struct {
  int agg[4];          /* level-2 aggregate in level-1 sites */
  int nv;              /* level-2 test vectors per chirality (2 nv <= 64, nv <= agg volume x N_v) */
  int smooth_m;        /* GMRES steps of the level-1 smoother (1..64) */
  int k_restart;       /* maximum FGMRES steps of the K-cycle (1..16) */
  double k_rtol;       /* relative residual target of the K-cycle */
  int coarse_m;        /* maximum level-2 GMRES steps (1..64) */
  double coarse_rtol;  /* relative residual target of the level-2 GMRES */
  int n_init;          /* initial smoother passes of the level-2 setup */
  int n_iter;          /* level-1 cycle-based setup iterations */
} tmg_level2_params;

/* Defaults: agg 2^4, nv 8, smoother 3 steps, K-cycle 10 steps / 0.1, level-2 GMRES 30 / 5e-2,
 * setup 5 + 3. */
int tmg_level2_defaults(tmg_level2_params *p);

/* Level-2 setup after tmg_setup, applied to D_c exactly like the fine setup is applied to D: from
 * the caller's nv level-1 vectors v1 ([nv][V_c][2 N_v] complex FP64, host or device), n_init
 * passes of v <- smoother(v) with normalisation, build P2 and D_cc, then n_iter passes of
 * v <- level-1 cycle(v) with normalisation and a rebuild.  A later tmg_setup drops level 2. */
int tmg_setup_level2(tmg_ctx *ctx, const tmg_level2_params *p, const double *v1, int where);

/* Copy out the orthonormalised level-2 basis ([nv][V_c][2 N_v] FP64). */
int tmg_get_vectors2(tmg_ctx *ctx, double *W2, int where);

/* Level-2 pieces in precision prec (F64 / F32): c2 = P2^dag c ([V_c2][2 nv] from [V_c][2 N_v]),
 * e = P2 c2, y = D_cc(mu) x. */
int tmg_restrict2(tmg_ctx *ctx, const double *c, double *c2, int prec, int where);
int tmg_prolong2(tmg_ctx *ctx, const double *c2, double *e, int prec, int where);
int tmg_coarse_apply2(tmg_ctx *ctx, const double *x, double *y, double mu, int prec, int where);

/* The level-1 K-cycle kernel on a level-1 vector b ([V_c][2 N_v]) in precision prec:
 * mode 0: x ~= D_c(mu)^-1 b (the three-level coarse solve); mode 1: x = level-1 cycle of b;
 * mode 2: x = smoother of b from zero (smooth_m GMRES steps). */
int tmg_kcycle(tmg_ctx *ctx, const double *b, double *x, double mu, int mode, int prec, int where);

/* The same K-cycle (modes 0 / 1 / 2, FP32) for n_rhs level-1 vectors b[n_rhs][V_c][2 N_v] in
 * lock-step, column n with twist mu_per_col[n] (or the context's mu when mu_per_col is NULL): the
 * coarse solve of the three-level batched solve.  Every D_c and D_cc application covers all columns
 * in one tensor-core launch; Gram-Schmidt, Givens rotations and stopping tests are per column, as
 * in tmg_kcycle.  Needs 1..32 columns and 2 N_v, 2 nv in {8, 16, 24, 32, 48, 64}.  Synchronises.
 * TMG_ERR_STATE before tmg_setup_level2, TMG_ERR_ARG for a bad count, mode, shape or pointer,
 * TMG_ERR_TIMEOUT if a tensor-core completion wait gave up. */
int tmg_kcycle_multi(tmg_ctx *ctx, const double *b, double *x, int n_rhs, const double *mu_per_col, int mode, int where);

/* ---- the non-degenerate doublet (Eq. 2, coarsened with P_ND = P x I2 as in Sec. 1.2) ----
 * Doublet vectors are flavour pairs: fine [2][V][4][3], coarse [2][V_c][2 N_v].  The operator
 * parameters are the context's mubar and epsbar; P (and P2 with three levels) come from the
 * single-flavour setup, which a caller runs with mu = mubar (the flavour-diagonal part of D_ND).
 *   tmg_sap_nd:          x <- k SAP sweeps on D_ND x = b (block MR on the flavour-coupled
 *                        Dirichlet block operator) starting from the given x;
 *   tmg_coarse_apply_nd: y = D_ND,c x = (D_c x I2 + i mubar G5_c x tau3 - epsbar I x tau1) x;
 *   tmg_coarse_solve_nd: x ~= D_ND,c^-1 b by the coarse GMRES of the cycle (with three levels
 *                        use tmg_kcycle_nd);
 *   tmg_kcycle_nd:       the level-1 K-cycle kernel on doublet level-1 vectors (modes as
 *                        tmg_kcycle);
 *   tmg_cycle_nd:        z = one doublet preconditioner cycle of r. */
int tmg_sap_nd(tmg_ctx *ctx, const double *b, double *x, int prec, int where);
int tmg_coarse_apply_nd(tmg_ctx *ctx, const double *x, double *y, int prec, int where);
int tmg_coarse_solve_nd(tmg_ctx *ctx, const double *b, double *x, int prec, int where);
int tmg_kcycle_nd(tmg_ctx *ctx, const double *b, double *x, int mode, int prec, int where);
int tmg_cycle_nd(tmg_ctx *ctx, const double *r, double *z, int where);

/* ---- solves ---- */
typedef struct {
  int iterations;        /* outer FGMRES (or CG) iterations summed over restarts/refinements */
  int refinements;       /* FP64 defect-correction restarts */
  int coarse_iterations; /* coarse GMRES steps summed over all cycles */
  double true_residual;  /* ||b - D x|| / ||b|| in FP64 at exit */
  double seconds;        /* wall time of the call */
} tmg_stats;

enum {
  TMG_SOLVE_MG_F64 = 0,   /* FGMRES + DD-alpha-AMG, everything in FP64                     */
  TMG_SOLVE_MG_MIXED = 1, /* FP64 defect correction around FGMRES + DD-alpha-AMG in the MG   */
                          /* params' fine/coarse precisions                                 */
  TMG_SOLVE_CG_F64 = 2,   /* CG on D D^dag in FP64 (comparator of Sec. 1.1 / Fig. 1)       */
  TMG_SOLVE_MG_BATCHED = 3, /* as TMG_SOLVE_MG_MIXED, all n_rhs (<= 32) columns in lock-step: */
                          /* one launch per operation for every column, FP32 coarse level    */
  TMG_SOLVE_ND_F64 = 4,   /* doublet D_ND x = b (Eq. 2), b and x [n_rhs][2][V][4][3], multigrid */
                          /* with P_ND = P x I2 (Sec. 1.2), everything in FP64                */
  TMG_SOLVE_ND_MIXED = 5, /* the same with FP64 defect correction around the MG params'      */
                          /* fine/coarse precisions                                          */
  TMG_SOLVE_CG_EO = 6     /* odd-even CG (Fig. 1's comparator): FP64 CG on Dhat Dhat^dag for  */
                          /* the odd sites, rhs b_o - H_oe M_e^-1 b_e, then x_e = M_e^-1 (b_e */
                          /* - H_eo x_o); needs no multigrid setup; Lx even                   */
};

/* Solve D(mu) x = b (relative FP64 residual tol) for n_rhs right-hand sides, one after another.
 * mu_per_col may override the twist per column (the same P serves every mu, Sec. 1.1).
 * x is an output (zero initial guess).  maxiter bounds the outer iterations. */
int tmg_solve(tmg_ctx *ctx, const double *b, double *x, int n_rhs, const double *mu_per_col,
              double tol, int method, int maxiter, tmg_stats *stats, int where);

/* ---- force (the HMC force terms of Sec. 2 and 3, solves in the two-step form of Sec. 1.1) ----
 * S = phi^dag (D D^dag)^-1 phi = ||D(mu)^-1 phi||^2.  F[V][4][3][3] (complex, lexicographic sites,
 * direction, row, column) is the traceless Hermitian field with dS/dt = sum_{x,mu} tr(H F) under
 * U_mu(x) -> exp(i t H_mu(x)) U_mu(x).
 *   tmg_force_xy: F from X = D^-dag Y and Y = D^-1 phi given by the caller (FP64 fine spinors);
 *   tmg_force:    solves Y = D(mu)^-1 phi and X = g5 D(-mu)^-1 g5 Y with the mixed-precision
 *                 multigrid (tolerance tol, needs tmg_setup), returns S in *action (may be NULL). */
int tmg_force_xy(tmg_ctx *ctx, const double *X, const double *Y, double *F, int where);
int tmg_force(tmg_ctx *ctx, const double *phi, double *F, double tol, double *action, tmg_stats *stats, int where);

/* Link update U_mu(x) <- exp(i step sum_a omega_a(x, mu) lambda_a / 2) U_mu(x) (lambda_a the Gell-Mann
 * matrices; the left-multiplied su(3) variation in which the force below is defined, i.e. the
 * molecular-dynamics link update of the HMC of Sec. 2).  omega: [V][4][8] real FP64, lexicographic
 * sites, host or device per `where`.  Computed in FP64 on the device (exp by Taylor series with
 * scaling and squaring, the product projected back onto SU(3)); the clover field and the compressed
 * copies are rebuilt, and an existing multigrid keeps its P but gets D_c (and D_cc) rebuilt for
 * the new field.  A following tmg_setup_update adapts P itself. */
int tmg_rotate_gauge(tmg_ctx *ctx, const double *omega, double step, int where);

/* Setup update (Sec. 2: after the gauge field has changed, the previous subspace is refined by one
 * setup iteration instead of a new setup): n_iter passes of v_j <- normalise(cycle(v_j)) on the
 * current operator, starting from the test vectors the last tmg_setup kept, each followed by a
 * rebuild of P and D_c; with three levels the level-2 basis gets n_iter passes of the level-1
 * cycle too.  n_iter = 0 only rebuilds P and D_c.  TMG_ERR_STATE without an earlier setup. */
int tmg_setup_update(tmg_ctx *ctx, int n_iter);

/* Shifted systems D(mu_k) x_k = b, k = 0 .. n_shift-1 (1..64) in the given order, one right-hand side
 * b ([V][4][3]) and x [n_shift][V][4][3], each solved by the mixed-precision multigrid to the FP64
 * residual tol with the same P (Sec. 1.1: one P serves every twist).  guess selects the initial
 * guess of system k > 0: 0 zero, 1 the solution x_{k-1}, 2 the first-order Taylor expansion of
 * Sec. 3, (Q + i mu + i delta)^-1 ~ (Q + i mu)^-1 - i delta (Q + i mu)^-2 with g5 D(mu) = Q + i mu:
 * x_k^0 = x_{k-1} - i (mu_k - mu_{k-1}) D(mu_{k-1})^-1 g5 x_{k-1}, the correction solved only to the
 * relative residual taylor_tol.  iterations (may be NULL) gets n_shift outer-iteration counts of the
 * systems themselves; stats sums every solve, the Taylor corrections included.  Shifted normal
 * equations (D^dag D + sigma) map to twists mu_k = sqrt(mu^2 + sigma) (Sec. 1.1). */
int tmg_solve_shifts(tmg_ctx *ctx, const double *b, double *x, int n_shift, const double *mu, double tol, int guess,
                     double taylor_tol, int *iterations, tmg_stats *stats, int where);

/* Multi-shift CG (the MMS-CG of Sec. 3): x_s = (A + sigma_s)^-1 b for n_shift (1..64) shifts
 * sigma_s >= 0 at once, FP64, with A = D(mu)^dag D(mu) (flavours = 1; b [V][4][3], x
 * [n_shift][V][4][3]) or A = Q_ND^2 = D_ND^dag D_ND, Q_ND = (g5 x tau1) D_ND (flavours = 2, Eqs. 2
 * and 4; b [2][V][4][3], x [n_shift][2][V][4][3]).  One Krylov space (the seed system A) serves all
 * shifts.  Stops when every shifted residual is <= tol ||b||; stats: seed iterations and the
 * largest recomputed residual ||b - (A + sigma_s) x_s|| / ||b||.  Needs no multigrid setup. */
int tmg_mms_cg(tmg_ctx *ctx, const double *b, double *x, int n_shift, const double *sigma, double tol, int flavours,
               tmg_stats *stats, int where);

/* Rational function of A (the RHMC approximation R of Eq. 5, for 1/sqrt(Q_ND^2)):
 * out = a prod_{l=1..n} (A + num_l)(A + den_l)^-1 phi, n <= 32, distinct den_l >= 0, evaluated
 * through its partial fractions a (phi + sum_l r_l (A + den_l)^-1 phi).  The coefficients
 * (Zolotarev's for 1/sqrt(x)) come from the caller.  As in Sec. 3, the shifted systems are split
 * between two solvers: shifts den_l >= mg_below go to one multi-shift CG (above; mg_below <= 0 sends
 * every shift there), the smaller, worse-conditioned ones to the mixed-precision multigrid (needs
 * tmg_setup), two solves per shift: one flavour, D^dag D + q = D(mu_q)^dag D(mu_q) with
 * mu_q = sqrt(mu^2 + q); doublet, Q_ND^2 + q = (Q_ND - i d)(Q_ND + i d), d = sqrt(q), with
 * Q_ND +- i d = (g5 x tau1)(D_ND +- i d g5 x tau1) solved by the doublet multigrid (P_ND = P x I2).
 * Same A, flavours and tolerance; stats sum both solvers. */
int tmg_rational_apply(tmg_ctx *ctx, const double *phi, double *out, int n, double a, const double *num,
                       const double *den, double tol, int flavours, double mg_below, tmg_stats *stats, int where);

/* Pseudofermion action S = phi^dag (D D^dag)^-1 phi = ||Y||^2, Y = D(mu)^-1 phi (Sec. 1.1, the
 * monomials of Sec. 2): one mixed-precision multigrid solve to tolerance tol.  phi, Y: FP64 fine
 * spinors (Y is written).  Y is what tmg_pf_force needs: the force is recomputed from it rather
 * than kept from the action call. */
int tmg_pf_action(tmg_ctx *ctx, const double *phi, double *Y, double tol, double *S, tmg_stats *stats, int where);

/* Force of that action from Y: solves X = D(mu)^-dag Y = g5 D(-mu)^-1 g5 Y (the second step of the
 * two-step D^dag D solve of Sec. 1.1) and writes f[V][4][8] = tr(lambda_a / 2 F_mu(x)), the su(3)
 * coefficients of the traceless Hermitian F with dS/dt = sum tr(H F) under U -> exp(i t H) U, so
 * that dS/domega_a(x, mu) = f_a(x, mu) at omega = 0 for tmg_rotate_gauge's parametrisation.
 * Force kernels per "force_prec" (tmg_tune). */
int tmg_pf_force(tmg_ctx *ctx, const double *Y, double *f, double tol, tmg_stats *stats, int where);

/* sigma_min(D_W) = min |lambda(Q)|, Q = g5 D_W at mu = 0 (the smallest singular value of the Wilson-clover
 * operator that fixes kappa in the workloads; the hermitian Q of Sec. 2, Eq. 3): Lanczos with full
 * reorthogonalisation on (Q^2 + mu_s^2)^-1 = (D(mu_s)^dag D(mu_s))^-1, each product computed by the
 * two-step solve of Sec. 1.1 (D(-mu_s) u = g5 b, then D(mu_s) v = g5 u) with solver `method`
 * (TMG_SOLVE_MG_F64 / MG_MIXED / CG_F64) to relative residual solve_tol.  The largest Ritz value
 * theta gives sigma = sqrt(1/theta - mu_s^2).  start: FP64 fine spinor (host/device); at most
 * max_steps (2..64) Lanczos steps, stopping once the Ritz residual is <= rtol theta.  Writes sigma,
 * the last relative Ritz residual and the number of solves; TMG_ERR_NOCONV if rtol was not reached
 * (sigma still holds the estimate).  mu_s > 0 keeps every solve well posed; choose it near the
 * expected sigma (1/theta - mu_s^2 loses relative accuracy when mu_s >> sigma). */
int tmg_sigma_min(tmg_ctx *ctx, const double *start, double mu_s, int max_steps, double rtol, double solve_tol,
                  int method, double *sigma, double *ritz_res, int *solves, int where);

/* ---- HMC (Sec. 2) ----
 * One molecular-dynamics trajectory of the Hasenbusch-split twisted-mass HMC: det[Q^2 + mu^2] (Eq. 3)
 * written as fermion monomials m = 0 .. n_mono-1, each a ratio det[D(mu)^dag D(mu)] /
 * det[D(mu')^dag D(mu')] (mu2[m] = mu' > 0) or a last det[D(mu)^dag D(mu)] (mu2[m] = 0), with
 * pseudofermion actions ||D(mu)^-dag D(mu')^dag phi||^2 and ||D(mu)^-1 phi||^2, plus the Wilson
 * plaquette gauge action beta sum (1 - Re tr P / 3) (the paper does not print its gauge action).
 * Every fermion monomial sits on the time scale level[m] (0 = outermost) of a nested second-order
 * minimal-norm integrator with steps[l] steps per call of scale l; the gauge action is on the
 * innermost scale n_levels-1.  The heat bath draws phi from the caller's Gaussian eta ([n_mono][V][4][3]
 * complex, seeded by the caller); the momenta P ([V][4][8] real su(3) coefficients, the caller's
 * Gaussians) are updated in place and the context's gauge field is left at the end of the trajectory
 * (the accept / reject step and restoring the old field, tmg_get_gauge / tmg_load_gauge, are the
 * caller's).  Solves: mixed-precision DD-alpha-AMG (needs tmg_setup) to tol_action (heat bath,
 * Hamiltonian) and tol_force (forces) -- Sec. 2 uses 1e-11 and 1e-9; the setup is updated by
 * setup_iters_start iterations at the start and setup_iters_force before every force of the monomial
 * with the smallest mu (Sec. 2: 3 and 1).  Writes dH = H_end - H_start. */
typedef struct {
  double beta;            /* gauge coupling */
  double tau;             /* trajectory length */
  int n_mono;             /* fermion monomials, 1..8 */
  double mu[8];           /* twist of each monomial's D(mu) */
  double mu2[8];          /* mu' of a ratio monomial, 0 for a det monomial */
  int level[8];           /* time scale of each fermion monomial */
  int n_levels;           /* time scales (1..8); the gauge action is on the last */
  int steps[8];           /* minimal-norm steps per call of each time scale */
  double tol_action;      /* heat bath and Hamiltonian solves */
  double tol_force;       /* force solves */
  int setup_iters_start;  /* setup-update iterations at the start (0: none) */
  int setup_iters_force;  /* setup-update iterations before each force of the lightest monomial */
  int keep_phi;           /* 1: skip the heat bath and reuse the pseudofermions of the context's
                             previous trajectory (eta unused; for reversibility checks) */
} tmg_hmc_params;

typedef struct {
  double H_start, H_end;  /* Hamiltonians (kinetic + gauge + fermion actions) */
  long long solves;       /* multigrid solves */
  long long outer_iterations;
  long long fermion_forces, gauge_forces, link_updates;
  double seconds;
} tmg_hmc_stats;

int tmg_hmc_trajectory(tmg_ctx *ctx, const tmg_hmc_params *p, double *P, const double *eta, double *dH,
                       tmg_hmc_stats *stats, int where);

/* Copy out the context's gauge field ([V][4][3][3] FP64 complex, lexicographic), e.g. to restore it
 * with tmg_load_gauge after a rejected trajectory. */
int tmg_get_gauge(tmg_ctx *ctx, double *U, int where);

/* Wilson plaquette action beta sum_{x, mu<nu} (1 - Re tr P_mu_nu(x) / 3) of the context's field, and
 * its force as su(3) coefficients f[V][4][8] = tr(lambda_a / 2 F), dS/dt = sum tr(H F) under
 * U -> exp(i t H) U. */
int tmg_gauge_action(tmg_ctx *ctx, double beta, double *S);
int tmg_gauge_force(tmg_ctx *ctx, double beta, double *f, int where);

/* Time `n_iter` back-to-back launches of the dslash kernel (y = D x, one column, storage
 * precision prec as in tmg_apply, so TMG_PREC_F16 is the all-FP16 form) on the context stream with
 * CUDA events; writes the mean milliseconds per launch.  Inputs are the library's internal fields (random data is not needed: the timing
 * does not depend on values). */
int tmg_bench_dslash(tmg_ctx *ctx, int prec, int n_iter, double *ms_per_launch);

/* Time `n_iter` back-to-back applications of the even-odd reduced operator Dhat (the two kernels of
 * one application; F64 with 12-real links or F32 with 8-real links) on the context stream with CUDA
 * events; writes the mean milliseconds per application. */
int tmg_bench_schur(tmg_ctx *ctx, int prec, int n_iter, double *ms_per_application);

/* Coarse solve that allocates nothing, for callers that cannot call cudaMalloc: code running
 * under CUDA stream capture, hosts whose memory manager forbids allocation on the call path, and
 * latency-critical loops.  (No counterpart in the paper: an interface addition.)  Same result as
 * tmg_coarse_solve, but b and x are DEVICE pointers to FP64 coarse vectors ([V_c][2 N_v] complex,
 * caller-owned) and all scratch comes from one fixed 32 MiB device array inside the library that
 * every GPU loading the library keeps until the process exits.  A coarse problem whose scratch
 * ((coarse_m + 13) x V_c x 2 N_v complex values plus partial sums) does not fit returns
 * TMG_ERR_ARG.  The first call on a device looks up the array's device address, so make it before
 * any stream capture.  Calls share the array: calls that overlap on the GPU race.  Stream-ordered
 * on the context stream; no host synchronisation. */
int tmg_coarse_solve_noalloc(tmg_ctx *ctx, const double *b, double *x, double mu, int prec);

/* Kernel classes timed by tmg_profile (CUDA events around every launch of the class, on the
 * context stream).  Not a paper quantity: measurement support. */
enum {
  TMG_PK_DSLASH_F64 = 0, TMG_PK_DSLASH_F32 = 1, TMG_PK_DSLASH_F16 = 2,
  TMG_PK_SAP_F64 = 3, TMG_PK_SAP_F32 = 4, TMG_PK_SAP_F16 = 5,
  TMG_PK_RESTRICT = 6, TMG_PK_PROLONG = 7, TMG_PK_COARSE = 8, TMG_PK_COARSE_SOLVE = 9,
  TMG_PK_EO_F64 = 10, TMG_PK_EO_F32 = 11, TMG_PK_COUNT = 12
};
/* enable != 0: reset the records and start timing every launch of the classes above;
 * enable == 0: stop (records are kept until the next call). */
int tmg_profile(tmg_ctx *ctx, int enable);
/* Launches recorded for class `kind` and their summed device time in milliseconds. */
int tmg_profile_read(tmg_ctx *ctx, int kind, long long *count, double *ms_total);

/* Launch-shape knobs (not paper quantities): "coarse_ctas_per_sm" (1..8, CTAs per SM of the
 * persistent coarse GMRES, capped by occupancy) and "coarse_gs_passes" (1 or 2 classical
 * Gram-Schmidt passes in the coarse GMRES; 0 = 1 in FP32, 2 in FP64), "kcycle_ctas_per_sm" (1..4,
 * CTAs per SM of the persistent level-1 K-cycle), "cycle_graph" (1, the default: the preconditioner
 * cycle inside the outer FGMRES is captured once per set of buffers and parameters as a CUDA graph
 * and replayed with one launch; 0: launched kernel by kernel), "tc_steps_per_range" (1, 2 or 4 K = 8
 * steps accumulated in one tensor-memory range by tmg_coarse_apply_multi; 1 keeps FP32-level
 * accuracy for any N_v), "tc_pipeline" (1, the default: for 2 N_v <= 32 the tensor-core apply stacks
 * the hi and lo TF32 parts of each stencil block in one 128-row operand and the columns' parts in one
 * operand, one MMA per K step, with double-buffered shared and tensor memory; 0: the unstacked
 * kernel, three MMAs per K step), "coarse_grid" / "kcycle_grid" (absolute CTA count of the persistent coarse
 * GMRES / K-cycle, capped by residency; 0 = the per-SM knobs), "outer_gs_fused" (1, the default:
 * the outer FGMRES's first Gram-Schmidt update and second set of dot products share one sweep over
 * the basis for up to 10 basis vectors; 0: separate kernels), "outer_gs_passes" (1, the default, or 2:
 * classical Gram-Schmidt passes of the outer FGMRES and of the batched solve), "coarse_overlap" (1, the default: the coarse GMRES updates the Hessenberg
 * column of step j on one warp per CTA while the other warps run the stencil of step j+1; 0: the
 * update follows each step and all warps run the stencil), "batched_coarse_tc" (1, the default: the
 * two-level batched solve's coarse GMRES applies D_c to all columns at once on the tensor cores,
 * tcgen05 split TF32 as tmg_coarse_apply_multi, two launches per Arnoldi step; 0: one persistent
 * CUDA-core kernel), "coarse_block_cache" (1, the default: each CTA of the persistent coarse GMRES
 * copies as many of its own coarse sites' stencil blocks as fit into shared memory once per solve,
 * with one bounded bulk copy, and reads them from there at every step; 0: every step reads the
 * stencil from L2), "coarse_eo" (0, the default, or 1: the coarse GMRES of the single-flavour
 * cycle solves the odd-even reduced system S x_o = b_o - A_oe A_ee^-1 b_e, S = A_oo - A_oe A_ee^-1
 * A_eo, with per-site inverses (A_self + i mu G5_c)^-1 computed on the GPU for each twist and kept
 * for up to 16 (twist, precision) pairs, then sets x_e = A_ee^-1 (b_e - A_eo x_o); needs even
 * coarse extents, else the plain form runs; not a construction of the paper; the allocation-free
 * tmg_coarse_solve_noalloc keeps the plain form), "batched_coarse_m" (0, the default: the batched
 * solve's coarse GMRES takes at most coarse_m steps; 1..64: at most that many, e.g. when coarse_m
 * is sized for the odd-even reduced single-column solve), "eo_stage" (1, the default: the FP32 even-odd kernels copy
 * each CTA's tile of the clover field / clover inverse into shared memory with bulk copies while
 * the neighbour loads run; 0: direct loads), "force_prec" (TMG_PREC_F64, the default: the force kernels of
 * tmg_force / tmg_force_xy / tmg_pf_force read FP64 X, Y and links; TMG_PREC_F32: they read FP32
 * copies of X, Y and the 12-real FP32 links and sum every product in FP64; F is returned in FP64
 * either way).  TMG_ERR_ARG for an unknown key or
 * value. */
int tmg_tune(tmg_ctx *ctx, const char *key, double value);

/* Autotuner (not a paper quantity): after tmg_setup (and tmg_setup_level2), time the coarse solve of
 * the cycle for every allowed launch shape ("coarse_ctas_per_sm" x "coarse_gs_passes", or with
 * three levels "kcycle_ctas_per_sm") on a fixed right-hand side with the stopping test disabled,
 * keep the fastest shape in the context and write its time per coarse solve (ms) to *best_ms
 * (may be NULL).  CUDA events on the context stream; synchronises. */
int tmg_autotune(tmg_ctx *ctx, double *best_ms);

/* Number of preconditioner-cycle CUDA graphs the context holds (0 when "cycle_graph" is off or
 * capture is not available). */
int tmg_graph_count(const tmg_ctx *ctx, int *n);

/* Number of CUDA kernels this context has launched so far (every launcher counts its launches;
 * lets a caller count the kernels inside a timed region).  Not a paper quantity. */
int tmg_launch_count(const tmg_ctx *ctx, long long *n);

#ifdef __cplusplus
}
#endif
#endif /* TMG_H */
