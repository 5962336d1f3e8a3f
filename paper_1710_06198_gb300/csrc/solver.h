// Host-side solver runtime of libtmg (internal): adaptive setup, the DD-alpha-AMG cycle of Eq. 1,
// the device-resident coarse GMRES, the outer flexible GMRES with FP64 defect correction, and the
// FP64 CG comparator.
#pragma once
#include "tmg_host.h"

namespace tmg {

struct SolveStats {
  int iterations = 0;
  int refinements = 0;
  int coarse_iterations = 0;
  double true_residual = 0.0;
};

// Adaptive setup from nv FP64 lexicographic vectors on the device (Sec. 1.1, Sec. 2).
void mg_setup(Ctx& c, const double* v0_lex);
// Setup update after the gauge field changed: n_iter cycle-based iterations from the kept vectors.
void mg_setup_update(Ctx& c, int n_iter);
// Level-2 setup (three levels) from nv2 FP64 level-1 vectors on the device, parameters in c.l2p.
void mg_setup2(Ctx& c, const double* v1_dev);
// z = M_MG r in the fine storage precision of the multigrid parameters (r is not modified).
void mg_cycle(Ctx& c, const void* r, void* z, double mu);
// Solve D(mu) x = b on FP64 internal fields (b, x: F64 storage).  Returns a tmg_status.
// nf = 2: the doublet D_ND (Eq. 2) on F64 fields [2][12 V] (mu unused; mubar, epsbar of the context).
// use_x0: x holds the initial guess (multigrid methods; CG always starts from zero).
int solve_one(Ctx& c, int method, const void* b, void* x, double mu, double tol, int maxiter, SolveStats& st,
              int nf = 1, bool use_x0 = false);
// D(c.mu) x = b by the odd-even CG on the Schur operator (FP64); b, x lexicographic on the device.
int cg_eo_solve(Ctx& c, const double* b_lex, double* x_lex, double tol, int maxiter, SolveStats& st);
// Multi-shift CG on A + sigma_s, A = D^dag D (nf = 1) or Q_ND^2 (nf = 2), FP64 internal fields.
int mms_cg_solve(Ctx& c, const void* b, void* X, int ns, const double* sigma, double tol, int maxiter, int nf,
                 SolveStats& st);
// Shifted systems D(mu_k) x_k = b in order with zero / previous-solution / first-order Taylor
// initial guesses (guess 0 / 1 / 2); see solver.cu.
int solve_shifts(Ctx& c, const void* b, void* X, int n, const double* mu, double tol, int guess, double taylor_tol,
                 int maxiter, SolveStats& st, int* iters);
// sigma_min(D_W) by Lanczos on (D(mu_s)^dag D(mu_s))^-1 from the FP64 field `start` (two solves of
// method `method` per step, to solve_tol); see solver.cu.
double sigma_min_lanczos(Ctx& c, const void* start, double mu_s, int k, double rtol, double solve_tol, int method,
                         double* ritz_res, int* solves, int* steps);
// HMC (hmc.cu): one trajectory on device momenta P_dev and Gaussians eta (lexicographic FP64)
int hmc_trajectory(Ctx& c, const tmg_hmc_params& p, double* P_dev, const double* eta_lex_dev, double* dH,
                   tmg_hmc_stats* stats);
double gauge_action(Ctx& c, double beta);
void gauge_force(Ctx& c, double beta, double* f_lex);
// clover, compressed copies, even-odd data and coarse operators after the links changed
void gauge_changed(Ctx& c);
// Launch-shape autotuner of the coarse solve (coarse_ctas_per_sm, coarse_gs_passes; with three
// levels kcycle_ctas_per_sm); keeps the fastest shape, returns its time per coarse solve in ms.
double autotune(Ctx& c);
// z = doublet cycle of r (fields [2][12 V] in the fine storage precision)
void mg_cycle_nd(Ctx& c, const void* r, void* z);
// ncol systems D(mu_c) x_c = b_c (F64 fields, column c at c * 12 V) solved in lock-step.
int solve_batched(Ctx& c, int ncol, const void* b, void* x, const double* mu, double tol, int maxiter, SolveStats& st);

}  // namespace tmg
