// Hasenbusch-split HMC trajectory (Sec. 2 of arXiv:1710.06198): det[Q^2 + mu^2] split into ratios
// det[(Q^2 + mu_i^2)/(Q^2 + mu'_i^2)] and a last det[Q^2 + mu_N^2] (Eq. 3), every fermion monomial on
// its own time scale of a nested second-order minimal-norm integrator with the gauge action
// innermost, the solves by the mixed-precision DD-alpha-AMG of this library, and the multigrid
// setup updated during the trajectory (three setup iterations at its start, one before every force
// of the lightest monomial, Sec. 2).  With Q^2 + m^2 = D(m)^dag D(m):
//   det:   S = ||D(mu)^-1 phi||^2,               F from (X, Y) = (D^-dag Y, D^-1 phi);
//   ratio: S = ||D(mu)^-dag D(mu')^dag phi||^2,  F from (Y - phi, X), Y = D(mu)^-dag D(mu')^dag phi,
//          X = D(mu)^-1 Y  (dS/dt = 2 Re (phi - Y)^dag (dD/dt) X);
//   gauge: S_g = beta sum_{x, mu<nu} (1 - Re tr P_mu_nu / 3) (Wilson plaquette action),
//          F = (beta / 3) TH[(W - W^dag) / (2 i)], W = U_mu(x) x (its six staples).
// Momenta P[V][4][8] (lexicographic sites, su(3) coefficients), kinetic energy sum P_a^2 / 2,
// P -= e f with f_a = tr(lambda_a / 2 F); the link update U <- exp(i t P) U is tmg_rotate_gauge's
// kernel.  One minimal-norm step of size e on a time scale:
//   P -= lam e f; inner(e / 2); P -= (1 - 2 lam) e f; inner(e / 2); P -= lam e f.
#include <chrono>
#include <cmath>
#include <vector>

#include "solver.h"

namespace tmg {

namespace {

constexpr double kLambdaMN = 0.1931833275037836;

struct M3d { cpx<double> m[9]; };

__device__ __forceinline__ M3d ld_link(const Geom& g, const double2* __restrict__ U, int s, int mu) {
  M3d r;
#pragma unroll
  for (int k = 0; k < 9; k++) { const double2 v = U[(size_t)(mu * 9 + k) * g.V + s]; r.m[k] = {v.x, v.y}; }
  return r;
}
__device__ __forceinline__ M3d mm(const M3d& a, const M3d& b) {
  M3d r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) r.m[3 * i + j] = a.m[3 * i] * b.m[j] + a.m[3 * i + 1] * b.m[3 + j] + a.m[3 * i + 2] * b.m[6 + j];
  return r;
}
__device__ __forceinline__ M3d dg(const M3d& a) {
  M3d r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) r.m[3 * i + j] = conj(a.m[3 * j + i]);
  return r;
}

// per-CTA partial sums of sum_{mu<nu} (1 - Re tr P_mu_nu(x) / 3)
__global__ void k_plaquette_sum(Geom g, const double2* __restrict__ U, double* __restrict__ part) {
  double acc = 0.0;
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int c[4];
    site_coords(g, s, c);
    for (int mu = 0; mu < 4; mu++)
      for (int nu = mu + 1; nu < 4; nu++) {
        const M3d a = ld_link(g, U, s, mu), b = ld_link(g, U, neighbour(g, c, mu, +1), nu);
        const M3d cc = ld_link(g, U, neighbour(g, c, nu, +1), mu), d = ld_link(g, U, s, nu);
        const M3d P = mm(mm(a, b), mm(dg(cc), dg(d)));
        acc += 1.0 - (P.m[0].re + P.m[4].re + P.m[8].re) / 3.0;
      }
  }
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
    part[blockIdx.x] = t;
  }
}

// f[lex][mu][8] of the Wilson gauge force, (beta / 3) TH[(W - W^dag) / (2 i)]
__global__ void k_gauge_force(Geom g, const double2* __restrict__ U, double beta, double* __restrict__ f) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  M3d S;
  for (int k = 0; k < 9; k++) S.m[k] = mk(0.0, 0.0);
  const int sp = neighbour(g, c, mu, +1);
  for (int nu = 0; nu < 4; nu++) {
    if (nu == mu) continue;
    const int sn = neighbour(g, c, nu, +1), sm = neighbour(g, c, nu, -1);
    int cm[4];
    site_coords(g, sm, cm);
    const int spm = neighbour(g, cm, mu, +1);   // x + mu - nu
    const M3d up = mm(mm(ld_link(g, U, sp, nu), dg(ld_link(g, U, sn, mu))), dg(ld_link(g, U, s, nu)));
    const M3d lo = mm(mm(dg(ld_link(g, U, spm, nu)), dg(ld_link(g, U, sm, mu))), ld_link(g, U, sm, nu));
    for (int k = 0; k < 9; k++) S.m[k] = S.m[k] + up.m[k] + lo.m[k];
  }
  const M3d W = mm(ld_link(g, U, s, mu), S);
  cpx<double> h[9];
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      // (W - W^dag) / (2 i) entry (i, j) = (W_ij - conj(W_ji)) / (2 i)
      const cpx<double> d = W.m[3 * i + j] - conj(W.m[3 * j + i]);
      h[3 * i + j] = mk(0.5 * d.im, -0.5 * d.re);
    }
  const double tr = (h[0].re + h[4].re + h[8].re) / 3.0;
  h[0].re -= tr;
  h[4].re -= tr;
  h[8].re -= tr;
  double a[8];
  algebra_coeffs(h, a);
  const size_t lex = lex_index(g, c);
  for (int k = 0; k < 8; k++) f[(lex * 4 + mu) * 8 + k] = (beta / 3.0) * a[k];
}

int grid_of(const Ctx& c, size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, (size_t)c.sms * 8)); }

}  // namespace

double gauge_action(Ctx& c, double beta) {
  const int G = grid_of(c, c.g.V);
  DBuf part;
  part.alloc(G * sizeof(double));
  ++c.launches, k_plaquette_sum<<<G, 256, 0, c.stream>>>(c.g, c.op[0].U.as<double2>(), part.as<double>());
  TMG_CHECK_LAUNCH();
  std::vector<double> h(G);
  TMG_CUDA(cudaMemcpyAsync(h.data(), part.p, G * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  TMG_CUDA(cudaStreamSynchronize(c.stream));
  double s = 0.0;
  for (double v : h) s += v;
  return beta * s;
}

void gauge_force(Ctx& c, double beta, double* f_lex) {
  ++c.launches, k_gauge_force<<<dim3((c.g.V + 127) / 128, 4), 128, 0, c.stream>>>(c.g, c.op[0].U.as<double2>(), beta, f_lex);
  TMG_CHECK_LAUNCH();
}

// After the links moved: clover, compressed copies, even-odd data and the coarse operators.
void gauge_changed(Ctx& c) {
  build_clover(c);
  convert_op_precisions(c);
  c.eo.ready = false;
  if (c.mg_ready) {
    build_coarse(c);
    if (c.l2_ready) build_coarse_c(c);
  }
}

namespace {

struct Hmc {
  Ctx& c;
  const tmg_hmc_params& p;
  size_t n;          // complex numbers of a fine field
  size_t np;         // doubles of the momenta / force fields
  double* P;         // momenta (device, lexicographic [V][4][8])
  DBuf& phi;
  DBuf Y, X, t, f;
  int lightest = 0;
  tmg_hmc_stats st{};

  Hmc(Ctx& c_, const tmg_hmc_params& p_, double* P_) : c(c_), p(p_), P(P_), phi(c_.hmc_phi) {
    n = (size_t)12 * c.g.V;
    np = (size_t)32 * c.g.V;
    phi.alloc((size_t)p.n_mono * n * 16);
    Y.alloc(n * 16);
    X.alloc(n * 16);
    t.alloc(n * 16);
    f.alloc(np * sizeof(double));
    for (int m = 1; m < p.n_mono; m++)
      if (p.mu[m] < p.mu[lightest]) lightest = m;
  }
  void* phim(int m) { return phi.as<char>() + (size_t)m * n * 16; }

  // x = D(mu)^-1 b (dag false) or D(mu)^-dag b = g5 D(-mu)^-1 g5 b (dag true), mixed multigrid
  void solve(const void* b, void* x, double mu, bool dag, double tol) {
    SolveStats s{};
    int rc;
    if (!dag) {
      rc = solve_one(c, TMG_SOLVE_MG_MIXED, b, x, mu, tol, 100000, s);
    } else {
      blas_copy(c, b, t.p, TMG_PREC_F64, n);
      gamma5_inplace(c, t.p, TMG_PREC_F64);
      rc = solve_one(c, TMG_SOLVE_MG_MIXED, t.p, x, -mu, tol, 100000, s);
      gamma5_inplace(c, x, TMG_PREC_F64);
    }
    st.solves++;
    st.outer_iterations += s.iterations;
    if (rc != TMG_OK) throw Error{rc, "hmc: a solve did not converge"};
  }

  void heatbath(const double* eta_lex) {
    for (int m = 0; m < p.n_mono; m++) {
      spinor_from_lex(c, eta_lex + (size_t)m * 2 * n, X.p, TMG_PREC_F64);
      if (p.mu2[m] == 0.0) {
        dslash(c, TMG_PREC_F64, phim(m), X.p, nullptr, p.mu[m], 0, 0);                 // phi = D(mu) eta
      } else {
        dslash(c, TMG_PREC_F64, Y.p, X.p, nullptr, p.mu[m], 0, 1);                     // D(mu)^dag eta
        solve(Y.p, phim(m), p.mu2[m], true, p.tol_action);                              // D(mu')^-dag ...
      }
    }
  }

  double fermion_action(int m) {
    if (p.mu2[m] == 0.0) {
      solve(phim(m), Y.p, p.mu[m], false, p.tol_action);
    } else {
      dslash(c, TMG_PREC_F64, X.p, phim(m), nullptr, p.mu2[m], 0, 1);                  // D(mu')^dag phi
      solve(X.p, Y.p, p.mu[m], true, p.tol_action);
    }
    return blas_norm2(c, Y.p, TMG_PREC_F64, n);
  }

  double kinetic() { return 0.5 * blas_norm2(c, P, TMG_PREC_F64, np / 2); }

  double hamiltonian(bool start, const double* eta_lex) {
    double h = kinetic() + gauge_action(c, p.beta);
    if (start) {   // the heat bath makes each fermion action ||eta||^2 exactly
      for (int m = 0; m < p.n_mono; m++) h += blas_norm2(c, eta_lex + (size_t)m * 2 * n, TMG_PREC_F64, n);
    } else {
      for (int m = 0; m < p.n_mono; m++) h += fermion_action(m);
    }
    return h;
  }

  // P -= e f for every monomial of time scale `level` (the gauge action lives on the last one)
  void update_P(int level, double e) {
    if (level == p.n_levels - 1) {
      gauge_force(c, p.beta, f.as<double>());
      blas_axpy(c, -e, 0.0, f.p, P, TMG_PREC_F64, np / 2);
      st.gauge_forces++;
    }
    for (int m = 0; m < p.n_mono; m++) {
      if (p.level[m] != level) continue;
      if (m == lightest && p.setup_iters_force > 0) mg_setup_update(c, p.setup_iters_force);
      if (p.mu2[m] == 0.0) {
        solve(phim(m), Y.p, p.mu[m], false, p.tol_force);
        solve(Y.p, X.p, p.mu[m], true, p.tol_force);
        force_from_xy(c, X.p, Y.p, f.as<double>(), 1);
      } else {
        dslash(c, TMG_PREC_F64, X.p, phim(m), nullptr, p.mu2[m], 0, 1);
        solve(X.p, Y.p, p.mu[m], true, p.tol_force);
        solve(Y.p, X.p, p.mu[m], false, p.tol_force);
        blas_axpy(c, -1.0, 0.0, phim(m), Y.p, TMG_PREC_F64, n);                        // Y - phi
        force_from_xy(c, Y.p, X.p, f.as<double>(), 1);
      }
      blas_axpy(c, -e, 0.0, f.p, P, TMG_PREC_F64, np / 2);
      st.fermion_forces++;
    }
  }

  void evolve(int level, double tt) {
    if (level == p.n_levels) {
      rotate_gauge(c, P, tt);
      gauge_changed(c);
      st.link_updates++;
      return;
    }
    const int ns = p.steps[level];
    const double e = tt / ns;
    for (int i = 0; i < ns; i++) {
      update_P(level, kLambdaMN * e);
      evolve(level + 1, 0.5 * e);
      update_P(level, (1.0 - 2.0 * kLambdaMN) * e);
      evolve(level + 1, 0.5 * e);
      update_P(level, kLambdaMN * e);
    }
  }
};

}  // namespace

int hmc_trajectory(Ctx& c, const tmg_hmc_params& p, double* P_dev, const double* eta_lex_dev, double* dH,
                   tmg_hmc_stats* stats) {
  const auto t0 = std::chrono::steady_clock::now();
  if (p.keep_phi && (c.hmc_nmono != p.n_mono || c.hmc_phi.bytes < (size_t)p.n_mono * 12 * c.g.V * 16))
    throw Error{TMG_ERR_STATE, "hmc: keep_phi without pseudofermions of an earlier trajectory"};
  Hmc h(c, p, P_dev);
  if (p.setup_iters_start > 0) mg_setup_update(c, p.setup_iters_start);
  if (!p.keep_phi) h.heatbath(eta_lex_dev);
  c.hmc_nmono = p.n_mono;
  const double H0 = h.hamiltonian(!p.keep_phi, eta_lex_dev);
  h.evolve(0, p.tau);
  const double H1 = h.hamiltonian(false, nullptr);
  TMG_CUDA(cudaStreamSynchronize(c.stream));
  *dH = H1 - H0;
  h.st.H_start = H0;
  h.st.H_end = H1;
  h.st.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  if (stats) *stats = h.st;
  return TMG_OK;
}

}  // namespace tmg
