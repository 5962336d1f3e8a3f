// Pseudofermion force of S = phi^dag (D D^dag)^-1 phi = ||D(mu)^-1 phi||^2 (the force terms of
// the HMC of Sec. 2 and 3 of arXiv:1710.06198, built from solves of D^dag D in the two-step form
// of Sec. 1.1).  With Y = D^-1 phi and X = D^-dag Y, dS/dt = -2 Re X^dag (dD/dt) Y under
// U_mu(x) -> exp(i t H) U_mu(x); the kernels build G with X^dag (dD/dt) Y = sum tr(H G) and
// return F = traceless Hermitian part of -2 G, so that dS/dt = sum tr(H F).
//
//   k_force_lambda : per site y and plane (a < b), Lam_ab(y)[b', a'] = sum_{s,t} sigma_ab[s][t]
//                    Y(y)[t][b'] conj(X(y)[s][a']), the colour matrix of X^dag (sigma_ab x M) Y.
//   k_force_link   : one thread per link (x, mu): the hopping-term derivative, and the clover
//                    derivative gathered from the 16 leaf insertions of each of the 3 planes that
//                    contain mu (leaves of Q_ab with +1, of Q_ba with -1, coefficient i c_sw / 16).
//   k_force_project: F = traceless Hermitian part of -2 G, written in lexicographic order.
#include "tmg_host.h"

namespace tmg {

namespace {

template <typename R>
struct M3 { cpx<R> m[9]; };

template <typename R>
__device__ __forceinline__ M3<R> mmul(const M3<R>& a, const M3<R>& b) {
  M3<R> r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) {
      cpx<R> acc = a.m[i * 3] * b.m[j];
      acc = acc + a.m[i * 3 + 1] * b.m[3 + j];
      acc = acc + a.m[i * 3 + 2] * b.m[6 + j];
      r.m[i * 3 + j] = acc;
    }
  return r;
}
template <typename R>
__device__ __forceinline__ M3<R> mdag(const M3<R>& a) {
  M3<R> r;
#pragma unroll
  for (int i = 0; i < 3; i++)
#pragma unroll
    for (int j = 0; j < 3; j++) r.m[i * 3 + j] = conj(a.m[j * 3 + i]);
  return r;
}
template <typename R>
__device__ __forceinline__ M3<R> mident() {
  M3<R> r;
#pragma unroll
  for (int k = 0; k < 9; k++) r.m[k] = mk<R>(k % 4 == 0 ? R(1) : R(0), R(0));
  return r;
}
template <typename R, class G>
__device__ __forceinline__ M3<R> load_link(const G& U, int s, int mu) {
  Link<R> l;
  U.load(s, mu, l);
  M3<R> r;
#pragma unroll
  for (int k = 0; k < 9; k++) r.m[k] = l.m[k];
  return r;
}

// plane index of (a < b): (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
__device__ __forceinline__ int plane_index(int a, int b) {
  return a == 0 ? b - 1 : (a == 1 ? b + 1 : 5);
}

// sigma_ab (a < b) restricted to chirality chi, chiral basis (see k_fields.cu):
// spatial (j,k): -eps_jkl s_l; (k,t): +s_k for chi = 0, -s_k for chi = 1.
template <typename R>
__device__ __forceinline__ void sigma_chi(int a, int b, int chi, cpx<R> sg[4]) {
  int l;
  R sign;
  if (b == 3) { l = a; sign = chi == 0 ? R(1) : R(-1); }
  else { l = 3 - a - b; sign = (a == 0 && b == 2) ? R(1) : R(-1); }
  cpx<R> p[4];
  const R o = 1, z = 0;
  if (l == 0) { p[0] = mk<R>(z, z); p[1] = mk<R>(o, z); p[2] = mk<R>(o, z); p[3] = mk<R>(z, z); }
  else if (l == 1) { p[0] = mk<R>(z, z); p[1] = mk<R>(z, -o); p[2] = mk<R>(z, o); p[3] = mk<R>(z, z); }
  else { p[0] = mk<R>(o, z); p[1] = mk<R>(z, z); p[2] = mk<R>(z, z); p[3] = mk<R>(-o, z); }
#pragma unroll
  for (int k = 0; k < 4; k++) sg[k] = sign * p[k];
}

// The four counter-clockwise (rho -> sig) leaves ending at the corner y, as lists of
// (offset along rho, offset along sig, direction is sig, daggered).
__constant__ int c_leaf_or[4][4] = {{0, 1, 0, 0}, {0, -1, -1, -1}, {-1, -1, -1, 0}, {0, 0, 1, 0}};
__constant__ int c_leaf_os[4][4] = {{0, 0, 1, 0}, {0, 1, 0, 0}, {0, -1, -1, -1}, {-1, -1, -1, 0}};
__constant__ int c_leaf_sig[4][4] = {{0, 1, 0, 1}, {1, 0, 1, 0}, {0, 1, 0, 1}, {1, 0, 1, 0}};
__constant__ int c_leaf_dag[4][4] = {{0, 0, 1, 1}, {0, 1, 1, 0}, {1, 1, 0, 0}, {1, 0, 0, 1}};

__device__ __forceinline__ int shifted_site(const Geom& g, const int c[4], int r, int dr, int sg, int ds) {
  int d[4] = {c[0], c[1], c[2], c[3]};
  d[r] = (d[r] + dr + 2 * g.L[r]) % g.L[r];
  d[sg] = (d[sg] + ds + 2 * g.L[sg]) % g.L[sg];
  return site_index(g, d);
}

template <typename R, class S, typename T2>
__global__ void k_force_lambda(Geom g, S X, S Y, T2* __restrict__ lam) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  Spinor<R> x, y;
  X.load(s, x);
  Y.load(s, y);
  for (int a = 0; a < 4; a++)
    for (int b = a + 1; b < 4; b++) {
      const int p = plane_index(a, b);
      cpx<R> L[9];
      for (int k = 0; k < 9; k++) L[k] = mk<R>(0, 0);
      for (int chi = 0; chi < 2; chi++) {
        cpx<R> sg[4];
        sigma_chi<R>(a, b, chi, sg);
        for (int si = 0; si < 2; si++)
          for (int ti = 0; ti < 2; ti++) {
            const cpx<R> w = sg[si * 2 + ti];
            if (w.re == R(0) && w.im == R(0)) continue;
            const int s_ = 2 * chi + si, t_ = 2 * chi + ti;
            for (int bb = 0; bb < 3; bb++)
              for (int aa = 0; aa < 3; aa++)
                L[bb * 3 + aa] = L[bb * 3 + aa] + w * (y.c[t_ * 3 + bb] * conj(x.c[s_ * 3 + aa]));
          }
      }
      for (int k = 0; k < 9; k++) {
        T2 o;
        o.x = L[k].re;
        o.y = L[k].im;
        lam[((size_t)p * 9 + k) * g.V + s] = o;
      }
    }
}

// full-spinor (1 + sgn g_mu) applied to p (chiral basis; see spin_project in tmg_internal.cuh)
template <typename R>
__device__ __forceinline__ void proj_full(int mu, int sgn, const Spinor<R>& p, Spinor<R>& o) {
  // (1 - s g) p = [h ; -s B^dag h], h = p_up - s B p_dn ; here s = -sgn so that (1 + sgn g) is formed
  cpx<R> h[6];
  spin_project(mu, -sgn, p, h);
  Spinor<R> acc;
  for (int k = 0; k < 12; k++) acc.c[k] = mk<R>(0, 0);
  spin_reconstruct_add(mu, -sgn, h, acc);
  o = acc;
}

template <typename R, class GT, class S, typename T2>
__global__ void k_force_link(Geom g, GT U, S X, S Y, const T2* __restrict__ lam, R csw, T2* __restrict__ G) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  const SiteCoord sc = decode_site(g, s);
  const int sf = nbr_fwd(g, sc, mu);
  cpx<R> Gm[9];
  // ---- hopping term: G = (i sgn / 2) (A2 - A1)
  {
    const M3<R> u = load_link<R>(U, s, mu);
    const R sgn = (mu == 3 && c[3] == g.L[3] - 1 && g.tbc < 0) ? R(-1) : R(1);
    Spinor<R> xs, ys, xf, yf, uy, P, W, ux;
    X.load(s, xs);
    Y.load(s, ys);
    X.load(sf, xf);
    Y.load(sf, yf);
    for (int sp = 0; sp < 4; sp++)
      for (int a = 0; a < 3; a++) {
        cpx<R> t1 = mk<R>(0, 0), t2 = mk<R>(0, 0);
        for (int b = 0; b < 3; b++) {
          t1 = t1 + u.m[a * 3 + b] * yf.c[sp * 3 + b];
          t2 = t2 + u.m[a * 3 + b] * xf.c[sp * 3 + b];
        }
        uy.c[sp * 3 + a] = t1;
        ux.c[sp * 3 + a] = t2;
      }
    proj_full(mu, -1, uy, P);   // (1 - g_mu) U Y(x+mu)
    proj_full(mu, +1, ys, W);   // (1 + g_mu) Y(x)
    for (int i = 0; i < 3; i++)
      for (int j = 0; j < 3; j++) {
        // A1[i][j] = sum_s P[s][i] conj(X[s][j]) ; A2[i][j] = sum_s W[s][i] conj(UX[s][j])
        cpx<R> a1 = mk<R>(0, 0), a2 = mk<R>(0, 0);
        for (int sp = 0; sp < 4; sp++) {
          a1 = a1 + P.c[sp * 3 + i] * conj(xs.c[sp * 3 + j]);
          a2 = a2 + W.c[sp * 3 + i] * conj(ux.c[sp * 3 + j]);
        }
        Gm[i * 3 + j] = mul_i((R(0.5) * sgn) * (a2 - a1));
      }
  }
  // ---- clover term
  if (csw != R(0)) {
    const cpx<R> coef = mk<R>(0, csw / R(16));
    for (int nu = 0; nu < 4; nu++) {
      if (nu == mu) continue;
      const int a = min(mu, nu), b = max(mu, nu), p = plane_index(a, b);
      for (int orient = 0; orient < 2; orient++) {
        const int rho = orient == 0 ? a : b, sig = orient == 0 ? b : a;
        const R sign = orient == 0 ? R(1) : R(-1);
        for (int leaf = 0; leaf < 4; leaf++) {
          for (int k = 0; k < 4; k++) {
            const int dk = c_leaf_sig[leaf][k] ? sig : rho;
            if (dk != mu) continue;
            // corner y = x - offset of factor k
            int yc[4] = {c[0], c[1], c[2], c[3]};
            yc[rho] = (yc[rho] - c_leaf_or[leaf][k] + 2 * g.L[rho]) % g.L[rho];
            yc[sig] = (yc[sig] - c_leaf_os[leaf][k] + 2 * g.L[sig]) % g.L[sig];
            const int ys = site_index(g, yc);
            M3<R> f[4];
            for (int q = 0; q < 4; q++) {
              const int site = shifted_site(g, yc, rho, c_leaf_or[leaf][q], sig, c_leaf_os[leaf][q]);
              const M3<R> l = load_link<R>(U, site, c_leaf_sig[leaf][q] ? sig : rho);
              f[q] = c_leaf_dag[leaf][q] ? mdag(l) : l;
            }
            M3<R> L;
            for (int e = 0; e < 9; e++) {
              const T2 v = lam[((size_t)p * 9 + e) * g.V + ys];
              L.m[e] = mk<R>(v.x, v.y);
            }
            M3<R> after = mident<R>(), before = mident<R>();
            for (int q = k + 1; q < 4; q++) after = mmul(after, f[q]);
            for (int q = 0; q < k; q++) before = mmul(before, f[q]);
            M3<R> M;
            cpx<R> ph;
            if (!c_leaf_dag[leaf][k]) {
              M = mmul(mmul(mmul(f[k], after), L), before);
              ph = mk<R>(0, 1);
            } else {
              M = mmul(mmul(mmul(after, L), before), f[k]);
              ph = mk<R>(0, -1);
            }
            const cpx<R> w = (sign * coef) * ph;
            for (int e = 0; e < 9; e++) Gm[e] = Gm[e] + w * M.m[e];
          }
        }
      }
    }
  }
  for (int e = 0; e < 9; e++) {
    T2 o;
    o.x = Gm[e].re;
    o.y = Gm[e].im;
    G[((size_t)mu * 9 + e) * g.V + s] = o;
  }
}

// FP32 storage read into FP64 registers: the force kernels then sum every outer product and leaf
// product in FP64 while moving half the bytes of the FP64 fields.
struct SpinorF32in64 {
  float4* p; int V;
  __device__ __forceinline__ void load(int s, Spinor<double>& o) const {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const float4 v = __ldg(p + (size_t)k * V + s);
      o.c[2 * k] = {(double)v.x, (double)v.y};
      o.c[2 * k + 1] = {(double)v.z, (double)v.w};
    }
  }
};
struct GaugeF32in64 {
  float4* p; int V;
  __device__ __forceinline__ void load(int s, int mu, Link<double>& u) const {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      const float4 v = __ldg(p + (size_t)(mu * 3 + k) * V + s);
      u.m[2 * k] = {(double)v.x, (double)v.y};
      u.m[2 * k + 1] = {(double)v.z, (double)v.w};
    }
    reconstruct_row2(u);
  }
};

// F = traceless Hermitian part of -2 G, lexicographic output [V][4][3][3] (alg = 0) or its su(3)
// coefficients [V][4][8] (alg = 1)
template <typename T2>
__global__ void k_force_project(Geom g, const T2* __restrict__ G, double2* __restrict__ F, int alg) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  const int lex = lex_index(g, c);
  cpx<double> m[9], h[9];
  for (int e = 0; e < 9; e++) { const T2 v = G[((size_t)mu * 9 + e) * g.V + s]; m[e] = mk(-2.0 * v.x, -2.0 * v.y); }
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) h[i * 3 + j] = 0.5 * (m[i * 3 + j] + conj(m[j * 3 + i]));
  const double tr = (h[0].re + h[4].re + h[8].re) / 3.0;
  h[0].re -= tr;
  h[4].re -= tr;
  h[8].re -= tr;
  if (alg) {
    double f[8];
    algebra_coeffs(h, f);
    double* out = reinterpret_cast<double*>(F) + ((size_t)lex * 4 + mu) * 8;
    for (int a = 0; a < 8; a++) out[a] = f[a];
    return;
  }
  for (int e = 0; e < 9; e++) F[((size_t)lex * 4 + mu) * 9 + e] = make_double2(h[e].re, h[e].im);
}

}  // namespace

// F (lexicographic [V][4][3][3], or its su(3) coefficients [V][4][8] when alg != 0; device) from
// internal F64 fields X, Y (tbc/clover from the context).  With c.force_prec == TMG_PREC_F32 the
// kernels read FP32 copies of X, Y and the 12-real FP32 links and accumulate in FP64.
void force_from_xy(Ctx& c, const void* X, const void* Y, double* F_lex, int alg) {
  const size_t V = c.g.V;
  const dim3 grid1((c.g.V + 127) / 128), grid4((c.g.V + 127) / 128, 4);
  c.fw_t.alloc(V * (6 * 9 + 4 * 9) * sizeof(double2) + (c.force_prec == TMG_PREC_F32 ? 2 * 12 * V * sizeof(float2) : 0));
  double2* lam = c.fw_t.as<double2>();
  double2* G = lam + V * 6 * 9;
  if (c.force_prec == TMG_PREC_F32) {
    float2* x32 = reinterpret_cast<float2*>(G + V * 4 * 9);
    float2* y32 = x32 + 12 * V;
    convert_field(c, X, TMG_PREC_F64, x32, TMG_PREC_F32, 12 * V);
    convert_field(c, Y, TMG_PREC_F64, y32, TMG_PREC_F32, 12 * V);
    const SpinorF32in64 xs{(float4*)x32, c.g.V}, ys{(float4*)y32, c.g.V};
    ++c.launches, k_force_lambda<double><<<grid1, 128, 0, c.stream>>>(c.g, xs, ys, lam);
    TMG_CHECK_LAUNCH();
    ++c.launches, k_force_link<double><<<grid4, 128, 0, c.stream>>>(c.g, GaugeF32in64{c.op[1].U.as<float4>(), c.g.V}, xs, ys,
                                                                    lam, c.csw, G);
    TMG_CHECK_LAUNCH();
  } else {
    const SpinorF64 xs{(double2*)X, c.g.V}, ys{(double2*)Y, c.g.V};
    ++c.launches, k_force_lambda<double><<<grid1, 128, 0, c.stream>>>(c.g, xs, ys, lam);
    TMG_CHECK_LAUNCH();
    ++c.launches, k_force_link<double><<<grid4, 128, 0, c.stream>>>(c.g, GaugeF64{c.op[0].U.as<double2>(), c.g.V}, xs, ys,
                                                                    lam, c.csw, G);
    TMG_CHECK_LAUNCH();
  }
  ++c.launches, k_force_project<<<grid4, 128, 0, c.stream>>>(c.g, (const double2*)G, (double2*)F_lex, alg);
  TMG_CHECK_LAUNCH();
}

}  // namespace tmg
