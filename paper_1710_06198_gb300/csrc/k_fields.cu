// Field layout conversion, clover construction and complex BLAS kernels of libtmg.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "tmg_host.h"

namespace tmg {

static inline int grid_for(const Ctx& c, size_t n, int threads = 256) {
  size_t b = (n + threads - 1) / threads;
  size_t cap = (size_t)c.sms * 16;
  return (int)std::max<size_t>(1, std::min(b, cap));
}

// ------------------------------------------------------------------ SU(3) check of a loaded field
// max(|U U^dag - 1|_max, |det U - 1|) of one link (row-major 3x3, interleaved re/im); a non-finite
// entry gives +inf.
__host__ __device__ inline double su3_defect_one(const double* u) {
  double d = 0.0;
  for (int k = 0; k < 18; k++)
    if (!(u[k] == u[k]) || u[k] > 1e300 || u[k] < -1e300) return HUGE_VAL;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      double re = (i == j) ? -1.0 : 0.0, im = 0.0;
      for (int k = 0; k < 3; k++) {   // sum_k U_ik conj(U_jk)
        const double ar = u[2 * (3 * i + k)], ai = u[2 * (3 * i + k) + 1];
        const double br = u[2 * (3 * j + k)], bi = u[2 * (3 * j + k) + 1];
        re += ar * br + ai * bi;
        im += ai * br - ar * bi;
      }
      d = fmax(d, fmax(fabs(re), fabs(im)));
    }
  auto R = [&](int i, int j) { return u[2 * (3 * i + j)]; };
  auto I = [&](int i, int j) { return u[2 * (3 * i + j) + 1]; };
  // det = sum over the first row of U_0j times its cofactor
  double dr = 0.0, di = 0.0;
  for (int j = 0; j < 3; j++) {
    const int a = (j + 1) % 3, b = (j + 2) % 3;
    const double cr = R(1, a) * R(2, b) - I(1, a) * I(2, b) - (R(1, b) * R(2, a) - I(1, b) * I(2, a));
    const double ci = R(1, a) * I(2, b) + I(1, a) * R(2, b) - (R(1, b) * I(2, a) + I(1, b) * R(2, a));
    dr += R(0, j) * cr - I(0, j) * ci;
    di += R(0, j) * ci + I(0, j) * cr;
  }
  return fmax(d, hypot(dr - 1.0, di));
}

double su3_defect_host(const double* U, size_t n_links, long long* at) {
  const unsigned hw = std::thread::hardware_concurrency();
  const int nt = (int)std::max<size_t>(1, std::min<size_t>({(size_t)(hw ? hw : 1), (size_t)32, n_links / 4096 + 1}));
  std::vector<double> worst(nt, 0.0);
  std::vector<long long> idx(nt, -1);
  std::vector<std::thread> th;
  for (int t = 0; t < nt; t++)
    th.emplace_back([&, t] {
      const size_t a = n_links * t / nt, b = n_links * (t + 1) / nt;
      for (size_t l = a; l < b; l++) {
        const double d = su3_defect_one(U + 18 * l);
        if (d > worst[t] || idx[t] < 0) { worst[t] = d; idx[t] = (long long)l; }
      }
    });
  for (auto& x : th) x.join();
  double w = 0.0;
  long long i = -1;
  for (int t = 0; t < nt; t++)
    if (idx[t] >= 0 && (i < 0 || worst[t] > w)) { w = worst[t]; i = idx[t]; }
  if (at) *at = i;
  return w;
}

// per-CTA maximum defect and the index where it occurs
__global__ void k_su3_defect(const double* __restrict__ U, size_t n, double* __restrict__ wout, long long* __restrict__ iout) {
  double w = -1.0;
  long long wi = -1;
  for (size_t l = blockIdx.x * (size_t)blockDim.x + threadIdx.x; l < n; l += (size_t)gridDim.x * blockDim.x) {
    double u[18];
    for (int k = 0; k < 18; k++) u[k] = U[18 * l + k];
    const double d = su3_defect_one(u);
    if (d > w) { w = d; wi = (long long)l; }
  }
  __shared__ double sw[256];
  __shared__ long long si[256];
  sw[threadIdx.x] = w;
  si[threadIdx.x] = wi;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o && sw[threadIdx.x + o] > sw[threadIdx.x]) {
      sw[threadIdx.x] = sw[threadIdx.x + o];
      si[threadIdx.x] = si[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) { wout[blockIdx.x] = sw[0]; iout[blockIdx.x] = si[0]; }
}

double su3_defect_device(Ctx& c, const double* U_dev, size_t n_links, long long* at) {
  const int G = grid_for(c, n_links);
  DBuf buf;
  buf.alloc((size_t)G * (sizeof(double) + sizeof(long long)));
  double* w = buf.as<double>();
  long long* ix = reinterpret_cast<long long*>(w + G);
  ++c.launches, k_su3_defect<<<G, 256, 0, c.stream>>>(U_dev, n_links, w, ix);
  TMG_CHECK_LAUNCH();
  std::vector<double> hw(G);
  std::vector<long long> hi(G);
  TMG_CUDA(cudaMemcpyAsync(hw.data(), w, G * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  TMG_CUDA(cudaMemcpyAsync(hi.data(), ix, G * sizeof(long long), cudaMemcpyDeviceToHost, c.stream));
  TMG_CUDA(cudaStreamSynchronize(c.stream));
  double best = 0.0;
  long long bi = -1;
  for (int b = 0; b < G; b++)
    if (hi[b] >= 0 && (bi < 0 || hw[b] > best)) { best = hw[b]; bi = hi[b]; }
  if (at) *at = bi;
  return best;
}

// ------------------------------------------------------------------ link update U <- exp(i A) U
// A = step * sum_a omega_a lambda_a / 2 (lambda_a: Gell-Mann matrices), the su(3) direction of one
// link.  exp(i A) by Taylor series with scaling and squaring: the matrix is divided by 2^s so that
// its Frobenius norm is at most 1/2, summed to order 14 (truncation below 3e-17 relative), then
// squared s times.  The product is projected back onto SU(3) (rows 0, 1 orthonormalised, row 2 =
// conj(row0 x row1)) so that repeated updates stay special unitary.
__device__ void su3_from_algebra(const double* w, double step, cpx<double> A[9]) {
  const double r3 = 0.57735026918962576451;   // 1 / sqrt(3)
  const double h = 0.5 * step;
  A[0] = mk(h * (w[2] + r3 * w[7]), 0.0);
  A[4] = mk(h * (-w[2] + r3 * w[7]), 0.0);
  A[8] = mk(h * (-2.0 * r3 * w[7]), 0.0);
  A[1] = mk(h * w[0], -h * w[1]);
  A[3] = conj(A[1]);
  A[2] = mk(h * w[3], -h * w[4]);
  A[6] = conj(A[2]);
  A[5] = mk(h * w[5], -h * w[6]);
  A[7] = conj(A[5]);
}

__device__ void m3mul(const cpx<double> a[9], const cpx<double> b[9], cpx<double> r[9]) {
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) r[3 * i + j] = a[3 * i] * b[j] + a[3 * i + 1] * b[3 + j] + a[3 * i + 2] * b[6 + j];
}

__device__ void exp_i_hermitian3(const cpx<double> A[9], cpx<double> E[9]) {
  double nrm = 0.0;
  for (int k = 0; k < 9; k++) nrm += A[k].re * A[k].re + A[k].im * A[k].im;
  nrm = sqrt(nrm);
  int sq = 0;
  double scale = 1.0;
  while (nrm * scale > 0.5 && sq < 60) { scale *= 0.5; sq++; }
  cpx<double> B[9];
  for (int k = 0; k < 9; k++) B[k] = mul_i(scale * A[k]);   // i A / 2^s
  // Horner: E = I + B (I + B/2 (I + B/3 (... (I + B/14))))
  for (int k = 0; k < 9; k++) E[k] = mk(k % 4 == 0 ? 1.0 : 0.0, 0.0);
  for (int n = 14; n >= 1; n--) {
    cpx<double> T[9];
    m3mul(B, E, T);
    for (int k = 0; k < 9; k++) E[k] = mk((k % 4 == 0 ? 1.0 : 0.0) + T[k].re / n, T[k].im / n);
  }
  for (int q = 0; q < sq; q++) {
    cpx<double> T[9];
    m3mul(E, E, T);
    for (int k = 0; k < 9; k++) E[k] = T[k];
  }
}

__device__ void reunitarise3(cpx<double> u[9]) {
  double n0 = 0.0;
  for (int b = 0; b < 3; b++) n0 += u[b].re * u[b].re + u[b].im * u[b].im;
  n0 = 1.0 / sqrt(n0);
  for (int b = 0; b < 3; b++) u[b] = n0 * u[b];
  cpx<double> ov = mk(0.0, 0.0);
  for (int b = 0; b < 3; b++) ov = ov + cmul_conj(u[b], u[3 + b]);
  for (int b = 0; b < 3; b++) u[3 + b] = u[3 + b] - ov * u[b];
  double n1 = 0.0;
  for (int b = 0; b < 3; b++) n1 += u[3 + b].re * u[3 + b].re + u[3 + b].im * u[3 + b].im;
  n1 = 1.0 / sqrt(n1);
  for (int b = 0; b < 3; b++) u[3 + b] = n1 * u[3 + b];
  u[6] = conj(u[1] * u[5] - u[2] * u[4]);
  u[7] = conj(u[2] * u[3] - u[0] * u[5]);
  u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

// omega: lexicographic [V][4][8] algebra coefficients; U: internal F64 [4][9][V]
__global__ void k_rotate_links(Geom g, const double* __restrict__ omega, double step, double2* __restrict__ U) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  const int mu = blockIdx.y;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  const size_t lex = lex_index(g, c);
  double w[8];
  for (int a = 0; a < 8; a++) w[a] = omega[(lex * 4 + mu) * 8 + a];
  cpx<double> A[9], E[9], u[9], r[9];
  su3_from_algebra(w, step, A);
  exp_i_hermitian3(A, E);
  for (int k = 0; k < 9; k++) { const double2 v = U[(size_t)(mu * 9 + k) * g.V + s]; u[k] = mk(v.x, v.y); }
  m3mul(E, u, r);
  reunitarise3(r);
  for (int k = 0; k < 9; k++) U[(size_t)(mu * 9 + k) * g.V + s] = make_double2(r[k].re, r[k].im);
}

void rotate_gauge(Ctx& c, const double* omega_dev, double step) {
  const dim3 grid((c.g.V + 127) / 128, 4);
  ++c.launches, k_rotate_links<<<grid, 128, 0, c.stream>>>(c.g, omega_dev, step, c.op[0].U.as<double2>());
  TMG_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ gauge field
// lex [V][4][9] complex -> internal F64 [4][9][V]
__global__ void k_gauge_lex_to_f64(Geom g, const double2* __restrict__ lex, double2* __restrict__ out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int c[4];
    site_coords(g, s, c);
    const int i = lex_index(g, c);
    for (int k = 0; k < 36; k++) out[(size_t)k * g.V + s] = lex[(size_t)i * 36 + k];
  }
}

// internal F64 [4][9][V] -> lex [V][4][9] complex
__global__ void k_gauge_f64_to_lex(Geom g, const double2* __restrict__ in, double2* __restrict__ lex) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int c[4];
    site_coords(g, s, c);
    const int i = lex_index(g, c);
    for (int k = 0; k < 36; k++) lex[(size_t)i * 36 + k] = in[(size_t)k * g.V + s];
  }
}

void gauge_internal_to_lex(Ctx& c, double* lex_dev) {
  ++c.launches, k_gauge_f64_to_lex<<<grid_for(c, c.g.V), 256, 0, c.stream>>>(c.g, c.op[0].U.as<double2>(), (double2*)lex_dev);
  TMG_CHECK_LAUNCH();
}

void gauge_lex_to_internal(Ctx& c, const double* lex_dev) {
  c.op[0].U.alloc((size_t)36 * c.g.V * sizeof(double2));
  ++c.launches, k_gauge_lex_to_f64<<<grid_for(c, c.g.V), 256, 0, c.stream>>>(c.g, (const double2*)lex_dev, c.op[0].U.as<double2>());
  TMG_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ clover
// Leaves of the clover, all counter-clockwise in the (mu, nu) plane, ending at x.
struct M3 { cpx<double> m[9]; };

__device__ __forceinline__ M3 m3_load(const Geom& g, const double2* U, int s, int mu) {
  M3 r;
  for (int k = 0; k < 9; k++) { double2 v = U[(size_t)(mu * 9 + k) * g.V + s]; r.m[k] = {v.x, v.y}; }
  return r;
}
__device__ __forceinline__ M3 m3_mul(const M3& a, const M3& b) {
  M3 r;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) {
      cpx<double> acc = mk(0.0, 0.0);
      for (int k = 0; k < 3; k++) acc = acc + a.m[i * 3 + k] * b.m[k * 3 + j];
      r.m[i * 3 + j] = acc;
    }
  return r;
}
__device__ __forceinline__ M3 m3_dag(const M3& a) {
  M3 r;
  for (int i = 0; i < 3; i++)
    for (int j = 0; j < 3; j++) r.m[i * 3 + j] = conj(a.m[j * 3 + i]);
  return r;
}
__device__ __forceinline__ M3 m3_add(const M3& a, const M3& b) {
  M3 r;
  for (int k = 0; k < 9; k++) r.m[k] = a.m[k] + b.m[k];
  return r;
}

__device__ __forceinline__ int step(const Geom& g, int s, int mu, int dir) {
  SiteCoord sc = decode_site(g, s);
  return dir > 0 ? nbr_fwd(g, sc, mu) : nbr_bwd(g, sc, mu);
}

// sigma_mu_nu restricted to chirality chi (2x2), for mu < nu, in the chiral basis:
// spatial (j,k): -eps_jkl s_l for both chiralities; (k,t): +s_k for chi = 0, -s_k for chi = 1.
__device__ __forceinline__ void sigma_block(int mu, int nu, int chi, cpx<double> sg[4]) {
  int l;
  double sign;
  if (nu == 3) { l = mu; sign = chi == 0 ? 1.0 : -1.0; }
  else {
    l = 3 - mu - nu;                               // the remaining spatial direction
    const double eps = (mu == 0 && nu == 1) ? 1.0 : (mu == 0 && nu == 2) ? -1.0 : 1.0;  // eps_{mu nu l}
    sign = -eps;
  }
  // Pauli matrix s_l (l = 0, 1, 2 -> s1, s2, s3)
  cpx<double> p[4];
  if (l == 0) { p[0] = mk(0., 0.); p[1] = mk(1., 0.); p[2] = mk(1., 0.); p[3] = mk(0., 0.); }
  else if (l == 1) { p[0] = mk(0., 0.); p[1] = mk(0., -1.); p[2] = mk(0., 1.); p[3] = mk(0., 0.); }
  else { p[0] = mk(1., 0.); p[1] = mk(0., 0.); p[2] = mk(0., 0.); p[3] = mk(-1., 0.); }
  for (int k = 0; k < 4; k++) sg[k] = sign * p[k];
}

// A(x) = (4 + m0) + (i c_sw / 16) sum_{mu<nu} sigma_mu_nu (x) (Q_mu_nu - Q_mu_nu^dag)
// (equal to the sum over all ordered pairs with 1/32, since Q_nu_mu = Q_mu_nu^dag).
__global__ void k_clover_build(Geom g, const double2* __restrict__ U, double diag, double csw,
                               double2* __restrict__ A) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  cpx<double> blk[2][36];  // full 6x6 per chirality
  for (int chi = 0; chi < 2; chi++)
    for (int k = 0; k < 36; k++) blk[chi][k] = mk(0.0, 0.0);
  if (csw != 0.0) {
    for (int mu = 0; mu < 4; mu++) {
      for (int nu = mu + 1; nu < 4; nu++) {
        const int xpm = step(g, s, mu, +1), xpn = step(g, s, nu, +1);
        const int xmm = step(g, s, mu, -1), xmn = step(g, s, nu, -1);
        const int xmm_pn = step(g, xmm, nu, +1), xmm_mn = step(g, xmm, nu, -1);
        const int xpm_mn = step(g, xpm, nu, -1);
        const M3 Um = m3_load(g, U, s, mu), Un = m3_load(g, U, s, nu);
        const M3 Un_pm = m3_load(g, U, xpm, nu), Um_pn = m3_load(g, U, xpn, mu);
        const M3 Um_mm = m3_load(g, U, xmm, mu), Un_mm = m3_load(g, U, xmm, nu);
        const M3 Um_mm_pn = m3_load(g, U, xmm_pn, mu);
        const M3 Um_mm_mn = m3_load(g, U, xmm_mn, mu), Un_mm_mn = m3_load(g, U, xmm_mn, nu);
        const M3 Um_mn = m3_load(g, U, xmn, mu), Un_mn = m3_load(g, U, xmn, nu);
        const M3 Un_pm_mn = m3_load(g, U, xpm_mn, nu);
        M3 q = m3_mul(m3_mul(m3_mul(Um, Un_pm), m3_dag(Um_pn)), m3_dag(Un));
        q = m3_add(q, m3_mul(m3_mul(m3_mul(Un, m3_dag(Um_mm_pn)), m3_dag(Un_mm)), Um_mm));
        q = m3_add(q, m3_mul(m3_mul(m3_mul(m3_dag(Um_mm), m3_dag(Un_mm_mn)), Um_mm_mn), Un_mn));
        q = m3_add(q, m3_mul(m3_mul(m3_mul(m3_dag(Un_mn), Um_mn), Un_pm_mn), m3_dag(Um)));
        // F = Q - Q^dag, then i c_sw / 16 * F
        cpx<double> f[9];
        for (int a = 0; a < 3; a++)
          for (int b = 0; b < 3; b++) {
            cpx<double> v = q.m[a * 3 + b] - conj(q.m[b * 3 + a]);
            f[a * 3 + b] = mul_i((csw / 16.0) * v);
          }
        for (int chi = 0; chi < 2; chi++) {
          cpx<double> sg[4];
          sigma_block(mu, nu, chi, sg);
          for (int si = 0; si < 2; si++)
            for (int ti = 0; ti < 2; ti++)
              for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                  const int i = si * 3 + a, j = ti * 3 + b;
                  blk[chi][i * 6 + j] = blk[chi][i * 6 + j] + sg[si * 2 + ti] * f[a * 3 + b];
                }
        }
      }
    }
  }
  for (int chi = 0; chi < 2; chi++) {
    double v[36];
    for (int i = 0; i < 6; i++) v[i] = diag + blk[chi][i * 6 + i].re;
    for (int i = 1; i < 6; i++)
      for (int j = 0; j < i; j++) {
        const int t = 6 + 2 * tri_index(i, j);
        v[t] = blk[chi][i * 6 + j].re;
        v[t + 1] = blk[chi][i * 6 + j].im;
      }
    for (int k = 0; k < 18; k++) A[(size_t)(chi * 18 + k) * g.V + s] = make_double2(v[2 * k], v[2 * k + 1]);
  }
}

void build_clover(Ctx& c) {
  c.op[0].A.alloc((size_t)36 * c.g.V * sizeof(double2));
  const double m0 = 1.0 / (2.0 * c.kappa) - 4.0;
  ++c.launches, k_clover_build<<<(c.g.V + 127) / 128, 128, 0, c.stream>>>(c.g, c.op[0].U.as<double2>(), 4.0 + m0, c.csw,
                                                             c.op[0].A.as<double2>());
  TMG_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ precision copies
__global__ void k_gauge_f64_to_low(Geom g, const double2* __restrict__ U, float4* __restrict__ U32,
                                   short4* __restrict__ U16) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    for (int mu = 0; mu < 4; mu++) {
      for (int k = 0; k < 3; k++) {  // rows 0, 1 = complex 0..5, two per chunk
        const double2 a = U[(size_t)(mu * 9 + 2 * k) * g.V + s];
        const double2 b = U[(size_t)(mu * 9 + 2 * k + 1) * g.V + s];
        U32[(size_t)(mu * 3 + k) * g.V + s] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
        auto q = [](double v) { return (short)__double2int_rn(fmin(1.0, fmax(-1.0, v)) * 32767.0); };
        U16[(size_t)(mu * 3 + k) * g.V + s] = make_short4(q(a.x), q(a.y), q(b.x), q(b.y));
      }
    }
  }
}

__global__ void k_clover_f64_to_low(Geom g, const double2* __restrict__ A, float4* __restrict__ A32,
                                    short4* __restrict__ A16, float* __restrict__ sc16) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    double m = 0.0;
    for (int k = 0; k < 36; k++) {
      const double2 v = A[(size_t)k * g.V + s];
      m = fmax(m, fmax(fabs(v.x), fabs(v.y)));
    }
    const float scale = (float)m;
    sc16[s] = scale;
    const double inv = m > 0 ? 32767.0 / (double)scale : 0.0;
    for (int chi = 0; chi < 2; chi++)
      for (int k = 0; k < 9; k++) {
        const double2 a = A[(size_t)(chi * 18 + 2 * k) * g.V + s];
        const double2 b = A[(size_t)(chi * 18 + 2 * k + 1) * g.V + s];
        A32[(size_t)(chi * 9 + k) * g.V + s] = make_float4((float)a.x, (float)a.y, (float)b.x, (float)b.y);
        auto q = [inv](double v) { return (short)__double2int_rn(fmin(32767.0, fmax(-32767.0, v * inv))); };
        A16[(size_t)(chi * 9 + k) * g.V + s] = make_short4(q(a.x), q(a.y), q(b.x), q(b.y));
      }
  }
}

void convert_op_precisions(Ctx& c) {
  const size_t V = c.g.V;
  c.op[1].U.alloc(V * 12 * sizeof(float4));
  c.op[2].U.alloc(V * 12 * sizeof(short4));
  c.op[1].A.alloc(V * 18 * sizeof(float4));
  c.op[2].A.alloc(V * 18 * sizeof(short4));
  c.op[2].Ascale.alloc(V * sizeof(float));
  ++c.launches, k_gauge_f64_to_low<<<grid_for(c, V), 256, 0, c.stream>>>(c.g, c.op[0].U.as<double2>(), c.op[1].U.as<float4>(),
                                                           c.op[2].U.as<short4>());
  TMG_CHECK_LAUNCH();
  ++c.launches, k_clover_f64_to_low<<<grid_for(c, V), 256, 0, c.stream>>>(c.g, c.op[0].A.as<double2>(), c.op[1].A.as<float4>(),
                                                            c.op[2].A.as<short4>(), c.op[2].Ascale.as<float>());
  TMG_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ spinor lex <-> internal

template <typename T2>
__global__ void k_spinor_from_lex(Geom g, const double2* __restrict__ lex, T2* __restrict__ out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int c[4];
    site_coords(g, s, c);
    const int i = lex_index(g, c);
    for (int k = 0; k < 12; k++) {
      const double2 v = lex[(size_t)i * 12 + k];
      T2 o;
      o.x = v.x; o.y = v.y;
      out[spinor_flat(g.V, s, k)] = o;
    }
  }
}

template <typename T2>
__global__ void k_spinor_to_lex(Geom g, const T2* __restrict__ in, double2* __restrict__ lex) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int c[4];
    site_coords(g, s, c);
    const int i = lex_index(g, c);
    for (int k = 0; k < 12; k++) {
      const T2 v = in[spinor_flat(g.V, s, k)];
      lex[(size_t)i * 12 + k] = make_double2((double)v.x, (double)v.y);
    }
  }
}

// lex FP64 <-> 16-bit fixed-point spinors with a per-site FP32 norm (value = q / 32767 * norm,
// norm = the site's largest |component|, rounding to nearest-even)
__global__ void k_spinor_lex_to_h16(Geom g, const double2* __restrict__ lex, SpinorF16 out) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int c[4];
    site_coords(g, s, c);
    const int i = lex_index(g, c);
    Spinor<float> v;
    for (int k = 0; k < 12; k++) {
      const double2 z = lex[(size_t)i * 12 + k];
      v.c[k] = {(float)z.x, (float)z.y};
    }
    out.store(s, v);
  }
}

__global__ void k_spinor_h16_to_lex(Geom g, SpinorF16 in, double2* __restrict__ lex) {
  for (int s = blockIdx.x * blockDim.x + threadIdx.x; s < g.V; s += gridDim.x * blockDim.x) {
    int c[4];
    site_coords(g, s, c);
    const int i = lex_index(g, c);
    Spinor<float> v;
    in.load(s, v);
    for (int k = 0; k < 12; k++) lex[(size_t)i * 12 + k] = make_double2((double)v.c[k].re, (double)v.c[k].im);
  }
}

SpinorF16 spinor_h16(const Ctx& c, void* p) {
  return SpinorF16{(int4*)p, reinterpret_cast<float*>((char*)p + (size_t)48 * c.g.V), c.g.V};
}

void spinor_from_lex(Ctx& c, const double* lex_dev, void* dst, int prec) {
  if (prec == PREC_H16) {
    ++c.launches, k_spinor_lex_to_h16<<<grid_for(c, c.g.V), 256, 0, c.stream>>>(c.g, (const double2*)lex_dev, spinor_h16(c, dst));
    TMG_CHECK_LAUNCH();
    return;
  }
  if (prec == TMG_PREC_F64)
    ++c.launches, k_spinor_from_lex<double2><<<grid_for(c, c.g.V), 256, 0, c.stream>>>(c.g, (const double2*)lex_dev, (double2*)dst);
  else
    ++c.launches, k_spinor_from_lex<float2><<<grid_for(c, c.g.V), 256, 0, c.stream>>>(c.g, (const double2*)lex_dev, (float2*)dst);
  TMG_CHECK_LAUNCH();
}

void spinor_to_lex(Ctx& c, const void* src, int prec, double* lex_dev) {
  if (prec == PREC_H16) {
    ++c.launches, k_spinor_h16_to_lex<<<grid_for(c, c.g.V), 256, 0, c.stream>>>(c.g, spinor_h16(c, (void*)src), (double2*)lex_dev);
    TMG_CHECK_LAUNCH();
    return;
  }
  if (prec == TMG_PREC_F64)
    ++c.launches, k_spinor_to_lex<double2><<<grid_for(c, c.g.V), 256, 0, c.stream>>>(c.g, (const double2*)src, (double2*)lex_dev);
  else
    ++c.launches, k_spinor_to_lex<float2><<<grid_for(c, c.g.V), 256, 0, c.stream>>>(c.g, (const float2*)src, (double2*)lex_dev);
  TMG_CHECK_LAUNCH();
}

template <typename A2, typename B2>
__global__ void k_convert(const A2* __restrict__ a, B2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const A2 v = a[i];
    B2 o;
    o.x = v.x; o.y = v.y;
    b[i] = o;
  }
}

void convert_field(Ctx& c, const void* src, int psrc, void* dst, int pdst, size_t n) {
  const int gr = grid_for(c, n);
  if (psrc == TMG_PREC_F64 && pdst == TMG_PREC_F32) ++c.launches, k_convert<<<gr, 256, 0, c.stream>>>((const double2*)src, (float2*)dst, n);
  else if (psrc == TMG_PREC_F32 && pdst == TMG_PREC_F64) ++c.launches, k_convert<<<gr, 256, 0, c.stream>>>((const float2*)src, (double2*)dst, n);
  else if (psrc == TMG_PREC_F64) ++c.launches, k_convert<<<gr, 256, 0, c.stream>>>((const double2*)src, (double2*)dst, n);
  else ++c.launches, k_convert<<<gr, 256, 0, c.stream>>>((const float2*)src, (float2*)dst, n);
  TMG_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ BLAS-1
// Element arithmetic runs in the data's own precision (FP32 fields never touch the FP64 pipes,
// which are a small fraction of the FP32 rate on this GPU); dot products accumulate per thread in
// the data precision and reduce across threads in FP64.
template <typename T2> struct ScalarOf;
template <> struct ScalarOf<float2> { using T = float; };
template <> struct ScalarOf<double2> { using T = double; };

template <typename T2>
__global__ void k_axpy(double ar_, double ai_, const T2* __restrict__ x, T2* __restrict__ y, size_t n) {
  using S = typename ScalarOf<T2>::T;
  const S ar = (S)ar_, ai = (S)ai_;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T2 a = x[i];
    T2 b = y[i];
    b.x += ar * a.x - ai * a.y;
    b.y += ar * a.y + ai * a.x;
    y[i] = b;
  }
}
template <typename T2>
__global__ void k_xpay(const T2* __restrict__ x, double ar_, double ai_, T2* __restrict__ y, size_t n) {
  using S = typename ScalarOf<T2>::T;
  const S ar = (S)ar_, ai = (S)ai_;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T2 a = x[i];
    const T2 b = y[i];
    T2 o;
    o.x = a.x + (ar * b.x - ai * b.y);
    o.y = a.y + (ar * b.y + ai * b.x);
    y[i] = o;
  }
}
template <typename T2>
__global__ void k_scale(double ar_, double ai_, T2* __restrict__ x, size_t n) {
  using S = typename ScalarOf<T2>::T;
  const S ar = (S)ar_, ai = (S)ai_;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T2 b = x[i];
    T2 o;
    o.x = ar * b.x - ai * b.y;
    o.y = ar * b.y + ai * b.x;
    x[i] = o;
  }
}
// y += a x with x, y of any precision; the arithmetic runs in the destination's precision
template <typename X2, typename Y2>
__global__ void k_axpy_mixed(double a_, const X2* __restrict__ x, Y2* __restrict__ y, size_t n) {
  using S = typename ScalarOf<Y2>::T;
  const S a = (S)a_;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const X2 v = x[i];
    Y2 b = y[i];
    b.x += a * (S)v.x;
    b.y += a * (S)v.y;
    y[i] = b;
  }
}

void blas_zero(Ctx& c, void* x, int prec, size_t n) {
  TMG_CUDA(cudaMemsetAsync(x, 0, n * (prec == TMG_PREC_F64 ? 16 : 8), c.stream));
}
void blas_copy(Ctx& c, const void* x, void* y, int prec, size_t n) {
  TMG_CUDA(cudaMemcpyAsync(y, x, n * (prec == TMG_PREC_F64 ? 16 : 8), cudaMemcpyDeviceToDevice, c.stream));
}
void blas_axpy(Ctx& c, double ar, double ai, const void* x, void* y, int prec, size_t n) {
  const int gr = grid_for(c, n);
  if (prec == TMG_PREC_F64) ++c.launches, k_axpy<double2><<<gr, 256, 0, c.stream>>>(ar, ai, (const double2*)x, (double2*)y, n);
  else ++c.launches, k_axpy<float2><<<gr, 256, 0, c.stream>>>(ar, ai, (const float2*)x, (float2*)y, n);
  TMG_CHECK_LAUNCH();
}
void blas_xpay(Ctx& c, const void* x, double ar, double ai, void* y, int prec, size_t n) {
  const int gr = grid_for(c, n);
  if (prec == TMG_PREC_F64) ++c.launches, k_xpay<double2><<<gr, 256, 0, c.stream>>>((const double2*)x, ar, ai, (double2*)y, n);
  else ++c.launches, k_xpay<float2><<<gr, 256, 0, c.stream>>>((const float2*)x, ar, ai, (float2*)y, n);
  TMG_CHECK_LAUNCH();
}
void blas_scale(Ctx& c, double ar, double ai, void* x, int prec, size_t n) {
  const int gr = grid_for(c, n);
  if (prec == TMG_PREC_F64) ++c.launches, k_scale<double2><<<gr, 256, 0, c.stream>>>(ar, ai, (double2*)x, n);
  else ++c.launches, k_scale<float2><<<gr, 256, 0, c.stream>>>(ar, ai, (float2*)x, n);
  TMG_CHECK_LAUNCH();
}
// g5 = diag(1, 1, -1, -1): spins 2, 3 are the complex components 6..11, i.e. component pairs 3..5,
// which form the contiguous second half [6 V, 12 V) of a field's flat complex array.
void gamma5_inplace(Ctx& c, void* x, int prec) {
  const size_t half = (size_t)6 * c.g.V;
  blas_scale(c, -1.0, 0.0, (char*)x + half * (prec == TMG_PREC_F64 ? 16 : 8), prec, half);
}

void blas_axpy_mixed(Ctx& c, double a, const void* x, int px, void* y, int py, size_t n) {
  const int gr = grid_for(c, n);
  if (px == TMG_PREC_F32 && py == TMG_PREC_F64) ++c.launches, k_axpy_mixed<<<gr, 256, 0, c.stream>>>(a, (const float2*)x, (double2*)y, n);
  else if (px == TMG_PREC_F64 && py == TMG_PREC_F32) ++c.launches, k_axpy_mixed<<<gr, 256, 0, c.stream>>>(a, (const double2*)x, (float2*)y, n);
  else if (px == TMG_PREC_F64) ++c.launches, k_axpy_mixed<<<gr, 256, 0, c.stream>>>(a, (const double2*)x, (double2*)y, n);
  else ++c.launches, k_axpy_mixed<<<gr, 256, 0, c.stream>>>(a, (const float2*)x, (float2*)y, n);
  TMG_CHECK_LAUNCH();
}

// Block-level reduction of two doubles; result valid in thread 0.
__device__ __forceinline__ void block_reduce2(double& a, double& b) {
  __shared__ double sa[32], sb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) { sa[w] = a; sb[w] = b; }
  __syncthreads();
  const int nw = (blockDim.x + 31) >> 5;
  if (w == 0) {
    a = l < nw ? sa[l] : 0.0;
    b = l < nw ? sb[l] : 0.0;
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_down_sync(0xffffffffu, a, o);
      b += __shfl_down_sync(0xffffffffu, b, o);
    }
  }
}

template <typename T2>
__global__ void k_dot_partial(const T2* __restrict__ x, const T2* __restrict__ y, size_t n, double* __restrict__ part) {
  using S = typename ScalarOf<T2>::T;
  S re = 0, im = 0;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const T2 a = x[i], b = y[i];
    re += a.x * b.x + a.y * b.y;
    im += a.x * b.y - a.y * b.x;
  }
  double dre = re, dim = im;
  block_reduce2(dre, dim);
  if (threadIdx.x == 0) { part[2 * blockIdx.x] = dre; part[2 * blockIdx.x + 1] = dim; }
}

__global__ void k_reduce_final(const double* __restrict__ part, int nparts, double* __restrict__ out) {
  double re = 0.0, im = 0.0;
  for (int i = threadIdx.x; i < nparts; i += blockDim.x) { re += part[2 * i]; im += part[2 * i + 1]; }
  block_reduce2(re, im);
  if (threadIdx.x == 0) { out[0] = re; out[1] = im; }
}

void blas_dot_dev(Ctx& c, const void* x, const void* y, int prec, size_t n, double* out_dev) {
  // enough CTAs to fill the GPU; each thread then sums ~n / (4 * 152 * 256) products
  const int gr = std::min(grid_for(c, n), 4 * c.sms);
  c.red.alloc((size_t)2 * 4096 * sizeof(double));
  if (prec == TMG_PREC_F64) ++c.launches, k_dot_partial<double2><<<gr, 256, 0, c.stream>>>((const double2*)x, (const double2*)y, n, c.red.as<double>());
  else ++c.launches, k_dot_partial<float2><<<gr, 256, 0, c.stream>>>((const float2*)x, (const float2*)y, n, c.red.as<double>());
  TMG_CHECK_LAUNCH();
  ++c.launches, k_reduce_final<<<1, 256, 0, c.stream>>>(c.red.as<double>(), gr, out_dev);
  TMG_CHECK_LAUNCH();
}

void blas_dot(Ctx& c, const void* x, const void* y, int prec, size_t n, double* re, double* im) {
  c.red_out.alloc(64 * sizeof(double));
  blas_dot_dev(c, x, y, prec, n, c.red_out.as<double>());
  double h[2];
  TMG_CUDA(cudaMemcpyAsync(h, c.red_out.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  TMG_CUDA(cudaStreamSynchronize(c.stream));
  *re = h[0];
  if (im) *im = h[1];
}

double blas_norm2(Ctx& c, const void* x, int prec, size_t n) {
  double re, im;
  blas_dot(c, x, x, prec, n, &re, &im);
  return re;
}

}  // namespace tmg
