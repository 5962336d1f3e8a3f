// Solver runtime of libtmg: the DD-alpha-AMG cycle of Eq. 1 (coarse-grid correction, then k SAP
// sweeps), its adaptive setup (Sec. 1.1 and Sec. 2 of arXiv:1710.06198), the coarse solve, and the
// flexible outer Krylov solver (Sec. 1.1) with FP64 residual recomputation at every restart.
//
// The coarse GMRES is one persistent cooperative kernel (k_coarse_gmres.cu), so a cycle issues
// its kernels without a single host synchronisation.
#include <algorithm>
#include <cmath>
#include <complex>
#include <vector>

#include "solver.h"

#include <cstdint>
#include <cstring>

namespace tmg {

namespace {

constexpr int MAXM = 64;     // largest Krylov cycle
constexpr int NPART = 1024;  // reduction partials per vector (>= CTAs of a reduction launch)

// ---- multi-vector reductions on flat complex arrays ---------------------------------------------
// part[i * NPART + b] = partial of <v_i, w> over the chunk of block b (grid: NPART x count)
template <typename T2> struct ScalarOf;
template <> struct ScalarOf<float2> { using T = float; };
template <> struct ScalarOf<double2> { using T = double; };

template <typename T2>
__global__ void k_mdot_partial(const T2* __restrict__ Vb, size_t stride, const T2* __restrict__ w, size_t n,
                               double2* __restrict__ part, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = typename ScalarOf<T2>::T;
  const int i = blockIdx.y;
  const T2* v = Vb + (size_t)i * stride;
  S tre = 0, tim = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const T2 a = v[e], b = w[e];
    tre += a.x * b.x + a.y * b.y;
    tim += a.x * b.y - a.y * b.x;
  }
  double re = tre, im = tim;
  __shared__ double sre[32], sim[32];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
  if (lane == 0) { sre[wp] = re; sim[wp] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) { a += sre[k]; b += sim[k]; }
    part[(size_t)i * NPART + blockIdx.x] = make_double2(a, b);
  }
}

// out[i] = sum_b part[i * NPART + b], one CTA per i (grid: count)
__global__ void k_mdot_final(const double2* __restrict__ part, int np, int count, double2* __restrict__ out,
                             const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int i = blockIdx.x;
  double a = 0, b = 0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) { const double2 v = part[(size_t)i * NPART + k]; a += v.x; b += v.y; }
  __shared__ double sa[32], sb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) { sa[threadIdx.x >> 5] = a; sb[threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0, tb = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) { ta += sa[k]; tb += sb[k]; }
    out[i] = make_double2(ta, tb);
  }
}

// First Gram-Schmidt pass's update fused with the second pass's dot products (count <= 10):
// w -= sum_i coef[i] v_i, then part[i * NPART + b] = partial of <v_i, w> over block b's elements,
// with each v_i read once for both.
constexpr int FUSED_MAX = 10;

template <typename T2>
__global__ void __launch_bounds__(256, 2) k_mgs_update_dot(const T2* __restrict__ Vb, size_t stride, int count,
                                                        const double2* __restrict__ coef, T2* __restrict__ w, size_t n,
                                                        double2* __restrict__ part) {
  using S = typename ScalarOf<T2>::T;
  __shared__ S cfr[FUSED_MAX], cfi[FUSED_MAX];
  __shared__ double sre[FUSED_MAX][8], sim[FUSED_MAX][8];
  for (int i = threadIdx.x; i < count; i += blockDim.x) { cfr[i] = (S)coef[i].x; cfi[i] = (S)coef[i].y; }
  __syncthreads();
  S dr[FUSED_MAX], di[FUSED_MAX];
#pragma unroll
  for (int i = 0; i < FUSED_MAX; i++) { dr[i] = 0; di[i] = 0; }
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    T2 v[FUSED_MAX];
    S xr = w[e].x, xi = w[e].y;
#pragma unroll
    for (int i = 0; i < FUSED_MAX; i++) {
      if (i < count) {
        v[i] = Vb[(size_t)i * stride + e];
        xr -= cfr[i] * v[i].x - cfi[i] * v[i].y;
        xi -= cfr[i] * v[i].y + cfi[i] * v[i].x;
      }
    }
    T2 o;
    o.x = xr;
    o.y = xi;
    w[e] = o;
#pragma unroll
    for (int i = 0; i < FUSED_MAX; i++) {
      if (i < count) {
        dr[i] += v[i].x * xr + v[i].y * xi;
        di[i] += v[i].x * xi - v[i].y * xr;
      }
    }
  }
  const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
#pragma unroll
  for (int i = 0; i < FUSED_MAX; i++) {
    if (i < count) {
      double re = dr[i], im = di[i];
      for (int o = 16; o > 0; o >>= 1) {
        re += __shfl_down_sync(0xffffffffu, re, o);
        im += __shfl_down_sync(0xffffffffu, im, o);
      }
      if (lane == 0) { sre[i][wp] = re; sim[i][wp] = im; }
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    double a = 0, b = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) { a += sre[i][k]; b += sim[i][k]; }
    part[(size_t)i * NPART + blockIdx.x] = make_double2(a, b);
  }
}

// w -= sum_i coef[i] v_i  (coef on the device); optionally partial ||w||^2 into part[b]
template <typename T2>
__global__ void k_mgs_update(const T2* __restrict__ Vb, size_t stride, int count, const double2* __restrict__ coef,
                             T2* __restrict__ w, size_t n, double2* __restrict__ npart, const int* __restrict__ skip) {
  if (skip && *skip) return;
  using S = typename ScalarOf<T2>::T;
  __shared__ S cfr[MAXM + 1], cfi[MAXM + 1];
  for (int i = threadIdx.x; i < count; i += blockDim.x) { cfr[i] = (S)coef[i].x; cfi[i] = (S)coef[i].y; }
  __syncthreads();
  S snn = 0;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    S xr = w[e].x, xi = w[e].y;
    for (int i = 0; i < count; i++) {
      const T2 v = Vb[(size_t)i * stride + e];
      xr -= cfr[i] * v.x - cfi[i] * v.y;
      xi -= cfr[i] * v.y + cfi[i] * v.x;
    }
    T2 o;
    o.x = xr;
    o.y = xi;
    w[e] = o;
    snn += xr * xr + xi * xi;
  }
  double nn = snn;
  if (!npart) return;
  __shared__ double s[32];
  for (int o = 16; o > 0; o >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, o);
  if ((threadIdx.x & 31) == 0) s[threadIdx.x >> 5] = nn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) a += s[k];
    npart[blockIdx.x] = make_double2(a, 0.0);
  }
}

// x = sum_{i<k} coef[i] z_i   (k read from the device when kdev != null)
template <typename T2>
__global__ void k_combine(const T2* __restrict__ Zb, size_t stride, int count, const int* __restrict__ kdev,
                          const double2* __restrict__ coef, T2* __restrict__ x, size_t n) {
  using S = typename ScalarOf<T2>::T;
  const int k = kdev ? *kdev : count;
  __shared__ S cfr[MAXM], cfi[MAXM];
  for (int i = threadIdx.x; i < k; i += blockDim.x) { cfr[i] = (S)coef[i].x; cfi[i] = (S)coef[i].y; }
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    S xr = 0, xi = 0;
    for (int i = 0; i < k; i++) {
      const T2 v = Zb[(size_t)i * stride + e];
      xr += cfr[i] * v.x - cfi[i] * v.y;
      xi += cfr[i] * v.y + cfi[i] * v.x;
    }
    T2 o;
    o.x = xr;
    o.y = xi;
    x[e] = o;
  }
}

// ---- column-batched variants: column c of a field at c * n elements, partials [c][i][NPART]
__global__ void k_mdot_partial_b(const float2* __restrict__ Vb, size_t istride, const float2* __restrict__ w,
                                 size_t n, double2* __restrict__ part) {
  const int i = blockIdx.y, c = blockIdx.z;
  const float2* v = Vb + (size_t)i * istride + (size_t)c * n;
  const float2* wc = w + (size_t)c * n;
  float tre = 0.f, tim = 0.f;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float2 a = v[e], b = wc[e];
    tre += a.x * b.x + a.y * b.y;
    tim += a.x * b.y - a.y * b.x;
  }
  double re = tre, im = tim;
  __shared__ double sre[32], sim[32];
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_down_sync(0xffffffffu, re, o);
    im += __shfl_down_sync(0xffffffffu, im, o);
  }
  if ((threadIdx.x & 31) == 0) { sre[threadIdx.x >> 5] = re; sim[threadIdx.x >> 5] = im; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) { a += sre[k]; b += sim[k]; }
    part[((size_t)c * (MAXM + 1) + i) * NPART + blockIdx.x] = make_double2(a, b);
  }
}

// out[c][i] = sum_b part[c][i][b]; grid (count, ncol)
__global__ void k_mdot_final_b(const double2* __restrict__ part, int np, double2* __restrict__ out) {
  const int i = blockIdx.x, c = blockIdx.y;
  const double2* p = part + ((size_t)c * (MAXM + 1) + i) * NPART;
  double a = 0, b = 0;
  for (int k = threadIdx.x; k < np; k += blockDim.x) { a += p[k].x; b += p[k].y; }
  __shared__ double sa[32], sb[32];
  for (int o = 16; o > 0; o >>= 1) {
    a += __shfl_down_sync(0xffffffffu, a, o);
    b += __shfl_down_sync(0xffffffffu, b, o);
  }
  if ((threadIdx.x & 31) == 0) { sa[threadIdx.x >> 5] = a; sb[threadIdx.x >> 5] = b; }
  __syncthreads();
  if (threadIdx.x == 0) {
    double ta = 0, tb = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) { ta += sa[k]; tb += sb[k]; }
    out[(size_t)c * (MAXM + 1) + i] = make_double2(ta, tb);
  }
}

// w_c -= sum_i coef[c][i] v_i,c ; optional partial ||w_c||^2 into npart[c][b]; grid (G, ncol)
__global__ void k_mgs_update_b(const float2* __restrict__ Vb, size_t istride, int count, const double2* __restrict__ coef,
                               float2* __restrict__ w, size_t n, double* __restrict__ npart) {
  const int c = blockIdx.y;
  __shared__ float cfr[MAXM + 1], cfi[MAXM + 1];
  for (int i = threadIdx.x; i < count; i += blockDim.x) {
    cfr[i] = (float)coef[(size_t)c * (MAXM + 1) + i].x;
    cfi[i] = (float)coef[(size_t)c * (MAXM + 1) + i].y;
  }
  __syncthreads();
  float snn = 0.f;
  float2* wc = w + (size_t)c * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float2 q = wc[e];
    for (int i = 0; i < count; i++) {
      const float2 v = Vb[(size_t)i * istride + (size_t)c * n + e];
      q.x -= cfr[i] * v.x - cfi[i] * v.y;
      q.y -= cfr[i] * v.y + cfi[i] * v.x;
    }
    wc[e] = q;
    snn += q.x * q.x + q.y * q.y;
  }
  if (!npart) return;
  double nn = snn;
  __shared__ double sh[32];
  for (int o = 16; o > 0; o >>= 1) nn += __shfl_down_sync(0xffffffffu, nn, o);
  if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = nn;
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) a += sh[k];
    npart[(size_t)c * NPART + blockIdx.x] = a;
  }
}

// x_c = sum_{i<k} coef[c][i] z_i,c ; grid (G, ncol)
__global__ void k_combine_b(const float2* __restrict__ Zb, size_t istride, int k, const double2* __restrict__ coef,
                            float2* __restrict__ x, size_t n) {
  const int c = blockIdx.y;
  __shared__ float cfr[MAXM], cfi[MAXM];
  for (int i = threadIdx.x; i < k; i += blockDim.x) {
    cfr[i] = (float)coef[(size_t)c * (MAXM + 1) + i].x;
    cfi[i] = (float)coef[(size_t)c * (MAXM + 1) + i].y;
  }
  __syncthreads();
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    float xr = 0.f, xi = 0.f;
    for (int i = 0; i < k; i++) {
      const float2 v = Zb[(size_t)i * istride + (size_t)c * n + e];
      xr += cfr[i] * v.x - cfi[i] * v.y;
      xi += cfr[i] * v.y + cfi[i] * v.x;
    }
    x[(size_t)c * n + e] = make_float2(xr, xi);
  }
}

// y_c = s_c x_c for ncol FP32 columns of n complex each (s on the device); grid (G, ncol)
__global__ void k_scale_cols(const float2* __restrict__ x, float2* __restrict__ y, const double* __restrict__ sc, size_t n) {
  const int c = blockIdx.y;
  const float s = (float)sc[c];
  const float2* xc = x + (size_t)c * n;
  float2* yc = y + (size_t)c * n;
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float2 v = xc[e];
    yc[e] = make_float2(s * v.x, s * v.y);
  }
}

size_t esize(int prec) { return prec == TMG_PREC_F64 ? 16 : 8; }

int red_grid(const Ctx& c, size_t n) {
  return (int)std::min<size_t>(std::min<size_t>(NPART, (size_t)4 * c.sms), std::max<size_t>(1, (n + 255) / 256));
}

template <typename F>
void dispatch(int prec, F&& f) {
  if (prec == TMG_PREC_F64) f(double2{});
  else f(float2{});
}

// grid for element-wise kernels
int egrid(const Ctx& c, size_t n) { return (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, (size_t)c.sms * 8)); }

}  // namespace

// ---------------------------------------------------------------- cycle (Eq. 1)
static int storage(int prec) { return prec == TMG_PREC_F64 ? TMG_PREC_F64 : TMG_PREC_F32; }

// z = P D_c^-1 P^dag r, then k SAP sweeps on D z = r starting from z (pf: fine precision of the
// SAP / P operations, pc: coarse precision).
// nf = 2: the doublet cycle (P_ND = P x I2, D_ND,c, SAP on D_ND); fields [2][12 V], mu unused.
static void cycle_p(Ctx& c, int pf, int pc, const void* r, void* z, double mu, int nf = 1) {
  const size_t nco = (size_t)c.cl.nc * c.cl.nd;
  const size_t nfi = (size_t)12 * c.g.V, ef = esize(storage(pf)), ec = esize(pc);
  c.cw_cr.alloc(nf * nco * ec);
  c.cw_ce.alloc(nf * nco * ec);
  for (int f = 0; f < nf; f++) restrict_(c, pf, (const char*)r + f * nfi * ef, (char*)c.cw_cr.p + f * nco * ec, pc);
  if (nf == 2) {
    if (c.l2_ready) kcycle(c, pc, c.cw_cr.p, c.cw_ce.p, c.mubar, 0, 2);
    else coarse_gmres_persistent_nd(c, pc, c.cw_cr.p, c.cw_ce.p);
  } else {
    if (c.l2_ready) kcycle(c, pc, c.cw_cr.p, c.cw_ce.p, mu, 0);   // three levels: the level-1 K-cycle
    else coarse_gmres_persistent(c, pc, c.cw_cr.p, c.cw_ce.p, mu);
  }
  for (int f = 0; f < nf; f++) prolong(c, pf, (const char*)c.cw_ce.p + f * nco * ec, pc, (char*)z + f * nfi * ef, 0);
  if (nf == 2) sap_sweeps_nd(c, pf, z, r, c.mg.sap_sweeps);
  else sap_sweeps(c, pf, z, r, nullptr, mu, c.mg.sap_sweeps);
}

// ---------------------------------------------------------------- cycle as a CUDA graph
// The cycle's launches (P^dag, the persistent coarse solve, P, the SAP sweeps) are captured once per
// key and replayed with one cudaGraphLaunch.  The key holds everything the launches bake in, so a
// changed parameter, knob or (re)allocated buffer leads to a new capture instead of a stale graph.
static std::vector<unsigned long long> cycle_key(const Ctx& c, int pf, int pc, const void* r, const void* z, double mu,
                                                 int nf) {
  auto u = [](const void* p) { return (unsigned long long)(uintptr_t)p; };
  auto d = [](double v) {
    unsigned long long b;
    memcpy(&b, &v, sizeof b);
    return b;
  };
  std::vector<unsigned long long> k = {u(r), u(z), (unsigned long long)pf, (unsigned long long)pc, (unsigned long long)nf,
                                       d(mu), d(c.mubar), d(c.epsbar), d(c.ndshift), (unsigned long long)(c.g.tbc + 2),
                                       (unsigned long long)c.l2_ready, (unsigned long long)c.mg.sap_sweeps,
                                       (unsigned long long)c.mg.sap_mr, (unsigned long long)c.mg.coarse_m, d(c.mg.coarse_rtol),
                                       (unsigned long long)c.coarse_ctas_per_sm, (unsigned long long)c.coarse_gs_passes,
                                       (unsigned long long)c.kcycle_ctas_per_sm, (unsigned long long)c.coarse_grid,
                                       (unsigned long long)c.kcycle_grid, (unsigned long long)c.coarse_overlap,
                                       (unsigned long long)c.coarse_block_cache, (unsigned long long)c.coarse_eo,
                                       (unsigned long long)(c.coarse_eo ? c.cl.version : 0), (unsigned long long)c.l2p.smooth_m,
                                       (unsigned long long)c.l2p.k_restart, d(c.l2p.k_rtol), (unsigned long long)c.l2p.coarse_m,
                                       d(c.l2p.coarse_rtol), (unsigned long long)c.tc_pipeline,
                                       (unsigned long long)c.tc_steps_per_range};
  for (int i = 0; i < 3; i++) {
    k.push_back(u(c.op[i].U.p));
    k.push_back(u(c.op[i].A.p));
    k.push_back(u(c.op[i].Ascale.p));
  }
  for (const DBuf* b : {&c.cl.W64, &c.cl.W32, &c.cl.Dc64, &c.cl.Dc32, &c.cl.nbr, &c.cl2.W64, &c.cl2.W32, &c.cl2.Dc64,
                        &c.cl2.Dc32, &c.cl2.nbr, &c.cw_cr, &c.cw_ce, &c.cw_V, &c.cw_w, &c.cw_part, &c.coarse_iter_dev,
                        &c.kw, &c.kbw, &c.l2_iter_dev, &c.tc_err}) {
    k.push_back(u(b->p));
    k.push_back((unsigned long long)b->bytes);
  }
  return k;
}

static void cycle_run(Ctx& c, int pf, int pc, const void* r, void* z, double mu, int nf = 1) {
  if (!c.cycle_graphs || c.prof.on) {
    cycle_p(c, pf, pc, r, z, mu, nf);
    return;
  }
  std::vector<unsigned long long> key = cycle_key(c, pf, pc, r, z, mu, nf);
  for (auto& e : c.graphs.g)
    if (e.key == key) {
      TMG_CUDA(cudaGraphLaunch(e.exec, c.stream));
      c.launches += e.kernels;
      return;
    }
  // miss: run the cycle eagerly (its result is this call's result and every buffer it needs is now
  // allocated), then capture the same launches for the next call with this key
  cycle_p(c, pf, pc, r, z, mu, nf);
  if (cycle_key(c, pf, pc, r, z, mu, nf) != key) return;   // the eager run allocated: capture next time
  if (!c.graphs.cap) TMG_CUDA(cudaStreamCreateWithFlags(&c.graphs.cap, cudaStreamNonBlocking));
  if (c.graphs.g.size() >= 64) c.graphs.clear();
  cudaStream_t saved = c.stream;
  const long long l0 = c.launches;
  cudaGraph_t graph = nullptr;
  c.stream = c.graphs.cap;
  cudaError_t err = cudaStreamBeginCapture(c.graphs.cap, cudaStreamCaptureModeRelaxed);
  if (err == cudaSuccess) {
    try {
      cycle_p(c, pf, pc, r, z, mu, nf);
    } catch (const Error&) {
      err = cudaErrorStreamCaptureInvalidated;
    }
    const cudaError_t e2 = cudaStreamEndCapture(c.graphs.cap, &graph);
    if (err == cudaSuccess) err = e2;
  }
  c.stream = saved;
  const long long kernels = c.launches - l0;
  c.launches = l0;
  cudaGraphExec_t exec = nullptr;
  if (err == cudaSuccess && graph) err = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (err != cudaSuccess || !exec) {
    cudaGetLastError();   // clear the capture error; this context runs the cycle eagerly from now on
    c.cycle_graphs = 0;
    return;
  }
  c.graphs.g.push_back(CycleGraph{key, exec, kernels});
}

void mg_cycle(Ctx& c, const void* r, void* z, double mu) { cycle_p(c, c.mg.prec_fine, c.mg.prec_coarse, r, z, mu); }

// ---------------------------------------------------------------- launch-shape autotuner
// Times the persistent coarse solve (and, with three levels, the K-cycle) for every allowed launch
// shape on a fixed right-hand side with the stopping test disabled (fixed work per call), keeps the
// fastest shape in the context and returns its time in milliseconds.
double autotune(Ctx& c) {
  const int pc = c.mg.prec_coarse;
  const size_t n = (size_t)c.cl.nc * c.cl.nd;
  DBuf b, x;
  b.alloc(n * esize(pc));
  x.alloc(n * esize(pc));
  std::vector<double> ones(2 * n, 0.0);
  for (size_t i = 0; i < n; i++) ones[2 * i] = 1.0;
  DBuf h;
  h.alloc(2 * n * sizeof(double));
  TMG_CUDA(cudaMemcpyAsync(h.p, ones.data(), 2 * n * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  convert_field(c, h.p, TMG_PREC_F64, b.p, pc, n);
  cudaEvent_t e0, e1;
  TMG_CUDA(cudaEventCreate(&e0));
  TMG_CUDA(cudaEventCreate(&e1));
  const bool prof = c.prof.on;
  c.prof.on = false;
  auto time_of = [&](auto&& run) {
    run();
    std::vector<float> t(3);
    for (auto& v : t) {
      TMG_CUDA(cudaEventRecord(e0, c.stream));
      run();
      TMG_CUDA(cudaEventRecord(e1, c.stream));
      TMG_CUDA(cudaEventSynchronize(e1));
      TMG_CUDA(cudaEventElapsedTime(&v, e0, e1));
    }
    std::sort(t.begin(), t.end());
    return (double)t[1];
  };
  double best = 0.0;
  const double rtol = c.mg.coarse_rtol;
  c.mg.coarse_rtol = 0.0;
  try {
    if (c.l2_ready) {
      const double krtol = c.l2p.k_rtol;
      c.l2p.k_rtol = 0.0;
      int best_k = c.kcycle_ctas_per_sm, best_g = 0;
      best = 1e30;
      for (int k = 1; k <= 4; k++) {
        c.kcycle_ctas_per_sm = k;
        c.kcycle_grid = 0;
        const double t = time_of([&] { kcycle(c, pc, b.p, x.p, c.mu, 0); });
        if (t < best) { best = t; best_k = k; best_g = 0; }
      }
      for (int g : {c.sms / 4, c.sms / 2}) {   // fewer CTAs than SMs: cheaper grid-wide barriers
        c.kcycle_ctas_per_sm = 1;
        c.kcycle_grid = g;
        const double t = time_of([&] { kcycle(c, pc, b.p, x.p, c.mu, 0); });
        if (t < best) { best = t; best_k = 1; best_g = g; }
      }
      c.kcycle_ctas_per_sm = best_k;
      c.kcycle_grid = best_g;
      c.l2p.k_rtol = krtol;
    } else {
      int best_ctas = c.coarse_ctas_per_sm, best_pass = c.coarse_gs_passes, best_g = 0, best_ovl = c.coarse_overlap;
      best = 1e30;
      // grids of k CTAs per SM, and grids smaller than the SM count (cheaper grid-wide barriers),
      // with and without the Hessenberg update overlapped with the next stencil
      const int grids[] = {0, 0, 0, 0, c.sms / 4, c.sms / 2};
      for (int ovl = 0; ovl <= 1; ovl++)
        for (int gi = 0; gi < 6; gi++)
          for (int pass = (pc == TMG_PREC_F64 ? 2 : 1); pass <= 2; pass++) {
            c.coarse_ctas_per_sm = gi < 4 ? gi + 1 : 1;
            c.coarse_grid = grids[gi];
            c.coarse_gs_passes = pass;
            c.coarse_overlap = ovl;
            const double t = time_of([&] { coarse_gmres_persistent(c, pc, b.p, x.p, c.mu); });
            if (t < best) { best = t; best_ctas = c.coarse_ctas_per_sm; best_pass = pass; best_g = grids[gi]; best_ovl = ovl; }
          }
      c.coarse_ctas_per_sm = best_ctas;
      c.coarse_gs_passes = best_pass;
      c.coarse_grid = best_g;
      c.coarse_overlap = best_ovl;
    }
  } catch (...) {
    c.mg.coarse_rtol = rtol;
    c.prof.on = prof;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    throw;
  }
  c.mg.coarse_rtol = rtol;
  c.prof.on = prof;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return best;
}
void mg_cycle_nd(Ctx& c, const void* r, void* z) { cycle_p(c, c.mg.prec_fine, c.mg.prec_coarse, r, z, 0.0, 2); }

// ---------------------------------------------------------------- setup
static void set_vectors2(Ctx& c, int pc);
static void set_vectors(Ctx& c, int sp) {
  const size_t n = (size_t)12 * c.g.V;
  const size_t es = esize(sp);
  for (int j = 0; j < c.cl.nv; j++)
    convert_field(c, (const char*)c.sv_raw.p + j * n * es, sp, c.cl.W64.as<double2>() + j * n, TMG_PREC_F64, n);
  orthonormalise(c, c.cl.W64.p);
  convert_field(c, c.cl.W64.p, TMG_PREC_F64, c.cl.W32.p, TMG_PREC_F32, n * c.cl.nv);
  build_coarse(c);
}

void mg_setup(Ctx& c, const double* v0_lex) {
  c.l2_ready = false;
  const int nv = c.mg.nv;
  c.cl.nv = nv;
  c.cl.nd = 2 * nv;
  c.cl.nc = c.g.nblk;
  for (int mu = 0; mu < 4; mu++) c.cl.cgeom[mu] = c.g.NB[mu];
  const size_t n = (size_t)12 * c.g.V;
  const int pf = c.mg.prec_fine, sp = storage(pf);
  const size_t es = esize(sp);
  c.cl.W64.alloc(nv * n * 16);
  c.cl.W32.alloc(nv * n * 8);
  c.sv_raw.alloc(nv * n * es);
  c.fw_t.alloc(2 * n * es);
  char* raw = (char*)c.sv_raw.p;
  void* xb = c.fw_t.p;
  void* bb = (char*)c.fw_t.p + n * es;
  for (int j = 0; j < nv; j++) spinor_from_lex(c, v0_lex + (size_t)j * 24 * c.g.V, raw + j * n * es, sp);
  for (int pass = 0; pass < c.mg.n_init; pass++) {
    for (int j = 0; j < nv; j++) {
      void* vj = raw + j * n * es;
      blas_copy(c, vj, bb, sp, n);
      blas_zero(c, xb, sp, n);
      sap_sweeps(c, pf, xb, bb, nullptr, c.mu, c.mg.sap_sweeps);
      const double nrm = std::sqrt(blas_norm2(c, xb, sp, n));
      if (!(nrm > 0.0) || !std::isfinite(nrm)) throw Error{TMG_ERR_BREAKDOWN, "setup: test vector vanished"};
      blas_copy(c, xb, vj, sp, n);
      blas_scale(c, 1.0 / nrm, 0.0, vj, sp, n);
    }
  }
  set_vectors(c, sp);
  c.mg_ready = true;
  for (int it = 0; it < c.mg.n_iter; it++) {
    for (int j = 0; j < nv; j++) {
      void* vj = raw + j * n * es;
      cycle_p(c, pf, c.mg.prec_coarse, vj, xb, c.mu);
      const double nrm = std::sqrt(blas_norm2(c, xb, sp, n));
      if (!(nrm > 0.0) || !std::isfinite(nrm)) throw Error{TMG_ERR_BREAKDOWN, "setup: test vector vanished"};
      blas_copy(c, xb, vj, sp, n);
      blas_scale(c, 1.0 / nrm, 0.0, vj, sp, n);
    }
    set_vectors(c, sp);
  }
  TMG_CUDA(cudaStreamSynchronize(c.stream));
}

// Setup update (Sec. 2: the subspace of the previous setup is refined by one setup iteration
// whenever the gauge field has moved): n_iter passes of v_j <- normalise(cycle(v_j)) on the current
// operator, starting from the raw test vectors the last setup kept, each pass followed by a
// rebuild of P and D_c; with three levels the level-2 vectors then get the same number of passes
// of the level-1 cycle.
void mg_setup_update(Ctx& c, int n_iter) {
  const size_t n = (size_t)12 * c.g.V;
  const int pf = c.mg.prec_fine, sp = storage(pf);
  const size_t es = esize(sp);
  const bool three = c.l2_ready;
  c.l2_ready = false;   // level 1 alone while its vectors move (the level-2 basis refers to them)
  set_vectors(c, sp);   // P and D_c of the current field from the kept vectors
  c.fw_t.alloc(2 * n * es);
  char* raw = (char*)c.sv_raw.p;
  void* xb = c.fw_t.p;
  for (int it = 0; it < n_iter; it++) {
    for (int j = 0; j < c.cl.nv; j++) {
      void* vj = raw + j * n * es;
      cycle_p(c, pf, c.mg.prec_coarse, vj, xb, c.mu);
      const double nrm = std::sqrt(blas_norm2(c, xb, sp, n));
      if (!(nrm > 0.0) || !std::isfinite(nrm)) throw Error{TMG_ERR_BREAKDOWN, "setup update: test vector vanished"};
      blas_copy(c, xb, vj, sp, n);
      blas_scale(c, 1.0 / nrm, 0.0, vj, sp, n);
    }
    set_vectors(c, sp);
  }
  if (three) {
    const int pc = c.mg.prec_coarse;
    const size_t n1 = (size_t)c.cl.nc * c.cl.nd;
    const size_t ec = esize(pc);
    set_vectors2(c, pc);
    c.l2_ready = true;
    DBuf tmp;
    tmp.alloc(n1 * ec);
    char* raw2 = (char*)c.sv2.p;
    for (int it = 0; it < n_iter; it++) {
      for (int j = 0; j < c.cl2.nv; j++) {
        void* vj = raw2 + j * n1 * ec;
        kcycle(c, pc, vj, tmp.p, c.mu, 1);
        const double nrm = std::sqrt(blas_norm2(c, tmp.p, pc, n1));
        if (!(nrm > 0.0) || !std::isfinite(nrm)) throw Error{TMG_ERR_BREAKDOWN, "setup update: level-2 vector vanished"};
        blas_copy(c, tmp.p, vj, pc, n1);
        blas_scale(c, 1.0 / nrm, 0.0, vj, pc, n1);
      }
      set_vectors2(c, pc);
    }
  }
  TMG_CUDA(cudaStreamSynchronize(c.stream));
}

// ---------------------------------------------------------------- level-2 setup (three levels)
static void set_vectors2(Ctx& c, int pc) {
  const size_t n1 = (size_t)c.cl.nc * c.cl.nd;
  convert_field(c, c.sv2.p, pc, c.cl2.W64.p, TMG_PREC_F64, n1 * c.cl2.nv);
  orthonormalise_c(c);
  convert_field(c, c.cl2.W64.p, TMG_PREC_F64, c.cl2.W32.p, TMG_PREC_F32, n1 * c.cl2.nv);
  build_coarse_c(c);
}

void mg_setup2(Ctx& c, const double* v1_dev) {
  const tmg_level2_params& p = c.l2p;
  c.l2_ready = false;
  Coarse2& q = c.cl2;
  for (int mu = 0; mu < 4; mu++) {
    q.agg[mu] = p.agg[mu];
    q.cgeom[mu] = c.g.NB[mu] / p.agg[mu];
  }
  q.nv = p.nv;
  q.nd = 2 * p.nv;
  q.nc = q.cgeom[0] * q.cgeom[1] * q.cgeom[2] * q.cgeom[3];
  const size_t n1 = (size_t)c.cl.nc * c.cl.nd;
  const int pc = c.mg.prec_coarse;
  const size_t es = esize(pc);
  q.W64.alloc(p.nv * n1 * 16);
  q.W32.alloc(p.nv * n1 * 8);
  c.sv2.alloc(p.nv * n1 * es);
  DBuf tmp;
  tmp.alloc(n1 * es);
  char* raw = (char*)c.sv2.p;
  convert_field(c, v1_dev, TMG_PREC_F64, raw, pc, n1 * p.nv);
  auto normalise_into = [&](void* vj) {
    const double nrm = std::sqrt(blas_norm2(c, tmp.p, pc, n1));
    if (!(nrm > 0.0) || !std::isfinite(nrm)) throw Error{TMG_ERR_BREAKDOWN, "level-2 setup: test vector vanished"};
    blas_copy(c, tmp.p, vj, pc, n1);
    blas_scale(c, 1.0 / nrm, 0.0, vj, pc, n1);
  };
  for (int pass = 0; pass < p.n_init; pass++)
    for (int j = 0; j < p.nv; j++) {
      void* vj = raw + j * n1 * es;
      kcycle(c, pc, vj, tmp.p, c.mu, 2);
      normalise_into(vj);
    }
  set_vectors2(c, pc);
  c.l2_ready = true;
  for (int it = 0; it < p.n_iter; it++) {
    for (int j = 0; j < p.nv; j++) {
      void* vj = raw + j * n1 * es;
      kcycle(c, pc, vj, tmp.p, c.mu, 1);
      normalise_into(vj);
    }
    set_vectors2(c, pc);
  }
  TMG_CUDA(cudaStreamSynchronize(c.stream));
}

// ---------------------------------------------------------------- outer flexible GMRES
// One FGMRES cycle of at most m steps on D(mu) e = r from zero (vectors in storage sp, operator
// precision op, preconditioner = cycle in (pf, pc)).  Host-side Givens; dots accumulate in FP64.
static void fgmres_cycle(Ctx& c, int sp, int op, int pf, int pc, const void* r, void* e, double mu, int m,
                         double rtol, int& steps, int nf = 1) {
  const size_t n = (size_t)nf * 12 * c.g.V;
  const size_t es = esize(sp);
  c.fw_V.alloc((m + 1) * n * es);
  c.fw_Z.alloc(m * n * es);
  c.fw_w.alloc(n * es);
  c.fw_part.alloc(sizeof(double2) * NPART * (MAXM + 2));
  c.fw_h.alloc(sizeof(double2) * 2 * (MAXM + 1));
  double2* part = c.fw_part.as<double2>();
  double2* hdev = c.fw_h.as<double2>();
  const int rg = red_grid(c, n);
  std::vector<std::complex<double>> H((m + 1) * m), cs(m), sn(m), g(m + 1), y(m);
  const double beta = std::sqrt(blas_norm2(c, r, sp, n));
  steps = 0;
  if (!(beta > 0.0)) {
    blas_zero(c, e, sp, n);
    return;
  }
  char* V = (char*)c.fw_V.p;
  char* Z = (char*)c.fw_Z.p;
  blas_copy(c, r, V, sp, n);
  blas_scale(c, 1.0 / beta, 0.0, V, sp, n);
  g[0] = beta;
  int k = 0;
  for (int j = 0; j < m; j++) {
    void* vj = V + j * n * es;
    void* zj = Z + j * n * es;
    cycle_run(c, pf, pc, vj, zj, mu, nf);
    if (nf == 2) dslash_nd(c, op, c.fw_w.p, zj);
    else dslash(c, op, c.fw_w.p, zj, nullptr, mu, 0, 0);
    std::vector<double2> hc(j + 1), hc2(j + 1, make_double2(0.0, 0.0));
    std::vector<double2> nn_parts(NPART);
    // classical Gram-Schmidt, two passes (the second restores the orthogonality the first loses in
    // FP32), or one pass when outer_gs_passes = 1
    const int npass = c.outer_gs_passes == 1 ? 1 : 2;
    dispatch(sp, [&](auto tag) {
      using T2 = decltype(tag);
      if (npass == 2 && c.outer_gs_fused && j + 1 <= FUSED_MAX) {
        // classical Gram-Schmidt, two passes, with pass 1's update and pass 2's dots in one sweep
        ++c.launches, k_mdot_partial<T2><<<dim3(rg, j + 1), 256, 0, c.stream>>>((const T2*)V, n, (const T2*)c.fw_w.p, n, part, nullptr);
        ++c.launches, k_mdot_final<<<j + 1, 256, 0, c.stream>>>(part, rg, j + 1, hdev, nullptr);
        ++c.launches, k_mgs_update_dot<T2><<<rg, 256, 0, c.stream>>>((const T2*)V, n, j + 1, hdev, (T2*)c.fw_w.p, n, part);
        ++c.launches, k_mdot_final<<<j + 1, 256, 0, c.stream>>>(part, rg, j + 1, hdev + (MAXM + 1), nullptr);
        ++c.launches, k_mgs_update<T2><<<rg, 256, 0, c.stream>>>((const T2*)V, n, j + 1, hdev + (MAXM + 1), (T2*)c.fw_w.p, n,
                                                   part + NPART * (MAXM + 1), nullptr);
        TMG_CHECK_LAUNCH();
      } else {
        for (int pass = 0; pass < npass; pass++) {
          ++c.launches, k_mdot_partial<T2><<<dim3(rg, j + 1), 256, 0, c.stream>>>((const T2*)V, n, (const T2*)c.fw_w.p, n, part, nullptr);
          ++c.launches, k_mdot_final<<<j + 1, 256, 0, c.stream>>>(part, rg, j + 1, hdev + pass * (MAXM + 1), nullptr);
          ++c.launches, k_mgs_update<T2><<<rg, 256, 0, c.stream>>>((const T2*)V, n, j + 1, hdev + pass * (MAXM + 1), (T2*)c.fw_w.p, n,
                                                     pass == npass - 1 ? part + NPART * (MAXM + 1) : nullptr, nullptr);
          TMG_CHECK_LAUNCH();
        }
      }
    });
    TMG_CUDA(cudaMemcpyAsync(hc.data(), hdev, sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost, c.stream));
    if (npass == 2)
      TMG_CUDA(cudaMemcpyAsync(hc2.data(), hdev + (MAXM + 1), sizeof(double2) * (j + 1), cudaMemcpyDeviceToHost, c.stream));
    TMG_CUDA(cudaMemcpyAsync(nn_parts.data(), part + NPART * (MAXM + 1), sizeof(double2) * rg, cudaMemcpyDeviceToHost, c.stream));
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    double nn = 0.0;
    for (int q = 0; q < rg; q++) nn += nn_parts[q].x;
    const double hn = std::sqrt(nn);
    std::complex<double>* h = &H[j * (m + 1)];
    for (int i = 0; i <= j; i++) h[i] = std::complex<double>(hc[i].x + hc2[i].x, hc[i].y + hc2[i].y);
    h[j + 1] = hn;
    for (int i = 0; i < j; i++) {
      const std::complex<double> a = h[i], b = h[i + 1];
      h[i] = std::conj(cs[i]) * a + std::conj(sn[i]) * b;
      h[i + 1] = -sn[i] * a + cs[i] * b;
    }
    const std::complex<double> a = h[j], b = h[j + 1];
    const double den = std::sqrt(std::norm(a) + std::norm(b));
    if (!std::isfinite(den)) throw Error{TMG_ERR_BREAKDOWN, "fgmres: non-finite Hessenberg entry"};
    cs[j] = den > 0 ? a / den : 1.0;
    sn[j] = den > 0 ? b / den : 0.0;
    h[j] = den;
    h[j + 1] = 0.0;
    g[j + 1] = -sn[j] * g[j];
    g[j] = std::conj(cs[j]) * g[j];
    k = j + 1;
    if (std::abs(g[j + 1]) <= rtol * beta || hn == 0.0) break;
    blas_copy(c, c.fw_w.p, V + (j + 1) * n * es, sp, n);
    blas_scale(c, 1.0 / hn, 0.0, V + (j + 1) * n * es, sp, n);
  }
  for (int i = k - 1; i >= 0; i--) {
    std::complex<double> acc = g[i];
    for (int l = i + 1; l < k; l++) acc -= H[l * (m + 1) + i] * y[l];
    y[i] = acc / H[i * (m + 1) + i];
  }
  std::vector<double2> yc(k);
  for (int i = 0; i < k; i++) yc[i] = make_double2(y[i].real(), y[i].imag());
  TMG_CUDA(cudaMemcpyAsync(hdev, yc.data(), sizeof(double2) * k, cudaMemcpyHostToDevice, c.stream));
  dispatch(sp, [&](auto tag) {
    using T2 = decltype(tag);
    ++c.launches, k_combine<T2><<<egrid(c, n), 256, 0, c.stream>>>((const T2*)Z, n, k, nullptr, hdev, (T2*)e, n);
    TMG_CHECK_LAUNCH();
  });
  TMG_CUDA(cudaStreamSynchronize(c.stream));
  steps = k;
}

// ---------------------------------------------------------------- CG comparator (FP64)
// CG on D D^dag y = b with x = D^dag y accumulated directly: q = D^dag p, x += a q, r -= a D q.
static int cg_solve(Ctx& c, const void* b, void* x, double mu, double tol, int maxiter, SolveStats& st) {
  const size_t n = (size_t)12 * c.g.V;
  c.fw_t.alloc(3 * n * 16);
  c.fw_r64.alloc(n * 16);
  void* r = c.fw_r64.p;
  void* p = c.fw_t.p;
  void* q = (char*)c.fw_t.p + n * 16;
  void* Aq = (char*)c.fw_t.p + 2 * n * 16;
  blas_zero(c, x, TMG_PREC_F64, n);
  blas_copy(c, b, r, TMG_PREC_F64, n);
  blas_copy(c, b, p, TMG_PREC_F64, n);
  const double bn2 = blas_norm2(c, b, TMG_PREC_F64, n);
  if (!std::isfinite(bn2)) throw Error{TMG_ERR_BREAKDOWN, "cg: right-hand side is not finite"};
  if (!(bn2 > 0.0)) return TMG_OK;
  double rr = bn2;
  int it = 0;
  while (it < maxiter && rr > tol * tol * bn2) {
    dslash(c, TMG_PREC_F64, q, p, nullptr, mu, 0, 1);
    dslash(c, TMG_PREC_F64, Aq, q, nullptr, mu, 0, 0);
    const double qq = blas_norm2(c, q, TMG_PREC_F64, n);
    if (!(qq > 0.0) || !std::isfinite(qq)) throw Error{TMG_ERR_BREAKDOWN, "cg: breakdown"};
    const double a = rr / qq;
    blas_axpy(c, a, 0.0, q, x, TMG_PREC_F64, n);
    blas_axpy(c, -a, 0.0, Aq, r, TMG_PREC_F64, n);
    const double rr_new = blas_norm2(c, r, TMG_PREC_F64, n);
    blas_xpay(c, r, rr_new / rr, 0.0, p, TMG_PREC_F64, n);
    rr = rr_new;
    it++;
  }
  dslash(c, TMG_PREC_F64, r, x, b, mu, 1, 0);
  st.iterations = it;
  st.true_residual = std::sqrt(blas_norm2(c, r, TMG_PREC_F64, n) / bn2);
  return st.true_residual <= tol ? TMG_OK : TMG_ERR_NOCONV;
}

// ---------------------------------------------------------------- solve
int solve_one(Ctx& c, int method, const void* b, void* x, double mu, double tol, int maxiter, SolveStats& st, int nf,
              bool use_x0) {
  if (method == TMG_SOLVE_CG_F64) return cg_solve(c, b, x, mu, tol, maxiter, st);
  const size_t n = (size_t)nf * 12 * c.g.V;
  // r = b - D x in FP64 (D_ND for the doublet)
  auto residual = [&](void* r) {
    if (nf == 2) {
      dslash_nd(c, TMG_PREC_F64, r, x);
      blas_xpay(c, b, -1.0, 0.0, r, TMG_PREC_F64, n);
    } else {
      dslash(c, TMG_PREC_F64, r, x, b, mu, 1, 0);
    }
  };
  const bool f64 = method == TMG_SOLVE_MG_F64;
  const int pf = f64 ? TMG_PREC_F64 : c.mg.prec_fine;
  const int pc = f64 ? TMG_PREC_F64 : c.mg.prec_coarse;
  const int sp = storage(pf);
  const int op = pf;
  const size_t es = esize(sp);
  c.fw_r64.alloc(n * 16);
  c.fw_e.alloc(n * es);
  c.fw_x.alloc(n * es);
  int c0 = 0, c1 = 0;
  if (c.coarse_iter_dev.p) TMG_CUDA(cudaMemcpyAsync(&c0, c.coarse_iter_dev.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  if (use_x0) {
    residual(c.fw_r64.p);            // start from the caller's x
  } else {
    blas_zero(c, x, TMG_PREC_F64, n);
    blas_copy(c, b, c.fw_r64.p, TMG_PREC_F64, n);
  }
  const double bn = std::sqrt(blas_norm2(c, b, TMG_PREC_F64, n));
  if (!std::isfinite(bn)) throw Error{TMG_ERR_BREAKDOWN, "solve: right-hand side is not finite"};
  if (!(bn > 0.0)) return TMG_OK;
  int rc = TMG_OK;
  while (true) {
    const double rn = std::sqrt(blas_norm2(c, c.fw_r64.p, TMG_PREC_F64, n));
    if (!std::isfinite(rn)) {
      rc = TMG_ERR_BREAKDOWN;
      break;
    }
    st.true_residual = rn / bn;
    if (rn <= tol * bn) break;
    if (st.iterations >= maxiter) {
      rc = TMG_ERR_NOCONV;
      break;
    }
    // unit-norm residual in the working precision
    convert_field(c, c.fw_r64.p, TMG_PREC_F64, c.fw_x.p, sp, n);
    blas_scale(c, 1.0 / rn, 0.0, c.fw_x.p, sp, n);
    double target = tol * bn / rn;
    if (!f64) target = std::max(target, 1e-6);
    int k = 0;
    fgmres_cycle(c, sp, op, pf, pc, c.fw_x.p, c.fw_e.p, mu, std::min(c.mg.restart, MAXM), target, k, nf);
    st.iterations += k;
    blas_axpy_mixed(c, rn, c.fw_e.p, sp, x, TMG_PREC_F64, n);
    residual(c.fw_r64.p);
    st.refinements++;
    if (k == 0) {
      rc = TMG_ERR_BREAKDOWN;
      break;
    }
  }
  if (c.coarse_iter_dev.p) {
    TMG_CUDA(cudaMemcpyAsync(&c1, c.coarse_iter_dev.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    st.coarse_iterations = c1 - c0;
  }
  return rc;
}

// ---------------------------------------------------------------- odd-even CG (FP64)
// D(mu) x = b through the even-odd reduction (Sec. 1.2; the odd-even CG of Fig. 1): CG on
// Dhat Dhat^dag y = rhs_o with x_o = Dhat^dag y, rhs_o = b_o - H_oe M_e^-1 b_e, then
// x_e = M_e^-1 (b_e - H_eo x_o).  b, x: lexicographic FP64 full-lattice fields on the device.
int cg_eo_solve(Ctx& c, const double* b_lex, double* x_lex, double tol, int maxiter, SolveStats& st) {
  eo_prepare(c);
  const size_t h = (size_t)c.g.V / 2, n = 12 * h;
  DBuf buf;
  buf.alloc(8 * n * 16);
  char* base = buf.as<char>();
  void* be = base;
  void* bo = base + n * 16;
  void* xo = base + 2 * n * 16;
  void* r = base + 3 * n * 16;
  void* p = base + 4 * n * 16;
  void* q = base + 5 * n * 16;
  void* Aq = base + 6 * n * 16;
  void* t = base + 7 * n * 16;
  eo_from_lex(c, b_lex, be, 0, TMG_PREC_F64);
  eo_from_lex(c, b_lex, bo, 1, TMG_PREC_F64);
  const double bn2 = blas_norm2(c, be, TMG_PREC_F64, n) + blas_norm2(c, bo, TMG_PREC_F64, n);
  if (!std::isfinite(bn2)) throw Error{TMG_ERR_BREAKDOWN, "cg_eo: right-hand side is not finite"};
  blas_zero(c, xo, TMG_PREC_F64, n);
  if (!(bn2 > 0.0)) {
    blas_zero(c, t, TMG_PREC_F64, n);
    eo_to_lex(c, t, x_lex, 0, TMG_PREC_F64, 1);
    return TMG_OK;
  }
  // rhs_o = b_o - H_oe M_e^-1 b_e
  eo_kernel(c, TMG_PREC_F64, 0, t, nullptr, be, 1.0, 1, 0);
  eo_kernel(c, TMG_PREC_F64, 1, r, bo, t, 1.0, 0, 0);
  blas_copy(c, r, p, TMG_PREC_F64, n);
  const double rhs2 = blas_norm2(c, r, TMG_PREC_F64, n);
  double rr = rhs2;
  int it = 0;
  // the odd-site system is solved until its residual is tol ||b||: the reconstruction keeps the
  // even-site residual at rounding level, so the full residual follows the odd one
  while (it < maxiter && rr > tol * tol * bn2) {
    eo_apply(c, TMG_PREC_F64, q, p, t, 1);
    eo_apply(c, TMG_PREC_F64, Aq, q, t, 0);
    const double qq = blas_norm2(c, q, TMG_PREC_F64, n);
    if (!(qq > 0.0) || !std::isfinite(qq)) throw Error{TMG_ERR_BREAKDOWN, "cg_eo: breakdown"};
    const double a = rr / qq;
    blas_axpy(c, a, 0.0, q, xo, TMG_PREC_F64, n);
    blas_axpy(c, -a, 0.0, Aq, r, TMG_PREC_F64, n);
    const double rr_new = blas_norm2(c, r, TMG_PREC_F64, n);
    blas_xpay(c, r, rr_new / rr, 0.0, p, TMG_PREC_F64, n);
    rr = rr_new;
    it++;
  }
  // x_e = M_e^-1 (b_e - H_eo x_o)
  eo_kernel(c, TMG_PREC_F64, 0, t, xo, be, -1.0, 1, 0);
  eo_to_lex(c, t, x_lex, 0, TMG_PREC_F64, 0);
  eo_to_lex(c, xo, x_lex, 1, TMG_PREC_F64, 0);
  eo_check(c);
  // true residual of the full system with the full-lattice FP64 operator
  c.fw_t.alloc(2 * 12 * (size_t)c.g.V * 16);
  void* xf = c.fw_t.p;
  void* rf = c.fw_t.as<char>() + 12 * (size_t)c.g.V * 16;
  void* bf = c.fw_r64.p;
  c.fw_r64.alloc(12 * (size_t)c.g.V * 16);
  bf = c.fw_r64.p;
  spinor_from_lex(c, x_lex, xf, TMG_PREC_F64);
  spinor_from_lex(c, b_lex, bf, TMG_PREC_F64);
  dslash(c, TMG_PREC_F64, rf, xf, bf, c.mu, 1, 0);
  st.iterations = it;
  st.true_residual = std::sqrt(blas_norm2(c, rf, TMG_PREC_F64, 12 * (size_t)c.g.V) / bn2);
  return st.true_residual <= tol ? TMG_OK : TMG_ERR_NOCONV;
}

// ---------------------------------------------------------------- multi-shift CG (FP64)
// x_s = (A + sigma_s)^-1 b for all shifts at once with A = D(mu)^dag D(mu) (nf = 1) or
// A = Q_ND^2 = D_ND^dag D_ND, Q_ND = (g5 x tau1) D_ND (nf = 2, Eqs. 2 and 4): the comparator of the
// rational approximation's shifted solves (Sec. 3, MMS-CG).  The Krylov space is that of the seed
// system A x = b; system s keeps a residual collinear with the seed's, r_s = zeta_s r, with the
// shifted coefficients from the seed's alpha, beta (the recurrences of the shifted-CG
// literature).  X: ns internal FP64 fields (nf flavours each).  Stops when every shifted residual is
// <= tol ||b||; st.iterations = seed iterations, st.true_residual = the largest recomputed
// ||b - (A + sigma_s) x_s|| / ||b||.
int mms_cg_solve(Ctx& c, const void* b, void* X, int ns, const double* sigma, double tol, int maxiter, int nf,
                 SolveStats& st) {
  const size_t n1 = (size_t)12 * c.g.V, n = nf * n1;
  DBuf buf;
  buf.alloc((size_t)(4 + ns) * n * 16);
  char* base = buf.as<char>();
  void* r = base;
  void* p = base + n * 16;
  void* Ap = base + 2 * n * 16;
  void* t = base + 3 * n * 16;
  auto ps = [&](int s) { return (void*)(base + (size_t)(4 + s) * n * 16); };
  auto xs = [&](int s) { return (void*)((char*)X + (size_t)s * n * 16); };
  // y = g5 tau1 v for doublet fields [2][12 V]
  auto g5_tau1 = [&](const void* v, void* y) {
    blas_copy(c, v, (char*)y + n1 * 16, TMG_PREC_F64, n1);
    blas_copy(c, (const char*)v + n1 * 16, y, TMG_PREC_F64, n1);
    gamma5_inplace(c, y, TMG_PREC_F64);
    gamma5_inplace(c, (char*)y + n1 * 16, TMG_PREC_F64);
  };
  auto applyA = [&](const void* v, void* out) {
    if (nf == 1) {
      dslash(c, TMG_PREC_F64, t, v, nullptr, c.mu, 0, 0);
      dslash(c, TMG_PREC_F64, out, t, nullptr, c.mu, 0, 1);
    } else {
      dslash_nd(c, TMG_PREC_F64, out, v);
      g5_tau1(out, t);
      dslash_nd(c, TMG_PREC_F64, out, t);
      g5_tau1(out, t);
      blas_copy(c, t, out, TMG_PREC_F64, n);
    }
  };
  const double bn2 = blas_norm2(c, b, TMG_PREC_F64, n);
  if (!std::isfinite(bn2)) throw Error{TMG_ERR_BREAKDOWN, "mms_cg: right-hand side is not finite"};
  for (int s = 0; s < ns; s++) blas_zero(c, xs(s), TMG_PREC_F64, n);
  if (!(bn2 > 0.0)) return TMG_OK;
  blas_copy(c, b, r, TMG_PREC_F64, n);
  blas_copy(c, b, p, TMG_PREC_F64, n);
  for (int s = 0; s < ns; s++) blas_copy(c, b, ps(s), TMG_PREC_F64, n);
  std::vector<double> zc(ns, 1.0), zo(ns, 1.0);
  std::vector<char> active(ns, 1);
  double alpha_old = 1.0, beta_old = 0.0, rr = bn2;
  int it = 0, n_active = ns;
  while (it < maxiter && n_active > 0) {
    applyA(p, Ap);
    double pre, pim;
    blas_dot(c, p, Ap, TMG_PREC_F64, n, &pre, &pim);
    if (!(pre > 0.0) || !std::isfinite(pre)) throw Error{TMG_ERR_BREAKDOWN, "mms_cg: breakdown"};
    const double alpha = rr / pre;
    blas_axpy(c, -alpha, 0.0, Ap, r, TMG_PREC_F64, n);
    const double rr_new = blas_norm2(c, r, TMG_PREC_F64, n);
    const double beta = rr_new / rr;
    for (int s = 0; s < ns; s++) {
      if (!active[s]) continue;
      const double zn = zc[s] * zo[s] * alpha_old /
                        (alpha * beta_old * (zo[s] - zc[s]) + zo[s] * alpha_old * (1.0 + sigma[s] * alpha));
      const double as = alpha * zn / zc[s];
      const double bs = beta * (zn / zc[s]) * (zn / zc[s]);
      blas_axpy(c, as, 0.0, ps(s), xs(s), TMG_PREC_F64, n);
      blas_scale(c, bs, 0.0, ps(s), TMG_PREC_F64, n);
      blas_axpy(c, zn, 0.0, r, ps(s), TMG_PREC_F64, n);
      zo[s] = zc[s];
      zc[s] = zn;
      if (std::fabs(zn) * std::sqrt(rr_new) <= tol * std::sqrt(bn2)) {
        active[s] = 0;
        n_active--;
      }
    }
    blas_xpay(c, r, beta, 0.0, p, TMG_PREC_F64, n);
    alpha_old = alpha;
    beta_old = beta;
    rr = rr_new;
    it++;
  }
  st.iterations = it;
  double worst = 0.0;
  for (int s = 0; s < ns; s++) {   // recomputed residuals b - (A + sigma_s) x_s
    applyA(xs(s), Ap);
    blas_axpy(c, sigma[s], 0.0, xs(s), Ap, TMG_PREC_F64, n);
    blas_xpay(c, b, -1.0, 0.0, Ap, TMG_PREC_F64, n);
    worst = std::max(worst, std::sqrt(blas_norm2(c, Ap, TMG_PREC_F64, n) / bn2));
  }
  st.true_residual = worst;
  return n_active == 0 ? TMG_OK : TMG_ERR_NOCONV;
}

// ---------------------------------------------------------------- shifted systems, Taylor guesses
// D(mu_k) x_k = b for k = 0 .. n-1 in order, every x_k to the FP64 residual tol by the mixed
// multigrid.  guess 0: every solve from zero; 1: x_k starts from x_{k-1}; 2: first-order Taylor
// expansion in the twist (Sec. 3: (Q + i mu + i delta)^-1 ~ (Q + i mu)^-1 - i delta (Q + i mu)^-2
// with g5 D(mu) = Q + i mu): x_k^0 = x_{k-1} - i (mu_k - mu_{k-1}) D(mu_{k-1})^-1 g5 x_{k-1}, the
// correction solved only to taylor_tol.  X: n internal FP64 columns.  st accumulates all solves
// (the Taylor corrections included); iters[k] gets the outer iterations of system k alone.
int solve_shifts(Ctx& c, const void* b, void* X, int n, const double* mu, double tol, int guess, double taylor_tol,
                 int maxiter, SolveStats& st, int* iters) {
  const size_t nf = (size_t)12 * c.g.V;
  DBuf tb, tt;
  if (guess == 2) {
    tb.alloc(nf * 16);
    tt.alloc(nf * 16);
  }
  int rc = TMG_OK;
  for (int k = 0; k < n; k++) {
    void* xk = (char*)X + (size_t)k * nf * 16;
    bool x0 = false;
    if (k > 0 && guess >= 1) {
      const void* xp = (const char*)X + (size_t)(k - 1) * nf * 16;
      blas_copy(c, xp, xk, TMG_PREC_F64, nf);
      if (guess == 2) {
        blas_copy(c, xp, tb.p, TMG_PREC_F64, nf);
        gamma5_inplace(c, tb.p, TMG_PREC_F64);
        SolveStats s1{};
        const int r1 = solve_one(c, TMG_SOLVE_MG_MIXED, tb.p, tt.p, mu[k - 1], taylor_tol, maxiter, s1);
        if (r1 != TMG_OK && r1 != TMG_ERR_NOCONV) return r1;
        st.iterations += s1.iterations;
        st.refinements += s1.refinements;
        st.coarse_iterations += s1.coarse_iterations;
        blas_axpy(c, 0.0, -(mu[k] - mu[k - 1]), tt.p, xk, TMG_PREC_F64, nf);   // x -= i delta t
      }
      x0 = true;
    }
    SolveStats sk{};
    const int r = solve_one(c, TMG_SOLVE_MG_MIXED, b, xk, mu[k], tol, maxiter, sk, 1, x0);
    if (iters) iters[k] = sk.iterations;
    st.iterations += sk.iterations;
    st.refinements += sk.refinements;
    st.coarse_iterations += sk.coarse_iterations;
    st.true_residual = std::max(st.true_residual, sk.true_residual);
    if (r != TMG_OK && rc == TMG_OK) rc = r;
  }
  return rc;
}

// ---------------------------------------------------------------- smallest singular value of D_W
// Eigenvalues of a small symmetric matrix (row-major n x n, n <= 64) by cyclic Jacobi rotations;
// on return a holds them on its diagonal and z the eigenvectors in its columns.
static void jacobi_eig(std::vector<double>& a, std::vector<double>& z, int n) {
  z.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; i++) z[(size_t)i * n + i] = 1.0;
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; i++)
      for (int j = 0; j < n; j++) (i == j ? diag : off) += a[(size_t)i * n + j] * a[(size_t)i * n + j];
    if (off <= 1e-30 * diag) break;
    for (int p = 0; p < n; p++)
      for (int q = p + 1; q < n; q++) {
        const double apq = a[(size_t)p * n + q];
        if (apq == 0.0) continue;
        const double th = (a[(size_t)q * n + q] - a[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
        const double cth = 1.0 / std::sqrt(t * t + 1.0), sth = t * cth;
        for (int k = 0; k < n; k++) {   // columns p, q
          const double akp = a[(size_t)k * n + p], akq = a[(size_t)k * n + q];
          a[(size_t)k * n + p] = cth * akp - sth * akq;
          a[(size_t)k * n + q] = sth * akp + cth * akq;
        }
        for (int k = 0; k < n; k++) {   // rows p, q
          const double apk = a[(size_t)p * n + k], aqk = a[(size_t)q * n + k];
          a[(size_t)p * n + k] = cth * apk - sth * aqk;
          a[(size_t)q * n + k] = sth * apk + cth * aqk;
        }
        for (int k = 0; k < n; k++) {
          const double zkp = z[(size_t)k * n + p], zkq = z[(size_t)k * n + q];
          z[(size_t)k * n + p] = cth * zkp - sth * zkq;
          z[(size_t)k * n + q] = sth * zkp + cth * zkq;
        }
      }
  }
}

// sigma_min(D_W) = min |lambda(Q)|, Q = g5 D_W: Lanczos with full reorthogonalisation on
// A = (D(mu_s)^dag D(mu_s))^-1 = (Q^2 + mu_s^2)^-1, each product computed by the two-step solve of
// Sec. 1.1 (D(-mu_s) u = g5 b, then D(mu_s) v = g5 u).  The largest Ritz value theta of A gives
// sigma_min^2 = 1/theta - mu_s^2.  Stops when the Ritz residual beta_j |s_j| <= rtol theta or after k
// steps; *ritz_res gets the last relative Ritz residual, *solves the number of solves.
double sigma_min_lanczos(Ctx& c, const void* start, double mu_s, int k, double rtol, double solve_tol, int method,
                         double* ritz_res, int* solves, int* steps_out) {
  const size_t n = (size_t)12 * c.g.V;
  k = std::max(2, std::min(k, 64));
  DBuf Vb, w, t, u;
  Vb.alloc((size_t)(k + 1) * n * 16);
  w.alloc(n * 16);
  t.alloc(n * 16);
  u.alloc(n * 16);
  char* V = Vb.as<char>();
  auto vec = [&](int j) { return (void*)(V + (size_t)j * n * 16); };
  blas_copy(c, start, vec(0), TMG_PREC_F64, n);
  const double n0 = std::sqrt(blas_norm2(c, vec(0), TMG_PREC_F64, n));
  if (!(n0 > 0.0) || !std::isfinite(n0)) throw Error{TMG_ERR_ARG, "sigma_min: start vector is zero or not finite"};
  blas_scale(c, 1.0 / n0, 0.0, vec(0), TMG_PREC_F64, n);
  std::vector<double> alpha, beta;
  int nsolve = 0;
  double theta = 0.0, res = 1.0;
  int j = 0;
  for (; j < k; j++) {
    // w = A v_j
    blas_copy(c, vec(j), t.p, TMG_PREC_F64, n);
    gamma5_inplace(c, t.p, TMG_PREC_F64);
    SolveStats s1{}, s2{};
    // bounded inner solves: a stalled solve ends with its best iterate instead of running on
    const int maxit = method == TMG_SOLVE_CG_F64 ? 200000 : 4000;
    int rc = solve_one(c, method, t.p, u.p, -mu_s, solve_tol, maxit, s1);
    if (rc != TMG_OK && rc != TMG_ERR_NOCONV) throw Error{rc, "sigma_min: inner solve failed"};
    gamma5_inplace(c, u.p, TMG_PREC_F64);
    rc = solve_one(c, method, u.p, w.p, mu_s, solve_tol, maxit, s2);
    if (rc != TMG_OK && rc != TMG_ERR_NOCONV) throw Error{rc, "sigma_min: inner solve failed"};
    nsolve += 2;
    double are, aim;
    blas_dot(c, vec(j), w.p, TMG_PREC_F64, n, &are, &aim);
    alpha.push_back(are);
    // full reorthogonalisation (twice) against v_0 .. v_j
    for (int pass = 0; pass < 2; pass++)
      for (int i = 0; i <= j; i++) {
        double hr, hi;
        blas_dot(c, vec(i), w.p, TMG_PREC_F64, n, &hr, &hi);
        blas_axpy(c, -hr, -hi, vec(i), w.p, TMG_PREC_F64, n);
      }
    const double b = std::sqrt(blas_norm2(c, w.p, TMG_PREC_F64, n));
    // Ritz values of the (j+1) x (j+1) tridiagonal
    const int m = j + 1;
    std::vector<double> T((size_t)m * m, 0.0), Z;
    for (int i = 0; i < m; i++) {
      T[(size_t)i * m + i] = alpha[i];
      if (i + 1 < m) T[(size_t)i * m + i + 1] = T[(size_t)(i + 1) * m + i] = beta[i];
    }
    jacobi_eig(T, Z, m);
    int imax = 0;
    for (int i = 1; i < m; i++)
      if (T[(size_t)i * m + i] > T[(size_t)imax * m + imax]) imax = i;
    theta = T[(size_t)imax * m + imax];
    res = theta > 0.0 ? b * std::fabs(Z[(size_t)(m - 1) * m + imax]) / theta : 1.0;
    if (res <= rtol || !(b > 0.0) || j + 1 == k) {
      j++;
      break;
    }
    beta.push_back(b);
    blas_copy(c, w.p, vec(j + 1), TMG_PREC_F64, n);
    blas_scale(c, 1.0 / b, 0.0, vec(j + 1), TMG_PREC_F64, n);
  }
  if (ritz_res) *ritz_res = res;
  if (solves) *solves = nsolve;
  if (steps_out) *steps_out = j;
  const double s2 = 1.0 / theta - mu_s * mu_s;
  return s2 > 0.0 ? std::sqrt(s2) : 0.0;
}

// ---------------------------------------------------------------- batched cycle (and its graph)
// z = M v for ncol FP32 columns: P^dag, the batched coarse solve (three levels: the lock-step
// K-cycle, or one K-cycle per column where the tensor-core apply does not cover the level shapes),
// P, SAP; one launch per operation for every column.
static void batched_cycle_p(Ctx& c, int pf, int ncol, const void* v, void* z, void* cr, void* ce, const float* mu_dev,
                            const double* mu) {
  restrict_mrhs(c, ncol, v, cr);
  if (c.l2_ready && kcycle_batched_ok(c, ncol)) {
    kcycle_batched(c, ncol, cr, ce, mu_dev, 0);
  } else if (c.l2_ready) {
    const size_t nco = (size_t)c.cl.nc * c.cl.nd;
    for (int col = 0; col < ncol; col++)
      kcycle(c, TMG_PREC_F32, (const float2*)cr + col * nco, (float2*)ce + col * nco, mu[col], 0);
  } else if (c.batched_tc && coarse_gmres_batched_tc_ok(c, ncol)) {
    coarse_gmres_batched_tc(c, ncol, cr, ce, mu_dev);
  } else {
    coarse_gmres_batched(c, ncol, cr, ce, mu_dev);
  }
  prolong_mrhs(c, ncol, ce, z);
  sap_mrhs(c, pf, ncol, z, v, mu_dev, c.mg.sap_sweeps);
}

// The batched cycle replayed as a CUDA graph, captured once per key like the single-column cycle:
// buffer addresses, column count, twists baked into host-side launches, parameters and knobs.
static void batched_cycle_run(Ctx& c, int pf, int ncol, const void* v, void* z, void* cr, void* ce, const float* mu_dev,
                              const double* mu) {
  if (!c.cycle_graphs || c.prof.on) {
    batched_cycle_p(c, pf, ncol, v, z, cr, ce, mu_dev, mu);
    return;
  }
  auto keyf = [&]() {
    std::vector<unsigned long long> k = cycle_key(c, pf, c.mg.prec_coarse, v, z, 0.0, 1);
    auto u = [](const void* p) { return (unsigned long long)(uintptr_t)p; };
    k.push_back(0xBA7C4ull);
    k.push_back((unsigned long long)ncol);
    k.push_back((unsigned long long)c.batched_tc);
    k.push_back((unsigned long long)c.batched_coarse_m);
    k.push_back(u(cr));
    k.push_back(u(ce));
    k.push_back(u(mu_dev));
    if (c.l2_ready)
      for (int col = 0; col < ncol; col++) {
        unsigned long long b;
        memcpy(&b, &mu[col], sizeof b);
        k.push_back(b);
      }
    return k;
  };
  std::vector<unsigned long long> key = keyf();
  for (auto& e : c.graphs.g)
    if (e.key == key) {
      TMG_CUDA(cudaGraphLaunch(e.exec, c.stream));
      c.launches += e.kernels;
      return;
    }
  batched_cycle_p(c, pf, ncol, v, z, cr, ce, mu_dev, mu);
  if (keyf() != key) return;
  if (!c.graphs.cap) TMG_CUDA(cudaStreamCreateWithFlags(&c.graphs.cap, cudaStreamNonBlocking));
  if (c.graphs.g.size() >= 64) c.graphs.clear();
  cudaStream_t saved = c.stream;
  const long long l0 = c.launches;
  cudaGraph_t graph = nullptr;
  c.stream = c.graphs.cap;
  cudaError_t err = cudaStreamBeginCapture(c.graphs.cap, cudaStreamCaptureModeRelaxed);
  if (err == cudaSuccess) {
    try {
      batched_cycle_p(c, pf, ncol, v, z, cr, ce, mu_dev, mu);
    } catch (const Error&) {
      err = cudaErrorStreamCaptureInvalidated;
    }
    const cudaError_t e2 = cudaStreamEndCapture(c.graphs.cap, &graph);
    if (err == cudaSuccess) err = e2;
  }
  c.stream = saved;
  const long long kernels = c.launches - l0;
  c.launches = l0;
  cudaGraphExec_t exec = nullptr;
  if (err == cudaSuccess && graph) err = cudaGraphInstantiate(&exec, graph, 0);
  if (graph) cudaGraphDestroy(graph);
  if (err != cudaSuccess || !exec) {
    cudaGetLastError();
    c.cycle_graphs = 0;
    return;
  }
  c.graphs.g.push_back(CycleGraph{key, exec, kernels});
}

// ---------------------------------------------------------------- batched mixed-precision solve
// All columns advance in lock-step: one launch per operation for every column (multi-column
// dslash, SAP, P, P^dag, and the batched coarse GMRES), per-column FGMRES recurrences on the host.
// The FP64 defect correction recomputes every column's true residual at each restart; columns
// that have converged keep a zero correction.
int solve_batched(Ctx& c, int ncol, const void* b64, void* x64, const double* mu, double tol, int maxiter,
                  SolveStats& st) {
  const size_t n = (size_t)12 * c.g.V;
  const int m = std::min(c.mg.restart, MAXM);
  const int pf = c.mg.prec_fine == TMG_PREC_F64 ? TMG_PREC_F32 : c.mg.prec_fine;
  const size_t nco = (size_t)c.cl.nc * c.cl.nd;
  const int rg = red_grid(c, n);
  // workspaces kept in the context: a repeated batched solve allocates nothing
  BatchWork& bw = c.bw;
  DBuf &r64 = bw.r64, &rin = bw.rin, &e = bw.e, &V = bw.V, &Z = bw.Z, &w = bw.w, &cr = bw.cr, &ce = bw.ce,
       &mu_dev = bw.mu, &part = bw.part, &hdev = bw.h, &npart = bw.npart, &inv_dev = bw.inv;
  inv_dev.alloc(ncol * sizeof(double));
  r64.alloc(ncol * n * 16);
  rin.alloc(ncol * n * 8);
  e.alloc(ncol * n * 8);
  V.alloc((size_t)(m + 1) * ncol * n * 8);
  Z.alloc((size_t)m * ncol * n * 8);
  w.alloc(ncol * n * 8);
  cr.alloc(ncol * nco * 8);
  ce.alloc(ncol * nco * 8);
  mu_dev.alloc(ncol * sizeof(float));
  part.alloc(sizeof(double2) * (size_t)ncol * (MAXM + 1) * NPART);
  hdev.alloc(sizeof(double2) * (size_t)2 * ncol * (MAXM + 1));
  npart.alloc(sizeof(double) * (size_t)ncol * NPART);
  std::vector<float> muf(ncol);
  for (int j = 0; j < ncol; j++) muf[j] = (float)mu[j];
  TMG_CUDA(cudaMemcpyAsync(mu_dev.p, muf.data(), ncol * sizeof(float), cudaMemcpyHostToDevice, c.stream));
  int c0 = 0, c1 = 0;
  if (c.coarse_iter_dev.p) TMG_CUDA(cudaMemcpyAsync(&c0, c.coarse_iter_dev.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  if (c.tc_err.p) TMG_CUDA(cudaMemsetAsync(c.tc_err.p, 0, sizeof(int), c.stream));
  std::vector<double> bn(ncol), rn(ncol);
  for (int j = 0; j < ncol; j++) {
    const char* bj = (const char*)b64 + j * n * 16;
    blas_zero(c, (char*)x64 + j * n * 16, TMG_PREC_F64, n);
    blas_copy(c, bj, r64.as<char>() + j * n * 16, TMG_PREC_F64, n);
    bn[j] = std::sqrt(blas_norm2(c, bj, TMG_PREC_F64, n));
    if (!std::isfinite(bn[j])) throw Error{TMG_ERR_BREAKDOWN, "batched solve: right-hand side is not finite"};
  }
  float2* Vp = V.as<float2>();
  float2* Zp = Z.as<float2>();
  const size_t istride = (size_t)ncol * n;
  int rc = TMG_OK;
  while (true) {
    bool all = true;
    double worst = 0.0;
    for (int j = 0; j < ncol; j++) {
      rn[j] = std::sqrt(blas_norm2(c, r64.as<char>() + j * n * 16, TMG_PREC_F64, n));
      if (!std::isfinite(rn[j])) throw Error{TMG_ERR_BREAKDOWN, "batched solve: residual is not finite"};
      const double rel = bn[j] > 0.0 ? rn[j] / bn[j] : 0.0;
      worst = std::max(worst, rel);
      if (rel > tol) all = false;
    }
    st.true_residual = worst;
    if (all) break;
    if (st.iterations >= maxiter) {
      rc = TMG_ERR_NOCONV;
      break;
    }
    // unit-norm FP32 residuals of the unconverged columns (converged ones: zero)
    for (int j = 0; j < ncol; j++) {
      char* rj = rin.as<char>() + j * n * 8;
      if (bn[j] > 0.0 && rn[j] > tol * bn[j]) {
        convert_field(c, r64.as<char>() + j * n * 16, TMG_PREC_F64, rj, TMG_PREC_F32, n);
        blas_scale(c, 1.0 / rn[j], 0.0, rj, TMG_PREC_F32, n);
      } else {
        blas_zero(c, rj, TMG_PREC_F32, n);
      }
    }
    // FGMRES(m) cycle on all columns; beta = 1 (or 0) per column
    std::vector<double> beta(ncol), target(ncol);
    for (int j = 0; j < ncol; j++) {
      const bool act = bn[j] > 0.0 && rn[j] > tol * bn[j];
      beta[j] = act ? 1.0 : 0.0;
      target[j] = act ? std::max(tol * bn[j] / rn[j], 1e-6) : 1.0;
    }
    blas_copy(c, rin.p, Vp, TMG_PREC_F32, ncol * n);
    std::vector<std::complex<double>> H((size_t)ncol * (m + 1) * m), cs((size_t)ncol * m), sn((size_t)ncol * m),
        g((size_t)ncol * (m + 1)), y((size_t)ncol * m);
    for (int j = 0; j < ncol; j++) g[(size_t)j * (m + 1)] = beta[j];
    std::vector<char> done(ncol);
    for (int j = 0; j < ncol; j++) done[j] = beta[j] == 0.0;
    int k = 0;
    for (int it = 0; it < m; it++) {
      float2* vj = Vp + (size_t)it * istride;
      float2* zj = Zp + (size_t)it * istride;
      // z = M v (one batched cycle, replayed as a graph)
      batched_cycle_run(c, pf, ncol, vj, zj, cr.p, ce.p, mu_dev.as<float>(), mu);
      dslash_mrhs(c, pf, ncol, w.p, zj, nullptr, mu_dev.as<float>(), 0);
      const int npass = c.outer_gs_passes == 1 ? 1 : 2;   // classical Gram-Schmidt passes
      for (int pass = 0; pass < npass; pass++) {
        ++c.launches, k_mdot_partial_b<<<dim3(rg, it + 1, ncol), 256, 0, c.stream>>>(Vp, istride, w.as<float2>(), n, part.as<double2>());
        ++c.launches, k_mdot_final_b<<<dim3(it + 1, ncol), 256, 0, c.stream>>>(part.as<double2>(), rg,
                                                                               hdev.as<double2>() + (size_t)pass * ncol * (MAXM + 1));
        ++c.launches, k_mgs_update_b<<<dim3(rg, ncol), 256, 0, c.stream>>>(Vp, istride, it + 1,
                                                                            hdev.as<double2>() + (size_t)pass * ncol * (MAXM + 1),
                                                                            w.as<float2>(), n, pass == npass - 1 ? npart.as<double>() : nullptr);
        TMG_CHECK_LAUNCH();
      }
      std::vector<double2> hc((size_t)2 * ncol * (MAXM + 1), make_double2(0.0, 0.0));
      std::vector<double> nn((size_t)ncol * NPART);
      TMG_CUDA(cudaMemcpyAsync(hc.data(), hdev.p, sizeof(double2) * (size_t)npass * ncol * (MAXM + 1), cudaMemcpyDeviceToHost,
                               c.stream));
      TMG_CUDA(cudaMemcpyAsync(nn.data(), npart.p, sizeof(double) * nn.size(), cudaMemcpyDeviceToHost, c.stream));
      TMG_CUDA(cudaStreamSynchronize(c.stream));
      k = it + 1;
      bool all_done = true;
      std::vector<double> inv(ncol, 0.0);
      for (int j = 0; j < ncol; j++) {
        double s2 = 0.0;
        for (int q = 0; q < rg; q++) s2 += nn[(size_t)j * NPART + q];
        const double hn = std::sqrt(s2);
        std::complex<double>* h = &H[((size_t)j * m + it) * (m + 1)];
        for (int i = 0; i <= it; i++) {
          const double2 a1 = hc[(size_t)j * (MAXM + 1) + i], a2 = hc[(size_t)ncol * (MAXM + 1) + (size_t)j * (MAXM + 1) + i];
          h[i] = std::complex<double>(a1.x + a2.x, a1.y + a2.y);
        }
        h[it + 1] = hn;
        std::complex<double>* csj = &cs[(size_t)j * m];
        std::complex<double>* snj = &sn[(size_t)j * m];
        std::complex<double>* gj = &g[(size_t)j * (m + 1)];
        for (int i = 0; i < it; i++) {
          const std::complex<double> a = h[i], bb = h[i + 1];
          h[i] = std::conj(csj[i]) * a + std::conj(snj[i]) * bb;
          h[i + 1] = -snj[i] * a + csj[i] * bb;
        }
        const std::complex<double> a = h[it], bb = h[it + 1];
        const double den = std::sqrt(std::norm(a) + std::norm(bb));
        csj[it] = den > 0 ? a / den : 1.0;
        snj[it] = den > 0 ? bb / den : 0.0;
        h[it] = den;
        h[it + 1] = 0.0;
        gj[it + 1] = -snj[it] * gj[it];
        gj[it] = std::conj(csj[it]) * gj[it];
        if (!done[j] && (std::abs(gj[it + 1]) <= target[j] * beta[j] || hn == 0.0)) done[j] = 1;
        all_done = all_done && done[j];
        inv[j] = hn > 0.0 ? 1.0 / hn : 0.0;
      }
      if (all_done || it == m - 1) break;
      // v_{it+1} = w / h_{it+1,it} for every column in one launch
      float2* vn = Vp + (size_t)(it + 1) * istride;
      TMG_CUDA(cudaMemcpyAsync(inv_dev.p, inv.data(), ncol * sizeof(double), cudaMemcpyHostToDevice, c.stream));
      ++c.launches, k_scale_cols<<<dim3(egrid(c, n), ncol), 256, 0, c.stream>>>(w.as<float2>(), vn, inv_dev.as<double>(), n);
      TMG_CHECK_LAUNCH();
    }
    // per-column back substitution (only over the steps each column has: all columns used k steps)
    std::vector<double2> yc((size_t)ncol * (MAXM + 1));
    for (int j = 0; j < ncol; j++) {
      std::complex<double>* yj = &y[(size_t)j * m];
      const std::complex<double>* gj = &g[(size_t)j * (m + 1)];
      for (int i = k - 1; i >= 0; i--) {
        std::complex<double> acc = gj[i];
        for (int l = i + 1; l < k; l++) acc -= H[((size_t)j * m + l) * (m + 1) + i] * yj[l];
        const std::complex<double> d = H[((size_t)j * m + i) * (m + 1) + i];
        yj[i] = std::abs(d) > 0.0 ? acc / d : 0.0;
        yc[(size_t)j * (MAXM + 1) + i] = make_double2(yj[i].real(), yj[i].imag());
      }
    }
    TMG_CUDA(cudaMemcpyAsync(hdev.p, yc.data(), sizeof(double2) * yc.size(), cudaMemcpyHostToDevice, c.stream));
    ++c.launches, k_combine_b<<<dim3(egrid(c, n), ncol), 256, 0, c.stream>>>(Zp, istride, k, hdev.as<double2>(), e.as<float2>(), n);
    TMG_CHECK_LAUNCH();
    st.iterations += k;
    st.refinements++;
    for (int j = 0; j < ncol; j++) {
      if (beta[j] == 0.0) continue;
      char* xj = (char*)x64 + j * n * 16;
      blas_axpy_mixed(c, rn[j], e.as<char>() + j * n * 8, TMG_PREC_F32, xj, TMG_PREC_F64, n);
      dslash(c, TMG_PREC_F64, r64.as<char>() + j * n * 16, xj, (const char*)b64 + j * n * 16, mu[j], 1, 0);
    }
  }
  if (c.coarse_iter_dev.p) {
    TMG_CUDA(cudaMemcpyAsync(&c1, c.coarse_iter_dev.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    st.coarse_iterations = c1 - c0;
  }
  if (c.tc_err.p) {
    int herr = 0;
    TMG_CUDA(cudaMemcpyAsync(&herr, c.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    if (herr) throw Error{TMG_ERR_TIMEOUT, "batched solve: a tensor-core completion wait gave up"};
  }
  return rc;
}

}  // namespace tmg
