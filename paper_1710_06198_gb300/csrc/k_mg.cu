// Multigrid kernels of the DD-alpha-AMG preconditioner (Eq. 1 of arXiv:1710.06198):
//   - SAP smoother M: one CTA per lattice block of one colour; residual, block MR solve on the
//     Dirichlet block operator in shared memory, update (Sec. 1.1, Schwarz alternating procedure);
//   - restriction P^dag and prolongation P over aggregates (= blocks), Gamma5-compatible: test
//     vectors are split into chirality halves (G5 P = P G5_c);
//   - coarse operator D_c = P^dag D P as a 9-point stencil (setup), and its application with the
//     twist i mu G5_c added on the fly (D_c(mu) = D_c + i mu G5_c);
//   - per-aggregate, per-chirality Gram-Schmidt of the test vectors in FP64.
#include <algorithm>
#include <vector>

#include "dslash_core.cuh"
#include "tmg_host.h"

namespace tmg {

// Reduction of N values (per thread) over the CTA; every thread gets the totals.  Warp sums use
// shuffles and the cross-warp sum (one thread per value) runs in the kernel's precision R: the
// FP32 kernels use no FP64 arithmetic, which GB300 issues at a small fraction of the FP32 rate.
// red: shared scratch of at least 33 * N doubles.
template <int N, typename R>
__device__ __forceinline__ void cta_allreduce(R (&v)[N], double* red_d) {
  R* red = reinterpret_cast<R*>(red_d);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < N; i++) {
    R a = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[w * N + i] = a;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    R a = 0;
    for (int k = 0; k < nw; k++) a += red[k * N + i];
    red[32 * N + i] = a;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; i++) v[i] = red[32 * N + i];
  __syncthreads();
}

// One-barrier variant for the block solvers (at most 8 warps): the warp sums go to half `parity`
// of the scratch (8 N values of R each) and, after one barrier, every thread adds the warps' values
// itself.  Consecutive calls alternate the parity; any two calls with the same parity must be
// separated by another CTA barrier of the caller (the block solvers have one before each MR step's
// operator), so no warp overwrites a half that another is still reading.
template <int N, typename R>
__device__ __forceinline__ void cta_allreduce_db(R (&v)[N], double* red_d, int parity) {
  R* red = reinterpret_cast<R*>(red_d) + parity * 8 * N;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < N; i++) {
    R a = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[w * N + i] = a;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; i++) {
    R a = 0;
    for (int k = 0; k < nw; k++) a += red[k * N + i];
    v[i] = a;
  }
}

// k-th block of the given colour (colour = parity of the block coordinates; NB[0] is even).
__device__ __forceinline__ int colour_block(const Geom& g, int colour, int k) {
  const int half = g.NB[0] >> 1;
  const int row = k / half, j = k - row * half;
  const int b1 = row % g.NB[1], r2 = row / g.NB[1];
  const int b2 = r2 % g.NB[2], b3 = r2 / g.NB[2];
  const int b0 = 2 * j + ((colour + b1 + b2 + b3) & 1);
  return row * g.NB[0] + b0;
}

// ------------------------------------------------------------------ SAP
// For every block of one colour: r = b - D x on the block (neighbours from global x), then n_mr
// minimal-residual steps e += a r, r -= a D_B r with the Dirichlet block operator D_B (hops that
// leave the block are dropped), then x += e.  Blocks of one colour never touch, so the CTAs of a
// launch are independent; the other colour's x is only read.
// Multi-column form (MC): CTA (block, column) = (blockIdx.x / ncol, blockIdx.x % ncol),
// column c of x and b with twist mu_col[c]; the columns of a block run on neighbouring CTAs, so
// its links and clover come from DRAM about once per launch.
template <typename R, class S, class G, class C, bool MC = false>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 2 : 1) k_sap_block(Geom g, int colour, S x, S b, G U, C A, R tw, int n_mr,
                                                                           int ncol, const float* __restrict__ mu_col) {
  // shared memory: r [12][VB] complex; for FP32 arithmetic also the block's links, reconstructed
  // once to 18 reals, [4][9][VB] complex (the MR steps then never touch global memory for links)
  extern __shared__ double smem_d[];
  cpx<R>* rs = reinterpret_cast<cpx<R>*>(smem_d);
  constexpr bool kCacheLinks = sizeof(R) == 4;
  cpx<R>* ls = rs + 12 * g.VB;
  double* red = smem_d + (sizeof(cpx<R>) * (kCacheLinks ? 48 : 12) * g.VB) / sizeof(double);
  int kblk = blockIdx.x;
  if constexpr (MC) {
    const int col = blockIdx.x % ncol;
    kblk = blockIdx.x / ncol;
    x = x.column(col);
    b = b.column(col);
    tw = (R)mu_col[col];
  }
  const int blk = colour_block(g, colour, kblk);
  const int t = threadIdx.x;
  const int s = blk * g.VB + t;
  const SiteCoord sc = decode_site(g, s);
  if (kCacheLinks) {
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      Link<R> u;
      U.load(s, mu, u);
#pragma unroll
      for (int k = 0; k < 9; k++) ls[(mu * 9 + k) * g.VB + t] = u.m[k];
    }
  }
  Spinor<R> r;
  {
    Spinor<R> dx, bs;
    apply_D_site<R>(g, sc, s, x, U, A, tw, dx);
    b.load(s, bs);
#pragma unroll
    for (int k = 0; k < 12; k++) r.c[k] = bs.c[k] - dx.c[k];
  }
  Spinor<R> e;
#pragma unroll
  for (int k = 0; k < 12; k++) e.c[k] = mk<R>(0, 0);
  for (int it = 0; it < n_mr; it++) {
#pragma unroll
    for (int k = 0; k < 12; k++) rs[k * g.VB + t] = r.c[k];
    __syncthreads();
    // p = D_B r
    Spinor<R> acc;
#pragma unroll
    for (int k = 0; k < 12; k++) acc.c[k] = mk<R>(0, 0);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      if (sc.l[mu] + 1 < g.B[mu]) {
        const int tf = t + g.ls[mu];
        Spinor<R> p;
#pragma unroll
        for (int k = 0; k < 12; k++) p.c[k] = rs[k * g.VB + tf];
        cpx<R> h[6], uh[6];
        spin_project(mu, +1, p, h);
        Link<R> u;
        if (kCacheLinks) {
#pragma unroll
          for (int k = 0; k < 9; k++) u.m[k] = ls[(mu * 9 + k) * g.VB + t];
        } else {
          U.load(s, mu, u);
        }
        su3_mul_half(u, false, h, uh);
        spin_reconstruct_add(mu, +1, uh, acc);
      }
      if (sc.l[mu] > 0) {
        const int tb = t - g.ls[mu];
        Spinor<R> p;
#pragma unroll
        for (int k = 0; k < 12; k++) p.c[k] = rs[k * g.VB + tb];
        cpx<R> h[6], uh[6];
        spin_project(mu, -1, p, h);
        Link<R> u;
        if (kCacheLinks) {
#pragma unroll
          for (int k = 0; k < 9; k++) u.m[k] = ls[(mu * 9 + k) * g.VB + tb];
        } else {
          U.load(s - g.ls[mu], mu, u);
        }
        su3_mul_half(u, true, h, uh);
        spin_reconstruct_add(mu, -1, uh, acc);
      }
    }
    Spinor<R> p;
#pragma unroll
    for (int chi = 0; chi < 2; chi++) {
      CloverBlock<R> a;
      A.load(s, chi, a);
      clover_mul(a, chi == 0 ? tw : -tw, &r.c[6 * chi], &p.c[6 * chi]);
    }
#pragma unroll
    for (int k = 0; k < 12; k++) p.c[k] = p.c[k] - R(0.5) * acc.c[k];
    R v[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 12; k++) {
      v[0] += p.c[k].re * p.c[k].re + p.c[k].im * p.c[k].im;
      const cpx<R> q = cmul_conj(p.c[k], r.c[k]);
      v[1] += q.re;
      v[2] += q.im;
    }
    cta_allreduce_db<3, R>(v, red, it & 1);
    const cpx<R> alpha = v[0] > R(0) ? mk(v[1] / v[0], v[2] / v[0]) : mk<R>(0, 0);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      e.c[k] = e.c[k] + alpha * r.c[k];
      r.c[k] = r.c[k] - alpha * p.c[k];
    }
  }
  Spinor<R> xs;
  x.load(s, xs);
#pragma unroll
  for (int k = 0; k < 12; k++) xs.c[k] = xs.c[k] + e.c[k];
  x.store(s, xs);
}

// SAP on the non-degenerate doublet (Eq. 2): the same colouring and block MR, on flavour pairs.
// The block operator is [[D_B(mubar), -epsbar], [-epsbar, D_B(-mubar)]] (the flavour mixing is
// site-local; the shifted doublet adds i delta g5 to it); MR step lengths come from inner products
// over both flavours.
template <typename R, class S, class G, class C>
__global__ void __launch_bounds__(256, 1) k_sap_block_nd(Geom g, int colour, S xu, S xd, S bu, S bd, G U, C A, R mubar,
                                                         R epsbar, R delta, int n_mr) {
  // shared memory: r [2][12][VB] complex; for FP32 arithmetic also the block's links [4][9][VB]
  extern __shared__ double smem_d[];
  cpx<R>* rs = reinterpret_cast<cpx<R>*>(smem_d);
  constexpr bool kCacheLinks = sizeof(R) == 4;
  cpx<R>* ls = rs + 24 * g.VB;
  double* red = smem_d + (sizeof(cpx<R>) * (kCacheLinks ? 60 : 24) * g.VB) / sizeof(double);
  const int blk = colour_block(g, colour, blockIdx.x);
  const int t = threadIdx.x;
  const int s = blk * g.VB + t;
  const SiteCoord sc = decode_site(g, s);
  if (kCacheLinks) {
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      Link<R> u;
      U.load(s, mu, u);
#pragma unroll
      for (int k = 0; k < 9; k++) ls[(mu * 9 + k) * g.VB + t] = u.m[k];
    }
  }
  Spinor<R> r[2];
  {
    Spinor<R> du, dd, xs_u, xs_d, bs;
    apply_D_site<R>(g, sc, s, xu, U, A, mubar, du);
    apply_D_site<R>(g, sc, s, xd, U, A, -mubar, dd);
    xu.load(s, xs_u);
    xd.load(s, xs_d);
    bu.load(s, bs);
#pragma unroll
    for (int k = 0; k < 12; k++) r[0].c[k] = bs.c[k] - (du.c[k] + nd_mix(epsbar, delta, k, xs_d.c[k]));
    bd.load(s, bs);
#pragma unroll
    for (int k = 0; k < 12; k++) r[1].c[k] = bs.c[k] - (dd.c[k] + nd_mix(epsbar, delta, k, xs_u.c[k]));
  }
  Spinor<R> e[2];
#pragma unroll
  for (int f = 0; f < 2; f++)
#pragma unroll
    for (int k = 0; k < 12; k++) e[f].c[k] = mk<R>(0, 0);
  for (int it = 0; it < n_mr; it++) {
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
      for (int k = 0; k < 12; k++) rs[(f * 12 + k) * g.VB + t] = r[f].c[k];
    __syncthreads();
    Spinor<R> acc[2];
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
      for (int k = 0; k < 12; k++) acc[f].c[k] = mk<R>(0, 0);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      if (sc.l[mu] + 1 < g.B[mu]) {
        const int tf = t + g.ls[mu];
        Link<R> u;
        if (kCacheLinks) {
#pragma unroll
          for (int k = 0; k < 9; k++) u.m[k] = ls[(mu * 9 + k) * g.VB + t];
        } else {
          U.load(s, mu, u);
        }
#pragma unroll
        for (int f = 0; f < 2; f++) {
          Spinor<R> p;
#pragma unroll
          for (int k = 0; k < 12; k++) p.c[k] = rs[(f * 12 + k) * g.VB + tf];
          cpx<R> h[6], uh[6];
          spin_project(mu, +1, p, h);
          su3_mul_half(u, false, h, uh);
          spin_reconstruct_add(mu, +1, uh, acc[f]);
        }
      }
      if (sc.l[mu] > 0) {
        const int tb = t - g.ls[mu];
        Link<R> u;
        if (kCacheLinks) {
#pragma unroll
          for (int k = 0; k < 9; k++) u.m[k] = ls[(mu * 9 + k) * g.VB + tb];
        } else {
          U.load(s - g.ls[mu], mu, u);
        }
#pragma unroll
        for (int f = 0; f < 2; f++) {
          Spinor<R> p;
#pragma unroll
          for (int k = 0; k < 12; k++) p.c[k] = rs[(f * 12 + k) * g.VB + tb];
          cpx<R> h[6], uh[6];
          spin_project(mu, -1, p, h);
          su3_mul_half(u, true, h, uh);
          spin_reconstruct_add(mu, -1, uh, acc[f]);
        }
      }
    }
    Spinor<R> q[2];
#pragma unroll
    for (int chi = 0; chi < 2; chi++) {
      CloverBlock<R> a;
      A.load(s, chi, a);
      clover_mul(a, chi == 0 ? mubar : -mubar, &r[0].c[6 * chi], &q[0].c[6 * chi]);
      clover_mul(a, chi == 0 ? -mubar : mubar, &r[1].c[6 * chi], &q[1].c[6 * chi]);
    }
#pragma unroll
    for (int k = 0; k < 12; k++) {
      const cpx<R> q0 = q[0].c[k] - R(0.5) * acc[0].c[k] + nd_mix(epsbar, delta, k, r[1].c[k]);
      const cpx<R> q1 = q[1].c[k] - R(0.5) * acc[1].c[k] + nd_mix(epsbar, delta, k, r[0].c[k]);
      q[0].c[k] = q0;
      q[1].c[k] = q1;
    }
    R v[3] = {0, 0, 0};
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
      for (int k = 0; k < 12; k++) {
        v[0] += q[f].c[k].re * q[f].c[k].re + q[f].c[k].im * q[f].c[k].im;
        const cpx<R> w = cmul_conj(q[f].c[k], r[f].c[k]);
        v[1] += w.re;
        v[2] += w.im;
      }
    cta_allreduce_db<3, R>(v, red, it & 1);
    const cpx<R> alpha = v[0] > R(0) ? mk(v[1] / v[0], v[2] / v[0]) : mk<R>(0, 0);
#pragma unroll
    for (int f = 0; f < 2; f++)
#pragma unroll
      for (int k = 0; k < 12; k++) {
        e[f].c[k] = e[f].c[k] + alpha * r[f].c[k];
        r[f].c[k] = r[f].c[k] - alpha * q[f].c[k];
      }
  }
  Spinor<R> xs;
  xu.load(s, xs);
#pragma unroll
  for (int k = 0; k < 12; k++) xs.c[k] = xs.c[k] + e[0].c[k];
  xu.store(s, xs);
  xd.load(s, xs);
#pragma unroll
  for (int k = 0; k < 12; k++) xs.c[k] = xs.c[k] + e[1].c[k];
  xd.store(s, xs);
}

template <typename R, class S, class G, class C>
static void launch_sap_nd(Ctx& c, S xu, S xd, S bu, S bd, G U, C A, R mubar, R epsbar, R delta, int n_sweeps, int kind) {
  const size_t smem = sizeof(cpx<R>) * (sizeof(R) == 4 ? 60 : 24) * c.g.VB + 33 * 3 * sizeof(double);
  if (smem > 48 * 1024)
    TMG_CUDA(cudaFuncSetAttribute(k_sap_block_nd<R, S, G, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  for (int sw = 0; sw < n_sweeps; sw++)
    for (int colour = 0; colour < 2; colour++) {
      ProfScope ps(c, kind);
      ++c.launches, k_sap_block_nd<R, S, G, C><<<c.g.nblk / 2, c.g.VB, smem, c.stream>>>(c.g, colour, xu, xd, bu, bd, U, A, mubar,
                                                                                     epsbar, delta, c.mg.sap_mr);
      TMG_CHECK_LAUNCH();
    }
}

void sap_sweeps_nd(Ctx& c, int prec, void* x, const void* b, int n_sweeps) {
  const size_t col = (size_t)12 * c.g.V;
  if (prec == TMG_PREC_F64) {
    double2* xp = (double2*)x;
    double2* bp = (double2*)b;
    launch_sap_nd<double>(c, SpinorF64{xp, c.g.V}, SpinorF64{xp + col, c.g.V}, SpinorF64{bp, c.g.V}, SpinorF64{bp + col, c.g.V},
                          GaugeF64{c.op[0].U.as<double2>(), c.g.V}, CloverF64{c.op[0].A.as<double2>(), c.g.V}, c.mubar, c.epsbar,
                          c.ndshift, n_sweeps, PK_SAP_F64);
  } else {
    float4* xp = (float4*)x;
    float4* bp = (float4*)b;
    const size_t col4 = col / 2;   // float4 per flavour column
    if (prec == TMG_PREC_F32)
      launch_sap_nd<float>(c, SpinorF32{xp, c.g.V}, SpinorF32{xp + col4, c.g.V}, SpinorF32{bp, c.g.V}, SpinorF32{bp + col4, c.g.V},
                           GaugeF32{c.op[1].U.as<float4>(), c.g.V}, CloverF32{c.op[1].A.as<float4>(), c.g.V}, (float)c.mubar,
                           (float)c.epsbar, (float)c.ndshift, n_sweeps, PK_SAP_F32);
    else
      launch_sap_nd<float>(c, SpinorF32{xp, c.g.V}, SpinorF32{xp + col4, c.g.V}, SpinorF32{bp, c.g.V}, SpinorF32{bp + col4, c.g.V},
                           GaugeF16{c.op[2].U.as<short4>(), c.g.V},
                           CloverF16{c.op[2].A.as<short4>(), c.op[2].Ascale.as<float>(), c.g.V}, (float)c.mubar,
                           (float)c.epsbar, (float)c.ndshift, n_sweeps, PK_SAP_F16);
  }
}

template <typename R, class S, class G, class C>
static void launch_sap(Ctx& c, S x, S b, G U, C A, R tw, int n_sweeps, int kind) {
  const size_t smem = sizeof(cpx<R>) * (sizeof(R) == 4 ? 48 : 12) * c.g.VB + 33 * 3 * sizeof(double);
  if (smem > 48 * 1024) {
    TMG_CUDA(cudaFuncSetAttribute(k_sap_block<R, S, G, C>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  }
  for (int sw = 0; sw < n_sweeps; sw++)
    for (int colour = 0; colour < 2; colour++) {
      ProfScope ps(c, kind);
      ++c.launches, k_sap_block<R, S, G, C><<<c.g.nblk / 2, c.g.VB, smem, c.stream>>>(c.g, colour, x, b, U, A, tw, c.mg.sap_mr,
                                                                                   1, nullptr);
      TMG_CHECK_LAUNCH();
    }
}

// The same sweeps for ncol FP32 columns [col][12 V] (column c with twist mu_col_dev[c]), one launch
// per colour for all columns.
template <class G, class C>
static void launch_sap_mrhs(Ctx& c, int ncol, float4* x, const float4* b, G U, C A, const float* mu_col_dev, int n_sweeps,
                            int kind) {
  using S = SpinorF32;
  const size_t smem = sizeof(cpx<float>) * 48 * c.g.VB + 33 * 3 * sizeof(double);
  if (smem > 48 * 1024)
    TMG_CUDA(cudaFuncSetAttribute(k_sap_block<float, S, G, C, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const unsigned grid = (unsigned)(c.g.nblk / 2) * (unsigned)ncol;
  for (int sw = 0; sw < n_sweeps; sw++)
    for (int colour = 0; colour < 2; colour++) {
      ProfScope ps(c, kind);
      ++c.launches, k_sap_block<float, S, G, C, true><<<grid, c.g.VB, smem, c.stream>>>(c.g, colour, S{x, c.g.V}, S{(float4*)b, c.g.V},
                                                                                  U, A, 0.f, c.mg.sap_mr, ncol, mu_col_dev);
      TMG_CHECK_LAUNCH();
    }
}

void sap_mrhs(Ctx& c, int prec, int ncol, void* x, const void* b, const float* mu_col_dev, int n_sweeps) {
  if (prec == TMG_PREC_F16)
    launch_sap_mrhs(c, ncol, (float4*)x, (const float4*)b, GaugeF16{c.op[2].U.as<short4>(), c.g.V},
                    CloverF16{c.op[2].A.as<short4>(), c.op[2].Ascale.as<float>(), c.g.V}, mu_col_dev, n_sweeps, PK_SAP_F16);
  else
    launch_sap_mrhs(c, ncol, (float4*)x, (const float4*)b, GaugeF32{c.op[1].U.as<float4>(), c.g.V},
                    CloverF32{c.op[1].A.as<float4>(), c.g.V}, mu_col_dev, n_sweeps, PK_SAP_F32);
}

void sap_sweeps(Ctx& c, int prec, void* x, const void* b, void* /*r_scratch*/, double mu, int n_sweeps) {
  if (prec == TMG_PREC_F64)
    launch_sap<double>(c, SpinorF64{(double2*)x, c.g.V}, SpinorF64{(double2*)b, c.g.V},
                       GaugeF64{c.op[0].U.as<double2>(), c.g.V}, CloverF64{c.op[0].A.as<double2>(), c.g.V}, mu, n_sweeps, PK_SAP_F64);
  else if (prec == TMG_PREC_F32)
    launch_sap<float>(c, SpinorF32{(float4*)x, c.g.V}, SpinorF32{(float4*)b, c.g.V},
                      GaugeF32{c.op[1].U.as<float4>(), c.g.V}, CloverF32{c.op[1].A.as<float4>(), c.g.V}, (float)mu,
                      n_sweeps, PK_SAP_F32);
  else
    launch_sap<float>(c, SpinorF32{(float4*)x, c.g.V}, SpinorF32{(float4*)b, c.g.V},
                      GaugeF16{c.op[2].U.as<short4>(), c.g.V},
                      CloverF16{c.op[2].A.as<short4>(), c.op[2].Ascale.as<float>(), c.g.V}, (float)mu, n_sweeps,
                      PK_SAP_F16);
}

// ------------------------------------------------------------------ restriction P^dag
// out[blk][chi * nv + j] = sum_{s in blk} W_j(s)_chi^dag r(s)_chi, test vectors handled in chunks of
// 8 to bound the registers.
// One round of a warp-wide multi-value reduction: of the 2 O values a lane still holds, it keeps
// the upper O if bit O of its lane index is set and the lower O otherwise, adding the partner's
// copy of the kept half.  After rounds O = 16, 8, 4, 2, 1 on 32 values, lane l holds in v[0] the
// warp sum of value l.
template <int O, typename R>
__device__ __forceinline__ void warp_transpose_reduce(R (&v)[32], int lane) {
  const bool upper = (lane & O) != 0;
#pragma unroll
  for (int i = 0; i < O; i++) {
    const R send = upper ? v[i] : v[i + O];
    const R keep = upper ? v[i + O] : v[i];
    v[i] = keep + __shfl_xor_sync(0xffffffffu, send, O);
  }
}

template <typename R, class S, typename OUT2>
__global__ void __launch_bounds__(256) k_restrict(Geom g, S r, S W, int nv, OUT2* __restrict__ out) {
  extern __shared__ double red[];
  const int blk = blockIdx.x;
  const int s = blk * g.VB + threadIdx.x;
  Spinor<R> rv;
  r.load(s, rv);
  const int nd = 2 * nv;
  for (int j0 = 0; j0 < nv; j0 += 8) {
    R v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = 0;
#pragma unroll
    for (int jj = 0; jj < 8; jj++) {
      const int j = j0 + jj;
      if (j < nv) {
        const S w = W.column(j);
        Spinor<R> wv;
        w.load(s, wv);
#pragma unroll
        for (int k = 0; k < 12; k++) {
          const cpx<R> q = cmul_conj(wv.c[k], rv.c[k]);
          const int chi = k / 6;
          v[(chi * 8 + jj) * 2] += q.re;
          v[(chi * 8 + jj) * 2 + 1] += q.im;
        }
      }
    }
    // warp sums by a butterfly in which every lane ends up holding the sum of one of the 32 values
    // (31 shuffles instead of 32 x 5), then one sum over the warps per value, in the kernel's
    // precision R (no FP64 arithmetic in the FP32 kernel)
    const int lane = threadIdx.x & 31, wp = threadIdx.x >> 5;
    warp_transpose_reduce<16>(v, lane);
    warp_transpose_reduce<8>(v, lane);
    warp_transpose_reduce<4>(v, lane);
    warp_transpose_reduce<2>(v, lane);
    warp_transpose_reduce<1>(v, lane);
    R* redr = reinterpret_cast<R*>(red);
    redr[wp * 32 + lane] = v[0];
    __syncthreads();
    if (threadIdx.x < 32) {
      R t = 0;
      for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += redr[k * 32 + threadIdx.x];
      redr[32 * 32 + threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x < 16) {
      const int chi = threadIdx.x / 8, jj = threadIdx.x % 8, j = j0 + jj;
      if (j < nv) {
        OUT2 o;
        o.x = redr[32 * 32 + (chi * 8 + jj) * 2];
        o.y = redr[32 * 32 + (chi * 8 + jj) * 2 + 1];
        out[(size_t)blk * nd + chi * nv + j] = o;
      }
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------ prolongation P
// e(s)_chi (+)= sum_j W_j(s)_chi c[blk][chi * nv + j]
template <typename R, class S, typename IN2>
__global__ void __launch_bounds__(256) k_prolong(Geom g, const IN2* __restrict__ cv, S W, int nv, S e, int accumulate) {
  extern __shared__ double smem_p[];
  cpx<R>* cs = reinterpret_cast<cpx<R>*>(smem_p);
  const int blk = blockIdx.x;
  const int nd = 2 * nv;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) {
    const IN2 v = cv[(size_t)blk * nd + i];
    cs[i] = mk<R>((R)v.x, (R)v.y);
  }
  __syncthreads();
  const int s = blk * g.VB + threadIdx.x;
  Spinor<R> out;
  if (accumulate) e.load(s, out);
  else {
#pragma unroll
    for (int k = 0; k < 12; k++) out.c[k] = mk<R>(0, 0);
  }
  for (int j = 0; j < nv; j++) {
    const S w = W.column(j);
    Spinor<R> wv;
    w.load(s, wv);
    const cpx<R> cp = cs[j], cm = cs[nv + j];
#pragma unroll
    for (int k = 0; k < 6; k++) out.c[k] = out.c[k] + wv.c[k] * cp;
#pragma unroll
    for (int k = 6; k < 12; k++) out.c[k] = out.c[k] + wv.c[k] * cm;
  }
  e.store(s, out);
}

// W_j pointer stride: F32 spinor = 6 V float4; F64 spinor = 12 V double2 (6 chunks of 2).
void restrict_(Ctx& c, int prec, const void* r, void* cvec, int cprec) {
  ProfScope ps(c, PK_RESTRICT);
  const int nv = c.cl.nv;
  const size_t smem = 33 * 32 * sizeof(double);   // per-warp sums (8 x 32) and the 32 totals
  if (prec == TMG_PREC_F64) {
    SpinorF64 rs{(double2*)r, c.g.V}, ws{c.cl.W64.as<double2>(), c.g.V};
    if (cprec == TMG_PREC_F64) ++c.launches, k_restrict<double><<<c.g.nblk, c.g.VB, smem, c.stream>>>(c.g, rs, ws, nv, (double2*)cvec);
    else ++c.launches, k_restrict<double><<<c.g.nblk, c.g.VB, smem, c.stream>>>(c.g, rs, ws, nv, (float2*)cvec);
  } else {
    SpinorF32 rs{(float4*)r, c.g.V}, ws{c.cl.W32.as<float4>(), c.g.V};
    if (cprec == TMG_PREC_F64) ++c.launches, k_restrict<float><<<c.g.nblk, c.g.VB, smem, c.stream>>>(c.g, rs, ws, nv, (double2*)cvec);
    else ++c.launches, k_restrict<float><<<c.g.nblk, c.g.VB, smem, c.stream>>>(c.g, rs, ws, nv, (float2*)cvec);
  }
  TMG_CHECK_LAUNCH();
}

void prolong(Ctx& c, int prec, const void* cvec, int cprec, void* e, int accumulate) {
  ProfScope ps(c, PK_PROLONG);
  const int nv = c.cl.nv;
  if (prec == TMG_PREC_F64) {
    SpinorF64 es{(double2*)e, c.g.V}, ws{c.cl.W64.as<double2>(), c.g.V};
    const size_t smem = 2 * nv * sizeof(cpx<double>);
    if (cprec == TMG_PREC_F64) ++c.launches, k_prolong<double><<<c.g.nblk, c.g.VB, smem, c.stream>>>(c.g, (const double2*)cvec, ws, nv, es, accumulate);
    else ++c.launches, k_prolong<double><<<c.g.nblk, c.g.VB, smem, c.stream>>>(c.g, (const float2*)cvec, ws, nv, es, accumulate);
  } else {
    SpinorF32 es{(float4*)e, c.g.V}, ws{c.cl.W32.as<float4>(), c.g.V};
    const size_t smem = 2 * nv * sizeof(cpx<float>);
    if (cprec == TMG_PREC_F64) ++c.launches, k_prolong<float><<<c.g.nblk, c.g.VB, smem, c.stream>>>(c.g, (const double2*)cvec, ws, nv, es, accumulate);
    else ++c.launches, k_prolong<float><<<c.g.nblk, c.g.VB, smem, c.stream>>>(c.g, (const float2*)cvec, ws, nv, es, accumulate);
  }
  TMG_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ coarse operator apply
// Coarse site a = block index; stencil slot d: 0 self, 1 + 2 mu: +mu face, 2 + 2 mu: -mu face.
__device__ __forceinline__ int coarse_nbr(const Geom& g, int a, int d) {
  if (d == 0) return a;
  const int mu = (d - 1) >> 1, dir = ((d - 1) & 1) ? -1 : 1;
  int b[4], q = a;
  b[0] = q % g.NB[0]; q /= g.NB[0];
  b[1] = q % g.NB[1]; q /= g.NB[1];
  b[2] = q % g.NB[2]; b[3] = q / g.NB[2];
  b[mu] += dir;
  if (b[mu] < 0) b[mu] += g.NB[mu];
  if (b[mu] >= g.NB[mu]) b[mu] -= g.NB[mu];
  return b[0] + g.NB[0] * (b[1] + g.NB[1] * (b[2] + g.NB[2] * b[3]));
}

// y[a][k] = sum_d sum_l Dc[a][d][l][k] x[nbr(a, d)][l] + i mu g5c[k] x[a][k]
template <typename R, typename T2>
__global__ void __launch_bounds__(128) k_coarse_apply(Geom g, int nd, int nv, const T2* __restrict__ Dc,
                                                      const T2* __restrict__ x, T2* __restrict__ y, R mu,
                                                      const int* __restrict__ skip) {
  if (skip && *skip) return;
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= g.nblk * nd) return;
  const int a = idx / nd, k = idx - a * nd;
  cpx<R> acc = mk<R>(0, 0);
  for (int d = 0; d < 9; d++) {
    const int nb = coarse_nbr(g, a, d);
    const T2* blk = Dc + ((size_t)(a * 9 + d) * nd) * nd + k;
    const T2* xv = x + (size_t)nb * nd;
    for (int l = 0; l < nd; l++) {
      const T2 m = blk[(size_t)l * nd];
      const T2 v = xv[l];
      acc = acc + mk<R>((R)m.x, (R)m.y) * mk<R>((R)v.x, (R)v.y);
    }
  }
  const T2 xs = x[(size_t)a * nd + k];
  const R tw = k < nv ? mu : -mu;
  acc = acc + tw * mul_i(mk<R>((R)xs.x, (R)xs.y));
  T2 o;
  o.x = acc.re;
  o.y = acc.im;
  y[(size_t)a * nd + k] = o;
}

void coarse_apply(Ctx& c, int cprec, const void* x, void* y, double mu, const int* skip) {
  ProfScope ps(c, PK_COARSE);
  const int nd = c.cl.nd;
  const int n = c.g.nblk * nd;
  if (cprec == TMG_PREC_F64)
    ++c.launches, k_coarse_apply<double, double2><<<(n + 127) / 128, 128, 0, c.stream>>>(c.g, nd, c.cl.nv, c.cl.Dc64.as<double2>(),
                                                                            (const double2*)x, (double2*)y, mu, skip);
  else
    ++c.launches, k_coarse_apply<float, float2><<<(n + 127) / 128, 128, 0, c.stream>>>(c.g, nd, c.cl.nv, c.cl.Dc32.as<float2>(),
                                                                          (const float2*)x, (float2*)y, (float)mu, skip);
  TMG_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ coarse operator build (FP64)
// Column l = (chi_l, j_l) of all 9 stencil blocks of every aggregate:
//   w = W_{j_l} projected on chirality chi_l (P e_l on every aggregate at once),
//   self:  P^dag [ A w - 1/2 (hops inside the aggregate) ],   twist excluded,
//   +mu:   P^dag [ -1/2 (1 - g_mu) U_mu(x) w(x+mu) on the +mu face ],
//   -mu:   P^dag [ -1/2 (1 + g_mu) U_mu(x-mu)^dag w(x-mu) on the -mu face ].
__global__ void __launch_bounds__(256) k_coarse_build_col(Geom g, int nv, int l, const double2* __restrict__ W,
                                                          GaugeF64 U, CloverF64 A, double2* __restrict__ Dc) {
  extern __shared__ double red[];
  const int blk = blockIdx.x;
  const int t = threadIdx.x;
  const int s = blk * g.VB + t;
  const int nd = 2 * nv;
  const SiteCoord sc = decode_site(g, s);
  const int chi_l = l / nv, j_l = l % nv;
  const SpinorF64 wl{const_cast<double2*>(W) + (size_t)j_l * 12 * g.V, g.V};
  auto loadw = [&](int site, Spinor<double>& o) {
    wl.load(site, o);
#pragma unroll
    for (int k = 0; k < 12; k++)
      if (k / 6 != chi_l) o.c[k] = mk(0.0, 0.0);
  };
  const int tcoord = coord(g, sc, 3);
  for (int d = 0; d < 9; d++) {
    Spinor<double> h;
#pragma unroll
    for (int k = 0; k < 12; k++) h.c[k] = mk(0.0, 0.0);
    if (d == 0) {
      Spinor<double> acc;
#pragma unroll
      for (int k = 0; k < 12; k++) acc.c[k] = mk(0.0, 0.0);
      for (int mu = 0; mu < 4; mu++) {
        if (sc.l[mu] + 1 < g.B[mu]) {
          Spinor<double> p;
          loadw(s + g.ls[mu], p);
          cpx<double> hh[6], uh[6];
          spin_project(mu, +1, p, hh);
          Link<double> u;
          U.load(s, mu, u);
          su3_mul_half(u, false, hh, uh);
          spin_reconstruct_add(mu, +1, uh, acc);
        }
        if (sc.l[mu] > 0) {
          Spinor<double> p;
          loadw(s - g.ls[mu], p);
          cpx<double> hh[6], uh[6];
          spin_project(mu, -1, p, hh);
          Link<double> u;
          U.load(s - g.ls[mu], mu, u);
          su3_mul_half(u, true, hh, uh);
          spin_reconstruct_add(mu, -1, uh, acc);
        }
      }
      Spinor<double> ws;
      loadw(s, ws);
      for (int chi = 0; chi < 2; chi++) {
        CloverBlock<double> a;
        A.load(s, chi, a);
        clover_mul(a, 0.0, &ws.c[6 * chi], &h.c[6 * chi]);
      }
#pragma unroll
      for (int k = 0; k < 12; k++) h.c[k] = h.c[k] - 0.5 * acc.c[k];
    } else {
      const int mu = (d - 1) >> 1;
      const bool fwd = ((d - 1) & 1) == 0;
      const bool on_face = fwd ? (sc.l[mu] == g.B[mu] - 1) : (sc.l[mu] == 0);
      if (on_face) {
        Spinor<double> acc;
#pragma unroll
        for (int k = 0; k < 12; k++) acc.c[k] = mk(0.0, 0.0);
        Spinor<double> p;
        cpx<double> hh[6], uh[6];
        Link<double> u;
        if (fwd) {
          loadw(nbr_fwd(g, sc, mu), p);
          spin_project(mu, +1, p, hh);
          U.load(s, mu, u);
          su3_mul_half(u, false, hh, uh);
          if (mu == 3 && tcoord == g.L[3] - 1 && g.tbc < 0)
            for (int k = 0; k < 6; k++) uh[k] = neg(uh[k]);
          spin_reconstruct_add(mu, +1, uh, acc);
        } else {
          const int sb = nbr_bwd(g, sc, mu);
          loadw(sb, p);
          spin_project(mu, -1, p, hh);
          U.load(sb, mu, u);
          su3_mul_half(u, true, hh, uh);
          if (mu == 3 && tcoord == 0 && g.tbc < 0)
            for (int k = 0; k < 6; k++) uh[k] = neg(uh[k]);
          spin_reconstruct_add(mu, -1, uh, acc);
        }
#pragma unroll
        for (int k = 0; k < 12; k++) h.c[k] = -0.5 * acc.c[k];
      }
    }
    // column entries k = (chi_k, j_k): <W_j P_chi, h> over the aggregate, in chunks of 8 vectors
    for (int j0 = 0; j0 < nv; j0 += 8) {
      double v[32];
#pragma unroll
      for (int i = 0; i < 32; i++) v[i] = 0.0;
#pragma unroll
      for (int jj = 0; jj < 8; jj++) {
        const int j = j0 + jj;
        if (j < nv) {
          const SpinorF64 wj{const_cast<double2*>(W) + (size_t)j * 12 * g.V, g.V};
          Spinor<double> wv;
          wj.load(s, wv);
#pragma unroll
          for (int k = 0; k < 12; k++) {
            const cpx<double> q = cmul_conj(wv.c[k], h.c[k]);
            v[((k / 6) * 8 + jj) * 2] += q.re;
            v[((k / 6) * 8 + jj) * 2 + 1] += q.im;
          }
        }
      }
      cta_allreduce<32, double>(v, red);
      if (t < 16) {
        const int chi = t / 8, jj = t % 8, j = j0 + jj;
        if (j < nv) {
          const int k = chi * nv + j;
          Dc[((size_t)(blk * 9 + d) * nd + l) * nd + k] = make_double2(v[(chi * 8 + jj) * 2], v[(chi * 8 + jj) * 2 + 1]);
        }
      }
    }
  }
}

template <typename A2, typename B2>
__global__ void k_copy_convert(const A2* __restrict__ a, B2* __restrict__ b, size_t n) {
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n; i += (size_t)gridDim.x * blockDim.x) {
    const A2 v = a[i];
    B2 o;
    o.x = v.x;
    o.y = v.y;
    b[i] = o;
  }
}

void build_coarse(Ctx& c) {
  const int nd = c.cl.nd;
  ++c.cl.version;                    // per-site inverses of the old stencil are stale
  {
    std::vector<int> nb((size_t)c.g.nblk * 9);
    for (int a = 0; a < c.g.nblk; a++) {
      int b[4], q = a;
      b[0] = q % c.g.NB[0]; q /= c.g.NB[0];
      b[1] = q % c.g.NB[1]; q /= c.g.NB[1];
      b[2] = q % c.g.NB[2]; b[3] = q / c.g.NB[2];
      nb[(size_t)a * 9] = a;
      for (int mu = 0; mu < 4; mu++)
        for (int dir = 0; dir < 2; dir++) {
          int bb[4] = {b[0], b[1], b[2], b[3]};
          bb[mu] = (bb[mu] + (dir == 0 ? 1 : c.g.NB[mu] - 1)) % c.g.NB[mu];
          nb[(size_t)a * 9 + 1 + 2 * mu + dir] = bb[0] + c.g.NB[0] * (bb[1] + c.g.NB[1] * (bb[2] + c.g.NB[2] * bb[3]));
        }
    }
    c.cl.nbr.alloc(nb.size() * sizeof(int));
    TMG_CUDA(cudaMemcpyAsync(c.cl.nbr.p, nb.data(), nb.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream));
    TMG_CUDA(cudaStreamSynchronize(c.stream));
  }
  const size_t n = (size_t)c.g.nblk * 9 * nd * nd;
  c.cl.Dc64.alloc(n * sizeof(double2));
  c.cl.Dc32.alloc(n * sizeof(float2));
  const size_t smem = 33 * 32 * sizeof(double);
  for (int l = 0; l < nd; l++) {
    ++c.launches, k_coarse_build_col<<<c.g.nblk, c.g.VB, smem, c.stream>>>(c.g, c.cl.nv, l, c.cl.W64.as<double2>(),
                                                              GaugeF64{c.op[0].U.as<double2>(), c.g.V},
                                                              CloverF64{c.op[0].A.as<double2>(), c.g.V}, c.cl.Dc64.as<double2>());
    TMG_CHECK_LAUNCH();
  }
  ++c.launches, k_copy_convert<<<c.sms * 8, 256, 0, c.stream>>>(c.cl.Dc64.as<double2>(), c.cl.Dc32.as<float2>(), n);
  TMG_CHECK_LAUNCH();
}

// ------------------------------------------------------------------ orthonormalisation (FP64)
// One CTA per (aggregate, chirality): modified Gram-Schmidt over j = 0..nv-1, applied twice.
// The 6 complex entries of a site's chirality half of W_j are handled by the site's thread.
__global__ void __launch_bounds__(256) k_orthonormalise(Geom g, int nv, double2* __restrict__ W) {
  extern __shared__ double red[];
  const int blk = blockIdx.x >> 1, chi = blockIdx.x & 1;
  const int s = blk * g.VB + threadIdx.x;
  // complex index of (site s, component k) in a F64 spinor field: 2 ((k/2) V + s) + (k % 2)
  auto at = [&](int j, int k) -> double2& {
    return W[(size_t)j * 12 * g.V + 2 * ((size_t)(k >> 1) * g.V + s) + (k & 1)];
  };
  for (int pass = 0; pass < 2; pass++) {
    for (int j = 0; j < nv; j++) {
      cpx<double> wj[6];
      for (int k = 0; k < 6; k++) { const double2 v = at(j, 6 * chi + k); wj[k] = mk(v.x, v.y); }
      for (int i = 0; i < j; i++) {
        double v[2] = {0.0, 0.0};
        cpx<double> wi[6];
        for (int k = 0; k < 6; k++) {
          const double2 q = at(i, 6 * chi + k);
          wi[k] = mk(q.x, q.y);
          const cpx<double> z = cmul_conj(wi[k], wj[k]);
          v[0] += z.re;
          v[1] += z.im;
        }
        cta_allreduce<2, double>(v, red);
        const cpx<double> ov = mk(v[0], v[1]);
        for (int k = 0; k < 6; k++) wj[k] = wj[k] - ov * wi[k];
      }
      double n2[1] = {0.0};
      for (int k = 0; k < 6; k++) n2[0] += wj[k].re * wj[k].re + wj[k].im * wj[k].im;
      cta_allreduce<1, double>(n2, red);
      const double inv = n2[0] > 0.0 ? 1.0 / sqrt(n2[0]) : 0.0;
      for (int k = 0; k < 6; k++) at(j, 6 * chi + k) = make_double2(inv * wj[k].re, inv * wj[k].im);
      __syncthreads();
    }
  }
}

void orthonormalise(Ctx& c, void* W64) {
  const size_t smem = 33 * 2 * sizeof(double);
  ++c.launches, k_orthonormalise<<<2 * c.g.nblk, c.g.VB, smem, c.stream>>>(c.g, c.cl.nv, (double2*)W64);
  TMG_CHECK_LAUNCH();
}

// y += (are + i aim) G5_c x on coarse vectors ([nc][nd], dofs [+: nv | -: nv])
template <typename T2>
__global__ void k_coarse_g5_axpy(const T2* __restrict__ x, T2* __restrict__ y, size_t n, int nd, double are, double aim) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const int k = (int)(e % nd);
    const double s = k < nd / 2 ? 1.0 : -1.0;
    const T2 v = x[e];
    T2 o = y[e];
    o.x += s * (are * v.x - aim * v.y);
    o.y += s * (are * v.y + aim * v.x);
    y[e] = o;
  }
}

void coarse_g5_axpy(Ctx& c, int prec, double are, double aim, const void* x, void* y) {
  const size_t n = (size_t)c.cl.nc * c.cl.nd;
  const int G = (int)std::max<size_t>(1, std::min<size_t>((n + 255) / 256, (size_t)c.sms * 8));
  if (prec == TMG_PREC_F64)
    ++c.launches, k_coarse_g5_axpy<double2><<<G, 256, 0, c.stream>>>((const double2*)x, (double2*)y, n, c.cl.nd, are, aim);
  else
    ++c.launches, k_coarse_g5_axpy<float2><<<G, 256, 0, c.stream>>>((const float2*)x, (float2*)y, n, c.cl.nd, are, aim);
  TMG_CHECK_LAUNCH();
}

}  // namespace tmg
