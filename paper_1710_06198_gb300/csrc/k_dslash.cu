// Fine-grid operator kernels: y = D(mu) x with the clover and twisted-mass term fused into the
// epilogue of the hopping term (Sec. 1.1 of arXiv:1710.06198: D(+-mu) = D +- i mu G5), and the
// non-degenerate doublet of Eq. 2.
//
// One thread per site; all loads are 16-byte vectors from structure-of-arrays fields, so a warp
// reads 32 consecutive sites of one component chunk in one transaction.  The hopping term uses the
// rank-2 spin projectors (1 -+ g_mu): project to a half spinor, multiply by the link (compressed
// links are reconstructed in registers), and rebuild the lower spin pair from the upper one.
#include "tmg_host.h"
#include "dslash_core.cuh"

namespace tmg {

// mode 0: y = D x; mode 1: y = b - D x; mode 2: y = hopping term only (-1/2 sum ...).
// dagger: y = g5 D(-mu) g5 x = D(mu)^dag x.
template <typename R, class S, class G, class C>
__global__ void __launch_bounds__(128) k_dslash(Geom g, S y, S x, S b, G U, C A, R mu, int mode, int dagger) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const SiteCoord sc = decode_site(g, s);
  Spinor<R> acc;
  hopping_sum<R>(g, sc, s, x, U, dagger != 0, acc);
  Spinor<R> out;
  if (mode == 2) {
#pragma unroll
    for (int k = 0; k < 12; k++) out.c[k] = R(-0.5) * acc.c[k];
  } else {
    Spinor<R> xs;
    x.load(s, xs);
    if (dagger) apply_g5(xs);
    const R tw = dagger ? -mu : mu;
#pragma unroll
    for (int chi = 0; chi < 2; chi++) {
      CloverBlock<R> a;
      A.load(s, chi, a);
      clover_mul(a, chi == 0 ? tw : -tw, &xs.c[6 * chi], &out.c[6 * chi]);
    }
#pragma unroll
    for (int k = 0; k < 12; k++) out.c[k] = out.c[k] - R(0.5) * acc.c[k];
  }
  if (dagger) apply_g5(out);
  if (mode == 1) {
    Spinor<R> bs;
    b.load(s, bs);
#pragma unroll
    for (int k = 0; k < 12; k++) out.c[k] = bs.c[k] - out.c[k];
  }
  y.store(s, out);
}

// Non-degenerate doublet (Eq. 2): y_u = D(mubar) x_u - epsbar x_d, y_d = D(-mubar) x_d - epsbar x_u,
// plus i delta g5 x_d / i delta g5 x_u for the shifted doublet (delta = the context's ndshift).
// Both flavours of a site are handled by one thread so the links and clover are read once.
template <typename R, class S, class G, class C>
__global__ void __launch_bounds__(128) k_dslash_nd(Geom g, S yu, S yd, S xu, S xd, G U, C A, R mubar, R epsbar,
                                                   R delta) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const SiteCoord sc = decode_site(g, s);
  Spinor<R> acc_u, acc_d;
  hopping_sum<R>(g, sc, s, xu, U, false, acc_u);
  hopping_sum<R>(g, sc, s, xd, U, false, acc_d);
  Spinor<R> su, sd, ou, od;
  xu.load(s, su);
  xd.load(s, sd);
#pragma unroll
  for (int chi = 0; chi < 2; chi++) {
    CloverBlock<R> a;
    A.load(s, chi, a);
    clover_mul(a, chi == 0 ? mubar : -mubar, &su.c[6 * chi], &ou.c[6 * chi]);
    clover_mul(a, chi == 0 ? -mubar : mubar, &sd.c[6 * chi], &od.c[6 * chi]);
  }
#pragma unroll
  for (int k = 0; k < 12; k++) {
    ou.c[k] = ou.c[k] - R(0.5) * acc_u.c[k] + nd_mix(epsbar, delta, k, sd.c[k]);
    od.c[k] = od.c[k] - R(0.5) * acc_d.c[k] + nd_mix(epsbar, delta, k, su.c[k]);
  }
  yu.store(s, ou);
  yd.store(s, od);
}

static SpinorF64 sp64(const Ctx& c, const void* p) { return SpinorF64{(double2*)p, c.g.V}; }
static SpinorF32 sp32(const Ctx& c, const void* p) { return SpinorF32{(float4*)p, c.g.V}; }

void dslash(Ctx& c, int prec, void* y, const void* x, const void* b, double mu, int mode, int dagger) {
  const int threads = 128;
  const int blocks = (c.g.V + threads - 1) / threads;
  if (!b) b = x;
  ProfScope ps(c, prec == PREC_H16 ? PK_DSLASH_F16 : PK_DSLASH_F64 + prec);
  if (prec == PREC_H16) {
    // all-FP16 storage: fixed-point spinors with per-site norms, FP16 links and clover; FP32 math
    ++c.launches, k_dslash<float><<<blocks, threads, 0, c.stream>>>(c.g, spinor_h16(c, y), spinor_h16(c, (void*)x),
                                                      spinor_h16(c, (void*)b),
                                                      GaugeF16{c.op[2].U.as<short4>(), c.g.V},
                                                      CloverF16{c.op[2].A.as<short4>(), c.op[2].Ascale.as<float>(), c.g.V},
                                                      (float)mu, mode, dagger);
  } else if (prec == TMG_PREC_F64) {
    ++c.launches, k_dslash<double><<<blocks, threads, 0, c.stream>>>(c.g, sp64(c, y), sp64(c, x), sp64(c, b),
                                                       GaugeF64{c.op[0].U.as<double2>(), c.g.V},
                                                       CloverF64{c.op[0].A.as<double2>(), c.g.V}, mu, mode, dagger);
  } else if (prec == TMG_PREC_F32) {
    ++c.launches, k_dslash<float><<<blocks, threads, 0, c.stream>>>(c.g, sp32(c, y), sp32(c, x), sp32(c, b),
                                                      GaugeF32{c.op[1].U.as<float4>(), c.g.V},
                                                      CloverF32{c.op[1].A.as<float4>(), c.g.V}, (float)mu, mode, dagger);
  } else {
    ++c.launches, k_dslash<float><<<blocks, threads, 0, c.stream>>>(c.g, sp32(c, y), sp32(c, x), sp32(c, b),
                                                      GaugeF16{c.op[2].U.as<short4>(), c.g.V},
                                                      CloverF16{c.op[2].A.as<short4>(), c.op[2].Ascale.as<float>(), c.g.V},
                                                      (float)mu, mode, dagger);
  }
  TMG_CHECK_LAUNCH();
}

void dslash_nd(Ctx& c, int prec, void* y, const void* x) {
  const int threads = 128;
  const int blocks = (c.g.V + threads - 1) / threads;
  const size_t col = (size_t)12 * c.g.V;
  if (prec == TMG_PREC_F64) {
    const double2* xp = (const double2*)x;
    double2* yp = (double2*)y;
    ++c.launches, k_dslash_nd<double><<<blocks, threads, 0, c.stream>>>(c.g, sp64(c, yp), sp64(c, yp + col), sp64(c, xp), sp64(c, xp + col),
                                                          GaugeF64{c.op[0].U.as<double2>(), c.g.V},
                                                          CloverF64{c.op[0].A.as<double2>(), c.g.V}, c.mubar, c.epsbar, c.ndshift);
  } else {
    const float2* xp = (const float2*)x;
    float2* yp = (float2*)y;
    if (prec == TMG_PREC_F32)
      ++c.launches, k_dslash_nd<float><<<blocks, threads, 0, c.stream>>>(c.g, sp32(c, yp), sp32(c, yp + col), sp32(c, xp), sp32(c, xp + col),
                                                           GaugeF32{c.op[1].U.as<float4>(), c.g.V},
                                                           CloverF32{c.op[1].A.as<float4>(), c.g.V}, (float)c.mubar, (float)c.epsbar, (float)c.ndshift);
    else
      ++c.launches, k_dslash_nd<float><<<blocks, threads, 0, c.stream>>>(c.g, sp32(c, yp), sp32(c, yp + col), sp32(c, xp), sp32(c, xp + col),
                                                           GaugeF16{c.op[2].U.as<short4>(), c.g.V},
                                                           CloverF16{c.op[2].A.as<short4>(), c.op[2].Ascale.as<float>(), c.g.V},
                                                           (float)c.mubar, (float)c.epsbar, (float)c.ndshift);
  }
  TMG_CHECK_LAUNCH();
}

}  // namespace tmg
