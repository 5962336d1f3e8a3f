// Device building blocks of the Wilson hopping term shared by the dslash, SAP and coarse-build
// kernels.
#pragma once
#include "tmg_internal.cuh"

namespace tmg {

template <typename R>
__device__ __forceinline__ void apply_g5(Spinor<R>& p) {
#pragma unroll
  for (int k = 6; k < 12; k++) p.c[k] = neg(p.c[k]);
}

// hopping sum  acc = sum_mu [(1 - g_mu) U_mu(x) p(x+mu) + (1 + g_mu) U_mu(x-mu)^dag p(x-mu)]
template <typename R, class S, class G>
__device__ __forceinline__ void hopping_sum(const Geom& g, const SiteCoord& sc, int s, const S& x, const G& U,
                                            bool g5in, Spinor<R>& acc) {
#pragma unroll
  for (int k = 0; k < 12; k++) acc.c[k] = mk<R>(0, 0);
  const int t = coord(g, sc, 3);
#pragma unroll
  for (int mu = 0; mu < 4; mu++) {
    {
      const int sf = nbr_fwd(g, sc, mu);
      Spinor<R> p;
      x.load(sf, p);
      if (g5in) apply_g5(p);
      cpx<R> h[6], uh[6];
      spin_project(mu, +1, p, h);
      Link<R> u;
      U.load(s, mu, u);
      su3_mul_half(u, false, h, uh);
      if (mu == 3 && t == g.L[3] - 1 && g.tbc < 0) {
#pragma unroll
        for (int k = 0; k < 6; k++) uh[k] = neg(uh[k]);
      }
      spin_reconstruct_add(mu, +1, uh, acc);
    }
    {
      const int sb = nbr_bwd(g, sc, mu);
      Spinor<R> p;
      x.load(sb, p);
      if (g5in) apply_g5(p);
      cpx<R> h[6], uh[6];
      spin_project(mu, -1, p, h);
      Link<R> u;
      U.load(sb, mu, u);
      su3_mul_half(u, true, h, uh);
      if (mu == 3 && t == 0 && g.tbc < 0) {
#pragma unroll
        for (int k = 0; k < 6; k++) uh[k] = neg(uh[k]);
      }
      spin_reconstruct_add(mu, -1, uh, acc);
    }
  }
}


// D x at site s: (A + i tw g5) x(s) - 1/2 hopping_sum (full lattice operator, twist tw).
template <typename R, class S, class G, class C>
__device__ __forceinline__ void apply_D_site(const Geom& g, const SiteCoord& sc, int s, const S& x, const G& U,
                                             const C& A, R tw, Spinor<R>& out) {
  Spinor<R> acc;
  hopping_sum<R>(g, sc, s, x, U, false, acc);
  Spinor<R> xs;
  x.load(s, xs);
#pragma unroll
  for (int chi = 0; chi < 2; chi++) {
    CloverBlock<R> a;
    A.load(s, chi, a);
    clover_mul(a, chi == 0 ? tw : -tw, &xs.c[6 * chi], &out.c[6 * chi]);
  }
#pragma unroll
  for (int k = 0; k < 12; k++) out.c[k] = out.c[k] - R(0.5) * acc.c[k];
}

}  // namespace tmg
