// The coarse solve D_c^-1 of Eq. 1 (arXiv:1710.06198) as ONE persistent cooperative kernel:
// GMRES from zero, at most m steps, stopping once the Givens estimate of the relative residual
// reaches rtol; classical Gram-Schmidt with an optional second pass.
//
// Every CTA stays resident for the whole solve; phases are separated by grid-wide barriers of a
// cooperative launch (two per step: the dot products' partials, then w and its norm).  Each CTA
// owns a range of coarse sites: it computes their stencil rows and owns those elements of every
// vector, so the stencil needs no barrier of its own.  The small sequential work (Hessenberg
// column, Givens rotations, stopping test) is repeated identically by every CTA from the same
// reduced values, so no extra barrier is needed to broadcast it; CTA 0 alone keeps the rotated
// Hessenberg for the back substitution.  Vectors, reductions and rotations are all in the coarse
// precision S (FP32 or FP64): FP64 is far slower than FP32 on GB300, so the FP32 path uses none.
#include <cooperative_groups.h>

#include "tmg_host.h"
#include "level2.cuh"

namespace cg = cooperative_groups;

namespace tmg {

namespace {

constexpr int CMAXM = 64;

template <typename S>
struct CplxT;
template <> struct CplxT<float> { using T2 = float2; };
template <> struct CplxT<double> { using T2 = double2; };

template <typename S>
struct CgArgs {
  int nd, nv, nc, m, passes;
  int nf;                            // flavours: 1, or 2 for the doublet (vectors [nf][nc][nd])
  const typename CplxT<S>::T2* Dc;   // [nc][9][nd(l)][nd(k)]
  const int* nbr;                    // [nc][9]
  const typename CplxT<S>::T2* b;
  typename CplxT<S>::T2* x;
  typename CplxT<S>::T2* V;          // (m + 1) x n basis
  typename CplxT<S>::T2* w;          // 2 x n: w of even and of odd steps
  typename CplxT<S>::T2* rows;       // [nf][nc][9][nd] partial stencil rows
  S mu;                              // twist (doublet: mubar, flavour 1 gets -mubar)
  S epsbar;                          // doublet flavour mixing -epsbar tau1 (unused for nf = 1)
  S delta;                           // shifted doublet: + i delta G5 x tau1 (0 for Eq. 2 itself)
  double rtol;
  double2* part;                     // [2][CMAXM + 1][grid] dot partials (by pass parity; pairs of S)
  double* npart;                     // [grid] norm partials (values of S)
  double2* R;                        // rotated Hessenberg, column-major (CMAXM + 1) x CMAXM (pairs of S)
  double2* y;                        // solution coefficients (pairs of S)
  int* counter;                      // accumulated step count
  int rows_smem;                     // 1: the own sites' stencil rows live in dynamic shared memory
                                     // (ceil(nc / grid) * nf * 9 * nd values); 0: in rows
  int blk_cache;                     // own stencil blocks copied once per launch into dynamic shared
  int cache_off;                     // memory (from the first own block on), at byte offset cache_off
  int eo;                            // 1: solve the odd-even reduced system (nf = 1, even extents)
  int cg[4];                         // coarse lattice extents (site = x + X (y + Y (z + Z t)))
  const typename CplxT<S>::T2* inv;  // eo: per-site (A_self + i mu G5_c)^-1, [nc][nd(l)][nd(k)]
  typename CplxT<S>::T2* te;         // eo: even-site intermediate A_ee^-1 (...) [n]
  typename CplxT<S>::T2* rb;         // eo: reduced right-hand side [n]
  int overlap;                       // 1: the Hessenberg update of step j runs during the stencil of
                                     // step j+1 (warp 0 of every CTA); 0: after step j, all warps stencil
};

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Sum of one value per thread over the CTA (result returned to every thread).
template <typename A>
__device__ __forceinline__ A cta_sum(A v, A* sh) {
  v = warp_sum(v);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (lane == 0) sh[w] = v;
  __syncthreads();
  A t = 0;
  for (int k = 0; k < (int)(blockDim.x >> 5); k++) t += sh[k];
  __syncthreads();
  return t;
}

// One stencil task, by one warp: out[k] = scale * (sum_l blk[l][k] x[l] + (-epsbar + i delta g5_k) xo[k])
// for the nd rows k of one (nd x nd) block (xo: the doublet's other flavour on the self block, or
// null; g5_k = +1 for the first nd / 2 rows, -1 for the others).
// FP32 blocks whose half width divides 32 are read as float4 (two rows per load) with the columns
// split over lane groups, so every lane keeps all its loads in flight at once; the group partial
// sums are combined with shuffles.  Other shapes: lanes are rows and every column is one coalesced
// read.
template <typename S>
__device__ __forceinline__ void stencil_task(const typename CplxT<S>::T2* __restrict__ blk,
                                             const typename CplxT<S>::T2* __restrict__ xv, int nd, S scale,
                                             const typename CplxT<S>::T2* xo, S epsbar, S delta,
                                             typename CplxT<S>::T2* __restrict__ out, int lane) {
  using T2 = typename CplxT<S>::T2;
  const int half = nd >> 1;
  if constexpr (sizeof(S) == 4) {
    if (half > 0 && (32 % half) == 0) {
      const int groups = 32 / half;
      const int kp = lane % half, lg = lane / half;
      const float4* bl = reinterpret_cast<const float4*>(blk);
      float ar0 = 0.f, ai0 = 0.f, ar1 = 0.f, ai1 = 0.f;
#pragma unroll 16
      for (int l = lg; l < nd; l += groups) {
        const float4 m = bl[(size_t)l * half + kp];
        const float2 v = xv[l];
        ar0 += m.x * v.x - m.y * v.y;
        ai0 += m.x * v.y + m.y * v.x;
        ar1 += m.z * v.x - m.w * v.y;
        ai1 += m.z * v.y + m.w * v.x;
      }
      for (int o = half; o < 32; o <<= 1) {
        ar0 += __shfl_xor_sync(0xffffffffu, ar0, o);
        ai0 += __shfl_xor_sync(0xffffffffu, ai0, o);
        ar1 += __shfl_xor_sync(0xffffffffu, ar1, o);
        ai1 += __shfl_xor_sync(0xffffffffu, ai1, o);
      }
      if (lg == 0) {
        const int k = 2 * kp;
        if (xo) {
          const float2 a0 = xo[k], a1 = xo[k + 1];
          const float d0 = k < half ? delta : -delta, d1 = k + 1 < half ? delta : -delta;
          ar0 += -epsbar * a0.x - d0 * a0.y;
          ai0 += -epsbar * a0.y + d0 * a0.x;
          ar1 += -epsbar * a1.x - d1 * a1.y;
          ai1 += -epsbar * a1.y + d1 * a1.x;
        }
        out[k] = make_float2(ar0 * scale, ai0 * scale);
        out[k + 1] = make_float2(ar1 * scale, ai1 * scale);
      }
      return;
    }
  }
  for (int k = lane; k < nd; k += 32) {
    S ar = 0, ai = 0;
#pragma unroll 16
    for (int l = 0; l < nd; l++) {
      const T2 m = blk[(size_t)l * nd + k];
      const T2 v = xv[l];
      ar += m.x * v.x - m.y * v.y;
      ai += m.x * v.y + m.y * v.x;
    }
    if (xo) {
      const S d = k < half ? delta : -delta;
      ar += -epsbar * xo[k].x - d * xo[k].y;
      ai += -epsbar * xo[k].y + d * xo[k].x;
    }
    T2 o;
    o.x = ar * scale;
    o.y = ai * scale;
    out[k] = o;
  }
}

// One-dimensional bulk copy global -> shared memory completing on an mbarrier, and a wait on it
// that gives up after about a second (the caller then falls back to global loads).
__device__ __forceinline__ uint32_t gm_smem_addr(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void gm_bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  const uint32_t b = gm_smem_addr(bar);
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(gm_smem_addr(dst)), "l"(src), "r"(bytes), "r"(b)
               : "memory");
}
__device__ __forceinline__ bool gm_bulk_wait(uint64_t* bar) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t0));
  for (unsigned it = 0; it < (1u << 26); it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(gm_smem_addr(bar)), "r"(0u), "r"(20000u)
        : "memory");
    if (done) return true;
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    if (t - t0 > 1000000000ull) return false;
  }
  return false;
}

// Parity of a coarse site from its coordinates (x fastest).
__device__ __forceinline__ int coarse_site_parity(const int cg[4], int site) {
  const int x = site % cg[0];
  site /= cg[0];
  const int y = site % cg[1];
  site /= cg[1];
  const int z = site % cg[2];
  return (x + y + z + site / cg[2]) & 1;
}

// Precision-generic helpers of the persistent solvers: the FP32 path keeps its reductions, Givens
// rotations and least-squares solve in FP32 (GB300 issues FP64 at a small fraction of the FP32
// rate, and one FP64 Givens chain per step costs more than the step's stencil).
template <typename S>
__device__ __forceinline__ typename CplxT<S>::T2 mk2(S x, S y) {
  typename CplxT<S>::T2 r;
  r.x = x;
  r.y = y;
  return r;
}
__device__ __forceinline__ float sq(float v) { return sqrtf(v); }
__device__ __forceinline__ double sq(double v) { return sqrt(v); }
__device__ __forceinline__ float rsq(float v) { return rsqrtf(v); }
__device__ __forceinline__ double rsq(double v) { return rsqrt(v); }

// GMRES from zero on the operator of a (any level): grid-wide phases, the caller's grid must be a
// cooperative launch; a.x is complete after the caller's next grid barrier.
template <typename S, bool EO = false>
__device__ void gmres_dev(const CgArgs<S>& a) {
  using T2 = typename CplxT<S>::T2;
  using A2 = T2;   // reductions, rotations and the least-squares solve in the vectors' precision
  cg::grid_group grid = cg::this_grid();
  // the FP64-sized scratch of the launch holds the FP32 path's partials and rotations as well
  A2* const part_base = reinterpret_cast<A2*>(a.part);
  S* const npart = reinterpret_cast<S*>(a.npart);
  A2* const Rm = reinterpret_cast<A2*>(a.R);
  A2* const ym = reinterpret_cast<A2*>(a.y);
  __shared__ S sh[32];
  __shared__ A2 hcol[CMAXM + 2];
  __shared__ A2 cs[CMAXM], sn[CMAXM], gv[CMAXM + 1];
  __shared__ A2 hp[CMAXM + 1];
  __shared__ int s_done, s_k;
  __shared__ S s_beta, s_hn;
  const int n1 = a.nc * a.nd, n = a.nf * n1;
  const int G = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = G * blockDim.x;
  // Coarse sites [s0, s1) of every flavour belong to this CTA: it computes their stencil rows, sums
  // them into w and is the only CTA that reads or writes those elements of the basis and of w until
  // the next grid barrier.  Own element t in [0, nown) is flavour t / own, offset t % own.
  const int s0 = (int)(((long long)blockIdx.x * a.nc) / G), s1 = (int)(((long long)(blockIdx.x + 1) * a.nc) / G);
  const int own = (s1 - s0) * a.nd, nown = a.nf * own;
#define GM_OWN_E(t) ((t) >= own ? n1 + s0 * a.nd + ((t) - own) : s0 * a.nd + (t))
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  // stencil rows of (flavour f, own site): in shared memory when the launch provides it (the rows
  // are written and read by this CTA only, so they never need a trip through L2), else global
  extern __shared__ __align__(16) unsigned char gm_dyn[];
  T2* const rows_sm = reinterpret_cast<T2*>(gm_dyn);
  T2* const rows_g = a.rows_smem ? rows_sm : a.rows;          // (flavour, site) row block origin:
  const int rows_site0 = a.rows_smem ? s0 : 0;                  // own sites only in shared memory
  const int rows_nsite = a.rows_smem ? s1 - s0 : a.nc;
#define GM_ROW_BASE(f, site) (rows_g + ((size_t)((f) * rows_nsite + (site) - rows_site0) * 9) * a.nd)
  // The stencil does not change during the solve: the CTA's first ncache own blocks (contiguous in
  // Dc) are copied once into shared memory and read from there at every step; the rest come from
  // L2.  The copy runs while the right-hand side's norm is reduced.
  __shared__ __align__(8) uint64_t s_cache_bar;
  __shared__ int s_cache_ok;
  T2* const blk_sm = reinterpret_cast<T2*>(gm_dyn + a.cache_off);
  const int ncache = min(a.blk_cache, (s1 - s0) * 9);
  if (ncache > 0) {
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(gm_smem_addr(&s_cache_bar)), "r"(1));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      gm_bulk_copy(blk_sm, a.Dc + (size_t)s0 * 9 * a.nd * a.nd, (uint32_t)((size_t)ncache * a.nd * a.nd * sizeof(T2)),
                   &s_cache_bar);
    }
  }

  // ---- odd-even reduced system (a.eo, one flavour, even coarse extents): the basis and w live on
  // the odd sites (their even entries stay zero).  GM_HOP_ROWS: hop products (blocks d = 1..8) of the
  // own sites of parity P applied to X, scaled by SC, into those sites' rows (the first NCACHED own
  // blocks from shared memory); GM_INV_TASKS: per own even site, OUT = A_ee^-1 IN.
#define GM_HOP_ROWS(P, X, SC, W0, NW, NCACHED)                                                        \
  for (int t = (W0); t < (s1 - s0) * 8; t += (NW)) {                                                 \
    const int site = s0 + t / 8, d = 1 + (t & 7);                                                    \
    if (coarse_site_parity(a.cg, site) != (P)) continue;                                             \
    const int t9 = site * 9 + d, lb = t9 - s0 * 9;                                                   \
    const T2* blk = lb < (NCACHED) ? blk_sm + (size_t)lb * a.nd * a.nd : a.Dc + (size_t)t9 * a.nd * a.nd; \
    stencil_task<S>(blk, (X) + (size_t)a.nbr[t9] * a.nd, a.nd, (SC), nullptr, (S)0, (S)0,            \
                    GM_ROW_BASE(0, site) + (size_t)d * a.nd, lane);                                  \
  }
#define GM_INV_TASKS(IN, OUT)                                                                        \
  for (int t = warp; t < s1 - s0; t += nwarp) {                                                      \
    const int site = s0 + t;                                                                         \
    if (coarse_site_parity(a.cg, site) != 0) continue;                                               \
    stencil_task<S>(a.inv + (size_t)site * a.nd * a.nd, (IN), a.nd, (S)1, nullptr, (S)0, (S)0, (OUT), lane); \
  }
  const T2* bsrc = a.b;
  if (EO) {
    // reduced right-hand side r_o = b_o - A_oe A_ee^-1 b_e
    GM_INV_TASKS(a.b + (size_t)site * a.nd, a.te + (size_t)site * a.nd);
    grid.sync();                                     // A_ee^-1 b_e complete
    GM_HOP_ROWS(1, a.te, (S)-1, warp, nwarp, 0);
    __syncthreads();
    for (int t = threadIdx.x; t < nown; t += blockDim.x) {
      const int e = GM_OWN_E(t), site = e / a.nd, k = e - site * a.nd;
      T2 o = mk2<S>(0, 0);
      if (coarse_site_parity(a.cg, site) == 1) {
        o = a.b[e];
        const T2* rw = GM_ROW_BASE(0, site) + k;
        for (int d = 1; d < 9; d++) { const T2 r = rw[(size_t)d * a.nd]; o.x += r.x; o.y += r.y; }
      }
      a.rb[e] = o;
    }
    grid.sync();                                     // r_o complete
    bsrc = a.rb;
  }

  // beta = ||b|| (of the reduced right-hand side for the odd-even system)
  {
    S nn = 0;
    for (int e = tid; e < n; e += nth) { const T2 v = bsrc[e]; nn += v.x * v.x + v.y * v.y; }
    const S t = cta_sum((S)nn, sh);
    if (threadIdx.x == 0) npart[blockIdx.x] = t;
  }
  grid.sync();
  if (warp == 0) {
    S t = 0;
    for (int q = lane; q < G; q += 32) t += npart[q];
    t = warp_sum(t);
    if (lane == 0) s_beta = sq(t);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_done = !(s_beta > (S)0);
    s_k = 0;
    s_hn = 1.0;
    for (int i = 0; i <= CMAXM; i++) gv[i] = mk2<S>(0, 0);
    gv[0] = mk2<S>(s_beta, (S)0);
  }
  __syncthreads();
  {
    const S inv = s_beta > (S)0 ? (S)1 / s_beta : (S)0;
    for (int e = tid; e < n; e += nth) { T2 v = bsrc[e]; v.x *= inv; v.y *= inv; a.V[e] = v; }
  }
  grid.sync();                                       // v_0 complete
  // Hessenberg column j: previous rotations [[conj c, conj s], [-s, c]] applied down the new column
  // (the running entry stays in registers), then the new rotation from (running entry, h_{j+1,j}),
  // the residual estimate and the stopping test.  Run by one thread of every CTA from the same
  // reduced values, so every CTA takes the same decision.
  auto hessenberg_update = [&](int j) {
    const S hn = s_hn;
    A2 x0 = hcol[0];
    for (int i = 0; i < j; i++) {
      const A2 x1 = hcol[i + 1];
      const A2 c = cs[i], s = sn[i];
      hcol[i] = mk2<S>(c.x * x0.x + c.y * x0.y + s.x * x1.x + s.y * x1.y,
                       c.x * x0.y - c.y * x0.x + s.x * x1.y - s.y * x1.x);
      x0 = mk2<S>(-(s.x * x0.x - s.y * x0.y) + (c.x * x1.x - c.y * x1.y),
                  -(s.x * x0.y + s.y * x0.x) + (c.x * x1.y + c.y * x1.x));
    }
    // one reciprocal square root instead of a square root and four divisions
    const A2 p = x0;
    const S n2 = p.x * p.x + p.y * p.y + hn * hn;
    const S inv = n2 > (S)0 ? rsq(n2) : (S)0;
    const S den = n2 * inv;
    const A2 c = n2 > (S)0 ? mk2<S>(p.x * inv, p.y * inv) : mk2<S>(1, 0);
    const A2 sr = mk2<S>(hn * inv, (S)0);
    cs[j] = c;
    sn[j] = sr;
    hcol[j] = mk2<S>(den, (S)0);
    hcol[j + 1] = mk2<S>(0, 0);
    const A2 g = gv[j];
    gv[j + 1] = mk2<S>(-(sr.x * g.x), -(sr.x * g.y));
    gv[j] = mk2<S>(c.x * g.x + c.y * g.y, c.x * g.y - c.y * g.x);
    if (blockIdx.x == 0)
      for (int i = 0; i <= j; i++) Rm[(size_t)j * (CMAXM + 1) + i] = hcol[i];
    s_k = j + 1;
    const S res2 = gv[j + 1].x * gv[j + 1].x + gv[j + 1].y * gv[j + 1].y;
    const S lim = (S)a.rtol * s_beta;
    if (res2 <= lim * lim || !(hn > (S)0) || !(den > (S)0) || j == a.m - 1) s_done = 1;
  };
  // Warp 0 of every CTA keeps out of the stencil products so that its first thread can update the
  // Hessenberg column of the previous step meanwhile: the stencil of step j only needs the norm
  // h_{j,j-1} (known before the rotations), and if the rotations of step j-1 stop the solve, the
  // stencil rows of step j are simply not used.
  const bool ovl = a.overlap != 0;
  const int swarp = ovl ? warp - 1 : warp, snwarp = ovl ? nwarp - 1 : nwarp;
  const int ntask = a.nf * (s1 - s0) * 9;
  int cached = 0;                                    // own blocks readable from shared memory
  if (ncache > 0) {
    if (threadIdx.x == 0) s_cache_ok = gm_bulk_wait(&s_cache_bar) ? 1 : 0;
    __syncthreads();
    cached = s_cache_ok ? ncache : 0;
  }
  // s_done is read only right after a barrier (or before the loop, where it is settled): the
  // thread that updates the Hessenberg column may set it while other warps are still starting a
  // step.  Every CTA sets it from the same reduced values, so all take the same grid barriers.
  const bool zero_rhs = s_done;
  for (int j = 0; j < a.m && !zero_rhs; j++) {
    // v_j = v_0, or the previous step's orthogonalised w scaled by 1 / h_{j,j-1}.  w alternates
    // between two buffers: a CTA writes w_j while its neighbours may still read w_{j-1} for
    // their stencil rows.
    const T2* src = j == 0 ? a.V : a.w + (size_t)((j - 1) & 1) * n;
    T2* wj = a.w + (size_t)(j & 1) * n;
    const S scale = j == 0 ? (S)1 : (S)1 / s_hn;
    T2* vj = a.V + (size_t)j * n;
    if (EO) {
      // (1a) t_e = A_ee^-1 A_eo src on the own even sites (unscaled: the scale enters in 1b)
      if (ovl && warp == 0) {
        if (lane == 0 && j > 0) hessenberg_update(j - 1);
      } else {
        GM_HOP_ROWS(0, src, (S)1, swarp, snwarp, cached);
      }
      __syncthreads();                               // own rows and the previous column complete
      if (s_done) break;                             // the previous step met the stopping test
      for (int t = threadIdx.x; t < nown; t += blockDim.x) {
        const int e = GM_OWN_E(t), site = e / a.nd, k = e - site * a.nd;
        if (coarse_site_parity(a.cg, site) != 0) continue;
        T2* rw = GM_ROW_BASE(0, site) + k;
        S ar = 0, ai = 0;
        for (int d = 1; d < 9; d++) { const T2 r = rw[(size_t)d * a.nd]; ar += r.x; ai += r.y; }
        rw[0] = mk2<S>(ar, ai);                      // slot 0 of an even site: the input of A_ee^-1
      }
      __syncthreads();
      GM_INV_TASKS(GM_ROW_BASE(0, site), a.te + (size_t)site * a.nd);
      grid.sync();                                   // t_e complete
      // (1b) rows of w_o = A_oo v_o - A_oe t_e on the own odd sites, v = scale * src
      for (int t = warp; t < (s1 - s0) * 9; t += nwarp) {
        const int site = s0 + t / 9, d = t - (t / 9) * 9;
        if (coarse_site_parity(a.cg, site) != 1) continue;
        const int t9 = site * 9 + d, lb = t9 - s0 * 9;
        const T2* blk = lb < cached ? blk_sm + (size_t)lb * a.nd * a.nd : a.Dc + (size_t)t9 * a.nd * a.nd;
        const T2* xv = d == 0 ? src + (size_t)site * a.nd : a.te + (size_t)a.nbr[t9] * a.nd;
        stencil_task<S>(blk, xv, a.nd, d == 0 ? scale : -scale, nullptr, (S)0, (S)0,
                        GM_ROW_BASE(0, site) + (size_t)d * a.nd, lane);
      }
      __syncthreads();
    } else {
      if (ovl && warp == 0) {
        if (lane == 0 && j > 0) hessenberg_update(j - 1);
      } else {
        // (1) stencil products of the own sites, one warp per (flavour, site, stencil block): lanes
        //     are rows, so every column of a block is one coalesced read.  The doublet's flavour
        //     mixing is added to the self block's row.
        for (int t = swarp; t < ntask; t += snwarp) {
          const int f = t / ((s1 - s0) * 9);
          const int t9 = s0 * 9 + (t - f * (s1 - s0) * 9);
          const int site = t9 / 9;
          const int lb = t9 - s0 * 9;                // own block index
          const T2* blk = lb < cached ? blk_sm + (size_t)lb * a.nd * a.nd : a.Dc + (size_t)t9 * a.nd * a.nd;
          const T2* xv = src + (size_t)f * n1 + (size_t)a.nbr[t9] * a.nd;
          const T2* xo = (a.nf == 2 && t9 == site * 9) ? src + (size_t)(1 - f) * n1 + (size_t)site * a.nd : nullptr;
          stencil_task<S>(blk, xv, a.nd, scale, xo, a.epsbar, a.delta,
                          GM_ROW_BASE(f, site) + (size_t)(t9 - site * 9) * a.nd, lane);
        }
      }
      __syncthreads();                               // own rows and the previous column complete
      if (s_done) break;                             // the previous step met the stopping test
    }
    // (2) own elements: v_j, w = sum of the 9 partial rows + twist, then <v_i, w> partials
    for (int t = threadIdx.x; t < nown; t += blockDim.x) {
      const int e = GM_OWN_E(t);
      const int f = e / n1, e1f = e - f * n1;
      const int site = e1f / a.nd, k = e1f - site * a.nd;
      if (EO && coarse_site_parity(a.cg, site) == 0) {   // reduced system: even entries stay zero
        if (j > 0) vj[e] = mk2<S>(0, 0);
        wj[e] = mk2<S>(0, 0);
        continue;
      }
      T2 xs = src[e];
      xs.x *= scale;
      xs.y *= scale;
      if (j > 0) vj[e] = xs;
      S ar = 0, ai = 0;
      const T2* rw = GM_ROW_BASE(f, site) + k;
      for (int d = 0; d < 9; d++) { const T2 r = rw[(size_t)d * a.nd]; ar += r.x; ai += r.y; }
      const S tw = (k < a.nv) == (f == 0) ? a.mu : -a.mu;
      T2 o;
      o.x = ar - tw * xs.y;
      o.y = ai + tw * xs.x;
      wj[e] = o;
    }
    if (threadIdx.x == 0)
      for (int i = 0; i <= j + 1; i++) hcol[i] = mk2<S>(0, 0);
    __syncthreads();
    for (int pass = 0; pass < a.passes; pass++) {
      // partial <v_i, w> over the own chunk, one warp per basis vector.  Consecutive passes write
      // alternate halves of the partials: only a CTA barrier separates one pass's reads from the
      // next pass's writes, so a CTA may start pass p+1 while others still sum the partials of p.
      A2* part = part_base + (size_t)(pass & 1) * (CMAXM + 1) * G;
      for (int i = warp; i <= j; i += nwarp) {
        const T2* vi = a.V + (size_t)i * n;
        S re = 0, im = 0;
        for (int t = lane; t < nown; t += 32) {
          const int e = GM_OWN_E(t);
          const T2 p = vi[e], q = wj[e];
          re += p.x * q.x + p.y * q.y;
          im += p.x * q.y - p.y * q.x;
        }
        const S dre = warp_sum((S)re), dim = warp_sum((S)im);
        if (lane == 0) part[(size_t)i * G + blockIdx.x] = mk2<S>(dre, dim);
      }
      grid.sync();                                   // partials complete
      for (int i = warp; i <= j; i += nwarp) {
        S re = 0, im = 0;
#pragma unroll 8
        for (int q = lane; q < G; q += 32) { const A2 v = part[(size_t)i * G + q]; re += v.x; im += v.y; }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) {
          hp[i] = mk2<S>(re, im);
          hcol[i] = mk2<S>(hcol[i].x + re, hcol[i].y + im);
        }
      }
      __syncthreads();
      // w -= sum_i h_i v_i on the own chunk and, in the last pass, ||w||^2
      S nn = 0;
      for (int t = threadIdx.x; t < nown; t += blockDim.x) {
        const int e = GM_OWN_E(t);
        T2 q = wj[e];
        S qr = q.x, qi = q.y;
        #pragma unroll 4
        for (int i = 0; i <= j; i++) {
          const T2 p = a.V[(size_t)i * n + e];
          const S hr = (S)hp[i].x, hi = (S)hp[i].y;
          qr -= hr * p.x - hi * p.y;
          qi -= hr * p.y + hi * p.x;
        }
        q.x = qr;
        q.y = qi;
        wj[e] = q;
        nn += qr * qr + qi * qi;
      }
      if (pass == a.passes - 1) {
        const S t = cta_sum((S)nn, sh);
        if (threadIdx.x == 0) npart[blockIdx.x] = t;
      } else {
        __syncthreads();
      }
    }
    grid.sync();                                     // w and norm partials complete
    if (warp == 0) {
      S t = 0;
#pragma unroll 8
      for (int q = lane; q < G; q += 32) t += npart[q];
      t = warp_sum(t);
      if (lane == 0) {
        s_hn = sq(t);
        s_k = j + 1;
        // without overlap, and for the last allowed step (no following stencil to hide it behind),
        // the column update runs here
        if (!ovl || j == a.m - 1) hessenberg_update(j);
      }
    }
    __syncthreads();
    if (!ovl && s_done) break;                       // every CTA decided alike from the same values
  }
  // a step whose column update was deferred and that ended the loop by reaching m: done above;
  // a stop found after the stencil of the next step: done in that stencil phase
  grid.sync();                                       // rotated Hessenberg stored by CTA 0
  const int k = s_k;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; i--) {
      A2 acc = gv[i];
      for (int l = i + 1; l < k; l++) {
        const A2 h = Rm[(size_t)l * (CMAXM + 1) + i], yl = ym[l];
        acc.x -= h.x * yl.x - h.y * yl.y;
        acc.y -= h.x * yl.y + h.y * yl.x;
      }
      const A2 d = Rm[(size_t)i * (CMAXM + 1) + i];
      const S dn = d.x * d.x + d.y * d.y;
      ym[i] = dn > (S)0 ? mk2<S>((acc.x * d.x + acc.y * d.y) / dn, (acc.y * d.x - acc.x * d.y) / dn)
                        : mk2<S>(0, 0);
    }
    if (a.counter) *a.counter += k;
  }
  grid.sync();                                       // coefficients ready
  __shared__ S yr[CMAXM], yi[CMAXM];
  for (int i = threadIdx.x; i < k; i += blockDim.x) { yr[i] = ym[i].x; yi[i] = ym[i].y; }
  __syncthreads();
  for (int e = tid; e < n; e += nth) {
    S xr = 0, xi = 0;
    #pragma unroll 4
    for (int i = 0; i < k; i++) {
      const T2 v = a.V[(size_t)i * n + e];
      xr += yr[i] * v.x - yi[i] * v.y;
      xi += yr[i] * v.y + yi[i] * v.x;
    }
    T2 o;
    o.x = xr;
    o.y = xi;
    a.x[e] = o;
  }
  if (EO) {
    // x_e = A_ee^-1 (b_e - A_eo x_o) on the own even sites (the loop above left x_e = 0)
    grid.sync();                                     // x_o complete
    GM_HOP_ROWS(0, a.x, (S)-1, warp, nwarp, cached);
    __syncthreads();
    for (int t = threadIdx.x; t < nown; t += blockDim.x) {
      const int e = GM_OWN_E(t), site = e / a.nd, k = e - site * a.nd;
      if (coarse_site_parity(a.cg, site) != 0) continue;
      T2* rw = GM_ROW_BASE(0, site) + k;
      T2 o = a.b[e];
      for (int d = 1; d < 9; d++) { const T2 r = rw[(size_t)d * a.nd]; o.x += r.x; o.y += r.y; }
      rw[0] = o;
    }
    __syncthreads();
    GM_INV_TASKS(GM_ROW_BASE(0, site), a.x + (size_t)site * a.nd);
  }
  // a copy that missed its deadline must still land before the CTA's shared memory goes away
  if (ncache > 0 && !cached && threadIdx.x == 0) gm_bulk_wait(&s_cache_bar);
}

#undef GM_OWN_E
#undef GM_ROW_BASE
#undef GM_HOP_ROWS
#undef GM_INV_TASKS

template <typename S>
__global__ void __launch_bounds__(256, 2) k_coarse_gmres(CgArgs<S> a) {
  if (a.eo) gmres_dev<S, true>(a);
  else gmres_dev<S, false>(a);
}

// ---- third level: the level-1 K-cycle as one persistent cooperative kernel.
// FGMRES on D_c (right-preconditioned, flexible, from zero, at most kr steps) whose preconditioner
// is the level-1 cycle: z = P2 gmres_L2(P2^dag v), then z += gmres_sm(v - D_c z) (smooth_m steps).
constexpr int KMAXR = 16;

template <typename S>
struct KcArgs {
  using T2 = typename CplxT<S>::T2;
  L2Geom q;
  CgArgs<S> sm;        // level-1 operator; smoother GMRES (b = r, x = es unless mode 2)
  CgArgs<S> l2;        // level-2 operator; level-2 GMRES (b = c2, x = e2)
  const T2* W2;        // level-2 basis [nv2][nc1 nd1]
  const T2* b;
  T2* x;
  T2* V;               // FGMRES basis (kr + 1) x n1
  T2* Z;               // preconditioned vectors kr x n1
  T2* t;               // D_c z work vector
  int kr, passes, mode;
  double krtol;
  double2* part;       // [2][KMAXR + 1][G] (by pass parity)
  double* npart;       // [G]
  double2* R;          // (KMAXR + 1) x KMAXR rotated Hessenberg (CTA 0)
  double2* y;          // [KMAXR]
  int* counter;        // FGMRES steps
};

// dst = D(mu) src (sub == nullptr) or dst = sub - D(mu) src on the operator of op; grid-wide, dst
// complete after the caller's next grid barrier.
template <typename S>
__device__ void stencil_dev(const CgArgs<S>& op, const typename CplxT<S>::T2* src, typename CplxT<S>::T2* dst,
                            const typename CplxT<S>::T2* sub) {
  using T2 = typename CplxT<S>::T2;
  cg::grid_group grid = cg::this_grid();
  const int lane = threadIdx.x & 31, nwarp = blockDim.x >> 5;
  const int gwarp = blockIdx.x * nwarp + (threadIdx.x >> 5), nwarps_total = gridDim.x * nwarp;
  const int n1 = op.nc * op.nd;
  for (int task = gwarp; task < op.nf * op.nc * 9; task += nwarps_total) {
    const int f = task / (op.nc * 9), t9 = task - f * op.nc * 9;
    const int site = t9 / 9;
    const T2* blk = op.Dc + (size_t)t9 * op.nd * op.nd;
    const T2* xv = src + (size_t)f * n1 + (size_t)op.nbr[t9] * op.nd;
    const T2* xo = (op.nf == 2 && t9 == site * 9) ? src + (size_t)(1 - f) * n1 + (size_t)site * op.nd : nullptr;
    stencil_task<S>(blk, xv, op.nd, (S)1, xo, op.epsbar, op.delta, op.rows + (size_t)task * op.nd, lane);
  }
  grid.sync();
  const int n = op.nf * n1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int f = e / n1, e1f = e - f * n1;
    const int site = e1f / op.nd, k = e1f - site * op.nd;
    S ar = 0, ai = 0;
    const T2* rw = op.rows + ((size_t)(f * op.nc + site) * 9) * op.nd + k;
    for (int d = 0; d < 9; d++) { const T2 r = rw[(size_t)d * op.nd]; ar += r.x; ai += r.y; }
    const T2 xs = src[e];
    const S tw = (k < op.nv) == (f == 0) ? op.mu : -op.mu;
    ar -= tw * xs.y;
    ai += tw * xs.x;
    T2 o;
    if (sub) {
      const T2 s0 = sub[e];
      o.x = s0.x - ar;
      o.y = s0.y - ai;
    } else {
      o.x = ar;
      o.y = ai;
    }
    dst[e] = o;
  }
}

// c2 = P2^dag v (grid-wide, one thread per level-2 dof)
template <typename S>
__device__ void restrict2_dev(const L2Geom& q, const typename CplxT<S>::T2* W, const typename CplxT<S>::T2* v,
                              typename CplxT<S>::T2* c2) {
  using T2 = typename CplxT<S>::T2;
  const size_t n1 = (size_t)q.nc1 * q.nd1;
  const int nd2 = 2 * q.nv2;
  for (int o = blockIdx.x * blockDim.x + threadIdx.x; o < q.nc2 * nd2; o += gridDim.x * blockDim.x) {
    const int a2 = o / nd2, r = o - a2 * nd2, chi = r / q.nv2, j = r - chi * q.nv2;
    S re = 0, im = 0;
    for (int t = 0; t < q.avol; t++) {
      const size_t base = (size_t)l2_member(q, a2, t) * q.nd1 + chi * q.nv1;
      for (int k = 0; k < q.nv1; k++) {
        const T2 w = W[(size_t)j * n1 + base + k];
        const T2 x = v[base + k];
        re += w.x * x.x + w.y * x.y;
        im += w.x * x.y - w.y * x.x;
      }
    }
    T2 out;
    out.x = re;
    out.y = im;
    c2[o] = out;
  }
}

// z = P2 c2 (grid-wide, one thread per level-1 dof)
template <typename S>
__device__ void prolong2_dev(const L2Geom& q, const typename CplxT<S>::T2* W, const typename CplxT<S>::T2* c2,
                             typename CplxT<S>::T2* z) {
  using T2 = typename CplxT<S>::T2;
  const int n1 = q.nc1 * q.nd1;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n1; e += gridDim.x * blockDim.x) {
    const int a1 = e / q.nd1, k = e - a1 * q.nd1;
    int c[4];
    l1_coords(q, a1, c);
    const T2* cv = c2 + (size_t)l2_agg_of(q, c) * 2 * q.nv2 + (k < q.nv1 ? 0 : q.nv2);
    S re = 0, im = 0;
    for (int j = 0; j < q.nv2; j++) {
      const T2 w = W[(size_t)j * n1 + e];
      const T2 v = cv[j];
      re += w.x * v.x - w.y * v.y;
      im += w.x * v.y + w.y * v.x;
    }
    T2 out;
    out.x = re;
    out.y = im;
    z[e] = out;
  }
}

// z = level-1 cycle of v (grid-wide; z complete on return)
template <typename S>
__device__ void l1_cycle_dev(const KcArgs<S>& a, const typename CplxT<S>::T2* v, typename CplxT<S>::T2* z) {
  using T2 = typename CplxT<S>::T2;
  cg::grid_group grid = cg::this_grid();
  const size_t n1 = (size_t)a.q.nc1 * a.q.nd1, n2 = (size_t)a.q.nc2 * 2 * a.q.nv2;
  for (int f = 0; f < a.sm.nf; f++) restrict2_dev<S>(a.q, a.W2, v + f * n1, const_cast<T2*>(a.l2.b) + f * n2);
  grid.sync();
  gmres_dev(a.l2);
  grid.sync();
  for (int f = 0; f < a.sm.nf; f++) prolong2_dev<S>(a.q, a.W2, a.l2.x + f * n2, z + f * n1);
  grid.sync();
  stencil_dev(a.sm, z, const_cast<T2*>(a.sm.b), v);
  grid.sync();
  gmres_dev(a.sm);
  grid.sync();
  const int n = (int)(a.sm.nf * n1);
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    T2 o = z[e];
    const T2 d = a.sm.x[e];
    o.x += d.x;
    o.y += d.y;
    z[e] = o;
  }
  grid.sync();
}

template <typename S>
__global__ void __launch_bounds__(256) k_kcycle(KcArgs<S> a) {
  using T2 = typename CplxT<S>::T2;
  cg::grid_group grid = cg::this_grid();
  if (a.mode == 2) {              // smoother from zero
    gmres_dev(a.sm);
    return;
  }
  if (a.mode == 1) {              // one level-1 cycle
    l1_cycle_dev(a, a.b, a.x);
    return;
  }
  using A2 = T2;                  // reductions and rotations in the vectors' precision, as gmres_dev
  A2* const part_base = reinterpret_cast<A2*>(a.part);
  S* const npart = reinterpret_cast<S*>(a.npart);
  A2* const Rm = reinterpret_cast<A2*>(a.R);
  A2* const ym = reinterpret_cast<A2*>(a.y);
  __shared__ S sh[32];
  __shared__ A2 hcol[KMAXR + 2], hp[KMAXR + 1];
  __shared__ A2 cs[KMAXR], sn[KMAXR], gv[KMAXR + 1];
  __shared__ int s_done, s_k;
  __shared__ S s_beta, s_hn;
  const int n = a.sm.nf * a.q.nc1 * a.q.nd1;
  const int G = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = G * blockDim.x;
  const int chunk = (n + G - 1) / G;
  const int e0 = min(n, blockIdx.x * chunk), e1 = min(n, e0 + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  {
    S nn = 0;
    for (int e = tid; e < n; e += nth) { const T2 v = a.b[e]; nn += v.x * v.x + v.y * v.y; }
    const S t = cta_sum((S)nn, sh);
    if (threadIdx.x == 0) npart[blockIdx.x] = t;
  }
  grid.sync();
  if (warp == 0) {
    S t = 0;
    for (int q = lane; q < G; q += 32) t += npart[q];
    t = warp_sum(t);
    if (lane == 0) s_beta = sq(t);
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    s_done = !(s_beta > (S)0);
    s_k = 0;
    for (int i = 0; i <= KMAXR; i++) gv[i] = mk2<S>(0, 0);
    gv[0] = mk2<S>(s_beta, (S)0);
  }
  __syncthreads();
  {
    const S inv = s_beta > (S)0 ? (S)1 / s_beta : (S)0;
    for (int e = tid; e < n; e += nth) { T2 v = a.b[e]; v.x *= inv; v.y *= inv; a.V[e] = v; }
  }
  grid.sync();
  for (int j = 0; j < a.kr && !s_done; j++) {
    T2* vj = a.V + (size_t)j * n;
    T2* zj = a.Z + (size_t)j * n;
    l1_cycle_dev(a, vj, zj);                         // z_j = M v_j (ends with a grid barrier)
    stencil_dev(a.sm, zj, a.t, (const T2*)nullptr);  // w = D_c z_j
    grid.sync();
    if (threadIdx.x == 0)
      for (int i = 0; i <= j + 1; i++) hcol[i] = mk2<S>(0, 0);
    __syncthreads();
    for (int pass = 0; pass < a.passes; pass++) {
      A2* part = part_base + (size_t)(pass & 1) * (KMAXR + 1) * G;   // alternate halves, as in gmres_dev
      for (int i = warp; i <= j; i += nwarp) {
        const T2* vi = a.V + (size_t)i * n;
        S re = 0, im = 0;
        for (int e = e0 + lane; e < e1; e += 32) {
          const T2 p = vi[e], q = a.t[e];
          re += p.x * q.x + p.y * q.y;
          im += p.x * q.y - p.y * q.x;
        }
        const S dre = warp_sum((S)re), dim = warp_sum((S)im);
        if (lane == 0) part[(size_t)i * G + blockIdx.x] = mk2<S>(dre, dim);
      }
      grid.sync();
      for (int i = warp; i <= j; i += nwarp) {
        S re = 0, im = 0;
        for (int q = lane; q < G; q += 32) { const A2 v = part[(size_t)i * G + q]; re += v.x; im += v.y; }
        re = warp_sum(re);
        im = warp_sum(im);
        if (lane == 0) {
          hp[i] = mk2<S>(re, im);
          hcol[i] = mk2<S>(hcol[i].x + re, hcol[i].y + im);
        }
      }
      __syncthreads();
      S nn = 0;
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        T2 q = a.t[e];
        S qr = q.x, qi = q.y;
        for (int i = 0; i <= j; i++) {
          const T2 p = a.V[(size_t)i * n + e];
          const S hr = (S)hp[i].x, hi = (S)hp[i].y;
          qr -= hr * p.x - hi * p.y;
          qi -= hr * p.y + hi * p.x;
        }
        q.x = qr;
        q.y = qi;
        a.t[e] = q;
        nn += qr * qr + qi * qi;
      }
      if (pass == a.passes - 1) {
        const S t = cta_sum((S)nn, sh);
        if (threadIdx.x == 0) npart[blockIdx.x] = t;
      } else {
        __syncthreads();
      }
    }
    grid.sync();
    if (warp == 0) {
      S t = 0;
      for (int q = lane; q < G; q += 32) t += npart[q];
      t = warp_sum(t);
      if (lane == 0) s_hn = sq(t);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      const S hn = s_hn;
      hcol[j + 1] = mk2<S>(hn, (S)0);
      for (int i = 0; i < j; i++) {
        const A2 x0 = hcol[i], x1 = hcol[i + 1];
        const A2 c = cs[i], s = sn[i];
        hcol[i] = mk2<S>(c.x * x0.x + c.y * x0.y + s.x * x1.x + s.y * x1.y,
                         c.x * x0.y - c.y * x0.x + s.x * x1.y - s.y * x1.x);
        hcol[i + 1] = mk2<S>(-(s.x * x0.x - s.y * x0.y) + (c.x * x1.x - c.y * x1.y),
                             -(s.x * x0.y + s.y * x0.x) + (c.x * x1.y + c.y * x1.x));
      }
      const A2 p = hcol[j], q = hcol[j + 1];
      const S den = sq(p.x * p.x + p.y * p.y + q.x * q.x + q.y * q.y);
      cs[j] = den > (S)0 ? mk2<S>(p.x / den, p.y / den) : mk2<S>(1, 0);
      sn[j] = den > (S)0 ? mk2<S>(q.x / den, q.y / den) : mk2<S>(0, 0);
      hcol[j] = mk2<S>(den, (S)0);
      hcol[j + 1] = mk2<S>(0, 0);
      const A2 g = gv[j];
      gv[j + 1] = mk2<S>(-(sn[j].x * g.x - sn[j].y * g.y), -(sn[j].x * g.y + sn[j].y * g.x));
      gv[j] = mk2<S>(cs[j].x * g.x + cs[j].y * g.y, cs[j].x * g.y - cs[j].y * g.x);
      if (blockIdx.x == 0)
        for (int i = 0; i <= j; i++) Rm[(size_t)j * (KMAXR + 1) + i] = hcol[i];
      s_k = j + 1;
      const S res = sq(gv[j + 1].x * gv[j + 1].x + gv[j + 1].y * gv[j + 1].y);
      if (res <= (S)a.krtol * s_beta || !(hn > (S)0) || !(den > (S)0) || j == a.kr - 1) s_done = 1;
    }
    __syncthreads();
    if (!s_done) {                                   // v_{j+1} = w / h_{j+1,j} on the own chunk
      const S inv = (S)1 / s_hn;
      T2* vn = a.V + (size_t)(j + 1) * n;
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        T2 q = a.t[e];
        q.x *= inv;
        q.y *= inv;
        vn[e] = q;
      }
    }
    grid.sync();
  }
  const int k = s_k;
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int i = k - 1; i >= 0; i--) {
      A2 acc = gv[i];
      for (int l = i + 1; l < k; l++) {
        const A2 h = Rm[(size_t)l * (KMAXR + 1) + i], yl = ym[l];
        acc.x -= h.x * yl.x - h.y * yl.y;
        acc.y -= h.x * yl.y + h.y * yl.x;
      }
      const A2 d = Rm[(size_t)i * (KMAXR + 1) + i];
      const S dn = d.x * d.x + d.y * d.y;
      ym[i] = dn > (S)0 ? mk2<S>((acc.x * d.x + acc.y * d.y) / dn, (acc.y * d.x - acc.x * d.y) / dn)
                        : mk2<S>(0, 0);
    }
    if (a.counter) *a.counter += k;
  }
  grid.sync();
  __shared__ S yr[KMAXR], yi[KMAXR];
  for (int i = threadIdx.x; i < k; i += blockDim.x) { yr[i] = ym[i].x; yi[i] = ym[i].y; }
  __syncthreads();
  for (int e = tid; e < n; e += nth) {
    S xr = 0, xi = 0;
    for (int i = 0; i < k; i++) {
      const T2 v = a.Z[(size_t)i * n + e];
      xr += yr[i] * v.x - yi[i] * v.y;
      xi += yr[i] * v.y + yi[i] * v.x;
    }
    T2 o;
    o.x = xr;
    o.y = xi;
    a.x[e] = o;
  }
}

// ---- batched version: ncol right-hand sides (each with its own twist) in lock-step.  Every
// stencil block is read once per group of 4 columns; Gram-Schmidt, Givens rotations and the
// stopping test are per column.  The loop ends when every column has converged (or after m steps).
// Layout: vectors [col][n]; basis V[i][col][n]; rows [col][nc * 9][nd].
constexpr int CB = 4;   // columns per register group in the stencil products
constexpr int BMAXC = 32;

struct CgbArgs {
  int nd, nv, nc, m, ncol;
  const float2* Dc;
  const int* nbr;
  const float2* b;
  float2* x;
  float2* V;
  float2* w;
  float2* rows;
  const float* mu;       // [ncol]
  float rtol;
  float2* part;          // [ncol][CMAXM + 1][G]
  float* npart;          // [ncol][G]
  float2* R;             // [ncol][(CMAXM + 1) * CMAXM]
  float2* y;             // [ncol][CMAXM]
  int* counter;
};

__global__ void __launch_bounds__(256) k_coarse_gmres_batched(CgbArgs a) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ float2 bsm[];
  // per column: cs[CMAXM], sn[CMAXM], gv[CMAXM + 1], hcol[CMAXM + 2], hp[CMAXM + 1]
  const int per = 5 * CMAXM + 4;
  __shared__ float sh[32];
  __shared__ float s_beta[BMAXC], s_hn[BMAXC];
  __shared__ int s_done[BMAXC], s_k[BMAXC], s_all;
  const int n = a.nc * a.nd;
  const int G = gridDim.x;
  const int tid = blockIdx.x * blockDim.x + threadIdx.x, nth = G * blockDim.x;
  const int chunk = (n + G - 1) / G;
  const int e0 = min(n, blockIdx.x * chunk), e1 = min(n, e0 + chunk);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int gwarp = blockIdx.x * nwarp + warp, nwarps_total = G * nwarp;
  const size_t cn = (size_t)a.ncol * n;   // stride of one basis index
  auto CS = [&](int c) { return bsm + (size_t)c * per; };
  auto SN = [&](int c) { return bsm + (size_t)c * per + CMAXM; };
  auto GV = [&](int c) { return bsm + (size_t)c * per + 2 * CMAXM; };
  auto HC = [&](int c) { return bsm + (size_t)c * per + 3 * CMAXM + 1; };
  auto HP = [&](int c) { return bsm + (size_t)c * per + 4 * CMAXM + 3; };

  for (int c = 0; c < a.ncol; c++) {
    float nn = 0;
    for (int e = tid; e < n; e += nth) { const float2 v = a.b[(size_t)c * n + e]; nn += v.x * v.x + v.y * v.y; }
    const float t = cta_sum(nn, sh);
    if (threadIdx.x == 0) a.npart[(size_t)c * G + blockIdx.x] = t;
  }
  grid.sync();
  for (int c = warp; c < a.ncol; c += nwarp) {
    float t = 0.f;
    for (int q = lane; q < G; q += 32) t += a.npart[(size_t)c * G + q];
    t = warp_sum(t);
    if (lane == 0) {
      s_beta[c] = sqrtf(t);
      s_done[c] = !(s_beta[c] > 0.f);
      s_k[c] = 0;
      s_hn[c] = 1.f;
      float2* gv = GV(c);
      for (int i = 0; i <= CMAXM; i++) gv[i] = make_float2(0.f, 0.f);
      gv[0] = make_float2(s_beta[c], 0.f);
    }
  }
  __syncthreads();
  for (int c = 0; c < a.ncol; c++) {
    const float inv = s_beta[c] > 0.f ? 1.f / s_beta[c] : 0.f;
    for (int e = tid; e < n; e += nth) {
      float2 v = a.b[(size_t)c * n + e];
      v.x *= inv;
      v.y *= inv;
      a.V[(size_t)c * n + e] = v;
    }
  }
  if (threadIdx.x == 0) {
    int all = 1;
    for (int c = 0; c < a.ncol; c++) all &= s_done[c];
    s_all = all;
  }
  grid.sync();
  for (int j = 0; j < a.m && !s_all; j++) {
    const float2* src = j == 0 ? a.V : a.w;
    float2* vj = a.V + (size_t)j * cn;
    // (1) stencil products for all columns: warp per (site, block), columns in groups of CB
    for (int task = gwarp; task < a.nc * 9; task += nwarps_total) {
      const int nb = a.nbr[task];
      const float2* blk = a.Dc + (size_t)task * a.nd * a.nd;
      for (int c0 = 0; c0 < a.ncol; c0 += CB) {
        float sc[CB];
#pragma unroll
        for (int q = 0; q < CB; q++) sc[q] = (c0 + q < a.ncol && j > 0) ? 1.f / s_hn[c0 + q] : 1.f;
        for (int k = lane; k < a.nd; k += 32) {
          float ar[CB], ai[CB];
#pragma unroll
          for (int q = 0; q < CB; q++) { ar[q] = 0.f; ai[q] = 0.f; }
#pragma unroll 4
          for (int l = 0; l < a.nd; l++) {
            const float2 m = blk[(size_t)l * a.nd + k];
#pragma unroll
            for (int q = 0; q < CB; q++) {
              if (c0 + q < a.ncol) {
                const float2 v = src[(size_t)(c0 + q) * n + (size_t)nb * a.nd + l];
                ar[q] += m.x * v.x - m.y * v.y;
                ai[q] += m.x * v.y + m.y * v.x;
              }
            }
          }
#pragma unroll
          for (int q = 0; q < CB; q++)
            if (c0 + q < a.ncol)
              a.rows[((size_t)(c0 + q) * a.nc * 9 + task) * a.nd + k] = make_float2(ar[q] * sc[q], ai[q] * sc[q]);
        }
      }
    }
    grid.sync();
    // (2) own chunk: v_j, w = sum of rows + twist, per column
    for (int c = 0; c < a.ncol; c++) {
      const float scale = j == 0 ? 1.f : 1.f / s_hn[c];
      const float mu = a.mu[c];
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        const int site = e / a.nd, k = e - site * a.nd;
        float2 xs = src[(size_t)c * n + e];
        xs.x *= scale;
        xs.y *= scale;
        if (j > 0) vj[(size_t)c * n + e] = xs;
        float ar = 0.f, ai = 0.f;
        for (int d = 0; d < 9; d++) {
          const float2 r = a.rows[((size_t)c * a.nc * 9 + (size_t)site * 9 + d) * a.nd + k];
          ar += r.x;
          ai += r.y;
        }
        const float tw = k < a.nv ? mu : -mu;
        a.w[(size_t)c * n + e] = make_float2(ar - tw * xs.y, ai + tw * xs.x);
      }
    }
    for (int c = threadIdx.x; c < a.ncol; c += blockDim.x)
      for (int i = 0; i <= j + 1; i++) HC(c)[i] = make_float2(0.f, 0.f);
    __syncthreads();
    // (3) dots <v_i, w> per column, partials per CTA
    for (int t = warp; t < (j + 1) * a.ncol; t += nwarp) {
      const int i = t / a.ncol, c = t - i * a.ncol;
      const float2* vi = a.V + (size_t)i * cn + (size_t)c * n;
      const float2* wc = a.w + (size_t)c * n;
      float re = 0.f, im = 0.f;
      for (int e = e0 + lane; e < e1; e += 32) {
        const float2 p = vi[e], q = wc[e];
        re += p.x * q.x + p.y * q.y;
        im += p.x * q.y - p.y * q.x;
      }
      const float dre = warp_sum(re), dim = warp_sum(im);
      if (lane == 0) a.part[((size_t)c * (CMAXM + 1) + i) * G + blockIdx.x] = make_float2(dre, dim);
    }
    grid.sync();
    for (int t = warp; t < (j + 1) * a.ncol; t += nwarp) {
      const int i = t / a.ncol, c = t - i * a.ncol;
      float re = 0.f, im = 0.f;
      for (int q = lane; q < G; q += 32) {
        const float2 v = a.part[((size_t)c * (CMAXM + 1) + i) * G + q];
        re += v.x;
        im += v.y;
      }
      re = warp_sum(re);
      im = warp_sum(im);
      if (lane == 0) {
        HP(c)[i] = make_float2(re, im);
        HC(c)[i] = make_float2(HC(c)[i].x + re, HC(c)[i].y + im);
      }
    }
    __syncthreads();
    // (4) update and norms on the own chunk
    for (int c = 0; c < a.ncol; c++) {
      float nn = 0.f;
      const float2* hp = HP(c);
      for (int e = e0 + threadIdx.x; e < e1; e += blockDim.x) {
        float2 q = a.w[(size_t)c * n + e];
        for (int i = 0; i <= j; i++) {
          const float2 p = a.V[(size_t)i * cn + (size_t)c * n + e];
          const float hr = (float)hp[i].x, hi = (float)hp[i].y;
          q.x -= hr * p.x - hi * p.y;
          q.y -= hr * p.y + hi * p.x;
        }
        a.w[(size_t)c * n + e] = q;
        nn += q.x * q.x + q.y * q.y;
      }
      const float t = cta_sum(nn, sh);
      if (threadIdx.x == 0) a.npart[(size_t)c * G + blockIdx.x] = t;
    }
    grid.sync();
    // (5) per column: norm, Givens, stopping test (one warp per column)
    for (int c = warp; c < a.ncol; c += nwarp) {
      float t = 0.f;
      for (int q = lane; q < G; q += 32) t += a.npart[(size_t)c * G + q];
      t = warp_sum(t);
      if (lane == 0 && !s_done[c]) {
        const float hn = sqrtf(t);
        s_hn[c] = hn > 0.f ? hn : 1.f;   // a broken-down column is finished; keep its scale finite
        float2* hcol = HC(c);
        float2* cs = CS(c);
        float2* sn = SN(c);
        float2* gv = GV(c);
        hcol[j + 1] = make_float2(hn, 0.f);
        for (int i = 0; i < j; i++) {
          const float2 x0 = hcol[i], x1 = hcol[i + 1];
          const float2 cc = cs[i], ss = sn[i];
          hcol[i] = make_float2(cc.x * x0.x + cc.y * x0.y + ss.x * x1.x + ss.y * x1.y,
                                 cc.x * x0.y - cc.y * x0.x + ss.x * x1.y - ss.y * x1.x);
          hcol[i + 1] = make_float2(-(ss.x * x0.x - ss.y * x0.y) + (cc.x * x1.x - cc.y * x1.y),
                                     -(ss.x * x0.y + ss.y * x0.x) + (cc.x * x1.y + cc.y * x1.x));
        }
        const float2 p = hcol[j], q = hcol[j + 1];
        const float den = sqrtf(p.x * p.x + p.y * p.y + q.x * q.x + q.y * q.y);
        cs[j] = den > 0.f ? make_float2(p.x / den, p.y / den) : make_float2(1.f, 0.f);
        sn[j] = den > 0.f ? make_float2(q.x / den, q.y / den) : make_float2(0.f, 0.f);
        hcol[j] = make_float2(den, 0.f);
        const float2 g = gv[j];
        gv[j + 1] = make_float2(-(sn[j].x * g.x - sn[j].y * g.y), -(sn[j].x * g.y + sn[j].y * g.x));
        gv[j] = make_float2(cs[j].x * g.x + cs[j].y * g.y, cs[j].x * g.y - cs[j].y * g.x);
        if (blockIdx.x == 0)
          for (int i = 0; i <= j; i++) a.R[(size_t)c * (CMAXM + 1) * CMAXM + (size_t)j * (CMAXM + 1) + i] = hcol[i];
        s_k[c] = j + 1;
        const float res = sqrtf(gv[j + 1].x * gv[j + 1].x + gv[j + 1].y * gv[j + 1].y);
        if (res <= (float)a.rtol * s_beta[c] || !(hn > 0.f) || !(den > 0.f)) s_done[c] = 1;
      } else if (lane == 0) {
        s_hn[c] = s_hn[c] > 0.f ? s_hn[c] : 1.f;   // a finished column keeps a harmless scale
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int all = 1;
      for (int c = 0; c < a.ncol; c++) all &= s_done[c];
      s_all = all || (j == a.m - 1);
    }
    __syncthreads();
  }
  grid.sync();
  if (blockIdx.x == 0) {
    for (int c = warp; c < a.ncol; c += nwarp) {
      if (lane != 0) continue;
      const int k = s_k[c];
      const float2* R = a.R + (size_t)c * (CMAXM + 1) * CMAXM;
      float2* y = a.y + (size_t)c * CMAXM;
      const float2* gv = GV(c);
      for (int i = k - 1; i >= 0; i--) {
        float2 acc = gv[i];
        for (int l = i + 1; l < k; l++) {
          const float2 h = R[(size_t)l * (CMAXM + 1) + i], yl = y[l];
          acc.x -= h.x * yl.x - h.y * yl.y;
          acc.y -= h.x * yl.y + h.y * yl.x;
        }
        const float2 d = R[(size_t)i * (CMAXM + 1) + i];
        const float dn = d.x * d.x + d.y * d.y;
        y[i] = dn > 0.f ? make_float2((acc.x * d.x + acc.y * d.y) / dn, (acc.y * d.x - acc.x * d.y) / dn)
                        : make_float2(0.f, 0.f);
      }
      if (a.counter) atomicAdd(a.counter, k);
    }
  }
  grid.sync();
  for (int c = 0; c < a.ncol; c++) {
    const int k = s_k[c];
    const float2* y = a.y + (size_t)c * CMAXM;
    for (int e = tid; e < n; e += nth) {
      float xr = 0.f, xi = 0.f;
      for (int i = 0; i < k; i++) {
        const float2 v = a.V[(size_t)i * cn + (size_t)c * n + e];
        const float yr = (float)y[i].x, yi = (float)y[i].y;
        xr += yr * v.x - yi * v.y;
        xi += yr * v.y + yi * v.x;
      }
      a.x[(size_t)c * n + e] = make_float2(xr, xi);
    }
  }
}

// CTAs of the persistent coarse GMRES: the "coarse_grid" knob if set, else "coarse_ctas_per_sm" per
// SM (at most one CTA per coarse site), both capped by the kernel's residency.  The allocating and
// the allocation-free launch both size their grid here, so they reduce in the same order.
// (A_self(a) + i mu G5_c)^-1 for every coarse site a, by Gauss-Jordan elimination with partial
// pivoting on the augmented matrix [A | I] in shared memory, one CTA per site; the result is stored
// like a stencil block (element (k, l) at l * nd + k).
template <typename S>
__global__ void __launch_bounds__(256) k_coarse_site_inverse(int nd, int nv, const typename CplxT<S>::T2* __restrict__ Dc,
                                                             S mu, typename CplxT<S>::T2* __restrict__ inv) {
  using T2 = typename CplxT<S>::T2;
  extern __shared__ __align__(16) unsigned char sinv_raw[];
  T2* const m = reinterpret_cast<T2*>(sinv_raw);   // [nd][2 nd], row-major
  T2* const fac = m + (size_t)nd * 2 * nd;          // [nd] elimination factors of the current column
  __shared__ int s_piv;
  const int w2 = 2 * nd;
  const T2* blk = Dc + (size_t)blockIdx.x * 9 * nd * nd;   // slot 0: the site's own block
  for (int q = threadIdx.x; q < nd * w2; q += blockDim.x) {
    const int r = q / w2, cc = q - r * w2;
    T2 v = mk2<S>(0, 0);
    if (cc < nd) {
      v = blk[(size_t)cc * nd + r];
      if (cc == r) v.y += r < nv ? mu : -mu;
    } else if (cc - nd == r) {
      v = mk2<S>(1, 0);
    }
    m[q] = v;
  }
  __syncthreads();
  for (int p = 0; p < nd; p++) {
    if (threadIdx.x == 0) {
      int best = p;
      S bv = m[(size_t)p * w2 + p].x * m[(size_t)p * w2 + p].x + m[(size_t)p * w2 + p].y * m[(size_t)p * w2 + p].y;
      for (int r = p + 1; r < nd; r++) {
        const T2 v = m[(size_t)r * w2 + p];
        const S a2 = v.x * v.x + v.y * v.y;
        if (a2 > bv) { bv = a2; best = r; }
      }
      s_piv = best;
    }
    __syncthreads();
    const int pr = s_piv;
    if (pr != p)
      for (int cc = threadIdx.x; cc < w2; cc += blockDim.x) {
        const T2 t = m[(size_t)p * w2 + cc];
        m[(size_t)p * w2 + cc] = m[(size_t)pr * w2 + cc];
        m[(size_t)pr * w2 + cc] = t;
      }
    __syncthreads();
    const T2 d = m[(size_t)p * w2 + p];
    const S dn = d.x * d.x + d.y * d.y;
    const T2 di = mk2<S>(d.x / dn, -d.y / dn);
    for (int r = threadIdx.x; r < nd; r += blockDim.x) fac[r] = m[(size_t)r * w2 + p];
    __syncthreads();
    for (int cc = threadIdx.x; cc < w2; cc += blockDim.x) {
      const T2 v = m[(size_t)p * w2 + cc];
      m[(size_t)p * w2 + cc] = mk2<S>(v.x * di.x - v.y * di.y, v.x * di.y + v.y * di.x);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < nd * w2; q += blockDim.x) {
      const int r = q / w2, cc = q - r * w2;
      if (r == p) continue;
      const T2 f = fac[r], v = m[(size_t)p * w2 + cc];
      T2 o = m[q];
      o.x -= f.x * v.x - f.y * v.y;
      o.y -= f.x * v.y + f.y * v.x;
      m[q] = o;
    }
    __syncthreads();
  }
  T2* out = inv + (size_t)blockIdx.x * nd * nd;
  for (int q = threadIdx.x; q < nd * nd; q += blockDim.x) {
    const int l = q / nd, k = q - l * nd;          // column l, row k
    out[q] = m[(size_t)k * w2 + nd + l];
  }
}

// The per-site inverses for mu in precision S, computed on first use and kept in one of the
// context's slots (least recently used slot reused; the cycle graphs, which may point at it, are
// dropped when a used slot is overwritten).
template <typename S>
const typename CplxT<S>::T2* site_inverse(Ctx& c, double mu) {
  using T2 = typename CplxT<S>::T2;
  const int prec = sizeof(S) == 8 ? TMG_PREC_F64 : TMG_PREC_F32;
  SiteInverse* pick = nullptr;
  for (auto& e : c.site_inv)
    if (e.used && e.mu == mu && e.prec == prec && e.version == c.cl.version) {
      e.stamp = ++c.site_inv_clock;
      return e.buf.as<T2>();
    }
  for (auto& e : c.site_inv)
    if (!pick || !e.used || (pick->used && e.stamp < pick->stamp)) {
      pick = &e;
      if (!e.used) break;
    }
  if (pick->used) c.graphs.clear();
  const int nd = c.cl.nd;
  pick->buf.alloc((size_t)c.cl.nc * nd * nd * sizeof(T2));
  const size_t smem = sizeof(T2) * ((size_t)nd * 2 * nd + nd);
  if (smem > 48 * 1024)
    TMG_CUDA(cudaFuncSetAttribute(k_coarse_site_inverse<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const T2* Dc = (const T2*)(sizeof(S) == 8 ? c.cl.Dc64.p : c.cl.Dc32.p);
  ++c.launches;
  k_coarse_site_inverse<S><<<c.cl.nc, 256, smem, c.stream>>>(nd, c.cl.nv, Dc, (S)mu, pick->buf.as<T2>());
  TMG_CHECK_LAUNCH();
  pick->used = true;
  pick->mu = mu;
  pick->prec = prec;
  pick->version = c.cl.version;
  pick->stamp = ++c.site_inv_clock;
  return pick->buf.as<T2>();
}

// Whether the odd-even coarse solve applies: asked for, one flavour, every coarse extent even.
inline bool coarse_eo_on(const Ctx& c, int nf) {
  if (!c.coarse_eo || nf != 1) return false;
  for (int mu = 0; mu < 4; mu++)
    if (c.cl.cgeom[mu] % 2) return false;
  return true;
}

template <typename S>
int coarse_grid_ctas(Ctx& c) {
  static int max_per_sm[2] = {-1, -1};
  int& mps = max_per_sm[sizeof(S) == 8];
  if (mps < 0) TMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mps, k_coarse_gmres<S>, 256, 0));
  return c.coarse_grid > 0 ? std::max(1, std::min(c.coarse_grid, c.sms * std::max(1, mps)))
                           : std::max(1, std::min(c.cl.nc, c.sms * std::max(1, std::min(mps, c.coarse_ctas_per_sm))));
}

// Dynamic shared memory for the own sites' stencil rows of a grid of G CTAs, or 0 when they do not
// fit (above 48 KB, or too large for every CTA of the grid to stay resident): then they go to the
// global rows buffer.
template <typename S>
size_t rows_smem_bytes(Ctx& c, int G, int nf) {
  using T2 = typename CplxT<S>::T2;
  const size_t per_cta = (size_t)((c.cl.nc + G - 1) / G) * nf * 9 * c.cl.nd * sizeof(T2);
  if (per_cta > 48 * 1024) return 0;
  static size_t cached_bytes[2] = {(size_t)-1, (size_t)-1};
  static int cached_mps[2] = {0, 0};
  const int t = sizeof(S) == 8;
  if (cached_bytes[t] != per_cta) {
    TMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&cached_mps[t], k_coarse_gmres<S>, 256, per_cta));
    cached_bytes[t] = per_cta;
  }
  return (size_t)cached_mps[t] * c.sms >= (size_t)G ? per_cta : 0;
}

// Shared-memory layout of a coarse GMRES launch of G CTAs: the own sites' stencil rows (when they
// fit), then as many of the own stencil blocks as the CTAs that share an SM leave room for.
template <typename S>
size_t coarse_smem_layout(Ctx& c, int G, int nf, CgArgs<S>& a) {
  using T2 = typename CplxT<S>::T2;
  const size_t rows = rows_smem_bytes<S>(c, G, nf);
  auto al = [](size_t v) { return (v + 127) & ~(size_t)127; };
  a.rows_smem = rows > 0;
  a.blk_cache = 0;
  const int per_sm = (G + c.sms - 1) / c.sms;
  static int cached_per_sm[2] = {-1, -1};
  static size_t cached_avail[2] = {0, 0};
  const int t = sizeof(S) == 8;
  if (cached_per_sm[t] != per_sm) {
    size_t avail = 0;
    TMG_CUDA(cudaOccupancyAvailableDynamicSMemPerBlock(&avail, k_coarse_gmres<S>, per_sm, 256));
    cached_avail[t] = avail;
    cached_per_sm[t] = per_sm;
    TMG_CUDA(cudaFuncSetAttribute(k_coarse_gmres<S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)avail));
  }
  const size_t avail = cached_avail[t];
  const size_t off = al(rows);
  a.cache_off = (int)off;
  const size_t blk_bytes = (size_t)c.cl.nd * c.cl.nd * sizeof(T2);
  if (!c.coarse_block_cache || avail <= off + blk_bytes) return rows;
  const int own_max = ((c.cl.nc + G - 1) / G) * 9;
  a.blk_cache = (int)std::min<size_t>((size_t)own_max, (avail - off) / blk_bytes);
  return off + (size_t)a.blk_cache * blk_bytes;
}

template <typename S>
void launch(Ctx& c, const void* b, void* x, double mu, const void* Dc, int nf = 1, double epsbar = 0.0) {
  using T2 = typename CplxT<S>::T2;
  const int m = std::min(c.mg.coarse_m, CMAXM);
  const size_t n = (size_t)nf * c.cl.nc * c.cl.nd;
  const int G = coarse_grid_ctas<S>(c);
  c.cw_V.alloc((m + 1) * n * sizeof(T2));
  c.cw_w.alloc(13 * n * sizeof(T2));   // w (two buffers), 9 rows, odd-even intermediate and right-hand side
  c.cw_part.alloc(sizeof(double2) * ((size_t)2 * (CMAXM + 1) * G + (CMAXM + 1) * CMAXM + CMAXM) + sizeof(double) * G);
  if (!c.coarse_iter_dev.p) {
    c.coarse_iter_dev.alloc(sizeof(int));
    TMG_CUDA(cudaMemsetAsync(c.coarse_iter_dev.p, 0, sizeof(int), c.stream));
  }
  CgArgs<S> a;
  a.nd = c.cl.nd;
  a.nv = c.cl.nv;
  a.nc = c.cl.nc;
  a.m = m;
  a.nf = nf;
  a.epsbar = (S)epsbar;
  a.delta = nf == 2 ? (S)c.ndshift : (S)0;
  a.overlap = c.coarse_overlap;
  const size_t smem = coarse_smem_layout<S>(c, G, nf, a);
  a.passes = c.coarse_gs_passes > 0 ? c.coarse_gs_passes : (sizeof(S) == 4 ? 1 : 2);
  a.Dc = (const T2*)Dc;
  a.nbr = c.cl.nbr.as<int>();
  a.b = (const T2*)b;
  a.x = (T2*)x;
  a.V = c.cw_V.as<T2>();
  a.w = c.cw_w.as<T2>();
  a.rows = a.w + 2 * n;
  a.te = a.w + 11 * n;
  a.rb = a.w + 12 * n;
  a.eo = coarse_eo_on(c, nf);
  for (int q = 0; q < 4; q++) a.cg[q] = c.cl.cgeom[q];
  a.inv = a.eo ? site_inverse<S>(c, mu) : nullptr;
  a.mu = (S)mu;
  a.rtol = c.mg.coarse_rtol;
  a.part = c.cw_part.as<double2>();
  a.R = a.part + (size_t)2 * (CMAXM + 1) * G;
  a.y = a.R + (size_t)(CMAXM + 1) * CMAXM;
  a.npart = reinterpret_cast<double*>(a.y + CMAXM);
  a.counter = c.coarse_iter_dev.as<int>();
  void* args[] = {&a};
  ++c.launches;
  TMG_CUDA(cudaLaunchCooperativeKernel((const void*)k_coarse_gmres<S>, dim3(G), dim3(256), args, smem, c.stream));
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

// Scratch layout used by coarse_gmres_on_scratch: basis V, the two w buffers and the 9 partial stencil rows, dot partials, R, y, norm partials,
// step counter, each 256-byte aligned.
template <typename S>
size_t scratch_layout(const Ctx& c, int G, size_t off[8]) {
  using T2 = typename CplxT<S>::T2;
  const int m = std::min(c.mg.coarse_m, CMAXM);
  const size_t n = (size_t)c.cl.nc * c.cl.nd;
  const size_t sz[7] = {(m + 1) * n * sizeof(T2), 11 * n * sizeof(T2), sizeof(double2) * 2 * (CMAXM + 1) * G,
                        sizeof(double2) * (CMAXM + 1) * CMAXM, sizeof(double2) * CMAXM, sizeof(double) * G, sizeof(int)};
  size_t o = 0;
  for (int i = 0; i < 7; i++) {
    off[i] = o;
    o = align256(o + sz[i]);
  }
  off[7] = o;
  return o;
}

template <typename S>
void launch_on(Ctx& c, const void* b, void* x, double mu, const void* Dc, char* scratch, int G) {
  using T2 = typename CplxT<S>::T2;
  size_t off[8];
  scratch_layout<S>(c, G, off);
  CgArgs<S> a;
  a.nd = c.cl.nd;
  a.nv = c.cl.nv;
  a.nc = c.cl.nc;
  a.m = std::min(c.mg.coarse_m, CMAXM);
  a.nf = 1;
  a.epsbar = (S)0;
  a.delta = (S)0;
  a.overlap = c.coarse_overlap;
  const size_t smem = coarse_smem_layout<S>(c, G, 1, a);
  a.passes = c.coarse_gs_passes > 0 ? c.coarse_gs_passes : (sizeof(S) == 4 ? 1 : 2);
  a.Dc = (const T2*)Dc;
  a.nbr = c.cl.nbr.as<int>();
  a.b = (const T2*)b;
  a.x = (T2*)x;
  a.V = (T2*)(scratch + off[0]);
  a.w = (T2*)(scratch + off[1]);
  a.rows = a.w + 2 * (size_t)c.cl.nc * c.cl.nd;
  a.eo = 0;                          // the allocation-free call keeps the plain form
  for (int q = 0; q < 4; q++) a.cg[q] = c.cl.cgeom[q];
  a.inv = nullptr;
  a.te = a.rb = nullptr;
  a.part = (double2*)(scratch + off[2]);
  a.R = (double2*)(scratch + off[3]);
  a.y = (double2*)(scratch + off[4]);
  a.npart = (double*)(scratch + off[5]);
  a.counter = (int*)(scratch + off[6]);
  a.mu = (S)mu;
  a.rtol = c.mg.coarse_rtol;
  TMG_CUDA(cudaMemsetAsync(a.counter, 0, sizeof(int), c.stream));   // the shared scratch keeps old contents
  void* args[] = {&a};
  ++c.launches;
  TMG_CUDA(cudaLaunchCooperativeKernel((const void*)k_coarse_gmres<S>, dim3(G), dim3(256), args, smem, c.stream));
}

}  // namespace

size_t coarse_gmres_scratch_bytes(Ctx& c, int cp) {
  size_t off[8];
  if (cp == TMG_PREC_F64) return scratch_layout<double>(c, coarse_grid_ctas<double>(c), off);
  return scratch_layout<float>(c, coarse_grid_ctas<float>(c), off);
}

void coarse_gmres_on_scratch(Ctx& c, int cp, const void* b, void* x, double mu, void* scratch) {
  if (cp == TMG_PREC_F64) launch_on<double>(c, b, x, mu, c.cl.Dc64.p, (char*)scratch, coarse_grid_ctas<double>(c));
  else launch_on<float>(c, b, x, mu, c.cl.Dc32.p, (char*)scratch, coarse_grid_ctas<float>(c));
}

void coarse_gmres_batched(Ctx& c, int ncol, const void* b, void* x, const float* mu_dev) {
  ProfScope ps(c, PK_COARSE_SOLVE);
  const int m = std::min(c.batched_coarse_m > 0 ? c.batched_coarse_m : c.mg.coarse_m, CMAXM);
  const size_t n = (size_t)c.cl.nc * c.cl.nd;
  const size_t smem = sizeof(float2) * (size_t)ncol * (5 * CMAXM + 4);
  if (smem > 48 * 1024)
    TMG_CUDA(cudaFuncSetAttribute(k_coarse_gmres_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int mps = 0;
  TMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mps, k_coarse_gmres_batched, 256, smem));
  if (mps < 1) throw Error{TMG_ERR_ARG, "batched coarse solve: too many columns for one CTA's shared memory"};
  const int G = std::max(1, std::min(c.cl.nc, c.sms * std::min(mps, 2)));
  c.cw_V.alloc((m + 1) * n * ncol * sizeof(float2));
  c.cw_w.alloc(10 * n * ncol * sizeof(float2));
  c.cw_part.alloc(sizeof(double2) * ((size_t)ncol * (CMAXM + 1) * G + (size_t)ncol * (CMAXM + 1) * CMAXM +
                                     (size_t)ncol * CMAXM) + sizeof(double) * (size_t)ncol * G);
  if (!c.coarse_iter_dev.p) {
    c.coarse_iter_dev.alloc(sizeof(int));
    TMG_CUDA(cudaMemsetAsync(c.coarse_iter_dev.p, 0, sizeof(int), c.stream));
  }
  CgbArgs a;
  a.nd = c.cl.nd;
  a.nv = c.cl.nv;
  a.nc = c.cl.nc;
  a.m = m;
  a.ncol = ncol;
  a.Dc = c.cl.Dc32.as<float2>();
  a.nbr = c.cl.nbr.as<int>();
  a.b = (const float2*)b;
  a.x = (float2*)x;
  a.V = c.cw_V.as<float2>();
  a.w = c.cw_w.as<float2>();
  a.rows = a.w + n * ncol;
  a.mu = mu_dev;
  a.rtol = c.mg.coarse_rtol;
  a.part = c.cw_part.as<float2>();
  a.R = a.part + (size_t)ncol * (CMAXM + 1) * G;
  a.y = a.R + (size_t)ncol * (CMAXM + 1) * CMAXM;
  a.npart = reinterpret_cast<float*>(a.y + (size_t)ncol * CMAXM);
  a.counter = c.coarse_iter_dev.as<int>();
  void* args[] = {&a};
  ++c.launches;
  TMG_CUDA(cudaLaunchCooperativeKernel((const void*)k_coarse_gmres_batched, dim3(G), dim3(256), args, smem, c.stream));
}

void coarse_gmres_persistent(Ctx& c, int cp, const void* b, void* x, double mu) {
  ProfScope ps(c, PK_COARSE_SOLVE);
  if (cp == TMG_PREC_F64) launch<double>(c, b, x, mu, c.cl.Dc64.p);
  else launch<float>(c, b, x, mu, c.cl.Dc32.p);
}

void coarse_gmres_persistent_nd(Ctx& c, int cp, const void* b, void* x) {
  ProfScope ps(c, PK_COARSE_SOLVE);
  if (cp == TMG_PREC_F64) launch<double>(c, b, x, c.mubar, c.cl.Dc64.p, 2, c.epsbar);
  else launch<float>(c, b, x, c.mubar, c.cl.Dc32.p, 2, c.epsbar);
}

namespace {

// ---- batched coarse GMRES with the stencil on the tensor cores.  Each Arnoldi step is two
// launches: the tcgen05 multi-RHS coarse operator W = D_c(mu_col) V_j for all columns (every
// stencil block is read once per step for all columns), then one cooperative kernel that
// orthogonalises W against V_0..V_j per column (three grid barriers: per-CTA dot partials, their
// totals reduced once across the grid, the norms), writes V_{j+1} and, on CTA 0,
// advances every unfinished column's Givens rotations and stopping test.  The rotations live in
// global memory between launches; once every column has stopped, the remaining launches of the
// step sequence return at once (a flag both kernels read on entry).  Same arithmetic as
// k_coarse_gmres_batched: one classical Gram-Schmidt pass, FP32 vectors, FP64 reductions.
struct BgtArgs {
  int nd, nv, nc, m, ncol;
  const float2* b;
  float2* x;
  float2* V;             // [(m + 1)][ncol][n]
  float2* W;             // [ncol][n]
  float rtol;
  float2* part;          // [ncol][CMAXM + 1][G]
  float* npart;          // [ncol][G]
  float2* cs;            // [ncol][CMAXM]
  float2* sn;            // [ncol][CMAXM]
  float2* gv;            // [ncol][CMAXM + 1]
  float2* R;             // [ncol][(CMAXM + 1) * CMAXM]
  float2* y;             // [ncol][CMAXM]
  float2* htot;          // [ncol][CMAXM + 1] Gram-Schmidt coefficients of the current step
  float* beta;           // [ncol]
  int* done;             // [ncol]
  int* kk;               // [ncol]: Krylov dimension reached
  int* all_done;
  int* counter;
  const int* skip_outer; // an enclosing solve's all-done flag (or null): every launch returns at once
};

// Lane l of the warp ends with the warp sum of v[l] (a butterfly over the five lane bits: at bit O
// each lane keeps one half of its values and adds the partner's copy of the same half).
template <int O>
__device__ __forceinline__ void transpose_sum_level(float (&v)[32], int lane) {
  const bool upper = (lane & O) != 0;
#pragma unroll
  for (int i = 0; i < O; i++) {
    const float mine = upper ? v[i + O] : v[i];
    const float other = upper ? v[i] : v[i + O];
    v[i] = mine + __shfl_xor_sync(0xffffffffu, other, O);
  }
}
__device__ __forceinline__ void warp_transpose_sum(float (&v)[32], int lane) {
  transpose_sum_level<16>(v, lane);
  transpose_sum_level<8>(v, lane);
  transpose_sum_level<4>(v, lane);
  transpose_sum_level<2>(v, lane);
  transpose_sum_level<1>(v, lane);
}

// Every CTA owns elements [e0, e1) of every column; the column loops below give whole columns to
// warps (lanes over the own elements), so the columns proceed in parallel.
struct BgtChunk {
  int e0, e1;
  __device__ BgtChunk(int n) {
    const int chunk = (n + gridDim.x - 1) / gridDim.x;
    e0 = min(n, (int)blockIdx.x * chunk);
    e1 = min(n, e0 + chunk);
  }
};

__global__ void __launch_bounds__(256) k_bgt_start(BgtArgs a) {
  if (a.skip_outer && *a.skip_outer) return;         // the same value in every CTA
  cg::grid_group grid = cg::this_grid();
  __shared__ float s_beta[BMAXC];
  const int n = a.nc * a.nd, G = gridDim.x;
  const BgtChunk ch(n);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  for (int c = warp; c < a.ncol; c += nwarp) {
    float nn = 0.f;
    for (int e = ch.e0 + lane; e < ch.e1; e += 32) {
      const float2 v = a.b[(size_t)c * n + e];
      nn += v.x * v.x + v.y * v.y;
    }
    nn = warp_sum(nn);
    if (lane == 0) a.npart[(size_t)c * G + blockIdx.x] = nn;
  }
  grid.sync();
  for (int c = warp; c < a.ncol; c += nwarp) {
    float t = 0.f;
    for (int q = lane; q < G; q += 32) t += a.npart[(size_t)c * G + q];
    t = warp_sum(t);
    if (lane == 0) s_beta[c] = sqrtf(t);
  }
  __syncthreads();
  for (int c = warp; c < a.ncol; c += nwarp) {
    const float inv = s_beta[c] > 0.f ? 1.f / s_beta[c] : 0.f;
    for (int e = ch.e0 + lane; e < ch.e1; e += 32) {
      float2 v = a.b[(size_t)c * n + e];
      v.x *= inv;
      v.y *= inv;
      a.V[(size_t)c * n + e] = v;
    }
  }
  if (blockIdx.x == 0) {
    for (int c = threadIdx.x; c < a.ncol; c += blockDim.x) {
      a.beta[c] = s_beta[c];
      a.done[c] = !(s_beta[c] > 0.f);
      a.kk[c] = 0;
      float2* gv = a.gv + (size_t)c * (CMAXM + 1);
      for (int i = 0; i <= CMAXM; i++) gv[i] = make_float2(0.f, 0.f);
      gv[0] = make_float2(s_beta[c], 0.f);
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      int all = 1;
      for (int c = 0; c < a.ncol; c++) all &= a.done[c];
      *a.all_done = all;
    }
  }
}

__global__ void __launch_bounds__(256, 2) k_bgt_arnoldi(BgtArgs a, int j) {
  if (*a.all_done || (a.skip_outer && *a.skip_outer)) return;   // the same values in every CTA: set by earlier launches
  cg::grid_group grid = cg::this_grid();
  extern __shared__ float2 hsm[];                    // [ncol][CMAXM + 1]
  __shared__ float s_hn[BMAXC];
  const int n = a.nc * a.nd, G = gridDim.x;
  const size_t cn = (size_t)a.ncol * n;
  const BgtChunk ch(n);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  const int ngrp = (j + 16) / 16;                    // groups of 16 basis vectors
  float* const partf = reinterpret_cast<float*>(a.part);
  // (1) per-CTA partials of <v_i, w>: one warp per (column, group of 16 basis vectors), every lane
  //     accumulating 16 complex products over its elements; one transpose-sum leaves value l of
  //     the group on lane l
  for (int t = warp; t < a.ncol * ngrp; t += nwarp) {
    const int c = t / ngrp, g0 = (t - c * ngrp) * 16;
    float v[32];
#pragma unroll
    for (int q = 0; q < 32; q++) v[q] = 0.f;
    for (int e = ch.e0 + lane; e < ch.e1; e += 32) {
      const float2 w = a.W[(size_t)c * n + e];
#pragma unroll
      for (int ii = 0; ii < 16; ii++) {
        if (g0 + ii <= j) {
          const float2 p = a.V[(size_t)(g0 + ii) * cn + (size_t)c * n + e];
          v[2 * ii] += p.x * w.x + p.y * w.y;
          v[2 * ii + 1] += p.x * w.y - p.y * w.x;
        }
      }
    }
    warp_transpose_sum(v, lane);
    const int i = g0 + (lane >> 1);
    if (i <= j) partf[(((size_t)c * (CMAXM + 1) + i) * G + blockIdx.x) * 2 + (lane & 1)] = v[0];
  }
  grid.sync();
  // (2) totals h_{i,j} per column: the (column, i) pairs spread over all warps of the grid
  const int npair = a.ncol * (j + 1);
  for (int p = blockIdx.x * nwarp + warp; p < npair; p += G * nwarp) {
    const int c = p / (j + 1), i = p - c * (j + 1);
    float re = 0.f, im = 0.f;
    for (int q = lane; q < G; q += 32) {
      const float2 v = a.part[((size_t)c * (CMAXM + 1) + i) * G + q];
      re += v.x;
      im += v.y;
    }
    re = warp_sum(re);
    im = warp_sum(im);
    if (lane == 0) a.htot[(size_t)c * (CMAXM + 1) + i] = make_float2(re, im);
  }
  grid.sync();
  // (3) w -= sum_i h_i v_i and the ||w||^2 partials on the own elements, a warp per column
  for (int p = threadIdx.x; p < npair; p += blockDim.x) {
    const int c = p / (j + 1), i = p - c * (j + 1);
    hsm[c * (CMAXM + 1) + i] = a.htot[(size_t)c * (CMAXM + 1) + i];
  }
  __syncthreads();
  for (int c = warp; c < a.ncol; c += nwarp) {
    const float2* hp = hsm + c * (CMAXM + 1);
    float nn = 0.f;
    for (int e = ch.e0 + lane; e < ch.e1; e += 32) {
      float2 q = a.W[(size_t)c * n + e];
#pragma unroll 4
      for (int i = 0; i <= j; i++) {
        const float2 p = a.V[(size_t)i * cn + (size_t)c * n + e];
        const float2 h = hp[i];
        q.x -= h.x * p.x - h.y * p.y;
        q.y -= h.x * p.y + h.y * p.x;
      }
      a.W[(size_t)c * n + e] = q;
      nn += q.x * q.x + q.y * q.y;
    }
    nn = warp_sum(nn);
    if (lane == 0) a.npart[(size_t)c * G + blockIdx.x] = nn;
  }
  grid.sync();
  // (4) h_{j+1,j} per column, then v_{j+1} = w / h_{j+1,j} on the own elements (zero for a column
  //     whose w vanished)
  for (int c = warp; c < a.ncol; c += nwarp) {
    float t = 0.f;
    for (int q = lane; q < G; q += 32) t += a.npart[(size_t)c * G + q];
    t = warp_sum(t);
    if (lane == 0) s_hn[c] = sqrtf(t);
  }
  __syncthreads();
  for (int c = warp; c < a.ncol; c += nwarp) {
    const float inv = s_hn[c] > 0.f ? 1.f / s_hn[c] : 0.f;
    float2* vn = a.V + (size_t)(j + 1) * cn + (size_t)c * n;
    for (int e = ch.e0 + lane; e < ch.e1; e += 32) {
      float2 q = a.W[(size_t)c * n + e];
      q.x *= inv;
      q.y *= inv;
      vn[e] = q;
    }
  }
  // (5) CTA 0: Hessenberg column j of every unfinished column, rotated by the column's previous
  //     Givens rotations, the new rotation, the residual estimate and the stopping test
  if (blockIdx.x != 0) return;
  for (int c = threadIdx.x; c < a.ncol; c += blockDim.x) {
    if (a.done[c]) continue;
    float2* hcol = hsm + c * (CMAXM + 1);
    float2* cs = a.cs + (size_t)c * CMAXM;
    float2* sn = a.sn + (size_t)c * CMAXM;
    float2* gv = a.gv + (size_t)c * (CMAXM + 1);
    const float hn = s_hn[c];
    float2 x0 = hcol[0];
    for (int i = 0; i < j; i++) {
      const float2 x1 = hcol[i + 1];
      const float2 cc = cs[i], ss = sn[i];
      hcol[i] = make_float2(cc.x * x0.x + cc.y * x0.y + ss.x * x1.x + ss.y * x1.y,
                            cc.x * x0.y - cc.y * x0.x + ss.x * x1.y - ss.y * x1.x);
      x0 = make_float2(-(ss.x * x0.x - ss.y * x0.y) + (cc.x * x1.x - cc.y * x1.y),
                       -(ss.x * x0.y + ss.y * x0.x) + (cc.x * x1.y + cc.y * x1.x));
    }
    const float den = sqrtf(x0.x * x0.x + x0.y * x0.y + hn * hn);
    const float2 cj = den > 0.f ? make_float2(x0.x / den, x0.y / den) : make_float2(1.f, 0.f);
    const float2 sj = den > 0.f ? make_float2(hn / den, 0.f) : make_float2(0.f, 0.f);
    cs[j] = cj;
    sn[j] = sj;
    hcol[j] = make_float2(den, 0.f);
    const float2 g = gv[j];
    gv[j + 1] = make_float2(-(sj.x * g.x - sj.y * g.y), -(sj.x * g.y + sj.y * g.x));
    gv[j] = make_float2(cj.x * g.x + cj.y * g.y, cj.x * g.y - cj.y * g.x);
    float2* R = a.R + (size_t)c * (CMAXM + 1) * CMAXM + (size_t)j * (CMAXM + 1);
    for (int i = 0; i <= j; i++) R[i] = hcol[i];
    a.kk[c] = j + 1;
    const float res = sqrtf(gv[j + 1].x * gv[j + 1].x + gv[j + 1].y * gv[j + 1].y);
    if (res <= a.rtol * a.beta[c] || !(hn > 0.f) || !(den > 0.f)) a.done[c] = 1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    int all = 1;
    for (int c = 0; c < a.ncol; c++) all &= a.done[c];
    *a.all_done = all || (j == a.m - 1);
  }
}

__global__ void __launch_bounds__(256) k_bgt_finish(BgtArgs a) {
  if (a.skip_outer && *a.skip_outer) return;
  cg::grid_group grid = cg::this_grid();
  __shared__ float2 ys[BMAXC][CMAXM];
  const int n = a.nc * a.nd;
  const size_t cn = (size_t)a.ncol * n;
  const BgtChunk ch(n);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
  if (blockIdx.x == 0) {
    // back substitution R y = g, one thread per column
    for (int c = threadIdx.x; c < a.ncol; c += blockDim.x) {
      const int k = a.kk[c];
      const float2* R = a.R + (size_t)c * (CMAXM + 1) * CMAXM;
      const float2* gv = a.gv + (size_t)c * (CMAXM + 1);
      float2* y = a.y + (size_t)c * CMAXM;
      for (int i = k - 1; i >= 0; i--) {
        float2 acc = gv[i];
        for (int l = i + 1; l < k; l++) {
          const float2 h = R[(size_t)l * (CMAXM + 1) + i], yl = y[l];
          acc.x -= h.x * yl.x - h.y * yl.y;
          acc.y -= h.x * yl.y + h.y * yl.x;
        }
        const float2 d = R[(size_t)i * (CMAXM + 1) + i];
        const float dn = d.x * d.x + d.y * d.y;
        y[i] = dn > 0.f ? make_float2((acc.x * d.x + acc.y * d.y) / dn, (acc.y * d.x - acc.x * d.y) / dn)
                        : make_float2(0.f, 0.f);
      }
      if (a.counter) atomicAdd(a.counter, k);
    }
  }
  grid.sync();
  for (int p = threadIdx.x; p < a.ncol * CMAXM; p += blockDim.x) {
    const int c = p / CMAXM, i = p - c * CMAXM;
    ys[c][i] = i < a.kk[c] ? a.y[(size_t)c * CMAXM + i] : make_float2(0.f, 0.f);
  }
  __syncthreads();
  // x = sum_i y_i v_i on the own elements, a warp per column
  for (int c = warp; c < a.ncol; c += nwarp) {
    const int k = a.kk[c];
    for (int e = ch.e0 + lane; e < ch.e1; e += 32) {
      float xr = 0.f, xi = 0.f;
#pragma unroll 4
      for (int i = 0; i < k; i++) {
        const float2 v = a.V[(size_t)i * cn + (size_t)c * n + e];
        const float2 y = ys[c][i];
        xr += y.x * v.x - y.y * v.y;
        xi += y.x * v.y + y.y * v.x;
      }
      a.x[(size_t)c * n + e] = make_float2(xr, xi);
    }
  }
}

}  // namespace

// Whether the tensor-core batched coarse solve covers this level: the tcgen05 coarse apply's block
// widths (2 N_v = 8 .. 64) and at most 32 columns.
bool coarse_gmres_batched_tc_ok(const Ctx& c, int ncol) { return tc_level_ok(c.cl.nd, ncol); }

namespace {

// Launch shape of the three batched-GMRES kernels for vectors of n elements: a cooperative grid of
// at most two CTAs per SM and no more CTAs than 32-element chunks.
struct BgtPlan {
  int G;
  size_t hsm;
};
BgtPlan bgt_plan(Ctx& c, size_t n, int ncol) {
  static int mps[3] = {-1, -1, -1};
  if (mps[0] < 0) {
    TMG_CUDA(cudaFuncSetAttribute(k_bgt_arnoldi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                  (int)(sizeof(float2) * BMAXC * (CMAXM + 1))));
    TMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mps[0], k_bgt_start, 256, 0));
    TMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mps[1], k_bgt_arnoldi, 256,
                                                           sizeof(float2) * BMAXC * (CMAXM + 1)));
    TMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mps[2], k_bgt_finish, 256, 0));
  }
  const int per_sm = std::min(2, std::min(mps[0], std::min(mps[1], mps[2])));
  if (per_sm < 1) throw Error{TMG_ERR_CUDA, "tensor-core batched coarse solve: kernels cannot be resident"};
  BgtPlan p;
  p.G = std::max(1, std::min((int)((n + 31) / 32), c.sms * per_sm));
  p.hsm = sizeof(float2) * (size_t)ncol * (CMAXM + 1);
  return p;
}

// Bytes of one solve's state (part, cs, sn, gv, R, y, htot, npart, beta, done, kk, all_done) and
// its carving from one allocation.
size_t bgt_state_bytes(int ncol, int G) {
  const size_t d2 = (size_t)ncol * ((CMAXM + 1) * G + 2 * CMAXM + (CMAXM + 1) + (CMAXM + 1) * CMAXM + CMAXM + (CMAXM + 1));
  const size_t bytes = sizeof(float2) * d2 + sizeof(float) * ((size_t)ncol * G + ncol) + sizeof(int) * (2 * (size_t)ncol + 1);
  return (bytes + 255) & ~(size_t)255;
}
void bgt_carve(BgtArgs& a, void* state, int ncol, int G) {
  a.part = reinterpret_cast<float2*>(state);
  a.cs = a.part + (size_t)ncol * (CMAXM + 1) * G;
  a.sn = a.cs + (size_t)ncol * CMAXM;
  a.gv = a.sn + (size_t)ncol * CMAXM;
  a.R = a.gv + (size_t)ncol * (CMAXM + 1);
  a.y = a.R + (size_t)ncol * (CMAXM + 1) * CMAXM;
  a.htot = a.y + (size_t)ncol * CMAXM;
  a.npart = reinterpret_cast<float*>(a.htot + (size_t)ncol * (CMAXM + 1));
  a.beta = a.npart + (size_t)ncol * G;
  a.done = reinterpret_cast<int*>(a.beta + ncol);
  a.kk = a.done + ncol;
  a.all_done = a.kk + ncol;
}

void ensure_counters(Ctx& c) {
  if (!c.coarse_iter_dev.p) {
    c.coarse_iter_dev.alloc(sizeof(int));
    TMG_CUDA(cudaMemsetAsync(c.coarse_iter_dev.p, 0, sizeof(int), c.stream));
  }
  if (!c.tc_err.p) {
    c.tc_err.alloc(sizeof(int));
    TMG_CUDA(cudaMemsetAsync(c.tc_err.p, 0, sizeof(int), c.stream));
  }
}

// A whole batched GMRES on level L: start, a.m Arnoldi steps (tensor-core apply of V_j, then the
// orthogonalisation kernel), and the solution x = V y.
void bgt_run(Ctx& c, const TcLevel& L, BgtArgs& a, const BgtPlan& pl, const float* mu_dev) {
  const size_t n = (size_t)L.nc * L.nd;
  int* tc_err = c.tc_err.as<int>();
  void* args[] = {&a};
  ++c.launches;
  TMG_CUDA(cudaLaunchCooperativeKernel((const void*)k_bgt_start, dim3(pl.G), dim3(256), args, 0, c.stream));
  for (int j = 0; j < a.m; j++) {
    coarse_apply_tc_level(c, L, a.ncol, a.V + (size_t)j * a.ncol * n, a.W, mu_dev, tc_err, a.all_done, a.skip_outer);
    void* sargs[] = {&a, &j};
    ++c.launches;
    TMG_CUDA(cudaLaunchCooperativeKernel((const void*)k_bgt_arnoldi, dim3(pl.G), dim3(256), sargs, pl.hsm, c.stream));
  }
  ++c.launches;
  TMG_CUDA(cudaLaunchCooperativeKernel((const void*)k_bgt_finish, dim3(pl.G), dim3(256), args, 0, c.stream));
}

BgtArgs bgt_args(const TcLevel& L, int ncol, int m, float rtol, const void* b, void* x, float2* V, float2* W, int* counter,
                 const int* skip_outer) {
  BgtArgs a;
  a.nd = L.nd;
  a.nv = L.nv;
  a.nc = L.nc;
  a.m = m;
  a.ncol = ncol;
  a.b = (const float2*)b;
  a.x = (float2*)x;
  a.V = V;
  a.W = W;
  a.rtol = rtol;
  a.counter = counter;
  a.skip_outer = skip_outer;
  return a;
}

}  // namespace

void coarse_gmres_batched_tc(Ctx& c, int ncol, const void* b, void* x, const float* mu_dev) {
  ProfScope ps(c, PK_COARSE_SOLVE);
  if (!coarse_gmres_batched_tc_ok(c, ncol)) throw Error{TMG_ERR_ARG, "tensor-core batched coarse solve: unsupported shape"};
  const int m = std::min(c.batched_coarse_m > 0 ? c.batched_coarse_m : c.mg.coarse_m, CMAXM);
  const TcLevel L = tc_level1(c);
  const size_t n = (size_t)L.nc * L.nd;
  const BgtPlan pl = bgt_plan(c, n, ncol);
  c.cw_V.alloc((m + 1) * n * ncol * sizeof(float2));
  c.cw_w.alloc(n * ncol * sizeof(float2));
  c.cw_state.alloc(bgt_state_bytes(ncol, pl.G));
  ensure_counters(c);
  BgtArgs a = bgt_args(L, ncol, m, (float)c.mg.coarse_rtol, b, x, c.cw_V.as<float2>(), c.cw_w.as<float2>(),
                       c.coarse_iter_dev.as<int>(), nullptr);
  bgt_carve(a, c.cw_state.p, ncol, pl.G);
  bgt_run(c, L, a, pl, mu_dev);
}

// ---- the level-1 K-cycle for ncol columns in lock-step (three levels, batched solve).  The same
// algorithm as k_kcycle (FGMRES on D_c, right-preconditioned by the level-1 cycle z = P2 gmres_L2(P2^dag v)
// followed by smooth_m GMRES steps on D_c from zero), with every column advancing together: each
// operator application is one tensor-core launch for all columns (every stencil block read once per
// step), every Gram-Schmidt step one cooperative launch, and the restriction, prolongation and
// vector updates one launch each.  Once every column of the FGMRES has stopped, the remaining
// launches return at once (they read its all-done flag).
namespace {

__global__ void __launch_bounds__(256) k_kb_restrict2(L2Geom q, const float2* __restrict__ W2, const float2* __restrict__ v,
                                                      float2* __restrict__ c2, size_t n1, size_t n2, const int* skip) {
  if (skip && *skip) return;
  restrict2_dev<float>(q, W2, v + blockIdx.y * n1, c2 + blockIdx.y * n2);
}

__global__ void __launch_bounds__(256) k_kb_prolong2(L2Geom q, const float2* __restrict__ W2, const float2* __restrict__ c2,
                                                     float2* __restrict__ z, size_t n1, size_t n2, const int* skip) {
  if (skip && *skip) return;
  prolong2_dev<float>(q, W2, c2 + blockIdx.y * n2, z + blockIdx.y * n1);
}

// out = u + s v (elementwise over n complex values)
__global__ void __launch_bounds__(256) k_kb_axpy(const float2* u, const float2* __restrict__ v, float2* out, size_t n, float s,
                                                 const int* skip) {
  if (skip && *skip) return;
  for (size_t e = (size_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (size_t)gridDim.x * blockDim.x) {
    const float2 a = u[e], b = v[e];
    out[e] = make_float2(a.x + s * b.x, a.y + s * b.y);
  }
}

}  // namespace

bool kcycle_batched_ok(const Ctx& c, int ncol) {
  return c.l2_ready && c.batched_tc && tc_level_ok(c.cl.nd, ncol) && tc_level_ok(c.cl2.nd, ncol);
}

void kcycle_batched(Ctx& c, int ncol, const void* b, void* x, const float* mu_dev, int mode) {
  ProfScope ps(c, PK_COARSE_SOLVE);
  if (!kcycle_batched_ok(c, ncol)) throw Error{TMG_ERR_ARG, "batched K-cycle: unsupported shape"};
  const tmg_level2_params& p = c.l2p;
  const TcLevel L1 = tc_level1(c), L2 = tc_level2(c);
  const size_t n1 = (size_t)L1.nc * L1.nd, n2 = (size_t)L2.nc * L2.nd, m1 = n1 * ncol, m2 = n2 * ncol;
  const int sm_m = std::max(1, std::min(p.smooth_m, CMAXM)), cm = std::max(1, std::min(p.coarse_m, CMAXM));
  const int kr = std::max(1, std::min(p.k_restart, KMAXR));
  const BgtPlan P1 = bgt_plan(c, n1, ncol), P2 = bgt_plan(c, n2, ncol);
  // one allocation: FGMRES basis V, preconditioned vectors Z and w; smoother basis and w; the
  // smoother's right-hand side and solution; the level-2 right-hand side, solution, basis and w;
  // the three solves' states
  const size_t vec[] = {(kr + 1) * m1, kr * m1, m1, (sm_m + 1) * m1, m1, m1, m1, m2, m2, (cm + 1) * m2, m2};
  const size_t nvec = sizeof(vec) / sizeof(vec[0]);
  size_t off[16], o = 0;
  for (size_t i = 0; i < nvec; i++) { off[i] = o; o += ((vec[i] * sizeof(float2)) + 255) & ~(size_t)255; }
  const size_t so = o, s1b = bgt_state_bytes(ncol, P1.G), s2b = bgt_state_bytes(ncol, P2.G);
  o += 2 * s1b + s2b;
  c.kbw.alloc(o);
  ensure_counters(c);
  if (!c.l2_iter_dev.p) {
    c.l2_iter_dev.alloc(sizeof(int));
    TMG_CUDA(cudaMemsetAsync(c.l2_iter_dev.p, 0, sizeof(int), c.stream));
  }
  char* base = (char*)c.kbw.p;
  auto v = [&](int i) { return (float2*)(base + off[i]); };
  float2 *oV = v(0), *oZ = v(1), *oW = v(2), *sV = v(3), *sW = v(4), *r1 = v(5), *es = v(6), *c2 = v(7), *e2 = v(8),
         *bV = v(9), *bW = v(10);
  const float2* W2 = c.cl2.W32.as<float2>();
  const L2Geom q = l2geom(c);
  auto smoother = [&](const void* rhs, void* out, const int* skip) {
    BgtArgs S = bgt_args(L1, ncol, sm_m, 0.f, rhs, out, sV, sW, nullptr, skip);
    bgt_carve(S, base + so + s1b, ncol, P1.G);
    bgt_run(c, L1, S, P1, mu_dev);
  };
  const int eb = 256;
  auto grid_for = [&](size_t n) { return (unsigned)std::max<size_t>(1, std::min<size_t>((n + eb - 1) / eb, (size_t)8 * c.sms)); };
  // z = level-1 cycle of v (all columns): level-2 correction, then the smoother on the residual
  auto l1_cycle = [&](const float2* vin, float2* z, const int* skip) {
    ++c.launches;
    k_kb_restrict2<<<dim3(grid_for(n2), ncol), eb, 0, c.stream>>>(q, W2, vin, c2, n1, n2, skip);
    BgtArgs B = bgt_args(L2, ncol, cm, (float)p.coarse_rtol, c2, e2, bV, bW, c.l2_iter_dev.as<int>(), skip);
    bgt_carve(B, base + so + 2 * s1b, ncol, P2.G);
    bgt_run(c, L2, B, P2, mu_dev);
    ++c.launches;
    k_kb_prolong2<<<dim3(grid_for(n1), ncol), eb, 0, c.stream>>>(q, W2, e2, z, n1, n2, skip);
    coarse_apply_tc_level(c, L1, ncol, z, sW, mu_dev, c.tc_err.as<int>(), skip, nullptr);
    ++c.launches;
    k_kb_axpy<<<grid_for(m1), eb, 0, c.stream>>>(vin, sW, r1, m1, -1.f, skip);
    smoother(r1, es, skip);
    ++c.launches;
    k_kb_axpy<<<grid_for(m1), eb, 0, c.stream>>>(z, es, z, m1, 1.f, skip);
  };
  if (mode == 2) {
    smoother(b, x, nullptr);
  } else if (mode == 1) {
    l1_cycle((const float2*)b, (float2*)x, nullptr);
  } else {
    BgtArgs A = bgt_args(L1, ncol, kr, (float)p.k_rtol, b, x, oV, oW, c.coarse_iter_dev.as<int>(), nullptr);
    bgt_carve(A, base + so, ncol, P1.G);
    void* args[] = {&A};
    ++c.launches;
    TMG_CUDA(cudaLaunchCooperativeKernel((const void*)k_bgt_start, dim3(P1.G), dim3(256), args, 0, c.stream));
    for (int j = 0; j < kr; j++) {
      float2* zj = oZ + (size_t)j * m1;
      l1_cycle(oV + (size_t)j * m1, zj, A.all_done);
      coarse_apply_tc_level(c, L1, ncol, zj, oW, mu_dev, c.tc_err.as<int>(), A.all_done, nullptr);
      void* sargs[] = {&A, &j};
      ++c.launches;
      TMG_CUDA(cudaLaunchCooperativeKernel((const void*)k_bgt_arnoldi, dim3(P1.G), dim3(256), sargs, P1.hsm, c.stream));
    }
    BgtArgs F = A;                                   // flexible GMRES: x = Z y
    F.V = oZ;
    void* fargs[] = {&F};
    ++c.launches;
    TMG_CUDA(cudaLaunchCooperativeKernel((const void*)k_bgt_finish, dim3(P1.G), dim3(256), fargs, 0, c.stream));
  }
  TMG_CHECK_LAUNCH();
}

}  // namespace tmg

namespace tmg {

namespace {

template <typename S>
void kcycle_launch(Ctx& c, const void* b, void* x, double mu, int mode, int nf, double epsbar) {
  using T2 = typename CplxT<S>::T2;
  const tmg_level2_params& p = c.l2p;
  const size_t n1 = (size_t)nf * c.cl.nc * c.cl.nd, n2 = (size_t)nf * c.cl2.nc * c.cl2.nd;
  static int max_per_sm[2] = {-1, -1};
  int& mps = max_per_sm[sizeof(S) == 8];
  if (mps < 0) TMG_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&mps, k_kcycle<S>, 256, 0));
  if (mps < 1) throw Error{TMG_ERR_CUDA, "K-cycle kernel cannot be resident"};
  const int G = c.kcycle_grid > 0 ? std::max(1, std::min(c.kcycle_grid, c.sms * mps))
                                  : c.sms * std::max(1, std::min(mps, c.kcycle_ctas_per_sm));
  const int sm_m = std::min(p.smooth_m, CMAXM), cm = std::min(p.coarse_m, CMAXM), kr = std::min(p.k_restart, KMAXR);
  // one scratch allocation, carved 256-byte aligned
  const size_t vec_elems[] = {(kr + 1) * n1, kr * n1, n1, n1, n1, (sm_m + 1) * n1, 11 * n1, n2, n2, (cm + 1) * n2, 11 * n2};
  const size_t nvec = sizeof(vec_elems) / sizeof(vec_elems[0]);
  const size_t d2_elems[] = {(size_t)2 * (KMAXR + 1) * G, (size_t)(KMAXR + 1) * KMAXR, KMAXR,
                             (size_t)2 * (CMAXM + 1) * G, (size_t)(CMAXM + 1) * CMAXM, CMAXM,
                             (size_t)2 * (CMAXM + 1) * G, (size_t)(CMAXM + 1) * CMAXM, CMAXM};
  const size_t nd2 = sizeof(d2_elems) / sizeof(d2_elems[0]);
  size_t off[32], o = 0;
  auto al = [](size_t v) { return (v + 255) & ~(size_t)255; };
  for (size_t i = 0; i < nvec; i++) { off[i] = o; o = al(o + vec_elems[i] * sizeof(T2)); }
  for (size_t i = 0; i < nd2; i++) { off[nvec + i] = o; o = al(o + d2_elems[i] * sizeof(double2)); }
  off[nvec + nd2] = o;
  o = al(o + 3 * (size_t)G * sizeof(double));
  c.kw.alloc(o);
  if (!c.l2_iter_dev.p) {
    c.l2_iter_dev.alloc(sizeof(int));
    TMG_CUDA(cudaMemsetAsync(c.l2_iter_dev.p, 0, sizeof(int), c.stream));
  }
  if (!c.coarse_iter_dev.p) {
    c.coarse_iter_dev.alloc(sizeof(int));
    TMG_CUDA(cudaMemsetAsync(c.coarse_iter_dev.p, 0, sizeof(int), c.stream));
  }
  char* base = (char*)c.kw.p;
  auto vec = [&](int i) { return (T2*)(base + off[i]); };
  auto d2 = [&](int i) { return (double2*)(base + off[nvec + i]); };
  double* npart = (double*)(base + off[nvec + nd2]);
  const int passes = c.coarse_gs_passes > 0 ? c.coarse_gs_passes : (sizeof(S) == 4 ? 1 : 2);

  KcArgs<S> a;
  a.q = l2geom(c);
  CgArgs<S>& s = a.sm;
  s.nd = c.cl.nd;
  s.nv = c.cl.nv;
  s.nc = c.cl.nc;
  s.m = sm_m;
  s.nf = nf;
  s.epsbar = (S)epsbar;
  s.delta = nf == 2 ? (S)c.ndshift : (S)0;
  s.overlap = c.coarse_overlap;
  s.rows_smem = 0;
  s.blk_cache = 0;
  s.cache_off = 0;
  s.eo = 0;
  s.inv = nullptr;
  s.te = s.rb = nullptr;
  s.passes = passes;
  s.Dc = (const T2*)(sizeof(S) == 8 ? c.cl.Dc64.p : c.cl.Dc32.p);
  s.nbr = c.cl.nbr.as<int>();
  s.b = mode == 2 ? (const T2*)b : vec(3);
  s.x = mode == 2 ? (T2*)x : vec(4);
  s.V = vec(5);
  s.w = vec(6);
  s.rows = s.w + 2 * n1;
  s.mu = (S)mu;
  s.rtol = 0.0;
  s.part = d2(3);
  s.R = d2(4);
  s.y = d2(5);
  s.npart = npart + G;
  s.counter = nullptr;
  CgArgs<S>& l = a.l2;
  l.nd = c.cl2.nd;
  l.nv = c.cl2.nv;
  l.nc = c.cl2.nc;
  l.m = cm;
  l.nf = nf;
  l.epsbar = (S)epsbar;
  l.delta = nf == 2 ? (S)c.ndshift : (S)0;
  l.overlap = c.coarse_overlap;
  l.rows_smem = 0;
  l.blk_cache = 0;
  l.cache_off = 0;
  l.eo = 0;
  l.inv = nullptr;
  l.te = l.rb = nullptr;
  l.passes = passes;
  l.Dc = (const T2*)(sizeof(S) == 8 ? c.cl2.Dc64.p : c.cl2.Dc32.p);
  l.nbr = c.cl2.nbr.as<int>();
  l.b = vec(7);
  l.x = vec(8);
  l.V = vec(9);
  l.w = vec(10);
  l.rows = l.w + 2 * n2;
  l.mu = (S)mu;
  l.rtol = p.coarse_rtol;
  l.part = d2(6);
  l.R = d2(7);
  l.y = d2(8);
  l.npart = npart + 2 * G;
  l.counter = c.l2_iter_dev.as<int>();
  a.W2 = (const T2*)(sizeof(S) == 8 ? c.cl2.W64.p : c.cl2.W32.p);
  a.b = (const T2*)b;
  a.x = (T2*)x;
  a.V = vec(0);
  a.Z = vec(1);
  a.t = vec(2);
  a.kr = kr;
  a.passes = passes;
  a.mode = mode;
  a.krtol = p.k_rtol;
  a.part = d2(0);
  a.R = d2(1);
  a.y = d2(2);
  a.npart = npart;
  a.counter = c.coarse_iter_dev.as<int>();
  void* args[] = {&a};
  ++c.launches;
  TMG_CUDA(cudaLaunchCooperativeKernel((const void*)k_kcycle<S>, dim3(G), dim3(256), args, 0, c.stream));
}

}  // namespace

void kcycle(Ctx& c, int prec, const void* b, void* x, double mu, int mode, int nf) {
  ProfScope ps(c, PK_COARSE_SOLVE);
  if (!c.l2_ready && mode != 2) throw Error{TMG_ERR_STATE, "K-cycle: level 2 not built"};
  const double eb = nf == 2 ? c.epsbar : 0.0;
  if (nf == 2) mu = c.mubar;
  if (prec == TMG_PREC_F64) kcycle_launch<double>(c, b, x, mu, mode, nf, eb);
  else kcycle_launch<float>(c, b, x, mu, mode, nf, eb);
}

}  // namespace tmg
