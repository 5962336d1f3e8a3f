// Third level of the DD-alpha-AMG hierarchy (the paper runs three levels, Sec. 1.2): the level-1
// operator D_c is aggregated again.  Level-1 vectors are [nc1][nd1] complex with the level-1 sites
// in lexicographic order of the level-1 lattice (dims NB of the fine geometry); level-2 aggregates
// are agg2-shaped blocks of level-1 sites; level-1 dofs split into chirality halves [+ | -]
// (G5_c), so P2 is G5-compatible exactly like the fine P.
//
//   k_restrict_c   : c2[a2][chi nv2 + j] = sum_{a1 in a2, k in chi} conj(W2_j[a1][k]) r[a1][k]
//   k_prolong_c    : e[a1][k] = sum_j W2_j[a1][k] c2[a2(a1)][chi(k) nv2 + j]
//   k_ortho_c      : per (level-2 aggregate, chirality) modified Gram-Schmidt, twice, in FP64
//   k_dc_pieces    : the 9 pieces of D_c w (aggregate-Dirichlet self part and the 8 face hops),
//                    used column by column to build D_cc = P2^dag D_c P2 (setup)
#include "tmg_host.h"
#include "level2.cuh"

namespace tmg {

namespace {

// one CTA per level-2 aggregate, one thread per output (chi, j) (2 nv2 <= 64)
template <typename T2, typename W2T>
__global__ void k_restrict_c(L2Geom q, const T2* __restrict__ r, const W2T* __restrict__ W, T2* __restrict__ out) {
  const int a2 = blockIdx.x;
  const int o = threadIdx.x;
  if (o >= 2 * q.nv2) return;
  const int chi = o / q.nv2, j = o - chi * q.nv2;
  const size_t n1 = (size_t)q.nc1 * q.nd1;
  double re = 0.0, im = 0.0;
  for (int t = 0; t < q.avol; t++) {
    const int a1 = l2_member(q, a2, t);
    for (int k = chi * q.nv1; k < (chi + 1) * q.nv1; k++) {
      const W2T w = W[(size_t)j * n1 + (size_t)a1 * q.nd1 + k];
      const T2 x = r[(size_t)a1 * q.nd1 + k];
      re += (double)w.x * x.x + (double)w.y * x.y;
      im += (double)w.x * x.y - (double)w.y * x.x;
    }
  }
  T2 v;
  v.x = re;
  v.y = im;
  out[(size_t)a2 * 2 * q.nv2 + o] = v;
}

// one thread per level-1 element (a1, k)
template <typename T2, typename W2T>
__global__ void k_prolong_c(L2Geom q, const T2* __restrict__ c2, const W2T* __restrict__ W, T2* __restrict__ e) {
  const size_t n1 = (size_t)q.nc1 * q.nd1;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= n1) return;
  const int a1 = (int)(idx / q.nd1), k = (int)(idx - (size_t)a1 * q.nd1);
  int c[4];
  l1_coords(q, a1, c);
  const int a2 = l2_agg_of(q, c);
  const int chi = k / q.nv1;
  double re = 0.0, im = 0.0;
  for (int j = 0; j < q.nv2; j++) {
    const W2T w = W[(size_t)j * n1 + idx];
    const T2 v = c2[(size_t)a2 * 2 * q.nv2 + chi * q.nv2 + j];
    re += (double)w.x * v.x - (double)w.y * v.y;
    im += (double)w.x * v.y + (double)w.y * v.x;
  }
  T2 o;
  o.x = re;
  o.y = im;
  e[idx] = o;
}

// one CTA (128 threads) per (aggregate, chirality); elements of the aggregate's chirality half are
// strided over the threads
__global__ void k_ortho_c(L2Geom q, double2* __restrict__ W) {
  __shared__ double red[64];
  const int a2 = blockIdx.x >> 1, chi = blockIdx.x & 1;
  const size_t n1 = (size_t)q.nc1 * q.nd1;
  const int len = q.avol * q.nv1;
  auto at = [&](int j, int e) -> double2& {
    const int t = e / q.nv1, k = chi * q.nv1 + (e - t * q.nv1);
    return W[(size_t)j * n1 + (size_t)l2_member(q, a2, t) * q.nd1 + k];
  };
  auto cta_sum2 = [&](double& a, double& b) {
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) { red[2 * w] = a; red[2 * w + 1] = b; }
    __syncthreads();
    a = 0.0;
    b = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); k++) { a += red[2 * k]; b += red[2 * k + 1]; }
    __syncthreads();
  };
  for (int pass = 0; pass < 2; pass++)
    for (int j = 0; j < q.nv2; j++) {
      for (int i = 0; i < j; i++) {
        double re = 0.0, im = 0.0;
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
          const double2 a = at(i, e), b = at(j, e);
          re += a.x * b.x + a.y * b.y;
          im += a.x * b.y - a.y * b.x;
        }
        cta_sum2(re, im);
        for (int e = threadIdx.x; e < len; e += blockDim.x) {
          const double2 a = at(i, e);
          double2& b = at(j, e);
          b.x -= re * a.x - im * a.y;
          b.y -= re * a.y + im * a.x;
        }
        __syncthreads();
      }
      double nn = 0.0, dummy = 0.0;
      for (int e = threadIdx.x; e < len; e += blockDim.x) { const double2 b = at(j, e); nn += b.x * b.x + b.y * b.y; }
      cta_sum2(nn, dummy);
      const double inv = nn > 0.0 ? 1.0 / sqrt(nn) : 0.0;
      for (int e = threadIdx.x; e < len; e += blockDim.x) {
        double2& b = at(j, e);
        b.x *= inv;
        b.y *= inv;
      }
      __syncthreads();
    }
}

// 9 pieces of D_c w for the level-1 vector w = W2_j restricted to chirality chi_l (column l of
// the level-2 basis): piece 0 = self block + hops inside the level-2 aggregate; piece 1 + 2 mu
// (2 + 2 mu) = the +mu (-mu) hop for sites on that face of their aggregate (zero elsewhere).
// out[piece][a1][k]; one thread per (a1, k).
__global__ void k_dc_pieces(L2Geom q, const double2* __restrict__ Dc, const int* __restrict__ nbr,
                            const double2* __restrict__ W, int l, double2* __restrict__ out) {
  const size_t n1 = (size_t)q.nc1 * q.nd1;
  const size_t idx = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
  if (idx >= n1) return;
  const int a1 = (int)(idx / q.nd1), k = (int)(idx - (size_t)a1 * q.nd1);
  const int chi_l = l / q.nv2, j_l = l - chi_l * q.nv2;
  int c[4];
  l1_coords(q, a1, c);
  const double2* wj = W + (size_t)j_l * n1;
  double2 self = make_double2(0.0, 0.0);
  for (int d = 0; d < 9; d++) {
    const int b1 = nbr[a1 * 9 + d];
    const double2* blk = Dc + ((size_t)(a1 * 9 + d) * q.nd1) * q.nd1 + k;   // column l' stride nd1
    double re = 0.0, im = 0.0;
    for (int kk = chi_l * q.nv1; kk < (chi_l + 1) * q.nv1; kk++) {
      const double2 m = blk[(size_t)kk * q.nd1];
      const double2 v = wj[(size_t)b1 * q.nd1 + kk];
      re += m.x * v.x - m.y * v.y;
      im += m.x * v.y + m.y * v.x;
    }
    bool inner = true;
    if (d > 0) {
      const int mu = (d - 1) >> 1;
      const bool fwd = ((d - 1) & 1) == 0;
      const int lc = c[mu] % q.A[mu];
      inner = fwd ? (lc != q.A[mu] - 1) : (lc != 0);
    }
    if (inner) { self.x += re; self.y += im; }
    if (d > 0) out[(size_t)d * n1 + idx] = inner ? make_double2(0.0, 0.0) : make_double2(re, im);
  }
  out[idx] = self;
}

// one CTA per (level-2 aggregate, piece): the 2 nv2 rows of column l of the piece's block
__global__ void k_restrict_pieces(L2Geom q, const double2* __restrict__ pieces, const double2* __restrict__ W, int l,
                                  double2* __restrict__ Dcc) {
  const int a2 = blockIdx.x, d = blockIdx.y;
  const int o = threadIdx.x;
  if (o >= 2 * q.nv2) return;
  const int chi = o / q.nv2, j = o - chi * q.nv2;
  const size_t n1 = (size_t)q.nc1 * q.nd1;
  const double2* r = pieces + (size_t)d * n1;
  double re = 0.0, im = 0.0;
  for (int t = 0; t < q.avol; t++) {
    const int a1 = l2_member(q, a2, t);
    for (int k = chi * q.nv1; k < (chi + 1) * q.nv1; k++) {
      const double2 w = W[(size_t)j * n1 + (size_t)a1 * q.nd1 + k];
      const double2 x = r[(size_t)a1 * q.nd1 + k];
      re += w.x * x.x + w.y * x.y;
      im += w.x * x.y - w.y * x.x;
    }
  }
  const int nd2 = 2 * q.nv2;
  Dcc[((size_t)(a2 * 9 + d) * nd2 + l) * nd2 + o] = make_double2(re, im);
}

// y[a][k] = sum_d sum_l Dc[a][d][l][k] x[nbr[a][d]][l] + i mu g5[k] x[a][k], one thread per (a, k)
template <typename R, typename T2>
__global__ void __launch_bounds__(128) k_coarse_apply_tab(int nc, int nd, int nv, const T2* __restrict__ Dc,
                                                          const int* __restrict__ nbr, const T2* __restrict__ x,
                                                          T2* __restrict__ y, R mu) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= nc * nd) return;
  const int a = idx / nd, k = idx - a * nd;
  R re = 0, im = 0;
  for (int d = 0; d < 9; d++) {
    const T2* blk = Dc + ((size_t)(a * 9 + d) * nd) * nd + k;
    const T2* xv = x + (size_t)nbr[a * 9 + d] * nd;
    for (int l = 0; l < nd; l++) {
      const T2 m = blk[(size_t)l * nd];
      const T2 v = xv[l];
      re += (R)m.x * (R)v.x - (R)m.y * (R)v.y;
      im += (R)m.x * (R)v.y + (R)m.y * (R)v.x;
    }
  }
  const T2 xs = x[idx];
  const R tw = k < nv ? mu : -mu;
  T2 o;
  o.x = re - tw * (R)xs.y;
  o.y = im + tw * (R)xs.x;
  y[idx] = o;
}

}  // namespace

L2Geom l2geom(const Ctx& c) {
  L2Geom q{};
  for (int mu = 0; mu < 4; mu++) {
    q.NB[mu] = c.g.NB[mu];
    q.A[mu] = c.cl2.agg[mu];
    q.NA[mu] = c.g.NB[mu] / c.cl2.agg[mu];
  }
  q.nc1 = c.cl.nc;
  q.nd1 = c.cl.nd;
  q.nv1 = c.cl.nv;
  q.nv2 = c.cl2.nv;
  q.nc2 = c.cl2.nc;
  q.avol = c.cl2.agg[0] * c.cl2.agg[1] * c.cl2.agg[2] * c.cl2.agg[3];
  return q;
}

void restrict_c(Ctx& c, int prec, const void* r, void* c2) {
  const L2Geom q = l2geom(c);
  const int threads = ((2 * q.nv2 + 31) / 32) * 32;
  if (prec == TMG_PREC_F64)
    ++c.launches, k_restrict_c<double2, double2><<<q.nc2, threads, 0, c.stream>>>(q, (const double2*)r, c.cl2.W64.as<double2>(), (double2*)c2);
  else
    ++c.launches, k_restrict_c<float2, float2><<<q.nc2, threads, 0, c.stream>>>(q, (const float2*)r, c.cl2.W32.as<float2>(), (float2*)c2);
  TMG_CHECK_LAUNCH();
}

void coarse_apply_c(Ctx& c, int prec, const void* x, void* y, double mu) {
  const int n = c.cl2.nc * c.cl2.nd;
  if (prec == TMG_PREC_F64)
    ++c.launches, k_coarse_apply_tab<double, double2><<<(n + 127) / 128, 128, 0, c.stream>>>(
                      c.cl2.nc, c.cl2.nd, c.cl2.nv, c.cl2.Dc64.as<double2>(), c.cl2.nbr.as<int>(), (const double2*)x, (double2*)y, mu);
  else
    ++c.launches, k_coarse_apply_tab<float, float2><<<(n + 127) / 128, 128, 0, c.stream>>>(
                      c.cl2.nc, c.cl2.nd, c.cl2.nv, c.cl2.Dc32.as<float2>(), c.cl2.nbr.as<int>(), (const float2*)x, (float2*)y, (float)mu);
  TMG_CHECK_LAUNCH();
}

void prolong_c(Ctx& c, int prec, const void* c2, void* e) {
  const L2Geom q = l2geom(c);
  const size_t n1 = (size_t)q.nc1 * q.nd1;
  const int blocks = (int)((n1 + 127) / 128);
  if (prec == TMG_PREC_F64)
    ++c.launches, k_prolong_c<double2, double2><<<blocks, 128, 0, c.stream>>>(q, (const double2*)c2, c.cl2.W64.as<double2>(), (double2*)e);
  else
    ++c.launches, k_prolong_c<float2, float2><<<blocks, 128, 0, c.stream>>>(q, (const float2*)c2, c.cl2.W32.as<float2>(), (float2*)e);
  TMG_CHECK_LAUNCH();
}

void orthonormalise_c(Ctx& c) {
  const L2Geom q = l2geom(c);
  ++c.launches, k_ortho_c<<<2 * q.nc2, 128, 0, c.stream>>>(q, c.cl2.W64.as<double2>());
  TMG_CHECK_LAUNCH();
}

void build_coarse_c(Ctx& c) {
  const L2Geom q = l2geom(c);
  const int nd2 = 2 * q.nv2;
  const size_t n1 = (size_t)q.nc1 * q.nd1;
  const size_t nb = (size_t)q.nc2 * 9 * nd2 * nd2;
  c.cl2.Dc64.alloc(nb * sizeof(double2));
  c.cl2.Dc32.alloc(nb * sizeof(float2));
  DBuf pieces;
  pieces.alloc(9 * n1 * sizeof(double2));
  const int threads = ((nd2 + 31) / 32) * 32;
  for (int l = 0; l < nd2; l++) {
    ++c.launches, k_dc_pieces<<<(int)((n1 + 127) / 128), 128, 0, c.stream>>>(q, c.cl.Dc64.as<double2>(), c.cl.nbr.as<int>(),
                                                                          c.cl2.W64.as<double2>(), l, pieces.as<double2>());
    TMG_CHECK_LAUNCH();
    ++c.launches, k_restrict_pieces<<<dim3(q.nc2, 9), threads, 0, c.stream>>>(q, pieces.as<double2>(), c.cl2.W64.as<double2>(), l,
                                                                         c.cl2.Dc64.as<double2>());
    TMG_CHECK_LAUNCH();
  }
  convert_field(c, c.cl2.Dc64.p, TMG_PREC_F64, c.cl2.Dc32.p, TMG_PREC_F32, nb);
  // level-2 neighbour table
  std::vector<int> nbv((size_t)q.nc2 * 9);
  for (int a = 0; a < q.nc2; a++) {
    int b[4], t = a;
    b[0] = t % q.NA[0]; t /= q.NA[0];
    b[1] = t % q.NA[1]; t /= q.NA[1];
    b[2] = t % q.NA[2]; b[3] = t / q.NA[2];
    nbv[(size_t)a * 9] = a;
    for (int mu = 0; mu < 4; mu++)
      for (int dir = 0; dir < 2; dir++) {
        int bb[4] = {b[0], b[1], b[2], b[3]};
        bb[mu] = (bb[mu] + (dir == 0 ? 1 : q.NA[mu] - 1)) % q.NA[mu];
        nbv[(size_t)a * 9 + 1 + 2 * mu + dir] = bb[0] + q.NA[0] * (bb[1] + q.NA[1] * (bb[2] + q.NA[2] * bb[3]));
      }
  }
  c.cl2.nbr.alloc(nbv.size() * sizeof(int));
  TMG_CUDA(cudaMemcpyAsync(c.cl2.nbr.p, nbv.data(), nbv.size() * sizeof(int), cudaMemcpyHostToDevice, c.stream));
  TMG_CUDA(cudaStreamSynchronize(c.stream));
}

}  // namespace tmg
