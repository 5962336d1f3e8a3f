// Multi-right-hand-side ("batched") versions of the fine-level kernels: many columns with their
// own twist mu_c (multi-shift systems map to twists, Sec. 1.1: the same P serves every mu) go
// through one launch per operation.
//
//   k_dslash_mrhs : every thread loops over the columns of its site, so the site's links and
//                   clover are fetched from DRAM once and re-read from L1 for the other columns;
//   k_sap_mrhs    : one CTA per (block of a colour, column);
//   k_restrict_mrhs / k_prolong_mrhs: one CTA per (aggregate, column).
// Column c of a batched field starts at c * 12 V complex numbers (F32 storage, see
// tmg_internal.cuh).
#include "dslash_core.cuh"
#include "tmg_host.h"

namespace tmg {

namespace {

template <class G, class C>
__global__ void __launch_bounds__(128) k_dslash_mrhs(Geom g, int ncol, SpinorF32 y, SpinorF32 x, SpinorF32 b,
                                                     G U, C A, const float* __restrict__ mu_col, int mode) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  const SiteCoord sc = decode_site(g, s);
  for (int col = 0; col < ncol; col++) {
    const SpinorF32 xc = x.column(col), yc = y.column(col);
    Spinor<float> out;
    apply_D_site<float>(g, sc, s, xc, U, A, mu_col[col], out);
    if (mode == 1) {
      Spinor<float> bs;
      b.column(col).load(s, bs);
#pragma unroll
      for (int k = 0; k < 12; k++) out.c[k] = bs.c[k] - out.c[k];
    }
    yc.store(s, out);
  }
}

// k-th block of the given colour (colour = parity of the block coordinates; NB[0] is even).
__device__ __forceinline__ int colour_block_b(const Geom& g, int colour, int k) {
  const int half = g.NB[0] >> 1;
  const int row = k / half, j = k - row * half;
  const int b1 = row % g.NB[1], r2 = row / g.NB[1];
  const int b2 = r2 % g.NB[2], b3 = r2 / g.NB[2];
  const int b0 = 2 * j + ((colour + b1 + b2 + b3) & 1);
  return row * g.NB[0] + b0;
}

// CTA all-reduce of N floats, in FP32 throughout (red: shared scratch of at least 33 * N doubles)
template <int N>
__device__ __forceinline__ void cta_allreduce_f(float (&v)[N], double* red_d) {
  float* red = reinterpret_cast<float*>(red_d);
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
#pragma unroll
  for (int i = 0; i < N; i++) {
    float a = v[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
    if (lane == 0) red[w * N + i] = a;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < N; i += blockDim.x) {
    float a = 0.f;
    for (int k = 0; k < nw; k++) a += red[k * N + i];
    red[32 * N + i] = a;
  }
  __syncthreads();
#pragma unroll
  for (int i = 0; i < N; i++) v[i] = red[32 * N + i];
  __syncthreads();
}

// Same block solve as k_sap_block (k_mg.cu), one column per blockIdx.y with its own twist.
template <class G, class C>
__global__ void __launch_bounds__(256, 2) k_sap_mrhs(Geom g, int colour, SpinorF32 x, SpinorF32 b, G U, C A,
                                                     const float* __restrict__ mu_col, int n_mr) {
  extern __shared__ double smem_d[];
  cpx<float>* rs = reinterpret_cast<cpx<float>*>(smem_d);
  double* red = smem_d + (sizeof(cpx<float>) * 12 * g.VB) / sizeof(double);
  const int col = blockIdx.y;
  const float tw = mu_col[col];
  const SpinorF32 xc = x.column(col), bc = b.column(col);
  const int blk = colour_block_b(g, colour, blockIdx.x);
  const int t = threadIdx.x;
  const int s = blk * g.VB + t;
  const SiteCoord sc = decode_site(g, s);
  Spinor<float> r;
  {
    Spinor<float> dx, bs;
    apply_D_site<float>(g, sc, s, xc, U, A, tw, dx);
    bc.load(s, bs);
#pragma unroll
    for (int k = 0; k < 12; k++) r.c[k] = bs.c[k] - dx.c[k];
  }
  Spinor<float> e;
#pragma unroll
  for (int k = 0; k < 12; k++) e.c[k] = mk<float>(0, 0);
  for (int it = 0; it < n_mr; it++) {
#pragma unroll
    for (int k = 0; k < 12; k++) rs[k * g.VB + t] = r.c[k];
    __syncthreads();
    Spinor<float> acc;
#pragma unroll
    for (int k = 0; k < 12; k++) acc.c[k] = mk<float>(0, 0);
#pragma unroll
    for (int mu = 0; mu < 4; mu++) {
      if (sc.l[mu] + 1 < g.B[mu]) {
        const int tf = t + g.ls[mu];
        Spinor<float> p;
#pragma unroll
        for (int k = 0; k < 12; k++) p.c[k] = rs[k * g.VB + tf];
        cpx<float> h[6], uh[6];
        spin_project(mu, +1, p, h);
        Link<float> u;
        U.load(s, mu, u);
        su3_mul_half(u, false, h, uh);
        spin_reconstruct_add(mu, +1, uh, acc);
      }
      if (sc.l[mu] > 0) {
        const int tb = t - g.ls[mu];
        Spinor<float> p;
#pragma unroll
        for (int k = 0; k < 12; k++) p.c[k] = rs[k * g.VB + tb];
        cpx<float> h[6], uh[6];
        spin_project(mu, -1, p, h);
        Link<float> u;
        U.load(s - g.ls[mu], mu, u);
        su3_mul_half(u, true, h, uh);
        spin_reconstruct_add(mu, -1, uh, acc);
      }
    }
    Spinor<float> p;
#pragma unroll
    for (int chi = 0; chi < 2; chi++) {
      CloverBlock<float> a;
      A.load(s, chi, a);
      clover_mul(a, chi == 0 ? tw : -tw, &r.c[6 * chi], &p.c[6 * chi]);
    }
#pragma unroll
    for (int k = 0; k < 12; k++) p.c[k] = p.c[k] - 0.5f * acc.c[k];
    float v[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 12; k++) {
      v[0] += p.c[k].re * p.c[k].re + p.c[k].im * p.c[k].im;
      const cpx<float> q = cmul_conj(p.c[k], r.c[k]);
      v[1] += q.re;
      v[2] += q.im;
    }
    cta_allreduce_f<3>(v, red);
    const cpx<float> alpha = v[0] > 0.f ? mk(v[1] / v[0], v[2] / v[0]) : mk<float>(0, 0);
#pragma unroll
    for (int k = 0; k < 12; k++) {
      e.c[k] = e.c[k] + alpha * r.c[k];
      r.c[k] = r.c[k] - alpha * p.c[k];
    }
  }
  Spinor<float> xs;
  xc.load(s, xs);
#pragma unroll
  for (int k = 0; k < 12; k++) xs.c[k] = xs.c[k] + e.c[k];
  xc.store(s, xs);
}

// out[col][blk][chi * nv + j] = <W_j P_chi, r_col> over the aggregate
__global__ void __launch_bounds__(256) k_restrict_mrhs(Geom g, SpinorF32 r, SpinorF32 W, int nv, float2* __restrict__ out) {
  extern __shared__ double red[];
  const int blk = blockIdx.x, col = blockIdx.y;
  const int s = blk * g.VB + threadIdx.x;
  Spinor<float> rv;
  r.column(col).load(s, rv);
  const int nd = 2 * nv;
  float2* o = out + (size_t)col * g.nblk * nd;
  for (int j0 = 0; j0 < nv; j0 += 8) {
    float v[32];
#pragma unroll
    for (int i = 0; i < 32; i++) v[i] = 0;
#pragma unroll
    for (int jj = 0; jj < 8; jj++) {
      const int j = j0 + jj;
      if (j < nv) {
        Spinor<float> wv;
        W.column(j).load(s, wv);
#pragma unroll
        for (int k = 0; k < 12; k++) {
          const cpx<float> q = cmul_conj(wv.c[k], rv.c[k]);
          v[((k / 6) * 8 + jj) * 2] += q.re;
          v[((k / 6) * 8 + jj) * 2 + 1] += q.im;
        }
      }
    }
    cta_allreduce_f<32>(v, red);
    if (threadIdx.x < 16) {
      const int chi = threadIdx.x / 8, jj = threadIdx.x % 8, j = j0 + jj;
      if (j < nv) o[(size_t)blk * nd + chi * nv + j] = make_float2(v[(chi * 8 + jj) * 2], v[(chi * 8 + jj) * 2 + 1]);
    }
  }
}

// e_col(s)_chi = sum_j W_j(s)_chi c_col[blk][chi * nv + j]
__global__ void __launch_bounds__(256) k_prolong_mrhs(Geom g, const float2* __restrict__ cv, SpinorF32 W, int nv, SpinorF32 e) {
  extern __shared__ double smem_p[];
  cpx<float>* cs = reinterpret_cast<cpx<float>*>(smem_p);
  const int blk = blockIdx.x, col = blockIdx.y;
  const int nd = 2 * nv;
  const float2* c = cv + (size_t)col * g.nblk * nd;
  for (int i = threadIdx.x; i < nd; i += blockDim.x) cs[i] = mk(c[(size_t)blk * nd + i].x, c[(size_t)blk * nd + i].y);
  __syncthreads();
  const int s = blk * g.VB + threadIdx.x;
  Spinor<float> out;
#pragma unroll
  for (int k = 0; k < 12; k++) out.c[k] = mk<float>(0, 0);
  for (int j = 0; j < nv; j++) {
    Spinor<float> wv;
    W.column(j).load(s, wv);
    const cpx<float> cp = cs[j], cm = cs[nv + j];
#pragma unroll
    for (int k = 0; k < 6; k++) out.c[k] = out.c[k] + wv.c[k] * cp;
#pragma unroll
    for (int k = 6; k < 12; k++) out.c[k] = out.c[k] + wv.c[k] * cm;
  }
  e.column(col).store(s, out);
}

}  // namespace

void dslash_mrhs(Ctx& c, int prec, int ncol, void* y, const void* x, const void* b, const float* mu_col_dev, int mode) {
  ProfScope ps(c, prec == TMG_PREC_F16 ? PK_DSLASH_F16 : PK_DSLASH_F32);
  const int blocks = (c.g.V + 127) / 128;
  const SpinorF32 ys{(float4*)y, c.g.V}, xs{(float4*)x, c.g.V}, bs{(float4*)(b ? b : x), c.g.V};
  if (prec == TMG_PREC_F16)
    ++c.launches, k_dslash_mrhs<<<blocks, 128, 0, c.stream>>>(c.g, ncol, ys, xs, bs, GaugeF16{c.op[2].U.as<short4>(), c.g.V},
                                                      CloverF16{c.op[2].A.as<short4>(), c.op[2].Ascale.as<float>(), c.g.V}, mu_col_dev, mode);
  else
    ++c.launches, k_dslash_mrhs<<<blocks, 128, 0, c.stream>>>(c.g, ncol, ys, xs, bs, GaugeF32{c.op[1].U.as<float4>(), c.g.V},
                                                      CloverF32{c.op[1].A.as<float4>(), c.g.V}, mu_col_dev, mode);
  TMG_CHECK_LAUNCH();
}

void sap_mrhs(Ctx& c, int prec, int ncol, void* x, const void* b, const float* mu_col_dev, int n_sweeps) {
  const size_t smem = sizeof(cpx<float>) * 12 * c.g.VB + 33 * 3 * sizeof(double);
  const SpinorF32 xs{(float4*)x, c.g.V}, bs{(float4*)b, c.g.V};
  const dim3 grid(c.g.nblk / 2, ncol);
  for (int sw = 0; sw < n_sweeps; sw++)
    for (int colour = 0; colour < 2; colour++) {
      ProfScope ps(c, prec == TMG_PREC_F16 ? PK_SAP_F16 : PK_SAP_F32);
      if (prec == TMG_PREC_F16)
        ++c.launches, k_sap_mrhs<<<grid, c.g.VB, smem, c.stream>>>(c.g, colour, xs, bs, GaugeF16{c.op[2].U.as<short4>(), c.g.V},
                                                          CloverF16{c.op[2].A.as<short4>(), c.op[2].Ascale.as<float>(), c.g.V},
                                                          mu_col_dev, c.mg.sap_mr);
      else
        ++c.launches, k_sap_mrhs<<<grid, c.g.VB, smem, c.stream>>>(c.g, colour, xs, bs, GaugeF32{c.op[1].U.as<float4>(), c.g.V},
                                                          CloverF32{c.op[1].A.as<float4>(), c.g.V}, mu_col_dev, c.mg.sap_mr);
      TMG_CHECK_LAUNCH();
    }
}

void restrict_mrhs(Ctx& c, int ncol, const void* r, void* cvec) {
  ProfScope ps(c, PK_RESTRICT);
  const size_t smem = 33 * 32 * sizeof(double);
  ++c.launches, k_restrict_mrhs<<<dim3(c.g.nblk, ncol), c.g.VB, smem, c.stream>>>(
      c.g, SpinorF32{(float4*)r, c.g.V}, SpinorF32{c.cl.W32.as<float4>(), c.g.V}, c.cl.nv, (float2*)cvec);
  TMG_CHECK_LAUNCH();
}

void prolong_mrhs(Ctx& c, int ncol, const void* cvec, void* e) {
  ProfScope ps(c, PK_PROLONG);
  const size_t smem = 2 * c.cl.nv * sizeof(cpx<float>);
  ++c.launches, k_prolong_mrhs<<<dim3(c.g.nblk, ncol), c.g.VB, smem, c.stream>>>(
      c.g, (const float2*)cvec, SpinorF32{c.cl.W32.as<float4>(), c.g.V}, c.cl.nv, SpinorF32{(float4*)e, c.g.V});
  TMG_CHECK_LAUNCH();
}

}  // namespace tmg
