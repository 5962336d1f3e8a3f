// Multi-right-hand-side ("batched") versions of the fine-level kernels: many columns with their
// own twist mu_c (multi-shift systems map to twists, Sec. 1.1: the same P serves every mu) go
// through one launch per operation.
//
//   k_dslash_mrhs : every thread loops over the columns of its site, so the site's links and
//                   clover are fetched from DRAM once and re-read from L1 for the other columns;
//   k_restrict_mrhs / k_prolong_mrhs: one CTA per (aggregate, column), the column index running
//                   fastest over the CTAs, so the CTAs that share an aggregate's test vectors run
//                   together and find them in L2 (read from DRAM about once per launch instead of
//                   once per column).
// (The multi-column SAP is k_sap_block's multi-column form, k_mg.cu.)
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

// out[col][blk][chi * nv + j] = <W_j P_chi, r_col> over the aggregate
__global__ void __launch_bounds__(256) k_restrict_mrhs(Geom g, int ncol, SpinorF32 r, SpinorF32 W, int nv,
                                                       float2* __restrict__ out) {
  extern __shared__ double red[];
  const int blk = blockIdx.x / ncol, col = blockIdx.x % ncol;
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
__global__ void __launch_bounds__(256) k_prolong_mrhs(Geom g, int ncol, const float2* __restrict__ cv, SpinorF32 W, int nv,
                                                      SpinorF32 e) {
  extern __shared__ double smem_p[];
  cpx<float>* cs = reinterpret_cast<cpx<float>*>(smem_p);
  const int blk = blockIdx.x / ncol, col = blockIdx.x % ncol;
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

void restrict_mrhs(Ctx& c, int ncol, const void* r, void* cvec) {
  ProfScope ps(c, PK_RESTRICT);
  const size_t smem = 33 * 32 * sizeof(double);
  ++c.launches, k_restrict_mrhs<<<(unsigned)c.g.nblk * (unsigned)ncol, c.g.VB, smem, c.stream>>>(
      c.g, ncol, SpinorF32{(float4*)r, c.g.V}, SpinorF32{c.cl.W32.as<float4>(), c.g.V}, c.cl.nv, (float2*)cvec);
  TMG_CHECK_LAUNCH();
}

void prolong_mrhs(Ctx& c, int ncol, const void* cvec, void* e) {
  ProfScope ps(c, PK_PROLONG);
  const size_t smem = 2 * c.cl.nv * sizeof(cpx<float>);
  ++c.launches, k_prolong_mrhs<<<(unsigned)c.g.nblk * (unsigned)ncol, c.g.VB, smem, c.stream>>>(
      c.g, ncol, (const float2*)cvec, SpinorF32{c.cl.W32.as<float4>(), c.g.V}, c.cl.nv, SpinorF32{(float4*)e, c.g.V});
  TMG_CHECK_LAUNCH();
}

}  // namespace tmg
