// Even-odd reduced twisted-mass operator (the paper's simulations use the even-odd reduced
// operator, Sec. 1.2; its CG comparator is an odd-even CG, Fig. 1):
//
//   D(mu) = M(mu) + H,  M(mu) = (4 + m0) + C(x) + i mu g5 (site-local),  H = -1/2 sum_mu hops,
//   Dhat(mu) x_o = M_o x_o - H_oe M_e^-1 H_eo x_o          (Schur complement on the odd sites).
//
// Fields live on half lattices: the sites of one parity p = (x + y + z + t) mod 2 in lexicographic
// order, half-site index i = lex / 2 (Lx even).  Two kernels make one application of Dhat:
//   k_eo_even: t_e = M_e^-1 (b_e + c H_eo x_o)   (c = 1 for Dhat; b and x optional)
//   k_eo_odd : y_o = [M_o x_o | x_o] - H_oe t_e
// with the clover field of the odd sites and the inverse (A + i s mu)^-1 of every even site's two
// chirality blocks (s = +1 / -1) prepared once per (gauge field, kappa, c_sw, mu).  Dhat(mu)^dag =
// g5 Dhat(-mu) g5 uses the same data: M_chi(-mu) = M_chi(mu)^dag because A is Hermitian.
//
// Storage: FP64 links as rows 0 and 1 (12 reals, row 2 = conj(row0 x row1)); FP32 links in 8 reals,
// (U01, U02, U10, arg U00, arg U20): |U00| and |U20| follow from the unit norms of row 0 and of
// column 0, and the four remaining entries from the cofactor relations conj(U) = cof(U) of SU(3),
// e.g. U11 = -(conj(U00) U01 U10 + conj(U02) conj(U20)) / (|U01|^2 + |U02|^2).
//
// Staging: the site-local stream of each CTA (the clover inverse in k_eo_even, the clover field in
// k_eo_odd: contiguous chunks of the structure-of-arrays fields) is copied into shared memory by
// one-dimensional bulk copies (cp.async.bulk, the TMA engine) issued at kernel entry and completed
// on an mbarrier; the gathered neighbour spinors and links are loaded while those copies are in
// flight, and the site-local matrix is read from shared memory afterwards.  The mbarrier wait is
// bounded in wall time; a wait that gives up sets an error flag and the CTA waits (again bounded)
// for its copies before it exits.
#include "tmg_host.h"

namespace tmg {

namespace {

struct EoGeom {
  int L[4];
  int half;
  int tbc;
};

__device__ __forceinline__ void eo_coords(const EoGeom& g, int p, int i, int c[4]) {
  int l = 2 * i;
  c[0] = l % g.L[0]; l /= g.L[0];
  c[1] = l % g.L[1]; l /= g.L[1];
  c[2] = l % g.L[2]; c[3] = l / g.L[2];
  if (((c[0] + c[1] + c[2] + c[3]) & 1) != p) c[0] += 1;
}

__device__ __forceinline__ int eo_index(const EoGeom& g, const int c[4]) {
  return (c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]))) >> 1;
}

__device__ __forceinline__ int eo_nbr(const EoGeom& g, const int c[4], int mu, int dir) {
  int d[4] = {c[0], c[1], c[2], c[3]};
  int v = d[mu] + dir;
  if (v < 0) v += g.L[mu];
  if (v >= g.L[mu]) v -= g.L[mu];
  d[mu] = v;
  return eo_index(g, d);
}

// ---- link formats on a half lattice: [mu][chunk][half]
struct EoGaugeF64 {   // rows 0, 1 as 6 double2
  const double2* p; int half;
  __device__ __forceinline__ void load(int i, int mu, Link<double>& u) const {
#pragma unroll
    for (int k = 0; k < 6; k++) { const double2 v = __ldg(p + (size_t)(mu * 6 + k) * half + i); u.m[k] = {v.x, v.y}; }
    reconstruct_row2(u);
  }
};

struct EoGaugeF32x8 {   // 8 reals: (U01, U02), (U10, arg U00, arg U20)
  const float4* p; int half;
  __device__ __forceinline__ void load(int i, int mu, Link<float>& u) const {
    const float4 a = __ldg(p + (size_t)(mu * 2) * half + i);
    const float4 b = __ldg(p + (size_t)(mu * 2 + 1) * half + i);
    const cpx<float> a1 = {a.x, a.y}, a2 = {a.z, a.w}, b0 = {b.x, b.y};
    const float n12 = a.x * a.x + a.y * a.y + a.z * a.z + a.w * a.w;       // |U01|^2 + |U02|^2
    const float r0 = sqrtf(fmaxf(0.f, 1.f - n12));
    float s0, c0, s2, c2;
    sincosf(b.z, &s0, &c0);
    sincosf(b.w, &s2, &c2);
    const cpx<float> a0 = {r0 * c0, r0 * s0};
    const float r2 = sqrtf(fmaxf(0.f, n12 - (b.x * b.x + b.y * b.y)));    // 1 - |U00|^2 - |U10|^2
    const cpx<float> cc = {r2 * c2, r2 * s2};
    const float inv = 1.f / n12;
    const cpx<float> u11 = neg(inv * (conj(a0) * a1 * b0 + conj(a2) * conj(cc)));
    const cpx<float> u12 = inv * (conj(a1) * conj(cc) - conj(a0) * a2 * b0);
    u.m[0] = a0; u.m[1] = a1; u.m[2] = a2;
    u.m[3] = b0; u.m[4] = u11; u.m[5] = u12;
    u.m[6] = cc;
    u.m[7] = conj(a2 * b0 - a0 * u12);
    u.m[8] = conj(a0 * u11 - a1 * b0);
  }
};

// ---- clover inverse of the even sites: per chirality the full 6 x 6 complex (A + i s mu)^-1,
//      element (r, c) at complex index r * 6 + c, [chi][36 complex][half]
template <typename R> struct InvBlock { cpx<R> m[36]; };

// y = Minv x (dag = 0) or Minv^dag x (dag = 1) for one chirality block
template <typename R>
__device__ __forceinline__ void inv_mul(const InvBlock<R>& a, bool dag, const cpx<R>* x, cpx<R>* y) {
#pragma unroll
  for (int r = 0; r < 6; r++) {
    cpx<R> acc = mk<R>(0, 0);
#pragma unroll
    for (int c = 0; c < 6; c++) acc = acc + (dag ? cmul_conj(a.m[c * 6 + r], x[c]) : a.m[r * 6 + c] * x[c]);
    y[r] = acc;
  }
}

// hop sum acc = sum_mu [(1 - g_mu) U_mu(x) v(x+mu) + (1 + g_mu) U_mu(x-mu)^dag v(x-mu)] at the site
// c (parity p, half index i) from the other parity's field v; Uown: links of parity p, Uoth: of 1-p
template <typename R, class S, class G>
__device__ __forceinline__ void eo_hops(const EoGeom& g, const int c[4], int i, const S& v, const G& Uown,
                                        const G& Uoth, bool g5in, Spinor<R>& acc) {
#pragma unroll
  for (int k = 0; k < 12; k++) acc.c[k] = mk<R>(0, 0);
#pragma unroll
  for (int mu = 0; mu < 4; mu++) {
    {
      const int jf = eo_nbr(g, c, mu, +1);
      Spinor<R> q;
      v.load(jf, q);
      if (g5in) {
#pragma unroll
        for (int k = 6; k < 12; k++) q.c[k] = neg(q.c[k]);
      }
      cpx<R> h[6], uh[6];
      spin_project(mu, +1, q, h);
      Link<R> u;
      Uown.load(i, mu, u);
      su3_mul_half(u, false, h, uh);
      if (mu == 3 && c[3] == g.L[3] - 1 && g.tbc < 0) {
#pragma unroll
        for (int k = 0; k < 6; k++) uh[k] = neg(uh[k]);
      }
      spin_reconstruct_add(mu, +1, uh, acc);
    }
    {
      const int jb = eo_nbr(g, c, mu, -1);
      Spinor<R> q;
      v.load(jb, q);
      if (g5in) {
#pragma unroll
        for (int k = 6; k < 12; k++) q.c[k] = neg(q.c[k]);
      }
      cpx<R> h[6], uh[6];
      spin_project(mu, -1, q, h);
      Link<R> u;
      Uoth.load(jb, mu, u);
      su3_mul_half(u, true, h, uh);
      if (mu == 3 && c[3] == 0 && g.tbc < 0) {
#pragma unroll
        for (int k = 0; k < 6; k++) uh[k] = neg(uh[k]);
      }
      spin_reconstruct_add(mu, -1, uh, acc);
    }
  }
}

// ---- bulk-copy staging (one-dimensional cp.async.bulk into shared memory, mbarrier completion)
constexpr unsigned long long kStageWaitNs = 1000000000ull;   // 1 s

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ unsigned long long gtimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}
__device__ __forceinline__ bool stage_wait(uint32_t bar, uint32_t phase) {
  const unsigned long long t0 = gtimer();
  for (unsigned it = 0; it < (1u << 26); it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase), "r"(20000u)
        : "memory");
    if (done) return true;
    if (gtimer() - t0 > kStageWaitNs) return false;
  }
  return false;
}

// Thread 0 copies `nchunk` chunks of `tile` 16-byte elements each, chunk k from src + k * stride
// (elements), into dst + k * tile; the mbarrier completes when all bytes have landed.
__device__ __forceinline__ void stage_issue(const float4* src, size_t stride, int nchunk, int tile, float4* dst,
                                            uint64_t* bar) {
  const uint32_t b = smem_addr(bar);
  const uint32_t bytes = (uint32_t)nchunk * (uint32_t)tile * 16u;
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(b), "r"(bytes) : "memory");
  for (int k = 0; k < nchunk; k++) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(smem_addr(dst + (size_t)k * tile)), "l"(src + (size_t)k * stride), "r"((uint32_t)tile * 16u), "r"(b)
                 : "memory");
  }
}

template <typename R> struct Vec4Of;
template <> struct Vec4Of<float> { using T = float4; };
template <> struct Vec4Of<double> { using T = double2; };

// ---------------------------------------------------------------- kernels
// t_e = M_e^-1 (b_e + hc H_eo x_o), H = -1/2 sum hops; x or b may be null.  dagger: the blocks of
// Dhat(mu)^dag = g5 Dhat(-mu) g5 (input g5 x, Minv^dag); t is then the intermediate of that form.
// STAGE (FP32 only): the CTA's tile of the inverse field is bulk-copied into shared memory.
template <typename R, class S, class G, bool STAGE>
__global__ void __launch_bounds__(128) k_eo_even(EoGeom g, S t, S x, S b, G Ue, G Uo,
                                                 const typename Vec4Of<R>::T* __restrict__ Minv, R hc, int dagger,
                                                 int* err) {
  using V4 = typename Vec4Of<R>::T;
  constexpr int kPer = sizeof(R) == 4 ? 18 : 36;   // 16-byte elements per chirality block
  extern __shared__ float4 sh_stage[];
  __shared__ uint64_t bar;
  const int i0 = blockIdx.x * blockDim.x;
  const int tile = min((int)blockDim.x, g.half - i0);
  if constexpr (STAGE) {
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar)), "r"(1));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0)
      stage_issue(reinterpret_cast<const float4*>(Minv) + i0, (size_t)g.half, 2 * kPer, tile, sh_stage, &bar);
  }
  const int i = i0 + threadIdx.x;
  const bool live = i < g.half;
  int c[4] = {0, 0, 0, 0};
  Spinor<R> h;
  if (live) {
    eo_coords(g, 0, i, c);
    if (x.p) {
      Spinor<R> acc;
      eo_hops<R>(g, c, i, x, Ue, Uo, dagger != 0, acc);
#pragma unroll
      for (int k = 0; k < 12; k++) h.c[k] = (R(-0.5) * hc) * acc.c[k];
    } else {
#pragma unroll
      for (int k = 0; k < 12; k++) h.c[k] = mk<R>(0, 0);
    }
    if (b.p) {
      Spinor<R> bs;
      b.load(i, bs);
      if (dagger) {
#pragma unroll
        for (int k = 6; k < 12; k++) bs.c[k] = neg(bs.c[k]);
      }
#pragma unroll
      for (int k = 0; k < 12; k++) h.c[k] = h.c[k] + bs.c[k];
    }
  }
  bool ok = true;
  if constexpr (STAGE) {
    ok = stage_wait(smem_addr(&bar), 0);
    if (!ok && threadIdx.x == 0) atomicExch(err, 1);
  }
  if (live && ok) {
    Spinor<R> out;
#pragma unroll
    for (int chi = 0; chi < 2; chi++) {
      InvBlock<R> a;
#pragma unroll
      for (int k = 0; k < kPer; k++) {
        V4 v;
        if constexpr (STAGE) v = sh_stage[(size_t)(chi * kPer + k) * tile + threadIdx.x];
        else v = __ldg(Minv + (size_t)(chi * kPer + k) * g.half + i);
        if constexpr (sizeof(R) == 4) {
          a.m[2 * k] = {v.x, v.y};
          a.m[2 * k + 1] = {v.z, v.w};
        } else {
          a.m[k] = {v.x, v.y};
        }
      }
      inv_mul(a, dagger != 0, &h.c[6 * chi], &out.c[6 * chi]);
    }
    t.store(i, out);
  }
  if constexpr (STAGE) {
    if (!ok) stage_wait(smem_addr(&bar), 0);   // let the copies land before the CTA's memory goes away
  }
}

// y_o = [M_o(mu) x_o  (usem) | x_o] - H_oe t_e; dagger: y = g5 [M_o(-mu) g5 x - H_oe t] with t from the
// dagger form of k_eo_even.  STAGE: the CTA's tile of the clover field is bulk-copied into shared memory.
template <typename R, class S, class G, class C, bool STAGE>
__global__ void __launch_bounds__(128) k_eo_odd(EoGeom g, S y, S x, S t, G Uo, G Ue, C Ao, R mu, int usem,
                                                int dagger, int* err) {
  extern __shared__ float4 sh_stage[];
  __shared__ uint64_t bar;
  const int i0 = blockIdx.x * blockDim.x;
  const int tile = min((int)blockDim.x, g.half - i0);
  if constexpr (STAGE) {
    if (threadIdx.x == 0) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(&bar)), "r"(1));
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    __syncthreads();
    if (threadIdx.x == 0 && usem) stage_issue(reinterpret_cast<const float4*>(Ao.p) + i0, (size_t)g.half, 18, tile, sh_stage, &bar);
  }
  const int i = i0 + threadIdx.x;
  const bool live = i < g.half;
  int c[4] = {0, 0, 0, 0};
  Spinor<R> acc, xs;
  if (live) {
    eo_coords(g, 1, i, c);
    eo_hops<R>(g, c, i, t, Uo, Ue, false, acc);
    x.load(i, xs);
    if (dagger) {
#pragma unroll
      for (int k = 6; k < 12; k++) xs.c[k] = neg(xs.c[k]);
    }
  }
  bool ok = true;
  if constexpr (STAGE) {
    if (usem) {
      ok = stage_wait(smem_addr(&bar), 0);
      if (!ok && threadIdx.x == 0) atomicExch(err, 1);
    }
  }
  if (live && ok) {
    Spinor<R> out;
    if (usem) {
      const R tw = dagger ? -mu : mu;
#pragma unroll
      for (int chi = 0; chi < 2; chi++) {
        CloverBlock<R> a;
        if constexpr (STAGE) {
#pragma unroll
          for (int k = 0; k < 9; k++) {
            const float4 v = sh_stage[(size_t)(chi * 9 + k) * tile + threadIdx.x];
            a.v[4 * k] = v.x; a.v[4 * k + 1] = v.y; a.v[4 * k + 2] = v.z; a.v[4 * k + 3] = v.w;
          }
        } else {
          Ao.load(i, chi, a);
        }
        clover_mul(a, chi == 0 ? tw : -tw, &xs.c[6 * chi], &out.c[6 * chi]);
      }
    } else {
#pragma unroll
      for (int k = 0; k < 12; k++) out.c[k] = xs.c[k];
    }
#pragma unroll
    for (int k = 0; k < 12; k++) out.c[k] = out.c[k] + R(0.5) * acc.c[k];
    if (dagger) {
#pragma unroll
      for (int k = 6; k < 12; k++) out.c[k] = neg(out.c[k]);
    }
    y.store(i, out);
  }
  if constexpr (STAGE) {
    if (usem && !ok) stage_wait(smem_addr(&bar), 0);
  }
}

// ---------------------------------------------------------------- preparation
// links of parity p from the internal block-major FP64 links: FP64 12-real and FP32 8-real
__global__ void k_eo_pack_links(Geom g, EoGeom e, const double2* __restrict__ U, double2* __restrict__ U64e,
                                double2* __restrict__ U64o, float4* __restrict__ U32e, float4* __restrict__ U32o) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int i = eo_index(e, c);
  double2* U64 = p ? U64o : U64e;
  float4* U32 = p ? U32o : U32e;
  for (int mu = 0; mu < 4; mu++) {
    double2 m[9];
    for (int k = 0; k < 9; k++) m[k] = U[(size_t)(mu * 9 + k) * g.V + s];
    for (int k = 0; k < 6; k++) U64[(size_t)(mu * 6 + k) * e.half + i] = m[k];
    U32[(size_t)(mu * 2) * e.half + i] = make_float4((float)m[1].x, (float)m[1].y, (float)m[2].x, (float)m[2].y);
    U32[(size_t)(mu * 2 + 1) * e.half + i] =
        make_float4((float)m[3].x, (float)m[3].y, (float)atan2(m[0].y, m[0].x), (float)atan2(m[6].y, m[6].x));
  }
}

// odd sites: the clover field A (FP64 and FP32); even sites: (A_chi + i s mu)^-1, s = +1 / -1 for
// chi = 0 / 1, by Gauss-Jordan elimination with partial pivoting in FP64
__global__ void k_eo_pack_clover(Geom g, EoGeom e, const double2* __restrict__ A, double mu, double2* __restrict__ Ao64,
                                 float4* __restrict__ Ao32, double2* __restrict__ Mi64, float4* __restrict__ Mi32,
                                 int* __restrict__ singular) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= g.V) return;
  int c[4];
  site_coords(g, s, c);
  const int p = (c[0] + c[1] + c[2] + c[3]) & 1;
  const int i = eo_index(e, c);
  for (int chi = 0; chi < 2; chi++) {
    double v[36];
    for (int k = 0; k < 18; k++) {
      const double2 q = A[(size_t)(chi * 18 + k) * g.V + s];
      v[2 * k] = q.x;
      v[2 * k + 1] = q.y;
    }
    if (p == 1) {
      for (int k = 0; k < 18; k++) Ao64[(size_t)(chi * 18 + k) * e.half + i] = make_double2(v[2 * k], v[2 * k + 1]);
      for (int k = 0; k < 9; k++)
        Ao32[(size_t)(chi * 9 + k) * e.half + i] =
            make_float4((float)v[4 * k], (float)v[4 * k + 1], (float)v[4 * k + 2], (float)v[4 * k + 3]);
      continue;
    }
    // dense 6 x 6: M = A + i s mu, then [M | I] -> [I | M^-1]
    cpx<double> m[6][6], inv[6][6];
    for (int r = 0; r < 6; r++)
      for (int q = 0; q < 6; q++) inv[r][q] = mk(r == q ? 1.0 : 0.0, 0.0);
    for (int r = 0; r < 6; r++) m[r][r] = mk(v[r], chi == 0 ? mu : -mu);
    for (int r = 1; r < 6; r++)
      for (int q = 0; q < r; q++) {
        const int t = 6 + 2 * tri_index(r, q);
        m[r][q] = mk(v[t], v[t + 1]);
        m[q][r] = mk(v[t], -v[t + 1]);
      }
    for (int col = 0; col < 6; col++) {
      int piv = col;
      double best = 0.0;
      for (int r = col; r < 6; r++) {
        const double a = m[r][col].re * m[r][col].re + m[r][col].im * m[r][col].im;
        if (a > best) { best = a; piv = r; }
      }
      if (!(best > 0.0)) { atomicExch(singular, 1); best = 1.0; }
      if (piv != col)
        for (int q = 0; q < 6; q++) {
          const cpx<double> t1 = m[col][q]; m[col][q] = m[piv][q]; m[piv][q] = t1;
          const cpx<double> t2 = inv[col][q]; inv[col][q] = inv[piv][q]; inv[piv][q] = t2;
        }
      const cpx<double> d = m[col][col];
      const double dn = d.re * d.re + d.im * d.im;
      const cpx<double> di = dn > 0.0 ? mk(d.re / dn, -d.im / dn) : mk(0.0, 0.0);
      for (int q = 0; q < 6; q++) { m[col][q] = di * m[col][q]; inv[col][q] = di * inv[col][q]; }
      for (int r = 0; r < 6; r++) {
        if (r == col) continue;
        const cpx<double> f = m[r][col];
        for (int q = 0; q < 6; q++) { m[r][q] = m[r][q] - f * m[col][q]; inv[r][q] = inv[r][q] - f * inv[col][q]; }
      }
    }
    for (int r = 0; r < 6; r++)
      for (int q = 0; q < 6; q++) Mi64[(size_t)(chi * 36 + r * 6 + q) * e.half + i] = make_double2(inv[r][q].re, inv[r][q].im);
    for (int k = 0; k < 18; k++) {
      const cpx<double> a = inv[(2 * k) / 6][(2 * k) % 6], b = inv[(2 * k + 1) / 6][(2 * k + 1) % 6];
      Mi32[(size_t)(chi * 18 + k) * e.half + i] = make_float4((float)a.re, (float)a.im, (float)b.re, (float)b.im);
    }
  }
}

// full-lattice lexicographic FP64 <-> half-lattice internal field of parity p (F64 or F32)
template <typename T2>
__global__ void k_eo_from_lex(EoGeom e, int p, const double2* __restrict__ lex, T2* __restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.half) return;
  int c[4];
  eo_coords(e, p, i, c);
  const size_t l = (size_t)c[0] + (size_t)e.L[0] * (c[1] + (size_t)e.L[1] * (c[2] + (size_t)e.L[2] * c[3]));
  for (int k = 0; k < 12; k++) {
    const double2 v = lex[l * 12 + k];
    T2 o;
    o.x = v.x;
    o.y = v.y;
    out[spinor_flat(e.half, i, k)] = o;
  }
}

template <typename T2>
__global__ void k_eo_to_lex(EoGeom e, int p, const T2* __restrict__ in, double2* __restrict__ lex, int zero_other) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= e.half) return;
  int c[4];
  eo_coords(e, p, i, c);
  const size_t l = (size_t)c[0] + (size_t)e.L[0] * (c[1] + (size_t)e.L[1] * (c[2] + (size_t)e.L[2] * c[3]));
  for (int k = 0; k < 12; k++) {
    const T2 v = in[spinor_flat(e.half, i, k)];
    lex[l * 12 + k] = make_double2((double)v.x, (double)v.y);
  }
  if (zero_other) {   // the partner site of the other parity (x +- 1 in the same lexicographic pair)
    const size_t lo = l ^ 1;
    for (int k = 0; k < 12; k++) lex[lo * 12 + k] = make_double2(0.0, 0.0);
  }
}

EoGeom eo_geom(const Ctx& c) {
  EoGeom e;
  for (int mu = 0; mu < 4; mu++) e.L[mu] = c.g.L[mu];
  e.half = c.g.V / 2;
  e.tbc = c.g.tbc;
  return e;
}

}  // namespace

// Prepare the even-odd data for the context's field and twist (no-op when current).
void eo_prepare(Ctx& c) {
  EoData& d = c.eo;
  if (d.ready && d.mu == c.mu) return;
  if (c.g.L[0] % 2) throw Error{TMG_ERR_ARG, "even-odd operator: Lx must be even"};
  const EoGeom e = eo_geom(c);
  const size_t h = e.half;
  if (!d.ready) {
    d.U64[0].alloc(h * 24 * sizeof(double2));
    d.U64[1].alloc(h * 24 * sizeof(double2));
    d.U32[0].alloc(h * 8 * sizeof(float4));
    d.U32[1].alloc(h * 8 * sizeof(float4));
  }
  d.Ao64.alloc(h * 36 * sizeof(double2));
  d.Ao32.alloc(h * 18 * sizeof(float4));
  d.Mi64.alloc(h * 72 * sizeof(double2));
  d.Mi32.alloc(h * 36 * sizeof(float4));
  d.flag.alloc(2 * sizeof(int));
  TMG_CUDA(cudaMemsetAsync(d.flag.p, 0, 2 * sizeof(int), c.stream));
  const int G = (c.g.V + 127) / 128;
  if (!d.ready) {
    ++c.launches, k_eo_pack_links<<<G, 128, 0, c.stream>>>(c.g, e, c.op[0].U.as<double2>(), d.U64[0].as<double2>(),
                                                           d.U64[1].as<double2>(), d.U32[0].as<float4>(), d.U32[1].as<float4>());
    TMG_CHECK_LAUNCH();
  }
  ++c.launches, k_eo_pack_clover<<<G, 128, 0, c.stream>>>(c.g, e, c.op[0].A.as<double2>(), c.mu, d.Ao64.as<double2>(),
                                                          d.Ao32.as<float4>(), d.Mi64.as<double2>(), d.Mi32.as<float4>(),
                                                          d.flag.as<int>());
  TMG_CHECK_LAUNCH();
  int sing = 0;
  TMG_CUDA(cudaMemcpyAsync(&sing, d.flag.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  TMG_CUDA(cudaStreamSynchronize(c.stream));
  if (sing) throw Error{TMG_ERR_BREAKDOWN, "even-odd operator: a site block A + i mu g5 is singular"};
  d.ready = true;
  d.mu = c.mu;
}

static int eo_err_flag(Ctx& c) {
  int f = 0;
  TMG_CUDA(cudaMemcpyAsync(&f, c.eo.flag.as<int>() + 1, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
  TMG_CUDA(cudaStreamSynchronize(c.stream));
  return f;
}

// One even-odd kernel pair on half-lattice fields of precision prec (F64: 12-real links; F32:
// 8-real links).  which = 0: t = M_e^-1 (b + hc H_eo x) (x, b may be null); which = 1: y = [M_o x |
// x] - H_oe t.  dagger selects the blocks of Dhat^dag.
void eo_kernel(Ctx& c, int prec, int which, void* out, const void* x, const void* bt, double hc, int usem, int dagger) {
  const EoGeom e = eo_geom(c);
  const int threads = 128, blocks = (e.half + threads - 1) / threads;
  EoData& d = c.eo;
  int* err = d.flag.as<int>() + 1;
  const bool stage = c.eo_stage != 0;
  static bool smem_set = false;
  if (stage && !smem_set) {   // the staged inverse tile needs more than the default 48 KB
    TMG_CUDA(cudaFuncSetAttribute((const void*)k_eo_even<float, SpinorF32, EoGaugeF32x8, true>,
                                  cudaFuncAttributeMaxDynamicSharedMemorySize, 36 * threads * (int)sizeof(float4)));
    smem_set = true;
  }
  ProfScope ps(c, prec == TMG_PREC_F64 ? PK_EO_F64 : PK_EO_F32);
  if (prec == TMG_PREC_F64) {
    const SpinorF64 o{(double2*)out, e.half}, xs{(double2*)x, e.half}, bs{(double2*)bt, e.half};
    const EoGaugeF64 Ue{d.U64[0].as<double2>(), e.half}, Uo{d.U64[1].as<double2>(), e.half};
    if (which == 0)
      ++c.launches, k_eo_even<double, SpinorF64, EoGaugeF64, false><<<blocks, threads, 0, c.stream>>>(
                        e, o, xs, bs, Ue, Uo, d.Mi64.as<double2>(), hc, dagger, err);
    else
      ++c.launches, k_eo_odd<double, SpinorF64, EoGaugeF64, CloverF64, false><<<blocks, threads, 0, c.stream>>>(
                        e, o, xs, bs, Uo, Ue, CloverF64{d.Ao64.as<double2>(), e.half}, c.mu, usem, dagger, err);
  } else {
    const SpinorF32 o{(float4*)out, e.half}, xs{(float4*)x, e.half}, bs{(float4*)bt, e.half};
    const EoGaugeF32x8 Ue{d.U32[0].as<float4>(), e.half}, Uo{d.U32[1].as<float4>(), e.half};
    if (which == 0) {
      if (stage)
        ++c.launches, k_eo_even<float, SpinorF32, EoGaugeF32x8, true><<<blocks, threads, 36 * threads * sizeof(float4), c.stream>>>(
                          e, o, xs, bs, Ue, Uo, d.Mi32.as<float4>(), (float)hc, dagger, err);
      else
        ++c.launches, k_eo_even<float, SpinorF32, EoGaugeF32x8, false><<<blocks, threads, 0, c.stream>>>(
                          e, o, xs, bs, Ue, Uo, d.Mi32.as<float4>(), (float)hc, dagger, err);
    } else {
      if (stage)
        ++c.launches, k_eo_odd<float, SpinorF32, EoGaugeF32x8, CloverF32, true><<<blocks, threads, 18 * threads * sizeof(float4), c.stream>>>(
                          e, o, xs, bs, Uo, Ue, CloverF32{d.Ao32.as<float4>(), e.half}, (float)c.mu, usem, dagger, err);
      else
        ++c.launches, k_eo_odd<float, SpinorF32, EoGaugeF32x8, CloverF32, false><<<blocks, threads, 0, c.stream>>>(
                          e, o, xs, bs, Uo, Ue, CloverF32{d.Ao32.as<float4>(), e.half}, (float)c.mu, usem, dagger, err);
    }
  }
  TMG_CHECK_LAUNCH();
}

// y_o = Dhat x_o (dagger: Dhat^dag) on half-lattice fields; t: half-lattice scratch (even sites)
void eo_apply(Ctx& c, int prec, void* y, const void* x, void* t, int dagger) {
  eo_kernel(c, prec, 0, t, x, nullptr, 1.0, 1, dagger);
  eo_kernel(c, prec, 1, y, x, t, 1.0, 1, dagger);
}

void eo_check(Ctx& c) {
  if (eo_err_flag(c)) throw Error{TMG_ERR_TIMEOUT, "even-odd operator: a staging wait gave up"};
}

void eo_from_lex(Ctx& c, const double* lex, void* out, int parity, int prec) {
  const EoGeom e = eo_geom(c);
  const int G = (e.half + 127) / 128;
  if (prec == TMG_PREC_F64)
    ++c.launches, k_eo_from_lex<double2><<<G, 128, 0, c.stream>>>(e, parity, (const double2*)lex, (double2*)out);
  else
    ++c.launches, k_eo_from_lex<float2><<<G, 128, 0, c.stream>>>(e, parity, (const double2*)lex, (float2*)out);
  TMG_CHECK_LAUNCH();
}

void eo_to_lex(Ctx& c, const void* in, double* lex, int parity, int prec, int zero_other) {
  const EoGeom e = eo_geom(c);
  const int G = (e.half + 127) / 128;
  if (prec == TMG_PREC_F64)
    ++c.launches, k_eo_to_lex<double2><<<G, 128, 0, c.stream>>>(e, parity, (const double2*)in, (double2*)lex, zero_other);
  else
    ++c.launches, k_eo_to_lex<float2><<<G, 128, 0, c.stream>>>(e, parity, (const float2*)in, (double2*)lex, zero_other);
  TMG_CHECK_LAUNCH();
}

}  // namespace tmg
