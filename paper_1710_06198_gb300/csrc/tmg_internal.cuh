// Internal definitions of libtmg: geometry, complex arithmetic, field storage formats.
//
// Site ordering on the device ("block-major"): the lattice is cut into blocks (the SAP blocks,
// which are also the fine aggregates); sites are numbered block by block,
//   s = blk * VB + loc,
// blk = lexicographic block coordinate, loc = lexicographic coordinate inside the block.  A block
// is then a contiguous range of every field, so one CTA per block reads its block with fully
// coalesced loads, the SAP block solve and the restriction P^dag touch only their own range, and
// the coarse site index equals blk.
//
// Field formats (structure of arrays: component chunk k of site s at ptr[k * V + s]):
//   spinor F64 :  6 chunks of 2 double2 (two complex per chunk, spin-major colour-minor order)
//   spinor F32 :  6 float4  (two complex per chunk)
//   spinor F16 :  3 int4 (8 x int16 fixed point, value = q / 32767 * norm) + float norm[s]
//   links  F64 : per direction 9 double2 (row-major SU(3))
//   links  F32 : per direction 3 float4  (rows 0 and 1; row 2 = conj(row0 x row1))
//   links  F16 : per direction 3 short4  (rows 0 and 1, fixed point scale 1)
//   clover F64 : per chirality 18 double2 = 6 real diagonal (3 double2) + 15 complex lower triangle
//   clover F32 : per chirality 9 float4 (same 36 reals)
//   clover F16 : per chirality 9 short4 + float scale per site (value = q / 32767 * scale)
// The clover field stores A(x) = (4 + m0) + C(x), block-diagonal in chirality (g5 diagonal).
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace tmg {

struct Geom {
  int L[4];    // x, y, z, t
  int B[4];    // block dims
  int NB[4];   // blocks per direction
  int ls[4];   // stride of a local coordinate inside a block: 1, B0, B0 B1, B0 B1 B2
  int bs[4];   // stride of a block coordinate: 1, NB0, NB0 NB1, NB0 NB1 NB2
  int VB;      // sites per block
  int nblk;    // number of blocks
  int V;       // sites
  int tbc;     // time boundary sign
};

// Coordinates of one site, decoded once; neighbours are then found without divisions.
struct SiteCoord {
  int blk, loc;
  int l[4], b[4];
};

__device__ __forceinline__ SiteCoord decode_site(const Geom& g, int s) {
  SiteCoord sc;
  sc.blk = s / g.VB;
  sc.loc = s - sc.blk * g.VB;
  int loc = sc.loc, blk = sc.blk;
  sc.l[0] = loc % g.B[0]; loc /= g.B[0];
  sc.l[1] = loc % g.B[1]; loc /= g.B[1];
  sc.l[2] = loc % g.B[2]; sc.l[3] = loc / g.B[2];
  sc.b[0] = blk % g.NB[0]; blk /= g.NB[0];
  sc.b[1] = blk % g.NB[1]; blk /= g.NB[1];
  sc.b[2] = blk % g.NB[2]; sc.b[3] = blk / g.NB[2];
  return sc;
}

__device__ __forceinline__ int coord(const Geom& g, const SiteCoord& sc, int mu) {
  return sc.b[mu] * g.B[mu] + sc.l[mu];
}

// site index of the neighbour in direction +mu
__device__ __forceinline__ int nbr_fwd(const Geom& g, const SiteCoord& sc, int mu) {
  int loc = sc.loc, blk = sc.blk;
  if (sc.l[mu] + 1 < g.B[mu]) {
    loc += g.ls[mu];
  } else {
    loc -= (g.B[mu] - 1) * g.ls[mu];
    blk += (sc.b[mu] + 1 < g.NB[mu]) ? g.bs[mu] : -(g.NB[mu] - 1) * g.bs[mu];
  }
  return blk * g.VB + loc;
}

// site index of the neighbour in direction -mu
__device__ __forceinline__ int nbr_bwd(const Geom& g, const SiteCoord& sc, int mu) {
  int loc = sc.loc, blk = sc.blk;
  if (sc.l[mu] > 0) {
    loc -= g.ls[mu];
  } else {
    loc += (g.B[mu] - 1) * g.ls[mu];
    blk += (sc.b[mu] > 0) ? -g.bs[mu] : (g.NB[mu] - 1) * g.bs[mu];
  }
  return blk * g.VB + loc;
}

// ------------------------------------------------------------------ complex
template <typename R> struct cpx { R re, im; };

template <typename R> __host__ __device__ __forceinline__ cpx<R> mk(R a, R b) { return {a, b}; }
template <typename R> __device__ __forceinline__ cpx<R> operator+(cpx<R> a, cpx<R> b) { return {a.re + b.re, a.im + b.im}; }
template <typename R> __device__ __forceinline__ cpx<R> operator-(cpx<R> a, cpx<R> b) { return {a.re - b.re, a.im - b.im}; }
template <typename R> __device__ __forceinline__ cpx<R> operator*(cpx<R> a, cpx<R> b) {
  return {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
}
template <typename R> __device__ __forceinline__ cpx<R> operator*(R s, cpx<R> a) { return {s * a.re, s * a.im}; }
template <typename R> __device__ __forceinline__ cpx<R> conj(cpx<R> a) { return {a.re, -a.im}; }
template <typename R> __device__ __forceinline__ cpx<R> mul_i(cpx<R> a) { return {-a.im, a.re}; }     // i a
template <typename R> __device__ __forceinline__ cpx<R> mul_mi(cpx<R> a) { return {a.im, -a.re}; }    // -i a
template <typename R> __device__ __forceinline__ cpx<R> neg(cpx<R> a) { return {-a.re, -a.im}; }
// conj(a) * b
template <typename R> __device__ __forceinline__ cpx<R> cmul_conj(cpx<R> a, cpx<R> b) {
  return {a.re * b.re + a.im * b.im, a.re * b.im - a.im * b.re};
}

// ------------------------------------------------------------------ geometry
__device__ __forceinline__ void site_coords(const Geom& g, int s, int c[4]) {
  int blk = s / g.VB, loc = s - blk * g.VB;
  int l0 = loc % g.B[0]; loc /= g.B[0];
  int l1 = loc % g.B[1]; loc /= g.B[1];
  int l2 = loc % g.B[2]; int l3 = loc / g.B[2];
  int b0 = blk % g.NB[0]; blk /= g.NB[0];
  int b1 = blk % g.NB[1]; blk /= g.NB[1];
  int b2 = blk % g.NB[2]; int b3 = blk / g.NB[2];
  c[0] = b0 * g.B[0] + l0; c[1] = b1 * g.B[1] + l1;
  c[2] = b2 * g.B[2] + l2; c[3] = b3 * g.B[3] + l3;
}

__device__ __forceinline__ int site_index(const Geom& g, const int c[4]) {
  int b0 = c[0] / g.B[0], l0 = c[0] - b0 * g.B[0];
  int b1 = c[1] / g.B[1], l1 = c[1] - b1 * g.B[1];
  int b2 = c[2] / g.B[2], l2 = c[2] - b2 * g.B[2];
  int b3 = c[3] / g.B[3], l3 = c[3] - b3 * g.B[3];
  int blk = b0 + g.NB[0] * (b1 + g.NB[1] * (b2 + g.NB[2] * b3));
  int loc = l0 + g.B[0] * (l1 + g.B[1] * (l2 + g.B[2] * l3));
  return blk * g.VB + loc;
}

__device__ __forceinline__ int lex_index(const Geom& g, const int c[4]) {
  return c[0] + g.L[0] * (c[1] + g.L[1] * (c[2] + g.L[2] * c[3]));
}

// neighbour of site with coordinates c in direction mu, +1 or -1 (periodic wrap)
__device__ __forceinline__ int neighbour(const Geom& g, const int c[4], int mu, int dir) {
  int d[4] = {c[0], c[1], c[2], c[3]};
  int v = d[mu] + dir;
  if (v < 0) v += g.L[mu];
  if (v >= g.L[mu]) v -= g.L[mu];
  d[mu] = v;
  return site_index(g, d);
}

// ------------------------------------------------------------------ spinor storage
// internal flat complex index of (site s, component k) = 2 ((k/2) V + s) + (k%2)
__device__ __forceinline__ size_t spinor_flat(int V, int s, int k) {
  return 2 * ((size_t)(k >> 1) * V + s) + (k & 1);
}

// A spinor in registers: 12 complex, index spin*3 + colour.
template <typename R> struct Spinor { cpx<R> c[12]; };

// F64 and F32 spinors share one logical order of their 12 V complex numbers: component pair k
// (complex 2k, 2k+1) of site s sits at complex index 2 (k V + s) + {0, 1}.  Element-wise BLAS and
// precision conversion therefore treat a field as a flat complex array.
struct SpinorF64 {
  double2* p; int V;
  // the j-th field of a contiguous array of fields
  __host__ __device__ __forceinline__ SpinorF64 column(int j) const { return SpinorF64{p + (size_t)j * 12 * V, V}; }
  __device__ __forceinline__ void load(int s, Spinor<double>& o) const {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      const double2* q = p + 2 * ((size_t)k * V + s);
      double2 a = __ldg(q), b = __ldg(q + 1);
      o.c[2 * k] = {a.x, a.y}; o.c[2 * k + 1] = {b.x, b.y};
    }
  }
  __device__ __forceinline__ void store(int s, const Spinor<double>& o) const {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      double2* q = p + 2 * ((size_t)k * V + s);
      q[0] = make_double2(o.c[2 * k].re, o.c[2 * k].im);
      q[1] = make_double2(o.c[2 * k + 1].re, o.c[2 * k + 1].im);
    }
  }
};

struct SpinorF32 {
  float4* p; int V;
  __host__ __device__ __forceinline__ SpinorF32 column(int j) const { return SpinorF32{p + (size_t)j * 6 * V, V}; }
  __device__ __forceinline__ void load(int s, Spinor<float>& o) const {
#pragma unroll
    for (int k = 0; k < 6; k++) {
      float4 v = __ldg(p + (size_t)k * V + s);
      o.c[2 * k] = {v.x, v.y}; o.c[2 * k + 1] = {v.z, v.w};
    }
  }
  __device__ __forceinline__ void store(int s, const Spinor<float>& o) const {
#pragma unroll
    for (int k = 0; k < 6; k++)
      p[(size_t)k * V + s] = make_float4(o.c[2 * k].re, o.c[2 * k].im, o.c[2 * k + 1].re, o.c[2 * k + 1].im);
  }
};

struct SpinorF16 {
  int4* p; float* nrm; int V;
  __device__ __forceinline__ void load(int s, Spinor<float>& o) const {
    const float sc = __ldg(nrm + s) * (1.0f / 32767.0f);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      int4 v = __ldg(p + (size_t)k * V + s);
      int w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
      for (int h = 0; h < 4; h++) {
        short lo = (short)(w[h] & 0xffff), hi = (short)((unsigned)w[h] >> 16);
        int r = 8 * k + 2 * h;  // real index
        // real index r, r+1 belong to complex r/2
        o.c[r / 2] = {sc * (float)lo, sc * (float)hi};
      }
    }
  }
  __device__ __forceinline__ void store(int s, const Spinor<float>& o) const {
    float m = 0.f;
#pragma unroll
    for (int k = 0; k < 12; k++) m = fmaxf(m, fmaxf(fabsf(o.c[k].re), fabsf(o.c[k].im)));
    nrm[s] = m;
    const float inv = m > 0.f ? 32767.0f / m : 0.f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      int w[4];
#pragma unroll
      for (int h = 0; h < 4; h++) {
        const cpx<float> z = o.c[4 * k + h];
        int lo = __float2int_rn(z.re * inv), hi = __float2int_rn(z.im * inv);
        w[h] = (lo & 0xffff) | ((unsigned)(hi & 0xffff) << 16);
      }
      p[(size_t)k * V + s] = make_int4(w[0], w[1], w[2], w[3]);
    }
  }
};

template <int PREC> struct SpinorOf;
template <> struct SpinorOf<0> { using T = SpinorF64; using R = double; };
template <> struct SpinorOf<1> { using T = SpinorF32; using R = float; };
template <> struct SpinorOf<2> { using T = SpinorF16; using R = float; };

// ------------------------------------------------------------------ SU(3) links
template <typename R> struct Link { cpx<R> m[9]; };

template <typename R> __device__ __forceinline__ void reconstruct_row2(Link<R>& u) {
  // row2 = conj(row0 x row1)
  u.m[6] = conj(u.m[1] * u.m[5] - u.m[2] * u.m[4]);
  u.m[7] = conj(u.m[2] * u.m[3] - u.m[0] * u.m[5]);
  u.m[8] = conj(u.m[0] * u.m[4] - u.m[1] * u.m[3]);
}

struct GaugeF64 {
  double2* p; int V;
  __device__ __forceinline__ void load(int s, int mu, Link<double>& u) const {
#pragma unroll
    for (int k = 0; k < 9; k++) { double2 v = __ldg(p + (size_t)(mu * 9 + k) * V + s); u.m[k] = {v.x, v.y}; }
  }
};

struct GaugeF32 {
  float4* p; int V;
  __device__ __forceinline__ void load(int s, int mu, Link<float>& u) const {
#pragma unroll
    for (int k = 0; k < 3; k++) {
      float4 v = __ldg(p + (size_t)(mu * 3 + k) * V + s);
      u.m[2 * k] = {v.x, v.y}; u.m[2 * k + 1] = {v.z, v.w};
    }
    reconstruct_row2(u);
  }
};

struct GaugeF16 {
  short4* p; int V;
  __device__ __forceinline__ void load(int s, int mu, Link<float>& u) const {
    const float sc = 1.0f / 32767.0f;
#pragma unroll
    for (int k = 0; k < 3; k++) {
      short4 v = __ldg(p + (size_t)(mu * 3 + k) * V + s);
      u.m[2 * k] = {sc * v.x, sc * v.y}; u.m[2 * k + 1] = {sc * v.z, sc * v.w};
    }
    reconstruct_row2(u);
  }
};

template <int PREC> struct GaugeOf;
template <> struct GaugeOf<0> { using T = GaugeF64; };
template <> struct GaugeOf<1> { using T = GaugeF32; };
template <> struct GaugeOf<2> { using T = GaugeF16; };

// ------------------------------------------------------------------ clover
// 36 reals per chirality: d[0..5] real diagonal, then 15 complex lower-triangle entries (i > j) in
// the order (1,0) (2,0) (2,1) (3,0) (3,1) (3,2) (4,0) .. (5,4).
template <typename R> struct CloverBlock { R v[36]; };

__host__ __device__ __forceinline__ int tri_index(int i, int j) { return i * (i - 1) / 2 + j; }  // i > j

struct CloverF64 {
  double2* p; int V;
  __device__ __forceinline__ void load(int s, int chi, CloverBlock<double>& a) const {
#pragma unroll
    for (int k = 0; k < 18; k++) { double2 v = __ldg(p + (size_t)(chi * 18 + k) * V + s); a.v[2 * k] = v.x; a.v[2 * k + 1] = v.y; }
  }
};
struct CloverF32 {
  float4* p; int V;
  __device__ __forceinline__ void load(int s, int chi, CloverBlock<float>& a) const {
#pragma unroll
    for (int k = 0; k < 9; k++) {
      float4 v = __ldg(p + (size_t)(chi * 9 + k) * V + s);
      a.v[4 * k] = v.x; a.v[4 * k + 1] = v.y; a.v[4 * k + 2] = v.z; a.v[4 * k + 3] = v.w;
    }
  }
};
struct CloverF16 {
  short4* p; float* scale; int V;
  __device__ __forceinline__ void load(int s, int chi, CloverBlock<float>& a) const {
    const float sc = __ldg(scale + s) * (1.0f / 32767.0f);
#pragma unroll
    for (int k = 0; k < 9; k++) {
      short4 v = __ldg(p + (size_t)(chi * 9 + k) * V + s);
      a.v[4 * k] = sc * v.x; a.v[4 * k + 1] = sc * v.y; a.v[4 * k + 2] = sc * v.z; a.v[4 * k + 3] = sc * v.w;
    }
  }
};
template <int PREC> struct CloverOf;
template <> struct CloverOf<0> { using T = CloverF64; };
template <> struct CloverOf<1> { using T = CloverF32; };
template <> struct CloverOf<2> { using T = CloverF16; };

// Flavour mixing of the doublet for spinor component k (spin-major, so k < 6 has g5 = +1):
// (-epsbar + i delta g5) v, i.e. -epsbar tau1 of Eq. 2 plus the i delta G5 x tau1 of the shifted
// systems (Q_ND + i delta = (G5 x tau1)(D_ND + i delta G5 x tau1)).
template <typename R>
__device__ __forceinline__ cpx<R> nd_mix(R epsbar, R delta, int k, cpx<R> v) {
  const R d = k < 6 ? delta : -delta;
  return {-epsbar * v.re - d * v.im, -epsbar * v.im + d * v.re};
}

// y = (A_chi + i tw) x for one chirality block (x, y: 6 complex).  A is Hermitian.
template <typename R>
__device__ __forceinline__ void clover_mul(const CloverBlock<R>& a, R tw, const cpx<R>* x, cpx<R>* y) {
#pragma unroll
  for (int i = 0; i < 6; i++) y[i] = mk(a.v[i] * x[i].re - tw * x[i].im, a.v[i] * x[i].im + tw * x[i].re);
#pragma unroll
  for (int i = 1; i < 6; i++) {
#pragma unroll
    for (int j = 0; j < i; j++) {
      const int t = 6 + 2 * tri_index(i, j);
      const cpx<R> l = mk(a.v[t], a.v[t + 1]);   // A_ij (i > j);  A_ji = conj(A_ij)
      y[i] = y[i] + l * x[j];
      y[j] = y[j] + cmul_conj(l, x[i]);
    }
  }
}

// su(3) coefficients f_a = tr(lambda_a / 2 F) of a traceless Hermitian F (row-major 3x3; lambda_a
// the Gell-Mann matrices)
__device__ __forceinline__ void algebra_coeffs(const cpx<double> h[9], double f[8]) {
  f[0] = h[1].re;
  f[1] = -h[1].im;
  f[2] = 0.5 * (h[0].re - h[4].re);
  f[3] = h[2].re;
  f[4] = -h[2].im;
  f[5] = h[5].re;
  f[6] = -h[5].im;
  f[7] = (h[0].re + h[4].re - 2.0 * h[8].re) * 0.28867513459481288225;   // 1 / (2 sqrt 3)
}

// ------------------------------------------------------------------ gamma algebra (chiral basis)
// g_mu = [[0, B_mu], [B_mu^dag, 0]]: B_x = -i s1, B_y = -i s2, B_z = -i s3, B_t = 1.
// (1 - s g_mu) psi = [h ; -s B^dag h] with h = psi_up - s B psi_dn   (s = +1 forward, -1 backward)
// returns h (2 spins x 3 colours) for the projector (1 - sgn * g_mu)
template <typename R>
__device__ __forceinline__ void spin_project(int mu, int sgn, const Spinor<R>& p, cpx<R> h[6]) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const cpx<R> u0 = p.c[a], u1 = p.c[3 + a], d0 = p.c[6 + a], d1 = p.c[9 + a];
    cpx<R> b0, b1;  // B psi_dn
    switch (mu) {
      case 0: b0 = mul_mi(d1); b1 = mul_mi(d0); break;      // -i s1 d
      case 1: b0 = neg(d1); b1 = d0; break;                 // -i s2 d = [[0,-1],[1,0]] d
      case 2: b0 = mul_mi(d0); b1 = mul_i(d1); break;       // -i s3 d
      default: b0 = d0; b1 = d1; break;                     // 1 d
    }
    if (sgn > 0) { h[a] = u0 - b0; h[3 + a] = u1 - b1; }
    else         { h[a] = u0 + b0; h[3 + a] = u1 + b1; }
  }
}

// acc += coef * (1 - sgn g_mu) psi reconstructed from uh = U h (2 spins x 3 colours):
// upper = uh, lower = -sgn B^dag uh
template <typename R>
__device__ __forceinline__ void spin_reconstruct_add(int mu, int sgn, const cpx<R> uh[6], Spinor<R>& acc) {
#pragma unroll
  for (int a = 0; a < 3; a++) {
    const cpx<R> h0 = uh[a], h1 = uh[3 + a];
    cpx<R> c0, c1;  // B^dag h
    switch (mu) {
      case 0: c0 = mul_i(h1); c1 = mul_i(h0); break;        // (i s1) h
      case 1: c0 = h1; c1 = neg(h0); break;                 // (-i s2)^dag = i s2 = [[0,1],[-1,0]]
      case 2: c0 = mul_i(h0); c1 = mul_mi(h1); break;       // i s3
      default: c0 = h0; c1 = h1; break;
    }
    acc.c[a] = acc.c[a] + h0;
    acc.c[3 + a] = acc.c[3 + a] + h1;
    if (sgn > 0) { acc.c[6 + a] = acc.c[6 + a] - c0; acc.c[9 + a] = acc.c[9 + a] - c1; }
    else         { acc.c[6 + a] = acc.c[6 + a] + c0; acc.c[9 + a] = acc.c[9 + a] + c1; }
  }
}

// uh = U h (colour) for both spins;  dag: uh = U^dag h
template <typename R>
__device__ __forceinline__ void su3_mul_half(const Link<R>& u, bool dag, const cpx<R> h[6], cpx<R> uh[6]) {
#pragma unroll
  for (int s = 0; s < 2; s++) {
#pragma unroll
    for (int a = 0; a < 3; a++) {
      cpx<R> acc = mk<R>(0, 0);
#pragma unroll
      for (int b = 0; b < 3; b++) {
        if (!dag) acc = acc + u.m[a * 3 + b] * h[s * 3 + b];
        else acc = acc + cmul_conj(u.m[b * 3 + a], h[s * 3 + b]);
      }
      uh[s * 3 + a] = acc;
    }
  }
}

}  // namespace tmg
