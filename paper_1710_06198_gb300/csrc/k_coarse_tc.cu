// Multi-right-hand-side coarse operator Y = D_c(mu_n) X on the 5th-generation tensor cores
// (tcgen05, accumulators in tensor memory), the one dense block contraction of the DD-alpha-AMG
// hot path (Eq. 1: D_c = P^dag D P is a 9-point stencil of dense (2 N_v)^2 complex blocks).
//
// One CTA (4 warps) per coarse site.  For each of the 9 stencil blocks the CTA stages, in shared
// memory and in the canonical K-major no-swizzle core-matrix layout,
//   A = real embedding of the complex block, [[Re A, -Im A], [Im A, Re A]] (2 nd x 2 nd, rows
//       zero-padded to M = 128),
//   B = real embedding of the neighbour's column vectors [Re x; Im x] (N columns, padded to 16/32),
// and one elected thread issues tcgen05.mma kind::tf32.  FP32 accuracy comes from split TF32:
// v = hi + lo with hi = tf32(v), lo = tf32(v - hi), and A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi
// (the dropped A_lo B_lo term is below FP32 rounding).  Each group of R consecutive K = 8 steps
// (R = 1 by default, "tc_steps_per_range" of tmg_tune) accumulates its products in its own TMEM
// column range, and the partial results are summed in FP32 registers after tcgen05.ld: with R = 1
// the tensor core never adds more than 24 products into one accumulator, which keeps its
// accumulation rounding below the FP32 tolerance for any N_v.  The twist i mu_n G5_c is added in
// the epilogue.
//
// For 2 N_v <= 32 a pipelined form (k_coarse_apply_tc2) stacks the split parts instead: one M = 128
// operand [A_hi; A_lo], one N = 2 NPAD operand [B_hi | B_lo], one MMA per K step, and two operand and
// accumulator buffers so that staging, MMAs and read-back of consecutive tiles overlap.
//
// Every wait on the MMA-completion mbarrier is bounded; a wait that gives up sets *err and the
// CTA still frees its tensor memory before returning.
#include <algorithm>

#include "tmg_host.h"

namespace tmg {

namespace {

constexpr int TC_M = 128;
constexpr unsigned kSpinLimit = 1u << 26;
constexpr uint64_t kWaitNs = 1000000000ull;   // 1 s
constexpr uint32_t kSuspendHintNs = 1000;     // each poll suspends for at most ~1 us

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ float tf32_round(float v) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(v));
  return __uint_as_float(r);
}

// float offset of element (row r, k) in a K-major core-matrix tile with KP columns:
// core matrix = 8 rows x 4 floats (128 bytes, rows 16 bytes apart); core matrices adjacent in K
// are 128 bytes apart (leading byte offset), adjacent in rows KP/4 * 128 bytes apart (stride).
__device__ __forceinline__ int core_off(int r, int k, int KP) {
  return ((r >> 3) * (KP >> 2) + (k >> 2)) * 32 + (r & 7) * 4 + (k & 3);
}

// shared-memory matrix descriptor: start address, leading / stride byte offsets (>> 4), version 1,
// no swizzle
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((addr >> 4) & 0x3FFF);
  d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// instruction descriptor of kind::tf32: D F32, A and B TF32, both K-major, shape M x N
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
  return t;
}

// Wait for the mbarrier phase; gives up after kWaitNs of wall time (and after kSpinLimit polls),
// so a completion that never arrives costs at most about a second instead of hanging the kernel.
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity) {
  const uint64_t t0 = global_ns();
  for (unsigned it = 0; it < kSpinLimit; it++) {
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(mbar), "r"(parity), "r"(kSuspendHintNs)
        : "memory");
    if (done) return true;
    if (global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// 16 consecutive TMEM columns of the warp's 32 lanes into registers, without waiting (the caller
// issues tmem_wait_ld before reading them), so several loads can be in flight at once
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// Per-thread share of one raw tile: the stencil block (ND x ND complex) and the neighbour's column
// vectors (ncol <= NPAD columns of ND complex) with 128 threads.  ND (= 2 N_v) and the padded K are
// compile-time constants so that the per-element index arithmetic reduces to shifts and constant
// multiplies.
template <int ND, int NPAD>
struct RawTile {
  static constexpr int kA = (ND * ND + 127) / 128;
  static constexpr int kB = (NPAD * ND + 127) / 128;
  float2 a[kA];
  float2 b[kB];
};

// The backward-hop blocks are not read: by the Gamma5_c-hermiticity of D_c (twist excluded) the
// block of site x for the hop -mu is G5_c B^dag G5_c with B the +mu block of site x - mu (the
// stencil's slot 2 + 2 mu holds the -mu hop, slot 1 + 2 mu the +mu hop, for every coarse extent), so
// a backward tile is staged from that forward block: transposed addresses at load, and at store the
// conjugate with the sign s_k s_l of the chirality halves.  Only the self and forward blocks (5 of
// 9) are read from memory.
__device__ __forceinline__ bool tc_backward(int d) { return d >= 2 && (d & 1) == 0; }

// Element assignment shared by load_tile and store_tile: chunk q * 4 + warp of a tile is one 8 x 4
// patch (8 rows of the result, 4 consecutive K) and lane L takes element (L / 4, L % 4) of it, so
// each warp-wide shared-memory store fills one 128-byte core matrix (no bank conflicts).
template <int ND, int NPAD>
__device__ __forceinline__ void load_tile(RawTile<ND, NPAD>& t, const float2* __restrict__ blk, const float2* __restrict__ X,
                                          size_t n, int nbr_site, int ncol, int tid, bool tr) {
  const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
  for (int q = 0; q < RawTile<ND, NPAD>::kA; q++) {
    const int ch = q * 4 + warp;                   // patch of the block: rows kb*8.., columns lb*4..
    if (ch < ND * ND / 32) {
      const int k = (ch % (ND / 8)) * 8 + (lane >> 2), l = (ch / (ND / 8)) * 4 + (lane & 3);
      t.a[q] = blk[tr ? (size_t)k * ND + l : (size_t)l * ND + k];
    }
  }
#pragma unroll
  for (int q = 0; q < RawTile<ND, NPAD>::kB; q++) {
    const int ch = q * 4 + warp;                   // patch of the columns: col cb*8.., entries lb*4..
    if (ch < NPAD * ND / 32) {
      const int col = (ch % (NPAD / 8)) * 8 + (lane >> 2), l = (ch / (NPAD / 8)) * 4 + (lane & 3);
      if (col < ncol) t.b[q] = X[(size_t)col * n + (size_t)nbr_site * ND + l];
    }
  }
}

template <int ND, int NPAD>
__device__ __forceinline__ void store_tile(const RawTile<ND, NPAD>& t, float* Ahi, float* Alo, float* Bhi, float* Blo, int ncol,
                                           int tid, bool tr) {
  constexpr int KP = ((2 * ND + 7) / 8) * 8;
  const int warp = tid >> 5, lane = tid & 31;
  // A real embedding: row r < ND -> (Re, -Im); row ND + r -> (Im, Re)
#pragma unroll
  for (int q = 0; q < RawTile<ND, NPAD>::kA; q++) {
    const int ch = q * 4 + warp;
    if (ch < ND * ND / 32) {
      const int k = (ch % (ND / 8)) * 8 + (lane >> 2), l = (ch / (ND / 8)) * 4 + (lane & 3);
      float2 z = t.a[q];
      if (tr) {                                    // backward hop: s_k s_l conj(B_lk)
        const float sg = ((k < ND / 2) == (l < ND / 2)) ? 1.f : -1.f;
        z = make_float2(sg * z.x, -sg * z.y);
      }
      const float re_h = tf32_round(z.x), im_h = tf32_round(z.y);
      const float re_l = tf32_round(z.x - re_h), im_l = tf32_round(z.y - im_h);
      const int o00 = core_off(k, l, KP), o01 = core_off(k, ND + l, KP);
      const int o10 = core_off(ND + k, l, KP), o11 = core_off(ND + k, ND + l, KP);
      Ahi[o00] = re_h;
      Ahi[o01] = -im_h;
      Ahi[o10] = im_h;
      Ahi[o11] = re_h;
      Alo[o00] = re_l;
      Alo[o01] = -im_l;
      Alo[o10] = im_l;
      Alo[o11] = re_l;
    }
  }
  // B: column vectors of the neighbour (NPAD rows of K-major data)
#pragma unroll
  for (int q = 0; q < RawTile<ND, NPAD>::kB; q++) {
    const int ch = q * 4 + warp;
    if (ch < NPAD * ND / 32) {
      const int col = (ch % (NPAD / 8)) * 8 + (lane >> 2), l = (ch / (NPAD / 8)) * 4 + (lane & 3);
      if (col < ncol) {
        const float2 z = t.b[q];
        const float re_h = tf32_round(z.x), im_h = tf32_round(z.y);
        const int o0 = core_off(col, l, KP), o1 = core_off(col, ND + l, KP);
        Bhi[o0] = re_h;
        Bhi[o1] = im_h;
        Blo[o0] = tf32_round(z.x - re_h);
        Blo[o1] = tf32_round(z.y - im_h);
      }
    }
  }
}

// Persistent CTAs: CTA b handles coarse sites b, b + G, b + 2 G, ...; the 9 stencil tiles of its
// sites form one sequence, and the global loads of tile t + 1 are issued into registers while the
// MMAs of tile t run.  Tensor memory, the mbarrier and the zero padding of the operand tiles are set
// up once per CTA.
template <int ND, int NPAD, int R>
__global__ void __launch_bounds__(128) k_coarse_apply_tc(int nc, int nv, int ncol, const float2* __restrict__ Dc,
                                                         const int* __restrict__ nbr, const float2* __restrict__ X,
                                                         float2* __restrict__ Y, const float* __restrict__ mu,
                                                         int* __restrict__ err, const int* __restrict__ skip,
                                                         const int* __restrict__ skip2) {
  // the caller's "nothing left to do" flags, written by earlier launches: every thread reads the
  // same values and returns before any tensor memory is allocated
  if ((skip && *skip) || (skip2 && *skip2)) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  constexpr int KP = ((2 * ND + 7) / 8) * 8;             // K padded to the MMA step
  constexpr int nsteps = KP / 8;                          // K = 8 MMA steps per stencil block
  constexpr int nranges = (nsteps + R - 1) / R;           // R consecutive K steps share one TMEM range
  constexpr uint32_t kCols = nranges * NPAD <= 32 ? 32 : nranges * NPAD <= 64 ? 64 : nranges * NPAD <= 128 ? 128
                             : nranges * NPAD <= 256 ? 256 : 512;
  float* Ahi = reinterpret_cast<float*>(sm);
  float* Alo = Ahi + TC_M * KP;
  float* Bhi = Alo + TC_M * KP;
  float* Blo = Bhi + NPAD * KP;
  uint64_t* mbar = reinterpret_cast<uint64_t*>(Blo + NPAD * KP);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
  volatile int* s_ok = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t n = (size_t)nc * ND;
  const int my_sites = blockIdx.x < nc ? (nc - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int ntiles = 9 * my_sites;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(kCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // rows >= 2 ND of A, K columns >= 2 ND and B columns >= ncol stay zero for the whole kernel
  for (int i = tid; i < 2 * TC_M * KP; i += blockDim.x) Ahi[i] = 0.f;
  for (int i = tid; i < 2 * NPAD * KP; i += blockDim.x) Bhi[i] = 0.f;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = idesc_tf32(TC_M, NPAD);
  constexpr uint32_t lbo = 128, sbo = (uint32_t)(KP / 4) * 128;
  bool ok = true;
  float acc[NPAD];
#pragma unroll
  for (int i = 0; i < NPAD; i++) acc[i] = 0.f;

  // two raw tiles in registers (when they fit: up to 16 float2 per thread each): tile t + 2's global
  // loads are issued as soon as tile t has been stored to shared memory, so each load has two
  // tiles' worth of MMAs and TMEM reads to land; larger tiles keep one register tile, loaded one
  // tile ahead
  constexpr bool kTwoAhead = RawTile<ND, NPAD>::kA + RawTile<ND, NPAD>::kB <= 16;
  RawTile<ND, NPAD> rawA, rawB;
  auto tile_site = [&](int t) { return blockIdx.x + (t / 9) * gridDim.x; };
  auto load_t = [&](RawTile<ND, NPAD>& r, int t) {
    const int st = tile_site(t), dt = t % 9;
    const int nb = nbr[st * 9 + dt];
    const bool bw = tc_backward(dt);
    load_tile<ND, NPAD>(r, Dc + (size_t)(bw ? nb * 9 + dt - 1 : st * 9 + dt) * ND * ND, X, n, nb, ncol, tid, bw);
  };
  if (ntiles > 0) load_t(rawA, 0);
  if (kTwoAhead && ntiles > 1) load_t(rawB, 1);
  auto tile_step = [&](int t, RawTile<ND, NPAD>& raw, int tnext) {
    const int site = tile_site(t), d = t % 9;
    store_tile<ND, NPAD>(raw, Ahi, Alo, Bhi, Blo, ncol, tid, tc_backward(d));
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");   // generic-proxy writes -> MMA reads
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const uint32_t aH = smem_u32(Ahi), aL = smem_u32(Alo), bH = smem_u32(Bhi), bL = smem_u32(Blo);
#pragma unroll
      for (int s = 0; s < nsteps; s++) {
        const uint32_t koff = (uint32_t)s * 2 * 128;     // two core matrices per K = 8 step
        const uint32_t dcol = tmem + (uint32_t)((s / R) * NPAD);
        const uint64_t dAh = smem_desc(aH + koff, lbo, sbo), dAl = smem_desc(aL + koff, lbo, sbo);
        const uint64_t dBh = smem_desc(bH + koff, lbo, sbo), dBl = smem_desc(bL + koff, lbo, sbo);
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(dcol), "l"(dAh), "l"(dBh), "r"(idesc), "r"((s % R) ? 1u : 0u));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(dcol), "l"(dAh), "l"(dBl), "r"(idesc), "r"(1u));
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(dcol), "l"(dAl), "l"(dBh), "r"(idesc), "r"(1u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar))
                   : "memory");
    }
    // the loads of tile tnext go out into the registers this tile has just left
    if (tnext < ntiles) load_t(raw, tnext);
    // the MMAs read shared memory asynchronously: thread 0 waits (bounded) for their completion,
    // then the whole CTA learns the outcome at one barrier, so every thread leaves the loop together
    if (tid == 0) {
      const bool done = mbar_wait(smem_u32(mbar), (uint32_t)(t & 1));
      *s_ok = done ? 1 : 0;
      if (!done) atomicExch(err, 1);
    }
    __syncthreads();
    ok = *s_ok != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && warp * 32 < 2 * ND) {
      // warp w reads TMEM lanes 32 w .. 32 w + 31 (rows of the real-embedded result), one column
      // range per K step, and sums them in FP32 (warps above row 2 ND hold only padding); up to 64
      // columns are loaded before each wait
      constexpr int X16 = NPAD / 16, RB = 4 / X16;
#pragma unroll
      for (int s2 = 0; s2 < nranges; s2 += RB) {
        uint32_t r[RB * X16][16];
#pragma unroll
        for (int q = 0; q < RB; q++)
          if (s2 + q < nranges)
#pragma unroll
            for (int h = 0; h < X16; h++)
              tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)((s2 + q) * NPAD + h * 16), r[q * X16 + h]);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < RB; q++)
          if (s2 + q < nranges)
#pragma unroll
            for (int h = 0; h < X16; h++)
#pragma unroll
              for (int i = 0; i < 16; i++) acc[h * 16 + i] += __uint_as_float(r[q * X16 + h][i]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();   // TMEM reads and shared-memory tiles consumed before the next tile's MMAs
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && d == 8) {
      // epilogue of this site: twist and store, then a fresh accumulator
      const int r = warp * 32 + lane;
      if (r < 2 * ND) {
        const bool imag = r >= ND;
        const int k = imag ? r - ND : r;
        float xo[NPAD];
#pragma unroll
        for (int col = 0; col < NPAD; col++) {
          const float2* xp = X + (size_t)col * n + (size_t)site * ND + k;
          xo[col] = col < ncol ? (imag ? xp->x : xp->y) : 0.f;
        }
#pragma unroll
        for (int col = 0; col < NPAD; col++) {
          if (col < ncol) {
            const float tw = k < nv ? mu[col] : -mu[col];
            float* yp = reinterpret_cast<float*>(Y + (size_t)col * n + (size_t)site * ND + k);
            if (!imag) yp[0] = acc[col] - tw * xo[col];
            else yp[1] = acc[col] + tw * xo[col];
          }
        }
      }
#pragma unroll
      for (int i = 0; i < NPAD; i++) acc[i] = 0.f;
    }
  };
  if (kTwoAhead) {
    for (int t = 0; t < ntiles && ok; t += 2) {
      tile_step(t, rawA, t + 2);
      if (t + 1 < ntiles && ok) tile_step(t + 1, rawB, t + 3);
    }
  } else {
    for (int t = 0; t < ntiles && ok; t++) tile_step(t, rawA, t + 1);
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kCols));
  }
}

// ---- pipelined form for 4 ND <= 128 (N_v <= 16).  The hi and lo parts of the split stencil block
// are stacked in one M = 128 operand, A' = [A_hi; A_lo] (rows 0 .. 2 ND - 1 and 2 ND .. 4 ND - 1 of
// the real embedding), and the neighbour's columns side by side in one N = 2 NPAD operand,
// B' = [B_hi | B_lo].  One MMA per K = 8 step then yields all four products A_hi B_hi, A_hi B_lo,
// A_lo B_hi, A_lo B_lo (TMEM lanes: hi / lo rows; columns: hi / lo right-hand sides), whose sum is
// the product of the split values; no row of the MMA is padding when N_v = 16.
//
// Two operand buffers in shared memory and two accumulator buffers in tensor memory, each with its
// own completion mbarrier: while the MMAs of tile t run, the CTA reads tile t - 1's accumulators,
// issues the global loads of tile t + 2 and, in the next iteration, stages tile t + 1 into the
// other buffer.
// Per-thread element map of the stacked form, computed once per kernel (the same element assignment
// as load_tile / store_tile): for each register slot of a raw tile, its offset in the global block
// or column vector and its shared-memory offset in A' / B' (-1: nothing to load or store).  The other
// copies of an element (Im rows, lo rows, Im columns) sit at compile-time distances from it.
template <int ND, int NPAD>
struct StackedMap {
  static constexpr int kA = RawTile<ND, NPAD>::kA, kB = RawTile<ND, NPAD>::kB, KP = 2 * ND;
  static constexpr int CC = (ND / 4) * 32;               // + ND along K
  static constexpr int CR = (ND / 8) * (KP / 4) * 32;    // + ND rows
  static constexpr int CB = (NPAD / 8) * (KP / 4) * 32;  // + NPAD rows (columns of B')
  int sa[kA], ga[kA], gt[kA], sb[kB];
  float sg[kA];                                          // chirality sign s_k s_l of a backward tile
  size_t gb[kB];
  __device__ __forceinline__ StackedMap(int tid, int ncol, size_t n) {
    const int warp = tid >> 5, lane = tid & 31;
#pragma unroll
    for (int q = 0; q < kA; q++) {
      const int ch = q * 4 + warp;
      const int k = (ch % (ND / 8)) * 8 + (lane >> 2), l = (ch / (ND / 8)) * 4 + (lane & 3);
      const bool in = ch < ND * ND / 32;
      sa[q] = in ? core_off(k, l, KP) : -1;
      ga[q] = in ? l * ND + k : 0;
      gt[q] = in ? k * ND + l : 0;
      sg[q] = ((k < ND / 2) == (l < ND / 2)) ? 1.f : -1.f;
    }
#pragma unroll
    for (int q = 0; q < kB; q++) {
      const int ch = q * 4 + warp;
      const int col = (ch % (NPAD / 8)) * 8 + (lane >> 2), l = (ch / (NPAD / 8)) * 4 + (lane & 3);
      const bool in = ch < NPAD * ND / 32 && col < ncol;
      sb[q] = in ? core_off(col, l, KP) : -1;
      gb[q] = in ? (size_t)col * n + l : 0;
    }
  }
  __device__ __forceinline__ void load(RawTile<ND, NPAD>& t, const float2* __restrict__ blk, const float2* __restrict__ xv,
                                       bool tr) const {
#pragma unroll
    for (int q = 0; q < kA; q++)
      if (sa[q] >= 0) t.a[q] = blk[tr ? gt[q] : ga[q]];
#pragma unroll
    for (int q = 0; q < kB; q++)
      if (sb[q] >= 0) t.b[q] = xv[gb[q]];
  }
  // A' = [A_hi; A_lo] (real embedding rows (Re, -Im) / (Im, Re)), B' = [B_hi | B_lo]
  __device__ __forceinline__ void store(const RawTile<ND, NPAD>& t, float* A, float* B, bool tr) const {
#pragma unroll
    for (int q = 0; q < kA; q++) {
      if (sa[q] >= 0) {
        float2 z = t.a[q];
        if (tr) z = make_float2(sg[q] * z.x, -sg[q] * z.y);   // backward hop: s_k s_l conj(B_lk)
        const float re_h = tf32_round(z.x), im_h = tf32_round(z.y);
        const float re_l = tf32_round(z.x - re_h), im_l = tf32_round(z.y - im_h);
        float* a = A + sa[q];
        a[0] = re_h;
        a[CC] = -im_h;
        a[CR] = im_h;
        a[CR + CC] = re_h;
        a[2 * CR] = re_l;
        a[2 * CR + CC] = -im_l;
        a[3 * CR] = im_l;
        a[3 * CR + CC] = re_l;
      }
    }
#pragma unroll
    for (int q = 0; q < kB; q++) {
      if (sb[q] >= 0) {
        const float2 z = t.b[q];
        const float re_h = tf32_round(z.x), im_h = tf32_round(z.y);
        float* b = B + sb[q];
        b[0] = re_h;
        b[CC] = im_h;
        b[CB] = tf32_round(z.x - re_h);
        b[CB + CC] = tf32_round(z.y - im_h);
      }
    }
  }
};

__host__ __device__ constexpr uint32_t tmem_cols_pow2(int n) { return n <= 32 ? 32 : n <= 64 ? 64 : n <= 128 ? 128 : n <= 256 ? 256 : 512; }

// Shared-memory bytes and TMEM columns of the pipelined kernel.
template <int ND, int NPAD, int R>
struct Tc2Shape {
  static constexpr int KP = 2 * ND, NS = KP / 8, NR = (NS + R - 1) / R, NB = 2 * NPAD;
  static constexpr int TCOLS = NR * NB;                    // accumulator columns of one buffer
  static constexpr int ASZ = TC_M * KP, BSZ = NB * KP;     // floats of one operand buffer
  static constexpr int SCR = 2 * ND * (NPAD + 1);          // epilogue scratch (floats)
  static constexpr size_t smem = sizeof(float) * (size_t)(2 * (ASZ + BSZ) + SCR) + 64;
  static constexpr uint32_t cols = tmem_cols_pow2(2 * TCOLS);
};

template <int ND, int NPAD, int R>
__global__ void __launch_bounds__(128) k_coarse_apply_tc2(int nc, int nv, int ncol, const float2* __restrict__ Dc,
                                                          const int* __restrict__ nbr, const float2* __restrict__ X,
                                                          float2* __restrict__ Y, const float* __restrict__ mu,
                                                          int* __restrict__ err, const int* __restrict__ skip,
                                                          const int* __restrict__ skip2) {
  using Sh = Tc2Shape<ND, NPAD, R>;
  static_assert(4 * ND <= TC_M, "stacked hi / lo rows must fit one M = 128 tile");
  if ((skip && *skip) || (skip2 && *skip2)) return;
  extern __shared__ __align__(1024) unsigned char sm[];
  float* const opnd = reinterpret_cast<float*>(sm);        // [2][A' (ASZ) | B' (BSZ)]
  float* const scratch = opnd + 2 * (Sh::ASZ + Sh::BSZ);   // [2 ND][NPAD + 1]
  uint64_t* const mbar = reinterpret_cast<uint64_t*>(scratch + Sh::SCR);   // [2]
  uint32_t* const tslot = reinterpret_cast<uint32_t*>(mbar + 2);
  volatile int* const s_ok = reinterpret_cast<volatile int*>(tslot + 1);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const size_t n = (size_t)nc * ND;
  const int my_sites = blockIdx.x < nc ? (nc - 1 - blockIdx.x) / gridDim.x + 1 : 0;
  const int ntiles = 9 * my_sites;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tslot)), "r"(Sh::cols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar)), "r"(1));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mbar + 1)), "r"(1));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  // rows >= 4 ND of A' and columns >= ncol of either half of B' stay zero for the whole kernel
  for (int i = tid; i < 2 * (Sh::ASZ + Sh::BSZ); i += blockDim.x) opnd[i] = 0.f;
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  constexpr uint32_t idesc = idesc_tf32(TC_M, Sh::NB);
  constexpr uint32_t lbo = 128, sbo = (uint32_t)(Sh::KP / 4) * 128;
  bool ok = true;
  float acc[NPAD];
#pragma unroll
  for (int i = 0; i < NPAD; i++) acc[i] = 0.f;

  constexpr bool kTwoAhead = RawTile<ND, NPAD>::kA + RawTile<ND, NPAD>::kB <= 16;
  RawTile<ND, NPAD> rawA, rawB;
  auto tile_site = [&](int t) { return blockIdx.x + (t / 9) * gridDim.x; };
  const StackedMap<ND, NPAD> map(tid, ncol, n);
  auto load_t = [&](RawTile<ND, NPAD>& r, int t) {
    const int st = tile_site(t), dt = t % 9;
    const int nb = nbr[st * 9 + dt];
    const bool bw = tc_backward(dt);
    map.load(r, Dc + (size_t)(bw ? nb * 9 + dt - 1 : st * 9 + dt) * ND * ND, X + (size_t)nb * ND, bw);
  };
  // thread 0 issues the MMAs of tile t (operand and accumulator buffer t & 1) once every thread's
  // shared-memory stores are visible to the tensor core
  auto issue = [&](int t) {
    const int bb = t & 1;
    float* const A = opnd + bb * (Sh::ASZ + Sh::BSZ);
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (tid == 0) {
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      // the descriptor's address field counts 16-byte units: K step s adds 2 * 128 / 16
      const uint64_t dA0 = smem_desc(smem_u32(A), lbo, sbo), dB0 = smem_desc(smem_u32(A + Sh::ASZ), lbo, sbo);
#pragma unroll
      for (int s = 0; s < Sh::NS; s++) {
        const uint32_t dcol = tmem + (uint32_t)(bb * Sh::TCOLS + (s / R) * Sh::NB);
        const uint64_t dA = dA0 + (uint64_t)(s * 16), dB = dB0 + (uint64_t)(s * 16);
        asm volatile("{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n"
                     ::"r"(dcol), "l"(dA), "l"(dB), "r"(idesc), "r"((s % R) ? 1u : 0u));
      }
      asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(mbar + bb))
                   : "memory");
    }
  };
  // site epilogue: rows 2 ND .. 4 ND - 1 (the lo part of A') hand their sums to rows 0 .. 2 ND - 1
  // through shared memory; those add the twist and store
  auto epilogue = [&](int site) {
    const int L = warp * 32 + lane;
    if (L >= 2 * ND && L < 4 * ND) {
#pragma unroll
      for (int i = 0; i < NPAD; i++) scratch[(L - 2 * ND) * (NPAD + 1) + i] = acc[i];
    }
    __syncthreads();
    if (L < 2 * ND) {
      const bool imag = L >= ND;
      const int k = imag ? L - ND : L;
      // the site's own entries for the twist term: all loads in flight before the first use
      float xo[NPAD];
#pragma unroll
      for (int col = 0; col < NPAD; col++) {
        const float2* xp = X + (size_t)col * n + (size_t)site * ND + k;
        xo[col] = col < ncol ? (imag ? xp->x : xp->y) : 0.f;
      }
#pragma unroll
      for (int col = 0; col < NPAD; col++) {
        if (col < ncol) {
          const float tw = k < nv ? mu[col] : -mu[col];
          const float v = acc[col] + scratch[L * (NPAD + 1) + col];
          float* yp = reinterpret_cast<float*>(Y + (size_t)col * n + (size_t)site * ND + k);
          if (!imag) yp[0] = v - tw * xo[col];
          else yp[1] = v + tw * xo[col];
        }
      }
    }
#pragma unroll
    for (int i = 0; i < NPAD; i++) acc[i] = 0.f;
  };
  // wait (bounded) for tile u's MMAs, add its accumulators to acc, free its buffers
  auto drain = [&](int u) {
    const int bu = u & 1;
    if (tid == 0) {
      const bool done = mbar_wait(smem_u32(mbar + bu), (uint32_t)((u >> 1) & 1));
      *s_ok = done ? 1 : 0;
      if (!done) atomicExch(err, 1);
    }
    __syncthreads();
    ok = *s_ok != 0;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (ok && warp * 32 < 4 * ND) {
      constexpr int X16 = Sh::NB / 16, RB = X16 >= 4 ? 1 : 4 / X16;
#pragma unroll
      for (int s2 = 0; s2 < Sh::NR; s2 += RB) {
        uint32_t r[RB * X16][16];
#pragma unroll
        for (int q = 0; q < RB; q++)
          if (s2 + q < Sh::NR)
#pragma unroll
            for (int h = 0; h < X16; h++)
              tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)(bu * Sh::TCOLS + (s2 + q) * Sh::NB + h * 16),
                        r[q * X16 + h]);
        tmem_wait_ld();
#pragma unroll
        for (int q = 0; q < RB; q++)
          if (s2 + q < Sh::NR)
#pragma unroll
            for (int h = 0; h < X16 / 2; h++)
#pragma unroll
              for (int i = 0; i < 16; i++)
                acc[h * 16 + i] += __uint_as_float(r[q * X16 + h][i]) + __uint_as_float(r[q * X16 + X16 / 2 + h][i]);
      }
    }
    // no CTA barrier here: the next issue's barrier orders these TMEM reads before the MMAs that
    // reuse the buffer, and this tile's operand buffer is free since the wait above
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    if (ok && u % 9 == 8) epilogue(tile_site(u));
  };
  int issued = 0, drained = 0;   // tiles whose MMAs were issued / whose accumulators were read
  auto step = [&](int t, RawTile<ND, NPAD>& raw) {
    float* const A = opnd + (t & 1) * (Sh::ASZ + Sh::BSZ);
    map.store(raw, A, A + Sh::ASZ, tc_backward(t % 9));   // buffer t & 1: tile t - 2 drained
    issue(t);
    issued = t + 1;
    const int tn = kTwoAhead ? t + 2 : t + 1;        // the registers just stored take the next loads
    if (tn < ntiles) load_t(raw, tn);
    if (t >= 1) {
      drain(t - 1);
      if (ok) drained = t;
    }
  };
  if (ntiles > 0) load_t(rawA, 0);
  if (kTwoAhead && ntiles > 1) load_t(rawB, 1);
  if (kTwoAhead) {
    for (int t = 0; t < ntiles && ok; t += 2) {
      step(t, rawA);
      if (t + 1 < ntiles && ok) step(t + 1, rawB);
    }
  } else {
    for (int t = 0; t < ntiles && ok; t++) step(t, rawA);
  }
  if (ok && ntiles > 0) {
    drain(ntiles - 1);
    if (ok) drained = ntiles;
  }
  // after a wait that gave up, let every issued MMA finish (bounded) before the tensor memory goes
  if (tid == 0)
    for (int u = drained; u < issued; u++) mbar_wait(smem_u32(mbar + (u & 1)), (uint32_t)((u >> 1) & 1));
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(Sh::cols));
  }
}

template <int ND, int NPAD>
void launch_tc2(Ctx& c, const TcLevel& L, int ncol, const void* X, void* Y, const float* mu_dev, int* err_dev, const int* skip,
                const int* skip2) {
  constexpr int R = NPAD <= 16 ? 2 : 4;   // K steps per accumulator range: at most 32 products per TMEM sum
  using Sh = Tc2Shape<ND, NPAD, R>;
  // persistent CTAs: two per SM when both tensor memory (512 columns) and shared memory allow
  const int per_sm = (Sh::cols <= 256 && Sh::smem <= 113 * 1024) ? 2 : 1;
  const int grid = std::max(1, std::min(L.nc, per_sm * c.sms));
  TMG_CUDA(cudaFuncSetAttribute(k_coarse_apply_tc2<ND, NPAD, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)Sh::smem));
  ++c.launches, k_coarse_apply_tc2<ND, NPAD, R><<<grid, 128, Sh::smem, c.stream>>>(L.nc, L.nv, ncol, L.Dc, L.nbr, (const float2*)X,
                                                                                (float2*)Y, mu_dev, err_dev, skip, skip2);
}

template <int ND, int NPAD, int R>
void launch_tc(Ctx& c, const TcLevel& L, int ncol, const void* X, void* Y, const float* mu_dev, int* err_dev, const int* skip,
               const int* skip2) {
  constexpr int KP = ((2 * ND + 7) / 8) * 8;
  constexpr int cols = ((KP / 8 + R - 1) / R) * NPAD;
  const size_t smem = sizeof(float) * (size_t)(2 * TC_M * KP + 2 * NPAD * KP) + 32;
  // persistent CTAs, as many as can be resident: tensor memory (512 columns per SM) holds two CTAs
  // when one needs at most 256 columns, shared memory two when one needs at most 113 KB
  const int per_sm = (cols <= 256 && smem <= 113 * 1024) ? 2 : 1;
  const int grid = std::max(1, std::min(L.nc, per_sm * c.sms));
  TMG_CUDA(cudaFuncSetAttribute(k_coarse_apply_tc<ND, NPAD, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  ++c.launches, k_coarse_apply_tc<ND, NPAD, R><<<grid, 128, smem, c.stream>>>(L.nc, L.nv, ncol, L.Dc, L.nbr, (const float2*)X,
                                                                           (float2*)Y, mu_dev, err_dev, skip, skip2);
}

template <int ND, int NPAD>
void launch_tc_r(Ctx& c, const TcLevel& L, int ncol, const void* X, void* Y, const float* mu_dev, int* err_dev,
                 const int* skip, const int* skip2) {
  if (c.tc_steps_per_range >= 4) launch_tc<ND, NPAD, 4>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2);
  else if (c.tc_steps_per_range == 2) launch_tc<ND, NPAD, 2>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2);
  else launch_tc<ND, NPAD, 1>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2);
}

template <int ND>
void launch_tc_nd(Ctx& c, const TcLevel& L, int ncol, const void* X, void* Y, const float* mu_dev, int* err_dev,
                  const int* skip, const int* skip2) {
  if constexpr (4 * ND <= TC_M) {
    if (c.tc_pipeline) {
      if (ncol <= 16) launch_tc2<ND, 16>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2);
      else launch_tc2<ND, 32>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2);
      return;
    }
  }
  if (ncol <= 16) launch_tc_r<ND, 16>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2);
  else launch_tc_r<ND, 32>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2);
}

}  // namespace

bool tc_level_ok(int nd, int ncol) {
  return ncol >= 1 && ncol <= 32 && (nd == 8 || nd == 16 || nd == 24 || nd == 32 || nd == 48 || nd == 64);
}

TcLevel tc_level1(const Ctx& c) { return TcLevel{c.cl.nc, c.cl.nv, c.cl.nd, c.cl.Dc32.as<float2>(), c.cl.nbr.as<int>()}; }
TcLevel tc_level2(const Ctx& c) { return TcLevel{c.cl2.nc, c.cl2.nv, c.cl2.nd, c.cl2.Dc32.as<float2>(), c.cl2.nbr.as<int>()}; }

// Y = D(mu_col) X for ncol FP32 vectors ([col][nc * nd] complex) of level L on the tensor cores;
// the launch does nothing when a skip flag is given and nonzero on the device.
void coarse_apply_tc_level(Ctx& c, const TcLevel& L, int ncol, const void* X, void* Y, const float* mu_dev, int* err_dev,
                           const int* skip, const int* skip2) {
  ProfScope ps(c, PK_COARSE);
  if (!tc_level_ok(L.nd, ncol)) throw Error{TMG_ERR_ARG, "tensor-core coarse apply: 1..32 columns, N_v 4, 8, 12, 16, 24 or 32"};
  switch (L.nd) {
    case 8: launch_tc_nd<8>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2); break;
    case 16: launch_tc_nd<16>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2); break;
    case 24: launch_tc_nd<24>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2); break;
    case 32: launch_tc_nd<32>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2); break;
    case 48: launch_tc_nd<48>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2); break;
    default: launch_tc_nd<64>(c, L, ncol, X, Y, mu_dev, err_dev, skip, skip2); break;
  }
  TMG_CHECK_LAUNCH();
}

// Y = D_c(mu_col) X on level 1
void coarse_apply_tc(Ctx& c, int ncol, const void* X, void* Y, const float* mu_dev, int* err_dev, const int* skip) {
  coarse_apply_tc_level(c, tc_level1(c), ncol, X, Y, mu_dev, err_dev, skip, nullptr);
}

}  // namespace tmg
