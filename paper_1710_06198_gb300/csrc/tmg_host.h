// Host-side context and kernel launchers of libtmg (internal).
#pragma once
#include <cuda_runtime.h>
#include <string>
#include <vector>

#include "tmg_internal.cuh"
#include "../../include/tmg.h"

namespace tmg {

// Error carried from a launcher up to the C ABI.
struct Error {
  int code;
  std::string msg;
};

#define TMG_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw ::tmg::Error{e_ == cudaErrorMemoryAllocation ? TMG_ERR_OOM : TMG_ERR_CUDA,       \
                         std::string(#call) + ": " + cudaGetErrorString(e_)};                \
  } while (0)

#define TMG_CHECK_LAUNCH() TMG_CUDA(cudaGetLastError())

// Owning device buffer.
struct DBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DBuf() = default;
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  ~DBuf() { release(); }
  void alloc(size_t n) {
    if (n <= bytes && p) return;
    release();
    if (n == 0) return;
    TMG_CUDA(cudaMalloc(&p, n));
    bytes = n;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T> T* as() const { return reinterpret_cast<T*>(p); }
};

// Internal storage code of an all-FP16 fine field: spinors as 16-bit fixed point with one FP32
// norm per site (SpinorF16), links and clover in their FP16 forms.  Not a public precision: the
// ABI's TMG_PREC_F16 selects it for operator applications.
constexpr int PREC_H16 = 3;

// Bytes of one fine spinor column in storage precision prec (H16: 3 int4 + 1 float per site).
inline size_t spinor_col_bytes(const Geom& g, int prec) {
  return prec == TMG_PREC_F64 ? (size_t)192 * g.V : prec == PREC_H16 ? (size_t)52 * g.V : (size_t)96 * g.V;
}

// Fine spinor field (one or more columns) in F64, F32 or H16 storage; complex count per column 12 V.
struct Field {
  int prec = 1;       // TMG_PREC_F64, TMG_PREC_F32 or PREC_H16
  int ncol = 1;
  DBuf buf;
  size_t col_elems(const Geom& g) const { return (size_t)12 * g.V; }
  size_t elem_bytes() const { return prec == TMG_PREC_F64 ? 16 : 8; }
  void create(const Geom& g, int prec_, int ncol_ = 1) {
    prec = prec_;
    ncol = ncol_;
    buf.alloc(spinor_col_bytes(g, prec) * ncol);
  }
  void* col(const Geom& g, int j) const { return (char*)buf.p + spinor_col_bytes(g, prec) * j; }
};

// Coarse vector: [ncoarse][nd] complex in F64 or F32.
struct CField {
  int prec = 1;
  size_t n = 0;       // complex entries per column
  DBuf buf;
  void create(int prec_, size_t n_) {
    prec = prec_;
    n = n_;
    buf.alloc(n * (prec == TMG_PREC_F64 ? 16 : 8));
  }
};

// Gauge-dependent operator data in one storage precision.
struct OpData {
  DBuf U;       // links
  DBuf A;       // clover (4 + m0 + C)
  DBuf Ascale;  // F16 clover scale per site
};

// Multigrid level data (fine level 0 -> coarse level 1).
struct Coarse {
  int nv = 0, nd = 0, nc = 0;  // test vectors, dofs per coarse site, coarse sites
  int cgeom[4];                // coarse lattice dims
  DBuf W64, W32;               // orthonormalised test vectors, F64 and F32 ([nv] spinor fields)
  DBuf Dc64, Dc32;             // coarse stencil [nc][9][nd(col l)][nd(row k)]
  DBuf nbr;                    // coarse neighbour table [nc][9] (slot 0 self, 1 + 2 mu: +mu, 2 + 2 mu: -mu)
  unsigned long long version = 0;   // bumped whenever the stencil is rebuilt
};

// Per-site inverses (A_self + i mu G5_c)^-1 of the coarse stencil for the odd-even coarse solve,
// kept for a few (mu, precision) pairs; a captured cycle refers to an entry by address.
struct SiteInverse {
  bool used = false;
  double mu = 0.0;
  int prec = 0;
  unsigned long long version = 0, stamp = 0;
  DBuf buf;
};
constexpr int kSiteInverseSlots = 16;

// Level 2 of the three-level hierarchy: aggregates of level-1 sites (Sec. 1.2 runs three levels).
struct Coarse2 {
  int agg[4] = {1, 1, 1, 1};   // level-2 aggregate in level-1 sites
  int nv = 0, nd = 0, nc = 0;  // level-2 test vectors, dofs per level-2 site, level-2 sites
  int cgeom[4];                // level-2 lattice dims
  DBuf W64, W32;               // orthonormalised level-2 basis, [nv][nc1 * nd1]
  DBuf Dc64, Dc32;             // level-2 stencil [nc][9][nd(col)][nd(row)]
  DBuf nbr;                    // level-2 neighbour table [nc][9]
};

// Optional per-kernel-class timing with CUDA events on the context stream (tmg_profile).
enum { PK_DSLASH_F64 = 0, PK_DSLASH_F32, PK_DSLASH_F16, PK_SAP_F64, PK_SAP_F32, PK_SAP_F16, PK_RESTRICT,
       PK_PROLONG, PK_COARSE, PK_COARSE_SOLVE, PK_EO_F64, PK_EO_F32, PK_COUNT };

struct Prof {
  bool on = false;
  std::vector<cudaEvent_t> pool;             // free events
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> recs[PK_COUNT];
  ~Prof() {
    for (auto& v : recs)
      for (auto& p : v) { cudaEventDestroy(p.first); cudaEventDestroy(p.second); }
    for (auto e : pool) cudaEventDestroy(e);
  }
  cudaEvent_t get() {
    if (!pool.empty()) { cudaEvent_t e = pool.back(); pool.pop_back(); return e; }
    cudaEvent_t e;
    TMG_CUDA(cudaEventCreate(&e));
    return e;
  }
  void reset() {
    for (auto& v : recs) {
      for (auto& p : v) { pool.push_back(p.first); pool.push_back(p.second); }
      v.clear();
    }
  }
};

// Workspaces of the lock-step batched solve (solver.cu), grown on demand and kept between calls.
struct BatchWork {
  DBuf r64, rin, e, V, Z, w, cr, ce, mu, part, h, npart, inv;
};

// Even-odd reduced operator data (k_eo.cu): half-lattice links (FP64 12-real, FP32 8-real) of both
// parities, the odd sites' clover field and the even sites' inverse (A + i mu g5)^-1, for the
// context's field and the twist mu they were built at.
struct EoData {
  bool ready = false;   // links and clover packed for the current gauge field, kappa and c_sw
  double mu = 0.0;      // twist of the stored inverse
  DBuf U64[2], U32[2];
  DBuf Ao64, Ao32, Mi64, Mi32;
  DBuf flag;            // [0] singular block found, [1] a staging wait gave up
  DBuf t, w;            // half-lattice work fields
};

// Captured CUDA graphs of the preconditioner cycle (solver.cu), keyed by everything the captured
// launches bake in: buffer addresses, twists, parameters and launch-shape knobs.
struct CycleGraph {
  std::vector<unsigned long long> key;
  cudaGraphExec_t exec = nullptr;
  long long kernels = 0;   // launches inside the graph (added to Ctx::launches per replay)
};

struct GraphCache {
  std::vector<CycleGraph> g;
  cudaStream_t cap = nullptr;   // private stream used only while capturing
  void clear() {
    for (auto& e : g)
      if (e.exec) cudaGraphExecDestroy(e.exec);
    g.clear();
  }
  ~GraphCache() {
    clear();
    if (cap) cudaStreamDestroy(cap);
  }
};

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Geom g{};
  double kappa = 0.125, csw = 0.0, mu = 0.0, mubar = 0.0, epsbar = 0.0;
  double ndshift = 0.0;   // delta of the shifted doublet D_ND + i delta G5 x tau1 (0: Eq. 2 itself)
  bool gauge_loaded = false;
  OpData op[3];          // F64, F32, F16
  DBuf U_lex;            // staging for a host gauge field
  tmg_mg_params mg{};
  bool mg_ready = false;
  Coarse cl;
  tmg_level2_params l2p{};
  bool l2_ready = false;   // level 2 built: the coarse solve of the cycle is the level-1 K-cycle
  Coarse2 cl2;
  DBuf kw;                 // K-cycle scratch (k_coarse_gmres.cu)
  DBuf kbw;                // batched K-cycle scratch (k_coarse_gmres.cu)
  DBuf sv2;                // raw level-1 test vectors of the level-2 setup
  DBuf l2_iter_dev;        // device counter of level-2 GMRES steps (K-cycle steps go to coarse_iter_dev)
  // solver workspaces (solver.cu)
  DBuf cw_V, cw_w, cw_state, cw_part, cw_cr, cw_ce;   // coarse GMRES
  DBuf fw_V, fw_Z, fw_w, fw_r64, fw_e, fw_x, fw_t, fw_part, fw_h;  // outer FGMRES / CG
  DBuf sv_raw;           // raw (un-orthonormalised) test vectors of the setup
  DBuf coarse_iter_dev;  // device counter of coarse GMRES steps
  // scratch
  DBuf red;              // reduction partials (doubles)
  DBuf red_out;          // reduction results (doubles)
  DBuf stage_a, stage_b; // FP64 lex staging for host vectors
  std::string err;
  int sms = 152;
  long long launches = 0;  // kernels launched by this context (all launchers count)
  // launch-shape tuning knobs (tmg_tune)
  int coarse_ctas_per_sm = 2;   // CTAs per SM of the persistent coarse GMRES (bounded by occupancy)
  int coarse_gs_passes = 0;     // classical Gram-Schmidt passes in the coarse GMRES (0: 1 for FP32, 2 for FP64)
  int kcycle_ctas_per_sm = 1;   // CTAs per SM of the persistent level-1 K-cycle
  int force_prec = TMG_PREC_F64;   // force kernels: all FP64 (TMG_PREC_F64) or FP32 inputs with FP64 sums
  int outer_gs_fused = 1;       // outer FGMRES: fuse pass 1's update with pass 2's dot products
  int outer_gs_passes = 1;      // outer FGMRES: classical Gram-Schmidt passes (1 or 2)
  int coarse_grid = 0;          // CTAs of the persistent coarse GMRES (0: coarse_ctas_per_sm x SMs)
  int kcycle_grid = 0;          // CTAs of the persistent K-cycle (0: kcycle_ctas_per_sm x SMs)
  int tc_steps_per_range = 1;   // K steps sharing one TMEM accumulator range in the tensor-core coarse apply
  int tc_pipeline = 1;          // tensor-core coarse apply for 2 N_v <= 32: stacked hi / lo operands, double-buffered
  int cycle_graphs = 1;         // replay the preconditioner cycle of the outer FGMRES as a CUDA graph
  GraphCache graphs;
  Prof prof;
  EoData eo;
  BatchWork bw;
  DBuf hmc_phi;                 // pseudofermions of the last HMC trajectory (hmc.cu)
  int hmc_nmono = 0;
  int eo_stage = 1;             // FP32 even-odd kernels stage the site-local clover stream by bulk copies
  int coarse_overlap = 1;       // coarse GMRES: overlap the Hessenberg update with the next stencil
  int batched_tc = 1;           // batched coarse solve: stencil on the tensor cores (k_coarse_tc.cu)
  int coarse_block_cache = 1;   // coarse GMRES: own stencil blocks copied once into shared memory
  int coarse_eo = 0;            // coarse GMRES on the odd-even reduced system (one flavour, even extents)
  int batched_coarse_m = 0;     // GMRES steps of the batched coarse solve (0: the multigrid's coarse_m)
  SiteInverse site_inv[kSiteInverseSlots];
  unsigned long long site_inv_clock = 0;
  DBuf tc_err;                  // set by a tensor-core completion wait that gave up (batched solve)
};

// Records a start event on construction and an end event on destruction when profiling is on.
struct ProfScope {
  Ctx& c;
  int kind;
  cudaEvent_t a = nullptr;
  ProfScope(Ctx& c_, int kind_) : c(c_), kind(kind_) {
    if (c.prof.on) {
      a = c.prof.get();
      TMG_CUDA(cudaEventRecord(a, c.stream));
    }
  }
  ~ProfScope() {
    if (a) {
      cudaEvent_t b = c.prof.get();
      cudaEventRecord(b, c.stream);
      c.prof.recs[kind].push_back({a, b});
    }
  }
};

// ---------------------------------------------------------------- launchers (k_fields.cu)
// Largest SU(3) defect max(|U U^dag - 1|_max, |det U - 1|) over n_links FP64 3x3 complex links
// ([n][3][3] interleaved), on the host (threads) or on the device (U a device pointer); *at gets
// the index of the worst link (the first NaN link if there is one; NaN makes the result NaN).
double su3_defect_host(const double* U, size_t n_links, long long* at);
double su3_defect_device(Ctx& c, const double* U_dev, size_t n_links, long long* at);
void gauge_lex_to_internal(Ctx& c, const double* lex_dev);
void gauge_internal_to_lex(Ctx& c, double* lex_dev);
// U_mu(x) <- exp(i step sum_a omega_a lambda_a / 2) U_mu(x) on the internal F64 links, omega
// lexicographic [V][4][8] on the device; the caller rebuilds clover and compressed copies
void rotate_gauge(Ctx& c, const double* omega_dev, double step);
void build_clover(Ctx& c);
void convert_op_precisions(Ctx& c);
// lex FP64 [V][12] complex -> internal field column (prec F64, F32 or PREC_H16)
void spinor_from_lex(Ctx& c, const double* lex_dev, void* dst, int prec);
void spinor_to_lex(Ctx& c, const void* src, int prec, double* lex_dev);
// view of an H16 spinor column: 3 int4 chunks per site, then the per-site norms
SpinorF16 spinor_h16(const Ctx& c, void* p);
void convert_field(Ctx& c, const void* src, int psrc, void* dst, int pdst, size_t n_complex);

// complex BLAS on flat arrays of n complex numbers (prec F64: double2, F32: float2)
void blas_zero(Ctx& c, void* x, int prec, size_t n);
void blas_copy(Ctx& c, const void* x, void* y, int prec, size_t n);
// y = a x + y
void blas_axpy(Ctx& c, double are, double aim, const void* x, void* y, int prec, size_t n);
// y = x + a y
void blas_xpay(Ctx& c, const void* x, double are, double aim, void* y, int prec, size_t n);
// x = a x
void blas_scale(Ctx& c, double are, double aim, void* x, int prec, size_t n);
// x = g5 x on a fine field
void gamma5_inplace(Ctx& c, void* x, int prec);
// y_prec_dst += a * x_prec_src (mixed precision accumulate, F32 -> F64 typical)
void blas_axpy_mixed(Ctx& c, double a, const void* x, int px, void* y, int py, size_t n);
// result[0] = re <x, y>, result[1] = im <x, y> into device doubles (FP64 accumulation)
void blas_dot_dev(Ctx& c, const void* x, const void* y, int prec, size_t n, double* out_dev);
double blas_norm2(Ctx& c, const void* x, int prec, size_t n);
void blas_dot(Ctx& c, const void* x, const void* y, int prec, size_t n, double* re, double* im);

// ---------------------------------------------------------------- dslash (k_dslash.cu)
// mode 0: y = op x ; mode 1: y = b - op x ; mode 2: y = hopping(x)
void dslash(Ctx& c, int prec, void* y, const void* x, const void* b, double mu, int mode, int dagger);
// non-degenerate doublet (Eq. 2) on F64 / F32 fields with 2 flavour columns
void dslash_nd(Ctx& c, int prec, void* y, const void* x);

// ---------------------------------------------------------------- even-odd operator (k_eo.cu)
// (re)build the even-odd data for the current field and c.mu
void eo_prepare(Ctx& c);
// y_o = Dhat(mu) x_o (dagger: Dhat^dag) on half-lattice fields of precision F64 / F32; t: scratch
void eo_apply(Ctx& c, int prec, void* y, const void* x, void* t, int dagger);
// which = 0: out = M_e^-1 (bt + hc H_eo x); which = 1: out = [M_o x | x] - H_oe bt (usem selects)
void eo_kernel(Ctx& c, int prec, int which, void* out, const void* x, const void* bt, double hc, int usem, int dagger);
// TMG_ERR_TIMEOUT if a staging wait of an even-odd kernel gave up (synchronises)
void eo_check(Ctx& c);
// full-lattice lexicographic FP64 <-> half-lattice field of one parity
void eo_from_lex(Ctx& c, const double* lex, void* out, int parity, int prec);
void eo_to_lex(Ctx& c, const void* in, double* lex, int parity, int prec, int zero_other);

// ---------------------------------------------------------------- force (k_force.cu)
// F (lexicographic [V][4][3][3] complex, device) of S = ||D^-1 phi||^2 from internal F64 fields
// X = D^-dag D^-1 phi and Y = D^-1 phi
// alg = 0: F as [V][4][3][3] complex; alg = 1: f[V][4][8] = tr(lambda_a / 2 F) (real), the
// su(3) coefficients of the force
void force_from_xy(Ctx& c, const void* X, const void* Y, double* F_lex, int alg = 0);

// ---------------------------------------------------------------- multigrid (k_mg.cu)
void sap_sweeps(Ctx& c, int prec, void* x, const void* b, void* r_scratch, double mu, int n_sweeps);
void restrict_(Ctx& c, int prec, const void* r, void* cvec, int cprec);
void prolong(Ctx& c, int prec, const void* cvec, int cprec, void* e, int accumulate);
// skip: optional device flag; when it is non-zero the launch does nothing
void coarse_apply(Ctx& c, int cprec, const void* x, void* y, double mu, const int* skip = nullptr);
void orthonormalise(Ctx& c, void* W64);
// y += (are + i aim) G5_c x on level-1 coarse vectors
void coarse_g5_axpy(Ctx& c, int prec, double are, double aim, const void* x, void* y);
// x ~= D_c(mu)^-1 b: one persistent cooperative GMRES kernel (k_coarse_gmres.cu)
void coarse_gmres_persistent(Ctx& c, int cprec, const void* b, void* x, double mu);
// the same on doublet coarse vectors [2][nc][nd] with D_ND,c = D_c x I2 + i mubar G5_c x tau3 - epsbar tau1
void coarse_gmres_persistent_nd(Ctx& c, int cprec, const void* b, void* x);
// SAP sweeps on the doublet (Eq. 2) for fields [2][12 V] in precision prec (mubar, epsbar of the context)
void sap_sweeps_nd(Ctx& c, int prec, void* x, const void* b, int n_sweeps);
// ncol columns in lock-step (FP32 coarse vectors [col][nc * nd], twists mu_dev[ncol] on the device)
void coarse_gmres_batched(Ctx& c, int ncol, const void* b, void* x, const float* mu_dev);
// multi-column fine-level kernels (k_batch.cu), FP32 spinors [col][12 V], twists per column
void dslash_mrhs(Ctx& c, int prec, int ncol, void* y, const void* x, const void* b, const float* mu_col_dev, int mode);
void sap_mrhs(Ctx& c, int prec, int ncol, void* x, const void* b, const float* mu_col_dev, int n_sweeps);
void restrict_mrhs(Ctx& c, int ncol, const void* r, void* cvec);
void prolong_mrhs(Ctx& c, int ncol, const void* cvec, void* e);
// Y = D_c(mu_col) X for ncol <= 32 FP32 coarse vectors on the tensor cores (k_coarse_tc.cu);
// err_dev (device int) is set to 1 if a bounded wait gave up
void coarse_apply_tc(Ctx& c, int ncol, const void* X, void* Y, const float* mu_dev, int* err_dev,
                     const int* skip = nullptr);
bool coarse_gmres_batched_tc_ok(const Ctx& c, int ncol);
void coarse_gmres_batched_tc(Ctx& c, int ncol, const void* b, void* x, const float* mu_dev);
// One coarse level as the tensor-core apply sees it: sites, test vectors, dofs per site, FP32
// stencil [nc][9][nd][nd] and neighbour table [nc][9].
struct TcLevel {
  int nc, nv, nd;
  const float2* Dc;
  const int* nbr;
};
bool tc_level_ok(int nd, int ncol);
TcLevel tc_level1(const Ctx& c);
TcLevel tc_level2(const Ctx& c);
void coarse_apply_tc_level(Ctx& c, const TcLevel& L, int ncol, const void* X, void* Y, const float* mu_dev, int* err_dev,
                           const int* skip, const int* skip2);
// The same solve on caller-provided device scratch (no allocation): bytes needed, and the launch.
size_t coarse_gmres_scratch_bytes(Ctx& c, int cprec);
void coarse_gmres_on_scratch(Ctx& c, int cprec, const void* b, void* x, double mu, void* scratch);
void build_coarse(Ctx& c);

// ---------------------------------------------------------------- level 2 (k_level2.cu)
// level-1 vectors [nc1][nd1] <-> level-2 vectors [nc2][nd2] in precision F64 / F32
void restrict_c(Ctx& c, int prec, const void* r, void* c2);
void prolong_c(Ctx& c, int prec, const void* c2, void* e);
// per (level-2 aggregate, level-1 chirality) modified Gram-Schmidt, twice, on cl2.W64
void orthonormalise_c(Ctx& c);
// cl2.Dc64 / Dc32 / nbr from cl.Dc64 and cl2.W64
void build_coarse_c(Ctx& c);
// y = D_cc(mu) x on level 2
void coarse_apply_c(Ctx& c, int prec, const void* x, void* y, double mu);
// Level-1 K-cycle as one persistent cooperative kernel (k_coarse_gmres.cu), precision F64 / F32:
// mode 0: x ~= D_c(mu)^-1 b by FGMRES preconditioned by the level-1 cycle (the coarse solve of the
//         three-level cycle); mode 1: x = level-1 cycle applied to b; mode 2: x = smoother applied
//         to b from zero (GMRES steps on D_c).
//         nf = 2: the same on doublet vectors [2][nc1][nd1] with D_ND,c and D_ND,cc (mu = mubar, the
//         context's epsbar).
void kcycle(Ctx& c, int prec, const void* b, void* x, double mu, int mode, int nf = 1);
// The same (one flavour, FP32, modes 0 / 1 / 2) for ncol columns [col][nc1 * nd1] in lock-step, each
// with its twist mu_dev[col] on the device: the operator applications on the tensor cores.
bool kcycle_batched_ok(const Ctx& c, int ncol);
void kcycle_batched(Ctx& c, int ncol, const void* b, void* x, const float* mu_dev, int mode);

}  // namespace tmg

// The opaque handle of the C ABI.
struct tmg_ctx {
  tmg::Ctx c;
  tmg::Field fin, fout;   // per-call conversion buffers
};
