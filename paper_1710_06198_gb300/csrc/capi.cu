// C ABI of libtmg (declared in include/tmg.h).  Every entry point validates its arguments, runs
// the work on the context stream and converts exceptions from the launchers into status codes.
#include <chrono>
#include <string>
#include <cstring>
#include <new>

#include "tmg_host.h"
#include "solver.h"
#include <algorithm>
#include <vector>

using namespace tmg;

namespace {

int fail(tmg_ctx* ctx, int code, const std::string& msg) {
  if (ctx) ctx->c.err = msg;
  return code;
}

template <typename F>
int guarded(tmg_ctx* ctx, F&& f) {
  if (!ctx) return TMG_ERR_ARG;
  try {
    TMG_CUDA(cudaSetDevice(ctx->c.device));
    return f();
  } catch (const tmg::Error& e) {
    return fail(ctx, e.code, e.msg);
  } catch (const std::bad_alloc&) {
    return fail(ctx, TMG_ERR_OOM, "host allocation failed");
  } catch (const std::exception& e) {
    return fail(ctx, TMG_ERR_CUDA, e.what());
  }
}

bool valid_prec(int p) { return p == TMG_PREC_F64 || p == TMG_PREC_F32 || p == TMG_PREC_F16; }
bool valid_where(int w) { return w == TMG_HOST || w == TMG_DEVICE; }

// Bring an FP64 lexicographic array (host or device) onto the device; returns a device pointer.
const double* stage_in(Ctx& c, DBuf& stage, const double* p, size_t n_doubles, int where) {
  if (where == TMG_DEVICE) return p;
  stage.alloc(n_doubles * sizeof(double));
  TMG_CUDA(cudaMemcpyAsync(stage.p, p, n_doubles * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  return stage.as<double>();
}

double* stage_out_ptr(Ctx& c, DBuf& stage, double* p, size_t n_doubles, int where) {
  if (where == TMG_DEVICE) return p;
  stage.alloc(n_doubles * sizeof(double));
  return stage.as<double>();
}

void stage_out_finish(Ctx& c, DBuf& stage, double* p, size_t n_doubles, int where) {
  if (where == TMG_DEVICE) return;
  TMG_CUDA(cudaMemcpyAsync(p, stage.p, n_doubles * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  TMG_CUDA(cudaStreamSynchronize(c.stream));
}

int storage_of(int prec) { return prec == TMG_PREC_F64 ? TMG_PREC_F64 : TMG_PREC_F32; }

// in (n_in complex, FP64) -> op in precision prec -> out (n_out complex, FP64)
template <typename F>
int level2_op(tmg_ctx* ctx, const char* name, const double* in, double* out, size_t n_in, size_t n_out, int prec,
                     int where, F&& op) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!in || !out || (prec != TMG_PREC_F64 && prec != TMG_PREC_F32) || !valid_where(where))
      return fail(ctx, TMG_ERR_ARG, std::string(name) + ": bad argument");
    if (!c.l2_ready) return fail(ctx, TMG_ERR_STATE, std::string(name) + ": no level-2 setup");
    const double* d = stage_in(c, c.stage_a, in, 2 * n_in, where);
    tmg::CField xi, yo;
    xi.create(prec, n_in);
    yo.create(prec, n_out);
    convert_field(c, d, TMG_PREC_F64, xi.buf.p, prec, n_in);
    op(xi.buf.p, yo.buf.p);
    double* o = stage_out_ptr(c, c.stage_b, out, 2 * n_out, where);
    convert_field(c, yo.buf.p, prec, o, TMG_PREC_F64, n_out);
    stage_out_finish(c, c.stage_b, out, 2 * n_out, where);
    return TMG_OK;
  });
}

// coarse doublet vectors in (FP64) -> op in precision prec -> out
template <typename F>
int coarse_nd_op(tmg_ctx* ctx, const char* name, const double* in, double* out, int prec, int where, F&& op) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!in || !out || (prec != TMG_PREC_F64 && prec != TMG_PREC_F32) || !valid_where(where))
      return fail(ctx, TMG_ERR_ARG, std::string(name) + ": bad argument");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, std::string(name) + ": no setup");
    const size_t n = (size_t)2 * c.cl.nc * c.cl.nd;
    const double* d = stage_in(c, c.stage_a, in, 2 * n, where);
    tmg::CField xi, yo;
    xi.create(prec, n);
    yo.create(prec, n);
    convert_field(c, d, TMG_PREC_F64, xi.buf.p, prec, n);
    op(xi.buf.p, yo.buf.p);
    double* o = stage_out_ptr(c, c.stage_b, out, 2 * n, where);
    convert_field(c, yo.buf.p, prec, o, TMG_PREC_F64, n);
    stage_out_finish(c, c.stage_b, out, 2 * n, where);
    return TMG_OK;
  });
}

}  // namespace

extern "C" {

const char* tmg_version(void) { return "tmg 0.1 (sm_103a)"; }

const char* tmg_last_error(const tmg_ctx* ctx) { return ctx ? ctx->c.err.c_str() : "null context"; }

int tmg_create(tmg_ctx** out, const int dims[4], const int block[4], int device, void* stream) {
  if (!out || !dims || !block) return TMG_ERR_ARG;
  *out = nullptr;
  Geom g{};
  long long V = 1;
  int VB = 1, nblk = 1;
  for (int mu = 0; mu < 4; mu++) {
    if (dims[mu] <= 0 || block[mu] <= 0 || dims[mu] % block[mu]) return TMG_ERR_ARG;
    const int nb = dims[mu] / block[mu];
    if (nb < 2 || nb % 2) return TMG_ERR_ARG;
    g.L[mu] = dims[mu];
    g.B[mu] = block[mu];
    g.NB[mu] = nb;
    V *= dims[mu];
    VB *= block[mu];
    nblk *= nb;
  }
  if (V > (1LL << 30) / 12 || VB % 32 || VB > 256) return TMG_ERR_ARG;
  g.ls[0] = 1; g.bs[0] = 1;
  for (int mu = 1; mu < 4; mu++) {
    g.ls[mu] = g.ls[mu - 1] * g.B[mu - 1];
    g.bs[mu] = g.bs[mu - 1] * g.NB[mu - 1];
  }
  g.VB = VB;
  g.nblk = nblk;
  g.V = (int)V;
  g.tbc = -1;
  tmg_ctx* ctx = new (std::nothrow) tmg_ctx();
  if (!ctx) return TMG_ERR_OOM;
  ctx->c.device = device;
  ctx->c.stream = (cudaStream_t)stream;
  ctx->c.g = g;
  tmg_mg_defaults(&ctx->c.mg);
  const int rc = guarded(ctx, [&]() -> int {
    int sms = 0;
    TMG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    ctx->c.sms = sms > 0 ? sms : 152;
    return TMG_OK;
  });
  if (rc != TMG_OK) {
    delete ctx;
    return rc;
  }
  *out = ctx;
  return TMG_OK;
}

int tmg_destroy(tmg_ctx* ctx) {
  if (!ctx) return TMG_ERR_ARG;
  cudaSetDevice(ctx->c.device);
  cudaStreamSynchronize(ctx->c.stream);
  delete ctx;
  return TMG_OK;
}

int tmg_set_params(tmg_ctx* ctx, double kappa, double csw, double mu, double mubar, double epsbar) {
  return guarded(ctx, [&]() -> int {
    if (!(kappa > 0.0) || !std::isfinite(csw) || !std::isfinite(mu) || !std::isfinite(mubar) || !std::isfinite(epsbar))
      return fail(ctx, TMG_ERR_ARG, "invalid operator parameters");
    Ctx& c = ctx->c;
    const bool rebuild = c.gauge_loaded && (kappa != c.kappa || csw != c.csw);
    c.kappa = kappa;
    c.csw = csw;
    c.mu = mu;
    c.mubar = mubar;
    c.epsbar = epsbar;
    if (rebuild) {
      build_clover(c);
      convert_op_precisions(c);
      c.mg_ready = false;
      c.eo.ready = false;
    }
    return TMG_OK;
  });
}

int tmg_set_ndshift(tmg_ctx* ctx, double delta) {
  return guarded(ctx, [&]() -> int {
    if (!std::isfinite(delta)) return fail(ctx, TMG_ERR_ARG, "tmg_set_ndshift: delta not finite");
    ctx->c.ndshift = delta;
    return TMG_OK;
  });
}

int tmg_check_links(const double* U, long long n_links, double* worst, long long* worst_index) {
  if (!U || n_links < 0) return TMG_ERR_ARG;
  long long at = -1;
  const double w = tmg::su3_defect_host(U, (size_t)n_links, &at);
  if (worst) *worst = w;
  if (worst_index) *worst_index = at;
  return w <= TMG_SU3_TOL ? TMG_OK : TMG_ERR_ARG;
}

int tmg_load_gauge(tmg_ctx* ctx, const double* U, int where, int t_bc) {
  return guarded(ctx, [&]() -> int {
    if (!U || !valid_where(where) || (t_bc != 1 && t_bc != -1)) return fail(ctx, TMG_ERR_ARG, "tmg_load_gauge: bad argument");
    Ctx& c = ctx->c;
    const size_t n = (size_t)c.g.V * 72;
    // every link must be special unitary: the compressed link formats rebuild row 2 from rows 0
    // and 1, which is exact for SU(3) only
    long long at = -1;
    double defect = 0.0;
    if (where == TMG_HOST) defect = su3_defect_host(U, (size_t)c.g.V * 4, &at);
    else defect = su3_defect_device(c, U, (size_t)c.g.V * 4, &at);
    if (!(defect <= TMG_SU3_TOL))
      return fail(ctx, TMG_ERR_ARG, "tmg_load_gauge: link " + std::to_string(at) + " (site " + std::to_string(at / 4) +
                                        ", direction " + std::to_string(at % 4) + ") is not in SU(3): max(|U U^dag - 1|, |det U - 1|) = " +
                                        std::to_string(defect));
    c.g.tbc = t_bc;
    const double* d = stage_in(c, c.U_lex, U, n, where);
    gauge_lex_to_internal(c, d);
    build_clover(c);
    convert_op_precisions(c);
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    c.U_lex.release();
    c.gauge_loaded = true;
    c.eo.ready = false;
    c.mg_ready = false;
    return TMG_OK;
  });
}

int tmg_apply(tmg_ctx* ctx, int op, const double* x, double* y, int n_rhs, const double* mu_per_col, int prec,
              int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!x || !y || n_rhs <= 0 || !valid_prec(prec) || !valid_where(where) || op < 0 || op > 5)
      return fail(ctx, TMG_ERR_ARG, "tmg_apply: bad argument");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_apply: no gauge field loaded");
    if (op == TMG_OP_DHAT || op == TMG_OP_DHAT_DAG) {
      if (prec == TMG_PREC_F16) return fail(ctx, TMG_ERR_ARG, "tmg_apply: the even-odd operator has F64 and F32 forms");
      const size_t col = (size_t)24 * c.g.V;
      const size_t hb = (size_t)12 * (c.g.V / 2) * (prec == TMG_PREC_F64 ? 16 : 8);
      const double mu0 = c.mu;
      DBuf w;
      w.alloc(3 * hb);
      for (int j = 0; j < n_rhs; j++) {
        c.mu = mu_per_col ? mu_per_col[j] : mu0;
        try {
          eo_prepare(c);
        } catch (...) {
          c.mu = mu0;
          throw;
        }
        const double* xd = stage_in(c, c.stage_a, x + j * col, col, where);
        eo_from_lex(c, xd, w.p, 1, prec);
        eo_apply(c, prec, w.as<char>() + hb, w.p, w.as<char>() + 2 * hb, op == TMG_OP_DHAT_DAG);
        double* yd = stage_out_ptr(c, c.stage_b, y + j * col, col, where);
        eo_to_lex(c, w.as<char>() + hb, yd, 1, prec, 1);
        stage_out_finish(c, c.stage_b, y + j * col, col, where);
      }
      c.mu = mu0;
      eo_check(c);
      return TMG_OK;
    }
    // FP16 storage of D, D^dag and the hopping term: spinors too are 16-bit fixed point
    const bool h16 = prec == TMG_PREC_F16 && op != TMG_OP_DND;
    const int sp = h16 ? PREC_H16 : storage_of(prec);
    const int kp = h16 ? PREC_H16 : prec;
    const int nfl = op == TMG_OP_DND ? 2 : 1;
    const size_t col = (size_t)24 * c.g.V;  // doubles per flavour column
    if (op == TMG_OP_D && prec == TMG_PREC_F32 && n_rhs > 1) {
      // all columns through the multi-column kernel (links and clover fetched once per site)
      ctx->fin.create(c.g, sp, n_rhs);
      ctx->fout.create(c.g, sp, n_rhs);
      const double* xd = stage_in(c, c.stage_a, x, col * n_rhs, where);
      for (int j = 0; j < n_rhs; j++) spinor_from_lex(c, xd + j * col, ctx->fin.col(c.g, j), sp);
      std::vector<float> mus(n_rhs, (float)c.mu);
      if (mu_per_col)
        for (int j = 0; j < n_rhs; j++) mus[j] = (float)mu_per_col[j];
      DBuf mu_dev;
      mu_dev.alloc(n_rhs * sizeof(float));
      TMG_CUDA(cudaMemcpyAsync(mu_dev.p, mus.data(), n_rhs * sizeof(float), cudaMemcpyHostToDevice, c.stream));
      dslash_mrhs(c, prec, n_rhs, ctx->fout.buf.p, ctx->fin.buf.p, nullptr, mu_dev.as<float>(), 0);
      double* yd = stage_out_ptr(c, c.stage_b, y, col * n_rhs, where);
      for (int j = 0; j < n_rhs; j++) spinor_to_lex(c, ctx->fout.col(c.g, j), sp, yd + j * col);
      stage_out_finish(c, c.stage_b, y, col * n_rhs, where);
      TMG_CUDA(cudaStreamSynchronize(c.stream));
      return TMG_OK;
    }
    ctx->fin.create(c.g, sp, nfl);
    ctx->fout.create(c.g, sp, nfl);
    for (int j = 0; j < n_rhs; j++) {
      const size_t off = (size_t)j * nfl * col;
      const double* xd = x + off;
      if (where == TMG_HOST) {
        c.stage_a.alloc(nfl * col * sizeof(double));
        TMG_CUDA(cudaMemcpyAsync(c.stage_a.p, x + off, nfl * col * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        xd = c.stage_a.as<double>();
      }
      for (int f = 0; f < nfl; f++) spinor_from_lex(c, xd + f * col, ctx->fin.col(c.g, f), sp);
      const double mu = mu_per_col ? mu_per_col[j] : c.mu;
      if (op == TMG_OP_D) dslash(c, kp, ctx->fout.col(c.g, 0), ctx->fin.col(c.g, 0), nullptr, mu, 0, 0);
      else if (op == TMG_OP_DDAG) dslash(c, kp, ctx->fout.col(c.g, 0), ctx->fin.col(c.g, 0), nullptr, mu, 0, 1);
      else if (op == TMG_OP_HOP) dslash(c, kp, ctx->fout.col(c.g, 0), ctx->fin.col(c.g, 0), nullptr, mu, 2, 0);
      else dslash_nd(c, prec, ctx->fout.buf.p, ctx->fin.buf.p);
      double* yd = where == TMG_DEVICE ? y + off : nullptr;
      if (where == TMG_HOST) {
        c.stage_b.alloc(nfl * col * sizeof(double));
        yd = c.stage_b.as<double>();
      }
      for (int f = 0; f < nfl; f++) spinor_to_lex(c, ctx->fout.col(c.g, f), sp, yd + f * col);
      if (where == TMG_HOST) {
        TMG_CUDA(cudaMemcpyAsync(y + off, yd, nfl * col * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
        TMG_CUDA(cudaStreamSynchronize(c.stream));
      }
    }
    return TMG_OK;
  });
}

int tmg_bench_dslash(tmg_ctx* ctx, int prec, int n_iter, double* ms) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!ms || n_iter <= 0 || !valid_prec(prec)) return fail(ctx, TMG_ERR_ARG, "tmg_bench_dslash: bad argument");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_bench_dslash: no gauge field loaded");
    const int sp = prec == TMG_PREC_F16 ? PREC_H16 : storage_of(prec);
    const int kp = prec == TMG_PREC_F16 ? PREC_H16 : prec;
    ctx->fin.create(c.g, sp, 1);
    ctx->fout.create(c.g, sp, 1);
    TMG_CUDA(cudaMemsetAsync(ctx->fin.buf.p, 0, spinor_col_bytes(c.g, sp), c.stream));
    for (int i = 0; i < 3; i++) dslash(c, kp, ctx->fout.buf.p, ctx->fin.buf.p, nullptr, c.mu, 0, 0);
    cudaEvent_t e0, e1;
    TMG_CUDA(cudaEventCreate(&e0));
    TMG_CUDA(cudaEventCreate(&e1));
    TMG_CUDA(cudaEventRecord(e0, c.stream));
    for (int i = 0; i < n_iter; i++) dslash(c, kp, ctx->fout.buf.p, ctx->fin.buf.p, nullptr, c.mu, 0, 0);
    TMG_CUDA(cudaEventRecord(e1, c.stream));
    TMG_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    TMG_CUDA(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    *ms = (double)t / n_iter;
    return TMG_OK;
  });
}

int tmg_bench_schur(tmg_ctx* ctx, int prec, int n_iter, double* ms) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!ms || n_iter <= 0 || (prec != TMG_PREC_F64 && prec != TMG_PREC_F32))
      return fail(ctx, TMG_ERR_ARG, "tmg_bench_schur: bad argument");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_bench_schur: no gauge field loaded");
    eo_prepare(c);
    const size_t hb = (size_t)12 * (c.g.V / 2) * (prec == TMG_PREC_F64 ? 16 : 8);
    DBuf w;
    w.alloc(3 * hb);
    TMG_CUDA(cudaMemsetAsync(w.p, 0, 3 * hb, c.stream));
    for (int i = 0; i < 3; i++) eo_apply(c, prec, w.as<char>() + hb, w.p, w.as<char>() + 2 * hb, 0);
    cudaEvent_t e0, e1;
    TMG_CUDA(cudaEventCreate(&e0));
    TMG_CUDA(cudaEventCreate(&e1));
    TMG_CUDA(cudaEventRecord(e0, c.stream));
    for (int i = 0; i < n_iter; i++) eo_apply(c, prec, w.as<char>() + hb, w.p, w.as<char>() + 2 * hb, 0);
    TMG_CUDA(cudaEventRecord(e1, c.stream));
    TMG_CUDA(cudaEventSynchronize(e1));
    float t = 0.f;
    TMG_CUDA(cudaEventElapsedTime(&t, e0, e1));
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    eo_check(c);
    *ms = (double)t / n_iter;
    return TMG_OK;
  });
}

int tmg_profile(tmg_ctx* ctx, int enable) {
  return guarded(ctx, [&]() -> int {
    TMG_CUDA(cudaStreamSynchronize(ctx->c.stream));
    ctx->c.prof.reset();
    ctx->c.prof.on = enable != 0;
    return TMG_OK;
  });
}

int tmg_profile_read(tmg_ctx* ctx, int kind, long long* count, double* ms_total) {
  return guarded(ctx, [&]() -> int {
    if (kind < 0 || kind >= PK_COUNT || !count || !ms_total) return fail(ctx, TMG_ERR_ARG, "tmg_profile_read: bad argument");
    TMG_CUDA(cudaStreamSynchronize(ctx->c.stream));
    double t = 0.0;
    for (auto& p : ctx->c.prof.recs[kind]) {
      float ms = 0.f;
      TMG_CUDA(cudaEventElapsedTime(&ms, p.first, p.second));
      t += ms;
    }
    *count = (long long)ctx->c.prof.recs[kind].size();
    *ms_total = t;
    return TMG_OK;
  });
}

int tmg_force_xy(tmg_ctx* ctx, const double* X, const double* Y, double* F, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!X || !Y || !F || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_force_xy: bad argument");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_force_xy: no gauge field loaded");
    const size_t col = (size_t)24 * c.g.V;
    tmg::Field xf, yf;
    xf.create(c.g, TMG_PREC_F64, 1);
    yf.create(c.g, TMG_PREC_F64, 1);
    spinor_from_lex(c, stage_in(c, c.stage_a, X, col, where), xf.buf.p, TMG_PREC_F64);
    spinor_from_lex(c, stage_in(c, c.stage_b, Y, col, where), yf.buf.p, TMG_PREC_F64);
    const size_t nf = (size_t)c.g.V * 4 * 9 * 2;
    DBuf fo;
    double* fd = where == TMG_DEVICE ? F : (fo.alloc(nf * sizeof(double)), fo.as<double>());
    force_from_xy(c, xf.buf.p, yf.buf.p, fd);
    if (where == TMG_HOST) {
      TMG_CUDA(cudaMemcpyAsync(F, fd, nf * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    }
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    return TMG_OK;
  });
}

int tmg_force(tmg_ctx* ctx, const double* phi, double* F, double tol, double* action, tmg_stats* stats, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!phi || !F || !(tol > 0.0) || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_force: bad argument");
    if (!c.gauge_loaded || !c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_force: needs a gauge field and a setup");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t col = (size_t)24 * c.g.V;
    const size_t n = (size_t)12 * c.g.V;
    tmg::Field pf, yf, xf, tf;
    pf.create(c.g, TMG_PREC_F64, 1);
    yf.create(c.g, TMG_PREC_F64, 1);
    xf.create(c.g, TMG_PREC_F64, 1);
    tf.create(c.g, TMG_PREC_F64, 1);
    spinor_from_lex(c, stage_in(c, c.stage_a, phi, col, where), pf.buf.p, TMG_PREC_F64);
    SolveStats s1{}, s2{};
    // Y = D(mu)^-1 phi ; X = D(mu)^-dag Y = g5 D(-mu)^-1 g5 Y (the same P serves both signs of mu)
    int rc = solve_one(c, TMG_SOLVE_MG_MIXED, pf.buf.p, yf.buf.p, c.mu, tol, 100000, s1);
    if (rc != TMG_OK) return fail(ctx, rc, "tmg_force: solve for Y failed");
    blas_copy(c, yf.buf.p, tf.buf.p, TMG_PREC_F64, n);
    gamma5_inplace(c, tf.buf.p, TMG_PREC_F64);
    rc = solve_one(c, TMG_SOLVE_MG_MIXED, tf.buf.p, xf.buf.p, -c.mu, tol, 100000, s2);
    if (rc != TMG_OK) return fail(ctx, rc, "tmg_force: solve for X failed");
    gamma5_inplace(c, xf.buf.p, TMG_PREC_F64);
    if (action) *action = blas_norm2(c, yf.buf.p, TMG_PREC_F64, n);
    const size_t nf = (size_t)c.g.V * 4 * 9 * 2;
    DBuf fo;
    double* fd = where == TMG_DEVICE ? F : (fo.alloc(nf * sizeof(double)), fo.as<double>());
    force_from_xy(c, xf.buf.p, yf.buf.p, fd);
    if (where == TMG_HOST) {
      TMG_CUDA(cudaMemcpyAsync(F, fd, nf * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    }
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    if (stats) {
      stats->iterations = s1.iterations + s2.iterations;
      stats->refinements = s1.refinements + s2.refinements;
      stats->coarse_iterations = s1.coarse_iterations + s2.coarse_iterations;
      stats->true_residual = std::max(s1.true_residual, s2.true_residual);
      stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    }
    return TMG_OK;
  });
}

static void fill_stats(tmg_stats* stats, const SolveStats& a, const SolveStats& b, std::chrono::steady_clock::time_point t0) {
  if (!stats) return;
  stats->iterations = a.iterations + b.iterations;
  stats->refinements = a.refinements + b.refinements;
  stats->coarse_iterations = a.coarse_iterations + b.coarse_iterations;
  stats->true_residual = std::max(a.true_residual, b.true_residual);
  stats->seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

int tmg_rotate_gauge(tmg_ctx* ctx, const double* omega, double step, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!omega || !valid_where(where) || !std::isfinite(step)) return fail(ctx, TMG_ERR_ARG, "tmg_rotate_gauge: bad argument");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_rotate_gauge: no gauge field loaded");
    const double* w = stage_in(c, c.stage_a, omega, (size_t)c.g.V * 32, where);
    rotate_gauge(c, w, step);
    build_clover(c);
    convert_op_precisions(c);
    c.eo.ready = false;
    if (c.mg_ready) {            // keep the hierarchy consistent with the new field: same P, new D_c
      build_coarse(c);
      if (c.l2_ready) build_coarse_c(c);
    }
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    if (where == TMG_HOST) c.stage_a.release();
    return TMG_OK;
  });
}

int tmg_setup_update(tmg_ctx* ctx, int n_iter) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (n_iter < 0 || n_iter > 100) return fail(ctx, TMG_ERR_ARG, "tmg_setup_update: n_iter out of range");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_setup_update: no earlier setup to update");
    mg_setup_update(c, n_iter);
    return TMG_OK;
  });
}

int tmg_pf_action(tmg_ctx* ctx, const double* phi, double* Y, double tol, double* S, tmg_stats* stats, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!phi || !Y || !(tol > 0.0) || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_pf_action: bad argument");
    if (!c.gauge_loaded || !c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_pf_action: needs a gauge field and a setup");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t col = (size_t)24 * c.g.V;
    const size_t n = (size_t)12 * c.g.V;
    tmg::Field pf, yf;
    pf.create(c.g, TMG_PREC_F64, 1);
    yf.create(c.g, TMG_PREC_F64, 1);
    spinor_from_lex(c, stage_in(c, c.stage_a, phi, col, where), pf.buf.p, TMG_PREC_F64);
    SolveStats s1{}, s0{};
    const int rc = solve_one(c, TMG_SOLVE_MG_MIXED, pf.buf.p, yf.buf.p, c.mu, tol, 100000, s1);
    if (rc != TMG_OK) return fail(ctx, rc, "tmg_pf_action: solve for Y failed");
    if (S) *S = blas_norm2(c, yf.buf.p, TMG_PREC_F64, n);
    double* yd = stage_out_ptr(c, c.stage_b, Y, col, where);
    spinor_to_lex(c, yf.buf.p, TMG_PREC_F64, yd);
    stage_out_finish(c, c.stage_b, Y, col, where);
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    fill_stats(stats, s1, s0, t0);
    return TMG_OK;
  });
}

int tmg_pf_force(tmg_ctx* ctx, const double* Y, double* f, double tol, tmg_stats* stats, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!Y || !f || !(tol > 0.0) || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_pf_force: bad argument");
    if (!c.gauge_loaded || !c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_pf_force: needs a gauge field and a setup");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t col = (size_t)24 * c.g.V;
    const size_t n = (size_t)12 * c.g.V;
    tmg::Field yf, xf, tf;
    yf.create(c.g, TMG_PREC_F64, 1);
    xf.create(c.g, TMG_PREC_F64, 1);
    tf.create(c.g, TMG_PREC_F64, 1);
    spinor_from_lex(c, stage_in(c, c.stage_a, Y, col, where), yf.buf.p, TMG_PREC_F64);
    // X = D(mu)^-dag Y = g5 D(-mu)^-1 g5 Y: the second solve of the two-step D^dag D scheme
    blas_copy(c, yf.buf.p, tf.buf.p, TMG_PREC_F64, n);
    gamma5_inplace(c, tf.buf.p, TMG_PREC_F64);
    SolveStats s2{}, s0{};
    const int rc = solve_one(c, TMG_SOLVE_MG_MIXED, tf.buf.p, xf.buf.p, -c.mu, tol, 100000, s2);
    if (rc != TMG_OK) return fail(ctx, rc, "tmg_pf_force: solve for X failed");
    gamma5_inplace(c, xf.buf.p, TMG_PREC_F64);
    const size_t nf = (size_t)c.g.V * 4 * 8;
    DBuf fo;
    double* fd = where == TMG_DEVICE ? f : (fo.alloc(nf * sizeof(double)), fo.as<double>());
    force_from_xy(c, xf.buf.p, yf.buf.p, fd, 1);
    if (where == TMG_HOST) TMG_CUDA(cudaMemcpyAsync(f, fd, nf * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    fill_stats(stats, s2, s0, t0);
    return TMG_OK;
  });
}

int tmg_sigma_min(tmg_ctx* ctx, const double* start, double mu_s, int max_steps, double rtol, double solve_tol,
                  int method, double* sigma, double* ritz_res, int* solves, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!start || !sigma || !(mu_s > 0.0) || max_steps < 2 || max_steps > 64 || !(rtol > 0.0) || !(solve_tol > 0.0) ||
        !valid_where(where) || (method != TMG_SOLVE_MG_F64 && method != TMG_SOLVE_MG_MIXED && method != TMG_SOLVE_CG_F64))
      return fail(ctx, TMG_ERR_ARG, "tmg_sigma_min: bad argument");
    if (!c.gauge_loaded || (method != TMG_SOLVE_CG_F64 && !c.mg_ready))
      return fail(ctx, TMG_ERR_STATE, "tmg_sigma_min: needs a gauge field (and a setup for multigrid solves)");
    const size_t col = (size_t)24 * c.g.V;
    tmg::Field sf;
    sf.create(c.g, TMG_PREC_F64, 1);
    spinor_from_lex(c, stage_in(c, c.stage_a, start, col, where), sf.buf.p, TMG_PREC_F64);
    int ns = 0, steps = 0;
    double rr = 0.0;
    *sigma = sigma_min_lanczos(c, sf.buf.p, mu_s, max_steps, rtol, solve_tol, method, &rr, &ns, &steps);
    if (ritz_res) *ritz_res = rr;
    if (solves) *solves = ns;
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    return rr <= rtol ? TMG_OK : TMG_ERR_NOCONV;
  });
}

int tmg_solve_shifts(tmg_ctx* ctx, const double* b, double* x, int n_shift, const double* mu, double tol, int guess,
                     double taylor_tol, int* iterations, tmg_stats* stats, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!b || !x || !mu || n_shift < 1 || n_shift > 64 || !(tol > 0.0) || guess < 0 || guess > 2 ||
        (guess == 2 && !(taylor_tol > 0.0)) || !valid_where(where))
      return fail(ctx, TMG_ERR_ARG, "tmg_solve_shifts: bad argument");
    for (int k = 0; k < n_shift; k++)
      if (!std::isfinite(mu[k])) return fail(ctx, TMG_ERR_ARG, "tmg_solve_shifts: twist not finite");
    if (!c.gauge_loaded || !c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_solve_shifts: needs a gauge field and a setup");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t col = (size_t)24 * c.g.V;
    tmg::Field bf, xf;
    bf.create(c.g, TMG_PREC_F64, 1);
    xf.create(c.g, TMG_PREC_F64, n_shift);
    spinor_from_lex(c, stage_in(c, c.stage_a, b, col, where), bf.buf.p, TMG_PREC_F64);
    SolveStats st{};
    const int rc = solve_shifts(c, bf.buf.p, xf.buf.p, n_shift, mu, tol, guess, taylor_tol, 100000, st, iterations);
    double* xd = stage_out_ptr(c, c.stage_b, x, col * n_shift, where);
    for (int k = 0; k < n_shift; k++) spinor_to_lex(c, xf.col(c.g, k), TMG_PREC_F64, xd + k * col);
    stage_out_finish(c, c.stage_b, x, col * n_shift, where);
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    SolveStats s0{};
    fill_stats(stats, st, s0, t0);
    if (stats) stats->true_residual = st.true_residual;
    return rc == TMG_OK ? TMG_OK : fail(ctx, rc, "tmg_solve_shifts: a shifted solve did not converge");
  });
}

int tmg_mms_cg(tmg_ctx* ctx, const double* b, double* x, int n_shift, const double* sigma, double tol, int flavours,
               tmg_stats* stats, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!b || !x || !sigma || n_shift < 1 || n_shift > 64 || !(tol > 0.0) || (flavours != 1 && flavours != 2) ||
        !valid_where(where))
      return fail(ctx, TMG_ERR_ARG, "tmg_mms_cg: bad argument");
    for (int s = 0; s < n_shift; s++)
      if (!(sigma[s] >= 0.0) || !std::isfinite(sigma[s])) return fail(ctx, TMG_ERR_ARG, "tmg_mms_cg: shifts must be >= 0");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_mms_cg: no gauge field loaded");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t col = (size_t)24 * c.g.V;
    const int nf = flavours;
    tmg::Field bf, xf;
    bf.create(c.g, TMG_PREC_F64, nf);
    xf.create(c.g, TMG_PREC_F64, nf * n_shift);
    const double* bd = stage_in(c, c.stage_a, b, col * nf, where);
    for (int f = 0; f < nf; f++) spinor_from_lex(c, bd + f * col, bf.col(c.g, f), TMG_PREC_F64);
    SolveStats st{}, s0{};
    const int rc = mms_cg_solve(c, bf.buf.p, xf.buf.p, n_shift, sigma, tol, 1000000, nf, st);
    double* xd = stage_out_ptr(c, c.stage_b, x, col * nf * n_shift, where);
    for (int k = 0; k < nf * n_shift; k++) spinor_to_lex(c, xf.col(c.g, k), TMG_PREC_F64, xd + k * col);
    stage_out_finish(c, c.stage_b, x, col * nf * n_shift, where);
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    fill_stats(stats, st, s0, t0);
    if (stats) stats->true_residual = st.true_residual;
    return rc == TMG_OK ? TMG_OK : fail(ctx, rc, "tmg_mms_cg: not converged");
  });
}

int tmg_rational_apply(tmg_ctx* ctx, const double* phi, double* out, int n, double a, const double* num,
                       const double* den, double tol, int flavours, double mg_below, tmg_stats* stats, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!phi || !out || !num || !den || n < 1 || n > 32 || !(tol > 0.0) || !std::isfinite(a) ||
        (flavours != 1 && flavours != 2) || !valid_where(where) || std::isnan(mg_below))
      return fail(ctx, TMG_ERR_ARG, "tmg_rational_apply: bad argument");
    bool any_mg = false;
    for (int l = 0; l < n; l++) any_mg = any_mg || den[l] < mg_below;
    if (any_mg && !c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_rational_apply: multigrid shifts need a setup");
    for (int l = 0; l < n; l++) {
      if (!(den[l] >= 0.0) || !std::isfinite(num[l])) return fail(ctx, TMG_ERR_ARG, "tmg_rational_apply: bad coefficients");
      for (int k = 0; k < l; k++)
        if (den[k] == den[l]) return fail(ctx, TMG_ERR_ARG, "tmg_rational_apply: repeated denominator shift");
    }
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_rational_apply: no gauge field loaded");
    const auto t0 = std::chrono::steady_clock::now();
    // partial fractions a prod (x + num_l)/(x + den_l) = a (1 + sum_l r_l / (x + den_l))
    std::vector<double> r(n);
    for (int l = 0; l < n; l++) {
      double pr = 1.0;
      for (int k = 0; k < n; k++) {
        pr *= num[k] - den[l];
        if (k != l) pr /= den[k] - den[l];
      }
      r[l] = pr;
    }
    const size_t col = (size_t)24 * c.g.V;
    const size_t nn = (size_t)flavours * 12 * c.g.V;
    const int nf = flavours;
    tmg::Field bf, xf;
    bf.create(c.g, TMG_PREC_F64, nf);
    xf.create(c.g, TMG_PREC_F64, nf * n);
    const double* bd = stage_in(c, c.stage_a, phi, col * nf, where);
    for (int f = 0; f < nf; f++) spinor_from_lex(c, bd + f * col, bf.col(c.g, f), TMG_PREC_F64);
    SolveStats st{}, s0{};
    // shifts at or above mg_below: one multi-shift CG; below it: the multigrid, two solves per shift
    std::vector<double> sh_cg;
    std::vector<int> at_cg, at_mg;
    for (int l = 0; l < n; l++) {
      if (den[l] < mg_below) at_mg.push_back(l);
      else { at_cg.push_back(l); sh_cg.push_back(den[l]); }
    }
    int rc = TMG_OK;
    tmg::Field cgf;
    if (!at_cg.empty()) {
      cgf.create(c.g, TMG_PREC_F64, nf * (int)at_cg.size());
      rc = mms_cg_solve(c, bf.buf.p, cgf.buf.p, (int)at_cg.size(), sh_cg.data(), tol, 1000000, nf, st);
      for (size_t i = 0; i < at_cg.size(); i++)
        blas_copy(c, cgf.col(c.g, (int)i * nf), xf.col(c.g, at_cg[i] * nf), TMG_PREC_F64, nn);
    }
    if (!at_mg.empty()) {
      tmg::Field tf, uf;
      tf.create(c.g, TMG_PREC_F64, nf);
      uf.create(c.g, TMG_PREC_F64, nf);
      const size_t n1 = (size_t)12 * c.g.V;
      // y = g5 x (one flavour) or (g5 x tau1) x (doublet)
      auto g5t = [&](const void* x, void* y) {
        if (nf == 1) {
          blas_copy(c, x, y, TMG_PREC_F64, n1);
        } else {
          blas_copy(c, x, (char*)y + n1 * 16, TMG_PREC_F64, n1);
          blas_copy(c, (const char*)x + n1 * 16, y, TMG_PREC_F64, n1);
        }
        for (int f = 0; f < nf; f++) gamma5_inplace(c, (char*)y + f * n1 * 16, TMG_PREC_F64);
      };
      const double shift0 = c.ndshift;
      try {
        for (int l : at_mg) {
          SolveStats s1{}, s2{};
          int r1, r2;
          g5t(bf.buf.p, tf.buf.p);
          if (nf == 1) {
            // D^dag D + q = D(mu_q)^dag D(mu_q), mu_q = sqrt(mu^2 + q): two-step solve of Sec. 1.1
            const double mq = std::sqrt(c.mu * c.mu + den[l]);
            r1 = solve_one(c, TMG_SOLVE_MG_MIXED, tf.buf.p, uf.buf.p, -mq, tol, 100000, s1);
            g5t(uf.buf.p, tf.buf.p);
            r2 = solve_one(c, TMG_SOLVE_MG_MIXED, tf.buf.p, xf.col(c.g, l), mq, tol, 100000, s2);
          } else {
            // Q_ND^2 + q = (Q_ND - i delta)(Q_ND + i delta), Q_ND +- i delta = (g5 x tau1)(D_ND +- i delta g5 x tau1)
            const double dl = std::sqrt(den[l]);
            c.ndshift = dl;
            r1 = solve_one(c, TMG_SOLVE_MG_MIXED, tf.buf.p, uf.buf.p, 0.0, tol, 100000, s1, 2);
            g5t(uf.buf.p, tf.buf.p);
            c.ndshift = -dl;
            r2 = solve_one(c, TMG_SOLVE_MG_MIXED, tf.buf.p, xf.col(c.g, l * nf), 0.0, tol, 100000, s2, 2);
            c.ndshift = shift0;
          }
          if (rc == TMG_OK && r1 != TMG_OK) rc = r1;
          if (rc == TMG_OK && r2 != TMG_OK) rc = r2;
          st.iterations += s1.iterations + s2.iterations;
          st.true_residual = std::max(st.true_residual, std::max(s1.true_residual, s2.true_residual));
        }
      } catch (...) {
        c.ndshift = shift0;
        throw;
      }
    }
    for (int l = 0; l < n; l++) blas_axpy(c, r[l], 0.0, xf.col(c.g, l * nf), bf.buf.p, TMG_PREC_F64, nn);
    blas_scale(c, a, 0.0, bf.buf.p, TMG_PREC_F64, nn);
    double* od = stage_out_ptr(c, c.stage_b, out, col * nf, where);
    for (int f = 0; f < nf; f++) spinor_to_lex(c, bf.col(c.g, f), TMG_PREC_F64, od + f * col);
    stage_out_finish(c, c.stage_b, out, col * nf, where);
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    fill_stats(stats, st, s0, t0);
    if (stats) stats->true_residual = st.true_residual;
    return rc == TMG_OK ? TMG_OK : fail(ctx, rc, "tmg_rational_apply: a shifted solve did not converge");
  });
}

int tmg_hmc_trajectory(tmg_ctx* ctx, const tmg_hmc_params* p, double* P, const double* eta, double* dH,
                       tmg_hmc_stats* stats, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!p || !P || !eta || !dH || !valid_where(where) || p->n_mono < 1 || p->n_mono > 8 || p->n_levels < 1 ||
        p->n_levels > 8 || !(p->tau > 0.0) || !std::isfinite(p->beta) || !(p->tol_action > 0.0) ||
        !(p->tol_force > 0.0) || p->setup_iters_start < 0 || p->setup_iters_force < 0)
      return fail(ctx, TMG_ERR_ARG, "tmg_hmc_trajectory: bad argument");
    for (int l = 0; l < p->n_levels; l++)
      if (p->steps[l] < 1 || p->steps[l] > 10000) return fail(ctx, TMG_ERR_ARG, "tmg_hmc_trajectory: steps out of range");
    for (int m = 0; m < p->n_mono; m++)
      if (!std::isfinite(p->mu[m]) || !(p->mu2[m] >= 0.0) || p->level[m] < 0 || p->level[m] >= p->n_levels)
        return fail(ctx, TMG_ERR_ARG, "tmg_hmc_trajectory: bad monomial");
    if (!c.gauge_loaded || !c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_hmc_trajectory: needs a gauge field and a setup");
    const size_t np = (size_t)32 * c.g.V, ne = (size_t)p->n_mono * 24 * c.g.V;
    DBuf Pd, Ed;
    double* Pp = P;
    const double* Ep = eta;
    if (where == TMG_HOST) {
      Pd.alloc(np * sizeof(double));
      Ed.alloc(ne * sizeof(double));
      TMG_CUDA(cudaMemcpyAsync(Pd.p, P, np * sizeof(double), cudaMemcpyHostToDevice, c.stream));
      TMG_CUDA(cudaMemcpyAsync(Ed.p, eta, ne * sizeof(double), cudaMemcpyHostToDevice, c.stream));
      Pp = Pd.as<double>();
      Ep = Ed.as<double>();
    }
    const int rc = hmc_trajectory(c, *p, Pp, Ep, dH, stats);
    if (where == TMG_HOST) {
      TMG_CUDA(cudaMemcpyAsync(P, Pp, np * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      TMG_CUDA(cudaStreamSynchronize(c.stream));
    }
    return rc;
  });
}

int tmg_get_gauge(tmg_ctx* ctx, double* U, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!U || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_get_gauge: bad argument");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_get_gauge: no gauge field loaded");
    const size_t n = (size_t)c.g.V * 72;
    double* d = stage_out_ptr(c, c.stage_b, U, n, where);
    gauge_internal_to_lex(c, d);
    stage_out_finish(c, c.stage_b, U, n, where);
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    return TMG_OK;
  });
}

int tmg_gauge_action(tmg_ctx* ctx, double beta, double* S) {
  return guarded(ctx, [&]() -> int {
    if (!S || !std::isfinite(beta)) return fail(ctx, TMG_ERR_ARG, "tmg_gauge_action: bad argument");
    if (!ctx->c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_gauge_action: no gauge field loaded");
    *S = gauge_action(ctx->c, beta);
    return TMG_OK;
  });
}

int tmg_gauge_force(tmg_ctx* ctx, double beta, double* f, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!f || !std::isfinite(beta) || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_gauge_force: bad argument");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_gauge_force: no gauge field loaded");
    const size_t n = (size_t)c.g.V * 32;
    double* d = stage_out_ptr(c, c.stage_b, f, n, where);
    gauge_force(c, beta, d);
    stage_out_finish(c, c.stage_b, f, n, where);
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    return TMG_OK;
  });
}

int tmg_tune(tmg_ctx* ctx, const char* key, double value) {
  return guarded(ctx, [&]() -> int {
    if (!key) return fail(ctx, TMG_ERR_ARG, "tmg_tune: null key");
    const std::string k(key);
    const int v = (int)value;
    if (k == "coarse_ctas_per_sm" && v >= 1 && v <= 8) ctx->c.coarse_ctas_per_sm = v;
    else if (k == "coarse_gs_passes" && (v >= 0 && v <= 2)) ctx->c.coarse_gs_passes = v;
    else if (k == "kcycle_ctas_per_sm" && v >= 1 && v <= 4) ctx->c.kcycle_ctas_per_sm = v;
    else if (k == "tc_steps_per_range" && (v == 1 || v == 2 || v == 4)) ctx->c.tc_steps_per_range = v;
    else if (k == "tc_pipeline" && (v == 0 || v == 1)) ctx->c.tc_pipeline = v;
    else if (k == "coarse_grid" && v >= 0 && v <= 4096) ctx->c.coarse_grid = v;
    else if (k == "eo_stage" && (v == 0 || v == 1)) ctx->c.eo_stage = v;
    else if (k == "coarse_overlap" && (v == 0 || v == 1)) ctx->c.coarse_overlap = v;
    else if (k == "batched_coarse_tc" && (v == 0 || v == 1)) ctx->c.batched_tc = v;
    else if (k == "coarse_block_cache" && (v == 0 || v == 1)) ctx->c.coarse_block_cache = v;
    else if (k == "coarse_eo" && (v == 0 || v == 1)) ctx->c.coarse_eo = v;
    else if (k == "batched_coarse_m" && v >= 0 && v <= 64) ctx->c.batched_coarse_m = v;
    else if (k == "outer_gs_fused" && (v == 0 || v == 1)) ctx->c.outer_gs_fused = v;
    else if (k == "outer_gs_passes" && (v == 1 || v == 2)) ctx->c.outer_gs_passes = v;
    else if (k == "force_prec" && (v == TMG_PREC_F64 || v == TMG_PREC_F32)) ctx->c.force_prec = v;
    else if (k == "kcycle_grid" && v >= 0 && v <= 4096) ctx->c.kcycle_grid = v;
    else if (k == "cycle_graph" && (v == 0 || v == 1)) {
      ctx->c.cycle_graphs = v;
      if (!v) ctx->c.graphs.clear();
    }
    else return fail(ctx, TMG_ERR_ARG, "tmg_tune: unknown key or value out of range: " + k);
    return TMG_OK;
  });
}

int tmg_autotune(tmg_ctx* ctx, double* best_ms) {
  return guarded(ctx, [&]() -> int {
    if (!ctx->c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_autotune: no setup");
    const double t = autotune(ctx->c);
    if (best_ms) *best_ms = t;
    return TMG_OK;
  });
}

int tmg_graph_count(const tmg_ctx* ctx, int* n) {
  if (!ctx || !n) return TMG_ERR_ARG;
  *n = (int)ctx->c.graphs.g.size();
  return TMG_OK;
}

int tmg_launch_count(const tmg_ctx* ctx, long long* n) {
  if (!ctx || !n) return TMG_ERR_ARG;
  *n = ctx->c.launches;
  return TMG_OK;
}

int tmg_mg_defaults(tmg_mg_params* p) {
  if (!p) return TMG_ERR_ARG;
  p->nv = 8;
  p->sap_sweeps = 3;
  p->sap_mr = 4;
  p->coarse_m = 30;
  p->coarse_rtol = 5e-2;
  p->n_init = 5;
  p->n_iter = 3;
  p->restart = 10;
  p->prec_fine = TMG_PREC_F32;
  p->prec_coarse = TMG_PREC_F32;
  return TMG_OK;
}

int tmg_setup(tmg_ctx* ctx, const tmg_mg_params* p, const double* v0, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!p || !v0 || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_setup: bad argument");
    if (p->nv < 2 || p->nv > 32 || p->sap_sweeps < 0 || p->sap_mr < 0 || p->coarse_m < 1 || p->coarse_m > 64 ||
        p->restart < 1 || p->restart > 64 || p->n_init < 0 || p->n_iter < 0 || !valid_prec(p->prec_fine) ||
        (p->prec_coarse != TMG_PREC_F64 && p->prec_coarse != TMG_PREC_F32) || !(p->coarse_rtol >= 0.0))
      return fail(ctx, TMG_ERR_ARG, "tmg_setup: invalid multigrid parameters");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_setup: no gauge field loaded");
    c.mg = *p;
    const size_t n = (size_t)p->nv * 24 * c.g.V;
    const double* d = stage_in(c, c.stage_a, v0, n, where);
    mg_setup(c, d);
    if (where == TMG_HOST) c.stage_a.release();
    return TMG_OK;
  });
}

int tmg_get_vectors(tmg_ctx* ctx, double* W, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!W || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_get_vectors: bad argument");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_get_vectors: no setup");
    const size_t col = (size_t)24 * c.g.V;
    const size_t n = col * c.cl.nv;
    double* d = stage_out_ptr(c, c.stage_b, W, n, where);
    for (int j = 0; j < c.cl.nv; j++)
      spinor_to_lex(c, c.cl.W64.as<double2>() + (size_t)j * 12 * c.g.V, TMG_PREC_F64, d + j * col);
    stage_out_finish(c, c.stage_b, W, n, where);
    return TMG_OK;
  });
}

// Fine vector in -> internal field (F64 or F32 storage)
static void fine_in(tmg_ctx* ctx, const double* x, int where, tmg::Field& f, int sp) {
  Ctx& c = ctx->c;
  const size_t col = (size_t)24 * c.g.V;
  const double* d = stage_in(c, c.stage_a, x, col, where);
  f.create(c.g, sp, 1);
  spinor_from_lex(c, d, f.buf.p, sp);
}

static void fine_out(tmg_ctx* ctx, const tmg::Field& f, int sp, double* y, int where) {
  Ctx& c = ctx->c;
  const size_t col = (size_t)24 * c.g.V;
  double* d = stage_out_ptr(c, c.stage_b, y, col, where);
  spinor_to_lex(c, f.buf.p, sp, d);
  stage_out_finish(c, c.stage_b, y, col, where);
}

int tmg_sap(tmg_ctx* ctx, const double* b, double* x, int prec, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!b || !x || !valid_prec(prec) || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_sap: bad argument");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_sap: no gauge field loaded");
    const int sp = storage_of(prec);
    fine_in(ctx, b, where, ctx->fin, sp);
    fine_in(ctx, x, where, ctx->fout, sp);
    tmg::Field r;
    r.create(c.g, sp, 1);
    sap_sweeps(c, prec, ctx->fout.buf.p, ctx->fin.buf.p, r.buf.p, c.mu, c.mg.sap_sweeps);
    fine_out(ctx, ctx->fout, sp, x, where);
    return TMG_OK;
  });
}

int tmg_restrict(tmg_ctx* ctx, const double* r, double* cv, int prec, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!r || !cv || !valid_prec(prec) || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_restrict: bad argument");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_restrict: no setup");
    const int sp = storage_of(prec);
    fine_in(ctx, r, where, ctx->fin, sp);
    const size_t n = (size_t)c.cl.nc * c.cl.nd;
    tmg::CField out;
    out.create(TMG_PREC_F64, n);
    restrict_(c, prec, ctx->fin.buf.p, out.buf.p, TMG_PREC_F64);
    double* d = stage_out_ptr(c, c.stage_b, cv, 2 * n, where);
    blas_copy(c, out.buf.p, d, TMG_PREC_F64, n);
    stage_out_finish(c, c.stage_b, cv, 2 * n, where);
    return TMG_OK;
  });
}

int tmg_prolong(tmg_ctx* ctx, const double* cv, double* e, int prec, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!cv || !e || !valid_prec(prec) || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_prolong: bad argument");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_prolong: no setup");
    const int sp = storage_of(prec);
    const size_t n = (size_t)c.cl.nc * c.cl.nd;
    const double* d = stage_in(c, c.stage_a, cv, 2 * n, where);
    ctx->fout.create(c.g, sp, 1);
    prolong(c, prec, d, TMG_PREC_F64, ctx->fout.buf.p, 0);
    fine_out(ctx, ctx->fout, sp, e, where);
    return TMG_OK;
  });
}

int tmg_coarse_apply(tmg_ctx* ctx, const double* x, double* y, double mu, int prec, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!x || !y || (prec != TMG_PREC_F64 && prec != TMG_PREC_F32) || !valid_where(where))
      return fail(ctx, TMG_ERR_ARG, "tmg_coarse_apply: bad argument");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_coarse_apply: no setup");
    const size_t n = (size_t)c.cl.nc * c.cl.nd;
    const double* d = stage_in(c, c.stage_a, x, 2 * n, where);
    tmg::CField xi, yo;
    xi.create(prec, n);
    yo.create(prec, n);
    convert_field(c, d, TMG_PREC_F64, xi.buf.p, prec, n);
    coarse_apply(c, prec, xi.buf.p, yo.buf.p, mu);
    double* o = stage_out_ptr(c, c.stage_b, y, 2 * n, where);
    convert_field(c, yo.buf.p, prec, o, TMG_PREC_F64, n);
    stage_out_finish(c, c.stage_b, y, 2 * n, where);
    return TMG_OK;
  });
}

int tmg_coarse_apply_multi(tmg_ctx* ctx, const double* x, double* y, int n_rhs, const double* mu_per_col, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!x || !y || n_rhs < 1 || n_rhs > 32 || !valid_where(where))
      return fail(ctx, TMG_ERR_ARG, "tmg_coarse_apply_multi: bad argument (1..32 columns)");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_coarse_apply_multi: no setup");
    if (2 * c.cl.nd > 128) return fail(ctx, TMG_ERR_ARG, "tmg_coarse_apply_multi: N_v > 32");
    const size_t n = (size_t)c.cl.nc * c.cl.nd;
    const double* d = stage_in(c, c.stage_a, x, 2 * n * n_rhs, where);
    tmg::CField xi, yo;
    xi.create(TMG_PREC_F32, n * n_rhs);
    yo.create(TMG_PREC_F32, n * n_rhs);
    convert_field(c, d, TMG_PREC_F64, xi.buf.p, TMG_PREC_F32, n * n_rhs);
    std::vector<float> mus(n_rhs, (float)c.mu);
    if (mu_per_col)
      for (int j = 0; j < n_rhs; j++) mus[j] = (float)mu_per_col[j];
    DBuf aux;
    aux.alloc(sizeof(float) * 32 + sizeof(int));
    TMG_CUDA(cudaMemcpyAsync(aux.p, mus.data(), n_rhs * sizeof(float), cudaMemcpyHostToDevice, c.stream));
    int* err = reinterpret_cast<int*>(aux.as<float>() + 32);
    TMG_CUDA(cudaMemsetAsync(err, 0, sizeof(int), c.stream));
    coarse_apply_tc(c, n_rhs, xi.buf.p, yo.buf.p, aux.as<float>(), err);
    int herr = 0;
    TMG_CUDA(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    double* o = stage_out_ptr(c, c.stage_b, y, 2 * n * n_rhs, where);
    convert_field(c, yo.buf.p, TMG_PREC_F32, o, TMG_PREC_F64, n * n_rhs);
    stage_out_finish(c, c.stage_b, y, 2 * n * n_rhs, where);
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    if (herr) return fail(ctx, TMG_ERR_TIMEOUT, "tmg_coarse_apply_multi: a tensor-core completion wait gave up");
    return TMG_OK;
  });
}

int tmg_coarse_solve_multi(tmg_ctx* ctx, const double* b, double* x, int n_rhs, const double* mu_per_col, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!b || !x || n_rhs < 1 || n_rhs > 32 || !valid_where(where))
      return fail(ctx, TMG_ERR_ARG, "tmg_coarse_solve_multi: bad argument (1..32 columns)");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_coarse_solve_multi: no setup");
    const size_t n = (size_t)c.cl.nc * c.cl.nd;
    const double* d = stage_in(c, c.stage_a, b, 2 * n * n_rhs, where);
    tmg::CField bi, xo;
    bi.create(TMG_PREC_F32, n * n_rhs);
    xo.create(TMG_PREC_F32, n * n_rhs);
    convert_field(c, d, TMG_PREC_F64, bi.buf.p, TMG_PREC_F32, n * n_rhs);
    std::vector<float> mus(n_rhs, (float)c.mu);
    if (mu_per_col)
      for (int j = 0; j < n_rhs; j++) mus[j] = (float)mu_per_col[j];
    DBuf mu_dev;
    mu_dev.alloc(sizeof(float) * 32);
    TMG_CUDA(cudaMemcpyAsync(mu_dev.p, mus.data(), n_rhs * sizeof(float), cudaMemcpyHostToDevice, c.stream));
    const bool tc = c.batched_tc && coarse_gmres_batched_tc_ok(c, n_rhs);
    if (tc) {
      if (!c.tc_err.p) c.tc_err.alloc(sizeof(int));
      TMG_CUDA(cudaMemsetAsync(c.tc_err.p, 0, sizeof(int), c.stream));
      coarse_gmres_batched_tc(c, n_rhs, bi.buf.p, xo.buf.p, mu_dev.as<float>());
    } else {
      coarse_gmres_batched(c, n_rhs, bi.buf.p, xo.buf.p, mu_dev.as<float>());
    }
    TMG_CHECK_LAUNCH();
    int herr = 0;
    if (tc) TMG_CUDA(cudaMemcpyAsync(&herr, c.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    double* o = stage_out_ptr(c, c.stage_b, x, 2 * n * n_rhs, where);
    convert_field(c, xo.buf.p, TMG_PREC_F32, o, TMG_PREC_F64, n * n_rhs);
    stage_out_finish(c, c.stage_b, x, 2 * n * n_rhs, where);
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    if (herr) return fail(ctx, TMG_ERR_TIMEOUT, "tmg_coarse_solve_multi: a tensor-core completion wait gave up");
    return TMG_OK;
  });
}

int tmg_kcycle_multi(tmg_ctx* ctx, const double* b, double* x, int n_rhs, const double* mu_per_col, int mode, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!b || !x || n_rhs < 1 || n_rhs > 32 || mode < 0 || mode > 2 || !valid_where(where))
      return fail(ctx, TMG_ERR_ARG, "tmg_kcycle_multi: bad argument (1..32 columns, mode 0..2)");
    if (!c.mg_ready || !c.l2_ready) return fail(ctx, TMG_ERR_STATE, "tmg_kcycle_multi: no level-2 setup");
    if (!kcycle_batched_ok(c, n_rhs)) return fail(ctx, TMG_ERR_ARG, "tmg_kcycle_multi: level shapes not covered by the tensor-core apply");
    const size_t n = (size_t)c.cl.nc * c.cl.nd;
    const double* d = stage_in(c, c.stage_a, b, 2 * n * n_rhs, where);
    tmg::CField bi, xo;
    bi.create(TMG_PREC_F32, n * n_rhs);
    xo.create(TMG_PREC_F32, n * n_rhs);
    convert_field(c, d, TMG_PREC_F64, bi.buf.p, TMG_PREC_F32, n * n_rhs);
    std::vector<float> mus(n_rhs, (float)c.mu);
    if (mu_per_col)
      for (int j = 0; j < n_rhs; j++) mus[j] = (float)mu_per_col[j];
    DBuf mu_dev;
    mu_dev.alloc(sizeof(float) * 32);
    TMG_CUDA(cudaMemcpyAsync(mu_dev.p, mus.data(), n_rhs * sizeof(float), cudaMemcpyHostToDevice, c.stream));
    if (!c.tc_err.p) c.tc_err.alloc(sizeof(int));
    TMG_CUDA(cudaMemsetAsync(c.tc_err.p, 0, sizeof(int), c.stream));
    kcycle_batched(c, n_rhs, bi.buf.p, xo.buf.p, mu_dev.as<float>(), mode);
    int herr = 0;
    TMG_CUDA(cudaMemcpyAsync(&herr, c.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    double* o = stage_out_ptr(c, c.stage_b, x, 2 * n * n_rhs, where);
    convert_field(c, xo.buf.p, TMG_PREC_F32, o, TMG_PREC_F64, n * n_rhs);
    stage_out_finish(c, c.stage_b, x, 2 * n * n_rhs, where);
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    if (herr) return fail(ctx, TMG_ERR_TIMEOUT, "tmg_kcycle_multi: a tensor-core completion wait gave up");
    return TMG_OK;
  });
}

int tmg_coarse_solve(tmg_ctx* ctx, const double* b, double* x, double mu, int prec, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!b || !x || (prec != TMG_PREC_F64 && prec != TMG_PREC_F32) || !valid_where(where))
      return fail(ctx, TMG_ERR_ARG, "tmg_coarse_solve: bad argument");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_coarse_solve: no setup");
    const size_t n = (size_t)c.cl.nc * c.cl.nd;
    const double* d = stage_in(c, c.stage_a, b, 2 * n, where);
    tmg::CField bi, xo;
    bi.create(prec, n);
    xo.create(prec, n);
    convert_field(c, d, TMG_PREC_F64, bi.buf.p, prec, n);
    coarse_gmres_persistent(c, prec, bi.buf.p, xo.buf.p, mu);
    double* o = stage_out_ptr(c, c.stage_b, x, 2 * n, where);
    convert_field(c, xo.buf.p, prec, o, TMG_PREC_F64, n);
    stage_out_finish(c, c.stage_b, x, 2 * n, where);
    return TMG_OK;
  });
}

// ---------------------------------------------------------------- third level
int tmg_level2_defaults(tmg_level2_params* p) {
  if (!p) return TMG_ERR_ARG;
  for (int mu = 0; mu < 4; mu++) p->agg[mu] = 2;
  p->nv = 8;
  p->smooth_m = 3;
  p->k_restart = 10;
  p->k_rtol = 1e-1;
  p->coarse_m = 30;
  p->coarse_rtol = 5e-2;
  p->n_init = 5;
  p->n_iter = 3;
  return TMG_OK;
}

int tmg_setup_level2(tmg_ctx* ctx, const tmg_level2_params* p, const double* v1, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!p || !v1 || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_setup_level2: bad argument");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_setup_level2: no fine setup");
    int avol = 1;
    for (int mu = 0; mu < 4; mu++) {
      if (p->agg[mu] < 1 || c.g.NB[mu] % p->agg[mu]) return fail(ctx, TMG_ERR_ARG, "tmg_setup_level2: aggregate does not tile the level-1 lattice");
      avol *= p->agg[mu];
    }
    if (p->nv < 1 || 2 * p->nv > 64 || p->nv > avol * c.cl.nv || p->smooth_m < 1 || p->smooth_m > 64 || p->k_restart < 1 ||
        p->k_restart > 16 || p->coarse_m < 1 || p->coarse_m > 64 || !(p->k_rtol >= 0.0) || !(p->coarse_rtol >= 0.0) ||
        p->n_init < 0 || p->n_iter < 0)
      return fail(ctx, TMG_ERR_ARG, "tmg_setup_level2: invalid level-2 parameters");
    c.l2p = *p;
    const size_t n = (size_t)p->nv * 2 * c.cl.nc * c.cl.nd;
    const double* d = stage_in(c, c.stage_a, v1, n, where);
    mg_setup2(c, d);
    if (where == TMG_HOST) c.stage_a.release();
    return TMG_OK;
  });
}

int tmg_get_vectors2(tmg_ctx* ctx, double* W2, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!W2 || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_get_vectors2: bad argument");
    if (!c.l2_ready) return fail(ctx, TMG_ERR_STATE, "tmg_get_vectors2: no level-2 setup");
    const size_t n = (size_t)c.cl2.nv * 2 * c.cl.nc * c.cl.nd;
    double* d = stage_out_ptr(c, c.stage_b, W2, n, where);
    TMG_CUDA(cudaMemcpyAsync(d, c.cl2.W64.p, n * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    stage_out_finish(c, c.stage_b, W2, n, where);
    if (where == TMG_DEVICE) TMG_CUDA(cudaStreamSynchronize(c.stream));
    return TMG_OK;
  });
}

int tmg_restrict2(tmg_ctx* ctx, const double* cv, double* c2, int prec, int where) {
  if (!ctx) return TMG_ERR_ARG;
  Ctx& c = ctx->c;
  return level2_op(ctx, "tmg_restrict2", cv, c2, (size_t)c.cl.nc * c.cl.nd, (size_t)c.cl2.nc * c.cl2.nd, prec, where,
                   [&](const void* x, void* y) { restrict_c(c, prec, x, y); });
}

int tmg_prolong2(tmg_ctx* ctx, const double* c2, double* e, int prec, int where) {
  if (!ctx) return TMG_ERR_ARG;
  Ctx& c = ctx->c;
  return level2_op(ctx, "tmg_prolong2", c2, e, (size_t)c.cl2.nc * c.cl2.nd, (size_t)c.cl.nc * c.cl.nd, prec, where,
                   [&](const void* x, void* y) { prolong_c(c, prec, x, y); });
}

int tmg_coarse_apply2(tmg_ctx* ctx, const double* x, double* y, double mu, int prec, int where) {
  if (!ctx) return TMG_ERR_ARG;
  Ctx& c = ctx->c;
  const size_t n2 = (size_t)c.cl2.nc * c.cl2.nd;
  return level2_op(ctx, "tmg_coarse_apply2", x, y, n2, n2, prec, where,
                   [&](const void* a, void* b) { coarse_apply_c(c, prec, a, b, mu); });
}

int tmg_kcycle(tmg_ctx* ctx, const double* b, double* x, double mu, int mode, int prec, int where) {
  if (!ctx) return TMG_ERR_ARG;
  Ctx& c = ctx->c;
  if (mode < 0 || mode > 2) return fail(ctx, TMG_ERR_ARG, "tmg_kcycle: mode must be 0, 1 or 2");
  const size_t n1 = (size_t)c.cl.nc * c.cl.nd;
  return level2_op(ctx, "tmg_kcycle", b, x, n1, n1, prec, where,
                   [&](const void* bb, void* xx) { kcycle(c, prec, bb, xx, mu, mode); });
}

// ---------------------------------------------------------------- doublet pieces
int tmg_sap_nd(tmg_ctx* ctx, const double* b, double* x, int prec, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!b || !x || !valid_prec(prec) || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_sap_nd: bad argument");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_sap_nd: no setup");
    const int sp = storage_of(prec);
    const size_t col = (size_t)24 * c.g.V;
    tmg::Field bf, xf;
    bf.create(c.g, sp, 2);
    xf.create(c.g, sp, 2);
    const double* bd = stage_in(c, c.stage_a, b, 2 * col, where);
    for (int f = 0; f < 2; f++) spinor_from_lex(c, bd + f * col, bf.col(c.g, f), sp);
    const double* xd = stage_in(c, c.stage_a, x, 2 * col, where);
    for (int f = 0; f < 2; f++) spinor_from_lex(c, xd + f * col, xf.col(c.g, f), sp);
    sap_sweeps_nd(c, prec, xf.buf.p, bf.buf.p, c.mg.sap_sweeps);
    double* o = stage_out_ptr(c, c.stage_b, x, 2 * col, where);
    for (int f = 0; f < 2; f++) spinor_to_lex(c, xf.col(c.g, f), sp, o + f * col);
    stage_out_finish(c, c.stage_b, x, 2 * col, where);
    return TMG_OK;
  });
}

int tmg_coarse_apply_nd(tmg_ctx* ctx, const double* x, double* y, int prec, int where) {
  if (!ctx) return TMG_ERR_ARG;
  Ctx& c = ctx->c;
  return coarse_nd_op(ctx, "tmg_coarse_apply_nd", x, y, prec, where, [&](const void* xi, void* yo) {
    const size_t n1 = (size_t)c.cl.nc * c.cl.nd, es = prec == TMG_PREC_F64 ? 16 : 8;
    const char* xu = (const char*)xi;
    char* yu = (char*)yo;
    coarse_apply(c, prec, xu, yu, c.mubar);
    coarse_apply(c, prec, xu + n1 * es, yu + n1 * es, -c.mubar);
    blas_axpy(c, -c.epsbar, 0.0, xu + n1 * es, yu, prec, n1);
    blas_axpy(c, -c.epsbar, 0.0, xu, yu + n1 * es, prec, n1);
    if (c.ndshift != 0.0) {   // i delta G5_c x tau1 of the shifted doublet
      coarse_g5_axpy(c, prec, 0.0, c.ndshift, xu + n1 * es, yu);
      coarse_g5_axpy(c, prec, 0.0, c.ndshift, xu, yu + n1 * es);
    }
  });
}

int tmg_coarse_solve_nd(tmg_ctx* ctx, const double* b, double* x, int prec, int where) {
  if (!ctx) return TMG_ERR_ARG;
  Ctx& c = ctx->c;
  return coarse_nd_op(ctx, "tmg_coarse_solve_nd", b, x, prec, where,
                      [&](const void* bi, void* xo) { coarse_gmres_persistent_nd(c, prec, bi, xo); });
}

int tmg_kcycle_nd(tmg_ctx* ctx, const double* b, double* x, int mode, int prec, int where) {
  if (!ctx) return TMG_ERR_ARG;
  Ctx& c = ctx->c;
  if (mode < 0 || mode > 2) return fail(ctx, TMG_ERR_ARG, "tmg_kcycle_nd: mode must be 0, 1 or 2");
  if (!c.l2_ready) return fail(ctx, TMG_ERR_STATE, "tmg_kcycle_nd: no level-2 setup");
  return coarse_nd_op(ctx, "tmg_kcycle_nd", b, x, prec, where,
                      [&](const void* bi, void* xo) { kcycle(c, prec, bi, xo, c.mubar, mode, 2); });
}

int tmg_cycle_nd(tmg_ctx* ctx, const double* r, double* z, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!r || !z || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_cycle_nd: bad argument");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_cycle_nd: no setup");
    const int sp = storage_of(c.mg.prec_fine);
    const size_t col = (size_t)24 * c.g.V;
    tmg::Field rf, zf;
    rf.create(c.g, sp, 2);
    zf.create(c.g, sp, 2);
    const double* rd = stage_in(c, c.stage_a, r, 2 * col, where);
    for (int f = 0; f < 2; f++) spinor_from_lex(c, rd + f * col, rf.col(c.g, f), sp);
    mg_cycle_nd(c, rf.buf.p, zf.buf.p);
    double* o = stage_out_ptr(c, c.stage_b, z, 2 * col, where);
    for (int f = 0; f < 2; f++) spinor_to_lex(c, zf.col(c.g, f), sp, o + f * col);
    stage_out_finish(c, c.stage_b, z, 2 * col, where);
    return TMG_OK;
  });
}

int tmg_cycle(tmg_ctx* ctx, const double* r, double* z, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!r || !z || !valid_where(where)) return fail(ctx, TMG_ERR_ARG, "tmg_cycle: bad argument");
    if (!c.mg_ready) return fail(ctx, TMG_ERR_STATE, "tmg_cycle: no setup");
    const int sp = storage_of(c.mg.prec_fine);
    fine_in(ctx, r, where, ctx->fin, sp);
    ctx->fout.create(c.g, sp, 1);
    mg_cycle(c, ctx->fin.buf.p, ctx->fout.buf.p, c.mu);
    fine_out(ctx, ctx->fout, sp, z, where);
    return TMG_OK;
  });
}

int tmg_solve(tmg_ctx* ctx, const double* b, double* x, int n_rhs, const double* mu_per_col, double tol, int method,
              int maxiter, tmg_stats* stats, int where) {
  return guarded(ctx, [&]() -> int {
    Ctx& c = ctx->c;
    if (!b || !x || n_rhs <= 0 || !(tol > 0.0) || maxiter <= 0 || !valid_where(where) || method < 0 || method > 6)
      return fail(ctx, TMG_ERR_ARG, "tmg_solve: bad argument");
    if (!c.gauge_loaded) return fail(ctx, TMG_ERR_STATE, "tmg_solve: no gauge field loaded");
    if (method != TMG_SOLVE_CG_F64 && method != TMG_SOLVE_CG_EO && !c.mg_ready)
      return fail(ctx, TMG_ERR_STATE, "tmg_solve: no multigrid setup");
    const auto t0 = std::chrono::steady_clock::now();
    const size_t col = (size_t)24 * c.g.V;
    tmg_stats acc{};
    int rc = TMG_OK;
    if (method == TMG_SOLVE_CG_EO) {
      const double mu0 = c.mu;
      for (int j = 0; j < n_rhs; j++) {
        c.mu = mu_per_col ? mu_per_col[j] : mu0;
        const double* bd = stage_in(c, c.stage_a, b + j * col, col, where);
        double* xd = stage_out_ptr(c, c.stage_b, x + j * col, col, where);
        SolveStats st{};
        int r;
        try {
          r = cg_eo_solve(c, bd, xd, tol, maxiter, st);
        } catch (...) {
          c.mu = mu0;
          throw;
        }
        stage_out_finish(c, c.stage_b, x + j * col, col, where);
        if (r != TMG_OK && rc == TMG_OK) rc = r;
        acc.iterations += st.iterations;
        acc.true_residual = std::max(acc.true_residual, st.true_residual);
      }
      c.mu = mu0;
      TMG_CUDA(cudaStreamSynchronize(c.stream));
      acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (stats) *stats = acc;
      if (rc != TMG_OK) c.err = "odd-even CG did not converge";
      return rc;
    }
    if (method == TMG_SOLVE_MG_BATCHED) {
      if (n_rhs > 32) return fail(ctx, TMG_ERR_ARG, "tmg_solve: at most 32 columns per batched solve");
      tmg::Field bf, xf;
      bf.create(c.g, TMG_PREC_F64, n_rhs);
      xf.create(c.g, TMG_PREC_F64, n_rhs);
      const double* bd = stage_in(c, c.stage_a, b, col * n_rhs, where);
      for (int j = 0; j < n_rhs; j++) spinor_from_lex(c, bd + j * col, bf.col(c.g, j), TMG_PREC_F64);
      std::vector<double> mus(n_rhs, c.mu);
      if (mu_per_col)
        for (int j = 0; j < n_rhs; j++) mus[j] = mu_per_col[j];
      SolveStats st{};
      rc = solve_batched(c, n_rhs, bf.buf.p, xf.buf.p, mus.data(), tol, maxiter, st);
      double* out = stage_out_ptr(c, c.stage_b, x, col * n_rhs, where);
      for (int j = 0; j < n_rhs; j++) spinor_to_lex(c, xf.col(c.g, j), TMG_PREC_F64, out + j * col);
      stage_out_finish(c, c.stage_b, x, col * n_rhs, where);
      TMG_CUDA(cudaStreamSynchronize(c.stream));
      acc.iterations = st.iterations;
      acc.refinements = st.refinements;
      acc.coarse_iterations = st.coarse_iterations;
      acc.true_residual = st.true_residual;
      acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
      if (stats) *stats = acc;
      if (rc != TMG_OK && c.err.empty()) c.err = "solver did not converge";
      return rc;
    }
    // doublet methods: every column is a flavour pair [2][V][4][3]
    const int nf = (method == TMG_SOLVE_ND_F64 || method == TMG_SOLVE_ND_MIXED) ? 2 : 1;
    const int m1 = nf == 2 ? (method == TMG_SOLVE_ND_F64 ? TMG_SOLVE_MG_F64 : TMG_SOLVE_MG_MIXED) : method;
    const size_t ccol = nf * col;
    for (int j = 0; j < n_rhs; j++) {
      const double mu = mu_per_col ? mu_per_col[j] : c.mu;
      tmg::Field bf, xf;
      bf.create(c.g, TMG_PREC_F64, nf);
      const double* bd = b + j * ccol;
      if (where == TMG_HOST) {
        c.stage_a.alloc(ccol * sizeof(double));
        TMG_CUDA(cudaMemcpyAsync(c.stage_a.p, b + j * ccol, ccol * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        bd = c.stage_a.as<double>();
      }
      for (int f = 0; f < nf; f++) spinor_from_lex(c, bd + f * col, bf.col(c.g, f), TMG_PREC_F64);
      xf.create(c.g, TMG_PREC_F64, nf);
      SolveStats st{};
      const int r = solve_one(c, m1, bf.buf.p, xf.buf.p, mu, tol, maxiter, st, nf);
      if (r != TMG_OK && rc == TMG_OK) rc = r;
      acc.iterations += st.iterations;
      acc.refinements += st.refinements;
      acc.coarse_iterations += st.coarse_iterations;
      acc.true_residual = std::max(acc.true_residual, st.true_residual);
      double* out = where == TMG_DEVICE ? x + j * ccol : nullptr;
      if (where == TMG_HOST) {
        c.stage_b.alloc(ccol * sizeof(double));
        out = c.stage_b.as<double>();
      }
      for (int f = 0; f < nf; f++) spinor_to_lex(c, xf.col(c.g, f), TMG_PREC_F64, out + f * col);
      if (where == TMG_HOST) {
        TMG_CUDA(cudaMemcpyAsync(x + j * ccol, out, ccol * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
      }
    }
    TMG_CUDA(cudaStreamSynchronize(c.stream));
    acc.seconds = std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (stats) *stats = acc;
    if (rc != TMG_OK && c.err.empty()) c.err = "solver did not converge";
    return rc;
  });
}

}  // extern "C"
