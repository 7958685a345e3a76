// C ABI of libfmmpc (declared in include/fmmpc.h).  Every entry point validates its
// arguments, runs on the handle's stream and turns internal exceptions into FMMPC_ERR_*
// codes; nothing is thrown across the boundary.
#include <chrono>
#include <cmath>
#include <cstring>
#include <numeric>

#include "handle.cuh"

using namespace fmmpc;

namespace fmmpc {
int set_global_error(int code, const char *msg);
}

namespace {

thread_local char g_global_error[512];

int fail(fmmpc_handle *h, const Error &e) {
  if (h) h->err = e.msg;
  else set_global_error(e.code, e.msg.c_str());
  return e.code;
}

template <typename F>
int guarded(fmmpc_handle *h, F &&f) {
  try {
    return f();
  } catch (const Error &e) {
    return fail(h, e);
  } catch (const std::bad_alloc &) {
    return fail(h, Error(FMMPC_ERR_OOM, "host allocation failed"));
  } catch (const std::exception &e) {
    return fail(h, Error(FMMPC_ERR_CUDA, e.what()));
  }
}

void setup(fmmpc_handle &H, const fmmpc_grid &g, const fmmpc_params &p) {
  require(g.nx == g.ny, "grid: nx must equal ny");
  // the BEM inverse is a dense 4n x 4n FP64 matrix: n <= 4096 keeps it at 2.1 GB
  require(g.nx >= 4 && g.nx <= 4096, "grid: 4 <= nx <= 4096");
  const double wx = g.x1 - g.x0, wy = g.y1 - g.y0;
  require(wx > 0 && std::fabs(wx - wy) <= 1e-12 * wx, "grid: the domain must be a square");
  require(p.p == 4 || p.p == 6 || p.p == 8 || p.p == 10 || p.p == 12 || p.p == 16,
          "params: p must be one of 4, 6, 8, 10, 12, 16");
  require(p.leaf_max >= 16, "params: leaf_max >= 16");
  require(p.theta > 0.0 && p.theta < 1.0, "params: 0 < theta < 1");
  require(p.n_rhs >= 1 && p.n_rhs <= 64, "params: 1 <= n_rhs <= 64");
  require(p.precision >= FMMPC_PREC_FP64 && p.precision <= FMMPC_PREC_MIXED_TF32, "params: unknown precision");
  // leaf level: split at the centre lines while a cell holds more than leaf_max nodes
  const int n = g.nx;
  int L = 0, s = n;
  while ((int64_t)s * s > p.leaf_max) {
    require(s % 2 == 0, "grid: a centre-line split would cut a row of nodes (nx must be m 2^L)");
    s /= 2;
    ++L;
  }
  require(s == 4 || s == 8 || s == 16, "grid: leaf side must be 4, 8 or 16 nodes");
  Geo &G = H.g;
  G.n = n;
  G.m = s;
  G.L = L;
  G.lg = 0;
  while ((1 << G.lg) < n) ++G.lg;
  require((1 << G.lg) == n, "grid: nx must be a power of two");
  G.p = p.p;
  int tn = (int)std::lround(p.theta * 1000.0), td = 1000;
  int gc = std::gcd(tn, td);
  G.tnum = tn / gc;
  G.tden = td / gc;
  require(G.tnum > 0 && G.tnum < G.tden, "params: theta rounds outside (0, 1)");
  G.x0 = g.x0;
  G.y0 = g.y0;
  G.side = wx;
  G.h = wx / (n + 1);
  G.lnh = std::log(G.h);
  G.NG = 4 * n;
  G.ncell = level_offset(L + 1);
  G.nbcell = blevel_offset(L + 1);
  G.nleaf = int64_t(1) << (2 * L);
  G.nbleaf = 4 * (int64_t(1) << L);
  H.prec = p.precision;
  H.nrhs_max = p.n_rhs;

  auto t0 = std::chrono::steady_clock::now();
  DevPool tmp;
  try {
    build_tree(G, H.tree, H.stream, H.pool, tmp);
    build_lists(G, H.lists, H.st, H.stream, H.pool, tmp);
    G.R = H.st.R;
    G.pad = G.R * G.m;
    G.npad = n + 2 * G.pad;
    init_fmm(H);
    init_tc_p2p(H);
    init_tc_m2l(H, tmp);
    init_bem(H, tmp);
    FMMPC_CUDA(cudaStreamSynchronize(H.stream));
  } catch (...) {
    cudaStreamSynchronize(H.stream);
    tmp.release();
    throw;
  }
  tmp.release();
  H.t_setup_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

void check_rhs(const fmmpc_handle *h, int32_t n_rhs) {
  require(n_rhs >= 1 && n_rhs <= h->nrhs_max, "n_rhs must be in [1, params.n_rhs]");
}

void ensure_stage(fmmpc_handle &H) {
  if (H.stage_in) return;
  const size_t N = (size_t)H.g.n * H.g.n * H.nrhs_max;
  H.stage_in = H.pool.get<double>(N);
  H.stage_out = H.pool.get<double>(N);
  H.stage_g = H.pool.get<double>((size_t)4 * H.g.n * H.nrhs_max);
}

void release(fmmpc_handle *h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  for (auto &e : h->gcache) cudaGraphExecDestroy(e.exec);
  clear_solve_graphs(*h);
  if (h->cstream) cudaStreamDestroy(h->cstream);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  if (h->gev_in) cudaEventDestroy(h->gev_in);
  if (h->gev_out) cudaEventDestroy(h->gev_out);
  if (h->sstream) cudaStreamDestroy(h->sstream);
  if (h->sstream2) cudaStreamDestroy(h->sstream2);
  if (h->sstream3) cudaStreamDestroy(h->sstream3);
  for (auto e : h->sev)
    if (e) cudaEventDestroy(e);
  for (int k = 0; k <= fmmpc_handle::NSTAGE; ++k)
    if (h->ev[k]) cudaEventDestroy(h->ev[k]);
  if (h->kw.hbuf) cudaFreeHost(h->kw.hbuf);
  h->kpool.release();
  h->pool.release();
  delete h;
}

}  // namespace

namespace fmmpc {
int create_handle(fmmpc_handle **out, const fmmpc_grid &g, const fmmpc_params &prm, void *stream) {
  fmmpc_handle *h = nullptr;
  try {
    h = new fmmpc_handle();
  } catch (...) {
    return set_global_error(FMMPC_ERR_OOM, "host allocation failed");
  }
  h->stream = (cudaStream_t)stream;
  int rc = guarded(h, [&] {
    setup(*h, g, prm);
    return FMMPC_OK;
  });
  if (rc != FMMPC_OK) {
    set_global_error(rc, h->err.c_str());
    release(h);
    return rc;
  }
  *out = h;
  return FMMPC_OK;
}

int set_global_error(int code, const char *msg) {
  std::strncpy(g_global_error, msg ? msg : "", sizeof(g_global_error) - 1);
  g_global_error[sizeof(g_global_error) - 1] = 0;
  return code;
}
}  // namespace fmmpc

extern "C" {

int fmmpc_create(fmmpc_handle **out, const fmmpc_grid *g, const fmmpc_params *prm, void *stream) {
  if (!out || !g || !prm) return set_global_error(FMMPC_ERR_INVALID, "fmmpc_create: NULL argument");
  *out = nullptr;
  fmmpc_params p = *prm;
  if (p.autotune) {
    // tune on a smooth synthetic right-hand side (a few Gaussian bumps) of this grid
    int rc = FMMPC_OK;
    try {
      const int n = g->nx;
      require(n >= 4 && n <= 4096 && g->ny == n, "fmmpc_create: grid outside the supported range");
      std::vector<double> f((size_t)n * n);
      for (int j = 0; j < n; ++j)
        for (int i = 0; i < n; ++i) {
          const double x = (i + 1.0) / (n + 1), y = (j + 1.0) / (n + 1);
          f[(size_t)j * n + i] = std::exp(-((x - 0.3) * (x - 0.3) + (y - 0.6) * (y - 0.6)) / 0.005) -
                                 0.7 * std::exp(-((x - 0.7) * (x - 0.7) + (y - 0.35) * (y - 0.35)) / 0.002) +
                                 0.3 * std::sin(3.0 * x) * std::cos(2.0 * y);
        }
      DevPool tmp;
      double *fd = tmp.get<double>(f.size());
      cudaStream_t s = (cudaStream_t)stream;
      FMMPC_CUDA(cudaMemcpyAsync(fd, f.data(), sizeof(double) * f.size(), cudaMemcpyHostToDevice, s));
      fmmpc_solve_opts o{FMMPC_FGMRES, 30, 100, 1e-8, 1};
      std::vector<fmmpc_tune_entry> rep;
      fmmpc_params best = p;
      try {
        rc = autotune(*g, p, o, fd, 1e-5, stream, best, rep, false);
      } catch (...) {
        cudaStreamSynchronize(s);
        tmp.release();
        throw;
      }
      cudaStreamSynchronize(s);
      tmp.release();
      p = best;
      p.autotune = 0;
    } catch (const Error &e) {
      return set_global_error(e.code, e.msg.c_str());
    }
    if (rc != FMMPC_OK) return rc;
  }
  return create_handle(out, *g, p, stream);
}

int fmmpc_apply(fmmpc_handle *h, const double *r_dev, double *z_dev, int32_t n_rhs) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(r_dev && z_dev && r_dev != z_dev, "apply: r and z must be distinct device buffers");
    check_rhs(h, n_rhs);
    apply_fmm(*h, PART_FULL, r_dev, z_dev, n_rhs);
    return FMMPC_OK;
  });
}

int fmmpc_apply_host(fmmpc_handle *h, const double *r_host, double *z_host, int32_t n_rhs) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(r_host && z_host, "apply_host: NULL buffer");
    check_rhs(h, n_rhs);
    ensure_stage(*h);
    const size_t bytes = sizeof(double) * (size_t)h->g.n * h->g.n * n_rhs;
    FMMPC_CUDA(cudaMemcpyAsync(h->stage_in, r_host, bytes, cudaMemcpyHostToDevice, h->stream));
    apply_fmm(*h, PART_FULL, h->stage_in, h->stage_out, n_rhs);
    FMMPC_CUDA(cudaMemcpyAsync(z_host, h->stage_out, bytes, cudaMemcpyDeviceToHost, h->stream));
    FMMPC_CUDA(cudaStreamSynchronize(h->stream));
    return FMMPC_OK;
  });
}

int fmmpc_apply_part(fmmpc_handle *h, int32_t part, const double *r_dev, double *out_dev, int32_t n_rhs) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(r_dev && out_dev, "apply_part: NULL buffer");
    require(part >= PART_FULL && part <= PART_Q, "apply_part: unknown part");
    check_rhs(h, n_rhs);
    apply_fmm(*h, part, r_dev, out_dev, n_rhs);
    return FMMPC_OK;
  });
}

int fmmpc_apply_bc(fmmpc_handle *h, const double *f_dev, const double *g_dev, double *u_dev, int32_t n_rhs) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(f_dev && g_dev && u_dev && f_dev != u_dev, "apply_bc: f, g, u must be device buffers, u distinct from f");
    check_rhs(h, n_rhs);
    struct Restore {  // the single-layer equations of Sec. 4.1, whatever form the handle uses
      fmmpc_handle *h;
      int form;
      ~Restore() {
        h->bc_g = nullptr;
        h->bem_form = form;
      }
    } restore{h, h->bem_form};
    h->bem_form = 0;
    h->bc_g = g_dev;
    apply_fmm(*h, PART_BC, f_dev, u_dev, n_rhs);
    return FMMPC_OK;
  });
}

int fmmpc_apply_transpose(fmmpc_handle *h, const double *zb_dev, double *rb_dev, int32_t n_rhs) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(zb_dev && rb_dev && zb_dev != rb_dev, "apply_transpose: zb and rb must be distinct device buffers");
    check_rhs(h, n_rhs);
    if (h->bem_form != FMMPC_BEM_SINGLE_LAYER)
      throw Error(FMMPC_ERR_UNSUPPORTED, "apply_transpose: the single-layer correction only");
    init_bem_transpose(*h);
    struct Restore {
      fmmpc_handle *h;
      ~Restore() { h->trans_pass = false; }
    } restore{h};
    h->trans_pass = true;
    apply_fmm(*h, PART_TRANS, zb_dev, rb_dev, n_rhs);
    return FMMPC_OK;
  });
}

int fmmpc_set_bem_form(fmmpc_handle *h, int32_t form) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(form == FMMPC_BEM_SINGLE_LAYER || form == FMMPC_BEM_DOUBLE_LAYER, "set_bem_form: unknown form");
    if (form == FMMPC_BEM_DOUBLE_LAYER) init_bem_dl(*h);
    if (form != h->bem_form) {
      for (auto &e : h->gcache) cudaGraphExecDestroy(e.exec);  // captured with the other form
      h->gcache.clear();
      clear_solve_graphs(*h);
    }
    h->bem_form = form;
    return FMMPC_OK;
  });
}

int fmmpc_spmv(fmmpc_handle *h, const double *x_dev, double *y_dev, int32_t n_rhs) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(x_dev && y_dev && x_dev != y_dev, "spmv: x and y must be distinct device buffers");
    check_rhs(h, n_rhs);
    spmv5(*h, x_dev, y_dev, n_rhs);
    return FMMPC_OK;
  });
}

int fmmpc_solve(fmmpc_handle *h, const double *f_dev, const double *g_dev, double *u_dev, int32_t n_rhs,
                const fmmpc_solve_opts *opts, fmmpc_solve_info *info) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(f_dev && u_dev && opts, "solve: NULL argument");
    check_rhs(h, n_rhs);
    fmmpc_solve_info tmp{};
    int st = solve(*h, f_dev, g_dev, u_dev, n_rhs, *opts, tmp);
    if (info) *info = tmp;
    if (st != FMMPC_OK) h->err = (st == FMMPC_ERR_NOT_CONVERGED) ? "solve: not converged within maxit"
                                                                  : "solve: NaN or Inf in a residual";
    return st;
  });
}

int fmmpc_solve_host(fmmpc_handle *h, const double *f_host, const double *g_host, double *u_host,
                     int32_t n_rhs, const fmmpc_solve_opts *opts, fmmpc_solve_info *info) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(f_host && u_host && opts, "solve_host: NULL argument");
    check_rhs(h, n_rhs);
    ensure_stage(*h);
    const size_t N = (size_t)h->g.n * h->g.n * n_rhs;
    double *gdev = nullptr;
    FMMPC_CUDA(cudaMemcpyAsync(h->stage_in, f_host, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    FMMPC_CUDA(cudaMemcpyAsync(h->stage_out, u_host, sizeof(double) * N, cudaMemcpyHostToDevice, h->stream));
    if (g_host) {
      gdev = h->stage_g;
      FMMPC_CUDA(cudaMemcpyAsync(gdev, g_host, sizeof(double) * 4 * h->g.n * n_rhs, cudaMemcpyHostToDevice, h->stream));
    }
    fmmpc_solve_info tmp{};
    int st = solve(*h, h->stage_in, gdev, h->stage_out, n_rhs, *opts, tmp);
    FMMPC_CUDA(cudaMemcpyAsync(u_host, h->stage_out, sizeof(double) * N, cudaMemcpyDeviceToHost, h->stream));
    FMMPC_CUDA(cudaStreamSynchronize(h->stream));
    if (info) *info = tmp;
    return st;
  });
}

int fmmpc_query(const fmmpc_handle *h, int32_t what, int64_t *value) {
  if (!h || !value) return FMMPC_ERR_INVALID;
  switch (what) {
    case 0: *value = h->g.L; break;
    case 1: *value = h->g.m; break;
    case 2: *value = h->lists.n_m2l; break;
    case 3: *value = h->lists.n_p2p; break;
    case 4: *value = h->lists.n_m2l_vb; break;
    case 5: *value = h->lists.n_p2p_vb; break;
    case 6: *value = h->g.NG; break;
    case 7: *value = h->g.ncell; break;
    case 8: *value = (int64_t)h->g.n * h->g.n; break;
    case 9: *value = h->st.count; break;
    case 10: *value = h->launches; break;
    case 11: *value = (int64_t)(h->pool.bytes + h->kpool.bytes); break;
    case 12: {  // device-side error flags of the tensor-core kernels (bounded waits that gave up)
      int e = 0, e2 = 0;
      cudaStreamSynchronize(h->stream);
      if (h->tcp.err && cudaMemcpy(&e, h->tcp.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FMMPC_ERR_CUDA;
      if (h->tcm.err && cudaMemcpy(&e2, h->tcm.err, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
        return FMMPC_ERR_CUDA;
      *value = e | (e2 << 8);
      break;
    }
    case 13: *value = (h->tcp.enabled && h->p2p_engine == 0) ? 1 : 0; break;
    case 14: *value = h->tcm.enabled ? (h->tcm.kind == 0 ? 1 : 2) : 0; break;
    default: return FMMPC_ERR_INVALID;
  }
  return FMMPC_OK;
}

int fmmpc_export(fmmpc_handle *h, int32_t what, void *dst, int64_t bytes) {
  if (!h || !dst) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    const int64_t N = (int64_t)h->g.n * h->g.n;
    const void *src = nullptr;
    int64_t need = 0;
    switch (what) {
      case 0: src = h->tree.keys; need = 4 * N; break;
      case 1: src = h->tree.perm; need = 4 * N; break;
      case 2: src = h->tree.cell_start; need = 4 * h->g.ncell; break;
      case 3: src = h->lists.m2l; need = 12 * h->lists.n_m2l; break;
      case 4: src = h->lists.p2p; need = 8 * h->lists.n_p2p; break;
      case 5: src = h->lists.m2l_vb; need = 12 * h->lists.n_m2l_vb; break;
      case 6: src = h->lists.p2p_vb; need = 8 * h->lists.n_p2p_vb; break;
      default: throw Error(FMMPC_ERR_INVALID, "export: unknown array");
    }
    require(bytes >= need, "export: destination too small");
    if (need) FMMPC_CUDA(cudaMemcpyAsync(dst, src, need, cudaMemcpyDeviceToHost, h->stream));
    FMMPC_CUDA(cudaStreamSynchronize(h->stream));
    return FMMPC_OK;
  });
}

int fmmpc_set_p2p_engine(fmmpc_handle *h, int32_t engine) {
  if (!h || engine < 0 || engine > 1) return FMMPC_ERR_INVALID;
  h->p2p_engine = engine;
  for (auto &e : h->gcache) cudaGraphExecDestroy(e.exec);  // captured graphs used the old engine
  h->gcache.clear();
  clear_solve_graphs(*h);
  return FMMPC_OK;
}

int fmmpc_set_operator(fmmpc_handle *h, int32_t op, const double *a_dev) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(op >= FMMPC_OP_FD5 && op <= FMMPC_OP_Q1, "set_operator: unknown operator");
    require(op != FMMPC_OP_FD5_VAR || a_dev, "set_operator: the variable-coefficient operator needs a");
    const int n = h->g.n;
    if (op == FMMPC_OP_FD5_VAR) {
      const size_t na = (size_t)(n + 2) * (n + 2);
      if (!h->acoef) h->acoef = h->pool.get<double>(na);
      FMMPC_CUDA(cudaMemcpyAsync(h->acoef, a_dev, sizeof(double) * na, cudaMemcpyDeviceToDevice, h->stream));
    }
    if (op == FMMPC_OP_Q1 && !h->q1tab) {
      // Thomas coefficients of (1/6) tridiag(1, 4, 1): cp[k] and 1 / (pivot k)
      std::vector<double> t(2 * (size_t)n);
      double cprev = 0.0;
      for (int k = 0; k < n; ++k) {
        const double den = 4.0 / 6.0 - (k ? cprev / 6.0 : 0.0);
        t[n + k] = 1.0 / den;
        cprev = t[k] = (1.0 / 6.0) / den;
      }
      h->q1tab = h->pool.get<double>(t.size());
      FMMPC_CUDA(cudaMemcpyAsync(h->q1tab, t.data(), sizeof(double) * t.size(), cudaMemcpyHostToDevice, h->stream));
      FMMPC_CUDA(cudaStreamSynchronize(h->stream));
    }
    h->op = op;
    clear_solve_graphs(*h);  // they hold the previous operator
    return FMMPC_OK;
  });
}

int fmmpc_set_graphs(fmmpc_handle *h, int32_t on) {
  if (!h) return FMMPC_ERR_INVALID;
  h->graphs = on != 0;
  return FMMPC_OK;
}

int fmmpc_set_timing(fmmpc_handle *h, int32_t on) {
  if (!h) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    if (on && !h->ev[0])
      for (int k = 0; k <= fmmpc_handle::NSTAGE; ++k) FMMPC_CUDA(cudaEventCreate(&h->ev[k]));
    require(on >= 0 && on <= 2, "set_timing: mode must be 0, 1 or 2");
    h->timing = on;
    return FMMPC_OK;
  });
}

int fmmpc_get_timing(fmmpc_handle *h, float *ms, int32_t cap, int32_t *count) {
  if (!h || !ms || !count) return FMMPC_ERR_INVALID;
  return guarded(h, [&] {
    require(h->timing, "get_timing: timing is off");
    FMMPC_CUDA(cudaStreamSynchronize(h->stream));
    const int ns = fmmpc_handle::NSTAGE;
    *count = ns;
    if (h->timing == 2) {  // only M2L (5 -> 6) and P2P (9 -> 10)
      for (int k = 0; k < ns && k < cap; ++k) ms[k] = 0.0f;
      const int pairs[2][2] = {{5, 6}, {9, 10}};
      for (auto &pr : pairs)
        if (pr[0] < cap && h->stage_hit[pr[0]] && h->stage_hit[pr[1]])
          FMMPC_CUDA(cudaEventElapsedTime(&ms[pr[0]], h->ev[pr[0]], h->ev[pr[1]]));
      return FMMPC_OK;
    }
    for (int k = 0; k < ns && k < cap; ++k) {
      ms[k] = 0.0f;
      if (!h->stage_hit[k]) continue;
      int nx = k + 1;  // next stage that ran (or the end mark)
      while (nx < ns && !h->stage_hit[nx]) ++nx;
      FMMPC_CUDA(cudaEventElapsedTime(&ms[k], h->ev[k], h->ev[nx]));
    }
    return FMMPC_OK;
  });
}

void fmmpc_destroy(fmmpc_handle *h) { release(h); }

int fmmpc_autotune(const fmmpc_grid *g, const fmmpc_params *base, const fmmpc_solve_opts *opts, const double *f_dev,
                   double tol, void *stream, fmmpc_params *best, fmmpc_tune_entry *report, int32_t cap,
                   int32_t *count) {
  if (!g || !base || !opts || !f_dev || !best || !(tol > 0.0)) return set_global_error(FMMPC_ERR_INVALID, "autotune: bad argument");
  try {
    std::vector<fmmpc_tune_entry> rep;
    fmmpc_params b = *base;
    int rc = autotune(*g, *base, *opts, f_dev, tol, stream, b, rep, report && cap > 0);
    if (rc != FMMPC_OK) return rc;
    *best = b;
    if (count) *count = (int32_t)rep.size();
    for (int i = 0; report && i < cap && i < (int)rep.size(); ++i) report[i] = rep[i];
    return FMMPC_OK;
  } catch (const Error &e) {
    return set_global_error(e.code, e.msg.c_str());
  }
}

}  // extern "C"

struct fmmpc_batch {
  std::vector<fmmpc_handle *> hs;
  std::vector<cudaStream_t> streams;
  cudaStream_t user = nullptr;
  cudaEvent_t ev = nullptr;
  std::string err;
};

extern "C" {

void fmmpc_destroy_batched(fmmpc_batch *b) {
  if (!b) return;
  for (auto *h : b->hs) fmmpc_destroy(h);
  for (auto s : b->streams) cudaStreamDestroy(s);
  if (b->ev) cudaEventDestroy(b->ev);
  delete b;
}

int fmmpc_create_batched(fmmpc_batch **out, int32_t nprob, const fmmpc_grid *grids, const fmmpc_params *prm,
                         void *stream) {
  if (!out || !grids || !prm || nprob < 1) return set_global_error(FMMPC_ERR_INVALID, "create_batched: bad argument");
  *out = nullptr;
  fmmpc_batch *b = new (std::nothrow) fmmpc_batch();
  if (!b) return set_global_error(FMMPC_ERR_OOM, "host allocation failed");
  b->user = (cudaStream_t)stream;
  if (cudaEventCreateWithFlags(&b->ev, cudaEventDisableTiming) != cudaSuccess) {
    fmmpc_destroy_batched(b);
    return set_global_error(FMMPC_ERR_CUDA, "create_batched: event creation failed");
  }
  for (int i = 0; i < nprob; ++i) {
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
      fmmpc_destroy_batched(b);
      return set_global_error(FMMPC_ERR_CUDA, "create_batched: stream creation failed");
    }
    b->streams.push_back(s);
    fmmpc_handle *h = nullptr;
    const int rc = fmmpc_create(&h, &grids[i], prm, s);  // autotunes per grid when prm->autotune
    if (rc != FMMPC_OK) {
      fmmpc_destroy_batched(b);
      return rc;
    }
    b->hs.push_back(h);
  }
  *out = b;
  return FMMPC_OK;
}

int fmmpc_solve_batched(fmmpc_batch *b, const double *const *f_dev, const double *const *g_dev, double *const *u_dev,
                        const fmmpc_solve_opts *opts, fmmpc_solve_info *infos) {
  if (!b || !f_dev || !u_dev || !opts) return FMMPC_ERR_INVALID;
  try {
    // order the problem streams after the caller's stream, and the caller's after them
    FMMPC_CUDA(cudaEventRecord(b->ev, b->user));
    for (auto s : b->streams) FMMPC_CUDA(cudaStreamWaitEvent(s, b->ev, 0));
    const int rc = solve_batched(b->hs, f_dev, g_dev, u_dev, *opts, infos);
    for (auto s : b->streams) {
      FMMPC_CUDA(cudaEventRecord(b->ev, s));
      FMMPC_CUDA(cudaStreamWaitEvent(b->user, b->ev, 0));
    }
    if (rc != FMMPC_OK) b->err = "solve_batched: a problem did not converge (see infos)";
    return rc;
  } catch (const Error &e) {
    b->err = e.msg;
    return e.code;
  }
}

int fmmpc_batch_query(const fmmpc_batch *b, int32_t prob, int32_t what, int64_t *value) {
  if (!b || prob < 0 || prob >= (int)b->hs.size()) return FMMPC_ERR_INVALID;
  if (what == 100) {
    if (!value) return FMMPC_ERR_INVALID;
    *value = b->hs[prob]->g.p;
    return FMMPC_OK;
  }
  return fmmpc_query(b->hs[prob], what, value);
}

const char *fmmpc_batch_last_error(const fmmpc_batch *b) { return b ? b->err.c_str() : ""; }

const char *fmmpc_last_error(const fmmpc_handle *h) {
  return h ? h->err.c_str() : g_global_error;
}

int fmmpc_near_field_noalloc(int32_t n, double side, int32_t leaf_max, double theta, const double *r_dev,
                             double *out_dev, void *stream) {
  return near_field_noalloc(n, side, leaf_max, theta, r_dev, out_dev, stream);
}

const char *fmmpc_version(void) { return "fmmpc 0.1 sm_103a"; }

}  // extern "C"
