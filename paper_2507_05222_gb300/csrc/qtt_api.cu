// extern "C" entry points of include/qtt.h: argument checks, error translation, handle
// management.  No C++ exception crosses this file's functions.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <memory>
#include <string>

#include <cuda_profiler_api.h>

#include "qtt_algebra.h"
#include "qtt_case.h"
#include "qtt_nn.h"

namespace qtt {

static thread_local std::string g_last_error;
void set_last_error(const std::string& msg) { g_last_error = msg; }

}  // namespace qtt

using namespace qtt;

#define API_BEGIN try {
#define API_END                                        \
  }                                                    \
  catch (const qtt::Error& e) {                        \
    set_last_error(e.what());                          \
    return e.code;                                     \
  }                                                    \
  catch (const std::bad_alloc&) {                      \
    set_last_error("host allocation failed");          \
    return QTT_ERR_ALLOC;                              \
  }                                                    \
  catch (const std::exception& e) {                    \
    set_last_error(e.what());                          \
    return QTT_ERR_CUDA;                               \
  }                                                    \
  set_last_error("");                                  \
  return QTT_OK;

namespace {

void check_mps(const qtt_mps* x, const char* what) {
  if (!x) throw Error(QTT_ERR_ARG, std::string(what) + ": null MPS");
}

void check_trunc(const qtt_trunc& t) {
  if (t.chi_max < 1) throw Error(QTT_ERR_ARG, "trunc: chi_max must be >= 1");
  if (!(t.rel_tol >= 0.0) || !std::isfinite(t.rel_tol)) throw Error(QTT_ERR_ARG, "trunc: rel_tol must be >= 0");
  prec_digits(t.prec);
  if (t.apply != QTT_APPLY_GRAM && t.apply != QTT_APPLY_SKETCH) throw Error(QTT_ERR_ARG, "trunc: apply must be 0 or 1");
}

void check_solve_opts(const qtt_solve_opts& o, const char* what) {
  if (!(o.max_sweeps >= 0 && o.cg_max_iter >= 0 && o.rel_tol >= 0.0 && o.cg_tol >= 0.0 && std::isfinite(o.rel_tol) &&
        std::isfinite(o.cg_tol) && std::isfinite(o.stall) && o.stall < 1.0))
    throw Error(QTT_ERR_ARG, std::string(what) +
                                 ": solve options need max_sweeps, cg_max_iter >= 0, rel_tol, cg_tol >= 0, stall < 1");
}

void fill_solve_info(const AlsCtl& h, qtt_solve_info* info) {
  info->sweeps = h.sweeps;
  info->cg_iters = h.cg_total < 0 ? -1 : h.cg_total;
  info->rel_residual = h.res;
  info->status = h.status;
}

// QTT_OK for a solve that met its tolerance or stopped at its bond's floor; the error codes of
// include/qtt.h otherwise.  `floor_ok` = false makes a stall an error too (poisson_solve).
int solve_status_code(int status, bool floor_ok = false) {
  switch (status) {
    case QTT_SOLVE_CONVERGED: return QTT_OK;
    case QTT_SOLVE_STALLED: return floor_ok ? QTT_OK : QTT_ERR_NOT_CONVERGED;
    case QTT_SOLVE_MAX_SWEEPS: return QTT_ERR_NOT_CONVERGED;
    case QTT_SOLVE_NONFINITE: return QTT_ERR_NONFINITE;
    case QTT_SOLVE_TIMEOUT: return QTT_ERR_TIMEOUT;
    default: return QTT_ERR_CUDA;
  }
}

std::string solve_status_text(const AlsCtl& h) {
  static const char* names[] = {"converged", "stalled above the tolerance", "out of sweeps", "non-finite residual",
                                "a CG grid barrier timed out"};
  const char* s = (h.status >= 0 && h.status <= 4) ? names[h.status] : "did not finish";
  return std::string(s) + " after " + std::to_string(h.sweeps) + " sweeps, relative residual " +
         std::to_string(h.res);
}

cudaMemcpyKind kind_in(int kind) {
  if (kind == QTT_HOST) return cudaMemcpyHostToDevice;
  if (kind == QTT_DEVICE) return cudaMemcpyDeviceToDevice;
  throw Error(QTT_ERR_ARG, "pointer kind must be QTT_HOST or QTT_DEVICE");
}

cudaMemcpyKind kind_out(int kind) {
  if (kind == QTT_HOST) return cudaMemcpyDeviceToHost;
  if (kind == QTT_DEVICE) return cudaMemcpyDeviceToDevice;
  throw Error(QTT_ERR_ARG, "pointer kind must be QTT_HOST or QTT_DEVICE");
}

// Collects the discarded weight of the roundings of one call when the caller asked for it.
struct DiscScope {
  Ctx& c;
  DBuf acc;
  DiscScope(Ctx& ctx, bool on) : c(ctx) {
    if (on) {
      acc.reset(&c, 1);
      fill(c, acc.p, 1, 0.0);
      c.disc_acc = acc.p;
    }
  }
  ~DiscScope() { c.disc_acc = nullptr; }
  DiscScope(const DiscScope&) = delete;
  DiscScope& operator=(const DiscScope&) = delete;
};

// max bond, norm (right-canonical result: the norm of its first core) and discarded norm
// (sqrt of the accumulated weight; -1 when the result is a variational fit).
void fill_info(Ctx& c, const qtt_mps* y, qtt_round_info* info, const DiscScope* disc) {
  if (!info) return;
  int mb = 1;
  for (int b : y->bonds) mb = std::max(mb, b);
  info->max_bond = mb;
  DBuf d(&c, 1);
  dot_dev(c, y, y, d.p);
  double v[2] = {0.0, -1.0};
  QTT_CUDA(cudaMemcpyAsync(&v[0], d.p, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  if (disc && disc->acc.p)
    QTT_CUDA(cudaMemcpyAsync(&v[1], disc->acc.p, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  info->norm = std::sqrt(std::max(v[0], 0.0));
  info->discarded_norm = v[1] >= 0.0 ? std::sqrt(v[1]) : -1.0;
}

__global__ void k_reorder(const double* __restrict__ src, double* __restrict__ dst, int ne, int nx, int ordering,
                          int inverse) {
  const int n = ne + nx;
  const int64_t total = int64_t(1) << n;
  for (int64_t q = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; q < total; q += int64_t(gridDim.x) * blockDim.x) {
    int64_t i = 0, j = 0;
    int p = 0;
    if (ordering == QTT_ORDER_SEQUENTIAL) {
      i = q >> nx;
      j = q & ((int64_t(1) << nx) - 1);
    } else {
      for (int l = 0; l < (ne > nx ? ne : nx); ++l) {
        if (l < ne) {
          int64_t bit = (q >> (n - 1 - p)) & 1;
          i |= bit << (ne - 1 - l);
          ++p;
        }
        if (l < nx) {
          int64_t bit = (q >> (n - 1 - p)) & 1;
          j |= bit << (nx - 1 - l);
          ++p;
        }
      }
    }
    int64_t f = (i << nx) | j;  // row-major field index
    if (inverse) dst[f] = src[q];
    else dst[q] = src[f];
  }
}

}  // namespace

extern "C" {

int qtt_ctx_create(qtt_ctx** out, int device, void* cuda_stream, qtt_alloc_fn alloc, qtt_free_fn free_fn, void* user) {
  API_BEGIN
  QTT_CHECK_ARG(out != nullptr, "ctx_create: out is null");
  QTT_CHECK_ARG((alloc == nullptr) == (free_fn == nullptr), "ctx_create: give both alloc and free or neither");
  int ndev = 0;
  QTT_CUDA(cudaGetDeviceCount(&ndev));
  QTT_CHECK_ARG(device >= 0 && device < ndev, "ctx_create: no such device");
  QTT_CUDA(cudaSetDevice(device));
  std::unique_ptr<Ctx> c(new Ctx);
  c->device = device;
  c->stream = static_cast<cudaStream_t>(cuda_stream);
  QTT_CUDA(cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, device));
  c->pool = new Pool(alloc, free_fn, user);
  c->root = c.get();
  c->alloc_fn = alloc;
  c->free_fn = free_fn;
  c->alloc_user = user;
  init_tile_counters(*c);
  *out = reinterpret_cast<qtt_ctx*>(c.release());
  API_END
}

void qtt_ctx_destroy(qtt_ctx* ctx) {
  if (!ctx) return;
  Ctx* c = reinterpret_cast<Ctx*>(ctx);
  cudaStreamSynchronize(c->stream);
  destroy_workers(*c);
  for (auto e : c->prof.free_events) cudaEventDestroy(e);
  for (int k = 0; k < KC_N; ++k)
    for (auto& pr : c->prof.pending[k]) {
      cudaEventDestroy(pr.e0);
      cudaEventDestroy(pr.e1);
    }
  free_tile_counters(*c);
  free_autotuner(*c);
  if (c->prof.dev_flops) cudaFree(c->prof.dev_flops);
  if (c->side) cudaStreamDestroy(c->side);
  delete c->pool;
  delete c;
}

int qtt_ctx_sync(qtt_ctx* ctx) {
  API_BEGIN
  QTT_CHECK_ARG(ctx, "ctx is null");
  QTT_CUDA(cudaStreamSynchronize(reinterpret_cast<Ctx*>(ctx)->stream));
  API_END
}

const char* qtt_last_error(void) { return g_last_error.c_str(); }

int qtt_profiler_range(int start) {
  API_BEGIN
  if (start) QTT_CUDA(cudaProfilerStart());
  else QTT_CUDA(cudaProfilerStop());
  API_END
}

int64_t qtt_ctx_kernel_launches(qtt_ctx* ctx) { return ctx ? reinterpret_cast<Ctx*>(ctx)->launches : 0; }

size_t qtt_ctx_pool_bytes(qtt_ctx* ctx) {
  if (!ctx) return 0;
  const Ctx* c = reinterpret_cast<Ctx*>(ctx);
  size_t b = c->pool->held();
  for (const Ctx* w : c->workers) b += w->pool->held();
  return b;
}

int qtt_ctx_profile(qtt_ctx* ctx, int on, double* ms_out, double* flops_out, int64_t* launches_out) {
  API_BEGIN
  QTT_CHECK_ARG(ctx, "ctx is null");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  Profiler& P = c.prof;
  if (P.dev_flops) {
    double f = 0.0;
    QTT_CUDA(cudaMemcpy(&f, P.dev_flops, sizeof(double), cudaMemcpyDeviceToHost));
    QTT_CUDA(cudaMemset(P.dev_flops, 0, sizeof(double)));
    P.flops[KC_CG] += f;
  } else if (on) {
    QTT_CUDA(cudaMalloc(&P.dev_flops, sizeof(double)));
    QTT_CUDA(cudaMemset(P.dev_flops, 0, sizeof(double)));
  }
  for (auto& row : P.phase_ms)
    for (double& v : row) v = 0.0;
  for (int k = 0; k < KC_N; ++k) {
    double ms = 0.0;
    for (auto& sp : P.pending[k]) {
      float t = 0.f;
      QTT_CUDA(cudaEventElapsedTime(&t, sp.e0, sp.e1));
      ms += t;
      if (k < KC_KERNEL_CLASSES) P.phase_ms[sp.phase < 0 ? KC_PHASES : sp.phase][k] += t;
      P.free_events.push_back(sp.e0);
      P.free_events.push_back(sp.e1);
    }
    P.pending[k].clear();
    if (ms_out) ms_out[k] = ms;
    if (flops_out) flops_out[k] = P.flops[k];
    if (launches_out) launches_out[k] = P.launches[k];
    P.flops[k] = 0.0;
    P.launches[k] = 0;
  }
  for (int i = 0; i <= KC_PHASES; ++i) {
    P.phase_launches[i] = P.acc_phase_launches[i];
    P.acc_phase_launches[i] = 0;
  }
  P.phase = -1;
  P.on = on != 0;
  API_END
}

int qtt_ctx_profile_phases(qtt_ctx* ctx, double* ms_out, int64_t* launches_out) {
  API_BEGIN
  QTT_CHECK_ARG(ctx, "ctx is null");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  for (int i = 0; i <= KC_PHASES; ++i) {
    for (int k = 0; k < KC_KERNEL_CLASSES; ++k)
      if (ms_out) ms_out[i * KC_KERNEL_CLASSES + k] = c.prof.phase_ms[i][k];
    if (launches_out) launches_out[i] = c.prof.phase_launches[i];
  }
  API_END
}

// ------------------------------------------------------------------ MPS / MPO

int qtt_mps_create(qtt_ctx* ctx, int n, int d, const int* bonds, const double* cores, int kind, qtt_mps** out) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && out && bonds, "mps_create: null argument");
  QTT_CHECK_ARG(n >= 1 && n <= 64 && d >= 1 && d <= 16, "mps_create: n in [1, 64], d in [1, 16]");
  std::vector<int> b(bonds, bonds + n + 1);
  QTT_CHECK_ARG(b[0] == 1 && b[n] == 1, "mps_create: bonds[0] and bonds[n] must be 1");
  for (int v : b) QTT_CHECK_ARG(v >= 1 && v <= 4096, "mps_create: bonds must be in [1, 4096]");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  std::unique_ptr<qtt_mps> x(new_mps(&c, n, d, b));
  if (cores) {
    cudaMemcpyKind k = kind_in(kind);
    int64_t src = 0;
    for (int i = 0; i < n; ++i) {
      int64_t sz = int64_t(b[i]) * d * b[i + 1];
      QTT_CUDA(cudaMemcpyAsync(x->core(i), cores + src, sz * sizeof(double), k, c.stream));
      src += sz;
    }
    if (kind == QTT_HOST) QTT_CUDA(cudaStreamSynchronize(c.stream));
  } else {
    fill(c, x->buf.p, x->off[n], 0.0);
  }
  *out = x.release();
  API_END
}

int qtt_mps_free(qtt_mps* x) {
  API_BEGIN
  if (x) free_mps(x);
  API_END
}

int qtt_mps_n(const qtt_mps* x) { return x ? x->n : 0; }
int qtt_mps_d(const qtt_mps* x) { return x ? x->d : 0; }

int qtt_mps_bonds(const qtt_mps* x, int* bonds_out) {
  API_BEGIN
  check_mps(x, "mps_bonds");
  QTT_CHECK_ARG(bonds_out, "mps_bonds: null output");
  std::memcpy(bonds_out, x->bonds.data(), x->bonds.size() * sizeof(int));
  API_END
}

int64_t qtt_mps_size(const qtt_mps* x) {
  if (!x) return 0;
  int64_t s = 0;
  for (int k = 0; k < x->n; ++k) s += int64_t(x->bonds[k]) * x->d * x->bonds[k + 1];
  return s;
}

int qtt_mps_get_cores(const qtt_mps* x, double* dst, int kind) {
  API_BEGIN
  check_mps(x, "mps_get_cores");
  QTT_CHECK_ARG(dst, "mps_get_cores: null destination");
  Ctx& c = *x->ctx;
  cudaMemcpyKind k = kind_out(kind);
  int64_t o = 0;
  for (int i = 0; i < x->n; ++i) {
    int64_t sz = int64_t(x->bonds[i]) * x->d * x->bonds[i + 1];
    QTT_CUDA(cudaMemcpyAsync(dst + o, x->core(i), sz * sizeof(double), k, c.stream));
    o += sz;
  }
  if (kind == QTT_HOST) QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

const double* qtt_mps_device_ptr(const qtt_mps* x) { return x ? x->buf.p : nullptr; }

int qtt_mps_copy(const qtt_mps* x, qtt_mps** out) {
  API_BEGIN
  check_mps(x, "mps_copy");
  QTT_CHECK_ARG(out, "mps_copy: null output");
  *out = mps_copy(*x->ctx, x);
  API_END
}

int qtt_mpo_create(qtt_ctx* ctx, int n, int d, const int* bonds, const double* cores, int kind, qtt_mpo** out) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && out && bonds, "mpo_create: null argument");
  QTT_CHECK_ARG(n >= 1 && n <= 64 && d >= 1 && d <= 4, "mpo_create: n in [1, 64], d in [1, 4]");
  std::vector<int> b(bonds, bonds + n + 1);
  QTT_CHECK_ARG(b[0] == 1 && b[n] == 1, "mpo_create: bonds[0] and bonds[n] must be 1");
  for (int v : b) QTT_CHECK_ARG(v >= 1 && v <= 256, "mpo_create: bonds must be in [1, 256]");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  std::unique_ptr<qtt_mpo> m(new_mpo(&c, n, d, b));
  if (cores) {
    cudaMemcpyKind k = kind_in(kind);
    int64_t src = 0;
    for (int i = 0; i < n; ++i) {
      int64_t sz = int64_t(b[i]) * d * d * b[i + 1];
      QTT_CUDA(cudaMemcpyAsync(m->core(i), cores + src, sz * sizeof(double), k, c.stream));
      src += sz;
    }
    if (kind == QTT_HOST) QTT_CUDA(cudaStreamSynchronize(c.stream));
  } else {
    fill(c, m->buf.p, m->off[n], 0.0);
  }
  *out = m.release();
  API_END
}

int qtt_mpo_free(qtt_mpo* m) {
  API_BEGIN
  if (m) free_mpo(m);
  API_END
}

int qtt_mpo_bonds(const qtt_mpo* m, int* bonds_out) {
  API_BEGIN
  QTT_CHECK_ARG(m && bonds_out, "mpo_bonds: null argument");
  std::memcpy(bonds_out, m->bonds.data(), m->bonds.size() * sizeof(int));
  API_END
}

int qtt_mpo_get_cores(const qtt_mpo* m, double* dst, int kind) {
  API_BEGIN
  QTT_CHECK_ARG(m && dst, "mpo_get_cores: null argument");
  Ctx& c = *m->ctx;
  cudaMemcpyKind k = kind_out(kind);
  int64_t o = 0;
  for (int i = 0; i < m->n; ++i) {
    int64_t sz = int64_t(m->bonds[i]) * m->d * m->d * m->bonds[i + 1];
    QTT_CUDA(cudaMemcpyAsync(dst + o, m->core(i), sz * sizeof(double), k, c.stream));
    o += sz;
  }
  if (kind == QTT_HOST) QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

// ------------------------------------------------------------------ TT operations

int qtt_encode(qtt_ctx* ctx, const double* dense, int kind, int n, int d, qtt_trunc tr, qtt_mps** out,
               qtt_round_info* info) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && dense && out, "encode: null argument");
  QTT_CHECK_ARG(n >= 1 && d >= 2 && std::pow(double(d), n) <= double(int64_t(1) << 31), "encode: d^n must be <= 2^31");
  check_trunc(tr);
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  int64_t N = 1;
  for (int i = 0; i < n; ++i) N *= d;
  DBuf buf(&c, size_t(N));
  QTT_CUDA(cudaMemcpyAsync(buf.p, dense, N * sizeof(double), kind_in(kind), c.stream));
  DiscScope disc(c, info != nullptr);
  qtt_mps* y = encode_dense(c, buf.p, n, d, tr.chi_max, tr.rel_tol);
  fill_info(c, y, info, &disc);
  *out = y;
  API_END
}

int qtt_decode(qtt_ctx* ctx, const qtt_mps* x, double* dense, int kind) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && dense, "decode: null argument");
  check_mps(x, "decode");
  QTT_CHECK_ARG(std::pow(double(x->d), x->n) <= double(int64_t(1) << 26), "decode: at most 2^26 values");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  int64_t N = 1;
  for (int i = 0; i < x->n; ++i) N *= x->d;
  if (kind == QTT_DEVICE) {
    decode_dense(c, x, dense);
  } else {
    DBuf buf(&c, size_t(N));
    decode_dense(c, x, buf.p);
    QTT_CUDA(cudaMemcpyAsync(dense, buf.p, N * sizeof(double), kind_out(kind), c.stream));
    QTT_CUDA(cudaStreamSynchronize(c.stream));
  }
  API_END
}

int qtt_field_to_vector(qtt_ctx* ctx, const double* src, double* dst, int kind, int n_eta, int n_xi, int ordering,
                        int inverse) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && src && dst && src != dst, "field_to_vector: null or aliased buffers");
  QTT_CHECK_ARG(n_eta >= 1 && n_xi >= 1 && n_eta + n_xi <= 30, "field_to_vector: grid bits");
  QTT_CHECK_ARG(ordering == QTT_ORDER_SEQUENTIAL || ordering == QTT_ORDER_INTERLEAVED, "field_to_vector: ordering");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  int64_t N = int64_t(1) << (n_eta + n_xi);
  DBuf a(&c, size_t(N)), b(&c, size_t(N));
  QTT_CUDA(cudaMemcpyAsync(a.p, src, N * sizeof(double), kind_in(kind), c.stream));
  int grid = int(std::min<int64_t>((N + 255) / 256, 65535 * 4));
  k_reorder<<<grid, 256, 0, c.stream>>>(a.p, b.p, n_eta, n_xi, ordering, inverse);
  after_launch(c, "reorder");
  QTT_CUDA(cudaMemcpyAsync(dst, b.p, N * sizeof(double), kind_out(kind), c.stream));
  if (kind == QTT_HOST) QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

int qtt_round(qtt_ctx* ctx, const qtt_mps* x, qtt_trunc tr, qtt_mps** out, qtt_round_info* info) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && out, "round: null argument");
  check_mps(x, "round");
  check_trunc(tr);
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  DigitsScope prec(c, prec_digits(tr.prec));
  DiscScope disc(c, info != nullptr);
  qtt_mps* y = round_any(c, x, tr.chi_max, tr.rel_tol);
  fill_info(c, y, info, &disc);
  *out = y;
  API_END
}

int mps_axpby_round(qtt_ctx* ctx, double alpha, const qtt_mps* x, double beta, const qtt_mps* y, qtt_trunc tr,
                    qtt_mps** out, qtt_round_info* info) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && out, "axpby: null argument");
  check_mps(x, "axpby x");
  check_mps(y, "axpby y");
  QTT_CHECK_ARG(x->n == y->n && x->d == y->d, "axpby: x and y differ in n or d");
  QTT_CHECK_ARG(std::isfinite(alpha) && std::isfinite(beta), "axpby: non-finite coefficient");
  check_trunc(tr);
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  DigitsScope prec(c, prec_digits(tr.prec));
  std::unique_ptr<qtt_mps, void (*)(qtt_mps*)> s(direct_sum(c, alpha, x, beta, y), free_mps);
  DiscScope disc(c, info != nullptr);
  qtt_mps* z = round_any(c, s.get(), tr.chi_max, tr.rel_tol);
  fill_info(c, z, info, &disc);
  *out = z;
  API_END
}

int mpo_apply_round(qtt_ctx* ctx, const qtt_mpo* M, const qtt_mps* x, qtt_trunc tr, qtt_mps** out,
                    qtt_round_info* info) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && M && out, "apply: null argument");
  check_mps(x, "apply x");
  QTT_CHECK_ARG(M->n == x->n && M->d == x->d, "apply: operator and vector differ in n or d");
  check_trunc(tr);
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  DigitsScope prec(c, prec_digits(tr.prec));
  qtt_mps* y;
  DiscScope disc(c, info != nullptr);
  if (tr.rel_tol > 0.0) {
    std::unique_ptr<qtt_mps, void (*)(qtt_mps*)> e(mpo_mps_exact(c, M, x), free_mps);
    y = round_any(c, e.get(), tr.chi_max, tr.rel_tol);
  } else if (tr.apply == QTT_APPLY_SKETCH) {
    y = apply_round_sketch(c, M, x, tr.chi_max, 0.0);
  } else {
    y = apply_round_gram(c, M, x, tr.chi_max, 0.0);
  }
  fill_info(c, y, info, &disc);
  *out = y;
  API_END
}

int mps_hadamard_round(qtt_ctx* ctx, const qtt_mps* a, const qtt_mps* b, qtt_trunc tr, const qtt_mps* init, int sweeps,
                       qtt_mps** out, qtt_round_info* info) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && out, "hadamard: null argument");
  check_mps(a, "hadamard a");
  check_mps(b, "hadamard b");
  QTT_CHECK_ARG(a->n == b->n && a->d == b->d, "hadamard: a and b differ in n or d");
  QTT_CHECK_ARG(sweeps >= 0 && sweeps <= 1000, "hadamard: sweeps in [0, 1000]");
  check_trunc(tr);
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  DigitsScope prec(c, prec_digits(tr.prec));
  qtt_mps* y;
  bool canonical;
  if (init) {
    QTT_CHECK_ARG(init->n == a->n && init->d == a->d, "hadamard: init shape");
    y = mps_copy(c, init);
    canonical = false;
  } else {
    y = zipup_hadamard(c, a, b, tr.chi_max);
    canonical = true;
  }
  std::unique_ptr<qtt_mps, void (*)(qtt_mps*)> guard(y, free_mps);
  fit(c, {Term::had(1.0, a, b)}, y, sweeps, canonical);
  fill_info(c, y, info, nullptr);
  *out = guard.release();
  API_END
}

int qtt_sym_eig(qtt_ctx* ctx, int n, const double* S, double* w, double* V) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && S && w && V, "sym_eig: null argument");
  QTT_CHECK_ARG(n >= 1 && n <= 256, "sym_eig: n in [1, 256]");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  size_t nn = size_t(n) * n;
  DBuf dS(&c, nn), dw(&c, size_t(n)), dV(&c, nn);
  QTT_CUDA(cudaMemcpyAsync(dS.p, S, nn * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  eigh(c, n, dS.p, dw.p, dV.p);
  QTT_CUDA(cudaMemcpyAsync(w, dw.p, n * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaMemcpyAsync(V, dV.p, nn * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

int qtt_qr(qtt_ctx* ctx, int m, int n, int trans, const double* A, double* Q, double* R, int path) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && A && Q, "qr: null argument");
  QTT_CHECK_ARG(m >= 1 && n >= 1 && int64_t(m) * n <= (int64_t(1) << 22), "qr: m, n >= 1 and m n <= 2^22");
  QTT_CHECK_ARG(path >= 0 && path <= 2, "qr: path must be 0, 1 or 2");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  const int kk = std::min(m, n);
  const size_t mn = size_t(m) * n;
  DBuf dA(&c, mn), dQ(&c, size_t(m) * kk), dR(&c, size_t(kk) * n);
  QTT_CUDA(cudaMemcpyAsync(dA.p, A, mn * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  qr(c, 1, m, n, trans, dA.p, 0, dQ.p, 0, R ? dR.p : nullptr, 0, path);
  QTT_CUDA(cudaMemcpyAsync(Q, dQ.p, size_t(m) * kk * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  if (R) QTT_CUDA(cudaMemcpyAsync(R, dR.p, size_t(kk) * n * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

int qtt_dgemm(qtt_ctx* ctx, int m, int n, int k, const double* A, const double* B, double* C, int path) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && A && B && C, "dgemm: null argument");
  QTT_CHECK_ARG(m >= 1 && n >= 1 && k >= 1 && int64_t(m) * k <= (int64_t(1) << 26) &&
                    int64_t(k) * n <= (int64_t(1) << 26) && int64_t(m) * n <= (int64_t(1) << 26),
                "dgemm: sizes must be >= 1 with each operand at most 2^26 values");
  QTT_CHECK_ARG(path >= 0 && path <= 3, "dgemm: path must be 0, 1, 2 or 3");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  DBuf dA(&c, size_t(m) * k), dB(&c, size_t(k) * n), dC(&c, size_t(m) * n);
  QTT_CUDA(cudaMemcpyAsync(dA.p, A, size_t(m) * k * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  QTT_CUDA(cudaMemcpyAsync(dB.p, B, size_t(k) * n * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  if (path >= 2) {
    const int saved = c.gemm_mode;
    c.gemm_mode = path;          // 2: digit products on mma.sync, 3: on tcgen05
    try {
      gemm_ozaki(c, 1, m, n, k, 1.0, dA.p, 0, k, 1, dB.p, 0, n, 1, 0.0, dC.p, 0, n, 1);
    } catch (...) {
      c.gemm_mode = saved;
      throw;
    }
    c.gemm_mode = saved;
  } else {
    const int saved = c.gemm_mode;
    if (path == 1) c.gemm_mode = 1;
    try {
      gemm(c, 1, m, n, k, 1.0, dA.p, 0, k, 1, dB.p, 0, n, 1, 0.0, dC.p, 0, n, 1);
    } catch (...) {
      c.gemm_mode = saved;
      throw;
    }
    c.gemm_mode = saved;
  }
  QTT_CUDA(cudaMemcpyAsync(C, dC.p, size_t(m) * n * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

int qtt_ctx_set_gemm_mode(qtt_ctx* ctx, int mode) {
  API_BEGIN
  QTT_CHECK_ARG(ctx, "ctx is null");
  QTT_CHECK_ARG(mode >= 0 && mode <= 3,
                "gemm mode must be 0 (tensor cores for large products), 1 (FP64 pipe), 2 (digit products on "
                "mma.sync) or 3 (digit products on tcgen05)");
  reinterpret_cast<Ctx*>(ctx)->gemm_mode = mode;
  API_END
}

int qtt_ctx_set_autotune(qtt_ctx* ctx, int on) {
  API_BEGIN
  QTT_CHECK_ARG(ctx, "ctx is null");
  QTT_CHECK_ARG(on == 0 || on == 1 || on == -1, "autotune: on must be 1, 0 or -1 (clear the table)");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  if (on == -1) {
    c.tuned.clear();
    c.autotune = false;
  } else {
    c.autotune = on == 1;
  }
  API_END
}

int qtt_ctx_set_precision(qtt_ctx* ctx, int prec) {
  API_BEGIN
  QTT_CHECK_ARG(ctx, "ctx is null");
  reinterpret_cast<Ctx*>(ctx)->digits = prec_digits(prec);
  API_END
}

int qtt_ctx_autotune_table(qtt_ctx* ctx, int max_rows, int64_t* rows, int* count) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && count, "autotune_table: null argument");
  QTT_CHECK_ARG(max_rows >= 0 && (max_rows == 0 || rows), "autotune_table: rows needed for max_rows > 0");
  *count = int(autotune_table(*reinterpret_cast<Ctx*>(ctx), max_rows, rows));
  API_END
}

int qtt_check_recip(qtt_ctx* ctx, int n, const double* x, double* err2) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && x && err2 && n >= 1 && n <= (1 << 24), "check_recip: arguments");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  DBuf dx(&c, size_t(n)), de(&c, 2);
  QTT_CUDA(cudaMemcpyAsync(dx.p, x, size_t(n) * sizeof(double), cudaMemcpyHostToDevice, c.stream));
  check_recip(c, n, dx.p, de.p);
  QTT_CUDA(cudaMemcpyAsync(err2, de.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

int mps_dot(qtt_ctx* ctx, const qtt_mps* a, const qtt_mps* b, double* out_host) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && out_host, "dot: null argument");
  check_mps(a, "dot a");
  check_mps(b, "dot b");
  QTT_CHECK_ARG(a->n == b->n && a->d == b->d, "dot: a and b differ in n or d");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  DBuf d(&c, 1);
  dot_dev(c, a, b, d.p);
  QTT_CUDA(cudaMemcpyAsync(out_host, d.p, sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

int poisson_solve(qtt_ctx* ctx, const qtt_mpo* A, const qtt_mps* b, qtt_mps* x_inout, const qtt_solve_opts* opts,
                  qtt_solve_info* info) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && A && opts, "poisson_solve: null argument");
  check_mps(b, "poisson_solve b");
  check_mps(x_inout, "poisson_solve x");
  QTT_CHECK_ARG(A->n == b->n && b->n == x_inout->n && A->d == b->d && b->d == x_inout->d, "poisson_solve: shapes");
  check_solve_opts(*opts, "poisson_solve");
  for (int k = 1; k < x_inout->n; ++k)
    QTT_CHECK_ARG(x_inout->bonds[k] <= x_inout->d * x_inout->bonds[k + 1] &&
                      x_inout->bonds[k] <= x_inout->d * x_inout->bonds[k - 1],
                  "poisson_solve: x bonds must satisfy r_k <= d r_{k+-1}");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  DBuf ctl(&c, kAlsCtlDoubles);
  AlsCtl* cp = reinterpret_cast<AlsCtl*>(ctl.p);
  als(c, A, {Term::vec(1.0, b)}, x_inout, *opts, false, cp);
  AlsCtl h;
  QTT_CUDA(cudaMemcpyAsync(&h, cp, sizeof(AlsCtl), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  if (info) fill_solve_info(h, info);
  const int rc = solve_status_code(h.status);
  if (rc != QTT_OK) {
    set_last_error("poisson_solve: " + solve_status_text(h));
    return rc;
  }
  API_END
}

// ------------------------------------------------------------------ case

int qtt_case_create(qtt_ctx* ctx, const qtt_case_params* p, qtt_case** out) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && p && out, "case_create: null argument");
  QTT_CHECK_ARG(p->poisson_warm == 0 || p->poisson_warm == 1, "case_create: poisson_warm must be 0 or 1");
  QTT_CHECK_ARG(p->apply == QTT_APPLY_GRAM || p->apply == QTT_APPLY_SKETCH, "case_create: apply must be 0 or 1");
  QTT_CHECK_ARG(p->apply != QTT_APPLY_SKETCH || 2 * p->chi <= 256, "case_create: the sketched products need chi <= 128");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  std::unique_ptr<qtt_case> h(new qtt_case);
  h->ctx = &c;
  h->cs = build_case(c, *p);
  *out = h.release();
  API_END
}

int qtt_case_free(qtt_case* h) {
  API_BEGIN
  if (h) {
    delete h->cs;
    delete h;
  }
  API_END
}

int qtt_case_set_state(qtt_case* h, const qtt_mps* u, const qtt_mps* v, const qtt_mps* p) {
  API_BEGIN
  QTT_CHECK_ARG(h, "case_set_state: null case");
  check_mps(u, "case_set_state u");
  check_mps(v, "case_set_state v");
  check_mps(p, "case_set_state p");
  Case& cs = *h->cs;
  Ctx& c = *h->ctx;
  const int n = cs.P.n_eta + cs.P.n_xi;
  for (const qtt_mps* x : {u, v, p}) {
    QTT_CHECK_ARG(x->n == n && x->d == 2, "case_set_state: field must have n_eta + n_xi cores of size 2");
    for (int k = 1; k < n; ++k)
      QTT_CHECK_ARG(x->bonds[k] <= 2 * x->bonds[k + 1] && x->bonds[k] <= 2 * x->bonds[k - 1],
                    "case_set_state: bonds must satisfy r_k <= 2 r_{k+-1}");
  }
  // Same bond profile as the current state: copy into the existing buffers (a captured step
  // graph, which refers to these addresses, stays valid).  Otherwise new buffers.
  const bool same = cs.u && cs.v && cs.p && cs.u->bonds == u->bonds && cs.v->bonds == v->bonds &&
                    cs.p->bonds == p->bonds;
  if (same) {
    copy(c, cs.u->buf.p, u->buf.p, u->off[n]);
    copy(c, cs.v->buf.p, v->buf.p, v->off[n]);
    copy(c, cs.p->buf.p, p->buf.p, p->off[n]);
    right_orthonormalize(c, cs.u);
    right_orthonormalize(c, cs.v);
    right_orthonormalize(c, cs.p);
  } else {
    cs.drop_graph();   // the captured step refers to the old state buffers
    qtt_mps* nu = mps_copy(c, u);
    qtt_mps* nv = mps_copy(c, v);
    qtt_mps* np = mps_copy(c, p);
    right_orthonormalize(c, nu);
    right_orthonormalize(c, nv);
    right_orthonormalize(c, np);
    if (cs.u) free_mps(cs.u);
    if (cs.v) free_mps(cs.v);
    if (cs.p) free_mps(cs.p);
    if (cs.p_prev) free_mps(cs.p_prev);
    cs.u = nu;
    cs.v = nv;
    cs.p = np;
    cs.p_prev = mps_copy(c, np);
  }
  cs.prev_valid = false;   // no previous pressure: the next step starts its Poisson solve from p
  API_END
}

int qtt_case_get_state(qtt_case* h, qtt_mps** u, qtt_mps** v, qtt_mps** p) {
  API_BEGIN
  QTT_CHECK_ARG(h, "case_get_state: null case");
  Case& cs = *h->cs;
  QTT_CHECK_ARG(cs.u && cs.v && cs.p, "case_get_state: state not set");
  if (u) *u = mps_copy(*h->ctx, cs.u);
  if (v) *v = mps_copy(*h->ctx, cs.v);
  if (p) *p = mps_copy(*h->ctx, cs.p);
  API_END
}

int qtt_case_get_operator(qtt_case* h, int which, qtt_mpo** out) {
  API_BEGIN
  QTT_CHECK_ARG(h && out, "case_get_operator: null argument");
  Case& cs = *h->cs;
  const qtt_mpo* ops[8] = {cs.Dx, cs.Dz, cs.Dxp, cs.Dzp, cs.H, cs.Ap, cs.Px, cs.Pz};
  QTT_CHECK_ARG(which >= 0 && which < 8, "case_get_operator: which in [0, 7]");
  const qtt_mpo* m = ops[which];
  qtt_mpo* r = new_mpo(h->ctx, m->n, m->d, m->bonds);
  copy(*h->ctx, r->buf.p, m->buf.p, m->off[m->n]);
  *out = r;
  API_END
}

int qtt_case_get_vector(qtt_case* h, int which, qtt_mps** out) {
  API_BEGIN
  QTT_CHECK_ARG(h && out, "case_get_vector: null argument");
  Case& cs = *h->cs;
  const qtt_mps* vs[8] = {cs.bcx_u, cs.bcz_u, cs.bcx_v, cs.bcz_v, cs.JbcLap_u, cs.JbcLap_v, cs.bcdiv_w, cs.absJ};
  QTT_CHECK_ARG(which >= 0 && which < 8, "case_get_vector: which in [0, 7]");
  *out = vs[which] ? mps_copy(*h->ctx, vs[which]) : nullptr;
  API_END
}

// Reads the device records of nsteps steps of one case: fills per_step (may be null), adds the
// replayed kernels to the launch count, returns the most severe outcome over the steps
// (timeout, non-finite, out of sweeps) with its message in msg.
static int read_step_records(Ctx& c, Case& cs, const double* hrec, int nsteps, bool forces, qtt_step_info* per_step,
                             const char* who, std::string& msg) {
  int rc = QTT_OK;
  for (int s = 0; s < nsteps; ++s) {
    const double* r = &hrec[size_t(s) * kStepRecDoubles];
    AlsCtl h[3];
    std::memcpy(h, r, sizeof(h));
    const int finite = r[kStepRecFinite] != 0.0;
    if (per_step) {
      fill_solve_info(h[0], &per_step[s].u);
      fill_solve_info(h[1], &per_step[s].v);
      fill_solve_info(h[2], &per_step[s].p);
      per_step[s].finite = finite;
      per_step[s].cd = forces ? r[kStepRecForces] : 0.0;
      per_step[s].cl = forces ? r[kStepRecForces + 1] : 0.0;
    }
    if (cs.use_graph && !(s == 0 && cs.last_first_eager))
      c.root->launches += cs.graph_launches + int64_t(h[0].sweeps) * cs.body_launches[0] +
                                          int64_t(h[1].sweeps) * cs.body_launches[1] +
                                          int64_t(h[2].sweeps) * cs.body_launches[2];
    for (int i = 0; i < 3; ++i) {
      const int e = solve_status_code(h[i].status, true);
      const char* which[3] = {"u momentum", "v momentum", "Poisson"};
      if (e != QTT_OK && (rc == QTT_OK || e == QTT_ERR_TIMEOUT || (e == QTT_ERR_NONFINITE && rc != QTT_ERR_TIMEOUT))) {
        rc = e;
        msg = std::string(who) + ": " + which[i] + " solve of step " + std::to_string(s) + ": " +
              solve_status_text(h[i]);
      }
    }
    if (!finite && rc != QTT_ERR_TIMEOUT) {
      rc = QTT_ERR_NONFINITE;
      msg = std::string(who) + ": the new velocity of step " + std::to_string(s) + " is not finite";
    }
  }
  return rc;
}

// more severe of two outcomes: timeout > non-finite > any other error > OK
static int more_severe(int a, int b) {
  auto rank = [](int e) { return e == QTT_OK ? 0 : e == QTT_ERR_TIMEOUT ? 3 : e == QTT_ERR_NONFINITE ? 2 : 1; };
  return rank(b) > rank(a) ? b : a;
}

int fractional_step(qtt_ctx* ctx, qtt_case* h, int nsteps, int with_forces, qtt_step_info* per_step) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && h, "fractional_step: null argument");
  QTT_CHECK_ARG(nsteps >= 0, "fractional_step: nsteps >= 0");
  Case& cs = *h->cs;
  QTT_CHECK_ARG(cs.u && cs.v && cs.p, "fractional_step: state not set");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  if (nsteps == 0) {
    set_last_error("");
    return QTT_OK;
  }
  const bool forces = with_forces && per_step;
  DBuf rec(&c, size_t(nsteps) * kStepRecDoubles);
  fill(c, rec.p, int64_t(nsteps) * kStepRecDoubles, 0.0);
  run_steps(c, cs, nsteps, forces, rec.p);
  std::vector<double> hrec(size_t(nsteps) * kStepRecDoubles);
  QTT_CUDA(cudaMemcpyAsync(hrec.data(), rec.p, hrec.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  std::string msg;
  const int rc = read_step_records(c, cs, hrec.data(), nsteps, forces, per_step, "fractional_step", msg);
  if (rc != QTT_OK) {
    set_last_error(msg);
    return rc;
  }
  API_END
}

int fractional_step_batch(qtt_ctx* ctx, int ncases, qtt_case* const* cases, int nsteps, int with_forces,
                          qtt_step_info* per_step, int* status) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && cases && ncases >= 1, "fractional_step_batch: null argument or ncases < 1");
  QTT_CHECK_ARG(nsteps >= 0, "fractional_step_batch: nsteps >= 0");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  std::vector<Case*> cs;
  for (int i = 0; i < ncases; ++i) {
    QTT_CHECK_ARG(cases[i] && cases[i]->ctx == &c, "fractional_step_batch: every case must belong to ctx");
    Case* p = cases[i]->cs;
    QTT_CHECK_ARG(p->u && p->v && p->p, "fractional_step_batch: state not set");
    QTT_CHECK_ARG(p->use_graph, "fractional_step_batch: every case must replay its step graph");
    for (Case* q : cs) QTT_CHECK_ARG(q != p, "fractional_step_batch: a case appears twice");
    cs.push_back(p);
  }
  if (status)
    for (int i = 0; i < ncases; ++i) status[i] = QTT_OK;
  if (nsteps == 0) {
    set_last_error("");
    return QTT_OK;
  }
  const bool forces = with_forces && per_step;
  const int64_t nrec = int64_t(ncases) * nsteps * kStepRecDoubles;
  DBuf rec(&c, size_t(nrec));
  fill(c, rec.p, nrec, 0.0);
  run_steps_batch(c, cs, nsteps, forces, rec.p);
  std::vector<double> hrec(static_cast<size_t>(nrec));
  QTT_CUDA(cudaMemcpyAsync(hrec.data(), rec.p, hrec.size() * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  int rc = QTT_OK;
  std::string first;
  for (int i = 0; i < ncases; ++i) {
    std::string msg;
    const std::string who = "fractional_step_batch: case " + std::to_string(i);
    const int e = read_step_records(c, *cs[i], hrec.data() + int64_t(i) * nsteps * kStepRecDoubles, nsteps, forces,
                                    per_step ? per_step + int64_t(i) * nsteps : nullptr, who.c_str(), msg);
    if (status) status[i] = e;
    if (more_severe(rc, e) != rc) {
      rc = e;
      first = msg;
    }
  }
  if (rc != QTT_OK) {
    set_last_error(first);
    return rc;
  }
  API_END
}

// ---------------------------------------------------------------- learned warm start

int64_t qtt_nn_param_count(int c_in, int width, int depth) {
  if (c_in < 1 || width < 1 || depth < 1) return -1;
  return nn_param_count(c_in, width, depth);
}

int qtt_nn_create(qtt_ctx* ctx, int c_in, int width, int depth, const float* params, qtt_nn** out) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && params && out, "nn_create: null argument");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  std::unique_ptr<Net> net(new Net(c, c_in, width, depth, params));
  qtt_nn* h = new qtt_nn;
  h->ctx = &c;
  h->net = net.release();
  *out = h;
  API_END
}

int qtt_nn_free(qtt_nn* nn) {
  API_BEGIN
  if (nn) {
    delete nn->net;
    delete nn;
  }
  API_END
}

int qtt_nn_get_params(const qtt_nn* nn, float* dst) {
  API_BEGIN
  QTT_CHECK_ARG(nn && dst, "nn_get_params: null argument");
  Net& n = *nn->net;
  QTT_CUDA(cudaMemcpyAsync(dst, n.params, size_t(n.nparam) * sizeof(float), cudaMemcpyDeviceToHost, n.ctx->stream));
  QTT_CUDA(cudaStreamSynchronize(n.ctx->stream));
  API_END
}

int qtt_nn_get_grad(const qtt_nn* nn, float* dst) {
  API_BEGIN
  QTT_CHECK_ARG(nn && dst, "nn_get_grad: null argument");
  Net& n = *nn->net;
  QTT_CUDA(cudaMemcpyAsync(dst, n.grad, size_t(n.nparam) * sizeof(float), cudaMemcpyDeviceToHost, n.ctx->stream));
  QTT_CUDA(cudaStreamSynchronize(n.ctx->stream));
  API_END
}

int qtt_nn_set_scaling(qtt_nn* nn, const float* in_shift, const float* in_scale, float out_scale) {
  API_BEGIN
  QTT_CHECK_ARG(nn && in_shift && in_scale, "nn_set_scaling: null argument");
  nn->net->set_scaling(in_shift, in_scale, out_scale);
  API_END
}

static void check_nn_shape(const Net& n, int B, int H, int W) {
  QTT_CHECK_ARG(B >= 1 && H >= 1 && W >= 1 && int64_t(B) * std::max(n.c_in, n.width) * H * W <= (int64_t(1) << 30),
                "nn: B, H, W >= 1 and at most 2^30 activations per layer");
}

int qtt_nn_predict(qtt_nn* nn, int B, int H, int W, const float* x, int xkind, float* y, int ykind) {
  API_BEGIN
  QTT_CHECK_ARG(nn && x && y, "nn_predict: null argument");
  Net& n = *nn->net;
  check_nn_shape(n, B, H, W);
  Ctx& c = *n.ctx;
  const int64_t nx = int64_t(B) * n.c_in * H * W, ny = int64_t(B) * H * W;
  DBuf xb(&c, size_t((nx + 1) / 2)), yb(&c, size_t((ny + 1) / 2));
  float* xd = reinterpret_cast<float*>(xb.p);
  float* yd = reinterpret_cast<float*>(yb.p);
  QTT_CUDA(cudaMemcpyAsync(xd, x, size_t(nx) * sizeof(float), kind_in(xkind), c.stream));
  n.predict(B, H, W, xd, yd);
  QTT_CUDA(cudaMemcpyAsync(y, yd, size_t(ny) * sizeof(float), kind_out(ykind), c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

int qtt_nn_train_step(qtt_nn* nn, int B, int H, int W, const float* x, const float* y, int kind, float lr,
                      float* loss) {
  API_BEGIN
  QTT_CHECK_ARG(nn && x && y, "nn_train_step: null argument");
  QTT_CHECK_ARG(std::isfinite(lr) && lr > 0.f, "nn_train_step: lr must be positive");
  Net& n = *nn->net;
  check_nn_shape(n, B, H, W);
  Ctx& c = *n.ctx;
  const int64_t nx = int64_t(B) * n.c_in * H * W, ny = int64_t(B) * H * W;
  DBuf xb(&c, size_t((nx + 1) / 2)), yb(&c, size_t((ny + 1) / 2)), lb(&c, 1);
  float* xd = reinterpret_cast<float*>(xb.p);
  float* yd = reinterpret_cast<float*>(yb.p);
  QTT_CUDA(cudaMemcpyAsync(xd, x, size_t(nx) * sizeof(float), kind_in(kind), c.stream));
  QTT_CUDA(cudaMemcpyAsync(yd, y, size_t(ny) * sizeof(float), kind_in(kind), c.stream));
  const float l = n.train_step(B, H, W, xd, yd, lr, reinterpret_cast<float*>(lb.p));
  if (loss) *loss = l;
  if (!std::isfinite(l)) throw Error(QTT_ERR_NONFINITE, "nn_train_step: the loss is not finite");
  API_END
}

int qtt_grid_restrict(qtt_ctx* ctx, int Hc, int Wc, int levels, const double* fine, int fkind, float* coarse,
                      int ckind) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && fine && coarse, "grid_restrict: null argument");
  QTT_CHECK_ARG(Hc >= 1 && Wc >= 1 && levels >= 0 && levels <= 12 &&
                    (int64_t(Hc) * Wc << (2 * levels)) <= (int64_t(1) << 32),
                "grid_restrict: Hc, Wc >= 1, 0 <= levels <= 12, at most 2^32 fine values");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  const int64_t nf = int64_t(Hc) * Wc << (2 * levels), nc = int64_t(Hc) * Wc;
  DBuf fb(&c, size_t(nf)), cb(&c, size_t((nc + 1) / 2));
  QTT_CUDA(cudaMemcpyAsync(fb.p, fine, size_t(nf) * sizeof(double), kind_in(fkind), c.stream));
  grid_restrict(c, Hc, Wc, levels, fb.p, reinterpret_cast<float*>(cb.p));
  QTT_CUDA(cudaMemcpyAsync(coarse, cb.p, size_t(nc) * sizeof(float), kind_out(ckind), c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

int qtt_grid_prolong(qtt_ctx* ctx, int Hc, int Wc, int levels, const float* coarse, int ckind, double* fine,
                     int fkind) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && fine && coarse, "grid_prolong: null argument");
  QTT_CHECK_ARG(Hc >= 1 && Wc >= 1 && levels >= 0 && levels <= 12 &&
                    (int64_t(Hc) * Wc << (2 * levels)) <= (int64_t(1) << 32),
                "grid_prolong: Hc, Wc >= 1, 0 <= levels <= 12, at most 2^32 fine values");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  const int64_t nf = int64_t(Hc) * Wc << (2 * levels), nc = int64_t(Hc) * Wc;
  DBuf fb(&c, size_t(nf)), cb(&c, size_t((nc + 1) / 2));
  QTT_CUDA(cudaMemcpyAsync(cb.p, coarse, size_t(nc) * sizeof(float), kind_in(ckind), c.stream));
  grid_prolong(c, Hc, Wc, levels, reinterpret_cast<float*>(cb.p), fb.p);
  QTT_CUDA(cudaMemcpyAsync(fine, fb.p, size_t(nf) * sizeof(double), kind_out(fkind), c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  API_END
}

int qtt_field_moments(qtt_ctx* ctx, int64_t n, const float* x, int kind, double* mean, double* rms) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && x && mean && rms && n >= 1, "field_moments: null argument or n < 1");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  DBuf xb(&c, size_t((n + 1) / 2)), ob(&c, 2);
  QTT_CUDA(cudaMemcpyAsync(xb.p, x, size_t(n) * sizeof(float), kind_in(kind), c.stream));
  field_moments(c, n, reinterpret_cast<float*>(xb.p), ob.p);
  double h[2];
  QTT_CUDA(cudaMemcpyAsync(h, ob.p, sizeof(h), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  *mean = h[0];
  *rms = h[1];
  API_END
}

int qtt_case_phase_ms(qtt_case* h, double* ms4) {
  API_BEGIN
  QTT_CHECK_ARG(h && ms4, "case_phase_ms: null argument");
  Case& cs = *h->cs;
  QTT_CHECK_ARG(cs.ph_ev[4] != nullptr, "case_phase_ms: no step has run");
  QTT_CUDA(cudaEventSynchronize(cs.ph_ev[4]));
  for (int i = 0; i < 4; ++i) {
    float t = 0.f;
    QTT_CUDA(cudaEventElapsedTime(&t, cs.ph_ev[i], cs.ph_ev[i + 1]));
    ms4[i] = t;
  }
  API_END
}

int qtt_ctx_set_wait_limit(qtt_ctx* ctx, double seconds) {
  API_BEGIN
  QTT_CHECK_ARG(ctx, "ctx is null");
  QTT_CHECK_ARG(seconds > 0.0 && seconds <= 3600.0, "wait limit must be in (0, 3600] seconds");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  c.wait_ns = static_cast<unsigned long long>(std::max(1.0, seconds * 1e9));
  API_END
}

int qtt_ctx_set_cg_mode(qtt_ctx* ctx, int mode) {
  API_BEGIN
  QTT_CHECK_ARG(ctx, "ctx is null");
  QTT_CHECK_ARG(mode >= 0 && mode <= 3,
                "cg mode must be 0 (one kernel per solve, tensor-core contractions at full-bond sites), 1 (one kernel "
                "per stage), 2 (one FP64 kernel per solve) or 3 (one kernel per solve, tensor cores wherever it fits)");
  reinterpret_cast<Ctx*>(ctx)->cg_mode = mode;
  API_END
}

int qtt_case_use_graph(qtt_case* h, int enable) {
  API_BEGIN
  QTT_CHECK_ARG(h, "case_use_graph: null case");
  h->cs->drop_graph();
  h->cs->use_graph = enable != 0;
  API_END
}

int qtt_case_forces(qtt_ctx* ctx, qtt_case* h, double* cd, double* cl) {
  API_BEGIN
  QTT_CHECK_ARG(ctx && h && cd && cl, "case_forces: null argument");
  Case& cs = *h->cs;
  QTT_CHECK_ARG(cs.u && cs.v && cs.p, "case_forces: state not set");
  Ctx& c = *reinterpret_cast<Ctx*>(ctx);
  DBuf o(&c, 2);
  case_forces(c, cs, o.p);
  double hv[2];
  QTT_CUDA(cudaMemcpyAsync(hv, o.p, 2 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  *cd = hv[0];
  *cl = hv[1];
  API_END
}

int qtt_strouhal(const double* t, const double* cl, int n, double* st) {
  API_BEGIN
  QTT_CHECK_ARG(t && cl && st && n >= 2, "strouhal: need at least two samples");
  double mean = 0;
  for (int i = 0; i < n; ++i) mean += cl[i];
  mean /= n;
  std::vector<double> tc;
  for (int i = 0; i + 1 < n; ++i) {
    double a = cl[i] - mean, b = cl[i + 1] - mean;
    if (a < 0 && b >= 0) tc.push_back(t[i] - a * (t[i + 1] - t[i]) / (b - a));
  }
  if (tc.size() < 2) {
    *st = std::nan("");
  } else {
    double per = (tc.back() - tc.front()) / double(tc.size() - 1);
    *st = 1.0 / per;
  }
  API_END
}

}  // extern "C"
