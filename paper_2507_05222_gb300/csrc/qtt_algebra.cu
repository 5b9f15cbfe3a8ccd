// TT algebra of the QTT fractional-step method (arXiv:2507.05222, Sec. II) on the GPU:
// rounding, sums, MPO-MPS products, Hadamard products (variational fit, Table I), the
// single-site ALS solver (Sec. II.A.4), inner products, dense encode/decode (Fig. 1).
//
// Every operation is a host-side sequence of device kernels on the context stream; the host
// never waits on the device inside an operation except where a data-dependent bond must be
// known (rel_tol > 0 rounding, used at operator set-up).
#include <algorithm>
#include <cmath>
#include <memory>

#include "qtt_algebra.h"

namespace qtt {

// ------------------------------------------------------------------ handles

qtt_mps* new_mps(Ctx* c, int n, int d, const std::vector<int>& bonds) {
  QTT_CHECK_ARG(n >= 1 && d >= 1 && int(bonds.size()) == n + 1, "mps: bad shape");
  std::unique_ptr<qtt_mps> x(new qtt_mps);
  x->ctx = c;
  x->n = n;
  x->d = d;
  x->bonds = bonds;
  x->off.assign(n + 1, 0);
  int64_t tot = 0;
  for (int k = 0; k < n; ++k) {
    QTT_CHECK_ARG(bonds[k] >= 1 && bonds[k + 1] >= 1, "mps: bonds must be >= 1");
    x->off[k] = tot;
    int64_t sz = int64_t(bonds[k]) * d * bonds[k + 1];
    tot += (sz + 3) / 4 * 4;  // 32-byte aligned cores
  }
  x->off[n] = tot;
  x->buf.reset(c, size_t(tot));
  return x.release();
}

qtt_mpo* new_mpo(Ctx* c, int n, int d, const std::vector<int>& bonds) {
  QTT_CHECK_ARG(n >= 1 && d >= 1 && int(bonds.size()) == n + 1, "mpo: bad shape");
  std::unique_ptr<qtt_mpo> m(new qtt_mpo);
  m->ctx = c;
  m->n = n;
  m->d = d;
  m->bonds = bonds;
  m->off.assign(n + 1, 0);
  int64_t tot = 0;
  for (int k = 0; k < n; ++k) {
    m->off[k] = tot;
    int64_t sz = int64_t(bonds[k]) * d * d * bonds[k + 1];
    tot += (sz + 3) / 4 * 4;
  }
  m->off[n] = tot;
  m->buf.reset(c, size_t(tot));
  return m.release();
}

void free_mps(qtt_mps* x) { delete x; }
void free_mpo(qtt_mpo* m) { delete m; }

// ------------------------------------------------------------------ small kernels

namespace {

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return int(std::max<int64_t>(1, std::min<int64_t>(g, 65535 * 8)));
}

// Core k of alpha x (+) beta y (Sec. II.A.1): first core [ax | by], last [x ; y], middle
// block diagonal; alpha/beta are applied on the first core only.
__global__ void k_direct_sum(const double* __restrict__ X, int xr0, int xr1, const double* __restrict__ Y, int yr0,
                             int yr1, int d, int first, int last, double alpha, double beta, double* __restrict__ Z) {
  int zr0 = first ? 1 : xr0 + yr0;
  int zr1 = last ? 1 : xr1 + yr1;
  int64_t total = int64_t(zr0) * d * zr1;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    int a = int(e / (int64_t(d) * zr1));
    int s = int((e / zr1) % d);
    int b = int(e % zr1);
    double v = 0.0;
    if (first && last) {
      v = alpha * X[s] + beta * Y[s];
    } else if (first) {
      v = (b < xr1) ? alpha * X[s * xr1 + b] : beta * Y[s * yr1 + (b - xr1)];
    } else if (last) {
      v = (a < xr0) ? X[a * d + s] : Y[(a - xr0) * d + s];
    } else {
      if (a < xr0 && b < xr1) v = X[(int64_t(a) * d + s) * xr1 + b];
      else if (a >= xr0 && b >= xr1) v = Y[(int64_t(a - xr0) * d + s) * yr1 + (b - xr1)];
    }
    Z[e] = v;
  }
}

// diag(a) as an MPO core: W(a, s', s, b) = delta_{s s'} A(a, s, b) (copy tensor, Sec. II.A.3).
__global__ void k_diag_core(const double* __restrict__ A, int r0, int d, int r1, double* __restrict__ W) {
  int64_t total = int64_t(r0) * d * d * r1;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    int b = int(e % r1);
    int s = int((e / r1) % d);
    int so = int((e / (int64_t(r1) * d)) % d);
    int a = int(e / (int64_t(r1) * d * d));
    W[e] = (s == so) ? A[(int64_t(a) * d + s) * r1 + b] : 0.0;
  }
}

// *acc += the discarded weight of a Gram rounding cut: trace(rho) minus the kept eigenvalues
// w[0..bk) (sigma^2 each).  The kept eigenpairs are refined to FP64 and their sum is
// insensitive to how the discarded subspace is resolved, which the discarded eigenvalues
// themselves (FP32 Jacobi, not refined) are not.
__global__ void k_disc_add(const double* rho, const double* w, int nv, int bk, double* acc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double tr = 0.0, kept = 0.0;
  for (int i = 0; i < nv; ++i) tr += rho[int64_t(i) * nv + i];
  for (int i = 0; i < bk; ++i) kept += w[i];
  *acc += fmax(tr - kept, 0.0);
}

// *acc += the sum of the discarded eigenvalues w[bk..nv) of a cut whose eigenpairs were refined
// in factored form (each Rayleigh quotient then accurate on its own scale).
__global__ void k_disc_add_tail(const double* w, int nv, int bk, double* acc) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double s = 0.0;
  for (int i = bk; i < nv; ++i) s += fmax(w[i], 0.0);
  *acc += s;
}

// One core (l0, d, l1) of the sketch tensor train.  l0 == d l1 (the sketch as wide as the
// right space it sketches): the identity map, so that the sketch spans that space exactly.
// Else i.i.d. N(0, s^2) entries by the Box-Muller transform of two uniforms, each the top 53 bits
// of SplitMix64 (Steele, Lea and Flood 2014) at counter seed + 2i + 1 and seed + 2i + 2.
__device__ __forceinline__ uint64_t splitmix64(uint64_t x) {
  uint64_t z = x * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_sketch_core(int l0, int d, int l1, uint64_t seed, double s, double* __restrict__ out) {
  const int64_t n = int64_t(l0) * d * l1;
  const bool ident = int64_t(l0) == int64_t(d) * l1;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    if (ident) {
      const int64_t l = i / (int64_t(d) * l1), sm = i % (int64_t(d) * l1);
      out[i] = (l == sm) ? 1.0 : 0.0;
    } else {
      const double u1 = (double(splitmix64(seed + 2 * uint64_t(i) + 1) >> 11) + 1.0) * 0x1.0p-53;  // (0, 1]
      const double u2 = double(splitmix64(seed + 2 * uint64_t(i) + 2) >> 11) * 0x1.0p-53;          // [0, 1)
      out[i] = s * sqrt(-2.0 * log(u1)) * cospi(2.0 * u2);
    }
  }
}

__global__ void k_add_value(double* acc, double v) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *acc += v;
}

__global__ void k_sqrt(const double* in, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = sqrt(fmax(*in, 0.0));
}

}  // namespace

// Discarded weight of one rounding cut, added to the context's accumulator when a caller asked
// for it (qtt_round_info.discarded_norm).
static void add_discarded(Ctx& c, const double* rho_dev, const double* w_dev, int nv, int bk) {
  if (!c.disc_acc || bk >= nv) return;
  k_disc_add<<<1, 1, 0, c.stream>>>(rho_dev, w_dev, nv, bk, c.disc_acc);
  after_launch(c, "disc_add");
}

void sqrt_dev(Ctx& c, const double* in, double* out) {
  k_sqrt<<<1, 1, 0, c.stream>>>(in, out);
  after_launch(c, "sqrt");
}

void direct_sum_core(Ctx& c, const double* X, int xr0, int xr1, const double* Y, int yr0, int yr1, int d, bool first,
                     bool last, double alpha, double beta, double* Z, int64_t zsize) {
  k_direct_sum<<<grid_for(zsize, 256), 256, 0, c.stream>>>(X, xr0, xr1, Y, yr0, yr1, d, first ? 1 : 0, last ? 1 : 0,
                                                           alpha, beta, Z);
  after_launch(c, "direct_sum");
}

qtt_mps* direct_sum(Ctx& c, double alpha, const qtt_mps* x, double beta, const qtt_mps* y) {
  QTT_CHECK_ARG(x->n == y->n && x->d == y->d, "direct sum: shape mismatch");
  const int n = x->n, d = x->d;
  std::vector<int> b(n + 1);
  b[0] = 1;
  b[n] = 1;
  for (int k = 1; k < n; ++k) b[k] = x->bonds[k] + y->bonds[k];
  qtt_mps* z = new_mps(&c, n, d, b);
  for (int k = 0; k < n; ++k)
    direct_sum_core(c, x->core(k), x->bonds[k], x->bonds[k + 1], y->core(k), y->bonds[k], y->bonds[k + 1], d, k == 0,
                    k == n - 1, alpha, beta, z->core(k), int64_t(b[k]) * d * b[k + 1]);
  return z;
}

qtt_mpo* diag_mpo(Ctx& c, const qtt_mps* a) {
  qtt_mpo* m = new_mpo(&c, a->n, a->d, a->bonds);
  for (int k = 0; k < a->n; ++k) {
    int64_t tot = int64_t(a->bonds[k]) * a->d * a->d * a->bonds[k + 1];
    k_diag_core<<<grid_for(tot, 256), 256, 0, c.stream>>>(a->core(k), a->bonds[k], a->d, a->bonds[k + 1], m->core(k));
    after_launch(c, "diag_core");
  }
  return m;
}

// y = M x without rounding: B[k]((a w), s', (b v)) = sum_s M[k](w, s', s, v) A[k](a, s, b)
// (Sec. II.A.2; fused bond index (x-bond slow, MPO-bond fast)).
void mpo_mps_exact_into(Ctx& c, const qtt_mpo* M, const qtt_mps* x, qtt_mps* y) {
  QTT_CHECK_ARG(M->n == x->n && M->d == x->d && y->n == x->n && y->d == x->d, "mpo-mps: shape mismatch");
  const int n = x->n, d = x->d;
  for (int k = 0; k <= n; ++k) QTT_CHECK_ARG(y->bonds[k] == x->bonds[k] * M->bonds[k], "mpo-mps: output bonds");
  for (int k = 0; k < n; ++k) {
    int a0 = x->bonds[k], a1 = x->bonds[k + 1], w0 = M->bonds[k], w1 = M->bonds[k + 1];
    einsum(c, "wtsv,asb->awtbv", 1.0, tv(M->core(k), {w0, d, d, w1}), tv(x->core(k), {a0, d, a1}), 0.0,
           tv(y->core(k), {a0, w0, d, a1, w1}));
  }
}

qtt_mps* mpo_mps_exact(Ctx& c, const qtt_mpo* M, const qtt_mps* x) {
  QTT_CHECK_ARG(M->n == x->n && M->d == x->d, "mpo-mps: shape mismatch");
  const int n = x->n, d = x->d;
  std::vector<int> b(n + 1);
  for (int k = 0; k <= n; ++k) b[k] = x->bonds[k] * M->bonds[k];
  std::unique_ptr<qtt_mps, void (*)(qtt_mps*)> y(new_mps(&c, n, d, b), free_mps);
  mpo_mps_exact_into(c, M, x, y.get());
  return y.release();
}

qtt_mpo* mpo_mpo_exact(Ctx& c, const qtt_mpo* A, const qtt_mpo* B) {
  QTT_CHECK_ARG(A->n == B->n && A->d == B->d, "mpo-mpo: shape mismatch");
  const int n = A->n, d = A->d;
  std::vector<int> b(n + 1);
  for (int k = 0; k <= n; ++k) b[k] = A->bonds[k] * B->bonds[k];
  qtt_mpo* m = new_mpo(&c, n, d, b);
  for (int k = 0; k < n; ++k) {
    int a0 = A->bonds[k], a1 = A->bonds[k + 1], b0 = B->bonds[k], b1 = B->bonds[k + 1];
    einsum(c, "asrb,crtd->acstbd", 1.0, tv(A->core(k), {a0, d, d, a1}), tv(B->core(k), {b0, d, d, b1}), 0.0,
           tv(m->core(k), {a0, b0, d, d, a1, b1}));
  }
  return m;
}

qtt_mps* mps_copy(Ctx& c, const qtt_mps* x) {
  qtt_mps* y = new_mps(&c, x->n, x->d, x->bonds);
  copy(c, y->buf.p, x->buf.p, x->off[x->n]);
  return y;
}

void mps_scale(Ctx& c, qtt_mps* x, double s) { axpby(c, x->core_size(0), 0.0, x->core(0), s, x->core(0)); }

// View an MPO as an MPS with physical dimension d^2 (no copy of values; a new handle).
qtt_mps* mpo_as_mps(Ctx& c, const qtt_mpo* m) {
  qtt_mps* x = new_mps(&c, m->n, m->d * m->d, m->bonds);
  copy(c, x->buf.p, m->buf.p, m->off[m->n]);
  return x;
}

qtt_mpo* mps_as_mpo(Ctx& c, const qtt_mps* x, int d) {
  QTT_CHECK_ARG(x->d == d * d, "mps_as_mpo: physical size");
  qtt_mpo* m = new_mpo(&c, x->n, d, x->bonds);
  copy(c, m->buf.p, x->buf.p, x->off[x->n]);
  return m;
}

// ------------------------------------------------------------------ structural ranks

std::vector<int> left_struct(const std::vector<int>& pre, int d) {
  std::vector<int> m(pre.size());
  m[0] = 1;
  for (size_t k = 1; k < pre.size(); ++k) {
    int64_t v = std::min<int64_t>(pre[k], int64_t(d) * m[k - 1]);
    m[k] = int(v);
  }
  return m;
}

static int kept(const std::vector<double>& sig, int chi, double eps, int strct) {
  int b = std::min<int>(chi, strct);
  b = std::min<int>(b, int(sig.size()));
  if (eps > 0.0 && !sig.empty()) {
    int cnt = 0;
    for (double s : sig)
      if (s > eps * sig[0]) ++cnt;
    b = std::min(b, cnt);
  }
  return std::max(b, 1);
}

// ------------------------------------------------------------------ accurate rounding (QR + SVD)
// TT-rounding (Sec. II.A): left-to-right Householder QR, right-to-left truncated SVD
// (one-sided Jacobi, FP64).  Reads singular values on the host at every cut.

qtt_mps* round_svd(Ctx& c, const qtt_mps* x_in, int chi, double eps) {
  const int n = x_in->n, d = x_in->d;
  std::vector<int> pre = x_in->bonds;
  std::vector<int> m = left_struct(pre, d);
  // working copy of the cores with the current bonds
  std::vector<DBuf> core(n);
  std::vector<int> b = pre;
  for (int k = 0; k < n; ++k) {
    core[k].reset(&c, size_t(x_in->core_size(k)) + 4);
    copy(c, core[k].p, x_in->core(k), int64_t(b[k]) * d * b[k + 1]);
  }
  // left-to-right orthogonalisation
  for (int k = 0; k + 1 < n; ++k) {
    int rows = b[k] * d, cols = b[k + 1];
    int kk = std::min(rows, cols);
    DBuf Q(&c, size_t(rows) * kk), R(&c, size_t(kk) * cols);
    qr(c, 1, rows, cols, 0, core[k].p, 0, Q.p, 0, R.p, 0);
    core[k] = std::move(Q);
    DBuf nxt(&c, size_t(kk) * d * b[k + 2]);
    einsum(c, "ab,bsc->asc", 1.0, tv(R.p, {kk, cols}), tv(core[k + 1].p, {cols, d, b[k + 2]}), 0.0,
           tv(nxt.p, {kk, d, b[k + 2]}));
    core[k + 1] = std::move(nxt);
    b[k + 1] = kk;
  }
  // right-to-left truncation
  std::vector<int> out_b(n + 1);
  out_b[0] = 1;
  out_b[n] = 1;
  for (int k = n - 1; k >= 1; --k) {
    int r0 = b[k], r1 = out_b[k + 1];
    int cols = d * r1;
    // Y = core (r0 x cols).  SVD of the taller orientation.
    int mm = std::max(r0, cols), nn = std::min(r0, cols);
    DBuf U(&c, size_t(mm) * nn), S(&c, size_t(nn)), V(&c, size_t(nn) * nn), T(&c, size_t(r0) * cols);
    bool tall = r0 >= cols;
    if (tall) {
      svd_small(c, r0, cols, core[k].p, U.p, S.p, V.p);  // Y = U S V^T, right vectors = V columns
    } else {
      int64_t dims[2] = {r0, cols};
      int perm[2] = {1, 0};
      permute(c, core[k].p, 2, dims, perm, T.p, 1.0, 0.0);  // Y^T (cols x r0)
      svd_small(c, cols, r0, T.p, U.p, S.p, V.p);           // Y^T = U S V^T: right vectors of Y = U columns
    }
    std::vector<double> sig(nn);
    QTT_CUDA(cudaMemcpyAsync(sig.data(), S.p, nn * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    QTT_CUDA(cudaStreamSynchronize(c.stream));
    int nz = 0;
    for (double s : sig)
      if (s > 0.0) ++nz;
    int bk = kept(sig, chi, eps, std::min(m[k], cols));
    bk = std::max(1, std::min(bk, std::max(nz, 1)));
    if (c.disc_acc) {
      double disc = 0.0;
      for (int i = bk; i < nn; ++i) disc += sig[i] * sig[i];
      k_add_value<<<1, 1, 0, c.stream>>>(c.disc_acc, disc);
      after_launch(c, "add_value");
    }
    DBuf newcore(&c, size_t(bk) * cols), carry(&c, size_t(r0) * bk);
    // right singular vectors (cols x bk) -> new core = their transpose (bk x cols);
    // carry = left vectors * S (r0 x bk)
    const double* Rv = tall ? V.p : U.p;        // (cols x nn) row-major, first bk columns
    const double* Lv = tall ? U.p : V.p;        // (r0 x nn)
    QTT_CUDA(cudaMemcpy2DAsync(T.p, bk * sizeof(double), Rv, nn * sizeof(double), bk * sizeof(double), cols,
                               cudaMemcpyDeviceToDevice, c.stream));
    {
      int64_t dims[2] = {cols, bk};
      int perm[2] = {1, 0};
      permute(c, T.p, 2, dims, perm, newcore.p, 1.0, 0.0);
    }
    QTT_CUDA(cudaMemcpy2DAsync(carry.p, bk * sizeof(double), Lv, nn * sizeof(double), bk * sizeof(double), r0,
                               cudaMemcpyDeviceToDevice, c.stream));
    // scale columns by S: carry (r0 x bk) = carry * diag(S[:bk]) via einsum with a diag
    {
      DBuf Dg(&c, size_t(bk) * bk);
      fill(c, Dg.p, int64_t(bk) * bk, 0.0);
      QTT_CUDA(cudaMemcpy2DAsync(Dg.p, (bk + 1) * sizeof(double), S.p, sizeof(double), sizeof(double), bk,
                                 cudaMemcpyDeviceToDevice, c.stream));
      DBuf cs(&c, size_t(r0) * bk);
      einsum(c, "ab,bc->ac", 1.0, tv(carry.p, {r0, bk}), tv(Dg.p, {bk, bk}), 0.0, tv(cs.p, {r0, bk}));
      DBuf prev(&c, size_t(b[k - 1]) * d * bk);
      einsum(c, "asb,bc->asc", 1.0, tv(core[k - 1].p, {b[k - 1], d, r0}), tv(cs.p, {r0, bk}), 0.0,
             tv(prev.p, {b[k - 1], d, bk}));
      core[k - 1] = std::move(prev);
    }
    core[k] = std::move(newcore);
    out_b[k] = bk;
  }
  qtt_mps* y = new_mps(&c, n, d, out_b);
  for (int k = 0; k < n; ++k) copy(c, y->core(k), core[k].p, int64_t(out_b[k]) * d * out_b[k + 1]);
  return y;
}

// ------------------------------------------------------------------ Gram rounding
// Right-to-left TT-SVD of an explicit TT through left Gram matrices G_k = Y_{<k}^T Y_{<k}
// (density-matrix form): at core k, Z = Y[k] P_{k+1}, rho = Z^T G_k Z (d b x d b), the top
// b_k eigenvectors of rho are the new core (right singular vectors of the unfolding), and
// P_k = Z V.  Only (d chi)-sized eigenproblems appear, never the (pre-round) bond.

static std::vector<double> host_copy(Ctx& c, const double* p, int n) {
  std::vector<double> h(n);
  QTT_CUDA(cudaMemcpyAsync(h.data(), p, n * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  return h;
}

static int choose_rank(Ctx& c, const double* w_dev, int nw, int chi, double eps, int strct) {
  int b = std::min(std::min(chi, strct), nw);
  if (eps > 0.0) {
    std::vector<double> w = host_copy(c, w_dev, nw);
    std::vector<double> sig(nw);
    for (int i = 0; i < nw; ++i) sig[i] = std::sqrt(std::max(w[i], 0.0));
    b = kept(sig, chi, eps, strct);
  }
  return std::max(b, 1);
}

// Take the first b columns of V (nv x nv, row-major) as the rows of a (b x nv) core.
static void top_vectors_as_core(Ctx& c, const double* V, int nv, int b, double* core_out) {
  DBuf T(&c, size_t(nv) * b);
  QTT_CUDA(cudaMemcpy2DAsync(T.p, b * sizeof(double), V, nv * sizeof(double), b * sizeof(double), nv,
                             cudaMemcpyDeviceToDevice, c.stream));
  int64_t dims[2] = {nv, b};
  int perm[2] = {1, 0};
  permute(c, T.p, 2, dims, perm, core_out, 1.0, 0.0);
}

qtt_mps* round_gram(Ctx& c, const qtt_mps* y, int chi, double eps) {
  const int n = y->n, d = y->d;
  const std::vector<int>& R = y->bonds;
  std::vector<int> m = left_struct(R, d);
  if (n == 1) return mps_copy(c, y);
  // left Grams G_k (R_k x R_k), k = 0..n-1
  std::vector<DBuf> G(n);
  G[0].reset(&c, 1);
  fill(c, G[0].p, 1, 1.0);
  for (int k = 0; k + 1 < n; ++k) {
    int a0 = R[k], a1 = R[k + 1];
    DBuf T(&c, size_t(a0) * d * a1);
    einsum(c, "aA,asb->Asb", 1.0, tv(G[k].p, {a0, a0}), tv(y->core(k), {a0, d, a1}), 0.0, tv(T.p, {a0, d, a1}));
    G[k + 1].reset(&c, size_t(a1) * a1);
    einsum(c, "Asb,AsB->bB", 1.0, tv(T.p, {a0, d, a1}), tv(y->core(k), {a0, d, a1}), 0.0, tv(G[k + 1].p, {a1, a1}));
  }
  std::vector<int> ob(n + 1);
  ob[0] = 1;
  ob[n] = 1;
  std::vector<DBuf> out(n);
  DBuf P(&c, 1);
  fill(c, P.p, 1, 1.0);
  for (int k = n - 1; k >= 0; --k) {
    int a0 = R[k], a1 = R[k + 1], c1 = ob[k + 1];
    DBuf Z(&c, size_t(a0) * d * c1);
    einsum(c, "asb,bc->asc", 1.0, tv(y->core(k), {a0, d, a1}), tv(P.p, {a1, c1}), 0.0, tv(Z.p, {a0, d, c1}));
    if (k == 0) {
      out[0] = std::move(Z);
      break;
    }
    const int nv = d * c1;
    DBuf T(&c, size_t(a0) * nv), rho(&c, size_t(nv) * nv), w(&c, size_t(nv)), V(&c, size_t(nv) * nv);
    einsum(c, "aA,asc->Asc", 1.0, tv(G[k].p, {a0, a0}), tv(Z.p, {a0, d, c1}), 0.0, tv(T.p, {a0, d, c1}));
    einsum(c, "Asc,AtD->sctD", 1.0, tv(T.p, {a0, d, c1}), tv(Z.p, {a0, d, c1}), 0.0, tv(rho.p, {d, c1, d, c1}));
    eigh(c, nv, rho.p, w.p, V.p, std::min(std::min(chi, m[k]), nv));
    int bk = choose_rank(c, w.p, nv, chi, eps, std::min(m[k], nv));
    add_discarded(c, rho.p, w.p, nv, bk);
    out[k].reset(&c, size_t(bk) * nv);
    top_vectors_as_core(c, V.p, nv, bk, out[k].p);
    // P_k = Z V[:, :bk]  (a0 x bk)
    DBuf Pn(&c, size_t(a0) * bk);
    gemm(c, 1, a0, bk, nv, 1.0, Z.p, 0, nv, 1, V.p, 0, nv, 1, 0.0, Pn.p, 0, bk, 1);
    P = std::move(Pn);
    ob[k] = bk;
  }
  qtt_mps* z = new_mps(&c, n, d, ob);
  for (int k = 0; k < n; ++k) copy(c, z->core(k), out[k].p, int64_t(ob[k]) * d * ob[k + 1]);
  return z;
}

// Gram rounding of y = M x without forming y: the left Gram of y at bond k is kept in the
// factored index (w, a, w', a'), and Z = (M x)[k] P is contracted from M[k], X[k] directly.
std::vector<int> apply_bonds(const qtt_mpo* M, const qtt_mps* x, int chi) {
  const int n = x->n, d = x->d;
  std::vector<int> R(n + 1);
  for (int k = 0; k <= n; ++k) R[k] = M->bonds[k] * x->bonds[k];
  std::vector<int> m = left_struct(R, d);
  std::vector<int> ob(n + 1, 1);
  for (int k = n - 1; k >= 1; --k) ob[k] = std::max(1, std::min(std::min(chi, m[k]), d * ob[k + 1]));
  if (n == 1) ob = R;
  return ob;
}

qtt_mps* apply_round_gram(Ctx& c, const qtt_mpo* M, const qtt_mps* x, int chi, double eps, qtt_mps* into) {
  const int n = x->n, d = x->d;
  QTT_CHECK_ARG(M->n == n && M->d == d, "apply: shape mismatch");
  std::vector<int> R(n + 1);
  for (int k = 0; k <= n; ++k) R[k] = M->bonds[k] * x->bonds[k];
  std::vector<int> mstruct = left_struct(R, d);
  if (n == 1) {
    QTT_CHECK_ARG(!into, "apply into: single-core operands are not supported");
    qtt_mps* y = mpo_mps_exact(c, M, x);
    return y;
  }
  std::vector<DBuf> G(n);
  G[0].reset(&c, 1);
  fill(c, G[0].p, 1, 1.0);
  for (int k = 0; k + 1 < n; ++k) {
    int w0 = M->bonds[k], w1 = M->bonds[k + 1], a0 = x->bonds[k], a1 = x->bonds[k + 1];
    TV g = tv(G[k].p, {w0, a0, w0, a0});
    TV X = tv(x->core(k), {a0, d, a1});
    TV W = tv(M->core(k), {w0, d, d, w1});
    DBuf T1(&c, size_t(w0) * w0 * a0 * d * a1);
    einsum(c, "waWA,atb->wWAtb", 1.0, g, X, 0.0, tv(T1.p, {w0, w0, a0, d, a1}));
    DBuf T2(&c, size_t(w0) * a0 * a1 * d * w1);
    einsum(c, "wWAtb,wstv->WAbsv", 1.0, tv(T1.p, {w0, w0, a0, d, a1}), W, 0.0, tv(T2.p, {w0, a0, a1, d, w1}));
    DBuf T3(&c, size_t(a0) * a1 * w1 * d * w1);
    einsum(c, "WAbsv,WsTV->AbvTV", 1.0, tv(T2.p, {w0, a0, a1, d, w1}), W, 0.0, tv(T3.p, {a0, a1, w1, d, w1}));
    G[k + 1].reset(&c, size_t(w1) * a1 * w1 * a1);
    einsum(c, "AbvTV,ATB->vbVB", 1.0, tv(T3.p, {a0, a1, w1, d, w1}), X, 0.0, tv(G[k + 1].p, {w1, a1, w1, a1}));
  }
  std::vector<int> ob(n + 1);
  ob[0] = 1;
  ob[n] = 1;
  std::vector<DBuf> out(n);
  DBuf P(&c, 1);  // (w_{k+1}, a_{k+1}, c_{k+1})
  fill(c, P.p, 1, 1.0);
  for (int k = n - 1; k >= 0; --k) {
    int w0 = M->bonds[k], w1 = M->bonds[k + 1], a0 = x->bonds[k], a1 = x->bonds[k + 1], c1 = ob[k + 1];
    TV X = tv(x->core(k), {a0, d, a1});
    TV W = tv(M->core(k), {w0, d, d, w1});
    DBuf T1(&c, size_t(a0) * d * w1 * c1);
    einsum(c, "atb,vbc->atvc", 1.0, X, tv(P.p, {w1, a1, c1}), 0.0, tv(T1.p, {a0, d, w1, c1}));
    DBuf Z(&c, size_t(w0) * a0 * d * c1);
    einsum(c, "wstv,atvc->wasc", 1.0, W, tv(T1.p, {a0, d, w1, c1}), 0.0, tv(Z.p, {w0, a0, d, c1}));
    if (k == 0) {
      out[0] = std::move(Z);  // w0 = a0 = 1: (1, d, c1)
      break;
    }
    const int nv = d * c1;
    DBuf T2(&c, size_t(w0) * a0 * nv), rho(&c, size_t(nv) * nv), wv(&c, size_t(nv)), V(&c, size_t(nv) * nv);
    einsum(c, "waWA,wasc->WAsc", 1.0, tv(G[k].p, {w0, a0, w0, a0}), tv(Z.p, {w0, a0, d, c1}), 0.0,
           tv(T2.p, {w0, a0, d, c1}));
    einsum(c, "WAsc,WASC->scSC", 1.0, tv(T2.p, {w0, a0, d, c1}), tv(Z.p, {w0, a0, d, c1}), 0.0,
           tv(rho.p, {d, c1, d, c1}));
    eigh(c, nv, rho.p, wv.p, V.p, std::min(std::min(chi, mstruct[k]), nv));
    int bk = choose_rank(c, wv.p, nv, chi, eps, std::min(mstruct[k], nv));
    add_discarded(c, rho.p, wv.p, nv, bk);
    out[k].reset(&c, size_t(bk) * nv);
    top_vectors_as_core(c, V.p, nv, bk, out[k].p);
    DBuf Pn(&c, size_t(w0) * a0 * bk);
    gemm(c, 1, int64_t(w0) * a0, bk, nv, 1.0, Z.p, 0, nv, 1, V.p, 0, nv, 1, 0.0, Pn.p, 0, bk, 1);
    P = std::move(Pn);
    ob[k] = bk;
  }
  qtt_mps* z = into;
  if (z) QTT_CHECK_ARG(z->n == n && z->d == d && z->bonds == ob, "apply into: output bonds differ");
  else z = new_mps(&c, n, d, ob);
  for (int k = 0; k < n; ++k) copy(c, z->core(k), out[k].p, int64_t(ob[k]) * d * ob[k + 1]);
  return z;
}

// ------------------------------------------------------------------ sketched rounding of M x
// TT-SVD of y = M x (Sec. II.A.2 then the rounding of Sec. II.A) without squaring singular
// values.  The Gram rounding above resolves nothing below ~sqrt(eps) sigma_1 at a cut; on
// smooth fields the chi-th singular value of the middle cuts sits at 1e-9..1e-11 sigma_1, so
// its result there differs from the TT-SVD by ~1e-8.  Here:
//  1. a tensor train Omega (bonds sb_k = min(ell, d sb_{k+1})) sketches the right part of y at
//     every cut: W_k = y_{>=k} . Omega_{>=k}, (w_k a_k) x sb_k, contracted core by core; its
//     cores are identity maps while the sketch is as wide as the right space (which it then
//     spans exactly) and Gaussian where it compresses;
//  2. left to right, the next left unfolding T_k = F_{k-1} y[k] ((rho d) x (w a)) is kept as
//     it is while rho d <= sb_{k+1}, else replaced by its coefficients F_k = Q^T T_k in the
//     orthonormal basis Q of the sketched range T_k W_{k+1} (Householder QR): y's left part is
//     then Q_{<=k} F_k with Q_{<=k} orthonormal, up to the sketch's range error, which falls
//     with the (rank ell) tail of the cut's spectrum (<~1e-13 for the fields of the step);
//  3. right to left as in the Gram rounding, but each cut's matrix A_k = F_{k-1} Z_k
//     (rho x d c) is explicit, and its eigenpairs are refined in factored form
//     ((F X)^T (F X) instead of X^T S X), which resolves the tail to its own scale.
// The result does not depend on Omega beyond the sketch's range error, which is zero when ell
// reaches the product's largest bond (sketch_width).  Cost: the sketches and one QR of
// (rho d) x ell per middle site in place of the left Gram recurrence.

// Sketch width: the largest product bond max_k w_k a_k when the QR of a (d ell) x ell sketch
// supports it (every sketch then spans its cut's range exactly, for any input), else 2 chi + 32
// (the range error then falls with the cut spectra beyond that width), at most what the QR
// supports.
static int sketch_width(int chi, int d, const std::vector<int>& R) {
  int rmax = *std::max_element(R.begin(), R.end());
  int want = rmax;
  if (!qr_fits(d * want, want)) want = 2 * chi + 32;
  while (want > 16 && !qr_fits(d * want, want)) want -= 8;
  return std::max(want, 1);
}

qtt_mps* apply_round_sketch(Ctx& c, const qtt_mpo* M, const qtt_mps* x, int chi, double eps, qtt_mps* into) {
  const int n = x->n, d = x->d;
  QTT_CHECK_ARG(M->n == n && M->d == d, "apply: shape mismatch");
  if (n == 1) return apply_round_gram(c, M, x, chi, eps, into);
  if (int64_t(d) * chi > 256)
    throw Error(QTT_ERR_UNSUPPORTED, "apply (sketched rounding): d * chi must be <= 256 (eigensolver limit)");
  std::vector<int> R(n + 1);
  for (int k = 0; k <= n; ++k) R[k] = M->bonds[k] * x->bonds[k];
  std::vector<int> mstruct = left_struct(R, d);
  const int ell = sketch_width(chi, d, R);
  std::vector<int> sb(n + 1, 1);
  for (int k = n - 1; k >= 1; --k) sb[k] = int(std::min<int64_t>(ell, int64_t(d) * sb[k + 1]));
  // 1. right sketches W[k] (w_k, a_k, sb_k), k = n .. 1
  std::vector<DBuf> W(n + 1);
  W[n].reset(&c, 1);
  fill(c, W[n].p, 1, 1.0);
  for (int k = n - 1; k >= 1; --k) {
    int w0 = M->bonds[k], w1 = M->bonds[k + 1], a0 = x->bonds[k], a1 = x->bonds[k + 1], l0 = sb[k], l1 = sb[k + 1];
    DBuf Om(&c, size_t(l0) * d * l1);
    int64_t cnt = int64_t(l0) * d * l1;
    k_sketch_core<<<unsigned(std::min<int64_t>((cnt + 255) / 256, 1024)), 256, 0, c.stream>>>(
        l0, d, l1, 0x5EEDC0DEull * uint64_t(k + 1) << 20, 1.0 / std::sqrt(double(d) * l1), Om.p);
    after_launch(c, "sketch_core");
    DBuf T1(&c, size_t(a0) * d * w1 * l1), T2(&c, size_t(w0) * a0 * d * l1);
    einsum(c, "atb,vbl->atvl", 1.0, tv(x->core(k), {a0, d, a1}), tv(W[k + 1].p, {w1, a1, l1}), 0.0,
           tv(T1.p, {a0, d, w1, l1}));
    einsum(c, "wstv,atvl->wasl", 1.0, tv(M->core(k), {w0, d, d, w1}), tv(T1.p, {a0, d, w1, l1}), 0.0,
           tv(T2.p, {w0, a0, d, l1}));
    W[k].reset(&c, size_t(w0) * a0 * l0);
    einsum(c, "wasl,msl->wam", 1.0, tv(T2.p, {w0, a0, d, l1}), tv(Om.p, {l0, d, l1}), 0.0, tv(W[k].p, {w0, a0, l0}));
  }
  // 2. left-to-right coefficients F[k] (rho_k x w_{k+1} a_{k+1}), k = 0 .. n-2
  std::vector<DBuf> F(n);
  std::vector<int> rho(n, 1);
  {
    DBuf F0(&c, 1);
    fill(c, F0.p, 1, 1.0);
    const double* Fp = F0.p;
    int r = 1;
    for (int k = 0; k + 1 < n; ++k) {
      int w0 = M->bonds[k], w1 = M->bonds[k + 1], a0 = x->bonds[k], a1 = x->bonds[k + 1];
      DBuf T1(&c, size_t(r) * w0 * d * a1), T(&c, size_t(r) * d * w1 * a1);
      einsum(c, "rwa,atb->rwtb", 1.0, tv(const_cast<double*>(Fp), {r, w0, a0}), tv(x->core(k), {a0, d, a1}), 0.0,
             tv(T1.p, {r, w0, d, a1}));
      einsum(c, "rwtb,wstv->rsvb", 1.0, tv(T1.p, {r, w0, d, a1}), tv(M->core(k), {w0, d, d, w1}), 0.0,
             tv(T.p, {r, d, w1, a1}));
      const int rows = r * d, cols = w1 * a1, l = sb[k + 1];
      if (rows <= l) {
        F[k] = std::move(T);
        rho[k] = rows;
      } else {
        DBuf Y(&c, size_t(rows) * l), Q(&c, size_t(rows) * l);
        gemm(c, 1, rows, l, cols, 1.0, T.p, 0, cols, 1, W[k + 1].p, 0, l, 1, 0.0, Y.p, 0, l, 1);
        qr(c, 1, rows, l, 0, Y.p, 0, Q.p, 0, nullptr, 0);
        F[k].reset(&c, size_t(l) * cols);
        gemm(c, 1, l, cols, rows, 1.0, Q.p, 0, 1, l, T.p, 0, cols, 1, 0.0, F[k].p, 0, cols, 1);
        rho[k] = l;
      }
      Fp = F[k].p;
      r = rho[k];
      W[k + 1] = DBuf();   // no longer needed
    }
  }
  // 3. right-to-left truncation on the explicit cut matrices
  std::vector<int> ob(n + 1);
  ob[0] = 1;
  ob[n] = 1;
  std::vector<DBuf> out(n);
  DBuf P(&c, 1);  // (w_{k+1}, a_{k+1}, c_{k+1})
  fill(c, P.p, 1, 1.0);
  for (int k = n - 1; k >= 0; --k) {
    int w0 = M->bonds[k], w1 = M->bonds[k + 1], a0 = x->bonds[k], a1 = x->bonds[k + 1], c1 = ob[k + 1];
    TV X = tv(x->core(k), {a0, d, a1});
    TV Wm = tv(M->core(k), {w0, d, d, w1});
    DBuf T1(&c, size_t(a0) * d * w1 * c1);
    einsum(c, "atb,vbc->atvc", 1.0, X, tv(P.p, {w1, a1, c1}), 0.0, tv(T1.p, {a0, d, w1, c1}));
    DBuf Z(&c, size_t(w0) * a0 * d * c1);
    einsum(c, "wstv,atvc->wasc", 1.0, Wm, tv(T1.p, {a0, d, w1, c1}), 0.0, tv(Z.p, {w0, a0, d, c1}));
    if (k == 0) {
      out[0] = std::move(Z);
      break;
    }
    const int nv = d * c1, r = rho[k - 1], wa = w0 * a0;
    DBuf A(&c, size_t(r) * nv), S(&c, size_t(nv) * nv), wv(&c, size_t(nv)), V(&c, size_t(nv) * nv);
    gemm(c, 1, r, nv, wa, 1.0, F[k - 1].p, 0, wa, 1, Z.p, 0, nv, 1, 0.0, A.p, 0, nv, 1);
    F[k - 1] = DBuf();
    gemm(c, 1, nv, nv, r, 1.0, A.p, 0, 1, nv, A.p, 0, nv, 1, 0.0, S.p, 0, nv, 1);
    const int keep = std::min(std::min(chi, mstruct[k]), nv);
    eigh(c, nv, S.p, wv.p, V.p, keep, A.p, r);
    int bk = choose_rank(c, wv.p, nv, chi, eps, std::min(mstruct[k], nv));
    if (c.disc_acc && bk < nv) {
      k_disc_add_tail<<<1, 1, 0, c.stream>>>(wv.p, nv, bk, c.disc_acc);
      after_launch(c, "disc_add_tail");
    }
    out[k].reset(&c, size_t(bk) * nv);
    top_vectors_as_core(c, V.p, nv, bk, out[k].p);
    DBuf Pn(&c, size_t(wa) * bk);
    gemm(c, 1, wa, bk, nv, 1.0, Z.p, 0, nv, 1, V.p, 0, nv, 1, 0.0, Pn.p, 0, bk, 1);
    P = std::move(Pn);
    ob[k] = bk;
  }
  qtt_mps* z = into;
  if (z) QTT_CHECK_ARG(z->n == n && z->d == d && z->bonds == ob, "apply into: output bonds differ");
  else z = new_mps(&c, n, d, ob);
  for (int k = 0; k < n; ++k) copy(c, z->core(k), out[k].p, int64_t(ob[k]) * d * ob[k + 1]);
  return z;
}

// The accurate path keeps every core unfolding in one CTA's shared memory.
static bool svd_path_fits(const std::vector<int>& b, int d) {
  for (size_t k = 0; k + 1 < b.size(); ++k) {
    int64_t r0 = b[k], c = int64_t(d) * b[k + 1];
    int64_t mm = std::max(r0, c), nn = std::min(r0, c);
    if (mm * nn + nn * nn + 2 * nn > 26000) return false;
    if (int64_t(b[k]) * d * b[k + 1] + int64_t(b[k]) * d + b[k + 1] > 26000) return false;
  }
  return true;
}

// Rounding dispatcher.  rel_tol = 0: Gram rounding (structural ranks, no host sync).
// rel_tol > 0: thresholds below ~1e-7 sigma_1 cannot be resolved from Gram eigenvalues
// (they square the singular values), so the threshold is applied by the accurate QR + SVD
// path whenever the bonds (after a structural Gram pass, if needed) fit it.
qtt_mps* round_any(Ctx& c, const qtt_mps* y, int chi, double eps) {
  if (eps <= 0.0) return round_gram(c, y, chi, 0.0);
  if (svd_path_fits(y->bonds, y->d)) return round_svd(c, y, chi, eps);
  std::unique_ptr<qtt_mps, void (*)(qtt_mps*)> z(round_gram(c, y, chi, 0.0), free_mps);
  if (svd_path_fits(z->bonds, z->d)) return round_svd(c, z.get(), chi, eps);
  return round_gram(c, z.get(), chi, eps);
}

// ------------------------------------------------------------------ right-orthonormalisation

void right_orthonormalize(Ctx& c, qtt_mps* x) {
  const int n = x->n, d = x->d;
  for (int k = n - 1; k >= 1; --k) {
    int r0 = x->bonds[k], r1 = x->bonds[k + 1];
    int mrows = d * r1;  // QR of Y^T (d r1 x r0)
    QTT_CHECK_ARG(mrows >= r0, "right_orthonormalize: bond larger than d * right bond");
    DBuf Rm(&c, size_t(r0) * r0);
    qr(c, 1, mrows, r0, 1, x->core(k), 0, x->core(k), 0, Rm.p, 0);
    int p0 = x->bonds[k - 1];
    DBuf prev(&c, size_t(p0) * d * r0);
    einsum(c, "asb,cb->asc", 1.0, tv(x->core(k - 1), {p0, d, r0}), tv(Rm.p, {r0, r0}), 0.0, tv(prev.p, {p0, d, r0}));
    copy(c, x->core(k - 1), prev.p, int64_t(p0) * d * r0);
  }
}

// ------------------------------------------------------------------ fit engine (Table I)

int Term::rbond(int k) const {
  if (kind == VEC) return a->bonds[k];
  if (kind == HAD) return a->bonds[k] * b->bonds[k];
  return M->bonds[k] * a->bonds[k];
}

// Environment shapes: VEC (c, a); HAD (c, a, b); MPO (c, w, a).
size_t env_size(const Term& t, int cb, int k) {
  if (t.kind == Term::VEC) return size_t(cb) * t.a->bonds[k];
  if (t.kind == Term::HAD) return size_t(cb) * t.a->bonds[k] * t.b->bonds[k];
  return size_t(cb) * t.M->bonds[k] * t.a->bonds[k];
}

// L_{k+1} from L_k and the new (left-orthonormal) core C of the fitted tensor at site k.
void env_left(Ctx& c, const Term& t, const double* L, const double* C, int c0, int c1, int k, double* Lout) {
  const int d = t.a->d;
  if (t.kind == Term::VEC) {
    int a0 = t.a->bonds[k], a1 = t.a->bonds[k + 1];
    DBuf T(&c, size_t(c0) * d * a1);
    einsum(c, "ca,asb->csb", 1.0, tv(const_cast<double*>(L), {c0, a0}), tv(t.a->core(k), {a0, d, a1}), 0.0,
           tv(T.p, {c0, d, a1}));
    einsum(c, "csb,csd->db", 1.0, tv(T.p, {c0, d, a1}), tv(const_cast<double*>(C), {c0, d, c1}), 0.0,
           tv(Lout, {c1, a1}));
  } else if (t.kind == Term::HAD) {
    int a0 = t.a->bonds[k], a1 = t.a->bonds[k + 1], b0 = t.b->bonds[k], b1 = t.b->bonds[k + 1];
    DBuf T1(&c, size_t(c0) * b0 * d * a1);
    einsum(c, "cab,ase->cbse", 1.0, tv(const_cast<double*>(L), {c0, a0, b0}), tv(t.a->core(k), {a0, d, a1}), 0.0,
           tv(T1.p, {c0, b0, d, a1}));
    DBuf T2(&c, size_t(d) * c0 * a1 * b1);
    einsum(c, "cbse,bsf->scef", 1.0, tv(T1.p, {c0, b0, d, a1}), tv(t.b->core(k), {b0, d, b1}), 0.0,
           tv(T2.p, {d, c0, a1, b1}));
    einsum(c, "csd,scef->def", 1.0, tv(const_cast<double*>(C), {c0, d, c1}), tv(T2.p, {d, c0, a1, b1}), 0.0,
           tv(Lout, {c1, a1, b1}));
  } else {
    int w0 = t.M->bonds[k], w1 = t.M->bonds[k + 1], a0 = t.a->bonds[k], a1 = t.a->bonds[k + 1];
    DBuf T1(&c, size_t(c0) * w0 * d * a1);
    einsum(c, "cwa,atb->cwtb", 1.0, tv(const_cast<double*>(L), {c0, w0, a0}), tv(t.a->core(k), {a0, d, a1}), 0.0,
           tv(T1.p, {c0, w0, d, a1}));
    DBuf T2(&c, size_t(c0) * d * w1 * a1);
    einsum(c, "cwtb,wstv->csvb", 1.0, tv(T1.p, {c0, w0, d, a1}), tv(t.M->core(k), {w0, d, d, w1}), 0.0,
           tv(T2.p, {c0, d, w1, a1}));
    einsum(c, "csvb,csd->dvb", 1.0, tv(T2.p, {c0, d, w1, a1}), tv(const_cast<double*>(C), {c0, d, c1}), 0.0,
           tv(Lout, {c1, w1, a1}));
  }
}

// R_k from R_{k+1} and the new (right-orthonormal) core C at site k.
void env_right(Ctx& c, const Term& t, const double* R, const double* C, int c0, int c1, int k, double* Rout) {
  const int d = t.a->d;
  if (t.kind == Term::VEC) {
    int a0 = t.a->bonds[k], a1 = t.a->bonds[k + 1];
    DBuf T(&c, size_t(a0) * d * c1);
    einsum(c, "asb,db->asd", 1.0, tv(t.a->core(k), {a0, d, a1}), tv(const_cast<double*>(R), {c1, a1}), 0.0,
           tv(T.p, {a0, d, c1}));
    einsum(c, "asd,csd->ca", 1.0, tv(T.p, {a0, d, c1}), tv(const_cast<double*>(C), {c0, d, c1}), 0.0,
           tv(Rout, {c0, a0}));
  } else if (t.kind == Term::HAD) {
    int a0 = t.a->bonds[k], a1 = t.a->bonds[k + 1], b0 = t.b->bonds[k], b1 = t.b->bonds[k + 1];
    DBuf T1(&c, size_t(a0) * d * c1 * b1);
    einsum(c, "ase,def->asdf", 1.0, tv(t.a->core(k), {a0, d, a1}), tv(const_cast<double*>(R), {c1, a1, b1}), 0.0,
           tv(T1.p, {a0, d, c1, b1}));
    DBuf T2(&c, size_t(d) * a0 * c1 * b0);
    einsum(c, "asdf,bsf->sadb", 1.0, tv(T1.p, {a0, d, c1, b1}), tv(t.b->core(k), {b0, d, b1}), 0.0,
           tv(T2.p, {d, a0, c1, b0}));
    einsum(c, "sadb,csd->cab", 1.0, tv(T2.p, {d, a0, c1, b0}), tv(const_cast<double*>(C), {c0, d, c1}), 0.0,
           tv(Rout, {c0, a0, b0}));
  } else {
    int w0 = t.M->bonds[k], w1 = t.M->bonds[k + 1], a0 = t.a->bonds[k], a1 = t.a->bonds[k + 1];
    DBuf T1(&c, size_t(a0) * d * c1 * w1);
    einsum(c, "atb,dvb->atdv", 1.0, tv(t.a->core(k), {a0, d, a1}), tv(const_cast<double*>(R), {c1, w1, a1}), 0.0,
           tv(T1.p, {a0, d, c1, w1}));
    DBuf T2(&c, size_t(a0) * w0 * d * c1);
    einsum(c, "atdv,wstv->awsd", 1.0, tv(T1.p, {a0, d, c1, w1}), tv(t.M->core(k), {w0, d, d, w1}), 0.0,
           tv(T2.p, {a0, w0, d, c1}));
    einsum(c, "awsd,csd->cwa", 1.0, tv(T2.p, {a0, w0, d, c1}), tv(const_cast<double*>(C), {c0, d, c1}), 0.0,
           tv(Rout, {c0, w0, a0}));
  }
}

// out (c0, d, c1) (+)= coef * projection of the term onto the frames L (site k) and R (site k+1).
// `vec` (if non-null) replaces the term's own core at site k (used by the ALS matvec).
void local_target(Ctx& c, const Term& t, const double* L, const double* R, int c0, int c1, int k, double coef,
                  double beta, double* out, const double* vec) {
  const int d = t.a->d;
  if (t.kind == Term::VEC) {
    int a0 = t.a->bonds[k], a1 = t.a->bonds[k + 1];
    DBuf T(&c, size_t(c0) * d * a1);
    einsum(c, "ca,asb->csb", 1.0, tv(const_cast<double*>(L), {c0, a0}), tv(t.a->core(k), {a0, d, a1}), 0.0,
           tv(T.p, {c0, d, a1}));
    einsum(c, "csb,db->csd", coef, tv(T.p, {c0, d, a1}), tv(const_cast<double*>(R), {c1, a1}), beta,
           tv(out, {c0, d, c1}));
  } else if (t.kind == Term::HAD) {
    int a0 = t.a->bonds[k], a1 = t.a->bonds[k + 1], b0 = t.b->bonds[k], b1 = t.b->bonds[k + 1];
    DBuf T1(&c, size_t(c0) * b0 * d * a1);
    einsum(c, "cab,ase->cbse", 1.0, tv(const_cast<double*>(L), {c0, a0, b0}), tv(t.a->core(k), {a0, d, a1}), 0.0,
           tv(T1.p, {c0, b0, d, a1}));
    DBuf T2(&c, size_t(d) * c0 * a1 * b1);
    einsum(c, "cbse,bsf->scef", 1.0, tv(T1.p, {c0, b0, d, a1}), tv(t.b->core(k), {b0, d, b1}), 0.0,
           tv(T2.p, {d, c0, a1, b1}));
    einsum(c, "scef,def->csd", coef, tv(T2.p, {d, c0, a1, b1}), tv(const_cast<double*>(R), {c1, a1, b1}), beta,
           tv(out, {c0, d, c1}));
  } else {
    int w0 = t.M->bonds[k], w1 = t.M->bonds[k + 1], a0 = t.a->bonds[k], a1 = t.a->bonds[k + 1];
    const double* X = vec ? vec : t.a->core(k);
    DBuf T1(&c, size_t(c0) * w0 * d * a1);
    einsum(c, "cwa,atb->cwtb", 1.0, tv(const_cast<double*>(L), {c0, w0, a0}), tv(const_cast<double*>(X), {a0, d, a1}),
           0.0, tv(T1.p, {c0, w0, d, a1}));
    DBuf T2(&c, size_t(c0) * d * w1 * a1);
    einsum(c, "cwtb,wstv->csvb", 1.0, tv(T1.p, {c0, w0, d, a1}), tv(t.M->core(k), {w0, d, d, w1}), 0.0,
           tv(T2.p, {c0, d, w1, a1}));
    einsum(c, "csvb,dvb->csd", coef, tv(T2.p, {c0, d, w1, a1}), tv(const_cast<double*>(R), {c1, w1, a1}), beta,
           tv(out, {c0, d, c1}));
  }
}

struct Envs {
  std::vector<std::vector<DBuf>> L, R;  // [term][k]
};

static void init_envs(Ctx& c, const std::vector<Term>& terms, const qtt_mps* x, Envs& E) {
  const int n = x->n;
  E.L.clear();
  E.R.clear();
  E.L.resize(terms.size());
  E.R.resize(terms.size());
  for (size_t t = 0; t < terms.size(); ++t) {
    E.L[t].resize(n + 1);
    E.R[t].resize(n + 1);
    E.L[t][0].reset(&c, 1);
    fill(c, E.L[t][0].p, 1, 1.0);
    E.R[t][n].reset(&c, 1);
    fill(c, E.R[t][n].p, 1, 1.0);
    for (int k = n - 1; k >= 1; --k) {
      E.R[t][k].reset(&c, env_size(terms[t], x->bonds[k], k));
      env_right(c, terms[t], E.R[t][k + 1].p, x->core(k), x->bonds[k], x->bonds[k + 1], k, E.R[t][k].p);
    }
  }
}

static void local_sum(Ctx& c, const std::vector<Term>& terms, const Envs& E, const qtt_mps* x, int k, double* out) {
  for (size_t t = 0; t < terms.size(); ++t)
    local_target(c, terms[t], E.L[t][k].p, E.R[t][k + 1].p, x->bonds[k], x->bonds[k + 1], k, terms[t].coef,
                 t == 0 ? 0.0 : 1.0, out);
}

void fit(Ctx& c, const std::vector<Term>& terms, qtt_mps* x, int sweeps, bool canonical) {
  QTT_CHECK_ARG(!terms.empty(), "fit: no terms");
  for (const Term& t : terms) QTT_CHECK_ARG(t.a->n == x->n && t.a->d == x->d, "fit: term shape mismatch");
  const int n = x->n, d = x->d;
  if (!canonical) right_orthonormalize(c, x);
  if (n == 1) {
    Envs E;
    init_envs(c, terms, x, E);
    DBuf T(&c, size_t(x->core_size(0)));
    local_sum(c, terms, E, x, 0, T.p);
    copy(c, x->core(0), T.p, x->core_size(0));
    return;
  }
  Envs E;
  init_envs(c, terms, x, E);
  for (int sw = 0; sw < sweeps; ++sw) {
    for (int k = 0; k < n; ++k) {
      int r0 = x->bonds[k], r1 = x->bonds[k + 1];
      DBuf T(&c, size_t(r0) * d * r1);
      local_sum(c, terms, E, x, k, T.p);
      if (k < n - 1) {
        qr(c, 1, r0 * d, r1, 0, T.p, 0, x->core(k), 0, nullptr, 0);
        for (size_t t = 0; t < terms.size(); ++t) {
          E.L[t][k + 1].reset(&c, env_size(terms[t], r1, k + 1));
          env_left(c, terms[t], E.L[t][k].p, x->core(k), r0, r1, k, E.L[t][k + 1].p);
        }
      } else {
        copy(c, x->core(k), T.p, int64_t(r0) * d * r1);
      }
    }
    for (int k = n - 1; k >= 0; --k) {
      int r0 = x->bonds[k], r1 = x->bonds[k + 1];
      DBuf T(&c, size_t(r0) * d * r1);
      local_sum(c, terms, E, x, k, T.p);
      if (k > 0) {
        qr(c, 1, d * r1, r0, 1, T.p, 0, x->core(k), 0, nullptr, 0);
        for (size_t t = 0; t < terms.size(); ++t) {
          E.R[t][k].reset(&c, env_size(terms[t], r0, k));
          env_right(c, terms[t], E.R[t][k + 1].p, x->core(k), r0, r1, k, E.R[t][k].p);
        }
      } else {
        copy(c, x->core(k), T.p, int64_t(r0) * d * r1);
      }
    }
  }
}

// ------------------------------------------------------------------ zip-up (Hadamard start)

qtt_mps* zipup_hadamard(Ctx& c, const qtt_mps* a, const qtt_mps* b, int chi) {
  QTT_CHECK_ARG(a->n == b->n && a->d == b->d, "zipup: shape mismatch");
  const int n = a->n, d = a->d;
  std::vector<int> R(n + 1);
  for (int k = 0; k <= n; ++k) R[k] = a->bonds[k] * b->bonds[k];
  std::vector<int> ms = left_struct(R, d);
  std::vector<int> ob(n + 1);
  ob[0] = 1;
  ob[n] = 1;
  std::vector<DBuf> out(n);
  DBuf C(&c, 1);
  fill(c, C.p, 1, 1.0);
  for (int k = n - 1; k >= 0; --k) {
    int a0 = a->bonds[k], a1 = a->bonds[k + 1], b0 = b->bonds[k], b1 = b->bonds[k + 1], c1 = ob[k + 1];
    DBuf T1(&c, size_t(a0) * d * c1 * b1);
    einsum(c, "asA,cAB->ascB", 1.0, tv(a->core(k), {a0, d, a1}), tv(C.p, {c1, a1, b1}), 0.0,
           tv(T1.p, {a0, d, c1, b1}));
    DBuf T(&c, size_t(a0) * b0 * d * c1);
    einsum(c, "bsB,ascB->absc", 1.0, tv(b->core(k), {b0, d, b1}), tv(T1.p, {a0, d, c1, b1}), 0.0,
           tv(T.p, {a0, b0, d, c1}));
    if (k == 0) {
      out[0] = std::move(T);
      break;
    }
    const int nv = d * c1;
    DBuf rho(&c, size_t(nv) * nv), w(&c, size_t(nv)), V(&c, size_t(nv) * nv);
    gemm(c, 1, nv, nv, int64_t(a0) * b0, 1.0, T.p, 0, 1, nv, T.p, 0, nv, 1, 0.0, rho.p, 0, nv, 1);
    int bk = std::max(1, std::min(std::min(chi, ms[k]), nv));
    eigh(c, nv, rho.p, w.p, V.p, bk);
    out[k].reset(&c, size_t(bk) * nv);
    top_vectors_as_core(c, V.p, nv, bk, out[k].p);
    // C_new(beta, a, b) = sum_{s,c} T(a, b, s, c) V(sc, beta)
    DBuf Cn(&c, size_t(bk) * a0 * b0);
    gemm(c, 1, bk, int64_t(a0) * b0, nv, 1.0, V.p, 0, 1, nv, T.p, 0, 1, nv, 0.0, Cn.p, 0, int64_t(a0) * b0, 1);
    C = std::move(Cn);
    ob[k] = bk;
  }
  qtt_mps* z = new_mps(&c, n, d, ob);
  for (int k = 0; k < n; ++k) copy(c, z->core(k), out[k].p, int64_t(ob[k]) * d * ob[k + 1]);
  return z;
}

// ------------------------------------------------------------------ inner products, norms

void dot_dev(Ctx& c, const qtt_mps* a, const qtt_mps* b, double* out_dev) {
  QTT_CHECK_ARG(a->n == b->n && a->d == b->d, "dot: shape mismatch");
  const int n = a->n, d = a->d;
  DBuf E(&c, 1);
  fill(c, E.p, 1, 1.0);
  for (int k = 0; k < n; ++k) {
    int a0 = a->bonds[k], a1 = a->bonds[k + 1], b0 = b->bonds[k], b1 = b->bonds[k + 1];
    DBuf T(&c, size_t(b0) * d * a1);
    einsum(c, "ab,asc->bsc", 1.0, tv(E.p, {a0, b0}), tv(a->core(k), {a0, d, a1}), 0.0, tv(T.p, {b0, d, a1}));
    DBuf En(&c, size_t(a1) * b1);
    einsum(c, "bsc,bsd->cd", 1.0, tv(T.p, {b0, d, a1}), tv(b->core(k), {b0, d, b1}), 0.0, tv(En.p, {a1, b1}));
    E = std::move(En);
  }
  copy(c, out_dev, E.p, 1);
}

// ------------------------------------------------------------------ dense encode / decode

qtt_mps* encode_dense(Ctx& c, const double* dense_dev, int n, int d, int chi, double eps) {
  QTT_CHECK_ARG(n >= 1 && n <= 40, "encode: n");
  if (eps > 0.0) {
    std::unique_ptr<qtt_mps, void (*)(qtt_mps*)> z(encode_dense(c, dense_dev, n, d, chi, 0.0), free_mps);
    return round_any(c, z.get(), chi, eps);
  }
  auto powd = [&](int k) {
    int64_t p = 1;
    for (int i = 0; i < k; ++i) p *= d;
    return p;
  };
  std::vector<int> ob(n + 1);
  ob[0] = 1;
  ob[n] = 1;
  std::vector<DBuf> out(n);
  DBuf cur(&c, size_t(powd(n)));
  copy(c, cur.p, dense_dev, powd(n));
  for (int k = n - 1; k >= 1; --k) {
    int c1 = ob[k + 1];
    int nv = d * c1;
    int64_t rows = powd(k);
    DBuf rho(&c, size_t(nv) * nv), w(&c, size_t(nv)), V(&c, size_t(nv) * nv);
    gemm(c, 1, nv, nv, rows, 1.0, cur.p, 0, 1, nv, cur.p, 0, nv, 1, 0.0, rho.p, 0, nv, 1);
    int strct = int(std::min<int64_t>(rows, nv));
    eigh(c, nv, rho.p, w.p, V.p, std::min(chi, strct));
    int bk = choose_rank(c, w.p, nv, chi, eps, strct);
    add_discarded(c, rho.p, w.p, nv, bk);
    out[k].reset(&c, size_t(bk) * nv);
    top_vectors_as_core(c, V.p, nv, bk, out[k].p);
    DBuf nxt(&c, size_t(rows) * bk);
    gemm(c, 1, rows, bk, nv, 1.0, cur.p, 0, nv, 1, V.p, 0, nv, 1, 0.0, nxt.p, 0, bk, 1);
    cur = std::move(nxt);
    ob[k] = bk;
  }
  out[0] = std::move(cur);
  qtt_mps* z = new_mps(&c, n, d, ob);
  for (int k = 0; k < n; ++k) copy(c, z->core(k), out[k].p, int64_t(ob[k]) * d * ob[k + 1]);
  return z;
}

void decode_dense(Ctx& c, const qtt_mps* x, double* dense_dev) {
  const int n = x->n, d = x->d;
  DBuf t(&c, 1);
  fill(c, t.p, 1, 1.0);
  int64_t rows = 1;
  for (int k = 0; k < n; ++k) {
    int a0 = x->bonds[k], a1 = x->bonds[k + 1];
    DBuf nt(&c, size_t(rows) * d * a1);
    gemm(c, 1, rows, int64_t(d) * a1, a0, 1.0, t.p, 0, a0, 1, x->core(k), 0, int64_t(d) * a1, 1, 0.0, nt.p, 0,
         int64_t(d) * a1, 1);
    t = std::move(nt);
    rows *= d;
  }
  copy(c, dense_dev, t.p, rows);
}

}  // namespace qtt
