// Single-site ALS solver for symmetric positive definite TT systems A x = b (arXiv:2507.05222,
// Sec. II.A.4; the pressure Poisson and momentum solves of Sec. III.C), swept until the true
// relative residual meets a tolerance.
//
// Per site k the local system (r_{k-1} d r_k unknowns, Fig. 5) is solved by CG on the fast
// matvec L . x . W . R (one cooperative kernel per solve where the shapes allow it, qtt_cg.cu),
// preconditioned by the inverse of the local matrix's diagonal (the paper preconditions the local
// updates without saying how, App. G), warm-started from the current core; the core is split by
// QR and the R factor pushed into the neighbour.  A sweep is a left-to-right half-sweep followed by a right-to-left one.
//
// Stop rule (the paper leaves it open): after every sweep the residual r = A x - b of the
// un-truncated TT A x (+) (-b) is evaluated entry by entry -- A x is formed exactly (bond w r),
// both A x and b are reconstructed on the device as 2^n-entry vectors (the left and right halves
// of the train contracted separately and joined by one product) and the squared differences
// are summed in a fixed order.  Each entry carries only its own rounding, so the relative
// residual is resolved down to ~1e-15, where the expanded form ||Ax||^2 - 2<b,Ax> + ||b||^2
// cancels below ~1e-8.  A one-thread control kernel then decides: converged (res <= rel_tol),
// stalled (a sweep after the first gained less than the fraction `stall`), out of sweeps,
// non-finite, or one more sweep; it also sets the local CG tolerance of the next sweep
// (cg_tol * res).
//
// Inside a captured step the sweep loop is a conditional WHILE node: its body (one sweep, the
// residual, the control kernel) is captured once into the node's body graph and the control
// kernel sets the loop condition on the device, so a whole time step with data-dependent sweep
// counts replays without the host.  Outside a capture the host drives the same kernels and
// reads the loop flag after every sweep.
//
// Every buffer the body touches is allocated before the loop with the solve's fixed bonds and
// updated in place, so the addresses captured in the body stay valid on every iteration.
#include <algorithm>
#include <memory>

#include "qtt_algebra.h"

namespace qtt {

namespace {

// ------------------------------------------------------------------ per-stage CG
// CG for the ALS local systems, spread over CG_BLOCKS blocks, one kernel per stage (the path
// for shapes the cooperative kernels of qtt_cg.cu do not take, and CG mode 1).  State lives on
// the device so that the host never waits: rr is kept in two slots (iteration `it` reads slot
// it & 1 and writes slot (it + 1) & 1) because blocks of one kernel are not ordered with respect
// to each other.  Partial sums are reduced in a fixed order (deterministic results).
constexpr int CG_BLOCKS = 32;
constexpr int CG_THREADS = 256;

struct CGState {
  double rr[2], rz[2];
  double bb, tol2;
  int active;
  int count;
  double part[3][CG_BLOCKS];   // per-block partial sums
};

__device__ double block_sum_d(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

__device__ __forceinline__ double sum_parts(const double* part) {
  double s = 0.0;
  for (int i = 0; i < CG_BLOCKS; ++i) s += part[i];
  return s;
}

// Preconditioned residual z = D^-1 r (z = r without a preconditioner).
__device__ __forceinline__ double zval(const double* dinv, double r, int64_t e) { return dinv ? dinv[e] * r : r; }

// r = b - Ax, p = z; partial r.r, b.b and r.z per block.
__global__ void __launch_bounds__(CG_THREADS) k_cg_init1(int64_t n, const double* __restrict__ b,
                                                         const double* __restrict__ Ax, const double* __restrict__ dinv,
                                                         double* __restrict__ r, double* __restrict__ p, CGState* st) {
  __shared__ double red[32];
  double rr = 0, bb = 0, rz = 0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    double re = b[e] - Ax[e];
    const double ze = zval(dinv, re, e);
    r[e] = re;
    p[e] = ze;
    rr += re * re;
    rz += re * ze;
    bb += b[e] * b[e];
  }
  rr = block_sum_d(rr, red);
  bb = block_sum_d(bb, red);
  rz = block_sum_d(rz, red);
  if (threadIdx.x == 0) {
    st->part[0][blockIdx.x] = rr;
    st->part[1][blockIdx.x] = bb;
    st->part[2][blockIdx.x] = rz;
  }
}

__global__ void k_cg_init2(CGState* st, const double* tol) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double rr = sum_parts(st->part[0]), bb = sum_parts(st->part[1]), rz = sum_parts(st->part[2]);
  const double tol2 = *tol * *tol;
  st->rr[0] = rr;
  st->rz[0] = rz;
  st->bb = bb;
  st->tol2 = tol2;
  st->active = (rr > tol2 * bb && rr > 0.0) ? 1 : 0;
  st->count = 0;
}

// partial p.Ap
__global__ void __launch_bounds__(CG_THREADS) k_cg_pap(int64_t n, const double* __restrict__ p,
                                                       const double* __restrict__ Ap, CGState* st) {
  __shared__ double red[32];
  if (!st->active) return;
  double s = 0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    s += p[e] * Ap[e];
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) st->part[0][blockIdx.x] = s;
}

// alpha = rz / pAp; x += alpha p; r -= alpha Ap; partial r.r and r.z
__global__ void __launch_bounds__(CG_THREADS) k_cg_xr(int64_t n, int it, double* __restrict__ x, double* __restrict__ r,
                                                      const double* __restrict__ p, const double* __restrict__ Ap,
                                                      const double* __restrict__ dinv, CGState* st) {
  __shared__ double red[32];
  if (!st->active) return;
  const double pap = sum_parts(st->part[0]);
  if (!(pap > 0.0)) {                    // every block computes the same pap and stops here
    if (blockIdx.x == 0 && threadIdx.x == 0) st->active = 0;
    return;
  }
  const double alpha = st->rz[it & 1] / pap;
  double rn = 0, rzn = 0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    x[e] += alpha * p[e];
    double re = r[e] - alpha * Ap[e];
    r[e] = re;
    rn += re * re;
    rzn += re * zval(dinv, re, e);
  }
  rn = block_sum_d(rn, red);
  rzn = block_sum_d(rzn, red);
  if (threadIdx.x == 0) {
    st->part[1][blockIdx.x] = rn;
    st->part[2][blockIdx.x] = rzn;
  }
}

// beta = rz' / rz; p = z + beta p; block 0 records rr', rz', the count and the stopping test.
__global__ void __launch_bounds__(CG_THREADS) k_cg_p(int64_t n, int it, const double* __restrict__ r,
                                                     const double* __restrict__ dinv, double* __restrict__ p,
                                                     CGState* st) {
  if (!st->active) return;
  const double rn = sum_parts(st->part[1]), rzn = sum_parts(st->part[2]);
  const double beta = rzn / st->rz[it & 1];
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    p[e] = zval(dinv, r[e], e) + beta * p[e];
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    st->rr[(it + 1) & 1] = rn;
    st->rz[(it + 1) & 1] = rzn;
    st->count += 1;
    st->active = (rn > st->tol2 * st->bb && rn > 0.0) ? 1 : 0;
  }
}

// dinv[c, s, e] = 1 / sum_{w, v} L[c, w, c] W[w, s, s, v] R[e, v, e]: the inverse diagonal of
// the local matrix L . W . R (Fig. 5), 1 where that diagonal is not positive.
__global__ void k_local_dinv(const double* __restrict__ L, const double* __restrict__ W, const double* __restrict__ R,
                             int r0, int r1, int w0, int w1, int d, double* __restrict__ dinv) {
  const int64_t n = int64_t(r0) * d * r1;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const int e = int(i % r1), s = int((i / r1) % d), c = int(i / (int64_t(r1) * d));
    double acc = 0.0;
    for (int w = 0; w < w0; ++w) {
      const double l = L[(int64_t(c) * w0 + w) * r0 + c];
      double t = 0.0;
      for (int v = 0; v < w1; ++v) t = fma(W[((int64_t(w) * d + s) * d + s) * w1 + v], R[(int64_t(e) * w1 + v) * r1 + e], t);
      acc = fma(l, t, acc);
    }
    dinv[i] = acc > 0.0 ? 1.0 / acc : 1.0;
  }
}

__global__ void k_cg_accumulate(const CGState* st, int* total) {
  if (threadIdx.x == 0 && blockIdx.x == 0 && *total >= 0) *total += st->count;
}

// ------------------------------------------------------------------ residual and control

constexpr int RES_THREADS = 256;
constexpr int RES_MAX_BLOCKS = 1024;

// part[block] = sum over the block's entries of (a - b)^2 (b may be null: a^2), block sums in
// a fixed order.
__global__ void __launch_bounds__(RES_THREADS) k_sq_partials(int64_t n, const double* __restrict__ a,
                                                             const double* __restrict__ b, double* __restrict__ part) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) {
    const double v = b ? a[e] - b[e] : a[e];
    s = fma(v, v, s);
  }
  s = block_sum_d(s, red);
  if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// y += coef * a (.) b (dense)
__global__ void k_had_acc(int64_t n, double coef, const double* __restrict__ a, const double* __restrict__ b,
                          double* __restrict__ y) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    y[e] = fma(coef * a[e], b[e], y[e]);
}

struct AlsParams {
  double rel_tol, cg_tol, stall;
  int max_sweeps;
  int G;                 // partial sums per vector
};

__device__ __forceinline__ double sum_in_order(const double* p, int G) {
  double s = 0.0;
  for (int i = 0; i < G; ++i) s += p[i];
  return s;
}

// Residual of the warm start: ||b|| from part_b, ||A x0 - b|| from part_r; first decision.
__global__ void k_als_start(AlsCtl* ctl, const double* part_b, const double* part_r, AlsParams P,
                            cudaGraphConditionalHandle h, int set_h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double nb = sqrt(sum_in_order(part_b, P.G));
  if (!(nb > 0.0)) nb = 1.0;
  const double res = sqrt(sum_in_order(part_r, P.G)) / nb;
  int status = -1;
  if (!isfinite(res) || !isfinite(nb)) status = QTT_SOLVE_NONFINITE;
  else if (res <= P.rel_tol) status = QTT_SOLVE_CONVERGED;
  else if (P.max_sweeps <= 0) status = QTT_SOLVE_MAX_SWEEPS;
  ctl->res = res;
  ctl->nb = nb;
  ctl->cg_tol = P.cg_tol * res;
  ctl->sweeps = 0;
  ctl->status = status;
  ctl->cont = status < 0 ? 1 : 0;
  ctl->cg_total = 0;
  if (set_h) cudaGraphSetConditional(h, status < 0 ? 1u : 0u);
}

// After a sweep: the new residual and the stop rule.
__global__ void k_als_after_sweep(AlsCtl* ctl, const double* part_r, AlsParams P, cudaGraphConditionalHandle h,
                                  int set_h) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const double prev = ctl->res;
  const double res = sqrt(sum_in_order(part_r, P.G)) / ctl->nb;
  const int sweeps = ctl->sweeps + 1;
  int status = -1;
  if (ctl->cg_total < 0) status = QTT_SOLVE_TIMEOUT;
  else if (!isfinite(res)) status = QTT_SOLVE_NONFINITE;
  else if (res <= P.rel_tol) status = QTT_SOLVE_CONVERGED;
  else if (P.stall > 0.0 && sweeps >= 2 && !(res <= (1.0 - P.stall) * prev)) status = QTT_SOLVE_STALLED;
  else if (sweeps >= P.max_sweeps) status = QTT_SOLVE_MAX_SWEEPS;
  ctl->res = res;
  ctl->cg_tol = P.cg_tol * res;
  ctl->sweeps = sweeps;
  ctl->status = status;
  ctl->cont = status < 0 ? 1 : 0;
  if (set_h) cudaGraphSetConditional(h, status < 0 ? 1u : 0u);
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return int(std::max<int64_t>(1, std::min<int64_t>(g, 65535 * 8)));
}

// Side stream of a context: the body of a conditional node is captured there.
cudaStream_t side_stream(Ctx& c) {
  if (!c.side) QTT_CUDA(cudaStreamCreateWithFlags(&c.side, cudaStreamNonBlocking));
  return c.side;
}

struct Envs {
  std::vector<std::vector<DBuf>> L, R;  // [term][k]
};

}  // namespace

// ------------------------------------------------------------------ dense reconstruction

void decode_mid(Ctx& c, const qtt_mps* x, double* dense) {
  const int n = x->n, d = x->d;
  const int h = n / 2;
  // left half: T (rows x r_k), rows = d^k
  DBuf t(&c, 1);
  fill(c, t.p, 1, 1.0);
  int64_t rows = 1;
  for (int k = 0; k < h; ++k) {
    const int a0 = x->bonds[k], a1 = x->bonds[k + 1];
    DBuf nt(&c, size_t(rows) * d * a1);
    gemm(c, 1, rows, int64_t(d) * a1, a0, 1.0, t.p, 0, a0, 1, x->core(k), 0, int64_t(d) * a1, 1, 0.0, nt.p, 0,
         int64_t(d) * a1, 1);
    t = std::move(nt);
    rows *= d;
  }
  // right half: S (r_k x cols), cols = d^(n-k); core k as (r_k d) x r_{k+1} times S
  DBuf s(&c, 1);
  fill(c, s.p, 1, 1.0);
  int64_t cols = 1;
  for (int k = n - 1; k >= h; --k) {
    const int a0 = x->bonds[k], a1 = x->bonds[k + 1];
    DBuf ns(&c, size_t(a0) * d * cols);
    gemm(c, 1, int64_t(a0) * d, cols, a1, 1.0, x->core(k), 0, a1, 1, s.p, 0, cols, 1, 0.0, ns.p, 0, cols, 1);
    s = std::move(ns);
    cols *= d;
  }
  const int rh = x->bonds[h];
  gemm(c, 1, rows, cols, rh, 1.0, t.p, 0, rh, 1, s.p, 0, cols, 1, 0.0, dense, 0, cols, 1);
}

// ------------------------------------------------------------------ the solver

void als(Ctx& c, const qtt_mpo* A, const std::vector<Term>& rhs, qtt_mps* x, const qtt_solve_opts& o, bool canonical,
         AlsCtl* ctl, int64_t* body_launches) {
  QTT_CHECK_ARG(A->n == x->n && A->d == x->d, "als: operator shape");
  for (const Term& t : rhs) QTT_CHECK_ARG(t.a->n == x->n && t.a->d == x->d, "als: rhs shape");
  QTT_CHECK_ARG(o.max_sweeps >= 0 && o.cg_max_iter >= 0 && o.cg_tol >= 0.0 && o.rel_tol >= 0.0,
                "als: options must be non-negative");
  const int n = x->n, d = x->d;
  int64_t N = 1;
  for (int k = 0; k < n; ++k) {
    N *= d;
    if (N > (int64_t(1) << 30)) throw Error(QTT_ERR_UNSUPPORTED, "als: the residual needs d^n <= 2^30 entries");
  }
  if (!canonical) right_orthonormalize(c, x);
  Term opT;
  opT.kind = Term::MPO;
  opT.coef = 1.0;
  opT.M = A;
  opT.a = x;
  // environments with the solve's fixed bonds, updated in place by the sweeps
  std::vector<DBuf> LA(n + 1), RA(n + 1);
  for (int k = 0; k <= n; ++k) {
    LA[k].reset(&c, env_size(opT, x->bonds[k], k));
    RA[k].reset(&c, env_size(opT, x->bonds[k], k));
  }
  fill(c, LA[0].p, 1, 1.0);
  fill(c, RA[n].p, 1, 1.0);
  for (int k = n - 1; k >= 1; --k) env_right(c, opT, RA[k + 1].p, x->core(k), x->bonds[k], x->bonds[k + 1], k, RA[k].p);
  Envs E;
  E.L.resize(rhs.size());
  E.R.resize(rhs.size());
  for (size_t t = 0; t < rhs.size(); ++t) {
    E.L[t].resize(n + 1);
    E.R[t].resize(n + 1);
    for (int k = 0; k <= n; ++k) {
      E.L[t][k].reset(&c, env_size(rhs[t], x->bonds[k], k));
      E.R[t][k].reset(&c, env_size(rhs[t], x->bonds[k], k));
    }
    fill(c, E.L[t][0].p, 1, 1.0);
    fill(c, E.R[t][n].p, 1, 1.0);
    for (int k = n - 1; k >= 1; --k)
      env_right(c, rhs[t], E.R[t][k + 1].p, x->core(k), x->bonds[k], x->bonds[k + 1], k, E.R[t][k].p);
  }
  // residual set-up: b reconstructed once, A x into a fixed buffer
  const int G = std::min(RES_MAX_BLOCKS, std::max(1, 2 * c.num_sms));
  DBuf bd(&c, size_t(N)), ad(&c, size_t(N)), part(&c, size_t(2) * G);
  fill(c, bd.p, N, 0.0);
  for (const Term& t : rhs) {
    if (t.kind == Term::VEC) {
      decode_mid(c, t.a, ad.p);
      axpby(c, N, t.coef, ad.p, 1.0, bd.p);
    } else if (t.kind == Term::MPO) {
      std::unique_ptr<qtt_mps, void (*)(qtt_mps*)> y(mpo_mps_exact(c, t.M, t.a), free_mps);
      decode_mid(c, y.get(), ad.p);
      axpby(c, N, t.coef, ad.p, 1.0, bd.p);
    } else {
      DBuf bb(&c, size_t(N));
      decode_mid(c, t.a, ad.p);
      decode_mid(c, t.b, bb.p);
      k_had_acc<<<grid_for(N, 256), 256, 0, c.stream>>>(N, t.coef, ad.p, bb.p, bd.p);
      after_launch(c, "had_acc");
    }
  }
  std::vector<int> yb(n + 1);
  for (int k = 0; k <= n; ++k) yb[k] = x->bonds[k] * A->bonds[k];
  std::unique_ptr<qtt_mps, void (*)(qtt_mps*)> Ax(new_mps(&c, n, d, yb), free_mps);
  double* part_b = part.p;
  double* part_r = part.p + G;
  auto residual = [&]() {
    mpo_mps_exact_into(c, A, x, Ax.get());
    decode_mid(c, Ax.get(), ad.p);
    k_sq_partials<<<G, RES_THREADS, 0, c.stream>>>(N, ad.p, bd.p, part_r);
    after_launch(c, "sq_partials");
  };
  k_sq_partials<<<G, RES_THREADS, 0, c.stream>>>(N, bd.p, nullptr, part_b);
  after_launch(c, "sq_partials");
  AlsParams P;
  P.rel_tol = o.rel_tol;
  P.cg_tol = o.cg_tol;
  P.stall = o.stall;
  P.max_sweeps = o.max_sweeps;
  P.G = G;
  int* total = &ctl->cg_total;
  const double* cg_tol = &ctl->cg_tol;

  auto solve_site = [&](int k) {
    int r0 = x->bonds[k], r1 = x->bonds[k + 1];
    int64_t nel = int64_t(r0) * d * r1;
    const int w0 = A->bonds[k], w1 = A->bonds[k + 1];
    // mode 0: tensor-core contractions at full-bond sites (r0 r1 >= 4096, where they measured
    // faster: ~690 vs ~800 us per Poisson solve at bonds 64), FP64 elsewhere; mode 2: FP64 only;
    // mode 3: tensor cores wherever the kernel fits
    const int mode = c.root->cg_mode;
    const bool tc = (mode == 3 || (mode == 0 && int64_t(r0) * r1 >= 4096)) && cg_tc_fits(c, r0, r1, w0, w1, d);
    DBuf bvec(&c, nel), xk(&c, nel), dinv(&c, nel);
    for (size_t t = 0; t < rhs.size(); ++t)
      local_target(c, rhs[t], E.L[t][k].p, E.R[t][k + 1].p, r0, r1, k, rhs[t].coef, t == 0 ? 0.0 : 1.0, bvec.p);
    copy(c, xk.p, x->core(k), nel);
    k_local_dinv<<<grid_for(nel, 256), 256, 0, c.stream>>>(LA[k].p, A->core(k), RA[k + 1].p, r0, r1, w0, w1, d, dinv.p);
    after_launch(c, "local_dinv");
    if (tc || (mode != 1 && cg_persistent_fits(c, r0, r1, w0, w1, d))) {
      if (tc)
        cg_tc(c, LA[k].p, A->core(k), RA[k + 1].p, bvec.p, xk.p, r0, r1, w0, w1, d, o.cg_max_iter, cg_tol, total,
              dinv.p);
      else
        cg_persistent(c, LA[k].p, A->core(k), RA[k + 1].p, bvec.p, xk.p, r0, r1, w0, w1, d, o.cg_max_iter, cg_tol,
                      total, dinv.p);
      return xk;
    }
    DBuf Ax_(&c, nel), r(&c, nel), p(&c, nel), Ap(&c, nel), stbuf(&c, (sizeof(CGState) + 7) / 8);
    CGState* st = reinterpret_cast<CGState*>(stbuf.p);
    local_target(c, opT, LA[k].p, RA[k + 1].p, r0, r1, k, 1.0, 0.0, Ax_.p, xk.p);
    k_cg_init1<<<CG_BLOCKS, CG_THREADS, 0, c.stream>>>(nel, bvec.p, Ax_.p, dinv.p, r.p, p.p, st);
    after_launch(c, "cg_init1");
    k_cg_init2<<<1, 32, 0, c.stream>>>(st, cg_tol);
    after_launch(c, "cg_init2");
    for (int it = 0; it < o.cg_max_iter; ++it) {
      c.guard = &st->active;
      local_target(c, opT, LA[k].p, RA[k + 1].p, r0, r1, k, 1.0, 0.0, Ap.p, p.p);
      c.guard = nullptr;
      ProfScope ps(c, KC_CG);
      k_cg_pap<<<CG_BLOCKS, CG_THREADS, 0, c.stream>>>(nel, p.p, Ap.p, st);
      after_launch(c, "cg_pap");
      k_cg_xr<<<CG_BLOCKS, CG_THREADS, 0, c.stream>>>(nel, it, xk.p, r.p, p.p, Ap.p, dinv.p, st);
      after_launch(c, "cg_xr");
      k_cg_p<<<CG_BLOCKS, CG_THREADS, 0, c.stream>>>(nel, it, r.p, dinv.p, p.p, st);
      after_launch(c, "cg_p");
    }
    k_cg_accumulate<<<1, 1, 0, c.stream>>>(st, total);
    after_launch(c, "cg_accumulate");
    return xk;
  };

  auto sweep = [&]() {
    for (int k = 0; k < n; ++k) {
      int r0 = x->bonds[k], r1 = x->bonds[k + 1];
      DBuf xk = solve_site(k);
      if (k < n - 1) {
        DBuf Rm(&c, size_t(r1) * r1);
        qr(c, 1, r0 * d, r1, 0, xk.p, 0, x->core(k), 0, Rm.p, 0);
        int r2 = x->bonds[k + 2];
        DBuf nxt(&c, size_t(r1) * d * r2);
        einsum(c, "ab,bsc->asc", 1.0, tv(Rm.p, {r1, r1}), tv(x->core(k + 1), {r1, d, r2}), 0.0, tv(nxt.p, {r1, d, r2}));
        copy(c, x->core(k + 1), nxt.p, int64_t(r1) * d * r2);
        env_left(c, opT, LA[k].p, x->core(k), r0, r1, k, LA[k + 1].p);
        for (size_t t = 0; t < rhs.size(); ++t) env_left(c, rhs[t], E.L[t][k].p, x->core(k), r0, r1, k, E.L[t][k + 1].p);
      } else {
        copy(c, x->core(k), xk.p, int64_t(r0) * d * r1);
      }
    }
    for (int k = n - 1; k >= 0; --k) {
      int r0 = x->bonds[k], r1 = x->bonds[k + 1];
      DBuf xk = solve_site(k);
      if (k > 0) {
        DBuf Rm(&c, size_t(r0) * r0);
        qr(c, 1, d * r1, r0, 1, xk.p, 0, x->core(k), 0, Rm.p, 0);
        int p0 = x->bonds[k - 1];
        DBuf prev(&c, size_t(p0) * d * r0);
        einsum(c, "asb,cb->asc", 1.0, tv(x->core(k - 1), {p0, d, r0}), tv(Rm.p, {r0, r0}), 0.0,
               tv(prev.p, {p0, d, r0}));
        copy(c, x->core(k - 1), prev.p, int64_t(p0) * d * r0);
        env_right(c, opT, RA[k + 1].p, x->core(k), r0, r1, k, RA[k].p);
        for (size_t t = 0; t < rhs.size(); ++t)
          env_right(c, rhs[t], E.R[t][k + 1].p, x->core(k), r0, r1, k, E.R[t][k].p);
      } else {
        copy(c, x->core(k), xk.p, int64_t(r0) * d * r1);
      }
    }
  };

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  QTT_CUDA(cudaStreamIsCapturing(c.stream, &cap));
  const bool capturing = cap == cudaStreamCaptureStatusActive;
  cudaGraphConditionalHandle hnd = 0;
  cudaGraph_t graph = nullptr;
  if (capturing) {
    QTT_CUDA(cudaStreamGetCaptureInfo(c.stream, &cap, nullptr, &graph, nullptr, nullptr, nullptr));
    QTT_CUDA(cudaGraphConditionalHandleCreate(&hnd, graph, 0, 0));
  }
  residual();
  k_als_start<<<1, 1, 0, c.stream>>>(ctl, part_b, part_r, P, hnd, capturing ? 1 : 0);
  after_launch(c, "als_start");
  const int64_t l0 = c.root->launches;
  if (capturing) {
    const cudaGraphNode_t* deps = nullptr;
    const cudaGraphEdgeData* edges = nullptr;
    size_t ndeps = 0;
    QTT_CUDA(cudaStreamGetCaptureInfo(c.stream, &cap, nullptr, &graph, &deps, &edges, &ndeps));
    cudaGraphNodeParams np = {};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = hnd;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node;
    QTT_CUDA(cudaGraphAddNode(&node, graph, deps, edges, ndeps, &np));
    cudaGraph_t body = np.conditional.phGraph_out[0];
    QTT_CUDA(cudaStreamUpdateCaptureDependencies(c.stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
    cudaStream_t outer = c.stream;
    cudaStream_t bs = side_stream(c);
    QTT_CUDA(cudaStreamBeginCaptureToGraph(bs, body, nullptr, nullptr, 0, cudaStreamCaptureModeRelaxed));
    c.stream = bs;
    try {
      sweep();
      residual();
      k_als_after_sweep<<<1, 1, 0, c.stream>>>(ctl, part_r, P, hnd, 1);
      after_launch(c, "als_after_sweep");
    } catch (...) {
      cudaGraph_t g2 = nullptr;
      cudaStreamEndCapture(bs, &g2);
      c.stream = outer;
      throw;
    }
    c.stream = outer;
    cudaGraph_t g2 = nullptr;
    QTT_CUDA(cudaStreamEndCapture(bs, &g2));
  } else {
    for (int s = 0; s <= o.max_sweeps; ++s) {
      int cont = 0;
      QTT_CUDA(cudaMemcpyAsync(&cont, &ctl->cont, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
      QTT_CUDA(cudaStreamSynchronize(c.stream));
      if (!cont) break;
      sweep();
      residual();
      k_als_after_sweep<<<1, 1, 0, c.stream>>>(ctl, part_r, P, hnd, 0);
      after_launch(c, "als_after_sweep");
    }
  }
  if (body_launches) *body_launches = capturing ? c.root->launches - l0 : 0;
}

}  // namespace qtt
