// Internal TT algebra interface (see qtt_algebra.cu).
#pragma once

#include <vector>

#include "qtt_internal.h"

namespace qtt {

// One term of a target sum: coef * x, coef * (a (.) b) or coef * (M x).
struct Term {
  enum Kind { VEC = 0, HAD = 1, MPO = 2 };
  int kind = VEC;
  double coef = 1.0;
  const qtt_mps* a = nullptr;   // x for VEC and MPO, first factor for HAD
  const qtt_mps* b = nullptr;   // second factor for HAD
  const qtt_mpo* M = nullptr;   // operator for MPO
  int rbond(int k) const;
  static Term vec(double c, const qtt_mps* x) { Term t; t.kind = VEC; t.coef = c; t.a = x; return t; }
  static Term had(double c, const qtt_mps* x, const qtt_mps* y) {
    Term t; t.kind = HAD; t.coef = c; t.a = x; t.b = y; return t;
  }
  static Term mpo(double c, const qtt_mpo* m, const qtt_mps* x) {
    Term t; t.kind = MPO; t.coef = c; t.M = m; t.a = x; return t;
  }
};

std::vector<int> left_struct(const std::vector<int>& pre, int d);

qtt_mps* direct_sum(Ctx& c, double alpha, const qtt_mps* x, double beta, const qtt_mps* y);
void direct_sum_core(Ctx& c, const double* X, int xr0, int xr1, const double* Y, int yr0, int yr1, int d, bool first,
                     bool last, double alpha, double beta, double* Z, int64_t zsize);
qtt_mpo* diag_mpo(Ctx& c, const qtt_mps* a);
qtt_mps* mpo_mps_exact(Ctx& c, const qtt_mpo* M, const qtt_mps* x);
qtt_mpo* mpo_mpo_exact(Ctx& c, const qtt_mpo* A, const qtt_mpo* B);
qtt_mps* mps_copy(Ctx& c, const qtt_mps* x);
void mps_scale(Ctx& c, qtt_mps* x, double s);
qtt_mps* mpo_as_mps(Ctx& c, const qtt_mpo* m);
qtt_mpo* mps_as_mpo(Ctx& c, const qtt_mps* x, int d);

// TT-rounding, exact TT-SVD semantics (right to left, result right-canonical).
qtt_mps* round_svd(Ctx& c, const qtt_mps* x, int chi, double eps);    // QR + Jacobi SVD, FP64
qtt_mps* round_gram(Ctx& c, const qtt_mps* y, int chi, double eps);   // Gram / density matrix
qtt_mps* round_any(Ctx& c, const qtt_mps* y, int chi, double eps);
// y = round(M x) by Gram rounding; written into `into` (bonds apply_bonds(M, x, chi)) if given.
qtt_mps* apply_round_gram(Ctx& c, const qtt_mpo* M, const qtt_mps* x, int chi, double eps, qtt_mps* into = nullptr);
// The same product rounded through a sketched left orthogonalisation and factored eigenpair
// refinement (no squared singular values; d * chi <= 256).
qtt_mps* apply_round_sketch(Ctx& c, const qtt_mpo* M, const qtt_mps* x, int chi, double eps, qtt_mps* into = nullptr);
std::vector<int> apply_bonds(const qtt_mpo* M, const qtt_mps* x, int chi);

void right_orthonormalize(Ctx& c, qtt_mps* x);
// Variational fit of sum(terms) in place on x (fixed bonds), `sweeps` full sweeps.
void fit(Ctx& c, const std::vector<Term>& terms, qtt_mps* x, int sweeps, bool canonical);
qtt_mps* zipup_hadamard(Ctx& c, const qtt_mps* a, const qtt_mps* b, int chi);
// Environments of the fit / ALS sweeps (Table I): shapes VEC (c, a), HAD (c, a, b), MPO (c, w, a).
size_t env_size(const Term& t, int cb, int k);
// L_{k+1} from L_k and the left-orthonormal core C (c0, d, c1) of site k; R_k from R_{k+1}.
void env_left(Ctx& c, const Term& t, const double* L, const double* C, int c0, int c1, int k, double* Lout);
void env_right(Ctx& c, const Term& t, const double* R, const double* C, int c0, int c1, int k, double* Rout);
// out (c0, d, c1) = coef * projection of the term onto the frames L, R + beta out; `vec`, if
// given, replaces the term's own core at site k (the ALS matvec).
void local_target(Ctx& c, const Term& t, const double* L, const double* R, int c0, int c1, int k, double coef,
                  double beta, double* out, const double* vec = nullptr);

// Device record of one ALS solve (qtt_als.cu), written by the solve's control kernels.
struct AlsCtl {
  double res;       // true relative residual ||A x - b|| / ||b|| of the current iterate
  double nb;        // ||b|| (1 when b = 0)
  double cg_tol;    // relative tolerance of the local CG solves of the next sweep
  double pad;
  int sweeps;       // full sweeps done
  int status;       // QTT_SOLVE_* (-1 while running)
  int cont;         // 1 while another sweep follows
  int cg_total;     // CG iterations (negative once a grid barrier timed out)
};
static_assert(sizeof(AlsCtl) == 48, "AlsCtl layout");
constexpr int kAlsCtlDoubles = 6;

// ALS for A x = sum(rhs) under the stop rule of qtt_solve_opts; the outcome lands in *ctl
// (device memory of at least sizeof(AlsCtl)).  When c.stream is being captured, the sweeps
// become a conditional WHILE node of the graph (body = one sweep, the residual and the control
// kernel); otherwise the host launches sweep after sweep until the control kernel says stop
// (one device-to-host read per sweep).  *body_launches (if given) receives the kernel launches
// of one sweep.
void als(Ctx& c, const qtt_mpo* A, const std::vector<Term>& rhs, qtt_mps* x, const qtt_solve_opts& o, bool canonical,
         AlsCtl* ctl, int64_t* body_launches = nullptr);
// Dense value (d^n entries, first core = most significant digit) of x by contracting the left
// and right halves separately and joining them with one product (n <= 30).
void decode_mid(Ctx& c, const qtt_mps* x, double* dense);
// y = M x without rounding into an existing MPS with bonds x.bonds * M.bonds.
void mpo_mps_exact_into(Ctx& c, const qtt_mpo* M, const qtt_mps* x, qtt_mps* y);

// One ALS local CG solve as a single cooperative kernel (qtt_cg.cu): L (r0, w0, r0),
// W (w0, d, d, w1), R (r1, w1, r1), b and x (r0, d, r1; x in/out); *total_dev += iterations
// done, or a negative value if a grid barrier timed out; tol_dev: relative CG tolerance (device scalar);
// dinv (may be null): the preconditioner, the inverse of the local matrix's diagonal (r0, d, r1).
bool cg_persistent_fits(const Ctx& c, int r0, int r1, int w0, int w1, int d);
void cg_init_attributes();   // kernel attributes and occupancy, once (before any stream capture)
void cg_persistent(Ctx& c, const double* L, const double* W, const double* R, const double* b, double* x, int r0,
                   int r1, int w0, int w1, int d, int iters, const double* tol_dev, int* total_dev,
                   const double* dinv);
// The same solve with both contractions as exact digit-split products on the tensor cores
// (qtt_cg.cu, CG mode 2); the caller's own stream only (one CTA per SM), r0 <= 64, products on
// the tensor cores (gemm mode 0).
bool cg_tc_fits(const Ctx& c, int r0, int r1, int w0, int w1, int d);
void cg_tc_init_attributes();
void cg_tc(Ctx& c, const double* L, const double* W, const double* R, const double* b, double* x, int r0, int r1,
           int w0, int w1, int d, int iters, const double* tol_dev, int* total_dev, const double* dinv);

void dot_dev(Ctx& c, const qtt_mps* a, const qtt_mps* b, double* out_dev);
void sqrt_dev(Ctx& c, const double* in, double* out);
qtt_mps* encode_dense(Ctx& c, const double* dense_dev, int n, int d, int chi, double eps);
void decode_dense(Ctx& c, const qtt_mps* x, double* dense_dev);

}  // namespace qtt
