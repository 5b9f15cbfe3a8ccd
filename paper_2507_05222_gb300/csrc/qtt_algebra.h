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
std::vector<int> apply_bonds(const qtt_mpo* M, const qtt_mps* x, int chi);

void right_orthonormalize(Ctx& c, qtt_mps* x);
// Variational fit of sum(terms) in place on x (fixed bonds), `sweeps` full sweeps.
void fit(Ctx& c, const std::vector<Term>& terms, qtt_mps* x, int sweeps, bool canonical);
qtt_mps* zipup_hadamard(Ctx& c, const qtt_mps* a, const qtt_mps* b, int chi);
// ALS for A x = sum(rhs); returns total CG iterations (host-synchronising) unless
// cg_total_dev is given (then the count is written there on the device and 0 is returned).
int als(Ctx& c, const qtt_mpo* A, const std::vector<Term>& rhs, qtt_mps* x, int sweeps, int cg_iters, double cg_tol,
        bool canonical, int* cg_total_dev);

// One ALS local CG solve as a single cooperative kernel (qtt_cg.cu): L (r0, w0, r0),
// W (w0, d, d, w1), R (r1, w1, r1), b and x (r0, d, r1; x in/out); *total_dev += iterations
// done, or a negative value if a grid barrier timed out.
bool cg_persistent_fits(const Ctx& c, int r0, int r1, int w0, int w1, int d);
void cg_init_attributes();   // kernel attributes and occupancy, once (before any stream capture)
void cg_persistent(Ctx& c, const double* L, const double* W, const double* R, const double* b, double* x, int r0,
                   int r1, int w0, int w1, int d, int iters, double tol, int* total_dev);
// The same solve with both contractions as exact digit-split products on the tensor cores
// (qtt_cg.cu, CG mode 2); the caller's own stream only (one CTA per SM), r0 <= 64, products on
// the tensor cores (gemm mode 0).
bool cg_tc_fits(const Ctx& c, int r0, int r1, int w0, int w1, int d);
void cg_tc_init_attributes();
void cg_tc(Ctx& c, const double* L, const double* W, const double* R, const double* b, double* x, int r0, int r1,
           int w0, int w1, int d, int iters, double tol, int* total_dev);

void dot_dev(Ctx& c, const qtt_mps* a, const qtt_mps* b, double* out_dev);
void norm_dev(Ctx& c, const qtt_mps* y, double* out_dev);
void sqrt_dev(Ctx& c, const double* in, double* out);
qtt_mps* encode_dense(Ctx& c, const double* dense_dev, int n, int d, int chi, double eps);
void decode_dense(Ctx& c, const qtt_mps* x, double* dense_dev);

}  // namespace qtt
