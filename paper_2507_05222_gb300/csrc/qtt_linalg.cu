// Small dense factorisations for the QTT sweeps, one CTA per matrix, operands in shared
// memory:
//   * Householder QR in FP64 (gauge moves of the fit and ALS sweeps; the orthogonalisation
//     sweep of the accurate rounding), blocked and spread over a thread-block cluster of up
//     to 16 CTAs (one SM of GB300 retires only 2 FP64 FMAs per cycle, so a one-CTA QR of a
//     128 x 64 unfolding is bound at ~0.2 ms by that SM's FP64 pipe), one CTA for small or
//     wide matrices;
//   * one-sided (Hestenes) Jacobi SVD in FP64 for small accurate roundings (operator set-up,
//     rel_tol > 0);
//   * symmetric eigendecomposition: cyclic parallel Jacobi in FP32 (the FP32 pipe of GB300 is
//     ~70x the FP64 pipe) followed by FP64 refinement of all eigenpairs with the
//     Ogita-Aishima iteration (Ogita & Aishima, Japan J. Indust. Appl. Math. 35, 2018), whose
//     matrix products run on the FP64 GEMM path across many SMs.
// Every loop has a fixed upper bound; no kernel waits on another.
#include <cooperative_groups.h>

#include <algorithm>
#include <cmath>

#include "qtt_internal.h"

namespace cgrp = cooperative_groups;

namespace qtt {

namespace {

// Descending order with ties broken by index, NaN placed after every number: a strict total
// order, so the rank-counting sorts below always produce a permutation (with NaN values
// compared plainly, every comparison is false and several entries would share one rank).
__device__ __forceinline__ bool sort_before(double a, int ia, double b, int ib) {
  const bool na = isnan(a), nb = isnan(b);
  if (na || nb) return (na == nb) ? ia < ib : nb;
  return a > b || (a == b && ia < ib);
}

}  // namespace

namespace {

__device__ __forceinline__ double warp_sum(double v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sumf(float v) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Block-wide sum (all threads get the result).  red must hold 32 doubles.
__device__ double block_sum(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

// ------------------------------------------------------------------ Householder QR (FP64)
// A (m x n) = Q (m x kk) R (kk x n), kk = min(m, n).  Shared layout: column-major S[c*m + r].
// trans = 0: input row-major (m x n), Q written row-major (m x kk).
// trans = 1: the input buffer holds A^T row-major (n x m) -- i.e. exactly the column-major
//            image -- and Q^T (kk x m) is written row-major.  This serves right-to-left
//            sweeps, which factor the transpose of a core's (r_{k-1} x d r_k) unfolding.
// Q may alias the input when kk == n.  R (kk x n, row-major) is written if non-null.
__global__ void __launch_bounds__(256) k_qr(int m, int n, int trans, const double* __restrict__ Ain, double* Qall,
                                            double* __restrict__ Rall, int64_t in_stride, int64_t q_stride,
                                            int64_t r_stride) {
  extern __shared__ double sm[];
  const int kk = min(m, n);
  double* S = sm;                 // m*n
  double* v = S + size_t(m) * n;  // m (current reflector)
  double* tau = v + m;            // kk
  double* red = tau + kk;         // 32
  const double* A = Ain + blockIdx.x * in_stride;
  double* Q = Qall + blockIdx.x * q_stride;
  double* R = Rall ? Rall + blockIdx.x * r_stride : nullptr;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  for (int e = tid; e < m * n; e += nt) {
    if (trans) S[e] = A[e];
    else S[(e % n) * m + e / n] = A[e];
  }
  __syncthreads();
  for (int j = 0; j < kk; ++j) {
    double* x = S + j * m;
    double part = 0.0;
    for (int i = j + 1 + tid; i < m; i += nt) part += x[i] * x[i];
    double sigma = block_sum(part, red);
    double alpha = x[j];
    double beta, t, scale;
    if (sigma == 0.0) {
      t = 0.0; beta = alpha; scale = 0.0;
    } else {
      double nrm = sqrt(alpha * alpha + sigma);
      beta = alpha >= 0.0 ? -nrm : nrm;
      t = (beta - alpha) / beta;
      scale = 1.0 / (alpha - beta);
    }
    for (int i = j + tid; i < m; i += nt) v[i] = (i == j) ? 1.0 : x[i] * scale;
    if (tid == 0) tau[j] = t;
    __syncthreads();
    for (int i = j + tid; i < m; i += nt) x[i] = (i == j) ? beta : v[i];
    for (int c = j + 1 + warp; c < n; c += nwarps) {
      double* y = S + c * m;
      double w = 0.0;
      for (int i = j + lane; i < m; i += 32) w += v[i] * y[i];
      w = warp_sum(w) * t;
      for (int i = j + lane; i < m; i += 32) y[i] -= w * v[i];
    }
    __syncthreads();
  }
  if (R) {
    for (int e = tid; e < kk * n; e += nt) {
      int r = e / n, c = e % n;
      R[e] = (r <= c) ? S[c * m + r] : 0.0;
    }
  }
  __syncthreads();
  // Q = H_0 ... H_{kk-1} [I]_{:, :kk}, accumulated backwards in place in columns 0..kk-1.
  for (int j = kk - 1; j >= 0; --j) {
    double* x = S + j * m;
    for (int i = j + 1 + tid; i < m; i += nt) v[i] = x[i];
    __syncthreads();
    const double t = tau[j];
    for (int i = j + tid; i < m; i += nt) x[i] = (i == j) ? 1.0 - t : -t * v[i];
    for (int c = j + 1 + tid; c < kk; c += nt) S[c * m + j] = 0.0;
    __syncthreads();
    for (int c = j + 1 + warp; c < kk; c += nwarps) {
      double* y = S + c * m;
      double w = 0.0;
      for (int i = j + 1 + lane; i < m; i += 32) w += v[i] * y[i];
      w = warp_sum(w) * t;
      if (lane == 0) y[j] -= w;
      for (int i = j + 1 + lane; i < m; i += 32) y[i] -= w * v[i];
    }
    __syncthreads();
  }
  for (int e = tid; e < m * kk; e += nt) {
    if (trans) Q[e] = S[e];                      // Q^T row-major (kk x m)
    else Q[e] = S[(e % kk) * m + e / kk];        // Q row-major (m x kk)
  }
}

// ------------------------------------------------------------------ cluster Householder QR (FP64)
// Same factorisation and conventions as k_qr (beta = -sign(alpha) ||x||, unit-diagonal
// reflectors, thin Q), for m >= n, organised as a blocked right-looking QR over a cluster of
// cs CTAs.  CTA q owns columns [q nb, q nb + nb) and holds them in shared memory for the
// whole factorisation; panel p is CTA p's column block.
//   R phase, for p = 0 .. cs-1: CTA p factors its (already updated) panel with one warp and
//     forms the compact-WY factor T_p (H_{j0} ... H_{j0+w-1} = I - V_p T_p V_p^T); after a
//     cluster barrier every CTA q > p reads V_p and T_p from CTA p's shared memory (DSMEM)
//     and updates its columns, A_q <- (I - V_p T_p^T V_p^T) A_q.
//   Q phase: column block q of Q = H_0 ... H_{n-1} [I; 0] only sees panels p <= q, so each CTA
//     accumulates its own columns of Q backwards from the final V_p, T_p with no further
//     synchronisation; a last cluster barrier keeps every CTA's shared memory alive until the
//     others have read it.
// Shared layout (doubles): Acol | Qcol | Vb (m x nb each, column-major) | T | Tb | W | W2
// (nb x nb each) | tau (nb).
constexpr int QRC_THREADS = 256;

// 1/sqrt(q) and 1/x by Newton-Raphson from the hardware's approximate FP64 reciprocal (square
// root), two quadratically convergent steps each (~20 correct bits -> beyond 53).  An FP64
// division or square root is a sequence of ~10 dependent FP64 operations, ~650 cycles on this
// part; these take 3 x 64 (reciprocal) and 6 x 64 (reciprocal square root) cycles.  Results are
// within a few ulp of the correctly rounded ones (checked against CUDA's by qtt_check_recip).
__device__ __forceinline__ double rcp_nr(double x) {
  double y;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double e = fma(-x, y, 1.0);
  y = fma(y, e, y);
  e = fma(-x, y, 1.0);
  return fma(y, e, y);
}
__device__ __forceinline__ double rsqrt_nr(double x) {
  double y;
  asm("rsqrt.approx.ftz.f64 %0, %1;" : "=d"(y) : "d"(x));
  double r = fma(-x * y, y, 1.0);
  y = fma(0.5 * y, r, y);
  r = fma(-x * y, y, 1.0);
  return fma(0.5 * y, r, y);
}

// Householder scalars of a column with pivot alpha and sum of squares sigma below it (LAPACK
// convention): beta = -sign(alpha) ||x||, t = (beta - alpha) / beta = 1 + |alpha| / ||x||,
// scale = 1 / (alpha - beta) = sign(alpha) / (|alpha| + ||x||).  sigma = 0: identity reflector.
__device__ __forceinline__ void householder_scalars(double alpha, double sigma, double& beta, double& t,
                                                    double& scale) {
  if (sigma == 0.0) {
    t = 0.0;
    beta = alpha;
    scale = 0.0;
    return;
  }
  const double q = fma(alpha, alpha, sigma);
  const double g = rsqrt_nr(q);
  const double nrm = q * g;
  const double aa = fabs(alpha);
  beta = alpha >= 0.0 ? -nrm : nrm;
  t = fma(aa, g, 1.0);
  const double rd = rcp_nr(aa + nrm);
  scale = alpha >= 0.0 ? rd : -rd;
}

__global__ void k_check_recip(int n, const double* __restrict__ x, double* __restrict__ err) {
  // err[0] = max relative error of rcp_nr, err[1] of rsqrt_nr, against CUDA's 1/x, 1/sqrt(x)
  __shared__ double red[2][32];
  double e0 = 0.0, e1 = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = x[i];
    const double a = 1.0 / v, b = 1.0 / sqrt(v);
    e0 = fmax(e0, fabs(rcp_nr(v) - a) / fabs(a));
    e1 = fmax(e1, fabs(rsqrt_nr(v) - b) / fabs(b));
  }
  for (int o = 16; o > 0; o >>= 1) {
    e0 = fmax(e0, __shfl_xor_sync(0xffffffffu, e0, o));
    e1 = fmax(e1, __shfl_xor_sync(0xffffffffu, e1, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = e0;
    red[1][threadIdx.x >> 5] = e1;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double m0 = 0.0, m1 = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) {
      m0 = fmax(m0, red[0][w]);
      m1 = fmax(m1, red[1][w]);
    }
    err[0] = m0;
    err[1] = m1;
  }
}

__host__ __device__ constexpr size_t qrc_smem_doubles(int m, int nb) {
  return size_t(3) * m * nb + 4 * size_t(nb) * nb + nb;
}

// X(i, c) (i >= j0, c < ncols, column-major with leading dimension m) <- (I - V op(T) V^T) X,
// op(T) = T^T when transT, else T.  V: m x wp (rows >= j0 valid), T: wp x wp upper triangular
// with leading dimension nb.  Called by every thread of the CTA; ends with a CTA barrier.
__device__ void qrc_apply_block(int m, int nb, int j0, int wp, int ncols, const double* V, const double* T, bool transT,
                                double* X, double* W, double* W2) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nd = wp * ncols;
  int g = 32;
  while (g > 1 && g * nd > nt) g >>= 1;
  {
    const int dd = tid / g, gl = tid % g;
    double s = 0.0;
    if (dd < nd) {
      const int l = dd / ncols, c = dd % ncols;
      const double* vl = V + size_t(l) * m;
      const double* xc = X + size_t(c) * m;
      for (int i = j0 + gl; i < m; i += g) s += vl[i] * xc[i];
    }
    for (int o = g >> 1; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (dd < nd && gl == 0) W[dd] = s;
  }
  __syncthreads();
  if (tid < nd) {
    const int l = tid / ncols, c = tid % ncols;
    double s = 0.0;
    if (transT) {
      for (int l2 = 0; l2 <= l; ++l2) s += T[l2 * nb + l] * W[l2 * ncols + c];
    } else {
      for (int l2 = l; l2 < wp; ++l2) s += T[l * nb + l2] * W[l2 * ncols + c];
    }
    W2[tid] = s;
  }
  __syncthreads();
  const int mr = m - j0;
  for (int e = tid; e < mr * ncols; e += nt) {
    const int c = e / mr, i = j0 + e % mr;
    double s = 0.0;
    for (int l = 0; l < wp; ++l) s += V[size_t(l) * m + i] * W2[l * ncols + c];
    X[size_t(c) * m + i] -= s;
  }
  __syncthreads();
}

// Copy panel p's reflectors (unit diagonal, zeros above, from the factored columns src) and
// its T into the local buffers Vb, Tb.  Ends with a CTA barrier.
__device__ void qrc_fetch_panel(int m, int nb, int j0, int wp, const double* src, const double* srcT, double* Vb,
                                double* Tb) {
  const int tid = threadIdx.x, nt = blockDim.x;
  const int mr = m - j0;
  for (int e = tid; e < mr * wp; e += nt) {
    const int l = e / mr, i = j0 + e % mr;
    const int diag = j0 + l;
    Vb[size_t(l) * m + i] = (i < diag) ? 0.0 : (i == diag ? 1.0 : src[size_t(l) * m + i]);
  }
  for (int e = tid; e < wp * nb; e += nt) Tb[e] = srcT[e];
  __syncthreads();
}

__global__ void __launch_bounds__(QRC_THREADS) k_qr_cluster(int m, int n, int nb, int trans, const double* __restrict__ Ain,
                                                           double* Qall, double* __restrict__ Rall, int64_t in_stride,
                                                           int64_t q_stride, int64_t r_stride) {
  cgrp::cluster_group cl = cgrp::this_cluster();
  const int cs = int(cl.num_blocks());
  const int q = int(cl.block_rank());
  const int mat = blockIdx.x / cs;
  extern __shared__ double sm[];
  double* Acol = sm;
  double* Qcol = Acol + size_t(m) * nb;
  double* Vb = Qcol + size_t(m) * nb;
  double* T = Vb + size_t(m) * nb;
  double* Tb = T + nb * nb;
  double* W = Tb + nb * nb;
  double* W2 = W + nb * nb;
  double* tau = W2 + nb * nb;
  const double* A = Ain + mat * in_stride;
  double* Q = Qall + mat * q_stride;
  double* R = Rall ? Rall + mat * r_stride : nullptr;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps_all = nt >> 5;
  const int c0 = q * nb;
  const int w = max(0, min(nb, n - c0));
  for (int e = tid; e < m * w; e += nt) {
    if (trans) {
      const int c = e / m, i = e % m;
      Acol[size_t(c) * m + i] = A[int64_t(c0 + c) * m + i];
    } else {
      const int i = e / w, c = e % w;
      Acol[size_t(c) * m + i] = A[int64_t(i) * n + c0 + c];
    }
  }
  for (int e = tid; e < nb * nb; e += nt) T[e] = 0.0;
  __syncthreads();

  // ---- R phase
  for (int p = 0; p < cs; ++p) {
    const int j0 = p * nb;
    const int wp = max(0, min(nb, n - j0));
    if (p == q) {
      // Panel factorisation.  Warp 0 forms reflector j; the other panel columns are then updated
      // by one warp each (every warp sits on its own SM sub-partition and FP64 unit: one warp
      // issues at most one FP64 instruction per ~64 cycles on this part).
      for (int j = 0; j < w; ++j) {
        const int r = j0 + j;
        if (warp == 0) {
          double* x = Acol + size_t(j) * m;
          double part0 = 0.0, part1 = 0.0;
          int i = r + 1 + lane;
          for (; i + 32 < m; i += 64) {
            part0 = fma(x[i], x[i], part0);
            part1 = fma(x[i + 32], x[i + 32], part1);
          }
          if (i < m) part0 = fma(x[i], x[i], part0);
          const double sigma = warp_sum(part0 + part1);
          const double alpha = x[r];
          double beta, t, scale;
          householder_scalars(alpha, sigma, beta, t, scale);
          __syncwarp();
          for (int i2 = r + 1 + lane; i2 < m; i2 += 32) x[i2] *= scale;
          if (lane == 0) {
            x[r] = beta;
            tau[j] = t;
          }
        }
        __syncthreads();
        for (int jj = j + 1 + warp; jj < w; jj += nwarps_all) {
          const double* x = Acol + size_t(j) * m;
          double* y = Acol + size_t(jj) * m;
          double sdot = 0.0;
          for (int i = r + 1 + lane; i < m; i += 32) sdot = fma(x[i], y[i], sdot);
          sdot = (warp_sum(sdot) + y[r]) * tau[j];
          __syncwarp();
          if (lane == 0) y[r] -= sdot;
          for (int i = r + 1 + lane; i < m; i += 32) y[i] -= sdot * x[i];
        }
        __syncthreads();
      }
      // T: T_ii = tau_i, T_{0:i, i} = -tau_i T_{0:i, 0:i} z_{0:i, i} with z_{l,i} = v_l . v_i,
      // the w (w - 1) / 2 products one warp each, then the triangular recurrence in warp 0
      const int npair = w * (w - 1) / 2;
      for (int pidx = warp; pidx < npair; pidx += nwarps_all) {
        int i = 1, base = 0;
        while (base + i <= pidx) {
          base += i;
          ++i;
        }
        const int l = pidx - base;
        const double* vi = Acol + size_t(i) * m;
        const double* vl = Acol + size_t(l) * m;
        double sdot = 0.0;
        for (int row = j0 + i + 1 + lane; row < m; row += 32) sdot = fma(vl[row], vi[row], sdot);
        sdot = warp_sum(sdot) + vl[j0 + i];
        if (lane == 0) W[l * nb + i] = sdot;
      }
      __syncthreads();
      if (warp == 0) {
        for (int i = 0; i < w; ++i) {
          if (lane < i) {
            double sacc = 0.0;
            for (int l2 = lane; l2 < i; ++l2) sacc = fma(T[lane * nb + l2], W[l2 * nb + i], sacc);
            T[lane * nb + i] = -tau[i] * sacc;
          }
          if (lane == 0) T[i * nb + i] = tau[i];
          __syncwarp();
        }
      }
    }
    cl.sync();
    if (q > p) {
      qrc_fetch_panel(m, nb, j0, wp, cl.map_shared_rank(Acol, p), cl.map_shared_rank(T, p), Vb, Tb);
      qrc_apply_block(m, nb, j0, wp, w, Vb, Tb, true, Acol, W, W2);
    }
  }
  if (R) {
    for (int e = tid; e < n * w; e += nt) {
      const int r = e / w, c = e % w;
      R[int64_t(r) * n + c0 + c] = (r <= c0 + c) ? Acol[size_t(c) * m + r] : 0.0;
    }
  }

  // ---- Q phase: own columns of H_0 ... H_{n-1} [I; 0], panels q, q-1, ..., 0
  for (int e = tid; e < m * w; e += nt) {
    const int c = e / m, i = e % m;
    Qcol[size_t(c) * m + i] = (i == c0 + c) ? 1.0 : 0.0;
  }
  __syncthreads();
  for (int p = q; p >= 0; --p) {
    const int j0 = p * nb;
    const int wp = max(0, min(nb, n - j0));
    const double* srcA = (p == q) ? Acol : cl.map_shared_rank(Acol, p);
    const double* srcT = (p == q) ? T : cl.map_shared_rank(T, p);
    qrc_fetch_panel(m, nb, j0, wp, srcA, srcT, Vb, Tb);
    qrc_apply_block(m, nb, j0, wp, w, Vb, Tb, false, Qcol, W, W2);
  }
  for (int e = tid; e < m * w; e += nt) {
    if (trans) {
      const int c = e / m, i = e % m;
      Q[int64_t(c0 + c) * m + i] = Qcol[size_t(c) * m + i];   // Q^T row-major (n x m)
    } else {
      const int i = e / w, c = e % w;
      Q[int64_t(i) * n + c0 + c] = Qcol[size_t(c) * m + i];   // Q row-major (m x n)
    }
  }
  cl.sync();
}

// ------------------------------------------------------------------ one-sided Jacobi SVD (FP64)
// G: m x n row-major (m >= n).  Outputs U (m x n, row-major), s (n, descending), V (n x n,
// row-major, columns = right singular vectors).
__global__ void __launch_bounds__(256) k_svd_jacobi(int m, int n, const double* __restrict__ G, double* __restrict__ U,
                                                    double* __restrict__ s, double* __restrict__ Vout, int max_sweeps) {
  extern __shared__ double sm[];
  double* A = sm;                    // column-major m x n
  double* V = A + size_t(m) * n;     // column-major n x n
  double* nrm = V + size_t(n) * n;   // n
  int* order = reinterpret_cast<int*>(nrm + n);  // n
  __shared__ int rotated;
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
  for (int e = tid; e < m * n; e += nt) A[(e % n) * m + e / n] = G[e];
  for (int e = tid; e < n * n; e += nt) V[e] = ((e / n) == (e % n)) ? 1.0 : 0.0;
  __syncthreads();
  const int np = (n + 1) & ~1;  // players (a dummy when n is odd)
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    if (tid == 0) rotated = 0;
    __syncthreads();
    for (int r = 0; r < np - 1; ++r) {
      // round-robin pairs: (r, np-1) and ((r+k) mod (np-1), (r-k) mod (np-1)), k = 1..np/2-1
      for (int k = warp; k < np / 2; k += nwarps) {
        int p, q;
        if (k == 0) { p = r; q = np - 1; }
        else { p = (r + k) % (np - 1); q = (r - k + (np - 1)) % (np - 1); }
        if (p >= n || q >= n) continue;
        if (p > q) { int tmp = p; p = q; q = tmp; }
        double* ap = A + p * m;
        double* aq = A + q * m;
        double al = 0, be = 0, ga = 0;
        for (int i = lane; i < m; i += 32) {
          double x = ap[i], y = aq[i];
          al += x * x; be += y * y; ga += x * y;
        }
        al = warp_sum(al); be = warp_sum(be); ga = warp_sum(ga);
        if (ga == 0.0 || fabs(ga) <= 1e-15 * sqrt(al * be)) continue;
        double zeta = (be - al) / (2.0 * ga);
        double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
        double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
        for (int i = lane; i < m; i += 32) {
          double x = ap[i], y = aq[i];
          ap[i] = cs * x - sn * y;
          aq[i] = sn * x + cs * y;
        }
        double* vp = V + p * n;
        double* vq = V + q * n;
        for (int i = lane; i < n; i += 32) {
          double x = vp[i], y = vq[i];
          vp[i] = cs * x - sn * y;
          vq[i] = sn * x + cs * y;
        }
        if (lane == 0) rotated = 1;
      }
      __syncthreads();
    }
    if (!rotated) break;
    __syncthreads();
  }
  // singular values and a descending order (selection by rank counting, ties by index)
  for (int c = warp; c < n; c += nwarps) {
    double w = 0;
    for (int i = lane; i < m; i += 32) w += A[c * m + i] * A[c * m + i];
    w = warp_sum(w);
    if (lane == 0) nrm[c] = sqrt(w);
  }
  __syncthreads();
  for (int c = tid; c < n; c += nt) {
    int rank = 0;
    for (int o = 0; o < n; ++o)
      if (sort_before(nrm[o], o, nrm[c], c)) ++rank;
    order[rank] = c;
  }
  __syncthreads();
  for (int e = tid; e < n; e += nt) s[e] = nrm[order[e]];
  for (int e = tid; e < m * n; e += nt) {
    int r = e / n, k = e % n;
    int c = order[k];
    double sv = nrm[c];
    U[e] = sv > 0.0 ? A[c * m + r] / sv : 0.0;
  }
  for (int e = tid; e < n * n; e += nt) {
    int r = e / n, k = e % n;
    Vout[e] = V[order[k] * n + r];
  }
}

// ------------------------------------------------------------------ symmetric Jacobi (FP32)
// S: n x n FP64 row-major symmetric.  V (FP64 out, row-major n x n): eigenvectors as columns.
// With t0_dev != null only the trailing block S[t0:, t0:] is diagonalised (t0 read on the
// device) and Vout is the identity outside that block.  With guard != null and *guard == 0
// the kernel returns at once and leaves Vout untouched.  1024 threads per CTA.
// Parallel cyclic (round-robin) ordering: each round rotates n/2 disjoint pairs (p_k, q_k).
// The round's two-sided update A <- J^T A J is done in one pass over 2 x 2 blocks: block
// (k, l) of A (rows p_k, q_k; columns p_l, q_l) becomes R_k B R_l^T.  Only the upper triangle
// of A is kept: element (i, j) lives at (min, max), blocks k <= l cover every upper element
// once, so each is loaded and stored once per round with no mirror store.
// The eigenvector rows are independent under column rotations, so the grid's CTAs each keep a
// full copy of A and a slab of V's rows: every CTA runs the same rotations in the same order
// (no atomics, fixed reduction orders, so their A copies and decisions are bitwise equal) and
// rotates only its own slab, with no communication between CTAs.  Sweeps stop when the
// off-diagonal mass falls below off_tol2 of the total (squared Frobenius norms) -- the FP64
// refinement that follows only needs a start it converges from quadratically.
// Up to n = 160 A is stored as padded rows (n x (n + 1), upper triangle used); above, up to
// n = 256, as the packed upper triangle (n (n + 1) / 2 floats), which fits a CTA's shared memory.
constexpr int JAC_MAX_N_PADDED = 160, JAC_MAX_N = 256;
__device__ __forceinline__ int jac_aidx(bool packed, int i, int j, int n, int ld) {   // i <= j
  return packed ? (i * (2 * n - i - 1)) / 2 + j : i * ld + j;
}
__host__ __device__ constexpr size_t jac_a_floats(bool packed, int n) {
  return packed ? size_t(n) * (n + 1) / 2 : size_t(n) * (n + 1);
}
// blocks per thread: n <= 160: 80 pairs, 3240 blocks <= 4 x 1024; n <= 256: 8256 <= 9 x 1024
template <bool PACKED, int MAXB>
__global__ void __launch_bounds__(1024) k_jacobi_f32(int nfull, const double* __restrict__ S, double* __restrict__ Vout,
                                                     int max_sweeps, const int* __restrict__ t0_dev, float off_tol2,
                                                     const int* __restrict__ guard) {
  extern __shared__ float smf[];
  if (guard && *guard == 0) return;
  const int t0 = t0_dev ? *t0_dev : 0;
  const int n = nfull - t0;
  const int G = gridDim.x, g = blockIdx.x;
  const int tx = threadIdx.x, ty = threadIdx.y, tid = ty * 32 + tx;
  if (t0_dev) {
    for (int i = g + G * ty; i < nfull; i += 32 * G)
      for (int j = tx; j < nfull; j += 32)
        if (i < t0 || j < t0) Vout[size_t(i) * nfull + j] = (i == j) ? 1.0 : 0.0;
  }
  if (n <= 1) {
    if (n == 1 && g == 0 && tid == 0) Vout[size_t(t0) * nfull + t0] = 1.0;
    return;
  }
  const int ld = n + 1;                 // padded rows: column walks are bank-conflict free
  const int np = (n + 1) & ~1;
  const int npairs = np / 2;
  const int nblocks = npairs * (npairs + 1) / 2;
  const int r0 = (g * n) / G, r1 = ((g + 1) * n) / G;   // this CTA's rows of V
  float* A = smf;                       // upper triangle (padded rows or packed)
  float* V = A + jac_a_floats(PACKED, n);   // (r1 - r0) x ld: row i = component r0 + i
  const size_t poff = (jac_a_floats(PACKED, n) + size_t(n / G + 1) * ld + 1) & ~size_t(1);   // 8-byte aligned
  float2* cs = reinterpret_cast<float2*>(smf + poff);
  int2* pq = reinterpret_cast<int2*>(cs + npairs);
  __shared__ float red[2][32];
  for (int i = ty; i < n; i += 32)
    for (int j = i + tx; j < n; j += 32) A[jac_aidx(PACKED, i, j, n, ld)] = float(S[size_t(i + t0) * nfull + (j + t0)]);
  for (int i = ty; i < r1 - r0; i += 32)
    for (int j = tx; j < n; j += 32) V[i * ld + j] = (r0 + i == j) ? 1.0f : 0.0f;
  // this thread's blocks (k, l), k <= l, for blocks e = tid + 1024 b
  int bk[MAXB], bl[MAXB];
#pragma unroll
  for (int b = 0; b < MAXB; ++b) {
    int e = tid + 1024 * b, k = 0;
    bk[b] = -1; bl[b] = -1;
    if (e < nblocks) {
      while (e >= npairs - k) { e -= npairs - k; ++k; }
      bk[b] = k; bl[b] = k + e;
    }
  }
  __syncthreads();
  for (int sweep = 0; sweep < max_sweeps; ++sweep) {
    // convergence test: off-diagonal mass relative to the total (upper triangle counted twice)
    float off = 0.f, dia = 0.f;
    for (int i = ty; i < n; i += 32) {
      for (int j = i + tx; j < n; j += 32) {
        float a = A[jac_aidx(PACKED, i, j, n, ld)];
        if (j == i) dia += a * a; else off += a * a;
      }
    }
    off = warp_sumf(off);
    dia = warp_sumf(dia);
    if (tx == 0) { red[0][ty] = off; red[1][ty] = dia; }
    __syncthreads();
    float offs = 0.f, dias = 0.f;
    for (int i = 0; i < 32; ++i) { offs += red[0][i]; dias += red[1][i]; }
    __syncthreads();
    offs *= 2.f;
    if (!(offs > off_tol2 * (offs + dias))) break;
    for (int r = 0; r < np - 1; ++r) {
      if (tid < npairs) {
        const int k = tid;
        int p, q;
        if (k == 0) { p = r; q = np - 1; }
        else {
          p = r + k; if (p >= np - 1) p -= np - 1;
          q = r - k; if (q < 0) q += np - 1;
        }
        if (p > q) { int t2 = p; p = q; q = t2; }
        float c = 1.f, s = 0.f;
        if (q < n) {
          float apq = A[jac_aidx(PACKED, p, q, n, ld)];
          if (apq != 0.f) {
            float tau = (A[jac_aidx(PACKED, q, q, n, ld)] - A[jac_aidx(PACKED, p, p, n, ld)]) / (2.f * apq);
            float t = copysignf(1.f, tau) / (fabsf(tau) + sqrtf(1.f + tau * tau));
            // correctly rounded sqrt and division: c^2 + s^2 - 1 stays at the rounding level
            // with no bias, so V drifts from orthonormality like a random walk over the
            // ~n sweeps x n rounds of rotations rather than linearly
            c = 1.f / sqrtf(1.f + t * t);
            s = t * c;
          }
        }
        pq[k] = make_int2(p, q);
        cs[k] = make_float2(c, s);
      }
      __syncthreads();
      // A <- J^T A J: block (k, l) = R_k B R_l^T with R = [c -s; s c] acting on (p, q)
#pragma unroll
      for (int b = 0; b < MAXB; ++b) {
        if (bk[b] < 0) break;
        const int k = bk[b], l = bl[b];
        const int2 pq1 = pq[k], pq2 = pq[l];
        const float2 r1v = cs[k], r2v = cs[l];
        const int p1 = pq1.x, q1 = pq1.y, p2 = pq2.x, q2 = pq2.y;
        const float c1 = r1v.x, s1 = r1v.y, c2 = r2v.x, s2 = r2v.y;
        const bool h1 = q1 < n, h2 = q2 < n;   // a pair with q >= n is a lone index (odd n)
        // upper-triangle addresses of (p1, p2), (p1, q2), (q1, p2), (q1, q2); for k == l the
        // two off-diagonal entries are the same element
        const int a00 = p1 <= p2 ? jac_aidx(PACKED, p1, p2, n, ld) : jac_aidx(PACKED, p2, p1, n, ld);
        const int a01 = p1 <= q2 ? jac_aidx(PACKED, p1, q2, n, ld) : jac_aidx(PACKED, q2, p1, n, ld);
        const int a10 = q1 <= p2 ? jac_aidx(PACKED, q1, p2, n, ld) : jac_aidx(PACKED, p2, q1, n, ld);
        const int a11 = q1 <= q2 ? jac_aidx(PACKED, q1, q2, n, ld) : jac_aidx(PACKED, q2, q1, n, ld);
        const float b00 = A[a00];
        const float b01 = h2 ? A[a01] : 0.f;
        const float b10 = h1 ? A[a10] : 0.f;
        const float b11 = (h1 && h2) ? A[a11] : 0.f;
        const float t00 = c1 * b00 - s1 * b10, t01 = c1 * b01 - s1 * b11;
        const float t10 = s1 * b00 + c1 * b10, t11 = s1 * b01 + c1 * b11;
        const float n00 = c2 * t00 - s2 * t01, n01 = s2 * t00 + c2 * t01;
        const float n10 = c2 * t10 - s2 * t11, n11 = s2 * t10 + c2 * t11;
        A[a00] = n00;
        if (h2) A[a01] = n01;
        if (h1 && k != l) A[a10] = n10;
        if (h1 && h2) A[a11] = n11;
      }
      // columns p, q of this CTA's rows of V (independent of the A update): one (pair, row)
      // item per thread, rows fastest
      const int vrows = r1 - r0;
      for (int idx = tid; idx < npairs * vrows; idx += 1024) {
        const int k = idx / vrows, i = idx - k * vrows;
        const int2 pqk = pq[k];
        if (pqk.y >= n) continue;
        const float2 r = cs[k];
        float x = V[i * ld + pqk.x], y = V[i * ld + pqk.y];
        V[i * ld + pqk.x] = r.x * x - r.y * y;
        V[i * ld + pqk.y] = r.y * x + r.x * y;
      }
      __syncthreads();
    }
  }
  for (int i = ty; i < r1 - r0; i += 32)
    for (int j = tx; j < n; j += 32) Vout[size_t(r0 + i + t0) * nfull + (j + t0)] = double(V[i * ld + j]);
}

// First index of the sorted (descending) spectrum below tau * lambda_0; n if none.  Also
// raises a flag when the tail holds at least two eigenvalues and starts before index keep
// (else the refinement level is skipped: a tail made only of discarded vectors needs no
// resolution among its own pairs).
__global__ void k_tail_start(int n, const double* __restrict__ lam, double tau, int keep, int* t0, int* need) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  double top = lam[0];
  int s = n;
  if (top > 0.0) {
    for (int i = 1; i < n; ++i)
      if (lam[i] < tau * top) { s = i; break; }
  }
  *t0 = s;
  *need = (n - s >= 2 && s < keep) ? 1 : 0;
}

// One Ogita-Aishima correction, given XtX, SX = X^T A X (both n x n) and ||A||_F, in three
// short kernels spread over OA_BLOCKS blocks: eigenvalue estimates, the two residual norms
// (partial sums per block, reduced in a fixed order), then E with X <- X + X E.
constexpr int OA_BLOCKS = 64;

__global__ void k_oa_lambda(int n, const double* __restrict__ XtX, const double* __restrict__ SX,
                            double* __restrict__ lam, const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    lam[i] = SX[i * n + i] / XtX[i * n + i];
}

__global__ void __launch_bounds__(256) k_oa_norms(int n, const double* __restrict__ XtX, const double* __restrict__ SX,
                                                  const double* __restrict__ lam, double* __restrict__ part,
                                                  const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  __shared__ double red[32];
  double so = 0.0, ro = 0.0;
  const int64_t nn = int64_t(n) * n;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nn; e += int64_t(gridDim.x) * blockDim.x) {
    int i = int(e / n), j = int(e % n);
    double r = (i == j ? 1.0 : 0.0) - XtX[e];
    double sd = SX[e] - (i == j ? lam[i] : 0.0);
    so += sd * sd;
    ro += r * r;
  }
  so = block_sum(so, red);
  ro = block_sum(ro, red);
  if (threadIdx.x == 0) {
    part[blockIdx.x] = so;
    part[OA_BLOCKS + blockIdx.x] = ro;
  }
}

__global__ void __launch_bounds__(256) k_oa_E(int n, const double* __restrict__ XtX, const double* __restrict__ SX,
                                              const double* __restrict__ lam, const double* __restrict__ part,
                                              const double* __restrict__ anorm_dev, double* __restrict__ E,
                                              const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  double s2 = 0.0, r2 = 0.0;
  for (int i = 0; i < OA_BLOCKS; ++i) {
    s2 += part[i];
    r2 += part[OA_BLOCKS + i];
  }
  const double delta = 2.0 * (sqrt(s2) + (*anorm_dev) * sqrt(r2));
  const int64_t nn = int64_t(n) * n;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < nn; e += int64_t(gridDim.x) * blockDim.x) {
    int i = int(e / n), j = int(e % n);
    double r = (i == j ? 1.0 : 0.0) - XtX[e];
    double val;
    if (i == j) val = 0.5 * r;
    else {
      double d = lam[j] - lam[i];
      val = (fabs(d) > delta) ? (SX[e] + lam[j] * r) / d : 0.5 * r;
    }
    E[e] = val;
  }
}

// Order eigenpairs by decreasing eigenvalue: w[k] = lam[order[k]], V[:, k] = X[:, order[k]].
__global__ void __launch_bounds__(1024) k_sort_eig(int n, const double* __restrict__ lam, const double* __restrict__ X,
                                                   double* __restrict__ w, double* __restrict__ V) {
  extern __shared__ int ord[];
  const int tid = threadIdx.x, nt = blockDim.x;
  for (int c = tid; c < n; c += nt) {
    int rank = 0;
    for (int o = 0; o < n; ++o)
      if (sort_before(lam[o], o, lam[c], c)) ++rank;
    ord[rank] = c;
  }
  __syncthreads();
  for (int k = tid; k < n; k += nt) w[k] = lam[ord[k]];
  for (int e = tid; e < n * n; e += nt) {
    int r = e / n, k = e % n;
    V[e] = X[r * n + ord[k]];
  }
}

__global__ void k_copy_guarded(double* __restrict__ dst, const double* __restrict__ src, int64_t n,
                               const int* __restrict__ guard) {
  if (*guard == 0) return;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    dst[e] = src[e];
}

// Sc = S 2^-e with e = ilogb(max |S_ij|) (0 for a zero or non-finite matrix): a power-of-two
// scaling, exact, that brings the largest entry into [1, 2) so that the FP32 Jacobi and the
// squared norms of the refinement neither underflow nor overflow.  *e_out = e.
__global__ void k_scale_pow2(int64_t n, const double* __restrict__ S, double* __restrict__ Sc, int* e_out, int even) {
  __shared__ double red[32];
  __shared__ int es;
  double m = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, fabs(S[i]));
  for (int off = 16; off > 0; off >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < int(blockDim.x >> 5); ++w) t = fmax(t, red[w]);
    es = (t > 0.0 && isfinite(t)) ? ilogb(t) : 0;
    if (even && (es & 1)) es -= 1;   // largest entry then in [1, 4)
    *e_out = es;
  }
  __syncthreads();
  const int e = es;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) Sc[i] = ldexp(S[i], -e);
}

// Fc = F 2^(-e/2) for the even exponent e of k_scale_pow2.
__global__ void k_scale_pow2_half(int64_t n, const double* __restrict__ F, double* __restrict__ Fc,
                                  const int* __restrict__ e) {
  const int h = *e / 2;
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    Fc[i] = ldexp(F[i], -h);
}

// w[i] *= 2^e
__global__ void k_unscale_pow2(int n, double* __restrict__ w, const int* __restrict__ e) {
  for (int i = threadIdx.x; i < n; i += blockDim.x) w[i] = ldexp(w[i], *e);
}

__global__ void k_frob(int64_t n, const double* __restrict__ x, double* out) {
  __shared__ double red[32];
  double s = 0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s += x[e] * x[e];
  s = block_sum(s, red);
  if (threadIdx.x == 0) *out = sqrt(s);
}

}  // namespace

// Set the dynamic shared-memory limits of the one-CTA kernels up front (before any stream
// capture; they are otherwise set on first use).
static bool g_attr_qr = false, g_attr_svd = false, g_attr_jac = false;
static int g_qr_max_cluster = 0;  // largest cluster the cluster QR may use (0: none)
constexpr size_t QRC_SMEM_LIMIT = 200 * 1024;
void init_kernel_attributes() {
  if (!g_attr_qr) {
    QTT_CUDA(cudaFuncSetAttribute(k_qr, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    QTT_CUDA(cudaFuncSetAttribute(k_qr_cluster, cudaFuncAttributeMaxDynamicSharedMemorySize, int(QRC_SMEM_LIMIT)));
    // 16-CTA clusters are beyond the portable size 8: ask for them, keep them only if a
    // 16-CTA cluster of the largest shared-memory footprint can be resident.
    g_qr_max_cluster = 8;
    if (cudaFuncSetAttribute(k_qr_cluster, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) == cudaSuccess) {
      cudaLaunchConfig_t cfg = {};
      cfg.gridDim = dim3(16);
      cfg.blockDim = dim3(QRC_THREADS);
      cfg.dynamicSmemBytes = QRC_SMEM_LIMIT;
      cudaLaunchAttribute at[1];
      at[0].id = cudaLaunchAttributeClusterDimension;
      at[0].val.clusterDim.x = 16;
      at[0].val.clusterDim.y = 1;
      at[0].val.clusterDim.z = 1;
      cfg.attrs = at;
      cfg.numAttrs = 1;
      int nclusters = 0;
      if (cudaOccupancyMaxActiveClusters(&nclusters, k_qr_cluster, &cfg) == cudaSuccess && nclusters >= 1)
        g_qr_max_cluster = 16;
    }
    cudaGetLastError();
    g_attr_qr = true;
  }
  if (!g_attr_svd) {
    QTT_CUDA(cudaFuncSetAttribute(k_svd_jacobi, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    g_attr_svd = true;
  }
  if (!g_attr_jac) {
    QTT_CUDA(cudaFuncSetAttribute(k_jacobi_f32<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    QTT_CUDA(cudaFuncSetAttribute(k_jacobi_f32<true, 9>, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024));
    g_attr_jac = true;
  }
}

static void copy_guarded(Ctx& c, double* dst, const double* src, int64_t n, const int* guard) {
  int g = int(std::min<int64_t>((n + 255) / 256, 4096));
  k_copy_guarded<<<g, 256, 0, c.stream>>>(dst, src, n, guard);
  after_launch(c, "copy_guarded");
}

static size_t qr_smem(int m, int n) { return (size_t(m) * n + m + std::min(m, n) + 32) * sizeof(double); }

// Column block width and cluster size of the cluster QR for an m x n matrix (cs = 0: use the
// one-CTA kernel).  Panels of at least 4 columns; at most g_qr_max_cluster CTAs.
static void qr_cluster_shape(int m, int n, int& nb, int& cs) {
  nb = 0;
  cs = 0;
  if (m < n || n < 16 || g_qr_max_cluster < 2) return;
  int b = std::max(4, (n + g_qr_max_cluster - 1) / g_qr_max_cluster);
  int k = (n + b - 1) / b;
  if (k < 2 || b > 16 || qrc_smem_doubles(m, b) * sizeof(double) > QRC_SMEM_LIMIT) return;
  nb = b;
  cs = k;
}

bool qr_fits(int m, int n) {
  init_kernel_attributes();
  int nb = 0, cs = 0;
  qr_cluster_shape(m, n, nb, cs);
  return cs > 0 || qr_smem(m, n) <= 220 * 1024;
}

void qr(Ctx& c, int count, int m, int n, int trans, const double* A, int64_t in_stride, double* Q, int64_t q_stride,
        double* R, int64_t r_stride, int path) {
  DigitsScope fp64(c, kDigitsFP64);   // the decompositions and their refinement products stay FP64
  if (count <= 0 || n <= 0 || m <= 0) return;
  init_kernel_attributes();
  int kk = std::min(m, n);
  int nb = 0, cs = 0;
  if (path != 1) qr_cluster_shape(m, n, nb, cs);
  if (path == 2 && cs == 0)
    throw Error(QTT_ERR_UNSUPPORTED, "qr: no cluster shape for " + std::to_string(m) + "x" + std::to_string(n));
  ProfScope ps(c, KC_QR, double(count) * 8.0 * (double(m) * n * kk - 0.5 * (double(m) + n) * kk * kk + kk * kk * kk / 3.0));
  if (cs > 0) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(unsigned(count) * unsigned(cs));
    cfg.blockDim = dim3(QRC_THREADS);
    cfg.dynamicSmemBytes = qrc_smem_doubles(m, nb) * sizeof(double);
    cfg.stream = c.stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = unsigned(cs);
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    QTT_CUDA(cudaLaunchKernelEx(&cfg, k_qr_cluster, m, n, nb, trans, A, Q, R, in_stride, q_stride, r_stride));
    after_launch(c, "qr_cluster");
    return;
  }
  size_t sm = qr_smem(m, n);
  if (sm > 220 * 1024)
    throw Error(QTT_ERR_UNSUPPORTED, "qr: matrix " + std::to_string(m) + "x" + std::to_string(n) + " too large for one CTA");
  k_qr<<<count, 256, sm, c.stream>>>(m, n, trans, A, Q, R, in_stride, q_stride, r_stride);
  after_launch(c, "qr");
}

void check_recip(Ctx& c, int n, const double* x_dev, double* err_dev) {
  k_check_recip<<<1, 256, 0, c.stream>>>(n, x_dev, err_dev);
  after_launch(c, "check_recip");
}

// Accurate SVD of small matrices: G (m x n, m >= n) = U diag(s) V^T.
void svd_small(Ctx& c, int m, int n, const double* G, double* U, double* s, double* V) {
  DigitsScope fp64(c, kDigitsFP64);   // the decompositions and their refinement products stay FP64
  QTT_CHECK_ARG(m >= n, "svd: needs m >= n");
  size_t sm = (size_t(m) * n + size_t(n) * n + n) * sizeof(double) + n * sizeof(int);
  if (sm > 220 * 1024) throw Error(QTT_ERR_UNSUPPORTED, "svd: matrix too large for one CTA");
  init_kernel_attributes();
  k_svd_jacobi<<<1, 256, sm, c.stream>>>(m, n, G, U, s, V, 60);
  after_launch(c, "svd_jacobi");
}

static void oa_update(Ctx& c, int n, const double* XtX, const double* SX, const double* an, double* E, double* lam,
                      double* part, const int* guard) {
  k_oa_lambda<<<1, 256, 0, c.stream>>>(n, XtX, SX, lam, guard);
  after_launch(c, "oa_lambda");
  k_oa_norms<<<OA_BLOCKS, 256, 0, c.stream>>>(n, XtX, SX, lam, part, guard);
  after_launch(c, "oa_norms");
  k_oa_E<<<OA_BLOCKS, 256, 0, c.stream>>>(n, XtX, SX, lam, part, an, E, guard);
  after_launch(c, "oa_E");
}

// One Newton-Schulz step X <- X (3 I - X^T X) / 2 (squares ||X^T X - I||); honours c.guard.
static void newton_schulz(Ctx& c, int n, double* X, double* XtX, double* AX) {
  gemm(c, 1, n, n, n, 1.0, X, 0, 1, n, X, 0, n, 1, 0.0, XtX, 0, n, 1);
  gemm(c, 1, n, n, n, 1.0, X, 0, n, 1, XtX, 0, n, 1, 0.0, AX, 0, n, 1);
  axpby(c, int64_t(n) * n, -0.5, AX, 1.5, X);
}

// X^T S X into SX (n x n).  With a factor F (m x n row-major, S = F^T F) it is formed as
// (F X)^T (F X): each entry then carries an error relative to the product of the norms of its
// two columns of F X, not to ||S||, so pairs far down the spectrum keep their relative
// accuracy (the squared form resolves nothing below ~eps ||S||).  FX: m x n scratch.
static void xtsx(Ctx& c, int n, const double* S, const double* F, int m, const double* X, double* AX, double* FX,
                 double* SX) {
  if (F) {
    gemm(c, 1, m, n, n, 1.0, F, 0, n, 1, X, 0, n, 1, 0.0, FX, 0, n, 1);   // F X
    gemm(c, 1, n, n, m, 1.0, FX, 0, 1, n, FX, 0, n, 1, 0.0, SX, 0, n, 1); // (F X)^T (F X)
  } else {
    gemm(c, 1, n, n, n, 1.0, S, 0, n, 1, X, 0, n, 1, 0.0, AX, 0, n, 1);   // S X
    gemm(c, 1, n, n, n, 1.0, X, 0, 1, n, AX, 0, n, 1, 0.0, SX, 0, n, 1);  // X^T S X
  }
}

// One Ogita-Aishima iteration on X (n x n) for the symmetric S (or S = F^T F, see xtsx).
static void oa_iteration(Ctx& c, int n, const double* S, const double* F, int m, double* X, double* XtX, double* AX,
                         double* FX, double* SX, double* E, double* lam, const double* an, double* part) {
  gemm(c, 1, n, n, n, 1.0, X, 0, 1, n, X, 0, n, 1, 0.0, XtX, 0, n, 1);   // X^T X
  xtsx(c, n, S, F, m, X, AX, FX, SX);
  oa_update(c, n, XtX, SX, an, E, lam, part, c.guard);
  gemm(c, 1, n, n, n, 1.0, X, 0, n, 1, E, 0, n, 1, 0.0, AX, 0, n, 1);    // X E
  axpby(c, int64_t(n) * n, 1.0, AX, 1.0, X);
}

// Symmetric eigendecomposition to FP64 accuracy (absolute error ~ eps_64 ||S||) from FP32
// Jacobi sweeps: level 1 diagonalises S in FP32 and refines all pairs in FP64 (Ogita-Aishima);
// eigenvalues closer than the FP32 resolution (~1e-7 ||S||) stay lumped in a cluster, so
// levels 2 to 5 re-diagonalise the trailing block of X^T S X (the eigenvalues below 1e-3,
// 1e-6, 1e-9 and 1e-12 of the largest) on its own scale and refine again.  Levels with fewer
// than two tail eigenvalues are skipped on the device.  The levels are three decades apart:
// a pair just above a level's threshold tau has a gap of order tau times its relative
// spacing, while its coupling after the previous level is at that level's FP32 resolution
// (~1e-7 of the previous threshold), so the refinement starts from vector errors of ~1e-4 or
// less even for log-evenly spaced spectra; with levels five decades apart, spectra with ~10 %
// relative spacing between neighbours were left with eigenvalue errors near 1e-6 ||S||.
// Each tail level starts with one Newton-Schulz step on X: the last refinement of a level can
// take a large first-order step for a tail pair that the level could not yet resolve (its
// Rayleigh quotients drift apart by more than the threshold while their coupling is still at
// the previous level's FP32 resolution), which leaves X^T X - I near 1e-3.  The tail block of
// X^T S X is a Rayleigh-Ritz projection only for an orthonormal X; with X^T X - I at 1e-3 the
// re-diagonalised tail pairs keep couplings of ~1e-3 of their scale, and the same large step
// recurs in the next level's last refinement, where nothing repairs it.
// FP32 Jacobi stopping thresholds (squared off-diagonal mass over squared total) before the
// level-0 and the tail-level refinements.
#ifndef QTT_JAC_TOL2_FULL
#define QTT_JAC_TOL2_FULL 1e-12f
#endif
#ifndef QTT_JAC_TOL2_TAIL
#define QTT_JAC_TOL2_TAIL 1e-12f
#endif
#ifndef QTT_JAC_CTAS
#define QTT_JAC_CTAS 8
#endif
constexpr float JAC_TOL2_FULL = QTT_JAC_TOL2_FULL;
constexpr float JAC_TOL2_TAIL = QTT_JAC_TOL2_TAIL;

void eigh(Ctx& c, int n, const double* S, double* w, double* V, int keep, const double* F, int m) {
  DigitsScope fp64(c, kDigitsFP64);   // the decompositions and their refinement products stay FP64
  QTT_CHECK_ARG(n >= 1, "eigh: n >= 1");
  if (keep <= 0 || keep > n) keep = n;
  if (n > JAC_MAX_N) throw Error(QTT_ERR_UNSUPPORTED, "eigh: n > 256 not supported");
  const bool packed = n > JAC_MAX_N_PADDED;
  QTT_CHECK_ARG(!F || m >= 1, "eigh: factor needs m >= 1 rows");
  // FP32 Jacobi: QTT_JAC_CTAS CTAs share the eigenvector rows for the larger matrices (each
  // keeps all of A; 8: 16 rows each at n = 128)
  const int jac_ctas = n >= 64 ? QTT_JAC_CTAS : 1;
  const size_t npairs = size_t((n + 1) & ~1) / 2;
  const size_t smf = ((jac_a_floats(packed, n) + size_t(n / jac_ctas + 1) * (n + 1) + 1) & ~size_t(1)) * sizeof(float) +
                     npairs * (sizeof(float2) + sizeof(int2));
  auto jacobi = packed ? k_jacobi_f32<true, 9> : k_jacobi_f32<false, 4>;
  init_kernel_attributes();
  const size_t nn = size_t(n) * n;
  DBuf X(&c, nn), Xs(&c, nn), XtX(&c, nn), AX(&c, nn), SX(&c, nn), E(&c, nn), Y(&c, nn), lam(&c, size_t(n)),
      an(&c, 1), flags(&c, 2), part(&c, 2 * OA_BLOCKS), Ssc(&c, nn), FX(&c, F ? size_t(m) * n : 1),
      Fsc(&c, F ? size_t(m) * n : 1);
  int* t0 = reinterpret_cast<int*>(flags.p);
  int* need = t0 + 1;
  // work on S 2^-e (largest entry in [1, 2)): Gram matrices of small-norm trains (e.g. a field
  // held at zero with 1e-8 padding, norms ~1e-96) would otherwise vanish in FP32 and in the
  // squared norms of the refinement; the eigenvalues are scaled back at the end
  DBuf escale(&c, 1);
  int* eexp = reinterpret_cast<int*>(escale.p);
  k_scale_pow2<<<1, 1024, 0, c.stream>>>(int64_t(nn), S, Ssc.p, eexp, F ? 1 : 0);
  after_launch(c, "scale_pow2");
  S = Ssc.p;
  if (F) {   // F 2^(-e/2) with e even, so that (F X)^T (F X) is on the scale of S 2^-e
    k_scale_pow2_half<<<unsigned(std::min<int64_t>((int64_t(m) * n + 255) / 256, 1024)), 256, 0, c.stream>>>(int64_t(m) * n, F, Fsc.p, eexp);
    after_launch(c, "scale_pow2_half");
    F = Fsc.p;
  }
  {
    ProfScope ps(c, KC_EIG);
    jacobi<<<jac_ctas, dim3(32, 32), smf, c.stream>>>(n, S, X.p, packed ? 14 : 10, nullptr, JAC_TOL2_FULL, nullptr);
    after_launch(c, "jacobi_f32");
  }

  k_frob<<<1, 1024, 0, c.stream>>>(int64_t(n) * n, S, an.p);
  after_launch(c, "frob");
  // levels three decades apart in the eigenvalue; with a factor F the products resolve the
  // tail to its own scale, and levels continue down to 1e-27 of the largest (singular values of
  // F down to ~3e-14 of the largest), where the cut of a weakly truncated rounding can fall
  const double taus[10] = {0.0, 1e-3, 1e-6, 1e-9, 1e-12, 1e-15, 1e-18, 1e-21, 1e-24, 1e-27};
  const int kLevels = F ? 10 : 5;
  for (int level = 0; level < kLevels; ++level) {
    if (level > 0) {
      k_tail_start<<<1, 1, 0, c.stream>>>(n, lam.p, taus[level], keep, t0, need);
      after_launch(c, "tail_start");
      c.guard = need;
      newton_schulz(c, n, X.p, XtX.p, AX.p);
      xtsx(c, n, S, F, m, X.p, AX.p, FX.p, SX.p);
      c.guard = nullptr;
      {
        ProfScope ps(c, KC_EIG);
        jacobi<<<jac_ctas, dim3(32, 32), smf, c.stream>>>(n, SX.p, Y.p, packed ? 10 : 8, t0, JAC_TOL2_TAIL, need);
        after_launch(c, "jacobi_f32_tail");
      }
      c.guard = need;
      gemm(c, 1, n, n, n, 1.0, X.p, 0, n, 1, Y.p, 0, n, 1, 0.0, AX.p, 0, n, 1);
      copy_guarded(c, X.p, AX.p, int64_t(nn), need);
    }
    for (int it = 0; it < (level == 0 ? 3 : 2); ++it)
      oa_iteration(c, n, S, F, m, X.p, XtX.p, AX.p, FX.p, SX.p, E.p, lam.p, an.p, part.p);
    // eigenvalue estimates of the refined vectors, then sort (descending); a skipped level
    // leaves X and lam as they were, and the sort is then the identity
    gemm(c, 1, n, n, n, 1.0, X.p, 0, 1, n, X.p, 0, n, 1, 0.0, XtX.p, 0, n, 1);
    xtsx(c, n, S, F, m, X.p, AX.p, FX.p, SX.p);
    oa_update(c, n, XtX.p, SX.p, an.p, E.p, lam.p, part.p, c.guard);
    c.guard = nullptr;
    k_sort_eig<<<1, 1024, n * sizeof(int), c.stream>>>(n, lam.p, X.p, w, Xs.p);
    after_launch(c, "sort_eig");
    copy(c, X.p, Xs.p, int64_t(nn));
    copy(c, lam.p, w, n);
  }
  // Two Newton-Schulz steps: the first-order orthonormalisation of the refinement leaves
  // ~eps ||S|| / gap in X^T X - I for close pairs; each step squares it.
  for (int it = 0; it < 2; ++it) newton_schulz(c, n, X.p, XtX.p, AX.p);
  copy(c, V, X.p, int64_t(nn));
  k_unscale_pow2<<<1, 256, 0, c.stream>>>(n, w, eexp);
  after_launch(c, "unscale_pow2");
}

}  // namespace qtt
