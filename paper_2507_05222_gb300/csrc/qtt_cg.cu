// Local CG solve of one ALS site (Sec. II.A.4) as ONE cooperative kernel.
//
// The ALS local system at site k is A_loc x = b with
//     (A_loc x)[c, s, e] = sum_{w, a, t, v, b} L[c, w, a] x[a, t, b] W[w, s, t, v] R[e, v, b]
// (L, R: operator environments of the current sweep, W: the operator's core k).  Launching
// the three contractions and the CG vector updates one kernel at a time costs ~8 dependent
// launches per iteration; on GB300 a dependent FP64 instruction also costs ~64 cycles, so every
// launch pays a long serial tail.  Here the whole solve -- the initial residual and up to
// `iters` CG iterations -- runs in one grid of one CTA per SM, stages separated by a grid
// barrier:
//   A  T2[c, s, v, b] = sum_{w,t} (sum_a L[c, w, a] P[a, t, b]) W[w, s, t, v]
//      work item (c, block of b): L[c] and P[:, :, block] staged in shared memory;
//   B  out[c, s, e] = sum_{v,b} T2[c, s, v, b] R[e, v, b]   (+ the block's share of P . out)
//      work item (row (c, s), block of 16 e), 16 threads per output over K = w1 r1;
//   C  alpha = rr / pAp; x += alpha p; r -= alpha Ap; partial r.r
//   D  beta = rr' / rr; p = r + beta p; stopping test.
// The CG is the textbook one (Hestenes-Stiefel), with the same stopping rule and iteration
// count as the per-kernel path: stop once r.r <= tol^2 b.b, or when p.Ap is not positive.
// Every block sums the per-block partials in the same fixed order, so all blocks take the same
// decisions and results are deterministic.
//
// Barrier: an arrival counter in device memory (reset before the launch); a waiting block polls
// it for at most the context's wait limit (2 s unless set otherwise; global timer).  The
// cooperative launch makes every block resident, so the bound is only a safety net: on expiry
// the block sets the error flag,
// every block leaves at its next barrier, and the iteration count is overwritten with a
// negative value that the host turns into an error.  Data written by other blocks inside the
// kernel are read with ld.global.cg (L2).
#include <algorithm>

#include "qtt_algebra.h"
#include "qtt_ozaki_dev.cuh"

namespace qtt {

namespace {

constexpr int CGP_THREADS = 256;
constexpr int CGP_MAX_BOND = 128;
constexpr int CGP_MAX_W = 16;
constexpr int CGP_MAX_D = 4;

struct CgBar {
  unsigned int count;   // arrivals so far (monotonic within a launch)
  int error;            // set by a block that gave up waiting
  unsigned long long limit_ns;   // how long a block waits at one barrier (the context's wait limit)
};

struct CgArgs {
  int r0, r1, w0, w1, d, bt, iters;
  int eb, ch;     // stage B: e-block width (16, 8, 4, 2 or 1) and T2 row chunks per load
  const double* tol;   // relative tolerance (device scalar, read at launch)
  const double* L;
  const double* W;
  const double* R;
  const double* b;
  double* x;
  double* r;
  double* p;      // 2 x (r0 d r1): directions of even and odd iterations
  double* Ap;
  double* T2;
  double* part;   // 4 x gridDim.x
  const double* dinv;  // diagonal preconditioner (inverse of the local matrix's diagonal; may be null)
  CgBar* bar;
  int* total;     // += iterations done (may be null)
  double* flops;  // += (iterations + 1) * fpi when profiling (may be null)
  double fpi;     // flops of one operator application
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

// Barrier state before a launch: no arrivals, no error, the context's wait limit.
__global__ void k_bar_init(CgBar* b, unsigned long long limit_ns) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    b->count = 0;
    b->error = 0;
    b->limit_ns = limit_ns;
  }
}

__device__ __forceinline__ void red_release_add(unsigned int* p, unsigned int v) {
  asm volatile("red.release.gpu.global.add.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Grid barrier on a monotonic arrival counter: barrier number k completes when the counter
// reaches k * gridDim.x.  Returns false (in every thread of the block) once any block gave up.
__device__ bool grid_sync(CgBar* bar, unsigned int& target, int* flag) {
  target += gridDim.x;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    red_release_add(&bar->count, 1u);
    const unsigned long long t0 = global_ns();
    unsigned int spins = 0;
    const unsigned long long limit = bar->limit_ns;
    // limits below 0.1 ms (tests of the timeout path) are checked at every poll
    const unsigned int mask = limit < 100000ull ? 0u : 255u;
    while (ld_acquire(&bar->count) < target) {
      if ((++spins & mask) == 0u) {
        if (ld_volatile(&bar->error)) break;
        if (global_ns() - t0 > limit) {
          atomicExch(&bar->error, 1);
          break;
        }
      }
    }
    __threadfence();
    *flag = ld_volatile(&bar->error);
  }
  __syncthreads();
  return *flag == 0;
}

__device__ double block_reduce(double v, double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  double s = 0.0;
  for (int i = 0; i < nw; ++i) s += red[i];
  __syncthreads();
  return s;
}

// Sum of the gridDim.x partials part[0..G) in a fixed order (identical in every block).
__device__ double sum_partials(const double* part, double* red) {
  const int G = gridDim.x;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int i = threadIdx.x; i < G; i += 32) s += __ldcg(part + i);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) red[0] = s;
  }
  __syncthreads();
  const double s = red[0];
  __syncthreads();
  return s;
}

// Preconditioned residual z = D^-1 r at element g (z = r without a preconditioner); every place
// that forms z uses this one expression, so the values agree bit for bit.
__device__ __forceinline__ double zval(const double* dinv, const double* r, size_t g) {
  return dinv ? __ldg(dinv + g) * __ldcg(r + g) : __ldcg(r + g);
}

// Stage A: T2 = (L . P) . W, with P the vector P0 or, when Rv is given, P = z(Rv) + beta P0 formed
// on the fly (the CG direction update, computed exactly as its owners store it).
__device__ void stage_a(const CgArgs& a, const double* P0, const double* Rv, double beta, double* sL, double* sW,
                        double* sP, double* sT1) {
  const int r0 = a.r0, r1 = a.r1, w0 = a.w0, w1 = a.w1, d = a.d, bt = a.bt;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int nblk = (r1 + bt - 1) / bt;
  const int items = r0 * nblk;
  for (int item = blockIdx.x; item < items; item += gridDim.x) {
    const int c = item / nblk, b0 = (item % nblk) * bt, bw = min(bt, r1 - b0);
    for (int e = tid; e < w0 * r0; e += nt) sL[e] = __ldg(a.L + size_t(c) * w0 * r0 + e);
    // rows (a, t) of the P block, one warp per row and one lane per b (bt <= 32): coalesced,
    // no index division
    const int lane = tid & 31, warp = tid >> 5, nwarps = nt >> 5;
    if (lane < bw) {
#pragma unroll 4
      for (int row = warp; row < r0 * d; row += nwarps) {
        const size_t g = size_t(row) * r1 + b0 + lane;
        sP[row * bt + lane] = Rv ? fma(beta, __ldcg(P0 + g), zval(a.dinv, Rv, g)) : __ldcg(P0 + g);
      }
    }
    __syncthreads();
    for (int e = tid; e < w0 * d * bw; e += nt) {
      const int w = e / (d * bw), rem = e % (d * bw), t = rem / bw, bb = rem % bw;
      const double* lw = sL + w * r0;
      const double* pc = sP + t * bt + bb;
      double s = 0.0;
      for (int aa = 0; aa < r0; ++aa) s = fma(lw[aa], pc[aa * d * bt], s);
      sT1[(w * d + t) * bt + bb] = s;
    }
    __syncthreads();
    for (int e = tid; e < d * w1 * bw; e += nt) {
      const int s_ = e / (w1 * bw), rem = e % (w1 * bw), v = rem / bw, bb = rem % bw;
      double acc = 0.0;
      for (int w = 0; w < w0; ++w)
        for (int t = 0; t < d; ++t) acc = fma(sT1[(w * d + t) * bt + bb], sW[((w * d + s_) * d + t) * w1 + v], acc);
      a.T2[((size_t(c) * d + s_) * w1 + v) * r1 + b0 + bb] = acc;
    }
    __syncthreads();
  }
}

// Stage B: out = T2 . R^T; returns this block's share of P . out (0 if P is null).
// Block j works on the e-block j % NE (EB consecutive e, its rows of R staged in sR once per
// solve) and on the row chunks (RB rows each) j / NE, j / NE + NRG, ...; the T2 rows of up to
// CH chunks are loaded together (one L2 latency), then 16 outputs x 16 lanes per pass.
__device__ double stage_b(const CgArgs& a, const double* P, double* out, const double* sR, double* sT2) {
  const int r1 = a.r1, EB = a.eb, RB = 16 / a.eb, K = a.w1 * r1, Kp = K + 1;
  const int rows = a.r0 * a.d;
  const int NE = (r1 + EB - 1) / EB, NRG = gridDim.x / NE;
  const int eb = blockIdx.x % NE, rg = blockIdx.x / NE;
  const int tid = threadIdx.x, nt = blockDim.x;
  const int o = tid >> 4, l = tid & 15, i = o / EB, eo = o % EB;
  const int e = eb * EB + eo;
  double dot = 0.0;
  if (rg >= NRG) return dot;
  const int nchunks = (rows + RB - 1) / RB;
  for (int c0 = rg; c0 < nchunks; c0 += NRG * a.ch) {
    // load the T2 rows of chunks c0, c0 + NRG, ... (at most ch chunks)
    int nch = 0;
    for (int cc = c0; cc < nchunks && nch < a.ch; cc += NRG, ++nch) {
      const int row0 = cc * RB, nr = min(RB, rows - row0);
      const double* src = a.T2 + size_t(row0) * K;
      double* dst = sT2 + size_t(nch) * RB * K;
      for (int x = tid; x < nr * K; x += nt) dst[x] = __ldcg(src + x);
    }
    __syncthreads();
    for (int q = 0; q < nch; ++q) {
      const int row = (c0 + q * NRG) * RB + i;
      double s = 0.0;
      const bool ok = row < rows && e < r1;
      if (ok) {
        const double* t2 = sT2 + (size_t(q) * RB + i) * K;
        const double* rr = sR + size_t(eo) * Kp;
        for (int k = l; k < K; k += 16) s = fma(t2[k], rr[k], s);
      }
      for (int off = 8; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      if (ok && l == 0) {
        out[size_t(row) * r1 + e] = s;
        if (P) dot = fma(__ldcg(P + size_t(row) * r1 + e), s, dot);
      }
    }
    __syncthreads();
  }
  return dot;
}

// Written to *total when a barrier timed out; the host treats a negative count as a failed solve.
constexpr int CGP_POISON = -(1 << 29);

__global__ void __launch_bounds__(CGP_THREADS, 2) k_cg_persistent(CgArgs a) {
  extern __shared__ double sm[];
  const int r0 = a.r0, w0 = a.w0, w1 = a.w1, d = a.d, bt = a.bt;
  const int G = gridDim.x, tid = threadIdx.x, nt = blockDim.x;
  const int64_t nel = int64_t(r0) * d * a.r1;
  const int K = w1 * a.r1;
  double* sL = sm;                           // w0 x r0
  double* sW = sL + w0 * r0;                 // w0 x d x d x w1
  double* sP = sW + w0 * d * d * w1;         // r0 x d x bt
  double* sT1 = sP + r0 * d * bt;            // w0 x d x bt
  double* sR = sT1 + w0 * d * bt;            // eb x (K + 1): this block's rows of R
  double* sT2 = sR + size_t(a.eb) * (K + 1); // ch x (16 / eb) x K
  __shared__ double red[32];
  __shared__ int flag;
  unsigned int target = 0;
  double* part_pap = a.part;
  double* part_rr = a.part + G;
  double* part_bb = a.part + 2 * G;
  double* part_rz = a.part + 3 * G;
  for (int e = tid; e < w0 * d * d * w1; e += nt) sW[e] = __ldg(a.W + e);
  {
    const int NE = (a.r1 + a.eb - 1) / a.eb, e0 = (blockIdx.x % NE) * a.eb;
    for (int x = tid; x < a.eb * K; x += nt) {
      const int eo = x / K, k = x - eo * K;
      sR[size_t(eo) * (K + 1) + k] = (e0 + eo < a.r1) ? __ldg(a.R + size_t(e0 + eo) * K + k) : 0.0;
    }
  }
  __syncthreads();

  // ---- initial residual: r = b - A x, p_0 = r
  // The directions alternate between the two halves of a.p: p_it lives in half it & 1.
  bool ok = true;
  int count = 0;
  do {
    stage_a(a, a.x, nullptr, 0.0, sL, sW, sP, sT1);
    if (!(ok = grid_sync(a.bar, target, &flag))) break;
    stage_b(a, nullptr, a.Ap, sR, sT2);
    if (!(ok = grid_sync(a.bar, target, &flag))) break;
    double rr_p = 0.0, bb_p = 0.0, rz_p = 0.0;
    for (int64_t e = int64_t(blockIdx.x) * nt + tid; e < nel; e += int64_t(G) * nt) {
      const double be = __ldg(a.b + e);
      const double re = be - __ldcg(a.Ap + e);
      const double ze = a.dinv ? __ldg(a.dinv + e) * re : re;
      a.r[e] = re;
      a.p[e] = ze;
      rr_p = fma(re, re, rr_p);
      rz_p = fma(re, ze, rz_p);
      bb_p = fma(be, be, bb_p);
    }
    rr_p = block_reduce(rr_p, red);
    rz_p = block_reduce(rz_p, red);
    bb_p = block_reduce(bb_p, red);
    if (tid == 0) {
      part_rr[blockIdx.x] = rr_p;
      part_rz[blockIdx.x] = rz_p;
      part_bb[blockIdx.x] = bb_p;
    }
    if (!(ok = grid_sync(a.bar, target, &flag))) break;
    double rr = sum_partials(part_rr, red);
    double rz = sum_partials(part_rz, red);
    const double bb = sum_partials(part_bb, red);
    const double tol2 = __ldg(a.tol) * __ldg(a.tol);
    bool active = rr > tol2 * bb && rr > 0.0;
    double beta = 0.0;
    // Three barriers per iteration: after A (T2 and p_it complete), after B (Ap and the p.Ap
    // partials), after C (x, r and the r.r partials).  part_rr is read at the top of an
    // iteration and rewritten only in its stage C, two barriers later.
    for (int it = 0; it < a.iters && active; ++it) {
      double* pn = a.p + (it & 1) * nel;
      const double* po = a.p + ((it & 1) ^ 1) * nel;
      if (it == 0) {
        stage_a(a, pn, nullptr, 0.0, sL, sW, sP, sT1);
      } else {
        for (int64_t e = int64_t(blockIdx.x) * nt + tid; e < nel; e += int64_t(G) * nt)
          pn[e] = fma(beta, po[e], zval(a.dinv, a.r, e));
        stage_a(a, po, a.r, beta, sL, sW, sP, sT1);
      }
      if (!(ok = grid_sync(a.bar, target, &flag))) break;
      double pap_p = stage_b(a, pn, a.Ap, sR, sT2);
      pap_p = block_reduce(pap_p, red);
      if (tid == 0) part_pap[blockIdx.x] = pap_p;
      if (!(ok = grid_sync(a.bar, target, &flag))) break;
      const double pap = sum_partials(part_pap, red);
      if (!(pap > 0.0)) break;                       // same decision in every block
      const double alpha = rz / pap;
      double rn_p = 0.0, rzn_p = 0.0;
      for (int64_t e = int64_t(blockIdx.x) * nt + tid; e < nel; e += int64_t(G) * nt) {
        a.x[e] += alpha * pn[e];
        const double re = a.r[e] - alpha * __ldcg(a.Ap + e);
        a.r[e] = re;
        rn_p = fma(re, re, rn_p);
        rzn_p = fma(re, a.dinv ? __ldg(a.dinv + e) * re : re, rzn_p);
      }
      rn_p = block_reduce(rn_p, red);
      rzn_p = block_reduce(rzn_p, red);
      if (tid == 0) {
        part_rr[blockIdx.x] = rn_p;
        part_rz[blockIdx.x] = rzn_p;
      }
      if (!(ok = grid_sync(a.bar, target, &flag))) break;
      const double rn = sum_partials(part_rr, red);
      const double rzn = sum_partials(part_rz, red);
      beta = rzn / rz;
      rr = rn;
      rz = rzn;
      count += 1;
      active = rn > tol2 * bb && rn > 0.0;
    }
  } while (false);
  if (blockIdx.x == 0 && tid == 0 && a.total) {
    if (ok) *a.total += count;
    else *a.total = CGP_POISON;
  }
  if (blockIdx.x == 0 && tid == 0 && a.flops && ok) atomicAdd(a.flops, (count + 1) * a.fpi);
}

// Stage-A block of b.  Per work item the CTA does bt r0 w0 d FP64 FMAs at the SM's 2 per cycle,
// and never less than one dependent chain of r0 FMAs (~64 cycles each) per pass of its 256
// threads; items are dealt to the G CTAs round by round.  Larger blocks win ties.
int choose_bt(int r0, int r1, int w0, int d, int G) {
  int best = 32;
  double best_cost = 1e300;
  for (int bt : {32, 16, 8}) {
    const int items = r0 * ((r1 + bt - 1) / bt);
    const int rounds = (items + G - 1) / G;
    const double thr = 0.5 * double(bt) * r0 * w0 * d;
    const double lat = double((w0 * d * bt + CGP_THREADS - 1) / CGP_THREADS) * r0 * 64.0;
    const double cost = rounds * std::max(thr, lat);
    if (cost < best_cost * (1.0 - 1e-9)) {
      best_cost = cost;
      best = bt;
    }
  }
  return best;
}

// Shared memory of one block at most 110 KiB, so that two blocks fit an SM.
constexpr size_t CGP_SMEM_LIMIT = 110 * 1024;

struct CgPlan {
  int G, bt, eb, ch;
  size_t smem;
};

// Grid, stage-A block, stage-B e-block and chunking, shared memory; false if the solve does not
// fit this kernel (the caller then launches one kernel per stage).
bool cg_plan(const Ctx& c, int r0, int r1, int w0, int w1, int d, CgPlan& p) {
  if (!(r0 >= 1 && r1 >= 1 && r0 <= CGP_MAX_BOND && r1 <= CGP_MAX_BOND && w0 >= 1 && w1 >= 1 && w0 <= CGP_MAX_W &&
        w1 <= CGP_MAX_W && d >= 1 && d <= CGP_MAX_D))
    return false;
  // The cooperative launch needs every block resident.  The caller's own stream gets one CTA
  // per SM; a worker stream (two solves may run concurrently, next to short-lived kernels of
  // other streams) gets half the SMs, so that two persistent grids never hold more than one of
  // the two slots per SM that this kernel's register and shared-memory budget leaves.
  p.G = (&c == c.root) ? c.num_sms : std::max(1, c.num_sms / 2);
  const int K = w1 * r1;
  int eb = 16;
  while (eb > 1 && size_t(eb) * (K + 1) * sizeof(double) > 64 * 1024) eb >>= 1;
  const int NE = (r1 + eb - 1) / eb;
  if (NE > p.G) return false;
  const int NRG = p.G / NE, RB = 16 / eb, rows = r0 * d;
  const int nchunks = (rows + RB - 1) / RB;
  p.bt = choose_bt(r0, r1, w0, d, p.G);
  const size_t base = size_t(w0) * r0 + size_t(w0) * d * d * w1 + size_t(r0) * d * p.bt + size_t(w0) * d * p.bt +
                      size_t(eb) * (K + 1);
  const size_t per_ch = size_t(RB) * K;
  const size_t budget = CGP_SMEM_LIMIT / sizeof(double);
  if (base + per_ch > budget) return false;
  p.eb = eb;
  p.ch = int(std::min<size_t>((nchunks + NRG - 1) / NRG, (budget - base) / per_ch));
  p.smem = (base + size_t(p.ch) * per_ch) * sizeof(double);
  return true;
}

}  // namespace

static int g_cgp_per_sm = -1;

void cg_init_attributes() {
  if (g_cgp_per_sm >= 0) return;
  QTT_CUDA(cudaFuncSetAttribute(k_cg_persistent, cudaFuncAttributeMaxDynamicSharedMemorySize, int(CGP_SMEM_LIMIT)));
  int per_sm = 0;
  QTT_CUDA(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_persistent, CGP_THREADS, CGP_SMEM_LIMIT));
  g_cgp_per_sm = per_sm;
}

bool cg_persistent_fits(const Ctx& c, int r0, int r1, int w0, int w1, int d) {
  cg_init_attributes();
  CgPlan p;
  return g_cgp_per_sm >= 2 && cg_plan(c, r0, r1, w0, w1, d, p);
}

void cg_persistent(Ctx& c, const double* L, const double* W, const double* R, const double* b, double* x, int r0,
                   int r1, int w0, int w1, int d, int iters, const double* tol_dev, int* total_dev,
                   const double* dinv) {
  CgPlan pl;
  QTT_CHECK_ARG(cg_plan(c, r0, r1, w0, w1, d, pl), "cg_persistent: shape outside the supported range");
  cg_init_attributes();
  if (g_cgp_per_sm < 2) throw Error(QTT_ERR_UNSUPPORTED, "cg_persistent: fewer than two blocks fit an SM");
  const int G = pl.G, bt = pl.bt;
  const size_t smem = pl.smem;
  const int64_t nel = int64_t(r0) * d * r1;
  DBuf r(&c, nel), p(&c, 2 * nel), Ap(&c, nel), T2(&c, size_t(r0) * d * w1 * r1), part(&c, size_t(4) * G),
      bar(&c, (sizeof(CgBar) + 7) / 8);
  k_bar_init<<<1, 1, 0, c.stream>>>(reinterpret_cast<CgBar*>(bar.p), c.root->wait_ns);
  after_launch(c, "bar_init");
  CgArgs a;
  a.r0 = r0; a.r1 = r1; a.w0 = w0; a.w1 = w1; a.d = d; a.bt = bt; a.iters = iters;
  a.eb = pl.eb; a.ch = pl.ch;
  a.tol = tol_dev;
  a.L = L; a.W = W; a.R = R; a.b = b; a.x = x;
  a.r = r.p; a.p = p.p; a.Ap = Ap.p; a.T2 = T2.p; a.part = part.p; a.dinv = dinv;
  a.bar = reinterpret_cast<CgBar*>(bar.p);
  a.total = total_dev;
  a.flops = c.root->prof.on ? c.root->prof.dev_flops : nullptr;
  a.fpi = 2.0 * (double(r0) * w0 * r0 * d * r1 + double(r0) * d * w0 * d * w1 * r1 + double(r0) * d * w1 * r1 * r1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(G));
  cfg.blockDim = dim3(CGP_THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = c.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  ProfScope ps(c, KC_CG);
  QTT_CUDA(cudaLaunchKernelEx(&cfg, k_cg_persistent, a));
  after_launch(c, "cg_persistent");
}

// ------------------------------------------------------------------ tensor-core local solve
// The same CG with both contractions done as exact digit-split products on the bf16 tensor
// cores (the scheme of qtt_ozaki.cu: seven balanced 8-bit digits per row or column, group sums
// exact in FP32 over 64-wide k chunks, 128-bit fixed-point accumulation, one rounding per
// output).  Per solve, W and R are folded into
//     Q[(s, e), (w, t, b)] = sum_v W[w, s, t, v] R[e, v, b]
// so that the operator is two products:
//   A  T1[(c, w), (t, b)] = sum_a L[(c, w), a] P[a, (t, b)]
//   B  Ap[c, (s, e)]     = sum_{(w, t, b)} T1[c, (w, t, b)] Q[(s, e), (w, t, b)]
// Rows of L and of Q are split once per solve (before the launch); columns of P are split by
// the stage-A items themselves; rows of T1 need their whole row, so they are split in a phase
// of their own between two barriers.  Stage-A items (128 rows of L x 8 columns of P) live on
// CTAs [0, IA) and keep their digit slices of L in shared memory for the whole solve;
// stage-B items (16 rows of T1 x 8 columns) live on CTAs [IA, IA + IB), each warp taking
// whole k chunks and the CTA adding the warps' exact partials.  Stage C, the stopping rule,
// the deterministic partial sums and the bounded barrier are those of the FP64 kernel.

namespace {

constexpr int TC_AM = 128;          // stage-A item rows (8 warps x m16)
constexpr int TC_BM = 16;           // stage-B item rows (one m16 tile)
constexpr int TC_N = 8;             // item columns in both stages (one n8 tile)
constexpr int TC_KC = 64;           // k per exact FP32 group accumulation
constexpr int TC_LDB = TC_KC + 8;   // padded row of a stage-B digit slice (bf16)
constexpr int TC_THREADS = 256;
constexpr int TC_MAX_KPA = 64;      // stage-A k (= r0, padded) kept resident: r0 <= 64

struct CgTcArgs {
  int iters;
  int MA, NA, KA, KpA;      // stage A: rows (c, w) = r0 w0, columns (t, b) = d r1, k = a (r0)
  int MB, NB, KB, KpB;      // stage B: rows c = r0, columns (s, e) = d r1, k = (w, t, b)
  int IA, IB, nNA, nNB;
  const double* tol;        // relative tolerance (device scalar, read at launch)
  const __nv_bfloat16* La;  // [S][MA][KpA] digit slices of the rows of L
  const int* eL;            // [MA] scale exponents
  const __nv_bfloat16* Qd;  // [S][NB][KpB] digit slices of the rows of Q
  const int* eQ;            // [NB]
  __nv_bfloat16* Td;        // [S][MB][KpB] digit slices of the rows of T1 (every iteration)
  int* fT;                  // [MB] largest exponent field of each row of T1
  const double* b;
  double* x;
  double* r;
  double* p;                // 2 x nel: directions of even and odd iterations
  double* Ap;
  double* T1;               // MA x NA = MB x KB
  double* part;             // 4 x gridDim.x
  const double* dinv;       // diagonal preconditioner (may be null)
  CgBar* bar;
  int* total;
  double* flops;            // += (iterations + 1) * fpi when profiling (may be null)
  double fpi;               // FP64-equivalent flops of one operator application
};

__device__ __forceinline__ double tc_nan() { return __longlong_as_double(0x7ff8000000000000ll); }

// The seven digits of F into dst[s * sstride] (s = 0 most significant), as k_oz_digits.
__device__ __forceinline__ void tc_digits(long long F, __nv_bfloat16* dst, size_t sstride) {
#pragma unroll
  for (int s = OZ_S - 1; s >= 1; --s) {
    const long long dg = ((F + 128) & 255) - 128;
    F = (F - dg) >> 8;
    dst[s * sstride] = __float2bfloat16_rn(float(dg));
  }
  dst[0] = __float2bfloat16_rn(float(F));
}

// One warp: the exact product of a 16-row A tile and an 8-column B tile over one k chunk of
// kw <= 64 (a multiple of 16), digit slices in shared memory (row strides lda / ldb, slice
// strides sa / sb), added into the fixed-point accumulators.  The B fragments of all seven
// slices stay in registers; each A slice is loaded once and multiplied into the group
// accumulators it contributes to (group t = s + u, exact in FP32: at most 7 pairs x 64 k x 2^14).
__device__ __forceinline__ void tc_mma_chunk(const __nv_bfloat16* A, int lda, size_t sa, const __nv_bfloat16* B,
                                             int ldb, size_t sb, int kw, long long (&hi)[4],
                                             unsigned long long (&lo)[4]) {
  const int lane = threadIdx.x & 31;
  const int nk = kw / 16;
  uint32_t bf[OZ_S][4][2];
#pragma unroll
  for (int u = 0; u < OZ_S; ++u)
#pragma unroll
    for (int i = 0; i < 4; ++i)
      if (i < nk) ldsm_x2(bf[u][i], B + u * sb + (lane & 7) * ldb + 16 * i + ((lane >> 3) & 1) * 8);
  float c32[OZ_S][4];
#pragma unroll
  for (int g = 0; g < OZ_S; ++g)
#pragma unroll
    for (int q = 0; q < 4; ++q) c32[g][q] = 0.f;
#pragma unroll
  for (int s = 0; s < OZ_S; ++s)
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      if (i >= nk) continue;
      uint32_t af[4];
      ldsm_x4(af, A + s * sa + (lane & 15) * lda + 16 * i + (lane >> 4) * 8);
#pragma unroll
      for (int u = 0; u < OZ_S - s; ++u) mma_bf16(c32[s + u], af, bf[u][i][0], bf[u][i][1]);
    }
  // digit indices s + 1 and u + 1: group t = s + u + 2 enters shifted by 8 (S + 1 - t) bits
#pragma unroll
  for (int g = 0; g < OZ_S; ++g)
#pragma unroll
    for (int q = 0; q < 4; ++q)
      oz_acc(hi[q], lo[q], static_cast<long long>(__float2int_rz(c32[g][q])), 8 * (OZ_S - 1 - g));
}

// Shared memory of a stage-A CTA: L slices [S][128][KpA + 8], P slices [S][8][KpA + 8],
// P values [KpA][8], column exponent fields [8].
__host__ __device__ constexpr size_t tc_smem_a(int KpA) {
  return size_t(OZ_S) * (TC_AM + TC_N) * (KpA + 8) * 2 + size_t(KpA) * TC_N * 8 + 64;
}
// Shared memory of a stage-B CTA: per warp A slices [S][16][72] and B slices [S][8][72].
__host__ __device__ constexpr size_t tc_smem_b() { return size_t(8) * OZ_S * (TC_BM + TC_N) * TC_LDB * 2 + 64; }

// Stage A on the CTA's item: T1 for its 128 rows x 8 columns.  P = Rv + beta P0 (as its
// owners store it) or P0.
__device__ void tc_stage_a(const CgTcArgs& a, const double* P0, const double* Rv, double beta, unsigned char* sm) {
  const int ia = blockIdx.x;
  if (ia >= a.IA) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int ldA = a.KpA + 8;
  __nv_bfloat16* sLa = reinterpret_cast<__nv_bfloat16*>(sm);
  __nv_bfloat16* sPd = sLa + size_t(OZ_S) * TC_AM * ldA;
  double* sPv = reinterpret_cast<double*>(sPd + size_t(OZ_S) * TC_N * ldA);
  int* sF = reinterpret_cast<int*>(sPv + size_t(a.KpA) * TC_N);
  const int m0 = (ia / a.nNA) * TC_AM, n0 = (ia % a.nNA) * TC_N;
  if (tid < TC_N) sF[tid] = 0;
  __syncthreads();
  // column j = tid % 8 for every e this thread takes (the stride is a multiple of 8): a running
  // max per thread, then over the lanes of the same column, then one shared atomic per column
  // and warp
  int fmax = 0;
  for (int e = tid; e < a.KA * TC_N; e += TC_THREADS) {
    const int k = e / TC_N, j = e - k * TC_N, n = n0 + j;
    double v = 0.0;
    if (n < a.NA) {
      const size_t g = size_t(k) * a.NA + n;
      v = Rv ? fma(beta, __ldcg(P0 + g), zval(a.dinv, Rv, g)) : __ldcg(P0 + g);
    }
    sPv[e] = v;
    fmax = max(fmax, oz_field(v));
  }
  fmax = max(fmax, __shfl_xor_sync(0xffffffffu, fmax, 8));
  fmax = max(fmax, __shfl_xor_sync(0xffffffffu, fmax, 16));
  if (lane < TC_N) atomicMax(sF + lane, fmax);
  __syncthreads();
  for (int e = tid; e < a.KpA * TC_N; e += TC_THREADS) {
    const int k = e / TC_N, j = e - k * TC_N;
    const long long F = k < a.KA ? oz_fixed(sPv[e], oz_scale(sF[j])) : 0;
    tc_digits(F, sPd + size_t(j) * ldA + k, size_t(TC_N) * ldA);
  }
  __syncthreads();
  const int mw = m0 + warp * 16;
  if (mw < a.MA) {
    long long hi[4] = {0, 0, 0, 0};
    unsigned long long lo[4] = {0ull, 0ull, 0ull, 0ull};
    tc_mma_chunk(sLa + size_t(warp) * 16 * ldA, ldA, size_t(TC_AM) * ldA, sPd, ldA, size_t(TC_N) * ldA, a.KpA, hi,
                 lo);
    const int g = lane >> 2, tg = lane & 3;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int m = mw + g + (q >= 2 ? 8 : 0), j = 2 * tg + (q & 1), n = n0 + j;
      if (m >= a.MA || n >= a.NA) continue;
      const int fp = sF[j], el = __ldg(a.eL + m);
      a.T1[size_t(m) * a.NA + n] =
          (fp == 0x7ff || el > 1025) ? tc_nan() : fixed_to_double(hi[q], lo[q], el + oz_scale(fp) - 8 * (OZ_S + 1));
    }
  }
}

// Split phase: the digit slices of every row of T1 (one row per CTA at a time, all CTAs).
__device__ void tc_split_t1(const CgTcArgs& a, int* sred) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int row = blockIdx.x; row < a.MB; row += gridDim.x) {
    const double* src = a.T1 + size_t(row) * a.KB;
    int mx = 0;
    for (int k = tid; k < a.KB; k += TC_THREADS) mx = max(mx, oz_field(__ldcg(src + k)));
    for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (lane == 0) sred[warp] = mx;
    __syncthreads();
    mx = 0;
    for (int w = 0; w < TC_THREADS / 32; ++w) mx = max(mx, sred[w]);
    const int e = oz_scale(mx);
    for (int k = tid; k < a.KpB; k += TC_THREADS) {
      const long long F = k < a.KB ? oz_fixed(__ldcg(src + k), e) : 0;
      tc_digits(F, a.Td + size_t(row) * a.KpB + k, size_t(a.MB) * a.KpB);
    }
    if (tid == 0) a.fT[row] = mx;
    __syncthreads();
  }
}

// Stage B on the CTA's item: Ap for its 16 rows x 8 columns; returns this CTA's share of P . Ap
// (0 if P is null).
__device__ double tc_stage_b(const CgTcArgs& a, const double* P, unsigned char* sm) {
  const int ib = int(blockIdx.x) - a.IA;
  if (ib < 0 || ib >= a.IB) return 0.0;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int c0 = (ib / a.nNB) * TC_BM, n0 = (ib % a.nNB) * TC_N;
  const size_t per_warp = size_t(OZ_S) * (TC_BM + TC_N) * TC_LDB;
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(sm) + warp * per_warp;
  __nv_bfloat16* sB = sA + size_t(OZ_S) * TC_BM * TC_LDB;
  long long hi[4] = {0, 0, 0, 0};
  unsigned long long lo[4] = {0ull, 0ull, 0ull, 0ull};
  // k in pieces of 32 (KpB is a multiple of 64): 768 = 24 pieces, three per warp
  constexpr int KW = TC_KC / 2;
  const int nch = a.KpB / KW;
  for (int q = warp; q < nch; q += TC_THREADS / 32) {
    const int k0 = q * KW;
    // 16 rows of T1 and 8 rows of Q, 7 slices each, 32 k: 16-byte asynchronous copies
    for (int idx = lane; idx < OZ_S * TC_BM * 4; idx += 32) {   // (slice, row, 16-byte vector)
      const int c4 = idx & 3, sr = idx >> 2, s = sr >> 4, row = sr & 15, c = c0 + row;
      const bool in = c < a.MB;
      cp_async16(sA + (s * TC_BM + row) * TC_LDB + c4 * 8,
                 in ? a.Td + (size_t(s) * a.MB + c) * a.KpB + k0 + c4 * 8 : a.Td, in);
    }
    for (int idx = lane; idx < OZ_S * TC_N * 4; idx += 32) {
      const int c4 = idx & 3, sr = idx >> 2, s = sr >> 3, j = sr & 7, n = n0 + j;
      const bool in = n < a.NB;
      cp_async16(sB + (s * TC_N + j) * TC_LDB + c4 * 8,
                 in ? a.Qd + (size_t(s) * a.NB + n) * a.KpB + k0 + c4 * 8 : a.Qd, in);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncwarp();
    tc_mma_chunk(sA, TC_LDB, size_t(TC_BM) * TC_LDB, sB, TC_LDB, size_t(TC_N) * TC_LDB, KW, hi, lo);
    __syncwarp();
  }
  // add the warps' partials in warp order (exact), convert once per output
  __syncthreads();
  long long* xh = reinterpret_cast<long long*>(sm);
  unsigned long long* xl = reinterpret_cast<unsigned long long*>(sm) + (TC_THREADS * 4);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    xh[tid * 4 + q] = hi[q];
    xl[tid * 4 + q] = lo[q];
  }
  __syncthreads();
  double dot = 0.0;
  if (warp == 0) {
    const int g = lane >> 2, tg = lane & 3;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      long long H = 0;
      unsigned long long Lo = 0ull;
      for (int w = 0; w < TC_THREADS / 32; ++w) oz_add128(H, Lo, xh[(w * 32 + lane) * 4 + q], xl[(w * 32 + lane) * 4 + q]);
      const int c = c0 + g + (q >= 2 ? 8 : 0), n = n0 + 2 * tg + (q & 1);
      if (c >= a.MB || n >= a.NB) continue;
      const int ft = __ldcg(a.fT + c), eq = __ldg(a.eQ + n);
      const double v =
          (ft == 0x7ff || eq > 1025) ? tc_nan() : fixed_to_double(H, Lo, oz_scale(ft) + eq - 8 * (OZ_S + 1));
      const size_t idx = size_t(c) * a.NB + n;
      a.Ap[idx] = v;
      if (P) dot = fma(__ldcg(P + idx), v, dot);
    }
  }
  __syncthreads();   // the exchange buffer overlaps warp 0's digit slices
  return dot;
}

__global__ void __launch_bounds__(TC_THREADS, 1) k_cg_tc(CgTcArgs a) {
  extern __shared__ __align__(16) unsigned char tc_sm[];
  const int G = gridDim.x, tid = threadIdx.x, nt = blockDim.x;
  const int64_t nel = int64_t(a.MB) * a.NB;
  __shared__ double red[32];
  __shared__ int sred[TC_THREADS / 32];
  __shared__ int flag;
  unsigned int target = 0;
  double* part_pap = a.part;
  double* part_rr = a.part + G;
  double* part_bb = a.part + 2 * G;
  double* part_rz = a.part + 3 * G;
  // stage-A CTAs: their rows of the L slices, resident for the whole solve
  if (int(blockIdx.x) < a.IA) {
    const int ldA = a.KpA + 8, m0 = (int(blockIdx.x) / a.nNA) * TC_AM, v8 = a.KpA / 8;
    __nv_bfloat16* sLa = reinterpret_cast<__nv_bfloat16*>(tc_sm);
    for (int idx = tid; idx < OZ_S * TC_AM * v8; idx += nt) {
      const int s = idx / (TC_AM * v8), rem = idx - s * TC_AM * v8, row = rem / v8, c8 = rem - row * v8;
      const int m = m0 + row;
      const bool in = m < a.MA;
      cp_async16(sLa + (size_t(s) * TC_AM + row) * ldA + c8 * 8,
                 in ? a.La + (size_t(s) * a.MA + m) * a.KpA + c8 * 8 : a.La, in);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
  }
  bool ok = true;
  int count = 0;
  do {
    // ---- initial residual: r = b - A x, p_0 = r
    tc_stage_a(a, a.x, nullptr, 0.0, tc_sm);
    if (!(ok = grid_sync(a.bar, target, &flag))) break;
    tc_split_t1(a, sred);
    if (!(ok = grid_sync(a.bar, target, &flag))) break;
    tc_stage_b(a, nullptr, tc_sm);
    if (!(ok = grid_sync(a.bar, target, &flag))) break;
    double rr_p = 0.0, bb_p = 0.0, rz_p = 0.0;
    for (int64_t e = int64_t(blockIdx.x) * nt + tid; e < nel; e += int64_t(G) * nt) {
      const double be = __ldg(a.b + e);
      const double re = be - __ldcg(a.Ap + e);
      const double ze = a.dinv ? __ldg(a.dinv + e) * re : re;
      a.r[e] = re;
      a.p[e] = ze;
      rr_p = fma(re, re, rr_p);
      rz_p = fma(re, ze, rz_p);
      bb_p = fma(be, be, bb_p);
    }
    rr_p = block_reduce(rr_p, red);
    rz_p = block_reduce(rz_p, red);
    bb_p = block_reduce(bb_p, red);
    if (tid == 0) {
      part_rr[blockIdx.x] = rr_p;
      part_rz[blockIdx.x] = rz_p;
      part_bb[blockIdx.x] = bb_p;
    }
    if (!(ok = grid_sync(a.bar, target, &flag))) break;
    double rr = sum_partials(part_rr, red);
    double rz = sum_partials(part_rz, red);
    const double bb = sum_partials(part_bb, red);
    const double tol2 = __ldg(a.tol) * __ldg(a.tol);
    bool active = rr > tol2 * bb && rr > 0.0;
    double beta = 0.0;
    for (int it = 0; it < a.iters && active; ++it) {
      double* pn = a.p + (it & 1) * nel;
      const double* po = a.p + ((it & 1) ^ 1) * nel;
      if (it == 0) {
        tc_stage_a(a, pn, nullptr, 0.0, tc_sm);
      } else {
        for (int64_t e = int64_t(blockIdx.x) * nt + tid; e < nel; e += int64_t(G) * nt)
          pn[e] = fma(beta, po[e], zval(a.dinv, a.r, e));
        tc_stage_a(a, po, a.r, beta, tc_sm);
      }
      if (!(ok = grid_sync(a.bar, target, &flag))) break;
      tc_split_t1(a, sred);
      if (!(ok = grid_sync(a.bar, target, &flag))) break;
      double pap_p = tc_stage_b(a, pn, tc_sm);
      pap_p = block_reduce(pap_p, red);
      if (tid == 0) part_pap[blockIdx.x] = pap_p;
      if (!(ok = grid_sync(a.bar, target, &flag))) break;
      const double pap = sum_partials(part_pap, red);
      if (!(pap > 0.0)) break;
      const double alpha = rz / pap;
      double rn_p = 0.0, rzn_p = 0.0;
      for (int64_t e = int64_t(blockIdx.x) * nt + tid; e < nel; e += int64_t(G) * nt) {
        a.x[e] += alpha * pn[e];
        const double re = a.r[e] - alpha * __ldcg(a.Ap + e);
        a.r[e] = re;
        rn_p = fma(re, re, rn_p);
        rzn_p = fma(re, a.dinv ? __ldg(a.dinv + e) * re : re, rzn_p);
      }
      rn_p = block_reduce(rn_p, red);
      rzn_p = block_reduce(rzn_p, red);
      if (tid == 0) {
        part_rr[blockIdx.x] = rn_p;
        part_rz[blockIdx.x] = rzn_p;
      }
      if (!(ok = grid_sync(a.bar, target, &flag))) break;
      const double rn = sum_partials(part_rr, red);
      const double rzn = sum_partials(part_rz, red);
      beta = rzn / rz;
      rr = rn;
      rz = rzn;
      count += 1;
      active = rn > tol2 * bb && rn > 0.0;
    }
  } while (false);
  if (blockIdx.x == 0 && tid == 0 && a.total) {
    if (ok) *a.total += count;
    else *a.total = CGP_POISON;
  }
  if (blockIdx.x == 0 && tid == 0 && a.flops && ok) atomicAdd(a.flops, (count + 1) * a.fpi);
}

struct TcPlan {
  int MA, NA, KA, KpA, MB, NB, KB, KpB, IA, IB, nNA, nNB;
  size_t smem;
};

bool tc_plan(const Ctx& c, int r0, int r1, int w0, int w1, int d, TcPlan& p) {
  if (&c != c.root || c.root->gemm_mode == 1) return false;
  if (!(r0 >= 1 && r1 >= 1 && r0 <= TC_MAX_KPA && r1 <= CGP_MAX_BOND && w0 >= 1 && w1 >= 1 && w0 <= CGP_MAX_W &&
        w1 <= CGP_MAX_W && d >= 1 && d <= CGP_MAX_D))
    return false;
  p.MA = r0 * w0;
  p.NA = d * r1;
  p.KA = r0;
  p.KpA = (r0 + 15) / 16 * 16;
  p.MB = r0;
  p.NB = d * r1;
  p.KB = w0 * d * r1;
  p.KpB = (p.KB + TC_KC - 1) / TC_KC * TC_KC;
  p.nNA = (p.NA + TC_N - 1) / TC_N;
  p.nNB = (p.NB + TC_N - 1) / TC_N;
  p.IA = ((p.MA + TC_AM - 1) / TC_AM) * p.nNA;
  p.IB = ((p.MB + TC_BM - 1) / TC_BM) * p.nNB;
  p.smem = std::max(tc_smem_a(p.KpA), tc_smem_b());
  (void)w1;
  return p.IA + p.IB <= c.num_sms && p.smem <= 227 * 1024;
}

bool g_tc_attr = false;
bool g_tc_ok = false;

}  // namespace

void cg_tc_init_attributes() {
  if (g_tc_attr) return;
  g_tc_attr = true;
  const int smem = int(std::max(tc_smem_a(TC_MAX_KPA), tc_smem_b()));
  if (cudaFuncSetAttribute(k_cg_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_cg_tc, TC_THREADS, smem) == cudaSuccess)
    g_tc_ok = per_sm >= 1;
  cudaGetLastError();
}

bool cg_tc_fits(const Ctx& c, int r0, int r1, int w0, int w1, int d) {
  cg_tc_init_attributes();
  TcPlan p;
  return g_tc_ok && tc_plan(c, r0, r1, w0, w1, d, p);
}

void cg_tc(Ctx& c, const double* L, const double* W, const double* R, const double* b, double* x, int r0, int r1,
           int w0, int w1, int d, int iters, const double* tol_dev, int* total_dev, const double* dinv) {
  TcPlan pl;
  cg_tc_init_attributes();
  QTT_CHECK_ARG(g_tc_ok && tc_plan(c, r0, r1, w0, w1, d, pl), "cg_tc: shape outside the supported range");
  const int G = c.num_sms;
  const int64_t nel = int64_t(r0) * d * r1;
  auto halves = [](size_t n) { return (n * 2 + 7) / 8; };   // bf16 count -> doubles
  auto ints = [](size_t n) { return (n * 4 + 7) / 8; };
  DBuf La(&c, halves(size_t(OZ_S) * pl.MA * pl.KpA)), eL(&c, ints(pl.MA)), Q(&c, size_t(pl.NB) * pl.KB),
      Qd(&c, halves(size_t(OZ_S) * pl.NB * pl.KpB)), eQ(&c, ints(pl.NB)), Td(&c, halves(size_t(OZ_S) * pl.MB * pl.KpB)),
      fT(&c, ints(pl.MB)), r(&c, nel), p(&c, 2 * nel), Ap(&c, nel), T1(&c, size_t(pl.MA) * pl.NA),
      part(&c, size_t(4) * G), bar(&c, (sizeof(CgBar) + 7) / 8);
  // per solve: digit slices of the rows of L, Q = W x_v R and its rows' digit slices
  oz_split_rows(c, pl.MA, pl.KA, pl.KpA, L, pl.KA, 1, La.p, reinterpret_cast<int*>(eL.p));
  einsum(c, "wstv,evb->sewtb", 1.0, tv(const_cast<double*>(W), {w0, d, d, w1}),
         tv(const_cast<double*>(R), {r1, w1, r1}), 0.0, tv(Q.p, {d, r1, w0, d, r1}));
  oz_split_rows(c, pl.NB, pl.KB, pl.KpB, Q.p, pl.KB, 1, Qd.p, reinterpret_cast<int*>(eQ.p));
  k_bar_init<<<1, 1, 0, c.stream>>>(reinterpret_cast<CgBar*>(bar.p), c.root->wait_ns);
  after_launch(c, "bar_init");
  CgTcArgs a;
  a.iters = iters;
  a.MA = pl.MA; a.NA = pl.NA; a.KA = pl.KA; a.KpA = pl.KpA;
  a.MB = pl.MB; a.NB = pl.NB; a.KB = pl.KB; a.KpB = pl.KpB;
  a.IA = pl.IA; a.IB = pl.IB; a.nNA = pl.nNA; a.nNB = pl.nNB;
  a.tol = tol_dev;
  a.La = reinterpret_cast<const __nv_bfloat16*>(La.p);
  a.eL = reinterpret_cast<const int*>(eL.p);
  a.Qd = reinterpret_cast<const __nv_bfloat16*>(Qd.p);
  a.eQ = reinterpret_cast<const int*>(eQ.p);
  a.Td = reinterpret_cast<__nv_bfloat16*>(Td.p);
  a.fT = reinterpret_cast<int*>(fT.p);
  a.b = b; a.x = x; a.r = r.p; a.p = p.p; a.Ap = Ap.p; a.T1 = T1.p; a.part = part.p; a.dinv = dinv;
  a.bar = reinterpret_cast<CgBar*>(bar.p);
  a.total = total_dev;
  a.flops = c.root->prof.on ? c.root->prof.dev_flops : nullptr;
  a.fpi = 2.0 * (double(r0) * w0 * r0 * d * r1 + double(r0) * d * r1 * w0 * d * r1);
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(unsigned(G));
  cfg.blockDim = dim3(TC_THREADS);
  cfg.dynamicSmemBytes = pl.smem;
  cfg.stream = c.stream;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeCooperative;
  at[0].val.cooperative = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  ProfScope ps(c, KC_CG);
  QTT_CUDA(cudaLaunchKernelEx(&cfg, k_cg_tc, a));
  after_launch(c, "cg_tc");
}

}  // namespace qtt
