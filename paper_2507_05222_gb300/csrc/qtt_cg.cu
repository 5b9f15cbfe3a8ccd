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
// Barrier: an arrival counter in device memory (reset by the host before the launch); a
// waiting block polls it for at most 2 s (global timer).  The cooperative launch makes every
// block resident, so the bound is only a safety net: on expiry the block sets the error flag,
// every block leaves at its next barrier, and the iteration count is overwritten with a
// negative value that the host turns into an error.  Data written by other blocks inside the
// kernel are read with ld.global.cg (L2).
#include <algorithm>

#include "qtt_algebra.h"

namespace qtt {

namespace {

constexpr int CGP_THREADS = 256;
constexpr unsigned long long CGP_TIMEOUT_NS = 2000000000ull;   // 2 s per barrier
constexpr int CGP_MAX_BOND = 128;
constexpr int CGP_MAX_W = 16;
constexpr int CGP_MAX_D = 4;

struct CgBar {
  unsigned int count;   // arrivals so far (monotonic within a launch)
  int error;            // set by a block that gave up waiting
  int pad[2];
};

struct CgArgs {
  int r0, r1, w0, w1, d, bt, iters;
  int eb, ch;     // stage B: e-block width (16, 8, 4, 2 or 1) and T2 row chunks per load
  double tol2;
  const double* L;
  const double* W;
  const double* R;
  const double* b;
  double* x;
  double* r;
  double* p;      // 2 x (r0 d r1): directions of even and odd iterations
  double* Ap;
  double* T2;
  double* part;   // 3 x gridDim.x
  CgBar* bar;
  int* total;     // += iterations done (may be null)
};

__device__ __forceinline__ unsigned int ld_acquire(const unsigned int* p) {
  unsigned int v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ int ld_volatile(const int* p) { return *reinterpret_cast<const volatile int*>(p); }

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
    while (ld_acquire(&bar->count) < target) {
      if ((++spins & 255u) == 0u) {
        if (ld_volatile(&bar->error)) break;
        if (global_ns() - t0 > CGP_TIMEOUT_NS) {
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

// Stage A: T2 = (L . P) . W, with P the vector P0 or, when Rv is given, P = Rv + beta P0 formed
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
        sP[row * bt + lane] = Rv ? fma(beta, __ldcg(P0 + g), __ldcg(Rv + g)) : __ldcg(P0 + g);
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
    double rr_p = 0.0, bb_p = 0.0;
    for (int64_t e = int64_t(blockIdx.x) * nt + tid; e < nel; e += int64_t(G) * nt) {
      const double be = __ldg(a.b + e);
      const double re = be - __ldcg(a.Ap + e);
      a.r[e] = re;
      a.p[e] = re;
      rr_p = fma(re, re, rr_p);
      bb_p = fma(be, be, bb_p);
    }
    rr_p = block_reduce(rr_p, red);
    bb_p = block_reduce(bb_p, red);
    if (tid == 0) {
      part_rr[blockIdx.x] = rr_p;
      part_bb[blockIdx.x] = bb_p;
    }
    if (!(ok = grid_sync(a.bar, target, &flag))) break;
    double rr = sum_partials(part_rr, red);
    const double bb = sum_partials(part_bb, red);
    bool active = rr > a.tol2 * bb && rr > 0.0;
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
          pn[e] = fma(beta, po[e], a.r[e]);
        stage_a(a, po, a.r, beta, sL, sW, sP, sT1);
      }
      if (!(ok = grid_sync(a.bar, target, &flag))) break;
      double pap_p = stage_b(a, pn, a.Ap, sR, sT2);
      pap_p = block_reduce(pap_p, red);
      if (tid == 0) part_pap[blockIdx.x] = pap_p;
      if (!(ok = grid_sync(a.bar, target, &flag))) break;
      const double pap = sum_partials(part_pap, red);
      if (!(pap > 0.0)) break;                       // same decision in every block
      const double alpha = rr / pap;
      double rn_p = 0.0;
      for (int64_t e = int64_t(blockIdx.x) * nt + tid; e < nel; e += int64_t(G) * nt) {
        a.x[e] += alpha * pn[e];
        const double re = a.r[e] - alpha * __ldcg(a.Ap + e);
        a.r[e] = re;
        rn_p = fma(re, re, rn_p);
      }
      rn_p = block_reduce(rn_p, red);
      if (tid == 0) part_rr[blockIdx.x] = rn_p;
      if (!(ok = grid_sync(a.bar, target, &flag))) break;
      const double rn = sum_partials(part_rr, red);
      beta = rn / rr;
      rr = rn;
      count += 1;
      active = rn > a.tol2 * bb && rn > 0.0;
    }
  } while (false);
  if (blockIdx.x == 0 && tid == 0 && a.total) {
    if (ok) *a.total += count;
    else *a.total = CGP_POISON;
  }
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
                   int r1, int w0, int w1, int d, int iters, double tol, int* total_dev) {
  CgPlan pl;
  QTT_CHECK_ARG(cg_plan(c, r0, r1, w0, w1, d, pl), "cg_persistent: shape outside the supported range");
  cg_init_attributes();
  if (g_cgp_per_sm < 2) throw Error(QTT_ERR_UNSUPPORTED, "cg_persistent: fewer than two blocks fit an SM");
  const int G = pl.G, bt = pl.bt;
  const size_t smem = pl.smem;
  const int64_t nel = int64_t(r0) * d * r1;
  DBuf r(&c, nel), p(&c, 2 * nel), Ap(&c, nel), T2(&c, size_t(r0) * d * w1 * r1), part(&c, size_t(3) * G),
      bar(&c, (sizeof(CgBar) + 7) / 8);
  QTT_CUDA(cudaMemsetAsync(bar.p, 0, sizeof(CgBar), c.stream));
  CgArgs a;
  a.r0 = r0; a.r1 = r1; a.w0 = w0; a.w1 = w1; a.d = d; a.bt = bt; a.iters = iters;
  a.eb = pl.eb; a.ch = pl.ch;
  a.tol2 = tol * tol;
  a.L = L; a.W = W; a.R = R; a.b = b; a.x = x;
  a.r = r.p; a.p = p.p; a.Ap = Ap.p; a.T2 = T2.p; a.part = part.p;
  a.bar = reinterpret_cast<CgBar*>(bar.p);
  a.total = total_dev;
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

}  // namespace qtt
