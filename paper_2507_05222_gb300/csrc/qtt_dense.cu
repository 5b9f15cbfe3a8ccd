// Dense building blocks of the QTT library: device pool, FP64 batched GEMM (split-K),
// permutations, elementwise kernels, deterministic reductions and the einsum planner that
// turns every core contraction into (permute +) batched GEMM.
//
// FP64 on GB300 runs at ~1/70 of the FP32 rate (about 1.7 DFMA per clock per SM), so the
// GEMM kernel is bound by the FP64 pipe, not by memory: the design goal is enough CTAs
// (>= 2 x 152) for every contraction, which small core contractions only reach through
// split-K, and no host synchronisation between the many small launches.
#include <algorithm>
#include <cstring>
#include <numeric>

#include "qtt_internal.h"

namespace qtt {

// ------------------------------------------------------------------ pool

Pool::~Pool() {
  for (auto& ch : chunks_) {
    if (free_) free_(ch.first, user_);
    else cudaFree(ch.first);
  }
}

size_t Pool::size_class(size_t bytes) {
  if (bytes < 256) return 256;
  // 8 classes per power of two
  size_t p = 1;
  while (p * 2 <= bytes) p *= 2;
  size_t step = p / 8 < 256 ? 256 : p / 8;
  return (bytes + step - 1) / step * step;
}

void* Pool::raw_alloc(size_t bytes) {
  void* p = nullptr;
  if (alloc_) p = alloc_(bytes, user_);
  else if (cudaMalloc(&p, bytes) != cudaSuccess) p = nullptr;
  if (!p) throw Error(QTT_ERR_ALLOC, "device allocation of " + std::to_string(bytes) + " bytes failed");
  chunks_.push_back({p, bytes});
  held_ += bytes;
  return p;
}

void* Pool::get(size_t bytes) {
  size_t cls = size_class(bytes);
  if (capturing_) {
    auto& arena = cap_free_[capturing_];
    auto ci = arena.find(cls);
    if (ci != arena.end()) {
      void* p = ci->second;
      arena.erase(ci);
      live_[p] = cls;
      return p;
    }
    if (cls > cur_left_) {
      size_t chunk = std::max<size_t>(cls, size_t(64) << 20);
      cur_ = static_cast<char*>(raw_alloc(chunk));
      cur_left_ = chunk;
    }
    void* p = cur_;
    cur_ += cls;
    cur_left_ -= cls;
    live_[p] = cls;
    cap_owned_[p] = capturing_;
    return p;
  }
  auto it = free_blocks_.lower_bound(cls);
  if (it != free_blocks_.end() && it->first == cls) {
    void* p = it->second;
    free_blocks_.erase(it);
    live_[p] = cls;
    return p;
  }
  if (cls > cur_left_) {
    size_t chunk = std::max<size_t>(cls, size_t(64) << 20);
    cur_ = static_cast<char*>(raw_alloc(chunk));
    cur_left_ = chunk;
  }
  void* p = cur_;
  cur_ += cls;
  cur_left_ -= cls;
  live_[p] = cls;
  return p;
}

void Pool::put(void* p) {
  if (!p) return;
  auto it = live_.find(p);
  if (it == live_.end()) return;
  size_t cls = it->second;
  live_.erase(it);
  auto own = cap_owned_.find(p);
  if (own != cap_owned_.end()) {
    cap_free_[own->second].insert({cls, p});   // reserved for its graph: reused only by its captures
    return;
  }
  if (capturing_) {
    deferred_.push_back(p);
    live_[p] = cls;                               // keep its size until the capture ends
    return;
  }
  free_blocks_.insert({cls, p});
}

void Pool::begin_capture(const void* owner) {
  capturing_ = owner;
}

void Pool::end_capture() {
  capturing_ = nullptr;
  for (void* p : deferred_) {
    auto it = live_.find(p);
    if (it != live_.end()) {
      free_blocks_.insert({it->second, p});
      live_.erase(it);
    }
  }
  deferred_.clear();
}

void Pool::release_capture(const void* owner) {
  auto a = cap_free_.find(owner);
  if (a != cap_free_.end()) {
    for (auto& kv : a->second) {
      free_blocks_.insert(kv);
      cap_owned_.erase(kv.second);
    }
    cap_free_.erase(a);
  }
  // arena blocks still live (held by objects created during the capture) stay with their
  // holders and return to the ordinary free list when those are freed
  for (auto it = cap_owned_.begin(); it != cap_owned_.end();) {
    if (it->second == owner) it = cap_owned_.erase(it);
    else ++it;
  }
}

DBuf::DBuf(Ctx* c, size_t count) { reset(c, count); }
DBuf::~DBuf() {
  if (ctx && p) ctx->pool->put(p);
}
DBuf& DBuf::operator=(DBuf&& o) noexcept {
  if (this != &o) {
    if (ctx && p) ctx->pool->put(p);
    ctx = o.ctx; p = o.p; n = o.n;
    o.p = nullptr; o.n = 0;
  }
  return *this;
}
void DBuf::reset(Ctx* c, size_t count) {
  if (ctx && p) ctx->pool->put(p);
  ctx = c;
  n = count;
  p = count ? static_cast<double*>(c->pool->get(count * sizeof(double))) : nullptr;
}

void after_launch(Ctx& c, const char* what) {
  c.root->launches += 1;
  Profiler& pr = c.root->prof;
  if (pr.on) pr.acc_phase_launches[pr.phase < 0 ? KC_PHASES : pr.phase] += 1;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) throw Error(QTT_ERR_CUDA, std::string("launch of ") + what + ": " + cudaGetErrorString(e));
}

static cudaEvent_t take_event(Ctx& c) {
  Profiler& pr = c.root->prof;
  if (!pr.free_events.empty()) {
    cudaEvent_t e = pr.free_events.back();
    pr.free_events.pop_back();
    return e;
  }
  cudaEvent_t e;
  QTT_CUDA(cudaEventCreate(&e));
  return e;
}

ProfScope::ProfScope(Ctx& ctx, int kclass, double flops) : c(ctx), k(kclass) {
  Profiler& pr = c.root->prof;
  if (!pr.on) return;
  pr.flops[k] += flops;
  pr.launches[k] += 1;
  if (k >= KC_PH_APPLY) pr.phase = k - KC_PH_APPLY;
  e0 = take_event(c);
  cudaEventRecord(e0, c.stream);
}

ProfScope::~ProfScope() {
  if (!e0) return;
  Profiler& pr = c.root->prof;
  cudaEvent_t e1 = take_event(c);
  cudaEventRecord(e1, c.stream);
  pr.pending[k].push_back({e0, e1, pr.phase});
  // phase scopes are replaced by constructing the next one first: close only our own phase
  if (k >= KC_PH_APPLY && pr.phase == k - KC_PH_APPLY) pr.phase = -1;
}

void init_tile_counters(Ctx& c) {
  if (c.tile_ctr) return;
  QTT_CUDA(cudaMalloc(&c.tile_ctr, kTileCounters * sizeof(int)));
  QTT_CUDA(cudaMemsetAsync(c.tile_ctr, 0, kTileCounters * sizeof(int), c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
}

void free_tile_counters(Ctx& c) {
  if (c.tile_ctr) cudaFree(c.tile_ctr);
  c.tile_ctr = nullptr;
}

Ctx& worker(Ctx& c, int i) {
  while (int(c.workers.size()) <= i) {
    Ctx* w = new Ctx;
    w->device = c.device;
    w->num_sms = c.num_sms;
    w->root = c.root;
    w->alloc_fn = c.alloc_fn;
    w->free_fn = c.free_fn;
    w->alloc_user = c.alloc_user;
    cudaError_t e = cudaStreamCreateWithFlags(&w->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      delete w;
      throw Error(QTT_ERR_CUDA, std::string("worker stream: ") + cudaGetErrorString(e));
    }
    w->pool = new Pool(c.alloc_fn, c.free_fn, c.alloc_user);
    init_tile_counters(*w);
    cudaEvent_t j;
    QTT_CUDA(cudaEventCreateWithFlags(&j, cudaEventDisableTiming));
    c.ev_join.push_back(j);
    c.workers.push_back(w);
  }
  return *c.workers[i];
}

void fork(Ctx& c, int n) {
  for (int i = 0; i < n; ++i) worker(c, i);
  if (!c.ev_fork) QTT_CUDA(cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
  QTT_CUDA(cudaEventRecord(c.ev_fork, c.stream));
  for (int i = 0; i < n; ++i) QTT_CUDA(cudaStreamWaitEvent(c.workers[i]->stream, c.ev_fork, 0));
}

void join(Ctx& c, int n) {
  for (int i = 0; i < n; ++i) {
    QTT_CUDA(cudaEventRecord(c.ev_join[i], c.workers[i]->stream));
    QTT_CUDA(cudaStreamWaitEvent(c.stream, c.ev_join[i], 0));
  }
}

void destroy_workers(Ctx& c) {
  for (Ctx* w : c.workers) {
    cudaStreamSynchronize(w->stream);
    destroy_workers(*w);
    free_tile_counters(*w);
    delete w->pool;
    cudaStreamDestroy(w->stream);
    if (w->side) cudaStreamDestroy(w->side);
    delete w;
  }
  c.workers.clear();
  for (cudaEvent_t e : c.ev_join) cudaEventDestroy(e);
  c.ev_join.clear();
  if (c.ev_fork) cudaEventDestroy(c.ev_fork);
  c.ev_fork = nullptr;
}

TV tv(double* p, std::initializer_list<int64_t> dims) {
  TV t;
  t.p = p;
  for (int64_t d : dims) t.dim[t.nd++] = d;
  return t;
}

// ------------------------------------------------------------------ GEMM

namespace {

constexpr int GK = 16;   // k step staged in shared memory

// 256 threads (16 x 16); each thread owns a (T/16) x (T/16) block of outputs strided by 16, so
// that the shared-memory reads of B are consecutive across a warp and those of A are
// broadcasts.  T = 64 for large outputs, T = 32 to put more CTAs on small ones.
template <int T>
__global__ void __launch_bounds__(256) k_gemm(int64_t M, int64_t N, int64_t K, int64_t kchunk, int splits,
                                              int64_t batch, double alpha, const double* __restrict__ A,
                                              int64_t sAb, int64_t sAm, int64_t sAk,
                                              const double* __restrict__ B, int64_t sBb, int64_t sBk,
                                              int64_t sBn, double beta, double* __restrict__ C,
                                              int64_t sCb, int64_t sCm, int64_t sCn,
                                              double* __restrict__ W, int* __restrict__ tile_ctr,
                                              const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  constexpr int R = T / 16;          // outputs per thread per dimension
  constexpr int L = T * GK / 256;    // loads per thread per operand tile
  __shared__ double As[GK][T];
  __shared__ double Bs[GK][T];
  const int tx = threadIdx.x, ty = threadIdx.y;
  const int t = ty * 16 + tx;
  const int64_t n0 = int64_t(blockIdx.x) * T, m0 = int64_t(blockIdx.y) * T;
  const int64_t b = blockIdx.z / splits;
  const int sp = blockIdx.z % splits;
  const int64_t k0 = sp * kchunk;
  const int64_t k1 = min(K, k0 + kchunk);
  const double* Ab = A + b * sAb;
  const double* Bb = B + b * sBb;
  double acc[R][R];
#pragma unroll
  for (int i = 0; i < R; ++i)
#pragma unroll
    for (int j = 0; j < R; ++j) acc[i][j] = 0.0;
  const bool a_k_fast = (sAk == 1);
  const bool b_n_fast = (sBn == 1);
  for (int64_t kb = k0; kb < k1; kb += GK) {
#pragma unroll
    for (int i = 0; i < L; ++i) {
      int e = t + 256 * i;
      int mm, kk;
      if (a_k_fast) { mm = e / GK; kk = e % GK; } else { mm = e % T; kk = e / T; }
      int64_t gm = m0 + mm, gk = kb + kk;
      As[kk][mm] = (gm < M && gk < k1) ? Ab[gm * sAm + gk * sAk] : 0.0;
      int nn, kk2;
      if (b_n_fast) { kk2 = e / T; nn = e % T; } else { nn = e / GK; kk2 = e % GK; }
      int64_t gn = n0 + nn, gk2 = kb + kk2;
      Bs[kk2][nn] = (gn < N && gk2 < k1) ? Bb[gk2 * sBk + gn * sBn] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < GK; ++kk) {
      double a[R], bv[R];
#pragma unroll
      for (int i = 0; i < R; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < R; ++j) bv[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < R; ++i)
#pragma unroll
        for (int j = 0; j < R; ++j) acc[i][j] = fma(a[i], bv[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      if (W) {
        W[((int64_t(sp) * batch + b) * M + gm) * N + gn] = acc[i][j];
      } else {
        double* cp = C + b * sCb + gm * sCm + gn * sCn;
        *cp = (beta == 0.0) ? alpha * acc[i][j] : alpha * acc[i][j] + beta * (*cp);
      }
    }
  }
  if (!W || !tile_ctr) return;
  // Split-K fix-up without a second launch: the CTA that finishes a tile last (arrival counter)
  // sums the tile's partials over the splits in split order -- the order of k_splitk_reduce,
  // whichever CTA is last -- and resets the counter for the next GEMM on this stream.
  __shared__ int last;
  __threadfence();
  __syncthreads();
  const int64_t tile = (b * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  if (t == 0) last = (atomicAdd(tile_ctr + tile, 1) == splits - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
#pragma unroll
  for (int i = 0; i < R; ++i) {
    int64_t gm = m0 + ty + 16 * i;
    if (gm >= M) continue;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      int64_t gn = n0 + tx + 16 * j;
      if (gn >= N) continue;
      double s = 0.0;
      for (int q = 0; q < splits; ++q) s += __ldcg(W + ((int64_t(q) * batch + b) * M + gm) * N + gn);
      double* cp = C + b * sCb + gm * sCm + gn * sCn;
      *cp = (beta == 0.0) ? alpha * s : alpha * s + beta * (*cp);
    }
  }
  if (t == 0) tile_ctr[tile] = 0;
}

__global__ void k_splitk_reduce(int64_t batch, int64_t M, int64_t N, int splits, double alpha,
                                const double* __restrict__ W, double beta, double* __restrict__ C,
                                int64_t sCb, int64_t sCm, int64_t sCn, const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  int64_t total = batch * M * N;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    double s = 0.0;
    for (int sp = 0; sp < splits; ++sp) s += W[int64_t(sp) * total + e];
    int64_t b = e / (M * N), r = e % (M * N), m = r / N, n = r % N;
    double* cp = C + b * sCb + m * sCm + n * sCn;
    *cp = (beta == 0.0) ? alpha * s : alpha * s + beta * (*cp);
  }
}

int grid_for(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  return int(std::max<int64_t>(1, std::min<int64_t>(g, 65535 * 8)));
}

// Direct contraction for small problems: C[o] = alpha sum_k A[a(o) + ka(k)] B[b(o) + kb(k)]
// (+ beta C[o]), every operand read in place through per-label strides.  The output index is
// split over the output labels (row-major in the order given), the contracted index over the
// contracted labels; LPO lanes share one output (strided over k, four independent partial
// sums per lane, then a shuffle reduction in a fixed order).  One launch replaces the
// permutes, the GEMM and the split-K reduction of the general path.
constexpr int kDirectMaxLabels = 8;
constexpr int64_t kDirectMaxMacs = int64_t(1) << 18;
constexpr int64_t kDirectMaxK = 4096;
struct DirectArgs {
  int no = 0, nk = 0;
  int odim[kDirectMaxLabels], oa[kDirectMaxLabels], ob[kDirectMaxLabels], oc[kDirectMaxLabels];
  int kdim[kDirectMaxLabels], ka[kDirectMaxLabels], kb[kDirectMaxLabels];
  int nout = 0, K = 0;
  double alpha = 1.0, beta = 0.0;
};

template <int LPO>
__global__ void __launch_bounds__(256) k_contract_direct(DirectArgs a, const double* __restrict__ A,
                                                         const double* __restrict__ B, double* C,
                                                         const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int o = t / LPO, lane = t % LPO;
  const bool valid = o < a.nout;   // every lane of a warp stays for the shuffle reduction
  int r = valid ? o : 0, aoff = 0, boff = 0, coff = 0;
  for (int i = a.no - 1; i >= 0; --i) {
    const int ci = r % a.odim[i];
    r /= a.odim[i];
    aoff += ci * a.oa[i];
    boff += ci * a.ob[i];
    coff += ci * a.oc[i];
  }
  auto term = [&](int k) {
    int rk = k, ka = 0, kb = 0;
    for (int j = a.nk - 1; j >= 0; --j) {
      const int cj = rk % a.kdim[j];
      rk /= a.kdim[j];
      ka += cj * a.ka[j];
      kb += cj * a.kb[j];
    }
    return make_int2(ka, kb);
  };
  double s0 = 0.0, s1 = 0.0, s2 = 0.0, s3 = 0.0;
  int k = valid ? lane : a.K;
  for (; k + 3 * LPO < a.K; k += 4 * LPO) {
    const int2 o0 = term(k), o1 = term(k + LPO), o2 = term(k + 2 * LPO), o3 = term(k + 3 * LPO);
    s0 = fma(__ldg(A + aoff + o0.x), __ldg(B + boff + o0.y), s0);
    s1 = fma(__ldg(A + aoff + o1.x), __ldg(B + boff + o1.y), s1);
    s2 = fma(__ldg(A + aoff + o2.x), __ldg(B + boff + o2.y), s2);
    s3 = fma(__ldg(A + aoff + o3.x), __ldg(B + boff + o3.y), s3);
  }
  for (; k < a.K; k += LPO) {
    const int2 o0 = term(k);
    s0 = fma(__ldg(A + aoff + o0.x), __ldg(B + boff + o0.y), s0);
  }
  double v = (s0 + s1) + (s2 + s3);
  for (int off = LPO / 2; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off, LPO);
  if (valid && lane == 0) C[coff] = (a.beta == 0.0) ? a.alpha * v : a.alpha * v + a.beta * C[coff];
}

void contract_direct(Ctx& c, DirectArgs& a, const double* A, const double* B, double* C) {
  ProfScope ps(c, KC_GEMM, 2.0 * double(a.nout) * double(a.K));
  if (a.K >= 32) {
    k_contract_direct<32><<<grid_for(int64_t(a.nout) * 32, 256), 256, 0, c.stream>>>(a, A, B, C, c.guard);
  } else if (a.K >= 8) {
    k_contract_direct<8><<<grid_for(int64_t(a.nout) * 8, 256), 256, 0, c.stream>>>(a, A, B, C, c.guard);
  } else {
    k_contract_direct<1><<<grid_for(int64_t(a.nout), 256), 256, 0, c.stream>>>(a, A, B, C, c.guard);
  }
  after_launch(c, "contract_direct");
}

}  // namespace

namespace {

struct GemmArgs {
  int64_t batch, M, N, K;
  double alpha;
  const double* A;
  int64_t sAb, sAm, sAk;
  const double* B;
  int64_t sBb, sBk, sBn;
  double beta;
  double* C;
  int64_t sCb, sCm, sCn;
};

struct Plan {
  int T;
  int64_t splits, kchunk;
  double cost;
};

// FP64-pipe tile plan of tile size T with a given number of k splits (0: the split-K choice of
// the cost model below).
Plan plan_fp64(const Ctx& c, const GemmArgs& g, int T, int64_t want_splits) {
  const int64_t target = 2 * int64_t(c.num_sms);
  Plan p;
  p.T = T;
  const int64_t tiles = ((g.M + T - 1) / T) * ((g.N + T - 1) / T) * g.batch;
  int64_t splits = 1;
  if (want_splits > 0) {
    splits = want_splits;
  } else if (tiles < target && g.K > 2 * GK) {
    int64_t want = (target + tiles - 1) / tiles;
    int64_t maxs = (g.K + 2 * GK - 1) / (2 * GK);   // at least 32 k per split
    splits = std::max<int64_t>(1, std::min<int64_t>(want, maxs));
  }
  int64_t kchunk = (g.K + splits - 1) / splits;
  kchunk = (kchunk + GK - 1) / GK * GK;
  splits = (g.K + kchunk - 1) / kchunk;
  p.splits = splits;
  p.kchunk = kchunk;
  const int64_t per_sm = (tiles * splits + c.num_sms - 1) / c.num_sms;
  p.cost = double(per_sm) * T * T * double(kchunk) / 2.0 + (splits > 1 ? 3000.0 : 0.0);
  return p;
}

// Tile and split-K choice of the cost model.  On GB300 an SM retires 2 FP64 FMAs per cycle, so
// the FP64 pipe, not shared-memory or L2 traffic, bounds these kernels at any tile size >= 16:
// the time is about the FMA load of the busiest SM, ceil(CTAs / SMs) T^2 kchunk / 2 cycles,
// plus one more launch when K is split.  Each tile size is planned with split-K up to two CTAs
// per SM (at least 2 GK of k per split); the cheapest plan wins, ties going to the larger tile.
Plan heuristic_plan(const Ctx& c, const GemmArgs& g) {
  Plan best = plan_fp64(c, g, 64, 0);
  for (int T : {32, 16}) {
    Plan p = plan_fp64(c, g, T, 0);
    if (p.cost < best.cost * 0.97) best = p;
  }
  return best;
}

void launch_fp64(Ctx& c, const GemmArgs& g, const Plan& best) {
  const int T = best.T;
  const int splits = int(best.splits);
  const int64_t kchunk = best.kchunk;
  const int64_t batch = g.batch, M = g.M, N = g.N, K = g.K;
  ProfScope ps(c, KC_GEMM, 2.0 * double(batch) * double(M) * double(N) * double(K));
  dim3 grid(unsigned((N + T - 1) / T), unsigned((M + T - 1) / T), unsigned(batch * splits));
  QTT_CHECK_ARG(grid.y <= 65535 && grid.z <= 65535, "gemm grid too large");
  dim3 block(16, 16);
  DBuf W;
  if (splits > 1) W.reset(&c, size_t(splits) * batch * M * N);
  double* Wp = splits > 1 ? W.p : nullptr;
  const int64_t ntiles = int64_t(grid.x) * grid.y * batch;
  int* ctr = (splits > 1 && c.tile_ctr && ntiles <= kTileCounters) ? c.tile_ctr : nullptr;
  if (T == 64)
    k_gemm<64><<<grid, block, 0, c.stream>>>(M, N, K, kchunk, splits, batch, g.alpha, g.A, g.sAb, g.sAm, g.sAk, g.B,
                                             g.sBb, g.sBk, g.sBn, g.beta, g.C, g.sCb, g.sCm, g.sCn, Wp, ctr, c.guard);
  else if (T == 32)
    k_gemm<32><<<grid, block, 0, c.stream>>>(M, N, K, kchunk, splits, batch, g.alpha, g.A, g.sAb, g.sAm, g.sAk, g.B,
                                             g.sBb, g.sBk, g.sBn, g.beta, g.C, g.sCb, g.sCm, g.sCn, Wp, ctr, c.guard);
  else
    k_gemm<16><<<grid, block, 0, c.stream>>>(M, N, K, kchunk, splits, batch, g.alpha, g.A, g.sAb, g.sAm, g.sAk, g.B,
                                             g.sBb, g.sBk, g.sBn, g.beta, g.C, g.sCb, g.sCm, g.sCn, Wp, ctr, c.guard);
  after_launch(c, "gemm");
  if (splits > 1 && !ctr) {
    k_splitk_reduce<<<grid_for(batch * M * N, 256), 256, 0, c.stream>>>(batch, M, N, splits, g.alpha, W.p, g.beta,
                                                                        g.C, g.sCb, g.sCm, g.sCn, c.guard);
    after_launch(c, "splitk_reduce");
  }
}

GemmKey gemm_key(const Ctx& c, const GemmArgs& g) {
  return GemmKey{int64_t(c.root->gemm_mode), g.batch, g.M, g.N, g.K, g.sAb, g.sAm, g.sAk, g.sBb, g.sBk, g.sBn,
                 g.sCb, g.sCm, g.sCn, g.beta == 0.0 ? 0 : 1, int64_t(c.root->digits)};
}

// Largest element offset + 1 of a strided view (non-negative strides).
int64_t view_span(int64_t n0, int64_t s0, int64_t n1, int64_t s1, int64_t n2, int64_t s2) {
  return (n0 - 1) * s0 + (n1 - 1) * s1 + (n2 - 1) * s2 + 1;
}

// Times every candidate engine of one GEMM shape and returns the fastest: the FP64-pipe kernel
// at tile sizes 64, 32 and 16 (split-K as the cost model plans it, and unsplit), and the
// digit-split tensor-core product where the shape allows it.  The trials run on the tuner's
// own stream (outside any capture, so a step being captured is not disturbed) over scratch
// operands of the same shape and strides filled with constants; each candidate runs once to
// warm up, then three times between events, and keeps its fastest time.
GemmPick tune_gemm(Ctx& c, const GemmArgs& g, bool oz_ok) {
  Ctx& r = *c.root;
  GemmPick none{-1, 0, 0, 0.0, 0.0};
  if (g.sAb < 0 || g.sAm < 0 || g.sAk < 0 || g.sBb < 0 || g.sBk < 0 || g.sBn < 0 || g.sCb < 0 || g.sCm < 0 ||
      g.sCn < 0)
    return none;   // negative strides: the cost model decides
  if (!r.tune_stream) {
    QTT_CUDA(cudaStreamCreateWithFlags(&r.tune_stream, cudaStreamNonBlocking));
    QTT_CUDA(cudaMalloc(&r.tune_ctr, kTileCounters * sizeof(int)));
    QTT_CUDA(cudaMemsetAsync(r.tune_ctr, 0, kTileCounters * sizeof(int), r.tune_stream));
    QTT_CUDA(cudaEventCreate(&r.tune_ev[0]));
    QTT_CUDA(cudaEventCreate(&r.tune_ev[1]));
  }
  const int64_t na = view_span(g.batch, g.sAb, g.M, g.sAm, g.K, g.sAk);
  const int64_t nb = view_span(g.batch, g.sBb, g.K, g.sBk, g.N, g.sBn);
  const int64_t nc = view_span(g.batch, g.sCb, g.M, g.sCm, g.N, g.sCn);
  const size_t need = size_t(na + nb + nc);
  if (need > r.tune_cap) {
    QTT_CUDA(cudaStreamSynchronize(r.tune_stream));
    if (r.tune_buf) QTT_CUDA(cudaFree(r.tune_buf));
    r.tune_buf = nullptr;
    r.tune_cap = 0;
    QTT_CUDA(cudaMalloc(&r.tune_buf, need * sizeof(double)));
    r.tune_cap = need;
  }
  // a context of its own for the trials: the tuner's stream, pool and counters, no guard, no
  // profiling (a block of the context's pool may still be in use by work queued on its stream)
  if (!r.tune_pool) r.tune_pool = new Pool(r.alloc_fn, r.free_fn, r.alloc_user);
  Ctx t;
  t.device = c.device;
  t.stream = r.tune_stream;
  t.pool = r.tune_pool;
  t.num_sms = c.num_sms;
  t.root = &t;
  t.gemm_mode = r.gemm_mode;
  t.digits = r.digits;
  t.tile_ctr = r.tune_ctr;
  double* A = r.tune_buf;
  double* B = A + na;
  double* C = B + nb;
  fill(t, A, na, 0.75);
  fill(t, B, nb, -1.25);
  fill(t, C, nc, 0.5);
  GemmArgs h = g;
  h.A = A; h.B = B; h.C = C;
  auto time_of = [&](auto&& launch) {
    launch();
    float best = 1e30f;
    for (int rep = 0; rep < 3; ++rep) {
      QTT_CUDA(cudaEventRecord(r.tune_ev[0], t.stream));
      launch();
      QTT_CUDA(cudaEventRecord(r.tune_ev[1], t.stream));
      QTT_CUDA(cudaEventSynchronize(r.tune_ev[1]));
      float ms = 0.f;
      QTT_CUDA(cudaEventElapsedTime(&ms, r.tune_ev[0], r.tune_ev[1]));
      best = std::min(best, ms);
    }
    return double(best) * 1e6;   // ns
  };
  GemmPick pick{0, 64, 0, 1e300, 0.0};
  const Plan def = heuristic_plan(t, h);
  for (int T : {64, 32, 16}) {
    Plan pm = plan_fp64(t, h, T, 0);
    for (int64_t sp : {pm.splits, int64_t(1)}) {
      const Plan p = plan_fp64(t, h, T, sp);
      const double ns = time_of([&] { launch_fp64(t, h, p); });
      if (p.T == def.T && p.splits == def.splits) pick.default_ns = ns;
      if (ns < pick.best_ns) pick = GemmPick{0, p.T, p.splits, ns, pick.default_ns};
      if (pm.splits == 1) break;
    }
  }
  if (oz_ok) {
    const double ns = time_of([&] {
      gemm_ozaki(t, h.batch, h.M, h.N, h.K, h.alpha, h.A, h.sAb, h.sAm, h.sAk, h.B, h.sBb, h.sBk, h.sBn, h.beta, h.C,
                 h.sCb, h.sCm, h.sCn);
    });
    if (h.batch * h.M * h.N * h.K >= (int64_t(1) << 23)) pick.default_ns = ns;   // the cost model's engine
    if (ns < pick.best_ns) pick = GemmPick{1, 0, 0, ns, pick.default_ns};
  }
  QTT_CUDA(cudaStreamSynchronize(t.stream));
  r.tune_trials += 1;
  return pick;
}

}  // namespace

void gemm(Ctx& c, int64_t batch, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
          int64_t sAb, int64_t sAm, int64_t sAk, const double* B, int64_t sBb, int64_t sBk,
          int64_t sBn, double beta, double* C, int64_t sCb, int64_t sCm, int64_t sCn) {
  if (batch <= 0 || M <= 0 || N <= 0) return;
  if (K <= 0) {  // C = beta C
    if (beta == 1.0) return;
    // treat as a split-K reduction over zero partial sums
    DBuf W(&c, size_t(batch * M * N));
    fill(c, W.p, batch * M * N, 0.0);
    k_splitk_reduce<<<grid_for(batch * M * N, 256), 256, 0, c.stream>>>(batch, M, N, 1, alpha, W.p, beta, C, sCb, sCm, sCn, c.guard);
    after_launch(c, "splitk_reduce");
    return;
  }
  auto span = [](int64_t n0, int64_t s0, int64_t n1, int64_t s1, int64_t n2, int64_t s2) {
    return (n0 - 1) * std::abs(s0) + (n1 - 1) * std::abs(s1) + (n2 - 1) * std::abs(s2);
  };
  const int64_t kIntMax = (int64_t(1) << 31) - 1;
  if (batch * M * N * K <= kDirectMaxMacs && K <= kDirectMaxK && span(batch, sAb, M, sAm, K, sAk) < kIntMax &&
      span(batch, sBb, K, sBk, N, sBn) < kIntMax && span(batch, sCb, M, sCm, N, sCn) < kIntMax) {
    DirectArgs a;
    a.no = 3; a.nk = 1;
    a.odim[0] = int(batch); a.odim[1] = int(M); a.odim[2] = int(N);
    a.oa[0] = int(sAb); a.oa[1] = int(sAm); a.oa[2] = 0;
    a.ob[0] = int(sBb); a.ob[1] = 0; a.ob[2] = int(sBn);
    a.oc[0] = int(sCb); a.oc[1] = int(sCm); a.oc[2] = int(sCn);
    a.kdim[0] = int(K); a.ka[0] = int(sAk); a.kb[0] = int(sBk);
    a.nout = int(batch * M * N); a.K = int(K);
    a.alpha = alpha; a.beta = beta;
    contract_direct(c, a, A, B, C);
    return;
  }
  const GemmArgs g{batch, M, N, K, alpha, A, sAb, sAm, sAk, B, sBb, sBk, sBn, beta, C, sCb, sCm, sCn};
  const bool oz_ok = c.root->gemm_mode != 1 && M >= 16 && N >= 16 && K >= 16;
  Ctx& r = *c.root;
  if (r.digits < kDigitsFP64 && M >= 16 && N >= 16 && K >= 16) {   // reduced contraction precision
    gemm_ozaki(c, batch, M, N, K, alpha, A, sAb, sAm, sAk, B, sBb, sBk, sBn, beta, C, sCb, sCm, sCn);
    return;
  }
  if (r.autotune || !r.tuned.empty()) {
    const GemmKey key = gemm_key(c, g);
    auto it = r.tuned.find(key);
    if (it == r.tuned.end() && r.autotune) it = r.tuned.emplace(key, tune_gemm(c, g, oz_ok)).first;
    if (it != r.tuned.end()) {
      const GemmPick& pk = it->second;
      if (pk.engine == 1 && oz_ok) {
        gemm_ozaki(c, batch, M, N, K, alpha, A, sAb, sAm, sAk, B, sBb, sBk, sBn, beta, C, sCb, sCm, sCn);
        return;
      }
      if (pk.engine == 0) {
        launch_fp64(c, g, plan_fp64(c, g, pk.T, pk.splits));
        return;
      }
    }
  }
  if (oz_ok && batch * M * N * K >= (int64_t(1) << 23)) {
    gemm_ozaki(c, batch, M, N, K, alpha, A, sAb, sAm, sAk, B, sBb, sBk, sBn, beta, C, sCb, sCm, sCn);
    return;
  }
  launch_fp64(c, g, heuristic_plan(c, g));
}

// ------------------------------------------------------------------ GEMM autotuner

int prec_digits(int prec) {
  switch (prec) {
    case QTT_PREC_FP64: return kDigitsFP64;
    case QTT_PREC_FP32: return 3;
    case QTT_PREC_TF32: return 2;
    case QTT_PREC_BF16: return 1;
    default: throw Error(QTT_ERR_ARG, "precision must be QTT_PREC_FP64, _FP32, _TF32 or _BF16");
  }
}

void free_autotuner(Ctx& c) {
  if (c.tune_stream) cudaStreamSynchronize(c.tune_stream);
  if (c.tune_buf) cudaFree(c.tune_buf);
  if (c.tune_ctr) cudaFree(c.tune_ctr);
  for (auto& e : c.tune_ev)
    if (e) cudaEventDestroy(e);
  if (c.tune_stream) cudaStreamDestroy(c.tune_stream);
  delete c.tune_pool;
  c.tune_pool = nullptr;
  c.tune_buf = nullptr;
  c.tune_ctr = nullptr;
  c.tune_stream = nullptr;
  c.tune_cap = 0;
}

int64_t autotune_table(Ctx& c, int64_t max_rows, int64_t* rows) {
  Ctx& r = *c.root;
  int64_t i = 0;
  for (const auto& kv : r.tuned) {
    if (rows && i < max_rows) {
      int64_t* o = rows + i * kTuneRow;
      o[0] = kv.first[1]; o[1] = kv.first[2]; o[2] = kv.first[3]; o[3] = kv.first[4];
      o[4] = kv.second.engine; o[5] = kv.second.T; o[6] = kv.second.splits;
      o[7] = int64_t(kv.second.best_ns); o[8] = int64_t(kv.second.default_ns);
    }
    ++i;
  }
  return i;
}

// ------------------------------------------------------------------ permute / elementwise

namespace {

struct PermArgs {
  int nd;
  int64_t out_dim[8];
  int64_t in_stride[8];  // stride in the input of output axis i
};

__global__ void k_permute(const double* __restrict__ in, double* __restrict__ out, int64_t total, PermArgs a,
                          double alpha, double beta, const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    int64_t r = e, off = 0;
    for (int i = a.nd - 1; i >= 0; --i) {
      int64_t idx = r % a.out_dim[i];
      r /= a.out_dim[i];
      off += idx * a.in_stride[i];
    }
    double v = alpha * in[off];
    out[e] = (beta == 0.0) ? v : v + beta * out[e];
  }
}

__global__ void k_fill(double* x, int64_t n, double v) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x) x[e] = v;
}

__global__ void k_axpby(int64_t n, double a, const double* __restrict__ x, double b, double* __restrict__ y,
                        const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    y[e] = (b == 0.0) ? a * x[e] : a * x[e] + b * y[e];
}

// One block; fixed reduction tree, so the result is bitwise reproducible.
__global__ void __launch_bounds__(1024) k_dot(int64_t n, const double* __restrict__ x, const double* __restrict__ y,
                                              double* out) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t e = threadIdx.x; e < n; e += blockDim.x) s = fma(x[e], y[e], s);
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    s = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) *out = s;
  }
}

}  // namespace

void permute(Ctx& c, const double* in, int nd, const int64_t* in_dim, const int* perm, double* out, double alpha,
             double beta) {
  PermArgs a;
  a.nd = nd;
  int64_t stride[8];
  int64_t s = 1;
  for (int i = nd - 1; i >= 0; --i) { stride[i] = s; s *= in_dim[i]; }
  for (int i = 0; i < nd; ++i) { a.out_dim[i] = in_dim[perm[i]]; a.in_stride[i] = stride[perm[i]]; }
  int64_t total = s;
  if (total == 0) return;
  k_permute<<<grid_for(total, 256), 256, 0, c.stream>>>(in, out, total, a, alpha, beta, c.guard);
  after_launch(c, "permute");
}

void fill(Ctx& c, double* x, int64_t n, double v) {
  if (n <= 0) return;
  k_fill<<<grid_for(n, 256), 256, 0, c.stream>>>(x, n, v);
  after_launch(c, "fill");
}

void copy(Ctx& c, double* dst, const double* src, int64_t n) {
  if (n <= 0) return;
  QTT_CUDA(cudaMemcpyAsync(dst, src, size_t(n) * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
}

void axpby(Ctx& c, int64_t n, double a, const double* x, double b, double* y) {
  if (n <= 0) return;
  k_axpby<<<grid_for(n, 256), 256, 0, c.stream>>>(n, a, x, b, y, c.guard);
  after_launch(c, "axpby");
}

void dot(Ctx& c, int64_t n, const double* x, const double* y, double* out_dev) {
  k_dot<<<1, 1024, 0, c.stream>>>(n, x, y, out_dev);
  after_launch(c, "dot");
}

// ------------------------------------------------------------------ einsum planner

namespace {

struct Lab {
  char l;
  int64_t d;
};

std::vector<char> labels(const std::string& s) { return std::vector<char>(s.begin(), s.end()); }

int find(const std::vector<char>& v, char l) {
  for (size_t i = 0; i < v.size(); ++i)
    if (v[i] == l) return int(i);
  return -1;
}

// Is the label order of `have` equal to the concatenation g1 + g2 + g3?
bool is_order(const std::vector<char>& have, const std::vector<char>& g1, const std::vector<char>& g2,
              const std::vector<char>& g3) {
  std::vector<char> w(g1);
  w.insert(w.end(), g2.begin(), g2.end());
  w.insert(w.end(), g3.begin(), g3.end());
  return w == have;
}

// Permutation taking `from` label order to `to` label order: perm[i] = axis of to[i] in from.
std::vector<int> perm_of(const std::vector<char>& from, const std::vector<char>& to) {
  std::vector<int> p(to.size());
  for (size_t i = 0; i < to.size(); ++i) p[i] = find(from, to[i]);
  return p;
}

std::vector<char> cat3(const std::vector<char>& a, const std::vector<char>& b, const std::vector<char>& c) {
  std::vector<char> w(a);
  w.insert(w.end(), b.begin(), b.end());
  w.insert(w.end(), c.begin(), c.end());
  return w;
}

}  // namespace

void einsum(Ctx& c, const char* spec, double alpha, const TV& A, const TV& B, double beta, const TV& C) {
  std::string s(spec);
  size_t comma = s.find(','), arrow = s.find("->");
  QTT_CHECK_ARG(comma != std::string::npos && arrow != std::string::npos, "einsum spec");
  auto la = labels(s.substr(0, comma)), lb = labels(s.substr(comma + 1, arrow - comma - 1)),
       lc = labels(s.substr(arrow + 2));
  QTT_CHECK_ARG(int(la.size()) == A.nd && int(lb.size()) == B.nd && int(lc.size()) == C.nd,
                std::string("einsum rank mismatch: ") + spec);
  std::map<char, int64_t> dim;
  auto reg = [&](const std::vector<char>& l, const TV& t) {
    for (size_t i = 0; i < l.size(); ++i) {
      auto it = dim.find(l[i]);
      if (it == dim.end()) dim[l[i]] = t.dim[i];
      else QTT_CHECK_ARG(it->second == t.dim[i], std::string("einsum dim mismatch: ") + spec);
    }
  };
  reg(la, A); reg(lb, B); reg(lc, C);
  std::vector<char> batch, fa, fb, kk;
  for (char l : lc) {
    bool ia = find(la, l) >= 0, ib = find(lb, l) >= 0;
    QTT_CHECK_ARG(ia || ib, std::string("einsum output label not in inputs: ") + spec);
    if (ia && ib) batch.push_back(l);
    else if (ia) fa.push_back(l);
    else fb.push_back(l);
  }
  for (char l : la)
    if (find(lc, l) < 0) {
      QTT_CHECK_ARG(find(lb, l) >= 0, std::string("einsum: label summed in one operand only: ") + spec);
      kk.push_back(l);
    }
  for (char l : lb)
    if (find(lc, l) < 0) QTT_CHECK_ARG(find(la, l) >= 0, std::string("einsum: label summed in one operand only: ") + spec);
  auto prod = [&](const std::vector<char>& g) {
    int64_t p = 1;
    for (char l : g) p *= dim[l];
    return p;
  };
  int64_t Bt = prod(batch), M = prod(fa), N = prod(fb), K = prod(kk);
  if (Bt == 0 || M == 0 || N == 0) return;
  if (K >= 1 && Bt * M * N * K <= kDirectMaxMacs && K <= kDirectMaxK && lc.size() <= size_t(kDirectMaxLabels) &&
      kk.size() <= size_t(kDirectMaxLabels)) {
    // small problem: one direct launch, operands read in place
    auto stride_in = [&](const std::vector<char>& l, const TV& t, char x) -> int {
      int64_t st = 1;
      for (int i = int(l.size()) - 1; i >= 0; --i) {
        if (l[i] == x) return int(st);
        st *= t.dim[i];
      }
      return 0;
    };
    DirectArgs a;
    a.no = int(lc.size());
    for (int i = 0; i < a.no; ++i) {
      a.odim[i] = int(dim[lc[i]]);
      a.oa[i] = stride_in(la, A, lc[i]);
      a.ob[i] = stride_in(lb, B, lc[i]);
      a.oc[i] = stride_in(lc, C, lc[i]);
    }
    a.nk = int(kk.size());
    for (int j = 0; j < a.nk; ++j) {
      a.kdim[j] = int(dim[kk[j]]);
      a.ka[j] = stride_in(la, A, kk[j]);
      a.kb[j] = stride_in(lb, B, kk[j]);
    }
    a.nout = int(Bt * M * N);
    a.K = int(K);
    a.alpha = alpha;
    a.beta = beta;
    contract_direct(c, a, A.p, B.p, C.p);
    return;
  }
  // The contracted labels may be taken in the order of A or of B: pick the order that lets
  // both operands be read in place, if any.
  std::vector<char> kkB;
  for (char l : lb)
    if (find(kk, l) >= 0) kkB.push_back(l);
  auto fitsA = [&](const std::vector<char>& k) { return is_order(la, batch, fa, k) || is_order(la, batch, k, fa); };
  auto fitsB = [&](const std::vector<char>& k) { return is_order(lb, batch, k, fb) || is_order(lb, batch, fb, k); };
  if (!(fitsA(kk) && fitsB(kk)) && fitsA(kkB) && fitsB(kkB)) kk = kkB;
  else if (!fitsA(kk) && !fitsB(kk) && (fitsA(kkB) || fitsB(kkB))) kk = kkB;
  // --- operand A: [batch][fa][k] (row-major M x K) or [batch][k][fa] (K x M)
  const double* Ap = A.p;
  DBuf Atmp;
  int64_t sAm, sAk;
  if (is_order(la, batch, fa, kk)) { sAm = K; sAk = 1; }
  else if (is_order(la, batch, kk, fa)) { sAm = 1; sAk = M; }
  else {
    Atmp.reset(&c, size_t(A.size()));
    auto p = perm_of(la, cat3(batch, fa, kk));
    permute(c, A.p, A.nd, A.dim, p.data(), Atmp.p, 1.0, 0.0);
    Ap = Atmp.p; sAm = K; sAk = 1;
  }
  // --- operand B: [batch][k][fb] (K x N) or [batch][fb][k]
  const double* Bp = B.p;
  DBuf Btmp;
  int64_t sBk, sBn;
  if (is_order(lb, batch, kk, fb)) { sBk = N; sBn = 1; }
  else if (is_order(lb, batch, fb, kk)) { sBk = 1; sBn = K; }
  else {
    Btmp.reset(&c, size_t(B.size()));
    auto p = perm_of(lb, cat3(batch, kk, fb));
    permute(c, B.p, B.nd, B.dim, p.data(), Btmp.p, 1.0, 0.0);
    Bp = Btmp.p; sBk = N; sBn = 1;
  }
  // --- output C: [batch][fa][fb] or [batch][fb][fa]; otherwise a temporary + permute
  if (is_order(lc, batch, fa, fb)) {
    gemm(c, Bt, M, N, K, alpha, Ap, M * K, sAm, sAk, Bp, K * N, sBk, sBn, beta, C.p, M * N, N, 1);
  } else if (is_order(lc, batch, fb, fa)) {
    gemm(c, Bt, M, N, K, alpha, Ap, M * K, sAm, sAk, Bp, K * N, sBk, sBn, beta, C.p, M * N, 1, M);
  } else {
    DBuf Ct(&c, size_t(Bt * M * N));
    gemm(c, Bt, M, N, K, 1.0, Ap, M * K, sAm, sAk, Bp, K * N, sBk, sBn, 0.0, Ct.p, M * N, N, 1);
    auto from = cat3(batch, fa, fb);
    int64_t fdim[8];
    for (size_t i = 0; i < from.size(); ++i) fdim[i] = dim[from[i]];
    auto p = perm_of(from, lc);
    permute(c, Ct.p, int(from.size()), fdim, p.data(), C.p, alpha, beta);
  }
}

}  // namespace qtt
