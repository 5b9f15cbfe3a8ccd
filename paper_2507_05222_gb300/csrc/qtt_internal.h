// Internal declarations of the QTT GB300 library (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>
#include <array>
#include <map>
#include <stdexcept>
#include <string>
#include <vector>

#include "../../include/qtt.h"

namespace qtt {

// ------------------------------------------------------------------ errors

struct Error : std::runtime_error {
  int code;
  Error(int c, const std::string& m) : std::runtime_error(m), code(c) {}
};

void set_last_error(const std::string& msg);

#define QTT_CHECK_ARG(cond, msg)                                   \
  do {                                                             \
    if (!(cond)) throw ::qtt::Error(QTT_ERR_ARG, std::string(msg)); \
  } while (0)

#define QTT_CUDA(call)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      throw ::qtt::Error(QTT_ERR_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// ------------------------------------------------------------------ device memory pool

// Stream-ordered pool: every allocation and every kernel of a context use one stream, so a
// block freed on the host can be handed out again at once (work that uses the new owner is
// enqueued after the work of the old owner).  Large chunks come from the user allocator.
class Pool {
 public:
  Pool(qtt_alloc_fn a, qtt_free_fn f, void* user) : alloc_(a), free_(f), user_(user) {}
  ~Pool();
  void* get(size_t bytes);
  void put(void* p);
  size_t held() const { return held_; }
  // CUDA-graph capture: blocks handed out while capturing form an arena owned by the graph
  // being captured (key: its owner, one arena per captured case), reused among themselves
  // by later captures of the same owner and never handed to anyone else, so the graphs of
  // different cases may replay concurrently.  Blocks from before the capture that are freed
  // during it return to the ordinary free list only when the capture ends.
  // release_capture(owner) gives that owner's arena back once its graph is destroyed and its
  // last replay has finished.
  void begin_capture(const void* owner);
  void end_capture();
  void release_capture(const void* owner);

 private:
  static size_t size_class(size_t bytes);
  void* raw_alloc(size_t bytes);
  qtt_alloc_fn alloc_;
  qtt_free_fn free_;
  void* user_;
  std::multimap<size_t, void*> free_blocks_;  // class size -> block
  std::map<void*, size_t> live_;              // block -> class size
  const void* capturing_ = nullptr;           // owner of the capture in progress
  std::map<const void*, std::multimap<size_t, void*>> cap_free_;  // owner -> free arena blocks
  std::map<void*, const void*> cap_owned_;    // every arena block -> its owner
  std::vector<void*> deferred_;
  std::vector<std::pair<void*, size_t>> chunks_;
  char* cur_ = nullptr;
  size_t cur_left_ = 0;
  size_t held_ = 0;
};

struct Ctx;

// RAII device buffer from the context pool.
struct DBuf {
  Ctx* ctx = nullptr;
  double* p = nullptr;
  size_t n = 0;
  DBuf() = default;
  DBuf(Ctx* c, size_t count);
  ~DBuf();
  DBuf(const DBuf&) = delete;
  DBuf& operator=(const DBuf&) = delete;
  DBuf(DBuf&& o) noexcept : ctx(o.ctx), p(o.p), n(o.n) { o.p = nullptr; o.n = 0; }
  DBuf& operator=(DBuf&& o) noexcept;
  void reset(Ctx* c, size_t count);
};

// Kernel classes for the optional per-class timing (CUDA events around each launch).
enum KClass {
  KC_GEMM = 0, KC_QR = 1, KC_EIG = 2, KC_CG = 3, KC_OTHER = 4,
  // phases of the fractional step (nested around the kernels above)
  KC_PH_APPLY = 5, KC_PH_RHS = 6 /* with the momentum solves */, KC_PH_MOM = 7, KC_PH_POI = 8, KC_PH_PROJ = 9,
  KC_N = 10
};

constexpr int KC_KERNEL_CLASSES = KC_PH_APPLY;       // classes 0..4 are kernel classes
constexpr int KC_PHASES = KC_N - KC_PH_APPLY;         // classes 5..9 are step phases

struct Profiler {
  struct Span {
    cudaEvent_t e0, e1;
    int phase;  // step phase open when the span was enqueued (-1: none)
  };
  bool on = false;
  int phase = -1;
  std::vector<cudaEvent_t> free_events;
  std::vector<Span> pending[KC_N];
  double flops[KC_N] = {0};
  int64_t launches[KC_N] = {0};
  // Kernel-class time (ms) and launch counts split by step phase, filled by the last
  // read-out; row KC_PHASES collects what ran outside any phase.
  double phase_ms[KC_PHASES + 1][KC_KERNEL_CLASSES] = {};
  int64_t phase_launches[KC_PHASES + 1] = {0};
  int64_t acc_phase_launches[KC_PHASES + 1] = {0};
  // Flops of the cooperative CG solves, counted on the device (their iteration counts are
  // data dependent); one double of device memory, allocated when profiling is first turned on.
  double* dev_flops = nullptr;
};

// GEMM autotuner (qtt_dense.cu): shape key (gemm mode, batch, M, N, K, the nine strides,
// beta != 0, digits) and the engine picked for it by timing.
using GemmKey = std::array<int64_t, 16>;
struct GemmPick {
  int engine;          // 0 FP64-pipe tiles, 1 digit-split tensor-core product, -1 not tuned
  int T;               // FP64 tile size
  int64_t splits;      // FP64 k splits
  double best_ns;      // time of the pick
  double default_ns;   // time of the cost model's choice
};
constexpr int kTuneRow = 9;   // batch, M, N, K, engine, T, splits, best_ns, default_ns

struct Ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  Pool* pool = nullptr;
  int64_t launches = 0;
  int num_sms = 152;
  // Worker contexts run independent parts of a step concurrently: each has its own stream
  // and its own stream-ordered pool; `root` is the context the caller created (launch count
  // and profiler live there).  Outputs that cross streams are allocated from the parent
  // before fork(), so the fork event orders any earlier use of that memory.
  Ctx* root = nullptr;
  std::vector<Ctx*> workers;
  cudaEvent_t ev_fork = nullptr;
  std::vector<cudaEvent_t> ev_join;
  qtt_alloc_fn alloc_fn = nullptr;
  qtt_free_fn free_fn = nullptr;
  void* alloc_user = nullptr;
  // When non-null, GEMM / permute / reduction kernels read *guard first and return at once
  // if it is 0.  Set around the matrix-vector products of a CG solve so that iterations past
  // convergence cost only their launches (the iteration budget is fixed on the host).
  const int* guard = nullptr;
  // ALS local solves: 0 = one cooperative kernel per solve where the shapes allow it,
  // 1 = one kernel per contraction and CG update (read from the root context).
  int cg_mode = 0;
  // Matrix products: 0 = products of >= 2^23 multiply-adds on the tensor cores (digit
  // splitting, see qtt_ozaki.cu; engine kDigitProductsOnTc05), the rest on the FP64 pipe;
  // 1 = everything on the FP64 pipe; 2 = digit products on mma.sync; 3 = digit products on tcgen05.
  int gemm_mode = 0;
  // Digits of each operand the digit-split products keep (read from the root): kDigitsFP64 =
  // exact FP64 products; 3, 2, 1 = the reduced contraction precisions (QTT_PREC_FP32, _TF32,
  // _BF16), which also send every batched GEMM with M, N, K >= 16 to the digit-split product.
  int digits = 7;
  // Per-tile arrival counters of split-K GEMMs on this context's stream (kTileCounters ints,
  // zero between launches: the last CTA of a tile resets its counter).
  int* tile_ctr = nullptr;
  // Stream on which the body of a conditional graph node (the ALS sweep loop) is captured.
  cudaStream_t side = nullptr;
  // When non-null, every TT-SVD cut of a rounding adds its discarded sigma^2 here (device).
  double* disc_acc = nullptr;
  // Limit of every bounded device wait (grid barriers of the cooperative CG), read from root.
  unsigned long long wait_ns = 2000000000ull;
  Profiler prof;
  // GEMM autotuner (root context): when autotune is on, a GEMM shape met for the first time is
  // timed under every candidate engine on tune_stream and the fastest is kept in tuned; shapes
  // in tuned use their pick whether or not tuning is still on (also inside graph captures).
  bool autotune = false;
  std::map<GemmKey, GemmPick> tuned;
  int64_t tune_trials = 0;
  cudaStream_t tune_stream = nullptr;
  cudaEvent_t tune_ev[2] = {nullptr, nullptr};
  int* tune_ctr = nullptr;
  double* tune_buf = nullptr;
  size_t tune_cap = 0;
  Pool* tune_pool = nullptr;   // scratch of the trials: used on tune_stream only (the pools are stream-ordered)
};
// Rows of the autotuner's table (kTuneRow int64 each, at most max_rows written); returns the
// number of tuned shapes.
int64_t autotune_table(Ctx& c, int64_t max_rows, int64_t* rows);
void free_autotuner(Ctx& c);

constexpr int kTileCounters = 16384;
constexpr int kDigitsFP64 = 7;
int prec_digits(int prec);   // QTT_PREC_* -> digits (throws QTT_ERR_ARG for another value)

// Sets the root context's contraction digits for a scope (FP64 regions inside a reduced-
// precision step: eigen and QR refinement products, the Poisson phase).
struct DigitsScope {
  Ctx& r;
  int saved;
  DigitsScope(Ctx& c, int d) : r(*c.root), saved(c.root->digits) { r.digits = d; }
  ~DigitsScope() { r.digits = saved; }
};
void init_tile_counters(Ctx& c);   // allocate and zero c.tile_ctr (outside stream capture of c.stream)
void free_tile_counters(Ctx& c);

void after_launch(Ctx& c, const char* what);

Ctx& worker(Ctx& c, int i);     // i-th worker of c (created on first use)
void fork(Ctx& c, int n);       // workers 0..n-1 wait for the work enqueued on c so far
void join(Ctx& c, int n);       // c waits for everything enqueued on workers 0..n-1
void destroy_workers(Ctx& c);

// RAII bracket of one launch (or launch group) of class k when profiling is on.
struct ProfScope {
  Ctx& c;
  int k;
  cudaEvent_t e0 = nullptr;
  ProfScope(Ctx& ctx, int kclass, double flops = 0.0);
  ~ProfScope();
};

// ------------------------------------------------------------------ handles

}  // namespace qtt

struct qtt_mps {
  qtt::Ctx* ctx = nullptr;
  int n = 0, d = 2;
  std::vector<int> bonds;       // n + 1
  std::vector<int64_t> off;     // n + 1 offsets in doubles (off[n] = total)
  qtt::DBuf buf;
  double* core(int k) const { return buf.p + off[k]; }
  int64_t core_size(int k) const { return off[k + 1] - off[k]; }
};

struct qtt_mpo {
  qtt::Ctx* ctx = nullptr;
  int n = 0, d = 2;
  std::vector<int> bonds;
  std::vector<int64_t> off;
  qtt::DBuf buf;
  double* core(int k) const { return buf.p + off[k]; }
};

namespace qtt {

// Allocate an MPS with the given bonds (uninitialised cores).
qtt_mps* new_mps(Ctx* c, int n, int d, const std::vector<int>& bonds);
qtt_mpo* new_mpo(Ctx* c, int n, int d, const std::vector<int>& bonds);
void free_mps(qtt_mps* x);
void free_mpo(qtt_mpo* m);

// ------------------------------------------------------------------ tensor views and kernels

struct TV {            // row-major dense tensor view on the device
  double* p = nullptr;
  int nd = 0;
  int64_t dim[8] = {0};
  int64_t size() const {
    int64_t s = 1;
    for (int i = 0; i < nd; ++i) s *= dim[i];
    return s;
  }
};
TV tv(double* p, std::initializer_list<int64_t> dims);

// C = alpha * einsum(spec, A, B) + beta * C.  spec like "ab,bc->ac" (single-letter labels).
void einsum(Ctx& c, const char* spec, double alpha, const TV& A, const TV& B, double beta, const TV& C);

// Batched strided GEMM: C[b](m,n) = alpha sum_k A[b](m,k) B[b](k,n) + beta C[b](m,n).
void gemm(Ctx& c, int64_t batch, int64_t M, int64_t N, int64_t K, double alpha, const double* A,
          int64_t sAb, int64_t sAm, int64_t sAk, const double* B, int64_t sBb, int64_t sBk,
          int64_t sBn, double beta, double* C, int64_t sCb, int64_t sCm, int64_t sCn);

// out = alpha * permute(in) + beta * out; perm[i] = input axis of output axis i.
void permute(Ctx& c, const double* in, int nd, const int64_t* in_dim, const int* perm, double* out,
             double alpha, double beta);

// Elementwise helpers (device pointers, count n).
void fill(Ctx& c, double* x, int64_t n, double v);
// FP64-accurate product on the bf16 tensor cores (qtt_ozaki.cu); same arguments as gemm.
void gemm_ozaki(Ctx& c, int64_t batch, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sAb,
                int64_t sAm, int64_t sAk, const double* B, int64_t sBb, int64_t sBk, int64_t sBn, double beta,
                double* C, int64_t sCb, int64_t sCm, int64_t sCn);
void init_ozaki_attributes();   // kernel attributes, once (before any stream capture)
// The digit products of gemm_ozaki on the fifth-generation tensor cores (qtt_tc05.cu): the
// engine of gemm mode 0 when true, for every FP64 product whose padded k is a multiple of 16
// (mode 3 forces it, mode 2 forces the mma.sync kernel; the two give bit-identical results).
constexpr bool kDigitProductsOnTc05 = true;
void init_tc05_attributes();     // kernel attributes and the tensor-map encoder, once
bool tc05_fits(int64_t Kp);
void oz_gemm_tc05(Ctx& c, int64_t batch, int64_t M, int64_t N, int64_t Kp, int splits, int64_t ksplit,
                  const void* As, const int* ea, const void* Bs, const int* eb, double alpha, double beta, double* C,
                  int64_t sCb, int64_t sCm, int64_t sCn, double* W);
// Seven bf16 digit slices out[s][r][Kp] and scale exponents ex[r] of the R rows of X (K values
// each, strides sR, sK), as the tensor-core products use them (qtt_ozaki.cu).
void oz_split_rows(Ctx& c, int64_t R, int64_t K, int64_t Kp, const double* X, int64_t sR, int64_t sK, void* out,
                   int* ex);
void copy(Ctx& c, double* dst, const double* src, int64_t n);
void axpby(Ctx& c, int64_t n, double a, const double* x, double b, double* y);  // y = a x + b y
// Deterministic dot product into a device scalar.
void dot(Ctx& c, int64_t n, const double* x, const double* y, double* out_dev);

// ------------------------------------------------------------------ small dense linear algebra

// Householder QR of `count` matrices (strided): A (m x n) = Q (m x kk) R (kk x n), kk = min(m,n).
// trans = 1: the buffer holds A^T (n x m row-major) and Q^T (kk x m) is written.
// Max relative errors of the QR's Newton reciprocal / reciprocal square root against CUDA's
// correctly rounded 1/x and 1/sqrt(x) over x_dev[0..n): err_dev[0], err_dev[1].
void check_recip(Ctx& c, int n, const double* x_dev, double* err_dev);
// path: 0 = cluster QR when the shape allows it, else one CTA; 1 = one CTA; 2 = cluster only.
void qr(Ctx& c, int count, int m, int n, int trans, const double* A, int64_t in_stride, double* Q, int64_t q_stride,
        double* R, int64_t r_stride, int path = 0);
// Whether qr() supports an m x n matrix (cluster kernel or one CTA).
bool qr_fits(int m, int n);
// Accurate (one-sided Jacobi, FP64) SVD of a small m x n matrix, m >= n: U (m x n), s, V (n x n).
void svd_small(Ctx& c, int m, int n, const double* G, double* U, double* s, double* V);

// Symmetric eigendecomposition of an n x n FP64 matrix S (row-major): eigenvalues descending
// into w (n), eigenvectors as columns of V (n x n, row-major).  FP32 Jacobi, then FP64
// Ogita-Aishima refinement levels.  keep (0: n) bounds how many leading eigenvectors the
// caller uses: refinement levels whose tail starts at or after keep are skipped, so the
// trailing (discarded) vectors span the right subspace but are not resolved among themselves.
// F (optional, m x n row-major, S = F^T F): every refinement product X^T S X is then formed as
// (F X)^T (F X), which keeps eigenvalues far below ||S|| (squared singular values of F down to
// ~eps^2 ||S||) resolved to their own scale.
void eigh(Ctx& c, int n, const double* S, double* w, double* V, int keep = 0, const double* F = nullptr, int m = 0);
void init_kernel_attributes();

}  // namespace qtt
