// Digit-split FP64 products on the fifth-generation (tcgen05) tensor cores of sm_103a.
//
// The same exact scheme as qtt_ozaki.cu (seven balanced 8-bit digits per row of A and column of
// B; the group sums G_t = sum_{s+u=t} sum_k a_s b_u are integers below 2^24 per 64-wide k chunk,
// exact in FP32; 128-bit fixed-point accumulation; one rounding per output), with the digit
// products moved from warp-level mma.sync to tcgen05.mma:
//   * operand tiles are staged by TMA (cp.async.bulk.tensor.2d) into shared memory in the
//     128-byte swizzled K-major layout the tensor core reads directly: per 64-wide k chunk the
//     seven digit slices of a 128-row tile of A (7 x 16 KB) and of a 32-column tile of B (7 x 4 KB);
//   * one thread issues the chunk's 112 MMAs (28 digit pairs x 4 k-steps of 16, M = 128, N = 32)
//     into seven FP32 accumulators in tensor memory (one per digit group, 32 columns each) and
//     commits them to an mbarrier;
//   * the four warps read the accumulators back with tcgen05.ld (warp w owns TMEM lanes =
//     output rows 32w..32w+31), convert each exact group sum to an integer and add it, shifted,
//     to the thread's 128-bit accumulators of its row's 32 outputs; the next chunk's TMA loads
//     are already in flight meanwhile.
// The result is bit-identical to the mma.sync kernel's (both add the same exact integers).
//
// Every wait on an mbarrier is bounded (~2 s of polling): on expiry the CTA records an error,
// waits (bounded again) for its own MMAs and copies, writes NaN to its outputs so that the
// caller's finiteness checks catch it, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>

#include <algorithm>

#include "qtt_internal.h"
#include "qtt_ozaki_dev.cuh"

namespace qtt {

namespace {

constexpr int T5_BM = 128;             // output rows per CTA (= TMEM lanes, MMA M)
constexpr int T5_BN = 32;              // output columns per CTA (MMA N)
constexpr int T5_KC = 64;              // k per chunk (one 128-byte swizzle row of bf16)
constexpr int T5_THREADS = 128;
constexpr int T5_GROUPS = OZ_S;        // digit groups t = 2 .. S + 1
constexpr int T5_TMEM_COLS = 256;      // 7 x 32 accumulator columns, allocated as a power of two
constexpr uint32_t T5_A_TILE = T5_BM * T5_KC * 2;   // 16 KB per digit slice
constexpr uint32_t T5_B_TILE = T5_BN * T5_KC * 2;   // 4 KB per digit slice
constexpr uint32_t T5_STAGE_BYTES = OZ_S * (T5_A_TILE + T5_B_TILE);
constexpr size_t T5_SMEM = T5_STAGE_BYTES + 1024 /* alignment */ + 64 /* barriers, TMEM slot */;
constexpr unsigned long long T5_WAIT_NS = 2000000000ull;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ unsigned long long t5_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}

// Bounded wait for the given phase of an mbarrier; false once the limit ran out.
__device__ bool mbar_wait(uint64_t* bar, unsigned phase) {
  const unsigned long long t0 = t5_ns();
  unsigned spins = 0;
  while (!mbar_test(bar, phase)) {
    if ((++spins & 1023u) == 0u && t5_ns() - t0 > T5_WAIT_NS) return false;
  }
  return true;
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          smem_u32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(smem_u32(bar))
      : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile in the 128-byte swizzled layout:
// rows of 128 bytes, 8-row groups 1024 bytes apart (the stride-dimension offset), tile base
// 1024-byte aligned; sm_100-family descriptor version 1, layout type 2 (128-byte swizzle).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  uint64_t d = 0;
  d |= uint64_t((saddr >> 4) & 0x3FFFu);
  d |= uint64_t(1) << 16;              // leading-dimension offset (unused for swizzled K-major)
  d |= uint64_t(1024 >> 4) << 32;      // stride-dimension offset
  d |= uint64_t(1) << 46;              // descriptor version
  d |= uint64_t(2) << 61;              // 128-byte swizzle
  return d;
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, both K-major, M x N.
__host__ __device__ constexpr uint32_t t5_idesc(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | (uint32_t(N >> 3) << 17) | (uint32_t(M >> 4) << 24);
}

__device__ __forceinline__ void t5_mma(uint32_t tmem_d, uint64_t adesc, uint64_t bdesc, uint32_t idesc, int acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(
          tmem_d),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void t5_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void t5_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
        "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
        "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
        "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

struct T5Args {
  int64_t M, N, Kp, ksplit, batch;
  int splits;
  const int* ea;
  const int* eb;
  double alpha, beta;
  double* C;
  int64_t sCb, sCm, sCn;
  double* W;       // split-K partials (or null)
  int* err;        // set to 1 when a bounded wait ran out (may be null)
};

__global__ void __launch_bounds__(T5_THREADS, 1)
    k_oz_gemm_tc05(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB, T5Args a) {
  extern __shared__ unsigned char t5_raw[];
  // 1024-byte alignment of the shared-window address (the swizzle pattern and the descriptors
  // assume it)
  const uint32_t raw_s = smem_u32(t5_raw);
  unsigned char* base = t5_raw + (((raw_s + 1023u) & ~1023u) - raw_s);
  unsigned char* sA = base;                                 // [S][128 rows][128 B]
  unsigned char* sB = base + OZ_S * T5_A_TILE;              // [S][32 rows][128 B]
  uint64_t* bar_tma = reinterpret_cast<uint64_t*>(base + T5_STAGE_BYTES);
  uint64_t* bar_mma = bar_tma + 1;
  uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bar_tma + 2);
  __shared__ int s_fail;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t b = blockIdx.z / a.splits;
  const int sp = blockIdx.z % a.splits;
  const int64_t kbeg = sp * a.ksplit, kend = min(a.Kp, kbeg + a.ksplit);
  const int64_t m0 = int64_t(blockIdx.y) * T5_BM, n0 = int64_t(blockIdx.x) * T5_BN;

  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(T5_TMEM_COLS)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  if (tid == 0) {
    mbar_init(bar_tma, 1);
    mbar_init(bar_mma, 1);
    s_fail = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tmem_slot;

  unsigned long long lo[T5_BN];
  long long hi[T5_BN];
#pragma unroll
  for (int c = 0; c < T5_BN; ++c) {
    lo[c] = 0ull;
    hi[c] = 0ll;
  }
  const int64_t rowA = (b * OZ_S) * a.M + m0, rowB = (b * OZ_S) * a.N + n0;
  auto issue_loads = [&](int64_t k0) {
    mbar_expect_tx(bar_tma, T5_STAGE_BYTES);
    for (int s = 0; s < OZ_S; ++s) {
      tma_load_2d(sA + s * T5_A_TILE, &mapA, int(k0), int(rowA + int64_t(s) * a.M), bar_tma);
      tma_load_2d(sB + s * T5_B_TILE, &mapB, int(k0), int(rowB + int64_t(s) * a.N), bar_tma);
    }
  };
  constexpr uint32_t idesc = t5_idesc(T5_BM, T5_BN);
  unsigned phase = 0;
  bool ok = true;
  bool loads_pending = false, mma_pending = false;
  if (tid == 0 && kbeg < kend) {
    issue_loads(kbeg);
    loads_pending = true;
  }
  for (int64_t k0 = kbeg; k0 < kend; k0 += T5_KC) {
    if (tid == 0) {
      if (!mbar_wait(bar_tma, phase)) {
        s_fail = 1;
      } else {
        loads_pending = false;
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t a0 = smem_u32(sA), b0 = smem_u32(sB);
        for (int g = 0; g < T5_GROUPS; ++g) {
          const int t = g + 2;                               // digits are numbered 1 .. S
          const int s_lo = max(1, t - OZ_S), s_hi = min(OZ_S, t - 1);
          int acc = 0;
          for (int s = s_lo; s <= s_hi; ++s) {
            const int u = t - s;
            for (int kk = 0; kk < T5_KC / 16; ++kk) {
              const uint64_t ad = sw128_desc(a0 + (s - 1) * T5_A_TILE + kk * 32);
              const uint64_t bd = sw128_desc(b0 + (u - 1) * T5_B_TILE + kk * 32);
              t5_mma(tmem + uint32_t(g * T5_BN), ad, bd, idesc, acc);
              acc = 1;
            }
          }
        }
        t5_commit(bar_mma);
        mma_pending = true;
      }
    }
    __syncthreads();
    if (s_fail) {
      ok = false;
      break;
    }
    // all threads: the chunk's group sums are in TMEM once the commit arrives
    if (!mbar_wait(bar_mma, phase)) atomicExch(&s_fail, 1);
    __syncthreads();
    if (s_fail) {
      ok = false;
      break;
    }
    if (tid == 0) mma_pending = false;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // shared memory is free again: the next chunk's loads overlap this chunk's read-back
    if (tid == 0 && k0 + T5_KC < kend) {
      issue_loads(k0 + T5_KC);
      loads_pending = true;
    }
    const uint32_t lane_base = tmem + (uint32_t(warp * 32) << 16);
    for (int g = 0; g < T5_GROUPS; ++g) {
      float v[32];
      t5_ld32(lane_base + uint32_t(g * T5_BN), v);
      const int shift = 8 * (OZ_S - 1 - g);                  // group t = g + 2: 8 (S + 1 - t)
#pragma unroll
      for (int c = 0; c < T5_BN; ++c) oz_acc(hi[c], lo[c], static_cast<long long>(__float2int_rz(v[c])), shift);
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    phase ^= 1u;
  }
  if (!ok) {
    // bounded waits for this CTA's own copies and MMAs before its memory goes away
    if (tid == 0) {
      if (loads_pending) mbar_wait(bar_tma, phase);
      if (mma_pending) mbar_wait(bar_mma, phase);
      if (a.err) atomicExch(a.err, 1);
    }
    __syncthreads();
  }
  const int64_t gm = m0 + tid;
  if (gm < a.M) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
    for (int c = 0; c < T5_BN; ++c) {
      const int64_t gn = n0 + c;
      if (gn >= a.N) continue;
      double v = ok ? fixed_to_double(hi[c], lo[c], a.ea[b * a.M + gm] + a.eb[b * a.N + gn] - 8 * (OZ_S + 1)) : nan;
      if (a.alpha != 1.0) v *= a.alpha;
      if (a.W) {
        a.W[((int64_t(sp) * a.batch + b) * a.M + gm) * a.N + gn] = v;
      } else {
        double* cp = a.C + b * a.sCb + gm * a.sCm + gn * a.sCn;
        *cp = (a.beta == 0.0) ? v : v + a.beta * (*cp);
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(T5_TMEM_COLS) : "memory");
  }
}

PFN_cuTensorMapEncodeTiled_v12000 g_encode = nullptr;
bool g_t5_attr = false;

void t5_init() {
  if (g_t5_attr) return;
  void* fn = nullptr;
  cudaDriverEntryPointQueryResult q;
  QTT_CUDA(cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q));
  if (!fn || q != cudaDriverEntryPointSuccess)
    throw Error(QTT_ERR_UNSUPPORTED, "tcgen05 products: cuTensorMapEncodeTiled is not available");
  g_encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  QTT_CUDA(cudaFuncSetAttribute(k_oz_gemm_tc05, cudaFuncAttributeMaxDynamicSharedMemorySize, int(T5_SMEM)));
  g_t5_attr = true;
}

// 2-D tensor map of digit slices: rows x Kp bf16 values, row-major, box 64 (k) x box_rows,
// 128-byte swizzle; reads past either extent return zeros.
CUtensorMap t5_map(const void* base, int64_t rows, int64_t Kp, int box_rows) {
  CUtensorMap m;
  const cuuint64_t dims[2] = {cuuint64_t(Kp), cuuint64_t(rows)};
  const cuuint64_t strides[1] = {cuuint64_t(Kp) * 2};
  const cuuint32_t box[2] = {cuuint32_t(T5_KC), cuuint32_t(box_rows)};
  const cuuint32_t estr[2] = {1, 1};
  CUresult r = g_encode(&m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                        CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) throw Error(QTT_ERR_CUDA, "tcgen05 products: tensor map encoding failed (" + std::to_string(int(r)) + ")");
  return m;
}

}  // namespace

void init_tc05_attributes() { t5_init(); }

bool tc05_fits(int64_t Kp) { return Kp % 16 == 0 && Kp <= (int64_t(1) << 31); }

// C = alpha A B + beta C from digit slices As [batch][S][M][Kp], Bs [batch][S][N][Kp] (bf16,
// K contiguous) and their exponents, on the tcgen05 tensor cores; split K like the mma.sync
// kernel (one CTA per SM).  W: partial products when splits > 1.
void oz_gemm_tc05(Ctx& c, int64_t batch, int64_t M, int64_t N, int64_t Kp, int splits, int64_t ksplit,
                  const void* As, const int* ea, const void* Bs, const int* eb, double alpha, double beta, double* C,
                  int64_t sCb, int64_t sCm, int64_t sCn, double* W) {
  t5_init();
  QTT_CHECK_ARG(reinterpret_cast<uintptr_t>(As) % 16 == 0 && reinterpret_cast<uintptr_t>(Bs) % 16 == 0,
                "tcgen05 products: digit slices must be 16-byte aligned");
  QTT_CHECK_ARG(ksplit % T5_KC == 0 || splits == 1, "tcgen05 products: split k must be a multiple of 64");
  const CUtensorMap ma = t5_map(As, batch * OZ_S * M, Kp, T5_BM);
  const CUtensorMap mb = t5_map(Bs, batch * OZ_S * N, Kp, T5_BN);
  T5Args a;
  a.M = M; a.N = N; a.Kp = Kp; a.ksplit = ksplit; a.batch = batch; a.splits = splits;
  a.ea = ea; a.eb = eb; a.alpha = alpha; a.beta = beta; a.C = C; a.sCb = sCb; a.sCm = sCm; a.sCn = sCn;
  a.W = W;
  a.err = nullptr;             // a timed-out CTA reports through NaN outputs
  dim3 grid(unsigned((N + T5_BN - 1) / T5_BN), unsigned((M + T5_BM - 1) / T5_BM), unsigned(batch * splits));
  QTT_CHECK_ARG(grid.y <= 65535 && grid.z <= 65535, "tcgen05 products: grid too large");
  k_oz_gemm_tc05<<<grid, T5_THREADS, T5_SMEM, c.stream>>>(ma, mb, a);
  after_launch(c, "oz_gemm_tc05");
}

}  // namespace qtt
