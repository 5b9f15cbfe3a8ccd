// FP64 matrix products on the tensor cores by exact digit splitting (the Ozaki scheme:
// Ozaki, Ogita, Oishi & Rump, Numer. Algorithms 59, 2012; Mukunoki et al., ISC 2020).
//
// On GB300 the FP64 pipe retires ~1 TFLOP/s while bf16 tensor-core MMA (even the legacy
// mma.sync path used here) retires ~600 TFLOP/s, so a large FP64 product can be done as a
// handful of exact bf16 products:
//   * every row i of A is scaled by 2^-e_i (|A_ik| 2^-e_i <= 1/2) and written as S = 7
//     balanced base-256 digits, A_ik = 2^e_i sum_s a_s 2^-8s + r, |a_s| <= 128,
//     |r| <= 2^-57 2^e_i; columns of B likewise (exponents f_j, digits b_u);
//   * digits are integers of at most 8 bits, exact in bf16; a digit product is exact in FP32, and
//     every sum of (t - 1) <= 7 digit products over at most 64 k stays below 2^24, so the tensor
//     core's FP32 accumulation of G_t = sum_{s+u=t} sum_k a_s b_u is exact for t <= 8;
//   * C_ij = 2^(e_i + f_j) sum_{t=2}^{S+1} 2^-8t G_t, accumulated exactly as a 128-bit integer
//     (integer adds only) and converted to FP64 once per output.
// Dropped digit products (s + u > S + 1) and the splitting remainders bound the error by
// ~2^-53 max_k |A_ik| sum_k |B_kj| (the FP64 GEMM bound is k eps sum_k |A_ik||B_kj|): the two
// agree to rounding for operands whose rows (columns) do not span many orders of magnitude.
#include <cuda_bf16.h>

#include <algorithm>

#include "qtt_internal.h"
#include "qtt_ozaki_dev.cuh"

namespace qtt {

namespace {

constexpr int OZ_KC = 64;          // k per chunk of exact FP32 accumulation
constexpr int OZ_BM = 128;         // rows of A per CTA (8 warps x 16)
constexpr int OZ_BN = 32;          // columns of B per CTA (4 n8 tiles)
constexpr int OZ_THREADS = 256;

// Exponent of each row r of X (R rows of K values, strides sR, sK; batch stride sB):
// ex[b R + r] = e with max_k |X_rk| 2^-e < 1/2 (0 for a zero row).  One warp per row.
__global__ void k_oz_rowexp(int64_t batch, int64_t R, int64_t K, const double* __restrict__ X, int64_t sB, int64_t sR,
                            int64_t sK, int* __restrict__ ex, const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  const int64_t wid = (blockIdx.x * int64_t(blockDim.x) + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (wid >= batch * R) return;
  const int64_t b = wid / R, r = wid - b * R;
  const double* x = X + b * sB + r * sR;
  // largest exponent field of the row (integer operations only: the FP64 unit is slow here)
  int mx = 0;
  for (int64_t k = lane; k < K; k += 32)
    mx = max(mx, int((static_cast<unsigned long long>(__double_as_longlong(x[k * sK])) >> 52) & 0x7ff));
  for (int o = 16; o > 0; o >>= 1) mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  // max |x| < 2^(mx - 1022), so e = mx - 1021 gives |x| 2^-e < 1/2 (rows of zeros and subnormals:
  // e = 0, their digits vanish -- an absolute error below 2^-1021)
  if (lane == 0) ex[b * R + r] = mx > 0 ? mx - 1021 : 0;
}

// The S digits of every element, by integer arithmetic on the FP64 bit pattern: the element
// as a fixed-point integer F = round(x 2^(8S - e)) (|F| < 2^(8S-1)), then balanced base-256
// digits from the least significant up, d = ((F + 128) mod 256) - 128, F = (F - d) / 256; what
// is left is the most significant digit, |d_1| <= 128.  Written as
// out[((b S + s) R + r) Kp + k] (digit s + 1, bf16; zero for K <= k < Kp).  Threads walk k
// fastest when X is contiguous along k, else r fastest, so that the reads coalesce.
__global__ void k_oz_digits(int64_t batch, int64_t R, int64_t K, int64_t Kp, const double* __restrict__ X, int64_t sB,
                            int64_t sR, int64_t sK, const int* __restrict__ ex, __nv_bfloat16* __restrict__ out,
                            const int* __restrict__ guard, int P) {
  if (guard && *guard == 0) return;
  const int64_t total = batch * R * Kp;
  const bool kfast = (sK == 1) || (sR != 1);
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < total; i += int64_t(gridDim.x) * blockDim.x) {
    int64_t b, r, k;
    if (kfast) {
      k = i % Kp;
      const int64_t br = i / Kp;
      r = br % R;
      b = br / R;
    } else {
      r = i % R;
      const int64_t bk = i / R;
      k = bk % Kp;
      b = bk / Kp;
    }
    const long long F0 = (k < K) ? oz_fixed(X[b * sB + r * sR + k * sK], ex[b * R + r]) : 0;
    long long F = F0;
    __nv_bfloat16* o = out + ((b * OZ_S) * R + r) * Kp + k;
#pragma unroll
    for (int s = OZ_S - 1; s >= 1; --s) {
      const long long dg = ((F + 128) & 255) - 128;
      F = (F - dg) >> 8;
      if (s < P) o[int64_t(s) * R * Kp] = __float2bfloat16_rn(float(dg));
    }
    o[0] = __float2bfloat16_rn(float(F));   // |F| <= 128
  }
}

// C = alpha A B + beta C from the digit slices of A (rows) and of B (columns).  CTA tile
// 128 x 32, warp w owns rows 16w..16w+15 and all 32 columns (four m16n8k16 tiles).  Shared
// memory holds the S digit slices of the tile for one k chunk, rows padded by 8 bf16 (16 bytes)
// so that ldmatrix rows fall on distinct banks.  Split K: blockIdx.z = b splits + sp covers
// k in [sp ksplit, (sp + 1) ksplit); with splits > 1 the (alpha-scaled) partial products go to
// W[((sp batch + b) M + m) N + n] for k_oz_reduce.
__global__ void __launch_bounds__(OZ_THREADS)
    k_oz_gemm(int64_t M, int64_t N, int64_t Kp, int kc, int splits, int64_t ksplit, int64_t batch,
              const __nv_bfloat16* __restrict__ As, const int* __restrict__ ea, const __nv_bfloat16* __restrict__ Bs,
              const int* __restrict__ eb, double alpha, double beta, double* __restrict__ C, int64_t sCb, int64_t sCm,
              int64_t sCn, double* __restrict__ W, const int* __restrict__ guard, int P) {
  if (guard && *guard == 0) return;
  extern __shared__ __align__(16) unsigned char oz_smem[];
  const int lds = kc + 8;
  __nv_bfloat16* sA = reinterpret_cast<__nv_bfloat16*>(oz_smem);   // [S][BM][lds]
  __nv_bfloat16* sB = sA + size_t(OZ_S) * OZ_BM * lds;              // [S][BN][lds]
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int64_t b = blockIdx.z / splits;
  const int sp = blockIdx.z % splits;
  const int64_t kbeg = sp * ksplit, kend = min(Kp, kbeg + ksplit);
  const int64_t m0 = int64_t(blockIdx.y) * OZ_BM, n0 = int64_t(blockIdx.x) * OZ_BN;
  // Exact fixed-point accumulators (value = hi 2^64 + lo, in units of 2^-64 2^(e_i + f_j)):
  // each group sum G_t (an integer below 2^24 per chunk) enters shifted left by 8 (8 - t) bits,
  // with integer adds only -- the FP64 pipe is touched once per output, at the end.
  unsigned long long lo[4][4];
  long long hi[4][4];
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      lo[i][q] = 0ull;
      hi[i][q] = 0ll;
    }
  for (int64_t k0 = kbeg; k0 < kend; k0 += kc) {
    const int kw = int(kend - k0 < int64_t(kc) ? kend - k0 : int64_t(kc));   // multiple of 16
    const int v8 = kw / 8;                                                    // 16-byte vectors per row
    __syncthreads();
    for (int idx = threadIdx.x; idx < P * OZ_BM * v8; idx += OZ_THREADS) {
      const int s = idx / (OZ_BM * v8), rem = idx - s * OZ_BM * v8, row = rem / v8, c8 = rem - row * v8;
      const int64_t gm = m0 + row;
      const bool in = gm < M;
      cp_async16(sA + (size_t(s) * OZ_BM + row) * lds + c8 * 8,
                 in ? As + ((b * OZ_S + s) * M + gm) * Kp + k0 + c8 * 8 : As, in);
    }
    for (int idx = threadIdx.x; idx < P * OZ_BN * v8; idx += OZ_THREADS) {
      const int s = idx / (OZ_BN * v8), rem = idx - s * OZ_BN * v8, row = rem / v8, c8 = rem - row * v8;
      const int64_t gn = n0 + row;
      const bool in = gn < N;
      cp_async16(sB + (size_t(s) * OZ_BN + row) * lds + c8 * 8,
                 in ? Bs + ((b * OZ_S + s) * N + gn) * Kp + k0 + c8 * 8 : Bs, in);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    for (int t = 2; t <= P + 1; ++t) {
      float c32[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) c32[i][q] = 0.f;
      const int s_lo = max(1, t - P), s_hi = min(P, t - 1);
      for (int s = s_lo; s <= s_hi; ++s) {
        const int u = t - s;
        const __nv_bfloat16* a_base = sA + (size_t(s - 1) * OZ_BM + warp * 16) * lds;
        const __nv_bfloat16* b_base = sB + size_t(u - 1) * OZ_BN * lds;
        for (int kk = 0; kk < kw; kk += 16) {
          uint32_t a[4];
          ldsm_x4(a, a_base + (lane & 15) * lds + kk + (lane >> 4) * 8);
          uint32_t b01[4], b23[4];
          ldsm_x4(b01, b_base + ((lane >> 4) * 8 + (lane & 7)) * lds + kk + ((lane >> 3) & 1) * 8);
          ldsm_x4(b23, b_base + (16 + (lane >> 4) * 8 + (lane & 7)) * lds + kk + ((lane >> 3) & 1) * 8);
          mma_bf16(c32[0], a, b01[0], b01[1]);
          mma_bf16(c32[1], a, b01[2], b01[3]);
          mma_bf16(c32[2], a, b23[0], b23[1]);
          mma_bf16(c32[3], a, b23[2], b23[3]);
        }
      }
      const int shift = 8 * (OZ_S + 1 - t);   // 0 .. 48
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          // exact integer, |G| < 2^24; the 32-bit conversion stays off the FP64 unit
          const long long G = static_cast<long long>(__float2int_rz(c32[i][q]));
          unsigned long long add_lo;
          long long add_hi;
          if (shift >= 32) {
            const long long v = G << (shift - 32);            // |v| < 2^40: value v 2^32
            add_lo = static_cast<unsigned long long>(v) << 32;
            add_hi = v >> 32;
          } else {
            const long long v = G << shift;                   // |v| < 2^56
            add_lo = static_cast<unsigned long long>(v);
            add_hi = v >> 63;                                 // sign extension
          }
          const unsigned long long nl = lo[i][q] + add_lo;
          hi[i][q] += add_hi + (nl < add_lo ? 1 : 0);
          lo[i][q] = nl;
        }
    }
  }
  const int g = lane >> 2, tg = lane & 3;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int64_t gm = m0 + warp * 16 + g + (q >= 2 ? 8 : 0);
      const int64_t gn = n0 + i * 8 + 2 * tg + (q & 1);
      if (gm >= M || gn >= N) continue;
      double v = fixed_to_double(hi[i][q], lo[i][q], ea[b * M + gm] + eb[b * N + gn] - 8 * (OZ_S + 1));
      if (alpha != 1.0) v *= alpha;
      if (W) {
        W[((int64_t(sp) * batch + b) * M + gm) * N + gn] = v;
      } else {
        double* cp = C + b * sCb + gm * sCm + gn * sCn;
        *cp = (beta == 0.0) ? v : v + beta * (*cp);
      }
    }
}

// C = sum over splits of W + beta C (fixed summation order: deterministic).
__global__ void k_oz_reduce(int64_t batch, int64_t M, int64_t N, int splits, const double* __restrict__ W, double beta,
                            double* __restrict__ C, int64_t sCb, int64_t sCm, int64_t sCn,
                            const int* __restrict__ guard) {
  if (guard && *guard == 0) return;
  const int64_t total = batch * M * N;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    const int64_t b = e / (M * N), mn = e - b * M * N, m = mn / N, n = mn - m * N;
    double v = 0.0;
    for (int sp = 0; sp < splits; ++sp) v += W[int64_t(sp) * total + e];
    double* cp = C + b * sCb + m * sCm + n * sCn;
    *cp = (beta == 0.0) ? v : v + beta * (*cp);
  }
}

size_t oz_smem_bytes(int kc) { return size_t(OZ_S) * (OZ_BM + OZ_BN) * (kc + 8) * sizeof(__nv_bfloat16); }

bool g_oz_attr = false;

}  // namespace

void init_ozaki_attributes() {
  if (g_oz_attr) return;
  QTT_CUDA(cudaFuncSetAttribute(k_oz_gemm, cudaFuncAttributeMaxDynamicSharedMemorySize, int(oz_smem_bytes(OZ_KC))));
  g_oz_attr = true;
}

void gemm_ozaki(Ctx& c, int64_t batch, int64_t M, int64_t N, int64_t K, double alpha, const double* A, int64_t sAb,
                int64_t sAm, int64_t sAk, const double* B, int64_t sBb, int64_t sBk, int64_t sBn, double beta,
                double* C, int64_t sCb, int64_t sCm, int64_t sCn) {
  QTT_CHECK_ARG(batch >= 1 && M >= 1 && N >= 1 && K >= 1, "gemm_ozaki: empty product");
  init_ozaki_attributes();
  const int P = c.root->digits;   // digits of each operand the product uses (7: FP64-exact)
  const int64_t Kp = (K + 15) / 16 * 16;
  const int kc = int(std::min<int64_t>(OZ_KC, Kp));
  // digit slices (bf16) and exponents, carved from the pool in doubles
  const size_t a_half = size_t(batch) * OZ_S * M * Kp, b_half = size_t(batch) * OZ_S * N * Kp;
  DBuf sa(&c, (a_half * 2 + 7) / 8), sb(&c, (b_half * 2 + 7) / 8), e(&c, (size_t(batch) * (M + N) * 4 + 7) / 8);
  __nv_bfloat16* As = reinterpret_cast<__nv_bfloat16*>(sa.p);
  __nv_bfloat16* Bs = reinterpret_cast<__nv_bfloat16*>(sb.p);
  int* ea = reinterpret_cast<int*>(e.p);
  int* eb = ea + batch * M;
  ProfScope ps(c, KC_GEMM, 2.0 * double(batch) * double(M) * double(N) * double(K));
  {
    const int64_t wa = batch * M, wb = batch * N;
    k_oz_rowexp<<<unsigned((wa * 32 + 255) / 256), 256, 0, c.stream>>>(batch, M, K, A, sAb, sAm, sAk, ea, c.guard);
    after_launch(c, "oz_rowexp_a");
    k_oz_rowexp<<<unsigned((wb * 32 + 255) / 256), 256, 0, c.stream>>>(batch, N, K, B, sBb, sBn, sBk, eb, c.guard);
    after_launch(c, "oz_rowexp_b");
    const int64_t ta = batch * M * Kp, tb = batch * N * Kp;
    k_oz_digits<<<unsigned(std::min<int64_t>((ta + 255) / 256, 8192)), 256, 0, c.stream>>>(batch, M, K, Kp, A, sAb,
                                                                                          sAm, sAk, ea, As, c.guard, P);
    after_launch(c, "oz_digits_a");
    k_oz_digits<<<unsigned(std::min<int64_t>((tb + 255) / 256, 8192)), 256, 0, c.stream>>>(batch, N, K, Kp, B, sBb,
                                                                                          sBn, sBk, eb, Bs, c.guard, P);
    after_launch(c, "oz_digits_b");
  }
  // Split K (in whole chunks) until the grid covers the SMs once: this kernel holds one CTA per
  // SM (its shared memory), and products such as (c s) x (e f) x d have few output tiles but a
  // long k.
  const int64_t tiles = ((N + OZ_BN - 1) / OZ_BN) * ((M + OZ_BM - 1) / OZ_BM) * batch;
  const int64_t nchunks = (Kp + kc - 1) / kc;
  int64_t splits = 1;
  if (tiles < c.num_sms) splits = std::min<int64_t>(nchunks, (c.num_sms + tiles - 1) / tiles);
  const int64_t ksplit = (nchunks + splits - 1) / splits * kc;
  splits = (Kp + ksplit - 1) / ksplit;
  dim3 grid(unsigned((N + OZ_BN - 1) / OZ_BN), unsigned((M + OZ_BM - 1) / OZ_BM), unsigned(batch * splits));
  QTT_CHECK_ARG(grid.y <= 65535 && grid.z <= 65535, "gemm_ozaki: grid too large");
  DBuf Wb;
  if (splits > 1) Wb.reset(&c, size_t(splits) * batch * M * N);
  const int mode = c.root->gemm_mode;
  if (P == OZ_S && (mode == 3 || (mode == 0 && kDigitProductsOnTc05)) && !c.guard && tc05_fits(Kp)) {
    oz_gemm_tc05(c, batch, M, N, Kp, int(splits), ksplit, As, ea, Bs, eb, alpha, beta, C, sCb, sCm, sCn,
                 splits > 1 ? Wb.p : nullptr);
  } else {
    k_oz_gemm<<<grid, OZ_THREADS, oz_smem_bytes(kc), c.stream>>>(M, N, Kp, kc, int(splits), ksplit, batch, As, ea, Bs,
                                                                 eb, alpha, beta, C, sCb, sCm, sCn,
                                                                 splits > 1 ? Wb.p : nullptr, c.guard, P);
    after_launch(c, "oz_gemm");
  }
  if (splits > 1) {
    const int64_t total = batch * M * N;
    const int64_t blocks = std::min<int64_t>((total + 255) / 256, 4096);
    k_oz_reduce<<<unsigned(blocks), 256, 0, c.stream>>>(batch, M, N, int(splits), Wb.p, beta, C, sCb, sCm, sCn,
                                                        c.guard);
    after_launch(c, "oz_reduce");
  }
}

// Digit slices out[s][r][Kp] (bf16, s = 0..OZ_S-1) and scale exponents ex[r] of the R rows of X
// (K values each, strides sR, sK; zero digits for K <= k < Kp).
void oz_split_rows(Ctx& c, int64_t R, int64_t K, int64_t Kp, const double* X, int64_t sR, int64_t sK, void* out,
                   int* ex) {
  k_oz_rowexp<<<unsigned((R * 32 + 255) / 256), 256, 0, c.stream>>>(1, R, K, X, 0, sR, sK, ex, c.guard);
  after_launch(c, "oz_rowexp");
  const int64_t t = R * Kp;
  k_oz_digits<<<unsigned(std::min<int64_t>((t + 255) / 256, 8192)), 256, 0, c.stream>>>(
      1, R, K, Kp, X, 0, sR, sK, ex, static_cast<__nv_bfloat16*>(out), c.guard, OZ_S);
  after_launch(c, "oz_digits");
}

}  // namespace qtt
