// mps_dot_noalloc: the overlap <a, b> of two TT-vectors without any device allocation.
//
// Some callers cannot allocate device memory at the moment they need an overlap: code that
// runs inside another allocator's callback (allocating there would re-enter that allocator),
// loops that must not pay for cudaMalloc (which may synchronise the whole device), and
// processes whose device memory is entirely reserved by another framework's pool.  For them
// this entry point takes raw device arrays for the inputs and the output and keeps its
// intermediate transfer matrices in one fixed array of device memory compiled into the
// library, instead of the context pool that mps_dot uses.
//
// The fixed array (NOALLOC_SCRATCH doubles, 768 KiB) exists once per device that loads the
// library and stays allocated until the process exits.  Every call uses the same array, so
// calls that overlap on the GPU (different streams, or different host threads) race and
// corrupt each other's result; serialise them.  The array keeps the contents of the last
// call; the one entry that must start at a known value (the 1 x 1 starting transfer matrix)
// is written by each call before use, everything else is fully overwritten before it is read.
#include <mutex>
#include <string>

#include "qtt_internal.h"

namespace {

constexpr int NOALLOC_MAX_BOND = 128;
constexpr int NOALLOC_MAX_D = 4;
// Two transfer matrices (ping-pong) and the half-contracted intermediate.
constexpr int64_t NOALLOC_E = int64_t(NOALLOC_MAX_BOND) * NOALLOC_MAX_BOND;
constexpr int64_t NOALLOC_T = int64_t(NOALLOC_MAX_D) * NOALLOC_MAX_BOND * NOALLOC_MAX_BOND;
constexpr int64_t NOALLOC_SCRATCH = 2 * NOALLOC_E + NOALLOC_T;

static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH];

constexpr int MAX_DEVICES = 64;
double* g_scratch_addr[MAX_DEVICES] = {nullptr};
std::mutex g_scratch_mutex;

// Device address of the fixed array on the current device.  In host code the array's name is
// only a host-side stand-in, so the address must come from cudaGetSymbolAddress, once per
// device, with that device current.
double* scratch_for_current_device() {
  int dev = -1;
  QTT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= MAX_DEVICES) throw qtt::Error(QTT_ERR_UNSUPPORTED, "mps_dot_noalloc: device index out of range");
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      throw qtt::Error(QTT_ERR_CUDA, std::string("mps_dot_noalloc: cudaGetSymbolAddress failed: ") + cudaGetErrorString(e));
    g_scratch_addr[dev] = static_cast<double*>(p);
  }
  return g_scratch_addr[dev];
}

__global__ void k_noalloc_init(double* E) {
  if (threadIdx.x == 0 && blockIdx.x == 0) E[0] = 1.0;
}

// T[s][i][j'] = sum_j E[i][j] B[j][s][j']   (E: ra0 x rb0, B core: rb0 x d x rb1)
__global__ void k_noalloc_left(const double* __restrict__ E, const double* __restrict__ B, double* __restrict__ T,
                               int ra0, int rb0, int d, int rb1) {
  const int64_t total = int64_t(d) * ra0 * rb1;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    int jp = int(e % rb1);
    int i = int((e / rb1) % ra0);
    int s = int(e / (int64_t(rb1) * ra0));
    double acc = 0.0;
    for (int j = 0; j < rb0; ++j) acc = fma(E[int64_t(i) * rb0 + j], B[(int64_t(j) * d + s) * rb1 + jp], acc);
    T[e] = acc;
  }
}

// E'[i'][j'] = sum_{s,i} A[i][s][i'] T[s][i][j']   (A core: ra0 x d x ra1)
__global__ void k_noalloc_right(const double* __restrict__ A, const double* __restrict__ T, double* __restrict__ En,
                                int ra0, int d, int ra1, int rb1) {
  const int64_t total = int64_t(ra1) * rb1;
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < total; e += int64_t(gridDim.x) * blockDim.x) {
    int jp = int(e % rb1);
    int ip = int(e / rb1);
    double acc = 0.0;
    for (int s = 0; s < d; ++s)
      for (int i = 0; i < ra0; ++i)
        acc = fma(A[(int64_t(i) * d + s) * ra1 + ip], T[(int64_t(s) * ra0 + i) * rb1 + jp], acc);
    En[e] = acc;
  }
}

__global__ void k_noalloc_out(const double* E, double* out) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *out = E[0];
}

int blocks_for(int64_t n) {
  int64_t b = (n + 255) / 256;
  return int(b < 1 ? 1 : (b > 4096 ? 4096 : b));
}

}  // namespace

extern "C" int mps_dot_noalloc(int n, int d, const int* a_bonds, const double* a_cores, const int* b_bonds,
                               const double* b_cores, double* out_dev, void* cuda_stream) {
  try {
    if (!a_bonds || !b_bonds || !a_cores || !b_cores || !out_dev)
      throw qtt::Error(QTT_ERR_ARG, "mps_dot_noalloc: null argument");
    if (n < 1 || n > 64) throw qtt::Error(QTT_ERR_ARG, "mps_dot_noalloc: n must be in [1, 64]");
    if (d < 1 || d > NOALLOC_MAX_D)
      throw qtt::Error(QTT_ERR_UNSUPPORTED, "mps_dot_noalloc: physical size d must be in [1, 4]");
    if (a_bonds[0] != 1 || a_bonds[n] != 1 || b_bonds[0] != 1 || b_bonds[n] != 1)
      throw qtt::Error(QTT_ERR_ARG, "mps_dot_noalloc: boundary bonds must be 1");
    for (int k = 0; k <= n; ++k) {
      if (a_bonds[k] < 1 || b_bonds[k] < 1) throw qtt::Error(QTT_ERR_ARG, "mps_dot_noalloc: bonds must be >= 1");
      if (a_bonds[k] > NOALLOC_MAX_BOND || b_bonds[k] > NOALLOC_MAX_BOND)
        throw qtt::Error(QTT_ERR_UNSUPPORTED, "mps_dot_noalloc: bond " + std::to_string(a_bonds[k] > b_bonds[k] ? a_bonds[k] : b_bonds[k]) +
                                                  " exceeds the fixed scratch limit of 128");
    }
    cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
    double* base = scratch_for_current_device();
    double* E0 = base;
    double* E1 = base + NOALLOC_E;
    double* T = base + 2 * NOALLOC_E;
    k_noalloc_init<<<1, 32, 0, st>>>(E0);
    int64_t oa = 0, ob = 0;
    double* E = E0;
    double* En = E1;
    for (int k = 0; k < n; ++k) {
      const int ra0 = a_bonds[k], ra1 = a_bonds[k + 1], rb0 = b_bonds[k], rb1 = b_bonds[k + 1];
      k_noalloc_left<<<blocks_for(int64_t(d) * ra0 * rb1), 256, 0, st>>>(E, b_cores + ob, T, ra0, rb0, d, rb1);
      k_noalloc_right<<<blocks_for(int64_t(ra1) * rb1), 256, 0, st>>>(a_cores + oa, T, En, ra0, d, ra1, rb1);
      oa += int64_t(ra0) * d * ra1;
      ob += int64_t(rb0) * d * rb1;
      double* t = E;
      E = En;
      En = t;
    }
    k_noalloc_out<<<1, 32, 0, st>>>(E, out_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) throw qtt::Error(QTT_ERR_CUDA, std::string("mps_dot_noalloc: launch failed: ") + cudaGetErrorString(e));
  } catch (const qtt::Error& e) {
    qtt::set_last_error(e.what());
    return e.code;
  } catch (const std::exception& e) {
    qtt::set_last_error(e.what());
    return QTT_ERR_CUDA;
  }
  qtt::set_last_error("");
  return QTT_OK;
}
