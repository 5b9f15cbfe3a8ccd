// Learned warm start of the Poisson solve: a small convolutional network on a coarse (eta, xi)
// grid, trained on states the solver itself produces, predicting the pressure change of the
// next step (the growth direction standing in for the paper's unspecified preconditioner of
// the Poisson sweeps, Sec. IV.C / App. G).  Hand-written FP32 kernels: 3 x 3 convolution
// forward, its data and weight gradients, ReLU mask, squared-error loss, Adam (Kingma & Ba
// 2015), and the coarse/fine grid transfers.
//
// Convolution: y[n, o, i, j] = b[o] + sum_{c, a, e} w[o, c, a, e] x[n, c, i + a - 1, j + e - 1],
// zero outside the eta range (first axis: the wall and the far field are not neighbours),
// periodic in xi (second axis, angular).  Layout NCHW; parameters one flat vector, layer by
// layer: weights (c_out, c_in, 3, 3) then bias (c_out).
#include <algorithm>
#include <cmath>
#include <vector>

#include "qtt_internal.h"
#include "qtt_nn.h"

namespace qtt {

namespace {

constexpr float NN_B1 = 0.9f, NN_B2 = 0.999f, NN_EPS = 1e-8f;

unsigned nn_blocks(int64_t n, int t) { return unsigned(std::min<int64_t>((n + t - 1) / t, 65535 * 8)); }

// input affine (x - shift[c]) * scale[c] applied on load when shift/scale are given (layer 0)
__global__ void k_conv_fwd(int B, int ci, int co, int H, int W, const float* __restrict__ x,
                           const float* __restrict__ shift, const float* __restrict__ scale,
                           const float* __restrict__ w, const float* __restrict__ b, float* __restrict__ y, int relu) {
  const int64_t total = int64_t(B) * co * H * W;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int j = int(idx % W);
    const int i = int((idx / W) % H);
    const int o = int((idx / (int64_t(W) * H)) % co);
    const int n = int(idx / (int64_t(W) * H * co));
    float s = b[o];
    for (int c = 0; c < ci; ++c) {
      const float sh = shift ? shift[c] : 0.f, sc = scale ? scale[c] : 1.f;
      const float* xc = x + (int64_t(n) * ci + c) * H * W;
      const float* wc = w + (int64_t(o) * ci + c) * 9;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int ii = i + a - 1;
        if (ii < 0 || ii >= H) continue;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          int jj = j + e - 1;
          jj = jj < 0 ? jj + W : (jj >= W ? jj - W : jj);
          s = fmaf(wc[a * 3 + e], (xc[int64_t(ii) * W + jj] - sh) * sc, s);
        }
      }
    }
    y[idx] = relu ? fmaxf(s, 0.f) : s;
  }
}

// dx[n, c, i, j] = sum_{o, a, e} w[o, c, a, e] dy[n, o, i - a + 1, j - e + 1]
__global__ void k_conv_bwd_data(int B, int ci, int co, int H, int W, const float* __restrict__ dy,
                                const float* __restrict__ w, float* __restrict__ dx) {
  const int64_t total = int64_t(B) * ci * H * W;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int j = int(idx % W);
    const int i = int((idx / W) % H);
    const int c = int((idx / (int64_t(W) * H)) % ci);
    const int n = int(idx / (int64_t(W) * H * ci));
    float s = 0.f;
    for (int o = 0; o < co; ++o) {
      const float* dyo = dy + (int64_t(n) * co + o) * H * W;
      const float* wo = w + (int64_t(o) * ci + c) * 9;
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const int ii = i - a + 1;
        if (ii < 0 || ii >= H) continue;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
          int jj = j - e + 1;
          jj = jj < 0 ? jj + W : (jj >= W ? jj - W : jj);
          s = fmaf(wo[a * 3 + e], dyo[int64_t(ii) * W + jj], s);
        }
      }
    }
    dx[idx] = s;
  }
}

// One block per weight (o, c, a, e) -- blocks [0, co ci 9) -- and per bias o -- blocks
// [co ci 9, co ci 9 + co): dw = sum_{n, i, j} dy[n, o, i, j] x'[n, c, i + a - 1, j + e - 1] with the
// layer's input affine, db = sum dy[n, o, :, :].  Fixed summation order (per-thread strides,
// then a fixed tree): deterministic.
__global__ void k_conv_bwd_w(int B, int ci, int co, int H, int W, const float* __restrict__ x,
                             const float* __restrict__ shift, const float* __restrict__ scale,
                             const float* __restrict__ dy, float* __restrict__ dw, float* __restrict__ db) {
  __shared__ float red[32];
  const int blk = blockIdx.x;
  const bool bias = blk >= co * ci * 9;
  int o, c = 0, a = 0, e = 0;
  if (bias) {
    o = blk - co * ci * 9;
  } else {
    o = blk / (ci * 9);
    const int r = blk % (ci * 9);
    c = r / 9;
    a = (r % 9) / 3;
    e = r % 3;
  }
  const float sh = (!bias && shift) ? shift[c] : 0.f, sc = (!bias && scale) ? scale[c] : 1.f;
  const int64_t per = int64_t(H) * W, total = int64_t(B) * per;
  float s = 0.f;
  for (int64_t t = threadIdx.x; t < total; t += blockDim.x) {
    const int n = int(t / per);
    const int i = int((t % per) / W), j = int(t % W);
    const float g = dy[(int64_t(n) * co + o) * per + int64_t(i) * W + j];
    if (bias) {
      s += g;
    } else {
      const int ii = i + a - 1;
      if (ii < 0 || ii >= H) continue;
      int jj = j + e - 1;
      jj = jj < 0 ? jj + W : (jj >= W ? jj - W : jj);
      s = fmaf(g, (x[(int64_t(n) * ci + c) * per + int64_t(ii) * W + jj] - sh) * sc, s);
    }
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    float v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.f;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) {
      if (bias) db[o] = v;
      else dw[blk] = v;
    }
  }
}

__global__ void k_relu_mask(int64_t n, const float* __restrict__ act, float* __restrict__ g) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    if (!(act[i] > 0.f)) g[i] = 0.f;
}

// dpred = 2 (pred - y / out_scale) / n; *loss = mean squared difference (one block, fixed order)
__global__ void k_mse(int64_t n, const float* __restrict__ pred, const float* __restrict__ y, float inv_out,
                      float* __restrict__ dpred, float* __restrict__ loss) {
  __shared__ double red[32];
  double s = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const float d = pred[i] - y[i] * inv_out;
    dpred[i] = 2.f * d / float(n);
    s += double(d) * d;
  }
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x < 32) {
    double v = threadIdx.x < (blockDim.x >> 5) ? red[threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
    if (threadIdx.x == 0) *loss = float(v / double(n));
  }
}

__global__ void k_adam(int64_t n, float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, float lr, float bc1, float bc2) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x) {
    const float gi = g[i];
    const float mi = NN_B1 * m[i] + (1.f - NN_B1) * gi;
    const float vi = NN_B2 * v[i] + (1.f - NN_B2) * gi * gi;
    m[i] = mi;
    v[i] = vi;
    p[i] -= lr * (mi / bc1) / (sqrtf(vi / bc2) + NN_EPS);
  }
}

__global__ void k_scale(int64_t n, float* __restrict__ x, float s) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    x[i] *= s;
}

// coarse[I, J] = mean of the s x s block of fine (row-major (Hc s) x (Wc s)), s = 2^levels
__global__ void k_restrict(int Hc, int Wc, int s, const double* __restrict__ fine, float* __restrict__ coarse) {
  const int64_t total = int64_t(Hc) * Wc;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int I = int(idx / Wc), J = int(idx % Wc);
    const int64_t Wf = int64_t(Wc) * s;
    double acc = 0.0;
    for (int a = 0; a < s; ++a)
      for (int e = 0; e < s; ++e) acc += fine[(int64_t(I) * s + a) * Wf + int64_t(J) * s + e];
    coarse[idx] = float(acc / (double(s) * s));
  }
}

// one cell-centred bilinear doubling: (H x W) -> (2H x 2W), clamped in eta, periodic in xi
__global__ void k_prolong2(int H, int W, const double* __restrict__ c, double* __restrict__ f) {
  const int64_t total = int64_t(4) * H * W;
  for (int64_t idx = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; idx < total;
       idx += int64_t(gridDim.x) * blockDim.x) {
    const int i = int(idx / (2 * W)), j = int(idx % (2 * W));
    const int I = i >> 1, J = j >> 1;
    const int I2 = (i & 1) ? min(I + 1, H - 1) : max(I - 1, 0);
    const int J2 = (j & 1) ? (J + 1) % W : (J - 1 + W) % W;
    const double t1 = 0.75 * c[int64_t(I) * W + J] + 0.25 * c[int64_t(I2) * W + J];
    const double t2 = 0.75 * c[int64_t(I) * W + J2] + 0.25 * c[int64_t(I2) * W + J2];
    f[idx] = 0.75 * t1 + 0.25 * t2;
  }
}

__global__ void k_to_double(int64_t n, const float* __restrict__ x, double* __restrict__ y) {
  for (int64_t i = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; i < n; i += int64_t(gridDim.x) * blockDim.x)
    y[i] = double(x[i]);
}

// mean and root mean square (one block, fixed order)
__global__ void k_moments(int64_t n, const float* __restrict__ x, double* __restrict__ out) {
  __shared__ double red[2][32];
  double s = 0.0, q = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
    const double v = x[i];
    s += v;
    q += v * v;
  }
  for (int off = 16; off > 0; off >>= 1) {
    s += __shfl_xor_sync(0xffffffffu, s, off);
    q += __shfl_xor_sync(0xffffffffu, q, off);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = s;
    red[1][threadIdx.x >> 5] = q;
  }
  __syncthreads();
  if (threadIdx.x < 32) {
    double a = threadIdx.x < (blockDim.x >> 5) ? red[0][threadIdx.x] : 0.0;
    double b = threadIdx.x < (blockDim.x >> 5) ? red[1][threadIdx.x] : 0.0;
    for (int off = 16; off > 0; off >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, off);
      b += __shfl_xor_sync(0xffffffffu, b, off);
    }
    if (threadIdx.x == 0) {
      out[0] = a / double(n);
      out[1] = sqrt(b / double(n));
    }
  }
}

float* fbuf(DBuf& b, Ctx& c, int64_t nfloats) {
  b.reset(&c, size_t((nfloats + 1) / 2));
  return reinterpret_cast<float*>(b.p);
}

}  // namespace

int64_t nn_param_count(int c_in, int width, int depth) {
  int64_t n = 0;
  for (int k = 0; k < depth; ++k) {
    const int ci = k == 0 ? c_in : width, co = k == depth - 1 ? 1 : width;
    n += int64_t(co) * ci * 9 + co;
  }
  return n;
}

Net::Net(Ctx& c, int c_in_, int width_, int depth_, const float* params_host)
    : ctx(&c), c_in(c_in_), width(width_), depth(depth_) {
  QTT_CHECK_ARG(c_in >= 1 && c_in <= 64 && width >= 1 && width <= 256 && depth >= 1 && depth <= 16,
                "nn: 1 <= c_in <= 64, 1 <= width <= 256, 1 <= depth <= 16");
  nparam = nn_param_count(c_in, width, depth);
  for (int k = 0; k < depth; ++k) {
    const int ci = k == 0 ? c_in : width, co = k == depth - 1 ? 1 : width;
    ci_.push_back(ci);
    co_.push_back(co);
  }
  for (float** p : {&params, &m, &v, &grad}) QTT_CUDA(cudaMalloc(p, size_t(nparam) * sizeof(float)));
  QTT_CUDA(cudaMalloc(&shift, size_t(c_in) * sizeof(float)));
  QTT_CUDA(cudaMalloc(&scale, size_t(c_in) * sizeof(float)));
  QTT_CUDA(cudaMemcpyAsync(params, params_host, size_t(nparam) * sizeof(float), cudaMemcpyHostToDevice, c.stream));
  QTT_CUDA(cudaMemsetAsync(m, 0, size_t(nparam) * sizeof(float), c.stream));
  QTT_CUDA(cudaMemsetAsync(v, 0, size_t(nparam) * sizeof(float), c.stream));
  std::vector<float> zero(c_in, 0.f), one(c_in, 1.f);
  QTT_CUDA(cudaMemcpyAsync(shift, zero.data(), size_t(c_in) * sizeof(float), cudaMemcpyHostToDevice, c.stream));
  QTT_CUDA(cudaMemcpyAsync(scale, one.data(), size_t(c_in) * sizeof(float), cudaMemcpyHostToDevice, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
}

Net::~Net() {
  if (ctx) cudaStreamSynchronize(ctx->stream);
  for (float* p : {params, m, v, grad, shift, scale})
    if (p) cudaFree(p);
}

void Net::set_scaling(const float* in_shift, const float* in_scale, float out_scale_) {
  QTT_CHECK_ARG(std::isfinite(out_scale_) && out_scale_ != 0.f, "nn: out_scale must be finite and non-zero");
  for (int c = 0; c < c_in; ++c)
    QTT_CHECK_ARG(std::isfinite(in_shift[c]) && std::isfinite(in_scale[c]), "nn: non-finite input scaling");
  QTT_CUDA(cudaMemcpyAsync(shift, in_shift, size_t(c_in) * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  QTT_CUDA(cudaMemcpyAsync(scale, in_scale, size_t(c_in) * sizeof(float), cudaMemcpyHostToDevice, ctx->stream));
  QTT_CUDA(cudaStreamSynchronize(ctx->stream));
  out_scale = out_scale_;
}

// Forward pass over B samples of c_in x H x W; acts[k] = output of layer k (ReLU applied to
// all but the last).  Returns the last activation (B x H x W, in units of out_scale).
void Net::forward(int B, int H, int W, const float* x, std::vector<DBuf>& acts) {
  Ctx& c = *ctx;
  acts.resize(depth);
  int64_t off = 0;
  const float* in = x;
  for (int k = 0; k < depth; ++k) {
    const int ci = ci_[k], co = co_[k];
    float* out = fbuf(acts[k], c, int64_t(B) * co * H * W);
    const float* w = params + off;
    const float* b = w + int64_t(co) * ci * 9;
    k_conv_fwd<<<nn_blocks(int64_t(B) * co * H * W, 256), 256, 0, c.stream>>>(
        B, ci, co, H, W, in, k == 0 ? shift : nullptr, k == 0 ? scale : nullptr, w, b, out, k < depth - 1 ? 1 : 0);
    after_launch(c, "nn_conv_fwd");
    off += int64_t(co) * ci * 9 + co;
    in = out;
  }
}

void Net::predict(int B, int H, int W, const float* x, float* y) {
  std::vector<DBuf> acts;
  forward(B, H, W, x, acts);
  const int64_t n = int64_t(B) * H * W;
  QTT_CUDA(cudaMemcpyAsync(y, acts[depth - 1].p, size_t(n) * sizeof(float), cudaMemcpyDeviceToDevice, ctx->stream));
  if (out_scale != 1.f) {
    k_scale<<<nn_blocks(n, 256), 256, 0, ctx->stream>>>(n, y, out_scale);
    after_launch(*ctx, "nn_scale");
  }
}

float Net::train_step(int B, int H, int W, const float* x, const float* y, float lr, float* loss_dev) {
  Ctx& c = *ctx;
  std::vector<DBuf> acts;
  forward(B, H, W, x, acts);
  const int64_t per = int64_t(H) * W;
  DBuf dyb, dxb;
  float* dy = fbuf(dyb, c, int64_t(B) * per);
  k_mse<<<1, 1024, 0, c.stream>>>(int64_t(B) * per, reinterpret_cast<float*>(acts[depth - 1].p), y,
                                  1.f / out_scale, dy, loss_dev);
  after_launch(c, "nn_mse");
  // parameter offsets per layer
  std::vector<int64_t> offs(depth);
  int64_t off = 0;
  for (int k = 0; k < depth; ++k) {
    offs[k] = off;
    off += int64_t(co_[k]) * ci_[k] * 9 + co_[k];
  }
  for (int k = depth - 1; k >= 0; --k) {
    const int ci = ci_[k], co = co_[k];
    const float* in = k == 0 ? x : reinterpret_cast<float*>(acts[k - 1].p);
    float* dw = grad + offs[k];
    float* db = dw + int64_t(co) * ci * 9;
    k_conv_bwd_w<<<unsigned(co * ci * 9 + co), 256, 0, c.stream>>>(B, ci, co, H, W, in, k == 0 ? shift : nullptr,
                                                                   k == 0 ? scale : nullptr, dy, dw, db);
    after_launch(c, "nn_conv_bwd_w");
    if (k > 0) {
      float* dx = fbuf(dxb, c, int64_t(B) * ci * per);
      k_conv_bwd_data<<<nn_blocks(int64_t(B) * ci * per, 256), 256, 0, c.stream>>>(B, ci, co, H, W, dy,
                                                                                  params + offs[k], dx);
      after_launch(c, "nn_conv_bwd_data");
      k_relu_mask<<<nn_blocks(int64_t(B) * ci * per, 256), 256, 0, c.stream>>>(
          int64_t(B) * ci * per, reinterpret_cast<float*>(acts[k - 1].p), dx);
      after_launch(c, "nn_relu_mask");
      std::swap(dyb, dxb);
      dy = reinterpret_cast<float*>(dyb.p);
    }
  }
  ++t;
  const float bc1 = 1.f - std::pow(NN_B1, float(t)), bc2 = 1.f - std::pow(NN_B2, float(t));
  k_adam<<<nn_blocks(nparam, 256), 256, 0, c.stream>>>(nparam, params, grad, m, v, lr, bc1, bc2);
  after_launch(c, "nn_adam");
  float h = 0.f;
  QTT_CUDA(cudaMemcpyAsync(&h, loss_dev, sizeof(float), cudaMemcpyDeviceToHost, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  return h;
}

void grid_restrict(Ctx& c, int Hc, int Wc, int levels, const double* fine, float* coarse) {
  k_restrict<<<nn_blocks(int64_t(Hc) * Wc, 256), 256, 0, c.stream>>>(Hc, Wc, 1 << levels, fine, coarse);
  after_launch(c, "grid_restrict");
}

void grid_prolong(Ctx& c, int Hc, int Wc, int levels, const float* coarse, double* fine) {
  const int64_t nc = int64_t(Hc) * Wc;
  if (levels == 0) {
    k_to_double<<<nn_blocks(nc, 256), 256, 0, c.stream>>>(nc, coarse, fine);
    after_launch(c, "grid_to_double");
    return;
  }
  // ping-pong buffers hold every level but the last (at most nc 4^(levels - 1) values)
  const size_t cap = size_t(nc) << (2 * (levels - 1));
  DBuf a(&c, cap), b(&c, cap);
  k_to_double<<<nn_blocks(nc, 256), 256, 0, c.stream>>>(nc, coarse, a.p);
  after_launch(c, "grid_to_double");
  int H = Hc, W = Wc;
  double* cur = a.p;
  for (int l = 0; l < levels; ++l) {
    double* out = (l == levels - 1) ? fine : (cur == a.p ? b.p : a.p);
    k_prolong2<<<nn_blocks(int64_t(4) * H * W, 256), 256, 0, c.stream>>>(H, W, cur, out);
    after_launch(c, "grid_prolong2");
    cur = out;
    H *= 2;
    W *= 2;
  }
}

void field_moments(Ctx& c, int64_t n, const float* x, double* out_dev) {
  k_moments<<<1, 1024, 0, c.stream>>>(n, x, out_dev);
  after_launch(c, "field_moments");
}

}  // namespace qtt
