// Learned warm start (qtt_nn.cu): the network object and the grid transfers.
#pragma once

#include <vector>

#include "qtt_internal.h"

namespace qtt {

int64_t nn_param_count(int c_in, int width, int depth);

struct Net {
  Ctx* ctx = nullptr;
  int c_in = 0, width = 0, depth = 0;
  int64_t nparam = 0;
  int64_t t = 0;                 // Adam steps taken
  float out_scale = 1.f;         // the network predicts y / out_scale
  float *params = nullptr, *m = nullptr, *v = nullptr, *grad = nullptr;   // device, nparam each
  float *shift = nullptr, *scale = nullptr;                               // device, c_in each
  std::vector<int> ci_, co_;     // channels per layer

  Net(Ctx& c, int c_in, int width, int depth, const float* params_host);
  ~Net();
  void set_scaling(const float* in_shift, const float* in_scale, float out_scale);
  void forward(int B, int H, int W, const float* x, std::vector<DBuf>& acts);
  // y (device, B x H x W) = network(x) x out_scale
  void predict(int B, int H, int W, const float* x, float* y);
  // one Adam step on the mean squared error between network(x) and y / out_scale; returns the
  // loss before the step (loss_dev: one float of device scratch)
  float train_step(int B, int H, int W, const float* x, const float* y, float lr, float* loss_dev);
};

void grid_restrict(Ctx& c, int Hc, int Wc, int levels, const double* fine, float* coarse);
void grid_prolong(Ctx& c, int Hc, int Wc, int levels, const float* coarse, double* fine);
void field_moments(Ctx& c, int64_t n, const float* x, double* out_dev);   // out_dev[0] mean, [1] rms

}  // namespace qtt

struct qtt_nn {
  qtt::Ctx* ctx = nullptr;
  qtt::Net* net = nullptr;
};
