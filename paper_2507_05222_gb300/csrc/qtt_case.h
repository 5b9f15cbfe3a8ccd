// Internal cylinder-case state (see qtt_case.cu).
#pragma once

#include <utility>
#include <vector>

#include "qtt_algebra.h"

namespace qtt {

struct Case {
  qtt_case_params P{};
  double deta = 0, dxi = 0;
  std::vector<std::pair<int, int>> layout;  // (axis, level) per core; axis 0 = eta, 1 = xi
  // operators
  qtt_mpo *Dx = nullptr, *Dz = nullptr, *Dxp = nullptr, *Dzp = nullptr, *H = nullptr, *Ap = nullptr,
          *Px = nullptr, *Pz = nullptr, *Jdiag = nullptr;
  // boundary vectors (null when identically zero) and |J|
  qtt_mps *bcx_u = nullptr, *bcz_u = nullptr, *bcx_v = nullptr, *bcz_v = nullptr, *JbcLap_u = nullptr,
          *JbcLap_v = nullptr, *bcdiv_w = nullptr, *absJ = nullptr;
  // state
  qtt_mps *u = nullptr, *v = nullptr, *p = nullptr;
  qtt_mps* p_prev = nullptr;        // the pressure of the previous step (warm start extrapolation)
  bool prev_valid = false;          // p_prev holds a previous step's pressure (false after set_state)
  bool last_first_eager = false;    // the last run's first step ran eagerly (launches already counted)
  // CUDA graph of one step (captured on first use, replayed afterwards; invalidated when the
  // state buffers change).  The graph writes its per-step record (kStepRecDoubles) to rec.
  bool use_graph = true;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool graph_forces = false;
  int64_t graph_launches = 0;       // kernels of one replay outside the ALS sweep loops
  int64_t body_launches[3] = {0, 0, 0};  // kernels of one sweep of the u, v and p solves
  double* rec = nullptr;            // kStepRecDoubles doubles of device memory (cudaMalloc, once)
  std::vector<int*> tile_ctr;       // the graph's split-K tile counters (context, then workers)
  // Phase boundaries of the last step (timing events; external event nodes inside the graph):
  // start, after the MPO-MPS products, after the right sides + momentum, after the Poisson
  // solve, after the projection.
  cudaEvent_t ph_ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
  bool capturing = false;
  void mark(Ctx& c, int i);
  Ctx* ctx = nullptr;
  void drop_graph();
  ~Case();
};

// Record of one step (device): the AlsCtl of the u, v and p solves, a finiteness flag of the
// new velocity (1 or 0), then C_D, C_L.
constexpr int kStepRecFinite = 3 * kAlsCtlDoubles;
constexpr int kStepRecForces = kStepRecFinite + 1;
constexpr int kStepRecDoubles = kStepRecForces + 2;

Case* build_case(Ctx& c, const qtt_case_params& P);
// One step; writes its record to rec (device, kStepRecDoubles) and the forces when asked.
// extrapolate: warm-start the Poisson solve from 2 p^m - p^(m-1) (needs poisson_warm = 1).
void step(Ctx& c, Case& cs, double* rec, bool with_forces, bool extrapolate);
// nsteps steps, replaying the captured graph when cs.use_graph; records into rec_all (device,
// kStepRecDoubles per step).
void run_steps(Ctx& c, Case& cs, int nsteps, bool with_forces, double* rec_all);
// nsteps steps of every case (graph replays only), the cases' graphs replayed concurrently on
// their own streams; records into rec_all (device, case-major: case i, step s at
// (i * nsteps + s) * kStepRecDoubles).  The cases must be distinct.
void run_steps_batch(Ctx& c, const std::vector<Case*>& cases, int nsteps, bool with_forces, double* rec_all);
void case_forces(Ctx& c, Case& cs, double* out_dev);
void read_row(Ctx& c, const Case& cs, const qtt_mps* x, int64_t I, double* row_dev);
// *flag = 0 if any of x[0..n) is NaN or Inf (left untouched otherwise).
void check_finite(Ctx& c, const double* x, int64_t n, double* flag);

}  // namespace qtt

struct qtt_case {
  qtt::Ctx* ctx = nullptr;
  qtt::Case* cs = nullptr;
};
