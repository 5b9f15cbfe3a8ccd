// Internal cylinder-case state (see qtt_case.cu).
#pragma once

#include <utility>
#include <vector>

#include "qtt_internal.h"

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
  // CUDA graph of one step (captured on first use, replayed afterwards; invalidated when the
  // state buffers change).  The graph writes its per-step record (3 CG counts, C_D, C_L) to rec.
  bool use_graph = true;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  cudaStream_t gstream = nullptr;
  cudaEvent_t ev_in = nullptr, ev_out = nullptr;
  bool graph_forces = false;
  int64_t graph_launches = 0;
  double* rec = nullptr;        // 4 doubles of device memory (allocated with cudaMalloc once)
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

Case* build_case(Ctx& c, const qtt_case_params& P);
void step(Ctx& c, Case& cs, int* cg_dev, double* forces_dev);
// nsteps steps, replaying the captured graph when cs.use_graph; records (4 doubles per step:
// three CG counts packed as ints in the first 16 bytes, then C_D, C_L) into rec_all (device).
void run_steps(Ctx& c, Case& cs, int nsteps, bool with_forces, double* rec_all);
void case_forces(Ctx& c, Case& cs, double* out_dev);
void read_row(Ctx& c, const Case& cs, const qtt_mps* x, int64_t I, double* row_dev);

}  // namespace qtt

struct qtt_case {
  qtt::Ctx* ctx = nullptr;
  qtt::Case* cs = nullptr;
};
