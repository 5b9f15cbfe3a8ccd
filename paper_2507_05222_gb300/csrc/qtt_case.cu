// Cylinder case: analytic QTT grid fields and metric terms, curvilinear finite-difference
// operators and ghost-point boundary vectors (arXiv:2507.05222, Sec. III.B, App. A, App. E),
// the fractional step (Sec. III.C) and the wall forces (App. F).
//
// Operator set-up: the 1-D building blocks (carry-automaton shift MPOs, rank-1 exponential
// and rank-2 trigonometric MPS of the metric coefficients) are written out core by core on the
// host -- they are closed-form tables -- then placed in the 2-D bit layout; every product,
// sum and rounding (sigma < 1e-14 sigma_1) runs on the device.
#include <cmath>
#include <memory>

#include "qtt_algebra.h"
#include "qtt_case.h"

namespace qtt {

namespace {

// ------------------------------------------------------------------ host-side 1-D tables

struct HTT {                        // host TT: cores (r0, p, r1) with p = d (MPS) or d*d (MPO)
  std::vector<std::vector<double>> cores;
  std::vector<int> bonds;
  int p = 2;
};

HTT h_exp(int nb, double C, double lam) {
  HTT t;
  t.p = 2;
  t.bonds.assign(nb + 1, 1);
  for (int k = 0; k < nb; ++k) {
    double e = std::exp(lam * std::ldexp(1.0, nb - 1 - k));
    t.cores.push_back({1.0, e});
  }
  for (double& v : t.cores[0]) v *= C;
  return t;
}

// amp * trig(omega q + phase) with [cos(a+b), sin(a+b)] = [cos a, sin a] [[cos b, sin b], [-sin b, cos b]].
HTT h_trig(int nb, double om, double phase, bool is_sin, double amp) {
  HTT t;
  t.p = 2;
  t.bonds.assign(nb + 1, 2);
  t.bonds[0] = 1;
  t.bonds[nb] = 1;
  for (int k = 0; k < nb; ++k) {
    std::vector<double> full(2 * 2 * 2);
    for (int s = 0; s < 2; ++s) {
      double b = om * s * std::ldexp(1.0, nb - 1 - k);
      double cb = std::cos(b), sb = std::sin(b);
      // (left a, s, right c): rot(b)[a][c]
      full[(0 * 2 + s) * 2 + 0] = cb;
      full[(0 * 2 + s) * 2 + 1] = sb;
      full[(1 * 2 + s) * 2 + 0] = -sb;
      full[(1 * 2 + s) * 2 + 1] = cb;
    }
    t.cores.push_back(full);
  }
  // first core: contract the left vector amp [cos phase, sin phase]
  {
    std::vector<double> f(2 * 2, 0.0);
    double l0 = amp * std::cos(phase), l1 = amp * std::sin(phase);
    for (int s = 0; s < 2; ++s)
      for (int c = 0; c < 2; ++c) f[s * 2 + c] = l0 * t.cores[0][(0 * 2 + s) * 2 + c] + l1 * t.cores[0][(1 * 2 + s) * 2 + c];
    t.cores[0] = f;
  }
  // last core: select column 0 (cos) or 1 (sin)
  {
    int col = is_sin ? 1 : 0;
    int r0 = nb == 1 ? 1 : 2;
    std::vector<double> l(r0 * 2, 0.0);
    const std::vector<double>& src = t.cores[nb - 1];
    for (int a = 0; a < r0; ++a)
      for (int s = 0; s < 2; ++s) l[a * 2 + s] = src[(a * 2 + s) * 2 + col];
    t.cores[nb - 1] = l;
  }
  return t;
}

HTT h_const(int nb, double C) { return h_exp(nb, C, 0.0); }

HTT h_indicator(int nb, int64_t q) {
  HTT t;
  t.p = 2;
  t.bonds.assign(nb + 1, 1);
  for (int k = 0; k < nb; ++k) {
    int bit = int((q >> (nb - 1 - k)) & 1);
    std::vector<double> c(2, 0.0);
    c[bit] = 1.0;
    t.cores.push_back(c);
  }
  return t;
}

HTT h_scale(HTT t, double s) {
  for (double& v : t.cores[0]) v *= s;
  return t;
}

HTT h_identity_mpo(int nb) {
  HTT t;
  t.p = 4;
  t.bonds.assign(nb + 1, 1);
  for (int k = 0; k < nb; ++k) t.cores.push_back({1.0, 0.0, 0.0, 1.0});
  return t;
}

// (S f)_q = f_{q+step}: carry automaton, bond index = carry (borrow for step = -1); the least
// significant core receives carry 1; the most significant core keeps carry-out 0 only unless
// periodic.
HTT h_shift(int nb, int step, bool periodic) {
  HTT t;
  t.p = 4;
  t.bonds.assign(nb + 1, 2);
  t.bonds[0] = 1;
  t.bonds[nb] = 1;
  std::vector<double> W(2 * 4 * 2, 0.0);  // (cout, o, q, cin)
  for (int o = 0; o < 2; ++o)
    for (int cin = 0; cin < 2; ++cin) {
      int q, cout;
      if (step > 0) {
        int s = o + cin;
        q = s % 2;
        cout = s / 2;
      } else {
        int s = o - cin;
        q = (s + 2) % 2;
        cout = s < 0 ? 1 : 0;
      }
      W[((cout * 2 + o) * 2 + q) * 2 + cin] = 1.0;
    }
  for (int k = 0; k < nb; ++k) {
    int r0 = (k == 0) ? 1 : 2, r1 = (k == nb - 1) ? 1 : 2;
    std::vector<double> c(size_t(r0) * 4 * r1, 0.0);
    for (int a = 0; a < r0; ++a)
      for (int ph = 0; ph < 4; ++ph)
        for (int b = 0; b < r1; ++b) {
          double v = 0.0;
          for (int ca = 0; ca < 2; ++ca) {
            double lw = (k == 0) ? ((ca == 0 || periodic) ? 1.0 : 0.0) : (ca == a ? 1.0 : 0.0);
            if (lw == 0.0) continue;
            for (int cb = 0; cb < 2; ++cb) {
              double rw = (k == nb - 1) ? (cb == 1 ? 1.0 : 0.0) : (cb == b ? 1.0 : 0.0);
              if (rw == 0.0) continue;
              v += lw * rw * W[(ca * 4 + ph) * 2 + cb];
            }
          }
          c[(size_t(a) * 4 + ph) * r1 + b] = v;
        }
    t.cores.push_back(c);
  }
  return t;
}

HTT h_diag(const HTT& x) {
  HTT t;
  t.p = 4;
  t.bonds = x.bonds;
  for (size_t k = 0; k < x.cores.size(); ++k) {
    int r0 = x.bonds[k], r1 = x.bonds[k + 1];
    std::vector<double> c(size_t(r0) * 4 * r1, 0.0);
    for (int a = 0; a < r0; ++a)
      for (int s = 0; s < 2; ++s)
        for (int b = 0; b < r1; ++b) c[(size_t(a) * 4 + s * 2 + s) * r1 + b] = x.cores[k][(size_t(a) * 2 + s) * r1 + b];
    t.cores.push_back(c);
  }
  return t;
}

// Linear combination of 1-D TTs of equal shape by block cores (Sec. II.A.1).
HTT h_lin(const std::vector<std::pair<double, HTT>>& terms) {
  HTT out = terms[0].second;
  for (double& v : out.cores[0]) v *= terms[0].first;
  for (size_t t = 1; t < terms.size(); ++t) {
    const HTT& y = terms[t].second;
    double cf = terms[t].first;
    int n = int(out.cores.size()), p = out.p;
    HTT z;
    z.p = p;
    z.bonds.assign(n + 1, 1);
    for (int k = 1; k < n; ++k) z.bonds[k] = out.bonds[k] + y.bonds[k];
    for (int k = 0; k < n; ++k) {
      int xr0 = out.bonds[k], xr1 = out.bonds[k + 1], yr0 = y.bonds[k], yr1 = y.bonds[k + 1];
      int zr0 = z.bonds[k], zr1 = z.bonds[k + 1];
      std::vector<double> c(size_t(zr0) * p * zr1, 0.0);
      for (int a = 0; a < zr0; ++a)
        for (int s = 0; s < p; ++s)
          for (int b = 0; b < zr1; ++b) {
            double v = 0.0;
            if (n == 1) v = out.cores[k][s] + cf * y.cores[k][s];
            else if (k == 0) v = (b < xr1) ? out.cores[k][s * xr1 + b] : cf * y.cores[k][s * yr1 + (b - xr1)];
            else if (k == n - 1) v = (a < xr0) ? out.cores[k][a * p + s] : y.cores[k][(a - xr0) * p + s];
            else if (a < xr0 && b < xr1) v = out.cores[k][(size_t(a) * p + s) * xr1 + b];
            else if (a >= xr0 && b >= xr1) v = y.cores[k][(size_t(a - xr0) * p + s) * yr1 + (b - xr1)];
            c[(size_t(a) * p + s) * zr1 + b] = v;
          }
      z.cores.push_back(c);
    }
    out = z;
  }
  return out;
}

// Place a 1-D train on the eta bits and another on the xi bits of the 2-D layout: the bond
// after each core is (eta bond) x (xi bond), eta major; a core of one axis passes the other
// axis' bond through with an identity.
HTT h_combine(const HTT& fe, const HTT& fx, const std::vector<std::pair<int, int>>& layout) {
  HTT t;
  t.p = fe.p;
  int be = 1, bx = 1;
  t.bonds.push_back(1);
  const int p = fe.p;
  for (auto [ax, l] : layout) {
    if (ax == 0) {
      int a0 = fe.bonds[l], a1 = fe.bonds[l + 1];
      std::vector<double> c(size_t(a0) * bx * p * a1 * bx, 0.0);
      for (int a = 0; a < a0; ++a)
        for (int x = 0; x < bx; ++x)
          for (int s = 0; s < p; ++s)
            for (int b = 0; b < a1; ++b)
              c[((size_t(a * bx + x) * p + s) * a1 + b) * bx + x] = fe.cores[l][(size_t(a) * p + s) * a1 + b];
      t.cores.push_back(c);
      be = a1;
    } else {
      int a0 = fx.bonds[l], a1 = fx.bonds[l + 1];
      std::vector<double> c(size_t(be) * a0 * p * be * a1, 0.0);
      for (int x = 0; x < be; ++x)
        for (int a = 0; a < a0; ++a)
          for (int s = 0; s < p; ++s)
            for (int b = 0; b < a1; ++b)
              c[((size_t(x * a0 + a) * p + s) * be + x) * a1 + b] = fx.cores[l][(size_t(a) * p + s) * a1 + b];
      t.cores.push_back(c);
      bx = a1;
    }
    t.bonds.push_back(be * bx);
  }
  return t;
}

std::vector<std::pair<int, int>> make_layout(int ne, int nx, int ordering) {
  std::vector<std::pair<int, int>> lay;
  if (ordering == QTT_ORDER_SEQUENTIAL) {
    for (int l = 0; l < ne; ++l) lay.push_back({0, l});
    for (int l = 0; l < nx; ++l) lay.push_back({1, l});
  } else {
    for (int l = 0; l < std::max(ne, nx); ++l) {
      if (l < ne) lay.push_back({0, l});
      if (l < nx) lay.push_back({1, l});
    }
  }
  return lay;
}

qtt_mps* upload_mps(Ctx& c, const HTT& t) {
  qtt_mps* x = new_mps(&c, int(t.cores.size()), t.p, t.bonds);
  for (size_t k = 0; k < t.cores.size(); ++k)
    QTT_CUDA(cudaMemcpyAsync(x->core(int(k)), t.cores[k].data(), t.cores[k].size() * sizeof(double),
                             cudaMemcpyHostToDevice, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  return x;
}

qtt_mpo* upload_mpo(Ctx& c, const HTT& t) {
  qtt_mpo* m = new_mpo(&c, int(t.cores.size()), 2, t.bonds);
  for (size_t k = 0; k < t.cores.size(); ++k)
    QTT_CUDA(cudaMemcpyAsync(m->core(int(k)), t.cores[k].data(), t.cores[k].size() * sizeof(double),
                             cudaMemcpyHostToDevice, c.stream));
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  return m;
}

// ------------------------------------------------------------------ device-side combinators

using MpsP = std::unique_ptr<qtt_mps, void (*)(qtt_mps*)>;
using MpoP = std::unique_ptr<qtt_mpo, void (*)(qtt_mpo*)>;
MpsP mk(qtt_mps* x) { return MpsP(x, free_mps); }
MpoP mk(qtt_mpo* m) { return MpoP(m, free_mpo); }

constexpr double OP_EPS = 1e-14;
constexpr int BIG = 1 << 20;

qtt_mpo* round_op(Ctx& c, const qtt_mpo* M) {
  MpsP v = mk(mpo_as_mps(c, M));
  MpsP r = mk(round_any(c, v.get(), BIG, OP_EPS));
  return mps_as_mpo(c, r.get(), 2);
}

qtt_mpo* lin_op(Ctx& c, const std::vector<std::pair<double, const qtt_mpo*>>& terms) {
  MpsP acc = mk(mpo_as_mps(c, terms[0].second));
  mps_scale(c, acc.get(), terms[0].first);
  for (size_t t = 1; t < terms.size(); ++t) {
    MpsP y = mk(mpo_as_mps(c, terms[t].second));
    acc = mk(direct_sum(c, 1.0, acc.get(), terms[t].first, y.get()));
  }
  return mps_as_mpo(c, acc.get(), 2);
}

qtt_mpo* diag_times(Ctx& c, const qtt_mps* coef, const qtt_mpo* D) {
  MpoP dg = mk(diag_mpo(c, coef));
  return mpo_mpo_exact(c, dg.get(), D);
}

qtt_mps* had_round(Ctx& c, const qtt_mps* a, const qtt_mps* b) {
  MpoP dg = mk(diag_mpo(c, a));
  MpsP p = mk(mpo_mps_exact(c, dg.get(), b));
  return round_any(c, p.get(), BIG, OP_EPS);
}

qtt_mps* add_round(Ctx& c, const qtt_mps* a, const qtt_mps* b) {
  if (!a) return b ? mps_copy(c, b) : nullptr;
  if (!b) return mps_copy(c, a);
  MpsP s = mk(direct_sum(c, 1.0, a, 1.0, b));
  return round_any(c, s.get(), BIG, OP_EPS);
}

}  // namespace

// ------------------------------------------------------------------ case

void Case::mark(Ctx& c, int i) {
  if (!ph_ev[i]) QTT_CUDA(cudaEventCreate(&ph_ev[i]));
  if (capturing) QTT_CUDA(cudaEventRecordWithFlags(ph_ev[i], c.stream, cudaEventRecordExternal));
  else QTT_CUDA(cudaEventRecord(ph_ev[i], c.stream));
}

void Case::drop_graph() {
  if (gexec || graph) {
    if (gstream) cudaStreamSynchronize(gstream);
    if (gexec) cudaGraphExecDestroy(gexec);
    if (graph) cudaGraphDestroy(graph);
    gexec = nullptr;
    graph = nullptr;
    if (ctx) {
      ctx->pool->release_capture(this);
      for (Ctx* w : ctx->workers) w->pool->release_capture(this);
    }
  }
}

Case::~Case() {
  drop_graph();
  if (gstream) cudaStreamDestroy(gstream);
  if (ev_in) cudaEventDestroy(ev_in);
  if (ev_out) cudaEventDestroy(ev_out);
  for (auto& e : ph_ev)
    if (e) cudaEventDestroy(e);
  if (rec) cudaFree(rec);
  for (int* t : tile_ctr)
    if (t) cudaFree(t);
  for (qtt_mpo* m : {Dx, Dz, Dxp, Dzp, H, Ap, Px, Pz, Jdiag})
    if (m) free_mpo(m);
  for (qtt_mps* x : {bcx_u, bcz_u, bcx_v, bcz_v, JbcLap_u, JbcLap_v, bcdiv_w, absJ, u, v, p, p_prev})
    if (x) free_mps(x);
}

Case* build_case(Ctx& c, const qtt_case_params& P) {
  QTT_CHECK_ARG(P.n_eta >= 1 && P.n_xi >= 1 && P.n_eta + P.n_xi <= 40, "case: grid bits");
  QTT_CHECK_ARG(P.ordering == QTT_ORDER_SEQUENTIAL || P.ordering == QTT_ORDER_INTERLEAVED, "case: ordering");
  QTT_CHECK_ARG(P.R > 1.0 && P.D > 0.0 && P.Re > 0.0 && P.dt > 0.0 && P.chi >= 1, "case: parameters");
  std::unique_ptr<Case> cs(new Case);
  cs->P = P;
  const int ne = P.n_eta, nx = P.n_xi;
  const double Ne = std::ldexp(1.0, ne), Nx = std::ldexp(1.0, nx);
  const double de = 1.0 / (Ne + 1.0), dx = 1.0 / Nx;
  const double lnR = std::log(P.R), pi = M_PI, D = P.D;
  const double om = 2.0 * pi * dx;
  cs->deta = de;
  cs->dxi = dx;
  auto lay = make_layout(ne, nx, P.ordering);
  cs->layout = lay;
  auto m2 = [&](const HTT& fe, const HTT& fx) { return upload_mps(c, h_combine(fe, fx, lay)); };
  auto o2 = [&](const HTT& Me, const HTT& Mx) { return upload_mpo(c, h_combine(Me, Mx, lay)); };
  HTT Ie = h_identity_mpo(ne), Ix = h_identity_mpo(nx);
  HTT inv_r = h_exp(ne, (2.0 / D) * std::pow(P.R, -de), -lnR * de);        // 1 / r_i
  HTT r2 = h_exp(ne, (D / 2) * (D / 2) * std::pow(P.R, 2 * de), 2 * lnR * de);  // r_i^2
  HTT sin_x = h_trig(nx, om, 0.0, true, 1.0), cos_x = h_trig(nx, om, 0.0, false, 1.0);
  HTT one_x = h_const(nx, 1.0);
  MpsP cx_xi = mk(m2(h_scale(inv_r, -1.0 / (2 * pi)), sin_x));
  MpsP cx_eta = mk(m2(h_scale(inv_r, 1.0 / lnR), cos_x));
  MpsP cz_xi = mk(m2(h_scale(inv_r, 1.0 / (2 * pi)), cos_x));
  MpsP cz_eta = mk(m2(h_scale(inv_r, 1.0 / lnR), sin_x));
  cs->absJ = m2(h_scale(r2, 2 * pi * lnR), one_x);
  HTT Sxp = h_shift(nx, +1, true), Sxm = h_shift(nx, -1, true);
  HTT Sep = h_shift(ne, +1, false), Sem = h_shift(ne, -1, false);
  MpoP d_xi = mk(o2(Ie, h_lin({{1 / (2 * dx), Sxp}, {-1 / (2 * dx), Sxm}})));
  MpoP d_eta = mk(o2(h_lin({{1 / (2 * de), Sep}, {-1 / (2 * de), Sem}}), Ix));
  MpoP dd_xi = mk(o2(Ie, h_lin({{1 / (dx * dx), Sxp}, {-2 / (dx * dx), Ix}, {1 / (dx * dx), Sxm}})));
  MpoP dd_eta = mk(o2(h_lin({{1 / (de * de), Sep}, {-2 / (de * de), Ie}, {1 / (de * de), Sem}}), Ix));
  MpoP E0 = mk(o2(h_diag(h_indicator(ne, 0)), Ix));
  MpoP d_eta_p = mk(lin_op(c, {{1.0, d_eta.get()}, {-1 / (2 * de), E0.get()}}));   // ghost p_{-1} = p_0
  MpoP dd_eta_p = mk(lin_op(c, {{1.0, dd_eta.get()}, {1 / (de * de), E0.get()}}));
  auto curv = [&](const qtt_mps* c1, const qtt_mpo* D1, const qtt_mps* c2, const qtt_mpo* D2) {
    MpoP a = mk(diag_times(c, c1, D1)), b = mk(diag_times(c, c2, D2));
    MpoP s = mk(lin_op(c, {{1.0, a.get()}, {1.0, b.get()}}));
    return round_op(c, s.get());
  };
  cs->Dx = curv(cx_xi.get(), d_xi.get(), cx_eta.get(), d_eta.get());
  cs->Dz = curv(cz_xi.get(), d_xi.get(), cz_eta.get(), d_eta.get());
  cs->Dxp = curv(cx_xi.get(), d_xi.get(), cx_eta.get(), d_eta_p.get());
  cs->Dzp = curv(cz_xi.get(), d_xi.get(), cz_eta.get(), d_eta_p.get());
  // |J| Lap_h = (lnR / 2 pi) d_xixi + (2 pi / lnR) d_etaeta (g12 = 0, g/J constant)
  const double aX = lnR / (2 * pi), aE = 2 * pi / lnR, kk = P.dt / P.Re;
  cs->Jdiag = diag_mpo(c, cs->absJ);
  {
    MpoP s = mk(lin_op(c, {{1.0, cs->Jdiag}, {-kk * aX, dd_xi.get()}, {-kk * aE, dd_eta.get()}}));
    cs->H = round_op(c, s.get());
  }
  {
    MpoP s = mk(lin_op(c, {{-aX, dd_xi.get()}, {-aE, dd_eta_p.get()}}));
    cs->Ap = round_op(c, s.get());
  }
  {
    MpsP jw = mk(mps_copy(c, cs->absJ));
    mps_scale(c, jw.get(), -1.0 / P.dt);
    MpoP s1 = mk(diag_times(c, jw.get(), cs->Dx));
    cs->Px = round_op(c, s1.get());
    MpoP s2 = mk(diag_times(c, jw.get(), cs->Dz));
    cs->Pz = round_op(c, s2.get());
  }
  // ghost-point boundary vectors (Sec. III.A): op(f) = M f + bc
  HTT e0 = h_indicator(ne, 0), eN = h_indicator(ne, int64_t(Ne) - 1);
  const bool rot = P.rot != 0.0;
  std::unique_ptr<HTT> u_wall, v_wall, u_far;
  if (rot) {
    u_wall.reset(new HTT(h_trig(nx, om, 0.0, true, P.rot)));    // u_G = rot sin(theta)
    v_wall.reset(new HTT(h_trig(nx, om, 0.0, false, -P.rot)));  // v_G = -rot cos(theta)
  }
  if (P.u_inf != 0.0) u_far.reset(new HTT(h_const(nx, P.u_inf)));
  auto bc_eta = [&](const HTT* wall, const HTT* far, double sw, double sf) -> qtt_mps* {
    MpsP a(nullptr, free_mps), b(nullptr, free_mps);
    if (wall) a = mk(m2(h_scale(e0, sw), *wall));
    if (far) b = mk(m2(h_scale(eN, sf), *far));
    return add_round(c, a.get(), b.get());
  };
  MpsP b1u = mk(bc_eta(u_wall.get(), u_far.get(), -1 / (2 * de), 1 / (2 * de)));
  MpsP b1v(bc_eta(v_wall.get(), nullptr, -1 / (2 * de), 1 / (2 * de)), free_mps);
  MpsP b2u = mk(bc_eta(u_wall.get(), u_far.get(), 1 / (de * de), 1 / (de * de)));
  MpsP b2v(bc_eta(v_wall.get(), nullptr, 1 / (de * de), 1 / (de * de)), free_mps);
  auto had_or_null = [&](const qtt_mps* a, const qtt_mps* b) -> qtt_mps* {
    if (!a || !b) return nullptr;
    return had_round(c, a, b);
  };
  if (b1u) {
    cs->bcx_u = had_or_null(cx_eta.get(), b1u.get());
    cs->bcz_u = had_or_null(cz_eta.get(), b1u.get());
  }
  if (b1v) {
    cs->bcx_v = had_or_null(cx_eta.get(), b1v.get());
    cs->bcz_v = had_or_null(cz_eta.get(), b1v.get());
  }
  if (b2u) {
    cs->JbcLap_u = mps_copy(c, b2u.get());
    mps_scale(c, cs->JbcLap_u, aE);
  }
  if (b2v) {
    cs->JbcLap_v = mps_copy(c, b2v.get());
    mps_scale(c, cs->JbcLap_v, aE);
  }
  {
    MpsP bd(add_round(c, cs->bcx_u, cs->bcz_v), free_mps);
    if (bd) {
      MpsP jw = mk(mps_copy(c, cs->absJ));
      mps_scale(c, jw.get(), -1.0 / P.dt);
      cs->bcdiv_w = had_round(c, jw.get(), bd.get());
    }
  }
  cs->ctx = &c;
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  return cs.release();
}

// ------------------------------------------------------------------ forces (App. F)

namespace {

// Rows 0 and 1 of u, v and row 0 of p arrive dense (length N_xi).  Wall values are the
// analytic ghost values (eq:rot_bc).  One block reduces over the wall nodes.
__global__ void __launch_bounds__(1024) k_forces(int Nx, const double* __restrict__ u0, const double* __restrict__ u1,
                                                 const double* __restrict__ v0, const double* __restrict__ v1,
                                                 const double* __restrict__ p0, double rot, double deta, double dxi,
                                                 double lnR, double rw, double Re, double D, double* out) {
  __shared__ double red[2][32];
  const double pi = 3.141592653589793;
  double fd = 0.0, fl = 0.0;
  for (int j = threadIdx.x; j < Nx; j += blockDim.x) {
    double th = 2.0 * pi * j * dxi;
    double thp = 2.0 * pi * ((j + 1) % Nx) * dxi, thm = 2.0 * pi * ((j - 1 + Nx) % Nx) * dxi;
    double uw = rot * sin(th), vw = -rot * cos(th);
    double ue = (-3.0 * uw + 4.0 * u0[j] - u1[j]) / (2.0 * deta);
    double ve = (-3.0 * vw + 4.0 * v0[j] - v1[j]) / (2.0 * deta);
    double ux = (rot * sin(thp) - rot * sin(thm)) / (2.0 * dxi);
    double vx = (-rot * cos(thp) + rot * cos(thm)) / (2.0 * dxi);
    double cxx = -sin(th) / (2.0 * pi * rw), cxe = cos(th) / (lnR * rw);
    double czx = cos(th) / (2.0 * pi * rw), cze = sin(th) / (lnR * rw);
    double du_dx = cxx * ux + cxe * ue, du_dz = czx * ux + cze * ue;
    double dv_dx = cxx * vx + cxe * ve, dv_dz = czx * vx + cze * ve;
    double div = du_dx + dv_dz;
    double iso = -(p0[j] + 2.0 / (3.0 * Re) * div);
    double sxx = iso + 2.0 / Re * du_dx, szz = iso + 2.0 / Re * dv_dz, sxz = (du_dz + dv_dx) / Re;
    double nxv = cos(th), nzv = sin(th);
    fd += sxx * nxv + sxz * nzv;
    fl += sxz * nxv + szz * nzv;
  }
  for (int o = 16; o > 0; o >>= 1) {
    fd += __shfl_xor_sync(0xffffffffu, fd, o);
    fl += __shfl_xor_sync(0xffffffffu, fl, o);
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = fd;
    red[1][threadIdx.x >> 5] = fl;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    double a = 0, b = 0;
    for (int i = 0; i < int(blockDim.x >> 5); ++i) {
      a += red[0][i];
      b += red[1][i];
    }
    double ds = 0.5 * D * 2.0 * pi * dxi;
    out[0] = 2.0 * a * ds;
    out[1] = 2.0 * b * ds;
  }
}

__global__ void k_check_finite(const double* __restrict__ x, int64_t n, double* flag) {
  for (int64_t e = blockIdx.x * int64_t(blockDim.x) + threadIdx.x; e < n; e += int64_t(gridDim.x) * blockDim.x)
    if (!isfinite(x[e])) *flag = 0.0;
}

}  // namespace

// flag = 0 if any of x[0..n) is NaN or Inf (every writer writes 0, so the race is benign).
void check_finite(Ctx& c, const double* x, int64_t n, double* flag) {
  const int threads = 256;
  const int blocks = int(std::min<int64_t>((n + threads - 1) / threads, 4 * int64_t(c.num_sms)));
  k_check_finite<<<std::max(blocks, 1), threads, 0, c.stream>>>(x, n, flag);
  after_launch(c, "check_finite");
}

// Row I of a 2-D field (App. C): the eta-bit cores are sliced at the bits of I, the xi-bit
// cores kept; the result is decoded to the dense row (length 2^n_xi).
void read_row(Ctx& c, const Case& cs, const qtt_mps* x, int64_t I, double* row_dev) {
  const int ne = cs.P.n_eta;
  const int d = 2;
  DBuf t(&c, 1);
  fill(c, t.p, 1, 1.0);
  int64_t rows = 1;
  for (int k = 0; k < x->n; ++k) {
    int a0 = x->bonds[k], a1 = x->bonds[k + 1];
    auto [ax, l] = cs.layout[k];
    if (ax == 0) {
      int bit = int((I >> (ne - 1 - l)) & 1);
      DBuf nt(&c, size_t(rows) * a1);
      gemm(c, 1, rows, a1, a0, 1.0, t.p, 0, a0, 1, x->core(k) + bit * a1, 0, int64_t(d) * a1, 1, 0.0, nt.p, 0, a1, 1);
      t = std::move(nt);
    } else {
      DBuf nt(&c, size_t(rows) * d * a1);
      gemm(c, 1, rows, int64_t(d) * a1, a0, 1.0, t.p, 0, a0, 1, x->core(k), 0, int64_t(d) * a1, 1, 0.0, nt.p, 0,
           int64_t(d) * a1, 1);
      t = std::move(nt);
      rows *= d;
    }
  }
  copy(c, row_dev, t.p, rows);
}

void case_forces(Ctx& c, Case& cs, double* out_dev) {
  const int64_t Nx = int64_t(1) << cs.P.n_xi;
  DBuf rows(&c, size_t(5 * Nx));
  read_row(c, cs, cs.u, 0, rows.p);
  read_row(c, cs, cs.u, 1, rows.p + Nx);
  read_row(c, cs, cs.v, 0, rows.p + 2 * Nx);
  read_row(c, cs, cs.v, 1, rows.p + 3 * Nx);
  read_row(c, cs, cs.p, 0, rows.p + 4 * Nx);
  const double rw = 0.5 * cs.P.D;  // r at the wall ghost row: (D/2) R^0
  k_forces<<<1, 1024, 0, c.stream>>>(int(Nx), rows.p, rows.p + Nx, rows.p + 2 * Nx, rows.p + 3 * Nx, rows.p + 4 * Nx,
                                     cs.P.rot, cs.deta, cs.dxi, std::log(cs.P.R), rw, cs.P.Re, cs.P.D, out_dev);
  after_launch(c, "forces");
}

// ------------------------------------------------------------------ the fractional step

// Independent parts run on worker streams: the four MPO-MPS products (4 workers), the
// right-hand side and momentum solve of each velocity component (2 workers), the two
// projection fits (2 workers).  The Poisson solve couples u* and v* and runs on the caller's
// stream.  Results that cross streams are allocated before the fork.
void step(Ctx& c, Case& cs, double* rec, bool with_forces, bool extrapolate) {
  AlsCtl* ctl = reinterpret_cast<AlsCtl*>(rec);
  const qtt_case_params& P = cs.P;
  const int chi = P.chi;
  const double dt = P.dt;
  const int n = cs.u->n;
  // (i) convective derivatives (MPO-MPS products rounded to chi, Sec. II.A.2)
  cs.mark(c, 0);
  std::unique_ptr<ProfScope> ph(new ProfScope(c, KC_PH_APPLY));
  MpsP dxu = mk(new_mps(&c, n, 2, apply_bonds(cs.Dx, cs.u, chi)));
  MpsP dzu = mk(new_mps(&c, n, 2, apply_bonds(cs.Dz, cs.u, chi)));
  MpsP dxv = mk(new_mps(&c, n, 2, apply_bonds(cs.Dx, cs.v, chi)));
  MpsP dzv = mk(new_mps(&c, n, 2, apply_bonds(cs.Dz, cs.v, chi)));
  fork(c, 4);
  auto apply = P.apply == QTT_APPLY_SKETCH ? apply_round_sketch : apply_round_gram;
  apply(worker(c, 0), cs.Dx, cs.u, chi, 0.0, dxu.get());
  apply(worker(c, 1), cs.Dz, cs.u, chi, 0.0, dzu.get());
  apply(worker(c, 2), cs.Dx, cs.v, chi, 0.0, dxv.get());
  apply(worker(c, 3), cs.Dz, cs.v, chi, 0.0, dzv.get());
  join(c, 4);
  cs.mark(c, 1);
  // explicit right-hand sides (eq:intermediate_vel_eq), one fit each, warm start u (v), then
  // (ii) implicit momentum H v* = |J| (.) rhs + dt/Re |J| bcLap (ALS, warm start v^m)
  ph.reset(new ProfScope(c, KC_PH_RHS));
  std::vector<Term> tu = {Term::vec(1.0, cs.u), Term::had(-dt, cs.u, dxu.get()), Term::had(-dt, cs.v, dzu.get())};
  if (cs.bcx_u) tu.push_back(Term::had(-dt, cs.u, cs.bcx_u));
  if (cs.bcz_u) tu.push_back(Term::had(-dt, cs.v, cs.bcz_u));
  std::vector<Term> tv_ = {Term::vec(1.0, cs.v), Term::had(-dt, cs.u, dxv.get()), Term::had(-dt, cs.v, dzv.get())};
  if (cs.bcx_v) tv_.push_back(Term::had(-dt, cs.u, cs.bcx_v));
  if (cs.bcz_v) tv_.push_back(Term::had(-dt, cs.v, cs.bcz_v));
  MpsP rhs_u = mk(mps_copy(c, cs.u));
  MpsP rhs_v = mk(mps_copy(c, cs.v));
  MpsP us = mk(mps_copy(c, cs.u));
  MpsP vs = mk(mps_copy(c, cs.v));
  const double kk = dt / P.Re;
  std::vector<Term> mu = {Term::mpo(1.0, cs.Jdiag, rhs_u.get())};
  if (cs.JbcLap_u) mu.push_back(Term::vec(kk, cs.JbcLap_u));
  std::vector<Term> mv = {Term::mpo(1.0, cs.Jdiag, rhs_v.get())};
  if (cs.JbcLap_v) mv.push_back(Term::vec(kk, cs.JbcLap_v));
  // Poisson warm start: p^m, or (poisson_warm = 1, once a previous pressure exists) the
  // extrapolation 2 p^m - p^(m-1) fitted at the pressure's bonds from p^m, on a third worker
  // while the momentum solves run; p^m is kept as the next step's p^(m-1)
  const int nw = P.poisson_warm == 1 ? 3 : 2;
  MpsP pw = extrapolate ? mk(mps_copy(c, cs.p)) : MpsP(nullptr, free_mps);
  fork(c, nw);
  fit(worker(c, 0), tu, rhs_u.get(), P.fit_sweeps, true);
  fit(worker(c, 1), tv_, rhs_v.get(), P.fit_sweeps, true);
  als(worker(c, 0), cs.H, mu, us.get(), P.mom, true, ctl + 0, &cs.body_launches[0]);
  als(worker(c, 1), cs.H, mv, vs.get(), P.mom, true, ctl + 1, &cs.body_launches[1]);
  if (P.poisson_warm == 1) {
    Ctx& w2 = worker(c, 2);
    if (extrapolate) fit(w2, {Term::vec(2.0, cs.p), Term::vec(-1.0, cs.p_prev)}, pw.get(), P.fit_sweeps, true);
    copy(w2, cs.p_prev->buf.p, cs.p->buf.p, cs.p->off[n]);
    if (extrapolate) copy(w2, cs.p->buf.p, pw->buf.p, cs.p->off[n]);
  }
  join(c, nw);
  cs.mark(c, 2);
  // (iii) pressure Poisson, J-weighted (Sec. III.C): (-|J| Lap_h^p) p = -|J| (.) div(v*) / dt
  ph.reset(new ProfScope(c, KC_PH_POI));
  std::vector<Term> pr = {Term::mpo(1.0, cs.Px, us.get()), Term::mpo(1.0, cs.Pz, vs.get())};
  if (cs.bcdiv_w) pr.push_back(Term::vec(1.0, cs.bcdiv_w));
  {
    DigitsScope fp64(c, kDigitsFP64);   // the divergence and the Poisson solve stay FP64 at any precision
    als(c, cs.Ap, pr, cs.p, P.poi, true, ctl + 2, &cs.body_launches[2]);
  }
  // projection v = v* - dt grad_h p (one fit each, warm start v*)
  cs.mark(c, 3);
  ph.reset(new ProfScope(c, KC_PH_PROJ));
  MpsP un = mk(mps_copy(c, us.get()));
  MpsP vn = mk(mps_copy(c, vs.get()));
  fork(c, 2);
  fit(worker(c, 0), {Term::vec(1.0, us.get()), Term::mpo(-dt, cs.Dxp, cs.p)}, un.get(), P.fit_sweeps, true);
  fit(worker(c, 1), {Term::vec(1.0, vs.get()), Term::mpo(-dt, cs.Dzp, cs.p)}, vn.get(), P.fit_sweeps, true);
  join(c, 2);
  ph.reset();
  cs.mark(c, 4);
  // new state into the same buffers (the captured graph reads and writes these addresses)
  copy(c, cs.u->buf.p, un->buf.p, cs.u->off[n]);
  copy(c, cs.v->buf.p, vn->buf.p, cs.v->off[n]);
  fill(c, rec + kStepRecFinite, 1, 1.0);
  check_finite(c, cs.u->buf.p, cs.u->off[n], rec + kStepRecFinite);
  check_finite(c, cs.v->buf.p, cs.v->off[n], rec + kStepRecFinite);
  if (with_forces) case_forces(c, cs, rec + kStepRecForces);
}

static void capture(Ctx& c, Case& cs, bool with_forces) {
  cs.drop_graph();
  init_kernel_attributes();
  cg_init_attributes();
  cg_tc_init_attributes();
  init_ozaki_attributes();
  for (int i = 0; i < 4; ++i) worker(c, i);
  if (!cs.gstream) QTT_CUDA(cudaStreamCreateWithFlags(&cs.gstream, cudaStreamNonBlocking));
  if (!cs.ev_in) QTT_CUDA(cudaEventCreateWithFlags(&cs.ev_in, cudaEventDisableTiming));
  if (!cs.ev_out) QTT_CUDA(cudaEventCreateWithFlags(&cs.ev_out, cudaEventDisableTiming));
  if (!cs.rec) QTT_CUDA(cudaMalloc(&cs.rec, kStepRecDoubles * sizeof(double)));
  // The graph's own split-K tile counters and pool arena (one per case, for the context and
  // each worker), so that the graphs of different cases may replay concurrently.
  std::vector<Ctx*> tree{&c};
  for (Ctx* w : c.workers) tree.push_back(w);
  while (cs.tile_ctr.size() < tree.size()) {
    int* t = nullptr;
    QTT_CUDA(cudaMalloc(&t, kTileCounters * sizeof(int)));
    cs.tile_ctr.push_back(t);
    QTT_CUDA(cudaMemsetAsync(t, 0, kTileCounters * sizeof(int), c.stream));
  }
  QTT_CUDA(cudaStreamSynchronize(c.stream));
  std::vector<int*> saved_ctr;
  for (size_t i = 0; i < tree.size(); ++i) {
    saved_ctr.push_back(tree[i]->tile_ctr);
    tree[i]->tile_ctr = cs.tile_ctr[i];
  }
  auto restore_ctr = [&]() {
    for (size_t i = 0; i < tree.size(); ++i) tree[i]->tile_ctr = saved_ctr[i];
  };
  cudaStream_t saved = c.stream;
  const bool prof_on = c.root->prof.on;
  c.root->prof.on = false;   // no timing events inside a graph
  c.pool->begin_capture(&cs);
  for (Ctx* w : c.workers) w->pool->begin_capture(&cs);
  c.stream = cs.gstream;
  const int64_t n0 = c.root->launches;
  for (int i = 0; i < 5; ++i)
    if (!cs.ph_ev[i]) QTT_CUDA(cudaEventCreate(&cs.ph_ev[i]));
  cs.capturing = true;
  cudaError_t err = cudaStreamBeginCapture(cs.gstream, cudaStreamCaptureModeRelaxed);
  try {
    if (err != cudaSuccess) throw Error(QTT_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(err));
    step(c, cs, cs.rec, with_forces, cs.P.poisson_warm == 1);
  } catch (...) {
    cs.capturing = false;
    cudaGraph_t g = nullptr;
    cudaStreamEndCapture(cs.gstream, &g);
    if (g) cudaGraphDestroy(g);
    c.stream = saved;
    c.pool->end_capture();
    for (Ctx* w : c.workers) w->pool->end_capture();
    restore_ctr();
    c.root->prof.on = prof_on;
    c.root->launches = n0;
    throw;
  }
  err = cudaStreamEndCapture(cs.gstream, &cs.graph);
  cs.capturing = false;
  c.stream = saved;
  c.pool->end_capture();
  for (Ctx* w : c.workers) w->pool->end_capture();
  restore_ctr();
  c.root->prof.on = prof_on;
  cs.graph_launches = c.root->launches - n0 - cs.body_launches[0] - cs.body_launches[1] - cs.body_launches[2];
  c.root->launches = n0;
  if (err != cudaSuccess) throw Error(QTT_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(err));
  QTT_CUDA(cudaGraphInstantiate(&cs.gexec, cs.graph, 0));
  cs.graph_forces = with_forces;
}

// The first step after the state was set has no previous pressure: with the extrapolated warm
// start it runs eagerly from p^m (the captured graph always extrapolates).
static bool first_step_eager(const Case& cs) { return cs.P.poisson_warm == 1 && !cs.prev_valid; }

void run_steps(Ctx& c, Case& cs, int nsteps, bool with_forces, double* rec_all) {
  if (!cs.use_graph) {
    for (int s = 0; s < nsteps; ++s) {
      step(c, cs, rec_all + int64_t(kStepRecDoubles) * s, with_forces, cs.P.poisson_warm == 1 && cs.prev_valid);
      cs.prev_valid = true;
    }
    return;
  }
  int s0 = 0;
  cs.last_first_eager = false;
  if (nsteps > 0 && first_step_eager(cs)) {
    step(c, cs, rec_all, with_forces, false);
    cs.prev_valid = true;
    cs.last_first_eager = true;
    s0 = 1;
  }
  if (s0 < nsteps && (!cs.gexec || cs.graph_forces != with_forces)) capture(c, cs, with_forces);
  for (int s = s0; s < nsteps; ++s) {
    QTT_CUDA(cudaEventRecord(cs.ev_in, c.stream));
    QTT_CUDA(cudaStreamWaitEvent(cs.gstream, cs.ev_in, 0));
    QTT_CUDA(cudaGraphLaunch(cs.gexec, cs.gstream));
    QTT_CUDA(cudaEventRecord(cs.ev_out, cs.gstream));
    QTT_CUDA(cudaStreamWaitEvent(c.stream, cs.ev_out, 0));
    copy(c, rec_all + int64_t(kStepRecDoubles) * s, cs.rec, kStepRecDoubles);
  }
}

void run_steps_batch(Ctx& c, const std::vector<Case*>& cases, int nsteps, bool with_forces, double* rec_all) {
  // every graph first (captures are host work on the context's streams), then the replays:
  // one stream per case, ordered after the context stream, step s of every case enqueued
  // before step s + 1 of any
  // cases whose first step has no previous pressure take it eagerly, on the context stream,
  // before the replays start
  std::vector<char> eager0(cases.size(), 0);
  for (size_t i = 0; i < cases.size(); ++i) {
    cases[i]->last_first_eager = false;
    if (nsteps > 0 && first_step_eager(*cases[i])) {
      step(c, *cases[i], rec_all + int64_t(i) * nsteps * kStepRecDoubles, with_forces, false);
      cases[i]->prev_valid = true;
      cases[i]->last_first_eager = true;
      eager0[i] = 1;
    }
  }
  for (Case* cs : cases)
    if (!cs->gexec || cs->graph_forces != with_forces) capture(c, *cs, with_forces);
  QTT_CUDA(cudaEventRecord(cases[0]->ev_in, c.stream));
  for (Case* cs : cases) QTT_CUDA(cudaStreamWaitEvent(cs->gstream, cases[0]->ev_in, 0));
  for (int s = 0; s < nsteps; ++s)
    for (size_t i = 0; i < cases.size(); ++i) {
      Case& cs = *cases[i];
      if (s == 0 && eager0[i]) continue;
      QTT_CUDA(cudaGraphLaunch(cs.gexec, cs.gstream));
      double* dst = rec_all + (int64_t(i) * nsteps + s) * kStepRecDoubles;
      QTT_CUDA(cudaMemcpyAsync(dst, cs.rec, kStepRecDoubles * sizeof(double), cudaMemcpyDeviceToDevice, cs.gstream));
    }
  for (Case* cs : cases) {
    QTT_CUDA(cudaEventRecord(cs->ev_out, cs->gstream));
    QTT_CUDA(cudaStreamWaitEvent(c.stream, cs->ev_out, 0));
  }
}

}  // namespace qtt
