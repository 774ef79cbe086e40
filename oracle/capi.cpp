// C interface of the CPU oracle, loaded by the tests (ctypes) and by the
// timed CPU baseline of the benchmark.  TEST INFRASTRUCTURE ONLY (see scalar.h).
//
// Single-environment arrays are plain [nq] / [nv] / [nq + nv] vectors;
// batched arrays are environment-major ([B][...]).
#include <algorithm>
#include <atomic>
#include <cstring>
#include <thread>
#include <vector>

#include "integrator.h"

using namespace orc;

namespace {
Model& M(void* h) { return *static_cast<Model*>(h); }

template <class Fn> void parallel_for(int n, int nthreads, Fn fn) {
  nthreads = std::max(1, std::min(nthreads, n));
  if (nthreads == 1) { for (int i = 0; i < n; ++i) fn(i); return; }
  std::atomic<int> next(0);
  std::vector<std::thread> th;
  for (int t = 0; t < nthreads; ++t)
    th.emplace_back([&] {
      for (int i = next++; i < n; i = next++) fn(i);
    });
  for (auto& x : th) x.join();
}
Opts make_opts(double T, int NI, double rtol, double atol, double h0, int max_steps, int method) {
  Opts o;
  o.T = T; o.NI = NI; o.rtol = rtol; o.atol = atol; o.h0 = h0; o.max_steps = max_steps;
  o.method = (method >= METHOD_DOPRI5 && method <= METHOD_EULER) ? method : METHOD_DOPRI5;
  return o;
}
void put_stats(const Result& r, int* s) { s[0] = r.status; s[1] = r.nsteps; s[2] = r.nrej; s[3] = r.nrhs; }
}  // namespace

extern "C" {

void* orc_create(const double* body, int nbody, const double* geom, int ngeom, const double* pair, int npair,
                 const double* act, int nact, const double* opt, const double* qpos0, char* err, int errlen) {
  Model* m = new Model();
  std::string e = build_model(*m, body, nbody, geom, ngeom, pair, npair, act, nact, opt, qpos0);
  if (!e.empty()) {
    if (err && errlen > 0) { std::strncpy(err, e.c_str(), errlen - 1); err[errlen - 1] = 0; }
    delete m;
    return nullptr;
  }
  return m;
}
void orc_free(void* h) { delete static_cast<Model*>(h); }

void orc_dims(void* h, int* out) {
  Model& m = M(h);
  out[0] = m.nq; out[1] = m.nv; out[2] = m.nu; out[3] = m.nslot; out[4] = m.nrowmax; out[5] = (int)m.body.size();
}
double orc_body_invw(void* h, int b) { return M(h).body_invw[b]; }
double orc_pair_invw(void* h, int p) { return M(h).pair[p].invw; }

// Coefficients of scheme `method`: aq, av (7 x 7), b, bhat, c; returns the
// number of stages (stage 0 included).
int orc_tableau(int method, double* aq, double* av, double* b, double* bhat, double* c) {
  const Tableau& t = tableau_of(method);
  for (int i = 0; i < 7; ++i) {
    for (int j = 0; j < 7; ++j) { aq[7 * i + j] = t.aq[i][j]; av[7 * i + j] = t.av[i][j]; }
    b[i] = t.b[i]; bhat[i] = t.bhat[i]; c[i] = t.c[i];
  }
  return t.S;
}

int orc_kinematics(void* h, const double* q, double* R, double* p, double* com) {
  Model& m = M(h);
  Kin<double> k;
  kinematics(m, q, k);
  for (size_t b = 0; b < m.body.size(); ++b) {
    for (int i = 0; i < 9; ++i) R[9 * b + i] = k.R[b][i];
    for (int i = 0; i < 3; ++i) { p[3 * b + i] = k.p[b][i]; com[3 * b + i] = k.c[b][i]; }
  }
  return 0;
}
// Linear (3 x nv) and angular (3 x nv) Jacobians of a world point fixed to body b.
int orc_point_jacobian(void* h, const double* q, int b, const double* x, double* Jlin, double* Jang) {
  Model& m = M(h);
  Kin<double> k;
  kinematics(m, q, k);
  V3<double> xp = {x[0], x[1], x[2]};
  for (int i = 0; i < m.nv; ++i) {
    V3<double> pv = dof_point_vel(m, k, i, b, xp);
    const bool moves = m.anc[b][m.dof_body[i]];
    for (int r = 0; r < 3; ++r) {
      Jlin[r * m.nv + i] = pv[r];
      Jang[r * m.nv + i] = moves ? k.s[i][r] : 0.0;
    }
  }
  return 0;
}
int orc_mass(void* h, const double* q, double* Mout) {
  Model& m = M(h);
  Kin<double> k;
  kinematics(m, q, k);
  std::vector<double> Mm;
  crba(m, k, Mm);
  std::copy(Mm.begin(), Mm.end(), Mout);
  return 0;
}
int orc_bias(void* h, const double* q, const double* v, double* c) {
  Model& m = M(h);
  Kin<double> k;
  kinematics(m, q, k);
  std::vector<double> cc;
  rne(m, k, v, cc);
  std::copy(cc.begin(), cc.end(), c);
  return 0;
}
int orc_applied(void* h, const double* q, const double* v, const double* u, double* tau) {
  std::vector<double> t;
  applied(M(h), q, v, u, t);
  std::copy(t.begin(), t.end(), tau);
  return 0;
}
// out per slot (16): r, pos[3], n[3], t1[3], t2[3], bodyA, bodyB, pair
int orc_contacts(void* h, const double* q, double* out) {
  Model& m = M(h);
  Kin<double> k;
  kinematics(m, q, k);
  std::vector<Contact<double>> ct;
  contacts(m, k, ct);
  for (int s = 0; s < m.nslot; ++s) {
    double* o = out + 16 * s;
    o[0] = ct[s].r;
    for (int i = 0; i < 3; ++i) { o[1 + i] = ct[s].pos[i]; o[4 + i] = ct[s].n[i]; o[7 + i] = ct[s].t1[i]; o[10 + i] = ct[s].t2[i]; }
    o[13] = ct[s].bodyA; o[14] = ct[s].bodyB; o[15] = ct[s].pair;
  }
  return 0;
}
double orc_impedance(void* h, double r, int cfd) { return impedance<double>(M(h), r, cfd != 0); }

// Constraint rows of the included contacts; returns the number of rows.
int orc_rows(void* h, const double* q, const double* v, int cfd, double* J, double* aref, double* D, int* slot) {
  Model& m = M(h);
  Kin<double> k;
  kinematics(m, q, k);
  std::vector<Contact<double>> ct;
  contacts(m, k, ct);
  Rows<double> R;
  make_rows(m, k, ct, v, cfd != 0, R);
  std::copy(R.J.begin(), R.J.end(), J);
  std::copy(R.aref.begin(), R.aref.end(), aref);
  std::copy(R.D.begin(), R.D.end(), D);
  std::copy(R.slot.begin(), R.slot.end(), slot);
  return R.nr;
}
// info: nr, newton iterations, noconv, spd_fail
int orc_rhs(void* h, const double* q, const double* v, const double* u, int cfd, double* a, double* f, int* active, int* info) {
  Model& m = M(h);
  RhsDiag<double> dg;
  bool ok = rhs<double>(m, q, v, u, cfd != 0, a, &dg);
  if (f) std::copy(dg.f.begin(), dg.f.end(), f);
  if (active) for (int r = 0; r < dg.rows.nr; ++r) active[r] = dg.info.active[r];
  if (info) { info[0] = dg.rows.nr; info[1] = dg.info.iters; info[2] = dg.info.noconv; info[3] = dg.info.spd_fail; }
  return ok ? 0 : 1;
}
// Jacobians of F (or F~) w.r.t. q (nv x nq), v (nv x nv), u (nv x nu).
int orc_rhs_jacobian(void* h, const double* q, const double* v, const double* u, int cfd, double* Jq, double* Jv, double* Ju) {
  using D = Dual<double>;
  Model& m = M(h);
  const int nq = m.nq, nv = m.nv, nu = m.nu;
  std::vector<D> qd(nq), vd(nv), ud(std::max(nu, 1)), a(nv);
  for (int dir = 0; dir < nq + nv + nu; ++dir) {
    for (int i = 0; i < nq; ++i) qd[i] = D(q[i], dir == i ? 1.0 : 0.0);
    for (int i = 0; i < nv; ++i) vd[i] = D(v[i], dir == nq + i ? 1.0 : 0.0);
    for (int i = 0; i < nu; ++i) ud[i] = D(u[i], dir == nq + nv + i ? 1.0 : 0.0);
    rhs<D>(m, qd.data(), vd.data(), ud.data(), cfd != 0, a.data());
    for (int i = 0; i < nv; ++i) {
      if (dir < nq) Jq[i * nq + dir] = a[i].d;
      else if (dir < nq + nv) Jv[i * nv + dir - nq] = a[i].d;
      else Ju[i * nu + dir - nq - nv] = a[i].d;
    }
  }
  return 0;
}
void orc_integrate_pos(void* h, const double* q, const double* dlt, double* out) { integrate_pos<double>(M(h), q, dlt, out); }

int orc_rollout(void* h, const double* x0, const double* ctrl, double T, int NI, double rtol, double atol, double h0,
                int max_steps, double* xT, double* xb, int* stats, double* hlog, int hcap, int method) {
  std::vector<double> hl;
  Result r = rollout<double>(M(h), x0, ctrl, make_opts(T, NI, rtol, atol, h0, max_steps, method), xT, xb, nullptr, &hl,
                             nullptr, 0);
  put_stats(r, stats);
  if (hlog) for (int i = 0; i < std::min<int>(hcap, (int)hl.size()); ++i) hlog[i] = hl[i];
  return (int)hl.size();
}
int orc_replay(void* h, const double* x0, const double* ctrl, double T, int NI, const double* hlog, int n, double* xT,
               double* xb, int method) {
  Result r = rollout<double>(M(h), x0, ctrl, make_opts(T, NI, 0, 0, 0, 0, method), xT, xb, nullptr, nullptr, hlog, n);
  return r.nsteps;
}
// Error norm of a given embedded difference e (2 nv tangent components)
// between the states (q0, v0) and (q1, v1): the scalar the step controller
// compares with 1.
double orc_error_norm(void* h, const double* q0, const double* v0, const double* q1, const double* v1,
                      const double* e, double rtol, double atol) {
  return error_norm<double>(M(h), q0, v0, q1, v1, e, rtol, atol);
}
// Error norm of one DOPRI5 attempt of size hs from x = [q; v] (controls u):
// the value the adaptive controller compares with 1.
double orc_step_error(void* h, const double* x, const double* u, double hs, double rtol, double atol, int method) {
  Model& m = M(h);
  const int nq = m.nq, nv = m.nv;
  std::vector<double> a1(nv), q7(nq), v7(nv), a7(nv), e(2 * nv);
  StageRhs<double> f{m, false};
  f(x, x + nq, u, a1.data());
  rk_step(m, tableau_of(method), f, x, x + nq, a1.data(), u, hs, q7.data(), v7.data(), a7.data(), e.data());
  return error_norm<double>(m, x, x + nq, q7.data(), v7.data(), e.data(), rtol, atol);
}
int orc_step_jacobian(void* h, const double* q, const double* v, const double* u, double hs, int cfd, double* Jx,
                      double* Ju, int method) {
  Model& m = M(h);
  std::vector<double> A, B;
  step_jacobian(m, q, v, u, hs, cfd != 0, A, B, method);
  std::copy(A.begin(), A.end(), Jx);
  if (Ju && m.nu) std::copy(B.begin(), B.end(), Ju);
  return 0;
}
int orc_rollout_grad(void* h, const double* x0, const double* ctrl, double T, int NI, double rtol, double atol,
                     double h0, int max_steps, int cfd, const double* xT_bar, const double* xb_bar, double* xT,
                     double* x0_bar, double* ctrl_bar, int* stats, int method) {
  Result r = rollout_grad(M(h), x0, ctrl, make_opts(T, NI, rtol, atol, h0, max_steps, method), cfd != 0, xT_bar, xb_bar,
                          xT, x0_bar, ctrl_bar);
  put_stats(r, stats);
  return 0;
}

// Gradient along a given accepted step sequence (per environment: hlog[e][0:n[e]]);
// p_bar [B][np] (optional) receives the model-parameter gradients.
int orc_batch_replay_grad(void* h, int B, const double* x0, const double* ctrl, const double* T, int NI, const double* hlog,
                          int hstride, const int* n, int cfd, const double* xT_bar, const double* xb_bar, double* xT,
                          double* x0_bar, double* ctrl_bar, int nthreads, int method, double* p_bar) {
  Model& m = M(h);
  const int nx = m.nq + m.nv, nu = m.nu, np = n_params(m);
  parallel_for(B, nthreads, [&](int b) {
    rollout_grad(m, x0 + (size_t)b * nx, ctrl ? ctrl + (size_t)b * NI * nu : nullptr, make_opts(T[b], NI, 1, 1, 1, 1 << 30, method),
                 cfd != 0, xT_bar + (size_t)b * nx, xb_bar ? xb_bar + (size_t)b * (NI + 1) * nx : nullptr,
                 xT + (size_t)b * nx, x0_bar + (size_t)b * nx, ctrl_bar ? ctrl_bar + (size_t)b * NI * nu : nullptr,
                 hlog + (size_t)b * hstride, n[b], p_bar ? p_bar + (size_t)b * np : nullptr);
  });
  return 0;
}
// Number of model parameters of the adjoint (solref 2, solimp 4, one friction per pair).
int orc_nparams(void* h) { return n_params(M(h)); }
int orc_batch_rollout(void* h, int B, const double* x0, const double* ctrl, const double* T, int NI, double rtol,
                      double atol, double h0, int max_steps, double* xT, double* xb, int* stats, int nthreads, int method) {
  Model& m = M(h);
  const int nx = m.nq + m.nv, nu = m.nu;
  parallel_for(B, nthreads, [&](int b) {
    Result r = rollout<double>(m, x0 + (size_t)b * nx, ctrl ? ctrl + (size_t)b * NI * nu : nullptr,
                               make_opts(T[b], NI, rtol, atol, h0, max_steps, method), xT + (size_t)b * nx,
                               xb ? xb + (size_t)b * (NI + 1) * nx : nullptr, nullptr, nullptr, nullptr, 0);
    put_stats(r, stats + 4 * b);
  });
  return 0;
}
int orc_batch_grad(void* h, int B, const double* x0, const double* ctrl, const double* T, int NI, double rtol,
                   double atol, double h0, int max_steps, int cfd, const double* xT_bar, const double* xb_bar,
                   double* xT, double* x0_bar, double* ctrl_bar, int* stats, int nthreads, int method) {
  Model& m = M(h);
  const int nx = m.nq + m.nv, nu = m.nu;
  parallel_for(B, nthreads, [&](int b) {
    Result r = rollout_grad(m, x0 + (size_t)b * nx, ctrl ? ctrl + (size_t)b * NI * nu : nullptr,
                            make_opts(T[b], NI, rtol, atol, h0, max_steps, method), cfd != 0, xT_bar + (size_t)b * nx,
                            xb_bar ? xb_bar + (size_t)b * (NI + 1) * nx : nullptr, xT + (size_t)b * nx,
                            x0_bar + (size_t)b * nx, ctrl_bar ? ctrl_bar + (size_t)b * NI * nu : nullptr);
    put_stats(r, stats + 4 * b);
  });
  return 0;
}

// Floating-point operations of one adaptive rollout (counted scalar type).
// search = 1: the constraint solver's active-set search from the unconstrained
// acceleration is counted; 0: the solve is counted as started at its final
// active set (one Newton system and one residual check per right-hand side).
long long orc_count_flops(void* h, const double* x0, const double* ctrl, double T, int NI, double rtol, double atol,
                          double h0, int max_steps, int* stats, int search, int method) {
  Model& m = M(h);
  const int nx = m.nq + m.nv, nu = m.nu;
  std::vector<Cnt> xc(nx), uc((size_t)std::max(1, NI * nu)), xTc(nx);
  for (int i = 0; i < nx; ++i) xc[i] = Cnt(x0[i]);
  for (int i = 0; i < NI * nu; ++i) uc[i] = Cnt(ctrl[i]);
  g_flops = 0;
  g_count_search = search;
  Result r = rollout<Cnt>(m, xc.data(), uc.data(), make_opts(T, NI, rtol, atol, h0, max_steps, method), xTc.data(), nullptr,
                          nullptr, nullptr, nullptr, 0);
  put_stats(r, stats);
  return (long long)g_flops;
}

// Algorithmic work of the discrete adjoint of one rollout: for every accepted
// step, the step evaluated once in the counting derivative scalar (value and
// one tangent: the primal recompute plus the linearised step; by the
// transposition principle the reverse sweep of a linear map costs the same
// multiply-adds as the forward one).  The active-set searches are not counted
// (the derivative type searches in plain doubles).
long long orc_count_adjoint_flops(void* h, const double* x0, const double* ctrl, double T, int NI, double rtol,
                                  double atol, double h0, int max_steps, int* stats, int method) {
  using D = Dual<Cnt>;
  Model& m = M(h);
  const int nq = m.nq, nv = m.nv, nx = nq + nv, nu = m.nu;
  std::vector<StepRec> rec;
  std::vector<double> xT(nx);
  const Opts o = make_opts(T, NI, rtol, atol, h0, max_steps, method);
  Result r = rollout<double>(m, x0, ctrl, o, xT.data(), nullptr, &rec,
                             nullptr, nullptr, 0);
  put_stats(r, stats);
  std::vector<D> qd(nq), vd(nv), ud(std::max(nu, 1)), a1(nv), q7(nq), v7(nv), a7(nv), e(2 * nv);
  g_flops = 0;
  g_count_search = 0;
  for (const StepRec& s : rec) {
    for (int i = 0; i < nq; ++i) qd[i] = D(Cnt(s.q[i]), Cnt(1.0));
    for (int i = 0; i < nv; ++i) vd[i] = D(Cnt(s.v[i]), Cnt(1.0));
    for (int i = 0; i < nu; ++i) ud[i] = D(Cnt(ctrl[(size_t)s.k * nu + i]), Cnt(1.0));
    StageRhs<D> f{m, false};
    f(qd.data(), vd.data(), ud.data(), a1.data());
    rk_step(m, tableau_of(o.method), f, qd.data(), vd.data(), a1.data(), ud.data(), s.h, q7.data(), v7.data(), a7.data(),
            e.data());
  }
  return (long long)g_flops;
}

// Optimize-then-discretize (backsolve) gradient of a batch of rollouts
// (environment-major arrays); stats [B][8]: forward status, steps, rejects,
// rhs, then the backward solve's status, steps, rejects, 0.
int orc_batch_grad_otd(void* h, int B, const double* x0, const double* ctrl, const double* T, int NI, double rtol,
                       double atol, double h0, int max_steps, int cfd, const double* xT_bar, const double* xb_bar,
                       double* xT, double* x0_bar, double* ctrl_bar, int* stats, int nthreads, int method) {
  Model& m = M(h);
  const int nx = m.nq + m.nv, nu = m.nu;
  parallel_for(B, nthreads, [&](int b) {
    Result back;
    Result r = rollout_grad_otd(m, x0 + (size_t)b * nx, ctrl ? ctrl + (size_t)b * NI * nu : nullptr,
                                make_opts(T[b], NI, rtol, atol, h0, max_steps, method), cfd != 0, xT_bar + (size_t)b * nx,
                                xb_bar ? xb_bar + (size_t)b * (NI + 1) * nx : nullptr, xT + (size_t)b * nx,
                                x0_bar + (size_t)b * nx, ctrl_bar ? ctrl_bar + (size_t)b * NI * nu : nullptr, &back);
    put_stats(r, stats + 8 * b);
    put_stats(back, stats + 8 * b + 4);
    stats[8 * b + 7] = 0;
  });
  return 0;
}

}  // extern "C"
