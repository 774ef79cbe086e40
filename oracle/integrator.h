// Oracle time integration and discrete adjoint.
//
// TEST INFRASTRUCTURE ONLY (see scalar.h).
//
// Paper passages followed (arXiv 2506.14186):
//   Sec. 3.1           adaptive embedded Runge-Kutta: two orders give an error
//                      estimate, accept/reject, a controller picks the next step
//   App. B.1 (Fig. 12) PID step-size controller with P = 0.2, I = 0.4, D = 0
//   App. C.2           Dormand-Prince 5(4) (cited there) with quaternions
//                      integrated exactly; discretize-then-optimize gradient
//   Fig. 12, Sec. 3.1  Tsitouras 5(4) (the paper's default solver) and the
//                      fixed-step semi-implicit Euler of MuJoCo XLA
//   Sec. 4 (ST)        x' = sg(F) + F~ - sg(F~): values from F, derivatives
//                      from F~ evaluated on the F trajectory
// Step sizes of accepted steps are held constant in the derivative; rejected
// attempts contribute nothing.
#pragma once
#include <cmath>
#include <vector>

#include "dynamics.h"

namespace orc {

// Explicit one-step schemes on (q, v) as partitioned tableaus.  Stage s
// (s = 1 .. S-1) takes
//   V_s = v_n + h sum_{j<s} av[s][j] K_j,
//   Q_s = q_n (+) h sum_{j<=s} aq[s][j] V_j   (V_0 = v_n; a diagonal entry uses
//                                             the stage's own new velocity),
//   K_s = F(Q_s, V_s, u),
// and the last stage is the step's result (its K is the next step's K_0,
// first-same-as-last).  Adaptive schemes carry the weights e = b - bhat of the
// embedded error estimate.
enum { METHOD_DOPRI5 = 0, METHOD_TSIT5 = 1, METHOD_EULER = 2 };
struct Tableau {
  int S = 7;                      // stage evaluations per step, stage 0 included
  bool adaptive = true;
  double aq[7][7] = {}, av[7][7] = {};
  double b[7] = {}, bhat[7] = {}, c[7] = {};
};

// Dormand & Prince (1980) 5(4); row 7 equals the 5th-order weights (FSAL),
// bhat are the embedded 4th-order weights.
inline const Tableau& dopri5() {
  static const Tableau T = [] {
    Tableau t{};
    double (&a)[7][7] = t.av;
    a[1][0] = 1.0 / 5.0;
    a[2][0] = 3.0 / 40.0; a[2][1] = 9.0 / 40.0;
    a[3][0] = 44.0 / 45.0; a[3][1] = -56.0 / 15.0; a[3][2] = 32.0 / 9.0;
    a[4][0] = 19372.0 / 6561.0; a[4][1] = -25360.0 / 2187.0; a[4][2] = 64448.0 / 6561.0; a[4][3] = -212.0 / 729.0;
    a[5][0] = 9017.0 / 3168.0; a[5][1] = -355.0 / 33.0; a[5][2] = 46732.0 / 5247.0; a[5][3] = 49.0 / 176.0;
    a[5][4] = -5103.0 / 18656.0;
    a[6][0] = 35.0 / 384.0; a[6][1] = 0.0; a[6][2] = 500.0 / 1113.0; a[6][3] = 125.0 / 192.0;
    a[6][4] = -2187.0 / 6784.0; a[6][5] = 11.0 / 84.0;
    for (int i = 0; i < 7; ++i)
      for (int j = 0; j < 7; ++j) t.aq[i][j] = a[i][j];
    for (int j = 0; j < 7; ++j) t.b[j] = (j < 6) ? a[6][j] : 0.0;
    const double bh[7] = {5179.0 / 57600.0, 0.0, 7571.0 / 16695.0, 393.0 / 640.0, -92097.0 / 339200.0, 187.0 / 2100.0, 1.0 / 40.0};
    const double c[7] = {0.0, 1.0 / 5.0, 3.0 / 10.0, 4.0 / 5.0, 8.0 / 9.0, 1.0, 1.0};
    for (int j = 0; j < 7; ++j) { t.bhat[j] = bh[j]; t.c[j] = c[j]; }
    return t;
  }();
  return T;
}

// Tsitouras (2011) 5(4), the paper's default solver (Fig. 12): FSAL, row 7 =
// the 5th-order weights; e = b - bhat given directly (the pair's published
// error weights), bhat = b - e.
inline const Tableau& tsit5() {
  static const Tableau T = [] {
    Tableau t{};
    double (&a)[7][7] = t.av;
    a[1][0] = 0.161;
    a[2][0] = -0.008480655492356989; a[2][1] = 0.335480655492357;
    a[3][0] = 2.897153057105493; a[3][1] = -6.359448489975075; a[3][2] = 4.3622954328695815;
    a[4][0] = 5.325864828439257; a[4][1] = -11.748883564062828; a[4][2] = 7.4955393428898365;
    a[4][3] = -0.09249506636175525;
    a[5][0] = 5.86145544294642; a[5][1] = -12.92096931784711; a[5][2] = 8.159367898576159;
    a[5][3] = -0.071584973281401; a[5][4] = -0.028269050394068383;
    a[6][0] = 0.09646076681806523; a[6][1] = 0.01; a[6][2] = 0.4798896504144996; a[6][3] = 1.379008574103742;
    a[6][4] = -3.290069515436081; a[6][5] = 2.324710524099774;
    for (int i = 0; i < 7; ++i)
      for (int j = 0; j < 7; ++j) t.aq[i][j] = a[i][j];
    const double e[7] = {-0.00178001105222577714, -0.0008164344596567469, 0.007880878010261995, -0.1447110071732629,
                         0.5823571654525552, -0.45808210592918697, 0.015151515151515152};
    const double c[7] = {0.0, 0.161, 0.327, 0.9, 0.9800255409045097, 1.0, 1.0};
    for (int j = 0; j < 7; ++j) {
      t.b[j] = (j < 6) ? a[6][j] : 0.0;
      t.bhat[j] = t.b[j] - e[j];
      t.c[j] = c[j];
    }
    return t;
  }();
  return T;
}

// Semi-implicit (symplectic) Euler with a fixed step, the default integrator
// of MuJoCo XLA that the paper compares against (Sec. 3.1, Fig. 12):
// v_{n+1} = v_n + h F(q_n, v_n), q_{n+1} = q_n (+) h v_{n+1}.  One right-hand
// side per step; no error estimate.
inline const Tableau& euler_si() {
  static const Tableau T = [] {
    Tableau t{};
    t.S = 2;
    t.adaptive = false;
    t.av[1][0] = 1.0;
    t.aq[1][1] = 1.0;
    t.b[0] = 1.0; t.bhat[0] = 1.0; t.c[1] = 1.0;
    return t;
  }();
  return T;
}

inline const Tableau& tableau_of(int method) {
  return method == METHOD_TSIT5 ? tsit5() : method == METHOD_EULER ? euler_si() : dopri5();
}

// q (+) delta: positions advanced by a tangent increment.  Free joint:
// translation += delta[0:3] (world), quaternion <- normalize(quat * exp(delta[3:6] / 2))
// with the rotation increment in body coordinates.  Hinge: angle += delta.
template <class S> void integrate_pos(const Model& m, const S* q, const S* dlt, S* out) {
  for (const Body& B : m.body) {
    const S* x = q + B.qadr;
    const S* d = dlt + B.vadr;
    S* o = out + B.qadr;
    if (B.jtype == JNT_HINGE) { o[0] = x[0] + d[0]; continue; }
    for (int i = 0; i < 3; ++i) o[i] = x[i] + d[i];
    S th2 = d[3] * d[3] + d[4] * d[4] + d[5] * d[5];
    S cw, sk;   // cos(|th|/2), sin(|th|/2)/|th|
    if (val(th2) < 1e-12) {
      cw = 1.0 - th2 / 8.0 + th2 * th2 / 384.0;
      sk = 0.5 - th2 / 48.0 + th2 * th2 / 3840.0;
    } else {
      S th = sqrt(th2);
      cw = cos(0.5 * th);
      sk = sin(0.5 * th) / th;
    }
    S ew = cw, ex = sk * d[3], ey = sk * d[4], ez = sk * d[5];
    S w = x[3], a = x[4], b = x[5], c = x[6];
    S rw = w * ew - a * ex - b * ey - c * ez;
    S rx = w * ex + a * ew + b * ez - c * ey;
    S ry = w * ey - a * ez + b * ew + c * ex;
    S rz = w * ez + a * ey - b * ex + c * ew;
    S n = sqrt(rw * rw + rx * rx + ry * ry + rz * rz);
    o[3] = rw / n; o[4] = rx / n; o[5] = ry / n; o[6] = rz / n;
  }
}

// Magnitude of the coordinate belonging to tangent component i of the
// position part (free-joint rotation components have magnitude 1).
template <class S> S pos_magnitude(const Model& m, const S* q, int i) {
  const Body& B = m.body[m.dof_body[i]];
  if (B.jtype == JNT_HINGE) return fabs(q[B.qadr]);
  const int d = i - B.vadr;
  return d < 3 ? fabs(q[B.qadr + d]) : S(1.0);
}

// RMS error norm of the embedded difference e (2 nv tangent components).
template <class S>
S error_norm(const Model& m, const S* q0, const S* v0, const S* q1, const S* v1, const S* e, double rtol, double atol) {
  const int nv = m.nv;
  S acc = S(0.0);
  for (int i = 0; i < nv; ++i) {
    S sc = atol + rtol * smax(pos_magnitude(m, q0, i), pos_magnitude(m, q1, i));
    S r = e[i] / sc;
    acc = acc + r * r;
  }
  for (int i = 0; i < nv; ++i) {
    S sc = atol + rtol * smax(fabs(v0[i]), fabs(v1[i]));
    S r = e[nv + i] / sc;
    acc = acc + r * r;
  }
  return sqrt(acc / (2.0 * nv));
}

// Stage right-hand side.  Values always from F; with cfd and a derivative
// type, the tangent is taken from F~ at the same state (straight-through).
template <class S> struct StageRhs {
  const Model& m;
  bool cfd;
  bool noconv = false;
  bool operator()(const S* q, const S* v, const S* u, S* a) {
    bool ok = rhs<S>(m, q, v, u, false, a);
    if (!ok) noconv = true;
    return ok;
  }
};
template <> struct StageRhs<Dual<double>> {
  using D = Dual<double>;
  const Model& m;
  bool cfd;
  bool noconv = false;
  bool operator()(const D* q, const D* v, const D* u, D* a) {
    bool ok = rhs<D>(m, q, v, u, false, a);
    if (cfd) {
      std::vector<D> at(m.nv);
      rhs<D>(m, q, v, u, true, at.data());
      for (int i = 0; i < m.nv; ++i) a[i].d = at[i].d;   // ST: value of F, tangent of F~
    }
    if (!ok) noconv = true;
    return ok;
  }
};

// One attempt of size h of the scheme tb from (q, v) with stage-0 derivative
// a1.  Writes the result (q7, v7), its derivative a7 (FSAL) and, for adaptive
// schemes, the embedded difference e (2 nv tangent components; zero for a
// fixed-step scheme).
template <class S, class R>
void rk_step(const Model& m, const Tableau& tb, R& f, const S* q, const S* v, const S* a1, const S* u, double h,
             S* q7, S* v7, S* a7, S* e) {
  const int nv = m.nv, nq = m.nq, ns = tb.S;
  std::vector<std::vector<S>> ks_v(ns, std::vector<S>(nv)), ks_a(ns, std::vector<S>(nv));
  for (int i = 0; i < nv; ++i) { ks_v[0][i] = v[i]; ks_a[0][i] = a1[i]; }
  std::vector<S> dq(nv), qs(nq), vs(nv);
  for (int s = 1; s < ns; ++s) {
    for (int i = 0; i < nv; ++i) {
      S sv = S(0.0);
      for (int j = 0; j < s; ++j) {
        if (tb.av[s][j] == 0.0) continue;
        sv = sv + tb.av[s][j] * ks_a[j][i];
      }
      vs[i] = v[i] + h * sv;
      ks_v[s][i] = vs[i];
    }
    for (int i = 0; i < nv; ++i) {
      S sq = S(0.0);
      for (int j = 0; j <= s; ++j) {
        if (tb.aq[s][j] == 0.0) continue;
        sq = sq + tb.aq[s][j] * ks_v[j][i];
      }
      dq[i] = h * sq;
    }
    integrate_pos(m, q, dq.data(), qs.data());
    f(qs.data(), vs.data(), u, ks_a[s].data());
    if (s == ns - 1) {
      for (int i = 0; i < nq; ++i) q7[i] = qs[i];
      for (int i = 0; i < nv; ++i) { v7[i] = vs[i]; a7[i] = ks_a[s][i]; }
    }
  }
  for (int i = 0; i < nv; ++i) {
    S ep = S(0.0), ev = S(0.0);
    for (int j = 0; j < ns && tb.adaptive; ++j) {
      double w = tb.b[j] - tb.bhat[j];
      if (w == 0.0) continue;
      ep = ep + w * ks_v[j][i];
      ev = ev + w * ks_a[j][i];
    }
    e[i] = h * ep;
    e[nv + i] = h * ev;
  }
}

// The Dormand-Prince attempt (the default scheme).
template <class S, class R>
void dopri5_step(const Model& m, R& f, const S* q, const S* v, const S* a1, const S* u, double h,
                 S* q7, S* v7, S* a7, S* e) {
  rk_step(m, dopri5(), f, q, v, a1, u, h, q7, v7, a7, e);
}

struct Opts {
  double T = 1.0;
  int NI = 1;
  double rtol = 1e-6, atol = 1e-8, h0 = 1e-3;
  int max_steps = 100000;
  int method = METHOD_DOPRI5;   // fixed-step schemes take h0 for every step
};
struct Result {
  int status = ENV_OK, nsteps = 0, nrej = 0, nrhs = 0;
};
struct StepRec {
  std::vector<double> q, v;
  double h;
  int k;          // control interval of the step
  bool reached;   // the step ends on the boundary of interval k
};

inline double boundary_time(double T, int NI, int k) { return k >= NI ? T : T * k / NI; }

// Adaptive rollout (replay == nullptr) or replay of given accepted step sizes.
// x0 = [q; v], ctrl = [NI][nu].  xb (optional) receives the states at the NI+1
// interval boundaries; rec (optional) the accepted steps.
template <class S>
Result rollout(const Model& m, const S* x0, const S* ctrl, const Opts& o, S* xT, S* xb,
               std::vector<StepRec>* rec, std::vector<double>* hlog, const double* replay, int nreplay) {
  const int nq = m.nq, nv = m.nv, nx = nq + nv, nu = m.nu;
  Result res;
  std::vector<S> q(x0, x0 + nq), v(x0 + nq, x0 + nx), a1(nv), q7(nq), v7(nv), a7(nv), e(2 * nv);
  for (int i = 0; i < nx; ++i) xT[i] = x0[i];
  bool finite = true;
  for (int i = 0; i < nx; ++i) finite = finite && std::isfinite(val(x0[i]));
  if (xb) for (int i = 0; i < nx; ++i) xb[i] = x0[i];
  if (!finite) { res.status = ENV_NONFINITE; return res; }
  StageRhs<S> f{m, false};
  const Tableau& tb = tableau_of(o.method);
  auto uk = [&](int k) { return nu ? ctrl + (size_t)k * nu : ctrl; };
  int k = 0;
  double t = 0.0;
  f(q.data(), v.data(), uk(0), a1.data());
  res.nrhs = 1;
  double h = o.h0;
  double err_prev = 1.0;
  int attempts = 0, ir = 0;
  while (t < o.T) {
    if (replay) { if (ir >= nreplay) break; h = replay[ir]; }
    else if (attempts >= o.max_steps) { res.status = ENV_MAX_STEPS; break; }
    const double tn = boundary_time(o.T, o.NI, k + 1);
    const double hb = tn - t;
    const bool clamped = replay ? (h == hb) : (h >= hb || hb - h < 1e-12);
    const double ht = clamped ? hb : h;
    if (!replay && ht < 1e-12) { res.status = ENV_H_UNDERFLOW; break; }
    f.noconv = false;
    rk_step(m, tb, f, q.data(), v.data(), a1.data(), uk(k), ht, q7.data(), v7.data(), a7.data(), e.data());
    res.nrhs += tb.S - 1;
    ++attempts;
    double err = (replay || !tb.adaptive)
                     ? 0.0
                     : val(error_norm<S>(m, q.data(), v.data(), q7.data(), v7.data(), e.data(), o.rtol, o.atol));
    if (err <= 1.0) {
      if (f.noconv) { res.status = ENV_SOLVER_NOCONV; break; }
      if (rec) {
        StepRec r;
        r.q.resize(nq); r.v.resize(nv);
        for (int i = 0; i < nq; ++i) r.q[i] = val(q[i]);
        for (int i = 0; i < nv; ++i) r.v[i] = val(v[i]);
        r.h = ht; r.k = k; r.reached = false;
        rec->push_back(r);
      }
      if (hlog) hlog->push_back(ht);
      const bool reached = clamped || (t + ht >= tn);
      t = reached ? tn : t + ht;
      q = q7; v = v7; a1 = a7;
      ++res.nsteps;
      ++ir;
      if (tb.adaptive) {
        const double errf = std::max(err, 1e-10);
        double fac = 0.9 * std::pow(errf, -0.6 / 5.0) * std::pow(err_prev, 0.2 / 5.0);
        fac = std::min(10.0, std::max(0.2, fac));
        err_prev = errf;
        h = ht * fac;
      } else {
        h = o.h0;    // fixed step (the last step of an interval may have been shortened)
      }
      if (reached) {
        if (rec) rec->back().reached = true;
        ++k;
        if (xb) {
          for (int i = 0; i < nq; ++i) xb[(size_t)k * nx + i] = q[i];
          for (int i = 0; i < nv; ++i) xb[(size_t)k * nx + nq + i] = v[i];
        }
        if (k < o.NI) { f(q.data(), v.data(), uk(k), a1.data()); res.nrhs += 1; }
      }
    } else {
      ++res.nrej;
      const double fac = std::isfinite(err) ? std::max(0.2, 0.9 * std::pow(err, -1.0 / 5.0)) : 0.2;
      h = ht * fac;
    }
  }
  for (int i = 0; i < nq; ++i) xT[i] = q[i];
  for (int i = 0; i < nv; ++i) xT[nq + i] = v[i];
  return res;
}

// Jacobian of one accepted DOPRI5 step (h fixed) of the map
// (q, v, u) -> (q7, v7), by forward-mode derivatives, one input direction at a
// time.  Jx is nx x nx, Ju is nx x nu (row major).  With cfd the derivatives
// of every stage come from F~ (straight-through).
inline void step_jacobian(const Model& m, const double* q, const double* v, const double* u, double h, bool cfd,
                          std::vector<double>& Jx, std::vector<double>& Ju, int method = METHOD_DOPRI5) {
  using D = Dual<double>;
  const int nq = m.nq, nv = m.nv, nx = nq + nv, nu = m.nu;
  Jx.assign((size_t)nx * nx, 0.0);
  Ju.assign((size_t)nx * std::max(nu, 1), 0.0);
  std::vector<D> qd(nq), vd(nv), ud(std::max(nu, 1)), a1(nv), q7(nq), v7(nv), a7(nv), e(2 * nv);
  for (int dir = 0; dir < nx + nu; ++dir) {
    for (int i = 0; i < nq; ++i) qd[i] = D(q[i], dir == i ? 1.0 : 0.0);
    for (int i = 0; i < nv; ++i) vd[i] = D(v[i], dir == nq + i ? 1.0 : 0.0);
    for (int i = 0; i < nu; ++i) ud[i] = D(u[i], dir == nx + i ? 1.0 : 0.0);
    StageRhs<D> f{m, cfd};
    f(qd.data(), vd.data(), ud.data(), a1.data());
    rk_step(m, tableau_of(method), f, qd.data(), vd.data(), a1.data(), ud.data(), h, q7.data(), v7.data(), a7.data(),
            e.data());
    for (int i = 0; i < nq; ++i) {
      if (dir < nx) Jx[(size_t)i * nx + dir] = q7[i].d; else Ju[(size_t)i * nu + (dir - nx)] = q7[i].d;
    }
    for (int i = 0; i < nv; ++i) {
      if (dir < nx) Jx[(size_t)(nq + i) * nx + dir] = v7[i].d; else Ju[(size_t)(nq + i) * nu + (dir - nx)] = v7[i].d;
    }
  }
}

// Jacobian (nx x np, row major) of one accepted step (h fixed) with respect to
// the model parameters (par<S>, dynamics.h), one parameter direction at a
// time; with cfd the derivatives of every stage come from F~.
inline void step_jacobian_params(const Model& m, const double* q, const double* v, const double* u, double h,
                                 bool cfd, std::vector<double>& Jp, int method = METHOD_DOPRI5) {
  using D = Dual<double>;
  const int nq = m.nq, nv = m.nv, nu = m.nu, np = n_params(m);
  Jp.assign((size_t)(nq + nv) * np, 0.0);
  std::vector<D> qd(nq), vd(nv), ud(std::max(nu, 1)), a1(nv), q7(nq), v7(nv), a7(nv), e(2 * nv);
  for (int i = 0; i < nq; ++i) qd[i] = D(q[i], 0.0);
  for (int i = 0; i < nv; ++i) vd[i] = D(v[i], 0.0);
  for (int i = 0; i < nu; ++i) ud[i] = D(u[i], 0.0);
  for (int k = 0; k < np; ++k) {
    g_pdir = k;
    StageRhs<D> f{m, cfd};
    f(qd.data(), vd.data(), ud.data(), a1.data());
    rk_step(m, tableau_of(method), f, qd.data(), vd.data(), a1.data(), ud.data(), h, q7.data(), v7.data(), a7.data(),
            e.data());
    for (int i = 0; i < nq; ++i) Jp[(size_t)i * np + k] = q7[i].d;
    for (int i = 0; i < nv; ++i) Jp[(size_t)(nq + i) * np + k] = v7[i].d;
  }
  g_pdir = -1;
}

// Discrete adjoint (discretize-then-optimize) over the accepted steps of the
// adaptive rollout: x0_bar = d/dx0 <xT_bar, xT> + sum_k <xb_bar[k], x(t_k)>,
// ctrl_bar likewise for the piecewise-constant controls.
// With replay != nullptr the forward pass takes the given accepted step sizes
// instead of choosing them (the gradient of that frozen step sequence).
// With p_bar (n_params(m) entries) also the model-parameter gradient
// p_bar = sum over the accepted steps of (d step / d p)^T lambda_{n+1}.
inline Result rollout_grad(const Model& m, const double* x0, const double* ctrl, const Opts& o, bool cfd,
                           const double* xT_bar, const double* xb_bar, double* xT, double* x0_bar, double* ctrl_bar,
                           const double* replay = nullptr, int nreplay = 0, double* p_bar = nullptr) {
  const int nq = m.nq, nv = m.nv, nx = nq + nv, nu = m.nu;
  std::vector<StepRec> rec;
  Result res = rollout<double>(m, x0, ctrl, o, xT, nullptr, &rec, nullptr, replay, nreplay);
  std::vector<double> lam(xT_bar, xT_bar + nx), Jx, Ju, Jp, nl(nx);
  const int np = n_params(m);
  if (ctrl_bar) for (int i = 0; i < o.NI * nu; ++i) ctrl_bar[i] = 0.0;
  if (p_bar) for (int k = 0; k < np; ++k) p_bar[k] = 0.0;
  for (int n = (int)rec.size() - 1; n >= 0; --n) {
    const StepRec& r = rec[n];
    if (r.reached && xb_bar)
      for (int i = 0; i < nx; ++i) lam[i] += xb_bar[(size_t)(r.k + 1) * nx + i];
    const double* u = nu ? ctrl + (size_t)r.k * nu : ctrl;
    step_jacobian(m, r.q.data(), r.v.data(), u, r.h, cfd, Jx, Ju, o.method);
    if (p_bar) {
      step_jacobian_params(m, r.q.data(), r.v.data(), u, r.h, cfd, Jp, o.method);
      for (int k = 0; k < np; ++k) {
        double acc = 0;
        for (int i = 0; i < nx; ++i) acc += Jp[(size_t)i * np + k] * lam[i];
        p_bar[k] += acc;
      }
    }
    if (ctrl_bar)
      for (int j = 0; j < nu; ++j) {
        double s = 0;
        for (int i = 0; i < nx; ++i) s += Ju[(size_t)i * nu + j] * lam[i];
        ctrl_bar[(size_t)r.k * nu + j] += s;
      }
    for (int j = 0; j < nx; ++j) {
      double s = 0;
      for (int i = 0; i < nx; ++i) s += Jx[(size_t)i * nx + j] * lam[i];
      nl[j] = s;
    }
    lam = nl;
  }
  if (xb_bar) for (int i = 0; i < nx; ++i) lam[i] += xb_bar[i];
  for (int i = 0; i < nx; ++i) x0_bar[i] = lam[i];
  return res;
}

// ------------------------------------------------------------------ optimize-then-discretize
// Continuous adjoint (App. C.2 "Optimize-then-discretize", Eq. adjoint-
// equations; the straight-through variant of App. C.4): with x = (q, v),
// x' = f(x, u) = (G(q) v, F(q, v, u)) and a_x(T) = dL/dx(T),
//   a_x' = -a_x^T df/dx,   a_u' = -a_x^T df/du  (per control interval),
// integrated BACKWARD from T together with the state itself (backsolve: the
// state runs backward from x(T), constant memory).  With cfd the VJPs use F~
// (the state still follows F).  The backward solve takes its own adaptive
// steps (the scheme and PID controller of the forward pass) with the error
// norm over the state's 2 nv tangent components and every adjoint component.
// G(q): identity for translations and hinges, q' = q (x) (0, w) / 2 for the
// quaternion of a free joint (w: body angular velocity).  Interval-boundary
// cotangents xb_bar[k] enter as jumps of a_x at t_k; a_u is collected per
// interval.  In reversed time s = T - t: dx/ds = -f, da/ds = +(df/dx)^T a.

// Kinematic part of the adjoint right-hand side at (q, v): kq += (d(G v)/dq)^T aq,
// kv += G^T aq.
inline void kin_adjoint(const Model& m, const double* q, const double* v, const double* aq, double* kq, double* kv) {
  for (const Body& B : m.body) {
    const int qa = B.qadr, va = B.vadr;
    if (B.jtype == JNT_HINGE) { kv[va] += aq[qa]; continue; }
    for (int i = 0; i < 3; ++i) kv[va + i] += aq[qa + i];
    const double w = q[qa + 3], x = q[qa + 4], y = q[qa + 5], z = q[qa + 6];
    const double a = v[va + 3], b = v[va + 4], c = v[va + 5];
    const double Aw = aq[qa + 3], Ax = aq[qa + 4], Ay = aq[qa + 5], Az = aq[qa + 6];
    // q (x) (0, a, b, c) = (-x a - y b - z c, w a + y c - z b, w b - x c + z a, w c + x b - y a)
    kq[qa + 3] += 0.5 * (a * Ax + b * Ay + c * Az);
    kq[qa + 4] += 0.5 * (-a * Aw - c * Ay + b * Az);
    kq[qa + 5] += 0.5 * (-b * Aw + c * Ax - a * Az);
    kq[qa + 6] += 0.5 * (-c * Aw - b * Ax + a * Ay);
    kv[va + 3] += 0.5 * (-x * Aw + w * Ax + z * Ay - y * Az);
    kv[va + 4] += 0.5 * (-y * Aw - z * Ax + w * Ay + x * Az);
    kv[va + 5] += 0.5 * (-z * Aw + y * Ax - x * Ay + w * Az);
  }
}

// Adjoint right-hand side in reversed time at the stage state (q, v):
// (kq, kv, ku) = (df/dx)^T (aq, av) and (dF/du)^T av, with F (or F~).
inline void adjoint_rhs(const Model& m, const double* q, const double* v, const double* u, bool cfd,
                        const double* aq, const double* av, double* kq, double* kv, double* ku) {
  using D = Dual<double>;
  const int nq = m.nq, nv = m.nv, nu = m.nu;
  std::vector<D> qd(nq), vd(nv), ud(std::max(nu, 1)), acc(nv);
  for (int i = 0; i < nq; ++i) kq[i] = 0.0;
  for (int i = 0; i < nv; ++i) kv[i] = 0.0;
  for (int i = 0; i < nu; ++i) ku[i] = 0.0;
  for (int dir = 0; dir < nq + nv + nu; ++dir) {     // columns of dF/d(q, v, u), one derivative direction each
    for (int i = 0; i < nq; ++i) qd[i] = D(q[i], dir == i ? 1.0 : 0.0);
    for (int i = 0; i < nv; ++i) vd[i] = D(v[i], dir == nq + i ? 1.0 : 0.0);
    for (int i = 0; i < nu; ++i) ud[i] = D(u[i], dir == nq + nv + i ? 1.0 : 0.0);
    rhs<D>(m, qd.data(), vd.data(), ud.data(), cfd, acc.data());
    double s = 0.0;
    for (int i = 0; i < nv; ++i) s += acc[i].d * av[i];
    if (dir < nq) kq[dir] += s; else if (dir < nq + nv) kv[dir - nq] += s; else ku[dir - nq - nv] += s;
  }
  kin_adjoint(m, q, v, aq, kq, kv);
}

inline Result rollout_grad_otd(const Model& m, const double* x0, const double* ctrl, const Opts& o, bool cfd,
                               const double* xT_bar, const double* xb_bar, double* xT, double* x0_bar,
                               double* ctrl_bar, Result* back = nullptr) {
  const int nq = m.nq, nv = m.nv, nx = nq + nv, nu = m.nu;
  Result res = rollout<double>(m, x0, ctrl, o, xT, nullptr, nullptr, nullptr, nullptr, 0);
  const Tableau& tb = tableau_of(o.method);
  const int ns = tb.S;
  const int na = nx + nu;                               // adjoint components (a_q, a_v, a_u)
  std::vector<double> q(xT, xT + nq), v(xT + nq, xT + nx), a(na, 0.0);
  for (int i = 0; i < nx; ++i) a[i] = xT_bar[i];
  if (xb_bar) for (int i = 0; i < nx; ++i) a[i] += xb_bar[(size_t)o.NI * nx + i];
  if (ctrl_bar) for (int i = 0; i < o.NI * nu; ++i) ctrl_bar[i] = 0.0;
  std::vector<std::vector<double>> kv_(ns, std::vector<double>(nv)), kf(ns, std::vector<double>(nv)),
      ka(ns, std::vector<double>(na));
  std::vector<double> dq(nv), qs(nq), vs(nv), as(na), q7(nq), v7(nv), a7(na), tmpq(nq), tmpv(nv), tmpu(std::max(nu, 1));
  Result bres;
  StageRhs<double> f{m, false};
  int k = o.NI - 1;
  double t = o.T, h = o.h0, err_prev = 1.0;
  auto uk = [&](int kk) { return nu ? ctrl + (size_t)kk * nu : ctrl; };
  int attempts = 0;
  while (t > 0.0 && k >= 0) {
    if (attempts >= o.max_steps) { bres.status = ENV_MAX_STEPS; break; }
    const double tlo = boundary_time(o.T, o.NI, k);
    const double hb = t - tlo;
    const bool clamped = h >= hb || hb - h < 1e-12;
    const double ht = clamped ? hb : h;
    if (ht < 1e-12) { bres.status = ENV_H_UNDERFLOW; break; }
    const double* u = uk(k);
    // stage 0
    for (int i = 0; i < nv; ++i) kv_[0][i] = v[i];
    f(q.data(), v.data(), u, kf[0].data());
    adjoint_rhs(m, q.data(), v.data(), u, cfd, a.data(), a.data() + nq, ka[0].data(), ka[0].data() + nq,
                ka[0].data() + nx);
    for (int s = 1; s < ns; ++s) {
      for (int i = 0; i < nv; ++i) {
        double sv = 0.0;
        for (int j = 0; j < s; ++j) if (tb.av[s][j] != 0.0) sv += tb.av[s][j] * kf[j][i];
        vs[i] = v[i] - ht * sv;
        kv_[s][i] = vs[i];
      }
      for (int i = 0; i < nv; ++i) {
        double sq = 0.0;
        for (int j = 0; j <= s; ++j) if (tb.aq[s][j] != 0.0) sq += tb.aq[s][j] * kv_[j][i];
        dq[i] = -ht * sq;
      }
      integrate_pos(m, q.data(), dq.data(), qs.data());
      for (int i = 0; i < na; ++i) {
        double sa = 0.0;
        for (int j = 0; j < s; ++j) if (tb.av[s][j] != 0.0) sa += tb.av[s][j] * ka[j][i];
        as[i] = a[i] + ht * sa;
      }
      f(qs.data(), vs.data(), u, kf[s].data());
      adjoint_rhs(m, qs.data(), vs.data(), u, cfd, as.data(), as.data() + nq, ka[s].data(), ka[s].data() + nq,
                  ka[s].data() + nx);
      if (s == ns - 1) { q7 = qs; v7 = vs; a7 = as; }
    }
    ++attempts;
    double err = 0.0;
    if (tb.adaptive) {
      double acc = 0.0;
      for (int i = 0; i < nv; ++i) {
        double ep = 0.0, ev = 0.0;
        for (int j = 0; j < ns; ++j) {
          const double w = tb.b[j] - tb.bhat[j];
          ep += w * kv_[j][i];
          ev += w * kf[j][i];
        }
        ep *= ht; ev *= ht;
        const double sp = o.atol + o.rtol * std::max(val(pos_magnitude(m, q.data(), i)), val(pos_magnitude(m, q7.data(), i)));
        const double sv = o.atol + o.rtol * std::max(std::fabs(v[i]), std::fabs(v7[i]));
        acc += (ep / sp) * (ep / sp) + (ev / sv) * (ev / sv);
      }
      for (int i = 0; i < na; ++i) {
        double ea = 0.0;
        for (int j = 0; j < ns; ++j) ea += (tb.b[j] - tb.bhat[j]) * ka[j][i];
        ea *= ht;
        const double sa = o.atol + o.rtol * std::max(std::fabs(a[i]), std::fabs(a7[i]));
        acc += (ea / sa) * (ea / sa);
      }
      err = std::sqrt(acc / (2.0 * nv + na));
    }
    if (err <= 1.0) {
      q = q7; v = v7; a = a7;
      ++bres.nsteps;
      t = clamped ? tlo : t - ht;
      if (tb.adaptive) {
        const double errf = std::max(err, 1e-10);
        double fac = 0.9 * std::pow(errf, -0.6 / 5.0) * std::pow(err_prev, 0.2 / 5.0);
        fac = std::min(10.0, std::max(0.2, fac));
        err_prev = errf;
        h = ht * fac;
      } else {
        h = o.h0;
      }
      if (clamped) {                                  // reached the interval's lower boundary t_k
        if (ctrl_bar) for (int j = 0; j < nu; ++j) ctrl_bar[(size_t)k * nu + j] += a[nx + j];
        for (int j = 0; j < nu; ++j) a[nx + j] = 0.0;
        if (xb_bar) for (int i = 0; i < nx; ++i) a[i] += xb_bar[(size_t)k * nx + i];
        --k;
      }
    } else {
      ++bres.nrej;
      const double fac = std::isfinite(err) ? std::max(0.2, 0.9 * std::pow(err, -1.0 / 5.0)) : 0.2;
      h = ht * fac;
    }
  }
  for (int i = 0; i < nx; ++i) x0_bar[i] = a[i];
  if (back) *back = bres;
  return res;
}

}  // namespace orc
