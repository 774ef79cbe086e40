// Oracle forward dynamics v' = F(q, v, u) of the soft-contact rigid-body model.
//
// TEST INFRASTRUCTURE ONLY (see scalar.h).
//
// Paper passages followed (arXiv 2506.14186):
//   Sec. 2, Eq. (EOM)          v' = M^-1 (tau - c + J^T f)
//   Sec. 2 (Featherstone)      M by the composite-rigid-body algorithm, c by
//                              recursive Newton-Euler, both in world-frame
//                              spatial (Plucker) coordinates
//   Sec. 2.1 collision         signed distance r, contact active iff r < 0
//   Sec. 2.1 Eq. (primal)      relaxed Gauss principle with pyramidal cones
//   Sec. 2.1 a_ref             a_ref = -b (J v) - k d(r) r, b = 2/(d_w t_c),
//                              k = 1/(d_w^2 t_c^2 phi_d^2)
//   Sec. 2.1 impedance / R     d(r) solimp spline, R = A_hat (1-d)/d
//   Sec. 2.1 solver            exact Newton method on the convex primal
//   App. C.1 plane-box         box vertices against the plane, pos = v - r/2 n
//   Sec. 4 CFD                 d(r) continued for r > 0 by the solimp-CFD
//                              spline; ReLU of a_ref replaced by a softplus
//   Sec. 5.1, App. E.2         contact parameters (solref, solimp, friction)
//                              and body masses
//                              as differentiable model parameters
// Readings where the paper is silent are listed in the design notes of the
// repository (integrator, spline form, A_hat, solver stop rule, capsule-box).
#pragma once
#include <algorithm>
#include <array>
#include <type_traits>
#include <vector>

#include "model.h"
#include "scalar.h"

namespace orc {

template <class S> using V3 = std::array<S, 3>;
template <class S> using M3 = std::array<S, 9>;   // row major

template <class S> inline V3<S> vadd(const V3<S>& a, const V3<S>& b) { return {a[0] + b[0], a[1] + b[1], a[2] + b[2]}; }
template <class S> inline V3<S> vsub(const V3<S>& a, const V3<S>& b) { return {a[0] - b[0], a[1] - b[1], a[2] - b[2]}; }
template <class S> inline V3<S> vscl(const V3<S>& a, const S& s) { return {a[0] * s, a[1] * s, a[2] * s}; }
template <class S> inline S vdot(const V3<S>& a, const V3<S>& b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class S> inline V3<S> vcross(const V3<S>& a, const V3<S>& b) {
  return {a[1] * b[2] - a[2] * b[1], a[2] * b[0] - a[0] * b[2], a[0] * b[1] - a[1] * b[0]};
}
template <class S> inline V3<S> mvec(const M3<S>& R, const V3<S>& x) {
  return {R[0] * x[0] + R[1] * x[1] + R[2] * x[2], R[3] * x[0] + R[4] * x[1] + R[5] * x[2],
          R[6] * x[0] + R[7] * x[1] + R[8] * x[2]};
}
template <class S> inline V3<S> mtvec(const M3<S>& R, const V3<S>& x) {
  return {R[0] * x[0] + R[3] * x[1] + R[6] * x[2], R[1] * x[0] + R[4] * x[1] + R[7] * x[2],
          R[2] * x[0] + R[5] * x[1] + R[8] * x[2]};
}
template <class S> inline M3<S> mmul(const M3<S>& A, const M3<S>& B) {
  M3<S> C;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) C[3 * i + j] = A[3 * i] * B[j] + A[3 * i + 1] * B[3 + j] + A[3 * i + 2] * B[6 + j];
  return C;
}
template <class S> inline V3<S> cvec(const double* x) { return {S(x[0]), S(x[1]), S(x[2])}; }

// Rotation matrix of a quaternion (w, x, y, z), normalised first.
template <class S> M3<S> quat2mat(const S& w0, const S& x0, const S& y0, const S& z0) {
  S n = sqrt(w0 * w0 + x0 * x0 + y0 * y0 + z0 * z0);
  S w = w0 / n, x = x0 / n, y = y0 / n, z = z0 / n;
  return {1.0 - 2.0 * (y * y + z * z), 2.0 * (x * y - w * z), 2.0 * (x * z + w * y),
          2.0 * (x * y + w * z), 1.0 - 2.0 * (x * x + z * z), 2.0 * (y * z - w * x),
          2.0 * (x * z - w * y), 2.0 * (y * z + w * x), 1.0 - 2.0 * (x * x + y * y)};
}
// Rotation by angle th about the unit axis a (Rodrigues' formula).
template <class S> M3<S> axis_angle(const double* a, const S& th) {
  S s = sin(th), c1 = 1.0 - cos(th);
  M3<S> K = {S(0.0), S(-a[2]), S(a[1]), S(a[2]), S(0.0), S(-a[0]), S(-a[1]), S(a[0]), S(0.0)};
  M3<S> K2 = mmul(K, K);
  M3<S> R;
  for (int i = 0; i < 9; ++i) R[i] = (i % 4 == 0 ? S(1.0) : S(0.0)) + s * K[i] + c1 * K2[i];
  return R;
}

// ------------------------------------------------------------------ kinematics
template <class S> struct Kin {
  std::vector<M3<S>> R;      // body orientation (world)
  std::vector<V3<S>> p;      // body origin (world)
  std::vector<V3<S>> c;      // body centre of mass (world)
  std::vector<M3<S>> Iw;     // inertia about the COM, world axes
  std::vector<std::array<S, 6>> s;   // dof motion vectors (omega; v at world origin)
  std::vector<M3<S>> gR;
  std::vector<V3<S>> gp;
};

// Model parameters that the adjoint differentiates (the parameters of the
// system identification of Sec. 5.1 and App. E.2): solref (t_c, phi_d),
// solimp (d_o, d_w, width, midpoint), the friction coefficient of every pair,
// the mass of every body (its rotational inertia scaled in proportion: equal
// density, fixed shape), then the side length of every box geom (its edge
// along the geom's x axis; the half sizes scale together, and the inertia of
// a body whose only geom is the box scales with the square, mass fixed).
// par<S>(k, v) is the value v of parameter k; in the derivative scalar it
// carries a unit tangent when k is the direction being differentiated
// (g_pdir), else none.
enum { PAR_TC = 0, PAR_DAMP = 1, PAR_DO = 2, PAR_DW = 3, PAR_WIDTH = 4, PAR_MID = 5, PAR_MU0 = 6 };
extern thread_local int g_pdir;
template <class S> inline S par(int, double v) { return S(v); }
template <> inline Dual<double> par<Dual<double>>(int k, double v) { return Dual<double>(v, g_pdir == k ? 1.0 : 0.0); }
inline int par_mass(const Model& m, int b) { return PAR_MU0 + (int)m.pair.size() + b; }
inline int par_side(const Model& m, int j) { return par_mass(m, (int)m.body.size()) + j; }
inline int n_params(const Model& m) { return par_side(m, (int)m.box_geom.size()); }
// Whether S carries the tangent of body b's mass in this evaluation.
template <class S> inline bool mass_direction(const Model&, int) { return false; }
template <> inline bool mass_direction<Dual<double>>(const Model& m, int b) { return g_pdir == par_mass(m, b); }
// Whether S carries the tangent of the side of the box body b consists of.
template <class S> inline bool side_direction(const Model&, int) { return false; }
template <> inline bool side_direction<Dual<double>>(const Model& m, int b) {
  return m.body[b].sole_box >= 0 && g_pdir == par_side(m, m.body[b].sole_box);
}
// Half size i of geom g; for a box in the derivative scalar with g_pdir on
// its side length l = 2 h_0, the tangent dh_i/dl = h_i / (2 h_0).
template <class S> inline S half_size(const Model& m, int g, int i) { return S(m.geom[g].size[i]); }
template <> inline Dual<double> half_size<Dual<double>>(const Model& m, int g, int i) {
  const Geom& G = m.geom[g];
  const bool dir = G.box >= 0 && g_pdir == par_side(m, G.box);
  return Dual<double>(G.size[i], dir ? G.size[i] / (2.0 * G.size[0]) : 0.0);
}

// A_hat of pair P (the sum of its bodies' inverse weights); the derivative
// scalar carries its derivative with respect to the body mass g_pdir points at.
template <class S> inline S pair_invw(const Model& m, const Pair& P) { return S(P.invw); }
template <> inline Dual<double> pair_invw<Dual<double>>(const Model& m, const Pair& P) {
  const int c = g_pdir - par_mass(m, 0);
  return Dual<double>(P.invw, (c >= 0 && c < (int)P.dinvw.size()) ? P.dinvw[c] : 0.0);
}

template <class S> void kinematics(const Model& m, const S* q, Kin<S>& k) {
  const int nb = (int)m.body.size();
  k.R.resize(nb); k.p.resize(nb); k.c.resize(nb); k.Iw.resize(nb);
  k.s.assign(m.nv, std::array<S, 6>{});
  for (int b = 0; b < nb; ++b) {
    const Body& B = m.body[b];
    M3<S> Rp = {S(1.0), S(0.0), S(0.0), S(0.0), S(1.0), S(0.0), S(0.0), S(0.0), S(1.0)};
    V3<S> pp = {S(0.0), S(0.0), S(0.0)};
    if (B.parent >= 0) { Rp = k.R[B.parent]; pp = k.p[B.parent]; }
    if (B.jtype == JNT_FREE) {
      const S* x = q + B.qadr;
      k.p[b] = {x[0], x[1], x[2]};
      k.R[b] = quat2mat(x[3], x[4], x[5], x[6]);
    } else {
      M3<S> Ro = quat2mat(S(B.quat[0]), S(B.quat[1]), S(B.quat[2]), S(B.quat[3]));
      k.p[b] = vadd(pp, mvec(Rp, cvec<S>(B.pos)));
      k.R[b] = mmul(mmul(Rp, Ro), axis_angle(B.axis, q[B.qadr]));
    }
    k.c[b] = vadd(k.p[b], mvec(k.R[b], cvec<S>(B.com)));
    M3<S> RI;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) RI[3 * i + j] = k.R[b][3 * i + j] * B.inertia[j];
    if (mass_direction<S>(m, b)) {                      // inertia proportional to the mass
      const S scale = par<S>(par_mass(m, b), B.mass) / B.mass;
      for (int i = 0; i < 9; ++i) RI[i] = RI[i] * scale;
    }
    if (side_direction<S>(m, b)) {                      // inertia proportional to the side squared
      const Geom& G = m.geom[m.box_geom[B.sole_box]];
      const double l0 = 2.0 * G.size[0];
      const S lam = par<S>(par_side(m, B.sole_box), l0) / l0;
      for (int i = 0; i < 9; ++i) RI[i] = RI[i] * (lam * lam);
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        k.Iw[b][3 * i + j] = RI[3 * i] * k.R[b][3 * j] + RI[3 * i + 1] * k.R[b][3 * j + 1] + RI[3 * i + 2] * k.R[b][3 * j + 2];
    // motion vectors of this body's dofs
    if (B.jtype == JNT_FREE) {
      for (int d = 0; d < 3; ++d) {
        std::array<S, 6>& st = k.s[B.vadr + d];
        for (int i = 0; i < 6; ++i) st[i] = S(0.0);
        st[3 + d] = S(1.0);
        V3<S> w = {k.R[b][d], k.R[b][3 + d], k.R[b][6 + d]};   // body axis d in world
        V3<S> vo = vcross(k.p[b], w);
        std::array<S, 6>& sr = k.s[B.vadr + 3 + d];
        sr = {w[0], w[1], w[2], vo[0], vo[1], vo[2]};
      }
    } else {
      V3<S> w = mvec(k.R[b], cvec<S>(B.axis));
      V3<S> vo = vcross(k.p[b], w);
      k.s[B.vadr] = {w[0], w[1], w[2], vo[0], vo[1], vo[2]};
    }
  }
  const int ng = (int)m.geom.size();
  k.gR.resize(ng); k.gp.resize(ng);
  for (int g = 0; g < ng; ++g) {
    const Geom& G = m.geom[g];
    M3<S> Ro = quat2mat(S(G.quat[0]), S(G.quat[1]), S(G.quat[2]), S(G.quat[3]));
    k.gR[g] = mmul(k.R[G.body], Ro);
    k.gp[g] = vadd(k.p[G.body], mvec(k.R[G.body], cvec<S>(G.pos)));
  }
}

// Spatial inertia (6x6, ordering omega; v, reference point = world origin).
template <class S, class Ms> std::array<S, 36> spatial_inertia_of(const Kin<S>& k, int b, const Ms& mass) {
  const V3<S>& c = k.c[b];
  M3<S> cx = {S(0.0), -c[2], c[1], c[2], S(0.0), -c[0], -c[1], c[0], S(0.0)};
  std::array<S, 36> I;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      // I_c + m cx cx^T
      S cc = cx[3 * i] * cx[3 * j] + cx[3 * i + 1] * cx[3 * j + 1] + cx[3 * i + 2] * cx[3 * j + 2];
      I[6 * i + j] = k.Iw[b][3 * i + j] + mass * cc;
      I[6 * i + 3 + j] = mass * cx[3 * i + j];
      I[6 * (3 + i) + j] = mass * cx[3 * j + i];
      I[6 * (3 + i) + 3 + j] = (i == j) ? S(mass) : S(0.0);
    }
  return I;
}
template <class S> std::array<S, 36> spatial_inertia(const Model& m, const Kin<S>& k, int b) {
  // the mass as a derivative scalar only when it is the direction differentiated
  if (mass_direction<S>(m, b)) return spatial_inertia_of(k, b, par<S>(par_mass(m, b), m.body[b].mass));
  return spatial_inertia_of(k, b, m.body[b].mass);
}
template <class S> std::array<S, 6> mat6vec(const std::array<S, 36>& A, const std::array<S, 6>& x) {
  std::array<S, 6> y;
  for (int i = 0; i < 6; ++i) {
    S a = S(0.0);
    for (int j = 0; j < 6; ++j) a = a + A[6 * i + j] * x[j];
    y[i] = a;
  }
  return y;
}
template <class S> S dot6(const std::array<S, 6>& a, const std::array<S, 6>& b) {
  S r = S(0.0);
  for (int i = 0; i < 6; ++i) r = r + a[i] * b[i];
  return r;
}
// motion cross product  [w; v] x [w2; v2] = [w x w2; w x v2 + v x w2]
template <class S> std::array<S, 6> crm(const std::array<S, 6>& a, const std::array<S, 6>& b) {
  V3<S> w = {a[0], a[1], a[2]}, v = {a[3], a[4], a[5]}, w2 = {b[0], b[1], b[2]}, v2 = {b[3], b[4], b[5]};
  V3<S> x = vcross(w, w2), y = vadd(vcross(w, v2), vcross(v, w2));
  return {x[0], x[1], x[2], y[0], y[1], y[2]};
}
// force cross product  [w; v] x* [n; f] = [w x n + v x f; w x f]
template <class S> std::array<S, 6> crf(const std::array<S, 6>& a, const std::array<S, 6>& b) {
  V3<S> w = {a[0], a[1], a[2]}, v = {a[3], a[4], a[5]}, n = {b[0], b[1], b[2]}, f = {b[3], b[4], b[5]};
  V3<S> x = vadd(vcross(w, n), vcross(v, f)), y = vcross(w, f);
  return {x[0], x[1], x[2], y[0], y[1], y[2]};
}

// Joint-space inertia matrix by the composite-rigid-body algorithm.
template <class S> void crba(const Model& m, const Kin<S>& k, std::vector<S>& M) {
  const int nb = (int)m.body.size(), nv = m.nv;
  std::vector<std::array<S, 36>> Ic(nb);
  for (int b = 0; b < nb; ++b) Ic[b] = spatial_inertia(m, k, b);
  for (int b = nb - 1; b >= 0; --b)
    if (m.body[b].parent >= 0)
      for (int i = 0; i < 36; ++i) Ic[m.body[b].parent][i] = Ic[m.body[b].parent][i] + Ic[b][i];
  M.assign((size_t)nv * nv, S(0.0));
  for (int i = 0; i < nv; ++i) {
    const int bi = m.dof_body[i];
    std::array<S, 6> F = mat6vec(Ic[bi], k.s[i]);
    for (int j = 0; j <= i; ++j) {
      if (!m.anc[bi][m.dof_body[j]]) continue;
      S x = dot6(k.s[j], F);
      M[(size_t)i * nv + j] = x;
      M[(size_t)j * nv + i] = x;
    }
  }
}

// Bias force c(q, v) (Coriolis, centrifugal, gravity) by recursive Newton-Euler
// with zero joint acceleration; gravity enters as a base acceleration -g.
template <class S> void rne(const Model& m, const Kin<S>& k, const S* v, std::vector<S>& c) {
  const int nb = (int)m.body.size();
  std::vector<std::array<S, 6>> V(nb), A(nb), F(nb);
  for (int b = 0; b < nb; ++b) {
    const Body& B = m.body[b];
    std::array<S, 6> vb{}, ab{};
    if (B.parent >= 0) { vb = V[B.parent]; ab = A[B.parent]; }
    else {
      for (int i = 0; i < 6; ++i) { vb[i] = S(0.0); ab[i] = S(0.0); }
      for (int i = 0; i < 3; ++i) ab[3 + i] = S(-m.grav[i]);
    }
    for (int d = 0; d < B.nv; ++d)
      for (int i = 0; i < 6; ++i) vb[i] = vb[i] + k.s[B.vadr + d][i] * v[B.vadr + d];
    for (int d = 0; d < B.nv; ++d) {
      if (B.jtype == JNT_FREE && d < 3) continue;   // world-fixed translation axes
      std::array<S, 6> sd = crm(vb, k.s[B.vadr + d]);
      for (int i = 0; i < 6; ++i) ab[i] = ab[i] + sd[i] * v[B.vadr + d];
    }
    V[b] = vb; A[b] = ab;
    std::array<S, 36> I = spatial_inertia(m, k, b);
    std::array<S, 6> f1 = mat6vec(I, ab), f2 = crf(vb, mat6vec(I, vb));
    for (int i = 0; i < 6; ++i) F[b][i] = f1[i] + f2[i];
  }
  for (int b = nb - 1; b >= 0; --b)
    if (m.body[b].parent >= 0)
      for (int i = 0; i < 6; ++i) F[m.body[b].parent][i] = F[m.body[b].parent][i] + F[b][i];
  c.assign(m.nv, S(0.0));
  for (int i = 0; i < m.nv; ++i) c[i] = dot6(k.s[i], F[m.dof_body[i]]);
}

// Applied generalised forces: joint damping, motors (gear * u) and position
// servos (kp (u - q) - kd v) on hinge dofs.
template <class S> void applied(const Model& m, const S* q, const S* v, const S* u, std::vector<S>& tau) {
  tau.assign(m.nv, S(0.0));
  for (const Body& B : m.body)
    for (int d = 0; d < B.nv; ++d)
      if (B.damping != 0.0) tau[B.vadr + d] = tau[B.vadr + d] - B.damping * v[B.vadr + d];
  for (int i = 0; i < (int)m.act.size(); ++i) {
    const Act& a = m.act[i];
    if (a.type == ACT_MOTOR) tau[a.vadr] = tau[a.vadr] + a.gear * u[i];
    else tau[a.vadr] = tau[a.vadr] + a.kp * (u[i] - q[a.qadr]) - a.kd * v[a.vadr];
  }
}

// ------------------------------------------------------------------ collision
template <class S> struct Contact {
  S r;                 // signed distance (negative = penetration)
  V3<S> pos;           // contact point (world), midway between the surfaces
  V3<S> n, t1, t2;     // contact frame; n points from body B towards body A
  int bodyA, bodyB;    // bodyB = -1 for the world (plane)
  int pair;
};

// Box signed distance in box coordinates and its gradient (a subgradient
// inside); exact Euclidean distance outside.
template <class S, class H> S box_sdf(const V3<S>& y, const H* h, V3<S>& grad, bool& outside) {
  S qd[3];
  outside = false;
  for (int i = 0; i < 3; ++i) {
    qd[i] = fabs(y[i]) - h[i];
    if (val(qd[i]) > 0) outside = true;
  }
  if (outside) {
    S ss = S(0.0);
    for (int i = 0; i < 3; ++i)
      if (val(qd[i]) > 0) ss = ss + qd[i] * qd[i];
    S d = sqrt(ss);
    for (int i = 0; i < 3; ++i) {
      S g = val(qd[i]) > 0 ? qd[i] / d : S(0.0);
      grad[i] = val(y[i]) < 0 ? -g : g;
    }
    return d;
  }
  int k = 0;
  for (int i = 1; i < 3; ++i)
    if (val(qd[i]) > val(qd[k])) k = i;
  for (int i = 0; i < 3; ++i) grad[i] = S(0.0);
  grad[k] = val(y[k]) < 0 ? S(-1.0) : S(1.0);
  return qd[k];
}

// Frame (n, t1, t2) for a capsule-box contact normal: t1 is perpendicular to n
// and to the world z axis (x axis when n is closer to z than 60 degrees).
template <class S> void normal_frame(const V3<S>& n, V3<S>& t1, V3<S>& t2) {
  V3<S> ref = std::fabs(val(n[2])) < 0.5 ? V3<S>{S(0.0), S(0.0), S(1.0)} : V3<S>{S(1.0), S(0.0), S(0.0)};
  V3<S> t = vcross(n, ref);
  S l = sqrt(vdot(t, t));
  t1 = vscl(t, S(1.0) / l);
  t2 = vcross(n, t1);
}

template <class S>
void capsule_box(const Model& m, const Kin<S>& k, const Pair& P, Contact<S>& ct) {
  const Geom& C = m.geom[P.g1];
  const Geom& Bx = m.geom[P.g2];
  const double rc = C.size[0], L = C.size[1];
  const double* h = Bx.size;
  const S hS[3] = {half_size<S>(m, P.g2, 0), half_size<S>(m, P.g2, 1), half_size<S>(m, P.g2, 2)};
  V3<S> u = {k.gR[P.g1][0], k.gR[P.g1][3], k.gR[P.g1][6]};     // capsule axis = geom x
  // segment in box coordinates: y(s) = y0 + s w, s in [-L, L]
  V3<S> y0 = mtvec(k.gR[P.g2], vsub(k.gp[P.g1], k.gp[P.g2]));
  V3<S> w = mtvec(k.gR[P.g2], u);
  using P_t = double;
  auto dphi = [&](P_t s) {   // derivative of sdf(y(s)) along s (primal)
    V3<P_t> y = {val(y0[0]) + s * val(w[0]), val(y0[1]) + s * val(w[1]), val(y0[2]) + s * val(w[2])};
    V3<P_t> g; bool out;
    box_sdf<P_t>(y, h, g, out);
    return g[0] * val(w[0]) + g[1] * val(w[1]) + g[2] * val(w[2]);
  };
  // sdf(y(s)) is convex in s: bisection on the sign of its derivative.
  double s_star;
  if (dphi(-L) >= 0) s_star = -L;
  else if (dphi(L) <= 0) s_star = L;
  else {
    double lo = -L, hi = L;
    for (int it = 0; it < 200; ++it) {
      double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (dphi(mid) < 0) lo = mid; else hi = mid;
    }
    s_star = 0.5 * (lo + hi);
  }
  // Implicit-function refinement: s = s* - phi'(s*) / phi''(s*) carries
  // ds*/dtheta in derivative types (interior minimum in the edge/corner region
  // of the distance field only, where phi'' > 0).
  S s = S(s_star);
  {
    V3<double> y = {val(y0[0]) + s_star * val(w[0]), val(y0[1]) + s_star * val(w[1]), val(y0[2]) + s_star * val(w[2])};
    V3<double> g; bool out;
    double phi = box_sdf<double>(y, h, g, out);
    if (out && s_star > -L && s_star < L && phi > 0) {
      double gw = g[0] * val(w[0]) + g[1] * val(w[1]) + g[2] * val(w[2]);
      double ww = 0;
      for (int i = 0; i < 3; ++i)
        if (std::fabs(y[i]) > h[i]) ww += val(w[i]) * val(w[i]);
      double phi2 = (ww - gw * gw) / phi;
      if (phi2 > 1e-12) {
        V3<S> yS = vadd(y0, vscl(w, S(s_star)));
        V3<S> gS; bool o2;
        box_sdf<S>(yS, hS, gS, o2);
        S dS = vdot(gS, w);
        s = S(s_star) - dS / phi2;
      }
    }
  }
  V3<S> y = vadd(y0, vscl(w, s));
  V3<S> g; bool out;
  S dist = box_sdf<S>(y, hS, g, out);
  V3<S> nw = mvec(k.gR[P.g2], g);
  V3<S> x = vadd(k.gp[P.g1], vscl(u, s));
  ct.r = dist - rc;
  ct.n = nw;
  ct.pos = vsub(x, vscl(nw, S(rc) + 0.5 * ct.r));
  normal_frame(nw, ct.t1, ct.t2);
  ct.bodyA = C.body;
  ct.bodyB = Bx.body;
}

// All contact slots of the model, in pair order (every slot is evaluated;
// inclusion in the constraint problem is decided by the caller).
// Sphere / capsule pair (App. C.1's "removing discontinuities" pairs, the
// billiard of Sec. 4): each geom is a segment c + s u, |s| <= L along its
// local x (L = 0 for a sphere) of radius rad.  The closest points minimise
// |D + s ua - t ub|^2 (D = ca - cb) over the box |s| <= La, |t| <= Lb: every
// candidate of the optimality conditions (interior, each edge with the other
// variable clamped) is evaluated and the least distance taken.  With the set
// of clamped variables fixed, the free ones solve the reduced linear
// optimality conditions, re-solved in S so that derivative types carry
// ds/dtheta, dt/dtheta.  n points from geom 2 to geom 1, r = |d| - ra - rb,
// pos = pa - (ra + r/2) n.  Degenerate (not differentiable): crossing axes
// (|d| = 0), i.e. penetrations deeper than the radii.
template <class S>
void seg_seg(const Model& m, const Kin<S>& k, const Pair& P, Contact<S>& ct) {
  const Geom& A = m.geom[P.g1];
  const Geom& B = m.geom[P.g2];
  const double ra = A.size[0], La = A.type == GEOM_CAPSULE ? A.size[1] : 0.0;
  const double rb = B.size[0], Lb = B.type == GEOM_CAPSULE ? B.size[1] : 0.0;
  const V3<S> ua = {k.gR[P.g1][0], k.gR[P.g1][3], k.gR[P.g1][6]};
  const V3<S> ub = {k.gR[P.g2][0], k.gR[P.g2][3], k.gR[P.g2][6]};
  const V3<S> D = vsub(k.gp[P.g1], k.gp[P.g2]);
  const double c = val(vdot(ua, ub)), Du = val(vdot(D, ua)), Dv = val(vdot(D, ub));
  auto clampd = [](double x, double L) { return std::min(std::max(x, -L), L); };
  auto f = [&](double s, double t) {
    double d2 = 0;
    for (int i = 0; i < 3; ++i) {
      const double di = val(D[i]) + s * val(ua[i]) - t * val(ub[i]);
      d2 += di * di;
    }
    return d2;
  };
  double bs = 0, bt = 0, best = INFINITY;
  auto consider = [&](double s, double t) {
    if (std::fabs(s) > La || std::fabs(t) > Lb) return;
    const double v = f(s, t);
    if (v < best) { best = v; bs = s; bt = t; }
  };
  if (1.0 - c * c > 1e-12) {
    const double s0 = (c * Dv - Du) / (1.0 - c * c);
    consider(s0, Dv + s0 * c);
  }
  for (double s0 : {-La, La}) consider(s0, clampd(Dv + s0 * c, Lb));
  for (double t0 : {-Lb, Lb}) consider(clampd(t0 * c - Du, La), t0);
  const bool sfree = std::fabs(bs) < La, tfree = std::fabs(bt) < Lb;
  S s = S(bs), t = S(bt);
  const S cS = vdot(ua, ub), DuS = vdot(D, ua), DvS = vdot(D, ub);
  if (sfree && tfree) {            // Du + s - c t = 0, -Dv - c s + t = 0
    const S det = 1.0 - cS * cS;
    s = (cS * DvS - DuS) / det;
    t = DvS + cS * s;
  } else if (sfree) {
    s = S(bt) * cS - DuS;
  } else if (tfree) {
    t = DvS + S(bs) * cS;
  }
  const V3<S> pa = vadd(k.gp[P.g1], vscl(ua, s));
  const V3<S> d = vsub(vadd(D, vscl(ua, s)), vscl(ub, t));
  const S rho = sqrt(vdot(d, d));
  const V3<S> n = vscl(d, S(1.0) / rho);
  ct.r = rho - (ra + rb);
  ct.n = n;
  ct.pos = vsub(pa, vscl(n, S(ra) + 0.5 * ct.r));
  normal_frame(n, ct.t1, ct.t2);
  ct.bodyA = A.body;
  ct.bodyB = B.body;
}

template <class S> void contacts(const Model& m, const Kin<S>& k, std::vector<Contact<S>>& out) {
  out.resize(m.nslot);
  const V3<S> ez = {S(0.0), S(0.0), S(1.0)}, ex = {S(1.0), S(0.0), S(0.0)}, ey = {S(0.0), S(1.0), S(0.0)};
  for (int pi = 0; pi < (int)m.pair.size(); ++pi) {
    const Pair& P = m.pair[pi];
    const Geom& G = m.geom[P.g1];
    for (int j = 0; j < P.nslot; ++j) {
      Contact<S>& ct = out[P.slot0 + j];
      ct.pair = pi;
      if (P.g2 >= 0) {
        if (m.geom[P.g2].type == GEOM_BOX) capsule_box(m, k, P, ct);
        else seg_seg(m, k, P, ct);
        continue;
      }
      ct.bodyA = G.body; ct.bodyB = -1;
      ct.n = ez; ct.t1 = ex; ct.t2 = ey;
      V3<S> cpt;          // sphere centre / capsule end / box vertex
      double rad = 0.0;
      if (G.type == GEOM_SPHERE) { cpt = k.gp[P.g1]; rad = G.size[0]; }
      else if (G.type == GEOM_CAPSULE) {
        V3<S> e = {S(j == 0 ? -G.size[1] : G.size[1]), S(0.0), S(0.0)};
        cpt = vadd(k.gp[P.g1], mvec(k.gR[P.g1], e));
        rad = G.size[0];
      } else {
        const S h0 = half_size<S>(m, P.g1, 0), h1 = half_size<S>(m, P.g1, 1), h2 = half_size<S>(m, P.g1, 2);
        V3<S> e = {(j & 1) ? h0 : -h0, (j & 2) ? h1 : -h1, (j & 4) ? h2 : -h2};
        cpt = vadd(k.gp[P.g1], mvec(k.gR[P.g1], e));
      }
      ct.r = cpt[2] - rad;
      ct.pos = vsub(cpt, vscl(ez, S(rad) + 0.5 * ct.r));
    }
  }
}

// ------------------------------------------------------------------ impedance

// Polynomial spline of the solimp shape (midpoint mid, power pw) on x in [0,1].
template <class S, class M> S spline_shape(const S& x, const M& mid, double pw) {
  if (val(x) <= val(mid) && val(mid) > 0) return pow(x, pw) / pow(mid, pw - 1.0);
  return 1.0 - pow(1.0 - x, pw) / pow(1.0 - mid, pw - 1.0);
}
inline double clamp_imp(double d) { return std::min(std::max(d, 0.0), 0.9999); }
template <class S> S clamp_imp(const S& d) {
  if (val(d) < 0.0) return S(0.0);
  if (val(d) > 0.9999) return S(0.9999);
  return d;
}
// Impedance d(r): solimp spline for r < 0; for r >= 0 the CFD continuation
// (only when cfd is set; otherwise the solimp value at |r|).
template <class S> S impedance(const Model& m, const S& r, bool cfd) {
  if (cfd && val(r) >= 0) {
    const double dc = m.cfd[0], d0 = m.cfd[1], wc = m.cfd[2], mc = m.cfd[3], pc = m.cfd[4];
    S x = 1.0 - r / wc;
    if (val(x) < 0) x = S(0.0);
    return clamp_imp(dc + (d0 - dc) * spline_shape(x, mc, pc));
  }
  const S d_o = par<S>(PAR_DO, m.solimp[0]), d_w = par<S>(PAR_DW, m.solimp[1]), w = par<S>(PAR_WIDTH, m.solimp[2]);
  const S mid = par<S>(PAR_MID, m.solimp[3]);
  const double pw = m.solimp[4];
  S span, den_lo, den_hi;                  // model constants
  {
    FlopsPaused fp;
    span = d_w - d_o;
    den_lo = pow(mid, pw - 1.0);
    den_hi = pow(1.0 - mid, pw - 1.0);
  }
  S x = fabs(r) / w;
  if (val(x) > 1.0) x = S(1.0);
  // the solimp spline (spline_shape) with its midpoint denominators folded
  const S y = (val(x) <= val(mid) && val(mid) > 0) ? pow(x, pw) / den_lo : 1.0 - pow(1.0 - x, pw) / den_hi;
  return clamp_imp(d_o + span * y);
}
template <class S> S softplus(const S& x) {
  if (val(x) > 0) return x + log1p(exp(-x));
  return log1p(exp(x));
}

// ------------------------------------------------------------------ constraint rows
template <class S> struct Rows {
  int nr = 0;
  std::vector<S> J, aref, D;   // J row major nr x nv
  std::vector<int> slot;
};

// Point velocity of dof i at world point x on body b (zero unless dof i moves b).
template <class S> inline V3<S> dof_point_vel(const Model& m, const Kin<S>& k, int i, int b, const V3<S>& x) {
  if (b < 0 || !m.anc[b][m.dof_body[i]]) return {S(0.0), S(0.0), S(0.0)};
  const std::array<S, 6>& s = k.s[i];
  V3<S> w = {s[0], s[1], s[2]}, vo = {s[3], s[4], s[5]};
  return vadd(vo, vcross(w, x));
}

template <class S>
void make_rows(const Model& m, const Kin<S>& k, const std::vector<Contact<S>>& ct, const S* v, bool cfd, Rows<S>& R) {
  const int nv = m.nv;
  R.nr = 0; R.J.clear(); R.aref.clear(); R.D.clear(); R.slot.clear();
  const S tc = par<S>(PAR_TC, m.solref[0]), damp = par<S>(PAR_DAMP, m.solref[1]), dw = par<S>(PAR_DW, m.solimp[1]);
  S bcoef, kcoef;                          // model constants
  {
    FlopsPaused fp;
    bcoef = 2.0 / (dw * tc);
    kcoef = 1.0 / (dw * dw * tc * tc * damp * damp);
  }
  for (int si = 0; si < (int)ct.size(); ++si) {
    const Contact<S>& c = ct[si];
    const bool incl = cfd ? (val(c.r) < m.cfd[2]) : (val(c.r) < 0);
    if (!incl) continue;
    const Pair& P = m.pair[c.pair];
    // point Jacobians projected on the frame axes
    std::vector<S> jn(nv), j1(nv), j2(nv);
    for (int i = 0; i < nv; ++i) {
      V3<S> d = vsub(dof_point_vel(m, k, i, c.bodyA, c.pos), dof_point_vel(m, k, i, c.bodyB, c.pos));
      jn[i] = vdot(c.n, d); j1[i] = vdot(c.t1, d); j2[i] = vdot(c.t2, d);
    }
    S d = impedance(m, c.r, cfd);
    S pterm = cfd ? kcoef * d * (m.softplus_s * softplus(-c.r / m.softplus_s)) : -(kcoef * d * c.r);
    const int nrow = P.condim == 1 ? 1 : 4;
    const S mu = par<S>(PAR_MU0 + c.pair, P.mu);
    S Ahat;                                // model constant
    {
      FlopsPaused fp;
      Ahat = P.condim == 1 ? pair_invw<S>(m, P) : pair_invw<S>(m, P) * (1.0 + mu * mu);
    }
    S Dv = d / (Ahat * (1.0 - d));
    for (int e = 0; e < nrow; ++e) {
      S sgn = (e & 1) ? -mu : mu;
      const std::vector<S>& jt = (e < 2) ? j1 : j2;
      S jv = S(0.0);
      for (int i = 0; i < nv; ++i) {
        S ji = (nrow == 1) ? jn[i] : jn[i] + sgn * jt[i];
        R.J.push_back(ji);
        jv = jv + ji * v[i];
      }
      R.aref.push_back(-(bcoef * jv) + pterm);
      R.D.push_back(Dv);
      R.slot.push_back(si);
      ++R.nr;
    }
  }
}

// ------------------------------------------------------------------ linear algebra
// In-place Cholesky M = L L^T (lower triangle); returns false if not SPD.
template <class S> bool cholesky(std::vector<S>& A, int n) {
  for (int j = 0; j < n; ++j) {
    S s = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) s = s - A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(val(s) > 0)) return false;
    S l = sqrt(s);
    A[(size_t)j * n + j] = l;
    for (int i = j + 1; i < n; ++i) {
      S t = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) t = t - A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = t / l;
    }
  }
  return true;
}
template <class S> void chol_solve(const std::vector<S>& L, int n, std::vector<S>& x) {
  for (int i = 0; i < n; ++i) {
    S t = x[i];
    for (int k = 0; k < i; ++k) t = t - L[(size_t)i * n + k] * x[k];
    x[i] = t / L[(size_t)i * n + i];
  }
  for (int i = n - 1; i >= 0; --i) {
    S t = x[i];
    for (int k = i + 1; k < n; ++k) t = t - L[(size_t)k * n + i] * x[k];
    x[i] = t / L[(size_t)i * n + i];
  }
}

// ------------------------------------------------------------------ A_hat
// Translational inverse weight of every body at the reference pose,
// trace(Jc M(q0)^-1 Jc^T) / 3 (Jc: the body's COM point Jacobian), the
// reading of "an approximation to diag(J M^-1 J^T)" (Sec. 2.1).  In the
// derivative scalar with g_pdir on a body mass it carries the derivative of
// that model constant with respect to the mass.  Returns false if M(q0) is
// not positive definite.
template <class S> bool body_inverse_weights(const Model& m, std::vector<S>& invw) {
  const int nb = (int)m.body.size();
  std::vector<S> q(m.qpos0.begin(), m.qpos0.end());
  Kin<S> k;
  kinematics(m, q.data(), k);
  std::vector<S> M;
  crba(m, k, M);
  if (!cholesky(M, m.nv)) return false;
  invw.assign(nb, S(0.0));
  for (int b = 0; b < nb; ++b) {
    S tr = S(0.0);
    for (int ax = 0; ax < 3; ++ax) {
      std::vector<S> col(m.nv);
      for (int i = 0; i < m.nv; ++i) col[i] = dof_point_vel(m, k, i, b, k.c[b])[ax];
      std::vector<S> x = col;
      chol_solve(M, m.nv, x);
      for (int i = 0; i < m.nv; ++i) tr = tr + col[i] * x[i];
    }
    invw[b] = tr / 3.0;
  }
  return true;
}

// ------------------------------------------------------------------ solver
struct SolveInfo {
  int iters = 0;
  bool noconv = false;
  bool spd_fail = false;
  std::vector<char> active;
};

inline double primal(double x) { return x; }
inline Cnt primal(const Cnt& x) { return x; }
template <class T> inline double primal(const Dual<T>& x) { return val(x); }

// Exact line search: minimiser over alpha >= 0 of the convex piecewise
// quadratic phi(alpha) = 1/2 |a + alpha d - a0|_M^2 + sum_i 1/2 D_i min(0, z_i + alpha s_i)^2.
template <class P>
P exact_line_search(const P& c0, const P& c1, const std::vector<P>& z, const std::vector<P>& s, const std::vector<P>& D) {
  const int nr = (int)z.size();
  std::vector<char> act(nr);
  P slope0 = c0, slope1 = c1;
  std::vector<std::pair<double, int>> bp;
  for (int i = 0; i < nr; ++i) {
    act[i] = (val(z[i]) < 0) || (val(z[i]) == 0 && val(s[i]) < 0);
    if (act[i]) { slope0 = slope0 + D[i] * z[i] * s[i]; slope1 = slope1 + D[i] * s[i] * s[i]; }
    const bool toggles = act[i] ? (val(s[i]) > 0) : (val(s[i]) < 0 && val(z[i]) > 0);
    if (toggles) bp.push_back({val(-z[i] / s[i]), i});
  }
  std::sort(bp.begin(), bp.end());
  P alpha = -slope0 / slope1;
  for (const auto& b : bp) {
    if (val(alpha) <= b.first) break;
    const int i = b.second;
    if (act[i]) { slope0 = slope0 - D[i] * z[i] * s[i]; slope1 = slope1 - D[i] * s[i] * s[i]; }
    else { slope0 = slope0 + D[i] * z[i] * s[i]; slope1 = slope1 + D[i] * s[i] * s[i]; }
    act[i] = !act[i];
    alpha = -slope0 / slope1;
  }
  return val(alpha) < 0 ? P(0.0) : alpha;
}

// Newton method on the primal problem (Eq. primal) with exact line search,
// started from the unconstrained acceleration a0 = M^-1 (tau - c).  With the
// active set A of the iterate a, the Newton target is the minimiser of the
// quadratic of A, a_A = H_A^-1 (tau - c + J_A^T D_A a_ref,A); the search stops
// when the active set of a_A is A itself (then a_A is the exact minimiser: the
// gradient of the primal cost vanishes there), otherwise it moves to the exact
// line minimum between a and a_A.  Returns the final active set.
template <class P>
void newton_active_set(int nv, const std::vector<P>& M, const std::vector<P>& a0, const std::vector<P>& J,
                       const std::vector<P>& aref, const std::vector<P>& D, const std::vector<P>& rhs0, SolveInfo& info) {
  const int nr = (int)aref.size();
  std::vector<P> a = a0, z(nr), zt(nr), H, aA(nv), dlt(nv), s(nr);
  std::vector<char> act(nr), nxt(nr);
  auto residual = [&](const std::vector<P>& x, std::vector<P>& zz, std::vector<char>& st) {
    for (int r = 0; r < nr; ++r) {
      P t = P(0.0);
      for (int i = 0; i < nv; ++i) t = t + J[(size_t)r * nv + i] * x[i];
      zz[r] = t - aref[r];
      st[r] = val(zz[r]) < 0;
    }
  };
  info.noconv = true;
  residual(a, z, act);
  for (int it = 0; it <= 50; ++it) {
    info.iters = it + 1;
    // minimiser of the quadratic of the current active set
    H = M;
    for (int i = 0; i < nv; ++i) aA[i] = rhs0[i];
    for (int r = 0; r < nr; ++r) {
      if (!act[r]) continue;
      for (int i = 0; i < nv; ++i) {
        aA[i] = aA[i] + D[r] * aref[r] * J[(size_t)r * nv + i];
        for (int j = 0; j < nv; ++j) H[(size_t)i * nv + j] = H[(size_t)i * nv + j] + D[r] * J[(size_t)r * nv + i] * J[(size_t)r * nv + j];
      }
    }
    if (!cholesky(H, nv)) { info.spd_fail = true; break; }
    chol_solve(H, nv, aA);
    residual(aA, zt, nxt);
    if (nxt == act) { info.noconv = false; break; }
    // exact line search from a along the Newton direction aA - a
    for (int i = 0; i < nv; ++i) dlt[i] = aA[i] - a[i];
    P c0 = P(0.0), c1 = P(0.0);
    for (int i = 0; i < nv; ++i) {
      P md = P(0.0), mr = P(0.0);
      for (int j = 0; j < nv; ++j) { md = md + M[(size_t)i * nv + j] * dlt[j]; mr = mr + M[(size_t)i * nv + j] * (a[j] - a0[j]); }
      c0 = c0 + dlt[i] * mr;
      c1 = c1 + dlt[i] * md;
    }
    for (int r = 0; r < nr; ++r) {
      P t = P(0.0);
      for (int i = 0; i < nv; ++i) t = t + J[(size_t)r * nv + i] * dlt[i];
      s[r] = t;
    }
    P alpha = exact_line_search<P>(c0, c1, z, s, D);
    for (int i = 0; i < nv; ++i) a[i] = a[i] + alpha * dlt[i];
    residual(a, z, act);
  }
  info.active = act;
}

// Unique minimiser of the primal problem: Newton to find the active set A, then
// a = H_A^-1 (tau - c + J_A^T D_A a_ref,A) with H_A = M + J_A^T D_A J_A (the
// Newton target of the last iteration, recomputed in S).  In a derivative type
// this last solve carries the implicit-function derivative.
template <class S>
void solve_constraints(int nv, const std::vector<S>& M, const std::vector<S>& rhs0, const Rows<S>& R,
                       std::vector<S>& a, std::vector<S>& f, SolveInfo& info) {
  using P = typename PrimalOf<S>::type;
  const int nr = R.nr;
  std::vector<P> Mp(M.size()), rp(nv), Jp(R.J.size()), arp(nr), Dp(nr);
  for (size_t i = 0; i < M.size(); ++i) Mp[i] = primal(M[i]);
  for (int i = 0; i < nv; ++i) rp[i] = primal(rhs0[i]);
  for (size_t i = 0; i < R.J.size(); ++i) Jp[i] = primal(R.J[i]);
  for (int i = 0; i < nr; ++i) { arp[i] = primal(R.aref[i]); Dp[i] = primal(R.D[i]); }
  // Counting scalar without g_count_search: the search for the active set is
  // left out of the count and replaced by one residual check of the final
  // active set (nr dot products of length nv), i.e. the work of a solve whose
  // Newton iteration starts at the right active set.
  constexpr bool counting = std::is_same<S, Cnt>::value || std::is_same<S, Dual<Cnt>>::value;
  const bool skip = counting && !g_count_search;
  if (skip) ++g_flops_paused;
  std::vector<P> L = Mp, a0 = rp;
  if (!cholesky(L, nv)) { info.spd_fail = true; }
  chol_solve(L, nv, a0);
  newton_active_set<P>(nv, Mp, a0, Jp, arp, Dp, rp, info);
  if (skip) { --g_flops_paused; g_flops += (std::int64_t)nr * (2 * nv); }
  std::vector<S> H = M, b = rhs0;
  for (int r = 0; r < nr; ++r) {
    if (!info.active[r]) continue;
    for (int i = 0; i < nv; ++i) {
      b[i] = b[i] + R.D[r] * R.aref[r] * R.J[(size_t)r * nv + i];
      for (int j = 0; j < nv; ++j) H[(size_t)i * nv + j] = H[(size_t)i * nv + j] + R.D[r] * R.J[(size_t)r * nv + i] * R.J[(size_t)r * nv + j];
    }
  }
  if (!cholesky(H, nv)) info.spd_fail = true;
  chol_solve(H, nv, b);
  a = b;
  f.assign(nr, S(0.0));
  for (int r = 0; r < nr; ++r) {
    if (!info.active[r]) continue;
    S t = S(0.0);
    for (int i = 0; i < nv; ++i) t = t + R.J[(size_t)r * nv + i] * a[i];
    f[r] = R.D[r] * (R.aref[r] - t);
  }
}

// ------------------------------------------------------------------ right-hand side
template <class S> struct RhsDiag {
  std::vector<S> M, c, tau, f;
  std::vector<Contact<S>> ct;
  Rows<S> rows;
  SolveInfo info;
};

// v' = F(q, v, u) (cfd = false) or the CFD right-hand side F~ (cfd = true).
// Returns false if the solver did not converge or a factorisation failed.
template <class S>
bool rhs(const Model& m, const S* q, const S* v, const S* u, bool cfd, S* acc, RhsDiag<S>* dg = nullptr) {
  RhsDiag<S> local;
  RhsDiag<S>& D = dg ? *dg : local;
  Kin<S> k;
  kinematics(m, q, k);
  crba(m, k, D.M);
  rne(m, k, v, D.c);
  applied(m, q, v, u, D.tau);
  contacts(m, k, D.ct);
  make_rows(m, k, D.ct, v, cfd, D.rows);
  std::vector<S> rhs0(m.nv), a;
  for (int i = 0; i < m.nv; ++i) rhs0[i] = D.tau[i] - D.c[i];
  D.info = SolveInfo();
  solve_constraints(m.nv, D.M, rhs0, D.rows, a, D.f, D.info);
  for (int i = 0; i < m.nv; ++i) acc[i] = a[i];
  return !D.info.noconv && !D.info.spd_fail;
}

}  // namespace orc
