// Reverse mode (vector-Jacobian products) of the right-hand side
// v' = F(q, v, u) (or F~ of Sec. 4) and of one Dormand-Prince step, for one
// environment handled by a group of G lanes, like the forward code.
//
// rhs_vjp runs right after rhs() on the same inputs and reads the forward
// intermediates that rhs() left in the workspace (poses, motion vectors,
// inertias, body velocities and accelerations, forces, contact records,
// Jacobian rows, the Cholesky factor of H = M + J_A^T D_A J_A of the final
// active set, the solution and its residuals).  The cotangents of those
// intermediates live in a second per-environment workspace (LayoutBar).
//
// The derivative is the one the forward-mode derivative scalars of the
// tangent adjoint compute (the two agree to rounding):
//   * the constraint solve through its final active set A (implicit function
//     theorem: an = H_A^-1 (rhs0 + J_A^T D_A a_ref,A), everything else
//     piecewise constant);
//   * the capsule-box minimiser through the implicit function theorem where
//     it is an interior minimum outside the box, constant elsewhere;
//   * clamps and branches (impedance limits, spline pieces, small-angle
//     series) differentiated on the branch the values take.
// With the constraint solution an and y = H_A^-1 abar, the solve's VJP is
//   rhs0bar = y,  Mbar = -y an^T,  and for every active row r (z = J an - a_ref)
//   a_refbar_r = D_r (J_r y),  Dbar_r = -(J_r y) z_r,
//   Jbar_r = -D_r (z_r y + (J_r y) an)   (+ the a_ref term -bcoef a_refbar_r v).
// Every intermediate's cotangent is written by one lane of the group
// (reductions over children, dofs or slots are gathers by the owner), so the
// result does not depend on scheduling.
#pragma once
#include "dmx_device.cuh"

namespace dmx {

struct WsB {
  double* d;
  const LayoutBar* L;
  __device__ double* at(int off) const { return d + off; }
};

// ------------------------------------------------------------------ small VJP helpers
__device__ __forceinline__ void acc_cross(const double* a, const double* b, double* out) {
  out[0] += a[1] * b[2] - a[2] * b[1];
  out[1] += a[2] * b[0] - a[0] * b[2];
  out[2] += a[0] * b[1] - a[1] * b[0];
}
// Ibar += d/dI (ybar . inertia_apply(I, x)) for the 10-number spatial inertia.
__device__ __forceinline__ void inertia_grad(const double* yb, const double* x, double* Ibar) {
  const double w0 = x[0], w1 = x[1], w2 = x[2], v0 = x[3], v1 = x[4], v2 = x[5];
  Ibar[0] += yb[3] * v0 + yb[4] * v1 + yb[5] * v2;
  // h enters as h x v (angular part) and -(h x w) (linear part)
  Ibar[1] += (v1 * yb[2] - v2 * yb[1]) - (w1 * yb[5] - w2 * yb[4]);
  Ibar[2] += (v2 * yb[0] - v0 * yb[2]) - (w2 * yb[3] - w0 * yb[5]);
  Ibar[3] += (v0 * yb[1] - v1 * yb[0]) - (w0 * yb[4] - w1 * yb[3]);
  Ibar[4] += yb[0] * w0; Ibar[5] += yb[1] * w1; Ibar[6] += yb[2] * w2;
  Ibar[7] += yb[0] * w1 + yb[1] * w0; Ibar[8] += yb[0] * w2 + yb[2] * w0; Ibar[9] += yb[1] * w2 + yb[2] * w1;
}
// c = a x b (motion): abar, bbar += from cbar.  a = (w; v), b = (w2; v2).
__device__ __forceinline__ void crm6_vjp(const double* a, const double* b, const double* cb, double* ab, double* bb) {
  acc_cross(b, cb, ab);            // w2 x cw
  acc_cross(b + 3, cb + 3, ab);    // v2 x cv
  acc_cross(b, cb + 3, ab + 3);    // w2 x cv
  acc_cross(cb, a, bb);            // cw x w
  acc_cross(cb + 3, a + 3, bb);    // cv x v
  acc_cross(cb + 3, a, bb + 3);    // cv x w
}
// c = a x* b (force): a = (w; v), b = (n; f).
__device__ __forceinline__ void crf6_vjp(const double* a, const double* b, const double* cb, double* ab, double* bb) {
  acc_cross(b, cb, ab);            // n x cn
  acc_cross(b + 3, cb + 3, ab);    // f x cf
  acc_cross(b + 3, cb, ab + 3);    // f x cn
  acc_cross(cb, a, bb);            // cn x w
  acc_cross(cb, a + 3, bb + 3);    // cn x v
  acc_cross(cb + 3, a, bb + 3);    // cf x w
}
// qbar += (d R / d q)^T Rbar for R = quat_to_mat(q) = 1 + s P(q), s = 2 / |q|^2.
__device__ __forceinline__ void quat_to_mat_vjp(const double* q, const double* Rb, double* qb) {
  const double w = q[0], x = q[1], y = q[2], z = q[3];
  const double n2 = w * w + x * x + y * y + z * z, s = 2.0 / n2;
  const double P[9] = {-(y * y + z * z), x * y - w * z, x * z + w * y, x * y + w * z, -(x * x + z * z),
                       y * z - w * x,    x * z - w * y, y * z + w * x, -(x * x + y * y)};
  double sb = 0;
  for (int k = 0; k < 9; ++k) sb += Rb[k] * P[k];
  const double gw = -z * Rb[1] + y * Rb[2] + z * Rb[3] - x * Rb[5] - y * Rb[6] + x * Rb[7];
  const double gx = y * Rb[1] + z * Rb[2] + y * Rb[3] - 2 * x * Rb[4] - w * Rb[5] + z * Rb[6] + w * Rb[7] - 2 * x * Rb[8];
  const double gy = -2 * y * Rb[0] + x * Rb[1] + w * Rb[2] + x * Rb[3] + z * Rb[5] - w * Rb[6] + z * Rb[7] - 2 * y * Rb[8];
  const double gz = -2 * z * Rb[0] - w * Rb[1] + x * Rb[2] + w * Rb[3] - 2 * z * Rb[4] + y * Rb[5] + x * Rb[6] + y * Rb[7];
  const double c = -2.0 * sb * s / n2;   // ds/dq = -(s / n2) 2 q
  qb[0] += s * gw + c * w; qb[1] += s * gx + c * x; qb[2] += s * gy + c * y; qb[3] += s * gz + c * z;
}
// Rodrigues rotation about the unit axis a by theta and its theta-derivative.
__device__ __forceinline__ void rodrigues(const double* a, double sn, double cs, double* Rj, double* dR) {
  const double c1 = 1.0 - cs;
  Rj[0] = cs + c1 * a[0] * a[0];        Rj[1] = c1 * a[0] * a[1] - sn * a[2]; Rj[2] = c1 * a[0] * a[2] + sn * a[1];
  Rj[3] = c1 * a[0] * a[1] + sn * a[2]; Rj[4] = cs + c1 * a[1] * a[1];        Rj[5] = c1 * a[1] * a[2] - sn * a[0];
  Rj[6] = c1 * a[0] * a[2] - sn * a[1]; Rj[7] = c1 * a[1] * a[2] + sn * a[0]; Rj[8] = cs + c1 * a[2] * a[2];
  dR[0] = -sn + sn * a[0] * a[0];       dR[1] = sn * a[0] * a[1] - cs * a[2]; dR[2] = sn * a[0] * a[2] + cs * a[1];
  dR[3] = sn * a[0] * a[1] + cs * a[2]; dR[4] = -sn + sn * a[1] * a[1];       dR[5] = sn * a[1] * a[2] - cs * a[0];
  dR[6] = sn * a[0] * a[2] - cs * a[1]; dR[7] = sn * a[1] * a[2] + cs * a[0]; dR[8] = -sn + sn * a[2] * a[2];
}

// Value and derivative of the solimp spline shape on x in [0, 1].
__device__ __forceinline__ double spline_shape_d(double x, double mid, double pw, double* dy) {
  if (x <= mid && mid > 0) {
    const double den = (pw == 2.0) ? mid : ::pow(mid, pw - 1.0);
    double num, dn;
    if (pw == 2.0) { num = x * x; dn = 2.0 * x; }
    else if (pw == 4.0) { num = (x * x) * (x * x); dn = 4.0 * x * x * x; }
    else { num = ::pow(x, pw); dn = pw * ::pow(x, pw - 1.0); }
    *dy = dn / den;
    return num / den;
  }
  const double y = 1.0 - x;
  const double den = (pw == 2.0) ? (1.0 - mid) : ::pow(1.0 - mid, pw - 1.0);
  double num, dn;
  if (pw == 2.0) { num = y * y; dn = 2.0 * y; }
  else if (pw == 4.0) { num = (y * y) * (y * y); dn = 4.0 * y * y * y; }
  else { num = ::pow(y, pw); dn = pw * ::pow(y, pw - 1.0); }
  *dy = dn / den;
  return 1.0 - num / den;
}
// Impedance d(r) (solimp spline; with cfd and r >= 0 the CFD continuation)
// and its derivative, zero on the clamped pieces.
__device__ __forceinline__ double impedance_d(const DevModel& m, double r, bool cfd, double* dd) {
  double d, dr;
  if (cfd && r >= 0) {
    double x = 1.0 - r / m.cfd[2], dx = -1.0 / m.cfd[2];
    if (x < 0) { x = 0.0; dx = 0.0; }
    double dy;
    const double y = spline_shape_d(x, m.cfd[3], m.cfd[4], &dy);
    d = m.cfd[0] + (m.cfd[1] - m.cfd[0]) * y;
    dr = (m.cfd[1] - m.cfd[0]) * dy * dx;
  } else {
    double x = fabs(r) / m.solimp[2], dx = (r < 0 ? -1.0 : 1.0) / m.solimp[2];
    if (x > 1.0) { x = 1.0; dx = 0.0; }
    double dy;
    const double y = spline_shape_d(x, m.solimp[3], m.solimp[4], &dy);
    d = m.solimp[0] + (m.solimp[1] - m.solimp[0]) * y;
    dr = (m.solimp[1] - m.solimp[0]) * dy * dx;
  }
  if (d < 0.0) { *dd = 0.0; return 0.0; }
  if (d > 0.9999) { *dd = 0.0; return 0.9999; }
  *dd = dr;
  return d;
}
// softplus and its derivative (the logistic function), both branches as in softplus().
__device__ __forceinline__ double softplus_d(double x, double* ds) {
  if (x > 0) {
    const double e = ::exp(-x);
    *ds = 1.0 / (1.0 + e);
    return x + ::log1p(e);
  }
  const double e = ::exp(x);
  *ds = e / (1.0 + e);
  return ::log1p(e);
}

// rbar of the slot's impedance terms: ct[14] (a_ref position term) and
// ct[15] (D = d / (A_hat (1 - d))).
__device__ __forceinline__ double impedance_terms_vjp(const DevModel& m, double r, bool cfd, double ahat, double b14,
                                                      double b15) {
  double dd;
  const double d = impedance_d(m, r, cfd, &dd);
  double rb = 0.0, db;
  if (cfd) {
    double sg;
    const double sp = m.softplus * softplus_d(-r / m.softplus, &sg);
    db = b14 * m.kcoef * sp;
    rb -= b14 * m.kcoef * d * sg;
  } else {
    db = -b14 * m.kcoef * r;
    rb -= b14 * m.kcoef * d;
  }
  const double om = 1.0 - d;
  db += b15 / (ahat * om * om);
  return rb + db * dd;
}

// box_sdf VJP at y: ybar += from (distbar, grbar).
__device__ __forceinline__ void box_sdf_vjp(const double* y, const double* h, double distbar, const double* grbar,
                                            double* ybar) {
  double qd[3];
  bool out = false;
  for (int i = 0; i < 3; ++i) { qd[i] = fabs(y[i]) - h[i]; out = out || qd[i] > 0; }
  if (out) {
    double ss = 0.0;
    for (int i = 0; i < 3; ++i) if (qd[i] > 0) ss += qd[i] * qd[i];
    const double d = ::sqrt(ss), inv = 1.0 / d;
    double gg[3], ggb = 0.0;
    for (int i = 0; i < 3; ++i) {
      gg[i] = qd[i] > 0 ? (y[i] < 0 ? -qd[i] : qd[i]) * inv : 0.0;
      ggb += gg[i] * grbar[i];
    }
    // dist = |qd+|, grad = sgn qd+ / dist: d grad = (1 - g g^T) dy / dist on the outside axes
    for (int i = 0; i < 3; ++i)
      if (qd[i] > 0) ybar[i] += distbar * gg[i] + (grbar[i] - gg[i] * ggb) * inv;
    return;
  }
  int k = 0;
  if (qd[1] > qd[k]) k = 1;
  if (qd[2] > qd[k]) k = 2;
  ybar[k] += y[k] < 0 ? -distbar : distbar;
}

// Capsule-box contact record VJP.  cb: cotangents of (r, pos, n, t1, t2) in
// cb[0..12] (cb[0] already holds the impedance part of rbar).  Accumulates the
// pose cotangents of g1 (R1bar 9, c1bar 3) and g2 (R2bar 9, c2bar 3).
static __device__ void capsule_box_vjp(const DevModel& m, const double* gR, const double* gp, int g1, int g2,
                                const double* cb, double* b1, double* b2) {
  const double rc = m.g_size[g1][0], Lh = m.g_size[g1][1];
  const double* h = m.g_size[g2];
  const double* R1 = gR + 9 * g1; const double* R2 = gR + 9 * g2;
  const double* c1 = gp + 3 * g1; const double* c2 = gp + 3 * g2;
  const double dc[3] = {c1[0] - c2[0], c1[1] - c2[1], c1[2] - c2[2]};
  const double u[3] = {R1[0], R1[3], R1[6]};
  double y0[3], wv[3];
  matTvec3(R2, dc, y0);
  matTvec3(R2, u, wv);
  const double sv = capsule_box_s(y0, wv, Lh, h);
  const double phi2 = capsule_box_curv(y0, wv, sv, Lh, h);
  const double y[3] = {y0[0] + sv * wv[0], y0[1] + sv * wv[1], y0[2] + sv * wv[2]};
  double gr[3], n[3];
  const double dist = box_sdf(y, h, gr);
  matvec3(R2, gr, n);
  const double r = dist - rc, off = rc + 0.5 * r;
  double ref[3] = {0, 0, 1};
  if (fabs(n[2]) >= 0.5) { ref[0] = 1; ref[2] = 0; }
  double t1r[3], t1[3];
  cross3(n, ref, t1r);
  const double il = rsqrt_t(dot3(t1r, t1r));
  for (int i = 0; i < 3; ++i) t1[i] = t1r[i] * il;
  // reverse
  double nb[3] = {cb[4], cb[5], cb[6]}, t1b[3] = {cb[7], cb[8], cb[9]};
  const double* t2b = cb + 10;
  const double* posb = cb + 1;
  acc_cross(t1, t2b, nb);                    // t2 = n x t1
  acc_cross(t2b, n, t1b);
  const double tt = dot3(t1, t1b);
  double t1rb[3];
  for (int i = 0; i < 3; ++i) t1rb[i] = il * (t1b[i] - t1[i] * tt);
  acc_cross(ref, t1rb, nb);                  // t1r = n x ref
  double sb = dot3(u, posb), ub[3];          // pos = c1 + s u - off n
  for (int i = 0; i < 3; ++i) { b1[9 + i] += posb[i]; ub[i] = sv * posb[i]; nb[i] -= off * posb[i]; }
  const double rb = cb[0] - 0.5 * dot3(n, posb);
  double grb[3];                              // n = R2 gr
  matTvec3(R2, nb, grb);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) b2[3 * i + j] += nb[i] * gr[j];
  double yb[3] = {0, 0, 0};
  box_sdf_vjp(y, h, rb, grb, yb);            // dist = r + rc
  double y0b[3], wvb[3];
  for (int i = 0; i < 3; ++i) { y0b[i] = yb[i]; wvb[i] = sv * yb[i]; }
  sb += dot3(wv, yb);
  if (phi2 > 0) {
    // s = s*(y0, wv): ds = -(dslope/dy0 dy0 + dslope/dwv dwv) / phi'', with
    // dslope/dy0 = Hs wv and dslope/dwv = g + s Hs wv (Hs: Hessian of the field)
    double gv[3], a[3];
    box_sdf(y, h, gv);
    double qd[3], ss = 0.0;
    for (int i = 0; i < 3; ++i) { qd[i] = fabs(y[i]) - h[i]; if (qd[i] > 0) ss += qd[i] * qd[i]; }
    const double inv = 1.0 / ::sqrt(ss);
    const double gw = dot3(gv, wv);
    for (int i = 0; i < 3; ++i) a[i] = qd[i] > 0 ? (wv[i] - gv[i] * gw) * inv : 0.0;
    const double c = -sb / phi2;
    for (int i = 0; i < 3; ++i) { y0b[i] += c * a[i]; wvb[i] += c * (gv[i] + sv * a[i]); }
  }
  double dcb[3];                              // y0 = R2^T dc, wv = R2^T u
  matvec3(R2, y0b, dcb);
  double uw[3];
  matvec3(R2, wvb, uw);
  for (int i = 0; i < 3; ++i) {
    ub[i] += uw[i];
    for (int j = 0; j < 3; ++j) b2[3 * i + j] += dc[i] * y0b[j] + u[i] * wvb[j];
  }
  b1[0] += ub[0]; b1[3] += ub[1]; b1[6] += ub[2];   // u = first column of R1
  for (int i = 0; i < 3; ++i) { b1[9 + i] += dcb[i]; b2[9 + i] -= dcb[i]; }
}


// ------------------------------------------------------------------ right-hand side VJP
// Jacobian-entry cotangents of slot s (rows from r0) at dof i, folded back to
// the normal / tangent point Jacobians: jb = cotangents of (jn, j1, j2).
// pv = velocity direction of the contact point under dof i, sg = +1 when dof
// i moves the first geom's body, -1 the second's.  Returns false when the dof
// moves neither or both (no Jacobian entry).  With ya_i = an_i + bcoef v_i:
//   Jbar_r,i = -(D_r z_r y_i + D_r (J_r y) ya_i)   (active rows, else 0).
__device__ __forceinline__ bool slot_jbar(const DevModel& m, const Ws& w, const WsB& b, int s, int r0, int i,
                                          double yi, double yai, double* jb, double* pv, double* sg) {
  const Layout& L = *w.L;
  const LayoutBar& LB = *b.L;
  const int p = m.s_pair[s];
  const int bA = m.g_body[m.p_g1[p]];
  const int bB = m.p_g2[p] >= 0 ? m.g_body[m.p_g2[p]] : -1;
  const int bi = m.dof_body[i];
  const bool mA = (m.b_anc[bA] >> bi) & 1u;
  const bool mB = bB >= 0 && ((m.b_anc[bB] >> bi) & 1u);
  if (mA == mB) return false;
  const double* ct = w.at(L.ct) + 16 * s;
  const double* sv = w.at(L.sd) + 6 * i;
  cross3(sv, ct + 1, pv);
  pv[0] += sv[3]; pv[1] += sv[4]; pv[2] += sv[5];
  *sg = mA ? 1.0 : -1.0;
  const double* cz = b.at(LB.cz); const double* cj = b.at(LB.cj);
  if (m.p_condim[p] == 1) {
    jb[0] = -(cz[r0] * yi + cj[r0] * yai);
    jb[1] = 0.0; jb[2] = 0.0;
  } else {
    double e[4];
    for (int k = 0; k < 4; ++k) e[k] = -(cz[r0 + k] * yi + cj[r0 + k] * yai);
    const double mu = m.p_mu[p];
    jb[0] = (e[0] + e[1]) + (e[2] + e[3]);
    jb[1] = mu * (e[0] - e[1]);
    jb[2] = mu * (e[2] - e[3]);
  }
  return true;
}

// qbar, vbar, ubar += (dF/d(q, v, u))^T abar at the inputs of the rhs() call
// that immediately precedes this one (same q, v, u, cfd; st = its status).
template <int G>
__device__ void rhs_vjp(const Grp<G>& g, const DevModel& m, const Ws& w, const WsB& b, const double* q,
                        const double* v, const double* u, bool cfd, int st, const double* abar, double* qbar,
                        double* vbar, double* ubar) {
  const Layout& L = *w.L;
  const LayoutBar& LB = *b.L;
  const int nq = m.nq, nv = m.nv, nb = m.nbody;
  if (st == ENV_ROW_OVERFLOW) return;   // the rows were never built: no derivative
  const int* slotrow = w.i + L.slotrow;
  const int* rowid = w.i + L.rowid;
  const int* am = w.i + L.amask;
  const int nr = slotrow[m.nslot];
  const double thr = cfd ? m.cfd[2] : 0.0;
  const double* R = w.at(L.R); const double* P = w.at(L.p); const double* C = w.at(L.com);
  const double* S = w.at(L.sd); const double* Ib = w.at(L.Ib); const double* Ic = w.at(L.Ic);
  const double* F = w.at(L.F); const double* V = w.at(L.Vb); const double* A = w.at(L.Ab);
  const double* Fb = w.at(L.Fb); const double* gR = w.at(L.gR); const double* gp = w.at(L.gp);
  const double* an = w.at(L.an); const double* J = w.at(L.J); const double* Dr = w.at(L.Dr);
  const double* z = w.at(L.z); const double* CT = w.at(L.ct);
  double* Rb = b.at(LB.R); double* pb = b.at(LB.p); double* cR = b.at(LB.cR); double* cp = b.at(LB.cp);
  double* Sb = b.at(LB.S); double* Fd = b.at(LB.F); double* Ibb = b.at(LB.Ib); double* Icb = b.at(LB.Ic);
  double* Vbb = b.at(LB.V); double* Abb = b.at(LB.A); double* Fbb = b.at(LB.Fb); double* SB = b.at(LB.slot);
  double* y = b.at(LB.y); double* jy = b.at(LB.jy); double* cz = b.at(LB.cz); double* cj = b.at(LB.cj);
  double* qb = b.at(LB.q); double* vb = b.at(LB.v); double* ub = b.at(LB.u);
  for (int k = g.lane; k < LB.qn - LB.R; k += G) Rb[k] = 0.0;   // every right-hand-side cotangent
  for (int i = g.lane; i < nv; i += G) y[i] = abar[i];
  g.sync();
  // ---- constraint solve: y = H_A^-1 abar with the factor of the final set
  chol_solve(g, w.at(L.H), w.at(L.tmp2), y, nv);
  for (int r = g.lane; r < nr; r += G) {
    double t = 0.0;
    if (mask_has(am, rowid[r]))
      for (int i = 0; i < nv; ++i) t += J[r * nv + i] * y[i];
    jy[r] = t;
    cz[r] = mask_has(am, rowid[r]) ? Dr[r] * z[r] : 0.0;
    cj[r] = Dr[r] * t;
  }
  g.sync();
  // ---- per dof: a_ref's J v term, damping, bias force, CRBA products, contact Jacobians
  for (int i = g.lane; i < nv; i += G) {
    const int bi = m.dof_body[i];
    double acc = -m.b_damping[bi] * y[i];
    for (int r = 0; r < nr; ++r) acc -= m.bcoef * cj[r] * J[r * nv + i];
    vb[i] += acc;
    double* sbi = Sb + 6 * i;
    const double* fb = Fb + 6 * bi;
    for (int e = 0; e < 6; ++e) sbi[e] -= y[i] * fb[e];
    // M_kj = S_j . F_k for j <= k with dof j's body an ancestor of dof k's body
    double fd[6] = {0, 0, 0, 0, 0, 0};
    for (int j = 0; j <= i; ++j) {
      if (!((m.b_anc[bi] >> m.dof_body[j]) & 1u)) continue;
      const double wij = (i == j) ? -y[i] * an[i] : -(y[i] * an[j] + y[j] * an[i]);
      for (int e = 0; e < 6; ++e) fd[e] += wij * S[6 * j + e];
    }
    for (int e = 0; e < 6; ++e) Fd[6 * i + e] = fd[e];
    for (int k = i; k < nv; ++k) {
      if (!((m.b_anc[m.dof_body[k]] >> bi) & 1u)) continue;
      const double wki = (i == k) ? -y[i] * an[i] : -(y[k] * an[i] + y[i] * an[k]);
      for (int e = 0; e < 6; ++e) sbi[e] += wki * F[6 * k + e];
    }
    const double yai = an[i] + m.bcoef * v[i];
    for (int s = 0; s < m.nslot; ++s) {
      const int r0 = slotrow[s];
      if (r0 < 0) continue;
      double jb[3], pv[3], sg;
      if (!slot_jbar(m, w, b, s, r0, i, y[i], yai, jb, pv, &sg)) continue;
      const double* ct = CT + 16 * s;
      double pvb[3];
      for (int k = 0; k < 3; ++k) pvb[k] = sg * (jb[0] * ct[4 + k] + jb[1] * ct[7 + k] + jb[2] * ct[10 + k]);
      acc_cross(ct + 1, pvb, sbi);      // pv = S_ang x pos + S_lin
      sbi[3] += pvb[0]; sbi[4] += pvb[1]; sbi[5] += pvb[2];
    }
  }
  // ---- per slot: record cotangents, impedance terms, contact geometry
  for (int s = g.lane; s < m.nslot; s += G) {
    const int r0 = slotrow[s];
    if (r0 < 0) continue;
    const double* ct = CT + 16 * s;
    double* sb = SB + SLOTBAR * s;
    const int p = m.s_pair[s];
    const int nrow = m.p_condim[p] == 1 ? 1 : 4;
    double cb[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    for (int i = 0; i < nv; ++i) {
      double jb[3], pv[3], sg;
      if (!slot_jbar(m, w, b, s, r0, i, y[i], an[i] + m.bcoef * v[i], jb, pv, &sg)) continue;
      const double* sv = S + 6 * i;
      double pvb[3];
      for (int k = 0; k < 3; ++k) {
        cb[4 + k] += sg * jb[0] * pv[k];
        cb[7 + k] += sg * jb[1] * pv[k];
        cb[10 + k] += sg * jb[2] * pv[k];
        pvb[k] = sg * (jb[0] * ct[4 + k] + jb[1] * ct[7 + k] + jb[2] * ct[10 + k]);
      }
      acc_cross(pvb, sv, cb + 1);       // pos cotangent from S_ang x pos
    }
    double b14 = 0.0, b15 = 0.0;
    for (int e = 0; e < nrow; ++e) { b14 += cj[r0 + e]; b15 -= jy[r0 + e] * z[r0 + e]; }
    const double r = ct[0];
    if (r < thr) {
      const double ahat = m.p_condim[p] == 1 ? m.p_ahat[p] : m.p_ahat_edge[p];
      cb[0] += impedance_terms_vjp(m, r, cfd, ahat, b14, b15);
    }
    double* b1 = sb; double* b2 = sb + 12;
    const int g1 = m.p_g1[p];
    if (m.p_g2[p] >= 0) {
      capsule_box_vjp(m, gR, gp, g1, m.p_g2[p], cb, b1, b2);
    } else {
      // r = pt_z - rad, pos = (pt_x, pt_y, pt_z - rad - r / 2); fixed frame
      const double ptb[3] = {cb[1], cb[2], cb[0] + 0.5 * cb[3]};
      const int ty = m.g_type[g1];
      b1[9] += ptb[0]; b1[10] += ptb[1]; b1[11] += ptb[2];
      if (ty == GEOM_CAPSULE) {
        const double e = (m.s_idx[s] == 0) ? -m.g_size[g1][1] : m.g_size[g1][1];
        b1[0] += e * ptb[0]; b1[3] += e * ptb[1]; b1[6] += e * ptb[2];
      } else if (ty == GEOM_BOX) {
        const int j = m.s_idx[s];
        const double ex[3] = {(j & 1) ? m.g_size[g1][0] : -m.g_size[g1][0], (j & 2) ? m.g_size[g1][1] : -m.g_size[g1][1],
                              (j & 4) ? m.g_size[g1][2] : -m.g_size[g1][2]};
        for (int a = 0; a < 3; ++a)
          for (int c = 0; c < 3; ++c) b1[3 * a + c] += ptb[a] * ex[c];
      }
    }
  }
  g.sync();
  // ---- per body: geom poses -> body pose; bias-force and CRBA cotangents of its dofs
  for (int bb = g.lane; bb < nb; bb += G) {
    double* rb = Rb + 9 * bb; double* pbb = pb + 3 * bb;
    for (int gi = 0; gi < m.ngeom; ++gi) {
      if (m.g_body[gi] != bb) continue;
      double gRb[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, gpb[3] = {0, 0, 0};
      for (int s = 0; s < m.nslot; ++s) {
        if (slotrow[s] < 0) continue;
        const int p = m.s_pair[s];
        const double* src = nullptr;
        if (m.p_g1[p] == gi) src = SB + SLOTBAR * s;
        else if (m.p_g2[p] == gi) src = SB + SLOTBAR * s + 12;
        if (!src) continue;
        for (int k = 0; k < 9; ++k) gRb[k] += src[k];
        for (int k = 0; k < 3; ++k) gpb[k] += src[9 + k];
      }
      // gR = R_b Roff, gp = p_b + R_b gpos
      const double* Ro = m.g_Roff[gi]; const double* gpos = m.g_pos[gi];
      for (int i = 0; i < 3; ++i) {
        for (int j = 0; j < 3; ++j)
          rb[3 * i + j] += gRb[3 * i] * Ro[3 * j] + gRb[3 * i + 1] * Ro[3 * j + 1] + gRb[3 * i + 2] * Ro[3 * j + 2] +
                           gpb[i] * gpos[j];
        pbb[i] += gpb[i];
      }
    }
    const int va = m.b_vadr[bb], nd = m.b_nv[bb];
    const double* I = Ic + 10 * bb;
    double* fbb = Fbb + 6 * bb; double* icb = Icb + 10 * bb;
    for (int d = 0; d < nd; ++d) {
      const int i = va + d;
      for (int e = 0; e < 6; ++e) fbb[e] -= y[i] * S[6 * i + e];   // c_i = S_i . Fb
      inertia_grad(Fd + 6 * i, S + 6 * i, icb);                     // F_i = Ic S_i
      double t[6];
      inertia_apply(I, Fd + 6 * i, t);
      for (int e = 0; e < 6; ++e) Sb[6 * i + e] += t[e];
    }
  }
  g.sync();
  // accumulated forces and composite inertias: cotangents flow from parents to children
  for (int lev = 0; lev < m.nlevel; ++lev) {
    for (int k = m.level_start[lev] + g.lane; k < m.level_start[lev + 1]; k += G) {
      const int bb = m.level_list[k];
      const int par = m.b_parent[bb];
      if (par >= 0) {
        for (int e = 0; e < 6; ++e) Fbb[6 * bb + e] += Fbb[6 * par + e];
        for (int e = 0; e < 10; ++e) Icb[10 * bb + e] += Icb[10 * par + e];
      }
      for (int e = 0; e < 10; ++e) Ibb[10 * bb + e] += Icb[10 * bb + e];
    }
    g.sync();
  }
  // ---- recursive Newton-Euler (forward: V = V_parent + S v, A = A_parent + (V x S) v,
  // F = I A + V x* (I V)), reversed with the same split: per-body work for all
  // bodies at once, sums along the tree level by level
  for (int bb = g.lane; bb < nb; bb += G) {      // F's cotangent -> A, V (own terms)
    const double* vbv = V + 6 * bb; const double* abv = A + 6 * bb; const double* I = Ib + 10 * bb;
    const double* fbar = Fbb + 6 * bb;
    double* ibb = Ibb + 10 * bb;
    double abar6[6], vbar6[6] = {0, 0, 0, 0, 0, 0}, ivb[6] = {0, 0, 0, 0, 0, 0}, iv[6], t[6];
    inertia_apply(I, fbar, abar6);               // f1 = I ab
    inertia_grad(fbar, abv, ibb);
    inertia_apply(I, vbv, iv);                   // f2 = vb x* (I vb)
    crf6_vjp(vbv, iv, fbar, vbar6, ivb);
    inertia_apply(I, ivb, t);
    for (int e = 0; e < 6; ++e) vbar6[e] += t[e];
    inertia_grad(ivb, vbv, ibb);
    for (int e = 0; e < 6; ++e) { Vbb[6 * bb + e] = vbar6[e]; Abb[6 * bb + e] = abar6[e]; }
  }
  g.sync();
  for (int lev = m.nlevel - 1; lev >= 1; --lev) {   // A_child = A_parent + ...: gather into parents
    for (int k = m.level_start[lev - 1] + g.lane; k < m.level_start[lev]; k += G) {
      const int bb = m.level_list[k];
      for (int c = 0; c < m.child_count[bb]; ++c) {
        const int ch = m.child_list[m.child_start[bb] + c];
        for (int e = 0; e < 6; ++e) Abb[6 * bb + e] += Abb[6 * ch + e];
      }
    }
    g.sync();
  }
  for (int bb = g.lane; bb < nb; bb += G) {      // A's own term (V x S_d) v_d
    const double* vbv = V + 6 * bb; const double* abar6 = Abb + 6 * bb;
    const int va = m.b_vadr[bb], nd = m.b_nv[bb];
    const int d0 = (m.b_jtype[bb] == JNT_FREE) ? 3 : 0;
    for (int d = d0; d < nd; ++d) {
      const double* sd = S + 6 * (va + d);
      double cm[6];
      crm6(vbv, sd, cm);
      double s1 = 0.0, cb6[6];
      for (int e = 0; e < 6; ++e) { s1 += abar6[e] * cm[e]; cb6[e] = abar6[e] * v[va + d]; }
      vb[va + d] += s1;
      crm6_vjp(vbv, sd, cb6, Vbb + 6 * bb, Sb + 6 * (va + d));
    }
  }
  g.sync();
  for (int lev = m.nlevel - 1; lev >= 1; --lev) {   // V_child = V_parent + ...
    for (int k = m.level_start[lev - 1] + g.lane; k < m.level_start[lev]; k += G) {
      const int bb = m.level_list[k];
      for (int c = 0; c < m.child_count[bb]; ++c) {
        const int ch = m.child_list[m.child_start[bb] + c];
        for (int e = 0; e < 6; ++e) Vbb[6 * bb + e] += Vbb[6 * ch + e];
      }
    }
    g.sync();
  }
  for (int bb = g.lane; bb < nb; bb += G) {      // V's own term S_d v_d
    const double* vbar6 = Vbb + 6 * bb;
    const int va = m.b_vadr[bb], nd = m.b_nv[bb];
    for (int d = 0; d < nd; ++d) {
      const double* sd = S + 6 * (va + d);
      double s1 = 0.0;
      for (int e = 0; e < 6; ++e) { s1 += vbar6[e] * sd[e]; Sb[6 * (va + d) + e] += vbar6[e] * v[va + d]; }
      vb[va + d] += s1;
    }
  }
  g.sync();
  if (g.lane == 0) {
    for (int a = 0; a < m.nact; ++a) {
      const int vi = m.a_vadr[a];
      if (m.a_type[a] == ACT_MOTOR) ub[a] += m.a_gear[a] * y[vi];
      else { ub[a] += m.a_kp[a] * y[vi]; qb[m.a_qadr[a]] -= m.a_kp[a] * y[vi]; vb[vi] -= m.a_kd[a] * y[vi]; }
    }
  }
  // ---- kinematics (forward: local rotation Rl = Roff Rj(theta) or the free joint's
  // pose; R = R_parent Rl, p = p_parent + R_parent b_pos; then COMs, inertias,
  // motion vectors and geoms from (R, p)).  Own terms of every body first.
  for (int bb = g.lane; bb < nb; bb += G) {
    double* rb = Rb + 9 * bb; double* pbv = pb + 3 * bb;   // geom terms are already in
    const double* Rv = R + 9 * bb; const double* pv = P + 3 * bb; const double* c = C + 3 * bb;
    // spatial inertia about the origin: (m, m c, R diag(In) R^T + m (|c|^2 - c c^T))
    const double ms = m.b_mass[bb];
    const double* In = m.b_inertia[bb];
    const double* ib = Ibb + 10 * bb;
    double cb3[3] = {ms * ib[1], ms * ib[2], ms * ib[3]};
    const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
    for (int e = 0; e < 6; ++e) {
      const int i = ii[e], j = jj[e];
      const double be = ib[4 + e];
      for (int kk = 0; kk < 3; ++kk) {
        rb[3 * i + kk] += be * Rv[3 * j + kk] * In[kk];
        rb[3 * j + kk] += be * Rv[3 * i + kk] * In[kk];
      }
      if (i == j) for (int kk = 0; kk < 3; ++kk) cb3[kk] += be * ms * 2.0 * c[kk];
      cb3[i] -= be * ms * c[j];
      cb3[j] -= be * ms * c[i];
    }
    // c = R com + p
    for (int i = 0; i < 3; ++i) {
      for (int j = 0; j < 3; ++j) rb[3 * i + j] += cb3[i] * m.b_com[bb][j];
      pbv[i] += cb3[i];
    }
    // dof motion vectors
    const int va = m.b_vadr[bb];
    if (m.b_jtype[bb] == JNT_FREE) {
      for (int d = 0; d < 3; ++d) {
        const double* sbd = Sb + 6 * (va + 3 + d);
        const double sr[3] = {Rv[d], Rv[3 + d], Rv[6 + d]};
        double srb[3] = {sbd[0], sbd[1], sbd[2]};
        acc_cross(sbd + 3, pv, srb);           // lin = p x sr
        acc_cross(sr, sbd + 3, pbv);
        rb[d] += srb[0]; rb[3 + d] += srb[1]; rb[6 + d] += srb[2];
      }
    } else {
      const double* sbd = Sb + 6 * va;
      const double* ax = m.b_axis[bb];
      double sh[3];
      matvec3(Rv, ax, sh);
      double shb[3] = {sbd[0], sbd[1], sbd[2]};
      acc_cross(sbd + 3, pv, shb);             // lin = p x sh
      acc_cross(sh, sbd + 3, pbv);
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) rb[3 * i + j] += shb[i] * ax[j];
      // the local rotation, for the composition below
      double Rj[9], dRj[9], sn, cs;
      ::sincos(q[m.b_qadr[bb]], &sn, &cs);
      rodrigues(ax, sn, cs, Rj, dRj);
      matmul3(m.b_Roff[bb], Rj, cR + 9 * bb);
    }
  }
  g.sync();
  // composition, leaves to root: R_parent gets Rbar Rl^T + pbar b_pos^T, p_parent gets pbar
  for (int lev = m.nlevel - 1; lev >= 1; --lev) {
    for (int k = m.level_start[lev - 1] + g.lane; k < m.level_start[lev]; k += G) {
      const int bb = m.level_list[k];
      double* rb = Rb + 9 * bb; double* pbv = pb + 3 * bb;
      for (int c = 0; c < m.child_count[bb]; ++c) {
        const int ch = m.child_list[m.child_start[bb] + c];
        if (m.b_jtype[ch] == JNT_FREE) continue;
        const double* rc = Rb + 9 * ch; const double* pc = pb + 3 * ch;
        const double* Rl = cR + 9 * ch; const double* bp = m.b_pos[ch];
        for (int i = 0; i < 3; ++i) {
          for (int j = 0; j < 3; ++j)
            rb[3 * i + j] += rc[3 * i] * Rl[3 * j] + rc[3 * i + 1] * Rl[3 * j + 1] + rc[3 * i + 2] * Rl[3 * j + 2] +
                             pc[i] * bp[j];
          pbv[i] += pc[i];
        }
      }
    }
    g.sync();
  }
  // joint coordinates
  for (int bb = g.lane; bb < nb; bb += G) {
    const double* rb = Rb + 9 * bb; const double* pbv = pb + 3 * bb;
    const int qa = m.b_qadr[bb];
    if (m.b_jtype[bb] == JNT_FREE) {
      qb[qa] += pbv[0]; qb[qa + 1] += pbv[1]; qb[qa + 2] += pbv[2];
      quat_to_mat_vjp(q + qa + 3, rb, qb + qa + 3);
      continue;
    }
    // Rl bar = R_parent^T Rbar; Rj bar = Roff^T Rl bar; theta bar = <Rj bar, dRj/dtheta>
    const int par = m.b_parent[bb];
    double rl[9];
    if (par >= 0) {
      const double* Rp = R + 9 * par;
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) rl[3 * i + j] = Rp[i] * rb[j] + Rp[3 + i] * rb[3 + j] + Rp[6 + i] * rb[6 + j];
    } else {
      for (int e = 0; e < 9; ++e) rl[e] = rb[e];
    }
    double Rj[9], dRj[9], sn, cs;
    ::sincos(q[qa], &sn, &cs);
    rodrigues(m.b_axis[bb], sn, cs, Rj, dRj);
    const double* Ro = m.b_Roff[bb];
    double th = 0.0;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        th += (Ro[i] * rl[j] + Ro[3 + i] * rl[3 + j] + Ro[6 + i] * rl[6 + j]) * dRj[3 * i + j];
    qb[qa] += th;
  }
  g.sync();
  for (int i = g.lane; i < nq; i += G) qbar[i] += qb[i];
  for (int i = g.lane; i < nv; i += G) vbar[i] += vb[i];
  for (int a = g.lane; a < m.nu; a += G) ubar[a] += ub[a];
  g.sync();
}

// ------------------------------------------------------------------ integrator VJPs
// out = q (+) dq (integrate_pos): qbar += and dqbar = from outbar.
template <int G>
__device__ void integrate_pos_vjp(const Grp<G>& g, const DevModel& m, const double* q, const double* dq,
                                  const double* ob, double* qbar, double* dqbar) {
  for (int b = g.lane; b < m.nbody; b += G) {
    const int qa = m.b_qadr[b], va = m.b_vadr[b];
    if (m.b_jtype[b] == JNT_HINGE) { qbar[qa] += ob[qa]; dqbar[va] = ob[qa]; continue; }
    for (int k = 0; k < 3; ++k) { qbar[qa + k] += ob[qa + k]; dqbar[va + k] = ob[qa + k]; }
    const double* d = dq + va + 3;
    const double th2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    double cw, sk, dcw, dsk;   // and their derivatives with respect to th2
    if (th2 < 1e-2) {   // the series branch of integrate_pos
      cw = 1.0 + th2 * (-1.0 / 8.0 + th2 * (1.0 / 384.0 + th2 * (-1.0 / 46080.0 + th2 * (1.0 / 10321920.0))));
      sk = 0.5 + th2 * (-1.0 / 48.0 + th2 * (1.0 / 3840.0 + th2 * (-1.0 / 645120.0 + th2 * (1.0 / 185794560.0))));
      dcw = -1.0 / 8.0 + th2 * (2.0 / 384.0 + th2 * (-3.0 / 46080.0 + th2 * (4.0 / 10321920.0)));
      dsk = -1.0 / 48.0 + th2 * (2.0 / 3840.0 + th2 * (-3.0 / 645120.0 + th2 * (4.0 / 185794560.0)));
    } else {
      const double th = ::sqrt(th2);
      double sn, cs;
      ::sincos(0.5 * th, &sn, &cs);
      cw = cs;
      sk = sn / th;
      dcw = -sn / (4.0 * th);
      dsk = (0.5 * th * cs - sn) / (2.0 * th2 * th);
    }
    const double e[4] = {cw, sk * d[0], sk * d[1], sk * d[2]};
    const double* qq = q + qa + 3;
    double r[4];
    r[0] = qq[0] * e[0] - qq[1] * e[1] - qq[2] * e[2] - qq[3] * e[3];
    r[1] = qq[0] * e[1] + qq[1] * e[0] + qq[2] * e[3] - qq[3] * e[2];
    r[2] = qq[0] * e[2] - qq[1] * e[3] + qq[2] * e[0] + qq[3] * e[1];
    r[3] = qq[0] * e[3] + qq[1] * e[2] - qq[2] * e[1] + qq[3] * e[0];
    const double in = rsqrt_t(r[0] * r[0] + r[1] * r[1] + r[2] * r[2] + r[3] * r[3]);
    const double* o4 = ob + qa + 3;
    double oo = 0.0;
    for (int k = 0; k < 4; ++k) oo += r[k] * in * o4[k];
    double rb[4];
    for (int k = 0; k < 4; ++k) rb[k] = in * (o4[k] - r[k] * in * oo);   // out = r / |r|
    // r = qq (x) e: qqbar = rb (x) conj(e), ebar = conj(qq) (x) rb
    double* qb4 = qbar + qa + 3;
    qb4[0] += rb[0] * e[0] + rb[1] * e[1] + rb[2] * e[2] + rb[3] * e[3];
    qb4[1] += -rb[0] * e[1] + rb[1] * e[0] - rb[2] * e[3] + rb[3] * e[2];
    qb4[2] += -rb[0] * e[2] + rb[1] * e[3] + rb[2] * e[0] - rb[3] * e[1];
    qb4[3] += -rb[0] * e[3] - rb[1] * e[2] + rb[2] * e[1] + rb[3] * e[0];
    double eb[4];
    eb[0] = qq[0] * rb[0] + qq[1] * rb[1] + qq[2] * rb[2] + qq[3] * rb[3];
    eb[1] = qq[0] * rb[1] - qq[1] * rb[0] - qq[2] * rb[3] + qq[3] * rb[2];
    eb[2] = qq[0] * rb[2] + qq[1] * rb[3] - qq[2] * rb[0] - qq[3] * rb[1];
    eb[3] = qq[0] * rb[3] - qq[1] * rb[2] + qq[2] * rb[1] - qq[3] * rb[0];
    // e = (cw(th2), sk(th2) d)
    const double th2b = eb[0] * dcw + (eb[1] * d[0] + eb[2] * d[1] + eb[3] * d[2]) * dsk;
    for (int k = 0; k < 3; ++k) dqbar[va + 3 + k] = sk * eb[1 + k] + 2.0 * th2b * d[k];
  }
  g.sync();
}

}  // namespace dmx
