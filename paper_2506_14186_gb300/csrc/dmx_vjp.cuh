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
// Component e of d/dI (ybar . inertia_apply(I, x)) (the terms inertia_grad adds).
__device__ __forceinline__ double inertia_grad_comp(const double* yb, const double* x, int e) {
  const double w0 = x[0], w1 = x[1], w2 = x[2], v0 = x[3], v1 = x[4], v2 = x[5];
  switch (e) {
    case 0: return yb[3] * v0 + yb[4] * v1 + yb[5] * v2;
    case 1: return (v1 * yb[2] - v2 * yb[1]) - (w1 * yb[5] - w2 * yb[4]);
    case 2: return (v2 * yb[0] - v0 * yb[2]) - (w2 * yb[3] - w0 * yb[5]);
    case 3: return (v0 * yb[1] - v1 * yb[0]) - (w0 * yb[4] - w1 * yb[3]);
    case 4: return yb[0] * w0;
    case 5: return yb[1] * w1;
    case 6: return yb[2] * w2;
    case 7: return yb[0] * w1 + yb[1] * w0;
    case 8: return yb[0] * w2 + yb[2] * w0;
    default: return yb[1] * w2 + yb[2] * w1;
  }
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
// sv: the minimiser over the capsule axis that the forward evaluation found.
// VJP of seg_seg (dmx_device.cuh): cb = cotangents of (r, pos, n, t1, t2);
// b1 / b2 += pose cotangents (R 9, p 3) of geoms g1 / g2.  The free closest-
// point parameters follow the reduced optimality conditions
// F = (Du + s - c t, -Dv - c s + t) = 0: with lambda = A^-T (sbar, tbar),
// A = [[1, -c], [-c, 1]] restricted to the free ones, theta gets -lambda^T dF/dtheta.
static __device__ void seg_seg_vjp(const DevModel& m, const double* gR, const double* gp, int g1, int g2, double sv,
                                   double tv, const double* cb, double* b1, double* b2) {
  const double ra = m.g_size[g1][0];
  const double La = seg_half(m, g1), Lb = seg_half(m, g2);
  const double* R1 = gR + 9 * g1; const double* R2 = gR + 9 * g2;
  const double* c1 = gp + 3 * g1; const double* c2 = gp + 3 * g2;
  const double D[3] = {c1[0] - c2[0], c1[1] - c2[1], c1[2] - c2[2]};
  const double ua[3] = {R1[0], R1[3], R1[6]}, ub[3] = {R2[0], R2[3], R2[6]};
  double d[3], n[3];
  for (int i = 0; i < 3; ++i) d[i] = D[i] + sv * ua[i] - tv * ub[i];
  const double rho = ::sqrt(dot3(d, d));
  for (int i = 0; i < 3; ++i) n[i] = d[i] / rho;
  const double r = rho - (ra + m.g_size[g2][0]), off = ra + 0.5 * r;
  double ref[3] = {0, 0, 1};
  if (fabs(n[2]) >= 0.5) { ref[0] = 1; ref[2] = 0; }
  double t1r[3], t1[3];
  cross3(n, ref, t1r);
  const double il = rsqrt_t(dot3(t1r, t1r));
  for (int i = 0; i < 3; ++i) t1[i] = t1r[i] * il;
  // reverse: frame, position, distance
  double nb[3] = {cb[4], cb[5], cb[6]}, t1b[3] = {cb[7], cb[8], cb[9]};
  const double* t2b = cb + 10;
  const double* posb = cb + 1;
  acc_cross(t1, t2b, nb);                    // t2 = n x t1
  acc_cross(t2b, n, t1b);
  const double tt = dot3(t1, t1b);
  double t1rb[3];
  for (int i = 0; i < 3; ++i) t1rb[i] = il * (t1b[i] - t1[i] * tt);
  acc_cross(ref, t1rb, nb);                  // t1r = n x ref
  double c1b[3], uab[3], ubb[3] = {0, 0, 0}, Db[3];
  double sb = dot3(ua, posb), tb = 0.0;      // pos = c1 + s ua - off n
  for (int i = 0; i < 3; ++i) { c1b[i] = posb[i]; uab[i] = sv * posb[i]; nb[i] -= off * posb[i]; }
  const double rhob = cb[0] - 0.5 * dot3(n, posb);
  const double nn = dot3(nb, n);
  double db[3];
  for (int i = 0; i < 3; ++i) db[i] = (nb[i] - nn * n[i]) / rho + rhob * n[i];   // n = d / rho, rho = |d|
  for (int i = 0; i < 3; ++i) {             // d = D + s ua - t ub
    Db[i] = db[i];
    uab[i] += sv * db[i];
    ubb[i] -= tv * db[i];
  }
  sb += dot3(db, ua);
  tb -= dot3(db, ub);
  // implicit function of the free closest-point parameters
  const bool sf = fabs(sv) < La, tf = fabs(tv) < Lb;
  double ls = 0.0, lt = 0.0;
  const double c = dot3(ua, ub);
  if (sf && tf) {
    const double det = 1.0 - c * c;
    ls = (sb + c * tb) / det;
    lt = (tb + c * sb) / det;
  } else if (sf) {
    ls = sb;
  } else if (tf) {
    lt = tb;
  }
  if (sf || tf) {
    const double w = ls * tv + lt * sv;      // the c = ua . ub terms
    for (int i = 0; i < 3; ++i) {
      Db[i] += -ls * ua[i] + lt * ub[i];
      uab[i] += -ls * D[i] + w * ub[i];
      ubb[i] += lt * D[i] + w * ua[i];
    }
  }
  b1[0] += uab[0]; b1[3] += uab[1]; b1[6] += uab[2];   // u = first column of R
  b2[0] += ubb[0]; b2[3] += ubb[1]; b2[6] += ubb[2];
  for (int i = 0; i < 3; ++i) { b1[9 + i] += c1b[i] + Db[i]; b2[9 + i] -= Db[i]; }
}

static __device__ void capsule_box_vjp(const DevModel& m, const double* gR, const double* gp, int g1, int g2,
                                       double sv, const double* cb, double* b1, double* b2) {
  const double rc = m.g_size[g1][0], Lh = m.g_size[g1][1];
  const double* h = m.g_size[g2];
  const double* R1 = gR + 9 * g1; const double* R2 = gR + 9 * g2;
  const double* c1 = gp + 3 * g1; const double* c2 = gp + 3 * g2;
  const double dc[3] = {c1[0] - c2[0], c1[1] - c2[1], c1[2] - c2[2]};
  const double u[3] = {R1[0], R1[3], R1[6]};
  double y0[3], wv[3];
  matTvec3(R2, dc, y0);
  matTvec3(R2, u, wv);
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
__device__ __forceinline__ void slot_rows_bar(const DevModel& m, const WsB& b, int p, int r0, double yi, double yai,
                                              double* jb) {
  const LayoutBar& LB = *b.L;
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
}
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
  const double* ct = (w.xct ? w.xct : w.at(L.ct)) + 16 * s;
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
  const double* an = w.at(L.an); const double* J = w.xJ ? w.xJ : w.at(L.J); const double* Dr = w.at(L.Dr);
  const double* z = w.at(L.z); const double* CT = w.xct ? w.xct : w.at(L.ct);
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
      const int p = m.s_pair[s];
      const double* ct = CT + 16 * s;
      double pvb[3];
      if (m.p_g2[p] < 0) {
        // ground plane: frame (z, x, y) of the world, the dof moves the geom's body or nothing
        if (!((m.b_anc[m.g_body[m.p_g1[p]]] >> bi) & 1u)) continue;
        double jb[3];
        slot_rows_bar(m, b, p, r0, y[i], yai, jb);
        pvb[0] = jb[1]; pvb[1] = jb[2]; pvb[2] = jb[0];
      } else {
        double jb[3], pv[3], sg;
        if (!slot_jbar(m, w, b, s, r0, i, y[i], yai, jb, pv, &sg)) continue;
        for (int k = 0; k < 3; ++k) pvb[k] = sg * (jb[0] * ct[4 + k] + jb[1] * ct[7 + k] + jb[2] * ct[10 + k]);
      }
      acc_cross(ct + 1, pvb, sbi);      // pv = S_ang x pos + S_lin
      sbi[3] += pvb[0]; sbi[4] += pvb[1]; sbi[5] += pvb[2];
    }
  }
  // ---- per slot: record cotangents, impedance terms, contact geometry
  for (int s = g.lane; s < m.nslot; s += G) {
    const int r0 = slotrow[s];
    if (r0 < 0) continue;
    const double* ct = CT + 16 * s;
    double* sb = SB + m.s_barofs[s];
    const int p = m.s_pair[s];
    const int nrow = m.p_condim[p] == 1 ? 1 : 4;
    double cb[13] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
    if (m.p_g2[p] < 0) {
      // ground plane: the frame is fixed (no frame cotangents), pvb in the world frame
      const unsigned anc = m.b_anc[m.g_body[m.p_g1[p]]];
      for (int i = 0; i < nv; ++i) {
        if (!((anc >> m.dof_body[i]) & 1u)) continue;
        double jb[3];
        slot_rows_bar(m, b, p, r0, y[i], an[i] + m.bcoef * v[i], jb);
        const double pvb[3] = {jb[1], jb[2], jb[0]};
        acc_cross(pvb, S + 6 * i, cb + 1);   // pos cotangent from S_ang x pos
      }
    } else {
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
      const double* st = w.at(L.csv) + 2 * s;
      if (m.g_type[m.p_g2[p]] == GEOM_BOX) capsule_box_vjp(m, gR, gp, g1, m.p_g2[p], st[0], cb, b1, b2);
      else seg_seg_vjp(m, gR, gp, g1, m.p_g2[p], st[0], st[1], cb, b1, b2);
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
  // ---- per geom: pose cotangents gathered from its slots (one component per task)
  double* GB = b.at(LB.gb);
  for (int t = g.lane; t < 12 * m.ngeom; t += G) {
    const int gi = t / 12, c = t - 12 * gi;
    double acc = 0.0;
    for (int s = 0; s < m.nslot; ++s) {
      if (slotrow[s] < 0) continue;
      const int p = m.s_pair[s];
      if (m.p_g1[p] == gi) acc += SB[m.s_barofs[s] + c];
      else if (m.p_g2[p] == gi) acc += SB[m.s_barofs[s] + 12 + c];
    }
    GB[t] = acc;
  }
  g.sync();
  // ---- per body: geom poses -> body pose (gR = R_b Roff, gp = p_b + R_b gpos), one
  // entry per task; per dof and body component: bias-force (c_i = S_i . Fb) and
  // CRBA (F_i = Ic S_i) cotangents
  {
    const int n1 = 12 * nb, n2 = n1 + 6 * nv, n3 = n2 + 6 * nb, n4 = n3 + 10 * nb;
    for (int t = g.lane; t < n4; t += G) {
      if (t < n1) {
        const int bb = t / 12, c = t - 12 * bb;
        double acc = 0.0;
        for (int gi = 0; gi < m.ngeom; ++gi) {
          if (m.g_body[gi] != bb) continue;
          const double* gb = GB + 12 * gi;
          if (c < 9) {
            const int i = c / 3, j = c - 3 * (c / 3);
            const double* Ro = m.g_Roff[gi];
            acc += gb[3 * i] * Ro[3 * j] + gb[3 * i + 1] * Ro[3 * j + 1] + gb[3 * i + 2] * Ro[3 * j + 2] +
                   gb[9 + i] * m.g_pos[gi][j];
          } else {
            acc += gb[c];
          }
        }
        if (c < 9) Rb[9 * bb + c] += acc; else pb[3 * bb + c - 9] += acc;
      } else if (t < n2) {
        const int k = t - n1, i = k / 6, e = k - 6 * (k / 6);
        Sb[6 * i + e] += inertia_comp(Ic + 10 * m.dof_body[i], Fd + 6 * i, e);
      } else if (t < n3) {
        const int k = t - n2, bb = k / 6, e = k - 6 * (k / 6);
        double acc = 0.0;
        for (int d = 0; d < m.b_nv[bb]; ++d) { const int i = m.b_vadr[bb] + d; acc += y[i] * S[6 * i + e]; }
        Fbb[6 * bb + e] -= acc;
      } else {
        const int k = t - n3, bb = k / 10, e = k - 10 * (k / 10);
        double acc = 0.0;
        for (int d = 0; d < m.b_nv[bb]; ++d) {
          const int i = m.b_vadr[bb] + d;
          acc += inertia_grad_comp(Fd + 6 * i, S + 6 * i, e);
        }
        Icb[10 * bb + e] += acc;
      }
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
  // F's cotangent -> A, V (own terms), one body component per task:
  //   f1 = I A:          Abar = I fbar,  Ibar += grad(fbar, A)
  //   f2 = V x* (I V):   Vbar and (I V)bar from the force cross product, then
  //                      Vbar += I (I V)bar,  Ibar += grad((I V)bar, V)
  double* IV = b.at(LB.iv); double* IVB = b.at(LB.ivb);
  for (int t = g.lane; t < 6 * nb; t += G) {
    const int bb = t / 6, e = t - 6 * (t / 6);
    const double* I = Ib + 10 * bb;
    Abb[t] = inertia_comp(I, Fbb + 6 * bb, e);
    IV[t] = inertia_comp(I, V + 6 * bb, e);
  }
  g.sync();
  for (int t = g.lane; t < 6 * nb; t += G) {
    const int bb = t / 6, e = t - 6 * (t / 6);
    const double* a = V + 6 * bb; const double* iv = IV + 6 * bb; const double* fbar = Fbb + 6 * bb;
    const int k = e < 3 ? e : e - 3, k1 = nxt3(k), k2 = prv3(k);
    // c = a x* iv with a = (w; v), iv = (n; f): c_n = w x n + v x f, c_f = w x f
    double vb_e, ivb_e;
    if (e < 3) {
      vb_e = (iv[k1] * fbar[k2] - iv[k2] * fbar[k1]) + (iv[3 + k1] * fbar[3 + k2] - iv[3 + k2] * fbar[3 + k1]);
      ivb_e = fbar[k1] * a[k2] - fbar[k2] * a[k1];
    } else {
      vb_e = iv[3 + k1] * fbar[k2] - iv[3 + k2] * fbar[k1];
      ivb_e = (fbar[k1] * a[3 + k2] - fbar[k2] * a[3 + k1]) + (fbar[3 + k1] * a[k2] - fbar[3 + k2] * a[k1]);
    }
    Vbb[t] = vb_e;
    IVB[t] = ivb_e;
  }
  g.sync();
  for (int t = g.lane; t < 16 * nb; t += G) {
    if (t < 6 * nb) {
      const int bb = t / 6, e = t - 6 * (t / 6);
      Vbb[t] += inertia_comp(Ib + 10 * bb, IVB + 6 * bb, e);
    } else {
      const int k = t - 6 * nb, bb = k / 10, e = k - 10 * (k / 10);
      Ibb[10 * bb + e] += inertia_grad_comp(Fbb + 6 * bb, A + 6 * bb, e) + inertia_grad_comp(IVB + 6 * bb, V + 6 * bb, e);
    }
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
  // A's own term (V x S_d) v_d (d past the free joint's translations):
  //   vbar_d += Abar . (V x S_d);  with cb = Abar v_d:  Vbar_w += S_w x cb_w + S_v x cb_v,
  //   Vbar_v += S_w x cb_v;  Sbar_w += cb_w x V_w + cb_v x V_v,  Sbar_v += cb_v x V_w
  {
    const int n1 = nv, n2 = n1 + 6 * nv, n3 = n2 + 6 * nb;
    for (int t = g.lane; t < n3; t += G) {
      if (t < n1) {
        const int i = t, bb = m.dof_body[i];
        if (m.b_jtype[bb] == JNT_FREE && i - m.b_vadr[bb] < 3) continue;
        const double* vbv = V + 6 * bb; const double* sd = S + 6 * i; const double* ab6 = Abb + 6 * bb;
        double s1 = 0.0;
        for (int e = 0; e < 6; ++e) s1 += ab6[e] * crm_comp(vbv, sd, e);
        vb[i] += s1;
      } else if (t < n2) {
        const int k = t - n1, i = k / 6, e = k - 6 * (k / 6), bb = m.dof_body[i];
        if (m.b_jtype[bb] == JNT_FREE && i - m.b_vadr[bb] < 3) continue;
        const double* a = V + 6 * bb; const double* ab6 = Abb + 6 * bb;
        const double vd = v[i];
        const int c = e < 3 ? e : e - 3, c1 = nxt3(c), c2 = prv3(c);
        double r;
        if (e < 3)
          r = vd * ((ab6[c1] * a[c2] - ab6[c2] * a[c1]) + (ab6[3 + c1] * a[3 + c2] - ab6[3 + c2] * a[3 + c1]));
        else
          r = vd * (ab6[3 + c1] * a[c2] - ab6[3 + c2] * a[c1]);
        Sb[6 * i + e] += r;
      } else {
        const int k = t - n2, bb = k / 6, e = k - 6 * (k / 6);
        const double* ab6 = Abb + 6 * bb;
        const int c = e < 3 ? e : e - 3, c1 = nxt3(c), c2 = prv3(c);
        const int va = m.b_vadr[bb], nd = m.b_nv[bb];
        const int d0 = (m.b_jtype[bb] == JNT_FREE) ? 3 : 0;
        double acc = 0.0;
        for (int d = d0; d < nd; ++d) {
          const double* sd = S + 6 * (va + d);
          const double vd = v[va + d];
          if (e < 3)
            acc += vd * ((sd[c1] * ab6[c2] - sd[c2] * ab6[c1]) + (sd[3 + c1] * ab6[3 + c2] - sd[3 + c2] * ab6[3 + c1]));
          else
            acc += vd * (sd[c1] * ab6[3 + c2] - sd[c2] * ab6[3 + c1]);
        }
        Vbb[6 * bb + e] += acc;
      }
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
  // V's own term S_d v_d: vbar_d += Vbar . S_d, Sbar_d += Vbar v_d (per dof, per dof component)
  for (int t = g.lane; t < 7 * nv; t += G) {
    if (t < nv) {
      const int i = t;
      const double* vbar6 = Vbb + 6 * m.dof_body[i]; const double* sd = S + 6 * i;
      double s1 = 0.0;
      for (int e = 0; e < 6; ++e) s1 += vbar6[e] * sd[e];
      vb[i] += s1;
    } else {
      const int k = t - nv, i = k / 6, e = k - 6 * (k / 6);
      Sb[6 * i + e] += Vbb[6 * m.dof_body[i] + e] * v[i];
    }
  }
  g.sync();
  // actuators: motor tau += gear u; position servo tau += kp (u - q) - kd v
  if (g.lane == 0) {
    for (int a = 0; a < m.nact; ++a) {
      const int vi = m.a_vadr[a];
      if (m.a_type[a] == ACT_MOTOR) ub[a] += m.a_gear[a] * y[vi];
      else { ub[a] += m.a_kp[a] * y[vi]; qb[m.a_qadr[a]] -= m.a_kp[a] * y[vi]; vb[vi] -= m.a_kd[a] * y[vi]; }
    }
  }
  // ---- kinematics (forward: local rotation Rl = Roff Rj(theta) or the free joint's
  // pose; R = R_parent Rl, p = p_parent + R_parent b_pos; then COMs, inertias,
  // motion vectors and geoms from (R, p)).  Own terms of every body first, split
  // into tasks: per body the hinge's sine and cosine and the COM cotangent
  // (spatial inertia (m, m c, R diag(In) R^T + m (|c|^2 - c c^T)) -> c); then
  // one pose entry per task (inertia, COM and motion-vector terms) and one
  // local-rotation entry per task for the composition.
  double* SCb = b.at(LB.sc); double* TK = b.at(LB.tk);
  for (int t = g.lane; t < 4 * nb; t += G) {
    if (t < nb) {
      if (m.b_jtype[t] == JNT_HINGE) ::sincos(q[m.b_qadr[t]], &SCb[2 * t], &SCb[2 * t + 1]);
    } else {
      const int k = t - nb, bb = k / 3, r = k - 3 * (k / 3);
      const double ms = m.b_mass[bb];
      const double* ib = Ibb + 10 * bb; const double* c = C + 3 * bb;
      // Ibar as a symmetric matrix B (diagonal ib[4..6], (0,1) ib[7], (0,2) ib[8], (1,2) ib[9])
      const double Br[3] = {r == 0 ? 2.0 * ib[4] : (r == 1 ? ib[7] : ib[8]),
                            r == 0 ? ib[7] : (r == 1 ? 2.0 * ib[5] : ib[9]),
                            r == 0 ? ib[8] : (r == 1 ? ib[9] : 2.0 * ib[6])};
      const double tr = ib[4] + ib[5] + ib[6];
      cp[k] = ms * (ib[1 + r] + 2.0 * c[r] * tr - (Br[0] * c[0] + Br[1] * c[1] + Br[2] * c[2]));
    }
  }
  g.sync();
  for (int t = g.lane; t < 21 * nb; t += G) {
    if (t < 12 * nb) {
      const int bb = t / 12, comp = t - 12 * (t / 12);
      const double* Rv = R + 9 * bb; const double* pv = P + 3 * bb;
      const double* cb3 = cp + 3 * bb;
      const int va = m.b_vadr[bb];
      const bool fr = m.b_jtype[bb] == JNT_FREE;
      if (comp < 9) {
        const int r = comp / 3, kk = comp - 3 * (comp / 3);
        const double* ib = Ibb + 10 * bb;
        const double Br[3] = {r == 0 ? 2.0 * ib[4] : (r == 1 ? ib[7] : ib[8]),
                              r == 0 ? ib[7] : (r == 1 ? 2.0 * ib[5] : ib[9]),
                              r == 0 ? ib[8] : (r == 1 ? ib[9] : 2.0 * ib[6])};
        double val = m.b_inertia[bb][kk] * (Br[0] * Rv[kk] + Br[1] * Rv[3 + kk] + Br[2] * Rv[6 + kk]);
        val += cb3[r] * m.b_com[bb][kk];
        // motion vectors: free angular dof kk = column kk of R (lin = p x col);
        // hinge: sh = R axis (lin = p x sh)
        const double* sbd = Sb + 6 * (fr ? va + 3 + kk : va);
        const int r1 = nxt3(r), r2 = prv3(r);
        const double wb = sbd[r] + (sbd[3 + r1] * pv[r2] - sbd[3 + r2] * pv[r1]);
        val += fr ? wb : wb * m.b_axis[bb][kk];
        Rb[9 * bb + comp] += val;
      } else {
        const int r = comp - 9, r1 = nxt3(r), r2 = prv3(r);
        double val = cb3[r];
        if (fr) {
          for (int d = 0; d < 3; ++d) {
            const double* sv = Sb + 6 * (va + 3 + d) + 3;
            val += Rv[3 * r1 + d] * sv[r2] - Rv[3 * r2 + d] * sv[r1];
          }
        } else {
          const double* sv = Sb + 6 * va + 3;
          const double* ax = m.b_axis[bb];
          const double sh1 = Rv[3 * r1] * ax[0] + Rv[3 * r1 + 1] * ax[1] + Rv[3 * r1 + 2] * ax[2];
          const double sh2 = Rv[3 * r2] * ax[0] + Rv[3 * r2 + 1] * ax[1] + Rv[3 * r2 + 2] * ax[2];
          val += sh1 * sv[r2] - sh2 * sv[r1];
        }
        pb[3 * bb + r] += val;
      }
    } else {
      const int k = t - 12 * nb, bb = k / 9, e = k - 9 * (k / 9);
      if (m.b_jtype[bb] != JNT_HINGE) continue;
      const int i = e / 3, j = e - 3 * (e / 3);
      const double sn = SCb[2 * bb], cs = SCb[2 * bb + 1];
      const double* ax = m.b_axis[bb];
      double val;
      if (m.b_ident[bb]) {
        val = hinge_entry(ax, sn, cs, i, j);
      } else {
        const double* Ro = m.b_Roff[bb];
        val = Ro[3 * i] * hinge_entry(ax, sn, cs, 0, j) + Ro[3 * i + 1] * hinge_entry(ax, sn, cs, 1, j) +
              Ro[3 * i + 2] * hinge_entry(ax, sn, cs, 2, j);
      }
      cR[9 * bb + e] = val;
    }
  }
  g.sync();
  // composition, leaves to root: R_parent gets Rbar Rl^T + pbar b_pos^T, p_parent gets pbar
  // (one parent entry per task)
  for (int lev = m.nlevel - 1; lev >= 1; --lev) {
    for (int t = 12 * m.level_start[lev - 1] + g.lane; t < 12 * m.level_start[lev]; t += G) {
      const int kb = t / 12, comp = t - 12 * (t / 12);
      const int bb = m.level_list[kb];
      double acc = 0.0;
      for (int c = 0; c < m.child_count[bb]; ++c) {
        const int ch = m.child_list[m.child_start[bb] + c];
        if (m.b_jtype[ch] == JNT_FREE) continue;
        const double* rc = Rb + 9 * ch; const double* pc = pb + 3 * ch;
        if (comp < 9) {
          const int i = comp / 3, j = comp - 3 * (comp / 3);
          const double* Rl = cR + 9 * ch;
          acc += rc[3 * i] * Rl[3 * j] + rc[3 * i + 1] * Rl[3 * j + 1] + rc[3 * i + 2] * Rl[3 * j + 2] +
                 pc[i] * m.b_pos[ch][j];
        } else {
          acc += pc[comp - 9];
        }
      }
      if (comp < 9) Rb[9 * bb + comp] += acc; else pb[3 * bb + comp - 9] += acc;
    }
    g.sync();
  }
  // joint coordinates: free joints (translation, quaternion), one task per body;
  // hinges: theta bar = <Roff^T R_parent^T Rbar, dRj/dtheta>, one entry per task
  for (int t = g.lane; t < 10 * nb; t += G) {
    if (t < nb) {
      const int bb = t;
      if (m.b_jtype[bb] != JNT_FREE) continue;
      const double* rb = Rb + 9 * bb; const double* pbv = pb + 3 * bb;
      const int qa = m.b_qadr[bb];
      qb[qa] += pbv[0]; qb[qa + 1] += pbv[1]; qb[qa + 2] += pbv[2];
      quat_to_mat_vjp(q + qa + 3, rb, qb + qa + 3);
    } else {
      const int k = t - nb, bb = k / 9, e = k - 9 * (k / 9);
      if (m.b_jtype[bb] != JNT_HINGE) continue;
      const int i = e / 3, j = e - 3 * (e / 3);
      const double* rb = Rb + 9 * bb;
      const int par = m.b_parent[bb];
      double rl[3];   // column j of R_parent^T Rbar
      for (int kk = 0; kk < 3; ++kk)
        rl[kk] = par >= 0 ? R[9 * par + kk] * rb[j] + R[9 * par + 3 + kk] * rb[3 + j] + R[9 * par + 6 + kk] * rb[6 + j]
                          : rb[3 * kk + j];
      const double* Ro = m.b_Roff[bb];
      const double rjb = Ro[i] * rl[0] + Ro[3 + i] * rl[1] + Ro[6 + i] * rl[2];
      // dRj/dtheta (i, j) = sin (a_i a_j - delta_ij) + cos K_ij, K = [a]x
      const double* ax = m.b_axis[bb];
      const double sn = SCb[2 * bb], cs = SCb[2 * bb + 1];
      double dr = sn * ax[i] * ax[j];
      if (i == j) dr -= sn;
      else dr += (j == nxt3(i)) ? -cs * ax[3 - i - j] : cs * ax[3 - i - j];
      TK[k] = rjb * dr;
    }
  }
  g.sync();
  for (int bb = g.lane; bb < nb; bb += G) {
    if (m.b_jtype[bb] != JNT_HINGE) continue;
    const double* tk = TK + 9 * bb;
    qb[m.b_qadr[bb]] += (((tk[0] + tk[1]) + (tk[2] + tk[3])) + ((tk[4] + tk[5]) + (tk[6] + tk[7]))) + tk[8];
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
