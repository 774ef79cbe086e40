// Oracle model builder.  TEST INFRASTRUCTURE ONLY (see scalar.h).
#include "model.h"

#include <cmath>

#include "dynamics.h"

namespace orc {

thread_local std::int64_t g_flops = 0;
thread_local int g_flops_paused = 0;
thread_local int g_count_search = 1;
thread_local int g_pdir = -1;

static void normalize4(double* q) {
  double n = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3]);
  for (int i = 0; i < 4; ++i) q[i] /= n;
}
static void normalize3(double* a) {
  double n = std::sqrt(a[0] * a[0] + a[1] * a[1] + a[2] * a[2]);
  for (int i = 0; i < 3; ++i) a[i] /= n;
}

std::string build_model(Model& m, const double* body, int nbody, const double* geom, int ngeom,
                        const double* pair, int npair, const double* act, int nact,
                        const double* opt, const double* qpos0) {
  m = Model();
  for (int b = 0; b < nbody; ++b) {
    const double* r = body + 20 * b;
    Body B;
    B.parent = (int)r[0];
    B.jtype = (int)r[1];
    for (int i = 0; i < 3; ++i) { B.pos[i] = r[2 + i]; B.axis[i] = r[9 + i]; B.com[i] = r[13 + i]; B.inertia[i] = r[16 + i]; }
    for (int i = 0; i < 4; ++i) B.quat[i] = r[5 + i];
    B.mass = r[12];
    B.damping = r[19];
    if (B.parent >= b) return "body parent must precede the body";
    if (B.jtype == JNT_FREE && B.parent != -1) return "free joint only on a child of the world";
    if (B.jtype != JNT_FREE && B.jtype != JNT_HINGE) return "unknown joint type";
    normalize4(B.quat);
    if (B.jtype == JNT_HINGE) normalize3(B.axis);
    B.qadr = m.nq; B.vadr = m.nv;
    B.nq = B.jtype == JNT_FREE ? 7 : 1;
    B.nv = B.jtype == JNT_FREE ? 6 : 1;
    m.nq += B.nq; m.nv += B.nv;
    m.body.push_back(B);
  }
  for (int g = 0; g < ngeom; ++g) {
    const double* r = geom + 12 * g;
    Geom G;
    G.type = (int)r[0]; G.body = (int)r[1];
    for (int i = 0; i < 3; ++i) { G.pos[i] = r[2 + i]; G.size[i] = r[9 + i]; }
    for (int i = 0; i < 4; ++i) G.quat[i] = r[5 + i];
    if (G.body < 0 || G.body >= nbody) return "geom body out of range";
    normalize4(G.quat);
    if (G.type == GEOM_BOX) { G.box = (int)m.box_geom.size(); m.box_geom.push_back(g); }
    m.geom.push_back(G);
  }
  for (int b = 0; b < nbody; ++b) {
    int n = 0, last = -1;
    for (int g = 0; g < ngeom; ++g)
      if (m.geom[g].body == b) { ++n; last = g; }
    if (n == 1 && m.geom[last].type == GEOM_BOX) m.body[b].sole_box = m.geom[last].box;
  }
  int row = 0;
  for (int p = 0; p < npair; ++p) {
    const double* r = pair + 4 * p;
    Pair P;
    P.g1 = (int)r[0]; P.g2 = (int)r[1]; P.condim = (int)r[2]; P.mu = r[3];
    if (P.g1 < 0 || P.g1 >= ngeom || P.g2 >= ngeom) return "pair geom out of range";
    if (P.condim != 1 && P.condim != 3) return "condim must be 1 or 3";
    if (P.g2 >= 0) {
      const int t1 = m.geom[P.g1].type, t2 = m.geom[P.g2].type;
      const bool capbox = t1 == GEOM_CAPSULE && t2 == GEOM_BOX;
      const bool segseg = (t1 == GEOM_SPHERE || t1 == GEOM_CAPSULE) && (t2 == GEOM_SPHERE || t2 == GEOM_CAPSULE);
      if (!capbox && !segseg) return "geom pairs: capsule-box or sphere/capsule against sphere/capsule";
    }
    P.nslot = pair_slots(m, P);
    P.slot0 = m.nslot;
    P.row0 = row;
    m.nslot += P.nslot;
    row += P.nslot * (P.condim == 1 ? 1 : 4);
    m.pair.push_back(P);
  }
  m.nrowmax = row;
  for (int a = 0; a < nact; ++a) {
    const double* r = act + 5 * a;
    Act A;
    A.type = (int)r[0]; A.body = (int)r[1]; A.gear = r[2]; A.kp = r[3]; A.kd = r[4];
    if (A.body < 0 || A.body >= nbody || m.body[A.body].jtype != JNT_HINGE) return "actuator must drive a hinge";
    A.qadr = m.body[A.body].qadr; A.vadr = m.body[A.body].vadr;
    m.act.push_back(A);
  }
  m.nu = nact;
  for (int i = 0; i < 3; ++i) m.grav[i] = opt[i];
  m.solref[0] = opt[3]; m.solref[1] = opt[4];
  for (int i = 0; i < 5; ++i) { m.solimp[i] = opt[5 + i]; m.cfd[i] = opt[10 + i]; }
  m.softplus_s = opt[15];
  m.qpos0.assign(qpos0, qpos0 + m.nq);
  // ancestry and dof ownership
  m.anc.assign(nbody, std::vector<char>(nbody, 0));
  for (int b = 0; b < nbody; ++b)
    for (int j = b; j >= 0; j = m.body[j].parent) m.anc[b][j] = 1;
  m.dof_body.resize(m.nv);
  for (int b = 0; b < nbody; ++b)
    for (int d = 0; d < m.body[b].nv; ++d) m.dof_body[m.body[b].vadr + d] = b;
  // translational inverse weight of each body at qpos0: trace(Jc M^-1 Jc^T) / 3,
  // and its derivative with respect to every body mass (one derivative pass each)
  if (!body_inverse_weights(m, m.body_invw)) return "mass matrix at qpos0 is not positive definite";
  const int nmc = nbody + (int)m.box_geom.size();    // parameters M(q0) depends on: masses, box sides
  std::vector<std::vector<double>> dinv(nmc, std::vector<double>(nbody, 0.0));
  for (int c = 0; c < nmc; ++c) {
    g_pdir = par_mass(m, 0) + c;
    std::vector<Dual<double>> w;
    body_inverse_weights(m, w);
    for (int b = 0; b < nbody; ++b) dinv[c][b] = w[b].d;
  }
  g_pdir = -1;
  for (Pair& P : m.pair) {
    const int bA = m.geom[P.g1].body;
    const int bB = P.g2 >= 0 ? m.geom[P.g2].body : -1;
    P.invw = m.body_invw[bA] + (bB >= 0 ? m.body_invw[bB] : 0.0);
    P.dinvw.assign(nmc, 0.0);
    for (int c = 0; c < nmc; ++c) P.dinvw[c] = dinv[c][bA] + (bB >= 0 ? dinv[c][bB] : 0.0);
  }
  return "";
}

}  // namespace orc
