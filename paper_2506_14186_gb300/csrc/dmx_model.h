// Compiled model and per-environment workspace layout, shared by the host
// runtime (which fills them) and the device kernels (which read them).
#pragma once
#include <cstdint>

#ifdef __CUDACC__
#define DMX_HD __host__ __device__
#else
#define DMX_HD
#endif

namespace dmx {

// Capacity limits of the compiled model (checked by dmx_create_model).
constexpr int MAXB = 16;      // bodies
constexpr int MAXV = 24;      // dofs
constexpr int MAXQ = 32;      // position coordinates
constexpr int MAXG = 24;      // geoms
constexpr int MAXBOX = 4;     // box geoms (side-length parameters)
constexpr int MAXP = 24;      // contact pairs
constexpr int MAXS = 32;      // contact slots
constexpr int MAXU = 16;      // actuators
constexpr int MAXROWID = 128; // constraint rows over all slots (stable row ids)
// Constraint rows one right-hand side can hold (the included contacts' rows,
// compacted): the Jacobian and row arrays of the per-environment workspace
// are sized min(row ids, ROWCAP), which keeps shared memory per environment,
// hence warps per SM, independent of how many slots a model declares; a state
// with more included rows reports ENV_ROW_OVERFLOW.
constexpr int ROWCAP = 64;
constexpr int MAXLEV = 12;    // depth of the body tree
constexpr int MASKW = MAXROWID / 32;

enum { JNT_FREE = 0, JNT_HINGE = 1 };
enum { GEOM_SPHERE = 0, GEOM_CAPSULE = 1, GEOM_BOX = 2 };
enum { ACT_MOTOR = 0, ACT_POSITION = 1 };
// Model parameters the adjoint differentiates (dmx_rollout_grad_params): solref
// (t_c, phi_d), solimp (d_o, d_w, width, midpoint), then the friction
// coefficient of every pair.
enum { PAR_TC = 0, PAR_DAMP = 1, PAR_DO = 2, PAR_DW = 3, PAR_WIDTH = 4, PAR_MID = 5, PAR_MU0 = 6 };
enum { ENV_OK = 0, ENV_MAX_STEPS = 1, ENV_H_UNDERFLOW = 2, ENV_NONFINITE = 3, ENV_SOLVER_NOCONV = 4,
       ENV_ROW_OVERFLOW = 5 };

struct DevModel {
  int nbody, ngeom, npair, nact, nq, nv, nu, nslot, nrowid, nlevel;
  double grav[3];
  double bcoef, kcoef;               // a_ref = -bcoef (J v) - kcoef d(r) r
  double solref[2];                  // t_c, phi_d (bcoef = 2 / (d_w t_c), kcoef = 1 / (d_w^2 t_c^2 phi_d^2))
  double solimp[5];                  // d_o, d_w, width, midpoint, power
  double cfd[5];                     // d_c, d_0, w_c, m_c, p_c
  double softplus;
  // bodies (topological order)
  int b_parent[MAXB], b_jtype[MAXB], b_qadr[MAXB], b_vadr[MAXB], b_nv[MAXB];
  unsigned b_anc[MAXB];              // bit j: body j is this body or an ancestor
  double b_pos[MAXB][3], b_Roff[MAXB][9], b_axis[MAXB][3];
  double b_mass[MAXB], b_com[MAXB][3], b_inertia[MAXB][3], b_damping[MAXB];
  int b_ident[MAXB];                 // 1: b_Roff is exactly the identity
  int child_start[MAXB], child_count[MAXB], child_list[MAXB];
  int level_start[MAXLEV + 1], level_list[MAXB];
  int dof_body[MAXV];
  // geoms
  int g_type[MAXG], g_body[MAXG];
  double g_pos[MAXG][3], g_Roff[MAXG][9], g_size[MAXG][3];
  double g_bound[MAXG];              // bounding-sphere radius about the geom centre
  int g_box[MAXG];                   // index among the box geoms (side-length parameter), else -1
  int nbox;
  int b_solebox[MAXB];               // geom index of the body's only geom when it is a box (its inertia follows the side), else -1
  int g_ident[MAXG], g_zpos[MAXG];   // 1: g_Roff is exactly the identity / g_pos is exactly zero
  // pairs and slots
  int p_g1[MAXP], p_g2[MAXP], p_condim[MAXP], p_slot0[MAXP], p_nslot[MAXP], p_row0[MAXP];
  double p_mu[MAXP], p_ahat[MAXP], p_ahat_edge[MAXP];
  double p_dahat[MAXP][MAXB + MAXBOX];   // d A_hat / d (mass of each body, then side of each box)
  int s_pair[MAXS], s_idx[MAXS];
  int s_barofs[MAXS], nslotbar;      // adjoint: offset / total of the per-slot pose cotangents
                                     // (12 doubles for a plane slot, 24 for a geom pair)
  // actuators
  int a_type[MAXU], a_qadr[MAXU], a_vadr[MAXU];
  double a_gear[MAXU], a_kp[MAXU], a_kd[MAXU];
};

// Offsets (in doubles / ints) of one environment's shared-memory workspace.
struct Layout {
  int qn, vn, qs, vs, kv, ka, dq;
  int R, p, com, sd, Ib, Ic, F, Vb, Ab, Fb, iv, gR, gp;
  int M, H, rhs0, a, an, tmp, tmp2;
  int ct, csv, J, aref, Dr, z, s, u;   // csv: closest-point parameters of each geom-pair slot (2 per slot)
  int nd;                            // doubles per environment (padded to even)
  int xl, sc;                        // kinematics scratch, aliases of Ab..Fb (12 per body) and iv (2 per body)
  int rowid, slotrow, slist, amask, pmask, misc;
  int sinc, rowslot, alist;          // slot included (0/1), slot of each row, compacted active rows
  int ni;                            // ints per environment
  int rcap;                          // constraint-row capacity
  int xbar;                          // adjoint layout: state cotangent (nq + nv), else -1
  int ovl;                           // adjoint layout: start of the arrays the VJP never reads, else nd
};

DMX_HD inline Layout make_layout(const DevModel& m, int rcap) {
  Layout L{};
  int o = 0;
  const int nq = m.nq, nv = m.nv, nb = m.nbody, ng = m.ngeom, ns = m.nslot > 0 ? m.nslot : 1;
  auto take = [&](int n) { int r = o; o += n; return r; };
  L.qn = take(nq); L.vn = take(nv); L.qs = take(nq); L.vs = take(nv);
  L.kv = take(7 * nv); L.ka = take(7 * nv); L.dq = take(nv);
  L.R = take(9 * nb); L.p = take(3 * nb); L.com = take(3 * nb); L.sd = take(6 * nv);
  L.Ib = take(10 * nb); L.Ic = take(10 * nb); L.F = take(6 * nv);
  L.Vb = take(6 * nb); L.Ab = take(6 * nb); L.Fb = take(6 * nb); L.iv = take(6 * nb);
  // the bias-force arrays are free while the kinematics run: local transforms
  // (Ab and Fb are contiguous, 12 per body) and per-body scalars (iv)
  L.xl = L.Ab; L.sc = L.iv;
  L.gR = take(9 * ng); L.gp = take(3 * ng);
  L.M = take(nv * nv); L.H = take(nv * nv);
  L.rhs0 = take(nv); L.a = take(nv); L.an = take(nv); L.tmp = take(nv); L.tmp2 = take(nv);
  L.ct = take(16 * ns); L.csv = take(2 * ns);
  L.J = take(rcap * nv); L.aref = take(rcap); L.Dr = take(rcap); L.z = take(rcap); L.s = take(rcap);
  L.u = take(m.nu > 0 ? m.nu : 1);
  L.nd = (o + 1) & ~1;
  int i = 0;
  auto takei = [&](int n) { int r = i; i += n; return r; };
  L.rowid = takei(rcap); L.slotrow = takei(ns + 1); L.slist = takei(ns); L.amask = takei(MASKW);
  L.pmask = takei(MASKW);
  L.misc = takei(8);
  L.sinc = takei(ns); L.rowslot = takei(rcap); L.alist = takei(rcap);
  L.ni = (i + 3) & ~3;
  L.rcap = rcap;
  L.xbar = -1;
  L.ovl = L.nd;
  return L;
}

// Workspace of the reverse adjoint kernel when it restores stage snapshots:
// the same arrays, ordered so that everything the right-hand-side VJP reads
// (poses .. geom frames, the final Newton factor and solution, capsule-box
// minimisers, D and the residuals of the rows, controls) and the running
// state cotangent come first, and the arrays only the segment recompute uses
// (stage state, M, contact records, Jacobian rows, a_ref, line-search slopes)
// start at ovl.  During the reverse sweep the cotangent workspace occupies
// [ovl, ...): the VJP reads the contact records and Jacobian rows from the
// snapshot in device memory instead.
DMX_HD inline Layout make_layout_adj(const DevModel& m, int rcap) {
  Layout L = make_layout(m, rcap);
  int o = 0;
  const int nq = m.nq, nv = m.nv, nb = m.nbody, ng = m.ngeom, ns = m.nslot > 0 ? m.nslot : 1;
  auto take = [&](int n) { int r = o; o += n; return r; };
  L.R = take(9 * nb); L.p = take(3 * nb); L.com = take(3 * nb); L.sd = take(6 * nv);
  L.Ib = take(10 * nb); L.Ic = take(10 * nb); L.F = take(6 * nv);
  L.Vb = take(6 * nb); L.Ab = take(6 * nb); L.Fb = take(6 * nb); L.iv = take(6 * nb);
  L.xl = L.Ab; L.sc = L.iv;
  L.gR = take(9 * ng); L.gp = take(3 * ng);
  L.H = take(nv * nv);
  L.rhs0 = take(nv); L.a = take(nv); L.an = take(nv); L.tmp = take(nv); L.tmp2 = take(nv);
  L.csv = take(2 * ns); L.Dr = take(rcap); L.z = take(rcap);
  L.u = take(m.nu > 0 ? m.nu : 1);
  L.xbar = take(nq + nv);
  L.ovl = o;
  L.qn = take(nq); L.vn = take(nv); L.qs = take(nq); L.vs = take(nv);
  L.kv = take(7 * nv); L.ka = take(7 * nv); L.dq = take(nv);
  L.M = take(nv * nv);
  L.ct = take(16 * ns);
  L.J = take(rcap * nv); L.aref = take(rcap); L.s = take(rcap);
  L.nd = (o + 1) & ~1;
  return L;
}

// Offsets (in doubles) of one environment's adjoint workspace (reverse-mode
// adjoint kernel): cotangents of the right-hand side's intermediates, then
// the stage data and cotangents of one Dormand-Prince step.
struct LayoutBar {
  int R, p, cR, cp, S, F, Ib, Ic, V, A, Fb, slot, y, jy, cz, cj, q, v, u;   // right-hand side
  int gb, iv, ivb;                   // geom pose cotangents, I V and its cotangent per body
  int sc, tk;                        // hinge sine and cosine, theta-cotangent terms per body
  int qn, vst, dq, dqb, Qs, kab, kvb, Qb, Vb, qnb, vnb, ub, xb;            // one step
  int nd;                            // doubles per environment (padded to even)
};
constexpr int SLOTBAR = 24;          // at most per slot: pose cotangents of its two geoms (R 9 + p 3 each)

DMX_HD inline LayoutBar make_bar_layout(const DevModel& m, int rcap) {
  LayoutBar B{};
  int o = 0;
  const int nq = m.nq, nv = m.nv, nb = m.nbody, ns = m.nslot > 0 ? m.nslot : 1, nu = m.nu > 0 ? m.nu : 1;
  auto take = [&](int n) { int r = o; o += n; return r; };
  B.R = take(9 * nb); B.p = take(3 * nb); B.cR = take(9 * nb); B.cp = take(3 * nb);
  B.S = take(6 * nv); B.F = take(6 * nv); B.Ib = take(10 * nb); B.Ic = take(10 * nb);
  B.V = take(6 * nb); B.A = take(6 * nb); B.Fb = take(6 * nb);
  B.slot = take(m.nslotbar > 0 ? m.nslotbar : SLOTBAR * ns);
  B.y = take(nv); B.jy = take(rcap); B.cz = take(rcap); B.cj = take(rcap);
  B.q = take(nq); B.v = take(nv); B.u = take(nu);
  B.gb = take(12 * (m.ngeom > 0 ? m.ngeom : 1)); B.iv = take(6 * nb); B.ivb = take(6 * nb);
  B.sc = take(2 * nb); B.tk = take(9 * nb);
  B.qn = take(nq); B.vst = take(7 * nv); B.dq = take(nv); B.dqb = take(nv); B.Qs = take(nq);
  B.kab = take(6 * nv); B.kvb = take(6 * nv); B.Qb = take(nq); B.Vb = take(nv);
  B.qnb = take(nq); B.vnb = take(nv); B.ub = take(nu); B.xb = take(nq + nv);
  B.nd = (o + 1) & ~1;
  return B;
}

}  // namespace dmx
