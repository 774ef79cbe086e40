// Oracle model: a tree of rigid bodies with free and hinge joints, sphere /
// capsule / box geoms, contact pairs against the ground plane z = 0 (and
// capsule-box pairs), motor and PD actuators, and the soft-contact parameters
// solref / solimp / solimp-CFD of the paper (Sec. 2.1, Sec. 4).
//
// TEST INFRASTRUCTURE ONLY (see scalar.h).
//
// The model arrives as flat double records (layouts below), so the oracle
// shares no header or struct with the CUDA path.
//   body  (20): parent, jnt_type(0 free, 1 hinge), pos[3], quat[4], axis[3],
//               mass, com[3], inertia[3] (principal, body axes), damping
//   geom  (12): type(0 sphere, 1 capsule, 2 box), body, pos[3], quat[4], size[3]
//   pair   (4): geom1, geom2 (-1 = plane), condim (1 or 3), mu
//   act    (5): type(0 motor, 1 position servo), body (hinge), gear, kp, kd
//   opt   (16): gravity[3], solref[2], solimp[5], solimp_cfd[5], softplus width
#pragma once
#include <cmath>
#include <string>
#include <vector>

namespace orc {

enum { JNT_FREE = 0, JNT_HINGE = 1 };
enum { GEOM_SPHERE = 0, GEOM_CAPSULE = 1, GEOM_BOX = 2 };
enum { ACT_MOTOR = 0, ACT_POSITION = 1 };
enum { ENV_OK = 0, ENV_MAX_STEPS = 1, ENV_H_UNDERFLOW = 2, ENV_NONFINITE = 3, ENV_SOLVER_NOCONV = 4 };

struct Body {
  int parent, jtype;
  double pos[3], quat[4], axis[3], mass, com[3], inertia[3], damping;
  int qadr, vadr, nq, nv;
  int sole_box = -1;        // the body's only geom is box geom number sole_box (its inertia follows the size)
};
struct Geom {
  int type, body;
  int box = -1;             // index among the model's box geoms (side-length parameter), else -1
  double pos[3], quat[4], size[3];
};
struct Pair {
  int g1, g2, condim;
  double mu;
  int nslot, slot0, row0;   // contact slots and first constraint row of this pair
  double invw;              // approximate diag(J M^-1 J^T) for the normal row
  std::vector<double> dinvw; // its derivative w.r.t. the mass of each body, then the side of each box
};
struct Act {
  int type, body;
  double gear, kp, kd;
  int qadr, vadr;
};

struct Model {
  std::vector<Body> body;
  std::vector<Geom> geom;
  std::vector<Pair> pair;
  std::vector<Act> act;
  int nq = 0, nv = 0, nu = 0, nslot = 0, nrowmax = 0;
  double grav[3];
  double solref[2];      // time constant t_c, damping ratio phi_d
  double solimp[5];      // d_o, d_w, width, midpoint, power
  double cfd[5];         // d_c, d_0, w_c, m_c, p_c
  double softplus_s;     // width of the softplus that replaces the ReLU in a_ref (CFD)
  std::vector<double> qpos0;
  std::vector<std::vector<char>> anc;   // anc[b][j]: body j is b or an ancestor of b
  std::vector<int> dof_body;            // body owning each dof
  std::vector<double> body_invw;        // translational inverse weight at qpos0
  std::vector<int> box_geom;            // geom index of every box geom
};

// Builds the model; returns "" on success or an error message.
std::string build_model(Model& m, const double* body, int nbody, const double* geom, int ngeom,
                        const double* pair, int npair, const double* act, int nact,
                        const double* opt, const double* qpos0);

inline int pair_slots(const Model& m, const Pair& p) {
  const int t1 = m.geom[p.g1].type;
  if (p.g2 < 0) return t1 == GEOM_SPHERE ? 1 : t1 == GEOM_CAPSULE ? 2 : 8;
  return 1;   // capsule-box
}

}  // namespace orc
