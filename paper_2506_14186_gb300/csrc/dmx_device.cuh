// Device code of the forward dynamics v' = F(q, v, u) and of one adaptive
// Dormand-Prince attempt, for one environment handled by a group of G lanes
// of a warp (G = 1, 2, 4, 8, 16, 32).  Every per-environment array lives in
// shared memory; the G lanes split loops over bodies, dofs, contact slots,
// constraint rows and matrix entries, and meet at __syncwarp(group mask).
//
// Method (arXiv 2506.14186):
//   Sec. 2, Eq. (EOM)       v' = M^-1 (tau - c + J^T f); M by the composite-
//                           rigid-body algorithm, c by recursive Newton-Euler
//                           (world-frame spatial vectors, Featherstone)
//   Sec. 2.1                signed distances r (active iff r < 0), pyramidal
//                           rows, a_ref = -b (J v) - k d(r) r, impedance d(r)
//                           (solimp spline), R = A_hat (1 - d) / d, and the
//                           relaxed Gauss principle solved by exact Newton
//   App. C.1                plane-box from the box vertices, pos = v - r/2 n
//   Sec. 4                  contacts from distance: d(r) continued for r > 0,
//                           softplus in place of the ReLU of a_ref (backward)
//   Sec. 3.1, App. B, C.2   adaptive Dormand-Prince 5(4), PID controller,
//                           quaternions integrated exactly
//   Fig. 12                 Tsitouras 5(4) and fixed-step semi-implicit Euler
//
// GB300 notes: FP64 runs at 1/62 of the FP32 rate and a warp instruction costs
// the same whatever its active lanes, so work is split across the group where
// it parallelises and divisions are avoided (reciprocals, division-free
// breakpoint comparisons).  The Newton search starts from the active set of
// the previous right-hand side of the same environment (the minimiser is
// unique, so the start only changes the number of iterations).
#pragma once
#include <cuda_runtime.h>
#include <math.h>

#include <type_traits>

#include "dmx_dual.cuh"
#include "dmx_model.h"

namespace dmx {

// ------------------------------------------------------------------ lane groups
template <int G>
struct Grp {
  int lane;
  int base;                          // first warp lane of the group
  unsigned mask;
  __device__ Grp() {
    const int l = threadIdx.x & 31;
    lane = l & (G - 1);
    base = l & ~(G - 1);
    mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << base);
  }
  // bit k: predicate of the group's lane k
  __device__ unsigned ballot(bool p) const {
    const unsigned b = __ballot_sync(mask, p);
    return G == 32 ? b : (b >> base) & ((1u << G) - 1u);
  }
  __device__ unsigned ior(unsigned x) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x |= __shfl_xor_sync(mask, x, o);
    return x;
  }
  __device__ void sync() const {
    if (G > 1) __syncwarp(mask);
  }
  __device__ double sum(double x) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    return x;
  }
  __device__ int isum(int x) const {
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    return x;
  }
  __device__ int bcast(int x, int src) const { return G == 1 ? x : __shfl_sync(mask, x, src, G); }
  __device__ double bcast(double x, int src) const { return G == 1 ? x : __shfl_sync(mask, x, src, G); }
};

// (row, column) of the t-th entry of a lower triangle enumerated row by row
// ((0,0), (1,0), (1,1), (2,0), ...): the same for every matrix size.
struct TriTab {
  unsigned char e[MAXV * (MAXV + 1) / 2][2];
};
__host__ __device__ constexpr TriTab make_tri() {
  TriTab t{};
  int k = 0;
  for (int i = 0; i < MAXV; ++i)
    for (int j = 0; j <= i; ++j) { t.e[k][0] = (unsigned char)i; t.e[k][1] = (unsigned char)j; ++k; }
  return t;
}
static __constant__ TriTab c_tri_tab = make_tri();
#define c_tri c_tri_tab.e

// ------------------------------------------------------------------ small helpers
// Templated on the scalar types so that the same code runs on doubles (the
// forward path) and on derivative scalars (the adjoint); model constants
// stay double.
template <class A, class B, class C>
__device__ __forceinline__ void cross3(const A* a, const B* b, C* c) {
  c[0] = a[1] * b[2] - a[2] * b[1];
  c[1] = a[2] * b[0] - a[0] * b[2];
  c[2] = a[0] * b[1] - a[1] * b[0];
}
template <class A, class B>
__device__ __forceinline__ auto dot3(const A* a, const B* b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
template <class A, class B, class C>
__device__ __forceinline__ void matmul3(const A* M, const B* N, C* P) {
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) P[3 * i + j] = M[3 * i] * N[j] + M[3 * i + 1] * N[3 + j] + M[3 * i + 2] * N[6 + j];
}
template <class A, class B, class C>
__device__ __forceinline__ void matvec3(const A* M, const B* x, C* y) {
  y[0] = M[0] * x[0] + M[1] * x[1] + M[2] * x[2];
  y[1] = M[3] * x[0] + M[4] * x[1] + M[5] * x[2];
  y[2] = M[6] * x[0] + M[7] * x[1] + M[8] * x[2];
}
template <class A, class B, class C>
__device__ __forceinline__ void matTvec3(const A* M, const B* x, C* y) {
  y[0] = M[0] * x[0] + M[3] * x[1] + M[6] * x[2];
  y[1] = M[1] * x[0] + M[4] * x[1] + M[7] * x[2];
  y[2] = M[2] * x[0] + M[5] * x[1] + M[8] * x[2];
}
// rotation matrix of the normalised quaternion (w, x, y, z)
template <class T>
__device__ __forceinline__ void quat_to_mat(const T* q, T* R) {
  const T n2 = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] + q[3] * q[3];
  const T s = 2.0 / n2;   // 2 / |q|^2 folds the normalisation into the products
  const T w = q[0], x = q[1], y = q[2], z = q[3];
  const T xx = s * x * x, yy = s * y * y, zz = s * z * z;
  const T xy = s * x * y, xz = s * x * z, yz = s * y * z;
  const T wx = s * w * x, wy = s * w * y, wz = s * w * z;
  R[0] = 1.0 - (yy + zz); R[1] = xy - wz; R[2] = xz + wy;
  R[3] = xy + wz; R[4] = 1.0 - (xx + zz); R[5] = yz - wx;
  R[6] = xz - wy; R[7] = yz + wx; R[8] = 1.0 - (xx + yy);
}
// spatial inertia (10 numbers: m, h = m c, I_O xx yy zz xy xz yz about the world
// origin) applied to a motion vector (w; v): (I_O w + h x v; m v - h x w)
template <class T>
__device__ __forceinline__ void inertia_apply(const T* I, const T* x, T* y) {
  const T m = I[0], h0 = I[1], h1 = I[2], h2 = I[3];
  const T w0 = x[0], w1 = x[1], w2 = x[2], v0 = x[3], v1 = x[4], v2 = x[5];
  y[0] = I[4] * w0 + I[7] * w1 + I[8] * w2 + (h1 * v2 - h2 * v1);
  y[1] = I[7] * w0 + I[5] * w1 + I[9] * w2 + (h2 * v0 - h0 * v2);
  y[2] = I[8] * w0 + I[9] * w1 + I[6] * w2 + (h0 * v1 - h1 * v0);
  y[3] = m * v0 - (h1 * w2 - h2 * w1);
  y[4] = m * v1 - (h2 * w0 - h0 * w2);
  y[5] = m * v2 - (h0 * w1 - h1 * w0);
}
// motion cross product (w; v) x (w2; v2) = (w x w2; w x v2 + v x w2)
template <class T>
__device__ __forceinline__ void crm6(const T* a, const T* b, T* c) {
  T t[3];
  cross3(a, b, c);
  cross3(a, b + 3, c + 3);
  cross3(a + 3, b, t);
  c[3] += t[0]; c[4] += t[1]; c[5] += t[2];
}
// force cross product (w; v) x* (n; f) = (w x n + v x f; w x f)
template <class T>
__device__ __forceinline__ void crf6(const T* a, const T* b, T* c) {
  T t[3];
  cross3(a, b, c);
  cross3(a + 3, b + 3, t);
  c[0] += t[0]; c[1] += t[1]; c[2] += t[2];
  cross3(a, b + 3, c + 3);
}

// Single components (e = 0..5) of the spatial products above, so that the
// six components of a body's vector can go to six lanes.
__device__ __forceinline__ int nxt3(int k) { return k == 2 ? 0 : k + 1; }
__device__ __forceinline__ int prv3(int k) { return k == 0 ? 2 : k - 1; }
template <class T>
__device__ __forceinline__ T crm_comp(const T* a, const T* b, int e) {   // (a x b)_e, motion
  const int k = e < 3 ? e : e - 3, k1 = nxt3(k), k2 = prv3(k);
  const T* x = e < 3 ? b : b + 3;
  T r = a[k1] * x[k2] - a[k2] * x[k1];                                // (w x w2) or (w x v2)
  if (e >= 3) r += a[3 + k1] * b[k2] - a[3 + k2] * b[k1];             // + v x w2
  return r;
}
template <class T>
__device__ __forceinline__ T crf_comp(const T* a, const T* b, int e) {   // (a x* b)_e, force
  const int k = e < 3 ? e : e - 3, k1 = nxt3(k), k2 = prv3(k);
  const T* x = e < 3 ? b : b + 3;
  T r = a[k1] * x[k2] - a[k2] * x[k1];                                // (w x n) or (w x f)
  if (e < 3) r += a[3 + k1] * b[3 + k2] - a[3 + k2] * b[3 + k1];      // + v x f
  return r;
}
template <class T>
__device__ __forceinline__ T inertia_comp(const T* I, const T* x, int e) {   // (I x)_e, inertia_apply
  const int k = e < 3 ? e : e - 3, k1 = nxt3(k), k2 = prv3(k);
  if (e < 3)   // I_O row k (entry (k, j): 4 + k on the diagonal, else 6 + k + j) . w + h x v
    return I[k == 0 ? 4 : 6 + k] * x[0] + I[k == 1 ? 5 : 7 + k] * x[1] + I[k == 2 ? 6 : 8 + k] * x[2] +
           (I[1 + k1] * x[3 + k2] - I[1 + k2] * x[3 + k1]);
  return I[0] * x[3 + k] - (I[1 + k1] * x[k2] - I[1 + k2] * x[k1]);   // m v - h x w
}

// ------------------------------------------------------------------ workspace view
template <class T>
struct WsT {
  T* d;
  int* i;
  const Layout* L;
  // the right-hand-side VJP reads the contact records / Jacobian rows here
  // when set (a stage snapshot in device memory), else from the workspace
  const double* xct = nullptr;
  const double* xJ = nullptr;
  // derivative scalars: the model parameter (PAR_*) whose tangent this
  // evaluation carries, -1 for none
  int pdir = -1;
  __device__ T* at(int off) const { return d + off; }
};

// Value v of model parameter k; a derivative scalar carries a unit tangent
// when k is the direction pdir being differentiated.
// Parameter order: PAR_TC .. PAR_MID, mu of every pair, then the mass of
// every body (rotational inertia scaled in proportion).
__device__ __forceinline__ int par_mass(const DevModel& m, int b) { return PAR_MU0 + m.npair + b; }
// then the side length of every box geom (its edge along the geom's x axis;
// the half sizes scale together; the inertia of a body whose only geom is the
// box scales with the square)
__device__ __forceinline__ int par_side(const DevModel& m, int j) { return PAR_MU0 + m.npair + m.nbody + j; }
template <class T>
struct Par {
  static __device__ __forceinline__ double get(int, int, double v) { return v; }
  static __device__ __forceinline__ double bcoef(const DevModel& m, int) { return m.bcoef; }
  static __device__ __forceinline__ double kcoef(const DevModel& m, int) { return m.kcoef; }
  static __device__ __forceinline__ double ahat(const DevModel& m, int, int p) { return m.p_ahat[p]; }
  static __device__ __forceinline__ double ahat_edge(const DevModel& m, int, int p) { return m.p_ahat_edge[p]; }
  static __device__ __forceinline__ bool mass_dir(const DevModel&, int, int) { return false; }
  static __device__ __forceinline__ bool side_dir(const DevModel&, int, int) { return false; }
  static __device__ __forceinline__ double half(const DevModel& m, int, int g, int i) { return m.g_size[g][i]; }
};
template <>
struct Par<Dual> {
  static __device__ __forceinline__ Dual get(int pdir, int k, double v) { return Dual(v, pdir == k ? 1.0 : 0.0); }
  // bcoef = 2 / (d_w t_c), kcoef = 1 / (d_w^2 t_c^2 phi_d^2): values as
  // compiled, tangents by their logarithmic derivatives
  static __device__ __forceinline__ Dual bcoef(const DevModel& m, int pdir) {
    const double b = m.bcoef;
    return Dual(b, pdir == PAR_TC ? -b / m.solref[0] : pdir == PAR_DW ? -b / m.solimp[1] : 0.0);
  }
  static __device__ __forceinline__ Dual kcoef(const DevModel& m, int pdir) {
    const double k = m.kcoef;
    return Dual(k, pdir == PAR_TC ? -2.0 * k / m.solref[0]
                 : pdir == PAR_DAMP ? -2.0 * k / m.solref[1]
                 : pdir == PAR_DW ? -2.0 * k / m.solimp[1] : 0.0);
  }
  // d A_hat / d theta: non-zero for the body masses and box sides only
  static __device__ __forceinline__ double dahat(const DevModel& m, int pdir, int p) {
    const int b = pdir - par_mass(m, 0);
    return (b >= 0 && b < m.nbody + m.nbox) ? m.p_dahat[p][b] : 0.0;
  }
  static __device__ __forceinline__ Dual ahat(const DevModel& m, int pdir, int p) {
    return Dual(m.p_ahat[p], dahat(m, pdir, p));
  }
  // A_hat (1 + mu^2) of a pyramid-edge row
  static __device__ __forceinline__ Dual ahat_edge(const DevModel& m, int pdir, int p) {
    const double mu = m.p_mu[p];
    return Dual(m.p_ahat_edge[p], (pdir == PAR_MU0 + p ? 2.0 * mu * m.p_ahat[p] : 0.0) +
                                      dahat(m, pdir, p) * (1.0 + mu * mu));
  }
  static __device__ __forceinline__ bool mass_dir(const DevModel& m, int pdir, int b) { return pdir == par_mass(m, b); }
  static __device__ __forceinline__ bool side_dir(const DevModel& m, int pdir, int b) {
    return m.b_solebox[b] >= 0 && pdir == par_side(m, m.g_box[m.b_solebox[b]]);
  }
  // half size i of geom g: a box's carries dh_i/dl = h_i / (2 h_0) along its side l
  static __device__ __forceinline__ Dual half(const DevModel& m, int pdir, int g, int i) {
    const double h = m.g_size[g][i];
    return Dual(h, (m.g_box[g] >= 0 && pdir == par_side(m, m.g_box[g])) ? h / (2.0 * m.g_size[g][0]) : 0.0);
  }
};
using Ws = WsT<double>;

// Entry e (row-major) of the rotation of the quaternion x (w, x, y, z) with
// s = 2 / |x|^2 (the normalisation folded into the products).
template <class T>
__device__ __forceinline__ T quat_entry(const T* x, const T& s, int e) {
  const T w = x[0], a = x[1], b = x[2], c = x[3];
  switch (e) {
    case 0: return 1.0 - (s * b * b + s * c * c);
    case 1: return s * a * b - s * w * c;
    case 2: return s * a * c + s * w * b;
    case 3: return s * a * b + s * w * c;
    case 4: return 1.0 - (s * a * a + s * c * c);
    case 5: return s * b * c - s * w * a;
    case 6: return s * a * c - s * w * b;
    case 7: return s * b * c + s * w * a;
    default: return 1.0 - (s * a * a + s * b * b);
  }
}
// Entry (i, j) of the hinge rotation about the unit axis a by the angle with
// sine sn and cosine cs (Rodrigues: I + sin K + (1 - cos) K^2, K = [a]x).
template <class T>
__device__ __forceinline__ T hinge_entry(const double* a, const T& sn, const T& cs, int i, int j) {
  const T c1 = 1.0 - cs;
  T v = c1 * a[i] * a[j];
  if (i == j) return cs + v;
  const int k = 3 - i - j;                       // the third axis
  const bool pos = (j == nxt3(i));               // K_ij = -a_k for j = i + 1 (cyclic), else +a_k
  return pos ? v - sn * a[k] : v + sn * a[k];
}

// Kinematics: body poses, COMs, dof motion vectors, body spatial inertias, geom poses.
// Work is split into small tasks so that a group's lanes stay busy even for a
// single body: per-body scalars (hinge sine and cosine, the free joint's
// quaternion normalisation), then every entry of every local transform, then
// the composition along the tree level by level (one entry per task), then
// COMs, geom poses and dof motion vectors, then spatial inertias.
template <int G, class T>
__device__ void kinematics(const Grp<G>& g, const DevModel& m, const WsT<T>& w, const T* q) {
  const Layout& L = *w.L;
  T* R = w.at(L.R); T* P = w.at(L.p); T* C = w.at(L.com);
  T* S = w.at(L.sd); T* Ib = w.at(L.Ib);
  T* X = w.at(L.xl); T* SC = w.at(L.sc);
  const int nb = m.nbody;
  for (int b = g.lane; b < nb; b += G) {
    const T* x = q + m.b_qadr[b];
    if (m.b_jtype[b] == JNT_FREE) {
      SC[2 * b] = 2.0 / (x[3] * x[3] + x[4] * x[4] + x[5] * x[5] + x[6] * x[6]);
    } else {
      T sn, cs;
      sincos(x[0], &sn, &cs);
      SC[2 * b] = sn; SC[2 * b + 1] = cs;
    }
  }
  g.sync();
  // local transforms: free joint = world pose; hinge = rotation in the parent frame.
  // Bodies at the root are written straight into the world arrays.
  for (int t = g.lane; t < 12 * nb; t += G) {
    const int b = t / 12, e = t - 12 * b;
    const bool root = m.b_parent[b] < 0;
    T v;
    if (m.b_jtype[b] == JNT_FREE) {
      const T* x = q + m.b_qadr[b];
      v = e < 9 ? quat_entry(x + 3, SC[2 * b], e) : x[e - 9];
    } else if (e >= 9) {
      v = m.b_pos[b][e - 9];
    } else {
      const int i = e / 3, j = e - 3 * (e / 3);
      const T sn = SC[2 * b], cs = SC[2 * b + 1];
      if (m.b_ident[b]) {
        v = hinge_entry(m.b_axis[b], sn, cs, i, j);
      } else {
        const double* Ro = m.b_Roff[b];
        v = Ro[3 * i] * hinge_entry(m.b_axis[b], sn, cs, 0, j) + Ro[3 * i + 1] * hinge_entry(m.b_axis[b], sn, cs, 1, j) +
            Ro[3 * i + 2] * hinge_entry(m.b_axis[b], sn, cs, 2, j);
      }
    }
    if (root) { if (e < 9) R[9 * b + e] = v; else P[3 * b + e - 9] = v; }
    else X[12 * b + e] = v;
  }
  g.sync();
  // world poses: R = R_parent R_local, p = p_parent + R_parent p_local
  for (int lev = 1; lev < m.nlevel; ++lev) {
    for (int t = 12 * m.level_start[lev] + g.lane; t < 12 * m.level_start[lev + 1]; t += G) {
      const int k = t / 12, e = t - 12 * k;
      const int b = m.level_list[k], par = m.b_parent[b];
      const T* Rp = R + 9 * par; const T* xl = X + 12 * b;
      if (e < 9) {
        const int i = e / 3, j = e - 3 * (e / 3);
        R[9 * b + e] = Rp[3 * i] * xl[j] + Rp[3 * i + 1] * xl[3 + j] + Rp[3 * i + 2] * xl[6 + j];
      } else {
        const int i = e - 9;
        P[3 * b + i] = P[3 * par + i] + (Rp[3 * i] * xl[9] + Rp[3 * i + 1] * xl[10] + Rp[3 * i + 2] * xl[11]);
      }
    }
    g.sync();
  }
  // COMs (one component per task), geom poses (one entry per task), dof
  // motion vectors (w; v at the world origin, one dof per task)
  T* gR = w.at(L.gR); T* gp = w.at(L.gp);
  const int n1 = 3 * nb, n2 = n1 + 12 * m.ngeom, n3 = n2 + m.nv;
  for (int t = g.lane; t < n3; t += G) {
    if (t < n1) {
      const int b = t / 3, i = t - 3 * b;
      const T* Rb = R + 9 * b; const double* c = m.b_com[b];
      C[t] = (Rb[3 * i] * c[0] + Rb[3 * i + 1] * c[1] + Rb[3 * i + 2] * c[2]) + P[t];
    } else if (t < n2) {
      const int gi = (t - n1) / 12, e = t - n1 - 12 * gi;
      const int b = m.g_body[gi];
      const T* Rb = R + 9 * b;
      if (e < 9) {
        const int i = e / 3, j = e - 3 * (e / 3);
        const double* Ro = m.g_Roff[gi];
        gR[9 * gi + e] = m.g_ident[gi] ? Rb[e] : Rb[3 * i] * Ro[j] + Rb[3 * i + 1] * Ro[3 + j] + Rb[3 * i + 2] * Ro[6 + j];
      } else {
        const int i = e - 9;
        const double* gpos = m.g_pos[gi];
        gp[3 * gi + i] = m.g_zpos[gi] ? P[3 * b + i]
                                      : P[3 * b + i] + (Rb[3 * i] * gpos[0] + Rb[3 * i + 1] * gpos[1] + Rb[3 * i + 2] * gpos[2]);
      }
    } else {
      const int i = t - n2;
      const int b = m.dof_body[i];
      const T* Rb = R + 9 * b; const T* pb = P + 3 * b;
      T* st = S + 6 * i;
      if (m.b_jtype[b] == JNT_FREE) {
        const int d = i - m.b_vadr[b];
        if (d < 3) {
          st[0] = 0.0; st[1] = 0.0; st[2] = 0.0; st[3] = d == 0 ? 1.0 : 0.0; st[4] = d == 1 ? 1.0 : 0.0;
          st[5] = d == 2 ? 1.0 : 0.0;
        } else {
          st[0] = Rb[d - 3]; st[1] = Rb[d]; st[2] = Rb[d + 3];
          cross3(pb, st, st + 3);
        }
      } else {
        matvec3(Rb, m.b_axis[b], st);
        cross3(pb, st, st + 3);
      }
    }
  }
  g.sync();
  // spatial inertias about the world origin (m, m c, R diag(I) R^T + m (|c|^2 1 - c c^T)),
  // one entry per task
  for (int k = g.lane; k < 10 * nb; k += G) {
    const int b = k / 10, e = k - 10 * b;
    const auto ms = Par<T>::get(w.pdir, par_mass(m, b), m.b_mass[b]);
    const T* c = C + 3 * b;
    T v;
    if (e == 0) v = ms;
    else if (e < 4) v = ms * c[e - 1];
    else {
      const int ii[6] = {0, 1, 2, 0, 0, 1}, jj[6] = {0, 1, 2, 1, 2, 2};
      const int i = ii[e - 4], j = jj[e - 4];
      const T* Rb = R + 9 * b;
      const double* In = m.b_inertia[b];
      v = Rb[3 * i] * Rb[3 * j] * In[0] + Rb[3 * i + 1] * Rb[3 * j + 1] * In[1] + Rb[3 * i + 2] * Rb[3 * j + 2] * In[2];
      if (Par<T>::mass_dir(m, w.pdir, b)) v = v * (ms / m.b_mass[b]);   // inertia proportional to the mass
      if (Par<T>::side_dir(m, w.pdir, b)) {                             // ... and to the side squared
        const int gs = m.b_solebox[b];
        const double l0 = 2.0 * m.g_size[gs][0];
        const auto lam = Par<T>::get(w.pdir, par_side(m, m.g_box[gs]), l0) / l0;
        v = v * (lam * lam);
      }
      const T cc = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
      v += ms * ((i == j ? cc : T(0.0)) - c[i] * c[j]);
    }
    Ib[10 * b + e] = v;
  }
  g.sync();
}

// Composite-rigid-body algorithm: M (dense, both triangles).
template <int G, class T>
__device__ void crba(const Grp<G>& g, const DevModel& m, const WsT<T>& w) {
  const Layout& L = *w.L;
  const T* Ib = w.at(L.Ib); T* Ic = w.at(L.Ic);
  const T* S = w.at(L.sd); T* F = w.at(L.F); T* M = w.at(L.M);
  const int nv = m.nv;
  for (int lev = m.nlevel - 1; lev >= 0; --lev) {
    for (int k = m.level_start[lev] + g.lane; k < m.level_start[lev + 1]; k += G) {
      const int b = m.level_list[k];
      T acc[10];
      for (int e = 0; e < 10; ++e) acc[e] = Ib[10 * b + e];
      for (int c = 0; c < m.child_count[b]; ++c) {
        const int ch = m.child_list[m.child_start[b] + c];
        for (int e = 0; e < 10; ++e) acc[e] += Ic[10 * ch + e];
      }
      for (int e = 0; e < 10; ++e) Ic[10 * b + e] = acc[e];
    }
    g.sync();
  }
  for (int i = g.lane; i < nv; i += G) inertia_apply(Ic + 10 * m.dof_body[i], S + 6 * i, F + 6 * i);
  g.sync();
  for (int t = g.lane; t < nv * (nv + 1) / 2; t += G) {   // lower triangle
    const int i = c_tri[t][0], j = c_tri[t][1];
    T v = 0.0;
    if ((m.b_anc[m.dof_body[i]] >> m.dof_body[j]) & 1u) {
      const T* s = S + 6 * j; const T* f = F + 6 * i;
      v = s[0] * f[0] + s[1] * f[1] + s[2] * f[2] + s[3] * f[3] + s[4] * f[4] + s[5] * f[5];
    }
    M[i * nv + j] = v;
    M[j * nv + i] = v;
  }
  g.sync();
}

// Recursive Newton-Euler with zero joint acceleration: rhs0 = tau - c.
// Body velocities and velocity-product accelerations are sums along the path
// from the root: each body's own joint term is computed for all bodies at
// once, then added down the tree level by level (6 additions per body).  The
// per-body work is split by component (one body component per task).
template <int G, class T>
__device__ void rne_and_forces(const Grp<G>& g, const DevModel& m, const WsT<T>& w, const T* q, const T* v,
                               const T* u) {
  const Layout& L = *w.L;
  const T* Ib = w.at(L.Ib); const T* S = w.at(L.sd);
  T* V = w.at(L.Vb); T* A = w.at(L.Ab); T* Fb = w.at(L.Fb); T* IV = w.at(L.iv);
  const int nt = 6 * m.nbody;
  // own joint velocity S v
  for (int t = g.lane; t < nt; t += G) {
    const int b = t / 6, e = t - 6 * b;
    const int va = m.b_vadr[b], nd = m.b_nv[b];
    T x = 0.0;
    for (int d = 0; d < nd; ++d) x += S[6 * (va + d) + e] * v[va + d];
    V[t] = x;
  }
  g.sync();
  for (int lev = 1; lev < m.nlevel; ++lev) {
    for (int t = 6 * m.level_start[lev] + g.lane; t < 6 * m.level_start[lev + 1]; t += G) {
      const int k = t / 6, e = t - 6 * k;
      const int b = m.level_list[k], par = m.b_parent[b];
      if (par >= 0) V[6 * b + e] += V[6 * par + e];
    }
    g.sync();
  }
  // own velocity-product acceleration (vb x S_d) v_d (gravity at the roots)
  for (int t = g.lane; t < nt; t += G) {
    const int b = t / 6, e = t - 6 * b;
    const int va = m.b_vadr[b], nd = m.b_nv[b];
    T x = (m.b_parent[b] < 0 && e >= 3) ? T(-m.grav[e - 3]) : T(0.0);
    const int d0 = (m.b_jtype[b] == JNT_FREE) ? 3 : 0;   // world-fixed translation axes
    for (int d = d0; d < nd; ++d) x += crm_comp(V + 6 * b, S + 6 * (va + d), e) * v[va + d];
    A[t] = x;
  }
  g.sync();
  for (int lev = 1; lev < m.nlevel; ++lev) {
    for (int t = 6 * m.level_start[lev] + g.lane; t < 6 * m.level_start[lev + 1]; t += G) {
      const int k = t / 6, e = t - 6 * k;
      const int b = m.level_list[k], par = m.b_parent[b];
      if (par >= 0) A[6 * b + e] += A[6 * par + e];
    }
    g.sync();
  }
  // body forces I a + v x* (I v)
  for (int t = g.lane; t < nt; t += G) {
    const int b = t / 6, e = t - 6 * b;
    Fb[t] = inertia_comp(Ib + 10 * b, A + 6 * b, e);
    IV[t] = inertia_comp(Ib + 10 * b, V + 6 * b, e);
  }
  g.sync();
  for (int t = g.lane; t < nt; t += G) {
    const int b = t / 6, e = t - 6 * b;
    Fb[t] += crf_comp(V + 6 * b, IV + 6 * b, e);
  }
  g.sync();
  for (int lev = m.nlevel - 1; lev >= 1; --lev) {
    // children add into their parents; parents of one level are distinct bodies
    // of the level above, so sweep the level above and gather its children
    for (int t = 6 * m.level_start[lev - 1] + g.lane; t < 6 * m.level_start[lev]; t += G) {
      const int k = t / 6, e = t - 6 * k;
      const int b = m.level_list[k];
      for (int c = 0; c < m.child_count[b]; ++c) Fb[6 * b + e] += Fb[6 * m.child_list[m.child_start[b] + c] + e];
    }
    g.sync();
  }
  T* rhs0 = w.at(L.rhs0);
  for (int i = g.lane; i < m.nv; i += G) {
    const T* s = S + 6 * i; const T* f = Fb + 6 * m.dof_body[i];
    const T c = s[0] * f[0] + s[1] * f[1] + s[2] * f[2] + s[3] * f[3] + s[4] * f[4] + s[5] * f[5];
    const T tau = -m.b_damping[m.dof_body[i]] * v[i];
    rhs0[i] = tau - c;
  }
  g.sync();
  if (g.lane == 0) {
    for (int a = 0; a < m.nact; ++a) {
      const int vi = m.a_vadr[a];
      if (m.a_type[a] == ACT_MOTOR) rhs0[vi] += m.a_gear[a] * u[a];
      else rhs0[vi] += m.a_kp[a] * (u[a] - q[m.a_qadr[a]]) - m.a_kd[a] * v[vi];
    }
  }
  g.sync();
}

// ------------------------------------------------------------------ collision
// contact record (16 scalars): r, pos[3], n[3], t1[3], t2[3], d, pterm, D
template <class T, class H>
__device__ __forceinline__ T box_sdf(const T* y, const H* h, T* grad) {
  T qd[3];
  bool out = false;
  for (int i = 0; i < 3; ++i) { qd[i] = fabs(y[i]) - h[i]; out = out || value(qd[i]) > 0; }
  if (out) {
    T ss = 0.0;
    for (int i = 0; i < 3; ++i) if (value(qd[i]) > 0) ss += qd[i] * qd[i];
    const T d = sqrt(ss), inv = 1.0 / d;
    for (int i = 0; i < 3; ++i) {
      const T gg = value(qd[i]) > 0 ? qd[i] * inv : T(0.0);
      grad[i] = value(y[i]) < 0 ? -gg : gg;
    }
    return d;
  }
  int k = 0;
  if (value(qd[1]) > value(qd[k])) k = 1;
  if (value(qd[2]) > value(qd[k])) k = 2;
  grad[0] = 0.0; grad[1] = 0.0; grad[2] = 0.0;
  grad[k] = value(y[k]) < 0 ? -1.0 : 1.0;
  return qd[k];
}
// A number with the sign of the slope of the box distance field along
// y0 + s wv: outside the box the gradient is (sgn y_i max(|y_i| - h_i, 0))_i
// divided by the (positive) distance, so the division and the square root
// are left out; inside it is sgn(y_k) e_k for the axis k of the largest
// |y_k| - h_k (the same tie rule as box_sdf).
__device__ __forceinline__ double box_sdf_slope(const double* y0, const double* wv, double s, const double* h) {
  const double y[3] = {y0[0] + s * wv[0], y0[1] + s * wv[1], y0[2] + s * wv[2]};
  const double qd[3] = {fabs(y[0]) - h[0], fabs(y[1]) - h[1], fabs(y[2]) - h[2]};
  if (qd[0] > 0 || qd[1] > 0 || qd[2] > 0) {
    double num = 0.0;
    for (int i = 0; i < 3; ++i)
      if (qd[i] > 0) num += (y[i] < 0 ? -qd[i] : qd[i]) * wv[i];
    return num;
  }
  int k = 0;
  if (qd[1] > qd[k]) k = 1;
  if (qd[2] > qd[k]) k = 2;
  return y[k] < 0 ? -wv[k] : wv[k];
}

// Minimiser over the capsule axis s in [-Lh, Lh] of the box distance field
// along y0 + s wv (box frame), by bisection on its slope (values only).
__device__ __forceinline__ double capsule_box_s(const double* y0v, const double* wvv, double Lh, const double* h) {
  if (box_sdf_slope(y0v, wvv, -Lh, h) >= 0) return -Lh;
  if (box_sdf_slope(y0v, wvv, Lh, h) <= 0) return Lh;
  double lo = -Lh, hi = Lh;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (mid <= lo || mid >= hi) break;
    if (box_sdf_slope(y0v, wvv, mid, h) < 0) lo = mid; else hi = mid;
  }
  return 0.5 * (lo + hi);
}
// Curvature phi'' of the distance along the axis at an interior minimiser sv
// outside the box, where the minimiser moves with the poses (implicit
// function theorem: ds = -d(slope) / phi'').  Returns 0 where s is held
// constant (an end of the axis, inside the box, or a flat direction).
__device__ __forceinline__ double capsule_box_curv(const double* y0v, const double* wvv, double sv, double Lh,
                                                   const double* h) {
  double yv[3] = {y0v[0] + sv * wvv[0], y0v[1] + sv * wvv[1], y0v[2] + sv * wvv[2]}, gv[3];
  const double phi = box_sdf(yv, h, gv);
  bool outside = false;
  for (int i = 0; i < 3; ++i) outside = outside || (fabs(yv[i]) - h[i] > 0);
  if (!(outside && sv > -Lh && sv < Lh && phi > 0)) return 0.0;
  const double gw = gv[0] * wvv[0] + gv[1] * wvv[1] + gv[2] * wvv[2];
  double ww = 0;
  for (int i = 0; i < 3; ++i) if (fabs(yv[i]) > h[i]) ww += wvv[i] * wvv[i];
  const double phi2 = (ww - gw * gw) / phi;
  return phi2 > 1e-12 ? phi2 : 0.0;
}

// Capsule (geom g1) against box (geom g2): minimum over the capsule axis of
// the box distance field (convex along the axis; bisection on its slope, in
// values).  In derivative scalars the minimiser s carries ds/dtheta from the
// implicit function theorem (slope = 0 at an interior minimum of the smooth
// outside field: ds = -d(slope) / (d slope / ds)); elsewhere s is constant.
template <class T>
__device__ void capsule_box(const DevModel& m, const T* gR, const T* gp, int g1, int g2, double thr, T* ct,
                            T* s_out, int pdir = -1) {
  const double rc = m.g_size[g1][0], Lh = m.g_size[g1][1];
  const double* h = m.g_size[g2];
  // the box half sizes as the evaluation's scalars (a side-length tangent in derivative scalars)
  T hd[3];
  if constexpr (!std::is_same<T, double>::value)
    for (int i = 0; i < 3; ++i) hd[i] = Par<T>::half(m, pdir, g2, i);
  const auto* hT = [&]() {
    if constexpr (std::is_same<T, double>::value) return h; else return static_cast<const T*>(hd);
  }();
  const T* R1 = gR + 9 * g1; const T* R2 = gR + 9 * g2;
  const T* c1 = gp + 3 * g1; const T* c2 = gp + 3 * g2;
  T dc[3] = {c1[0] - c2[0], c1[1] - c2[1], c1[2] - c2[2]};
  const double reach = m.g_bound[g1] + m.g_bound[g2] + (thr > 0 ? thr : 0.0);
  const double dd = value(dc[0]) * value(dc[0]) + value(dc[1]) * value(dc[1]) + value(dc[2]) * value(dc[2]);
  if (dd > reach * reach) { ct[0] = 1e30; return; }   // cannot be within the threshold
  const T u[3] = {R1[0], R1[3], R1[6]};
  T y0[3], wv[3];
  matTvec3(R2, dc, y0);
  matTvec3(R2, u, wv);
  const double y0v[3] = {value(y0[0]), value(y0[1]), value(y0[2])}, wvv[3] = {value(wv[0]), value(wv[1]), value(wv[2])};
  const double sv = capsule_box_s(y0v, wvv, Lh, h);
  *s_out = T(sv);
  T s = sv;
  if constexpr (!std::is_same<T, double>::value) {
    const double phi2 = capsule_box_curv(y0v, wvv, sv, Lh, h);
    if (phi2 > 0) {
      T yT[3] = {y0[0] + sv * wv[0], y0[1] + sv * wv[1], y0[2] + sv * wv[2]}, gT[3];
      box_sdf(yT, hT, gT);
      const T slope = gT[0] * wv[0] + gT[1] * wv[1] + gT[2] * wv[2];
      s = T(sv, -slope.d / phi2);
    }
  }
  T y[3] = {y0[0] + s * wv[0], y0[1] + s * wv[1], y0[2] + s * wv[2]}, gr[3], n[3];
  const T dist = box_sdf(y, hT, gr);
  matvec3(R2, gr, n);
  const T r = dist - rc;
  ct[0] = r;
  const T off = rc + 0.5 * r;
  for (int i = 0; i < 3; ++i) { ct[1 + i] = c1[i] + s * u[i] - off * n[i]; ct[4 + i] = n[i]; }
  // tangent frame: t1 perpendicular to n and world z (world x when n is near z)
  double ref[3] = {0, 0, 1};
  if (fabs(value(n[2])) >= 0.5) { ref[0] = 1; ref[2] = 0; }
  T t1[3], t2[3];
  cross3(n, ref, t1);
  const T il = rsqrt_t(dot3(t1, t1));
  t1[0] *= il; t1[1] *= il; t1[2] *= il;
  cross3(n, t1, t2);
  for (int i = 0; i < 3; ++i) { ct[7 + i] = t1[i]; ct[10 + i] = t2[i]; }
}

// Spline of the solimp shape on x in [0, 1] (midpoint mid, power pw).
// Sphere / capsule pair (the billiard's ball-ball contact of Sec. 4, capsule
// pairs of App. C.1): geom g is the segment c + s u, |s| <= L along its local
// x (L = 0 for a sphere), radius rad.  Closest points: the least of the
// candidates of the box-constrained optimality conditions of
// |D + s ua - t ub|^2 (D = ca - cb): the interior point (non-parallel axes)
// and each edge with the other parameter clamped.  Decisions on values; with
// derivative scalars the free parameters are re-solved from the reduced
// optimality conditions (Du + s - c t = 0, -Dv - c s + t = 0), carrying
// ds/dtheta, dt/dtheta.  n from geom 2 to geom 1, r = |d| - ra - rb,
// pos = pa - (ra + r/2) n; tangent frame as for capsule-box.  st_out: s, t.
__device__ __forceinline__ double seg_half(const DevModel& m, int g) {
  return m.g_type[g] == GEOM_CAPSULE ? m.g_size[g][1] : 0.0;
}
__device__ __forceinline__ void seg_closest(double c, double Du, double Dv, double La, double Lb, const double* D,
                                            const double* ua, const double* ub, double* s_out, double* t_out) {
  double bs = 0.0, bt = 0.0, best = INFINITY;
  auto consider = [&](double s, double t) {
    if (fabs(s) > La || fabs(t) > Lb) return;
    double d2 = 0.0;
    for (int i = 0; i < 3; ++i) {
      const double di = D[i] + s * ua[i] - t * ub[i];
      d2 += di * di;
    }
    if (d2 < best) { best = d2; bs = s; bt = t; }
  };
  if (1.0 - c * c > 1e-12) {
    const double s0 = (c * Dv - Du) / (1.0 - c * c);
    consider(s0, Dv + s0 * c);
  }
  consider(-La, fmin(fmax(Dv - La * c, -Lb), Lb));
  consider(La, fmin(fmax(Dv + La * c, -Lb), Lb));
  consider(fmin(fmax(-Lb * c - Du, -La), La), -Lb);
  consider(fmin(fmax(Lb * c - Du, -La), La), Lb);
  *s_out = bs;
  *t_out = bt;
}
template <class T>
__device__ void seg_seg(const DevModel& m, const T* gR, const T* gp, int g1, int g2, double thr, T* ct, T* st_out) {
  const double ra = m.g_size[g1][0], rb = m.g_size[g2][0];
  const double La = seg_half(m, g1), Lb = seg_half(m, g2);
  const T* R1 = gR + 9 * g1; const T* R2 = gR + 9 * g2;
  const T* c1 = gp + 3 * g1; const T* c2 = gp + 3 * g2;
  const T D[3] = {c1[0] - c2[0], c1[1] - c2[1], c1[2] - c2[2]};
  const double reach = m.g_bound[g1] + m.g_bound[g2] + (thr > 0 ? thr : 0.0);
  const double Dv0[3] = {value(D[0]), value(D[1]), value(D[2])};
  if (Dv0[0] * Dv0[0] + Dv0[1] * Dv0[1] + Dv0[2] * Dv0[2] > reach * reach) { ct[0] = 1e30; return; }
  const T ua[3] = {R1[0], R1[3], R1[6]}, ub[3] = {R2[0], R2[3], R2[6]};
  const double uav[3] = {value(ua[0]), value(ua[1]), value(ua[2])}, ubv[3] = {value(ub[0]), value(ub[1]), value(ub[2])};
  const double cv = dot3(uav, ubv), Duv = dot3(Dv0, uav), Dvv = dot3(Dv0, ubv);
  double sv, tv;
  seg_closest(cv, Duv, Dvv, La, Lb, Dv0, uav, ubv, &sv, &tv);
  st_out[0] = T(sv);
  st_out[1] = T(tv);
  T s = sv, t = tv;
  if constexpr (!std::is_same<T, double>::value) {
    const bool sf = fabs(sv) < La, tf = fabs(tv) < Lb;
    const T c = dot3(ua, ub), Du = dot3(D, ua), Dv = dot3(D, ub);
    if (sf && tf) {
      s = (c * Dv - Du) / (1.0 - c * c);
      t = Dv + c * s;
    } else if (sf) {
      s = tv * c - Du;
    } else if (tf) {
      t = Dv + sv * c;
    }
  }
  T d[3], n[3];
  for (int i = 0; i < 3; ++i) d[i] = D[i] + s * ua[i] - t * ub[i];
  const T rho = sqrt(dot3(d, d));
  const T ir = 1.0 / rho;
  for (int i = 0; i < 3; ++i) n[i] = d[i] * ir;
  const T r = rho - (ra + rb);
  ct[0] = r;
  const T off = ra + 0.5 * r;
  for (int i = 0; i < 3; ++i) { ct[1 + i] = c1[i] + s * ua[i] - off * n[i]; ct[4 + i] = n[i]; }
  double ref[3] = {0, 0, 1};
  if (fabs(value(n[2])) >= 0.5) { ref[0] = 1; ref[2] = 0; }
  T t1[3], t2[3];
  cross3(n, ref, t1);
  const T il = rsqrt_t(dot3(t1, t1));
  t1[0] *= il; t1[1] *= il; t1[2] *= il;
  cross3(n, t1, t2);
  for (int i = 0; i < 3; ++i) { ct[7 + i] = t1[i]; ct[10 + i] = t2[i]; }
}

template <class T>
__device__ __forceinline__ T spline_shape(const T& x, double mid, double pw) {
  if (value(x) <= mid && mid > 0) {
    const T num = (pw == 2.0) ? x * x : (pw == 4.0 ? (x * x) * (x * x) : pow(x, pw));
    return num / ((pw == 2.0) ? mid : ::pow(mid, pw - 1.0));
  }
  const T y = 1.0 - x;
  const T num = (pw == 2.0) ? y * y : (pw == 4.0 ? (y * y) * (y * y) : pow(y, pw));
  return 1.0 - num / ((pw == 2.0) ? (1.0 - mid) : ::pow(1.0 - mid, pw - 1.0));
}
// The same shape with a derivative-scalar midpoint (parameter tangents).
__device__ __forceinline__ Dual spline_shape(const Dual& x, const Dual& mid, double pw) {
  if (value(x) <= value(mid) && value(mid) > 0) {
    const Dual num = (pw == 2.0) ? x * x : (pw == 4.0 ? (x * x) * (x * x) : pow(x, pw));
    return num / ((pw == 2.0) ? mid : pow(mid, pw - 1.0));
  }
  const Dual y = 1.0 - x;
  const Dual num = (pw == 2.0) ? y * y : (pw == 4.0 ? (y * y) * (y * y) : pow(y, pw));
  const Dual om = 1.0 - mid;
  return 1.0 - num / ((pw == 2.0) ? om : pow(om, pw - 1.0));
}
template <class T>
__device__ __forceinline__ T impedance(const DevModel& m, const T& r, bool cfd, int pdir = -1) {
  T d;
  if (cfd && value(r) >= 0) {
    T x = 1.0 - r / m.cfd[2];
    if (value(x) < 0) x = 0.0;
    d = m.cfd[0] + (m.cfd[1] - m.cfd[0]) * spline_shape(x, m.cfd[3], m.cfd[4]);
  } else {
    const auto d_o = Par<T>::get(pdir, PAR_DO, m.solimp[0]), d_w = Par<T>::get(pdir, PAR_DW, m.solimp[1]);
    const auto width = Par<T>::get(pdir, PAR_WIDTH, m.solimp[2]), mid = Par<T>::get(pdir, PAR_MID, m.solimp[3]);
    T x = fabs(r) / width;
    if (value(x) > 1.0) x = 1.0;
    d = d_o + (d_w - d_o) * spline_shape(x, mid, m.solimp[4]);
  }
  if (value(d) < 0.0) return T(0.0);
  if (value(d) > 0.9999) return T(0.9999);
  return d;
}
template <class T>
__device__ __forceinline__ T softplus(const T& x) { return value(x) > 0 ? x + log1p(exp(-x)) : log1p(exp(x)); }

// All contact slots, then the included ones (r < 0, or r < w_c for F~) and
// their per-slot impedance terms.
template <int G, class T>
__device__ void collide(const Grp<G>& g, const DevModel& m, const WsT<T>& w, bool cfd) {
  const Layout& L = *w.L;
  const T* gR = w.at(L.gR); const T* gp = w.at(L.gp);
  T* CT = w.at(L.ct);
  const double thr = cfd ? m.cfd[2] : 0.0;
  for (int s = g.lane; s < m.nslot; s += G) {
    T* ct = CT + 16 * s;
    const int p = m.s_pair[s], j = m.s_idx[s], g1 = m.p_g1[p];
    if (m.p_g2[p] >= 0) {
      if (m.g_type[m.p_g2[p]] == GEOM_BOX) capsule_box(m, gR, gp, g1, m.p_g2[p], thr, ct, w.at(L.csv) + 2 * s, w.pdir);
      else seg_seg(m, gR, gp, g1, m.p_g2[p], thr, ct, w.at(L.csv) + 2 * s);
    } else {
      const T* Rg = gR + 9 * g1; const T* cg = gp + 3 * g1;
      T pt[3];
      double rad = 0.0;
      const int ty = m.g_type[g1];
      if (ty == GEOM_SPHERE) { pt[0] = cg[0]; pt[1] = cg[1]; pt[2] = cg[2]; rad = m.g_size[g1][0]; }
      else if (ty == GEOM_CAPSULE) {
        const double e = (j == 0) ? -m.g_size[g1][1] : m.g_size[g1][1];
        pt[0] = cg[0] + e * Rg[0]; pt[1] = cg[1] + e * Rg[3]; pt[2] = cg[2] + e * Rg[6];
        rad = m.g_size[g1][0];
      } else {
        T t[3];
        if constexpr (std::is_same<T, double>::value) {
          const double ex[3] = {(j & 1) ? m.g_size[g1][0] : -m.g_size[g1][0],
                                (j & 2) ? m.g_size[g1][1] : -m.g_size[g1][1],
                                (j & 4) ? m.g_size[g1][2] : -m.g_size[g1][2]};
          matvec3(Rg, ex, t);
        } else {   // derivative scalars: the half sizes carry a side-length tangent
          const T h0 = Par<T>::half(m, w.pdir, g1, 0), h1 = Par<T>::half(m, w.pdir, g1, 1);
          const T h2 = Par<T>::half(m, w.pdir, g1, 2);
          const T ex[3] = {(j & 1) ? h0 : -h0, (j & 2) ? h1 : -h1, (j & 4) ? h2 : -h2};
          matvec3(Rg, ex, t);
        }
        pt[0] = cg[0] + t[0]; pt[1] = cg[1] + t[1]; pt[2] = cg[2] + t[2];
      }
      const T r = pt[2] - rad;
      ct[0] = r;
      ct[1] = pt[0]; ct[2] = pt[1]; ct[3] = pt[2] - (rad + 0.5 * r);
      ct[4] = 0.0; ct[5] = 0.0; ct[6] = 1.0; ct[7] = 1.0; ct[8] = 0.0; ct[9] = 0.0; ct[10] = 0.0; ct[11] = 1.0;
      ct[12] = 0.0;
    }
    const bool inc = value(ct[0]) < thr;
    w.i[L.sinc + s] = inc ? 1 : 0;
    if (inc) {
      const T r = ct[0];
      const T d = impedance(m, r, cfd, w.pdir);
      const int pr = m.s_pair[s];
      const auto ahat = m.p_condim[pr] == 1 ? Par<T>::ahat(m, w.pdir, pr) : Par<T>::ahat_edge(m, w.pdir, pr);
      const auto kc = Par<T>::kcoef(m, w.pdir);
      ct[13] = d;
      ct[14] = cfd ? kc * d * (m.softplus * softplus(-r / m.softplus)) : -(kc * d * r);
      ct[15] = d / (ahat * (1.0 - d));
    }
  }
  g.sync();
}

// Constraint rows of the included contacts (compacted in slot order).
// Returns the number of rows, or -1 when they exceed the workspace.
template <int G, class T>
__device__ int make_rows(const Grp<G>& g, const DevModel& m, const WsT<T>& w, const T* v, bool cfd) {
  const Layout& L = *w.L;
  const T* CT = w.at(L.ct); const T* S = w.at(L.sd);
  int* slotrow = w.i + L.slotrow; int* rowid = w.i + L.rowid; int* slist = w.i + L.slist;
  const int nv = m.nv;
  int* rowslot = w.i + L.rowslot;
  const int* sinc = w.i + L.sinc;
  if (g.lane == 0) {
    int n = 0, ns = 0;
    for (int s = 0; s < m.nslot; ++s) {
      const bool inc = sinc[s] != 0;
      slotrow[s] = inc ? n : -1;
      if (inc) {
        const int nrow = (m.p_condim[m.s_pair[s]] == 1) ? 1 : 4;
        for (int e = 0; e < nrow && n + e < L.rcap; ++e) rowslot[n + e] = s;
        n += nrow;
        slist[ns++] = s;
      }
    }
    slotrow[m.nslot] = n;
    w.i[L.misc] = ns;
  }
  g.sync();
  const int nr = slotrow[m.nslot];
  const int nincl = w.i[L.misc];
  if (nr > L.rcap) return -1;
  T* J = w.at(L.J);
  for (int idx = g.lane; idx < nincl * nv; idx += G) {   // included slots only
    const int si = idx / nv, i = idx - si * nv;
    const int s = slist[si];
    const int r0 = slotrow[s];
    const T* ct = CT + 16 * s;
    const int p = m.s_pair[s];
    const int bA = m.g_body[m.p_g1[p]];
    const int bB = m.p_g2[p] >= 0 ? m.g_body[m.p_g2[p]] : -1;
    const int bi = m.dof_body[i];
    const bool mA = (m.b_anc[bA] >> bi) & 1u;
    const bool mB = bB >= 0 && ((m.b_anc[bB] >> bi) & 1u);
    T jn = 0.0, j1 = 0.0, j2 = 0.0;
    if (mA != mB) {
      const T* sv = S + 6 * i;
      T pv[3];
      cross3(sv, ct + 1, pv);
      pv[0] += sv[3]; pv[1] += sv[4]; pv[2] += sv[5];
      const double sg = mA ? 1.0 : -1.0;
      if (bB < 0) {   // ground plane: the frame is the world's (z, x, y)
        jn = sg * pv[2]; j1 = sg * pv[0]; j2 = sg * pv[1];
      } else {
        jn = sg * dot3(ct + 4, pv); j1 = sg * dot3(ct + 7, pv); j2 = sg * dot3(ct + 10, pv);
      }
    }
    if (m.p_condim[p] == 1) {
      J[r0 * nv + i] = jn;
    } else {
      const auto mu = Par<T>::get(w.pdir, PAR_MU0 + p, m.p_mu[p]);
      J[r0 * nv + i] = jn + mu * j1;
      J[(r0 + 1) * nv + i] = jn - mu * j1;
      J[(r0 + 2) * nv + i] = jn + mu * j2;
      J[(r0 + 3) * nv + i] = jn - mu * j2;
    }
  }
  g.sync();
  T* aref = w.at(L.aref); T* Dr = w.at(L.Dr);
  for (int r = g.lane; r < nr; r += G) {   // one row per task
    const int s = rowslot[r];
    const int e = r - slotrow[s];
    const int p = m.s_pair[s];
    const int nrow = m.p_condim[p] == 1 ? 1 : 4;
    const T* ct = CT + 16 * s;
    T jv = 0.0;
    for (int i = 0; i < nv; ++i) jv += J[r * nv + i] * v[i];
    aref[r] = -(Par<T>::bcoef(m, w.pdir) * jv) + ct[14];
    Dr[r] = ct[15];
    rowid[r] = m.p_row0[p] + m.s_idx[s] * nrow + e;
  }
  g.sync();
  (void)nincl;
  return nr;
}

// ------------------------------------------------------------------ dense kernels
// H <- its Cholesky factor below the diagonal, invd <- 1 / diagonal of the
// factor.  Returns false if not SPD.
template <int G, class T>
__device__ bool cholesky(const Grp<G>& g, T* H, T* invd, int n) {
  bool ok = true;
  for (int k = 0; k < n; ++k) {
    const T hkk = H[k * n + k];
    ok = ok && (value(hkk) > 0);
    const T il = rsqrt_t(hkk);   // the diagonal of the factor is kept as its reciprocal
    for (int i = k + 1 + g.lane; i < n; i += G) H[i * n + k] *= il;
    if (g.lane == 0) invd[k] = il;
    g.sync();
    const int nt = n - k - 1;
    for (int t = g.lane; t < nt * (nt + 1) / 2; t += G) {   // lower triangle of the trailing block
      const int i = k + 1 + c_tri[t][0], j = k + 1 + c_tri[t][1];
      H[i * n + j] -= H[i * n + k] * H[j * n + k];
    }
    g.sync();
  }
  return ok;
}
// x <- H^-1 x with the factor from cholesky().
template <int G, class T>
__device__ void chol_solve(const Grp<G>& g, const T* H, const T* invd, T* x, int n) {
  for (int k = 0; k < n; ++k) {
    const T xk = x[k] * invd[k];
    g.sync();
    if (g.lane == 0) x[k] = xk;
    for (int i = k + 1 + g.lane; i < n; i += G) x[i] -= H[i * n + k] * xk;
    g.sync();
  }
  for (int k = n - 1; k >= 0; --k) {
    const T xk = x[k] * invd[k];
    g.sync();
    if (g.lane == 0) x[k] = xk;
    for (int i = g.lane; i < k; i += G) x[i] -= H[k * n + i] * xk;
    g.sync();
  }
}

__device__ __forceinline__ bool mask_has(const int* mk, int id) { return (mk[id >> 5] >> (id & 31)) & 1; }

// H = M + J_A^T D_A J_A, b = rhs0 + J_A^T D_A a_ref,A; factor; an = H^-1 b.
template <int G, class T>
__device__ bool solve_active(const Grp<G>& g, const DevModel& m, const WsT<T>& w, int nr, const int* act) {
  const Layout& L = *w.L;
  const int nv = m.nv;
  const T* M = w.at(L.M); T* H = w.at(L.H);
  const T* J = w.at(L.J); const T* aref = w.at(L.aref); const T* Dr = w.at(L.Dr);
  const T* rhs0 = w.at(L.rhs0); T* an = w.at(L.an);
  const int* rowid = w.i + L.rowid;
  int* alist = w.i + L.alist;
  // compacted list of the active rows (in row order)
  int na = 0;
  for (int r0 = 0; r0 < nr; r0 += G) {
    const int r = r0 + g.lane;
    const bool a = r < nr && mask_has(act, rowid[r]);
    const unsigned bits = g.ballot(a);
    if (a) alist[na + __popc(bits & ((1u << g.lane) - 1u))] = r;
    na += __popc(bits);
  }
  g.sync();
  // lower triangle of H, then b: one entry per task
  const int ntri = nv * (nv + 1) / 2;
  for (int t = g.lane; t < ntri + nv; t += G) {
    if (t < ntri) {
      const int i = c_tri[t][0], j = c_tri[t][1];
      T h = M[i * nv + j];
      for (int k = 0; k < na; ++k) {
        const int r = alist[k];
        h += Dr[r] * J[r * nv + i] * J[r * nv + j];
      }
      H[i * nv + j] = h;
    } else {
      const int i = t - ntri;
      T b = rhs0[i];
      for (int k = 0; k < na; ++k) {
        const int r = alist[k];
        b += Dr[r] * aref[r] * J[r * nv + i];
      }
      an[i] = b;
    }
  }
  g.sync();
  const bool ok = cholesky(g, H, w.at(L.tmp2), nv);
  chol_solve(g, H, w.at(L.tmp2), an, nv);
  return ok;
}

// z = J a - a_ref for every row; returns the active set {z < 0} in newmask.
template <int G, class T>
__device__ void residual_set(const Grp<G>& g, const DevModel& m, const WsT<T>& w, int nr, const T* a, int* newmask) {
  const Layout& L = *w.L;
  const int nv = m.nv;
  const T* J = w.at(L.J); const T* aref = w.at(L.aref);
  T* z = w.at(L.z);
  const int* rowid = w.i + L.rowid;
  unsigned bits[MASKW] = {0u, 0u, 0u, 0u};
  for (int r = g.lane; r < nr; r += G) {
    T t = 0.0;
    for (int i = 0; i < nv; ++i) t += J[r * nv + i] * a[i];
    const T zr = t - aref[r];
    z[r] = zr;
    if (value(zr) < 0) bits[rowid[r] >> 5] |= 1u << (rowid[r] & 31);
  }
  for (int k = 0; k < MASKW; ++k) newmask[k] = (int)g.ior(bits[k]);
  g.sync();
}

// Exact line search along d = an - a: minimiser over alpha >= 0 of the convex
// piecewise quadratic primal cost; breakpoints compared without divisions.
// The search only selects the next Newton iterate, so it runs on values.
template <int G, class T>
__device__ double line_search(const Grp<G>& g, const DevModel& m, const WsT<T>& w, int nr) {
  const Layout& L = *w.L;
  const int nv = m.nv;
  const T* M = w.at(L.M); const T* J = w.at(L.J); const T* Dr = w.at(L.Dr);
  const T* a = w.at(L.a); const T* an = w.at(L.an); const T* rhs0 = w.at(L.rhs0);
  T* dl = w.at(L.tmp); T* z = w.at(L.z); T* s = w.at(L.s);
  for (int i = g.lane; i < nv; i += G) dl[i] = an[i] - a[i];
  g.sync();
  double c0 = 0, c1 = 0;
  for (int i = g.lane; i < nv; i += G) {
    double ma = 0, md = 0;
    for (int j = 0; j < nv; ++j) { ma += value(M[i * nv + j]) * value(a[j]); md += value(M[i * nv + j]) * value(dl[j]); }
    c0 += value(dl[i]) * (ma - value(rhs0[i]));
    c1 += value(dl[i]) * md;
  }
  const T* aref = w.at(L.aref);
  for (int r = g.lane; r < nr; r += G) {
    double t = 0, u = 0;
    for (int i = 0; i < nv; ++i) { t += value(J[r * nv + i]) * value(dl[i]); u += value(J[r * nv + i]) * value(a[i]); }
    s[r] = t;
    z[r] = u - value(aref[r]);
  }
  g.sync();
  double s0 = 0, s1 = 0;
  for (int r = g.lane; r < nr; r += G) {
    const double zr = value(z[r]), sr = value(s[r]), dr = value(Dr[r]);
    const bool act = zr < 0 || (zr == 0 && sr < 0);
    if (act) { s0 += dr * zr * sr; s1 += dr * sr * sr; }
  }
  double slope0 = g.sum(c0) + g.sum(s0), slope1 = g.sum(c1) + g.sum(s1);
  // sweep the breakpoints below the current root (each row toggles at most once)
  unsigned tog[MASKW] = {0u, 0u, 0u, 0u};
  for (int iter = 0; iter <= nr; ++iter) {
    // candidate rows: active ones leaving (s > 0) or inactive ones entering (s < 0, z > 0)
    // with breakpoint -z/s below the root -slope0/slope1 (slope1 > 0)
    int best = -1;
    double bz = 0, bs = 1;
    for (int r = g.lane; r < nr; r += G) {
      if ((tog[r >> 5] >> (r & 31)) & 1u) continue;
      const double zr = value(z[r]), sr = value(s[r]);
      const bool act = zr < 0 || (zr == 0 && sr < 0);
      const bool cand = act ? (sr > 0) : (sr < 0 && zr > 0);
      if (!cand) continue;
      // -z/s < -slope0/slope1  <=>  z slope1 > s slope0 (s > 0) or z slope1 < s slope0 (s < 0)
      const double lhs = zr * slope1, rhs = sr * slope0;
      const bool below = sr > 0 ? (lhs > rhs) : (lhs < rhs);
      if (!below) continue;
      // smaller breakpoint: -z/s < -bz/bs  <=>  z bs * sign > bz s * sign with sign(s bs)
      if (best < 0) { best = r; bz = zr; bs = sr; continue; }
      const double l2 = zr * bs, r2 = bz * sr;
      const bool smaller = (sr * bs > 0) ? (l2 > r2) : (l2 < r2);
      if (smaller) { best = r; bz = zr; bs = sr; }
    }
    // group arg-min over lanes
#pragma unroll
    for (int o = G / 2; o > 0; o >>= 1) {
      const int ob = __shfl_xor_sync(g.mask, best, o);
      const double oz = __shfl_xor_sync(g.mask, bz, o), os = __shfl_xor_sync(g.mask, bs, o);
      if (ob >= 0) {
        bool take = best < 0;
        if (!take) {
          const double l2 = oz * bs, r2 = bz * os;
          take = (os * bs > 0) ? (l2 > r2) : (l2 < r2);
          if (!take && !(l2 != r2)) take = ob < best;   // tie: lowest row index
        }
        if (take) { best = ob; bz = oz; bs = os; }
      }
    }
    if (best < 0) break;
    const double zb = value(z[best]), sb = value(s[best]), db = value(Dr[best]);
    const bool act = zb < 0 || (zb == 0 && sb < 0);
    const double dz = db * zb * sb, ds = db * sb * sb;
    if (act) { slope0 -= dz; slope1 -= ds; } else { slope0 += dz; slope1 += ds; }
    tog[best >> 5] |= 1u << (best & 31);
  }
  const double alpha = -slope0 / slope1;
  return alpha < 0 ? 0.0 : alpha;
}

// Unique minimiser of the primal problem -> an (= v').  With the active set A
// of the current iterate, an = H_A^-1 b_A is the minimiser of A's quadratic;
// it is the solution as soon as its own active set is A (the gradient of the
// primal cost vanishes there).  Otherwise Newton moves to the exact line
// minimum between the iterate and an.  The first candidate set is the final
// set of the previous right-hand side of this environment (pmask): when it is
// still right, one factorisation finishes the solve; when not, Newton starts
// from its solution.  pmask receives the final set.  In derivative scalars the
// final solve with the final set carries the implicit-function derivative.
// Returns 0 or an ENV_* code.
template <int G, class T>
__device__ int solve_constraints(const Grp<G>& g, const DevModel& m, const WsT<T>& w, int nr) {
  const Layout& L = *w.L;
  const int nv = m.nv;
  int* pm = w.i + L.pmask; int* am = w.i + L.amask;
  T* a = w.at(L.a); const T* an = w.at(L.an);
  int cur[MASKW], nxt[MASKW];
  for (int k = 0; k < MASKW; ++k) cur[k] = pm[k];
  bool ok = true;
  int status = ENV_SOLVER_NOCONV;
  for (int it = 0; it <= 50; ++it) {
    ok = solve_active(g, m, w, nr, cur) && ok;
    residual_set(g, m, w, nr, an, nxt);
    bool same = true;
    for (int k = 0; k < MASKW; ++k) same = same && (nxt[k] == cur[k]);
    if (same) { status = ENV_OK; break; }
    if (it == 0) {
      // start point of the Newton search: the solution of the first candidate set
      for (int i = g.lane; i < nv; i += G) a[i] = an[i];
      for (int k = 0; k < MASKW; ++k) cur[k] = nxt[k];
      g.sync();
      continue;
    }
    const double alpha = line_search(g, m, w, nr);
    const T* dl = w.at(L.tmp);
    for (int i = g.lane; i < nv; i += G) a[i] += alpha * dl[i];
    g.sync();
    residual_set(g, m, w, nr, (const T*)a, cur);
  }
  g.sync();
  if (g.lane == 0)
    for (int k = 0; k < MASKW; ++k) { pm[k] = cur[k]; am[k] = cur[k]; }
  g.sync();
  if (!ok) return ENV_SOLVER_NOCONV;
  return status;
}

// v' = F(q, v, u) (or F~ with cfd) into out[nv].  Returns 0 or an ENV_* code.
template <int G, class T>
__device__ int rhs(const Grp<G>& g, const DevModel& m, const WsT<T>& w, const T* q, const T* v,
                                const T* u, bool cfd, T* out) {
  const Layout& L = *w.L;
  kinematics(g, m, w, q);
  crba(g, m, w);
  rne_and_forces(g, m, w, q, v, u);
  collide(g, m, w, cfd);
  const int nr = make_rows(g, m, w, v, cfd);
  if (nr < 0) return ENV_ROW_OVERFLOW;
  const int st = solve_constraints(g, m, w, nr);
  const T* an = w.at(L.an);
  for (int i = g.lane; i < m.nv; i += G) out[i] = an[i];
  g.sync();
  return st;
}

// ------------------------------------------------------------------ integrator
// Explicit one-step schemes as partitioned tableaus on (q, v).  Stage s
// (s = 1 .. S-1) takes V_s = v_n + h sum_{j<s} av[s][j] K_j and
// Q_s = q_n (+) h sum_{j<=s} aq[s][j] V_j (V_0 = v_n; a diagonal position
// coefficient uses the stage's own new velocity), K_s = F(Q_s, V_s, u); the
// last stage is the step's result and its K the next step's K_0 (first same
// as last).  e = b - bhat: weights of the embedded error estimate of the
// adaptive schemes.  nzq / nzv / enz: bit j set where the coefficient is
// non-zero, so that the stage sums skip zeros with an integer test.
enum { METHOD_DOPRI5 = 0, METHOD_TSIT5 = 1, METHOD_EULER = 2, NMETHOD = 3 };
struct Tab {
  int S, adaptive;
  double aq[7][7], av[7][7];
  double e[7];
  unsigned nzq[7], nzv[7], enz;
};
__host__ __device__ constexpr void finish_tab(Tab& t) {
  for (int s = 0; s < 7; ++s) {
    t.nzq[s] = 0u; t.nzv[s] = 0u;
    for (int j = 0; j < 7; ++j) {
      if (t.aq[s][j] != 0.0) t.nzq[s] |= 1u << j;
      if (t.av[s][j] != 0.0) t.nzv[s] |= 1u << j;
    }
  }
  t.enz = 0u;
  for (int j = 0; j < 7; ++j)
    if (t.e[j] != 0.0) t.enz |= 1u << j;
}
// Dormand & Prince (1980) 5(4): row 7 = the 5th-order weights b.
__host__ __device__ constexpr Tab make_dopri5() {
  Tab t{7, 1,
        {},
        {{0, 0, 0, 0, 0, 0, 0},
         {1.0 / 5.0, 0, 0, 0, 0, 0, 0},
         {3.0 / 40.0, 9.0 / 40.0, 0, 0, 0, 0, 0},
         {44.0 / 45.0, -56.0 / 15.0, 32.0 / 9.0, 0, 0, 0, 0},
         {19372.0 / 6561.0, -25360.0 / 2187.0, 64448.0 / 6561.0, -212.0 / 729.0, 0, 0, 0},
         {9017.0 / 3168.0, -355.0 / 33.0, 46732.0 / 5247.0, 49.0 / 176.0, -5103.0 / 18656.0, 0, 0},
         {35.0 / 384.0, 0.0, 500.0 / 1113.0, 125.0 / 192.0, -2187.0 / 6784.0, 11.0 / 84.0, 0}},
        {35.0 / 384.0 - 5179.0 / 57600.0, 0.0, 500.0 / 1113.0 - 7571.0 / 16695.0, 125.0 / 192.0 - 393.0 / 640.0,
         -2187.0 / 6784.0 + 92097.0 / 339200.0, 11.0 / 84.0 - 187.0 / 2100.0, -1.0 / 40.0},
        {}, {}, 0u};
  for (int s = 0; s < 7; ++s)
    for (int j = 0; j < 7; ++j) t.aq[s][j] = t.av[s][j];
  finish_tab(t);
  return t;
}
// Tsitouras (2011) 5(4) (the paper's default solver): row 7 = b, e its
// published error weights.
__host__ __device__ constexpr Tab make_tsit5() {
  Tab t{7, 1,
        {},
        {{0, 0, 0, 0, 0, 0, 0},
         {0.161, 0, 0, 0, 0, 0, 0},
         {-0.008480655492356989, 0.335480655492357, 0, 0, 0, 0, 0},
         {2.897153057105493, -6.359448489975075, 4.3622954328695815, 0, 0, 0, 0},
         {5.325864828439257, -11.748883564062828, 7.4955393428898365, -0.09249506636175525, 0, 0, 0},
         {5.86145544294642, -12.92096931784711, 8.159367898576159, -0.071584973281401, -0.028269050394068383, 0, 0},
         {0.09646076681806523, 0.01, 0.4798896504144996, 1.379008574103742, -3.290069515436081, 2.324710524099774,
          0}},
        {-0.00178001105222577714, -0.0008164344596567469, 0.007880878010261995, -0.1447110071732629,
         0.5823571654525552, -0.45808210592918697, 0.015151515151515152},
        {}, {}, 0u};
  for (int s = 0; s < 7; ++s)
    for (int j = 0; j < 7; ++j) t.aq[s][j] = t.av[s][j];
  finish_tab(t);
  return t;
}
// Semi-implicit Euler with a fixed step (the MuJoCo XLA integrator the paper
// compares against): v_{n+1} = v_n + h K_0, q_{n+1} = q_n (+) h v_{n+1}.
__host__ __device__ constexpr Tab make_euler() {
  Tab t{2, 0, {}, {}, {}, {}, {}, 0u};
  t.av[1][0] = 1.0;
  t.aq[1][1] = 1.0;
  finish_tab(t);
  return t;
}
struct TabSet {
  Tab t[NMETHOD];
};
__host__ __device__ constexpr TabSet make_tabs() { return TabSet{{make_dopri5(), make_tsit5(), make_euler()}}; }
static __constant__ TabSet c_tabs = make_tabs();
#define TAB(mt) (c_tabs.t[(mt)])

// q (+) dq for every joint (free: translation + body-frame rotation exponential).
template <int G, class T>
__device__ void integrate_pos(const Grp<G>& g, const DevModel& m, const T* q, const T* dq, T* out) {
  for (int b = g.lane; b < m.nbody; b += G) {
    const int qa = m.b_qadr[b], va = m.b_vadr[b];
    if (m.b_jtype[b] == JNT_HINGE) { out[qa] = q[qa] + dq[va]; continue; }
    out[qa] = q[qa] + dq[va]; out[qa + 1] = q[qa + 1] + dq[va + 1]; out[qa + 2] = q[qa + 2] + dq[va + 2];
    const T* d = dq + va + 3;
    const T th2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    T cw, sk;
    if (value(th2) < 1e-2) {
      // |dq| < 0.1 rad: Taylor series of cos(th/2) and sin(th/2)/th in th^2
      // (the next terms are below 3e-20): no square root, sine or division
      cw = 1.0 + th2 * (-1.0 / 8.0 + th2 * (1.0 / 384.0 + th2 * (-1.0 / 46080.0 + th2 * (1.0 / 10321920.0))));
      sk = 0.5 + th2 * (-1.0 / 48.0 + th2 * (1.0 / 3840.0 + th2 * (-1.0 / 645120.0 + th2 * (1.0 / 185794560.0))));
    } else {
      const T th = sqrt(th2);
      T sn, cs;
      sincos(0.5 * th, &sn, &cs);
      cw = cs;
      sk = sn / th;
    }
    const T ex = sk * d[0], ey = sk * d[1], ez = sk * d[2];
    const T w0 = q[qa + 3], a0 = q[qa + 4], b0 = q[qa + 5], c0 = q[qa + 6];
    const T rw = w0 * cw - a0 * ex - b0 * ey - c0 * ez;
    const T rx = w0 * ex + a0 * cw + b0 * ez - c0 * ey;
    const T ry = w0 * ey - a0 * ez + b0 * cw + c0 * ex;
    const T rz = w0 * ez + a0 * ey - b0 * ex + c0 * cw;
    const T in = rsqrt_t(rw * rw + rx * rx + ry * ry + rz * rz);
    out[qa + 3] = rw * in; out[qa + 4] = rx * in; out[qa + 5] = ry * in; out[qa + 6] = rz * in;
  }
  g.sync();
}

// Magnitude used by the error norm for tangent component i of the positions.
__device__ __forceinline__ double pos_mag(const DevModel& m, const double* q, int i) {
  const int b = m.dof_body[i];
  if (m.b_jtype[b] == JNT_HINGE) return fabs(q[m.b_qadr[b]]);
  const int d = i - m.b_vadr[b];
  return d < 3 ? fabs(q[m.b_qadr[b] + d]) : 1.0;
}

// The new stages of one step of scheme mt (TAB(mt)) of size h from (qn, vn)
// with ka[0] = F(qn, vn): stage velocities kv[s], derivatives ka[s], the
// result in (qs, vs) and its derivative in ka[(S-1) nv].  hook(s, status)
// runs after the right-hand side of stage s (the workspace then holds that
// evaluation).  Returns the worst stage status.
template <int G, class Hook>
__device__ int rk_stages(const Grp<G>& g, const DevModel& m, const Ws& w, const double* u, double h, int mt,
                         Hook&& hook) {
  const Layout& L = *w.L;
  const int nv = m.nv, S = TAB(mt).S;
  const double* qn = w.at(L.qn); const double* vn = w.at(L.vn);
  double* qs = w.at(L.qs); double* vs = w.at(L.vs);
  double* kv = w.at(L.kv); double* ka = w.at(L.ka); double* dq = w.at(L.dq);
  int st = 0;
  for (int i = g.lane; i < nv; i += G) kv[i] = vn[i];
  g.sync();
  for (int s = 1; s < S; ++s) {
    const unsigned mq = TAB(mt).nzq[s], mv = TAB(mt).nzv[s];
    for (int i = g.lane; i < nv; i += G) {
      double sq = 0, sv = 0;
      for (int j = 0; j < s; ++j) {
        if ((mq >> j) & 1u) sq += TAB(mt).aq[s][j] * kv[j * nv + i];
        if ((mv >> j) & 1u) sv += TAB(mt).av[s][j] * ka[j * nv + i];
      }
      const double vv = vn[i] + h * sv;
      if ((mq >> s) & 1u) sq += TAB(mt).aq[s][s] * vv;
      dq[i] = h * sq;
      vs[i] = vv;
      kv[s * nv + i] = vv;
    }
    g.sync();
    integrate_pos(g, m, qn, dq, qs);
    const int r = rhs(g, m, w, qs, vs, u, false, ka + s * nv);
    if (r > st) st = r;
    hook(s, r);
  }
  return st;
}

// One attempt of scheme mt of size h from (qn, vn) with ka[0] = F(qn, vn).
// Leaves the result in (qs, vs) and its derivative in ka[(S-1) nv]; returns
// the RMS error norm of the embedded estimate (NaN-safe: non-finite -> +inf;
// 0 for a fixed-step scheme) and the worst stage status.
template <int G>
__device__ double rk_attempt(const Grp<G>& g, const DevModel& m, const Ws& w, const double* u, double h, int mt,
                             double rtol, double atol, int* st_out) {
  const Layout& L = *w.L;
  const int nv = m.nv;
  const double* qn = w.at(L.qn); const double* vn = w.at(L.vn);
  const double* qs = w.at(L.qs); const double* vs = w.at(L.vs);
  const double* kv = w.at(L.kv); const double* ka = w.at(L.ka);
  const int st = rk_stages(g, m, w, u, h, mt, [](int, int) {});
  *st_out = st;
  if (!TAB(mt).adaptive) return 0.0;
  const unsigned enz = TAB(mt).enz;
  double acc = 0;
  for (int i = g.lane; i < nv; i += G) {
    double ep = 0, ev = 0;
    for (int j = 0; j < 7; ++j) {
      if (!((enz >> j) & 1u)) continue;
      const double c = TAB(mt).e[j];
      ep += c * kv[j * nv + i];
      ev += c * ka[j * nv + i];
    }
    ep *= h; ev *= h;
    const double sp = atol + rtol * fmax(pos_mag(m, qn, i), pos_mag(m, qs, i));
    const double sv = atol + rtol * fmax(fabs(vn[i]), fabs(vs[i]));
    const double r1 = ep / sp, r2 = ev / sv;
    acc += r1 * r1 + r2 * r2;
  }
  acc = g.sum(acc);
  const double err = sqrt(acc / (2.0 * nv));
  return isfinite(err) ? err : INFINITY;
}

}  // namespace dmx
