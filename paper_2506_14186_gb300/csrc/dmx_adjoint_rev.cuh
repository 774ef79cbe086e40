// Reverse-mode discrete adjoint of the taped rollout (discretize-then-
// optimize over the accepted steps, App. C.2), with the straight-through CFD
// treatment of Sec. 4: a group of G lanes per environment, like the forward
// kernels, persistent (groups take the next environment from a counter).
//
// For every accepted step, in reverse order, the step map
// (q_n, v_n, u) -> (q_{n+1}, v_{n+1}) of the taped scheme (Dormand-Prince,
// Tsitouras or semi-implicit Euler, dmx_device.cuh) with the taped step size
// h (held constant) is transposed stage by stage:
//   stage s state  V_s = v_n + h sum_{j<s} av_sj K_j,  Q_s = q_n (+) h sum_{j<=s} aq_sj V_j,
//   K_s = F(Q_s, V_s, u)  (s = 0..S-2),  (q_{n+1}, v_{n+1}) = (Q_{S-1}, V_{S-1}).
// Walking s = S-1..0, the stage cotangents (Qbar_s, Vbar_s) collect the
// contributions of the later stages, K_s's cotangent goes through the
// right-hand side VJP at (Q_s, V_s) (of F~ at the F stage states when cfd:
// straight-through), and (q_n, v_n, u) receive the rest.  The stage states
// come from a forward recompute of the segment between two checkpoints (the
// tape holds the state every K accepted steps), stored per step in a
// per-group buffer: q_n, V_0..V_{S-1} and t_n.
//
// Without the CFD right-hand side (cfd = 0) the reverse sweep needs the
// right-hand sides that the segment recompute already evaluated (same stage
// states, same inputs).  When P.snapbuf is given, the recompute copies the
// part of each stage's workspace that the VJP reads to device memory
// (K steps x (S - 1) stages per group) and the reverse sweep restores it instead of
// evaluating the right-hand side a second time: device memory traded for
// FP64 work.  The final active set of a stage does not depend on the
// warm start of its Newton search, so the restored workspace equals a
// recomputed one.
#pragma once
#include <cuda_runtime.h>

#include "dmx_adjoint.h"
#include "dmx_vjp.cuh"

namespace dmx {

__device__ __forceinline__ double rev_boundary(double T, int NI, int k) { return k >= NI ? T : T * k / NI; }
__device__ __forceinline__ int rev_interval(double T, int NI, double t) {
  int k = 0;
  while (k + 1 < NI && t >= rev_boundary(T, NI, k + 1)) ++k;
  return k;
}

// Workspace of the right-hand side just evaluated (status st) -> snapshot dst.
template <int G>
__device__ void snap_save(const Grp<G>& g, const DevModel& m, const Ws& w, double* dst, int st) {
  const Layout& L = *w.L;
  const SnapOff o = snap_offsets(m, L);
  const int nr = (st == ENV_ROW_OVERFLOW) ? 0 : w.i[L.slotrow + m.nslot];
  const double* d = w.d;
  for (int i = g.lane; i < o.n1; i += G) dst[i] = d[L.R + i];
  for (int i = g.lane; i < o.n2; i += G) dst[o.o2 + i] = d[L.H + i];
  for (int i = g.lane; i < 16 * m.nslot; i += G) dst[o.o3 + i] = d[L.ct + i];
  for (int i = g.lane; i < 2 * m.nslot; i += G) dst[o.o3 + 16 * m.nslot + i] = d[L.csv + i];
  for (int i = g.lane; i < nr * m.nv; i += G) dst[o.o4 + i] = d[L.J + i];
  for (int i = g.lane; i < nr; i += G) { dst[o.o5 + i] = d[L.Dr + i]; dst[o.o6 + i] = d[L.z + i]; }
  int* di = reinterpret_cast<int*>(dst + o.oi);
  if (g.lane == 0) { di[0] = st; di[1] = nr; }
  for (int i = g.lane; i <= m.nslot; i += G) di[2 + i] = w.i[L.slotrow + i];
  for (int i = g.lane; i < nr; i += G) di[3 + m.nslot + i] = w.i[L.rowid + i];
  for (int i = g.lane; i < MASKW; i += G) di[3 + m.nslot + L.rcap + i] = w.i[L.amask + i];
}
// Snapshot src -> workspace (the state rhs() leaves for rhs_vjp, except the
// contact records and Jacobian rows, which the VJP reads from the snapshot
// itself: see snap_view); returns the status.
template <int G>
__device__ int snap_restore(const Grp<G>& g, const DevModel& m, const Ws& w, const double* src) {
  const Layout& L = *w.L;
  const SnapOff o = snap_offsets(m, L);
  const int* si = reinterpret_cast<const int*>(src + o.oi);
  const int st = si[0], nr = si[1];
  double* d = w.d;
  for (int i = g.lane; i < o.n1; i += G) d[L.R + i] = src[i];
  for (int i = g.lane; i < o.n2; i += G) d[L.H + i] = src[o.o2 + i];
  for (int i = g.lane; i < 2 * m.nslot; i += G) d[L.csv + i] = src[o.o3 + 16 * m.nslot + i];
  for (int i = g.lane; i < nr; i += G) { d[L.Dr + i] = src[o.o5 + i]; d[L.z + i] = src[o.o6 + i]; }
  for (int i = g.lane; i <= m.nslot; i += G) w.i[L.slotrow + i] = si[2 + i];
  for (int i = g.lane; i < nr; i += G) w.i[L.rowid + i] = si[3 + m.nslot + i];
  for (int i = g.lane; i < MASKW; i += G) w.i[L.amask + i] = si[3 + m.nslot + L.rcap + i];
  g.sync();
  return st;
}
// The workspace view whose VJP reads the snapshot's contact records and rows.
__device__ __forceinline__ Ws snap_view(const DevModel& m, const Ws& w, const double* src) {
  const SnapOff o = snap_offsets(m, *w.L);
  Ws v = w;
  v.xct = src + o.o3;
  v.xJ = src + o.o4;
  return v;
}

// (qnb, vnb, ub) = transposed step map of scheme mt applied to (Qb, Vb) = the
// cotangent of (q_{n+1}, v_{n+1}); reads q_n from b.qn and V_0..V_{S-1} from
// b.vst.  Qb and Vb are consumed (left zero).  snaps: the step's S - 1 stage
// snapshots (SN doubles each), or null to evaluate each stage's right-hand
// side.  Returns the worst right-hand-side status.
template <int G>
__device__ int rk_step_vjp(const Grp<G>& g, const DevModel& m, const Ws& w, const WsB& b, const double* u,
                           double h, int mt, bool cfd, const double* snaps, int SN) {
  const Layout& L = *w.L;
  const LayoutBar& LB = *b.L;
  const int nv = m.nv, S = TAB(mt).S;
  const double* qn = b.at(LB.qn); const double* vst = b.at(LB.vst);
  double* dq = b.at(LB.dq); double* dqb = b.at(LB.dqb); double* Qs = b.at(LB.Qs);
  double* kab = b.at(LB.kab); double* kvb = b.at(LB.kvb);
  double* Qb = b.at(LB.Qb); double* Vb = b.at(LB.Vb);
  double* qnb = b.at(LB.qnb); double* vnb = b.at(LB.vnb); double* ub = b.at(LB.ub);
  int st = 0;
  for (int i = g.lane; i < 6 * nv; i += G) { kab[i] = 0.0; kvb[i] = 0.0; }
  for (int i = g.lane; i < m.nq; i += G) qnb[i] = 0.0;
  for (int i = g.lane; i < nv; i += G) vnb[i] = 0.0;
  for (int a = g.lane; a < m.nu; a += G) ub[a] = 0.0;
  g.sync();
  for (int s = S - 1; s >= 0; --s) {
    const unsigned mq = TAB(mt).nzq[s], mv = TAB(mt).nzv[s];
    if (s >= 1) {
      for (int i = g.lane; i < nv; i += G) {
        double sq = 0;
        for (int j = 0; j <= s; ++j)
          if ((mq >> j) & 1u) sq += TAB(mt).aq[s][j] * vst[j * nv + i];
        dq[i] = h * sq;
      }
      g.sync();
      if (s <= S - 2) integrate_pos(g, m, qn, (const double*)dq, Qs);
    } else {
      for (int i = g.lane; i < m.nq; i += G) Qs[i] = qn[i];
      g.sync();
    }
    if (s <= S - 2) {
      const double* Vs = vst + s * nv;
      const double* sn = snaps ? snaps + (size_t)s * SN : nullptr;
      const int r = sn ? snap_restore(g, m, w, sn) : rhs(g, m, w, (const double*)Qs, Vs, u, cfd, w.at(L.ka));
      if (r > st) st = r;
      rhs_vjp(g, m, sn ? snap_view(m, w, sn) : w, b, Qs, Vs, u, cfd, r, kab + s * nv, Qb, Vb, ub);
      for (int i = g.lane; i < nv; i += G) Vb[i] += kvb[s * nv + i];   // V_s in the later stages' positions
      g.sync();
    }
    if (s >= 1) {
      // positions first: a diagonal coefficient puts V_s into Q_s itself
      integrate_pos_vjp(g, m, qn, dq, Qb, qnb, dqb);
      for (int i = g.lane; i < nv; i += G) {
        for (int j = 0; j < s; ++j)
          if ((mq >> j) & 1u) kvb[j * nv + i] += h * TAB(mt).aq[s][j] * dqb[i];
        if ((mq >> s) & 1u) Vb[i] += h * TAB(mt).aq[s][s] * dqb[i];
        vnb[i] += Vb[i];
        for (int j = 0; j < s; ++j)
          if ((mv >> j) & 1u) kab[j * nv + i] += h * TAB(mt).av[s][j] * Vb[i];
      }
    } else {
      for (int i = g.lane; i < m.nq; i += G) qnb[i] += Qb[i];
      for (int i = g.lane; i < nv; i += G) vnb[i] += Vb[i];
    }
    g.sync();
    for (int i = g.lane; i < m.nq; i += G) Qb[i] = 0.0;
    for (int i = g.lane; i < nv; i += G) Vb[i] = 0.0;
    g.sync();
  }
  return st;
}

template <int G>
__global__ void __launch_bounds__(32, 1) k_adjoint_rev(AdjParams P) {
  extern __shared__ double smem[];
  __shared__ Layout sL;
  __shared__ LayoutBar sB;
  if (threadIdx.x == 0) { sL = P.L; sB = P.LB; }
  __syncthreads();
  const DevModel& m = *P.model;
  Grp<G> g;
  const int ngb = blockDim.x / G, gib = threadIdx.x / G;
  // doubles per environment and the cotangent workspace's offset in them (with
  // stage snapshots it overlays the arrays only the segment recompute uses)
  const int per = P.per;
  const Ws w{smem + (size_t)gib * per, reinterpret_cast<int*>(smem + (size_t)ngb * per) + (size_t)gib * sL.ni, &sL};
  const WsB b{smem + (size_t)gib * per + P.barofs, &sB};
  const int nq = m.nq, nv = m.nv, nx = nq + nv, nu = m.nu;
  const int RW = rev_row_doubles(m);
  const int mt = P.method, S = TAB(mt).S;
  double* seg = P.segbuf + (size_t)(blockIdx.x * ngb + gib) * P.K * RW;
  const bool use_snap = P.snapbuf != nullptr && P.cfd == 0;
  const int SN = P.SN;
  double* snb = use_snap ? P.snapbuf + (size_t)(blockIdx.x * ngb + gib) * P.K * (S - 1) * SN : nullptr;
  double* qn = w.at(sL.qn); double* vn = w.at(sL.vn); double* u = w.at(sL.u); double* ka = w.at(sL.ka);
  double* xbar = sL.xbar >= 0 ? w.at(sL.xbar) : b.at(sB.xb);   // kept across the recompute phases
  for (;;) {
    int env = 0;
    if (g.lane == 0) env = atomicAdd(P.queue, 1);
    env = g.bcast(env, 0);
    if (env >= P.B) break;
    const int N = P.tape_n[env];
    const double T = P.T[env];
    for (int i = g.lane; i < nx; i += G) xbar[i] = P.xT_bar[(size_t)i * P.B + env];
    if (P.ctrl_bar)
      for (int i = g.lane; i < P.NI * nu; i += G) P.ctrl_bar[(size_t)i * P.B + env] = 0.0;
    if (g.lane == 0) for (int k = 0; k < MASKW; ++k) w.i[sL.pmask + k] = 0;
    g.sync();
    int worst = 0;
    for (int c = N > 0 ? (N - 1) / P.K : -1; c >= 0; --c) {
      const int n0 = c * P.K, n1 = min(n0 + P.K, N);
      // ---- forward recompute of the segment from checkpoint c: q_n, V_0..V_5, t_n per step
      const double* ck = P.ckpt + (size_t)c * (nx + 1) * P.B;
      for (int i = g.lane; i < nq; i += G) qn[i] = ck[(size_t)i * P.B + env];
      for (int i = g.lane; i < nv; i += G) vn[i] = ck[(size_t)(nq + i) * P.B + env];
      double t = ck[(size_t)nx * P.B + env];
      int k = rev_interval(T, P.NI, t);
      for (int a = g.lane; a < nu; a += G) u[a] = P.ctrl[((size_t)k * nu + a) * P.B + env];
      g.sync();
      {
        const int st0 = rhs(g, m, w, (const double*)qn, (const double*)vn, (const double*)u, false, ka);
        if (use_snap) snap_save(g, m, w, snb, st0);
      }
      for (int n = n0; n < n1; ++n) {
        double* row = seg + (size_t)(n - n0) * RW;
        const double h = P.hlog[(size_t)n * P.B + env];
        double* sn_step = use_snap ? snb + (size_t)(n - n0) * (S - 1) * SN : nullptr;
        double* sn_next = (use_snap && n + 1 < n1) ? sn_step + (size_t)(S - 1) * SN : nullptr;
        rk_stages(g, m, w, (const double*)u, h, mt, [&](int s, int r) {
          if (s <= S - 2) { if (sn_step) snap_save(g, m, w, sn_step + (size_t)s * SN, r); }
          else if (sn_next) snap_save(g, m, w, sn_next, r);   // the last stage = stage 0 of the next step
        });
        const double* kv = w.at(sL.kv);
        for (int i = g.lane; i < nq; i += G) row[i] = qn[i];
        for (int i = g.lane; i < S * nv; i += G) row[nq + i] = kv[i];
        if (g.lane == 0) row[nq + 7 * nv] = t;
        if (n == n1 - 1) break;
        const double tn = rev_boundary(T, P.NI, k + 1);
        const bool reached = (h == tn - t) || (t + h >= tn);
        t = reached ? tn : t + h;
        const double* qs = w.at(sL.qs); const double* vs = w.at(sL.vs);
        g.sync();
        for (int i = g.lane; i < nq; i += G) qn[i] = qs[i];
        for (int i = g.lane; i < nv; i += G) { vn[i] = vs[i]; ka[i] = ka[(S - 1) * nv + i]; }
        g.sync();
        if (reached && k + 1 < P.NI) {
          ++k;
          for (int a = g.lane; a < nu; a += G) u[a] = P.ctrl[((size_t)k * nu + a) * P.B + env];
          g.sync();
          const int stb = rhs(g, m, w, (const double*)qn, (const double*)vn, (const double*)u, false, ka);
          if (sn_next) snap_save(g, m, w, sn_next, stb);   // the new control's stage 0
        }
      }
      __threadfence_block();
      g.sync();
      // ---- reverse sweep over the segment's steps
      double* bq = b.at(sB.qn); double* bv = b.at(sB.vst);
      double* Qb = b.at(sB.Qb); double* Vb = b.at(sB.Vb);
      for (int n = n1 - 1; n >= n0; --n) {
        const double* row = seg + (size_t)(n - n0) * RW;
        const double tn0 = row[nq + 7 * nv];
        const int kn = rev_interval(T, P.NI, tn0);
        const double h = P.hlog[(size_t)n * P.B + env];
        const double tb = rev_boundary(T, P.NI, kn + 1);
        const bool reached = (h == tb - tn0) || (tn0 + h >= tb);
        if (reached && P.xb_bar)
          for (int i = g.lane; i < nx; i += G) xbar[i] += P.xb_bar[((size_t)(kn + 1) * nx + i) * P.B + env];
        for (int i = g.lane; i < nq; i += G) bq[i] = row[i];
        for (int i = g.lane; i < S * nv; i += G) bv[i] = row[nq + i];
        for (int a = g.lane; a < nu; a += G) u[a] = P.ctrl[((size_t)kn * nu + a) * P.B + env];
        g.sync();
        for (int i = g.lane; i < nq; i += G) Qb[i] = xbar[i];
        for (int i = g.lane; i < nv; i += G) Vb[i] = xbar[nq + i];
        g.sync();
        const int st = rk_step_vjp(g, m, w, b, (const double*)u, h, mt, P.cfd != 0,
                                   use_snap ? snb + (size_t)(n - n0) * (S - 1) * SN : nullptr, SN);
        if (st > worst) worst = st;
        const double* qnb = b.at(sB.qnb); const double* vnb = b.at(sB.vnb); const double* ub = b.at(sB.ub);
        for (int i = g.lane; i < nq; i += G) xbar[i] = qnb[i];
        for (int i = g.lane; i < nv; i += G) xbar[nq + i] = vnb[i];
        if (P.ctrl_bar)
          for (int a = g.lane; a < nu; a += G) P.ctrl_bar[((size_t)kn * nu + a) * P.B + env] += ub[a];
        g.sync();
      }
      g.sync();
    }
    if (P.xb_bar)
      for (int i = g.lane; i < nx; i += G) xbar[i] += P.xb_bar[(size_t)i * P.B + env];
    g.sync();
    // a right-hand side whose rows overflowed the workspace has no derivative: mark the result
    const double bad = (worst == ENV_ROW_OVERFLOW) ? __longlong_as_double(0x7ff8000000000000ll) : 0.0;
    for (int i = g.lane; i < nx; i += G) P.x0_bar[(size_t)i * P.B + env] = xbar[i] + bad;
    g.sync();
  }
}

// (dF/d(q, v, u))^T abar for a batch of states (q [nq][B], v [nv][B],
// u [nu][B], abar [nv][B]) into qbar [nq][B], vbar [nv][B], ubar [nu][B]
// (ubar only when nu > 0); status [B] = rhs status.
template <int G>
__global__ void __launch_bounds__(32) k_eval_rhs_vjp(AdjParams P, const double* q, const double* v, const double* u,
                                                      const double* abar, double* qbar, double* vbar, double* ubar,
                                                      int* status) {
  extern __shared__ double smem[];
  __shared__ Layout sL;
  __shared__ LayoutBar sB;
  if (threadIdx.x == 0) { sL = P.L; sB = P.LB; }
  __syncthreads();
  const DevModel& m = *P.model;
  Grp<G> g;
  const int ngb = blockDim.x / G, gib = threadIdx.x / G;
  const int per = sL.nd + sB.nd;
  const Ws w{smem + (size_t)gib * per, reinterpret_cast<int*>(smem + (size_t)ngb * per) + (size_t)gib * sL.ni, &sL};
  const WsB b{smem + (size_t)gib * per + sL.nd, &sB};
  const int env = blockIdx.x * ngb + gib;
  if (env >= P.B) return;
  double* qs = b.at(sB.Qs); double* vs = b.at(sB.vst); double* uu = w.at(sL.u); double* ab = b.at(sB.kab);
  double* qb = b.at(sB.qnb); double* vb = b.at(sB.vnb); double* ub = b.at(sB.ub);
  for (int i = g.lane; i < m.nq; i += G) { qs[i] = q[(size_t)i * P.B + env]; qb[i] = 0.0; }
  for (int i = g.lane; i < m.nv; i += G) {
    vs[i] = v[(size_t)i * P.B + env]; ab[i] = abar[(size_t)i * P.B + env]; vb[i] = 0.0;
  }
  for (int i = g.lane; i < m.nu; i += G) { uu[i] = u[(size_t)i * P.B + env]; ub[i] = 0.0; }
  if (g.lane == 0) for (int k = 0; k < MASKW; ++k) w.i[sL.pmask + k] = 0;
  g.sync();
  const int st = rhs(g, m, w, (const double*)qs, (const double*)vs, (const double*)uu, P.cfd != 0, w.at(sL.ka));
  rhs_vjp(g, m, w, b, qs, vs, uu, P.cfd != 0, st, ab, qb, vb, ub);
  for (int i = g.lane; i < m.nq; i += G) qbar[(size_t)i * P.B + env] = qb[i];
  for (int i = g.lane; i < m.nv; i += G) vbar[(size_t)i * P.B + env] = vb[i];
  if (ubar)
    for (int i = g.lane; i < m.nu; i += G) ubar[(size_t)i * P.B + env] = ub[i];
  if (g.lane == 0) status[env] = st;
}
template <int G>
cudaError_t launch_eval_rhs_vjp_g(const AdjParams& P, const double* q, const double* v, const double* u,
                                  const double* abar, double* qbar, double* vbar, double* ubar, int* status,
                                  int threads, size_t smem, cudaStream_t st) {
  auto k = k_eval_rhs_vjp<G>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (int)(((size_t)P.B * G + threads - 1) / threads);
  k<<<blocks, threads, smem, st>>>(P, q, v, u, abar, qbar, vbar, ubar, status);
  return cudaGetLastError();
}

template <int G>
cudaError_t launch_adjoint_rev_g(const AdjParams& P, int blocks, int threads, size_t smem, cudaStream_t st) {
  auto k = k_adjoint_rev<G>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<blocks, threads, smem, st>>>(P);
  return cudaGetLastError();
}
template <int G>
int occupancy_adjoint_rev_g(int threads, size_t smem) {
  auto k = k_adjoint_rev<G>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
  return n;
}

}  // namespace dmx
