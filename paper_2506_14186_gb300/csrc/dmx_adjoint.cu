// Discrete adjoint of the taped rollout (discretize-then-optimize over the
// accepted steps, App. C.2), with the straight-through CFD treatment of Sec. 4.
//
// One warp per environment.  For every accepted step, in reverse order, the
// warp evaluates the step map (q_n, v_n, u) -> (q_{n+1}, v_{n+1}) once
// in forward-mode derivative scalars with ONE INPUT DIRECTION PER LANE: all
// lanes run the same instruction stream (the primal part is identical in
// every lane), so on GB300, where an FP64 warp instruction costs the same
// whatever its active lanes, one dual step yields 32 Jacobian columns.  The
// adjoint update is then lane-local: lane d gets
//   xbar_n[d] = sum_i xbar_{n+1}[i] * d x_{n+1}[i] / d input_d,
// and likewise the control cotangent of the step's interval.  Step sizes are
// held constant (they come from the tape).  The constraint solve is
// differentiated through its final active set (implicit function theorem: the
// derivative scalars flow through the last factorisation).  With cfd the
// stage derivatives come from the CFD right-hand side F~ evaluated at the
// stage states of F (straight-through: values of F, derivatives of F~).
//
// The states at the step starts are recomputed segment by segment from the
// checkpoints the forward pass stored every K accepted steps.
#include <cuda_runtime.h>

#include "dmx_adjoint.h"
#include "dmx_device.cuh"

namespace dmx {
template <int G> cudaError_t launch_adjoint_rev_g(const AdjParams&, int, int, size_t, cudaStream_t);
template <int G> int occupancy_adjoint_rev_g(int, size_t);
template <int G>
cudaError_t launch_eval_rhs_vjp_g(const AdjParams&, const double*, const double*, const double*, const double*, double*,
                                  double*, double*, int*, int, size_t, cudaStream_t);
}  // namespace dmx

namespace dmx {

constexpr int ADJ_WARPS = 2;          // warps (environments) per block
constexpr int ADJ_WS = 4096;          // per-lane workspace (derivative scalars)
constexpr int ADJ_WI = 512;           // per-lane workspace (ints)

__device__ __forceinline__ double adj_boundary(double T, int NI, int k) { return k >= NI ? T : T * k / NI; }
__device__ __forceinline__ int adj_interval(double T, int NI, double t) {
  int k = 0;
  while (k + 1 < NI && t >= adj_boundary(T, NI, k + 1)) ++k;
  return k;
}

// One step of scheme mt (TAB(mt)) of size h in derivative scalars from (qn, vn)
// in the dual workspace; leaves the result in (qs, vs).  Stage derivatives of
// F; with cfd the tangents of F~ replace them (straight-through).
__device__ int dual_step(const Grp<1>& g, const DevModel& m, const WsT<Dual>& w, const Dual* u, double h, int mt,
                         bool cfd, int* maskF, int* maskC) {
  const Layout& L = *w.L;
  const int nv = m.nv, S = TAB(mt).S;
  const Dual* qn = w.at(L.qn); const Dual* vn = w.at(L.vn);
  Dual* qs = w.at(L.qs); Dual* vs = w.at(L.vs);
  Dual* kv = w.at(L.kv); Dual* ka = w.at(L.ka); Dual* dq = w.at(L.dq);
  int* pm = w.i + L.pmask;
  int st = 0;
  for (int s = 0; s < S; ++s) {
    if (s == 0) {
      for (int i = 0; i < m.nq; ++i) qs[i] = qn[i];
      for (int i = 0; i < nv; ++i) vs[i] = vn[i];
    } else {
      const unsigned mq = TAB(mt).nzq[s], mv = TAB(mt).nzv[s];
      for (int i = 0; i < nv; ++i) {
        Dual sq = 0.0, sv = 0.0;
        for (int j = 0; j < s; ++j) {
          if ((mq >> j) & 1u) sq += TAB(mt).aq[s][j] * kv[j * nv + i];
          if ((mv >> j) & 1u) sv += TAB(mt).av[s][j] * ka[j * nv + i];
        }
        vs[i] = vn[i] + h * sv;
        if ((mq >> s) & 1u) sq += TAB(mt).aq[s][s] * vs[i];
        dq[i] = h * sq;
      }
      integrate_pos(g, m, qn, (const Dual*)dq, qs);
    }
    for (int i = 0; i < nv; ++i) kv[s * nv + i] = vs[i];
    if (s == S - 1) break;                      // the last stage's derivative is not part of the step
    for (int k = 0; k < MASKW; ++k) pm[k] = maskF[k];
    int r = rhs(g, m, w, (const Dual*)qs, (const Dual*)vs, u, false, ka + s * nv);
    for (int k = 0; k < MASKW; ++k) maskF[k] = pm[k];
    if (r > st) st = r;
    if (cfd) {
      Dual* tmpa = w.at(L.tmp);                 // F~ into tmp, keep the values of F
      for (int k = 0; k < MASKW; ++k) pm[k] = maskC[k];
      r = rhs(g, m, w, (const Dual*)qs, (const Dual*)vs, u, true, tmpa);
      for (int k = 0; k < MASKW; ++k) maskC[k] = pm[k];
      if (r > st) st = r;
      for (int i = 0; i < nv; ++i) ka[s * nv + i].d = tmpa[i].d;
    }
  }
  return st;
}

__global__ void __launch_bounds__(32 * ADJ_WARPS) k_adjoint(AdjParams P) {
  __shared__ Layout sL;
  __shared__ double s_xbar[ADJ_WARPS][MAXQ + MAXV];
  __shared__ double s_t[ADJ_WARPS];
  if (threadIdx.x == 0) sL = P.L;
  __syncthreads();
  const DevModel& m = *P.model;
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int gwarp = blockIdx.x * ADJ_WARPS + wib;
  const unsigned full = 0xffffffffu;
  const int nq = m.nq, nv = m.nv, nx = nq + nv, nu = m.nu, D = nx + nu + (P.p_bar ? P.np : 0);
  const int npass = (D + 31) / 32;
  Grp<1> g;                                     // every lane is a group of one
  Dual wsd[ADJ_WS];
  int wsi[ADJ_WI];
  WsT<Dual> wd{wsd, wsi, &sL};
  const WsT<double> wp{reinterpret_cast<double*>(wsd), wsi, &sL};
  double* xbar = s_xbar[wib];
  double* seg = P.segbuf + (size_t)gwarp * P.K * (nx + 1);
  int maskF[MASKW], maskC[MASKW];
  for (;;) {
    int env = 0;
    if (lane == 0) env = atomicAdd(P.queue, 1);
    env = __shfl_sync(full, env, 0);
    if (env >= P.B) break;
    const int N = P.tape_n[env];
    const double T = P.T[env];
    for (int i = lane; i < nx; i += 32) xbar[i] = P.xT_bar[(size_t)i * P.B + env];
    if (P.ctrl_bar)
      for (int i = lane; i < P.NI * nu; i += 32) P.ctrl_bar[(size_t)i * P.B + env] = 0.0;
    for (int k = 0; k < MASKW; ++k) { maskF[k] = 0; maskC[k] = 0; }
    double pacc[4] = {0.0, 0.0, 0.0, 0.0};       // this lane's parameter directions
    __syncwarp();
    for (int c = N > 0 ? (N - 1) / P.K : -1; c >= 0; --c) {
      const int n0 = c * P.K, n1 = min(n0 + P.K, N);
      // ---- forward recompute of the segment from checkpoint c (values, every lane)
      const double* ck = P.ckpt + (size_t)c * (nx + 1) * P.B;
      double* qn = wp.at(sL.qn); double* vn = wp.at(sL.vn);
      for (int i = 0; i < nq; ++i) qn[i] = ck[(size_t)i * P.B + env];
      for (int i = 0; i < nv; ++i) vn[i] = ck[(size_t)(nq + i) * P.B + env];
      double t = ck[(size_t)nx * P.B + env];
      int k = adj_interval(T, P.NI, t);
      double* u = wp.at(sL.u);
      for (int a = 0; a < nu; ++a) u[a] = P.ctrl[((size_t)k * nu + a) * P.B + env];
      for (int kk = 0; kk < MASKW; ++kk) wsi[sL.pmask + kk] = maskF[kk];
      rhs(g, m, wp, (const double*)qn, (const double*)vn, (const double*)u, false, wp.at(sL.ka));
      for (int n = n0; n < n1; ++n) {
        if (lane == 0) {
          double* row = seg + (size_t)(n - n0) * (nx + 1);
          for (int i = 0; i < nq; ++i) row[i] = qn[i];
          for (int i = 0; i < nv; ++i) row[nq + i] = vn[i];
          row[nx] = t;
        }
        if (n == n1 - 1) break;
        const double h = P.hlog[(size_t)n * P.B + env];
        int st;
        rk_attempt(g, m, wp, (const double*)u, h, P.method, 1.0, 1.0, &st);
        const double tn = adj_boundary(T, P.NI, k + 1);
        const bool reached = (h == tn - t) || (t + h >= tn);
        t = reached ? tn : t + h;
        const double* qs = wp.at(sL.qs); const double* vs = wp.at(sL.vs);
        double* ka = wp.at(sL.ka);
        for (int i = 0; i < nq; ++i) qn[i] = qs[i];
        for (int i = 0; i < nv; ++i) { vn[i] = vs[i]; ka[i] = ka[(TAB(P.method).S - 1) * nv + i]; }
        if (reached && k + 1 < P.NI) {
          ++k;
          for (int a = 0; a < nu; ++a) u[a] = P.ctrl[((size_t)k * nu + a) * P.B + env];
          rhs(g, m, wp, (const double*)qn, (const double*)vn, (const double*)u, false, ka);
        }
      }
      for (int kk = 0; kk < MASKW; ++kk) maskF[kk] = wsi[sL.pmask + kk];
      __syncwarp();
      // ---- reverse sweep over the segment's steps
      for (int n = n1 - 1; n >= n0; --n) {
        const double* row = seg + (size_t)(n - n0) * (nx + 1);
        const double tn0 = row[nx];
        const int kn = adj_interval(T, P.NI, tn0);
        const double h = P.hlog[(size_t)n * P.B + env];
        const double tb = adj_boundary(T, P.NI, kn + 1);
        const bool reached = (h == tb - tn0) || (tn0 + h >= tb);
        if (reached && P.xb_bar)
          for (int i = lane; i < nx; i += 32) xbar[i] += P.xb_bar[((size_t)(kn + 1) * nx + i) * P.B + env];
        __syncwarp();
        double gdir[4];
        for (int p = 0; p < npass; ++p) {
          const int d = p * 32 + lane;
          wd.pdir = (d >= nx + nu && d < D) ? d - nx - nu : -1;   // a model-parameter direction
          Dual* qd = wd.at(sL.qn); Dual* vd = wd.at(sL.vn); Dual* ud = wd.at(sL.u);
          for (int i = 0; i < nq; ++i) qd[i] = Dual(row[i], d == i ? 1.0 : 0.0);
          for (int i = 0; i < nv; ++i) vd[i] = Dual(row[nq + i], d == nq + i ? 1.0 : 0.0);
          for (int a = 0; a < nu; ++a) ud[a] = Dual(P.ctrl[((size_t)kn * nu + a) * P.B + env], d == nx + a ? 1.0 : 0.0);
          dual_step(g, m, wd, (const Dual*)ud, h, P.method, P.cfd != 0, maskF, maskC);
          const Dual* qs = wd.at(sL.qs); const Dual* vs = wd.at(sL.vs);
          double acc = 0.0;
          for (int i = 0; i < nq; ++i) acc += xbar[i] * qs[i].d;
          for (int i = 0; i < nv; ++i) acc += xbar[nq + i] * vs[i].d;
          gdir[p] = acc;
        }
        __syncwarp();
        for (int p = 0; p < npass; ++p) {
          const int d = p * 32 + lane;
          if (d < nx) xbar[d] = gdir[p];
          else if (d < nx + nu) { if (P.ctrl_bar) P.ctrl_bar[((size_t)kn * nu + (d - nx)) * P.B + env] += gdir[p]; }
          else if (d < D) pacc[p] += gdir[p];
        }
        __syncwarp();
      }
    }
    for (int p = 0; p < npass; ++p) {
      const int d = p * 32 + lane;
      if (d >= nx + nu && d < D) P.p_bar[(size_t)(d - nx - nu) * P.B + env] = pacc[p];
    }
    if (P.xb_bar)
      for (int i = lane; i < nx; i += 32) xbar[i] += P.xb_bar[(size_t)i * P.B + env];
    __syncwarp();
    for (int i = lane; i < nx; i += 32) P.x0_bar[(size_t)i * P.B + env] = xbar[i];
    __syncwarp();
  }
  (void)s_t;
}

cudaError_t launch_adjoint(const AdjParams& P, int blocks, cudaStream_t st) {
  k_adjoint<<<blocks, 32 * ADJ_WARPS, 0, st>>>(P);
  return cudaGetLastError();
}

// Sum of every row of x [n][B]: block k strides over row k, then a fixed
// shuffle tree and a fixed shared-memory sum (the same order every call).
__global__ void __launch_bounds__(256) k_row_sums(const double* x, int B, double* out) {
  __shared__ double part[8];
  const double* row = x + (size_t)blockIdx.x * B;
  double acc = 0.0;
  for (int e = threadIdx.x; e < B; e += blockDim.x) acc += row[e];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += part[w];
    out[blockIdx.x] = s;
  }
}
// Derivative of every body's translational inverse weight at qpos0 (the
// A_hat model constant, trace(Jc M^-1 Jc^T) / 3) with respect to the
// model parameter pdir (a body mass): the set-up computation of
// k_body_invweight in derivative scalars, one environment, one lane, the
// workspace in device memory (ws: nd derivative scalars then ni ints).
__global__ void k_body_invweight_tangent(const DevModel* mp, const double* qpos0, int rcap, int pdir, Dual* ws,
                                         Dual* scratch, double* dinvw) {
  __shared__ Layout sL;
  const DevModel& m = *mp;
  if (threadIdx.x != 0) return;
  sL = make_layout(m, rcap);
  Grp<1> g;
  WsT<Dual> w{ws, reinterpret_cast<int*>(ws + sL.nd), &sL};
  w.pdir = pdir;
  Dual* q = scratch;
  Dual* col = scratch + m.nq;
  Dual* x = col + m.nv;
  for (int i = 0; i < m.nq; ++i) q[i] = Dual(qpos0[i], 0.0);
  kinematics(g, m, w, q);
  crba(g, m, w);
  Dual* H = w.at(sL.H); const Dual* M = w.at(sL.M);
  for (int i = 0; i < m.nv * m.nv; ++i) H[i] = M[i];
  cholesky(g, H, w.at(sL.tmp2), m.nv);
  const Dual* S = w.at(sL.sd); const Dual* C = w.at(sL.com);
  for (int b = 0; b < m.nbody; ++b) {
    Dual tr = 0.0;
    for (int ax = 0; ax < 3; ++ax) {
      for (int i = 0; i < m.nv; ++i) {
        const bool moves = (m.b_anc[b] >> m.dof_body[i]) & 1u;
        Dual pv[3] = {0.0, 0.0, 0.0};
        if (moves) {
          cross3(S + 6 * i, C + 3 * b, pv);
          pv[0] += S[6 * i + 3]; pv[1] += S[6 * i + 4]; pv[2] += S[6 * i + 5];
        }
        col[i] = pv[ax];
        x[i] = pv[ax];
      }
      chol_solve(g, H, w.at(sL.tmp2), x, m.nv);
      for (int i = 0; i < m.nv; ++i) tr += col[i] * x[i];
    }
    dinvw[b] = (tr / 3.0).d;
  }
}

cudaError_t launch_body_invweight_tangent(const DevModel* m, const double* qpos0, int rcap, int pdir, void* ws,
                                          void* scratch, double* dinvw, cudaStream_t st) {
  k_body_invweight_tangent<<<1, 32, 0, st>>>(m, qpos0, rcap, pdir, static_cast<Dual*>(ws),
                                             static_cast<Dual*>(scratch), dinvw);
  return cudaGetLastError();
}

cudaError_t launch_row_sums(const double* x, int n, int B, double* out, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_row_sums<<<n, 256, 0, st>>>(x, B, out);
  return cudaGetLastError();
}
int adjoint_warps_per_block() { return ADJ_WARPS; }
int adjoint_workspace_limit() { return ADJ_WS; }
int adjoint_int_limit() { return ADJ_WI; }

cudaError_t launch_adjoint_rev(int G, const AdjParams& P, int blocks, int threads, size_t smem, cudaStream_t st) {
  switch (G) {
    case 2: return launch_adjoint_rev_g<2>(P, blocks, threads, smem, st);
    case 4: return launch_adjoint_rev_g<4>(P, blocks, threads, smem, st);
    case 8: return launch_adjoint_rev_g<8>(P, blocks, threads, smem, st);
    case 16: return launch_adjoint_rev_g<16>(P, blocks, threads, smem, st);
    case 32: return launch_adjoint_rev_g<32>(P, blocks, threads, smem, st);
  }
  return cudaErrorInvalidValue;
}
int adjoint_rev_occupancy(int G, int threads, size_t smem) {
  switch (G) {
    case 2: return occupancy_adjoint_rev_g<2>(threads, smem);
    case 4: return occupancy_adjoint_rev_g<4>(threads, smem);
    case 8: return occupancy_adjoint_rev_g<8>(threads, smem);
    case 16: return occupancy_adjoint_rev_g<16>(threads, smem);
    case 32: return occupancy_adjoint_rev_g<32>(threads, smem);
  }
  return 0;
}
cudaError_t launch_eval_rhs_vjp(int G, const AdjParams& P, const double* q, const double* v, const double* u,
                                const double* abar, double* qbar, double* vbar, double* ubar, int* status, int threads,
                                size_t smem, cudaStream_t st) {
  switch (G) {
    case 2: return launch_eval_rhs_vjp_g<2>(P, q, v, u, abar, qbar, vbar, ubar, status, threads, smem, st);
    case 4: return launch_eval_rhs_vjp_g<4>(P, q, v, u, abar, qbar, vbar, ubar, status, threads, smem, st);
    case 8: return launch_eval_rhs_vjp_g<8>(P, q, v, u, abar, qbar, vbar, ubar, status, threads, smem, st);
    case 16: return launch_eval_rhs_vjp_g<16>(P, q, v, u, abar, qbar, vbar, ubar, status, threads, smem, st);
    case 32: return launch_eval_rhs_vjp_g<32>(P, q, v, u, abar, qbar, vbar, ubar, status, threads, smem, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dmx
