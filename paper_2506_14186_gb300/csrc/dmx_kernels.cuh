// Rollout kernels: the persistent refill form (one launch integrates every
// environment to its horizon; a group of G lanes takes the next environment
// from an atomic counter when its own is done) and the plain form (one launch
// performs one step attempt of every environment, state kept in HBM).
//
// Step logic (Sec. 3.1, App. B): attempt h = min(h_prop, next boundary - t)
// (steps never straddle a control change; a step that would leave less than
// 1e-12 s before the boundary is stretched to it); accept iff the RMS error
// norm <= 1; PID factor 0.9 err^-(P+I)/5 err_prev^(P/5) clipped to [0.2, 10]
// with P = 0.2, I = 0.4; on rejection h *= max(0.2, 0.9 err^-1/5).  A
// fixed-step scheme (semi-implicit Euler) accepts every step and proposes h0
// after each.
#pragma once
#include <cuda_runtime.h>

#include "dmx_device.cuh"
#include "dmx_kernels.h"

namespace dmx {

__device__ __forceinline__ double boundary_time(double T, int NI, int k) { return k >= NI ? T : T * k / NI; }

struct EnvState {
  double t, h, lerrp, T;   // lerrp: log of the previous accepted step's error norm
  int k, nacc, nrej, att, st, done;
};

template <int G>
__device__ void load_ctrl(const Grp<G>& g, const DevModel& m, const Ws& w, const RolloutParams& P, int env, int k) {
  double* u = w.at(w.L->u);
  for (int a = g.lane; a < m.nu; a += G) u[a] = P.ctrl[((size_t)k * m.nu + a) * P.B + env];
  g.sync();
}

template <int G>
__device__ void store_state(const Grp<G>& g, const DevModel& m, const Ws& w, const RolloutParams& P, int env,
                            double* dst /* [nx][B] */) {
  const double* qn = w.at(w.L->qn); const double* vn = w.at(w.L->vn);
  for (int i = g.lane; i < m.nq; i += G) dst[(size_t)i * P.B + env] = qn[i];
  for (int i = g.lane; i < m.nv; i += G) dst[(size_t)(m.nq + i) * P.B + env] = vn[i];
}

template <int G>
__device__ void write_checkpoint(const Grp<G>& g, const DevModel& m, const Ws& w, const RolloutParams& P, int env,
                                 int c, double t) {
  const int nx = m.nq + m.nv;
  double* ck = P.ckpt + (size_t)c * (nx + 1) * P.B;
  store_state(g, m, w, P, env, ck);
  if (g.lane == 0) ck[(size_t)nx * P.B + env] = t;
}

// Initial state, first right-hand side; returns the initial environment state.
template <int G>
__device__ void env_start(const Grp<G>& g, const DevModel& m, const Ws& w, const RolloutParams& P, int env,
                          EnvState& s) {
  const Layout& L = *w.L;
  double* qn = w.at(L.qn); double* vn = w.at(L.vn);
  bool fin = true;
  for (int i = g.lane; i < m.nq; i += G) { qn[i] = P.x0[(size_t)i * P.B + env]; fin = fin && isfinite(qn[i]); }
  for (int i = g.lane; i < m.nv; i += G) { vn[i] = P.x0[(size_t)(m.nq + i) * P.B + env]; fin = fin && isfinite(vn[i]); }
  int bad = fin ? 0 : 1;
  bad = g.isum(bad);
  if (g.lane == 0) for (int k = 0; k < MASKW; ++k) w.i[L.pmask + k] = 0;
  g.sync();
  s.t = 0.0; s.h = P.h0; s.lerrp = 0.0; s.T = P.T[env];
  s.k = 0; s.nacc = 0; s.nrej = 0; s.att = 0; s.st = ENV_OK; s.done = 0;
  if (P.xb) store_state(g, m, w, P, env, P.xb);
  if (P.ckpt) write_checkpoint(g, m, w, P, env, 0, 0.0);
  if (bad) { s.st = ENV_NONFINITE; s.done = 1; return; }
  if (m.nu) load_ctrl(g, m, w, P, env, 0);
  const int st = rhs(g, m, w, qn, vn, w.at(L.u), false, w.at(L.ka));
  if (st != ENV_OK) { s.st = st; s.done = 1; }
}

// One step attempt with its bookkeeping.
template <int G>
__device__ void env_attempt(const Grp<G>& g, const DevModel& m, const Ws& w, const RolloutParams& P, int env,
                            EnvState& s) {
  const Layout& L = *w.L;
  if (s.t >= s.T) { s.done = 1; return; }
  if (s.att >= P.max_steps) { s.st = ENV_MAX_STEPS; s.done = 1; return; }
  const double tn = boundary_time(s.T, P.NI, s.k + 1);
  const double hb = tn - s.t;
  const bool clamped = s.h >= hb || hb - s.h < 1e-12;
  const double ht = clamped ? hb : s.h;
  if (ht < 1e-12) { s.st = ENV_H_UNDERFLOW; s.done = 1; return; }
  int stage_st = 0;
  const int mt = P.method;
  const double err = rk_attempt(g, m, w, w.at(L.u), ht, mt, P.rtol, P.atol, &stage_st);
  ++s.att;
  if (err <= 1.0) {
    if (stage_st != ENV_OK) { s.st = stage_st; s.done = 1; return; }
    if (P.hlog && g.lane == 0) P.hlog[(size_t)s.nacc * P.B + env] = ht;
    const bool reached = clamped || (s.t + ht >= tn);
    s.t = reached ? tn : s.t + ht;
    double* qn = w.at(L.qn); double* vn = w.at(L.vn);
    const double* qs = w.at(L.qs); const double* vs = w.at(L.vs);
    double* ka = w.at(L.ka);
    const int last = (TAB(mt).S - 1) * m.nv;
    for (int i = g.lane; i < m.nq; i += G) qn[i] = qs[i];
    for (int i = g.lane; i < m.nv; i += G) { vn[i] = vs[i]; ka[i] = ka[last + i]; }
    g.sync();
    ++s.nacc;
    if (TAB(mt).adaptive) {
      const double errf = fmax(err, 1e-10);
      // 0.9 err^-(P+I)/5 err_prev^(P/5) as one exponential of the logs (the
      // previous log is carried over)
      const double lerr = log(errf);
      double fac = 0.9 * exp(-(0.6 / 5.0) * lerr + (0.2 / 5.0) * s.lerrp);
      fac = fmin(10.0, fmax(0.2, fac));
      s.lerrp = lerr;
      s.h = ht * fac;
    } else {
      s.h = P.h0;   // fixed step (the last step of an interval may have been shortened)
    }
    if (P.ckpt && (s.nacc % P.K) == 0) write_checkpoint(g, m, w, P, env, s.nacc / P.K, s.t);
    if (reached) {
      ++s.k;
      if (P.xb) store_state(g, m, w, P, env, P.xb + (size_t)s.k * (m.nq + m.nv) * P.B);
      if (s.k < P.NI) {
        if (m.nu) load_ctrl(g, m, w, P, env, s.k);
        const int st = rhs(g, m, w, qn, vn, w.at(L.u), false, ka);
        if (st != ENV_OK) { s.st = st; s.done = 1; return; }
      }
    }
    if (s.t >= s.T) s.done = 1;
  } else {
    ++s.nrej;
    const double fac = isfinite(err) ? fmax(0.2, 0.9 * pow(err, -1.0 / 5.0)) : 0.2;
    s.h = ht * fac;
  }
}

template <int G>
__device__ void env_finish(const Grp<G>& g, const DevModel& m, const Ws& w, const RolloutParams& P, int env,
                           const EnvState& s) {
  store_state(g, m, w, P, env, P.xT);
  if (g.lane == 0) {
    if (P.nsteps) P.nsteps[env] = s.nacc;
    if (P.nrej) P.nrej[env] = s.nrej;
    if (P.status) P.status[env] = s.st;
    if (P.tape_n) P.tape_n[env] = s.nacc;
  }
}

// Plain form: per-environment integrator state kept in HBM between launches.
template <int G>
__device__ void load_step_state(const Grp<G>& g, const DevModel& m, const Ws& w, const RolloutParams& P,
                                const StepState& S, int env, EnvState& s) {
  const Layout& L = *w.L;
  double* qn = w.at(L.qn); double* vn = w.at(L.vn); double* ka = w.at(L.ka);
  for (int i = g.lane; i < m.nq; i += G) qn[i] = S.q[(size_t)i * P.B + env];
  for (int i = g.lane; i < m.nv; i += G) { vn[i] = S.v[(size_t)i * P.B + env]; ka[i] = S.ka0[(size_t)i * P.B + env]; }
  if (g.lane == 0)
    for (int k = 0; k < MASKW; ++k) w.i[L.pmask + k] = S.pmask[(size_t)k * P.B + env];
  s.t = S.t[env]; s.h = S.h[env]; s.lerrp = S.lerrp[env]; s.T = P.T[env];
  s.k = S.k[env]; s.nacc = S.nacc[env]; s.nrej = S.nrej[env]; s.att = S.att[env]; s.st = S.st[env];
  s.done = S.done[env];
  g.sync();
  if (m.nu) load_ctrl(g, m, w, P, env, s.k < P.NI ? s.k : P.NI - 1);
}
template <int G>
__device__ void save_step_state(const Grp<G>& g, const DevModel& m, const Ws& w, const RolloutParams& P,
                                const StepState& S, int env, const EnvState& s) {
  const Layout& L = *w.L;
  const double* qn = w.at(L.qn); const double* vn = w.at(L.vn); const double* ka = w.at(L.ka);
  for (int i = g.lane; i < m.nq; i += G) S.q[(size_t)i * P.B + env] = qn[i];
  for (int i = g.lane; i < m.nv; i += G) { S.v[(size_t)i * P.B + env] = vn[i]; S.ka0[(size_t)i * P.B + env] = ka[i]; }
  if (g.lane == 0) {
    for (int k = 0; k < MASKW; ++k) S.pmask[(size_t)k * P.B + env] = w.i[L.pmask + k];
    S.t[env] = s.t; S.h[env] = s.h; S.lerrp[env] = s.lerrp;
    S.k[env] = s.k; S.nacc[env] = s.nacc; S.nrej[env] = s.nrej; S.att[env] = s.att; S.st[env] = s.st;
    S.done[env] = s.done;
  }
}

template <int G>
__device__ Ws group_workspace(const RolloutParams& P, const Layout* L) {
  extern __shared__ double smem[];
  const int ngb = blockDim.x / G;
  const int gib = threadIdx.x / G;
  Ws w;
  w.d = smem + (size_t)gib * L->nd;
  w.i = reinterpret_cast<int*>(smem + (size_t)ngb * L->nd) + (size_t)gib * L->ni;
  w.L = L;
  return w;
}

// Persistent form: loop { take next env; integrate it to T }.
template <int G>
__global__ void __launch_bounds__(32, 1) k_rollout_persistent(RolloutParams P) {
  __shared__ Layout sL;
  if (threadIdx.x == 0) sL = P.L;
  __syncthreads();
  const DevModel& m = *P.model;
  Grp<G> g;
  const Ws w = group_workspace<G>(P, &sL);
  // One loop level: every pass makes one step attempt of the group's
  // environment, taking the next environment first when the group has none.
  // The groups of a warp thus meet at every attempt; with a per-environment
  // inner loop, a group whose environment finished would wait at that loop's
  // exit (where the warp reconverges) for the warp's slowest environment.
  EnvState s;
  int env = -1;
  for (;;) {
    if (env < 0) {
      int e = 0;
      if (g.lane == 0) e = atomicAdd(P.queue, 1);
      e = g.bcast(e, 0);
      if (e >= P.B) break;
      env = e;
      env_start(g, m, w, P, env, s);
    }
    if (!s.done) env_attempt(g, m, w, P, env, s);
    if (s.done) {
      env_finish(g, m, w, P, env, s);
      env = -1;
    }
  }
}

// Plain form, initialisation launch: state of every environment into HBM.
template <int G>
__global__ void __launch_bounds__(32, 1) k_step_init(RolloutParams P, StepState S) {
  __shared__ Layout sL;
  if (threadIdx.x == 0) sL = P.L;
  __syncthreads();
  const DevModel& m = *P.model;
  Grp<G> g;
  const Ws w = group_workspace<G>(P, &sL);
  const int env = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  if (env >= P.B) return;
  EnvState s;
  env_start(g, m, w, P, env, s);
  save_step_state(g, m, w, P, S, env, s);
  if (s.done) {
    env_finish(g, m, w, P, env, s);
    if (g.lane == 0) atomicSub(S.active, 1);
  }
}

// Plain form, one attempt of every unfinished environment.
template <int G>
__global__ void __launch_bounds__(32, 1) k_step(RolloutParams P, StepState S) {
  __shared__ Layout sL;
  if (threadIdx.x == 0) sL = P.L;
  __syncthreads();
  const DevModel& m = *P.model;
  Grp<G> g;
  const Ws w = group_workspace<G>(P, &sL);
  const int env = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  if (env >= P.B) return;
  if (S.done[env]) return;
  EnvState s;
  load_step_state(g, m, w, P, S, env, s);
  env_attempt(g, m, w, P, env, s);
  save_step_state(g, m, w, P, S, env, s);
  if (s.done) {
    env_finish(g, m, w, P, env, s);
    if (g.lane == 0) atomicSub(S.active, 1);
  }
}

// Right-hand side of a batch of states (q [nq][B], v [nv][B], u [nu][B]) into
// a [nv][B]; info [4][B]: status, rows, active rows, Newton solves.
template <int G>
__global__ void __launch_bounds__(32, 1) k_eval_rhs(RolloutParams P, const double* q, const double* v, const double* u,
                                                  int cfd, double* a, int* info) {
  __shared__ Layout sL;
  if (threadIdx.x == 0) sL = P.L;
  __syncthreads();
  const DevModel& m = *P.model;
  Grp<G> g;
  const Ws w = group_workspace<G>(P, &sL);
  const int env = (blockIdx.x * blockDim.x + threadIdx.x) / G;
  if (env >= P.B) return;
  double* qs = w.at(sL.qs); double* vs = w.at(sL.vs); double* uu = w.at(sL.u);
  for (int i = g.lane; i < m.nq; i += G) qs[i] = q[(size_t)i * P.B + env];
  for (int i = g.lane; i < m.nv; i += G) vs[i] = v[(size_t)i * P.B + env];
  for (int i = g.lane; i < m.nu; i += G) uu[i] = u[(size_t)i * P.B + env];
  if (g.lane == 0) for (int k = 0; k < MASKW; ++k) w.i[sL.pmask + k] = 0;
  g.sync();
  double* res = w.at(sL.ka);
  const int st = rhs(g, m, w, qs, vs, uu, cfd != 0, res);
  for (int i = g.lane; i < m.nv; i += G) a[(size_t)i * P.B + env] = res[i];
  if (g.lane == 0) {
    int nact = 0;
    for (int k = 0; k < MASKW; ++k) nact += __popc(w.i[sL.amask + k]);
    info[env] = st;
    info[P.B + env] = w.i[sL.slotrow + m.nslot];
    info[2 * P.B + env] = nact;
    info[3 * P.B + env] = 0;
  }
}

template <int G>
cudaError_t launch_eval_rhs_g(const RolloutParams& P, const double* q, const double* v, const double* u, int cfd,
                              double* a, int* info, int threads, size_t smem, cudaStream_t st) {
  auto k = k_eval_rhs<G>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const int blocks = (int)(((size_t)P.B * G + threads - 1) / threads);
  k<<<blocks, threads, smem, st>>>(P, q, v, u, cfd, a, info);
  return cudaGetLastError();
}

template <int G>
cudaError_t launch_persistent_g(const RolloutParams& P, int blocks, int threads, size_t smem, cudaStream_t st) {
  auto k = k_rollout_persistent<G>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k<<<blocks, threads, smem, st>>>(P);
  return cudaGetLastError();
}
template <int G>
int occupancy_g(int threads, size_t smem) {
  auto k = k_rollout_persistent<G>;
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, k, threads, smem) != cudaSuccess) return 0;
  return n;
}
template <int G>
cudaError_t launch_step_g(const RolloutParams& P, const StepState& S, bool init, int threads, size_t smem,
                          cudaStream_t st) {
  const int blocks = (int)(((size_t)P.B * G + threads - 1) / threads);
  if (init) {
    auto k = k_step_init<G>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<blocks, threads, smem, st>>>(P, S);
  } else {
    auto k = k_step<G>;
    cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    k<<<blocks, threads, smem, st>>>(P, S);
  }
  return cudaGetLastError();
}

}  // namespace dmx
