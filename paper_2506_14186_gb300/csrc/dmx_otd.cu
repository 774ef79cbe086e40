// Optimize-then-discretize gradient (App. C.2, Eq. adjoint-equations:
// BacksolveAdjoint), with the straight-through CFD variant of App. C.4.
//
// With x = (q, v), x' = f(x, u) = (G(q) v, F(q, v, u)) and a_x(T) = dL/dx(T),
// the continuous adjoint a_x' = -a_x^T df/dx, a_u' = -a_x^T df/du is integrated
// BACKWARD from T together with the state itself (constant memory: only x(T)
// is needed), in reversed time s = T - t: dx/ds = -f, da/ds = +(df/dx)^T a.
// The backward solve takes its own adaptive steps (the forward scheme's
// tableau, error norm over the state's 2 nv tangent components and every
// adjoint component, the PID controller of App. B), never straddling a
// control-interval boundary; boundary cotangents enter as jumps of a_x, the
// control adjoint is collected per interval.  df/dx^T a = (d(G v)/dq^T a_q +
// dF/dq^T a_v, G^T a_q + dF/dv^T a_v): the F part is the right-hand-side VJP
// (of F~ when cfd: straight-through, the state still follows F), the G part
// the quaternion kinematics q' = q (x) (0, w) / 2 of a free joint (identity
// for translations and hinges).
//
// A group of G lanes per environment, persistent (groups take the next
// environment from a counter), workspaces in shared memory: the forward
// right-hand side, its cotangent workspace and the stage data of the
// augmented state.
#include <cuda_runtime.h>

#include <algorithm>
#include <string>

#include "dmx.h"
#include "dmx_adjoint.h"
#include "dmx_runtime.h"
#include "dmx_vjp.cuh"

namespace dmx {

struct OtdParams {
  const DevModel* model;
  Layout L;
  LayoutBar LB;
  int B, NI, max_steps, cfd, method;
  double rtol, atol, h0;
  const double* xT;       // [nx][B] states at T
  const double* ctrl;     // [NI][nu][B]
  const double* T;        // [B]
  const double* xT_bar;   // [nx][B]
  const double* xb_bar;   // [NI+1][nx][B] or null
  double* x0_bar;         // [nx][B]
  double* ctrl_bar;       // [NI][nu][B] or null
  int* steps;             // [B] accepted backward steps, or null
  int* status;            // [B] DMX_ENV_* of the backward solve, or null
  int per, barofs, otdofs, na;   // doubles per environment; cotangent and augmented-state offsets; nx + nu
  int* queue;
};

__device__ __forceinline__ double otd_boundary(double T, int NI, int k) { return k >= NI ? T : T * k / NI; }

// Kinematic part of the adjoint right-hand side: kq += (d(G v)/dq)^T aq,
// kv += G^T aq (one body per task).
template <int G>
__device__ void kin_adjoint(const Grp<G>& g, const DevModel& m, const double* q, const double* v, const double* aq,
                            double* kq, double* kv) {
  for (int b = g.lane; b < m.nbody; b += G) {
    const int qa = m.b_qadr[b], va = m.b_vadr[b];
    if (m.b_jtype[b] == JNT_HINGE) { kv[va] += aq[qa]; continue; }
    for (int i = 0; i < 3; ++i) kv[va + i] += aq[qa + i];
    const double w = q[qa + 3], x = q[qa + 4], y = q[qa + 5], z = q[qa + 6];
    const double a = v[va + 3], bb = v[va + 4], c = v[va + 5];
    const double Aw = aq[qa + 3], Ax = aq[qa + 4], Ay = aq[qa + 5], Az = aq[qa + 6];
    kq[qa + 3] += 0.5 * (a * Ax + bb * Ay + c * Az);
    kq[qa + 4] += 0.5 * (-a * Aw - c * Ay + bb * Az);
    kq[qa + 5] += 0.5 * (-bb * Aw + c * Ax - a * Az);
    kq[qa + 6] += 0.5 * (-c * Aw - bb * Ax + a * Ay);
    kv[va + 3] += 0.5 * (-x * Aw + w * Ax + z * Ay - y * Az);
    kv[va + 4] += 0.5 * (-y * Aw - z * Ax + w * Ay + x * Az);
    kv[va + 5] += 0.5 * (-z * Aw + y * Ax - x * Ay + w * Az);
  }
  g.sync();
}

// Stage s of the augmented backward step: F at (qs, vs) into kf, the adjoint
// right-hand side at (qs, vs, as) into ka (nq + nv + nu).  Returns the worst
// right-hand-side status.
template <int G>
__device__ int otd_stage(const Grp<G>& g, const DevModel& m, const Ws& w, const WsB& b, const double* qs,
                         const double* vs, const double* u, const double* as, bool cfd, double* kf, double* ka) {
  const LayoutBar& LB = *b.L;
  const int nq = m.nq, nv = m.nv, nu = m.nu;
  int st = rhs(g, m, w, qs, vs, u, false, kf);
  if (cfd) {
    const int s2 = rhs(g, m, w, qs, vs, u, true, w.at(w.L->tmp));   // F~ for the derivative
    if (s2 > st) st = s2;
  }
  double* qb = b.at(LB.qnb); double* vb = b.at(LB.vnb); double* ub = b.at(LB.ub);
  for (int i = g.lane; i < nq; i += G) qb[i] = 0.0;
  for (int i = g.lane; i < nv; i += G) vb[i] = 0.0;
  for (int i = g.lane; i < nu; i += G) ub[i] = 0.0;
  g.sync();
  rhs_vjp(g, m, w, b, qs, vs, u, cfd, st, as + nq, qb, vb, ub);
  for (int i = g.lane; i < nq; i += G) ka[i] = qb[i];
  for (int i = g.lane; i < nv; i += G) ka[nq + i] = vb[i];
  for (int i = g.lane; i < nu; i += G) ka[nq + nv + i] = ub[i];
  g.sync();
  kin_adjoint(g, m, qs, vs, as, ka, ka + nq);
  return st;
}

template <int G>
__global__ void __launch_bounds__(32, 1) k_adjoint_otd(OtdParams P) {
  extern __shared__ double smem[];
  __shared__ Layout sL;
  __shared__ LayoutBar sB;
  if (threadIdx.x == 0) { sL = P.L; sB = P.LB; }
  __syncthreads();
  const DevModel& m = *P.model;
  Grp<G> g;
  const int ngb = blockDim.x / G, gib = threadIdx.x / G;
  const Ws w{smem + (size_t)gib * P.per, reinterpret_cast<int*>(smem + (size_t)ngb * P.per) + (size_t)gib * sL.ni,
             &sL};
  const WsB b{smem + (size_t)gib * P.per + P.barofs, &sB};
  const int nq = m.nq, nv = m.nv, nx = nq + nv, nu = m.nu, na = P.na;
  const int mt = P.method, S = TAB(mt).S;
  double* a = w.d + P.otdofs;          // adjoint (a_q, a_v, a_u)
  double* as = a + na;                 // stage adjoint
  double* a7 = as + na;                // result of the attempt
  double* ka = a7 + na;                // [S][na] adjoint stage derivatives
  double* qn = w.at(sL.qn); double* vn = w.at(sL.vn);
  double* qs = w.at(sL.qs); double* vs = w.at(sL.vs);
  double* kv = w.at(sL.kv); double* kf = w.at(sL.ka); double* dq = w.at(sL.dq);
  double* u = w.at(sL.u);
  for (;;) {
    int env = 0;
    if (g.lane == 0) env = atomicAdd(P.queue, 1);
    env = g.bcast(env, 0);
    if (env >= P.B) break;
    const double T = P.T[env];
    for (int i = g.lane; i < nq; i += G) qn[i] = P.xT[(size_t)i * P.B + env];
    for (int i = g.lane; i < nv; i += G) vn[i] = P.xT[(size_t)(nq + i) * P.B + env];
    for (int i = g.lane; i < na; i += G) {
      double x = i < nx ? P.xT_bar[(size_t)i * P.B + env] : 0.0;
      if (i < nx && P.xb_bar) x += P.xb_bar[((size_t)P.NI * nx + i) * P.B + env];
      a[i] = x;
    }
    if (P.ctrl_bar)
      for (int i = g.lane; i < P.NI * nu; i += G) P.ctrl_bar[(size_t)i * P.B + env] = 0.0;
    if (g.lane == 0) for (int k = 0; k < MASKW; ++k) w.i[sL.pmask + k] = 0;
    g.sync();
    int k = P.NI - 1, steps = 0, attempts = 0, status = ENV_OK;
    double t = T, h = P.h0, lerrp = 0.0;
    while (t > 0.0 && k >= 0) {
      if (attempts >= P.max_steps) { status = ENV_MAX_STEPS; break; }
      const double tlo = otd_boundary(T, P.NI, k);
      const double hb = t - tlo;
      const bool clamped = h >= hb || hb - h < 1e-12;
      const double ht = clamped ? hb : h;
      if (ht < 1e-12) { status = ENV_H_UNDERFLOW; break; }
      for (int i = g.lane; i < nu; i += G) u[i] = P.ctrl[((size_t)k * nu + i) * P.B + env];
      for (int i = g.lane; i < nv; i += G) kv[i] = vn[i];
      g.sync();
      int st = otd_stage(g, m, w, b, qn, vn, u, a, P.cfd != 0, kf, ka);
      for (int s = 1; s < S; ++s) {
        const unsigned mq = TAB(mt).nzq[s], mv = TAB(mt).nzv[s];
        for (int i = g.lane; i < nv; i += G) {
          double sq = 0, sv = 0;
          for (int j = 0; j < s; ++j) {
            if ((mq >> j) & 1u) sq += TAB(mt).aq[s][j] * kv[j * nv + i];
            if ((mv >> j) & 1u) sv += TAB(mt).av[s][j] * kf[j * nv + i];
          }
          const double vv = vn[i] - ht * sv;
          if ((mq >> s) & 1u) sq += TAB(mt).aq[s][s] * vv;
          dq[i] = -ht * sq;
          vs[i] = vv;
          kv[s * nv + i] = vv;
        }
        for (int i = g.lane; i < na; i += G) {
          double sa = 0;
          for (int j = 0; j < s; ++j)
            if ((mv >> j) & 1u) sa += TAB(mt).av[s][j] * ka[j * na + i];
          as[i] = a[i] + ht * sa;
        }
        g.sync();
        integrate_pos(g, m, qn, dq, qs);
        const int r = otd_stage(g, m, w, b, qs, vs, u, as, P.cfd != 0, kf + s * nv, ka + s * na);
        if (r > st) st = r;
      }
      ++attempts;
      // the result is the last stage: (qs, vs) and as
      for (int i = g.lane; i < na; i += G) a7[i] = as[i];
      double err = 0.0;
      if (TAB(mt).adaptive) {
        const unsigned enz = TAB(mt).enz;
        double acc = 0.0;
        for (int i = g.lane; i < nv; i += G) {
          double ep = 0, ev = 0;
          for (int j = 0; j < 7; ++j) {
            if (!((enz >> j) & 1u)) continue;
            ep += TAB(mt).e[j] * kv[j * nv + i];
            ev += TAB(mt).e[j] * kf[j * nv + i];
          }
          ep *= ht; ev *= ht;
          const double sp = P.atol + P.rtol * fmax(pos_mag(m, qn, i), pos_mag(m, qs, i));
          const double sv = P.atol + P.rtol * fmax(fabs(vn[i]), fabs(vs[i]));
          acc += (ep / sp) * (ep / sp) + (ev / sv) * (ev / sv);
        }
        for (int i = g.lane; i < na; i += G) {
          double ea = 0;
          for (int j = 0; j < 7; ++j)
            if ((enz >> j) & 1u) ea += TAB(mt).e[j] * ka[j * na + i];
          ea *= ht;
          const double sa = P.atol + P.rtol * fmax(fabs(a[i]), fabs(a7[i]));
          acc += (ea / sa) * (ea / sa);
        }
        acc = g.sum(acc);
        err = sqrt(acc / (2.0 * nv + na));
        if (!isfinite(err)) err = INFINITY;
      }
      g.sync();
      if (err <= 1.0) {
        if (st != ENV_OK) { status = st; break; }
        for (int i = g.lane; i < nq; i += G) qn[i] = qs[i];
        for (int i = g.lane; i < nv; i += G) vn[i] = vs[i];
        for (int i = g.lane; i < na; i += G) a[i] = a7[i];
        g.sync();
        ++steps;
        t = clamped ? tlo : t - ht;
        if (TAB(mt).adaptive) {
          const double lerr = log(fmax(err, 1e-10));
          double fac = 0.9 * exp(-(0.6 / 5.0) * lerr + (0.2 / 5.0) * lerrp);
          fac = fmin(10.0, fmax(0.2, fac));
          lerrp = lerr;
          h = ht * fac;
        } else {
          h = P.h0;
        }
        if (clamped) {                       // reached the interval's lower boundary t_k
          for (int j = g.lane; j < nu; j += G) {
            if (P.ctrl_bar) P.ctrl_bar[((size_t)k * nu + j) * P.B + env] += a[nx + j];
            a[nx + j] = 0.0;
          }
          if (P.xb_bar)
            for (int i = g.lane; i < nx; i += G) a[i] += P.xb_bar[((size_t)k * nx + i) * P.B + env];
          g.sync();
          --k;
        }
      } else {
        h = ht * (isfinite(err) ? fmax(0.2, 0.9 * pow(err, -1.0 / 5.0)) : 0.2);
      }
    }
    for (int i = g.lane; i < nx; i += G) P.x0_bar[(size_t)i * P.B + env] = a[i];
    if (g.lane == 0) {
      if (P.steps) P.steps[env] = steps;
      if (P.status) P.status[env] = status;
    }
    g.sync();
  }
}

template <int G>
static cudaError_t launch_otd_g(const OtdParams& P, int blocks, size_t smem, cudaStream_t st, int* occ) {
  auto k = k_adjoint_otd<G>;
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  if (occ) {
    *occ = 0;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, 32, smem);
  }
  k<<<blocks, 32, smem, st>>>(P);
  return cudaGetLastError();
}
static cudaError_t launch_otd(int G, const OtdParams& P, int blocks, size_t smem, cudaStream_t st, int* occ) {
  switch (G) {
    case 8: return launch_otd_g<8>(P, blocks, smem, st, occ);
    case 16: return launch_otd_g<16>(P, blocks, smem, st, occ);
    case 32: return launch_otd_g<32>(P, blocks, smem, st, occ);
  }
  return cudaErrorInvalidValue;
}

}  // namespace dmx

#define OTD_CK(x)                                                                                 \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess) return dmx_fail(DMX_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" dmx_status dmx_rollout_grad_otd(dmx_model* m, const dmx_otd_args* a, void* stream) {
  using namespace dmx;
  if (!m || !a) return dmx_fail(DMX_ERR_INVALID, "null argument");
  if (a->B < 0 || a->NI < 1 || a->max_steps < 1 || !(a->rtol >= 0) || !(a->atol > 0) || !(a->h0 > 0))
    return dmx_fail(DMX_ERR_INVALID, "bad sizes or tolerances");
  if (a->method < DMX_METHOD_DOPRI5 || a->method > DMX_METHOD_EULER) return dmx_fail(DMX_ERR_INVALID, "unknown method");
  if (a->B == 0) return DMX_OK;
  const int nu = m->host.nu;
  if (!a->xT || !a->T || !a->xT_bar || !a->x0_bar || (nu && (!a->ctrl || !a->ctrl_bar)))
    return dmx_fail(DMX_ERR_INVALID, "xT, T, xT_bar, x0_bar (and ctrl, ctrl_bar) are required");
  int cur = 0;
  if (cudaGetDevice(&cur) != cudaSuccess || cur != m->device) return dmx_fail(DMX_ERR_INVALID, "model belongs to another device");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  OtdParams P{};
  P.model = m->dev;
  P.L = layout_for(m, a->cfd);
  P.LB = make_bar_layout(m->host, P.L.rcap);
  P.B = a->B; P.NI = a->NI; P.max_steps = a->max_steps; P.cfd = a->cfd; P.method = a->method;
  P.rtol = a->rtol; P.atol = a->atol; P.h0 = a->h0;
  P.xT = a->xT; P.ctrl = a->ctrl; P.T = a->T; P.xT_bar = a->xT_bar; P.xb_bar = a->xb_bar;
  P.x0_bar = a->x0_bar; P.ctrl_bar = nu ? a->ctrl_bar : nullptr; P.steps = a->steps; P.status = a->status;
  P.na = m->host.nq + m->host.nv + nu;
  P.barofs = P.L.nd;
  P.otdofs = P.L.nd + P.LB.nd;
  P.per = (P.otdofs + (3 + 7) * P.na + 1) & ~1;
  // lanes: the fewest of 8 / 16 / 32 whose workspace fits, more when the batch leaves SMs idle
  int G = 8;
  const int want = 4 * 32 * m->nsm;
  while (G < 32 && (long long)a->B * G < want) G <<= 1;
  size_t smem = 0;
  for (;; G <<= 1) {
    smem = (size_t)(32 / G) * ((size_t)P.per * 8 + (size_t)P.L.ni * 4);
    if ((int)smem <= m->smem_max - 2048) break;
    if (G == 32) return dmx_fail(DMX_ERR_INVALID, "OTD workspace does not fit shared memory");
  }
  int occ = 0;
  OTD_CK(launch_otd(G, P, 0, smem, st, &occ));
  const int gpb = 32 / G;
  const int blocks = std::min((a->B + gpb - 1) / gpb, m->nsm * std::max(occ, 1));
  int* q = nullptr;
  OTD_CK(cudaMallocAsync(reinterpret_cast<void**>(&q), sizeof(int), st));
  OTD_CK(cudaMemsetAsync(q, 0, sizeof(int), st));
  P.queue = q;
  OTD_CK(launch_otd(G, P, blocks, smem, st, nullptr));
  OTD_CK(cudaFreeAsync(q, st));
  return DMX_OK;
}
