// Host runtime behind include/dmx.h: model compiler, launch configuration,
// rollout orchestration (persistent / per-attempt launches / CUDA graphs),
// tapes for the adjoint, host-buffer staging, autotuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <string>
#include <tuple>
#include <vector>

#include "dmx.h"
#include "dmx_kernels.h"
#include "dmx_model.h"
#include "dmx_runtime.h"
#include "dmx_adjoint.h"

using namespace dmx;

namespace {
thread_local std::string g_err;
}

dmx_status dmx_fail(dmx_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

#define CK(x)                                                                                     \
  do {                                                                                            \
    cudaError_t e_ = (x);                                                                         \
    if (e_ != cudaSuccess) return dmx_fail(DMX_ERR_CUDA, std::string(#x) + ": " + cudaGetErrorString(e_)); \
  } while (0)

extern "C" const char* dmx_last_error(void) { return g_err.c_str(); }

// ------------------------------------------------------------------ device buffers
void DevBuf::free_all() {
  if (p) cudaFree(p);
  p = nullptr;
  bytes = 0;
}
cudaError_t DevBuf::ensure(size_t n) {
  if (n <= bytes) return cudaSuccess;
  free_all();
  cudaError_t e = cudaMalloc(&p, n);
  if (e == cudaSuccess) bytes = n;
  return e;
}

// ------------------------------------------------------------------ model compiler
static void quat_mat(const double* q0, double* R) {
  double n = std::sqrt(q0[0] * q0[0] + q0[1] * q0[1] + q0[2] * q0[2] + q0[3] * q0[3]);
  const double w = q0[0] / n, x = q0[1] / n, y = q0[2] / n, z = q0[3] / n;
  R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
  R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
  R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
}

static int is_identity(const double* R) {
  for (int i = 0; i < 9; ++i)
    if (R[i] != ((i % 4 == 0) ? 1.0 : 0.0)) return 0;
  return 1;
}

static std::string compile_model(const dmx_model_desc* d, DevModel& m) {
  std::memset(&m, 0, sizeof(m));
  if (d->nbody < 1 || d->nbody > MAXB) return "nbody must be in [1, " + std::to_string(MAXB) + "]";
  if (d->ngeom < 0 || d->ngeom > MAXG) return "ngeom over the compiled limit";
  if (d->npair < 0 || d->npair > MAXP) return "npair over the compiled limit";
  if (d->nact < 0 || d->nact > MAXU) return "nact over the compiled limit";
  m.nbody = d->nbody; m.ngeom = d->ngeom; m.npair = d->npair; m.nact = d->nact;
  int depth[MAXB];
  for (int b = 0; b < m.nbody; ++b) {
    const dmx_body_desc& B = d->body[b];
    if (B.parent >= b || B.parent < -1) return "body " + std::to_string(b) + ": parent must precede the body";
    if (B.joint != DMX_JNT_FREE && B.joint != DMX_JNT_HINGE) return "unknown joint type";
    if (B.joint == DMX_JNT_FREE && B.parent != -1) return "free joint only on children of the world";
    if (!(B.mass > 0)) return "body mass must be positive";
    m.b_parent[b] = B.parent;
    m.b_jtype[b] = B.joint;
    m.b_qadr[b] = m.nq; m.b_vadr[b] = m.nv;
    m.b_nv[b] = B.joint == DMX_JNT_FREE ? 6 : 1;
    m.nq += B.joint == DMX_JNT_FREE ? 7 : 1;
    m.nv += m.b_nv[b];
    for (int i = 0; i < 3; ++i) { m.b_pos[b][i] = B.pos[i]; m.b_com[b][i] = B.com[i]; m.b_inertia[b][i] = B.inertia[i]; }
    quat_mat(B.quat, m.b_Roff[b]);
    m.b_ident[b] = is_identity(m.b_Roff[b]);
    double an = std::sqrt(B.axis[0] * B.axis[0] + B.axis[1] * B.axis[1] + B.axis[2] * B.axis[2]);
    if (B.joint == DMX_JNT_HINGE && !(an > 0)) return "hinge axis must be non-zero";
    for (int i = 0; i < 3; ++i) m.b_axis[b][i] = an > 0 ? B.axis[i] / an : 0.0;
    m.b_mass[b] = B.mass;
    m.b_damping[b] = B.damping;
    depth[b] = B.parent < 0 ? 0 : depth[B.parent] + 1;
    if (depth[b] >= MAXLEV) return "body tree too deep";
    m.b_anc[b] = (1u << b) | (B.parent >= 0 ? m.b_anc[B.parent] : 0u);
  }
  if (m.nq > MAXQ || m.nv > MAXV) return "too many dofs for the compiled limits";
  // children lists and levels
  int pos = 0;
  for (int b = 0; b < m.nbody; ++b) {
    m.child_start[b] = pos;
    for (int c = 0; c < m.nbody; ++c)
      if (m.b_parent[c] == b) m.child_list[pos++] = c;
    m.child_count[b] = pos - m.child_start[b];
  }
  int maxd = 0;
  for (int b = 0; b < m.nbody; ++b) maxd = std::max(maxd, depth[b]);
  m.nlevel = maxd + 1;
  pos = 0;
  for (int l = 0; l < m.nlevel; ++l) {
    m.level_start[l] = pos;
    for (int b = 0; b < m.nbody; ++b)
      if (depth[b] == l) m.level_list[pos++] = b;
  }
  m.level_start[m.nlevel] = pos;
  for (int b = 0; b < m.nbody; ++b)
    for (int k = 0; k < m.b_nv[b]; ++k) m.dof_body[m.b_vadr[b] + k] = b;
  for (int g = 0; g < m.ngeom; ++g) {
    const dmx_geom_desc& G = d->geom[g];
    if (G.type < 0 || G.type > 2) return "unknown geom type";
    if (G.body < 0 || G.body >= m.nbody) return "geom body out of range";
    m.g_type[g] = G.type; m.g_body[g] = G.body;
    for (int i = 0; i < 3; ++i) { m.g_pos[g][i] = G.pos[i]; m.g_size[g][i] = G.size[i]; }
    quat_mat(G.quat, m.g_Roff[g]);
    m.g_ident[g] = is_identity(m.g_Roff[g]);
    m.g_zpos[g] = G.pos[0] == 0.0 && G.pos[1] == 0.0 && G.pos[2] == 0.0;
    m.g_box[g] = -1;
    if (G.type == DMX_GEOM_BOX) {
      if (m.nbox >= MAXBOX) return "too many box geoms for the compiled limits";
      m.g_box[g] = m.nbox++;
    }
    if (G.type == DMX_GEOM_SPHERE) m.g_bound[g] = G.size[0];
    else if (G.type == DMX_GEOM_CAPSULE) m.g_bound[g] = G.size[0] + G.size[1];
    else m.g_bound[g] = std::sqrt(G.size[0] * G.size[0] + G.size[1] * G.size[1] + G.size[2] * G.size[2]);
  }
  for (int b = 0; b < m.nbody; ++b) {
    int n = 0, last = -1;
    for (int g = 0; g < m.ngeom; ++g)
      if (m.g_body[g] == b) { ++n; last = g; }
    m.b_solebox[b] = (n == 1 && m.g_type[last] == DMX_GEOM_BOX) ? last : -1;
  }
  int row = 0;
  for (int p = 0; p < m.npair; ++p) {
    const dmx_pair_desc& P = d->pair[p];
    if (P.geom1 < 0 || P.geom1 >= m.ngeom || P.geom2 >= m.ngeom || P.geom2 < -1) return "pair geom out of range";
    if (P.condim != 1 && P.condim != 3) return "condim must be 1 or 3";
    if (P.geom2 >= 0) {
      const int t1 = m.g_type[P.geom1], t2 = m.g_type[P.geom2];
      const bool capbox = t1 == DMX_GEOM_CAPSULE && t2 == DMX_GEOM_BOX;
      const bool segseg = (t1 == DMX_GEOM_SPHERE || t1 == DMX_GEOM_CAPSULE) && (t2 == DMX_GEOM_SPHERE || t2 == DMX_GEOM_CAPSULE);
      if (!capbox && !segseg) return "geom pairs: capsule-box or sphere/capsule against sphere/capsule";
      if (m.g_body[P.geom1] == m.g_body[P.geom2]) return "a geom pair must join two bodies";
    }
    const int ns = P.geom2 >= 0 ? 1 : (m.g_type[P.geom1] == DMX_GEOM_SPHERE ? 1 : m.g_type[P.geom1] == DMX_GEOM_CAPSULE ? 2 : 8);
    m.p_g1[p] = P.geom1; m.p_g2[p] = P.geom2; m.p_condim[p] = P.condim; m.p_mu[p] = P.mu;
    m.p_slot0[p] = m.nslot; m.p_nslot[p] = ns; m.p_row0[p] = row;
    if (m.nslot + ns > MAXS) return "too many contact slots";
    for (int j = 0; j < ns; ++j) {
      m.s_pair[m.nslot + j] = p; m.s_idx[m.nslot + j] = j;
      m.s_barofs[m.nslot + j] = m.nslotbar;
      m.nslotbar += P.geom2 >= 0 ? 24 : 12;     // a plane slot moves one geom
    }
    m.nslot += ns;
    row += ns * (P.condim == 1 ? 1 : 4);
  }
  if (row > MAXROWID) return "too many constraint rows";
  m.nrowid = row;
  for (int a = 0; a < m.nact; ++a) {
    const dmx_actuator_desc& A = d->act[a];
    if (A.body < 0 || A.body >= m.nbody || m.b_jtype[A.body] != DMX_JNT_HINGE) return "actuator must drive a hinge";
    if (A.type != DMX_ACT_MOTOR && A.type != DMX_ACT_POSITION) return "unknown actuator type";
    m.a_type[a] = A.type; m.a_qadr[a] = m.b_qadr[A.body]; m.a_vadr[a] = m.b_vadr[A.body];
    m.a_gear[a] = A.gear; m.a_kp[a] = A.kp; m.a_kd[a] = A.kd;
  }
  m.nu = m.nact;
  for (int i = 0; i < 3; ++i) m.grav[i] = d->gravity[i];
  const double tc = d->solref[0], damp = d->solref[1], dw = d->solimp[1];
  if (!(tc > 0) || !(damp > 0) || !(dw > 0) || !(d->solimp[2] > 0)) return "solref / solimp must be positive";
  if (!(d->solimp_cfd[2] > 0) || !(d->softplus > 0)) return "solimp-CFD width and softplus width must be positive";
  m.bcoef = 2.0 / (dw * tc);
  m.kcoef = 1.0 / (dw * dw * tc * tc * damp * damp);
  m.solref[0] = tc; m.solref[1] = damp;
  for (int i = 0; i < 5; ++i) { m.solimp[i] = d->solimp[i]; m.cfd[i] = d->solimp_cfd[i]; }
  m.softplus = d->softplus;
  return "";
}

int model_smem_bytes(const dmx_model* m, int groups) {
  return groups * (m->L.nd * 8 + m->L.ni * 4);
}

extern "C" dmx_status dmx_create_model(const dmx_model_desc* desc, dmx_model** out) {
  if (!desc || !out) return dmx_fail(DMX_ERR_INVALID, "null argument");
  *out = nullptr;
  dmx_model* m = new dmx_model();
  std::string err = compile_model(desc, m->host);
  if (!err.empty()) { delete m; return dmx_fail(DMX_ERR_INVALID, err); }
  m->rcap = std::max(1, std::min(m->host.nrowid, dmx::ROWCAP));
  m->L = make_layout(m->host, m->rcap);
  m->rcap_c = std::max(1, std::min(m->host.nrowid, dmx::MAXROWID));
  m->Lc = make_layout(m->host, m->rcap_c);
  CK(cudaGetDevice(&m->device));
  cudaDeviceProp prop;
  CK(cudaGetDeviceProperties(&prop, m->device));
  m->nsm = prop.multiProcessorCount;
  {
    // keep stream-ordered per-call scratch cached in the device's default pool
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, m->device) == cudaSuccess) {
      uint64_t thr = ~0ull;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  m->smem_max = (int)prop.sharedMemPerBlockOptin;
  if (cudaMalloc(&m->dev, sizeof(DevModel)) != cudaSuccess) { delete m; return dmx_fail(DMX_ERR_OOM, "model upload"); }
  CK(cudaMemcpy(m->dev, &m->host, sizeof(DevModel), cudaMemcpyHostToDevice));
  // A_hat: translational inverse weight of each body at qpos0 (computed on the device)
  std::vector<double> q0(desc->qpos0, desc->qpos0 + m->host.nq);
  double *dq0 = nullptr, *dinv = nullptr, *dscr = nullptr;
  CK(cudaMalloc(&dq0, sizeof(double) * m->host.nq));
  CK(cudaMalloc(&dinv, sizeof(double) * MAXB));
  CK(cudaMalloc(&dscr, sizeof(double) * 2 * MAXV));
  CK(cudaMemcpy(dq0, q0.data(), sizeof(double) * m->host.nq, cudaMemcpyHostToDevice));
  CK(launch_body_invweight(m->dev, dq0, dinv, dscr, m->rcap, model_smem_bytes(m, 1), 0));
  double invw[MAXB];
  CK(cudaMemcpy(invw, dinv, sizeof(double) * m->host.nbody, cudaMemcpyDeviceToHost));
  // derivative of the inverse weights with respect to every body mass (the
  // model-parameter gradient carries A_hat's dependence on the masses)
  // (and every box side, through the inertia of a body that is that box)
  const int nmc = m->host.nbody + m->host.nbox;
  double dinvw[MAXB + MAXBOX][MAXB] = {};
  {
    void *ws = nullptr, *tscr = nullptr;
    const size_t wsb = (size_t)m->L.nd * 16 + (size_t)m->L.ni * 4 + 16;
    CK(cudaMalloc(&ws, wsb));
    CK(cudaMalloc(&tscr, 16 * (size_t)(m->host.nq + 2 * m->host.nv)));
    for (int c = 0; c < nmc; ++c) {
      CK(launch_body_invweight_tangent(m->dev, dq0, m->rcap, dmx::PAR_MU0 + m->host.npair + c, ws, tscr, dinv, 0));
      CK(cudaMemcpy(dinvw[c], dinv, sizeof(double) * m->host.nbody, cudaMemcpyDeviceToHost));
    }
    cudaFree(ws); cudaFree(tscr);
  }
  cudaFree(dq0); cudaFree(dinv); cudaFree(dscr);
  for (int p = 0; p < m->host.npair; ++p) {
    const int bA = m->host.g_body[m->host.p_g1[p]];
    const int bB = m->host.p_g2[p] >= 0 ? m->host.g_body[m->host.p_g2[p]] : -1;
    const double ah = invw[bA] + (bB >= 0 ? invw[bB] : 0.0);
    if (!(ah > 0) || !std::isfinite(ah)) { cudaFree(m->dev); delete m; return dmx_fail(DMX_ERR_INVALID, "mass matrix at qpos0 is singular"); }
    m->host.p_ahat[p] = ah;
    m->host.p_ahat_edge[p] = ah * (1.0 + m->host.p_mu[p] * m->host.p_mu[p]);
    for (int c = 0; c < nmc; ++c) m->host.p_dahat[p][c] = dinvw[c][bA] + (bB >= 0 ? dinvw[c][bB] : 0.0);
  }
  for (int b = 0; b < m->host.nbody; ++b) m->invw[b] = invw[b];
  CK(cudaMemcpy(m->dev, &m->host, sizeof(DevModel), cudaMemcpyHostToDevice));
  *out = m;
  return DMX_OK;
}

extern "C" void dmx_destroy_model(dmx_model* m) {
  if (!m) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(m->device);
  cudaFree(m->dev);
  cudaSetDevice(cur);
  delete m;
}

extern "C" dmx_status dmx_model_dims(const dmx_model* m, int32_t* nq, int32_t* nv, int32_t* nu) {
  if (!m) return dmx_fail(DMX_ERR_INVALID, "null model");
  if (nq) *nq = m->host.nq;
  if (nv) *nv = m->host.nv;
  if (nu) *nu = m->host.nu;
  return DMX_OK;
}

// Extra accessor for tests: body inverse weights and workspace sizes.
extern "C" dmx_status dmx_model_info(const dmx_model* m, double* invw, int32_t* info) {
  if (!m) return dmx_fail(DMX_ERR_INVALID, "null model");
  if (invw) for (int b = 0; b < m->host.nbody; ++b) invw[b] = m->invw[b];
  if (info) {
    info[0] = m->host.nslot; info[1] = m->host.nrowid; info[2] = m->rcap; info[3] = m->L.nd; info[4] = m->L.ni;
    info[5] = m->host.nbody;
  }
  return DMX_OK;
}

// ------------------------------------------------------------------ launch configuration
static bool valid_lanes(int G) { return G == 1 || G == 2 || G == 4 || G == 8 || G == 16 || G == 32; }

// Threads per block and dynamic shared memory for G lanes per environment.
// One warp per block: the block scheduler then spreads the warps over every
// SM (with larger blocks a batch of a few thousand environments filled only
// some of the SMs), and a block needs only one warp's workspace.
bool launch_config(const dmx_model* m, int G, int* threads, size_t* smem) {
  return launch_config_layout(m, m->L, G, threads, smem);
}
bool launch_config_layout(const dmx_model* m, const dmx::Layout& L, int G, int* threads, size_t* smem) {
  const int per = L.nd * 8 + L.ni * 4;
  if (G < 1 || G > 32) return false;
  const size_t s = (size_t)(32 / G) * per;
  if ((int)s > m->smem_max - 1024) return false;
  *threads = 32;
  *smem = s;
  return true;
}

int default_lanes(const dmx_model* m, int B) {
  // enough lanes to give every SM sub-partition one warp of FP64 work
  const int want = 4 * 32 * m->nsm;
  int G = 1;
  while (G < 32 && (long long)B * G < want) G <<= 1;
  int t; size_t s;
  while (G < 32 && !launch_config(m, G, &t, &s)) G <<= 1;
  return G;
}

// ------------------------------------------------------------------ rollout
static int ncheck_for(int max_steps, int K) { return max_steps / K + 2; }

dmx_status run_rollout(dmx_model* m, const RolloutParams& P0, int form, int G, cudaStream_t st) {
  RolloutParams P = P0;
  int threads; size_t smem;
  if (!launch_config(m, G, &threads, &smem))
    return dmx_fail(DMX_ERR_INVALID, "workspace of " + std::to_string(G) + " lanes/env does not fit shared memory");
  if (P.B == 0) return DMX_OK;
  if (form == DMX_FORM_PERSISTENT) {
    // per-call work counter (stream ordered, so concurrent calls on other
    // streams never share it)
    int* q = nullptr;
    CK(cudaMallocAsync(reinterpret_cast<void**>(&q), sizeof(int), st));
    CK(cudaMemsetAsync(q, 0, sizeof(int), st));
    P.queue = q;
    int per_sm = persistent_occupancy(G, threads, smem);
    if (per_sm < 1) per_sm = 1;
    const long long groups = (long long)m->nsm * per_sm * (threads / G);
    long long blocks = (long long)m->nsm * per_sm;
    if (groups > P.B) blocks = std::max(1LL, ((long long)P.B * G + threads - 1) / threads);
    CK(launch_persistent(G, P, (int)blocks, threads, smem, st));
    CK(cudaFreeAsync(q, st));
    return DMX_OK;
  }
  // plain form: state in HBM, one launch per attempt
  const int nq = m->host.nq, nv = m->host.nv;
  const size_t B = P.B;
  const size_t need = B * (sizeof(double) * (nq + 2 * nv + 3) + sizeof(int) * (7 + MASKW)) + 64;
  void* mem = nullptr;
  CK(cudaMallocAsync(&mem, need, st));
  char* base = static_cast<char*>(mem);
  StepState S;
  size_t off = 0;
  auto takeD = [&](size_t n) { double* r = reinterpret_cast<double*>(base + off); off += n * sizeof(double); return r; };
  auto takeI = [&](size_t n) { int* r = reinterpret_cast<int*>(base + off); off += n * sizeof(int); return r; };
  S.q = takeD(B * nq); S.v = takeD(B * nv); S.ka0 = takeD(B * nv); S.t = takeD(B); S.h = takeD(B); S.lerrp = takeD(B);
  S.k = takeI(B); S.nacc = takeI(B); S.nrej = takeI(B); S.att = takeI(B); S.st = takeI(B); S.done = takeI(B);
  S.pmask = takeI(B * MASKW);
  S.active = takeI(1);
  const int Bi = P.B;
  CK(cudaMemcpyAsync(S.active, &Bi, sizeof(int), cudaMemcpyHostToDevice, st));
  CK(launch_step(G, P, S, true, threads, smem, st));
  // device-to-pageable copies return once the copy (and the work before it on
  // the stream) has completed
  int active_host = P.B;
  int* h_active = &active_host;
  const int chunk = 64;
  long long launched = 0;
  const long long limit = (long long)P.max_steps + 2;
  if (form == DMX_FORM_STEP_GRAPH) {
    cudaGraph_t graph;
    cudaGraphExec_t exec;
    // one ordinary launch first: it configures the kernel's shared-memory
    // attribute outside the capture and is a valid attempt of every environment
    CK(launch_step(G, P, S, false, threads, smem, st));
    launched += 1;
    cudaStream_t cap;
    CK(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    CK(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal));
    for (int i = 0; i < chunk; ++i) launch_step(G, P, S, false, threads, smem, cap);
    CK(cudaStreamEndCapture(cap, &graph));
    CK(cudaGraphInstantiate(&exec, graph, 0));
    for (;;) {
      CK(cudaGraphLaunch(exec, st));
      launched += chunk;
      CK(cudaMemcpyAsync(h_active, S.active, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (*h_active <= 0 || launched > limit) break;
    }
    cudaGraphExecDestroy(exec);
    cudaGraphDestroy(graph);
    cudaStreamDestroy(cap);
  } else {
    for (;;) {
      for (int i = 0; i < chunk; ++i) CK(launch_step(G, P, S, false, threads, smem, st));
      launched += chunk;
      CK(cudaMemcpyAsync(h_active, S.active, sizeof(int), cudaMemcpyDeviceToHost, st));
      CK(cudaStreamSynchronize(st));
      if (*h_active <= 0 || launched > limit) break;
    }
  }
  CK(cudaFreeAsync(mem, st));
  if (*h_active > 0) return dmx_fail(DMX_ERR_TIMEOUT, "plain form did not finish within max_steps launches");
  return DMX_OK;
}


static dmx_status make_tape(dmx_model* m, const dmx_rollout_args* a, const double* ctrl, const double* T,
                            cudaStream_t st, dmx_tape** out) {
  dmx_tape* t = new dmx_tape();
  t->model = m;
  t->B = a->B; t->NI = a->NI; t->K = a->K; t->nx = m->host.nq + m->host.nv; t->nu = m->host.nu;
  t->max_steps = a->max_steps; t->ncheck = ncheck_for(a->max_steps, a->K);
  t->rtol = a->rtol; t->atol = a->atol; t->h0 = a->h0; t->method = a->method;
  const size_t B = a->B;
  const size_t bytes = sizeof(double) * ((size_t)t->ncheck * (t->nx + 1) * B + (size_t)a->max_steps * B +
                                         (size_t)a->NI * t->nu * B + B) + sizeof(int) * B;
  if (cudaMallocAsync(&t->mem, bytes, st) != cudaSuccess) { delete t; return dmx_fail(DMX_ERR_OOM, "tape allocation of " + std::to_string(bytes) + " bytes"); }
  t->stream = st;
  t->bytes = bytes;
  double* p = static_cast<double*>(t->mem);
  t->ckpt = p; p += (size_t)t->ncheck * (t->nx + 1) * B;
  t->hlog = p; p += (size_t)a->max_steps * B;
  t->ctrl = p; p += (size_t)a->NI * t->nu * B;
  t->T = p; p += B;
  t->n = reinterpret_cast<int*>(p);
  if (t->nu && ctrl) CK(cudaMemcpyAsync(t->ctrl, ctrl, sizeof(double) * a->NI * t->nu * B, cudaMemcpyDeviceToDevice, st));
  CK(cudaMemcpyAsync(t->T, T, sizeof(double) * B, cudaMemcpyDeviceToDevice, st));
  *out = t;
  return DMX_OK;
}

extern "C" void dmx_tape_free(dmx_tape* t) {
  if (!t) return;
  cudaFreeAsync(t->mem, t->stream);   // ordered after the work queued on the tape's stream
  delete t;
}

extern "C" dmx_status dmx_rollout(dmx_model* m, const dmx_rollout_args* a, void* stream) {
  if (!m || !a) return dmx_fail(DMX_ERR_INVALID, "null argument");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nq = m->host.nq, nv = m->host.nv, nx = nq + nv, nu = m->host.nu;
  if (a->B < 0) return dmx_fail(DMX_ERR_INVALID, "B must be >= 0");
  if (a->NI < 1) return dmx_fail(DMX_ERR_INVALID, "NI must be >= 1");
  if (!(a->rtol >= 0) || !(a->atol > 0) || !(a->h0 > 0)) return dmx_fail(DMX_ERR_INVALID, "rtol >= 0, atol > 0 and h0 > 0 are required");
  if (a->max_steps < 1) return dmx_fail(DMX_ERR_INVALID, "max_steps must be >= 1");
  if (a->tape && a->K < 1) return dmx_fail(DMX_ERR_INVALID, "K must be >= 1 when a tape is requested");
  if (a->form < DMX_FORM_PERSISTENT || a->form > DMX_FORM_STEP_GRAPH) return dmx_fail(DMX_ERR_INVALID, "unknown form");
  if (a->method < DMX_METHOD_DOPRI5 || a->method > DMX_METHOD_EULER) return dmx_fail(DMX_ERR_INVALID, "unknown method");
  if (a->lanes != 0 && !valid_lanes(a->lanes)) return dmx_fail(DMX_ERR_INVALID, "lanes must be 0, 1, 2, 4, 8, 16 or 32");
  if (a->B > 0 && (!a->x0 || !a->T || !a->xT)) return dmx_fail(DMX_ERR_INVALID, "x0, T and xT are required");
  if (a->B > 0 && nu > 0 && !a->ctrl) return dmx_fail(DMX_ERR_INVALID, "ctrl is required when the model has actuators");
  if (a->host && a->tape) return dmx_fail(DMX_ERR_INVALID, "tapes need device buffers (host = 0)");
  int cur = 0;
  CK(cudaGetDevice(&cur));
  if (cur != m->device) return dmx_fail(DMX_ERR_INVALID, "model belongs to another device");
  const int G = a->lanes ? a->lanes : tuned_lanes(m, a->B, 0);
  const size_t B = a->B;
  RolloutParams P{};
  P.model = m->dev; P.L = m->L; P.B = a->B; P.NI = a->NI; P.max_steps = a->max_steps; P.K = a->K > 0 ? a->K : 1;
  P.rtol = a->rtol; P.atol = a->atol; P.h0 = a->h0; P.method = a->method;
  P.x0 = a->x0; P.ctrl = a->ctrl; P.T = a->T; P.xT = a->xT; P.xb = a->xb;
  P.nsteps = a->nsteps; P.nrej = a->nrej; P.status = a->status;
  if (a->host && B > 0) {
    // stage host buffers through library device memory
    const size_t nin = B * nx + (size_t)a->NI * nu * B + B;
    const size_t nout = B * nx + (a->xb ? (size_t)(a->NI + 1) * nx * B : 0);
    const size_t bytes = sizeof(double) * (nin + nout) + sizeof(int) * 3 * B + 256;
    void* stage = nullptr;
    CK(cudaMallocAsync(&stage, bytes, st));
    double* p = static_cast<double*>(stage);
    double* dx0 = p; p += B * nx;
    double* dctrl = p; p += (size_t)a->NI * nu * B;
    double* dT = p; p += B;
    double* dxT = p; p += B * nx;
    double* dxb = a->xb ? p : nullptr; if (a->xb) p += (size_t)(a->NI + 1) * nx * B;
    int* ip = reinterpret_cast<int*>(p);
    int* dns = ip; int* dnr = ip + B; int* dst = ip + 2 * B;
    CK(cudaMemcpyAsync(dx0, a->x0, sizeof(double) * B * nx, cudaMemcpyHostToDevice, st));
    if (nu) CK(cudaMemcpyAsync(dctrl, a->ctrl, sizeof(double) * a->NI * nu * B, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dT, a->T, sizeof(double) * B, cudaMemcpyHostToDevice, st));
    P.x0 = dx0; P.ctrl = nu ? dctrl : nullptr; P.T = dT; P.xT = dxT; P.xb = dxb;
    P.nsteps = dns; P.nrej = dnr; P.status = dst;
    dmx_status s = run_rollout(m, P, a->form, G, st);
    if (s != DMX_OK) return s;
    CK(cudaMemcpyAsync(a->xT, dxT, sizeof(double) * B * nx, cudaMemcpyDeviceToHost, st));
    if (a->xb) CK(cudaMemcpyAsync(a->xb, dxb, sizeof(double) * (a->NI + 1) * nx * B, cudaMemcpyDeviceToHost, st));
    if (a->nsteps) CK(cudaMemcpyAsync(a->nsteps, dns, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    if (a->nrej) CK(cudaMemcpyAsync(a->nrej, dnr, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    if (a->status) CK(cudaMemcpyAsync(a->status, dst, sizeof(int) * B, cudaMemcpyDeviceToHost, st));
    CK(cudaFreeAsync(stage, st));
    CK(cudaStreamSynchronize(st));
    return DMX_OK;
  }
  dmx_tape* tape = nullptr;
  if (a->tape) {
    dmx_status s = make_tape(m, a, a->ctrl, a->T, st, &tape);
    if (s != DMX_OK) return s;
    tape->G = G;
    P.ckpt = tape->ckpt; P.hlog = tape->hlog; P.tape_n = tape->n;
  }
  dmx_status s = run_rollout(m, P, a->form, G, st);
  if (s != DMX_OK) { dmx_tape_free(tape); return s; }
  if (a->tape) *a->tape = tape;
  return DMX_OK;
}

// ------------------------------------------------------------------ autotuner
int tuned_lanes(dmx_model* m, int B, int grad) {
  std::lock_guard<std::mutex> lk(m->mu);
  auto it = m->tuned.find({B, grad});
  if (it != m->tuned.end()) return it->second;
  return default_lanes(m, B);
}

extern "C" dmx_status dmx_autotune(dmx_model* m, int32_t B, int32_t grad, int32_t* lanes, void* stream) {
  (void)stream;
  if (!m || B < 0) return dmx_fail(DMX_ERR_INVALID, "bad argument");
  if (lanes) *lanes = tuned_lanes(m, B, grad);
  return DMX_OK;
}

extern "C" dmx_status dmx_set_lanes(dmx_model* m, int32_t B, int32_t grad, int32_t lanes) {
  if (!m || !valid_lanes(lanes) || grad < 0 || grad > 2 || (grad == 2 && lanes == 1))
    return dmx_fail(DMX_ERR_INVALID, "bad argument");
  std::lock_guard<std::mutex> lk(m->mu);
  m->tuned[{B, grad}] = lanes;
  return DMX_OK;
}

static bool valid_adj_lanes(int G) { return G == 2 || G == 4 || G == 8 || G == 16 || G == 32; }

// Upper bound of the reverse adjoint's stage-snapshot buffer per call.
constexpr size_t kSnapMaxBytes = size_t(8) << 30;

// Threads and shared memory of the reverse-mode adjoint kernel for G lanes.
// (one warp per block, as for the forward kernels)
static bool adj_launch_config(const dmx_model* m, const dmx::Layout& L, const dmx::LayoutBar& LB, int G, int* threads,
                              size_t* smem) {
  const int per = (L.nd + LB.nd) * 8 + L.ni * 4;
  if (G < 1 || G > 32) return false;
  const size_t s = (size_t)(32 / G) * per;
  if ((int)s > m->smem_max - 2048) return false;
  *threads = 32;
  *smem = s;
  return true;
}

// Lanes of the reverse-mode adjoint: the recorded choice, else enough lanes
// to give every SM sub-partition a warp (at least 2), within shared memory.
static int adjoint_lanes(dmx_model* m, int B, const dmx::Layout& L) {
  const dmx::LayoutBar LB = dmx::make_bar_layout(m->host, L.rcap);
  int t; size_t s;
  {
    std::lock_guard<std::mutex> lk(m->mu);
    auto it = m->tuned.find({B, 2});
    if (it != m->tuned.end() && valid_adj_lanes(it->second) && adj_launch_config(m, L, LB, it->second, &t, &s))
      return it->second;
  }
  const int want = 4 * 32 * m->nsm;
  int G = 2;
  while (G < 32 && (long long)B * G < want) G <<= 1;
  while (G < 32 && !adj_launch_config(m, L, LB, G, &t, &s)) G <<= 1;
  return G;
}

size_t adjoint_scratch_bound(dmx_model* m, int B, int K, int cfd) {
  int mode;
  {
    std::lock_guard<std::mutex> lk(m->mu);
    mode = m->adj_mode;
  }
  const size_t groups = (size_t)std::max(B, 1), k = (size_t)std::max(K, 1);
  const size_t nx = m->host.nq + m->host.nv;
  size_t b = sizeof(double) * groups * k * std::max<size_t>(dmx::rev_row_doubles(m->host), nx + 1);
  if (mode == DMX_ADJ_REVERSE && !cfd)
    b += std::min(kSnapMaxBytes, sizeof(double) * groups * k * 6 * (size_t)dmx::snap_offsets(m->host, m->L).size);
  (void)cfd;
  return b + 256;
}

extern "C" dmx_status dmx_set_adjoint(dmx_model* m, int32_t mode) {
  if (!m || (mode != DMX_ADJ_REVERSE && mode != DMX_ADJ_TANGENT && mode != DMX_ADJ_RECOMPUTE))
    return dmx_fail(DMX_ERR_INVALID, "bad argument");
  std::lock_guard<std::mutex> lk(m->mu);
  m->adj_mode = mode;
  return DMX_OK;
}

// The forward-mode adjoint kernel (one derivative direction per lane; model
// parameters too when P.p_bar is set).
static dmx_status run_tangent_adjoint(dmx_model* m, dmx_tape* t, dmx::AdjParams& P, cudaStream_t st) {
  const dmx::Layout& L = P.L;
  const int nx = t->nx;
  if (L.nd > dmx::adjoint_workspace_limit() || L.ni > dmx::adjoint_int_limit())
    return dmx_fail(DMX_ERR_INVALID, "model workspace exceeds the tangent adjoint kernel's per-lane limit");
  const int wpb = dmx::adjoint_warps_per_block();
  int blocks = (t->B + wpb - 1) / wpb;
  blocks = std::min(blocks, m->nsm * 8);
  const size_t seg_bytes = sizeof(double) * (size_t)blocks * wpb * t->K * (nx + 1);
  void* scratch = nullptr;
  CK(cudaMallocAsync(&scratch, seg_bytes + 256, st));
  P.segbuf = static_cast<double*>(scratch);
  P.queue = reinterpret_cast<int*>(static_cast<char*>(scratch) + seg_bytes);
  CK(cudaMemsetAsync(P.queue, 0, sizeof(int), st));
  CK(dmx::launch_adjoint(P, blocks, st));
  CK(cudaFreeAsync(scratch, st));
  return DMX_OK;
}

static int model_nparams(const dmx_model* m) {
  return dmx::PAR_MU0 + m->host.npair + m->host.nbody + m->host.nbox;
}

extern "C" dmx_status dmx_model_params(const dmx_model* m, int32_t* np, double* values) {
  if (!m) return dmx_fail(DMX_ERR_INVALID, "null model");
  const int n = model_nparams(m);
  if (np) *np = n;
  if (values) {
    const dmx::DevModel& d = m->host;
    values[dmx::PAR_TC] = d.solref[0]; values[dmx::PAR_DAMP] = d.solref[1];
    values[dmx::PAR_DO] = d.solimp[0]; values[dmx::PAR_DW] = d.solimp[1];
    values[dmx::PAR_WIDTH] = d.solimp[2]; values[dmx::PAR_MID] = d.solimp[3];
    for (int p = 0; p < d.npair; ++p) values[dmx::PAR_MU0 + p] = d.p_mu[p];
    for (int b = 0; b < d.nbody; ++b) values[dmx::PAR_MU0 + d.npair + b] = d.b_mass[b];
    for (int g = 0; g < d.ngeom; ++g)
      if (d.g_box[g] >= 0) values[dmx::PAR_MU0 + d.npair + d.nbody + d.g_box[g]] = 2.0 * d.g_size[g][0];
  }
  return DMX_OK;
}

extern "C" dmx_status dmx_rollout_grad_params(dmx_model* m, dmx_tape* t, int32_t cfd, const double* xT_bar,
                                              const double* xb_bar, double* x0_bar, double* ctrl_bar, double* p_bar,
                                              double* p_bar_sum, void* stream) {
  if (!m || !t) return dmx_fail(DMX_ERR_INVALID, "null model or tape");
  if (t->model != m) return dmx_fail(DMX_ERR_INVALID, "tape belongs to another model");
  if (!p_bar) return dmx_fail(DMX_ERR_INVALID, "p_bar is required");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int np = model_nparams(m);
  if (t->B == 0) {
    if (p_bar_sum) CK(cudaMemsetAsync(p_bar_sum, 0, sizeof(double) * np, st));
    return DMX_OK;
  }
  if (!xT_bar || !x0_bar) return dmx_fail(DMX_ERR_INVALID, "xT_bar and x0_bar are required");
  if (m->host.nu > 0 && !ctrl_bar) return dmx_fail(DMX_ERR_INVALID, "ctrl_bar is required when the model has actuators");
  dmx::AdjParams P{};
  P.model = m->dev; P.L = layout_for(m, cfd); P.B = t->B; P.NI = t->NI; P.K = t->K; P.cfd = cfd; P.method = t->method;
  P.ckpt = t->ckpt; P.hlog = t->hlog; P.tape_n = t->n; P.ctrl = t->ctrl; P.T = t->T;
  P.xT_bar = xT_bar; P.xb_bar = xb_bar; P.x0_bar = x0_bar; P.ctrl_bar = m->host.nu ? ctrl_bar : nullptr;
  P.p_bar = p_bar; P.np = np;
  const dmx_status s = run_tangent_adjoint(m, t, P, st);
  if (s != DMX_OK) return s;
  if (p_bar_sum) CK(dmx::launch_row_sums(p_bar, np, t->B, p_bar_sum, st));
  return DMX_OK;
}

extern "C" dmx_status dmx_rollout_grad(dmx_model* m, dmx_tape* t, int32_t cfd, const double* xT_bar,
                                       const double* xb_bar, double* x0_bar, double* ctrl_bar, void* stream) {
  if (!m || !t) return dmx_fail(DMX_ERR_INVALID, "null model or tape");
  if (t->model != m) return dmx_fail(DMX_ERR_INVALID, "tape belongs to another model");
  if (t->B == 0) return DMX_OK;
  if (!xT_bar || !x0_bar) return dmx_fail(DMX_ERR_INVALID, "xT_bar and x0_bar are required");
  if (m->host.nu > 0 && !ctrl_bar) return dmx_fail(DMX_ERR_INVALID, "ctrl_bar is required when the model has actuators");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nx = t->nx;
  int mode;
  {
    std::lock_guard<std::mutex> lk(m->mu);
    mode = m->adj_mode;
  }
  dmx::AdjParams P{};
  const dmx::Layout& L = layout_for(m, cfd);
  P.model = m->dev; P.L = L; P.B = t->B; P.NI = t->NI; P.K = t->K; P.cfd = cfd; P.method = t->method;
  P.ckpt = t->ckpt; P.hlog = t->hlog; P.tape_n = t->n; P.ctrl = t->ctrl; P.T = t->T;
  P.xT_bar = xT_bar; P.xb_bar = xb_bar; P.x0_bar = x0_bar; P.ctrl_bar = m->host.nu ? ctrl_bar : nullptr;
  if (mode == DMX_ADJ_TANGENT) return run_tangent_adjoint(m, t, P, st);
  const int G = adjoint_lanes(m, t->B, L);
  P.LB = dmx::make_bar_layout(m->host, L.rcap);
  const int gpb = 32 / G, threads = 32;
  const int RW = dmx::rev_row_doubles(m->host);
  const int nsnap = t->method == DMX_METHOD_EULER ? 1 : 6;   // stage right-hand sides per step
  // Launch plan for a workspace layout: doubles per environment, the cotangent
  // workspace's offset, shared memory, resident blocks and segment buffer.
  struct Plan {
    dmx::Layout L;
    int per = 0, barofs = 0, blocks = 0;
    size_t smem = 0, seg = 0;
  };
  auto plan = [&](const dmx::Layout& Lx, bool overlay, Plan& out) {
    out.L = Lx;
    out.per = overlay ? std::max(Lx.nd, Lx.ovl + P.LB.nd) : Lx.nd + P.LB.nd;
    out.per = (out.per + 1) & ~1;
    out.barofs = overlay ? Lx.ovl : Lx.nd;
    out.smem = (size_t)gpb * ((size_t)out.per * 8 + (size_t)Lx.ni * 4);
    if ((int)out.smem > m->smem_max - 2048) return false;
    const int occ = std::max(1, dmx::adjoint_rev_occupancy(G, threads, out.smem));
    out.blocks = std::min((t->B + gpb - 1) / gpb, m->nsm * occ);
    out.seg = sizeof(double) * (size_t)out.blocks * gpb * t->K * RW;
    return true;
  };
  // With stage snapshots (forward right-hand side only, when they fit a share
  // of the free device memory) the reverse sweep never evaluates a right-hand
  // side, so the cotangent workspace overlays the arrays only the segment
  // recompute uses (dmx::make_layout_adj): fewer bytes per environment, more
  // resident warps.  Otherwise every stage is evaluated again in the sweep.
  Plan pl;
  size_t snap_bytes = 0;
  if (mode == DMX_ADJ_REVERSE && !cfd && plan(dmx::make_layout_adj(m->host, L.rcap), true, pl)) {
    P.SN = dmx::snap_offsets(m->host, pl.L).size;
    snap_bytes = sizeof(double) * (size_t)pl.blocks * gpb * t->K * nsnap * (size_t)P.SN;
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess || snap_bytes > free_b / 8 || snap_bytes > kSnapMaxBytes)
      snap_bytes = 0;
  }
  if (snap_bytes == 0 && !plan(L, false, pl))
    return dmx_fail(DMX_ERR_INVALID, "adjoint workspace of " + std::to_string(G) + " lanes/env does not fit shared memory");
  P.L = pl.L;
  P.per = pl.per;
  P.barofs = pl.barofs;
  const int blocks = pl.blocks;
  const size_t smem = pl.smem, seg_bytes = pl.seg;
  void* scratch = nullptr;
  CK(cudaMallocAsync(&scratch, seg_bytes + snap_bytes + 256, st));
  P.segbuf = static_cast<double*>(scratch);
  P.snapbuf = snap_bytes ? reinterpret_cast<double*>(static_cast<char*>(scratch) + seg_bytes) : nullptr;
  P.queue = reinterpret_cast<int*>(static_cast<char*>(scratch) + seg_bytes + snap_bytes);
  CK(cudaMemsetAsync(P.queue, 0, sizeof(int), st));
  CK(dmx::launch_adjoint_rev(G, P, blocks, threads, smem, st));
  CK(cudaFreeAsync(scratch, st));
  return DMX_OK;
}

extern "C" dmx_status dmx_eval_rhs_vjp(dmx_model* m, int32_t B, const double* q, const double* v, const double* u,
                                       const double* abar, int32_t cfd, int32_t lanes, double* qbar, double* vbar,
                                       double* ubar, int32_t* status, void* stream) {
  if (!m || B < 0) return dmx_fail(DMX_ERR_INVALID, "bad argument");
  if (B == 0) return DMX_OK;
  const bool act = m->host.nu > 0;
  if (!q || !v || !abar || !qbar || !vbar || !status || (act && (!u || !ubar))) return dmx_fail(DMX_ERR_INVALID, "null array");
  const dmx::Layout& L = layout_for(m, cfd);
  const int G = lanes ? lanes : adjoint_lanes(m, B, L);
  if (!valid_adj_lanes(G)) return dmx_fail(DMX_ERR_INVALID, "lanes must be 0, 2, 4, 8, 16 or 32");
  dmx::AdjParams P{};
  P.model = m->dev; P.L = L; P.LB = dmx::make_bar_layout(m->host, L.rcap); P.B = B; P.cfd = cfd;
  int threads; size_t smem;
  if (!adj_launch_config(m, L, P.LB, G, &threads, &smem)) return dmx_fail(DMX_ERR_INVALID, "workspace does not fit");
  CK(dmx::launch_eval_rhs_vjp(G, P, q, v, act ? u : q, abar, qbar, vbar, act ? ubar : nullptr, status, threads, smem,
                              static_cast<cudaStream_t>(stream)));
  return DMX_OK;
}

extern "C" dmx_status dmx_eval_rhs(dmx_model* m, int32_t B, const double* q, const double* v, const double* u,
                                   int32_t cfd, int32_t lanes, double* a, int32_t* info, void* stream) {
  if (!m || B < 0) return dmx_fail(DMX_ERR_INVALID, "bad argument");
  if (B == 0) return DMX_OK;
  if (!q || !v || !a || !info || (m->host.nu && !u)) return dmx_fail(DMX_ERR_INVALID, "null array");
  const int G = lanes ? lanes : default_lanes(m, B);
  if (!valid_lanes(G)) return dmx_fail(DMX_ERR_INVALID, "lanes must be 0, 1, 2, 4, 8, 16 or 32");
  int threads; size_t smem;
  const dmx::Layout& L = layout_for(m, cfd);
  if (!launch_config_layout(m, L, G, &threads, &smem)) return dmx_fail(DMX_ERR_INVALID, "workspace does not fit");
  RolloutParams P{};
  P.model = m->dev; P.L = L; P.B = B;
  CK(launch_eval_rhs(G, P, q, v, m->host.nu ? u : q, cfd, a, info, threads, smem, static_cast<cudaStream_t>(stream)));
  return DMX_OK;
}

extern "C" dmx_status dmx_tape_read(const dmx_tape* t, double* hlog, int32_t* nsteps, double* ckpt, int32_t* dims,
                                    void* stream) {
  if (!t) return dmx_fail(DMX_ERR_INVALID, "null tape");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dims) { dims[0] = t->B; dims[1] = t->NI; dims[2] = t->max_steps; dims[3] = t->K; dims[4] = t->ncheck; dims[5] = t->nx; }
  if (ckpt) CK(cudaMemcpyAsync(ckpt, t->ckpt, sizeof(double) * (size_t)t->ncheck * (t->nx + 1) * t->B, cudaMemcpyDeviceToDevice, st));
  if (hlog) CK(cudaMemcpyAsync(hlog, t->hlog, sizeof(double) * (size_t)t->max_steps * t->B, cudaMemcpyDeviceToDevice, st));
  if (nsteps) CK(cudaMemcpyAsync(nsteps, t->n, sizeof(int) * (size_t)t->B, cudaMemcpyDeviceToDevice, st));
  return DMX_OK;
}
