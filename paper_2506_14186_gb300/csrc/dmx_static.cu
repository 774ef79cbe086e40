// dmx_rollout_static: the plain (one launch per step attempt) rollout with
// its per-environment integrator state in a fixed device array compiled into
// the library, for callers that must not allocate device memory during the
// call (see include/dmx.h).  Host code only; the kernels are the ordinary
// plain-form kernels, given the array's device address.
#include <cuda_runtime.h>

#include <mutex>
#include <string>

#include "dmx.h"
#include "dmx_kernels.h"
#include "dmx_model.h"
#include "dmx_runtime.h"

namespace {

// Every GPU that loads the library holds this array until the process exits.
static __device__ __align__(256) unsigned char g_static_scratch[DMX_STATIC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {};

// Device address of the array on the current device, looked up once per
// device with that device current (the host-side name is only a stand-in).
dmx_status scratch_address(int device, void** out) {
  if (device < 0 || device >= kMaxDevices) return dmx_fail(DMX_ERR_INVALID, "device ordinal out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[device]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess || !p)
      return dmx_fail(DMX_ERR_CUDA, std::string("cudaGetSymbolAddress(static scratch): ") + cudaGetErrorString(e));
    g_addr[device] = p;
  }
  *out = g_addr[device];
  return DMX_OK;
}

}  // namespace

extern "C" dmx_status dmx_rollout_static(dmx_model* m, const dmx_rollout_args* a, void* stream) {
  using namespace dmx;
  if (!m || !a) return dmx_fail(DMX_ERR_INVALID, "null argument");
  const cudaStream_t st = static_cast<cudaStream_t>(stream);
  const int nq = m->host.nq, nv = m->host.nv, nu = m->host.nu;
  if (a->B < 0) return dmx_fail(DMX_ERR_INVALID, "B must be >= 0");
  if (a->NI < 1) return dmx_fail(DMX_ERR_INVALID, "NI must be >= 1");
  if (!(a->rtol >= 0) || !(a->atol > 0) || !(a->h0 > 0)) return dmx_fail(DMX_ERR_INVALID, "rtol >= 0, atol > 0 and h0 > 0 are required");
  if (a->max_steps < 1) return dmx_fail(DMX_ERR_INVALID, "max_steps must be >= 1");
  if (a->host) return dmx_fail(DMX_ERR_INVALID, "dmx_rollout_static takes device buffers only (host = 0)");
  if (a->tape) return dmx_fail(DMX_ERR_INVALID, "dmx_rollout_static records no tape (tape must be NULL)");
  if (a->B > 0 && (!a->x0 || !a->T || !a->xT)) return dmx_fail(DMX_ERR_INVALID, "x0, T and xT are required");
  if (a->B > 0 && nu > 0 && !a->ctrl) return dmx_fail(DMX_ERR_INVALID, "ctrl is required when the model has actuators");
  const int G = a->lanes ? a->lanes : default_lanes(m, a->B);
  if (G != 1 && G != 2 && G != 4 && G != 8 && G != 16 && G != 32)
    return dmx_fail(DMX_ERR_INVALID, "lanes must be 0, 1, 2, 4, 8, 16 or 32");
  int threads;
  size_t smem;
  if (!launch_config(m, G, &threads, &smem))
    return dmx_fail(DMX_ERR_INVALID, "workspace of " + std::to_string(G) + " lanes/env does not fit shared memory");
  // per-environment state: q, v, derivative at the step start, t, h, previous
  // error (doubles); interval, counters, status, done, warm-start set (ints)
  const size_t B = (size_t)a->B;
  const size_t dbl = B * (size_t)(nq + 2 * nv + 3) * sizeof(double);
  const size_t need = dbl + B * (size_t)(6 + MASKW) * sizeof(int) + 2 * sizeof(int);
  if (need > (size_t)DMX_STATIC_SCRATCH_BYTES)
    return dmx_fail(DMX_ERR_INVALID, "B = " + std::to_string(a->B) + " needs " + std::to_string(need) +
                                         " bytes of state; the static scratch holds " +
                                         std::to_string((long long)DMX_STATIC_SCRATCH_BYTES));
  if (B == 0) return DMX_OK;
  int device = 0;
  if (cudaGetDevice(&device) != cudaSuccess) return dmx_fail(DMX_ERR_CUDA, "cudaGetDevice");
  if (device != m->device) return dmx_fail(DMX_ERR_INVALID, "model belongs to another device");
  void* base = nullptr;
  dmx_status s = scratch_address(device, &base);
  if (s != DMX_OK) return s;
  char* p = static_cast<char*>(base);
  StepState S;
  size_t off = 0;
  auto takeD = [&](size_t n) { double* r = reinterpret_cast<double*>(p + off); off += n * sizeof(double); return r; };
  auto takeI = [&](size_t n) { int* r = reinterpret_cast<int*>(p + off); off += n * sizeof(int); return r; };
  S.q = takeD(B * nq); S.v = takeD(B * nv); S.ka0 = takeD(B * nv); S.t = takeD(B); S.h = takeD(B); S.lerrp = takeD(B);
  S.k = takeI(B); S.nacc = takeI(B); S.nrej = takeI(B); S.att = takeI(B); S.st = takeI(B); S.done = takeI(B);
  S.pmask = takeI(B * MASKW);
  S.active = takeI(1);
  RolloutParams P{};
  P.model = m->dev; P.L = m->L; P.B = a->B; P.NI = a->NI; P.max_steps = a->max_steps; P.K = 1;
  P.rtol = a->rtol; P.atol = a->atol; P.h0 = a->h0; P.method = a->method;
  P.x0 = a->x0; P.ctrl = a->ctrl; P.T = a->T; P.xT = a->xT; P.xb = a->xb;
  P.nsteps = a->nsteps; P.nrej = a->nrej; P.status = a->status;
  // the unfinished-environment counter must start at B; every other field is
  // written by the initialisation launch before any attempt reads it
  int active = a->B;
  if (cudaMemcpyAsync(S.active, &active, sizeof(int), cudaMemcpyHostToDevice, st) != cudaSuccess)
    return dmx_fail(DMX_ERR_CUDA, "counter upload");
  cudaError_t e = launch_step(G, P, S, true, threads, smem, st);
  if (e != cudaSuccess) return dmx_fail(DMX_ERR_CUDA, std::string("init launch: ") + cudaGetErrorString(e));
  const long long limit = (long long)a->max_steps + 2;
  long long launched = 0;
  for (;;) {
    for (int i = 0; i < 64; ++i) {
      e = launch_step(G, P, S, false, threads, smem, st);
      if (e != cudaSuccess) return dmx_fail(DMX_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    }
    launched += 64;
    if (cudaMemcpyAsync(&active, S.active, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
      return dmx_fail(DMX_ERR_CUDA, "counter read-back");
    if (active <= 0) break;
    if (launched > limit) return dmx_fail(DMX_ERR_TIMEOUT, "did not finish within max_steps launches");
  }
  return DMX_OK;
}
