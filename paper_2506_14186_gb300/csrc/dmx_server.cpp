// Request server: continuous batching of rollout and gradient requests.
//
// dmx_submit queues a request (host buffers) and returns at once.  A worker
// thread admits queued requests in arrival order as soon as an in-flight slot
// and enough of the device-memory budget are free, and issues each admitted
// request on its own CUDA stream: stream-ordered allocation of its device
// state (inputs, outputs, tape), host-to-device copies, the persistent
// rollout kernel, the adjoint kernel for gradient requests, device-to-host
// copies, stream-ordered release, and a host callback that stamps the
// completion time and frees the slot.  Requests that arrive while others run
// are therefore admitted while those are still on the device, and their
// kernels overlap.  Each environment's arithmetic does not depend on what else
// runs, so a request's result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "dmx.h"
#include "dmx_runtime.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DONE = 2, REQ_FAILED = 3 };

}  // namespace

struct dmx_server;

struct ServerRequest {
  uint64_t ticket = 0;
  dmx_request r{};
  size_t bytes = 0;
  double t_submit = 0, t_done = 0;
  std::atomic<int> state{REQ_QUEUED};
  dmx_status err = DMX_OK;
  std::string msg;
  dmx_server* srv = nullptr;
};

struct dmx_server {
  dmx_server_cfg cfg{};
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ServerRequest*> queue;
  std::map<uint64_t, ServerRequest*> reqs;
  int inflight = 0;
  int64_t mem_used = 0;
  uint64_t next_ticket = 1, issued = 0;
  bool stop = false;
};

// Device bytes a request holds while it runs (inputs, outputs, tape, adjoint scratch).
static size_t request_bytes(const dmx_request& r) {
  int32_t nq = 0, nv = 0, nu = 0;
  dmx_model_dims(r.model, &nq, &nv, &nu);
  const size_t nx = nq + nv, B = r.B;
  size_t d = B * nx * 2 + (size_t)r.NI * nu * B + B;     // x0, xT, ctrl, T
  if (r.grad) {
    const size_t K = r.K > 0 ? r.K : 32;
    d += B * nx * 2 + (size_t)r.NI * nu * B;             // xT_bar, x0_bar, ctrl_bar
    d += (size_t)(r.max_steps / K + 2) * (nx + 1) * B + (size_t)r.max_steps * B + (size_t)r.NI * nu * B + B;  // tape
  }
  size_t extra = 0;
  if (r.grad) extra = adjoint_scratch_bound(r.model, r.B, r.K > 0 ? r.K : 32, r.cfd);   // segment buffers, snapshots
  return d * sizeof(double) + extra + 2 * B * sizeof(int) + 4096;
}

static void CUDART_CB on_done(void* p) {
  ServerRequest* q = static_cast<ServerRequest*>(p);
  dmx_server* s = q->srv;
  std::lock_guard<std::mutex> lk(s->mu);
  q->t_done = now_s();
  q->state = REQ_DONE;
  s->inflight -= 1;
  s->mem_used -= (int64_t)q->bytes;
  s->cv.notify_all();
}

// Issues one admitted request on `st`; on failure the request is marked failed.
static void issue(dmx_server* s, ServerRequest* q, cudaStream_t st) {
  const dmx_request& r = q->r;
  auto fail = [&](dmx_status e, const std::string& m) {
    std::lock_guard<std::mutex> lk(s->mu);
    q->err = e;
    q->msg = m;
    q->t_done = now_s();
    q->state = REQ_FAILED;
    s->inflight -= 1;
    s->mem_used -= (int64_t)q->bytes;
    s->cv.notify_all();
  };
  int32_t nq = 0, nv = 0, nu = 0;
  dmx_model_dims(r.model, &nq, &nv, &nu);
  const size_t nx = nq + nv, B = r.B;
  const size_t n_x = nx * B, n_u = (size_t)r.NI * nu * B;
  const size_t doubles = 2 * n_x + n_u + B + (r.grad ? 2 * n_x + n_u : 0);
  void* mem = nullptr;
  if (cudaMallocAsync(&mem, doubles * sizeof(double) + 2 * B * sizeof(int) + 256, st) != cudaSuccess)
    return fail(DMX_ERR_OOM, "request device state");
  double* p = static_cast<double*>(mem);
  double* x0 = p; p += n_x;
  double* xT = p; p += n_x;
  double* ctrl = p; p += n_u;
  double* T = p; p += B;
  double *xTb = nullptr, *x0b = nullptr, *cb = nullptr;
  if (r.grad) { xTb = p; p += n_x; x0b = p; p += n_x; cb = p; p += n_u; }
  int* status = reinterpret_cast<int*>(p);
  int* nsteps = status + B;
  bool ok = cudaMemcpyAsync(x0, r.x0, n_x * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (nu) ok = ok && cudaMemcpyAsync(ctrl, r.ctrl, n_u * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess;
  ok = ok && cudaMemcpyAsync(T, r.T, B * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (r.grad) ok = ok && cudaMemcpyAsync(xTb, r.xT_bar, n_x * sizeof(double), cudaMemcpyHostToDevice, st) == cudaSuccess;
  if (!ok) { cudaFreeAsync(mem, st); return fail(DMX_ERR_CUDA, "request upload"); }
  dmx_rollout_args a{};
  a.B = r.B; a.x0 = x0; a.ctrl = nu ? ctrl : nullptr; a.T = T; a.NI = r.NI; a.rtol = r.rtol; a.atol = r.atol;
  a.h0 = r.h0; a.max_steps = r.max_steps; a.K = r.K > 0 ? r.K : 32; a.form = DMX_FORM_PERSISTENT; a.lanes = 0;
  a.host = 0; a.xT = xT; a.xb = nullptr; a.nsteps = nsteps; a.nrej = nullptr; a.status = status;
  dmx_tape* tape = nullptr;
  a.tape = r.grad ? &tape : nullptr;
  dmx_status e = dmx_rollout(r.model, &a, st);
  if (e == DMX_OK && r.grad) {
    e = dmx_rollout_grad(r.model, tape, r.cfd, xTb, nullptr, x0b, nu ? cb : nullptr, st);
    dmx_tape_free(tape);   // stream ordered after the adjoint
  }
  if (e != DMX_OK) { cudaFreeAsync(mem, st); return fail(e, dmx_last_error()); }
  ok = cudaMemcpyAsync(r.xT, xT, n_x * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess;
  if (r.status) ok = ok && cudaMemcpyAsync(r.status, status, B * sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess;
  if (r.grad) {
    ok = ok && cudaMemcpyAsync(r.x0_bar, x0b, n_x * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess;
    if (nu) ok = ok && cudaMemcpyAsync(r.ctrl_bar, cb, n_u * sizeof(double), cudaMemcpyDeviceToHost, st) == cudaSuccess;
  }
  ok = ok && cudaFreeAsync(mem, st) == cudaSuccess;
  ok = ok && cudaLaunchHostFunc(st, on_done, q) == cudaSuccess;
  if (!ok) return fail(DMX_ERR_CUDA, "request issue");
}

static void worker_loop(dmx_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    while (!s->queue.empty()) {
      ServerRequest* q = s->queue.front();
      if (s->inflight >= s->cfg.max_inflight || s->mem_used + (int64_t)q->bytes > s->cfg.device_bytes) break;
      s->queue.pop_front();
      s->inflight += 1;
      s->mem_used += (int64_t)q->bytes;
      q->state = REQ_RUNNING;
      cudaStream_t st = s->streams[s->issued++ % s->streams.size()];
      lk.unlock();
      issue(s, q, st);
      lk.lock();
    }
    if (s->stop && s->queue.empty() && s->inflight == 0) break;
    s->cv.wait_for(lk, std::chrono::milliseconds(2));
  }
}

extern "C" dmx_status dmx_server_create(const dmx_server_cfg* cfg, dmx_server** out) {
  if (!cfg || !out) return dmx_fail(DMX_ERR_INVALID, "null argument");
  if (cfg->device_bytes <= 0 || cfg->max_inflight < 1 || cfg->nstreams < 1)
    return dmx_fail(DMX_ERR_INVALID, "device_bytes, max_inflight and nstreams must be positive");
  dmx_server* s = new dmx_server();
  s->cfg = *cfg;
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return dmx_fail(DMX_ERR_CUDA, "cudaGetDevice"); }
  for (int i = 0; i < cfg->nstreams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      delete s;
      return dmx_fail(DMX_ERR_CUDA, "stream creation");
    }
    s->streams.push_back(st);
  }
  s->worker = std::thread(worker_loop, s);
  *out = s;
  return DMX_OK;
}

extern "C" dmx_status dmx_submit(dmx_server* s, const dmx_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return dmx_fail(DMX_ERR_INVALID, "null argument");
  if (!r->model || r->B < 0 || r->NI < 1 || r->max_steps < 1 || !(r->rtol > 0) || !(r->atol > 0) || !(r->h0 > 0))
    return dmx_fail(DMX_ERR_INVALID, "bad request sizes or tolerances");
  int32_t nu = 0;
  dmx_model_dims(r->model, nullptr, nullptr, &nu);
  if (r->B > 0 && (!r->x0 || !r->T || !r->xT || (nu && !r->ctrl)))
    return dmx_fail(DMX_ERR_INVALID, "x0, T, xT (and ctrl) are required");
  if (r->grad && (!r->xT_bar || !r->x0_bar || (nu && !r->ctrl_bar)))
    return dmx_fail(DMX_ERR_INVALID, "gradient requests need xT_bar, x0_bar (and ctrl_bar)");
  ServerRequest* q = new ServerRequest();
  q->r = *r;
  q->bytes = request_bytes(*r);
  q->srv = s;
  if ((int64_t)q->bytes > s->cfg.device_bytes) {
    const size_t b = q->bytes;
    delete q;
    return dmx_fail(DMX_ERR_INVALID, "request needs " + std::to_string(b) + " device bytes, more than the server budget");
  }
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->stop) { delete q; return dmx_fail(DMX_ERR_INVALID, "server is shutting down"); }
    q->ticket = s->next_ticket++;
    q->t_submit = now_s();
    if (r->B == 0) { q->state = REQ_DONE; q->t_done = q->t_submit; }
    else s->queue.push_back(q);
    s->reqs[q->ticket] = q;
    *ticket = q->ticket;
  }
  s->cv.notify_all();
  return DMX_OK;
}

extern "C" dmx_status dmx_poll(dmx_server* s, uint64_t ticket, double* latency_s) {
  if (!s) return dmx_fail(DMX_ERR_INVALID, "null server");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->reqs.find(ticket);
  if (it == s->reqs.end()) return dmx_fail(DMX_ERR_INVALID, "unknown ticket");
  ServerRequest* q = it->second;
  const int st = q->state.load();
  if (st == REQ_QUEUED || st == REQ_RUNNING) return DMX_NOT_READY;
  if (latency_s) *latency_s = q->t_done - q->t_submit;
  const dmx_status e = st == REQ_DONE ? DMX_OK : q->err;
  if (st == REQ_FAILED) dmx_fail(e, q->msg);
  s->reqs.erase(it);
  delete q;
  return e;
}

extern "C" dmx_status dmx_server_destroy(dmx_server* s, double timeout_s) {
  if (!s) return DMX_OK;
  const double deadline = now_s() + timeout_s;
  {
    std::unique_lock<std::mutex> lk(s->mu);
    s->stop = true;
    s->cv.notify_all();
    while (!(s->queue.empty() && s->inflight == 0)) {
      if (now_s() > deadline) return dmx_fail(DMX_ERR_TIMEOUT, "requests still running; server not destroyed");
      s->cv.wait_for(lk, std::chrono::milliseconds(2));
    }
  }
  s->worker.join();
  for (cudaStream_t st : s->streams) {
    cudaStreamSynchronize(st);
    cudaStreamDestroy(st);
  }
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return DMX_OK;
}
