// Request server: continuous batching of rollout and gradient requests.
//
// dmx_submit queues a request (host buffers) and returns at once.  A worker
// thread admits queued requests in arrival order as soon as an in-flight slot
// and enough of the device-memory budget are free, and issues each admitted
// request on one of the server's CUDA streams: copy of its inputs into the
// slot's page-locked staging block, stream-ordered allocation of its device
// state, host-to-device copies, the persistent rollout kernel, the adjoint
// kernel for gradient requests, device-to-host copies into the staging block,
// stream-ordered release, and a host callback that hands the request back to
// the worker.  The worker then copies the outputs into the caller's buffers,
// stamps the completion time and frees the slot.  No call of the worker waits
// for device work (every copy the device sees is between device memory and
// page-locked memory), so requests that arrive while others run are admitted
// and issued while those are still on the device, and their kernels overlap.
// Each environment's arithmetic does not depend on what else runs, so a
// request's result is the same alone and in the mix.
#include <cuda_runtime.h>

#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
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

enum { REQ_QUEUED = 0, REQ_RUNNING = 1, REQ_DEVICE_DONE = 2, REQ_DONE = 3, REQ_FAILED = 4 };

constexpr size_t kStageAlign = 256;
constexpr int64_t kDefaultStagePerSlot = 32ll << 20;

size_t align_up(size_t n) { return (n + kStageAlign - 1) & ~(kStageAlign - 1); }

// Sizes of one request's arrays (doubles, except the int status array).
struct Sizes {
  size_t nx = 0, nu = 0, B = 0, n_x = 0, n_u = 0;
};
Sizes sizes_of(const dmx_request& r) {
  int32_t nq = 0, nv = 0, nu = 0;
  dmx_model_dims(r.model, &nq, &nv, &nu);
  Sizes z;
  z.nx = nq + nv; z.nu = nu; z.B = r.B;
  z.n_x = z.nx * z.B; z.n_u = (size_t)r.NI * z.nu * z.B;
  return z;
}

// Byte offsets of a request's arrays inside its staging block (the same
// layout is used for the device state).
struct StageLayout {
  size_t x0, ctrl, T, xTb, xT, x0b, cb, status, nsteps, bytes;
};
StageLayout stage_layout(const dmx_request& r) {
  const Sizes z = sizes_of(r);
  StageLayout L{};
  size_t o = 0;
  auto take = [&](size_t n) { size_t at = o; o += align_up(n); return at; };
  L.x0 = take(z.n_x * sizeof(double));
  L.ctrl = take(z.n_u * sizeof(double));
  L.T = take(z.B * sizeof(double));
  L.xTb = take(r.grad ? z.n_x * sizeof(double) : 0);
  L.xT = take(z.n_x * sizeof(double));
  L.x0b = take(r.grad ? z.n_x * sizeof(double) : 0);
  L.cb = take(r.grad ? z.n_u * sizeof(double) : 0);
  L.status = take(z.B * sizeof(int32_t));
  L.nsteps = take(z.B * sizeof(int32_t));   // device only (not copied back)
  L.bytes = o;
  return L;
}

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
  char* stage = nullptr;          // page-locked staging block of the request's slot
};

struct dmx_server {
  dmx_server_cfg cfg{};
  int device = 0;
  std::vector<cudaStream_t> streams;
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<ServerRequest*> queue;
  std::deque<ServerRequest*> finished;      // device work done, outputs still in staging
  std::map<uint64_t, ServerRequest*> reqs;
  void* stage_mem = nullptr;
  size_t slot_bytes = 0;
  std::vector<char*> free_slots;
  int inflight = 0;
  int64_t mem_used = 0;
  uint64_t next_ticket = 1, issued = 0;
  bool stop = false;
};

// Device bytes a request holds while it runs (inputs, outputs, tape, adjoint scratch).
static size_t request_bytes(const dmx_request& r) {
  const Sizes z = sizes_of(r);
  const size_t B = z.B, nx = z.nx;
  size_t d = 0;
  if (r.grad) {
    const size_t K = r.K > 0 ? r.K : 32;
    d += (size_t)(r.max_steps / K + 2) * (nx + 1) * B + (size_t)r.max_steps * B + z.n_u + B;   // tape
  }
  size_t extra = 0;
  if (r.grad) extra = adjoint_scratch_bound(r.model, r.B, r.K > 0 ? r.K : 32, r.cfd);   // segment buffers, snapshots
  return stage_layout(r).bytes + d * sizeof(double) + extra + 4096;
}

static void CUDART_CB on_device_done(void* p) {
  ServerRequest* q = static_cast<ServerRequest*>(p);
  dmx_server* s = q->srv;
  std::lock_guard<std::mutex> lk(s->mu);
  q->state = REQ_DEVICE_DONE;
  s->finished.push_back(q);
  s->cv.notify_all();
}

// Releases the slot, budget and staging block of a request (lock held).
static void release(dmx_server* s, ServerRequest* q) {
  s->inflight -= 1;
  s->mem_used -= (int64_t)q->bytes;
  if (q->stage) s->free_slots.push_back(q->stage);
  q->stage = nullptr;
}

// Issues one admitted request on `st`; on failure the request is marked failed.
static void issue(dmx_server* s, ServerRequest* q, cudaStream_t st) {
  const dmx_request& r = q->r;
  bool enqueued = false;   // copies from or to the staging block are queued on st
  auto fail = [&](dmx_status e, const std::string& m) {
    if (enqueued) cudaStreamSynchronize(st);   // the staging block is reused once released
    std::lock_guard<std::mutex> lk(s->mu);
    q->err = e;
    q->msg = m;
    q->t_done = now_s();
    q->state = REQ_FAILED;
    release(s, q);
    s->cv.notify_all();
  };
  const Sizes z = sizes_of(r);
  const StageLayout L = stage_layout(r);
  char* h = q->stage;
  // inputs into the page-locked block (host copies: the caller's buffers may be pageable)
  std::memcpy(h + L.x0, r.x0, z.n_x * sizeof(double));
  if (z.nu) std::memcpy(h + L.ctrl, r.ctrl, z.n_u * sizeof(double));
  std::memcpy(h + L.T, r.T, z.B * sizeof(double));
  if (r.grad) std::memcpy(h + L.xTb, r.xT_bar, z.n_x * sizeof(double));
  void* mem = nullptr;
  if (cudaMallocAsync(&mem, L.bytes, st) != cudaSuccess) return fail(DMX_ERR_OOM, "request device state");
  char* d = static_cast<char*>(mem);
  const size_t in_bytes = L.xT;   // x0, ctrl, T, xT_bar are contiguous at the start of the layout
  enqueued = true;
  if (cudaMemcpyAsync(d, h, in_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess) {
    cudaFreeAsync(mem, st);
    return fail(DMX_ERR_CUDA, "request upload");
  }
  double* x0 = reinterpret_cast<double*>(d + L.x0);
  double* ctrl = reinterpret_cast<double*>(d + L.ctrl);
  double* T = reinterpret_cast<double*>(d + L.T);
  double* xTb = reinterpret_cast<double*>(d + L.xTb);
  double* xT = reinterpret_cast<double*>(d + L.xT);
  double* x0b = reinterpret_cast<double*>(d + L.x0b);
  double* cb = reinterpret_cast<double*>(d + L.cb);
  int* status = reinterpret_cast<int*>(d + L.status);
  int* nsteps = reinterpret_cast<int*>(d + L.nsteps);
  dmx_rollout_args a{};
  a.B = r.B; a.x0 = x0; a.ctrl = z.nu ? ctrl : nullptr; a.T = T; a.NI = r.NI; a.rtol = r.rtol; a.atol = r.atol;
  a.h0 = r.h0; a.max_steps = r.max_steps; a.K = r.K > 0 ? r.K : 32; a.form = DMX_FORM_PERSISTENT; a.lanes = 0;
  a.host = 0; a.xT = xT; a.xb = nullptr; a.nsteps = nsteps; a.nrej = nullptr; a.status = status;
  dmx_tape* tape = nullptr;
  a.tape = r.grad ? &tape : nullptr;
  dmx_status e = dmx_rollout(r.model, &a, st);
  if (e == DMX_OK && r.grad) {
    e = dmx_rollout_grad(r.model, tape, r.cfd, xTb, nullptr, x0b, z.nu ? cb : nullptr, st);
    dmx_tape_free(tape);   // stream ordered after the adjoint
  }
  if (e != DMX_OK) { cudaFreeAsync(mem, st); return fail(e, dmx_last_error()); }
  // outputs (xT, x0_bar, ctrl_bar, status) are contiguous from L.xT on
  const size_t out_bytes = L.status + z.B * sizeof(int32_t) - L.xT;
  bool ok = cudaMemcpyAsync(h + L.xT, d + L.xT, out_bytes, cudaMemcpyDeviceToHost, st) == cudaSuccess;
  ok = ok && cudaFreeAsync(mem, st) == cudaSuccess;
  ok = ok && cudaLaunchHostFunc(st, on_device_done, q) == cudaSuccess;
  if (!ok) return fail(DMX_ERR_CUDA, "request issue");
}

// Outputs of a request whose device work has finished: staging -> caller
// buffers, then the request is done (lock held; the copies are host memcpys).
static void finish(dmx_server* s, ServerRequest* q) {
  const dmx_request& r = q->r;
  const Sizes z = sizes_of(r);
  const StageLayout L = stage_layout(r);
  const char* h = q->stage;
  std::memcpy(r.xT, h + L.xT, z.n_x * sizeof(double));
  if (r.status) std::memcpy(r.status, h + L.status, z.B * sizeof(int32_t));
  if (r.grad) {
    std::memcpy(r.x0_bar, h + L.x0b, z.n_x * sizeof(double));
    if (z.nu) std::memcpy(r.ctrl_bar, h + L.cb, z.n_u * sizeof(double));
  }
  q->t_done = now_s();
  q->state = REQ_DONE;
  release(s, q);
}

static void worker_loop(dmx_server* s) {
  cudaSetDevice(s->device);
  std::unique_lock<std::mutex> lk(s->mu);
  for (;;) {
    while (!s->finished.empty()) {
      ServerRequest* q = s->finished.front();
      s->finished.pop_front();
      finish(s, q);
    }
    while (!s->queue.empty()) {
      ServerRequest* q = s->queue.front();
      if (s->inflight >= s->cfg.max_inflight || s->free_slots.empty() ||
          s->mem_used + (int64_t)q->bytes > s->cfg.device_bytes)
        break;
      s->queue.pop_front();
      s->inflight += 1;
      s->mem_used += (int64_t)q->bytes;
      q->stage = s->free_slots.back();
      s->free_slots.pop_back();
      q->state = REQ_RUNNING;
      cudaStream_t st = s->streams[s->issued++ % s->streams.size()];
      lk.unlock();
      issue(s, q, st);
      lk.lock();
      while (!s->finished.empty()) {   // hand back finished requests between issues
        ServerRequest* f = s->finished.front();
        s->finished.pop_front();
        finish(s, f);
      }
    }
    if (s->stop && s->queue.empty() && s->inflight == 0) break;
    s->cv.wait_for(lk, std::chrono::milliseconds(2));
  }
}

extern "C" dmx_status dmx_server_create(const dmx_server_cfg* cfg, dmx_server** out) {
  if (!cfg || !out) return dmx_fail(DMX_ERR_INVALID, "null argument");
  if (cfg->device_bytes <= 0 || cfg->max_inflight < 1 || cfg->nstreams < 1 || cfg->host_stage_bytes < 0)
    return dmx_fail(DMX_ERR_INVALID, "device_bytes, max_inflight and nstreams must be positive");
  dmx_server* s = new dmx_server();
  s->cfg = *cfg;
  if (cudaGetDevice(&s->device) != cudaSuccess) { delete s; return dmx_fail(DMX_ERR_CUDA, "cudaGetDevice"); }
  const int64_t total = cfg->host_stage_bytes > 0 ? cfg->host_stage_bytes : kDefaultStagePerSlot * cfg->max_inflight;
  s->slot_bytes = (size_t)(total / cfg->max_inflight) & ~(kStageAlign - 1);
  if (s->slot_bytes < kStageAlign) { delete s; return dmx_fail(DMX_ERR_INVALID, "host_stage_bytes too small"); }
  if (cudaHostAlloc(&s->stage_mem, s->slot_bytes * cfg->max_inflight, cudaHostAllocPortable) != cudaSuccess) {
    delete s;
    return dmx_fail(DMX_ERR_OOM, "page-locked staging of " + std::to_string(s->slot_bytes * cfg->max_inflight) + " bytes");
  }
  for (int i = cfg->max_inflight - 1; i >= 0; --i) s->free_slots.push_back(static_cast<char*>(s->stage_mem) + i * s->slot_bytes);
  for (int i = 0; i < cfg->nstreams; ++i) {
    cudaStream_t st;
    if (cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
      for (cudaStream_t x : s->streams) cudaStreamDestroy(x);
      cudaFreeHost(s->stage_mem);
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
  if (!r->model || r->B < 0 || r->NI < 1 || r->max_steps < 1 || !(r->rtol >= 0) || !(r->atol > 0) || !(r->h0 > 0))
    return dmx_fail(DMX_ERR_INVALID, "bad request sizes or tolerances");
  int32_t nu = 0;
  dmx_model_dims(r->model, nullptr, nullptr, &nu);
  if (r->B > 0 && (!r->x0 || !r->T || !r->xT || (nu && !r->ctrl)))
    return dmx_fail(DMX_ERR_INVALID, "x0, T, xT (and ctrl) are required");
  if (r->grad && (!r->xT_bar || !r->x0_bar || (nu && !r->ctrl_bar)))
    return dmx_fail(DMX_ERR_INVALID, "gradient requests need xT_bar, x0_bar (and ctrl_bar)");
  const size_t stage = stage_layout(*r).bytes;
  if (stage > s->slot_bytes)
    return dmx_fail(DMX_ERR_INVALID, "request needs " + std::to_string(stage) + " bytes of host staging, more than the " +
                                         std::to_string(s->slot_bytes) + " of one in-flight slot");
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
  if (st == REQ_QUEUED || st == REQ_RUNNING || st == REQ_DEVICE_DONE) return DMX_NOT_READY;
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
  cudaFreeHost(s->stage_mem);
  for (auto& kv : s->reqs) delete kv.second;
  delete s;
  return DMX_OK;
}
