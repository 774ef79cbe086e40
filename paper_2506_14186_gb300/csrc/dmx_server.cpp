// Request server (continuous batching of rollout / gradient requests).
#include "dmx.h"
#include "dmx_runtime.h"

struct dmx_server {
  int dummy;
};

extern "C" dmx_status dmx_server_create(const dmx_server_cfg* cfg, dmx_server** out) {
  (void)cfg; (void)out;
  return dmx_fail(DMX_ERR_UNIMPLEMENTED, "server not built yet");
}
extern "C" dmx_status dmx_submit(dmx_server* s, const dmx_request* r, uint64_t* ticket) {
  (void)s; (void)r; (void)ticket;
  return dmx_fail(DMX_ERR_UNIMPLEMENTED, "server not built yet");
}
extern "C" dmx_status dmx_poll(dmx_server* s, uint64_t ticket, double* latency_s) {
  (void)s; (void)ticket; (void)latency_s;
  return dmx_fail(DMX_ERR_UNIMPLEMENTED, "server not built yet");
}
extern "C" dmx_status dmx_server_destroy(dmx_server* s, double timeout_s) {
  (void)s; (void)timeout_s;
  return DMX_OK;
}
