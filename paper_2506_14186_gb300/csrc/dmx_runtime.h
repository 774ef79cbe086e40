// Library-internal structures of the host runtime.
#pragma once
#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <string>
#include <utility>

#include "dmx.h"
#include "dmx_kernels.h"
#include "dmx_model.h"

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  cudaError_t ensure(size_t n);
  void free_all();
};

struct dmx_model {
  dmx::DevModel host;
  dmx::DevModel* dev = nullptr;
  dmx::Layout L;                              // workspace of the forward right-hand side (rows: rcap)
  dmx::Layout Lc;                             // workspace of the CFD right-hand side F~ (rows: rcap_c)
  int device = 0, nsm = 0, smem_max = 0, rcap = 0, rcap_c = 0;
  double invw[dmx::MAXB];
  std::mutex mu;
  std::map<std::pair<int, int>, int> tuned;   // (B, kind) -> lanes per environment
  int adj_mode = DMX_ADJ_REVERSE;             // adjoint kernel of dmx_rollout_grad
};

struct dmx_tape {
  dmx_model* model = nullptr;
  int B = 0, NI = 1, K = 1, nx = 0, nu = 0, max_steps = 0, ncheck = 0, G = 1;
  int method = 0;           // integration scheme of the taped rollout (DMX_METHOD_*)
  double rtol = 0, atol = 0, h0 = 0;
  void* mem = nullptr;
  size_t bytes = 0;
  double* ckpt = nullptr;   // [ncheck][nx+1][B]
  double* hlog = nullptr;   // [max_steps][B]
  double* ctrl = nullptr;   // [NI][nu][B]
  double* T = nullptr;      // [B]
  int* n = nullptr;         // [B] accepted steps
  cudaStream_t stream = nullptr;   // allocation stream (stream-ordered free)
};

dmx_status dmx_fail(dmx_status s, const std::string& msg);
bool launch_config(const dmx_model* m, int G, int* threads, size_t* smem);
bool launch_config_layout(const dmx_model* m, const dmx::Layout& L, int G, int* threads, size_t* smem);
// Workspace layout of a right-hand side with (cfd = 1) or without the CFD
// contacts: F~ includes every slot within w_c, so it may need more rows.
inline const dmx::Layout& layout_for(const dmx_model* m, int cfd) { return cfd ? m->Lc : m->L; }
int default_lanes(const dmx_model* m, int B);
int tuned_lanes(dmx_model* m, int B, int grad);
dmx_status run_rollout(dmx_model* m, const dmx::RolloutParams& P, int form, int G, cudaStream_t st);
int model_smem_bytes(const dmx_model* m, int groups);
// Upper bound of the device scratch that dmx_rollout_grad allocates for B
// environments with checkpoint interval K (segment buffers and, for the
// reverse kernel without CFD, the stage snapshots).
size_t adjoint_scratch_bound(dmx_model* m, int B, int K, int cfd);

namespace dmx {
int persistent_occupancy(int G, int threads, size_t smem);
}
