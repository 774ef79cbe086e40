// Parameter block and launcher of the adjoint kernel (dmx_adjoint.cu).
#pragma once
#include <cuda_runtime.h>

#include "dmx_model.h"

namespace dmx {

struct AdjParams {
  const DevModel* model;
  Layout L;
  LayoutBar LB;           // reverse-mode kernel: cotangent workspace
  int B, NI, K, cfd;
  const double* ckpt;     // [ncheck][nx+1][B] tape checkpoints (state, time)
  const double* hlog;     // [max_steps][B] accepted step sizes
  const int* tape_n;      // [B] accepted steps
  const double* ctrl;     // [NI][nu][B] controls of the taped rollout
  const double* T;        // [B] horizons
  const double* xT_bar;   // [nx][B]
  const double* xb_bar;   // [NI+1][nx][B] or null
  double* x0_bar;         // [nx][B]
  double* ctrl_bar;       // [NI][nu][B] or null
  double* segbuf;         // per warp (tangent) or group (reverse): recomputed steps of a segment
  int* queue;             // next environment
};

cudaError_t launch_adjoint(const AdjParams& P, int blocks, cudaStream_t st);
// reverse-mode kernel, G lanes per environment (G = 2, 4, 8, 16, 32)
cudaError_t launch_adjoint_rev(int G, const AdjParams& P, int blocks, int threads, size_t smem, cudaStream_t st);
int adjoint_rev_occupancy(int G, int threads, size_t smem);
cudaError_t launch_eval_rhs_vjp(int G, const AdjParams& P, const double* q, const double* v, const double* u,
                                const double* abar, double* qbar, double* vbar, double* ubar, int* status, int threads,
                                size_t smem, cudaStream_t st);
int adjoint_warps_per_block();
int adjoint_workspace_limit();
int adjoint_int_limit();

}  // namespace dmx
