// Kernel parameter blocks and launchers (host side of dmx_kernels.cu).
#pragma once
#include <cuda_runtime.h>

#include "dmx_model.h"

namespace dmx {

struct RolloutParams {
  const DevModel* model;
  Layout L;
  int B, NI, max_steps, K;
  int method;           // METHOD_* integration scheme (dmx_device.cuh)
  double rtol, atol, h0;
  const double* x0;     // [nx][B]
  const double* ctrl;   // [NI][nu][B]
  const double* T;      // [B]
  double* xT;           // [nx][B]
  double* xb;           // [NI+1][nx][B] or null
  int* nsteps;          // [B] or null
  int* nrej;            // [B] or null
  int* status;          // [B] or null
  double* ckpt;         // [ncheck][nx+1][B] or null (tape: state and time every K accepted steps)
  double* hlog;         // [max_steps][B] or null (tape: accepted step sizes)
  int* tape_n;          // [B] or null (tape: accepted steps)
  int* queue;           // persistent form: next environment
};

// Plain (one launch per attempt) form: integrator state in HBM.
struct StepState {
  double* q;            // [nq][B]
  double* v;            // [nv][B]
  double* ka0;          // [nv][B] derivative at the step start (first same as last)
  double* t;
  double* h;
  double* lerrp;        // log of the previous accepted error norm (step-size controller)
  int* k;
  int* nacc;
  int* nrej;
  int* att;
  int* st;
  int* done;
  int* pmask;           // [MASKW][B] warm-start active set
  int* active;          // unfinished environments
};

cudaError_t launch_persistent(int G, const RolloutParams& P, int blocks, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_step(int G, const RolloutParams& P, const StepState& S, bool init, int threads, size_t smem,
                        cudaStream_t st);
cudaError_t launch_eval_rhs(int G, const RolloutParams& P, const double* q, const double* v, const double* u, int cfd,
                            double* a, int* info, int threads, size_t smem, cudaStream_t st);
cudaError_t launch_body_invweight(const DevModel* m, const double* qpos0, double* invw, double* scratch, int rcap,
                                  size_t smem, cudaStream_t st);

}  // namespace dmx
