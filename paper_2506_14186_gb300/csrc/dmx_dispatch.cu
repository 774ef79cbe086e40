// Host launchers: dispatch on the lane count, model set-up kernel, tableau upload.
#include <cuda_runtime.h>

#include "dmx_kernels.cuh"

namespace dmx {

#define DMX_DECLARE(G)                                                                                   \
  extern template cudaError_t launch_persistent_g<G>(const RolloutParams&, int, int, size_t, cudaStream_t); \
  extern template cudaError_t launch_step_g<G>(const RolloutParams&, const StepState&, bool, int, size_t, cudaStream_t); \
  extern template int occupancy_g<G>(int, size_t); \
  extern template cudaError_t launch_eval_rhs_g<G>(const RolloutParams&, const double*, const double*, const double*, \
                                                   int, double*, int*, int, size_t, cudaStream_t);
DMX_DECLARE(1)
DMX_DECLARE(2)
DMX_DECLARE(4)
DMX_DECLARE(8)
DMX_DECLARE(16)
DMX_DECLARE(32)

// Model set-up: translational inverse weight of every body at qpos0,
// trace(Jc M^-1 Jc^T) / 3 (one environment, one lane).
__global__ void k_body_invweight(const DevModel* mp, const double* qpos0, double* invw, double* scratch, int rcap) {
  extern __shared__ double smem[];
  __shared__ Layout sL;
  const DevModel& m = *mp;
  if (threadIdx.x != 0) return;
  sL = make_layout(m, rcap);
  Grp<1> g;
  Ws w;
  w.d = smem;
  w.i = reinterpret_cast<int*>(smem + sL.nd);
  w.L = &sL;
  kinematics(g, m, w, qpos0);
  crba(g, m, w);
  double* H = w.at(sL.H); const double* M = w.at(sL.M);
  for (int i = 0; i < m.nv * m.nv; ++i) H[i] = M[i];
  cholesky(g, H, w.at(sL.tmp2), m.nv);
  const double* S = w.at(sL.sd); const double* C = w.at(sL.com);
  double* col = scratch;
  double* x = scratch + m.nv;
  for (int b = 0; b < m.nbody; ++b) {
    double tr = 0;
    for (int ax = 0; ax < 3; ++ax) {
      for (int i = 0; i < m.nv; ++i) {
        const bool moves = (m.b_anc[b] >> m.dof_body[i]) & 1u;
        double pv[3] = {0, 0, 0};
        if (moves) {
          cross3(S + 6 * i, C + 3 * b, pv);
          pv[0] += S[6 * i + 3]; pv[1] += S[6 * i + 4]; pv[2] += S[6 * i + 5];
        }
        col[i] = pv[ax];
        x[i] = pv[ax];
      }
      chol_solve(g, H, w.at(sL.tmp2), x, m.nv);
      for (int i = 0; i < m.nv; ++i) tr += col[i] * x[i];
    }
    invw[b] = tr / 3.0;
  }
}

cudaError_t launch_persistent(int G, const RolloutParams& P, int blocks, int threads, size_t smem, cudaStream_t st) {
  switch (G) {
    case 1: return launch_persistent_g<1>(P, blocks, threads, smem, st);
    case 2: return launch_persistent_g<2>(P, blocks, threads, smem, st);
    case 4: return launch_persistent_g<4>(P, blocks, threads, smem, st);
    case 8: return launch_persistent_g<8>(P, blocks, threads, smem, st);
    case 16: return launch_persistent_g<16>(P, blocks, threads, smem, st);
    case 32: return launch_persistent_g<32>(P, blocks, threads, smem, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t launch_eval_rhs(int G, const RolloutParams& P, const double* q, const double* v, const double* u, int cfd,
                            double* a, int* info, int threads, size_t smem, cudaStream_t st) {
  switch (G) {
    case 1: return launch_eval_rhs_g<1>(P, q, v, u, cfd, a, info, threads, smem, st);
    case 2: return launch_eval_rhs_g<2>(P, q, v, u, cfd, a, info, threads, smem, st);
    case 4: return launch_eval_rhs_g<4>(P, q, v, u, cfd, a, info, threads, smem, st);
    case 8: return launch_eval_rhs_g<8>(P, q, v, u, cfd, a, info, threads, smem, st);
    case 16: return launch_eval_rhs_g<16>(P, q, v, u, cfd, a, info, threads, smem, st);
    case 32: return launch_eval_rhs_g<32>(P, q, v, u, cfd, a, info, threads, smem, st);
  }
  return cudaErrorInvalidValue;
}
int persistent_occupancy(int G, int threads, size_t smem) {
  switch (G) {
    case 1: return occupancy_g<1>(threads, smem);
    case 2: return occupancy_g<2>(threads, smem);
    case 4: return occupancy_g<4>(threads, smem);
    case 8: return occupancy_g<8>(threads, smem);
    case 16: return occupancy_g<16>(threads, smem);
    case 32: return occupancy_g<32>(threads, smem);
  }
  return 0;
}
cudaError_t launch_step(int G, const RolloutParams& P, const StepState& S, bool init, int threads, size_t smem,
                        cudaStream_t st) {
  switch (G) {
    case 1: return launch_step_g<1>(P, S, init, threads, smem, st);
    case 2: return launch_step_g<2>(P, S, init, threads, smem, st);
    case 4: return launch_step_g<4>(P, S, init, threads, smem, st);
    case 8: return launch_step_g<8>(P, S, init, threads, smem, st);
    case 16: return launch_step_g<16>(P, S, init, threads, smem, st);
    case 32: return launch_step_g<32>(P, S, init, threads, smem, st);
  }
  return cudaErrorInvalidValue;
}
cudaError_t launch_body_invweight(const DevModel* m, const double* qpos0, double* invw, double* scratch, int rcap,
                                  size_t smem, cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(k_body_invweight, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_body_invweight<<<1, 32, smem, st>>>(m, qpos0, invw, scratch, rcap);
  return cudaGetLastError();
}

}  // namespace dmx
