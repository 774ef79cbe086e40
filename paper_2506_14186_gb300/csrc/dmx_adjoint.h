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
  int method;             // METHOD_* integration scheme of the taped rollout
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
  double* snapbuf;        // reverse mode: per group, K steps x (S - 1) stage snapshots of SN doubles (or null)
  int SN;                 // doubles per snapshot
  int per, barofs;        // reverse mode: doubles per environment, offset of the cotangent workspace
  double* p_bar;          // tangent mode: [np][B] model-parameter gradients, or null
  int np;                 // model parameters differentiated when p_bar is set
  int* queue;             // next environment
};

// Offsets (doubles) of one stage snapshot: the part of a right-hand-side
// workspace that its VJP reads (poses .. geom frames, the Cholesky factor of
// the final Newton system with the solution, contact records, the used
// Jacobian rows with D and the residuals, then as ints: status, rows,
// slot->row map, row ids, final active set).
struct SnapOff {
  int n1, o2, n2, o3, o4, o5, o6, oi, size;
};
__host__ __device__ inline SnapOff snap_offsets(const DevModel& m, const Layout& L) {
  SnapOff o{};
  o.n1 = L.gp + 3 * m.ngeom - L.R;
  o.o2 = o.n1;
  o.n2 = L.tmp2 + m.nv - L.H;
  o.o3 = o.o2 + o.n2;
  o.o4 = o.o3 + 18 * m.nslot;          // contact records, then the closest-point parameters (2 per slot)
  o.o5 = o.o4 + L.rcap * m.nv;
  o.o6 = o.o5 + L.rcap;
  o.oi = o.o6 + L.rcap;
  const int nints = 3 + m.nslot + L.rcap + MASKW;
  o.size = (o.oi + (nints + 1) / 2 + 1) & ~1;
  return o;
}

// Doubles per recomputed step in the reverse kernel's segment buffer: q_n,
// the stage velocities V_0..V_6, t_n.
__host__ __device__ inline int rev_row_doubles(const DevModel& m) { return m.nq + 7 * m.nv + 1; }

cudaError_t launch_adjoint(const AdjParams& P, int blocks, cudaStream_t st);
// out[k] = sum over e of x[k][e] (k < n, e < B): one block per row, fixed order.
cudaError_t launch_row_sums(const double* x, int n, int B, double* out, cudaStream_t st);
// d (translational inverse weight of every body at qpos0) / d (parameter
// pdir) into dinvw[nbody]; ws: Layout(rcap).nd derivative scalars (16 bytes)
// + ni ints of device memory, scratch: nq + 2 nv derivative scalars.
cudaError_t launch_body_invweight_tangent(const DevModel* m, const double* qpos0, int rcap, int pdir, void* ws,
                                          void* scratch, double* dinvw, cudaStream_t st);
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
