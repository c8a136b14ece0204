// mf_solver.h -- CG state and the asynchronous solver engine shared by mf_cg_solve (one
// request, host waits on the stream) and the server (many requests, host polls events).
#pragma once
#include <cuda_runtime.h>

#include "mf_internal.h"

namespace mf {

struct RedScratch;

// Workspace layout of a solve (all device pointers inside the caller's workspace).
struct SolveWs {
  CgState* st;
  RedScratch *sc1, *sc2, *sc3;
  double* hist;
  double* scal;          // [0] inner <r,r>, [1] outer ||b||^2, [2] outer ||r||^2
  double* apart;         // split-dual iteration: per-CTA partials of <p, A p> from the apply
  float *dinv, *dtab;    // Jacobi preconditioning: inverse diagonal, scratch of its computation
  float* dinv_active;    // dinv when the solve is preconditioned, else null
  void *r, *p, *q;       // CG vectors of the (inner) element type
  void *r64, *q64, *b64; // mixed: FP64 outer residual, A x, masked b
  void* d32;             // mixed: inner solution
  void* xdd;             // FP64 solver with double-float vectors: the iterate
};

// Host copy of the scalars each phase reports (pinned memory when used asynchronously).
struct HostMirror {
  CgState st;
  double bn2, rn2;
  double pad[6];
};

enum { PH_INNER = 1, PH_OUTER = 2, PH_DONE = 3 };

struct SolverEngine {
  const mf_operator* op = nullptr;
  int mixed = 0, elem_in = 8;
  cudaStream_t s = nullptr;
  SolveWs w{};
  const void* b = nullptr;
  void* x = nullptr;
  void* x_in = nullptr;
  // inner_rtol 0: 0.1 with reliable updates (a residual replacement every decade, the
  // replacement interval of Clark et al.), 1e-3 for the restarted inner CG
  double rtol = 0.0, inner_rtol = 0.0;
  int maxit = 0, chunk = 20, max_outer = 60;
  int form = MF_CG_SPLIT_DUAL; // MF_CG_SPLIT_DUAL, MF_CG_ASSEMBLED or MF_CG_SPLIT_DUAL_FUSED
  int vt = 8;                  // element type of the CG vectors (8, 4 or ELEM_DD), set at start
  int precond = MF_PRECOND_NONE;
  // mixed: continue the inner CG across defect-correction steps (reliable updates: the FP32
  // residual replaced by the FP64 one, the search direction kept) instead of restarting it;
  // the inner vectors then stay scaled by 1/||b|| for the whole solve
  bool reliable = true;
  HostMirror* hm = nullptr;
  int phase = 0, total_it = 0, outer = 0;
  double bn = 0.0, rel = 0.0;
  mf_status status = MF_OK;
  cudaGraphExec_t exec = nullptr;
  cudaGraph_t graph = nullptr;
  bool record = false, cancel = false;
  bool external = false; // inner CG iterations are run by a batch (the server), not by chunks
  bool idle = false;     // the last advance enqueued nothing (external inner CG waiting for a batch)
  int hist_off = 0;
};

size_t solve_ws_layout(const mf_operator* op, int mixed, char* base, SolveWs* w);

// A continuous batch of CG solves of one class (degree, path, kind, vector element type and
// launch variant): descriptors of all members in device memory, and the CTA counts of the
// batched launches.  batch_plan_build stages the descriptors in host (pinned) memory and
// copies them on stream s; batch_iteration enqueues one CG iteration of every member (four
// launches); batch_gather_states copies every member's CgState to states_dev[i].
struct BatchPlan {
  int n = 0, elem = 0, vk = 0;
  const mf_operator* op0 = nullptr;
  char* dev = nullptr;
  size_t jobs_off = 0, block0_off = 0, vec_off = 0;
  long long apply_blocks = 0, up_blocks = 0, pp_blocks = 0;
};
size_t batch_plan_bytes(int n, int vk);
mf_status batch_plan_build(BatchPlan* plan, const BatchMember* m, int n, int elem, void* dev, void* host_stage,
                           cudaStream_t s);
mf_status batch_iteration(const BatchPlan& plan, cudaStream_t s);
mf_status batch_gather_states(const BatchPlan& plan, CgState* states_dev, cudaStream_t s);
// the members a SolverEngine in the inner phase contributes to a batch
BatchMember engine_batch_member(const SolverEngine* e);
mf_status engine_init(SolverEngine* e, const mf_operator* op, int mixed, const void* b, void* x, double rtol, int maxit,
                      void* ws, cudaStream_t s, HostMirror* hm);
// Enqueue the first phase (ends with a D2H copy into e->hm).
mf_status engine_start(SolverEngine* e);
// Called once the last enqueued D2H copy has landed: decides and enqueues the next phase, or
// marks the engine done (e->phase == PH_DONE, result in e->status).
mf_status engine_advance(SolverEngine* e);
void engine_release(SolverEngine* e);

} // namespace mf
