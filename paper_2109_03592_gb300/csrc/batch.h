// Batched mixed-precision PCG engine (see batch.cu): the host side used by
// sem_pcg_solve_batch and by the request server.
#pragma once

#include "sem_internal.h"

namespace sem {
namespace batch {

// One request inside an engine (mirrors the single-request reliable-update solve).
struct Req {
  sem_mesh* m = nullptr;
  struct Workspace* ws = nullptr;
  bool own_ws = false;        // ws was allocated for this request (the mesh's was in use)
  const double* b = nullptr;  // device, FP64
  double* x = nullptr;        // device, FP64 (in: initial guess, out: solution)
  sem_solve_opts o{};         // prec SEM_MIXED, refine 0, defaults filled in
  sem_solve_result* out = nullptr;
  double bnorm = 0.0, scale = 0.0;
  int outer = 0, slot = -1;
  bool finished = false;
  sem_status status = SEM_OK;
  void* user = nullptr;  // owner's cookie
};

class EngineImpl;

// A batch of up to 32 requests of one odd order N, advanced together by one
// CUDA graph per step.
class Engine {
 public:
  explicit Engine(int N);
  ~Engine();
  sem_status init(cudaStream_t user);
  // Order the engine after `user` (a cached engine serving another call).
  sem_status attach(cudaStream_t user);
  // FP64 set-up of a request and its activation in a free slot; SEM_ERR_BUSY
  // when every slot is taken.  The request may finish inside add() (b = 0 or
  // x already converged).
  sem_status add(Req* q);
  // add() for several requests at once, their FP64 set-up overlapping on the
  // GPU; takes at most the free slots (*taken: how many, in order).
  sem_status add_many(Req* const* qs, int count, int* taken);
  // One graph launch, then the FP64 work of the requests that paused.
  sem_status step();
  bool idle() const;
  int order() const;
  // After a failure: drop every request the engine holds (each request's own
  // workspace goes back to its mesh, to be freed with it) once their streams
  // are idle, so that the engine keeps no pointer to a request or mesh the
  // caller releases next.  The requests are left unfinished.
  void abandon();

 private:
  EngineImpl* impl_;
};

}  // namespace batch
}  // namespace sem
