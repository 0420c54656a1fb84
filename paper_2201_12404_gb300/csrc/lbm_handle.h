// Host-side state behind an lbm_handle (shared by the host translation units).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_ops.h"

struct lbm_domain {
  lbm::TileMaps maps;  // halo tiles of (rho, psi) and q for the collide kernel's TMA loads
  lbm_params p{};
  const lbm::Ops* ops = nullptr;
  lbm::DevDomain dev{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int parity = 0;
  int64_t steps = 0;
  int64_t launches = 0;
  bool poisoned = false;
  std::string err;
  // error flags: device word, pinned host mirror, event marking the mirror's copy
  unsigned int* h_flags = nullptr;
  cudaEvent_t flags_ev = nullptr;
  bool flags_pending = false;
  // timing
  bool timing = false;
  std::vector<cudaEvent_t> ev_pool;
  struct Mark { int kind; cudaEvent_t a, b; };
  std::vector<Mark> marks;
  double ms[2] = {0, 0};
  int64_t cnt[2] = {0, 0};
  bool record_gamma = false;
  bool gamma_recorded = false;  // a step has run with recording on since the buffer was made
  // CUDA graphs of two consecutive steps starting at parity p (the three kernels of
  // parity p, then of 1 - p), replayed by lbm_step when timing is off.  A graph holds
  // the kernel arguments of its capture, so it is keyed by the only device pointer
  // that changes after creation, the gamma record (nullptr while not recording).
  cudaGraphExec_t step_graph[2] = {nullptr, nullptr};
  float* step_graph_gamma[2] = {nullptr, nullptr};
  bool graphs_ok = true;   // cleared if capture or instantiation fails: plain launches then
  int64_t plain_steps = 0; // steps launched one kernel at a time (the launchers set their
                           // kernel attributes on first use, outside any capture)
};

// Mark the domain's error word as copied to the host after work enqueued on `stream`
// (defined in lbm_api.cu); lbm_step / lbm_synchronize report it.
lbm_status lbm_internal_enqueue_flag_copy(lbm_domain* h, cudaStream_t stream);
