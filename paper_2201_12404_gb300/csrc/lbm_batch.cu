// Host side of the batched persistent stepping (lbm_batch_* in include/lbm.h):
// work lists, cooperative launch, CUDA-graph capture, and the tile-shape tuner.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <cstring>
#include <fstream>
#include <map>
#include <sstream>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_batch.h"
#include "lbm_handle.h"

using lbm::BatchArgs;
using lbm::BatchItem;
using lbm::BatchVariant;
using lbm::DevDomain;

struct lbm_batch {
  std::vector<lbm_domain*> doms;
  int precision = LBM_FP32;
  cudaStream_t stream = nullptr;
  const BatchVariant* variants = nullptr;
  int nvariants = 0;
  int chosen = 0;
  // device buffers
  DevDomain* d_jobs = nullptr;
  int* d_parity = nullptr;
  BatchItem* d_items = nullptr;  // the tiles of every job's interior
  unsigned int* d_sync = nullptr;  // [0] arrivals, [1] generation, [2] error word
  int n_k2 = 0, grid = 0;
  std::map<int64_t, cudaGraphExec_t> graphs;
  bool use_graph = true;
  unsigned int poll_limit = lbm::kBarrierPollsDefault;
  int skip_arrival = 0;
  bool poisoned = false;
  int64_t launches = 0;
  std::string err;
};

static thread_local std::string g_batch_error = "no error";

namespace {

lbm_status bfail(lbm_batch* b, lbm_status st, const std::string& msg) {
  b->err = msg;
  if (st != LBM_ERR_INVALID_ARG) b->poisoned = true;
  return st;
}

#define B_CUDA(b, call)                                                                                 \
  do {                                                                                                  \
    cudaError_t e_ = (call);                                                                            \
    if (e_ != cudaSuccess)                                                                              \
      return bfail((b), e_ == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,                   \
                   std::string(#call) + ": " + cudaGetErrorString(e_));                                 \
  } while (0)

// Work list of a tile shape: the tiles of every job's interior (each pass walks
// them; pass 1 writes the ghost images of its nodes itself).
void build_items(const std::vector<lbm_domain*>& doms, int bx, int by, std::vector<BatchItem>& k2) {
  k2.clear();
  for (int j = 0; j < (int)doms.size(); ++j) {
    const DevDomain& d = doms[j]->dev;
    for (int ty = 0; ty < (d.ny + by - 1) / by; ++ty)
      for (int tx = 0; tx < (d.nx + bx - 1) / bx; ++tx) k2.push_back({j, tx, ty});
  }
}

// Upload the work lists of variant v and size the cooperative grid.
lbm_status select_variant(lbm_batch* b, int v) {
  const BatchVariant& var = b->variants[v];
  std::vector<BatchItem> k2;
  build_items(b->doms, var.bx, var.by, k2);
  if (b->d_items) { cudaFree(b->d_items); b->d_items = nullptr; }
  B_CUDA(b, cudaMalloc(&b->d_items, k2.size() * sizeof(BatchItem)));
  B_CUDA(b, cudaMemcpy(b->d_items, k2.data(), k2.size() * sizeof(BatchItem), cudaMemcpyHostToDevice));
  b->n_k2 = (int)k2.size();
  int dev = 0, sms = 0, per_sm = 0;
  B_CUDA(b, cudaGetDevice(&dev));
  B_CUDA(b, cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  B_CUDA(b, cudaFuncSetAttribute(var.kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)var.dyn_smem));
  B_CUDA(b, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, var.kernel, var.bx * var.by, var.dyn_smem));
  if (per_sm < 1) return bfail(b, LBM_ERR_CUDA, "the batch kernel cannot be resident on an SM");
  b->grid = std::max(1, std::min(per_sm * sms, b->n_k2));
  b->chosen = v;
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
  return LBM_OK;
}

BatchArgs make_args(lbm_batch* b, const DevDomain* jobs, int* parity, int nsteps) {
  BatchArgs a;
  a.jobs = jobs;
  a.parity = parity;
  a.njobs = (int)b->doms.size();
  a.k2 = b->d_items;
  a.n_k2 = b->n_k2;
  a.barrier = b->d_sync;
  a.error = b->d_sync + 2;
  a.nsteps = nsteps;
  a.poll_limit = b->poll_limit;
  a.skip_arrival = b->skip_arrival;
  return a;
}

cudaError_t launch(lbm_batch* b, BatchArgs a, cudaStream_t s) {
  const BatchVariant& var = b->variants[b->chosen];
  void* params[] = {&a};
  return cudaLaunchCooperativeKernel(var.kernel, dim3(b->grid), dim3(var.bx, var.by), params, var.dyn_smem, s);
}

}  // namespace

extern "C" {

lbm_status lbm_batch_create(const lbm_handle* domains, int32_t count, lbm_batch_handle* out) {
  if (!out) { g_batch_error = "out is NULL"; return LBM_ERR_INVALID_ARG; }
  *out = nullptr;
  if (!domains || count < 1) { g_batch_error = "need at least one domain"; return LBM_ERR_INVALID_ARG; }
  for (int j = 0; j < count; ++j) {
    lbm_domain* h = domains[j];
    if (!h) { g_batch_error = "NULL domain"; return LBM_ERR_INVALID_ARG; }
    if (h->poisoned) { g_batch_error = "a domain is in an error state"; return LBM_ERR_STATE; }
    if (h->p.lattice != LBM_D2Q9) { g_batch_error = "batches hold D2Q9 domains"; return LBM_ERR_INVALID_ARG; }
    if (h->p.precision != domains[0]->p.precision) { g_batch_error = "all domains of a batch share one precision"; return LBM_ERR_INVALID_ARG; }
    for (int k = 0; k < j; ++k)
      if (domains[k] == h) { g_batch_error = "a domain appears twice"; return LBM_ERR_INVALID_ARG; }
  }
  lbm_batch* b = new lbm_batch();
  b->doms.assign(domains, domains + count);
  b->precision = domains[0]->p.precision;
  b->stream = domains[0]->stream;
  b->nvariants = lbm::batch_variants(b->precision, &b->variants);
  auto bail = [&](lbm_status st) {
    g_batch_error = b->err;
    lbm_batch_destroy(b);
    return st;
  };
  for (lbm_domain* h : b->doms)
    if (cudaStreamSynchronize(h->stream) != cudaSuccess) { b->err = "cudaStreamSynchronize failed"; return bail(LBM_ERR_CUDA); }
  std::vector<DevDomain> jobs(count);
  std::vector<int> parity(count);
  for (int j = 0; j < count; ++j) {
    jobs[j] = b->doms[j]->dev;
    jobs[j].gamma_out = nullptr;
    parity[j] = b->doms[j]->parity;
  }
  lbm_status st;
  if (cudaMalloc(&b->d_jobs, count * sizeof(DevDomain)) != cudaSuccess ||
      cudaMalloc(&b->d_parity, count * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&b->d_sync, 4 * sizeof(unsigned int)) != cudaSuccess) {
    b->err = "cudaMalloc failed";
    return bail(LBM_ERR_OOM);
  }
  if (cudaMemcpy(b->d_jobs, jobs.data(), count * sizeof(DevDomain), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_parity, parity.data(), count * sizeof(int), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemset(b->d_sync, 0, 4 * sizeof(unsigned int)) != cudaSuccess) {
    b->err = "cudaMemcpy failed";
    return bail(LBM_ERR_CUDA);
  }
  if ((st = select_variant(b, 0)) != LBM_OK) return bail(st);
  *out = b;
  return LBM_OK;
}

lbm_status lbm_batch_destroy(lbm_batch_handle b) {
  if (!b) return LBM_OK;
  if (b->stream) cudaStreamSynchronize(b->stream);
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  if (b->d_jobs) cudaFree(b->d_jobs);
  if (b->d_parity) cudaFree(b->d_parity);
  if (b->d_items) cudaFree(b->d_items);
  if (b->d_sync) cudaFree(b->d_sync);
  delete b;
  return LBM_OK;
}

lbm_status lbm_batch_step(lbm_batch_handle b, int64_t nsteps) {
  if (!b) return LBM_ERR_INVALID_ARG;
  if (b->poisoned) return LBM_ERR_STATE;
  if (nsteps < 0 || nsteps > (int64_t)1 << 30) return bfail(b, LBM_ERR_INVALID_ARG, "nsteps out of range");
  if (nsteps == 0) return LBM_OK;
  for (lbm_domain* h : b->doms)
    if (h->poisoned) return bfail(b, LBM_ERR_STATE, "a domain of the batch is in an error state");
  BatchArgs a = make_args(b, b->d_jobs, b->d_parity, (int)nsteps);
  bool launched = false;
  if (b->use_graph) {
    auto it = b->graphs.find(nsteps);
    if (it == b->graphs.end()) {
      cudaGraph_t g = nullptr;
      cudaGraphExec_t ge = nullptr;
      bool ok = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
      if (ok) {
        const cudaError_t le = launch(b, a, b->stream);
        const cudaError_t ce = cudaStreamEndCapture(b->stream, &g);
        ok = le == cudaSuccess && ce == cudaSuccess && g &&
             cudaGraphInstantiate(&ge, g, 0) == cudaSuccess;
        if (g) cudaGraphDestroy(g);
      }
      cudaGetLastError();
      if (ok) {
        if (b->graphs.size() >= 8) {
          cudaGraphExecDestroy(b->graphs.begin()->second);
          b->graphs.erase(b->graphs.begin());
        }
        it = b->graphs.emplace(nsteps, ge).first;
      } else {
        b->use_graph = false;  // capture of the cooperative launch refused: launch directly from now on
      }
    }
    if (b->use_graph) {
      B_CUDA(b, cudaGraphLaunch(it->second, b->stream));
      launched = true;
    }
  }
  if (!launched) B_CUDA(b, launch(b, a, b->stream));
  b->launches += 1;
  for (lbm_domain* h : b->doms) {
    h->parity ^= (int)(nsteps & 1);
    h->steps += nsteps;
    h->launches += 1;
    lbm_internal_enqueue_flag_copy(h, b->stream);
  }
  return LBM_OK;
}

lbm_status lbm_batch_synchronize(lbm_batch_handle b) {
  if (!b) return LBM_ERR_INVALID_ARG;
  if (b->poisoned) return LBM_ERR_STATE;
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  unsigned int e = 0;
  B_CUDA(b, cudaMemcpy(&e, b->d_sync + 2, sizeof(e), cudaMemcpyDeviceToHost));
  if (e & 2u) return bfail(b, LBM_ERR_TIMEOUT, "a bounded grid-barrier wait of the batch kernel gave up");
  lbm_status worst = LBM_OK;
  for (lbm_domain* h : b->doms) {
    const lbm_status st = lbm_synchronize(h);
    if (st != LBM_OK && worst == LBM_OK) worst = st;
  }
  return worst;
}

lbm_status lbm_batch_set_wait(lbm_batch_handle b, uint32_t poll_limit, int32_t skip_arrival) {
  if (!b) return LBM_ERR_INVALID_ARG;
  if (b->poisoned) return LBM_ERR_STATE;
  b->poll_limit = poll_limit ? poll_limit : lbm::kBarrierPollsDefault;
  b->skip_arrival = skip_arrival ? 1 : 0;
  // the captured graphs hold the previous arguments
  for (auto& kv : b->graphs) cudaGraphExecDestroy(kv.second);
  b->graphs.clear();
  return LBM_OK;
}

lbm_status lbm_batch_info(lbm_batch_handle b, int32_t* block_x, int32_t* block_y, int32_t* grid_blocks,
                          int32_t* graph_captured) {
  if (!b) return LBM_ERR_INVALID_ARG;
  if (block_x) *block_x = b->variants[b->chosen].bx;
  if (block_y) *block_y = b->variants[b->chosen].by;
  if (grid_blocks) *grid_blocks = b->grid;
  if (graph_captured) *graph_captured = b->use_graph ? 1 : 0;
  return LBM_OK;
}

lbm_status lbm_batch_tune(lbm_batch_handle b, int32_t trial_steps, const char* cache_path) {
  if (!b) return LBM_ERR_INVALID_ARG;
  if (b->poisoned) return LBM_ERR_STATE;
  if (trial_steps < 1) return bfail(b, LBM_ERR_INVALID_ARG, "trial_steps must be >= 1");
  // size class: total nodes rounded to a power of two, job count, precision
  long long nodes = 0;
  for (lbm_domain* h : b->doms) nodes += h->dev.N;
  int lg = 0;
  while ((1ll << (lg + 1)) <= nodes) ++lg;
  std::ostringstream key;
  key << "d2q9_p" << b->precision << "_n2^" << lg << "_j" << b->doms.size();
  // cached choice
  if (cache_path) {
    std::ifstream in(cache_path);
    std::string line;
    while (std::getline(in, line)) {
      char k[128];
      int bx = 0, by = 0;
      if (std::sscanf(line.c_str(), " {\"key\": \"%127[^\"]\", \"block\": [%d, %d]", k, &bx, &by) == 3 && key.str() == k) {
        for (int v = 0; v < b->nvariants; ++v)
          if (b->variants[v].bx == bx && b->variants[v].by == by) return select_variant(b, v);
      }
    }
  }
  // time every variant on clones of the jobs (the jobs themselves are not advanced)
  B_CUDA(b, cudaStreamSynchronize(b->stream));
  const int count = (int)b->doms.size();
  std::vector<DevDomain> clones(count);
  std::vector<void*> owned;
  auto free_all = [&]() { for (void* p : owned) cudaFree(p); owned.clear(); };
  for (int j = 0; j < count; ++j) {
    const lbm_domain* h = b->doms[j];
    DevDomain c = h->dev;
    const size_t fb = (size_t)h->ops->Q * h->dev.N * h->ops->pop_bytes;
    const size_t ab = (size_t)(2 + 2 * h->ops->D) * h->dev.PN * h->ops->aux_bytes;
    void *f = nullptr, *aux = nullptr, *fl = nullptr, *rw = nullptr;
    if (cudaMalloc(&f, fb) != cudaSuccess || cudaMalloc(&aux, ab) != cudaSuccess || cudaMalloc(&fl, 64) != cudaSuccess) {
      if (f) cudaFree(f);
      if (aux) cudaFree(aux);
      free_all();
      return bfail(b, LBM_ERR_OOM, "no memory for the tuning clones");
    }
    owned.push_back(f); owned.push_back(aux); owned.push_back(fl);
    cudaMemcpyAsync(f, h->dev.f, fb, cudaMemcpyDeviceToDevice, b->stream);
    cudaMemsetAsync(aux, 0, ab, b->stream);
    cudaMemsetAsync(fl, 0, 64, b->stream);
    c.f = f;
    c.aux = aux;
    c.flags = (unsigned int*)fl;
    c.guards = (unsigned long long*)((char*)fl + 8);
    c.gamma_out = nullptr;
    if (h->dev.rho_w[0]) {
      if (cudaMalloc(&rw, 2 * (size_t)h->dev.N * sizeof(float)) != cudaSuccess) { free_all(); return bfail(b, LBM_ERR_OOM, "no memory for the tuning clones"); }
      owned.push_back(rw);
      cudaMemcpyAsync(rw, h->dev.rho_w[0], 2 * (size_t)h->dev.N * sizeof(float), cudaMemcpyDeviceToDevice, b->stream);
      c.rho_w[0] = (float*)rw;
      c.rho_w[1] = (float*)rw + h->dev.N;
    }
    clones[j] = c;
  }
  DevDomain* d_clones = nullptr;
  int* d_par = nullptr;
  unsigned int* d_sync2 = nullptr;
  if (cudaMalloc(&d_clones, count * sizeof(DevDomain)) != cudaSuccess || cudaMalloc(&d_par, count * sizeof(int)) != cudaSuccess ||
      cudaMalloc(&d_sync2, 4 * sizeof(unsigned int)) != cudaSuccess) {
    if (d_clones) cudaFree(d_clones);
    if (d_par) cudaFree(d_par);
    free_all();
    return bfail(b, LBM_ERR_OOM, "no memory for the tuning clones");
  }
  owned.push_back(d_clones); owned.push_back(d_par); owned.push_back(d_sync2);
  B_CUDA(b, cudaMemcpyAsync(d_clones, clones.data(), count * sizeof(DevDomain), cudaMemcpyHostToDevice, b->stream));
  B_CUDA(b, cudaMemcpyAsync(d_par, b->d_parity, count * sizeof(int), cudaMemcpyDeviceToDevice, b->stream));
  B_CUDA(b, cudaMemsetAsync(d_sync2, 0, 4 * sizeof(unsigned int), b->stream));
  cudaEvent_t e0, e1;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  int best = b->chosen;
  float best_ms = 1e30f;
  const int keep = b->chosen;
  for (int v = 0; v < b->nvariants; ++v) {
    lbm_status st = select_variant(b, v);
    if (st != LBM_OK) { free_all(); return st; }
    BatchArgs a = make_args(b, d_clones, d_par, 1);
    a.barrier = d_sync2;
    a.error = d_sync2 + 2;
    launch(b, a, b->stream);  // warm-up step
    a.nsteps = trial_steps;
    cudaEventRecord(e0, b->stream);
    launch(b, a, b->stream);
    cudaEventRecord(e1, b->stream);
    if (cudaEventSynchronize(e1) != cudaSuccess) { free_all(); return bfail(b, LBM_ERR_CUDA, "tuning launch failed"); }
    float ms = 0;
    cudaEventElapsedTime(&ms, e0, e1);
    if (ms < best_ms) { best_ms = ms; best = v; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamSynchronize(b->stream);
  free_all();
  (void)keep;
  lbm_status st = select_variant(b, best);
  if (st != LBM_OK) return st;
  if (cache_path) {
    std::ofstream outf(cache_path, std::ios::app);
    // one JSON object per line
    outf << "{\"key\": \"" << key.str() << "\", \"block\": [" << b->variants[best].bx << ", " << b->variants[best].by
         << "], \"ms_per_step\": " << best_ms / trial_steps << "}\n";
  }
  return LBM_OK;
}

const char* lbm_batch_last_error(lbm_batch_handle b) {
  if (!b) return g_batch_error.c_str();
  return b->err.empty() ? "no error" : b->err.c_str();
}

}  // extern "C"
