// Host side of the C ABI declared in include/lbm.h: parameter validation,
// device memory, the step loop, field I/O, diagnostics and timing.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_handle.h"
#include "lbm_ops.h"
#include "lbm_phys.h"

using lbm::DevDomain;
using lbm::Ops;
using lbm::Phys;

static thread_local std::string g_create_error = "no error";

namespace {

#ifdef LBM_BOUNDS_CHECK
const char* kVersion =
    "liblbm: entropic MRT two-phase LBM, D2Q9/D3Q27, FP64/FP32/FP16-deviation, A-A streaming, sm_103a, bounds-checked";
#else
const char* kVersion = "liblbm: entropic MRT two-phase LBM, D2Q9/D3Q27, FP64/FP32/FP16-deviation, A-A streaming, sm_103a";
#endif

using lbm::EosCoeffs;
using lbm::eos_coeffs;
using lbm::pr_p;

std::string validate(const lbm_params* p) {
  if (!p) return "params is NULL";
  if (p->lattice != LBM_D2Q9 && p->lattice != LBM_D3Q27) return "lattice must be LBM_D2Q9 or LBM_D3Q27";
  if (p->precision != LBM_FP64 && p->precision != LBM_FP32 && p->precision != LBM_FP16DEV)
    return "precision must be LBM_FP64, LBM_FP32 or LBM_FP16DEV";
  const bool d3 = p->lattice == LBM_D3Q27;
  if (p->nx < 5 || p->ny < 5) return "nx and ny must be >= 5 (stencil radius 2)";
  if (d3 && p->nz < 5) return "nz must be >= 5 for D3Q27";
  if (!d3 && p->nz != 1) return "nz must be 1 for D2Q9";
  if ((double)p->nx * p->ny * p->nz > 4.0e9) return "domain larger than 4e9 nodes";
  if (!(p->a > 0) || !(p->b > 0) || !(p->R > 0)) return "EOS a, b, R must be > 0";
  if (!(p->T_over_Tc > 0) || !(p->T_over_Tc < 1.5)) return "T_over_Tc must lie in (0, 1.5)";
  if (!std::isfinite(p->acentric)) return "acentric factor must be finite";
  if (!(p->kappa >= 0) || !std::isfinite(p->kappa)) return "kappa must be >= 0";
  if (!(p->nu_liquid > 0) || !(p->nu_vapour > 0)) return "viscosities must be > 0";
  if (!(p->rho_vapour > 0) || !(p->rho_liquid > p->rho_vapour)) return "need rho_liquid > rho_vapour > 0";
  for (int k = 0; k < 3; ++k) if (!std::isfinite(p->body_force[k])) return "body_force must be finite";
  for (int k = 0; k < 6; ++k)
    if (p->bc[k] != LBM_BC_PERIODIC && p->bc[k] != LBM_BC_BOUNCEBACK) return "bc entries must be 0 or 1";
  for (int a = 0; a < (d3 ? 3 : 2); ++a)
    if ((p->bc[2 * a] == LBM_BC_PERIODIC) != (p->bc[2 * a + 1] == LBM_BC_PERIODIC))
      return "periodic faces must come in pairs";
  if (!d3 && (p->body_force[2] != 0.0)) return "body_force[2] must be 0 in 2-D";
  if (p->gamma_mode != LBM_GAMMA_ENTROPIC && p->gamma_mode != LBM_GAMMA_FIXED) return "gamma_mode must be 0 or 1";
  if (p->gamma_mode == LBM_GAMMA_FIXED && !std::isfinite(p->gamma_value)) return "gamma_value must be finite";
  if (p->eos_fp64 < 0 || p->eos_fp64 > 2) return "eos_fp64 must be 0, 1 or 2";
  if ((p->dev_alloc == nullptr) != (p->dev_free == nullptr)) return "set both dev_alloc and dev_free, or neither";
  return "";
}

struct Sizes { int D, Q; long long N, PN; int px, py, pz; size_t f_bytes, aux_bytes, gamma_bytes, rho_w_bytes; };

Sizes sizes_of(const lbm_params& p, const Ops* ops) {
  Sizes s;
  s.D = p.lattice == LBM_D3Q27 ? 3 : 2;
  s.Q = s.D == 3 ? 27 : 9;
  s.N = (long long)p.nx * p.ny * (s.D == 3 ? p.nz : 1);
  s.px = lbm::padded_x(p.nx);
  s.py = p.ny + 4;
  s.pz = s.D == 3 ? p.nz + 4 : 1;
  s.PN = (long long)s.px * s.py * s.pz;
  s.f_bytes = (size_t)s.Q * s.N * ops->pop_bytes;
  s.aux_bytes = (size_t)lbm::aux_fields_per_node(s.D) * s.PN * ops->aux_bytes;
  s.gamma_bytes = (size_t)s.N * sizeof(float);
  s.rho_w_bytes = p.precision == LBM_FP16DEV ? 2 * (size_t)s.N * sizeof(float) : 0;
  return s;
}

const Ops* ops_for(const lbm_params& p) {
  if (p.lattice == LBM_D2Q9)
    return p.precision == LBM_FP64 ? &lbm::ops_d2q9_fp64
                                   : (p.precision == LBM_FP16DEV ? &lbm::ops_d2q9_fp16dev : &lbm::ops_d2q9_fp32);
  return p.precision == LBM_FP64 ? &lbm::ops_d3q27_fp64
                                 : (p.precision == LBM_FP16DEV ? &lbm::ops_d3q27_fp16dev : &lbm::ops_d3q27_fp32);
}

lbm_status fail(lbm_domain* h, lbm_status st, const std::string& msg) {
  h->err = msg;
  if (st != LBM_ERR_INVALID_ARG) h->poisoned = true;
  return st;
}

lbm_status cuda_fail(lbm_domain* h, cudaError_t e, const char* where) {
  return fail(h, e == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA,
              std::string(where) + ": " + cudaGetErrorString(e));
}

#define LBM_CUDA(h, call)                                     \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((h), e_, #call);  \
  } while (0)

// Scratch buffers of the host-buffer calls come from a pool of the library's own
// that keeps up to kScratchKeep bytes across synchronisations.  The default pool
// hands its memory back at every synchronisation, and mapping a few GB again on
// the next call costs up to a fifth of a second.
constexpr uint64_t kScratchKeep = 4ull << 30;

cudaMemPool_t scratch_pool() {
  static std::mutex mu;
  static cudaMemPool_t pools[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(mu);
  if (!pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    uint64_t keep = kScratchKeep;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    pools[dev] = pool;
  }
  return pools[dev];
}

// Stream-ordered scratch allocation on h's stream (freed with cudaFreeAsync).
template <typename T>
cudaError_t scratch_alloc(lbm_domain* h, T** p, size_t bytes) {
  cudaMemPool_t pool = scratch_pool();
  if (!pool) return cudaMallocAsync((void**)p, bytes, h->stream);
  return cudaMallocFromPoolAsync((void**)p, bytes, pool, h->stream);
}

// Device memory a domain keeps for its lifetime: the caller's allocator when
// lbm_params sets one, cudaMalloc otherwise.
cudaError_t keep_alloc(const lbm_params& p, void** ptr, size_t bytes) {
  if (!p.dev_alloc) return cudaMalloc(ptr, bytes);
  *ptr = p.dev_alloc(bytes, p.alloc_ctx);
  if (!*ptr) return cudaErrorMemoryAllocation;
  if ((uintptr_t)*ptr % 256 != 0) {
    p.dev_free(*ptr, p.alloc_ctx);
    *ptr = nullptr;
    return cudaErrorInvalidValue;
  }
  return cudaSuccess;
}

void keep_free(const lbm_params& p, void* ptr) {
  if (!ptr) return;
  if (p.dev_alloc) p.dev_free(ptr, p.alloc_ctx);
  else cudaFree(ptr);
}

#define LBM_LIVE(h)                                                               \
  do {                                                                            \
    if (!(h)) return LBM_ERR_INVALID_ARG;                                         \
    if ((h)->poisoned) return LBM_ERR_STATE;                                      \
  } while (0)

cudaEvent_t take_event(lbm_domain* h) {
  if (!h->ev_pool.empty()) {
    cudaEvent_t e = h->ev_pool.back();
    h->ev_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Fold finished timing marks into the sums (synchronous).
lbm_status drain_marks(lbm_domain* h) {
  for (auto& m : h->marks) {
    float t = 0;
    LBM_CUDA(h, cudaEventSynchronize(m.b));
    LBM_CUDA(h, cudaEventElapsedTime(&t, m.a, m.b));
    h->ms[m.kind] += t;
    h->cnt[m.kind] += 1;
    h->ev_pool.push_back(m.a);
    h->ev_pool.push_back(m.b);
  }
  h->marks.clear();
  return LBM_OK;
}

// Status for the device error word: bit 0 instability, bit 1 a bounded wait gave up,
// bit 2 an out-of-range index caught by a bounds-checked build.
lbm_status flags_status(lbm_domain* h, unsigned int flags) {
  if (flags & 4u) return fail(h, LBM_ERR_BOUNDS, "a kernel computed an index outside its buffer (bounds-checked build)");
  if (flags & 2u) return fail(h, LBM_ERR_TIMEOUT, "a bounded device-side wait for a TMA tile gave up");
  if (flags & 1u) return fail(h, LBM_ERR_UNSTABLE, "non-finite or non-positive density in the domain");
  return LBM_OK;
}

// Check the error flags copied by earlier steps without waiting for the GPU.
lbm_status poll_flags(lbm_domain* h, bool wait) {
  if (!h->flags_pending) return LBM_OK;
  if (wait) {
    LBM_CUDA(h, cudaEventSynchronize(h->flags_ev));
  } else {
    cudaError_t q = cudaEventQuery(h->flags_ev);
    if (q == cudaErrorNotReady) return LBM_OK;
    if (q != cudaSuccess) return cuda_fail(h, q, "cudaEventQuery");
  }
  h->flags_pending = false;
  return flags_status(h, *h->h_flags);
}

lbm_status enqueue_flag_copy(lbm_domain* h, cudaStream_t stream) {
  LBM_CUDA(h, cudaMemcpyAsync(h->h_flags, h->dev.flags, sizeof(unsigned int), cudaMemcpyDeviceToHost, stream));
  LBM_CUDA(h, cudaEventRecord(h->flags_ev, stream));
  h->flags_pending = true;
  return LBM_OK;
}

lbm_status launch_k(lbm_domain* h, int kind) {
  cudaEvent_t a = nullptr, b = nullptr;
  if (h->timing) {
    a = take_event(h);
    b = take_event(h);
    LBM_CUDA(h, cudaEventRecord(a, h->stream));
  }
  if (kind == 0) {
    // pass 1 and the q planes it feeds, timed together
    h->ops->moments_eos(h->dev, h->parity, h->stream);
    h->ops->qflux(h->dev, h->maps, h->stream);
    h->launches += 1;
  } else {
    h->ops->collide_stream(h->dev, h->maps, h->parity, h->stream);
  }
  h->launches += 1;
  LBM_CUDA(h, cudaGetLastError());
  if (h->timing) {
    LBM_CUDA(h, cudaEventRecord(b, h->stream));
    h->marks.push_back({kind, a, b});
  }
  return LBM_OK;
}

// Launch the graph of two steps from the current parity, capturing it first if
// there is none for this parity and gamma record.  *replayed is false (and nothing
// was enqueued) when capture is not possible on this stream; the domain then keeps
// to plain launches.
lbm_status launch_pair_graph(lbm_domain* h, bool* replayed) {
  *replayed = false;
  const int p = h->parity;
  if (!h->step_graph[p] || h->step_graph_gamma[p] != h->dev.gamma_out) {
    if (h->step_graph[p]) {
      cudaGraphExecDestroy(h->step_graph[p]);
      h->step_graph[p] = nullptr;
    }
    if (cudaStreamBeginCapture(h->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      cudaGetLastError();
      h->graphs_ok = false;
      return LBM_OK;
    }
    for (int k = 0; k < 2; ++k) {
      const int par = p ^ k;
      h->ops->moments_eos(h->dev, par, h->stream);
      h->ops->qflux(h->dev, h->maps, h->stream);
      h->ops->collide_stream(h->dev, h->maps, par, h->stream);
    }
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamEndCapture(h->stream, &g);
    cudaGraphExec_t exec = nullptr;
    if (e == cudaSuccess && g) e = cudaGraphInstantiate(&exec, g, 0);
    if (g) cudaGraphDestroy(g);
    if (e != cudaSuccess || !exec) {
      cudaGetLastError();  // the failed capture left nothing on the stream
      h->graphs_ok = false;
      return LBM_OK;
    }
    h->step_graph[p] = exec;
    h->step_graph_gamma[p] = (float*)h->dev.gamma_out;
  }
  LBM_CUDA(h, cudaGraphLaunch(h->step_graph[p], h->stream));
  h->launches += 6;
  *replayed = true;
  return LBM_OK;
}

// Run pass 1 for the current state (refreshes the auxiliary fields).
lbm_status refresh_aux(lbm_domain* h) {
  h->ops->moments_eos(h->dev, h->parity, h->stream);
  h->launches += 1;
  LBM_CUDA(h, cudaGetLastError());
  return LBM_OK;
}

// ---- Maxwell construction (host) ----
// In density: int_{rv}^{rl} (Psat - P)/rho^2 drho = [ -Psat/rho - G(rho) ]_{rv}^{rl}, with the
// antiderivative of P/rho^2 for Peng-Robinson
//   G(rho) = RT ln(rho/(1 - b rho)) + aalpha/(2 sqrt2 b) ln|(rho - r1)/(rho - r2)|,
// r1,2 = (1 +- sqrt2)/b the roots of 1 + 2 b rho - b^2 rho^2.
double antideriv(const EosCoeffs& e, double rho) {
  const double s2 = std::sqrt(2.0);
  const double r1 = (1.0 + s2) / e.b, r2 = (1.0 - s2) / e.b;
  return e.RT * std::log(rho / (1.0 - e.b * rho)) + e.aalpha / (2.0 * s2 * e.b) * std::log(std::fabs((rho - r1) / (rho - r2)));
}

double dpdrho(const EosCoeffs& e, double rho) {
  const double h = 1e-7 * std::max(rho, 1e-6);
  return (pr_p(e, rho + h) - pr_p(e, rho - h)) / (2 * h);
}

// root of P(rho) = target on [lo, hi] where P - target changes sign
double bisect_p(const EosCoeffs& e, double target, double lo, double hi) {
  double flo = pr_p(e, lo) - target;
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double fm = pr_p(e, mid) - target;
    if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
    if (hi - lo <= 1e-15 * hi) break;
  }
  return 0.5 * (lo + hi);
}

// Pass 1 for the current state, then a block-partial maximum (field 4 of the
// [block][5] layout, at most N blocks) reduced by diag_final_kernel; *out = the maximum.
template <typename Partial>
lbm_status reduce_max(lbm_handle h, Partial partial, double* out) {
  lbm_status st = refresh_aux(h);
  if (st != LBM_OK) return st;
  const long long nblk = (h->dev.N + 255) / 256;
  double* buf = nullptr;
  LBM_CUDA(h, scratch_alloc(h, &buf, (size_t)(nblk * 5 + 5) * sizeof(double)));
  const int nb = partial(buf);
  lbm::launch_diag_final(buf, nb, buf + nblk * 5, h->stream);
  h->launches += 2;
  LBM_CUDA(h, cudaGetLastError());
  double res[5];
  LBM_CUDA(h, cudaMemcpyAsync(res, buf + nblk * 5, sizeof(res), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaFreeAsync(buf, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  *out = res[4];
  return LBM_OK;
}

}  // namespace

lbm_status lbm_internal_enqueue_flag_copy(lbm_domain* h, cudaStream_t stream) {
  if (h->flags_pending) return LBM_OK;
  return enqueue_flag_copy(h, stream);
}

namespace {
lbm_status init_from_device_fields(lbm_handle h, double* buf);
}  // namespace

extern "C" {

const char* lbm_version(void) { return kVersion; }

lbm_status lbm_default_params(lbm_params* p) {
  if (!p) return LBM_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->lattice = LBM_D2Q9;
  p->precision = LBM_FP32;
  p->nx = 64; p->ny = 64; p->nz = 1;
  p->a = 0.003; p->b = 0.095; p->R = 1.0; p->T_over_Tc = 0.8; p->acentric = 0.344;
  p->kappa = 0.0;
  p->nu_liquid = 0.1; p->nu_vapour = 0.1; p->rho_liquid = 1.0; p->rho_vapour = 0.5;
  p->gamma_mode = LBM_GAMMA_ENTROPIC; p->gamma_value = 2.0;
  p->eos_fp64 = 1;
  p->stream = nullptr;
  return LBM_OK;
}

size_t lbm_footprint_bytes(const lbm_params* p) {
  if (!validate(p).empty()) return 0;
  Sizes s = sizes_of(*p, ops_for(*p));
  return s.f_bytes + s.aux_bytes + s.rho_w_bytes + sizeof(unsigned int) + 2 * sizeof(unsigned long long);
}

lbm_status lbm_psi_sign_changes(const lbm_params* p, double changes[3], int* n, double* s0) {
  if (!p || !changes || !n || !s0) { g_create_error = "NULL argument"; return LBM_ERR_INVALID_ARG; }
  if (!(p->a > 0) || !(p->b > 0) || !(p->R > 0) || !(p->T_over_Tc > 0)) {
    g_create_error = "the sign changes need a, b, R, T/Tc > 0";
    return LBM_ERR_INVALID_ARG;
  }
  lbm::psi_sign_changes(eos_coeffs(*p), changes, s0);
  *n = 0;
  for (int k = 0; k < 3; ++k) *n += std::isfinite(changes[k]) ? 1 : 0;
  return LBM_OK;
}

lbm_status lbm_coexistence(const lbm_params* p, double* rho_vapour, double* rho_liquid, double* p_sat) {
  if (!p || !rho_vapour || !rho_liquid) { g_create_error = "NULL argument"; return LBM_ERR_INVALID_ARG; }
  if (!(p->a > 0) || !(p->b > 0) || !(p->R > 0) || !(p->T_over_Tc > 0) || !(p->T_over_Tc < 1)) {
    g_create_error = "coexistence needs a, b, R > 0 and 0 < T/Tc < 1";
    return LBM_ERR_INVALID_ARG;
  }
  const EosCoeffs e = eos_coeffs(*p);
  // spinodals: the local maximum (vapour side) and minimum (liquid side) of P(rho) on (0, 1/b)
  const double rmax = 1.0 / e.b;
  const int M = 200000;
  double r_spv = -1, r_spl = -1;
  double prev = dpdrho(e, rmax * 1e-6);
  for (int k = 1; k <= M; ++k) {
    const double r = rmax * (1e-6 + (0.999 - 1e-6) * k / M);
    const double d = dpdrho(e, r);
    if (r_spv < 0 && prev > 0 && d <= 0) r_spv = r;
    else if (r_spv > 0 && prev < 0 && d >= 0) { r_spl = r; break; }
    prev = d;
  }
  if (r_spv < 0 || r_spl < 0) { g_create_error = "no two-phase region at this temperature"; return LBM_ERR_INVALID_ARG; }
  const double p_hi = pr_p(e, r_spv), p_lo = std::max(pr_p(e, r_spl), 1e-300);
  double rv = 0, rl = 0;
  auto area = [&](double Ps) {
    rv = bisect_p(e, Ps, 0.0, r_spv);
    rl = bisect_p(e, Ps, r_spl, rmax * 0.999999);
    return (-Ps / rl - antideriv(e, rl)) - (-Ps / rv - antideriv(e, rv));
  };
  double lo = p_lo + 1e-12 * (p_hi - p_lo), hi = p_hi - 1e-12 * (p_hi - p_lo);
  double flo = area(lo);
  for (int it = 0; it < 200; ++it) {
    const double mid = 0.5 * (lo + hi);
    const double fm = area(mid);
    if ((fm < 0) == (flo < 0)) { lo = mid; flo = fm; } else { hi = mid; }
    if (hi - lo <= 1e-16 * hi) break;
  }
  const double Ps = 0.5 * (lo + hi);
  area(Ps);
  *rho_vapour = rv;
  *rho_liquid = rl;
  if (p_sat) *p_sat = Ps;
  return LBM_OK;
}

lbm_status lbm_create_domain(const lbm_params* p, lbm_handle* out) {
  if (!out) { g_create_error = "out is NULL"; return LBM_ERR_INVALID_ARG; }
  *out = nullptr;
  const std::string why = validate(p);
  if (!why.empty()) { g_create_error = why; return LBM_ERR_INVALID_ARG; }
  {
    // refuse a domain that cannot fit before allocating any of it
    size_t free_b = 0, total_b = 0;
    const cudaError_t e = cudaMemGetInfo(&free_b, &total_b);
    if (e != cudaSuccess) { g_create_error = std::string("cudaMemGetInfo: ") + cudaGetErrorString(e); return LBM_ERR_CUDA; }
    const size_t need = lbm_footprint_bytes(p);
    if (need > free_b) {
      g_create_error = "domain needs " + std::to_string(need) + " bytes of device memory, " + std::to_string(free_b) +
                       " are free";
      return LBM_ERR_OOM;
    }
  }

  lbm_domain* h = new lbm_domain();
  h->p = *p;
  h->ops = ops_for(*p);
  const Sizes s = sizes_of(*p, h->ops);
  DevDomain& d = h->dev;
  lbm::fill_geometry(d, *p, s.D, h->ops->pop_bytes);
  lbm::fill_phys(d, *p, s.D);

  auto bail = [&](cudaError_t err, const char* where) {
    g_create_error = std::string(where) + ": " + cudaGetErrorString(err);
    lbm_status st = err == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
    lbm_destroy(h);
    return st;
  };
  cudaError_t err;
  if (p->stream) {
    h->stream = (cudaStream_t)p->stream;
  } else {
    if ((err = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking)) != cudaSuccess) return bail(err, "cudaStreamCreate");
    h->own_stream = true;
  }
  if ((err = keep_alloc(*p, &d.f, s.f_bytes)) != cudaSuccess) return bail(err, "allocating the populations");
  if ((err = keep_alloc(*p, &d.aux, s.aux_bytes)) != cudaSuccess) return bail(err, "allocating the auxiliary fields");
  if (s.rho_w_bytes) {
    void* rw = nullptr;
    if ((err = keep_alloc(*p, &rw, s.rho_w_bytes)) != cudaSuccess) return bail(err, "allocating rho_w");
    d.rho_w[0] = (float*)rw;
    d.rho_w[1] = d.rho_w[0] + s.N;
    if ((err = cudaMemsetAsync(d.rho_w[0], 0, s.rho_w_bytes, h->stream)) != cudaSuccess) return bail(err, "cudaMemset(rho_w)");
  }
  {
    void* fl = nullptr;
    if ((err = keep_alloc(*p, &fl, sizeof(unsigned int) + sizeof(unsigned long long) * 2)) != cudaSuccess)
      return bail(err, "allocating the error words");
    d.flags = (unsigned int*)fl;
  }
  d.guards = (unsigned long long*)((char*)d.flags + sizeof(unsigned long long));
  if ((err = cudaMemsetAsync(d.flags, 0, sizeof(unsigned int) + sizeof(unsigned long long) * 2, h->stream)) != cudaSuccess)
    return bail(err, "cudaMemset(flags)");
  if ((err = cudaMemsetAsync(d.aux, 0, s.aux_bytes, h->stream)) != cudaSuccess) return bail(err, "cudaMemset(aux)");
  {
    const char* why = nullptr;
    if (!lbm::make_tile_maps(&h->maps, d, s.D, h->ops->aux_bytes, &why)) {
      g_create_error = why;
      lbm_destroy(h);
      return LBM_ERR_CUDA;
    }
  }
  if ((err = cudaMallocHost(&h->h_flags, sizeof(unsigned int))) != cudaSuccess) return bail(err, "cudaMallocHost");
  *h->h_flags = 0;
  if ((err = cudaEventCreateWithFlags(&h->flags_ev, cudaEventDisableTiming)) != cudaSuccess) return bail(err, "cudaEventCreate");
  if ((err = cudaStreamSynchronize(h->stream)) != cudaSuccess) return bail(err, "cudaStreamSynchronize");
  *out = h;
  return LBM_OK;
}

lbm_status lbm_destroy(lbm_handle h) {
  if (!h) return LBM_OK;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (auto& m : h->marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
  for (auto e : h->ev_pool) cudaEventDestroy(e);
  for (auto& g : h->step_graph)
    if (g) cudaGraphExecDestroy(g);
  keep_free(h->p, h->dev.f);
  keep_free(h->p, h->dev.aux);
  keep_free(h->p, h->dev.rho_w[0]);
  keep_free(h->p, h->dev.flags);
  keep_free(h->p, h->dev.gamma_out);
  if (h->h_flags) cudaFreeHost(h->h_flags);
  if (h->flags_ev) cudaEventDestroy(h->flags_ev);
  if (h->own_stream && h->stream) cudaStreamDestroy(h->stream);
  delete h;
  return LBM_OK;
}

lbm_status lbm_init_fields(lbm_handle h, const double* rho, const double* ux, const double* uy, const double* uz) {
  LBM_LIVE(h);
  const int D = h->ops->D;
  if (!rho || !ux || !uy || (D == 3 && !uz)) return fail(h, LBM_ERR_INVALID_ARG, "NULL field array");
  const size_t nb = (size_t)h->dev.N * sizeof(double);
  double* buf = nullptr;
  LBM_CUDA(h, scratch_alloc(h, &buf, nb * (1 + D)));
  LBM_CUDA(h, cudaMemcpyAsync(buf, rho, nb, cudaMemcpyHostToDevice, h->stream));
  LBM_CUDA(h, cudaMemcpyAsync(buf + h->dev.N, ux, nb, cudaMemcpyHostToDevice, h->stream));
  LBM_CUDA(h, cudaMemcpyAsync(buf + 2 * h->dev.N, uy, nb, cudaMemcpyHostToDevice, h->stream));
  if (D == 3) LBM_CUDA(h, cudaMemcpyAsync(buf + 3 * h->dev.N, uz, nb, cudaMemcpyHostToDevice, h->stream));
  return init_from_device_fields(h, buf);
}

lbm_status lbm_init_drop_on_film(lbm_handle h, const lbm_drop_on_film* g) {
  LBM_LIVE(h);
  if (!g) return fail(h, LBM_ERR_INVALID_ARG, "geometry is NULL");
  if (!(g->radius > 0) || !(g->width > 0) || !std::isfinite(g->speed) || !(g->noise >= 0) || !std::isfinite(g->film) ||
      !std::isfinite(g->gap))
    return fail(h, LBM_ERR_INVALID_ARG, "drop-on-film needs radius > 0, width > 0, noise >= 0 and finite film, gap, speed");
  const int D = h->ops->D;
  double* buf = nullptr;
  LBM_CUDA(h, scratch_alloc(h, &buf, (size_t)h->dev.N * sizeof(double) * (1 + D)));
  h->ops->drop_on_film(h->dev, *g, h->p.rho_liquid, h->p.rho_vapour, buf, buf + h->dev.N, h->stream);
  h->launches += 1;
  return init_from_device_fields(h, buf);
}

}  // extern "C"

namespace {
// Populations at rest in the reported sense for the float64 fields in the device
// buffer buf = [rho | ux | uy (| uz)], which this frees.
lbm_status init_from_device_fields(lbm_handle h, double* buf) {
  const int D = h->ops->D;
  double* uz_d = D == 3 ? buf + 3 * h->dev.N : nullptr;
  // the (rho, psi) pairs of the density field, the force they give, the bare velocity
  // u - F/(2 rho), and the equilibrium there, so that the reported velocity is u
  h->ops->aux_density(h->dev, buf, h->stream);
  h->parity = 0;
  h->ops->bare_velocity(h->dev, buf, buf + h->dev.N, h->stream);
  h->ops->init_equilibrium(h->dev, buf, buf + h->dev.N, buf + 2 * h->dev.N, uz_d, h->stream);
  h->launches += 3;
  LBM_CUDA(h, cudaGetLastError());
  LBM_CUDA(h, cudaFreeAsync(buf, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->steps = 0;
  return LBM_OK;
}
}  // namespace

extern "C" {

lbm_status lbm_step(lbm_handle h, int64_t nsteps) {
  LBM_LIVE(h);
  if (nsteps < 0) return fail(h, LBM_ERR_INVALID_ARG, "nsteps < 0");
  lbm_status st = poll_flags(h, false);
  if (st != LBM_OK) return st;
  if (h->record_gamma && !h->dev.gamma_out) {
    // (gamma, omega) per node
    void* g = nullptr;
    LBM_CUDA(h, keep_alloc(h->p, &g, 2 * (size_t)h->dev.N * sizeof(float)));
    h->dev.gamma_out = (float*)g;
    LBM_CUDA(h, cudaMemsetAsync(h->dev.gamma_out, 0, 2 * (size_t)h->dev.N * sizeof(float), h->stream));
  }
  if (h->record_gamma && nsteps > 0) h->gamma_recorded = true;
  DevDomain saved = h->dev;
  if (!h->record_gamma) h->dev.gamma_out = nullptr;
  for (int64_t s = 0; s < nsteps;) {
    if (!h->timing && h->graphs_ok && h->plain_steps >= 2 && nsteps - s >= 2) {
      bool replayed = false;
      if ((st = launch_pair_graph(h, &replayed)) != LBM_OK) break;
      if (replayed) {
        h->steps += 2;  // two steps: the parity is back where it was
        s += 2;
        continue;
      }
    }
    if ((st = launch_k(h, 0)) != LBM_OK) break;
    if ((st = launch_k(h, 1)) != LBM_OK) break;
    h->parity ^= 1;
    h->steps += 1;
    h->plain_steps += 1;
    s += 1;
  }
  h->dev.gamma_out = saved.gamma_out;
  if (st != LBM_OK) return st;
  if (nsteps > 0 && !h->flags_pending) return enqueue_flag_copy(h, h->stream);
  return LBM_OK;
}

lbm_status lbm_synchronize(lbm_handle h) {
  LBM_LIVE(h);
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  lbm_status st = poll_flags(h, true);
  if (st != LBM_OK) return st;
  // flags of the most recent steps
  LBM_CUDA(h, cudaMemcpy(h->h_flags, h->dev.flags, sizeof(unsigned int), cudaMemcpyDeviceToHost));
  return flags_status(h, *h->h_flags);
}

lbm_status lbm_read_macroscopic(lbm_handle h, double* rho, double* ux, double* uy, double* uz) {
  LBM_LIVE(h);
  const int D = h->ops->D;
  if (!rho || !ux || !uy || (D == 3 && !uz)) return fail(h, LBM_ERR_INVALID_ARG, "NULL field array");
  lbm_status st = refresh_aux(h);
  if (st != LBM_OK) return st;
  const size_t nb = (size_t)h->dev.N * sizeof(double);
  double* buf = nullptr;
  LBM_CUDA(h, scratch_alloc(h, &buf, nb * (1 + D)));
  h->ops->macroscopic(h->dev, h->parity, buf, buf + h->dev.N, h->stream);
  h->launches += 1;
  LBM_CUDA(h, cudaGetLastError());
  LBM_CUDA(h, cudaMemcpyAsync(rho, buf, nb, cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaMemcpyAsync(ux, buf + h->dev.N, nb, cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaMemcpyAsync(uy, buf + 2 * h->dev.N, nb, cudaMemcpyDeviceToHost, h->stream));
  if (D == 3) LBM_CUDA(h, cudaMemcpyAsync(uz, buf + 3 * h->dev.N, nb, cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaFreeAsync(buf, h->stream));
  return lbm_synchronize(h);
}

lbm_status lbm_read_populations(lbm_handle h, double* host, size_t count) {
  LBM_LIVE(h);
  const size_t want = (size_t)h->ops->Q * h->dev.N;
  if (!host || count != want) return fail(h, LBM_ERR_INVALID_ARG, "populations buffer must hold Q*N doubles");
  double* buf = nullptr;
  LBM_CUDA(h, scratch_alloc(h, &buf, want * sizeof(double)));
  h->ops->canonical_read(h->dev, h->parity, buf, h->stream);
  h->launches += 1;
  LBM_CUDA(h, cudaGetLastError());
  LBM_CUDA(h, cudaMemcpyAsync(host, buf, want * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaFreeAsync(buf, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_read_populations_window(lbm_handle h, const int64_t origin[3], const int64_t extent[3], double* host,
                                       size_t count) {
  LBM_LIVE(h);
  if (!origin || !extent || !host) return fail(h, LBM_ERR_INVALID_ARG, "window origin, extent and buffer are required");
  const long long n[3] = {h->dev.nx, h->dev.ny, h->dev.nz};
  int o[3], e[3];
  for (int a = 0; a < 3; ++a) {
    if (origin[a] < 0 || origin[a] >= n[a] || extent[a] < 1 || extent[a] > n[a])
      return fail(h, LBM_ERR_INVALID_ARG, "window needs 0 <= origin < n and 1 <= extent <= n on every axis");
    o[a] = (int)origin[a];
    e[a] = (int)extent[a];
  }
  const size_t m = (size_t)e[0] * e[1] * e[2];
  const size_t want = (size_t)h->ops->Q * m;
  if (count != want) return fail(h, LBM_ERR_INVALID_ARG, "window buffer must hold Q*ex*ey*ez doubles");
  double* buf = nullptr;
  LBM_CUDA(h, scratch_alloc(h, &buf, want * sizeof(double)));
  h->ops->canonical_window(h->dev, h->parity, o, e, buf, h->stream);
  h->launches += 1;
  LBM_CUDA(h, cudaGetLastError());
  LBM_CUDA(h, cudaMemcpyAsync(host, buf, want * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaFreeAsync(buf, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  return LBM_OK;
}

lbm_status lbm_write_populations(lbm_handle h, const double* host, size_t count) {
  LBM_LIVE(h);
  const size_t want = (size_t)h->ops->Q * h->dev.N;
  if (!host || count != want) return fail(h, LBM_ERR_INVALID_ARG, "populations buffer must hold Q*N doubles");
  double* buf = nullptr;
  LBM_CUDA(h, scratch_alloc(h, &buf, want * sizeof(double)));
  LBM_CUDA(h, cudaMemcpyAsync(buf, host, want * sizeof(double), cudaMemcpyHostToDevice, h->stream));
  h->ops->canonical_write(h->dev, buf, h->stream);
  h->launches += 1;
  LBM_CUDA(h, cudaGetLastError());
  LBM_CUDA(h, cudaFreeAsync(buf, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  h->parity = 0;
  return LBM_OK;
}

lbm_status lbm_read_diag(lbm_handle h, double* mass, double* momentum3, double* max_u, double* gamma_field) {
  LBM_LIVE(h);
  const long long nblk = (h->dev.N + 255) / 256;
  double* buf = nullptr;
  LBM_CUDA(h, scratch_alloc(h, &buf, (size_t)(nblk * 5 + 5) * sizeof(double)));
  int nb = h->ops->diag_partial(h->dev, h->parity, buf, h->stream);
  lbm::launch_diag_final(buf, nb, buf + nblk * 5, h->stream);
  h->launches += 2;
  LBM_CUDA(h, cudaGetLastError());
  double out[5];
  LBM_CUDA(h, cudaMemcpyAsync(out, buf + nblk * 5, sizeof(out), cudaMemcpyDeviceToHost, h->stream));
  LBM_CUDA(h, cudaFreeAsync(buf, h->stream));
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  if (mass) *mass = out[0];
  if (momentum3) { momentum3[0] = out[1]; momentum3[1] = out[2]; momentum3[2] = out[3]; }
  if (max_u) *max_u = out[4];
  if (gamma_field) {
    if (h->dev.gamma_out) {
      std::vector<float> g(2 * (size_t)h->dev.N);
      LBM_CUDA(h, cudaMemcpy(g.data(), h->dev.gamma_out, g.size() * sizeof(float), cudaMemcpyDeviceToHost));
      for (long long k = 0; k < h->dev.N; ++k) gamma_field[k] = g[2 * k];
    } else {
      for (long long k = 0; k < h->dev.N; ++k) gamma_field[k] = 0.0;
    }
  }
  return LBM_OK;
}

lbm_status lbm_max_speed(lbm_handle h, double* max_u) {
  LBM_LIVE(h);
  if (!max_u) return fail(h, LBM_ERR_INVALID_ARG, "max_u is NULL");
  return reduce_max(h, [&](double* buf) { return h->ops->max_speed_partial(h->dev, h->parity, buf, h->stream); }, max_u);
}

lbm_status lbm_interface_width(lbm_handle h, double* width, double* max_grad) {
  LBM_LIVE(h);
  if (!width) return fail(h, LBM_ERR_INVALID_ARG, "width is NULL");
  double g = 0;
  const lbm_status st = reduce_max(h, [&](double* buf) { return h->ops->grad_partial(h->dev, buf, h->stream); }, &g);
  if (st != LBM_OK) return st;
  *width = g > 0 ? (h->p.rho_liquid - h->p.rho_vapour) / g : INFINITY;
  if (max_grad) *max_grad = g;
  return LBM_OK;
}

lbm_status lbm_crown_radius(lbm_handle h, int32_t layer, double* radius) {
  LBM_LIVE(h);
  if (!radius) return fail(h, LBM_ERR_INVALID_ARG, "radius is NULL");
  const int last = h->dev.pz > 1 ? h->dev.nz : h->dev.ny;
  if (layer < 0 || layer >= last) return fail(h, LBM_ERR_INVALID_ARG, "layer outside the domain's last axis");
  const double mid = 0.5 * (h->p.rho_liquid + h->p.rho_vapour);
  return reduce_max(h, [&](double* buf) { return h->ops->crown_partial(h->dev, layer, mid, buf, h->stream); }, radius);
}

lbm_status lbm_read_relaxation(lbm_handle h, double* two_over_omega_gamma) {
  LBM_LIVE(h);
  if (!two_over_omega_gamma) return fail(h, LBM_ERR_INVALID_ARG, "output is NULL");
  if (!h->dev.gamma_out || !h->gamma_recorded)
    return fail(h, LBM_ERR_INVALID_ARG, "no step has run with gamma recording on (lbm_record_gamma)");
  std::vector<float> g(2 * (size_t)h->dev.N);
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  LBM_CUDA(h, cudaMemcpy(g.data(), h->dev.gamma_out, g.size() * sizeof(float), cudaMemcpyDeviceToHost));
  for (long long k = 0; k < h->dev.N; ++k) two_over_omega_gamma[k] = 2.0 / ((double)g[2 * k + 1] * (double)g[2 * k]);
  return LBM_OK;
}

lbm_status lbm_record_gamma(lbm_handle h, int enable) {
  LBM_LIVE(h);
  h->record_gamma = enable != 0;
  return LBM_OK;
}

lbm_status lbm_guard_count(lbm_handle h, uint64_t* count) {
  LBM_LIVE(h);
  if (!count) return fail(h, LBM_ERR_INVALID_ARG, "count is NULL");
  unsigned long long c = 0;
  LBM_CUDA(h, cudaStreamSynchronize(h->stream));
  LBM_CUDA(h, cudaMemcpy(&c, h->dev.guards, sizeof(c), cudaMemcpyDeviceToHost));
  *count = c;
  return LBM_OK;
}

lbm_status lbm_set_timing(lbm_handle h, int enable) {
  LBM_LIVE(h);
  lbm_status st = drain_marks(h);
  if (st != LBM_OK) return st;
  h->timing = enable != 0;
  h->ms[0] = h->ms[1] = 0;
  h->cnt[0] = h->cnt[1] = 0;
  return LBM_OK;
}

lbm_status lbm_kernel_times(lbm_handle h, double ms[2], int64_t count[2]) {
  LBM_LIVE(h);
  lbm_status st = drain_marks(h);
  if (st != LBM_OK) return st;
  if (ms) { ms[0] = h->ms[0]; ms[1] = h->ms[1]; }
  if (count) { count[0] = h->cnt[0]; count[1] = h->cnt[1]; }
  return LBM_OK;
}

int64_t lbm_launch_count(lbm_handle h) { return h ? h->launches : 0; }

const char* lbm_last_error(lbm_handle h) {
  if (!h) return g_create_error.c_str();
  return h->err.empty() ? "no error" : h->err.c_str();
}

}  // extern "C"
