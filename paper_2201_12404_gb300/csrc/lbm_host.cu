// Page-locked host buffers for the calls that take host arrays (lbm_init_fields,
// lbm_read_macroscopic, lbm_read/write_populations).
//
// On a Grace host the GPU reads and writes host memory over NVLink-C2C, and a
// buffer made of small pages can copy several times slower than the link allows
// when the GPU touches it for the first time in a while: what the copy engines
// pay is address translation, not bandwidth.  Buffers of at least half a
// transparent huge page are mapped on a huge-page boundary, sized in whole huge
// pages and advised for huge pages before their first touch, so that a few large
// pages cover a field of ~0.5 GB; smaller ones use the system's pages.  Both are
// then registered (page-locked) with the CUDA runtime.  Where the kernel gives no
// huge pages the buffer is still page-locked, with the system's page size.
#include <cuda_runtime.h>
#include <sys/mman.h>
#include <unistd.h>

#include <cstdint>
#include <cstdio>
#include <cstring>
#include <map>
#include <mutex>

#include "lbm.h"

namespace {

std::mutex g_mu;

// aligned start -> mapped length of every live buffer
std::map<void*, size_t>& live() {
  static std::map<void*, size_t> m;
  return m;
}

// Bytes of a transparent huge page as the kernel reports them, or 0 when huge
// pages are switched off or the kernel does not say.
size_t huge_page_bytes() {
  FILE* e = std::fopen("/sys/kernel/mm/transparent_hugepage/enabled", "r");
  if (!e) return 0;
  char mode[128] = {};
  const size_t n = std::fread(mode, 1, sizeof(mode) - 1, e);
  std::fclose(e);
  mode[n] = 0;
  if (std::strstr(mode, "[never]")) return 0;
  FILE* f = std::fopen("/sys/kernel/mm/transparent_hugepage/hpage_pmd_size", "r");
  if (!f) return 0;
  unsigned long long v = 0;
  const int got = std::fscanf(f, "%llu", &v);
  std::fclose(f);
  return got == 1 ? (size_t)v : 0;
}

}  // namespace

extern "C" lbm_status lbm_host_alloc(size_t bytes, void** out) {
  if (!out) return LBM_ERR_INVALID_ARG;
  *out = nullptr;
  if (bytes == 0) return LBM_ERR_INVALID_ARG;
  const long sys_page = sysconf(_SC_PAGESIZE);
  const size_t page = sys_page > 0 ? (size_t)sys_page : 4096;
  const size_t huge = huge_page_bytes();
  // huge pages for buffers of at least half a huge page (512 MB pages on a 64 KB-page
  // Arm kernel would waste most of their memory on small buffers); pages otherwise
  const size_t unit = huge > page && huge % page == 0 && bytes >= huge / 2 ? huge : page;
  if (bytes > SIZE_MAX - 2 * unit) return LBM_ERR_INVALID_ARG;
  const size_t length = (bytes + unit - 1) / unit * unit;
  // map one unit more than needed, keep the aligned part, return the rest
  const size_t span = length + (unit > page ? unit : 0);
  void* m = mmap(nullptr, span, PROT_READ | PROT_WRITE, MAP_PRIVATE | MAP_ANONYMOUS, -1, 0);
  if (m == MAP_FAILED) return LBM_ERR_OOM;
  const uintptr_t b = (uintptr_t)m, a = (b + unit - 1) / unit * unit;
  if (a > b) munmap(m, a - b);
  if (b + span > a + length) munmap((void*)(a + length), b + span - (a + length));
  void* p = (void*)a;
#ifdef MADV_HUGEPAGE
  if (unit > page) madvise(p, length, MADV_HUGEPAGE);  // advice only: small pages where none are free
#endif
  // first touch now, so that the pages (huge where the kernel can) exist before they are locked
  std::memset(p, 0, length);
  if (cudaHostRegister(p, length, cudaHostRegisterDefault) != cudaSuccess) {
    cudaGetLastError();
    munmap(p, length);
    return LBM_ERR_CUDA;
  }
  {
    std::lock_guard<std::mutex> lock(g_mu);
    live()[p] = length;
  }
  *out = p;
  return LBM_OK;
}

extern "C" lbm_status lbm_host_free(void* p) {
  if (!p) return LBM_OK;
  size_t length = 0;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    auto it = live().find(p);
    if (it == live().end()) return LBM_ERR_INVALID_ARG;
    length = it->second;
    live().erase(it);
  }
  const cudaError_t e = cudaHostUnregister(p);
  munmap(p, length);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return LBM_ERR_CUDA;
  }
  return LBM_OK;
}
