// The library's own allocations: device scratch, tables and page-locked
// record buffers of handles and ensembles (never the caller's field arrays).
// Every one goes through these functions, which keep the number and bytes of
// the live ones, so that a test can check that each error path releases what
// it had taken, and which can be told to fail the n-th allocation from now on
// as if the device were out of memory: the call returns
// cudaErrorMemoryAllocation without allocating and without touching the
// device, so the injected failure involves no GPU fault.
#include <cuda_runtime.h>

#include <mutex>
#include <unordered_map>

#include "../../include/u1u1.h"
#include "host_internal.h"

namespace u1u1 {
namespace {

struct AllocBook {
  std::mutex mu;
  std::unordered_map<void*, size_t> live;  // pointer -> bytes, device and host
  long long bytes = 0;
  long long countdown = 0;  // > 0: the allocation that brings it to zero fails
};

AllocBook& book() {
  static AllocBook* b = new AllocBook();  // never destroyed: frees may run during exit
  return *b;
}

template <typename F>
cudaError_t counted_alloc(void** p, size_t bytes, F&& allocate) {
  AllocBook& b = book();
  std::lock_guard<std::mutex> g(b.mu);
  *p = nullptr;
  if (b.countdown > 0 && --b.countdown == 0) return cudaErrorMemoryAllocation;
  const cudaError_t e = allocate(p, bytes);
  if (e == cudaSuccess && *p) {
    b.live[*p] = bytes;
    b.bytes += (long long)bytes;
  }
  return e;
}

void forget(void* p) {
  AllocBook& b = book();
  std::lock_guard<std::mutex> g(b.mu);
  auto it = b.live.find(p);
  if (it == b.live.end()) return;
  b.bytes -= (long long)it->second;
  b.live.erase(it);
}

}  // namespace

cudaError_t dev_alloc_bytes(void** p, size_t bytes) {
  return counted_alloc(p, bytes, [](void** q, size_t n) { return cudaMalloc(q, n); });
}

cudaError_t host_alloc_bytes(void** p, size_t bytes) {
  return counted_alloc(p, bytes, [](void** q, size_t n) { return cudaMallocHost(q, n); });
}

void dev_free(void* p) {
  if (!p) return;
  forget(p);
  cudaFree(p);
}

void host_free(void* p) {
  if (!p) return;
  forget(p);
  cudaFreeHost(p);
}

}  // namespace u1u1

using namespace u1u1;

extern "C" int u1u1_inject_alloc_failure(int nth) {
  if (nth < 0) return fail(U1U1_ERR_INVALID_ARG, "nth must be >= 0");
  AllocBook& b = book();
  std::lock_guard<std::mutex> g(b.mu);
  b.countdown = nth;
  return U1U1_OK;
}

extern "C" int u1u1_live_allocations(int64_t* count, int64_t* bytes) {
  if (!count || !bytes) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  AllocBook& b = book();
  std::lock_guard<std::mutex> g(b.mu);
  *count = (int64_t)b.live.size();
  *bytes = (int64_t)b.bytes;
  return U1U1_OK;
}
