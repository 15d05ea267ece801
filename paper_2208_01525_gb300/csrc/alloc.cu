// The library's own allocations: device scratch, tables and page-locked
// record buffers of handles and ensembles (never the caller's field arrays).
// Every one goes through these functions, which keep the number and bytes of
// the live ones, so that a test can check that each error path releases what
// it had taken, and which can be told to fail the n-th allocation from now on
// as if the device were out of memory: the call returns
// cudaErrorMemoryAllocation without allocating and without touching the
// device, so the injected failure involves no GPU fault.
//
// As a debugging aid in place of a device memory checker, allocations can
// also be made with guard zones: a fixed byte pattern on each side of the
// block handed out, checked on request, so that a kernel or a copy that
// writes past either end of a library buffer is caught by a test.
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>
#include <unordered_map>
#include <vector>

#include "../../include/u1u1.h"
#include "host_internal.h"

namespace u1u1 {
namespace {

constexpr unsigned char GUARD_BYTE = 0xA5;

struct Block {
  void* base;    // what cudaMalloc / cudaMallocHost returned
  size_t bytes;  // bytes handed out
  size_t guard;  // guard bytes on each side
  bool host;     // page-locked host memory
};

struct AllocBook {
  std::mutex mu;
  std::unordered_map<void*, Block> live;  // pointer handed out -> its block
  long long bytes = 0;
  long long countdown = 0;  // > 0: the allocation that brings it to zero fails
  size_t guard = 0;         // guard bytes of allocations made from now on
};

AllocBook& book() {
  static AllocBook* b = new AllocBook();  // never destroyed: frees may run during exit
  return *b;
}

// Fill the guard zones of a block with the pattern.
cudaError_t fill_guards(const Block& k) {
  char* base = (char*)k.base;
  char* tail = base + k.guard + k.bytes;
  if (k.host) {
    memset(base, GUARD_BYTE, k.guard);
    memset(tail, GUARD_BYTE, k.guard);
    return cudaSuccess;
  }
  cudaError_t e = cudaMemset(base, GUARD_BYTE, k.guard);
  if (e == cudaSuccess) e = cudaMemset(tail, GUARD_BYTE, k.guard);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();  // patterns in place before any kernel of any stream
  return e;
}

cudaError_t counted_alloc(void** p, size_t bytes, bool host) {
  AllocBook& b = book();
  std::lock_guard<std::mutex> g(b.mu);
  *p = nullptr;
  if (b.countdown > 0 && --b.countdown == 0) return cudaErrorMemoryAllocation;
  Block k{nullptr, bytes, b.guard, host};
  const size_t total = bytes + 2 * k.guard;
  cudaError_t e = host ? cudaMallocHost(&k.base, total) : cudaMalloc(&k.base, total);
  if (e != cudaSuccess || !k.base) return e;
  if (k.guard) {
    e = fill_guards(k);
    if (e != cudaSuccess) {
      if (host) cudaFreeHost(k.base); else cudaFree(k.base);
      return e;
    }
  }
  *p = (char*)k.base + k.guard;
  b.live[*p] = k;
  b.bytes += (long long)bytes;
  return cudaSuccess;
}

// Forget a pointer handed out and return the block to free (the pointer
// itself if the library did not hand it out).
void* forget(void* p) {
  AllocBook& b = book();
  std::lock_guard<std::mutex> g(b.mu);
  auto it = b.live.find(p);
  if (it == b.live.end()) return p;
  void* base = it->second.base;
  b.bytes -= (long long)it->second.bytes;
  b.live.erase(it);
  return base;
}

}  // namespace

cudaError_t dev_alloc_bytes(void** p, size_t bytes) { return counted_alloc(p, bytes, false); }

cudaError_t host_alloc_bytes(void** p, size_t bytes) { return counted_alloc(p, bytes, true); }

void dev_free(void* p) {
  if (!p) return;
  cudaFree(forget(p));
}

void host_free(void* p) {
  if (!p) return;
  cudaFreeHost(forget(p));
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

extern "C" int u1u1_set_alloc_guard(int64_t guard_bytes) {
  if (guard_bytes < 0 || guard_bytes % 256 != 0 || guard_bytes > (int64_t)1 << 30)
    return fail(U1U1_ERR_INVALID_ARG, "guard_bytes must be a multiple of 256 in [0, 2^30]");
  AllocBook& b = book();
  std::lock_guard<std::mutex> g(b.mu);
  b.guard = (size_t)guard_bytes;
  return U1U1_OK;
}

extern "C" int u1u1_inject_guard_damage(void) {
  AllocBook& b = book();
  std::lock_guard<std::mutex> g(b.mu);
  for (const auto& kv : b.live) {
    const Block& k = kv.second;
    if (!k.guard) continue;
    char* tail = (char*)k.base + k.guard + k.bytes;  // first byte of the tail guard
    if (k.host) {
      *tail = 0;
      return U1U1_OK;
    }
    cudaError_t e = cudaMemset(tail, 0, 1);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    return e == cudaSuccess ? U1U1_OK : cuda_fail(e, "guard damage");
  }
  return fail(U1U1_ERR_STATE, "no live allocation has guard zones");
}

extern "C" int u1u1_check_alloc_guards(int64_t* corrupted) {
  if (!corrupted) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  AllocBook& b = book();
  std::lock_guard<std::mutex> g(b.mu);
  cudaError_t e = cudaDeviceSynchronize();  // every kernel and copy that could still write has finished
  if (e != cudaSuccess) return cuda_fail(e, "device synchronize");
  int64_t bad = 0;
  std::vector<unsigned char> buf;
  for (const auto& kv : b.live) {
    const Block& k = kv.second;
    if (!k.guard) continue;
    const unsigned char* zone[2] = {(const unsigned char*)k.base, (const unsigned char*)k.base + k.guard + k.bytes};
    bool ok = true;
    for (int side = 0; side < 2 && ok; ++side) {
      const unsigned char* z = zone[side];
      if (!k.host) {
        buf.resize(k.guard);
        e = cudaMemcpy(buf.data(), z, k.guard, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(e, "guard read");
        z = buf.data();
      }
      for (size_t i = 0; i < k.guard; ++i)
        if (z[i] != GUARD_BYTE) {
          ok = false;
          break;
        }
    }
    if (!ok) ++bad;
  }
  *corrupted = bad;
  return U1U1_OK;
}
