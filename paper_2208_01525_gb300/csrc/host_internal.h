// Host-side internals shared by the C-ABI translation units (api.cu,
// ensemble.cu): the lattice handle, error reporting and coefficients.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>

#include "../../include/u1u1.h"
#include "u1u1_internal.cuh"

namespace u1u1 {


extern thread_local std::string g_last_error;
int fail(int code, const char* fmt, ...);
int cuda_fail(cudaError_t e, const char* where);

#define U1U1_CUDA_TRY(expr, where)                      \
  do {                                                  \
    cudaError_t e_ = (expr);                            \
    if (e_ != cudaSuccess) return ::u1u1::cuda_fail(e_, where); \
  } while (0)

// The library's device and page-locked host allocations, counted, with an
// injectable failure (alloc.cu).  Frees of NULL are no-ops.
cudaError_t dev_alloc_bytes(void** p, size_t bytes);
cudaError_t host_alloc_bytes(void** p, size_t bytes);
void dev_free(void* p);
void host_free(void* p);
template <typename P>
cudaError_t dev_alloc(P** p, size_t bytes) {
  return dev_alloc_bytes((void**)p, bytes);
}
template <typename P>
cudaError_t host_alloc(P** p, size_t bytes) {
  return host_alloc_bytes((void**)p, bytes);
}

// A named range on the host timeline around an entry point's enqueue work,
// for profilers that read NVTX (free when none is attached).
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// step coefficients of step n (Eqs. 12, 19, 22), FP64
void coeffs(const u1u1_params* p, int64_t n, double out[6]);
// the kernels' coefficient block for step n
template <typename T>
Coef<T> make_coef(const u1u1_params* p, int64_t n);
// host epilogue of a detection record (Sec. III.A, Eqs. 31-35)
void to_strings(const u1u1_params* p, const RawRecord& r, u1u1_strings* s);

}  // namespace u1u1

struct u1u1_lattice {
  using BlockPartial = u1u1::BlockPartial;
  using CellPartial = u1u1::CellPartial;
  using RawRecord = u1u1::RawRecord;
  u1u1_params p;
  size_t V;
  size_t esize;
  void* pos[2][U1U1_NPOS];
  void* mom[U1U1_NMOM];
  int cur;
  int64_t n;
  int kernel;       // U1U1_KERNEL_*
  int tile_waves;   // z-chunk target of the tiled kernel (tuning knob)
  int overlap_tol;
  // scratch (owned)
  uint8_t* faces;
  uint32_t* masks;  // packed pierced-cell bits, two sectors
  BlockPartial* partials;
  int npartials;
  CellPartial* cpartials;
  int ncpartials;
  unsigned long long* ge4;  // census counters of cells with value >= 4
  uint32_t* mpq;      // bound-state cell bits (segments), lazily allocated
  int* seg_label;     // component labels (segments), lazily allocated
  int* seg_size;
  u1u1::SegCounts* seg_counts;
  RawRecord* ring;
  RawRecord* scratch_rec;
  int* tma_status;      // device word: U1U1_ERR_TIMEOUT after a tensor-copy wait ran out
  int* host_status;     // pinned copy of it, read after a synchronisation
  RawRecord* host_rec;  // pinned, RING_CAP entries
  int64_t rec_written;
  int64_t rec_read;
  int ensemble_box;  // nonzero: owned by an ensemble, whose tables hold its parameters
};

namespace u1u1 {
// validate, allocate the handle and its scratch (no kernel launched)
int lattice_create(const u1u1_params* p, const u1u1_buffers* b, u1u1_lattice** out);
void lattice_free_scratch(u1u1_lattice* h);
// release a handle and its scratch (the ensemble's path for its boxes)
void lattice_destroy(u1u1_lattice* h);
// enqueue the random-phase initial conditions into buffer 0 (and zero the rest)
cudaError_t lattice_init_fields(u1u1_lattice* h, cudaStream_t st);
}  // namespace u1u1
