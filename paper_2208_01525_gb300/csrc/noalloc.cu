// String detection for callers that cannot allocate device memory.
//
// u1u1_detect_strings_noalloc runs the same windings kernel, cell pass and
// finalize as u1u1_detect_strings, but without a lattice handle: its scratch
// (per-site winding bytes, packed cell masks, block partials, the census
// counters and the result record) is carved out of one file-scope static device array, so the call
// itself never calls cudaMalloc, cudaFree or any allocating routine.
#include <cuda.h>
#include <cuda_runtime.h>
#include <string.h>

#include <mutex>

#include "../../include/u1u1.h"
#include "host_internal.h"
#include "u1u1_internal.cuh"

using namespace u1u1;

namespace {

constexpr size_t NOALLOC_BYTES = 48ull << 20;  // 48 MiB on every GPU that loads the library

// The scratch array.  In host code this name is only a host-side stand-in:
// its device address comes from cudaGetSymbolAddress, once per device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_BYTES];

constexpr int MAX_DEVICES = 64;
void* g_scratch_addr[MAX_DEVICES] = {};
unsigned long long g_scratch_ctx[MAX_DEVICES] = {};  // context the address belongs to
std::mutex g_scratch_mu;

size_t round_up(size_t v) { return (v + 255) & ~(size_t)255; }

// Unique id of the calling thread's current context, 0 when there is none
// (or the driver entry points are unavailable).  Neither query allocates.
unsigned long long current_context_id() {
  using GetCurrentFn = CUresult (*)(CUcontext*);
  using GetIdFn = CUresult (*)(CUcontext, unsigned long long*);
  static const GetCurrentFn get_current = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (GetCurrentFn) nullptr;
    }
    return reinterpret_cast<GetCurrentFn>(p);
  }();
  static const GetIdFn get_id = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (GetIdFn) nullptr;
    }
    return reinterpret_cast<GetIdFn>(p);
  }();
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (!get_current || !get_id || get_current(&ctx) != CUDA_SUCCESS || !ctx || get_id(ctx, &id) != CUDA_SUCCESS)
    return 0;
  return id;
}

// Device address of the scratch array on the current device.  Set up on
// the first call per device, with that device current; looked up again
// only when the device's context has changed since (after a
// cudaDeviceReset the module may be loaded at another address).
int scratch_address(void** out) {
  int dev = 0;
  U1U1_CUDA_TRY(cudaGetDevice(&dev), "cudaGetDevice");
  if (dev < 0 || dev >= MAX_DEVICES) return fail(U1U1_ERR_NOT_SUPPORTED, "device index %d out of range", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  const unsigned long long ctx = current_context_id();
  if (!g_scratch_addr[dev] || ctx == 0 || ctx != g_scratch_ctx[dev]) {
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetSymbolAddress of the static scratch array");
    g_scratch_addr[dev] = ptr;
    g_scratch_ctx[dev] = current_context_id();
  }
  *out = g_scratch_addr[dev];
  return U1U1_OK;
}

template <typename T>
int run_detect(const u1u1_params* p, const void* const fields[U1U1_NFIELDS], int64_t n, int tol, unsigned char* base,
               u1u1_strings* out, cudaStream_t st) {
  const size_t V = (size_t)p->nx * p->ny * p->nz;
  const int nblocks = wind_grid_blocks(p->nx, p->ny, p->nz);
  const int ncblocks = cells_grid_blocks();
  // carve the scratch: face bytes, cell masks, block partials, cell partials,
  // census counters, record
  const size_t off_faces = 0;
  const size_t off_masks = off_faces + round_up(2 * V);
  const size_t off_part = off_masks + round_up(2 * sizeof(uint32_t) * cell_mask_words(p->nx, p->ny, p->nz));
  const size_t off_cpart = off_part + round_up(sizeof(BlockPartial) * (size_t)(nblocks + FIN_STAGE_BLOCKS));
  const size_t off_ge4 = off_cpart + round_up(sizeof(CellPartial) * (size_t)ncblocks);
  const size_t off_rec = off_ge4 + round_up(2 * sizeof(unsigned long long));
  const size_t need = off_rec + round_up(sizeof(RawRecord));
  if (need > NOALLOC_BYTES)
    return fail(U1U1_ERR_INVALID_ARG, "lattice %dx%dx%d needs %zu bytes of scratch; the static array holds %zu", p->nx,
                p->ny, p->nz, need, NOALLOC_BYTES);
  uint8_t* faces = base + off_faces;
  uint32_t* masks = (uint32_t*)(base + off_masks);
  BlockPartial* part = (BlockPartial*)(base + off_part);
  CellPartial* cpart = (CellPartial*)(base + off_cpart);
  unsigned long long* ge4 = (unsigned long long*)(base + off_ge4);
  RawRecord* rec = (RawRecord*)(base + off_rec);
  // every scratch word read below is first written by the same call (face
  // bytes and masks for every site, one partial per block, the record; the
  // cell pass clears the census counters with a memset), so nothing needs
  // clearing here

  // the windings read only the ten position fields
  PosView<T> v;
  for (int f = 0; f < U1U1_NPOS; ++f) v.pos[f] = (const T*)fields[f];
  v.nx = p->nx;
  v.ny = p->ny;
  v.nz = p->nz;
  cudaError_t e = launch_windings<T>(v, (T)p->dx, part, faces, nullptr, st);
  if (e != cudaSuccess) return cuda_fail(e, "windings kernel");
  e = launch_cells(faces, p->nx, p->ny, p->nz, tol, nullptr, nullptr, masks, cpart, st, nullptr, ge4);
  if (e != cudaSuccess) return cuda_fail(e, "cell overlap kernel");
  e = launch_finalize(part, nblocks, cpart, ncblocks, rec, (long long)n, 0, 0, 1, tol, st, ge4);
  if (e != cudaSuccess) return cuda_fail(e, "finalize kernel");
  RawRecord r;
  U1U1_CUDA_TRY(cudaMemcpyAsync(&r, rec, sizeof(RawRecord), cudaMemcpyDeviceToHost, st), "record copy");
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  to_strings(p, r, out);
  return U1U1_OK;
}

}  // namespace

extern "C" int u1u1_detect_strings_noalloc(const u1u1_params* p, const void* const fields[U1U1_NFIELDS], int64_t n,
                                           int overlap_tol, u1u1_strings* out, void* stream) {
  int rc = u1u1_check_params(p);
  if (rc) return rc;
  if (!fields || !out) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  for (int f = 0; f < U1U1_NFIELDS; ++f) {
    if (!fields[f]) return fail(U1U1_ERR_INVALID_ARG, "fields[%d] is NULL", f);
    if ((uintptr_t)fields[f] % 256 != 0) return fail(U1U1_ERR_INVALID_ARG, "fields[%d] is not 256-byte aligned", f);
  }
  if (overlap_tol < 0 || overlap_tol > 1) return fail(U1U1_ERR_INVALID_ARG, "overlap tolerance must be 0 or 1");
  const double sites = (double)p->nx * p->ny * p->nz;
  if (sites > (double)U1U1_NOALLOC_MAX_SITES)
    return fail(U1U1_ERR_INVALID_ARG, "lattice of %.0f sites exceeds the %d-site limit of the allocation-free entry point",
                sites, U1U1_NOALLOC_MAX_SITES);
  void* base = nullptr;
  rc = scratch_address(&base);
  if (rc) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  return p->precision == U1U1_FP64 ? run_detect<double>(p, fields, n, overlap_tol, (unsigned char*)base, out, st)
                                   : run_detect<float>(p, fields, n, overlap_tol, (unsigned char*)base, out, st);
}
