// Bound-state segments of the robust method (Sec. III.B, Eq. 38): connected
// components of the fast method's pq cells on the periodic lattice, cells
// joined when they share a face, an edge or a corner.
//
// Lock-free union-find with link-by-index: every label points to a smaller
// or equal site index of the same component, a union links the larger of two
// roots under the smaller with atomicMin and retries when it lost a race, and
// finds halve paths.  The root of every component is its smallest site index,
// so the labelling is deterministic.  Every loop carries an iteration limit
// that records an error instead of spinning.
#include <stdint.h>

#include "u1u1_internal.cuh"

namespace u1u1 {

namespace {

constexpr int CCL_THREADS = 256;
constexpr int CCL_LIMIT = 1 << 24;

struct Box {
  int nx, ny, nz, words;
  __device__ bool bit(const uint32_t* m, int x, int y, int z) const {
    return (m[((long long)z * ny + y) * words + (x >> 5)] >> (x & 31)) & 1u;
  }
};

__device__ __forceinline__ int find_root(volatile int* label, int x, int* err) {
  for (int it = 0; it < CCL_LIMIT; ++it) {
    const int p = label[x];
    if (p == x) return x;
    const int gp = label[p];
    if (gp != p) label[x] = gp;  // path halving: gp is an ancestor of x
    x = gp;
  }
  atomicExch(err, 1);
  return x;
}

__device__ __forceinline__ void unite(int* label, int a, int b, int* err) {
  volatile int* vl = label;
  for (int it = 0; it < CCL_LIMIT; ++it) {
    a = find_root(vl, a, err);
    b = find_root(vl, b, err);
    if (a == b) return;
    if (a < b) {
      const int t = a;
      a = b;
      b = t;
    }
    const int old = atomicMin(&label[a], b);  // link the larger root under the smaller
    if (old == a) return;
    a = old;  // a was linked elsewhere meanwhile: continue from there
  }
  atomicExch(err, 1);
}

__global__ void k_ccl_init(const uint32_t* __restrict__ mpq, Box b, int* label, int* size) {
  const long long V = (long long)b.nx * b.ny * b.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % b.nx), y = (int)((i / b.nx) % b.ny), z = (int)(i / ((long long)b.nx * b.ny));
    label[i] = b.bit(mpq, x, y, z) ? (int)i : -1;
    size[i] = 0;
  }
}

__global__ void k_ccl_merge(const uint32_t* __restrict__ mpq, Box b, int* label, SegCounts* counts) {
  const long long V = (long long)b.nx * b.ny * b.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(i % b.nx), y = (int)((i / b.nx) % b.ny), z = (int)(i / ((long long)b.nx * b.ny));
    if (!b.bit(mpq, x, y, z)) continue;
    // the 13 neighbours that come after the cell in (z, y, x) order; the
    // other 13 are covered from the neighbour's side
    for (int dz = 0; dz <= 1; ++dz)
      for (int dy = (dz ? -1 : 0); dy <= 1; ++dy)
        for (int dx = (dz || dy ? -1 : 1); dx <= 1; ++dx) {
          const int xx = x + dx < 0 ? b.nx - 1 : (x + dx >= b.nx ? 0 : x + dx);
          const int yy = y + dy < 0 ? b.ny - 1 : (y + dy >= b.ny ? 0 : y + dy);
          const int zz = z + dz >= b.nz ? 0 : z + dz;
          if (b.bit(mpq, xx, yy, zz))
            unite(label, (int)i, (int)(xx + (long long)b.nx * (yy + (long long)b.ny * zz)), &counts->err);
        }
  }
}

__global__ void k_ccl_flatten(Box b, int* label, int* size, SegCounts* counts) {
  const long long V = (long long)b.nx * b.ny * b.nz;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    if (label[i] < 0) continue;
    const int r = find_root(label, (int)i, &counts->err);
    label[i] = r;
    atomicAdd(&size[r], 1);
  }
}

__global__ void k_ccl_stats(Box b, const int* __restrict__ label, const int* __restrict__ size, int min_cells,
                            SegCounts* counts) {
  const long long V = (long long)b.nx * b.ny * b.nz;
  unsigned long long cells = 0, comps = 0, segs = 0, len = 0, big = 0;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < V; i += (long long)gridDim.x * blockDim.x) {
    if (label[i] != (int)i) continue;  // roots only
    const unsigned long long n = (unsigned long long)size[i];
    cells += n;
    comps += 1;
    if (n > (unsigned long long)min_cells) {
      segs += 1;
      len += n - 1;  // a segment of n cells is (n - 1) dx long
    }
    big = n > big ? n : big;
  }
  for (int o = 16; o > 0; o >>= 1) {
    cells += __shfl_down_sync(0xffffffffu, cells, o);
    comps += __shfl_down_sync(0xffffffffu, comps, o);
    segs += __shfl_down_sync(0xffffffffu, segs, o);
    len += __shfl_down_sync(0xffffffffu, len, o);
    const unsigned long long ob = __shfl_down_sync(0xffffffffu, big, o);
    big = ob > big ? ob : big;
  }
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&counts->n_cells, cells);
    atomicAdd(&counts->n_components, comps);
    atomicAdd(&counts->n_segments, segs);
    atomicAdd(&counts->sum_len, len);
    atomicMax(&counts->largest, big);
  }
}

}  // namespace

cudaError_t launch_segments(const uint32_t* mpq, int nx, int ny, int nz, int min_cells, int* label, int* size,
                            SegCounts* counts, cudaStream_t st) {
  const Box b{nx, ny, nz, (nx + 31) / 32};
  cudaError_t e = cudaMemsetAsync(counts, 0, sizeof(SegCounts), st);
  if (e != cudaSuccess) return e;
  const int grid = 152 * 8;
  k_ccl_init<<<grid, CCL_THREADS, 0, st>>>(mpq, b, label, size);
  k_ccl_merge<<<grid, CCL_THREADS, 0, st>>>(mpq, b, label, counts);
  k_ccl_flatten<<<grid, CCL_THREADS, 0, st>>>(b, label, size, counts);
  k_ccl_stats<<<grid, CCL_THREADS, 0, st>>>(b, label, size, min_cells, counts);
  return cudaGetLastError();
}

}  // namespace u1u1
