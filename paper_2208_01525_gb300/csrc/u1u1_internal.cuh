// Internal declarations shared by the kernels and the C-ABI host code of
// libu1u1.  Nothing here is part of the public interface (include/u1u1.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/u1u1.h"

namespace u1u1 {

constexpr int RING_CAP = 1024;  // detection records kept on the device per lattice

// ---------------------------------------------------------------------------
// Reduction record layout.  Every measuring kernel writes one partial per
// block; a single-block finalize kernel merges them in a fixed order into a
// RawRecord, so results are bit-reproducible for a given launch shape.
// ---------------------------------------------------------------------------
enum SumIdx {
  S_KIN_P, S_KIN_Q, S_GRAD_P, S_GRAD_Q, S_EL_P, S_EL_Q, S_MAG_P, S_MAG_Q, S_POT, S_VINT,
  S_LAG, S_ENERGY, S_RL_NUM, S_RL_DEN, S_RPQ_NUM, S_RPQ_DEN,
  S_GAUSS_P, S_GAUSS_Q, S_CHARGE_P, S_CHARGE_Q,
  S_POT_P, S_POT_Q,  // c_n lambda_s/4 (|phi_s|^2 - sigma_s^2)^2 per sector
  NSUM
};
enum MaxIdx {
  M_GAUSS_P, M_GAUSS_Q, M_NEG_PHIMIN_P, M_PHIMAX_P, M_NEG_PHIMIN_Q, M_PHIMAX_Q,
  NMAX
};
enum CntIdx {
  C_NP, C_NQ, C_NZP, C_NZQ, C_NPQ_PLAQ, C_FLAGGED, C_MAXW, C_NAN,
  C_W2P, C_W2Q,  // plaquettes with |W| >= 2 per sector
  NCNT
};

struct BlockPartial {
  double sum[NSUM];
  double comp[NSUM];  // Neumaier compensation terms of the block's sums
  double mx[NMAX];
  long long cnt[NCNT];
};

struct CellPartial {
  long long pq[2];  // p-anchored and q-anchored overlap counts
};

struct RawRecord {
  double sum[NSUM];
  double mx[NMAX];
  long long cnt[NCNT];
  long long cells[4];  // overlap p-anchored, q-anchored; cells with value >= 4, p and q
  long long n;
  int has_diag, has_gauss, has_strings, tol;
};
// bytes moved device -> host per detection record read
static_assert(sizeof(RawRecord) == 360, "record layout changed: update the benchmark's byte count");

// Bits of a per-site, per-sector "face byte": |W| (saturated at 3) of the
// three plaquettes anchored at the site, plus a branch-cut flag.
__host__ __device__ constexpr int FACE_SHIFT(int k) { return 2 * k; }
constexpr unsigned FACE_FLAG = 0x40u;

// ---------------------------------------------------------------------------
// Per-step coefficients, evaluated on the host in FP64 and rounded to T.
// ---------------------------------------------------------------------------
template <typename T>
struct Coef {
  // scalar kick: pi+ = kPa pi + kP1 (sum(fwd + bwd) - 6 phi) - g phi,
  // g = kgl[s] (|phi_s|^2 - sigma_s^2) - kgk (|phi_o|^2 - sigma_o^2)
  T kPa, kP1, kgl[2], kgk;
  // gauge kick: E+ = kEa E - kE1 C + kE2 Im[phi^* U phi(x+i)]
  T kEa, kE1, kE2[2];
  T deta, dx;
  // diagnostics
  T inv_dx2;        // 1/dx^2 (gradient energy)
  T el_f[2];        // 1/(2 e^2 c_n)
  T mag_f[2];       // 1/(2 e^2 c_n dx^2) (F is stored times dx)
  T cV;             // c_n
  T lam4[2], sig2[2], kappa;
  T inv_dx;         // Gauss divergence
  T qG[2];          // 2 e^2 c~_{n-1}, Gauss charge factor
};

// Tensor maps of the ten position fields of one position buffer for the
// FP32 tiled kernels' tensor copies (box: one ring slot of one field); kept
// in a kernel parameter or, for ensembles, in device memory.  `enabled` is 0
// when they could not be made (FP64, lattices without an interior tile, no
// driver entry point); the kernels then fill every ring slot by cp.async.
struct TmaPlan {
  CUtensorMap map[U1U1_NPOS];
  int enabled;
  unsigned extra_bytes;  // failure-detection test hook: 0 in normal runs
  long long limit_ns;    // limit of a wait for a slot's copies (2 s)
  int* status;           // device word of the launching handle (or ensemble):
                         // set to U1U1_ERR_TIMEOUT when a wait ran out
};
template <typename T>
void make_tma_plan(const T* const pin[U1U1_NPOS], int nx, int ny, int nz, TmaPlan* tp);

// Raw field pointers of one lattice (positions double-buffered).
template <typename T>
struct LatticeView {
  const T* pin[U1U1_NPOS];  // positions at step n
  T* pout[U1U1_NPOS];       // positions at step n+1 (other buffer)
  T* mom[U1U1_NMOM];        // momenta, in place
  int nx, ny, nz;
};

// Read-only view of the ten position fields (windings kernel).
template <typename T>
struct PosView {
  const T* pos[U1U1_NPOS];
  int nx, ny, nz;
};

// Outputs of a measuring kernel.
struct MeasureOut {
  BlockPartial* partial;  // one per block
  uint8_t* faces;         // 2 * V bytes (sector-major) or nullptr
  int8_t* windings;       // 6 * V signed windings or nullptr
};

// ---------------------------------------------------------------------------
// Launchers (defined in the .cu files, called by the host API).
// ---------------------------------------------------------------------------
template <typename T>
cudaError_t launch_init(const LatticeView<T>& v, T* pos1[U1U1_NPOS], uint64_t seed, double sigma_p,
                        double sigma_q, cudaStream_t st);

// Simple kernel family: mode bits
enum { MODE_WRITE = 1, MODE_MEASURE = 2, MODE_GAUSS = 4 };
int simple_grid_blocks();  // fixed grid of the simple kernels (partials needed)
template <typename T>
cudaError_t launch_simple(int mode, const LatticeView<T>& v, const Coef<T>& c, const MeasureOut& mo,
                          cudaStream_t st);

// Tiled z-marching kernel (FP32 and FP64).
// waves: CTAs per SM-slot the z-chunking aims at (tuning knob; grid about
// 152 x 3 x waves CTAs).
// A measuring launch (MODE_MEASURE) with mo.faces set also runs the windings
// kernel on v.pin, whose block partials follow the step kernel's.
constexpr int TILE_WAVES_DEFAULT = 32;
// Test hook: make every tensor-copy wait of the single-lattice kernels run
// out (enable) after limit_ns, or restore normal copies; the limit applies to
// launches enqueued from then on either way.
int tma_inject_timeout(int enable, long long limit_ns);
int tiled_grid_blocks(int nx, int ny, int nz, int sizeof_t, int waves = TILE_WAVES_DEFAULT);
// block partials a tiled measuring launch writes (with or without windings)
int tiled_measure_blocks(int nx, int ny, int nz, int sizeof_t, int waves, bool windings);
// status: the caller's device status word, which a kernel whose wait for a
// tensor copy into shared memory ran out sets to U1U1_ERR_TIMEOUT (the kernel
// then finishes on stale data); required.
template <typename T>
cudaError_t launch_tiled(int mode, const LatticeView<T>& v, const Coef<T>& c, const MeasureOut& mo,
                         cudaStream_t st, int waves, int* status);

// Windings kernel (k_wind.cu): face bytes, optional int8 windings and one
// block partial (counts only) per block.
int wind_grid_blocks(int nx, int ny, int nz);
template <typename T>
cudaError_t launch_windings(const PosView<T>& v, T dx, BlockPartial* part, uint8_t* faces, int8_t* windings,
                            cudaStream_t st);

// ---------------------------------------------------------------------------
// Ensembles: per-box tables for the batched kernels.
// ---------------------------------------------------------------------------
template <typename T>
struct EnsBox {
  T* pos[2][U1U1_NPOS];
  T* mom[U1U1_NMOM];
  int nx, ny, nz;
  int gx, gy, lz, gz, ntiles;  // tile grid of this box
  long long coef0;             // first row of this box in the coefficient table
  const TmaPlan* tma[2];       // tensor maps of each position buffer (device memory)
  T dx;                        // lattice spacing (windings)
};
struct EnsDyn {                // device-side step index, current buffer and records written
  long long n;
  long long rec;
  int cur;
  int pad;
};
// Detection resources of one ensemble box (the scratch of its handle) and
// the grids of its passes, which are those of a single lattice of the same
// shape, so that a box's records equal those of the box stepped alone.
struct EnsDet {
  BlockPartial* part;        // measuring partials, then windings partials, then stage slots
  uint8_t* faces;            // 2 V face bytes
  uint32_t* masks;           // 2 x cell_mask_words pierced-cell words
  CellPartial* counts;       // one overlap partial, accumulated atomically
  unsigned long long* ge4;   // census counters
  RawRecord* ring;           // the handle's record ring (RING_CAP entries)
  int mgx, mgy, mgz, mlz;    // measuring tile grid (the default chunking)
  int wtx, wty, wtz, wlz;    // windings window grid
  int nmeas, nwind;          // block partials of each pass
  int words;                 // mask words per row
  int tol;                   // overlap tolerance
  int nx, ny, nz;
};
// index of the entry of a prefix table pre[0..n] (pre[0] = 0 <= r < pre[n])
// that holds r: the largest i < n with pre[i] <= r
__device__ __forceinline__ int ens_list_index(const long long* pre, int n, long long r) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (pre[mid] <= r) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}
struct EnsSched {              // one run's work-item order
  const int* order;            // sorted position -> box (steps descending)
  const int* steps;            // steps of each box (box index)
  const long long* box_prefix; // nboxes + 1 cumulative tiles in sorted order
  const long long* step_off;   // smax + 1 cumulative items before each step
  int nboxes, smax;
  long long total;
};
constexpr int ENS_LZ = 32;     // default z-chunk of an ensemble work item

// Each box's two step views (input buffer 0 and 1) for ensembles of up to
// ENS_VIEW_MAX boxes, passed to the ensemble step kernels as one kernel
// parameter.  The tile body then reads a box's field pointers from the
// parameter bank, as a single lattice's kernel does, instead of from a
// per-thread copy, which the copy plan's run-time field index keeps in local
// memory (measured: a 1024^3 box stepped 4% faster).  Larger ensembles use
// the per-thread copy.  56 x 2 views of 256 bytes stay inside the 32 KB
// kernel-parameter limit.
constexpr int ENS_VIEW_MAX = 56;
template <typename T>
struct EnsViews {
  LatticeView<T> v[ENS_VIEW_MAX][2];
};

int ens_tile_grid(int nx, int ny, int nz, int* gx, int* gy, int* lz, int* gz, int item_lz = ENS_LZ);
// kstart (nullable): per box, the run step its first item of this launch
// advances (a launch covering a segment of a run between detection steps);
// use_tma: interior tiles' ring slots filled by tensor copies
// views (host memory, nullable): the boxes' step views when the ensemble
// has at most ENS_VIEW_MAX boxes
template <typename T>
cudaError_t launch_ens_persistent(const EnsBox<T>* boxes, const EnsDyn* dyn, const Coef<T>* coef, const EnsSched& sc,
                                  const int* kstart, unsigned long long* ticket, unsigned* done, int* err,
                                  long long limit_ns, int inject, int use_tma, const EnsViews<T>* views,
                                  cudaStream_t st);
template <typename T>
cudaError_t launch_ens_step(const EnsBox<T>* boxes, const EnsDyn* dyn, const Coef<T>* coef, const EnsSched& sc,
                            int k, long long items, const EnsViews<T>* views, cudaStream_t st);
// de: detection cadence of the run (0: none), for the record counters
cudaError_t launch_ens_advance(EnsDyn* dyn, const int* steps, int nboxes, int de, cudaStream_t st);

// Batched detection at run step k over the boxes list[0..nlist) (every one
// of them detects at k); pre: per-list-entry prefix sums of the launch's
// work items.  The measuring step (writes step k and the diagnostic sums),
// the windings of its input positions, cells and overlap, the finalize into
// each box's record ring.
template <typename T>
cudaError_t launch_ens_measure(const EnsBox<T>* boxes, const EnsDet* det, const EnsDyn* dyn, const Coef<T>* coef,
                               const int* list, const long long* pre, int nlist, long long items, int k,
                               const EnsViews<T>* views, cudaStream_t st);
template <typename T>
cudaError_t launch_ens_windings(const EnsBox<T>* boxes, const EnsDet* det, const EnsDyn* dyn, const int* list,
                                const long long* pre, int nlist, long long items, int k, cudaStream_t st);
// pre_c: prefix sums of each box's mask words (the cell pass: one warp per
// word of 32 cells), pre_o: of its groups of 32 mask words (the overlap)
cudaError_t launch_ens_cells(const EnsDet* det, const int* list, const long long* pre_c, const long long* pre_o,
                             int nlist, long long items_c, long long items_o, cudaStream_t st);
cudaError_t launch_ens_finalize(const EnsDet* det, const EnsDyn* dyn, const int* list, int nlist, int k, int de,
                                bool stage, cudaStream_t st);
void tiled_grid_dims(int nx, int ny, int nz, int sizeof_t, int waves, int* gx, int* gy, int* gz, int* lz);
void wind_grid_dims(int nx, int ny, int nz, int* tx, int* ty, int* tz, int* lz);

// Cells and overlap from face bytes; masks holds 2 * cell_mask_words words.
int cells_grid_blocks();
size_t cell_mask_words(int nx, int ny, int nz);
// mpq (optional, cell_mask_words words): the p-anchored bound-state cells.
// ge4 (optional, 2 counters): cells of value >= 4 per sector.
cudaError_t launch_cells(const uint8_t* faces, int nx, int ny, int nz, int tol, uint8_t* cell_p,
                         uint8_t* cell_q, uint32_t* masks, CellPartial* part, cudaStream_t st,
                         uint32_t* mpq = nullptr, unsigned long long* ge4 = nullptr);

// Connected components of the bound-state cells (robust method).
struct SegCounts {
  unsigned long long n_cells, n_components, n_segments, sum_len, largest;
  int err;  // nonzero when a union-find loop hit its iteration limit
  int pad;
};
cudaError_t launch_segments(const uint32_t* mpq, int nx, int ny, int nz, int min_cells, int* label, int* size,
                            SegCounts* counts, cudaStream_t st);

// The FP32 link-phase routine on n values (check entry point).
cudaError_t launch_link_phase(const float* th, float* sn, float* cs, long long n, cudaStream_t st);
cudaError_t launch_link_phase64(const double* th, double* sn, double* cs, long long n, cudaStream_t st);
cudaError_t launch_edge_phase(const float* re, const float* im, float* out, long long n, cudaStream_t st);

// Merge partials into a record.  part must have room for nblocks +
// FIN_STAGE_BLOCKS entries: above FIN_STAGE_MIN partials a first stage of
// FIN_STAGE_BLOCKS CTAs merges contiguous slices of them into the entries
// after the last one (fixed slices and order: the result is reproducible).
constexpr int FIN_STAGE_BLOCKS = 128;
constexpr int FIN_STAGE_MIN = 2048;
cudaError_t launch_finalize(BlockPartial* part, int nblocks, const CellPartial* cpart,
                            int ncblocks, RawRecord* rec, long long n, int has_diag, int has_gauss,
                            int has_strings, int tol, cudaStream_t st,
                            const unsigned long long* ge4 = nullptr);

}  // namespace u1u1
