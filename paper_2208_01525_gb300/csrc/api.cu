// C ABI of libu1u1 (include/u1u1.h): parameter handling, lattice handles,
// the step loop, detection and diagnostics orchestration, record ring,
// host epilogue of Sec. III.A (Eqs. 31-37) and checkpoint I/O.
#include <cuda.h>
#include <cuda_runtime.h>
#include <stdint.h>
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <string>

#include "../../include/u1u1.h"
#include "host_internal.h"
#include "state_copy.cuh"
#include "u1u1_internal.cuh"

using namespace u1u1;

namespace u1u1 {

thread_local std::string g_last_error;

int fail(int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return code;
}

int cuda_fail(cudaError_t e, const char* where) {
  return fail(e == cudaErrorMemoryAllocation ? U1U1_ERR_OUT_OF_MEMORY : U1U1_ERR_CUDA, "%s: %s", where,
              cudaGetErrorString(e));
}

}  // namespace u1u1

namespace {
constexpr double TWO_PI = 6.283185307179586476925286766559;
// z-chunk targets the autotuner tries for the tiled kernel
// (more waves: shorter z-chunks, so neighbouring tiles stay closer in z
// and their halo rows are still in L2; fewer: fewer prologue planes)
constexpr int AUTOTUNE_WAVES[] = {8, 16, 32, 64, 128, 256};
constexpr int N_AUTOTUNE_WAVES = (int)(sizeof(AUTOTUNE_WAVES) / sizeof(AUTOTUNE_WAVES[0]));
}  // namespace



// ---------------------------------------------------------------------------
// parameters and coefficients
// ---------------------------------------------------------------------------

extern "C" const char* u1u1_version(void) { return "0.1.0"; }

extern "C" const char* u1u1_last_error(void) { return g_last_error.c_str(); }

extern "C" int u1u1_params_default(u1u1_params* p) {
  if (!p) return fail(U1U1_ERR_INVALID_ARG, "params pointer is NULL");
  memset(p, 0, sizeof(*p));
  p->nx = p->ny = p->nz = 64;
  p->dx = 0.5;
  p->deta = 0.1;
  p->eta0 = 1.0;
  p->m = 0.5;
  p->eta_ref = 1.0;
  p->beta = 1.0;
  p->alpha = 2.0;
  p->lambda_p = p->lambda_q = 2.0;
  p->e_p = p->e_q = 1.0;
  p->sigma_p = p->sigma_q = 1.0;
  p->kappa = 0.9;
  p->seed = 1;
  p->precision = U1U1_FP32;
  return U1U1_OK;
}

extern "C" int u1u1_check_params(const u1u1_params* p) {
  if (!p) return fail(U1U1_ERR_INVALID_ARG, "params pointer is NULL");
  if (p->nx < 4 || p->ny < 4 || p->nz < 4)
    return fail(U1U1_ERR_INVALID_ARG, "lattice sides must be >= 4 (got %d x %d x %d)", p->nx, p->ny, p->nz);
  if (p->nx % 4 != 0) return fail(U1U1_ERR_INVALID_ARG, "nx must be a multiple of 4 (got %d)", p->nx);
  if ((double)p->nx * p->ny * p->nz > 9.0e18)
    return fail(U1U1_ERR_INVALID_ARG, "lattice too large");
  if (!(p->dx > 0.0) || !isfinite(p->dx)) return fail(U1U1_ERR_INVALID_ARG, "dx must be > 0");
  if (!(p->deta > 0.0) || !isfinite(p->deta)) return fail(U1U1_ERR_INVALID_ARG, "deta must be > 0");
  if (!(p->m >= 0.0 && p->m < 1.0)) return fail(U1U1_ERR_INVALID_ARG, "m must be in [0, 1)");
  if (p->m != 0.0 && !(p->eta0 > 0.0)) return fail(U1U1_ERR_INVALID_ARG, "eta0 must be > 0 in an expanding background");
  if (!(p->eta_ref > 0.0) || !isfinite(p->eta_ref)) return fail(U1U1_ERR_INVALID_ARG, "eta_ref must be > 0");
  if (!isfinite(p->beta) || !isfinite(p->alpha)) return fail(U1U1_ERR_INVALID_ARG, "beta and alpha must be finite");
  if (!(p->e_p > 0.0) || !(p->e_q > 0.0)) return fail(U1U1_ERR_INVALID_ARG, "e_p and e_q must be > 0");
  if (!isfinite(p->lambda_p) || !isfinite(p->lambda_q) || !isfinite(p->kappa) || !isfinite(p->sigma_p) ||
      !isfinite(p->sigma_q))
    return fail(U1U1_ERR_INVALID_ARG, "couplings must be finite");
  if (p->precision != U1U1_FP32 && p->precision != U1U1_FP64)
    return fail(U1U1_ERR_INVALID_ARG, "precision must be U1U1_FP32 or U1U1_FP64");
  return U1U1_OK;
}

void u1u1::coeffs(const u1u1_params* p, int64_t n, double out[6]) {
  double eta = p->eta0 + (double)n * p->deta;
  double pm = (p->m == 0.0) ? 0.0 : p->m / (1.0 - p->m);
  double a = (pm == 0.0) ? 1.0 : pow(eta / p->eta_ref, pm);
  double c = pow(a, 2.0 * p->beta);
  double delta = 0.5 * p->alpha * pm * p->deta / eta;
  double omega = delta * (1.0 - p->beta);
  out[0] = eta;
  out[1] = a;
  out[2] = c;
  out[3] = delta;
  out[4] = omega;
  out[5] = c * (1.0 + delta) / (1.0 + omega);
}

extern "C" int u1u1_coefficients(const u1u1_params* p, int64_t n, double out[6]) {
  int rc = u1u1_check_params(p);
  if (rc) return rc;
  if (!out) return fail(U1U1_ERR_INVALID_ARG, "out is NULL");
  double eta = p->eta0 + (double)n * p->deta;
  if (p->m != 0.0 && !(eta > 0.0)) return fail(U1U1_ERR_INVALID_ARG, "eta_n <= 0 at step %lld", (long long)n);
  coeffs(p, n, out);
  return U1U1_OK;
}

extern "C" size_t u1u1_field_bytes(const u1u1_params* p) {
  if (!p || p->nx <= 0 || p->ny <= 0 || p->nz <= 0) return 0;
  size_t es = p->precision == U1U1_FP64 ? 8 : 4;
  return (size_t)p->nx * p->ny * p->nz * es;
}

extern "C" void u1u1_abi_sizes(size_t out[4]) {
  if (!out) return;
  out[0] = sizeof(u1u1_params);
  out[1] = sizeof(u1u1_buffers);
  out[2] = sizeof(u1u1_strings);
  out[3] = sizeof(u1u1_diag);
}

template <typename T>
Coef<T> u1u1::make_coef(const u1u1_params* p, int64_t n) {
  double cf[6];
  coeffs(p, n, cf);
  const double c = cf[2], delta = cf[3], omega = cf[4];
  const double dx = p->dx, deta = p->deta;
  const double lam[2] = {p->lambda_p, p->lambda_q};
  const double e[2] = {p->e_p, p->e_q};
  const double sig[2] = {p->sigma_p, p->sigma_q};
  Coef<T> k;
  const double kPb = deta / (1.0 + delta);
  k.kPa = (T)((1.0 - delta) / (1.0 + delta));
  k.kP1 = (T)(kPb / (dx * dx));
  for (int s = 0; s < 2; ++s) k.kgl[s] = (T)(kPb * c * 0.5 * lam[s]);
  k.kgk = (T)(kPb * c * p->kappa);
  const double kEb = deta / (1.0 + omega);
  k.kEa = (T)((1.0 - omega) / (1.0 + omega));
  k.kE1 = (T)(kEb / (dx * dx));
  for (int s = 0; s < 2; ++s) k.kE2[s] = (T)(kEb * 2.0 * e[s] * e[s] * c / dx);
  k.deta = (T)deta;
  k.dx = (T)dx;
  k.inv_dx2 = (T)(1.0 / (dx * dx));
  k.inv_dx = (T)(1.0 / dx);
  for (int s = 0; s < 2; ++s) {
    k.el_f[s] = (T)(1.0 / (2.0 * e[s] * e[s] * c));
    k.mag_f[s] = (T)(1.0 / (2.0 * e[s] * e[s] * c * dx * dx));
    k.lam4[s] = (T)(0.25 * lam[s]);
    k.sig2[s] = (T)(sig[s] * sig[s]);
  }
  k.cV = (T)c;
  k.kappa = (T)p->kappa;
  double etam = p->eta0 + (double)(n - 1) * p->deta;
  double ct = 0.0;
  if (p->m == 0.0 || etam > 0.0) {
    double cm[6];
    coeffs(p, n - 1, cm);
    ct = cm[5];
  }
  for (int s = 0; s < 2; ++s) k.qG[s] = (T)(2.0 * e[s] * e[s] * ct);
  return k;
}

// ---------------------------------------------------------------------------
// handle lifecycle
// ---------------------------------------------------------------------------

static int check_buffers(const u1u1_params* p, const u1u1_buffers* b) {
  if (!b) return fail(U1U1_ERR_BAD_BUFFER, "buffers pointer is NULL");
  for (int k = 0; k < 2; ++k)
    for (int f = 0; f < U1U1_NPOS; ++f) {
      if (!b->pos[k][f]) return fail(U1U1_ERR_BAD_BUFFER, "pos[%d][%d] is NULL", k, f);
      if ((uintptr_t)b->pos[k][f] % 256 != 0) return fail(U1U1_ERR_BAD_BUFFER, "pos[%d][%d] is not 256-byte aligned", k, f);
    }
  for (int f = 0; f < U1U1_NMOM; ++f) {
    if (!b->mom[f]) return fail(U1U1_ERR_BAD_BUFFER, "mom[%d] is NULL", f);
    if ((uintptr_t)b->mom[f] % 256 != 0) return fail(U1U1_ERR_BAD_BUFFER, "mom[%d] is not 256-byte aligned", f);
  }
  (void)p;
  return U1U1_OK;
}

void u1u1::lattice_free_scratch(u1u1_lattice* h) {
  if (!h) return;
  dev_free(h->faces);
  dev_free(h->ge4);
  dev_free(h->masks);
  dev_free(h->mpq);
  dev_free(h->seg_label);
  dev_free(h->seg_size);
  dev_free(h->seg_counts);
  dev_free(h->partials);
  dev_free(h->cpartials);
  dev_free(h->ring);
  dev_free(h->scratch_rec);
  dev_free(h->tma_status);
  host_free(h->host_rec);
  host_free(h->host_status);
}

int u1u1::lattice_create(const u1u1_params* p, const u1u1_buffers* b, u1u1_lattice** out) {
  int rc = u1u1_check_params(p);
  if (rc) return rc;
  if (!out) return fail(U1U1_ERR_INVALID_ARG, "out is NULL");
  rc = check_buffers(p, b);
  if (rc) return rc;
  u1u1_lattice* h = (u1u1_lattice*)calloc(1, sizeof(u1u1_lattice));
  if (!h) return fail(U1U1_ERR_OUT_OF_MEMORY, "host allocation failed");
  h->p = *p;
  h->V = (size_t)p->nx * p->ny * p->nz;
  h->esize = p->precision == U1U1_FP64 ? 8 : 4;
  memcpy(h->pos, b->pos, sizeof(h->pos));
  memcpy(h->mom, b->mom, sizeof(h->mom));
  h->kernel = U1U1_KERNEL_AUTO;
  h->overlap_tol = 1;
  h->tile_waves = TILE_WAVES_DEFAULT;
  h->npartials = simple_grid_blocks();
  for (int w : AUTOTUNE_WAVES) {  // room for every grid the tuner may choose
    const int tb = tiled_measure_blocks(p->nx, p->ny, p->nz, (int)h->esize, w, true);
    if (tb > h->npartials) h->npartials = tb;
  }
  h->ncpartials = cells_grid_blocks();
  cudaError_t e = cudaSuccess;
  if (e == cudaSuccess) e = dev_alloc(&h->faces, 2 * h->V);
  if (e == cudaSuccess) e = dev_alloc(&h->ge4, 2 * sizeof(unsigned long long));
  if (e == cudaSuccess)
    e = dev_alloc(&h->masks, 2 * sizeof(uint32_t) * cell_mask_words(p->nx, p->ny, p->nz));
  // block partials, plus the finalize's first-stage slots after the last one
  if (e == cudaSuccess)
    e = dev_alloc(&h->partials, sizeof(BlockPartial) * (size_t)(h->npartials + FIN_STAGE_BLOCKS));
  if (e == cudaSuccess) e = dev_alloc(&h->cpartials, sizeof(CellPartial) * (size_t)h->ncpartials);
  if (e == cudaSuccess) e = dev_alloc(&h->ring, sizeof(RawRecord) * RING_CAP);
  if (e == cudaSuccess) e = dev_alloc(&h->scratch_rec, sizeof(RawRecord));
  if (e == cudaSuccess) e = host_alloc(&h->host_rec, sizeof(RawRecord) * RING_CAP);
  if (e == cudaSuccess) e = dev_alloc(&h->tma_status, sizeof(int));
  if (e == cudaSuccess) e = host_alloc(&h->host_status, sizeof(int));
  if (e != cudaSuccess) {
    lattice_free_scratch(h);
    free(h);
    cudaGetLastError();
    return fail(e == cudaErrorMemoryAllocation ? U1U1_ERR_OUT_OF_MEMORY : U1U1_ERR_CUDA,
                "scratch allocation: %s", cudaGetErrorString(e));
  }
  *out = h;
  return U1U1_OK;
}

template <typename T>
static LatticeView<T> view(const u1u1_lattice* h) {
  LatticeView<T> v;
  for (int f = 0; f < U1U1_NPOS; ++f) {
    v.pin[f] = (const T*)h->pos[h->cur][f];
    v.pout[f] = (T*)h->pos[1 - h->cur][f];
  }
  for (int f = 0; f < U1U1_NMOM; ++f) v.mom[f] = (T*)h->mom[f];
  v.nx = h->p.nx;
  v.ny = h->p.ny;
  v.nz = h->p.nz;
  return v;
}

template <typename T>
static cudaError_t init_fields_t(u1u1_lattice* h, cudaStream_t st) {
  LatticeView<T> v = view<T>(h);
  T* pos1[U1U1_NPOS];
  for (int f = 0; f < U1U1_NPOS; ++f) pos1[f] = (T*)h->pos[1][f];
  return launch_init<T>(v, pos1, h->p.seed, h->p.sigma_p, h->p.sigma_q, st);
}

cudaError_t u1u1::lattice_init_fields(u1u1_lattice* h, cudaStream_t st) {
  return h->esize == 8 ? init_fields_t<double>(h, st) : init_fields_t<float>(h, st);
}

extern "C" int u1u1_init_lattice(const u1u1_params* p, const u1u1_buffers* b, void* stream,
                                 u1u1_lattice** out) {
  u1u1_lattice* h = nullptr;
  int rc = lattice_create(p, b, &h);
  if (rc) return rc;
  h->cur = 0;
  h->n = 0;
  cudaStream_t st = (cudaStream_t)stream;
  // the handle's status word, cleared on the stream its launches will use
  cudaError_t e = cudaMemsetAsync(h->tma_status, 0, sizeof(int), st);
  if (e == cudaSuccess) e = lattice_init_fields(h, st);
  if (e != cudaSuccess) {
    lattice_free_scratch(h);
    free(h);
    return cuda_fail(e, "initial conditions");
  }
  *out = h;
  return U1U1_OK;
}

extern "C" int u1u1_attach_lattice(const u1u1_params* p, const u1u1_buffers* b, int64_t n, int current,
                                   u1u1_lattice** out) {
  if (current != 0 && current != 1) return fail(U1U1_ERR_INVALID_ARG, "current must be 0 or 1");
  u1u1_lattice* h = nullptr;
  int rc = lattice_create(p, b, &h);
  if (rc) return rc;
  h->cur = current;
  h->n = n;
  // no stream is given: clear the status word and wait for it, so that
  // launches on any stream see it cleared
  cudaError_t e = cudaMemset(h->tma_status, 0, sizeof(int));
  if (e == cudaSuccess) e = cudaStreamSynchronize(cudaStreamLegacy);
  if (e != cudaSuccess) {
    lattice_destroy(h);
    return cuda_fail(e, "status word");
  }
  *out = h;
  return U1U1_OK;
}

void u1u1::lattice_destroy(u1u1_lattice* h) {
  if (!h) return;
  lattice_free_scratch(h);
  free(h);
}

extern "C" void u1u1_destroy(u1u1_lattice* h) {
  if (!h || h->ensemble_box) return;  // a box handle is released with its ensemble
  lattice_destroy(h);
}

extern "C" int u1u1_current(const u1u1_lattice* h, int64_t* n, int* current) {
  if (!h) return fail(U1U1_ERR_INVALID_ARG, "handle is NULL");
  if (n) *n = h->n;
  if (current) *current = h->cur;
  return U1U1_OK;
}

extern "C" int u1u1_set_kernel(u1u1_lattice* h, int kernel) {
  if (!h) return fail(U1U1_ERR_INVALID_ARG, "handle is NULL");
  if (kernel < U1U1_KERNEL_AUTO || kernel > U1U1_KERNEL_TILED) return fail(U1U1_ERR_INVALID_ARG, "unknown kernel %d", kernel);
  h->kernel = kernel;
  return U1U1_OK;
}

extern "C" int u1u1_set_tile_waves(u1u1_lattice* h, int waves) {
  if (!h) return fail(U1U1_ERR_INVALID_ARG, "handle is NULL");
  bool known = false;
  for (int w : AUTOTUNE_WAVES) known = known || w == waves;
  if (!known) return fail(U1U1_ERR_INVALID_ARG, "wave target %d is not one the tuner tries", waves);
  h->tile_waves = waves;
  return U1U1_OK;
}

extern "C" int u1u1_inject_copy_timeout(int enable, int64_t limit_ns) {
  if (limit_ns < 1000) return fail(U1U1_ERR_INVALID_ARG, "wait limit must be >= 1000 ns");
  tma_inject_timeout(enable, (long long)limit_ns);
  return U1U1_OK;
}

extern "C" int u1u1_get_kernel(const u1u1_lattice* h, int* kernel) {
  if (!h || !kernel) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  *kernel = h->kernel;
  return U1U1_OK;
}

extern "C" int u1u1_set_overlap_tol(u1u1_lattice* h, int tol) {
  if (!h) return fail(U1U1_ERR_INVALID_ARG, "handle is NULL");
  if (tol < 0 || tol > 1) return fail(U1U1_ERR_INVALID_ARG, "overlap tolerance must be 0 or 1");
  h->overlap_tol = tol;
  return U1U1_OK;
}

// ---------------------------------------------------------------------------
// stepping and measuring
// ---------------------------------------------------------------------------

static bool use_tiled(const u1u1_lattice* h) { return h->kernel != U1U1_KERNEL_SIMPLE; }

// z-chunking of a tiled launch: the tuned one for plain steps; the measuring
// passes keep the default, since their block partials and finalize grow
// with the number of CTAs (at 1024^3 a 256-wave chunking that made the plain
// step 0.2 ms faster made a detection step 4.6 ms slower)
static int launch_waves(const u1u1_lattice* h, int mode) {
  return (mode & MODE_MEASURE) ? TILE_WAVES_DEFAULT : h->tile_waves;
}

template <typename T>
static cudaError_t run_kernel(u1u1_lattice* h, int mode, const MeasureOut& mo, cudaStream_t st) {
  LatticeView<T> v = view<T>(h);
  Coef<T> c = make_coef<T>(&h->p, h->n);
  if (use_tiled(h)) return launch_tiled<T>(mode, v, c, mo, st, launch_waves(h, mode), h->tma_status);
  return launch_simple<T>(mode, v, c, mo, st);
}

// block partials of a measuring launch: the step kernel's, plus (tiled
// path, when windings are taken) the windings kernel's
static int measure_blocks(const u1u1_lattice* h, bool windings) {
  return use_tiled(h) ? tiled_measure_blocks(h->p.nx, h->p.ny, h->p.nz, (int)h->esize,
                                             launch_waves(h, MODE_MEASURE), windings)
                      : simple_grid_blocks();
}

static cudaError_t dispatch(u1u1_lattice* h, int mode, const MeasureOut& mo, cudaStream_t st) {
  return h->esize == 8 ? run_kernel<double>(h, mode, mo, st) : run_kernel<float>(h, mode, mo, st);
}

// Windings, face bytes and counts of the current positions for a
// standalone detection (Sec. III.A): on the tiled path the windings kernel
// alone, which reads the ten position fields once and neither the momenta
// nor any step arithmetic; the simple kernel family takes its own windings
// in a measuring pass.  Returns the number of block partials written.
template <typename T>
static cudaError_t windings_t(u1u1_lattice* h, int8_t* windings, cudaStream_t st) {
  PosView<T> pv;
  for (int f = 0; f < U1U1_NPOS; ++f) pv.pos[f] = (const T*)h->pos[h->cur][f];
  pv.nx = h->p.nx;
  pv.ny = h->p.ny;
  pv.nz = h->p.nz;
  return launch_windings<T>(pv, (T)h->p.dx, h->partials, h->faces, windings, st);
}

static cudaError_t strings_pass(u1u1_lattice* h, int8_t* windings, cudaStream_t st, int* nblocks) {
  if (!use_tiled(h)) {
    *nblocks = simple_grid_blocks();
    MeasureOut mo{h->partials, h->faces, windings};
    return dispatch(h, MODE_MEASURE, mo, st);
  }
  *nblocks = wind_grid_blocks(h->p.nx, h->p.ny, h->p.nz);
  return h->esize == 8 ? windings_t<double>(h, windings, st) : windings_t<float>(h, windings, st);
}

extern "C" int u1u1_step(u1u1_lattice* h, int nsteps, int detect_every, void* stream) {
  const NvtxRange range("u1u1_step");
  if (!h) return fail(U1U1_ERR_INVALID_ARG, "handle is NULL");
  if (nsteps < 0) return fail(U1U1_ERR_INVALID_ARG, "nsteps must be >= 0");
  if (detect_every < 0) return fail(U1U1_ERR_INVALID_ARG, "detect_every must be >= 0");
  if (h->p.m != 0.0) {
    double eta_last = h->p.eta0 + (double)(h->n + nsteps) * h->p.deta;
    double eta_first = h->p.eta0 + (double)h->n * h->p.deta;
    if (!(eta_first > 0.0) || !(eta_last > 0.0)) return fail(U1U1_ERR_INVALID_ARG, "conformal time must stay > 0");
  }
  cudaStream_t st = (cudaStream_t)stream;
  for (int k = 0; k < nsteps; ++k) {
    bool det = detect_every > 0 && (h->n % detect_every) == 0;
    MeasureOut mo{nullptr, nullptr, nullptr};
    int mode = MODE_WRITE;
    if (det) {
      mode |= MODE_MEASURE;
      mo.partial = h->partials;
      mo.faces = h->faces;
    }
    cudaError_t e = dispatch(h, mode, mo, st);
    if (e != cudaSuccess) return cuda_fail(e, "step kernel");
    if (det) {
      e = launch_cells(h->faces, h->p.nx, h->p.ny, h->p.nz, h->overlap_tol, nullptr, nullptr, h->masks,
                       h->cpartials, st, nullptr, h->ge4);
      if (e != cudaSuccess) return cuda_fail(e, "cell overlap kernel");
      RawRecord* slot = h->ring + (h->rec_written % RING_CAP);
      e = launch_finalize(h->partials, measure_blocks(h, true), h->cpartials, h->ncpartials, slot, (long long)h->n,
                          1, 0, 1, h->overlap_tol, st, h->ge4);
      if (e != cudaSuccess) return cuda_fail(e, "finalize kernel");
      h->rec_written++;
    }
    h->cur ^= 1;
    h->n++;
  }
  return U1U1_OK;
}

// Cooling (Eqs. 27-30) reuses the step kernel: with the old momenta weighted
// by zero, a kick of size dt equal to the flow's right-hand side, and a drift
// of weight one, a leapfrog step is exactly one forward-Euler cooling step.
template <typename T>
static Coef<T> make_cool_coef(const u1u1_params* p, double dt) {
  Coef<T> k;
  memset(&k, 0, sizeof(k));
  const double dx = p->dx;
  const double lam[2] = {p->lambda_p, p->lambda_q};
  const double e[2] = {p->e_p, p->e_q};
  const double sig[2] = {p->sigma_p, p->sigma_q};
  k.kPa = (T)0;
  k.kP1 = (T)(dt / (dx * dx));
  for (int s = 0; s < 2; ++s) k.kgl[s] = (T)(dt * 0.5 * lam[s]);
  k.kgk = (T)0;  // no kappa term in the cooling flow
  k.kEa = (T)0;
  k.kE1 = (T)(dt / (dx * dx));
  for (int s = 0; s < 2; ++s) k.kE2[s] = (T)(dt * 2.0 * e[s] * e[s] / dx);
  k.deta = (T)1;
  k.dx = (T)dx;
  for (int s = 0; s < 2; ++s) k.sig2[s] = (T)(sig[s] * sig[s]);
  return k;
}

template <typename T>
static cudaError_t cool_t(u1u1_lattice* h, double dt, int nsteps, cudaStream_t st) {
  const Coef<T> c = make_cool_coef<T>(&h->p, dt);
  const MeasureOut mo{nullptr, nullptr, nullptr};
  for (int k = 0; k < nsteps; ++k) {
    LatticeView<T> v = view<T>(h);
    cudaError_t e = use_tiled(h) ? launch_tiled<T>(MODE_WRITE, v, c, mo, st, h->tile_waves, h->tma_status)
                                 : launch_simple<T>(MODE_WRITE, v, c, mo, st);
    if (e != cudaSuccess) return e;
    h->cur ^= 1;
  }
  const size_t bytes = h->V * h->esize;
  for (int f = 0; f < U1U1_NMOM; ++f) {
    cudaError_t e = cudaMemsetAsync(h->mom[f], 0, bytes, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

extern "C" int u1u1_cool(u1u1_lattice* h, double dt, int nsteps, void* stream) {
  if (!h) return fail(U1U1_ERR_INVALID_ARG, "handle is NULL");
  if (!(dt > 0.0) || !isfinite(dt)) return fail(U1U1_ERR_INVALID_ARG, "dt must be > 0");
  if (nsteps < 0) return fail(U1U1_ERR_INVALID_ARG, "nsteps must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e = h->esize == 8 ? cool_t<double>(h, dt, nsteps, st) : cool_t<float>(h, dt, nsteps, st);
  if (e != cudaSuccess) return cuda_fail(e, "cooling");
  return U1U1_OK;
}

extern "C" int u1u1_set_params(u1u1_lattice* h, const u1u1_params* p, int64_t n) {
  if (!h) return fail(U1U1_ERR_INVALID_ARG, "handle is NULL");
  if (h->ensemble_box)
    return fail(U1U1_ERR_STATE, "the handle is a box of an ensemble, whose coefficient tables hold its parameters");
  int rc = u1u1_check_params(p);
  if (rc) return rc;
  if (p->nx != h->p.nx || p->ny != h->p.ny || p->nz != h->p.nz || p->precision != h->p.precision)
    return fail(U1U1_ERR_INVALID_ARG, "lattice sides and precision must stay the same");
  u1u1_params q = *p;
  q.seed = h->p.seed;
  h->p = q;
  h->n = n;
  return U1U1_OK;
}

// host epilogue (Sec. III.A): raw sums and counts -> estimators
static double sqrt_ratio(double num, double den) {
  if (den == 0.0) return INFINITY;
  double r = num / den;
  return r >= 0.0 ? sqrt(r) : NAN;
}

void u1u1::to_strings(const u1u1_params* p, const RawRecord& r, u1u1_strings* s) {
  memset(s, 0, sizeof(*s));
  double cf[6];
  coeffs(p, r.n, cf);
  s->n = r.n;
  s->eta = cf[0];
  s->n_p = r.cnt[C_NP];
  s->n_q = r.cnt[C_NQ];
  s->nonzero_p = r.cnt[C_NZP];
  s->nonzero_q = r.cnt[C_NZQ];
  s->n_pq_plaq = r.cnt[C_NPQ_PLAQ];
  s->n_pq_cell = r.cells[0];
  s->n_pq_cell_q = r.cells[1];
  s->n_flagged = r.cnt[C_FLAGGED];
  s->max_abs_w = (int32_t)r.cnt[C_MAXW];
  s->overlap_tol = r.tol;
  s->n_w2_p = r.cnt[C_W2P];
  s->n_w2_q = r.cnt[C_W2Q];
  s->n_cells_ge4_p = r.cells[2];
  s->n_cells_ge4_q = r.cells[3];
  const double dx = p->dx;
  const double vol = (double)p->nx * p->ny * p->nz * dx * dx * dx;
  s->L_pq = dx * (double)s->n_pq_cell;
  s->L_p = dx * (double)s->n_p - s->L_pq;
  s->L_q = dx * (double)s->n_q - s->L_pq;
  double tot = s->L_p + s->L_q + s->L_pq;
  s->xi_p = sqrt_ratio(vol, s->L_p);
  s->xi_q = sqrt_ratio(vol, s->L_q);
  s->xi_pq = sqrt_ratio(vol, s->L_pq);
  s->xi_w = sqrt_ratio(vol, tot);
  s->f_total = tot != 0.0 ? s->L_pq / tot : NAN;
  s->f_p = s->L_p != 0.0 ? s->L_pq / s->L_p : NAN;
}

static void to_diag(const u1u1_params* p, const RawRecord& r, u1u1_diag* d) {
  memset(d, 0, sizeof(*d));
  double cf[6];
  coeffs(p, r.n, cf);
  d->n = r.n;
  d->eta = cf[0];
  d->a = cf[1];
  d->kin_p = r.sum[S_KIN_P];
  d->kin_q = r.sum[S_KIN_Q];
  d->grad_p = r.sum[S_GRAD_P];
  d->grad_q = r.sum[S_GRAD_Q];
  d->el_p = r.sum[S_EL_P];
  d->el_q = r.sum[S_EL_Q];
  d->mag_p = r.sum[S_MAG_P];
  d->mag_q = r.sum[S_MAG_Q];
  d->pot = r.sum[S_POT];
  d->vint = r.sum[S_VINT];
  d->pot_p = r.sum[S_POT_P];
  d->pot_q = r.sum[S_POT_Q];
  // the Lagrangian and energy densities are linear in the component
  // densities, so their lattice sums are formed from the component sums
  d->lag = (d->kin_p - d->grad_p + d->el_p - d->mag_p) + (d->kin_q - d->grad_q + d->el_q - d->mag_q) - d->pot;
  d->energy = (d->kin_p + d->grad_p + d->el_p + d->mag_p) + (d->kin_q + d->grad_q + d->el_q + d->mag_q) + d->pot;
  d->rl_num = r.sum[S_RL_NUM];
  d->rl_den = r.sum[S_RL_DEN];
  d->rpq_num = r.sum[S_RPQ_NUM];
  d->rpq_den = r.sum[S_RPQ_DEN];
  const double dx3 = p->dx * p->dx * p->dx;
  const double vol = (double)p->nx * p->ny * p->nz * dx3;
  const double mu = TWO_PI * p->sigma_p * p->sigma_p;
  d->lag_total = dx3 * d->lag;
  d->energy_total = dx3 * d->energy;
  d->xi_l = sqrt_ratio(-mu * vol, d->lag_total);
  d->lag_p = dx3 * ((d->kin_p - d->grad_p + d->el_p - d->mag_p) - d->pot_p);
  d->lag_q = dx3 * ((d->kin_q - d->grad_q + d->el_q - d->mag_q) - d->pot_q);
  d->xi_l_p = sqrt_ratio(-TWO_PI * p->sigma_p * p->sigma_p * vol, d->lag_p);
  d->xi_l_q = sqrt_ratio(-TWO_PI * p->sigma_q * p->sigma_q * vol, d->lag_q);
  d->R_l = d->rl_den != 0.0 ? d->rl_num / d->rl_den : NAN;
  d->v2_l = 2.0 * d->R_l / (1.0 + d->R_l);
  d->R_pq = d->rpq_den != 0.0 ? d->rpq_num / d->rpq_den : NAN;
  d->v2_pq = 2.0 * d->R_pq / (1.0 + d->R_pq);
  d->has_gauss = r.has_gauss;
  if (r.has_gauss) {
    d->gauss_sum_p = r.sum[S_GAUSS_P];
    d->gauss_sum_q = r.sum[S_GAUSS_Q];
    d->charge_sum_p = r.sum[S_CHARGE_P];
    d->charge_sum_q = r.sum[S_CHARGE_Q];
    d->gauss_max_p = r.mx[M_GAUSS_P];
    d->gauss_max_q = r.mx[M_GAUSS_Q];
    d->gauss_rel_p = d->charge_sum_p != 0.0 ? d->gauss_sum_p / d->charge_sum_p : NAN;
    d->gauss_rel_q = d->charge_sum_q != 0.0 ? d->gauss_sum_q / d->charge_sum_q : NAN;
  } else {
    d->gauss_sum_p = d->gauss_sum_q = d->charge_sum_p = d->charge_sum_q = NAN;
    d->gauss_max_p = d->gauss_max_q = d->gauss_rel_p = d->gauss_rel_q = NAN;
  }
  d->phi_min_p = -r.mx[M_NEG_PHIMIN_P];
  d->phi_max_p = r.mx[M_PHIMAX_P];
  d->phi_min_q = -r.mx[M_NEG_PHIMIN_Q];
  d->phi_max_q = r.mx[M_PHIMAX_Q];
  d->nan_count = r.cnt[C_NAN];
}

// A tiled kernel of this handle whose wait for a tensor copy into shared
// memory ran out of time finished on stale data and set the handle's status
// word; read it in the order of `st` (which this synchronises) and report
// it once.  Other handles' words are not touched.
static int check_tma_timeout(u1u1_lattice* h, cudaStream_t st) {
  U1U1_CUDA_TRY(cudaMemcpyAsync(h->host_status, h->tma_status, sizeof(int), cudaMemcpyDeviceToHost, st),
                "status copy");
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  if (*h->host_status == 0) return U1U1_OK;
  U1U1_CUDA_TRY(cudaMemsetAsync(h->tma_status, 0, sizeof(int), st), "status reset");
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  return fail(U1U1_ERR_TIMEOUT, "a tiled kernel's wait for a tensor copy into shared memory ran out (2 s); "
                                "the fields written since may be wrong");
}

static int read_scratch(u1u1_lattice* h, RawRecord* r, cudaStream_t st) {
  U1U1_CUDA_TRY(cudaMemcpyAsync(h->host_rec, h->scratch_rec, sizeof(RawRecord), cudaMemcpyDeviceToHost, st),
                "record copy");
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  *r = h->host_rec[0];
  return check_tma_timeout(h, st);
}

extern "C" int u1u1_detect_strings(u1u1_lattice* h, int overlap_tol, uint8_t* cell_p, uint8_t* cell_q,
                                   int8_t* windings, u1u1_strings* out, void* stream) {
  const NvtxRange range("u1u1_detect_strings");
  if (!h) return fail(U1U1_ERR_INVALID_ARG, "handle is NULL");
  if (overlap_tol < 0 || overlap_tol > 1) return fail(U1U1_ERR_INVALID_ARG, "overlap tolerance must be 0 or 1");
  if (!out) return fail(U1U1_ERR_INVALID_ARG, "out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  int nblocks = 0;
  cudaError_t e = strings_pass(h, windings, st, &nblocks);
  if (e != cudaSuccess) return cuda_fail(e, "windings kernel");
  e = launch_cells(h->faces, h->p.nx, h->p.ny, h->p.nz, overlap_tol, cell_p, cell_q, h->masks, h->cpartials, st,
                   nullptr, h->ge4);
  if (e != cudaSuccess) return cuda_fail(e, "cell overlap kernel");
  e = launch_finalize(h->partials, nblocks, h->cpartials, h->ncpartials, h->scratch_rec, (long long)h->n, 0, 0, 1,
                      overlap_tol, st, h->ge4);
  if (e != cudaSuccess) return cuda_fail(e, "finalize kernel");
  RawRecord r;
  int rc = read_scratch(h, &r, st);
  if (rc) return rc;
  to_strings(&h->p, r, out);
  return U1U1_OK;
}

extern "C" int u1u1_pq_segments(u1u1_lattice* h, int overlap_tol, int min_cells, int32_t* labels_out,
                                u1u1_segments* out, void* stream) {
  const NvtxRange range("u1u1_pq_segments");
  if (!h || !out) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (overlap_tol < 0 || overlap_tol > 1) return fail(U1U1_ERR_INVALID_ARG, "overlap tolerance must be 0 or 1");
  if (min_cells < 0) return fail(U1U1_ERR_INVALID_ARG, "min_cells must be >= 0");
  if (h->V > 2147483647ull) return fail(U1U1_ERR_NOT_SUPPORTED, "component labels need fewer than 2^31 sites");
  cudaStream_t st = (cudaStream_t)stream;
  if (!h->seg_size) {
    cudaError_t e = cudaSuccess;
    if (e == cudaSuccess) e = dev_alloc(&h->mpq, sizeof(uint32_t) * cell_mask_words(h->p.nx, h->p.ny, h->p.nz));
    if (e == cudaSuccess) e = dev_alloc(&h->seg_label, sizeof(int) * h->V);
    if (e == cudaSuccess) e = dev_alloc(&h->seg_size, sizeof(int) * h->V);
    if (e == cudaSuccess) e = dev_alloc(&h->seg_counts, sizeof(SegCounts));
    if (e != cudaSuccess) {
      dev_free(h->mpq);
      dev_free(h->seg_label);
      dev_free(h->seg_size);
      dev_free(h->seg_counts);
      h->mpq = nullptr;
      h->seg_label = h->seg_size = nullptr;
      h->seg_counts = nullptr;
      cudaGetLastError();
      return fail(e == cudaErrorMemoryAllocation ? U1U1_ERR_OUT_OF_MEMORY : U1U1_ERR_CUDA, "segment scratch: %s",
                  cudaGetErrorString(e));
    }
  }
  int nblocks = 0;
  cudaError_t e = strings_pass(h, nullptr, st, &nblocks);
  if (e != cudaSuccess) return cuda_fail(e, "windings kernel");
  e = launch_cells(h->faces, h->p.nx, h->p.ny, h->p.nz, overlap_tol, nullptr, nullptr, h->masks, h->cpartials, st,
                   h->mpq);
  if (e != cudaSuccess) return cuda_fail(e, "cell overlap kernel");
  int* label = labels_out ? (int*)labels_out : h->seg_label;
  e = launch_segments(h->mpq, h->p.nx, h->p.ny, h->p.nz, min_cells, label, h->seg_size, h->seg_counts, st);
  if (e != cudaSuccess) return cuda_fail(e, "segment kernels");
  SegCounts c;
  U1U1_CUDA_TRY(cudaMemcpyAsync(&c, h->seg_counts, sizeof(SegCounts), cudaMemcpyDeviceToHost, st), "segment counts");
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  if (c.err) return fail(U1U1_ERR_CUDA, "component labelling hit its iteration limit");
  memset(out, 0, sizeof(*out));
  out->n = h->n;
  out->overlap_tol = overlap_tol;
  out->min_cells = min_cells;
  out->n_cells = (int64_t)c.n_cells;
  out->n_components = (int64_t)c.n_components;
  out->n_segments = (int64_t)c.n_segments;
  out->largest = (int64_t)c.largest;
  out->L_pq = h->p.dx * (double)c.sum_len;
  out->l_pq = c.n_segments ? out->L_pq / (double)c.n_segments : NAN;
  const double vol = (double)h->V * h->p.dx * h->p.dx * h->p.dx;
  out->xi_pq = sqrt_ratio(vol, out->L_pq);
  return U1U1_OK;
}

extern "C" int u1u1_diagnostics(u1u1_lattice* h, u1u1_diag* out, void* stream) {
  const NvtxRange range("u1u1_diagnostics");
  if (!h) return fail(U1U1_ERR_INVALID_ARG, "handle is NULL");
  if (!out) return fail(U1U1_ERR_INVALID_ARG, "out is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  MeasureOut mo{h->partials, nullptr, nullptr};  // no windings
  cudaError_t e = dispatch(h, MODE_MEASURE | MODE_GAUSS, mo, st);
  if (e != cudaSuccess) return cuda_fail(e, "diagnostics kernel");
  e = launch_finalize(h->partials, measure_blocks(h, false), nullptr, 0, h->scratch_rec, (long long)h->n, 1, 1, 0,
                      0, st);
  if (e != cudaSuccess) return cuda_fail(e, "finalize kernel");
  RawRecord r;
  int rc = read_scratch(h, &r, st);
  if (rc) return rc;
  to_diag(&h->p, r, out);
  return U1U1_OK;
}

extern "C" int u1u1_read_records(u1u1_lattice* h, u1u1_strings* s_out, u1u1_diag* d_out, int max, int* count,
                                 int64_t* lost, void* stream) {
  if (!h || !count) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  if (max < 0) return fail(U1U1_ERR_INVALID_ARG, "max must be >= 0");
  cudaStream_t st = (cudaStream_t)stream;
  int64_t avail = h->rec_written - h->rec_read;
  int64_t dropped = 0;
  if (avail > RING_CAP) {
    dropped = avail - RING_CAP;
    h->rec_read += dropped;
    avail = RING_CAP;
  }
  int64_t take = avail < max ? avail : max;
  // copy only the records being read: one contiguous run, or two when the
  // run wraps around the end of the ring
  int64_t first = h->rec_read % RING_CAP;
  int64_t run1 = take < RING_CAP - first ? take : RING_CAP - first;
  if (run1 > 0)
    U1U1_CUDA_TRY(cudaMemcpyAsync(h->host_rec + first, h->ring + first, sizeof(RawRecord) * run1,
                                  cudaMemcpyDeviceToHost, st), "record ring copy");
  if (take > run1)
    U1U1_CUDA_TRY(cudaMemcpyAsync(h->host_rec, h->ring, sizeof(RawRecord) * (take - run1),
                                  cudaMemcpyDeviceToHost, st), "record ring copy");
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  if (int rc = check_tma_timeout(h, st)) return rc;
  for (int64_t k = 0; k < take; ++k) {
    const RawRecord& r = h->host_rec[(h->rec_read + k) % RING_CAP];
    if (s_out) to_strings(&h->p, r, &s_out[k]);
    if (d_out) to_diag(&h->p, r, &d_out[k]);
  }
  h->rec_read += take;
  *count = (int)take;
  if (lost) *lost = dropped;
  return U1U1_OK;
}

// ---------------------------------------------------------------------------
// state transfer and checkpoints
// ---------------------------------------------------------------------------

// Host spans that the SMs copy directly: page-locked host memory mapped into
// the device's address space, 16-byte aligned, a whole number of 16-byte
// words, and lying inside one allocation (so no access can leave it).  On
// the GB300's CPU-GPU link such copies ran at 193 GB/s device to host and
// 211 GB/s host to device over twenty 4 GiB buffers, against 91-136 and
// 148-152 GB/s for the copy engines; every other host pointer (pageable
// memory, odd offsets) goes through the copy engines.
namespace {
using PointerGetAttributeFn = CUresult (*)(void*, CUpointer_attribute, CUdeviceptr);

PointerGetAttributeFn pointer_get_attribute() {
  static const PointerGetAttributeFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuPointerGetAttribute", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (PointerGetAttributeFn) nullptr;
    }
    return reinterpret_cast<PointerGetAttributeFn>(p);
  }();
  return fn;
}

bool mapped_host_span(const void* p, size_t bytes, void** dev) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type != cudaMemoryTypeHost || !at.devicePointer || bytes == 0) return false;
  const uintptr_t d = (uintptr_t)at.devicePointer;
  if ((d | (uintptr_t)bytes) & 15u) return false;
  const PointerGetAttributeFn get = pointer_get_attribute();
  if (!get) return false;
  CUdeviceptr start = 0;
  size_t size = 0;
  if (get(&start, CU_POINTER_ATTRIBUTE_RANGE_START_ADDR, (CUdeviceptr)d) != CUDA_SUCCESS ||
      get(&size, CU_POINTER_ATTRIBUTE_RANGE_SIZE, (CUdeviceptr)d) != CUDA_SUCCESS)
    return false;
  if (d < (uintptr_t)start || d - (uintptr_t)start > size || bytes > size - (d - (uintptr_t)start)) return false;
  *dev = at.devicePointer;
  return true;
}

// fields whose host span qualifies go to one SM copy launch, the rest to
// one copy-engine transfer each
int transfer_state(const u1u1_lattice* h, void* const dev[U1U1_NFIELDS], const void* const host[U1U1_NFIELDS],
                   bool upload, cudaStream_t st) {
  const size_t bytes = h->V * h->esize;
  for (int f = 0; f < U1U1_NFIELDS; ++f)  // every pointer checked before any copy is enqueued
    if (!host[f]) return fail(U1U1_ERR_INVALID_ARG, "host[%d] is NULL", f);
  XferTable t{};
  for (int f = 0; f < U1U1_NFIELDS; ++f) {
    void* hd = nullptr;
    if (mapped_host_span(host[f], bytes, &hd)) {
      t.src[t.m] = upload ? hd : dev[f];
      t.dst[t.m] = upload ? dev[f] : hd;
      ++t.m;
    } else if (upload) {
      U1U1_CUDA_TRY(cudaMemcpyAsync(dev[f], host[f], bytes, cudaMemcpyHostToDevice, st), "state upload");
    } else {
      U1U1_CUDA_TRY(cudaMemcpyAsync(const_cast<void*>(host[f]), dev[f], bytes, cudaMemcpyDeviceToHost, st),
                    "state download");
    }
  }
  U1U1_CUDA_TRY(launch_state_copy(t, (long long)(bytes / 16), st), upload ? "state upload" : "state download");
  return U1U1_OK;
}

void state_fields(const u1u1_lattice* h, void* dev[U1U1_NFIELDS]) {
  for (int f = 0; f < U1U1_NFIELDS; ++f) dev[f] = f < U1U1_NPOS ? h->pos[h->cur][f] : h->mom[f - U1U1_NPOS];
}
}  // namespace

extern "C" int u1u1_upload_state(u1u1_lattice* h, const void* const host[U1U1_NFIELDS], void* stream) {
  if (!h || !host) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  void* dev[U1U1_NFIELDS];
  state_fields(h, dev);
  return transfer_state(h, dev, host, true, (cudaStream_t)stream);
}

extern "C" int u1u1_download_state(const u1u1_lattice* h, void* const host[U1U1_NFIELDS], void* stream) {
  if (!h || !host) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  void* dev[U1U1_NFIELDS];
  state_fields(h, dev);
  return transfer_state(h, dev, host, false, (cudaStream_t)stream);
}

extern "C" int u1u1_host_span_mapped(const void* host, size_t bytes, int* mapped) {
  if (!host || !mapped) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  void* dev = nullptr;
  *mapped = mapped_host_span(host, bytes, &dev) ? 1 : 0;
  return U1U1_OK;
}

namespace {
const char CKPT_MAGIC[8] = {'U', '1', 'U', '1', 'C', 'K', 'P', '1'};
}

extern "C" int u1u1_save(const u1u1_lattice* h, const char* path, void* stream) {
  if (!h || !path) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  FILE* f = fopen(path, "wb");
  if (!f) return fail(U1U1_ERR_IO, "cannot open %s for writing", path);
  size_t bytes = h->V * h->esize;
  void* buf = malloc(bytes);
  if (!buf) {
    fclose(f);
    return fail(U1U1_ERR_OUT_OF_MEMORY, "host buffer of %zu bytes", bytes);
  }
  int rc = U1U1_OK;
  int64_t n = h->n;
  if (fwrite(CKPT_MAGIC, 8, 1, f) != 1 || fwrite(&h->p, sizeof(h->p), 1, f) != 1 || fwrite(&n, 8, 1, f) != 1)
    rc = fail(U1U1_ERR_IO, "write failed on %s", path);
  for (int k = 0; k < U1U1_NFIELDS && rc == U1U1_OK; ++k) {
    const void* src = k < U1U1_NPOS ? h->pos[h->cur][k] : h->mom[k - U1U1_NPOS];
    cudaError_t e = cudaMemcpy(buf, src, bytes, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) rc = cuda_fail(e, "checkpoint download");
    else if (fwrite(buf, 1, bytes, f) != bytes) rc = fail(U1U1_ERR_IO, "write failed on %s", path);
  }
  free(buf);
  if (fclose(f) != 0 && rc == U1U1_OK) rc = fail(U1U1_ERR_IO, "close failed on %s", path);
  return rc;
}

extern "C" int u1u1_load(u1u1_lattice* h, const char* path, void* stream) {
  if (!h || !path) return fail(U1U1_ERR_INVALID_ARG, "NULL argument");
  cudaStream_t st = (cudaStream_t)stream;
  U1U1_CUDA_TRY(cudaStreamSynchronize(st), "stream synchronize");
  FILE* f = fopen(path, "rb");
  if (!f) return fail(U1U1_ERR_IO, "cannot open %s", path);
  char magic[8];
  u1u1_params p;
  int64_t n;
  if (fread(magic, 8, 1, f) != 1 || memcmp(magic, CKPT_MAGIC, 8) != 0 || fread(&p, sizeof(p), 1, f) != 1 ||
      fread(&n, 8, 1, f) != 1) {
    fclose(f);
    return fail(U1U1_ERR_IO, "%s is not a u1u1 checkpoint", path);
  }
  if (p.nx != h->p.nx || p.ny != h->p.ny || p.nz != h->p.nz || p.precision != h->p.precision) {
    fclose(f);
    return fail(U1U1_ERR_INVALID_ARG, "checkpoint lattice %dx%dx%d/%d does not match the handle", p.nx, p.ny, p.nz,
                p.precision);
  }
  // a resumed run continues bit for bit only under the parameters it was
  // saved with (a phase switched by u1u1_set_params included)
  const struct {
    const char* name;
    double file, handle;
  } phys[] = {{"dx", p.dx, h->p.dx},           {"deta", p.deta, h->p.deta},
              {"eta0", p.eta0, h->p.eta0},     {"m", p.m, h->p.m},
              {"eta_ref", p.eta_ref, h->p.eta_ref}, {"beta", p.beta, h->p.beta},
              {"alpha", p.alpha, h->p.alpha},  {"lambda_p", p.lambda_p, h->p.lambda_p},
              {"lambda_q", p.lambda_q, h->p.lambda_q}, {"e_p", p.e_p, h->p.e_p},
              {"e_q", p.e_q, h->p.e_q},        {"sigma_p", p.sigma_p, h->p.sigma_p},
              {"sigma_q", p.sigma_q, h->p.sigma_q}, {"kappa", p.kappa, h->p.kappa}};
  for (const auto& q : phys)
    if (q.file != q.handle) {
      fclose(f);
      return fail(U1U1_ERR_INVALID_ARG, "checkpoint %s = %.17g, the handle's %.17g", q.name, q.file, q.handle);
    }
  size_t bytes = h->V * h->esize;
  // the rest of the file must be exactly the 20 fields: a truncated or
  // overlong file is refused before anything is written
  const long start = ftell(f);
  long end = -1;
  if (start >= 0 && fseek(f, 0, SEEK_END) == 0) end = ftell(f);
  if (end < 0 || fseek(f, start, SEEK_SET) != 0 ||
      (unsigned long long)(end - start) != (unsigned long long)bytes * U1U1_NFIELDS) {
    fclose(f);
    return fail(U1U1_ERR_IO, "%s holds %lld bytes of fields, %llu expected", path, (long long)(end - start),
                (unsigned long long)bytes * U1U1_NFIELDS);
  }
  void* buf = malloc(bytes);
  if (!buf) {
    fclose(f);
    return fail(U1U1_ERR_OUT_OF_MEMORY, "host buffer of %zu bytes", bytes);
  }
  int rc = U1U1_OK;
  for (int k = 0; k < U1U1_NFIELDS && rc == U1U1_OK; ++k) {
    void* dst = k < U1U1_NPOS ? h->pos[h->cur][k] : h->mom[k - U1U1_NPOS];
    if (fread(buf, 1, bytes, f) != bytes) rc = fail(U1U1_ERR_IO, "short read on %s", path);
    else {
      // staged from the pageable buffer before the call returns, ordered on st
      cudaError_t e = cudaMemcpyAsync(dst, buf, bytes, cudaMemcpyHostToDevice, st);
      if (e != cudaSuccess) rc = cuda_fail(e, "checkpoint upload");
    }
  }
  if (rc == U1U1_OK) {
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) rc = cuda_fail(e, "stream synchronize");
  }
  free(buf);
  fclose(f);
  if (rc == U1U1_OK) h->n = n;
  return rc;
}

// ---------------------------------------------------------------------------
// check entry points
// ---------------------------------------------------------------------------

extern "C" int u1u1_eval_link_phase(const float* theta, float* sin_out, float* cos_out, int64_t n, void* stream) {
  if (n < 0) return fail(U1U1_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return U1U1_OK;
  if (!theta || !sin_out || !cos_out) return fail(U1U1_ERR_INVALID_ARG, "NULL array");
  cudaError_t e = launch_link_phase(theta, sin_out, cos_out, (long long)n, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "link phase kernel");
  return U1U1_OK;
}

extern "C" int u1u1_eval_link_phase64(const double* theta, double* sin_out, double* cos_out, int64_t n,
                                      void* stream) {
  if (n < 0) return fail(U1U1_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return U1U1_OK;
  if (!theta || !sin_out || !cos_out) return fail(U1U1_ERR_INVALID_ARG, "NULL array");
  cudaError_t e = launch_link_phase64(theta, sin_out, cos_out, (long long)n, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "link phase kernel");
  return U1U1_OK;
}

extern "C" int u1u1_eval_edge_phase(const float* re, const float* im, float* out, int64_t n, void* stream) {
  if (n < 0) return fail(U1U1_ERR_INVALID_ARG, "n must be >= 0");
  if (n == 0) return U1U1_OK;
  if (!re || !im || !out) return fail(U1U1_ERR_INVALID_ARG, "NULL array");
  cudaError_t e = launch_edge_phase(re, im, out, (long long)n, (cudaStream_t)stream);
  if (e != cudaSuccess) return cuda_fail(e, "edge phase kernel");
  return U1U1_OK;
}

template Coef<float> u1u1::make_coef<float>(const u1u1_params*, int64_t);
template Coef<double> u1u1::make_coef<double>(const u1u1_params*, int64_t);

// ---------------------------------------------------------------------------
// autotuner
// ---------------------------------------------------------------------------

namespace {

void tune_key(const u1u1_lattice* h, char* key, size_t n) {
  cudaDeviceProp prop;
  int dev = 0;
  cudaGetDevice(&dev);
  if (cudaGetDeviceProperties(&prop, dev) != cudaSuccess) snprintf(prop.name, sizeof(prop.name), "unknown");
  char name[64];  // the device name, cut to 63 characters
  snprintf(name, sizeof(name), "%.63s", prop.name);
  for (char* c = name; *c; ++c)
    if (*c == ' ') *c = '_';
  snprintf(key, n, "%s/%dx%dx%d/%s", name, h->p.nx, h->p.ny, h->p.nz, h->esize == 8 ? "fp64" : "fp32");
}

// cache lines: "<key> <kernel> <waves>"
bool cache_lookup(const char* path, const char* key, int* kernel, int* waves) {
  if (!path) return false;
  FILE* f = fopen(path, "r");
  if (!f) return false;
  char k[256];
  int kk = 0, ww = 0;
  bool found = false;
  while (fscanf(f, "%255s %d %d", k, &kk, &ww) == 3)
    if (strcmp(k, key) == 0) {
      *kernel = kk;
      *waves = ww;
      found = true;
    }
  fclose(f);
  return found;
}

}  // namespace

extern "C" int u1u1_autotune(u1u1_lattice* h, const char* cache_path, int* kernel_out, int* waves_out, void* stream) {
  if (!h) return fail(U1U1_ERR_INVALID_ARG, "handle is NULL");
  cudaStream_t st = (cudaStream_t)stream;
  char key[256];
  tune_key(h, key, sizeof(key));
  int kernel = 0, waves = 0;
  if (cache_lookup(cache_path, key, &kernel, &waves)) {
    // accept only choices the tuner itself can make: the block-partial
    // buffers are sized for the candidate grids, and a larger one would
    // overrun them
    bool known = kernel == U1U1_KERNEL_SIMPLE;
    if (kernel == U1U1_KERNEL_TILED)
      for (int w : AUTOTUNE_WAVES) known = known || w == waves;
    if (!known)
      return fail(U1U1_ERR_INVALID_ARG, "autotune cache %s: entry '%s %d %d' is not a choice the tuner makes",
                  cache_path, key, kernel, waves);
    h->kernel = kernel;
    h->tile_waves = kernel == U1U1_KERNEL_TILED ? waves : TILE_WAVES_DEFAULT;
  } else {
    // time one plain step per candidate on the handle's own state: the step
    // reads the current position buffer, writes the other one and updates
    // the momenta, which are saved here and restored after every trial, so
    // the state is unchanged afterwards
    const size_t bytes = h->V * h->esize;
    void* save = nullptr;
    cudaError_t e = dev_alloc(&save, bytes * U1U1_NMOM);
    if (e != cudaSuccess) {
      cudaGetLastError();
      return fail(U1U1_ERR_OUT_OF_MEMORY, "autotune needs %zu bytes to save the momenta", bytes * U1U1_NMOM);
    }
    auto copy_mom = [&](bool to_save) -> cudaError_t {
      for (int f = 0; f < U1U1_NMOM; ++f) {
        char* s = (char*)save + (size_t)f * bytes;
        cudaError_t r = to_save ? cudaMemcpyAsync(s, h->mom[f], bytes, cudaMemcpyDeviceToDevice, st)
                                : cudaMemcpyAsync(h->mom[f], s, bytes, cudaMemcpyDeviceToDevice, st);
        if (r != cudaSuccess) return r;
      }
      return cudaSuccess;
    };
    const int kernel0 = h->kernel, waves0 = h->tile_waves;
    struct Cand { int kernel, waves; };
    Cand cands[N_AUTOTUNE_WAVES + 1];
    int nc = 0;
    for (int w : AUTOTUNE_WAVES) cands[nc++] = {U1U1_KERNEL_TILED, w};
    cands[nc++] = {U1U1_KERNEL_SIMPLE, TILE_WAVES_DEFAULT};
    float best = 1e30f;
    int bk = U1U1_KERNEL_TILED, bw = TILE_WAVES_DEFAULT;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = U1U1_OK;
    if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess) rc = cuda_fail(e, "events");
    if (!rc && (e = copy_mom(true)) != cudaSuccess) rc = cuda_fail(e, "autotune save");
    const MeasureOut none{nullptr, nullptr, nullptr};
    for (int k = 0; k < nc && !rc; ++k) {
      h->kernel = cands[k].kernel;
      h->tile_waves = cands[k].waves;
      float ms_best = 1e30f;
      for (int rep = 0; rep < 3 && !rc; ++rep) {  // the first repetition also warms up
        if ((e = copy_mom(false)) != cudaSuccess) { rc = cuda_fail(e, "autotune restore"); break; }
        cudaEventRecord(e0, st);
        if ((e = dispatch(h, MODE_WRITE, none, st)) != cudaSuccess) { rc = cuda_fail(e, "autotune step"); break; }
        cudaEventRecord(e1, st);
        if ((e = cudaEventSynchronize(e1)) != cudaSuccess) { rc = cuda_fail(e, "autotune sync"); break; }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        if (rep > 0 && ms < ms_best) ms_best = ms;
      }
      if (ms_best < best) {
        best = ms_best;
        bk = cands[k].kernel;
        bw = cands[k].waves;
      }
    }
    if (!rc && (e = copy_mom(false)) != cudaSuccess) rc = cuda_fail(e, "autotune restore");
    // the save buffer is read by copies on st: wait for them on every path
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess && !rc) rc = cuda_fail(e, "autotune sync");
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    dev_free(save);
    if (rc) {
      h->kernel = kernel0;
      h->tile_waves = waves0;
      return rc;
    }
    h->kernel = bk;
    h->tile_waves = bw;
    if (cache_path) {
      FILE* f = fopen(cache_path, "a");
      if (!f) return fail(U1U1_ERR_IO, "cannot append to %s", cache_path);
      fprintf(f, "%s %d %d\n", key, bk, bw);
      fclose(f);
    }
  }
  if (kernel_out) *kernel_out = h->kernel;
  if (waves_out) *waves_out = h->tile_waves;
  return U1U1_OK;
}
