/*
 * u1u1.h -- C ABI of libu1u1, a single-GPU (sm_103a) implementation of the
 * lattice time step and string diagnostics of the U(1)xU(1) model of
 * Correia & Martins, "Multitension strings in high-resolution U(1)xU(1)
 * simulations" (arXiv:2208.01525).
 *
 * Model (Sec. II): two complex scalars phi (sector p) and psi (sector q),
 * each with its own U(1) gauge field, A for p and B for q, coupled only
 * through the potential of Eq. 4,
 *   V = lambda_p/4 (|phi|^2 - sigma_p^2)^2 + lambda_q/4 (|psi|^2 - sigma_q^2)^2
 *       - kappa (|phi|^2 - sigma_p^2)(|psi|^2 - sigma_q^2).
 * Background (Sec. III): comoving periodic lattice, temporal gauge, power-law
 * FLRW expansion a ~ t^m, couplings scaled as lambda, kappa ~ a^{-2(1-beta)}
 * and e ~ a^{-(1-beta)} (Eq. 12).  Time step: the damped leapfrog of
 * Eqs. 17-26 (scalar kick, gauge kick, drift).
 *
 * Conventions fixed by this library where the paper is silent:
 *   - link variable U_i(x) = exp(-i dx A_i(x)); the gauge coupling is
 *     absorbed into A, so e^2 appears only in the current of Eq. 20 and in
 *     the 1/(2 e^2) gauge energy;
 *   - F_ij(x) = (A_j(x+i) - A_j(x) - A_i(x+j) + A_i(x)) / dx and the curl
 *     term of Eq. 20 is -sum_{j != i} (F_ij(x) - F_ij(x-j)) / dx;
 *   - a(eta) = (eta / eta_ref)^{m/(1-m)}, c_n = a_n^{2 beta},
 *     delta_n = (alpha/2) m/(1-m) deta/eta_n (Eq. 19), omega_n = delta_n (1-beta)
 *     (Eq. 22), eta_n = eta0 + n deta.
 *
 * Data layout.  A lattice of nx*ny*nz sites; every field is a separate
 * contiguous array of nx*ny*nz elements of the lattice precision (float or
 * double), site (x, y, z) at index x + nx*(y + ny*z).  Twenty fields make the
 * state: ten "position" fields at integer time n and ten momenta at n-1/2,
 * in the order of the U1U1_POS_* and U1U1_MOM_* constants below.  Position
 * fields are double-buffered (ping-pong): a step reads buffer `current` and
 * writes buffer `1 - current`; momenta are updated in place.
 *
 * Ownership.  The caller allocates and owns every field array (device
 * memory; 256-byte aligned base addresses) and must keep them alive, and not
 * write them, while a lattice handle uses them.  The handle owns only
 * metadata and its scratch memory (2 bytes per site for plaquette-winding
 * bytes plus small reduction buffers), released by u1u1_destroy.
 *
 * Errors.  Every int-returning call returns U1U1_OK (0) or a negative
 * U1U1_ERR_* code and never throws; u1u1_last_error() returns a message for
 * the calling thread's last failure.  A CUDA failure is reported as
 * U1U1_ERR_CUDA with the CUDA error string in the message.
 *
 * Streams.  `stream` arguments are cudaStream_t values passed as void*
 * (NULL = the legacy default stream).  Calls that only enqueue work return
 * before it runs; calls that fill host structs synchronise that stream.
 */
#ifndef U1U1_H
#define U1U1_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes ------------------------------------------------------ */
#define U1U1_OK 0
#define U1U1_ERR_INVALID_ARG (-1)   /* a parameter is out of its documented range */
#define U1U1_ERR_BAD_BUFFER (-2)    /* NULL or misaligned field array, or size mismatch */
#define U1U1_ERR_OUT_OF_MEMORY (-3) /* scratch allocation failed */
#define U1U1_ERR_CUDA (-4)          /* a CUDA runtime call or kernel launch failed */
#define U1U1_ERR_TIMEOUT (-5)       /* a bounded device-side wait ran out */
#define U1U1_ERR_NAN (-6)           /* a diagnostic pass found NaN in the state */
#define U1U1_ERR_NOT_SUPPORTED (-7) /* request valid but not implemented for this configuration */
#define U1U1_ERR_STATE (-8)         /* call not valid in the handle's current state */
#define U1U1_ERR_IO (-9)            /* file could not be read or written */

/* ---- precision --------------------------------------------------------- */
#define U1U1_FP32 0 /* float fields, FP32 arithmetic, compensated FP64 global sums */
#define U1U1_FP64 1 /* double fields and arithmetic throughout */

/* ---- field order ------------------------------------------------------- */
enum {
  U1U1_POS_PHI_RE = 0, U1U1_POS_PHI_IM, U1U1_POS_PSI_RE, U1U1_POS_PSI_IM,
  U1U1_POS_A0, U1U1_POS_A1, U1U1_POS_A2, U1U1_POS_B0, U1U1_POS_B1, U1U1_POS_B2,
  U1U1_NPOS
};
enum {
  U1U1_MOM_PI_RE = 0, U1U1_MOM_PI_IM, U1U1_MOM_PSI_RE, U1U1_MOM_PSI_IM,
  U1U1_MOM_E0, U1U1_MOM_E1, U1U1_MOM_E2, U1U1_MOM_H0, U1U1_MOM_H1, U1U1_MOM_H2,
  U1U1_NMOM
};
#define U1U1_NFIELDS (U1U1_NPOS + U1U1_NMOM)

/* ---- parameters (names follow the paper's symbols) ---------------------- */
typedef struct {
  int nx, ny, nz;       /* lattice sides; nx % 4 == 0; each >= 4 */
  double dx;            /* comoving lattice spacing Delta x (> 0) */
  double deta;          /* conformal time step Delta eta (> 0) */
  double eta0;          /* conformal time of step 0 (> 0 when m != 0) */
  double m;             /* a ~ t^m: 0 flat (a = 1), 1/2 radiation, 2/3 matter; 0 <= m < 1 */
  double eta_ref;       /* a(eta_ref) = 1 (> 0) */
  double beta;          /* Eq. 12: 1 physical, 0 constant comoving width, < 0 core growth */
  double alpha;         /* Hubble damping factor of Eq. 19 (the paper uses 2) */
  double lambda_p, lambda_q; /* lambda_0 per sector */
  double e_p, e_q;      /* e_0 per sector (> 0) */
  double sigma_p, sigma_q;   /* vacuum expectation values */
  double kappa;         /* kappa_0 of Eq. 4 */
  uint64_t seed;        /* random-phase initial conditions */
  int precision;        /* U1U1_FP32 or U1U1_FP64 */
} u1u1_params;

/* Caller-owned device field arrays (see "Data layout"). */
typedef struct {
  void* pos[2][U1U1_NPOS]; /* ping-pong position buffers */
  void* mom[U1U1_NMOM];    /* momenta, updated in place */
} u1u1_buffers;

/* Result of the fast string detection (Sec. III.A-B). */
typedef struct {
  int64_t n;            /* step index of the detected state */
  double eta;           /* its conformal time */
  int64_t n_p, n_q;     /* sum over plaquettes of |W| per sector */
  int64_t nonzero_p, nonzero_q; /* plaquettes with W != 0 per sector */
  int64_t n_pq_plaq;    /* plaquettes with W_p != 0 and W_q != 0 (exact overlap) */
  int64_t n_pq_cell;    /* p-pierced cells with a q-pierced cell within overlap_tol */
  int64_t n_pq_cell_q;  /* the same anchored on q-pierced cells (symmetry check) */
  int64_t n_flagged;    /* plaquette windings within 1e-4 of the +-pi branch cut */
  int32_t max_abs_w;    /* largest |W| seen */
  int32_t overlap_tol;  /* cell displacement allowed by the overlap (0 or 1) */
  int64_t n_w2_p, n_w2_q;           /* plaquettes with |W| >= 2 per sector (higher-winding census) */
  int64_t n_cells_ge4_p, n_cells_ge4_q; /* cells of value >= 4, e.g. a (2,0) string (Sec. III.B) */
  double L_p, L_q, L_pq;      /* dx * counts, L_s with L_pq subtracted */
  double xi_p, xi_q, xi_pq;   /* Eq. 31; +inf when the length is 0 */
  double xi_w;                /* Eq. 32 */
  double f_total, f_p;        /* Eqs. 34-35; NaN when undefined */
} u1u1_strings;

/* Network diagnostics of Sec. III.A on the state at integer time n.  The
 * momenta enter as the mean of their squares at n-1/2 and n+1/2. */
typedef struct {
  int64_t n;
  double eta, a;
  double kin_p, kin_q, grad_p, grad_q, el_p, el_q, mag_p, mag_q; /* lattice sums */
  double pot, vint;     /* sum c_n V and sum kappa(|phi|^2-sigma_p^2)(|psi|^2-sigma_q^2) */
  double pot_p, pot_q;  /* sum c_n lambda_s/4 (|phi_s|^2 - sigma_s^2)^2 per sector */
  double lag, energy;   /* sum of the Lagrangian and of the energy density */
  double rl_num, rl_den, rpq_num, rpq_den; /* Eq. 37 sums, W = L and W = V_int */
  double lag_total, energy_total; /* the sums times dx^3 */
  double xi_l;          /* Eq. 33 with mu = 2 pi sigma_p^2 */
  double lag_p, lag_q;  /* per-sector Lagrangian sums (own kinetic, gradient, gauge and
                           self-potential terms, the interaction term left out), times dx^3 */
  double xi_l_p, xi_l_q; /* Eq. 33 per sector with mu_s = 2 pi sigma_s^2, for unequal tensions */
  double R_l, v2_l, R_pq, v2_pq; /* Eqs. 36-37 */
  int32_t has_gauss;    /* 1 when the Gauss fields below were computed */
  double gauss_sum_p, gauss_sum_q, charge_sum_p, charge_sum_q;
  double gauss_max_p, gauss_max_q, gauss_rel_p, gauss_rel_q; /* rel = sum|G| / sum|rho| */
  double phi_min_p, phi_max_p, phi_min_q, phi_max_q;
  int64_t nan_count;    /* NaN entries among the 20 fields */
} u1u1_diag;

/* Bound-state segments of the robust method (Sec. III.B, Eq. 38). */
typedef struct {
  int64_t n;            /* step index of the state */
  int32_t overlap_tol;  /* cell overlap tolerance used for the pq cells */
  int32_t min_cells;    /* a component counts as a segment when it has more cells */
  int64_t n_cells;      /* pq cells (p-anchored fast-method overlap) */
  int64_t n_components; /* connected components of the pq cells */
  int64_t n_segments;   /* N_pq: components with more than min_cells cells */
  int64_t largest;      /* cells in the largest component */
  double L_pq;          /* dx * sum over segments of (N_cells - 1) */
  double l_pq;          /* L_pq / N_pq (Eq. 38); NaN when there is no segment */
  double xi_pq;         /* sqrt(V / L_pq); +inf when L_pq = 0 */
} u1u1_segments;

typedef struct u1u1_lattice u1u1_lattice;
typedef struct u1u1_ensemble u1u1_ensemble;

/* ---- library information ------------------------------------------------ */

/* Version string "major.minor.patch"; static storage. */
const char* u1u1_version(void);

/* Message of the calling thread's last failed call ("" if none). */
const char* u1u1_last_error(void);

/* ---- host-only helpers (no GPU needed) ---------------------------------- */

/* Fill *p with the paper's equal-tension values (Sec. IV): lambda = 2,
 * e = 1, sigma = 1, kappa = 0.9, alpha = 2, dx = 0.5, deta = 0.1,
 * radiation era (m = 1/2), beta = 1, eta0 = 1, eta_ref = 1, 64^3, FP32. */
int u1u1_params_default(u1u1_params* p);

/* Validate *p; U1U1_ERR_INVALID_ARG with a message naming the field. */
int u1u1_check_params(const u1u1_params* p);

/* Step coefficients of step n (Eqs. 12, 19, 22): out[0] = eta_n, out[1] = a_n,
 * out[2] = c_n = a_n^{2 beta}, out[3] = delta_n, out[4] = omega_n,
 * out[5] = c_n (1 + delta_n)/(1 + omega_n) (Gauss-law charge factor). */
int u1u1_coefficients(const u1u1_params* p, int64_t n, double out[6]);

/* Bytes of one field array for *p (nx*ny*nz times the element size);
 * 0 for a NULL or empty lattice. */
size_t u1u1_field_bytes(const u1u1_params* p);

/* sizeof of the public structs, for bindings to check their mirrors:
 * out[0] u1u1_params, out[1] u1u1_buffers, out[2] u1u1_strings,
 * out[3] u1u1_diag. */
void u1u1_abi_sizes(size_t out[4]);

/* ---- single lattice ----------------------------------------------------- */

/* Create a handle over caller buffers *b and enqueue the random-phase
 * initial conditions of Sec. III on `stream`: phi_s = sigma_s e^{i theta},
 * theta = 2 pi u, u the top 53 bits (times 2^-53) of draw number `site` of
 * the SplitMix64 generator (Steele, Lea & Flood 2014) whose state starts at
 * seed ^ (s << 62) (s = 0 for p, 1 for q); every other field zero, in both
 * position buffers.  The state is then at step n = 0 in buffer 0.
 * Errors: INVALID_ARG, BAD_BUFFER, OUT_OF_MEMORY, CUDA. */
int u1u1_init_lattice(const u1u1_params* p, const u1u1_buffers* b, void* stream,
                      u1u1_lattice** out);

/* Create a handle over buffers that already hold a state at step n in
 * position buffer `current` (0 or 1).  Enqueues nothing. */
int u1u1_attach_lattice(const u1u1_params* p, const u1u1_buffers* b, int64_t n, int current,
                        u1u1_lattice** out);

/* Release the handle and its scratch (not the caller's buffers).  A box
 * handle of an ensemble (u1u1_ensemble_lattice) is left alone: it is
 * released by u1u1_ensemble_destroy. */
void u1u1_destroy(u1u1_lattice* h);

/* Current step index and position buffer of the handle's state. */
int u1u1_current(const u1u1_lattice* h, int64_t* n, int* current);

/* Enqueue nsteps (>= 0) leapfrog steps (Eqs. 17-26).  Each step whose input
 * index n satisfies detect_every > 0 and n % detect_every == 0 is fused with
 * the detection of that input state: plaquette windings of both sectors
 * (Sec. III.A), the fast cell overlap (Sec. III.B, tolerance set by
 * u1u1_set_overlap_tol, default 1) and the diagnostic sums (Eqs. 33, 36-37,
 * without the Gauss-law fields); the result is appended to the handle's
 * record ring (read with u1u1_read_records).  Asynchronous on `stream`.
 * Each enqueued launch carries the values of the step it was enqueued for:
 * the coefficients of step n (Eqs. 12, 19, 22), the position buffer it reads
 * and writes, and (detection steps) the record-ring slot.  The call may be
 * recorded by stream capture, but a replay of such a graph repeats exactly
 * the captured launches with those captured values: it neither advances the
 * handle's step index nor re-evaluates the coefficients, and with an odd
 * nsteps it reads the position buffer the capture started from while the
 * momenta advance in place.  For replayed steps use the ensemble API, whose
 * graphs read coefficients and buffers from device tables.
 * Errors: INVALID_ARG, CUDA. */
int u1u1_step(u1u1_lattice* h, int nsteps, int detect_every, void* stream);

/* Diffusive cooling (Sec. III, Eqs. 27-30): nsteps >= 0 forward-Euler steps
 * of size dt > 0 of the first-order flow, per sector,
 *   d phi / dt = D^- D^+ phi - lambda/2 (|phi|^2 - sigma^2) phi,
 *   d A_i / dt = -sum_j (F_ij(x) - F_ij(x-j)) / dx + 2 e^2 Im[phi^* D_i^+ phi],
 * with lambda_0, e_0 and no kappa term, as printed; afterwards every
 * momentum and electric field is zero.  The step index is unchanged.
 * Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
int u1u1_cool(u1u1_lattice* h, double dt, int nsteps, void* stream);

/* Replace the time-dependent parameters of a handle (m, eta0, eta_ref,
 * deta, beta, alpha, couplings and vacuum values) by those of *p and set its
 * step index to n, keeping the lattice, precision, seed, buffers and the
 * current state: this chains the phases of a run schedule (damping with
 * m_damp, core growth with beta < 0, physical evolution; Sec. V, Table 3).
 * Errors: INVALID_ARG (invalid parameters or a different lattice/precision),
 * STATE (the handle is a box of an ensemble, whose device tables were built
 * from the box's parameters at creation). */
int u1u1_set_params(u1u1_lattice* h, const u1u1_params* p, int64_t n);

/* Overlap tolerance (0: same cell, 1: one cell in any of the 26 directions)
 * used by fused detection steps. */
int u1u1_set_overlap_tol(u1u1_lattice* h, int tol);

/* Fast string detection on the current state without stepping (Sec. III.A-B):
 * the plaquette windings of the current positions, the cells, the overlap
 * and the counts (the momenta are not read).
 * Optional device outputs (NULL to skip): cell_p, cell_q (uint8 per site:
 * sum over the cell's six faces of |W|, each |W| counted up to 3; any
 * alignment, 16-byte aligned arrays take the vectorised pass),
 * windings (int8, 6 arrays of nx*ny*nz: sector-major, plane (x,y), (x,z),
 * (y,z), the plaquette anchored at each site).  *out is filled on the host
 * (synchronises `stream`).  Errors: INVALID_ARG, CUDA, TIMEOUT (a tiled
 * step kernel of this handle had a bounded wait for its shared-memory tensor
 * copies run out since the handle's last check; each handle keeps its own
 * status, so a timeout is reported only by the handle whose launch it hit). */
int u1u1_detect_strings(u1u1_lattice* h, int overlap_tol, uint8_t* cell_p, uint8_t* cell_q,
                        int8_t* windings, u1u1_strings* out, void* stream);

/* Robust-method bound-state segments on the current state (Sec. III.B,
 * Eq. 38): the fast method's p-anchored pq cells (tolerance overlap_tol, 0
 * or 1) are split into connected components on the periodic lattice, cells
 * joined when they share a face, an edge or a corner (the connectivity
 * filter's rule); a component of N cells is a segment of length (N - 1) dx
 * (the off-by-one correction) and counts when N > min_cells (the paper uses
 * 41 at 4096^3).  labels_out (optional device int32 array of nx*ny*nz)
 * receives each pq cell's component label -- the smallest site index of its
 * component -- and -1 elsewhere.  Scratch (8 bytes per site) is allocated on
 * the handle's first call.  *out is filled on the host (synchronises
 * `stream`).  Errors: INVALID_ARG, NOT_SUPPORTED (more than 2^31 - 1
 * sites), OUT_OF_MEMORY, CUDA. */
int u1u1_pq_segments(u1u1_lattice* h, int overlap_tol, int min_cells, int32_t* labels_out, u1u1_segments* out,
                     void* stream);

/* All diagnostics of Sec. III.A on the current state, including the Gauss
 * law residual per sector at n-1/2 (Eqs. 9-10), without stepping.  Fills
 * *out on the host (synchronises `stream`).  Errors: CUDA, TIMEOUT (as for
 * u1u1_detect_strings). */
int u1u1_diagnostics(u1u1_lattice* h, u1u1_diag* out, void* stream);

/* Copy up to max records of fused detection steps not read yet, oldest
 * first, into s_out[] and d_out[] (either may be NULL); *count receives the
 * number copied and *lost (may be NULL) the number overwritten in the
 * device ring (capacity 1024) before they were read.  Synchronises `stream`.
 * Errors: INVALID_ARG, CUDA, TIMEOUT (a step kernel of this handle had a
 * bounded wait for its shared-memory tensor copies run out since the
 * handle's last check). */
int u1u1_read_records(u1u1_lattice* h, u1u1_strings* s_out, u1u1_diag* d_out, int max, int* count,
                      int64_t* lost, void* stream);

/* Copy the whole state between the handle's device buffers and 20 host
 * arrays (field order POS then MOM; each u1u1_field_bytes long; pinned
 * memory recommended).  Upload writes the current position buffer.  Arrays
 * for which u1u1_host_span_mapped reports 1 are copied by one kernel on the
 * SMs through their mapped device address (faster than the copy engines
 * over the CPU-GPU link); the others by one copy-engine transfer each.
 * Both calls are asynchronous on `stream`; the host arrays must stay valid
 * until the stream reaches them.  Errors: INVALID_ARG (NULL handle, table
 * or entry), CUDA. */
int u1u1_upload_state(u1u1_lattice* h, const void* const host[U1U1_NFIELDS], void* stream);
int u1u1_download_state(const u1u1_lattice* h, void* const host[U1U1_NFIELDS], void* stream);

/* *mapped = 1 when the host span [host, host + bytes) is page-locked host
 * memory mapped into the device's address space, 16-byte aligned, a whole
 * number of 16-byte words long and inside one allocation, so that state
 * transfers through it run on the SMs; 0 otherwise (copy engines).
 * Synchronous, no device work.  Errors: INVALID_ARG (NULL pointer). */
int u1u1_host_span_mapped(const void* host, size_t bytes, int* mapped);

/* Checkpoint / resume: write or read the parameters, step index and all 20
 * fields to or from a file; resuming continues bit for bit.  Synchronous.
 * u1u1_load writes the fields into the handle's current position buffer and
 * momenta and sets its step index.  It refuses, before writing anything, a
 * file whose lattice, precision or physical parameters (all but the seed)
 * differ from the handle's (INVALID_ARG, naming the first that differs),
 * and a file that is not a checkpoint or whose length is not exactly that
 * of the 20 fields (IO).
 * Errors: IO, INVALID_ARG, OUT_OF_MEMORY (host buffer), CUDA. */
int u1u1_save(const u1u1_lattice* h, const char* path, void* stream);
int u1u1_load(u1u1_lattice* h, const char* path, void* stream);

/* ---- kernel selection ---------------------------------------------------- */

/* Step kernel used by a handle: U1U1_KERNEL_AUTO picks the tuned one,
 * U1U1_KERNEL_SIMPLE is one thread per site with cached global loads,
 * U1U1_KERNEL_TILED the z-marching shared-memory kernel. */
/* Autotuner: choose the step kernel and the tiled kernel's z-chunking for
 * this handle's lattice by timing one plain step of each candidate (tiled
 * kernel with 8, 16, 32, 64, 128 or 256 target waves of CTAs; the simple kernel) on
 * the handle's own state, saving and restoring the momenta around every
 * trial so the state is unchanged (needs 10 field arrays of temporary device
 * memory).  The choice is applied to the handle and, when cache_path is not
 * NULL, looked up first in / appended to that text file, keyed by GPU name,
 * lattice and precision.  *kernel_out and *waves_out (may be NULL) receive
 * the choice.  A cache entry for this key that names a choice the tuner
 * does not make (another kernel id or wave count) is refused with
 * INVALID_ARG and the handle is left unchanged.  Synchronises `stream`.
 * Errors: INVALID_ARG, OUT_OF_MEMORY, IO, CUDA. */
int u1u1_autotune(u1u1_lattice* h, const char* cache_path, int* kernel_out, int* waves_out, void* stream);

#define U1U1_KERNEL_AUTO 0
#define U1U1_KERNEL_SIMPLE 1
#define U1U1_KERNEL_TILED 2
int u1u1_set_kernel(u1u1_lattice* h, int kernel);
int u1u1_get_kernel(const u1u1_lattice* h, int* kernel);
/* z-chunking of the tiled kernel's plain steps, as a target of `waves` x
 * (SMs x 3 resident CTAs) CTAs per launch: one of the tuner's candidates
 * (8, 16, 32, 64, 128, 256), else INVALID_ARG (the block-partial buffers are
 * sized for those grids).  Measuring passes keep the default chunking.  Lets
 * a caller reproduce a tuned choice without timing. */
int u1u1_set_tile_waves(u1u1_lattice* h, int waves);

/* Failure-detection test hook for the single-lattice tiled kernels' bounded
 * waits on their tensor copies into shared memory (process-wide; launches
 * enqueued afterwards see it).
 * enable = 1 makes every ring slot expect 16 bytes more than its copies
 * deliver, so every such wait runs out after limit_ns (the kernel finishes
 * on the delivered data and the next synchronising call of the handle that
 * launched it returns TIMEOUT);
 * enable = 0 restores normal copies.  limit_ns (>= 1000) is the wait limit
 * from then on; the default is 2 s.  No GPU fault or hang is involved.
 * Errors: INVALID_ARG. */
int u1u1_inject_copy_timeout(int enable, int64_t limit_ns);

/* Failure-detection test hook and accounting for the library's own
 * allocations: device scratch, tables and page-locked record buffers of
 * handles and ensembles (never the caller's field arrays).
 * u1u1_inject_alloc_failure(nth): nth >= 1 makes the nth allocation the
 * library attempts from now on fail as if the device were out of memory
 * (nothing is allocated and the device is not touched); the call that
 * needed it releases what it had taken and returns OUT_OF_MEMORY, leaving
 * the handle or ensemble it was called on as it was.  The hook fires once;
 * nth = 0 disarms it.  Process-wide.  Errors: INVALID_ARG (nth < 0).
 * u1u1_live_allocations: number and total bytes of the library allocations
 * held at the moment by every handle and ensemble of the process.  Neither
 * call needs a GPU. */
int u1u1_inject_alloc_failure(int nth);
int u1u1_live_allocations(int64_t* count, int64_t* bytes);

/* Debugging aid in place of a device memory checker.  With guard_bytes > 0
 * (a multiple of 256, at most 2^30) every library allocation made from then
 * on is handed out with guard_bytes of a fixed byte pattern (0xA5) on each
 * side, so that the blocks keep their 256-byte alignment; 0 turns guards off
 * for later allocations (earlier ones keep theirs).  Filling the guards
 * synchronises the device.  u1u1_check_alloc_guards synchronises the device
 * and sets *corrupted to the number of live allocations with a changed
 * guard byte, i.e. one that a kernel or a copy wrote past either end of.
 * Process-wide.  Errors: INVALID_ARG, CUDA. */
int u1u1_set_alloc_guard(int64_t guard_bytes);
int u1u1_check_alloc_guards(int64_t* corrupted);
/* Test hook for the check above: sets the first byte of the tail guard of one
 * live guarded allocation to 0 (memory the library owns, so nothing is
 * accessed out of bounds), so that the next check reports one corrupted
 * allocation.  Errors: STATE (no guarded allocation is live), CUDA. */
int u1u1_inject_guard_damage(void);

/* ---- ensembles of independent boxes ---------------------------------------- */

/* How u1u1_ensemble_run schedules the boxes' steps. */
#define U1U1_ENS_PERSISTENT 0 /* one persistent launch covers every step of every box */
#define U1U1_ENS_PER_STEP 1   /* one launch per step covering all boxes still running */
#define U1U1_ENS_UNBATCHED 2  /* one launch per box per step, box after box (reference loop) */

/* Create an ensemble of nboxes independent lattices (batched independent
 * realisations, e.g. uneven box sizes, eras, beta and seeds): per_box[b] and
 * buffers[b] are as for u1u1_init_lattice, every box gets its random-phase
 * initial conditions on `stream`, and all boxes share one precision.
 * horizon (0 = 8192) bounds the step index any box may reach; the per-step
 * coefficients of every box up to it are tabulated on the device at
 * creation.  Errors: INVALID_ARG, BAD_BUFFER, OUT_OF_MEMORY, CUDA. */
int u1u1_ensemble_create(const u1u1_params* per_box, int nboxes, const u1u1_buffers* buffers, int horizon,
                         void* stream, u1u1_ensemble** out);

/* Advance box b by steps[b] >= 0 leapfrog steps (Eqs. 17-26), all boxes
 * together, scheduled by `mode`.  With detect_every > 0, each step of a box
 * whose input index n satisfies n % detect_every == 0 is fused with the
 * detection of that input state, exactly as u1u1_step does for one lattice
 * (windings, cells, fast overlap with the tolerance of the box's handle as
 * set when the run is enqueued, and the diagnostic sums of Sec. III.A), and
 * the record is appended to the box's record ring, read with
 * u1u1_read_records on the box's handle (u1u1_ensemble_lattice); the
 * records equal those of the box stepped alone with u1u1_step.  In the
 * batched modes the detection steps of all boxes at one run step go through
 * one launch of each pass (measuring step, windings, cells, overlap,
 * finalize).  In U1U1_ENS_PERSISTENT mode one launch of about as many CTAs
 * as fit on the GPU takes (box, step, tile) work items from an ordered
 * ticket counter -- one such launch per stretch of plain steps between
 * detection steps; an item of step k of a box waits until every item of
 * step k-1 of that box is done (bounded wait: after the limit set by
 * u1u1_ensemble_set_wait_limit the kernel records U1U1_ERR_TIMEOUT, read
 * with u1u1_ensemble_status, and returns).  With use_graph != 0 the work of
 * this (steps, detect_every, mode) combination, and of each box's step index
 * modulo detect_every, is captured once into a CUDA graph and replayed on
 * later calls with the same combination (coefficients, buffers and record
 * slots come from device tables).  Asynchronous on `stream`.
 * Errors: INVALID_ARG, STATE (step horizon reached, or an earlier run timed
 * out), CUDA. */
int u1u1_ensemble_run(u1u1_ensemble* e, const int* steps, int detect_every, int mode, int use_graph, void* stream);

/* Borrow the handle of box b (for detection, diagnostics, state transfer);
 * it stays owned by the ensemble and valid until u1u1_ensemble_destroy
 * (u1u1_destroy leaves it alone; u1u1_set_params refuses it). */
int u1u1_ensemble_lattice(u1u1_ensemble* e, int box, u1u1_lattice** h);

/* Device status word of the last persistent run: U1U1_OK or
 * U1U1_ERR_TIMEOUT (a wait for another work item, or for a tensor copy into
 * shared memory, ran out of time).  Synchronises `stream`. */
int u1u1_ensemble_status(u1u1_ensemble* e, int* status, void* stream);

/* Wait limit of the persistent kernel's per-item dependency wait, in
 * nanoseconds (default 2e9). */
int u1u1_ensemble_set_wait_limit(u1u1_ensemble* e, int64_t ns);

/* Fault injection for tests of the bounded wait: when enabled, the first
 * work item of step 1 of the first box in the next persistent run waits for
 * a completion count that is never reached, so the run ends with
 * U1U1_ERR_TIMEOUT after the wait limit instead of hanging. */
int u1u1_ensemble_inject_unreachable_wait(u1u1_ensemble* e, int enable);

/* Autotuner for ensembles: times a probe run of probe_steps steps of every
 * box for each work-item z-chunk (16, 32, 64, 128 planes) and schedule
 * (persistent with and without tensor copies of interior tiles, per-step),
 * each timed as a CUDA-graph replay after a capturing run, restoring every
 * box's state and step index after each trial (needs a
 * temporary copy of the ensemble state), keeps the fastest z-chunk and
 * tensor-copy choice and returns the fastest schedule in *mode_out for
 * later u1u1_ensemble_run calls.  Synchronises `stream`.
 * Errors: INVALID_ARG, STATE, OUT_OF_MEMORY, CUDA. */
int u1u1_ensemble_autotune(u1u1_ensemble* e, int probe_steps, int* mode_out, int* item_lz_out, void* stream);

/* Set the ensemble's tuning knobs without timing (reproduces a tuned
 * choice): item_lz, the work-item z-chunk (16, 32, 64 or 128 planes), and
 * persistent_tma, whether the persistent kernel fills the ring slots of
 * interior tiles by tensor copies (1, the default) or by cp.async (0).
 * Results are the same either way.  Drops captured graphs; synchronises
 * `stream`.  Errors: INVALID_ARG, CUDA. */
int u1u1_ensemble_set_tuning(u1u1_ensemble* e, int item_lz, int persistent_tma, void* stream);

/* The ensemble's current tuning knobs (either output may be NULL).
 * Errors: INVALID_ARG. */
int u1u1_ensemble_get_tuning(const u1u1_ensemble* e, int* item_lz, int* persistent_tma);

void u1u1_ensemble_destroy(u1u1_ensemble* e);

/* ---- detection without device allocation ------------------------------------ */

/* Largest lattice, in sites, accepted by u1u1_detect_strings_noalloc. */
#define U1U1_NOALLOC_MAX_SITES 16777216 /* 256^3 */

/* Fast string detection (same windings, cells, overlap and counts as
 * u1u1_detect_strings) for callers that cannot allocate device memory:
 * code that runs while a framework owns the whole device pool, inside an
 * allocator or memory-pressure callback, or under a policy that forbids
 * allocation after start-up.  It needs no lattice handle and calls no
 * cudaMalloc, cudaFree or other allocating routine; its scratch (winding
 * bytes, cell masks, block partials, one record) is a fixed static device
 * array inside the library, 48 MiB on every GPU that loads the library,
 * held until the process exits.  This entry point is an engineering
 * addition: the paper has no counterpart.
 * Arguments: p, the lattice parameters; fields, the 20 device field arrays
 * of the state (U1U1_POS_* then U1U1_MOM_* order, layout as for a lattice,
 * 256-byte aligned; only the ten position fields are read); n, the step
 * index the record reports;
 * overlap_tol, 0 or 1; *out, filled on the host.  Synchronises `stream`.
 * Limits: at most U1U1_NOALLOC_MAX_SITES sites, and the scratch the shape
 * needs must fit the array (every cubic box up to 256^3 does); larger
 * requests return U1U1_ERR_INVALID_ARG with the byte count in the message.
 * Set-up: the first call on a device, with that device current, looks up
 * the array's device address (cudaGetSymbolAddress); make that first call
 * before any stream capture.  The lookup is repeated only when the device's
 * context has changed since (e.g. after cudaDeviceReset).  All calls share the one array, which keeps
 * the last call's contents: calls that overlap on the GPU (several streams
 * or threads) race and must be serialised by the caller.
 * Errors: INVALID_ARG, NOT_SUPPORTED (device index >= 64), CUDA. */
int u1u1_detect_strings_noalloc(const u1u1_params* p, const void* const fields[U1U1_NFIELDS], int64_t n,
                                int overlap_tol, u1u1_strings* out, void* stream);

/* ---- check entry points ---------------------------------------------------- */

/* Measured FP64 arithmetic rate of the current device, in TFLOP/s (two
 * operations per fused multiply-add): every thread of a full-occupancy grid
 * runs eight independent chains of dependent FP64 FMAs, timed with CUDA
 * events on `stream` over runs of at least 50 ms (best of several).  The
 * ceiling of the FP64 step, which is bound by the FP64 pipe rather than by
 * HBM (Sec. III, Eqs. 17-26 in double precision); a measurement helper with
 * no counterpart in the paper.  Changes no device setting and allocates no
 * device memory.  Synchronises `stream`.  Errors: INVALID_ARG, CUDA. */
int u1u1_fp64_fma_rate(double* tflops, void* stream);

/* Evaluate, on n device values theta, the FP32 routine the kernels use for
 * the link variable U = exp(-i theta) (sin and cos of theta: reduction by
 * 2 pi split in two floats, then the hardware sine and cosine), writing
 * sin_out[k] and cos_out[k] (device arrays).  Lets tests bound its error against a double-precision
 * reference.  Asynchronous on `stream`.  Errors: INVALID_ARG, CUDA. */
int u1u1_eval_link_phase(const float* theta, float* sin_out, float* cos_out, int64_t n, void* stream);

/* Evaluate, on n device angles theta[k], the FP64 routine the FP64 kernels
 * use for the link variable U = exp(-i theta) (Sec. III, Eqs. 17-21): the
 * table-driven method (theta = m 2 pi / 1024 + r, a table of sin and cos at
 * the multiples, short Taylor polynomials in r), writing sin_out[k] and
 * cos_out[k] (device arrays).  Lets tests bound its error against a
 * correctly rounded reference.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, CUDA. */
int u1u1_eval_link_phase64(const double* theta, double* sin_out, double* cos_out, int64_t n, void* stream);

/* Evaluate, on n device pairs (re[k], im[k]), the FP32 routine the kernels
 * use for the gauge-invariant edge phase chi = arg(re + i im) in [-pi, pi]
 * of the plaquette windings (Sec. III.A: octant reduction and a minimax
 * polynomial), writing out[k] (device array).  Lets tests bound its error
 * against a double-precision arctangent.  Asynchronous on `stream`.
 * Errors: INVALID_ARG, CUDA. */
int u1u1_eval_edge_phase(const float* re, const float* im, float* out, int64_t n, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* U1U1_H */
