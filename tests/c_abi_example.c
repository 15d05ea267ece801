/* A plain C caller of libu1u1: no Python and no C++.  It allocates the 30
 * field arrays with the CUDA runtime, creates a lattice with random-phase
 * initial conditions (Sec. III), takes 32 leapfrog steps with detection fused
 * into every 16th (Eqs. 17-26, Sec. III.A), reads the detection records, runs
 * the standalone string detection (Sec. III.A-B) and diagnostics (Eqs. 33-37)
 * on the final state, and prints the results as one line of key=value pairs,
 * which tests/test_c_abi_example.py compares with the Python binding's.
 *
 * usage: c_abi_example [side]   (a cube of side^3 sites, FP32; default 32) */
#include <cuda_runtime_api.h>
#include <stdio.h>
#include <stdlib.h>

#include "u1u1.h"

#define CHECK(call)                                                              \
  do {                                                                           \
    int rc_ = (call);                                                            \
    if (rc_ != U1U1_OK) {                                                        \
      fprintf(stderr, "%s failed (%d): %s\n", #call, rc_, u1u1_last_error());    \
      return 1;                                                                  \
    }                                                                            \
  } while (0)

int main(int argc, char** argv) {
  const int side = argc > 1 ? atoi(argv[1]) : 32;
  u1u1_params p;
  CHECK(u1u1_params_default(&p));
  p.nx = p.ny = p.nz = side;
  p.m = 0.5; /* radiation era */
  p.beta = 1.0;
  p.eta0 = 1.0;
  p.eta_ref = 1.0 + 0.1 * 32; /* a = 1 after the 32 steps */
  p.seed = 7;
  p.precision = U1U1_FP32;
  CHECK(u1u1_check_params(&p));

  /* the caller owns the fields: two position buffers and the momenta */
  const size_t bytes = u1u1_field_bytes(&p);
  u1u1_buffers b;
  for (int k = 0; k < 2; ++k)
    for (int f = 0; f < U1U1_NPOS; ++f)
      if (cudaMalloc(&b.pos[k][f], bytes) != cudaSuccess) return 2;
  for (int f = 0; f < U1U1_NMOM; ++f)
    if (cudaMalloc(&b.mom[f], bytes) != cudaSuccess) return 2;

  u1u1_lattice* h = NULL;
  CHECK(u1u1_init_lattice(&p, &b, NULL, &h));
  CHECK(u1u1_step(h, 32, 16, NULL));

  u1u1_strings rs[4];
  u1u1_diag rd[4];
  int count = 0;
  int64_t lost = 0;
  CHECK(u1u1_read_records(h, rs, rd, 4, &count, &lost, NULL));
  u1u1_strings s;
  CHECK(u1u1_detect_strings(h, 1, NULL, NULL, NULL, &s, NULL));
  u1u1_diag d;
  CHECK(u1u1_diagnostics(h, &d, NULL));
  int64_t n = 0;
  int cur = 0;
  CHECK(u1u1_current(h, &n, &cur));

  printf("records=%d lost=%lld n=%lld current=%d", count, (long long)lost, (long long)n, cur);
  for (int r = 0; r < count; ++r)
    printf(" rec%d_n=%lld rec%d_n_p=%lld rec%d_n_q=%lld rec%d_energy=%.17g", r, (long long)rs[r].n, r,
           (long long)rs[r].n_p, r, (long long)rs[r].n_q, r, rd[r].energy);
  printf(" n_p=%lld n_q=%lld n_pq_plaq=%lld n_pq_cell=%lld xi_w=%.17g energy=%.17g lag=%.17g\n",
         (long long)s.n_p, (long long)s.n_q, (long long)s.n_pq_plaq, (long long)s.n_pq_cell, s.xi_w, d.energy,
         d.lag);

  u1u1_destroy(h);
  for (int k = 0; k < 2; ++k)
    for (int f = 0; f < U1U1_NPOS; ++f) cudaFree(b.pos[k][f]);
  for (int f = 0; f < U1U1_NMOM; ++f) cudaFree(b.mom[f]);
  return 0;
}
