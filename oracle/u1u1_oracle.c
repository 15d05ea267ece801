/*
 * u1u1_oracle.c -- plain, slow, FP64 CPU oracle for the U(1)xU(1) lattice
 * Abelian-Higgs step of Correia & Martins, "Multitension strings in
 * high-resolution U(1)xU(1) simulations" (arXiv:2208.01525).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the package's smoke check and
 * the CPU-baseline leg of the benchmark may load this code.  It shares no
 * source, header, table or helper with the CUDA library; the two agree on
 * nothing but the field order of the state array (a data format) and the
 * published SplitMix64 generator, which each side writes out on its own.
 *
 * Everything is double precision, loops are plain z-y-x triple loops, and the
 * leapfrog step is three separate passes over the lattice (scalar kick, gauge
 * kick, drift) with no fusion, exactly in the order of Sec. III.
 *
 * Conventions (the paper leaves them implicit; the readings are listed in the
 * design notes of the repository):
 *   - sector s = 0 is the p sector (phi, Pi, A, E), s = 1 the q sector
 *     (psi, Psi, B, H); the equations are identical per sector (Sec. II,
 *     the phi<->psi exchange symmetry after Eq. 10).
 *   - the gauge coupling is absorbed into the link field: the link variable
 *     is U_i(x) = exp(-i dx A_i(x)), the forward covariant difference is
 *     D_i^+ phi = (U_i(x) phi(x+i) - phi(x)) / dx, and e^2 appears only in
 *     the current term of Eq. 20 and in the 1/(2 e^2) gauge energy.
 *   - F_ij(x) = (A_j(x+i) - A_j(x) - A_i(x+j) + A_i(x)) / dx (forward
 *     lattice curl) and the "-d_i^- F_ij" term of Eq. 20 is read as
 *     -sum_{j != i} (F_ij(x) - F_ij(x-j)) / dx.
 *   - kappa in Eq. 17 is kappa_0, so it scales with a^{2 beta} like lambda
 *     (Eq. 12).
 *
 * State layout (shared data format, not code): one double array of
 * 20 * V entries, V = nx*ny*nz, field-major, site index x + nx*(y + ny*z):
 *   0..3   phi_re, phi_im, psi_re, psi_im          (scalars, time n)
 *   4..6   A_0, A_1, A_2                           (p links, time n)
 *   7..9   B_0, B_1, B_2                           (q links, time n)
 *   10..13 Pi_re, Pi_im, Psi_re, Psi_im            (momenta, time n-1/2)
 *   14..16 E_0, E_1, E_2                           (time n-1/2)
 *   17..19 H_0, H_1, H_2                           (time n-1/2)
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

#define ORC_NFIELDS 20

typedef struct {
  int nx, ny, nz;
  double dx, deta, eta0;
  double m;        /* a ~ t^m in cosmic time; 0 gives a flat a = 1 */
  double eta_ref;  /* a(eta_ref) = 1 */
  double beta;     /* PRS exponent (Eq. 12) */
  double alpha;    /* damping factor of Eq. 19 */
  double lambda[2], e[2], sigma[2], kappa;
  uint64_t seed;
} orc_params;

/* ---- indexing ---------------------------------------------------------- */

static long wrapi(long i, long n) {
  long r = i % n;
  return r < 0 ? r + n : r;
}

/* site index of (x, y, z) on the periodic box */
static long sidx(const orc_params* p, long x, long y, long z) {
  return wrapi(x, p->nx) + (long)p->nx * (wrapi(y, p->ny) + (long)p->ny * wrapi(z, p->nz));
}

/* site index of x shifted by d (in {-1, +1}) along direction i */
static long shift(const orc_params* p, long site, int i, int d) {
  long V2 = (long)p->nx * p->ny;
  long x = site % p->nx, y = (site / p->nx) % p->ny, z = site / V2;
  if (i == 0) x += d;
  else if (i == 1) y += d;
  else z += d;
  return sidx(p, x, y, z);
}

static long nsites(const orc_params* p) { return (long)p->nx * p->ny * p->nz; }

static int f_phi(int s, int c) { return 2 * s + c; }
static int f_A(int s, int i) { return 4 + 3 * s + i; }
static int f_pi(int s, int c) { return 10 + 2 * s + c; }
static int f_E(int s, int i) { return 14 + 3 * s + i; }

/* ---- complex helpers --------------------------------------------------- */

typedef struct { double re, im; } cplx;

static cplx cmul(cplx a, cplx b) {
  cplx r = {a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re};
  return r;
}
static cplx cconj(cplx a) { cplx r = {a.re, -a.im}; return r; }
static double cabs2(cplx a) { return a.re * a.re + a.im * a.im; }

static cplx get_phi(const orc_params* p, const double* st, int s, long site) {
  long V = nsites(p);
  cplx r = {st[f_phi(s, 0) * V + site], st[f_phi(s, 1) * V + site]};
  return r;
}
static double get_A(const orc_params* p, const double* st, int s, int i, long site) {
  return st[f_A(s, i) * nsites(p) + site];
}

/* link variable U_i(x) = exp(-i dx A_i(x)) */
static cplx link_U(const orc_params* p, const double* st, int s, int i, long site) {
  double th = p->dx * get_A(p, st, s, i, site);
  cplx r = {cos(th), -sin(th)};
  return r;
}

/* F_ij(x), forward lattice curl of the link field of sector s */
static double plaq_F(const orc_params* p, const double* st, int s, int i, int j, long site) {
  long xi = shift(p, site, i, +1), xj = shift(p, site, j, +1);
  return (get_A(p, st, s, j, xi) - get_A(p, st, s, j, site)
          - get_A(p, st, s, i, xj) + get_A(p, st, s, i, site)) / p->dx;
}

/* ---- time-dependent coefficients (Sec. III, Eqs. 12, 19, 22) ------------ */

/* out[0] = eta_n, out[1] = a_n, out[2] = c_n = a_n^{2 beta},
 * out[3] = delta_n, out[4] = omega_n,
 * out[5] = c_n (1 + delta_n) / (1 + omega_n), the charge factor of the
 *          conserved half-step Gauss constraint. */
void orc_coeffs(const orc_params* p, long n, double* out) {
  double eta = p->eta0 + (double)n * p->deta;
  double pm = (p->m == 0.0) ? 0.0 : p->m / (1.0 - p->m); /* d ln a / d ln eta */
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

/* ---- random-phase initial conditions (Sec. III) ------------------------- */

/* SplitMix64 (Steele, Lea & Flood, OOPSLA 2014): output number k (k = 0, 1,
 * ...) of the generator whose 64-bit state starts at x0; the state advances
 * by the odd constant 0x9E3779B97F4A7C15 per draw and each output is the
 * state passed through the generator's two xor-shift-multiply rounds. */
static uint64_t splitmix64_at(uint64_t x0, uint64_t k) {
  uint64_t z = x0 + (k + 1) * 0x9E3779B97F4A7C15ULL;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
  return z ^ (z >> 31);
}

/* |phi_s| = sigma_s with a uniform random phase per site; momenta, links and
 * electric fields zero.  theta = 2 pi u with u the top 53 bits (times 2^-53)
 * of draw number `site` of the SplitMix64 stream that starts at
 * seed ^ (s << 62), one stream per sector. */
void orc_init(const orc_params* p, double* st) {
  long V = nsites(p);
  memset(st, 0, sizeof(double) * ORC_NFIELDS * (size_t)V);
  for (int s = 0; s < 2; ++s) {
    uint64_t x0 = p->seed ^ ((uint64_t)s << 62);
    for (long site = 0; site < V; ++site) {
      double u = (double)(splitmix64_at(x0, (uint64_t)site) >> 11) * (1.0 / 9007199254740992.0);
      double th = (2.0 * M_PI) * u;
      st[f_phi(s, 0) * V + site] = p->sigma[s] * cos(th);
      st[f_phi(s, 1) * V + site] = p->sigma[s] * sin(th);
    }
  }
}

/* ---- the three passes of one leapfrog step (Sec. III) ------------------ */

/* Scalar kick, Eqs. 17-18: new momenta (time n+1/2) of both sectors into
 * pi_new[4 * V] (field order Pi_re, Pi_im, Psi_re, Psi_im). */
void orc_scalar_kick(const orc_params* p, const double* st, long n, double* pi_new) {
  long V = nsites(p);
  double cf[6];
  orc_coeffs(p, n, cf);
  double c = cf[2], delta = cf[3];
  double inv_dx2 = 1.0 / (p->dx * p->dx);
#pragma omp parallel for schedule(static)
  for (long z = 0; z < p->nz; ++z)
    for (long y = 0; y < p->ny; ++y)
      for (long x = 0; x < p->nx; ++x) {
        long site = sidx(p, x, y, z);
        for (int s = 0; s < 2; ++s) {
          int o = 1 - s;
          cplx f = get_phi(p, st, s, site);
          cplx lap = {0.0, 0.0};
          for (int i = 0; i < 3; ++i) {
            long xp = shift(p, site, i, +1), xm = shift(p, site, i, -1);
            cplx fwd = cmul(link_U(p, st, s, i, site), get_phi(p, st, s, xp));
            cplx bwd = cmul(cconj(link_U(p, st, s, i, xm)), get_phi(p, st, s, xm));
            lap.re += fwd.re + bwd.re - 2.0 * f.re;
            lap.im += fwd.im + bwd.im - 2.0 * f.im;
          }
          lap.re *= inv_dx2;
          lap.im *= inv_dx2;
          double r_self = cabs2(f) - p->sigma[s] * p->sigma[s];
          double r_other = cabs2(get_phi(p, st, o, site)) - p->sigma[o] * p->sigma[o];
          double g = c * (0.5 * p->lambda[s] * r_self - p->kappa * r_other);
          double pr = st[f_pi(s, 0) * V + site], pi = st[f_pi(s, 1) * V + site];
          pi_new[(2 * s + 0) * V + site] =
              ((1.0 - delta) * pr + p->deta * (lap.re - g * f.re)) / (1.0 + delta);
          pi_new[(2 * s + 1) * V + site] =
              ((1.0 - delta) * pi + p->deta * (lap.im - g * f.im)) / (1.0 + delta);
        }
      }
}

/* Gauge kick, Eqs. 20-21: new electric fields (time n+1/2) into
 * E_new[6 * V] (field order E_0..2, H_0..2). */
void orc_gauge_kick(const orc_params* p, const double* st, long n, double* E_new) {
  long V = nsites(p);
  double cf[6];
  orc_coeffs(p, n, cf);
  double c = cf[2], omega = cf[4];
#pragma omp parallel for schedule(static)
  for (long z = 0; z < p->nz; ++z)
    for (long y = 0; y < p->ny; ++y)
      for (long x = 0; x < p->nx; ++x) {
        long site = sidx(p, x, y, z);
        for (int s = 0; s < 2; ++s) {
          cplx f = get_phi(p, st, s, site);
          for (int i = 0; i < 3; ++i) {
            long xp = shift(p, site, i, +1);
            /* current Im[phi^* D_i^+ phi] = Im[phi^*(x) U_i(x) phi(x+i)] / dx */
            cplx t = cmul(cconj(f), cmul(link_U(p, st, s, i, site), get_phi(p, st, s, xp)));
            double J = t.im / p->dx;
            double curl = 0.0;
            for (int j = 0; j < 3; ++j) {
              if (j == i) continue;
              long xmj = shift(p, site, j, -1);
              curl += (plaq_F(p, st, s, i, j, site) - plaq_F(p, st, s, i, j, xmj)) / p->dx;
            }
            double Eold = st[f_E(s, i) * V + site];
            double e2 = p->e[s] * p->e[s];
            E_new[(3 * s + i) * V + site] =
                ((1.0 - omega) * Eold + p->deta * (-curl + 2.0 * e2 * c * J)) / (1.0 + omega);
          }
        }
      }
}

/* Drift, Eqs. 23-26, then the new momenta replace the old ones. */
void orc_drift(const orc_params* p, double* st, const double* pi_new, const double* E_new) {
  long V = nsites(p);
  for (int s = 0; s < 2; ++s) {
    for (int c = 0; c < 2; ++c)
      for (long site = 0; site < V; ++site) {
        double v = pi_new[(2 * s + c) * V + site];
        st[f_phi(s, c) * V + site] += p->deta * v;
        st[f_pi(s, c) * V + site] = v;
      }
    for (int i = 0; i < 3; ++i)
      for (long site = 0; site < V; ++site) {
        double v = E_new[(3 * s + i) * V + site];
        st[f_A(s, i) * V + site] += p->deta * v;
        st[f_E(s, i) * V + site] = v;
      }
  }
}

/* nsteps leapfrog steps starting from step index n0.  work must hold
 * 10 * V doubles. */
void orc_step(const orc_params* p, double* st, long n0, int nsteps, double* work) {
  long V = nsites(p);
  for (int k = 0; k < nsteps; ++k) {
    long n = n0 + k;
    orc_scalar_kick(p, st, n, work);
    orc_gauge_kick(p, st, n, work + 4 * V);
    orc_drift(p, st, work, work + 4 * V);
  }
}

/* ---- diffusive cooling (Sec. III, Eqs. 27-30) --------------------------- */

/* Forward-Euler steps of the first-order flow
 *   d phi / dt = D^- D^+ phi - lambda/2 (|phi|^2 - sigma^2) phi
 *   d A_i / dt = -sum_j d_j^- F_ij + 2 e^2 Im[phi^* D_i^+ phi]
 * per sector, with no kappa term, as printed.  Momenta are left untouched.
 * work must hold 10 * V doubles. */
void orc_cool(const orc_params* p, double* st, double dt, int nsteps, double* work) {
  long V = nsites(p);
  orc_params q = *p;
  /* the flow is the a = 1, undamped limit of the kicks with kappa = 0 and
   * zero old momenta: (lap - g phi) and (-curl + 2 e^2 J) */
  q.m = 0.0;
  q.beta = 1.0;
  q.kappa = 0.0;
  q.deta = 1.0;
  double* tmp = (double*)malloc(sizeof(double) * ORC_NFIELDS * (size_t)V);
  for (int k = 0; k < nsteps; ++k) {
    memcpy(tmp, st, sizeof(double) * ORC_NFIELDS * (size_t)V);
    memset(tmp + 10 * V, 0, sizeof(double) * 10 * (size_t)V);
    orc_scalar_kick(&q, tmp, 0, work);
    orc_gauge_kick(&q, tmp, 0, work + 4 * V);
    for (int s = 0; s < 2; ++s) {
      for (int c = 0; c < 2; ++c)
        for (long site = 0; site < V; ++site)
          st[f_phi(s, c) * V + site] += dt * work[(2 * s + c) * V + site];
      for (int i = 0; i < 3; ++i)
        for (long site = 0; site < V; ++site)
          st[f_A(s, i) * V + site] += dt * work[4 * V + (3 * s + i) * V + site];
    }
  }
  free(tmp);
}

/* ---- gauge-invariant plaquette windings (Sec. III.A) -------------------- */

/* Edge phase chi_i(x) = arg(phi^*(x) U_i(x) phi(x+i)) in (-pi, pi].
 * *near_cut is set when pi - |chi| < 1e-4 or the product is exactly 0. */
static double edge_chi(const orc_params* p, const double* st, int s, int i, long site,
                       int* near_cut) {
  long xp = shift(p, site, i, +1);
  cplx t = cmul(cconj(get_phi(p, st, s, site)),
                cmul(link_U(p, st, s, i, site), get_phi(p, st, s, xp)));
  double chi = atan2(t.im, t.re);
  if (M_PI - fabs(chi) < 1e-4 || (t.re == 0.0 && t.im == 0.0)) *near_cut = 1;
  return chi;
}

/* Winding of every plaquette of both sectors: W[(3 s + k) V + x] for the
 * plaquette anchored at x in plane k = 0 (x,y), 1 (x,z), 2 (y,z), oriented
 * x -> x+i -> x+i+j -> x+j with i < j:
 *   W = rint{ [chi_i(x) + chi_j(x+i) - chi_i(x+j) - chi_j(x)
 *             + dx (A_i(x) + A_j(x+i) - A_i(x+j) - A_j(x))] / (2 pi) }.
 * flag[...] = 1 when one of the four edges is within 1e-4 of the branch cut. */
void orc_windings(const orc_params* p, const double* st, signed char* W, unsigned char* flag) {
  static const int PI_[3] = {0, 0, 1}, PJ_[3] = {1, 2, 2};
  long V = nsites(p);
  for (int s = 0; s < 2; ++s)
    for (int k = 0; k < 3; ++k) {
      int i = PI_[k], j = PJ_[k];
      for (long site = 0; site < V; ++site) {
        long xi = shift(p, site, i, +1), xj = shift(p, site, j, +1);
        int cut = 0;
        double tot = edge_chi(p, st, s, i, site, &cut) + edge_chi(p, st, s, j, xi, &cut)
                   - edge_chi(p, st, s, i, xj, &cut) - edge_chi(p, st, s, j, site, &cut);
        tot += p->dx * (get_A(p, st, s, i, site) + get_A(p, st, s, j, xi)
                        - get_A(p, st, s, i, xj) - get_A(p, st, s, j, site));
        W[(3 * s + k) * V + site] = (signed char)lrint(tot / (2.0 * M_PI));
        flag[(3 * s + k) * V + site] = (unsigned char)cut;
      }
    }
}

/* Cell arrays of the fast method (Sec. III.B): the value of cell x (the cube
 * with corners x + {0,1}^3) is the sum over its six faces of |W|; a straight
 * unit string pierces two faces and gives 2.  Saturates at 255. */
void orc_cells(const orc_params* p, const signed char* W, unsigned char* cells) {
  long V = nsites(p);
  for (int s = 0; s < 2; ++s)
    for (long site = 0; site < V; ++site) {
      long xp = shift(p, site, 0, +1), yp = shift(p, site, 1, +1), zp = shift(p, site, 2, +1);
      const signed char* w = W + 3 * s * V;
      int v = abs(w[0 * V + site]) + abs(w[0 * V + zp])   /* (x,y) faces at z, z+1 */
            + abs(w[1 * V + site]) + abs(w[1 * V + yp])   /* (x,z) faces at y, y+1 */
            + abs(w[2 * V + site]) + abs(w[2 * V + xp]);  /* (y,z) faces at x, x+1 */
      cells[s * V + site] = (unsigned char)(v > 255 ? 255 : v);
    }
}

/* Fast bound-state count (Sec. III.B): number of cells x with anchor[x] > 0
 * and other[y] > 0 for some y in x + {-tol..tol}^3. */
long orc_overlap(const orc_params* p, const unsigned char* anchor, const unsigned char* other,
                 int tol) {
  long count = 0;
  for (long z = 0; z < p->nz; ++z)
    for (long y = 0; y < p->ny; ++y)
      for (long x = 0; x < p->nx; ++x) {
        if (anchor[sidx(p, x, y, z)] == 0) continue;
        int hit = 0;
        for (int dz = -tol; dz <= tol && !hit; ++dz)
          for (int dy = -tol; dy <= tol && !hit; ++dy)
            for (int dx = -tol; dx <= tol && !hit; ++dx)
              if (other[sidx(p, x + dx, y + dy, z + dz)] > 0) hit = 1;
        count += hit;
      }
  return count;
}

/* The fast method's bound-state cells (Sec. III.B): mask[x] = 1 when
 * anchor[x] > 0 and other[y] > 0 for some y in x + {-tol..tol}^3. */
void orc_pq_mask(const orc_params* p, const unsigned char* anchor, const unsigned char* other, int tol,
                 unsigned char* mask) {
  for (long z = 0; z < p->nz; ++z)
    for (long y = 0; y < p->ny; ++y)
      for (long x = 0; x < p->nx; ++x) {
        long site = sidx(p, x, y, z);
        int hit = 0;
        if (anchor[site] > 0)
          for (int dz = -tol; dz <= tol && !hit; ++dz)
            for (int dy = -tol; dy <= tol && !hit; ++dy)
              for (int dx = -tol; dx <= tol && !hit; ++dx)
                if (other[sidx(p, x + dx, y + dy, z + dz)] > 0) hit = 1;
        mask[site] = (unsigned char)hit;
      }
}

/* Connected components of a cell mask on the periodic lattice, cells joined
 * when they share a face, an edge or a corner (26 neighbours): the
 * connectivity filter of the robust method (Sec. III.B).  label[x] is the
 * smallest site index of x's component, -1 outside the mask.  Breadth-first
 * search from every unlabelled mask cell in increasing index order, so the
 * start of each search is the smallest index of its component. */
void orc_components(const orc_params* p, const unsigned char* mask, long* label) {
  long V = nsites(p);
  long* queue = (long*)malloc(sizeof(long) * (size_t)V);
  for (long i = 0; i < V; ++i) label[i] = -1;
  for (long start = 0; start < V; ++start) {
    if (!mask[start] || label[start] >= 0) continue;
    long head = 0, tail = 0;
    queue[tail++] = start;
    label[start] = start;
    while (head < tail) {
      long c = queue[head++];
      long cx = c % p->nx, cy = (c / p->nx) % p->ny, cz = c / ((long)p->nx * p->ny);
      for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
          for (int dx = -1; dx <= 1; ++dx) {
            long nb = sidx(p, cx + dx, cy + dy, cz + dz);
            if (mask[nb] && label[nb] < 0) {
              label[nb] = start;
              queue[tail++] = nb;
            }
          }
    }
  }
  free(queue);
}

/* ---- network diagnostics (Sec. III.A, Eqs. 33, 36-37; Sec. IV) ---------- */

/* Neumaier compensated sum */
typedef struct { double s, c; } nsum;
static void nadd(nsum* a, double v) {
  double t = a->s + v;
  if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
  else a->c += (v - t) + a->s;
  a->s = t;
}

enum {
  D_KIN_P, D_KIN_Q, D_GRAD_P, D_GRAD_Q, D_EL_P, D_EL_Q, D_MAG_P, D_MAG_Q, D_POT, D_VINT,
  D_LAG, D_ENERGY, D_RL_NUM, D_RL_DEN, D_RPQ_NUM, D_RPQ_DEN,
  D_GAUSS_SUM_P, D_GAUSS_SUM_Q, D_CHARGE_SUM_P, D_CHARGE_SUM_Q,
  D_POT_P, D_POT_Q,
  D_NSUMS, /* compensated sums above, extrema below */
  D_GAUSS_MAX_P = D_NSUMS, D_GAUSS_MAX_Q, D_PHI_MIN_P, D_PHI_MAX_P, D_PHI_MIN_Q, D_PHI_MAX_Q,
  D_NAN, D_NOUT
};

int orc_diag_count(void) { return D_NOUT; }

/* Per-site diagnostic terms on the state at integer time n, summed over the
 * lattice (raw lattice sums; the dx^3 volume element is applied by the
 * caller).  The momenta enter as the mean of the squares at n-1/2 (stored)
 * and n+1/2 (recomputed here with the two kicks, not written back):
 *   kin_s  = (|pi^-|^2 + |pi^+|^2) / 2
 *   grad_s = sum_i |D_i^+ phi_s|^2
 *   el_s   = sum_i (E_i^-^2 + E_i^+^2) / 2 / (2 e_s^2 c_n)
 *   mag_s  = sum_{i<j} F_ij^2 / (2 e_s^2 c_n)
 *   pot    = c_n V(phi, psi), V of Eq. 4 with lambda_0, kappa_0
 *   pot_s  = c_n lambda_s/4 (|phi_s|^2 - sigma_s^2)^2, the self-potential of sector s
 *   vint   = kappa_0 (|phi|^2 - sigma_p^2)(|psi|^2 - sigma_q^2)
 *   L_x    = sum_s (kin - grad + el - mag) - pot           (Lagrangian)
 *   H_x    = sum_s (kin + grad + el + mag) + pot           (energy)
 * velocity estimator sums (Eq. 37) with weight W = L_x and W = vint:
 *   num = (kin_p + kin_q) W,  den = (grad_p + grad_q) W.
 * Gauss law (Eqs. 9-10) at time n-1/2 per sector:
 *   G(x) = sum_i (E_i(x) - E_i(x-i)) / dx - 2 e^2 ct_{n-1} Im[phi^{n*} pi^{n-1/2}]
 * with ct the charge factor of orc_coeffs; reported as sum |G|, sum |rho| (rho the charge term) and
 * max |G|.  work must hold 10 * V doubles. */
void orc_diagnostics(const orc_params* p, const double* st, long n, double* out, double* work) {
  static const int PI_[3] = {0, 0, 1}, PJ_[3] = {1, 2, 2};
  long V = nsites(p);
  double cf[6], cfm[6];
  orc_coeffs(p, n, cf);
  double c = cf[2];
  int have_prev = (p->eta0 + (double)(n - 1) * p->deta) > 0.0;
  orc_coeffs(p, n - 1, cfm);
  double ct_prev = have_prev ? cfm[5] : 0.0;

  orc_scalar_kick(p, st, n, work);
  orc_gauge_kick(p, st, n, work + 4 * V);
  const double* pi_new = work;
  const double* E_new = work + 4 * V;

  nsum acc[D_NSUMS];
  memset(acc, 0, sizeof(acc));
  double gmax[2] = {0.0, 0.0};
  double phimin[2] = {INFINITY, INFINITY}, phimax[2] = {0.0, 0.0};
  double nan_count = 0.0;

  for (long site = 0; site < V; ++site) {
    double kin[2], grad[2], el[2], mag[2], mod2[2];
    for (int s = 0; s < 2; ++s) {
      cplx f = get_phi(p, st, s, site);
      mod2[s] = cabs2(f);
      double pm2 = st[f_pi(s, 0) * V + site] * st[f_pi(s, 0) * V + site]
                 + st[f_pi(s, 1) * V + site] * st[f_pi(s, 1) * V + site];
      double pp2 = pi_new[(2 * s) * V + site] * pi_new[(2 * s) * V + site]
                 + pi_new[(2 * s + 1) * V + site] * pi_new[(2 * s + 1) * V + site];
      kin[s] = 0.5 * (pm2 + pp2);
      grad[s] = 0.0;
      double e2sum = 0.0;
      for (int i = 0; i < 3; ++i) {
        long xp = shift(p, site, i, +1);
        cplx fwd = cmul(link_U(p, st, s, i, site), get_phi(p, st, s, xp));
        cplx d = {(fwd.re - f.re) / p->dx, (fwd.im - f.im) / p->dx};
        grad[s] += cabs2(d);
        double em = st[f_E(s, i) * V + site], ep = E_new[(3 * s + i) * V + site];
        e2sum += 0.5 * (em * em + ep * ep);
      }
      double g = 1.0 / (2.0 * p->e[s] * p->e[s] * c);
      el[s] = g * e2sum;
      double f2 = 0.0;
      for (int k = 0; k < 3; ++k) {
        double F = plaq_F(p, st, s, PI_[k], PJ_[k], site);
        f2 += F * F;
      }
      mag[s] = g * f2;
    }
    double rp = mod2[0] - p->sigma[0] * p->sigma[0];
    double rq = mod2[1] - p->sigma[1] * p->sigma[1];
    double V0 = 0.25 * p->lambda[0] * rp * rp + 0.25 * p->lambda[1] * rq * rq - p->kappa * rp * rq;
    double pot = c * V0;
    double vint = p->kappa * rp * rq;
    double L = (kin[0] - grad[0] + el[0] - mag[0]) + (kin[1] - grad[1] + el[1] - mag[1]) - pot;
    double H = (kin[0] + grad[0] + el[0] + mag[0]) + (kin[1] + grad[1] + el[1] + mag[1]) + pot;
    double kt = kin[0] + kin[1], gt = grad[0] + grad[1];

    nadd(&acc[D_KIN_P], kin[0]);
    nadd(&acc[D_KIN_Q], kin[1]);
    nadd(&acc[D_GRAD_P], grad[0]);
    nadd(&acc[D_GRAD_Q], grad[1]);
    nadd(&acc[D_EL_P], el[0]);
    nadd(&acc[D_EL_Q], el[1]);
    nadd(&acc[D_MAG_P], mag[0]);
    nadd(&acc[D_MAG_Q], mag[1]);
    nadd(&acc[D_POT], pot);
    nadd(&acc[D_POT_P], c * 0.25 * p->lambda[0] * rp * rp);
    nadd(&acc[D_POT_Q], c * 0.25 * p->lambda[1] * rq * rq);
    nadd(&acc[D_VINT], vint);
    nadd(&acc[D_LAG], L);
    nadd(&acc[D_ENERGY], H);
    nadd(&acc[D_RL_NUM], kt * L);
    nadd(&acc[D_RL_DEN], gt * L);
    nadd(&acc[D_RPQ_NUM], kt * vint);
    nadd(&acc[D_RPQ_DEN], gt * vint);

    for (int s = 0; s < 2; ++s) {
      double div = 0.0;
      for (int i = 0; i < 3; ++i) {
        long xm = shift(p, site, i, -1);
        div += (st[f_E(s, i) * V + site] - st[f_E(s, i) * V + xm]) / p->dx;
      }
      /* Im[phi^{n-1*} pi] = Im[phi^{n*} pi] because phi^n - phi^{n-1} is
       * deta pi and Im|pi|^2 = 0; the stored phi^n is used directly */
      double pr = st[f_pi(s, 0) * V + site], pi = st[f_pi(s, 1) * V + site];
      double fr = st[f_phi(s, 0) * V + site], fi = st[f_phi(s, 1) * V + site];
      double rho = 2.0 * p->e[s] * p->e[s] * ct_prev * (fr * pi - fi * pr);
      double G = div - rho;
      nadd(&acc[D_GAUSS_SUM_P + s], fabs(G));
      nadd(&acc[D_CHARGE_SUM_P + s], fabs(rho));
      if (fabs(G) > gmax[s]) gmax[s] = fabs(G);
      double mod = sqrt(mod2[s]);
      if (mod < phimin[s]) phimin[s] = mod;
      if (mod > phimax[s]) phimax[s] = mod;
    }
    for (int f = 0; f < ORC_NFIELDS; ++f)
      if (isnan(st[f * V + site])) nan_count += 1.0;
  }
  for (int k = 0; k < D_NSUMS; ++k) out[k] = acc[k].s + acc[k].c;
  out[D_GAUSS_MAX_P] = gmax[0];
  out[D_GAUSS_MAX_Q] = gmax[1];
  out[D_PHI_MIN_P] = phimin[0];
  out[D_PHI_MAX_P] = phimax[0];
  out[D_PHI_MIN_Q] = phimin[1];
  out[D_PHI_MAX_Q] = phimax[1];
  out[D_NAN] = nan_count;
}

/* ---- threading control for the timed CPU baseline ----------------------- */

#ifdef _OPENMP
#include <omp.h>
#endif

void orc_set_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

int orc_max_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}
