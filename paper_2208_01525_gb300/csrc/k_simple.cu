// Initial conditions, the one-thread-per-site step/measure kernel, the cell
// overlap kernel and the reduction finalize kernel.
//
// k_simple is the plain form of the hot path: each thread updates whole
// sites (grid-stride), reading every neighbour value straight from global
// memory through the read-only cache and recomputing link phases it needs.
// It is the precision reference for the tiled kernel and the fallback shape
// for lattices too small to tile.
#include <stdint.h>

#include "reduce.cuh"
#include "site_math.cuh"
#include "state_copy.cuh"
#include "u1u1_internal.cuh"

namespace u1u1 {

namespace {

constexpr int SIMPLE_THREADS = 256;
constexpr int SIMPLE_BLOCKS = 152 * 8;

__device__ __forceinline__ int wrapc(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

struct Geo {
  int nx, ny, nz;
  __device__ long long idx(int x, int y, int z) const {
    return (long long)x + (long long)nx * ((long long)y + (long long)ny * z);
  }
  __device__ long long nb(int x, int y, int z, int ox, int oy, int oz) const {
    return idx(wrapc(x + ox, nx), wrapc(y + oy, ny), wrapc(z + oz, nz));
  }
};

// ---- initial conditions (Sec. III) ----------------------------------------

// SplitMix64 (Steele, Lea & Flood 2014): output number k of the generator
// whose state starts at x0 (the state advances by 0x9E3779B97F4A7C15 per
// draw; the output mixes the state with two xor-shift-multiply rounds).
__device__ __forceinline__ uint64_t splitmix64_draw(uint64_t x0, uint64_t k) {
  uint64_t z = x0 + (k + 1ull) * 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

template <typename T>
__global__ void k_init(LatticeView<T> v, LatticeView<T> v1, uint64_t seed, double sig_p, double sig_q) {
  const long long V = (long long)v.nx * v.ny * v.nz;
  T* pos0[U1U1_NPOS];
  for (int f = 0; f < U1U1_NPOS; ++f) pos0[f] = const_cast<T*>(v.pin[f]);
  for (long long site = blockIdx.x * (long long)blockDim.x + threadIdx.x; site < V;
       site += (long long)gridDim.x * blockDim.x) {
    for (int s = 0; s < 2; ++s) {
      uint64_t x0 = seed ^ ((uint64_t)s << 62);
      double u = (double)(splitmix64_draw(x0, (uint64_t)site) >> 11) * (1.0 / 9007199254740992.0);
      double th = (2.0 * 3.14159265358979323846) * u;
      double sn, cs;
      sincos(th, &sn, &cs);
      double sg = s == 0 ? sig_p : sig_q;
      pos0[2 * s][site] = (T)(sg * cs);
      pos0[2 * s + 1][site] = (T)(sg * sn);
      v1.pout[2 * s][site] = (T)0;
      v1.pout[2 * s + 1][site] = (T)0;
    }
    for (int f = 4; f < U1U1_NPOS; ++f) {
      pos0[f][site] = (T)0;
      v1.pout[f][site] = (T)0;
    }
    for (int f = 0; f < U1U1_NMOM; ++f) v.mom[f][site] = (T)0;
  }
}

// ---- the simple step / measure kernel ------------------------------------

template <typename T>
__device__ __forceinline__ T ld(const T* p, long long i) { return __ldg(p + i); }

// Edge product conj(phi(a)) U_d(a) phi(b) of sector s, link value Aval.
template <typename T>
__device__ __forceinline__ void edge_product(const LatticeView<T>& v, int s, long long a, long long b,
                                             T Aval, T dx, T* re, T* im) {
  T sn, cs;
  link_sincos<T>(dx * Aval, &sn, &cs);
  T br, bi;
  transport_fwd<T>(cs, sn, ld(v.pin[2 * s], b), ld(v.pin[2 * s + 1], b), &br, &bi);
  T ar = ld(v.pin[2 * s], a), ai = ld(v.pin[2 * s + 1], a);
  *re = ar * br + ai * bi;
  *im = ar * bi - ai * br;
}

template <typename T, int MODE>
__global__ void __launch_bounds__(SIMPLE_THREADS)
k_simple(LatticeView<T> v, Coef<T> c, MeasureOut mo) {
  constexpr bool WRITE = (MODE & MODE_WRITE) != 0;
  constexpr bool MEAS = (MODE & MODE_MEASURE) != 0;
  constexpr bool GAUSS = (MODE & MODE_GAUSS) != 0;
  static_assert(!(WRITE && GAUSS), "Gauss needs unmodified neighbour momenta");
  const Geo g{v.nx, v.ny, v.nz};
  const long long V = (long long)v.nx * v.ny * v.nz;
  ThreadAcc acc;
  if (MEAS) acc.zero();

  for (long long site = blockIdx.x * (long long)blockDim.x + threadIdx.x; site < V;
       site += (long long)gridDim.x * blockDim.x) {
    const int x = (int)(site % v.nx);
    const int y = (int)((site / v.nx) % v.ny);
    const int z = (int)(site / ((long long)v.nx * v.ny));
    long long xp[3], xm[3];
    xp[0] = g.nb(x, y, z, 1, 0, 0); xm[0] = g.nb(x, y, z, -1, 0, 0);
    xp[1] = g.nb(x, y, z, 0, 1, 0); xm[1] = g.nb(x, y, z, 0, -1, 0);
    xp[2] = g.nb(x, y, z, 0, 0, 1); xm[2] = g.nb(x, y, z, 0, 0, -1);

    SectorIn<T> in[2];
    T pr[2], pim[2], E[2][3];
    for (int s = 0; s < 2; ++s) {
      const T* Fr = v.pin[2 * s];
      const T* Fi = v.pin[2 * s + 1];
      const T* A0 = v.pin[4 + 3 * s];
      const T* A1 = v.pin[5 + 3 * s];
      const T* A2 = v.pin[6 + 3 * s];
      SectorIn<T>& q = in[s];
      q.fr = ld(Fr, site);
      q.fi = ld(Fi, site);
      for (int i = 0; i < 3; ++i) {
        const T* Ai = v.pin[4 + 3 * s + i];
        q.A[i] = ld(Ai, site);
        T sn, cs;
        link_sincos<T>(c.dx * q.A[i], &sn, &cs);
        transport_fwd<T>(cs, sn, ld(Fr, xp[i]), ld(Fi, xp[i]), &q.fwr[i], &q.fwi[i]);
        link_sincos<T>(c.dx * ld(Ai, xm[i]), &sn, &cs);
        transport_bwd<T>(cs, sn, ld(Fr, xm[i]), ld(Fi, xm[i]), &q.bwr[i], &q.bwi[i]);
      }
      q.F[0] = curl_ft<T>(ld(A1, xp[0]), q.A[1], ld(A0, xp[1]), q.A[0]);
      q.F[1] = curl_ft<T>(ld(A2, xp[0]), q.A[2], ld(A0, xp[2]), q.A[0]);
      q.F[2] = curl_ft<T>(ld(A2, xp[1]), q.A[2], ld(A1, xp[2]), q.A[1]);
      q.Fm[0] = curl_ft<T>(ld(A1, g.nb(x, y, z, 1, -1, 0)), ld(A1, xm[1]), q.A[0], ld(A0, xm[1]));
      q.Fm[1] = curl_ft<T>(q.A[1], ld(A1, xm[0]), ld(A0, g.nb(x, y, z, -1, 1, 0)), ld(A0, xm[0]));
      q.Fm[2] = curl_ft<T>(ld(A2, g.nb(x, y, z, 1, 0, -1)), ld(A2, xm[2]), q.A[0], ld(A0, xm[2]));
      q.Fm[3] = curl_ft<T>(q.A[2], ld(A2, xm[0]), ld(A0, g.nb(x, y, z, -1, 0, 1)), ld(A0, xm[0]));
      q.Fm[4] = curl_ft<T>(ld(A2, g.nb(x, y, z, 0, 1, -1)), ld(A2, xm[2]), q.A[1], ld(A1, xm[2]));
      q.Fm[5] = curl_ft<T>(q.A[2], ld(A2, xm[1]), ld(A1, g.nb(x, y, z, 0, -1, 1)), ld(A1, xm[1]));
      pr[s] = v.mom[2 * s][site];
      pim[s] = v.mom[2 * s + 1][site];
      for (int i = 0; i < 3; ++i) E[s][i] = v.mom[4 + 3 * s + i][site];
    }

    T mod2[2] = {in[0].fr * in[0].fr + in[0].fi * in[0].fi, in[1].fr * in[1].fr + in[1].fi * in[1].fi};
    T rr[2] = {mod2[0] - c.sig2[0], mod2[1] - c.sig2[1]};
    T prn[2], pin_[2], En[2][3];
    for (int s = 0; s < 2; ++s) {
      scalar_kick<T>(in[s], rr[s], rr[1 - s], pr[s], pim[s], c, s, &prn[s], &pin_[s]);
      gauge_kick<T>(in[s], E[s], c, s, En[s]);
    }

    if (WRITE) {
      for (int s = 0; s < 2; ++s) {
        v.mom[2 * s][site] = prn[s];
        v.mom[2 * s + 1][site] = pin_[s];
        v.pout[2 * s][site] = in[s].fr + c.deta * prn[s];
        v.pout[2 * s + 1][site] = in[s].fi + c.deta * pin_[s];
        for (int i = 0; i < 3; ++i) {
          v.mom[4 + 3 * s + i][site] = En[s][i];
          v.pout[4 + 3 * s + i][site] = in[s].A[i] + c.deta * En[s][i];
        }
      }
    }

    if (MEAS) {
      // diagnostic densities
      SectorDiag<T> d[2];
      for (int s = 0; s < 2; ++s) d[s] = sector_diag<T>(in[s], pr[s], pim[s], prn[s], pin_[s], E[s], En[s], c, s);
      T rp = rr[0], rq = rr[1];
      T pot = c.cV * (c.lam4[0] * rp * rp + c.lam4[1] * rq * rq - c.kappa * rp * rq);
      T vint = c.kappa * rp * rq;
      T L = (d[0].kin - d[0].grad + d[0].el - d[0].mag) + (d[1].kin - d[1].grad + d[1].el - d[1].mag) - pot;
      T kt = d[0].kin + d[1].kin, gt = d[0].grad + d[1].grad;
      acc.s[S_KIN_P] += (double)d[0].kin;
      acc.s[S_KIN_Q] += (double)d[1].kin;
      acc.s[S_GRAD_P] += (double)d[0].grad;
      acc.s[S_GRAD_Q] += (double)d[1].grad;
      acc.s[S_EL_P] += (double)d[0].el;
      acc.s[S_EL_Q] += (double)d[1].el;
      acc.s[S_MAG_P] += (double)d[0].mag;
      acc.s[S_MAG_Q] += (double)d[1].mag;
      acc.s[S_POT] += (double)pot;
      acc.s[S_POT_P] += (double)(c.cV * c.lam4[0] * rp * rp);
      acc.s[S_POT_Q] += (double)(c.cV * c.lam4[1] * rq * rq);
      acc.s[S_VINT] += (double)vint;
      acc.s[S_RL_NUM] += (double)(kt * L);
      acc.s[S_RL_DEN] += (double)(gt * L);
      acc.s[S_RPQ_NUM] += (double)(kt * vint);
      acc.s[S_RPQ_DEN] += (double)(gt * vint);
      for (int s = 0; s < 2; ++s) {
        T m = sqrt(mod2[s]);
        acc.mx[s == 0 ? M_NEG_PHIMIN_P : M_NEG_PHIMIN_Q] = fmax(acc.mx[s == 0 ? M_NEG_PHIMIN_P : M_NEG_PHIMIN_Q], -(double)m);
        acc.mx[s == 0 ? M_PHIMAX_P : M_PHIMAX_Q] = fmax(acc.mx[s == 0 ? M_PHIMAX_P : M_PHIMAX_Q], (double)m);
      }
      long long nan = 0;
      for (int f = 0; f < U1U1_NPOS; ++f) nan += isnan(ld(v.pin[f], site)) ? 1 : 0;
      for (int s = 0; s < 2; ++s) {
        nan += isnan(pr[s]) ? 1 : 0;
        nan += isnan(pim[s]) ? 1 : 0;
        for (int i = 0; i < 3; ++i) nan += isnan(E[s][i]) ? 1 : 0;
      }
      acc.cnt[C_NAN] += nan;

      if (GAUSS) {
        for (int s = 0; s < 2; ++s) {
          T div = T(0);
          for (int i = 0; i < 3; ++i) div += E[s][i] - v.mom[4 + 3 * s + i][xm[i]];
          div *= c.inv_dx;
          T rho = c.qG[s] * (in[s].fr * pim[s] - in[s].fi * pr[s]);
          T G = div - rho;
          acc.s[s == 0 ? S_GAUSS_P : S_GAUSS_Q] += fabs((double)G);
          acc.s[s == 0 ? S_CHARGE_P : S_CHARGE_Q] += fabs((double)rho);
          acc.mx[s == 0 ? M_GAUSS_P : M_GAUSS_Q] = fmax(acc.mx[s == 0 ? M_GAUSS_P : M_GAUSS_Q], fabs((double)G));
        }
      }

      // plaquette windings of both sectors (Sec. III.A)
      int W[2][3];
      bool cutk[2][3];
      for (int s = 0; s < 2; ++s) {
        const SectorIn<T>& q = in[s];
        bool cut_own[3] = {false, false, false};
        T chi_own[3];
        for (int i = 0; i < 3; ++i) chi_own[i] = edge_chi<T>(current_re(q, i), current_im(q, i), &cut_own[i]);
        // neighbour edges: chi_1(x+x), chi_0(x+y), chi_2(x+x), chi_0(x+z), chi_2(x+y), chi_1(x+z)
        T re, im;
        bool c1x = false, c0y = false, c2x = false, c0z = false, c2y = false, c1z = false;
        edge_product<T>(v, s, xp[0], g.nb(x, y, z, 1, 1, 0), ld(v.pin[5 + 3 * s], xp[0]), c.dx, &re, &im);
        T chi1_xpx = edge_chi<T>(re, im, &c1x);
        edge_product<T>(v, s, xp[1], g.nb(x, y, z, 1, 1, 0), ld(v.pin[4 + 3 * s], xp[1]), c.dx, &re, &im);
        T chi0_xpy = edge_chi<T>(re, im, &c0y);
        edge_product<T>(v, s, xp[0], g.nb(x, y, z, 1, 0, 1), ld(v.pin[6 + 3 * s], xp[0]), c.dx, &re, &im);
        T chi2_xpx = edge_chi<T>(re, im, &c2x);
        edge_product<T>(v, s, xp[2], g.nb(x, y, z, 1, 0, 1), ld(v.pin[4 + 3 * s], xp[2]), c.dx, &re, &im);
        T chi0_xpz = edge_chi<T>(re, im, &c0z);
        edge_product<T>(v, s, xp[1], g.nb(x, y, z, 0, 1, 1), ld(v.pin[6 + 3 * s], xp[1]), c.dx, &re, &im);
        T chi2_xpy = edge_chi<T>(re, im, &c2y);
        edge_product<T>(v, s, xp[2], g.nb(x, y, z, 0, 1, 1), ld(v.pin[5 + 3 * s], xp[2]), c.dx, &re, &im);
        T chi1_xpz = edge_chi<T>(re, im, &c1z);
        W[s][0] = plaquette_winding<T>(chi_own[0], chi1_xpx, chi0_xpy, chi_own[1], c.dx, q.F[0]);
        W[s][1] = plaquette_winding<T>(chi_own[0], chi2_xpx, chi0_xpz, chi_own[2], c.dx, q.F[1]);
        W[s][2] = plaquette_winding<T>(chi_own[1], chi2_xpy, chi1_xpz, chi_own[2], c.dx, q.F[2]);
        cutk[s][0] = cut_own[0] || c1x || c0y || cut_own[1];
        cutk[s][1] = cut_own[0] || c2x || c0z || cut_own[2];
        cutk[s][2] = cut_own[1] || c2y || c1z || cut_own[2];
      }
      for (int s = 0; s < 2; ++s) {
        unsigned byte = 0;
        for (int k = 0; k < 3; ++k) {
          int a = abs(W[s][k]);
          acc.cnt[s == 0 ? C_NP : C_NQ] += a;
          acc.cnt[s == 0 ? C_NZP : C_NZQ] += (a != 0);
          acc.cnt[C_FLAGGED] += cutk[s][k] ? 1 : 0;
          acc.cnt[C_MAXW] = max(acc.cnt[C_MAXW], (long long)a);
          acc.cnt[s == 0 ? C_W2P : C_W2Q] += (a >= 2);
          byte |= (unsigned)min(a, 3) << FACE_SHIFT(k);
          if (cutk[s][k]) byte |= FACE_FLAG;
          if (mo.windings) mo.windings[(3 * s + k) * V + site] = (int8_t)max(-127, min(127, W[s][k]));
        }
        if (mo.faces) mo.faces[s * V + site] = (uint8_t)byte;
      }
      for (int k = 0; k < 3; ++k) acc.cnt[C_NPQ_PLAQ] += (W[0][k] != 0 && W[1][k] != 0) ? 1 : 0;
    }
  }

  if (MEAS) {
    __shared__ ReduceSmem<SIMPLE_THREADS / 32> sm;
    block_reduce<SIMPLE_THREADS / 32>(acc, sm, mo.partial + blockIdx.x);
  }
}

__global__ void k_link_phase(const float* __restrict__ th, float* sn, float* cs, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    link_sincos<float>(th[i], &sn[i], &cs[i]);
}

__global__ void k_link_phase64(const double* __restrict__ th, double* sn, double* cs, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    link_sincos<double>(th[i], &sn[i], &cs[i]);
}

__global__ void k_edge_phase(const float* __restrict__ re, const float* __restrict__ im, float* out, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
    out[i] = edge_phase<float>(re[i], im[i]);
}

// One launch moves every field of the table; 16-byte words, grid-stride.
__global__ void __launch_bounds__(256) k_state_copy(const __grid_constant__ XferTable t, long long n16) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (int f = 0; f < t.m; ++f) {
    const uint4* __restrict__ src = static_cast<const uint4*>(t.src[f]);
    uint4* __restrict__ dst = static_cast<uint4*>(t.dst[f]);
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n16; i += stride) dst[i] = src[i];
  }
}

}  // namespace

cudaError_t launch_state_copy(const XferTable& t, long long n16, cudaStream_t st) {
  if (t.m <= 0 || n16 <= 0) return cudaSuccess;
  k_state_copy<<<152 * 8, 256, 0, st>>>(t, n16);
  return cudaGetLastError();
}

cudaError_t launch_edge_phase(const float* re, const float* im, float* out, long long n, cudaStream_t st) {
  k_edge_phase<<<152 * 4, 256, 0, st>>>(re, im, out, n);
  return cudaGetLastError();
}

cudaError_t launch_link_phase(const float* th, float* sn, float* cs, long long n, cudaStream_t st) {
  k_link_phase<<<152 * 4, 256, 0, st>>>(th, sn, cs, n);
  return cudaGetLastError();
}

cudaError_t launch_link_phase64(const double* th, double* sn, double* cs, long long n, cudaStream_t st) {
  k_link_phase64<<<152 * 4, 256, 0, st>>>(th, sn, cs, n);
  return cudaGetLastError();
}

// ---- launchers ---------------------------------------------------------------

template <typename T>
cudaError_t launch_init(const LatticeView<T>& v, T* pos1[U1U1_NPOS], uint64_t seed, double sigma_p,
                        double sigma_q, cudaStream_t st) {
  LatticeView<T> v1 = v;
  for (int f = 0; f < U1U1_NPOS; ++f) v1.pout[f] = pos1[f];
  k_init<T><<<152 * 8, 256, 0, st>>>(v, v1, seed, sigma_p, sigma_q);
  return cudaGetLastError();
}

int simple_grid_blocks() { return SIMPLE_BLOCKS; }

template <typename T>
cudaError_t launch_simple(int mode, const LatticeView<T>& v, const Coef<T>& c, const MeasureOut& mo,
                          cudaStream_t st) {
  switch (mode) {
    case MODE_WRITE:
      k_simple<T, MODE_WRITE><<<SIMPLE_BLOCKS, SIMPLE_THREADS, 0, st>>>(v, c, mo);
      break;
    case MODE_WRITE | MODE_MEASURE:
      k_simple<T, MODE_WRITE | MODE_MEASURE><<<SIMPLE_BLOCKS, SIMPLE_THREADS, 0, st>>>(v, c, mo);
      break;
    case MODE_MEASURE | MODE_GAUSS:
      k_simple<T, MODE_MEASURE | MODE_GAUSS><<<SIMPLE_BLOCKS, SIMPLE_THREADS, 0, st>>>(v, c, mo);
      break;
    case MODE_MEASURE:
      k_simple<T, MODE_MEASURE><<<SIMPLE_BLOCKS, SIMPLE_THREADS, 0, st>>>(v, c, mo);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  return cudaGetLastError();
}

template cudaError_t launch_init<float>(const LatticeView<float>&, float* [U1U1_NPOS], uint64_t, double,
                                        double, cudaStream_t);
template cudaError_t launch_init<double>(const LatticeView<double>&, double* [U1U1_NPOS], uint64_t,
                                         double, double, cudaStream_t);
template cudaError_t launch_simple<float>(int, const LatticeView<float>&, const Coef<float>&,
                                          const MeasureOut&, cudaStream_t);
template cudaError_t launch_simple<double>(int, const LatticeView<double>&, const Coef<double>&,
                                           const MeasureOut&, cudaStream_t);

}  // namespace u1u1
