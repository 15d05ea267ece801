// Tiled z-marching kernel for the fused leapfrog step (Sec. III, Eqs. 17-26),
// optionally fused with plaquette-winding detection (Sec. III.A) and the
// diagnostic sums (Eqs. 33, 36-37).
//
// Each CTA owns a TX x TY column of sites and marches up a chunk of z-planes.
// The ten position fields of planes z, z+1 (read) and z+2 (in flight) sit
// in a three-plane shared-memory ring with a one-site halo in x and y, filled
// with cp.async (16-byte chunks for the interior, element copies for the x
// halo).  Per plane, phase 1 computes every site-local quantity a neighbour
// needs -- the backward-transported scalars conj(U_i) phi, the plaquette
// curls dx F_ij and, when detecting, the gauge-invariant edge phases -- once,
// including the halo points, into shared memory; phase 2 assembles the kicks
// and the drift from those and streams momenta (in place) and positions (to
// the other ping-pong buffer) out.  Quantities of the plane below the
// current one (z-direction backward terms) are carried in registers, so each
// position value is read from HBM once per step and each link phase is
// evaluated once.
#include <cuda.h>
#include <stdint.h>
#include <string.h>

#include "reduce.cuh"
#include "site_math.cuh"
#include "u1u1_internal.cuh"

namespace u1u1 {

namespace {

__device__ __forceinline__ int wrapm(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem));
}
template <int BYTES>
__device__ __forceinline__ void cp_async_small(void* smem, const void* gmem) {
  unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }
__device__ __forceinline__ void cp_async_wait0() { asm volatile("cp.async.wait_group 0;\n" ::); }

// ---- tensor-memory-access (TMA) copies of the position ring ----------------
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ long long gtimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}
__device__ __forceinline__ void mbar_init(unsigned long long* m) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(m)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* m, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(m)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* m, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(m)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of m to complete, for at most `limit` ns (2 s);
// true when it did.  Past the limit the launching handle's status word is
// set to U1U1_ERR_TIMEOUT for the host and the CTA's flag is set, after which
// the CTA's later waits give up at once
// (they still return, so every thread reaches every barrier) and the
// thread that issues the copies issues no more (re-arming a slot whose phase
// never completed would be an arrival too many); the CTA finishes on stale
// data.  A timed-out wait has given the slot's copies the whole limit to
// land before the CTA can exit.
// (The plan's status pointer is read only on that path: for ensembles the
// plan lives in device memory, and a load per wait would sit on every
// plane's critical path.)
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* m, unsigned parity, volatile int* cta_fail,
                                                  long long limit, const TmaPlan* plan) {
  if (mbar_try_wait(m, parity)) return true;
  if (*cta_fail) return false;
  const long long t0 = gtimer_ns();
  while (!mbar_try_wait(m, parity)) {
    if (gtimer_ns() - t0 > limit) {
      int* status = plan->status;
      if (status) atomicExch(status, U1U1_ERR_TIMEOUT);
      *cta_fail = 1;
      return false;
    }
  }
  return true;
}

// tensor copy of the box at (x, y, z) of `map` into shared memory at dst,
// completing on m
__device__ __forceinline__ void tma_load_3d(void* dst, const CUtensorMap* map, int x, int y, int z,
                                            unsigned long long* m) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];"
      ::"r"(smem_u32(dst)), "l"((unsigned long long)map), "r"(x), "r"(y), "r"(z), "r"(smem_u32(m))
      : "memory");
}

template <typename T, int TX, int TY>
struct Tile {
  static constexpr int VEC = 16 / sizeof(T);  // elements per 16-byte chunk
  static constexpr int RS = TX + 2 * VEC;     // smem row stride (elements)
  static constexpr int ROWS = TY + 2;         // rows ly = -1 .. TY
  static constexpr int PLANE = ROWS * RS;     // one field, one plane
  // field stride of the position ring: a plane rounded up to 128 bytes, the
  // alignment of a tensor-copy destination
  static constexpr int PSTRIDE = (PLANE * (int)sizeof(T) + 127) / 128 * 128 / (int)sizeof(T);
  static constexpr int OFF = VEC;             // column of lx = 0
  static constexpr int NT = TX * TY;
  static constexpr int CH = TX / VEC;         // interior chunks per row
  static_assert(TX % VEC == 0, "TX must be a multiple of the 16-byte vector");
  static __device__ __forceinline__ int at(int ly, int lx) { return (ly + 1) * RS + OFF + lx; }
};

// Sums a thread accumulates per site: all but the Lagrangian and the energy
// (formed from the component sums on the host), the Gauss-law sums only in
// the variant that computes the residual.
__host__ __device__ constexpr bool acc_used(int k, bool gauss) {
  return k != S_LAG && k != S_ENERGY &&
         (gauss || (k != S_GAUSS_P && k != S_GAUSS_Q && k != S_CHARGE_P && k != S_CHARGE_Q));
}
// slot of sum k among the accumulated ones
__host__ __device__ constexpr int acc_slot(int k, bool gauss) {
  int j = 0;
  for (int i = 0; i < k; ++i) j += acc_used(i, gauss) ? 1 : 0;
  return j;
}

// Shared memory of one CTA; the detection and Gauss arrays shrink to one
// element when the kernel variant does not use them.
template <typename T, int TX, int TY, bool MEAS = true, bool GAUSS = true>
struct Smem {
  using TL = Tile<T, TX, TY>;
  static constexpr int PG = GAUSS ? TL::PLANE : 1;
  T pos[3][U1U1_NPOS][TL::PSTRIDE];    // position ring
  T P[2][2][2][TL::PLANE];             // [sector][dir 0,1][re,im] conj(U_i) phi
  T Ft[2][3][TL::PLANE];               // [sector][plane] dx F at this plane
  T Eg[2][2][PG];                      // [sector][dir 0,1] E for the Gauss divergence
  // per-warp running sums of the detection densities, compensated (value,
  // correction) pairs in the working precision: adding in FP64 here would
  // run on GB300's narrow FP64 pipe once per warp, sum and plane
  T wsum[MEAS ? TL::NT / 32 : 1][NSUM];
  T wcmp[MEAS ? TL::NT / 32 : 1][NSUM];
  // FP32 detection: each thread keeps plain sums over up to ACC_PLANES
  // planes in registers (NACC of them), folded into the warp sums once per
  // ACC_PLANES planes.  Registers rather than shared memory: the measuring
  // variants run at two CTAs per SM and have the registers to spare, and a
  // shared-memory read-modify-write per sum and site cost 2.5 ms per
  // detection step and 4 ms per diagnostics pass at 1024^3.
  static constexpr bool ACC = MEAS && sizeof(T) == 4;
  static constexpr int NACC = acc_slot(NSUM, GAUSS);
  // completion of the tensor copies into each ring slot (interior tiles),
  // and whether a wait for them gave up
  unsigned long long mbar[3];
  int tma_fail;
};

// Planes a thread sums in plain FP32 before its partials join the warp's
// compensated sums (bounds that stage's rounding by 15 ulp of the partial).
constexpr int ACC_PLANES = 16;

// Copy plan of one thread: every copy moves one 16-byte chunk of one row of
// one field.  A row of the smem ring holds TX + 2 VEC elements: the chunk
// ending at x0-1 (left halo), the TX interior elements and the chunk starting
// at x0+TX (right halo), so the x halo comes for free with 16-byte copies.
// The per-plane part of a copy is only the z offset; everything else is
// computed once per CTA.
template <typename T, int TX, int TY>
struct CopyPlan {
  using TL = Tile<T, TX, TY>;
  static constexpr int PER_ROW = TL::CH + 2;
  static constexpr int JOBS = U1U1_NPOS * TL::ROWS * PER_ROW;
  static constexpr int NJ = (JOBS + TL::NT - 1) / TL::NT;
  const T* g[NJ];   // global address of the chunk in plane z = 0
  int s[NJ];        // element offset inside one ring buffer (-1: no job)

  __device__ void init(const LatticeView<T>& v, int x0, int y0) {
#pragma unroll
    for (int k = 0; k < NJ; ++k) {
      const int job = threadIdx.x + k * TL::NT;
      s[k] = -1;
      g[k] = nullptr;
      if (job < JOBS) {
        const int f = job / (TL::ROWS * PER_ROW);
        const int r = (job / PER_ROW) % TL::ROWS;
        const int c = job % PER_ROW;  // 0: left halo chunk, 1..CH: interior, CH+1: right halo
        const int gy = wrapm(y0 + r - 1, v.ny);
        const int gx = wrapm(x0 + (c - 1) * TL::VEC, v.nx);
        g[k] = v.pin[f] + (long long)gy * v.nx + gx;
        s[k] = f * TL::PSTRIDE + r * TL::RS + c * TL::VEC;
      }
    }
  }
  __device__ __forceinline__ void issue(T* ring_buf, long long zoff) const {
#pragma unroll
    for (int k = 0; k < NJ; ++k)
      if (s[k] >= 0) cp_async16(ring_buf + s[k], g[k] + zoff);
  }
};
// Halo point handled by thread tid, or -1: the TX + TY halo points of a
// plane go to the first threads, so they cost one or two warp passes
// (spreading them over all warps costs one pass per warp, measured slower).
template <int NT, int NH>
__device__ __forceinline__ int halo_point(int tid) {
  static_assert(NH <= NT, "more halo points than threads");
  return tid < NH ? tid : -1;
}

// Momentum loads.  Within one kernel launch a tile's momenta may have been
// written by another CTA (persistent ensemble kernel), so that variant
// bypasses L1 (ld.global.cg); the per-step kernels use plain loads.
template <bool COHERENT, typename T>
__device__ __forceinline__ T ld_mom(const T* p) {
  if (COHERENT) return __ldcg(p);
  return *p;
}

// A field store of the step: streaming (st.global.cs) or plain.
template <bool STREAM, typename T>
__device__ __forceinline__ void st_field(T* p, T x) {
  if (STREAM)
    __stcs(p, x);
  else
    *p = x;
}

// One tile column (tile (bx, by), planes [z0, z1)) of a step or measuring
// pass; `bid` indexes the block partial of a measuring pass.
// HOOKS: the plan's test-hook fields are read (single-lattice kernels, whose
// plan is a kernel parameter); ensemble kernels, whose plans live in device
// memory, use the exact slot size and the 2 s limit instead.
// STREAM: the step's stores (new positions, momenta) are streaming stores,
// evict-first in L2, which leaves L2 to the position planes that
// neighbouring tiles re-read as halos.  Measured at 1024^3: the plain step
// 27.59 against 28.18 ms, DRAM reads +2.0 % instead of +3.0 % over the
// algorithmic bytes.  The measuring step keeps plain stores (35.5 against
// 35.2 ms per launch with streaming stores), and so do the ensemble kernels:
// with streaming stores their 32-plane work items ran 2 % slower and
// 64-plane ones no faster.
template <typename T, int TX, int TY, int MODE, bool COHERENT, bool HOOKS = true, bool STREAM = false>
__device__ __forceinline__ void tile_run(unsigned char* smem_raw, const LatticeView<T>& v, const Coef<T>& c,
                                         const MeasureOut& mo, int bx, int by, int z0, int z1, int bid,
                                         const TmaPlan* tma) {
  using TL = Tile<T, TX, TY>;
  constexpr bool WRITE = (MODE & MODE_WRITE) != 0;
  constexpr bool MEAS = (MODE & MODE_MEASURE) != 0;
  constexpr bool GAUSS = (MODE & MODE_GAUSS) != 0;
  static_assert(!(WRITE && GAUSS), "Gauss needs unmodified neighbour momenta");
  using SM = Smem<T, TX, TY, MEAS, GAUSS>;
  SM& sm = *reinterpret_cast<SM*>(smem_raw);

  const int tid = threadIdx.x;
  const int lx = tid % TX, ly = tid / TX;
  const int x0 = bx * TX, y0 = by * TY;
  const int gx = x0 + lx, gy = y0 + ly;
  const bool active = gx < v.nx && gy < v.ny;
  const long long plane = (long long)v.nx * v.ny;
  const long long V = plane * v.nz;
  const T dx = c.dx;

  T mx[NMAX];
  int cnt[NCNT];
  T racc[SM::ACC ? SM::NACC : 1];
#pragma unroll
  for (int k = 0; k < (SM::ACC ? SM::NACC : 1); ++k) racc[k] = T(0);
  if (MEAS) {
    if ((tid & 31) == 0)
      for (int k = 0; k < NSUM; ++k) sm.wsum[tid >> 5][k] = sm.wcmp[tid >> 5][k] = T(0);

#pragma unroll
    for (int k = 0; k < NMAX; ++k) mx[k] = -INFINITY;  // -inf is representable in T
#pragma unroll
    for (int k = 0; k < NCNT; ++k) cnt[k] = 0;
  }

  // ---- prologue: planes z0-1, z0, z0+1 in flight; backward-z carries ----
  // Interior tiles (the halo inside the lattice) load their ring slots with
  // one tensor copy per field, issued by thread 0 and completing on the
  // slot's mbarrier; tiles at the lattice's edges, whose halo wraps around,
  // use the cp.async plan.  So does the Gauss-residual variant: with tensor
  // copies it ran 15% slower (the other variants gain or break even).
  const bool use_tma = !GAUSS && x0 >= TL::VEC && x0 + TX + TL::VEC <= v.nx && y0 >= 1 && y0 + TY + 1 <= v.ny &&
                       tma != nullptr && tma->enabled;
  constexpr unsigned SLOT_BYTES = U1U1_NPOS * TL::ROWS * TL::RS * sizeof(T);
  const unsigned slot_expect = (HOOKS && use_tma) ? SLOT_BYTES + tma->extra_bytes : SLOT_BYTES;
  const long long wait_limit = (HOOKS && use_tma) ? tma->limit_ns : 2000000000LL;
  unsigned phase = 0u;  // bit k: parity of slot k's next completion
  CopyPlan<T, TX, TY> cpl;
  auto zoff = [&](int z) { return (long long)wrapm(z, v.nz) * plane; };
  auto tma_issue = [&](int slot, int z) {  // thread 0 only
    mbar_expect_tx(&sm.mbar[slot], slot_expect);
#pragma unroll
    for (int f = 0; f < U1U1_NPOS; ++f)
      tma_load_3d(&sm.pos[slot][f][0], &tma->map[f], x0 - TL::VEC, y0 - 1, wrapm(z, v.nz), &sm.mbar[slot]);
  };
  bool copies_ok = true;  // every wait of this thread completed
  auto tma_wait = [&](int slot) {
    copies_ok = mbar_wait_bounded(&sm.mbar[slot], (phase >> slot) & 1u, &sm.tma_fail, wait_limit, tma) && copies_ok;
    phase ^= 1u << slot;
  };
  if (use_tma) {
    if (tid == 0) {
      // order any earlier generic accesses to the ring before the copies
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      sm.tma_fail = 0;
#pragma unroll
      for (int k = 0; k < 3; ++k) mbar_init(&sm.mbar[k]);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
#pragma unroll
      for (int k = 0; k < 3; ++k) tma_issue(k, z0 - 1 + k);
    }
    __syncthreads();  // the barriers are initialised before anyone waits
    tma_wait(0);
    tma_wait(1);
  } else {
    cpl.init(v, x0, y0);
    cpl.issue(&sm.pos[0][0][0], zoff(z0 - 1));
    cp_async_commit();
    cpl.issue(&sm.pos[1][0][0], zoff(z0));
    cp_async_commit();
    cpl.issue(&sm.pos[2][0][0], zoff(z0 + 1));
    cp_async_commit();
    cp_async_wait1();
  }
  __syncthreads();

  // carries: conj(U_2) phi, dx F_02, dx F_12 at (x, z-1), and E_2(x, z-1)
  T cP2r[2], cP2i[2], cF02[2], cF12[2], cE2[2];
  {
    const int a = TL::at(ly, lx);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      T sn, cs;
      link_sincos<T>(dx * sm.pos[0][6 + 3 * s][a], &sn, &cs);
      transport_bwd<T>(cs, sn, sm.pos[0][2 * s][a], sm.pos[0][2 * s + 1][a], &cP2r[s], &cP2i[s]);
      const T* A0 = sm.pos[0][4 + 3 * s];
      const T* A1 = sm.pos[0][5 + 3 * s];
      const T* A2 = sm.pos[0][6 + 3 * s];
      cF02[s] = curl_ft<T>(A2[TL::at(ly, lx + 1)], A2[a], sm.pos[1][4 + 3 * s][a], A0[a]);
      cF12[s] = curl_ft<T>(A2[TL::at(ly + 1, lx)], A2[a], sm.pos[1][5 + 3 * s][a], A1[a]);
      cE2[s] = T(0);
      if (GAUSS && active)
        cE2[s] = ld_mom<COHERENT>(&v.mom[6 + 3 * s][(long long)wrapm(z0 - 1, v.nz) * plane + (long long)gy * v.nx + gx]);
    }
  }

  // momenta of the next plane, issued a plane ahead so that their loads are
  // in flight across the barrier and phase 1 (consumed in phase 2)
  T npr[2], npim[2], nE[2][3];
  auto load_mom = [&](int zz) {
    const long long gs = (long long)zz * plane + (long long)gy * v.nx + gx;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      npr[s] = active ? ld_mom<COHERENT>(&v.mom[2 * s][gs]) : T(0);
      npim[s] = active ? ld_mom<COHERENT>(&v.mom[2 * s + 1][gs]) : T(0);
#pragma unroll
      for (int i = 0; i < 3; ++i) nE[s][i] = active ? ld_mom<COHERENT>(&v.mom[4 + 3 * s + i][gs]) : T(0);
    }
  };
  load_mom(z0);

  for (int z = z0; z < z1; ++z) {
    const int it = z - z0;
    const int bc = (it + 1) % 3, bn = (it + 2) % 3, bf = it % 3;
    // plane z+1 (the only copy in flight) has landed; after the barrier
    // every thread is done with iteration z-1, so buffer bf (plane z-1) and
    // the per-plane shared arrays may be overwritten
    if (use_tma) tma_wait(bn);
    else cp_async_wait0();
    __syncthreads();
    if (z + 2 <= z1) {
      if (use_tma) {
        if (tid == 0 && copies_ok) {
          // the slot's last reads were generic loads: order them before the
          // tensor copy's writes
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
          tma_issue(bf, z + 2);
        }
      } else {
        cpl.issue(&sm.pos[bf][0][0], zoff(z + 2));
        cp_async_commit();
      }
    }

    const long long gsite = (long long)z * plane + (long long)gy * v.nx + gx;
    // momenta of the own site, loaded during the previous plane
    T pr[2], pim[2], E[2][3];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      pr[s] = npr[s];
      pim[s] = npim[s];
#pragma unroll
      for (int i = 0; i < 3; ++i) E[s][i] = nE[s][i];
    }

    // ---- phase 1: site-local quantities of plane z ----
    const int a = TL::at(ly, lx);
    T cs_[2][3], sn_[2][3], F[2][3], P2r[2], P2i[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T* fr = sm.pos[bc][2 * s];
      const T* fi = sm.pos[bc][2 * s + 1];
      const T* A0 = sm.pos[bc][4 + 3 * s];
      const T* A1 = sm.pos[bc][5 + 3 * s];
      const T* A2 = sm.pos[bc][6 + 3 * s];
#pragma unroll
      for (int i = 0; i < 3; ++i) link_sincos<T>(dx * sm.pos[bc][4 + 3 * s + i][a], &sn_[s][i], &cs_[s][i]);
      T pr0, pi0, pr1, pi1;
      transport_bwd<T>(cs_[s][0], sn_[s][0], fr[a], fi[a], &pr0, &pi0);
      transport_bwd<T>(cs_[s][1], sn_[s][1], fr[a], fi[a], &pr1, &pi1);
      transport_bwd<T>(cs_[s][2], sn_[s][2], fr[a], fi[a], &P2r[s], &P2i[s]);
      sm.P[s][0][0][a] = pr0;
      sm.P[s][0][1][a] = pi0;
      sm.P[s][1][0][a] = pr1;
      sm.P[s][1][1][a] = pi1;
      F[s][0] = curl_ft<T>(A1[TL::at(ly, lx + 1)], A1[a], A0[TL::at(ly + 1, lx)], A0[a]);
      F[s][1] = curl_ft<T>(A2[TL::at(ly, lx + 1)], A2[a], sm.pos[bn][4 + 3 * s][a], A0[a]);
      F[s][2] = curl_ft<T>(A2[TL::at(ly + 1, lx)], A2[a], sm.pos[bn][5 + 3 * s][a], A1[a]);
      sm.Ft[s][0][a] = F[s][0];
      sm.Ft[s][1][a] = F[s][1];
      sm.Ft[s][2][a] = F[s][2];
      if (GAUSS) {
        sm.Eg[s][0][a] = E[s][0];
        sm.Eg[s][1][a] = E[s][1];
      }
    }
    // halo points: left column (lx = -1) and bottom row (ly = -1).  A step
    // gives each of the first TX + TY threads one point, both sectors; a
    // measuring pass, whose own-site work is longer, spreads the 2 (TX + TY)
    // (point, sector) tasks over all warps, one single-sector pass each
    // (measured: 3% faster for the measuring pass, 1.5% slower for the step).
    constexpr int HT = 2 * (TX + TY), NW = TL::NT / 32, HPW = (HT + NW - 1) / NW;
    const int hj = MEAS ? ((tid & 31) < HPW ? (tid >> 5) * HPW + (tid & 31) : HT) : tid;
    if (MEAS ? hj < HT : halo_point<TL::NT, TX + TY>(tid) >= 0) {
      const int h = hj % (TX + TY);
      const bool left = h < TY;
      const int hy = left ? h : -1;
      const int hx = left ? -1 : h - TY;
      const int ha = TL::at(hy, hx);
#pragma unroll
      for (int s = (MEAS ? hj / (TX + TY) : 0); s < (MEAS ? hj / (TX + TY) + 1 : 2); ++s) {
        const T* fr = sm.pos[bc][2 * s];
        const T* fi = sm.pos[bc][2 * s + 1];
        const T* A0 = sm.pos[bc][4 + 3 * s];
        const T* A1 = sm.pos[bc][5 + 3 * s];
        const T* A2 = sm.pos[bc][6 + 3 * s];
        const int d = left ? 0 : 1;
        T sn, cs, br, bi;
        link_sincos<T>(dx * sm.pos[bc][4 + 3 * s + d][ha], &sn, &cs);
        transport_bwd<T>(cs, sn, fr[ha], fi[ha], &br, &bi);
        sm.P[s][d][0][ha] = br;
        sm.P[s][d][1][ha] = bi;
        sm.Ft[s][0][ha] = curl_ft<T>(A1[TL::at(hy, hx + 1)], A1[ha], A0[TL::at(hy + 1, hx)], A0[ha]);
        if (left)
          sm.Ft[s][1][ha] = curl_ft<T>(A2[TL::at(hy, hx + 1)], A2[ha], sm.pos[bn][4 + 3 * s][ha], A0[ha]);
        else
          sm.Ft[s][2][ha] = curl_ft<T>(A2[TL::at(hy + 1, hx)], A2[ha], sm.pos[bn][5 + 3 * s][ha], A1[ha]);
        if (GAUSS) {
          const long long hs = (long long)z * plane + (long long)wrapm(y0 + hy, v.ny) * v.nx + wrapm(x0 + hx, v.nx);
          sm.Eg[s][d][ha] = ld_mom<COHERENT>(&v.mom[4 + 3 * s + d][hs]);
        }
      }
    }

    // forward transports U_i phi(x+i) of the own site
    SectorIn<T> in[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      SectorIn<T>& q = in[s];
      q.fr = sm.pos[bc][2 * s][a];
      q.fi = sm.pos[bc][2 * s + 1][a];
      const int ax = TL::at(ly, lx + 1), ay = TL::at(ly + 1, lx);
      transport_fwd<T>(cs_[s][0], sn_[s][0], sm.pos[bc][2 * s][ax], sm.pos[bc][2 * s + 1][ax], &q.fwr[0], &q.fwi[0]);
      transport_fwd<T>(cs_[s][1], sn_[s][1], sm.pos[bc][2 * s][ay], sm.pos[bc][2 * s + 1][ay], &q.fwr[1], &q.fwi[1]);
      transport_fwd<T>(cs_[s][2], sn_[s][2], sm.pos[bn][2 * s][a], sm.pos[bn][2 * s + 1][a], &q.fwr[2], &q.fwi[2]);
      q.A[0] = sm.pos[bc][4 + 3 * s][a];
      q.A[1] = sm.pos[bc][5 + 3 * s][a];
      q.A[2] = sm.pos[bc][6 + 3 * s][a];
      q.F[0] = F[s][0];
      q.F[1] = F[s][1];
      q.F[2] = F[s][2];
    }

    __syncthreads();

    // ---- phase 2: assemble the update of the own site ----
    T tv[NSUM];  // this site's diagnostic densities (zero when inactive)
    if (MEAS) {
#pragma unroll
      for (int k = 0; k < NSUM; ++k) tv[k] = T(0);
    }
    if (active) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        SectorIn<T>& q = in[s];
        const int axm = TL::at(ly, lx - 1), aym = TL::at(ly - 1, lx);
        q.bwr[0] = sm.P[s][0][0][axm];
        q.bwi[0] = sm.P[s][0][1][axm];
        q.bwr[1] = sm.P[s][1][0][aym];
        q.bwi[1] = sm.P[s][1][1][aym];
        q.bwr[2] = cP2r[s];
        q.bwi[2] = cP2i[s];
        q.Fm[0] = sm.Ft[s][0][aym];
        q.Fm[1] = sm.Ft[s][0][axm];
        q.Fm[2] = cF02[s];
        q.Fm[3] = sm.Ft[s][1][axm];
        q.Fm[4] = cF12[s];
        q.Fm[5] = sm.Ft[s][2][aym];
      }
      T mod2[2] = {in[0].fr * in[0].fr + in[0].fi * in[0].fi, in[1].fr * in[1].fr + in[1].fi * in[1].fi};
      T rr[2] = {mod2[0] - c.sig2[0], mod2[1] - c.sig2[1]};
      T prn[2], pin_[2], En[2][3];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        scalar_kick<T>(in[s], rr[s], rr[1 - s], pr[s], pim[s], c, s, &prn[s], &pin_[s]);
        gauge_kick<T>(in[s], E[s], c, s, En[s]);
      }
      if (WRITE) {
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          st_field<STREAM>(&v.mom[2 * s][gsite], prn[s]);
          st_field<STREAM>(&v.mom[2 * s + 1][gsite], pin_[s]);
          st_field<STREAM>(&v.pout[2 * s][gsite], in[s].fr + c.deta * prn[s]);
          st_field<STREAM>(&v.pout[2 * s + 1][gsite], in[s].fi + c.deta * pin_[s]);
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            st_field<STREAM>(&v.mom[4 + 3 * s + i][gsite], En[s][i]);
            st_field<STREAM>(&v.pout[4 + 3 * s + i][gsite], in[s].A[i] + c.deta * En[s][i]);
          }
        }
      }
      if (MEAS) {
        SectorDiag<T> d[2];
#pragma unroll
        for (int s = 0; s < 2; ++s) d[s] = sector_diag<T>(in[s], pr[s], pim[s], prn[s], pin_[s], E[s], En[s], c, s);
        const T rp = rr[0], rq = rr[1];
        const T pot = c.cV * (c.lam4[0] * rp * rp + c.lam4[1] * rq * rq - c.kappa * rp * rq);
        const T vint = c.kappa * rp * rq;
        const T L = (d[0].kin - d[0].grad + d[0].el - d[0].mag) + (d[1].kin - d[1].grad + d[1].el - d[1].mag) - pot;
        const T kt = d[0].kin + d[1].kin, gt = d[0].grad + d[1].grad;
        // the Lagrangian and energy sums are formed from the component sums
        // on the host; only the weighted sums of Eq. 37 need L per site
        tv[S_KIN_P] = d[0].kin;
        tv[S_KIN_Q] = d[1].kin;
        tv[S_GRAD_P] = d[0].grad;
        tv[S_GRAD_Q] = d[1].grad;
        tv[S_EL_P] = d[0].el;
        tv[S_EL_Q] = d[1].el;
        tv[S_MAG_P] = d[0].mag;
        tv[S_MAG_Q] = d[1].mag;
        tv[S_POT] = pot;
        tv[S_POT_P] = c.cV * c.lam4[0] * rp * rp;
        tv[S_POT_Q] = c.cV * c.lam4[1] * rq * rq;
        tv[S_VINT] = vint;
        tv[S_RL_NUM] = kt * L;
        tv[S_RL_DEN] = gt * L;
        tv[S_RPQ_NUM] = kt * vint;
        tv[S_RPQ_DEN] = gt * vint;
        // extremes of |phi|^2 (|phi| after the block's last plane: the
        // square root is monotonic and correctly rounded)
#pragma unroll
        for (int s = 0; s < 2; ++s) {
          mx[s == 0 ? M_NEG_PHIMIN_P : M_NEG_PHIMIN_Q] = fmax(mx[s == 0 ? M_NEG_PHIMIN_P : M_NEG_PHIMIN_Q], -mod2[s]);
          mx[s == 0 ? M_PHIMAX_P : M_PHIMAX_Q] = fmax(mx[s == 0 ? M_PHIMAX_P : M_PHIMAX_Q], mod2[s]);
        }
        // NaN entries among the site's 20 fields, counted one by one only
        // where the site's ten new momenta do not sum to a finite number:
        // every one of its own fields enters one of them (phi and pi the
        // scalar kick, A and E the gauge kick) with a coefficient that
        // keeps a NaN or an infinity non-finite, so no NaN field is missed
        // (a non-finite neighbour or an overflow only triggers a recount
        // that finds nothing); ten additions instead of twenty
        T all = (prn[0] + pin_[0]) + (prn[1] + pin_[1]);
#pragma unroll
        for (int s = 0; s < 2; ++s) all += En[s][0] + En[s][1] + En[s][2];
        if (!isfinite(all)) {
          int nan = 0;
#pragma unroll
          for (int f = 0; f < U1U1_NPOS; ++f) nan += isnan(sm.pos[bc][f][a]) ? 1 : 0;
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            nan += isnan(pr[s]) + isnan(pim[s]) + isnan(E[s][0]) + isnan(E[s][1]) + isnan(E[s][2]);
          }
          cnt[C_NAN] += nan;
        }

        if (GAUSS) {
#pragma unroll
          for (int s = 0; s < 2; ++s) {
            T div = (E[s][0] - sm.Eg[s][0][TL::at(ly, lx - 1)]) + (E[s][1] - sm.Eg[s][1][TL::at(ly - 1, lx)]) +
                    (E[s][2] - cE2[s]);
            div *= c.inv_dx;
            const T rho = c.qG[s] * (in[s].fr * pim[s] - in[s].fi * pr[s]);
            const T G = div - rho;
            mx[s == 0 ? M_GAUSS_P : M_GAUSS_Q] = fmax(mx[s == 0 ? M_GAUSS_P : M_GAUSS_Q], fabs(G));
            tv[s == 0 ? S_GAUSS_P : S_GAUSS_Q] = fabs(G);
            tv[s == 0 ? S_CHARGE_P : S_CHARGE_Q] = fabs(rho);
          }
        }
      }
    }
    if (MEAS) {
      // one row of 32 sites per warp.  FP32: add the site's densities to the
      // thread's plain partials and, every ACC_PLANES planes and at the last
      // plane, reduce those across the warp into the warp's compensated sums.
      // FP64: reduce every plane.
      const bool fold = !SM::ACC || ((z - z0) % ACC_PLANES) == ACC_PLANES - 1 || z == z1 - 1;
#pragma unroll
      for (int k = 0; k < NSUM; ++k) {
        if (!acc_used(k, GAUSS)) continue;
        T v2 = tv[k];
        if (SM::ACC) {
          T& acc = racc[SM::ACC ? acc_slot(k, GAUSS) : 0];
          v2 += acc;
          acc = fold ? T(0) : v2;
        }
        if (fold) {
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) v2 += __shfl_down_sync(0xffffffffu, v2, o);
          if ((tid & 31) == 0) {  // Kahan step
            const T y = v2 - sm.wcmp[tid >> 5][k];
            const T t = sm.wsum[tid >> 5][k] + y;
            sm.wcmp[tid >> 5][k] = (t - sm.wsum[tid >> 5][k]) - y;
            sm.wsum[tid >> 5][k] = t;
          }
        }
      }
    }
    // carries for plane z+1
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      cP2r[s] = P2r[s];
      cP2i[s] = P2i[s];
      cF02[s] = F[s][1];
      cF12[s] = F[s][2];
      cE2[s] = E[s][2];
    }
    if (z + 1 < z1) load_mom(z + 1);
  }
  cp_async_wait0();

  if (MEAS) {
    // The block's partial: the warps' compensated sums are already in
    // shared memory, so only the extremes (in the working precision) and
    // the counts (32-bit, like each thread's own: a warp adds 32 of them) are
    // reduced across each warp; then one thread per quantity merges the
    // warps in a fixed order, the sums by Neumaier in FP64.  Nothing
    // per-thread goes through GB300's narrow FP64 pipe, so the cost of a
    // block's epilogue no longer grows the detection step when z-chunks
    // are short and blocks many.
    constexpr int NW = TL::NT / 32;
    const int lane = tid & 31, warp = tid >> 5;
    // |phi| from the extremes of |phi|^2 (-inf: no site of this block)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const int kn = s == 0 ? M_NEG_PHIMIN_P : M_NEG_PHIMIN_Q, kx = s == 0 ? M_PHIMAX_P : M_PHIMAX_Q;
      if (mx[kn] != -INFINITY) mx[kn] = -sqrt(-mx[kn]);
      if (mx[kx] != -INFINITY) mx[kx] = sqrt(mx[kx]);
    }
#pragma unroll
    for (int k = 0; k < NMAX; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) mx[k] = fmax(mx[k], __shfl_down_sync(0xffffffffu, mx[k], o));
    }
#pragma unroll
    for (int k = 0; k < NCNT; ++k) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const int u = __shfl_down_sync(0xffffffffu, cnt[k], o);
        cnt[k] = k == C_MAXW ? max(cnt[k], u) : cnt[k] + u;
      }
    }
    struct EpiSmem {
      double mx[NW][NMAX];
      long long cnt[NW][NCNT];
    };
    static_assert(sizeof(EpiSmem) <= sizeof(sm.pos), "epilogue scratch must fit in the position ring");
    __syncthreads();  // the ring is no longer read; every warp's sums are final
    EpiSmem& es = *reinterpret_cast<EpiSmem*>(&sm.pos[0][0][0]);
    if (lane == 0) {
#pragma unroll
      for (int k = 0; k < NMAX; ++k) es.mx[warp][k] = (double)mx[k];
#pragma unroll
      for (int k = 0; k < NCNT; ++k) es.cnt[warp][k] = cnt[k];
    }
    __syncthreads();
    BlockPartial* out = mo.partial + bid;
    if (tid < NSUM) {
      double sum = 0.0, comp = 0.0;
      for (int w = 0; w < NW; ++w) neumaier_add(sum, comp, (double)sm.wsum[w][tid] - (double)sm.wcmp[w][tid]);
      out->sum[tid] = sum;
      out->comp[tid] = comp;
    } else if (tid < NSUM + NMAX) {
      const int k = tid - NSUM;
      double m = -INFINITY;
      for (int w = 0; w < NW; ++w) m = fmax(m, es.mx[w][k]);
      out->mx[k] = m;
    } else if (tid < NSUM + NMAX + NCNT) {
      const int k = tid - NSUM - NMAX;
      long long n = 0;
      for (int w = 0; w < NW; ++w) n = k == C_MAXW ? max(n, es.cnt[w][k]) : n + es.cnt[w][k];
      out->cnt[k] = n;
    }
  }
}

template <typename T, int TX, int TY, int MODE>
__global__ void __launch_bounds__(TX* TY, sizeof(T) == 8 ? 1 : (MODE == MODE_WRITE ? 3 : 2))
k_tiled(LatticeView<T> v, Coef<T> c, MeasureOut mo, int lz, int band_rows, const __grid_constant__ TmaPlan tma) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  // The hardware hands out blocks in linear order.  With band_rows = 0 that
  // order is z-chunk by z-chunk over the whole plane of tiles.  With
  // band_rows > 0 a band of that many tile rows (one resident wave) is taken
  // through all its z-chunks before the next band starts, so that a tile's
  // y-neighbours run at the same time and the halo rows they share are still
  // in L2.  Every (tile, chunk) is taken exactly once either way.
  const int gx = gridDim.x, gy = gridDim.y, gz = gridDim.z;
  const int lin = (blockIdx.z * gy + blockIdx.y) * gx + blockIdx.x;
  int bx = blockIdx.x, by = blockIdx.y, bzc = blockIdx.z;
  if (band_rows > 0) {
    const int per_band = band_rows * gx * gz;
    const int band = lin / per_band;
    const int tiles_b = min(band_rows, gy - band * band_rows) * gx;  // the last band may be shorter
    const int rem = lin - band * per_band;
    bzc = rem / tiles_b;
    bx = (rem % tiles_b) % gx;
    by = band * band_rows + (rem % tiles_b) / gx;
  }
  const int z0 = bzc * lz;
  const int z1 = min(z0 + lz, v.nz);
  tile_run<T, TX, TY, MODE, false, true, MODE == MODE_WRITE>(smem_raw, v, c, mo, bx, by, z0, z1, lin, &tma);
}

template <typename T>
struct TileShape {
  static constexpr int TX = 32, TY = 8;
};

// The z-chunk length follows from the number of CTAs aimed at: 152 SMs x 3
// resident CTAs x `waves`.  About 32 waves (the default) keeps neighbouring
// tiles close in z, so halo rows are still in L2 when the neighbour needs
// them (measured 4% faster than 8 waves at 1024^3); at least 32 planes per
// chunk keep the extra prologue plane below 3%.  The autotuner may pick
// another value per lattice shape.
constexpr int MIN_LZ = 32;

struct Grid {
  int gx, gy, gz, lz;
};

template <typename T>
Grid tiled_grid(int nx, int ny, int nz, int waves) {
  constexpr int TX = TileShape<T>::TX, TY = TileShape<T>::TY;
  Grid g;
  g.gx = (nx + TX - 1) / TX;
  g.gy = (ny + TY - 1) / TY;
  const int tiles = g.gx * g.gy;
  const long long target = 152LL * 3 * (waves > 0 ? waves : TILE_WAVES_DEFAULT);
  int chunks = (int)((target + tiles - 1) / tiles);
  if (chunks < 1) chunks = 1;
  int lz = (nz + chunks - 1) / chunks;
  if (lz < MIN_LZ) lz = MIN_LZ;
  if (lz > nz) lz = nz;
  g.lz = lz;
  g.gz = (nz + lz - 1) / lz;
  return g;
}

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime
// (no link against the driver library); null when unavailable
using EncodeTiledFn = CUresult (*)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                   const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                   CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);
EncodeTiledFn encode_tiled() {
  static const EncodeTiledFn fn = [] {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess) {
      cudaGetLastError();
      return (EncodeTiledFn) nullptr;
    }
    return reinterpret_cast<EncodeTiledFn>(p);
  }();
  return fn;
}

// Tensor maps of the step's input position fields for the FP32 tiled kernel:
// a 3D view (x, y, z) of each field, box = one ring slot of one field.  The
// plan stays disabled (every tile then uses cp.async) for FP64, for
// lattices too small to have an interior tile, and when encoding fails.
// bytes each ring slot of the single-lattice kernels expects on top of what
// its copies deliver (0, or 16 while the timeout test hook is on), and the
// limit of a wait for them; both travel in the kernel parameter
unsigned g_inject_extra_bytes = 0u;
long long g_wait_limit_ns = 2000000000LL;

template <typename T>
void make_plan(const T* const pin[U1U1_NPOS], int nx, int ny, int nz, TmaPlan* tp) {
  memset(tp, 0, sizeof(*tp));
  tp->limit_ns = 2000000000LL;
  if (sizeof(T) != 4) return;
  using TL = Tile<T, TileShape<T>::TX, TileShape<T>::TY>;
  if (nx < TileShape<T>::TX + 2 * TL::VEC || ny < TileShape<T>::TY + 2) return;
  const EncodeTiledFn enc = encode_tiled();
  if (!enc) return;
  const cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)ny, (cuuint64_t)nz};
  const cuuint64_t strides[2] = {(cuuint64_t)nx * sizeof(T), (cuuint64_t)nx * ny * sizeof(T)};
  const cuuint32_t box[3] = {(cuuint32_t)TL::RS, (cuuint32_t)TL::ROWS, 1u};
  const cuuint32_t estride[3] = {1u, 1u, 1u};
  for (int f = 0; f < U1U1_NPOS; ++f) {
    if (enc(&tp->map[f], CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, const_cast<T*>(pin[f]), dims, strides, box, estride,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
      return;
  }
  tp->enabled = 1;
}

template <typename T, int MODE>
cudaError_t launch_mode(const LatticeView<T>& v, const Coef<T>& c, const MeasureOut& mo, cudaStream_t st,
                        int waves, int* status) {
  constexpr int TX = TileShape<T>::TX, TY = TileShape<T>::TY;
  constexpr bool MEAS = (MODE & MODE_MEASURE) != 0;
  constexpr bool GAUSS = (MODE & MODE_GAUSS) != 0;
  const size_t bytes = sizeof(Smem<T, TX, TY, MEAS, GAUSS>);
  // the dynamic shared-memory limit is a per-device function attribute;
  // the resident CTAs per device size the plain step's bands
  static bool configured[64] = {};
  static int resident[64] = {};
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    e = cudaFuncSetAttribute(k_tiled<T, TX, TY, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    // three plain-step CTAs of about 72 KB per SM need the largest
    // shared-memory carveout; the two-CTA measuring variants keep the
    // driver's choice (more L1 for their cached loads: forcing it made the
    // diagnostics pass 15% slower)
    if (MODE == MODE_WRITE) {
      e = cudaFuncSetAttribute(k_tiled<T, TX, TY, MODE>, cudaFuncAttributePreferredSharedMemoryCarveout,
                               (int)cudaSharedmemCarveoutMaxShared);
      if (e != cudaSuccess) return e;
    }
    int sms = 0, per_sm = 0;
    e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_tiled<T, TX, TY, MODE>, TX * TY, bytes);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) {
      resident[dev] = sms * (per_sm > 0 ? per_sm : 1);
      configured[dev] = true;
    }
  }
  Grid g = tiled_grid<T>(v.nx, v.ny, v.nz, waves);
  dim3 grid(g.gx, g.gy, g.gz);
  TmaPlan tp;
  make_plan<T>(v.pin, v.nx, v.ny, v.nz, &tp);
  tp.extra_bytes = g_inject_extra_bytes;
  tp.limit_ns = g_wait_limit_ns;
  tp.status = status;
  // plain steps: bands of one resident wave of tiles (measured at 1024^3,
  // 256 waves: 28.23 ms against 28.57 in z-chunk order; bands of 0.75 or 1.25
  // waves gave 28.67 and 28.59).  The measuring passes keep the z-chunk
  // order, which fixes the order in which their block partials are merged.
  int band_rows = 0;
  if (MODE == MODE_WRITE && dev >= 0 && dev < 64 && resident[dev] > 0)
    band_rows = min(g.gy, max(1, (resident[dev] + g.gx / 2) / g.gx));
  k_tiled<T, TX, TY, MODE><<<grid, TX * TY, bytes, st>>>(v, c, mo, g.lz, band_rows, tp);
  return cudaGetLastError();
}

}  // namespace

template <typename T>
void make_tma_plan(const T* const pin[U1U1_NPOS], int nx, int ny, int nz, TmaPlan* tp) {
  make_plan<T>(pin, nx, ny, nz, tp);
}
template void make_tma_plan<float>(const float* const*, int, int, int, TmaPlan*);
template void make_tma_plan<double>(const double* const*, int, int, int, TmaPlan*);

int tma_inject_timeout(int enable, long long limit_ns) {
  g_inject_extra_bytes = enable ? 16u : 0u;
  g_wait_limit_ns = limit_ns;
  return 0;
}

int tiled_grid_blocks(int nx, int ny, int nz, int sizeof_t, int waves) {
  Grid g = sizeof_t == 8 ? tiled_grid<double>(nx, ny, nz, waves) : tiled_grid<float>(nx, ny, nz, waves);
  return g.gx * g.gy * g.gz;
}

void tiled_grid_dims(int nx, int ny, int nz, int sizeof_t, int waves, int* gx, int* gy, int* gz, int* lz) {
  Grid g = sizeof_t == 8 ? tiled_grid<double>(nx, ny, nz, waves) : tiled_grid<float>(nx, ny, nz, waves);
  *gx = g.gx;
  *gy = g.gy;
  *gz = g.gz;
  *lz = g.lz;
}

// ---------------------------------------------------------------------------
// Ensemble kernels: many independent boxes in one launch.
// ---------------------------------------------------------------------------

namespace {

__device__ __forceinline__ long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return (long long)t;
}

// largest i in [0, n) with a[i] <= r (a ascending, a[0] = 0 <= r)
__device__ __forceinline__ int upper_index(const long long* a, int n, long long r) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (a[mid] <= r) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// USE_TMA: fill interior tiles' ring slots by tensor copies from the box's
// plan (tensor copies read through L2, so they see the positions another
// CTA of the same persistent launch wrote and fenced); a compile-time
// choice, since the tensor-copy path costs registers even where it is not
// taken
// A box's step view (input buffer cur) built in the thread: the fallback for
// ensembles too large for the parameter table of views
template <typename T>
__device__ __forceinline__ LatticeView<T> box_view(const EnsBox<T>& B, int cur) {
  LatticeView<T> v;
#pragma unroll
  for (int f = 0; f < U1U1_NPOS; ++f) {
    v.pin[f] = B.pos[cur][f];
    v.pout[f] = B.pos[cur ^ 1][f];
  }
#pragma unroll
  for (int f = 0; f < U1U1_NMOM; ++f) v.mom[f] = B.mom[f];
  v.nx = B.nx;
  v.ny = B.ny;
  v.nz = B.nz;
  return v;
}

template <typename T, bool COHERENT, bool USE_TMA>
__device__ __forceinline__ void ens_run_item(unsigned char* smem, const EnsBox<T>& B, const LatticeView<T>& v, int cur,
                                             const Coef<T>& c, long long t) {
  constexpr int TX = TileShape<T>::TX, TY = TileShape<T>::TY;
  const int bx = (int)(t % B.gx);
  const int by = (int)((t / B.gx) % B.gy);
  const int bz = (int)(t / ((long long)B.gx * B.gy));
  const int z0 = bz * B.lz;
  const int z1 = min(z0 + B.lz, B.nz);
  MeasureOut mo{nullptr, nullptr, nullptr};
  tile_run<T, TX, TY, MODE_WRITE, COHERENT, false>(smem, v, c, mo, bx, by, z0, z1, 0, USE_TMA ? B.tma[cur] : nullptr);
}

// Persistent ensemble kernel: CTAs take work items (step k, box, tile) in
// ticket order, step-major, boxes with more steps first.  An item of step k
// waits until all items of step k-1 of its box are done.  Every wait is
// bounded: past limit_ns the kernel records U1U1_ERR_TIMEOUT and all CTAs
// return.  Deadlock freedom: tickets are taken only by running CTAs and an
// item depends only on items with smaller tickets.
//
// VIEWS (all three ensemble kernels): each box's step view is read from the
// kernel-parameter table `views`; otherwise it is built in the thread from
// the box record.  A compile-time choice, so that each instantiation holds
// one copy of the tile body and the view path keeps no local view copy.
template <typename T, bool USE_TMA, bool VIEWS>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 3)
k_ens_persistent(const EnsBox<T>* __restrict__ boxes, const EnsDyn* __restrict__ dyn, const Coef<T>* __restrict__ coef,
                 EnsSched sc, const int* __restrict__ kstart, unsigned long long* ticket, unsigned* done, int* err,
                 long long limit_ns, int inject, const __grid_constant__ EnsViews<T> views) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ Coef<T> cs;
  __shared__ long long s_t;
  __shared__ int s_box, s_k, s_go;
  for (;;) {
    if (threadIdx.x == 0) {
      const long long tk = (long long)atomicAdd(ticket, 1ull);
      int go = (tk < sc.total) && (*(volatile int*)err == 0);
      int box = 0, k = 0;
      long long t = 0;
      if (go) {
        k = upper_index(sc.step_off, sc.smax + 1, tk);
        const long long r = tk - sc.step_off[k];
        const int si = upper_index(sc.box_prefix, sc.nboxes + 1, r);
        box = sc.order[si];
        t = r - sc.box_prefix[si];
        unsigned need = (unsigned)k * (unsigned)boxes[box].ntiles;
        if (inject && si == 0 && k == 1 && t == 0) need = 0xFFFFFFFFu;  // a count no run reaches
        if (need > 0) {
          const long long t0 = globaltimer_ns();
          while (*(volatile unsigned*)&done[box] < need) {
            if (*(volatile int*)err != 0) {
              go = 0;
              break;
            }
            if (globaltimer_ns() - t0 > limit_ns) {
              atomicExch(err, U1U1_ERR_TIMEOUT);
              go = 0;
              break;
            }
            __nanosleep(256);
          }
          __threadfence();
        }
        if (kstart) k += kstart[box];  // the run step of this item
        if (go) cs = coef[boxes[box].coef0 + dyn[box].n + k];
      }
      s_go = go;
      s_box = box;
      s_k = k;
      s_t = t;
    }
    __syncthreads();
    if (!s_go) break;
    const EnsBox<T>& B = boxes[s_box];
    const int cur = (dyn[s_box].cur + s_k) & 1;
    if constexpr (VIEWS)
      ens_run_item<T, true, USE_TMA>(smem_raw, B, views.v[s_box][cur], cur, cs, s_t);
    else
      ens_run_item<T, true, USE_TMA>(smem_raw, B, box_view(B, cur), cur, cs, s_t);
    __syncthreads();
    if (threadIdx.x == 0) {
      __threadfence();
      atomicAdd(&done[s_box], 1u);
    }
  }
}

// One step k of every box that still has steps: one CTA per work item.
template <typename T, bool VIEWS>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 3)
k_ens_step(const EnsBox<T>* __restrict__ boxes, const EnsDyn* __restrict__ dyn, const Coef<T>* __restrict__ coef,
           EnsSched sc, int k, const __grid_constant__ EnsViews<T> views) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ Coef<T> cs;
  const long long r = blockIdx.x;
  const int si = upper_index(sc.box_prefix, sc.nboxes + 1, r);
  const int box = sc.order[si];
  if (threadIdx.x == 0) cs = coef[boxes[box].coef0 + dyn[box].n + k];
  __syncthreads();
  const int cur = (dyn[box].cur + k) & 1;
  if constexpr (VIEWS)
    ens_run_item<T, false, true>(smem_raw, boxes[box], views.v[box][cur], cur, cs, r - sc.box_prefix[si]);
  else
    ens_run_item<T, false, true>(smem_raw, boxes[box], box_view(boxes[box], cur), cur, cs, r - sc.box_prefix[si]);
}

// Measuring step k (a step fused with the diagnostic sums) of the boxes in
// list[0..nlist), one CTA per tile of any of them, in the tile grid and
// partial slots of a single lattice's measuring launch.  The CTA of a box's
// first tile also clears the box's overlap and census counters for the
// passes that follow in stream order.
template <typename T, bool VIEWS>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 1 : 2)
k_ens_measure(const EnsBox<T>* __restrict__ boxes, const EnsDet* __restrict__ det, const EnsDyn* __restrict__ dyn,
              const Coef<T>* __restrict__ coef, const int* __restrict__ list, const long long* __restrict__ pre,
              int nlist, int k, const __grid_constant__ EnsViews<T> views) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  __shared__ Coef<T> cs;
  const long long r = blockIdx.x;
  const int si = ens_list_index(pre, nlist, r);
  const int b = list[si];
  const long long t = r - pre[si];
  const EnsBox<T>& B = boxes[b];
  const EnsDet& D = det[b];
  if (threadIdx.x == 0) cs = coef[B.coef0 + dyn[b].n + k];
  if (t == 0 && threadIdx.x < 2) {
    D.counts->pq[threadIdx.x] = 0;
    D.ge4[threadIdx.x] = 0ull;
  }
  __syncthreads();
  const int cur = (dyn[b].cur + k) & 1;
  const int bx = (int)(t % D.mgx), by = (int)((t / D.mgx) % D.mgy), bz = (int)(t / ((long long)D.mgx * D.mgy));
  const int z0 = bz * D.mlz, z1 = min(z0 + D.mlz, B.nz);
  MeasureOut mo{D.part, nullptr, nullptr};
  constexpr int TX = TileShape<T>::TX, TY = TileShape<T>::TY;
  if constexpr (VIEWS) {
    tile_run<T, TX, TY, MODE_WRITE | MODE_MEASURE, false, false>(smem_raw, views.v[b][cur], cs, mo, bx, by, z0, z1,
                                                                 (int)t, B.tma[cur]);
  } else {
    const LatticeView<T> v = box_view(B, cur);
    tile_run<T, TX, TY, MODE_WRITE | MODE_MEASURE, false, false>(smem_raw, v, cs, mo, bx, by, z0, z1, (int)t,
                                                                 B.tma[cur]);
  }
}

// After a run: advance each box's step index, buffer parity and count of
// records written (the steps n0 <= n < n0 + steps with n % de == 0).
__global__ void k_ens_advance(EnsDyn* dyn, const int* steps, int nboxes, int de) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b < nboxes) {
    if (de > 0) {
      const long long n0 = dyn[b].n;
      const long long k1 = (de - n0 % de) % de;  // first detection step of the run
      if (steps[b] > k1) dyn[b].rec += (steps[b] - 1 - k1) / de + 1;
    }
    dyn[b].n += steps[b];
    dyn[b].cur ^= (steps[b] & 1);
  }
}

template <typename T>
size_t ens_smem_bytes() {
  return sizeof(Smem<T, TileShape<T>::TX, TileShape<T>::TY, false, false>);
}

// The dynamic shared-memory limit is a per-device function attribute; the
// caller keeps one `configured` array per kernel (kernels of one signature
// share a function-pointer type, so a static here would be shared by them).
template <typename KernelT>
cudaError_t set_smem_attr(KernelT kernel, size_t bytes, bool (&configured)[64]) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 0 || dev >= 64 || !configured[dev]) {
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (e != cudaSuccess) return e;
    if (dev >= 0 && dev < 64) configured[dev] = true;
  }
  return cudaSuccess;
}

}  // namespace

int ens_tile_grid(int nx, int ny, int nz, int* gx, int* gy, int* lz, int* gz, int item_lz) {
  *gx = (nx + 31) / 32;
  *gy = (ny + 7) / 8;
  if (item_lz < 1) item_lz = ENS_LZ;
  *lz = nz < item_lz ? nz : item_lz;
  *gz = (nz + *lz - 1) / *lz;
  return *gx * *gy * *gz;
}

// the view table a launch passes: the ensemble's, or an empty one (the
// kernels then build each box's view in the thread)
template <typename T>
const EnsViews<T>& views_or_empty(const EnsViews<T>* views) {
  static const EnsViews<T> empty{};
  return views ? *views : empty;
}

template <typename T, bool USE_TMA, bool VIEWS>
cudaError_t launch_ens_persistent_t(const EnsBox<T>* boxes, const EnsDyn* dyn, const Coef<T>* coef,
                                    const EnsSched& sc, const int* kstart, unsigned long long* ticket, unsigned* done,
                                    int* err, long long limit_ns, int inject, const EnsViews<T>* views,
                                    cudaStream_t st) {
  static bool configured[64] = {};
  const size_t bytes = ens_smem_bytes<T>();
  cudaError_t e = set_smem_attr(k_ens_persistent<T, USE_TMA, VIEWS>, bytes, configured);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
  if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
  if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ens_persistent<T, USE_TMA, VIEWS>, 256,
                                                         bytes)) != cudaSuccess)
    return e;
  long long grid = (long long)sms * (per_sm > 0 ? per_sm : 1);
  if (grid > sc.total) grid = sc.total;
  if (grid < 1) return cudaSuccess;
  k_ens_persistent<T, USE_TMA, VIEWS><<<(unsigned)grid, 256, bytes, st>>>(boxes, dyn, coef, sc, kstart, ticket, done,
                                                                          err, limit_ns, inject,
                                                                          views_or_empty(views));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ens_persistent(const EnsBox<T>* boxes, const EnsDyn* dyn, const Coef<T>* coef, const EnsSched& sc,
                                  const int* kstart, unsigned long long* ticket, unsigned* done, int* err,
                                  long long limit_ns, int inject, int use_tma, const EnsViews<T>* views,
                                  cudaStream_t st) {
  if (use_tma)
    return views ? launch_ens_persistent_t<T, true, true>(boxes, dyn, coef, sc, kstart, ticket, done, err, limit_ns,
                                                          inject, views, st)
                 : launch_ens_persistent_t<T, true, false>(boxes, dyn, coef, sc, kstart, ticket, done, err, limit_ns,
                                                           inject, views, st);
  return views ? launch_ens_persistent_t<T, false, true>(boxes, dyn, coef, sc, kstart, ticket, done, err, limit_ns,
                                                         inject, views, st)
               : launch_ens_persistent_t<T, false, false>(boxes, dyn, coef, sc, kstart, ticket, done, err, limit_ns,
                                                          inject, views, st);
}

template <typename T, bool VIEWS>
cudaError_t launch_ens_measure_t(const EnsBox<T>* boxes, const EnsDet* det, const EnsDyn* dyn, const Coef<T>* coef,
                                 const int* list, const long long* pre, int nlist, long long items, int k,
                                 const EnsViews<T>* views, cudaStream_t st) {
  const size_t bytes = sizeof(Smem<T, TileShape<T>::TX, TileShape<T>::TY, true, false>);
  static bool configured[64] = {};
  cudaError_t e = set_smem_attr(k_ens_measure<T, VIEWS>, bytes, configured);
  if (e != cudaSuccess) return e;
  if (items <= 0) return cudaSuccess;
  k_ens_measure<T, VIEWS><<<(unsigned)items, 256, bytes, st>>>(boxes, det, dyn, coef, list, pre, nlist, k,
                                                               views_or_empty(views));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ens_measure(const EnsBox<T>* boxes, const EnsDet* det, const EnsDyn* dyn, const Coef<T>* coef,
                               const int* list, const long long* pre, int nlist, long long items, int k,
                               const EnsViews<T>* views, cudaStream_t st) {
  return views ? launch_ens_measure_t<T, true>(boxes, det, dyn, coef, list, pre, nlist, items, k, views, st)
               : launch_ens_measure_t<T, false>(boxes, det, dyn, coef, list, pre, nlist, items, k, views, st);
}

template <typename T, bool VIEWS>
cudaError_t launch_ens_step_t(const EnsBox<T>* boxes, const EnsDyn* dyn, const Coef<T>* coef, const EnsSched& sc,
                              int k, long long items, const EnsViews<T>* views, cudaStream_t st) {
  const size_t bytes = ens_smem_bytes<T>();
  static bool configured[64] = {};
  cudaError_t e = set_smem_attr(k_ens_step<T, VIEWS>, bytes, configured);
  if (e != cudaSuccess) return e;
  if (items <= 0) return cudaSuccess;
  k_ens_step<T, VIEWS><<<(unsigned)items, 256, bytes, st>>>(boxes, dyn, coef, sc, k, views_or_empty(views));
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_ens_step(const EnsBox<T>* boxes, const EnsDyn* dyn, const Coef<T>* coef, const EnsSched& sc,
                            int k, long long items, const EnsViews<T>* views, cudaStream_t st) {
  return views ? launch_ens_step_t<T, true>(boxes, dyn, coef, sc, k, items, views, st)
               : launch_ens_step_t<T, false>(boxes, dyn, coef, sc, k, items, views, st);
}

cudaError_t launch_ens_advance(EnsDyn* dyn, const int* steps, int nboxes, int de, cudaStream_t st) {
  k_ens_advance<<<(nboxes + 127) / 128, 128, 0, st>>>(dyn, steps, nboxes, de);
  return cudaGetLastError();
}

template cudaError_t launch_ens_persistent<float>(const EnsBox<float>*, const EnsDyn*, const Coef<float>*,
                                                  const EnsSched&, const int*, unsigned long long*, unsigned*, int*,
                                                  long long, int, int, const EnsViews<float>*, cudaStream_t);
template cudaError_t launch_ens_persistent<double>(const EnsBox<double>*, const EnsDyn*, const Coef<double>*,
                                                   const EnsSched&, const int*, unsigned long long*, unsigned*, int*,
                                                   long long, int, int, const EnsViews<double>*, cudaStream_t);
template cudaError_t launch_ens_measure<float>(const EnsBox<float>*, const EnsDet*, const EnsDyn*, const Coef<float>*,
                                               const int*, const long long*, int, long long, int,
                                               const EnsViews<float>*, cudaStream_t);
template cudaError_t launch_ens_measure<double>(const EnsBox<double>*, const EnsDet*, const EnsDyn*,
                                                const Coef<double>*, const int*, const long long*, int, long long, int,
                                                const EnsViews<double>*, cudaStream_t);
template cudaError_t launch_ens_step<float>(const EnsBox<float>*, const EnsDyn*, const Coef<float>*, const EnsSched&,
                                            int, long long, const EnsViews<float>*, cudaStream_t);
template cudaError_t launch_ens_step<double>(const EnsBox<double>*, const EnsDyn*, const Coef<double>*,
                                             const EnsSched&, int, long long, const EnsViews<double>*, cudaStream_t);

template <typename T>
cudaError_t launch_tiled(int mode, const LatticeView<T>& v, const Coef<T>& c, const MeasureOut& mo,
                         cudaStream_t st, int waves, int* status) {
  if (!status) return cudaErrorInvalidValue;  // a copy timeout must reach its caller
  cudaError_t e;
  switch (mode) {
    case MODE_WRITE:
      return launch_mode<T, MODE_WRITE>(v, c, mo, st, waves, status);
    case MODE_WRITE | MODE_MEASURE:
      e = launch_mode<T, MODE_WRITE | MODE_MEASURE>(v, c, mo, st, waves, status);
      break;
    case MODE_MEASURE:
      e = launch_mode<T, MODE_MEASURE>(v, c, mo, st, waves, status);
      break;
    case MODE_MEASURE | MODE_GAUSS:
      e = launch_mode<T, MODE_MEASURE | MODE_GAUSS>(v, c, mo, st, waves, status);
      break;
    default:
      return cudaErrorInvalidValue;
  }
  if (e != cudaSuccess || !mo.faces) return e;
  // windings on the step's input positions (a writing step leaves them in
  // place: it writes the other position buffer)
  PosView<T> pv;
  for (int f = 0; f < U1U1_NPOS; ++f) pv.pos[f] = v.pin[f];
  pv.nx = v.nx;
  pv.ny = v.ny;
  pv.nz = v.nz;
  return launch_windings<T>(pv, c.dx, mo.partial + tiled_grid_blocks(v.nx, v.ny, v.nz, (int)sizeof(T), waves),
                            mo.faces, mo.windings, st);
}

int tiled_measure_blocks(int nx, int ny, int nz, int sizeof_t, int waves, bool windings) {
  return tiled_grid_blocks(nx, ny, nz, sizeof_t, waves) + (windings ? wind_grid_blocks(nx, ny, nz) : 0);
}

template cudaError_t launch_tiled<float>(int, const LatticeView<float>&, const Coef<float>&, const MeasureOut&,
                                         cudaStream_t, int, int*);
template cudaError_t launch_tiled<double>(int, const LatticeView<double>&, const Coef<double>&,
                                          const MeasureOut&, cudaStream_t, int, int*);

}  // namespace u1u1
