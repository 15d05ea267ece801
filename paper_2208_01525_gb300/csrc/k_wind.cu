// Plaquette windings of both sectors (Sec. III.A) for the tiled measuring
// passes.
//
// The windings are taken on the positions (phi^n, A^n) the step kernel reads;
// a step writes its positions to the other buffer, so this kernel reads them
// after (or before) the fused step at no risk and the step kernel keeps no
// winding state.  Doing it here rather than inside the step kernel costs one
// more read of the ten position fields (40 B/site in FP32) but lets the edge
// phases run at the occupancy of a small kernel: inside the step kernel they
// lengthened every thread's dependency chain at two resident CTAs per SM.
//
// Per-site phases.  With alpha(x) = arg phi(x), the edge phase
// chi_i(x) = arg(conj(phi(x)) U_i(x) phi(x+i)) is the principal value of
// d_i(x) = alpha(x+i) - alpha(x) - theta_i(x), theta_i = dx A_i, i.e.
// chi_i = d_i - 2 pi k_i with the integer k_i = rint(d_i / 2 pi).  Around a
// plaquette the alpha differences cancel exactly and the thetas cancel
// against those of the curl term, so the winding of plaquette (x; i, j) is the
// integer
//   W_ij(x) = -(k_i(x) + k_j(x+i) - k_i(x+j) - k_j(x)),
// equal to the rounded sum of the four chi plus dx^2 F_ij over 2 pi.  That
// takes one arctangent per site and sector instead of one per link; the k
// and the flag depend on the rounding of d only within rounding of an odd
// multiple of pi, where chi is within rounding of +-pi and the edge is
// flagged (pi - |chi| < 1e-4).  A zero field makes alpha undefined: alpha is
// stored as NaN there, so every edge touching the site is flagged and every
// plaquette with such an edge gets W = 0.  The k are kept as floating-point
// integers: their four-term sums are exact, and each winding is converted
// to an integer once.
//
// CTA: 12 warps x 32 lanes on a (32 x 12)-site window that advances by 31 in
// x and 11 in y, so that lane 31 and warp 11 hold the right column and the
// top row of the tile's halo.  The halo threads compute edges they do not
// emit: 12 rows waste 1/12 of them against 1/8 for 8 rows (measured at
// 1024^3, FP32: the standalone string detection 16.02 against 16.25 ms; 16
// rows, which fit one CTA per SM, took 17.0 ms).  Each thread computes alpha of its own site once
// per sector and plane, and the branch integers of its own three edges.
// alpha of x+1 comes by warp shuffle, alpha of the row above from a
// three-plane shared ring (one barrier per plane), alpha of z+1 from the
// thread's next plane, whose raw fields are prefetched a plane ahead.  Each
// row publishes its k_0 and k_2 (and cut bits) in a two-plane ring; the row
// below reads them after the next barrier.  So the CTA marches a chunk of
// planes [z0, z1) and emits the face byte of plane z-1 at plane z, when the
// row above's edges of plane z-1 and its own k_0 and k_1 of plane z complete
// the 01, 02 and 12 plaquettes.
#include <stdint.h>

#include "reduce.cuh"
#include "site_math.cuh"
#include "u1u1_internal.cuh"

namespace u1u1 {

namespace {

constexpr int WW = 32;        // window width (lanes)
constexpr int WH = 12;        // window height (warps)
constexpr int WOX = WW - 1;   // output columns per tile
constexpr int WOY = WH - 1;   // output rows per tile
constexpr int WNT = WW * WH;  // threads per CTA
constexpr int WIND_MIN_LZ = 32;
constexpr int WIND_TARGET_CTAS = 152 * 2 * 16;  // 2 resident CTAs per SM, about 16 waves

// What the row below needs of a site: alpha of each plane (three-plane
// ring), and, one plane later, the branch integers of edges 0 and 2 with
// their cut bits (two-plane ring).
template <typename T>
struct WindEdges {
  T k0[2][WNT], k2[2][WNT];
  uint8_t cut[2][WNT];  // bit 0: edge 0, bit 2: edge 2
};

template <typename T>
struct WindSmem {
  T al[3][2][WNT];      // by plane index mod 3
  WindEdges<T> e[2];    // by plane index mod 2
  int cnt[WH][NCNT];
};

// alpha = arg(re + i im), NaN for a zero field
template <typename T>
__device__ __forceinline__ T site_phase(T re, T im) {
  const T a = edge_phase<T>(re, im);
  return (re == T(0) && im == T(0)) ? T(NAN) : a;
}

template <typename T> __device__ __forceinline__ int round_int(T x);
template <> __device__ __forceinline__ int round_int<float>(float x) { return __float2int_rn(x); }  // NaN -> 0
template <> __device__ __forceinline__ int round_int<double>(double x) { return __double2int_rn(x); }

// |chi| > pi - 1e-4 in units of 2 pi: |d / 2 pi - k| > 1/2 - 1e-4 / (2 pi)
template <typename T> __device__ __forceinline__ T cut_frac();
template <> __device__ __forceinline__ float cut_frac<float>() { return 0.49998408451f; }
template <> __device__ __forceinline__ double cut_frac<double>() { return 0.49998408450991098; }

// Branch integer k of the edge from a site of phase a_t to a site of phase
// a_h across a link of angle theta, as a floating-point integer (sums of a
// few k are exact), and whether the edge is flagged (near the cut, or a zero
// field at either end: then d and k are NaN and the test below fails; a
// plaquette with such an edge gets W = 0).
template <typename T>
__device__ __forceinline__ T edge_k(T a_h, T a_t, T theta, unsigned* cut) {
  const T t = ((a_h - a_t) - theta) * Consts<T>::inv_two_pi();
  const T k = rint_t<T>(t);
  *cut = (fabs(t - k) <= cut_frac<T>()) ? 0u : 1u;
  return k;
}

// One window column (tile (bx, by), planes [bz lz, bz lz + lz)) of the
// windings pass; its counts go to the block partial *p.
template <typename T>
__device__ __forceinline__ void windings_tile(const PosView<T>& v, T dx, int lz, int bx, int by, int bz,
                                              BlockPartial* p, uint8_t* faces, int8_t* windings) {
  __shared__ WindSmem<T> sm;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, t = threadIdx.x;
  const int nx = v.nx, ny = v.ny, nz = v.nz;
  const int x0 = bx * WOX, y0 = by * WOY;
  const int z0 = bz * lz, z1 = min(z0 + lz, nz);
  const int gx = (x0 + lane) % nx, gy = (y0 + w) % ny;
  const bool out = lane < WOX && w < WOY && x0 + lane < nx && y0 + w < ny;
  const long long plane = (long long)nx * ny;
  const long long V = plane * nz;
  const long long col = (long long)gy * nx + gx;
  const int ty = w + 1 < WH ? t + WW : t;  // the row above (the top row reads itself; unused)

  int cnt[NCNT];
#pragma unroll
  for (int k = 0; k < NCNT; ++k) cnt[k] = 0;

  // own alpha and A of the current plane; raw fields of the next plane
  T al[2], A[2][3], nfr[2], nfi[2], nA[2][3];
  auto load_plane = [&](int zz, T fr_[2], T fi_[2], T A_[2][3]) {
    const long long o = (long long)(zz >= nz ? zz - nz : zz) * plane + col;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      fr_[s] = __ldg(v.pos[2 * s] + o);
      fi_[s] = __ldg(v.pos[2 * s + 1] + o);
#pragma unroll
      for (int i = 0; i < 3; ++i) A_[s][i] = __ldg(v.pos[4 + 3 * s + i] + o);
    }
  };
  {
    T fr[2], fi[2];
    load_plane(z0, fr, fi, A);
    load_plane(z0 + 1, nfr, nfi, nA);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      al[s] = site_phase<T>(fr[s], fi[s]);
      sm.al[z0 % 3][s][t] = al[s];
    }
  }
  // the plane below's plaquettes, short of the edges of this plane (and, for
  // 01 and 12, of the row above): W01 = P01 + k0(x+y), W02 = P02 + k0(x+z),
  // W12 = P12 - k2(x+y) + k1(x+z); cut bits likewise
  T P01[2] = {T(0), T(0)}, P02[2] = {T(0), T(0)}, P12[2] = {T(0), T(0)};
  unsigned pc[2] = {0u, 0u};  // bit 0: 01, bit 1: 02, bit 2: 12

  for (int z = z0; z <= z1; ++z) {
    const bool last = z == z1;
    // next plane: alpha from the prefetched fields, into the ring; prefetch
    // the plane after it
    T aln[2], An[2][3];
    if (!last) {
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        aln[s] = site_phase<T>(nfr[s], nfi[s]);
#pragma unroll
        for (int i = 0; i < 3; ++i) An[s][i] = nA[s][i];
        sm.al[(z + 1) % 3][s][t] = aln[s];
      }
      if (z + 1 < z1) load_plane(z + 2, nfr, nfi, nA);
    }
    __syncthreads();
    const WindEdges<T>& eb = sm.e[(z + 1) & 1];  // the row above's edges of plane z-1
    WindEdges<T>& ec = sm.e[z & 1];              // this row's edges of plane z

    unsigned nzm[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      // own edges 0 and 1 of this plane
      const T ax = __shfl_down_sync(0xffffffffu, al[s], 1);
      const T ay = sm.al[z % 3][s][ty];
      unsigned c0, c1;
      const T k0 = edge_k<T>(ax, al[s], dx * A[s][0], &c0);
      const T k1 = edge_k<T>(ay, al[s], dx * A[s][1], &c1);

      // finish and emit the plane below
      if (z > z0 && out) {
        const long long gs = (long long)(z - 1) * plane + col;
        const unsigned cy = eb.cut[s][ty];
        const int W0 = round_int<T>(P01[s] + eb.k0[s][ty]);  // NaN (flagged) -> 0
        const int W1 = round_int<T>(P02[s] + k0);
        const int W2 = round_int<T>(P12[s] - eb.k2[s][ty] + k1);
        const unsigned ckm = pc[s] | (cy & 1u) | (c0 << 1) | ((c1 | (cy >> 2)) << 2);
        const int a0 = abs(W0), a1 = abs(W1), a2 = abs(W2);
        unsigned byte = (unsigned)min(a0, 3) | ((unsigned)min(a1, 3) << FACE_SHIFT(1)) |
                        ((unsigned)min(a2, 3) << FACE_SHIFT(2));
        nzm[s] = (byte | (byte >> 1)) & 0x15u;  // bit 2k: |W_k| >= 1
        cnt[s == 0 ? C_NP : C_NQ] += a0 + a1 + a2;
        cnt[s == 0 ? C_NZP : C_NZQ] += __popc(nzm[s]);
        cnt[s == 0 ? C_W2P : C_W2Q] += __popc((byte >> 1) & 0x15u);  // |W_k| >= 2
        cnt[C_FLAGGED] += __popc(ckm);
        cnt[C_MAXW] = max(cnt[C_MAXW], max(a0, max(a1, a2)));
        if (ckm) byte |= FACE_FLAG;
        faces[s * V + gs] = (uint8_t)byte;
        if (windings) {
          windings[(3 * s + 0) * V + gs] = (int8_t)max(-127, min(127, W0));
          windings[(3 * s + 1) * V + gs] = (int8_t)max(-127, min(127, W1));
          windings[(3 * s + 2) * V + gs] = (int8_t)max(-127, min(127, W2));
        }
      }
      if (last) continue;

      // own edge 2; publish edges 0 and 2 for the row below
      unsigned c2;
      const T k2 = edge_k<T>(aln[s], al[s], dx * A[s][2], &c2);
      ec.k0[s][t] = k0;
      ec.k2[s][t] = k2;
      ec.cut[s][t] = (uint8_t)(c0 | (c2 << 2));
      // edges 1 and 2 of x + x by shuffle
      const unsigned cb = c1 | (c2 << 1);
      const T k1x = __shfl_down_sync(0xffffffffu, k1, 1);
      const T k2x = __shfl_down_sync(0xffffffffu, k2, 1);
      const unsigned cx = __shfl_down_sync(0xffffffffu, cb, 1);
      P01[s] = -(k0 + k1x - k1);  // + k_0 of the row above
      P02[s] = -(k0 + k2x - k2);  // + k_0 of the plane above
      P12[s] = -(k1 - k2);        // - k_2 of the row above + k_1 of the plane above
      pc[s] = (c0 | (cx & 1u) | c1) | ((c0 | (cx >> 1) | c2) << 1) | ((c1 | c2) << 2);
      al[s] = aln[s];
#pragma unroll
      for (int i = 0; i < 3; ++i) A[s][i] = An[s][i];
    }
    if (z > z0 && out) cnt[C_NPQ_PLAQ] += __popc(nzm[0] & nzm[1]);
  }

  // block reduction of the counts (maximum for C_MAXW)
#pragma unroll
  for (int k = 0; k < NCNT; ++k) {
    int vk = cnt[k];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const int u = __shfl_down_sync(0xffffffffu, vk, o);
      vk = (k == C_MAXW) ? max(vk, u) : vk + u;
    }
    if (lane == 0) sm.cnt[w][k] = vk;
  }
  __syncthreads();
  if (t < NSUM) {
    p->sum[t] = 0.0;
    p->comp[t] = 0.0;
  } else if (t < NSUM + NMAX) {
    p->mx[t - NSUM] = -INFINITY;
  } else if (t < NSUM + NMAX + NCNT) {
    const int k = t - NSUM - NMAX;
    long long acc = 0;
    for (int ww = 0; ww < WH; ++ww) acc = (k == C_MAXW) ? max(acc, (long long)sm.cnt[ww][k]) : acc + sm.cnt[ww][k];
    p->cnt[k] = acc;
  }
}

template <typename T>
__global__ void __launch_bounds__(WNT, sizeof(T) == 8 ? 1 : 2)
k_windings(PosView<T> v, T dx, int lz, BlockPartial* part, uint8_t* faces, int8_t* windings) {
  BlockPartial* p = part + ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  windings_tile<T>(v, dx, lz, blockIdx.x, blockIdx.y, blockIdx.z, p, faces, windings);
}

// Windings of the boxes of an ensemble that detect at step k of a run, one
// CTA per window column of any of them: the same windows, chunking and
// partial slots as a single lattice's pass, on each box's input positions
// of step k.
template <typename T>
__global__ void __launch_bounds__(WNT, sizeof(T) == 8 ? 1 : 2)
k_ens_windings(const EnsBox<T>* __restrict__ boxes, const EnsDet* __restrict__ det, const EnsDyn* __restrict__ dyn,
               const int* __restrict__ list, const long long* __restrict__ pre, int nlist, int k) {
  const long long r = blockIdx.x;
  const int si = ens_list_index(pre, nlist, r);
  const int b = list[si];
  const long long t = r - pre[si];
  const EnsBox<T>& B = boxes[b];
  const EnsDet& D = det[b];
  const int bx = (int)(t % D.wtx), by = (int)((t / D.wtx) % D.wty), bz = (int)(t / ((long long)D.wtx * D.wty));
  PosView<T> v;
  const int par = (dyn[b].cur + k) & 1;
#pragma unroll
  for (int f = 0; f < U1U1_NPOS; ++f) v.pos[f] = B.pos[par][f];
  v.nx = B.nx;
  v.ny = B.ny;
  v.nz = B.nz;
  windings_tile<T>(v, B.dx, D.wlz, bx, by, bz, D.part + D.nmeas + t, D.faces, nullptr);
}

void wind_grid(int nx, int ny, int nz, dim3* grid, int* lz) {
  const int tx = (nx + WOX - 1) / WOX, ty = (ny + WOY - 1) / WOY;
  const long long tiles = (long long)tx * ty;
  int chunks = (int)((WIND_TARGET_CTAS + tiles - 1) / tiles);
  chunks = max(1, min(chunks, nz / WIND_MIN_LZ));
  const int l = (nz + chunks - 1) / chunks;
  *lz = l;
  *grid = dim3(tx, ty, (nz + l - 1) / l);
}

}  // namespace

int wind_grid_blocks(int nx, int ny, int nz) {
  dim3 g;
  int lz;
  wind_grid(nx, ny, nz, &g, &lz);
  return (int)(g.x * g.y * g.z);
}

void wind_grid_dims(int nx, int ny, int nz, int* tx, int* ty, int* tz, int* lz) {
  dim3 g;
  wind_grid(nx, ny, nz, &g, lz);
  *tx = (int)g.x;
  *ty = (int)g.y;
  *tz = (int)g.z;
}

template <typename T>
cudaError_t launch_ens_windings(const EnsBox<T>* boxes, const EnsDet* det, const EnsDyn* dyn, const int* list,
                                const long long* pre, int nlist, long long items, int k, cudaStream_t st) {
  if (items <= 0) return cudaSuccess;
  k_ens_windings<T><<<(unsigned)items, WNT, 0, st>>>(boxes, det, dyn, list, pre, nlist, k);
  return cudaGetLastError();
}
template cudaError_t launch_ens_windings<float>(const EnsBox<float>*, const EnsDet*, const EnsDyn*, const int*,
                                                const long long*, int, long long, int, cudaStream_t);
template cudaError_t launch_ens_windings<double>(const EnsBox<double>*, const EnsDet*, const EnsDyn*, const int*,
                                                 const long long*, int, long long, int, cudaStream_t);

template <typename T>
cudaError_t launch_windings(const PosView<T>& v, T dx, BlockPartial* part, uint8_t* faces, int8_t* windings,
                            cudaStream_t st) {
  dim3 g;
  int lz;
  wind_grid(v.nx, v.ny, v.nz, &g, &lz);
  k_windings<T><<<g, WNT, 0, st>>>(v, dx, lz, part, faces, windings);
  return cudaGetLastError();
}

template cudaError_t launch_windings<float>(const PosView<float>&, float, BlockPartial*, uint8_t*, int8_t*,
                                            cudaStream_t);
template cudaError_t launch_windings<double>(const PosView<double>&, double, BlockPartial*, uint8_t*, int8_t*,
                                             cudaStream_t);

}  // namespace u1u1
