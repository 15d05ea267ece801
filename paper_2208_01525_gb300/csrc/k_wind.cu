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
// CTA: 8 warps x 32 lanes on a (32 x 8)-site window that advances by 31 in x
// and 7 in y, so that lane 31 and warp 7 hold the right column and the top
// row of the tile's halo: every thread computes the three edge phases of its
// own site per sector and no thread does extra halo work.  Neighbours in x
// come by warp shuffle, neighbours in y through a double-buffered shared
// plane (one barrier per plane), neighbours in z from the same thread's
// previous plane.  The CTA marches a chunk of planes [z0, z1) and emits the
// face byte of plane z-1 at plane z, like the step kernel's measuring pass
// did.
#include <stdint.h>

#include "reduce.cuh"
#include "site_math.cuh"
#include "u1u1_internal.cuh"

namespace u1u1 {

namespace {

constexpr int WW = 32;        // window width (lanes)
constexpr int WH = 8;         // window height (warps)
constexpr int WOX = WW - 1;   // output columns per tile
constexpr int WOY = WH - 1;   // output rows per tile
constexpr int WNT = WW * WH;  // threads per CTA
constexpr int WIND_MIN_LZ = 32;
constexpr int WIND_TARGET_CTAS = 152 * 4 * 16;  // 4 resident CTAs per SM, about 16 waves

// What the row below needs of a site: chi_0, chi_2, A_0, A_2 and the flags.
template <typename T>
struct WindRow {
  T chi0[2][WNT], chi2[2][WNT], a0[2][WNT], a2[2][WNT];
  uint8_t fl[2][WNT];
};

template <typename T>
struct WindSmem {
  WindRow<T> row[2];  // by plane parity
  int cnt[WH][NCNT];
};

// The three edge phases chi_i(x) = arg(conj(phi(x)) U_i(x) phi(x+i)) of one
// sector at one site, with their branch-cut bits (bit i: edge i).  Since
// |U_i| = 1 and arg U_i = -theta_i, chi_i is the principal value of
// alpha_i - theta_i with alpha_i = arg(conj(phi(x)) phi(x+i)) and
// theta_i = dx A_i(x): one arctangent and a reduction by the nearest multiple
// of 2 pi (2 pi split in two floats, Cody & Waite), instead of the link
// variable's cosine and sine, a transport and an arctangent.  Equal to the
// direct form up to rounding; the two can pick different branches only
// within rounding of +-pi, where the edge is flagged either way.
template <typename T> struct TwoPi;
template <> struct TwoPi<float> {
  static __device__ __forceinline__ float hi() { return 6.28318548202514648f; }   // fl(2 pi)
  static __device__ __forceinline__ float lo() { return -1.74845553e-07f; }       // 2 pi - fl(2 pi)
};
template <> struct TwoPi<double> {
  static __device__ __forceinline__ double hi() { return 6.28318530717958623; }
  static __device__ __forceinline__ double lo() { return 2.44929359829470641e-16; }
};

template <typename T>
__device__ __forceinline__ unsigned edge_phases(T fr, T fi, const T nbr[3], const T nbi[3], const T A[3], T dx,
                                                T chi[3]) {
  unsigned f = 0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const T zr = fr * nbr[i] + fi * nbi[i], zi = fr * nbi[i] - fi * nbr[i];
    T d = edge_phase<T>(zr, zi) - dx * A[i];
    const T k = rint_t<T>(d * Consts<T>::inv_two_pi());
    d = fma(-k, TwoPi<T>::hi(), d);
    d = fma(-k, TwoPi<T>::lo(), d);
    chi[i] = d;
    const bool cut = Consts<T>::pi() - fabs(d) < T(1e-4) || (zr == T(0) && zi == T(0));
    f |= cut ? (1u << i) : 0u;
  }
  return f;
}

template <typename T>
__global__ void __launch_bounds__(WNT, sizeof(T) == 8 ? 2 : 4)
k_windings(PosView<T> v, T dx, int lz, BlockPartial* part, uint8_t* faces, int8_t* windings) {
  __shared__ WindSmem<T> sm;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nx = v.nx, ny = v.ny, nz = v.nz;
  const int x0 = blockIdx.x * WOX, y0 = blockIdx.y * WOY;
  const int z0 = blockIdx.z * lz, z1 = min(z0 + lz, nz);
  const int gx = (x0 + lane) % nx, gy = (y0 + w) % ny;
  const int gyn = gy + 1 == ny ? 0 : gy + 1;
  const bool out = lane < WOX && w < WOY && x0 + lane < nx && y0 + w < ny;
  const long long plane = (long long)nx * ny;
  const long long V = plane * nz;
  const long long col = (long long)gy * nx + gx, coln = (long long)gyn * nx + gx;

  int cnt[NCNT];
#pragma unroll
  for (int k = 0; k < NCNT; ++k) cnt[k] = 0;

  // own phi and A of the current plane (loaded one plane ahead)
  T fr[2], fi[2], A[2][3];
  {
    const long long o = (long long)z0 * plane + col;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      fr[s] = __ldg(v.pos[2 * s] + o);
      fi[s] = __ldg(v.pos[2 * s + 1] + o);
#pragma unroll
      for (int i = 0; i < 3; ++i) A[s][i] = __ldg(v.pos[4 + 3 * s + i] + o);
    }
  }
  // plaquettes of the plane below still waiting for this plane's chi_0, chi_1
  int pW01[2] = {0, 0};
  T pS02[2] = {T(0), T(0)}, pS12[2] = {T(0), T(0)};
  unsigned pcut[2] = {0u, 0u};

  for (int z = z0; z <= z1; ++z) {
    const int zc = z == nz ? 0 : z;            // plane z1 may wrap
    const int zn = zc + 1 == nz ? 0 : zc + 1;  // plane above
    const long long oc = (long long)zc * plane, on = (long long)zn * plane;
    const bool last = z == z1;
    // neighbours of the own site: x+1 by shuffle, y+1 and z+1 from memory
    T nbr[2][3], nbi[2][3], An[2][3];
    T frn[2], fin[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      nbr[s][0] = __shfl_down_sync(0xffffffffu, fr[s], 1);
      nbi[s][0] = __shfl_down_sync(0xffffffffu, fi[s], 1);
      nbr[s][1] = __ldg(v.pos[2 * s] + oc + coln);
      nbi[s][1] = __ldg(v.pos[2 * s + 1] + oc + coln);
      frn[s] = __ldg(v.pos[2 * s] + on + col);
      fin[s] = __ldg(v.pos[2 * s + 1] + on + col);
      nbr[s][2] = frn[s];
      nbi[s][2] = fin[s];
#pragma unroll
      for (int i = 0; i < 3; ++i) An[s][i] = last ? T(0) : __ldg(v.pos[4 + 3 * s + i] + on + col);
    }
    T chi[2][3];
    unsigned f[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) f[s] = edge_phases<T>(fr[s], fi[s], nbr[s], nbi[s], A[s], dx, chi[s]);

    // finish and emit the plane below
    if (z > z0 && out) {
      const long long gs = (long long)(z - 1) * plane + col;
      unsigned nzm[2];
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const int W0 = pW01[s];
        const int W1 = (int)rint_t<T>((pS02[s] - chi[s][0]) * Consts<T>::inv_two_pi());
        const int W2 = (int)rint_t<T>((pS12[s] - chi[s][1]) * Consts<T>::inv_two_pi());
        // flagged plaquettes: an edge of this plane or of the plane above on the cut
        const unsigned ckm = (pcut[s] & 1u) | (((pcut[s] & 2u) || (f[s] & 1u)) ? 2u : 0u) |
                             (((pcut[s] & 4u) || (f[s] & 2u)) ? 4u : 0u);
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
      cnt[C_NPQ_PLAQ] += __popc(nzm[0] & nzm[1]);
    }
    if (last) break;

    // exchange with the row below: it needs chi_0, chi_2, A_0, A_2, flags
    WindRow<T>& r = sm.row[z & 1];
    const int t = threadIdx.x;
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      r.chi0[s][t] = chi[s][0];
      r.chi2[s][t] = chi[s][2];
      r.a0[s][t] = A[s][0];
      r.a2[s][t] = A[s][2];
      r.fl[s][t] = (uint8_t)f[s];
    }
    __syncthreads();
    const int ty = w + 1 < WH ? t + WW : t;  // the top row reads itself (its results are not used)
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const T c1x = __shfl_down_sync(0xffffffffu, chi[s][1], 1);
      const T c2x = __shfl_down_sync(0xffffffffu, chi[s][2], 1);
      const T a1x = __shfl_down_sync(0xffffffffu, A[s][1], 1);
      const T a2x = __shfl_down_sync(0xffffffffu, A[s][2], 1);
      const unsigned fx = __shfl_down_sync(0xffffffffu, f[s], 1);
      const T c0y = r.chi0[s][ty], c2y = r.chi2[s][ty], a0y = r.a0[s][ty], a2y = r.a2[s][ty];
      const unsigned fy = r.fl[s][ty];
      const T F01 = curl_ft<T>(a1x, A[s][1], a0y, A[s][0]);
      const T F02 = curl_ft<T>(a2x, A[s][2], An[s][0], A[s][0]);
      const T F12 = curl_ft<T>(a2y, A[s][2], An[s][1], A[s][1]);
      pW01[s] = plaquette_winding<T>(chi[s][0], c1x, c0y, chi[s][1], dx, F01);
      pS02[s] = (chi[s][0] + c2x) - chi[s][2] + dx * F02;
      pS12[s] = (chi[s][1] + c2y) - chi[s][2] + dx * F12;
      const unsigned f0 = f[s];
      pcut[s] = (((f0 & 3u) || (fx & 2u) || (fy & 1u)) ? 1u : 0u) | (((f0 & 5u) || (fx & 4u)) ? 2u : 0u) |
                (((f0 & 6u) || (fy & 4u)) ? 4u : 0u);
      fr[s] = frn[s];
      fi[s] = fin[s];
#pragma unroll
      for (int i = 0; i < 3; ++i) A[s][i] = An[s][i];
    }
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
  BlockPartial* p = part + ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
  const int t = threadIdx.x;
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
