// Cell arrays, fast bound-state overlap (Sec. III.B) and the deterministic
// reduction finalize.
//
// Pass 1 (k_cellbits) turns the per-site face bytes written by the measuring
// kernels into cell values c_s(x) = sum over the six faces of cell x of |W|
// (optionally stored as uint8 cell arrays) and into one bit per cell and
// sector ("pierced"), packed 32 cells of a lattice row per word with a warp
// ballot.  Pass 2 (k_overlap) counts p-pierced cells that have a q-pierced
// cell in their (2 tol + 1)^3 neighbourhood -- a box, so the neighbourhood
// test is an OR of shifted words over 3 x 3 rows -- and the same with the
// roles swapped, with popcounts.
#include <stdint.h>

#include "reduce.cuh"
#include "u1u1_internal.cuh"

namespace u1u1 {

namespace {

constexpr int ROWS_PER_BLOCK = 8;
constexpr int BITS_BLOCKS_Y = 2048;
constexpr int OVL_THREADS = 256;
constexpr int OVL_BLOCKS = 152 * 8;

__device__ __forceinline__ int face_w(const uint8_t* f, long long i, int k) { return (f[i] >> FACE_SHIFT(k)) & 3; }

__global__ void __launch_bounds__(32 * ROWS_PER_BLOCK)
k_cellbits(const uint8_t* __restrict__ faces, int nx, int ny, int nz, int words, uint8_t* cell_p, uint8_t* cell_q,
           uint32_t* mp, uint32_t* mq, unsigned long long* ge4) {
  const long long V = (long long)nx * ny * nz;
  const long long nrows = (long long)ny * nz;
  const int lane = threadIdx.x;
  const int w = blockIdx.x;
  const int x = w * 32 + lane;
  unsigned long long n4[2] = {0ull, 0ull};  // this warp's cells of value >= 4 (lane 0)
  for (long long row = (long long)blockIdx.y * ROWS_PER_BLOCK + threadIdx.y; row < nrows;
       row += (long long)gridDim.y * ROWS_PER_BLOCK) {
    const int y = (int)(row % ny), z = (int)(row / ny);
    int c[2] = {0, 0};
    if (x < nx) {
      const long long i = row * nx + x;
      const long long ix = row * nx + (x + 1 == nx ? 0 : x + 1);
      const long long iy = ((long long)z * ny + (y + 1 == ny ? 0 : y + 1)) * nx + x;
      const long long iz = ((long long)(z + 1 == nz ? 0 : z + 1) * ny + y) * nx + x;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const uint8_t* f = faces + s * V;
        c[s] = face_w(f, i, 0) + face_w(f, iz, 0) + face_w(f, i, 1) + face_w(f, iy, 1) + face_w(f, i, 2) +
               face_w(f, ix, 2);
      }
      if (cell_p) cell_p[i] = (uint8_t)c[0];
      if (cell_q) cell_q[i] = (uint8_t)c[1];
    }
    const uint32_t bp = __ballot_sync(0xffffffffu, c[0] > 0);
    const uint32_t bq = __ballot_sync(0xffffffffu, c[1] > 0);
    if (lane == 0) {
      mp[row * words + w] = bp;
      mq[row * words + w] = bq;
    }
    if (ge4) {
      // census of cells pierced by winding two or more (value >= 4)
      n4[0] += (unsigned long long)__popc(__ballot_sync(0xffffffffu, c[0] >= 4));
      n4[1] += (unsigned long long)__popc(__ballot_sync(0xffffffffu, c[1] >= 4));
    }
  }
  if (ge4) {
    // one atomic per block and sector: the dense early network has value-4
    // cells in most rows, and per-row atomics on two counters serialised
    __shared__ unsigned long long s4[ROWS_PER_BLOCK][2];
    if (lane == 0) {
      s4[threadIdx.y][0] = n4[0];
      s4[threadIdx.y][1] = n4[1];
    }
    __syncthreads();
    if (threadIdx.y == 0 && lane < 2) {
      unsigned long long t = 0;
      for (int r = 0; r < ROWS_PER_BLOCK; ++r) t += s4[r][lane];
      if (t) atomicAdd(&ge4[lane], t);
    }
  }
}

constexpr int BITS4_THREADS = 256;
constexpr int BITS4_BLOCKS = 152 * 8;

// k_cellbits for rows whose length nx is a multiple of 32, sixteen cells
// per lane: 16-byte loads of the face bytes of the row, of the row above
// (y+1) and of the plane above (z+1), so that each lane has 48 bytes per
// sector in flight (four-byte loads left the pass at 1.2 TB/s).  The x+1
// face byte of the sixteenth cell comes from the next lane (from memory at
// a segment's end).  A warp covers a 512-cell segment of one row; two lanes'
// sixteen pierced bits form one mask word.
constexpr int SEG16 = 512;

__device__ __forceinline__ uint32_t cells4(uint32_t own, uint32_t nxt, uint32_t up, uint32_t ab) {
  // four cells, one byte each: six 2-bit |W| fields summed bytewise (at most
  // 18, so no carry crosses a byte)
  const uint32_t M = 0x03030303u;
  const uint32_t ox = (own >> 8) | (nxt << 24);  // byte j: face byte of x + j + 1
  return (own & M) + (ab & M) + ((own >> 2) & M) + ((up >> 2) & M) + ((own >> 4) & M) + ((ox >> 4) & M);
}

__global__ void __launch_bounds__(BITS4_THREADS)
k_cellbits16(const uint8_t* __restrict__ faces, int nx, int ny, int nz, int words, uint8_t* cell_p, uint8_t* cell_q,
             uint32_t* mp, uint32_t* mq, unsigned long long* ge4) {
  const long long V = (long long)nx * ny * nz;
  const long long nrows = (long long)ny * nz;
  const int lane = threadIdx.x & 31;
  const int segs = (nx + SEG16 - 1) / SEG16;
  const long long items = nrows * segs;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  unsigned long long n4[2] = {0ull, 0ull};
  for (long long it = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; it < items; it += nwarps) {
    const long long row = it / segs;
    const int sg = (int)(it % segs);
    const int y = (int)(row % ny), z = (int)(row / ny);
    const int x = sg * SEG16 + 16 * lane;  // this lane's first cell
    const bool act = x < nx;               // whole pairs of lanes (nx % 32 == 0)
    const long long rb = row * nx;
    const long long rby = ((long long)z * ny + (y + 1 == ny ? 0 : y + 1)) * nx;
    const long long rbz = ((long long)(z + 1 == nz ? 0 : z + 1) * ny + y) * nx;
    uint32_t bits[2], n4b[2];
    uint4 cv[2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      const uint8_t* f = faces + s * V;
      const uint4 z4 = make_uint4(0u, 0u, 0u, 0u);
      const uint4 own = act ? __ldg((const uint4*)(f + rb + x)) : z4;
      const uint4 up = act ? __ldg((const uint4*)(f + rby + x)) : z4;
      const uint4 ab = act ? __ldg((const uint4*)(f + rbz + x)) : z4;
      uint32_t nxt = __shfl_down_sync(0xffffffffu, own.x, 1);
      if (act && (lane == 31 || x + 16 >= nx)) nxt = __ldg((const uint32_t*)(f + rb + (x + 16 >= nx ? 0 : x + 16)));
      const uint32_t c0 = cells4(own.x, own.y, up.x, ab.x);
      const uint32_t c1 = cells4(own.y, own.z, up.y, ab.y);
      const uint32_t c2 = cells4(own.z, own.w, up.z, ab.z);
      const uint32_t c3 = cells4(own.w, nxt, up.w, ab.w);
      cv[s] = make_uint4(c0, c1, c2, c3);
      // bit 7 of byte j set when cell j is > 0 (>= 4): adding 127 (124) cannot
      // carry out of a byte below 129; the multiply gathers bit 0 of bytes
      // 0..3 into bits 0..3
      uint32_t b = 0, g = 0;
      const uint32_t cs[4] = {c0, c1, c2, c3};
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        b |= ((((cs[k] + 0x7F7F7F7Fu) & 0x80808080u) >> 7) * 0x01020408u >> 24) << (4 * k);
        g += __popc((cs[k] + 0x7C7C7C7Cu) & 0x80808080u);
      }
      bits[s] = b;
      n4b[s] = g;
    }
    if (act) {
      if (cell_p) *(uint4*)(cell_p + rb + x) = cv[0];
      if (cell_q) *(uint4*)(cell_q + rb + x) = cv[1];
    }
    // two lanes' sixteen bits form one word
    const uint32_t wp = (bits[0] << (16 * (lane & 1))) | __shfl_xor_sync(0xffffffffu, bits[0] << (16 * (lane & 1)), 1);
    const uint32_t wq = (bits[1] << (16 * (lane & 1))) | __shfl_xor_sync(0xffffffffu, bits[1] << (16 * (lane & 1)), 1);
    if (act && (lane & 1) == 0) {
      const long long wi = row * words + sg * (SEG16 / 32) + (lane >> 1);
      mp[wi] = wp;
      mq[wi] = wq;
    }
    if (act) {
      n4[0] += n4b[0];
      n4[1] += n4b[1];
    }
  }
  if (ge4) {
    __shared__ unsigned long long s4[BITS4_THREADS / 32][2];
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      unsigned long long v = n4[s];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
      if (lane == 0) s4[threadIdx.x >> 5][s] = v;
    }
    __syncthreads();
    if (threadIdx.x < 2) {
      unsigned long long t = 0;
      for (int w = 0; w < BITS4_THREADS / 32; ++w) t += s4[w][threadIdx.x];
      if (t) atomicAdd(&ge4[threadIdx.x], t);
    }
  }
}

// Bits of the row (y, z) dilated by one cell in x, periodic in x.
__device__ __forceinline__ uint32_t xdilate(const uint32_t* m, long long rowbase, int w, int words, int nx) {
  const uint32_t cur = m[rowbase + w];
  const int last_bit_row = (nx - 1) & 31;                  // bit of x = nx-1 in the last word
  const uint32_t left_in = (w > 0) ? (m[rowbase + w - 1] >> 31) & 1u
                                   : (m[rowbase + words - 1] >> last_bit_row) & 1u;
  const int top = (w < words - 1) ? 31 : last_bit_row;      // last valid bit of this word
  const uint32_t right_in = (w < words - 1) ? (m[rowbase + w + 1] & 1u) : (m[rowbase] & 1u);
  uint32_t d = cur | (cur << 1) | (cur >> 1) | left_in | (right_in << top);
  const uint32_t valid = (top == 31) ? 0xffffffffu : ((1u << (top + 1)) - 1u);
  return d & valid;
}

__global__ void __launch_bounds__(OVL_THREADS)
k_overlap(const uint32_t* __restrict__ mp, const uint32_t* __restrict__ mq, int nx, int ny, int nz, int words,
          int tol, CellPartial* part, uint32_t* mpq) {
  const long long nw = (long long)ny * nz * words;
  long long cnt[2] = {0, 0};
  for (long long idx = blockIdx.x * (long long)blockDim.x + threadIdx.x; idx < nw;
       idx += (long long)gridDim.x * blockDim.x) {
    const int w = (int)(idx % words);
    const long long row = idx / words;
    const int y = (int)(row % ny), z = (int)(row / ny);
    const uint32_t p = mp[idx], q = mq[idx];
    if (tol == 0) {
      cnt[0] += __popc(p & q);
      cnt[1] += __popc(p & q);
      if (mpq) mpq[idx] = p & q;
      continue;
    }
    if ((p | q) == 0) {
      if (mpq) mpq[idx] = 0u;
      continue;
    }
    uint32_t dq = 0, dp = 0;
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = z + dz < 0 ? nz - 1 : (z + dz >= nz ? 0 : z + dz);
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = y + dy < 0 ? ny - 1 : (y + dy >= ny ? 0 : y + dy);
        const long long rb = ((long long)zz * ny + yy) * words;
        if (p) dq |= xdilate(mq, rb, w, words, nx);
        if (q) dp |= xdilate(mp, rb, w, words, nx);
      }
    }
    cnt[0] += __popc(p & dq);
    cnt[1] += __popc(q & dp);
    if (mpq) mpq[idx] = p & dq;  // the p-anchored bound-state cells
  }
  __shared__ long long sm[OVL_THREADS / 32][2];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  for (int a = 0; a < 2; ++a) {
    const long long v = warp_sum_ll(cnt[a]);
    if (lane == 0) sm[warp][a] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    long long v = 0;
    for (int k = 0; k < OVL_THREADS / 32; ++k) v += sm[k][threadIdx.x];
    part[blockIdx.x].pq[threadIdx.x] = v;
  }
}

// k_overlap for rows of exactly 32 mask words (nx = 1024): one warp per row,
// lane = word, so the words left and right of a lane's word come by shuffle
// (periodic in x within the warp) and each of the nine neighbour rows costs
// one load per mask.
__global__ void __launch_bounds__(OVL_THREADS)
k_overlap_row32(const uint32_t* __restrict__ mp, const uint32_t* __restrict__ mq, int ny, int nz, int tol,
                CellPartial* part, uint32_t* mpq) {
  const long long nrows = (long long)ny * nz;
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  long long cnt[2] = {0, 0};
  for (long long row = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; row < nrows; row += nwarps) {
    const int y = (int)(row % ny), z = (int)(row / ny);
    const long long idx = row * 32 + lane;
    const uint32_t p = mp[idx], q = mq[idx];
    if (tol == 0) {
      cnt[0] += __popc(p & q);
      cnt[1] += __popc(p & q);
      if (mpq) mpq[idx] = p & q;
      continue;
    }
    if (__all_sync(0xffffffffu, (p | q) == 0)) {
      if (mpq) mpq[idx] = 0u;
      continue;
    }
    // union of the 3 x 3 rows' bits, then dilation in x once
    uint32_t uq = 0, up = 0;
#pragma unroll
    for (int dz = -1; dz <= 1; ++dz) {
      const int zz = z + dz < 0 ? nz - 1 : (z + dz >= nz ? 0 : z + dz);
#pragma unroll
      for (int dy = -1; dy <= 1; ++dy) {
        const int yy = y + dy < 0 ? ny - 1 : (y + dy >= ny ? 0 : y + dy);
        const long long rb = ((long long)zz * ny + yy) * 32;
        uq |= mq[rb + lane];
        up |= mp[rb + lane];
      }
    }
    const uint32_t lq = __shfl_sync(0xffffffffu, uq, (lane + 31) & 31), rq = __shfl_sync(0xffffffffu, uq, (lane + 1) & 31);
    const uint32_t lp = __shfl_sync(0xffffffffu, up, (lane + 31) & 31), rp = __shfl_sync(0xffffffffu, up, (lane + 1) & 31);
    const uint32_t dq = uq | (uq << 1) | (uq >> 1) | (lq >> 31) | (rq << 31);
    const uint32_t dp = up | (up << 1) | (up >> 1) | (lp >> 31) | (rp << 31);
    cnt[0] += __popc(p & dq);
    cnt[1] += __popc(q & dp);
    if (mpq) mpq[idx] = p & dq;  // the p-anchored bound-state cells
  }
  __shared__ long long sm[OVL_THREADS / 32][2];
  const int warp = threadIdx.x >> 5;
  for (int a = 0; a < 2; ++a) {
    const long long v = warp_sum_ll(cnt[a]);
    if (lane == 0) sm[warp][a] = v;
  }
  __syncthreads();
  if (threadIdx.x < 2) {
    long long v = 0;
    for (int k = 0; k < OVL_THREADS / 32; ++k) v += sm[k][threadIdx.x];
    part[blockIdx.x].pq[threadIdx.x] = v;
  }
}

// ---- finalize: fixed-order compensated merge of the block partials --------

constexpr int FIN_THREADS = 256;

__device__ __forceinline__ void merge_pair(double& s, double& c, double s2, double c2) {
  neumaier_add(s, c, s2);
  c += c2;
}

// First stage: CTA j merges the contiguous slice j of the partials into
// mid[j].  Warp w takes the quantities w, w + 8, ...; its lanes run over the
// slice with a stride of 32 and merge their results in a fixed shuffle tree.
__device__ __forceinline__ void fin_stage_body(const BlockPartial* __restrict__ part, int nb,
                                               BlockPartial* __restrict__ mid, int j, int nj) {
  const int per = (nb + nj - 1) / nj;
  const int b0 = j * per, b1 = min(nb, b0 + per);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  BlockPartial* out = mid + j;
  constexpr int NQ = NSUM + NMAX + NCNT;
  for (int q = warp; q < NQ; q += FIN_THREADS / 32) {
    if (q < NSUM) {
      double s = 0.0, c = 0.0;
      for (int b = b0 + lane; b < b1; b += 32) merge_pair(s, c, part[b].sum[q], part[b].comp[q]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const double s2 = __shfl_down_sync(0xffffffffu, s, o), c2 = __shfl_down_sync(0xffffffffu, c, o);
        merge_pair(s, c, s2, c2);
      }
      if (lane == 0) {
        out->sum[q] = s;
        out->comp[q] = c;
      }
    } else if (q < NSUM + NMAX) {
      const int k = q - NSUM;
      double m = -INFINITY;
      for (int b = b0 + lane; b < b1; b += 32) m = fmax(m, part[b].mx[k]);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_down_sync(0xffffffffu, m, o));
      if (lane == 0) out->mx[k] = m;
    } else {
      const int k = q - NSUM - NMAX;
      long long v = 0;
      for (int b = b0 + lane; b < b1; b += 32) v = (k == C_MAXW) ? max(v, part[b].cnt[k]) : v + part[b].cnt[k];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        const long long u = __shfl_down_sync(0xffffffffu, v, o);
        v = (k == C_MAXW) ? max(v, u) : v + u;
      }
      if (lane == 0) out->cnt[k] = v;
    }
  }
}

__global__ void __launch_bounds__(FIN_THREADS)
k_fin_stage(const BlockPartial* __restrict__ part, int nb, BlockPartial* __restrict__ mid) {
  fin_stage_body(part, nb, mid, blockIdx.x, gridDim.x);
}

// Second (or only) stage: one CTA merges nb partials in a fixed tree.
__device__ __forceinline__ void finalize_body(const BlockPartial* __restrict__ part, int nb,
                                              const CellPartial* __restrict__ cpart, int ncb, RawRecord* rec,
                                              long long n, int has_diag, int has_gauss, int has_strings, int tol,
                                              const unsigned long long* __restrict__ ge4) {
  __shared__ double ss[FIN_THREADS], sc[FIN_THREADS];
  __shared__ long long sl[FIN_THREADS];
  const int t = threadIdx.x;
  for (int k = 0; k < NSUM; ++k) {
    double s = 0.0, c = 0.0;
    if (part)
      for (int b = t; b < nb; b += FIN_THREADS) merge_pair(s, c, part[b].sum[k], part[b].comp[k]);
    ss[t] = s;
    sc[t] = c;
    __syncthreads();
    for (int h = FIN_THREADS / 2; h > 0; h >>= 1) {
      if (t < h) {
        double a = ss[t], ac = sc[t];
        merge_pair(a, ac, ss[t + h], sc[t + h]);
        ss[t] = a;
        sc[t] = ac;
      }
      __syncthreads();
    }
    if (t == 0) rec->sum[k] = ss[0] + sc[0];
    __syncthreads();
  }
  for (int k = 0; k < NMAX; ++k) {
    double m = -INFINITY;
    if (part)
      for (int b = t; b < nb; b += FIN_THREADS) m = fmax(m, part[b].mx[k]);
    ss[t] = m;
    __syncthreads();
    for (int h = FIN_THREADS / 2; h > 0; h >>= 1) {
      if (t < h) ss[t] = fmax(ss[t], ss[t + h]);
      __syncthreads();
    }
    if (t == 0) rec->mx[k] = ss[0];
    __syncthreads();
  }
  for (int k = 0; k < NCNT + 2; ++k) {
    long long v = 0;
    if (k < NCNT) {
      if (part)
        for (int b = t; b < nb; b += FIN_THREADS) v = (k == C_MAXW) ? max(v, part[b].cnt[k]) : v + part[b].cnt[k];
    } else if (cpart) {
      for (int b = t; b < ncb; b += FIN_THREADS) v += cpart[b].pq[k - NCNT];
    }
    sl[t] = v;
    __syncthreads();
    for (int h = FIN_THREADS / 2; h > 0; h >>= 1) {
      if (t < h) sl[t] = (k == C_MAXW) ? max(sl[t], sl[t + h]) : sl[t] + sl[t + h];
      __syncthreads();
    }
    if (t == 0) {
      if (k < NCNT) rec->cnt[k] = sl[0];
      else rec->cells[k - NCNT] = sl[0];
    }
    __syncthreads();
  }
  if (t == 0) {
    rec->cells[2] = ge4 ? (long long)ge4[0] : 0;
    rec->cells[3] = ge4 ? (long long)ge4[1] : 0;
    rec->n = n;
    rec->has_diag = has_diag;
    rec->has_gauss = has_gauss;
    rec->has_strings = has_strings;
    rec->tol = tol;
  }
}

__global__ void __launch_bounds__(FIN_THREADS)
k_finalize(const BlockPartial* __restrict__ part, int nb, const CellPartial* __restrict__ cpart, int ncb,
           RawRecord* rec, long long n, int has_diag, int has_gauss, int has_strings, int tol,
           const unsigned long long* __restrict__ ge4) {
  finalize_body(part, nb, cpart, ncb, rec, n, has_diag, has_gauss, has_strings, tol, ge4);
}

// ---- batched detection of ensemble boxes -----------------------------------
// The boxes of list[0..nlist) detect at the same run step.  Their cell values
// and overlap counts are integers, so the batched passes (bytewise cell
// values, one mask word per warp; 32 mask words per warp for the overlap,
// counts added atomically per box) give exactly the single-lattice counts.

constexpr int ENS_CELL_THREADS = 256;
constexpr int ENS_CELL_BLOCKS = 152 * 8;

__global__ void __launch_bounds__(ENS_CELL_THREADS)
k_ens_cellbits(const EnsDet* __restrict__ det, const int* __restrict__ list, const long long* __restrict__ pre,
               int nlist, long long items) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long u = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; u < items; u += nwarps) {
    const int si = ens_list_index(pre, nlist, u);
    const EnsDet& D = det[list[si]];
    const long long lu = u - pre[si];
    const int nx = D.nx, ny = D.ny, nz = D.nz, words = D.words;
    const long long V = (long long)nx * ny * nz;
    const long long nw = (long long)words * ny * nz;
    const int w = (int)(lu % words);
    const long long row = lu / words;
    const int y = (int)(row % ny), z = (int)(row / ny);
    const int x = w * 32 + lane;
    int c[2] = {0, 0};
    if (x < nx) {
      const long long i = row * nx + x;
      const long long ix = row * nx + (x + 1 == nx ? 0 : x + 1);
      const long long iy = ((long long)z * ny + (y + 1 == ny ? 0 : y + 1)) * nx + x;
      const long long iz = ((long long)(z + 1 == nz ? 0 : z + 1) * ny + y) * nx + x;
#pragma unroll
      for (int s = 0; s < 2; ++s) {
        const uint8_t* f = D.faces + s * V;
        c[s] = face_w(f, i, 0) + face_w(f, iz, 0) + face_w(f, i, 1) + face_w(f, iy, 1) + face_w(f, i, 2) +
               face_w(f, ix, 2);
      }
    }
    const uint32_t bp = __ballot_sync(0xffffffffu, c[0] > 0);
    const uint32_t bq = __ballot_sync(0xffffffffu, c[1] > 0);
    const int g0 = __popc(__ballot_sync(0xffffffffu, c[0] >= 4));
    const int g1 = __popc(__ballot_sync(0xffffffffu, c[1] >= 4));
    if (lane == 0) {
      D.masks[row * words + w] = bp;
      D.masks[nw + row * words + w] = bq;
      if (g0) atomicAdd(&D.ge4[0], (unsigned long long)g0);
      if (g1) atomicAdd(&D.ge4[1], (unsigned long long)g1);
    }
  }
}

__global__ void __launch_bounds__(ENS_CELL_THREADS)
k_ens_overlap(const EnsDet* __restrict__ det, const int* __restrict__ list, const long long* __restrict__ pre,
              int nlist, long long items) {
  const int lane = threadIdx.x & 31;
  const long long nwarps = ((long long)gridDim.x * blockDim.x) >> 5;
  for (long long u = (blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5; u < items; u += nwarps) {
    const int si = ens_list_index(pre, nlist, u);
    const EnsDet& D = det[list[si]];
    const int nx = D.nx, ny = D.ny, nz = D.nz, words = D.words;
    const long long nw = (long long)words * ny * nz;
    const uint32_t* mp = D.masks;
    const uint32_t* mq = D.masks + nw;
    const long long idx = (u - pre[si]) * 32 + lane;
    long long cp = 0, cq = 0;
    if (idx < nw) {
      const int w = (int)(idx % words);
      const long long row = idx / words;
      const int y = (int)(row % ny), z = (int)(row / ny);
      const uint32_t p = mp[idx], q = mq[idx];
      if (D.tol == 0) {
        cp = cq = __popc(p & q);
      } else if ((p | q) != 0) {
        uint32_t dq = 0, dp = 0;
        for (int dz = -1; dz <= 1; ++dz) {
          const int zz = z + dz < 0 ? nz - 1 : (z + dz >= nz ? 0 : z + dz);
          for (int dy = -1; dy <= 1; ++dy) {
            const int yy = y + dy < 0 ? ny - 1 : (y + dy >= ny ? 0 : y + dy);
            const long long rb = ((long long)zz * ny + yy) * words;
            if (p) dq |= xdilate(mq, rb, w, words, nx);
            if (q) dp |= xdilate(mp, rb, w, words, nx);
          }
        }
        cp = __popc(p & dq);
        cq = __popc(q & dp);
      }
    }
    cp = warp_sum_ll(cp);
    cq = warp_sum_ll(cq);
    if (lane == 0) {
      if (cp) atomicAdd((unsigned long long*)&D.counts->pq[0], (unsigned long long)cp);
      if (cq) atomicAdd((unsigned long long*)&D.counts->pq[1], (unsigned long long)cq);
    }
  }
}

__global__ void __launch_bounds__(FIN_THREADS)
k_ens_fin_stage(const EnsDet* __restrict__ det, const int* __restrict__ list) {
  const EnsDet& D = det[list[blockIdx.y]];
  const int nb = D.nmeas + D.nwind;
  if (nb <= FIN_STAGE_MIN) return;
  fin_stage_body(D.part, nb, D.part + nb, blockIdx.x, gridDim.x);
}

// One CTA per box: the record of run step k goes to the box's ring slot
// rec + (number of the box's detections before k in this run).
__global__ void __launch_bounds__(FIN_THREADS)
k_ens_finalize(const EnsDet* __restrict__ det, const EnsDyn* __restrict__ dyn, const int* __restrict__ list, int k,
               int de, int ring_cap) {
  const int b = list[blockIdx.x];
  const EnsDet& D = det[b];
  const int nb = D.nmeas + D.nwind;
  const bool staged = nb > FIN_STAGE_MIN;
  const long long n0 = dyn[b].n;
  const long long k1 = (de - n0 % de) % de;
  const long long slot = (dyn[b].rec + (k - k1) / de) % ring_cap;
  finalize_body(staged ? D.part + nb : D.part, staged ? FIN_STAGE_BLOCKS : nb, D.counts, 1, D.ring + slot, n0 + k,
                1, 0, 1, D.tol, D.ge4);
}

}  // namespace

int cells_grid_blocks() { return OVL_BLOCKS; }

size_t cell_mask_words(int nx, int ny, int nz) { return (size_t)((nx + 31) / 32) * ny * nz; }

cudaError_t launch_cells(const uint8_t* faces, int nx, int ny, int nz, int tol, uint8_t* cell_p, uint8_t* cell_q,
                         uint32_t* masks, CellPartial* part, cudaStream_t st, uint32_t* mpq,
                         unsigned long long* ge4) {
  const int words = (nx + 31) / 32;
  const size_t nw = cell_mask_words(nx, ny, nz);
  uint32_t* mp = masks;
  uint32_t* mq = masks + nw;
  const long long nrows = (long long)ny * nz;
  long long gy = (nrows + ROWS_PER_BLOCK - 1) / ROWS_PER_BLOCK;
  if (gy > BITS_BLOCKS_Y) gy = BITS_BLOCKS_Y;
  dim3 block(32, ROWS_PER_BLOCK), grid(words, (unsigned)gy);
  if (ge4) {
    cudaError_t e0 = cudaMemsetAsync(ge4, 0, 2 * sizeof(unsigned long long), st);
    if (e0 != cudaSuccess) return e0;
  }
  // the sixteen-cell kernel stores optional cell arrays as 16-byte chunks
  const bool al16 = ((uintptr_t)cell_p % 16 == 0) && ((uintptr_t)cell_q % 16 == 0);
  if (nx % 32 == 0 && al16)
    k_cellbits16<<<BITS4_BLOCKS, BITS4_THREADS, 0, st>>>(faces, nx, ny, nz, words, cell_p, cell_q, mp, mq, ge4);
  else
    k_cellbits<<<grid, block, 0, st>>>(faces, nx, ny, nz, words, cell_p, cell_q, mp, mq, ge4);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  if (words == 32 && nx == 1024)
    k_overlap_row32<<<OVL_BLOCKS, OVL_THREADS, 0, st>>>(mp, mq, ny, nz, tol, part, mpq);
  else
    k_overlap<<<OVL_BLOCKS, OVL_THREADS, 0, st>>>(mp, mq, nx, ny, nz, words, tol, part, mpq);
  return cudaGetLastError();
}

cudaError_t launch_ens_cells(const EnsDet* det, const int* list, const long long* pre_c, const long long* pre_o,
                             int nlist, long long items_c, long long items_o, cudaStream_t st) {
  if (items_c <= 0) return cudaSuccess;
  k_ens_cellbits<<<ENS_CELL_BLOCKS, ENS_CELL_THREADS, 0, st>>>(det, list, pre_c, nlist, items_c);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_ens_overlap<<<ENS_CELL_BLOCKS, ENS_CELL_THREADS, 0, st>>>(det, list, pre_o, nlist, items_o);
  return cudaGetLastError();
}

cudaError_t launch_ens_finalize(const EnsDet* det, const EnsDyn* dyn, const int* list, int nlist, int k, int de,
                                bool stage, cudaStream_t st) {
  if (nlist <= 0) return cudaSuccess;
  if (stage) {
    k_ens_fin_stage<<<dim3(FIN_STAGE_BLOCKS, nlist), FIN_THREADS, 0, st>>>(det, list);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  k_ens_finalize<<<nlist, FIN_THREADS, 0, st>>>(det, dyn, list, k, de, RING_CAP);
  return cudaGetLastError();
}

cudaError_t launch_finalize(BlockPartial* part, int nblocks, const CellPartial* cpart, int ncblocks,
                            RawRecord* rec, long long n, int has_diag, int has_gauss, int has_strings, int tol,
                            cudaStream_t st, const unsigned long long* ge4) {
  const BlockPartial* src = part;
  int nsrc = nblocks;
  if (part && nblocks > FIN_STAGE_MIN) {
    BlockPartial* mid = part + nblocks;
    k_fin_stage<<<FIN_STAGE_BLOCKS, FIN_THREADS, 0, st>>>(part, nblocks, mid);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    src = mid;
    nsrc = FIN_STAGE_BLOCKS;
  }
  k_finalize<<<1, FIN_THREADS, 0, st>>>(src, nsrc, cpart, ncblocks, rec, n, has_diag, has_gauss, has_strings, tol,
                                        ge4);
  return cudaGetLastError();
}

}  // namespace u1u1
