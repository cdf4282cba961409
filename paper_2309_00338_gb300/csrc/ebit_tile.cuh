// Tiled sweep kernel: one split sweep (Sec. 2.1-2.4) for a tile of the grid,
// marker-centric and bit-parallel in shared memory.
//
// Tile (sweep coordinates): vertices i in [i0, i0+64), j in [j0, j0+32) with
// their aligned edge (i,j), unaligned edge (i,j) and cell (i,j).  The region
// held in shared memory is the tile plus a halo, vertices
// [i0-4, i0+67] x [j0-2, j0+34] (72 x 37): candidate chords for line k come
// from cells k-2..k, their end markers' neighbours lie one cell further, the
// neighbours' next markers (points 1 and 4 when a neighbour is too close) one
// more, and the centre rule looks at landings on edges k-1..k+1.
//
// Colours are kept as bit rows (3 words per region row).  Marker sets,
// interface cells and new four-marker cells are word-level XORs of them, and
// all per-marker work runs from compacted lists, so a tile costs in
// proportion to the interface it holds:
//   P0 colour bits of the region (funnel shifts of the stored rows; for the y
//      sweep a warp-ballot transpose)
//   P1 marker bit sets; a tile with no marker in its region only copies its
//      colour words (P7)
//   P2 moved point of every marker (the only global reads of fractions and
//      velocities); corner flips (Fig. 5) by XOR into the new colour bits;
//      every aligned edge a marker lands on is claimed once
//   P3 landings on the claimed edges (Sec. 2.4), new aligned markers; list of
//      the interface cells whose chords can cross the tile's grid lines
//   P4 each chord of such a cell that crosses a grid line k of the tile
//      becomes a candidate of unaligned edge (k, j): references to A, B and
//      points 1-4, centre-rule verdicts; candidates are linked per edge
//   P5 circle fits (Sec. 2.2) of all candidates, one per thread, so the FP64
//      pipe sees full warps
//   P6 one marker per edge from its linked candidates; new unaligned markers
//   P7 centre colours of the new four-marker cells (Sec. 2.3); colour words
#pragma once
#include "ebit_device.cuh"

namespace ebit {

constexpr int kTI = 64, kTJ = 32;
constexpr int kRX = kTI + 8, kRY = kTJ + 5, kRN = kRX * kRY;
constexpr int kRW = 3;                 // words per region bit row (72 columns used)
constexpr int kRB = kRY * kRW;         // words per region bit plane
constexpr int kNVE = (kTI + 1) * kTJ;  // unaligned edges k in [i0, i0+64], rows j0..j0+31
constexpr int kTileThreads = 256;
constexpr int kCandCap = 256;          // candidates per tile; an edge beyond it is done in place
constexpr uint16_t kKindV = 0x8000;    // marker reference: region index | kKindV if unaligned

template <typename R> constexpr int tile_min_blocks();
template <> constexpr int tile_min_blocks<float>() { return 3; }
template <> constexpr int tile_min_blocks<double>() { return 2; }

// Candidate of one unaligned edge: chord ends A (left of the line) and B,
// point 1 (p1) with the next marker beyond it (q1) in case p1 is too close to
// A, likewise 4; references to moved markers held in the tile.
enum { CF_P1 = 1, CF_Q1 = 2, CF_P4 = 4, CF_Q4 = 8, CF_OWNED = 16 };
struct Cand {
  double y;
  uint16_t a, b, p1, q1, p4, q4;
  uint16_t edge;  // (j - j0) * (kTI + 1) + (k - i0)
  uint8_t fl, ord;
  int8_t vr, vl, kind;
};

// Shared memory of one tile (dynamic).
template <typename R>
struct TileMem {
  union {
    Cand cand[kCandCap];   // P4-P6
    uint16_t ld[kRN];      // P2-P3: claimed landing edges
  };
  R hfx[kRN];              // moved aligned marker: fraction
  R vfx[kRN];              // moved unaligned marker: fraction along the sweep
  R vfy[kRN];              // ... and across it (the marker's own fraction)
  int head[kNVE];          // first linked candidate of an unaligned edge, -1: none
  uint32_t kb[kRB];        // old corner colours
  uint32_t kn[kRB];        // new corner colours
  uint32_t zb[kRB];        // old centre colours (bit lx of row ly: cell (lx, ly))
  uint32_t hm[kRB];        // aligned markers (bit lx of row ly: edge (lx, ly))
  uint32_t vm[kRB];        // unaligned markers
  uint32_t claim[kRB];     // aligned edges some marker lands on
  uint32_t hc[kRB];        // unaligned edges with a linked candidate
  uint32_t ovf[kRB];       // unaligned edges done in place
  uint16_t lh[kRN];        // aligned marker list; in P3-P4 the interface-cell list
  uint16_t lv[kRN];        // unaligned marker list
  uint16_t le[kCandCap];   // unaligned edges with a linked candidate
  int16_t next[kCandCap];  // candidate links
  int8_t hix[kRN];         // moved aligned marker: ix - ri0
  int8_t vix[kRN];         // moved unaligned marker: ix - ri0
  int8_t lsrc[kRN];        // landing: kept source - i (kNoSrc: none)
  uint8_t vrl[kNVE];       // centre verdicts of an edge: bits 0-1 right + 1, bits 2-3 left + 1
};

template <typename R>
constexpr size_t tile_smem_bytes() {
  return sizeof(TileMem<R>);
}

__device__ __forceinline__ int getb(const uint32_t* w, int lx, int ly) {
  return (w[ly * kRW + (lx >> 5)] >> (lx & 31)) & 1;
}

// Bits [a, b] (inclusive, region columns) within word wi; empty if a > b.
__device__ __forceinline__ uint32_t span_mask(int wi, int a, int b) {
  const int lo = max(a - 32 * wi, 0), hi = min(b - 32 * wi, 31);
  if (lo > hi) return 0u;
  const uint32_t up = hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u);
  return up & ~((1u << lo) - 1u);
}

// Word wi of row ly shifted right by one column (bit b = column 32 wi + b + 1).
__device__ __forceinline__ uint32_t shr1(const uint32_t* w, int ly, int wi) {
  uint32_t v = w[ly * kRW + wi] >> 1;
  if (wi + 1 < kRW) v |= w[ly * kRW + wi + 1] << 31;
  return v;
}

// Bits x0 .. x0+31 of a stored row of nw words (bits outside the row read 0).
__device__ __forceinline__ uint32_t row_bits(const uint32_t* __restrict__ row, int nw, int x0) {
  const int q = x0 >> 5, r = x0 & 31;
  const uint32_t a = (q >= 0 && q < nw) ? __ldg(&row[q]) : 0u;
  const uint32_t b = (q + 1 >= 0 && q + 1 < nw) ? __ldg(&row[q + 1]) : 0u;
  return r ? ((a >> r) | (b << (32 - r))) : a;
}

// Appends the set bits of plane word t as region indices.
__device__ __forceinline__ void push_bits(uint32_t bits, int t, uint16_t* list, int* count) {
  if (!bits) return;
  int base = atomicAdd(count, __popc(bits));
  const int row0 = (t / kRW) * kRX + 32 * (t % kRW);
  while (bits) {
    const int b = __ffs(bits) - 1;
    bits &= bits - 1;
    list[base++] = (uint16_t)(row0 + b);
  }
}

__device__ __forceinline__ int verdict_r(uint8_t c) { return (int)(c & 3) - 1; }
__device__ __forceinline__ int verdict_l(uint8_t c) { return (int)((c >> 2) & 3) - 1; }
__device__ __forceinline__ uint8_t verdicts(int vr, int vl) {
  return (uint8_t)((vr + 1) | ((vl + 1) << 2));
}

// Accessor of the tile for the shared sweep logic (beyond, walk,
// new_unaligned).  Indices are clamped into the region; the kernel only asks
// inside it.
template <typename R>
struct TViewB {
  const TileMem<R>* m;
  int ri0, rj0, nx_, ny_;
  __device__ __forceinline__ int tnx() const { return nx_; }
  __device__ __forceinline__ int tny() const { return ny_; }
  __device__ __forceinline__ int cx(int i) const {
    return (int)min((unsigned)(i - ri0), (unsigned)(kRX - 1));
  }
  __device__ __forceinline__ int cy(int j) const {
    return (int)min((unsigned)(j - rj0), (unsigned)(kRY - 1));
  }
  __device__ __forceinline__ int k(int i, int j) const { return getb(m->kb, cx(i), cy(j)); }
  __device__ __forceinline__ int z(int i, int j) const { return getb(m->zb, cx(i), cy(j)); }
  __device__ __forceinline__ int knew(int i, int j) const { return getb(m->kn, cx(i), cy(j)); }
  __device__ __forceinline__ uint16_t ref(Mk mk) const {
    return (uint16_t)((cy(mk.j) * kRX + cx(mk.i)) | (mk.kind ? kKindV : 0));
  }
  __device__ __forceinline__ AP<R> moved(Mk mk) const {
    const int t = cy(mk.j) * kRX + cx(mk.i);
    AP<R> p;
    p.jy = mk.j;
    if (mk.kind == 0) {
      p.ix = m->hix[t] + ri0;
      p.fx = m->hfx[t];
      p.fy = R(0);
    } else {
      p.ix = m->vix[t] + ri0;
      p.fx = m->vfx[t];
      p.fy = m->vfy[t];
    }
    return p;
  }
  __device__ __forceinline__ Landing<R> landing(int i, int j) const {
    const int s = m->lsrc[cy(j) * kRX + cx(i)];
    Landing<R> L;
    L.present = knew(i, j) ^ knew(i + 1, j);
    L.kept_src = s == kNoSrc ? -1 : i + s;
    L.kept_fx = R(0);
    L.cancelled = 0;
    L.invariant = 0;
    return L;
  }
  // Moved point of a referenced marker relative to vertex (k, j).
  __device__ __forceinline__ void xy(uint16_t r, int k, int j, double* X, double* Y) const {
    const int t = r & (kKindV - 1), ly = t / kRX;
    if (r & kKindV) {
      *X = (double)(m->vix[t] + ri0 - k) + (double)m->vfx[t];
      *Y = (double)(rj0 + ly - j) + (double)m->vfy[t];
    } else {
      *X = (double)(m->hix[t] + ri0 - k) + (double)m->hfx[t];
      *Y = (double)(rj0 + ly - j) + 0.0;
    }
  }
};

// The tile with origin (i0, j0) of one grid (one block runs it).
template <typename R, int AX>
__device__ __forceinline__ void sweep_tile(const GView<R, AX>& G, const Buf<R>& out, int line_only,
                                           unsigned long long* ctr, unsigned long long* cfl_bits,
                                           int* status, const int i0, const int j0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileMem<R>& M = *reinterpret_cast<TileMem<R>*>(smem_raw);
  __shared__ int s_nh, s_nv, s_nd, s_nc, s_ncand, s_ne;
  __shared__ int s_cnt[D_NUSED];
  __shared__ unsigned long long s_dmax;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kWarps = kTileThreads / 32;
  const int tnx = G.tnx(), tny = G.tny();
  const int ri0 = i0 - 4, rj0 = j0 - 2;
  const long long P = G.d.P;
  if (tid < D_NUSED) s_cnt[tid] = 0;
  if (tid == 0) {
    s_nh = s_nv = s_nd = s_nc = s_ncand = s_ne = 0;
    s_dmax = 0ull;
  }
  int cnt[D_NUSED];
#pragma unroll
  for (int c = 0; c < D_NUSED; ++c) cnt[c] = 0;
  R dmax = R(0);
  auto owned = [&](int x, int y) { return x >= i0 && x < i0 + kTI && y >= j0 && y < j0 + kTJ; };
  // region columns / rows inside the grid
  const int vx0 = max(0, -ri0), vx1 = min(kRX - 1, tnx - ri0);  // vertices
  const int ex1 = min(kRX - 2, tnx - 1 - ri0);                   // aligned edges, cells
  const int vy0 = max(0, -rj0), vy1 = min(kRY - 1, tny - rj0);  // vertex rows
  const int ey1 = min(kRY - 2, tny - 1 - rj0);                   // unaligned edges, cells
  const int ty1 = min(kTJ + 1, ey1);                              // last cell row of the tile

  // P0: colour bits of the region
  if (AX == 0) {
    for (int t = tid; t < 2 * kRB; t += kTileThreads) {
      const int zpl = t >= kRB, u = zpl ? t - kRB : t;
      const int ly = u / kRW, wi = u % kRW;
      const int y = rj0 + ly, x0 = ri0 + 32 * wi;
      uint32_t v = 0u;
      if (!zpl && ly >= vy0 && ly <= vy1)
        v = row_bits(G.K + (long long)y * G.d.kw, G.d.kw, x0) & span_mask(wi, vx0, vx1);
      if (zpl && ly >= vy0 && ly <= ey1)
        v = row_bits(G.Z + (long long)y * G.d.zw, G.d.zw, x0) & span_mask(wi, vx0, ex1);
      (zpl ? M.zb : M.kb)[u] = v;
    }
  } else {
    // region column lx is stored row ri0 + lx and region row ly stored
    // column rj0 + ly: a warp reads 32 stored rows and transposes by ballots
    const int c0 = rj0 >> 5;  // first stored word of the region's rows
    for (int g = warp; g < 2 * kRW; g += kWarps) {
      const int zpl = g >= kRW, gw = zpl ? g - kRW : g;
      const int lx = 32 * gw + lane, yr = ri0 + lx;
      const uint32_t* base = zpl ? G.Z : G.K;
      const int nw = zpl ? G.d.zw : G.d.kw;
      const bool col_ok = lx >= vx0 && lx <= (zpl ? ex1 : vx1);
      const int row1 = zpl ? ey1 : vy1;
      uint32_t w0 = 0u, w1 = 0u, w2 = 0u;
      if (col_ok) {
        const uint32_t* r = base + (long long)yr * nw;
        if (c0 >= 0 && c0 < nw) w0 = __ldg(&r[c0]);
        if (c0 + 1 >= 0 && c0 + 1 < nw) w1 = __ldg(&r[c0 + 1]);
        if (c0 + 2 >= 0 && c0 + 2 < nw) w2 = __ldg(&r[c0 + 2]);
      }
      uint32_t* dst = zpl ? M.zb : M.kb;
      for (int ly = 0; ly < kRY; ++ly) {
        const int xr = rj0 + ly;
        const int q = (xr >> 5) - c0, b = xr & 31;
        const uint32_t wq = q == 0 ? w0 : (q == 1 ? w1 : w2);
        const int bit = (ly >= vy0 && ly <= row1) ? (int)((wq >> b) & 1u) : 0;
        const uint32_t word = __ballot_sync(0xffffffffu, bit);
        if (lane == 0) dst[ly * kRW + gw] = word;
      }
    }
  }
  __syncthreads();

  // P1: marker sets
  int mine = 0;
  for (int t = tid; t < kRB; t += kTileThreads) {
    const int ly = t / kRW, wi = t % kRW;
    uint32_t h = 0u, v = 0u;
    if (ly >= vy0 && ly <= vy1) h = (M.kb[t] ^ shr1(M.kb, ly, wi)) & span_mask(wi, vx0, ex1);
    if (ly >= vy0 && ly <= ey1) v = (M.kb[t] ^ M.kb[t + kRW]) & span_mask(wi, vx0, vx1);
    M.hm[t] = h;
    M.vm[t] = v;
    M.kn[t] = M.kb[t];
    M.claim[t] = 0u;
    M.hc[t] = 0u;
    M.ovf[t] = 0u;
    mine |= (h | v) != 0u;
  }
  const bool busy = __syncthreads_or(mine) != 0;
  const TViewB<R> TV{&M, ri0, rj0, tnx, tny};

  if (busy) {
    for (int t = tid; t < kRB; t += kTileThreads) {
      push_bits(M.hm[t], t, M.lh, &s_nh);
      push_bits(M.vm[t], t, M.lv, &s_nv);
    }
    for (int e = tid; e < kNVE; e += kTileThreads) {
      M.head[e] = -1;
      M.vrl[e] = 0;
    }
    __syncthreads();

    // P2: moved points, corner flips, landing claims
    const int nh = s_nh, nv = s_nv;
    for (int w = tid; w < nh; w += kTileThreads) {
      const int id = M.lh[w], lx = id % kRX, ly = id / kRX;
      const int x = ri0 + lx, y = rj0 + ly;
      Flags f;
      const AP<R> p = G.advect(Mk{0, x, y}, f);
      M.hix[id] = (int8_t)(p.ix - ri0);
      M.hfx[id] = p.fx;
      if (owned(x, y)) {
        cnt[D_CFL] += f.cfl;
        cnt[D_WALL_CLAMP] += f.clamp;
        dmax = fmax(dmax, dabs_of<R>(f));
      }
      // a marker moving right passes vertex x+1, one moving left vertex x
      if (p.ix == x + 1) atomicXor(&M.kn[ly * kRW + ((lx + 1) >> 5)], 1u << ((lx + 1) & 31));
      else if (p.ix == x - 1) atomicXor(&M.kn[ly * kRW + (lx >> 5)], 1u << (lx & 31));
      const int dl = p.ix - ri0;
      if (dl >= 1 && dl <= kRX - 3) {
        const uint32_t bit = 1u << (dl & 31);
        if (!(atomicOr(&M.claim[ly * kRW + (dl >> 5)], bit) & bit))
          M.ld[atomicAdd(&s_nd, 1)] = (uint16_t)(ly * kRX + dl);
      }
    }
    for (int w = tid; w < nv; w += kTileThreads) {
      const int id = M.lv[w], lx = id % kRX, ly = id / kRX;
      const int x = ri0 + lx, y = rj0 + ly;
      Flags f;
      const AP<R> p = G.advect(Mk{1, x, y}, f);
      M.vix[id] = (int8_t)(p.ix - ri0);
      M.vfx[id] = p.fx;
      M.vfy[id] = p.fy;
      if (owned(x, y)) {
        if (x >= 1 && x <= tnx - 1) {
          cnt[D_CFL] += f.cfl;
          dmax = fmax(dmax, dabs_of<R>(f));
        } else {  // a wall marker normal to the sweep stays
          if (AX) out.sH[(long long)x * P + y] = p.fy;
          else out.sV[(long long)y * P + x] = p.fy;
        }
      }
    }
    __syncthreads();

    // P3: landings on the claimed aligned edges
    const int nd = s_nd;
    for (int w = tid; w < nd; w += kTileThreads) {
      const int id = M.ld[w], dl = id % kRX, ly = id / kRX;
      const int x = ri0 + dl, y = rj0 + ly;
      R fx[3];
      int src[3];
      int n = 0;
      for (int e = dl - 1; e <= dl + 1; ++e) {
        if (!getb(M.hm, e, ly)) continue;
        const int ie = ly * kRX + e;
        if (M.hix[ie] == dl) {
          fx[n] = M.hfx[ie];
          src[n] = ri0 + e;
          ++n;
        }
      }
      const Landing<R> L = choose_landing(n, fx, src, getb(M.kn, dl, ly) ^ getb(M.kn, dl + 1, ly));
      M.lsrc[id] = L.kept_src < 0 ? kNoSrc : (int8_t)(L.kept_src - x);
      if (owned(x, y)) {
        cnt[D_CANCELLED] += L.cancelled;
        cnt[D_INVARIANT] += L.invariant;
        if (L.present) {
          if (AX) out.sV[(long long)x * P + y] = L.kept_fx;
          else out.sH[(long long)y * P + x] = L.kept_fx;
        }
      }
    }
    for (int t = tid; t < kTJ * kRW; t += kTileThreads) {
      const int ly = 2 + t / kRW, wi = t % kRW, u = ly * kRW + wi;
      // owned aligned edges that gain a marker none landed on (the colour
      // bookkeeping excludes it): counted, fraction 0.5
      if (ly <= vy1) {
        uint32_t bad = (M.kn[u] ^ shr1(M.kn, ly, wi)) & ~M.claim[u] &
                       span_mask(wi, 4, min(kTI + 3, ex1));
        while (bad) {
          const int b = __ffs(bad) - 1;
          bad &= bad - 1;
          const int x = ri0 + 32 * wi + b, y = rj0 + ly;
          cnt[D_INVARIANT] += 1;
          if (AX) out.sV[(long long)x * P + y] = R(0.5);
          else out.sH[(long long)y * P + x] = R(0.5);
        }
      }
      // interface cells (corner colours not all equal) whose chords can
      // cross a grid line k in [i0, i0+64]: cells k-2..k
      if (ly <= ty1) {
        const uint32_t a = M.kb[u], b = M.kb[u + kRW];
        const uint32_t ic = ((a ^ shr1(M.kb, ly, wi)) | (b ^ shr1(M.kb, ly + 1, wi)) | (a ^ b)) &
                            span_mask(wi, max(2, vx0), min(kTI + 4, ex1));
        push_bits(ic, u, M.lh, &s_nc);
      }
    }
    __syncthreads();

    // P4: candidates
    const int nc = s_nc;
    const int kmin = max(1, i0), kmax = min(tnx - 1, i0 + kTI);
    for (int w = tid; w < nc; w += kTileThreads) {
      const int id = M.lh[w], lx = id % kRX, ly = id / kRX;
      const int c = ri0 + lx, j = rj0 + ly;
      int seg[2][2];
      const int ns = cell_segments(TV, c, j, seg);
      for (int t = 0; t < ns; ++t) {
        const Mk ma = edge_marker(c, j, seg[t][0]);
        const Mk mb = edge_marker(c, j, seg[t][1]);
        const int ia = TV.moved(ma).ix, ib = TV.moved(mb).ix;
        const int klo = max(min(ia, ib) + 1, kmin), khi = min(max(ia, ib), kmax);
        for (int k = klo; k <= khi; ++k) {
          const int e = (j - j0) * (kTI + 1) + (k - i0);
          const int ex = k - ri0, eu = ly * kRW + (ex >> 5);
          const uint32_t ebit = 1u << (ex & 31);
          const int slot = atomicAdd(&s_ncand, 1);
          if (slot >= kCandCap) {
            atomicOr(&M.ovf[eu], ebit);
            continue;
          }
          const bool a_left = ia < k;
          const Mk mA = a_left ? ma : mb, mB = a_left ? mb : ma;
          Cand& C = M.cand[slot];
          C.a = TV.ref(mA);
          C.b = TV.ref(mB);
          uint8_t fl = k < i0 + kTI ? CF_OWNED : 0;
          int c1i = 0, c1j = 0, c4i = 0, c4j = 0;
          const Mk n1 = beyond(TV, mA, c, j, &c1i, &c1j);
          const Mk n4 = beyond(TV, mB, c, j, &c4i, &c4j);
          if (n1.kind >= 0) {
            C.p1 = TV.ref(n1);
            fl |= CF_P1;
            int oi, oj;
            const Mk nn = beyond(TV, n1, c1i, c1j, &oi, &oj);
            if (nn.kind >= 0) {
              C.q1 = TV.ref(nn);
              fl |= CF_Q1;
            }
          }
          if (n4.kind >= 0) {
            C.p4 = TV.ref(n4);
            fl |= CF_P4;
            int oi, oj;
            const Mk nn = beyond(TV, n4, c4i, c4j, &oi, &oj);
            if (nn.kind >= 0) {
              C.q4 = TV.ref(nn);
              fl |= CF_Q4;
            }
          }
          C.fl = fl;
          C.edge = (uint16_t)e;
          C.ord = (uint8_t)((c - (k - 2)) * 2 + t);
          const int lr = walk(TV, mB, n4, k);
          const int ll = walk(TV, mA, n1, k - 1);
          C.vr = (int8_t)(lr < 0 ? -1 : !TV.knew(k, lr));
          C.vl = (int8_t)(ll < 0 ? -1 : !TV.knew(k, ll));
          M.next[slot] = (int16_t)atomicExch(&M.head[e], slot);
          if (!(atomicOr(&M.hc[eu], ebit) & ebit)) M.le[atomicAdd(&s_ne, 1)] = (uint16_t)e;
        }
      }
    }
    __syncthreads();

    // P5: circle fits, one candidate per thread
    const int ncand = min(s_ncand, kCandCap);
    for (int ci = tid; ci < ncand; ci += kTileThreads) {
      Cand& C = M.cand[ci];
      const int k = i0 + C.edge % (kTI + 1), j = j0 + C.edge / (kTI + 1);
      if (getb(M.ovf, k - ri0, j - rj0)) continue;  // the edge is done in place
      double ax, ay, bx, by, p1x = 0.0, p1y = 0.0, p4x = 0.0, p4y = 0.0;
      TV.xy(C.a, k, j, &ax, &ay);
      TV.xy(C.b, k, j, &bx, &by);
      bool h1 = false, h4 = false;
      if (C.fl & CF_P1) {
        TV.xy(C.p1, k, j, &p1x, &p1y);
        h1 = true;
        const double ex = p1x - ax, ey = p1y - ay;
        if (ex * ex + ey * ey < kMinSep2) {
          if (C.fl & CF_Q1) TV.xy(C.q1, k, j, &p1x, &p1y);
          else h1 = false;
        }
      }
      if (C.fl & CF_P4) {
        TV.xy(C.p4, k, j, &p4x, &p4y);
        h4 = true;
        const double ex = p4x - bx, ey = p4y - by;
        if (ex * ex + ey * ey < kMinSep2) {
          if (C.fl & CF_Q4) TV.xy(C.q4, k, j, &p4x, &p4y);
          else h4 = false;
        }
      }
      double y;
      const int kind = fit_crossing(ax, ay, bx, by, h1, p1x, p1y, h4, p4x, p4y, line_only != 0, &y);
      C.y = y;
      C.kind = (int8_t)kind;
      if (C.fl & CF_OWNED) {  // static indices keep the counters in registers
        cnt[D_FIT_ONLINE] += kind == D_FIT_ONLINE;
        cnt[D_FIT_LINE] += kind == D_FIT_LINE;
        cnt[D_FIT_ONE] += kind == D_FIT_ONE;
        cnt[D_FIT_TWO] += kind == D_FIT_TWO;
      }
    }
    __syncthreads();

    // P6: one marker per unaligned edge (Sec. 2.4)
    const int ne = s_ne;
    for (int w = tid; w < ne; w += kTileThreads) {
      const int e = M.le[w];
      const int k = i0 + e % (kTI + 1), j = j0 + e / (kTI + 1);
      const int ex = k - ri0, ey = j - rj0;
      if (getb(M.ovf, ex, ey)) continue;
      double cy[6];
      int cvr[6], cvl[6], ord[6];
      int n = 0;
      for (int s = M.head[e]; s >= 0 && n < 6; s = M.next[s]) {
        cy[n] = M.cand[s].y;
        cvr[n] = M.cand[s].vr;
        cvl[n] = M.cand[s].vl;
        ord[n] = M.cand[s].ord;
        ++n;
      }
      const bool own = k < i0 + kTI;
      const int present = getb(M.kn, ex, ey) ^ getb(M.kn, ex, ey + 1);
      const NewV<R> nv = select_candidates<R>(n, cy, cvr, cvl, ord, present);
      if (own) {
        cnt[D_CANCELLED] += nv.cancelled;
        cnt[D_INVARIANT] += nv.invariant;
      }
      M.vrl[e] = verdicts(nv.vr, nv.vl);
      if (own && nv.present) {
        if (AX) out.sH[(long long)k * P + j] = nv.s;
        else out.sV[(long long)j * P + k] = nv.s;
      }
    }
    for (int t = tid; t < kTJ * kRW; t += kTileThreads) {
      const int ly = 2 + t / kRW, wi = t % kRW, u = ly * kRW + wi;
      if (ly > ty1) continue;
      // edges whose candidates did not fit in the tile's list: in place
      uint32_t o = M.ovf[u];
      while (o) {
        const int b = __ffs(o) - 1;
        o &= o - 1;
        const int k = ri0 + 32 * wi + b, j = rj0 + ly;
        const int e = (j - j0) * (kTI + 1) + (k - i0);
        const bool own = k < i0 + kTI;
        int oc[D_NUSED];
#pragma unroll
        for (int c = 0; c < D_NUSED; ++c) oc[c] = 0;
        const NewV<R> nv = new_unaligned<R>(TV, line_only != 0, k, j, own ? oc : nullptr);
#pragma unroll
        for (int c = 0; c < D_NUSED; ++c) cnt[c] += oc[c];
        M.vrl[e] = verdicts(nv.vr, nv.vl);
        if (own && nv.present) {
          if (AX) out.sH[(long long)k * P + j] = nv.s;
          else out.sV[(long long)j * P + k] = nv.s;
        }
      }
      // owned interior edges that gain a marker without a candidate: counted,
      // fraction 0.5
      uint32_t miss = (M.kn[u] ^ M.kn[u + kRW]) & ~M.hc[u] & ~M.ovf[u] &
                      span_mask(wi, max(4, 1 - ri0), min(kTI + 3, tnx - 1 - ri0));
      while (miss) {
        const int b = __ffs(miss) - 1;
        miss &= miss - 1;
        const int k = ri0 + 32 * wi + b, j = rj0 + ly;
        cnt[D_INVARIANT] += 1;
        if (AX) out.sH[(long long)k * P + j] = R(0.5);
        else out.sV[(long long)j * P + k] = R(0.5);
      }
    }
    __syncthreads();
  }

  // P7: colour words (one warp per word, one lane per bit)
  for (int w = warp; w < 64; w += kWarps) {
    // sweep coordinates of this lane's vertex / cell, and the stored word
    int i, j, row, word;
    if (AX) {
      i = i0 + w;
      j = j0 + lane;
      row = i;
      word = j0 >> 5;
    } else {
      i = i0 + 32 * (w & 1) + lane;
      j = j0 + (w >> 1);
      row = j;
      word = (i0 >> 5) + (w & 1);
    }
    const int lx = i - ri0, ly = j - rj0;
    const bool vin = i <= tnx && j <= tny;
    const unsigned kw = __ballot_sync(0xffffffffu, vin && getb(M.kn, lx, ly));
    if (lane == 0 && row <= G.d.ny && word < G.d.kw) out.K[(long long)row * G.d.kw + word] = kw;
    int zc = 0;
    const bool cin = i < tnx && j < tny;
    if (cin) {
      zc = getb(M.zb, lx, ly);
      if (busy) {
        const int q = getb(M.kn, lx, ly) | (getb(M.kn, lx + 1, ly) << 1) |
                      (getb(M.kn, lx + 1, ly + 1) << 2) | (getb(M.kn, lx, ly + 1) << 3);
        if (q == 5 || q == 10) {
          const int e = (j - j0) * (kTI + 1) + (i - i0);
          const int a = (i >= 1) ? verdict_r(M.vrl[e]) : -1;
          const int b = (i + 1 <= tnx - 1) ? verdict_l(M.vrl[e + 1]) : -1;
          if (a >= 0) {
            zc = a;
            cnt[D_ZSET] += 1;
            if (b >= 0 && b != a) cnt[D_ZCONFLICT] += 1;
          } else if (b >= 0) {
            zc = b;
            cnt[D_ZSET] += 1;
          }
        }
      }
    }
    const unsigned zw = __ballot_sync(0xffffffffu, cin && zc);
    if (lane == 0 && row < G.d.ny && word < G.d.zw) out.Z[(long long)row * G.d.zw + word] = zw;
  }

  // block-level counters
#pragma unroll
  for (int c = 0; c < D_NUSED; ++c) {
    const int s = __reduce_add_sync(0xffffffffu, cnt[c]);
    if (s != 0 && lane == 0) atomicAdd(&s_cnt[c], s);
  }
  if (dmax > R(0)) atomicMax(&s_dmax, (unsigned long long)__double_as_longlong((double)dmax));
  __syncthreads();
  if (tid < D_NUSED && s_cnt[tid] != 0) atomicAdd(&ctr[tid], (unsigned long long)s_cnt[tid]);
  if (tid == 0) {
    if (s_dmax) atomicMax(cfl_bits, s_dmax);
    if (s_cnt[D_CFL]) atomicOr(status, ST_CFL);
    if (s_cnt[D_INVARIANT]) atomicOr(status, ST_INVARIANT);
  }
}

// One grid: block (bx, by) runs the tile at (64 bx, 32 by).
template <typename R, int AX>
__global__ void __launch_bounds__(kTileThreads, tile_min_blocks<R>())
k_sweep_tile(GView<R, AX> G, Buf<R> out, int line_only, unsigned long long* ctr,
             unsigned long long* cfl_bits, int* status) {
  sweep_tile<R, AX>(G, out, line_only, ctr, cfl_bits, status, blockIdx.x * kTI, blockIdx.y * kTJ);
}

// Many grids in one launch: per-grid sweep descriptors and a list of work
// items (grid, tile); a grid whose descriptor is inactive for this launch
// (its split order puts the other direction first this step) is skipped.
template <typename R, int AX>
struct SweepDesc {
  GView<R, AX> G;
  Buf<R> out;
  unsigned long long* ctr;
  unsigned long long* cfl_bits;
  int* status;
  int line_only;
  int active;
};

struct WorkItem {
  int grid, tx, ty;
};

template <typename R, int AX>
__global__ void __launch_bounds__(kTileThreads, tile_min_blocks<R>())
k_sweep_tile_batch(const SweepDesc<R, AX>* __restrict__ descs, const WorkItem* __restrict__ items) {
  const WorkItem it = items[blockIdx.x];
  const SweepDesc<R, AX>& D = descs[it.grid];
  if (!D.active) return;
  sweep_tile<R, AX>(D.G, D.out, D.line_only, D.ctr, D.cfl_bits, D.status, it.tx * kTI, it.ty * kTJ);
}

}  // namespace ebit
