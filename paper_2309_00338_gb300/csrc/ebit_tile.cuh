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
constexpr int kCandCap = 255;          // candidates per tile of the one-grid kernels (an
                                       // edge beyond it is done in place)
// A candidate list of CAP entries links them through heads of 8 bits (CAP
// <= 255) or 16 bits; the all-ones head marks an edge without a candidate.
template <int CAP> __host__ __device__ constexpr int head_bits() { return CAP <= 255 ? 8 : 16; }
template <int CAP> __host__ __device__ constexpr uint32_t head_none() {
  return (1u << head_bits<CAP>()) - 1u;
}
constexpr uint16_t kKindV = 0x8000;    // marker reference: region index | kKindV if unaligned

// Block shape: 7 warps per tile; tiles resident per SM as shared memory
// allows (4 in the FP32 form, 3 in the FP64 form).
template <typename R> __host__ __device__ constexpr int tile_threads() { return 224; }
template <typename R> __host__ __device__ constexpr int tile_min_blocks();
template <> __host__ __device__ constexpr int tile_min_blocks<float>() { return 4; }
template <> __host__ __device__ constexpr int tile_min_blocks<double>() { return 3; }
// Candidates per tile of the batched kernels: many small grids of uneven
// sizes hold more interface per tile than one large grid, and the longer
// list (16-bit heads) still leaves 4 (FP32) / 3 (FP64) tiles per SM.
template <typename R> __host__ __device__ constexpr int batch_cand_cap() {
  return sizeof(R) == 4 ? 511 : 383;
}

// Candidate of one unaligned edge: chord ends A (left of the line) and B,
// points 1 (p1) and 4 (p4); references to moved markers held in the tile.
// The marker beyond point 1 (or 4), used where that point is too close to A
// (B), and the centre-rule verdicts, used where the edge borders a new
// four-marker cell, are rare: they are formed from these references when
// needed (the chord's cell is k - 2 + ord / 2 of row j).
enum { CF_P1 = 1, CF_P4 = 4, CF_OWNED = 16 };
struct Cand {
  double y;
  float sf;  // the crossing as an FP32 marker fraction (FP32 state only)
  uint16_t a, b, p1, p4;
  uint16_t edge;  // (j - j0) * (kTI + 1) + (k - i0)
  uint8_t fl, ord;
  int8_t kind;
};

// Shared memory of one tile (dynamic).  Arrays whose phases do not overlap
// share storage: the marker lists of P1-P3 with the candidates of P4-P6, the
// aligned / unaligned marker bit sets of P1-P3 with the candidate bit sets of
// P4-P6, and the interface-cell list of P3-P4 with the verdicts of P6-P7.
template <typename R, int CAP = kCandCap>
struct TileMem {
  static_assert(CAP <= 65534, "candidate slots fit the 16-bit heads");
  static constexpr int kCap = CAP;
  union {
    struct {
      uint16_t ld[kRN];        // P2-P3: claimed landing edges
      uint16_t lv[kRN];        // P1-P2: unaligned marker list
    } p;
    struct {
      Cand cand[CAP];          // P4-P6
      int16_t next[CAP];       // candidate links
      uint16_t le[CAP];        // P5-P6: unaligned edges with a linked candidate
    } c;
  } u;
  R hfx[kRN];              // moved aligned marker: fraction
  R vfx[kRN];              // moved unaligned marker: fraction along the sweep (the one
                           // across it is the marker's own, read from the state)
  alignas(16) uint32_t head[kNVE * head_bits<CAP>() / 32];  // first linked candidate of
                                                            // unaligned edges
                                        // 4m .. 4m+3 (8 bits each, 0xff: none)
  uint32_t kb[kRB];        // old corner colours
  uint32_t kn[kRB];        // new corner colours
  uint32_t zb[kRB];        // old centre colours (bit lx of row ly: cell (lx, ly))
  union {
    uint32_t hm[kRB];      // P1-P3: aligned markers (bit lx of row ly: edge (lx, ly))
    uint32_t hc[kRB];      // P4-P6: unaligned edges with a linked candidate
  };
  union {
    uint32_t vm[kRB];      // P1-P3: unaligned markers
    uint32_t ovf[kRB];     // P4-P6: unaligned edges done in place
  };
  uint32_t claim[kRB];     // aligned edges some marker lands on
  // 2-bit codes (planes 0 and 1): moved aligned / unaligned marker ix - x + 1,
  // landing kept source - i + 2 (0: none)
  uint32_t hq[2][kRB];
  uint32_t vq[2][kRB];
  uint32_t lq[2][kRB];
  union {
    uint16_t lh[kRN];      // P1-P2 aligned marker list; P3-P4 the interface-cell list
    alignas(16) uint8_t vrl[kNVE];  // P5-P7: centre verdicts of an edge: bits 0-1
                                    // right + 1, bits 2-3 left + 1
  };
};

template <typename R, int CAP = kCandCap>
constexpr size_t tile_smem_bytes() {
  return sizeof(TileMem<R, CAP>);
}

__device__ __forceinline__ int getb(const uint32_t* w, int lx, int ly) {
  return (w[ly * kRW + (lx >> 5)] >> (lx & 31)) & 1;
}

// 2-bit code of region entry (lx, ly) held in two bit planes.
__device__ __forceinline__ int get2(const uint32_t (&q)[2][kRB], int lx, int ly) {
  const int w = ly * kRW + (lx >> 5), b = lx & 31;
  return ((q[0][w] >> b) & 1) | (((q[1][w] >> b) & 1) << 1);
}
__device__ __forceinline__ void put2(uint32_t (&q)[2][kRB], int lx, int ly, int code) {
  const int w = ly * kRW + (lx >> 5);
  const uint32_t bit = 1u << (lx & 31);
  if (code & 1) atomicOr(&q[0][w], bit);
  if (code & 2) atomicOr(&q[1][w], bit);
}

// Word wi of row ly shifted right by one column (bit b = column 32 wi + b + 1).
__device__ __forceinline__ uint32_t shr1(const uint32_t* w, int ly, int wi) {
  uint32_t v = w[ly * kRW + wi] >> 1;
  if (wi + 1 < kRW) v |= w[ly * kRW + wi + 1] << 31;
  return v;
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

constexpr unsigned kFull = 0xffffffffu;

// Exclusive offset of this lane's n in a block-shared list counter; one
// shared atomic per warp.  All 32 lanes call it.
__device__ __forceinline__ int warp_alloc(int n, int* count, int lane) {
  int incl = n;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int v = __shfl_up_sync(kFull, incl, o);
    if (lane >= o) incl += v;
  }
  const int total = __shfl_sync(kFull, incl, 31);
  int base = 0;
  if (lane == 31 && total) base = atomicAdd(count, total);
  return __shfl_sync(kFull, base, 31) + incl - n;
}

// Adds the lanes' v to the block's counter c, one shared atomic per warp (all
// 32 lanes call it).  Counts are kept per phase so that no counter stays live
// in registers across the kernel.
__device__ __forceinline__ void flush_count(int* s_cnt, int c, int v, int lane) {
  const int s = __reduce_add_sync(kFull, v);
  if (s != 0 && lane == 0) atomicAdd(&s_cnt[c], s);
}

// push_bits for a whole warp (all 32 lanes call it).
__device__ __forceinline__ void push_bits_warp(uint32_t bits, int t, uint16_t* list, int* count,
                                               int lane) {
  int base = warp_alloc(__popc(bits), count, lane);
  const int row0 = (t / kRW) * kRX + 32 * (t % kRW);
  while (bits) {
    const int b = __ffs(bits) - 1;
    bits &= bits - 1;
    list[base++] = (uint16_t)(row0 + b);
  }
}

// 32 x 32 bit transpose across a warp: lane r holds row r (bit c = element
// (r, c)); returns column `lane` (bit r = element (r, lane)).
__device__ __forceinline__ uint32_t transpose32(uint32_t x, int lane) {
#pragma unroll
  for (int q = 0; q < 5; ++q) {
    const int s = 16 >> q;
    const uint32_t m = q == 0 ? 0x0000ffffu : q == 1 ? 0x00ff00ffu : q == 2 ? 0x0f0f0f0fu
                     : q == 3 ? 0x33333333u : 0x55555555u;
    const uint32_t y = __shfl_xor_sync(kFull, x, s);
    x = (lane & s) ? ((x & ~m) | ((y & ~m) >> s)) : ((x & m) | ((y & m) << s));
  }
  return x;
}

// Bits c0 .. c0+31 of region row ly (c0 + 32 < 32 kRW).
__device__ __forceinline__ uint32_t bits32(const uint32_t* w, int ly, int c0) {
  const int q = c0 >> 5, r = c0 & 31;
  const uint32_t a = w[ly * kRW + q];
  return r ? ((a >> r) | (w[ly * kRW + q + 1] << (32 - r))) : a;
}

// Bits b of a 32-column window starting at column c0 with c0 + b <= last.
__device__ __forceinline__ uint32_t upto32(int c0, int last) {
  const int n = last - c0 + 1;
  return n <= 0 ? 0u : (n >= 32 ? kFull : ((1u << n) - 1u));
}


// Accessor of the tile for the shared sweep logic (beyond, walk,
// new_unaligned).  Indices are clamped into the region; the kernel only asks
// inside it.
template <typename R, int AX, int LD, int CAP = kCandCap>
struct TViewB {
  const TileMem<R, CAP>* m;
  const GView<R, AX, LD>* g;  // an unaligned marker's own fraction is read from the state
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
  // The marker of a reference.
  __device__ __forceinline__ Mk mk(uint16_t r) const {
    const int t = r & (kKindV - 1), ly = t / kRX;
    return Mk{(r & kKindV) ? 1 : 0, ri0 + t - ly * kRX, rj0 + ly};
  }
  // The marker beyond point 1 (side 0) or point 4 (side 1) of candidate C on
  // the unaligned edge (k, j): points 1 and 4 are the markers beyond A and B
  // seen from the chord's cell, and this is the one beyond them in turn.
  template <class CandT>
  __device__ __forceinline__ Mk next_beyond(const CandT& C, int side, int k, int j) const {
    const int c = k - 2 + (C.ord >> 1);
    int ci = 0, cj = 0, oi = 0, oj = 0;
    const Mk n = beyond(*this, mk(side ? C.b : C.a), c, j, &ci, &cj);
    if (n.kind < 0) return n;
    return beyond(*this, n, ci, cj, &oi, &oj);
  }
  __device__ __forceinline__ AP<R> moved(Mk mk) const {
    const int lx = cx(mk.i), ly = cy(mk.j), t = ly * kRX + lx;
    AP<R> p;
    p.jy = mk.j;
    if (mk.kind == 0) {
      p.ix = mk.i + get2(m->hq, lx, ly) - 1;
      p.fx = m->hfx[t];
      p.fy = R(0);
    } else {
      p.ix = mk.i + get2(m->vq, lx, ly) - 1;
      p.fx = m->vfx[t];
      p.fy = g->v(mk.i, mk.j);
    }
    return p;
  }
  __device__ __forceinline__ Landing<R> landing(int i, int j) const {
    const int c = get2(m->lq, cx(i), cy(j));
    Landing<R> L;
    L.present = knew(i, j) ^ knew(i + 1, j);
    L.kept_src = c == 0 ? -1 : i + c - 2;
    L.kept_fx = R(0);
    L.cancelled = 0;
    L.invariant = 0;
    return L;
  }
  // Moved point of a referenced marker relative to vertex (k, j).
  __device__ __forceinline__ void xy(uint16_t r, int k, int j, double* X, double* Y) const {
    const int t = r & (kKindV - 1), ly = t / kRX, lx = t - ly * kRX;
    // the same values as (double)n + (double)f; the conversions run on the
    // integer pipe and an aligned marker's y needs no addition
    if (r & kKindV) {
      *X = i2d(ri0 + lx + get2(m->vq, lx, ly) - 1 - k) + to_d<R>(m->vfx[t]);
      *Y = i2d(rj0 + ly - j) + to_d<R>(g->v(ri0 + lx, rj0 + ly));
    } else {
      *X = i2d(ri0 + lx + get2(m->hq, lx, ly) - 1 - k) + to_d<R>(m->hfx[t]);
      *Y = i2d(rj0 + ly - j);
    }
  }
  // An unaligned marker's own fraction (its y in the sweep), read from the
  // state; 0 for an aligned marker.
  __device__ __forceinline__ R own_fraction(uint16_t r) const {
    if (!(r & kKindV)) return R(0);
    const int t = r & (kKindV - 1), ly = t / kRX, lx = t - ly * kRX;
    return g->v(ri0 + lx, rj0 + ly);
  }
  // The point in the FP32 form, given its own fraction fy: the exact sums by
  // integer operations where they are exact (add_nf), and a float estimate
  // (Xf, Yf) within 2^-22 of each coordinate.
  __device__ __forceinline__ void xyf(uint16_t r, int k, int j, float fy, double* X, double* Y,
                                      float* Xf, float* Yf) const {
    const int t = r & (kKindV - 1), ly = t / kRX, lx = t - ly * kRX;
    const int ny = rj0 + ly - j;
    int nx;
    float fx;
    if (r & kKindV) {
      nx = ri0 + lx + get2(m->vq, lx, ly) - 1 - k;
      fx = (float)m->vfx[t];
      *Y = add_nf(ny, fy);
    } else {
      nx = ri0 + lx + get2(m->hq, lx, ly) - 1 - k;
      fx = (float)m->hfx[t];
      fy = 0.0f;
      *Y = i2d(ny);
    }
    *X = add_nf(nx, fx);
    *Xf = (float)nx + fx;
    *Yf = (float)ny + fy;
  }
};

// One marker per edge from its linked candidates (the rule of
// select_candidates, Sec. 2.4), in registers: candidates ranked by (position,
// generation order).
// *kept receives the slot of the kept candidate (-1: none); its centre-rule
// verdicts are formed by the caller where they are needed.
template <typename R, int CAP>
__device__ __forceinline__ NewV<R> select_linked(const TileMem<R, CAP>& M, int s, int present,
                                                 int* kept) {
  *kept = -1;
  if (s >= 0 && M.u.c.next[s] < 0 && present) {
    // one candidate on an edge that keeps a marker: it is the marker (the
    // common case, without the ranking below)
    const Cand& C = M.u.c.cand[s];
    NewV<R> one;
    *kept = s;
    one.present = 1;
    one.vr = -1;
    one.vl = -1;
    one.cancelled = 0;
    one.invariant = 0;
    if constexpr (sizeof(R) == 4) one.s = C.sf;
    else one.s = to_fraction<R>(C.y);
    return one;
  }
  double cy[6];
  float sf[6];
  long long key[6];
  int ord[6], sl[6];
  int n = 0;
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    if (s >= 0) {
      const Cand& C = M.u.c.cand[s];
      cy[q] = C.y;
      sf[q] = C.sf;
      key[q] = okey(C.y);
      ord[q] = C.ord;
      sl[q] = s;
      n = q + 1;
      s = M.u.c.next[s];
    } else {
      cy[q] = 0.0;
      sf[q] = 0.0f;
      key[q] = 0;
      ord[q] = 0;
      sl[q] = -1;
    }
  }
  int rank[6];
#pragma unroll
  for (int t = 0; t < 6; ++t) {
    int r = 0;
#pragma unroll
    for (int u = 0; u < 6; ++u)
      if (u != t && u < n && (key[u] < key[t] || (key[u] == key[t] && ord[u] < ord[t]))) ++r;
    rank[t] = r;
  }
  NewV<R> out;
  out.present = present;
  out.vr = -1;
  out.vl = -1;
  out.s = R(0.5);
  out.cancelled = 0;
  out.invariant = 0;
  int want = -1;  // rank of the kept candidate
  if (present && (n & 1)) {
    want = n / 2;
    out.cancelled = n / 2;  // the pairs around the middle one
  } else if (!present && !(n & 1)) {
    out.cancelled = n / 2;
  } else {
    out.invariant = 1;
    if (present && n > 0) {  // the candidate nearest the edge's middle, first in rank order
      double bd = 0.0;
#pragma unroll
      for (int t = 0; t < 6; ++t)
        if (t < n) {
          const double d = fabs(cy[t] - 0.5);
          if (want < 0 || d < bd || (d == bd && rank[t] < want)) {
            bd = d;
            want = rank[t];
          }
        }
    }
  }
  if (want >= 0) {
    double ysel = 0.0;
    float fsel = 0.0f;
#pragma unroll
    for (int t = 0; t < 6; ++t)
      if (t < n && rank[t] == want) {
        ysel = cy[t];
        fsel = sf[t];
        *kept = sl[t];
      }
    if constexpr (sizeof(R) == 4) out.s = fsel;  // to_fraction<float>, taken in the fit phase
    else out.s = to_fraction<R>(ysel);
  }
  return out;
}

// The tile with origin (i0, j0) of one grid (one block runs it).
template <typename R, int AX, int LD, int CAP = kCandCap>
__device__ __forceinline__ void sweep_tile(const GView<R, AX, LD>& G, const Buf<R>& out, int line_only,
                                           unsigned long long* ctr, unsigned long long* cfl_bits,
                                           int* status, const int i0, const int j0) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  TileMem<R, CAP>& M = *reinterpret_cast<TileMem<R, CAP>*>(smem_raw);
  constexpr int kHB = head_bits<CAP>(), kHPW = 32 / kHB;  // head bits, heads per word
  constexpr uint32_t kHNone = head_none<CAP>();
  __shared__ int s_nh, s_nv, s_nd, s_nc, s_ncand, s_ne, s_novf;
  __shared__ int s_cnt[D_NUSED];
  __shared__ unsigned long long s_dmax;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int kTileThreads = tile_threads<R>();
  constexpr int kWarps = kTileThreads / 32;
  const int tnx = G.tnx(), tny = G.tny();
  const int ri0 = i0 - 4, rj0 = j0 - 2;
  const long long P = G.d.P;
  if (tid < D_NUSED) s_cnt[tid] = 0;
  if (tid == 0) {
    s_nh = s_nv = s_nd = s_nc = s_ncand = s_ne = s_novf = 0;
    s_dmax = 0ull;
  }
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
        v = row_bits<LD>(G.K + (long long)y * G.d.kw, G.d.kw, x0) & span_mask(wi, vx0, vx1);
      if (zpl && ly >= vy0 && ly <= ey1)
        v = row_bits<LD>(G.Z + (long long)y * G.d.zw, G.d.zw, x0) & span_mask(wi, vx0, ex1);
      (zpl ? M.zb : M.kb)[u] = v;
    }
  } else {
    // region column lx is stored row ri0 + lx and region row ly stored column
    // rj0 + ly: a warp reads three words of 32 stored rows and transposes them
    const int c0 = rj0 >> 5;  // stored word holding region rows 0 and 1
    for (int g = warp; g < 2 * kRW; g += kWarps) {
      const int zpl = g >= kRW, gw = zpl ? g - kRW : g;
      const int lx = 32 * gw + lane, yr = ri0 + lx;
      const uint32_t* base = zpl ? G.Z : G.K;
      const int nw = zpl ? G.d.zw : G.d.kw;
      const int row1 = zpl ? ey1 : vy1;
      uint32_t w[3] = {0u, 0u, 0u};
      if (lx >= vx0 && lx <= (zpl ? ex1 : vx1)) {
        const uint32_t* r = base + (long long)yr * nw;
#pragma unroll
        for (int q = 0; q < 3; ++q)
          if (c0 + q >= 0 && c0 + q < nw) w[q] = ld_state<LD>(&r[c0 + q]);
      }
      uint32_t* dst = zpl ? M.zb : M.kb;
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const uint32_t col = transpose32(w[q], lane);
        const int ly = 32 * (c0 + q) + lane - rj0;
        if (ly >= 0 && ly < kRY) dst[ly * kRW + gw] = (ly >= vy0 && ly <= row1) ? col : 0u;
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
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      M.hq[q][t] = 0u;
      M.vq[q][t] = 0u;
      M.lq[q][t] = 0u;
    }
    mine |= (h | v) != 0u;
  }
  const bool busy = __syncthreads_or(mine) != 0;
  const TViewB<R, AX, LD, CAP> TV{&M, &G, ri0, rj0, tnx, tny};

  if (busy) {
    for (int t0 = warp * 32; t0 < kRB; t0 += kTileThreads) {
      const int t = t0 + lane;
      push_bits_warp(t < kRB ? M.hm[t] : 0u, t, M.lh, &s_nh, lane);
      push_bits_warp(t < kRB ? M.vm[t] : 0u, t, M.u.p.lv, &s_nv, lane);
    }
    static_assert(sizeof(M.head) % 16 == 0, "vector initialisation");
    for (int e = tid; e < (int)(sizeof(M.head) / 16); e += kTileThreads)
      reinterpret_cast<uint4*>(M.head)[e] = make_uint4(~0u, ~0u, ~0u, ~0u);
    __syncthreads();

    // P2: moved points (aligned and unaligned markers in one pass), corner
    // flips, landing claims
    const int nh = s_nh, nm = s_nh + s_nv;
    int n_cfl = 0, n_clamp = 0;
    R dmax = R(0);
    for (int w0 = warp * 32; w0 < nm; w0 += kTileThreads) {
      const int w = w0 + lane;
      int claimed = -1;
      if (w < nh) {
        const int id = M.lh[w], lx = id % kRX, ly = id / kRX;
        const int x = ri0 + lx, y = rj0 + ly;
        Flags f;
        const AP<R> p = G.advect(Mk{0, x, y}, f);
        put2(M.hq, lx, ly, p.ix - x + 1);
        M.hfx[id] = p.fx;
        if (owned(x, y)) {
          n_cfl += f.cfl;
          n_clamp += f.clamp;
          dmax = fmax(dmax, dabs_of<R>(f));
        }
        // a marker moving right passes vertex x+1, one moving left vertex x
        if (p.ix == x + 1) atomicXor(&M.kn[ly * kRW + ((lx + 1) >> 5)], 1u << ((lx + 1) & 31));
        else if (p.ix == x - 1) atomicXor(&M.kn[ly * kRW + (lx >> 5)], 1u << (lx & 31));
        const int dl = p.ix - ri0;
        if (dl >= 1 && dl <= kRX - 3) {
          const uint32_t bit = 1u << (dl & 31);
          if (!(atomicOr(&M.claim[ly * kRW + (dl >> 5)], bit) & bit)) claimed = ly * kRX + dl;
        }
      } else if (w < nm) {
        const int id = M.u.p.lv[w - nh], lx = id % kRX, ly = id / kRX;
        const int x = ri0 + lx, y = rj0 + ly;
        Flags f;
        const AP<R> p = G.advect(Mk{1, x, y}, f);
        put2(M.vq, lx, ly, p.ix - x + 1);
        M.vfx[id] = p.fx;
        if (owned(x, y)) {
          if (x >= 1 && x <= tnx - 1) {
            n_cfl += f.cfl;
            dmax = fmax(dmax, dabs_of<R>(f));
          } else {  // a wall marker normal to the sweep stays
            if (AX) { if (in_range((long long)x * P + y, G.d.nH())) out.sH[(long long)x * P + y] = p.fy; }
            else if (in_range((long long)y * P + x, G.d.nV())) out.sV[(long long)y * P + x] = p.fy;
          }
        }
      }
      const unsigned cm = __ballot_sync(kFull, claimed >= 0);
      if (cm) {
        const int leader = __ffs(cm) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(&s_nd, __popc(cm));
        base = __shfl_sync(kFull, base, leader);
        if (claimed >= 0) M.u.p.ld[base + __popc(cm & ((1u << lane) - 1u))] = (uint16_t)claimed;
      }
    }
    flush_count(s_cnt, D_CFL, n_cfl, lane);
    flush_count(s_cnt, D_WALL_CLAMP, n_clamp, lane);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) dmax = fmax(dmax, __shfl_xor_sync(kFull, dmax, o));
    if (lane == 0 && dmax > R(0))
      atomicMax(&s_dmax, (unsigned long long)__double_as_longlong((double)dmax));
    __syncthreads();

    // P3: landings on the claimed aligned edges
    // landings on warps 0-4, the word pass (owned edges without a landing,
    // interface cells) on warps 5-7 at the same time
    const int nd = s_nd;
    int n_canc = 0, n_inv = 0;
    constexpr int kSplit = kTileThreads - kTJ * kRW;  // 96 words on the last three warps
    static_assert(kSplit > 0 && kSplit % 32 == 0, "warp split");
    for (int w = tid; w < nd && tid < kSplit; w += kSplit) {
      const int id = M.u.p.ld[w], dl = id % kRX, ly = id / kRX;
      const int x = ri0 + dl, y = rj0 + ly;
      bool valid[3];
      R fx[3];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const int e = dl - 1 + q, ie = ly * kRX + e;
        valid[q] = getb(M.hm, e, ly) && e + get2(M.hq, e, ly) - 1 == dl;
        fx[q] = valid[q] ? M.hfx[ie] : R(0);
      }
      const Landing<R> L =
          choose_landing3<R>(valid, fx, x, getb(M.kn, dl, ly) ^ getb(M.kn, dl + 1, ly));
      if (L.kept_src >= 0) put2(M.lq, dl, ly, L.kept_src - x + 2);
      if (owned(x, y)) {
        n_canc += L.cancelled;
        n_inv += L.invariant;
        if (L.present) {
          if (AX) { if (in_range((long long)x * P + y, G.d.nV())) out.sV[(long long)x * P + y] = L.kept_fx; }
          else if (in_range((long long)y * P + x, G.d.nH())) out.sH[(long long)y * P + x] = L.kept_fx;
        }
      }
    }
    if (tid >= kSplit) {
      const int t = tid - kSplit;  // one word each
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
          n_inv += 1;
          if (AX) { if (in_range((long long)x * P + y, G.d.nV())) out.sV[(long long)x * P + y] = R(0.5); }
          else if (in_range((long long)y * P + x, G.d.nH())) out.sH[(long long)y * P + x] = R(0.5);
        }
      }
      // interface cells (corner colours not all equal) whose chords can
      // cross a grid line k in [i0, i0+64]: cells k-2..k
      uint32_t ic = 0u;
      if (ly <= ty1) {
        const uint32_t a = M.kb[u], b = M.kb[u + kRW];
        ic = ((a ^ shr1(M.kb, ly, wi)) | (b ^ shr1(M.kb, ly + 1, wi)) | (a ^ b)) &
             span_mask(wi, max(2, vx0), min(kTI + 4, ex1));
      }
      push_bits_warp(ic, u, M.lh, &s_nc, lane);
    }
    flush_count(s_cnt, D_CANCELLED, n_canc, lane);
    flush_count(s_cnt, D_INVARIANT, n_inv, lane);
    __syncthreads();
    // the marker sets are dead: their storage becomes the candidate sets
    for (int t = tid; t < kRB; t += kTileThreads) {
      M.hc[t] = 0u;
      M.ovf[t] = 0u;
    }
    __syncthreads();

    // P4: candidates.  A thread takes one interface cell: counts the grid
    // lines its moved chords cross, takes that many slots, then fills them.
    const int nc = s_nc;
    const int kmin = max(1, i0), kmax = min(tnx - 1, i0 + kTI);
    for (int w0 = warp * 32; w0 < nc; w0 += kTileThreads) {
      const int w = w0 + lane;
      int c = 0, j = 0, ly = 0, ns = 0, ncross = 0;
      int seg[2][2] = {{0, 0}, {0, 0}};
      int ia[2] = {0, 0}, ib[2] = {0, 0};
      if (w < nc) {
        const int id = M.lh[w], lx = id % kRX;
        ly = id / kRX;
        c = ri0 + lx;
        j = rj0 + ly;
        ns = cell_segments(TV, c, j, seg);
#pragma unroll
        for (int t = 0; t < 2; ++t)
          if (t < ns) {
            ia[t] = TV.moved(edge_marker(c, j, seg[t][0])).ix;
            ib[t] = TV.moved(edge_marker(c, j, seg[t][1])).ix;
            ncross += max(0, min(max(ia[t], ib[t]), kmax) - max(min(ia[t], ib[t]) + 1, kmin) + 1);
          }
      }
      int slot = warp_alloc(ncross, &s_ncand, lane);
#pragma unroll
      for (int t = 0; t < 2; ++t) {
        if (t >= ns) continue;
        const Mk ma = edge_marker(c, j, seg[t][0]);
        const Mk mb = edge_marker(c, j, seg[t][1]);
        const int klo = max(min(ia[t], ib[t]) + 1, kmin), khi = min(max(ia[t], ib[t]), kmax);
        for (int k = klo; k <= khi; ++k, ++slot) {
          const int e = (j - j0) * (kTI + 1) + (k - i0);
          const int ex = k - ri0, eu = ly * kRW + (ex >> 5);
          const uint32_t ebit = 1u << (ex & 31);
          if (slot >= CAP) {
            atomicOr(&M.ovf[eu], ebit);
            continue;
          }
          const bool a_left = ia[t] < k;
          const Mk mA = a_left ? ma : mb, mB = a_left ? mb : ma;
          Cand& C = M.u.c.cand[slot];
          C.a = TV.ref(mA);
          C.b = TV.ref(mB);
          uint8_t fl = k < i0 + kTI ? CF_OWNED : 0;
          int c1i = 0, c1j = 0, c4i = 0, c4j = 0;
          const Mk n1 = beyond(TV, mA, c, j, &c1i, &c1j);
          const Mk n4 = beyond(TV, mB, c, j, &c4i, &c4j);
          if (n1.kind >= 0) {
            C.p1 = TV.ref(n1);
            fl |= CF_P1;
          }
          if (n4.kind >= 0) {
            C.p4 = TV.ref(n4);
            fl |= CF_P4;
          }
          C.fl = fl;
          C.edge = (uint16_t)e;
          C.ord = (uint8_t)((c - (k - 2)) * 2 + t);
          {  // push the slot on the edge's list: a head of kHB bits in a shared word
            uint32_t* hw = &M.head[e / kHPW];
            const int sh = (e % kHPW) * kHB;
            uint32_t old = *hw, seen;
            do {  // each retry follows another thread's successful update
              seen = old;
              old = atomicCAS(hw, seen, (seen & ~(kHNone << sh)) | ((uint32_t)slot << sh));
            } while (old != seen);
            const uint32_t prev = (seen >> sh) & kHNone;
            M.u.c.next[slot] = prev == kHNone ? (int16_t)-1 : (int16_t)prev;
          }
          atomicOr(&M.hc[eu], ebit);
        }
      }
    }
    __syncthreads();

    // P5: circle fits (Sec. 2.2).  Lanes 2m and 2m+1 fit the circles through
    // point 1 and point 4 of one candidate and the even lane combines them,
    // as fit_crossing does; the warps that take candidates rotate with the
    // block so that the FP64 work spreads over the SM's sub-partitions.  The
    // last three warps first list the edges with linked candidates.
    const int ncand = min(s_ncand, CAP);
    // the interface-cell list is dead: its storage becomes the verdicts of P6
    for (int e = tid; e < kNVE / 16; e += kTileThreads)
      reinterpret_cast<uint4*>(M.vrl)[e] = make_uint4(0u, 0u, 0u, 0u);
    if (warp >= kWarps - 3) {
      const int t = (warp - (kWarps - 3)) * 32 + lane;  // kTJ * kRW = 96 words
      const int u = (2 + t / kRW) * kRW + t % kRW;
      push_bits_warp(M.hc[u], u, M.u.c.le, &s_ne, lane);
      const int no = __reduce_add_sync(kFull, __popc(M.ovf[u]));  // edges done in place
      if (no != 0 && lane == 0) atomicAdd(&s_novf, no);
    }
    const int rot = (int)((blockIdx.x + blockIdx.y) & 3u);
    int n_fit[4] = {0, 0, 0, 0};  // D_FIT_ONLINE .. D_FIT_TWO
    const int vt = (((warp + rot) % kWarps) << 5) | lane;
    for (int b0 = 0; b0 < 2 * ncand; b0 += kTileThreads) {
      const int item = b0 + vt, side = item & 1;
      Cand& C = M.u.c.cand[min(item >> 1, CAP - 1)];
      int k = 0, j = 0;
      bool act = item < 2 * ncand;
      if (act) {
        k = i0 + C.edge % (kTI + 1);
        j = j0 + C.edge / (kTI + 1);
        act = !getb(M.ovf, k - ri0, j - rj0);  // else the edge is done in place
      }
      // the pair shares the chord: the even lane converts A and forms cx,
      // the odd lane B and cy, and they swap (shuffles instead of FP64 work)
      double px = 0.0, py = 0.0;
      float pxf = 0.0f, pyf = 0.0f, fy_t = 0.0f;
      if (act) {
        if constexpr (sizeof(R) == 4) {
          // the state reads this lane needs, issued together
          const uint8_t fl = C.fl;
          const float fy_ab = TV.own_fraction(side ? C.b : C.a);
          if (fl & (side ? CF_P4 : CF_P1)) fy_t = TV.own_fraction(side ? C.p4 : C.p1);
          TV.xyf(side ? C.b : C.a, k, j, fy_ab, &px, &py, &pxf, &pyf);
        } else {
          TV.xy(side ? C.b : C.a, k, j, &px, &py);
        }
      }
      const double ox = __shfl_xor_sync(kFull, px, 1), oy = __shfl_xor_sync(kFull, py, 1);
      const float oxf = __shfl_xor_sync(kFull, pxf, 1), oyf = __shfl_xor_sync(kFull, pyf, 1);
      const float bxf = side ? pxf : oxf, byf = side ? pyf : oyf;  // B, estimated in float
      const double ax = side ? ox : px, ay = side ? oy : py;
      const double bx = side ? px : ox, by = side ? py : oy;
      const double dd = side ? by - ay : bx - ax;
      const double od = __shfl_xor_sync(kFull, dd, 1);
      const double cx = side ? od : dd, cy = side ? dd : od;
      const double sq = dd * dd, osq = __shfl_xor_sync(kFull, sq, 1);
      const double c2 = side ? osq + sq : sq + osq;  // cx*cx + cy*cy
      const double x0 = -ax;
      const bool online = d_eq0(bx);
      double ys = 0.0;
      bool ok = false;
      if (act && !online) {
        const uint8_t fl = C.fl;
        if (!line_only && !d_below_sep(c2) && (fl & (side ? CF_P4 : CF_P1))) {
          if constexpr (sizeof(R) == 4) {
            // the third point's offsets from A exactly; its distance from B
            // only where a float estimate (error below 2e-6 per component)
            // does not already put it clearly past the minimum separation
            double rx, ry, r2;
            bool tfar;
            auto third = [&](uint16_t ref, float fy) {
              double X, Y;
              float Xf, Yf;
              TV.xyf(ref, k, j, fy, &X, &Y, &Xf, &Yf);
              rx = X - ax;
              ry = Y - ay;
              r2 = rx * rx + ry * ry;
              const float txf = Xf - bxf, tyf = Yf - byf;
              if (txf * txf + tyf * tyf >= 1.5e-4f) {
                tfar = true;
              } else {
                const double tx = X - bx, ty = Y - by;
                tfar = !d_below_sep(tx * tx + ty * ty);
              }
            };
            third(side ? C.p4 : C.p1, fy_t);
            bool use = true;
            if (side ? !tfar : d_below_sep(r2)) {  // too close to B (A): the next marker
              const Mk q = TV.next_beyond(C, side, k, j);
              if (q.kind >= 0) {
                const uint16_t qr = TV.ref(q);
                third(qr, TV.own_fraction(qr));
              } else {
                use = false;
              }
            }
            if (use) ok = circle_cross_r(ay, x0, cx, cy, c2, rx, ry, r2, tfar, &ys);
          } else {
            double X, Y;
            TV.xy(side ? C.p4 : C.p1, k, j, &X, &Y);
            FitPt T = fit_pt(X, Y, ax, ay, bx, by);
            bool use = true;
            if (d_below_sep(side ? T.t2 : T.r2)) {  // too close to A (B): the next marker
              const Mk q = TV.next_beyond(C, side, k, j);
              if (q.kind >= 0) {
                TV.xy(TV.ref(q), k, j, &X, &Y);
                T = fit_pt(X, Y, ax, ay, bx, by);
              } else {
                use = false;
              }
            }
            if (use) ok = circle_cross(ay, x0, cx, cy, c2, T, &ys);
          }
        }
      }
      const double yo = __shfl_xor_sync(kFull, ys, 1);
      const bool oko = __shfl_xor_sync(kFull, (int)ok, 1) != 0;
      if (act && side == 0) {
        double y;
        int kind;
        if (online) {
          y = by;
          kind = D_FIT_ONLINE;
        } else if (ok && oko) {
          y = 0.5 * (ys + yo);
          kind = D_FIT_TWO;
        } else if (ok || oko) {
          y = ok ? ys : yo;
          kind = D_FIT_ONE;
        } else {  // no circle: the chord's own crossing
          y = ay + (x0 * cy) / cx;
          kind = D_FIT_LINE;
        }
        C.y = y;
        if (sizeof(R) == 4) C.sf = to_fraction<float>(y);  // here, where the FP64 pipe is busy anyway
        C.kind = (int8_t)kind;
        if (C.fl & CF_OWNED) {  // static indices keep the counters in registers
#pragma unroll
          for (int q = 0; q < 4; ++q) n_fit[q] += kind == D_FIT_ONLINE + q;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) flush_count(s_cnt, D_FIT_ONLINE + q, n_fit[q], lane);
    __syncthreads();

    // P6: one marker per unaligned edge (Sec. 2.4)
    const int ne = s_ne;
    n_canc = 0;
    n_inv = 0;
    for (int w = tid; w < ne && tid < kSplit; w += kSplit) {
      const int id = M.u.c.le[w], ex = id % kRX, ey = id / kRX;
      if (getb(M.ovf, ex, ey)) continue;
      const int k = ri0 + ex, j = rj0 + ey;
      const int e = (j - j0) * (kTI + 1) + (k - i0);
      const bool own = k < i0 + kTI;
      const int present = getb(M.kn, ex, ey) ^ getb(M.kn, ex, ey + 1);
      const uint32_t hd = (M.head[e / kHPW] >> ((e % kHPW) * kHB)) & kHNone;
      int kept;
      const NewV<R> nv = select_linked<R>(M, hd == kHNone ? -1 : (int)hd, present, &kept);
      if (own) {
        n_canc += nv.cancelled;
        n_inv += nv.invariant;
      }
      // centre-rule verdicts of the kept candidate (Sec. 2.3), for the cells
      // either side of the edge that have four markers after the sweep (the
      // only ones whose centre colour the rule sets)
      int vr = -1, vl = -1;
      if (kept >= 0) {
        auto four = [&](int x) {  // cell (x, ey) of the region, new colours
          const int a = getb(M.kn, x, ey), b = getb(M.kn, x + 1, ey);
          const int c = getb(M.kn, x + 1, ey + 1), d = getb(M.kn, x, ey + 1);
          return a != b && b != c && c != d;
        };
        const bool fr = four(ex), fl = four(ex - 1);
        if (fr || fl) {
          const Cand& C = M.u.c.cand[kept];
          const Mk none{-1, 0, 0};
          if (fr) {
            const int lr = walk(TV, TV.mk(C.b), (C.fl & CF_P4) ? TV.mk(C.p4) : none, k);
            vr = lr < 0 ? -1 : !TV.knew(k, lr);
          }
          if (fl) {
            const int ll = walk(TV, TV.mk(C.a), (C.fl & CF_P1) ? TV.mk(C.p1) : none, k - 1);
            vl = ll < 0 ? -1 : !TV.knew(k, ll);
          }
        }
      }
      M.vrl[e] = verdicts(vr, vl);
      if (own && nv.present) {
        if (AX) { if (in_range((long long)k * P + j, G.d.nH())) out.sH[(long long)k * P + j] = nv.s; }
        else if (in_range((long long)j * P + k, G.d.nV())) out.sV[(long long)j * P + k] = nv.s;
      }
    }
    if (tid >= kSplit && 2 + (tid - kSplit) / kRW <= ty1) {  // rows of unaligned edges only
      const int t = tid - kSplit;
      const int ly = 2 + t / kRW, wi = t % kRW, u = ly * kRW + wi;
      // owned interior edges that gain a marker without a candidate: counted,
      // fraction 0.5
      uint32_t miss = (M.kn[u] ^ M.kn[u + kRW]) & ~M.hc[u] & ~M.ovf[u] &
                      span_mask(wi, max(4, 1 - ri0), min(kTI + 3, tnx - 1 - ri0));
      while (miss) {
        const int b = __ffs(miss) - 1;
        miss &= miss - 1;
        const int k = ri0 + 32 * wi + b, j = rj0 + ly;
        n_inv += 1;
        if (AX) { if (in_range((long long)k * P + j, G.d.nH())) out.sH[(long long)k * P + j] = R(0.5); }
        else if (in_range((long long)j * P + k, G.d.nV())) out.sV[(long long)j * P + k] = R(0.5);
      }
    }
    // edges whose candidates did not fit in the tile's list are done in
    // place by the generic logic, spread over all threads: overflow edge m
    // (in word order) goes to thread m mod the block size
    for (int m = tid; m < s_novf; m += kTileThreads) {
      int u = 2 * kRW, r = m;
      for (; u < kRB; ++u) {
        const int c = __popc(M.ovf[u]);
        if (r < c) break;
        r -= c;
      }
      if (u >= kRB) break;  // not reached: s_novf counts these words' bits
      uint32_t o = M.ovf[u];
      for (; r > 0; --r) o &= o - 1;
      const int b = __ffs(o) - 1, ly = u / kRW, wi = u % kRW;
      const int k = ri0 + 32 * wi + b, j = rj0 + ly;
      const int e = (j - j0) * (kTI + 1) + (k - i0);
      const bool own = k < i0 + kTI;
      int oc[D_NUSED];
#pragma unroll
      for (int c = 0; c < D_NUSED; ++c) oc[c] = 0;
      const NewV<R> nv = new_unaligned<R>(TV, line_only != 0, k, j, own ? oc : nullptr);
      for (int c = 0; c < D_NUSED; ++c)
        if (oc[c]) atomicAdd(&s_cnt[c], oc[c]);
      M.vrl[e] = verdicts(nv.vr, nv.vl);
      if (own && nv.present) {
        if (AX) { if (in_range((long long)k * P + j, G.d.nH())) out.sH[(long long)k * P + j] = nv.s; }
        else if (in_range((long long)j * P + k, G.d.nV())) out.sV[(long long)j * P + k] = nv.s;
      }
    }
    flush_count(s_cnt, D_CANCELLED, n_canc, lane);
    flush_count(s_cnt, D_INVARIANT, n_inv, lane);
    __syncthreads();
  }

  // P7: colour words.  Lane L of warp ow (0 or 1) takes tile row j0 + L and
  // the 32 vertices / cells i0 + 32 ow + b; the y sweep transposes them into
  // stored rows.  Centre colours of new four-marker cells (all four edges
  // with a marker) come from the verdicts of edges i (right) and i+1 (left);
  // the right one wins.
  int n_zset = 0, n_zconf = 0;
  if (warp < 2) {
    const int ow = warp, ly = 2 + lane, cx0 = 4 + 32 * ow;
    const int j = rj0 + ly;
    uint32_t kw = bits32(M.kn, ly, cx0);
    uint32_t zw = bits32(M.zb, ly, cx0);
    const uint32_t vmask = ly <= vy1 ? upto32(cx0, vx1) : 0u;
    const uint32_t cmask = ly <= ey1 ? upto32(cx0, ex1) : 0u;
    if (busy && cmask) {
      const uint32_t a1 = bits32(M.kn, ly, cx0 + 1);
      const uint32_t b0 = bits32(M.kn, ly + 1, cx0), b1 = bits32(M.kn, ly + 1, cx0 + 1);
      uint32_t fm = (kw ^ a1) & (b0 ^ b1) & (kw ^ b0) & cmask;
      while (fm) {
        const int b = __ffs(fm) - 1;
        fm &= fm - 1;
        const int i = i0 + 32 * ow + b;
        const int e = (j - j0) * (kTI + 1) + (i - i0);
        const int a = (i >= 1) ? verdict_r(M.vrl[e]) : -1;
        const int bl = (i + 1 <= tnx - 1) ? verdict_l(M.vrl[e + 1]) : -1;
        int zc = -1;
        if (a >= 0) {
          zc = a;
          n_zset += 1;
          if (bl >= 0 && bl != a) n_zconf += 1;
        } else if (bl >= 0) {
          zc = bl;
          n_zset += 1;
        }
        if (zc >= 0) zw = zc ? (zw | (1u << b)) : (zw & ~(1u << b));
      }
    }
    kw &= vmask;
    zw &= cmask;
    if (AX) {
      kw = transpose32(kw, lane);
      zw = transpose32(zw, lane);
      const int row = i0 + 32 * ow + lane, word = j0 >> 5;
      if (row <= G.d.ny && word < G.d.kw) out.K[(long long)row * G.d.kw + word] = kw;
      if (row < G.d.ny && word < G.d.zw) out.Z[(long long)row * G.d.zw + word] = zw;
    } else {
      const int word = (i0 >> 5) + ow;
      if (j <= G.d.ny && word < G.d.kw) out.K[(long long)j * G.d.kw + word] = kw;
      if (j < G.d.ny && word < G.d.zw) out.Z[(long long)j * G.d.zw + word] = zw;
    }
  }

  flush_count(s_cnt, D_ZSET, n_zset, lane);
  flush_count(s_cnt, D_ZCONFLICT, n_zconf, lane);

  // block counters to the grid's
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
__global__ void __launch_bounds__(tile_threads<R>(), tile_min_blocks<R>())
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
__global__ void __launch_bounds__(tile_threads<R>(), tile_min_blocks<R>())
k_sweep_tile_batch(const SweepDesc<R, AX>* __restrict__ descs, const WorkItem* __restrict__ items) {
  const WorkItem it = items[blockIdx.x];
  const SweepDesc<R, AX>& D = descs[it.grid];
  if (!D.active) return;
  sweep_tile<R, AX>(D.G, D.out, D.line_only, D.ctr, D.cfl_bits, D.status, it.tx * kTI, it.ty * kTJ);
}

// Square grids only: a grid's tiles are the same in both sweep directions, so
// one launch can take the first (or second) sweep of every grid, each tile in
// the direction its grid's split order puts there (x first on even steps):
// the x descriptor when it is active for this launch, else the y one.
template <typename R, int CAP = kCandCap>
__global__ void __launch_bounds__(tile_threads<R>(), tile_min_blocks<R>())
k_sweep_tile_both(const SweepDesc<R, 0>* __restrict__ dx, const SweepDesc<R, 1>* __restrict__ dy,
                  const WorkItem* __restrict__ items) {
  const WorkItem it = items[blockIdx.x];
  const SweepDesc<R, 0>& X = dx[it.grid];
  if (X.active) {
    sweep_tile<R, 0, 0, CAP>(X.G, X.out, X.line_only, X.ctr, X.cfl_bits, X.status, it.tx * kTI,
                             it.ty * kTJ);
  } else {
    const SweepDesc<R, 1>& Y = dy[it.grid];
    sweep_tile<R, 1, 0, CAP>(Y.G, Y.out, Y.line_only, Y.ctr, Y.cfl_bits, Y.status, it.tx * kTI,
                             it.ty * kTJ);
  }
}

}  // namespace ebit
