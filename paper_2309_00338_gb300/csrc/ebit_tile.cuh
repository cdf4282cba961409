// Tiled sweep kernel: one split sweep (Sec. 2.1-2.4) for a tile of the grid,
// with everything the tile depends on staged in shared memory.
//
// Tile (sweep coordinates): vertices i in [i0, i0+64), j in [j0, j0+32) with
// their aligned edge (i,j), unaligned edge (i,j) and cell (i,j).  The region
// held in shared memory is the tile plus a halo, vertices
// [i0-4, i0+67] x [j0-2, j0+34]: candidate chords for line k come from cells
// k-2..k, their end markers' neighbours lie one cell further, the
// neighbours' next markers (points 1 and 4 when a neighbour is too close)
// one more, and the centre rule looks at landings on edges k-1..k+1.
//
// Phases (barrier between each), every quantity computed once per tile:
//   P0 colours of the region; a tile with no marker in its region only copies
//   P1 moved point of every marker in the region (the only global reads of
//      fractions and velocities, and only where a marker exists)
//   P2 new corner colour of every region vertex
//   P3 landings on aligned edges; writes the tile's new aligned markers
//   P4 compact list of the unaligned edges with candidate chords
//   P5a per listed edge: its crossing chords become candidates (points 1-4
//      in integer + fraction form, centre-rule verdicts) in one dense array;
//      integer and shared-memory work only
//   P5b circle fits of the candidates, one candidate per thread, so the FP64
//      pipe sees full warps
//   P5c per listed edge: one marker per edge from its candidates
//   P6 writes new corner and centre colour words and unaligned markers;
//      block-level counter reduction
#pragma once
#include "ebit_device.cuh"

namespace ebit {

constexpr int kTI = 64, kTJ = 32;
constexpr int kRX = kTI + 8, kRY = kTJ + 5, kRN = kRX * kRY;
constexpr int kNVE = (kTI + 1) * kTJ;  // unaligned edges k in [i0, i0+64], rows j0..j0+31
constexpr int kTileThreads = 256;
constexpr int kCandCap = 192;          // candidates held per tile; beyond, an edge fits in place
constexpr uint16_t kInPlace = 0xffff;

// A moved point in vertex-local integer + fraction form: x = dx + fx, y = dy + fy.
template <typename R>
struct PP {
  int8_t dx, dy;
  R fx, fy;
};

template <typename R>
__device__ __forceinline__ PP<R> pp_of(const AP<R>& p, int k, int j) {
  PP<R> q;
  q.dx = (int8_t)(p.ix - k);
  q.dy = (int8_t)(p.jy - j);
  q.fx = p.fx;
  q.fy = p.fy;
  return q;
}

template <typename R>
__device__ __forceinline__ void pp_xy(const PP<R>& q, double* X, double* Y) {
  *X = (double)(int)q.dx + (double)q.fx;
  *Y = (double)(int)q.dy + (double)q.fy;
}

// Candidate of one unaligned edge: chord ends A, B; point 1 (p1) with the
// next marker beyond it (q1) in case p1 is too close to A; likewise 4.
enum { CF_P1 = 1, CF_Q1 = 2, CF_P4 = 4, CF_Q4 = 8, CF_OWNED = 16, CF_UNUSED = 128 };
template <typename R>
struct Cand {
  PP<R> a, b, p1, q1, p4, q4;
  double y;
  uint8_t fl;
  int8_t vr, vl, kind;
};

template <typename R>
constexpr size_t tile_smem_bytes() {
  return sizeof(Cand<R>) * kCandCap + sizeof(R) * (4 * kRN + kNVE) + 2 * (2 * kRN + 2 * kNVE) +
         (5 * kRN + 4 * kNVE);
}

// The tile with origin (i0, j0) of one grid (one block runs it).
template <typename R, int AX>
__device__ __forceinline__ void sweep_tile(const GView<R, AX>& G, const Buf<R>& out, int line_only,
                                           unsigned long long* ctr, unsigned long long* cfl_bits,
                                           int* status, const int i0, const int j0) {
  extern __shared__ __align__(16) unsigned char smem[];
  Cand<R>* cand = reinterpret_cast<Cand<R>*>(smem);
  R* hfx = reinterpret_cast<R*>(cand + kCandCap);
  R* vfx = hfx + kRN;
  R* vfy = vfx + kRN;
  R* lfx = vfy + kRN;
  R* vs = lfx + kRN;
  int16_t* hix = reinterpret_cast<int16_t*>(vs + kNVE);
  int16_t* vix = hix + kRN;
  uint16_t* list = reinterpret_cast<uint16_t*>(vix + kRN);
  uint16_t* ebase = list + kNVE;
  uint8_t* kb = reinterpret_cast<uint8_t*>(ebase + kNVE);
  uint8_t* kn = kb + kRN;
  uint8_t* zb = kn + kRN;
  uint8_t* lpres = zb + kRN;
  int8_t* lsrc = reinterpret_cast<int8_t*>(lpres + kRN);
  int8_t* vr = lsrc + kRN;
  int8_t* vl = vr + kNVE;
  uint8_t* vp = reinterpret_cast<uint8_t*>(vl + kNVE);
  uint8_t* ecount = vp + kNVE;
  __shared__ int s_nlist, s_ncand;
  __shared__ int s_cnt[D_NUSED];
  __shared__ unsigned long long s_dmax;

  const int tid = threadIdx.x;
  const int tnx = G.tnx(), tny = G.tny();
  const int ri0 = i0 - 4, rj0 = j0 - 2;
  if (tid < D_NUSED) s_cnt[tid] = 0;
  if (tid == 0) {
    s_nlist = 0;
    s_ncand = 0;
    s_dmax = 0ull;
  }
  int cnt[D_NUSED];
#pragma unroll
  for (int c = 0; c < D_NUSED; ++c) cnt[c] = 0;
  R dmax = R(0);
  auto owned = [&](int x, int y) { return x >= i0 && x < i0 + kTI && y >= j0 && y < j0 + kTJ; };
  // region entry t -> (lx, ly): consecutive threads walk along real rows
  auto coord = [&](int t, int* lx, int* ly) {
    if (AX) { *lx = t / kRY; *ly = t % kRY; } else { *lx = t % kRX; *ly = t / kRX; }
  };

  // P0: colours
  for (int t = tid; t < kRN; t += kTileThreads) {
    int lx, ly;
    coord(t, &lx, &ly);
    const int id = ly * kRX + lx, x = ri0 + lx, y = rj0 + ly;
    kb[id] = (x >= 0 && x <= tnx && y >= 0 && y <= tny) ? (uint8_t)G.k(x, y) : 0;
    zb[id] = (x >= 0 && x < tnx && y >= 0 && y < tny) ? (uint8_t)G.z(x, y) : 0;
  }
  __syncthreads();
  int any = 0;
  for (int t = tid; t < kRN && !any; t += kTileThreads) {
    int lx, ly;
    coord(t, &lx, &ly);
    const int id = ly * kRX + lx, x = ri0 + lx, y = rj0 + ly;
    if (x >= 0 && x < tnx && y >= 0 && y <= tny && lx + 1 < kRX && kb[id] != kb[id + 1]) any = 1;
    if (x >= 0 && x <= tnx && y >= 0 && y < tny && ly + 1 < kRY && kb[id] != kb[id + kRX]) any = 1;
  }
  const int busy = __syncthreads_or(any);

  const TView<R, kRX, kRY> TV{kb, kn, zb, hix, hfx, vix, vfx, vfy, lpres, lsrc, lfx,
                              ri0, rj0, tnx, tny};
  if (!busy) {
    for (int t = tid; t < kRN; t += kTileThreads) kn[t] = kb[t];
    for (int v = tid; v < kNVE; v += kTileThreads) {
      vr[v] = -1;
      vl[v] = -1;
      vp[v] = 0;
    }
    __syncthreads();
  } else {
    // P1: moved points
    for (int t = tid; t < kRN; t += kTileThreads) {
      int lx, ly;
      coord(t, &lx, &ly);
      const int id = ly * kRX + lx, x = ri0 + lx, y = rj0 + ly;
      if (x >= 0 && x < tnx && y >= 0 && y <= tny && lx + 1 < kRX && kb[id] != kb[id + 1]) {
        Flags f;
        const AP<R> p = G.advect(Mk{0, x, y}, f);
        hix[id] = (int16_t)(p.ix - ri0);
        hfx[id] = p.fx;
        if (owned(x, y)) {
          cnt[D_CFL] += f.cfl;
          cnt[D_WALL_CLAMP] += f.clamp;
          dmax = fmax(dmax, dabs_of<R>(f));
        }
      }
      if (x >= 0 && x <= tnx && y >= 0 && y < tny && ly + 1 < kRY && kb[id] != kb[id + kRX]) {
        Flags f;
        const AP<R> p = G.advect(Mk{1, x, y}, f);
        vix[id] = (int16_t)(p.ix - ri0);
        vfx[id] = p.fx;
        vfy[id] = p.fy;
        if (owned(x, y) && x >= 1 && x <= tnx - 1) {
          cnt[D_CFL] += f.cfl;
          dmax = fmax(dmax, dabs_of<R>(f));
        }
      }
    }
    __syncthreads();
    // P2: new corner colours (Fig. 5)
    for (int t = tid; t < kRN; t += kTileThreads) {
      int lx, ly;
      coord(t, &lx, &ly);
      const int id = ly * kRX + lx, x = ri0 + lx, y = rj0 + ly;
      if (lx < 1 || lx > kRX - 2 || x < 0 || x > tnx || y < 0 || y > tny) continue;
      const int c = kb[id];
      int r = c;
      if (x >= 1 && kb[id - 1] != c && hix[id - 1] + ri0 >= x) r ^= 1;
      if (x < tnx && kb[id + 1] != c && hix[id] + ri0 < x) r ^= 1;
      kn[id] = (uint8_t)r;
    }
    __syncthreads();
    // P3: landings on aligned edges (Sec. 2.4)
    for (int t = tid; t < kRN; t += kTileThreads) {
      int lx, ly;
      coord(t, &lx, &ly);
      const int id = ly * kRX + lx, x = ri0 + lx, y = rj0 + ly;
      if (lx < 2 || lx > kRX - 3 || x < 0 || x >= tnx || y < 0 || y > tny) continue;
      R fx[3];
      int src[3];
      int n = 0;
      for (int e = x - 1; e <= x + 1; ++e) {
        const int ie = id + (e - x);
        if (e < 0 || e >= tnx || kb[ie] == kb[ie + 1]) continue;
        if (hix[ie] + ri0 == x) { fx[n] = hfx[ie]; src[n] = e; ++n; }
      }
      const Landing<R> L = choose_landing(n, fx, src, kn[id] ^ kn[id + 1]);
      lpres[id] = (uint8_t)L.present;
      lsrc[id] = L.kept_src < 0 ? kNoSrc : (int8_t)(L.kept_src - x);
      lfx[id] = L.kept_fx;
      if (owned(x, y)) {
        cnt[D_CANCELLED] += L.cancelled;
        cnt[D_INVARIANT] += L.invariant;
        if (L.present) {
          if (AX) out.sV[(long long)x * G.d.P + y] = L.kept_fx;
          else out.sH[(long long)y * G.d.P + x] = L.kept_fx;
        }
      }
    }
    // P4: unaligned edges with candidate chords
    for (int v = tid; v < kNVE; v += kTileThreads) {
      vr[v] = -1;
      vl[v] = -1;
      vp[v] = 0;
    }
    __syncthreads();
    for (int v = tid; v < kNVE; v += kTileThreads) {
      const int k = i0 + v % (kTI + 1), j = j0 + v / (kTI + 1);
      if (k < 1 || k > tnx - 1 || j >= tny) continue;
      bool active = TV.knew(k, j) != TV.knew(k, j + 1);
      for (int c = max(k - 2, 0); c <= k && !active; ++c)
        if (c < tnx && edge_mask(corner_mask(TV, c, j)) != 0) active = true;
      if (active) list[atomicAdd(&s_nlist, 1)] = (uint16_t)v;
    }
    __syncthreads();
    const int nl = s_nlist;
    // P5a: candidates of each listed edge
    for (int w = tid; w < nl; w += kTileThreads) {
      const int v = list[w];
      const int k = i0 + v % (kTI + 1), j = j0 + v / (kTI + 1);
      const bool own = k < i0 + kTI;
      int n = 0;
      for (int c = max(k - 2, 0); c <= k && c < tnx; ++c) {
        int seg[2][2];
        const int ns = cell_segments(TV, c, j, seg);
        for (int t = 0; t < ns; ++t) {
          const int ia = TV.moved(edge_marker(c, j, seg[t][0])).ix;
          const int ib = TV.moved(edge_marker(c, j, seg[t][1])).ix;
          n += (k > min(ia, ib) && k <= max(ia, ib));
        }
      }
      const int base = n ? atomicAdd(&s_ncand, n) : 0;
      ecount[w] = (uint8_t)n;
      if (base + n > kCandCap) {
        // no room: this edge fits and selects in place; its reserved slots
        // below the cap stay empty
        for (int s = base; s < kCandCap; ++s) cand[s].fl = CF_UNUSED;
        ebase[w] = kInPlace;
        const NewV<R> nv = new_unaligned<R>(TV, line_only != 0, k, j, own ? cnt : nullptr);
        vp[v] = (uint8_t)nv.present;
        vs[v] = nv.s;
        vr[v] = (int8_t)nv.vr;
        vl[v] = (int8_t)nv.vl;
        continue;
      }
      ebase[w] = (uint16_t)base;
      int m = 0;
      for (int c = max(k - 2, 0); c <= k && c < tnx; ++c) {
        int seg[2][2];
        const int ns = cell_segments(TV, c, j, seg);
        for (int t = 0; t < ns; ++t) {
          const Mk ma = edge_marker(c, j, seg[t][0]);
          const Mk mb = edge_marker(c, j, seg[t][1]);
          const AP<R> pa = TV.moved(ma), pb = TV.moved(mb);
          if (!(k > min(pa.ix, pb.ix) && k <= max(pa.ix, pb.ix))) continue;
          const bool a_left = pa.ix < k;
          const Mk mA = a_left ? ma : mb, mB = a_left ? mb : ma;
          Cand<R>& C = cand[base + m];
          C.a = pp_of(a_left ? pa : pb, k, j);
          C.b = pp_of(a_left ? pb : pa, k, j);
          uint8_t fl = own ? CF_OWNED : 0;
          int c1i = 0, c1j = 0, c4i = 0, c4j = 0;
          const Mk n1 = beyond(TV, mA, c, j, &c1i, &c1j);
          const Mk n4 = beyond(TV, mB, c, j, &c4i, &c4j);
          if (n1.kind >= 0) {
            C.p1 = pp_of(TV.moved(n1), k, j);
            fl |= CF_P1;
            int oi, oj;
            const Mk nn = beyond(TV, n1, c1i, c1j, &oi, &oj);
            if (nn.kind >= 0) { C.q1 = pp_of(TV.moved(nn), k, j); fl |= CF_Q1; }
          }
          if (n4.kind >= 0) {
            C.p4 = pp_of(TV.moved(n4), k, j);
            fl |= CF_P4;
            int oi, oj;
            const Mk nn = beyond(TV, n4, c4i, c4j, &oi, &oj);
            if (nn.kind >= 0) { C.q4 = pp_of(TV.moved(nn), k, j); fl |= CF_Q4; }
          }
          C.fl = fl;
          const int lr = walk(TV, mB, n4, k);
          const int ll = walk(TV, mA, n1, k - 1);
          C.vr = (int8_t)(lr < 0 ? -1 : !TV.knew(k, lr));
          C.vl = (int8_t)(ll < 0 ? -1 : !TV.knew(k, ll));
          ++m;
        }
      }
    }
    __syncthreads();
    // P5b: circle fits (Sec. 2.2), one candidate per thread
    const int nc = min(s_ncand, kCandCap);
    for (int ci = tid; ci < nc; ci += kTileThreads) {
      Cand<R>& C = cand[ci];
      if (C.fl & CF_UNUSED) continue;
      double ax, ay, bx, by, p1x = 0.0, p1y = 0.0, p4x = 0.0, p4y = 0.0;
      pp_xy(C.a, &ax, &ay);
      pp_xy(C.b, &bx, &by);
      bool h1 = false, h4 = false;
      if (C.fl & CF_P1) {
        pp_xy(C.p1, &p1x, &p1y);
        h1 = true;
        const double ex = p1x - ax, ey = p1y - ay;
        if (ex * ex + ey * ey < kMinSep2) {
          if (C.fl & CF_Q1) pp_xy(C.q1, &p1x, &p1y); else h1 = false;
        }
      }
      if (C.fl & CF_P4) {
        pp_xy(C.p4, &p4x, &p4y);
        h4 = true;
        const double ex = p4x - bx, ey = p4y - by;
        if (ex * ex + ey * ey < kMinSep2) {
          if (C.fl & CF_Q4) pp_xy(C.q4, &p4x, &p4y); else h4 = false;
        }
      }
      double y;
      const int kind = fit_crossing(ax, ay, bx, by, h1, p1x, p1y, h4, p4x, p4y, line_only != 0, &y);
      C.y = y;
      C.kind = (int8_t)kind;
      if (C.fl & CF_OWNED) cnt[kind] += 1;
    }
    __syncthreads();
    // P5c: one marker per edge (Sec. 2.4)
    for (int w = tid; w < nl; w += kTileThreads) {
      if (ebase[w] == kInPlace) continue;
      const int v = list[w];
      const int k = i0 + v % (kTI + 1), j = j0 + v / (kTI + 1);
      const int n = ecount[w], base = ebase[w];
      double cy[6];
      int cvr[6], cvl[6], ord[6];
      for (int t = 0; t < n; ++t) {
        cy[t] = cand[base + t].y;
        cvr[t] = cand[base + t].vr;
        cvl[t] = cand[base + t].vl;
        ord[t] = t;
      }
      const NewV<R> nv = select_candidates<R>(n, cy, cvr, cvl, ord, TV.knew(k, j) ^ TV.knew(k, j + 1),
                                              k < i0 + kTI ? cnt : nullptr);
      vp[v] = (uint8_t)nv.present;
      vs[v] = nv.s;
      vr[v] = (int8_t)nv.vr;
      vl[v] = (int8_t)nv.vl;
    }
    __syncthreads();
  }

  // P6: colour words (one warp per word, one lane per bit), unaligned markers
  const int warp = tid >> 5, lane = tid & 31;
  for (int w = warp; w < 64; w += kTileThreads / 32) {
    // sweep coordinates of this lane's vertex / cell, and the real word
    int i, j, row, word;
    if (AX) { i = i0 + w; j = j0 + lane; row = i; word = j0 >> 5; }
    else { i = i0 + 32 * (w & 1) + lane; j = j0 + (w >> 1); row = j; word = (i0 >> 5) + (w & 1); }
    const bool vin = i <= tnx && j <= tny;
    const unsigned kw = __ballot_sync(0xffffffffu, vin && TV.knew(i, j));
    if (lane == 0 && row <= G.d.ny && word < G.d.kw) out.K[(long long)row * G.d.kw + word] = kw;
    int zc = 0;
    const bool cin = i < tnx && j < tny;
    if (cin) {
      zc = TV.z(i, j);
      const int q = TV.knew(i, j) | (TV.knew(i + 1, j) << 1) | (TV.knew(i + 1, j + 1) << 2) |
                    (TV.knew(i, j + 1) << 3);
      if (q == 5 || q == 10) {
        const int vrow = (j - j0) * (kTI + 1);
        const int a = (i >= 1) ? vr[vrow + (i - i0)] : -1;
        const int b = (i + 1 <= tnx - 1) ? vl[vrow + (i + 1 - i0)] : -1;
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
    const unsigned zw = __ballot_sync(0xffffffffu, cin && zc);
    if (lane == 0 && row < G.d.ny && word < G.d.zw) out.Z[(long long)row * G.d.zw + word] = zw;
  }
  if (busy) {
    for (int v = tid; v < kTI * kTJ; v += kTileThreads) {
      const int k = i0 + v % kTI, j = j0 + v / kTI;
      if (k > tnx || j >= tny) continue;
      const int vi = (j - j0) * (kTI + 1) + (k - i0);
      R val;
      bool put = false;
      if (k >= 1 && k <= tnx - 1) {
        put = vp[vi] != 0;
        val = vs[vi];
      } else if (TV.k(k, j) != TV.k(k, j + 1)) {  // wall marker normal to the sweep stays
        put = true;
        val = G.v(k, j);
      }
      if (put) {
        if (AX) out.sH[(long long)k * G.d.P + j] = val;
        else out.sV[(long long)j * G.d.P + k] = val;
      }
    }
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
__global__ void __launch_bounds__(kTileThreads)
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
__global__ void __launch_bounds__(kTileThreads)
k_sweep_tile_batch(const SweepDesc<R, AX>* __restrict__ descs, const WorkItem* __restrict__ items) {
  const WorkItem it = items[blockIdx.x];
  const SweepDesc<R, AX>& D = descs[it.grid];
  if (!D.active) return;
  sweep_tile<R, AX>(D.G, D.out, D.line_only, D.ctr, D.cfl_bits, D.status, it.tx * kTI, it.ty * kTJ);
}

}  // namespace ebit
