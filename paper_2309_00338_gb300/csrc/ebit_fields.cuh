// Fused fields kernel: volume fractions C, height-function curvature kappa,
// the area (per-tile partial sums, added up by the launch's last tile) and
// the marker counts of a state (Sec. 2.5), one
// 64x32 tile of cells per block with a 3-cell halo for the 7x3 height
// stencils.
//
// Colours are read as bit rows; full, empty and interface cells are word
// operations on them.  FP64 work is confined to interface cells: a full or
// empty cell has C equal to its corner colour exactly, so full cells are
// counted as integers and only interface fractions enter the double partial
// sums.  The interface cells are listed in region order (a deterministic scan)
// and each thread sums its list entries in order, then fixed shuffle and block
// orders, which keeps the sums deterministic.
#pragma once
#include "ebit_device.cuh"

namespace ebit {

constexpr int kFX = 64, kFY = 32, kFH = 3;
constexpr int kFRX = kFX + 2 * kFH, kFRY = kFY + 2 * kFH;  // region cells (70 x 38)
constexpr int kFVX = kFRX + 1, kFVY = kFRY + 1;            // region vertices (71 x 39)
constexpr int kFW = 3;                                     // words per region bit row
// Threads per tile and blocks per SM the kernel is compiled for: eight float
// tiles of 256 threads (32 registers, a few spilled, 12% faster than the five
// that 48 registers allow; 384 or 512 threads per tile were slower); the
// double form's shared memory admits seven at most, and it gains nothing.
template <typename R> __host__ __device__ constexpr int field_threads() { return 256; }
template <typename R> __host__ __device__ constexpr int fields_min_blocks() { return sizeof(R) == 4 ? 8 : 5; }

// Reference-phase area of cell (i,j) in cell units from its corner mask q,
// centre colour and marker fractions; double arithmetic.  The one-minus
// terms are formed once and each case then takes a few operations, so that a
// warp whose cells fall in different cases repeats little FP64 work.
template <typename R>
__device__ double fraction_of(int q, int zc, const R* __restrict__ sH, const R* __restrict__ sV,
                              const Dims& d, int i, int j) {
  const int em = edge_mask(q);
  // exact conversions on the integer pipe
  const long long q0 = (long long)j * d.P + i, q2 = q0 + d.P;  // sH of edges 0, 2; sV of 3, 1 at q0, q0 + 1
  const double s0 = in_range(q0, d.nH()) ? to_d<R>(__ldg(&sH[q0])) : 0.0;
  const double s1 = in_range(q0 + 1, d.nV()) ? to_d<R>(__ldg(&sV[q0 + 1])) : 0.0;
  const double s2 = in_range(q2, d.nH()) ? to_d<R>(__ldg(&sH[q2])) : 0.0;
  const double s3 = in_range(q0, d.nV()) ? to_d<R>(__ldg(&sV[q0])) : 0.0;
  // legs of the triangle cut off at corner c: (s3, s0) (1-s0, s1) (1-s1, 1-s2)
  // (s2, 1-s3); a one-minus is formed only for the legs that take it
  auto tri = [&](int c) {
    const double xa = c == 0 ? s3 : c == 1 ? s0 : c == 2 ? s1 : s2;
    const double xb = c == 0 ? s0 : c == 1 ? s1 : c == 2 ? s2 : s3;
    const double a = (c == 1 || c == 2) ? 1.0 - xa : xa;
    const double b = (c >= 2) ? 1.0 - xb : xb;
    return 0.5 * (a * b);
  };
  if (em != 15) {
    const int e1 = __ffs(em) - 1, e2 = 31 - __clz(em);
    const int c0 = q & 1;
    if (e2 - e1 == 2) {  // opposite edges: a trapezoid
      const double xa = e1 == 0 ? s0 : s3;
      const double xb = e1 == 0 ? s2 : s1;
      const double a = c0 ? xa : 1.0 - xa;
      const double b = c0 ? xb : 1.0 - xb;
      return 0.5 * (a + b);
    }
    const int c = (e1 == 0 && e2 == 3) ? 0 : e2;
    const double T = tri(c);
    return ((q >> c) & 1) ? T : 1.0 - T;
  }
  // four markers: the two corners of the other colour than the centre are cut
  // off (corners 1 and 3 when corner 0 has the centre's colour, else 0 and 2)
  const int ca = ((q & 1) == zc) ? 1 : 0;
  const double Tsum = tri(ca) + tri(ca + 2);
  return zc == 0 ? Tsum : 1.0 - Tsum;
}

__device__ __forceinline__ int fgetb(const uint32_t* w, int lx, int ly) {
  return (w[ly * kFW + (lx >> 5)] >> (lx & 31)) & 1;
}
__device__ __forceinline__ uint32_t fshr1(const uint32_t* w, int ly, int wi) {
  uint32_t v = w[ly * kFW + wi] >> 1;
  if (wi + 1 < kFW) v |= w[ly * kFW + wi + 1] << 31;
  return v;
}

// Dense stores of four consecutive values of a row (16-byte aligned for float).
__device__ __forceinline__ void store4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void store4(double* p, double a, double b, double c, double d) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}

// Where the tiles' area partials are summed: with `done` set, the last tile
// of the launch to finish (counted on *done, which it then resets to 0) adds
// all n partials in a fixed order (thread t takes partials t, t + 256, ...,
// then a tree over the threads), so the area does not depend on which tile
// finishes last, and no separate reduction launch is needed.
struct AreaSum {
  unsigned* done = nullptr;
  long long n = 0;
  double scale = 0.0;
  double* area = nullptr;
};

// The tile (bx, by) of one grid; its area partial goes to partial[slot].
// With ghf_list, the interface cells left without a 7x3 stencil are
// appended to it (ghf_count, zeroed before the launch, counts them): one
// global atomic per tile reserves its slice.
template <typename R>
__device__ __forceinline__ void fields_tile(const uint32_t* __restrict__ K,
                                            const uint32_t* __restrict__ Z,
                                            const R* __restrict__ sH, const R* __restrict__ sV,
                                            const Dims& d, R dx, R* C, R* kappa, double* partial,
                                            long long slot, unsigned long long* ctr, int bx, int by,
                                            int* ghf_list = nullptr, unsigned* ghf_count = nullptr,
                                            AreaSum sum = AreaSum()) {
  constexpr int kFieldThreads = field_threads<R>();
  __shared__ uint32_t kw[kFVY * kFW];  // vertex colours
  __shared__ uint32_t zw[kFRY * kFW];  // centre colours
  __shared__ uint32_t fw[kFRY * kFW];  // full cells
  __shared__ uint32_t iw[kFRY * kFW];  // interface cells
  __shared__ R cs[kFRY * kFRX];        // fractions of the region
  __shared__ uint16_t lst[kFRY * kFRX];
  __shared__ int s_woff[kFieldThreads / 32];
  __shared__ double s_wsum[kFieldThreads / 32];
  __shared__ int s_cnt[D_NUSED];
  __shared__ unsigned long long s_full;
  __shared__ unsigned s_nghf, s_ghf_base;
  __shared__ int s_last;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = bx * kFX, j0 = by * kFY;
  const int rx0 = i0 - kFH, ry0 = j0 - kFH;
  if (tid < D_NUSED) s_cnt[tid] = 0;
  if (tid == 0) {
    s_full = 0ull;
    s_nghf = 0u;
  }
  // region columns / rows inside the grid
  const int vx0 = max(0, -rx0), vx1 = min(kFVX - 1, d.nx - rx0);  // vertices
  const int cx1 = min(kFRX - 1, d.nx - 1 - rx0);                  // cells
  const int vy0 = max(0, -ry0), vy1 = min(kFVY - 1, d.ny - ry0);
  const int cy1 = min(kFRY - 1, d.ny - 1 - ry0);
  int cnt[D_NUSED];
#pragma unroll
  for (int c = 0; c < D_NUSED; ++c) cnt[c] = 0;

  // colour bits
  for (int t = tid; t < (kFVY + kFRY) * kFW; t += kFieldThreads) {
    const bool zpl = t >= kFVY * kFW;
    const int u = zpl ? t - kFVY * kFW : t;
    const int ly = u / kFW, wi = u % kFW, y = ry0 + ly, x0 = rx0 + 32 * wi;
    uint32_t v = 0u;
    if (!zpl && ly >= vy0 && ly <= vy1)
      v = row_bits(K + (long long)y * d.kw, d.kw, x0) & span_mask(wi, vx0, vx1);
    if (zpl && ly >= vy0 && ly <= cy1)
      v = row_bits(Z + (long long)y * d.zw, d.zw, x0) & span_mask(wi, vx0, cx1);
    (zpl ? zw : kw)[u] = v;
  }
  __syncthreads();

  // full / interface cells; the tile's full cells and markers are counted
  int full = 0;
  for (int t = tid; t < kFRY * kFW; t += kFieldThreads) {
    const int ly = t / kFW, wi = t % kFW;
    uint32_t f = 0u, ic = 0u;
    if (ly >= vy0 && ly <= cy1) {
      const uint32_t a = kw[t], a1 = fshr1(kw, ly, wi), b = kw[t + kFW], b1 = fshr1(kw, ly + 1, wi);
      const uint32_t cm = span_mask(wi, vx0, cx1);
      f = a & a1 & b & b1 & cm;
      ic = (a | a1 | b | b1) & ~f & cm;
    }
    fw[t] = f;
    iw[t] = ic;
    if (ly >= kFH && ly < kFH + kFY) {
      const uint32_t tile = span_mask(wi, kFH, kFH + kFX - 1);
      full += __popc(f & tile);
      // markers on the tile's vertices' right and upper edges
      if (ly <= vy1) {
        const uint32_t a = kw[t];
        cnt[D_NH] += __popc((a ^ fshr1(kw, ly, wi)) & tile & span_mask(wi, vx0, cx1));
        if (ly + 1 <= vy1) cnt[D_NV] += __popc((a ^ kw[t + kFW]) & tile & span_mask(wi, vx0, vx1));
      }
    }
  }
  {
    const int fsum = __reduce_add_sync(0xffffffffu, full);
    if (lane == 0 && fsum) atomicAdd(&s_full, (unsigned long long)fsum);
  }
  __syncthreads();

  // interface list in region order: per-warp scans of the word counts
  constexpr int kWords = kFRY * kFW;  // 114
  int pos = 0, n = 0;
  uint32_t mybits = 0u;
  if (warp < (kWords + 31) / 32) {
    const int t = warp * 32 + lane;
    mybits = t < kWords ? iw[t] : 0u;
    n = __popc(mybits);
    int incl = n;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int v = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += v;
    }
    pos = incl - n;
    if (lane == 31) s_woff[warp] = incl;
  }
  // fractions of full and empty cells, a warp per region row
  for (int ly = warp; ly < kFRY; ly += kFieldThreads / 32) {
#pragma unroll
    for (int w = 0; w < kFW; ++w) {
      const int lx = 32 * w + lane;
      const uint32_t f = fw[ly * kFW + w], ic = iw[ly * kFW + w];
      if (lx < kFRX && !((ic >> lane) & 1u)) cs[ly * kFRX + lx] = ((f >> lane) & 1u) ? R(1) : R(0);
    }
  }
  __syncthreads();
  if (warp < (kWords + 31) / 32) {
    for (int w = 0; w < warp; ++w) pos += s_woff[w];
    const int t = warp * 32 + lane;
    const int row0 = (t / kFW) * kFRX + 32 * (t % kFW);
    while (mybits) {
      const int b = __ffs(mybits) - 1;
      mybits &= mybits - 1;
      lst[pos++] = (uint16_t)(row0 + b);
    }
  }
  int nlist = 0;
#pragma unroll
  for (int w = 0; w < (kWords + 31) / 32; ++w) nlist += s_woff[w];
  __syncthreads();

  // interface fractions (FP64 on full warps) and the tile's area
  double acc = 0.0;
  for (int e = tid; e < nlist; e += kFieldThreads) {
    const int t = lst[e];
    const int lx = t % kFRX, ly = t / kFRX;
    const int q = fgetb(kw, lx, ly) | (fgetb(kw, lx + 1, ly) << 1) |
                  (fgetb(kw, lx + 1, ly + 1) << 2) | (fgetb(kw, lx, ly + 1) << 3);
    const double f = fraction_of(q, fgetb(zw, lx, ly), sH, sV, d, rx0 + lx, ry0 + ly);
    cs[t] = (R)f;
    if (lx >= kFH && lx < kFH + kFX && ly >= kFH && ly < kFH + kFY) acc = acc + f;
  }
  // area partial: warps holding interface cells reduce in a fixed shuffle
  // order (adding 0.0 from the other lanes changes nothing)
  if (__any_sync(0xffffffffu, !d_eq0(acc))) {
    for (int o = 16; o > 0; o >>= 1) acc = acc + __shfl_down_sync(0xffffffffu, acc, o);
  } else {
    acc = 0.0;
  }
  if (lane == 0) s_wsum[warp] = acc;
  __syncthreads();
  // the tile's partial, and its count towards the launch's last tile, by the
  // last thread: it has no global stores in flight to fence, and it rarely
  // has curvature work, so the fence and the counter's round trip overlap
  // the other threads' curvature
  if (tid == kFieldThreads - 1) {
    double p = 0.0;
    for (int w = 0; w < kFieldThreads / 32; ++w) p = p + s_wsum[w];
    if (s_full) p = p + (double)s_full;
    partial[slot] = p;
    s_last = 0;
    if (sum.done) {
      __threadfence();  // the partial is visible before the count says so
      s_last = atomicAdd(sum.done, 1u) == (unsigned)(sum.n - 1);
    }
  }

  // height-function curvature of the tile's interface cells
  for (int e = tid; e < nlist; e += kFieldThreads) {
    const int ci = lst[e];
    const int lx = ci % kFRX, ly = ci / kFRX;
    if (lx < kFH || lx >= kFH + kFX || ly < kFH || ly >= kFH + kFY) continue;
    const int i = rx0 + lx, j = ry0 + ly;
    const int q = fgetb(kw, lx, ly) | (fgetb(kw, lx + 1, ly) << 1) |
                  (fgetb(kw, lx + 1, ly + 1) << 2) | (fgetb(kw, lx, ly + 1) << 3);
    R out = R(NAN);
    int seg[2][2];
    const int ns = segments(q, edge_mask(q) == 15 ? fgetb(zw, lx, ly) : 0, seg);
    const long long q0 = (long long)j * d.P + i, q2 = q0 + d.P;
    const R px[4] = {in_range(q0, d.nH()) ? __ldg(&sH[q0]) : R(0), R(1),
                     in_range(q2, d.nH()) ? __ldg(&sH[q2]) : R(0), R(0)};
    const R py[4] = {R(0), in_range(q0 + 1, d.nV()) ? __ldg(&sV[q0 + 1]) : R(0), R(1),
                     in_range(q0, d.nV()) ? __ldg(&sV[q0]) : R(0)};
    R ax = R(0), ay = R(0);
#pragma unroll
    for (int s = 0; s < 2; ++s) {
      if (s >= ns) break;
      const int a = seg[s][0], b = seg[s][1];
      ax = ax + fabs(px[b] - px[a]);
      ay = ay + fabs(py[b] - py[a]);
    }
    const bool ycol = ax >= ay;
    const bool inside = ycol ? (i - 1 >= 0 && i + 1 <= d.nx - 1 && j - 3 >= 0 && j + 3 <= d.ny - 1)
                             : (j - 1 >= 0 && j + 1 <= d.ny - 1 && i - 3 >= 0 && i + 3 <= d.nx - 1);
    bool valid = inside;
    R h[3];
    if (inside) {
      int orient[3];
#pragma unroll
      for (int m = -1; m <= 1; ++m) {
        R a = R(0);
#pragma unroll
        for (int s = -3; s <= 3; ++s)
          a = a + (ycol ? cs[(ly + s) * kFRX + lx + m] : cs[(ly + m) * kFRX + lx + s]);
        h[m + 1] = a;
        const R lo = ycol ? cs[(ly - 3) * kFRX + lx + m] : cs[(ly + m) * kFRX + lx - 3];
        const R hi = ycol ? cs[(ly + 3) * kFRX + lx + m] : cs[(ly + m) * kFRX + lx + 3];
        orient[m + 1] = (one_bits(lo) && zero_bits(hi)) ? 1 : (zero_bits(lo) && one_bits(hi)) ? -1 : 0;
      }
      valid = orient[0] != 0 && orient[0] == orient[1] && orient[1] == orient[2];
    }
    if (valid) {
      const R hp = (h[2] - h[0]) * R(0.5);
      const R hpp = (h[2] - h[1]) - (h[1] - h[0]);
      const R qv = R(1) + hp * hp;
      const R den = dx * (qv * sqrt(qv));
      out = -hpp / den;
    } else {
      cnt[D_HF_INVALID] += 1;
      if (ghf_list) {  // flag the entry for the generalised fallbacks
        lst[e] = (uint16_t)(ci | 0x8000);
        atomicAdd(&s_nghf, 1u);
      }
    }
    if (in_range((long long)j * d.P + i, d.nV())) kappa[(long long)j * d.P + i] = out;
  }
  // dense outputs: C everywhere, kappa = NaN away from the interface (the
  // interface cells' kappa is written above)
  const bool vec = ((reinterpret_cast<uintptr_t>(C) | reinterpret_cast<uintptr_t>(kappa)) & 15) == 0;
  for (int g = tid; g < kFX * kFY / 4; g += kFieldThreads) {
    const int lx0 = (g % (kFX / 4)) * 4, ly0 = g / (kFX / 4);
    const int i = i0 + lx0, j = j0 + ly0;
    if (j >= d.ny || i >= d.nx) continue;
    const int lx = lx0 + kFH, ly = ly0 + kFH;
    const R* c = &cs[ly * kFRX + lx];
    const uint32_t ib = (iw[ly * kFW + (lx >> 5)] >> (lx & 31)) |
                        ((lx & 31) > 28 ? iw[ly * kFW + (lx >> 5) + 1] << (32 - (lx & 31)) : 0u);
    if (!in_range((long long)j * d.P + min(i + 3, d.nx - 1), d.nV())) continue;  // this group's last cell
    R* Cp = C + (long long)j * d.P + i;
    R* Kp = kappa + (long long)j * d.P + i;
    if (vec && i + 3 < d.nx) {
      store4(Cp, c[0], c[1], c[2], c[3]);
      if (!(ib & 15u)) store4(Kp, R(NAN), R(NAN), R(NAN), R(NAN));
      else
        for (int m = 0; m < 4; ++m)
          if (!((ib >> m) & 1u)) Kp[m] = R(NAN);
    } else {
      for (int m = 0; m < 4 && i + m < d.nx; ++m) {
        Cp[m] = c[m];
        if (!((ib >> m) & 1u)) Kp[m] = R(NAN);
      }
    }
  }
  // the counters this kernel keeps (markers, cells without a height stencil)
  for (const int c : {(int)D_NH, (int)D_NV, (int)D_HF_INVALID}) {
    const int s = __reduce_add_sync(0xffffffffu, cnt[c]);
    if (s != 0 && lane == 0) atomicAdd(&s_cnt[c], s);
  }
  __syncthreads();
  if (tid < D_NUSED && s_cnt[tid] != 0) atomicAdd(&ctr[tid], (unsigned long long)s_cnt[tid]);
  if (ghf_list) {
    const unsigned nflag = s_nghf;  // final: its atomics precede the last barrier
    if (nflag != 0u) {              // the same in every thread
      __syncthreads();              // every thread has read it
      if (tid == 0) {
        s_ghf_base = atomicAdd(ghf_count, nflag);
        s_nghf = 0u;
      }
      __syncthreads();
      for (int e = tid; e < nlist; e += kFieldThreads) {
        const int ci = lst[e];
        if (!(ci & 0x8000)) continue;
        const int t = ci & 0x7fff;
        const int i = rx0 + t % kFRX, j = ry0 + t / kFRX;
        ghf_list[s_ghf_base + atomicAdd(&s_nghf, 1u)] = j * d.nx + i;
      }
    }
  }
  __syncthreads();
  if (s_last) {  // the same in every thread of the block: set before a barrier
    static_assert(field_threads<R>() == 256, "the fixed area order assumes 256 threads");
    __shared__ double red[256];
    __threadfence();
    double a = 0.0;
    long long b = tid;
    for (; b + 7 * 256 < sum.n; b += 8 * 256) {  // eight loads in flight, added in order
      double v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) v[u] = __ldcg(&partial[b + u * 256]);
#pragma unroll
      for (int u = 0; u < 8; ++u) a = a + v[u];
    }
    for (; b < sum.n; b += 256) a = a + __ldcg(&partial[b]);
    red[tid] = a;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
      if (tid < s) red[tid] = red[tid] + red[tid + s];
      __syncthreads();
    }
    if (tid == 0) {
      *sum.area = red[0] * sum.scale;
      *sum.done = 0u;  // ready for the next launch (stream order)
    }
  }
}

template <typename R>
__global__ void __launch_bounds__(field_threads<R>(), fields_min_blocks<R>())
k_fields_tile(const uint32_t* __restrict__ K, const uint32_t* __restrict__ Z,
              const R* __restrict__ sH, const R* __restrict__ sV, Dims d, R dx, R* C, R* kappa,
              double* partial, unsigned long long* ctr, int* ghf_list, unsigned* ghf_count,
              AreaSum sum) {
  fields_tile<R>(K, Z, sH, sV, d, dx, C, kappa, partial,
                 (long long)blockIdx.y * gridDim.x + blockIdx.x, ctr, blockIdx.x, blockIdx.y, ghf_list,
                 ghf_count, sum);
}

// Many grids in one launch (work items: grid, tile).
template <typename R>
struct FieldDesc {
  const uint32_t* K;
  const uint32_t* Z;
  const R* sH;
  const R* sV;
  Dims d;
  R dx;
  R* C;
  R* kappa;
  double* partial;
  unsigned long long* ctr;
  int tiles_x;
  int* ghf_list;         // EBIT_CURV_GHF grids: their list of cells without a 7x3 stencil
  unsigned* ghf_count;   // (null otherwise)
};

struct FieldItem {
  int grid, tx, ty;
};

template <typename R>
__global__ void __launch_bounds__(field_threads<R>(), fields_min_blocks<R>())
k_fields_tile_batch(const FieldDesc<R>* __restrict__ descs, const FieldItem* __restrict__ items) {
  const FieldItem it = items[blockIdx.x];
  const FieldDesc<R>& D = descs[it.grid];
  fields_tile<R>(D.K, D.Z, D.sH, D.sV, D.d, D.dx, D.C, D.kappa, D.partial,
                 (long long)it.ty * D.tiles_x + it.tx, D.ctr, it.tx, it.ty, D.ghf_list, D.ghf_count);
}

}  // namespace ebit
