// Fused fields kernel: volume fractions C, height-function curvature kappa,
// the area partial sums and the marker counts of a state (Sec. 2.5), one
// 64x32 tile of cells per block with a 3-cell halo of fractions in shared
// memory for the 7x3 height stencils.
//
// FP64 work is confined to interface cells: a full or empty cell has C equal
// to its corner colour exactly, so full cells are counted as integers and only
// interface fractions enter the double partial sums (in a fixed order per
// thread, then fixed shuffle and block orders), which keeps the sums
// deterministic.
#pragma once
#include "ebit_device.cuh"

namespace ebit {

constexpr int kFX = 64, kFY = 32, kFH = 3;
constexpr int kFRX = kFX + 2 * kFH, kFRY = kFY + 2 * kFH;  // region cells
constexpr int kFVX = kFRX + 1, kFVY = kFRY + 1;            // region vertices
constexpr int kFieldThreads = 256;

__device__ __forceinline__ int kbit_of(const uint32_t* K, const Dims& d, int x, int y) {
  return (__ldg(&K[(long long)y * d.kw + (x >> 5)]) >> (x & 31)) & 1;
}

// Reference-phase area of cell (i,j) in cell units from its corner mask q,
// centre colour and marker fractions; double arithmetic.
template <typename R>
__device__ double fraction_of(int q, int zc, const R* __restrict__ sH, const R* __restrict__ sV,
                              const Dims& d, int i, int j) {
  const int em = edge_mask(q);
  const double s0 = (double)__ldg(&sH[(long long)j * d.P + i]);
  const double s1 = (double)__ldg(&sV[(long long)j * d.P + i + 1]);
  const double s2 = (double)__ldg(&sH[(long long)(j + 1) * d.P + i]);
  const double s3 = (double)__ldg(&sV[(long long)j * d.P + i]);
  auto tri = [&](int c) {
    double a, b;
    switch (c) {
      case 0: a = s3; b = s0; break;
      case 1: a = 1.0 - s0; b = s1; break;
      case 2: a = 1.0 - s1; b = 1.0 - s2; break;
      default: a = s2; b = 1.0 - s3; break;
    }
    return 0.5 * (a * b);
  };
  if (em != 15) {
    const int e1 = __ffs(em) - 1, e2 = 31 - __clz(em);
    const int c0 = q & 1;
    if (e2 - e1 == 2) {
      if (e1 == 0) return c0 ? 0.5 * (s0 + s2) : 0.5 * ((1.0 - s0) + (1.0 - s2));
      return c0 ? 0.5 * (s3 + s1) : 0.5 * ((1.0 - s3) + (1.0 - s1));
    }
    const int c = (e1 == 0 && e2 == 3) ? 0 : e2;
    const double T = tri(c);
    return ((q >> c) & 1) ? T : 1.0 - T;
  }
  double Tsum = 0.0;
  bool first = true;
  for (int c = 0; c < 4; ++c)
    if (((q >> c) & 1) != zc) {
      if (first) { Tsum = tri(c); first = false; } else { Tsum = Tsum + tri(c); }
    }
  return zc == 0 ? Tsum : 1.0 - Tsum;
}

// The tile (bx, by) of one grid; its area partial goes to partial[slot].
template <typename R>
__device__ __forceinline__ void fields_tile(const uint32_t* __restrict__ K,
                                            const uint32_t* __restrict__ Z,
                                            const R* __restrict__ sH, const R* __restrict__ sV,
                                            const Dims& d, R dx, R* C, R* kappa, double* partial,
                                            long long slot, unsigned long long* ctr, int bx, int by) {
  __shared__ uint8_t kb[kFVY * kFVX];
  __shared__ uint8_t zb[kFRY * kFRX];
  __shared__ R cs[kFRY * kFRX];
  __shared__ uint16_t lst[kFRY * kFRX];  // interface cells of the region, in region order
  __shared__ double s_wsum[kFieldThreads / 32];
  __shared__ int s_wcnt[kFieldThreads / 32];
  __shared__ int s_cnt[D_NUSED];
  __shared__ int s_nlist;
  __shared__ unsigned long long s_full;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int i0 = bx * kFX, j0 = by * kFY;
  const int rx0 = i0 - kFH, ry0 = j0 - kFH;
  if (tid < D_NUSED) s_cnt[tid] = 0;
  if (tid == 0) {
    s_full = 0ull;
    s_nlist = 0;
  }
  for (int t = tid; t < kFVX * kFVY; t += kFieldThreads) {
    const int x = rx0 + t % kFVX, y = ry0 + t / kFVX;
    kb[t] = (x >= 0 && x <= d.nx && y >= 0 && y <= d.ny) ? (uint8_t)kbit_of(K, d, x, y) : 0;
  }
  for (int t = tid; t < kFRX * kFRY; t += kFieldThreads) {
    const int x = rx0 + t % kFRX, y = ry0 + t / kFRX;
    zb[t] = (x >= 0 && x < d.nx && y >= 0 && y < d.ny)
                ? (uint8_t)((__ldg(&Z[(long long)y * d.zw + (x >> 5)]) >> (x & 31)) & 1)
                : 0;
  }
  __syncthreads();
  auto qmask = [&](int lx, int ly) {
    const int v = ly * kFVX + lx;
    return kb[v] | (kb[v + 1] << 1) | (kb[v + kFVX + 1] << 2) | (kb[v + kFVX] << 3);
  };
  // fractions: full and empty cells directly; interface cells go to a list
  // built in region order (ballot prefix sums), so that their FP64 work runs
  // on full warps and the area sum has a fixed order
  int full = 0;
  for (int base = 0; base < kFRX * kFRY; base += kFieldThreads) {
    const int t = base + tid;
    bool iface = false;
    if (t < kFRX * kFRY) {
      const int lx = t % kFRX, ly = t / kFRX;
      const int x = rx0 + lx, y = ry0 + ly;
      R c = R(0);
      if (x >= 0 && x < d.nx && y >= 0 && y < d.ny) {
        const int q = qmask(lx, ly);
        if (q == 15) {
          c = R(1);
          full += lx >= kFH && lx < kFH + kFX && ly >= kFH && ly < kFH + kFY;
        } else if (q != 0) {
          iface = true;
        }
      }
      cs[t] = c;
    }
    const unsigned b = __ballot_sync(0xffffffffu, iface);
    if (lane == 0) s_wcnt[warp] = __popc(b);
    __syncthreads();
    int off = s_nlist;
    for (int w = 0; w < warp; ++w) off += s_wcnt[w];
    if (iface) lst[off + __popc(b & ((1u << lane) - 1u))] = (uint16_t)t;
    __syncthreads();
    if (tid == 0) {
      int tot = 0;
      for (int w = 0; w < kFieldThreads / 32; ++w) tot += s_wcnt[w];
      s_nlist += tot;
    }
    __syncthreads();
  }
  const int nlist = s_nlist;
  double acc = 0.0;
  for (int e = tid; e < nlist; e += kFieldThreads) {
    const int t = lst[e];
    const int lx = t % kFRX, ly = t / kFRX;
    const double f = fraction_of(qmask(lx, ly), zb[t], sH, sV, d, rx0 + lx, ry0 + ly);
    cs[t] = (R)f;
    if (lx >= kFH && lx < kFH + kFX && ly >= kFH && ly < kFH + kFY) acc = acc + f;
  }
  __syncthreads();
  int cnt[D_NUSED];
#pragma unroll
  for (int c = 0; c < D_NUSED; ++c) cnt[c] = 0;
  // dense pass: C, marker counts, kappa = NaN away from the interface
  for (int t = tid; t < kFX * kFY; t += kFieldThreads) {
    const int i = i0 + t % kFX, j = j0 + t / kFX;
    if (i > d.nx || j > d.ny) continue;
    const int lx = t % kFX + kFH, ly = t / kFX + kFH;
    const int v = ly * kFVX + lx;
    if (i < d.nx) cnt[D_NH] += kb[v] != kb[v + 1];
    if (j < d.ny) cnt[D_NV] += kb[v] != kb[v + kFVX];
    if (i >= d.nx || j >= d.ny) continue;
    const int ci = ly * kFRX + lx;
    C[(long long)j * d.P + i] = cs[ci];
    const int q = qmask(lx, ly);
    if (q == 0 || q == 15) kappa[(long long)j * d.P + i] = R(NAN);
  }
  // height-function curvature of the tile's interface cells, from the list
  for (int e = tid; e < nlist; e += kFieldThreads) {
    const int ci = lst[e];
    const int lx = ci % kFRX, ly = ci / kFRX;
    if (lx < kFH || lx >= kFH + kFX || ly < kFH || ly >= kFH + kFY) continue;
    const int i = rx0 + lx, j = ry0 + ly;
    const int q = qmask(lx, ly);
    R out = R(NAN);
    {
      int seg[2][2];
      const int ns = segments(q, edge_mask(q) == 15 ? zb[ci] : 0, seg);
      const R px[4] = {__ldg(&sH[(long long)j * d.P + i]), R(1), __ldg(&sH[(long long)(j + 1) * d.P + i]), R(0)};
      const R py[4] = {R(0), __ldg(&sV[(long long)j * d.P + i + 1]), R(1), __ldg(&sV[(long long)j * d.P + i])};
      R ax = R(0), ay = R(0);
      for (int s = 0; s < ns; ++s) {
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
        for (int m = -1; m <= 1; ++m) {
          R a = R(0);
          for (int s = -3; s <= 3; ++s)
            a = a + (ycol ? cs[(ly + s) * kFRX + lx + m] : cs[(ly + m) * kFRX + lx + s]);
          h[m + 1] = a;
          const R lo = ycol ? cs[(ly - 3) * kFRX + lx + m] : cs[(ly + m) * kFRX + lx - 3];
          const R hi = ycol ? cs[(ly + 3) * kFRX + lx + m] : cs[(ly + m) * kFRX + lx + 3];
          orient[m + 1] = (lo == R(1) && hi == R(0)) ? 1 : (lo == R(0) && hi == R(1)) ? -1 : 0;
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
      }
    }
    kappa[(long long)j * d.P + i] = out;
  }
  // area partial: warps holding interface cells reduce in a fixed shuffle
  // order (adding 0.0 from the other lanes changes nothing)
  if (__any_sync(0xffffffffu, acc != 0.0)) {
    for (int o = 16; o > 0; o >>= 1) acc = acc + __shfl_down_sync(0xffffffffu, acc, o);
  } else {
    acc = 0.0;
  }
  if (lane == 0) s_wsum[warp] = acc;
  const int fw = __reduce_add_sync(0xffffffffu, full);
  if (lane == 0 && fw) atomicAdd(&s_full, (unsigned long long)fw);
#pragma unroll
  for (int c = 0; c < D_NUSED; ++c) {
    const int s = __reduce_add_sync(0xffffffffu, cnt[c]);
    if (s != 0 && lane == 0) atomicAdd(&s_cnt[c], s);
  }
  __syncthreads();
  if (tid == 0) {
    double p = 0.0;
    for (int w = 0; w < kFieldThreads / 32; ++w) p = p + s_wsum[w];
    if (s_full) p = p + (double)s_full;
    partial[slot] = p;
  }
  if (tid < D_NUSED && s_cnt[tid] != 0) atomicAdd(&ctr[tid], (unsigned long long)s_cnt[tid]);
}

template <typename R>
__global__ void __launch_bounds__(kFieldThreads)
k_fields_tile(const uint32_t* __restrict__ K, const uint32_t* __restrict__ Z,
              const R* __restrict__ sH, const R* __restrict__ sV, Dims d, R dx, R* C, R* kappa,
              double* partial, unsigned long long* ctr) {
  fields_tile<R>(K, Z, sH, sV, d, dx, C, kappa, partial,
                 (long long)blockIdx.y * gridDim.x + blockIdx.x, ctr, blockIdx.x, blockIdx.y);
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
};

struct FieldItem {
  int grid, tx, ty;
};

template <typename R>
__global__ void __launch_bounds__(kFieldThreads)
k_fields_tile_batch(const FieldDesc<R>* __restrict__ descs, const FieldItem* __restrict__ items) {
  const FieldItem it = items[blockIdx.x];
  const FieldDesc<R>& D = descs[it.grid];
  fields_tile<R>(D.K, D.Z, D.sH, D.sV, D.d, D.dx, D.C, D.kappa, D.partial,
                 (long long)it.ty * D.tiles_x + it.tx, D.ctr, it.tx, it.ty);
}

}  // namespace ebit
