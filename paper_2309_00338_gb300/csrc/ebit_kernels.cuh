// Kernels of the EBIT step besides the tiled sweep and the fused fields: the
// thread-per-vertex gather sweep (two passes, kept for differential testing),
// the area sum, initialisation and state I/O.
// Threads map to vertices of the real grid: a warp is 32 consecutive x of one
// row, aligned to 32, so colour bits pack into 32-bit words with a ballot.
#pragma once
#include "ebit_device.cuh"

namespace ebit {

constexpr int kBlockY = 8;  // blocks are 32 x kBlockY threads

__device__ __forceinline__ void flush_counters(const int* cnt, unsigned long long* ctr) {
#pragma unroll
  for (int c = 0; c < D_NUSED; ++c) {
    const int v = __reduce_add_sync(0xffffffffu, cnt[c]);
    if (v != 0 && (threadIdx.x & 31) == 0) atomicAdd(&ctr[c], (unsigned long long)v);
  }
}

__device__ __forceinline__ void raise_status(int* status, const int* cnt) {
  if (cnt[D_CFL]) atomicOr(status, ST_CFL);
  if (cnt[D_INVARIANT]) atomicOr(status, ST_INVARIANT);
}

// Pass 1 of a sweep.  Thread at real vertex (x,y) = sweep vertex (i,j):
//   new corner colour of vertex (i,j), new aligned marker on edge (i,j),
//   new unaligned marker on edge (i,j) with the centre-rule verdicts it gives
//   to the cells right (from_left) and left (from_right) of it.
template <typename R, int AX>
__global__ void __launch_bounds__(32 * kBlockY)
k_sweep(GView<R, AX> S, Buf<R> out, int line_only, int8_t* from_left, int8_t* from_right,
        unsigned long long* ctr, unsigned long long* cfl_bits, int* status) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.y;
  const Dims& d = S.d;
  const bool in = x <= d.nx && y <= d.ny;
  const int i = AX ? y : x, j = AX ? x : y;
  const int tnx = S.tnx(), tny = S.tny();
  int cnt[D_NUSED];
#pragma unroll
  for (int c = 0; c < D_NUSED; ++c) cnt[c] = 0;
  double dmax = 0.0;
  int kb = 0;
  if (in) {
    kb = S.k(i, j);
    // Anything to do?  Only if a colour changes along vertex rows j, j+1
    // within columns i-2..i+2 (all markers this thread looks at live there).
    bool busy = false;
    const int c0 = max(i - 2, 0), c1 = min(i + 2, tnx);
    const int ref = S.k(c0, j);
    for (int r = j; r <= min(j + 1, tny) && !busy; ++r)
      for (int c = c0; c <= c1; ++c)
        if (S.k(c, r) != ref) { busy = true; break; }
    if (busy) {
      kb = S.knew(i, j);
      if (i < tnx) {
        if (S.k(i, j) != S.k(i + 1, j)) {
          Flags f;
          S.advect(Mk{0, i, j}, f);
          cnt[D_CFL] += f.cfl;
          cnt[D_WALL_CLAMP] += f.clamp;
          dmax = fmax(dmax, (double)dabs_of<R>(f));
        }
        const Landing<R> L = S.landing(i, j);
        cnt[D_CANCELLED] += L.cancelled;
        cnt[D_INVARIANT] += L.invariant;
        if (L.present) {
          if (AX) out.sV[(long long)i * d.P + j] = L.kept_fx;
          else out.sH[(long long)j * d.P + i] = L.kept_fx;
        }
      }
      if (j < tny) {
        const bool had = S.k(i, j) != S.k(i, j + 1);
        if (i >= 1 && i <= tnx - 1) {
          if (had) {
            Flags f;
            S.advect(Mk{1, i, j}, f);
            cnt[D_CFL] += f.cfl;
            dmax = fmax(dmax, (double)dabs_of<R>(f));
          }
          const NewV<R> nv = new_unaligned<R>(S, line_only != 0, i, j, cnt);
          if (nv.present) {
            if (AX) out.sH[(long long)i * d.P + j] = nv.s;
            else out.sV[(long long)j * d.P + i] = nv.s;
          }
          // verdict slots are indexed by real cell
          const long long cr = AX ? (long long)i * d.nx + j : (long long)j * d.nx + i;
          const long long cl = AX ? (long long)(i - 1) * d.nx + j : (long long)j * d.nx + (i - 1);
          from_left[cr] = (int8_t)nv.vr;
          from_right[cl] = (int8_t)nv.vl;
        } else if (had) {  // wall marker normal to the sweep stays
          if (AX) out.sH[(long long)i * d.P + j] = S.v(i, j);
          else out.sV[(long long)j * d.P + i] = S.v(i, j);
        }
      }
    }
  }
  const unsigned word = __ballot_sync(0xffffffffu, in && kb);
  if (threadIdx.x == 0 && y <= d.ny && x <= d.nx) out.K[(long long)y * d.kw + (x >> 5)] = word;
  flush_counters(cnt, ctr);
  raise_status(status, cnt);
  if (dmax > 0.0) atomicMax(cfl_bits, (unsigned long long)__double_as_longlong(dmax));
}

// Pass 2 of a sweep: centre colour vertices of cells with four markers after
// the sweep (Sec. 2.3); the verdict from the cell's left (bottom) edge wins.
template <typename R, int AX>
__global__ void __launch_bounds__(32 * kBlockY)
k_centre(GView<R, AX> Snew, const uint32_t* __restrict__ Zold, uint32_t* Zout,
         const int8_t* __restrict__ from_left, const int8_t* __restrict__ from_right,
         unsigned long long* ctr) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.y;
  const Dims& d = Snew.d;
  const bool in = x < d.nx && y < d.ny;
  int cnt[D_NUSED];
#pragma unroll
  for (int c = 0; c < D_NUSED; ++c) cnt[c] = 0;
  int zb = 0;
  if (in) {
    const long long cell = (long long)y * d.nx + x;
    zb = (__ldg(&Zold[(long long)y * d.zw + (x >> 5)]) >> (x & 31)) & 1;
    const int i = AX ? y : x, j = AX ? x : y;
    const int q = corner_mask(Snew, i, j);
    if (q == 5 || q == 10) {
      const int a = (i >= 1) ? from_left[cell] : -1;
      const int b = (i + 1 <= Snew.tnx() - 1) ? from_right[cell] : -1;
      if (a >= 0) {
        zb = a;
        cnt[D_ZSET] += 1;
        if (b >= 0 && b != a) cnt[D_ZCONFLICT] += 1;
      } else if (b >= 0) {
        zb = b;
        cnt[D_ZSET] += 1;
      }
    }
  }
  const unsigned word = __ballot_sync(0xffffffffu, in && zb);
  if (threadIdx.x == 0 && y < d.ny && x < d.nx) Zout[(long long)y * d.zw + (x >> 5)] = word;
  flush_counters(cnt, ctr);
}

__device__ __forceinline__ int kbit(const uint32_t* K, const Dims& d, int x, int y) {
  return (__ldg(&K[(long long)y * d.kw + (x >> 5)]) >> (x & 31)) & 1;
}

// Sum of the per-block partials in a fixed order (one block of kAreaThreads;
// a thread adds every kAreaThreads-th partial, then a tree over the threads).
// 256 threads: 1024 took 12.6 us at 4096^2 against 10.5.
constexpr int kAreaThreads = 256;
__global__ void __launch_bounds__(kAreaThreads)
k_area(const double* __restrict__ partial, long long n, double scale, double* area) {
  __shared__ double red[kAreaThreads];
  double acc = 0.0;
  for (long long b = threadIdx.x; b < n; b += kAreaThreads) acc = acc + partial[b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = kAreaThreads / 2; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *area = red[0] * scale;
}

// ---------------------------------------------------------------------------
// Initialisation (Sec. 3.2).
// ---------------------------------------------------------------------------
struct SceneDev {
  const double* circ;   // 3 per circle: xc, yc, r
  int ncircles;
  int has_curve;
  double y0;
  int nmodes;
  const double* amp;
  const double* phase;
  int nlines;  // half-planes, each toggling where la x + lb y <= lc
  double la[4], lb[4], lc[4];
  const double* notch;  // 4 per notch: x0, x1, y0, y1
  int nnotches;
};

__device__ double curve_h(const SceneDev& sc, double x) {
  double acc = sc.y0;
  for (int k = 1; k <= sc.nmodes; ++k) {
    const double arg = (6.283185307179586 * (double)k) * x + sc.phase[k - 1];
    acc = acc + sc.amp[k - 1] * cos(arg);
  }
  return acc;
}

__device__ __forceinline__ bool in_circle(const SceneDev& sc, int c, double x, double y) {
  const double ddx = x - sc.circ[3 * c], ddy = y - sc.circ[3 * c + 1];
  const double r = sc.circ[3 * c + 2];
  return ddx * ddx + ddy * ddy <= r * r;
}
__device__ __forceinline__ bool in_line(const SceneDev& sc, int l, double x, double y) {
  return sc.la[l] * x + sc.lb[l] * y <= sc.lc[l];
}
__device__ __forceinline__ bool in_notch(const SceneDev& sc, double x, double y) {
  for (int b = 0; b < sc.nnotches; ++b) {
    const double* q = sc.notch + 4 * b;
    if (x >= q[0] && x <= q[1] && y >= q[2] && y <= q[3]) return true;
  }
  return false;
}
// The scene's phase at a point: curve, half-planes and circles toggle it,
// then the notches cut it out.
__device__ bool scene_inside(const SceneDev& sc, double x, double y) {
  bool p = false;
  if (sc.has_curve) p ^= y <= curve_h(sc, x);
  for (int l = 0; l < sc.nlines; ++l) p ^= in_line(sc, l, x, y);
  for (int c = 0; c < sc.ncircles; ++c) p ^= in_circle(sc, c, x, y);
  return p && !in_notch(sc, x, y);
}
// The first half-plane whose inside test differs at the two ends of an edge, or -1.
__device__ __forceinline__ int line_crossing(const SceneDev& sc, double xa, double ya, double xb,
                                             double yb) {
  for (int l = 0; l < sc.nlines; ++l)
    if (in_line(sc, l, xa, ya) != in_line(sc, l, xb, yb)) return l;
  return -1;
}
// Does the axis-aligned edge (xa, ya)-(xb, yb), xa <= xb, ya <= yb, touch a notch?
__device__ __forceinline__ bool touches_notch(const SceneDev& sc, double xa, double ya, double xb,
                                              double yb) {
  for (int b = 0; b < sc.nnotches; ++b) {
    const double* q = sc.notch + 4 * b;
    if (xb >= q[0] && xa <= q[1] && yb >= q[2] && ya <= q[3]) return true;
  }
  return false;
}

// Curve heights at the vertex columns (hv[i], x = i dx) and at the cell-centre
// columns (hv[nx + 1 + i], x = (i + 0.5) dx): the curve depends on x only, so
// each column's height is evaluated once.
__global__ void k_curve_cols(SceneDev sc, int nx, double dx, double* hv) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i <= nx) hv[i] = curve_h(sc, i * dx);
  if (i < nx) hv[nx + 1 + i] = curve_h(sc, (i + 0.5) * dx);
}

// Base phase of vertices (K) and cell centres (Z) from the curve and line.
__global__ void __launch_bounds__(32 * kBlockY)
k_init_base(SceneDev sc, Dims d, double dx, const double* hv, uint32_t* K, uint32_t* Z) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.y;
  int pk = 0, pz = 0;
  if (x <= d.nx && y <= d.ny) {
    if (sc.has_curve) pk ^= (y * dx) <= hv[x];
    for (int l = 0; l < sc.nlines; ++l) pk ^= in_line(sc, l, x * dx, y * dx);
  }
  if (x < d.nx && y < d.ny) {
    const double cx = (x + 0.5) * dx, cy = (y + 0.5) * dx;
    if (sc.has_curve) pz ^= cy <= hv[d.nx + 1 + x];
    for (int l = 0; l < sc.nlines; ++l) pz ^= in_line(sc, l, cx, cy);
  }
  const unsigned wk = __ballot_sync(0xffffffffu, (x <= d.nx && y <= d.ny) && pk);
  const unsigned wz = __ballot_sync(0xffffffffu, (x < d.nx && y < d.ny) && pz);
  if (threadIdx.x == 0 && y <= d.ny && x <= d.nx) K[(long long)y * d.kw + (x >> 5)] = wk;
  if (threadIdx.x == 0 && y < d.ny && x < d.nx) Z[(long long)y * d.zw + (x >> 5)] = wz;
}

// Notches: vertices and cell centres inside a box leave the reference phase
// (after the curve, line and circles have set it).
__global__ void __launch_bounds__(32 * kBlockY)
k_init_notch(SceneDev sc, Dims d, double dx, uint32_t* K, uint32_t* Z) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.y;
  const bool vk = x <= d.nx && y <= d.ny && in_notch(sc, x * dx, y * dx);
  const bool vz = x < d.nx && y < d.ny && in_notch(sc, (x + 0.5) * dx, (y + 0.5) * dx);
  const unsigned mk = __ballot_sync(0xffffffffu, vk);
  const unsigned mz = __ballot_sync(0xffffffffu, vz);
  if (threadIdx.x == 0 && mk) K[(long long)y * d.kw + (x >> 5)] &= ~mk;
  if (threadIdx.x == 0 && mz) Z[(long long)y * d.zw + (x >> 5)] &= ~mz;
}

__device__ __forceinline__ void circle_box(const SceneDev& sc, int c, const Dims& d, double dx,
                                           int* i0, int* i1, int* j0, int* j1) {
  const double xc = sc.circ[3 * c], yc = sc.circ[3 * c + 1], r = sc.circ[3 * c + 2];
  *i0 = max(0, (int)floor((xc - r) / dx) - 1);
  *i1 = min(d.nx, (int)ceil((xc + r) / dx) + 1);
  *j0 = max(0, (int)floor((yc - r) / dx) - 1);
  *j1 = min(d.ny, (int)ceil((yc + r) / dx) + 1);
}

// One block per circle: toggle the vertices and centres inside it.
__global__ void k_init_circles(SceneDev sc, Dims d, double dx, uint32_t* K, uint32_t* Z) {
  const int c = blockIdx.x;
  int i0, i1, j0, j1;
  circle_box(sc, c, d, dx, &i0, &i1, &j0, &j1);
  const int w = i1 - i0 + 1;
  const long long n = (long long)w * (j1 - j0 + 1);
  for (long long t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = i0 + (int)(t % w), j = j0 + (int)(t / w);
    if (in_circle(sc, c, i * dx, j * dx)) atomicXor(&K[(long long)j * d.kw + (i >> 5)], 1u << (i & 31));
    if (i < d.nx && j < d.ny && in_circle(sc, c, (i + 0.5) * dx, (j + 0.5) * dx))
      atomicXor(&Z[(long long)j * d.zw + (i >> 5)], 1u << (i & 31));
  }
}

// One block per circle: lowest circle index whose own inside test differs at
// the two ends of an edge.
__global__ void k_init_owner(SceneDev sc, Dims d, double dx, int* ownH, int* ownV) {
  const int c = blockIdx.x;
  int i0, i1, j0, j1;
  circle_box(sc, c, d, dx, &i0, &i1, &j0, &j1);
  const int w = i1 - i0 + 1;
  const long long n = (long long)w * (j1 - j0 + 1);
  for (long long t = threadIdx.x; t < n; t += blockDim.x) {
    const int i = i0 + (int)(t % w), j = j0 + (int)(t / w);
    const bool here = in_circle(sc, c, i * dx, j * dx);
    if (i < d.nx && here != in_circle(sc, c, (i + 1) * dx, j * dx))
      atomicMin(&ownH[(long long)j * d.P + i], c);
    if (j < d.ny && here != in_circle(sc, c, i * dx, (j + 1) * dx))
      atomicMin(&ownV[(long long)j * d.P + i], c);
  }
}

template <typename R>
__device__ __forceinline__ R finish_fraction(double s) {
  if (!(s >= 0.0)) s = 0.0;
  if (s >= 1.0) s = below_one<double>();
  R r = (R)s;
  if (r >= R(1)) r = below_one<R>();
  return r;
}

// Marker fraction of every edge whose end colours differ.
template <typename R>
__global__ void __launch_bounds__(32 * kBlockY)
k_init_roots(SceneDev sc, Dims d, double dx, const uint32_t* __restrict__ K,
             const double* __restrict__ hv, const int* __restrict__ ownH,
             const int* __restrict__ ownV, R* sH, R* sV) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.y;
  if (x > d.nx || y > d.ny) return;
  const double xi = x * dx, yj = y * dx;
  if (x < d.nx && kbit(K, d, x, y) != kbit(K, d, x + 1, y)) {
    double s = 0.5;
    if (sc.nnotches && touches_notch(sc, xi, yj, (x + 1) * dx, yj)) {
      // bisection on the scene's phase along the edge
      const bool side0 = scene_inside(sc, xi, yj);
      double lo = 0.0, hi = 1.0;
      for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (scene_inside(sc, xi + mid * dx, yj) == side0) lo = mid; else hi = mid;
      }
      s = 0.5 * (lo + hi);
    } else if (sc.has_curve && ((yj <= hv[x]) != (yj <= hv[x + 1]))) {
      const bool side0 = yj <= hv[x];
      double lo = 0.0, hi = 1.0;
      for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if ((yj <= curve_h(sc, xi + mid * dx)) == side0) lo = mid; else hi = mid;
      }
      s = 0.5 * (lo + hi);
    } else if (const int l = line_crossing(sc, xi, yj, (x + 1) * dx, yj); l >= 0) {
      const double xr = (sc.lc[l] - sc.lb[l] * yj) / sc.la[l];
      s = (xr - xi) / dx;
    } else {
      const int o = ownH[(long long)y * d.P + x];
      if (o < sc.ncircles) {
        const double ddy = yj - sc.circ[3 * o + 1];
        const double r = sc.circ[3 * o + 2];
        const double disc = r * r - ddy * ddy;
        const double sq = sqrt(disc > 0.0 ? disc : 0.0);
        const double root = in_circle(sc, o, xi, yj) ? sc.circ[3 * o] + sq : sc.circ[3 * o] - sq;
        s = (root - xi) / dx;
      }
    }
    sH[(long long)y * d.P + x] = finish_fraction<R>(s);
  }
  if (y < d.ny && kbit(K, d, x, y) != kbit(K, d, x, y + 1)) {
    double s = 0.5;
    if (sc.nnotches && touches_notch(sc, xi, yj, xi, (y + 1) * dx)) {
      const bool side0 = scene_inside(sc, xi, yj);
      double lo = 0.0, hi = 1.0;
      for (int it = 0; it < 60; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (scene_inside(sc, xi, yj + mid * dx) == side0) lo = mid; else hi = mid;
      }
      s = 0.5 * (lo + hi);
    } else if (sc.has_curve && ((yj <= hv[x]) != (((y + 1) * dx) <= hv[x]))) {
      s = (hv[x] - yj) / dx;
    } else if (const int l = line_crossing(sc, xi, yj, xi, (y + 1) * dx); l >= 0) {
      const double yr = (sc.lc[l] - sc.la[l] * xi) / sc.lb[l];
      s = (yr - yj) / dx;
    } else {
      const int o = ownV[(long long)y * d.P + x];
      if (o < sc.ncircles) {
        const double ddx = xi - sc.circ[3 * o];
        const double r = sc.circ[3 * o + 2];
        const double disc = r * r - ddx * ddx;
        const double sq = sqrt(disc > 0.0 ? disc : 0.0);
        const double root = in_circle(sc, o, xi, yj) ? sc.circ[3 * o + 1] + sq : sc.circ[3 * o + 1] - sq;
        s = (root - yj) / dx;
      }
    }
    sV[(long long)y * d.P + x] = finish_fraction<R>(s);
  }
}

// ---------------------------------------------------------------------------
// State I/O: bytes <-> packed bits, doubles <-> pitched state fractions.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(32 * kBlockY)
k_pack_bits(const uint8_t* __restrict__ src, int w, int h, int words, uint32_t* dst) {
  const int x = blockIdx.x * 32 + threadIdx.x;
  const int y = blockIdx.y * kBlockY + threadIdx.y;
  const bool in = x < w && y < h;
  const unsigned word = __ballot_sync(0xffffffffu, in && src[(long long)y * w + x] != 0);
  if (threadIdx.x == 0 && y < h && x < w) dst[(long long)y * words + (x >> 5)] = word;
}

__global__ void k_unpack_bits(const uint32_t* __restrict__ src, int w, int h, int words, uint8_t* dst) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)w * h) return;
  const int x = (int)(t % w), y = (int)(t / w);
  dst[t] = (src[(long long)y * words + (x >> 5)] >> (x & 31)) & 1;
}

template <typename R>
__global__ void k_load_frac(const double* __restrict__ src, int w, int h, long long P, R* dst) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)w * h) return;
  const int x = (int)(t % w), y = (int)(t / w);
  double s = src[t];
  R r = (R)s;
  if (!(r >= R(0))) r = R(0);
  if (r >= R(1)) r = below_one<R>();
  dst[(long long)y * P + x] = r;
}

template <typename R>
__global__ void k_store_frac(const R* __restrict__ src, int w, int h, long long P, double* dst) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)w * h) return;
  const int x = (int)(t % w), y = (int)(t / w);
  dst[t] = (double)src[(long long)y * P + x];
}

}  // namespace ebit
