// Kernels besides the tiled sweep and the fused fields: initialisation and
// state I/O.
// Threads map to vertices of the real grid: a warp is 32 consecutive x of one
// row, aligned to 32, so colour bits pack into 32-bit words with a ballot.
#pragma once
#include "ebit_device.cuh"

namespace ebit {

constexpr int kBlockY = 8;  // blocks are 32 x kBlockY threads

__device__ __forceinline__ int kbit(const uint32_t* K, const Dims& d, int x, int y) {
  return (__ldg(&K[(long long)y * d.kw + (x >> 5)]) >> (x & 31)) & 1;
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

// A pitched field (h rows of `pitch` words of type W) to a dense one (h rows
// of w words): one word per thread and row, rows by a grid-stride loop (the
// grid's y extent is capped).  W = uint4 when the dense rows are whole
// 16-byte words and the destination is 16-byte aligned (the pitched rows
// always are), else the element type itself.
template <typename W>
__global__ void k_unpitch(const W* __restrict__ src, long long pitch, W* __restrict__ dst, long long w,
                          int h) {
  const long long x = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= w) return;
  for (long long y = blockIdx.y; y < h; y += gridDim.y) dst[y * w + x] = src[y * pitch + x];
}

}  // namespace ebit
