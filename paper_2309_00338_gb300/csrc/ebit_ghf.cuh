// Generalised height-function fallbacks (Sec. 2.5 takes its curvature from
// the generalised height-function method, Popinet 2009).  The fused fields
// kernel computes the standard 7x3 height-function curvature; interface
// cells without a valid stencil are left NaN there and, when the context
// asks for the generalised method, listed by that kernel (each tile stages
// its cells in shared memory and reserves its slice of the list with one
// atomic; a separate listing pass over kappa was latency-bound at 44-70 us
// at 4096^2).  One more launch gives the listed cells a value:
//
//   k_ghf_fit   one thread per listed cell, in turn: the standard stencil
//               along the other direction; a parabola fitted to the valid
//               heights of both directions ("mixed heights"); a parabola
//               fitted to the markers on the edges of the 3x3 block of cells
//               (the markers lie on the interface, where the volume-of-fluid
//               form would fit fragment centroids).
//
// The listed cells are a few per cent of the interface cells, so the fits
// (in the context precision, in cell units relative to the cell) run on
// compacted work.
#pragma once
#include "ebit_device.cuh"

namespace ebit {

// counters of the fallbacks, after the ones the other kernels use
constexpr int D_HF_OTHER = 13, D_HF_MIXED = 14, D_HF_MARKERS = 15;
static_assert(D_NUSED <= D_HF_OTHER && D_HF_MARKERS < kCounters, "counter slots");

constexpr int kGhfThreads = 128;  // k_ghf_fit block

__device__ __forceinline__ int kbit(const uint32_t* __restrict__ K, int kw, int i, int j, long long n) {
  const long long q = (long long)j * kw + (i >> 5);
  return in_range(q, n) ? (__ldg(&K[q]) >> (i & 31)) & 1 : 0;
}

// Read-only view of the state and fractions of one context.
template <typename R>
struct GhfView {
  const uint32_t* K;
  const uint32_t* Z;
  const R* sH;
  const R* sV;
  const R* C;
  Dims d;
  __device__ int k(int i, int j) const { return kbit(K, d.kw, i, j, d.nK()); }
  __device__ int z(int i, int j) const { return kbit(Z, d.zw, i, j, d.nZ()); }
  __device__ R c(int i, int j) const {
    const long long q = (long long)j * d.P + i;
    return in_range(q, d.nV()) ? __ldg(&C[q]) : R(0);
  }
  __device__ R h(int i, int j) const {
    const long long q = (long long)j * d.P + i;
    return in_range(q, d.nH()) ? __ldg(&sH[q]) : R(0);
  }
  __device__ R v(int i, int j) const {
    const long long q = (long long)j * d.P + i;
    return in_range(q, d.nV()) ? __ldg(&sV[q]) : R(0);
  }
};

// The fractions a listed cell's stencils read: the vertical arm
// v[m+1][t+3] = C(i+m, j+t) and the horizontal arm h[m+1][t+3] = C(i+t, j+m),
// m = -1..1, t = -3..3, loaded together (independent loads) for the columns
// that lie inside the domain (vin / hin).
template <typename R>
struct Cross {
  R v[3][7], h[3][7];
  bool vin[3], hin[3];
  __device__ void load(const GhfView<R>& S, int i, int j) {
#pragma unroll
    for (int m = -1; m <= 1; ++m) {
      vin[m + 1] = i + m >= 0 && i + m <= S.d.nx - 1 && j - 3 >= 0 && j + 3 <= S.d.ny - 1;
      hin[m + 1] = j + m >= 0 && j + m <= S.d.ny - 1 && i - 3 >= 0 && i + 3 <= S.d.nx - 1;
#pragma unroll
      for (int t = -3; t <= 3; ++t) {
        v[m + 1][t + 3] = vin[m + 1] ? S.c(i + m, j + t) : R(0);
        h[m + 1][t + 3] = hin[m + 1] ? S.c(i + t, j + m) : R(0);
      }
    }
  }
  // The column of seven cells through (i+m, j-3..j+3) (ycol) or the row
  // (i-3..i+3, j+m): its count of reference-phase cells (summed in that
  // order) and orientation: 1 = reference phase at the low end only, -1 = at
  // the high end only, 0 = not a valid height (mixed end cell, equal ends,
  // or outside the domain).
  __device__ __forceinline__ int column(int m, bool ycol, R* hsum) const {
    if (!(ycol ? vin[m + 1] : hin[m + 1])) return 0;
    R acc = R(0);
#pragma unroll
    for (int t = 0; t < 7; ++t) acc = acc + (ycol ? v[m + 1][t] : h[m + 1][t]);
    *hsum = acc;
    const R lo = ycol ? v[m + 1][0] : h[m + 1][0], hi = ycol ? v[m + 1][6] : h[m + 1][6];
    return (one_bits(lo) && zero_bits(hi)) ? 1 : (zero_bits(lo) && one_bits(hi)) ? -1 : 0;
  }
};

// Points of a fit, kept only when at least half a cell from every point
// already kept, with the least-squares sums (unit weights) accumulated in that
// order in the frame of origin (ox, oy), unit normal (nx, ny) and tangent
// (ny, -nx).  Arithmetic in R, coordinates in cell units relative to the
// cell's lower-left corner.
template <typename R>
struct ParabolaFit {
  R ox, oy, nx, ny;
  R X[24], Y[24];
  int np;
  R S0, S1, S2, S3, S4, T0, T1, T2;
  __device__ void reset() {
    np = 0;
    S0 = S1 = S2 = S3 = S4 = T0 = T1 = T2 = R(0);
  }
  __device__ void add(R x, R y) {
    for (int p = 0; p < np; ++p) {
      const R ex = x - X[p], ey = y - Y[p];
      if (ex * ex + ey * ey < R(0.25)) return;
    }
    if (np >= 24) return;
    X[np] = x;
    Y[np] = y;
    ++np;
    const R ddx = x - ox, ddy = y - oy;
    const R sv = ddx * ny - ddy * nx;
    const R zv = ddx * nx + ddy * ny;
    const R s2 = sv * sv;
    S0 = S0 + R(1);
    S1 = S1 + sv;
    S2 = S2 + s2;
    S3 = S3 + s2 * sv;
    S4 = S4 + s2 * s2;
    T0 = T0 + zv;
    T1 = T1 + zv * sv;
    T2 = T2 + zv * s2;
  }
  // z = a s^2 + b s + c by Cramer's rule; kappa = -2a / (1 + b^2)^(3/2) / dx
  __device__ bool kappa(R dx, R* out) const {
    if (np < 3) return false;
    const R m00 = S2 * S0 - S1 * S1;
    const R m01 = S3 * S0 - S1 * S2;
    const R m02 = S3 * S1 - S2 * S2;
    const R det = S4 * m00 - S3 * m01 + S2 * m02;
    // regular: |det| above 1e-3 of its Hadamard bound S4 S2 S0, in both precisions
    const R eps = R(1e-3);
    if (!(fabs(det) > eps * (S4 * S2 * S0))) return false;
    const R u1 = T1 * S0 - S1 * T0;
    const R da = T2 * m00 - S3 * u1 + S2 * (T1 * S1 - S2 * T0);
    const R db = S4 * u1 - T2 * m01 + S2 * (S3 * T0 - T1 * S2);
    const R a = da / det, b = db / det;
    const R q = R(1) + b * b;
    *out = (R(-2) * a) / (q * sqrt(q)) / dx;
    return isfinite(*out);
  }
};

template <typename R>
__global__ void __launch_bounds__(kGhfThreads, 6)
    k_ghf_fit(GhfView<R> S, R dx, const int* __restrict__ list, const unsigned* __restrict__ count,
              R* __restrict__ kappa, unsigned long long* __restrict__ ctr) {
  __shared__ unsigned s_cnt[3];
  if (threadIdx.x < 3) s_cnt[threadIdx.x] = 0;
  __syncthreads();
  const unsigned n = *count;
  unsigned got[3] = {0, 0, 0};
  for (unsigned e = blockIdx.x * kGhfThreads + threadIdx.x; e < n; e += gridDim.x * kGhfThreads) {
    const int idx = __ldg(&list[e]);
    const int i = idx % S.d.nx, j = idx / S.d.nx;
    const int c[4] = {S.k(i, j), S.k(i + 1, j), S.k(i + 1, j + 1), S.k(i, j + 1)};
    const int q = c[0] | (c[1] << 1) | (c[2] << 2) | (c[3] << 3);
    int seg[2][2];
    const int ns = segments(q, edge_mask(q) == 15 ? S.z(i, j) : 0, seg);
    const R px[4] = {S.h(i, j), R(1), S.h(i, j + 1), R(0)};
    const R py[4] = {R(0), S.v(i + 1, j), R(1), S.v(i, j)};
    R ax = R(0), ay = R(0);
    for (int t = 0; t < ns; ++t) {
      ax = ax + fabs(px[seg[t][1]] - px[seg[t][0]]);
      ay = ay + fabs(py[seg[t][1]] - py[seg[t][0]]);
    }
    Cross<R> X;
    X.load(S, i, j);
    // 1. the standard stencil along the other direction
    const bool ycol = !(ax >= ay);
    {
      R h[3];
      int o[3];
#pragma unroll
      for (int m = -1; m <= 1; ++m) o[m + 1] = X.column(m, ycol, &h[m + 1]);
      if (o[0] != 0 && o[0] == o[1] && o[1] == o[2]) {
        const R hp = (h[2] - h[0]) * R(0.5);
        const R hpp = (h[2] - h[1]) - (h[1] - h[0]);
        const R qv = R(1) + hp * hp;
        const R den = dx * (qv * sqrt(qv));
        if (in_range((long long)j * S.d.P + i, S.d.nV())) kappa[(long long)j * S.d.P + i] = -hpp / den;
        ++got[0];
        continue;
      }
    }
    // the frame: the cell's single segment A->B, origin at its midpoint,
    // normal perpendicular to it and turned away from the reference-phase
    // corners (their colour-signed offsets from the centre sum into the
    // reference phase)
    if (ns != 1) continue;
    const int ea = seg[0][0], eb = seg[0][1];
    ParabolaFit<R> F;
    F.ox = (px[ea] + px[eb]) * R(0.5);
    F.oy = (py[ea] + py[eb]) * R(0.5);
    R n0x = py[eb] - py[ea], n0y = -(px[eb] - px[ea]);
    const int gx = (2 * c[1] - 1) + (2 * c[2] - 1) - (2 * c[0] - 1) - (2 * c[3] - 1);
    const int gy = (2 * c[2] - 1) + (2 * c[3] - 1) - (2 * c[0] - 1) - (2 * c[1] - 1);
    const R dot = n0x * (R)gx + n0y * (R)gy;
    if (dot == R(0)) continue;
    if (dot > R(0)) {
      n0x = -n0x;
      n0y = -n0y;
    }
    const R len = sqrt(n0x * n0x + n0y * n0y);
    if (!(len > R(0))) continue;
    F.nx = n0x / len;
    F.ny = n0y / len;
    // 2. mixed heights: the valid columns of both directions' stencils
    F.reset();
#pragma unroll
    for (int dir = 0; dir < 2; ++dir) {
      const bool yc = dir == 0;
#pragma unroll
      for (int m = -1; m <= 1; ++m) {
        R h = R(0);
        const int o = X.column(m, yc, &h);
        if (o == 0) continue;
        const R pos = o == 1 ? R(-3) + h : R(4) - h;
        const R mid = (R)m + R(0.5);
        if (yc) F.add(mid, pos);
        else F.add(pos, mid);
      }
    }
    R kv;
    if (F.kappa(dx, &kv)) {
      if (in_range((long long)j * S.d.P + i, S.d.nV())) kappa[(long long)j * S.d.P + i] = kv;
      ++got[1];
      continue;
    }
    // 3. the markers on the edges of the 3x3 block
    F.reset();
    for (int b = j - 1; b <= j + 2; ++b)
      for (int a = i - 1; a <= i + 1; ++a)
        if (a >= 0 && a < S.d.nx && b >= 0 && b <= S.d.ny && S.k(a, b) != S.k(a + 1, b))
          F.add((R)(a - i) + S.h(a, b), (R)(b - j));
    for (int b = j - 1; b <= j + 1; ++b)
      for (int a = i - 1; a <= i + 2; ++a)
        if (a >= 0 && a <= S.d.nx && b >= 0 && b < S.d.ny && S.k(a, b) != S.k(a, b + 1))
          F.add((R)(a - i), (R)(b - j) + S.v(a, b));
    if (F.kappa(dx, &kv)) {
      if (in_range((long long)j * S.d.P + i, S.d.nV())) kappa[(long long)j * S.d.P + i] = kv;
      ++got[2];
    }
  }
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    const unsigned s = __reduce_add_sync(0xffffffffu, got[t]);
    if (s && (threadIdx.x & 31) == 0) atomicAdd(&s_cnt[t], s);
  }
  __syncthreads();
  if (threadIdx.x < 3 && s_cnt[threadIdx.x])
    atomicAdd(&ctr[D_HF_OTHER + threadIdx.x], (unsigned long long)s_cnt[threadIdx.x]);
}

}  // namespace ebit
