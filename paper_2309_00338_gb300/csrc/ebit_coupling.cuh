// Hand-off to a one-fluid flow solver (Sec. 2.5).  The volume fraction C
// stands in for the Heaviside function of the property law (Eq. 8), and the
// surface term sigma kappa n delta_S of Eq. 6 is applied on the faces as
// sigma kappa_f grad C, with kappa_f the mean of the two cells' valid
// heights-based curvatures (one valid: that one; neither: no force).
//
// A pure stream: C and kappa are read once, rho, mu, fx and fy written once
// (24 bytes per cell in float, 48 in double).  One thread per column walks a
// strip of rows and carries the row below in registers; the left neighbour
// comes from the next lane down, so only the first row of a strip and lane 0
// re-read a value, and those hit in cache.
#pragma once
#include "ebit_device.cuh"

namespace ebit {

constexpr int kCT = 128;  // columns per block
constexpr int kCR = 16;   // rows per block

template <typename R>
struct Fluids {
  R r1, r2, m1, m2, sg, h;
};

// sigma kappa_f (C_b - C_a) / h for the face between cell a (low side) and
// cell b (high side); NaN marks a cell without a valid curvature.
template <typename R>
__device__ __forceinline__ R face_force(const Fluids<R>& f, R ka, R kb, R ca, R cb) {
  const bool va = !isnan(ka), vb = !isnan(kb);
  const R kf = va && vb ? (ka + kb) * R(0.5) : va ? ka : vb ? kb : R(0);
  return f.sg * kf * (cb - ca) / f.h;
}

// C, kap: pitched fields (row pitch d.P).  rho, mu: ny x nx; fx: ny x (nx+1);
// fy: (ny+1) x nx; any output may be null.  Thread column i runs over
// 0..nx: cell i for i < nx, and the right wall face of fx for i = nx.  Block
// rows cover 0..ny, row ny carrying only the top wall of fy.
template <typename R>
__global__ void __launch_bounds__(kCT) k_coupling(const R* __restrict__ C, const R* __restrict__ kap,
                                                  Dims d, Fluids<R> f, R* __restrict__ rho,
                                                  R* __restrict__ mu, R* __restrict__ fx,
                                                  R* __restrict__ fy) {
  const int i = blockIdx.x * kCT + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int j0 = blockIdx.y * kCR;
  const int j1 = min(j0 + kCR, d.ny + 1);
  const bool cell = i < d.nx;
  const R nan = R(__int_as_float(0x7fc00000));
  const long long wx = (long long)d.nx + 1;
  R cb = R(0), kb = nan;  // row below, column i
  if (j0 > 0 && cell) {
    cb = __ldg(&C[(long long)(j0 - 1) * d.P + i]);
    kb = __ldg(&kap[(long long)(j0 - 1) * d.P + i]);
  }
#pragma unroll 4
  for (int j = j0; j < j1; ++j) {  // trip count uniform across the block
    const bool row = j < d.ny;
    R c = R(0), k = nan;
    if (row && cell) {
      c = __ldg(&C[(long long)j * d.P + i]);
      k = __ldg(&kap[(long long)j * d.P + i]);
    }
    R cl = __shfl_up_sync(0xffffffffu, c, 1), kl = __shfl_up_sync(0xffffffffu, k, 1);
    if (lane == 0 && row && cell && i > 0) {
      cl = __ldg(&C[(long long)j * d.P + i - 1]);
      kl = __ldg(&kap[(long long)j * d.P + i - 1]);
    }
    if (row) {
      if (cell && rho) rho[(long long)j * d.nx + i] = c * f.r1 + (R(1) - c) * f.r2;
      if (cell && mu) mu[(long long)j * d.nx + i] = c * f.m1 + (R(1) - c) * f.m2;
      if (i <= d.nx && fx)
        fx[(long long)j * wx + i] = (i == 0 || i == d.nx) ? R(0) : face_force(f, kl, k, cl, c);
    }
    if (cell && fy)
      fy[(long long)j * d.nx + i] = (j == 0 || j == d.ny) ? R(0) : face_force(f, kb, k, cb, c);
    cb = c;
    kb = k;
  }
}

}  // namespace ebit
