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
  R r1, r2, m1, m2, sh;  // sh = sigma / dx, formed once in R
};

// Tests on the integer pipe (FP64 compares and arithmetic run on the narrow
// FP64 pipe, which would otherwise bound the double form).
__device__ __forceinline__ bool nan_bits(float x) { return (__float_as_uint(x) & 0x7fffffffu) > 0x7f800000u; }
__device__ __forceinline__ bool nan_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull) > 0x7ff0000000000000ull;
}
__device__ __forceinline__ bool one_bits(float x) { return __float_as_uint(x) == 0x3f800000u; }
__device__ __forceinline__ bool one_bits(double x) {
  return (unsigned long long)__double_as_longlong(x) == 0x3ff0000000000000ull;
}
__device__ __forceinline__ bool zero_bits(float x) { return (__float_as_uint(x) << 1) == 0u; }
__device__ __forceinline__ bool zero_bits(double x) {
  return ((unsigned long long)__double_as_longlong(x) << 1) == 0ull;
}

// c a + (1 - c) b; a pure cell (c = 1 or c = 0) gives a or b, which is what
// the expression evaluates to there.
template <typename R>
__device__ __forceinline__ R mix(R c, R a, R b) {
  if (one_bits(c)) return a;
  if (zero_bits(c)) return b;
  return c * a + (R(1) - c) * b;
}

// (sigma/dx) kappa_f (C_b - C_a) for the face between cell a (low side) and
// cell b (high side); NaN marks a cell without a valid curvature.  With no
// valid curvature on either side kappa_f = 0 and the force is zero.
template <typename R>
__device__ __forceinline__ R face_force(const Fluids<R>& f, R ka, R kb, R ca, R cb) {
  const bool va = !nan_bits(ka), vb = !nan_bits(kb);
  if (!va && !vb) return R(0);
  const R kf = va && vb ? (ka + kb) * R(0.5) : va ? ka : kb;
  return f.sh * kf * (cb - ca);
}

// C, kap: pitched fields (row pitch d.P).  rho, mu: ny x nx; fx: ny x (nx+1);
// fy: (ny+1) x nx; any output may be null.  Thread column i runs over
// 0..nx: cell i for i < nx, and the right wall face of fx for i = nx.  Block
// rows cover 0..ny, row ny carrying only the top wall of fy.  Rows are taken
// NB at a time, all their loads issued before any is used, so that each
// thread keeps 2 NB loads in flight.
template <typename R, int CR = kCR, int NB = 16 / sizeof(R) * 2>
__global__ void __launch_bounds__(kCT) k_coupling(const R* __restrict__ C, const R* __restrict__ kap,
                                                  Dims d, Fluids<R> f, R* __restrict__ rho,
                                                  R* __restrict__ mu, R* __restrict__ fx,
                                                  R* __restrict__ fy) {
  static_assert(CR % NB == 0, "strip of whole batches");
  const int i = blockIdx.x * kCT + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int j0 = blockIdx.y * CR;
  const int jc = min(j0 + CR, d.ny);      // cell rows of the strip end here
  const int j1 = min(j0 + CR, d.ny + 1);  // face rows end here
  const bool cell = i < d.nx;
  const bool left = lane == 0 && cell && i > 0;  // lane 0 reads its left neighbour itself
  const R nan = R(__int_as_float(0x7fc00000));
  const long long wx = (long long)d.nx + 1;
  R cb = R(0), kb = nan;  // row below, column i
  if (j0 > 0 && cell) {
    cb = __ldg(&C[(long long)(j0 - 1) * d.P + i]);
    kb = __ldg(&kap[(long long)(j0 - 1) * d.P + i]);
  }
  for (int jb = j0; jb < j1; jb += NB) {  // trip count uniform across the block
    R c[NB], k[NB], cl[NB], kl[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = jb + q;
      c[q] = R(0);
      k[q] = nan;
      cl[q] = R(0);
      kl[q] = nan;
      if (j < jc && cell) {
        c[q] = __ldg(&C[(long long)j * d.P + i]);
        k[q] = __ldg(&kap[(long long)j * d.P + i]);
      }
      if (j < jc && left) {
        cl[q] = __ldg(&C[(long long)j * d.P + i - 1]);
        kl[q] = __ldg(&kap[(long long)j * d.P + i - 1]);
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = jb + q;
      const R cs = __shfl_up_sync(0xffffffffu, c[q], 1), ks = __shfl_up_sync(0xffffffffu, k[q], 1);
      if (lane != 0) {
        cl[q] = cs;
        kl[q] = ks;
      }
      if (j < jc) {
        if (cell && rho) rho[(long long)j * d.nx + i] = mix(c[q], f.r1, f.r2);
        if (cell && mu) mu[(long long)j * d.nx + i] = mix(c[q], f.m1, f.m2);
        if (i <= d.nx && fx)
          fx[(long long)j * wx + i] =
              (i == 0 || i == d.nx) ? R(0) : face_force(f, kl[q], k[q], cl[q], c[q]);
      }
      if (j < j1 && cell && fy)
        fy[(long long)j * d.nx + i] =
            (j == 0 || j == d.ny) ? R(0) : face_force(f, kb, k[q], cb, c[q]);
      cb = c[q];
      kb = k[q];
    }
  }
}

}  // namespace ebit
