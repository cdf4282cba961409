// Hand-off to a one-fluid flow solver (Sec. 2.5).  The volume fraction C
// stands in for the Heaviside function of the property law (Eq. 8), and the
// surface term sigma kappa n delta_S of Eq. 6 is applied on the faces as
// sigma kappa_f grad C, with kappa_f the mean of the two cells' valid
// heights-based curvatures (one valid: that one; neither: no force).
//
// A pure stream: C and kappa are read once, rho, mu, fx and fy written once
// (24 bytes per cell in float, 48 in double).  A thread walks a strip of rows
// and carries the row below in registers; the left neighbour comes from the
// next lane down, so only the first row of a strip and lane 0 re-read a
// value, and those hit in cache.
#pragma once
#include <type_traits>

#include "ebit_device.cuh"

namespace ebit {

constexpr int kCT = 128;  // threads per block
constexpr int kCR = 16;   // rows per block of the double kernel

template <typename R>
struct Fluids {
  R r1, r2, m1, m2, sh;  // sh = sigma / dx, formed once in R
};

// rho or mu of a cell: c a + (1 - c) b (Eq. 8 with C for H).
template <typename R>
__device__ __forceinline__ R mix(R c, R a, R b) {
  return c * a + (R(1) - c) * b;
}

// (sigma/dx) kappa_f (C_b - C_a) for the face between cell a (low side) and
// cell b (high side); NaN marks a cell without a valid curvature, and with
// none on either side kappa_f = 0.  Branch-free for the float form: on the
// wide FP32 pipe the arithmetic costs less than tests, and the formulas give
// the pure-phase and zero values themselves.
template <typename R>
__device__ __forceinline__ R face_force(const Fluids<R>& f, R ka, R kb, R ca, R cb) {
  const bool va = !nan_bits(ka), vb = !nan_bits(kb);
  const R kf = va ? (vb ? (ka + kb) * R(0.5) : ka) : (vb ? kb : R(0));
  return f.sh * kf * (cb - ca);
}

// C, kap: pitched fields (row pitch d.P).  rho, mu: ny x nx; fx: ny x (nx+1);
// fy: (ny+1) x nx; any output may be null.  Thread t owns the column pair
// i0 = 2t, i0 + 1 (cells below nx; face columns up to nx, so the right wall
// face belongs to the last pair), reads both with one 8- or 16-byte load
// (rows are pitched to 32 elements, i0 is even) and, when nx is even, stores
// the pair of rho, mu and fy with one vector store.  Block rows cover 0..ny,
// row ny carrying only the top wall of fy.  Rows are taken NB at a time, all
// their loads issued before any is used.
constexpr int kCR2 = 8;  // rows per block of the column-pair kernel

template <typename R, int CR = kCR2, int NB = 4>
__global__ void __launch_bounds__(kCT) k_coupling(const R* __restrict__ C, const R* __restrict__ kap,
                                                  Dims d, Fluids<R> f, R* __restrict__ rho,
                                                  R* __restrict__ mu, R* __restrict__ fx,
                                                  R* __restrict__ fy) {
  static_assert(CR % NB == 0, "strip of whole batches");
  using R2 = typename std::conditional<sizeof(R) == 4, float2, double2>::type;
  const int i0 = 2 * (blockIdx.x * kCT + threadIdx.x);
  const int lane = threadIdx.x & 31;
  const int j0 = blockIdx.y * CR;
  const int jc = min(j0 + CR, d.ny);      // cell rows of the strip end here
  const int j1 = min(j0 + CR, d.ny + 1);  // face rows end here
  const bool c0 = i0 < d.nx, c1 = i0 + 1 < d.nx;
  const bool left = lane == 0 && c0 && i0 > 0;  // lane 0 reads its left neighbour itself
  const R nan = R(__int_as_float(0x7fc00000));
  const long long wx = (long long)d.nx + 1;
  const bool pairs = (d.nx & 1) == 0;  // rows of nx elements keep pairs aligned
  auto load = [&](const R* p, int row, R* a, R* b) {
    if (c1) {
      const R2 v = __ldg(reinterpret_cast<const R2*>(p + (long long)row * d.P + i0));
      *a = v.x;
      *b = v.y;
    } else if (c0) {
      *a = __ldg(p + (long long)row * d.P + i0);
    }
  };
  R cb0 = R(0), kb0 = nan, cb1 = R(0), kb1 = nan;  // row below, columns i0, i0 + 1
  if (j0 > 0) {
    load(C, j0 - 1, &cb0, &cb1);
    load(kap, j0 - 1, &kb0, &kb1);
  }
  for (int jb = j0; jb < j1; jb += NB) {  // trip count uniform across the block
    R ca[NB], cc[NB], ka[NB], kc[NB], cl[NB], kl[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = jb + q;
      ca[q] = cc[q] = cl[q] = R(0);
      ka[q] = kc[q] = kl[q] = nan;
      if (j < jc) {
        load(C, j, &ca[q], &cc[q]);
        load(kap, j, &ka[q], &kc[q]);
      }
      if (j < jc && left) {
        cl[q] = __ldg(&C[(long long)j * d.P + i0 - 1]);
        kl[q] = __ldg(&kap[(long long)j * d.P + i0 - 1]);
      }
    }
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = jb + q;
      const R cs = __shfl_up_sync(0xffffffffu, cc[q], 1), ks = __shfl_up_sync(0xffffffffu, kc[q], 1);
      if (lane != 0) {
        cl[q] = cs;
        kl[q] = ks;
      }
      const long long o = (long long)j * d.nx + i0;
      if (j < jc) {
        if (c1 && pairs) {
          if (rho) *reinterpret_cast<R2*>(rho + o) = R2{mix(ca[q], f.r1, f.r2), mix(cc[q], f.r1, f.r2)};
          if (mu) *reinterpret_cast<R2*>(mu + o) = R2{mix(ca[q], f.m1, f.m2), mix(cc[q], f.m1, f.m2)};
        } else {
          if (c0 && rho) rho[o] = mix(ca[q], f.r1, f.r2);
          if (c0 && mu) mu[o] = mix(ca[q], f.m1, f.m2);
          if (c1 && rho) rho[o + 1] = mix(cc[q], f.r1, f.r2);
          if (c1 && mu) mu[o + 1] = mix(cc[q], f.m1, f.m2);
        }
        if (fx) {
          R* px = fx + (long long)j * wx + i0;
          if (i0 <= d.nx)
            px[0] = (i0 == 0 || i0 == d.nx) ? R(0) : face_force(f, kl[q], ka[q], cl[q], ca[q]);
          if (i0 + 1 <= d.nx) px[1] = (i0 + 1 == d.nx) ? R(0) : face_force(f, ka[q], kc[q], ca[q], cc[q]);
        }
      }
      if (fy && j < j1) {
        const bool wall = j == 0 || j == d.ny;
        const R y0 = wall ? R(0) : face_force(f, kb0, ka[q], cb0, ca[q]);
        const R y1 = wall ? R(0) : face_force(f, kb1, kc[q], cb1, cc[q]);
        if (c1 && pairs) {
          *reinterpret_cast<R2*>(fy + o) = R2{y0, y1};
        } else {
          if (c0) fy[o] = y0;
          if (c1) fy[o + 1] = y1;
        }
      }
      cb0 = ca[q];
      kb0 = ka[q];
      cb1 = cc[q];
      kb1 = kc[q];
    }
  }
}

// The double form.  On this part the FP64 pipe retires a warp instruction
// every 16 cycles, so FP64 work issued by a warp in which only a few lanes
// hold a mixed cell or a face with a valid curvature would bound the kernel.
// Instead every lane settles pure cells and force-free faces with integer
// tests and stores them, and queues the rest in per-warp rings in shared
// memory; whenever a ring holds 32 items the warp evaluates them with every
// lane busy and stores the results.  The arithmetic is the one above: a face
// with one valid curvature k queues (k, k), whose mean (k + k) / 2 is k.
struct FaceRing {
  static constexpr int kCap = 128;  // >= 31 left over + 64 queued per row
  double ka[kCap], kb[kCap], ca[kCap], cb[kCap];
  double* out[kCap];
};
struct MixRing {
  static constexpr int kCap = 64;  // >= 31 left over + 32 queued per row
  double c[kCap];
  long long idx[kCap];
};

__device__ __forceinline__ void face_push(FaceRing& F, unsigned& tail, bool need, double ka, double kb,
                                          double ca, double cb, double* out) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned m = __ballot_sync(0xffffffffu, need);
  if (need) {
    const unsigned s = (tail + __popc(m & ((1u << lane) - 1u))) & (FaceRing::kCap - 1);
    F.ka[s] = ka;
    F.kb[s] = kb;
    F.ca[s] = ca;
    F.cb[s] = cb;
    F.out[s] = out;
  }
  tail += __popc(m);
}

__device__ __forceinline__ void face_run(const FaceRing& F, unsigned head, const Fluids<double>& f) {
  const unsigned s = (head + (threadIdx.x & 31)) & (FaceRing::kCap - 1);
  const double kf = (F.ka[s] + F.kb[s]) * 0.5;
  *F.out[s] = f.sh * kf * (F.cb[s] - F.ca[s]);
}

__device__ __forceinline__ void mix_run(const MixRing& M, unsigned head, const Fluids<double>& f,
                                        double* __restrict__ rho, double* __restrict__ mu) {
  const unsigned s = (head + (threadIdx.x & 31)) & (MixRing::kCap - 1);
  const double c = M.c[s];
  const double o = 1.0 - c;
  if (rho) rho[M.idx[s]] = c * f.r1 + o * f.r2;
  if (mu) mu[M.idx[s]] = c * f.m1 + o * f.m2;
}

// Same grid, layouts and outputs as k_coupling.
template <int CR = kCR, int NB = 2>
__global__ void __launch_bounds__(kCT) k_coupling_q(const double* __restrict__ C,
                                                    const double* __restrict__ kap, Dims d,
                                                    Fluids<double> f, double* __restrict__ rho,
                                                    double* __restrict__ mu, double* __restrict__ fx,
                                                    double* __restrict__ fy) {
  static_assert(CR % NB == 0, "strip of whole batches");
  __shared__ FaceRing face_ring[kCT / 32];
  __shared__ MixRing mix_ring[kCT / 32];
  FaceRing& F = face_ring[threadIdx.x >> 5];
  MixRing& M = mix_ring[threadIdx.x >> 5];
  unsigned fh = 0, ft = 0, mh = 0, mt = 0;  // ring heads and tails, warp-uniform
  const int i = blockIdx.x * kCT + threadIdx.x;
  const int lane = threadIdx.x & 31;
  const int j0 = blockIdx.y * CR;
  const int jc = min(j0 + CR, d.ny);
  const int j1 = min(j0 + CR, d.ny + 1);
  const bool cell = i < d.nx;
  const bool left = lane == 0 && cell && i > 0;
  const double nan = __longlong_as_double(0x7ff8000000000000ll);
  const long long wx = (long long)d.nx + 1;
  const bool props = rho || mu;
  double cb = 0.0, kb = nan;
  if (j0 > 0 && cell) {
    cb = __ldg(&C[(long long)(j0 - 1) * d.P + i]);
    kb = __ldg(&kap[(long long)(j0 - 1) * d.P + i]);
  }
  for (int jb = j0; jb < j1; jb += NB) {
    double c[NB], k[NB], cl[NB], kl[NB];
#pragma unroll
    for (int q = 0; q < NB; ++q) {
      const int j = jb + q;
      c[q] = 0.0;
      k[q] = nan;
      cl[q] = 0.0;
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
      const double cs = __shfl_up_sync(0xffffffffu, c[q], 1);
      const double ks = __shfl_up_sync(0xffffffffu, k[q], 1);
      if (lane != 0) {
        cl[q] = cs;
        kl[q] = ks;
      }
      const bool vk = !nan_bits(k[q]);
      // cell properties
      const bool cell_row = cell && j < jc && props;
      const bool pure1 = one_bits(c[q]), pure0 = zero_bits(c[q]);
      if (cell_row && (pure1 || pure0)) {
        const long long o = (long long)j * d.nx + i;
        if (rho) rho[o] = pure1 ? f.r1 : f.r2;
        if (mu) mu[o] = pure1 ? f.m1 : f.m2;
      }
      const bool mneed = cell_row && !pure1 && !pure0;
      {
        const unsigned m = __ballot_sync(0xffffffffu, mneed);
        if (mneed) {
          const unsigned s = (mt + __popc(m & ((1u << lane) - 1u))) & (MixRing::kCap - 1);
          M.c[s] = c[q];
          M.idx[s] = (long long)j * d.nx + i;
        }
        mt += __popc(m);
      }
      // vertical face (i, j) between cells (i-1, j) and (i, j)
      const bool xrow = fx && j < jc && i <= d.nx;
      const bool vl = !nan_bits(kl[q]);
      const bool xneed = xrow && i > 0 && i < d.nx && (vl || vk);
      if (xrow && !xneed) fx[(long long)j * wx + i] = 0.0;
      face_push(F, ft, xneed, vl ? kl[q] : k[q], vk ? k[q] : kl[q], cl[q], c[q],
                xneed ? fx + (long long)j * wx + i : nullptr);
      // horizontal face (i, j) between cells (i, j-1) and (i, j)
      const bool yrow = fy && cell && j < j1;
      const bool vb = !nan_bits(kb);
      const bool yneed = yrow && j > 0 && j < d.ny && (vb || vk);
      if (yrow && !yneed) fy[(long long)j * d.nx + i] = 0.0;
      face_push(F, ft, yneed, vb ? kb : k[q], vk ? k[q] : kb, cb, c[q],
                yneed ? fy + (long long)j * d.nx + i : nullptr);
      cb = c[q];
      kb = k[q];
      __syncwarp();
      while (ft - fh >= 32) {
        face_run(F, fh, f);
        fh += 32;
      }
      if (mt - mh >= 32) {
        mix_run(M, mh, f, rho, mu);
        mh += 32;
      }
      __syncwarp();
    }
  }
  if ((unsigned)lane < ft - fh) face_run(F, fh, f);
  if ((unsigned)lane < mt - mh) mix_run(M, mh, f, rho, mu);
}

}  // namespace ebit
