// Device code of the EBIT step (Pan et al., arXiv:2309.00338, Sec. 2.1-2.5).
//
// State of one grid in HBM (element pitch P, a multiple of 32, for the edge
// and cell arrays):
//   K  corner colour vertices, 1 bit per vertex, rows of kw 32-bit words
//   Z  centre colour vertices, 1 bit per cell, rows of zw words
//   sH marker fraction on horizontal edge (i,j), row j, element i
//   sV marker fraction on vertical edge (i,j),   row j, element i
// A marker exists exactly where the corner colours at the ends of its edge
// differ (Sec. 2.4); fractions of edges without a marker are don't-care.
//
// One split sweep is written once, for the x direction, in "sweep
// coordinates": AX = 0 reads the grid as it is, AX = 1 reads it transposed
// (vertex (i,j) is stored vertex (j,i), horizontal and vertical edges swap),
// which turns the y sweep into an x sweep.  Every decision is taken with the
// exact integer predicate "left of grid line k" <=> ix < k on moved points
// stored as (grid line index, fraction), so corner flips and chord crossings
// agree.  The library is compiled with -fmad=false: every expression below is
// the sequence of IEEE operations it spells.
//
// The sweep logic (segments, neighbours, centre rule, circle fit, candidate
// selection) is written against an accessor A that answers, in sweep
// coordinates: tnx/tny, old colours k/z, moved(marker), knew (new corner
// colour) and landing (aligned markers landing on an edge).  GView answers
// from global memory by recomputation; the tiled sweep kernel's accessor
// from shared memory, where each answer was computed once.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace ebit {

enum {
  D_NH = 0, D_NV, D_CANCELLED, D_ZSET, D_ZCONFLICT, D_FIT_ONLINE, D_FIT_LINE, D_FIT_ONE,
  D_FIT_TWO, D_WALL_CLAMP, D_INVARIANT, D_HF_INVALID, D_CFL, D_NUSED
};
constexpr int kCounters = 16;
enum { ST_CFL = 1, ST_INVARIANT = 2, ST_TIMEOUT = 4 };

// Two points closer than 0.01 cell do not define a usable circle (Sec. 2.2).
constexpr double kMinSep2 = 1e-4;

template <typename R> __device__ __forceinline__ R below_one();
template <> __device__ __forceinline__ float below_one<float>() { return __int_as_float(0x3f7fffff); }
template <> __device__ __forceinline__ double below_one<double>() {
  return __longlong_as_double(0x3fefffffffffffffLL);
}

// Pointers of one state buffer.
template <typename R>
struct Buf {
  uint32_t* K;
  uint32_t* Z;
  R* sH;
  R* sV;
};

struct Dims {
  int nx, ny;     // cells
  int kw, zw;     // words per row of K and Z
  long long P;    // element pitch of sH, sV, C, kappa
  // extents of the arrays, in elements
  __host__ __device__ long long nK() const { return (long long)(ny + 1) * kw; }
  __host__ __device__ long long nZ() const { return (long long)ny * zw; }
  __host__ __device__ long long nH() const { return (long long)(ny + 1) * P; }
  __host__ __device__ long long nV() const { return (long long)ny * P; }  // also C and kappa
  __host__ __device__ long long nW() const { return (long long)(ny + 1) * (nx + 1); }
};

struct Mk {
  int kind;  // 0 horizontal edge, 1 vertical edge, -1 none
  int i, j;
};

// A moved point: grid line ix at or left of it and fraction fx in [0,1);
// y = jy + fy is unchanged by the sweep.
template <typename R>
struct AP {
  int ix;
  R fx;
  int jy;
  R fy;
};

// CFL and wall flags of one moved marker; dabs is |d| in the state precision
// (a float |d| converts to double exactly, so the largest one is the same).
struct Flags {
  int cfl = 0, clamp = 0;
  float dabs = 0.0f;
  double dabs64 = 0.0;
};

// Aligned markers landing on an edge (Sec. 2.4).
template <typename R>
struct Landing {
  int present, kept_src, cancelled, invariant;
  R kept_fx;
};

// Bits [a, b] (inclusive, columns of a row of 32-bit words) within word wi;
// empty if a > b.
__device__ __forceinline__ uint32_t span_mask(int wi, int a, int b) {
  const int lo = max(a - 32 * wi, 0), hi = min(b - 32 * wi, 31);
  if (lo > hi) return 0u;
  const uint32_t up = hi == 31 ? 0xffffffffu : ((1u << (hi + 1)) - 1u);
  return up & ~((1u << lo) - 1u);
}

// Loads of the state a kernel advances.  LD = 0: through the read-only
// (non-coherent) cache, for kernels that never write what they read; LD = 1:
// cached in L2 only (coherent), for a kernel that reads, after a fenced count
// of finished tiles, what other blocks of the same launch wrote.
template <int LD, typename T>
__device__ __forceinline__ T ld_state(const T* p) {
  if constexpr (LD != 0) return __ldcg(p);
  else return __ldg(p);
}

// Bits x0 .. x0+31 of a stored row of nw words (bits outside the row read 0).
template <int LD = 0>
__device__ __forceinline__ uint32_t row_bits(const uint32_t* __restrict__ row, int nw, int x0) {
  const int q = x0 >> 5, r = x0 & 31;
  const uint32_t a = (q >= 0 && q < nw) ? ld_state<LD>(&row[q]) : 0u;
  const uint32_t b = (q + 1 >= 0 && q + 1 < nw) ? ld_state<LD>(&row[q + 1]) : 0u;
  return r ? ((a >> r) | (b << (32 - r))) : a;
}

// ---------------------------------------------------------------------------
// Cell topology.  Corner c of cell (i,j) counter-clockwise from (i,j); edge e
// joins corners e and e+1 (0 bottom, 1 right, 2 top, 3 left).
// ---------------------------------------------------------------------------
__device__ __forceinline__ int edge_mask(int q) { return (q ^ ((q >> 1) | ((q & 1) << 3))) & 15; }

// Segments of the implicit connectivity (Sec. 2.3, Fig. 4): two markers are
// joined; with four, each corner whose colour differs from the centre colour
// is cut off by the segment joining the markers of its two edges.
__device__ __forceinline__ int segments(int q, int zc, int seg[2][2]) {
  const int em = edge_mask(q);
  if (em == 0) return 0;
  if (em != 15) {
    seg[0][0] = __ffs(em) - 1;
    seg[0][1] = 31 - __clz(em);
    return 1;
  }
  // four markers: q is 5 or 10.  The corners of the other colour than the
  // centre are cut off, in corner order: corners 1 and 3 (segments 0-1, 2-3)
  // when corner 0 has the centre's colour, else corners 0 and 2 (segments
  // 3-0, 1-2).
  if ((q & 1) == zc) {
    seg[0][0] = 0; seg[0][1] = 1;
    seg[1][0] = 2; seg[1][1] = 3;
  } else {
    seg[0][0] = 3; seg[0][1] = 0;
    seg[1][0] = 1; seg[1][1] = 2;
  }
  return 2;
}

__device__ __forceinline__ Mk edge_marker(int ci, int cj, int e) {
  Mk m;
  m.kind = e & 1;
  m.i = ci + (e == 1);
  m.j = cj + (e == 2);
  return m;
}

template <class A>
__device__ __forceinline__ int corner_mask(const A& S, int i, int j) {
  return S.k(i, j) | (S.k(i + 1, j) << 1) | (S.k(i + 1, j + 1) << 2) | (S.k(i, j + 1) << 3);
}

template <class A>
__device__ __forceinline__ int cell_segments(const A& S, int i, int j, int seg[2][2]) {
  const int q = corner_mask(S, i, j);
  return segments(q, edge_mask(q) == 15 ? S.z(i, j) : 0, seg);
}

template <class A>
__device__ int partner(const A& S, int ci, int cj, int e) {
  int seg[2][2];
  const int n = cell_segments(S, ci, cj, seg);
#pragma unroll
  for (int t = 0; t < 2; ++t) {
    if (t >= n) break;
    if (seg[t][0] == e) return seg[t][1];
    if (seg[t][1] == e) return seg[t][0];
  }
  return -1;
}

// The marker next to m along the interface on the far side of m's edge, seen
// from cell (ci,cj); writes the cell it lies in.
template <class A>
__device__ Mk beyond(const A& S, Mk m, int ci, int cj, int* oi_, int* oj_) {
  int oi, oj, oe;
  if (m.kind == 0) {
    oi = m.i;
    if (cj == m.j) { oj = m.j - 1; oe = 2; } else { oj = m.j; oe = 0; }
  } else {
    oj = m.j;
    if (ci == m.i) { oi = m.i - 1; oe = 1; } else { oi = m.i; oe = 3; }
  }
  Mk none{-1, 0, 0};
  if (oi < 0 || oj < 0 || oi >= S.tnx() || oj >= S.tny()) return none;
  const int pe = partner(S, oi, oj, oe);
  if (pe < 0) return none;
  *oi_ = oi;
  *oj_ = oj;
  return edge_marker(oi, oj, pe);
}

// ---------------------------------------------------------------------------
// Advection along the sweep (Eq. 4).
// ---------------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ R dabs_of(const Flags& f) {
  return sizeof(R) == 4 ? (R)f.dabs : (R)f.dabs64;
}

// Velocity by linear interpolation along the marker's edge (the bilinear
// interpolation of Sec. 2.1 on a grid line); displacement in cells, clipped to
// one cell with the CFL flag raised beyond it.
template <typename R>
__device__ __forceinline__ R displacement(R s, R ua, R ub, R lam, Flags& f) {
  const R vel = (R(1) - s) * ua + s * ub;
  R d = vel * lam;
  const R ad = fabs(d);
  if (sizeof(R) == 4) {
    if (ad == ad && (float)ad > f.dabs) f.dabs = (float)ad;
  } else {
    if (ad == ad && (double)ad > f.dabs64) f.dabs64 = (double)ad;
  }
  if (!(fabs(d) <= R(1))) {
    f.cfl = 1;
    d = (d > R(0)) ? R(1) : R(-1);
  }
  return d;
}

// Moved point of an aligned marker on edge (i, line) with fraction s, given the
// velocities at the edge's ends; nx = number of cells along the sweep.
template <typename R>
__device__ __forceinline__ AP<R> move_aligned(int i, int line, R s, R ua, R ub, R lam, int nx,
                                               Flags& f) {
  const R d = displacement(s, ua, ub, lam, f);
  const R t = s + d;
  const R fl = floor(t);
  R fx = t - fl;
  int sh = (int)fl;
  if (sh > 1) { sh = 1; fx = below_one<R>(); }
  if (fx >= R(1)) fx = below_one<R>();
  int ix = i + sh;
  // markers cannot leave the domain: they stop at the wall
  if (ix < 0) { ix = 0; fx = R(0); f.clamp = 1; }
  else if (ix > nx - 1) { ix = nx - 1; fx = below_one<R>(); f.clamp = 1; }
  AP<R> p;
  p.ix = ix;
  p.fx = fx;
  p.jy = line;
  p.fy = R(0);
  return p;
}

// Moved point (the gray point of Fig. 2c) of an unaligned marker on vertical
// edge (i, row); markers on the two walls normal to the sweep stay.
template <typename R>
__device__ __forceinline__ AP<R> move_unaligned(int i, int row, R s, R ua, R ub, R lam, int nx,
                                                 Flags& f) {
  AP<R> p;
  p.jy = row;
  p.fy = s;
  if (i == 0 || i == nx) {
    p.ix = i;
    p.fx = R(0);
    return p;
  }
  const R d = displacement(s, ua, ub, lam, f);
  const R fl = floor(d);
  R fx = d - fl;
  if (fx >= R(1)) fx = below_one<R>();
  p.ix = i + (int)fl;
  p.fx = fx;
  return p;
}

// Order-preserving integer keys of a float / double (-0 and +0 equal).
__device__ __forceinline__ long long okey(double x) {
  const long long b = __double_as_longlong(x);
  if (b >= 0) return b;
  return b == (long long)(1ull << 63) ? 0 : (b ^ 0x7fffffffffffffffLL);
}
__device__ __forceinline__ long long okey(float x) {
  const int b = __float_as_int(x);
  if (b >= 0) return b;
  return b == (int)0x80000000 ? 0 : (long long)(b ^ 0x7fffffff);
}

// Aligned markers landing on edge (i, j), from edges i-1, i, i+1 (slot q for
// edge i-1+q, present in valid): kept only where the new end colours differ;
// an odd count keeps the median by (fraction, source edge).  Ranks in
// registers instead of a sort.
template <typename R>
__device__ __forceinline__ Landing<R> choose_landing3(const bool valid[3], const R fx[3], int i,
                                                      int present) {
  const int n = (int)valid[0] + (int)valid[1] + (int)valid[2];
  long long key[3];
  int rank[3];
#pragma unroll
  for (int t = 0; t < 3; ++t) key[t] = okey(fx[t]);
#pragma unroll
  for (int t = 0; t < 3; ++t) {
    int r = 0;
#pragma unroll
    for (int u = 0; u < 3; ++u)  // sources are distinct: ties in fraction go by source edge
      if (u != t && valid[u] && (key[u] < key[t] || (key[u] == key[t] && u < t))) ++r;
    rank[t] = r;
  }
  Landing<R> L;
  L.present = present;
  L.kept_src = -1;
  L.kept_fx = R(0.5);
  L.cancelled = 0;
  L.invariant = 0;
  int want = -1;
  if (present && (n & 1)) {
    want = n / 2;
    L.cancelled = n / 2;  // the pairs around the middle one
  } else if (!present && !(n & 1)) {
    L.cancelled = n / 2;
  } else {
    L.invariant = 1;
    if (present && n > 0) {  // nearest the edge's middle, first in rank order
      double bd = 0.0;
#pragma unroll
      for (int t = 0; t < 3; ++t)
        if (valid[t]) {
          const double d = fabs((double)fx[t] - 0.5);
          if (want < 0 || d < bd || (d == bd && rank[t] < want)) {
            bd = d;
            want = rank[t];
          }
        }
    }
  }
  if (want >= 0) {
#pragma unroll
    for (int t = 0; t < 3; ++t)
      if (valid[t] && rank[t] == want) {
        L.kept_src = i - 1 + t;
        L.kept_fx = fx[t];
      }
  }
  return L;
}

// ---------------------------------------------------------------------------
// IEEE predicates on finite doubles, evaluated on the bit pattern so that they
// run on the integer pipe rather than the (narrow) FP64 pipe: x > 0, x < 0,
// x == 0, 0 <= x <= 1, and s < kMinSep2 for s >= +0.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long dbits(double x) { return __double_as_longlong(x); }
__device__ __forceinline__ bool d_gt0(double x) { return dbits(x) > 0; }
__device__ __forceinline__ bool d_lt0(double x) { return (dbits(x) ^ (long long)(1ull << 63)) > 0; }
__device__ __forceinline__ bool d_eq0(double x) { return (dbits(x) << 1) == 0; }
__device__ __forceinline__ bool d_in01(double x) {
  const unsigned long long b = (unsigned long long)dbits(x);
  return b <= 0x3ff0000000000000ull || b == 0x8000000000000000ull;
}
__device__ __forceinline__ bool d_below_sep(double s) { return dbits(s) < dbits(kMinSep2); }

// Debug builds (EBIT_CHECK): the step kernels check each global index
// against the extent of its array; a miss sets the check word (read by
// ebit_check_status) and the access is skipped.  Release builds compile the
// checks away.
#ifdef EBIT_CHECK
static __device__ unsigned ebit_check_word;
__device__ __forceinline__ bool in_range(long long idx, long long n) {
  if (idx >= 0 && idx < n) return true;
  atomicOr(&ebit_check_word, 1u);
  return false;
}
#else
__device__ __forceinline__ bool in_range(long long, long long) { return true; }
#endif

// Value tests on the integer pipe for either precision (a double compare
// would take a slot of the narrow FP64 pipe): NaN, exactly 1, +-0.
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

// Exact conversions to double by integer operations: a float (any finite
// value) and a small integer.
__device__ __forceinline__ double f2d(float f) {
  const unsigned u = __float_as_uint(f);
  const unsigned long long sign = (unsigned long long)(u & 0x80000000u) << 32;
  int e = (int)((u >> 23) & 0xffu);
  unsigned m = u & 0x7fffffu;
  if (e == 0) {
    if (m == 0) return __longlong_as_double((long long)sign);
    const int sh = __clz(m) - 8;  // bring the leading one to bit 23
    m = (m << sh) & 0x7fffffu;
    e = 1 - sh;
  }
  return __longlong_as_double(
      (long long)(sign | ((unsigned long long)(e + 896) << 52) | ((unsigned long long)m << 29)));
}
__device__ __forceinline__ double i2d(int n) {
  if (n == 0) return 0.0;
  const unsigned long long sign = n < 0 ? (1ull << 63) : 0ull;
  const unsigned a = n < 0 ? (unsigned)(-n) : (unsigned)n;
  const int p = 31 - __clz(a);
  const unsigned long long mant = ((unsigned long long)a << (52 - p)) & 0xfffffffffffffull;
  return __longlong_as_double((long long)(sign | ((unsigned long long)(1023 + p) << 52) | mant));
}
template <typename R> __device__ __forceinline__ double to_d(R x);
template <> __device__ __forceinline__ double to_d<float>(float x) { return f2d(x); }
template <> __device__ __forceinline__ double to_d<double>(double x) { return x; }

// (double)n + (double)f for an integer |n| <= 7 and a float 0 <= f < 1, the
// value the FP64 addition gives.  When f >= 2^-26 the sum has at most 53
// significant bits, so it is exact and is formed by integer operations;
// smaller f take the FP64 addition.
__device__ __forceinline__ double add_nf(int n, float f) {
  const unsigned u = __float_as_uint(f);
  if (u == 0u) return i2d(n);
  const int e = (int)(u >> 23);
  if (e < 101 || n < -7 || n > 7) return i2d(n) + f2d(f);
  const int sh = 150 - e;  // f = m 2^-sh with 24 <= sh <= 49
  const long long S = (long long)n * (1ll << sh) + (long long)((u & 0x7fffffu) | 0x800000u);
  const unsigned long long sign = S < 0 ? (1ull << 63) : 0ull;
  const unsigned long long a = S < 0 ? (unsigned long long)(-S) : (unsigned long long)S;
  const int p = 63 - __clzll((long long)a);  // leading bit; p <= sh + 3 <= 52
  const unsigned long long mant = (a << (52 - p)) & 0xfffffffffffffull;
  return __longlong_as_double((long long)(sign | ((unsigned long long)(1023 + p - sh) << 52) | mant));
}

// ---------------------------------------------------------------------------
// Circle fit (Sec. 2.2, Fig. 3).  Coordinates in cells relative to vertex
// (k,j): the grid line is x = 0, the edge's band 0 <= y <= 1.  Circle through
// A, B, T with origin at A: kap (x^2+y^2) + al x + be y = 0 (a line when
// kap = 0).  The crossing wanted lies on the arc A..B that does not contain
// T, i.e. on the other side of chord AB from T.
// ---------------------------------------------------------------------------

// A third point T of a circle through A and B with its offsets r = T - A and
// t = T - B and their squared lengths.
struct FitPt {
  double rx, ry, r2, tx, ty, t2;
};

__device__ __forceinline__ FitPt fit_pt(double X, double Y, double Ax, double Ay, double Bx,
                                        double By) {
  FitPt p;
  p.rx = X - Ax;
  p.ry = Y - Ay;
  p.r2 = p.rx * p.rx + p.ry * p.ry;
  p.tx = X - Bx;
  p.ty = Y - By;
  p.t2 = p.tx * p.tx + p.ty * p.ty;
  return p;
}

// q = B - A, q2 = |q|^2; (rx, ry) = T - A with r2 = |T - A|^2; t_far: T is
// at least the minimum separation away from B.
__device__ __forceinline__ bool circle_cross_r(double Ay, double x0, double qx, double qy,
                                               double q2, double rx, double ry, double r2,
                                               bool t_far, double* y) {
  if (d_below_sep(r2) || !t_far) return false;
  const double kap = qx * ry - qy * rx;
  const double al = r2 * qy - q2 * ry;
  const double be = q2 * rx - r2 * qx;
  const double c0 = x0 * (kap * x0 + al);
  const double disc = be * be - 4.0 * kap * c0;
  if (d_lt0(disc)) return false;
  const double sq = sqrt(disc);
  const double h = -0.5 * (be + copysign(sq, be));
  if (d_eq0(h)) return false;
  const double ya = c0 / h;
  double yrel = ya;
  if (!d_eq0(kap)) {
    // the far root is formed only when the near one lies on T's side
    const bool kpos = d_gt0(kap);
    const double sa = qx * ya - qy * x0;
    if (kpos ? d_gt0(sa) : d_lt0(sa)) {
      const double yb = h / kap;
      const double sb = qx * yb - qy * x0;
      if (!(kpos ? d_gt0(sb) : d_lt0(sb))) yrel = yb;
    }
  }
  const double best = Ay + yrel;
  if (!d_in01(best)) return false;
  *y = best;
  return true;
}

__device__ __forceinline__ bool circle_cross(double Ay, double x0, double qx, double qy, double q2,
                                             const FitPt& T, double* y) {
  return circle_cross_r(Ay, x0, qx, qy, q2, T.rx, T.ry, T.r2, !d_below_sep(T.t2), y);
}

// Returns the fit kind (D_FIT_*) and the crossing ordinate; T1 (point 1) is
// used when h1, T4 (point 4) when h4.
__device__ __forceinline__ int fit_crossing(double Ax, double Ay, double Bx, double By, bool h1,
                                            const FitPt& T1, bool h4, const FitPt& T4,
                                            bool line_only, double* y) {
  if (d_eq0(Bx)) {
    *y = By;
    return D_FIT_ONLINE;
  }
  const double cx = Bx - Ax, cy = By - Ay;
  const double x0 = -Ax;
  const double c2 = cx * cx + cy * cy;
  if (!line_only && !d_below_sep(c2)) {
    double ys0 = 0.0, ys1 = 0.0;
    int n = 0;
    if (h1 && circle_cross(Ay, x0, cx, cy, c2, T1, &ys0)) ++n;
    if (h4) {
      double t;
      if (circle_cross(Ay, x0, cx, cy, c2, T4, &t)) {
        if (n == 0) ys0 = t; else ys1 = t;
        ++n;
      }
    }
    if (n == 2) {
      *y = 0.5 * (ys0 + ys1);
      return D_FIT_TWO;
    }
    if (n == 1) {
      *y = ys0;
      return D_FIT_ONE;
    }
  }
  // no circle: the chord's own crossing
  *y = Ay + (x0 * cy) / cx;
  return D_FIT_LINE;
}

template <typename R>
__device__ __forceinline__ R to_fraction(double y) {
  R s = (R)y;
  if (!(s >= R(0))) s = R(0);
  if (s >= R(1)) s = below_one<R>();
  return s;
}

template <typename R>
__device__ __forceinline__ void local_xy(const AP<R>& p, int k, int j, double* X, double* Y) {
  *X = i2d(p.ix - k) + to_d<R>(p.fx);
  *Y = i2d(p.jy - j) + to_d<R>(p.fy);
}

// Centre rule (Sec. 2.3): from the new unaligned marker follow the moved
// interface through m0 then m1 while they stay in column col; the first
// aligned marker met that survives the sweep is the partner.  Returns the
// partner's line, or -1 when no aligned marker is reached.
template <class A>
__device__ int walk(const A& S, Mk m0, Mk m1, int col) {
  Mk pts[2] = {m0, m1};
  for (int t = 0; t < 2; ++t) {
    const Mk m = pts[t];
    if (m.kind < 0) return -1;
    const auto p = S.moved(m);
    if (p.ix != col) return -1;
    if (m.kind == 0) {
      const auto L = S.landing(p.ix, m.j);
      return (L.present && L.kept_src == m.i) ? m.j : -1;
    }
  }
  return -1;
}

// Point 1 (near = A) or 4 (near = B) of a fit: the moved marker nb next to
// the chord (found in cell ci,cj), or the marker beyond it when nb is closer
// than the minimum separation to the near end.
template <class A>
__device__ bool far_point(const A& S, Mk nb, int ci, int cj, int k, int j, double ax, double ay,
                          double bx, double by, bool near_a, FitPt* T) {
  if (nb.kind < 0) return false;
  double X, Y;
  local_xy(S.moved(nb), k, j, &X, &Y);
  *T = fit_pt(X, Y, ax, ay, bx, by);
  if (d_below_sep(near_a ? T->r2 : T->t2)) {
    int oi = 0, oj = 0;
    const Mk nn = beyond(S, nb, ci, cj, &oi, &oj);
    if (nn.kind < 0) return false;
    local_xy(S.moved(nn), k, j, &X, &Y);
    *T = fit_pt(X, Y, ax, ay, bx, by);
  }
  return true;
}

// New unaligned marker on interior vertical edge (k,j) (Fig. 2c/2d): the
// moved chords of the old segments of cells k-2..k that cross line k are the
// candidates; one is kept where the new end colours differ.  cnt (nullable)
// receives the fit kinds, cancellations and invariant breaks.
template <typename R>
struct NewV {
  int present, vr, vl;
  int cancelled, invariant;  // candidate pairs cancelled; 1 if the count breaks parity
  R s;
};

// One marker per edge (Sec. 2.4): candidates sorted by (position, generation
// order); an odd count on an edge whose new end colours differ keeps the
// median, an even count on an edge whose colours agree cancels in pairs.
template <typename R>
__device__ NewV<R> select_candidates(int n, double* cy, int* cvr, int* cvl, int* ord, int present) {
  for (int a = 1; a < n; ++a)
    for (int b = a; b > 0 && (cy[b] < cy[b - 1] || (cy[b] == cy[b - 1] && ord[b] < ord[b - 1])); --b) {
      const double t = cy[b]; cy[b] = cy[b - 1]; cy[b - 1] = t;
      int u = cvr[b]; cvr[b] = cvr[b - 1]; cvr[b - 1] = u;
      u = cvl[b]; cvl[b] = cvl[b - 1]; cvl[b - 1] = u;
      u = ord[b]; ord[b] = ord[b - 1]; ord[b - 1] = u;
    }
  NewV<R> out;
  out.present = present;
  out.vr = -1;
  out.vl = -1;
  out.s = R(0.5);
  out.cancelled = 0;
  out.invariant = 0;
  int pick = -1;
  if (present && (n & 1)) {
    pick = n / 2;
    out.cancelled = n / 2;
  } else if (!present && !(n & 1)) {
    out.cancelled = n / 2;
  } else {
    out.invariant = 1;
    if (present && n > 0) {
      pick = 0;
      for (int t = 1; t < n; ++t)
        if (fabs(cy[t] - 0.5) < fabs(cy[pick] - 0.5)) pick = t;
    }
  }
  if (pick >= 0) {
    out.s = to_fraction<R>(cy[pick]);
    out.vr = cvr[pick];
    out.vl = cvl[pick];
  }
  return out;
}

template <typename R, class A>
__device__ NewV<R> new_unaligned(const A& S, bool line_only, int k, int j, int* cnt) {
  double cy[6];
  int cvr[6], cvl[6], ord[6];
  int n = 0;
  for (int c = k - 2; c <= k; ++c) {
    if (c < 0 || c >= S.tnx()) continue;
    int seg[2][2];
    const int ns = cell_segments(S, c, j, seg);
    for (int t = 0; t < ns; ++t) {
      const Mk ma = edge_marker(c, j, seg[t][0]);
      const Mk mb = edge_marker(c, j, seg[t][1]);
      const AP<R> pa = S.moved(ma), pb = S.moved(mb);
      const int lo = min(pa.ix, pb.ix), hi = max(pa.ix, pb.ix);
      if (!(k > lo && k <= hi)) continue;
      const bool a_left = pa.ix < k;
      const Mk mA = a_left ? ma : mb, mB = a_left ? mb : ma;
      const AP<R> A_ = a_left ? pa : pb, B_ = a_left ? pb : pa;
      int c1i = 0, c1j = 0, c4i = 0, c4j = 0;
      const Mk n1 = beyond(S, mA, c, j, &c1i, &c1j);
      const Mk n4 = beyond(S, mB, c, j, &c4i, &c4j);
      double ax, ay, bx, by;
      local_xy(A_, k, j, &ax, &ay);
      local_xy(B_, k, j, &bx, &by);
      FitPt t1{}, t4{};
      const bool h1 = far_point(S, n1, c1i, c1j, k, j, ax, ay, bx, by, true, &t1);
      const bool h4 = far_point(S, n4, c4i, c4j, k, j, ax, ay, bx, by, false, &t4);
      double y;
      const int kind = fit_crossing(ax, ay, bx, by, h1, t1, h4, t4, line_only, &y);
      if (cnt) cnt[kind] += 1;
      const int lr = walk(S, mB, n4, k);
      const int ll = walk(S, mA, n1, k - 1);
      cy[n] = y;
      cvr[n] = lr < 0 ? -1 : !S.knew(k, lr);
      cvl[n] = ll < 0 ? -1 : !S.knew(k, ll);
      ord[n] = n;
      ++n;
    }
  }
  const NewV<R> out = select_candidates<R>(n, cy, cvr, cvl, ord, S.knew(k, j) ^ S.knew(k, j + 1));
  if (cnt) {
    cnt[D_CANCELLED] += out.cancelled;
    cnt[D_INVARIANT] += out.invariant;
  }
  return out;
}

// ---------------------------------------------------------------------------
// Accessor over a state in global memory (sweep coordinates), recomputing.
// ---------------------------------------------------------------------------
template <typename R, int AX, int LD = 0>
struct GView {
  const uint32_t* __restrict__ K;
  const uint32_t* __restrict__ Z;
  const R* __restrict__ sH;
  const R* __restrict__ sV;
  const R* __restrict__ w;  // velocity component along the sweep, (ny+1)x(nx+1)
  Dims d;
  R lam;
  __device__ __forceinline__ int tnx() const { return AX ? d.ny : d.nx; }
  __device__ __forceinline__ int tny() const { return AX ? d.nx : d.ny; }
  __device__ __forceinline__ int kreal(int x, int y) const {
    const long long q = (long long)y * d.kw + (x >> 5);
    return in_range(q, d.nK()) ? (ld_state<LD>(&K[q]) >> (x & 31)) & 1 : 0;
  }
  __device__ __forceinline__ int k(int i, int j) const { return AX ? kreal(j, i) : kreal(i, j); }
  __device__ __forceinline__ int z(int i, int j) const {
    const int x = AX ? j : i, y = AX ? i : j;
    const long long q = (long long)y * d.zw + (x >> 5);
    return in_range(q, d.nZ()) ? (ld_state<LD>(&Z[q]) >> (x & 31)) & 1 : 0;
  }
  __device__ __forceinline__ R h(int i, int j) const {
    const long long q = AX ? (long long)i * d.P + j : (long long)j * d.P + i;
    return in_range(q, AX ? d.nV() : d.nH()) ? ld_state<LD>(AX ? &sV[q] : &sH[q]) : R(0);
  }
  __device__ __forceinline__ R v(int i, int j) const {
    const long long q = AX ? (long long)i * d.P + j : (long long)j * d.P + i;
    return in_range(q, AX ? d.nH() : d.nV()) ? ld_state<LD>(AX ? &sH[q] : &sV[q]) : R(0);
  }
  __device__ __forceinline__ R vel(int i, int j) const {
    const long long q = AX ? (long long)i * (d.nx + 1) + j : (long long)j * (d.nx + 1) + i;
    return in_range(q, d.nW()) ? __ldg(&w[q]) : R(0);
  }
  __device__ AP<R> advect(Mk m, Flags& f) const {
    if (m.kind == 0)
      return move_aligned(m.i, m.j, h(m.i, m.j), vel(m.i, m.j), vel(m.i + 1, m.j), lam, tnx(), f);
    if (m.i == 0 || m.i == tnx())  // wall: no velocity needed
      return move_unaligned(m.i, m.j, v(m.i, m.j), R(0), R(0), lam, tnx(), f);
    return move_unaligned(m.i, m.j, v(m.i, m.j), vel(m.i, m.j), vel(m.i, m.j + 1), lam, tnx(), f);
  }
  __device__ AP<R> moved(Mk m) const {
    Flags f;
    return advect(m, f);
  }
  // L2 prefetch of what advect(m) reads.
  __device__ __forceinline__ void prefetch(Mk m) const {
    const R* s;
    const R* w0;
    const R* w1;
    if (m.kind == 0) {
      s = AX ? &sV[(long long)m.i * d.P + m.j] : &sH[(long long)m.j * d.P + m.i];
      w0 = AX ? &w[(long long)m.i * (d.nx + 1) + m.j] : &w[(long long)m.j * (d.nx + 1) + m.i];
      w1 = AX ? w0 + (d.nx + 1) : w0 + 1;
    } else {
      s = AX ? &sH[(long long)m.i * d.P + m.j] : &sV[(long long)m.j * d.P + m.i];
      w0 = AX ? &w[(long long)m.i * (d.nx + 1) + m.j] : &w[(long long)m.j * (d.nx + 1) + m.i];
      w1 = AX ? w0 + 1 : w0 + (d.nx + 1);
    }
    asm volatile("prefetch.global.L2 [%0];" ::"l"(s));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(w0));
    asm volatile("prefetch.global.L2 [%0];" ::"l"(w1));
  }
  // New corner colour (Sec. 2.3, Fig. 5): vertex i of line j flips once for
  // each aligned marker that passes it; only markers of edges i-1 and i can.
  __device__ int knew(int i, int j) const {
    const int c = k(i, j);
    int r = c;
    if (i >= 1 && k(i - 1, j) != c && moved(Mk{0, i - 1, j}).ix >= i) r ^= 1;
    if (i < tnx() && k(i + 1, j) != c && moved(Mk{0, i, j}).ix < i) r ^= 1;
    return r;
  }
  __device__ Landing<R> landing(int i, int j) const {
    bool valid[3];
    R fx[3];
#pragma unroll
    for (int q = 0; q < 3; ++q) {
      const int e = i - 1 + q;
      valid[q] = false;
      fx[q] = R(0);
      if (e < 0 || e >= tnx() || k(e, j) == k(e + 1, j)) continue;
      const AP<R> p = moved(Mk{0, e, j});
      if (p.ix == i) {
        valid[q] = true;
        fx[q] = p.fx;
      }
    }
    return choose_landing3<R>(valid, fx, i, knew(i, j) ^ knew(i + 1, j));
  }
};


}  // namespace ebit
