// EBIT oracle: a plain, slow, single-threaded CPU restatement of one EBIT
// interface time step, written from the paper (Pan et al., Sec. 2.1-2.5).
//
// TEST INFRASTRUCTURE ONLY.  Only tests/, the smoke check and the CPU-baseline
// leg of bench.py load this code.  It shares no code, header, table or
// constant with the CUDA library, and the library never calls it.
//
// Structure follows the paper's order:
//   init        - colour vertices from the scene, markers by root finding
//                 (Sec. 3.2, marker initialisation)
//   sweep_x     - one direction-split sweep along x (Sec. 2.1, Fig. 2):
//                 aligned markers move by Eq. 4; unaligned markers are moved
//                 (gray points) and replaced by the crossings of the moved
//                 interface with the vertical grid lines, placed by the circle
//                 fit of Sec. 2.2; corner colour vertices flip when a marker
//                 passes them and the centre colour vertex follows the rule of
//                 Sec. 2.3; a marker exists only where the colours of its edge
//                 differ, so two markers meeting on one edge vanish (Sec. 2.4)
//   the y sweep - the same routine applied to the transposed state
//   fraction    - reference-phase area of each cell from the straight
//                 segments joining its markers (Sec. 2.5)
//   curvature   - standard 7x3 height functions on the fractions (Sec. 2.5)
// Readings of passages that the paper leaves open are stated where they are
// used; each one is listed in the design notes of the repository.
//
// Pinned statistically, not exactly: the centre colour that the rule of
// Sec. 2.3 gives a cell that becomes a saddle (four markers) in a sweep.  The
// paper prints no value for it; the pins check the loop counts it implies
// (merging along x, two loops along the diagonal) and, under uniform
// translation where the exact shape is known, that the saddle cells' centre
// colours equal the exact phase at the cell centre in at least 97% of the
// cell-steps (a rule taking the wrong corner fails that).  The GPU must agree
// with this code bit for bit.
//
// Floating point: built with -ffp-contract=off so that every expression is the
// sequence of IEEE operations written here.  R is the state precision (double
// for the FP64 form, float for the FP32 form); the circle fit and the fraction
// arithmetic are double in both forms.

#include "ebit_oracle.h"

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <limits>
#include <vector>

namespace {

template <typename R>
inline R below_one() { return std::nextafter(R(1), R(0)); }

template <typename R>
struct State {
  int nx = 0, ny = 0;
  std::vector<uint8_t> K, Z;
  std::vector<R> sH, sV;
  State(int nx_, int ny_)
      : nx(nx_), ny(ny_), K((size_t)(nx_ + 1) * (ny_ + 1)), Z((size_t)nx_ * ny_),
        sH((size_t)nx_ * (ny_ + 1)), sV((size_t)(nx_ + 1) * ny_) {}
  uint8_t& k(int i, int j) { return K[(size_t)j * (nx + 1) + i]; }
  uint8_t kc(int i, int j) const { return K[(size_t)j * (nx + 1) + i]; }
  uint8_t& z(int i, int j) { return Z[(size_t)j * nx + i]; }
  uint8_t zc(int i, int j) const { return Z[(size_t)j * nx + i]; }
  R& h(int i, int j) { return sH[(size_t)j * nx + i]; }
  R hc(int i, int j) const { return sH[(size_t)j * nx + i]; }
  R& v(int i, int j) { return sV[(size_t)j * (nx + 1) + i]; }
  R vc(int i, int j) const { return sV[(size_t)j * (nx + 1) + i]; }
  // A marker sits on an edge exactly when the colour vertices at its two ends
  // differ (Sec. 2.4).
  bool hasH(int i, int j) const { return kc(i, j) != kc(i + 1, j); }
  bool hasV(int i, int j) const { return kc(i, j) != kc(i, j + 1); }
};

template <typename R>
State<R> load(int nx, int ny, const uint8_t* K, const uint8_t* Z, const double* sH,
              const double* sV) {
  State<R> S(nx, ny);
  for (size_t t = 0; t < S.K.size(); ++t) S.K[t] = K[t] ? 1 : 0;
  for (size_t t = 0; t < S.Z.size(); ++t) S.Z[t] = Z[t] ? 1 : 0;
  for (size_t t = 0; t < S.sH.size(); ++t) S.sH[t] = (R)sH[t];
  for (size_t t = 0; t < S.sV.size(); ++t) S.sV[t] = (R)sV[t];
  return S;
}

template <typename R>
void store(const State<R>& S, uint8_t* K, uint8_t* Z, double* sH, double* sV) {
  std::copy(S.K.begin(), S.K.end(), K);
  std::copy(S.Z.begin(), S.Z.end(), Z);
  for (size_t t = 0; t < S.sH.size(); ++t) sH[t] = (double)S.sH[t];
  for (size_t t = 0; t < S.sV.size(); ++t) sV[t] = (double)S.sV[t];
}

// ---------------------------------------------------------------------------
// Cell topology (Sec. 2.3, Fig. 4).  Corners are numbered counter-clockwise
// 0=(i,j) 1=(i+1,j) 2=(i+1,j+1) 3=(i,j+1); edge e joins corner e and corner
// e+1 (mod 4): 0 bottom, 1 right, 2 top, 3 left.
// ---------------------------------------------------------------------------
struct Mk {
  int kind;  // 0: horizontal edge (i,j); 1: vertical edge (i,j); -1: none
  int i, j;
};

inline Mk edge_marker(int ci, int cj, int e) {
  switch (e) {
    case 0: return {0, ci, cj};
    case 1: return {1, ci + 1, cj};
    case 2: return {0, ci, cj + 1};
    default: return {1, ci, cj};
  }
}

template <typename R>
void corners(const State<R>& S, int i, int j, int c[4]) {
  c[0] = S.kc(i, j);
  c[1] = S.kc(i + 1, j);
  c[2] = S.kc(i + 1, j + 1);
  c[3] = S.kc(i, j + 1);
}

// Segments of the implicit connectivity.  With two markers the segment joins
// them.  With four markers the corners alternate in colour; the centre colour
// vertex selects the pairing: each corner whose colour differs from the centre
// is cut off by the segment joining the markers on its two edges.
template <typename R>
int cell_segments(const State<R>& S, int i, int j, int seg[2][2]) {
  int c[4];
  corners(S, i, j, c);
  int pres[4], n = 0;
  for (int e = 0; e < 4; ++e) {
    pres[e] = c[e] != c[(e + 1) & 3];
    n += pres[e];
  }
  if (n == 0) return 0;
  if (n == 2) {
    int a = -1, b = -1;
    for (int e = 0; e < 4; ++e)
      if (pres[e]) {
        if (a < 0) a = e; else b = e;
      }
    seg[0][0] = a;
    seg[0][1] = b;
    return 1;
  }
  const int zc = S.zc(i, j);
  int m = 0;
  for (int q = 0; q < 4; ++q)
    if (c[q] != zc) {
      seg[m][0] = (q + 3) & 3;
      seg[m][1] = q;
      ++m;
    }
  return m;
}

template <typename R>
int partner_edge(const State<R>& S, int ci, int cj, int e) {
  int seg[2][2];
  const int n = cell_segments(S, ci, cj, seg);
  for (int t = 0; t < n; ++t) {
    if (seg[t][0] == e) return seg[t][1];
    if (seg[t][1] == e) return seg[t][0];
  }
  return -1;
}

// The marker next to m along the interface, on the far side of m's edge as
// seen from cell (ci,cj); kind -1 if that side is outside the domain.
template <typename R>
Mk other_neighbour(const State<R>& S, Mk m, int ci, int cj, int* fi = nullptr, int* fj = nullptr) {
  int oi, oj, oe;
  if (m.kind == 0) {
    oi = m.i;
    if (cj == m.j) { oj = m.j - 1; oe = 2; } else { oj = m.j; oe = 0; }
  } else {
    oj = m.j;
    if (ci == m.i) { oi = m.i - 1; oe = 1; } else { oi = m.i; oe = 3; }
  }
  if (oi < 0 || oj < 0 || oi >= S.nx || oj >= S.ny) return {-1, 0, 0};
  const int pe = partner_edge(S, oi, oj, oe);
  if (pe < 0) return {-1, 0, 0};
  if (fi) { *fi = oi; *fj = oj; }
  return edge_marker(oi, oj, pe);
}

// ---------------------------------------------------------------------------
// Advection along x (Sec. 2.1, Eq. 4).  An advected point is kept as the index
// ix of the vertical grid line at or left of it plus a fraction fx in [0,1),
// so that "left of line k" is the exact integer test ix < k.
// ---------------------------------------------------------------------------
template <typename R>
struct AP {
  int ix;
  R fx;
  int jy;  // y = jy + fy in cell units (unchanged by an x sweep)
  R fy;
};

struct MoveFlags {
  int cfl = 0, clamp = 0;
  double dabs = 0.0;
};

// Marker velocity: bilinear interpolation of the vertex values (Sec. 2.1);
// on a grid line it is the linear interpolation between the two end vertices
// of the marker's edge.  Displacement in cell units d = u dt/dx; |d| <= 1 is
// the CFL limit of the method (Sec. 2.6) and larger values are flagged and
// clipped.
template <typename R>
R displacement(R s, R ua, R ub, R lam, MoveFlags* f) {
  const R vel = (R(1) - s) * ua + s * ub;
  R d = vel * lam;
  const double ad = std::fabs((double)d);
  if (ad == ad && ad > f->dabs) f->dabs = ad;
  if (!(std::fabs(d) <= R(1))) {
    f->cfl = 1;
    d = (d > R(0)) ? R(1) : R(-1);
  }
  return d;
}

template <typename R>
AP<R> advect(const State<R>& S, const R* u, R lam, Mk m, MoveFlags* f) {
  const int nx = S.nx;
  if (m.kind == 0) {
    // Aligned marker: moves along its own horizontal line.
    const R s = S.hc(m.i, m.j);
    const R d = displacement(s, u[(size_t)m.j * (nx + 1) + m.i],
                             u[(size_t)m.j * (nx + 1) + m.i + 1], lam, f);
    const R t = s + d;
    const R fl = std::floor(t);
    R fx = t - fl;
    int sh = (int)fl;
    if (sh > 1) { sh = 1; fx = below_one<R>(); }  // s+d rounded up to 2
    if (fx >= R(1)) fx = below_one<R>();          // t+1 rounded up to 1
    int ix = m.i + sh;
    // Reading: markers cannot leave the domain; they stop at the wall.
    if (ix < 0) { ix = 0; fx = R(0); f->clamp = 1; }
    else if (ix > nx - 1) { ix = nx - 1; fx = below_one<R>(); f->clamp = 1; }
    return {ix, fx, m.j, R(0)};
  }
  const R s = S.vc(m.i, m.j);
  // Reading: markers on the two walls normal to the sweep stay on the wall.
  if (m.i == 0 || m.i == nx) return {m.i, R(0), m.j, s};
  // Unaligned marker: moved off its grid line to the gray point of Fig. 2c.
  const R d = displacement(s, u[(size_t)m.j * (nx + 1) + m.i],
                           u[(size_t)(m.j + 1) * (nx + 1) + m.i], lam, f);
  const R fl = std::floor(d);
  R fx = d - fl;
  if (fx >= R(1)) fx = below_one<R>();
  return {m.i + (int)fl, fx, m.j, s};
}

// ---------------------------------------------------------------------------
// Circle fit (Sec. 2.2, Fig. 3).  Coordinates are in cell units relative to
// the vertex (k,j) at the bottom of the grid segment being crossed, so the
// grid line is x = 0 and the band of the edge is 0 <= y <= 1.
// ---------------------------------------------------------------------------
struct P2 {
  double x, y;
};

// Circle through A, B and T written with origin at A as
//     kap (x^2 + y^2) + al x + be y = 0,
// which stays well defined as the three points become collinear (kap -> 0,
// the circle becomes the line through them).  Its crossings with x = 0 solve
// kap y^2 + be y + c0 = 0.  The interface runs P1-A-B-P4, so the crossing
// wanted is the one on the arc from A to B that does not hold T, i.e. the
// root on the other side of the chord AB from T (the sign of kap is the side
// of T).  That root is returned if it lies in the band.
// Reading: a circle needs three distinct points.  Points closer than 0.01
// cell (an interface passing next to a grid vertex puts a horizontal and a
// vertical marker almost on top of each other) do not determine a circle to
// any useful accuracy.  The sweep therefore takes as points 1 and 4 the next
// markers at least that far from A and B, and a circle whose points are still
// closer than that is not used.
const double kMinSep2 = 1e-4;  // (0.01 cell)^2

bool circle_cross(P2 A, P2 B, P2 T, double* y) {
  const double qx = B.x - A.x, qy = B.y - A.y;
  const double rx = T.x - A.x, ry = T.y - A.y;
  const double tx = T.x - B.x, ty = T.y - B.y;
  const double q2 = qx * qx + qy * qy;
  const double r2 = rx * rx + ry * ry;
  if (r2 < kMinSep2 || tx * tx + ty * ty < kMinSep2) return false;
  const double kap = qx * ry - qy * rx;
  const double al = r2 * qy - q2 * ry;
  const double be = q2 * rx - r2 * qx;
  const double x0 = -A.x;
  const double c0 = x0 * (kap * x0 + al);
  const double disc = be * be - 4.0 * kap * c0;
  if (!(disc >= 0.0)) return false;  // the circle misses the grid line
  const double sq = std::sqrt(disc);
  const double h = -0.5 * (be + std::copysign(sq, be));
  if (h == 0.0) return false;  // coincident points: no circle
  const double ya = c0 / h;  // root that tends to the chord's crossing as kap -> 0
  double yrel = ya;
  if (kap != 0.0) {
    const double yb = h / kap;
    // side of the chord: cross((qx,qy), (x0, y)); T's side has the sign of kap
    const double sa = qx * ya - qy * x0;
    const double sb = qx * yb - qy * x0;
    const bool a_with_T = (sa > 0.0 && kap > 0.0) || (sa < 0.0 && kap < 0.0);
    const bool b_with_T = (sb > 0.0 && kap > 0.0) || (sb < 0.0 && kap < 0.0);
    if (a_with_T && !b_with_T) yrel = yb;
  }
  const double best = A.y + yrel;
  if (!(best >= 0.0 && best <= 1.0)) return false;  // outside the band
  *y = best;
  return true;
}

// New unaligned marker on the crossing of the moved chord A'B' with the grid
// line.  A' is left of the line (x < 0), B' at or right of it.  P1 is the
// moved neighbour beyond A', P4 the one beyond B' (points 1-4 of Fig. 3): the
// circles (P1,A',B') and (A',B',P4) are intersected with the line and the
// surviving crossings averaged; with none, the chord crossing is used (the
// straight-line fit of the first EBIT version).
int fit_crossing(P2 A, P2 B, const P2* P1, const P2* P4, bool line_only, double* y) {
  if (B.x == 0.0) {
    *y = B.y;
    return ORC_FIT_ONLINE;
  }
  const double x0 = -A.x;
  const double ystar = A.y + (x0 * (B.y - A.y)) / (B.x - A.x);
  const double cx = B.x - A.x, cy = B.y - A.y;
  // a chord shorter than the minimum separation: its own crossing is within
  // O(len^2 * curvature) of the interface
  if (!line_only && cx * cx + cy * cy >= kMinSep2) {
    double ys[2];
    int n = 0;
    if (P1 && circle_cross(A, B, *P1, &ys[n])) ++n;
    if (P4 && circle_cross(A, B, *P4, &ys[n])) ++n;
    if (n == 2) {
      *y = 0.5 * (ys[0] + ys[1]);
      return ORC_FIT_TWO;
    }
    if (n == 1) {
      *y = ys[0];
      return ORC_FIT_ONE;
    }
  }
  *y = ystar;
  return ORC_FIT_LINE;
}

template <typename R>
R to_fraction(double y) {
  R s = (R)y;
  if (!(s >= R(0))) s = R(0);
  if (s >= R(1)) s = below_one<R>();
  return s;
}

template <typename R>
P2 local(const AP<R>& p, int k, int j) {
  return {(double)(p.ix - k) + (double)p.fx, (double)(p.jy - j) + (double)p.fy};
}

// ---------------------------------------------------------------------------
// One sweep along x.
// ---------------------------------------------------------------------------
template <typename R>
void sweep_x(State<R>& S, const R* u, R lam, bool line_only, int64_t* ctr, double* maxcfl) {
  const int nx = S.nx, ny = S.ny;
  State<R> N = S;
  std::fill(N.sH.begin(), N.sH.end(), R(0));
  for (int j = 0; j < ny; ++j)
    for (int i = 1; i < nx; ++i) N.v(i, j) = R(0);

  auto move = [&](Mk m) {
    MoveFlags f;
    return advect(S, u, lam, m, &f);
  };

  // 1. Aligned markers move along their line (Eq. 4, Fig. 2b).  A corner
  //    colour vertex flips once for each marker that passes it (Fig. 5):
  //    marker from edge i to edge ix passes the vertices min(i,ix)+1..max(i,ix).
  struct Land {
    int i, j;
    R fx;
    int src;
  };
  std::vector<Land> land;
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i) {
      if (!S.hasH(i, j)) continue;
      MoveFlags f;
      const AP<R> p = advect(S, u, lam, {0, i, j}, &f);
      ctr[ORC_CFL] += f.cfl;
      ctr[ORC_WALL_CLAMP] += f.clamp;
      *maxcfl = std::max(*maxcfl, f.dabs);
      for (int kk = std::min(i, p.ix) + 1; kk <= std::max(i, p.ix); ++kk) N.k(kk, j) ^= 1;
      land.push_back({p.ix, j, p.fx, i});
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 1; i < nx; ++i) {
      if (!S.hasV(i, j)) continue;
      MoveFlags f;
      advect(S, u, lam, {1, i, j}, &f);
      ctr[ORC_CFL] += f.cfl;
      *maxcfl = std::max(*maxcfl, f.dabs);
    }

  // 2. Landed aligned markers.  An edge keeps a marker only if its end
  //    colours differ; two markers on one edge therefore cancel (Sec. 2.4).
  //    Reading: three on one edge keep the middle one.
  std::sort(land.begin(), land.end(), [](const Land& a, const Land& b) {
    if (a.j != b.j) return a.j < b.j;
    if (a.i != b.i) return a.i < b.i;
    if (a.fx != b.fx) return a.fx < b.fx;
    return a.src < b.src;
  });
  std::vector<int32_t> keep((size_t)nx * (ny + 1), -1);  // source edge kept
  std::vector<uint8_t> landed((size_t)nx * (ny + 1), 0);
  for (size_t a = 0; a < land.size();) {
    size_t b = a;
    while (b < land.size() && land[b].i == land[a].i && land[b].j == land[a].j) ++b;
    const int i = land[a].i, j = land[a].j;
    const size_t n = b - a;
    const bool present = N.hasH(i, j);
    landed[(size_t)j * nx + i] = 1;
    if (present && (n & 1)) {
      ctr[ORC_CANCELLED] += (int64_t)(n / 2);  // the pairs around the middle one
      const Land& m = land[a + n / 2];
      N.h(i, j) = m.fx;
      keep[(size_t)j * nx + i] = m.src;
    } else if (!present && !(n & 1)) {
      ctr[ORC_CANCELLED] += (int64_t)(n / 2);
    } else {
      ctr[ORC_INVARIANT] += 1;
      if (present) {
        size_t best = a;
        for (size_t t = a; t < b; ++t)
          if (std::fabs((double)land[t].fx - 0.5) < std::fabs((double)land[best].fx - 0.5))
            best = t;
        N.h(i, j) = land[best].fx;
        keep[(size_t)j * nx + i] = land[best].src;
      }
    }
    a = b;
  }
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (N.hasH(i, j) && !landed[(size_t)j * nx + i]) {
        ctr[ORC_INVARIANT] += 1;
        N.h(i, j) = R(0.5);
      }

  auto survives = [&](Mk m, const AP<R>& p) {
    return N.hasH(p.ix, m.j) && keep[(size_t)m.j * nx + p.ix] == m.i;
  };
  // Centre rule of Sec. 2.3 (reading): from the new unaligned marker, follow
  // the moved interface into the cell through the listed moved points while
  // they stay in the cell's column; the first aligned marker met that still
  // exists after the sweep is the partner, and the segment joining the two
  // cuts off the corner at (k, line of the partner).  Returns that line or -1
  // (no aligned marker reached: the paper's step (3), nothing to update).
  auto walk = [&](Mk m0, Mk m1, int col) -> int {
    const Mk pts[2] = {m0, m1};
    for (int t = 0; t < 2; ++t) {
      const Mk m = pts[t];
      if (m.kind < 0) return -1;
      const AP<R> p = move(m);
      if (p.ix != col) return -1;
      if (m.kind == 0) return survives(m, p) ? m.j : -1;
    }
    return -1;
  };

  // 3. Moved chords of the old segments crossing interior vertical lines give
  //    the candidates for the new unaligned markers (Fig. 2c/2d).
  struct Cand {
    int k, j, order;
    double y;
    int vr, vl;  // centre colour for the cell right / left of the edge, or -1
  };
  std::vector<Cand> cand;
  int order = 0;
  for (int j = 0; j < ny; ++j)
    for (int c = 0; c < nx; ++c) {
      int seg[2][2];
      const int ns = cell_segments(S, c, j, seg);
      for (int t = 0; t < ns; ++t) {
        const Mk ma = edge_marker(c, j, seg[t][0]);
        const Mk mb = edge_marker(c, j, seg[t][1]);
        const AP<R> pa = move(ma), pb = move(mb);
        const int lo = std::max(std::min(pa.ix, pb.ix) + 1, 1);
        const int hi = std::min(std::max(pa.ix, pb.ix), nx - 1);
        for (int k = lo; k <= hi; ++k) {
          const bool a_left = pa.ix < k;
          const Mk mA = a_left ? ma : mb, mB = a_left ? mb : ma;
          const AP<R> A = a_left ? pa : pb, B = a_left ? pb : pa;
          int c1i = 0, c1j = 0, c4i = 0, c4j = 0;
          const Mk n1 = other_neighbour(S, mA, c, j, &c1i, &c1j);
          const Mk n4 = other_neighbour(S, mB, c, j, &c4i, &c4j);
          const P2 a = local(A, k, j), b = local(B, k, j);
          // points 1 and 4 of Fig. 3: the next markers along the interface
          // beyond A and B that are at least the minimum separation away
          auto far_point = [&](Mk nb, int ci, int cj, P2 from, P2* out) -> bool {
            if (nb.kind < 0) return false;
            P2 q = local(move(nb), k, j);
            const double ex = q.x - from.x, ey = q.y - from.y;
            if (ex * ex + ey * ey < kMinSep2) {
              const Mk nn = other_neighbour(S, nb, ci, cj);
              if (nn.kind < 0) return false;
              q = local(move(nn), k, j);
            }
            *out = q;
            return true;
          };
          P2 q1{0, 0}, q4{0, 0};
          const bool h1 = far_point(n1, c1i, c1j, a, &q1);
          const bool h4 = far_point(n4, c4i, c4j, b, &q4);
          double y = 0.0;
          const int kind = fit_crossing(a, b, h1 ? &q1 : nullptr, h4 ? &q4 : nullptr,
                                        line_only, &y);
          ctr[kind] += 1;
          const int lr = walk(mB, n4, k);
          const int ll = walk(mA, n1, k - 1);
          const int vr = lr < 0 ? -1 : !N.kc(k, lr);
          const int vl = ll < 0 ? -1 : !N.kc(k, ll);
          cand.push_back({k, j, order++, y, vr, vl});
        }
      }
    }

  // 4. One marker per edge: keep a candidate only where the new colours of
  //    the edge's ends differ (Sec. 2.4).  Reading: an odd count keeps the
  //    median by position.
  std::sort(cand.begin(), cand.end(), [](const Cand& a, const Cand& b) {
    if (a.j != b.j) return a.j < b.j;
    if (a.k != b.k) return a.k < b.k;
    if (a.y != b.y) return a.y < b.y;
    return a.order < b.order;
  });
  std::vector<int8_t> from_left((size_t)nx * ny, -1), from_right((size_t)nx * ny, -1);
  std::vector<uint8_t> got((size_t)(nx + 1) * ny, 0);
  for (size_t a = 0; a < cand.size();) {
    size_t b = a;
    while (b < cand.size() && cand[b].k == cand[a].k && cand[b].j == cand[a].j) ++b;
    const int k = cand[a].k, j = cand[a].j;
    const size_t n = b - a;
    const bool present = N.hasV(k, j);
    got[(size_t)j * (nx + 1) + k] = 1;
    const Cand* pick = nullptr;
    if (present && (n & 1)) {
      ctr[ORC_CANCELLED] += (int64_t)(n / 2);
      pick = &cand[a + n / 2];
    } else if (!present && !(n & 1)) {
      ctr[ORC_CANCELLED] += (int64_t)(n / 2);
    } else {
      ctr[ORC_INVARIANT] += 1;
      if (present) {
        pick = &cand[a];
        for (size_t t = a; t < b; ++t)
          if (std::fabs(cand[t].y - 0.5) < std::fabs(pick->y - 0.5)) pick = &cand[t];
      }
    }
    if (pick) {
      N.v(k, j) = to_fraction<R>(pick->y);
      from_left[(size_t)j * nx + k] = (int8_t)pick->vr;       // cell (k,j)
      from_right[(size_t)j * nx + k - 1] = (int8_t)pick->vl;  // cell (k-1,j)
    }
    a = b;
  }
  for (int j = 0; j < ny; ++j)
    for (int k = 1; k < nx; ++k)
      if (N.hasV(k, j) && !got[(size_t)j * (nx + 1) + k]) {
        ctr[ORC_INVARIANT] += 1;
        N.v(k, j) = R(0.5);
      }
  // Wall markers stay; their colours cannot change because no aligned marker
  // crosses a wall, so presence there is unchanged.

  // 5. Centre colour vertices of cells with four markers after the sweep.
  //    Reading: when the two unaligned markers of a cell disagree, the one on
  //    the cell's left edge decides.
  for (int j = 0; j < ny; ++j)
    for (int c = 0; c < nx; ++c) {
      int q[4];
      corners(N, c, j, q);
      const bool four = q[0] != q[1] && q[1] != q[2] && q[2] != q[3] && q[3] != q[0];
      if (!four) continue;
      const int a = from_left[(size_t)j * nx + c], b = from_right[(size_t)j * nx + c];
      if (a >= 0) {
        N.z(c, j) = (uint8_t)a;
        ctr[ORC_ZSET] += 1;
        if (b >= 0 && b != a) ctr[ORC_ZCONFLICT] += 1;
      } else if (b >= 0) {
        N.z(c, j) = (uint8_t)b;
        ctr[ORC_ZSET] += 1;
      }
    }
  S = std::move(N);
}

// The y sweep is the x sweep of the transposed grid: vertex (i,j) becomes
// (j,i), so horizontal edges become vertical edges and vice versa.
template <typename R>
State<R> transposed(const State<R>& S) {
  State<R> T(S.ny, S.nx);
  for (int j = 0; j <= S.ny; ++j)
    for (int i = 0; i <= S.nx; ++i) T.k(j, i) = S.kc(i, j);
  for (int j = 0; j < S.ny; ++j)
    for (int i = 0; i < S.nx; ++i) T.z(j, i) = S.zc(i, j);
  for (int j = 0; j <= S.ny; ++j)
    for (int i = 0; i < S.nx; ++i) T.v(j, i) = S.hc(i, j);
  for (int j = 0; j < S.ny; ++j)
    for (int i = 0; i <= S.nx; ++i) T.h(j, i) = S.vc(i, j);
  return T;
}

template <typename R>
void sweep(State<R>& S, int axis, const double* vel, double lam, bool line_only,
           int64_t* ctr, double* maxcfl) {
  const int nx = S.nx, ny = S.ny;
  std::vector<R> w((size_t)(nx + 1) * (ny + 1));
  const R lamR = (R)lam;
  if (axis == 0) {
    for (size_t t = 0; t < w.size(); ++t) w[t] = (R)vel[t];
    sweep_x(S, w.data(), lamR, line_only, ctr, maxcfl);
  } else {
    // transposed vertex (a,b) is vertex (b,a): velocity index b*(nx+1)+a
    for (int a = 0; a <= nx; ++a)
      for (int b = 0; b <= ny; ++b) w[(size_t)a * (ny + 1) + b] = (R)vel[(size_t)b * (nx + 1) + a];
    State<R> T = transposed(S);
    sweep_x(T, w.data(), lamR, line_only, ctr, maxcfl);
    S = transposed(T);
  }
}

// ---------------------------------------------------------------------------
// Volume fraction (Sec. 2.5): reference-phase area of the cell bounded by the
// straight segments joining its markers, in cell units.  Double arithmetic.
// ---------------------------------------------------------------------------
template <typename R>
double cell_fraction(const State<R>& S, int i, int j) {
  int c[4];
  corners(S, i, j, c);
  const double s[4] = {(double)S.hc(i, j), (double)S.vc(i + 1, j), (double)S.hc(i, j + 1),
                       (double)S.vc(i, j)};
  int pres[4], n = 0;
  for (int e = 0; e < 4; ++e) {
    pres[e] = c[e] != c[(e + 1) & 3];
    n += pres[e];
  }
  if (n == 0) return (double)c[0];
  // Triangle cut off at corner q: legs along edge (q+3)%4 and edge q.
  auto tri = [&](int q) {
    double a, b;
    switch (q) {
      case 0: a = s[3]; b = s[0]; break;
      case 1: a = 1.0 - s[0]; b = s[1]; break;
      case 2: a = 1.0 - s[1]; b = 1.0 - s[2]; break;
      default: a = s[2]; b = 1.0 - s[3]; break;
    }
    return 0.5 * (a * b);
  };
  if (n == 2) {
    int e1 = -1, e2 = -1;
    for (int e = 0; e < 4; ++e)
      if (pres[e]) {
        if (e1 < 0) e1 = e; else e2 = e;
      }
    if (e2 - e1 == 2) {
      if (e1 == 0) {  // bottom and top: trapezoid measured from the left side
        return c[0] ? 0.5 * (s[0] + s[2]) : 0.5 * ((1.0 - s[0]) + (1.0 - s[2]));
      }
      // right and left: trapezoid measured from the bottom side
      return c[0] ? 0.5 * (s[3] + s[1]) : 0.5 * ((1.0 - s[3]) + (1.0 - s[1]));
    }
    const int q = (e1 == 0 && e2 == 3) ? 0 : e2;
    const double T = tri(q);
    return c[q] ? T : 1.0 - T;
  }
  const int zc = S.zc(i, j);
  double Tsum = 0.0;
  bool first = true;
  for (int q = 0; q < 4; ++q)
    if (c[q] != zc) {
      if (first) { Tsum = tri(q); first = false; } else { Tsum = Tsum + tri(q); }
    }
  return zc == 0 ? Tsum : 1.0 - Tsum;
}

template <typename R>
double fraction(const State<R>& S, double dx, double* C) {
  double acc = 0.0;
  for (int j = 0; j < S.ny; ++j)
    for (int i = 0; i < S.nx; ++i) {
      const double f = cell_fraction(S, i, j);
      C[(size_t)j * S.nx + i] = (double)(R)f;
      acc += f;
    }
  return acc * (dx * dx);
}

// ---------------------------------------------------------------------------
// Height-function curvature (Sec. 2.5): the standard 7x3 height functions,
// and, when asked for, the generalised fallbacks of the height-function
// method the paper cites (Popinet 2009): the stencil along the other
// direction, then a parabola fitted to the heights of both directions
// ("mixed heights"), then a parabola fitted to the markers of the 3x3 block
// (where the volume-of-fluid form fits interface-fragment centroids, the
// markers give points that lie on the interface).
//
// Precision (reading): the heights and the fits run in the state precision R.
// Their inputs are the state's own fractions and marker positions, which the
// FP32 form holds to 2^-24; a three-parameter parabola fitted over a window of
// about three cells with points at least half a cell apart has normal
// equations of moderate condition once the ill-determined ones are refused
// (the regularity test below), so float arithmetic moves kappa by ~1e-6
// relative (1e-4 at most), while the fit's own error against the curvature of
// the interface it samples is ~3e-2 (kappa r - 1 on disks of 3-8 cells).  The
// pins compare the two forms' fallback curvatures to show exactly that.
// ---------------------------------------------------------------------------

// Curvature of the parabola z = a s^2 + b s + c fitted by weighted least
// squares to the points (X, Y) (cell units), in the frame with origin (ox, oy)
// and unit normal (nx, ny) pointing out of the reference phase (tangent
// (ny, -nx)), evaluated at s = 0: kappa = -2a / (1 + b^2)^(3/2) / dx, which is
// +1/R for a reference-phase drop of radius R.  The normal equations are
// solved by Cramer's rule, in the arithmetic R.  Returns false when the
// system is ill-determined (|det| <= 1e-3 S4 S2 S0).
template <typename R>
bool parabola_kappa(int n, const R* X, const R* Y, const R* W, R ox, R oy, R nx, R ny, R dx,
                    R* kappa) {
  R S0 = R(0), S1 = R(0), S2 = R(0), S3 = R(0), S4 = R(0), T0 = R(0), T1 = R(0), T2 = R(0);
  for (int p = 0; p < n; ++p) {
    const R ddx = X[p] - ox, ddy = Y[p] - oy;
    const R sv = ddx * ny - ddy * nx;  // along the tangent (ny, -nx)
    const R zv = ddx * nx + ddy * ny;  // along the normal
    const R w = W[p];
    const R s2 = sv * sv;
    S0 = S0 + w;
    S1 = S1 + w * sv;
    S2 = S2 + w * s2;
    S3 = S3 + w * (s2 * sv);
    S4 = S4 + w * (s2 * s2);
    T0 = T0 + w * zv;
    T1 = T1 + w * (zv * sv);
    T2 = T2 + w * (zv * s2);
  }
  const R m00 = S2 * S0 - S1 * S1;
  const R m01 = S3 * S0 - S1 * S2;
  const R m02 = S3 * S1 - S2 * S2;
  const R det = S4 * m00 - S3 * m01 + S2 * m02;
  // regular: |det| above 1e-3 of the product of the diagonal of the (positive
  // definite) normal matrix, which bounds it (Hadamard); the same test in
  // both precisions
  const R eps = R(1e-3);
  if (!(std::fabs(det) > eps * (S4 * S2 * S0))) return false;
  const R u1 = T1 * S0 - S1 * T0;
  const R da = T2 * m00 - S3 * u1 + S2 * (T1 * S1 - S2 * T0);
  const R db = S4 * u1 - T2 * m01 + S2 * (S3 * T0 - T1 * S2);
  const R a = da / det, b = db / det;
  const R q = R(1) + b * b;
  *kappa = (R(-2) * a) / (q * std::sqrt(q)) / dx;
  return std::isfinite(*kappa);
}

template <typename R>
void curvature(const State<R>& S, const double* Cd, double dx, double* kappa, int64_t* ctr,
               bool ghf) {
  const int nx = S.nx, ny = S.ny;
  std::vector<R> C((size_t)nx * ny);
  for (size_t t = 0; t < C.size(); ++t) C[t] = (R)Cd[t];
  auto cf = [&](int i, int j) { return C[(size_t)j * nx + i]; };
  const R dxR = (R)dx;
  const R nanv = std::numeric_limits<R>::quiet_NaN();
  // The column of seven cells through (i+m, j-3..j+3) (ycol) or the row
  // (i-3..i+3, j+m): its count h of reference-phase cells and its
  // orientation: 1 when the low end is reference phase and the high end is
  // not, -1 for the reverse, 0 when the column is not a valid height (an end
  // cell is mixed, both ends agree, or it leaves the domain).
  auto column = [&](int i, int j, int m, bool ycol, R* h) -> int {
    const bool in = ycol ? (i + m >= 0 && i + m <= nx - 1 && j - 3 >= 0 && j + 3 <= ny - 1)
                         : (j + m >= 0 && j + m <= ny - 1 && i - 3 >= 0 && i + 3 <= nx - 1);
    if (!in) return 0;
    R acc = R(0);
    for (int t = -3; t <= 3; ++t) acc = acc + (ycol ? cf(i + m, j + t) : cf(i + t, j + m));
    *h = acc;
    const R lo = ycol ? cf(i + m, j - 3) : cf(i - 3, j + m);
    const R hi = ycol ? cf(i + m, j + 3) : cf(i + 3, j + m);
    return (lo == R(1) && hi == R(0)) ? 1 : (lo == R(0) && hi == R(1)) ? -1 : 0;
  };
  // The standard 7x3 stencil: three valid columns of one orientation.
  auto stencil = [&](int i, int j, bool ycol, double* out) -> bool {
    R h[3];
    int orient[3];
    for (int m = -1; m <= 1; ++m) orient[m + 1] = column(i, j, m, ycol, &h[m + 1]);
    if (orient[0] == 0 || orient[0] != orient[1] || orient[1] != orient[2]) return false;
    // h counts reference-phase cells in the column, so for either
    // orientation kappa = -h'' / (dx (1 + h'^2)^(3/2)) is positive for a
    // reference-phase drop.
    const R hp = (h[2] - h[0]) * R(0.5);
    const R hpp = (h[2] - h[1]) - (h[1] - h[0]);
    const R q = R(1) + hp * hp;
    const R den = dxR * (q * std::sqrt(q));
    *out = (double)(-hpp / den);
    return true;
  };
  const R one = R(1), zero = R(0);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      double& out = kappa[(size_t)j * nx + i];
      int c[4];
      corners(S, i, j, c);
      if (c[0] == c[1] && c[1] == c[2] && c[2] == c[3]) {
        out = (double)nanv;
        continue;
      }
      // Orientation from the cell's own segments: heights are taken along y
      // when the segments are at least as long in x as in y.
      const R px[4] = {S.hc(i, j), one, S.hc(i, j + 1), zero};
      const R py[4] = {zero, S.vc(i + 1, j), one, S.vc(i, j)};
      int seg[2][2];
      const int ns = cell_segments(S, i, j, seg);
      R ax = R(0), ay = R(0);
      for (int t = 0; t < ns; ++t) {
        const int a = seg[t][0], b = seg[t][1];
        ax = ax + std::fabs(px[b] - px[a]);
        ay = ay + std::fabs(py[b] - py[a]);
      }
      const bool ycol = ax >= ay;
      if (stencil(i, j, ycol, &out)) continue;
      ctr[ORC_HF_INVALID] += 1;
      out = (double)nanv;
      if (!ghf) continue;
      // 1. the standard stencil along the other direction
      if (stencil(i, j, !ycol, &out)) {
        ctr[ORC_HF_OTHER] += 1;
        continue;
      }
      out = (double)nanv;
      // The fits work in the state precision, in cell units relative to the
      // cell's lower-left corner.  The frame needs the cell's single segment
      // A->B: origin at its midpoint, normal perpendicular to it, turned
      // away from the reference-phase corners (their offsets from the cell
      // centre, each signed by colour, sum to a vector into the reference
      // phase).
      if (ns != 1) continue;
      const int ea = seg[0][0], eb = seg[0][1];
      const R Ax = px[ea], Ay = py[ea], Bx = px[eb], By = py[eb];
      const R ox = (Ax + Bx) * R(0.5), oy = (Ay + By) * R(0.5);
      R n0x = By - Ay, n0y = -(Bx - Ax);
      static const int sxc[4] = {-1, 1, 1, -1}, syc[4] = {-1, -1, 1, 1};
      int gx = 0, gy = 0;
      for (int q = 0; q < 4; ++q) {
        gx += (2 * c[q] - 1) * sxc[q];
        gy += (2 * c[q] - 1) * syc[q];
      }
      const R dot = n0x * (R)gx + n0y * (R)gy;
      if (dot == R(0)) continue;
      if (dot > R(0)) {
        n0x = -n0x;
        n0y = -n0y;
      }
      const R len = std::sqrt(n0x * n0x + n0y * n0y);
      if (!(len > R(0))) continue;
      const R unx = n0x / len, uny = n0y / len;
      // Points kept only when at least half a cell from every point already
      // kept (independent positions).
      R X[32], Y[32], W[32];  // at most 24 markers on the 3x3 block
      int np = 0;
      auto add = [&](R x, R y) {
        for (int p = 0; p < np; ++p) {
          const R ex = x - X[p], ey = y - Y[p];
          if (ex * ex + ey * ey < R(0.25)) return;
        }
        X[np] = x;
        Y[np] = y;
        W[np] = R(1);
        ++np;
      };
      // 2. mixed heights: every valid column of the cell's stencils in both
      // directions gives the interface point on its centre line
      for (int dir = 0; dir < 2; ++dir) {
        const bool yc = dir == 0;
        for (int m = -1; m <= 1; ++m) {
          R h = R(0);
          const int o = column(i, j, m, yc, &h);
          if (o == 0) continue;
          const R pos = o == 1 ? R(-3) + h : R(4) - h;
          const R mid = (R)m + R(0.5);
          if (yc) add(mid, pos);
          else add(pos, mid);
        }
      }
      R kv = R(0);
      if (np >= 3 && parabola_kappa<R>(np, X, Y, W, ox, oy, unx, uny, dxR, &kv)) {
        out = (double)kv;
        ctr[ORC_HF_MIXED] += 1;
        continue;
      }
      // 3. the markers on the edges of the 3x3 block of cells around the
      // cell (interface points on the grid lines)
      np = 0;
      for (int b = j - 1; b <= j + 2; ++b)
        for (int a = i - 1; a <= i + 1; ++a)
          if (a >= 0 && a < nx && b >= 0 && b <= ny && S.hasH(a, b))
            add((R)(a - i) + S.hc(a, b), (R)(b - j));
      for (int b = j - 1; b <= j + 1; ++b)
        for (int a = i - 1; a <= i + 2; ++a)
          if (a >= 0 && a <= nx && b >= 0 && b < ny && S.hasV(a, b))
            add((R)(a - i), (R)(b - j) + S.vc(a, b));
      if (np >= 3 && parabola_kappa<R>(np, X, Y, W, ox, oy, unx, uny, dxR, &kv)) {
        out = (double)kv;
        ctr[ORC_HF_MARKERS] += 1;
      }
    }
}

// ---------------------------------------------------------------------------
// Initialisation (Sec. 3.2): colour vertices from the scene, markers by root
// finding on edges whose end colours differ.
// ---------------------------------------------------------------------------
struct Scene {
  const orc_scene* s;
  double curve_h(double x) const {
    double acc = s->y0;
    for (int k = 1; k <= s->nmodes; ++k) {
      const double arg = (6.283185307179586 * (double)k) * x + s->phase[k - 1];
      acc = acc + s->amp[k - 1] * std::cos(arg);
    }
    return acc;
  }
  bool in_curve(double x, double y) const { return y <= curve_h(x); }
  bool in_line(int l, double x, double y) const { return s->la[l] * x + s->lb[l] * y <= s->lc[l]; }
  bool in_circle(int c, double x, double y) const {
    const double ddx = x - s->xc[c], ddy = y - s->yc[c];
    return ddx * ddx + ddy * ddy <= s->r[c] * s->r[c];
  }
  bool in_notch(double x, double y) const {
    for (int b = 0; b < s->nnotches; ++b) {
      const double* q = s->notch + 4 * b;
      if (x >= q[0] && x <= q[1] && y >= q[2] && y <= q[3]) return true;
    }
    return false;
  }
  // The scene's phase at a point: curve, half-planes and circles toggle it,
  // then the notches cut it out.
  bool inside(double x, double y) const {
    bool p = false;
    if (s->has_curve) p ^= in_curve(x, y);
    for (int l = 0; l < s->nlines; ++l) p ^= in_line(l, x, y);
    for (int c = 0; c < s->ncircles; ++c) p ^= in_circle(c, x, y);
    return p && !in_notch(x, y);
  }
  // Does the edge from (xa, ya) to (xb, yb) (axis-aligned, xa <= xb, ya <= yb)
  // touch a notch box?
  bool touches_notch(double xa, double ya, double xb, double yb) const {
    for (int b = 0; b < s->nnotches; ++b) {
      const double* q = s->notch + 4 * b;
      if (xb >= q[0] && xa <= q[1] && yb >= q[2] && ya <= q[3]) return true;
    }
    return false;
  }
};

template <typename R>
void init(State<R>& S, double dx, const orc_scene* sc) {
  const int nx = S.nx, ny = S.ny;
  const Scene P{sc};
  // colour of every vertex and cell centre: curve, half-planes, then each
  // circle toggles inside itself
  std::vector<double> hcol(nx + 1);
  if (sc->has_curve)
    for (int i = 0; i <= nx; ++i) hcol[i] = P.curve_h(i * dx);
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      int p = 0;
      if (sc->has_curve) p ^= (j * dx) <= hcol[i];
      for (int l = 0; l < sc->nlines; ++l) p ^= P.in_line(l, i * dx, j * dx);
      S.k(i, j) = (uint8_t)p;
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double x = (i + 0.5) * dx, y = (j + 0.5) * dx;
      int p = 0;
      if (sc->has_curve) p ^= P.in_curve(x, y);
      for (int l = 0; l < sc->nlines; ++l) p ^= P.in_line(l, x, y);
      S.z(i, j) = (uint8_t)p;
    }
  auto bbox = [&](int c, int* i0, int* i1, int* j0, int* j1) {
    *i0 = std::max(0, (int)std::floor((sc->xc[c] - sc->r[c]) / dx) - 1);
    *i1 = std::min(nx, (int)std::ceil((sc->xc[c] + sc->r[c]) / dx) + 1);
    *j0 = std::max(0, (int)std::floor((sc->yc[c] - sc->r[c]) / dx) - 1);
    *j1 = std::min(ny, (int)std::ceil((sc->yc[c] + sc->r[c]) / dx) + 1);
  };
  for (int c = 0; c < sc->ncircles; ++c) {
    int i0, i1, j0, j1;
    bbox(c, &i0, &i1, &j0, &j1);
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i) {
        if (P.in_circle(c, i * dx, j * dx)) S.k(i, j) ^= 1;
        if (i < nx && j < ny && P.in_circle(c, (i + 0.5) * dx, (j + 0.5) * dx)) S.z(i, j) ^= 1;
      }
  }
  // notches: vertices and cell centres inside a box leave the reference phase
  if (sc->nnotches)
    for (int j = 0; j <= ny; ++j)
      for (int i = 0; i <= nx; ++i) {
        if (P.in_notch(i * dx, j * dx)) S.k(i, j) = 0;
        if (i < nx && j < ny && P.in_notch((i + 0.5) * dx, (j + 0.5) * dx)) S.z(i, j) = 0;
      }
  // Owner of each edge's marker: a notch when the edge touches one of the
  // boxes, else the curve, then the half-plane and then the circle of lowest
  // index whose own inside test differs at the two ends of the edge.
  const int OWN_NOTCH = -4, OWN_NONE = -3, OWN_CURVE = -2, OWN_LINE = -10;  // line l: -10 - l
  std::vector<int32_t> ownH((size_t)nx * (ny + 1), OWN_NONE), ownV((size_t)(nx + 1) * ny, OWN_NONE);
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i) {
      if (!S.hasH(i, j)) continue;
      int32_t& o = ownH[(size_t)j * nx + i];
      if (sc->nnotches && P.touches_notch(i * dx, j * dx, (i + 1) * dx, j * dx)) o = OWN_NOTCH;
      else if (sc->has_curve && ((j * dx) <= hcol[i]) != ((j * dx) <= hcol[i + 1])) o = OWN_CURVE;
      else
        for (int l = 0; l < sc->nlines; ++l)
          if (P.in_line(l, i * dx, j * dx) != P.in_line(l, (i + 1) * dx, j * dx)) {
            o = OWN_LINE - l;
            break;
          }
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      if (!S.hasV(i, j)) continue;
      int32_t& o = ownV[(size_t)j * (nx + 1) + i];
      if (sc->nnotches && P.touches_notch(i * dx, j * dx, i * dx, (j + 1) * dx)) o = OWN_NOTCH;
      else if (sc->has_curve && ((j * dx) <= hcol[i]) != (((j + 1) * dx) <= hcol[i])) o = OWN_CURVE;
      else
        for (int l = 0; l < sc->nlines; ++l)
          if (P.in_line(l, i * dx, j * dx) != P.in_line(l, i * dx, (j + 1) * dx)) {
            o = OWN_LINE - l;
            break;
          }
    }
  for (int c = 0; c < sc->ncircles; ++c) {
    int i0, i1, j0, j1;
    bbox(c, &i0, &i1, &j0, &j1);
    for (int j = j0; j <= j1; ++j)
      for (int i = i0; i <= i1; ++i) {
        if (i < nx && S.hasH(i, j) && ownH[(size_t)j * nx + i] == OWN_NONE &&
            P.in_circle(c, i * dx, j * dx) != P.in_circle(c, (i + 1) * dx, j * dx))
          ownH[(size_t)j * nx + i] = c;
        if (j < ny && S.hasV(i, j) && ownV[(size_t)j * (nx + 1) + i] == OWN_NONE &&
            P.in_circle(c, i * dx, j * dx) != P.in_circle(c, i * dx, (j + 1) * dx))
          ownV[(size_t)j * (nx + 1) + i] = c;
      }
  }
  auto finish = [](double s) {
    if (!(s >= 0.0)) s = 0.0;
    if (s >= 1.0) s = below_one<double>();
    R r = (R)s;
    if (r >= R(1)) r = below_one<R>();
    return r;
  };
  std::fill(S.sH.begin(), S.sH.end(), R(0));
  std::fill(S.sV.begin(), S.sV.end(), R(0));
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i) {
      if (!S.hasH(i, j)) continue;
      const int32_t o = ownH[(size_t)j * nx + i];
      const double xi = i * dx, yj = j * dx;
      double s = 0.5;
      if (o == OWN_NOTCH) {
        // bisection on the scene's phase along the edge
        const bool side0 = P.inside(xi, yj);
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 60; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (P.inside(xi + mid * dx, yj) == side0) lo = mid; else hi = mid;
        }
        s = 0.5 * (lo + hi);
      } else if (o == OWN_CURVE) {
        // bisection on the edge until the bracket is below 2^-52
        const bool side0 = yj <= hcol[i];
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 60; ++it) {
          const double mid = 0.5 * (lo + hi);
          if ((yj <= P.curve_h(xi + mid * dx)) == side0) lo = mid; else hi = mid;
        }
        s = 0.5 * (lo + hi);
      } else if (o <= OWN_LINE) {
        const int l = OWN_LINE - o;
        const double x = (sc->lc[l] - sc->lb[l] * yj) / sc->la[l];
        s = (x - xi) / dx;
      } else if (o >= 0) {
        const double ddy = yj - sc->yc[o];
        const double disc = sc->r[o] * sc->r[o] - ddy * ddy;
        const double sq = std::sqrt(disc > 0.0 ? disc : 0.0);
        const double root = P.in_circle(o, xi, yj) ? sc->xc[o] + sq : sc->xc[o] - sq;
        s = (root - xi) / dx;
      }
      S.h(i, j) = finish(s);
    }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i) {
      if (!S.hasV(i, j)) continue;
      const int32_t o = ownV[(size_t)j * (nx + 1) + i];
      const double xi = i * dx, yj = j * dx;
      double s = 0.5;
      if (o == OWN_NOTCH) {
        const bool side0 = P.inside(xi, yj);
        double lo = 0.0, hi = 1.0;
        for (int it = 0; it < 60; ++it) {
          const double mid = 0.5 * (lo + hi);
          if (P.inside(xi, yj + mid * dx) == side0) lo = mid; else hi = mid;
        }
        s = 0.5 * (lo + hi);
      } else if (o == OWN_CURVE) {
        s = (hcol[i] - yj) / dx;
      } else if (o <= OWN_LINE) {
        const int l = OWN_LINE - o;
        const double y = (sc->lc[l] - sc->la[l] * xi) / sc->lb[l];
        s = (y - yj) / dx;
      } else if (o >= 0) {
        const double ddx = xi - sc->xc[o];
        const double disc = sc->r[o] * sc->r[o] - ddx * ddx;
        const double sq = std::sqrt(disc > 0.0 ? disc : 0.0);
        const double root = P.in_circle(o, xi, yj) ? sc->yc[o] + sq : sc->yc[o] - sq;
        s = (root - yj) / dx;
      }
      S.v(i, j) = finish(s);
    }
}

// Endpoints of a cell's marker on edge e, cell units relative to vertex (i,j).
template <typename R>
P2 edge_point(const State<R>& S, int i, int j, int e) {
  switch (e) {
    case 0: return {(double)S.hc(i, j), 0.0};
    case 1: return {1.0, (double)S.vc(i + 1, j)};
    case 2: return {(double)S.hc(i, j + 1), 1.0};
    default: return {0.0, (double)S.vc(i, j)};
  }
}

// Oriented segments (reference phase on the left), absolute cell units.
template <typename R>
int oriented_segments(const State<R>& S, int i, int j, P2 out[2][2]) {
  int seg[2][2];
  const int ns = cell_segments(S, i, j, seg);
  int c[4];
  corners(S, i, j, c);
  for (int t = 0; t < ns; ++t) {
    const int a = seg[t][0], b = seg[t][1];
    P2 P = edge_point(S, i, j, a), Q = edge_point(S, i, j, b);
    bool flip;
    if (b - a == 2) {
      // a=0,b=2: the left corners lie left of P->Q; a=1,b=3: the bottom ones
      flip = !c[0];
    } else {
      // a = (q+3)%4, b = q or a=0,b=3 (q=0): the cut corner lies right of the
      // segment going from edge (q+3)%4 to edge q
      const int q = (a == 0 && b == 3) ? 0 : b;
      const P2 from = edge_point(S, i, j, (q + 3) & 3), to = edge_point(S, i, j, q);
      P = from;
      Q = to;
      flip = c[q] != 0;
    }
    if (flip) std::swap(P, Q);
    out[t][0] = {P.x + i, P.y + j};
    out[t][1] = {Q.x + i, Q.y + j};
  }
  return ns;
}

template <typename R>
int64_t loops(const State<R>& S, double dx, int64_t* n_open, double* area, double* xy,
              int64_t cap, int64_t* n_written) {
  const int nx = S.nx, ny = S.ny;
  // signed shoelace area over all oriented segments (Green's theorem)
  double acc = 0.0;
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      P2 sg[2][2];
      const int ns = oriented_segments(S, i, j, sg);
      for (int t = 0; t < ns; ++t) acc += 0.5 * (sg[t][0].x * sg[t][1].y - sg[t][1].x * sg[t][0].y);
    }
  *area = acc * dx * dx;
  // trace polylines marker to marker
  auto id = [&](Mk m) -> int64_t {
    return m.kind == 0 ? (int64_t)m.j * nx + m.i
                       : (int64_t)nx * (ny + 1) + (int64_t)m.j * (nx + 1) + m.i;
  };
  auto has = [&](Mk m) { return m.kind == 0 ? S.hasH(m.i, m.j) : S.hasV(m.i, m.j); };
  auto cells_of = [&](Mk m, int cc[2][2], int ce[2]) {
    if (m.kind == 0) {
      cc[0][0] = m.i; cc[0][1] = m.j - 1; ce[0] = 2;
      cc[1][0] = m.i; cc[1][1] = m.j; ce[1] = 0;
    } else {
      cc[0][0] = m.i - 1; cc[0][1] = m.j; ce[0] = 1;
      cc[1][0] = m.i; cc[1][1] = m.j; ce[1] = 3;
    }
  };
  auto nbr = [&](Mk m, int side) -> Mk {
    int cc[2][2], ce[2];
    cells_of(m, cc, ce);
    const int ci = cc[side][0], cj = cc[side][1];
    if (ci < 0 || cj < 0 || ci >= nx || cj >= ny) return {-1, 0, 0};
    const int pe = partner_edge(S, ci, cj, ce[side]);
    if (pe < 0) return {-1, 0, 0};
    return edge_marker(ci, cj, pe);
  };
  auto pos = [&](Mk m) -> P2 {
    return m.kind == 0 ? P2{(m.i + (double)S.hc(m.i, m.j)) * dx, m.j * dx}
                       : P2{m.i * dx, (m.j + (double)S.vc(m.i, m.j)) * dx};
  };
  std::vector<uint8_t> seen((size_t)nx * (ny + 1) + (size_t)(nx + 1) * ny, 0);
  int64_t closed = 0, open = 0, w = 0;
  auto emit = [&](P2 p) {
    if (xy && w < cap) { xy[2 * w] = p.x; xy[2 * w + 1] = p.y; }
    ++w;
  };
  auto trace = [&](Mk start, int side) {
    // walk from start leaving through `side`; returns true if it closes
    Mk prev = start, cur = nbr(start, side);
    emit(pos(start));
    seen[id(start)] = 1;
    while (cur.kind >= 0) {
      if (cur.kind == start.kind && cur.i == start.i && cur.j == start.j) {
        emit(pos(start));
        return true;
      }
      seen[id(cur)] = 1;
      emit(pos(cur));
      Mk a = nbr(cur, 0), b = nbr(cur, 1);
      Mk next = (a.kind == prev.kind && a.i == prev.i && a.j == prev.j) ? b : a;
      prev = cur;
      cur = next;
    }
    return false;
  };
  auto visit = [&](Mk m) {
    if (!has(m) || seen[id(m)]) return;
    // open chains are traced from one of their ends
    Mk end = m;
    int side = 1;
    {
      Mk prev = {-1, 0, 0}, cur = m;
      int64_t guard = 0;
      while (true) {
        Mk a = nbr(cur, 0), b = nbr(cur, 1);
        if (a.kind < 0 || b.kind < 0) { end = cur; side = a.kind < 0 ? 1 : 0; break; }
        Mk next = (a.kind == prev.kind && a.i == prev.i && a.j == prev.j) ? b : a;
        prev = cur;
        cur = next;
        if ((cur.kind == m.kind && cur.i == m.i && cur.j == m.j) || ++guard > (int64_t)seen.size()) {
          end = m;
          side = 1;
          break;
        }
      }
    }
    const bool isclosed = trace(end, side);
    if (isclosed) ++closed; else ++open;
    emit({std::nan(""), std::nan("")});
  };
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i) visit({0, i, j});
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i) visit({1, i, j});
  *n_open = open;
  if (n_written) *n_written = w;
  return closed;
}

// ---------------------------------------------------------------------------
// Symmetric difference of two interface reconstructions (Sec. 3.2, Eqs. 15
// and 16): E_sym = |A| + |B| - 2 |A n B|, A and B the reference-phase regions
// bounded by the straight segments joining the markers of two states on the
// same grid.  Cell by cell, each region is one convex polygon or (a saddle
// whose centre is not reference phase) two corner triangles, so A n B is a
// sum of convex-convex intersections (Sutherland-Hodgman clipping).
// ---------------------------------------------------------------------------
struct Poly {
  int n = 0;
  P2 v[12];
};

double poly_area(const Poly& p) {
  double a = 0.0;
  for (int t = 0; t < p.n; ++t) {
    const P2 &u = p.v[t], &w = p.v[(t + 1) % p.n];
    a += u.x * w.y - w.x * u.y;
  }
  return 0.5 * a;
}

// p clipped to the left of the directed edge a->b (the inside of a
// counter-clockwise convex polygon).
Poly clip_left(const Poly& p, P2 a, P2 b) {
  Poly out;
  auto side = [&](P2 q) { return (b.x - a.x) * (q.y - a.y) - (b.y - a.y) * (q.x - a.x); };
  for (int t = 0; t < p.n; ++t) {
    const P2 cur = p.v[t], nxt = p.v[(t + 1) % p.n];
    const double sc = side(cur), sn = side(nxt);
    if (sc >= 0.0) out.v[out.n++] = cur;
    if ((sc >= 0.0) != (sn >= 0.0)) {
      const double w = sc / (sc - sn);
      out.v[out.n++] = {cur.x + w * (nxt.x - cur.x), cur.y + w * (nxt.y - cur.y)};
    }
  }
  return out;
}

double convex_overlap(const Poly& p, const Poly& q) {
  Poly r = p;
  for (int t = 0; t < q.n && r.n > 0; ++t) r = clip_left(r, q.v[t], q.v[(t + 1) % q.n]);
  return r.n >= 3 ? poly_area(r) : 0.0;
}

// Reference-phase pieces of cell (i,j) in cell units, counter-clockwise.
template <typename R>
int cell_pieces(const State<R>& S, int i, int j, Poly out[2]) {
  int c[4];
  corners(S, i, j, c);
  const P2 corner[4] = {{0, 0}, {1, 0}, {1, 1}, {0, 1}};
  P2 mk[4];
  int pres[4], n = 0;
  for (int e = 0; e < 4; ++e) {
    pres[e] = c[e] != c[(e + 1) & 3];
    n += pres[e];
    mk[e] = edge_point(S, i, j, e);
  }
  if (n == 4 && S.zc(i, j) == 0) {
    // two reference-phase corners cut off by their segments
    int m = 0;
    for (int q = 0; q < 4; ++q)
      if (c[q] == 1) {
        out[m].n = 3;
        out[m].v[0] = mk[(q + 3) & 3];
        out[m].v[1] = corner[q];
        out[m].v[2] = mk[q];
        ++m;
      }
    return m;
  }
  // one convex piece: the boundary walked counter-clockwise, keeping the
  // reference-phase corners and every marker
  Poly p;
  for (int q = 0; q < 4; ++q) {
    if (c[q] == 1) p.v[p.n++] = corner[q];
    if (pres[q]) p.v[p.n++] = mk[q];
  }
  if (p.n < 3) return 0;
  out[0] = p;
  return 1;
}

template <typename R>
double sym_diff(const State<R>& A, const State<R>& B, double dx) {
  double a = 0.0, b = 0.0, ab = 0.0;
  for (int j = 0; j < A.ny; ++j)
    for (int i = 0; i < A.nx; ++i) {
      Poly pa[2], pb[2];
      const int na = cell_pieces(A, i, j, pa), nb = cell_pieces(B, i, j, pb);
      for (int s = 0; s < na; ++s) a += poly_area(pa[s]);
      for (int t = 0; t < nb; ++t) b += poly_area(pb[t]);
      for (int s = 0; s < na; ++s)
        for (int t = 0; t < nb; ++t) ab += convex_overlap(pa[s], pb[t]);
    }
  return (a + b - 2.0 * ab) * (dx * dx);
}

template <typename R>
int do_step(int nx, int ny, double dx, int64_t step_index, bool line_only, bool ghf, uint8_t* K,
            uint8_t* Z, double* sH, double* sV, const double* u, const double* v, double dt,
            double* C, double* kappa, int64_t* counters, double* stats) {
  State<R> S = load<R>(nx, ny, K, Z, sH, sV);
  int64_t ctr[ORC_NCOUNTERS] = {0};
  double maxcfl = 0.0;
  const double lam = dt / dx;
  // Direction splitting (Sec. 2.1): x then y on even steps, y then x on odd.
  if ((step_index & 1) == 0) {
    sweep(S, 0, u, lam, line_only, ctr, &maxcfl);
    sweep(S, 1, v, lam, line_only, ctr, &maxcfl);
  } else {
    sweep(S, 1, v, lam, line_only, ctr, &maxcfl);
    sweep(S, 0, u, lam, line_only, ctr, &maxcfl);
  }
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i) ctr[ORC_N_H] += S.hasH(i, j);
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i) ctr[ORC_N_V] += S.hasV(i, j);
  const double area = fraction(S, dx, C);
  curvature(S, C, dx, kappa, ctr, ghf);
  store(S, K, Z, sH, sV);
  if (counters)
    for (int t = 0; t < ORC_NCOUNTERS; ++t) counters[t] = ctr[t];
  if (stats) {
    stats[0] = area;
    stats[1] = maxcfl;
  }
  return ctr[ORC_INVARIANT] ? 4 : (ctr[ORC_CFL] ? 3 : 0);
}

}  // namespace

extern "C" {

int orc_init(int nx, int ny, double dx, int prec, const orc_scene* scene, uint8_t* K, uint8_t* Z,
             double* sH, double* sV) {
  if (nx < 1 || ny < 1 || !(dx > 0.0) || !scene) return -1;
  if (prec == 0) {
    State<double> S(nx, ny);
    init(S, dx, scene);
    store(S, K, Z, sH, sV);
  } else {
    State<float> S(nx, ny);
    init(S, dx, scene);
    store(S, K, Z, sH, sV);
  }
  return 0;
}

int orc_sweep(int nx, int ny, int prec, int axis, uint8_t* K, uint8_t* Z, double* sH, double* sV,
              const double* vel, double lam, int64_t* counters, double* max_cfl) {
  if (nx < 1 || ny < 1) return -1;
  int64_t ctr[ORC_NCOUNTERS] = {0};
  double mc = 0.0;
  const bool line_only = (prec & 2) != 0;
  if ((prec & 1) == 0) {
    State<double> S = load<double>(nx, ny, K, Z, sH, sV);
    sweep(S, axis, vel, lam, line_only, ctr, &mc);
    store(S, K, Z, sH, sV);
  } else {
    State<float> S = load<float>(nx, ny, K, Z, sH, sV);
    sweep(S, axis, vel, lam, line_only, ctr, &mc);
    store(S, K, Z, sH, sV);
  }
  if (counters)
    for (int t = 0; t < ORC_NCOUNTERS; ++t) counters[t] = ctr[t];
  if (max_cfl) *max_cfl = mc;
  return 0;
}

int orc_step(int nx, int ny, double dx, int prec, int64_t step_index, uint8_t* K, uint8_t* Z,
             double* sH, double* sV, const double* u, const double* v, double dt, double* C,
             double* kappa, int64_t* counters, double* stats) {
  if (nx < 1 || ny < 1 || !(dx > 0.0)) return -1;
  const bool line_only = (prec & 2) != 0, ghf = (prec & 4) != 0;
  if ((prec & 1) == 0)
    return do_step<double>(nx, ny, dx, step_index, line_only, ghf, K, Z, sH, sV, u, v, dt, C,
                           kappa, counters, stats);
  return do_step<float>(nx, ny, dx, step_index, line_only, ghf, K, Z, sH, sV, u, v, dt, C, kappa,
                        counters, stats);
}

int orc_fraction(int nx, int ny, double dx, int prec, const uint8_t* K, const uint8_t* Z,
                 const double* sH, const double* sV, double* C, double* area) {
  double a;
  if ((prec & 1) == 0) a = fraction(load<double>(nx, ny, K, Z, sH, sV), dx, C);
  else a = fraction(load<float>(nx, ny, K, Z, sH, sV), dx, C);
  if (area) *area = a;
  return 0;
}

int orc_curvature(int nx, int ny, double dx, int prec, const uint8_t* K, const uint8_t* Z,
                  const double* sH, const double* sV, const double* C, double* kappa,
                  int64_t* counts) {
  int64_t ctr[ORC_NCOUNTERS] = {0};
  const bool ghf = (prec & 4) != 0;
  if ((prec & 1) == 0) curvature(load<double>(nx, ny, K, Z, sH, sV), C, dx, kappa, ctr, ghf);
  else curvature(load<float>(nx, ny, K, Z, sH, sV), C, dx, kappa, ctr, ghf);
  if (counts) {
    counts[0] = ctr[ORC_HF_INVALID];
    counts[1] = ctr[ORC_HF_OTHER];
    counts[2] = ctr[ORC_HF_MIXED];
    counts[3] = ctr[ORC_HF_MARKERS];
  }
  return 0;
}

int orc_parabola_kappa(int n, const double* X, const double* Y, const double* W, double ox,
                       double oy, double nx, double ny, double dx, double* kappa) {
  if (n < 3 || n > 64) return 0;
  return parabola_kappa<double>(n, X, Y, W, ox, oy, nx, ny, dx, kappa) ? 1 : 0;
}

}  // extern "C"

namespace {

// Properties and surface-tension source (the coupling of Sec. 2.5): the
// fraction C stands in for the Heaviside function of Eq. 8, and the surface
// term sigma kappa n delta_S of Eq. 6 becomes sigma kappa grad(C) at the
// faces, with the face curvature the mean of the two cells' valid
// heights-based curvatures (one valid: that one; none: 0) and the face
// gradient (C_b - C_a) / dx.  The definition written out in double for both
// precision forms: the library's FP32 form computes the same quantities in
// float and is compared with this within its rounding.
void coupling(int nx, int ny, double dx, const double* C, const double* kappa, double rho1,
              double rho2, double mu1, double mu2, double sigma, double* rho, double* mu,
              double* fx, double* fy) {
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i < nx; ++i) {
      const double c = C[(size_t)j * nx + i];
      rho[(size_t)j * nx + i] = c * rho1 + (1.0 - c) * rho2;
      mu[(size_t)j * nx + i] = c * mu1 + (1.0 - c) * mu2;
    }
  auto face = [&](size_t a, size_t b) -> double {  // cells a (low side), b (high side)
    const double ka = kappa[a], kb = kappa[b];
    const bool va = !std::isnan(ka), vb = !std::isnan(kb);
    double kf = 0.0;
    if (va && vb) kf = 0.5 * (ka + kb);
    else if (va) kf = ka;
    else if (vb) kf = kb;
    return sigma * kf * (C[b] - C[a]) / dx;
  };
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i)
      fx[(size_t)j * (nx + 1) + i] =
          (i == 0 || i == nx) ? 0.0 : face((size_t)j * nx + i - 1, (size_t)j * nx + i);
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i)
      fy[(size_t)j * nx + i] =
          (j == 0 || j == ny) ? 0.0 : face((size_t)(j - 1) * nx + i, (size_t)j * nx + i);
}

}  // namespace

extern "C" {

int orc_coupling(int nx, int ny, double dx, int prec, const double* C, const double* kappa,
                 double rho1, double rho2, double mu1, double mu2, double sigma,
                 double* rho, double* mu, double* fx, double* fy) {
  (void)prec;  // the same definition in double for both forms
  coupling(nx, ny, dx, C, kappa, rho1, rho2, mu1, mu2, sigma, rho, mu, fx, fy);
  return 0;
}

int orc_fit(const double* A, const double* B, const double* P1, int has_p1, const double* P4,
            int has_p4, double* y_out) {
  const P2 a{A[0], A[1]}, b{B[0], B[1]};
  const P2 p1{has_p1 ? P1[0] : 0.0, has_p1 ? P1[1] : 0.0};
  const P2 p4{has_p4 ? P4[0] : 0.0, has_p4 ? P4[1] : 0.0};
  return fit_crossing(a, b, has_p1 ? &p1 : nullptr, has_p4 ? &p4 : nullptr, false, y_out);
}

int64_t orc_loops(int nx, int ny, double dx, int prec, const uint8_t* K, const uint8_t* Z,
                  const double* sH, const double* sV, int64_t* n_open, double* area, double* xy,
                  int64_t cap, int64_t* n_written) {
  if ((prec & 1) == 0)
    return loops(load<double>(nx, ny, K, Z, sH, sV), dx, n_open, area, xy, cap, n_written);
  return loops(load<float>(nx, ny, K, Z, sH, sV), dx, n_open, area, xy, cap, n_written);
}

double orc_sym_diff(int nx, int ny, double dx, int prec, const uint8_t* K1, const uint8_t* Z1,
                    const double* sH1, const double* sV1, const uint8_t* K2, const uint8_t* Z2,
                    const double* sH2, const double* sV2) {
  if ((prec & 1) == 0)
    return sym_diff(load<double>(nx, ny, K1, Z1, sH1, sV1), load<double>(nx, ny, K2, Z2, sH2, sV2), dx);
  return sym_diff(load<float>(nx, ny, K1, Z1, sH1, sV1), load<float>(nx, ny, K2, Z2, sH2, sV2), dx);
}

double orc_shape_error(int nx, int ny, double dx, const uint8_t* K, const double* sH,
                       const double* sV, double xc, double yc, double R) {
  double e = 0.0;
  auto kk = [&](int i, int j) { return K[(size_t)j * (nx + 1) + i]; };
  for (int j = 0; j <= ny; ++j)
    for (int i = 0; i < nx; ++i)
      if (kk(i, j) != kk(i + 1, j)) {
        const double x = (i + sH[(size_t)j * nx + i]) * dx, y = j * dx;
        e = std::max(e, std::fabs(std::sqrt((x - xc) * (x - xc) + (y - yc) * (y - yc)) - R));
      }
  for (int j = 0; j < ny; ++j)
    for (int i = 0; i <= nx; ++i)
      if (kk(i, j) != kk(i, j + 1)) {
        const double x = i * dx, y = (j + sV[(size_t)j * (nx + 1) + i]) * dx;
        e = std::max(e, std::fabs(std::sqrt((x - xc) * (x - xc) + (y - yc) * (y - yc)) - R));
      }
  return e;
}

}  // extern "C"
