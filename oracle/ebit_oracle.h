/*
 * EBIT oracle: C interface of the plain CPU restatement of one EBIT interface
 * step (Pan et al., "An Edge-based Interface Tracking (EBIT) Method for
 * Multiphase-flow Simulation with Surface Tension", Sec. 2.1-2.5).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark may load this library.  The product path
 * (libebit.so and its Python binding) never calls it and shares no code,
 * header or table with it.
 *
 * Grid conventions (all arrays row-major, j is the slow index):
 *   vertex (i,j)   at (i*dx, j*dx),   0<=i<=nx, 0<=j<=ny
 *   K[j*(nx+1)+i]  colour vertex of that corner, 1 = reference phase
 *   Z[j*nx+i]      colour vertex of the centre of cell (i,j)
 *   sH[j*nx+i]     edge-local fraction of the marker on the horizontal edge
 *                  (i,j)->(i+1,j); marker at x=(i+s)dx; meaningful only
 *                  where K differs at the two ends of the edge
 *   sV[j*(nx+1)+i] same for the vertical edge (i,j)->(i,j+1); y=(j+s)dx
 *   u,v            velocity components at the vertices, (ny+1)*(nx+1)
 * prec: 0 = FP64 throughout; 1 = FP32 state, FP32 advection arithmetic,
 *       FP64 circle fit and FP64 fraction arithmetic (values exchanged here
 *       as doubles that are exactly representable in FP32).
 *       Flags or-ed into prec: 2 = straight-line fit (EBIT-SL), 4 = the
 *       generalised height-function fallbacks for curvature.
 */
#ifndef EBIT_ORACLE_H
#define EBIT_ORACLE_H
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef struct {
  int32_t ncircles;          /* circles toggle the phase inside (r^2 >= d^2) */
  const double *xc, *yc, *r;
  int32_t has_curve;         /* reference phase where y <= h(x)            */
  double y0;                 /* h(x) = y0 + sum_k amp[k-1] cos(2 pi k x + phase[k-1]) */
  int32_t nmodes;
  const double *amp, *phase;
  int32_t nlines;            /* 0..4 half-planes; each toggles the phase    */
  double la[4], lb[4], lc[4];/*   where la*x + lb*y <= lc                   */
  int32_t nnotches;          /* boxes cut out of the reference phase after the */
  const double* notch;       /* toggles: x0, x1, y0, y1 per box (closed)       */
} orc_scene;

/* Diagnostic counters written by orc_step / orc_sweep (summed over sweeps). */
enum {
  ORC_N_H = 0,         /* markers on horizontal edges after the step       */
  ORC_N_V,             /* markers on vertical edges after the step         */
  ORC_CANCELLED,       /* marker pairs removed because two met on an edge  */
  ORC_ZSET,            /* centre colour vertices set by the centre rule    */
  ORC_ZCONFLICT,       /* cells whose two unaligned markers disagreed      */
  ORC_FIT_ONLINE,      /* crossings that fall exactly on an advected point */
  ORC_FIT_LINE,        /* crossings where no circle survived (chord)       */
  ORC_FIT_ONE,         /* crossings placed by one circle                   */
  ORC_FIT_TWO,         /* crossings placed by the mean of two circles      */
  ORC_WALL_CLAMP,      /* aligned markers stopped at a domain wall         */
  ORC_INVARIANT,       /* colour/marker parity mismatches (must stay 0)    */
  ORC_HF_INVALID,      /* interface cells without a valid 7x3 height stencil */
  ORC_CFL,             /* markers whose displacement exceeded one cell     */
  ORC_HF_OTHER,        /* of those without a 7x3 stencil (generalised mode): */
  ORC_HF_MIXED,        /*   resolved by the other direction's stencil, by a  */
  ORC_HF_MARKERS,      /*   mixed-heights fit, by a fit to nearby markers    */
  ORC_NCOUNTERS = 16
};

int orc_init(int nx, int ny, double dx, int prec, const orc_scene* scene,
             uint8_t* K, uint8_t* Z, double* sH, double* sV);

/* One direction-split sweep: axis 0 = x (moves along x with u), 1 = y. */
int orc_sweep(int nx, int ny, int prec, int axis, uint8_t* K, uint8_t* Z,
              double* sH, double* sV, const double* vel, double lam,
              int64_t* counters, double* max_cfl);

/* Full step: sweeps in the order x,y when step_index is even, y,x when odd;
 * then fractions and curvature.  C and kappa are ny*nx; stats[0] = area
 * sum(C)*dx^2, stats[1] = largest |u| dt / dx seen. */
int orc_step(int nx, int ny, double dx, int prec, int64_t step_index,
             uint8_t* K, uint8_t* Z, double* sH, double* sV,
             const double* u, const double* v, double dt,
             double* C, double* kappa, int64_t* counters, double* stats);

int orc_fraction(int nx, int ny, double dx, int prec, const uint8_t* K,
                 const uint8_t* Z, const double* sH, const double* sV,
                 double* C, double* area);

/* Curvature of the fractions C; counts[4] (or NULL) receives the interface
 * cells without a valid 7x3 stencil and, with flag 4, how many of them the
 * other direction, mixed heights and the markers of the 3x3 block resolved.  The
 * heights and the fallback fits run in the state precision (double for the FP64
 * form, float for the FP32 form): their rounding stays far below the error of
 * the fits themselves (see the curvature section of the implementation). */
int orc_curvature(int nx, int ny, double dx, int prec, const uint8_t* K,
                  const uint8_t* Z, const double* sH, const double* sV,
                  const double* C, double* kappa, int64_t* counts);

/* Weighted least-squares parabola through n points (X, Y in cell units) in
 * the frame of origin (ox, oy) and unit normal (nx, ny) (out of the reference
 * phase); kappa at the origin, divided by dx.  Returns 1 if the fit is
 * regular (test hook of the generalised fallbacks). */
int orc_parabola_kappa(int n, const double* X, const double* Y, const double* W, double ox,
                       double oy, double nx, double ny, double dx, double* kappa);

/* Hand-off to a one-fluid Navier-Stokes solver (Sec. 2.5: the surface term
 * of Eq. 6 and the property law of Eq. 8, with the fractions standing in for
 * the Heaviside function):
 * rho = C rho1 + (1 - C) rho2 and mu likewise per cell (ny*nx), and the
 * surface-tension source sigma kappa grad(C) on the faces: fx on the
 * (nx+1)*ny vertical faces, fy on the nx*(ny+1) horizontal ones, zero on the
 * walls: f = sigma kappa_f (C_b - C_a) / dx.  Double arithmetic in both
 * precision forms (prec is accepted and ignored). */
int orc_coupling(int nx, int ny, double dx, int prec, const double* C, const double* kappa,
                 double rho1, double rho2, double mu1, double mu2, double sigma,
                 double* rho, double* mu, double* fx, double* fy);

/* Vertex-local circle fit of one crossing (test hook).  Points are (x,y)
 * pairs in cell units relative to the vertex on the grid line x = 0; A has
 * x < 0, B has x >= 0; has_p1 / has_p4 select the optional neighbours.
 * Returns the fit kind (ORC_FIT_*) and writes the crossing ordinate. */
int orc_fit(const double* A, const double* B, const double* P1, int has_p1,
            const double* P4, int has_p4, double* y_out);

/* Interface polylines traced through the per-cell segments.  Returns the
 * number of closed loops; writes the number of open chains, the signed
 * shoelace area (reference phase on the left, dx^2 units applied) and, if
 * xy is non-null, up to cap vertices (x,y pairs, domain units) of all
 * polylines, each polyline terminated by a (NaN,NaN) pair. */
int64_t orc_loops(int nx, int ny, double dx, int prec, const uint8_t* K,
                  const uint8_t* Z, const double* sH, const double* sV,
                  int64_t* n_open, double* area, double* xy, int64_t cap,
                  int64_t* n_written);

/* E_sym (Eqs. 15-16): |A| + |B| - 2 |A n B| of the reference-phase regions
 * of two states of the same grid (domain units: dx^2 applied). */
double orc_sym_diff(int nx, int ny, double dx, int prec, const uint8_t* K1,
                    const uint8_t* Z1, const double* sH1, const double* sV1,
                    const uint8_t* K2, const uint8_t* Z2, const double* sH2,
                    const double* sV2);

/* E_shape (Eq. 14): max over markers of |dist(marker, centre) - R|. */
double orc_shape_error(int nx, int ny, double dx, const uint8_t* K,
                       const double* sH, const double* sV, double xc,
                       double yc, double R);

#ifdef __cplusplus
}
#endif
#endif
