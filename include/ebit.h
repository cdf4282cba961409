/*
 * ebit.h - C ABI of libebit.so: the Edge-Based Interface Tracking (EBIT) step
 * of Pan, Long, Chirco, Scardovelli, Popinet & Zaleski (arXiv:2309.00338) on
 * one GB300 GPU (sm_103a).
 *
 * Grid (all arrays row-major, j is the slow index; dx is the cell size):
 *   vertex (i,j) at (i*dx, j*dx), 0 <= i <= nx, 0 <= j <= ny
 *   horizontal edge (i,j): (i,j)->(i+1,j), i < nx;  vertical edge (i,j): (i,j)->(i,j+1), j < ny
 *   a marker on an edge is an edge-local fraction s in [0,1) from the edge's
 *   first vertex; it exists exactly where the corner colour vertices at the
 *   two ends of the edge differ (Sec. 2.4).
 *   colour vertex 1 = reference phase.
 *
 * Precision: EBIT_FP64 - everything double.  EBIT_FP32 - marker fractions,
 * velocities, advection arithmetic, fractions C and curvature stored and
 * computed in float; circle fit (Sec. 2.2) and fraction areas in double.
 * Velocity and output buffers have the element type of the context precision.
 *
 * Errors: every call returns an ebit_status; no exception crosses the ABI.
 * Calls are asynchronous on the context's stream unless stated; failures that
 * kernels detect (CFL > 1, invariant breaks) are recorded in a device status
 * word and returned by the next synchronising call (ebit_sync,
 * ebit_fraction/ebit_curvature with a host output, ebit_diagnostics,
 * ebit_get_state).  ebit_last_error() gives a message for the calling thread.
 * A context is used by one host thread at a time.
 */
#ifndef EBIT_H
#define EBIT_H
#include <stddef.h>
#include <stdint.h>
#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  EBIT_OK = 0,
  EBIT_EAGAIN = 1,       /* result not ready yet (server)                    */
  EBIT_EINVAL = -1,      /* bad argument                                     */
  EBIT_ENOMEM = -2,      /* device or host allocation failed                 */
  EBIT_ECFL = -3,        /* a marker moved more than one cell in a sweep     */
  EBIT_EINVARIANT = -4,  /* colour/marker parity broken (must not happen)    */
  EBIT_ECUDA = -5,       /* CUDA runtime error                               */
  EBIT_ETIMEOUT = -6,    /* a bounded wait ran out                           */
  EBIT_EFULL = -7,       /* request can never fit the server's memory budget */
  EBIT_ECANCELLED = -8   /* the request was cancelled (ebit_cancel)          */
} ebit_status;

typedef enum { EBIT_FP64 = 0, EBIT_FP32 = 1 } ebit_precision;

/* flags: EBIT_FIT_LINE places unaligned markers on the chord crossing only
 * (the straight-line fit of the first EBIT version, Sec. 2.2).
 * EBIT_CURV_GHF gives the interface cells without a valid 7x3 height stencil
 * a curvature from the generalised height-function method Sec. 2.5 cites:
 * the stencil along the other direction, else a least-squares parabola
 * through the valid heights of both directions, else one through the markers
 * on the edges of the 3x3 block of cells (fits in the context precision, in
 * cell units relative to the cell).  The fields kernel lists those cells (a
 * list of nx*ny int32 in the context) and one more launch fits them.  Also
 * accepted in server requests. */
#define EBIT_FIT_LINE 1u
#define EBIT_CURV_GHF 2u

typedef struct {
  int32_t nx, ny;   /* cells; 1 <= nx, ny <= 32768                           */
  double dx;        /* cell size (> 0)                                       */
  int32_t prec;     /* ebit_precision                                        */
  uint32_t flags;
} ebit_grid;

typedef struct { double xc, yc, r; } ebit_circle;          /* toggles phase where d^2 <= r^2 */
typedef struct {                                             /* reference phase where y <= h(x) */
  double y0;                                                 /* h = y0 + sum_k amp[k-1] cos(2 pi k x + phase[k-1]) */
  int32_t nmodes;
  const double *amp, *phase;
} ebit_curve;
typedef struct { double a, b, c; } ebit_halfplane;          /* toggles phase where a x + b y <= c */
typedef struct { double x0, x1, y0, y1; } ebit_notch;       /* cuts the closed box [x0,x1]x[y0,y1] out
                                                               of the reference phase (Zalesak's
                                                               slotted disk, Sec. 3.4) */
typedef struct {
  const ebit_circle* circles;   /* host pointer, ncircles entries (may be NULL if 0) */
  int32_t ncircles;
  const ebit_curve* curve;      /* host pointer or NULL                     */
  const ebit_halfplane* line;   /* host pointer to max(nlines, 1) half-planes, or NULL */
  const ebit_notch* notches;    /* host pointer, nnotches entries (may be NULL if 0);
                                   applied after the curve, half-planes and circles */
  int32_t nnotches;
  int32_t nlines;               /* half-planes at line (0 or 1: one), at most 4; a
                                   band between parallel lines is two of them */
} ebit_scene;

/* Host copy of a state.  K: (ny+1)*(nx+1) bytes, Z: ny*nx bytes (0/1),
 * sH: (ny+1)*nx doubles, sV: ny*(nx+1) doubles (values where no marker exists
 * are unspecified on output and ignored on input).  Caller owns the arrays. */
typedef struct {
  int32_t nx, ny;
  uint8_t* K;
  uint8_t* Z;
  double* sH;
  double* sV;
  int64_t step_index;   /* even: next step sweeps x then y; odd: y then x */
} ebit_state_host;

/* Diagnostics of the last step (sums over both sweeps). */
enum {
  EBIT_D_NH = 0, EBIT_D_NV, EBIT_D_CANCELLED, EBIT_D_ZSET, EBIT_D_ZCONFLICT,
  EBIT_D_FIT_ONLINE, EBIT_D_FIT_LINE, EBIT_D_FIT_ONE, EBIT_D_FIT_TWO,
  EBIT_D_WALL_CLAMP, EBIT_D_INVARIANT, EBIT_D_HF_INVALID, EBIT_D_CFL,
  /* with EBIT_CURV_GHF: of the EBIT_D_HF_INVALID cells, those resolved by the
   * other direction, by mixed heights, by the markers fit */
  EBIT_D_HF_OTHER, EBIT_D_HF_MIXED, EBIT_D_HF_MARKERS,
  EBIT_D_COUNT = 16
};
typedef struct {
  int64_t c[EBIT_D_COUNT];
  double area;      /* sum C dx^2 of the current state                       */
  double max_cfl;   /* largest |u| dt / dx met by a marker in the last step  */
} ebit_diag;

typedef struct ebit_ctx ebit_ctx;

/* Initialisation (Sec. 3.2): colour vertices from the scene, markers by root
 * finding on edges whose end colours differ, then fractions and curvature.
 * Allocates all device state of the context (owned by it).  stream: a
 * cudaStream_t (NULL = legacy default stream).  Shapes closer than one cell
 * to each other are outside the supported input. */
ebit_status ebit_init(ebit_ctx** out, const ebit_grid* grid, const ebit_scene* scene,
                      void* stream);

/* An empty context (all colours 0, no markers) to be filled by ebit_load_state. */
ebit_status ebit_create(ebit_ctx** out, const ebit_grid* grid, void* stream);

/* Copies a host state in (synchronous); recomputes fractions and curvature.
 * FP32 contexts round the fractions to float. */
ebit_status ebit_load_state(ebit_ctx* ctx, const ebit_state_host* st);

/* Copies the current state out (synchronous). */
ebit_status ebit_get_state(ebit_ctx* ctx, ebit_state_host* st);

/* One EBIT time step (Sec. 2.1-2.5): direction-split advection (x then y on
 * even steps, y then x on odd steps) of the markers by Eq. 4 with the circle
 * fit (Sec. 2.2), corner and centre colour-vertex update (Sec. 2.3),
 * automatic topology change (Sec. 2.4), then volume fractions and
 * height-function curvature (Sec. 2.5).
 * u, v: DEVICE pointers, (ny+1)*(nx+1) contiguous, context precision,
 * velocity at the vertices; must stay valid until the step completes on the
 * stream.  dt: time step (any sign).  Asynchronous. */
ebit_status ebit_step(ebit_ctx* ctx, const void* u, const void* v, double dt);

/* One sweep only (axis 0 = x with u, 1 = y with v); does not update fractions,
 * curvature or the step index.  For tests. */
ebit_status ebit_sweep(ebit_ctx* ctx, int axis, const void* vel, double dt);

/* Volume fractions C (Sec. 2.5) of the current state.  C_dev: DEVICE buffer of
 * ny*nx elements (context precision) or NULL; area_host: if non-NULL receives
 * sum C dx^2 (synchronises the stream and reports deferred errors). */
ebit_status ebit_fraction(ebit_ctx* ctx, void* C_dev, double* area_host);

/* Volume fractions C (Sec. 2.5) of the current state straight into a HOST
 * buffer, for callers that take C every step: C_host is ny*nx elements
 * (context precision), row-major, pinned (page-locked) for the copy to run
 * asynchronously; the caller owns it.  copy_stream: a cudaStream_t of the
 * caller (NULL: the context's stream) on which the copy runs, ordered after
 * the work queued so far on the context's stream; the caller learns that
 * C_host is filled by synchronising copy_stream (or an event recorded on it).
 * The next fields computation of this context (ebit_step, ebit_fields) waits
 * on the device for the copy before overwriting C, so the next step's sweeps
 * overlap the copy.  ebit_destroy waits for a copy still in flight.
 * Asynchronous; EBIT_EINVAL for a NULL context or buffer. */
ebit_status ebit_fraction_to_host(ebit_ctx* ctx, void* C_host, void* copy_stream);

/* The area sum C dx^2 of the current state copied to area_host (host memory;
 * pinned memory keeps the copy asynchronous) on the context's stream, without
 * waiting: the value is there once the stream reaches the copy (after an
 * event recorded behind it, or ebit_sync).  For callers that read every
 * step's result while the next step runs.  EBIT_EINVAL for NULL arguments;
 * deferred device errors are reported by the next synchronising call. */
ebit_status ebit_area_async(ebit_ctx* ctx, double* area_host);

/* Height-function curvature (Sec. 2.5) of the current state, NaN where the
 * 7x3 stencil is invalid or the cell holds no interface.  kappa_dev: DEVICE
 * buffer of ny*nx elements or NULL; n_invalid_host: if non-NULL receives the
 * number of interface cells without a valid stencil (synchronises). */
ebit_status ebit_curvature(ebit_ctx* ctx, void* kappa_dev, int32_t* n_invalid_host);

/* Zero-copy access to the context's fraction and curvature buffers (device
 * pointers, row pitch in elements); valid until the next step or destroy. */
ebit_status ebit_fields(ebit_ctx* ctx, const void** C, const void** kappa, int64_t* pitch);

/* Material properties and surface tension of the two phases; phase 1 is the
 * reference phase (colour 1). */
typedef struct { double rho1, rho2, mu1, mu2, sigma; } ebit_fluids;

/* Hand-off to a one-fluid Navier-Stokes solver (Sec. 2.5), from the
 * context's current fractions C and curvature kappa:
 *   rho = C rho1 + (1 - C) rho2,  mu = C mu1 + (1 - C) mu2        (Eq. 8,
 *   with C in place of the Heaviside function), per cell, ny*nx;
 *   fx = sigma kappa_f (C(i,j) - C(i-1,j)) / dx on the vertical faces,
 *   ny*(nx+1), face (i,j) between cells (i-1,j) and (i,j);
 *   fy = sigma kappa_f (C(i,j) - C(i,j-1)) / dx on the horizontal faces,
 *   (ny+1)*nx, face (i,j) between cells (i,j-1) and (i,j)
 * (the surface term sigma kappa n delta_S of Eq. 6 as a face force density
 * sigma kappa grad C, the form whose pressure balance is exact; evaluated as
 * (sigma/dx) kappa_f dC with sigma/dx formed once).  kappa_f is
 * the mean of the two cells' curvatures when both are valid, the valid one
 * when one is, and 0 when neither is; wall faces carry 0.
 * Outputs: caller-owned DEVICE buffers, contiguous row-major, element type of
 * the context precision; any may be NULL (not written).  Arithmetic in the
 * context precision.  Asynchronous on the context's stream; EBIT_EINVAL for a
 * NULL ctx or fluids. */
ebit_status ebit_coupling(ebit_ctx* ctx, const ebit_fluids* fluids, void* rho_dev, void* mu_dev,
                          void* fx_dev, void* fy_dev);

/* Counters of the last step (synchronous). */
ebit_status ebit_diagnostics(ebit_ctx* ctx, ebit_diag* out);

/* Waits for the context's stream; returns and clears a deferred error. */
ebit_status ebit_sync(ebit_ctx* ctx);

/* Waits for the context's work (and a fraction copy still in flight), then
 * frees all its device memory.  NULL is ignored. */
void ebit_destroy(ebit_ctx* ctx);

/* Debug builds (libebit_check.so, compiled with EBIT_CHECK) check every
 * global index of the step kernels (sweeps, fields, fallback fits, of
 * contexts and of servers) against its array and skip an access out of
 * range; *misses receives
 * nonzero if any happened since the library was loaded.  Release builds
 * report 0.  Synchronous; EBIT_EINVAL for a NULL argument. */
ebit_status ebit_check_status(uint32_t* misses);

/* Message of the last failure on the calling thread (never NULL). */
const char* ebit_last_error(void);

/* Per-kernel timing for profiling.  When on, the context records a pair of
 * CUDA events on its stream around every kernel it launches for a step;
 * ebit_timings (synchronous) returns, per kernel kind, the summed duration in
 * milliseconds and the number of launches since the last call, then resets.
 * Kinds: EBIT_K_SWEEP (a split sweep), EBIT_K_CENTRE (reserved, always 0),
 * EBIT_K_FIELDS (fractions, curvature and area
 * sum, added up by the launch's last tile), EBIT_K_AREA (reserved, always 0),
 * EBIT_K_COUPLING (ebit_coupling),
 * EBIT_K_GHF (list and fits of the generalised fallbacks). */
enum { EBIT_K_SWEEP = 0, EBIT_K_CENTRE, EBIT_K_FIELDS, EBIT_K_AREA, EBIT_K_COUPLING, EBIT_K_GHF,
       EBIT_K_COUNT = 8 };
ebit_status ebit_set_timing(ebit_ctx* ctx, int on);
ebit_status ebit_timings(ebit_ctx* ctx, double* ms, int64_t* launches);

/* Volume fractions without allocating device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc (a solver that allocates all device memory at start-up and
 * forbids allocation inside its time loop, or a host framework that owns every
 * device buffer).  It computes C, the area sum C dx^2 and the marker counts of
 * a state held in the caller's device buffers, in the byte layout of
 * ebit_state_host: K (ny+1)*(nx+1) bytes, Z ny*nx bytes, sH (ny+1)*nx and
 * sV ny*(nx+1) elements of the grid precision.  Outputs (device): C ny*nx
 * elements, *area one double, marker_counts two int64 {horizontal, vertical}
 * or NULL.  Asynchronous on stream.
 * Scratch: a 1 MiB array inside the library that every GPU loading the
 * library holds until exit; it limits grids to 131072 blocks of 32x8 vertices
 * (about 5790x5790 cells) and larger grids return EBIT_EINVAL.  The first call
 * on a device looks up the array's device address (make it before any stream
 * capture) and keeps it for the life of the process: after a cudaDeviceReset
 * in this process that address is stale, so do not call this entry point on a
 * device that has been reset.  It calls no cudaMalloc/cudaFree.  All calls
 * share the array, so calls that overlap on the GPU (different streams, or
 * other host threads) race and must be serialised by the caller. */
ebit_status ebit_fraction_noalloc(const ebit_grid* grid, const uint8_t* K, const uint8_t* Z,
                                  const void* sH, const void* sV, void* C, double* area,
                                  int64_t* marker_counts, void* stream);

/* ------------------------------------------------------------------------
 * Batched steps and serving.  A server owns one CUDA stream and one worker
 * thread on its device.  Requests (an n x n unit-square grid of circles, an
 * analytic velocity field and a number of steps) are admitted while the sum
 * of their device footprints stays within the budget; every admitted grid
 * advances one EBIT step per batch step, in one captured launch sequence for
 * all of them (continuous batching: requests join and leave between batch
 * steps).  The results stay on the server until polled.  Submit and poll are
 * thread-safe.
 * ------------------------------------------------------------------------ */
typedef enum {
  EBIT_FIELD_VORTEX = 0,    /* u = -sin^2(pi x) sin(2 pi y), v = sin^2(pi y) sin(2 pi x),
                               times cos(pi t / period): time-reversed at t = period */
  EBIT_FIELD_CELLULAR = 1,  /* u = sin(pi x) cos(pi y), v = -cos(pi x) sin(pi y) */
  EBIT_FIELD_ROTATION = 2   /* u = -omega (y - cy) + drift_u, v = omega (x - cx) + drift_v */
} ebit_field_kind;

typedef struct {
  int32_t n;                   /* grid side, n x n cells, dx = 1/n */
  int32_t prec;                /* ebit_precision */
  uint32_t flags;              /* EBIT_FIT_LINE and/or EBIT_CURV_GHF, or 0 */
  const ebit_circle* circles;  /* host array, copied by ebit_submit */
  int32_t ncircles;
  int32_t field;               /* ebit_field_kind */
  double period;               /* vortex period T (> 0 for EBIT_FIELD_VORTEX) */
  double omega, cx, cy, drift_u, drift_v;  /* rotation parameters */
  int32_t steps;
  double cfl;                  /* dt = cfl dx / max|u| at t = 0, 0 < cfl <= 1 */
  void* C_out;                 /* optional HOST buffer of n*n elements (request
                                  precision) receiving the final fractions; must
                                  stay valid until the result has been polled */
  int32_t fault_after;         /* fault injection for testing the server's failure
                                  isolation: from step fault_after on, dt is
                                  multiplied by fault_dt_factor (ignored when
                                  fault_dt_factor is 0); a factor that takes a
                                  marker past one cell makes the request fail with
                                  EBIT_ECFL, which stops it and no other */
  double fault_dt_factor;
  int32_t fault_wait;          /* fault injection for the persistent schedules:
                                  nonzero makes, from step fault_after on, the
                                  count this grid's second-sweep tiles wait for
                                  one more than its first sweep can reach; the
                                  waits run out after the server's wait budget
                                  and the request stops with EBIT_ETIMEOUT */
} ebit_request;

typedef struct {
  int32_t status;              /* EBIT_OK, or why the request failed or stopped:
                                  EBIT_ECFL / EBIT_EINVARIANT (detected after the
                                  batch step that raised it; the request stops
                                  there), EBIT_ETIMEOUT (a device-side wait of a
                                  persistent batch step ran out), EBIT_ECANCELLED
                                  (ebit_cancel, or queued when the server was
                                  destroyed), EBIT_ECUDA */
  int64_t steps;               /* steps done */
  double area0, area;          /* sum C dx^2 at admission and at the end */
  double e_area;               /* |area - area0| / area0 (Eq. 13) */
  double queue_ms;             /* submission to admission */
  double run_ms;               /* admission to completion */
  double step_p50_ms, step_p99_ms;  /* latency of the batch steps it took part in */
  int64_t counters[EBIT_D_COUNT];   /* diagnostics summed over its steps */
  int64_t cell_updates;        /* n*n*steps */
} ebit_result;

/* CTA schedules of a batch step: the order of the (grid, tile) work items,
 * and how the two sweeps run.  The first three issue one launch per sweep
 * (every grid's first sweep, then every grid's second); the persistent ones
 * run both sweeps of all grids in one launch of resident blocks that take
 * the work items in order from a device counter, a grid's second-sweep tiles
 * starting once its first sweep is done (a device-side wait bounded by the
 * server's wait budget). */
typedef enum {
  EBIT_SCHED_LARGEST_FIRST = 0,  /* grid by grid, largest grids first */
  EBIT_SCHED_INTERLEAVED = 1,    /* tile t of every grid, then tile t+1, largest first */
  EBIT_SCHED_SMALLEST_FIRST = 2, /* grid by grid, smallest grids first */
  EBIT_SCHED_PERSISTENT_LARGEST_FIRST = 3,   /* the orders above, persistent */
  EBIT_SCHED_PERSISTENT_INTERLEAVED = 4,
  EBIT_SCHED_PERSISTENT_SMALLEST_FIRST = 5,
  EBIT_SCHED_COUNT = 6
} ebit_schedule;

typedef struct {
  int32_t max_instances;       /* 0: no limit besides the budget */
  int32_t use_graphs;          /* replay each batch step as a CUDA graph */
  int32_t device;              /* CUDA device ordinal */
  int32_t autotune;            /* 1: time every schedule on the first steps of a new set of
                                  grids and keep the fastest (cached per set signature);
                                  0: use `schedule` */
  int32_t schedule;            /* ebit_schedule when autotune is 0 */
  int32_t wait_budget_ms;      /* bound of each device-side wait of a persistent
                                  batch step (0: 1000 ms) */
} ebit_server_opts;

typedef struct {
  int64_t queued, running, batch_steps, cell_updates;
  double busy_ms;              /* GPU time of the batch steps */
  size_t bytes_in_use;
  int32_t schedule;            /* ebit_schedule of the current set of grids */
  int32_t tuned_sets;          /* set signatures whose schedule the autotuner has chosen */
  double tune_ms[EBIT_SCHED_COUNT];  /* step time of each schedule, last tuning (0: not timed) */
  /* Host time of the worker with no batch step in flight (ms): rebuilding the
     launch plan and its graph for a new set of grids (plans: how many times;
     plan_graph_ms: the part spent capturing the launch sequence and updating
     or instantiating its graph), admitting requests while no grid runs and
     taking out cancelled ones, and retiring finished grids (results copied
     out, memory freed). */
  int64_t plans;
  double plan_ms, plan_graph_ms, admit_idle_ms, retire_ms;
} ebit_server_stats;

typedef struct ebit_server ebit_server;

/* hbm_budget: device bytes the admitted requests may use together.  opts may
 * be NULL (graphs on, autotuned schedules, device 0).  No CUDA call happens
 * before the first admissible submission. */
ebit_status ebit_server_create(ebit_server** out, size_t hbm_budget, const ebit_server_opts* opts);
/* EBIT_EINVAL for a malformed request; EBIT_EFULL if it can never fit the
 * budget.  Otherwise queues it and returns its ticket. */
ebit_status ebit_submit(ebit_server* s, const ebit_request* req, uint64_t* ticket);
/* EBIT_EAGAIN while the request is queued or running; EBIT_OK with the result
 * once (the result is then released); EBIT_EINVAL for an unknown ticket. */
ebit_status ebit_poll(ebit_server* s, uint64_t ticket, ebit_result* out);
/* Cancels a request: a queued one is dropped at once, a running one leaves
 * the batch before the next batch step (the steps done so far are reported).
 * Its result (status EBIT_ECANCELLED) is then polled as usual; the other
 * requests are not affected.  EBIT_EINVAL for an unknown or finished ticket.
 * Thread-safe. */
ebit_status ebit_cancel(ebit_server* s, uint64_t ticket);
/* A snapshot of the server's counters (ebit_server_stats).  Thread-safe;
 * EBIT_EINVAL for NULL arguments. */
ebit_status ebit_server_stats_get(ebit_server* s, ebit_server_stats* out);
/* Cancels queued requests, finishes nothing further, frees everything. */
void ebit_server_destroy(ebit_server* s);

/* Device bytes a context of this grid allocates (for admission control). */
size_t ebit_footprint(const ebit_grid* grid);

#ifdef __cplusplus
}
#endif
#endif
