// Host side of the C ABI declared in include/ebit.h: context allocation, the
// launch sequence of one EBIT step, state I/O and error reporting.
#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ebit.h"
#include "ebit_ctx.hpp"
#include "ebit_kernels.cuh"
#include "ebit_tile.cuh"
#include "ebit_fields.cuh"
#include "ebit_coupling.cuh"
#include "ebit_ghf.cuh"

namespace {

thread_local std::string g_err;

ebit_status fail(ebit_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return s;
}

#define EBIT_CK(call)                                                                  \
  do {                                                                                 \
    cudaError_t e_ = (call);                                                           \
    if (e_ != cudaSuccess) return fail(EBIT_ECUDA, "%s: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

using namespace ebit_detail;

}  // namespace

namespace {

// Brackets a launch with events when timing is on.
struct Timed {
  ebit_ctx* c;
  ebit_ctx::Mark* m = nullptr;
  Timed(ebit_ctx* c_, int kind) : c(c_) {
    if (!c->timing) return;
    if (c->marks_used == c->marks.size()) {
      ebit_ctx::Mark k{};
      if (cudaEventCreate(&k.a) != cudaSuccess || cudaEventCreate(&k.b) != cudaSuccess) return;
      c->marks.push_back(k);
    }
    m = &c->marks[c->marks_used++];
    m->kind = kind;
    cudaEventRecord(m->a, c->stream);
  }
  ~Timed() {
    if (m) cudaEventRecord(m->b, c->stream);
  }
};

ebit_status dalloc(ebit_ctx* c, void** p, size_t bytes) {
  cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(EBIT_ENOMEM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
  }
  c->allocs.push_back(*p);
  e = cudaMemsetAsync(*p, 0, bytes ? bytes : 16, c->stream);
  if (e != cudaSuccess) return fail(EBIT_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  return EBIT_OK;
}

ebit_status alloc_ctx(ebit_ctx* c) {
  const Layout& L = c->L;
  ebit_status s;
#define EBIT_AL(ptr, bytes) \
  if ((s = dalloc(c, (void**)&(ptr), (bytes))) != EBIT_OK) return s
  for (int b = 0; b < 2; ++b) {
    EBIT_AL(c->K[b], L.k_bytes);
    EBIT_AL(c->Z[b], L.z_bytes);
    EBIT_AL(c->sH[b], L.h_bytes);
    EBIT_AL(c->sV[b], L.v_bytes);
  }
  EBIT_AL(c->C, L.field_bytes);
  EBIT_AL(c->kappa, L.field_bytes);
  EBIT_AL(c->partial, L.partial_count * sizeof(double));
  EBIT_AL(c->area, sizeof(double));
  EBIT_AL(c->area_done, sizeof(unsigned));
  EBIT_AL(c->ctr, ebit::kCounters * sizeof(unsigned long long));
  EBIT_AL(c->cfl_bits, sizeof(unsigned long long));
  EBIT_AL(c->status, sizeof(int));
  if (c->grid.flags & EBIT_CURV_GHF) {
    EBIT_AL(c->ghf_list, (size_t)c->grid.nx * c->grid.ny * sizeof(int));
    EBIT_AL(c->ghf_count, sizeof(unsigned));
  }
#undef EBIT_AL
  return EBIT_OK;
}

void free_ctx(ebit_ctx* c) {
  for (void* p : c->allocs) cudaFree(p);
  c->allocs.clear();
}

template <typename R>
ebit_status launch_fields(ebit_ctx* c) {
  const Layout& L = c->L;
  const int b = c->cur;
  const dim3 fgrid((L.d.nx + 1 + ebit::kFX - 1) / ebit::kFX, (L.d.ny + 1 + ebit::kFY - 1) / ebit::kFY);
  const bool ghf = (c->grid.flags & EBIT_CURV_GHF) != 0;
  if (c->c_read_pending) {  // C is still being copied to the host
    EBIT_CK(cudaStreamWaitEvent(c->stream, c->ev_c_read, 0));
    c->c_read_pending = false;
  }
  if (ghf) EBIT_CK(cudaMemsetAsync(c->ghf_count, 0, sizeof(unsigned), c->stream));
  {
    Timed t(c, EBIT_K_FIELDS);
    ebit::AreaSum sum;
    sum.done = c->area_done;
    sum.n = (long long)fgrid.x * fgrid.y;
    sum.scale = c->grid.dx * c->grid.dx;
    sum.area = c->area;
    ebit::k_fields_tile<R><<<fgrid, ebit::field_threads<R>(), 0, c->stream>>>(
        c->K[b], c->Z[b], (const R*)c->sH[b], (const R*)c->sV[b], L.d, (R)c->grid.dx, (R*)c->C,
        (R*)c->kappa, c->partial, c->ctr, ghf ? c->ghf_list : nullptr, ghf ? c->ghf_count : nullptr, sum);
  }
  if (ghf) {
    Timed t(c, EBIT_K_GHF);
    const ebit::GhfView<R> S{c->K[b], c->Z[b], (const R*)c->sH[b], (const R*)c->sV[b],
                             (const R*)c->C, L.d};
    const long long cells = (long long)L.d.nx * L.d.ny;
    const int blocks = (int)std::min<long long>((cells + ebit::kGhfThreads - 1) / ebit::kGhfThreads,
                                                152LL * 8);
    ebit::k_ghf_fit<R><<<blocks, ebit::kGhfThreads, 0, c->stream>>>(
        S, (R)c->grid.dx, c->ghf_list, c->ghf_count, (R*)c->kappa, c->ctr);
  }
  EBIT_CK(cudaGetLastError());
  return EBIT_OK;
}

ebit_status fields(ebit_ctx* c) {
  return c->grid.prec == EBIT_FP32 ? launch_fields<float>(c) : launch_fields<double>(c);
}

template <typename R>
ebit_status launch_coupling(ebit_ctx* c, const ebit_fluids* fl, void* rho, void* mu, void* fx,
                            void* fy) {
  const Layout& L = c->L;
  const ebit::Fluids<R> f{(R)fl->rho1, (R)fl->rho2, (R)fl->mu1, (R)fl->mu2,
                          (R)fl->sigma / (R)c->grid.dx};
  {
    Timed t(c, EBIT_K_COUPLING);
    if constexpr (sizeof(R) == 8) {
      const dim3 grid((L.d.nx + 1 + ebit::kCT - 1) / ebit::kCT, (L.d.ny + 1 + ebit::kCR - 1) / ebit::kCR);
      ebit::k_coupling_q<<<grid, ebit::kCT, 0, c->stream>>>((const R*)c->C, (const R*)c->kappa, L.d, f,
                                                            (R*)rho, (R*)mu, (R*)fx, (R*)fy);
    } else {
      // column pairs 0..nx/2 (the last pair holds the right wall face)
      const dim3 grid((L.d.nx / 2 + 1 + ebit::kCT - 1) / ebit::kCT,
                      (L.d.ny + 1 + ebit::kCR2 - 1) / ebit::kCR2);
      ebit::k_coupling<R><<<grid, ebit::kCT, 0, c->stream>>>((const R*)c->C, (const R*)c->kappa, L.d,
                                                             f, (R*)rho, (R*)mu, (R*)fx, (R*)fy);
    }
  }
  EBIT_CK(cudaGetLastError());
  return EBIT_OK;
}

template <typename R, int AX>
ebit_status launch_sweep(ebit_ctx* c, const void* vel, double lam) {
  const Layout& L = c->L;
  const int src = c->cur, dst = 1 - c->cur;
  const int line_only = (c->grid.flags & EBIT_FIT_LINE) ? 1 : 0;
  ebit::GView<R, AX> S{c->K[src], c->Z[src], (const R*)c->sH[src], (const R*)c->sV[src],
                       (const R*)vel, L.d, (R)lam};
  ebit::Buf<R> out{c->K[dst], c->Z[dst], (R*)c->sH[dst], (R*)c->sV[dst]};
  {
    constexpr size_t smem = ebit::tile_smem_bytes<R>();
    static bool attr = false;  // once per instantiation and process
    if (!attr) {
      EBIT_CK(cudaFuncSetAttribute(ebit::k_sweep_tile<R, AX>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      attr = true;
    }
    const int tnx = AX ? L.d.ny : L.d.nx, tny = AX ? L.d.nx : L.d.ny;
    const dim3 grid((tnx + 1 + ebit::kTI - 1) / ebit::kTI, (tny + 1 + ebit::kTJ - 1) / ebit::kTJ);
    Timed t(c, EBIT_K_SWEEP);
    ebit::k_sweep_tile<R, AX><<<grid, ebit::tile_threads<R>(), smem, c->stream>>>(
        S, out, line_only, c->ctr, c->cfl_bits, c->status);
  }
  EBIT_CK(cudaGetLastError());
  c->cur = dst;
  return EBIT_OK;
}

ebit_status sweep(ebit_ctx* c, int axis, const void* vel, double lam) {
  if (c->grid.prec == EBIT_FP32)
    return axis == 0 ? launch_sweep<float, 0>(c, vel, lam) : launch_sweep<float, 1>(c, vel, lam);
  return axis == 0 ? launch_sweep<double, 0>(c, vel, lam) : launch_sweep<double, 1>(c, vel, lam);
}

ebit_status reset_counters(ebit_ctx* c) {
  EBIT_CK(cudaMemsetAsync(c->ctr, 0, ebit::kCounters * sizeof(unsigned long long), c->stream));
  EBIT_CK(cudaMemsetAsync(c->cfl_bits, 0, sizeof(unsigned long long), c->stream));
  return EBIT_OK;
}

ebit_status take_status(ebit_ctx* c) {
  int st = 0;
  EBIT_CK(cudaMemcpyAsync(&st, c->status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  EBIT_CK(cudaStreamSynchronize(c->stream));
  if (st) {
    EBIT_CK(cudaMemsetAsync(c->status, 0, sizeof(int), c->stream));
    EBIT_CK(cudaStreamSynchronize(c->stream));
    if (st & ebit::ST_INVARIANT) return fail(EBIT_EINVARIANT, "colour/marker parity broken");
    if (st & ebit::ST_CFL) return fail(EBIT_ECFL, "a marker moved more than one cell in a sweep");
  }
  return EBIT_OK;
}

ebit_status new_ctx(ebit_ctx** out, const ebit_grid* grid, void* stream) {
  if (!out) return fail(EBIT_EINVAL, "out is NULL");
  *out = nullptr;
  if (!valid_grid(grid)) return fail(EBIT_EINVAL, "invalid grid");
  ebit_ctx* c = new (std::nothrow) ebit_ctx;
  if (!c) return fail(EBIT_ENOMEM, "host allocation failed");
  c->grid = *grid;
  c->L = layout_of(grid);
  c->stream = (cudaStream_t)stream;
  const ebit_status s = alloc_ctx(c);
  if (s != EBIT_OK) {
    free_ctx(c);
    delete c;
    return s;
  }
  *out = c;
  return EBIT_OK;
}

template <typename R>
ebit_status init_scene(ebit_ctx* c, const ebit_scene* scene) {
  const Layout& L = c->L;
  const double dx = c->grid.dx;
  ebit::SceneDev sc{};
  std::vector<double> circ;
  for (int t = 0; t < scene->ncircles; ++t) {
    circ.push_back(scene->circles[t].xc);
    circ.push_back(scene->circles[t].yc);
    circ.push_back(scene->circles[t].r);
  }
  std::vector<double> notch;
  for (int b = 0; b < scene->nnotches; ++b) {
    notch.push_back(scene->notches[b].x0);
    notch.push_back(scene->notches[b].x1);
    notch.push_back(scene->notches[b].y0);
    notch.push_back(scene->notches[b].y1);
  }
  std::vector<double> curve;
  if (scene->curve) {
    for (int k = 0; k < scene->curve->nmodes; ++k) curve.push_back(scene->curve->amp[k]);
    for (int k = 0; k < scene->curve->nmodes; ++k) curve.push_back(scene->curve->phase[k]);
  }
  // scene arrays and scratch: stream-ordered allocations freed at the end of
  // the call, so that setting up a grid does not wait for work on other
  // streams (a batch step of the server runs while it admits new grids)
  std::vector<void*> tmp;
  auto talloc = [&](void** p, size_t bytes) -> ebit_status {
    cudaError_t e = cudaMallocAsync(p, bytes ? bytes : 16, c->stream);
    if (e != cudaSuccess) { cudaGetLastError(); return fail(EBIT_ENOMEM, "cudaMallocAsync: %s", cudaGetErrorString(e)); }
    tmp.push_back(*p);
    return EBIT_OK;
  };
  auto cleanup = [&]() {
    for (void* p : tmp) cudaFreeAsync(p, c->stream);
    cudaStreamSynchronize(c->stream);
  };
  double *dcirc = nullptr, *dcurve = nullptr, *hv = nullptr, *dnotch = nullptr;
  int *ownH = nullptr, *ownV = nullptr;
  ebit_status s;
  if ((s = talloc((void**)&dcirc, circ.size() * sizeof(double))) != EBIT_OK ||
      (s = talloc((void**)&dcurve, curve.size() * sizeof(double))) != EBIT_OK ||
      (s = talloc((void**)&dnotch, notch.size() * sizeof(double))) != EBIT_OK ||
      (s = talloc((void**)&hv, (size_t)(2 * c->grid.nx + 1) * sizeof(double))) != EBIT_OK ||
      (s = talloc((void**)&ownH, (size_t)(c->grid.ny + 1) * L.d.P * sizeof(int))) != EBIT_OK ||
      (s = talloc((void**)&ownV, (size_t)(c->grid.ny + 1) * L.d.P * sizeof(int))) != EBIT_OK) {
    cleanup();
    return s;
  }
  auto run = [&]() -> ebit_status {
    if (!circ.empty())
      EBIT_CK(cudaMemcpyAsync(dcirc, circ.data(), circ.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (!curve.empty())
      EBIT_CK(cudaMemcpyAsync(dcurve, curve.data(), curve.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    if (!notch.empty())
      EBIT_CK(cudaMemcpyAsync(dnotch, notch.data(), notch.size() * sizeof(double), cudaMemcpyHostToDevice, c->stream));
    sc.notch = dnotch;
    sc.nnotches = scene->nnotches;
    EBIT_CK(cudaMemsetAsync(ownH, 0x7f, (size_t)(c->grid.ny + 1) * L.d.P * sizeof(int), c->stream));
    EBIT_CK(cudaMemsetAsync(ownV, 0x7f, (size_t)(c->grid.ny + 1) * L.d.P * sizeof(int), c->stream));
    sc.circ = dcirc;
    sc.ncircles = scene->ncircles;
    if (scene->curve) {
      sc.has_curve = 1;
      sc.y0 = scene->curve->y0;
      sc.nmodes = scene->curve->nmodes;
      sc.amp = dcurve;
      sc.phase = dcurve + scene->curve->nmodes;
    }
    if (scene->line) {
      sc.nlines = scene->nlines > 1 ? scene->nlines : 1;
      for (int l = 0; l < sc.nlines; ++l) {
        sc.la[l] = scene->line[l].a;
        sc.lb[l] = scene->line[l].b;
        sc.lc[l] = scene->line[l].c;
      }
    }
    const int b = c->cur;
    if (sc.has_curve) ebit::k_curve_cols<<<(c->grid.nx + 1 + 255) / 256, 256, 0, c->stream>>>(sc, c->grid.nx, dx, hv);
    ebit::k_init_base<<<L.grid, L.block, 0, c->stream>>>(sc, L.d, dx, hv, c->K[b], c->Z[b]);
    if (sc.ncircles > 0) {
      ebit::k_init_circles<<<sc.ncircles, 256, 0, c->stream>>>(sc, L.d, dx, c->K[b], c->Z[b]);
      ebit::k_init_owner<<<sc.ncircles, 256, 0, c->stream>>>(sc, L.d, dx, ownH, ownV);
    }
    if (sc.nnotches > 0) ebit::k_init_notch<<<L.grid, L.block, 0, c->stream>>>(sc, L.d, dx, c->K[b], c->Z[b]);
    ebit::k_init_roots<R><<<L.grid, L.block, 0, c->stream>>>(sc, L.d, dx, c->K[b], hv, ownH, ownV,
                                                            (R*)c->sH[b], (R*)c->sV[b]);
    EBIT_CK(cudaGetLastError());
    return EBIT_OK;
  };
  s = run();
  cleanup();
  return s;
}

template <typename R>
ebit_status load_state(ebit_ctx* c, const ebit_state_host* st) {
  const Layout& L = c->L;
  const int nx = c->grid.nx, ny = c->grid.ny;
  const size_t nk = (size_t)(nx + 1) * (ny + 1), nz = (size_t)nx * ny;
  const size_t nh = (size_t)nx * (ny + 1), nv = (size_t)(nx + 1) * ny;
  uint8_t *dk = nullptr, *dz = nullptr;
  double *dh = nullptr, *dv = nullptr;
  std::vector<void*> tmp;
  ebit_status s = EBIT_OK;
  auto talloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) { cudaGetLastError(); return false; }
    tmp.push_back(*p);
    return true;
  };
  if (!talloc((void**)&dk, nk) || !talloc((void**)&dz, nz) || !talloc((void**)&dh, nh * 8) ||
      !talloc((void**)&dv, nv * 8)) {
    s = fail(EBIT_ENOMEM, "cudaMalloc failed in load_state");
  } else {
    const int b = c->cur;
    const int T = 256;
    cudaMemcpyAsync(dk, st->K, nk, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(dz, st->Z, nz, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(dh, st->sH, nh * 8, cudaMemcpyHostToDevice, c->stream);
    cudaMemcpyAsync(dv, st->sV, nv * 8, cudaMemcpyHostToDevice, c->stream);
    ebit::k_pack_bits<<<dim3((nx + 1 + 31) / 32, (ny + 1 + ebit::kBlockY - 1) / ebit::kBlockY), L.block, 0, c->stream>>>(
        dk, nx + 1, ny + 1, L.d.kw, c->K[b]);
    ebit::k_pack_bits<<<dim3((nx + 31) / 32, (ny + ebit::kBlockY - 1) / ebit::kBlockY), L.block, 0, c->stream>>>(
        dz, nx, ny, L.d.zw, c->Z[b]);
    ebit::k_load_frac<R><<<(unsigned)((nh + T - 1) / T), T, 0, c->stream>>>(dh, nx, ny + 1, L.d.P, (R*)c->sH[b]);
    ebit::k_load_frac<R><<<(unsigned)((nv + T - 1) / T), T, 0, c->stream>>>(dv, nx + 1, ny, L.d.P, (R*)c->sV[b]);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = fail(EBIT_ECUDA, "load_state: %s", cudaGetErrorString(e));
  }
  cudaStreamSynchronize(c->stream);
  for (void* p : tmp) cudaFree(p);
  if (s != EBIT_OK) return s;
  c->step_index = st->step_index;
  if ((s = reset_counters(c)) != EBIT_OK) return s;
  if ((s = fields(c)) != EBIT_OK) return s;
  EBIT_CK(cudaStreamSynchronize(c->stream));
  return EBIT_OK;
}

template <typename R>
ebit_status get_state(ebit_ctx* c, ebit_state_host* st) {
  const Layout& L = c->L;
  const int nx = c->grid.nx, ny = c->grid.ny;
  const size_t nk = (size_t)(nx + 1) * (ny + 1), nz = (size_t)nx * ny;
  const size_t nh = (size_t)nx * (ny + 1), nv = (size_t)(nx + 1) * ny;
  uint8_t *dk = nullptr, *dz = nullptr;
  double *dh = nullptr, *dv = nullptr;
  std::vector<void*> tmp;
  ebit_status s = EBIT_OK;
  auto talloc = [&](void** p, size_t bytes) -> bool {
    if (cudaMalloc(p, bytes ? bytes : 16) != cudaSuccess) { cudaGetLastError(); return false; }
    tmp.push_back(*p);
    return true;
  };
  if (!talloc((void**)&dk, nk) || !talloc((void**)&dz, nz) || !talloc((void**)&dh, nh * 8) ||
      !talloc((void**)&dv, nv * 8)) {
    s = fail(EBIT_ENOMEM, "cudaMalloc failed in get_state");
  } else {
    const int b = c->cur;
    const int T = 256;
    ebit::k_unpack_bits<<<(unsigned)((nk + T - 1) / T), T, 0, c->stream>>>(c->K[b], nx + 1, ny + 1, L.d.kw, dk);
    ebit::k_unpack_bits<<<(unsigned)((nz + T - 1) / T), T, 0, c->stream>>>(c->Z[b], nx, ny, L.d.zw, dz);
    ebit::k_store_frac<R><<<(unsigned)((nh + T - 1) / T), T, 0, c->stream>>>((const R*)c->sH[b], nx, ny + 1, L.d.P, dh);
    ebit::k_store_frac<R><<<(unsigned)((nv + T - 1) / T), T, 0, c->stream>>>((const R*)c->sV[b], nx + 1, ny, L.d.P, dv);
    cudaMemcpyAsync(st->K, dk, nk, cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(st->Z, dz, nz, cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(st->sH, dh, nh * 8, cudaMemcpyDeviceToHost, c->stream);
    cudaMemcpyAsync(st->sV, dv, nv * 8, cudaMemcpyDeviceToHost, c->stream);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) s = fail(EBIT_ECUDA, "get_state: %s", cudaGetErrorString(e));
  }
  cudaError_t e = cudaStreamSynchronize(c->stream);
  for (void* p : tmp) cudaFree(p);
  if (s != EBIT_OK) return s;
  if (e != cudaSuccess) return fail(EBIT_ECUDA, "get_state: %s", cudaGetErrorString(e));
  st->step_index = c->step_index;
  return take_status(c);
}

}  // namespace

void ebit_detail_set_error(const char* msg) { g_err = msg; }

extern "C" {

const char* ebit_last_error(void) { return g_err.c_str(); }

size_t ebit_footprint(const ebit_grid* grid) {
  if (!valid_grid(grid)) return 0;
  return layout_of(grid).total();
}

ebit_status ebit_create(ebit_ctx** out, const ebit_grid* grid, void* stream) {
  ebit_status s = new_ctx(out, grid, stream);
  if (s != EBIT_OK) return s;
  if ((s = fields(*out)) != EBIT_OK) return s;
  return EBIT_OK;
}

ebit_status ebit_init(ebit_ctx** out, const ebit_grid* grid, const ebit_scene* scene, void* stream) {
  const Range range("ebit_init");
  if (!scene || scene->ncircles < 0 || (scene->ncircles > 0 && !scene->circles) ||
      (scene->curve && (scene->curve->nmodes < 0 || (scene->curve->nmodes > 0 &&
                                                     (!scene->curve->amp || !scene->curve->phase)))) ||
      (scene->line && scene->line->a == 0.0 && scene->line->b == 0.0 && scene->line->c < 0.0) ||
      scene->nnotches < 0 || (scene->nnotches > 0 && !scene->notches) || scene->nlines < 0 ||
      scene->nlines > 4)
    return fail(EBIT_EINVAL, "invalid scene");
  ebit_status s = new_ctx(out, grid, stream);
  if (s != EBIT_OK) return s;
  ebit_ctx* c = *out;
  s = c->grid.prec == EBIT_FP32 ? init_scene<float>(c, scene) : init_scene<double>(c, scene);
  if (s == EBIT_OK) s = reset_counters(c);
  if (s == EBIT_OK) s = fields(c);
  if (s != EBIT_OK) {
    ebit_destroy(c);
    *out = nullptr;
  }
  return s;
}

ebit_status ebit_load_state(ebit_ctx* c, const ebit_state_host* st) {
  if (!c || !st || !st->K || !st->Z || !st->sH || !st->sV) return fail(EBIT_EINVAL, "NULL argument");
  if (st->nx != c->grid.nx || st->ny != c->grid.ny) return fail(EBIT_EINVAL, "state size mismatch");
  return c->grid.prec == EBIT_FP32 ? load_state<float>(c, st) : load_state<double>(c, st);
}

ebit_status ebit_get_state(ebit_ctx* c, ebit_state_host* st) {
  if (!c || !st || !st->K || !st->Z || !st->sH || !st->sV) return fail(EBIT_EINVAL, "NULL argument");
  if (st->nx != c->grid.nx || st->ny != c->grid.ny) return fail(EBIT_EINVAL, "state size mismatch");
  return c->grid.prec == EBIT_FP32 ? get_state<float>(c, st) : get_state<double>(c, st);
}

ebit_status ebit_step(ebit_ctx* c, const void* u, const void* v, double dt) {
  const Range range("ebit_step");
  if (!c || !u || !v) return fail(EBIT_EINVAL, "NULL argument");
  if (!(dt == dt)) return fail(EBIT_EINVAL, "dt is NaN");
  ebit_status s = reset_counters(c);
  if (s != EBIT_OK) return s;
  const double lam = dt / c->grid.dx;
  const bool x_first = (c->step_index & 1) == 0;
  if ((s = sweep(c, x_first ? 0 : 1, x_first ? u : v, lam)) != EBIT_OK) return s;
  if ((s = sweep(c, x_first ? 1 : 0, x_first ? v : u, lam)) != EBIT_OK) return s;
  if ((s = fields(c)) != EBIT_OK) return s;
  c->step_index += 1;
  return EBIT_OK;
}

ebit_status ebit_sweep(ebit_ctx* c, int axis, const void* vel, double dt) {
  if (!c || !vel || (axis != 0 && axis != 1)) return fail(EBIT_EINVAL, "bad argument");
  ebit_status s = reset_counters(c);
  if (s != EBIT_OK) return s;
  return sweep(c, axis, vel, dt / c->grid.dx);
}

// The context's pitched C or kappa (ny rows of P elements) into the caller's
// dense ny x nx device array, on the context's stream.
static ebit_status unpitch(ebit_ctx* c, const void* src, void* dst) {
  const Layout& L = c->L;
  const long long row_bytes = (long long)c->grid.nx * L.esz, pitch_bytes = (long long)L.d.P * L.esz;
  const int h = c->grid.ny;
  const unsigned gy = (unsigned)std::min(h, 65535);
  if (row_bytes % 16 == 0 && ((uintptr_t)dst & 15u) == 0) {
    const long long w = row_bytes / 16;
    const dim3 grid((unsigned)((w + 255) / 256), gy);
    ebit::k_unpitch<uint4><<<grid, 256, 0, c->stream>>>((const uint4*)src, pitch_bytes / 16, (uint4*)dst, w, h);
  } else if (L.esz == 4) {
    const dim3 grid((unsigned)((c->grid.nx + 255) / 256), gy);
    ebit::k_unpitch<float><<<grid, 256, 0, c->stream>>>((const float*)src, L.d.P, (float*)dst, c->grid.nx, h);
  } else {
    const dim3 grid((unsigned)((c->grid.nx + 255) / 256), gy);
    ebit::k_unpitch<double><<<grid, 256, 0, c->stream>>>((const double*)src, L.d.P, (double*)dst, c->grid.nx, h);
  }
  EBIT_CK(cudaGetLastError());
  return EBIT_OK;
}

ebit_status ebit_fraction(ebit_ctx* c, void* C_dev, double* area_host) {
  if (!c) return fail(EBIT_EINVAL, "NULL context");
  if (C_dev) {
    const ebit_status s = unpitch(c, c->C, C_dev);
    if (s != EBIT_OK) return s;
  }
  if (area_host) {
    EBIT_CK(cudaMemcpyAsync(area_host, c->area, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    return take_status(c);
  }
  return EBIT_OK;
}

ebit_status ebit_fraction_to_host(ebit_ctx* c, void* C_host, void* copy_stream) {
  if (!c || !C_host) return fail(EBIT_EINVAL, "NULL argument");
  const Layout& L = c->L;
  cudaStream_t cs = copy_stream ? (cudaStream_t)copy_stream : c->stream;
  if (!c->ev_queued) {
    EBIT_CK(cudaEventCreateWithFlags(&c->ev_queued, cudaEventDisableTiming));
    EBIT_CK(cudaEventCreateWithFlags(&c->ev_c_read, cudaEventDisableTiming));
  }
  if (cs != c->stream) {
    EBIT_CK(cudaEventRecord(c->ev_queued, c->stream));
    EBIT_CK(cudaStreamWaitEvent(cs, c->ev_queued, 0));
    // a copy still pending from an earlier call comes first, so that the
    // single event the next fields launch waits for covers both
    if (c->c_read_pending) EBIT_CK(cudaStreamWaitEvent(cs, c->ev_c_read, 0));
  }
  EBIT_CK(cudaMemcpy2DAsync(C_host, (size_t)c->grid.nx * L.esz, c->C, (size_t)L.d.P * L.esz,
                            (size_t)c->grid.nx * L.esz, c->grid.ny, cudaMemcpyDeviceToHost, cs));
  if (cs != c->stream) {
    EBIT_CK(cudaEventRecord(c->ev_c_read, cs));
    c->c_read_pending = true;
  }
  return EBIT_OK;
}

ebit_status ebit_check_status(uint32_t* misses) {
  if (!misses) return fail(EBIT_EINVAL, "NULL argument");
#ifdef EBIT_CHECK
  unsigned w = 0;
  EBIT_CK(cudaMemcpyFromSymbol(&w, ebit::ebit_check_word, sizeof w));
  *misses = w | server_check_misses();
#else
  *misses = 0;
#endif
  return EBIT_OK;
}

ebit_status ebit_area_async(ebit_ctx* c, double* area_host) {
  if (!c || !area_host) return fail(EBIT_EINVAL, "NULL argument");
  EBIT_CK(cudaMemcpyAsync(area_host, c->area, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  return EBIT_OK;
}

ebit_status ebit_curvature(ebit_ctx* c, void* kappa_dev, int32_t* n_invalid_host) {
  if (!c) return fail(EBIT_EINVAL, "NULL context");
  if (kappa_dev) {
    const ebit_status s = unpitch(c, c->kappa, kappa_dev);
    if (s != EBIT_OK) return s;
  }
  if (n_invalid_host) {
    unsigned long long n = 0;
    EBIT_CK(cudaMemcpyAsync(&n, c->ctr + ebit::D_HF_INVALID, sizeof n, cudaMemcpyDeviceToHost, c->stream));
    ebit_status s = take_status(c);
    *n_invalid_host = (int32_t)n;
    return s;
  }
  return EBIT_OK;
}

ebit_status ebit_coupling(ebit_ctx* c, const ebit_fluids* fl, void* rho, void* mu, void* fx,
                          void* fy) {
  const Range range("ebit_coupling");
  if (!c || !fl) return fail(EBIT_EINVAL, "NULL argument");
  return c->grid.prec == EBIT_FP32 ? launch_coupling<float>(c, fl, rho, mu, fx, fy)
                                   : launch_coupling<double>(c, fl, rho, mu, fx, fy);
}

ebit_status ebit_fields(ebit_ctx* c, const void** C, const void** kappa, int64_t* pitch) {
  if (!c) return fail(EBIT_EINVAL, "NULL context");
  if (C) *C = c->C;
  if (kappa) *kappa = c->kappa;
  if (pitch) *pitch = c->L.d.P;
  return EBIT_OK;
}

ebit_status ebit_diagnostics(ebit_ctx* c, ebit_diag* out) {
  if (!c || !out) return fail(EBIT_EINVAL, "NULL argument");
  unsigned long long ctr[ebit::kCounters], bits = 0;
  double area = 0.0;
  EBIT_CK(cudaMemcpyAsync(ctr, c->ctr, sizeof ctr, cudaMemcpyDeviceToHost, c->stream));
  EBIT_CK(cudaMemcpyAsync(&bits, c->cfl_bits, sizeof bits, cudaMemcpyDeviceToHost, c->stream));
  EBIT_CK(cudaMemcpyAsync(&area, c->area, sizeof area, cudaMemcpyDeviceToHost, c->stream));
  EBIT_CK(cudaStreamSynchronize(c->stream));
  for (int t = 0; t < EBIT_D_COUNT; ++t) out->c[t] = (int64_t)ctr[t];
  out->area = area;
  double m;
  std::memcpy(&m, &bits, sizeof m);
  out->max_cfl = m;
  return take_status(c);
}

ebit_status ebit_sync(ebit_ctx* c) {
  if (!c) return fail(EBIT_EINVAL, "NULL context");
  EBIT_CK(cudaStreamSynchronize(c->stream));
  return take_status(c);
}

ebit_status ebit_set_timing(ebit_ctx* c, int on) {
  if (!c) return fail(EBIT_EINVAL, "NULL context");
  c->timing = on != 0;
  return EBIT_OK;
}

ebit_status ebit_timings(ebit_ctx* c, double* ms, int64_t* launches) {
  if (!c || !ms || !launches) return fail(EBIT_EINVAL, "NULL argument");
  EBIT_CK(cudaStreamSynchronize(c->stream));
  for (int k = 0; k < EBIT_K_COUNT; ++k) { ms[k] = 0.0; launches[k] = 0; }
  for (size_t t = 0; t < c->marks_used; ++t) {
    float e = 0.0f;
    EBIT_CK(cudaEventElapsedTime(&e, c->marks[t].a, c->marks[t].b));
    ms[c->marks[t].kind] += e;
    launches[c->marks[t].kind] += 1;
  }
  c->marks_used = 0;
  return EBIT_OK;
}

void ebit_destroy(ebit_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  if (c->ev_c_read) {  // a copy of C to the host may still run on the caller's stream
    cudaEventSynchronize(c->ev_c_read);
    cudaEventDestroy(c->ev_c_read);
    cudaEventDestroy(c->ev_queued);
  }
  for (auto& m : c->marks) {
    cudaEventDestroy(m.a);
    cudaEventDestroy(m.b);
  }
  free_ctx(c);
  delete c;
}

}  // extern "C"
