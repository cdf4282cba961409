// Batched EBIT steps over many grids and the request-serving loop
// (ebit_server_create / ebit_submit / ebit_poll / ebit_server_destroy).
//
// A batch step advances every admitted grid by one EBIT step with a fixed
// launch sequence per precision: a copy of the per-grid sweep descriptors
// from pinned host memory, the sweeps (each tile in the direction its grid's
// split order puts there: the grids are square, so their x and y tiles are
// the same work items), the fields launch and the area launch.  The sweeps
// are either one persistent launch for both sweeps of all grids (a grid's
// second-sweep tiles wait, bounded, for its first sweep) or two launches, the
// first sweeps of all grids and then the second.  Work items are (grid, tile)
// pairs in the order of a CTA schedule; an online autotuner picks the order
// and the persistent or two-launch form per set of grids (ebit_schedule).
// The sequence is captured once per set of admitted grids (and schedule) as a
// CUDA graph and replayed every step.  Grids keep their state in the same
// buffer across a step (first sweep A->B, second B->A).
//
// Serving: one worker thread owns the GPU.  Between batch steps it retires
// finished, failed and cancelled grids (results copied to the host, memory
// freed).  It admits queued requests, first come first served among those
// that fit, while the sum of their device footprints stays within the budget:
// continuous batching.  With grids running, admission happens while a batch
// step runs on the server's stream (the new grids are set up on a second
// stream and join from the next step), so it overlaps the GPU work; only a
// server with no grid running admits between steps.  The launch plan's
// buffers only grow and its graph is updated in place where the launch
// sequence keeps its shape, so a new set of grids costs little host time.  The
// last launch of a batch step copies every grid's status word into host-mapped
// memory; a grid whose step raised a CFL or invariant error leaves the batch
// with that status, and the others carry on unchanged.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <set>
#include <thread>
#include <vector>

#include "ebit.h"
#include "ebit_ctx.hpp"
#include "ebit_fields.cuh"
#include "ebit_ghf.cuh"
#include "ebit_persist.cuh"
#include "ebit_tile.cuh"

namespace {

ebit_status fail_s(ebit_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  ebit_detail_set_error(buf);
  return s;
}

double now_ms() {
  using namespace std::chrono;
  return duration<double, std::milli>(steady_clock::now().time_since_epoch()).count();
}

// Analytic velocity fields at the vertices of an n x n unit-square grid.
template <typename R>
__global__ void k_velocity(int kind, int n, double dx, double omega, double cx, double cy,
                           double du, double dv, R* u, R* v) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  const long long m = (long long)(n + 1) * (n + 1);
  if (t >= m) return;
  const int i = (int)(t % (n + 1)), j = (int)(t / (n + 1));
  const double x = i * dx, y = j * dx;
  double a, b;
  if (kind == EBIT_FIELD_VORTEX) {
    const double sx = sinpi(x), sy = sinpi(y);
    a = -(sx * sx) * sinpi(2.0 * y);
    b = (sy * sy) * sinpi(2.0 * x);
  } else if (kind == EBIT_FIELD_CELLULAR) {
    a = sinpi(x) * cospi(y);
    b = -cospi(x) * sinpi(y);
  } else {
    a = -omega * (y - cy) + du;
    b = omega * (x - cx) + dv;
  }
  u[t] = (R)a;
  v[t] = (R)b;
}

struct AreaDesc {
  const double* partial;
  long long n;
  double scale;
  double* area;
};

// Zeroes the generalised-HF list counts of the grids that have one, before
// the batched fields launch lists into them.
template <typename R>
__global__ void k_ghf_reset(const ebit::FieldDesc<R>* __restrict__ descs, int n) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n && descs[g].ghf_count) *descs[g].ghf_count = 0u;
}

__global__ void k_area_batch(const AreaDesc* __restrict__ descs) {
  const AreaDesc D = descs[blockIdx.x];
  __shared__ double red[256];
  double acc = 0.0;
  for (long long b = threadIdx.x; b < D.n; b += 256) acc = acc + D.partial[b];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) *D.area = red[0] * D.scale;
}

// Every grid's status word, gathered into host-mapped memory at the end of a
// batch step (one thread per grid).
__global__ void k_status_gather(int* const* __restrict__ status, int n, int* out) {
  const int g = blockIdx.x * blockDim.x + threadIdx.x;
  if (g < n) out[g] = *status[g];
}

struct Instance {
  uint64_t ticket = 0;
  ebit_request req{};
  std::vector<ebit_circle> circles;
  ebit_ctx* ctx = nullptr;
  void* u = nullptr;
  void* v = nullptr;
  size_t bytes = 0;
  int64_t done = 0;
  double dt = 0.0, dx = 0.0;
  double area0 = 0.0;
  double t_submit = 0.0, t_admit = 0.0;
  std::vector<float> lat_ms;
  ebit_status failed = EBIT_OK;  // set when a batch step it took part in failed,
                                 // its status word reported an error, or it was cancelled
};

size_t request_bytes(const ebit_request& r) {
  ebit_grid g{r.n, r.n, 1.0 / r.n, r.prec, r.flags};
  const size_t esz = r.prec == EBIT_FP32 ? 4 : 8;
  return ebit_footprint(&g) + 2 * (size_t)(r.n + 1) * (r.n + 1) * esz + (1u << 20);
}

double field_umax(const ebit_request& r) {
  if (r.field == EBIT_FIELD_VORTEX || r.field == EBIT_FIELD_CELLULAR) return 1.0;
  double m = 0.0;
  for (int a = 0; a < 2; ++a)
    for (int b = 0; b < 2; ++b) {
      m = std::max(m, std::fabs(-r.omega * (b - r.cy) + r.drift_u));
      m = std::max(m, std::fabs(r.omega * (a - r.cx) + r.drift_v));
    }
  return m > 0.0 ? m : 1.0;
}

// Launch plan of one precision for the current set of grids.
template <typename R>
struct Group {
  std::vector<Instance*> inst;
  ebit::SweepDesc<R, 0>* h_s0 = nullptr;  // pinned: [first-x | second-x] descriptors
  ebit::SweepDesc<R, 1>* h_s1 = nullptr;  // pinned: [first-y | second-y]
  ebit::SweepDesc<R, 0>* d_s0 = nullptr;
  ebit::SweepDesc<R, 1>* d_s1 = nullptr;
  ebit::WorkItem* d_items0 = nullptr;
  ebit::FieldDesc<R>* d_fd = nullptr;
  ebit::FieldItem* d_fitems = nullptr;
  AreaDesc* d_ad = nullptr;
  int n_items0 = 0, n_fitems = 0;
  std::vector<int> ghf;  // grids with EBIT_CURV_GHF (fits after the fields launch)
  // persistent schedules: [next item | first-sweep tiles done per grid], the
  // counts the second sweeps wait for (pinned copy refreshed every step)
  unsigned* d_ctl = nullptr;
  unsigned* d_need = nullptr;
  unsigned* h_need = nullptr;
  std::vector<unsigned> tiles;  // per grid: tiles of one sweep
  int persist_blocks = 0;
  // Capacities in bytes of the buffers above.  They only grow: a new set of
  // grids reuses them, so a plan rebuild neither frees (cudaFree waits for
  // the device) nor pins new host memory (slow) unless the set outgrew them.
  size_t c_s0 = 0, c_s1 = 0, c_items0 = 0, c_fd = 0, c_fitems = 0, c_ad = 0, c_ctl = 0, c_need = 0;
  size_t hc_s0 = 0, hc_s1 = 0, hc_need = 0;
  // pinned staging of the plan's tables (copied to the device buffers above)
  ebit::WorkItem* h_items0 = nullptr;
  ebit::FieldItem* h_fitems = nullptr;
  ebit::FieldDesc<R>* h_fd = nullptr;
  AreaDesc* h_ad = nullptr;
  size_t hc_items0 = 0, hc_fitems = 0, hc_fd = 0, hc_ad = 0;
  int per_sm = -1, sms = 0;  // occupancy of the persistent sweep, queried once

  void release() {
    for (void* p : {(void*)h_s0, (void*)h_s1, (void*)h_need, (void*)h_items0, (void*)h_fitems,
                    (void*)h_fd, (void*)h_ad})
      if (p) cudaFreeHost(p);
    for (void* p : {(void*)d_s0, (void*)d_s1, (void*)d_items0, (void*)d_fd,
                    (void*)d_fitems, (void*)d_ad, (void*)d_ctl, (void*)d_need})
      if (p) cudaFree(p);
    *this = Group<R>();
  }

  // At least `bytes` of device (pinned host) memory at *p, reallocated only
  // when the capacity is short (then doubled, so that a growing set of grids
  // reallocates rarely).
  static ebit_status grow_dev(void** p, size_t* cap, size_t bytes) {
    if (bytes <= *cap && *p) return EBIT_OK;
    if (*p) cudaFree(*p);
    *p = nullptr;
    *cap = 0;
    const size_t want = std::max<size_t>(256, 2 * bytes);
    if (cudaMalloc(p, want) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return fail_s(EBIT_ENOMEM, "cudaMalloc (batch plan)");
    }
    *cap = want;
    return EBIT_OK;
  }
  static ebit_status grow_host(void** p, size_t* cap, size_t bytes) {
    if (bytes <= *cap && *p) return EBIT_OK;
    if (*p) cudaFreeHost(*p);
    *p = nullptr;
    *cap = 0;
    const size_t want = std::max<size_t>(256, 2 * bytes);
    if (cudaMallocHost(p, want) != cudaSuccess) {
      cudaGetLastError();
      *p = nullptr;
      return fail_s(EBIT_ENOMEM, "cudaMallocHost (batch plan)");
    }
    *cap = want;
    return EBIT_OK;
  }

  ebit_status build(const std::vector<Instance*>& all, int prec, int schedule, cudaStream_t st) {
    inst.clear();
    ghf.clear();
    tiles.clear();
    n_items0 = n_fitems = 0;
    persist_blocks = 0;
    for (Instance* in : all)
      if (in->req.prec == prec) inst.push_back(in);
    if (inst.empty()) return EBIT_OK;
    if (schedule == EBIT_SCHED_SMALLEST_FIRST)
      std::stable_sort(inst.begin(), inst.end(),
                       [](const Instance* a, const Instance* b) { return a->req.n < b->req.n; });
    else
      std::stable_sort(inst.begin(), inst.end(),
                       [](const Instance* a, const Instance* b) { return a->req.n > b->req.n; });
    const size_t n = inst.size();
    // per grid, its sweep and field tiles (row order within the grid)
    tiles.assign(n, 0u);
    std::vector<int> ntx(n), nfx(n), nft(n);
    size_t total0 = 0, totalf = 0;
    for (size_t g = 0; g < n; ++g) {
      const ebit::Dims& d = inst[g]->ctx->L.d;
      ntx[g] = (d.nx + 1 + ebit::kTI - 1) / ebit::kTI;
      tiles[g] = (unsigned)(ntx[g] * ((d.ny + 1 + ebit::kTJ - 1) / ebit::kTJ));
      nfx[g] = (d.nx + 1 + ebit::kFX - 1) / ebit::kFX;
      nft[g] = nfx[g] * ((d.ny + 1 + ebit::kFY - 1) / ebit::kFY);
      total0 += tiles[g];
      totalf += (size_t)nft[g];
    }
    ebit_status s;
    if ((s = grow_host((void**)&h_items0, &hc_items0, total0 * sizeof(ebit::WorkItem))) != EBIT_OK) return s;
    if ((s = grow_host((void**)&h_fitems, &hc_fitems, totalf * sizeof(ebit::FieldItem))) != EBIT_OK) return s;
    if ((s = grow_host((void**)&h_fd, &hc_fd, n * sizeof(ebit::FieldDesc<R>))) != EBIT_OK) return s;
    if ((s = grow_host((void**)&h_ad, &hc_ad, n * sizeof(AreaDesc))) != EBIT_OK) return s;
    // the work items in the order of the CTA schedule, written straight into
    // pinned memory: grid by grid, or round robin (tile t of every grid
    // before tile t+1)
    n_items0 = (int)order_items(h_items0, tiles, ntx, schedule);
    std::vector<unsigned> nft_u(nft.begin(), nft.end());
    n_fitems = (int)order_items(h_fitems, nft_u, nfx, schedule);
    for (size_t g = 0; g < n; ++g) {
      const ebit_ctx* c = inst[g]->ctx;
      const ebit::Dims& d = c->L.d;
      const int b = c->cur;
      const bool gh = (c->grid.flags & EBIT_CURV_GHF) != 0;
      h_fd[g] = ebit::FieldDesc<R>{c->K[b], c->Z[b], (const R*)c->sH[b], (const R*)c->sV[b], d,
                                   (R)c->grid.dx, (R*)c->C, (R*)c->kappa, c->partial, c->ctr, nfx[g],
                                   gh ? c->ghf_list : nullptr, gh ? c->ghf_count : nullptr};
      if (gh) ghf.push_back((int)g);
      h_ad[g] = AreaDesc{c->partial, (long long)nft[g], c->grid.dx * c->grid.dx, c->area};
    }
    // the copies run on the server's stream before the step's launches; the
    // pinned sources stay untouched until the next plan, which the worker
    // builds only once that step has finished
    auto dput = [&](void** p, size_t* cap, const void* src, size_t bytes) -> ebit_status {
      const ebit_status g = grow_dev(p, cap, bytes);
      if (g != EBIT_OK) return g;
      if (src && cudaMemcpyAsync(*p, src, bytes, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return fail_s(EBIT_ECUDA, "cudaMemcpyAsync (batch plan)");
      return EBIT_OK;
    };
    if ((s = dput((void**)&d_items0, &c_items0, h_items0, total0 * sizeof(ebit::WorkItem))) != EBIT_OK) return s;
    if ((s = dput((void**)&d_fitems, &c_fitems, h_fitems, totalf * sizeof(ebit::FieldItem))) != EBIT_OK) return s;
    if ((s = dput((void**)&d_fd, &c_fd, h_fd, n * sizeof(ebit::FieldDesc<R>))) != EBIT_OK) return s;
    if ((s = dput((void**)&d_ad, &c_ad, h_ad, n * sizeof(AreaDesc))) != EBIT_OK) return s;
    if ((s = dput((void**)&d_s0, &c_s0, nullptr, 2 * n * sizeof(ebit::SweepDesc<R, 0>))) != EBIT_OK) return s;
    if ((s = dput((void**)&d_s1, &c_s1, nullptr, 2 * n * sizeof(ebit::SweepDesc<R, 1>))) != EBIT_OK) return s;
    if ((s = dput((void**)&d_ctl, &c_ctl, nullptr, (n + 1) * sizeof(unsigned))) != EBIT_OK) return s;
    if ((s = dput((void**)&d_need, &c_need, nullptr, n * sizeof(unsigned))) != EBIT_OK) return s;
    if ((s = grow_host((void**)&h_s0, &hc_s0, 2 * n * sizeof(ebit::SweepDesc<R, 0>))) != EBIT_OK) return s;
    if ((s = grow_host((void**)&h_s1, &hc_s1, 2 * n * sizeof(ebit::SweepDesc<R, 1>))) != EBIT_OK) return s;
    if ((s = grow_host((void**)&h_need, &hc_need, n * sizeof(unsigned))) != EBIT_OK) return s;
    // resident blocks of the persistent launch (more would only wait for a slot)
    int dev = 0;
    if (per_sm < 0 &&
        (cudaGetDevice(&dev) != cudaSuccess ||
         cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
         cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, ebit::k_sweep_persistent<R>,
                                                       ebit::tile_threads<R>(),
                                                       ebit::tile_smem_bytes<R, ebit::batch_cand_cap<R>()>()) != cudaSuccess)) {
      cudaGetLastError();
      per_sm = -1;
      return fail_s(EBIT_ECUDA, "occupancy of the persistent sweep");
    }
    persist_blocks = (int)std::min<long long>(2LL * n_items0, (long long)std::max(1, per_sm) * sms);
    return EBIT_OK;
  }

  // Writes the tiles of all grids to out in the order of the CTA schedule
  // (grid g has count[g] tiles, ncol[g] per tile row, in row order): grid by
  // grid, or round robin (tile t of every grid before tile t+1).  Returns
  // how many it wrote.
  template <typename Item>
  static size_t order_items(Item* out, const std::vector<unsigned>& count, const std::vector<int>& ncol,
                            int schedule) {
    size_t k = 0;
    const size_t n = count.size();
    if (schedule != EBIT_SCHED_INTERLEAVED) {
      for (size_t g = 0; g < n; ++g) {
        const int nr = (int)(count[g] / ncol[g]);
        for (int ty = 0; ty < nr; ++ty)
          for (int tx = 0; tx < ncol[g]; ++tx) out[k++] = Item{(int)g, tx, ty};
      }
      return k;
    }
    // round robin: each grid's next tile (column, row) advanced in turn
    std::vector<int> cx(n, 0), cy(n, 0);
    unsigned longest = 0;
    for (size_t g = 0; g < n; ++g) longest = std::max(longest, count[g]);
    for (unsigned t = 0; t < longest; ++t)
      for (size_t g = 0; g < n; ++g) {
        if (t >= count[g]) continue;
        out[k++] = Item{(int)g, cx[g], cy[g]};
        if (++cx[g] == ncol[g]) {
          cx[g] = 0;
          ++cy[g];
        }
      }
    return k;
  }

  // Descriptors of the coming step: lam and the split order of every grid.
  void fill() {
    const size_t n = inst.size();
    for (size_t g = 0; g < n; ++g) {
      Instance* in = inst[g];
      ebit_ctx* c = in->ctx;
      const int A = c->cur, B = 1 - c->cur;
      const double t = in->done * in->dt;
      double dte = in->req.field == EBIT_FIELD_VORTEX ? in->dt * std::cos(M_PI * t / in->req.period) : in->dt;
      if (in->req.fault_dt_factor != 0.0 && in->done >= in->req.fault_after) dte *= in->req.fault_dt_factor;
      const R lam = (R)(dte / c->grid.dx);
      const int x_first = ((c->step_index & 1) == 0);
      const int lo = (c->grid.flags & EBIT_FIT_LINE) ? 1 : 0;
      auto gv0 = [&](int s) {
        return ebit::GView<R, 0>{c->K[s], c->Z[s], (const R*)c->sH[s], (const R*)c->sV[s], (const R*)in->u, c->L.d, lam};
      };
      auto gv1 = [&](int s) {
        return ebit::GView<R, 1>{c->K[s], c->Z[s], (const R*)c->sH[s], (const R*)c->sV[s], (const R*)in->v, c->L.d, lam};
      };
      auto buf = [&](int s) { return ebit::Buf<R>{c->K[s], c->Z[s], (R*)c->sH[s], (R*)c->sV[s]}; };
      // first sweep A -> B, second sweep B -> A
      h_s0[g] = ebit::SweepDesc<R, 0>{gv0(A), buf(B), c->ctr, c->cfl_bits, c->status, lo, x_first};
      h_s1[g] = ebit::SweepDesc<R, 1>{gv1(A), buf(B), c->ctr, c->cfl_bits, c->status, lo, !x_first};
      h_s1[n + g] = ebit::SweepDesc<R, 1>{gv1(B), buf(A), c->ctr, c->cfl_bits, c->status, lo, x_first};
      h_s0[n + g] = ebit::SweepDesc<R, 0>{gv0(B), buf(A), c->ctr, c->cfl_bits, c->status, lo, !x_first};
      const bool unreachable = in->req.fault_wait != 0 && in->done >= in->req.fault_after;
      h_need[g] = tiles[g] + (unreachable ? 1u : 0u);
    }
  }

  // The launch sequence of one step on stream st.
  ebit_status launch(cudaStream_t st, bool persistent, unsigned long long budget_ns) {
    if (inst.empty()) return EBIT_OK;
    const size_t n = inst.size();
    constexpr size_t smem = ebit::tile_smem_bytes<R, ebit::batch_cand_cap<R>()>();
    cudaMemcpyAsync(d_s0, h_s0, 2 * n * sizeof(ebit::SweepDesc<R, 0>), cudaMemcpyHostToDevice, st);
    cudaMemcpyAsync(d_s1, h_s1, 2 * n * sizeof(ebit::SweepDesc<R, 1>), cudaMemcpyHostToDevice, st);
    // the requests' grids are square, so the x and y tiles of a grid are the
    // same work items (each tile swept in the direction its grid's split
    // order gives): either one persistent launch for both sweeps of all
    // grids, or the first sweeps of all grids in one launch and the second
    // sweeps in the next
    if (persistent) {
      cudaMemcpyAsync(d_need, h_need, n * sizeof(unsigned), cudaMemcpyHostToDevice, st);
      cudaMemsetAsync(d_ctl, 0, (n + 1) * sizeof(unsigned), st);
      const ebit::PersistCtl P{d_ctl, d_need, n_items0, (int)n, budget_ns};
      ebit::k_sweep_persistent<R><<<persist_blocks, ebit::tile_threads<R>(), smem, st>>>(d_s0, d_s1, d_items0, P);
    } else {
      ebit::k_sweep_tile_both<R, ebit::batch_cand_cap<R>()><<<n_items0, ebit::tile_threads<R>(), smem, st>>>(d_s0, d_s1, d_items0);
      ebit::k_sweep_tile_both<R, ebit::batch_cand_cap<R>()><<<n_items0, ebit::tile_threads<R>(), smem, st>>>(d_s0 + n, d_s1 + n, d_items0);
    }
    if (!ghf.empty()) k_ghf_reset<R><<<(unsigned)((n + 127) / 128), 128, 0, st>>>(d_fd, (int)n);
    ebit::k_fields_tile_batch<R><<<n_fitems, ebit::field_threads<R>(), 0, st>>>(d_fd, d_fitems);
    k_area_batch<<<(unsigned)n, 256, 0, st>>>(d_ad);
    for (const int g : ghf) {  // the state is back in the buffer the plan was built on
      const ebit_ctx* c = inst[g]->ctx;
      const int b = c->cur;
      const ebit::GhfView<R> S{c->K[b], c->Z[b], (const R*)c->sH[b], (const R*)c->sV[b], (const R*)c->C, c->L.d};
      const long long cells = (long long)c->L.d.nx * c->L.d.ny;
      const int blocks = (int)std::min<long long>((cells + ebit::kGhfThreads - 1) / ebit::kGhfThreads, 152LL * 8);
      ebit::k_ghf_fit<R><<<blocks, ebit::kGhfThreads, 0, st>>>(S, (R)c->grid.dx, c->ghf_list, c->ghf_count,
                                                              (R*)c->kappa, c->ctr);
    }
    const cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? EBIT_OK : fail_s(EBIT_ECUDA, "batch launch: %s", cudaGetErrorString(e));
  }
};

}  // namespace

unsigned ebit_detail::server_check_misses() {
#ifdef EBIT_CHECK
  unsigned w = 0;
  if (cudaMemcpyFromSymbol(&w, ebit::ebit_check_word, sizeof w) != cudaSuccess) {
    cudaGetLastError();
    return 1u;
  }
  return w;
#else
  return 0u;
#endif
}

namespace {

template <typename R>
ebit_status set_batch_attributes() {
  constexpr size_t smem = ebit::tile_smem_bytes<R, ebit::batch_cand_cap<R>()>();
  if (cudaFuncSetAttribute(ebit::k_sweep_tile_both<R, ebit::batch_cand_cap<R>()>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
      cudaFuncSetAttribute(ebit::k_sweep_persistent<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return fail_s(EBIT_ECUDA, "cudaFuncSetAttribute (batch)");
  }
  return EBIT_OK;
}

}  // namespace

struct ebit_server {
  size_t budget = 0, in_use = 0;
  ebit_server_opts opts{};
  std::mutex mu;
  std::condition_variable cv;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<std::unique_ptr<Instance>> queue;
  std::vector<std::unique_ptr<Instance>> active;
  std::map<uint64_t, ebit_result> done;
  std::map<uint64_t, int> pending;  // tickets queued or running
  std::set<uint64_t> cancels;       // running tickets to cancel at the next step boundary
  std::thread worker;
  bool started = false;
  // statistics
  int64_t batch_steps = 0, cell_updates = 0;
  double busy_ms = 0.0;
  // host time the worker spends with no batch step in flight
  int64_t plans = 0;
  double plan_ms = 0.0, plan_graph_ms = 0.0, admit_idle_ms = 0.0, retire_ms = 0.0;
  // worker-only
  cudaStream_t stream = nullptr;        // batch steps
  cudaStream_t admit_stream = nullptr;  // initialisation of admitted grids
  cudaEvent_t ev_a = nullptr, ev_b = nullptr;
  Group<float> g32;
  Group<double> g64;
  // status words of the grids of the current plan, gathered each step
  int** d_status = nullptr;  // device array of the grids' status pointers
  int* h_status = nullptr;   // host-mapped copy written by k_status_gather
  int* h_status_dev = nullptr;
  int** h_status_ptrs = nullptr;  // pinned staging of d_status
  size_t status_cap = 0;     // grids the two status buffers hold (they only grow)
  std::vector<Instance*> stepping;  // the grids of the step in flight, plan order
  bool dirty = true;   // the set of grids changed: new plans, new schedule choice
  bool replan = false; // same set, another schedule (autotuning)
  cudaGraphExec_t graph = nullptr;
  // CTA-schedule autotuner: the first kTuneSteps steps of a new set of grids
  // run under each schedule in turn (the work and its results do not depend
  // on the order, so no step is wasted); the fastest is kept for the set and
  // for later sets with the same signature
  static constexpr int kTuneSteps = 2;
  int sched = EBIT_SCHED_LARGEST_FIRST;
  bool tuning = false;
  uint64_t sig = 0;
  double tune_acc[EBIT_SCHED_COUNT] = {0.0, 0.0, 0.0};
  int tune_cnt[EBIT_SCHED_COUNT] = {0, 0, 0};
  double last_tune_ms[EBIT_SCHED_COUNT] = {0.0, 0.0, 0.0};
  std::map<uint64_t, int> tuned;

  uint64_t signature(const std::vector<Instance*>& all) const;
  void tune_after(float ms);

  void run();
  void take_admissible(std::vector<std::unique_ptr<Instance>>& out);  // caller holds mu
  void admit_all(std::vector<std::unique_ptr<Instance>>& admitted);
  ebit_status admit(Instance* in);
  void retire(size_t idx);
  ebit_status plan();
  ebit_status launch_all();
  ebit_status step_launch();
  ebit_status step_finish();
  void release_status();
};

ebit_status ebit_server::admit(Instance* in) {
  const ebit_request& r = in->req;
  ebit_grid g{r.n, r.n, 1.0 / r.n, r.prec, r.flags};
  ebit_scene sc{in->circles.empty() ? nullptr : in->circles.data(), (int32_t)in->circles.size(), nullptr, nullptr};
  // the grid is set up on the admission stream, so that a batch step in
  // flight on the server's stream goes on meanwhile; its context keeps that
  // stream for its own calls (area, status) between batch steps
  ebit_status s = ebit_init(&in->ctx, &g, &sc, admit_stream);
  if (s != EBIT_OK) return s;
  const size_t esz = r.prec == EBIT_FP32 ? 4 : 8;
  const size_t vb = (size_t)(r.n + 1) * (r.n + 1) * esz;
  if (cudaMalloc(&in->u, vb) != cudaSuccess || cudaMalloc(&in->v, vb) != cudaSuccess) {
    cudaGetLastError();
    return fail_s(EBIT_ENOMEM, "velocity allocation");
  }
  const int nb = (int)(((long long)(r.n + 1) * (r.n + 1) + 255) / 256);
  if (r.prec == EBIT_FP32)
    k_velocity<float><<<nb, 256, 0, admit_stream>>>(r.field, r.n, 1.0 / r.n, r.omega, r.cx, r.cy, r.drift_u, r.drift_v, (float*)in->u, (float*)in->v);
  else
    k_velocity<double><<<nb, 256, 0, admit_stream>>>(r.field, r.n, 1.0 / r.n, r.omega, r.cx, r.cy, r.drift_u, r.drift_v, (double*)in->u, (double*)in->v);
  in->dx = 1.0 / r.n;
  in->dt = r.cfl * in->dx / field_umax(r);
  if ((s = ebit_fraction(in->ctx, nullptr, &in->area0)) != EBIT_OK) return s;
  cudaMemsetAsync(in->ctx->ctr, 0, ebit::kCounters * sizeof(unsigned long long), admit_stream);
  if (cudaStreamSynchronize(admit_stream) != cudaSuccess) return fail_s(EBIT_ECUDA, "admission");
  in->t_admit = now_ms();
  return EBIT_OK;
}

void ebit_server::retire(size_t idx) {
  Instance* in = active[idx].get();
  const cudaStream_t cs = in->ctx->stream;
  ebit_result res{};
  res.status = EBIT_OK;
  res.steps = in->done;
  res.area0 = in->area0;
  unsigned long long ctr[ebit::kCounters] = {0};
  ebit_status s = ebit_fraction(in->ctx, nullptr, &res.area);
  // a CFL or invariant status was already taken into `failed`; the copy of
  // the results below still runs
  if (s == EBIT_ECFL || s == EBIT_EINVARIANT) s = EBIT_OK;
  if (s == EBIT_OK) {
    cudaMemcpyAsync(ctr, in->ctx->ctr, sizeof ctr, cudaMemcpyDeviceToHost, cs);
    if (in->req.C_out)
      cudaMemcpy2DAsync(in->req.C_out, (size_t)in->req.n * (in->req.prec == EBIT_FP32 ? 4 : 8),
                        in->ctx->C, (size_t)in->ctx->L.d.P * in->ctx->L.esz,
                        (size_t)in->req.n * in->ctx->L.esz, in->req.n, cudaMemcpyDeviceToHost, cs);
    if (cudaStreamSynchronize(cs) != cudaSuccess) s = EBIT_ECUDA;
  }
  res.status = in->failed != EBIT_OK ? in->failed : s;
  for (int t = 0; t < EBIT_D_COUNT; ++t) res.counters[t] = (int64_t)ctr[t];
  res.e_area = in->area0 != 0.0 ? std::fabs(res.area - in->area0) / in->area0 : 0.0;
  res.run_ms = now_ms() - in->t_admit;
  res.queue_ms = in->t_admit - in->t_submit;
  res.cell_updates = (int64_t)in->req.n * in->req.n * in->done;
  std::vector<float> l = in->lat_ms;
  if (!l.empty()) {
    std::sort(l.begin(), l.end());
    res.step_p50_ms = l[(size_t)(0.50 * (l.size() - 1))];
    res.step_p99_ms = l[(size_t)(0.99 * (l.size() - 1))];
  }
  ebit_destroy(in->ctx);
  cudaFree(in->u);
  cudaFree(in->v);
  {
    std::lock_guard<std::mutex> lk(mu);
    done[in->ticket] = res;
    pending.erase(in->ticket);
    cancels.erase(in->ticket);
    in_use -= in->bytes;
  }
  active.erase(active.begin() + idx);
  dirty = true;
  cv.notify_all();
}

void ebit_server::release_status() {
  if (d_status) cudaFree(d_status);
  if (h_status) cudaFreeHost(h_status);
  if (h_status_ptrs) cudaFreeHost(h_status_ptrs);
  d_status = nullptr;
  h_status = nullptr;
  h_status_ptrs = nullptr;
  h_status_dev = nullptr;
  status_cap = 0;
}

// Launch plans (and the captured graph) for the current set of grids.
ebit_status ebit_server::plan() {
  std::vector<Instance*> all;
  for (auto& p : active) all.push_back(p.get());
  ebit_status s;
  if (dirty) {
    sig = signature(all);
    tuning = false;
    if (!opts.autotune) {
      sched = (opts.schedule >= 0 && opts.schedule < EBIT_SCHED_COUNT) ? opts.schedule : 0;
    } else {
      const auto it = tuned.find(sig);
      if (it != tuned.end()) {
        sched = it->second;
      } else {
        tuning = true;
        sched = 0;
        for (int q = 0; q < EBIT_SCHED_COUNT; ++q) {
          tune_acc[q] = 0.0;
          tune_cnt[q] = 0;
        }
      }
    }
  }
  if (!dirty && !replan) return EBIT_OK;
  const double t0 = now_ms();
  // nothing of an earlier plan is still being copied from the pinned staging
  // (a plan whose step was never launched leaves its copies queued)
  if (cudaStreamSynchronize(stream) != cudaSuccess) return fail_s(EBIT_ECUDA, "plan: stream");
  // the previous step's graph is updated in place when the new launch
  // sequence has its shape (same kernels, same nodes), else replaced; it is
  // destroyed on every path that does not keep it
  struct ExecGuard {
    cudaGraphExec_t e;
    ~ExecGuard() {
      if (e) cudaGraphExecDestroy(e);
    }
  } old{graph};
  graph = nullptr;
  // the work-item order of the schedule (its persistent twin has the same)
  const int order = sched % EBIT_SCHED_PERSISTENT_LARGEST_FIRST;
  if ((s = g32.build(all, EBIT_FP32, order, stream)) != EBIT_OK) return s;
  if ((s = g64.build(all, EBIT_FP64, order, stream)) != EBIT_OK) return s;
  // the status words in plan order: the float group's grids, then the double group's
  stepping.clear();
  stepping.insert(stepping.end(), g32.inst.begin(), g32.inst.end());
  stepping.insert(stepping.end(), g64.inst.begin(), g64.inst.end());
  const size_t n = stepping.size();
  std::vector<int*> ptrs(n);
  for (size_t g = 0; g < n; ++g) ptrs[g] = stepping[g]->ctx->status;
  if (n > status_cap) {
    release_status();
    const size_t cap = std::max<size_t>(64, 2 * n);
    if (cudaMalloc((void**)&d_status, cap * sizeof(int*)) != cudaSuccess ||
        cudaMallocHost((void**)&h_status_ptrs, cap * sizeof(int*)) != cudaSuccess ||
        cudaHostAlloc((void**)&h_status, cap * sizeof(int), cudaHostAllocMapped) != cudaSuccess ||
        cudaHostGetDevicePointer((void**)&h_status_dev, h_status, 0) != cudaSuccess) {
      cudaGetLastError();
      return fail_s(EBIT_ENOMEM, "status plan");
    }
    status_cap = cap;
  }
  std::memset(h_status, 0, n * sizeof(int));
  std::memcpy(h_status_ptrs, ptrs.data(), n * sizeof(int*));
  if (cudaMemcpyAsync(d_status, h_status_ptrs, n * sizeof(int*), cudaMemcpyHostToDevice, stream) != cudaSuccess)
    return fail_s(EBIT_ECUDA, "status plan upload");
  const double tg = now_ms();
  if (opts.use_graphs) {
    cudaGraph_t gr = nullptr;
    if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
      return fail_s(EBIT_ECUDA, "begin capture");
    const ebit_status s1 = launch_all();
    if (cudaStreamEndCapture(stream, &gr) != cudaSuccess || s1 != EBIT_OK)
      return fail_s(EBIT_ECUDA, "capture of the batch step");
    cudaError_t e = cudaErrorUnknown;
    if (old.e) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(old.e, gr, &info) == cudaSuccess) {
        graph = old.e;
        old.e = nullptr;
        e = cudaSuccess;
      } else {
        cudaGetLastError();  // another shape: instantiated anew below
      }
    }
    if (!graph) e = cudaGraphInstantiate(&graph, gr, 0);
    cudaGraphDestroy(gr);
    if (e != cudaSuccess) {
      graph = nullptr;
      return fail_s(EBIT_ECUDA, "graph instantiate: %s", cudaGetErrorString(e));
    }
  }
  dirty = false;
  replan = false;
  {
    const double t1 = now_ms();
    std::lock_guard<std::mutex> lk(mu);
    plans += 1;
    plan_ms += t1 - t0;
    plan_graph_ms += t1 - tg;
  }
  return EBIT_OK;
}

// The launches of one batch step on the server's stream (captured into the
// graph, or issued directly when graphs are off).
ebit_status ebit_server::launch_all() {
  const bool persistent = sched >= EBIT_SCHED_PERSISTENT_LARGEST_FIRST;
  const unsigned long long budget_ns =
      (unsigned long long)(opts.wait_budget_ms > 0 ? opts.wait_budget_ms : 1000) * 1000000ull;
  ebit_status a = g32.launch(stream, persistent, budget_ns);
  if (a != EBIT_OK) return a;
  if ((a = g64.launch(stream, persistent, budget_ns)) != EBIT_OK) return a;
  const size_t n = stepping.size();
  k_status_gather<<<(unsigned)((n + 127) / 128), 128, 0, stream>>>(d_status, (int)n, h_status_dev);
  return cudaGetLastError() == cudaSuccess ? EBIT_OK : fail_s(EBIT_ECUDA, "status gather launch");
}

// Enqueues one batch step of the planned grids; returns without waiting.
ebit_status ebit_server::step_launch() {
  const ebit_detail::Range range("ebit_server_step");
  ebit_status s = plan();
  if (s != EBIT_OK) return s;
  g32.fill();
  g64.fill();
  cudaEventRecord(ev_a, stream);
  if (graph) {
    if (cudaGraphLaunch(graph, stream) != cudaSuccess) return fail_s(EBIT_ECUDA, "graph launch");
  } else if ((s = launch_all()) != EBIT_OK) {
    return s;
  }
  cudaEventRecord(ev_b, stream);
  return EBIT_OK;
}

// Waits for the step in flight and accounts it; grids whose status word
// reports an error are marked failed (they leave the batch).
ebit_status ebit_server::step_finish() {
  if (cudaEventSynchronize(ev_b) != cudaSuccess) return fail_s(EBIT_ECUDA, "batch step");
  float ms = 0.0f;
  cudaEventElapsedTime(&ms, ev_a, ev_b);
  if (tuning) tune_after(ms);
  int64_t cells = 0;
  for (size_t g = 0; g < stepping.size(); ++g) {
    Instance* in = stepping[g];
    in->lat_ms.push_back(ms);
    in->done += 1;
    in->ctx->step_index += 1;
    cells += (int64_t)in->req.n * in->req.n;
    const int st = ((volatile int*)h_status)[g];
    if (st && in->failed == EBIT_OK)
      in->failed = (st & ebit::ST_TIMEOUT) ? EBIT_ETIMEOUT
                 : (st & ebit::ST_INVARIANT) ? EBIT_EINVARIANT : EBIT_ECFL;
  }
  std::lock_guard<std::mutex> lk(mu);
  batch_steps += 1;
  cell_updates += cells;
  busy_ms += ms;
  return EBIT_OK;
}

// Coarse signature of a set of grids: the number of grids and the total cell
// count per precision, on a logarithmic scale.
uint64_t ebit_server::signature(const std::vector<Instance*>& all) const {
  uint64_t cnt[2] = {0, 0}, cells[2] = {0, 0};
  for (const Instance* in : all) {
    const int p = in->req.prec == EBIT_FP32 ? 1 : 0;
    cnt[p] += 1;
    cells[p] += (uint64_t)in->req.n * in->req.n;
  }
  auto lg = [](uint64_t v) { return v ? (uint64_t)(64 - __builtin_clzll(v)) : 0ull; };
  return lg(cnt[0]) | (lg(cnt[1]) << 8) | (lg(cells[0]) << 16) | (lg(cells[1]) << 24);
}

void ebit_server::tune_after(float ms) {
  tune_acc[sched] += ms;
  tune_cnt[sched] += 1;
  if (tune_cnt[sched] < kTuneSteps) return;
  if (sched + 1 < EBIT_SCHED_COUNT) {
    sched += 1;
    replan = true;
    return;
  }
  int best = 0;
  for (int q = 0; q < EBIT_SCHED_COUNT; ++q) {
    last_tune_ms[q] = tune_acc[q] / tune_cnt[q];
    if (last_tune_ms[q] < last_tune_ms[best]) best = q;
  }
  tuned[sig] = best;
  tuning = false;
  if (best != sched) {
    sched = best;
    replan = true;
  }
}

// Moves the queued requests that fit the budget (first come first served
// among those that fit) to out; the caller holds mu.
void ebit_server::take_admissible(std::vector<std::unique_ptr<Instance>>& out) {
  for (auto it = queue.begin(); it != queue.end();) {
    const bool room = in_use + (*it)->bytes <= budget &&
                      (opts.max_instances <= 0 ||
                       (int)(active.size() + out.size()) < opts.max_instances);
    if (room) {
      in_use += (*it)->bytes;
      out.push_back(std::move(*it));
      it = queue.erase(it);
    } else {
      ++it;
    }
  }
}

void ebit_server::admit_all(std::vector<std::unique_ptr<Instance>>& admitted) {
  for (auto& in : admitted) {
    const ebit_status s = admit(in.get());
    if (s != EBIT_OK) {
      ebit_result r{};
      r.status = s;
      if (in->ctx) ebit_destroy(in->ctx);
      if (in->u) cudaFree(in->u);
      if (in->v) cudaFree(in->v);
      std::lock_guard<std::mutex> lk(mu);
      done[in->ticket] = r;
      pending.erase(in->ticket);
      in_use -= in->bytes;
      cv.notify_all();
      continue;
    }
    active.push_back(std::move(in));
    dirty = true;
  }
  admitted.clear();
}

void ebit_server::run() {
  cudaSetDevice(opts.device);
  if (cudaStreamCreateWithFlags(&stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&admit_stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&ev_a) != cudaSuccess || cudaEventCreate(&ev_b) != cudaSuccess ||
      set_batch_attributes<float>() != EBIT_OK || set_batch_attributes<double>() != EBIT_OK) {
    std::lock_guard<std::mutex> lk(mu);
    for (auto& q : queue) {
      ebit_result r{};
      r.status = EBIT_ECUDA;
      done[q->ticket] = r;
      pending.erase(q->ticket);
    }
    queue.clear();
    stop = true;
    cv.notify_all();
    return;
  }
  for (;;) {
    // between batch steps (nothing in flight): cancellations, and admission
    // when no grid runs
    std::vector<std::unique_ptr<Instance>> admitted;
    std::set<uint64_t> cancel_now;
    {
      std::unique_lock<std::mutex> lk(mu);
      if (active.empty())
        cv.wait(lk, [&] { return stop || !queue.empty(); });
      if (stop && queue.empty() && active.empty()) break;
      if (stop) {
        // cancel what is queued; finish nothing further
        for (auto& q : queue) {
          ebit_result r{};
          r.status = EBIT_ECANCELLED;
          done[q->ticket] = r;
          pending.erase(q->ticket);
        }
        queue.clear();
      }
      // with grids running, what fits is admitted while their next step
      // runs (below), not here with the GPU idle
      if (active.empty()) take_admissible(admitted);
      cancel_now.swap(cancels);
    }
    const double ta = now_ms();
    admit_all(admitted);
    for (size_t i = active.size(); i-- > 0;)
      if (cancel_now.count(active[i]->ticket)) {
        active[i]->failed = EBIT_ECANCELLED;
        retire(i);
      }
    {
      std::lock_guard<std::mutex> lk(mu);
      admit_idle_ms += now_ms() - ta;
    }
    if (stop) {
      while (!active.empty()) retire(active.size() - 1);
      continue;
    }
    if (active.empty()) continue;
    ebit_status s = step_launch();
    if (s == EBIT_OK) {
      // while the step runs: admit what arrived meanwhile (those grids join
      // from the next step on)
      std::vector<std::unique_ptr<Instance>> more;
      {
        std::lock_guard<std::mutex> lk(mu);
        take_admissible(more);
      }
      // the step in flight keeps its own grid list (stepping); the plan is
      // rebuilt before the next one
      if (!more.empty()) admit_all(more);
      s = step_finish();
    }
    if (s != EBIT_OK) {
      // fail every running request and carry on with an empty set
      for (auto& in : active) {
        in->failed = s;
        in->req.steps = (int32_t)in->done;
      }
    }
    const double tr = now_ms();
    for (size_t i = active.size(); i-- > 0;)
      if (active[i]->done >= active[i]->req.steps || active[i]->failed != EBIT_OK) retire(i);
    {
      std::lock_guard<std::mutex> lk(mu);
      retire_ms += now_ms() - tr;
    }
  }
  if (graph) cudaGraphExecDestroy(graph);
  g32.release();
  g64.release();
  release_status();
  cudaEventDestroy(ev_a);
  cudaEventDestroy(ev_b);
  cudaStreamDestroy(admit_stream);
  cudaStreamDestroy(stream);
}

extern "C" {

ebit_status ebit_server_create(ebit_server** out, size_t hbm_budget, const ebit_server_opts* opts) {
  if (!out) return fail_s(EBIT_EINVAL, "out is NULL");
  *out = nullptr;
  if (hbm_budget == 0) return fail_s(EBIT_EINVAL, "zero memory budget");
  ebit_server* s = new (std::nothrow) ebit_server;
  if (!s) return fail_s(EBIT_ENOMEM, "host allocation failed");
  s->budget = hbm_budget;
  if (opts) {
    s->opts = *opts;
  } else {
    s->opts.use_graphs = 1;
    s->opts.autotune = 1;
  }
  *out = s;
  return EBIT_OK;
}

ebit_status ebit_submit(ebit_server* s, const ebit_request* r, uint64_t* ticket) {
  if (!s || !r || !ticket) return fail_s(EBIT_EINVAL, "NULL argument");
  if (r->n < 1 || r->n > ebit_detail::kMaxSide || (r->prec != EBIT_FP32 && r->prec != EBIT_FP64) ||
      r->steps < 0 || !(r->cfl > 0.0 && r->cfl <= 1.0) || r->ncircles < 0 ||
      (r->ncircles > 0 && !r->circles) ||
      (r->field != EBIT_FIELD_VORTEX && r->field != EBIT_FIELD_CELLULAR && r->field != EBIT_FIELD_ROTATION) ||
      (r->field == EBIT_FIELD_VORTEX && !(r->period > 0.0)) || (r->flags & ~(EBIT_FIT_LINE | EBIT_CURV_GHF)))
    return fail_s(EBIT_EINVAL, "invalid request");
  auto in = std::make_unique<Instance>();
  in->req = *r;
  in->circles.assign(r->circles, r->circles + r->ncircles);
  in->req.circles = nullptr;
  in->bytes = request_bytes(*r);
  if (in->bytes > s->budget)
    return fail_s(EBIT_EFULL, "request needs %zu bytes, more than the whole budget (%zu)", in->bytes, s->budget);
  in->t_submit = now_ms();
  std::lock_guard<std::mutex> lk(s->mu);
  if (s->stop) return fail_s(EBIT_EINVAL, "server is shutting down");
  in->ticket = s->next_ticket++;
  *ticket = in->ticket;
  s->pending[in->ticket] = 1;
  s->queue.push_back(std::move(in));
  if (!s->started) {
    s->started = true;
    s->worker = std::thread([s] { s->run(); });
  }
  s->cv.notify_all();
  return EBIT_OK;
}

ebit_status ebit_poll(ebit_server* s, uint64_t ticket, ebit_result* out) {
  if (!s || !out) return fail_s(EBIT_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  auto it = s->done.find(ticket);
  if (it != s->done.end()) {
    *out = it->second;
    s->done.erase(it);
    return EBIT_OK;
  }
  if (s->pending.count(ticket)) return EBIT_EAGAIN;
  return fail_s(EBIT_EINVAL, "unknown ticket %llu", (unsigned long long)ticket);
}

ebit_status ebit_cancel(ebit_server* s, uint64_t ticket) {
  if (!s) return fail_s(EBIT_EINVAL, "NULL server");
  std::lock_guard<std::mutex> lk(s->mu);
  if (!s->pending.count(ticket)) return fail_s(EBIT_EINVAL, "unknown or finished ticket %llu",
                                               (unsigned long long)ticket);
  for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
    if ((*it)->ticket == ticket) {  // not admitted yet: dropped at once
      ebit_result r{};
      r.status = EBIT_ECANCELLED;
      r.queue_ms = now_ms() - (*it)->t_submit;
      s->done[ticket] = r;
      s->pending.erase(ticket);
      s->queue.erase(it);
      s->cv.notify_all();
      return EBIT_OK;
    }
  s->cancels.insert(ticket);  // running: leaves before the next batch step
  return EBIT_OK;
}

ebit_status ebit_server_stats_get(ebit_server* s, ebit_server_stats* out) {
  if (!s || !out) return fail_s(EBIT_EINVAL, "NULL argument");
  std::lock_guard<std::mutex> lk(s->mu);
  out->queued = (int64_t)s->queue.size();
  out->running = (int64_t)s->pending.size() - (int64_t)s->queue.size();
  out->batch_steps = s->batch_steps;
  out->cell_updates = s->cell_updates;
  out->busy_ms = s->busy_ms;
  out->bytes_in_use = s->in_use;
  out->schedule = s->sched;
  out->tuned_sets = (int32_t)s->tuned.size();
  for (int q = 0; q < EBIT_SCHED_COUNT; ++q) out->tune_ms[q] = s->last_tune_ms[q];
  out->plans = s->plans;
  out->plan_ms = s->plan_ms;
  out->plan_graph_ms = s->plan_graph_ms;
  out->admit_idle_ms = s->admit_idle_ms;
  out->retire_ms = s->retire_ms;
  return EBIT_OK;
}

void ebit_server_destroy(ebit_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv.notify_all();
  if (s->worker.joinable()) s->worker.join();
  delete s;
}

}  // extern "C"
