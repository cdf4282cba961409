// Internal: the device layout of one EBIT context, shared by the translation
// units of libebit.so (not part of the exported interface).
#pragma once
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include <cstddef>
#include <cstdint>
#include <vector>

#include "ebit.h"
#include "ebit_device.cuh"

namespace ebit_detail {

// The index-check word of the server's kernels (debug builds; 0 otherwise).
unsigned server_check_misses();

// NVTX range over a host call (visible in profilers that record NVTX; a
// no-op otherwise).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
  Range(const Range&) = delete;
  Range& operator=(const Range&) = delete;
};

constexpr int kMaxSide = 32768;
constexpr int kBlockX = 32, kBlockY = 8;  // thread blocks of the per-vertex kernels

struct Layout {
  ebit::Dims d;
  size_t esz;
  size_t k_bytes, z_bytes, h_bytes, v_bytes, field_bytes, partial_count, ghf_bytes;
  dim3 grid, block;
  size_t total() const {
    return 2 * (k_bytes + z_bytes + h_bytes + v_bytes) + 2 * field_bytes +
           partial_count * sizeof(double) + ghf_bytes + 4096;
  }
};

inline bool valid_grid(const ebit_grid* g) {
  return g && g->nx >= 1 && g->ny >= 1 && g->nx <= kMaxSide && g->ny <= kMaxSide && g->dx > 0.0 &&
         (g->prec == EBIT_FP64 || g->prec == EBIT_FP32) &&
         (g->flags & ~(EBIT_FIT_LINE | EBIT_CURV_GHF)) == 0;
}

inline Layout layout_of(const ebit_grid* g) {
  Layout L;
  L.d.nx = g->nx;
  L.d.ny = g->ny;
  L.d.kw = (g->nx + 1 + 31) / 32;
  L.d.zw = (g->nx + 31) / 32;
  L.d.P = ((long long)g->nx + 1 + 31) / 32 * 32;
  L.esz = g->prec == EBIT_FP32 ? 4 : 8;
  L.k_bytes = (size_t)(g->ny + 1) * L.d.kw * 4;
  L.z_bytes = (size_t)g->ny * L.d.zw * 4;
  L.h_bytes = (size_t)(g->ny + 1) * L.d.P * L.esz;
  L.v_bytes = (size_t)g->ny * L.d.P * L.esz;
  L.field_bytes = (size_t)g->ny * L.d.P * L.esz;
  L.ghf_bytes = (g->flags & EBIT_CURV_GHF) ? (size_t)g->nx * g->ny * sizeof(int) + 256 : 0;
  L.block = dim3(kBlockX, kBlockY);
  L.grid = dim3((g->nx + 1 + kBlockX - 1) / kBlockX, (g->ny + 1 + kBlockY - 1) / kBlockY);
  L.partial_count = (size_t)L.grid.x * L.grid.y;
  return L;
}

}  // namespace ebit_detail

struct ebit_ctx {
  ebit_grid grid;
  ebit_detail::Layout L;
  cudaStream_t stream = nullptr;
  uint32_t* K[2] = {nullptr, nullptr};
  uint32_t* Z[2] = {nullptr, nullptr};
  void* sH[2] = {nullptr, nullptr};
  void* sV[2] = {nullptr, nullptr};
  int cur = 0;  // buffer holding the current state
  void* C = nullptr;
  void* kappa = nullptr;
  double* partial = nullptr;
  double* area = nullptr;
  unsigned* area_done = nullptr;    // tiles of the fields launch done (reset by its last tile)
  unsigned long long* ctr = nullptr;
  unsigned long long* cfl_bits = nullptr;
  int* status = nullptr;
  int* ghf_list = nullptr;          // EBIT_CURV_GHF: cells left without kappa
  unsigned* ghf_count = nullptr;
  int64_t step_index = 0;
  // ebit_fraction_to_host: the copy of C on the caller's stream, which the
  // next fields launch waits for
  cudaEvent_t ev_queued = nullptr, ev_c_read = nullptr;
  bool c_read_pending = false;
  std::vector<void*> allocs;
  // per-kernel event timing (off unless ebit_set_timing)
  bool timing = false;
  struct Mark {
    cudaEvent_t a, b;
    int kind;
  };
  std::vector<Mark> marks;
  size_t marks_used = 0;
};

// Error message of the calling thread (reported by ebit_last_error).
__attribute__((visibility("hidden"))) void ebit_detail_set_error(const char* msg);
