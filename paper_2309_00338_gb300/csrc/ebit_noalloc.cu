// ebit_fraction_noalloc: the volume-fraction kernel for callers that cannot
// allocate device memory.
//
// Some callers of this library cannot call cudaMalloc: a host solver that
// allocates all of its device memory once at start-up and forbids allocation
// inside its time loop (cudaMalloc can synchronise the device, fail under a
// fixed memory budget, and fragment a pool the host framework manages), or a
// framework that hands this library only the buffers it owns.  For them this
// entry point computes fractions, total area and marker counts of a state held
// in the caller's own device buffers, and allocates nothing: its scratch (the
// per-block area partial sums and two marker counters) lives in the file-scope
// array below, which every GPU that loads the library holds until the process
// exits.
#include <cstdarg>
#include <cstdio>
#include <mutex>

#include "ebit.h"

// Sets the message returned by ebit_last_error() (defined with the other
// entry points; hidden from the exported interface).
__attribute__((visibility("hidden"))) void ebit_detail_set_error(const char* msg);

namespace {

constexpr int kBX = 32, kBY = 8;
// Scratch: kMaxBlocks area partials (as double bit patterns) then 2 counters.
constexpr long long kMaxBlocks = 1 << 17;  // 131072 blocks of 32x8 vertices (1 MiB)
static __device__ __align__(256) unsigned long long g_noalloc_scratch[kMaxBlocks + 2];

std::mutex g_mu;
void* g_addr[1024] = {};  // scratch device address per device ordinal

ebit_status fail_na(ebit_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  ebit_detail_set_error(buf);
  return s;
}

// Device address of the scratch array on the current device.  The first call
// on a device looks it up (with that device current) and caches it for the
// life of the process; a cudaDeviceReset would make the cached address stale,
// which the header tells callers.
ebit_status scratch_address(unsigned long long** out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail_na(EBIT_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= 1024) return fail_na(EBIT_ECUDA, "device ordinal %d out of range", dev);
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p)
      return fail_na(EBIT_ECUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = static_cast<unsigned long long*>(g_addr[dev]);
  return EBIT_OK;
}

__device__ __forceinline__ int emask(int q) { return (q ^ ((q >> 1) | ((q & 1) << 3))) & 15; }

// Reference-phase area of cell (i,j) from its markers and colour vertices
// (Sec. 2.5), byte layout of ebit_state_host, double arithmetic.
template <typename R>
__device__ double frac_bytes(const uint8_t* K, const uint8_t* Z, const R* sH, const R* sV, int nx,
                             int i, int j) {
  const long long w = nx + 1;
  const int q = (K[j * w + i] != 0) | ((K[j * w + i + 1] != 0) << 1) |
                ((K[(j + 1) * w + i + 1] != 0) << 2) | ((K[(j + 1) * w + i] != 0) << 3);
  const int em = emask(q);
  if (em == 0) return (double)(q & 1);
  const double s0 = (double)sH[(long long)j * nx + i];
  const double s1 = (double)sV[(long long)j * w + i + 1];
  const double s2 = (double)sH[(long long)(j + 1) * nx + i];
  const double s3 = (double)sV[(long long)j * w + i];
  auto tri = [&](int c) {
    double a, b;
    switch (c) {
      case 0: a = s3; b = s0; break;
      case 1: a = 1.0 - s0; b = s1; break;
      case 2: a = 1.0 - s1; b = 1.0 - s2; break;
      default: a = s2; b = 1.0 - s3; break;
    }
    return 0.5 * (a * b);
  };
  if (em != 15) {
    const int e1 = __ffs(em) - 1, e2 = 31 - __clz(em);
    const int c0 = q & 1;
    if (e2 - e1 == 2) {
      if (e1 == 0) return c0 ? 0.5 * (s0 + s2) : 0.5 * ((1.0 - s0) + (1.0 - s2));
      return c0 ? 0.5 * (s3 + s1) : 0.5 * ((1.0 - s3) + (1.0 - s1));
    }
    const int c = (e1 == 0 && e2 == 3) ? 0 : e2;
    const double T = tri(c);
    return ((q >> c) & 1) ? T : 1.0 - T;
  }
  const int zc = Z[(long long)j * nx + i] != 0;
  double Tsum = 0.0;
  bool first = true;
  for (int c = 0; c < 4; ++c)
    if (((q >> c) & 1) != zc) {
      if (first) { Tsum = tri(c); first = false; } else { Tsum = Tsum + tri(c); }
    }
  return zc == 0 ? Tsum : 1.0 - Tsum;
}

template <typename R>
__global__ void __launch_bounds__(kBX * kBY)
k_fraction_noalloc(const uint8_t* __restrict__ K, const uint8_t* __restrict__ Z,
                   const R* __restrict__ sH, const R* __restrict__ sV, int nx, int ny, R* C,
                   unsigned long long* scratch) {
  __shared__ double red[kBX * kBY];
  const int x = blockIdx.x * kBX + threadIdx.x;
  const int y = blockIdx.y * kBY + threadIdx.y;
  const int t = threadIdx.y * kBX + threadIdx.x;
  const long long w = nx + 1;
  double f = 0.0;
  if (x < nx && y < ny) {
    f = frac_bytes(K, Z, sH, sV, nx, x, y);
    C[(long long)y * nx + x] = (R)f;
  }
  int nh = (x < nx && y <= ny) ? ((K[y * w + x] != 0) != (K[y * w + x + 1] != 0)) : 0;
  int nv = (x <= nx && y < ny) ? ((K[y * w + x] != 0) != (K[(y + 1) * w + x] != 0)) : 0;
  nh = __reduce_add_sync(0xffffffffu, nh);
  nv = __reduce_add_sync(0xffffffffu, nv);
  if ((threadIdx.x & 31) == 0) {
    if (nh) atomicAdd(&scratch[kMaxBlocks], (unsigned long long)nh);
    if (nv) atomicAdd(&scratch[kMaxBlocks + 1], (unsigned long long)nv);
  }
  red[t] = f;
  __syncthreads();
  for (int s = (kBX * kBY) / 2; s > 0; s >>= 1) {
    if (t < s) red[t] = red[t] + red[t + s];
    __syncthreads();
  }
  if (t == 0)
    scratch[(long long)blockIdx.y * gridDim.x + blockIdx.x] = (unsigned long long)__double_as_longlong(red[0]);
}

// Fixed-order sum of the partials; copies the counters out.
__global__ void k_area_noalloc(const unsigned long long* scratch, long long n, double scale,
                               double* area, long long* counts) {
  __shared__ double red[256];
  double acc = 0.0;
  for (long long b = threadIdx.x; b < n; b += 256) acc = acc + __longlong_as_double((long long)scratch[b]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int s = 128; s > 0; s >>= 1) {
    if ((int)threadIdx.x < s) red[threadIdx.x] = red[threadIdx.x] + red[threadIdx.x + s];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    *area = red[0] * scale;
    if (counts) {
      counts[0] = (long long)scratch[kMaxBlocks];
      counts[1] = (long long)scratch[kMaxBlocks + 1];
    }
  }
}

}  // namespace

extern "C" ebit_status ebit_fraction_noalloc(const ebit_grid* grid, const uint8_t* K,
                                             const uint8_t* Z, const void* sH, const void* sV,
                                             void* C, double* area, int64_t* marker_counts,
                                             void* stream) {
  if (!grid || grid->nx < 1 || grid->ny < 1 || !(grid->dx > 0.0) ||
      (grid->prec != EBIT_FP64 && grid->prec != EBIT_FP32))
    return fail_na(EBIT_EINVAL, "invalid grid");
  if (!K || !Z || !sH || !sV || !C || !area) return fail_na(EBIT_EINVAL, "NULL buffer");
  const dim3 block(kBX, kBY);
  const dim3 g((grid->nx + 1 + kBX - 1) / kBX, (grid->ny + 1 + kBY - 1) / kBY);
  const long long nblocks = (long long)g.x * g.y;
  if (nblocks > kMaxBlocks)
    return fail_na(EBIT_EINVAL,
                   "grid %dx%d needs %lld blocks of 32x8 vertices; the no-allocation scratch holds "
                   "at most %lld (about 5790x5790 cells)",
                   grid->nx, grid->ny, nblocks, kMaxBlocks);
  unsigned long long* scratch = nullptr;
  ebit_status s = scratch_address(&scratch);
  if (s != EBIT_OK) return s;
  cudaStream_t st = (cudaStream_t)stream;
  // the counters accumulate with atomics: they must start at zero; the
  // partials are all written before they are read
  cudaError_t e = cudaMemsetAsync(scratch + kMaxBlocks, 0, 2 * sizeof(unsigned long long), st);
  if (e != cudaSuccess) return fail_na(EBIT_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
  if (grid->prec == EBIT_FP32)
    k_fraction_noalloc<float><<<g, block, 0, st>>>(K, Z, (const float*)sH, (const float*)sV,
                                                   grid->nx, grid->ny, (float*)C, scratch);
  else
    k_fraction_noalloc<double><<<g, block, 0, st>>>(K, Z, (const double*)sH, (const double*)sV,
                                                    grid->nx, grid->ny, (double*)C, scratch);
  k_area_noalloc<<<1, 256, 0, st>>>(scratch, nblocks, grid->dx * grid->dx, area,
                                    (long long*)marker_counts);
  e = cudaGetLastError();
  if (e != cudaSuccess) return fail_na(EBIT_ECUDA, "launch: %s", cudaGetErrorString(e));
  return EBIT_OK;
}
