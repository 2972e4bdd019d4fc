// Allocation-free field-energy reduction (declared in include/pic.h as
// pic_field_energy_noalloc).
//
// Some callers cannot call cudaMalloc: processes whose device memory is
// planned up front by another allocator (a serving loop that admits work
// against a fixed memory budget, or a host framework whose caching allocator
// owns the device), where a stray allocation can fail or fragment the plan.  This entry point lets them reduce field
// energy with no allocation at all: its scratch (one FP64 partial sum per
// block) is a file-scope __device__ array that every GPU loading this
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cstdint>
#include <mutex>
#include <string>

#include "../../include/pic.h"

namespace {
constexpr int kMaxBlocks = 65536;  // scratch: 512 KiB of doubles
}

// One partial sum per block.  Every call writes all partials it later reads,
// so nothing needs clearing between calls; two calls that overlap on the GPU
// share this array and race.  In host code this name is only a stand-in for
// the device array: its device address comes from cudaGetSymbolAddress.
static __device__ __align__(256) double g_partials[kMaxBlocks];

namespace pg_internal {
void set_last_error(const std::string &msg);
}

namespace {

constexpr int kThreads = 256;
constexpr int kItems = 8;                           // field points per thread
constexpr long long kPointsPerBlock = (long long)kThreads * kItems;
constexpr double kEps0 = 8.8541878128e-12;
constexpr double kMu0 = 1.0 / (kEps0 * 299792458.0 * 299792458.0);

// Device addresses of g_partials, one per device, looked up on the first
// call made with that device current.
std::mutex g_mu;
void *g_addr[64];

template <class R>
__global__ void __launch_bounds__(kThreads) k_energy_partials(const R *ex, const R *ey, const R *ez,
                                                              const R *bx, const R *by, const R *bz,
                                                              long long n, double *partials) {
  const long long base = (long long)blockIdx.x * kPointsPerBlock + threadIdx.x;
  double e2 = 0.0, b2 = 0.0;
#pragma unroll
  for (int q = 0; q < kItems; ++q) {
    const long long o = base + (long long)q * kThreads;
    if (o < n) {
      const double a = ex[o], b = ey[o], c = ez[o];
      const double u = bx[o], v = by[o], w = bz[o];
      e2 += a * a + b * b + c * c;
      b2 += u * u + v * v + w * w;
    }
  }
  double s = 0.5 * kEps0 * e2 + 0.5 * b2 / kMu0;
#pragma unroll
  for (int d = 16; d > 0; d >>= 1) s += __shfl_xor_sync(0xffffffffu, s, d);
  __shared__ double warp_sum[kThreads / 32];
  if ((threadIdx.x & 31) == 0) warp_sum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int q = 0; q < kThreads / 32; ++q) t += warp_sum[q];
    partials[blockIdx.x] = t;
  }
}

// Sums the partials in a fixed order (deterministic) and scales by the cell
// volume.
__global__ void __launch_bounds__(kThreads) k_energy_final(const double *partials, int nb,
                                                           double volume, double *out) {
  double s = 0.0;
  for (int b = threadIdx.x; b < nb; b += kThreads) s += partials[b];
  __shared__ double part[kThreads];
  part[threadIdx.x] = s;
  __syncthreads();
  for (int w = kThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = part[0] * volume;
}

int fail(int code, const std::string &m) {
  pg_internal::set_last_error(m);  // readable through pic_last_error()
  return code;
}

// Address of g_partials on the current device (first call per device looks
// it up; that call must not be made during a stream capture).
int scratch_address(double **out) {
  int dev = -1;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return fail(PIC_ECUDA, std::string("cudaGetDevice: ") + cudaGetErrorString(e));
  if (dev < 0 || dev >= 64) return fail(PIC_EINVAL, "device ordinal above 63");
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_addr[dev]) {
    void *p = nullptr;
    e = cudaGetSymbolAddress(&p, g_partials);
    if (e != cudaSuccess || !p)
      return fail(PIC_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
    g_addr[dev] = p;
  }
  *out = (double *)g_addr[dev];
  return PIC_OK;
}

}  // namespace

extern "C" {

int pic_field_energy_noalloc(int precision, const void *Ex, const void *Ey, const void *Ez,
                             const void *Bx, const void *By, const void *Bz, long long n,
                             double cell_volume, double *d_out, void *stream) {
  if (precision != PIC_FP32 && precision != PIC_FP64)
    return fail(PIC_EINVAL, "precision must be PIC_FP32 or PIC_FP64");
  if (!Ex || !Ey || !Ez || !Bx || !By || !Bz || !d_out)
    return fail(PIC_EINVAL, "null device pointer");
  if (n < 0) return fail(PIC_EINVAL, "negative point count");
  const long long nb = (n + kPointsPerBlock - 1) / kPointsPerBlock;
  if (nb > kMaxBlocks)
    return fail(PIC_EINVAL, "n = " + std::to_string(n) + " exceeds the maximum of " +
                                std::to_string((long long)kMaxBlocks * kPointsPerBlock) +
                                " field points of the static scratch");
  double *partials = nullptr;
  int rc = scratch_address(&partials);
  if (rc) return rc;
  cudaStream_t s = (cudaStream_t)stream;
  if (nb > 0) {
    if (precision == PIC_FP32)
      k_energy_partials<float><<<(int)nb, kThreads, 0, s>>>(
          (const float *)Ex, (const float *)Ey, (const float *)Ez, (const float *)Bx,
          (const float *)By, (const float *)Bz, n, partials);
    else
      k_energy_partials<double><<<(int)nb, kThreads, 0, s>>>(
          (const double *)Ex, (const double *)Ey, (const double *)Ez, (const double *)Bx,
          (const double *)By, (const double *)Bz, n, partials);
  }
  k_energy_final<<<1, kThreads, 0, s>>>(partials, (int)nb, cell_volume, d_out);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(PIC_ECUDA, std::string("launch: ") + cudaGetErrorString(e));
  return PIC_OK;
}

}  // extern "C"
