// pm_shrink_static: the lightcone compaction of pm_shrink for callers that
// must not allocate device memory.  Its scratch (keep flags, per-block keep
// counts and offsets, the survivor count) lives in one file-scope device
// array sized for at most PM_SHRINK_STATIC_MAX_PARTICLES particles; every
// GPU that loads the library holds it (about 4.1 MB) until the process exits.
#include <cmath>
#include <mutex>
#include <string>

#include "pm_kernels.cuh"

namespace {

constexpr long long kMaxN = PM_SHRINK_STATIC_MAX_PARTICLES;
constexpr long long kChunk = pm::PART_CHUNK;  // particles per block of the compaction kernels
constexpr long long kMaxBlocks = (kMaxN + kChunk - 1) / kChunk;
constexpr size_t kFlagsOff = 0;                                   // u8 per particle
constexpr size_t kCountsOff = (size_t)kMaxN;                      // u32 per block
constexpr size_t kOffsetsOff = kCountsOff + 4 * kMaxBlocks;       // u64 per block
constexpr size_t kKeepOff = kOffsetsOff + 8 * kMaxBlocks;         // u64 survivor count
constexpr size_t kBytes = kKeepOff + 256;

static __device__ __align__(256) unsigned char g_shrink_scratch[kBytes];

// Device address of g_shrink_scratch per device.  In host code the symbol
// name is only a host-side stand-in, so the address is looked up once per
// device with that device current.
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_dev[kMaxDevices] = {};
std::mutex g_scratch_mu;
// the last failure's text, per calling thread: concurrent failing calls do
// not overwrite each other's message
thread_local std::string g_static_err;

pm_status static_fail(pm_status code, const std::string& msg) {
  g_static_err = msg;
  return code;
}

}  // namespace

extern "C" const char* pm_shrink_static_error(void) { return g_static_err.c_str(); }

extern "C" pm_status pm_shrink_static(const float* pos4_in, const float* mom4_in, int64_t n,
                                      int32_t n_mesh, double box_mpch, double omega_m,
                                      double omega_l, double buffer_cells, double a,
                                      float* pos4_keep, float* mom4_keep, float* pos4_leave,
                                      float* mom4_leave, int64_t* n_keep_out, void* stream) {
  if (n < 0 || n_mesh < 4 || !(box_mpch > 0) || !(omega_m > 0) || !(a > 0) || !n_keep_out ||
      !std::isfinite(box_mpch) || !std::isfinite(omega_m) || !std::isfinite(omega_l) ||
      !std::isfinite(buffer_cells) || !std::isfinite(a))
    return static_fail(PM_EINVAL, "pm_shrink_static: bad argument");
  if (n > kMaxN)
    return static_fail(PM_EINVAL,
                       "pm_shrink_static: n = " + std::to_string((long long)n) +
                           " exceeds the static scratch limit of " +
                           std::to_string(kMaxN) + " particles");
  if (n > 0 && (!pos4_in || !mom4_in || !pos4_keep || !mom4_keep || !pos4_leave || !mom4_leave))
    return static_fail(PM_EINVAL, "pm_shrink_static: NULL particle buffer");
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_fail(PM_ECUDA, cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return static_fail(PM_EINVAL, "device index too large");
  unsigned char* scratch = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_scratch_mu);
    if (!g_scratch_dev[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_shrink_scratch);
      if (e != cudaSuccess)
        return static_fail(PM_ECUDA, std::string("cudaGetSymbolAddress: ") +
                                         cudaGetErrorString(e));
      g_scratch_dev[dev] = (unsigned char*)p;
    }
    scratch = g_scratch_dev[dev];
  }
  if (n == 0) {
    *n_keep_out = 0;
    return PM_OK;
  }
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* flags = scratch + kFlagsOff;
  unsigned int* counts = (unsigned int*)(scratch + kCountsOff);
  unsigned long long* offs = (unsigned long long*)(scratch + kOffsetsOff);
  unsigned long long* nkeep = (unsigned long long*)(scratch + kKeepOff);
  const double R = pm::shrink_radius_cells(n_mesh, box_mpch, omega_m, omega_l, buffer_cells, a);
  float klo, khi;
  pm::shrink_keep_bounds(n_mesh, R, &klo, &khi);
  const int nblk = pm::gkd_blocks(n);
  // every flag, count, offset and the survivor count are written before they
  // are read, so nothing left over from an earlier call needs clearing
  pm::launch_flag(st, (const float4*)pos4_in, n, klo, khi, flags, counts,
                  pm::KeepBall{0, 0.0, 0.0});
  pm::launch_scan_blocks(st, counts, offs, nblk, nkeep);
  pm::launch_scatter(st, (const float4*)pos4_in, (const float4*)mom4_in, n, flags, offs,
                     (float4*)pos4_keep, (float4*)mom4_keep, (float4*)pos4_leave,
                     (float4*)mom4_leave, 0, (float)a);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(PM_ECUDA, cudaGetErrorString(e));
  unsigned long long h = 0;
  e = cudaMemcpyAsync(&h, nkeep, sizeof(h), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return static_fail(PM_ECUDA, cudaGetErrorString(e));
  *n_keep_out = (int64_t)h;
  return PM_OK;
}
