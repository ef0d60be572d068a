// Allocation-free variant of the system-observables reduction.
//
// md_observables_noalloc() computes U, K, T, the pressure tensor and the
// heat flux of caller-supplied per-particle arrays without allocating any
// device memory.  It is meant for host programs that cannot call cudaMalloc
// once they are running: engines that hand all device memory to their own
// fixed-size pool at start-up (so that memory use cannot grow behind their
// back), and programs that must not pay the device-wide synchronisation
// that cudaMalloc / cudaFree can trigger in the middle of a pipelined run.
//
// Its scratch (one row of partial sums per CTA plus the completion counter
// of the last-CTA reduction) lives in the file-scope array below, sized for
// kNoAllocBlocks CTAs.  Every GPU that loads the library holds it until the
// process exits.  Host code cannot use the array's name as a device
// address, so the first call on each device looks the address up with
// cudaGetSymbolAddress (that device current) and clears the counter on the
// caller's stream, ahead of its own launch; that first call should come
// before any stream capture.  All calls on a device
// share the one array: calls that overlap on the GPU race and must be
// ordered by the caller (one stream, or events).
#include <cstdint>
#include <mutex>

#include "common.cuh"

namespace {

constexpr int kNoAllocBlocks = 1024;  // CTAs of the grid-stride reduction
constexpr int kNoAllocThreads = 256;
constexpr int kObsRed = 11;           // K, U, V*sigma[6], V*q[3]
constexpr int kCounterSlot = kNoAllocBlocks * kObsRed;  // one double-sized word
constexpr int kScratchWords = kCounterSlot + 32;        // 256-byte tail for the counter
constexpr int kMaxDevices = 64;
constexpr int64_t kMaxAtoms = (int64_t(1) << 27) - 1;   // library-wide atom limit

static __device__ __align__(256) double g_noalloc_scratch[kScratchWords];

std::mutex g_setup_mutex;
double *g_scratch_ptr[kMaxDevices] = {};

// Deterministic reduction: per-thread FP64 sums, warp shuffles, one row per
// CTA in the scratch, and the last CTA to finish sums the rows in CTA order
// and writes [U, K, T, sigma xx yy zz xy xz yz, q x y z] to obs.
__global__ void __launch_bounds__(kNoAllocThreads)
    k_obs_noalloc(int64_t n, double volume, const double *__restrict__ v, const double *__restrict__ epot,
                  const double *__restrict__ W, const double *__restrict__ mass_of, double *obs,
                  double *scratch) {
  __shared__ double red[kNoAllocThreads / 32][kObsRed];
  __shared__ double tot[kObsRed];
  __shared__ int last;
  unsigned *counter = reinterpret_cast<unsigned *>(scratch + kCounterSlot);
  double acc[kObsRed];
#pragma unroll
  for (int q = 0; q < kObsRed; ++q) acc[q] = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
       i += (int64_t)gridDim.x * blockDim.x) {
    const double m = mass_of[i];
    const double vx = v[i], vy = v[n + i], vz = v[2 * n + i];
    double w[6];
#pragma unroll
    for (int q = 0; q < 6; ++q) w[q] = W[q * n + i];
    const double ke = 0.5 * m * (vx * vx + vy * vy + vz * vz);
    const double E = ke + epot[i];
    acc[0] += ke;
    acc[1] += epot[i];
    acc[2] += m * vx * vx + w[0];
    acc[3] += m * vy * vy + w[1];
    acc[4] += m * vz * vz + w[2];
    acc[5] += m * vx * vy + w[3];
    acc[6] += m * vx * vz + w[4];
    acc[7] += m * vy * vz + w[5];
    acc[8] += E * vx + w[0] * vx + w[3] * vy + w[4] * vz;
    acc[9] += E * vy + w[3] * vx + w[1] * vy + w[5] * vz;
    acc[10] += E * vz + w[4] * vx + w[5] * vy + w[2] * vz;
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int q = 0; q < kObsRed; ++q) {
    const double s = otf::warp_sum(acc[q]);
    if (lane == 0) red[warp][q] = s;
  }
  __syncthreads();
  if (threadIdx.x < kObsRed) {
    double s = 0.0;
    for (int w = 0; w < kNoAllocThreads / 32; ++w) s += red[w][threadIdx.x];
    scratch[blockIdx.x * kObsRed + threadIdx.x] = s;
  }
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  __syncthreads();
  if (!last) return;
  __threadfence();
  for (int q = warp; q < kObsRed; q += kNoAllocThreads / 32) {
    double s = 0.0;
    for (int b = lane; b < (int)gridDim.x; b += 32) s += __ldcg(scratch + b * kObsRed + q);
    s = otf::warp_sum(s);
    if (lane == 0) tot[q] = s;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    obs[0] = tot[1];
    obs[1] = tot[0];
    obs[2] = n > 1 ? 2.0 * tot[0] / (3.0 * (double)n - 3.0) : 0.0;
    for (int a = 0; a < 6; ++a) obs[3 + a] = tot[2 + a] / volume;
    for (int a = 0; a < 3; ++a) obs[9 + a] = tot[8 + a] / volume;
    *counter = 0u;  // ready for the next call
  }
}

// Device address of the scratch on the current device; the first call on a
// device looks it up and zeroes the completion counter on `stream` (the
// stream the caller's launch follows on, so the two are ordered whatever
// kind of stream it is).
int scratch_for_current_device(cudaStream_t stream, double **out) {
  int dev = 0;
  OTF_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    otf::set_error("md_observables_noalloc: device %d beyond the %d supported", dev, kMaxDevices);
    return MD_EINVAL;
  }
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_ptr[dev]) {
    double *p = nullptr;
    OTF_CUDA(cudaGetSymbolAddress(reinterpret_cast<void **>(&p), g_noalloc_scratch));
    OTF_CUDA(cudaMemsetAsync(p + kCounterSlot, 0, sizeof(double), stream));
    g_scratch_ptr[dev] = p;
  }
  *out = g_scratch_ptr[dev];
  return MD_OK;
}

}  // namespace

extern "C" {

int md_observables_noalloc(int64_t n, double volume, const double *v, const double *epot, const double *W,
                           const double *mass_of, double *obs, void *cuda_stream) {
  otf::clear_error();
  if (n < 2 || n > kMaxAtoms) {
    otf::set_error("md_observables_noalloc: n = %lld outside [2, %lld]", (long long)n, (long long)kMaxAtoms);
    return MD_EINVAL;
  }
  if (!(volume > 0.0) || !v || !epot || !W || !mass_of || !obs) {
    otf::set_error("md_observables_noalloc: volume must be positive and every array non-null");
    return MD_EINVAL;
  }
  double *scratch = nullptr;
  int rc = scratch_for_current_device((cudaStream_t)cuda_stream, &scratch);
  if (rc) return rc;
  const int64_t want = (n + kNoAllocThreads - 1) / kNoAllocThreads;
  const int blocks = (int)(want < kNoAllocBlocks ? want : kNoAllocBlocks);
  k_obs_noalloc<<<blocks, kNoAllocThreads, 0, (cudaStream_t)cuda_stream>>>(n, volume, v, epot, W, mass_of, obs,
                                                                          scratch);
  OTF_LAUNCH_CHECK();
  return MD_OK;
}

}  // extern "C"
