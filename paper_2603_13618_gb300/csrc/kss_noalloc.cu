// kss_noalloc.cu -- the allocation-free entry point kss_step_f32_noalloc (see
// include/kss.h).
//
// Some callers cannot allocate device memory: a host that hands the library
// buffers it manages itself (a memory pool, a simulation framework with its own
// allocator, memory registered for another device API), or code that must not
// allocate at all once it is running.  They still need the fused step, whose
// kernel writes per-CTA partial sums and a CTA completion counter to global
// scratch memory.  This entry point keeps that scratch in a fixed-size array
// with static storage on the device instead of allocating it, so the call itself
// never calls cudaMalloc, cudaFree or any allocating routine; the caller supplies
// every input and output buffer.
#include <cuda_runtime.h>

#include <mutex>

#include "../../include/kss.h"
#include "launch.h"

namespace {

// Scratch of the fused step: the CTA completion counter (first 256 bytes), then
// 3 doubles of partial sums and 4 uint32 of partial counts per CTA.
constexpr size_t kCounterBytes = 256;
constexpr size_t kScratchBytes =
    kCounterBytes + size_t(KSS_NOALLOC_MAX_BLOCKS) * (3 * sizeof(double) + 4 * sizeof(uint32_t));

// Every GPU that loads this library holds this array until the process exits.
// Every call shares it and it keeps the last call's contents.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mutex;
void* g_scratch_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device (host code cannot use the
// symbol itself: on the host it names a stand-in, not device memory).  Looked up
// once per device, with that device current.
cudaError_t scratch_address(int dev, void** out) {
  std::lock_guard<std::mutex> lock(g_mutex);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return e;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return cudaSuccess;
}

bool std_sensor(int s) { return s == KSS_S_KN || s == KSS_S_KL || s == KSS_S_NEQ; }

float round_down_f32(double t) {
  float r = static_cast<float>(t);
  if (static_cast<double>(r) > t) r = nextafterf(r, -__builtin_huge_valf());
  return r;
}

}  // namespace

extern "C" int kss_step_f32_noalloc(const float* f_in, float* f_out, int32_t nx, int32_t ny,
                                    int32_t pitch, double tau, int32_t refine_sensor,
                                    double refine_threshold, int32_t switch_sensor,
                                    double switch_threshold, int32_t tile, int32_t record_sensor,
                                    float* sensor_out, uint8_t* flags, int32_t* tile_counts,
                                    double* sums, unsigned long long* counts, void* stream) {
  if (!f_in || !f_out || !flags || !tile_counts || !sums || !counts) return KSS_ERR_ARG;
  if (nx < 1 || ny < 1 || pitch < nx || pitch % 32 != 0) return KSS_ERR_ARG;
  if ((long long)pitch * ny > 0x7fffffffLL) return KSS_ERR_ARG;
  if (!(tau > 0.5)) return KSS_ERR_ARG;
  if (tile != 8 && tile != 16 && tile != 32 && tile != 64) return KSS_ERR_ARG;
  if (!std_sensor(refine_sensor) || !std_sensor(switch_sensor)) return KSS_ERR_ARG;
  if (sensor_out && !std_sensor(record_sensor)) return KSS_ERR_ARG;
  if (((uintptr_t)f_in | (uintptr_t)f_out | (uintptr_t)sensor_out) % 16 != 0) return KSS_ERR_ARG;
  if ((uintptr_t)flags % 4 != 0) return KSS_ERR_ARG;
  // the pull step reads neighbouring rows of f_in while other CTAs write f_out, so the
  // two population ranges must not overlap (an in-place step would read new values)
  {
    const uintptr_t bytes = uintptr_t(9) * uintptr_t(pitch) * uintptr_t(ny) * sizeof(float);
    const uintptr_t a = reinterpret_cast<uintptr_t>(f_in), b = reinterpret_cast<uintptr_t>(f_out);
    if (a < b + bytes && b < a + bytes) return KSS_ERR_ARG;
  }

  const dim3 grid = kss::step_grid<float>(nx, ny, tile);
  const long long nblocks = (long long)grid.x * grid.y;
  if (nblocks > KSS_NOALLOC_MAX_BLOCKS) return KSS_ERR_NOALLOC_CAPACITY;

  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return KSS_ERR_CUDA;
  void* base = nullptr;
  if (scratch_address(dev, &base) != cudaSuccess) return KSS_ERR_CUDA;
  unsigned char* scratch = static_cast<unsigned char*>(base);
  cudaStream_t s = static_cast<cudaStream_t>(stream);

  kss::StepParams<float> p{};
  p.src = f_in;
  p.dst = f_out;
  p.rec = sensor_out;
  p.flags = flags;
  p.tiles = tile_counts;
  p.done = reinterpret_cast<uint32_t*>(scratch);
  p.part_sum = reinterpret_cast<double*>(scratch + kCounterBytes);
  p.part_cnt = reinterpret_cast<uint32_t*>(scratch + kCounterBytes +
                                           size_t(KSS_NOALLOC_MAX_BLOCKS) * 3 * sizeof(double));
  p.stat_sums = sums;
  p.stat_counts = counts;
  p.plane = (long long)pitch * ny;
  p.pitch = pitch;
  p.nx = nx;
  p.ny = ny;
  p.tile = tile;
  p.bands = kss::step_bands(tile);
  p.ntx = (nx + tile - 1) / tile;
  p.nty = (ny + tile - 1) / tile;
  p.omega = float(1.0 / tau);
  p.tau = float(tau);
  p.thr_r = round_down_f32(refine_threshold);
  p.switch_on = switch_threshold >= 0.0;
  p.thr_s = p.switch_on ? round_down_f32(switch_threshold) : 0.f;
  p.refine_s = refine_sensor;
  p.switch_s = switch_sensor;
  for (int k = 0; k < kss::S_COUNT; ++k) p.rec_slot[k] = -1;
  if (sensor_out) p.rec_slot[record_sensor] = 0;

  // the completion counter must start at zero (the last CTA of a finished call
  // resets it, but a call must not depend on the previous one)
  if (cudaMemsetAsync(p.done, 0, sizeof(uint32_t), s) != cudaSuccess) return KSS_ERR_CUDA;
  kss::step_kernel<float, kss::MODE_STD, true, true><<<grid, kss::kThreads, 0, s>>>(p);
  return cudaGetLastError() == cudaSuccess ? KSS_OK : KSS_ERR_CUDA;
}
