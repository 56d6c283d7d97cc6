// godec_mul_ZB_noalloc: the streaming product Y = Z B with its scratch in a
// fixed device array instead of memory allocated per call.
//
// Some callers cannot allocate device memory while they run: a host
// application that reserves all GPU memory at start-up and forbids plugins
// to allocate afterwards, or a latency-critical loop where an allocation may
// synchronise the device or fragment a pool.  For them this entry point keeps
// the padded copy of B, the split-K partial products and the padded result in
// one file-scope array of kNoAllocScratchBytes bytes.  The array belongs to the
// library's device code: a GPU holds it from the moment that code is loaded there
// (under CUDA's default lazy loading, at the first use of the library's kernels or
// symbols on that device) until the process exits.
#include <mutex>

#include "godec_internal.cuh"

namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;   // 32 MiB per device
static __device__ __align__(256) unsigned char g_mul_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices];
std::mutex g_scratch_mu;

size_t align256(size_t b) { return (b + 255) & ~size_t(255); }

// Device address of the array on the current device (host code cannot use the symbol
// itself: it names a host-side stand-in).  Outside stream capture the address is looked
// up again on every call, so a new primary context (after cudaDeviceReset) is picked
// up; while `st` is capturing, the address cached by an earlier call on this device is
// used, and a first call under capture is refused.
godec_status scratch_address(cudaStream_t st, void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) {
    godec::set_static_error("godec_mul_ZB_noalloc: cudaGetDevice: %s", cudaGetErrorString(e));
    return GODEC_ERR_CUDA;
  }
  if (dev < 0 || dev >= kMaxDevices) {
    godec::set_static_error("godec_mul_ZB_noalloc: device ordinal %d above %d", dev, kMaxDevices - 1);
    return GODEC_ERR_UNSUPPORTED;
  }
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  e = cudaStreamIsCapturing(st, &cap);
  if (e != cudaSuccess) {
    godec::set_static_error("godec_mul_ZB_noalloc: cudaStreamIsCapturing: %s", cudaGetErrorString(e));
    return GODEC_ERR_CUDA;
  }
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (cap != cudaStreamCaptureStatusNone && !g_scratch_addr[dev]) {
    godec::set_static_error("godec_mul_ZB_noalloc: the first call on device %d must come before any stream "
                            "capture", dev);
    return GODEC_ERR_STATE;
  }
  if (cap == cudaStreamCaptureStatusNone) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_mul_scratch);
    if (e != cudaSuccess || !p) {
      godec::set_static_error("godec_mul_ZB_noalloc: cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      return GODEC_ERR_CUDA;
    }
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return GODEC_OK;
}

}  // namespace

extern "C" godec_status godec_mul_ZB_noalloc(const float* Z, int64_t m, int64_t n, int64_t ldz,
                                             const float* B, int32_t r, float* Y, void* stream) {
  using namespace godec;
  if (!Z || !B || !Y || m < 1 || n < 1 || ldz < n || (ldz * 4) % 16 || r < 1 || r > GODEC_MAX_RANK ||
      (reinterpret_cast<uintptr_t>(Z) & 15)) {
    set_static_error("godec_mul_ZB_noalloc: invalid argument");
    return GODEC_ERR_ARG;
  }
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  const int RP = (r + 7) / 8 * 8;
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    set_static_error("godec_mul_ZB_noalloc: no CUDA device");
    return GODEC_ERR_CUDA;
  }
  int splits;
  int64_t kchunk;
  prod_geometry(m, n, nsm, &splits, &kchunk);
  const int64_t tiles = prod_tiles(m);
  const size_t bytes_b = align256((size_t)n * RP * sizeof(float));
  const size_t bytes_p = align256((size_t)splits * m * RP * sizeof(float));
  const size_t bytes_y = align256((size_t)m * RP * sizeof(float));
  const size_t bytes_c = align256((size_t)tiles * sizeof(unsigned));
  if (bytes_b + bytes_p + bytes_y + bytes_c > kNoAllocScratchBytes) {
    set_static_error("godec_mul_ZB_noalloc: m=%lld n=%lld r=%d needs %zu bytes of scratch, above the "
                     "fixed %zu", (long long)m, (long long)n, r, bytes_b + bytes_p + bytes_y + bytes_c,
                     kNoAllocScratchBytes);
    return GODEC_ERR_UNSUPPORTED;
  }
  if (prepare_stream_kernels() != cudaSuccess) {
    set_static_error("godec_mul_ZB_noalloc: kernel set-up failed");
    return GODEC_ERR_CUDA;
  }
  void* base = nullptr;
  godec_status s = scratch_address(st, &base);
  if (s) return s;
  char* p = reinterpret_cast<char*>(base);
  float* Bp = reinterpret_cast<float*>(p);
  float* part = reinterpret_cast<float*>(p + bytes_b);
  float* Yp = reinterpret_cast<float*>(p + bytes_b + bytes_p);
  unsigned* cnt = reinterpret_cast<unsigned*>(p + bytes_b + bytes_p + bytes_y);
  // Every scratch element read below is written first in the same call (all K x RP
  // of Bp, all splits x m x RP partials, all m x RP of Yp), except the per-tile
  // arrival counters, which must start at zero: clear them on every call.
  cudaError_t e = cudaMemsetAsync(cnt, 0, (size_t)tiles * sizeof(unsigned), st);
  if (e != cudaSuccess) {
    set_static_error("godec_mul_ZB_noalloc: clearing the tile counters: %s", cudaGetErrorString(e));
    return GODEC_ERR_CUDA;
  }
  launch_pad_copy(B, n, r, r, Bp, RP, st);
  ProdArgs pa{};
  pa.Z = Z;
  pa.rows = m;
  pa.K = n;
  pa.ld = ldz;
  pa.B = Bp;
  pa.part = part;
  pa.splits = splits;
  pa.kchunk = kchunk;
  pa.counters = cnt;
  pa.out = Yp;
  pa.RP = RP;
  launch_prod(pa, st);
  launch_unpad_copy(Yp, m, RP, Y, r, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) {
    set_static_error("godec_mul_ZB_noalloc: %s", cudaGetErrorString(e));
    return GODEC_ERR_CUDA;
  }
  return GODEC_OK;
}
