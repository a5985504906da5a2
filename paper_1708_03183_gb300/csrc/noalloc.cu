// Hilbert seed ranking that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need the ranking: a host
// framework that owns every device allocation through its own pool, or code running where a
// cudaMalloc would synchronise the device or is not permitted.  For them slt_seed_rank_noalloc
// ranks caller-provided points with caller-provided output and keeps its scratch (sort keys,
// values, their double buffers, radix histograms and the bounding box) in one file-scope device
// array of fixed size, which every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>
#include <stdint.h>

#include <mutex>

#include "internal.h"

namespace {

constexpr int64_t kMaxPoints = int64_t(1) << 20;  // 1,048,576 points
constexpr int64_t kRsTile = 2048;                  // items per radix block (sort.cu)
constexpr int64_t kMaxBlocks = (kMaxPoints + kRsTile - 1) / kRsTile;
// layout (bytes): box 4 x u64 | keys | vals | tkeys | tvals (n u32 each) | hist | offs (256 blocks + 1)
constexpr int64_t kBoxBytes = 256;
constexpr int64_t kVecBytes = kMaxPoints * 4;
constexpr int64_t kHistInts = 256 * kMaxBlocks + 1;
constexpr int64_t kScratchBytes = kBoxBytes + 4 * kVecBytes + 2 * ((kHistInts * 4 + 255) / 256 * 256);

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_addr[kMaxDevices] = {};

// Device address of g_scratch on the current device.  A call outside stream capture looks it
// up afresh (a cudaDeviceReset reloads the module, and the array may then sit elsewhere); a call
// on a capturing stream uses the address found by the last earlier call on that device.
unsigned char* scratch_address(cudaStream_t s) {
  int dev = 0;
  SLT_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) slt::fail(SLT_ERR_UNSUPPORTED, "device index beyond 63");
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
    (void)cudaGetLastError();
    cs = cudaStreamCaptureStatusActive;  // unknown: keep the address already found
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (cs == cudaStreamCaptureStatusNone || !g_addr[dev]) {
    void* p = nullptr;
    SLT_CUDA(cudaGetSymbolAddress(&p, g_scratch));
    g_addr[dev] = static_cast<unsigned char*>(p);
  }
  return g_addr[dev];
}

}  // namespace

extern "C" int slt_seed_rank_noalloc(const double* d_xy, int64_t n, int32_t* d_rank, void* stream) {
  try {
    if (n < 0) slt::fail(SLT_ERR_ARG, "n must be >= 0");
    if (n > kMaxPoints)
      slt::fail(SLT_ERR_ARG, "slt_seed_rank_noalloc ranks at most 1048576 points (fixed scratch); use slt_inspect");
    if (n > 0 && (!d_xy || !d_rank)) slt::fail(SLT_ERR_ARG, "null argument");
    if (n == 0) return SLT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char* base = scratch_address(s);
    auto* box = reinterpret_cast<unsigned long long*>(base);
    auto* keys = reinterpret_cast<uint32_t*>(base + kBoxBytes);
    auto* vals = keys + kMaxPoints;
    auto* tkeys = vals + kMaxPoints;
    auto* tvals = tkeys + kMaxPoints;
    auto* hist = reinterpret_cast<int32_t*>(base + kBoxBytes + 4 * kVecBytes);
    auto* offs = hist + (kHistInts * 4 + 255) / 256 * 256 / 4;
    slt::launch_bbox_init(box, s);  // the previous call's box must not leak into this one
    slt::launch_bbox(d_xy, n, box, s);
    slt::launch_hilbert_keys(d_xy, n, box, keys, vals, s);
    slt::radix_sort_pairs_with(keys, vals, n, 32, tkeys, tvals, hist, offs, s);
    slt::launch_rank_from_order(vals, n, d_rank, s);
    SLT_CUDA(cudaGetLastError());
  } catch (const slt::Error& e) {
    slt::set_error(e.msg);
    return e.code;
  } catch (...) {
    slt::set_error("unexpected exception");
    return SLT_ERR_CUDA;
  }
  return SLT_OK;
}
