// Host-side state shared by the launchers: the TMA tensor maps of input images
// (encoded once per pointer, shape and pitch), the multiprocessor count per
// device, the poll limit of the kernels' bounded waits, and the stream-ordered
// memory pool of the calls that need scratch.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <atomic>
#include <cstring>
#include <mutex>

#include "fbf_internal.h"

namespace fbf {
namespace {

PFN_cuTensorMapEncodeTiled_v12000 encoder() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static std::once_flag once;
  std::call_once(once, [] {
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
  });
  return fn;
}

struct MapEntry {
  int dev = -1;
  const void *ptr = nullptr;
  int Wd = 0, H = 0, bw = 0, bh = 0;
  size_t pitch = 0;
  bool ok = false;
  CUtensorMap map;
};
constexpr int kMapSlots = 64;
std::mutex g_map_mu;
MapEntry g_maps[kMapSlots];
int g_map_next = 0;

constexpr int kMaxDev = 64;
std::atomic<int> g_sms[kMaxDev];
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDev] = {};

// Default poll limit of the tensor-core kernels' bounded waits (about a second
// of polling on GB300), or the limit set by fbf_set_wait_limit.
constexpr unsigned int kDefaultPolls = 1u << 22;
std::atomic<long long> g_polls{-1};

}  // namespace

bool cached_box_map(const void *ptr, int Wd, int H, size_t pitch, int bw, int bh, CUtensorMap *out) {
  if ((reinterpret_cast<uintptr_t>(ptr) & 15) != 0 || (pitch & 15) != 0) return false;
  if (pitch >= (1ull << 40) || Wd <= 0 || H <= 0) return false;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return false;
  std::lock_guard<std::mutex> lock(g_map_mu);
  for (const MapEntry &e : g_maps)
    if (e.dev == dev && e.ptr == ptr && e.Wd == Wd && e.H == H && e.pitch == pitch && e.bw == bw && e.bh == bh) {
      if (e.ok) *out = e.map;
      return e.ok;
    }
  MapEntry &e = g_maps[g_map_next];
  g_map_next = (g_map_next + 1) % kMapSlots;
  e.dev = dev;
  e.ptr = ptr;
  e.Wd = Wd;
  e.H = H;
  e.pitch = pitch;
  e.bw = bw;
  e.bh = bh;
  e.ok = false;
  std::memset(&e.map, 0, sizeof(e.map));
  PFN_cuTensorMapEncodeTiled_v12000 enc = encoder();
  if (enc) {
    const cuuint64_t dims[2] = {(cuuint64_t)Wd, (cuuint64_t)H};
    const cuuint64_t strides[1] = {(cuuint64_t)pitch};
    const cuuint32_t box[2] = {(cuuint32_t)bw, (cuuint32_t)bh};
    const cuuint32_t estr[2] = {1, 1};
    e.ok = enc(&e.map, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(ptr), dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
               CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
  }
  if (e.ok) *out = e.map;
  return e.ok;
}

int sm_count(int dev) {
  if (dev < 0 || dev >= kMaxDev) return 0;
  int v = g_sms[dev].load(std::memory_order_relaxed);
  if (v <= 0) {
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    g_sms[dev].store(v, std::memory_order_relaxed);
  }
  return v;
}

// The library's own stream-ordered pool per device, created on first use,
// keeping the memory it has reserved (release threshold: unlimited) so that a
// call's scratch is re-used by the next call instead of being mapped again.
static cudaMemPool_t scratch_pool(int dev) {
  std::lock_guard<std::mutex> lock(g_pool_mu);
  if (!g_pools[dev]) {
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.handleTypes = cudaMemHandleTypeNone;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = dev;
    cudaMemPool_t pool = nullptr;
    if (cudaMemPoolCreate(&pool, &props) != cudaSuccess) return nullptr;
    unsigned long long keep = ~0ull;
    cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep);
    g_pools[dev] = pool;
  }
  return g_pools[dev];
}

fbf_status scratch_alloc(void **p, size_t bytes, cudaStream_t s) {
  *p = nullptr;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return FBF_ERR_CUDA;
  cudaMemPool_t pool = scratch_pool(dev);
  if (!pool) return FBF_ERR_CUDA;
  return cudaMallocFromPoolAsync(p, bytes, pool, s) == cudaSuccess ? FBF_OK : FBF_ERR_CUDA;
}

fbf_status scratch_free(void *p, cudaStream_t s) {
  if (!p) return FBF_OK;
  return cudaFreeAsync(p, s) == cudaSuccess ? FBF_OK : FBF_ERR_CUDA;
}

unsigned int wait_polls() {
  const long long p = g_polls.load(std::memory_order_relaxed);
  return p < 0 ? kDefaultPolls : (unsigned int)p;
}

}  // namespace fbf

extern "C" fbf_status fbf_set_wait_limit(long long polls) {
  if (polls > 0xFFFFFFFFll) return FBF_ERR_RANGE;
  fbf::g_polls.store(polls < 0 ? -1 : polls, std::memory_order_relaxed);
  return FBF_OK;
}
