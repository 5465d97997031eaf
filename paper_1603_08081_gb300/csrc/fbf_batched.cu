// Batched filtering of many uneven images, each with its own spatial and range
// parameters (its own W, K and coefficients), in one persistent launch that is
// captured in a CUDA graph.
//
// fbf_plan_create fits every image's coefficients (Algorithm 2, host FP64),
// uploads a table of per-image parameters, and lists every (image, tile) work
// item sorted by estimated cost (K x taps per tile, largest first).  The
// persistent kernel runs one CTA per SM; each CTA repeatedly takes the next
// item from a global counter (one atomicAdd per tile, no waiting), copies that
// image's taps and coefficients to shared memory, and runs the fused FP32 tile
// body (32 x 192 outputs, W <= 32, tap count at run time).  The graph holds a
// memset of the counter followed by the kernel, so fbf_filter_batched is one
// cudaGraphLaunch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fbf_fp32_kernel.cuh"
#include "fbf_internal.h"

namespace fbf {
namespace {

constexpr int kBBX = 32, kBBY = 192, kBNT = 256, kBNBUF = 1, kBWCAP = 32;

struct ImageParams {
  const unsigned char *in;
  float *out;
  size_t in_pitch, out_pitch;
  int H, Wd, W, K, twoT, tiles_x;
  float T;
  int pad_;
  u64 w2[TAPS_MAX];
  float d[FBF_KMAX];
};

struct BatchArgs {
  const ImageParams *imgs;
  const int2 *items;  // (image, tile index within the image)
  int nitems;
  int border;
  int *counter;
};

__global__ void __launch_bounds__(kBNT, 1) fbf_batched_kernel(const __grid_constant__ BatchArgs b) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Layout Lmax = make_layout(kBBX, kBBY, kBWCAP, kBNBUF, kBWCAP);
  u64 *w2s = reinterpret_cast<u64 *>(smem + Lmax.bytes);
  float *ds = reinterpret_cast<float *>(w2s + TAPS_MAX);
  int *item_s = reinterpret_cast<int *>(ds + FBF_KMAX);
  for (;;) {
    if (threadIdx.x == 0) *item_s = atomicAdd(b.counter, 1);
    __syncthreads();
    const int it = *item_s;
    if (it >= b.nitems) break;
    const int2 w = b.items[it];
    const ImageParams &P = b.imgs[w.x];
    const int W = P.W, K = P.K;
    for (int i = threadIdx.x; i < 2 * W + 1; i += kBNT) w2s[i] = P.w2[i];
    for (int i = threadIdx.x; i < K; i += kBNT) ds[i] = P.d[i];
    __syncthreads();
    const K1View v{P.in, P.in_pitch, P.out, P.out_pitch, P.H, P.Wd, W, K, P.twoT, b.border, P.T, w2s, ds};
    const int ty = w.y / P.tiles_x, tx = w.y - ty * P.tiles_x;
    k1_tile<kBBX, kBBY, kBNT, kBNBUF, kBWCAP, 0>(v, ty * kBBY, tx * kBBX, smem);
    __syncthreads();  // the next item overwrites the taps, coefficients and item slot
  }
}

size_t batched_smem_bytes() {
  const Layout Lmax = make_layout(kBBX, kBBY, kBWCAP, kBNBUF, kBWCAP);
  return Lmax.bytes + TAPS_MAX * sizeof(u64) + FBF_KMAX * sizeof(float) + 16;
}

}  // namespace
}  // namespace fbf

using namespace fbf;

struct fbf_plan {
  int device = 0;
  int n_images = 0, n_items = 0;
  ImageParams *d_imgs = nullptr;
  int2 *d_items = nullptr;
  int *d_counter = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

static void plan_free(fbf_plan *p) {
  if (!p) return;
  if (p->exec) cudaGraphExecDestroy(p->exec);
  if (p->graph) cudaGraphDestroy(p->graph);
  if (p->d_imgs) cudaFree(p->d_imgs);
  if (p->d_items) cudaFree(p->d_items);
  if (p->d_counter) cudaFree(p->d_counter);
  delete p;
}

extern "C" fbf_status fbf_plan_create(const fbf_image_desc *descs, int n, fbf_form form, fbf_border border,
                                      fbf_plan **out) {
  if (!out) return FBF_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (n < 0 || (n > 0 && !descs)) return FBF_ERR_INVALID_ARGUMENT;
  if (border != FBF_BORDER_REFLECT && border != FBF_BORDER_TRUNCATE) return FBF_ERR_INVALID_ARGUMENT;
  if (form != FBF_FORM_AUTO && form != FBF_FORM_FP32) {
    if (form == FBF_FORM_TC_FP16 || form == FBF_FORM_TC_BF16 || form == FBF_FORM_TC_FP16_SINGLE)
      return FBF_ERR_UNSUPPORTED;
    return FBF_ERR_INVALID_ARGUMENT;
  }
  std::vector<ImageParams> imgs(n);
  struct Item {
    int img, tile;
    double cost;
  };
  std::vector<Item> items;
  for (int i = 0; i < n; ++i) {
    const fbf_image_desc &d = descs[i];
    fbf_coeffs c;
    fbf_status st = fbf_fit_coeffs(d.range, d.sigma_r, d.T, d.eps, d.K_fixed, d.levels, &c);
    if (st != FBF_OK) return st;
    fbf_params prm;
    prm.spatial = d.spatial;
    prm.sigma_s = d.sigma_s;
    prm.W = d.W;
    prm.border = border;
    prm.form = FBF_FORM_FP32;
    prm.coeffs = &c;
    FilterArgs a;
    st = pack_filter_args(&prm, d.d_in, FBF_U8, d.H, d.Wd, d.in_pitch, d.d_out, d.out_pitch, &a);
    if (st != FBF_OK) return st;
    ImageParams &P = imgs[i];
    std::memset(&P, 0, sizeof(P));
    P.in = static_cast<const unsigned char *>(d.d_in);
    P.out = d.d_out;
    P.in_pitch = d.in_pitch;
    P.out_pitch = d.out_pitch;
    P.H = d.H;
    P.Wd = d.Wd;
    P.W = a.W;
    P.K = a.K;
    P.twoT = a.twoT;
    P.T = a.T;
    P.tiles_x = (d.Wd + kBBX - 1) / kBBX;
    std::memcpy(P.w2, a.w2, sizeof(P.w2));
    std::memcpy(P.d, a.d, sizeof(P.d));
    const int ntiles = d.H > 0 && d.Wd > 0 ? P.tiles_x * ((d.H + kBBY - 1) / kBBY) : 0;
    const double cost = (double)a.K * (2 * a.W + 1) + 8.0;  // per tile: harmonics x taps (+ staging)
    for (int t = 0; t < ntiles; ++t) items.push_back({i, t, cost});
  }
  std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });

  fbf_plan *p = new fbf_plan();
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    plan_free(p);
    return FBF_ERR_CUDA;
  }
  p->n_images = n;
  p->n_items = (int)items.size();
  std::vector<int2> h_items(items.size());
  for (size_t k = 0; k < items.size(); ++k) h_items[k] = make_int2(items[k].img, items[k].tile);
  bool okc = cudaMalloc(&p->d_imgs, sizeof(ImageParams) * std::max(n, 1)) == cudaSuccess &&
             cudaMalloc(&p->d_items, sizeof(int2) * std::max<size_t>(items.size(), 1)) == cudaSuccess &&
             cudaMalloc(&p->d_counter, sizeof(int)) == cudaSuccess;
  if (okc && n > 0)
    okc = cudaMemcpy(p->d_imgs, imgs.data(), sizeof(ImageParams) * n, cudaMemcpyHostToDevice) == cudaSuccess;
  if (okc && !items.empty())
    okc = cudaMemcpy(p->d_items, h_items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice) ==
          cudaSuccess;
  if (!okc) {
    plan_free(p);
    return FBF_ERR_CUDA;
  }

  // Capture: counter reset + one persistent launch (one CTA per SM).
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, p->device);
  const int grid = std::max(1, std::min(p->n_items, sms));
  const size_t smem = batched_smem_bytes();
  if (cudaFuncSetAttribute(fbf_batched_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
      cudaSuccess) {
    plan_free(p);
    return FBF_ERR_CUDA;
  }
  BatchArgs args{p->d_imgs, p->d_items, p->n_items, (int)border, p->d_counter};
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    plan_free(p);
    return FBF_ERR_CUDA;
  }
  bool okg = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
  if (okg) {
    cudaMemsetAsync(p->d_counter, 0, sizeof(int), cs);
    if (p->n_items > 0) fbf_batched_kernel<<<grid, kBNT, smem, cs>>>(args);
    okg = cudaStreamEndCapture(cs, &p->graph) == cudaSuccess && p->graph;
  }
  if (okg) okg = cudaGraphInstantiate(&p->exec, p->graph, 0) == cudaSuccess;
  cudaStreamDestroy(cs);
  if (!okg) {
    plan_free(p);
    return FBF_ERR_CUDA;
  }
  *out = p;
  return FBF_OK;
}

extern "C" fbf_status fbf_filter_batched(fbf_plan *plan, cudaStream_t stream) {
  if (!plan || !plan->exec) return FBF_ERR_INVALID_ARGUMENT;
  return cuda_status(cudaGraphLaunch(plan->exec, stream));
}

extern "C" fbf_status fbf_plan_destroy(fbf_plan *plan) {
  if (!plan) return FBF_ERR_INVALID_ARGUMENT;
  plan_free(plan);
  return FBF_OK;
}

extern "C" fbf_status fbf_plan_size(const fbf_plan *plan, int *n_images, int *n_items) {
  if (!plan) return FBF_ERR_INVALID_ARGUMENT;
  if (n_images) *n_images = plan->n_images;
  if (n_items) *n_items = plan->n_items;
  return FBF_OK;
}
