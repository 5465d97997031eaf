// Batched filtering of many uneven images, each with its own spatial and range
// parameters (its own W, K and coefficients), replayed as one CUDA graph.
//
// fbf_plan_create fits every image's coefficients (Algorithm 2, host FP64) and
// prepares the candidate schedules that apply to the plan's form, each
// captured in its own graph:
//
//   PERSISTENT       one launch, one CTA per SM; each CTA repeatedly takes
//                    the next (image, tile) item from a global counter (one
//                    atomicAdd per tile, no waiting), copies that image's taps
//                    and coefficients to shared memory and runs the fused
//                    FP32 tile body with run-time taps.  Items are sorted by
//                    estimated cost (K x taps per tile, largest first).  32 x
//                    192 tiles, any W <= 32 (a candidate only then);
//   PERSISTENT_WIDE  the same with 64 x 96 tiles (when every W <= 16);
//   PER_IMAGE_FP32   one launch per image of the single-image FP32 kernel
//                    (compile-time tap counts, running sums for box windows);
//   PER_IMAGE_FORM   one launch per image in the plan's form (AUTO: the
//                    per-image choice of fbf_filter; the tensor-core forms);
//   PERSISTENT_TC    one launch of the second tensor-core layout (single FP16
//                    form) over cost-sorted (image, tile) items of every
//                    image, CTA b taking items b, b + #SMs, ... (fbf_tc2_batched.cu).
//
// Autotuning: when more than one candidate applies (forms AUTO and FP32), the
// plan replays every candidate's graph on its own images (writing the
// outputs), times it with CUDA events and keeps the fastest; the others are
// released.  fbf_plan_schedule reports the choice and its time.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "fbf_fp32_kernel.cuh"
#include "fbf_internal.h"

namespace fbf {
namespace {

constexpr int kBNT = 256;

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

template <int BX, int BY, int NBUF, int WCAP>
__global__ void __launch_bounds__(kBNT, 1) fbf_batched_kernel(const __grid_constant__ BatchArgs b) {
  extern __shared__ __align__(128) unsigned char smem[];
  const Layout Lmax = make_layout(BX, BY, WCAP, NBUF, WCAP);
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
    k1_tile<BX, BY, kBNT, NBUF, WCAP, 0>(v, ty * BY, tx * BX, smem);
    __syncthreads();  // the next item overwrites the taps, coefficients and item slot
  }
}

template <int BX, int BY, int NBUF, int WCAP>
size_t batched_smem_bytes() {
  const Layout Lmax = make_layout(BX, BY, WCAP, NBUF, WCAP);
  return Lmax.bytes + TAPS_MAX * sizeof(u64) + FBF_KMAX * sizeof(float) + 16;
}

// Device tables of one persistent schedule.
struct Persistent {
  ImageParams *d_imgs = nullptr;
  int2 *d_items = nullptr;
  int *d_counter = nullptr;
  int n_items = 0;
  void release() {
    if (d_imgs) cudaFree(d_imgs);
    if (d_items) cudaFree(d_items);
    if (d_counter) cudaFree(d_counter);
    d_imgs = nullptr;
    d_items = nullptr;
    d_counter = nullptr;
  }
};

struct Candidate {
  fbf_schedule kind = FBF_SCHEDULE_PERSISTENT;
  Persistent tables;
  Tc2BatchTables tc2[3];  // persistent tensor-core launches: W <= 16, 17..32, 33..48
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  double ms = 0.0;
  void release() {
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    exec = nullptr;
    graph = nullptr;
    tables.release();
    for (Tc2BatchTables &t : tc2) t.release();
  }
};

}  // namespace
}  // namespace fbf

using namespace fbf;

struct fbf_plan {
  int device = 0;
  int n_images = 0, n_items = 0;
  Candidate chosen;
};

namespace fbf {
namespace {

// Per-image tables and cost-sorted work list for BX x BY tiles.
template <int BX, int BY>
fbf_status build_persistent(const std::vector<FilterArgs> &args, Persistent *t) {
  const int n = (int)args.size();
  std::vector<ImageParams> imgs(n);
  struct Item {
    int img, tile;
    double cost;
  };
  std::vector<Item> items;
  for (int i = 0; i < n; ++i) {
    const FilterArgs &a = args[i];
    ImageParams &P = imgs[i];
    std::memset(&P, 0, sizeof(P));
    P.in = static_cast<const unsigned char *>(a.in);
    P.out = a.out;
    P.in_pitch = a.in_pitch;
    P.out_pitch = a.out_pitch;
    P.H = a.H;
    P.Wd = a.Wd;
    P.W = a.W;
    P.K = a.K;
    P.twoT = a.twoT;
    P.T = a.T;
    P.tiles_x = (a.Wd + BX - 1) / BX;
    std::memcpy(P.w2, a.w2, sizeof(P.w2));
    std::memcpy(P.d, a.d, sizeof(P.d));
    const int ntiles = a.H > 0 && a.Wd > 0 ? P.tiles_x * ((a.H + BY - 1) / BY) : 0;
    const double cost = (double)a.K * (2 * a.W + 1) + 8.0;  // per tile: harmonics x taps (+ staging)
    for (int t = 0; t < ntiles; ++t) items.push_back({i, t, cost});
  }
  std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });
  std::vector<int2> h_items(items.size());
  for (size_t k = 0; k < items.size(); ++k) h_items[k] = make_int2(items[k].img, items[k].tile);
  t->n_items = (int)items.size();
  bool ok = cudaMalloc(&t->d_imgs, sizeof(ImageParams) * std::max(n, 1)) == cudaSuccess &&
            cudaMalloc(&t->d_items, sizeof(int2) * std::max<size_t>(items.size(), 1)) == cudaSuccess &&
            cudaMalloc(&t->d_counter, sizeof(int)) == cudaSuccess;
  if (ok && n > 0)
    ok = cudaMemcpy(t->d_imgs, imgs.data(), sizeof(ImageParams) * n, cudaMemcpyHostToDevice) == cudaSuccess;
  if (ok && !items.empty())
    ok = cudaMemcpy(t->d_items, h_items.data(), sizeof(int2) * items.size(), cudaMemcpyHostToDevice) ==
         cudaSuccess;
  return ok ? FBF_OK : FBF_ERR_CUDA;
}

// Capture of a persistent schedule: counter reset + one launch (one CTA per SM).
template <int BX, int BY, int NBUF, int WCAP>
fbf_status capture_persistent(int device, int border, Candidate *c, cudaStream_t cs) {
  int sms = 0;
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
  const int grid = std::max(1, std::min(c->tables.n_items, sms));
  const size_t smem = batched_smem_bytes<BX, BY, NBUF, WCAP>();
  auto kern = fbf_batched_kernel<BX, BY, NBUF, WCAP>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return FBF_ERR_CUDA;
  BatchArgs args{c->tables.d_imgs, c->tables.d_items, c->tables.n_items, border, c->tables.d_counter};
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FBF_ERR_CUDA;
  cudaMemsetAsync(c->tables.d_counter, 0, sizeof(int), cs);
  if (c->tables.n_items > 0) kern<<<grid, kBNT, smem, cs>>>(args);
  if (cudaStreamEndCapture(cs, &c->graph) != cudaSuccess || !c->graph) return FBF_ERR_CUDA;
  return cudaGraphInstantiate(&c->exec, c->graph, 0) == cudaSuccess ? FBF_OK : FBF_ERR_CUDA;
}

// Capture of the persistent tensor-core schedule: one persistent launch per
// window band present in the batch (W <= 16, 17..32, 33..48), in that order,
// each over its images' tables with the instantiation sized for its band --
// an image runs on the same kernel as its single-image launch would, instead
// of the one the batch's widest window needs (9-10% slower at W = 9 and 15 on
// the 32-window instantiation).  The launches run once before the capture for
// the kernels' one-time host set-up.
fbf_status capture_persistent_tc(const std::vector<FilterArgs> &args, int mode, Candidate *c, cudaStream_t cs) {
  std::vector<FilterArgs> band[3];
  for (const FilterArgs &a : args) band[a.W <= 16 ? 0 : a.W <= 32 ? 1 : 2].push_back(a);
  for (int b = 0; b < 3; ++b) {
    const fbf_status st = c->tc2[b].build(band[b].data(), (int)band[b].size());
    if (st != FBF_OK) return st;
  }
  auto launch_all = [&]() -> fbf_status {
    for (int b = 0; b < 3; ++b) {
      const fbf_status st = launch_tc2_batch(c->tc2[b], mode, cs);
      if (st != FBF_OK) return st;
    }
    return FBF_OK;
  };
  fbf_status st = launch_all();
  if (st != FBF_OK) return st;
  if (cudaStreamSynchronize(cs) != cudaSuccess) return FBF_ERR_CUDA;
  if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return FBF_ERR_CUDA;
  st = launch_all();
  cudaGraph_t g = nullptr;
  const bool ended = cudaStreamEndCapture(cs, &g) == cudaSuccess;
  c->graph = g;
  if (st != FBF_OK) return st;
  if (!ended || !g) return FBF_ERR_CUDA;
  return cudaGraphInstantiate(&c->exec, c->graph, 0) == cudaSuccess ? FBF_OK : FBF_ERR_CUDA;
}

// Capture of one single-image launch per image in `form`, in image order on
// one branch (nbranch = 1) or spread over nbranch concurrent branches of the
// graph: images by decreasing cost (pixels x harmonics), each to the branch
// with the least cost so far; the branches fork from and join the capturing
// stream.  Every launch runs once before the capture, so that the kernels'
// one-time host set-up (function attributes, driver entry points) happens
// outside it.
fbf_status capture_per_image(const std::vector<FilterArgs> &args, fbf_form form, int nbranch, Candidate *c,
                             cudaStream_t cs) {
  for (const FilterArgs &a : args) {
    if (a.H == 0 || a.Wd == 0) continue;
    const fbf_status st = launch_filter(a, form, FBF_U8, cs);
    if (st != FBF_OK) return st;
  }
  if (cudaStreamSynchronize(cs) != cudaSuccess) return FBF_ERR_CUDA;
  std::vector<int> order;
  for (int i = 0; i < (int)args.size(); ++i)
    if (args[i].H > 0 && args[i].Wd > 0) order.push_back(i);
  auto cost = [&](int i) { return (double)args[i].H * args[i].Wd * args[i].K; };
  if (nbranch > 1) std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost(x) > cost(y); });
  // side[b - 1] is branch b; branch 0 is the capturing stream; ev[0] forks, ev[b] joins branch b
  std::vector<cudaStream_t> side(nbranch > 1 ? nbranch - 1 : 0, nullptr);
  std::vector<cudaEvent_t> ev(side.size() + 1, nullptr);
  bool ok = true;
  for (auto &s : side) ok = ok && cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess;
  for (auto &e : ev) ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
  fbf_status st = ok ? FBF_OK : FBF_ERR_CUDA;
  bool capturing = false;
  if (st == FBF_OK) {
    capturing = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) == cudaSuccess;
    if (!capturing) st = FBF_ERR_CUDA;
  }
  bool forked = false;
  if (st == FBF_OK && !side.empty()) {
    forked = cudaEventRecord(ev[0], cs) == cudaSuccess;
    for (auto &s : side) forked = forked && cudaStreamWaitEvent(s, ev[0], 0) == cudaSuccess;
    if (!forked) st = FBF_ERR_CUDA;
  }
  std::vector<double> load(side.size() + 1, 0.0);
  for (size_t k = 0; k < order.size() && st == FBF_OK; ++k) {
    const int i = order[k];
    size_t b = 0;
    for (size_t j = 1; j < load.size(); ++j)
      if (load[j] < load[b]) b = j;
    load[b] += cost(i);
    st = launch_filter(args[i], form, FBF_U8, b == 0 ? cs : side[b - 1]);
  }
  if (forked)  // every branch rejoins the capturing stream, also after a failed launch
    for (size_t b = 1; b < ev.size(); ++b)
      if (cudaEventRecord(ev[b], side[b - 1]) != cudaSuccess || cudaStreamWaitEvent(cs, ev[b], 0) != cudaSuccess)
        st = FBF_ERR_CUDA;
  cudaGraph_t g = nullptr;
  const bool ended = capturing && cudaStreamEndCapture(cs, &g) == cudaSuccess;
  c->graph = g;
  for (auto &e : ev)
    if (e) cudaEventDestroy(e);
  for (auto &s : side)
    if (s) cudaStreamDestroy(s);
  if (st != FBF_OK) return st;
  if (!ended || !g) return FBF_ERR_CUDA;
  return cudaGraphInstantiate(&c->exec, c->graph, 0) == cudaSuccess ? FBF_OK : FBF_ERR_CUDA;
}

#ifndef FBF_PLAN_BRANCHES
#define FBF_PLAN_BRANCHES 4
#endif
constexpr int kPlanBranches = FBF_PLAN_BRANCHES;  // concurrent branches of the *_STREAMS schedules

// Mean time of three replays of a candidate's graph (after one untimed replay).
fbf_status time_candidate(Candidate *c, cudaStream_t cs) {
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    return FBF_ERR_CUDA;
  }
  constexpr int kReps = 3;
  bool ok = cudaGraphLaunch(c->exec, cs) == cudaSuccess && cudaEventRecord(e0, cs) == cudaSuccess;
  for (int r = 0; ok && r < kReps; ++r) ok = cudaGraphLaunch(c->exec, cs) == cudaSuccess;
  ok = ok && cudaEventRecord(e1, cs) == cudaSuccess && cudaEventSynchronize(e1) == cudaSuccess;
  float ms = 0.f;
  if (ok) ok = cudaEventElapsedTime(&ms, e0, e1) == cudaSuccess;
  c->ms = ms / kReps;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  return ok ? FBF_OK : FBF_ERR_CUDA;
}

}  // namespace
}  // namespace fbf

static void plan_free(fbf_plan *p) {
  if (!p) return;
  p->chosen.release();
  delete p;
}

// Plan creation: `only` < 0 autotunes over the form's candidate schedules,
// otherwise captures that one schedule (which must be a candidate of the form).
static fbf_status plan_create(const fbf_image_desc *descs, int n, fbf_form form, fbf_border border, int only,
                              fbf_plan **out) {
  if (!out) return FBF_ERR_INVALID_ARGUMENT;
  *out = nullptr;
  if (n < 0 || (n > 0 && !descs)) return FBF_ERR_INVALID_ARGUMENT;
  if (border != FBF_BORDER_REFLECT && border != FBF_BORDER_TRUNCATE) return FBF_ERR_INVALID_ARGUMENT;
  const bool tc = is_tc_form(form);
  if (form != FBF_FORM_AUTO && form != FBF_FORM_FP32 && !tc) return FBF_ERR_INVALID_ARGUMENT;

  std::vector<FilterArgs> args(n);
  int wmax = 0;
  for (int i = 0; i < n; ++i) {
    const fbf_image_desc &d = descs[i];
    if (d.spatial == FBF_SPATIAL_GAUSSIAN_RECURSIVE) return FBF_ERR_UNSUPPORTED;  // single-image calls only
    fbf_coeffs c;
    fbf_status st = fbf_fit_coeffs(d.range, d.sigma_r, d.T, d.eps, d.K_fixed, d.levels, &c);
    if (st != FBF_OK) return st;
    fbf_params prm;
    prm.spatial = d.spatial;
    prm.sigma_s = d.sigma_s;
    prm.W = d.W;
    prm.border = border;
    prm.form = form;
    prm.coeffs = &c;
    st = pack_filter_args(&prm, d.d_in, FBF_U8, d.H, d.Wd, d.in_pitch, d.d_out, d.out_pitch, &args[i]);
    if (st != FBF_OK) return st;
    wmax = std::max(wmax, args[i].W);
  }

  fbf_plan *p = new fbf_plan();
  if (cudaGetDevice(&p->device) != cudaSuccess) {
    plan_free(p);
    return FBF_ERR_CUDA;
  }
  p->n_images = n;
  int n_items = 0;  // (image, tile) items of the 32 x 192 tiling, reported by fbf_plan_size
  for (const FilterArgs &a : args)
    if (a.H > 0 && a.Wd > 0) n_items += ((a.Wd + 31) / 32) * ((a.H + 191) / 192);
  p->n_items = n_items;
  cudaStream_t cs = nullptr;
  if (cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    plan_free(p);
    return FBF_ERR_CUDA;
  }

  // Candidate schedules of this form.
  std::vector<fbf_schedule> kinds;
  if (tc) {
    bool t_ok = true;  // the persistent tensor-core kernel's 2T-phase table holds 2T <= 510
    for (const FilterArgs &a : args) t_ok = t_ok && a.twoT >= 2 && a.twoT <= 510;
    const bool single = form == FBF_FORM_TC_FP16_SINGLE || form == FBF_FORM_TC_BF16_SINGLE;
    if (single && t_ok) kinds.push_back(FBF_SCHEDULE_PERSISTENT_TC);
    kinds.push_back(FBF_SCHEDULE_PER_IMAGE_FORM);
    kinds.push_back(FBF_SCHEDULE_PER_IMAGE_FORM_STREAMS);
  } else {
    if (wmax <= 32) kinds.push_back(FBF_SCHEDULE_PERSISTENT);  // its 32 x 192 tiles stage W <= 32
    if (wmax <= 16) kinds.push_back(FBF_SCHEDULE_PERSISTENT_WIDE);
    kinds.push_back(FBF_SCHEDULE_PER_IMAGE_FP32);
    kinds.push_back(FBF_SCHEDULE_PER_IMAGE_FP32_STREAMS);
    if (form == FBF_FORM_AUTO) {
      kinds.push_back(FBF_SCHEDULE_PER_IMAGE_FORM);
      kinds.push_back(FBF_SCHEDULE_PER_IMAGE_FORM_STREAMS);
    }
  }

  if (only >= 0) {
    if (std::find(kinds.begin(), kinds.end(), (fbf_schedule)only) == kinds.end()) {
      cudaStreamDestroy(cs);
      plan_free(p);
      return FBF_ERR_INVALID_ARGUMENT;
    }
    kinds.assign(1, (fbf_schedule)only);
  }

  fbf_status st = FBF_OK;
  std::vector<Candidate> cands;
  for (fbf_schedule k : kinds) {
    Candidate c;
    c.kind = k;
    if (k == FBF_SCHEDULE_PERSISTENT) {
      st = build_persistent<32, 192>(args, &c.tables);
      if (st == FBF_OK) st = capture_persistent<32, 192, 1, 32>(p->device, (int)border, &c, cs);
    } else if (k == FBF_SCHEDULE_PERSISTENT_WIDE) {
      st = build_persistent<64, 96>(args, &c.tables);
      if (st == FBF_OK) st = capture_persistent<64, 96, 1, 16>(p->device, (int)border, &c, cs);
    } else if (k == FBF_SCHEDULE_PERSISTENT_TC) {
      st = capture_persistent_tc(args, tc_mode(form), &c, cs);
    } else {
      const bool fp32 = k == FBF_SCHEDULE_PER_IMAGE_FP32 || k == FBF_SCHEDULE_PER_IMAGE_FP32_STREAMS;
      const bool streams = k == FBF_SCHEDULE_PER_IMAGE_FP32_STREAMS || k == FBF_SCHEDULE_PER_IMAGE_FORM_STREAMS;
      st = capture_per_image(args, fp32 ? FBF_FORM_FP32 : form, streams ? kPlanBranches : 1, &c, cs);
    }
    cands.push_back(c);
    if (st != FBF_OK) break;
  }
  // Autotune: replay and time every candidate, keep the fastest.  Three rounds
  // over all candidates, each candidate's best round kept: candidates within
  // a fraction of a percent of each other (the persistent launch and the
  // per-image launches on branches, on uneven batches) are then not decided
  // by their order or by one round's noise.
  size_t best = 0;
  if (st == FBF_OK && cands.size() > 1) {
    constexpr int kRounds = 3;
    std::vector<float> best_ms(cands.size(), 0.f);
    for (int round = 0; round < kRounds && st == FBF_OK; ++round)
      for (size_t i = 0; i < cands.size() && st == FBF_OK; ++i) {
        st = time_candidate(&cands[i], cs);
        if (round == 0 || cands[i].ms < best_ms[i]) best_ms[i] = cands[i].ms;
      }
    for (size_t i = 0; i < cands.size(); ++i) cands[i].ms = best_ms[i];
    for (size_t i = 1; i < cands.size(); ++i)
      if (cands[i].ms < cands[best].ms) best = i;
  }
  cudaStreamDestroy(cs);
  for (size_t i = 0; i < cands.size(); ++i)
    if (st != FBF_OK || i != best) cands[i].release();
  if (st != FBF_OK) {
    plan_free(p);
    return st;
  }
  p->chosen = cands[best];
  *out = p;
  return FBF_OK;
}

extern "C" fbf_status fbf_plan_create(const fbf_image_desc *descs, int n, fbf_form form, fbf_border border,
                                      fbf_plan **out) {
  return plan_create(descs, n, form, border, -1, out);
}

extern "C" fbf_status fbf_plan_create_schedule(const fbf_image_desc *descs, int n, fbf_form form,
                                               fbf_border border, fbf_schedule schedule, fbf_plan **out) {
  if (out) *out = nullptr;
  if ((int)schedule < 0 || (int)schedule > (int)FBF_SCHEDULE_PERSISTENT_TC) return FBF_ERR_INVALID_ARGUMENT;
  return plan_create(descs, n, form, border, (int)schedule, out);
}

extern "C" fbf_status fbf_filter_batched(fbf_plan *plan, cudaStream_t stream) {
  if (!plan || !plan->chosen.exec) return FBF_ERR_INVALID_ARGUMENT;
  return cuda_status(cudaGraphLaunch(plan->chosen.exec, stream));
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

extern "C" fbf_status fbf_plan_schedule(const fbf_plan *plan, fbf_schedule *schedule, double *ms) {
  if (!plan) return FBF_ERR_INVALID_ARGUMENT;
  if (schedule) *schedule = plan->chosen.kind;
  if (ms) *ms = plan->chosen.ms;
  return FBF_OK;
}
