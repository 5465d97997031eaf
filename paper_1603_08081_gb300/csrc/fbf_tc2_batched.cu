// Persistent batched launches of the second tensor-core layout (batched
// plans): the device tables of a batch, and one instantiation per window band
// chosen by the batch's largest W.
#include <algorithm>
#include <cstring>
#include <vector>

#include "fbf_tc2_kernel.cuh"

namespace fbf {

namespace {
size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }
}  // namespace

fbf_status Tc2BatchTables::build(const FilterArgs *args, int n) {
  release();
  std::vector<FilterArgs> imgs(n > 0 ? n : 0);
  std::vector<CUtensorMap> maps(imgs.size());
  std::vector<int> ok(imgs.size(), 0);
  struct Item {
    int img, tile;
    double cost;
  };
  std::vector<Item> items;
  wmax = 0;
  for (int i = 0; i < n; ++i) {
    FilterArgs a = args[i];
    std::memset(&maps[i], 0, sizeof(CUtensorMap));
    const int BYv = tc2::kLanes - 2 * a.W;
    if (a.W < 0 || a.W > FBF_WMAX || BYv < 1 || a.twoT < 2 || a.twoT > tc2::kTrigEntries) return FBF_ERR_RANGE;
    a.tiles_x = (a.Wd + tc2::kBX - 1) / tc2::kBX;
    a.ntiles = a.H > 0 && a.Wd > 0 ? a.tiles_x * ((a.H + BYv - 1) / BYv) : 0;
    imgs[i] = a;
    if (a.ntiles == 0) continue;
    wmax = std::max(wmax, a.W);
    ok[i] = cached_box_map(a.in, a.Wd, a.H, a.in_pitch, tc2::kBoxW, tc2::kLanes, &maps[i]) ? 1 : 0;
    // harmonics (plus the prologue's two) x (row chunks + the fixed per-harmonic work)
    const double cost = (a.K + 2.0) * (tc2::kx_of(a.W) / 16 + 8.0);
    for (int t = 0; t < a.ntiles; ++t) items.push_back({i, t, cost});
  }
  std::stable_sort(items.begin(), items.end(), [](const Item &x, const Item &y) { return x.cost > y.cost; });
  const size_t o_maps = align_up(sizeof(FilterArgs) * imgs.size(), 128);
  const size_t o_ok = o_maps + sizeof(CUtensorMap) * maps.size();
  const size_t o_items = align_up(o_ok + sizeof(int) * ok.size(), 16);
  const size_t bytes = std::max<size_t>(o_items + sizeof(int2) * items.size(), 16);
  std::vector<unsigned char> host(bytes, 0);
  if (!imgs.empty()) {
    std::memcpy(host.data(), imgs.data(), sizeof(FilterArgs) * imgs.size());
    std::memcpy(host.data() + o_maps, maps.data(), sizeof(CUtensorMap) * maps.size());
    std::memcpy(host.data() + o_ok, ok.data(), sizeof(int) * ok.size());
  }
  int2 *hi = reinterpret_cast<int2 *>(host.data() + o_items);
  for (size_t k = 0; k < items.size(); ++k) hi[k] = make_int2(items[k].img, items[k].tile);
  if (cudaMalloc(&mem, bytes) != cudaSuccess) {
    mem = nullptr;
    return FBF_ERR_CUDA;
  }
  if (cudaMemcpy(mem, host.data(), bytes, cudaMemcpyHostToDevice) != cudaSuccess) {
    release();
    return FBF_ERR_CUDA;
  }
  unsigned char *base = static_cast<unsigned char *>(mem);
  b.imgs = reinterpret_cast<const FilterArgs *>(base);
  b.maps = reinterpret_cast<const CUtensorMap *>(base + o_maps);
  b.map_ok = reinterpret_cast<const int *>(base + o_ok);
  b.items = reinterpret_cast<const int2 *>(base + o_items);
  b.nitems = (int)items.size();
  return FBF_OK;
}

void Tc2BatchTables::release() {
  if (mem) cudaFree(mem);
  mem = nullptr;
  b = Tc2Batch{};
  wmax = 0;
}

fbf_status launch_tc2_batch(const Tc2BatchTables &t, int mode, cudaStream_t s) {
  if (mode != 2 && mode != 3) return FBF_ERR_UNSUPPORTED;  // the single FP16 and BF16 forms
  if (t.b.nitems <= 0) return FBF_OK;
  if (mode == 3) {
    if (t.wmax <= 16) return tc2::launch_batch_cfg<1, 1, 4, 0>(t.b, s);
    if (t.wmax <= 32) return tc2::launch_batch_cfg<1, 1, 6, 0>(t.b, s);
    if (t.wmax <= 48) return tc2::launch_batch_cfg<1, 1, 8, 1>(t.b, s);
    return FBF_ERR_UNSUPPORTED;
  }
  if (t.wmax <= 16) return tc2::launch_batch_cfg<0, 1, 4, 0>(t.b, s);
  if (t.wmax <= 32) return tc2::launch_batch_cfg<0, 1, 6, 0>(t.b, s);
  if (t.wmax <= 48) return tc2::launch_batch_cfg<0, 1, 8, 1>(t.b, s);
  return FBF_ERR_UNSUPPORTED;
}

}  // namespace fbf
