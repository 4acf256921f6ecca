// gs_field.cu -- the session: a Gaussian field resident on the device with its Adam state and
// registered images, the field update of Sec. IV-B, hierarchical image weighting (Eq. 3-4),
// Local & Semi-Global iteration allocation (Eq. 5), the per-image learning rate (Eq. 6-8), and
// optimisation steps replayed from captured CUDA graphs.
//
// Readings where the paper is silent (the same ones throughout the library):
//  * overlap M[i][j] = tracks shared by images i and j / min(track counts);
//  * hierarchy layers = breadth-first depth over M > 0 from the new image; unreachable images
//    weigh 0; key images = the N_m highest positive weights (ties: lower id);
//  * Eq. 5 rounded by largest remainder (ties: lower id) so the key images get exactly T_I / 2;
//    the other half is split evenly over the non-key images, the remainder going to distinct
//    images drawn by a partial Fisher-Yates shuffle; with no other image, Eq. 5 spreads all T_I;
//    the T_I view slots are then Fisher-Yates shuffled;
//  * random draws: SplitMix64 seeded with seed ^ ((new_id + 1) * 0x9E3779B97F4A7C15), a draw in
//    [0, k) is next() mod k;
//  * a step over several views uses the mean of their Eq. 8 rates; the rate scales the mean
//    positions' Adam group by the scene extent (3DGS), the other groups keep the 3DGS rates;
//  * new Gaussians (Sec. IV-B) follow the 3DGS initialisation: isotropic log-scale from the
//    mean squared distance to the 3 nearest sparse points, identity rotation, opacity 0.1,
//    DC colour from the point colour, higher SH zero.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstring>
#include <memory>
#include <mutex>
#include <numeric>
#include <unordered_map>
#include <vector>

#include "gs_engine.h"

namespace gs {

namespace {

struct SplitMix64 {
  unsigned long long s;
  explicit SplitMix64(unsigned long long seed) : s(seed) {}
  unsigned long long next() {
    s += 0x9E3779B97F4A7C15ull;
    unsigned long long z = s;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
  }
  unsigned long long below(unsigned long long k) { return next() % k; }
};

struct Image {
  gs_camera cam;
  DevBuf rgb;
  std::vector<long long> tracks;  // sorted, unique
  int T = 0;                      // iterations trained (Eq. 7)
};

// A captured step bakes in every device address and workspace layout it touches; the key holds
// all of them so any reallocation or layout change forces a new capture.
struct GraphKey {
  std::vector<int> sizes;            // W, H per view
  std::vector<unsigned long long> sig;  // buffer addresses and layout sizes
  bool operator==(const GraphKey& o) const { return sizes == o.sizes && sig == o.sig; }
};

struct GraphEntry {
  GraphKey key;
  cudaGraphExec_t exec = nullptr;
  bool timing = false;
};

}  // namespace

// Autotuned tilings, shared by every session of the process: a step's cost depends on the device
// and on the size of its view set, not on the session, so a class is tuned once per device.
// Class = (device, floor(log2(total pixels of the step's views))).
struct TuneCache {
  std::mutex mu;
  std::vector<std::pair<std::pair<int, int>, Tiling>> entries;
  bool find(std::pair<int, int> key, Tiling* out) {
    std::lock_guard<std::mutex> lock(mu);
    for (auto& e : entries)
      if (e.first == key) {
        *out = e.second;
        return true;
      }
    return false;
  }
  void put(std::pair<int, int> key, const Tiling& t) {
    std::lock_guard<std::mutex> lock(mu);
    for (auto& e : entries)
      if (e.first == key) {
        e.second = t;
        return;
      }
    entries.push_back({key, t});
  }
  void clear() {
    std::lock_guard<std::mutex> lock(mu);
    entries.clear();
  }
};

TuneCache& tune_cache() {
  static TuneCache c;
  return c;
}

// The schedule of Sec. IV-C/IV-D on the host: Eq. 6-8 rates, Eq. 3-4 weights, the key images and
// Eq. 5 with the semi-global half, over an overlap matrix M (n x n) and the images' iteration
// counts T (Eq. 7).  The session and gs_schedule_plan both use it.
struct Schedule {
  const gs_field_config& cfg;
  const std::vector<std::vector<float>>& M;
  const std::vector<int>& T;
  int n() const { return (int)M.size(); }

  double lr_current(int Tj) const {
    const double t = Tj > cfg.T_a ? 1.0 : (double)Tj / (double)cfg.T_a;
    return std::exp(std::log((double)cfg.eta0) * (1.0 - t) + std::log((double)cfg.etaf) * t);
  }
  // Eq. 8
  double lr_image(int j) const {
    double acc = lr_current(T[j]);
    int cnt = 0;
    for (int i = 0; i < n(); ++i) {
      if (i == j || !(M[i][j] > 0.f)) continue;
      acc += (double)M[i][j] * lr_current(T[i]);
      ++cnt;
    }
    return acc / (double)(cnt + 1);
  }

  // Eq. 3-4
  void weights(int nw, std::vector<double>& w) const {
    const int N = n();
    w.assign(N, 0.0);
    std::vector<int> layer(N, 0);
    w[nw] = 1.0;
    layer[nw] = 1;
    std::vector<int> prev = {nw};
    int k = 1;
    while (!prev.empty()) {
      ++k;
      std::vector<int> next;
      for (int i = 0; i < N; ++i) {
        if (layer[i]) continue;
        for (int j : prev)
          if (M[j][i] > 0.f) {
            next.push_back(i);
            break;
          }
      }
      for (int i : next) layer[i] = k;
      for (int i : next) {
        if (k == 2) {
          w[i] = w[nw] * (double)M[i][nw];
        } else {
          double s = 0;
          for (int j : prev) s += w[j] * (double)M[j][i];
          w[i] = s / (double)prev.size();
        }
      }
      prev = next;
    }
  }

  static std::vector<int> key_images(const std::vector<double>& w, int n_m) {
    std::vector<int> cand;
    for (int i = 0; i < (int)w.size(); ++i)
      if (w[i] > 0.0) cand.push_back(i);
    std::sort(cand.begin(), cand.end(), [&](int a, int b) { return w[a] != w[b] ? w[a] > w[b] : a < b; });
    if ((int)cand.size() > n_m) cand.resize(n_m);
    return cand;
  }

  static std::vector<int> largest_remainder(const std::vector<double>& shares, const std::vector<int>& ids, int total) {
    double s = 0;
    for (double x : shares) s += x;
    std::vector<double> exact(shares.size());
    std::vector<int> base(shares.size());
    int used = 0;
    for (size_t k = 0; k < shares.size(); ++k) {
      exact[k] = (double)total * shares[k] / s;
      base[k] = (int)std::floor(exact[k]);
      used += base[k];
    }
    std::vector<size_t> order(shares.size());
    std::iota(order.begin(), order.end(), 0);
    std::sort(order.begin(), order.end(), [&](size_t a, size_t b) {
      const double ra = exact[a] - base[a], rb = exact[b] - base[b];
      return ra != rb ? ra > rb : ids[a] < ids[b];
    });
    for (int q = 0; q < total - used && q < (int)order.size(); ++q) base[order[q]] += 1;
    return base;
  }

  // Eq. 5 + the semi-global half; returns the shuffled view slots
  std::vector<int> allocate(int nw, int* n_keys) const {
    std::vector<double> w;
    weights(nw, w);
    std::vector<int> keys = key_images(w, cfg.N_m);
    if (n_keys) *n_keys = (int)keys.size();
    std::vector<double> shares;
    for (int i : keys) shares.push_back(1.0 - std::exp(-w[i]));
    std::vector<char> is_key((size_t)n(), 0);
    for (int i : keys) is_key[i] = 1;
    std::vector<int> others;
    for (int i = 0; i < n(); ++i)
      if (!is_key[i]) others.push_back(i);
    SplitMix64 rng(cfg.seed ^ ((unsigned long long)(nw + 1) * 0x9E3779B97F4A7C15ull));
    std::vector<int> iters((size_t)n(), 0);
    const int T_I = cfg.T_I;
    if (!others.empty()) {
      std::vector<int> tk = largest_remainder(shares, keys, T_I / 2);
      for (size_t q = 0; q < keys.size(); ++q) iters[keys[q]] = tk[q];
      const int half = T_I - T_I / 2;
      const int per = half / (int)others.size(), rem = half % (int)others.size();
      std::vector<int> arr = others;
      for (int i = 0; i < rem; ++i) {
        const int j = i + (int)rng.below((unsigned long long)(arr.size() - i));
        std::swap(arr[i], arr[j]);
      }
      for (int i : others) iters[i] = per;
      for (int i = 0; i < rem; ++i) iters[arr[i]] += 1;
    } else {
      std::vector<int> tk = largest_remainder(shares, keys, T_I);
      for (size_t q = 0; q < keys.size(); ++q) iters[keys[q]] = tk[q];
    }
    std::vector<int> slots;
    for (int i = 0; i < n(); ++i)
      for (int q = 0; q < iters[i]; ++q) slots.push_back(i);
    for (int i = (int)slots.size() - 1; i > 0; --i) {
      const int j = (int)rng.below((unsigned long long)(i + 1));
      std::swap(slots[i], slots[j]);
    }
    return slots;
  }
};

struct Field {
  gs_field_config cfg;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  std::unique_ptr<Raster> r;
  int n = 0, stride = 0;
  DevBuf params, adam_m, adam_v;
  DevBuf dstat;  // densification statistics: norm sums, counts (2 rows of stride)
  DevBuf dens_tmp;
  long long densify_round = 0;
  long long adam_step = 0;
  std::vector<Image> images;
  std::vector<std::vector<float>> M;  // overlap matrix
  // sparse points of all registered images, hashed by cells (the field update of Sec. IV-B)
  DevBuf pts_xyz, pts_next, grid_keys, grid_head, new_rgb, far_flags, far_off, far_count;
  // the same points in cells of kCoarseCells x grid_cell, for the 3-NN search where points are sparse
  DevBuf pts_next_c, grid_keys_c, grid_head_c;
  long long n_points = 0;
  unsigned grid_slots = 0;
  float grid_cell = 1.f;
  bool grid_ready = false;
  unsigned* count_h = nullptr;  // pinned
  // per-step buffers
  DevBuf step_img, step_last, step_dimg, step_T, step_gp;
  std::vector<GraphEntry> graphs;
  bool sized_for_views = false;
  std::vector<int> last_sizes;
  Tiling sized_tiling;  // tiling of the last sizing step
  Tiling last_tiling;   // tiling of the last step

  double last_loss = 0.0;
  unsigned long long last_pairs = 0, last_blended = 0, last_instances = 0;
  double last_load_std = 0.0;
  int last_kernels = 0;
  // the last run of steps: device time between events recorded before its first and after its last
  // step (no readback inside), its steps, and the bytes staged to and read from the device
  cudaEvent_t run_ev[2] = {nullptr, nullptr};
  double last_run_ms = 0.0;
  long long last_run_steps = 0;
  unsigned long long last_h2d_bytes = 0, last_d2h_bytes = 0;
  DevBuf hwc_stage;  // an interleaved host image on its way to the planar layout
  size_t own_bytes = 0;
  // snapshot (gs_field_snapshot / gs_field_restore)
  DevBuf snap_p, snap_m, snap_v;
  DevBuf canary_flags;  // scratch of the guard-word check
  int snap_n = -1, snap_stride = 0;
  long long snap_step = 0;
  std::vector<int> snap_T;

  size_t bytes_in_use() const { return own_bytes + (r ? r->bytes_in_use : 0); }

  ~Field() {
    if (own_stream && stream) cudaStreamDestroy(stream);
    for (auto& g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    params.release(&own_bytes);
    adam_m.release(&own_bytes);
    adam_v.release(&own_bytes);
    dstat.release(&own_bytes);
    dens_tmp.release(&own_bytes);
    for (auto& im : images) im.rgb.release(&own_bytes);
    step_img.release(&own_bytes);
    step_last.release(&own_bytes);
    step_dimg.release(&own_bytes);
    step_T.release(&own_bytes);
    step_gp.release(&own_bytes);
    snap_p.release(&own_bytes);
    snap_m.release(&own_bytes);
    snap_v.release(&own_bytes);
    canary_flags.release(&own_bytes);
    hwc_stage.release(&own_bytes);
    for (cudaEvent_t& e : run_ev)
      if (e) cudaEventDestroy(e);
    DevBuf* pts[] = {&pts_xyz,   &pts_next,  &grid_keys,  &grid_head,   &new_rgb,
                     &far_flags, &far_off,   &far_count,  &pts_next_c,  &grid_keys_c, &grid_head_c};
    for (DevBuf* b : pts) b->release(&own_bytes);
    if (count_h) cudaFreeHost(count_h);
  }

  // Every device buffer of the session (its own, its images', its rasterizer's) for the guard-word
  // check, in a fixed order.
  std::vector<CanaryRef> canary_refs() const {
    std::vector<CanaryRef> v = {
        {"params", &params}, {"adam_m", &adam_m}, {"adam_v", &adam_v}, {"dstat", &dstat}, {"dens_tmp", &dens_tmp},
        {"pts_xyz", &pts_xyz}, {"pts_next", &pts_next}, {"grid_keys", &grid_keys}, {"grid_head", &grid_head},
        {"new_rgb", &new_rgb}, {"far_flags", &far_flags}, {"far_off", &far_off}, {"far_count", &far_count},
        {"pts_next_c", &pts_next_c}, {"grid_keys_c", &grid_keys_c}, {"grid_head_c", &grid_head_c},
        {"step_img", &step_img}, {"step_last", &step_last}, {"step_dimg", &step_dimg}, {"step_T", &step_T},
        {"step_gp", &step_gp}, {"snap_p", &snap_p}, {"snap_m", &snap_m}, {"snap_v", &snap_v}};
    for (const Image& im : images) v.push_back({"image rgb", &im.rgb});
    if (r) {
      const Raster& R = *r;
      const CanaryRef rr[] = {
          {"step params", &R.sp_d}, {"views", &R.views_d}, {"ledger", &R.ledger_d}, {"control + scan state", &R.zeroA},
          {"histograms + sort state + ranges", &R.zeroB}, {"xyo", &R.xyo}, {"conic", &R.conic}, {"rgb", &R.rgb},
          {"depth", &R.depth}, {"radius", &R.radius}, {"rect", &R.rect}, {"count", &R.count}, {"offsets", &R.offsets},
          {"clamp", &R.clamp}, {"g2s", &R.g2s}, {"keys0", &R.keys0}, {"keys1", &R.keys1}, {"vals0", &R.vals0},
          {"vals1", &R.vals1}, {"ginst", &R.ginst}, {"ckpt", &R.ckpt}, {"cmask", &R.cmask}, {"order", &R.order},
          {"tile_chunks", &R.tile_chunks}, {"inst_rec", &R.inst_rec}, {"carry", &R.carry}, {"partials", &R.partials},
          {"block_sums", &R.block_sums}, {"raster image", &R.own_image}, {"raster last", &R.own_last},
          {"raster dimage", &R.own_dimage}};
      v.insert(v.end(), std::begin(rr), std::end(rr));
    }
    v.push_back({"hwc staging", &hwc_stage});
    return v;
  }

  gs_status check_guard_words() {
    const std::vector<CanaryRef> refs = canary_refs();
    gs_status s = canary_flags.reserve(((refs.size() + 31) / 32) * 4, &own_bytes);
    if (s) return s;
    return check_canaries(refs.data(), (int)refs.size(), static_cast<unsigned*>(canary_flags.p), stream);
  }

  PointGridDev grid_dev(bool coarse = false) const {
    PointGridDev g;
    g.xyz = static_cast<const float*>(pts_xyz.p);
    g.keys = static_cast<unsigned long long*>((coarse ? grid_keys_c : grid_keys).p);
    g.head = static_cast<int*>((coarse ? grid_head_c : grid_head).p);
    g.next = static_cast<const int*>((coarse ? pts_next_c : pts_next).p);
    g.mask = grid_slots ? grid_slots - 1u : 0u;
    g.cell = coarse ? gs::kCoarseCells * grid_cell : grid_cell;
    return g;
  }

  // Points first..first+count-1 into both grids.
  void insert_points(long long first, long long count) {
    launch_insert_points(grid_dev(false), static_cast<int*>(pts_next.p), first, count, stream);
    launch_insert_points(grid_dev(true), static_cast<int*>(pts_next_c.p), first, count, stream);
  }

  // Room for `want` sparse points: the point arrays keep their contents; a larger hash table is
  // rebuilt from every point registered so far.
  gs_status reserve_points(long long want) {
    gs_status s;
    if ((long long)(pts_xyz.bytes / 12) < want) {
      const long long cap = std::max<long long>(want, std::max<long long>(2 * (long long)(pts_xyz.bytes / 12), 65536));
      const size_t grow = (size_t)cap * 20 - pts_xyz.bytes - pts_next.bytes - pts_next_c.bytes;
      if (cfg.hbm_budget_bytes && bytes_in_use() + grow > cfg.hbm_budget_bytes)
        return fail(GS_ERR_BUDGET, "registering the sparse points would exceed hbm_budget_bytes");
      DevBuf nx, nn, nc;
      if ((s = nx.reserve((size_t)cap * 12, &own_bytes)) || (s = nn.reserve((size_t)cap * 4, &own_bytes)) ||
          (s = nc.reserve((size_t)cap * 4, &own_bytes))) {
        nx.release(&own_bytes);
        nn.release(&own_bytes);
        nc.release(&own_bytes);
        return s;
      }
      if (n_points > 0) {
        cudaMemcpyAsync(nx.p, pts_xyz.p, (size_t)n_points * 12, cudaMemcpyDeviceToDevice, stream);
        cudaMemcpyAsync(nn.p, pts_next.p, (size_t)n_points * 4, cudaMemcpyDeviceToDevice, stream);
        cudaMemcpyAsync(nc.p, pts_next_c.p, (size_t)n_points * 4, cudaMemcpyDeviceToDevice, stream);
      }
      cudaStreamSynchronize(stream);
      pts_xyz.release(&own_bytes);
      pts_next.release(&own_bytes);
      pts_next_c.release(&own_bytes);
      pts_xyz = nx;
      pts_next = nn;
      pts_next_c = nc;
    }
    if ((long long)grid_slots < 2 * want) {
      unsigned long long slots = 1024;
      while ((long long)slots < 2 * want) slots <<= 1;
      if (slots > (1ull << 31)) return fail(GS_ERR_CAPACITY, "too many sparse points");
      const size_t bytes = (size_t)slots * 24;
      const size_t have = grid_keys.bytes + grid_head.bytes + grid_keys_c.bytes + grid_head_c.bytes;
      if (cfg.hbm_budget_bytes && bytes > have && bytes_in_use() + (bytes - have) > cfg.hbm_budget_bytes)
        return fail(GS_ERR_BUDGET, "growing the point grid would exceed hbm_budget_bytes");
      DevBuf* tables[] = {&grid_keys, &grid_head, &grid_keys_c, &grid_head_c};
      for (DevBuf* b : tables) b->release(&own_bytes);
      if ((s = grid_keys.reserve((size_t)slots * 8, &own_bytes)) || (s = grid_head.reserve((size_t)slots * 4, &own_bytes)) ||
          (s = grid_keys_c.reserve((size_t)slots * 8, &own_bytes)) ||
          (s = grid_head_c.reserve((size_t)slots * 4, &own_bytes))) {
        grid_slots = 0;
        return s;
      }
      grid_slots = (unsigned)slots;
      cudaMemsetAsync(grid_keys.p, 0xFF, (size_t)slots * 8, stream);
      cudaMemsetAsync(grid_head.p, 0xFF, (size_t)slots * 4, stream);
      cudaMemsetAsync(grid_keys_c.p, 0xFF, (size_t)slots * 8, stream);
      cudaMemsetAsync(grid_head_c.p, 0xFF, (size_t)slots * 4, stream);
      insert_points(0, n_points);
    }
    return GS_OK;
  }

  std::vector<unsigned long long> signature() const {
    const Raster& R = *r;
    std::vector<unsigned long long> v;
    const DevBuf* bufs[] = {&params, &adam_m, &adam_v, &dstat, &step_img, &step_dimg, &step_last, &step_T, &step_gp,
                            &R.sp_d, &R.views_d, &R.zeroA, &R.zeroB, &R.xyo, &R.conic, &R.rgb, &R.depth, &R.radius,
                            &R.rect, &R.count, &R.offsets, &R.clamp, &R.g2s, &R.keys0, &R.keys1, &R.vals0, &R.vals1, &R.ginst,
                            &R.inst_rec, &R.carry,
                            &R.ckpt, &R.cmask, &R.order, &R.tile_chunks, &R.partials, &R.block_sums};
    for (const DevBuf* b : bufs) v.push_back((unsigned long long)(uintptr_t)b->p);
    const unsigned long long lay[] = {(unsigned long long)stride, R.m_cap, (unsigned long long)(uintptr_t)R.dstat, (unsigned long long)R.passes,
                                      (unsigned long long)R.n_tiles, R.zeroA_bytes, R.zeroB_bytes, R.sort_state_bytes,
                                      R.ranges_bytes, R.chunk_bytes, (unsigned long long)R.timing,
                                      (unsigned long long)R.tiling.tw, (unsigned long long)R.tiling.th,
                                      (unsigned long long)R.tiling.batch};
    v.insert(v.end(), std::begin(lay), std::end(lay));
    return v;
  }

  void drop_graphs() {
    for (auto& g : graphs)
      if (g.exec) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }

  float scene_extent() const {
    if (cfg.scene_extent > 0.f) return cfg.scene_extent;
    if (images.empty()) return 1.f;
    double c[3] = {0, 0, 0};
    std::vector<std::array<double, 3>> centres;
    for (const auto& im : images) {
      std::array<double, 3> p;
      for (int a = 0; a < 3; ++a)
        p[a] = -(im.cam.R[a] * im.cam.t[0] + im.cam.R[3 + a] * im.cam.t[1] + im.cam.R[6 + a] * im.cam.t[2]);
      centres.push_back(p);
      for (int a = 0; a < 3; ++a) c[a] += p[a];
    }
    for (int a = 0; a < 3; ++a) c[a] /= (double)centres.size();
    double rmax = 0;
    for (auto& p : centres) rmax = std::max(rmax, std::sqrt((p[0] - c[0]) * (p[0] - c[0]) + (p[1] - c[1]) * (p[1] - c[1]) +
                                                             (p[2] - c[2]) * (p[2] - c[2])));
    return (float)std::max(1.0, 1.1 * rmax);
  }

  // Grow parameter / Adam buffers to hold `want` Gaussians (stride multiple of 32).
  gs_status reserve_gaussians(long long want) {
    if (want <= stride) return GS_OK;
    long long ns = std::max<long long>(want, (long long)stride * 2);
    ns = std::max<long long>(ns, 1024);
    ns = (ns + 31) / 32 * 32;
    if (ns > (1 << 28)) return fail(GS_ERR_CAPACITY, "field capacity limit");
    const size_t bytes = (size_t)ns * kNumParams * 4;
    const size_t growth = 3 * (bytes - (size_t)stride * kNumParams * 4);
    if (cfg.hbm_budget_bytes && bytes_in_use() + growth > cfg.hbm_budget_bytes)
      return fail(GS_ERR_BUDGET, "growing the field would exceed hbm_budget_bytes");
    DevBuf np, nm, nv;
    gs_status s;
    if ((s = np.reserve(bytes, &own_bytes)) || (s = nm.reserve(bytes, &own_bytes)) || (s = nv.reserve(bytes, &own_bytes))) {
      np.release(&own_bytes);
      nm.release(&own_bytes);
      nv.release(&own_bytes);
      return s;
    }
    cudaMemsetAsync(np.p, 0, bytes, stream);
    cudaMemsetAsync(nm.p, 0, bytes, stream);
    cudaMemsetAsync(nv.p, 0, bytes, stream);
    if (n > 0) {
      cudaMemcpy2DAsync(np.p, ns * 4, params.p, (size_t)stride * 4, (size_t)n * 4, kNumParams, cudaMemcpyDeviceToDevice, stream);
      cudaMemcpy2DAsync(nm.p, ns * 4, adam_m.p, (size_t)stride * 4, (size_t)n * 4, kNumParams, cudaMemcpyDeviceToDevice, stream);
      cudaMemcpy2DAsync(nv.p, ns * 4, adam_v.p, (size_t)stride * 4, (size_t)n * 4, kNumParams, cudaMemcpyDeviceToDevice, stream);
    }
    DevBuf nd;
    if ((s = nd.reserve((size_t)ns * 8, &own_bytes))) {
      np.release(&own_bytes);
      nm.release(&own_bytes);
      nv.release(&own_bytes);
      return s;
    }
    cudaMemsetAsync(nd.p, 0, (size_t)ns * 8, stream);
    if (n > 0 && dstat.p)
      cudaMemcpy2DAsync(nd.p, ns * 4, dstat.p, (size_t)stride * 4, (size_t)n * 4, 2, cudaMemcpyDeviceToDevice, stream);
    cudaStreamSynchronize(stream);
    params.release(&own_bytes);
    adam_m.release(&own_bytes);
    adam_v.release(&own_bytes);
    dstat.release(&own_bytes);
    params = np;
    adam_m = nm;
    adam_v = nv;
    dstat = nd;
    stride = (int)ns;
    drop_graphs();
    sized_for_views = false;
    return GS_OK;
  }

  // Eq. 6-7
  std::vector<int> image_T() const {
    std::vector<int> t;
    t.reserve(images.size());
    for (const Image& im : images) t.push_back(im.T);
    return t;
  }
  double lr_image(int j) const {
    const std::vector<int> t = image_T();
    return Schedule{cfg, M, t}.lr_image(j);
  }
  void weights(int nw, std::vector<double>& w) const {
    const std::vector<int> t = image_T();
    Schedule{cfg, M, t}.weights(nw, w);
  }
  std::vector<int> key_images(const std::vector<double>& w, int n_m) const { return Schedule::key_images(w, n_m); }
  std::vector<int> allocate(int nw, int* n_keys) const {
    const std::vector<int> t = image_T();
    return Schedule{cfg, M, t}.allocate(nw, n_keys);
  }

  gs_status ensure_step_buffers(long long pix) {
    gs_status s;
    if ((s = step_img.reserve(pix * 12, &own_bytes)) || (s = step_dimg.reserve(pix * 12, &own_bytes)) ||
        (s = step_last.reserve(pix * 4, &own_bytes)) || (s = step_T.reserve(pix * 4, &own_bytes)) ||
        (s = step_gp.reserve(pix * 4, &own_bytes)))
      return s;
    return GS_OK;
  }

  // Enqueue one whole step (forward, loss, backward + Adam); no readback, no synchronisation
  // (except the sizing step, which reads the instance count back mid-step).
  gs_status enqueue_step(bool size_exactly) {
    gs_status s;
    Raster& R = *r;
    R.upload(stream);
    if ((s = R.enqueue_forward_head(stream, static_cast<float*>(params.p), stride, size_exactly))) return s;
    if ((s = R.enqueue_forward_tail(stream, static_cast<float*>(step_img.p), static_cast<float*>(step_T.p),
                                    static_cast<unsigned*>(step_last.p), static_cast<unsigned*>(step_gp.p))))
      return s;
    R.enqueue_loss(stream, static_cast<float*>(step_img.p), static_cast<float*>(step_dimg.p), true);
    R.enqueue_backward(stream, static_cast<float*>(params.p), static_cast<float*>(step_img.p),
                       static_cast<unsigned*>(step_last.p), static_cast<float*>(step_dimg.p), nullptr,
                       static_cast<float*>(adam_m.p), static_cast<float*>(adam_v.p), nullptr);
    return GS_OK;
  }

  // Views of the next step: workspace sizes, and the mean of their Eq. 8 rates.
  std::vector<int> cur_sizes;
  gs_status setup_views(const int* ids, int nv, double* lr_mean) {
    if (nv <= 0 || nv > kMaxViews) return fail(GS_ERR_CAPACITY, "views per step must be in 1..32");
    if (n <= 0) return fail(GS_ERR_STATE, "the field has no Gaussians");
    std::vector<gs_camera> cams(nv);
    std::vector<const float*> tg(nv);
    cur_sizes.clear();
    double lr_sum = 0;
    for (int k = 0; k < nv; ++k) {
      if (ids[k] < 0 || ids[k] >= (int)images.size()) return fail(GS_ERR_INVALID_ARG, "view id out of range");
      cams[k] = images[ids[k]].cam;
      tg[k] = static_cast<const float*>(images[ids[k]].rgb.p);
      cur_sizes.push_back(cams[k].width);
      cur_sizes.push_back(cams[k].height);
      lr_sum += lr_image(ids[k]);
    }
    Raster& R = *r;
    gs_status s;
    if ((s = R.set_views(cams.data(), nv, tg.data()))) return s;
    R.stride = stride;
    R.n = n;
    R.dstat = cfg.densify_stats ? static_cast<float*>(dstat.p) : nullptr;
    if ((s = R.ensure_records(stride)) || (s = ensure_step_buffers(R.n_pix)) || (s = R.ensure_instances(R.m_cap)))
      return s;
    *lr_mean = lr_sum / nv;
    return GS_OK;
  }

  // Fill the staging parameters of a step (after Raster::stage) for Adam step `t`.
  // With batch_scaling a step over B views scales every rate by sqrt(B) and raises the betas to
  // the power B (Zhao et al. 2024, large-batch 3DGS training).
  void fill_params(int nv, double lr_mean, long long t) {
    StepParams& P = *r->sp_h;
    P.n = n;
    P.n_views = nv;
    for (int a = 0; a < 3; ++a) P.bg[a] = cfg.bg[a];
    P.lambda_ssim = cfg.lambda_ssim;
    P.lambda_l1 = cfg.lambda_l1 >= 0.f ? cfg.lambda_l1 : 1.f - cfg.lambda_ssim;
    P.lambda_load = cfg.lambda_load;
    double scale = 1.0, b1 = cfg.beta1, b2 = cfg.beta2;
    if (cfg.batch_scaling && nv > 1) {
      scale = std::sqrt((double)nv);
      b1 = std::pow(b1, (double)nv);
      b2 = std::pow(b2, (double)nv);
    }
    P.lr[0] = (float)(scale * lr_mean * (double)scene_extent());
    P.lr[1] = (float)(scale * cfg.lr_scale);
    P.lr[2] = (float)(scale * cfg.lr_rot);
    P.lr[3] = (float)(scale * cfg.lr_opacity);
    P.lr[4] = (float)(scale * cfg.lr_sh_dc);
    P.lr[5] = (float)(scale * cfg.lr_sh_rest);
    P.beta1 = (float)b1;
    P.beta2 = (float)b2;
    P.eps = cfg.adam_eps;
    P.step_size_scale = (float)(1.0 / (1.0 - std::pow(b1, (double)t)));
    P.bc2_sqrt = (float)std::sqrt(1.0 - std::pow(b2, (double)t));
    P.adam = 1;
    P.sparse = cfg.sparse_adam ? 1 : 0;
  }

  // Enqueue the prepared step: the sizing launch for new view sizes, else a graph replay (captured
  // on first use) or an eager launch.
  gs_status enqueue_prepared(int nv) {
    Raster& R = *r;
    gs_status s;
    const bool first = !sized_for_views || cur_sizes != last_sizes || !(sized_tiling == R.tiling);
    if (first) {
      if ((s = enqueue_step(true))) return s;
      sized_for_views = true;
      last_sizes = cur_sizes;
      sized_tiling = R.tiling;
      return GS_OK;
    }
    if (!cfg.use_graph) return enqueue_step(false);
    GraphKey key{cur_sizes, signature()};
    GraphEntry* ge = nullptr;
    for (auto& g : graphs)
      if (g.key == key && g.timing == R.timing) ge = &g;
    if (!ge) {
      TraceRange trace("graph capture");
      if (graphs.size() >= 8) drop_graphs();
      cudaGraph_t graph;
      std::unique_lock<std::mutex> lock(alloc_capture_mutex());
      cudaError_t e = cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("begin capture: ") + cudaGetErrorString(e));
      // The pinned staging copy is captured: each replay re-reads sp_h / views_h.
      gs_status cs = enqueue_step(false);
      e = cudaStreamEndCapture(stream, &graph);
      lock.unlock();
      if (cs) return cs;
      if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("end capture: ") + cudaGetErrorString(e));
      GraphEntry g;
      g.key = key;
      g.timing = R.timing;
      e = cudaGraphInstantiate(&g.exec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("instantiate: ") + cudaGetErrorString(e));
      graphs.push_back(g);
      ge = &graphs.back();
    }
    (void)nv;
    cudaError_t e = cudaGraphLaunch(ge->exec, stream);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("graph launch: ") + cudaGetErrorString(e));
    return GS_OK;
  }

  bool auto_tiling() const { return cfg.tiling.tile_w == 0 && cfg.tiling.tile_h == 0 && cfg.tiling.batch == 0; }
  Tiling fixed_tiling() const {
    if (auto_tiling()) return Tiling{};
    return Tiling{cfg.tiling.tile_w, cfg.tiling.tile_h, cfg.tiling.batch};
  }

  std::pair<int, int> view_class(const int* ids, int nv) const {
    long long pix = 0;
    for (int k = 0; k < nv; ++k)
      if (ids[k] >= 0 && ids[k] < (int)images.size())
        pix += (long long)images[ids[k]].cam.width * images[ids[k]].cam.height;
    int b = 0;
    while ((pix >> b) > 1) ++b;
    int dev = 0;
    cudaGetDevice(&dev);
    return {dev, b};
  }

  // Time every compiled tiling on these views (the whole step with the projection backward in
  // its write-nothing mode, so the field is untouched) and remember the fastest for the class.
  gs_status autotune(const int* ids, int nv, int reps, gs_autotune_result* out) {
    Raster& R = *r;
    gs_status s;
    if (nv <= 0 || nv > kMaxViews) return fail(GS_ERR_CAPACITY, "views per step must be in 1..32");
    if (n <= 0) return fail(GS_ERR_STATE, "the field has no Gaussians");
    if (reps < 1) return fail(GS_ERR_INVALID_ARG, "reps must be >= 1");
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
    Tiling cand[GS_MAX_TILINGS];
    const int nc = std::min(tiling_candidates(cand, GS_MAX_TILINGS), GS_MAX_TILINGS);
    float ms[GS_MAX_TILINGS];
    const Tiling keep = R.tiling;
    const bool keep_timing = R.timing;
    R.timing = false;  // the per-kernel events are for real steps only
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    int best = -1;
    s = GS_OK;
    for (int c = 0; c < nc && !s; ++c) {
      ms[c] = INFINITY;
      R.tiling = cand[c];
      double lr_mean = 0;
      gs_status cs = setup_views(ids, nv, &lr_mean);
      if (cs == GS_ERR_OOM || cs == GS_ERR_BUDGET || cs == GS_ERR_CAPACITY) continue;  // this candidate does not fit
      if (cs) {
        s = cs;
        break;
      }
      if ((s = R.stage(stream))) break;
      fill_params(nv, lr_mean, adam_step + 1);
      R.sp_h->adam = 2;  // the projection backward runs but writes nothing
      std::memcpy(R.views_h, R.views.data(), sizeof(ViewDev) * nv);
      R.reset_ledger(stream);
      R.upload(stream);
      float* img = static_cast<float*>(step_img.p);
      float* dimg = static_cast<float*>(step_dimg.p);
      for (int rep = 0; rep <= reps && !s; ++rep) {  // rep 0: sizing + warm-up
        if (rep == 1) cudaEventRecord(e0, stream);
        cs = R.enqueue_forward_head(stream, static_cast<float*>(params.p), stride, rep == 0);
        if (cs == GS_ERR_OOM || cs == GS_ERR_BUDGET || cs == GS_ERR_CAPACITY) break;
        if ((s = cs)) break;
        if ((s = R.enqueue_forward_tail(stream, img, static_cast<float*>(step_T.p), static_cast<unsigned*>(step_last.p),
                                        static_cast<unsigned*>(step_gp.p))))
          break;
        R.enqueue_loss(stream, img, dimg, true);
        R.enqueue_backward(stream, static_cast<float*>(params.p), img, static_cast<unsigned*>(step_last.p), dimg,
                           nullptr, static_cast<float*>(adam_m.p), static_cast<float*>(adam_v.p), nullptr);
        if (rep == reps) {
          cudaEventRecord(e1, stream);
          R.read_ledger(stream);
          e = cudaStreamSynchronize(stream);
          if (e != cudaSuccess) {
            s = fail(GS_ERR_CUDA, std::string("autotune: ") + cudaGetErrorString(e));
            break;
          }
          if (R.ledger_h->error & kErrTimeout) {
            s = fail(GS_ERR_TIMEOUT, "a device-side wait (decoupled look-back) timed out");
            break;
          }
          float t = 0.f;
          if (cudaEventElapsedTime(&t, e0, e1) == cudaSuccess && R.ledger_h->skip == 0u) {
            ms[c] = t / (float)reps;
            if (best < 0 || ms[c] < ms[best]) best = c;
          }
        }
      }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    R.timing = keep_timing;
    R.reset_ledger(stream);
    sized_for_views = false;  // the next step sizes its buffers for its own tiling
    if (s) {
      R.tiling = keep;
      return s;
    }
    if (best < 0) {
      R.tiling = keep;
      return fail(GS_ERR_OOM, "autotune: no tiling fits");
    }
    R.tiling = cand[best];
    tune_cache().put(view_class(ids, nv), cand[best]);
    if (out) {
      out->chosen = gs_tiling{cand[best].tw, cand[best].th, cand[best].batch};
      out->n_candidates = nc;
      for (int c = 0; c < nc; ++c) {
        out->candidates[c] = gs_tiling{cand[c].tw, cand[c].th, cand[c].batch};
        out->ms[c] = ms[c];
      }
    }
    if (!auto_tiling()) R.tiling = fixed_tiling();
    return GS_OK;
  }

  // Tiling of a step over these views: the configured one, else the class's autotuned one
  // (tuning the class first if `may_tune`).
  gs_status pick_tiling(const int* ids, int nv, bool may_tune) {
    Raster& R = *r;
    if (!auto_tiling()) {
      R.tiling = fixed_tiling();
      return GS_OK;
    }
    Tiling t;
    if (tune_cache().find(view_class(ids, nv), &t)) {
      R.tiling = t;
      return GS_OK;
    }
    if (!may_tune) return fail(GS_ERR_STATE, "tiling of this view class not tuned");
    return autotune(ids, nv, 3, nullptr);
  }

  // Run `count` steps (views of step k: groups[k]) enqueued back to back, with one
  // synchronisation at the end.  Returns how many completed (a prefix); the caller re-runs the
  // rest.  T_j and the Adam step count are advanced only for completed steps.
  gs_status run_steps(const std::vector<std::vector<int>>& groups, size_t first_group, size_t count, size_t* done,
                      double* loss_sum) {
    TraceRange trace("run of steps");
    Raster& R = *r;
    gs_status s;
    const long long step0 = adam_step;
    // tune any view class not seen yet before the run starts (tuning synchronises)
    for (size_t k = 0; k < count; ++k) {
      const std::vector<int>& ids = groups[first_group + k];
      if ((s = pick_tiling(ids.data(), (int)ids.size(), true))) return s;
    }
    std::vector<int> T0;
    for (auto& im : images) T0.push_back(im.T);
    for (cudaEvent_t& e : run_ev)
      if (!e && cudaEventCreate(&e) != cudaSuccess) return fail(GS_ERR_CUDA, "event creation failed");
    R.reset_ledger(stream);
    cudaEventRecord(run_ev[0], stream);
    for (size_t k = 0; k < count; ++k) {
      const std::vector<int>& ids = groups[first_group + k];
      double lr_mean = 0;
      if ((s = pick_tiling(ids.data(), (int)ids.size(), false))) return s;
      if ((s = setup_views(ids.data(), (int)ids.size(), &lr_mean))) return s;
      if (lr_override) lr_mean = (*lr_override)[first_group + k];
      if ((s = R.stage(stream))) return s;  // waits only for the previous step's parameter upload
      fill_params((int)ids.size(), lr_mean, adam_step + 1);
      std::memcpy(R.views_h, R.views.data(), sizeof(ViewDev) * ids.size());
      if ((s = enqueue_prepared((int)ids.size()))) return s;
      ++adam_step;
      last_tiling = R.tiling;
      for (int id : ids) images[id].T += 1;  // tentative: Eq. 7 counts for the next steps' rates
    }
    cudaEventRecord(run_ev[1], stream);
    R.read_ledger(stream);
    R.enqueue_readback(stream);
    cudaError_t e = cudaStreamSynchronize(stream);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("step: ") + cudaGetErrorString(e));
    {
      float ms = 0.f;
      last_run_ms = cudaEventElapsedTime(&ms, run_ev[0], run_ev[1]) == cudaSuccess ? (double)ms : 0.0;
      last_run_steps = (long long)count;
      // per step: the staged step parameters and views; per run: the ledger and control block
      last_h2d_bytes = (unsigned long long)count * (sizeof(StepParams) + sizeof(ViewDev) * (size_t)R.views.size());
      last_d2h_bytes = sizeof(Ledger) + sizeof(Control);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("step launch: ") + cudaGetErrorString(e));
    const Ledger& Lg = *R.ledger_h;
    if (Lg.error & kErrTimeout) return fail(GS_ERR_TIMEOUT, "a device-side wait (decoupled look-back) timed out");
    if (cfg.debug_canaries && (s = check_guard_words())) return s;
    const size_t ok = std::min<size_t>(Lg.steps_ok, count);
    // commit the completed prefix only
    adam_step = step0 + (long long)ok;
    for (size_t j = 0; j < images.size(); ++j) images[j].T = j < T0.size() ? T0[j] : 0;
    for (size_t k = 0; k < ok; ++k)
      for (int id : groups[first_group + k]) images[id].T += 1;
    if (ok < count) {
      // a step overflowed the instance buffers: grow them for the next try
      if ((s = R.ensure_instances(Lg.m_need + Lg.m_need / 4 + 1024))) return s;
      drop_graphs();
    }
    *done = ok;
    *loss_sum += Lg.loss_sum;
    last_pairs = ok ? Lg.pairs / ok : 0;
    last_blended = ok ? Lg.blended / ok : 0;
    last_instances = ok ? Lg.instances / ok : 0;
    last_kernels = kStepLaunchesBase + R.passes + (R.dstat ? 1 : 0);
    sum_pairs += Lg.pairs;
    if (ok && Lg.last_gp_pixels) {  // Eq. 9: std of G_p over the pixels some Gaussian reaches
      const double mean = (double)Lg.last_gp_sum / (double)Lg.last_gp_pixels;
      const double var = (double)Lg.last_gp_sq / (double)Lg.last_gp_pixels - mean * mean;
      last_load_std = std::sqrt(std::max(0.0, var));
    }
    if (ok == count && count > 0) {
      last_loss = R.ctl_h->loss;
      R.collect_times();
      R.have_forward = true;
    }
    return GS_OK;
  }

  // Steps in runs of up to `chunk`, re-running whatever an overflow skipped.
  gs_status run_all(const std::vector<std::vector<int>>& groups, size_t chunk, double* loss_sum) {
    size_t g = 0;
    int stalls = 0;
    while (g < groups.size()) {
      size_t done = 0;
      gs_status s = run_steps(groups, g, std::min(chunk, groups.size() - g), &done, loss_sum);
      if (s) return s;
      g += done;
      stalls = done ? 0 : stalls + 1;
      if (stalls > 3) return fail(GS_ERR_CAPACITY, "instance buffers kept overflowing");
    }
    return GS_OK;
  }

  unsigned long long sum_pairs = 0;
  const std::vector<double>* lr_override = nullptr;  // per step of a run: the position rate before x extent

  gs_status step(const int* ids, int nv, float* out_loss) {
    std::vector<std::vector<int>> groups(1, std::vector<int>(ids, ids + nv));
    double loss_sum = 0;
    gs_status s = run_all(groups, 1, &loss_sum);
    if (s) return s;
    if (out_loss) *out_loss = (float)last_loss;
    return GS_OK;
  }
};

}  // namespace gs

using gs::fail;
using gs::Field;

static Field* F(gs_field* f) { return reinterpret_cast<Field*>(f); }
static const Field* F(const gs_field* f) { return reinterpret_cast<const Field*>(f); }

extern "C" {

void gs_field_config_default(gs_field_config* c) {
  if (!c) return;
  std::memset(c, 0, sizeof(*c));
  c->T_I = 200;
  c->N_m = 10;
  c->T_a = 200;
  c->batch_views = 1;
  c->use_graph = 1;
  c->async_steps = 16;
  c->eta0 = 1.6e-4f;
  c->etaf = 1.6e-6f;
  c->lambda_ssim = 0.2f;
  c->lambda_l1 = -1.f;  // 1 - lambda_ssim
  c->lambda_load = 0.f;
  c->lr_scale = 5e-3f;
  c->lr_rot = 1e-3f;
  c->lr_opacity = 0.05f;
  c->lr_sh_dc = 2.5e-3f;
  c->lr_sh_rest = 2.5e-3f / 20.f;
  c->beta1 = 0.9f;
  c->beta2 = 0.999f;
  c->adam_eps = 1e-15f;
  c->seed = 0;
  c->initial_capacity = 0;
}

gs_status gs_field_init(const gs_field_config* cfg, void* stream, gs_field** out) {
  if (!cfg || !out) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  *out = nullptr;
  if (cfg->T_I <= 0 || cfg->N_m <= 0 || cfg->T_a <= 0 || cfg->batch_views <= 0 || cfg->batch_views > gs::kMaxViews ||
      !(cfg->eta0 > 0.f) || !(cfg->etaf > 0.f) || cfg->lambda_ssim < 0.f || cfg->lambda_ssim > 1.f ||
      !(cfg->lambda_load >= 0.f) || !(cfg->lambda_l1 >= 0.f || cfg->lambda_l1 == -1.f))
    return fail(GS_ERR_INVALID_ARG, "invalid field configuration");
  const bool tiling_auto = cfg->tiling.tile_w == 0 && cfg->tiling.tile_h == 0 && cfg->tiling.batch == 0;
  if (!tiling_auto && !gs::tiling_supported(gs::Tiling{cfg->tiling.tile_w, cfg->tiling.tile_h, cfg->tiling.batch}))
    return fail(GS_ERR_INVALID_ARG, "configured tiling not among gs_tiling_candidates");
  Field* f = new (std::nothrow) Field();
  if (!f) return fail(GS_ERR_OOM, "host allocation failed");
  f->cfg = *cfg;
  f->stream = static_cast<cudaStream_t>(stream);
  if (!f->stream) {
    // Graph capture needs a non-legacy stream.
    if (cudaStreamCreateWithFlags(&f->stream, cudaStreamNonBlocking) != cudaSuccess) {
      delete f;
      return fail(GS_ERR_CUDA, "stream creation failed");
    }
    f->own_stream = true;
  }
  f->r.reset(new (std::nothrow) gs::Raster());
  if (!f->r || !f->r->sp_h || !f->r->sp_d.p) {
    delete f;
    return fail(GS_ERR_OOM, "raster allocation failed");
  }
  if (cfg->initial_capacity > 0) {
    gs_status s = f->reserve_gaussians(cfg->initial_capacity);
    if (s) {
      delete f;
      return s;
    }
  }
  *out = reinterpret_cast<gs_field*>(f);
  return GS_OK;
}

gs_status gs_field_destroy(gs_field* f) {
  if (!f) return GS_OK;
  cudaStreamSynchronize(F(f)->stream);
  delete F(f);
  return GS_OK;
}

gs_status gs_field_set_gaussians(gs_field* ff, const float* host, int64_t n, int64_t src_stride) {
  gs::TraceRange trace("gs_field_set_gaussians");
  Field* f = F(ff);
  if (!f || (!host && n > 0) || n < 0 || src_stride < n) return fail(GS_ERR_INVALID_ARG, "bad arguments");
  gs_status s = f->reserve_gaussians(std::max<int64_t>(n, 1));
  if (s) return s;
  const size_t bytes = (size_t)f->stride * gs::kNumParams * 4;
  cudaMemsetAsync(f->params.p, 0, bytes, f->stream);
  cudaMemsetAsync(f->adam_m.p, 0, bytes, f->stream);
  cudaMemsetAsync(f->adam_v.p, 0, bytes, f->stream);
  cudaMemsetAsync(f->dstat.p, 0, (size_t)f->stride * 8, f->stream);
  if (n > 0)
    cudaMemcpy2DAsync(f->params.p, (size_t)f->stride * 4, host, (size_t)src_stride * 4, (size_t)n * 4, gs::kNumParams,
                      cudaMemcpyHostToDevice, f->stream);
  cudaError_t e = cudaStreamSynchronize(f->stream);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  f->n = (int)n;
  f->adam_step = 0;
  return GS_OK;
}

gs_status gs_field_get_gaussians(gs_field* ff, float* host, float* host_m, float* host_v, int64_t dst_stride,
                                 int64_t* out_n) {
  Field* f = F(ff);
  if (!f) return fail(GS_ERR_INVALID_ARG, "NULL field");
  if (out_n) *out_n = f->n;
  if (!host && !host_m && !host_v) return GS_OK;
  if (dst_stride < f->n) return fail(GS_ERR_INVALID_ARG, "dst_stride < n");
  cudaStreamSynchronize(f->stream);
  const gs::DevBuf* src[3] = {&f->params, &f->adam_m, &f->adam_v};
  float* dst[3] = {host, host_m, host_v};
  for (int k = 0; k < 3; ++k) {
    if (!dst[k] || f->n == 0) continue;
    cudaError_t e = cudaMemcpy2D(dst[k], (size_t)dst_stride * 4, src[k]->p, (size_t)f->stride * 4, (size_t)f->n * 4,
                                 gs::kNumParams, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  }
  return GS_OK;
}

// Copy an image into the planar device layout: straight for a planar source, through the transpose
// kernel (and the staging buffer, for a host source) for an interleaved one.
static gs_status upload_image(Field* f, float* dst, const float* rgb, int on_device, bool hwc, size_t npix) {
  const size_t bytes = npix * 12;
  cudaError_t e;
  if (!hwc) {
    e = cudaMemcpyAsync(dst, rgb, bytes, on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, f->stream);
    return e == cudaSuccess ? GS_OK : fail(GS_ERR_CUDA, cudaGetErrorString(e));
  }
  const float* src = rgb;
  if (!on_device) {
    // Page-locked host memory the device can address: the layout kernel reads it over the host
    // link itself (NVLink-C2C on Grace-Blackwell), with no staging copy in device memory.
    cudaPointerAttributes pa;
    if (cudaPointerGetAttributes(&pa, rgb) == cudaSuccess && pa.type == cudaMemoryTypeHost && pa.devicePointer) {
      gs::launch_hwc_to_chw_host(static_cast<const float*>(pa.devicePointer), dst, (long long)npix, f->stream);
      e = cudaGetLastError();
      return e == cudaSuccess ? GS_OK : fail(GS_ERR_CUDA, std::string("image layout: ") + cudaGetErrorString(e));
    }
    cudaGetLastError();  // an unregistered pointer is not an error here
    gs_status s = f->hwc_stage.reserve(bytes, &f->own_bytes);
    if (s) return s;
    e = cudaMemcpyAsync(f->hwc_stage.p, rgb, bytes, cudaMemcpyHostToDevice, f->stream);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
    src = static_cast<const float*>(f->hwc_stage.p);
  }
  gs::launch_hwc_to_chw(src, dst, (long long)npix, f->stream);
  e = cudaGetLastError();
  return e == cudaSuccess ? GS_OK : fail(GS_ERR_CUDA, std::string("image layout: ") + cudaGetErrorString(e));
}

static gs_status add_image_impl(gs_field* ff, const gs_camera* cam, const float* rgb, int on_device, bool hwc,
                                const float* pts_xyz, const float* pts_rgb, int32_t n_pts, const int32_t* tracks,
                                int32_t* out_id) {
  Field* f = F(ff);
  if (!f || !cam || !rgb) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  if (n_pts < 0 || (n_pts > 0 && (!pts_xyz || !pts_rgb))) return fail(GS_ERR_INVALID_ARG, "bad sparse points");
  if (cam->width <= 0 || cam->height <= 0 || !(cam->fx > 0.f) || !(cam->fy > 0.f))
    return fail(GS_ERR_INVALID_ARG, "bad camera");
  if (f->images.size() >= 4096) return fail(GS_ERR_CAPACITY, "image registry full (4096)");
  const size_t npix = (size_t)cam->width * cam->height;
  const size_t img_bytes = npix * 3 * 4;
  const size_t stage_grow = (hwc && !on_device && f->hwc_stage.bytes < img_bytes) ? img_bytes - f->hwc_stage.bytes : 0;
  if (f->cfg.hbm_budget_bytes && f->bytes_in_use() + img_bytes + stage_grow > f->cfg.hbm_budget_bytes)
    return fail(GS_ERR_BUDGET, "registering the image would exceed hbm_budget_bytes");
  gs::Image im;
  im.cam = *cam;
  gs_status s = im.rgb.reserve(img_bytes, &f->own_bytes);
  if (s) return s;
  if ((s = upload_image(f, static_cast<float*>(im.rgb.p), rgb, on_device, hwc, npix))) {
    im.rgb.release(&f->own_bytes);
    return s;
  }
  cudaError_t e;
  if (tracks && n_pts > 0) {
    im.tracks.assign(tracks, tracks + n_pts);
    std::sort(im.tracks.begin(), im.tracks.end());
    im.tracks.erase(std::unique(im.tracks.begin(), im.tracks.end()), im.tracks.end());
  }
  const int id = (int)f->images.size();
  f->images.push_back(std::move(im));
  // overlap row / column
  for (auto& row : f->M) row.push_back(0.f);
  f->M.push_back(std::vector<float>(f->images.size(), 0.f));
  const auto& tn = f->images[id].tracks;
  for (int i = 0; i < id; ++i) {
    const auto& ti = f->images[i].tracks;
    if (ti.empty() || tn.empty()) continue;
    size_t a = 0, b = 0, shared = 0;
    while (a < ti.size() && b < tn.size()) {
      if (ti[a] < tn[b]) ++a;
      else if (ti[a] > tn[b]) ++b;
      else {
        ++shared;
        ++a;
        ++b;
      }
    }
    const float m = (float)shared / (float)std::min(ti.size(), tn.size());
    f->M[i][id] = m;
    f->M[id][i] = m;
  }
  // Field update (Sec. IV-B), on the device: points farther than the threshold from every earlier
  // sparse point become new Gaussians (3DGS initialisation); all of the image's points then join
  // the sparse set.
  float thr = f->cfg.add_dist_thresh > 0.f ? f->cfg.add_dist_thresh : 0.01f * f->scene_extent();
  if (!f->grid_ready) {
    f->grid_cell = std::max(thr, 1e-6f);
    f->grid_ready = true;
  }
  if (n_pts > 0) {
    if (!f->count_h && cudaMallocHost(&f->count_h, sizeof(unsigned)) != cudaSuccess) {
      f->count_h = nullptr;
      return fail(GS_ERR_OOM, "pinned allocation failed");
    }
    if ((s = f->reserve_points(f->n_points + n_pts)) || (s = f->new_rgb.reserve((size_t)n_pts * 12, &f->own_bytes)) ||
        (s = f->far_flags.reserve((size_t)n_pts * 4, &f->own_bytes)) ||
        (s = f->far_off.reserve((size_t)n_pts * 4, &f->own_bytes)) || (s = f->far_count.reserve(4, &f->own_bytes))) {
      if (out_id) *out_id = id;
      return s;
    }
    float* xyz_new = static_cast<float*>(f->pts_xyz.p) + 3 * f->n_points;
    cudaMemcpyAsync(xyz_new, pts_xyz, (size_t)n_pts * 12, cudaMemcpyHostToDevice, f->stream);
    cudaMemcpyAsync(f->new_rgb.p, pts_rgb, (size_t)n_pts * 12, cudaMemcpyHostToDevice, f->stream);
    const gs::PointGridDev g = f->grid_dev();
    const int ring = (int)std::min(16.f, std::max(1.f, std::ceil(thr / f->grid_cell)));
    unsigned* far = static_cast<unsigned*>(f->far_flags.p);
    unsigned* off = static_cast<unsigned*>(f->far_off.p);
    gs::launch_far_points(g, xyz_new, n_pts, thr * thr, ring, far, f->stream);
    f->insert_points(f->n_points, n_pts);
    gs::launch_scan_flags(far, n_pts, off, static_cast<unsigned*>(f->far_count.p), f->stream);
    cudaMemcpyAsync(f->count_h, f->far_count.p, sizeof(unsigned), cudaMemcpyDeviceToHost, f->stream);
    e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("field update: ") + cudaGetErrorString(e));
    const long long first_pt = f->n_points;
    f->n_points += n_pts;
    const unsigned fresh = *f->count_h;
    if (fresh > 0) {
      s = f->reserve_gaussians((long long)f->n + (long long)fresh);
      if (s) {
        if (out_id) *out_id = id;
        return s;
      }
      const double C0 = 0.5 * std::sqrt(1.0 / 3.14159265358979323846);
      gs::launch_init_gaussians(f->grid_dev(false), f->grid_dev(true), xyz_new, static_cast<const float*>(f->new_rgb.p), n_pts, first_pt, far,
                                off, static_cast<float*>(f->params.p), static_cast<float*>(f->adam_m.p),
                                static_cast<float*>(f->adam_v.p), f->stride, f->n, (float)std::log(0.1 / 0.9), C0,
                                f->stream);
      e = cudaStreamSynchronize(f->stream);
      if (e == cudaSuccess) e = cudaGetLastError();
      if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("field update: ") + cudaGetErrorString(e));
      f->n += (int)fresh;
    }
  } else {
    cudaStreamSynchronize(f->stream);
  }
  if (out_id) *out_id = id;
  return GS_OK;
}

gs_status gs_add_image(gs_field* f, const gs_camera* cam, const float* rgb_hwc, int rgb_on_device, const float* pts_xyz,
                       const float* pts_rgb, int32_t n_pts, const int32_t* pt_track_ids, int32_t* out_image_id) {
  gs::TraceRange trace("gs_add_image");
  return add_image_impl(f, cam, rgb_hwc, rgb_on_device, true, pts_xyz, pts_rgb, n_pts, pt_track_ids, out_image_id);
}

gs_status gs_add_image_chw(gs_field* f, const gs_camera* cam, const float* rgb_chw, int rgb_on_device,
                           const float* pts_xyz, const float* pts_rgb, int32_t n_pts, const int32_t* pt_track_ids,
                           int32_t* out_image_id) {
  gs::TraceRange trace("gs_add_image");
  return add_image_impl(f, cam, rgb_chw, rgb_on_device, false, pts_xyz, pts_rgb, n_pts, pt_track_ids, out_image_id);
}

static gs_status set_image_impl(gs_field* ff, int32_t id, const gs_camera* cam, const float* rgb, int on_device,
                                bool hwc) {
  Field* f = F(ff);
  if (!f || id < 0 || id >= (int)f->images.size()) return fail(GS_ERR_INVALID_ARG, "bad image id");
  gs::Image& im = f->images[id];
  if (cam) {
    if (cam->width != im.cam.width || cam->height != im.cam.height) return fail(GS_ERR_INVALID_ARG, "size change");
    im.cam = *cam;
  }
  if (rgb) {
    const size_t npix = (size_t)im.cam.width * im.cam.height;
    if (hwc && !on_device && f->cfg.hbm_budget_bytes && f->hwc_stage.bytes < npix * 12 &&
        f->bytes_in_use() + (npix * 12 - f->hwc_stage.bytes) > f->cfg.hbm_budget_bytes)
      return fail(GS_ERR_BUDGET, "the staging buffer would exceed hbm_budget_bytes");
    gs_status s = upload_image(f, static_cast<float*>(im.rgb.p), rgb, on_device, hwc, npix);
    if (s) return s;
  }
  return GS_OK;
}

gs_status gs_set_image(gs_field* f, int32_t id, const gs_camera* cam, const float* rgb_hwc, int rgb_on_device) {
  gs::TraceRange trace("gs_set_image");
  return set_image_impl(f, id, cam, rgb_hwc, rgb_on_device, true);
}

gs_status gs_set_image_chw(gs_field* f, int32_t id, const gs_camera* cam, const float* rgb_chw, int rgb_on_device) {
  gs::TraceRange trace("gs_set_image");
  return set_image_impl(f, id, cam, rgb_chw, rgb_on_device, false);
}

gs_status gs_select_neighbors(gs_field* ff, int32_t id, int32_t k, int32_t* out_ids, float* out_w, int32_t* out_n) {
  Field* f = F(ff);
  if (!f || id < 0 || id >= (int)f->images.size() || k < 0 || !out_ids) return fail(GS_ERR_INVALID_ARG, "bad arguments");
  std::vector<double> w;
  f->weights(id, w);
  std::vector<int> keys = f->key_images(w, k + 1);
  for (size_t q = 0; q < keys.size(); ++q) {
    out_ids[q] = keys[q];
    if (out_w) out_w[q] = (float)w[keys[q]];
  }
  if (out_n) *out_n = (int)keys.size();
  return GS_OK;
}

gs_status gs_optimize_step(gs_field* ff, const int32_t* ids, int32_t nv, float* out_loss) {
  gs::TraceRange trace("gs_optimize_step");
  Field* f = F(ff);
  if (!f || !ids) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  std::vector<int> v(ids, ids + nv);
  return f->step(v.data(), nv, out_loss);
}

gs_status gs_integrate(gs_field* ff, int32_t id, gs_integrate_stats* st) {
  gs::TraceRange trace("gs_integrate");
  Field* f = F(ff);
  if (!f || id < 0 || id >= (int)f->images.size()) return fail(GS_ERR_INVALID_ARG, "bad image id");
  int nk = 0;
  std::vector<int> slots = f->allocate(id, &nk);
  const int B = f->cfg.batch_views;
  std::vector<std::vector<int>> groups;
  for (size_t q = 0; q < slots.size(); q += B)
    groups.emplace_back(slots.begin() + q, slots.begin() + std::min(slots.size(), q + (size_t)B));
  const size_t chunk = f->cfg.async_steps > 0 ? (size_t)f->cfg.async_steps : 1;
  const unsigned long long pairs0 = f->sum_pairs;
  double loss_sum = 0;
  gs_status s = f->run_all(groups, chunk, &loss_sum);
  if (s) return s;
  if (st) {
    st->iterations = (int)slots.size();
    st->steps = (int)groups.size();
    st->key_images = nk;
    st->new_gaussians = 0;
    st->mean_loss = groups.empty() ? 0.0 : loss_sum / (double)groups.size();
    st->pairs = f->sum_pairs - pairs0;
  }
  return GS_OK;
}

gs_status gs_initial_training(gs_field* ff, int32_t iterations, int32_t max_steps, gs_integrate_stats* st) {
  gs::TraceRange trace("gs_initial_training");
  Field* f = F(ff);
  if (!f || iterations < 0 || max_steps <= 0) return fail(GS_ERR_INVALID_ARG, "bad arguments");
  if (f->images.empty()) return fail(GS_ERR_STATE, "no registered image");
  // views drawn uniformly by SplitMix64; 3DGS's exponential position-rate schedule over max_steps
  gs::SplitMix64 rng(f->cfg.seed ^ 0x5048415345310000ull);
  const int B = f->cfg.batch_views;
  const int n_img = (int)f->images.size();
  std::vector<std::vector<int>> groups;
  std::vector<double> lrs;
  for (int done = 0; done < iterations; done += B) {
    std::vector<int> ids;
    for (int k = 0; k < B && done + k < iterations; ++k) ids.push_back((int)rng.below((unsigned long long)n_img));
    const double u = std::min(1.0, (double)groups.size() / (double)max_steps);
    lrs.push_back(std::exp(std::log((double)f->cfg.eta0) * (1.0 - u) + std::log((double)f->cfg.etaf) * u));
    groups.push_back(std::move(ids));
  }
  const size_t chunk = f->cfg.async_steps > 0 ? (size_t)f->cfg.async_steps : 1;
  const unsigned long long pairs0 = f->sum_pairs;
  double loss_sum = 0;
  f->lr_override = &lrs;
  gs_status s = f->run_all(groups, chunk, &loss_sum);
  f->lr_override = nullptr;
  if (s) return s;
  if (st) {
    st->iterations = iterations;
    st->steps = (int)groups.size();
    st->key_images = 0;
    st->new_gaussians = 0;
    st->mean_loss = groups.empty() ? 0.0 : loss_sum / (double)groups.size();
    st->pairs = f->sum_pairs - pairs0;
  }
  return GS_OK;
}

gs_status gs_field_densify_stats(gs_field* ff, float* host_sum, float* host_count) {
  Field* f = F(ff);
  if (!f) return fail(GS_ERR_INVALID_ARG, "NULL field");
  cudaError_t e = cudaStreamSynchronize(f->stream);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  const float* d = static_cast<const float*>(f->dstat.p);
  if (f->n > 0 && host_sum && cudaMemcpy(host_sum, d, (size_t)f->n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(GS_ERR_CUDA, "reading the statistics failed");
  if (f->n > 0 && host_count &&
      cudaMemcpy(host_count, d + f->stride, (size_t)f->n * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(GS_ERR_CUDA, "reading the statistics failed");
  return GS_OK;
}

gs_status gs_field_corrupt_guard(gs_field* ff, int32_t index, char* out_name, int32_t name_cap) {
  Field* f = F(ff);
  if (!f) return fail(GS_ERR_INVALID_ARG, "field is NULL");
  cudaError_t e = cudaStreamSynchronize(f->stream);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  std::vector<gs::CanaryRef> allocated;
  for (const gs::CanaryRef& c : f->canary_refs())
    if (c.buf->p) allocated.push_back(c);
  if (index < 0 || index >= (int32_t)allocated.size())
    return fail(GS_ERR_INVALID_ARG, "index must be in 0.." + std::to_string((long long)allocated.size() - 1));
  const gs::DevBuf* b = allocated[(size_t)index].buf;
  // one guard word of the allocation (inside it: the bytes behind the usable size)
  e = cudaMemset(static_cast<char*>(b->p) + b->bytes + 4 * (index % 64), 0, 4);
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  if (out_name && name_cap > 0) {
    std::strncpy(out_name, allocated[(size_t)index].name, (size_t)name_cap - 1);
    out_name[name_cap - 1] = '\0';
  }
  return GS_OK;
}

gs_status gs_field_densify(gs_field* ff, const gs_densify_params* prm, gs_densify_result* out) {
  gs::TraceRange trace("gs_field_densify");
  Field* f = F(ff);
  if (!f || !prm) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  if (!(prm->grad_thresh >= 0.f) || !(prm->percent_dense > 0.f) || !(prm->min_opacity > 0.f) ||
      !(prm->min_opacity < 1.f) || !(prm->max_scale > 0.f))
    return fail(GS_ERR_INVALID_ARG, "bad densification parameters");
  cudaError_t e = cudaStreamSynchronize(f->stream);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  const int n = f->n;
  gs_densify_result res{n, n, 0, 0, 0};
  if (n > 0) {
    const double extent = (double)f->scene_extent();
    gs::DensifyThresholds th;
    th.grad = prm->grad_thresh;
    th.ls_dense = (float)std::log((double)prm->percent_dense * extent);
    th.ls_big = (float)std::log((double)prm->max_scale * extent);
    th.logit_min = (float)std::log((double)prm->min_opacity / (1.0 - (double)prm->min_opacity));
    th.ls_shrink = (float)std::log(1.6);
    th.seed_base = f->cfg.seed ^ ((unsigned long long)f->densify_round * 0x9E3779B97F4A7C15ull);
    // scratch: counts a, b, c; offsets a, b, c; totals (3) + candidates (2)
    gs_status s = f->dens_tmp.reserve((size_t)6 * n * 4 + 64, &f->own_bytes);
    if (s) return s;
    unsigned* tmp = static_cast<unsigned*>(f->dens_tmp.p);
    unsigned *ca = tmp, *cb = tmp + n, *cc = tmp + 2 * (size_t)n;
    unsigned *oa = tmp + 3 * (size_t)n, *ob = tmp + 4 * (size_t)n, *oc = tmp + 5 * (size_t)n;
    unsigned* tot = tmp + 6 * (size_t)n;  // [0..2] totals, [3..4] clone / split candidates
    cudaMemsetAsync(tot, 0, 64, f->stream);
    gs::launch_densify_count(n, f->stride, static_cast<const float*>(f->params.p), static_cast<const float*>(f->dstat.p),
                             th, ca, cb, cc, tot + 3, f->stream);
    gs::launch_scan_flags(ca, n, oa, tot, f->stream);
    gs::launch_scan_flags(cb, n, ob, tot + 1, f->stream);
    gs::launch_scan_flags(cc, n, oc, tot + 2, f->stream);
    unsigned h[5];
    e = cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, f->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(f->stream);
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("densify: ") + cudaGetErrorString(e));
    const long long n2 = (long long)h[0] + h[1] + h[2];
    const long long stride2 = std::max<long long>(1024, (std::max<long long>(n2, 1) + 31) / 32 * 32);
    const size_t bytes = (size_t)stride2 * gs::kNumParams * 4;
    if (f->cfg.hbm_budget_bytes && f->bytes_in_use() + 3 * bytes > f->cfg.hbm_budget_bytes + 3 * f->params.bytes)
      return fail(GS_ERR_BUDGET, "densification would exceed hbm_budget_bytes");
    gs::DevBuf np, nm, nv, nd;
    if ((s = np.reserve(bytes, &f->own_bytes)) || (s = nm.reserve(bytes, &f->own_bytes)) ||
        (s = nv.reserve(bytes, &f->own_bytes)) || (s = nd.reserve((size_t)stride2 * 8, &f->own_bytes))) {
      np.release(&f->own_bytes);
      nm.release(&f->own_bytes);
      nv.release(&f->own_bytes);
      nd.release(&f->own_bytes);
      return s;
    }
    cudaMemsetAsync(np.p, 0, bytes, f->stream);
    cudaMemsetAsync(nm.p, 0, bytes, f->stream);
    cudaMemsetAsync(nv.p, 0, bytes, f->stream);
    cudaMemsetAsync(nd.p, 0, (size_t)stride2 * 8, f->stream);
    gs::launch_densify_write(n, f->stride, static_cast<const float*>(f->params.p), static_cast<const float*>(f->adam_m.p),
                             static_cast<const float*>(f->adam_v.p), static_cast<const float*>(f->dstat.p), th, oa, ob,
                             oc, tot, (int)stride2, static_cast<float*>(np.p), static_cast<float*>(nm.p),
                             static_cast<float*>(nv.p), f->stream);
    e = cudaStreamSynchronize(f->stream);
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("densify: ") + cudaGetErrorString(e));
    f->params.release(&f->own_bytes);
    f->adam_m.release(&f->own_bytes);
    f->adam_v.release(&f->own_bytes);
    f->dstat.release(&f->own_bytes);
    f->params = np;
    f->adam_m = nm;
    f->adam_v = nv;
    f->dstat = nd;
    f->stride = (int)stride2;
    f->n = (int)n2;
    f->drop_graphs();
    f->sized_for_views = false;
    ++f->densify_round;
    res.n_after = n2;
    res.cloned = h[1];
    res.split = h[4];
    res.pruned = (long long)n + h[3] + 2ll * h[4] - n2 - h[4];  // results made minus results kept
  }
  if (out) *out = res;
  return GS_OK;
}

gs_status gs_render(gs_field* ff, const gs_camera* cam, float* out_rgb, float* out_T) {
  gs::TraceRange trace("gs_render");
  Field* f = F(ff);
  if (!f || !cam || !out_rgb) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  if (f->n <= 0) return fail(GS_ERR_STATE, "the field has no Gaussians");
  gs::Raster& R = *f->r;
  gs_status s;
  R.tiling = f->fixed_tiling();  // renders use the configured tiling, else the default one
  if ((s = R.set_views(cam, 1, nullptr))) return s;
  R.stride = f->stride;
  R.n = f->n;
  if ((s = R.ensure_records(f->stride)) || (s = f->ensure_step_buffers(R.n_pix)) || (s = R.ensure_instances(R.m_cap)))
    return s;
  if ((s = R.stage(f->stream))) return s;
  gs::StepParams& P = *R.sp_h;
  P.n = f->n;
  P.n_views = 1;
  for (int a = 0; a < 3; ++a) P.bg[a] = f->cfg.bg[a];
  P.adam = 0;
  R.reset_ledger(f->stream);
  R.upload(f->stream);
  if ((s = R.enqueue_forward_head(f->stream, static_cast<float*>(f->params.p), f->stride, true))) return s;
  if ((s = R.enqueue_forward_tail(f->stream, out_rgb, out_T, static_cast<unsigned*>(f->step_last.p), nullptr))) return s;
  f->sized_for_views = false;
  R.enqueue_readback(f->stream);
  cudaError_t e = cudaStreamSynchronize(f->stream);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, std::string("render: ") + cudaGetErrorString(e));
  return R.check_control();
}

gs_status gs_field_stats(const gs_field* ff, size_t* n_gaussians, size_t* bytes_in_use) {
  const Field* f = F(ff);
  if (!f) return fail(GS_ERR_INVALID_ARG, "NULL field");
  if (n_gaussians) *n_gaussians = (size_t)f->n;
  if (bytes_in_use) *bytes_in_use = f->bytes_in_use();
  return GS_OK;
}

gs_status gs_field_info_get(const gs_field* ff, gs_field_info* out) {
  const Field* f = F(ff);
  if (!f || !out) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  out->n_gaussians = f->n;
  out->capacity = f->stride;
  out->n_images = (int64_t)f->images.size();
  out->adam_step = f->adam_step;
  out->bytes_in_use = f->bytes_in_use();
  out->last_pairs = f->last_pairs;
  out->last_blended = f->last_blended;
  out->last_instances = (int64_t)f->last_instances;
  out->last_kernels = f->last_kernels;
  out->pad = 0;
  out->last_loss = f->last_loss;
  out->last_load_std = f->last_load_std;
  out->last_tiling = gs_tiling{f->last_tiling.tw, f->last_tiling.th, f->last_tiling.batch};
  out->pad2 = 0;
  out->last_run_ms = f->last_run_ms;
  out->last_run_steps = f->last_run_steps;
  out->last_h2d_bytes = f->last_h2d_bytes;
  out->last_d2h_bytes = f->last_d2h_bytes;
  return GS_OK;
}

gs_status gs_image_info(const gs_field* ff, int32_t id, int32_t* out_T, float* row, int32_t row_len) {
  const Field* f = F(ff);
  if (!f || id < 0 || id >= (int)f->images.size()) return fail(GS_ERR_INVALID_ARG, "bad image id");
  if (out_T) *out_T = f->images[id].T;
  if (row)
    for (int i = 0; i < row_len && i < (int)f->images.size(); ++i) row[i] = f->M[id][i];
  return GS_OK;
}

gs_status gs_schedule_plan(const gs_field_config* cfg, const float* Mh, const int32_t* Th, int32_t n,
                           int32_t new_id, int32_t* out_slots, int32_t* out_n_slots, int32_t* out_keys,
                           int32_t* out_n_keys, float* out_w, float* out_lr) {
  if (!cfg || !Mh || !Th || !out_slots || !out_n_slots || (out_keys && !out_n_keys))
    return fail(GS_ERR_INVALID_ARG, "gs_schedule_plan: a required pointer is NULL");
  if (n < 1 || new_id < 0 || new_id >= n || cfg->T_I < 1 || cfg->N_m < 1)
    return fail(GS_ERR_INVALID_ARG, "gs_schedule_plan: need n >= 1, 0 <= new_id < n, T_I >= 1, N_m >= 1");
  std::vector<std::vector<float>> M((size_t)n, std::vector<float>((size_t)n));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) M[i][j] = Mh[(size_t)i * n + j];
  const std::vector<int> T(Th, Th + n);
  const gs::Schedule sc{*cfg, M, T};
  int nk = 0;
  const std::vector<int> slots = sc.allocate(new_id, &nk);
  if ((int)slots.size() > cfg->T_I) return fail(GS_ERR_INVALID_ARG, "gs_schedule_plan: more slots than T_I");
  std::copy(slots.begin(), slots.end(), out_slots);
  *out_n_slots = (int32_t)slots.size();
  std::vector<double> w;
  sc.weights(new_id, w);
  if (out_keys) {
    const std::vector<int> keys = gs::Schedule::key_images(w, cfg->N_m);
    std::copy(keys.begin(), keys.end(), out_keys);
    *out_n_keys = (int32_t)keys.size();
  }
  for (int i = 0; i < n; ++i) {
    if (out_w) out_w[i] = (float)w[i];
    if (out_lr) out_lr[i] = (float)sc.lr_image(i);
  }
  return GS_OK;
}

gs_status gs_image_lr(const gs_field* ff, int32_t id, float* out_lr) {
  const Field* f = F(ff);
  if (!f || !out_lr || id < 0 || id >= (int)f->images.size()) return fail(GS_ERR_INVALID_ARG, "bad arguments");
  *out_lr = (float)f->lr_image(id);
  return GS_OK;
}

gs_status gs_field_snapshot(gs_field* ff) {
  gs::TraceRange trace("gs_field_snapshot");
  Field* f = F(ff);
  if (!f) return fail(GS_ERR_INVALID_ARG, "NULL field");
  const size_t bytes = (size_t)f->stride * gs::kNumParams * 4;
  if (f->cfg.hbm_budget_bytes && f->snap_p.bytes < bytes &&
      f->bytes_in_use() + 3 * (bytes - f->snap_p.bytes) > f->cfg.hbm_budget_bytes)
    return fail(GS_ERR_BUDGET, "a snapshot would exceed hbm_budget_bytes");
  gs_status s;
  if ((s = f->snap_p.reserve(bytes, &f->own_bytes)) || (s = f->snap_m.reserve(bytes, &f->own_bytes)) ||
      (s = f->snap_v.reserve(bytes, &f->own_bytes)))
    return s;
  if (bytes) {
    cudaMemcpyAsync(f->snap_p.p, f->params.p, bytes, cudaMemcpyDeviceToDevice, f->stream);
    cudaMemcpyAsync(f->snap_m.p, f->adam_m.p, bytes, cudaMemcpyDeviceToDevice, f->stream);
    cudaMemcpyAsync(f->snap_v.p, f->adam_v.p, bytes, cudaMemcpyDeviceToDevice, f->stream);
  }
  f->snap_n = f->n;
  f->snap_stride = f->stride;
  f->snap_step = f->adam_step;
  f->snap_T.clear();
  for (auto& im : f->images) f->snap_T.push_back(im.T);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  return GS_OK;
}

gs_status gs_field_restore(gs_field* ff) {
  gs::TraceRange trace("gs_field_restore");
  Field* f = F(ff);
  if (!f) return fail(GS_ERR_INVALID_ARG, "NULL field");
  if (f->snap_n < 0) return fail(GS_ERR_STATE, "no snapshot");
  // the field may have grown (stride) since the snapshot: copy rows with their pitches
  const gs::DevBuf* src[3] = {&f->snap_p, &f->snap_m, &f->snap_v};
  gs::DevBuf* dst[3] = {&f->params, &f->adam_m, &f->adam_v};
  for (int k = 0; k < 3; ++k) {
    if (f->snap_n == 0) continue;
    cudaMemcpy2DAsync(dst[k]->p, (size_t)f->stride * 4, src[k]->p, (size_t)f->snap_stride * 4, (size_t)f->snap_n * 4,
                      gs::kNumParams, cudaMemcpyDeviceToDevice, f->stream);
  }
  f->n = f->snap_n;
  f->adam_step = f->snap_step;
  cudaMemsetAsync(f->dstat.p, 0, (size_t)f->stride * 8, f->stream);  // statistics are not part of a snapshot
  for (size_t j = 0; j < f->images.size(); ++j) f->images[j].T = j < f->snap_T.size() ? f->snap_T[j] : 0;
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  return GS_OK;
}

gs_status gs_field_set_timing(gs_field* ff, int enable) {
  Field* f = F(ff);
  if (!f) return fail(GS_ERR_INVALID_ARG, "NULL field");
  f->r->timing = enable != 0;
  std::memset(f->r->acc_ms, 0, sizeof(f->r->acc_ms));
  f->r->timed_steps = 0;
  return GS_OK;
}

gs_status gs_field_autotune(gs_field* ff, const int32_t* ids, int32_t nv, int32_t reps, gs_autotune_result* out) {
  gs::TraceRange trace("gs_field_autotune");
  Field* f = F(ff);
  if (!f || !ids) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < nv; ++k)
    if (ids[k] < 0 || ids[k] >= (int)f->images.size()) return fail(GS_ERR_INVALID_ARG, "view id out of range");
  std::vector<int> v(ids, ids + std::max(nv, 0));
  return f->autotune(v.data(), nv, reps, out);
}

gs_status gs_autotune_clear(void) {
  gs::tune_cache().clear();
  return GS_OK;
}

gs_status gs_field_kernel_times(gs_field* ff, float out_ms[9], int64_t* out_steps) {
  Field* f = F(ff);
  if (!f || !out_ms) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  for (int k = 0; k < gs::kNumKernels; ++k) out_ms[k] = (float)f->r->acc_ms[k];
  if (out_steps) *out_steps = f->r->timed_steps;
  return GS_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------------------------
// Checkpoint / resume of a session in a file.
// ---------------------------------------------------------------------------------------------
namespace {

struct FileHeader {
  char magic[8];
  uint32_t version, cfg_bytes, camera_bytes, nparams;
};
constexpr char kMagic[8] = {'G', 'S', 'F', 'I', 'E', 'L', 'D', '1'};

struct File {
  FILE* f = nullptr;
  bool ok = true;
  ~File() {
    if (f) fclose(f);
  }
  void put(const void* p, size_t n) {
    if (ok && n && fwrite(p, 1, n, f) != n) ok = false;
  }
  void get(void* p, size_t n) {
    if (ok && n && fread(p, 1, n, f) != n) ok = false;
  }
  template <class T>
  void put(const T& v) {
    put(&v, sizeof(T));
  }
  template <class T>
  void get(T& v) {
    get(&v, sizeof(T));
  }
};

}  // namespace

extern "C" gs_status gs_field_save(gs_field* ff, const char* path) {
  gs::TraceRange trace("gs_field_save");
  Field* f = F(ff);
  if (!f || !path) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  cudaError_t e = cudaStreamSynchronize(f->stream);
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  File out;
  out.f = fopen(path, "wb");
  if (!out.f) return fail(GS_ERR_IO, std::string("cannot write ") + path);
  FileHeader h;
  std::memcpy(h.magic, kMagic, 8);
  h.version = 3;
  h.cfg_bytes = sizeof(gs_field_config);
  h.camera_bytes = sizeof(gs_camera);
  h.nparams = gs::kNumParams;
  out.put(h);
  out.put(f->cfg);
  out.put((int64_t)f->n);
  out.put((int64_t)f->adam_step);
  out.put((int32_t)f->images.size());
  std::vector<float> buf;
  for (const auto& im : f->images) {
    out.put(im.cam);
    out.put((int32_t)im.T);
    out.put((int64_t)im.tracks.size());
    out.put(im.tracks.data(), im.tracks.size() * sizeof(long long));
    buf.resize((size_t)3 * im.cam.width * im.cam.height);
    if (cudaMemcpy(buf.data(), im.rgb.p, buf.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(GS_ERR_CUDA, "reading an image back failed");
    out.put(buf.data(), buf.size() * 4);
  }
  for (const auto& row : f->M) out.put(row.data(), row.size() * 4);
  out.put((int64_t)f->n_points);
  out.put(f->grid_cell);
  out.put((int32_t)f->grid_ready);
  buf.resize((size_t)3 * f->n_points);
  if (f->n_points && cudaMemcpy(buf.data(), f->pts_xyz.p, buf.size() * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(GS_ERR_CUDA, "reading the sparse points back failed");
  out.put(buf.data(), buf.size() * 4);
  const gs::DevBuf* src[3] = {&f->params, &f->adam_m, &f->adam_v};
  buf.resize((size_t)gs::kNumParams * f->n);
  for (const gs::DevBuf* b : src) {
    if (f->n && cudaMemcpy2D(buf.data(), (size_t)f->n * 4, b->p, (size_t)f->stride * 4, (size_t)f->n * 4, gs::kNumParams,
                             cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(GS_ERR_CUDA, "reading the Gaussians back failed");
    out.put(buf.data(), buf.size() * 4);
  }
  out.put((int64_t)f->densify_round);
  buf.resize((size_t)2 * f->n);
  if (f->n && cudaMemcpy2D(buf.data(), (size_t)f->n * 4, f->dstat.p, (size_t)f->stride * 4, (size_t)f->n * 4, 2,
                           cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(GS_ERR_CUDA, "reading the densification statistics back failed");
  out.put(buf.data(), buf.size() * 4);
  if (!out.ok) return fail(GS_ERR_IO, std::string("short write to ") + path);
  return GS_OK;
}

extern "C" gs_status gs_field_load(const char* path, void* stream, gs_field** out_field) {
  gs::TraceRange trace("gs_field_load");
  if (!path || !out_field) return fail(GS_ERR_INVALID_ARG, "NULL argument");
  *out_field = nullptr;
  File in;
  in.f = fopen(path, "rb");
  if (!in.f) return fail(GS_ERR_IO, std::string("cannot read ") + path);
  FileHeader h;
  in.get(h);
  if (!in.ok || std::memcmp(h.magic, kMagic, 8) != 0 || h.version != 3 || h.cfg_bytes != sizeof(gs_field_config) ||
      h.camera_bytes != sizeof(gs_camera) || h.nparams != (uint32_t)gs::kNumParams)
    return fail(GS_ERR_IO, std::string(path) + " is not a saved field of this library");
  gs_field_config cfg;
  in.get(cfg);
  int64_t n = 0, adam_step = 0;
  int32_t n_images = 0;
  in.get(n);
  in.get(adam_step);
  in.get(n_images);
  if (!in.ok || n < 0 || n_images < 0 || n_images > 4096) return fail(GS_ERR_IO, "corrupt field file");
  gs_field* ffield = nullptr;
  gs_status s = gs_field_init(&cfg, stream, &ffield);
  if (s) return s;
  std::unique_ptr<Field> f(F(ffield));
  std::vector<float> buf;
  for (int32_t k = 0; k < n_images; ++k) {
    gs::Image im;
    int32_t T = 0;
    int64_t nt = 0;
    in.get(im.cam);
    in.get(T);
    in.get(nt);
    if (!in.ok || nt < 0 || im.cam.width <= 0 || im.cam.height <= 0) return fail(GS_ERR_IO, "corrupt field file");
    im.T = T;
    im.tracks.resize((size_t)nt);
    in.get(im.tracks.data(), (size_t)nt * sizeof(long long));
    buf.resize((size_t)3 * im.cam.width * im.cam.height);
    in.get(buf.data(), buf.size() * 4);
    if (!in.ok) return fail(GS_ERR_IO, "corrupt field file");
    if ((s = im.rgb.reserve(buf.size() * 4, &f->own_bytes))) return s;
    if (cudaMemcpy(im.rgb.p, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(GS_ERR_CUDA, "uploading an image failed");
    f->images.push_back(std::move(im));
  }
  f->M.assign(n_images, std::vector<float>(n_images, 0.f));
  for (auto& row : f->M) in.get(row.data(), row.size() * 4);
  int64_t n_points = 0;
  int32_t grid_ready = 0;
  in.get(n_points);
  in.get(f->grid_cell);
  in.get(grid_ready);
  if (!in.ok || n_points < 0) return fail(GS_ERR_IO, "corrupt field file");
  buf.resize((size_t)3 * n_points);
  in.get(buf.data(), buf.size() * 4);
  if (!in.ok) return fail(GS_ERR_IO, "corrupt field file");
  f->grid_ready = grid_ready != 0;
  if (n_points > 0) {
    if ((s = f->reserve_points(n_points))) return s;
    if (cudaMemcpy(f->pts_xyz.p, buf.data(), buf.size() * 4, cudaMemcpyHostToDevice) != cudaSuccess)
      return fail(GS_ERR_CUDA, "uploading the sparse points failed");
    f->n_points = n_points;
    f->insert_points(0, n_points);
  }
  if ((s = f->reserve_gaussians(std::max<int64_t>(n, 1)))) return s;
  gs::DevBuf* dst[3] = {&f->params, &f->adam_m, &f->adam_v};
  buf.resize((size_t)gs::kNumParams * n);
  for (gs::DevBuf* b : dst) {
    in.get(buf.data(), buf.size() * 4);
    if (!in.ok) return fail(GS_ERR_IO, "corrupt field file");
    cudaMemsetAsync(b->p, 0, (size_t)f->stride * gs::kNumParams * 4, f->stream);
    if (n && cudaMemcpy2DAsync(b->p, (size_t)f->stride * 4, buf.data(), (size_t)n * 4, (size_t)n * 4, gs::kNumParams,
                               cudaMemcpyHostToDevice, f->stream) != cudaSuccess)
      return fail(GS_ERR_CUDA, "uploading the Gaussians failed");
    cudaStreamSynchronize(f->stream);
  }
  int64_t densify_round = 0;
  in.get(densify_round);
  buf.resize((size_t)2 * n);
  in.get(buf.data(), buf.size() * 4);
  if (!in.ok || densify_round < 0) return fail(GS_ERR_IO, "corrupt field file");
  if (n && cudaMemcpy2D(f->dstat.p, (size_t)f->stride * 4, buf.data(), (size_t)n * 4, (size_t)n * 4, 2,
                        cudaMemcpyHostToDevice) != cudaSuccess)
    return fail(GS_ERR_CUDA, "uploading the densification statistics failed");
  f->densify_round = densify_round;
  f->n = (int)n;
  f->adam_step = adam_step;
  cudaError_t e = cudaStreamSynchronize(f->stream);
  if (e == cudaSuccess) e = cudaGetLastError();
  if (e != cudaSuccess) return fail(GS_ERR_CUDA, cudaGetErrorString(e));
  *out_field = reinterpret_cast<gs_field*>(f.release());
  return GS_OK;
}
