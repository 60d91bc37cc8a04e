// api.cpp -- the C ABI (include/shell.h): handles, batches, device memory, launches.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <numeric>
#include <vector>

#include "amg_setup.h"
#include "halo.h"
#include "host_mesh.h"
#include "internal.h"

using namespace shl;

namespace {

#define CK(call)                          \
  do {                                    \
    cudaError_t e_ = (call);              \
    if (e_ != cudaSuccess) {              \
      last_cuda_error() = e_;             \
      return SHELL_ERR_CUDA;              \
    }                                     \
  } while (0)

cudaError_t &last_cuda_error() {
  static thread_local cudaError_t e = cudaSuccess;
  return e;
}

int check_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return SHELL_ERR_NO_DEVICE;
  }
  int major = 0, minor = 0;
  if (cudaDeviceGetAttribute(&major, cudaDevAttrComputeCapabilityMajor, dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&minor, cudaDevAttrComputeCapabilityMinor, dev) != cudaSuccess) {
    cudaGetLastError();
    return SHELL_ERR_NO_DEVICE;
  }
  if (major != 10 || minor != 3) return SHELL_ERR_NO_DEVICE;
  return SHELL_OK;
}

// ---------------------------------------------------------------- device memory
struct Mem {
  shell_alloc_fn alloc = nullptr;
  shell_free_fn free = nullptr;
  void *user = nullptr;
  cudaStream_t st = nullptr;
  void *get(size_t bytes) const {
    if (bytes == 0) bytes = 256;
    if (alloc) return alloc(bytes, (void *)st, user);
    void *p = nullptr;
    if (cudaMallocAsync(&p, bytes, st) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    return p;
  }
  void put(void *p, size_t bytes) const {
    if (!p) return;
    if (free)
      free(p, bytes, (void *)st, user);
    else
      cudaFreeAsync(p, st);
  }
};

// carve one allocation into 256-byte aligned arrays: first pass sizes, second pass assigns
struct Carver {
  char *base = nullptr;
  size_t off = 0;
  template <typename T>
  T *take(size_t n) {
    off = (off + 255) & ~size_t(255);
    T *p = base ? reinterpret_cast<T *>(base + off) : nullptr;
    off += n * sizeof(T);
    return p;
  }
};

// gather lists of one matrix: device arrays carved from a block, then uploaded
void halo_take(Carver &C, const HostHalo &H, HaloDev &D) {
  D = HaloDev{};
  if (H.col.empty()) return;
  D.col = C.take<int32_t>(H.col.size());
  D.own = C.take<int32_t>(H.own.size());
  D.c16 = C.take<uint16_t>(H.c16.size());
  D.max = H.max;
}

cudaError_t halo_upload(const HostHalo &H, const HaloDev &D, cudaStream_t st) {
  if (H.col.empty()) return cudaSuccess;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(D.col, H.col.data(), 4 * H.col.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  if ((e = cudaMemcpyAsync(D.own, H.own.data(), 4 * H.own.size(), cudaMemcpyHostToDevice, st)) != cudaSuccess) return e;
  return cudaMemcpyAsync(D.c16, H.c16.data(), 2 * H.c16.size(), cudaMemcpyHostToDevice, st);
}

}  // namespace

struct shell_batch;

struct shell_handle {
  int nv = 0, nt = 0, ne = 0, model = 0;
  shell_material mat{};
  shell_options opt{};
  Mem mem;
  void *block = nullptr;
  size_t block_bytes = 0;
  Inst h{};                 // descriptor with device pointers
  Inst *d_inst = nullptr;   // device copy
  double *d_stage = nullptr;  // [2][V][3] staging for row-major state transfers
  double *d_energy = nullptr; // [4]
  double *d_forces = nullptr; // [V][3]
  shell_batch *batch = nullptr;  // user batch holding this handle
  int32_t slot = -1;
  shell_batch *solo = nullptr;   // private batch used by shell_step
  std::vector<Tile> tiles;       // force tiles of this instance (inst index filled by the batch)
  Tile *d_tiles = nullptr;       // the same tiles on the device (inst index 0 = d_inst)
  void *amg_block = nullptr;     // multigrid hierarchy (device), if any
  size_t amg_bytes = 0;
  int64_t vcycle_bytes = 0;      // algorithmic bytes of one FP32 V-cycle
  double est_iters = 64.0;       // scheduling estimate (PCG iterations per step)
  long long meas_ns = 0;         // longest device solve time of the last call's steps (0 = never run)
  int meas_team = 0;             // team size it ran with
  // longest solve time, with its team size, of each of the last kHist calls: the schedule plans for the
  // slowest of them, so that an instance whose step cost varies (one or two refinement rounds) is not
  // given a team sized for its cheap steps
  static constexpr int kHist = 4;
  long long hist_ns[kHist] = {0, 0, 0, 0};
  int hist_team[kHist] = {0, 0, 0, 0};
  int hist_n = 0;
  int64_t nnz = 0, nnz_pad = 0;
  InstStatus last_status{};
};

struct shell_batch {
  shell_options opt{};
  Mem mem;
  size_t budget = 0, used = 0;
  std::vector<shell_handle *> slots;
  bool dirty = true;
  bool solo = false;
  // device tables
  void *tbl = nullptr;
  size_t tbl_bytes = 0;
  Inst *d_insts = nullptr;
  Tile *d_tiles64 = nullptr;   // force tiles of FP64 instances
  int n_tiles64 = 0;
  Sched sched{};
  int grid = 0;
  int prec = 0;     // solve-kernel variant: 0 mixed, 1 FP64 only, 2 FP32-refinement only
  int n_teams = 0;
  int n_active = 0;
  InstStatus *d_status_out = nullptr;
  int32_t *d_abort_out = nullptr;
  long long *d_offs = nullptr;     // first row of each active instance in the packed state layout
  long long rows_total = 0;
  double *d_pack = nullptr;        // packed states [rows][3] x, then [rows][3] v (allocated on first use)
  size_t pack_bytes = 0;
  std::vector<int> active;   // slot ids in table order
  std::vector<cudaEvent_t> events;
  std::vector<float> step_ms;
  cudaGraphExec_t gexec = nullptr;
  bool graph_tried = false;
  bool profiling = false;
  int occ = 0;                 // CTAs per SM of the solve launch (0 = the occupancy maximum)
  bool cluster_off = false;    // set if a cluster launch was refused
  int policy = 0;              // 0 flat teams, 1 one-cluster teams
  int occ_launch = 3;          // occupancy variant of the current plan
  int chord_max = 1;           // solve launches per step (exact backward Euler: the largest nl_max)
  double plan_T = 0.0;         // makespan the current flat plan was built for (ns, or model units)
  double share_scale = 1.0;    // multiplier of the CTA share given to large instances
  std::vector<cudaEvent_t> pev;   // 3 per profiled step
  double kern_ms[2] = {0.0, 0.0};
  unsigned long long wait_ns = (unsigned long long)kMaxTeamWaitMs * 1000000ull;   // team-barrier wait bound
};

namespace {

// Device properties queried once (atomics: handles may be created on several threads; racing threads
// compute the same value).
// CTAs per SM of the solve variant compiled for `occ` (FP32: variants for 3, 4, 5; others one variant)
int blocks_per_sm_cached(int prec, int occ = 3) {
  static std::atomic<int> n[4][6] = {{-1, -1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1, -1}, {-1, -1, -1, -1, -1, -1},
                                     {-1, -1, -1, -1, -1, -1}};
  occ = std::max(1, std::min(5, occ));
  int v = n[prec][occ].load();
  if (v < 0) {
    v = std::max(1, solve_blocks_per_sm(prec, occ));
    n[prec][occ].store(v);
  }
  return v;
}
int max_occ(int prec) { return prec == 2 ? blocks_per_sm_cached(2, 5) : blocks_per_sm_cached(prec, 2); }
int max_clusters_cached(int prec) {
  static std::atomic<int> n[4] = {-1, -1, -1, -1};
  int v = n[prec].load();
  if (v < 0) {
    v = std::max(0, solve_max_clusters(prec, kCluster));
    n[prec].store(v);
  }
  return v;
}
int num_sms() {
  static std::atomic<int> n{-1};
  int v = n.load();
  if (v < 0) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
    n.store(v);
  }
  return v;
}

void destroy_graph(shell_batch *b) {
  if (b->gexec) {
    cudaGraphExecDestroy(b->gexec);
    b->gexec = nullptr;
  }
  b->graph_tried = false;
}

// The step kernel's variant with the Newton tangent also carries the projection of per-component constraints.
static bool uses_nt_variant(const Inst &I) { return (I.nl_newton && I.nl_max > 1) || I.fix != nullptr; }

// Build the force tile lists and the persistent-solve schedule for the resident instances.
int rebuild_tables(shell_batch *b) {
  destroy_graph(b);
  b->active.clear();
  for (size_t k = 0; k < b->slots.size(); ++k)
    if (b->slots[k]) b->active.push_back((int)k);
  const int n = (int)b->active.size();
  b->n_active = n;
  b->chord_max = 1;
  for (int k : b->active) b->chord_max = std::max(b->chord_max, b->slots[k]->h.nl_max);
  if (n == 0) {
    b->dirty = false;
    return SHELL_OK;
  }
  std::vector<Inst> insts(n);
  std::vector<Tile> t64;   // force tiles of the FP64 instances (FP32 ones evaluate forces in the step kernel)
  for (int k = 0; k < n; ++k) {
    shell_handle *h = b->slots[b->active[k]];
    insts[k] = h->h;
    if (h->h.precision != SHELL_FP64) continue;
    for (Tile t : h->tiles) {
      t.inst = k;
      t64.push_back(t);
    }
  }
  // ---- solve-kernel variant by the precisions present, then the schedule: teams of CTAs, each working
  // through a list of instances
  bool any64 = false, any32 = false, anynt = false;
  for (int k = 0; k < n; ++k) {
    const Inst &hk = b->slots[b->active[k]]->h;
    (hk.precision == SHELL_FP64 ? any64 : any32) = true;
    anynt = anynt || uses_nt_variant(hk);
  }
  // a batch with a Newton instance, or one with per-component constraints, runs the variant that carries the
  // Newton tangent and the projection
  b->prec = anynt ? 3 : (any64 && any32) ? 0 : (any64 ? 1 : 2);
  // default occupancy: the 3-CTA variant for FP32 (fewest spills), else the variant's maximum
  const int occ_def = b->prec == 2 ? blocks_per_sm_cached(2, 3) : max_occ(b->prec);
  const int occ = (b->occ > 0) ? std::min(b->occ, max_occ(b->prec)) : occ_def;
  b->occ_launch = occ;
  // team policy: flat (multi-CTA teams of any size, cooperative launch, global barriers) or clusters
  // (multi-CTA teams are exactly one 8-CTA cluster and use the hardware cluster barrier; non-cooperative)
  const bool use_clusters = b->policy == 1 && !b->cluster_off && max_clusters_cached(b->prec) > 0;
  const int CS = use_clusters ? kCluster : 0;
  int G = num_sms() * occ;
  if (CS) G = std::max(CS, std::min(G, max_clusters_cached(b->prec) * CS) / CS * CS);
  // Team-time model of an instance of B row blocks (chunks) on c CTAs: t(c) = w ceil(B/c)/B (1 + beta (c-1)).
  // Every CTA of a team takes its share of whole blocks in each phase, so the phase ends with the CTAs that
  // hold ceil(B/c) blocks: the time falls in steps, and the smallest c of a step is the one to use; beta is
  // the barrier overhead per extra CTA. w (the one-CTA time) is measured (the last solve time, divided by
  // the model's factor for the team it ran with) once the instance has run, else rows x iterations.
  constexpr double kBeta = 0.04;
  const double beta = kBeta * b->share_scale;
  auto cmax = [&](int k) { return std::max(1, b->slots[b->active[k]]->h.n_chunks); };
  auto factor = [&](int k, int c) {
    const double B = cmax(k);
    return std::ceil(B / c) / B * (1.0 + beta * (c - 1));
  };
  std::vector<double> work(n);
  bool measured = true;
  for (int k = 0; k < n; ++k) measured &= b->slots[b->active[k]]->meas_ns > 0;
  for (int k = 0; k < n; ++k) {
    shell_handle *h = b->slots[b->active[k]];
    if (measured) {
      work[k] = 0.0;
      for (int q = 0; q < std::min(h->hist_n, shell_handle::kHist); ++q) {
        const int c = std::max(1, std::min(cmax(k), h->hist_team[q]));
        work[k] = std::max(work[k], (double)h->hist_ns[q] / factor(k, c));
      }
    } else {
      work[k] = (double)h->nv * std::max(1.0, h->est_iters) * (h->h.amg_levels > 0 ? 6.0 : 1.0);
    }
  }
  std::vector<int> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::sort(order.begin(), order.end(), [&](int a, int c) { return work[a] > work[c]; });
  std::vector<int> team_size, team_of(n, -1);
  std::vector<std::vector<int>> team_inst;
  std::vector<int32_t> queue;   // one-CTA instances taken dynamically (flat policy)
  int used = 0;
  auto t_of = [&](int k, int c) { return work[k] * factor(k, c); };
  if (CS) {
    // one-cluster teams for instances that want at least half a cluster, single CTAs for the rest
    double total = 0.0;
    for (double w : work) total += w;
    const double share = total / G;
    for (int k : order) {
      if (work[k] / share < CS / 2.0) break;
      int left_small = 0;
      for (int q = 0; q < n; ++q)
        if (team_of[q] < 0 && q != k) ++left_small;
      if ((G - used - (left_small > 0 ? 1 : 0)) / CS * CS < CS) break;
      team_of[k] = (int)team_size.size();
      team_size.push_back(CS);
      team_inst.push_back({k});
      used += CS;
    }
  } else {
    // makespan T: instances slower than T on one CTA get the smallest team that meets T; the others are
    // packed first-fit-decreasing onto single CTAs of capacity T; bisect for the smallest T that fits G
    auto team_for = [&](int k, double T) {
      int c = 1;
      while (c < cmax(k) && t_of(k, c) > T) ++c;
      return c;
    };
    auto plan = [&](double T, std::vector<int> *sizes, std::vector<std::vector<int>> *bins) -> int {
      int need = 0;
      std::vector<double> load;
      std::vector<std::vector<int>> bl;
      for (int k : order) {
        if (t_of(k, 1) > T) {
          const int c = team_for(k, T);
          need += c;
          if (sizes) sizes->push_back(c);
        } else {
          size_t q = 0;
          while (q < load.size() && load[q] + t_of(k, 1) > T) ++q;
          if (q == load.size()) {
            load.push_back(0.0);
            bl.emplace_back();
          }
          load[q] += t_of(k, 1);
          bl[q].push_back(k);
        }
      }
      if (bins) *bins = bl;
      return need + (int)load.size();
    };
    double lo = 0.0, hi = 0.0;
    for (int k = 0; k < n; ++k) {
      double best = t_of(k, 1);
      for (int c = 2; c <= cmax(k); ++c) best = std::min(best, t_of(k, c));
      lo = std::max(lo, best);
      hi += work[k];
    }
    if (plan(lo, nullptr, nullptr) > G) {
      for (int it = 0; it < 60 && hi > lo * (1.0 + 1e-3); ++it) {
        const double mid = 0.5 * (lo + hi);
        (plan(mid, nullptr, nullptr) <= G ? hi : lo) = mid;
      }
    } else {
      hi = lo;
    }
    std::vector<int> sizes;
    std::vector<std::vector<int>> bins;
    plan(hi, &sizes, &bins);
    b->plan_T = measured ? hi : 0.0;
    int q = 0;
    for (int k : order) {
      if (t_of(k, 1) > hi) {
        team_of[k] = (int)team_size.size();
        team_size.push_back(sizes[q++]);
        team_inst.push_back({k});
        used += team_size.back();
      }
    }
    // the one-CTA instances are not bound to the bins the plan sized: they form a queue in decreasing work,
    // served by one-CTA workers (every CTA the multi-CTA teams leave, at least as many as the bins) and by the
    // CTAs of the multi-CTA teams once their instance is done, so that the estimates' errors even out
    for (int k : order)
      if (t_of(k, 1) <= hi) queue.push_back(k);
    const int workers = queue.empty() ? 0 : std::max((int)bins.size(), G - used);
    for (int w = 0; w < workers; ++w) {
      team_size.push_back(1);
      team_inst.push_back({});
      used += 1;
    }
  }
  if (CS) {
    // the rest: single-CTA teams, longest-processing-time first
    std::vector<int> small;
    for (int k : order)
      if (team_of[k] < 0) small.push_back(k);
    if (!small.empty()) {
      const int n1 = std::max(1, std::min((int)small.size(), G - used));
      const int first = (int)team_size.size();
      std::vector<double> load(n1, 0.0);
      for (int q = 0; q < n1; ++q) {
        team_size.push_back(1);
        team_inst.push_back({});
      }
      for (int k : small) {
        int best = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        load[best] += work[k];
        team_inst[first + best].push_back(k);
        team_of[k] = first + best;
      }
      used += n1;
    }
  }
  const int n_teams = (int)team_size.size();
  const int grid = CS ? (used + CS - 1) / CS * CS : used;   // whole clusters; spare CTAs return at once
  std::vector<int32_t> cta_team(grid, -1), cta_rank(grid, 0), tsize(n_teams), tptr(n_teams + 1, 0), tlist;
  int c = 0;
  for (int t = 0; t < n_teams; ++t) {
    tsize[t] = team_size[t];
    for (int r = 0; r < team_size[t]; ++r) {
      cta_team[c] = t;
      cta_rank[c] = r;
      ++c;
    }
    for (int k : team_inst[t]) tlist.push_back(k);
    tptr[t + 1] = (int32_t)tlist.size();
  }
  b->grid = grid;
  b->n_teams = n_teams;
  // ---- one device table block
  Carver cv;
  auto layout = [&](Carver &C) {
    b->d_insts = C.take<Inst>(n);
    b->d_tiles64 = C.take<Tile>(t64.size());
    b->sched.cta_team = C.take<int32_t>(grid);
    b->sched.cta_rank = C.take<int32_t>(grid);
    b->sched.team_size = C.take<int32_t>(n_teams);
    b->sched.team_ptr = C.take<int32_t>(n_teams + 1);
    b->sched.team_list = C.take<int32_t>(tlist.size());
    b->sched.bar = C.take<unsigned int>((size_t)kBarWords * n_teams);
    b->sched.abort_flag = C.take<int32_t>(1);
    b->sched.cluster_ok = C.take<int32_t>(grid / (CS ? CS : 1) + 1);
    b->sched.queue = C.take<int32_t>(std::max<size_t>(1, queue.size()));
    b->sched.queue_ctr = C.take<unsigned int>(1);
    b->d_status_out = C.take<InstStatus>(n);
    b->d_abort_out = C.take<int32_t>(1);
    b->d_offs = C.take<long long>(n + 1);
  };
  layout(cv);
  if (cv.off > b->tbl_bytes) {
    if (b->tbl) b->mem.put(b->tbl, b->tbl_bytes);
    b->tbl_bytes = cv.off + 4096;
    b->tbl = b->mem.get(b->tbl_bytes);
    if (!b->tbl) {
      b->tbl_bytes = 0;
      return SHELL_ERR_OOM;
    }
  }
  Carver real;
  real.base = (char *)b->tbl;
  layout(real);
  b->sched.n_ctas = grid;
  b->sched.cluster = CS;
  cudaStream_t st = b->mem.st;
  CK(cudaMemcpyAsync(b->d_insts, insts.data(), sizeof(Inst) * n, cudaMemcpyHostToDevice, st));
  if (!t64.empty()) CK(cudaMemcpyAsync(b->d_tiles64, t64.data(), sizeof(Tile) * t64.size(), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(b->sched.cta_team, cta_team.data(), 4 * grid, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(b->sched.cta_rank, cta_rank.data(), 4 * grid, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(b->sched.team_size, tsize.data(), 4 * n_teams, cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(b->sched.team_ptr, tptr.data(), 4 * (n_teams + 1), cudaMemcpyHostToDevice, st));
  CK(cudaMemcpyAsync(b->sched.team_list, tlist.data(), 4 * tlist.size(), cudaMemcpyHostToDevice, st));
  b->sched.n_queue = (int32_t)queue.size();
  if (!queue.empty())
    CK(cudaMemcpyAsync(b->sched.queue, queue.data(), 4 * queue.size(), cudaMemcpyHostToDevice, st));
  std::vector<long long> offs(n + 1, 0);
  for (int k = 0; k < n; ++k) offs[k + 1] = offs[k] + b->slots[b->active[k]]->nv;
  b->rows_total = offs[n];
  CK(cudaMemcpyAsync(b->d_offs, offs.data(), sizeof(long long) * (n + 1), cudaMemcpyHostToDevice, st));
  CK(cudaMemsetAsync(b->sched.bar, 0, sizeof(unsigned int) * kBarWords * n_teams, st));
  CK(cudaMemsetAsync(b->sched.abort_flag, 0, sizeof(int32_t), st));
  CK(cudaStreamSynchronize(st));   // host vectors above go out of scope
  b->n_tiles64 = (int)t64.size();
  b->dirty = false;
  return SHELL_OK;
}

// the solve launch; if the driver refuses the cluster launch, fall back to plain global team barriers (the
// team layout stays valid: whole-cluster teams become flat global-barrier teams)
cudaError_t solve_launch(shell_batch *b, cudaStream_t st, int chord_k) {
  b->sched.chord_k = chord_k;
  b->sched.wait_ns = b->wait_ns;
  if (b->sched.n_queue > 0) {   // the queue of one-CTA instances starts at its head in every launch
    cudaError_t e = cudaMemsetAsync(b->sched.queue_ctr, 0, sizeof(unsigned int), st);
    if (e != cudaSuccess) return e;
  }
  cudaError_t e = launch_solve(b->d_insts, b->sched, b->grid, b->prec, b->occ_launch, st);
  if (e != cudaSuccess && b->sched.cluster > 0) {
    cudaGetLastError();
    b->cluster_off = true;
    b->sched.cluster = 0;
    e = launch_solve(b->d_insts, b->sched, b->grid, b->prec, b->occ_launch, st);
  }
  return e;
}

// one step: one persistent launch (forces, right-hand side, solve, commit of every FP32-refinement instance;
// FP64 instances take their forces from a force launch just before it), repeated for the chord iterations of
// exact backward-Euler instances (instances whose step is done skip the later launches)
int launch_step(shell_batch *b) {
  cudaStream_t st = b->mem.st;
  for (int k = 0; k < b->chord_max; ++k) {
    CK(launch_forces(b->d_insts, b->d_tiles64, b->n_tiles64, 0, 0, st, k));
    CK(solve_launch(b, st, k));
  }
  return SHELL_OK;
}

// capture one step into a CUDA graph (falls back to direct launches if capture is refused)
void try_capture(shell_batch *b) {
  b->graph_tried = true;
  cudaStream_t st = b->mem.st;
  if (st == nullptr) return;   // the legacy default stream cannot be captured
  cudaGraph_t g = nullptr;
  if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
    cudaGetLastError();
    return;
  }
  int rc = launch_step(b);
  cudaError_t e = cudaStreamEndCapture(st, &g);
  if (rc != SHELL_OK || e != cudaSuccess || !g) {
    cudaGetLastError();
    if (g) cudaGraphDestroy(g);
    return;
  }
  if (cudaGraphInstantiate(&b->gexec, g, 0) != cudaSuccess) {
    cudaGetLastError();
    b->gexec = nullptr;
  }
  cudaGraphDestroy(g);
}

// Device address of a host buffer that the GPU can read and write in place: page-locked memory
// (cudaHostAlloc, cudaHostRegister, torch's pinned tensors) is mapped into the device's address space under
// unified addressing. Null for pageable memory, or memory not mapped for the current device.
static double *mapped_host(const void *p) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? static_cast<double *>(a.devicePointer) : nullptr;
}

// Packed state copies of the resident instances, enqueued on the batch's stream (no synchronisation): with xin,
// host -> device and unpack; else pack and device -> host into x, v. The tables must be current.
// Page-locked host buffers are read (written) in place by the unpack (pack) kernel over the host link, with
// no staging copy; pageable ones go through a device staging buffer and two copies each way.
static int enqueue_states(shell_batch *b, double *x, double *v, const double *xin, const double *vin) {
  cudaStream_t st = b->mem.st;
  {
    double *mx = mapped_host(xin ? xin : x), *mv = mapped_host(xin ? vin : v);
    if (mx && mv) {
      CK(launch_pack_states(b->d_insts, b->n_active, b->d_offs, b->rows_total, mx, mv, xin ? 1 : 0, st));
      return SHELL_OK;
    }
  }
  const size_t n3 = 3 * (size_t)b->rows_total;
  const size_t n3a = (n3 + 1) & ~size_t(1);   // v starts on a 16-byte boundary (vector state kernel)
  const size_t need = 8 * (n3a + n3);
  if (b->pack_bytes < need) {
    if (b->d_pack) b->mem.put(b->d_pack, b->pack_bytes);
    b->d_pack = (double *)b->mem.get(need);
    b->pack_bytes = b->d_pack ? need : 0;
    if (!b->d_pack) return SHELL_ERR_OOM;
  }
  double *dx = b->d_pack, *dv = b->d_pack + n3a;
  if (xin) {
    CK(cudaMemcpyAsync(dx, xin, 8 * n3, cudaMemcpyHostToDevice, st));
    CK(cudaMemcpyAsync(dv, vin, 8 * n3, cudaMemcpyHostToDevice, st));
    CK(launch_pack_states(b->d_insts, b->n_active, b->d_offs, b->rows_total, dx, dv, 1, st));
  } else {
    CK(launch_pack_states(b->d_insts, b->n_active, b->d_offs, b->rows_total, dx, dv, 0, st));
    CK(cudaMemcpyAsync(x, dx, 8 * n3, cudaMemcpyDeviceToHost, st));
    CK(cudaMemcpyAsync(v, dv, 8 * n3, cudaMemcpyDeviceToHost, st));
  }
  return SHELL_OK;
}

// Step the batch n_steps times. xin/vin (host [rows][3], both or neither): states copied in before the steps;
// xout/vout: states copied out after them; all enqueued on the batch's stream ahead of one synchronisation.
int batch_step(shell_batch *b, int n_steps, shell_step_stats *stats, const double *xin = nullptr,
               const double *vin = nullptr, double *xout = nullptr, double *vout = nullptr) {
  if (n_steps < 0) return SHELL_ERR_INVALID_ARG;
  if (b->dirty) {
    int rc = rebuild_tables(b);
    if (rc != SHELL_OK) return rc;
  }
  const int n = b->n_active;
  if (n == 0 || n_steps == 0) {
    if (n > 0 && xin) {
      int rc = enqueue_states(b, nullptr, nullptr, xin, vin);
      if (rc != SHELL_OK) return rc;
    }
    if (n > 0 && xout) {
      int rc = enqueue_states(b, xout, vout, nullptr, nullptr);
      if (rc != SHELL_OK) return rc;
    }
    if (n > 0 && (xin || xout)) CK(cudaStreamSynchronize(b->mem.st));
    if (stats)
      for (size_t k = 0; k < b->slots.size(); ++k) stats[k] = shell_step_stats{0, 0, 0, SHELL_OK, 0, 0.0, 0, 0.0, 0, 0};
    return SHELL_OK;
  }
  cudaStream_t st = b->mem.st;
  // statuses before the call (cumulative counters)
  std::vector<InstStatus> before(n), after(n);
  for (int k = 0; k < n; ++k) before[k] = b->slots[b->active[k]]->last_status;
  if (!b->graph_tried) try_capture(b);
  if (xin) {   // after the capture, which records only the step
    int rc = enqueue_states(b, nullptr, nullptr, xin, vin);
    if (rc != SHELL_OK) return rc;
  }
  const int n_ev = std::min(n_steps, 4096) + 1;
  while ((int)b->events.size() < n_ev) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    b->events.push_back(e);
  }
  const int ev_stride = (n_steps + n_ev - 2) / (n_ev - 1);
  int ev = 0;
  CK(cudaEventRecord(b->events[ev++], st));
  // profiled steps: events around the force launches and the solve launch of every chord iteration
  const int n_prof = b->profiling ? std::min(n_steps, std::max(1, 4096 / b->chord_max)) : 0;
  const int pev_per_step = 3 * b->chord_max;
  while ((int)b->pev.size() < pev_per_step * n_prof) {
    cudaEvent_t e;
    CK(cudaEventCreate(&e));
    b->pev.push_back(e);
  }
  for (int s = 0; s < n_steps; ++s) {
    if (s < n_prof) {
      for (int k = 0; k < b->chord_max; ++k) {
        const int e0 = pev_per_step * s + 3 * k;
        CK(cudaEventRecord(b->pev[e0], st));
        CK(launch_forces(b->d_insts, b->d_tiles64, b->n_tiles64, 0, 0, st, k));   // FP64 instances only
        CK(cudaEventRecord(b->pev[e0 + 1], st));
        CK(solve_launch(b, st, k));
        CK(cudaEventRecord(b->pev[e0 + 2], st));
      }
    } else if (b->gexec) {
      CK(cudaGraphLaunch(b->gexec, st));
    } else {
      int rc = launch_step(b);
      if (rc != SHELL_OK) return rc;
    }
    if ((s + 1) % ev_stride == 0 && ev < n_ev) CK(cudaEventRecord(b->events[ev++], st));
  }
  if (xout) {
    int rc = enqueue_states(b, xout, vout, nullptr, nullptr);
    if (rc != SHELL_OK) return rc;
  }
  CK(launch_gather_status(b->d_insts, n, b->d_status_out, b->sched.abort_flag, b->d_abort_out, st));
  int32_t aborted = 0;
  CK(cudaMemcpyAsync(after.data(), b->d_status_out, sizeof(InstStatus) * n, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(&aborted, b->d_abort_out, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  b->kern_ms[0] = b->kern_ms[1] = 0.0;
  for (int s = 0; s < n_prof * b->chord_max; ++s) {
    float f = 0.f, v = 0.f;
    cudaEventElapsedTime(&f, b->pev[3 * s], b->pev[3 * s + 1]);
    cudaEventElapsedTime(&v, b->pev[3 * s + 1], b->pev[3 * s + 2]);
    b->kern_ms[0] += f;
    b->kern_ms[1] += v;
  }
  b->step_ms.clear();
  for (int k = 1; k < ev; ++k) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, b->events[k - 1], b->events[k]);
    b->step_ms.push_back(ms / ev_stride);
  }
  int first_err = SHELL_OK;
  if (aborted) {
    first_err = SHELL_ERR_TIMEOUT;
    CK(cudaMemsetAsync(b->sched.bar, 0, sizeof(unsigned int) * kBarWords * b->n_teams, st));
    CK(cudaMemsetAsync(b->sched.abort_flag, 0, sizeof(int32_t), st));
    CK(cudaStreamSynchronize(st));
  }
  if (stats)
    for (size_t k = 0; k < b->slots.size(); ++k) stats[k] = shell_step_stats{0, 0, 0, SHELL_OK, 0, 0.0, 0, 0.0, 0, 0};
  for (int k = 0; k < n; ++k) {
    shell_handle *h = b->slots[b->active[k]];
    const InstStatus &a = after[k];
    const InstStatus &z = before[k];
    h->last_status = a;
    const int done = a.steps_done - z.steps_done;
    if (a.err != SHELL_OK && first_err == SHELL_OK) first_err = a.err;
    if (done > 0) {
      const double it = double(a.total_iters - z.total_iters + 2 * (a.total_rounds - z.total_rounds)) / done;
      h->est_iters = std::max(1.0, it);
      // results do not depend on the schedule, so re-plan freely when the work estimate moved: on the first
      // measurement, and when the measured solve time leaves the planned makespan (below)
      const bool first_meas = h->meas_ns == 0;
      h->meas_ns = std::max(a.max_ns, a.last_ns);
      h->meas_team = a.team_size;
      h->hist_ns[h->hist_n % shell_handle::kHist] = h->meas_ns;
      h->hist_team[h->hist_n % shell_handle::kHist] = a.team_size;
      h->hist_n++;
      if (first_meas) b->dirty = true;
      // by more than the timing noise
      if (b->policy == 0 && b->plan_T > 0 && h->meas_ns > 1.05 * b->plan_T) b->dirty = true;
    }
    if (stats) {
      shell_step_stats &o = stats[b->active[k]];
      o.steps_done = done;
      o.pcg_iterations = a.last_iters;
      o.refine_rounds = a.last_rounds;
      o.status = a.err;
      o.total_pcg_iterations = a.total_iters - z.total_iters;
      o.rel_residual = a.rel_res;
      o.total_refine_rounds = a.total_rounds - z.total_rounds;
      o.last_solve_us = a.last_ns * 1e-3;
      o.team_ctas = a.team_size;
      o.nl_iterations = h->h.nl_max > 1 ? a.nl_iters : 0;
    }
  }
  return first_err;
}

int batch_new(const shell_options *opt, size_t budget, bool solo, shell_batch **out) {
  shell_batch *b = new (std::nothrow) shell_batch();
  if (!b) return SHELL_ERR_OOM;
  b->opt = *opt;
  b->mem.alloc = opt->alloc;
  b->mem.free = opt->free;
  b->mem.user = opt->alloc_user;
  b->mem.st = (cudaStream_t)opt->cuda_stream;
  b->budget = budget;
  b->solo = solo;
  *out = b;
  return SHELL_OK;
}

void batch_free(shell_batch *b) {
  if (!b) return;
  if (b->d_pack) b->mem.put(b->d_pack, b->pack_bytes);
  destroy_graph(b);
  for (cudaEvent_t e : b->events) cudaEventDestroy(e);
  for (cudaEvent_t e : b->pev) cudaEventDestroy(e);
  if (b->tbl) b->mem.put(b->tbl, b->tbl_bytes);
  for (shell_handle *h : b->slots)
    if (h && !b->solo) {
      h->batch = nullptr;
      h->slot = -1;
    }
  delete b;
}

void fill_default_tolerances(shell_options *o) {
  if (!(o->pcg_rtol > 0.0)) o->pcg_rtol = (o->precision == SHELL_FP64) ? 1e-13 : 1e-6;
  // FP32 refinement target: below 3e-7 of ||b|| the FP32 force rounding, not the solve, sets the error against
  // FP64 (batch256, 100 steps: max rel_x 2.2e-7 at targets 1e-8, 1e-7 and 3e-7 alike), so tighter targets
  // only cost inner iterations (12.1 -> 8.7 per step from 1e-8 to 3e-7)
  if (!(o->refine_rtol > 0.0)) o->refine_rtol = 3e-7;
  if (o->pcg_max_it <= 0) o->pcg_max_it = 20000;
  if (o->refine_max <= 0) o->refine_max = 20;
}

bool planar(const double *X, int nv, const int32_t *tris, int nt) {
  // normal of the largest triangle; every vertex within 1e-9 * extent of its plane
  double best = -1.0, n[3] = {0, 0, 1};
  const double *o = X;
  for (int t = 0; t < nt; ++t) {
    const double *a = X + 3 * tris[3 * t], *b = X + 3 * tris[3 * t + 1], *c = X + 3 * tris[3 * t + 2];
    double u[3] = {b[0] - a[0], b[1] - a[1], b[2] - a[2]}, v[3] = {c[0] - a[0], c[1] - a[1], c[2] - a[2]};
    double w[3] = {u[1] * v[2] - u[2] * v[1], u[2] * v[0] - u[0] * v[2], u[0] * v[1] - u[1] * v[0]};
    double l = std::sqrt(w[0] * w[0] + w[1] * w[1] + w[2] * w[2]);
    if (l > best) {
      best = l;
      n[0] = w[0] / l;
      n[1] = w[1] / l;
      n[2] = w[2] / l;
      o = a;
    }
  }
  double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300};
  for (int i = 0; i < nv; ++i)
    for (int c = 0; c < 3; ++c) {
      lo[c] = std::min(lo[c], X[3 * i + c]);
      hi[c] = std::max(hi[c], X[3 * i + c]);
    }
  double ext = std::max(hi[0] - lo[0], std::max(hi[1] - lo[1], hi[2] - lo[2]));
  for (int i = 0; i < nv; ++i) {
    double d = (X[3 * i] - o[0]) * n[0] + (X[3 * i + 1] - o[1]) * n[1] + (X[3 * i + 2] - o[2]) * n[2];
    if (std::fabs(d) > 1e-9 * ext) return false;
  }
  return true;
}

std::vector<double> to_soa(const double *aos, int nv) {
  std::vector<double> s((size_t)3 * nv);
  for (int i = 0; i < nv; ++i)
    for (int c = 0; c < 3; ++c) s[(size_t)c * nv + i] = aos[3 * i + c];
  return s;
}

// Multigrid preconditioner: download the assembled FP64 matrix, build the smoothed-aggregation hierarchy
// on the host (the matrix is constant, so this happens once) and upload its levels: the transfers with the
// smoother folded in (Ps in SELL-32, Rs with 4 lanes per row), the coarse operators with 4 lanes per row,
// the dense operator of the coarse end of the cycle, and (FP32 instances) the gather lists of every product.
// Per-component constraints (fixb: fixed-component bits per vertex, empty if none has fixed and free ones): the
// hierarchy is built from A with the diagonal of each such vertex doubled. A itself can be nearly singular then
// (with nothing pinned, a rigid motion costs only its mass), and a cycle of A amplifies those motions, which the
// projected system has removed; the doubled diagonal ties the constrained vertices down instead. Level 0 then
// carries that matrix's values, and the instance's inverse diagonal (Jacobi, and the level-0 pre-smoothing
// done in the residual and update phases) becomes its own, so the cycle stays symmetric.
int setup_amg(shell_handle *h, const HostTopo &T, int mode, bool stage, const std::vector<uint8_t> &fixb) {
  Inst &I = h->h;
  cudaStream_t st = h->mem.st;
  if (mode == SHELL_PRECOND_JACOBI) return SHELL_OK;
  const int nv = I.nv;
  const size_t nnz_pad = (size_t)T.sl_ptr[T.n_slices];
  std::vector<double> val(nnz_pad), mass(nv);
  CK(cudaMemcpyAsync(val.data(), I.val64, 8 * nnz_pad, cudaMemcpyDeviceToHost, st));
  CK(cudaMemcpyAsync(mass.data(), I.mass, 8 * (size_t)nv, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  HostCsr A;
  A.n = A.m = nv;
  A.ptr = T.row_ptr;
  A.col.resize(T.row_ptr[nv]);
  A.val.resize(T.row_ptr[nv]);
  std::vector<double> q;
  for (int r = 0; r < nv; ++r) {
    const int s = r / 32, l = r % 32;
    for (int k = 0; k < T.row_ptr[r + 1] - T.row_ptr[r]; ++k) {
      const int pos = T.sl_ptr[s] + 32 * k + l;
      A.col[T.row_ptr[r] + k] = T.sl_col[pos];
      A.val[T.row_ptr[r] + k] = val[pos];
    }
    const double d = val[T.diag_pos[r]];
    if (mass[r] > 0 && T.row_ptr[r + 1] - T.row_ptr[r] > 1) q.push_back((d - mass[r]) / mass[r]);
  }
  if (mode == SHELL_PRECOND_AUTO) {
    if (nv < 256 || q.empty()) return SHELL_OK;
    std::nth_element(q.begin(), q.begin() + q.size() / 2, q.end());
    if (q[q.size() / 2] <= 30.0) return SHELL_OK;
  }
  bool own0 = false;   // level 0 differs from the step matrix (doubled diagonals)
  for (int r = 0; r < (int)fixb.size(); ++r) {
    if (fixb[r] == 0 || fixb[r] == 7) continue;
    for (int k = A.ptr[r]; k < A.ptr[r + 1]; ++k)
      if (A.col[k] == r) A.val[k] *= 2.0;
    val[T.diag_pos[r]] *= 2.0;
    own0 = true;
  }
  HostAmg H;
  build_amg(A, &H);
  const int L = (int)H.levels.size();
  if (L < 2) return SHELL_OK;
  // one V(1,1) cycle reads every level operator above the dense level, Ps and Rs once (8 B per FP32
  // nonzero with its column); per row of level vectors (16 B each, AoS float4) the down step reads b, x, the
  // row sum and writes r, the up step reads x, r, D^-1 and writes y, and the level above writes b and x:
  // 136 B; the dense operator (or the dense coarsest inverse) once
  const int top = H.dense_level > 0 ? H.dense_level : L - 1;
  h->vcycle_bytes = 0;
  for (int l = 0; l < top; ++l) {
    const HostAmgLevel &V = H.levels[l];
    h->vcycle_bytes += 8 * (int64_t)V.A.val.size() + 136 * (int64_t)V.A.n;
    h->vcycle_bytes += 8 * (int64_t)(V.Ps.val.size() + V.Rs.val.size());
  }
  h->vcycle_bytes += 136 * (int64_t)H.levels[top].A.n;
  h->vcycle_bytes += 4 * (int64_t)(H.dense_level > 0 ? H.dense.size() : H.coarse_inv.size());
  std::vector<HostSell> As(L), Ps(L), Rs(L);
  for (int l = 0; l < L; ++l) {
    if (l > 0) As[l] = to_sell4(H.levels[l].A);
    if (l < L - 1) {
      Ps[l] = to_sell(H.levels[l].Ps);
      Rs[l] = to_sell4(H.levels[l].Rs);
    }
  }
  // gather lists for the FP32 products (level 0 shares the instance's)
  const bool stage32 = stage && I.precision != SHELL_FP64;
  std::vector<HostHalo> Ha(L), Hp(L), Hr(L);
  for (int l = 0; stage32 && l < L; ++l) {
    const HostAmgLevel &V = H.levels[l];
    if (l > 0) build_halo(V.A.n, V.A.n, As[l].sl_ptr, As[l].sl_col, V.A.ptr, true, &Ha[l], 4);
    if (l < L - 1) {
      build_halo(V.Ps.n, V.Ps.m, Ps[l].sl_ptr, Ps[l].sl_col, V.Ps.ptr, false, &Hp[l]);
      build_halo(V.Rs.n, V.Rs.m, Rs[l].sl_ptr, Rs[l].sl_col, V.Rs.ptr, false, &Hr[l], 4);
    }
  }
  const int nc = H.levels[L - 1].A.n;
  std::vector<AmgDev> lev(L);
  double *cinv64 = nullptr, *dense64 = nullptr;
  float *cinv32 = nullptr, *dense32 = nullptr;
  AmgDev *d_lev = nullptr;
  auto layout = [&](Carver &C) {
    for (int l = 0; l < L; ++l) {
      AmgDev &D = lev[l];
      const int n = H.levels[l].A.n;
      D.n = n;
      D.n_next = (l < L - 1) ? H.levels[l + 1].A.n : 0;
      D.omega = H.levels[l].omega;
      if (l > 0) {
        D.a_ptr = C.take<int32_t>(As[l].sl_ptr.size());
        D.a_col = C.take<int32_t>(As[l].sl_col.size());
        D.a_val32 = C.take<float>(As[l].val.size());
        D.a_val64 = C.take<double>(As[l].val.size());
        D.rs32 = C.take<float>(n);
        D.dinv32 = C.take<float>(n);
        D.dinv64 = C.take<double>(n);
      } else {
        D.a_ptr = I.sl_ptr;
        D.a_col = I.sl_col;
        D.a_val32 = own0 ? C.take<float>(nnz_pad) : I.val32;
        D.a_val64 = own0 ? C.take<double>(nnz_pad) : I.val64;
        D.rs32 = own0 ? C.take<float>(n) : I.rs32;
        D.dinv32 = I.dinv32;
        D.dinv64 = I.dinv64;
      }
      if (l > 0)
        halo_take(C, Ha[l], D.ha);
      else
        D.ha = I.h0;
      halo_take(C, Hp[l], D.hp);
      halo_take(C, Hr[l], D.hr);
      if (l < L - 1) {
        D.p_ptr = C.take<int32_t>(Ps[l].sl_ptr.size());
        D.p_col = C.take<int32_t>(Ps[l].sl_col.size());
        D.p_val32 = C.take<float>(Ps[l].val.size());
        D.p_val64 = C.take<double>(Ps[l].val.size());
        D.r_ptr = C.take<int32_t>(Rs[l].sl_ptr.size());
        D.r_col = C.take<int32_t>(Rs[l].sl_col.size());
        D.r_val32 = C.take<float>(Rs[l].val.size());
        D.r_val64 = C.take<double>(Rs[l].val.size());
      }
      D.b = C.take<double>(4 * (size_t)n);
      D.x = C.take<double>(4 * (size_t)n);
      D.r = C.take<double>(4 * (size_t)n);
      D.y = C.take<double>(4 * (size_t)n);
    }
    cinv64 = C.take<double>(H.coarse_inv.size());
    cinv32 = C.take<float>(H.coarse_inv.size());
    dense64 = C.take<double>(H.dense.size());
    dense32 = C.take<float>(H.dense.size());
    d_lev = C.take<AmgDev>(L);
  };
  Carver sz;
  layout(sz);
  h->amg_bytes = sz.off;
  h->amg_block = h->mem.get(h->amg_bytes);
  if (!h->amg_block) return SHELL_ERR_OOM;
  Carver real;
  real.base = (char *)h->amg_block;
  layout(real);
  std::vector<std::vector<float>> keep32;   // host staging kept alive until the stream synchronises
  auto up = [&](void *dst, const void *src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  auto f32 = [&](const std::vector<double> &v) -> const float * {
    keep32.emplace_back(v.begin(), v.end());
    return keep32.back().data();
  };
  for (int l = 0; l < L; ++l) {
    const AmgDev &D = lev[l];
    if (l > 0) {
      CK(up(D.a_ptr, As[l].sl_ptr.data(), 4 * As[l].sl_ptr.size()));
      CK(up(D.a_col, As[l].sl_col.data(), 4 * As[l].sl_col.size()));
      CK(up(D.a_val64, As[l].val.data(), 8 * As[l].val.size()));
      CK(up(D.a_val32, f32(As[l].val), 4 * As[l].val.size()));
      CK(up(D.rs32, f32(H.levels[l].rowsum), 4 * (size_t)D.n));
      CK(up(D.dinv64, H.levels[l].dinv.data(), 8 * (size_t)D.n));
      CK(up(D.dinv32, f32(H.levels[l].dinv), 4 * (size_t)D.n));
    } else if (own0) {
      CK(up(D.a_val64, val.data(), 8 * nnz_pad));
      CK(up(D.a_val32, f32(val), 4 * nnz_pad));
      CK(up(D.rs32, f32(H.levels[0].rowsum), 4 * (size_t)D.n));
      CK(up(D.dinv64, H.levels[0].dinv.data(), 8 * (size_t)D.n));
      CK(up(D.dinv32, f32(H.levels[0].dinv), 4 * (size_t)D.n));
    }
    if (l < L - 1) {
      CK(up(D.p_ptr, Ps[l].sl_ptr.data(), 4 * Ps[l].sl_ptr.size()));
      CK(up(D.p_col, Ps[l].sl_col.data(), 4 * Ps[l].sl_col.size()));
      CK(up(D.p_val64, Ps[l].val.data(), 8 * Ps[l].val.size()));
      CK(up(D.p_val32, f32(Ps[l].val), 4 * Ps[l].val.size()));
      CK(up(D.r_ptr, Rs[l].sl_ptr.data(), 4 * Rs[l].sl_ptr.size()));
      CK(up(D.r_col, Rs[l].sl_col.data(), 4 * Rs[l].sl_col.size()));
      CK(up(D.r_val64, Rs[l].val.data(), 8 * Rs[l].val.size()));
      CK(up(D.r_val32, f32(Rs[l].val), 4 * Rs[l].val.size()));
    }
    if (l > 0) CK(halo_upload(Ha[l], D.ha, st));
    CK(halo_upload(Hp[l], D.hp, st));
    CK(halo_upload(Hr[l], D.hr, st));
    CK(cudaMemsetAsync(D.b, 0, 32 * (size_t)D.n, st));
    CK(cudaMemsetAsync(D.x, 0, 32 * (size_t)D.n, st));
    CK(cudaMemsetAsync(D.r, 0, 32 * (size_t)D.n, st));
    CK(cudaMemsetAsync(D.y, 0, 32 * (size_t)D.n, st));
  }
  CK(up(cinv64, H.coarse_inv.data(), 8 * H.coarse_inv.size()));
  CK(up(cinv32, f32(H.coarse_inv), 4 * H.coarse_inv.size()));
  CK(up(dense64, H.dense.data(), 8 * H.dense.size()));
  CK(up(dense32, f32(H.dense), 4 * H.dense.size()));
  CK(up(d_lev, lev.data(), sizeof(AmgDev) * L));
  I.amg_levels = L;
  I.amg_coarse_n = nc;
  I.amg_coarse_sweeps = H.coarse_sweeps;
  I.amg_dense_level = H.dense_level;
  I.amg_dense_n = H.dense_n;
  I.amg_dense64 = dense64;
  I.amg_dense32 = dense32;
  I.amg = d_lev;
  I.amg_cinv64 = cinv64;
  I.amg_cinv32 = cinv32;
  CK(up(h->d_inst, &I, sizeof(Inst)));
  CK(cudaStreamSynchronize(st));
  return SHELL_OK;
}

}  // namespace

extern "C" {

void shell_default_options(shell_options *o) {
  if (!o) return;
  std::memset(o, 0, sizeof(*o));
  o->dt = 1e-2;
  o->precision = SHELL_FP64;
  o->pcg_rtol = 0.0;      // precision default: 1e-13 (FP64) / 1e-6 (FP32 inner)
  o->refine_rtol = 0.0;   // 3e-7
  o->pcg_max_it = 20000;
  o->refine_max = 20;
}

const char *shell_strerror(int code) {
  switch (code) {
    case SHELL_OK: return "ok";
    case SHELL_ERR_INVALID_ARG: return "invalid argument";
    case SHELL_ERR_NON_MANIFOLD: return "mesh is not manifold";
    case SHELL_ERR_BAD_ORIENTATION: return "triangles are not consistently oriented";
    case SHELL_ERR_DEGENERATE: return "degenerate rest triangle or stencil";
    case SHELL_ERR_SINGULAR_OPERATOR: return "singular smoothed-hinge fit (L_p C_p)";
    case SHELL_ERR_OOM: return "device memory allocation failed";
    case SHELL_ERR_BUDGET: return "batch memory budget exceeded";
    case SHELL_ERR_NOT_CONVERGED: return "linear solve did not converge within its iteration cap";
    case SHELL_ERR_NONFINITE: return "non-finite value in the step";
    case SHELL_ERR_TIMEOUT: return "device-side wait timed out";
    case SHELL_ERR_CUDA: return cudaGetErrorString(last_cuda_error());
    case SHELL_ERR_NO_DEVICE: return "no CUDA device of compute capability 10.3";
    case SHELL_ERR_BUSY: return "handle is resident in a batch";
    case SHELL_ERR_STATIC_LIMIT: return "request exceeds the static scratch of shell_step_noalloc (2048 CTAs)";
    default: return "unknown error";
  }
}

int shell_create(const shell_mesh *mesh, const shell_material *mat, int32_t model, const shell_bc *bc,
                 const shell_options *opt_in, shell_handle **out) {
  if (!mesh || !mat || !out || !mesh->tris || !mesh->rest_xyz) return SHELL_ERR_INVALID_ARG;
  *out = nullptr;
  if (mesh->n_verts < 3 || mesh->n_tris < 1) return SHELL_ERR_INVALID_ARG;
  if (model < SHELL_EP || model > SHELL_SS) return SHELL_ERR_INVALID_ARG;
  if (!(mat->E > 0) || !(mat->nu >= 0 && mat->nu < 0.5) || !(mat->thickness > 0) || !(mat->density > 0))
    return SHELL_ERR_INVALID_ARG;
  shell_options opt;
  if (opt_in)
    opt = *opt_in;
  else
    shell_default_options(&opt);
  if (!(opt.dt > 0) || (opt.precision != SHELL_FP64 && opt.precision != SHELL_FP32_REFINE))
    return SHELL_ERR_INVALID_ARG;
  fill_default_tolerances(&opt);
  const int nv = mesh->n_verts, nt = mesh->n_tris;
  if (bc && ((bc->n_clamped > 0 && !bc->clamped_edges) || (bc->n_loads > 0 && (!bc->load_vtx || !bc->load_f))))
    return SHELL_ERR_INVALID_ARG;
  if (bc)
    for (int k = 0; k < bc->n_loads; ++k)
      if (bc->load_vtx[k] < 0 || bc->load_vtx[k] >= nv) return SHELL_ERR_INVALID_ARG;
  // fixed components per vertex: pinned and clamped-edge vertices have all three; a vertex with fixed and free
  // components makes the instance's solves projected
  std::vector<uint8_t> fixb(nv, 0);
  bool partial = false;
  if (bc) {
    for (int i = 0; i < nv; ++i) {
      if (bc->fixed_dofs && (bc->fixed_dofs[i] & ~7u)) return SHELL_ERR_INVALID_ARG;
      fixb[i] = (bc->pinned && bc->pinned[i]) ? 7 : (bc->fixed_dofs ? bc->fixed_dofs[i] : 0);
    }
    for (int k = 0; k < 2 * bc->n_clamped; ++k) {
      if (bc->clamped_edges[k] < 0 || bc->clamped_edges[k] >= nv) return SHELL_ERR_INVALID_ARG;
      fixb[bc->clamped_edges[k]] = 7;
    }
    for (int i = 0; i < nv; ++i) partial = partial || (fixb[i] != 0 && fixb[i] != 7);
  }
  int rc = check_device();
  if (rc != SHELL_OK) return rc;

  const bool plate = (model == SHELL_EP || model == SHELL_FP || model == SHELL_SP);
  if (plate && !planar(mesh->rest_xyz, nv, mesh->tris, nt)) return SHELL_ERR_INVALID_ARG;

  HostTopo T;
  rc = build_topology(nv, nt, mesh->tris, bc ? bc->n_clamped : 0, bc ? bc->clamped_edges : nullptr, model, &T);
  if (rc != SHELL_OK) return rc;

  shell_handle *h = new (std::nothrow) shell_handle();
  if (!h) return SHELL_ERR_OOM;
  h->nv = nv;
  h->nt = nt;
  h->ne = T.ne;
  h->model = model;
  h->mat = *mat;
  h->opt = opt;
  h->mem.alloc = opt.alloc;
  h->mem.free = opt.free;
  h->mem.user = opt.alloc_user;
  h->mem.st = (cudaStream_t)opt.cuda_stream;
  cudaStream_t st = h->mem.st;

  Inst &I = h->h;
  I.nv = nv;
  I.nt = nt;
  I.ne = T.ne;
  I.model = model;
  I.precision = opt.precision;
  I.kt = T.kt;
  I.n_slices = T.n_slices;
  I.rows_per_thread = 1;
  const int chunk = kBlock * I.rows_per_thread;
  I.n_chunks = (nv + chunk - 1) / chunk;
  I.pcg_max_it = opt.pcg_max_it;
  I.refine_max = opt.refine_max;
  I.nl_max = 0;        // linearised step until shell_set_nonlinear
  I.nl_rtol = 1e-8;
  I.dt = opt.dt;
  I.pcg_rtol = opt.pcg_rtol;
  I.refine_rtol = opt.refine_rtol;
  I.mu = mat->E / (2.0 * (1.0 + mat->nu));
  I.lam = mat->E * mat->nu / (1.0 - mat->nu * mat->nu);
  I.n_slots = T.n_slots;
  I.n_local = T.n_local;
  const size_t nnz_pad = (size_t)T.sl_ptr[T.n_slices];
  h->nnz = T.nnz;
  h->nnz_pad = (int64_t)nnz_pad;
  const int ne = T.ne;
  const int n_loads = bc ? bc->n_loads : 0;

  HostHalo H0;   // gather lists of the matrix for the FP32 products
  if (I.precision != SHELL_FP64 && !opt.no_staging) build_halo(nv, nv, T.sl_ptr, T.sl_col, T.row_ptr, true, &H0);

  for (int s0 = 0; s0 < nt; s0 += kForceBlock) h->tiles.push_back({0, 0, s0, std::min(kForceBlock, nt - s0)});
  for (int s0 = 0; s0 < ne; s0 += kForceBlock) h->tiles.push_back({0, 1, s0, std::min(kForceBlock, ne - s0)});

  // ---- persistent block
  auto layout = [&](Carver &C) {
    I.x = C.take<double>(3 * (size_t)nv);
    I.v = C.take<double>(3 * (size_t)nv);
    I.vprev = C.take<double>(3 * (size_t)nv);
    I.vprev2 = C.take<double>(3 * (size_t)nv);
    I.vprev3 = C.take<double>(3 * (size_t)nv);
    I.xk = C.take<double>(3 * (size_t)nv);
    I.vk = C.take<double>(3 * (size_t)nv);
    I.rest = C.take<double>(3 * (size_t)nv);
    I.fext = C.take<double>(3 * (size_t)nv);
    I.mass = C.take<double>(nv);
    I.pinned = C.take<uint8_t>(nv);
    I.fix = partial ? C.take<uint8_t>(nv) : nullptr;
    I.t_idx = C.take<int32_t>(6 * (size_t)nt);
    I.t_bc = C.take<uint8_t>(3 * (size_t)nt);
    I.t_mode = C.take<uint8_t>(nt);
    I.t_L64 = C.take<double>(18 * (size_t)nt);
    I.t_L32 = C.take<float>(18 * (size_t)nt);
    I.t_W64 = C.take<double>(6 * (size_t)nt);
    I.t_W32 = C.take<float>(6 * (size_t)nt);
    I.t_k064 = C.take<double>(3 * (size_t)nt);
    I.t_k032 = C.take<float>(3 * (size_t)nt);
    I.t_n64 = C.take<double>(3 * (size_t)nt);
    I.t_n32 = C.take<float>(3 * (size_t)nt);
    I.m_D64 = C.take<double>(3 * (size_t)nt);
    I.m_D32 = C.take<float>(3 * (size_t)nt);
    I.m_G64 = C.take<double>(3 * (size_t)nt);
    I.m_At64 = C.take<double>(nt);
    I.m_At32 = C.take<float>(nt);
    I.m_T = C.take<double>(10 * (size_t)nt);
    I.e_idx = C.take<int32_t>(4 * (size_t)ne);
    I.e_mode = C.take<uint8_t>(ne);
    I.e_L64 = C.take<double>(4 * (size_t)ne);
    I.e_L32 = C.take<float>(4 * (size_t)ne);
    I.e_w64 = C.take<double>(ne);
    I.e_w32 = C.take<float>(ne);
    I.e_k064 = C.take<double>(ne);
    I.e_k032 = C.take<float>(ne);
    I.e_n64 = C.take<double>(3 * (size_t)ne);
    I.e_n32 = C.take<float>(3 * (size_t)ne);
    I.vtx_ptr = C.take<int32_t>(nv + 1);
    I.vtx_slot = C.take<int32_t>(T.vtx_slot.size());
    I.contrib = C.take<double>(3 * (size_t)T.n_slots);
    I.sl_ptr = C.take<int32_t>(T.n_slices + 1);
    I.sl_col = C.take<int32_t>(nnz_pad);
    I.val64 = C.take<double>(nnz_pad);
    I.val32 = C.take<float>(nnz_pad);
    I.dinv64 = C.take<double>(nv);
    I.dinv32 = C.take<float>(nv);
    I.rs32 = C.take<float>(nv);
    I.diag_pos = C.take<int32_t>(nv);
    halo_take(C, H0, I.h0);
    I.b = C.take<double>(3 * (size_t)nv);
    I.sol = C.take<double>(3 * (size_t)nv);
    I.r64 = C.take<double>(3 * (size_t)nv);
    I.g64 = C.take<double>(4 * (size_t)nv);
    I.r = C.take<double>(3 * (size_t)nv);
    I.p = C.take<double>(3 * (size_t)nv);
    I.s = C.take<double>(3 * (size_t)nv);
    I.w = C.take<double>(3 * (size_t)nv);
    I.xs = C.take<double>(3 * (size_t)nv);
    I.g = C.take<double>(4 * (size_t)nv);
    I.part = C.take<double>(8 * (size_t)I.n_chunks);
    I.ebuf = C.take<double>(2 * (size_t)(nt + ne));
    I.status = C.take<InstStatus>(1);
    I.err_flags = C.take<int32_t>(1);
    h->d_inst = C.take<Inst>(1);
    h->d_stage = C.take<double>(6 * (size_t)nv);
    h->d_energy = C.take<double>(4);
    h->d_forces = h->d_stage;   // shares the staging area
    h->d_tiles = C.take<Tile>(h->tiles.size());
  };
  Carver sizer;
  layout(sizer);
  h->block_bytes = sizer.off;
  h->block = h->mem.get(h->block_bytes);
  if (!h->block) {
    delete h;
    return SHELL_ERR_OOM;
  }
  Carver real;
  real.base = (char *)h->block;
  layout(real);

  // ---- temporary block: assembly sources, local matrices, point loads
  int32_t *d_lv = nullptr;
  double *d_lf = nullptr;
  auto tlayout = [&](Carver &C) {
    I.asm_ptr = C.take<int32_t>(nnz_pad + 1);
    I.asm_src = C.take<int32_t>(T.asm_src.size());
    I.local = C.take<double>(T.n_local);
    d_lv = C.take<int32_t>(n_loads);
    d_lf = C.take<double>(3 * (size_t)n_loads);
  };
  Carver tsz;
  tlayout(tsz);
  void *tmp = h->mem.get(tsz.off);
  if (!tmp) {
    h->mem.put(h->block, h->block_bytes);
    delete h;
    return SHELL_ERR_OOM;
  }
  Carver treal;
  treal.base = (char *)tmp;
  tlayout(treal);

  auto fail = [&](int code) {
    cudaStreamSynchronize(st);
    h->mem.put(tmp, tsz.off);
    h->mem.put(h->block, h->block_bytes);
    delete h;
    return code;
  };
#define CKF(call)                     \
  do {                                \
    cudaError_t e_ = (call);          \
    if (e_ != cudaSuccess) {          \
      last_cuda_error() = e_;         \
      return fail(SHELL_ERR_CUDA);    \
    }                                 \
  } while (0)

  // ---- uploads
  std::vector<double> rest = to_soa(mesh->rest_xyz, nv);
  std::vector<double> x0 = to_soa(mesh->init_xyz ? mesh->init_xyz : mesh->rest_xyz, nv);
  std::vector<double> v0 = mesh->init_vel ? to_soa(mesh->init_vel, nv) : std::vector<double>((size_t)3 * nv, 0.0);
  std::vector<uint8_t> pin(nv, 0);
  for (int i = 0; i < nv; ++i) pin[i] = fixb[i] == 7 ? 1 : 0;
  auto up = [&](void *dst, const void *src, size_t bytes) {
    return bytes ? cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st) : cudaSuccess;
  };
  CKF(up(I.rest, rest.data(), 8 * rest.size()));
  CKF(up(I.x, x0.data(), 8 * x0.size()));
  CKF(up(I.v, v0.data(), 8 * v0.size()));
  CKF(up(I.vprev, v0.data(), 8 * v0.size()));
  CKF(up(I.vprev2, v0.data(), 8 * v0.size()));
  CKF(up(I.vprev3, v0.data(), 8 * v0.size()));
  CKF(up(I.pinned, pin.data(), nv));
  if (partial) CKF(up(I.fix, fixb.data(), nv));
  CKF(up(I.t_idx, T.t_idx.data(), 4 * T.t_idx.size()));
  CKF(up(I.t_bc, T.t_bc.data(), T.t_bc.size()));
  CKF(up(I.e_idx, T.e_idx.data(), 4 * T.e_idx.size()));
  CKF(up(I.vtx_ptr, T.vtx_ptr.data(), 4 * T.vtx_ptr.size()));
  CKF(up(I.vtx_slot, T.vtx_slot.data(), 4 * T.vtx_slot.size()));
  CKF(up(I.sl_ptr, T.sl_ptr.data(), 4 * T.sl_ptr.size()));
  CKF(up(I.sl_col, T.sl_col.data(), 4 * T.sl_col.size()));
  CKF(up(I.diag_pos, T.diag_pos.data(), 4 * T.diag_pos.size()));
  CKF(halo_upload(H0, I.h0, st));
  CKF(up(I.asm_ptr, T.asm_ptr.data(), 4 * T.asm_ptr.size()));
  CKF(up(I.asm_src, T.asm_src.data(), 4 * T.asm_src.size()));
  if (n_loads) {
    CKF(up(d_lv, bc->load_vtx, 4 * (size_t)n_loads));
    CKF(up(d_lf, bc->load_f, 24 * (size_t)n_loads));
  }
  CKF(cudaMemsetAsync(I.val64, 0, 8 * nnz_pad, st));
  CKF(cudaMemsetAsync(I.val32, 0, 4 * nnz_pad, st));
  CKF(cudaMemsetAsync(I.t_mode, MODE_NONE, nt, st));
  CKF(cudaMemsetAsync(I.status, 0, sizeof(InstStatus), st));
  CKF(cudaMemsetAsync(I.err_flags, 0, sizeof(int32_t), st));
  CKF(cudaMemsetAsync(I.g, 0, 32 * (size_t)nv, st));
  CKF(cudaMemsetAsync(I.g64, 0, 32 * (size_t)nv, st));
  CKF(up(h->d_inst, &I, sizeof(Inst)));
  CKF(up(h->d_tiles, h->tiles.data(), sizeof(Tile) * h->tiles.size()));
  // ---- device precompute and assembly (FP64)
  const double g[3] = {bc ? bc->gravity[0] : 0.0, bc ? bc->gravity[1] : 0.0, bc ? bc->gravity[2] : 0.0};
  CKF(launch_precompute(h->d_inst, I, mat->E, mat->nu, mat->thickness, mat->density, st));
  CKF(launch_mass(h->d_inst, I, mat->density, g, n_loads, d_lv, d_lf, st));
  CKF(launch_assemble(h->d_inst, I, st));
  int32_t flags = 0;
  CKF(cudaMemcpyAsync(&flags, I.err_flags, 4, cudaMemcpyDeviceToHost, st));
  CKF(cudaStreamSynchronize(st));
  h->mem.put(tmp, tsz.off);
  I.asm_ptr = nullptr;
  I.asm_src = nullptr;
  I.local = nullptr;
  cudaMemcpyAsync(h->d_inst, &I, sizeof(Inst), cudaMemcpyHostToDevice, st);
  cudaStreamSynchronize(st);
  if (flags) {
    h->mem.put(h->block, h->block_bytes);
    delete h;
    return (flags & 1) ? SHELL_ERR_DEGENERATE : SHELL_ERR_SINGULAR_OPERATOR;
  }
#undef CKF
  rc = setup_amg(h, T, opt.preconditioner, !opt.no_staging, partial ? fixb : std::vector<uint8_t>());
  if (rc != SHELL_OK) {
    if (h->amg_block) h->mem.put(h->amg_block, h->amg_bytes);
    h->mem.put(h->block, h->block_bytes);
    delete h;
    return rc;
  }
  // ---- private batch for shell_step
  rc = batch_new(&opt, (size_t)-1, true, &h->solo);
  if (rc != SHELL_OK) {
    h->mem.put(h->block, h->block_bytes);
    delete h;
    return rc;
  }
  h->solo->slots.push_back(h);
  *out = h;
  return SHELL_OK;
}

int shell_step(shell_handle *h, int32_t n_steps, shell_step_stats *stats) {
  if (!h || n_steps < 0) return SHELL_ERR_INVALID_ARG;
  if (h->batch) return SHELL_ERR_BUSY;
  return batch_step(h->solo, n_steps, stats);
}

// shell_step for callers that cannot allocate: the launch scratch is the static array of kernels_solve.cu
int shell_step_noalloc(shell_handle *h, int32_t n_steps, shell_step_stats *stats) {
  if (!h || n_steps < 0) return SHELL_ERR_INVALID_ARG;
  if (h->batch) return SHELL_ERR_BUSY;
  const bool newton = uses_nt_variant(h->h);
  const int prec = newton ? 3 : (h->h.precision == SHELL_FP64 ? 1 : 2);
  int team = std::max(1, std::min(num_sms() * blocks_per_sm_cached(prec, prec == 2 ? 3 : 2), h->h.n_chunks));
  if (team > static_max_ctas()) return SHELL_ERR_STATIC_LIMIT;
  const InstStatus before = h->last_status;
  InstStatus after{};
  int32_t aborted = 0;
  cudaError_t e = launch_step_static(h->d_inst, h->d_tiles, (int)h->tiles.size(), h->h.precision != SHELL_FP64,
                                     newton, team, n_steps, std::max(1, h->h.nl_max), &after, &aborted, h->mem.st);
  if (e != cudaSuccess) {
    last_cuda_error() = e;
    return SHELL_ERR_CUDA;
  }
  h->last_status = after;
  if (stats) {
    stats->steps_done = after.steps_done - before.steps_done;
    stats->pcg_iterations = after.last_iters;
    stats->refine_rounds = after.last_rounds;
    stats->status = after.err;
    stats->total_pcg_iterations = after.total_iters - before.total_iters;
    stats->rel_residual = after.rel_res;
    stats->total_refine_rounds = after.total_rounds - before.total_rounds;
    stats->last_solve_us = after.last_ns * 1e-3;
    stats->team_ctas = after.team_size;
    stats->nl_iterations = h->h.nl_max > 1 ? after.nl_iters : 0;
  }
  if (aborted) return SHELL_ERR_TIMEOUT;
  return after.err;
}

static int run_forces64(shell_handle *h, int want_energy) {
  cudaStream_t st = h->mem.st;
  cudaError_t e = launch_forces(h->d_inst, h->d_tiles, (int)h->tiles.size(), want_energy, 0, st);
  if (e != cudaSuccess) {
    last_cuda_error() = e;
    return SHELL_ERR_CUDA;
  }
  return SHELL_OK;
}

// exact backward Euler: chord iterations per step (<= 1: linearised step) and their tolerance
int shell_set_nonlinear(shell_handle *h, int32_t max_iters, double rtol) {
  if (!h || max_iters < 0 || !(rtol >= 0.0)) return SHELL_ERR_INVALID_ARG;
  h->h.nl_max = max_iters;
  h->h.nl_rtol = rtol;
  CK(cudaMemcpyAsync(h->d_inst, &h->h, sizeof(Inst), cudaMemcpyHostToDevice, h->mem.st));
  CK(cudaStreamSynchronize(h->mem.st));
  // batches hold copies of the descriptor and plan their launches per step by it
  if (h->batch) h->batch->dirty = true;
  if (h->solo) h->solo->dirty = true;
  return SHELL_OK;
}

int shell_set_newton(shell_handle *h, int32_t on) {
  if (!h) return SHELL_ERR_INVALID_ARG;
  h->h.nl_newton = on ? 1 : 0;
  CK(cudaMemcpyAsync(h->d_inst, &h->h, sizeof(Inst), cudaMemcpyHostToDevice, h->mem.st));
  CK(cudaStreamSynchronize(h->mem.st));
  if (h->batch) h->batch->dirty = true;
  if (h->solo) h->solo->dirty = true;
  return SHELL_OK;
}

// Eq. 64 quasi-static Newton-Raphson: one step of the handle's iteration machinery in its static mode (no
// inertia in the residual, Newton tangent, eps_u limiter, absolute residual test), then the handle's
// nonlinear settings are restored
int shell_solve_static(shell_handle *h, double eps_f, double eps_u, int32_t max_iters, shell_step_stats *stats) {
  if (!h || !(eps_f > 0.0) || !(eps_u >= 0.0) || max_iters < 1) return SHELL_ERR_INVALID_ARG;
  if (h->batch) return SHELL_ERR_BUSY;
  const Inst saved = h->h;
  h->h.nl_max = max_iters + 1;   // up to max_iters solves, then a launch that tests the last iterate
  h->h.nl_rtol = 0.0;
  h->h.nl_atol = eps_f;
  h->h.nl_eps_u = eps_u;
  h->h.nl_newton = 1;
  h->h.nl_static = 1;
  CK(cudaMemcpyAsync(h->d_inst, &h->h, sizeof(Inst), cudaMemcpyHostToDevice, h->mem.st));
  if (h->solo) h->solo->dirty = true;
  const int rc = shell_step(h, 1, stats);
  h->h.nl_max = saved.nl_max;
  h->h.nl_rtol = saved.nl_rtol;
  h->h.nl_atol = saved.nl_atol;
  h->h.nl_eps_u = saved.nl_eps_u;
  h->h.nl_newton = saved.nl_newton;
  h->h.nl_static = saved.nl_static;
  CK(cudaMemcpyAsync(h->d_inst, &h->h, sizeof(Inst), cudaMemcpyHostToDevice, h->mem.st));
  CK(cudaStreamSynchronize(h->mem.st));
  if (h->solo) h->solo->dirty = true;
  return rc;
}

int shell_energy(shell_handle *h, double out[4]) {
  if (!h || !out) return SHELL_ERR_INVALID_ARG;
  int rc = run_forces64(h, 1);
  if (rc != SHELL_OK) return rc;
  cudaStream_t st = h->mem.st;
  CK(launch_energy_reduce(h->d_inst, h->h, h->d_energy, st));
  CK(cudaMemcpyAsync(out, h->d_energy, 32, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SHELL_OK;
}

int shell_forces(shell_handle *h, double *out_xyz) {
  if (!h || !out_xyz) return SHELL_ERR_INVALID_ARG;
  int rc = run_forces64(h, 0);
  if (rc != SHELL_OK) return rc;
  cudaStream_t st = h->mem.st;
  CK(launch_gather_forces(h->d_inst, h->h, h->d_forces, st));
  CK(cudaMemcpyAsync(out_xyz, h->d_forces, 24 * (size_t)h->nv, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SHELL_OK;
}

int shell_apply_matrix(shell_handle *h, const double *in, double *out) {
  if (!h || !in || !out) return SHELL_ERR_INVALID_ARG;
  cudaStream_t st = h->mem.st;
  const size_t n3 = 3 * (size_t)h->nv;
  CK(cudaMemcpyAsync(h->d_stage, in, 8 * n3, cudaMemcpyHostToDevice, st));
  CK(launch_matvec64(h->d_inst, h->h, h->d_stage, h->d_stage + n3, st));
  CK(cudaMemcpyAsync(out, h->d_stage + n3, 8 * n3, cudaMemcpyDeviceToHost, st));
  CK(cudaStreamSynchronize(st));
  return SHELL_OK;
}

int shell_get_state(shell_handle *h, double *x, double *v) {
  if (!h) return SHELL_ERR_INVALID_ARG;
  cudaStream_t st = h->mem.st;
  const size_t n3 = 3 * (size_t)h->nv;
  if (x) {
    CK(launch_soa_to_aos(h->h.x, h->d_stage, h->nv, st));
    CK(cudaMemcpyAsync(x, h->d_stage, 8 * n3, cudaMemcpyDeviceToHost, st));
  }
  if (v) {
    CK(launch_soa_to_aos(h->h.v, h->d_stage + n3, h->nv, st));
    CK(cudaMemcpyAsync(v, h->d_stage + n3, 8 * n3, cudaMemcpyDeviceToHost, st));
  }
  CK(cudaStreamSynchronize(st));
  return SHELL_OK;
}

int shell_set_state(shell_handle *h, const double *x, const double *v) {
  if (!h) return SHELL_ERR_INVALID_ARG;
  cudaStream_t st = h->mem.st;
  const size_t n3 = 3 * (size_t)h->nv;
  if (x) {
    CK(cudaMemcpyAsync(h->d_stage, x, 8 * n3, cudaMemcpyHostToDevice, st));
    CK(launch_aos_to_soa(h->d_stage, h->h.x, h->nv, st));
  }
  if (v) {
    CK(cudaMemcpyAsync(h->d_stage + n3, v, 8 * n3, cudaMemcpyHostToDevice, st));
    CK(launch_aos_to_soa(h->d_stage + n3, h->h.v, h->nv, st));
  }
  // a new state clears a previous step failure
  CK(cudaMemsetAsync(&h->h.status->err, 0, sizeof(int32_t), st));
  h->last_status.err = SHELL_OK;
  CK(cudaStreamSynchronize(st));
  return SHELL_OK;
}

int shell_get_state_device(shell_handle *h, double *d_x, double *d_v) {
  if (!h) return SHELL_ERR_INVALID_ARG;
  cudaStream_t st = h->mem.st;
  if (d_x) CK(launch_soa_to_aos(h->h.x, d_x, h->nv, st));
  if (d_v) CK(launch_soa_to_aos(h->h.v, d_v, h->nv, st));
  return SHELL_OK;
}

int shell_set_state_device(shell_handle *h, const double *d_x, const double *d_v) {
  if (!h) return SHELL_ERR_INVALID_ARG;
  cudaStream_t st = h->mem.st;
  if (d_x) CK(launch_aos_to_soa(d_x, h->h.x, h->nv, st));
  if (d_v) CK(launch_aos_to_soa(d_v, h->h.v, h->nv, st));
  return SHELL_OK;
}

int shell_info(shell_handle *h, int64_t out[9]) {
  if (!h || !out) return SHELL_ERR_INVALID_ARG;
  out[0] = h->nv;
  out[1] = h->nt;
  out[2] = (h->model == SHELL_EP || h->model == SHELL_ES) ? h->ne : h->nt;
  out[3] = (int64_t)h->block_bytes;
  out[4] = h->nnz;
  out[5] = h->nnz_pad;
  out[6] = h->h.n_slots;
  out[7] = h->h.amg_levels;
  out[8] = h->vcycle_bytes;
  out[3] = (int64_t)(h->block_bytes + h->amg_bytes);
  return SHELL_OK;
}

int shell_destroy(shell_handle *h) {
  if (!h) return SHELL_ERR_INVALID_ARG;
  if (h->batch) return SHELL_ERR_BUSY;
  cudaStreamSynchronize(h->mem.st);
  batch_free(h->solo);
  if (h->amg_block) h->mem.put(h->amg_block, h->amg_bytes);
  h->mem.put(h->block, h->block_bytes);
  cudaStreamSynchronize(h->mem.st);
  delete h;
  return SHELL_OK;
}

int shell_topology_summary(int32_t nv, int32_t nt, const int32_t *tris, int32_t n_clamped, const int32_t *clamped,
                           int32_t model, int64_t out[8]) {
  if (!tris || !out || nv < 3 || nt < 1 || model < SHELL_EP || model > SHELL_SS) return SHELL_ERR_INVALID_ARG;
  if (n_clamped > 0 && !clamped) return SHELL_ERR_INVALID_ARG;
  HostTopo T;
  int rc = build_topology(nv, nt, tris, n_clamped, clamped, model, &T);
  if (rc != SHELL_OK) return rc;
  int64_t bad = 0;
  int64_t virt = 0;
  for (int t = 0; t < nt; ++t) {
    bool v = false;
    for (int j = 0; j < 6; ++j) {
      int q = T.t_idx[(size_t)j * nt + t];
      if (q >= nv || (j < 3 && q < 0) || q < -1) ++bad;
      if (j >= 3 && q < 0) {
        v = true;
        if (T.t_bc[(size_t)(j - 3) * nt + t] == 0) ++bad;
      }
      if (j >= 3 && q >= 0 && T.t_bc[(size_t)(j - 3) * nt + t] != 0) ++bad;
    }
    virt += v;
  }
  for (int e = 0; e < T.ne; ++e)
    for (int j = 0; j < 4; ++j) {
      int q = T.e_idx[(size_t)j * T.ne + e];
      if (q >= nv || q < (j == 3 ? -1 : 0)) ++bad;
      if (j == 3 && (q < 0) != (e >= T.ne_int)) ++bad;
    }
  if ((int)T.vtx_ptr.size() != nv + 1 || T.vtx_ptr[0] != 0) ++bad;
  for (int i = 0; i < nv && !bad; ++i)
    for (int q = T.vtx_ptr[i]; q < T.vtx_ptr[i + 1]; ++q)
      if (T.vtx_slot[q] < 0 || T.vtx_slot[q] >= T.n_slots || (q > T.vtx_ptr[i] && T.vtx_slot[q] <= T.vtx_slot[q - 1]))
        ++bad;
  const int64_t nnz_pad = T.sl_ptr[T.n_slices];
  for (int s = 0; s < T.n_slices; ++s)
    if ((T.sl_ptr[s + 1] - T.sl_ptr[s]) % 32 != 0) ++bad;
  for (int64_t p = 0; p < nnz_pad; ++p)
    if (T.sl_col[p] < 0 || T.sl_col[p] >= nv) ++bad;
  for (int i = 0; i < nv; ++i) {
    int d = T.diag_pos[i];
    int s = i / 32;
    if (d < T.sl_ptr[s] || d >= T.sl_ptr[s + 1] || T.sl_col[d] != i || (d - T.sl_ptr[s]) % 32 != i % 32) ++bad;
  }
  if ((int64_t)T.asm_ptr.size() != nnz_pad + 1 || T.asm_ptr[nnz_pad] != (int64_t)T.asm_src.size()) ++bad;
  for (int32_t q : T.asm_src)
    if (q < 0 || q >= T.n_local) ++bad;
  out[0] = T.ne_int;
  out[1] = T.ne - T.ne_int;
  out[2] = virt;
  out[3] = T.nnz;
  out[4] = nnz_pad;
  out[5] = T.n_slots;
  out[6] = (int64_t)T.asm_src.size();
  out[7] = bad;
  return SHELL_OK;
}

// ---------------------------------------------------------------- batches
int shell_batch_create(const shell_options *opt, size_t budget, shell_batch **out) {
  if (!out) return SHELL_ERR_INVALID_ARG;
  *out = nullptr;
  int rc = check_device();
  if (rc != SHELL_OK) return rc;
  shell_options o;
  if (opt)
    o = *opt;
  else
    shell_default_options(&o);
  return batch_new(&o, budget, false, out);
}

int shell_batch_admit(shell_batch *b, shell_handle *h, int32_t *slot) {
  if (!b || !h) return SHELL_ERR_INVALID_ARG;
  if (h->batch) return SHELL_ERR_BUSY;
  if (b->used + h->block_bytes + h->amg_bytes > b->budget) return SHELL_ERR_BUDGET;
  int k = -1;
  for (size_t q = 0; q < b->slots.size(); ++q)
    if (!b->slots[q]) {
      k = (int)q;
      break;
    }
  if (k < 0) {
    k = (int)b->slots.size();
    b->slots.push_back(nullptr);
  }
  b->slots[k] = h;
  h->batch = b;
  h->slot = k;
  b->used += h->block_bytes + h->amg_bytes;
  b->dirty = true;
  if (slot) *slot = k;
  return SHELL_OK;
}

int shell_batch_retire(shell_batch *b, int32_t slot) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot]) return SHELL_ERR_INVALID_ARG;
  shell_handle *h = b->slots[slot];
  cudaStreamSynchronize(b->mem.st);
  b->slots[slot] = nullptr;
  h->batch = nullptr;
  h->slot = -1;
  b->used -= h->block_bytes + h->amg_bytes;
  b->dirty = true;
  return SHELL_OK;
}

int shell_batch_step_states(shell_batch *b, int32_t n_steps, const double *x_in, const double *v_in, double *x_out,
                            double *v_out, shell_step_stats *stats) {
  if (!b || (!x_in) != (!v_in) || (!x_out) != (!v_out)) return SHELL_ERR_INVALID_ARG;
  return batch_step(b, n_steps, stats, x_in, v_in, x_out, v_out);
}

int shell_batch_step(shell_batch *b, int32_t n_steps, shell_step_stats *stats) {
  if (!b) return SHELL_ERR_INVALID_ARG;
  return batch_step(b, n_steps, stats);
}

int shell_batch_capacity(shell_batch *b) { return b ? (int)b->slots.size() : 0; }

// packed state transfer of every resident instance (rows in increasing slot order)
static int batch_states(shell_batch *b, double *x, double *v, const double *xin, const double *vin) {
  if (!b) return SHELL_ERR_INVALID_ARG;
  if (b->dirty) {
    int rc = rebuild_tables(b);
    if (rc != SHELL_OK) return rc;
  }
  if (b->n_active == 0) return SHELL_OK;
  int rc = enqueue_states(b, x, v, xin, vin);
  if (rc != SHELL_OK) return rc;
  CK(cudaStreamSynchronize(b->mem.st));
  return SHELL_OK;
}

int shell_batch_get_states(shell_batch *b, double *x, double *v) {
  if (!x || !v) return SHELL_ERR_INVALID_ARG;
  return batch_states(b, x, v, nullptr, nullptr);
}

int shell_batch_set_states(shell_batch *b, const double *x, const double *v) {
  if (!x || !v) return SHELL_ERR_INVALID_ARG;
  return batch_states(b, nullptr, nullptr, x, v);
}

int shell_batch_state_layout(shell_batch *b, int32_t *slots, int64_t *row_offsets) {
  if (!b) return SHELL_ERR_INVALID_ARG;
  int k = 0;
  int64_t off = 0;
  for (size_t q = 0; q < b->slots.size(); ++q)
    if (b->slots[q]) {
      if (slots) slots[k] = (int32_t)q;
      if (row_offsets) row_offsets[k] = off;
      off += b->slots[q]->nv;
      ++k;
    }
  if (row_offsets) row_offsets[k] = off;
  return k;
}

int shell_batch_step_times(shell_batch *b, float *out_ms, int32_t n) {
  if (!b || !out_ms || n < 0) return SHELL_ERR_INVALID_ARG;
  for (int k = 0; k < n && k < (int)b->step_ms.size(); ++k) out_ms[k] = b->step_ms[k];
  return std::min<int>(n, (int)b->step_ms.size());
}

// Autotuner: the results of a batch do not depend on its launch shape (every reduction has a fixed order
// independent of the team layout), so candidate shapes are tried on real, committed steps and timed with
// CUDA events; the fastest is kept.
constexpr int kSettleCalls = 3;   // calls of steps_per_trial steps after the trials (see include/shell.h)

int shell_batch_autotune(shell_batch *b, int32_t steps_per_trial, double *out_ms, int32_t *out_choice) {
  if (!b || steps_per_trial < 1) return SHELL_ERR_INVALID_ARG;
  if (b->dirty) {
    int rc = rebuild_tables(b);
    if (rc != SHELL_OK) return rc;
  }
  if (b->n_active == 0) return SHELL_OK;
  const int occ_max = max_occ(b->prec);
  int occs[3] = {1, std::max(1, occ_max / 2), occ_max};
  if (b->prec == 2) {   // the FP32 variants compiled for 3, 4 and 5 CTAs per SM
    occs[0] = blocks_per_sm_cached(2, 3);
    occs[1] = blocks_per_sm_cached(2, 4);
    occs[2] = blocks_per_sm_cached(2, 5);
  }
  const double scales[3] = {0.5, 1.0, 2.0};
  double best = 1e300;
  int best_k = 0;
  for (int k = 0; k < 12; ++k) {
    const int pol = k < 9 ? 0 : 1;
    const int oi = k < 9 ? k / 3 : 2, si = k % 3;
    if ((pol == 0 && oi > 0 && occs[oi] == occs[oi - 1]) || (pol == 1 && max_clusters_cached(b->prec) == 0)) {
      if (out_ms) out_ms[k] = -1.0;
      continue;
    }
    b->policy = pol;
    b->occ = occs[oi];
    b->share_scale = scales[si];
    b->dirty = true;
    int rc = batch_step(b, steps_per_trial, nullptr);
    if (rc != SHELL_OK) return rc;
    double ms = 0.0;
    for (float t : b->step_ms) ms += t;
    ms /= std::max<size_t>(1, b->step_ms.size());
    if (pol == 1 && b->cluster_off) ms = 1e300;   // the cluster launch was refused (the steps still ran)
    if (out_ms) out_ms[k] = ms < 1e299 ? ms : -2.0;
    if (ms < best) {
      best = ms;
      best_k = k;
    }
  }
  b->policy = best_k < 9 ? 0 : 1;
  b->occ = occs[best_k < 9 ? best_k / 3 : 2];
  b->share_scale = scales[best_k % 3];
  // settle: the schedule of the chosen shape is planned from measured times, and those measured under the
  // trials' other shapes predict it poorly; one call with the chosen shape replaces them, then further calls
  // re-plan from the chosen shape's own times
  for (int q = 0; q < kSettleCalls; ++q) {
    b->dirty = true;
    int rc = batch_step(b, steps_per_trial, nullptr);
    if (rc != SHELL_OK) return rc;
    if (q == 0)
      for (int i : b->active) {
        shell_handle *h = b->slots[i];
        h->hist_ns[0] = h->meas_ns;
        h->hist_team[0] = h->meas_team;
        h->hist_n = 1;
      }
  }
  b->dirty = true;
  if (out_choice) {
    out_choice[0] = b->occ;
    out_choice[1] = (int32_t)std::lround(b->share_scale * 100.0);
    out_choice[2] = b->policy;
  }
  return SHELL_OK;
}

int shell_batch_set_launch(shell_batch *b, int32_t ctas_per_sm, int32_t share_x100, int32_t clusters) {
  if (!b || ctas_per_sm < 1 || share_x100 < 1) return SHELL_ERR_INVALID_ARG;
  b->occ = ctas_per_sm;
  b->share_scale = share_x100 / 100.0;
  b->policy = clusters ? 1 : 0;
  b->dirty = true;
  return SHELL_OK;
}

int shell_batch_set_profiling(shell_batch *b, int32_t on) {
  if (!b) return SHELL_ERR_INVALID_ARG;
  b->profiling = on != 0;
  return SHELL_OK;
}

int shell_batch_set_wait_limit(shell_batch *b, int64_t ns) {
  if (!b) return SHELL_ERR_INVALID_ARG;
  b->wait_ns = ns > 0 ? (unsigned long long)ns : (unsigned long long)kMaxTeamWaitMs * 1000000ull;
  destroy_graph(b);   // the captured launches hold the previous bound
  return SHELL_OK;
}

int shell_batch_kernel_times(shell_batch *b, double out_ms[2]) {
  if (!b || !out_ms) return SHELL_ERR_INVALID_ARG;
  out_ms[0] = b->kern_ms[0];
  out_ms[1] = b->kern_ms[1];
  return SHELL_OK;
}

int shell_batch_destroy(shell_batch *b) {
  if (!b) return SHELL_ERR_INVALID_ARG;
  cudaStreamSynchronize(b->mem.st);
  batch_free(b);
  return SHELL_OK;
}

}  // extern "C"
