// Host side of the C ABI declared in include/esdp.h: validation, device
// workspace, launch planning (tile shapes, actions split, rows per thread),
// the autotuner, and the drivers of the sweep, bid-curve and adjoint kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <map>
#include <mutex>
#include <numeric>
#include <queue>
#include <string>
#include <vector>

#include "../../include/esdp.h"
#include "esdp_internal.h"

using namespace esdp;

namespace {

constexpr size_t kSmemLimit = 227 * 1024;

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

// One planned sweep launch over a subset of the assets.
struct Plan {
  SweepShape shape;
  std::vector<int> asset_ids;       // context asset index of each launch asset
  std::vector<AssetDev> adev;
  std::vector<WorkItem> items;
  std::vector<int> cta_items;
  int n_steps = 0;
  int n_flags = 0;
  int sm_E = 0, sm_R = 0, sm_C = 0, sm_V = 0, sm_P = 0, sm_X = 0, sm_A = 0, sm_A2 = 0;
  int tmem_cols = 0;
  AssetDev* d_assets = nullptr;
  WorkItem* d_items = nullptr;
  int* d_cta = nullptr;
  int* d_flags = nullptr;
  double* d_item_c = nullptr;
  int max_rows = 0;                 // max T*K over the launch's assets
  bool uploaded = false;
};

struct TuneKey {
  std::vector<long long> sig;
  bool operator<(const TuneKey& o) const { return sig < o.sig; }
};
std::mutex g_tune_mu;
std::map<TuneKey, std::pair<int, int>> g_tune_cache;  // (R, block)

}  // namespace

struct esdp_ctx {
  int device = 0;
  int n_sm = 0;
  uint32_t flags = 0;
  std::vector<esdp_asset> assets;
  // concatenated input offsets per asset
  std::vector<long long> off_price, off_trans, off_cost, off_terminal, off_v1;
  long long n_price = 0, n_trans = 0, n_cost = 0, n_terminal = 0, n_v1 = 0;
  // device workspace
  std::vector<void*> allocs;
  float* d_e = nullptr;           // concatenated action energies
  std::vector<long long> off_e;
  std::vector<float> fx_e;        // per asset: fixed-point scale of rho * e_a in the adjoint
  std::vector<float*> d_ev;       // per asset
  std::vector<void*> d_policy;    // per asset (full policy) or nullptr
  std::vector<float*> d_ckpt;     // per asset or nullptr
  std::vector<double*> d_rho;     // per asset [T][K] row sums of trans
  std::vector<double*> d_off;     // per asset [T+2] level c_t
  std::vector<double*> d_evoff;   // per asset [T][K] EV_t - EV'_t
  std::vector<float*> d_refh;     // per asset [T+2] reference EV' entries
  std::vector<float*> d_ptrans;   // per asset [T][K][Kp4] transposed transition matrices
  float* d_in_price = nullptr;    // host-mode input copies
  float* d_in_trans = nullptr;
  float* d_in_cost = nullptr;
  float* d_in_terminal = nullptr;
  float* d_v1 = nullptr;          // host-mode V1
  float* d_obj_mu = nullptr;      // host-mode esdp_objective staging: mu0 (max K floats)
  double* d_obj_J = nullptr;      // ... and J
  int* d_status = nullptr;
  void* bid_scr = nullptr;        // bid-curve scratch (host-mode outputs, packed form), grown on demand
  size_t bid_scr_bytes = 0;
  void* grad_scr = nullptr;       // esdp_grad workspace, grown on demand
  size_t grad_scr_bytes = 0;
  // inputs of the last solve (device pointers)
  const float* last_price = nullptr;
  const float* last_trans = nullptr;
  const float* last_cost = nullptr;
  const float* last_terminal = nullptr;
  const float* last_v1 = nullptr;
  bool solved = false;
  std::vector<int> prep_tc;       // per asset: tc flag of its last P preparation (-1: none)
  Plan main;
  // per asset: launch plans of the gradient's segment re-sweeps, keyed by
  // the number of segments swept together in one launch
  std::vector<std::map<int, Plan>> seg_plans;
  std::string err;
  unsigned long long timeout_ns = 5ull * 1000 * 1000 * 1000;
  // ESDP_TIME_SWEEP: events recorded around the sweep launch of esdp_solve
  cudaEvent_t ev_sweep[2] = {nullptr, nullptr};
  bool sweep_recorded = false;
  // per-CTA phase cycle counters of the last main sweep (ESDP_PHASE_CLOCKS builds)
  unsigned long long* d_phase = nullptr;
  int phase_grid = 0;
};

namespace {

int fail(esdp_ctx* c, int code, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return code;
}

int cuda_fail(esdp_ctx* c, cudaError_t e, const char* what) {
  return fail(c, ESDP_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                                     \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return cuda_fail(c, e_, what);  \
  } while (0)

template <class T>
int dalloc(esdp_ctx* c, T** out, size_t count) {
  *out = nullptr;
  if (count == 0) return ESDP_OK;
  void* p = nullptr;
  cudaError_t e = cudaMalloc(&p, count * sizeof(T));
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(c, ESDP_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T),
                cudaGetErrorString(e));
  }
  c->allocs.push_back(p);
  *out = static_cast<T*>(p);
  return ESDP_OK;
}

size_t mnk_of(const esdp_asset& a) { return (size_t)a.n_modes * a.N * a.K; }

int round_up(int x, int r) { return (x + r - 1) / r * r; }

int validate_asset(esdp_ctx* c, const esdp_asset& a, int i) {
  if (a.T < 1 || a.N < 2 || a.K < 1 || a.A < 1)
    return fail(c, ESDP_EINVAL, "asset %d: T, K, A must be >= 1 and N >= 2", i);
  if (a.N > (1 << 24))  // SoC indices are exact in float32 (bid-curve predicate)
    return fail(c, ESDP_EINVAL, "asset %d: N must be at most 2^24", i);
  if (a.D_dis < 0 || a.D_chg < 0 || a.D_dis + a.D_chg + 1 != a.A)
    return fail(c, ESDP_EINVAL, "asset %d: A must equal D_dis + D_chg + 1", i);
  if (a.D_dis > a.N - 1 || a.D_chg > a.N - 1)
    return fail(c, ESDP_EINVAL, "asset %d: the action band is wider than the SoC grid", i);
  if (a.n_modes != 1 && a.n_modes != 2)
    return fail(c, ESDP_EINVAL, "asset %d: n_modes must be 1 or 2", i);
  if (a.policy_bytes != 0 && a.policy_bytes != 2 && a.policy_bytes != 4)
    return fail(c, ESDP_EINVAL, "asset %d: policy_bytes must be 0, 2 or 4", i);
  if (a.policy_bytes == 2 && a.A > 32767)
    return fail(c, ESDP_EINVAL, "asset %d: int16 policy needs A <= 32767", i);
  if (a.ckpt_every < 0) return fail(c, ESDP_EINVAL, "asset %d: ckpt_every < 0", i);
  if (!(a.eta_c > 0.0 && a.eta_c <= 1.0 && a.eta_d > 0.0 && a.eta_d <= 1.0))
    return fail(c, ESDP_EINVAL, "asset %d: efficiencies must lie in (0, 1]", i);
  if (!(a.s_max > 0.0) || !std::isfinite(a.s_max) || !(a.tau > 0.0) || !std::isfinite(a.switch_cost))
    return fail(c, ESDP_EINVAL, "asset %d: s_max and tau must be positive and finite", i);
  if (a.s0 < 0 || a.s0 >= a.N) return fail(c, ESDP_EINVAL, "asset %d: s0 outside the grid", i);
  if ((long long)a.K * a.K > 16384)
    return fail(c, ESDP_EINVAL, "asset %d: K = %d exceeds the supported 128", i, a.K);
  return ESDP_OK;
}

// ------------------------------------------------------------------ planning

struct AssetChoice {
  int nb, parts, W, n_tiles, rows, rs;
};

int asset_ev_path(const esdp_asset& a, int W) { return ev_path(W, a.n_modes, a.K, ev_force()); }

size_t smem_need(const esdp_asset& a, const AssetChoice& ch, int R) {
  return sweep_smem_layout(a.n_modes, a.K, ch.W, a.A, R, asset_ev_path(a, ch.W) == kEvTc).bytes;
}

int n_chunks_min(const esdp_asset& a, int R) {
  if (a.n_modes == 1) return round_up(a.A, R) / R;
  const int m0 = round_up(a.D_dis + 1, R) / R + round_up(a.D_chg, R) / R;
  const int m1 = round_up(a.D_dis, R) / R + round_up(a.D_chg + 1, R) / R;
  return std::min(m0, m1);
}

// Pick rows per tile and the action split for one asset given the share of
// the grid (CTAs) it should occupy.
bool choose_asset(const esdp_asset& a, int R, int block, double cta_share, AssetChoice* out) {
  const int KM = ((a.K + 1) / 2) * a.n_modes;  // max-plus threads per row block: price-state pairs
  const int nb_max = block / KM;
  if (nb_max < 1) return false;
  const double rows_per_cta = a.N / std::max(cta_share, 1e-9);
  int nb = (int)std::ceil(rows_per_cta / R);
  nb = std::max(1, std::min(nb, nb_max));
  for (; nb >= 1; --nb) {
    AssetChoice ch;
    ch.nb = nb;
    ch.W = nb * R;
    ch.n_tiles = (a.N + ch.W - 1) / ch.W;
    ch.rows = ch.W + a.A + R;
    ch.rs = (a.A + 2 * R) | 1;
    ch.parts = pick_parts(KM * nb, block, n_chunks_min(a, R));
    if (ch.parts < 1) continue;
    const int dmax = std::max(a.D_dis, a.D_chg);
    const int nw = 2 * ((dmax + ch.W - 1) / ch.W) + 1;
    if (nw + 1 > block) continue;  // one thread per neighbour wait + the reference tile
    if (smem_need(a, ch, R) > kSmemLimit) continue;
    *out = ch;
    return true;
  }
  return false;
}

double item_cost(const esdp_asset& a, const AssetChoice& ch, int s0, int s1, int R) {
  const double rows = round_up(s1 - s0, R);
  const double evals = rows * a.K * a.n_modes * a.A;
  const double ev = rows * a.K * a.n_modes * a.K;
  const double stage_fixed = (ch.rows + 2.0 * ch.rs) * a.K * a.n_modes + 2000.0;
  return (evals + 2.0 * ev) / std::max(1, ch.parts) + stage_fixed;
}

int build_plan(esdp_ctx* c, const std::vector<int>& ids, int R, int block, int grid_cap,
               Plan* plan) {
  plan->shape.R = R;
  {
    std::vector<esdp_asset> launch_assets;
    for (int id : ids) launch_assets.push_back(c->assets[id]);
    plan->shape.kh = getenv("ESDP_NO_KH") ? 0 : sweep_kh(launch_assets.begin(), launch_assets.end());
  }
  plan->shape.block = block;
  plan->asset_ids = ids;
  plan->adev.clear();
  plan->items.clear();
  // grid share per asset proportional to its work per stage
  double total = 0;
  for (int id : ids) {
    const esdp_asset& a = c->assets[id];
    total += (double)a.n_modes * a.N * a.K * a.A;
  }
  std::vector<AssetChoice> ch(ids.size());
  int flag_base = 0;
  // the launch's carve-up must hold every asset: take the largest region sizes
  long long need_E = 0, need_R = 0, need_C = 0, need_V = 0, need_P = 0, need_X = 0;
  long long need_A = 0, need_foot = 0;  // tcgen05 operand part; footprint of its 128-row blocks
  int tmem_cols = 0;
  for (size_t j = 0; j < ids.size(); ++j) {
    const esdp_asset& a = c->assets[ids[j]];
    const double work = (double)a.n_modes * a.N * a.K * a.A;
    const double share = grid_cap * work / total;
    if (!choose_asset(a, R, block, share, &ch[j]))
      return fail(c, ESDP_EINVAL,
                  "asset %d (K=%d, modes=%d, A=%d) does not fit a %d-thread tile in shared memory",
                  ids[j], a.K, a.n_modes, a.A, block);
    {
      const bool tc = asset_ev_path(a, ch[j].W) == kEvTc;
      const SweepSmem L = sweep_smem_layout(a.n_modes, a.K, ch[j].W, a.A, R, tc);
      const long long endX = L.X + ((long long)a.n_modes * ch[j].W * a.K + 31) / 32 * 32;
      need_A = std::max<long long>(need_A, L.A2 - L.A);
      if (tc) {
        const long long mw64 = ((long long)a.n_modes * ch[j].W + 63) / 64 * 64;
        need_foot = std::max<long long>(need_foot, mw64 / 8 * (a.K / 4) * kCmA);
        int cols = 32;
        while (cols < a.K) cols *= 2;
        tmem_cols = std::max(tmem_cols, cols);
      }
      need_E = std::max<long long>(need_E, L.Rt - L.E);
      need_R = std::max<long long>(need_R, L.C - L.Rt);
      need_C = std::max<long long>(need_C, L.V - L.C);
      need_V = std::max<long long>(need_V, L.P - L.V);
      need_P = std::max<long long>(need_P, L.X - L.P);
      need_X = std::max<long long>(need_X, endX - L.X);
    }
    AssetDev d{};
    d.T = a.T; d.N = a.N; d.K = a.K; d.A = a.A; d.D_dis = a.D_dis; d.D_chg = a.D_chg;
    d.M = a.n_modes;
    d.policy_bytes = a.policy_bytes;
    d.nb = ch[j].nb; d.parts = ch[j].parts; d.W = ch[j].W; d.n_tiles = ch[j].n_tiles;
    d.flag_base = flag_base;
    const int dmax = std::max(a.D_dis, a.D_chg);
    const int reach = (dmax + d.W - 1) / d.W;
    d.wait_lo = -reach;
    d.wait_hi = reach;
    d.t_hi = a.T; d.t_lo = 1;
    d.rows = ch[j].rows; d.rs = ch[j].rs;
    d.sw = (float)a.switch_cost;
    d.off_price = c->off_price[ids[j]];
    d.off_trans = c->off_trans[ids[j]];
    d.off_cost = c->off_cost[ids[j]];
    d.off_terminal = c->off_terminal[ids[j]];
    d.off_v1 = c->off_v1[ids[j]];
    d.e = c->d_e + c->off_e[ids[j]];
    d.ref_row = a.N / 2;
    d.ref_tile = d.ref_row / d.W;
    d.ref_hist = c->d_refh[ids[j]];
    d.rho = c->d_rho[ids[j]];
    d.off = c->d_off[ids[j]];
    d.evoff = c->d_evoff[ids[j]];
    d.c_start = nullptr;
    d.ptrans = c->d_ptrans[ids[j]];
    {
      // the prep kernel lays P out for the path of the plan that runs it
      const int path = asset_ev_path(a, d.W);
      d.tc = (d.ptrans != nullptr && path == kEvTc) ? 1 : 0;
      d.mma = path == kEvMma ? 1 : 0;
    }
    plan->max_rows = std::max(plan->max_rows, a.T * a.K);
    plan->adev.push_back(d);
    for (int tI = 0; tI < d.n_tiles; ++tI) {
      WorkItem w;
      w.asset = (int)j;
      w.tile = tI;
      w.s0 = tI * d.W;
      w.s1 = std::min(a.N, w.s0 + d.W);
      plan->items.push_back(w);
    }
    flag_base += d.n_tiles;
  }
  plan->n_flags = flag_base;
  if (plan->shape.kh == 0)
    for (const AssetDev& d : plan->adev)
      if ((d.K & 3) != 0 || d.parts == 1) {
        plan->shape.kh = -1;
        break;
      }
  plan->sm_A = 0;
  plan->sm_A2 = (int)need_A;
  plan->sm_E = 2 * (int)need_A;
  plan->sm_R = plan->sm_E + (int)need_E;
  plan->sm_C = plan->sm_R + (int)need_R;
  plan->sm_V = plan->sm_C + (int)need_C;
  plan->sm_P = plan->sm_V + (int)need_V;
  plan->sm_X = plan->sm_P + (int)need_P;
  plan->tmem_cols = tmem_cols;
  plan->shape.smem =
      (size_t)std::max<long long>(plan->sm_X + need_X, plan->sm_A2 + need_foot) * sizeof(float);
  if (plan->shape.smem > kSmemLimit)
    return fail(c, ESDP_EINVAL, "shared memory plan of %zu bytes exceeds the limit",
                plan->shape.smem);
  // co-resident grid (cooperative launch) and LPT assignment of the items
  int per_sm = sweep_max_blocks_per_sm(R, plan->shape.kh, block, plan->shape.smem);
  if (per_sm < 1) return fail(c, ESDP_EINVAL, "sweep kernel does not fit on an SM");
  int grid = std::min((int)plan->items.size(), std::min(grid_cap, per_sm * c->n_sm));
  grid = std::max(grid, 1);
  plan->shape.grid = grid;
  std::vector<int> order(plan->items.size());
  std::iota(order.begin(), order.end(), 0);
  std::vector<double> cost(plan->items.size());
  for (size_t i = 0; i < plan->items.size(); ++i) {
    const WorkItem& w = plan->items[i];
    cost[i] = item_cost(c->assets[ids[w.asset]], ch[w.asset], w.s0, w.s1, R) *
              c->assets[ids[w.asset]].T;
  }
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
  using Slot = std::pair<double, int>;
  std::priority_queue<Slot, std::vector<Slot>, std::greater<Slot>> heap;
  for (int g = 0; g < grid; ++g) heap.push({0.0, g});
  std::vector<std::vector<int>> per(grid);
  for (int i : order) {
    Slot s = heap.top();
    heap.pop();
    per[s.second].push_back(i);
    heap.push({s.first + cost[i], s.second});
  }
  std::vector<WorkItem> items;
  plan->cta_items.assign(grid + 1, 0);
  for (int g = 0; g < grid; ++g) {
    // items of one CTA in (asset, tile) order
    std::sort(per[g].begin(), per[g].end());
    for (int i : per[g]) items.push_back(plan->items[i]);
    plan->cta_items[g + 1] = (int)items.size();
  }
  plan->items = items;
  plan->n_steps = 0;
  for (const AssetDev& d : plan->adev) plan->n_steps = std::max(plan->n_steps, d.t_hi - d.t_lo + 1);
  plan->uploaded = false;
  return ESDP_OK;
}

void free_plan(Plan* p) {
  cudaFree(p->d_assets);
  cudaFree(p->d_items);
  cudaFree(p->d_cta);
  cudaFree(p->d_flags);
  cudaFree(p->d_item_c);
  p->d_item_c = nullptr;
  p->d_assets = nullptr;
  p->d_items = nullptr;
  p->d_cta = nullptr;
  p->d_flags = nullptr;
  p->uploaded = false;
}

int upload_plan(esdp_ctx* c, Plan* p, cudaStream_t st) {
  if (!p->d_assets) {
    CK(cudaMalloc(&p->d_assets, p->adev.size() * sizeof(AssetDev)), "cudaMalloc plan");
    CK(cudaMalloc(&p->d_items, p->items.size() * sizeof(WorkItem)), "cudaMalloc plan");
    CK(cudaMalloc(&p->d_cta, p->cta_items.size() * sizeof(int)), "cudaMalloc plan");
    CK(cudaMalloc(&p->d_flags, std::max(1, p->n_flags) * sizeof(int)), "cudaMalloc plan");
    CK(cudaMalloc(&p->d_item_c, std::max<size_t>(1, p->items.size()) * sizeof(double)),
       "cudaMalloc plan");
  }
  CK(cudaMemcpyAsync(p->d_assets, p->adev.data(), p->adev.size() * sizeof(AssetDev),
                     cudaMemcpyHostToDevice, st), "upload plan");
  CK(cudaMemcpyAsync(p->d_items, p->items.data(), p->items.size() * sizeof(WorkItem),
                     cudaMemcpyHostToDevice, st), "upload plan");
  CK(cudaMemcpyAsync(p->d_cta, p->cta_items.data(), p->cta_items.size() * sizeof(int),
                     cudaMemcpyHostToDevice, st), "upload plan");
  // the host vectors must outlive the copies
  CK(cudaStreamSynchronize(st), "upload plan");
  p->uploaded = true;
  return ESDP_OK;
}

// prep = false: the row sums and the prepared P of the plan's assets are
// already in place (a gradient re-sweep of the last solve's inputs).
// d_assets: the plan's asset descriptors on the device, when not the plan's
// own uploaded copy (the gradient's per-segment descriptors).
int run_plan(esdp_ctx* c, Plan* p, const float* price, const float* trans, const float* cost,
             const float* terminal, float* v1, cudaStream_t st, bool prep = true,
             const AssetDev* d_assets = nullptr) {
  if (!p->uploaded) {
    int rc = upload_plan(c, p, st);
    if (rc) return rc;
  }
  SweepParams sp{};
  sp.assets = d_assets ? d_assets : p->d_assets;
  sp.items = p->d_items;
  sp.cta_items = p->d_cta;
  sp.price = price;
  sp.trans = trans;
  sp.cost = cost;
  sp.terminal = terminal;
  sp.v1 = v1;
  sp.n_steps = p->n_steps;
  sp.flags = p->d_flags;
  sp.status = c->d_status;
  sp.timeout_ns = c->timeout_ns;
  // test hook: make every wait of the next launches run into its time limit
  sp.wait_extra = getenv("ESDP_INJECT_STALL") ? 1000000 : 0;
  sp.item_c = p->d_item_c;
  sp.sm_E = p->sm_E;
  sp.sm_R = p->sm_R;
  sp.sm_C = p->sm_C;
  sp.sm_V = p->sm_V;
  sp.sm_P = p->sm_P;
  sp.sm_X = p->sm_X;
  sp.sm_A = p->sm_A;
  sp.sm_A2 = p->sm_A2;
  sp.tmem_cols = p->tmem_cols;
  CK(cudaMemsetAsync(p->d_flags, 0, std::max(1, p->n_flags) * sizeof(int), st), "reset flags");
  // a gradient's segment re-sweeps keep the status word of the whole call
  // (reset once by esdp_grad), so an earlier segment's error is not lost
  if (!d_assets) CK(cudaMemsetAsync(c->d_status, 0, sizeof(int), st), "reset status");
  if (prep) {
    CK(launch_rowsums(p->d_assets, (int)p->adev.size(), p->max_rows, trans, st), "row sums");
    for (size_t j = 0; j < p->adev.size(); ++j) c->prep_tc[p->asset_ids[j]] = p->adev[j].tc;
  }
#ifdef ESDP_PHASE_CLOCKS
  if (p == &c->main) {
    if (c->phase_grid < p->shape.grid) {
      cudaFree(c->d_phase);
      c->d_phase = nullptr;
      c->phase_grid = 0;
      CK(cudaMalloc(&c->d_phase, (size_t)p->shape.grid * (kPhases + 1) * 8), "phase counters");
      c->phase_grid = p->shape.grid;
    }
    CK(cudaMemsetAsync(c->d_phase, 0, (size_t)c->phase_grid * (kPhases + 1) * 8, st),
       "phase counters");
    sp.phase_clk = c->d_phase;
  }
#endif
  const bool timed = p == &c->main && c->ev_sweep[0] != nullptr;
  if (timed) CK(cudaEventRecord(c->ev_sweep[0], st), "sweep timing event");
  CK(launch_sweep(p->shape, sp, st), "sweep launch");
  if (timed) {
    CK(cudaEventRecord(c->ev_sweep[1], st), "sweep timing event");
    c->sweep_recorded = true;
  }
  return ESDP_OK;
}

// Fill the buffer pointers of a main-launch asset.
void bind_main(esdp_ctx* c, Plan* p) {
  for (size_t j = 0; j < p->adev.size(); ++j) {
    const int id = p->asset_ids[j];
    const esdp_asset& a = c->assets[id];
    AssetDev& d = p->adev[j];
    d.t_hi = a.T;
    d.t_lo = 1;
    d.v_start = nullptr;
    d.ev = c->d_ev[id];
    d.ev_keep = (c->flags & ESDP_KEEP_EV) ? 1 : 0;
    d.policy = c->d_policy[id];
    d.policy_bytes = c->d_policy[id] ? a.policy_bytes : 0;
    d.policy_t_base = 1;
    d.ckpt_every = a.ckpt_every;
    d.ckpt = c->d_ckpt[id];
    d.v_keep = nullptr;
  }
  p->n_steps = 0;
  for (const AssetDev& d : p->adev) p->n_steps = std::max(p->n_steps, d.t_hi - d.t_lo + 1);
  p->uploaded = false;
}

std::vector<long long> signature(const esdp_ctx* c, const std::vector<int>& ids) {
  std::vector<long long> s;
  for (int id : ids) {
    const esdp_asset& a = c->assets[id];
    s.insert(s.end(), {a.T, a.N, a.K, a.A, a.D_dis, a.n_modes});
  }
  s.push_back(c->n_sm);
  return s;
}

int plan_default(esdp_ctx* c, const std::vector<int>& ids, Plan* plan) {
  // cached autotune result first
  {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    auto it = g_tune_cache.find(TuneKey{signature(c, ids)});
    if (it != g_tune_cache.end())
      return build_plan(c, ids, it->second.first, it->second.second, c->n_sm, plan);
  }
  // heuristic: largest thread-row window that keeps every SM busy
  int best_rc = ESDP_EINVAL;
  double best_score = 1e300;
  Plan best;
  for (int R : {8, 10, 12, 9, 6, 4}) {
    for (int block : {256, 512, 384, 128}) {
      Plan p;
      std::string keep = c->err;
      int rc = build_plan(c, ids, R, block, c->n_sm, &p);
      if (rc) {
        c->err = keep;
        continue;
      }
      // modelled time: max CTA load, with a mild preference for larger R
      std::vector<double> load(p.shape.grid, 0.0);
      for (int g = 0; g < p.shape.grid; ++g)
        for (int i = p.cta_items[g]; i < p.cta_items[g + 1]; ++i) {
          const WorkItem& w = p.items[i];
          const esdp_asset& a = c->assets[ids[w.asset]];
          AssetChoice ch{p.adev[w.asset].nb, p.adev[w.asset].parts, p.adev[w.asset].W,
                         p.adev[w.asset].n_tiles, p.adev[w.asset].rows, p.adev[w.asset].rs};
          load[g] += item_cost(a, ch, w.s0, w.s1, R) * a.T;
        }
      double mx = *std::max_element(load.begin(), load.end());
      const double util = 1.0 + 3.0 / R;  // loads + argmax per evaluation
      const double score = mx * util;
      if (score < best_score) {
        best_score = score;
        best = p;
        best_rc = ESDP_OK;
      }
    }
  }
  if (best_rc) return fail(c, ESDP_EINVAL, "no launch shape fits these assets");
  *plan = best;
  return ESDP_OK;
}

int scan_inputs(esdp_ctx* c, const float* price, const float* trans, const float* cost,
                const float* terminal) {
  for (long long i = 0; i < c->n_price; ++i)
    if (!std::isfinite(price[i])) return fail(c, ESDP_EINVAL, "price[%lld] is not finite", i);
  for (long long i = 0; i < c->n_cost; ++i)
    if (!std::isfinite(cost[i])) return fail(c, ESDP_EINVAL, "cost[%lld] is not finite", i);
  for (long long i = 0; i < c->n_terminal; ++i)
    if (!std::isfinite(terminal[i]))
      return fail(c, ESDP_EINVAL, "terminal[%lld] is not finite", i);
  for (size_t id = 0; id < c->assets.size(); ++id) {
    const esdp_asset& a = c->assets[id];
    const float* P = trans + c->off_trans[id];
    for (long long r = 0; r < (long long)a.T * a.K; ++r) {
      double sum = 0;
      for (int k2 = 0; k2 < a.K; ++k2) {
        const float v = P[r * a.K + k2];
        if (!std::isfinite(v) || v < 0.f)
          return fail(c, ESDP_EINVAL, "asset %zu: transition entry %lld is negative or not finite",
                      id, r * a.K + k2);
        sum += v;
      }
      if ((c->flags & ESDP_CHECK_ROWS) && std::fabs(sum - 1.0) > 1e-5)
        return fail(c, ESDP_EINVAL, "asset %zu: transition row %lld sums to %.8f", id, r, sum);
    }
  }
  return ESDP_OK;
}

}  // namespace

// =================================================================== C ABI

extern "C" {

int esdp_version(void) { return 1; }

const char* esdp_last_error(const esdp_ctx* c) {
  return c ? c->err.c_str() : "no context";
}

int esdp_create(const esdp_asset* assets, int32_t n_assets, uint32_t flags, esdp_ctx** out) {
  if (!out) return ESDP_EINVAL;
  *out = nullptr;
  if (!assets || n_assets < 1) return ESDP_EINVAL;
  esdp_ctx* c = new (std::nothrow) esdp_ctx;
  if (!c) return ESDP_ENOMEM;
  *out = c;
  c->flags = flags;
  c->assets.assign(assets, assets + n_assets);
  for (int i = 0; i < n_assets; ++i) {
    int rc = validate_asset(c, c->assets[i], i);
    if (rc) return rc;
  }
  if (const char* env = getenv("ESDP_TIMEOUT_MS")) {
    const long long ms = atoll(env);
    if (ms > 0) c->timeout_ns = (unsigned long long)ms * 1000000ull;
  }
  if (getenv("ESDP_FAIL_ALLOC")) return fail(c, ESDP_ENOMEM, "allocation failure injected");
  CK(cudaGetDevice(&c->device), "cudaGetDevice");
  if (flags & ESDP_TIME_SWEEP) {
    CK(cudaEventCreate(&c->ev_sweep[0]), "sweep timing event");
    CK(cudaEventCreate(&c->ev_sweep[1]), "sweep timing event");
  }
  int coop = 0;
  CK(cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, c->device), "device attribute");
  if (!coop) return fail(c, ESDP_ECUDA, "device has no cooperative launch support");
  CK(cudaDeviceGetAttribute(&c->n_sm, cudaDevAttrMultiProcessorCount, c->device), "SM count");
  // offsets of the concatenated arrays
  long long op = 0, ot = 0, oc = 0, om = 0, oe = 0;
  for (const esdp_asset& a : c->assets) {
    c->off_price.push_back(op);
    c->off_trans.push_back(ot);
    c->off_cost.push_back(oc);
    c->off_terminal.push_back(om);
    c->off_v1.push_back(om);
    c->off_e.push_back(oe);
    op += (long long)a.T * a.K;
    ot += (long long)a.T * a.K * a.K;
    oc += a.A;
    om += (long long)mnk_of(a);
    oe += a.A;
  }
  c->n_price = op;
  c->n_trans = ot;
  c->n_cost = oc;
  c->n_terminal = om;
  c->n_v1 = om;
  int rc;
  // action energies (eq. 2), computed in double and rounded once
  std::vector<float> e(oe);
  for (size_t id = 0; id < c->assets.size(); ++id) {
    const esdp_asset& a = c->assets[id];
    const double delta = a.s_max / (double)(a.N - 1);
    for (int j = 0; j < a.A; ++j) {
      const int d = j - a.D_dis;
      double en = 0.0;
      if (d < 0) en = -(double)d * delta * a.eta_d;
      if (d > 0) en = -(double)d * delta / a.eta_c;
      e[c->off_e[id] + j] = (float)en;
    }
    // 2^(32 - ceil(log2 max|e_a|)): |rho e_a| in these units stays below |rho| 2^32
    float emax = 0.f;
    for (int j = 0; j < a.A; ++j) emax = std::max(emax, std::fabs(e[c->off_e[id] + j]));
    int ex = 0;
    if (emax > 0.f) std::frexp(emax, &ex);
    c->fx_e.push_back(std::ldexp(1.f, 32 - ex));
  }
  if ((rc = dalloc(c, &c->d_e, e.size()))) return rc;
  CK(cudaMemcpy(c->d_e, e.data(), e.size() * sizeof(float), cudaMemcpyHostToDevice), "copy e");
  if ((rc = dalloc(c, &c->d_status, 1))) return rc;
  CK(cudaMemset(c->d_status, 0, sizeof(int)), "status");
  for (const esdp_asset& a : c->assets) {
    float* ev = nullptr;
    const size_t L = mnk_of(a);
    if ((rc = dalloc(c, &ev, (flags & ESDP_KEEP_EV) ? L * a.T : 2 * L))) return rc;
    c->d_ev.push_back(ev);
    void* pol = nullptr;
    if (a.policy_bytes > 0 && a.ckpt_every == 0) {
      char* pp = nullptr;
      if ((rc = dalloc(c, &pp, L * a.T * a.policy_bytes))) return rc;
      pol = pp;
    }
    c->d_policy.push_back(pol);
    float* ck = nullptr;
    if (a.ckpt_every > 0 && a.T > a.ckpt_every) {
      const int nck = (a.T - 1) / a.ckpt_every;
      if ((rc = dalloc(c, &ck, L * nck))) return rc;
    }
    c->d_ckpt.push_back(ck);
    double *rho = nullptr, *off = nullptr, *evoff = nullptr;
    float* refh = nullptr;
    if ((rc = dalloc(c, &rho, (size_t)a.T * a.K))) return rc;
    if ((rc = dalloc(c, &off, (size_t)a.T + 2))) return rc;
    if ((rc = dalloc(c, &evoff, (size_t)a.T * a.K))) return rc;
    if ((rc = dalloc(c, &refh, (size_t)a.T + 2))) return rc;
    c->d_rho.push_back(rho);
    c->d_off.push_back(off);
    c->d_evoff.push_back(evoff);
    c->d_refh.push_back(refh);
    float* pt = nullptr;
    // room for either layout: the tile size of the plan picks the EV path
    const size_t per = std::max(tc_shape(a.K) ? 2 * (size_t)a.K * a.K : (size_t)0,
                                (size_t)a.K * p_stride(a.K));
    if ((rc = dalloc(c, &pt, (size_t)a.T * per))) return rc;
    c->d_ptrans.push_back(pt);
  }
  if (!(flags & ESDP_DEVICE_PTRS)) {
    if ((rc = dalloc(c, &c->d_in_price, c->n_price))) return rc;
    if ((rc = dalloc(c, &c->d_in_trans, c->n_trans))) return rc;
    if ((rc = dalloc(c, &c->d_in_cost, c->n_cost))) return rc;
    if ((rc = dalloc(c, &c->d_in_terminal, c->n_terminal))) return rc;
  }
  // V_1 lands here when the caller passes no output (the gradient needs it)
  if ((rc = dalloc(c, &c->d_v1, c->n_v1))) return rc;
  int k_max = 1;
  for (const esdp_asset& a : c->assets) k_max = std::max(k_max, (int)a.K);
  if ((rc = dalloc(c, &c->d_obj_mu, (size_t)k_max))) return rc;
  if ((rc = dalloc(c, &c->d_obj_J, (size_t)1))) return rc;
  std::vector<int> ids(c->assets.size());
  std::iota(ids.begin(), ids.end(), 0);
  if ((rc = plan_default(c, ids, &c->main))) return rc;
  bind_main(c, &c->main);
  c->seg_plans.resize(c->assets.size());
  c->prep_tc.assign(c->assets.size(), -1);
  return ESDP_OK;
}

int esdp_sweep_ms(esdp_ctx* c, float* ms) {
  if (!c || !ms) return ESDP_EINVAL;
  if (!c->ev_sweep[0]) return fail(c, ESDP_ESTATE, "context made without ESDP_TIME_SWEEP");
  if (!c->sweep_recorded) return fail(c, ESDP_ESTATE, "no sweep launched yet");
  CK(cudaEventSynchronize(c->ev_sweep[1]), "sweep timing");
  CK(cudaEventElapsedTime(ms, c->ev_sweep[0], c->ev_sweep[1]), "sweep timing");
  return ESDP_OK;
}

int esdp_phase_clocks(esdp_ctx* c, double* cycles, int32_t n_phases) {
  if (!c || !cycles || n_phases < kPhases) return ESDP_EINVAL;
#ifdef ESDP_PHASE_CLOCKS
  if (!c->d_phase || !c->solved) return fail(c, ESDP_ESTATE, "no instrumented sweep has run");
  std::vector<unsigned long long> h((size_t)c->phase_grid * (kPhases + 1));
  CK(cudaDeviceSynchronize(), "phase counters");
  CK(cudaMemcpy(h.data(), c->d_phase, h.size() * 8, cudaMemcpyDeviceToHost), "phase counters");
  double stages = 0;
  std::vector<double> sum(kPhases, 0.0);
  for (int g = 0; g < c->phase_grid; ++g) {
    stages += (double)h[(size_t)g * (kPhases + 1) + kPhases];
    for (int i = 0; i < kPhases; ++i) sum[i] += (double)h[(size_t)g * (kPhases + 1) + i];
  }
  for (int i = 0; i < kPhases; ++i) cycles[i] = stages > 0 ? sum[i] / stages : 0.0;
  return ESDP_OK;
#else
  (void)cycles;
  return fail(c, ESDP_ESTATE, "library built without ESDP_PHASE_CLOCKS");
#endif
}

void esdp_destroy(esdp_ctx* c) {
  if (!c) return;
  cudaDeviceSynchronize();
  cudaFree(c->d_phase);
  for (cudaEvent_t& e : c->ev_sweep)
    if (e) cudaEventDestroy(e);
  free_plan(&c->main);
  for (auto& m : c->seg_plans)
    for (auto& kv : m) free_plan(&kv.second);
  for (void* p : c->allocs) cudaFree(p);
  cudaFree(c->bid_scr);
  cudaFree(c->grad_scr);
  delete c;
}

int esdp_solve(esdp_ctx* c, const float* price, const float* trans, const float* cost,
               const float* terminal, float* V1, void* stream) {
  if (!c) return ESDP_EINVAL;
  if (!price || !trans || !cost || !terminal) return fail(c, ESDP_EINVAL, "null input array");
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = (c->flags & ESDP_DEVICE_PTRS) != 0;
  const float *dp = price, *dt = trans, *dc = cost, *dm = terminal;
  float* dv = V1 ? V1 : c->d_v1;
  if (!dev) {
    if (!(c->flags & ESDP_NO_VALIDATE)) {
      int rc = scan_inputs(c, price, trans, cost, terminal);
      if (rc) return rc;
    }
    CK(cudaMemcpyAsync(c->d_in_price, price, c->n_price * 4, cudaMemcpyHostToDevice, st), "H2D");
    CK(cudaMemcpyAsync(c->d_in_trans, trans, c->n_trans * 4, cudaMemcpyHostToDevice, st), "H2D");
    CK(cudaMemcpyAsync(c->d_in_cost, cost, c->n_cost * 4, cudaMemcpyHostToDevice, st), "H2D");
    CK(cudaMemcpyAsync(c->d_in_terminal, terminal, c->n_terminal * 4, cudaMemcpyHostToDevice, st),
       "H2D");
    dp = c->d_in_price;
    dt = c->d_in_trans;
    dc = c->d_in_cost;
    dm = c->d_in_terminal;
    dv = c->d_v1;
  }
  int rc = run_plan(c, &c->main, dp, dt, dc, dm, dv, st);
  if (rc) return rc;
  if (c->flags & ESDP_KEEP_EV) {
    // the kept EV'_t become the reported EV_t (level added back, in double)
    for (size_t id = 0; id < c->assets.size(); ++id) {
      const esdp_asset& a = c->assets[id];
      CK(launch_ev_restore(c->d_ev[id], c->d_evoff[id], a.T, a.n_modes * a.N, a.K, st),
         "EV restore");
    }
  }
  c->last_price = dp;
  c->last_trans = dt;
  c->last_cost = dc;
  c->last_terminal = dm;
  c->last_v1 = dv;
  c->solved = true;
  if (!dev) {
    if (V1) CK(cudaMemcpyAsync(V1, c->d_v1, c->n_v1 * 4, cudaMemcpyDeviceToHost, st), "D2H");
    int status = 0;
    CK(cudaMemcpyAsync(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost, st), "D2H");
    CK(cudaStreamSynchronize(st), "solve");
    if (status) {
      c->solved = false;
      return fail(c, status, "device reported status %d during the sweep", status);
    }
    if (V1)
      for (long long i = 0; i < c->n_v1; ++i)
        if (std::isnan(V1[i])) return fail(c, ESDP_ENUMERIC, "V1[%lld] is NaN", i);
  }
  return ESDP_OK;
}

int esdp_status(esdp_ctx* c, void* stream) {
  if (!c) return ESDP_EINVAL;
  int status = 0;
  CK(cudaMemcpyAsync(&status, c->d_status, sizeof(int), cudaMemcpyDeviceToHost,
                     (cudaStream_t)stream), "status");
  CK(cudaStreamSynchronize((cudaStream_t)stream), "status");
  return status;
}

int esdp_launch_info(const esdp_ctx* c, int32_t* grid, int32_t* block, int32_t* items,
                     int32_t* rows_per_tile, int32_t* parts, int32_t* rows_per_thread,
                     int32_t* ev_path) {
  if (!c) return ESDP_EINVAL;
  if (ev_path) {
    const AssetDev* d = c->main.adev.empty() ? nullptr : &c->main.adev[0];
    *ev_path = !d ? -1 : d->tc ? kEvTc : d->mma ? kEvMma : kEvSimt;
  }
  if (grid) *grid = c->main.shape.grid;
  if (block) *block = c->main.shape.block;
  if (items) *items = (int32_t)c->main.items.size();
  if (rows_per_tile) *rows_per_tile = c->main.adev.empty() ? 0 : c->main.adev[0].W;
  if (parts) *parts = c->main.adev.empty() ? 0 : c->main.adev[0].parts;
  if (rows_per_thread) *rows_per_thread = c->main.shape.R;
  return ESDP_OK;
}

static int check_asset_t(esdp_ctx* c, int32_t asset, int32_t t) {
  if (asset < 0 || asset >= (int32_t)c->assets.size())
    return fail(c, ESDP_EINVAL, "asset index %d out of range", asset);
  if (t < 1 || t > c->assets[asset].T) return fail(c, ESDP_EINVAL, "stage %d out of range", t);
  if (!c->solved) return fail(c, ESDP_ESTATE, "no solve has completed");
  return ESDP_OK;
}

int esdp_policy(esdp_ctx* c, int32_t asset, int32_t t, void* out, void* stream) {
  if (!c || !out) return ESDP_EINVAL;
  int rc = check_asset_t(c, asset, t);
  if (rc) return rc;
  if (!c->d_policy[asset])
    return fail(c, ESDP_ESTATE, "the context keeps no full policy for asset %d", asset);
  const esdp_asset& a = c->assets[asset];
  const size_t bytes = mnk_of(a) * a.policy_bytes;
  const char* src = static_cast<const char*>(c->d_policy[asset]) + (size_t)(t - 1) * bytes;
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = (c->flags & ESDP_DEVICE_PTRS) != 0;
  CK(cudaMemcpyAsync(out, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st),
     "policy copy");
  if (!dev) CK(cudaStreamSynchronize(st), "policy copy");
  return ESDP_OK;
}

int esdp_expected_value(esdp_ctx* c, int32_t asset, int32_t t, float* out, void* stream) {
  if (!c || !out) return ESDP_EINVAL;
  int rc = check_asset_t(c, asset, t);
  if (rc) return rc;
  if (!(c->flags & ESDP_KEEP_EV)) return fail(c, ESDP_ESTATE, "context made without ESDP_KEEP_EV");
  const esdp_asset& a = c->assets[asset];
  const size_t L = mnk_of(a);
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = (c->flags & ESDP_DEVICE_PTRS) != 0;
  CK(cudaMemcpyAsync(out, c->d_ev[asset] + (size_t)(t - 1) * L, L * 4,
                     dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st), "EV copy");
  if (!dev) CK(cudaStreamSynchronize(st), "EV copy");
  return ESDP_OK;
}

namespace {

// Device scratch of the bid-curve entry points: grown on demand (the free of
// a smaller one synchronises the device), kept until esdp_destroy.
void* bid_scratch(esdp_ctx* c, size_t bytes) {
  if (bytes <= c->bid_scr_bytes) return c->bid_scr;
  cudaFree(c->bid_scr);
  c->bid_scr = nullptr;
  c->bid_scr_bytes = 0;
  void* p = nullptr;
  if (getenv("ESDP_FAIL_ALLOC") || cudaMalloc(&p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  c->bid_scr = p;
  c->bid_scr_bytes = bytes;
  return p;
}

int check_bid_call(esdp_ctx* c, int32_t asset, int32_t t0, int32_t t1) {
  if (asset < 0 || asset >= (int32_t)c->assets.size())
    return fail(c, ESDP_EINVAL, "asset index %d out of range", asset);
  const esdp_asset& a = c->assets[asset];
  if (t0 < 1 || t1 > a.T + 1 || t1 <= t0) return fail(c, ESDP_EINVAL, "bad stage range");
  if (!c->solved) return fail(c, ESDP_ESTATE, "no solve has completed");
  if (!(c->flags & ESDP_KEEP_EV)) return fail(c, ESDP_ESTATE, "context made without ESDP_KEEP_EV");
  return ESDP_OK;
}

cudaError_t run_hull(esdp_ctx* c, int32_t asset, int32_t t0, int32_t t1, int* d_n, int* d_idx,
                     float* d_sl, cudaStream_t st) {
  const esdp_asset& a = c->assets[asset];
  HullParams hp{};
  hp.ev = c->d_ev[asset] + (size_t)(t0 - 1) * mnk_of(a);
  hp.n_t = t1 - t0;
  hp.M = a.n_modes;
  hp.N = a.N;
  hp.K = a.K;
  hp.delta = a.s_max / (double)(a.N - 1);
  hp.n_bp = d_n;
  hp.idx = d_idx;
  hp.slope = d_sl;
  return launch_hull(hp, st);
}

}  // namespace

int esdp_bid_curves(esdp_ctx* c, int32_t asset, int32_t t0, int32_t t1, int32_t* n_bp,
                    int32_t* bp_idx, float* slope, void* stream) {
  if (!c || !n_bp || !bp_idx || !slope) return ESDP_EINVAL;
  int rc = check_bid_call(c, asset, t0, t1);
  if (rc) return rc;
  const esdp_asset& a = c->assets[asset];
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = (c->flags & ESDP_DEVICE_PTRS) != 0;
  const size_t nh = (size_t)(t1 - t0) * a.n_modes * a.K;
  int* d_n = n_bp;
  int* d_idx = bp_idx;
  float* d_sl = slope;
  if (!dev) {
    char* scr = (char*)bid_scratch(c, nh * 4 * (1 + 2 * (size_t)a.N));
    if (!scr) return fail(c, ESDP_ENOMEM, "bid-curve scratch allocation failed");
    d_n = (int*)scr;
    d_idx = d_n + nh;
    d_sl = (float*)(d_idx + nh * a.N);
  }
  cudaError_t e = run_hull(c, asset, t0, t1, d_n, d_idx, d_sl, st);
  if (e == cudaSuccess && !dev) {
    e = cudaMemcpyAsync(n_bp, d_n, nh * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(bp_idx, d_idx, nh * a.N * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(slope, d_sl, nh * a.N * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "bid curves");
  return ESDP_OK;
}

int esdp_bid_curves_packed(esdp_ctx* c, int32_t asset, int32_t t0, int32_t t1, int64_t* offsets,
                           int32_t* bp_idx, float* slope, int64_t cap, void* stream) {
  if (!c || !offsets || !bp_idx || !slope || cap < 0) return ESDP_EINVAL;
  int rc = check_bid_call(c, asset, t0, t1);
  if (rc) return rc;
  const esdp_asset& a = c->assets[asset];
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = (c->flags & ESDP_DEVICE_PTRS) != 0;
  const size_t nh = (size_t)(t1 - t0) * a.n_modes * a.K;
  const size_t rows = nh * (size_t)a.N;
  // scratch: padded rows (counts, indices, slopes), then in host mode the
  // offsets and the packed arrays (worst case: every point a vertex)
  const size_t pad_bytes = (nh + 2 * rows) * 4;
  const size_t off_at = (pad_bytes + 15) / 16 * 16;
  const size_t bytes = dev ? pad_bytes : off_at + (nh + 1) * 8 + 2 * rows * 4;
  char* scr = (char*)bid_scratch(c, bytes);
  if (!scr) return fail(c, ESDP_ENOMEM, "bid-curve scratch allocation failed");
  int* d_n = (int*)scr;
  int* d_idx = d_n + nh;
  float* d_sl = (float*)(d_idx + rows);
  long long* d_off = (long long*)offsets;
  int* d_pi = bp_idx;
  float* d_ps = slope;
  long long d_cap = cap;
  if (!dev) {
    d_off = (long long*)(scr + off_at);
    d_pi = (int*)(d_off + nh + 1);
    d_ps = (float*)(d_pi + rows);
    d_cap = (long long)rows;
  }
  cudaError_t e = run_hull(c, asset, t0, t1, d_n, d_idx, d_sl, st);
  if (e == cudaSuccess)
    e = launch_pack_bids(d_n, d_idx, d_sl, a.N, (int)nh, d_off, d_cap, d_pi, d_ps, st);
  if (e == cudaSuccess && !dev) {
    e = cudaMemcpyAsync(offsets, d_off, (nh + 1) * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    if (e == cudaSuccess) {
      const long long total = (long long)offsets[nh];
      if (total > cap)
        return fail(c, ESDP_EINVAL, "cap %lld is below the %lld vertices", (long long)cap, total);
      e = cudaMemcpyAsync(bp_idx, d_pi, (size_t)total * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(slope, d_ps, (size_t)total * 4, cudaMemcpyDeviceToHost, st);
      if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    }
  }
  if (e != cudaSuccess) return cuda_fail(c, e, "packed bid curves");
  return ESDP_OK;
}

int esdp_bids_at(esdp_ctx* c, int32_t asset, int32_t t0, int32_t t1, int32_t s_idx,
                 const int32_t* n_bp, const int32_t* bp_idx, int32_t* n_pts, double* p_mw,
                 float* price, void* stream) {
  if (!c || !n_bp || !bp_idx || !n_pts || !p_mw || !price) return ESDP_EINVAL;
  if (asset < 0 || asset >= (int32_t)c->assets.size())
    return fail(c, ESDP_EINVAL, "asset index %d out of range", asset);
  const esdp_asset& a = c->assets[asset];
  if (t0 < 1 || t1 > a.T + 1 || t1 <= t0) return fail(c, ESDP_EINVAL, "bad stage range");
  if (s_idx < 0 || s_idx >= a.N) return fail(c, ESDP_EINVAL, "SoC index %d outside the grid", s_idx);
  if (!c->solved) return fail(c, ESDP_ESTATE, "no solve has completed");
  if (!(c->flags & ESDP_KEEP_EV)) return fail(c, ESDP_ESTATE, "context made without ESDP_KEEP_EV");
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = (c->flags & ESDP_DEVICE_PTRS) != 0;
  const int n_t = t1 - t0;
  const size_t L = mnk_of(a);
  const size_t nh = (size_t)n_t * a.n_modes * a.K;
  const int* d_nbp = n_bp;
  const int* d_idx = bp_idx;
  int* d_np = n_pts;
  double* d_p = p_mw;
  float* d_pr = price;
  std::vector<void*> tmp;
  if (!dev) {
    const size_t sizes[5] = {nh * 4, nh * a.N * 4, nh * 4, nh * a.A * 8, nh * a.A * 4};
    void* q[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    for (int i = 0; i < 5; ++i)
      if (cudaMalloc(&q[i], sizes[i]) != cudaSuccess) {
        for (void* x : q) cudaFree(x);
        cudaGetLastError();
        return fail(c, ESDP_ENOMEM, "bid allocation failed");
      }
    tmp.assign(q, q + 5);
    d_nbp = (const int*)q[0];
    d_idx = (const int*)q[1];
    d_np = (int*)q[2];
    d_p = (double*)q[3];
    d_pr = (float*)q[4];
    cudaError_t e = cudaMemcpyAsync(q[0], n_bp, sizes[0], cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(q[1], bp_idx, sizes[1], cudaMemcpyHostToDevice, st);
    if (e != cudaSuccess) {
      for (void* x : tmp) cudaFree(x);
      return cuda_fail(c, e, "bid inputs");
    }
  }
  BidsAtParams bp{};
  bp.ev = c->d_ev[asset] + (size_t)(t0 - 1) * L;
  bp.n_bp = d_nbp;
  bp.idx = d_idx;
  bp.n_t = n_t;
  bp.M = a.n_modes;
  bp.N = a.N;
  bp.K = a.K;
  bp.s = s_idx;
  bp.D_dis = a.D_dis;
  bp.D_chg = a.D_chg;
  bp.A = a.A;
  bp.delta = a.s_max / (double)(a.N - 1);
  bp.eta_c = a.eta_c;
  bp.eta_d = a.eta_d;
  bp.tau = a.tau;
  bp.n_pts = d_np;
  bp.p_mw = d_p;
  bp.price = d_pr;
  cudaError_t e = launch_bids_at(bp, st);
  if (e == cudaSuccess && !dev) {
    e = cudaMemcpyAsync(n_pts, d_np, nh * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(p_mw, d_p, nh * a.A * 8, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(price, d_pr, nh * a.A * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  }
  for (void* x : tmp) cudaFree(x);
  if (e != cudaSuccess) return cuda_fail(c, e, "bids at a SoC state");
  return ESDP_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ adjoint

namespace {

__global__ void objective_kernel(const float* v1, const float* mu0, int K, int s0, double* J) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    double acc = 0.0;
    for (int k = 0; k < K; ++k) acc += (double)mu0[k] * (double)v1[(size_t)s0 * K + k];
    *J = acc;
  }
}

__global__ void init_rho_kernel(float* rho, const float* mu0, int K, int s0) {
  const int k = threadIdx.x;
  if (k < K) rho[(size_t)s0 * K + k] = mu0[k];
}

__global__ void to_float_kernel(const double* src, float* dst, long long n) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (float)src[i];
}

// The gradient re-sweeps its checkpoint segments B at a time as the assets
// of one persistent launch (they are independent: each starts from its own
// checkpoint), holding the policies, values and post-decision occupancies of
// those B segments at once:
// B = ESDP_GRAD_SEGMENTS, else as many as 1 GiB of slots holds; the groups
// have equal sizes except the last (b_last segments).
void grad_groups(const esdp_asset& a, int* B_out, int* b_last_out, int* nseg_out) {
  const int T = a.T;
  const int C = a.ckpt_every > 0 ? std::min((int)a.ckpt_every, T) : T;
  const int nseg = (T + C - 1) / C;
  const size_t L = mnk_of(a);
  const int pb = a.policy_bytes > 0 ? a.policy_bytes : 4;
  const size_t slot_bytes = L * C * pb + L * (C + 1) * 4 + L * C * 4 + 2 * L * 4 +
                            (size_t)(T + 2) * 8 + (size_t)C * kDtSplit * (a.K + 1) * a.K * 8;
  int B = (int)std::max<size_t>(1, std::min<size_t>(nseg, (size_t(1) << 30) / slot_bytes));
  if (const char* f = getenv("ESDP_GRAD_SEGMENTS")) B = std::max(1, std::min(nseg, atoi(f)));
  const int ngrp = (nseg + B - 1) / B;
  B = (nseg + ngrp - 1) / ngrp;
  *B_out = B;
  *b_last_out = nseg - (ngrp - 1) * B;
  *nseg_out = nseg;
}

}  // namespace

extern "C" int esdp_grad(esdp_ctx* c, int32_t asset, const float* mu0, double* J,
                         float* d_price, float* d_trans, double* d_eta, float* d_cost,
                         double* d_switch, float* d_terminal, float* d_mu0, void* stream) {
  if (!c || !mu0) return ESDP_EINVAL;
  if (asset < 0 || asset >= (int32_t)c->assets.size())
    return fail(c, ESDP_EINVAL, "asset index %d out of range", asset);
  if (!c->solved) return fail(c, ESDP_ESTATE, "no solve has completed");
  const esdp_asset& a = c->assets[asset];
  cudaStream_t st = (cudaStream_t)stream;
  const bool dev = (c->flags & ESDP_DEVICE_PTRS) != 0;
  const int T = a.T, K = a.K, M = a.n_modes, N = a.N;
  const size_t L = mnk_of(a);
  const int C = a.ckpt_every > 0 ? std::min(a.ckpt_every, T) : T;
  const int nseg = (T + C - 1) / C;
  if (a.ckpt_every > 0 && T > C && !c->d_ckpt[asset])
    return fail(c, ESDP_ESTATE, "no checkpoints kept");
  int rc;
  const int pb = a.policy_bytes > 0 ? a.policy_bytes : 4;
  int B, b_last, nseg_g;
  grad_groups(a, &B, &b_last, &nseg_g);
  const int ngrp = (nseg + B - 1) / B;
  // launch plans of B and of b_last segments (same shape rules as the main plan)
  Plan* gplan[2] = {nullptr, nullptr};
  for (int q = 0; q < 2; ++q) {
    const int b = q == 0 ? B : b_last;
    Plan& pl = c->seg_plans[asset][b];
    if (pl.adev.empty() && (rc = plan_default(c, std::vector<int>(b, asset), &pl))) return rc;
    gplan[q] = &pl;
  }
  // workspace: carved from the context's gradient scratch (kept across calls)
  void *seg_pol, *seg_v, *seg_post, *rho, *ev2, *dprice64, *acc, *bar, *d_mu, *dJ, *dtr, *dpr,
      *dcost64, *dco, *opart, *opart_cost, *opart_acc, *dsegs, *dtpart, *dtmass, *post_fx,
      *seg_off;
  const int MN = M * N;
  int ogrid = std::min(c->n_sm, std::max(1, (MN + 7) / 8));  // occupancy CTAs
  const int orows = (MN + ogrid - 1) / ogrid;
  ogrid = (MN + orows - 1) / orows;
  {
    void** outs[] = {&seg_pol, &seg_v, &seg_post, &rho, &ev2, &dprice64, &acc,
                     &bar, &d_mu, &dJ, &dtr, &dpr, &dcost64, &dco, &opart, &opart_cost,
                     &opart_acc, &dsegs, &dtpart, &dtmass, &post_fx, &seg_off};
    const size_t sizes[] = {L * C * pb * B, L * (C + 1) * 4 * B, L * C * 4 * B, L * 4, 2 * L * 4 * B,
                            (size_t)T * K * 8, 8 * 8, (size_t)ogrid * 4, (size_t)K * 4, 8,
                            (size_t)T * K * K * 4, (size_t)T * K * 4, (size_t)a.A * 8,
                            (size_t)a.A * 4, (size_t)C * ogrid * K * 8,
                            (size_t)ogrid * a.A * 8, (size_t)ogrid * 8 * 8,
                            (size_t)nseg * sizeof(AssetDev), (size_t)C * B * kDtSplit * K * K * 8,
                            (size_t)C * B * kDtSplit * K * 8, L * C * 8, (size_t)(T + 2) * 8 * B};
    size_t total = 0;
    for (size_t sz : sizes) total += (sz + 255) / 256 * 256;
    if (total > c->grad_scr_bytes) {
      cudaFree(c->grad_scr);  // synchronises: no earlier call still uses it
      c->grad_scr = nullptr;
      c->grad_scr_bytes = 0;
      if (getenv("ESDP_FAIL_ALLOC") || cudaMalloc(&c->grad_scr, total) != cudaSuccess) {
        cudaGetLastError();
        c->grad_scr = nullptr;
        return fail(c, ESDP_ENOMEM, "gradient scratch allocation failed");
      }
      c->grad_scr_bytes = total;
    }
    char* q = (char*)c->grad_scr;
    for (int i = 0; i < 22; ++i) {
      *outs[i] = q;
      q += (sizes[i] + 255) / 256 * 256;
    }
  }
  auto release = [&]() { cudaStreamSynchronize(st); };
  auto cfail = [&](cudaError_t e, const char* what) {
    release();
    return cuda_fail(c, e, what);
  };
  cudaError_t e;
  if ((e = cudaMemcpyAsync(d_mu, mu0, K * 4, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                           st)) != cudaSuccess)
    return cfail(e, "mu0 copy");
  cudaMemsetAsync(c->d_status, 0, sizeof(int), st);
  cudaMemsetAsync(rho, 0, L * 4, st);
  cudaMemsetAsync(dprice64, 0, (size_t)T * K * 8, st);
  cudaMemsetAsync(acc, 0, 64, st);
  cudaMemsetAsync(dcost64, 0, (size_t)a.A * 8, st);
  init_rho_kernel<<<1, 128, 0, st>>>((float*)rho, (const float*)d_mu, K, a.s0);
  objective_kernel<<<1, 32, 0, st>>>(c->last_v1 + c->off_v1[asset], (const float*)d_mu, K, a.s0,
                                      (double*)dJ);
  const float* price = c->last_price + c->off_price[asset];
  const float* trans = c->last_trans + c->off_trans[asset];
  const float* cost = c->last_cost + c->off_cost[asset];
  const float* terminal = c->last_terminal + c->off_terminal[asset];
  // the re-sweeps' asset descriptors, one per segment, uploaded together (a
  // host upload per segment would drain the stream before each re-sweep);
  // segment j runs as launch asset j % B of group j / B, in slot j % B of
  // the policy, value, EV and level buffers (the levels the re-sweep writes
  // go to the slot: the solve's own c_t stay as they are)
  std::vector<AssetDev> segs(nseg);
  for (int j = 0; j < nseg; ++j) {
    const int g = j / B, i = j % B;
    const int t_lo = 1 + j * C, t_hi = std::min(T, (j + 1) * C);
    AssetDev& d = segs[j];
    d = gplan[g == ngrp - 1 ? 1 : 0]->adev[i];
    d.t_hi = t_hi;
    d.t_lo = t_lo;
    d.v_start = (t_hi == T) ? nullptr : c->d_ckpt[asset] + (size_t)j * L;
    d.c_start = (t_hi == T) ? nullptr : c->d_off[asset] + t_hi + 1;
    d.ev = (float*)ev2 + (size_t)i * 2 * L;
    d.ev_keep = 0;
    d.policy = (char*)seg_pol + (size_t)i * L * C * pb;
    d.policy_bytes = pb;
    d.policy_t_base = t_lo;
    d.ckpt_every = 0;
    d.ckpt = nullptr;
    d.v_keep = (float*)seg_v + (size_t)i * L * (C + 1);
    d.off = (double*)seg_off + (size_t)i * (T + 2);
  }
  for (Plan* pl : gplan)
    if (!pl->uploaded && (rc = upload_plan(c, pl, st))) {  // once per context
      release();
      return rc;
    }
  if ((e = cudaMemcpyAsync(dsegs, segs.data(), (size_t)nseg * sizeof(AssetDev),
                           cudaMemcpyHostToDevice, st)) != cudaSuccess)
    return cfail(e, "segment descriptors");
  for (int j = 0; j < nseg; ++j) {
    const int t_lo = 1 + j * C, t_hi = std::min(T, (j + 1) * C);
    const int nt = t_hi - t_lo + 1;
    const int g = j / B, i = j % B;
    if (i == 0) {  // the group's re-sweeps
      Plan* pl = gplan[g == ngrp - 1 ? 1 : 0];
      pl->n_steps = 0;
      for (int jj = j; jj < std::min(nseg, j + B); ++jj)
        pl->n_steps = std::max(pl->n_steps, segs[jj].t_hi - segs[jj].t_lo + 1);
      // the last solve prepared the row sums and P of these transition
      // matrices; P again (once: the launch's assets are one asset) only if
      // this plan's tile size picks another EV path (operand layout)
      if (c->prep_tc[asset] != pl->adev[0].tc) {
        if ((e = launch_rowsums(pl->d_assets, 1, pl->max_rows, c->last_trans, st)) != cudaSuccess)
          return cfail(e, "row sums");
        c->prep_tc[asset] = pl->adev[0].tc;
      }
      if ((rc = run_plan(c, pl, c->last_price, c->last_trans, c->last_cost, c->last_terminal,
                         nullptr, st, false, (const AssetDev*)dsegs + j))) {
        release();
        return rc;
      }
    }
    float* slot_v = (float*)seg_v + (size_t)i * L * (C + 1);
    const void* slot_pol = (const char*)seg_pol + (size_t)i * L * C * pb;
    // V_{t_hi+1} after the segment's values, so V_{t+1} of stage t sits at t - t_lo + 1
    const float* vend = segs[j].v_start ? segs[j].v_start : terminal;
    if ((e = cudaMemcpyAsync(slot_v + (size_t)nt * L, vend, L * 4, cudaMemcpyDeviceToDevice,
                             st)) != cudaSuccess)
      return cfail(e, "segment copy");
    cudaMemsetAsync(post_fx, 0, L * nt * 8, st);
    cudaMemsetAsync(bar, 0, (size_t)ogrid * 4, st);
    OccParams op{};
    op.N = N; op.K = K; op.M = M; op.A = a.A; op.D_dis = a.D_dis;
    op.t_lo = t_lo; op.t_hi = t_hi;
    op.grid_rows = orows;
    const int grid = ogrid;
    op.delta = a.s_max / (double)(N - 1);
    op.eta_c = a.eta_c;
    op.eta_d = a.eta_d;
    op.sw = (float)a.switch_cost;
    op.price = price;
    op.trans = trans;
    op.cost = cost;
    op.e = c->d_e + c->off_e[asset];
    op.policy = slot_pol;
    op.policy_bytes = pb;
    op.rho = (float*)rho;
    op.post = (float*)seg_post + (size_t)i * L * C;
    op.post_fx = (unsigned long long*)post_fx;
    op.fx_e = c->fx_e[asset];
    op.d_price = (double*)dprice64;
    op.acc = (double*)acc;
    op.d_cost = (double*)dcost64;
    op.part = (long long*)opart;
    op.part_cost = (double*)opart_cost;
    op.part_acc = (double*)opart_acc;
    op.flags = (int*)bar;
    op.status = c->d_status;
    op.timeout_ns = c->timeout_ns;
    if ((e = launch_occupancy(op, grid, 256, st)) != cudaSuccess) return cfail(e, "occupancy");
    if ((e = launch_occ_reduce(op, grid, st)) != cudaSuccess) return cfail(e, "occupancy sums");
    // dJ/dP of the group's stages once its last segment's occupancy is in
    // (one launch over all of them: enough blocks to fill the SMs)
    if (i == B - 1 || j == nseg - 1) {
      const int g_lo = 1 + (j - i) * C;
      DTransParams dp{};
      dp.n_t = t_hi - g_lo + 1;
      dp.MN = MN;
      dp.K = K;
      dp.post = (const float*)seg_post;
      dp.vnext = (const float*)seg_v + L;
      dp.seg_len = C;
      dp.seg_stride = (long long)(L * (C + 1));
      dp.cnext = c->d_off[asset] + g_lo + 1;
      dp.d_trans = (float*)dtr + (size_t)(g_lo - 1) * K * K;
      dp.n_split = kDtSplit;
      dp.part = (double*)dtpart;
      dp.part_mass = (double*)dtmass;
      if ((e = launch_dtrans(dp, st)) != cudaSuccess) return cfail(e, "dtrans");
    }
  }
  const long long nP = (long long)T * K;
  to_float_kernel<<<(unsigned)((nP + 255) / 256), 256, 0, st>>>((const double*)dprice64,
                                                                  (float*)dpr, nP);
  if ((e = cudaGetLastError()) != cudaSuccess) return cfail(e, "convert");
  const cudaMemcpyKind k = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
  if (J) cudaMemcpyAsync(J, dJ, 8, k, st);
  if (d_price) cudaMemcpyAsync(d_price, dpr, nP * 4, k, st);
  if (d_trans) cudaMemcpyAsync(d_trans, dtr, (size_t)T * K * K * 4, k, st);
  if (d_eta) cudaMemcpyAsync(d_eta, acc, 16, k, st);
  if (d_cost) {
    to_float_kernel<<<(unsigned)((a.A + 255) / 256), 256, 0, st>>>((const double*)dcost64,
                                                                    (float*)dco, a.A);
    cudaMemcpyAsync(d_cost, dco, (size_t)a.A * 4, k, st);
  }
  if (d_switch) cudaMemcpyAsync(d_switch, (const double*)acc + 4, 8, k, st);
  // after the last segment the occupancy buffer holds rho_{T+1}
  if (d_terminal) cudaMemcpyAsync(d_terminal, rho, L * 4, k, st);
  if (d_mu0)
    cudaMemcpyAsync(d_mu0, c->last_v1 + c->off_v1[asset] + (size_t)a.s0 * K, (size_t)K * 4, k, st);
  int status = 0;
  cudaMemcpyAsync(&status, c->d_status, 4, cudaMemcpyDeviceToHost, st);
  e = cudaStreamSynchronize(st);
  release();
  if (e != cudaSuccess) return cuda_fail(c, e, "grad");
  if (status) return fail(c, status, "device reported status %d in the adjoint", status);
  return ESDP_OK;
}

extern "C" int esdp_objective(esdp_ctx* c, int32_t asset, const float* mu0, double* J,
                              void* stream) {
  if (!c || !mu0 || !J) return ESDP_EINVAL;
  if (asset < 0 || asset >= (int32_t)c->assets.size())
    return fail(c, ESDP_EINVAL, "asset index %d out of range", asset);
  if (!c->solved) return fail(c, ESDP_ESTATE, "no solve has completed");
  const esdp_asset& a = c->assets[asset];
  cudaStream_t st = (cudaStream_t)stream;
  const float* v1 = c->last_v1 + c->off_v1[asset];
  if (c->flags & ESDP_DEVICE_PTRS) {
    objective_kernel<<<1, 32, 0, st>>>(v1, mu0, a.K, a.s0, J);
    CK(cudaGetLastError(), "objective");
    return ESDP_OK;
  }
  CK(cudaMemcpyAsync(c->d_obj_mu, mu0, (size_t)a.K * 4, cudaMemcpyHostToDevice, st), "H2D");
  objective_kernel<<<1, 32, 0, st>>>(v1, c->d_obj_mu, a.K, a.s0, c->d_obj_J);
  CK(cudaGetLastError(), "objective");
  CK(cudaMemcpyAsync(J, c->d_obj_J, 8, cudaMemcpyDeviceToHost, st), "D2H");
  CK(cudaStreamSynchronize(st), "objective");
  return ESDP_OK;
}

// ---------------------------------------------------------------- autotuner

namespace {

struct ZeroInputs {
  const float *price, *trans, *cost, *terminal;
};

// Time every launch shape for the launch assets `ids` over their last
// `t_short` stages (zero inputs: the cost of the sweep does not depend on the
// values), best of four launches after a warm-up; records the fastest in the
// tuning cache (keyed by the assets' shapes) and returns it.
void tune_launch(esdp_ctx* c, const std::vector<int>& ids, int t_short, const ZeroInputs& z,
                 cudaStream_t st, int* best_R, int* best_block) {
  cudaEvent_t e0, e1;
  if (cudaEventCreate(&e0) != cudaSuccess) return;
  if (cudaEventCreate(&e1) != cudaSuccess) {
    cudaEventDestroy(e0);
    return;
  }
  // copies of one asset (the gradient's segment groups) each get their own
  // levels and reference entries, and P is prepared once for them
  const bool copies = ids.size() > 1 && ids[0] == ids[1];
  void* lvl_scr = nullptr;
  if (copies) {
    const esdp_asset& a = c->assets[ids[0]];
    const size_t per = (size_t)(a.T + 2) * 8 + (size_t)a.T * a.K * 8 + (size_t)(a.T + 2) * 4;
    if (cudaMalloc(&lvl_scr, per * ids.size()) != cudaSuccess) {
      cudaGetLastError();
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return;
    }
  }
  double best_ms = 1e300;
  for (int R : {4, 6, 8, 9, 10, 12}) {
    for (int block : {128, 256, 384, 512}) {
      Plan p;
      std::string keep = c->err;
      if (build_plan(c, ids, R, block, c->n_sm, &p)) {
        c->err = keep;
        continue;
      }
      char* q = (char*)lvl_scr;
      for (AssetDev& d : p.adev) {
        d.t_lo = std::max(1, d.t_hi - t_short + 1);
        d.ev_keep = 0;
        d.policy = nullptr;
        d.policy_bytes = 0;
        d.ckpt = nullptr;
        d.v_keep = nullptr;
        if (copies) {
          d.off = (double*)q;
          q += (size_t)(d.T + 2) * 8;
          d.evoff = (double*)q;
          q += (size_t)d.T * d.K * 8;
          d.ref_hist = (float*)q;
          q += (size_t)(d.T + 2) * 4;
        }
      }
      // double-buffered EV scratch per launch asset
      std::vector<float*> evs;
      bool ok = true;
      for (size_t j = 0; j < p.adev.size(); ++j) {
        float* ev = nullptr;
        if (cudaMalloc(&ev, 2 * mnk_of(c->assets[ids[j]]) * 4) != cudaSuccess) {
          cudaGetLastError();
          ok = false;
          break;
        }
        evs.push_back(ev);
        p.adev[j].ev = ev;
      }
      p.n_steps = 0;
      for (const AssetDev& d : p.adev) p.n_steps = std::max(p.n_steps, d.t_hi - d.t_lo + 1);
      double ms = 1e300;
      if (ok && copies) {
        ok = upload_plan(c, &p, st) == ESDP_OK &&
             launch_rowsums(p.d_assets, 1, p.max_rows, z.trans, st) == cudaSuccess;
        c->prep_tc[ids[0]] = p.adev[0].tc;
      }
      if (ok) {
        for (int rep = 0; rep < 5 && ok; ++rep) {
          cudaEventRecord(e0, st);
          if (run_plan(c, &p, z.price, z.trans, z.cost, z.terminal, nullptr, st, !copies)) {
            ok = false;
            break;
          }
          cudaEventRecord(e1, st);
          cudaEventSynchronize(e1);
          float f = 0.f;
          cudaEventElapsedTime(&f, e0, e1);
          if (rep > 0) ms = std::min(ms, (double)f);
        }
      }
      cudaStreamSynchronize(st);
      for (float* ev : evs) cudaFree(ev);
      free_plan(&p);
      if (ok && ms < best_ms) {
        best_ms = ms;
        *best_R = R;
        *best_block = block;
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(lvl_scr);
  if (best_ms < 1e300) {
    std::lock_guard<std::mutex> lk(g_tune_mu);
    g_tune_cache[TuneKey{signature(c, ids)}] = {*best_R, *best_block};
  }
}

}  // namespace

extern "C" int esdp_autotune(esdp_ctx* c, void* stream) {
  if (!c) return ESDP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // the timed candidates overwrite the context's row sums, prepared P and
  // level offsets, and a new shape can change the P layout: the results of an
  // earlier solve are no longer usable
  c->solved = false;
  std::vector<int> ids(c->assets.size());
  std::iota(ids.begin(), ids.end(), 0);
  // ESDP_SHAPE="R,block" pins the launch shape instead of timing candidates
  // (reproducible launches, e.g. for profiler captures)
  if (const char* f = getenv("ESDP_SHAPE")) {
    int R = 0, block = 0;
    if (sscanf(f, "%d,%d", &R, &block) != 2)
      return fail(c, ESDP_EINVAL, "ESDP_SHAPE must be \"R,block\"");
    Plan p;
    int rc = build_plan(c, ids, R, block, c->n_sm, &p);
    if (rc) return rc;
    free_plan(&p);
    g_tune_cache[TuneKey{signature(c, ids)}] = {R, block};
    free_plan(&c->main);
    if ((rc = build_plan(c, ids, R, block, c->n_sm, &c->main))) return rc;
    bind_main(c, &c->main);
    for (auto& m : c->seg_plans) {
      for (auto& kv : m) free_plan(&kv.second);
      m.clear();
    }
    return ESDP_OK;
  }
  // time every candidate on zero inputs over a short horizon (the cost of
  // the sweep does not depend on the values): best of four launches after a
  // warm-up, so that run-to-run noise rarely decides between close shapes
  float *zp = nullptr, *zt = nullptr, *zc = nullptr, *zm = nullptr;
  int rc;
  if ((rc = dalloc(c, &zp, c->n_price)) || (rc = dalloc(c, &zt, c->n_trans)) ||
      (rc = dalloc(c, &zc, c->n_cost)) || (rc = dalloc(c, &zm, c->n_terminal)))
    return rc;
  CK(cudaMemsetAsync(zp, 0, c->n_price * 4, st), "tune");
  CK(cudaMemsetAsync(zt, 0, c->n_trans * 4, st), "tune");
  CK(cudaMemsetAsync(zc, 0, c->n_cost * 4, st), "tune");
  CK(cudaMemsetAsync(zm, 0, c->n_terminal * 4, st), "tune");
  const ZeroInputs z{zp, zt, zc, zm};
  int best_R = c->main.shape.R, best_block = c->main.shape.block;
  tune_launch(c, ids, 16, z, st, &best_R, &best_block);
  // the gradient's segment re-sweeps: B (and b_last) copies of an asset
  // over C stages each
  for (size_t id = 0; id < c->assets.size(); ++id) {
    const esdp_asset& a = c->assets[id];
    if (a.ckpt_every <= 0 || a.T <= a.ckpt_every) continue;
    int B, b_last, nseg;
    grad_groups(a, &B, &b_last, &nseg);
    for (int b : {B, b_last}) {
      const std::vector<int> seg_ids(b, (int)id);
      bool have;
      {
        std::lock_guard<std::mutex> lk(g_tune_mu);
        have = g_tune_cache.count(TuneKey{signature(c, seg_ids)}) > 0;
      }
      int R = best_R, block = best_block;
      if (!have) tune_launch(c, seg_ids, std::min(16, (int)a.ckpt_every), z, st, &R, &block);
    }
  }
  free_plan(&c->main);
  if ((rc = build_plan(c, ids, best_R, best_block, c->n_sm, &c->main))) return rc;
  bind_main(c, &c->main);
  for (auto& m : c->seg_plans) {
    for (auto& kv : m) free_plan(&kv.second);
    m.clear();
  }
  int status = 0;
  CK(cudaMemcpy(&status, c->d_status, 4, cudaMemcpyDeviceToHost), "status");
  if (status) return fail(c, status, "device reported status %d while tuning", status);
  return ESDP_OK;
}
