// esdp_solve_noalloc: the backward-induction sweep for one asset with no
// memory allocation at all.
//
// Some callers cannot call cudaMalloc: code running inside a host that owns
// the device memory pool (a plugin in an application with its own caching
// allocator, a process under a hard device-memory quota), or code that must
// not allocate on a latency-critical path.  This entry point takes the
// caller's inputs and outputs and keeps every piece of workspace the sweep
// needs (EV halo buffers, neighbour flags, status word, stage levels, launch
// plan) in one file-scope device array of fixed size, reserved when the
// library is loaded on a GPU and held until the process exits.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "../../include/esdp.h"
#include "esdp_internal.h"

namespace esdp {
namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;  // ESDP_NOALLOC_SCRATCH_BYTES
constexpr int kNoAllocMaxItems = 2048;
constexpr size_t kSmemLimit = 227 * 1024;

// The workspace.  Every call on a device reuses it; its contents persist
// between calls, so everything that must start at zero is cleared per call.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

// Grid energy of each action (eq. 2), in double then rounded once.
__global__ void energy_kernel(float* e, int A, int D_dis, double delta, double eta_c,
                              double eta_d) {
  for (int a = blockIdx.x * blockDim.x + threadIdx.x; a < A; a += gridDim.x * blockDim.x) {
    const int d = a - D_dis;
    double en = 0.0;
    if (d < 0) en = -(double)d * delta * eta_d;
    if (d > 0) en = -(double)d * delta / eta_c;
    e[a] = (float)en;
  }
}

int msg(char* buf, int32_t len, int code, const char* text) {
  if (buf && len > 0) {
    std::strncpy(buf, text, (size_t)len - 1);
    buf[len - 1] = '\0';
  }
  return code;
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

int chunks_min(const esdp_asset& a, int R) {
  auto ru = [R](int x) { return (x + R - 1) / R; };
  if (a.n_modes == 1) return ru(a.A);
  return std::min(ru(a.D_dis + 1) + ru(a.D_chg), ru(a.D_dis) + ru(a.D_chg + 1));
}

}  // namespace
}  // namespace esdp

using namespace esdp;

extern "C" int esdp_solve_noalloc(const esdp_asset* asset, const float* price, const float* trans,
                                  const float* cost, const float* terminal, float* V1,
                                  void* policy, void* stream, char* err, int32_t err_len) {
  char buf[256];
  if (!asset || !price || !trans || !cost || !terminal || !V1)
    return msg(err, err_len, ESDP_EINVAL, "null argument");
  const esdp_asset& a = *asset;
  if (a.T < 1 || a.N < 2 || a.K < 1 || a.K > 128 || a.A < 1 || a.D_dis < 0 || a.D_chg < 0 ||
      a.D_dis + a.D_chg + 1 != a.A || a.D_dis > a.N - 1 || a.D_chg > a.N - 1 ||
      (a.n_modes != 1 && a.n_modes != 2) || !(a.eta_c > 0 && a.eta_c <= 1) ||
      !(a.eta_d > 0 && a.eta_d <= 1) || !(a.s_max > 0) || !std::isfinite(a.s_max) ||
      !std::isfinite(a.switch_cost) || (policy && a.policy_bytes != 2 && a.policy_bytes != 4))
    return msg(err, err_len, ESDP_EINVAL, "invalid asset description");
  if (policy && a.policy_bytes == 2 && a.A > 32767)
    return msg(err, err_len, ESDP_EINVAL, "int16 policies need A <= 32767");
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess)
    return msg(err, err_len, ESDP_ECUDA, "no current CUDA device");
  // the device address of the workspace in the current context, looked up
  // on every call: a cached address would go stale after a device reset or
  // under another context of the same device
  void* base = nullptr;
  {
    const cudaError_t e = cudaGetSymbolAddress(&base, g_noalloc_scratch);
    if (e != cudaSuccess || !base) {
      snprintf(buf, sizeof(buf), "cudaGetSymbolAddress of the workspace failed: %s",
               cudaGetErrorString(e));
      return msg(err, err_len, ESDP_ECUDA, buf);
    }
  }
  // bounded device waits: the same limit and test hook as esdp_solve
  unsigned long long timeout_ns = 5ull * 1000 * 1000 * 1000;
  if (const char* env = std::getenv("ESDP_TIMEOUT_MS")) {
    const long long ms = std::atoll(env);
    if (ms > 0) timeout_ns = (unsigned long long)ms * 1000000ull;
  }
  const int wait_extra = std::getenv("ESDP_INJECT_STALL") ? 1000000 : 0;
  int n_sm = 0;
  if (cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return msg(err, err_len, ESDP_ECUDA, "device attribute query failed");

  // launch shape: R = 8 rows per thread, 512 threads, tiles sized to the grid
  const int R = 8, block = 512, M = a.n_modes, K = a.K, KM = ((K + 1) / 2) * M;
  const int nb_max = block / KM;
  if (nb_max < 1) return msg(err, err_len, ESDP_EINVAL, "K * n_modes exceeds 1024");
  int nb = std::max(1, std::min(nb_max, (a.N + n_sm * R - 1) / (n_sm * R)));
  int W = 0, tiles = 0, parts = 1, rows = 0, rs = 0;
  SweepSmem L{};
  for (; nb >= 1; --nb) {
    W = nb * R;
    tiles = (a.N + W - 1) / W;
    rows = W + a.A + R;
    rs = (a.A + 2 * R) | 1;
    const int reach = (std::max(a.D_dis, a.D_chg) + W - 1) / W;
    if (2 * reach + 2 > block) continue;
    parts = pick_parts(KM * nb, block, chunks_min(a, R));
    if (parts < 1) continue;
    L = sweep_smem_layout(M, K, W, a.A, R, false);  // no prepared P: SIMT / mma.sync EV
    if (L.bytes <= kSmemLimit) break;
  }
  if (nb < 1) return msg(err, err_len, ESDP_EINVAL, "no launch shape fits shared memory");
  if (tiles > kNoAllocMaxItems) {
    snprintf(buf, sizeof(buf), "%d tiles exceed the allocation-free limit of %d", tiles,
             kNoAllocMaxItems);
    return msg(err, err_len, ESDP_EINVAL, buf);
  }
  const size_t smem = L.bytes;
  const int kh = (a.K + 1) / 2 == 32 ? 32 : 0;
  const int per_sm = sweep_max_blocks_per_sm(R, kh, block, smem);
  if (per_sm < 1) return msg(err, err_len, ESDP_ECUDA, "sweep kernel does not fit on an SM");
  const int grid = std::min(tiles, per_sm * n_sm);

  // carve the workspace
  const size_t MNK = (size_t)M * a.N * K;
  size_t o = 0;
  auto take = [&](size_t bytes) {
    const size_t at = o;
    o = align256(o + bytes);
    return at;
  };
  const size_t o_asset = take(sizeof(AssetDev));
  const size_t o_items = take(sizeof(WorkItem) * tiles);
  const size_t o_cta = take(sizeof(int) * (grid + 1));
  const size_t o_flags = take(sizeof(int) * tiles);
  const size_t o_status = take(sizeof(int));
  const size_t o_itemc = take(sizeof(double) * tiles);
  const size_t o_e = take(sizeof(float) * a.A);
  const size_t o_rho = take(sizeof(double) * (size_t)a.T * K);
  const size_t o_off = take(sizeof(double) * ((size_t)a.T + 2));
  const size_t o_evoff = take(sizeof(double) * (size_t)a.T * K);
  const size_t o_refh = take(sizeof(float) * ((size_t)a.T + 2));
  const size_t o_ev = take(sizeof(float) * 2 * MNK);
  if (o > kNoAllocBytes) {
    snprintf(buf, sizeof(buf),
             "this asset needs %zu bytes of workspace; the allocation-free entry point "
             "reserves %zu (2*n_modes*N*K floats of EV plus per-stage data must fit)",
             o, kNoAllocBytes);
    return msg(err, err_len, ESDP_EINVAL, buf);
  }
  unsigned char* S = static_cast<unsigned char*>(base);

  // launch plan on the host stack, copied into the workspace
  AssetDev d{};
  d.T = a.T; d.N = a.N; d.K = K; d.A = a.A; d.D_dis = a.D_dis; d.D_chg = a.D_chg; d.M = M;
  d.policy_bytes = policy ? a.policy_bytes : 0;
  d.nb = nb; d.parts = parts; d.W = W; d.n_tiles = tiles; d.flag_base = 0;
  const int reach = (std::max(a.D_dis, a.D_chg) + W - 1) / W;
  d.wait_lo = -reach; d.wait_hi = reach;
  d.t_hi = a.T; d.t_lo = 1; d.ev_keep = 0; d.policy_t_base = 1; d.ckpt_every = 0;
  d.rows = rows; d.rs = rs; d.sw = (float)a.switch_cost;
  // no prepared P here: where the tile size (or ESDP_EV) picks a tensor path,
  // mma.sync takes it
  d.mma = (ev_path(W, M, K, ev_force()) != kEvSimt && (K & 7) == 0) ? 1 : 0;
  d.off_price = d.off_trans = d.off_cost = d.off_terminal = d.off_v1 = 0;
  d.e = reinterpret_cast<const float*>(S + o_e);
  d.v_start = nullptr;
  d.ev = reinterpret_cast<float*>(S + o_ev);
  d.policy = policy;
  d.v_keep = nullptr;
  d.ckpt = nullptr;
  d.ref_row = a.N / 2;
  d.ref_tile = d.ref_row / W;
  d.ref_hist = reinterpret_cast<float*>(S + o_refh);
  d.rho = reinterpret_cast<double*>(S + o_rho);
  d.off = reinterpret_cast<double*>(S + o_off);
  d.evoff = reinterpret_cast<double*>(S + o_evoff);
  d.c_start = nullptr;
  WorkItem items[kNoAllocMaxItems];
  int cta[kNoAllocMaxItems + 1];
  // contiguous runs of tiles per CTA, balanced to within one tile
  int k = 0;
  cta[0] = 0;
  for (int g = 0; g < grid; ++g) {
    const int n = tiles / grid + (g < tiles % grid ? 1 : 0);
    for (int j = 0; j < n; ++j, ++k) {
      items[k].asset = 0;
      items[k].tile = k;
      items[k].s0 = k * W;
      items[k].s1 = std::min(a.N, k * W + W);
    }
    cta[g + 1] = k;
  }
  cudaError_t e = cudaMemcpyAsync(S + o_asset, &d, sizeof(d), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S + o_items, items, sizeof(WorkItem) * tiles, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(S + o_cta, cta, sizeof(int) * (grid + 1), cudaMemcpyHostToDevice, st);
  // cleared on every call: neighbour flags and the status word
  if (e == cudaSuccess) e = cudaMemsetAsync(S + o_flags, 0, sizeof(int) * tiles, st);
  if (e == cudaSuccess) e = cudaMemsetAsync(S + o_status, 0, sizeof(int), st);
  if (e == cudaSuccess) {
    energy_kernel<<<1, 256, 0, st>>>(reinterpret_cast<float*>(S + o_e), a.A, a.D_dis,
                                     a.s_max / (double)(a.N - 1), a.eta_c, a.eta_d);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess)
    e = launch_rowsums(reinterpret_cast<const AssetDev*>(S + o_asset), 1, a.T * K, trans, st);
  SweepParams sp{};
  sp.assets = reinterpret_cast<const AssetDev*>(S + o_asset);
  sp.items = reinterpret_cast<const WorkItem*>(S + o_items);
  sp.cta_items = reinterpret_cast<const int*>(S + o_cta);
  sp.price = price;
  sp.trans = trans;
  sp.cost = cost;
  sp.terminal = terminal;
  sp.v1 = V1;
  sp.n_steps = a.T;
  sp.flags = reinterpret_cast<int*>(S + o_flags);
  sp.status = reinterpret_cast<int*>(S + o_status);
  sp.timeout_ns = timeout_ns;
  sp.wait_extra = wait_extra;
  sp.item_c = reinterpret_cast<double*>(S + o_itemc);
  sp.sm_E = L.E;
  sp.sm_R = L.Rt;
  sp.sm_C = L.C;
  sp.sm_V = L.V;
  sp.sm_P = L.P;
  sp.sm_X = L.X;
  SweepShape shape;
  shape.R = R;
  shape.kh = kh;
  shape.block = block;
  shape.grid = grid;
  shape.smem = smem;
  if (e == cudaSuccess) e = launch_sweep(shape, sp, st);
  int status = 0;
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(&status, S + o_status, sizeof(int), cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) {
    snprintf(buf, sizeof(buf), "CUDA error: %s", cudaGetErrorString(e));
    return msg(err, err_len, ESDP_ECUDA, buf);
  }
  if (status) {
    snprintf(buf, sizeof(buf), "device reported status %d", status);
    return msg(err, err_len, status, buf);
  }
  return msg(err, err_len, ESDP_OK, "");
}
