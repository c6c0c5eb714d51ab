// Persistent backward-induction sweep (Sec. III-B, Algorithm 1; eq. 5-6 with
// a Markov price chain).
//
// One cooperative launch runs every stage of every asset.  A work item is a
// tile of W consecutive SoC rows of one asset with all K price states and
// all modes.  Per stage t the item
//   1. waits (bounded spin) until the tiles whose rows it reads, and the
//      tiles that read its rows, have published EV_t;
//   2. stages EV_t rows [s0 - D_dis, s1 + D_chg) of every mode in shared
//      memory (out-of-grid rows = -inf: the infeasibility mask of Alg. 1);
//   3. builds the payoff table r[m][k][a] = price[t][k] e_a - cost[a]
//      (- switch cost) for its modes;
//   4. runs the banded max-plus over the action band with a register window
//      of R rows per thread and a chunked argmax (exact smallest index);
//   5. writes V_t (shared) and the policy, then contracts
//      EV_{t-1}[m][s][k] = sum_k2 P_{t-1}[k][k2] V_t[m][s][k2] for its own
//      rows (a pointwise-in-s product, so no halo is recomputed) and
//      publishes it with a release flag.
// V therefore never leaves the SM: only EV_{t-1} goes to L2, where the
// neighbouring tiles pick up their halos for stage t-1.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>

#include "../../include/esdp.h"
#include "esdp_internal.h"

namespace esdp {
namespace {

__device__ __forceinline__ unsigned long long now_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct Seg {
  int a0, len, src;
  float sw;
};

// Action segments of output mode m, in increasing action order.  Within a
// segment every action reads EV of the same source mode.
__device__ __forceinline__ void segments(const AssetDev& as, int m, Seg& g0, Seg& g1) {
  if (as.M == 1) {
    g0 = {0, as.A, 0, 0.f};
    g1 = {as.A, 0, 0, 0.f};
  } else if (m == 0) {  // discharge + idle stay in mode 0; charge -> mode 1
    g0 = {0, as.D_dis + 1, 0, 0.f};
    g1 = {as.D_dis + 1, as.D_chg, 1, 0.f};
  } else {              // discharge from mode 1 pays the switch; idle + charge -> mode 1
    g0 = {0, as.D_dis, 0, as.sw};
    g1 = {as.D_dis, as.D_chg + 1, 1, 0.f};
  }
}

__device__ __forceinline__ int round_up(int x, int r) { return (x + r - 1) / r * r; }

__device__ __forceinline__ size_t mnk(const AssetDev& as) {
  return (size_t)as.M * as.N * as.K;
}

__device__ __forceinline__ float* ev_ptr(const AssetDev& as, int t) {
  return as.ev_keep ? as.ev + (size_t)(t - 1) * mnk(as) : as.ev + (size_t)(t & 1) * mnk(as);
}

// Load P_t transposed: Ps[k2*K + k] = trans[t][k][k2].
__device__ __forceinline__ void load_trans(const SweepParams& p, const AssetDev& as, int t,
                                           float* Ps) {
  const int K = as.K;
  const float* P = p.trans + as.off_trans + (size_t)(t - 1) * K * K;
  for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
    const int k = i / K, k2 = i - k * K;
    Ps[k2 * K + k] = __ldg(P + i);
  }
}

// EV rows of the item from the V tile in shared memory (eq. 6).  `te` is
// the stage of the EV being produced; the reference entry is also kept in
// its own per-stage slot.
__device__ __forceinline__ void expectation(const AssetDev& as, const WorkItem& w, int te,
                                            const float* Ps, const float* Vs, float* dst) {
  const int K = as.K, M = as.M, W = as.W, N = as.N;
  const int Wt = w.s1 - w.s0;
  const int total = M * Wt * K;
  for (int i = threadIdx.x; i < total; i += blockDim.x) {
    const int k = i % K;
    const int r = (i / K) % Wt;
    const int m = i / (K * Wt);
    const float* v = Vs + (size_t)(m * W + r) * K;
    float acc = 0.f;
    for (int k2 = 0; k2 < K; ++k2) acc = fmaf(Ps[k2 * K + k], v[k2], acc);
    __stcg(dst + ((size_t)m * N + w.s0 + r) * K + k, acc);
    if (m == 0 && k == 0 && w.s0 + r == as.ref_row) __stcg(as.ref_hist + te, acc);
  }
}

__device__ __forceinline__ void publish(int* flag, int v) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(flag, v);
  }
}

// Wait until every neighbour tile has published at least `need` EV arrays.
// Returns false (uniformly over the CTA) if the launch is being abandoned.
__device__ bool wait_neighbours(const SweepParams& p, const AssetDev& as, const WorkItem& w,
                                int need, int* s_abort) {
  const int lo = max(0, w.tile + as.wait_lo);
  const int hi = min(as.n_tiles - 1, w.tile + as.wait_hi);
  const int n = hi - lo + 1;
  // one more thread waits for the tile that holds the reference row
  if ((int)threadIdx.x <= n) {
    const int tile = (int)threadIdx.x < n ? lo + (int)threadIdx.x : as.ref_tile;
    const int* f = p.flags + as.flag_base + tile;
    if (ld_acquire(f) < need) {
      const unsigned long long t0 = now_ns();
      while (true) {
        if (ld_acquire(f) >= need) break;
        if (*(volatile int*)p.status != 0) {
          *(volatile int*)s_abort = 1;
          break;
        }
        if (now_ns() - t0 > p.timeout_ns) {
          atomicCAS(p.status, 0, ESDP_ETIMEOUT);
          *(volatile int*)s_abort = 1;
          break;
        }
      }
    }
  }
  __threadfence();
  __syncthreads();
  return *(volatile int*)s_abort == 0;
}

template <int R>
__device__ void stage(const SweepParams& p, const AssetDev& as, const WorkItem& w, int it, int t,
                      float* Es, float* Rt, float* Vs, float* Ps, float* Xs, double* s_lvl,
                      float* s_delta) {
  const int K = as.K, M = as.M, N = as.N, rows = as.rows, rs = as.rs, W = as.W;
  const int tid = threadIdx.x, nth = blockDim.x;
  const float NEG = -CUDART_INF_F;

  // 0. level of this stage: c_t = c_{t+1} + EV'_t[ref], the same double on
  //    every tile of the asset; the payoff of price state k absorbs
  //    c_{t+1} rho_t[k] - c_t so that the float values stay centred
  if (tid == 0) {
    const double c_next = p.item_c[it];
    const double c_t = c_next + (double)__ldcg(as.ref_hist + t);
    s_lvl[0] = c_next;
    s_lvl[1] = c_t;
    p.item_c[it] = c_t;
    if (w.tile == 0) as.off[t] = c_t;
  }
  __syncthreads();
  for (int k = tid; k < K; k += nth) {
    const double cr = s_lvl[0] * as.rho[(size_t)(t - 1) * K + k];
    s_delta[k] = (float)(cr - s_lvl[1]);
    if (w.tile == 0) as.evoff[(size_t)(t - 1) * K + k] = cr;
  }

  // 1. EV_t tile with halo; rows outside the grid are infeasible (-inf)
  {
    const float* ev_t = ev_ptr(as, t);
    const long long g0 = (long long)(w.s0 - as.D_dis) * K;
    const long long lim = (long long)N * K;
    const int total = rows * K;
    for (int m = 0; m < M; ++m) {
      const float* src = ev_t + (size_t)m * N * K;
      float* dst = Es + (size_t)m * rows * K;
      for (int i = tid; i < total; i += nth) {
        const long long gi = g0 + i;
        dst[i] = (gi >= 0 && gi < lim) ? __ldcg(src + gi) : NEG;
      }
    }
  }
  __syncthreads();
  // 2. payoff table, padded per segment to a multiple of R with -inf
  {
    const float* price_t = p.price + as.off_price + (size_t)(t - 1) * K;
    const float* cost = p.cost + as.off_cost;
    const int total = M * K * rs;
    for (int i = tid; i < total; i += nth) {
      const int j = i % rs;
      const int mk = i / rs;
      const int k = mk % K, m = mk / K;
      Seg g0, g1;
      segments(as, m, g0, g1);
      const int L0p = round_up(g0.len, R);
      float v = NEG;
      int a = -1;
      float sw = 0.f;
      if (j < L0p) {
        if (j < g0.len) { a = g0.a0 + j; sw = g0.sw; }
      } else if (j - L0p < g1.len) {
        a = g1.a0 + (j - L0p);
        sw = g1.sw;
      }
      if (a >= 0)
        v = (fmaf(__ldg(price_t + k), __ldg(as.e + a), -__ldg(cost + a)) - sw) + s_delta[k];
      Rt[i] = v;
    }
  }
  if (t > as.t_lo) load_trans(p, as, t - 1, Ps);
  __syncthreads();

  // 3. banded max-plus with a register window of R rows
  const int MWK = M * W * K;
  int* Xi = reinterpret_cast<int*>(Xs + (size_t)as.parts * MWK);
  const int nact = K * as.nb * M * as.parts;
  if (tid < nact) {
    const int k = tid % K;
    int q = tid / K;
    const int b = q % as.nb;
    q /= as.nb;
    const int m = q % M;
    const int part = q / M;
    Seg g0, g1;
    segments(as, m, g0, g1);
    const int n0 = round_up(g0.len, R) / R;
    const int nc = n0 + round_up(g1.len, R) / R;
    const int c_lo = part * nc / as.parts, c_hi = (part + 1) * nc / as.parts;
    const float* rt = Rt + (size_t)(m * K + k) * rs;
    float best[R];
    int bc[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      best[j] = NEG;
      bc[j] = -1;
    }
    for (int c = c_lo; c < c_hi; ++c) {
      const bool second = c >= n0;
      const int u0 = (second ? c - n0 : c) * R;
      const int a0 = second ? g1.a0 : g0.a0;
      const int src = second ? g1.src : g0.src;
      const int toff = second ? n0 * R : 0;
      const float* eb = Es + ((size_t)src * rows + b * R + a0 + u0) * K + k;
      float wv[2 * R - 1];
#pragma unroll
      for (int x = 0; x < 2 * R - 1; ++x) wv[x] = eb[(size_t)x * K];
      float rr[R];
#pragma unroll
      for (int i = 0; i < R; ++i) rr[i] = rt[toff + u0 + i];
      float cm[R];
#pragma unroll
      for (int j = 0; j < R; ++j) cm[j] = rr[0] + wv[j];
#pragma unroll
      for (int i = 1; i < R; ++i) {
#pragma unroll
        for (int j = 0; j < R; ++j) cm[j] = fmaxf(cm[j], rr[i] + wv[i + j]);
      }
#pragma unroll
      for (int j = 0; j < R; ++j) {
        if (cm[j] > best[j]) {
          best[j] = cm[j];
          bc[j] = c;
        }
      }
    }
    // exact argmax: first action of the winning chunk that reproduces the max
    const int xo = part * MWK + (m * W + b * R) * K + k;
#pragma unroll
    for (int j = 0; j < R; ++j) {
      int arg = -1;
      if (bc[j] >= 0) {
        const int c = bc[j];
        const bool second = c >= n0;
        const int u0 = (second ? c - n0 : c) * R;
        const int a0 = second ? g1.a0 : g0.a0;
        const int src = second ? g1.src : g0.src;
        const int toff = second ? n0 * R : 0;
        const float* eb = Es + ((size_t)src * rows + b * R + j + a0 + u0) * K + k;
        for (int i = 0; i < R; ++i) {
          const float v = rt[toff + u0 + i] + eb[(size_t)i * K];
          if (v == best[j]) {
            arg = a0 + u0 + i;
            break;
          }
        }
      }
      Xs[xo + j * K] = best[j];
      Xi[xo + j * K] = arg;
    }
  }
  __syncthreads();

  // 4. combine the action parts (in increasing action order), store V_t and
  //    the policy
  {
    const size_t MNK = mnk(as);
    const int total = M * W * K;
    for (int i = tid; i < total; i += nth) {
      const int k = i % K;
      const int r = (i / K) % W;
      const int m = i / (K * W);
      const int s = w.s0 + r;
      if (s >= w.s1) continue;
      float bv = Xs[i];
      int ba = Xi[i];
      for (int q = 1; q < as.parts; ++q) {
        const float v = Xs[q * MWK + i];
        if (v > bv) {
          bv = v;
          ba = Xi[q * MWK + i];
        }
      }
      Vs[i] = bv;
      const size_t o = ((size_t)m * N + s) * K + k;
      if (as.policy) {
        const size_t po = (size_t)(t - as.policy_t_base) * MNK + o;
        if (as.policy_bytes == 2)
          __stcs(reinterpret_cast<short*>(as.policy) + po, (short)ba);
        else
          __stcs(reinterpret_cast<int*>(as.policy) + po, ba);
      }
      if (as.v_keep) __stcg(as.v_keep + (size_t)(t - as.t_lo) * MNK + o, bv);
      if (as.ckpt && as.ckpt_every > 0 && t > 1 && (t - 1) % as.ckpt_every == 0)
        __stcg(as.ckpt + (size_t)((t - 1) / as.ckpt_every - 1) * MNK + o, bv);
      if (t == 1 && p.v1) p.v1[as.off_v1 + o] = (float)((double)bv + s_lvl[1]);
    }
  }
  __syncthreads();

  // 5. EV_{t-1} for the item's own rows
  if (t > as.t_lo) expectation(as, w, t - 1, Ps, Vs, ev_ptr(as, t - 1));
}

template <int R>
__global__ void __launch_bounds__(kMaxBlock, 1) sweep_kernel(const SweepParams p) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  float* Es = smem + p.sm_E;
  float* Rt = smem + p.sm_R;
  float* Vs = smem + p.sm_V;
  float* Ps = smem + p.sm_P;
  float* Xs = smem + p.sm_X;
  __shared__ int s_abort;
  __shared__ double s_lvl[2];
  __shared__ float s_delta[128];
  const int i0 = p.cta_items[blockIdx.x], i1 = p.cta_items[blockIdx.x + 1];
  if (threadIdx.x == 0) s_abort = 0;
  __syncthreads();

  // prologue: EV_{t_hi} = P_{t_hi} V_{t_hi+1} for the item's rows
  for (int it = i0; it < i1; ++it) {
    const WorkItem w = p.items[it];
    const AssetDev& as = p.assets[w.asset];
    const float* vst = as.v_start ? as.v_start : p.terminal + as.off_terminal;
    load_trans(p, as, as.t_hi, Ps);
    const int Wt = w.s1 - w.s0, K = as.K;
    for (int i = threadIdx.x; i < as.M * Wt * K; i += blockDim.x) {
      const int k = i % K, r = (i / K) % Wt, m = i / (K * Wt);
      Vs[(m * as.W + r) * K + k] = __ldcg(vst + ((size_t)m * as.N + w.s0 + r) * K + k);
    }
    if (threadIdx.x == 0) {
      const double c0 = as.c_start ? *as.c_start : 0.0;
      p.item_c[it] = c0;
      if (w.tile == 0) as.off[as.t_hi + 1] = c0;
    }
    __syncthreads();
    expectation(as, w, as.t_hi, Ps, Vs, ev_ptr(as, as.t_hi));
    publish(p.flags + as.flag_base + w.tile, 1);
    __syncthreads();
  }

  for (int g = 0; g < p.n_steps; ++g) {
    for (int it = i0; it < i1; ++it) {
      const WorkItem w = p.items[it];
      const AssetDev& as = p.assets[w.asset];
      if (g > as.t_hi - as.t_lo) continue;
      if (!wait_neighbours(p, as, w, g + 1 + p.wait_extra, &s_abort)) return;
      stage<R>(p, as, w, it, as.t_hi - g, Es, Rt, Vs, Ps, Xs, s_lvl, s_delta);
      publish(p.flags + as.flag_base + w.tile, g + 2);
    }
  }
}

template <int R>
cudaError_t launch_R(const SweepShape& s, const SweepParams& p, cudaStream_t stream) {
  auto fn = sweep_kernel<R>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  SweepParams pp = p;
  void* args[] = {&pp};
  return cudaLaunchCooperativeKernel((const void*)fn, dim3(s.grid), dim3(s.block), args, s.smem,
                                     stream);
}

template <int R>
int max_blocks_R(int block, size_t smem) {
  auto fn = sweep_kernel<R>;
  if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess)
    return 0;
  int n = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, fn, block, smem) != cudaSuccess) return 0;
  return n;
}

// rho_t[k] = sum_k2 trans[t][k][k2] in double, for every asset of a launch
__global__ void rowsum_kernel(const AssetDev* assets, const float* trans) {
  const AssetDev& as = assets[blockIdx.y];
  const int K = as.K;
  const long long rows = (long long)as.T * K;
  const float* P = trans + as.off_trans;
  double* rho = as.rho;
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < rows;
       r += (long long)gridDim.x * blockDim.x) {
    double acc = 0.0;
    for (int k2 = 0; k2 < K; ++k2) acc += (double)__ldg(P + r * K + k2);
    rho[r] = acc;
  }
}

__global__ void ev_readout_kernel(const float* evp, const double* evoff, int M, int N, int K,
                                  float* out) {
  const long long n = (long long)M * N * K;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    out[i] = (float)((double)evp[i] + evoff[i % K]);
}

}  // namespace

cudaError_t launch_rowsums(const AssetDev* d_assets, int n_assets, int max_rows,
                           const float* trans, cudaStream_t stream) {
  if (n_assets == 0) return cudaSuccess;
  const int block = 128;
  const int gx = std::max(1, std::min(64, (max_rows + block - 1) / block));
  rowsum_kernel<<<dim3(gx, n_assets), block, 0, stream>>>(d_assets, trans);
  return cudaGetLastError();
}

cudaError_t launch_ev_readout(const float* evp, const double* evoff, int M, int N, int K,
                              float* out, cudaStream_t stream) {
  const long long n = (long long)M * N * K;
  const int block = 256;
  const int grid = (int)std::min<long long>(1184, (n + block - 1) / block);
  ev_readout_kernel<<<std::max(grid, 1), block, 0, stream>>>(evp, evoff, M, N, K, out);
  return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepShape& s, const SweepParams& p, cudaStream_t stream) {
  switch (s.R) {
    case 4: return launch_R<4>(s, p, stream);
    case 8: return launch_R<8>(s, p, stream);
    case 12: return launch_R<12>(s, p, stream);
    case 16: return launch_R<16>(s, p, stream);
    default: return cudaErrorInvalidValue;
  }
}

int sweep_max_blocks_per_sm(int R, int block, size_t smem) {
  switch (R) {
    case 4: return max_blocks_R<4>(block, smem);
    case 8: return max_blocks_R<8>(block, smem);
    case 12: return max_blocks_R<12>(block, smem);
    case 16: return max_blocks_R<16>(block, smem);
    default: return 0;
  }
}

}  // namespace esdp
