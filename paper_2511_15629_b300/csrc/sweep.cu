// Persistent backward-induction sweep (Sec. III-B, Algorithm 1; eq. 5-6 with
// a Markov price chain).
//
// One cooperative launch runs every stage of every asset.  A work item is a
// tile of W consecutive SoC rows of one asset with all K price states and
// all modes.  Per stage t the item
//   0. prefetches what does not depend on other tiles (P_{t-1} transposed via
//      cp.async, its prices and transition row sums);
//   1. waits (bounded spin) until the tiles whose rows it reads, the tiles
//      that read its rows and the tile holding the reference row have
//      published EV_t;
//   2. stages EV_t rows [s0 - D_dis, s1 + D_chg + R) of every mode in shared
//      memory with TMA bulk copies (rows outside the grid are -inf: the
//      infeasibility mask of Alg. 1), overlapped with building the payoff
//      table r[m][k][a] = price[t][k] e_a - cost[a] (- switch cost);
//   3. runs the banded max-plus: a thread owns R consecutive rows of one
//      (m, k) and slides a register window of EV values over the action band
//      (two evaluations per 3-input max), tracking the winning chunk of R
//      actions and recovering the exact smallest maximiser afterwards;
//   4. keeps V_t in shared memory, stores the policy, and contracts
//      EV_{t-1}[m][s][k] = sum_k2 P_{t-1}[k][k2] V_t[m][s][k2] for its own rows
//      (pointwise in s: no halo is recomputed), then publishes it.
// V never leaves the SM; EV goes to L2 where neighbours pick up their halos.
//
// Float32 values are kept centred: V'_t = V_t - c_t with a scalar level
// c_t = c_{t+1} + EV'_t[ref] carried in double (the same on every tile), and
// the payoff of price state k absorbs c_{t+1} rowsum(P_t)[k] - c_t.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cstdint>

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

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}

__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

__device__ __forceinline__ void mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
               "r"(bytes)
               : "memory");
}

__device__ __forceinline__ void bulk_load(void* dst, const void* src, uint32_t bytes,
                                          uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return ok != 0;
}

// Bounded wait for the bulk copies of this stage.  On expiry: report
// ESDP_ETIMEOUT, give the copies one more bounded wait, and tell the caller to
// abandon the launch.
__device__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, const SweepParams& p) {
  if (mbar_try_wait(bar, parity)) return true;
  unsigned long long t0 = now_ns();
  while (!mbar_try_wait(bar, parity)) {
    if (now_ns() - t0 > p.timeout_ns) {
      atomicCAS(p.status, 0, ESDP_ETIMEOUT);
      t0 = now_ns();
      while (!mbar_try_wait(bar, parity) && now_ns() - t0 <= p.timeout_ns) {
      }
      return false;
    }
  }
  return true;
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

// Issue the asynchronous load of P_t transposed: Ps[k2*Kp4 + k] = trans[t][k][k2].
__device__ __forceinline__ void prefetch_trans(const SweepParams& p, const AssetDev& as, int t,
                                               float* Ps) {
  const int K = as.K, Kp4 = (K + 3) & ~3;
  const float* P = p.trans + as.off_trans + (size_t)(t - 1) * K * K;
  for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
    const int k2 = i / K, k = i - k2 * K;
    cp_async4(Ps + k2 * Kp4 + k, P + (size_t)k * K + k2);
  }
}

// EV rows of the item (eq. 6) from V' in shared memory (row stride K+1):
// each thread forms 2 rows x 4 price states; the sum over k2 runs in
// ascending order with one fma per term.  `te` is the stage of the EV being
// produced; its reference entry also goes to its own per-stage slot.
__device__ __forceinline__ void expectation(const AssetDev& as, const WorkItem& w, int te,
                                            const float* Ps, const float* Vs, float* dst) {
  const int K = as.K, M = as.M, W = as.W, N = as.N, Kv = K + 1, Kp4 = (K + 3) & ~3;
  const int Wt = w.s1 - w.s0;
  const int G = (K + 3) >> 2;
  const int n_rows = M * Wt;
  const int units = ((n_rows + 1) >> 1) * G;
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int g = u % G, rp = u / G;
    const int L0 = 2 * rp, L1 = min(2 * rp + 1, n_rows - 1);
    const int m0 = L0 / Wt, r0 = L0 - m0 * Wt;
    const int m1 = L1 / Wt, r1 = L1 - m1 * Wt;
    const float* v0 = Vs + (m0 * W + r0) * Kv;
    const float* v1 = Vs + (m1 * W + r1) * Kv;
    const float* pp = Ps + 4 * g;
    float a0[4] = {0.f, 0.f, 0.f, 0.f}, a1[4] = {0.f, 0.f, 0.f, 0.f};
    for (int k2 = 0; k2 < K; ++k2) {
      const float4 q = *reinterpret_cast<const float4*>(pp + k2 * Kp4);
      const float x0 = v0[k2], x1 = v1[k2];
      a0[0] = fmaf(q.x, x0, a0[0]);
      a0[1] = fmaf(q.y, x0, a0[1]);
      a0[2] = fmaf(q.z, x0, a0[2]);
      a0[3] = fmaf(q.w, x0, a0[3]);
      a1[0] = fmaf(q.x, x1, a1[0]);
      a1[1] = fmaf(q.y, x1, a1[1]);
      a1[2] = fmaf(q.z, x1, a1[2]);
      a1[3] = fmaf(q.w, x1, a1[3]);
    }
    float* d0 = dst + ((size_t)m0 * N + w.s0 + r0) * K + 4 * g;
#pragma unroll
    for (int j = 0; j < 4; ++j)
      if (4 * g + j < K) __stcg(d0 + j, a0[j]);
    if (m0 == 0 && g == 0 && w.s0 + r0 == as.ref_row) __stcg(as.ref_hist + te, a0[0]);
    if (2 * rp + 1 < n_rows) {
      float* d1 = dst + ((size_t)m1 * N + w.s0 + r1) * K + 4 * g;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (4 * g + j < K) __stcg(d1 + j, a1[j]);
      if (m1 == 0 && g == 0 && w.s0 + r1 == as.ref_row) __stcg(as.ref_hist + te, a1[0]);
    }
  }
}

__device__ __forceinline__ void publish(int* flag, int v) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    st_release(flag, v);
  }
}

// Wait until every neighbour tile and the reference tile have published at
// least `need` EV arrays; the thread that waits for the reference tile also
// reads EV'_t[ref].  Returns false (uniformly over the CTA) if the launch is
// being abandoned.
__device__ bool wait_neighbours(const SweepParams& p, const AssetDev& as, const WorkItem& w,
                                int need, int t, int* s_abort, float* s_ref) {
  const int lo = max(0, w.tile + as.wait_lo);
  const int hi = min(as.n_tiles - 1, w.tile + as.wait_hi);
  const int n = hi - lo + 1;
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
    if ((int)threadIdx.x == n) *s_ref = __ldcg(as.ref_hist + t);
  }
  __syncthreads();
  return *(volatile int*)s_abort == 0;
}

struct Smem {
  float *Es, *Rt, *Ecol, *Ccol, *Vs, *Ps, *Xs;
  double* lvl;     // [2]: c_{t+1}, c_t
  float* lam;      // [K] prices of the stage
  float* delta;    // [K] level correction of the stage
  float* ref;      // EV'_t[ref]
  int* abort;
  uint64_t* bar;
};

// One stage of one work item.  Returns false if the launch is abandoned.
template <int R>
__device__ bool item_stage(const SweepParams& p, const AssetDev& as, const WorkItem& w, int it,
                           int g, const Smem& sm, uint32_t& parity) {
  const int t = as.t_hi - g;
  const int K = as.K, M = as.M, N = as.N, rows = as.rows, rs = as.rs, W = as.W;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5,
            nwarps = nth >> 5;
  const float NEG = -CUDART_INF_F;
  const bool tma = (K & 3) == 0;

  // 0. prefetch the inputs of the stage
  if (t > as.t_lo) prefetch_trans(p, as, t - 1, sm.Ps);
  float lam_k = 0.f;
  double rho_k = 0.0, c_next = 0.0;
  if (tid < K) {
    lam_k = __ldg(p.price + as.off_price + (size_t)(t - 1) * K + tid);
    rho_k = __ldg(as.rho + (size_t)(t - 1) * K + tid);
  }
  if (tid == 0) c_next = p.item_c[it];

  // 1. neighbours
  if (!wait_neighbours(p, as, w, g + 1 + p.wait_extra, t, sm.abort, sm.ref)) return false;

  // 2. EV_t tile: bulk copies of the rows inside the grid, -inf outside
  const float* ev_t = ev_ptr(as, t);
  const int g0row = w.s0 - as.D_dis;
  const int lo = max(g0row, 0), hi = min(g0row + rows, N);
  if (tma) {
    if (tid == 0) {
      asm volatile("fence.proxy.async;" ::: "memory");
      const uint32_t bytes = (uint32_t)(hi - lo) * K * 4u;
      mbar_expect_tx(sm.bar, bytes * M);
      for (int m = 0; m < M; ++m)
        bulk_load(sm.Es + ((size_t)m * rows + (lo - g0row)) * K, ev_t + ((size_t)m * N + lo) * K,
                  bytes, sm.bar);
    }
  } else {
    for (int m = 0; m < M; ++m) {
      const float* src = ev_t + ((size_t)m * N + lo) * K;
      float* dst = sm.Es + ((size_t)m * rows + (lo - g0row)) * K;
      const int n = (hi - lo) * K;
      for (int i = tid; i < n; i += nth) dst[i] = __ldcg(src + i);
    }
  }
  {
    const int below = (lo - g0row) * K, above0 = (hi - g0row) * K, total = rows * K;
    for (int m = 0; m < M; ++m) {
      float* e = sm.Es + (size_t)m * rows * K;
      for (int i = tid; i < below; i += nth) e[i] = NEG;
      for (int i = above0 + tid; i < total; i += nth) e[i] = NEG;
    }
  }
  // level of the stage and the per-state correction of the payoffs
  if (tid == 0) {
    const double c_t = c_next + (double)*sm.ref;
    sm.lvl[0] = c_next;
    sm.lvl[1] = c_t;
    p.item_c[it] = c_t;
    if (w.tile == 0) as.off[t] = c_t;
  }
  // payoff columns of each mode: e_a and -(cost_a + switch), -inf padding
  {
    const float* cost = p.cost + as.off_cost;
    for (int i = tid; i < M * rs; i += nth) {
      const int m = i / rs, j = i - m * rs;
      Seg g0, g1;
      segments(as, m, g0, g1);
      const int L0p = round_up(g0.len, R);
      int a = -1;
      float sw = 0.f;
      if (j < L0p) {
        if (j < g0.len) {
          a = g0.a0 + j;
          sw = g0.sw;
        }
      } else if (j - L0p < g1.len) {
        a = g1.a0 + (j - L0p);
        sw = g1.sw;
      }
      sm.Ecol[i] = a >= 0 ? __ldg(as.e + a) : 0.f;
      sm.Ccol[i] = a >= 0 ? -__ldg(cost + a) - sw : NEG;
    }
  }
  __syncthreads();
  if (tid < K) {
    const double cr = sm.lvl[0] * rho_k;
    sm.delta[tid] = (float)(cr - sm.lvl[1]);
    sm.lam[tid] = lam_k;
    if (w.tile == 0) as.evoff[(size_t)(t - 1) * K + tid] = cr;
  }
  __syncthreads();
  for (int row = warp; row < M * K; row += nwarps) {
    const int m = row / K, k = row - m * K;
    const float lam = sm.lam[k], dl = sm.delta[k];
    const float* ec = sm.Ecol + m * rs;
    const float* cc = sm.Ccol + m * rs;
    float* dst = sm.Rt + (size_t)row * rs;
    for (int j = lane; j < rs; j += 32) dst[j] = fmaf(lam, ec[j], cc[j]) + dl;
  }
  cp_async_wait_all();
  if (tma) {
    if (tid == 0 && !mbar_wait_bounded(sm.bar, parity, p)) *(volatile int*)sm.abort = 1;
    parity ^= 1u;
  }
  __syncthreads();
  if (*(volatile int*)sm.abort) return false;

  // 3. banded max-plus with a register window of R rows
  const int MWK = M * W * K;
  int* Xi = reinterpret_cast<int*>(sm.Xs + (size_t)as.parts * MWK);
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
    const float* rt = sm.Rt + (size_t)(m * K + k) * rs;
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
      const float* eb = sm.Es + ((size_t)src * rows + b * R + a0 + u0) * K + k;
      float wv[2 * R - 1];
#pragma unroll
      for (int x = 0; x < 2 * R - 1; ++x) wv[x] = eb[(size_t)x * K];
      float rr[R];
#pragma unroll
      for (int i = 0; i < R; ++i) rr[i] = rt[toff + u0 + i];
      float cm[R];
#pragma unroll
      for (int j = 0; j < R; ++j) cm[j] = fmaxf(rr[0] + wv[j], rr[1] + wv[j + 1]);
#pragma unroll
      for (int i = 2; i < R; i += 2) {
#pragma unroll
        for (int j = 0; j < R; ++j)
          cm[j] = max3f(cm[j], rr[i] + wv[i + j], rr[i + 1] + wv[i + 1 + j]);
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
        const float* eb = sm.Es + ((size_t)src * rows + b * R + j + a0 + u0) * K + k;
        const float* rp = rt + toff + u0;
        float v[R];
#pragma unroll
        for (int i = 0; i < R; ++i) v[i] = rp[i] + eb[(size_t)i * K];
        int first = R - 1;
#pragma unroll
        for (int i = R - 1; i >= 0; --i)
          if (v[i] == best[j]) first = i;
        arg = a0 + u0 + first;
      }
      sm.Xs[xo + j * K] = best[j];
      Xi[xo + j * K] = arg;
    }
  }
  __syncthreads();

  // 4. combine the action parts (in increasing action order); V'_t, policy
  {
    const size_t MNK = mnk(as);
    const int Wt = w.s1 - w.s0, Kv = K + 1;
    const double lvl = sm.lvl[1];
    for (int row = warp; row < M * Wt; row += nwarps) {
      const int m = row / Wt, r = row - m * Wt;
      const int s = w.s0 + r;
      for (int k = lane; k < K; k += 32) {
        const int i = (m * W + r) * K + k;
        float bv = sm.Xs[i];
        int ba = Xi[i];
        for (int qq = 1; qq < as.parts; ++qq) {
          const float v = sm.Xs[qq * MWK + i];
          if (v > bv) {
            bv = v;
            ba = Xi[qq * MWK + i];
          }
        }
        sm.Vs[(m * W + r) * Kv + k] = bv;
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
        if (t == 1 && p.v1) p.v1[as.off_v1 + o] = (float)((double)bv + lvl);
      }
    }
  }
  __syncthreads();

  // 5. EV'_{t-1} of the item's own rows
  if (t > as.t_lo) expectation(as, w, t - 1, sm.Ps, sm.Vs, ev_ptr(as, t - 1));
  return true;
}

template <int R>
__global__ void __launch_bounds__(kMaxBlock, 1) sweep_kernel(const SweepParams p) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  __shared__ int s_abort;
  __shared__ double s_lvl[2];
  __shared__ float s_lam[128];
  __shared__ float s_delta[128];
  __shared__ float s_ref;
  __shared__ __align__(8) uint64_t s_bar;
  Smem sm;
  sm.Es = smem + p.sm_E;
  sm.Rt = smem + p.sm_R;
  sm.Vs = smem + p.sm_V;
  sm.Ps = smem + p.sm_P;
  sm.Xs = smem + p.sm_X;
  sm.Ecol = smem + p.sm_C;
  sm.Ccol = sm.Ecol;
  sm.lvl = s_lvl;
  sm.lam = s_lam;
  sm.delta = s_delta;
  sm.ref = &s_ref;
  sm.abort = &s_abort;
  sm.bar = &s_bar;
  const int i0 = p.cta_items[blockIdx.x], i1 = p.cta_items[blockIdx.x + 1];
  if (threadIdx.x == 0) {
    s_abort = 0;
    mbar_init(&s_bar);
  }
  __syncthreads();
  uint32_t parity = 0;

  // prologue: EV'_{t_hi} = P_{t_hi} V'_{t_hi+1} for the item's rows
  for (int it = i0; it < i1; ++it) {
    const WorkItem w = p.items[it];
    const AssetDev& as = p.assets[w.asset];
    const float* vst = as.v_start ? as.v_start : p.terminal + as.off_terminal;
    prefetch_trans(p, as, as.t_hi, sm.Ps);
    const int Wt = w.s1 - w.s0, K = as.K;
    for (int i = threadIdx.x; i < as.M * Wt * K; i += blockDim.x) {
      const int k = i % K, r = (i / K) % Wt, m = i / (K * Wt);
      sm.Vs[(m * as.W + r) * (K + 1) + k] =
          __ldcg(vst + ((size_t)m * as.N + w.s0 + r) * K + k);
    }
    if (threadIdx.x == 0) {
      const double c0 = as.c_start ? *as.c_start : 0.0;
      p.item_c[it] = c0;
      if (w.tile == 0) as.off[as.t_hi + 1] = c0;
    }
    cp_async_wait_all();
    __syncthreads();
    expectation(as, w, as.t_hi, sm.Ps, sm.Vs, ev_ptr(as, as.t_hi));
    publish(p.flags + as.flag_base + w.tile, 1);
    __syncthreads();
  }

  for (int g = 0; g < p.n_steps; ++g) {
    for (int it = i0; it < i1; ++it) {
      const WorkItem w = p.items[it];
      const AssetDev& as = p.assets[w.asset];
      if (g > as.t_hi - as.t_lo) continue;
      sm.Ccol = sm.Ecol + as.M * as.rs;
      if (!item_stage<R>(p, as, w, it, g, sm, parity)) return;
      publish(p.flags + as.flag_base + w.tile, g + 2);
    }
  }
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
