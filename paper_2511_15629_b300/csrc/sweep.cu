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
//      memory with 16-byte cp.async copies by every thread (rows outside the
//      grid are -inf: the infeasibility mask of Alg. 1);
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
//
// The kernel is compiled as sweep_kernel<R, KH>: R rows per thread, and KH =
// 32 (every asset has K = 63 or 64: the shared EV row stride is a compile-time
// constant), -1 (the batch variant: paths that only launches with K not a
// multiple of 4 or one action part take) or 0 (general).  The variants give
// the same results; keeping rarely taken paths out of a variant keeps its
// loop's register allocation as it is.
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cstdint>

#include "../../include/esdp.h"
#include "esdp_internal.h"

namespace esdp {
namespace {

// Per-phase cycle counters of thread 0 (a build with -DESDP_PHASE_CLOCKS
// only; otherwise these compile to nothing).  PHASE_MARK(i) adds the cycles
// since the previous mark to phase i.
#ifdef ESDP_PHASE_CLOCKS
struct PhaseClock {
  unsigned long long last = 0, acc[kPhases + 1] = {};
};
#define PHASE_DECL PhaseClock& pc,
#define PHASE_ARG pc,
#define PHASE_MARK(i)                                    \
  do {                                                   \
    if (threadIdx.x == 0) {                              \
      const unsigned long long now_ = clock64();         \
      pc.acc[(i)] += now_ - pc.last;                     \
      pc.last = now_;                                    \
    }                                                    \
  } while (0)
#else
#define PHASE_DECL
#define PHASE_ARG
#define PHASE_MARK(i) \
  do {                \
  } while (0)
#endif

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

// Two independent round-to-nearest float32 operations per instruction
// (one per price state of a pair); each lane equals the scalar operation.
// (v, c) of this lane or of lane ^ d: the larger value, on equal values the
// smaller chunk index (-1, no feasible action, compares as the largest)
__device__ __forceinline__ void merge_part(float& v, int& c, int d) {
  const float ov = __shfl_xor_sync(0xffffffffu, v, d);
  const int oc = __shfl_xor_sync(0xffffffffu, c, d);
  if (ov > v || (ov == v && (unsigned)oc < (unsigned)c)) {
    v = ov;
    c = oc;
  }
}

__device__ __forceinline__ float2 add2(float2 a, float2 b) {
  unsigned long long x = *reinterpret_cast<unsigned long long*>(&a);
  unsigned long long y = *reinterpret_cast<unsigned long long*>(&b), r;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(x), "l"(y));
  return *reinterpret_cast<float2*>(&r);
}

__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) {
  unsigned long long x = *reinterpret_cast<unsigned long long*>(&a);
  unsigned long long y = *reinterpret_cast<unsigned long long*>(&b);
  unsigned long long z = *reinterpret_cast<unsigned long long*>(&c), r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(x), "l"(y), "l"(z));
  return *reinterpret_cast<float2*>(&r);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void cp_async4(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(dst)), "l"(src)
               : "memory");
}

__device__ __forceinline__ void cp_async8(void* dst, const void* src) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(smem_u32(dst)), "l"(src)
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

// Shared-memory regions and barriers of the sweep CTA.
struct Smem {
  float *Es, *Vs, *Ps, *Xs;
  float2* EC;      // [M][rs] (grid energy e_a, -(cost_a + switch)), -inf padding
  double* lvl;     // [2]: c_{t+1}, c_t
  float* lam;      // [K] prices of the stage
  double* rho;     // [K] row sums of P_{t-1}
  float* delta;    // [K] level correction of the stage
  float* ref;      // EV'_t[ref]
  int* abort;
  uint64_t* barP;  // transposed P bulk copy
  float *Ah, *Al;  // tcgen05 A operand: V' rows, tf32 hi and lo parts
  uint64_t* barM;  // tcgen05 products of the EV contraction
  uint32_t tmem;   // EV accumulator in tensor memory (lane 0, first column)
};

// Issue the asynchronous load of P_t transposed: Ps[k2*Kp4 + k] = trans[t][k][k2].
__device__ __forceinline__ void prefetch_trans(const SweepParams& p, const AssetDev& as, int t,
                                               float* Ps) {
  const int K = as.K, Kpt = p_stride(K);
  const float* P = p.trans + as.off_trans + (size_t)(t - 1) * K * K;
  for (int i = threadIdx.x; i < K * K; i += blockDim.x) {
    const int k2 = i / K, k = i - k2 * K;
    cp_async4(Ps + k2 * Kpt + k, P + (size_t)k * K + k2);
  }
}

// Start loading P_t into shared memory: one bulk copy of the prepared copy
// when there is one (transposed, or the tensor-core operand parts; completion
// on `bar`), else the cp.async gather of P_t^T above.  Returns true if a bulk
// copy was issued.
__device__ __forceinline__ bool load_trans_async(const SweepParams& p, const AssetDev& as, int t,
                                                 float* Ps, uint64_t* bar) {
  if (as.ptrans) {
    if (threadIdx.x == 0) {
      const int K = as.K;
      const uint32_t per = as.tc ? 2u * K * K : (uint32_t)K * p_stride(K);
      asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
      mbar_expect_tx(bar, per * 4u);
      bulk_load(Ps, as.ptrans + (size_t)(t - 1) * per, per * 4u, bar);
    }
    return true;
  }
  prefetch_trans(p, as, t, Ps);
  return false;
}

// EV rows of the item (eq. 6) from V' in shared memory (row stride K+1):
// each thread forms NR rows x 4 price states from float4 reads of P^T; the
// sum over k2 runs in ascending order with one fma per term.  `te` is the
// stage of the EV being produced; its reference entry also goes to its own
// per-stage slot.
template <int NR>
__device__ __forceinline__ void expectation_rows(const AssetDev& as, const WorkItem& w, int te,
                                                 const float* Ps, const float* Vs, float* dst) {
  const int K = as.K, M = as.M, W = as.W, N = as.N, Kv = v_stride(K), Kpt = p_stride(K);
  const int Wt = w.s1 - w.s0;
  const int G = (K + 3) >> 2;
  const int n_rows = M * Wt;
  const int units = ((n_rows + NR - 1) / NR) * G;
  for (int u = threadIdx.x; u < units; u += blockDim.x) {
    const int g = u % G, rp = u / G;
    const float* v[NR];
    int mm[NR], rr[NR];
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      const int L = min(NR * rp + q, n_rows - 1);
      mm[q] = L / Wt;
      rr[q] = L - mm[q] * Wt;
      v[q] = Vs + (mm[q] * W + rr[q]) * Kv;
    }
    const float* pp = Ps + 4 * g;
    float a[NR][4];
#pragma unroll
    for (int q = 0; q < NR; ++q) a[q][0] = a[q][1] = a[q][2] = a[q][3] = 0.f;
#pragma unroll 4
    for (int k2 = 0; k2 < K; ++k2) {
      const float4 pq = *reinterpret_cast<const float4*>(pp + k2 * Kpt);
#pragma unroll
      for (int q = 0; q < NR; ++q) {
        const float x = v[q][k2];
        a[q][0] = fmaf(pq.x, x, a[q][0]);
        a[q][1] = fmaf(pq.y, x, a[q][1]);
        a[q][2] = fmaf(pq.z, x, a[q][2]);
        a[q][3] = fmaf(pq.w, x, a[q][3]);
      }
    }
#pragma unroll
    for (int q = 0; q < NR; ++q) {
      if (NR * rp + q >= n_rows) break;
      float* d = dst + ((size_t)mm[q] * N + w.s0 + rr[q]) * K + 4 * g;
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (4 * g + j < K) __stcg(d + j, a[q][j]);
      if (mm[q] == 0 && g == 0 && w.s0 + rr[q] == as.ref_row) __stcg(as.ref_hist + te, a[q][0]);
    }
  }
}

__device__ __forceinline__ uint32_t to_tf32(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

// x = hi + lo with hi, lo exactly representable in tf32 (lo carries the next
// 11 bits): the products hi*hi + hi*lo + lo*hi keep float32 accuracy.
__device__ __forceinline__ void split_tf32(float x, uint32_t& hi, uint32_t& lo) {
  hi = to_tf32(x);
  lo = to_tf32(x - __uint_as_float(hi));
}

// V'_t entry (mode m, tile row r, state k) into the V tile and, on the
// tensor-core path, into the two A operand parts (row m * Wt + r).
__device__ __forceinline__ void put_v(float* Vs, float* Ah, float* Al, const AssetDev& as, int Wt,
                                      int m, int r, int k, float v) {
  Vs[(m * as.W + r) * v_stride(as.K) + k] = v;
  if (as.tc) {
    uint32_t hi, lo;
    split_tf32(v, hi, lo);
    const int o = tc_offset(m * Wt + r, k, as.K, kCmA);
    Ah[o] = __uint_as_float(hi);
    Al[o] = __uint_as_float(lo);
  }
}

__device__ __forceinline__ void mma_tf32(float (&d)[4], const uint32_t (&a)[4], uint32_t b0,
                                         uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, "
      "{%8,%9}, {%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// EV rows of the item on the tensor cores (K a multiple of 8): the dense
// product [M*Wt x K] = V' [M*Wt x K] . P^T [K x K] in 16x8x8 tf32 tiles,
// float32-accurate through the three-product split, float32 accumulation.
// A warp owns one 16-row block and two 8-column blocks at a time.
__device__ void expectation_mma(const AssetDev& as, const WorkItem& w, int te, const float* Ps,
                                const float* Vs, float* dst) {
  const int K = as.K, M = as.M, W = as.W, N = as.N, Kv = v_stride(K), Kpt = p_stride(K);
  const int Wt = w.s1 - w.s0, n_rows = M * Wt;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int gq = lane >> 2, tq = lane & 3;
  const int MT = (n_rows + 15) >> 4, NT2 = ((K >> 3) + 1) >> 1;
  for (int u = warp; u < MT * NT2; u += nwarps) {
    const int mt = u / NT2, nt = (u - mt * NT2) * 2;
    const bool two = nt + 1 < (K >> 3);
    // the two A rows of this lane (clamped: rows past the tile are computed, not stored)
    const int L0 = min(mt * 16 + gq, n_rows - 1), L1 = min(mt * 16 + gq + 8, n_rows - 1);
    const int m0 = L0 / Wt, r0 = L0 - m0 * Wt, m1 = L1 / Wt, r1 = L1 - m1 * Wt;
    const float* A0 = Vs + (m0 * W + r0) * Kv;
    const float* A1 = Vs + (m1 * W + r1) * Kv;
    // independent accumulators (by product term and by k-step parity) keep
    // the chains of dependent mma short; they are summed at the end
    float hh[2][2][4] = {}, xx[2][2][4] = {};  // [n-tile][k parity][frag]
    for (int k0 = 0; k0 < K; k0 += 8) {
      const int par = (k0 >> 3) & 1;
      uint32_t ah[4], al[4];
      split_tf32(A0[k0 + tq], ah[0], al[0]);
      split_tf32(A1[k0 + tq], ah[1], al[1]);
      split_tf32(A0[k0 + tq + 4], ah[2], al[2]);
      split_tf32(A1[k0 + tq + 4], ah[3], al[3]);
      const float* B = Ps + (k0 + tq) * Kpt + nt * 8 + gq;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (h == 1 && !two) break;
        uint32_t bh0, bl0, bh1, bl1;
        split_tf32(B[8 * h], bh0, bl0);
        split_tf32(B[4 * Kpt + 8 * h], bh1, bl1);
        if (par == 0) {
          mma_tf32(xx[h][0], al, bh0, bh1);
          mma_tf32(xx[h][0], ah, bl0, bl1);
          mma_tf32(hh[h][0], ah, bh0, bh1);
        } else {
          mma_tf32(xx[h][1], al, bh0, bh1);
          mma_tf32(xx[h][1], ah, bl0, bl1);
          mma_tf32(hh[h][1], ah, bh0, bh1);
        }
      }
    }
    float d0[4], d1[4];
#pragma unroll
    for (int f = 0; f < 4; ++f) {
      d0[f] = (hh[0][0][f] + hh[0][1][f]) + (xx[0][0][f] + xx[0][1][f]);
      d1[f] = (hh[1][0][f] + hh[1][1][f]) + (xx[1][0][f] + xx[1][1][f]);
    }
    // d[0..1]: row gq, columns 2tq, 2tq+1; d[2..3]: row gq + 8
#pragma unroll
    for (int hrow = 0; hrow < 2; ++hrow) {
      const int L = mt * 16 + gq + 8 * hrow;
      if (L >= n_rows) continue;
      const int m = L / Wt, r = L - m * Wt;
      float* drow = dst + ((size_t)m * N + w.s0 + r) * K;
      const int c0 = nt * 8 + 2 * tq;
      __stcg(drow + c0, d0[2 * hrow]);
      __stcg(drow + c0 + 1, d0[2 * hrow + 1]);
      if (two) {
        __stcg(drow + c0 + 8, d1[2 * hrow]);
        __stcg(drow + c0 + 9, d1[2 * hrow + 1]);
      }
      if (m == 0 && c0 == 0 && w.s0 + r == as.ref_row) __stcg(as.ref_hist + te, d0[2 * hrow]);
    }
  }
}

// ---- tcgen05 (5th-generation tensor cores, accumulator in tensor memory)

// Shared-memory operand descriptor: start address, leading (K-adjacent core
// matrices) and stride (8-row groups) byte offsets, descriptor version 1, no
// swizzle.
__device__ __forceinline__ uint64_t tc_desc(const float* p, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((smem_u32(p) >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
}

// D[128 x N] (+)= A . B^T, tf32 inputs, float32 accumulation in tensor memory
__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc,
                                       uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(bar))
      : "memory");
}

__device__ __forceinline__ void tc_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 16 consecutive float32 columns of this warp's 32 tensor-memory lanes
__device__ __forceinline__ void tc_load16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,"
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

// EV rows of the item on tcgen05: D[L][k] = sum_k2 A[L][k2] B[k][k2] with
// A the tile's V' rows (row L = m * Wt + r) and B = P_te, both split into tf32
// hi + lo parts; per k-step of 8 the products hi.lo, lo.hi and hi.hi
// accumulate in float32 in tensor memory (float32-accurate).  Blocks of 64
// rows (an M = 64 MMA keeps row i in lane 32 * (i / 16) + i % 16); thread 0
// issues the MMAs and commits them to `barM`, the warps of each lane quarter
// read their 16 rows back, 16 columns at a time, and store them.  A bounded
// wait that expires leaves ESDP_ETIMEOUT in the status word (the next
// neighbour wait then abandons the launch).
__device__ void expectation_tc(const SweepParams& p, const AssetDev& as, const WorkItem& w, int te,
                               const Smem& sm, uint32_t& parity_m) {
  const int K = as.K, N = as.N;
  const int Wt = w.s1 - w.s0, n_rows = as.M * Wt;
  const int nblk = (n_rows + 63) >> 6;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nwarps = blockDim.x >> 5;
  const int q = warp & 3, nq = (nwarps - q + 3) >> 2, wi = warp >> 2;
  float* dst = ev_ptr(as, te);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");  // V' parts -> tensor core
  for (int blk = 0; blk < nblk; ++blk) {
    tc_before_sync();
    __syncthreads();
    tc_after_sync();
    if (threadIdx.x == 0) {
      const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(K >> 3) << 17) |
                             ((uint32_t)(64 >> 4) << 24);
      const uint32_t sbo_a = (uint32_t)(K >> 2) * kCmA * 4u, sbo_b = (uint32_t)(K >> 2) * kCmB * 4u;
      const int o = blk * 8 * (K >> 2) * kCmA;  // 8 row groups per 64 rows
      // k-step st covers core-matrix columns 2st, 2st + 1: the start address
      // (16-byte units, low bits of the descriptor) advances by 2 cm floats
      const uint64_t ah = tc_desc(sm.Ah + o, kCmA * 4u, sbo_a);
      const uint64_t al = tc_desc(sm.Al + o, kCmA * 4u, sbo_a);
      const uint64_t bh = tc_desc(sm.Ps, kCmB * 4u, sbo_b);
      const uint64_t bl = tc_desc(sm.Ps + K * K, kCmB * 4u, sbo_b);
      for (int st = 0; st < (K >> 3); ++st) {
        const uint64_t da = (uint64_t)(st * kCmA / 2), db = (uint64_t)(st * kCmB / 2);
        tc_mma(sm.tmem, ah + da, bl + db, idesc, st > 0);
        tc_mma(sm.tmem, al + da, bh + db, idesc, 1u);
        tc_mma(sm.tmem, ah + da, bh + db, idesc, 1u);
      }
      tc_commit(sm.barM);
    }
    const int row0 = blk * 64 + 16 * q;  // first row of this warp's lane quarter
    if (row0 < n_rows && mbar_wait_bounded(sm.barM, parity_m, p)) {
      tc_after_sync();
      for (int c0 = 16 * wi; c0 < K; c0 += 16 * nq) {
        float v[16];
        tc_load16(sm.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
        const int L = row0 + lane;
        if (lane < 16 && L < n_rows) {
          const int m = L / Wt, r = L - m * Wt;
          float4* d4 = reinterpret_cast<float4*>(dst + ((size_t)m * N + w.s0 + r) * K + c0);
#pragma unroll
          for (int j = 0; j < 4; ++j)
            __stcg(d4 + j, make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]));
          if (m == 0 && c0 == 0 && w.s0 + r == as.ref_row) __stcg(as.ref_hist + te, v[0]);
        }
      }
    }
    parity_m ^= 1u;
  }
  tc_before_sync();
}


__device__ __forceinline__ void expectation(const SweepParams& p, const AssetDev& as,
                                            const WorkItem& w, int te, const Smem& sm,
                                            uint32_t& parity_m) {
  if (as.tc) {
    expectation_tc(p, as, w, te, sm, parity_m);
    return;
  }
  const float* Ps = sm.Ps;
  const float* Vs = sm.Vs;
  float* dst = ev_ptr(as, te);
  if (as.mma) {
    expectation_mma(as, w, te, Ps, Vs, dst);
    return;
  }
  const int n_rows = as.M * (w.s1 - w.s0), G = (as.K + 3) >> 2;
  if (((n_rows + 1) / 2) * G * 4 >= (int)blockDim.x * 3)
    expectation_rows<2>(as, w, te, Ps, Vs, dst);
  else
    expectation_rows<1>(as, w, te, Ps, Vs, dst);
}

// Release the item's EV rows.  Other CTAs read them with cp.async or plain
// loads (generic proxy) after an acquire of the flag, so the barrier and one
// release store order them; a reader through bulk copies (async proxy) would
// also need a proxy fence here.
__device__ __forceinline__ void publish(int* flag, int v) {
  __syncthreads();
  if (threadIdx.x == 0) st_release(flag, v);
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
      for (unsigned it = 1;; ++it) {
        if (ld_acquire(f) >= need) break;
        if ((it & 15u) == 0) {  // the abort checks cost a round trip: not every poll
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
    if ((int)threadIdx.x == n) *s_ref = __ldcg(as.ref_hist + t);
  }
  __syncthreads();
  return *(volatile int*)s_abort == 0;
}


// Payoff columns of each mode: (e_a, -(cost_a + switch)), -inf padding to a
// multiple of R per action segment; the payoff r = price*e_a - cost_a is
// formed in the max-plus itself.  They depend on the asset only.
template <int R>
__device__ void build_columns(const SweepParams& p, const AssetDev& as, float2* EC) {
  const int M = as.M, rs = as.rs;
  const float NEG = -CUDART_INF_F;
  const float* cost = p.cost + as.off_cost;
  for (int i = threadIdx.x; i < M * rs; i += blockDim.x) {
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
    EC[i] = a >= 0 ? make_float2(__ldg(as.e + a), -__ldg(cost + a) - sw) : make_float2(0.f, NEG);
  }
}

// One chunk of R actions for R rows and a pair of price states.  `eb` points
// at the EV pair of the chunk's first action for the first row (rows and
// actions both step by one EV row), `ecp` at the chunk's payoff columns.
// Each running maximum takes the chunk's R candidates in one chain of 3-input
// maxima; the chunk index is recorded where a maximum strictly rises, so the
// earliest chunk that attains it is kept.
// The chunk's window is wv[OFF .. OFF + 2R - 1) of registers the caller
// loaded (one chunk's 2R - 1 rows, or two consecutive chunks' 3R - 1).
template <int R, int OFF, int NW>
__device__ __forceinline__ void maxplus_core(const float2 (&wv)[NW], const float2* ecp, float2 lam,
                                             int c, float2 (&best)[R], int (&bx)[R],
                                             int (&by)[R]) {
  static_assert(OFF + 2 * R - 1 <= NW, "window");
  float2 rr[R];
#pragma unroll
  for (int i = 0; i < R; ++i) {
    const float2 e = ecp[i];
    rr[i] = fma2(lam, make_float2(e.x, e.x), make_float2(e.y, e.y));
  }
  float2 nm[R];
#pragma unroll
  for (int j = 0; j < R; ++j) {
    const float2 x = add2(rr[0], wv[OFF + j]), y = add2(rr[1], wv[OFF + j + 1]);
    nm[j] = make_float2(max3f(best[j].x, x.x, y.x), max3f(best[j].y, x.y, y.y));
  }
#pragma unroll
  for (int i = 2; i + 1 < R; i += 2) {
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const float2 x = add2(rr[i], wv[OFF + i + j]), y = add2(rr[i + 1], wv[OFF + i + 1 + j]);
      nm[j] = make_float2(max3f(nm[j].x, x.x, y.x), max3f(nm[j].y, x.y, y.y));
    }
  }
  if constexpr ((R & 1) != 0) {  // an odd R: the chunk's last action on its own
#pragma unroll
    for (int j = 0; j < R; ++j) {
      const float2 x = add2(rr[R - 1], wv[OFF + R - 1 + j]);
      nm[j] = make_float2(fmaxf(nm[j].x, x.x), fmaxf(nm[j].y, x.y));
    }
  }
#pragma unroll
  for (int j = 0; j < R; ++j) {
    if (nm[j].x > best[j].x) bx[j] = c;
    if (nm[j].y > best[j].y) by[j] = c;
    best[j] = nm[j];
  }
}

template <int R>
__device__ __forceinline__ void maxplus_chunk(const float2* eb, int Kh, const float2* ecp,
                                              float2 lam, int c, float2 (&best)[R], int (&bx)[R],
                                              int (&by)[R]) {
  float2 wv[2 * R - 1];
#pragma unroll
  for (int x = 0; x < 2 * R - 1; ++x) wv[x] = eb[(size_t)x * Kh];
  maxplus_core<R, 0>(wv, ecp, lam, c, best, bx, by);
}

// Two consecutive chunks c, c + 1 of one action segment: their windows
// overlap in R - 1 rows, so 3R - 1 rows are loaded once for both.
template <int R>
__device__ __forceinline__ void maxplus_pair(const float2* eb, int Kh, const float2* ecp,
                                             float2 lam, int c, float2 (&best)[R], int (&bx)[R],
                                             int (&by)[R]) {
  float2 wv[3 * R - 1];
#pragma unroll
  for (int x = 0; x < 3 * R - 1; ++x) wv[x] = eb[(size_t)x * Kh];
  maxplus_core<R, 0>(wv, ecp, lam, c, best, bx, by);
  maxplus_core<R, R>(wv, ecp + R, lam, c + 1, best, bx, by);
}

// Inputs of stage t of work item `it` that do not depend on other tiles:
// threads below K start copies of the price and the row sum of P_{t-1} of
// their state into shared memory (waited for in the stage with
// cp.async.wait_all), thread 0 takes the item's running level c_{t+1} (from
// shared memory when the item repeats, else from its global slot).
struct StageScalars {
  double c = 0.0;
  bool valid = false;
};

__device__ __forceinline__ void stage_scalars(const SweepParams& p, const AssetDev& as, int t,
                                              int it, const Smem& sm, double& c, bool same) {
  const int K = as.K, tid = threadIdx.x;
  if (tid < K) {
    cp_async4(sm.lam + tid, p.price + as.off_price + (size_t)(t - 1) * K + tid);
    cp_async8(sm.rho + tid, as.rho + (size_t)(t - 1) * K + tid);
  }
  if (tid == 0) c = same ? sm.lvl[1] : *(volatile double*)(p.item_c + it);
}

template <bool FLAT = false>
__device__ void item_outputs(const SweepParams& p, const AssetDev& as, const WorkItem& w, int t,
                             const Smem& sm, int first);

// A stage whose outputs are still to be written (it < 0: none).
struct Deferred {
  int it = -1, t = 0;
  WorkItem w{};
};

// One stage of one work item.  Returns false if the launch is abandoned.
template <int R, int KH>
__device__ bool item_stage(PHASE_DECL const SweepParams& p, const AssetDev& as,
                           const WorkItem& w, int it, int g, const Smem& sm,
                           uint32_t& parity_p, uint32_t& parity_m, bool p_pref,
                           const StageScalars& pre, const Deferred& def) {
  const int t = as.t_hi - g;
  const int K = as.K, M = as.M, N = as.N, rows = as.rows, rs = as.rs, W = as.W;
  const int tid = threadIdx.x, nth = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const float NEG = -CUDART_INF_F;
  // EV tile row stride: price states in pairs (a compile-time constant in
  // the launches whose assets all have K = 2 KH - 1 or 2 KH, so that the
  // register window is loaded with immediate offsets)
  const int Ke = KH > 0 ? 2 * KH : K + (K & 1);

  // 0. inputs of the stage: the bulk copy of P_{t-1} and the per-thread
  // scalars (price, row sum, running level) may already be in flight, issued
  // right after the previous stage's release
  const bool p_bulk = p_pref || (t > as.t_lo && load_trans_async(p, as, t - 1, sm.Ps, sm.barP));
  double c_next = pre.c;
  if (!pre.valid) stage_scalars(p, as, t, it, sm, c_next, false);
  PHASE_MARK(0);

  // 1. neighbours; meanwhile the warps that do not poll write the previous
  //    stage's outputs (its V' tile and indices are still in place)
  if (def.it >= 0) {
    const int n_wait = min(as.n_tiles - 1, w.tile + as.wait_hi) - max(0, w.tile + as.wait_lo) + 2;
    const int first = (n_wait + 31) & ~31;
    item_outputs<(KH < 0)>(p, as, def.w, def.t, sm, first < (int)blockDim.x ? first : 0);
  }
  if (!wait_neighbours(p, as, w, g + 1 + p.wait_extra, t, sm.abort, sm.ref)) {
    // abandoning the launch: first let this CTA's own copy of P_{t-1} land
    // (bounded), so that no bulk copy into its shared memory is in flight
    if (p_bulk && tid == 0) mbar_wait_bounded(sm.barP, parity_p, p);
    return false;
  }
  PHASE_MARK(1);

  // 2. EV_t tile: copies of the rows inside the grid, -inf outside
  const float* ev_t = ev_ptr(as, t);
  const int g0row = w.s0 - as.D_dis;
  const int lo = max(g0row, 0), hi = min(g0row + rows, N);
  if ((K & 3) == 0) {
    // 16-byte cp.async copies by every thread (generic proxy: the producers
    // need no proxy fence before their release)
    const int n16 = (hi - lo) * (K >> 2);
    for (int m = 0; m < M; ++m) {
      const float4* src = reinterpret_cast<const float4*>(ev_t + ((size_t)m * N + lo) * K);
      float4* dst = reinterpret_cast<float4*>(sm.Es + ((size_t)m * rows + (lo - g0row)) * K);
      for (int i = tid; i < n16; i += nth)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(dst + i)),
                     "l"(src + i)
                     : "memory");
    }
  } else if (KH < 0) {
    // (the batch variant) K not a multiple of 4: L2 loads of eight elements
    // per thread in flight before their shared stores (a row of odd K gets a
    // pad column)
    for (int m = 0; m < M; ++m) {
      const float* src = ev_t + ((size_t)m * N + lo) * K;
      float* dst = sm.Es + ((size_t)m * rows + (lo - g0row)) * Ke;
      const int n = (hi - lo) * K;
      for (int i0 = tid; i0 < n; i0 += 8 * nth) {
        float v[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + q * nth;
          v[q] = i < n ? __ldcg(src + i) : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int i = i0 + q * nth;
          if (i < n) dst[Ke == K ? i : i + i / K] = v[q];
        }
      }
      if (Ke != K)
        for (int r = tid; r < hi - lo; r += nth) dst[r * Ke + K] = NEG;  // pad column
    }
  } else {
    for (int m = 0; m < M; ++m) {
      const float* src = ev_t + ((size_t)m * N + lo) * K;
      float* dst = sm.Es + ((size_t)m * rows + (lo - g0row)) * Ke;
      const int n = (hi - lo) * K;
      if (Ke == K) {
        for (int i = tid; i < n; i += nth) dst[i] = __ldcg(src + i);
      } else {
        for (int i = tid; i < n; i += nth) {
          const int r = i / K;
          dst[i + r] = __ldcg(src + i);
        }
        for (int r = tid; r < hi - lo; r += nth) dst[r * Ke + K] = NEG;  // pad column
      }
    }
  }
  {
    const int below = (lo - g0row) * Ke, above0 = (hi - g0row) * Ke, total = rows * Ke;
    for (int m = 0; m < M; ++m) {
      float* e = sm.Es + (size_t)m * rows * Ke;
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
  cp_async_wait_all();
  __syncthreads();
  if (tid < K) {
    const double cr = sm.lvl[0] * sm.rho[tid];
    sm.delta[tid] = (float)(cr - sm.lvl[1]);
    if (w.tile == 0) as.evoff[(size_t)(t - 1) * K + tid] = cr;
  }
  if (tid == K && (K & 1)) sm.lam[K] = 0.f;  // pad state of an odd K
  if (p_bulk) {
    if (tid == 0 && !mbar_wait_bounded(sm.barP, parity_p, p)) *(volatile int*)sm.abort = 1;
    parity_p ^= 1u;
  }
  __syncthreads();
  if (*(volatile int*)sm.abort) return false;
  PHASE_MARK(2);

  // 3. banded max-plus.  A cell is (pair of price states, block of R rows,
  //    mode); its chunks of R actions are split over G = parts thread groups
  //    (contiguous ranges, or every G-th chunk, see below).  A warp holds
  //    L = 32/G cells in each of the G groups (lane = cell slot + L * part),
  //    so the parts of a cell meet in one warp and are merged by shuffles.
  //    Each lane slides a register window of EV pairs over its chunks: two
  //    evaluations per packed add and per 3-input max.
  const int Kh = KH > 0 ? KH : Ke >> 1;
  const int G = as.parts, lgL = 5 - (31 - __clz(G)), L = 32 >> (31 - __clz(G));
  const int ncell = Kh * as.nb * M;
  int* Xi = reinterpret_cast<int*>(sm.Xs);
  const int Wt = w.s1 - w.s0, Kv = v_stride(K);
  if (warp * L < ncell) {  // warp-uniform: every lane takes part in the shuffles
    const int part = lane >> lgL;
    const int cell = warp * L + (lane & (L - 1));
    const bool active = cell < ncell;
    const int cc = active ? cell : 0;
    const int kp = cc % Kh;
    int q = cc / Kh;
    const int b = q % as.nb;
    const int m = q / as.nb;
    const int k0 = 2 * kp;
    Seg g0, g1;
    segments(as, m, g0, g1);
    const int n0 = round_up(g0.len, R) / R;
    const int nc = n0 + round_up(g1.len, R) / R;
    // R >= 6: each part takes a contiguous range of chunks (consecutive
    // chunks share R - 1 window rows); R < 6: part p takes the chunks p,
    // p + G, p + 2G, ..., so that the lanes of a warp read rows R apart and
    // their shared-memory loads spread over the banks
    const int c_lo = R >= 6 ? part * nc / G : part;
    const int c_hi = !active ? c_lo : R >= 6 ? (part + 1) * nc / G : nc;
    const float2* ec = sm.EC + m * rs;
    const float2 lam = make_float2(sm.lam[k0], sm.lam[k0 + 1]);
    float2 best[R];
    int bx[R], by[R];
#pragma unroll
    for (int j = 0; j < R; ++j) {
      best[j] = make_float2(NEG, NEG);
      bx[j] = -1;
      by[j] = -1;
    }
    auto chunk = [&](int c, float2 (&bst)[R], int (&cx)[R], int (&cy)[R]) {
      const bool second = c >= n0;
      const int u0 = (second ? c - n0 : c) * R;
      const int a0 = second ? g1.a0 : g0.a0;
      const int src = second ? g1.src : g0.src;
      const int toff = second ? n0 * R : 0;
      const float2* eb =
          reinterpret_cast<const float2*>(sm.Es + ((size_t)src * rows + b * R + a0 + u0) * Ke) + kp;
      maxplus_chunk<R>(eb, Kh, ec + toff + u0, lam, c, bst, cx, cy);
    };
    // two chunks per iteration where the registers allow: independent loads
    // and max chains in flight
    int c = c_lo;
    if constexpr (R >= 6 && R <= 8) {
      // (for R = 4 the per-chunk windows measured faster: 1.86 vs 1.90 ms on
      // the two-mode 5-minute asset)
      for (; c + 1 < c_hi; c += 2) {
        if ((c >= n0) == (c + 1 >= n0)) {
          // both chunks in one action segment: one window of 3R - 1 rows
          const bool second = c >= n0;
          const int u0 = (second ? c - n0 : c) * R;
          const int a0 = second ? g1.a0 : g0.a0;
          const int src = second ? g1.src : g0.src;
          const int toff = second ? n0 * R : 0;
          const float2* eb = reinterpret_cast<const float2*>(
                                 sm.Es + ((size_t)src * rows + b * R + a0 + u0) * Ke) + kp;
          maxplus_pair<R>(eb, Kh, ec + toff + u0, lam, c, best, bx, by);
        } else {
          chunk(c, best, bx, by);
          chunk(c + 1, best, bx, by);
        }
      }
    }
    if constexpr (R < 6) {
      for (; c + G < c_hi; c += 2 * G) {
        chunk(c, best, bx, by);
        chunk(c + G, best, bx, by);
      }
      for (; c < c_hi; c += G) chunk(c, best, bx, by);
    } else {
      for (; c < c_hi; ++c) chunk(c, best, bx, by);
    }
    PHASE_MARK(3);
    // merge the parts of each cell: the larger value, on equal values the
    // earlier chunk
    for (int d = L; d < 32; d <<= 1) {
#pragma unroll
      for (int j = 0; j < R; ++j) {
        merge_part(best[j].x, bx[j], d);
        merge_part(best[j].y, by[j], d);
      }
    }
    // exact argmax of each entry e = 2 j + h (row j, state k0 + h), spread
    // over the parts: lane `part` takes e = part, part + G, ... in rounds, so
    // every lane of a warp runs the same code.  The first action of the
    // winning chunk that reproduces the max (the same two round-to-nearest
    // operations as the packed evaluation); V'_t = max + c_{t+1} rho_t[k] - c_t
    if (active) {
      // argmax of one entry (row j, state k0 + h) from its max bj and winning
      // chunk c, without stores, so that the loads of all of a lane's entries
      // can be in flight together; -1 for padding entries
      auto argmax_of = [&](int j, int h, float bj, int c) -> int {
        const int row = b * R + j, k = k0 + h;
        if (c < 0 || k >= K || row >= Wt) return -1;
        const float lk = h ? lam.y : lam.x;
        const bool second = c >= n0;
        const int u0 = (second ? c - n0 : c) * R;
        const int a0 = second ? g1.a0 : g0.a0;
        const int src = second ? g1.src : g0.src;
        const int toff = second ? n0 * R : 0;
        const float* eb = sm.Es + ((size_t)src * rows + row + a0 + u0) * Ke + k;
        const float2* ep = ec + toff + u0;
        float v[R];
#pragma unroll
        for (int i = 0; i < R; ++i) {
          const float2 ei = ep[i];
          v[i] = fmaf(lk, ei.x, ei.y) + eb[(size_t)i * Ke];
        }
        int first = R - 1;
#pragma unroll
        for (int i = R - 1; i >= 0; --i)
          if (v[i] == bj) first = i;
        return a0 + u0 + first;
      };
      // V'_t and the argmax of an entry into the V tile (and the tcgen05
      // operand parts) and the index tile; the asset fields are read once,
      // before any store (the descriptor lives in shared memory)
      const int tcv = as.tc;
      float* Vs = sm.Vs;
      float* Ah = sm.Ah;
      float* Al = sm.Al;
      auto store = [&](int j, int h, float bj, int arg) {
        const int row = b * R + j, k = k0 + h;
        if (k >= K || row >= Wt) return;
        const float v = bj + sm.delta[k];
        Vs[(m * W + row) * Kv + k] = v;
        if (tcv) {
          uint32_t hi, lo;
          split_tf32(v, hi, lo);
          const int o = tc_offset(m * Wt + row, k, K, kCmA);
          Ah[o] = __uint_as_float(hi);
          Al[o] = __uint_as_float(lo);
        }
        Xi[(m * W + row) * K + k] = arg;
      };
      if (G == 2) {
        // lane `part` takes state k0 + part of every row
        int arg[R];
#pragma unroll
        for (int j = 0; j < R; ++j)
          arg[j] = argmax_of(j, part, part ? best[j].y : best[j].x, part ? by[j] : bx[j]);
#pragma unroll
        for (int j = 0; j < R; ++j) store(j, part, part ? best[j].y : best[j].x, arg[j]);
      } else if (G == 4 && (R & 1) == 0) {
        // lane `part` takes state k0 + (part & 1) of the rows j = part/2 + 2i
        const int h = part & 1, jo = part >> 1;
        int arg[R / 2];
        float bv[R / 2];
#pragma unroll
        for (int i = 0; i < R / 2; ++i) {
          const float2 bb = jo ? best[2 * i + 1] : best[2 * i];
          const int cx = jo ? bx[2 * i + 1] : bx[2 * i], cy = jo ? by[2 * i + 1] : by[2 * i];
          bv[i] = h ? bb.y : bb.x;
          arg[i] = argmax_of(2 * i + jo, h, bv[i], h ? cy : cx);
        }
#pragma unroll
        for (int i = 0; i < R / 2; ++i) store(2 * i + jo, h, bv[i], arg[i]);
      } else if (KH < 0 && G == 1) {
        // (the batch variant) one lane holds both states of every row: where the two states won
        // in the same chunk, one scan reads each EV pair and payoff column
        // once (the same two round-to-nearest operations per candidate)
#pragma unroll
        for (int j = 0; j < R; ++j) {
          const int cx = bx[j], cy = by[j];
          int ax, ay;
          if (cx == cy && cx >= 0 && b * R + j < Wt) {
            const bool second = cx >= n0;
            const int u0 = (second ? cx - n0 : cx) * R;
            const int a0 = second ? g1.a0 : g0.a0;
            const int src = second ? g1.src : g0.src;
            const int toff = second ? n0 * R : 0;
            const float2* eb2 = reinterpret_cast<const float2*>(
                sm.Es + ((size_t)src * rows + b * R + j + a0 + u0) * Ke + k0);
            const float2* ep = ec + toff + u0;
            int fx = R - 1, fy = R - 1;
#pragma unroll
            for (int i = R - 1; i >= 0; --i) {
              const float2 ei = ep[i];
              const float2 ev = eb2[(size_t)i * (Ke >> 1)];
              if (fmaf(lam.x, ei.x, ei.y) + ev.x == best[j].x) fx = i;
              if (fmaf(lam.y, ei.x, ei.y) + ev.y == best[j].y) fy = i;
            }
            ax = a0 + u0 + fx;
            ay = a0 + u0 + fy;
          } else {
            ax = argmax_of(j, 0, best[j].x, cx);
            ay = argmax_of(j, 1, best[j].y, cy);
          }
          store(j, 0, best[j].x, ax);
          store(j, 1, best[j].y, ay);
        }
      } else {
#pragma unroll 2
        for (int e = part; e < 2 * R; e += G) {
          const int j = e >> 1, h = e & 1;
          float bj = 0.f;
          int c = -1;
#pragma unroll
          for (int jj = 0; jj < R; ++jj)
            if (jj == j) {
              bj = h ? best[jj].y : best[jj].x;
              c = h ? by[jj] : bx[jj];
            }
          store(j, h, bj, argmax_of(j, h, bj, c));
        }
      }
    }
  }
  __syncthreads();
  PHASE_MARK(4);

  // 5. EV'_{t-1} of the item's own rows
  if (t > as.t_lo) expectation(p, as, w, t - 1, sm, parity_m);
  PHASE_MARK(5);
  return true;
}

// The streaming outputs of a stage (policy, values kept for the adjoint,
// checkpoints, V_1), read from the V' tile and the argmax indices: written
// while the next stage of the CTA waits for its neighbours (or right after the
// release when no such stage follows).
// Run by the threads from `first` (a multiple of 32) on.
// FLAT (the batch variant): where the 16-byte path does not apply, the
// entries of each mode's rows are taken as one flat range (contiguous in the
// outputs and the index tile) by all threads, four loads ahead of their
// stores, instead of one row per warp (2.7x faster on the 256-asset batch).
template <bool FLAT>
__device__ void item_outputs(const SweepParams& p, const AssetDev& as, const WorkItem& w, int t,
                             const Smem& sm, int first) {
  const int K = as.K, M = as.M, N = as.N, W = as.W;
  const int lane = threadIdx.x & 31, warp = (threadIdx.x - first) >> 5,
            nwarps = (blockDim.x - first) >> 5;
  if ((int)threadIdx.x < first) return;
  const int* Xi = reinterpret_cast<const int*>(sm.Xs);
  const int Kv = v_stride(K);
  const size_t MNK = mnk(as);
  const int Wt = w.s1 - w.s0;
  const double lvl = sm.lvl[1];
  const bool ck = as.ckpt && as.ckpt_every > 0 && t > 1 && (t - 1) % as.ckpt_every == 0;
  short* pol16 = as.policy_bytes == 2 ? reinterpret_cast<short*>(as.policy) : nullptr;
  int* pol32 = as.policy_bytes == 4 ? reinterpret_cast<int*>(as.policy) : nullptr;
  const size_t pbase = (size_t)(t - as.policy_t_base) * MNK;
  float* vk = as.v_keep ? as.v_keep + (size_t)(t - as.t_lo) * MNK : nullptr;
  float* cp = ck ? as.ckpt + (size_t)((t - 1) / as.ckpt_every - 1) * MNK : nullptr;
  float* v1 = (t == 1 && p.v1) ? p.v1 + as.off_v1 : nullptr;
  const bool vec = (K & 3) == 0 && ((reinterpret_cast<uintptr_t>(as.policy) |
                                      reinterpret_cast<uintptr_t>(as.v_keep) |
                                      reinterpret_cast<uintptr_t>(as.ckpt)) & 15) == 0;
  if (vec) {
    // four states per thread: 16-byte shared reads and global stores (the
    // per-stage and per-row offsets are multiples of 4 elements; V_1 sits at
    // an arbitrary offset of the caller's array and is written per element)
    const int K4 = K >> 2, n = M * Wt * K4;
    for (int i = threadIdx.x - first; i < n; i += blockDim.x - first) {
      const int row = i / K4, k = (i - row * K4) << 2;
      const int m = row / Wt, r = row - m * Wt;
      const size_t o = ((size_t)m * N + w.s0 + r) * K + k;
      const float4 bv = *reinterpret_cast<const float4*>(sm.Vs + (m * W + r) * Kv + k);
      const int4 ba = *reinterpret_cast<const int4*>(Xi + (m * W + r) * K + k);
      if (pol32) __stcs(reinterpret_cast<int4*>(pol32 + pbase + o), ba);
      if (pol16)
        __stcs(reinterpret_cast<short4*>(pol16 + pbase + o),
               make_short4((short)ba.x, (short)ba.y, (short)ba.z, (short)ba.w));
      if (vk) __stcg(reinterpret_cast<float4*>(vk + o), bv);
      if (cp) __stcg(reinterpret_cast<float4*>(cp + o), bv);
      if (v1) {
        v1[o] = (float)((double)bv.x + lvl);
        v1[o + 1] = (float)((double)bv.y + lvl);
        v1[o + 2] = (float)((double)bv.z + lvl);
        v1[o + 3] = (float)((double)bv.w + lvl);
      }
    }
    return;
  }
  if constexpr (FLAT) {
    const int n = Wt * K, nt = (int)blockDim.x - first;
    for (int m = 0; m < M; ++m) {
      const size_t ob0 = ((size_t)m * N + w.s0) * K;
      const int* xi = Xi + m * W * K;
      for (int i0 = (int)threadIdx.x - first; i0 < n; i0 += 4 * nt) {
        int ba[4];
        float bv[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = i0 + q * nt;
          const int r = i / K, k = i - r * K;
          ba[q] = i < n ? xi[i] : 0;
          bv[q] = i < n ? sm.Vs[(m * W + r) * Kv + k] : 0.f;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = i0 + q * nt;
          if (i >= n) break;
          if (pol32) __stcs(pol32 + pbase + ob0 + i, ba[q]);
          if (pol16) __stcs(pol16 + pbase + ob0 + i, (short)ba[q]);
          if (vk) __stcg(vk + ob0 + i, bv[q]);
          if (cp) __stcg(cp + ob0 + i, bv[q]);
          if (v1) v1[ob0 + i] = (float)((double)bv[q] + lvl);
        }
      }
    }
    return;
  }
  for (int row = warp; row < M * Wt; row += nwarps) {
    const int m = row / Wt, r = row - m * Wt;
    const size_t ob = ((size_t)m * N + w.s0 + r) * K;
    const int ib = (m * W + r) * K, vb = (m * W + r) * Kv;
    for (int k = lane; k < K; k += 32) {
      const float bv = sm.Vs[vb + k];
      const int ba = Xi[ib + k];
      if (pol32) __stcs(pol32 + pbase + ob + k, ba);
      if (pol16) __stcs(pol16 + pbase + ob + k, (short)ba);
      if (vk) __stcg(vk + ob + k, bv);
      if (cp) __stcg(cp + ob + k, bv);
      if (v1) v1[ob + k] = (float)((double)bv + lvl);
    }
  }
}

// The persistent sweep of one CTA: its work items for every stage.  Returns
// early (uniformly over the CTA) when the launch is abandoned.
template <int R, int KH>
__device__ __forceinline__ void sweep_run(const SweepParams& p, const Smem& sm, AssetDev& s_as) {
  const int i0 = p.cta_items[blockIdx.x], i1 = p.cta_items[blockIdx.x + 1];
#ifdef ESDP_PHASE_CLOCKS
  PhaseClock pc;
#endif
  uint32_t parity_p = 0, parity_m = 0;
  // the work item's asset descriptor lives in shared memory: the loops that
  // store to global memory then need not reload its fields
  auto load_asset = [&](int a) {
    const int n = (int)(sizeof(AssetDev) / sizeof(int));
    const int* src = reinterpret_cast<const int*>(p.assets + a);
    int* dst = reinterpret_cast<int*>(&s_as);
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) dst[i] = src[i];
    __syncthreads();
  };
  int cur_asset = -1, cols_asset = -1;
  bool pref = false;
  StageScalars pre;

  // prologue: EV'_{t_hi} = P_{t_hi} V'_{t_hi+1} for the item's rows
  for (int it = i0; it < i1; ++it) {
    const WorkItem w = p.items[it];
    if (w.asset != cur_asset) {
      load_asset(w.asset);
      cur_asset = w.asset;
    }
    const AssetDev& as = s_as;
    const float* vst = as.v_start ? as.v_start : p.terminal + as.off_terminal;
    const bool pb = load_trans_async(p, as, as.t_hi, sm.Ps, sm.barP);
    const int Wt = w.s1 - w.s0, K = as.K;
    for (int i = threadIdx.x; i < as.M * Wt * K; i += blockDim.x) {
      const int k = i % K, r = (i / K) % Wt, m = i / (K * Wt);
      put_v(sm.Vs, sm.Ah, sm.Al, as, Wt, m, r, k,
            __ldcg(vst + ((size_t)m * as.N + w.s0 + r) * K + k));
    }
    if (threadIdx.x == 0) {
      const double c0 = as.c_start ? *as.c_start : 0.0;
      p.item_c[it] = c0;
      if (w.tile == 0) as.off[as.t_hi + 1] = c0;
    }
    cp_async_wait_all();
    if (pb) {
      if (threadIdx.x == 0 && !mbar_wait_bounded(sm.barP, parity_p, p)) *sm.abort = 1;
      parity_p ^= 1u;
    }
    __syncthreads();
    if (*(volatile int*)sm.abort) return;
    expectation(p, as, w, as.t_hi, sm, parity_m);
    publish(p.flags + as.flag_base + w.tile, 1);
    __syncthreads();
  }

  // the next work item's descriptor is read right after each release (off
  // the stage's critical path) and carried over
  int nx_idx = -1;
  WorkItem nx{};
  Deferred def;
#ifdef ESDP_PHASE_CLOCKS
  if (threadIdx.x == 0) pc.last = clock64();
#endif
  for (int g = 0; g < p.n_steps; ++g) {
    for (int it = i0; it < i1; ++it) {
      const WorkItem w = it == nx_idx ? nx : p.items[it];
      if (w.asset != cur_asset && def.it >= 0) {
        item_outputs<(KH < 0)>(p, s_as, def.w, def.t, sm, 0);  // before the descriptor changes
        def.it = -1;
      }
      if (w.asset != cur_asset) {
        load_asset(w.asset);
        cur_asset = w.asset;
      }
      const AssetDev& as = s_as;
      if (g > as.t_hi - as.t_lo) continue;
      if (w.asset != cols_asset) {
        build_columns<R>(p, as, sm.EC);  // read after the barriers of the stage
        cols_asset = w.asset;
      }
      if (!item_stage<R, KH>(PHASE_ARG p, as, w, it, g, sm, parity_p, parity_m, pref, pre, def))
        return;
      def.it = -1;
      publish(p.flags + as.flag_base + w.tile, g + 2);
      PHASE_MARK(6);
      // start the next stage's loads now when that stage is of the same
      // asset: their latency then overlaps the output stores and the wait
      {
        const int nit = it + 1 < i1 ? it + 1 : i0;
        const int ng = it + 1 < i1 ? g : g + 1;
        const int nt = as.t_hi - ng;
        nx = nit == it ? w : p.items[nit];
        nx_idx = nit;
        const bool next = ng < p.n_steps && nx.asset == w.asset && ng <= as.t_hi - as.t_lo;
        pref = next && as.ptrans != nullptr && nt > as.t_lo;
        if (pref) load_trans_async(p, as, nt - 1, sm.Ps, sm.barP);
        pre.valid = next;
        if (next) stage_scalars(p, as, nt, nit, sm, pre.c, nit == it);
        // this stage's outputs: during the next stage's wait when one follows
        // on this asset, else now
        if (next) {
          def.it = it;
          def.t = as.t_hi - g;
          def.w = w;
        } else {
          item_outputs<(KH < 0)>(p, as, w, as.t_hi - g, sm, 0);
        }
      }
      PHASE_MARK(7);
#ifdef ESDP_PHASE_CLOCKS
      if (threadIdx.x == 0) pc.acc[kPhases] += 1;  // stages counted
#endif
    }
  }
  if (def.it >= 0) item_outputs<(KH < 0)>(p, s_as, def.w, def.t, sm, 0);
#ifdef ESDP_PHASE_CLOCKS
  if (threadIdx.x == 0 && p.phase_clk)
    for (int i = 0; i <= kPhases; ++i) p.phase_clk[(size_t)blockIdx.x * (kPhases + 1) + i] = pc.acc[i];
#endif
}

template <int R, int KH>
__global__ void __launch_bounds__(kMaxBlock, 1) sweep_kernel(const SweepParams p) {
  extern __shared__ float4 smem4[];
  float* smem = reinterpret_cast<float*>(smem4);
  __shared__ int s_abort;
  __shared__ double s_lvl[2];
  __shared__ float s_lam[128];
  __shared__ float s_delta[128];
  __shared__ double s_rho[128];
  __shared__ float s_ref;
  __shared__ __align__(8) uint64_t s_barP;
  __shared__ __align__(8) uint64_t s_barM;
  __shared__ uint32_t s_tmem;
  __shared__ __align__(16) AssetDev s_as;
  Smem sm;
  sm.Es = smem + p.sm_E;
  sm.EC = reinterpret_cast<float2*>(smem + p.sm_C);
  sm.Vs = smem + p.sm_V;
  sm.Ps = smem + p.sm_P;
  sm.Xs = smem + p.sm_X;
  sm.Ah = smem + p.sm_A;
  sm.Al = smem + p.sm_A2;
  sm.lvl = s_lvl;
  sm.lam = s_lam;
  sm.delta = s_delta;
  sm.rho = s_rho;
  sm.ref = &s_ref;
  sm.abort = &s_abort;
  sm.barP = &s_barP;
  sm.barM = &s_barM;
  if (threadIdx.x == 0) {
    s_abort = 0;
    mbar_init(&s_barP);
    mbar_init(&s_barM);
  }
  // tensor memory for the EV accumulator: allocated by warp 0 for the whole
  // launch, freed on every way out
  if (p.tmem_cols > 0 && threadIdx.x < 32) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     smem_u32(&s_tmem)),
                 "r"(p.tmem_cols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  tc_before_sync();
  __syncthreads();
  tc_after_sync();
  sm.tmem = p.tmem_cols > 0 ? s_tmem : 0u;
  sweep_run<R, KH>(p, sm, s_as);
  tc_before_sync();
  __syncthreads();
  if (p.tmem_cols > 0 && threadIdx.x < 32) {
    tc_after_sync();
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(sm.tmem),
                 "r"(p.tmem_cols)
                 : "memory");
  }
}

// Instance preparation, per asset of a launch: rho_t[k] = sum_k2 P_t[k][k2]
// in double, and ptrans[t][k2][k] = P_t[k][k2] with rows padded to
// p_stride(K) (zeros), written in output order.
__global__ void rowsum_kernel(const AssetDev* assets, const float* trans) {
  const AssetDev& as = assets[blockIdx.y];
  const int K = as.K, Kpt = p_stride(K);
  const long long rows = (long long)as.T * K;
  const float* P = trans + as.off_trans;
  const long long stride = (long long)gridDim.x * blockDim.x;
  const long long first = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  for (long long r = first; r < rows; r += stride) {
    double acc = 0.0;
    for (int k2 = 0; k2 < K; ++k2) acc += (double)__ldg(P + r * K + k2);
    as.rho[r] = acc;
  }
  if (as.ptrans && as.tc) {
    // [T][hi, lo][K*K]: B(k, k2) = P_t[k][k2] in the tcgen05 operand layout
    const long long KK = (long long)K * K, n = (long long)as.T * KK;
    for (long long i = first; i < n; i += stride) {
      const long long t = i / KK;
      const int kk = (int)(i - t * KK), k = kk / K, k2 = kk - k * K;
      uint32_t hi, lo;
      split_tf32(__ldg(P + i), hi, lo);
      float* base = as.ptrans + t * 2 * KK;
      base[tc_offset(k, k2, K, kCmB)] = __uint_as_float(hi);
      base[KK + tc_offset(k, k2, K, kCmB)] = __uint_as_float(lo);
    }
  } else if (as.ptrans) {
    const long long n = rows * Kpt;  // [T][K][Kpt]
    for (long long i = first; i < n; i += stride) {
      const long long tk2 = i / Kpt;
      const int k = (int)(i - tk2 * Kpt);
      const long long t = tk2 / K;
      const int k2 = (int)(tk2 - t * K);
      as.ptrans[i] = k < K ? __ldg(P + (t * K + k) * K + k2) : 0.f;
    }
  }
}

template <int R, int KH>
cudaError_t launch_R(const SweepShape& s, const SweepParams& p, cudaStream_t stream) {
  auto fn = sweep_kernel<R, KH>;
  cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)s.smem);
  if (e != cudaSuccess) return e;
  SweepParams pp = p;
  void* args[] = {&pp};
  return cudaLaunchCooperativeKernel((const void*)fn, dim3(s.grid), dim3(s.block), args, s.smem,
                                     stream);
}

template <int R, int KH>
int max_blocks_R(int block, size_t smem) {
  auto fn = sweep_kernel<R, KH>;
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
  // enough threads for the prepared copy (about 32 elements per row), not
  // only for the row sums: its loads are then in flight together
  const int block = 128;
  const long long elems = (long long)max_rows * 32;
  const int gx = (int)std::max(1LL, std::min(2048LL, (elems + block - 1) / block));
  rowsum_kernel<<<dim3(gx, n_assets), block, 0, stream>>>(d_assets, trans);
  return cudaGetLastError();
}

cudaError_t launch_sweep(const SweepShape& s, const SweepParams& p, cudaStream_t stream) {
  if (s.kh == 32) {
    switch (s.R) {
      case 4: return launch_R<4, 32>(s, p, stream);
      case 6: return launch_R<6, 32>(s, p, stream);
      case 8: return launch_R<8, 32>(s, p, stream);
      case 9: return launch_R<9, 32>(s, p, stream);
      case 10: return launch_R<10, 32>(s, p, stream);
      case 12: return launch_R<12, 32>(s, p, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  if (s.kh == -1) {
    switch (s.R) {
      case 4: return launch_R<4, -1>(s, p, stream);
      case 6: return launch_R<6, -1>(s, p, stream);
      case 8: return launch_R<8, -1>(s, p, stream);
      case 9: return launch_R<9, -1>(s, p, stream);
      case 10: return launch_R<10, -1>(s, p, stream);
      case 12: return launch_R<12, -1>(s, p, stream);
      default: return cudaErrorInvalidValue;
    }
  }
  if (s.kh != 0) return cudaErrorInvalidValue;
  switch (s.R) {
    case 4: return launch_R<4, 0>(s, p, stream);
    case 6: return launch_R<6, 0>(s, p, stream);
    case 8: return launch_R<8, 0>(s, p, stream);
    case 9: return launch_R<9, 0>(s, p, stream);
    case 10: return launch_R<10, 0>(s, p, stream);
    case 12: return launch_R<12, 0>(s, p, stream);
    default: return cudaErrorInvalidValue;
  }
}

int sweep_max_blocks_per_sm(int R, int kh, int block, size_t smem) {
  if (kh == 32) {
    switch (R) {
      case 4: return max_blocks_R<4, 32>(block, smem);
      case 6: return max_blocks_R<6, 32>(block, smem);
      case 8: return max_blocks_R<8, 32>(block, smem);
      case 9: return max_blocks_R<9, 32>(block, smem);
      case 10: return max_blocks_R<10, 32>(block, smem);
      case 12: return max_blocks_R<12, 32>(block, smem);
      default: return 0;
    }
  }
  if (kh == -1) {
    switch (R) {
      case 4: return max_blocks_R<4, -1>(block, smem);
      case 6: return max_blocks_R<6, -1>(block, smem);
      case 8: return max_blocks_R<8, -1>(block, smem);
      case 9: return max_blocks_R<9, -1>(block, smem);
      case 10: return max_blocks_R<10, -1>(block, smem);
      case 12: return max_blocks_R<12, -1>(block, smem);
      default: return 0;
    }
  }
  switch (R) {
    case 4: return max_blocks_R<4, 0>(block, smem);
    case 6: return max_blocks_R<6, 0>(block, smem);
    case 8: return max_blocks_R<8, 0>(block, smem);
    case 9: return max_blocks_R<9, 0>(block, smem);
    case 10: return max_blocks_R<10, 0>(block, smem);
    case 12: return max_blocks_R<12, 0>(block, smem);
    default: return 0;
  }
}

}  // namespace esdp
