// Occupancy adjoint of the storage DP.
//
// J = sum_k mu0[k] V_1[0][s0][k] depends on the prices, the transition
// matrices and the efficiencies only through the payoffs and expectations of
// eq. 5-6.  Away from ties of the maximisation (envelope theorem) its
// derivatives are expectations under the state-occupancy distribution of the
// stored argmax policy:
//   rho_1[0][s0][k]        = mu0[k]
//   post_t[m'][s+d][k]    += rho_t[m][s][k]      (d, m' of the stored action)
//   rho_{t+1}[m][s][k2]    = sum_k post_t[m][s][k] P_t[k][k2]
//   dJ/dprice[t][k]        = sum_{m,s} rho_t[m][s][k] e_a
//   dJ/dP_t[k][k2]         = sum_{m,s} post_t[m][s][k] V_{t+1}[m][s][k2]
//   dJ/deta_c              = sum rho_t price[t][k] d delta / eta_c^2   (d > 0)
//   dJ/deta_d              = sum rho_t price[t][k] (-d) delta           (d < 0)
//   dJ/dcost[a]            = -sum_t sum rho_t [a_t = a]
//   dJ/dswitch             = -sum rho_t [m = 1, d < 0]                  (two modes)
//   dJ/dterminal           = rho_{T+1}, dJ/dmu0[k] = V_1[0][s0][k]  (taken by the host)
// occ_kernel runs the forward pass over a segment of stages in one
// cooperative launch (per stage, between the scatter and the contraction, a
// CTA waits only for the CTAs whose rows can scatter into its own: release
// flags and bounded acquire polls); dtrans_kernel then forms dJ/dP for the segment from
// the stored post-decision occupancies and values (a split-row reduction per
// stage and 32 x 32 output tile).
//
// The scatter adds with atomics, in 64-bit fixed point: integer addition is
// associative, so the sums do not depend on the order in which threads and
// CTAs arrive, and every other sum runs in a fixed order, so the gradients
// are the same bit for bit on every call.  Occupancy mass is counted in
// units of 2^-32 (entries up to 2^20 are accepted, sums must stay below
// 2^31), the rho * e_a terms of dJ/dprice in units chosen from the largest
// |e_a| so that they have the same range.
#include <cuda_runtime.h>

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

// This CTA's scatter of stage `epoch` is complete: its atomics on the
// post-decision occupancy are ordered before the flag by the CTA barrier and
// one release store at GPU scope (cumulative over what the barrier ordered
// before it; a separate fence ahead of the release cost 0.6 us per stage).
// The last warp releases: the first warp, whose threads poll the sources,
// is then not held up by the release's wait for the CTA's writes.
__device__ __forceinline__ void publish_stage(int* flags, int epoch) {
  __syncthreads();
  if (threadIdx.x == blockDim.x - 32) st_release(flags + blockIdx.x, epoch);
}

// Wait until every CTA that can scatter into this CTA's rows [r0, r1) has
// published stage `epoch`.  A target (m', s') receives from (m, s) with
// s' - D_chg <= s <= s' + D_dis in every mode m, so the sources are the CTAs
// covering rows m N + [lo, hi] of each mode.  Each thread polls a share of
// them with acquire loads, bounded by the timeout (status ESDP_ETIMEOUT).
__device__ bool wait_sources(const OccParams& p, int r0, int r1, int epoch, int* s_abort) {
  const int N = p.N, gr = p.grid_rows, D_chg = p.A - 1 - p.D_dis;
  const int m0 = r0 / N, m1 = (r1 - 1) / N;
  int s_lo = 0, s_hi = N - 1;  // the rows' SoC range (all of it across a mode boundary)
  if (m0 == m1) {
    s_lo = r0 - m0 * N;
    s_hi = r1 - 1 - m0 * N;
  }
  const int lo = max(0, s_lo - D_chg), hi = min(N - 1, s_hi + p.D_dis);
  // CTA range [c0_m, c1_m] of each mode's rows m N + [lo, hi]
  int total = 0;
  for (int m = 0; m < p.M; ++m) total += (m * N + hi) / gr - (m * N + lo) / gr + 1;
  for (int q = threadIdx.x; q < total; q += blockDim.x) {
    int rem = q, cta = 0;
    for (int m = 0; m < p.M; ++m) {
      const int c0 = (m * N + lo) / gr, c1 = (m * N + hi) / gr;
      if (rem <= c1 - c0) {
        cta = c0 + rem;
        break;
      }
      rem -= c1 - c0 + 1;
    }
    const unsigned long long t0 = now_ns();
    int polls = 0;
    while (ld_acquire(p.flags + cta) < epoch) {
      if ((++polls & 15) == 0) {
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
  __syncthreads();
  return *(volatile int*)s_abort == 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

constexpr float kFxRho = 4294967296.f;  // 2^32 units per unit of occupancy mass
constexpr double kFxRhoInv = 1.0 / 4294967296.0;
constexpr float kFxRhoInvF = 1.0f / 4294967296.0f;
constexpr int kPre = 4;  // entries per thread whose actions are loaded a stage ahead
constexpr float kFxMaxRho = 1048576.f;  // 2^20: larger entries are reported

__device__ __forceinline__ unsigned long long to_fx(float x, float scale) {
  return (unsigned long long)__float2ll_rn(x * scale);  // scale: a power of two
}

__global__ void __launch_bounds__(256) occ_kernel(const OccParams p) {
  // float32 per-state terms (few terms each: this part's FP64 pipe is 64x
  // slower than FP32), fixed-point shared sums, double from the warp sums on
  extern __shared__ double osm[];
  double* sacc = osm;                                       // [8] segment accumulators
  double* wacc = osm + 8;                                   // [8 warps][3] warp segment sums
  unsigned long long* skx = reinterpret_cast<unsigned long long*>(osm + 32);  // [K] dprice
  // [n_cc][A] cost partials of the segment: thread tid adds into copy
  // tid % n_cc, so that the many states that take the same action (full
  // charge, idle, full discharge) do not all hit one shared address
  unsigned long long* scx = skx + p.K;
  const int n_cc = p.n_cost_copies;
  float* Ps0 = reinterpret_cast<float*>(scx + (size_t)n_cc * p.A);  // [2][K][K]: P_t, P_{t+1}
  float* spost = Ps0 + 2 * p.K * p.K;  // [grid_rows][K] own converted rows (if own_smem)
  float* srho = spost + p.grid_rows * p.K;  // [grid_rows][K] own occupancy rows (if own_smem)
  __shared__ int s_abort;
  const int K = p.K, N = p.N, M = p.M, MN = M * N;
  const size_t MNK = (size_t)MN * K;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int r0 = blockIdx.x * p.grid_rows;
  const int r1 = min(MN, r0 + p.grid_rows);
  // d rho lam delta / eta_c^2 per charging step, d rho lam delta per discharging step
  const float coef_c = (float)(p.delta / (p.eta_c * p.eta_c)), coef_d = (float)p.delta;
  // own occupancy rows: in shared memory for the whole segment when they
  // fit (the scatter reads and the contraction writes only these rows)
  float* rho = p.own_smem ? srho - r0 * K : p.rho;
  if (tid == 0) s_abort = 0;
  for (int a = tid; a < n_cc * p.A; a += nth) scx[a] = 0ull;
  if (tid < 8) sacc[tid] = 0.0;  // summed over the segment
  for (int i = tid; i < p.K; i += nth) skx[i] = 0ull;
  if (p.own_smem)
    for (int i = r0 * K + tid; i < r1 * K; i += nth) srho[i - r0 * K] = p.rho[i];
  {  // P of the first stage; every later P_{t+1} is copied during stage t
    const float* P = p.trans + (size_t)(p.t_lo - 1) * K * K;
    for (int i = tid; i < K * K; i += nth) Ps0[i] = P[i];
  }
  __syncthreads();
  int epoch = 0;
  // lane 0 of each warp: the warp's segment sums and their compensations
  float wsum[3] = {0.f, 0.f, 0.f}, wcmp[3] = {0.f, 0.f, 0.f};
  // the stored actions of a thread's first kPre entries are loaded one stage
  // ahead, so that the scatter waits on no global load
  const int e0 = r0 * K + tid, e1 = r1 * K;
  auto action_at = [&](int ts_, int i) -> int {
    const size_t pi = (size_t)ts_ * MNK + i;
    return p.policy_bytes == 2 ? (int)__ldcg(reinterpret_cast<const short*>(p.policy) + pi)
                               : __ldcg(reinterpret_cast<const int*>(p.policy) + pi);
  };
  int apre[kPre];
#pragma unroll
  for (int j = 0; j < kPre; ++j) apre[j] = e0 + j * nth < e1 ? action_at(0, e0 + j * nth) : 0;
  for (int t = p.t_lo; t <= p.t_hi; ++t) {
    const int ts = t - p.t_lo;
    float* Ps = Ps0 + (ts & 1) * K * K;
    float* post = p.post + (size_t)ts * MNK;
    unsigned long long* post_fx = p.post_fx + (size_t)ts * MNK;
    unsigned long long* scx_t = scx + (size_t)(tid % n_cc) * p.A;
    const float* price_t = p.price + (size_t)(t - 1) * K;
    float dc = 0.f, dd = 0.f, dsw = 0.f;
    auto scatter = [&](int i, int a) {
      const float rv = rho[i];
      if (rv == 0.f) return;
      const int row = i / K, k = i - row * K;
      const int m = row / N, s = row - m * N;
      const int d = a - p.D_dis;
      if (a < 0 || a >= p.A || s + d < 0 || s + d >= N ||  // not a feasible stored action,
          !(fabsf(rv) <= kFxMaxRho)) {                      // or outside the fixed-point range
        atomicCAS(p.status, 0, ESDP_ENUMERIC);
        return;
      }
      const int m2 = (M == 2) ? (d < 0 ? 0 : (d > 0 ? 1 : m)) : 0;
      atomicAdd(post_fx + ((size_t)m2 * N + s + d) * K + k, to_fx(rv, kFxRho));
      const float lam = price_t[k];
      atomicAdd(&skx[k], to_fx(rv * p.e[a], p.fx_e));
      if (d > 0) dc = fmaf(rv * lam, (float)d * coef_c, dc);
      if (d < 0) dd = fmaf(rv * lam, (float)(-d) * coef_d, dd);
      atomicAdd(&scx_t[a], to_fx(-rv, kFxRho));
      if (M == 2 && m == 1 && d < 0) dsw -= rv;
    };
#pragma unroll
    for (int j = 0; j < kPre; ++j)
      if (e0 + j * nth < e1) scatter(e0 + j * nth, apre[j]);
    for (int i = e0 + kPre * nth; i < e1; i += nth) scatter(i, action_at(ts, i));
    // the scatter is complete once every thread is past the barrier of the
    // release; the stage's partial sums are formed after it, while the
    // sources are awaited
    ++epoch;
    publish_stage(p.flags, epoch);
    if (t < p.t_hi) {
      // P_{t+1} into the other buffer (its last reader, the contraction of
      // stage t - 1, is behind the barrier), waited for at the end of the stage
      const float* P = p.trans + (size_t)t * K * K;
      float* Pn = Ps0 + ((ts + 1) & 1) * K * K;
      for (int i = tid; i < K * K; i += nth)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(
                         (uint32_t)__cvta_generic_to_shared(Pn + i)),
                     "l"(P + i)
                     : "memory");
#pragma unroll
      for (int j = 0; j < kPre; ++j)
        if (e0 + j * nth < e1) apre[j] = action_at(ts + 1, e0 + j * nth);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dc += __shfl_xor_sync(0xffffffffu, dc, o);
      dd += __shfl_xor_sync(0xffffffffu, dd, o);
      dsw += __shfl_xor_sync(0xffffffffu, dsw, o);
    }
    if ((tid & 31) == 0) {  // the warp's segment sums: compensated float32, in stage order
      const float x[3] = {dc, dd, dsw};
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        const float y = x[q] - wcmp[q];
        const float u = wsum[q] + y;
        wcmp[q] = (u - wsum[q]) - y;
        wsum[q] = u;
      }
    }
    // this CTA's partials of the stage (and, once, of the segment's costs):
    // plain stores, added up after the launch in a fixed order; a K sum is
    // cleared by the thread that read it, before the next stage's scatter
    long long* pr = p.part + ((size_t)ts * gridDim.x + blockIdx.x) * K;
    for (int i = tid; i < K; i += nth) {
      pr[i] = (long long)skx[i];  // fixed point: turned into double by the reduction
      skx[i] = 0ull;
    }
    if (t == p.t_hi)
      for (int a = tid; a < p.A; a += nth) {
        unsigned long long sum = 0ull;  // the copies in order (integer: exact)
        for (int q = 0; q < n_cc; ++q) sum += scx[(size_t)q * p.A + a];
        p.part_cost[(size_t)blockIdx.x * p.A + a] = (double)(long long)sum * kFxRhoInv;
      }
    if (!wait_sources(p, r0, r1, epoch, &s_abort)) {
      asm volatile("cp.async.wait_all;" ::: "memory");  // no copy outlives the CTA
      return;
    }
    if (p.own_smem && K == 32 && (nth & 31) == 0) {
      // K = 32: a warp's entries of one pass are the 32 states of one row,
      // so each lane keeps its converted entry in a register and the row's
      // terms reach the other lanes by shuffles (no shared copy, no barrier);
      // each output is still summed in ascending k with one fma per term
      for (int i = e0; i < e1; i += nth) {
        const float v = __ll2float_rn((long long)__ldcg(post_fx + i)) * kFxRhoInvF;
        post[i] = v;
        const int k2 = i & 31;
        float acc = 0.f;
#pragma unroll 8
        for (int k = 0; k < 32; ++k) acc = fmaf(__shfl_sync(0xffffffffu, v, k), Ps[k * 32 + k2], acc);
        rho[i] = acc;
        if (t == p.t_hi) p.rho[i] = acc;  // the next segment starts from it
      }
    } else {
      // own rows of the post-decision occupancy, complete: fixed point to
      // float, for dJ/dP and (in shared memory when they fit) the contraction
      for (int i = e0; i < e1; i += nth) {
        // one rounding of the integer to float32, then an exact scaling by
        // 2^-32: the same value as through double, without this part's slow
        // FP64 pipe
        const float v = __ll2float_rn((long long)__ldcg(post_fx + i)) * kFxRhoInvF;
        post[i] = v;
        if (p.own_smem) spost[i - r0 * K] = v;
      }
      __syncthreads();
      // contraction of the post-decision occupancy with P_t (own rows); entry
      // i of rho is written here and read by the next scatter in the same
      // thread, and every other shared buffer of the next stage is reused only
      // behind its release barrier, so no barrier closes the stage
      for (int i = e0; i < e1; i += nth) {
        const int row = i / K, k2 = i - row * K;
        float acc = 0.f;
        if (p.own_smem) {
          // in ascending k, one fma per term; the loads of eight terms are
          // issued ahead of their fmas
          const float* prw = spost + (size_t)(row - r0) * K;
          int k = 0;
          for (; k + 8 <= K; k += 8) {
            float a8[8], b8[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              a8[j] = prw[k + j];
              b8[j] = Ps[(k + j) * K + k2];
            }
#pragma unroll
            for (int j = 0; j < 8; ++j) acc = fmaf(a8[j], b8[j], acc);
          }
          for (; k < K; ++k) acc = fmaf(prw[k], Ps[k * K + k2], acc);
        } else {
          const float* prw = post + (size_t)row * K;
          for (int k = 0; k < K; ++k) acc = fmaf(__ldcg(prw + k), Ps[k * K + k2], acc);
        }
        rho[i] = acc;
        if (p.own_smem && t == p.t_hi) p.rho[i] = acc;  // the next segment starts from it
      }
    }
    asm volatile("cp.async.wait_all;" ::: "memory");  // this thread's part of P_{t+1}
  }
  // the segment accumulators: the warps' sums added in warp order in double
  // (this part's FP64 pipe is slow: once per segment, off the stages' path)
  if ((tid & 31) == 0)
    for (int q = 0; q < 3; ++q) wacc[(tid >> 5) * 3 + q] = (double)wsum[q] - (double)wcmp[q];
  __syncthreads();
  if (tid == 0) {
    for (int wq = 0; wq < (nth >> 5); ++wq) {
      sacc[0] += wacc[wq * 3 + 0];
      sacc[1] += wacc[wq * 3 + 1];
      sacc[4] += wacc[wq * 3 + 2];
    }
    for (int q = 0; q < 8; ++q) p.part_acc[(size_t)blockIdx.x * 8 + q] = sacc[q];
  }
}

// dJ/dP_t = post_t^T V_{t+1} over all rows (m, s): one block per (stage,
// 32 x 32 tile of (k, k2), range of rows; n_split ranges).  The block stages
// its rows through shared memory 64 at a time (16-byte cp.async copies into
// a double buffer when K is a multiple of 4, so the next rows land while
// these are used); its 256 threads are four groups of 64, group g takes the
// rows g, g + 4, ... of each chunk, and thread (i, j) of a group keeps the
// 4 x 4 sums of k = kb + 4i.., k2 = k2b + 4j.. in registers (per row: two
// 16-byte shared reads, 16 fmas; the threads with j = 0 also sum the
// occupancy mass of their k).  The four groups' sums are added in double in
// group order; dtrans_finish_kernel adds the ranges in order plus c_{t+1}
// times the occupancy mass of k (V_{t+1} = V'_{t+1} + c_{t+1}).
constexpr int kDtRows = 64;  // rows per shared chunk
__device__ __forceinline__ void cp_async16(float* dst, const float* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(
                   (uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}
__global__ void __launch_bounds__(256) dtrans_kernel(const DTransParams p) {
  // [2][64][32] post rows (columns kb..kb+31), then [2][64][32] V' rows
  // (columns k2b..k2b+31); after the rows, the groups' sums [4][32][33]
  __shared__ __align__(16) float sbuf[4 * kDtRows * 32];
  __shared__ float sM[4][32];  // the groups' masses
  auto sP = [&](int b, int r, int c) -> float* { return sbuf + (b * kDtRows + r) * 32 + c; };
  auto sV = [&](int b, int r, int c) -> float* { return sbuf + ((2 + b) * kDtRows + r) * 32 + c; };
  auto sR = [&](int g, int j, int l) -> float& { return sbuf[(g * 32 + j) * 33 + l]; };
  const int K = p.K, MN = p.MN;
  const int tiles = (K + 31) / 32;
  const int ts = blockIdx.y, ty = blockIdx.x / tiles, tx = blockIdx.x % tiles;
  const int part = blockIdx.z;
  const int row0 = (int)((long long)MN * part / p.n_split);
  const int row1 = (int)((long long)MN * (part + 1) / p.n_split);
  const int kb = 32 * ty, k2b = 32 * tx;
  const int tid = threadIdx.x, grp = tid >> 6, lt = tid & 63;
  const int mi = (lt >> 3) * 4, ni = (lt & 7) * 4;
  const float* post = p.post + (size_t)ts * MN * K;
  const float* v = p.vnext + (size_t)(ts / p.seg_len) * p.seg_stride +
                   (size_t)(ts % p.seg_len) * MN * K;
  const bool vec = (K & 3) == 0;
  // chunk c of the range into buffer b: 64 rows x 32 columns of each array,
  // zeros outside the range and beyond K
  auto load_chunk = [&](int c, int b) {
    const int rbase = row0 + c * kDtRows;
    for (int q = tid; q < 2 * kDtRows * 8; q += 256) {
      const int arr = q >= kDtRows * 8, qq = q - arr * kDtRows * 8;
      const int r = qq >> 3, c4 = (qq & 7) * 4;
      const int row = rbase + r, col = (arr ? k2b : kb) + c4;
      float* dst = arr ? sV(b, r, c4) : sP(b, r, c4);
      const float* src = (arr ? v : post) + (size_t)row * K + col;
      if (vec && row < row1 && col + 4 <= K) {
        cp_async16(dst, src);
      } else {
#pragma unroll
        for (int e = 0; e < 4; ++e) dst[e] = (row < row1 && col + e < K) ? __ldg(src + e) : 0.f;
      }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
  };
  float acc[4][4], mass[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    mass[i] = 0.f;
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
  }
  const int nchunk = (row1 - row0 + kDtRows - 1) / kDtRows;
  if (nchunk > 0) load_chunk(0, 0);
  for (int c = 0; c < nchunk; ++c) {
    const int b = c & 1;
    if (c + 1 < nchunk) {
      load_chunk(c + 1, b ^ 1);  // its buffer was last read before the barrier below
      asm volatile("cp.async.wait_group 1;" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;" ::: "memory");
    }
    __syncthreads();
#pragma unroll 4
    for (int r = grp; r < kDtRows; r += 4) {
      const float4 a = *reinterpret_cast<const float4*>(sP(b, r, mi));
      const float4 x = *reinterpret_cast<const float4*>(sV(b, r, ni));
      const float av[4] = {a.x, a.y, a.z, a.w}, xv[4] = {x.x, x.y, x.z, x.w};
#pragma unroll
      for (int i = 0; i < 4; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(av[i], xv[j], acc[i][j]);
      }
      if (ni == 0) {
#pragma unroll
        for (int i = 0; i < 4; ++i) mass[i] += av[i];
      }
    }
    __syncthreads();  // buffer b is refilled two chunks on (and sR overlays the rows)
  }
#pragma unroll
  for (int i = 0; i < 4; ++i) {
#pragma unroll
    for (int j = 0; j < 4; ++j) sR(grp, mi + i, ni + j) = acc[i][j];
    if (ni == 0) sM[grp][mi + i] = mass[i];
  }
  __syncthreads();
  // this block's partial: [ts][part][k][k2] sums and [ts][part][k] masses
  double* ps = p.part + ((size_t)ts * p.n_split + part) * K * K;
  double* pm = p.part_mass + ((size_t)ts * p.n_split + part) * K;
  for (int e = tid; e < 32 * 32; e += 256) {
    const int j = e >> 5, l = e & 31;
    const int k = kb + j, kk2 = k2b + l;
    if (k >= K || kk2 >= K) continue;
    double sv = 0.0;
#pragma unroll
    for (int q = 0; q < 4; ++q) sv += (double)sR(q, j, l);
    ps[(size_t)k * K + kk2] = sv;
    if (tx == 0 && l == 0) {
      double sm = 0.0;
#pragma unroll
      for (int q = 0; q < 4; ++q) sm += (double)sM[q][j];
      pm[k] = sm;
    }
  }
}

// dJ/dP_t[k][k2] = sum of the row ranges in order + c_{t+1} mass_t[k]
__global__ void dtrans_finish_kernel(const DTransParams p) {
  const int K = p.K;
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i >= (long long)p.n_t * K * K) return;
  const int ts = (int)(i / ((long long)K * K));
  const int e = (int)(i - (long long)ts * K * K), k = e / K;
  double sv = 0.0, sm = 0.0;
  for (int q = 0; q < p.n_split; ++q) {
    sv += p.part[((size_t)ts * p.n_split + q) * K * K + e];
    sm += p.part_mass[((size_t)ts * p.n_split + q) * K + k];
  }
  p.d_trans[(size_t)ts * K * K + e] = (float)(sv + p.cnext[ts] * sm);
}

// Per-CTA partials of one segment into the accumulated gradients, one warp
// per output: (stage, state) -> d_price, the five accumulators, actions ->
// d_cost.  Lane l adds the partials l, l + 32, ... in order, then a fixed
// butterfly over the lanes: the same sum on every run.
__global__ void occ_reduce_kernel(const OccParams p, int grid) {
  const int K = p.K, n_t = p.t_hi - p.t_lo + 1;
  const int o = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  const int n_price = n_t * K;
  if (o >= n_price + 5 + p.A) return;  // whole warps
  double s = 0.0;
  if (o < n_price) {
    const int ts = o / K, k = o - ts * K;
    const double inv_fx_e = 1.0 / (double)p.fx_e;  // a power of two: exact
    for (int b = lane; b < grid; b += 32)
      s += (double)p.part[((size_t)ts * grid + b) * K + k] * inv_fx_e;
  } else if (o < n_price + 5) {
    const int q = o - n_price;
    for (int b = lane; b < grid; b += 32) s += p.part_acc[(size_t)b * 8 + q];
  } else {
    const int a = o - n_price - 5;
    for (int b = lane; b < grid; b += 32) s += p.part_cost[(size_t)b * p.A + a];
  }
  s = warp_sum(s);
  if (lane == 0) {
    if (o < n_price)
      p.d_price[(size_t)(p.t_lo - 1 + o / K) * K + o % K] += s;
    else if (o < n_price + 5)
      p.acc[o - n_price] += s;
    else
      p.d_cost[o - n_price - 5] += s;
  }
}

}  // namespace

cudaError_t launch_occ_reduce(const OccParams& p, int grid, cudaStream_t stream) {
  const int n = (p.t_hi - p.t_lo + 1) * p.K + 5 + p.A;  // outputs, one warp each
  occ_reduce_kernel<<<(n + 7) / 8, 256, 0, stream>>>(p, grid);
  return cudaGetLastError();
}

cudaError_t launch_occupancy(const OccParams& p, int grid, int block, cudaStream_t stream) {
  // segment sums, 8 warps x 3 stage sums, fixed-point K sums and copies of
  // the A cost sums, P_t and P_{t+1}, and (when they fit) the own converted
  // rows and the own occupancy rows
  OccParams pp = p;
  pp.n_cost_copies = (int)std::max<long long>(1, std::min<long long>(8, 16384 / std::max(1, p.A)));
  const size_t base = 32 * sizeof(double) +
                      ((size_t)p.K + (size_t)pp.n_cost_copies * p.A) * sizeof(unsigned long long) +
                      2 * (size_t)p.K * p.K * sizeof(float);
  const size_t own = 2 * (size_t)p.grid_rows * p.K * sizeof(float);
  pp.own_smem = base + own <= 160 * 1024 ? 1 : 0;
  const size_t smem = base + (pp.own_smem ? own : 0);
  cudaError_t e = cudaFuncSetAttribute(occ_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  void* args[] = {&pp};
  return cudaLaunchCooperativeKernel((const void*)occ_kernel, dim3(grid), dim3(block), args, smem,
                                     stream);
}

cudaError_t launch_dtrans(const DTransParams& p, cudaStream_t stream) {
  if (p.n_t == 0) return cudaSuccess;
  const int tiles = (p.K + 31) / 32;
  dtrans_kernel<<<dim3(tiles * tiles, p.n_t, p.n_split), 256, 0, stream>>>(p);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  const long long n = (long long)p.n_t * p.K * p.K;
  dtrans_finish_kernel<<<(unsigned)((n + 255) / 256), 256, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace esdp
