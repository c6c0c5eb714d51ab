// Stagewise-independent prices on the paper's own action grid (Sec. III-A,
// Algorithm 1, eq. 2 and 13):
//   V_{t-1}(s) = sum_k pi_t[k] max_a ( lam_t[k] p_a tau + V_t(sigma(s, a)) )
// with R price samples (lam_t[k], pi_t[k]) per stage, the power actions p_a of
// eq. 13 (grid steps delta*eta / delta/eta and the two end points -p_max,
// +p_max), next state sigma = s delta + F(p_a) tau (F = -p/eta discharging,
// -eta p charging), linear interpolation of V_t between the two neighbouring
// grid points when sigma is off the grid, and -inf outside [0, s_max].
//
// In the Markov form of the main sweep this is the rank-1 transition
// P_t[k][k2] = pi_{t+1}[k2]: the next-stage value is one vector over SoC for
// every price sample, so a stage needs no K x K contraction, only one
// weighted sum over the samples per SoC point.  This kernel exploits that:
// a tile of SoC rows stages a single column of V_t (its rows plus the action
// halo), forms the feasible, interpolated next values once per (row, action),
// and every price sample of the row reuses them; a thread owns one row and
// KG samples (6, 8 or 10: the least work per thread for the tile's rows,
// passes of the block x samples) and runs the max over all actions for them.
//
// Persistent cooperative launch over all stages; tiles synchronise with their
// neighbours only (release/acquire flags, bounded waits) as in the main sweep.
// Values are kept as V'_t = V_t - c_t in float32 with the scalar level c_t in
// double (every stage re-centres on a reference row).
#include <cuda_runtime.h>
#include <math_constants.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <vector>

#include "../../include/esdp.h"
#include "esdp_internal.h"

namespace esdp {
namespace {

constexpr int kIidBlock = 512;
constexpr int kIidKG = 8;  // price samples per thread (the smaller choice)
constexpr size_t kIidSmemLimit = 227 * 1024;

struct IidParams {
  int T, S, R, P, W, n_tiles, reach, groups;
  int dmin, span;            // halo rows of a tile: [s0 + dmin, s0 + dmin + span)
  int ref_tile, ref_row;
  const float* lam;          // [T][R]
  const float* pi;           // [T][R]
  const double* rho;         // [T] sum_k pi_t[k]
  const float* pay;          // [P] p_a * tau
  const int* dlo;            // [P] floor of the SoC shift in grid steps
  const float* bw;           // [P] weight of grid point dlo + 1 (0: on the grid)
  const int* smin;           // [P] feasible rows s of action a: smin[a] <= s <= smax[a]
  const int* smax;
  const float* terminal;     // [S] V_T, or nullptr for 0
  float* v;                  // [2][S] V'_t, t even / odd
  float* ref_hist;           // [T+1] V'_t[ref_row]
  int* flags;                // [n_tiles], zero at launch
  int* status;
  int* pol32;                // [T][S][R] argmax (action index) or nullptr
  short* pol16;
  float* v_out;              // [S] V_0
  float* v_all;              // [T+1][S] V_t of every stage, or nullptr
  const int* cta_first;      // [grid+1] contiguous tile ranges
  unsigned long long timeout_ns;
};

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

__device__ __forceinline__ unsigned long long pack2(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}

// a * b + c per lane of a float pair (two round-to-nearest FMAs)
__device__ __forceinline__ float2 fma2u(unsigned long long a, unsigned long long b,
                                        unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  float2 f;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(f.x), "=f"(f.y) : "l"(r));
  return f;
}

__device__ __forceinline__ float max3f(float a, float b, float c) {
  float r;
  asm("max.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
  return r;
}

// Release the tile's values: the barrier orders every thread's stores before
// thread 0's release store (cumulativity), consumers read after an acquire.
__device__ __forceinline__ void publish(int* flag, int v) {
  __syncthreads();
  if (threadIdx.x == 0) st_release(flag, v);
}

// Wait until the neighbour tiles within `reach` and the reference tile have
// published at least `need` stages; the thread that waits for the reference
// tile reads V'_t[ref].  Bounded: ESDP_ETIMEOUT in the status word and false.
__device__ bool iid_wait(const IidParams& p, int tile, int need, int t, float* s_ref,
                         int* s_abort) {
  const int lo = max(0, tile - p.reach), hi = min(p.n_tiles - 1, tile + p.reach);
  const int n = hi - lo + 1;
  if ((int)threadIdx.x <= n) {
    const int* f = p.flags + ((int)threadIdx.x < n ? lo + (int)threadIdx.x : p.ref_tile);
    if (ld_acquire(f) < need) {
      const unsigned long long t0 = now_ns();
      for (unsigned it = 1;; ++it) {
        if (ld_acquire(f) >= need) break;
        if ((it & 15u) == 0) {
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
    if ((int)threadIdx.x == n) *s_ref = __ldcg(p.ref_hist + t);
  }
  __syncthreads();
  return *(volatile int*)s_abort == 0;
}

template <bool kPol, int KG>
__global__ void __launch_bounds__(kIidBlock, 1) iid_kernel(const IidParams p) {
  extern __shared__ float4 ism4[];
  float* ism = reinterpret_cast<float*>(ism4);
  auto al = [](int x) { return (x + 31) & ~31; };
  const int Pp = (p.P + 3) & ~3;            // actions padded to a multiple of 4
  float* Vt = ism;                          // [span] halo column of V'_t - r_t
  float2* BP = reinterpret_cast<float2*>(Vt + al(p.span));  // [W][Pp] (next value, payoff)
  float* pay = reinterpret_cast<float*>(BP + (size_t)p.W * Pp);  // [P]
  float* red = pay + al(p.P);               // [W][groups] per-group expectations
  __shared__ float s_ref;
  __shared__ int s_abort;
  __shared__ double s_c;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int S = p.S, R = p.R, P = p.P, W = p.W, groups = p.groups;
  const int i0 = p.cta_first[blockIdx.x], i1 = p.cta_first[blockIdx.x + 1];
  const float NEG = -CUDART_INF_F;
  if (tid == 0) {
    s_abort = 0;
    s_c = 0.0;
  }
  for (int a = tid; a < P; a += nth) pay[a] = p.pay[a];
  __syncthreads();

  // prologue: V'_T = V_T (c_T = 0)
  for (int tile = i0; tile < i1; ++tile) {
    const int s0 = tile * W, s1 = min(S, s0 + W);
    for (int s = s0 + tid; s < s1; s += nth) {
      const float v = p.terminal ? __ldg(p.terminal + s) : 0.f;
      p.v[(size_t)(p.T & 1) * S + s] = v;
      if (p.v_all) p.v_all[(size_t)p.T * S + s] = v;
      if (s == p.ref_row) p.ref_hist[p.T] = v;
    }
    publish(p.flags + tile, 1);
  }

  const int rows_pass = nth / groups;  // rows of one pass of the max loop
  const int my_row = tid / groups, my_group = tid - my_row * groups;
  for (int g = 0; g < p.T; ++g) {
    const int t = p.T - g;  // V'_{t-1} from V'_t
    const float* vin = p.v + (size_t)(t & 1) * S;
    float* vout = p.v + (size_t)((t - 1) & 1) * S;
    const float* lam_t = p.lam + (size_t)(t - 1) * R;
    const float* pi_t = p.pi + (size_t)(t - 1) * R;
    for (int tile = i0; tile < i1; ++tile) {
      const int s0 = tile * W, s1 = min(S, s0 + W), Wt = s1 - s0;
      if (!iid_wait(p, tile, g + 1, t, &s_ref, &s_abort)) return;
      const float r = s_ref;
      if (tile == i0 && tid == 0) s_c = (s_c + (double)r) * p.rho[t - 1];  // c_{t-1}
      // 1. halo column of V'_t, re-centred on the reference row
      for (int i = tid; i < p.span; i += nth) {
        const int row = s0 + p.dmin + i;
        Vt[i] = (row >= 0 && row < S) ? __ldcg(vin + row) - r : 0.f;
      }
      __syncthreads();
      // 2. next value of every (row, action): on the grid, interpolated, or
      //    -inf when the next SoC leaves [0, s_max]
      for (int i = tid; i < Wt * Pp; i += nth) {
        const int rr = i / Pp, a = i - rr * Pp, s = s0 + rr;
        float b = NEG, pa = 0.f;  // padding actions: -inf
        if (a < P) {
          pa = pay[a];
          if (s >= __ldg(p.smin + a) && s <= __ldg(p.smax + a)) {
            const int j = s + __ldg(p.dlo + a) - (s0 + p.dmin);
            const float w = __ldg(p.bw + a);
            b = w == 0.f ? Vt[j] : fmaf(w, Vt[j + 1], (1.f - w) * Vt[j]);
          }
        }
        BP[rr * Pp + a] = make_float2(b, pa);
      }
      __syncthreads();
      // 3. max over the actions for KG price samples of one row; the
      //    smallest maximising action index (strict >)
      for (int rr = my_row; my_row < rows_pass && rr < Wt; rr += rows_pass) {
        const int k0 = my_group * KG;
        float lam[KG], best[KG];
        int arg[KG];
#pragma unroll
        for (int j = 0; j < KG; ++j) {
          lam[j] = k0 + j < R ? __ldg(lam_t + k0 + j) : 0.f;
          best[j] = NEG;
          arg[j] = -1;
        }
        const float2* Br = BP + rr * Pp;
        if constexpr (!kPol) {
          // four actions per step: two 16-byte reads of (next value, payoff);
          // each packed FMA forms two samples' candidates of one action (two
          // round-to-nearest FMAs, the same values as scalar fmaf)
          const float4* B4 = reinterpret_cast<const float4*>(Br);
          unsigned long long lam2[KG / 2];
#pragma unroll
          for (int j = 0; j < KG / 2; ++j) lam2[j] = pack2(lam[2 * j], lam[2 * j + 1]);
#pragma unroll 2
          for (int q = 0; q < (Pp >> 1); q += 2) {
            const float4 x = B4[q], y = B4[q + 1];
            const unsigned long long b0 = pack2(x.x, x.x), p0 = pack2(x.y, x.y);
            const unsigned long long b1 = pack2(x.z, x.z), p1 = pack2(x.w, x.w);
            const unsigned long long b2 = pack2(y.x, y.x), p2 = pack2(y.y, y.y);
            const unsigned long long b3 = pack2(y.z, y.z), p3 = pack2(y.w, y.w);
#pragma unroll
            for (int j = 0; j < KG / 2; ++j) {
              const float2 c0 = fma2u(lam2[j], p0, b0), c1 = fma2u(lam2[j], p1, b1);
              const float2 c2 = fma2u(lam2[j], p2, b2), c3 = fma2u(lam2[j], p3, b3);
              best[2 * j] = max3f(best[2 * j], c0.x, c1.x);
              best[2 * j + 1] = max3f(best[2 * j + 1], c0.y, c1.y);
              best[2 * j] = max3f(best[2 * j], c2.x, c3.x);
              best[2 * j + 1] = max3f(best[2 * j + 1], c2.y, c3.y);
            }
          }
        } else {
          // the same candidates two samples per packed FMA; the argmax with a
          // strict > over ascending actions (the smallest maximiser)
          unsigned long long lam2[KG / 2];
#pragma unroll
          for (int j = 0; j < KG / 2; ++j) lam2[j] = pack2(lam[2 * j], lam[2 * j + 1]);
          for (int a = 0; a < P; ++a) {
            const float2 bp = Br[a];
            const unsigned long long b2 = pack2(bp.x, bp.x), p2 = pack2(bp.y, bp.y);
#pragma unroll
            for (int j = 0; j < KG / 2; ++j) {
              const float2 c = fma2u(lam2[j], p2, b2);
              if (c.x > best[2 * j]) {
                best[2 * j] = c.x;
                arg[2 * j] = a;
              }
              if (c.y > best[2 * j + 1]) {
                best[2 * j + 1] = c.y;
                arg[2 * j + 1] = a;
              }
            }
          }
        }
        float part = 0.f;
#pragma unroll
        for (int j = 0; j < KG; ++j)
          if (k0 + j < R) part = fmaf(__ldg(pi_t + k0 + j), best[j], part);
        red[rr * groups + my_group] = part;
        if (kPol) {
          const size_t base = ((size_t)(t - 1) * S + s0 + rr) * R + k0;
#pragma unroll
          for (int j = 0; j < KG; ++j) {
            if (k0 + j >= R) break;
            if (p.pol32) p.pol32[base + j] = arg[j];
            if (p.pol16) p.pol16[base + j] = (short)arg[j];
          }
        }
      }
      __syncthreads();
      // 4. V'_{t-1}(s): the expectation over the samples, groups in order
      for (int rr = tid; rr < Wt; rr += nth) {
        float acc = 0.f;
        for (int q = 0; q < groups; ++q) acc += red[rr * groups + q];
        __stcg(vout + s0 + rr, acc);
        if (p.v_all) p.v_all[(size_t)(t - 1) * S + s0 + rr] = (float)((double)acc + s_c);
        if (s0 + rr == p.ref_row) __stcg(p.ref_hist + t - 1, acc);
      }
      publish(p.flags + tile, g + 2);
    }
  }
  // V_0 = V'_0 + c_0
  __syncthreads();
  const double c = s_c;
  for (int tile = i0; tile < i1; ++tile) {
    const int s0 = tile * W, s1 = min(S, s0 + W);
    for (int s = s0 + tid; s < s1; s += nth)
      p.v_out[s] = (float)((double)__ldcg(p.v + s) + c);  // V'_0 sits in buffer 0
  }
}

// ---- bid curves (eq. 8-11) and market clearing on the kept values

struct IidActions {  // per action
  const double* p;   // power level (MW)
  const double* f;   // SoC shift in grid steps F(p) tau / delta
  const float* ptf;  // float(p tau): energy sold (MWh), for the float32 filter
  const float* ff;   // float(f)
  int P, S;
  double tau;
};

// V_t at SoC position z (grid steps; feasible when -1e-9 <= z <= S-1+1e-9):
// the grid value within 1e-9 of a grid point, else linear interpolation,
// in double with round-to-nearest operations in a fixed order.
__device__ __forceinline__ double v_at(const float* v, int S, double z) {
  double j = floor(z);
  double b = __dsub_rn(z, j);
  if (b < 1e-9) return (double)v[max(0, min(S - 1, (int)j))];
  if (b > 1.0 - 1e-9) return (double)v[max(0, min(S - 1, (int)j + 1))];
  const int i = (int)j;
  return __dadd_rn(__dmul_rn(__dsub_rn(1.0, b), (double)v[i]), __dmul_rn(b, (double)v[i + 1]));
}

__device__ __forceinline__ bool feasible(double z, int S) {
  return z >= -1e-9 && z <= (double)(S - 1) + 1e-9;
}

// Upper concave envelope over the power levels of U(p_a) = V_t(s + f_a) for
// the feasible actions at grid SoC s (monotone chain, ascending p; a middle
// point is dropped when (y_j - y_i)(x_l - x_i) - (y_l - y_i)(x_j - x_i) <= 0 in
// double); bid price of segment q: -(y_{q+1} - y_q) / ((x_{q+1} - x_q) tau).
__global__ void iid_bids_kernel(const IidActions A, const float* v_all, int t0, int n_t,
                                int* n_bp, int* bp_action, float* bp_price) {
  const long long id = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (id >= (long long)n_t * A.S) return;
  const int tt = (int)(id / A.S), s = (int)(id - (long long)tt * A.S);
  const float* v = v_all + (size_t)(t0 + tt) * A.S;
  int* stk = bp_action + (size_t)id * A.P;
  auto y_of = [&](int a) { return v_at(v, A.S, __dadd_rn((double)s, A.f[a])); };
  int nh = 0;
  for (int l = 0; l < A.P; ++l) {
    if (!feasible(__dadd_rn((double)s, A.f[l]), A.S)) continue;
    const double xl = A.p[l], yl = y_of(l);
    while (nh >= 2) {
      const int i = stk[nh - 2], j = stk[nh - 1];
      const double xi = A.p[i], yi = y_of(i), xj = A.p[j], yj = y_of(j);
      const double cross = __dsub_rn(__dmul_rn(__dsub_rn(yj, yi), __dsub_rn(xl, xi)),
                                     __dmul_rn(__dsub_rn(yl, yi), __dsub_rn(xj, xi)));
      if (cross > 0.0) break;
      --nh;
    }
    stk[nh++] = l;
  }
  n_bp[id] = nh;
  float* pr = bp_price + (size_t)id * A.P;
  for (int q = 0; q + 1 < nh; ++q) {
    const int a = stk[q], b = stk[q + 1];
    const double dy = __dsub_rn(y_of(b), y_of(a));
    pr[q] = (float)(-__ddiv_rn(dy, __dmul_rn(__dsub_rn(A.p[b], A.p[a]), A.tau)));
  }
}

// Merit-order clearing of a price-taking storage against realised prices: at
// stage t the cleared power maximises lam_t p tau + U_t(p; s) over the
// actions (the vertex of the convexified bid curve where the bid price
// crosses lam_t; the first such action on ties), the SoC moves by F(p) tau
// (off the grid at the end points: V_t interpolated there) and the revenue
// lam_t p tau accrues.  One warp per price path: the lanes take the actions
// in turn and the warp reduces (larger value, on equal values the smaller
// action index).
// Float32 enclosure of the clearing value lam p tau + V_t(z + f_a) of action
// a: 0 = surely infeasible, 1 = surely feasible with the value in [lo, hi],
// 2 = feasibility undecided.  The float position zn = z + f carries an error
// of at most m = 2^-24 (|z| + |f| + |zn|) grid steps; within m of a grid
// point the double evaluation may snap or interpolate towards either
// neighbour, elsewhere it interpolates on the same two points with a weight
// within m of the float one; the float arithmetic adds a few roundings of the
// magnitudes involved.
__device__ __forceinline__ int clear_bounds(const IidActions& A, const float* v, float zf,
                                            float lf, int a, float& lo, float& hi) {
  const float U = 5.97e-8f;  // 2^-24, slightly rounded up
  const float ff = A.ff[a];
  const float zn = zf + ff;
  const float m = U * (fabsf(zf) + fabsf(ff) + fabsf(zn)) + 1e-7f;
  const float top = (float)(A.S - 1);
  if (zn < -m - 1e-6f || zn > top + m + 1e-6f) return 0;
  if (zn < m + 1e-6f || zn > top - m - 1e-6f) return 2;
  float vf, ev, mag;
  const float jr = rintf(zn);
  if (fabsf(zn - jr) <= m) {
    const int j = (int)jr;  // in [0, S-1]
    const float vj = v[j];
    const float dl = j > 0 ? fabsf(vj - v[j - 1]) : 0.f;
    const float dr = j < A.S - 1 ? fabsf(v[j + 1] - vj) : 0.f;
    vf = vj;
    ev = 2.01f * m * fmaxf(dl, dr) * 1.01f;
    mag = fabsf(vj);
  } else {
    const int j = (int)floorf(zn);  // in [0, S-2], zn - j in (m, 1 - m)
    const float b = zn - (float)j;
    const float v0 = v[j], v1 = v[j + 1];
    vf = (1.f - b) * v0 + b * v1;
    ev = 1.01f * (m + 1e-9f) * fabsf(v1 - v0);
    mag = fabsf(v0) + fabsf(v1);
  }
  const float pr = lf * A.ptf[a];
  const float val = pr + vf;
  const float err = 1.01f * (ev + U * (6.f * mag + 4.f * fabsf(pr) + 2.f * fabsf(val))) + 1e-30f;
  lo = val - err;
  hi = val + err;
  return 1;
}

// One warp per price path through all stages: at each stage the cleared
// action maximises lam_t p tau + V_t(z + f_a) over the feasible actions (the
// larger value, then the smaller index), exactly as in double.  A float32 pass
// first encloses every action's value; its best lower bound L over the surely
// feasible actions lies below the maximum, so only the actions whose upper
// bound reaches L (or whose feasibility is undecided) are evaluated in double.
__global__ void iid_clear_kernel(const IidActions A, const float* v_all, int T, const float* lam,
                                 int n_paths, double s0, double* revenue, double* s_end,
                                 int* actions) {
  const int lane = threadIdx.x & 31;
  const int path = (int)((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5);
  if (path >= n_paths) return;  // whole warps leave together
  double z = s0, rev = 0.0;
  for (int t = 1; t <= T; ++t) {
    const float* v = v_all + (size_t)t * A.S;
    const float lf = lam[(size_t)path * T + t - 1];
    const double l = (double)lf;
    const float zf = (float)z;
    float L = -INFINITY;
    for (int a = lane; a < A.P; a += 32) {
      float lo, hi;
      if (clear_bounds(A, v, zf, lf, a, lo, hi) == 1) L = fmaxf(L, lo);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) L = fmaxf(L, __shfl_xor_sync(0xffffffffu, L, o));
    double best = -INFINITY;
    int arg = 0x7fffffff;
    for (int a = lane; a < A.P; a += 32) {
      float lo, hi;
      const int kind = clear_bounds(A, v, zf, lf, a, lo, hi);
      if (kind == 0 || (kind == 1 && hi < L)) continue;
      const double zn = __dadd_rn(z, A.f[a]);
      if (!feasible(zn, A.S)) continue;
      const double val = __dadd_rn(__dmul_rn(l, __dmul_rn(A.p[a], A.tau)), v_at(v, A.S, zn));
      if (val > best) {
        best = val;
        arg = a;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const double ob = __shfl_xor_sync(0xffffffffu, best, o);
      const int oa = __shfl_xor_sync(0xffffffffu, arg, o);
      if (ob > best || (ob == best && oa < arg)) {
        best = ob;
        arg = oa;
      }
    }
    if (arg == 0x7fffffff) arg = 0;  // not reached: idle is always feasible
    rev = __dadd_rn(rev, __dmul_rn(l, __dmul_rn(A.p[arg], A.tau)));
    z = __dadd_rn(z, A.f[arg]);
    const double zr = rint(z);
    if (fabs(__dsub_rn(z, zr)) < 1e-9) z = zr;
    if (actions && lane == 0) actions[(size_t)path * T + t - 1] = arg;
  }
  if (lane == 0) {
    revenue[path] = rev;
    if (s_end) s_end[path] = z;
  }
}

// rho_t = sum_k pi_t[k] in double
__global__ void iid_rho_kernel(const float* pi, double* rho, int T, int R) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= T) return;
  double acc = 0.0;
  for (int k = 0; k < R; ++k) acc += (double)pi[(size_t)t * R + k];
  rho[t] = acc;
}

int msg(char* buf, int32_t len, int code, const char* text) {
  if (buf && len > 0) {
    std::strncpy(buf, text, (size_t)len - 1);
    buf[len - 1] = '\0';
  }
  return code;
}

// The action grid of eq. 13: -p_max, -(n_c-1) delta/eta, ..., -delta/eta, 0,
// delta eta, ..., (n_d-1) delta eta, p_max with n_c = ceil(p_max eta/delta) and
// n_d = ceil(p_max/(delta eta)).
std::vector<double> action_grid(const esdp_iid_problem& q) {
  const double delta = q.s_max / (double)(q.S - 1);
  const int n_c = (int)std::ceil(q.p_max * q.eta / delta - 1e-12);
  const int n_d = (int)std::ceil(q.p_max / (delta * q.eta) - 1e-12);
  std::vector<double> p;
  p.push_back(-q.p_max);
  for (int j = n_c - 1; j >= 1; --j) p.push_back(-(double)j * delta / q.eta);
  p.push_back(0.0);
  for (int j = 1; j <= n_d - 1; ++j) p.push_back((double)j * delta * q.eta);
  p.push_back(q.p_max);
  return p;
}

// Device time of the last successful esdp_solve_iid of this host thread.
thread_local double g_iid_sweep_ms = -1.0;

}  // namespace
}  // namespace esdp

using namespace esdp;

extern "C" int esdp_iid_actions(const esdp_iid_problem* q, double* p_hat, int32_t* n_actions) {
  if (!q || !n_actions || q->S < 2 || !(q->s_max > 0) || !(q->p_max > 0) || !(q->eta > 0) ||
      q->eta > 1 || !(q->tau > 0))
    return ESDP_EINVAL;
  const std::vector<double> p = action_grid(*q);
  *n_actions = (int32_t)p.size();
  if (p_hat) std::copy(p.begin(), p.end(), p_hat);
  return ESDP_OK;
}

extern "C" int esdp_solve_iid(const esdp_iid_problem* q, const float* lam_hat, const float* pi_hat,
                              const float* terminal, float* V0, float* V_all, void* policy,
                              uint32_t flags, void* stream, char* err, int32_t err_len) {
  char buf[256];
  if (!q || !lam_hat || !pi_hat || !V0) return msg(err, err_len, ESDP_EINVAL, "null argument");
  if (q->T < 1 || q->S < 2 || q->R < 1 || q->R > kIidKG * kIidBlock)
    return msg(err, err_len, ESDP_EINVAL, "T >= 1, S >= 2 and 1 <= R <= 4096 required");
  if (!(q->s_max > 0) || !(q->p_max > 0) || !(q->eta > 0) || q->eta > 1 || !(q->tau > 0))
    return msg(err, err_len, ESDP_EINVAL, "s_max, p_max, tau > 0 and 0 < eta <= 1 required");
  if (q->policy_bytes != 0 && q->policy_bytes != 2 && q->policy_bytes != 4)
    return msg(err, err_len, ESDP_EINVAL, "policy_bytes must be 0, 2 or 4");
  if (q->policy_bytes && !policy)
    return msg(err, err_len, ESDP_EINVAL, "policy_bytes > 0 needs a policy array");
  const bool dev = (flags & ESDP_DEVICE_PTRS) != 0;
  cudaStream_t st = (cudaStream_t)stream;
  const int T = q->T, S = q->S, R = q->R;
  const double delta = q->s_max / (double)(S - 1);
  const std::vector<double> p_hat = action_grid(*q);
  const int P = (int)p_hat.size();
  // per action: payoff coefficient, SoC shift f in grid steps (eq. 2), the
  // grid point below and the interpolation weight (shifts within 1e-9 of a
  // grid point are taken as on it), the feasible rows
  std::vector<float> pay(P), bw(P);
  std::vector<int> dlo(P), smin(P), smax(P);
  int dmin = 0, dmax = 0;
  for (int a = 0; a < P; ++a) {
    const double pa = p_hat[a];
    const double F = pa >= 0 ? -pa / q->eta : -q->eta * pa;
    const double f = F * q->tau / delta;
    double fl = std::floor(f), fr = f - fl;
    if (fr < 1e-9) fr = 0.0;
    if (fr > 1.0 - 1e-9) {
      fr = 0.0;
      fl += 1.0;
    }
    pay[a] = (float)(pa * q->tau);
    dlo[a] = (int)fl;
    bw[a] = (float)fr;
    smin[a] = (int)std::ceil(-f - 1e-9);
    smax[a] = (int)std::floor((double)(S - 1) - f + 1e-9);
    dmin = std::min(dmin, dlo[a]);
    dmax = std::max(dmax, dlo[a] + (fr > 0 ? 1 : 0));
  }
  const int groups8 = (R + 5) / 6;  // the largest group count, KG = 6 (shared memory)
  int dev_id = 0, n_sm = 0;
  cudaGetDevice(&dev_id);
  cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev_id);
  // one tile per SM where shared memory allows (rows beyond one pass of the
  // block are taken in further passes): the per-tile wait, halo load and
  // barriers then occur once per CTA and stage
  int W = std::max(1, (S + n_sm - 1) / n_sm);
  auto smem_of = [&](int w) {
    auto al = [](size_t x) { return (x + 31) / 32 * 32; };
    const size_t span = (size_t)w + (size_t)(dmax - dmin) + 2;
    const size_t Pp = (size_t)(P + 3) / 4 * 4;
    return (al(span) + 2 * (size_t)w * Pp + al(P) + al((size_t)w * groups8)) * sizeof(float);
  };
  while (W > 1 && smem_of(W) > kIidSmemLimit) --W;
  if (smem_of(W) > kIidSmemLimit)
    return msg(err, err_len, ESDP_EINVAL, "the action halo does not fit shared memory");
  const int n_tiles = (S + W - 1) / W;
  const int reach = (std::max(-dmin, dmax) + W - 1) / W;
  if (2 * reach + 2 > kIidBlock) return msg(err, err_len, ESDP_EINVAL, "action halo too wide");

  // workspace
  std::vector<void*> allocs;
  auto alloc = [&](void** p_, size_t bytes) {
    if (cudaMalloc(p_, std::max<size_t>(bytes, 16)) != cudaSuccess) {
      cudaGetLastError();
      return false;
    }
    allocs.push_back(*p_);
    return true;
  };
  auto cleanup = [&]() {
    cudaStreamSynchronize(st);
    for (void* a : allocs) cudaFree(a);
  };
  void *d_pay, *d_dlo, *d_bw, *d_smin, *d_smax, *d_v, *d_ref, *d_flags, *d_status, *d_rho, *d_cta;
  void *d_lam = nullptr, *d_pi = nullptr, *d_term = nullptr, *d_v0 = nullptr, *d_pol = nullptr,
       *d_vall = nullptr;
  const size_t pol_bytes = (size_t)q->policy_bytes * T * S * R;
  bool ok = alloc(&d_pay, P * 4) && alloc(&d_dlo, P * 4) && alloc(&d_bw, P * 4) &&
            alloc(&d_smin, P * 4) && alloc(&d_smax, P * 4) && alloc(&d_v, (size_t)2 * S * 4) &&
            alloc(&d_ref, (size_t)(T + 1) * 4) && alloc(&d_flags, (size_t)n_tiles * 4) &&
            alloc(&d_status, 4) && alloc(&d_rho, (size_t)T * 8) &&
            alloc(&d_cta, (size_t)(n_sm + 1) * 4);
  if (ok && !dev) {
    ok = alloc(&d_lam, (size_t)T * R * 4) && alloc(&d_pi, (size_t)T * R * 4) &&
         alloc(&d_v0, (size_t)S * 4) && (!terminal || alloc(&d_term, (size_t)S * 4)) &&
         (!q->policy_bytes || alloc(&d_pol, pol_bytes)) &&
         (!V_all || alloc(&d_vall, (size_t)(T + 1) * S * 4));
  }
  if (!ok) {
    cleanup();
    return msg(err, err_len, ESDP_ENOMEM, "device workspace allocation failed");
  }
  auto h2d = [&](void* d, const void* h, size_t n) {
    return cudaMemcpyAsync(d, h, n, cudaMemcpyHostToDevice, st) == cudaSuccess;
  };
  ok = h2d(d_pay, pay.data(), P * 4) && h2d(d_dlo, dlo.data(), P * 4) &&
       h2d(d_bw, bw.data(), P * 4) && h2d(d_smin, smin.data(), P * 4) &&
       h2d(d_smax, smax.data(), P * 4);
  if (ok && !dev) {
    ok = h2d(d_lam, lam_hat, (size_t)T * R * 4) && h2d(d_pi, pi_hat, (size_t)T * R * 4) &&
         (!terminal || h2d(d_term, terminal, (size_t)S * 4));
  }
  // samples per thread: the block takes rows in passes of kIidBlock / groups
  // rows; of 6, 8 and 10 samples the one with the least work per thread for a
  // tile (passes x samples) wins, 8 on ties
  auto work = [&](int kg) {
    const int g = (R + kg - 1) / kg, rows_pass = kIidBlock / g;
    return rows_pass < 1 ? 1 << 30 : ((W + rows_pass - 1) / rows_pass) * kg;
  };
  int KG = 8;
  if (work(10) < work(KG)) KG = 10;
  if (work(6) < work(KG)) KG = 6;
  const int groups = (R + KG - 1) / KG;
  // launch shape: one CTA per SM at most, contiguous tile ranges
  const bool pk = policy && q->policy_bytes;
  auto fn = KG == 10 ? (pk ? iid_kernel<true, 10> : iid_kernel<false, 10>)
            : KG == 6 ? (pk ? iid_kernel<true, 6> : iid_kernel<false, 6>)
                      : (pk ? iid_kernel<true, 8> : iid_kernel<false, 8>);
  const size_t smem = smem_of(W);
  cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, kIidBlock, smem);
  const int grid = std::max(1, std::min(n_tiles, std::min(n_sm, per_sm * n_sm)));
  std::vector<int> cta(grid + 1);
  for (int b = 0; b <= grid; ++b) cta[b] = (int)((long long)n_tiles * b / grid);
  ok = ok && h2d(d_cta, cta.data(), (size_t)(grid + 1) * 4) &&
       cudaMemsetAsync(d_flags, 0, (size_t)n_tiles * 4, st) == cudaSuccess &&
       cudaMemsetAsync(d_status, 0, 4, st) == cudaSuccess;
  if (!ok || per_sm < 1) {
    cleanup();
    return msg(err, err_len, ESDP_ECUDA, "workspace setup failed");
  }
  IidParams ip{};
  ip.T = T; ip.S = S; ip.R = R; ip.P = P; ip.W = W; ip.n_tiles = n_tiles; ip.reach = reach;
  ip.groups = groups;
  ip.dmin = dmin;
  ip.span = W + (dmax - dmin) + 2;
  ip.ref_row = S / 2;
  ip.ref_tile = ip.ref_row / W;
  ip.lam = (const float*)(dev ? lam_hat : d_lam);
  ip.pi = (const float*)(dev ? pi_hat : d_pi);
  ip.rho = (const double*)d_rho;
  ip.pay = (const float*)d_pay;
  ip.dlo = (const int*)d_dlo;
  ip.bw = (const float*)d_bw;
  ip.smin = (const int*)d_smin;
  ip.smax = (const int*)d_smax;
  ip.terminal = dev ? terminal : (const float*)d_term;
  ip.v = (float*)d_v;
  ip.ref_hist = (float*)d_ref;
  ip.flags = (int*)d_flags;
  ip.status = (int*)d_status;
  void* pol = dev ? policy : d_pol;
  ip.pol32 = q->policy_bytes == 4 ? (int*)pol : nullptr;
  ip.pol16 = q->policy_bytes == 2 ? (short*)pol : nullptr;
  ip.v_out = dev ? V0 : (float*)d_v0;
  ip.v_all = V_all ? (dev ? V_all : (float*)d_vall) : nullptr;
  ip.cta_first = (const int*)d_cta;
  ip.timeout_ns = 5ull * 1000 * 1000 * 1000;
  // device time of the sweep (events on the call's stream, the workspace set
  // up before them), kept per host thread for esdp_iid_last_sweep_ms
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  const bool timed = cudaEventCreate(&ev0) == cudaSuccess && cudaEventCreate(&ev1) == cudaSuccess &&
                     cudaEventRecord(ev0, st) == cudaSuccess;
  iid_rho_kernel<<<(T + 127) / 128, 128, 0, st>>>(ip.pi, (double*)d_rho, T, R);
  void* args[] = {&ip};
  cudaError_t e = cudaLaunchCooperativeKernel((const void*)fn, dim3(grid), dim3(kIidBlock), args,
                                              smem, st);
  const bool timed_end = timed && e == cudaSuccess && cudaEventRecord(ev1, st) == cudaSuccess;
  int status = 0;
  if (e == cudaSuccess) e = cudaMemcpyAsync(&status, d_status, 4, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess && !dev) {
    e = cudaMemcpyAsync(V0, d_v0, (size_t)S * 4, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && q->policy_bytes)
      e = cudaMemcpyAsync(policy, d_pol, pol_bytes, cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess && V_all)
      e = cudaMemcpyAsync(V_all, d_vall, (size_t)(T + 1) * S * 4, cudaMemcpyDeviceToHost, st);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  float ms = -1.f;
  if (e == cudaSuccess && timed_end && cudaEventElapsedTime(&ms, ev0, ev1) != cudaSuccess) ms = -1.f;
  if (ev0) cudaEventDestroy(ev0);
  if (ev1) cudaEventDestroy(ev1);
  cleanup();
  if (e != cudaSuccess) {
    std::snprintf(buf, sizeof(buf), "CUDA error: %s", cudaGetErrorString(e));
    return msg(err, err_len, ESDP_ECUDA, buf);
  }
  if (status) {
    std::snprintf(buf, sizeof(buf), "device reported status %d", status);
    return msg(err, err_len, status, buf);
  }
  g_iid_sweep_ms = ms;
  return ESDP_OK;
}

extern "C" double esdp_iid_last_sweep_ms(void) { return g_iid_sweep_ms; }

namespace {

// the per-action arrays of IidActions on the device
struct ActionsBuf {
  double* d = nullptr;
  IidActions a{};
};

int make_actions(const esdp_iid_problem& q, ActionsBuf* out, char* err, int32_t err_len) {
  const std::vector<double> p = action_grid(q);
  const int P = (int)p.size();
  const double delta = q.s_max / (double)(q.S - 1);
  // [p (double)][f (double)][float(p tau), float(f) as float pairs in P doubles]
  std::vector<double> h(3 * P);
  float* hf = reinterpret_cast<float*>(h.data() + 2 * P);
  for (int a = 0; a < P; ++a) {
    h[a] = p[a];
    const double F = p[a] >= 0 ? -p[a] / q.eta : -q.eta * p[a];
    h[P + a] = F * q.tau / delta;
    hf[a] = (float)(p[a] * q.tau);
    hf[P + a] = (float)h[P + a];
  }
  if (cudaMalloc(&out->d, 3 * P * sizeof(double)) != cudaSuccess) {
    cudaGetLastError();
    return msg(err, err_len, ESDP_ENOMEM, "allocation failed");
  }
  if (cudaMemcpy(out->d, h.data(), 3 * P * sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
    cudaFree(out->d);
    return msg(err, err_len, ESDP_ECUDA, "copy failed");
  }
  out->a.p = out->d;
  out->a.f = out->d + P;
  out->a.ptf = reinterpret_cast<const float*>(out->d + 2 * P);
  out->a.ff = out->a.ptf + P;
  out->a.P = P;
  out->a.S = q.S;
  out->a.tau = q.tau;
  return ESDP_OK;
}

int check_problem(const esdp_iid_problem* q, char* err, int32_t err_len) {
  if (!q || q->T < 1 || q->S < 2 || !(q->s_max > 0) || !(q->p_max > 0) || !(q->eta > 0) ||
      q->eta > 1 || !(q->tau > 0))
    return msg(err, err_len, ESDP_EINVAL, "invalid problem");
  return ESDP_OK;
}

}  // namespace

extern "C" int esdp_iid_bids(const esdp_iid_problem* q, const float* V_all, int32_t t0, int32_t t1,
                             int32_t* n_bp, int32_t* bp_action, float* bp_price, void* stream,
                             char* err, int32_t err_len) {
  int rc = check_problem(q, err, err_len);
  if (rc) return rc;
  if (!V_all || !n_bp || !bp_action || !bp_price || t0 < 1 || t1 <= t0 || t1 > q->T + 1)
    return msg(err, err_len, ESDP_EINVAL, "need V_all, outputs and 1 <= t0 < t1 <= T+1");
  ActionsBuf ab;
  if ((rc = make_actions(*q, &ab, err, err_len))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  const long long n = (long long)(t1 - t0) * q->S;
  iid_bids_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(ab.a, V_all, t0, t1 - t0, n_bp,
                                                               bp_action, bp_price);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(ab.d);
  if (e != cudaSuccess) return msg(err, err_len, ESDP_ECUDA, cudaGetErrorString(e));
  return ESDP_OK;
}

extern "C" int esdp_iid_clear(const esdp_iid_problem* q, const float* V_all, const float* lam_real,
                              int32_t n_paths, double s0, double* revenue, double* s_end,
                              int32_t* actions, void* stream, char* err, int32_t err_len) {
  int rc = check_problem(q, err, err_len);
  if (rc) return rc;
  if (!V_all || !lam_real || !revenue || n_paths < 1)
    return msg(err, err_len, ESDP_EINVAL, "need V_all, lam_real, revenue and n_paths >= 1");
  const double z0 = s0 / (q->s_max / (double)(q->S - 1));
  if (!(z0 >= -1e-9) || z0 > (double)(q->S - 1) + 1e-9)
    return msg(err, err_len, ESDP_EINVAL, "s0 outside [0, s_max]");
  ActionsBuf ab;
  if ((rc = make_actions(*q, &ab, err, err_len))) return rc;
  cudaStream_t st = (cudaStream_t)stream;
  iid_clear_kernel<<<(unsigned)(((long long)n_paths * 32 + 255) / 256), 256, 0, st>>>(
      ab.a, V_all, q->T, lam_real, n_paths, z0, revenue, s_end, actions);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(ab.d);
  if (e != cudaSuccess) return msg(err, err_len, ESDP_ECUDA, cudaGetErrorString(e));
  return ESDP_OK;
}
