// Convexified bid curves (Sec. II-C, eq. 10-11): for every (stage, mode,
// price state) the upper concave envelope of EV_t[m][.][k] over the SoC grid,
// i.e. the hypograph convex hull, by Andrew's monotone chain.  Its slopes are
// the monotone marginal values of stored energy from which the price-quantity
// bids are read.
//
// A block handles 32 envelopes (consecutive lanes take consecutive price
// states, so every load is one coalesced row of EV) with kSeg warps: warp q
// first builds the envelope of the q-th segment of the SoC grid of all 32,
// then warp 0 merges the segment envelopes.  Every strict vertex of the whole
// envelope is a strict vertex of its segment's envelope, so the chain over
// the concatenated segment vertices yields exactly the envelope of all points.
//
// A middle point j between i and l is dropped when
//     (y_j - y_i) * (l - i) - (y_l - y_i) * (j - i)  <= 0.
// Its exact sign is taken: in float32 when the value clears a rigorous
// rounding bound, otherwise in 128-bit integers on a common binary grid of the
// three values, and, for exponent spreads beyond 38 bits, by the double
// expression, which is exact up to its last subtraction (whose rounding
// cannot change the sign).  The vertex set is therefore a deterministic
// function of the float32 EV values.
#include <cuda_runtime.h>

#include "esdp_internal.h"

namespace esdp {
namespace {

constexpr int kSeg = 8;    // segments (warps) per block
constexpr int kWin = 16;   // stack entries cached per thread in shared memory

// float32 value as mantissa * 2^(e - 150) with a signed integer mantissa
__device__ __forceinline__ void decompose(float v, long long& m, int& e) {
  const unsigned u = __float_as_uint(v);
  const int eb = (u >> 23) & 0xff;
  const unsigned mant = u & 0x7fffffu;
  long long mm = eb ? (long long)(mant | 0x800000u) : (long long)mant;
  e = eb ? eb : 1;
  m = (u >> 31) ? -mm : mm;
}

// exact sign test of (yj - yi) * L - (yl - yi) * J <= 0
__device__ bool below_exact(float yi, float yj, float yl, int L, int J) {
  long long mi, mj, ml;
  int ei, ej, el;
  decompose(yi, mi, ei);
  decompose(yj, mj, ej);
  decompose(yl, ml, el);
  const int big = 1 << 20;
  const int emin = min(min(mi ? ei : big, mj ? ej : big), ml ? el : big);
  const int emax = max(max(mi ? ei : -big, mj ? ej : -big), ml ? el : -big);
  if (emin == big) return true;  // all three are zero: cross == 0
  if (emax - emin <= 38) {
    const long long Yi = mi ? mi * (1LL << (ei - emin)) : 0;
    const long long Yj = mj ? mj * (1LL << (ej - emin)) : 0;
    const long long Yl = ml ? ml * (1LL << (el - emin)) : 0;
    const __int128 cross = (__int128)(Yj - Yi) * L - (__int128)(Yl - Yi) * J;
    return cross <= 0;
  }
  const double dl = __dmul_rn(__dsub_rn((double)yj, (double)yi), (double)L);
  const double dr = __dmul_rn(__dsub_rn((double)yl, (double)yi), (double)J);
  return __dsub_rn(dl, dr) <= 0.0;
}

// true if point j lies on or below the chord from i to l
__device__ __forceinline__ bool below_chord(float yi, float yj, float yl, int i, int j, int l) {
  const float L = (float)(l - i), J = (float)(j - i);  // exact: grid sizes < 2^24
  const float lhs = __fmul_rn(__fsub_rn(yj, yi), L);
  const float rhs = __fmul_rn(__fsub_rn(yl, yi), J);
  const float cross = __fsub_rn(lhs, rhs);
  // each side carries at most two roundings, the difference one more:
  // |cross - exact| <= (2u + u^2)(|lhs| + |rhs|)(1 + u) + u |cross|, u = 2^-24
  // (taken as 5u, plus an absolute floor so that subnormal ranges always go
  // to the exact route)
  const float bound = 3.0e-7f * (fabsf(lhs) + fabsf(rhs)) + 1e-30f;
  if (cross > bound) return false;
  if (cross < -bound) return true;
  return below_exact(yi, yj, yl, l - i, j - i);
}

// Monotone chain over a stream of points (index, value) in increasing index
// order.  The stack lives in global memory at `stack`; its top kWin entries
// are mirrored in shared memory (slot-major, conflict-free) and the top two in
// registers.
struct Chain {
  int* stack;
  int* s_idx;    // this thread's column of the shared window
  float* s_y;
  const float* y;
  int K;
  int nh = 0, win = 0;
  int i_idx = 0, j_idx = 0;
  float yi = 0.f, yj = 0.f;

  __device__ __forceinline__ int slot(int pos) const {
    return (pos & (kWin - 1)) * (32 * kSeg);
  }

  __device__ __forceinline__ void push(int l, float yl) {
    while (nh >= 2 && below_chord(yi, yj, yl, i_idx, j_idx, l)) {
      --nh;  // j is on or below the chord (i, l)
      win = max(win - 1, 0);  // positions [nh - win, nh) are cached
      j_idx = i_idx;
      yj = yi;
      if (nh >= 2) {
        if (win >= 2) {
          i_idx = s_idx[slot(nh - 2)];
          yi = s_y[slot(nh - 2)];
        } else {
          i_idx = stack[nh - 2];
          yi = __ldg(y + (size_t)i_idx * K);
        }
      }
    }
    s_idx[slot(nh)] = l;
    s_y[slot(nh)] = yl;
    stack[nh] = l;
    ++nh;
    win = min(win + 1, kWin);
    if (nh == 1) {
      j_idx = l;
      yj = yl;
    } else {
      i_idx = j_idx;
      yi = yj;
      j_idx = l;
      yj = yl;
    }
  }
};

__global__ void __launch_bounds__(32 * kSeg) hull_kernel(const HullParams p) {
  __shared__ int s_idx[kWin * 32 * kSeg];
  __shared__ float s_y[kWin * 32 * kSeg];
  __shared__ int s_cnt[kSeg][32];
  const int lane = threadIdx.x & 31, q = threadIdx.x >> 5;
  const int n_h = p.n_t * p.M * p.K;
  const int h = blockIdx.x * 32 + lane;
  const bool valid = h < n_h;
  const int K = p.K, N = p.N;
  const int k = valid ? h % K : 0;
  const int tm = valid ? h / K : 0;  // stage-major, then mode
  const float* y = p.ev + (size_t)tm * N * K + k;
  int* row = p.idx + (size_t)(valid ? h : 0) * N;
  const int seg = (N + kSeg - 1) / kSeg;

  // 1. envelope of segment q of the hull, stacked in place in its own range
  if (valid) {
    const int l0 = q * seg, l1 = min(N, l0 + seg);
    Chain ch;
    ch.stack = row + l0;
    ch.s_idx = s_idx + threadIdx.x;
    ch.s_y = s_y + threadIdx.x;
    ch.y = y;
    ch.K = K;
    constexpr int kAhead = 8;
    float cur[kAhead], nxt[kAhead];
#pragma unroll
    for (int u = 0; u < kAhead; ++u) cur[u] = l0 + u < l1 ? __ldg(y + (size_t)(l0 + u) * K) : 0.f;
    for (int b = l0; b < l1; b += kAhead) {
#pragma unroll
      for (int u = 0; u < kAhead; ++u)
        nxt[u] = b + kAhead + u < l1 ? __ldg(y + (size_t)(b + kAhead + u) * K) : 0.f;
#pragma unroll
      for (int u = 0; u < kAhead; ++u)
        if (b + u < l1) ch.push(b + u, cur[u]);
#pragma unroll
      for (int u = 0; u < kAhead; ++u) cur[u] = nxt[u];
    }
    s_cnt[q][lane] = l0 < l1 ? ch.nh : 0;
  } else {
    s_cnt[q][lane] = 0;
  }
  __syncthreads();

  // 2. merge: the chain over the segment vertices in order, written in place
  //    (the output position never passes the entries still to be read)
  if (q == 0 && valid) {
    Chain ch;
    ch.stack = row;
    ch.s_idx = s_idx + threadIdx.x;
    ch.s_y = s_y + threadIdx.x;
    ch.y = y;
    ch.K = K;
    for (int s = 0; s < kSeg; ++s) {
      const int n = s_cnt[s][lane];
      for (int v = 0; v < n; ++v) {
        const int l = row[s * seg + v];
        ch.push(l, __ldg(y + (size_t)l * K));
      }
    }
    p.n_bp[h] = ch.nh;
    s_cnt[0][lane] = ch.nh;
  }
  __syncthreads();

  // 3. slopes between consecutive vertices, $ per MWh of stored energy
  if (valid) {
    const int nh = s_cnt[0][lane];
    float* sl = p.slope + (size_t)h * N;
    for (int v = q; v + 1 < nh; v += kSeg) {
      const int a = row[v], b = row[v + 1];
      const double ya = (double)__ldg(y + (size_t)a * K), yb = (double)__ldg(y + (size_t)b * K);
      sl[v] = (float)(__ddiv_rn(__dsub_rn(yb, ya), __dmul_rn((double)(b - a), p.delta)));
    }
  }
}

// Reported EV_t = EV'_t + evoff_t[k] for every kept stage, in place, as a
// float32 compensated sum: the level is split into hi + lo floats and the
// rounding error of EV' + hi (TwoSum) is carried into the final addition.
__device__ __forceinline__ float add_level(float a, float hi, float lo) {
  const float s = __fadd_rn(a, hi);
  const float bb = __fsub_rn(s, a);
  const float err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(hi, bb));
  return __fadd_rn(s, __fadd_rn(err, lo));
}

// grid.y = stage; rows of K values, float4 when K is a multiple of 4
__global__ void ev_restore_kernel(float* ev, const double* evoff, int MN, int K) {
  __shared__ float s_hi[128], s_lo[128];
  const int t = blockIdx.y;
  for (int k = threadIdx.x; k < K; k += blockDim.x) {
    const double o = evoff[(size_t)t * K + k];
    s_hi[k] = (float)o;
    s_lo[k] = (float)(o - (double)(float)o);
  }
  __syncthreads();
  float* e = ev + (size_t)t * MN * K;
  const int n = MN * K;
  if ((K & 3) == 0) {
    float4* e4 = reinterpret_cast<float4*>(e);
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n / 4; i += gridDim.x * blockDim.x) {
      const int k = (4 * i) % K;
      float4 v = e4[i];
      v.x = add_level(v.x, s_hi[k], s_lo[k]);
      v.y = add_level(v.y, s_hi[k + 1], s_lo[k + 1]);
      v.z = add_level(v.z, s_hi[k + 2], s_lo[k + 2]);
      v.w = add_level(v.w, s_hi[k + 3], s_lo[k + 3]);
      e4[i] = v;
    }
  } else {
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      const int k = i % K;
      e[i] = add_level(e[i], s_hi[k], s_lo[k]);
    }
  }
}

}  // namespace

cudaError_t launch_hull(const HullParams& p, cudaStream_t stream) {
  const int n_h = p.n_t * p.M * p.K;
  if (n_h == 0) return cudaSuccess;
  hull_kernel<<<(n_h + 31) / 32, 32 * kSeg, 0, stream>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_ev_restore(float* ev, const double* evoff, int n_t, int MN, int K,
                              cudaStream_t stream) {
  const long long n = (long long)MN * K;
  if (n == 0 || n_t == 0) return cudaSuccess;
  const int block = 256;
  const long long per = ((K & 3) == 0 ? n / 4 : n);
  const int gx = (int)((per + block - 1) / block < 64 ? (per + block - 1) / block : 64);
  ev_restore_kernel<<<dim3(gx, n_t), block, 0, stream>>>(ev, evoff, MN, K);
  return cudaGetLastError();
}

}  // namespace esdp
