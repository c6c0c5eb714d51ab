// Convexified bid curves (Sec. II-C, eq. 10-11): for every (stage, mode,
// price state) the upper concave envelope of EV_t[m][.][k] over the SoC grid,
// i.e. the hypograph convex hull, by Andrew's monotone chain.  Its slopes are
// the monotone marginal values of stored energy from which the price-quantity
// bids are read.
//
// One warp per envelope: the lanes build the hulls of 32 consecutive parts of
// the SoC grid and join them pairwise by upper bridges (details at the
// kernel).  The joined hull of two adjacent strict hulls is a prefix of the
// left one, the bridge, and a suffix of the right one, so every strict vertex
// of the whole envelope survives from its part's hull.
//
// A middle point j between i and l is dropped when
//     (y_j - y_i) * (l - i) - (y_l - y_i) * (j - i)  <= 0.
// Its exact sign is taken: in float32 when the value clears a rigorous
// rounding bound, otherwise by error-free float32 transformations (TwoSum,
// FMA residuals) where they settle it, else in 128-bit integers on a common
// binary grid of the three values, and, for exponent spreads beyond 38 bits,
// by the double expression, which is exact up to its last subtraction (whose
// rounding cannot change the sign).  The vertex set is therefore a deterministic
// function of the float32 EV values.
#include <cuda_runtime.h>

#include "esdp_internal.h"

namespace esdp {
namespace {


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

// rounding error of s = RN(a + b): a + b = s + err exactly (Knuth's TwoSum)
__device__ __forceinline__ float two_sum_err(float a, float b, float s) {
  const float bv = __fsub_rn(s, a);
  const float av = __fsub_rn(s, bv);
  return __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
}

// Exact sign of the cross product by error-free float32 transformations, for
// the near-collinear triples the rounded test leaves open.  With
// a = RN(yj - yi), b = RN(yl - yi) exact (TwoSum errors zero), the products
// split exactly as a L = lhs + e1, b J = rhs + e2 (FMA residuals, exact away
// from underflow), and lhs - rhs = d exactly (TwoSum error zero), so the cross
// product is d + e1 - e2.  Its sign is that of e1 - e2 when d = 0 and that of
// d when |d| > 2 max(|e1|, |e2|).  Returns 1 (on or below), 0 (above) or -1
// (not decided here).
__device__ __forceinline__ int below_near(float yi, float yj, float yl, float L, float J) {
  const float a = __fsub_rn(yj, yi), b = __fsub_rn(yl, yi);
  if (two_sum_err(yj, -yi, a) != 0.f || two_sum_err(yl, -yi, b) != 0.f) return -1;
  const float lhs = __fmul_rn(a, L), rhs = __fmul_rn(b, J);
  // residuals are exact unless the products are near the underflow range
  if ((lhs != 0.f && fabsf(lhs) < 1e-28f) || (rhs != 0.f && fabsf(rhs) < 1e-28f)) return -1;
  const float e1 = __fmaf_rn(a, L, -lhs), e2 = __fmaf_rn(b, J, -rhs);
  const float d = __fsub_rn(lhs, rhs);
  if (two_sum_err(lhs, -rhs, d) != 0.f) return -1;
  if (d == 0.f) return e1 <= e2;
  if (fabsf(d) > 2.f * fmaxf(fabsf(e1), fabsf(e2))) return d < 0.f;
  return -1;
}

// true if point j lies on or below the chord from i to l (SoC indices as
// float32, exact below 2^24, and so are their differences)
__device__ __forceinline__ bool below_chord(float yi, float yj, float yl, float xi, float xj,
                                            float xl) {
  const float L = __fsub_rn(xl, xi), J = __fsub_rn(xj, xi);
  const float lhs = __fmul_rn(__fsub_rn(yj, yi), L);
  const float rhs = __fmul_rn(__fsub_rn(yl, yi), J);
  const float cross = __fsub_rn(lhs, rhs);
  // each side carries at most two roundings, the difference one more:
  // |cross - exact| <= (2u + u^2)(|lhs| + |rhs|)(1 + u) + u |cross|, u = 2^-24
  // (taken as 5u, plus an absolute floor so that subnormal ranges always go
  // to the exact routes)
  const float bound = 3.0e-7f * (fabsf(lhs) + fabsf(rhs)) + 1e-30f;
  if (cross > bound) return false;
  if (cross < -bound) return true;
  const int near = below_near(yi, yj, yl, L, J);
  if (near >= 0) return near != 0;
  return below_exact(yi, yj, yl, (int)L, (int)J);
}

// One warp per envelope.  Lane l takes the points [l c, (l+1) c) of the SoC
// grid (c = ceil(N/32) rounded up to odd, so that the lanes' equal steps fall
// in distinct shared-memory banks) and builds their strict upper hull with the
// monotone chain.  Five levels then join adjacent groups of lanes: the leader
// of each pair finds the upper bridge of the left and the right hull by the
// tangent walk (drop the left end point while it lies on or below the chord
// from its predecessor to the right end point, drop the right end point while
// it lies on or below the chord from the left end point to its successor,
// until neither moves), and only trims the kept range of each lane's stack
// (no copying): the joined hull is the left hull up to the bridge and the
// right hull from it.  The surviving ranges are read out in order by a prefix
// sum and a binary search over the lanes, so that the index and slope rows
// are written coalesced.  With the exact orientation sign the vertex set is
// the unique set of strict vertices, the same as one monotone chain over all
// points.
//
// kStaged: a block of nw warps first copies the columns of its nw envelopes
// into shared memory (cp.async; consecutive threads read consecutive price
// states of one SoC row); each lane's stack then keeps the SoC index (16
// bits) and, in place of the column, the value of its vertices, so a pop or a
// walk step needs no dependent lookup.  N * 6 bytes per warp (four blocks of
// eight warps per SM at N = 1001).  For grids too long for that, the values
// are read in place and the slope row holds the stacks' indices as floats.
constexpr int kHullWarps = 8;
constexpr int kHullSmemBudget = 96 * 1024;  // dynamic shared memory per block

// SoC index (< 2^16) stored in 16 bits -> exact float32, without a
// conversion instruction: 2^23 + i has i as its low mantissa bits
__device__ __forceinline__ float index_float(unsigned short i) {
  return __fsub_rn(__uint_as_float(0x4B000000u + (unsigned)i), 8388608.f);
}

template <bool kStaged>
struct HullView {
  const float* y;          // in place: the envelope's column, stride K
  float* sv;               // staged: the column, overwritten by the stacks' values
  unsigned short* st16;    // staged: the stacks' SoC indices (lane l from position l*c)
  float* st;               // in place: the same as exact floats, in the slope row
  int K;
  int* lo;                 // [32] kept range [lo, hi) of each lane's stack
  int* hi;
  // SoC index of the stack entry at position pos, as an exact float
  __device__ __forceinline__ float xs(int pos) const {
    if constexpr (kStaged)
      return index_float(st16[pos]);
    else
      return st[pos];
  }
  __device__ __forceinline__ void push(int pos, int l, float xl) {
    if constexpr (kStaged)
      st16[pos] = (unsigned short)l;
    else
      st[pos] = xl;
  }
  // value of SoC point l before the local hulls
  __device__ __forceinline__ float point(int l) const {
    if constexpr (kStaged)
      return sv[l];
    else
      return __ldg(y + (size_t)l * K);
  }
  // value of the stack entry at position pos
  __device__ __forceinline__ float val(int pos) const {
    if constexpr (kStaged)
      return sv[pos];
    else
      return __ldg(y + (size_t)(int)st[pos] * K);
  }
  // SoC index of the stack entry at position pos
  __device__ __forceinline__ int xi(int pos) const {
    if constexpr (kStaged)
      return st16[pos];
    else
      return (int)st[pos];
  }
  // previous kept vertex of (l, i) within lanes >= lmin, or l = -1
  __device__ __forceinline__ void prev(int& l, int& i, int lmin) const {
    if (i > lo[l]) {
      --i;
      return;
    }
    for (int q = l - 1; q >= lmin; --q)
      if (hi[q] > lo[q]) {
        l = q;
        i = hi[q] - 1;
        return;
      }
    l = -1;
  }
  // next kept vertex of (l, i) within lanes < lend, or l = -1
  __device__ __forceinline__ void next(int& l, int& i, int lend) const {
    if (i + 1 < hi[l]) {
      ++i;
      return;
    }
    for (int q = l + 1; q < lend; ++q)
      if (hi[q] > lo[q]) {
        l = q;
        i = lo[q];
        return;
      }
    l = -1;
  }
};

// slope between two vertices, $ per MWh of stored energy
__device__ __forceinline__ float hull_slope(float xa, float ya, float xb, float yb, double delta) {
  return (float)(__ddiv_rn(__dsub_rn((double)yb, (double)ya),
                           __dmul_rn((double)__fsub_rn(xb, xa), delta)));
}

// blockDim.x = 32 << lg_nw
template <bool kStaged>
__global__ void __launch_bounds__(32 * kHullWarps) hull_kernel(const HullParams p, int lg_nw) {
  extern __shared__ float hull_smem[];  // staged: [nw][N] values, then [nw][N] 16-bit indices
  __shared__ int s_lo[kHullWarps][32], s_hi[kHullWarps][32], s_pre[kHullWarps][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int nw = 1 << lg_nw;
  const int n_h = p.n_t * p.M * p.K;
  const int K = p.K, N = p.N;
  const int h0 = blockIdx.x * nw;
  if constexpr (kStaged) {
    // thread -> envelope h0 + (tid mod nw), SoC rows tid/nw, tid/nw + 32, ...
    const int ww = threadIdx.x & (nw - 1), hh = h0 + ww;
    if (hh < n_h) {
      const float* col = p.ev + (size_t)(hh / K) * N * K + hh % K;
      const unsigned dst = (unsigned)__cvta_generic_to_shared(hull_smem + ww * N);
      for (int l = threadIdx.x >> lg_nw; l < N; l += 32)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(dst + 4u * (unsigned)l),
                     "l"(col + (size_t)l * K)
                     : "memory");
    }
    asm volatile("cp.async.wait_all;\n" ::: "memory");
    __syncthreads();
  }
  const int h = h0 + w;
  if (h >= n_h) return;  // whole warps, after the block's only barrier
  const int k = h % K, tm = h / K;  // stage-major, then mode
  int* row = p.idx + (size_t)h * N;
  float* sl = p.slope + (size_t)h * N;
  HullView<kStaged> v;
  v.K = K;
  v.lo = s_lo[w];
  v.hi = s_hi[w];
  if constexpr (kStaged) {
    v.y = nullptr;
    v.sv = hull_smem + w * N;
    v.st16 = reinterpret_cast<unsigned short*>(hull_smem + nw * N) + w * N;
    v.st = nullptr;
  } else {
    v.y = p.ev + (size_t)tm * N * K + k;
    v.sv = nullptr;
    v.st16 = nullptr;
    v.st = sl;  // scratch until the slopes
  }
  const int c = ((N + 31) / 32) | 1;

  // 1. local hull of the lane's points
  const int l0 = min(N, lane * c), l1 = min(N, l0 + c);
  int nh = 0;
  float xi = 0.f, xj = 0.f, yi = 0.f, yj = 0.f;
  float xl = (float)l0;
  for (int l = l0; l < l1; ++l, xl = __fadd_rn(xl, 1.f)) {
    const float yl = v.point(l);
    while (nh >= 2 && below_chord(yi, yj, yl, xi, xj, xl)) {
      --nh;
      xj = xi;
      yj = yi;
      if (nh >= 2) {
        xi = v.xs(l0 + nh - 2);
        yi = v.val(l0 + nh - 2);
      }
    }
    v.push(l0 + nh, l, xl);
    if constexpr (kStaged) v.sv[l0 + nh] = yl;  // position <= l: already read
    ++nh;
    if (nh == 1) {
      xj = xl;
      yj = yl;
    } else {
      xi = xj;
      yi = yj;
      xj = xl;
      yj = yl;
    }
  }
  v.lo[lane] = 0;
  v.hi[lane] = nh;
  __syncwarp();

  // 2. join the lanes' hulls pairwise: groups of 2, 4, ..., 32 lanes
  for (int d = 1; d < 32; d <<= 1) {
    if ((lane & (2 * d - 1)) == 0) {
      const int gl = lane, gm = lane + d, ge = lane + 2 * d;
      // right end of the left group, left end of the right group
      int la = -1, ia = 0, lb = -1, ib = 0;
      for (int q = gm - 1; q >= gl; --q)
        if (v.hi[q] > v.lo[q]) {
          la = q;
          ia = v.hi[q] - 1;
          break;
        }
      for (int q = gm; q < ge; ++q)
        if (v.hi[q] > v.lo[q]) {
          lb = q;
          ib = v.lo[q];
          break;
        }
      if (la >= 0 && lb >= 0) {
        float xa = v.xs(la * c + ia), ya = v.val(la * c + ia);
        float xb = v.xs(lb * c + ib), yb = v.val(lb * c + ib);
        for (bool moved = true; moved;) {
          moved = false;
          for (;;) {  // left end point on or below the chord (its predecessor, right end)?
            int lp = la, ip = ia;
            v.prev(lp, ip, gl);
            if (lp < 0) break;
            const float xp = v.xs(lp * c + ip), yp = v.val(lp * c + ip);
            if (!below_chord(yp, ya, yb, xp, xa, xb)) break;
            la = lp;
            ia = ip;
            xa = xp;
            ya = yp;
            moved = true;
          }
          for (;;) {  // right end point on or below the chord (left end, its successor)?
            int ln = lb, in = ib;
            v.next(ln, in, ge);
            if (ln < 0) break;
            const float xn = v.xs(ln * c + in), yn = v.val(ln * c + in);
            if (!below_chord(ya, yb, yn, xa, xb, xn)) break;
            lb = ln;
            ib = in;
            xb = xn;
            yb = yn;
            moved = true;
          }
        }
        v.hi[la] = ia + 1;
        for (int q = la + 1; q < gm; ++q) v.hi[q] = v.lo[q];
        for (int q = gm; q < lb; ++q) v.hi[q] = v.lo[q];
        v.lo[lb] = ib;
      }
    }
    __syncwarp();
  }

  // 3. read-out: vertex q of the envelope lies in the last lane whose
  // exclusive prefix of kept counts is <= q (empty lanes share the prefix of
  // the next non-empty one, so that lane is never empty)
  const int kept = v.hi[lane] - v.lo[lane];
  int pre = kept;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int t = __shfl_up_sync(0xffffffffu, pre, o);
    if (lane >= o) pre += t;
  }
  const int total = __shfl_sync(0xffffffffu, pre, 31);
  s_pre[w][lane] = pre - kept;
  if (lane == 0) p.n_bp[h] = total;
  __syncwarp();
  auto position = [&](int q) {  // stack position of vertex q
    int L = 0;
#pragma unroll
    for (int step = 16; step > 0; step >>= 1)
      if (s_pre[w][L + step] <= q) L += step;
    return L * c + v.lo[L] + q - s_pre[w][L];
  };
  if constexpr (kStaged) {
    for (int q = lane; q < total; q += 32) {
      const int pa = position(q);
      const float xa = v.xs(pa);
      row[q] = v.xi(pa);
      if (q + 1 < total) {
        const int pb = position(q + 1);
        sl[q] = hull_slope(xa, v.sv[pa], v.xs(pb), v.sv[pb], p.delta);
      }
    }
  } else {
    for (int q = lane; q < total; q += 32) row[q] = v.xi(position(q));
    __syncwarp();  // the slope row held the stacks
    for (int q = lane; q + 1 < total; q += 32) {
      const int a = row[q], b = row[q + 1];
      sl[q] = hull_slope((float)a, v.point(a), (float)b, v.point(b), p.delta);
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

// offsets[h] = sum of n_bp[0 .. h), offsets[n_h] = total: one block of 1024
// threads walks the counts in chunks, each chunk scanned by warp shuffles
// and a scan of the 32 warp sums, plus the running carry.
__global__ void __launch_bounds__(1024) offsets_kernel(const int* n_bp, int n_h,
                                                       long long* offsets) {
  __shared__ long long s_warp[32];
  __shared__ long long s_carry;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_carry = 0;
  __syncthreads();
  for (int base = 0; base < n_h; base += 1024) {
    const int i = base + threadIdx.x;
    const long long v = i < n_h ? n_bp[i] : 0;
    long long x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const long long y = __shfl_up_sync(0xffffffffu, x, o);
      if (lane >= o) x += y;
    }
    if (lane == 31) s_warp[w] = x;
    __syncthreads();
    if (w == 0) {
      long long z = s_warp[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const long long y = __shfl_up_sync(0xffffffffu, z, o);
        if (lane >= o) z += y;
      }
      s_warp[lane] = z;  // inclusive scan of the warp sums
    }
    __syncthreads();
    const long long carry = s_carry;
    const long long excl = carry + (w ? s_warp[w - 1] : 0) + x - v;
    if (i < n_h) offsets[i] = excl;
    __syncthreads();
    if (threadIdx.x == 1023) s_carry = excl + v;
    __syncthreads();
  }
  if (threadIdx.x == 0) offsets[n_h] = s_carry;
}

// one warp per envelope: its vertices and slopes from the padded rows to
// [offsets[h], offsets[h+1]) of the packed arrays (the envelope's last slot
// of `slope` is 0); nothing at or beyond cap is written
__global__ void pack_kernel(const int* n_bp, const int* idx, const float* slope, int N, int n_h,
                            const long long* offsets, long long cap, int* idx_out,
                            float* slope_out) {
  const int h = (int)((blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5);
  const int lane = threadIdx.x & 31;
  if (h >= n_h) return;
  const int n = n_bp[h];
  const long long o = offsets[h];
  const int* row = idx + (size_t)h * N;
  const float* sl = slope + (size_t)h * N;
  for (int j = lane; j < n; j += 32) {
    const long long d = o + j;
    if (d >= cap) break;
    idx_out[d] = row[j];
    slope_out[d] = j + 1 < n ? sl[j] : 0.f;
  }
}

}  // namespace

cudaError_t launch_hull(const HullParams& p, cudaStream_t stream) {
  const int n_h = p.n_t * p.M * p.K;
  if (n_h == 0) return cudaSuccess;
  const size_t per_warp = (size_t)p.N * 6;  // staged values and 16-bit stack indices
  int lg = 3;
  while (lg > 0 && (per_warp << lg) > (size_t)kHullSmemBudget) --lg;
  if (p.N <= 65536 && (per_warp << lg) <= (size_t)kHullSmemBudget) {
    const int nw = 1 << lg, smem = (int)(per_warp << lg);
    cudaError_t e = cudaFuncSetAttribute(hull_kernel<true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    hull_kernel<true><<<(n_h + nw - 1) / nw, 32 * nw, smem, stream>>>(p, lg);
  } else {
    hull_kernel<false><<<(n_h + kHullWarps - 1) / kHullWarps, 32 * kHullWarps, 0, stream>>>(p, 3);
  }
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

cudaError_t launch_pack_bids(const int* n_bp, const int* idx, const float* slope, int N, int n_h,
                             long long* offsets, long long cap, int* idx_out, float* slope_out,
                             cudaStream_t stream) {
  offsets_kernel<<<1, 1024, 0, stream>>>(n_bp, n_h, offsets);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess || n_h == 0) return e;
  const int warps_per_block = 8;
  pack_kernel<<<(n_h + warps_per_block - 1) / warps_per_block, 32 * warps_per_block, 0, stream>>>(
      n_bp, idx, slope, N, n_h, offsets, cap, idx_out, slope_out);
  return cudaGetLastError();
}

}  // namespace esdp

