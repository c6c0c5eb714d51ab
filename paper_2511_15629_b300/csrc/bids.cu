// Price-quantity bids at one SoC state from the SoC envelopes of the Markov
// sweep (eq. 8-11).  The envelope of EV_t[m][.][k] over the SoC grid (the
// vertices of the bid-curve kernel) is read inside the action window
// [s - D_dis, s + D_chg]; its vertices there, the window's two ends and s
// itself are mapped to grid power -- selling (x <= s) delivers
// (s - x) delta eta_d MWh, buying (x > s) takes (x - s) delta / eta_c MWh
// (eq. 2 with separate efficiencies) -- and the upper concave envelope of
// U(p) = E(x(p)) over power is taken with a monotone chain in double
// precision.  Each side alone is already concave (a concave function of a
// linear map of p); the chain only merges segments where the two sides meet,
// which happens when the buying price g eta_c exceeds the selling price
// g / eta_d, i.e. for negative marginal values g.  Segment q then sells at
// -(U_{q+1} - U_q) / ((p_{q+1} - p_q) tau), non-decreasing in q.
//
// One thread per (stage, mode, price state); O(A log N) work each.  Every
// quantity is formed by explicit round-to-nearest double operations in the
// order the comments give, so the result is a deterministic function of the
// float32 EV values and the vertex indices.
#include <cuda_runtime.h>

#include "esdp_internal.h"

namespace esdp {
namespace {

// envelope value at grid point x: the EV value at a vertex, else the chord of
// the two vertices around x, y_a + ((y_b - y_a) (x - a)) / (b - a).  v holds
// the n >= 2 vertex indices in increasing order, v[0] = 0, v[n-1] = N - 1.
__device__ __forceinline__ double envelope_at(const float* y, int K, const int* v, int n, int x) {
  int a = 0, b = n - 1;  // first vertex >= x
  while (a < b) {
    const int mid = (a + b) >> 1;
    if (v[mid] < x)
      a = mid + 1;
    else
      b = mid;
  }
  if (v[a] == x) return (double)y[(size_t)x * K];
  const int xa = v[a - 1], xb = v[a];
  const double ya = (double)y[(size_t)xa * K], yb = (double)y[(size_t)xb * K];
  return __dadd_rn(ya, __ddiv_rn(__dmul_rn(__dsub_rn(yb, ya), (double)(x - xa)),
                                 (double)(xb - xa)));
}

// grid power (MW, positive = selling) of moving from SoC index s to x:
// (((s - x) delta) eta_d) / tau for x <= s, (((s - x) delta) / eta_c) / tau
// for x > s
__device__ __forceinline__ double power_of(const BidsAtParams& p, int x) {
  const double e = __dmul_rn((double)(p.s - x), p.delta);
  return x <= p.s ? __ddiv_rn(__dmul_rn(e, p.eta_d), p.tau)
                  : __ddiv_rn(__ddiv_rn(e, p.eta_c), p.tau);
}

__global__ void __launch_bounds__(128) bids_at_kernel(const BidsAtParams p) {
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  const int n_h = p.n_t * p.M * p.K;
  if (h >= n_h) return;
  const int K = p.K, N = p.N;
  const int k = h % K, tm = h / K;  // stage-major, then mode
  const float* y = p.ev + (size_t)tm * N * K + k;
  const int* v = p.idx + (size_t)h * N;
  const int nv = p.n_bp[h];
  double* pw = p.p_mw + (size_t)h * p.A;
  float* pr = p.price + (size_t)h * p.A;
  int* xs = reinterpret_cast<int*>(pr);  // the chain's SoC indices until the prices
  // the vertex list must be an envelope's: 2..N strictly increasing indices
  // from 0 to N-1 (else no bid, n_pts = 0, and nothing outside the row is read)
  bool ok = nv >= 2 && nv <= N && v[0] == 0 && v[nv - 1] == N - 1;
  for (int j = 1; ok && j < nv; ++j) ok = v[j] > v[j - 1];
  if (!ok) {
    p.n_pts[h] = 0;
    return;
  }

  const int s = p.s, lo = max(0, s - p.D_dis), hi = min(N - 1, s + p.D_chg);
  // vertices strictly inside (lo, hi): v[jlo .. jhi]
  int jlo = 0, jhi = nv - 1;
  {
    int a = 0, b = nv;  // first vertex > lo
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (v[mid] <= lo)
        a = mid + 1;
      else
        b = mid;
    }
    jlo = a;
    a = 0;
    b = nv;  // first vertex >= hi
    while (a < b) {
      const int mid = (a + b) >> 1;
      if (v[mid] < hi)
        a = mid + 1;
      else
        b = mid;
    }
    jhi = a - 1;
  }

  // monotone chain over ascending power (descending SoC); the two top
  // entries in registers, the stack in the output rows
  int n = 0;
  double pi = 0.0, ui = 0.0, pj = 0.0, uj = 0.0;
  auto push = [&](int x) {
    const double px = power_of(p, x), ux = envelope_at(y, K, v, nv, x);
    while (n >= 2) {
      // (U_j - U_i)(p - p_i) - (U - U_i)(p_j - p_i) > 0 keeps j
      const double cross = __dsub_rn(__dmul_rn(__dsub_rn(uj, ui), __dsub_rn(px, pi)),
                                     __dmul_rn(__dsub_rn(ux, ui), __dsub_rn(pj, pi)));
      if (cross > 0.0) break;
      --n;
      pj = pi;
      uj = ui;
      if (n >= 2) {
        pi = pw[n - 2];
        ui = envelope_at(y, K, v, nv, xs[n - 2]);
      }
    }
    pw[n] = px;
    xs[n] = x;
    ++n;
    if (n == 1) {
      pj = px;
      uj = ux;
    } else {
      pi = pj;
      ui = uj;
      pj = px;
      uj = ux;
    }
  };
  push(hi);
  bool s_done = s == hi;
  for (int j = jhi; j >= jlo; --j) {
    const int x = v[j];
    if (!s_done && s > x) {
      push(s);
      s_done = true;
    }
    if (x == s) s_done = true;
    push(x);
  }
  if (lo != hi) {
    if (!s_done && s > lo) push(s);
    push(lo);
  }
  p.n_pts[h] = n;
  // prices, in place of the indices: entry q is read before it is overwritten
  int xa = xs[0];
  double ua = envelope_at(y, K, v, nv, xa);
  for (int q = 0; q + 1 < n; ++q) {
    const int xb = xs[q + 1];
    const double ub = envelope_at(y, K, v, nv, xb);
    pr[q] = (float)__ddiv_rn(-__dsub_rn(ub, ua), __dmul_rn(__dsub_rn(pw[q + 1], pw[q]), p.tau));
    xa = xb;
    ua = ub;
  }
}

}  // namespace

cudaError_t launch_bids_at(const BidsAtParams& p, cudaStream_t stream) {
  const int n_h = p.n_t * p.M * p.K;
  if (n_h == 0) return cudaSuccess;
  bids_at_kernel<<<(n_h + 127) / 128, 128, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace esdp
