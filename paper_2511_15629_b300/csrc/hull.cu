// Convexified bid curves (Sec. II-C, eq. 10-11): for every (stage, mode,
// price state) the upper concave envelope of EV_t[m][.][k] over the SoC grid,
// i.e. the hypograph convex hull, by Andrew's monotone chain.  Its slopes are
// the monotone marginal values of stored energy from which the price-quantity
// bids are read.
//
// One thread per envelope; consecutive threads take consecutive price states,
// so every step reads one coalesced row of EV.  The orientation test is the
// exact-order double expression
//     (y_j - y_i) * (l - i) - (y_l - y_i) * (j - i)  <= 0  -> drop j
// with round-to-nearest intrinsics (no contraction), so the vertex set is a
// deterministic function of the float32 EV values.
#include <cuda_runtime.h>

#include "esdp_internal.h"

namespace esdp {
namespace {

__global__ void hull_kernel(const HullParams p) {
  const int n_h = p.n_t * p.M * p.K;
  const int h = blockIdx.x * blockDim.x + threadIdx.x;
  if (h >= n_h) return;
  const int K = p.K, N = p.N;
  const int k = h % K;
  const int tm = h / K;  // stage-major, then mode
  const float* y = p.ev + (size_t)tm * N * K + k;
  // the reported EV_t: the float32 working value plus the stage level
  const double off = p.evoff[(size_t)(tm / p.M) * K + k];
  auto Y = [&](int s) -> double { return (double)(float)((double)__ldg(y + (size_t)s * K) + off); };
  int* stack = p.idx + (size_t)h * N;
  int nh = 0;
  // the two top vertices are kept in registers
  int i_idx = 0, j_idx = 0;
  double yi = 0.0, yj = 0.0;
  for (int l = 0; l < N; ++l) {
    const double yl = Y(l);
    while (nh >= 2) {
      const double lhs = __dmul_rn(__dsub_rn(yj, yi), (double)(l - i_idx));
      const double rhs = __dmul_rn(__dsub_rn(yl, yi), (double)(j_idx - i_idx));
      if (__dsub_rn(lhs, rhs) <= 0.0) {
        --nh;  // j is on or below the chord (i, l)
        j_idx = i_idx;
        yj = yi;
        if (nh >= 2) {
          i_idx = stack[nh - 2];
          yi = Y(i_idx);
        }
      } else {
        break;
      }
    }
    stack[nh] = l;
    ++nh;
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
  p.n_bp[h] = nh;
  float* sl = p.slope + (size_t)h * N;
  for (int q = 0; q + 1 < nh; ++q) {
    const int a = stack[q], b = stack[q + 1];
    const double ya = Y(a), yb = Y(b);
    sl[q] = (float)(__ddiv_rn(__dsub_rn(yb, ya), __dmul_rn((double)(b - a), p.delta)));
  }
}

}  // namespace

cudaError_t launch_hull(const HullParams& p, cudaStream_t stream) {
  const int n_h = p.n_t * p.M * p.K;
  if (n_h == 0) return cudaSuccess;
  const int block = 128;
  hull_kernel<<<(n_h + block - 1) / block, block, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace esdp
