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
// cooperative launch (one bounded grid barrier per stage, between the scatter
// and the contraction); dtrans_kernel then forms dJ/dP for the segment from
// the stored post-decision occupancies and values.
#include <cuda_runtime.h>

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

__device__ bool grid_barrier(int* bar, int target, int* status, unsigned long long timeout,
                             int* s_abort) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1);
    const unsigned long long t0 = now_ns();
    while (ld_acquire(bar) < target) {
      if (*(volatile int*)status != 0) {
        *(volatile int*)s_abort = 1;
        break;
      }
      if (now_ns() - t0 > timeout) {
        atomicCAS(status, 0, ESDP_ETIMEOUT);
        *(volatile int*)s_abort = 1;
        break;
      }
    }
    __threadfence();
  }
  __syncthreads();
  return *(volatile int*)s_abort == 0;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void __launch_bounds__(256) occ_kernel(const OccParams p) {
  extern __shared__ double osm[];
  double* sk = osm;                                          // [K] dprice partials, then [5]
  double* sc = osm + p.K + 5;                                // [A] cost partials (segment)
  float* Ps = reinterpret_cast<float*>(osm + p.K + 5 + p.A);  // [K][K]
  __shared__ int s_abort;
  const int K = p.K, N = p.N, M = p.M, MN = M * N;
  const size_t MNK = (size_t)MN * K;
  const int tid = threadIdx.x, nth = blockDim.x;
  const int r0 = blockIdx.x * p.grid_rows;
  const int r1 = min(MN, r0 + p.grid_rows);
  if (tid == 0) s_abort = 0;
  for (int a = tid; a < p.A; a += nth) sc[a] = 0.0;
  __syncthreads();
  int epoch = 0;
  for (int t = p.t_lo; t <= p.t_hi; ++t) {
    const int ts = t - p.t_lo;
    for (int i = tid; i < K + 5; i += nth) sk[i] = 0.0;
    __syncthreads();
    float* post = p.post + (size_t)ts * MNK;
    const float* price_t = p.price + (size_t)(t - 1) * K;
    double dc = 0.0, dd = 0.0, jr = 0.0, ms = 0.0, dsw = 0.0;
    for (int i = r0 * K + tid; i < r1 * K; i += nth) {
      const float rho = p.rho[i];
      if (rho == 0.f) continue;
      const int row = i / K, k = i - row * K;
      const int m = row / N, s = row - m * N;
      const size_t pi = (size_t)ts * MNK + i;
      const int a = p.policy_bytes == 2 ? (int)reinterpret_cast<const short*>(p.policy)[pi]
                                        : reinterpret_cast<const int*>(p.policy)[pi];
      const int d = a - p.D_dis;
      if (a < 0 || a >= p.A || s + d < 0 || s + d >= N) {  // not a feasible stored action
        atomicCAS(p.status, 0, ESDP_ENUMERIC);
        continue;
      }
      const int m2 = (M == 2) ? (d < 0 ? 0 : (d > 0 ? 1 : m)) : 0;
      atomicAdd(post + ((size_t)m2 * N + s + d) * K + k, rho);
      const double lam = (double)price_t[k];
      const double e = (double)p.e[a];
      atomicAdd(&sk[k], (double)rho * e);
      if (d > 0) dc += (double)rho * lam * ((double)d * p.delta / (p.eta_c * p.eta_c));
      if (d < 0) dd += (double)rho * lam * (-(double)d * p.delta);
      double r = lam * e - (double)p.cost[a];
      atomicAdd(&sc[a], -(double)rho);
      if (M == 2 && m == 1 && d < 0) {
        r -= (double)p.sw;
        dsw -= (double)rho;
      }
      jr += (double)rho * r;
      ms += (double)rho;
    }
    dc = warp_sum(dc);
    dd = warp_sum(dd);
    jr = warp_sum(jr);
    ms = warp_sum(ms);
    dsw = warp_sum(dsw);
    if ((tid & 31) == 0) {
      atomicAdd(&sk[K + 0], dc);
      atomicAdd(&sk[K + 1], dd);
      atomicAdd(&sk[K + 2], jr);
      atomicAdd(&sk[K + 3], ms);
      atomicAdd(&sk[K + 4], dsw);
    }
    __syncthreads();
    for (int k = tid; k < K; k += nth)
      if (sk[k] != 0.0) atomicAdd(&p.d_price[(size_t)(t - 1) * K + k], sk[k]);
    if (tid < 5 && sk[K + tid] != 0.0) atomicAdd(&p.acc[tid], sk[K + tid]);
    if (t == p.t_hi)  // the segment's cost partials, once
      for (int a = tid; a < p.A; a += nth)
        if (sc[a] != 0.0) atomicAdd(&p.d_cost[a], sc[a]);
    ++epoch;
    if (!grid_barrier(p.bar, epoch * (int)gridDim.x, p.status, p.timeout_ns, &s_abort)) return;
    // contraction of the post-decision occupancy with P_t (own rows)
    const float* P = p.trans + (size_t)(t - 1) * K * K;
    for (int i = tid; i < K * K; i += nth) Ps[i] = P[i];
    __syncthreads();
    for (int i = r0 * K + tid; i < r1 * K; i += nth) {
      const int row = i / K, k2 = i - row * K;
      const float* pr = post + (size_t)row * K;
      float acc = 0.f;
      for (int k = 0; k < K; ++k) acc = fmaf(__ldcg(pr + k), Ps[k * K + k2], acc);
      p.rho[i] = acc;
    }
    __syncthreads();
  }
}

__global__ void dtrans_kernel(const DTransParams p) {
  const int K = p.K;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  const int ts = blockIdx.y;
  if (e >= K * K) return;
  const int k = e / K, k2 = e - k * K;
  const float* post = p.post + (size_t)ts * p.MN * K;
  const float* v = p.vnext + (size_t)ts * p.MN * K;
  // V_{t+1} = V'_{t+1} + c_{t+1}: sum post * V' plus c_{t+1} times the mass
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float mass[4] = {0.f, 0.f, 0.f, 0.f};
  int row = 0;
  for (; row + 4 <= p.MN; row += 4) {
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const float w = __ldg(post + (size_t)(row + u) * K + k);
      if (w != 0.f) {
        acc[u] = fmaf(w, __ldg(v + (size_t)(row + u) * K + k2), acc[u]);
        mass[u] += w;
      }
    }
  }
  for (; row < p.MN; ++row) {
    const float w = __ldg(post + (size_t)row * K + k);
    if (w != 0.f) {
      acc[0] = fmaf(w, __ldg(v + (size_t)row * K + k2), acc[0]);
      mass[0] += w;
    }
  }
  const double sv = ((double)acc[0] + (double)acc[1]) + ((double)acc[2] + (double)acc[3]);
  const double sm = ((double)mass[0] + (double)mass[1]) + ((double)mass[2] + (double)mass[3]);
  p.d_trans[(size_t)ts * K * K + e] = (float)(sv + p.cnext[ts] * sm);
}

}  // namespace

cudaError_t launch_occupancy(const OccParams& p, int grid, int block, cudaStream_t stream) {
  const size_t smem =
      (size_t)(p.K + 5 + p.A) * sizeof(double) + (size_t)p.K * p.K * sizeof(float);
  cudaError_t e = cudaFuncSetAttribute(occ_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)smem);
  if (e != cudaSuccess) return e;
  OccParams pp = p;
  void* args[] = {&pp};
  return cudaLaunchCooperativeKernel((const void*)occ_kernel, dim3(grid), dim3(block), args, smem,
                                     stream);
}

cudaError_t launch_dtrans(const DTransParams& p, cudaStream_t stream) {
  if (p.n_t == 0) return cudaSuccess;
  const int block = 256;
  dim3 grid((p.K * p.K + block - 1) / block, p.n_t);
  dtrans_kernel<<<grid, block, 0, stream>>>(p);
  return cudaGetLastError();
}

}  // namespace esdp
