// Register-only issue-rate probe of the float32 instructions the max-plus
// loop is built from: scalar add, packed add (add.rn.f32x2), two- and
// three-input max, and the loop's own mix (two packed adds and two
// three-input maxima per four evaluations).  Each thread runs eight
// independent chains of inline-asm instructions (volatile, so none is merged
// or removed); a block of 1024 threads times its loop with clock64 between two
// barriers, which gives instructions and element operations per SM clock.
// The evaluation ceiling used in the roofline (128 lanes x 1 op per clock,
// two ops per evaluation) is checked against these rates.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "esdp.h"

namespace {

constexpr int kProbeThreads = 1024;
constexpr int kChains = 8;

__device__ __forceinline__ void op_add(float& a, float x) {
  asm volatile("add.rn.f32 %0, %0, %1;" : "+f"(a) : "f"(x));
}
__device__ __forceinline__ void op_add2(unsigned long long& a, unsigned long long x) {
  asm volatile("add.rn.f32x2 %0, %0, %1;" : "+l"(a) : "l"(x));
}
__device__ __forceinline__ void op_max(float& a, float x) {
  asm volatile("max.f32 %0, %0, %1;" : "+f"(a) : "f"(x));
}
__device__ __forceinline__ void op_max3(float& a, float x, float y) {
  asm volatile("max.f32 %0, %0, %1, %2;" : "+f"(a) : "f"(x), "f"(y));
}
// one step of the max-plus pattern for a pair of price states and two
// actions: s = r0 + w0, u = r1 + w1 (packed), then m.x = max(m.x, s.x, u.x),
// m.y = max(m.y, s.y, u.y)
__device__ __forceinline__ void op_eval4(float& mx, float& my, unsigned long long r0,
                                         unsigned long long w0, unsigned long long r1,
                                         unsigned long long w1) {
  asm volatile(
      "{\n\t.reg .b64 s, u;\n\t.reg .f32 sx, sy, ux, uy;\n\t"
      "add.rn.f32x2 s, %2, %3;\n\t"
      "add.rn.f32x2 u, %4, %5;\n\t"
      "mov.b64 {sx, sy}, s;\n\t"
      "mov.b64 {ux, uy}, u;\n\t"
      "max.f32 %0, %0, sx, ux;\n\t"
      "max.f32 %1, %1, sy, uy;\n\t}"
      : "+f"(mx), "+f"(my)
      : "l"(r0), "l"(w0), "l"(r1), "l"(w1));
}

__device__ __forceinline__ unsigned long long pack(float a, float b) {
  return (unsigned long long)__float_as_uint(a) | ((unsigned long long)__float_as_uint(b) << 32);
}

// out[0 .. gridDim.x): cycles of each block's timed loop; sink keeps results
__global__ void __launch_bounds__(kProbeThreads) alu_probe_kernel(int kind, int iters,
                                                                  long long* cycles, float* sink) {
  const float x = 1e-7f * (float)(threadIdx.x + 1), y = 2e-7f * (float)(blockIdx.x + 1);
  float a[kChains], b[kChains];
  unsigned long long p[kChains];
#pragma unroll
  for (int i = 0; i < kChains; ++i) {
    a[i] = x * (float)(i + 1);
    b[i] = y * (float)(i + 2);
    p[i] = pack(a[i], b[i]);
  }
  const unsigned long long px = pack(x, y), py = pack(y, x);
  __syncthreads();
  const long long t0 = clock64();
  switch (kind) {
    case 0:
      for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) op_add(a[i], x);
      break;
    case 1:
      for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) op_add2(p[i], px);
      break;
    case 2:
      for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) op_max(a[i], b[i]);
      break;
    case 3:
      for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; ++i) op_max3(a[i], b[i], x);
      break;
    default:
      for (int it = 0; it < iters; ++it)
#pragma unroll
        for (int i = 0; i < kChains; i += 2) op_eval4(a[i], a[i + 1], p[i], px, p[i + 1], py);
      break;
  }
  __syncthreads();
  const long long t1 = clock64();
  if (threadIdx.x == 0) cycles[blockIdx.x] = t1 - t0;
  float s = 0.f;
#pragma unroll
  for (int i = 0; i < kChains; ++i)
    s += a[i] + __uint_as_float((unsigned)p[i]) + __uint_as_float((unsigned)(p[i] >> 32));
  if (s == 12345.678f) sink[threadIdx.x] = s;  // practically never: keeps the chains live
}

}  // namespace

// Instructions and element operations per SM clock, median over one block
// per SM.  kind: 0 add.f32, 1 add.rn.f32x2, 2 max.f32, 3 three-input max.f32,
// 4 the max-plus mix (elements = evaluations).
extern "C" int esdp_alu_probe(int32_t kind, int32_t iters, double* instr_per_clk,
                              double* elem_per_clk, void* stream) {
  if (kind < 0 || kind > 4 || iters < 1 || !instr_per_clk || !elem_per_clk) return ESDP_EINVAL;
  int dev = 0, n_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return ESDP_ECUDA;
  long long* d_cyc = nullptr;
  float* d_sink = nullptr;
  if (cudaMalloc(&d_cyc, sizeof(long long) * n_sm) != cudaSuccess) return ESDP_ENOMEM;
  if (cudaMalloc(&d_sink, sizeof(float) * kProbeThreads) != cudaSuccess) {
    cudaFree(d_cyc);
    return ESDP_ENOMEM;
  }
  cudaStream_t st = (cudaStream_t)stream;
  alu_probe_kernel<<<n_sm, kProbeThreads, 0, st>>>(kind, iters, d_cyc, d_sink);
  std::vector<long long> cyc(n_sm);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(cyc.data(), d_cyc, sizeof(long long) * n_sm, cudaMemcpyDeviceToHost, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  cudaFree(d_cyc);
  cudaFree(d_sink);
  if (e != cudaSuccess) return ESDP_ECUDA;
  std::sort(cyc.begin(), cyc.end());
  const double c = (double)cyc[n_sm / 2];
  // instructions per loop iteration: kChains (kinds 0-3), or kChains / 2
  // steps of four instructions (kind 4); elements: two per packed add and per
  // three-input max, one evaluation per instruction of the mix
  const double n_instr = (double)kProbeThreads * iters * (kind == 4 ? 2.0 * kChains : kChains);
  const double n_elem = (kind == 1 || kind == 3) ? 2.0 * n_instr : n_instr;
  *instr_per_clk = n_instr / c;
  *elem_per_clk = n_elem / c;
  return ESDP_OK;
}
