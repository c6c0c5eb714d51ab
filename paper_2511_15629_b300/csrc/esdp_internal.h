// Internal structures shared by the host library and the kernels.
#pragma once

#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <cuda_runtime.h>

namespace esdp {

// Rows of the SoC grid a thread owns in the banded max-plus (its register
// window), one launch uses one value.
constexpr int kRowsPerThreadChoices[] = {4, 6, 8, 9, 10, 12};
constexpr int kMaxBlock = 512;
constexpr int kMaxWaits = 64;     // neighbour tiles a work item may wait on

// Per-asset parameters of one sweep launch (device-resident array).
struct AssetDev {
  int T, N, K, A, D_dis, D_chg, M;
  int policy_bytes;     // 0, 2, 4
  int nb;               // row blocks (of R rows) per tile
  int parts;            // the action chunks are split over this many thread groups
  int W;                // rows per tile = nb * R
  int n_tiles;
  int flag_base;        // first flag of this asset
  int wait_lo, wait_hi; // neighbour tiles [tile+wait_lo, tile+wait_hi] read our rows / we read theirs
  int t_hi, t_lo;       // stages swept: t_hi down to t_lo
  int ev_keep;          // 1: EV_t at ev + (t-1)*MNK; 0: double buffer ev + (t&1)*MNK
  int policy_t_base;    // policy of stage t at policy + (t - policy_t_base)*MNK
  int ckpt_every;       // > 0: V_t with (t-1) % C == 0, t > 1 -> ckpt[(t-1)/C - 1]
  int rows;             // EV tile rows in shared memory: W + A + R
  int rs;               // row stride of the payoff table (odd)
  float sw;             // switch cost
  // offsets into the launch's concatenated inputs (elements)
  long long off_price, off_trans, off_cost, off_terminal, off_v1;
  const float* e;       // [A] grid energy of each action (device)
  const float* v_start; // V_{t_hi+1} [M][N][K]; nullptr -> terminal input
  float* ev;            // EV buffers [*][M][N][K]
  void* policy;         // policy buffers or nullptr
  float* v_keep;        // V_t, t in [t_lo, t_hi], at (t - t_lo); or nullptr
  float* ckpt;          // checkpoints or nullptr
  // Level offsets.  The float32 working values are V'_t = V_t - c_t with a
  // scalar c_t per stage carried in double: c_t = c_{t+1} + EV'_t[ref].
  // EV_t = EV'_t + c_{t+1} rho_t[k] with rho_t[k] the row sums of P_t.
  int ref_tile;         // tile holding the reference row
  int ref_row;          // reference SoC row (mode 0, price state 0)
  float* ref_hist;      // [T+2]: EV'_t[0][ref_row][0] of every stage (one slot per stage)
  double* rho;          // [T][K] row sums of trans (double)
  double* off;          // [T+2]: off[t] = c_t (written by tile 0)
  double* evoff;        // [T][K]: EV_t - EV'_t = c_{t+1} rho_t[k] (written by tile 0)
  const double* c_start;  // c_{t_hi+1}, or nullptr for 0
  float* ptrans;        // prepared P_t per stage (prep kernel), or nullptr: with tc == 0
                        // [T][K][p_stride(K)] transposed and padded; with tc == 1
                        // [T][2][K*K] tf32 hi and lo parts in the tensor-core operand layout
  int tc;               // 1: EV contraction on tcgen05 (K a multiple of 16, ptrans prepared)
  int mma;              // 1: EV contraction on mma.sync m16n8k8 (K a multiple of 8, tc == 0)
};

// The EV contraction on tcgen05 (64-row MMAs with N = K, k-steps of 8) is
// built for K a multiple of 16 up to 128 (tensor-memory columns, operand
// layouts) and needs the prepared operand copy of P.
__host__ __device__ inline bool tc_shape(int K) { return K >= 16 && K <= 128 && (K & 15) == 0; }

// Unit that contracts EV_{t-1} = P_{t-1} V_t over the rows of a tile of W
// rows x M modes x K states (W M K^2 multiply-adds per stage).  The tensor
// paths repay their fixed cost (the tf32 operand split, MMA issue and
// completion, the read-back) only on large contractions with many states:
// on B300, FP32 SIMT was the faster for 16-row tiles at K = 16..64
// (W M K^2 <= 65,536, by 4-11 %) and for the 256-asset batch with K = 8..40
// on tiles of up to hundreds of rows (by 1.5 %), tcgen05 for 36-row tiles at
// K = 64 (147,456, by 8 %; mma.sync 2.6 % ahead of SIMT there).  So tiles
// with K >= 64 and from 98,304 multiply-adds take tcgen05 (K a multiple of
// 16) or mma.sync (K a multiple of 8).  `force`: 0 automatic; 1 SIMT,
// 2 tcgen05, 3 mma.sync where K allows it (else SIMT).
enum EvPath { kEvSimt = 0, kEvTc = 1, kEvMma = 2 };

// The `force` argument from the environment: ESDP_EV = "simt" | "tc" | "mma"
// pins a path (so that every path can be exercised on small grids); unset or
// any other value leaves the choice to the tile size.
inline int ev_force() {
  const char* f = std::getenv("ESDP_EV");
  if (!f) return 0;
  if (!std::strcmp(f, "simt")) return 1;
  if (!std::strcmp(f, "tc")) return 2;
  if (!std::strcmp(f, "mma")) return 3;
  return 0;
}
constexpr long long kTensorEvMinWork = 98304;
constexpr int kTensorEvMinK = 64;
inline int ev_path(int W, int M, int K, int force) {
  const bool tc_ok = tc_shape(K), mma_ok = (K & 7) == 0;
  if (force == 1) return kEvSimt;
  if (force == 2) return tc_ok ? kEvTc : kEvSimt;
  if (force == 3) return mma_ok ? kEvMma : kEvSimt;
  if (K < kTensorEvMinK || (long long)W * M * K * K < kTensorEvMinWork) return kEvSimt;
  return tc_ok ? kEvTc : (mma_ok ? kEvMma : kEvSimt);
}

// Offset (floats) of element (r, k) of a [rows x KK] tcgen05 operand in the
// K-major, unswizzled canonical layout: 8-row x 16-byte core matrices, the
// KK/4 core matrices of one 8-row group `cm` floats apart (leading byte
// offset 4 * cm), the 8-row groups KK/4 * cm floats apart (stride byte
// offset).  cm = 32 packs them (the prepared B operand); cm = 36 leaves a
// 16-byte gap that puts the 32 states of one row in 32 distinct banks (the A
// operand, written row by row by the sweep).
constexpr int kCmB = 32, kCmA = 36;
__host__ __device__ inline int tc_offset(int r, int k, int KK, int cm) {
  return (r >> 3) * (KK >> 2) * cm + (k >> 2) * cm + (r & 7) * 4 + (k & 3);
}

struct WorkItem {
  int asset, tile, s0, s1;  // rows [s0, s1) of the asset's SoC grid
};

struct SweepParams {
  const AssetDev* assets;
  const WorkItem* items;
  const int* cta_items;      // [grid + 1] prefix offsets into items
  const float* price;        // concatenated inputs
  const float* trans;
  const float* cost;
  const float* terminal;
  float* v1;                 // concatenated V_1 output or nullptr
  int n_steps;               // max over assets of t_hi - t_lo + 1
  int* flags;                // one per (asset, tile), zero at launch
  int* status;               // 0 or an ESDP_E* code
  unsigned long long timeout_ns;
  int wait_extra;            // 0; > 0 only in the stall test: waits for a value nobody publishes
  double* item_c;            // [items] running level c of each work item
  // shared-memory carve-up (floats), see sweep_smem_layout
  int sm_E, sm_R, sm_C, sm_V, sm_P, sm_X;
  int sm_A, sm_A2;           // tcgen05 A operand (V' split into tf32 hi and lo parts)
  int tmem_cols;             // tensor-memory columns of the EV accumulator (0: none)
  // per-CTA phase cycle sums [grid][kPhases + 1] (the last slot counts the
  // stages), written only by a library built with ESDP_PHASE_CLOCKS
  unsigned long long* phase_clk;
};

// Phases of one stage of one work item, as the per-phase clock counters of
// an ESDP_PHASE_CLOCKS build split it (cycles of thread 0 of the CTA).
constexpr int kPhases = 8;

// Row strides of the V' tile and of the transposed transition matrix in
// shared memory (and of the prepared transposed copy in global memory),
// padded so that tensor-core fragment loads and float4 reads are free of bank
// conflicts.
__host__ __device__ inline int v_stride(int K) { return K + 4; }
__host__ __device__ inline int p_stride(int K) { return ((K + 3) & ~3) + 8; }

// Shared-memory carve-up of the sweep kernel (offsets in floats, every region
// 128-byte aligned so that bulk copies and float4 accesses are aligned).
// With the tensor-core EV (tc), the two A operand parts come first: each
// holds the tile's M*W rows (rounded up to 8); a 64-row MMA reads past them
// into the regions that follow (rows it computes but nobody stores), so the
// carve-up extends at least whole 64-row blocks past the second part.
struct SweepSmem {
  int A, A2, E, Rt, C, V, P, X;
  size_t bytes;
};
inline SweepSmem sweep_smem_layout(int M, int K, int W, int A, int R, bool tc) {
  auto al = [](long long x) { return (int)((x + 31) / 32 * 32); };
  const int rows = W + A + R, rs = (A + 2 * R) | 1;
  const int mw8 = (M * W + 7) / 8 * 8, mw64 = (M * W + 63) / 64 * 64;
  SweepSmem s;
  const long long apart = (long long)(mw8 / 8) * (K / 4) * kCmA;  // A part (floats)
  s.A = 0;
  s.A2 = s.A + (tc ? al(apart) : 0);
  s.E = s.A2 + (tc ? al(apart) : 0);
  s.Rt = s.E + al((long long)M * rows * (K + (K & 1)));
  s.C = s.Rt;  // no payoff table: the payoffs are formed in registers
  s.V = s.C + al(2LL * M * rs);
  s.P = s.V + al((long long)M * W * v_stride(K));
  s.X = s.P + al(tc ? 2LL * K * K : (long long)K * p_stride(K));
  long long end = s.X + al((long long)M * W * K);  // argmax indices
  const long long foot = (long long)(mw64 / 8) * (K / 4) * kCmA;  // read by the 64-row blocks
  if (tc && end < (long long)s.A2 + foot) end = (long long)s.A2 + foot;
  s.bytes = (size_t)end * sizeof(float);
  return s;
}

// Threads of the max-plus phase: cells (price-state pairs x row blocks x
// modes) laid out over warps of 32/G cell slots x G action parts.
inline int maxplus_threads(int cells, int G) {
  const int L = 32 / G;
  return (cells + L - 1) / L * 32;
}

// The action split: the largest power of two G <= 32, at most half the
// chunks of R actions, whose max-plus threads fit the block; 0 if none does.
inline int pick_parts(int cells, int block, int chunks) {
  for (int G = 32; G >= 1; G >>= 1)
    if (G <= (chunks / 2 > 1 ? chunks / 2 : 1) && maxplus_threads(cells, G) <= block) return G;
  return 0;
}

// Launch shape of one sweep.
struct SweepShape {
  int R = 8;
  int kh = 0;       // 32: every asset has K = 63 or 64 (the kernel variant with a fixed EV row
                    // stride); -1: the variant with the paths only batches need (EV tiles of K
                    // not a multiple of 4 copied eight loads at a time, one-part recovery of both
                    // states per row), so that the other launches keep their code unchanged
  int block = 256;
  int grid = 0;
  size_t smem = 0;
};

cudaError_t launch_sweep(const SweepShape& shape, const SweepParams& p, cudaStream_t stream);
int sweep_max_blocks_per_sm(int R, int kh, int block, size_t smem);
// The kernel variant for a launch's assets: 32 when every asset has
// ceil(K / 2) = 32 price-state pairs, else 0 (row stride read at run time).
template <typename It>
inline int sweep_kh(It first, It last) {
  if (first == last) return 0;
  for (It i = first; i != last; ++i)
    if ((i->K + 1) / 2 != 32) return 0;
  return 32;
}
// Instance preparation for a launch: row sums (double) of every transition
// matrix and, where the asset has a buffer for it, the transposed padded copy
// ptrans[t][k2][k] = trans[t][k][k2].
cudaError_t launch_rowsums(const AssetDev* d_assets, int n_assets, int max_rows, const float* trans,
                           cudaStream_t stream);
// Bid-curve envelope kernel.
struct HullParams {
  const float* ev;   // EV_t of stage t0 at ev, stage stride MNK, layout [M][N][K]
  int n_t, M, N, K;
  double delta;      // SoC step (MWh): slopes in $ per MWh
  int* n_bp;         // [n_t][M][K]
  int* idx;          // [n_t][M][K][N]
  float* slope;      // [n_t][M][K][N]
};
cudaError_t launch_hull(const HullParams& p, cudaStream_t stream);
// Packed form of the bid curves: offsets[n_h + 1] (exclusive prefix of n_bp),
// then each envelope's vertices and slopes copied to [offsets[h], offsets[h+1])
// of idx_out / slope_out (entries at or beyond cap are not written).
cudaError_t launch_pack_bids(const int* n_bp, const int* idx, const float* slope, int N, int n_h,
                             long long* offsets, long long cap, int* idx_out, float* slope_out,
                             cudaStream_t stream);
// Price-quantity bids at SoC index s from the envelopes of the bid-curve
// kernel (one thread per (stage, mode, price state)).
struct BidsAtParams {
  const float* ev;      // reported EV_t of stage t0 at ev, stage stride MNK, layout [M][N][K]
  const int* n_bp;      // [n_t][M][K] envelope vertex counts
  const int* idx;       // [n_t][M][K][N] envelope vertex indices
  int n_t, M, N, K, s, D_dis, D_chg, A;
  double delta, eta_c, eta_d, tau;
  int* n_pts;           // [n_t][M][K] out
  double* p_mw;         // [n_t][M][K][A] out
  float* price;         // [n_t][M][K][A] out (first n_pts - 1 used)
};
cudaError_t launch_bids_at(const BidsAtParams& p, cudaStream_t stream);
// Kept EV'_t of n_t stages -> reported EV_t = float(EV'_t + evoff_t[k]), in place.
cudaError_t launch_ev_restore(float* ev, const double* evoff, int n_t, int MN, int K,
                              cudaStream_t stream);

// Occupancy adjoint kernels.
struct OccParams {
  int N, K, M, A, D_dis, t_lo, t_hi;
  int grid_rows;          // rows (m*N + s) per CTA
  double delta, eta_c, eta_d;
  float sw;
  const float* price;     // [T][K] of this asset
  const float* trans;     // [T][K][K]
  const float* cost;      // [A]
  const float* e;         // [A]
  const void* policy;     // stages t_lo..t_hi, [C][M][N][K]
  int policy_bytes;
  float* rho;             // [M][N][K], holds rho_{t_lo} on entry, rho_{t_hi+1} on exit
  float* post;            // [C][M][N][K], written by the kernel
  unsigned long long* post_fx;  // [C][M][N][K] the scatter's fixed-point sums, zero on entry
  float fx_e;             // fixed-point scale (a power of two) of the rho * e_a terms
  int own_smem;           // set by the launcher: own converted and occupancy rows in shared memory
  int n_cost_copies;      // set by the launcher: copies of the shared per-action cost sums
  double* d_price;        // [T][K] (accumulated)
  double* acc;            // [5]: d_eta_c, d_eta_d, (two unused slots), d_switch
  double* d_cost;         // [A] (accumulated)
  long long* part;        // [C][grid][K] per-CTA stage partials of dprice (fixed point, fx_e units)
  double* part_cost;      // [grid][A] per-CTA segment partials of d_cost
  double* part_acc;       // [grid][8] per-CTA segment partials of acc
  int* flags;             // [grid] last stage whose scatter each CTA published (zero on entry)
  int* status;
  unsigned long long timeout_ns;
};
cudaError_t launch_occupancy(const OccParams& p, int grid, int block, cudaStream_t stream);
// Adds the per-CTA partials of a segment (grid CTAs, stages t_lo..t_hi) to
// d_price, acc and d_cost, summing in a fixed order.
cudaError_t launch_occ_reduce(const OccParams& p, int grid, cudaStream_t stream);

struct DTransParams {
  int n_t, MN, K;
  const float* post;    // [n_t][MN][K]
  const float* vnext;   // V'_{t+1} of stage ts (0-based) at vnext + (ts / seg_len) * seg_stride
                        // + (ts % seg_len) * MN * K (segments of seg_len stages)
  int seg_len;
  long long seg_stride;
  const double* cnext;  // [n_t]: c_{t+1}, V_{t+1} = V'_{t+1} + c_{t+1}
  float* d_trans;       // [n_t][K][K]
  int n_split;          // row ranges per (stage, tile)
  double* part;         // [n_t][n_split][K][K] row-range partial sums (scratch)
  double* part_mass;    // [n_t][n_split][K] row-range occupancy masses (scratch)
};
constexpr int kDtSplit = 4;  // row ranges of the dJ/dP reduction
cudaError_t launch_dtrans(const DTransParams& p, cudaStream_t stream);

}  // namespace esdp
