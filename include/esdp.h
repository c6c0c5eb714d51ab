/*
 * esdp.h -- C ABI of the B300 (sm_103a) stochastic-DP library for energy
 * storage arbitrage.
 *
 * The library solves the discretized multistage stochastic storage problem
 * by backward induction (Sec. III-B, Algorithm 1), generalised from
 * stagewise-independent price samples (eq. 14) to a Markov chain of price
 * states with per-stage transition matrices:
 *
 *   stages t = 1..T; SoC grid s = 0..N-1 with step delta = s_max/(N-1)
 *   (eq. 12); price state k = 0..K-1 with price price[t][k]; optional mode
 *   m in {0,1} (1 iff the most recent non-idle action was a charge).
 *   Action a = 0..A-1 shifts the SoC by d = a - D_dis grid steps (the integer
 *   "recombining" interior of the action grid of eq. 13), A = D_dis+D_chg+1.
 *   Grid energy (eq. 2 with separate efficiencies):
 *       e_a = -d*delta*eta_d (d < 0, discharge)   e_a = -d*delta/eta_c (d > 0)
 *   Expectation (eq. 6):  EV_t[m][s][k] = sum_k2 trans[t][k][k2] V_{t+1}[m][s][k2]
 *   Bellman step (eq. 5 over the feasible set of eq. 4, 0 <= s+d <= N-1):
 *       V_t[m][s][k] = max_a  price[t][k]*e_a - cost[a]
 *                             - switch_cost*[m==1 && d<0] + EV_t[m'][s+d][k]
 *   with m' = 0 after a discharge, 1 after a charge, m when idle; the policy
 *   is the smallest maximising a.  V_{T+1} = terminal (zero in eq. 6).
 *   Bid curves (eq. 10-11): the upper concave envelope of EV_t[m][.][k]
 *   over the SoC grid; its slopes are the monotone marginal values.
 *
 * Array layouts (row-major, float32 unless stated, per asset, assets
 * concatenated in the order given to esdp_create):
 *   price    [T][K]            trans [T][K][K]   (trans[t] maps stage t -> t+1)
 *   cost     [A]               terminal [n_modes][N][K]
 *   V1       [n_modes][N][K]   policy [n_modes][N][K] per stage (int32/int16)
 *
 * Ownership and errors: the caller owns every buffer it passes; the context
 * owns its device workspace.  Without ESDP_DEVICE_PTRS all pointers are host
 * pointers and every call blocks until its result is in host memory; with
 * it, the array arguments of esdp_solve / esdp_grad are device pointers, the
 * work is queued on `stream` (a cudaStream_t, NULL = legacy default stream)
 * and the caller must keep the input buffers alive and unchanged until the
 * last call that uses them (esdp_grad and esdp_bid_curves read them again).
 * Every function returns ESDP_OK (0) or a negative ESDP_E* code and leaves a
 * message for esdp_last_error.  A call that fails leaves the context usable
 * unless the code is ESDP_ECUDA.
 */
#ifndef ESDP_H_
#define ESDP_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ESDP_OK 0
#define ESDP_EINVAL (-1)   /* bad shape, efficiency outside (0,1], negative
                              transition entry, NaN/Inf input, bad index */
#define ESDP_ENOMEM (-2)   /* device or host allocation failed */
#define ESDP_ECUDA (-3)    /* a CUDA call failed (message has the reason) */
#define ESDP_ETIMEOUT (-4) /* a device-side wait gave up (bounded spin) */
#define ESDP_ESTATE (-5)   /* result requested before the solve that makes it,
                              or not kept by the context's flags */
#define ESDP_ENUMERIC (-6) /* the solve produced a NaN */

/* esdp_create flags */
#define ESDP_DEVICE_PTRS 1u /* array arguments are device pointers, stream-ordered */
#define ESDP_KEEP_EV 2u     /* keep EV_t of every stage (esdp_bid_curves,
                               esdp_expected_value) */
#define ESDP_CHECK_ROWS 4u  /* reject transition rows whose sum is not 1 +- 1e-5 */
#define ESDP_NO_VALIDATE 8u /* skip the host-side NaN / sign scan of inputs
                               (only meaningful with host pointers) */
#define ESDP_TIME_SWEEP 16u /* record CUDA events around the persistent sweep
                               launch of every esdp_solve (esdp_sweep_ms) */

typedef struct esdp_ctx esdp_ctx;

typedef struct {
  int32_t T, N, K, A;     /* stages, SoC points (2..2^24), price states, actions */
  int32_t D_dis, D_chg;   /* action band: shifts -D_dis..+D_chg, A = D_dis+D_chg+1 */
  int32_t n_modes;        /* 1, or 2 = charge->discharge switch-cost flag */
  int32_t policy_bytes;   /* 4 (int32), 2 (int16) or 0 (policy not kept) */
  int32_t ckpt_every;     /* 0: keep the whole policy; C > 0: keep V every C
                             stages, esdp_grad recomputes policies per segment */
  int32_t s0;             /* initial SoC index of the objective J (esdp_grad) */
  double s_max;           /* MWh; delta = s_max/(N-1) */
  double tau;             /* stage length in hours (bid quantities in MW) */
  double eta_c, eta_d;    /* charge / discharge efficiency, in (0,1] */
  double switch_cost;     /* $ per charge->discharge switch (n_modes == 2) */
} esdp_asset;

/* Create a context for `n_assets` assets solved together (one persistent,
 * batched launch).  The asset description is the problem statement of
 * Sec. II-B (SoC bound s_max and grid of eq. 12, efficiencies of eq. 2, the
 * action band of eq. 13's integer interior); solving several assets in one
 * launch has no counterpart in the paper.  Validates the shapes (ESDP_EINVAL
 * with a message; on any failure after the context itself was allocated
 * *out is a context that carries the message and must still be destroyed;
 * *out is NULL when `out` or `assets` is NULL, n_assets < 1 or the context
 * could not be allocated), allocates the device
 * workspace on the current CUDA device (ESDP_ENOMEM) and picks tile shapes
 * (see esdp_autotune).  The caller owns *out and frees it with
 * esdp_destroy. */
int esdp_create(const esdp_asset* assets, int32_t n_assets, uint32_t flags, esdp_ctx** out);

/* Backward induction over all assets (Algorithm 1, eq. 5-6).
 * price [sum T*K], trans [sum T*K*K], cost [sum A], terminal [sum M*N*K]
 * in; V1 [sum M*N*K] out (may be NULL).  Policies (and EV_t with
 * ESDP_KEEP_EV) stay in the context.  ESDP_ETIMEOUT if a device wait gave up,
 * ESDP_ENUMERIC if V_1 holds a NaN (host-pointer mode only). */
int esdp_solve(esdp_ctx* ctx, const float* price, const float* trans, const float* cost,
               const float* terminal, float* V1, void* stream);

/* Policy of stage t (1..T) of `asset`: [n_modes][N][K] action indices as
 * int32 or int16 (policy_bytes), the smallest maximiser of the Bellman step
 * (eq. 5; Algorithm 1 keeps only the maximum, the argmax is this library's
 * addition).  `out` is a host or device pointer as the context's flags say;
 * the caller owns it.  ESDP_EINVAL for a bad asset or stage index,
 * ESDP_ESTATE when the context keeps no full policy (policy_bytes == 0 or
 * ckpt_every > 0) or before esdp_solve. */
int esdp_policy(esdp_ctx* ctx, int32_t asset, int32_t t, void* out, void* stream);

/* EV_t (1..T) of `asset`: [n_modes][N][K] float (needs ESDP_KEEP_EV). */
int esdp_expected_value(esdp_ctx* ctx, int32_t asset, int32_t t, float* out, void* stream);

/* Convexified bid curves (eq. 10-11) of stages t0 <= t < t1 (1-based): for
 * every (t, m, k) the vertices of the upper concave envelope of
 * EV_t[m][.][k] over the SoC grid, strictly-above-chord vertices only, both
 * ends always included.  Outputs, with n = t1 - t0:
 *   n_bp   [n][n_modes][K]      vertex count
 *   bp_idx [n][n_modes][K][N]   vertex SoC indices (first n_bp valid)
 *   slope  [n][n_modes][K][N]   envelope slope between vertices q and q+1 in
 *                               $ per MWh of stored energy (first n_bp-1 valid);
 *                               strictly decreasing (monotone bids).
 * Needs ESDP_KEEP_EV.  Device or host pointers as the context's flags say. */
int esdp_bid_curves(esdp_ctx* ctx, int32_t asset, int32_t t0, int32_t t1, int32_t* n_bp,
                    int32_t* bp_idx, float* slope, void* stream);

/* The same bid curves in packed form, without the padding of the per-
 * envelope rows: envelope h = ((t - t0) M + m) K + k owns entries
 * [offsets[h], offsets[h+1]) of bp_idx (its vertex SoC indices, ascending)
 * and of slope (the slope from each vertex to the next, $ per MWh of stored
 * energy; the envelope's last entry is 0).  offsets [n_h + 1] (int64,
 * offsets[0] = 0, offsets[n_h] = total vertices), bp_idx / slope [cap].
 * Host mode: copies back the offsets and exactly `total` entries, and
 * returns ESDP_EINVAL (offsets written, nothing else) when total > cap.
 * Device mode: stream-ordered, entries at or beyond cap are not written
 * (read offsets[n_h] to size the arrays; cap = n_h * N always suffices).
 * Needs ESDP_KEEP_EV and a completed solve.  Errors as esdp_bid_curves. */
int esdp_bid_curves_packed(esdp_ctx* ctx, int32_t asset, int32_t t0, int32_t t1,
                           int64_t* offsets, int32_t* bp_idx, float* slope, int64_t cap,
                           void* stream);

/* Price-quantity bids at SoC index s (0..N-1) for stages t0..t1-1 of an
 * asset (eq. 8-11 on the SoC envelope): for every (stage, mode, price state)
 * the envelope vertices that esdp_bid_curves returned for the same stages
 * and lie inside the action window [s - D_dis, s + D_chg] (clipped to the
 * grid), the window's two ends and s itself (values on the envelope, chords
 * interpolated) are mapped to grid power -- selling, x <= s:
 * p = (s - x) delta eta_d / tau; buying, x > s: p = (s - x) delta / (eta_c tau)
 * -- and the upper concave envelope of U(p) = E_t(x(p)) is taken over power.
 * Segment q, between breakpoints p_mw[q] < p_mw[q+1] (MW, ascending: buying
 * first), sells at price[q] = -(U_{q+1} - U_q) / ((p_{q+1} - p_q) tau) $/MWh,
 * non-decreasing in q; where the buying price g eta_c of a marginal value g
 * would exceed its selling price g / eta_d (g < 0) the envelope merges the
 * two sides.  Inputs n_bp [n][M][K], bp_idx [n][M][K][N] as esdp_bid_curves
 * wrote them (n = t1 - t0); outputs n_pts [n][M][K] (breakpoint count,
 * >= 1; 0 where the input was not a vertex list of 2..N strictly increasing
 * indices from 0 to N-1), p_mw [n][M][K][A] (double), price [n][M][K][A] (float, the first
 * n_pts - 1 used).  Needs ESDP_KEEP_EV and a completed solve.  Device or
 * host pointers as the context's flags say; host mode blocks.  Returns
 * ESDP_EINVAL (NULL pointer, bad asset, stage range or s), ESDP_ESTATE,
 * ESDP_ENOMEM or ESDP_ECUDA. */
int esdp_bids_at(esdp_ctx* ctx, int32_t asset, int32_t t0, int32_t t1, int32_t s,
                 const int32_t* n_bp, const int32_t* bp_idx, int32_t* n_pts, double* p_mw,
                 float* price, void* stream);

/* Objective J = sum_k mu0[k] V_1[0][s0][k] (mode 0, initial SoC index s0 of
 * the asset) from the V_1 of the last esdp_solve, summed in double on the
 * device.  mu0 [K] is the initial price-state distribution; J [1] (double).
 * Host mode blocks; device mode queues one tiny kernel on `stream`.
 * ESDP_ESTATE before the first solve, ESDP_EINVAL on a bad asset index. */
int esdp_objective(esdp_ctx* ctx, int32_t asset, const float* mu0, double* J, void* stream);

/* Objective J = sum_k mu0[k] V_1[0][s0][k] and its sensitivities by a
 * forward pass of the state-occupancy distribution under the stored argmax
 * policy (envelope theorem on eq. 5-6; exact away from ties).  With
 * ckpt_every = C > 0 the policies are recomputed from the V checkpoints, B
 * segments of C stages at a time as the assets of one persistent launch (the
 * segments are independent), holding B segments' policies, values and
 * post-decision occupancies at once: B = the environment variable
 * ESDP_GRAD_SEGMENTS, else as many as 1 GiB of that workspace holds (the
 * result does not depend on B); otherwise the whole horizon is recomputed
 * once.  Uses the inputs of the last esdp_solve.  In: mu0 [K].  Out (any may be NULL):
 *   J          [1]         double
 *   d_price    [T*K]       float   dJ/dprice[t][k]
 *   d_trans    [T*K*K]     float   dJ/dtrans[t][k][k2]
 *   d_eta      [2]         double  dJ/deta_c, dJ/deta_d
 *   d_cost     [A]         float   dJ/dcost[a] (the per-action cost array)
 *   d_switch   [1]         double  dJ/dswitch_cost (0 with one mode)
 *   d_terminal [n_modes*N*K] float dJ/dterminal = the occupancy after stage T
 *   d_mu0      [K]         float   dJ/dmu0[k] = V_1[0][s0][k]
 * Repeated calls on the same solve give the same bits (the occupancy is
 * scattered in 64-bit fixed point, 2^-32 units; ESDP_ENUMERIC if an
 * occupancy entry exceeds 2^20, e.g. from a mu0 far from a distribution).
 * Device or host pointers as the context's flags say; blocks until done. */
int esdp_grad(esdp_ctx* ctx, int32_t asset, const float* mu0, double* J, float* d_price,
              float* d_trans, double* d_eta, float* d_cost, double* d_switch, float* d_terminal,
              float* d_mu0, void* stream);

/* Re-time the candidate tile shapes / actions-per-warp on the device and
 * keep the fastest (results are cached per shape class for the process).
 * The paper has no counterpart (its sweep is one library broadcast per
 * stage); the shapes only change how the Bellman step of eq. 5 is tiled,
 * not its result up to float32 rounding of the EV contraction.  Launches
 * whose assets all have K = 63 or 64 use a kernel variant with the shared
 * EV row stride fixed at compile time (same results; ESDP_NO_KH=1 pins the
 * general variant).
 * The launches of esdp_grad's segment re-sweeps (B copies of an asset with
 * ckpt_every > 0) are timed the same way, once per shape of asset.
 * With the environment variable ESDP_SHAPE="R,block" (rows per thread
 * 4/6/8/9/10/12, threads per block) that shape is used without timing;
 * ESDP_EINVAL if it cannot be built for the context's assets.  The results
 * of an earlier esdp_solve are discarded (the timed launches reuse the
 * context's workspace): policy, EV, bid curves and esdp_grad answer
 * ESDP_ESTATE until the next solve. */
int esdp_autotune(esdp_ctx* ctx, void* stream);

/* Device time in milliseconds of the persistent sweep kernel of the last
 * esdp_solve (CUDA events recorded on its stream right before and after the
 * launch, so the input copies, the row-sum preparation and the EV level
 * restore are outside it); waits for that launch to finish.  A measurement
 * aid with no counterpart in the paper.  ESDP_ESTATE when the context was
 * made without ESDP_TIME_SWEEP or has not solved yet. */
int esdp_sweep_ms(esdp_ctx* ctx, float* ms);

/* Per-stage cycle counts of the phases of the last esdp_solve's sweep,
 * averaged over its CTAs and stages (clock64 of each CTA's first thread):
 * 0 inputs of the stage, 1 neighbour wait (other warps write the previous
 * stage's outputs meanwhile), 2 EV halo copy and stage level, 3 banded
 * max-plus loop, 4 part merge and argmax recovery, 5 EV contraction,
 * 6 release, 7 next-stage loads and output bookkeeping.  Only a library
 * built with -DESDP_PHASE_CLOCKS counts them (the package's build script
 * makes it as libesdp_phase.so); the regular library returns ESDP_ESTATE.
 * cycles [n_phases >= 8] out.  A measurement aid with no counterpart in the
 * paper. */
int esdp_phase_clocks(esdp_ctx* ctx, double* cycles, int32_t n_phases);

/* Device status word of the last launch: 0, or the ESDP_E* code a kernel
 * reported.  Synchronises `stream`. */
int esdp_status(esdp_ctx* ctx, void* stream);

/* Counters of the chosen launch shape: grid, block, work items, rows per
 * tile of asset 0, actions split (parts), R (rows per thread), and the unit
 * that contracts EV for asset 0 (ev_path: 0 FP32 SIMT, 1 tcgen05 split-tf32,
 * 2 mma.sync split-tf32; tiles with K >= 64 and at least 98,304
 * multiply-adds per stage, rows x modes x K^2, take a tensor path when K is
 * a multiple of 16 resp. 8;
 * the environment variable ESDP_EV = "simt" | "tc" | "mma" pins one where K
 * allows it).  Any pointer may be NULL. */
int esdp_launch_info(const esdp_ctx* ctx, int32_t* grid, int32_t* block, int32_t* items,
                     int32_t* rows_per_tile, int32_t* parts, int32_t* rows_per_thread,
                     int32_t* ev_path);

/* ---------------------------------------------------------------------
 * Stagewise-independent prices on the paper's own action grid (Sec. III-A,
 * Algorithm 1, eq. 2 and 13).  Per stage t = T..1:
 *   V_{t-1}(s) = sum_k pi_hat[t][k] max_a ( lam_hat[t][k] p_a tau + V_t(sigma) ),
 * actions p_a of eq. 13 (charge -p_max, -(n_c-1) delta/eta .. -delta/eta, idle
 * 0, discharge delta eta .. (n_d-1) delta eta, p_max; n_c = ceil(p_max eta /
 * delta), n_d = ceil(p_max / (delta eta)), delta = s_max/(S-1)), next state
 * sigma = s delta + F(p_a) tau with F(p) = -p/eta (p >= 0) or -eta p (p < 0),
 * V_t linearly interpolated between grid points off the grid, and -inf
 * (infeasible) outside [0, s_max].  In the Markov form of esdp_solve this is
 * the rank-1 transition P_t = 1 pi_hat_{t+1}^T with K = R price states.
 * --------------------------------------------------------------------- */
typedef struct {
  int32_t T;             /* stages */
  int32_t S;             /* SoC grid points */
  int32_t R;             /* price samples per stage, 1..4096 */
  int32_t policy_bytes;  /* 0 (values only), 2 or 4: argmax action index per (t, s, k) */
  double s_max;          /* MWh */
  double p_max;          /* MW */
  double eta;            /* efficiency of eq. 2, in (0, 1] */
  double tau;            /* stage length in hours */
} esdp_iid_problem;

/* The action grid of eq. 13 for a problem: writes the P power levels (MW,
 * ascending) to p_hat when it is not NULL and their count to *n_actions. */
int esdp_iid_actions(const esdp_iid_problem* problem, double* p_hat, int32_t* n_actions);

/* Backward induction over all T stages in one persistent launch.
 *   lam_hat, pi_hat [T][R]: price samples and probabilities of stages 1..T
 *   terminal [S] V_T (NULL: zero); V0 [S] out: V_0
 *   V_all [T+1][S] out: V_t of every stage t = 0..T (the input of
 *     esdp_iid_bids and esdp_iid_clear), or NULL
 *   policy [T][S][R] int32/int16 as policy_bytes says (stage t at t-1) or NULL
 * With flags & ESDP_DEVICE_PTRS the arrays are device pointers, else host
 * arrays.  Allocates its workspace, blocks until done; returns ESDP_OK or a
 * negative code with a message in err (err_len bytes, may be NULL). */
int esdp_solve_iid(const esdp_iid_problem* problem, const float* lam_hat, const float* pi_hat,
                   const float* terminal, float* V0, float* V_all, void* policy, uint32_t flags,
                   void* stream, char* err, int32_t err_len);

/* Convexified price-quantity bid curves of the paper (eq. 8-11): for every
 * delivery interval t in [t0, t1) and grid SoC s (the state s_{t-1}), the
 * upper concave envelope over the power levels p_a of U_t(p_a; s) =
 * V_t(s delta + F(p_a) tau) on the feasible actions (V_t interpolated off the
 * grid).  Outputs, with n = t1 - t0 (device pointers; V_all as written by
 * esdp_solve_iid):
 *   n_bp      [n][S]     vertex count
 *   bp_action [n][S][P]  action indices of the vertices, ascending power
 *   bp_price  [n][S][P]  bid price of the segment between vertices q and q+1,
 *                        -(U_{q+1} - U_q) / ((p_{q+1} - p_q) tau) in $/MWh,
 *                        non-decreasing in q (monotone bids)
 * The orientation test (y_j - y_i)(x_l - x_i) - (y_l - y_i)(x_j - x_i) <= 0
 * drops a point (collinear points are dropped) and runs in double with
 * round-to-nearest operations in that order.  Blocks until done. */
int esdp_iid_bids(const esdp_iid_problem* problem, const float* V_all, int32_t t0, int32_t t1,
                  int32_t* n_bp, int32_t* bp_action, float* bp_price, void* stream, char* err,
                  int32_t err_len);

/* Merit-order clearing of a price-taking storage against realised price
 * paths (device pointers): lam_real [n_paths][T]; starting SoC s0 (MWh).
 * At stage t the cleared power maximises lam_t p tau + V_t(s + F(p) tau)
 * over the feasible actions (a vertex of the stage's convexified bid curve;
 * the first on ties), the SoC moves (off the grid at the end-point actions)
 * and lam_t p tau accrues.  Outputs: revenue [n_paths] and s_end [n_paths]
 * (grid steps, double; may be NULL), actions [n_paths][T] or NULL.  Double
 * arithmetic.  Blocks until done. */
int esdp_iid_clear(const esdp_iid_problem* problem, const float* V_all, const float* lam_real,
                   int32_t n_paths, double s0, double* revenue, double* s_end, int32_t* actions,
                   void* stream, char* err, int32_t err_len);

/* Allocation-free solve of one asset.  The paper has no counterpart: this
 * entry point exists for callers that cannot call cudaMalloc, for example a
 * plug-in running inside an application that owns the device memory pool
 * through its own caching allocator, a process under a hard device-memory
 * quota, or code on a latency-critical path where an allocation could
 * stall.  It runs the same persistent sweep as esdp_solve but needs no
 * context and allocates nothing: its workspace
 * (EV halo buffers, neighbour flags, status word, stage levels, launch plan)
 * is one file-scope device array of ESDP_NOALLOC_SCRATCH_BYTES that every
 * GPU loading this library reserves until the process exits.
 *   asset: description as for esdp_create (policy_bytes 2 or 4 when `policy`
 *          is given; ckpt_every is ignored);
 *   price [T*K], trans [T*K*K], cost [A], terminal [n_modes*N*K]: device
 *          pointers, read only;  V1 [n_modes*N*K]: device pointer, written;
 *   policy: NULL, or a device buffer of T*n_modes*N*K int32/int16 entries;
 *   stream: cudaStream_t (NULL = legacy default stream);
 *   err/err_len: optional buffer for a message (always NUL-terminated).
 * The call is queued on `stream` and returns when it has finished; the
 * result code includes the device status word (ESDP_ETIMEOUT etc.).
 * Limits: the asset must fit the workspace, about 2*n_modes*N*K floats of EV
 * plus 2*T*K doubles of per-stage data (N*K up to roughly 1.9 million for one
 * mode and T = 288), and at most 2048 tiles; larger assets are rejected with
 * ESDP_EINVAL and a message that states the bytes needed.
 * Every call looks up the workspace address (cudaGetSymbolAddress) with
 * the caller's device current, so a new context or a device reset is
 * picked up; the first call on a device also loads the library's device
 * code there, so make that first call before any stream capture.  The
 * bounded device waits give up after ESDP_TIMEOUT_MS milliseconds (default
 * 5000) with ESDP_ETIMEOUT, as in esdp_solve.  Every call on a device shares the one
 * workspace: calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller. */
#define ESDP_NOALLOC_SCRATCH_BYTES (16u << 20)
int esdp_solve_noalloc(const esdp_asset* asset, const float* price, const float* trans,
                       const float* cost, const float* terminal, float* V1, void* policy,
                       void* stream, char* err, int32_t err_len);

/* Issue-rate probe of the float32 instructions of the max-plus loop (a
 * register-only kernel, one block of 1024 threads per SM of the current
 * device, clock64-timed): kind 0 add.f32, 1 add.rn.f32x2, 2 max.f32,
 * 3 three-input max.f32, 4 the loop's mix (two packed adds and two
 * three-input maxima per four evaluations).  Writes the median over SMs of
 * warp-lane instructions and of element operations (adds, maxima or
 * evaluations) per SM clock.  Blocks until done.  Returns ESDP_EINVAL for a
 * bad kind, iters < 1 or a NULL output, ESDP_ECUDA on a CUDA error. */
int esdp_alu_probe(int32_t kind, int32_t iters, double* instr_per_clk, double* elem_per_clk,
                   void* stream);

/* Device time in milliseconds (CUDA events on the call's stream) of the
 * sweep of the last successful esdp_solve_iid made by this host thread: the
 * stage-probability sums and the persistent Algorithm 1 launch, without the
 * workspace allocation and the copies around them; a negative value before
 * any such call.  A measurement aid with no counterpart in the paper. */
double esdp_iid_last_sweep_ms(void);

/* Free a context and its device workspace (no counterpart in the paper).
 * NULL is accepted.  The caller must not use the context afterwards, and no
 * work queued with it may still be running on the device. */
void esdp_destroy(esdp_ctx* ctx);
/* Message of the context's last failed call ("" if none; a static message
 * when ctx is NULL).  Owned by the context, valid until its next call. */
const char* esdp_last_error(const esdp_ctx* ctx);
int esdp_version(void);

#ifdef __cplusplus
}
#endif
#endif /* ESDP_H_ */
