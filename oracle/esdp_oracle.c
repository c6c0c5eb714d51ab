/*
 * FP64 reference oracle for discretized stochastic-DP storage arbitrage.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path links, loads or
 * calls this file: only the tests, the package's smoke check and the
 * benchmark's CPU-baseline leg do.  It shares no code, header, table or
 * helper with the CUDA library.
 *
 * Plain loops in double precision, in the order the paper states them, with
 * no blocking, fusion or reordering.  Build with -O2 -ffp-contract=off (no
 * fused multiply-add, so that results do not depend on the compiler).
 *
 * Problem (Sec. II-B, eq. 4-6, generalised to a Markov price chain):
 *   stages t = 1..T (array index t-1), SoC index s = 0..N-1 with step
 *   delta = s_max/(N-1) (eq. 12), price state k = 0..K-1, mode m < n_modes.
 *   Action a = 0..A-1 shifts the SoC by d = a - D_dis grid steps (the
 *   integer interior of the action grid of eq. 13).  Grid energy of the
 *   action, from the efficiency transition of eq. 2 with separate charge and
 *   discharge efficiencies:
 *       d < 0 (discharge): e_a = -d * delta * eta_d   (> 0, sold)
 *       d > 0 (charge):    e_a = -d * delta / eta_c   (< 0, bought)
 *   Payoff  r[t,k,a] = price[t,k] * e_a - cost[a]
 *                      - switch_cost * [n_modes == 2 && m == 1 && d < 0].
 *   Mode: m' = 0 after a discharge, 1 after a charge, unchanged when idle.
 *   Expectation (eq. 6 with a Markov chain):
 *       EV_t[m][s][k] = sum_k2 trans[t][k][k2] * V_{t+1}[m][s][k2]
 *   Bellman step (eq. 5, the feasibility interval of eq. 4 becomes
 *   0 <= s + d <= N-1):
 *       V_t[m][s][k] = max_a r[t,k,a] + EV_t[m'][s + d][k]
 *   policy = the smallest maximising a; gap = best - second best.
 *   Base case V_{T+1} = terminal (zero in eq. 6).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef struct {
  int32_t T, N, K, A, D_dis, D_chg, n_modes, pad_;
  double s_max, eta_c, eta_d, switch_cost;
} orc_problem;

#define IDX3(m, s, k, N, K) (((size_t)(m) * (size_t)(N) + (size_t)(s)) * (size_t)(K) + (size_t)(k))

/* Grid-side energy of action a (eq. 2). */
static double action_energy(const orc_problem* p, int a) {
  double delta = p->s_max / (double)(p->N - 1);
  int d = a - p->D_dis;
  if (d < 0) return -(double)d * delta * p->eta_d;
  if (d > 0) return -(double)d * delta / p->eta_c;
  return 0.0;
}

static int next_mode(const orc_problem* p, int m, int a) {
  int d = a - p->D_dis;
  if (p->n_modes < 2) return 0;
  if (d < 0) return 0;
  if (d > 0) return 1;
  return m;
}

static double payoff(const orc_problem* p, double price, const double* cost, int m, int a) {
  double r = price * action_energy(p, a) - cost[a];
  if (p->n_modes == 2 && m == 1 && a < p->D_dis) r -= p->switch_cost;
  return r;
}

static int check(const orc_problem* p) {
  if (p->T < 1 || p->N < 2 || p->K < 1 || p->A < 1) return -1;
  if (p->D_dis < 0 || p->D_chg < 0 || p->D_dis + p->D_chg + 1 != p->A) return -1;
  if (p->n_modes != 1 && p->n_modes != 2) return -1;
  return 0;
}

/* EV_t = trans_t applied to V_{t+1} over the price index (eq. 6). */
static void expectation(const orc_problem* p, const double* P, const double* Vn, double* EV, int nthreads) {
  int M = p->n_modes, N = p->N, K = p->K;
  (void)nthreads;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int s = 0; s < N; ++s)
    for (int m = 0; m < M; ++m)
      for (int k = 0; k < K; ++k) {
        double acc = 0.0;
        for (int k2 = 0; k2 < K; ++k2) acc += P[(size_t)k * K + k2] * Vn[IDX3(m, s, k2, N, K)];
        EV[IDX3(m, s, k, N, K)] = acc;
      }
}

/* One Bellman step (eq. 5) for stage t (1-based) given EV_t. */
static void bellman(const orc_problem* p, int t, const double* price, const double* cost, const double* EV,
                    double* V, int32_t* pol, double* gap, int nthreads) {
  int M = p->n_modes, N = p->N, K = p->K, A = p->A;
  (void)nthreads;
#pragma omp parallel for num_threads(nthreads) schedule(static)
  for (int s = 0; s < N; ++s)
    for (int m = 0; m < M; ++m)
      for (int k = 0; k < K; ++k) {
        double lam = price[(size_t)(t - 1) * K + k];
        double best = -INFINITY, second = -INFINITY;
        int arg = -1;
        for (int a = 0; a < A; ++a) {
          int s2 = s + (a - p->D_dis);
          if (s2 < 0 || s2 > N - 1) continue; /* infeasible (Alg. 1, infeasibility step) */
          int m2 = next_mode(p, m, a);
          double v = payoff(p, lam, cost, m, a) + EV[IDX3(m2, s2, k, N, K)];
          if (v > best) {
            second = best;
            best = v;
            arg = a;
          } else if (v > second) {
            second = v;
          }
        }
        size_t o = IDX3(m, s, k, N, K);
        V[o] = best;
        if (pol) pol[o] = arg;
        if (gap) gap[o] = best - second;
      }
}

/*
 * Backward induction over t = T..1.
 *   price[T*K], trans[T*K*K], cost[A], terminal[M*N*K]   (inputs)
 *   V_all[(T+1)*M*N*K]: V_t at block t-1, V_{T+1} at block T  (or NULL)
 *   EV_all[T*M*N*K]:    EV_t at block t-1                      (or NULL)
 *   policy[T*M*N*K], gap[T*M*N*K]                              (or NULL)
 *   V1[M*N*K]                                                  (required)
 */
int orc_solve(const orc_problem* p, const double* price, const double* trans, const double* cost,
              const double* terminal, double* V_all, double* EV_all, int32_t* policy, double* gap,
              double* V1, int nthreads) {
  if (check(p)) return -1;
  size_t L = (size_t)p->n_modes * p->N * p->K;
  double* Vn = (double*)malloc(L * sizeof(double));
  double* Vc = (double*)malloc(L * sizeof(double));
  double* EV = (double*)malloc(L * sizeof(double));
  if (!Vn || !Vc || !EV) {
    free(Vn); free(Vc); free(EV);
    return -2;
  }
  memcpy(Vn, terminal, L * sizeof(double));
  if (V_all) memcpy(V_all + (size_t)p->T * L, terminal, L * sizeof(double));
  for (int t = p->T; t >= 1; --t) {
    expectation(p, trans + (size_t)(t - 1) * p->K * p->K, Vn, EV, nthreads);
    if (EV_all) memcpy(EV_all + (size_t)(t - 1) * L, EV, L * sizeof(double));
    bellman(p, t, price, cost, EV, Vc, policy ? policy + (size_t)(t - 1) * L : NULL,
            gap ? gap + (size_t)(t - 1) * L : NULL, nthreads);
    if (V_all) memcpy(V_all + (size_t)(t - 1) * L, Vc, L * sizeof(double));
    double* tmp = Vn; Vn = Vc; Vc = tmp;
  }
  memcpy(V1, Vn, L * sizeof(double));
  free(Vn); free(Vc); free(EV);
  return 0;
}

/*
 * Upper concave envelope of the points (i, y[i*stride]), i = 0..N-1: the
 * hypograph convexification of eq. 10 done with Andrew's monotone chain (a
 * Graham-scan variant).  A point is kept only if it lies strictly above the
 * chord of its hull neighbours; points on the chord are dropped.  Both end
 * points are always vertices.  Returns the vertex count; idx receives the
 * vertex indices in increasing order.  The orientation value
 *   (y_j - y_i) * (l - i) - (y_l - y_i) * (j - i)
 * is evaluated in double precision in exactly this order.
 */
int orc_hull(int N, const double* y, int stride, int32_t* idx) {
  int h = 0;
  for (int l = 0; l < N; ++l) {
    while (h >= 2) {
      int i = idx[h - 2], j = idx[h - 1];
      double yi = y[(size_t)i * stride], yj = y[(size_t)j * stride], yl = y[(size_t)l * stride];
      double lhs = (yj - yi) * (double)(l - i);
      double rhs = (yl - yi) * (double)(j - i);
      double cross = lhs - rhs;
      if (cross <= 0.0) --h; /* j on or below chord (i, l): not a strict vertex */
      else break;
    }
    idx[h++] = l;
  }
  return h;
}

/*
 * Forward occupancy pass under a stored policy and the sensitivities of
 * J = sum_k mu0[k] V_1[0][s0][k] that follow from it (envelope theorem on
 * eq. 5-6; valid away from ties of the maximisation).
 *   rho_1[0][s0][k] = mu0[k];
 *   post_t[m'][s + d][k] += rho_t[m][s][k]        (d, m' from the policy)
 *   rho_{t+1}[m'][s][k2] = sum_k post_t[m'][s][k] * trans[t][k][k2]
 * Gradients (all in double):
 *   dprice[t][k]      = sum_{m,s} rho_t[m][s][k] * e_{pi}
 *   dtrans[t][k][k2]  = sum_{m,s} post_t[m][s][k] * V_{t+1}[m][s][k2]
 *   deta_c            = sum rho_t * price[t][k] * de/deta_c (charge: d*delta/eta_c^2)
 *   deta_d            = sum rho_t * price[t][k] * de/deta_d (discharge: -d*delta)
 *   dcost[a]          = -sum_t sum rho_t * [pi_t = a]       (cost[a] enters every payoff of a)
 *   dswitch           = -sum rho_t * [m = 1, d < 0]          (two modes)
 *   dterminal[m][s][k] = rho_{T+1}[m][s][k]                 (J holds E[V_{T+1}] linearly)
 *   exp_reward[t]     = sum rho_t * r  (so J = sum_t exp_reward + E[V_{T+1}])
 *   V_all: (T+1) blocks as produced by orc_solve (block t holds V_{t+1}).
 */
int orc_occupancy(const orc_problem* p, const double* price, const double* trans, const double* cost,
                  const int32_t* policy, const double* V_all, int s0, const double* mu0, double* J,
                  double* J_occ, double* dprice, double* dtrans, double* deta_c, double* deta_d,
                  double* exp_reward, double* mass, double* dcost, double* dswitch,
                  double* dterminal) {
  if (check(p)) return -1;
  int M = p->n_modes, N = p->N, K = p->K, T = p->T;
  size_t L = (size_t)M * N * K;
  double delta = p->s_max / (double)(N - 1);
  double* rho = (double*)calloc(L, sizeof(double));
  double* post = (double*)calloc(L, sizeof(double));
  if (!rho || !post) {
    free(rho); free(post);
    return -2;
  }
  double j = 0.0;
  for (int k = 0; k < K; ++k) {
    rho[IDX3(0, s0, k, N, K)] = mu0[k];
    j += mu0[k] * V_all[IDX3(0, s0, k, N, K)];
  }
  *J = j;
  double jo = 0.0, dc = 0.0, dd = 0.0, dsw = 0.0;
  for (int a = 0; a < p->A; ++a) dcost[a] = 0.0;
  for (int t = 1; t <= T; ++t) {
    const int32_t* pol = policy + (size_t)(t - 1) * L;
    const double* Vn = V_all + (size_t)t * L;
    const double* P = trans + (size_t)(t - 1) * K * K;
    double er = 0.0, ms = 0.0;
    memset(post, 0, L * sizeof(double));
    for (int k = 0; k < K; ++k) dprice[(size_t)(t - 1) * K + k] = 0.0;
    for (int m = 0; m < M; ++m)
      for (int s = 0; s < N; ++s)
        for (int k = 0; k < K; ++k) {
          double r0 = rho[IDX3(m, s, k, N, K)];
          if (r0 == 0.0) continue;
          int a = pol[IDX3(m, s, k, N, K)];
          int d = a - p->D_dis;
          int m2 = next_mode(p, m, a);
          double lam = price[(size_t)(t - 1) * K + k];
          post[IDX3(m2, s + d, k, N, K)] += r0;
          dprice[(size_t)(t - 1) * K + k] += r0 * action_energy(p, a);
          if (d > 0) dc += r0 * lam * ((double)d * delta / (p->eta_c * p->eta_c));
          if (d < 0) dd += r0 * lam * (-(double)d * delta);
          /* the payoff carries -cost[a] and, from mode 1 into a discharge, -switch_cost */
          dcost[a] -= r0;
          if (M == 2 && m == 1 && d < 0) dsw -= r0;
          er += r0 * payoff(p, lam, cost, m, a);
          ms += r0;
        }
    exp_reward[t - 1] = er;
    mass[t - 1] = ms;
    jo += er;
    for (int k = 0; k < K; ++k)
      for (int k2 = 0; k2 < K; ++k2) {
        double acc = 0.0;
        for (int m = 0; m < M; ++m)
          for (int s = 0; s < N; ++s) acc += post[IDX3(m, s, k, N, K)] * Vn[IDX3(m, s, k2, N, K)];
        dtrans[((size_t)(t - 1) * K + k) * K + k2] = acc;
      }
    for (int m = 0; m < M; ++m)
      for (int s = 0; s < N; ++s)
        for (int k2 = 0; k2 < K; ++k2) {
          double acc = 0.0;
          for (int k = 0; k < K; ++k) acc += post[IDX3(m, s, k, N, K)] * P[(size_t)k * K + k2];
          rho[IDX3(m, s, k2, N, K)] = acc;
        }
  }
  const double* VT1 = V_all + (size_t)T * L;
  for (size_t i = 0; i < L; ++i) jo += rho[i] * VT1[i];
  /* J depends on the terminal value through E[V_{T+1}]: the final occupancy */
  for (size_t i = 0; i < L; ++i) dterminal[i] = rho[i];
  *J_occ = jo;
  *deta_c = dc;
  *deta_d = dd;
  *dswitch = dsw;
  free(rho); free(post);
  return 0;
}

int orc_version(void) { return 1; }
