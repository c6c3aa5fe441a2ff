/*
 * pdilqr_oracle.h -- plain FP64 CPU oracle for the primal-dual iLQR hot path.
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, obviously-correct
 * definition that the CUDA path is checked against.  Only the test suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product library never links, loads or calls it, and it shares no code with
 * the product (no common headers, helpers or constants).
 *
 * Conventions (Sec. II-A/II-B of the paper, with the horizon re-indexed so
 * that N counts control intervals and the terminal cost sits on x_N):
 *   states   x_0..x_N   in R^n     controls u_0..u_{N-1} in R^m
 *   costates lam_0..lam_N in R^n
 * Every per-stage array has N+1 slots, row-major within a stage:
 *   A [N+1][n][n]  B [N+1][n][m]  c [N+1][n]   (slot N unused)
 *   Q [N+1][n][n]  q [N+1][n]                  (slot N = terminal Q_N, q_N)
 *   R [N+1][m][m]  S [N+1][m][n]  r [N+1][m]   (slot N unused)
 *   dx [N+1][n]  du [N+1][m] (slot N written 0)  dlam [N+1][n]
 *   K [N+1][m][n]  k [N+1][m] (slot N written 0)  P [N+1][n][n]  p [N+1][n]
 *
 * Parity status of each function is stated beside it; every function listed
 * here is pinned by a CPU test against something other than itself.
 */
#ifndef PDILQR_ORACLE_H
#define PDILQR_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

/* Sec. II-C, Eq. (lqr) backward recursion, forward rollout and
 * dlam_i = P_i dx_i + p_i.  s is dx_0 = xhat_0 - x_0 (Eq. QP).
 * K, kff, P, p may be NULL.  Returns 0, or -1 if some G_i is not SPD. */
int orc_riccati_solve(int n, int m, int N,
                      const double *A, const double *B, const double *c,
                      const double *Q, const double *R, const double *S,
                      const double *q, const double *r, const double *s,
                      double *dx, double *du, double *dlam,
                      double *K, double *kff, double *P, double *p);

/* Residual of the LQ KKT system (first-order conditions of Eq. QP with the
 * Lagrangian of Sec. II-B).  Writes the infinity norms of the residual, of
 * the KKT matrix (max absolute row sum), of z = (dx, du, dlam) and of the
 * right-hand side into out[0..3]. */
void orc_kkt_residual(int n, int m, int N,
                      const double *A, const double *B, const double *c,
                      const double *Q, const double *R, const double *S,
                      const double *q, const double *r, const double *s,
                      const double *dx, const double *du, const double *dlam,
                      double out[4]);

/* Relaxed barrier of Sec. II-F: value, first and second derivative. */
void orc_barrier(double xi, double mu, double delta, double out[3]);

/* ---------------------------------------------------------------------- */
/* Single-rigid-body (SRBD) quadruped model, Sec. III (equations are this
 * library's reading; the paper prints none).  One robot has n = m = 12;
 * the centralised multi-robot variant stacks nrob robots block-diagonally
 * (n = m = 12 nrob) and couples their positions with a ring formation cost
 * 0.5 w_form sum_a |p_a - p_{a+1 mod nrob} - d_a|^2 (nrob >= 2).  Per-stage
 * arrays then hold nrob robot blocks; contact is [N+1][nrob][4].          */
typedef struct {
    int nrob;             /* robots stacked in one state (1..16)       */
    double w_form;        /* formation weight (ignored when nrob == 1) */
    double d_form[16][3]; /* formation offsets d_a                     */
    double mass;          /* kg                                        */
    double inertia[3];    /* body inertia diagonal, kg m^2             */
    double dt;            /* explicit-Euler step, s                    */
    double gravity;       /* m/s^2, acts along -z                      */
    double foot[4][3];    /* nominal stance points r_j (world frame)   */
    double mu_fric;       /* friction coefficient of the cone          */
    double bar_mu;        /* relaxed-barrier weight mu                 */
    double bar_delta;     /* relaxed-barrier switch point delta        */
    double W[12];         /* stage state weight (diagonal)             */
    double Wu[12];        /* stage control weight (diagonal)           */
    double WN[12];        /* terminal state weight (diagonal)          */
} orc_srbd_params;

/* x_next = h(x, u) for one stage; contact[4 nrob] in {0,1}. */
void orc_srbd_step(const orc_srbd_params *prm, const double *x,
                   const double *u, const unsigned char *contact,
                   double *x_next);
/* Analytic Jacobians A = dh/dx (n x n), B = dh/du (n x m). */
void orc_srbd_jacobians(const orc_srbd_params *prm, const double *x,
                        const double *u, const unsigned char *contact,
                        double *A, double *B);
/* Stage cost l_k (tracking + barrier); terminal when u == NULL. */
double orc_srbd_cost(const orc_srbd_params *prm, const double *x,
                     const double *u, const unsigned char *contact,
                     const double *xref, const double *uref, int terminal);

/* Linearisation of Sec. II-B / II-F at (x, u, lam) over a horizon of N
 * intervals: A, B, defect c_k = h(x_k,u_k) - x_{k+1}, Gauss-Newton Q, R,
 * S (= 0 for this model), Lagrangian gradients q, r (costate terms
 * included).  xref [N+1][n], uref [N+1][m], contact [N+1][nrob][4]. */
void orc_srbd_linearize(const orc_srbd_params *prm, int N,
                        const double *x, const double *u, const double *lam,
                        const double *xref, const double *uref,
                        const unsigned char *contact,
                        double *A, double *B, double *c, double *Q,
                        double *R, double *S, double *q, double *r);

/* Total cost J and constraint violation theta (Eq. constraint
 * satisfaction, plus the initial-state term |xhat_0 - x_0|_2). */
void orc_srbd_merit(const orc_srbd_params *prm, int N, const double *x0hat,
                    const double *x, const double *u, const double *xref,
                    const double *uref, const unsigned char *contact,
                    double *J, double *theta);

/* Filter acceptance of Sec. II-E for one candidate. */
int orc_filter_accept(double J0, double th0, double dphi, double th_max,
                      double alpha, double Ja, double tha, double c_armijo);

typedef struct {
    int max_iters;        /* SQP iterations                                 */
    double tol_step;      /* stop when |dz|_inf < tol_step and             */
    double tol_theta;     /*      theta < tol_theta (0 disables stopping)  */
    double c_armijo;      /* Armijo constant                                */
    double theta_frac;    /* theta_max = theta_frac * max(1, theta_init)    */
    const double *alpha_replay; /* if non-NULL: use these step sizes        */
} orc_sqp_opts;

typedef struct {
    int iters;            /* SQP iterations performed (KKT solves)           */
    int status;           /* 0 ok, 1 line search found no step, 2 not SPD    */
    double alpha[32];     /* step size taken at each iteration               */
    double step[32];      /* |dz|_inf of the search direction per iteration  */
    double theta_it[32];  /* theta of the iterate at the start of each iter. */
    double J, theta;      /* merit at the returned iterate                   */
    double theta_max;
} orc_sqp_info;

/* Multiple-shooting SQP (Sec. II-B..II-E): linearise, solve the LQ KKT
 * system by Eq. (lqr), evaluate the ten step sizes 2^0..2^-9, take the
 * largest accepted one, update x, u, lam in place. */
int orc_srbd_sqp(const orc_srbd_params *prm, int N, const double *x0hat,
                 double *x, double *u, double *lam,
                 const double *xref, const double *uref,
                 const unsigned char *contact, const orc_sqp_opts *opt,
                 orc_sqp_info *info);

/* Linear time-varying model (test model for the SQP loop):
 *   h_k(x,u) = A_k x + B_k u + e_k,
 *   l_k = 0.5 x^T Q_k x + u^T S_k x + 0.5 u^T R_k u + gq_k^T x + gr_k^T u,
 *   l_N = 0.5 x^T Q_N x + gq_N^T x.
 * The SQP on it converges in one step with alpha = 1. */
double orc_ltv_cost(int n, int m, int N, const double *Q, const double *R,
                    const double *S, const double *gq, const double *gr,
                    const double *x, const double *u);
int orc_ltv_sqp(int n, int m, int N, const double *A, const double *B,
                const double *e, const double *Q, const double *R,
                const double *S, const double *gq, const double *gr,
                const double *x0hat, double *x, double *u, double *lam,
                const orc_sqp_opts *opt, orc_sqp_info *info);

#ifdef __cplusplus
}
#endif
#endif
