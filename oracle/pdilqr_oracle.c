/*
 * pdilqr_oracle.c -- plain FP64 CPU oracle (test infrastructure only).
 *
 * Written for readability, not speed: every loop follows the equation it
 * cites, with no blocking, fusion or reordering.  The CUDA path shares no
 * code with this file; only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark load it.
 */
#include "pdilqr_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- helpers */

/* out (r x c) = op(X) * op(Y); op = transpose when the flag is set.
 * X is stored (r x k) or (k x r), Y (k x c) or (c x k). */
static void mm(int r, int k, int c, const double *X, int tX, const double *Y,
               int tY, double *out)
{
    for (int i = 0; i < r; ++i)
        for (int j = 0; j < c; ++j) {
            double acc = 0.0;
            for (int l = 0; l < k; ++l) {
                double a = tX ? X[l * r + i] : X[i * k + l];
                double b = tY ? Y[j * k + l] : Y[l * c + j];
                acc += a * b;
            }
            out[i * c + j] = acc;
        }
}

/* y (r) = op(X) v */
static void mv(int r, int k, const double *X, int tX, const double *v,
               double *y)
{
    for (int i = 0; i < r; ++i) {
        double acc = 0.0;
        for (int l = 0; l < k; ++l)
            acc += (tX ? X[l * r + i] : X[i * k + l]) * v[l];
        y[i] = acc;
    }
}

/* In-place Cholesky G = L L^T (lower triangle kept).  0 ok, -1 not SPD. */
static int chol(int m, double *G)
{
    for (int j = 0; j < m; ++j) {
        double d = G[j * m + j];
        for (int l = 0; l < j; ++l) d -= G[j * m + l] * G[j * m + l];
        if (!(d > 0.0)) return -1;
        d = sqrt(d);
        G[j * m + j] = d;
        for (int i = j + 1; i < m; ++i) {
            double v = G[i * m + j];
            for (int l = 0; l < j; ++l) v -= G[i * m + l] * G[j * m + l];
            G[i * m + j] = v / d;
        }
    }
    return 0;
}

/* Solve L L^T X = Y for ncol right-hand sides stored as columns of Y
 * (m x ncol, row-major), in place. */
static void chol_solve(int m, const double *L, int ncol, double *Y)
{
    for (int col = 0; col < ncol; ++col) {
        for (int i = 0; i < m; ++i) {          /* L z = y */
            double v = Y[i * ncol + col];
            for (int l = 0; l < i; ++l) v -= L[i * m + l] * Y[l * ncol + col];
            Y[i * ncol + col] = v / L[i * m + i];
        }
        for (int i = m - 1; i >= 0; --i) {     /* L^T x = z */
            double v = Y[i * ncol + col];
            for (int l = i + 1; l < m; ++l) v -= L[l * m + i] * Y[l * ncol + col];
            Y[i * ncol + col] = v / L[i * m + i];
        }
    }
}

static double *dalloc(size_t count)
{
    return (double *)calloc(count ? count : 1, sizeof(double));
}

/* ------------------------------------------------- Riccati, Eq. (lqr) */

int orc_riccati_solve(int n, int m, int N,
                      const double *A, const double *B, const double *c,
                      const double *Q, const double *R, const double *S,
                      const double *q, const double *r, const double *s,
                      double *dx, double *du, double *dlam,
                      double *K_out, double *k_out, double *P_out,
                      double *p_out)
{
    const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
    double *P = dalloc((N + 1) * nn), *p = dalloc((N + 1) * (size_t)n);
    double *K = dalloc((N + 1) * nm), *kf = dalloc((N + 1) * (size_t)m);
    double *G = dalloc(mm_), *H = dalloc(nm), *h = dalloc(m);
    double *PB = dalloc(nm), *PA = dalloc(nn), *Pc = dalloc(n);
    double *tmp = dalloc(nn), *tmpv = dalloc(n);
    int status = 0;

    /* terminal value function: P_N = Q_N, p_N = q_N */
    memcpy(P + N * nn, Q + N * nn, nn * sizeof(double));
    memcpy(p + (size_t)N * n, q + (size_t)N * n, n * sizeof(double));

    for (int k = N - 1; k >= 0; --k) {
        const double *Ak = A + k * nn, *Bk = B + k * nm, *ck = c + (size_t)k * n;
        const double *Qk = Q + k * nn, *Rk = R + k * mm_, *Sk = S + k * nm;
        const double *qk = q + (size_t)k * n, *rk = r + (size_t)k * m;
        const double *P1 = P + (k + 1) * nn, *p1 = p + (size_t)(k + 1) * n;

        /* Pc = p_{k+1} + P_{k+1} c_k */
        mv(n, n, P1, 0, ck, Pc);
        for (int i = 0; i < n; ++i) Pc[i] += p1[i];
        /* G = R + B^T P B */
        mm(n, n, m, P1, 0, Bk, 0, PB);
        mm(m, n, m, Bk, 1, PB, 0, G);
        for (size_t i = 0; i < mm_; ++i) G[i] += Rk[i];
        /* H = S + B^T P A */
        mm(n, n, n, P1, 0, Ak, 0, PA);
        mm(m, n, n, Bk, 1, PA, 0, H);
        for (size_t i = 0; i < nm; ++i) H[i] += Sk[i];
        /* h = B^T (p + P c) + r */
        mv(m, n, Bk, 1, Pc, h);
        for (int i = 0; i < m; ++i) h[i] += rk[i];
        /* K = -G^{-1} H, k = -G^{-1} h */
        if (chol(m, G) != 0) { status = -1; break; }
        double *Kk = K + k * nm, *kk = kf + (size_t)k * m;
        for (size_t i = 0; i < nm; ++i) Kk[i] = -H[i];
        for (int i = 0; i < m; ++i) kk[i] = -h[i];
        chol_solve(m, G, n, Kk);
        chol_solve(m, G, 1, kk);
        /* P_k = Q + A^T P A + K^T H */
        double *Pk = P + k * nn, *pk = p + (size_t)k * n;
        mm(n, n, n, Ak, 1, PA, 0, Pk);
        mm(n, m, n, Kk, 1, H, 0, tmp);
        for (size_t i = 0; i < nn; ++i) Pk[i] += Qk[i] + tmp[i];
        /* p_k = q + A^T (p + P c) + K^T h */
        mv(n, n, Ak, 1, Pc, pk);
        mv(n, m, Kk, 1, h, tmpv);
        for (int i = 0; i < n; ++i) pk[i] += qk[i] + tmpv[i];
    }

    if (status == 0) {
        /* forward rollout: du_k = K dx_k + k, dx_{k+1} = A dx + B du + c */
        memcpy(dx, s, n * sizeof(double));
        for (int k = 0; k < N; ++k) {
            const double *xk = dx + (size_t)k * n;
            double *uk = du + (size_t)k * m, *x1 = dx + (size_t)(k + 1) * n;
            mv(m, n, K + k * nm, 0, xk, uk);
            for (int i = 0; i < m; ++i) uk[i] += kf[(size_t)k * m + i];
            mv(n, n, A + k * nn, 0, xk, x1);
            mv(n, m, B + k * nm, 0, uk, tmpv);
            for (int i = 0; i < n; ++i) x1[i] += tmpv[i] + c[(size_t)k * n + i];
        }
        for (int i = 0; i < m; ++i) du[(size_t)N * m + i] = 0.0;
        /* costates: dlam_k = P_k dx_k + p_k */
        for (int k = 0; k <= N; ++k) {
            double *lk = dlam + (size_t)k * n;
            mv(n, n, P + k * nn, 0, dx + (size_t)k * n, lk);
            for (int i = 0; i < n; ++i) lk[i] += p[(size_t)k * n + i];
        }
        if (K_out) memcpy(K_out, K, (N + 1) * nm * sizeof(double));
        if (k_out) memcpy(k_out, kf, (N + 1) * (size_t)m * sizeof(double));
        if (P_out) memcpy(P_out, P, (N + 1) * nn * sizeof(double));
        if (p_out) memcpy(p_out, p, (N + 1) * (size_t)n * sizeof(double));
    }

    free(P); free(p); free(K); free(kf); free(G); free(H); free(h);
    free(PB); free(PA); free(Pc); free(tmp); free(tmpv);
    return status;
}

/* --------------------------------------------------------- KKT residual */

static double amax(double a, double b) { return a > b ? a : b; }

void orc_kkt_residual(int n, int m, int N,
                      const double *A, const double *B, const double *c,
                      const double *Q, const double *R, const double *S,
                      const double *q, const double *r, const double *s,
                      const double *dx, const double *du, const double *dlam,
                      double out[4])
{
    const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
    double res = 0.0, knorm = 1.0, znorm = 0.0, rhs = 0.0;

    /* initial condition: dx_0 = s */
    for (int i = 0; i < n; ++i) {
        res = amax(res, fabs(s[i] - dx[i]));
        rhs = amax(rhs, fabs(s[i]));
    }
    for (int k = 0; k < N; ++k) {
        const double *Ak = A + k * nn, *Bk = B + k * nm, *Qk = Q + k * nn;
        const double *Rk = R + k * mm_, *Sk = S + k * nm;
        const double *xk = dx + (size_t)k * n, *uk = du + (size_t)k * m;
        const double *lk = dlam + (size_t)k * n, *l1 = dlam + (size_t)(k + 1) * n;
        /* d/dx_k: Q x + S^T u + q + A^T lam_{k+1} - lam_k = 0 */
        for (int i = 0; i < n; ++i) {
            double v = q[(size_t)k * n + i] - lk[i], row = 1.0;
            for (int j = 0; j < n; ++j) {
                v += Qk[i * n + j] * xk[j] + Ak[j * n + i] * l1[j];
                row += fabs(Qk[i * n + j]) + fabs(Ak[j * n + i]);
            }
            for (int j = 0; j < m; ++j) {
                v += Sk[j * n + i] * uk[j];
                row += fabs(Sk[j * n + i]);
            }
            res = amax(res, fabs(v));
            knorm = amax(knorm, row);
            rhs = amax(rhs, fabs(q[(size_t)k * n + i]));
        }
        /* d/du_k: S x + R u + r + B^T lam_{k+1} = 0 */
        for (int i = 0; i < m; ++i) {
            double v = r[(size_t)k * m + i], row = 0.0;
            for (int j = 0; j < n; ++j) {
                v += Sk[i * n + j] * xk[j] + Bk[j * m + i] * l1[j];
                row += fabs(Sk[i * n + j]) + fabs(Bk[j * m + i]);
            }
            for (int j = 0; j < m; ++j) {
                v += Rk[i * m + j] * uk[j];
                row += fabs(Rk[i * m + j]);
            }
            res = amax(res, fabs(v));
            knorm = amax(knorm, row);
            rhs = amax(rhs, fabs(r[(size_t)k * m + i]));
        }
        /* dynamics: A x + B u + c - x_{k+1} = 0 */
        for (int i = 0; i < n; ++i) {
            double v = c[(size_t)k * n + i] - dx[(size_t)(k + 1) * n + i];
            double row = 1.0;
            for (int j = 0; j < n; ++j) {
                v += Ak[i * n + j] * xk[j];
                row += fabs(Ak[i * n + j]);
            }
            for (int j = 0; j < m; ++j) {
                v += Bk[i * m + j] * uk[j];
                row += fabs(Bk[i * m + j]);
            }
            res = amax(res, fabs(v));
            knorm = amax(knorm, row);
            rhs = amax(rhs, fabs(c[(size_t)k * n + i]));
        }
    }
    /* terminal: Q_N x_N + q_N - lam_N = 0 */
    for (int i = 0; i < n; ++i) {
        const double *QN = Q + N * nn;
        double v = q[(size_t)N * n + i] - dlam[(size_t)N * n + i], row = 1.0;
        for (int j = 0; j < n; ++j) {
            v += QN[i * n + j] * dx[(size_t)N * n + j];
            row += fabs(QN[i * n + j]);
        }
        res = amax(res, fabs(v));
        knorm = amax(knorm, row);
        rhs = amax(rhs, fabs(q[(size_t)N * n + i]));
    }
    for (int k = 0; k <= N; ++k) {
        for (int i = 0; i < n; ++i) {
            znorm = amax(znorm, fabs(dx[(size_t)k * n + i]));
            znorm = amax(znorm, fabs(dlam[(size_t)k * n + i]));
        }
        if (k < N)
            for (int i = 0; i < m; ++i) znorm = amax(znorm, fabs(du[(size_t)k * m + i]));
    }
    out[0] = res; out[1] = knorm; out[2] = znorm; out[3] = rhs;
}

/* ----------------------------------------------- relaxed barrier, Sec. II-F */

void orc_barrier(double xi, double mu, double delta, double out[3])
{
    if (xi >= delta) {
        out[0] = -mu * log(xi);
        out[1] = -mu / xi;
        out[2] = mu / (xi * xi);
    } else {
        double t = (xi - 2.0 * delta) / delta;
        out[0] = 0.5 * mu * (t * t - 1.0) - mu * log(delta);
        out[1] = mu * t / delta;
        out[2] = mu / (delta * delta);
    }
}

/* ------------------------------------------------------------ SRBD model */
/* Per robot: x = [p, theta, v, omega], u = [f_0, f_1, f_2, f_3];
 *   p' = v,  theta' = omega,  v' = sum_j s_j f_j / mass + g,
 *   omega' = I^{-1} ( sum_j s_j (r_j - p) x f_j - omega x (I omega) ),
 * integrated by one explicit Euler step of length dt. */

static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* skew(a) b = a x b */
static void skew3(const double *a, double *M)
{
    M[0] = 0.0;   M[1] = -a[2]; M[2] = a[1];
    M[3] = a[2];  M[4] = 0.0;   M[5] = -a[0];
    M[6] = -a[1]; M[7] = a[0];  M[8] = 0.0;
}

static int srbd_n(const orc_srbd_params *prm) { return 12 * prm->nrob; }

void orc_srbd_step(const orc_srbd_params *prm, const double *x,
                   const double *u, const unsigned char *contact,
                   double *x_next)
{
    for (int b = 0; b < prm->nrob; ++b) {
        const double *xb = x + 12 * b, *ub = u + 12 * b;
        const unsigned char *sb = contact + 4 * b;
        const double *p = xb, *th = xb + 3, *v = xb + 6, *w = xb + 9;
        double f_sum[3] = {0, 0, 0}, tau[3] = {0, 0, 0};
        for (int j = 0; j < 4; ++j) {
            if (!sb[j]) continue;
            const double *f = ub + 3 * j;
            double arm[3], t[3];
            for (int i = 0; i < 3; ++i) arm[i] = prm->foot[j][i] - p[i];
            cross3(arm, f, t);
            for (int i = 0; i < 3; ++i) { f_sum[i] += f[i]; tau[i] += t[i]; }
        }
        double Iw[3], gyro[3];
        for (int i = 0; i < 3; ++i) Iw[i] = prm->inertia[i] * w[i];
        cross3(w, Iw, gyro);
        double *xn = x_next + 12 * b;
        for (int i = 0; i < 3; ++i) {
            double vdot = f_sum[i] / prm->mass - (i == 2 ? prm->gravity : 0.0);
            double wdot = (tau[i] - gyro[i]) / prm->inertia[i];
            xn[i] = p[i] + prm->dt * v[i];
            xn[3 + i] = th[i] + prm->dt * w[i];
            xn[6 + i] = v[i] + prm->dt * vdot;
            xn[9 + i] = w[i] + prm->dt * wdot;
        }
    }
}

void orc_srbd_jacobians(const orc_srbd_params *prm, const double *x,
                        const double *u, const unsigned char *contact,
                        double *A, double *B)
{
    const int n = srbd_n(prm), m = n;
    const double dt = prm->dt;
    memset(A, 0, sizeof(double) * n * n);
    memset(B, 0, sizeof(double) * n * m);
    for (int i = 0; i < n; ++i) A[i * n + i] = 1.0;
    for (int b = 0; b < prm->nrob; ++b) {
        const int o = 12 * b;
        const double *xb = x + o, *ub = u + o;
        const unsigned char *sb = contact + 4 * b;
        const double *p = xb, *w = xb + 9;
        /* dp'/dv = I, dtheta'/domega = I */
        for (int i = 0; i < 3; ++i) {
            A[(o + i) * n + (o + 6 + i)] += dt;
            A[(o + 3 + i) * n + (o + 9 + i)] += dt;
        }
        /* d omega'/dp = I^{-1} sum_j s_j skew(f_j)  [ (r-p) x f = r x f + f x p ] */
        double Fs[9];
        for (int j = 0; j < 4; ++j) {
            if (!sb[j]) continue;
            skew3(ub + 3 * j, Fs);
            for (int i = 0; i < 3; ++i)
                for (int l = 0; l < 3; ++l)
                    A[(o + 9 + i) * n + (o + l)] += dt * Fs[i * 3 + l] / prm->inertia[i];
        }
        /* d omega'/d omega = -I^{-1} ( skew(w) I - skew(I w) ) */
        double Sw[9], SIw[9], Iw[3];
        for (int i = 0; i < 3; ++i) Iw[i] = prm->inertia[i] * w[i];
        skew3(w, Sw);
        skew3(Iw, SIw);
        for (int i = 0; i < 3; ++i)
            for (int l = 0; l < 3; ++l) {
                double d = Sw[i * 3 + l] * prm->inertia[l] - SIw[i * 3 + l];
                A[(o + 9 + i) * n + (o + 9 + l)] -= dt * d / prm->inertia[i];
            }
        /* dv'/df_j = s_j I / mass,  d omega'/df_j = s_j I^{-1} skew(r_j - p) */
        for (int j = 0; j < 4; ++j) {
            if (!sb[j]) continue;
            double arm[3], Sa[9];
            for (int i = 0; i < 3; ++i) arm[i] = prm->foot[j][i] - p[i];
            skew3(arm, Sa);
            for (int i = 0; i < 3; ++i) {
                B[(o + 6 + i) * m + (o + 3 * j + i)] += dt / prm->mass;
                for (int l = 0; l < 3; ++l)
                    B[(o + 9 + i) * m + (o + 3 * j + l)] += dt * Sa[i * 3 + l] / prm->inertia[i];
            }
        }
    }
}

/* Friction pyramid of one stance foot: xi_c = G_c . f >= 0, five rows:
 * mu fz + fx, mu fz - fx, mu fz + fy, mu fz - fy, fz. */
static void cone_rows(double mu, double G[5][3])
{
    double rows[5][3] = {{1, 0, mu}, {-1, 0, mu}, {0, 1, mu}, {0, -1, mu}, {0, 0, 1}};
    memcpy(G, rows, sizeof(rows));
}

/* formation residual e_a = p_a - p_{a+1} - d_a for robot a (nrob >= 2) */
static void form_residual(const orc_srbd_params *prm, const double *x, int a,
                          double *e)
{
    int b = (a + 1) % prm->nrob;
    for (int i = 0; i < 3; ++i)
        e[i] = x[12 * a + i] - x[12 * b + i] - prm->d_form[a][i];
}

double orc_srbd_cost(const orc_srbd_params *prm, const double *x,
                     const double *u, const unsigned char *contact,
                     const double *xref, const double *uref, int terminal)
{
    const int n = srbd_n(prm);
    const double *Wx = terminal ? prm->WN : prm->W;
    double J = 0.0;
    for (int i = 0; i < n; ++i) {
        double d = x[i] - xref[i];
        J += 0.5 * Wx[i % 12] * d * d;
    }
    if (prm->nrob >= 2)
        for (int a = 0; a < prm->nrob; ++a) {
            double e[3];
            form_residual(prm, x, a, e);
            J += 0.5 * prm->w_form * (e[0] * e[0] + e[1] * e[1] + e[2] * e[2]);
        }
    if (!terminal) {
        double G[5][3];
        cone_rows(prm->mu_fric, G);
        for (int i = 0; i < n; ++i) {
            double d = u[i] - uref[i];
            J += 0.5 * prm->Wu[i % 12] * d * d;
        }
        for (int b = 0; b < prm->nrob; ++b)
            for (int j = 0; j < 4; ++j) {
                if (!contact[4 * b + j]) continue;
                const double *f = u + 12 * b + 3 * j;
                for (int c = 0; c < 5; ++c) {
                    double xi = G[c][0] * f[0] + G[c][1] * f[1] + G[c][2] * f[2];
                    double bv[3];
                    orc_barrier(xi, prm->bar_mu, prm->bar_delta, bv);
                    J += bv[0];
                }
            }
    }
    return J;
}

/* Cost gradient and Gauss-Newton Hessian of one stage (Sec. II-F):
 * gx = W (x - xref) [+ formation], Hxx = W [+ formation];
 * gu = Wu (u - uref) + sum B'(xi) grad xi, Huu = Wu + sum B''(xi) grad xi grad xi^T.
 * The model has no state-control cross term (S = 0). */
static void srbd_cost_derivs(const orc_srbd_params *prm, const double *x,
                             const double *u, const unsigned char *contact,
                             const double *xref, const double *uref,
                             int terminal, double *gx, double *Hxx,
                             double *gu, double *Huu)
{
    const int n = srbd_n(prm), m = n;
    const double *Wx = terminal ? prm->WN : prm->W;
    memset(Hxx, 0, sizeof(double) * n * n);
    for (int i = 0; i < n; ++i) {
        gx[i] = Wx[i % 12] * (x[i] - xref[i]);
        Hxx[i * n + i] = Wx[i % 12];
    }
    if (prm->nrob >= 2)
        for (int a = 0; a < prm->nrob; ++a) {
            int b = (a + 1) % prm->nrob;
            double e[3];
            form_residual(prm, x, a, e);
            for (int i = 0; i < 3; ++i) {
                int ia = 12 * a + i, ib = 12 * b + i;
                gx[ia] += prm->w_form * e[i];
                gx[ib] -= prm->w_form * e[i];
                Hxx[ia * n + ia] += prm->w_form;
                Hxx[ib * n + ib] += prm->w_form;
                Hxx[ia * n + ib] -= prm->w_form;
                Hxx[ib * n + ia] -= prm->w_form;
            }
        }
    if (terminal) return;
    memset(Huu, 0, sizeof(double) * m * m);
    for (int i = 0; i < m; ++i) {
        gu[i] = prm->Wu[i % 12] * (u[i] - uref[i]);
        Huu[i * m + i] = prm->Wu[i % 12];
    }
    double G[5][3];
    cone_rows(prm->mu_fric, G);
    for (int b = 0; b < prm->nrob; ++b)
        for (int j = 0; j < 4; ++j) {
            if (!contact[4 * b + j]) continue;
            const int o = 12 * b + 3 * j;
            const double *f = u + o;
            for (int c = 0; c < 5; ++c) {
                double xi = G[c][0] * f[0] + G[c][1] * f[1] + G[c][2] * f[2];
                double bv[3];
                orc_barrier(xi, prm->bar_mu, prm->bar_delta, bv);
                for (int i = 0; i < 3; ++i) {
                    gu[o + i] += bv[1] * G[c][i];
                    for (int l = 0; l < 3; ++l)
                        Huu[(o + i) * m + (o + l)] += bv[2] * G[c][i] * G[c][l];
                }
            }
        }
}

void orc_srbd_linearize(const orc_srbd_params *prm, int N,
                        const double *x, const double *u, const double *lam,
                        const double *xref, const double *uref,
                        const unsigned char *contact,
                        double *A, double *B, double *c, double *Q,
                        double *R, double *S, double *q, double *r)
{
    const int n = srbd_n(prm), m = n, nc = 4 * prm->nrob;
    const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
    double *hx = dalloc(n), *tmp = dalloc(n);
    memset(A, 0, sizeof(double) * (N + 1) * nn);
    memset(B, 0, sizeof(double) * (N + 1) * nm);
    memset(c, 0, sizeof(double) * (N + 1) * n);
    memset(R, 0, sizeof(double) * (N + 1) * mm_);
    memset(S, 0, sizeof(double) * (N + 1) * nm);
    memset(r, 0, sizeof(double) * (N + 1) * m);
    for (int k = 0; k < N; ++k) {
        const double *xk = x + (size_t)k * n, *uk = u + (size_t)k * m;
        const unsigned char *ck = contact + (size_t)k * nc;
        double *Ak = A + k * nn, *Bk = B + k * nm;
        orc_srbd_jacobians(prm, xk, uk, ck, Ak, Bk);
        /* defect b_k = h(x_k, u_k) - x_{k+1} */
        orc_srbd_step(prm, xk, uk, ck, hx);
        for (int i = 0; i < n; ++i) c[(size_t)k * n + i] = hx[i] - x[(size_t)(k + 1) * n + i];
        /* Hessian blocks and Lagrangian gradients:
         * q = grad_x l + A^T lam_{k+1} - lam_k,  r = grad_u l + B^T lam_{k+1} */
        double *qk = q + (size_t)k * n, *rk = r + (size_t)k * m;
        srbd_cost_derivs(prm, xk, uk, ck, xref + (size_t)k * n, uref + (size_t)k * m,
                         0, qk, Q + k * nn, rk, R + k * mm_);
        const double *l1 = lam + (size_t)(k + 1) * n, *l0 = lam + (size_t)k * n;
        mv(n, n, Ak, 1, l1, tmp);
        for (int i = 0; i < n; ++i) qk[i] += tmp[i] - l0[i];
        mv(m, n, Bk, 1, l1, tmp);
        for (int i = 0; i < m; ++i) rk[i] += tmp[i];
    }
    /* terminal: Q_N = grad^2 l_N, q_N = grad l_N - lam_N */
    srbd_cost_derivs(prm, x + (size_t)N * n, NULL, NULL, xref + (size_t)N * n, NULL,
                     1, q + (size_t)N * n, Q + N * nn, NULL, NULL);
    for (int i = 0; i < n; ++i) q[(size_t)N * n + i] -= lam[(size_t)N * n + i];
    free(hx); free(tmp);
}

void orc_srbd_merit(const orc_srbd_params *prm, int N, const double *x0hat,
                    const double *x, const double *u, const double *xref,
                    const double *uref, const unsigned char *contact,
                    double *J_out, double *theta_out)
{
    const int n = srbd_n(prm), m = n, nc = 4 * prm->nrob;
    double *hx = dalloc(n);
    double J = 0.0, theta = 0.0, d2 = 0.0;
    for (int i = 0; i < n; ++i) d2 += (x0hat[i] - x[i]) * (x0hat[i] - x[i]);
    theta += sqrt(d2);
    for (int k = 0; k < N; ++k) {
        const double *xk = x + (size_t)k * n, *uk = u + (size_t)k * m;
        const unsigned char *ck = contact + (size_t)k * nc;
        J += orc_srbd_cost(prm, xk, uk, ck, xref + (size_t)k * n, uref + (size_t)k * m, 0);
        orc_srbd_step(prm, xk, uk, ck, hx);
        d2 = 0.0;
        for (int i = 0; i < n; ++i) {
            double d = x[(size_t)(k + 1) * n + i] - hx[i];
            d2 += d * d;
        }
        theta += sqrt(d2);
    }
    J += orc_srbd_cost(prm, x + (size_t)N * n, NULL, NULL, xref + (size_t)N * n, NULL, 1);
    *J_out = J;
    *theta_out = theta;
    free(hx);
}

/* ------------------------------------------------ filter line search */
/* Sec. II-E: above theta_max a step must lower theta; below it, a descent
 * direction must satisfy Armijo (and keep theta under theta_max); a
 * non-descent direction must lower the cost or theta. */
int orc_filter_accept(double J0, double th0, double dphi, double th_max,
                      double alpha, double Ja, double tha, double c_armijo)
{
    if (!(isfinite(Ja) && isfinite(tha))) return 0;
    if (th0 > th_max) return tha < th0;
    if (dphi < 0.0) return (Ja <= J0 + c_armijo * alpha * dphi) && (tha <= th_max);
    return (Ja < J0) || (tha < th0);
}

/* A model seen by the SQP loop: linearisation, merit and cost gradient. */
typedef struct {
    int n, m, N;
    void (*linearize)(const void *ctx, const double *x, const double *u,
                      const double *lam, double *A, double *B, double *c,
                      double *Q, double *R, double *S, double *q, double *r);
    void (*merit)(const void *ctx, const double *x0hat, const double *x,
                  const double *u, double *J, double *theta);
    /* directional derivative of the cost (not the Lagrangian) along dz */
    double (*dcost)(const void *ctx, const double *x, const double *u,
                    const double *dx, const double *du);
    const void *ctx;
} sqp_model;

static int sqp_run(const sqp_model *mdl, const double *x0hat, double *x,
                   double *u, double *lam, const orc_sqp_opts *opt,
                   orc_sqp_info *info)
{
    const int n = mdl->n, m = mdl->m, N = mdl->N;
    const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
    const size_t S1 = (size_t)N + 1;
    double *A = dalloc(S1 * nn), *B = dalloc(S1 * nm), *c = dalloc(S1 * n);
    double *Q = dalloc(S1 * nn), *R = dalloc(S1 * mm_), *S = dalloc(S1 * nm);
    double *q = dalloc(S1 * n), *r = dalloc(S1 * m), *s = dalloc(n);
    double *dx = dalloc(S1 * n), *du = dalloc(S1 * m), *dl = dalloc(S1 * n);
    double *xt = dalloc(S1 * n), *ut = dalloc(S1 * m);
    memset(info, 0, sizeof(*info));

    double J0, th0;
    mdl->merit(mdl->ctx, x0hat, x, u, &J0, &th0);
    const double th_max = opt->theta_frac * (th0 > 1.0 ? th0 : 1.0);
    info->theta_max = th_max;

    for (int it = 0; it < opt->max_iters && it < 32; ++it) {
        mdl->linearize(mdl->ctx, x, u, lam, A, B, c, Q, R, S, q, r);
        for (int i = 0; i < n; ++i) s[i] = x0hat[i] - x[i];
        if (orc_riccati_solve(n, m, N, A, B, c, Q, R, S, q, r, s, dx, du, dl,
                              NULL, NULL, NULL, NULL) != 0) {
            info->status = 2;
            break;
        }
        info->iters = it + 1;
        double step = 0.0;
        for (size_t i = 0; i < S1 * n; ++i) step = amax(step, fabs(dx[i]));
        for (size_t i = 0; i < (size_t)N * m; ++i) step = amax(step, fabs(du[i]));
        info->step[it] = step;
        info->theta_it[it] = th0;
        const double dphi = mdl->dcost(mdl->ctx, x, u, dx, du);
        /* the ten step sizes 2^0 .. 2^-9; the largest accepted one wins */
        double alpha = 0.0;
        if (opt->alpha_replay) {
            alpha = opt->alpha_replay[it];
        } else {
            for (int t = 0; t < 10; ++t) {
                double a = ldexp(1.0, -t), Ja, tha;
                for (size_t i = 0; i < S1 * n; ++i) xt[i] = x[i] + a * dx[i];
                for (size_t i = 0; i < S1 * m; ++i) ut[i] = u[i] + a * du[i];
                mdl->merit(mdl->ctx, x0hat, xt, ut, &Ja, &tha);
                if (orc_filter_accept(J0, th0, dphi, th_max, a, Ja, tha, opt->c_armijo)) {
                    alpha = a;
                    break;
                }
            }
        }
        info->alpha[it] = alpha;
        if (alpha == 0.0) {
            /* no step accepted: converged if theta is at the rounding floor of
             * the iterate, (N+1) sqrt(n) u max(1, |x|_inf), u = 2^-52 */
            double xmax = 0.0;
            for (size_t i = 0; i < S1 * n; ++i) xmax = amax(xmax, fabs(x[i]));
            double floor_th = (double)(N + 1) * sqrt((double)n) * ldexp(1.0, -52) *
                              (xmax > 1.0 ? xmax : 1.0);
            if (!(opt->alpha_replay) && th0 <= floor_th) break;
            info->status = 1;
            break;
        }
        /* Eq. (linear_rollout) */
        for (size_t i = 0; i < S1 * n; ++i) x[i] += alpha * dx[i];
        for (size_t i = 0; i < (size_t)N * m; ++i) u[i] += alpha * du[i];
        for (size_t i = 0; i < S1 * n; ++i) lam[i] += alpha * dl[i];
        mdl->merit(mdl->ctx, x0hat, x, u, &J0, &th0);
        if (step < opt->tol_step && th0 < opt->tol_theta) break;
    }
    info->J = J0;
    info->theta = th0;

    free(A); free(B); free(c); free(Q); free(R); free(S); free(q); free(r); free(s);
    free(dx); free(du); free(dl); free(xt); free(ut);
    return info->status;
}

/* SRBD adapter */
typedef struct {
    const orc_srbd_params *prm;
    int N;
    const double *xref, *uref;
    const unsigned char *contact;
} srbd_ctx;

static void srbd_lin_cb(const void *ctx, const double *x, const double *u,
                        const double *lam, double *A, double *B, double *c,
                        double *Q, double *R, double *S, double *q, double *r)
{
    const srbd_ctx *t = (const srbd_ctx *)ctx;
    orc_srbd_linearize(t->prm, t->N, x, u, lam, t->xref, t->uref, t->contact,
                       A, B, c, Q, R, S, q, r);
}

static void srbd_merit_cb(const void *ctx, const double *x0hat, const double *x,
                          const double *u, double *J, double *theta)
{
    const srbd_ctx *t = (const srbd_ctx *)ctx;
    orc_srbd_merit(t->prm, t->N, x0hat, x, u, t->xref, t->uref, t->contact, J, theta);
}

static double srbd_dcost_cb(const void *ctx, const double *x, const double *u,
                            const double *dx, const double *du)
{
    const srbd_ctx *t = (const srbd_ctx *)ctx;
    const int n = srbd_n(t->prm), m = n, nc = 4 * t->prm->nrob, N = t->N;
    double *gx = dalloc(n), *gu = dalloc(m);
    double *Hx = dalloc((size_t)n * n), *Hu = dalloc((size_t)m * m);
    double dphi = 0.0;
    for (int k = 0; k <= N; ++k) {
        int term = (k == N);
        srbd_cost_derivs(t->prm, x + (size_t)k * n, term ? NULL : u + (size_t)k * m,
                         term ? NULL : t->contact + (size_t)k * nc, t->xref + (size_t)k * n,
                         term ? NULL : t->uref + (size_t)k * m, term, gx, Hx, gu, Hu);
        for (int i = 0; i < n; ++i) dphi += gx[i] * dx[(size_t)k * n + i];
        if (!term)
            for (int i = 0; i < m; ++i) dphi += gu[i] * du[(size_t)k * m + i];
    }
    free(gx); free(gu); free(Hx); free(Hu);
    return dphi;
}

int orc_srbd_sqp(const orc_srbd_params *prm, int N, const double *x0hat,
                 double *x, double *u, double *lam,
                 const double *xref, const double *uref,
                 const unsigned char *contact, const orc_sqp_opts *opt,
                 orc_sqp_info *info)
{
    srbd_ctx t = {prm, N, xref, uref, contact};
    sqp_model mdl = {srbd_n(prm), srbd_n(prm), N, srbd_lin_cb, srbd_merit_cb,
                     srbd_dcost_cb, &t};
    return sqp_run(&mdl, x0hat, x, u, lam, opt, info);
}

/* ------------------------------------------------------------ LTV model */
/* h_k(x,u) = A_k x + B_k u + e_k;
 * l_k = 0.5 x^T Q_k x + u^T S_k x + 0.5 u^T R_k u + gq_k^T x + gr_k^T u,
 * l_N = 0.5 x^T Q_N x + gq_N^T x.  All arrays use the N+1-slot layout. */
typedef struct {
    int n, m, N;
    const double *A, *B, *e, *Q, *R, *S, *gq, *gr;
} ltv_ctx;

static double ltv_stage(const ltv_ctx *t, int k, const double *x,
                        const double *u, double *gx, double *gu)
{
    const int n = t->n, m = t->m;
    const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
    const double *Q = t->Q + k * nn;
    double J = 0.0;
    for (int i = 0; i < n; ++i) {
        double v = t->gq[(size_t)k * n + i];
        for (int j = 0; j < n; ++j) v += Q[i * n + j] * x[j];
        if (k < t->N)
            for (int j = 0; j < m; ++j) v += t->S[k * nm + j * n + i] * u[j];
        gx[i] = v;
        J += x[i] * (0.5 * (v - t->gq[(size_t)k * n + i]) + t->gq[(size_t)k * n + i]);
    }
    if (k < t->N) {
        const double *R = t->R + k * mm_, *S = t->S + k * nm;
        for (int i = 0; i < m; ++i) {
            double v = t->gr[(size_t)k * m + i], vr = 0.0;
            for (int j = 0; j < m; ++j) vr += R[i * m + j] * u[j];
            for (int j = 0; j < n; ++j) v += S[i * n + j] * x[j];
            gu[i] = v + vr;
            J += u[i] * (0.5 * vr + t->gr[(size_t)k * m + i]);
        }
        /* x-part above counted 0.5 u^T S x; add the other half */
        for (int i = 0; i < m; ++i)
            for (int j = 0; j < n; ++j) J += 0.5 * u[i] * S[i * n + j] * x[j];
    }
    return J;
}

static void ltv_step(const ltv_ctx *t, int k, const double *x, const double *u,
                     double *xn)
{
    const int n = t->n, m = t->m;
    const double *A = t->A + (size_t)k * n * n, *B = t->B + (size_t)k * n * m;
    for (int i = 0; i < n; ++i) {
        double v = t->e[(size_t)k * n + i];
        for (int j = 0; j < n; ++j) v += A[i * n + j] * x[j];
        for (int j = 0; j < m; ++j) v += B[i * m + j] * u[j];
        xn[i] = v;
    }
}

static void ltv_lin_cb(const void *ctx, const double *x, const double *u,
                       const double *lam, double *A, double *B, double *c,
                       double *Q, double *R, double *S, double *q, double *r)
{
    const ltv_ctx *t = (const ltv_ctx *)ctx;
    const int n = t->n, m = t->m, N = t->N;
    const size_t nn = (size_t)n * n, nm = (size_t)n * m, mm_ = (size_t)m * m;
    memcpy(A, t->A, (N + 1) * nn * sizeof(double));
    memcpy(B, t->B, (N + 1) * nm * sizeof(double));
    memcpy(Q, t->Q, (N + 1) * nn * sizeof(double));
    memcpy(R, t->R, (N + 1) * mm_ * sizeof(double));
    memcpy(S, t->S, (N + 1) * nm * sizeof(double));
    memset(c, 0, (N + 1) * (size_t)n * sizeof(double));
    memset(r, 0, (N + 1) * (size_t)m * sizeof(double));
    double *hx = dalloc(n), *tmp = dalloc(n > m ? n : m);
    for (int k = 0; k <= N; ++k) {
        const double *xk = x + (size_t)k * n, *uk = u + (size_t)k * m;
        double *qk = q + (size_t)k * n, *rk = r + (size_t)k * m;
        ltv_stage(t, k, xk, uk, qk, rk);
        for (int i = 0; i < n; ++i) qk[i] -= lam[(size_t)k * n + i];
        if (k == N) break;
        ltv_step(t, k, xk, uk, hx);
        for (int i = 0; i < n; ++i) c[(size_t)k * n + i] = hx[i] - x[(size_t)(k + 1) * n + i];
        const double *l1 = lam + (size_t)(k + 1) * n;
        mv(n, n, A + k * nn, 1, l1, tmp);
        for (int i = 0; i < n; ++i) qk[i] += tmp[i];
        mv(m, n, B + k * nm, 1, l1, tmp);
        for (int i = 0; i < m; ++i) rk[i] += tmp[i];
    }
    free(hx); free(tmp);
}

static void ltv_merit_cb(const void *ctx, const double *x0hat, const double *x,
                         const double *u, double *J, double *theta)
{
    const ltv_ctx *t = (const ltv_ctx *)ctx;
    const int n = t->n, m = t->m, N = t->N;
    double *hx = dalloc(n), *gx = dalloc(n), *gu = dalloc(m);
    double Jv = 0.0, th = 0.0, d2 = 0.0;
    for (int i = 0; i < n; ++i) d2 += (x0hat[i] - x[i]) * (x0hat[i] - x[i]);
    th += sqrt(d2);
    for (int k = 0; k <= N; ++k) {
        Jv += ltv_stage(t, k, x + (size_t)k * n, u + (size_t)k * m, gx, gu);
        if (k == N) break;
        ltv_step(t, k, x + (size_t)k * n, u + (size_t)k * m, hx);
        d2 = 0.0;
        for (int i = 0; i < n; ++i) {
            double d = x[(size_t)(k + 1) * n + i] - hx[i];
            d2 += d * d;
        }
        th += sqrt(d2);
    }
    *J = Jv;
    *theta = th;
    free(hx); free(gx); free(gu);
}

static double ltv_dcost_cb(const void *ctx, const double *x, const double *u,
                           const double *dx, const double *du)
{
    const ltv_ctx *t = (const ltv_ctx *)ctx;
    const int n = t->n, m = t->m, N = t->N;
    double *gx = dalloc(n), *gu = dalloc(m), d = 0.0;
    for (int k = 0; k <= N; ++k) {
        ltv_stage(t, k, x + (size_t)k * n, u + (size_t)k * m, gx, gu);
        for (int i = 0; i < n; ++i) d += gx[i] * dx[(size_t)k * n + i];
        if (k < N)
            for (int i = 0; i < m; ++i) d += gu[i] * du[(size_t)k * m + i];
    }
    free(gx); free(gu);
    return d;
}

double orc_ltv_cost(int n, int m, int N, const double *Q, const double *R,
                    const double *S, const double *gq, const double *gr,
                    const double *x, const double *u)
{
    ltv_ctx t = {n, m, N, NULL, NULL, NULL, Q, R, S, gq, gr};
    double *gx = dalloc(n), *gu = dalloc(m), J = 0.0;
    for (int k = 0; k <= N; ++k) J += ltv_stage(&t, k, x + (size_t)k * n, u + (size_t)k * m, gx, gu);
    free(gx); free(gu);
    return J;
}

int orc_ltv_sqp(int n, int m, int N, const double *A, const double *B,
                const double *e, const double *Q, const double *R,
                const double *S, const double *gq, const double *gr,
                const double *x0hat, double *x, double *u, double *lam,
                const orc_sqp_opts *opt, orc_sqp_info *info)
{
    ltv_ctx t = {n, m, N, A, B, e, Q, R, S, gq, gr};
    sqp_model mdl = {n, m, N, ltv_lin_cb, ltv_merit_cb, ltv_dcost_cb, &t};
    return sqp_run(&mdl, x0hat, x, u, lam, opt, info);
}
