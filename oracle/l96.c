/*
 * FP64 reference integrators for the Lorenz-96 system (oracle; test
 * infrastructure only, never linked into the GPU library).
 *
 * Model (Section 3.1, Eq. "L-96"): dx_i/dt = (x_{i+1} - x_{i-2}) x_{i-1} - x_i + F
 * with periodic indices.  Time stepping is the classical four-stage
 * Runge-Kutta scheme (the paper does not name its integrator; RK4 is the
 * stepping the workloads prescribe):
 *     k1 = f(x), k2 = f(x + dt/2 k1), k3 = f(x + dt/2 k2), k4 = f(x + dt k3),
 *     x+ = x + dt/6 (k1 + 2 k2 + 2 k3 + k4).
 * The tangent-linear (TL) model is the derivative of one RK4 step with
 * respect to x (chain rule through the stages); the adjoint (AD) is its exact
 * transpose, run backward in time with the base stages recomputed from the
 * stored trajectory (Section 2.3, Algorithms 1-3: "integrate and store
 * trajectory", H_{k-1} tangent linear, H_{k-1}^T adjoint).
 *
 * Written for clarity, not speed: one state at a time, no blocking.
 */
#include <stdlib.h>
#include <string.h>

static int wrap(int i, int n) { i %= n; return i < 0 ? i + n : i; }

/* f(x): the L-96 tendency. */
void l96_rhs(int n, double F, const double *x, double *f)
{
    for (int i = 0; i < n; ++i) {
        double xp1 = x[wrap(i + 1, n)], xm2 = x[wrap(i - 2, n)], xm1 = x[wrap(i - 1, n)];
        f[i] = (xp1 - xm2) * xm1 - x[i] + F;
    }
}

/* Jacobian of f at X applied to v: d/de f(X + e v) at e = 0 (product rule). */
static void l96_jac(int n, const double *X, const double *v, double *out)
{
    for (int i = 0; i < n; ++i) {
        int ip1 = wrap(i + 1, n), im1 = wrap(i - 1, n), im2 = wrap(i - 2, n);
        out[i] = (v[ip1] - v[im2]) * X[im1] + (X[ip1] - X[im2]) * v[im1] - v[i];
    }
}

/* Transpose of the Jacobian applied to mu, written as a scatter: component
 * f_j depends on x_{j+1}, x_{j-2}, x_{j-1}, x_j, and each partial
 * derivative sends mu_j back to that variable. */
static void l96_jac_t(int n, const double *X, const double *mu, double *out)
{
    for (int i = 0; i < n; ++i) out[i] = 0.0;
    for (int j = 0; j < n; ++j) {
        int jp1 = wrap(j + 1, n), jm1 = wrap(j - 1, n), jm2 = wrap(j - 2, n);
        out[jp1] += mu[j] * X[jm1];                 /* df_j/dx_{j+1} =  x_{j-1} */
        out[jm2] -= mu[j] * X[jm1];                 /* df_j/dx_{j-2} = -x_{j-1} */
        out[jm1] += mu[j] * (X[jp1] - X[jm2]);      /* df_j/dx_{j-1} = x_{j+1} - x_{j-2} */
        out[j]   -= mu[j];                          /* df_j/dx_j     = -1 */
    }
}

/* Base RK4 stage states X1..X4 (each n) of the step starting at x. */
static void rk4_stages(int n, double dt, double F, const double *x, double *X /* 4n */, double *k /* n */)
{
    double *X1 = X, *X2 = X + n, *X3 = X + 2 * n, *X4 = X + 3 * n;
    memcpy(X1, x, sizeof(double) * n);
    l96_rhs(n, F, X1, k);
    for (int i = 0; i < n; ++i) X2[i] = x[i] + 0.5 * dt * k[i];
    l96_rhs(n, F, X2, k);
    for (int i = 0; i < n; ++i) X3[i] = x[i] + 0.5 * dt * k[i];
    l96_rhs(n, F, X3, k);
    for (int i = 0; i < n; ++i) X4[i] = x[i] + dt * k[i];
}

/* Nonlinear trajectory: traj[t*n + i] = x_i at step t, t = 0..T. */
void l96_nl(int n, int T, double dt, double F, const double *x0, double *traj)
{
    double *k1 = malloc(sizeof(double) * n), *k2 = malloc(sizeof(double) * n);
    double *k3 = malloc(sizeof(double) * n), *k4 = malloc(sizeof(double) * n);
    double *s = malloc(sizeof(double) * n);
    memcpy(traj, x0, sizeof(double) * n);
    for (int t = 0; t < T; ++t) {
        const double *x = traj + (size_t)t * n;
        double *xn = traj + (size_t)(t + 1) * n;
        l96_rhs(n, F, x, k1);
        for (int i = 0; i < n; ++i) s[i] = x[i] + 0.5 * dt * k1[i];
        l96_rhs(n, F, s, k2);
        for (int i = 0; i < n; ++i) s[i] = x[i] + 0.5 * dt * k2[i];
        l96_rhs(n, F, s, k3);
        for (int i = 0; i < n; ++i) s[i] = x[i] + dt * k3[i];
        l96_rhs(n, F, s, k4);
        for (int i = 0; i < n; ++i)
            xn[i] = x[i] + dt / 6.0 * (k1[i] + 2.0 * k2[i] + 2.0 * k3[i] + k4[i]);
    }
    free(k1); free(k2); free(k3); free(k4); free(s);
}

/* Tangent-linear trajectory: dxs[t*n + i] = (M_{0->t} dx0)_i, t = 0..T,
 * linearised about the stored trajectory traj. */
void l96_tl(int n, int T, double dt, double F, const double *traj, const double *dx0, double *dxs)
{
    double *X = malloc(sizeof(double) * 4 * n), *kb = malloc(sizeof(double) * n);
    double *d1 = malloc(sizeof(double) * n), *d2 = malloc(sizeof(double) * n);
    double *d3 = malloc(sizeof(double) * n), *d4 = malloc(sizeof(double) * n);
    double *s = malloc(sizeof(double) * n);
    memcpy(dxs, dx0, sizeof(double) * n);
    for (int t = 0; t < T; ++t) {
        const double *dx = dxs + (size_t)t * n;
        double *dxn = dxs + (size_t)(t + 1) * n;
        rk4_stages(n, dt, F, traj + (size_t)t * n, X, kb);
        l96_jac(n, X, dx, d1);                                        /* s1 = dx          */
        for (int i = 0; i < n; ++i) s[i] = dx[i] + 0.5 * dt * d1[i];  /* s2 = dx + dt/2 d1 */
        l96_jac(n, X + n, s, d2);
        for (int i = 0; i < n; ++i) s[i] = dx[i] + 0.5 * dt * d2[i];  /* s3 = dx + dt/2 d2 */
        l96_jac(n, X + 2 * n, s, d3);
        for (int i = 0; i < n; ++i) s[i] = dx[i] + dt * d3[i];        /* s4 = dx + dt d3   */
        l96_jac(n, X + 3 * n, s, d4);
        for (int i = 0; i < n; ++i)
            dxn[i] = dx[i] + dt / 6.0 * (d1[i] + 2.0 * d2[i] + 2.0 * d3[i] + d4[i]);
    }
    free(X); free(kb); free(d1); free(d2); free(d3); free(d4); free(s);
}

/* Adjoint: lam_T = forcing_T;  lam_t = M_t^T lam_{t+1} + forcing_t for
 * t = T-1..0; returns lam_0.  forcing is (T+1) x n (row t = forcing at step t).
 * Each step is the transpose of the TL step above, taken statement by
 * statement in reverse order. */
void l96_ad(int n, int T, double dt, double F, const double *traj, const double *forcing, double *lam0)
{
    double *X = malloc(sizeof(double) * 4 * n), *kb = malloc(sizeof(double) * n);
    double *lam = malloc(sizeof(double) * n), *lx = malloc(sizeof(double) * n);
    double *lk1 = malloc(sizeof(double) * n), *lk2 = malloc(sizeof(double) * n);
    double *lk3 = malloc(sizeof(double) * n), *lk4 = malloc(sizeof(double) * n);
    double *ls = malloc(sizeof(double) * n);
    memcpy(lam, forcing + (size_t)T * n, sizeof(double) * n);
    for (int t = T - 1; t >= 0; --t) {
        rk4_stages(n, dt, F, traj + (size_t)t * n, X, kb);
        /* dxn = dx + dt/6 (d1 + 2 d2 + 2 d3 + d4) */
        for (int i = 0; i < n; ++i) {
            lx[i] = lam[i];
            lk1[i] = dt / 6.0 * lam[i];
            lk2[i] = dt / 3.0 * lam[i];
            lk3[i] = dt / 3.0 * lam[i];
            lk4[i] = dt / 6.0 * lam[i];
        }
        /* d4 = J(X4) s4, s4 = dx + dt d3 */
        l96_jac_t(n, X + 3 * n, lk4, ls);
        for (int i = 0; i < n; ++i) { lx[i] += ls[i]; lk3[i] += dt * ls[i]; }
        /* d3 = J(X3) s3, s3 = dx + dt/2 d2 */
        l96_jac_t(n, X + 2 * n, lk3, ls);
        for (int i = 0; i < n; ++i) { lx[i] += ls[i]; lk2[i] += 0.5 * dt * ls[i]; }
        /* d2 = J(X2) s2, s2 = dx + dt/2 d1 */
        l96_jac_t(n, X + n, lk2, ls);
        for (int i = 0; i < n; ++i) { lx[i] += ls[i]; lk1[i] += 0.5 * dt * ls[i]; }
        /* d1 = J(X1) dx */
        l96_jac_t(n, X, lk1, ls);
        for (int i = 0; i < n; ++i) lam[i] = lx[i] + ls[i] + forcing[(size_t)t * n + i];
    }
    memcpy(lam0, lam, sizeof(double) * n);
    free(X); free(kb); free(lam); free(lx); free(lk1); free(lk2); free(lk3); free(lk4); free(ls);
}
