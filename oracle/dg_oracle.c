/*
 * dg_oracle.c -- plain FP64 CPU oracle of the nodal DG hot path of
 * arXiv:1609.00098 (Kidder et al., SpECTRE).
 *
 * TEST INFRASTRUCTURE ONLY (see dg_oracle.h).  Every routine restates the
 * paper's definitions directly, in the paper's order, with no blocking or
 * fusion.  Where the paper is silent the reading taken is stated at the
 * routine.  Compiled with -ffp-contract=off so each operation rounds once.
 */
#include "dg_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>

struct or_mesh {
    or_desc d;
    int na[3];          /* nodes per axis (n active, 1 inactive) */
    int nn;             /* nodes per element */
    long long E;        /* number of elements */
    double dx[3];       /* element widths */
    double x[OR_MAXN];  /* LGL nodes */
    double w[OR_MAXN];  /* LGL weights */
    double D[OR_MAXN * OR_MAXN];
    double Vinv[OR_MAXN * OR_MAXN];
    double t;           /* mesh time: enters only through analytic exterior states */
};

/* ------------------------------------------------------------------------ */
/* Legendre polynomials and LGL tables (Sec. 3.1, Lagrange basis on GLL nodes) */

/* P_N(x) and P_N'(x) by the three-term recurrence
 * (k+1) P_{k+1} = (2k+1) x P_k - k P_{k-1};  P'_{k+1} = P'_{k-1} + (2k+1) P_k */
static void legendre(int N, double x, double *P, double *dP)
{
    if (N == 0) { *P = 1.0; *dP = 0.0; return; }
    double pm = 1.0, p = x, dpm = 0.0, dp = 1.0;
    for (int k = 1; k < N; ++k) {
        double pn = ((2.0 * k + 1.0) * x * p - k * pm) / (k + 1.0);
        double dpn = dpm + (2.0 * k + 1.0) * p;
        pm = p; p = pn; dpm = dp; dp = dpn;
    }
    *P = p; *dP = dp;
}

int or_lgl(int n, double *x, double *w)
{
    if (n < 2 || n > OR_MAXN) return 1;
    const int N = n - 1;
    x[0] = -1.0; x[N] = 1.0;
    /* interior nodes: roots of P_N'.  Newton with the second derivative from
     * Legendre's equation (1-x^2) P'' = 2x P' - N(N+1) P, starting from the
     * Chebyshev-Lobatto points -cos(pi j / N). */
    for (int j = 1; j <= (N - 1) / 2 + ((N - 1) % 2); ++j) {
        double t = -cos(M_PI * j / N);
        for (int it = 0; it < 100; ++it) {
            double P, dP;
            legendre(N, t, &P, &dP);
            double d2P = (2.0 * t * dP - N * (N + 1.0) * P) / (1.0 - t * t);
            double dt = -dP / d2P;
            t += dt;
            if (fabs(dt) < 1e-16) break;
        }
        x[j] = t;
        x[N - j] = -t;
    }
    if (N % 2 == 0) x[N / 2] = 0.0;
    for (int j = 0; j <= N; ++j) {
        double P, dP;
        legendre(N, x[j], &P, &dP);
        w[j] = 2.0 / (N * (N + 1.0) * P * P);
    }
    return 0;
}

/* D_il = ell_l'(x_i) (eq:405) from barycentric weights lambda_j = 1/prod_{k!=j}(x_j-x_k):
 * D_il = (lambda_l/lambda_i)/(x_i-x_l) for i != l, and D_ii = -sum_{l!=i} D_il so
 * that D annihilates constants. */
int or_diffmat(int n, const double *x, double *D)
{
    if (n < 2 || n > OR_MAXN) return 1;
    double lam[OR_MAXN];
    for (int j = 0; j < n; ++j) {
        double p = 1.0;
        for (int k = 0; k < n; ++k)
            if (k != j) p *= (x[j] - x[k]);
        lam[j] = 1.0 / p;
    }
    for (int i = 0; i < n; ++i) {
        double s = 0.0;
        for (int l = 0; l < n; ++l) {
            if (l == i) continue;
            D[i * n + l] = (lam[l] / lam[i]) / (x[i] - x[l]);
            s += D[i * n + l];
        }
        D[i * n + i] = -s;
    }
    return 0;
}

/* Inverse of V[i][m] = P_m(x_i) by Gauss-Jordan elimination with partial pivoting. */
int or_legendre_vinv(int n, const double *x, double *Vinv)
{
    if (n < 1 || n > OR_MAXN) return 1;
    double A[OR_MAXN][2 * OR_MAXN];
    for (int i = 0; i < n; ++i) {
        for (int m = 0; m < n; ++m) {
            double P, dP;
            legendre(m, x[i], &P, &dP);
            A[i][m] = P;
            A[i][n + m] = (i == m) ? 1.0 : 0.0;
        }
    }
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (fabs(A[r][c]) > fabs(A[piv][c])) piv = r;
        if (A[piv][c] == 0.0) return 2;
        if (piv != c)
            for (int k = 0; k < 2 * n; ++k) { double t = A[c][k]; A[c][k] = A[piv][k]; A[piv][k] = t; }
        double inv = 1.0 / A[c][c];
        for (int k = 0; k < 2 * n; ++k) A[c][k] *= inv;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            double f = A[r][c];
            if (f == 0.0) continue;
            for (int k = 0; k < 2 * n; ++k) A[r][k] -= f * A[c][k];
        }
    }
    /* A now holds [I | V^{-1}] with V^{-1}[m][i] mapping nodal values to modes */
    for (int m = 0; m < n; ++m)
        for (int i = 0; i < n; ++i) Vinv[m * n + i] = A[m][n + i];
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Mesh: uniform periodic box of affine elements (eq:AffineMap). */

or_mesh *or_mesh_create(const or_desc *d)
{
    if (d->dim < 1 || d->dim > 3 || d->n < 2 || d->n > OR_MAXN) return NULL;
    if (d->flux < 0 || d->flux > 2 || (d->flux == 2 && d->system != 0)) return NULL;  /* Roe: Newtonian only */
    if (d->limiter < 0 || d->limiter > 3 || (d->limiter == 3 && (d->system != 0 || !(d->mrs_alpha >= 0.0))))
        return NULL;  /* MRS: Newtonian only, alpha~ >= 0 */
    int analytic = 0;
    for (int a = 0; a < d->dim; ++a) {
        if (d->bc[a] != 0 && d->bc[a] != 1) return NULL;
        analytic |= d->bc[a];
    }
    if (d->exact < 0 || d->exact > 1) return NULL;
    /* analytic exterior states: the isentropic vortex (Newtonian), no limiter */
    if (analytic && (d->exact != 1 || d->system != 0 || d->limiter != 0)) return NULL;
    or_mesh *m = (or_mesh *)calloc(1, sizeof(or_mesh));
    m->d = *d;
    m->nn = 1;
    m->E = 1;
    for (int a = 0; a < 3; ++a) {
        if (a >= d->dim) m->d.K[a] = 1;
        if (m->d.K[a] < 1) { free(m); return NULL; }
        m->na[a] = (a < d->dim) ? d->n : 1;
        m->nn *= m->na[a];
        m->E *= m->d.K[a];
        m->dx[a] = (d->hi[a] - d->lo[a]) / m->d.K[a];
    }
    or_lgl(d->n, m->x, m->w);
    or_diffmat(d->n, m->x, m->D);
    or_legendre_vinv(d->n, m->x, m->Vinv);
    return m;
}

void or_mesh_destroy(or_mesh *m) { free(m); }
void or_set_time(or_mesh *m, double t) { m->t = t; }
double or_get_time(const or_mesh *m) { return m->t; }
long long or_num_elements(const or_mesh *m) { return m->E; }
int or_nodes_per_element(const or_mesh *m) { return m->nn; }

static void elem_coords(const or_mesh *m, long long e, int *ec)
{
    ec[0] = (int)(e % m->d.K[0]);
    ec[1] = (int)((e / m->d.K[0]) % m->d.K[1]);
    ec[2] = (int)(e / ((long long)m->d.K[0] * m->d.K[1]));
}

static long long elem_index(const or_mesh *m, const int *ec)
{
    return ec[0] + (long long)m->d.K[0] * (ec[1] + (long long)m->d.K[1] * ec[2]);
}

/* periodic neighbour of element e along axis a, direction s = +1 or -1 */
static long long neighbour(const or_mesh *m, long long e, int a, int s)
{
    int ec[3];
    elem_coords(m, e, ec);
    ec[a] = (ec[a] + s + m->d.K[a]) % m->d.K[a];
    return elem_index(m, ec);
}

/* reference coordinate of node index i along axis a (0 on inactive axes) */
static double xbar(const or_mesh *m, int a, int i)
{
    return (a < m->d.dim) ? m->x[i] : 0.0;
}

/* quadrature weight of node index i along axis a (1 on inactive axes) */
static double wgt(const or_mesh *m, int a, int i)
{
    return (a < m->d.dim) ? m->w[i] : 1.0;
}

void or_node_coords(const or_mesh *m, double *xyz)
{
    const long long N = m->E * m->nn;
    for (long long e = 0; e < m->E; ++e) {
        int ec[3];
        elem_coords(m, e, ec);
        for (int k = 0; k < m->na[2]; ++k)
            for (int j = 0; j < m->na[1]; ++j)
                for (int i = 0; i < m->na[0]; ++i) {
                    int idx[3] = {i, j, k};
                    long long q = e * m->nn + i + m->na[0] * (j + m->na[1] * k);
                    for (int a = 0; a < 3; ++a) {
                        /* eq:AffineMap: x = a^k + (1 + xbar)(b^k - a^k)/2 */
                        double ak = m->d.lo[a] + ec[a] * m->dx[a];
                        double bk = ak + m->dx[a];
                        xyz[a * N + q] = ak + 0.5 * (1.0 + xbar(m, a, idx[a])) * (bk - ak);
                    }
                }
    }
}

/* ------------------------------------------------------------------------ */
/* Physics: primitive <-> conserved (Sec. 2.1.1, 2.1.2) */

static void prim2con_node(int system, double g, const double *pr, double *u)
{
    const double rho = pr[0], vx = pr[1], vy = pr[2], vz = pr[3], p = pr[4];
    const double v2 = vx * vx + vy * vy + vz * vz;
    if (system == 0) {
        /* U = [rho, rho v_i, E], E = rho eps + rho v^2/2, p = (g-1) rho eps */
        u[0] = rho;
        u[1] = rho * vx; u[2] = rho * vy; u[3] = rho * vz;
        u[4] = p / (g - 1.0) + 0.5 * rho * v2;
    } else {
        /* D = rho W, S_i = rho h W^2 v_i, tau = rho h W^2 - p - rho W, written as
         * tau = rho W (W-1) + rho eps W^2 + p (W^2-1) with W-1 = W^2 v^2/(W+1)
         * and W^2-1 = W^2 v^2, which loses no digits when eps << 1 and W ~ 1. */
        const double W = 1.0 / sqrt(1.0 - v2);
        const double W2v2 = W * W * v2;
        const double rhoeps = p / (g - 1.0);
        const double rhoh = rho + rhoeps + p;
        u[0] = rho * W;
        u[1] = rhoh * W * W * vx; u[2] = rhoh * W * W * vy; u[3] = rhoh * W * W * vz;
        u[4] = rho * W * (W2v2 / (W + 1.0)) + rhoeps * W * W + p * W2v2;
    }
}

void or_prim2con(int system, double gamma, long long count, const double *prim, double *cons)
{
    for (long long q = 0; q < count; ++q) {
        double pr[5], u[5];
        for (int v = 0; v < 5; ++v) pr[v] = prim[v * count + q];
        prim2con_node(system, gamma, pr, u);
        for (int v = 0; v < 5; ++v) cons[v * count + q] = u[v];
    }
}

/* SR con2prim (Sec. 2.1.2; the paper defers the method to a cited appendix).
 * Reading: with E = tau + D and s = |S|, solve f(p) = p - (g-1) rho eps(p) = 0
 * where v(p) = s/(E+p), W = 1/sqrt(1-v^2), rho = D/W and, from the definitions
 * of D, S, tau,
 *     rho eps = tau + D (1 - 1/W) - (E + p) v^2
 *             = tau - v^2 [ (E + p) - D W/(W+1) ]          (no cancellation at small v)
 * f is increasing with f'(p) = 1 - (g-1) v^2 (1 - D W/(E+p)).  The root lies in
 * [max(0, s-E), (g-1) tau] because tau >= rho eps for W >= 1.  Safeguarded
 * Newton: a step leaving the bracket is replaced by bisection, except a step
 * landing exactly on an end that is still its a-priori bound (at v = 0 the root
 * is the upper bound (g-1) tau itself); the bracket is
 * updated from the sign of f.  Stop once |dp| <= 2^-48 p, then take one more
 * Newton step so the result does not depend on the starting guess.
 * Returns 0 ok, 1 unphysical input, 2 no convergence. */
typedef struct { double f, df, v2, W; } c2p_eval;

static c2p_eval c2p_f(double g, double D, double s2, double tau, double p)
{
    c2p_eval r;
    const double Ep = tau + D + p;
    const double v2 = s2 / (Ep * Ep);
    const double W = 1.0 / sqrt(1.0 - v2);
    const double rhoeps = tau - v2 * (Ep - D * W / (W + 1.0));
    r.f = p - (g - 1.0) * rhoeps;
    r.df = 1.0 - (g - 1.0) * v2 * (1.0 - D * W / Ep);
    r.v2 = v2;
    r.W = W;
    return r;
}

static int c2p_node(double g, const double *u, double guess, double *pr, int *iters)
{
    const double D = u[0], Sx = u[1], Sy = u[2], Sz = u[3], tau = u[4];
    const double s2 = Sx * Sx + Sy * Sy + Sz * Sz;
    *iters = 0;
    if (!(D > 0.0) || !(tau > 0.0) || !(s2 < tau * (tau + 2.0 * D))) {
        for (int v = 0; v < 5; ++v) pr[v] = NAN;
        return 1;
    }
    const double E = tau + D;
    double plo = sqrt(s2) - E;
    if (plo < 0.0) plo = 0.0;
    double phi = (g - 1.0) * tau;
    double p = (guess >= 0.0) ? guess : phi;
    if (p < plo) p = plo;
    if (p > phi) p = phi;
    int status = 2;
    int lo_moved = 0, hi_moved = 0; /* an end still at its a-priori bound may be landed on */
    int it = 0;
    for (; it < 200; ++it) {
        c2p_eval r = c2p_f(g, D, s2, tau, p);
        if (r.f == 0.0) { status = 0; break; }
        if (r.f > 0.0) { phi = p; hi_moved = 1; } else { plo = p; lo_moved = 1; }
        double pn = p - r.f / r.df;
        if (!((pn > plo && pn < phi) || (pn == phi && !hi_moved) || (pn == plo && !lo_moved)))
            pn = 0.5 * (plo + phi);
        const double dp = fabs(pn - p);
        p = pn;
        if (dp <= 0x1p-48 * p) {
            /* one more Newton step from the converged iterate */
            c2p_eval r2 = c2p_f(g, D, s2, tau, p);
            p = p - r2.f / r2.df;
            it += 1;
            status = 0;
            break;
        }
        if (phi - plo <= 0.0) { status = 0; break; }
    }
    *iters = it + 1;
    const double Ep = E + p;
    pr[0] = D * sqrt(1.0 - s2 / (Ep * Ep));
    pr[1] = Sx / Ep;
    pr[2] = Sy / Ep;
    pr[3] = Sz / Ep;
    pr[4] = p;
    return status;
}

long long or_con2prim(long long count, double gamma, const double *cons, double *prim,
                      const double *guess, int *iters, int *status)
{
    long long fails = 0;
#pragma omp parallel for reduction(+ : fails) schedule(static)
    for (long long q = 0; q < count; ++q) {
        double u[5], pr[5];
        for (int v = 0; v < 5; ++v) u[v] = cons[v * count + q];
        int it;
        int st = c2p_node(gamma, u, guess ? guess[q] : -1.0, pr, &it);
        for (int v = 0; v < 5; ++v) prim[v * count + q] = pr[v];
        if (iters) iters[q] = it;
        if (status) status[q] = st;
        if (st) ++fails;
    }
    return fails;
}

/* Node primitives used by fluxes: (vx, vy, vz, p). */
static int node_prim(int system, double g, const double *u, double *P)
{
    if (system == 0) {
        /* Sec. 2.1.1: v = S/rho, p = (g-1)(E - rho v^2/2) */
        const double inv = 1.0 / u[0];
        P[0] = u[1] * inv;
        P[1] = u[2] * inv;
        P[2] = u[3] * inv;
        P[3] = (g - 1.0) * (u[4] - 0.5 * (u[1] * P[0] + u[2] * P[1] + u[3] * P[2]));
        return 0;
    }
    double pr[5];
    int it;
    int st = c2p_node(g, u, -1.0, pr, &it);
    P[0] = pr[1]; P[1] = pr[2]; P[2] = pr[3]; P[3] = pr[4];
    return st;
}

long long or_primitives(const or_mesh *m, const double *U, double *P)
{
    const int nn = m->nn;
    long long fails = 0;
#pragma omp parallel for reduction(+ : fails) schedule(static)
    for (long long e = 0; e < m->E; ++e) {
        for (int q = 0; q < nn; ++q) {
            double u[5], pp[4];
            for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + q];
            if (node_prim(m->d.system, m->d.gamma, u, pp)) ++fails;
            for (int c = 0; c < 4; ++c) P[(e * 4 + c) * nn + q] = pp[c];
        }
    }
    return fails;
}

/* Flux along axis a (Sec. 2.1.1 and 2.1.2 with alpha = 1, beta = 0):
 * F = [U0 v_a, S_i v_a + p delta_ia, (U4 + p) v_a]; U0 = rho (NE) or D (SR),
 * U4 = E (NE) or tau (SR).  Both systems share this form. */
static void flux_axis(const double *u, const double *P, int a, double *F)
{
    const double va = P[a], p = P[3];
    F[0] = u[0] * va;
    F[1] = u[1] * va;
    F[2] = u[2] * va;
    F[3] = u[3] * va;
    F[1 + a] = F[1 + a] + p;
    F[4] = (u[4] + p) * va;
}

/* Smallest and largest characteristic speeds along axis a (eq:CharDecomp).
 * NE: v_a -+ c with c^2 = g p / rho.  SR: the standard flat-space eigenvalues
 * lambda_-+ = [v_a (1-cs^2) -+ cs sqrt((1-v^2)(1 - v^2 cs^2 - v_a^2 (1-cs^2)))] / (1 - v^2 cs^2)
 * with cs^2 = g p/(rho h) and rho h = (tau + D + p)(1 - v^2). */
static void speeds_axis(int system, double g, const double *u, const double *P, int a,
                        double *lmin, double *lmax)
{
    const double va = P[a], p = P[3];
    if (system == 0) {
        const double c = sqrt(g * p / u[0]);
        *lmin = va - c;
        *lmax = va + c;
        return;
    }
    const double v2 = P[0] * P[0] + P[1] * P[1] + P[2] * P[2];
    const double rhoh = (u[4] + u[0] + p) * (1.0 - v2);
    const double cs2 = g * p / rhoh;
    const double cs = sqrt(cs2);
    double disc = (1.0 - v2) * (1.0 - v2 * cs2 - va * va * (1.0 - cs2));
    if (disc < 0.0) disc = 0.0;
    const double root = cs * sqrt(disc);
    const double den = 1.0 - v2 * cs2;
    *lmin = (va * (1.0 - cs2) - root) / den;
    *lmax = (va * (1.0 - cs2) + root) / den;
}

/* Numerical flux along +e_a between lower state L and upper state R (Sec. 3.2):
 * LLF (eq:LLF) or HLL with Davis speeds (eq:HLL). */
/* Roe flux for the Newtonian ideal gas (Sec. 3.2.3, eq:Roe): half the sum of the
 * physical fluxes minus half of sum_i alpha_i |lambda_i| e_i, with the flux
 * Jacobian along e_a evaluated at the Roe averages (eq:RoeAverages) of the
 * velocity and of the specific enthalpy h = (E + p)/rho.  Its eigenvalues are
 * u_n - c, u_n (three times), u_n + c with c^2 = (g-1)(h - |v|^2/2); the wave
 * strengths alpha_i are the jump U_R - U_L on the left eigenvectors, written in
 * the frame (normal, t1, t2) = (a, a+1, a+2). */
static void roe_flux(double g, int a, const double *uL, const double *PL, const double *uR, const double *PR,
                     const double *FL, const double *FR, double *Fs)
{
    const double sl = sqrt(uL[0]), sr = sqrt(uR[0]);
    const double wsum = sl + sr;
    double vh[3];
    for (int i = 0; i < 3; ++i) vh[i] = (sl * PL[i] + sr * PR[i]) / wsum;
    const double hL = (uL[4] + PL[3]) / uL[0], hR = (uR[4] + PR[3]) / uR[0];
    const double hh = (sl * hL + sr * hR) / wsum;
    const double q2 = vh[0] * vh[0] + vh[1] * vh[1] + vh[2] * vh[2];
    const double c2 = (g - 1.0) * (hh - 0.5 * q2);
    const double c = sqrt(c2);
    const int b = (a + 1) % 3, d = (a + 2) % 3;
    const double un = vh[a], ut1 = vh[b], ut2 = vh[d];
    const double j1 = uR[0] - uL[0], jn = uR[1 + a] - uL[1 + a];
    const double jt1 = uR[1 + b] - uL[1 + b], jt2 = uR[1 + d] - uL[1 + d], j5 = uR[4] - uL[4];
    const double al3 = jt1 - ut1 * j1;
    const double al4 = jt2 - ut2 * j1;
    const double j5b = j5 - al3 * ut1 - al4 * ut2;
    const double al2 = (g - 1.0) / c2 * (j1 * (hh - un * un) + un * jn - j5b);
    const double al1 = (j1 * (un + c) - jn - c * al2) / (2.0 * c);
    const double al5 = j1 - (al1 + al2);
    const double w1 = fabs(un - c) * al1, w2 = fabs(un) * al2, w5 = fabs(un + c) * al5;
    const double w3 = fabs(un) * al3, w4 = fabs(un) * al4;
    double D[5];
    D[0] = w1 + w2 + w5;
    D[1 + a] = w1 * (un - c) + w2 * un + w5 * (un + c);
    D[1 + b] = (w1 + w2 + w5) * ut1 + w3;
    D[1 + d] = (w1 + w2 + w5) * ut2 + w4;
    D[4] = w1 * (hh - un * c) + w2 * (0.5 * q2) + w3 * ut1 + w4 * ut2 + w5 * (hh + un * c);
    for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * D[v];
}

static void num_flux(const or_mesh *m, int a, const double *uL, const double *PL,
                     const double *uR, const double *PR, double *Fs, double *FL, double *FR)
{
    const int sys = m->d.system;
    const double g = m->d.gamma;
    double lminL, lmaxL, lminR, lmaxR;
    flux_axis(uL, PL, a, FL);
    flux_axis(uR, PR, a, FR);
    speeds_axis(sys, g, uL, PL, a, &lminL, &lmaxL);
    speeds_axis(sys, g, uR, PR, a, &lminR, &lmaxR);
    if (m->d.flux == 2) {
        roe_flux(g, a, uL, PL, uR, PR, FL, FR, Fs);
    } else if (m->d.flux == 0) {
        /* alpha = largest |lambda| on either side */
        double al = fmax(fmax(fabs(lminL), fabs(lmaxL)), fmax(fabs(lminR), fabs(lmaxR)));
        for (int v = 0; v < 5; ++v)
            Fs[v] = 0.5 * (FL[v] + FR[v]) - 0.5 * al * (uR[v] - uL[v]);
    } else {
        double cmin = fmin(fmin(lminL, lminR), 0.0);
        double cmax = fmax(fmax(lmaxL, lmaxR), 0.0);
        double den = cmax - cmin;
        if (den > 0.0) {
            for (int v = 0; v < 5; ++v)
                Fs[v] = (cmax * FL[v] - cmin * FR[v]) / den + (cmin * cmax / den) * (uR[v] - uL[v]);
        } else {
            for (int v = 0; v < 5; ++v) Fs[v] = 0.5 * (FL[v] + FR[v]);
        }
    }
}


/* Point-wise numerical flux along +e_axis for tests: fills Fs (numerical flux),
 * FL, FR (physical fluxes) and speeds[4] = (lmin_L, lmax_L, lmin_R, lmax_R). */
int or_num_flux(int system, double gamma, int flux, int axis, const double *uL, const double *uR,
                double *Fs, double *FL, double *FR, double *speeds)
{
    or_mesh m;
    memset(&m, 0, sizeof(m));
    m.d.system = system;
    m.d.gamma = gamma;
    m.d.flux = flux;
    double PL[4], PR[4];
    int st = node_prim(system, gamma, uL, PL) | node_prim(system, gamma, uR, PR);
    num_flux(&m, axis, uL, PL, uR, PR, Fs, FL, FR);
    speeds_axis(system, gamma, uL, PL, axis, &speeds[0], &speeds[1]);
    speeds_axis(system, gamma, uR, PR, axis, &speeds[2], &speeds[3]);
    return st;
}

/* ------------------------------------------------------------------------ */
/* Semi-discrete RHS, eq:411 with the affine map.  Reading of the signs: with
 * F = (F* - F).n_out and outward unit normals the strong form (eq:5) gives
 *   dU_ijk/dt = - sum_a (2/dx_a) sum_l D_{i_a l} F^a_l
 *               - sum_{faces containing the node} (2/dx_a)(1/w_end) (F* - F).n_out,
 * which is eq:411 once F at the lower faces is taken along +e_a.  The factor
 * sqrt(2gamma)/J of eq:411 is (dx_b dx_c/4)/(dx_a dx_b dx_c/8) = 2/dx_a.
 * Each face is evaluated once, in the +e_a orientation, and the same F* is used
 * by both elements, so the scheme conserves to roundoff. */

static long long node_id(const or_mesh *m, int i, int j, int k)
{
    return i + (long long)m->na[0] * (j + (long long)m->na[1] * k);
}

/* eq:isen_vortex at point x and time t; par = (beta, X0, Y0, U, V, W), P = rho^gamma */
static void isentropic_vortex(const double *par, double g, const double *x, double t, double *pr)
{
    const double pi = 3.14159265358979323846;
    const double beta = par[0];
    const double xt = x[0] - par[1] - par[3] * t;
    const double yt = x[1] - par[2] - par[4] * t;
    const double r2 = xt * xt + yt * yt;
    const double rho = pow(1.0 - (g - 1.0) * beta * beta / (8.0 * g * pi * pi) * exp(1.0 - r2), 1.0 / (g - 1.0));
    const double f = beta / (2.0 * pi) * exp(0.5 * (1.0 - r2));
    pr[0] = rho;
    pr[1] = par[3] - yt * f;
    pr[2] = par[4] + xt * f;
    pr[3] = par[5];
    pr[4] = pow(rho, g);
}

/* Exterior state of a boundary face node (Sec. 3.4: the interior numerical flux
 * with the exterior solution supplied): the analytic solution at time t at the
 * coordinates of the interior trace node (element e, node indices id),
 * conserved, and its primitives as node_prim recovers them. */
static void exterior_state(const or_mesh *m, long long e, const int *id, double t, double *u, double *P)
{
    int ec[3];
    elem_coords(m, e, ec);
    double x[3], pr[5];
    for (int a = 0; a < 3; ++a) {
        const double ak = m->d.lo[a] + ec[a] * m->dx[a];
        const double bk = ak + m->dx[a];
        x[a] = ak + 0.5 * (1.0 + xbar(m, a, id[a])) * (bk - ak);
    }
    isentropic_vortex(m->d.exact_par, m->d.gamma, x, t, pr);
    prim2con_node(0, m->d.gamma, pr, u);
    node_prim(0, m->d.gamma, u, P);
}

static long long rhs_at(const or_mesh *m, const double *U, double *R, double t)
{
    const int nn = m->nn, n = m->d.n, dim = m->d.dim;
    const long long E = m->E;
    double *P = (double *)malloc(sizeof(double) * 4 * nn * E);
    long long fails = or_primitives(m, U, P);

    /* volume term */
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < E; ++e) {
        double *F = (double *)malloc(sizeof(double) * 3 * 5 * nn);
        const double *Ue = U + e * 5 * nn;
        const double *Pe = P + e * 4 * nn;
        for (int q = 0; q < nn; ++q) {
            double u[5], pp[4], f[5];
            for (int v = 0; v < 5; ++v) u[v] = Ue[v * nn + q];
            for (int c = 0; c < 4; ++c) pp[c] = Pe[c * nn + q];
            for (int a = 0; a < dim; ++a) {
                flux_axis(u, pp, a, f);
                for (int v = 0; v < 5; ++v) F[(a * 5 + v) * nn + q] = f[v];
            }
        }
        for (int k = 0; k < m->na[2]; ++k)
            for (int j = 0; j < m->na[1]; ++j)
                for (int i = 0; i < m->na[0]; ++i) {
                    const int idx[3] = {i, j, k};
                    const long long q = node_id(m, i, j, k);
                    for (int v = 0; v < 5; ++v) {
                        double acc = 0.0;
                        for (int a = 0; a < dim; ++a) {
                            double s = 0.0;
                            for (int l = 0; l < n; ++l) {
                                int id2[3] = {i, j, k};
                                id2[a] = l;
                                s = s + m->D[idx[a] * n + l] * F[(a * 5 + v) * nn + node_id(m, id2[0], id2[1], id2[2])];
                            }
                            acc = acc + (2.0 / m->dx[a]) * s;
                        }
                        R[(e * 5 + v) * nn + q] = -acc;
                    }
                }
        free(F);
    }

    /* surface terms, one axis after another; on an analytic axis the faces at
     * lo and hi take the exterior state instead of the periodic neighbour */
    for (int a = 0; a < dim; ++a) {
        const double g = 2.0 / m->dx[a];
        const double liftN = g / m->w[n - 1];
        const double lift0 = g / m->w[0];
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const int analytic = m->d.bc[a] == 1;
#pragma omp parallel for schedule(static)
        for (long long e = 0; e < E; ++e) {
            const long long ep = neighbour(m, e, a, +1);
            int ec[3];
            elem_coords(m, e, ec);
            const int hi_bnd = analytic && ec[a] == m->d.K[a] - 1;
            const int lo_bnd = analytic && ec[a] == 0;
            for (int t1 = 0; t1 < m->na[c]; ++t1)
                for (int t0 = 0; t0 < m->na[b]; ++t0) {
                    int iL[3], iR[3];
                    iL[a] = n - 1; iR[a] = 0;
                    iL[b] = iR[b] = t0;
                    iL[c] = iR[c] = t1;
                    const long long qL = node_id(m, iL[0], iL[1], iL[2]);
                    const long long qR = node_id(m, iR[0], iR[1], iR[2]);
                    double uL[5], uR[5], PL[4], PR[4], Fs[5], FL[5], FR[5];
                    for (int v = 0; v < 5; ++v) uL[v] = U[(e * 5 + v) * nn + qL];
                    for (int cc = 0; cc < 4; ++cc) PL[cc] = P[(e * 4 + cc) * nn + qL];
                    if (hi_bnd) {
                        exterior_state(m, e, iL, t, uR, PR);
                    } else {
                        for (int v = 0; v < 5; ++v) uR[v] = U[(ep * 5 + v) * nn + qR];
                        for (int cc = 0; cc < 4; ++cc) PR[cc] = P[(ep * 4 + cc) * nn + qR];
                    }
                    num_flux(m, a, uL, PL, uR, PR, Fs, FL, FR);
                    for (int v = 0; v < 5; ++v) {
                        /* lower element: n_out = +e_a */
                        R[(e * 5 + v) * nn + qL] = R[(e * 5 + v) * nn + qL] - liftN * (Fs[v] - FL[v]);
                        /* upper element: n_out = -e_a, so (F*-F).n_out = -(F*_a - F_a) */
                        if (!hi_bnd)
                            R[(ep * 5 + v) * nn + qR] = R[(ep * 5 + v) * nn + qR] + lift0 * (Fs[v] - FR[v]);
                    }
                    if (lo_bnd) {
                        /* the element's lower face: exterior on the left, this element on the right */
                        for (int v = 0; v < 5; ++v) uR[v] = U[(e * 5 + v) * nn + qR];
                        for (int cc = 0; cc < 4; ++cc) PR[cc] = P[(e * 4 + cc) * nn + qR];
                        exterior_state(m, e, iR, t, uL, PL);
                        num_flux(m, a, uL, PL, uR, PR, Fs, FL, FR);
                        for (int v = 0; v < 5; ++v)
                            R[(e * 5 + v) * nn + qR] = R[(e * 5 + v) * nn + qR] + lift0 * (Fs[v] - FR[v]);
                    }
                }
        }
    }
    free(P);
    return fails;
}

long long or_rhs(const or_mesh *m, const double *U, double *R) { return rhs_at(m, U, R, m->t); }

double or_lambda_max(const or_mesh *m, const double *U)
{
    const int nn = m->nn;
    double lam = 0.0;
#pragma omp parallel for reduction(max : lam) schedule(static)
    for (long long e = 0; e < m->E; ++e) {
        for (int q = 0; q < nn; ++q) {
            double u[5], pp[4];
            for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + q];
            node_prim(m->d.system, m->d.gamma, u, pp);
            for (int a = 0; a < m->d.dim; ++a) {
                double lo, hi;
                speeds_axis(m->d.system, m->d.gamma, u, pp, a, &lo, &hi);
                double s = fmax(fabs(lo), fabs(hi));
                if (s > lam) lam = s;
            }
        }
    }
    return lam;
}

/* Sec. 3.4: dt = C dx_min / lambda_max; reading: dx_min is the smallest gap between
 * neighbouring LGL nodes on the physical grid, min_a (dx_a/2)(xbar_1 - xbar_0). */
double or_cfl_dt(const or_mesh *m, const double *U, double cfl)
{
    double dxmin = INFINITY;
    for (int a = 0; a < m->d.dim; ++a) {
        double h = 0.5 * m->dx[a] * (m->x[1] - m->x[0]);
        if (h < dxmin) dxmin = h;
    }
    return cfl * dxmin / or_lambda_max(m, U);
}

/* ------------------------------------------------------------------------ */
/* Limiter (Sec. 3.3.1, 3.3.2) */

static double minmod3(double a1, double a2, double a3)
{
    if (a1 > 0.0 && a2 > 0.0 && a3 > 0.0) return fmin(a1, fmin(a2, a3));
    if (a1 < 0.0 && a2 < 0.0 && a3 < 0.0) return fmax(a1, fmax(a2, a3));
    return 0.0;
}

/* eq:MinModB */
static double minmodB(double a1, double a2, double a3, double M, double h)
{
    if (fabs(a1) <= M * h * h) return a1;
    return minmod3(a1, a2, a3);
}

/* Summaries of one element and variable: U0 = LGL cell average; face means
 * (LGL-weighted over the face nodes); c1[a] = Legendre P_1 coefficient along
 * axis a of the average over the other axes, from the inverse Vandermonde
 * (exact for every degree, including N = 1). */
static void summaries(const or_mesh *m, const double *Uv, double *S)
{
    const int dim = m->d.dim, n = m->d.n;
    double norm = 1.0;
    for (int a = 0; a < dim; ++a) norm *= 2.0;
    double U0 = 0.0;
    for (int k = 0; k < m->na[2]; ++k)
        for (int j = 0; j < m->na[1]; ++j)
            for (int i = 0; i < m->na[0]; ++i)
                U0 = U0 + wgt(m, 0, i) * wgt(m, 1, j) * wgt(m, 2, k) * Uv[node_id(m, i, j, k)];
    S[0] = U0 / norm;
    for (int a = 0; a < 3; ++a) {
        S[1 + 2 * a] = S[0];
        S[2 + 2 * a] = S[0];
        S[7 + a] = 0.0;
    }
    for (int a = 0; a < dim; ++a) {
        const int b = (a + 1) % 3, c = (a + 2) % 3;
        const double fnorm = norm / 2.0;
        double ubar[OR_MAXN];
        for (int ia = 0; ia < n; ++ia) {
            double s = 0.0;
            for (int t1 = 0; t1 < m->na[c]; ++t1)
                for (int t0 = 0; t0 < m->na[b]; ++t0) {
                    int id[3];
                    id[a] = ia; id[b] = t0; id[c] = t1;
                    s = s + wgt(m, b, t0) * wgt(m, c, t1) * Uv[node_id(m, id[0], id[1], id[2])];
                }
            ubar[ia] = s / fnorm;
        }
        S[1 + 2 * a] = ubar[0];
        S[2 + 2 * a] = ubar[n - 1];
        double c1 = 0.0;
        for (int i = 0; i < n; ++i) c1 = c1 + m->Vinv[1 * n + i] * ubar[i];
        S[7 + a] = c1;
    }
}

void or_limiter_summaries(const or_mesh *m, const double *U, double *S)
{
    const int nn = m->nn;
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < m->E; ++e)
        for (int v = 0; v < 5; ++v) summaries(m, U + (e * 5 + v) * nn, S + (e * 5 + v) * 10);
}

static int unphysical_node(const double *u)
{
    const double D = u[0], tau = u[4];
    const double s2 = u[1] * u[1] + u[2] * u[2] + u[3] * u[3];
    return !(D > 0.0) || !(tau > 0.0) || !(s2 < tau * (tau + 2.0 * D));
}

/* Reading of the limiter:
 *  - summaries and neighbour means come from the pre-limit state of the stage;
 *  - each conserved variable is tested and limited on its own;
 *  - MinModN: the six face tests of Sec. 3.3.2 with tolerance 1e-8 and M = 0 in
 *    the detector; a variable failing any test is replaced by
 *    U0 + sum_a m_B(U_a, (U0+ - U0)/(dx/beta), (U0 - U0-)/(dx/beta); M)(x_a - x_a0)
 *    (eq:MinModSol, eq:MinModB), U_a = 2 c1_a / dx_a;
 *  - MinMod: every variable of every element is replaced that way;
 *  - SR: an element with an unphysical node is limited in every variable. */
/* Moment limiter of Moe, Rossmanith and Seal (Sec. 3.3.3, eq:MRSSol), Newtonian
 * system, in the reading used here:
 *   U -> U0 + Theta (U - U0) on the conserved variables, one Theta in [0, 1] per
 *   element, found from the primitives w = (rho, vx, vy, vz, p):
 *   w0      primitives of the LGL cell average U0 of the element;
 *   we_max, we_min  max and min of w over the element's nodes;
 *   M, m    max and min of the face neighbours' w0 (along the active axes),
 *           widened to w0 + alpha~ h^{3/2} and w0 - alpha~ h^{3/2}, h the largest
 *           element width;
 *   Theta = min over the components of min(1, |(M - w0)/(we_max - w0)|,
 *           |(m - w0)/(we_min - w0)|), a ratio counting 1 when its denominator is
 *           at the rounding level of w0 (|d| <= 1e-12 |w0|: a component that is
 *           constant over the element up to rounding says nothing).
 * The element's cell average is kept exactly. */
static long long limit_mrs(const or_mesh *m, double *U, unsigned char *troubled)
{
    const int nn = m->nn, dim = m->d.dim;
    const long long E = m->E;
    const double g = m->d.gamma;
    double h = 0.0;
    for (int a = 0; a < dim; ++a) h = fmax(h, m->dx[a]);
    const double wid = m->d.mrs_alpha * h * sqrt(h);
    /* per element: U0[5], w0[5], we_max[5], we_min[5] */
    double *T = (double *)malloc(sizeof(double) * 20 * E);
    double *S = (double *)malloc(sizeof(double) * 10 * 5 * E);
    or_limiter_summaries(m, U, S);
#pragma omp parallel for schedule(static)
    for (long long e = 0; e < E; ++e) {
        double *Te = T + 20 * e;
        for (int v = 0; v < 5; ++v) Te[v] = S[(e * 5 + v) * 10];
        double P0[4];
        node_prim(0, g, Te, P0);
        Te[5] = Te[0];
        for (int c = 0; c < 4; ++c) Te[6 + c] = P0[c];
        for (int c = 0; c < 5; ++c) {
            Te[10 + c] = -INFINITY;
            Te[15 + c] = INFINITY;
        }
        for (int q = 0; q < nn; ++q) {
            double u[5], P[4];
            for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + q];
            node_prim(0, g, u, P);
            const double w[5] = {u[0], P[0], P[1], P[2], P[3]};
            for (int c = 0; c < 5; ++c) {
                Te[10 + c] = fmax(Te[10 + c], w[c]);
                Te[15 + c] = fmin(Te[15 + c], w[c]);
            }
        }
    }
    long long count = 0;
#pragma omp parallel for reduction(+ : count) schedule(static)
    for (long long e = 0; e < E; ++e) {
        const double *Te = T + 20 * e;
        double theta = 1.0;
        for (int c = 0; c < 5; ++c) {
            const double w0 = Te[5 + c];
            double M = w0 + wid, mm = w0 - wid;
            for (int a = 0; a < dim; ++a)
                for (int sd = -1; sd <= 1; sd += 2) {
                    const double *Tn = T + 20 * neighbour(m, e, a, sd);
                    M = fmax(M, Tn[5 + c]);
                    mm = fmin(mm, Tn[5 + c]);
                }
            const double dmax = Te[10 + c] - w0, dmin = Te[15 + c] - w0;
            const double tiny = 1e-12 * fabs(w0);
            if (fabs(dmax) > tiny) theta = fmin(theta, fabs((M - w0) / dmax));
            if (fabs(dmin) > tiny) theta = fmin(theta, fabs((mm - w0) / dmin));
        }
        if (troubled) troubled[e] = theta < 1.0 ? 0x1f : 0;
        if (!(theta < 1.0)) continue;
        ++count;
        for (int v = 0; v < 5; ++v) {
            const double U0 = Te[v];
            for (int q = 0; q < nn; ++q) {
                double *x = U + (e * 5 + v) * nn + q;
                *x = U0 + theta * (*x - U0);
            }
        }
    }
    free(S);
    free(T);
    return count;
}

long long or_limit(const or_mesh *m, double *U, unsigned char *troubled)
{
    if (m->d.limiter == 0) {
        if (troubled) memset(troubled, 0, (size_t)m->E);
        return 0;
    }
    if (m->d.limiter == 3) return limit_mrs(m, U, troubled);
    const int nn = m->nn, dim = m->d.dim;
    const long long E = m->E;
    double *S = (double *)malloc(sizeof(double) * 10 * 5 * E);
    or_limiter_summaries(m, U, S);
    long long count = 0;
#pragma omp parallel for reduction(+ : count) schedule(static)
    for (long long e = 0; e < E; ++e) {
        int unphys = 0;
        if (m->d.system == 1) {
            for (int q = 0; q < nn && !unphys; ++q) {
                double u[5];
                for (int v = 0; v < 5; ++v) u[v] = U[(e * 5 + v) * nn + q];
                unphys = unphysical_node(u);
            }
        }
        unsigned char mask = 0;
        double slopes[5][3];
        for (int v = 0; v < 5; ++v) {
            const double *Se = S + (e * 5 + v) * 10;
            const double U0 = Se[0];
            int flag = (m->d.limiter == 2) || unphys;
            for (int a = 0; a < dim; ++a) {
                const double U0m = S[(neighbour(m, e, a, -1) * 5 + v) * 10];
                const double U0p = S[(neighbour(m, e, a, +1) * 5 + v) * 10];
                const double ulo = Se[1 + 2 * a], uhi = Se[2 + 2 * a];
                if (m->d.limiter == 1) {
                    const double vl = U0 - minmodB(U0 - ulo, U0 - U0m, U0p - U0, 0.0, m->dx[a]);
                    const double vr = U0 + minmodB(uhi - U0, U0 - U0m, U0p - U0, 0.0, m->dx[a]);
                    if (fabs(vl - ulo) > 1e-8 || fabs(vr - uhi) > 1e-8) flag = 1;
                }
                const double h = m->dx[a] / m->d.beta;
                slopes[v][a] = minmodB(2.0 * Se[7 + a] / m->dx[a], (U0p - U0) / h, (U0 - U0m) / h,
                                       m->d.tvb_M, m->dx[a]);
            }
            if (flag) mask |= (unsigned char)(1u << v);
        }
        if (troubled) troubled[e] = mask;
        if (!mask) continue;
        ++count;
        for (int v = 0; v < 5; ++v) {
            if (!(mask & (1u << v))) continue;
            const double U0 = S[(e * 5 + v) * 10];
            for (int k = 0; k < m->na[2]; ++k)
                for (int j = 0; j < m->na[1]; ++j)
                    for (int i = 0; i < m->na[0]; ++i) {
                        const int id[3] = {i, j, k};
                        double val = U0;
                        for (int a = 0; a < dim; ++a)
                            val = val + slopes[v][a] * (0.5 * m->dx[a] * m->x[id[a]]);
                        U[(e * 5 + v) * nn + node_id(m, i, j, k)] = val;
                    }
        }
    }
    free(S);
    return count;
}

/* Sec. 2.1.4, reading of the fix: D >= d_atm, tau >= tau_atm D, and
 * S^2 <= (1 - 1e-12) tau (tau + 2 D) -- the largest S^2 with a physical
 * primitive state is tau (tau + 2D), from tau + D >= sqrt(S^2 + D^2). */
long long or_fix(const or_mesh *m, double *U)
{
    if (m->d.system != 1) return 0;
    const int nn = m->nn;
    long long changed = 0;
#pragma omp parallel for reduction(+ : changed) schedule(static)
    for (long long e = 0; e < m->E; ++e) {
        for (int q = 0; q < nn; ++q) {
            double *D = &U[(e * 5 + 0) * nn + q];
            double *tau = &U[(e * 5 + 4) * nn + q];
            double *Sx = &U[(e * 5 + 1) * nn + q];
            double *Sy = &U[(e * 5 + 2) * nn + q];
            double *Sz = &U[(e * 5 + 3) * nn + q];
            int ch = 0;
            if (!(*D >= m->d.d_atm)) { *D = m->d.d_atm; ch = 1; }
            const double tmin = m->d.tau_atm * *D;
            if (!(*tau >= tmin)) { *tau = tmin; ch = 1; }
            const double s2 = *Sx * *Sx + *Sy * *Sy + *Sz * *Sz;
            const double s2max = (1.0 - 1e-12) * (*tau * (*tau + 2.0 * *D));
            if (s2 > s2max) {
                const double f = sqrt(s2max / s2);
                *Sx *= f; *Sy *= f; *Sz *= f;
                ch = 1;
            }
            changed += ch;
        }
    }
    return changed;
}

/* SSP-RK3 in Shu-Osher form (Sec. 3.4 cites Gottlieb-Shu; coefficients are the
 * standard three-stage ones):
 *   U1 = Un + dt L(Un);  U2 = 3/4 Un + 1/4 (U1 + dt L(U1));
 *   Un+1 = 1/3 Un + 2/3 (U2 + dt L(U2)),
 * with the limiter and then the SR fix applied after every stage (Sec. 3.3). */
long long or_rk3_step(or_mesh *m, double *U, double dt, unsigned char *troubled_last)
{
    const long long tot = m->E * 5 * m->nn;
    double *Un = (double *)malloc(sizeof(double) * tot);
    double *L = (double *)malloc(sizeof(double) * tot);
    memcpy(Un, U, sizeof(double) * tot);
    const double ca[3] = {0.0, 0.75, 1.0 / 3.0};
    const double cb[3] = {1.0, 0.25, 2.0 / 3.0};
    const double ct[3] = {0.0, 1.0, 0.5};  /* stage times t + ct dt of U, U1, U2 */
    long long fails = 0;
    for (int s = 0; s < 3; ++s) {
        fails += rhs_at(m, U, L, m->t + ct[s] * dt);
#pragma omp parallel for schedule(static)
        for (long long q = 0; q < tot; ++q) {
            const double y = U[q] + dt * L[q];
            U[q] = (s == 0) ? y : ca[s] * Un[q] + cb[s] * y;
        }
        or_limit(m, U, s == 2 ? troubled_last : NULL);
        or_fix(m, U);
    }
    m->t = m->t + dt;
    free(Un);
    free(L);
    return fails;
}

void or_norms(const or_mesh *m, const double *U, const double *V, double *l1, double *l2)
{
    const int nn = m->nn;
    double J = 1.0;
    for (int a = 0; a < m->d.dim; ++a) J *= 0.5 * m->dx[a];
    for (int v = 0; v < 5; ++v) {
        double s1 = 0.0, s2 = 0.0;
        for (long long e = 0; e < m->E; ++e)
            for (int k = 0; k < m->na[2]; ++k)
                for (int j = 0; j < m->na[1]; ++j)
                    for (int i = 0; i < m->na[0]; ++i) {
                        const long long q = (e * 5 + v) * nn + node_id(m, i, j, k);
                        const double wq = wgt(m, 0, i) * wgt(m, 1, j) * wgt(m, 2, k) * J;
                        const double d = U[q] - V[q];
                        s1 += wq * fabs(d);
                        s2 += wq * d * d;
                    }
        l1[v] = s1;
        l2[v] = sqrt(s2);
    }
}

void or_totals(const or_mesh *m, const double *U, double *tot)
{
    const int nn = m->nn;
    double J = 1.0;
    for (int a = 0; a < m->d.dim; ++a) J *= 0.5 * m->dx[a];
    for (int v = 0; v < 5; ++v) {
        double s = 0.0;
        for (long long e = 0; e < m->E; ++e)
            for (int k = 0; k < m->na[2]; ++k)
                for (int j = 0; j < m->na[1]; ++j)
                    for (int i = 0; i < m->na[0]; ++i)
                        s += wgt(m, 0, i) * wgt(m, 1, j) * wgt(m, 2, k) * J *
                             U[(e * 5 + v) * nn + node_id(m, i, j, k)];
        tot[v] = s;
    }
}
