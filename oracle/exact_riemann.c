/*
 * exact_riemann.c -- TEST INFRASTRUCTURE ONLY.
 *
 * Exact solution of the 1D Riemann problem for the Euler equations with a
 * gamma-law gas, used to pin the oracle on the shock-tube and gas-vacuum
 * problems (Sec. 2.3 of arXiv 1912.04855 compares against "the exact solution
 * of the corresponding Riemann problem").  Written from the standard wave
 * analysis: across a shock the Rankine-Hugoniot conditions hold, across a
 * rarefaction the Riemann invariant u +- 2c/(gamma-1) and the entropy are
 * constant; the star pressure is the root of f_L(p) + f_R(p) + u_R - u_L = 0,
 * found by Newton iteration; a vacuum on one side is bounded by the escape
 * front u +- 2c/(gamma-1).
 */
#include <math.h>

#include "cspht_oracle.h"

typedef struct {
    double g, rho, u, p, c;
} Side;

/* Velocity change across the wave that joins a side state to pressure ps,
 * and its derivative in ps. */
static void wave_fn(const Side *s, double ps, double *f, double *df)
{
    double g = s->g;
    if (ps > s->p) { /* shock */
        double A = 2.0 / ((g + 1.0) * s->rho), B = (g - 1.0) / (g + 1.0) * s->p;
        double q = sqrt(A / (ps + B));
        *f = (ps - s->p) * q;
        *df = q * (1.0 - 0.5 * (ps - s->p) / (ps + B));
    } else { /* rarefaction */
        double e = (g - 1.0) / (2.0 * g);
        *f = 2.0 * s->c / (g - 1.0) * (pow(ps / s->p, e) - 1.0);
        *df = 1.0 / (s->rho * s->c) * pow(ps / s->p, -(g + 1.0) / (2.0 * g));
    }
}

int orc_riemann_star(double g, double rl, double ul, double pl, double rr, double ur, double pr,
                     double *pstar, double *ustar)
{
    if (!(rl > 0.0 && rr > 0.0 && pl > 0.0 && pr > 0.0 && g > 1.0)) return ORC_EINVAL;
    Side L = {g, rl, ul, pl, sqrt(g * pl / rl)}, R = {g, rr, ur, pr, sqrt(g * pr / rr)};
    if (2.0 / (g - 1.0) * (L.c + R.c) <= ur - ul) return ORC_EINVAL; /* vacuum is generated */
    /* two-rarefaction estimate as the starting point */
    double e = (g - 1.0) / (2.0 * g);
    double num = L.c + R.c - 0.5 * (g - 1.0) * (ur - ul);
    double den = L.c / pow(pl, e) + R.c / pow(pr, e);
    double p = pow(num / den, 1.0 / e);
    if (!(p > 1e-14)) p = 1e-14;
    for (int it = 0; it < 200; ++it) {
        double fl, dfl, fr, dfr;
        wave_fn(&L, p, &fl, &dfl);
        wave_fn(&R, p, &fr, &dfr);
        double f = fl + fr + (ur - ul);
        double pn = p - f / (dfl + dfr);
        if (pn < 1e-14) pn = 1e-14;
        double ch = fabs(pn - p) / (0.5 * (pn + p));
        p = pn;
        if (ch < 1e-15) break;
    }
    double fl, dfl, fr, dfr;
    wave_fn(&L, p, &fl, &dfl);
    wave_fn(&R, p, &fr, &dfr);
    *pstar = p;
    *ustar = 0.5 * (ul + ur) + 0.5 * (fr - fl);
    return ORC_OK;
}

/* State inside the rarefaction fan of side s at x/t = xs; dir = +1 for a
 * left-facing (left side) fan, -1 for a right-facing fan. */
static void fan(const Side *s, double xs, int dir, double *rho, double *u, double *p)
{
    double g = s->g;
    double c = 2.0 / (g + 1.0) * (s->c + dir * 0.5 * (g - 1.0) * (s->u - xs));
    *u = 2.0 / (g + 1.0) * (dir * s->c + 0.5 * (g - 1.0) * s->u + xs);
    *rho = s->rho * pow(c / s->c, 2.0 / (g - 1.0));
    *p = s->p * pow(c / s->c, 2.0 * g / (g - 1.0));
}

static void sample_one(const Side *L, const Side *R, double ps, double us, double s, double *rho,
                       double *u, double *p)
{
    double g = L->g;
    double G6 = (g - 1.0) / (g + 1.0);
    if (s <= us) {
        if (ps > L->p) {
            double SL = L->u - L->c * sqrt((g + 1.0) / (2.0 * g) * ps / L->p + (g - 1.0) / (2.0 * g));
            if (s <= SL) { *rho = L->rho; *u = L->u; *p = L->p; }
            else { *rho = L->rho * (ps / L->p + G6) / (G6 * ps / L->p + 1.0); *u = us; *p = ps; }
        } else {
            double SH = L->u - L->c;
            double cs = L->c * pow(ps / L->p, (g - 1.0) / (2.0 * g));
            double ST = us - cs;
            if (s <= SH) { *rho = L->rho; *u = L->u; *p = L->p; }
            else if (s > ST) { *rho = L->rho * pow(ps / L->p, 1.0 / g); *u = us; *p = ps; }
            else fan(L, s, +1, rho, u, p);
        }
    } else {
        if (ps > R->p) {
            double SR = R->u + R->c * sqrt((g + 1.0) / (2.0 * g) * ps / R->p + (g - 1.0) / (2.0 * g));
            if (s >= SR) { *rho = R->rho; *u = R->u; *p = R->p; }
            else { *rho = R->rho * (ps / R->p + G6) / (G6 * ps / R->p + 1.0); *u = us; *p = ps; }
        } else {
            double SH = R->u + R->c;
            double cs = R->c * pow(ps / R->p, (g - 1.0) / (2.0 * g));
            double ST = us + cs;
            if (s >= SH) { *rho = R->rho; *u = R->u; *p = R->p; }
            else if (s < ST) { *rho = R->rho * pow(ps / R->p, 1.0 / g); *u = us; *p = ps; }
            else fan(R, s, -1, rho, u, p);
        }
    }
}

int orc_riemann_sample(double g, double rl, double ul, double pl, double rr, double ur, double pr,
                       const double *s, long n, double *rho, double *u, double *p)
{
    if (!(g > 1.0)) return ORC_EINVAL;
    int lvac = !(rl > 0.0 && pl > 0.0), rvac = !(rr > 0.0 && pr > 0.0);
    if (lvac && rvac) {
        for (long i = 0; i < n; ++i) rho[i] = u[i] = p[i] = 0.0;
        return ORC_OK;
    }
    Side L = {g, rl, ul, pl, lvac ? 0.0 : sqrt(g * pl / rl)};
    Side R = {g, rr, ur, pr, rvac ? 0.0 : sqrt(g * pr / rr)};
    if (rvac) { /* gas on the left expands into vacuum */
        double SH = ul - L.c, SF = ul + 2.0 * L.c / (g - 1.0);
        for (long i = 0; i < n; ++i) {
            if (s[i] <= SH) { rho[i] = rl; u[i] = ul; p[i] = pl; }
            else if (s[i] < SF) fan(&L, s[i], +1, &rho[i], &u[i], &p[i]);
            else rho[i] = u[i] = p[i] = 0.0;
        }
        return ORC_OK;
    }
    if (lvac) { /* gas on the right expands into vacuum */
        double SH = ur + R.c, SF = ur - 2.0 * R.c / (g - 1.0);
        for (long i = 0; i < n; ++i) {
            if (s[i] >= SH) { rho[i] = rr; u[i] = ur; p[i] = pr; }
            else if (s[i] > SF) fan(&R, s[i], -1, &rho[i], &u[i], &p[i]);
            else rho[i] = u[i] = p[i] = 0.0;
        }
        return ORC_OK;
    }
    double ps, us;
    int rc = orc_riemann_star(g, rl, ul, pl, rr, ur, pr, &ps, &us);
    if (rc) return rc;
    for (long i = 0; i < n; ++i) sample_one(&L, &R, ps, us, s[i], &rho[i], &u[i], &p[i]);
    return ORC_OK;
}
