/*
 * cspht_oracle.c -- TEST INFRASTRUCTURE ONLY.
 *
 * A plain, slow, single-precision-free (FP64) CPU definition of one CSPH-TVD
 * time step (Khrapov, Khoperskov & Khoperskov, arXiv 1912.04855).  Only the
 * test-suite, the smoke check and the CPU-baseline leg of the benchmark use
 * it; the CUDA library never links, calls or includes anything from here, and
 * this file includes nothing from the CUDA library.
 *
 * The step is written stage by stage in the paper's order, one whole-box loop
 * per stage, with no fusion or reordering:
 *
 *   stage 0  U^n, particles at the cell centres (xi = 0)           Sec. 2.2
 *   stage 1  predictor  U*  = U^n + dt Q(U^n, r^n),  r* (Eq. 5)
 *   stage 2  corrector  U~  = (U^n + U*)/2 + dt/2 Q(U*, r*), r^{n+1} (Eq. 6)
 *   Euler    U^{n+1} = U~ - dt/h (F+ - F- + G+ - G- + H+ - H-)      (Eq. 4)
 *            with faces reconstructed by Eq. 8 and a Riemann flux.
 *
 * Q is the modified-SPH force of Eq. 7 with phi = sqrt(2p).  Where the paper
 * is silent the following readings are used (they are the same readings the
 * CUDA path implements, written independently there):
 *   - force sign from the physics of Eqs. 2-3: dm/dt = -grad p - rho grad psi,
 *     dE/dt = -div(p u) - rho u.grad psi;
 *   - particle positions stored as offsets xi = r - x_cell, xi^n = 0;
 *   - Eq. 4 fluxes are advective only: F = a U with the face speed a;
 *   - density is not changed by the Lagrangian stage (Q_rho = 0);
 *   - smoothing kernel: M4 cubic spline, support 2h, with the weight
 *     G(r) = gt(r/h) / (C h^2), gt(q) = -W'(q)/q, and C fixed so that the
 *     27-point lattice gradient is exact on linear fields;
 *   - gravity: f_i = -D0_i[psi], the same 27-point operator on the static
 *     lattice (this makes hydrostatic states discrete equilibria);
 *   - vacuum: rho <= rho_vac means u = 0, p = 0, phi = 0 and Q = 0;
 *     pressure floor p = max(p, 0);
 *   - u_star = m_star / rho^n and u^{n+1} = m~ / rho^n (density is unchanged
 *     by the stage);
 *   - slopes Theta^n: limiter of one-sided differences of U^n (van Leer
 *     default, minmod, MC); U^{n+1/2} = (U^n + U~)/2;
 *   - face speed a = xi^{n+1}_d / dt; Lax-Friedrichs (default) or HLL flux
 *     on the advective system;
 *   - boundaries, per stage, one ghost layer, resolved z then y then x:
 *     periodic (wrap), outflow (copy of the boundary cell, incl. xi, ghost
 *     slope 0), inflow (fixed primitive state, ghost xi = dt u_in after the
 *     predictor, slope 0), reflecting wall (zero face flux, mirrored u and
 *     xi, hydrostatically extrapolated phi);
 *   - ghost psi: wrapped for periodic faces, linearly extrapolated otherwise;
 *   - dt = CFL h / max over gas cells of (max_d |u_d| + c).
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include "cspht_oracle.h"

/* ---------------------------------------------------------------- kernel */

/* M4 cubic spline in q = r/h (support 2): W ~ 1 - 1.5q^2 + 0.75q^3 (q < 1),
 * 0.25 (2-q)^3 (1 <= q < 2).  gt(q) = -W'(q)/q, the radial weight of the
 * SPH gradient (Eq. 7, the kernel W of Sec. 2.2). */
double orc_gtilde(double q)
{
    if (q < 1.0) return 3.0 - 2.25 * q;
    if (q < 2.0) return 0.75 * (2.0 - q) * (2.0 - q) / q;
    return 0.0;
}

/* Lattice normalisation: sum over the 26 neighbours of gt(|d|) d_x^2.
 * Written as the plain sum so that the constant follows from gt itself. */
double orc_norm_C(void)
{
    double s = 0.0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy && !dz) continue;
                double q = sqrt((double)(dx * dx + dy * dy + dz * dz));
                s += orc_gtilde(q) * dx * dx;
            }
    return s;
}

/* ----------------------------------------------------------------- state */

typedef struct {
    double U[5];   /* content carried by the particle: rho, mx, my, mz, E */
    double xi[3];  /* particle offset from its cell centre */
    double u[3];   /* velocity */
    double p, phi; /* pressure and phi = sqrt(2p) */
    int vac;       /* vacuum flag */
} Rec;

typedef struct {
    int cnt[3];
    int *map[3]; /* global index -> local index, -1 when not held */
    Rec *r;
} Stage;

typedef struct {
    const orc_cfg *c;
    const double *psi;
    const double *U; /* stage-0 content, full domain, SoA */
    double dt;
    double C;
    size_t N;
    Stage st[3]; /* st[0] U^n with primitives, st[1] predictor, st[2] corrector */
} Ctx;

/* Primitive recovery, Sec. 2.1 (EOS p = (gamma-1) rho eps) with the vacuum
 * threshold and the pressure floor. */
static void eos(const orc_cfg *c, Rec *r)
{
    double rho = r->U[0];
    if (!(rho > c->rho_vac)) {
        r->vac = 1;
        r->u[0] = r->u[1] = r->u[2] = 0.0;
        r->p = 0.0;
        r->phi = 0.0;
        return;
    }
    r->vac = 0;
    for (int e = 0; e < 3; ++e) r->u[e] = r->U[1 + e] / rho;
    double kin = 0.5 * (r->U[1] * r->u[0] + r->U[2] * r->u[1] + r->U[3] * r->u[2]);
    double p = (c->gamma - 1.0) * (r->U[4] - kin);
    if (p < 0.0) p = 0.0;
    r->p = p;
    r->phi = sqrt(2.0 * p);
}

static size_t gidx(const Ctx *x, int i, int j, int k)
{
    return ((size_t)k * x->c->n[1] + j) * x->c->n[0] + i;
}

static Rec rec_interior(const Ctx *x, int s, int i, int j, int k)
{
    const Stage *S = &x->st[s];
    int li = S->map[0][i], lj = S->map[1][j], lk = S->map[2][k];
    if (li < 0 || lj < 0 || lk < 0) abort(); /* a stage read outside what was computed */
    return S->r[((size_t)lk * S->cnt[1] + lj) * S->cnt[0] + li];
}

static int wrapi(int a, int n) { return ((a % n) + n) % n; }

/* Ghost psi (static): wrap across periodic faces, linear extrapolation
 * 2 psi_b - psi_m across every other face; resolved z, then y, then x. */
static double psi_at(const Ctx *x, int i, int j, int k)
{
    int id[3] = {i, j, k};
    for (int d = 2; d >= 0; --d) {
        int n = x->c->n[d];
        if (id[d] >= 0 && id[d] < n) continue;
        int side = id[d] < 0 ? 0 : 1;
        if (x->c->bc[2 * d + side] == ORC_BC_PERIODIC) {
            id[d] = wrapi(id[d], n);
            return psi_at(x, id[0], id[1], id[2]);
        }
        int b[3] = {id[0], id[1], id[2]}, m[3];
        b[d] = side ? n - 1 : 0;
        memcpy(m, b, sizeof m);
        if (n > 1) m[d] = side ? n - 2 : 1;
        return 2.0 * psi_at(x, b[0], b[1], b[2]) - psi_at(x, m[0], m[1], m[2]);
    }
    return x->psi[gidx(x, i, j, k)];
}

static Rec inflow_rec(const Ctx *x, int s, int face)
{
    const orc_cfg *c = x->c;
    const double *W = c->inflow[face];
    Rec r;
    double rho = W[0];
    r.U[0] = rho;
    for (int e = 0; e < 3; ++e) r.U[1 + e] = rho * W[1 + e];
    r.U[4] = W[4] / (c->gamma - 1.0) + 0.5 * rho * (W[1] * W[1] + W[2] * W[2] + W[3] * W[3]);
    if (!(rho > c->rho_vac)) {
        r.vac = 1;
        r.u[0] = r.u[1] = r.u[2] = 0.0;
        r.p = r.phi = 0.0;
    } else {
        r.vac = 0;
        for (int e = 0; e < 3; ++e) r.u[e] = W[1 + e];
        r.p = W[4] > 0.0 ? W[4] : 0.0;
        r.phi = sqrt(2.0 * r.p);
    }
    for (int e = 0; e < 3; ++e) r.xi[e] = s ? x->dt * r.u[e] : 0.0;
    return r;
}

static Rec get_rec(const Ctx *x, int s, int i, int j, int k);

/* Reflecting wall across the face normal to d.  b = boundary cell, m = the
 * cell beyond b (the mirror of the ghost through b's centre).  phi of the
 * ghost keeps the discrete hydrostatic balance of cell b:
 *   phi_b (phi_m - phi_g) + rho_b (psi_m - psi_g) = 0.                     */
static Rec wall_rec(const Ctx *x, int s, const int g[3], int d, int side)
{
    const orc_cfg *c = x->c;
    int n = c->n[d];
    int b[3] = {g[0], g[1], g[2]}, m[3];
    b[d] = side ? n - 1 : 0;
    memcpy(m, b, sizeof m);
    if (n > 1) m[d] = side ? n - 2 : 1;
    Rec rb = get_rec(x, s, b[0], b[1], b[2]);
    Rec rm = get_rec(x, s, m[0], m[1], m[2]);
    Rec r = rb;
    r.u[d] = -rb.u[d];
    r.xi[d] = -rb.xi[d];
    double rho_g = rb.U[0];
    if (rb.vac || !(rb.phi > 0.0)) {
        r.phi = 0.0;
        r.p = 0.0;
    } else {
        double psig = psi_at(x, g[0], g[1], g[2]);
        double psim = psi_at(x, m[0], m[1], m[2]);
        double phig = rm.phi + rb.U[0] * (psim - psig) / rb.phi;
        if (phig < 0.0) phig = 0.0;
        double ratio = phig / rb.phi;
        r.phi = phig;
        r.p = 0.5 * phig * phig;
        rho_g = rb.U[0] * ratio * ratio;
    }
    r.U[0] = rho_g;
    if (rb.vac) {
        for (int e = 0; e < 3; ++e) r.U[1 + e] = rb.U[1 + e];
        r.U[1 + d] = -rb.U[1 + d];
        r.U[4] = rb.U[4];
    } else {
        for (int e = 0; e < 3; ++e) r.U[1 + e] = rho_g * r.u[e];
        r.U[4] = r.p / (c->gamma - 1.0) +
                 0.5 * rho_g * (r.u[0] * r.u[0] + r.u[1] * r.u[1] + r.u[2] * r.u[2]);
    }
    return r;
}

/* Record of stage s at (i,j,k), resolving one ghost layer per stage. */
static Rec get_rec(const Ctx *x, int s, int i, int j, int k)
{
    const orc_cfg *c = x->c;
    int id[3] = {i, j, k};
    for (int d = 2; d >= 0; --d) {
        int n = c->n[d];
        if (id[d] >= 0 && id[d] < n) continue;
        int side = id[d] < 0 ? 0 : 1;
        int t = c->bc[2 * d + side];
        if (t == ORC_BC_PERIODIC) {
            id[d] = wrapi(id[d], n);
            return get_rec(x, s, id[0], id[1], id[2]);
        }
        if (t == ORC_BC_OUTFLOW) {
            id[d] = side ? n - 1 : 0;
            return get_rec(x, s, id[0], id[1], id[2]);
        }
        if (t == ORC_BC_INFLOW) return inflow_rec(x, s, 2 * d + side);
        return wall_rec(x, s, id, d, side);
    }
    return rec_interior(x, s, i, j, k);
}

/* ----------------------------------------------------------- Lagrangian */

/* D0_i[psi] = sum_j G(h|d_j|) h d_j psi_j: the 27-point gradient operator of
 * Eq. 7 on the static lattice, applied to the potential (gravity f = -D0). */
static void lattice_gravity(const Ctx *x, int i, int j, int k, double D0[3])
{
    const double h = x->c->h;
    D0[0] = D0[1] = D0[2] = 0.0;
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy && !dz) continue;
                int d[3] = {dx, dy, dz};
                double q0 = sqrt((double)(dx * dx + dy * dy + dz * dz));
                double G0 = orc_gtilde(q0) / (x->C * h * h);
                double ps = psi_at(x, i + dx, j + dy, k + dz);
                for (int e = 0; e < 3; ++e) D0[e] += G0 * (h * d[e]) * ps;
            }
}

/* Q_i of Eq. 7 for cell (i,j,k) from the records of stage s: the pressure
 * term phi_i sum_j phi_j G_ij (r_j - r_i), the pressure-work term
 * phi_i sum_j phi_j G_ij (r_j - r_i).(u_i + u_j)/2, and gravity with
 * f_i = -D0_i[psi] on the static lattice.  Q = (d mx, d my, d mz, d E)/dt. */
static void force(const Ctx *x, int s, int i, int j, int k, double Q[4])
{
    const double h = x->c->h;
    Rec ri = get_rec(x, s, i, j, k);
    Q[0] = Q[1] = Q[2] = Q[3] = 0.0;
    if (ri.vac) return;
    double P[3] = {0.0, 0.0, 0.0}, Wk = 0.0, D0[3];
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy && !dz) continue;
                int d[3] = {dx, dy, dz};
                Rec rj = get_rec(x, s, i + dx, j + dy, k + dz);
                double r[3], r2 = 0.0;
                for (int e = 0; e < 3; ++e) {
                    r[e] = h * d[e] + (rj.xi[e] - ri.xi[e]);
                    r2 += r[e] * r[e];
                }
                double G = orc_gtilde(sqrt(r2) / h) / (x->C * h * h);
                double ru = 0.0;
                for (int e = 0; e < 3; ++e) {
                    P[e] += G * r[e] * rj.phi;
                    ru += r[e] * 0.5 * (ri.u[e] + rj.u[e]);
                }
                Wk += G * ru * rj.phi;
            }
    lattice_gravity(x, i, j, k, D0);
    double rho = ri.U[0];
    for (int e = 0; e < 3; ++e) Q[e] = -ri.phi * P[e] - rho * D0[e];
    Q[3] = -ri.phi * Wk - rho * (ri.u[0] * D0[0] + ri.u[1] * D0[1] + ri.u[2] * D0[2]);
}

/* ------------------------------------------------------------- Eulerian */

static double limiter(int kind, double a, double b)
{
    if (!(a * b > 0.0)) return 0.0;
    if (kind == ORC_LIM_MINMOD) return fabs(a) < fabs(b) ? a : b;
    if (kind == ORC_LIM_MC) {
        double m = fabs(2.0 * a);
        if (fabs(2.0 * b) < m) m = fabs(2.0 * b);
        if (fabs(0.5 * (a + b)) < m) m = fabs(0.5 * (a + b));
        return a > 0.0 ? m : -m;
    }
    return 2.0 * a * b / (a + b); /* van Leer */
}

/* Slope Theta^n_d of the conserved components at cell c (which may be a
 * ghost only along d): periodic ghosts take the slope of the wrapped cell,
 * other ghosts have slope 0. */
static void slope(const Ctx *x, int d, const int c_in[3], double th[5])
{
    const orc_cfg *c = x->c;
    int cc[3] = {c_in[0], c_in[1], c_in[2]};
    int n = c->n[d];
    if (cc[d] < 0 || cc[d] >= n) {
        int side = cc[d] < 0 ? 0 : 1;
        if (c->bc[2 * d + side] != ORC_BC_PERIODIC) {
            for (int f = 0; f < 5; ++f) th[f] = 0.0;
            return;
        }
        cc[d] = wrapi(cc[d], n);
    }
    int lo[3] = {cc[0], cc[1], cc[2]}, hi[3] = {cc[0], cc[1], cc[2]};
    lo[d] -= 1;
    hi[d] += 1;
    Rec rm = get_rec(x, 0, lo[0], lo[1], lo[2]);
    Rec r0 = get_rec(x, 0, cc[0], cc[1], cc[2]);
    Rec rp = get_rec(x, 0, hi[0], hi[1], hi[2]);
    for (int f = 0; f < 5; ++f)
        th[f] = limiter(c->limiter, (rp.U[f] - r0.U[f]) / c->h, (r0.U[f] - rm.U[f]) / c->h);
}

/* Flux through the face between L and R = L + e_d at t_{n+1/2}:
 * Eq. 8 reconstruction with the particle offsets, then LF, HLL or the
 * swept-volume upwind flux (Sec. 2.2 names several Riemann solvers) on the
 * advective system F = a U. */
static void face_flux(const Ctx *x, int d, const int L[3], double F[5])
{
    const orc_cfg *c = x->c;
    const double h = c->h, dt = x->dt;
    int R[3] = {L[0], L[1], L[2]};
    R[d] += 1;
    if ((L[d] == -1 && c->bc[2 * d] == ORC_BC_WALL) ||
        (R[d] == c->n[d] && c->bc[2 * d + 1] == ORC_BC_WALL)) {
        for (int f = 0; f < 5; ++f) F[f] = 0.0;
        return;
    }
    double thL[5], thR[5];
    slope(x, d, L, thL);
    slope(x, d, R, thR);
    Rec a0 = get_rec(x, 0, L[0], L[1], L[2]), a2 = get_rec(x, 2, L[0], L[1], L[2]);
    Rec b0 = get_rec(x, 0, R[0], R[1], R[2]), b2 = get_rec(x, 2, R[0], R[1], R[2]);
    double xL = a2.xi[d], xR = b2.xi[d];
    double aL = xL / dt, aR = xR / dt;
    double UL[5], UR[5];
    for (int f = 0; f < 5; ++f) {
        UL[f] = 0.5 * (a0.U[f] + a2.U[f]) + 0.5 * (h - xL) * thL[f];
        UR[f] = 0.5 * (b0.U[f] + b2.U[f]) - 0.5 * (h + xR) * thR[f];
    }
    if (c->riemann == ORC_RIEMANN_HLL || c->riemann == ORC_RIEMANN_HLLC) { /* HLLC reads as HLL */
        double SL = aL < aR ? aL : aR, SR = aL < aR ? aR : aL;
        for (int f = 0; f < 5; ++f) {
            if (SL >= 0.0) F[f] = aL * UL[f];
            else if (SR <= 0.0) F[f] = aR * UR[f];
            else F[f] = (SR * aL * UL[f] - SL * aR * UR[f] + SL * SR * (UR[f] - UL[f])) / (SR - SL);
        }
        return;
    }
    if (c->riemann == ORC_RIEMANN_SWEPT) {
        /* the face moves with the mean offset of its two particles; the volume
           it sweeps carries the reconstructed state of the upwind side */
        double a = 0.5 * (aL + aR);
        for (int f = 0; f < 5; ++f) F[f] = a >= 0.0 ? a * UL[f] : a * UR[f];
        return;
    }
    double smax = fabs(aL) > fabs(aR) ? fabs(aL) : fabs(aR);
    for (int f = 0; f < 5; ++f)
        F[f] = 0.5 * (aL * UL[f] + aR * UR[f]) - 0.5 * smax * (UR[f] - UL[f]);
}

/* --------------------------------------------------------------- stages */

static int build_stage(Ctx *x, int s, const int lo[3], const int hi[3], int margin)
{
    Stage *S = &x->st[s];
    for (int d = 0; d < 3; ++d) {
        int n = x->c->n[d];
        int per = x->c->bc[2 * d] == ORC_BC_PERIODIC;
        S->map[d] = (int *)malloc(sizeof(int) * n);
        if (!S->map[d]) return -1;
        for (int a = 0; a < n; ++a) S->map[d][a] = -1;
        for (int a = lo[d] - margin; a < hi[d] + margin; ++a) {
            int g = a;
            if (g < 0 || g >= n) {
                if (!per) continue;
                g = wrapi(g, n);
            }
            S->map[d][g] = 0;
        }
        int cnt = 0;
        for (int a = 0; a < n; ++a)
            if (S->map[d][a] == 0) S->map[d][a] = cnt++;
        S->cnt[d] = cnt;
    }
    S->r = (Rec *)calloc((size_t)S->cnt[0] * S->cnt[1] * S->cnt[2], sizeof(Rec));
    return S->r ? 0 : -1;
}

static void free_stage(Stage *S)
{
    for (int d = 0; d < 3; ++d) free(S->map[d]);
    free(S->r);
    memset(S, 0, sizeof *S);
}

/* Inverse of a stage map: local index -> global index. */
static void inverse_map(const Stage *S, int d, int n, int *inv)
{
    for (int a = 0; a < n; ++a)
        if (S->map[d][a] >= 0) inv[S->map[d][a]] = a;
}

/* Stage 0 (step a1): primitive recovery of U^n on every cell held, with the
 * particles at the cell centres. */
static void run_primitives(Ctx *x)
{
    Stage *S = &x->st[0];
    int *inv[3];
    for (int d = 0; d < 3; ++d) {
        inv[d] = (int *)malloc(sizeof(int) * (S->cnt[d] ? S->cnt[d] : 1));
        inverse_map(S, d, x->c->n[d], inv[d]);
    }
#pragma omp parallel for collapse(2) schedule(static)
    for (int lk = 0; lk < S->cnt[2]; ++lk)
        for (int lj = 0; lj < S->cnt[1]; ++lj)
            for (int li = 0; li < S->cnt[0]; ++li) {
                size_t g = gidx(x, inv[0][li], inv[1][lj], inv[2][lk]);
                Rec r;
                for (int f = 0; f < 5; ++f) r.U[f] = x->U[(size_t)f * x->N + g];
                r.xi[0] = r.xi[1] = r.xi[2] = 0.0;
                eos(x->c, &r);
                S->r[((size_t)lk * S->cnt[1] + lj) * S->cnt[0] + li] = r;
            }
    for (int d = 0; d < 3; ++d) free(inv[d]);
}

/* Predictor (Eq. 5) on every cell held by stage 1. */
static void run_predictor(Ctx *x)
{
    Stage *S = &x->st[1];
    int *inv[3];
    for (int d = 0; d < 3; ++d) {
        inv[d] = (int *)malloc(sizeof(int) * (S->cnt[d] ? S->cnt[d] : 1));
        inverse_map(S, d, x->c->n[d], inv[d]);
    }
    const double dt = x->dt;
#pragma omp parallel for collapse(2) schedule(static)
    for (int lk = 0; lk < S->cnt[2]; ++lk)
        for (int lj = 0; lj < S->cnt[1]; ++lj)
            for (int li = 0; li < S->cnt[0]; ++li) {
                int i = inv[0][li], j = inv[1][lj], k = inv[2][lk];
                Rec r0 = rec_interior(x, 0, i, j, k);
                double Q[4];
                force(x, 0, i, j, k, Q);
                Rec r1;
                r1.U[0] = r0.U[0];
                for (int f = 1; f < 5; ++f) r1.U[f] = r0.U[f] + dt * Q[f - 1];
                eos(x->c, &r1);
                for (int e = 0; e < 3; ++e) r1.xi[e] = r0.xi[e] + dt * 0.5 * (r0.u[e] + r1.u[e]);
                S->r[((size_t)lk * S->cnt[1] + lj) * S->cnt[0] + li] = r1;
            }
    for (int d = 0; d < 3; ++d) free(inv[d]);
}

/* Corrector (Eq. 6) on every cell held by stage 2. */
static void run_corrector(Ctx *x)
{
    Stage *S = &x->st[2];
    int *inv[3];
    for (int d = 0; d < 3; ++d) {
        inv[d] = (int *)malloc(sizeof(int) * (S->cnt[d] ? S->cnt[d] : 1));
        inverse_map(S, d, x->c->n[d], inv[d]);
    }
    const double dt = x->dt;
#pragma omp parallel for collapse(2) schedule(static)
    for (int lk = 0; lk < S->cnt[2]; ++lk)
        for (int lj = 0; lj < S->cnt[1]; ++lj)
            for (int li = 0; li < S->cnt[0]; ++li) {
                int i = inv[0][li], j = inv[1][lj], k = inv[2][lk];
                Rec r0 = rec_interior(x, 0, i, j, k);
                Rec r1 = rec_interior(x, 1, i, j, k);
                double Q[4];
                force(x, 1, i, j, k, Q);
                Rec r2;
                r2.U[0] = 0.5 * (r0.U[0] + r1.U[0]);
                for (int f = 1; f < 5; ++f) r2.U[f] = 0.5 * (r0.U[f] + r1.U[f]) + 0.5 * dt * Q[f - 1];
                eos(x->c, &r2);
                for (int e = 0; e < 3; ++e)
                    r2.xi[e] = 0.5 * (r0.xi[e] + r1.xi[e]) + 0.5 * dt * 0.5 * (r0.u[e] + r2.u[e]);
                S->r[((size_t)lk * S->cnt[1] + lj) * S->cnt[0] + li] = r2;
            }
    for (int d = 0; d < 3; ++d) free(inv[d]);
}

static void ctx_init(Ctx *x, const orc_cfg *c, const double *psi, const double *U, double dt)
{
    memset(x, 0, sizeof *x);
    x->c = c;
    x->psi = psi;
    x->U = U;
    x->dt = dt;
    x->C = orc_norm_C();
    x->N = (size_t)c->n[0] * c->n[1] * c->n[2];
}

static int cfg_ok(const orc_cfg *c)
{
    for (int d = 0; d < 3; ++d) {
        if (c->n[d] < 1) return 0;
        int a = c->bc[2 * d] == ORC_BC_PERIODIC, b = c->bc[2 * d + 1] == ORC_BC_PERIODIC;
        if (a != b) return 0;
        if (!a && c->n[d] < 2) return 0;
    }
    return c->h > 0.0 && c->gamma > 1.0;
}

/* --------------------------------------------------------------- public */

int orc_step(const orc_cfg *c, const double *psi, const double *U, double dt, double *Uout,
             const int *box)
{
    if (!cfg_ok(c)) return ORC_EINVAL;
    Ctx x;
    ctx_init(&x, c, psi, U, dt);
    int lo[3] = {0, 0, 0}, hi[3] = {c->n[0], c->n[1], c->n[2]};
    if (box)
        for (int d = 0; d < 3; ++d) {
            lo[d] = box[2 * d];
            hi[d] = box[2 * d + 1];
            if (lo[d] < 0 || hi[d] > c->n[d] || lo[d] >= hi[d]) return ORC_EINVAL;
        }
    size_t N = x.N;
    if (!(dt > 0.0)) { /* a zero step leaves the state as it is */
        for (int k = lo[2]; k < hi[2]; ++k)
            for (int j = lo[1]; j < hi[1]; ++j)
                for (int i = lo[0]; i < hi[0]; ++i) {
                    size_t g = gidx(&x, i, j, k);
                    for (int f = 0; f < 5; ++f) Uout[f * N + g] = U[f * N + g];
                }
        return ORC_OK;
    }
    if (build_stage(&x, 0, lo, hi, 3) || build_stage(&x, 1, lo, hi, 2) ||
        build_stage(&x, 2, lo, hi, 1)) {
        for (int s = 0; s < 3; ++s) free_stage(&x.st[s]);
        return ORC_ENOMEM;
    }
    run_primitives(&x);
    run_predictor(&x);
    run_corrector(&x);
    const double h = c->h;
    int bad = 0;
#pragma omp parallel for collapse(2) schedule(static) reduction(| : bad)
    for (int k = lo[2]; k < hi[2]; ++k)
        for (int j = lo[1]; j < hi[1]; ++j)
            for (int i = lo[0]; i < hi[0]; ++i) {
                int cc[3] = {i, j, k};
                Rec r2 = rec_interior(&x, 2, i, j, k);
                double div[5] = {0, 0, 0, 0, 0};
                for (int d = 0; d < 3; ++d) {
                    int Lm[3] = {i, j, k};
                    Lm[d] -= 1;
                    double Fp[5], Fm[5];
                    face_flux(&x, d, cc, Fp);
                    face_flux(&x, d, Lm, Fm);
                    for (int f = 0; f < 5; ++f) div[f] += Fp[f] - Fm[f];
                }
                size_t g = gidx(&x, i, j, k);
                for (int f = 0; f < 5; ++f) {
                    double v = r2.U[f] - dt / h * div[f];
                    Uout[f * N + g] = v;
                    if (!isfinite(v)) bad = 1;
                }
            }
    for (int s = 0; s < 3; ++s) free_stage(&x.st[s]);
    return bad ? ORC_ENONFINITE : ORC_OK;
}

double orc_max_speed(const orc_cfg *c, const double *U)
{
    size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
    double smax = 0.0;
    for (size_t g = 0; g < N; ++g) {
        Rec r;
        for (int f = 0; f < 5; ++f) r.U[f] = U[f * N + g];
        eos(c, &r);
        if (r.vac) continue;
        double um = fabs(r.u[0]);
        if (fabs(r.u[1]) > um) um = fabs(r.u[1]);
        if (fabs(r.u[2]) > um) um = fabs(r.u[2]);
        double s = um + sqrt(c->gamma * r.p / r.U[0]);
        if (!(s <= smax)) smax = s; /* NaN propagates */
    }
    return smax;
}

double orc_dt(const orc_cfg *c, const double *U, double cfl)
{
    double s = orc_max_speed(c, U);
    return s > 0.0 ? cfl * c->h / s : 0.0;
}

int orc_run(const orc_cfg *c, const double *psi, double *U, long nsteps, double cfl, double t_end,
            double *t_io, long *steps_out)
{
    size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
    double *tmp = (double *)malloc(sizeof(double) * 5 * N);
    if (!tmp) return ORC_ENOMEM;
    double t = t_io ? *t_io : 0.0;
    long s = 0;
    int rc = ORC_OK;
    while ((nsteps < 0 || s < nsteps) && t < t_end) {
        double dt = orc_dt(c, U, cfl);
        int last = 0;
        if (dt >= t_end - t) { /* the last step lands exactly on t_end */
            dt = t_end - t;
            last = 1;
        }
        if (!(dt > 0.0)) break;
        rc = orc_step(c, psi, U, dt, tmp, NULL);
        memcpy(U, tmp, sizeof(double) * 5 * N);
        t = last ? t_end : t + dt;
        ++s;
        if (rc) break;
    }
    free(tmp);
    if (t_io) *t_io = t;
    if (steps_out) *steps_out = s;
    return rc;
}

/* Totals (times h^3) in a fixed order: mass, momentum, E, E + rho psi. */
void orc_totals(const orc_cfg *c, const double *psi, const double *U, double out[6])
{
    size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
    double v = c->h * c->h * c->h;
    for (int f = 0; f < 6; ++f) out[f] = 0.0;
    for (size_t g = 0; g < N; ++g) {
        for (int f = 0; f < 5; ++f) out[f] += U[f * N + g];
        out[5] += U[4 * N + g] + U[g] * psi[g];
    }
    for (int f = 0; f < 6; ++f) out[f] *= v;
}

/* Primitive (rho,u,v,w,p) -> conserved (rho,mx,my,mz,E), SoA, N cells. */
void orc_prim_to_cons(double gamma, const double *W, double *U, long N)
{
    for (long g = 0; g < N; ++g) {
        double rho = W[g], u = W[N + g], v = W[2 * N + g], w = W[3 * N + g], p = W[4 * N + g];
        U[g] = rho;
        U[N + g] = rho * u;
        U[2 * N + g] = rho * v;
        U[3 * N + g] = rho * w;
        U[4 * N + g] = p / (gamma - 1.0) + 0.5 * rho * (u * u + v * v + w * w);
    }
}

/* Primitive recovery of every cell: u (3N), p, phi, vacuum flag. */
void orc_eos(const orc_cfg *c, const double *U, double *u, double *p, double *phi, int *vac)
{
    size_t N = (size_t)c->n[0] * c->n[1] * c->n[2];
    for (size_t g = 0; g < N; ++g) {
        Rec r;
        for (int f = 0; f < 5; ++f) r.U[f] = U[f * N + g];
        eos(c, &r);
        for (int e = 0; e < 3; ++e) u[e * N + g] = r.u[e];
        p[g] = r.p;
        phi[g] = r.phi;
        vac[g] = r.vac;
    }
}

/* Q of Eq. 7 at every cell.  xi == NULL: particles at the cell centres
 * (stage-0 ghosts).  Otherwise the particles sit at x_cell + xi with the
 * content U, and ghosts follow the post-predictor rules (inflow xi = dt u). */
int orc_force(const orc_cfg *c, const double *psi, const double *U, const double *xi, double dt,
              double *Q)
{
    if (!cfg_ok(c)) return ORC_EINVAL;
    Ctx x;
    ctx_init(&x, c, psi, U, dt);
    size_t N = x.N;
    int s = 0;
    int lo[3] = {0, 0, 0}, hi[3] = {c->n[0], c->n[1], c->n[2]};
    if (build_stage(&x, 0, lo, hi, 0)) return ORC_ENOMEM;
    run_primitives(&x);
    if (xi) {
        if (build_stage(&x, 1, lo, hi, 0)) {
            free_stage(&x.st[0]);
            return ORC_ENOMEM;
        }
        for (int k = 0; k < c->n[2]; ++k)
            for (int j = 0; j < c->n[1]; ++j)
                for (int i = 0; i < c->n[0]; ++i) {
                    size_t g = gidx(&x, i, j, k);
                    Rec r;
                    for (int f = 0; f < 5; ++f) r.U[f] = U[f * N + g];
                    eos(c, &r);
                    for (int e = 0; e < 3; ++e) r.xi[e] = xi[e * N + g];
                    x.st[1].r[g] = r;
                }
        s = 1;
    }
    for (int k = 0; k < c->n[2]; ++k)
        for (int j = 0; j < c->n[1]; ++j)
            for (int i = 0; i < c->n[0]; ++i) {
                double q[4];
                force(&x, s, i, j, k, q);
                size_t g = gidx(&x, i, j, k);
                for (int e = 0; e < 4; ++e) Q[e * N + g] = q[e];
            }
    free_stage(&x.st[0]);
    free_stage(&x.st[1]);
    return ORC_OK;
}

/* The Lagrangian stage alone (Eqs. 5-6) on the whole domain: U*, xi*,
 * U~^{n+1}, xi^{n+1}. */
int orc_lagrange(const orc_cfg *c, const double *psi, const double *U, double dt, double *Us,
                 double *xis, double *Un, double *xin)
{
    if (!cfg_ok(c)) return ORC_EINVAL;
    Ctx x;
    ctx_init(&x, c, psi, U, dt);
    int lo[3] = {0, 0, 0}, hi[3] = {c->n[0], c->n[1], c->n[2]};
    if (build_stage(&x, 0, lo, hi, 0) || build_stage(&x, 1, lo, hi, 0) ||
        build_stage(&x, 2, lo, hi, 0)) {
        for (int s = 0; s < 3; ++s) free_stage(&x.st[s]);
        return ORC_ENOMEM;
    }
    run_primitives(&x);
    run_predictor(&x);
    run_corrector(&x);
    size_t N = x.N;
    for (size_t g = 0; g < N; ++g) {
        const Rec *a = &x.st[1].r[g], *b = &x.st[2].r[g];
        for (int f = 0; f < 5; ++f) {
            Us[f * N + g] = a->U[f];
            Un[f * N + g] = b->U[f];
        }
        for (int e = 0; e < 3; ++e) {
            xis[e * N + g] = a->xi[e];
            xin[e * N + g] = b->xi[e];
        }
    }
    for (int s = 0; s < 3; ++s) free_stage(&x.st[s]);
    return ORC_OK;
}
