/*
 * cspht_oracle.h -- TEST INFRASTRUCTURE ONLY.
 *
 * Declarations of the FP64 CPU oracle of the CSPH-TVD step (Sec. 2.2 of
 * arXiv 1912.04855) and of the exact Riemann solver used to pin it.  Only the
 * tests, the smoke check and the benchmark's CPU-baseline leg use these; the
 * CUDA library shares no header, code or table with them.
 *
 * Arrays are structure-of-arrays over N = nx*ny*nz cells, x fastest:
 * field f of cell (i,j,k) sits at [f*N + (k*ny + j)*nx + i].
 */
#ifndef CSPHT_ORACLE_H
#define CSPHT_ORACLE_H

#ifdef __cplusplus
extern "C" {
#endif

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_ENONFINITE = -4 };
enum { ORC_BC_PERIODIC = 0, ORC_BC_OUTFLOW = 1, ORC_BC_INFLOW = 2, ORC_BC_WALL = 3 };
enum { ORC_LIM_VANLEER = 0, ORC_LIM_MINMOD = 1, ORC_LIM_MC = 2 };
/* HLLC (named in Sec. 2.2) is read as HLL: on the advective system F = a U
 * every component moves with the one speed a, so there is no contact wave
 * between the HLL bounds S_L = min(a_L, a_R), S_R = max(a_L, a_R). */
enum { ORC_RIEMANN_LF = 0, ORC_RIEMANN_HLL = 1, ORC_RIEMANN_SWEPT = 2, ORC_RIEMANN_HLLC = 3 };

typedef struct {
    int n[3];             /* cells along x, y, z */
    double h;             /* cell size */
    double gamma;         /* adiabatic index */
    double rho_vac;       /* vacuum threshold */
    int bc[6];            /* faces -x,+x,-y,+y,-z,+z */
    double inflow[6][5];  /* primitive (rho,u,v,w,p) of INFLOW faces */
    int limiter;          /* ORC_LIM_* */
    int riemann;          /* ORC_RIEMANN_* */
} orc_cfg;

double orc_gtilde(double q);
double orc_norm_C(void);

int orc_step(const orc_cfg *c, const double *psi, const double *U, double dt, double *Uout,
             const int *box /* lo/hi per axis, or NULL for the whole grid */);
double orc_max_speed(const orc_cfg *c, const double *U);
double orc_dt(const orc_cfg *c, const double *U, double cfl);
int orc_run(const orc_cfg *c, const double *psi, double *U, long nsteps, double cfl, double t_end,
            double *t_io, long *steps_out);
void orc_totals(const orc_cfg *c, const double *psi, const double *U, double out[6]);
void orc_prim_to_cons(double gamma, const double *W, double *U, long N);
void orc_eos(const orc_cfg *c, const double *U, double *u, double *p, double *phi, int *vac);
int orc_force(const orc_cfg *c, const double *psi, const double *U, const double *xi, double dt,
              double *Q);
int orc_lagrange(const orc_cfg *c, const double *psi, const double *U, double dt, double *Us,
                 double *xis, double *Un, double *xin);

/* Exact Riemann solver of the 1D Euler equations (gamma law), including the
 * vacuum cases.  Star state of a non-vacuum problem: */
int orc_riemann_star(double gamma, double rl, double ul, double pl, double rr, double ur,
                     double pr, double *pstar, double *ustar);
/* Sampled solution at similarity coordinates s[i] = (x - x0)/t. */
int orc_riemann_sample(double gamma, double rl, double ul, double pl, double rr, double ur,
                       double pr, const double *s, long n, double *rho, double *u, double *p);

#ifdef __cplusplus
}
#endif
#endif
