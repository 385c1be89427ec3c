// opcount.cpp -- TEST AND MEASUREMENT INFRASTRUCTURE ONLY.
//
// Floating-point operation count of one CSPH-TVD step, taken from the oracle
// itself: this file compiles cspht_oracle.c unchanged with its `double`
// replaced by a type that counts the adds, subtracts, multiplies, divides and
// square roots it performs, then calls the oracle's own stage functions on a
// given state.  Nothing here computes any part of the step.
//
// Counting rule: an operation is counted when its result depends on the
// cell state (the conserved fields U and what the stages derive from them).
// Operations whose operands are all run constants -- h, gamma, the lattice
// normalisation C, the lattice geometry, the static potential psi -- or the
// step's scalar dt are folded: an implementation does them once per run or
// per step, not per cell.  (So the predictor's static-lattice weights and
// the gravity D0[psi] cost nothing per cell, while the corrector's weights
// at displaced positions are counted in full.)  Every value the method
// defines is counted once: the oracle computes every face flux twice (once
// from each neighbouring cell) and every slope twice (once per face that
// reads it), and those repeats are removed by counting the pieces apart.
// Negation, absolute value and comparisons are not counted.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

namespace opc {
unsigned long long n_add = 0, n_mul = 0, n_div = 0, n_sqrt = 0;
}

// A double with a flag that says whether it depends on the cell state.
struct ocd {
    double v;
    bool var;
    ocd() = default;
    ocd(double x) : v(x), var(false) {}
    ocd(double x, bool dep) : v(x), var(dep) {}
    ocd &operator+=(ocd b);
    ocd &operator-=(ocd b);
    ocd &operator*=(ocd b);
    ocd &operator/=(ocd b);
    ocd operator-() const { return ocd(-v, var); }
};
static inline ocd counted(double r, bool dep, unsigned long long &n) {
    if (dep) ++n;
    return ocd(r, dep);
}
static inline ocd operator+(ocd a, ocd b) { return counted(a.v + b.v, a.var || b.var, opc::n_add); }
static inline ocd operator-(ocd a, ocd b) { return counted(a.v - b.v, a.var || b.var, opc::n_add); }
static inline ocd operator*(ocd a, ocd b) { return counted(a.v * b.v, a.var || b.var, opc::n_mul); }
static inline ocd operator/(ocd a, ocd b) { return counted(a.v / b.v, a.var || b.var, opc::n_div); }
inline ocd &ocd::operator+=(ocd b) { return *this = *this + b; }
inline ocd &ocd::operator-=(ocd b) { return *this = *this - b; }
inline ocd &ocd::operator*=(ocd b) { return *this = *this * b; }
inline ocd &ocd::operator/=(ocd b) { return *this = *this / b; }
static inline bool operator<(ocd a, ocd b) { return a.v < b.v; }
static inline bool operator>(ocd a, ocd b) { return a.v > b.v; }
static inline bool operator<=(ocd a, ocd b) { return a.v <= b.v; }
static inline bool operator>=(ocd a, ocd b) { return a.v >= b.v; }
static inline bool operator==(ocd a, ocd b) { return a.v == b.v; }
static inline bool operator!=(ocd a, ocd b) { return a.v != b.v; }
static inline ocd sqrt(ocd a) { return counted(::sqrt(a.v), a.var, opc::n_sqrt); }
static inline ocd fabs(ocd a) { return ocd(::fabs(a.v), a.var); }
static inline bool isfinite(ocd a) { return ::isfinite(a.v) != 0; }

#define double ocd
#include "cspht_oracle.c"
#undef double

namespace {

// The oracle's configuration with plain doubles (the layout of orc_cfg).
struct cfg_in {
    int n[3];
    double h, gamma, rho_vac;
    int bc[6];
    double inflow[6][5];
    int limiter, riemann;
};

struct Counts {
    unsigned long long add, mul, div, sqrt_;
    unsigned long long flops() const { return add + mul + div + sqrt_; }
};

Counts snap() { return Counts{opc::n_add, opc::n_mul, opc::n_div, opc::n_sqrt}; }
Counts operator-(Counts a, Counts b) {
    return Counts{a.add - b.add, a.mul - b.mul, a.div - b.div, a.sqrt_ - b.sqrt_};
}
Counts operator+(Counts a, Counts b) {
    return Counts{a.add + b.add, a.mul + b.mul, a.div + b.div, a.sqrt_ + b.sqrt_};
}

void put(FILE *f, const char *name, Counts c, double N, bool comma = true) {
    fprintf(f, "  \"%s\": {\"flops\": %.4f, \"add\": %.4f, \"mul\": %.4f, \"div\": %.4f, \"sqrt\": %.4f}%s\n",
            name, c.flops() / N, c.add / N, c.mul / N, c.div / N, c.sqrt_ / N, comma ? "," : "");
}

}  // namespace

// Counts the operations of one step of the given state with time step dt and
// writes per-cell counts as JSON to `out_path`.  Returns 0 on success.
extern "C" int orc_opcount(const cfg_in *ci, const double *psi_in, const double *U_in, double dt_in,
                           const char *out_path) {
    orc_cfg c;
    memset(&c, 0, sizeof c);
    for (int d = 0; d < 3; ++d) c.n[d] = ci->n[d];
    c.h = ci->h;
    c.gamma = ci->gamma;
    c.rho_vac = ci->rho_vac;
    for (int f = 0; f < 6; ++f) {
        c.bc[f] = ci->bc[f];
        for (int k = 0; k < 5; ++k) c.inflow[f][k] = ci->inflow[f][k];
    }
    c.limiter = ci->limiter;
    c.riemann = ci->riemann;
    if (!cfg_ok(&c)) return -1;
    const size_t N = (size_t)c.n[0] * c.n[1] * c.n[2];
    ocd *psi = (ocd *)malloc(sizeof(ocd) * N), *U = (ocd *)malloc(sizeof(ocd) * 5 * N),
        *Uo = (ocd *)malloc(sizeof(ocd) * 5 * N);
    if (!psi || !U || !Uo) return -2;
    // the state is what the counted operations depend on; psi and dt are
    // a run constant and a per-step scalar
    for (size_t g = 0; g < N; ++g) psi[g] = ocd(psi_in[g], false);
    for (size_t g = 0; g < 5 * N; ++g) U[g] = ocd(U_in[g], true);
    const ocd dt = ocd(dt_in, false);

    // the whole step as the oracle runs it
    Counts t0 = snap();
    if (orc_step(&c, psi, U, dt, Uo, NULL) != ORC_OK) return -3;
    const Counts all = snap() - t0;

    // its stages, on the same stage boxes orc_step builds for the whole grid
    Ctx x;
    ctx_init(&x, &c, psi, U, dt);
    int lo[3] = {0, 0, 0}, hi[3] = {c.n[0], c.n[1], c.n[2]};
    if (build_stage(&x, 0, lo, hi, 3) || build_stage(&x, 1, lo, hi, 2) || build_stage(&x, 2, lo, hi, 1))
        return -2;
    t0 = snap();
    run_primitives(&x);
    const Counts prim = snap() - t0;
    t0 = snap();
    run_predictor(&x);
    const Counts pred = snap() - t0;
    t0 = snap();
    run_corrector(&x);
    const Counts corr = snap() - t0;

    // the static gravity D0[psi] (folded: psi is a run constant; kept as a
    // check that it costs nothing per cell)
    t0 = snap();
    for (int k = 0; k < c.n[2]; ++k)
        for (int j = 0; j < c.n[1]; ++j)
            for (int i = 0; i < c.n[0]; ++i) {
                ocd D0[3];
                lattice_gravity(&x, i, j, k, D0);
            }
    const Counts grav = snap() - t0;

    // the Euler stage as orc_step does it: two face fluxes per cell and axis
    t0 = snap();
    for (int k = 0; k < c.n[2]; ++k)
        for (int j = 0; j < c.n[1]; ++j)
            for (int i = 0; i < c.n[0]; ++i)
                for (int d = 0; d < 3; ++d) {
                    int cc[3] = {i, j, k}, Lm[3] = {i, j, k};
                    Lm[d] -= 1;
                    ocd F[5];
                    face_flux(&x, d, cc, F);
                    face_flux(&x, d, Lm, F);
                }
    const Counts faces_twice = snap() - t0;
    // each distinct face once (the upper face of every cell, plus the lower
    // face of the first cell along a non-periodic axis), and the slopes those
    // calls evaluate inside
    Counts faces_once{0, 0, 0, 0}, slopes_in_faces{0, 0, 0, 0};
    for (int k = 0; k < c.n[2]; ++k)
        for (int j = 0; j < c.n[1]; ++j)
            for (int i = 0; i < c.n[0]; ++i)
                for (int d = 0; d < 3; ++d) {
                    const int cc[3] = {i, j, k};
                    const bool first = cc[d] == 0 && c.bc[2 * d] != ORC_BC_PERIODIC;
                    for (int lower = 0; lower <= (first ? 1 : 0); ++lower) {
                        int L[3] = {i, j, k};
                        L[d] -= lower;
                        int R[3] = {L[0], L[1], L[2]};
                        R[d] += 1;
                        ocd F[5], th[5];
                        t0 = snap();
                        face_flux(&x, d, L, F);
                        faces_once = faces_once + (snap() - t0);
                        // a wall face returns before reading any slope
                        const bool wall = (L[d] == -1 && c.bc[2 * d] == ORC_BC_WALL) ||
                                          (R[d] == c.n[d] && c.bc[2 * d + 1] == ORC_BC_WALL);
                        if (!wall) {
                            t0 = snap();
                            slope(&x, d, L, th);
                            slope(&x, d, R, th);
                            slopes_in_faces = slopes_in_faces + (snap() - t0);
                        }
                    }
                }
    // each distinct slope once: every cell and axis
    t0 = snap();
    for (int k = 0; k < c.n[2]; ++k)
        for (int j = 0; j < c.n[1]; ++j)
            for (int i = 0; i < c.n[0]; ++i)
                for (int d = 0; d < 3; ++d) {
                    const int cc[3] = {i, j, k};
                    ocd th[5];
                    slope(&x, d, cc, th);
                }
    const Counts slopes_once = snap() - t0;

    // the signal speed of every cell (the next step's dt) and dt itself
    t0 = snap();
    ocd smax = orc_max_speed(&c, U);
    (void)(c.h * ocd(0.4) / smax);
    const Counts speed = snap() - t0;
    for (int s = 0; s < 3; ++s) free_stage(&x.st[s]);

    const Counts euler_oracle = all - prim - pred - corr;
    const Counts update = euler_oracle - faces_twice;
    const Counts flux = faces_once - slopes_in_faces;  // Eq. 8 states and the Riemann flux
    const Counts euler = flux + slopes_once + update;
    const Counts lag = prim + pred + corr;

    FILE *f = fopen(out_path, "w");
    if (!f) return -4;
    const double n = (double)N;
    fprintf(f, "{\n  \"cells\": %zu,\n", N);
    put(f, "oracle_step_as_written", all, n);
    put(f, "primitives", prim, n);
    put(f, "predictor_incl_gravity", pred, n);
    put(f, "corrector_incl_gravity", corr, n);
    put(f, "static_gravity", grav, n);
    put(f, "euler_as_written", euler_oracle, n);
    put(f, "euler_faces", flux, n);
    put(f, "euler_slopes", slopes_once, n);
    put(f, "euler_update", update, n);
    put(f, "signal_speed_and_dt", speed, n);
    put(f, "lagrange_kernel", lag, n);
    put(f, "euler_kernel", euler + speed, n);
    put(f, "step", lag + euler + speed, n, false);
    fprintf(f, "}\n");
    fclose(f);
    free(psi);
    free(U);
    free(Uo);
    return 0;
}
