// common.cuh -- layout, parameters and device helpers shared by the CUDA
// kernels of the CSPH-TVD step (arXiv 1912.04855, Sec. 2.2).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace cspht {

enum { BC_PERIODIC = 0, BC_OUTFLOW = 1, BC_INFLOW = 2, BC_WALL = 3 };
enum { LIM_VANLEER = 0, LIM_MINMOD = 1, LIM_MC = 2 };
enum { RIEMANN_LF = 0, RIEMANN_HLL = 1, RIEMANN_SWEPT = 2 };
enum { INJECT_NO_COPIES = 1 };
// device status bits
enum { ST_NONFINITE = 1, ST_NEGATIVE = 2, ST_CFL = 4, ST_TIMEOUT = 8 };

// Ghost depth of every padded array.  The stages use one layer (refilled
// after each stage); U^n carries a second layer so that TMA boxes with a
// two-cell halo see wrapped values on periodic axes.
constexpr int GH = 2;

// Padded structure-of-arrays layout.  Cell (i,j,k), i in [-GH, nx+GH), sits at
// ((k+GH)*py + (j+GH))*px + (i + ox); ox puts interior rows on a 32-byte
// boundary and px is a multiple of 32 bytes.
struct Grid {
    int n[3];
    int ox, px, py, pz;
    long long plane, total;
    __host__ __device__ __forceinline__ long long at(int i, int j, int k) const {
        return ((long long)(k + GH) * py + (j + GH)) * px + (i + ox);
    }
    __host__ __device__ __forceinline__ long long cells() const {
        return (long long)n[0] * n[1] * n[2];
    }
};

template <typename T>
inline Grid make_grid(int nx, int ny, int nz) {
    Grid g;
    g.n[0] = nx;
    g.n[1] = ny;
    g.n[2] = nz;
    int a = 32 / (int)sizeof(T);
    g.ox = a;
    g.px = ((g.ox + nx + GH + a - 1) / a) * a;
    g.py = ny + 2 * GH;
    g.pz = nz + 2 * GH;
    g.plane = (long long)g.px * g.py;
    g.total = g.plane * g.pz;
    return g;
}

// Physical and numerical parameters, passed by value to every kernel.
template <typename T>
struct Phys {
    T h, inv_h, gamma, gm1, inv_gm1, rho_vac;
    T inv_Ch2;     // 1 / (C h^2): weight G(r) = gt(r/h) / (C h^2)
    T w[4];        // static-lattice weight G(h|d|) = gt(|d|)/(C h^2) by |d|^2 = 1, 2, 3
    T gt[4];       // gt(|d|) by |d|^2 = 1, 2, 3 (cell units)
    int bc[6];
    T inW[6][5];   // inflow primitive (rho,u,v,w,p)
    T inU[6][5];   // inflow conserved
    T inPhi[6];    // inflow phi = sqrt(2p)
    int in_vac[6]; // inflow state is vacuum
    int limiter, riemann;
    int balance;   // CSPHT_BALANCE_*: compensated balance terms in FP32
};

// Per-handle control word in device memory.  k_dt writes dt at the start of a
// step; the Euler kernel accumulates the signal speed of the new state.
struct Ctrl {
    double t;      // simulated time of the state
    double t_end;  // clip target of cspht_run (+inf otherwise)
    double cfl;
    double dt;     // dt of the step in progress
    unsigned long long smax_cur;  // max signal speed of the state dt was taken from (bits)
    unsigned long long smax_next; // max signal speed of the state being produced (bits)
    long long steps;
    int status;
    int inject;      // test hook: bit 0 = the fused kernels post their copies' byte
                     // counts but issue no copy, so every copy wait runs out
    int spin_limit;  // polls a copy wait makes before it gives up (0 = MBAR_SPIN_LIMIT)
    int pad;
};

// M4 cubic spline weight gt(q) = -W'(q)/q (Eq. 7's kernel W, support 2h).
template <typename T>
__device__ __forceinline__ T gtilde(T q) {
    if (q < T(1)) return T(3) - T(2.25) * q;
    if (q < T(2)) {
        T a = T(2) - q;
        return T(0.75) * a * a / q;
    }
    return T(0);
}

// Primitive recovery (Sec. 2.1 EOS) with the vacuum threshold and p >= 0.
template <typename T>
struct Prim {
    T u[3], p, phi;
    bool vac;
};

template <typename T>
__device__ __forceinline__ Prim<T> eos(const Phys<T> &P, T rho, T mx, T my, T mz, T E) {
    Prim<T> r;
    if (!(rho > P.rho_vac)) {
        r.vac = true;
        r.u[0] = r.u[1] = r.u[2] = T(0);
        r.p = r.phi = T(0);
        return r;
    }
    r.vac = false;
    r.u[0] = mx / rho;
    r.u[1] = my / rho;
    r.u[2] = mz / rho;
    T kin = T(0.5) * (mx * r.u[0] + my * r.u[1] + mz * r.u[2]);
    T p = P.gm1 * (E - kin);
    if (p < T(0)) p = T(0);
    r.p = p;
    r.phi = sqrt(T(2) * p);
    return r;
}

// Signal speed max_d |u_d| + c of a gas cell (0 for vacuum); Delta t reduction.
template <typename T>
__device__ __forceinline__ double signal_speed(const Phys<T> &P, T rho, T mx, T my, T mz, T E) {
    Prim<T> q = eos(P, rho, mx, my, mz, E);
    if (q.vac) return 0.0;
    T um = fabs(q.u[0]);
    if (fabs(q.u[1]) > um) um = fabs(q.u[1]);
    if (fabs(q.u[2]) > um) um = fabs(q.u[2]);
    return (double)(um + sqrt(P.gamma * q.p / rho));
}

// TVD limiter of the one-sided slopes a = (U+ - U)/h, b = (U - U-)/h.
template <typename T>
__device__ __forceinline__ T limiter(int kind, T a, T b) {
    if (!(a * b > T(0))) return T(0);
    if (kind == LIM_MINMOD) return fabs(a) < fabs(b) ? a : b;
    if (kind == LIM_MC) {
        T m = fabs(T(2) * a);
        if (fabs(T(2) * b) < m) m = fabs(T(2) * b);
        if (fabs(T(0.5) * (a + b)) < m) m = fabs(T(0.5) * (a + b));
        return a > T(0) ? m : -m;
    }
    return T(2) * a * b / (a + b);
}

// Riemann flux of the advective system F = a U between the reconstructed
// states UL, UR with face speeds aL, aR.
template <typename T>
__device__ __forceinline__ T riemann_flux(int kind, T aL, T aR, T UL, T UR) {
    if (kind == RIEMANN_HLL) {
        T SL = aL < aR ? aL : aR, SR = aL < aR ? aR : aL;
        if (SL >= T(0)) return aL * UL;
        if (SR <= T(0)) return aR * UR;
        return (SR * aL * UL - SL * aR * UR + SL * SR * (UR - UL)) / (SR - SL);
    }
    if (kind == RIEMANN_SWEPT) {  // the face sweeps with the mean offset, carrying the upwind state
        const T a = T(0.5) * (aL + aR);
        return a >= T(0) ? a * UL : a * UR;
    }
    T s = fabs(aL) > fabs(aR) ? fabs(aL) : fabs(aR);
    return T(0.5) * (aL * UL + aR * UR) - T(0.5) * s * (UR - UL);
}

__device__ __forceinline__ void atomic_max_speed(unsigned long long *slot, double v) {
    // Non-negative doubles (and NaN, whose bits exceed +inf) order like their bits.
    atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}

__device__ __forceinline__ int wrap_idx(int a, int n) {
    a %= n;
    return a < 0 ? a + n : a;
}

}  // namespace cspht
