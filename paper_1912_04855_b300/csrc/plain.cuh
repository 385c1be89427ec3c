// plain.cuh -- the CSPH-TVD step as one kernel per paper kernel (Sec. 3):
// HFC (force Q of Eq. 7), SUL (updates of Eqs. 5-6), FGC (face fluxes of
// Eq. 8 and the Riemann flux), SUE (Eq. 4), each stage reading and writing
// global arrays, with the ghost layers refilled between stages.  This path
// is the straightforward GPU form of the method and the baseline the fused
// path is measured against.
#pragma once

#include "common.cuh"
#include "ghost.cuh"

namespace cspht {

struct Cell {
    int i, j, k;
};

// Interior cell of a (x, y, z) launch; false for the ragged tail.
__device__ __forceinline__ bool interior_cell(const Grid &G, Cell &c) {
    c.i = blockIdx.x * blockDim.x + threadIdx.x;
    c.j = blockIdx.y * blockDim.y + threadIdx.y;
    c.k = blockIdx.z;
    return c.i < G.n[0] && c.j < G.n[1];
}

// Primitive recovery of U^n on the whole padded box (ghosts included).
template <typename T>
__global__ void k_prim(Grid G, Phys<T> P, UPtr<T> U, T *__restrict__ ux, T *__restrict__ uy,
                       T *__restrict__ uz, T *__restrict__ phi) {
    int i = blockIdx.x * blockDim.x + threadIdx.x - 1;  // one ghost layer
    int j = blockIdx.y * blockDim.y + threadIdx.y - 1;
    int k = blockIdx.z - 1;
    if (i > G.n[0] || j > G.n[1]) return;
    long long c = G.at(i, j, k);
    Prim<T> q = eos(P, U.f[0][c], U.f[1][c], U.f[2][c], U.f[3][c], U.f[4][c]);
    ux[c] = q.u[0];
    uy[c] = q.u[1];
    uz[c] = q.u[2];
    phi[c] = q.phi;
}

// HFC: Q_i of Eq. 7 -- pressure phi_i sum_j phi_j G_ij r_ij, pressure work
// phi_i sum_j phi_j G_ij r_ij.(u_i+u_j)/2, gravity -rho_i D0_i[psi] and
// -rho_i u_i.D0_i[psi] on the static lattice.  DISP: particles displaced by
// xi (corrector); otherwise at the cell centres (predictor).
template <typename T, bool DISP>
__global__ void k_hfc(Grid G, Phys<T> P, const T *__restrict__ rho, const T *__restrict__ ux,
                      const T *__restrict__ uy, const T *__restrict__ uz, const T *__restrict__ phi,
                      const T *__restrict__ xx, const T *__restrict__ xy, const T *__restrict__ xz,
                      const T *__restrict__ psi, T *__restrict__ Q0, T *__restrict__ Q1,
                      T *__restrict__ Q2, T *__restrict__ Q3) {
    Cell cc;
    if (!interior_cell(G, cc)) return;
    long long c = G.at(cc.i, cc.j, cc.k);
    T rhoi = rho[c];
    if (!(rhoi > P.rho_vac)) {
        Q0[c] = Q1[c] = Q2[c] = Q3[c] = T(0);
        return;
    }
    T ui[3] = {ux[c], uy[c], uz[c]}, phii = phi[c];
    T xii[3] = {T(0), T(0), T(0)};
    if (DISP) {
        xii[0] = xx[c];
        xii[1] = xy[c];
        xii[2] = xz[c];
    }
    T Pp[3] = {T(0), T(0), T(0)}, Wk = T(0), D0[3] = {T(0), T(0), T(0)};
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy && !dz) continue;
                long long cj = c + dz * G.plane + dy * (long long)G.px + dx;
                int d[3] = {dx, dy, dz};
                T r[3];
                T Gw;
                int d2 = dx * dx + dy * dy + dz * dz;
                if (DISP) {
                    T xj[3] = {xx[cj], xy[cj], xz[cj]};
                    T r2 = T(0);
                    for (int e = 0; e < 3; ++e) {
                        r[e] = P.h * d[e] + (xj[e] - xii[e]);
                        r2 += r[e] * r[e];
                    }
                    Gw = gtilde<T>(sqrt(r2) / P.h) * P.inv_Ch2;
                } else {
                    for (int e = 0; e < 3; ++e) r[e] = P.h * d[e];
                    Gw = P.w[d2];
                }
                T phj = phi[cj];
                T uj[3] = {ux[cj], uy[cj], uz[cj]};
                T ru = T(0);
                for (int e = 0; e < 3; ++e) {
                    Pp[e] += Gw * r[e] * phj;
                    ru += r[e] * (T(0.5) * (ui[e] + uj[e]));
                }
                Wk += Gw * ru * phj;
                T G0 = P.w[d2];
                T ps = psi[cj];
                for (int e = 0; e < 3; ++e) D0[e] += G0 * (P.h * d[e]) * ps;
            }
    Q0[c] = -phii * Pp[0] - rhoi * D0[0];
    Q1[c] = -phii * Pp[1] - rhoi * D0[1];
    Q2[c] = -phii * Pp[2] - rhoi * D0[2];
    Q3[c] = -phii * Wk - rhoi * (ui[0] * D0[0] + ui[1] * D0[1] + ui[2] * D0[2]);
}

// SUL, predictor (Eq. 5): U* = U^n + dt Q (density unchanged), u* = m*/rho,
// xi* = dt (u^n + u*)/2.
template <typename T>
__global__ void k_sul_pred(Grid G, Phys<T> P, const Ctrl *__restrict__ ctrl, UPtr<T> U,
                           const T *__restrict__ Q0, const T *__restrict__ Q1,
                           const T *__restrict__ Q2, const T *__restrict__ Q3,
                           const T *__restrict__ u0x, const T *__restrict__ u0y,
                           const T *__restrict__ u0z, UPtr<T> Us, S1Ptr<T> S1) {
    Cell cc;
    if (!interior_cell(G, cc)) return;
    long long c = G.at(cc.i, cc.j, cc.k);
    T dt = (T)ctrl->dt;
    T rho = U.f[0][c];
    T m[3] = {U.f[1][c] + dt * Q0[c], U.f[2][c] + dt * Q1[c], U.f[3][c] + dt * Q2[c]};
    T E = U.f[4][c] + dt * Q3[c];
    Prim<T> q = eos(P, rho, m[0], m[1], m[2], E);
    T u0[3] = {u0x[c], u0y[c], u0z[c]};
    for (int e = 0; e < 3; ++e) {
        Us.f[1 + e][c] = m[e];
        S1.u[e][c] = q.u[e];
        S1.xi[e][c] = T(0) + dt * T(0.5) * (u0[e] + q.u[e]);
    }
    Us.f[4][c] = E;
    S1.rho[c] = rho;
    S1.phi[c] = q.phi;
}

// SUL, corrector (Eq. 6): U~ = (U^n + U*)/2 + dt/2 Q*, u~ = m~/rho,
// xi^{n+1} = xi*/2 + dt/2 (u^n + u~)/2.  A particle that moved more than h
// along an axis raises ST_CFL.
template <typename T>
__global__ void k_sul_corr(Grid G, Phys<T> P, Ctrl *__restrict__ ctrl, UPtr<T> U, UPtr<T> Us,
                           const T *__restrict__ Q0, const T *__restrict__ Q1,
                           const T *__restrict__ Q2, const T *__restrict__ Q3,
                           const T *__restrict__ u0x, const T *__restrict__ u0y,
                           const T *__restrict__ u0z, S1Ptr<T> S1, S2Ptr<T> S2) {
    Cell cc;
    if (!interior_cell(G, cc)) return;
    long long c = G.at(cc.i, cc.j, cc.k);
    T dt = (T)ctrl->dt;
    T rho = U.f[0][c];
    T Q[4] = {Q0[c], Q1[c], Q2[c], Q3[c]};
    T m[3], E;
    for (int e = 0; e < 3; ++e)
        m[e] = T(0.5) * (U.f[1 + e][c] + Us.f[1 + e][c]) + T(0.5) * dt * Q[e];
    E = T(0.5) * (U.f[4][c] + Us.f[4][c]) + T(0.5) * dt * Q[3];
    Prim<T> q = eos(P, T(0.5) * (rho + rho), m[0], m[1], m[2], E);
    T u0[3] = {u0x[c], u0y[c], u0z[c]};
    bool far = false;
    for (int e = 0; e < 3; ++e) {
        T xi = T(0.5) * (T(0) + S1.xi[e][c]) + T(0.5) * dt * (T(0.5) * (u0[e] + q.u[e]));
        S2.m[e][c] = m[e];
        S2.xi[e][c] = xi;
        far |= !(fabs(xi) <= P.h);
    }
    S2.E[c] = E;
    if (far) atomicOr(&ctrl->status, ST_CFL);
}

// Slope Theta^n_d of field f at cell (i,j,k) that may be a ghost along d only:
// periodic ghosts take the wrapped cell's slope, other ghosts have slope 0.
template <typename T>
__device__ __forceinline__ T slope_at(const Grid &G, const Phys<T> &P, const T *__restrict__ f, int d,
                                      int i, int j, int k) {
    int id[3] = {i, j, k};
    if (id[d] < 0 || id[d] >= G.n[d]) {
        if (P.bc[2 * d + (id[d] < 0 ? 0 : 1)] != BC_PERIODIC) return T(0);
        id[d] = wrap_idx(id[d], G.n[d]);
    }
    long long c = G.at(id[0], id[1], id[2]);
    long long s = d == 0 ? 1 : (d == 1 ? (long long)G.px : G.plane);
    T um = f[c - s], u0 = f[c], up = f[c + s];
    return limiter<T>(P.limiter, (up - u0) / P.h, (u0 - um) / P.h);
}

// FGC: flux through the face between L = (i,j,k) and R = L + e_d at
// t_{n+1/2}; Eq. 8 with U^{n+1/2} = (U^n + U~)/2, face speeds a = xi/dt.
// L runs over [-1, n_d - 1] along d.  Stored at L's padded index.
template <typename T>
__global__ void k_fgc(Grid G, Phys<T> P, const Ctrl *__restrict__ ctrl, int d, UPtr<T> U,
                      S2Ptr<T> S2, UPtr<T> F) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    int j = blockIdx.y * blockDim.y + threadIdx.y;
    int k = blockIdx.z;
    int id[3] = {i, j, k};
    id[d] -= 1;  // launch covers n_d + 1 faces along d
    int lim[3] = {G.n[0], G.n[1], G.n[2]};
    if (id[0] >= lim[0] || id[1] >= lim[1] || id[2] >= lim[2]) return;
    long long cL = G.at(id[0], id[1], id[2]);
    long long s = d == 0 ? 1 : (d == 1 ? (long long)G.px : G.plane);
    long long cR = cL + s;
    if ((id[d] == -1 && P.bc[2 * d] == BC_WALL) ||
        (id[d] + 1 == G.n[d] && P.bc[2 * d + 1] == BC_WALL)) {
        for (int f = 0; f < 5; ++f) F.f[f][cL] = T(0);
        return;
    }
    T dt = (T)ctrl->dt, h = P.h;
    T xL = S2.xi[d][cL], xR = S2.xi[d][cR];
    T aL = xL / dt, aR = xR / dt;
    int rid[3] = {id[0], id[1], id[2]};
    rid[d] += 1;
    for (int f = 0; f < 5; ++f) {
        T thL = slope_at(G, P, U.f[f], d, id[0], id[1], id[2]);
        T thR = slope_at(G, P, U.f[f], d, rid[0], rid[1], rid[2]);
        T tL = f == 0 ? U.f[0][cL] : (f == 4 ? S2.E[cL] : S2.m[f - 1][cL]);
        T tR = f == 0 ? U.f[0][cR] : (f == 4 ? S2.E[cR] : S2.m[f - 1][cR]);
        T UL = T(0.5) * (U.f[f][cL] + tL) + T(0.5) * (h - xL) * thL;
        T UR = T(0.5) * (U.f[f][cR] + tR) - T(0.5) * (h + xR) * thR;
        F.f[f][cL] = riemann_flux<T>(P.riemann, aL, aR, UL, UR);
    }
}

// Block-wide max of a double, then one atomic per block.
__device__ __forceinline__ void block_max_to(unsigned long long *slot, double v) {
    __shared__ double red[32];
    for (int o = 16; o > 0; o >>= 1) {
        double w = __shfl_xor_sync(0xffffffffu, v, o);
        v = (w > v || w != w) ? w : v;
    }
    int lane = (threadIdx.x + threadIdx.y * blockDim.x) & 31;
    int warp = (threadIdx.x + threadIdx.y * blockDim.x) >> 5;
    int nw = (blockDim.x * blockDim.y + 31) >> 5;
    if (lane == 0) red[warp] = v;
    __syncthreads();
    if (warp == 0) {
        v = lane < nw ? red[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) {
            double w = __shfl_xor_sync(0xffffffffu, v, o);
            v = (w > v || w != w) ? w : v;
        }
        if (lane == 0) atomic_max_speed(slot, v);
    }
}

// SUE (Eq. 4): U^{n+1} = U~ - dt/h sum_d (F_{+} - F_{-}).  Epilogue: signal
// speed of U^{n+1} for the next dt, and the status checks.  dt == 0 copies.
template <typename T>
__global__ void k_sue(Grid G, Phys<T> P, Ctrl *__restrict__ ctrl, UPtr<T> U, S2Ptr<T> S2,
                      UPtr<T> Fx, UPtr<T> Fy, UPtr<T> Fz, UPtr<T> Un) {
    Cell cc;
    bool in = interior_cell(G, cc);
    double sp = 0.0;
    if (in) {
        long long c = G.at(cc.i, cc.j, cc.k);
        T dt = (T)ctrl->dt;
        T v[5];
        if (dt > T(0)) {
            T base[5] = {U.f[0][c], S2.m[0][c], S2.m[1][c], S2.m[2][c], S2.E[c]};
            for (int f = 0; f < 5; ++f) {
                T div = T(0);
                div += Fx.f[f][c] - Fx.f[f][c - 1];
                div += Fy.f[f][c] - Fy.f[f][c - G.px];
                div += Fz.f[f][c] - Fz.f[f][c - G.plane];
                v[f] = base[f] - dt / P.h * div;
            }
        } else {
            for (int f = 0; f < 5; ++f) v[f] = U.f[f][c];
        }
        int st = 0;
        for (int f = 0; f < 5; ++f) {
            Un.f[f][c] = v[f];
            if (!isfinite((double)v[f])) st |= ST_NONFINITE;
        }
        if (v[0] < T(0)) st |= ST_NEGATIVE;
        if (st) atomicOr(&ctrl->status, st);
        sp = signal_speed(P, v[0], v[1], v[2], v[3], v[4]);
    }
    block_max_to(&ctrl->smax_next, sp);
}

}  // namespace cspht
