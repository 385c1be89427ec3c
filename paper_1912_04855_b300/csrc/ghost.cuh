// ghost.cuh -- one-layer ghost cells of each stage of the CSPH-TVD step.
//
// The boundary conditions are applied per stage (U^n, the predictor state,
// the corrector state), one axis at a time: x ghosts for interior (y,z), then
// y ghosts over x including its ghosts, then z ghosts over x and y including
// theirs.  A ghost out of range along several axes is therefore
// BC_z(BC_y(BC_x(...))).  Kinds: periodic (wrap), outflow (copy of the
// boundary cell b), inflow (fixed state, particle offset dt*u_in after the
// predictor), reflecting wall (normal velocity and offset mirrored, phi
// extrapolated hydrostatically from b and the next cell inward m:
// phi_g = phi_m + rho_b (psi_m - psi_g) / phi_b).
#pragma once

#include "common.cuh"

namespace cspht {

struct GhostSite {
    int g[3], b[3], m[3], src[3];  // ghost, boundary cell, next cell inward, periodic source
    int axis, side;
};

// Decomposes a thread index of the ghost pass along `a` into its site; the
// axes filled before `a` are covered including `depth` ghost layers.
__device__ __forceinline__ bool ghost_site(const Grid &G, int a, long long t, GhostSite &s,
                                           int depth = 1) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    int lob = b < a ? -depth : 0, lenb = G.n[b] + (b < a ? 2 * depth : 0);
    int loc = c < a ? -depth : 0, lenc = G.n[c] + (c < a ? 2 * depth : 0);
    long long lines = (long long)lenb * lenc;
    if (t >= 2 * lines) return false;
    int side = t >= lines ? 1 : 0;
    long long r = t - side * lines;
    int tb = (int)(r % lenb), tc = (int)(r / lenb);
    int n = G.n[a];
    s.g[b] = s.b[b] = s.m[b] = s.src[b] = lob + tb;
    s.g[c] = s.b[c] = s.m[c] = s.src[c] = loc + tc;
    s.g[a] = side ? n : -1;
    s.b[a] = side ? n - 1 : 0;
    s.m[a] = n > 1 ? (side ? n - 2 : 1) : s.b[a];
    s.src[a] = side ? 0 : n - 1;
    s.axis = a;
    s.side = side;
    return true;
}

inline long long ghost_pass_threads(const Grid &G, int a, int depth = 1) {
    int b = (a + 1) % 3, c = (a + 2) % 3;
    long long lenb = G.n[b] + (b < a ? 2 * depth : 0), lenc = G.n[c] + (c < a ? 2 * depth : 0);
    return 2 * lenb * lenc;
}

// Static potential: periodic wrap, otherwise linear extrapolation 2 psi_b - psi_m.
// Two layers, like U^n (the reflecting-wall rule of the second U^n layer on a
// periodic neighbour axis reads psi there); launch with depth 2.  The second
// layer continues the wrap or the extrapolation.
template <typename T>
__global__ void k_ghost_psi(Grid G, Phys<T> P, int a, T *__restrict__ psi) {
    GhostSite s;
    if (!ghost_site(G, a, blockIdx.x * (long long)blockDim.x + threadIdx.x, s, 2)) return;
    long long g = G.at(s.g[0], s.g[1], s.g[2]);
    int g2[3] = {s.g[0], s.g[1], s.g[2]};
    g2[a] += s.side ? 1 : -1;
    long long d2 = G.at(g2[0], g2[1], g2[2]);
    if (P.bc[2 * a + s.side] == BC_PERIODIC) {
        psi[g] = psi[G.at(s.src[0], s.src[1], s.src[2])];
        int w[3] = {g2[0], g2[1], g2[2]};
        w[a] = wrap_idx(w[a], G.n[a]);
        psi[d2] = psi[G.at(w[0], w[1], w[2])];
    } else {
        const T pb = psi[G.at(s.b[0], s.b[1], s.b[2])];
        psi[g] = T(2) * pb - psi[G.at(s.m[0], s.m[1], s.m[2])];
        psi[d2] = T(2) * psi[g] - pb;
    }
}

// Stage 0: conserved state U^n (5 fields).
template <typename T>
struct UPtr {
    T *f[5];
};

// Fills the first ghost layer by the face's rule and the second layer too:
// the wrapped cell on periodic faces, a copy of the first layer otherwise
// (no stage reads a non-periodic second layer).  Launch with depth 2.
template <typename T>
__device__ __forceinline__ void ghost_U_second(const Grid &G, int a, const GhostSite &s, int kind,
                                               UPtr<T> U) {
    int g2[3] = {s.g[0], s.g[1], s.g[2]};
    g2[a] += s.side ? 1 : -1;
    long long d2 = G.at(g2[0], g2[1], g2[2]);
    long long src;
    if (kind == BC_PERIODIC) {
        int w[3] = {g2[0], g2[1], g2[2]};
        w[a] = wrap_idx(w[a], G.n[a]);
        src = G.at(w[0], w[1], w[2]);
    } else {
        src = G.at(s.g[0], s.g[1], s.g[2]);
    }
    for (int f = 0; f < 5; ++f) U.f[f][d2] = U.f[f][src];
}

template <typename T>
__global__ void k_ghost_U(Grid G, Phys<T> P, int a, UPtr<T> U, const T *__restrict__ psi) {
    GhostSite s;
    if (!ghost_site(G, a, blockIdx.x * (long long)blockDim.x + threadIdx.x, s, 2)) return;
    long long g = G.at(s.g[0], s.g[1], s.g[2]);
    int face = 2 * a + s.side;
    int kind = P.bc[face];
    if (kind == BC_PERIODIC || kind == BC_OUTFLOW) {
        long long src = kind == BC_PERIODIC ? G.at(s.src[0], s.src[1], s.src[2])
                                            : G.at(s.b[0], s.b[1], s.b[2]);
        for (int f = 0; f < 5; ++f) U.f[f][g] = U.f[f][src];
        ghost_U_second(G, a, s, kind, U);
        return;
    }
    if (kind == BC_INFLOW) {
        for (int f = 0; f < 5; ++f) U.f[f][g] = P.inU[face][f];
        ghost_U_second(G, a, s, kind, U);
        return;
    }
    // reflecting wall
    long long b = G.at(s.b[0], s.b[1], s.b[2]), m = G.at(s.m[0], s.m[1], s.m[2]);
    T rb = U.f[0][b];
    Prim<T> qb = eos(P, rb, U.f[1][b], U.f[2][b], U.f[3][b], U.f[4][b]);
    Prim<T> qm = eos(P, U.f[0][m], U.f[1][m], U.f[2][m], U.f[3][m], U.f[4][m]);
    T u[3] = {qb.u[0], qb.u[1], qb.u[2]};
    u[a] = -u[a];
    if (qb.vac) {
        U.f[0][g] = rb;
        for (int e = 0; e < 3; ++e) U.f[1 + e][g] = e == a ? -U.f[1 + e][b] : U.f[1 + e][b];
        U.f[4][g] = U.f[4][b];
        ghost_U_second(G, a, s, kind, U);
        return;
    }
    T phig = T(0), rho_g = rb;
    if (qb.phi > T(0)) {
        phig = qm.phi + rb * (psi[m] - psi[g]) / qb.phi;
        if (phig < T(0)) phig = T(0);
        T ratio = phig / qb.phi;
        rho_g = rb * ratio * ratio;
    }
    T pg = T(0.5) * phig * phig;
    U.f[0][g] = rho_g;
    for (int e = 0; e < 3; ++e) U.f[1 + e][g] = rho_g * u[e];
    U.f[4][g] = pg / P.gm1 + T(0.5) * rho_g * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    ghost_U_second(G, a, s, kind, U);
}

// Stage 1 (after the predictor): particle density, velocity, phi, offset.
template <typename T>
struct S1Ptr {
    T *rho, *u[3], *phi, *xi[3];
};

template <typename T>
__global__ void k_ghost_S1(Grid G, Phys<T> P, int a, S1Ptr<T> S, const T *__restrict__ psi,
                           const Ctrl *__restrict__ ctrl) {
    GhostSite s;
    if (!ghost_site(G, a, blockIdx.x * (long long)blockDim.x + threadIdx.x, s)) return;
    long long g = G.at(s.g[0], s.g[1], s.g[2]);
    int face = 2 * a + s.side;
    int kind = P.bc[face];
    if (kind == BC_PERIODIC || kind == BC_OUTFLOW) {
        long long src = kind == BC_PERIODIC ? G.at(s.src[0], s.src[1], s.src[2])
                                            : G.at(s.b[0], s.b[1], s.b[2]);
        S.rho[g] = S.rho[src];
        S.phi[g] = S.phi[src];
        for (int e = 0; e < 3; ++e) {
            S.u[e][g] = S.u[e][src];
            S.xi[e][g] = S.xi[e][src];
        }
        return;
    }
    if (kind == BC_INFLOW) {
        T dt = (T)ctrl->dt;
        S.rho[g] = P.inW[face][0];
        S.phi[g] = P.inPhi[face];
        for (int e = 0; e < 3; ++e) {
            T ue = P.in_vac[face] ? T(0) : P.inW[face][1 + e];
            S.u[e][g] = ue;
            S.xi[e][g] = dt * ue;
        }
        return;
    }
    long long b = G.at(s.b[0], s.b[1], s.b[2]), m = G.at(s.m[0], s.m[1], s.m[2]);
    T rb = S.rho[b], phib = S.phi[b];
    for (int e = 0; e < 3; ++e) {
        S.u[e][g] = e == a ? -S.u[e][b] : S.u[e][b];
        S.xi[e][g] = e == a ? -S.xi[e][b] : S.xi[e][b];
    }
    T phig = T(0), rho_g = rb;
    if (rb > P.rho_vac && phib > T(0)) {
        phig = S.phi[m] + rb * (psi[m] - psi[g]) / phib;
        if (phig < T(0)) phig = T(0);
        T ratio = phig / phib;
        rho_g = rb * ratio * ratio;
    }
    S.rho[g] = rho_g;
    S.phi[g] = phig;
}

// Stage 2 (after the corrector): momentum and energy content and offset.
// Wall faces carry no flux, so their stage-2 ghosts are never read; they are
// filled with the mirrored values for completeness.
template <typename T>
struct S2Ptr {
    T *m[3], *E, *xi[3];
};

template <typename T>
__global__ void k_ghost_S2(Grid G, Phys<T> P, int a, S2Ptr<T> S, const Ctrl *__restrict__ ctrl) {
    GhostSite s;
    if (!ghost_site(G, a, blockIdx.x * (long long)blockDim.x + threadIdx.x, s)) return;
    long long g = G.at(s.g[0], s.g[1], s.g[2]);
    int face = 2 * a + s.side;
    int kind = P.bc[face];
    if (kind == BC_INFLOW) {
        T dt = (T)ctrl->dt;
        for (int e = 0; e < 3; ++e) {
            S.m[e][g] = P.inU[face][1 + e];
            S.xi[e][g] = P.in_vac[face] ? T(0) : dt * P.inW[face][1 + e];
        }
        S.E[g] = P.inU[face][4];
        return;
    }
    long long src = kind == BC_PERIODIC ? G.at(s.src[0], s.src[1], s.src[2])
                                        : G.at(s.b[0], s.b[1], s.b[2]);
    T sg = kind == BC_WALL ? T(-1) : T(1);
    for (int e = 0; e < 3; ++e) {
        S.m[e][g] = e == a ? sg * S.m[e][src] : S.m[e][src];
        S.xi[e][g] = e == a ? sg * S.xi[e][src] : S.xi[e][src];
    }
    S.E[g] = S.E[src];
}

}  // namespace cspht
