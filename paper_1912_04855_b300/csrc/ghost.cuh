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

// Values of the two ghost layers of U^n at site s (axis a): v1 for the first
// layer by the face's rule, v2 for the second -- the wrapped cell on periodic
// faces, a copy of the first layer otherwise (no stage reads a non-periodic
// second layer).  Reads interior cells and psi only.
template <typename T>
__device__ __forceinline__ void ghost_U_values(const Grid &G, const Phys<T> &P, int a, const GhostSite &s,
                                               UPtr<T> U, const T *__restrict__ psi, T v1[5], T v2[5]) {
    const int face = 2 * a + s.side;
    const int kind = P.bc[face];
    if (kind == BC_PERIODIC) {
        const long long src = G.at(s.src[0], s.src[1], s.src[2]);
        int w[3] = {s.g[0], s.g[1], s.g[2]};
        w[a] = wrap_idx(w[a] + (s.side ? 1 : -1), G.n[a]);
        const long long src2 = G.at(w[0], w[1], w[2]);
        for (int f = 0; f < 5; ++f) {
            v1[f] = U.f[f][src];
            v2[f] = U.f[f][src2];
        }
        return;
    }
    if (kind == BC_OUTFLOW) {
        const long long b = G.at(s.b[0], s.b[1], s.b[2]);
        for (int f = 0; f < 5; ++f) v1[f] = v2[f] = U.f[f][b];
        return;
    }
    if (kind == BC_INFLOW) {
        for (int f = 0; f < 5; ++f) v1[f] = v2[f] = P.inU[face][f];
        return;
    }
    // reflecting wall
    const long long g = G.at(s.g[0], s.g[1], s.g[2]);
    const long long b = G.at(s.b[0], s.b[1], s.b[2]), m = G.at(s.m[0], s.m[1], s.m[2]);
    const T rb = U.f[0][b];
    const Prim<T> qb = eos(P, rb, U.f[1][b], U.f[2][b], U.f[3][b], U.f[4][b]);
    const Prim<T> qm = eos(P, U.f[0][m], U.f[1][m], U.f[2][m], U.f[3][m], U.f[4][m]);
    if (qb.vac) {
        v1[0] = rb;
        for (int e = 0; e < 3; ++e) v1[1 + e] = e == a ? -U.f[1 + e][b] : U.f[1 + e][b];
        v1[4] = U.f[4][b];
    } else {
        T u[3] = {qb.u[0], qb.u[1], qb.u[2]};
        u[a] = -u[a];
        T phig = T(0), rho_g = rb;
        if (qb.phi > T(0)) {
            phig = qm.phi + rb * (psi[m] - psi[g]) / qb.phi;
            if (phig < T(0)) phig = T(0);
            const T ratio = phig / qb.phi;
            rho_g = rb * ratio * ratio;
        }
        const T pg = T(0.5) * phig * phig;
        v1[0] = rho_g;
        for (int e = 0; e < 3; ++e) v1[1 + e] = rho_g * u[e];
        v1[4] = pg / P.gm1 + T(0.5) * rho_g * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
    }
    for (int f = 0; f < 5; ++f) v2[f] = v1[f];
}

// One pass along axis a; launch with depth 2.
template <typename T>
__global__ void k_ghost_U(Grid G, Phys<T> P, int a, UPtr<T> U, const T *__restrict__ psi) {
    GhostSite s;
    if (!ghost_site(G, a, blockIdx.x * (long long)blockDim.x + threadIdx.x, s, 2)) return;
    T v1[5], v2[5];
    ghost_U_values(G, P, a, s, U, psi, v1, v2);
    int g2[3] = {s.g[0], s.g[1], s.g[2]};
    g2[a] += s.side ? 1 : -1;
    const long long g = G.at(s.g[0], s.g[1], s.g[2]), d2 = G.at(g2[0], g2[1], g2[2]);
    for (int f = 0; f < 5; ++f) {
        U.f[f][g] = v1[f];
        U.f[f][d2] = v2[f];
    }
}

// ---- the whole ghost shell in one pass, when the y and z faces are periodic
// or outflow.  Their rules are copies (a wrapped or the boundary cell), so an
// edge or corner ghost BC_z(BC_y(BC_x(.))) equals the x rule applied on the
// row its y and z map to, and every ghost depends on interior cells only: the
// three passes collapse into one launch with the same values.
__host__ __device__ __forceinline__ bool copy_faces_yz(const int bc[6]) {
    for (int f = 2; f < 6; ++f)
        if (bc[f] != BC_PERIODIC && bc[f] != BC_OUTFLOW) return false;
    return true;
}

// in-range source of coordinate c along an axis with copy-rule faces
__device__ __forceinline__ int copy_coord(int c, int n, int kind_lo, int kind_hi) {
    if (c < 0) return kind_lo == BC_PERIODIC ? wrap_idx(c, n) : 0;
    if (c >= n) return kind_hi == BC_PERIODIC ? wrap_idx(c, n) : n - 1;
    return c;
}

// Threads of the shell pass with `depth` layers: x faces over y, z including
// their ghosts, y faces over interior x and z including ghosts, z faces over
// interior x and y (the z faces are the last threads: zfaces = false leaves
// them out, for readers that wrap a periodic z instead of reading its ghosts).
inline long long shell_threads(const Grid &G, int depth, bool zfaces = true) {
    const long long ny = G.n[1], nz = G.n[2], nx = G.n[0];
    return 2 * (ny + 2 * depth) * (nz + 2 * depth) + 2 * nx * (nz + 2 * depth) + (zfaces ? 2 * nx * ny : 0);
}

// Decomposes thread t of the shell pass: the axis of the face, the side and
// the two other coordinates (the axis coordinate is the first ghost layer).
__device__ __forceinline__ bool shell_site(const Grid &G, int depth, long long t, int &a, int &side, int c[3]) {
    const long long nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const long long rx = 2 * (ny + 2 * depth) * (nz + 2 * depth), ry = 2 * nx * (nz + 2 * depth);
    if (t < rx) {
        a = 0;
        const long long per = (ny + 2 * depth) * (nz + 2 * depth);
        side = t >= per;
        t -= side * per;
        c[1] = (int)(t % (ny + 2 * depth)) - depth;
        c[2] = (int)(t / (ny + 2 * depth)) - depth;
    } else if ((t -= rx) < ry) {
        a = 1;
        const long long per = nx * (nz + 2 * depth);
        side = t >= per;
        t -= side * per;
        c[0] = (int)(t % nx);
        c[2] = (int)(t / nx) - depth;
    } else if ((t -= ry) < 2 * nx * ny) {
        a = 2;
        const long long per = nx * ny;
        side = t >= per;
        t -= side * per;
        c[0] = (int)(t % nx);
        c[1] = (int)(t / nx);
    } else {
        return false;
    }
    c[a] = side ? G.n[a] : -1;
    return true;
}

// The ghost site of axis a on the row that (c with its other coordinates
// mapped into range) lies on.
__device__ __forceinline__ GhostSite shell_ghost_site(const Grid &G, int a, int side, const int cm[3]) {
    GhostSite s;
    const int n = G.n[a];
    for (int d = 0; d < 3; ++d) s.g[d] = s.b[d] = s.m[d] = s.src[d] = cm[d];
    s.g[a] = side ? n : -1;
    s.b[a] = side ? n - 1 : 0;
    s.m[a] = n > 1 ? (side ? n - 2 : 1) : s.b[a];
    s.src[a] = side ? 0 : n - 1;
    s.axis = a;
    s.side = side;
    return s;
}

// An x-face ghost of the padded layout (make_grid: the row's first G.ox
// elements are one 32-byte sector of padding and ghosts): the sector of the
// row that holds the ghost layers, or nullptr when it also holds interior
// cells (the right face of a grid whose nx is not a multiple of G.ox).
// Writing the whole sector (the elements beyond the ghost layers are padding
// that no stage reads) lets the memory system take full sectors instead of
// merging partial ones.
template <typename T>
__device__ __forceinline__ T *x_ghost_sector(const Grid &G, T *field, int side, int y, int z) {
    static_assert(sizeof(T) * 4 == 16 || sizeof(T) * 2 == 16, "two 16-byte stores per sector");
    if (G.ox * (int)sizeof(T) != 32) return nullptr;
    if (side && (G.n[0] % G.ox != 0 || G.px < G.n[0] + 2 * G.ox)) return nullptr;
    T *p = field + G.at(side ? G.n[0] : -G.ox, y, z);
    return (reinterpret_cast<uintptr_t>(p) & 15u) ? nullptr : p;
}
// Fills a sector found by x_ghost_sector: inner is the first ghost layer's
// value, outer the second's (and the padding's).
template <typename T>
__device__ __forceinline__ void put_x_sector(T *p, int side, T inner, T outer) {
    constexpr int n = 32 / (int)sizeof(T);
    T v[n];
#pragma unroll
    for (int k = 0; k < n; ++k) v[k] = outer;
    v[side ? 0 : n - 1] = inner;
    if constexpr (sizeof(T) == 4) {
        reinterpret_cast<float4 *>(p)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4 *>(p)[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
        reinterpret_cast<double2 *>(p)[0] = make_double2(v[0], v[1]);
        reinterpret_cast<double2 *>(p)[1] = make_double2(v[2], v[3]);
    }
}

template <typename T>
__device__ __forceinline__ void ghost_U_shell_at(const Grid &G, const Phys<T> &P, const UPtr<T> &U,
                                                 const T *__restrict__ psi, long long t) {
    int a, side, c[3];
    if (!shell_site(G, 2, t, a, side, c)) return;
    int cm[3] = {c[0], c[1], c[2]};
    cm[1] = copy_coord(c[1], G.n[1], P.bc[2], P.bc[3]);
    cm[2] = copy_coord(c[2], G.n[2], P.bc[4], P.bc[5]);
    const GhostSite s = shell_ghost_site(G, a, side, cm);
    T v1[5], v2[5];
    ghost_U_values(G, P, a, s, U, psi, v1, v2);
    if (a == 0 && x_ghost_sector(G, U.f[0], side, c[1], c[2])) {
        for (int f = 0; f < 5; ++f)
            if (T *p = x_ghost_sector(G, U.f[f], side, c[1], c[2])) {
                put_x_sector(p, side, v1[f], v2[f]);
            } else {
                const long long g = G.at(c[0], c[1], c[2]);
                U.f[f][g] = v1[f];
                U.f[f][g + (side ? 1 : -1)] = v2[f];
            }
        return;
    }
    int g2[3] = {c[0], c[1], c[2]};
    g2[a] += side ? 1 : -1;
    const long long g = G.at(c[0], c[1], c[2]), d2 = G.at(g2[0], g2[1], g2[2]);
    for (int f = 0; f < 5; ++f) {
        U.f[f][g] = v1[f];
        U.f[f][d2] = v2[f];
    }
}

template <typename T>
__global__ void k_ghost_U_shell(Grid G, Phys<T> P, UPtr<T> U, const T *__restrict__ psi) {
    ghost_U_shell_at(G, P, U, psi, blockIdx.x * (long long)blockDim.x + threadIdx.x);
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

// Values (m[3], E, xi[3]) of the stage-2 ghost at site s (axis a).  axis_xi:
// of the offset only its component along a (the others are left 0 and not
// read; see ghost_S2_shell_at).
template <typename T>
__device__ __forceinline__ void ghost_S2_values(const Grid &G, const Phys<T> &P, int a, const GhostSite &s,
                                                S2Ptr<T> S, const Ctrl *__restrict__ ctrl, T v[7],
                                                bool axis_xi = false) {
    const int face = 2 * a + s.side;
    const int kind = P.bc[face];
    if (kind == BC_INFLOW) {
        const T dt = (T)ctrl->dt;
        for (int e = 0; e < 3; ++e) {
            v[e] = P.inU[face][1 + e];
            v[4 + e] = P.in_vac[face] ? T(0) : dt * P.inW[face][1 + e];
        }
        v[3] = P.inU[face][4];
        return;
    }
    const long long src = kind == BC_PERIODIC ? G.at(s.src[0], s.src[1], s.src[2])
                                              : G.at(s.b[0], s.b[1], s.b[2]);
    const T sg = kind == BC_WALL ? T(-1) : T(1);
    for (int e = 0; e < 3; ++e) {
        v[e] = e == a ? sg * S.m[e][src] : S.m[e][src];
        v[4 + e] = e == a ? sg * S.xi[e][src] : (axis_xi ? T(0) : S.xi[e][src]);
    }
    v[3] = S.E[src];
}

// Stores a stage-2 ghost; xi_axis >= 0: of the offset only that component.
template <typename T>
__device__ __forceinline__ void put_S2(S2Ptr<T> S, long long g, const T v[7], int xi_axis = -1) {
    for (int e = 0; e < 3; ++e) {
        S.m[e][g] = v[e];
        if (xi_axis < 0 || e == xi_axis) S.xi[e][g] = v[4 + e];
    }
    S.E[g] = v[3];
}

template <typename T>
__global__ void k_ghost_S2(Grid G, Phys<T> P, int a, S2Ptr<T> S, const Ctrl *__restrict__ ctrl) {
    GhostSite s;
    if (!ghost_site(G, a, blockIdx.x * (long long)blockDim.x + threadIdx.x, s)) return;
    T v[7];
    ghost_S2_values(G, P, a, s, S, ctrl, v);
    put_S2(S, G.at(s.g[0], s.g[1], s.g[2]), v);
}

// The stage-2 shell in one pass (y and z faces periodic or outflow; see
// k_ghost_U_shell).  axis_xi: on a face of axis a only m, E and the offset's
// component along a -- all that the fused Eulerian kernel reads of such a
// ghost (its x faces take xi_x, its y faces xi_y, its z faces xi_z, and its
// slopes m and E; the other components it reads at interior columns, rows
// and planes only) -- which leaves out 2 of the 7 fields' loads and stores.
template <typename T>
__device__ __forceinline__ void ghost_S2_shell_at(const Grid &G, const Phys<T> &P, const S2Ptr<T> &S,
                                                  const Ctrl *__restrict__ ctrl, long long t, bool axis_xi) {
    int a, side, c[3];
    if (!shell_site(G, 1, t, a, side, c)) return;
    int cm[3] = {c[0], c[1], c[2]};
    cm[1] = copy_coord(c[1], G.n[1], P.bc[2], P.bc[3]);
    cm[2] = copy_coord(c[2], G.n[2], P.bc[4], P.bc[5]);
    const GhostSite s = shell_ghost_site(G, a, side, cm);
    T v[7];
    ghost_S2_values(G, P, a, s, S, ctrl, v, axis_xi);
    if (a == 0) {  // x faces: whole sectors where the layout allows (x_ghost_sector)
        T *fld[7] = {S.m[0], S.m[1], S.m[2], S.E, S.xi[0], S.xi[1], S.xi[2]};
        const long long g = G.at(c[0], c[1], c[2]);
        for (int e = 0; e < (axis_xi ? 5 : 7); ++e) {
            if (T *p = x_ghost_sector(G, fld[e], side, c[1], c[2])) put_x_sector(p, side, v[e], v[e]);
            else fld[e][g] = v[e];
        }
        return;
    }
    put_S2(S, G.at(c[0], c[1], c[2]), v, axis_xi ? a : -1);
}

template <typename T>
__global__ void k_ghost_S2_shell(Grid G, Phys<T> P, S2Ptr<T> S, const Ctrl *__restrict__ ctrl, bool axis_xi) {
    ghost_S2_shell_at(G, P, S, ctrl, blockIdx.x * (long long)blockDim.x + threadIdx.x, axis_xi);
}

}  // namespace cspht
