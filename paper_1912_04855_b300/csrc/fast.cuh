// fast.cuh -- the CSPH-TVD step in two fused kernels.
//
//  k_lagrange: the whole Lagrangian stage (Eqs. 5-7): primitive recovery,
//    HFC + SUL predictor, the predictor-stage boundary layer, HFC + SUL
//    corrector.  A CTA owns a TX x TY column of cells and marches up a chunk
//    of z planes.  Two shared-memory rings of three planes hold the
//    primitives of U^n (tile + 2 halo) and the predictor particles (tile + 1
//    halo); only U^n and the precomputed lattice gravity are read from HBM,
//    only the corrector's content and offsets (m~, E~, xi) are written.
//  k_euler: the Eulerian stage (Eq. 8 reconstruction, Riemann flux, Eq. 4
//    update) for one cell per thread, plus the signal-speed reduction for the
//    next dt and the status checks.
#pragma once

#include "common.cuh"
#include "ghost.cuh"
#include "plain.cuh"

namespace cspht {

// Static lattice gravity D0_i[psi] = sum_j G(h|d|) h d psi_j (Eq. 7's f = -D0[psi]),
// computed once per handle: psi does not change.
template <typename T>
__global__ void k_gravity(Grid G, Phys<T> P, const T *__restrict__ psi, T *__restrict__ gx,
                          T *__restrict__ gy, T *__restrict__ gz) {
    Cell cc;
    if (!interior_cell(G, cc)) return;
    long long c = G.at(cc.i, cc.j, cc.k);
    T D0[3] = {T(0), T(0), T(0)};
    for (int dz = -1; dz <= 1; ++dz)
        for (int dy = -1; dy <= 1; ++dy)
            for (int dx = -1; dx <= 1; ++dx) {
                if (!dx && !dy && !dz) continue;
                int d[3] = {dx, dy, dz};
                T G0 = P.w[dx * dx + dy * dy + dz * dz];
                T ps = psi[c + dz * G.plane + dy * (long long)G.px + dx];
                for (int e = 0; e < 3; ++e) D0[e] += G0 * (P.h * d[e]) * ps;
            }
    gx[c] = D0[0];
    gy[c] = D0[1];
    gz[c] = D0[2];
}

template <typename T>
struct LagArgs {
    Grid G;
    Phys<T> P;
    const T *U[5];
    const T *psi;
    const T *grav[3];
    T *m[3];
    T *E;
    T *xi[3];
    Ctrl *ctrl;
    int zchunk;
};

// Coordinate of a tile position in the padded arrays: wrapped on periodic
// axes, clamped into the one-cell ghost layer otherwise (positions further
// out only feed values that the boundary fill overwrites).
__device__ __forceinline__ int map_coord(int a, int n, bool per) {
    if (per) return wrap_idx(a, n);
    return a < -1 ? -1 : (a > n ? n : a);
}

__device__ __forceinline__ int mod3(int a) { return ((a % 3) + 3) % 3; }

template <int TX, int TY>
struct LagShape {
    static constexpr int IX = TX + 4, IY = TY + 4, NI = IX * IY;  // U^n primitives
    static constexpr int PX = TX + 2, PY = TY + 2, NP = PX * PY;  // predictor particles
    static constexpr int NT = TX * TY;
    static constexpr int NIN = 5;  // rho, u, v, w, phi
    static constexpr int NPR = 8;  // rho, u, v, w, phi, xi_x, xi_y, xi_z
    template <typename T>
    static constexpr size_t smem_bytes() {
        return sizeof(T) * (3 * NIN * NI + 3 * NPR * NP);
    }
};

template <typename T, int TX, int TY>
__global__ void __launch_bounds__(TX *TY) k_lagrange(LagArgs<T> A) {
    using S = LagShape<TX, TY>;
    constexpr int IX = S::IX, NI = S::NI, PX = S::PX, PY = S::PY, NP = S::NP, NT = S::NT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sin = reinterpret_cast<T *>(smem_raw);  // [3][NIN][NI]
    T *spr = sin + 3 * S::NIN * NI;             // [3][NPR][NP]

    const Grid &G = A.G;
    const Phys<T> &P = A.P;
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const bool perx = P.bc[0] == BC_PERIODIC, pery = P.bc[2] == BC_PERIODIC,
               perz = P.bc[4] == BC_PERIODIC;
    const int tid = threadIdx.x;
    const int x0 = blockIdx.x * TX, y0 = blockIdx.y * TY;
    const int z0 = blockIdx.z * A.zchunk;
    const int z1 = min(z0 + A.zchunk, nz);
    const T dt = (T)A.ctrl->dt;
    if (!(dt > T(0))) return;  // a zero step: the Euler kernel copies U^n
    const T h = P.h, half_dt = T(0.5) * dt;

    auto IN = [&](int slot, int f, int t) -> T & { return sin[(slot * S::NIN + f) * NI + t]; };
    auto PR = [&](int slot, int f, int t) -> T & { return spr[(slot * S::NPR + f) * NP + t]; };

    // ---- U^n plane gz -> primitives in the input ring
    auto load_in = [&](int gz) {
        int slot = mod3(gz);
        int zz = map_coord(gz, nz, perz);
        for (int t = tid; t < NI; t += NT) {
            int ix = t % IX, iy = t / IX;
            int gx = map_coord(x0 - 2 + ix, nx, perx), gy = map_coord(y0 - 2 + iy, ny, pery);
            long long c = G.at(gx, gy, zz);
            T r = A.U[0][c];
            Prim<T> q = eos(P, r, A.U[1][c], A.U[2][c], A.U[3][c], A.U[4][c]);
            IN(slot, 0, t) = r;
            IN(slot, 1, t) = q.u[0];
            IN(slot, 2, t) = q.u[1];
            IN(slot, 3, t) = q.u[2];
            IN(slot, 4, t) = q.phi;
        }
    };

    // predictor position index -> (px, py); pass 0 = the TX x TY inner block
    // (thread tid owns inner position tid), pass 1 = the one-cell halo ring.
    auto pos_of = [&](int pass, int t, int &px, int &py) {
        if (pass == 0) {
            px = t % TX + 1;
            py = t / TX + 1;
        } else if (t < 2 * PX) {
            px = t % PX;
            py = t < PX ? 0 : PY - 1;
        } else {
            int r = t - 2 * PX;
            px = (r & 1) ? PX - 1 : 0;
            py = 1 + (r >> 1);
        }
    };

    // ---- predictor (Eq. 5) for plane p; own[] receives (U*+U)/2 of m, E and
    // u^n of the inner position owned by this thread.
    auto predict = [&](int p, T own[7]) {
        const int sl = mod3(p), sm = mod3(p - 1), sp = mod3(p + 1);
        const int zz = map_coord(p, nz, perz);
        for (int pass = 0; pass < 2; ++pass) {
            int t = tid;
            if (pass == 1 && t >= NP - NT) break;
            int px, py;
            pos_of(pass, t, px, py);
            const int ip = (py + 1) * IX + (px + 1);
            const T rhoi = IN(sl, 0, ip);
            const T ui[3] = {IN(sl, 1, ip), IN(sl, 2, ip), IN(sl, 3, ip)};
            const T phii = IN(sl, 4, ip);
            T Pp[3] = {T(0), T(0), T(0)}, Wk = T(0);
#pragma unroll
            for (int dz = -1; dz <= 1; ++dz) {
                const int s = dz < 0 ? sm : (dz > 0 ? sp : sl);
#pragma unroll
                for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                    for (int dx = -1; dx <= 1; ++dx) {
                        if (!dx && !dy && !dz) continue;
                        const int j = ip + dy * IX + dx;
                        const T w = P.w[dx * dx + dy * dy + dz * dz];
                        const T phj = IN(s, 4, j);
                        const T r[3] = {h * dx, h * dy, h * dz};
                        const T ru = r[0] * (T(0.5) * (ui[0] + IN(s, 1, j))) +
                                     r[1] * (T(0.5) * (ui[1] + IN(s, 2, j))) +
                                     r[2] * (T(0.5) * (ui[2] + IN(s, 3, j)));
                        const T wp = w * phj;
                        Pp[0] += wp * r[0];
                        Pp[1] += wp * r[1];
                        Pp[2] += wp * r[2];
                        Wk += wp * ru;
                    }
            }
            const int gx = map_coord(x0 - 1 + px, nx, perx), gy = map_coord(y0 - 1 + py, ny, pery);
            const long long c = G.at(gx, gy, zz);
            const T D0[3] = {A.grav[0][c], A.grav[1][c], A.grav[2][c]};
            T Q[4] = {T(0), T(0), T(0), T(0)};
            if (rhoi > P.rho_vac) {
                for (int e = 0; e < 3; ++e) Q[e] = -phii * Pp[e] - rhoi * D0[e];
                Q[3] = -phii * Wk - rhoi * (ui[0] * D0[0] + ui[1] * D0[1] + ui[2] * D0[2]);
            }
            const T m0[3] = {A.U[1][c], A.U[2][c], A.U[3][c]}, E0 = A.U[4][c];
            T ms[3], Es;
            for (int e = 0; e < 3; ++e) ms[e] = m0[e] + dt * Q[e];
            Es = E0 + dt * Q[3];
            Prim<T> q = eos(P, rhoi, ms[0], ms[1], ms[2], Es);
            const int pt = py * PX + px;
            PR(sl, 0, pt) = rhoi;
            for (int e = 0; e < 3; ++e) {
                PR(sl, 1 + e, pt) = q.u[e];
                PR(sl, 5 + e, pt) = dt * T(0.5) * (ui[e] + q.u[e]);
            }
            PR(sl, 4, pt) = q.phi;
            if (pass == 0) {
                for (int e = 0; e < 3; ++e) {
                    own[e] = T(0.5) * (m0[e] + ms[e]);
                    own[4 + e] = ui[e];
                }
                own[3] = T(0.5) * (E0 + Es);
            }
        }
    };

    // ---- predictor-stage ghost record g from b (boundary) and m (next inward)
    // along axis a of face `face`; slots may differ (z) or coincide (x, y).
    auto bc_record = [&](int face, int a, int sg, int tg, int sb, int tb, int smm, int tm,
                         long long cg, long long cm) {
        const int kind = P.bc[face];
        if (kind == BC_PERIODIC) return;
        if (kind == BC_OUTFLOW) {
            for (int f = 0; f < S::NPR; ++f) PR(sg, f, tg) = PR(sb, f, tb);
            return;
        }
        if (kind == BC_INFLOW) {
            PR(sg, 0, tg) = P.inW[face][0];
            PR(sg, 4, tg) = P.inPhi[face];
            for (int e = 0; e < 3; ++e) {
                T ue = P.in_vac[face] ? T(0) : P.inW[face][1 + e];
                PR(sg, 1 + e, tg) = ue;
                PR(sg, 5 + e, tg) = dt * ue;
            }
            return;
        }
        const T rb = PR(sb, 0, tb), phib = PR(sb, 4, tb);
        for (int e = 0; e < 3; ++e) {
            PR(sg, 1 + e, tg) = e == a ? -PR(sb, 1 + e, tb) : PR(sb, 1 + e, tb);
            PR(sg, 5 + e, tg) = e == a ? -PR(sb, 5 + e, tb) : PR(sb, 5 + e, tb);
        }
        T phig = T(0), rho_g = rb;
        if (rb > P.rho_vac && phib > T(0)) {
            phig = PR(smm, 4, tm) + rb * (A.psi[cm] - A.psi[cg]) / phib;
            if (phig < T(0)) phig = T(0);
            T ratio = phig / phib;
            rho_g = rb * ratio * ratio;
        }
        PR(sg, 0, tg) = rho_g;
        PR(sg, 4, tg) = phig;
    };

    // ---- x then y ghost columns/rows of predictor plane p (block-uniform branches)
    auto fill_xy = [&](int p) {
        const int sl = mod3(p);
        const int zz = map_coord(p, nz, perz);
        __syncthreads();
        if (!perx) {
            for (int side = 0; side < 2; ++side) {
                const int gxg = side ? nx : -1;
                const int pxg = gxg - (x0 - 1);
                if (pxg < 0 || pxg >= PX) continue;
                const int pxb = side ? pxg - 1 : pxg + 1;
                const int pxm = nx > 1 ? (side ? pxg - 2 : pxg + 2) : pxb;
                for (int py = tid; py < PY; py += NT) {
                    const int gy = y0 - 1 + py;
                    if (gy < 0 || gy >= ny) continue;
                    bc_record(side, 0, sl, py * PX + pxg, sl, py * PX + pxb, sl, py * PX + pxm,
                              G.at(gxg, gy, zz), G.at(side ? nx - 2 : 1, gy, zz));
                }
            }
        }
        __syncthreads();
        if (!pery) {
            for (int side = 0; side < 2; ++side) {
                const int gyg = side ? ny : -1;
                const int pyg = gyg - (y0 - 1);
                if (pyg < 0 || pyg >= PY) continue;
                const int pyb = side ? pyg - 1 : pyg + 1;
                const int pym = ny > 1 ? (side ? pyg - 2 : pyg + 2) : pyb;
                for (int px = tid; px < PX; px += NT) {
                    const int gx = map_coord(x0 - 1 + px, nx, false);
                    bc_record(2 + side, 1, sl, pyg * PX + px, sl, pyb * PX + px, sl, pym * PX + px,
                              G.at(gx, gyg, zz), G.at(gx, side ? ny - 2 : 1, zz));
                }
            }
        }
        __syncthreads();
    };

    // ---- z ghost plane pg (non-periodic z): from planes pb and pm
    auto fill_z = [&](int pg) {
        const int side = pg < 0 ? 0 : 1;
        const int pb = side ? nz - 1 : 0;
        const int pm = nz > 1 ? (side ? nz - 2 : 1) : pb;
        __syncthreads();
        for (int t = tid; t < NP; t += NT) {
            const int px = t % PX, py = t / PX;
            const int gx = map_coord(x0 - 1 + px, nx, false), gy = map_coord(y0 - 1 + py, ny, false);
            bc_record(4 + side, 2, mod3(pg), t, mod3(pb), t, mod3(pm), t, G.at(gx, gy, pg),
                      G.at(gx, gy, pm));
        }
        __syncthreads();
    };

    // ---- corrector (Eqs. 6-7 with displaced particles) for plane k
    const int tx = tid % TX, ty = tid / TX;
    auto correct = [&](int k, const T own[7]) {
        const int gx = x0 + tx, gy = y0 + ty;
        const int sl = mod3(k), sm = mod3(k - 1), sp = mod3(k + 1);
        const int pi = (ty + 1) * PX + (tx + 1);
        const T rhoi = PR(sl, 0, pi);
        const T ui[3] = {PR(sl, 1, pi), PR(sl, 2, pi), PR(sl, 3, pi)};
        const T phii = PR(sl, 4, pi);
        const T xii[3] = {PR(sl, 5, pi), PR(sl, 6, pi), PR(sl, 7, pi)};
        T Pp[3] = {T(0), T(0), T(0)}, Wk = T(0);
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const int s = dz < 0 ? sm : (dz > 0 ? sp : sl);
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz) continue;
                    const int j = pi + dy * PX + dx;
                    T r[3] = {h * dx + (PR(s, 5, j) - xii[0]), h * dy + (PR(s, 6, j) - xii[1]),
                              h * dz + (PR(s, 7, j) - xii[2])};
                    const T r2 = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
                    const T Gw = gtilde<T>(sqrt(r2) / h) * P.inv_Ch2;
                    const T phj = PR(s, 4, j);
                    const T ru = r[0] * (T(0.5) * (ui[0] + PR(s, 1, j))) +
                                 r[1] * (T(0.5) * (ui[1] + PR(s, 2, j))) +
                                 r[2] * (T(0.5) * (ui[2] + PR(s, 3, j)));
                    const T gp = Gw * phj;
                    Pp[0] += gp * r[0];
                    Pp[1] += gp * r[1];
                    Pp[2] += gp * r[2];
                    Wk += gp * ru;
                }
        }
        if (gx >= nx || gy >= ny) return;
        const long long c = G.at(gx, gy, k);
        const T D0[3] = {A.grav[0][c], A.grav[1][c], A.grav[2][c]};
        T Q[4] = {T(0), T(0), T(0), T(0)};
        if (rhoi > P.rho_vac) {
            for (int e = 0; e < 3; ++e) Q[e] = -phii * Pp[e] - rhoi * D0[e];
            Q[3] = -phii * Wk - rhoi * (ui[0] * D0[0] + ui[1] * D0[1] + ui[2] * D0[2]);
        }
        T m[3], E;
        for (int e = 0; e < 3; ++e) m[e] = own[e] + half_dt * Q[e];
        E = own[3] + half_dt * Q[3];
        Prim<T> q = eos(P, rhoi, m[0], m[1], m[2], E);
        bool far = false;
        for (int e = 0; e < 3; ++e) {
            T xi = T(0.5) * xii[e] + half_dt * (T(0.5) * (own[4 + e] + q.u[e]));
            A.m[e][c] = m[e];
            A.xi[e][c] = xi;
            far |= !(fabs(xi) <= h);
        }
        A.E[c] = E;
        if (far) atomicOr(&A.ctrl->status, ST_CFL);
    };

    // ---- prologue: predictor planes z0-1 and z0 (or 0, 1 and the z ghost -1)
    T cur[7], nxt[7], junk[7];
    int pnext;
    if (!perz && z0 == 0) {
        load_in(-1);
        load_in(0);
        load_in(1);
        __syncthreads();
        predict(0, cur);
        __syncthreads();
        load_in(2);
        __syncthreads();
        predict(1, nxt);
        fill_xy(0);
        fill_xy(1);
        fill_z(-1);
        pnext = 2;
    } else {
        load_in(z0 - 2);
        load_in(z0 - 1);
        load_in(z0);
        __syncthreads();
        predict(z0 - 1, junk);
        __syncthreads();
        load_in(z0 + 1);
        __syncthreads();
        predict(z0, cur);
        fill_xy(z0 - 1);
        fill_xy(z0);
        pnext = z0 + 1;
    }
    for (int k = z0; k < z1; ++k) {
        if (pnext == k + 1) {
            if (!perz && k + 1 == nz) {
                fill_z(nz);
            } else {
                load_in(k + 2);
                __syncthreads();
                predict(k + 1, nxt);
                fill_xy(k + 1);
            }
            ++pnext;
        }
        correct(k, cur);
#pragma unroll
        for (int e = 0; e < 7; ++e) cur[e] = nxt[e];
        __syncthreads();
    }
}

// Eulerian stage, one cell per thread: U^{n+1/2} = (U^n + U~)/2, Eq. 8
// reconstruction with the particle offsets, Riemann flux, Eq. 4 update.
template <typename T>
__global__ void k_euler(Grid G, Phys<T> P, Ctrl *__restrict__ ctrl, UPtr<T> U, S2Ptr<T> S2,
                        UPtr<T> Un) {
    Cell cc;
    const bool in = interior_cell(G, cc);
    double sp = 0.0;
    if (in) {
        const long long c = G.at(cc.i, cc.j, cc.k);
        const T dt = (T)ctrl->dt;
        T v[5];
        if (dt > T(0)) {
            const T h = P.h;
            T div[5] = {T(0), T(0), T(0), T(0), T(0)};
            const int id[3] = {cc.i, cc.j, cc.k};
#pragma unroll
            for (int d = 0; d < 3; ++d) {
                const long long s = d == 0 ? 1 : (d == 1 ? (long long)G.px : G.plane);
                const bool wall_lo = id[d] == 0 && P.bc[2 * d] == BC_WALL;
                const bool wall_hi = id[d] == G.n[d] - 1 && P.bc[2 * d + 1] == BC_WALL;
                const long long cm = c - s, cp = c + s;
                const T xm = S2.xi[d][cm], x0 = S2.xi[d][c], xp = S2.xi[d][cp];
                const T am = xm / dt, a0 = x0 / dt, ap = xp / dt;
                int im[3] = {cc.i, cc.j, cc.k}, ipp[3] = {cc.i, cc.j, cc.k};
                im[d] -= 1;
                ipp[d] += 1;
#pragma unroll
                for (int f = 0; f < 5; ++f) {
                    const T *uf = U.f[f];
                    const T th0 = slope_at(G, P, uf, d, cc.i, cc.j, cc.k);
                    const T thm = slope_at(G, P, uf, d, im[0], im[1], im[2]);
                    const T thp = slope_at(G, P, uf, d, ipp[0], ipp[1], ipp[2]);
                    const T tm = f == 0 ? uf[cm] : (f == 4 ? S2.E[cm] : S2.m[f - 1][cm]);
                    const T t0 = f == 0 ? uf[c] : (f == 4 ? S2.E[c] : S2.m[f - 1][c]);
                    const T tp = f == 0 ? uf[cp] : (f == 4 ? S2.E[cp] : S2.m[f - 1][cp]);
                    const T hm = T(0.5) * (uf[cm] + tm), h0 = T(0.5) * (uf[c] + t0),
                            hp = T(0.5) * (uf[cp] + tp);
                    // face c-1/2: L = c-1, R = c
                    T Fm = T(0);
                    if (!wall_lo) {
                        const T UL = hm + T(0.5) * (h - xm) * thm;
                        const T UR = h0 - T(0.5) * (h + x0) * th0;
                        Fm = riemann_flux<T>(P.riemann, am, a0, UL, UR);
                    }
                    T Fp = T(0);
                    if (!wall_hi) {
                        const T UL = h0 + T(0.5) * (h - x0) * th0;
                        const T UR = hp - T(0.5) * (h + xp) * thp;
                        Fp = riemann_flux<T>(P.riemann, a0, ap, UL, UR);
                    }
                    div[f] += Fp - Fm;
                }
            }
            const T base[5] = {U.f[0][c], S2.m[0][c], S2.m[1][c], S2.m[2][c], S2.E[c]};
            for (int f = 0; f < 5; ++f) v[f] = base[f] - dt / h * div[f];
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
