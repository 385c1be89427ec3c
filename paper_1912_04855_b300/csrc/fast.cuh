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
//    update) on the same tiling: in-plane slopes are computed once per cell
//    into shared memory, z slopes and z fluxes stay in registers along the
//    march; the epilogue reduces the signal speed for the next dt and checks
//    the state.
//
// Both kernels work in cell units: offsets xi^ = xi/h, and the Euler stage
// uses Courant-scaled fluxes G = (dt/h) F, which for the advective flux
// F = (xi/dt) U is G = xi^ U -- dt and h drop out of the face arithmetic.
// FP32 instantiations use the SFU reciprocal and reciprocal square root; FP64
// instantiations keep IEEE division and square root.
#pragma once

#include "common.cuh"
#include "ghost.cuh"
#include "plain.cuh"
#include "tma.cuh"

namespace cspht {

template <typename T>
struct alignas(4 * sizeof(T)) V4 {
    T x, y, z, w;
};

__device__ __forceinline__ float f_rcp(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double f_rcp(double x) { return 1.0 / x; }
__device__ __forceinline__ float f_sqrt(float x) { return x > 0.0f ? x * rsqrtf(x) : 0.0f; }
__device__ __forceinline__ double f_sqrt(double x) { return sqrt(x); }
// 1/sqrt(x) for x > 0
__device__ __forceinline__ float f_rsqrt(float x) { return rsqrtf(x); }
__device__ __forceinline__ double f_rsqrt(double x) { return 1.0 / sqrt(x); }

// The same for arguments known to be normal numbers (FP32: x >= 2^-126) or
// zero: the SFU instructions without the subnormal handling, which such an
// argument never needs (the result is the same).  FP64 as above.
__device__ __forceinline__ float f_rsqrt_n(float x) {
    float r;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double f_rsqrt_n(double x) { return 1.0 / sqrt(x); }
__device__ __forceinline__ float f_rcp_n(float x) {
    float r;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
    return r;
}
__device__ __forceinline__ double f_rcp_n(double x) { return 1.0 / x; }
// sqrt(x), 0 for x below the smallest normal number (FP32)
__device__ __forceinline__ float f_sqrt_n(float x) { return x >= 1.17549435e-38f ? x * f_rsqrt_n(x) : 0.0f; }
__device__ __forceinline__ double f_sqrt_n(double x) { return x > 0.0 ? sqrt(x) : 0.0; }

// Round-to-nearest operations the compiler may not contract or reorder.  The
// predictor's plane sums, the reconstruction and the fluxes use them, so a
// value computed at two places (two call sites, neighbouring tiles or z
// chunks) has the same bits in both: a face enters its two cells exactly.
__device__ __forceinline__ float r_add(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return __dadd_rn(a, b); }
__device__ __forceinline__ float r_sub(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ double r_sub(double a, double b) { return __dsub_rn(a, b); }
__device__ __forceinline__ float r_mul(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double r_mul(double a, double b) { return __dmul_rn(a, b); }
__device__ __forceinline__ float r_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
__device__ __forceinline__ double r_fma(double a, double b, double c) { return __fma_rn(a, b, c); }

// Error-free sum a + b = s + err (Knuth's TwoSum).  The round-to-nearest
// intrinsics are never contracted or reassociated by the compiler.
__device__ __forceinline__ float two_sum(float a, float b, float &err) {
    const float s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    err = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
    return s;
}

// The balance of the Lagrangian force, -(a b) - c d: the pressure term phi_i
// P (a = phi_i / (C h), b = the pressure sum) against the gravity term
// rho_i D0 (c = rho_i, d = D0[psi]).  In a hydrostatic state the two nearly
// cancel.  COMP (FP32 only) forms both products exactly (TwoProd with an
// fma) and adds them with TwoSum, so the difference is rounded once;
// otherwise it is the plain expression.
template <typename T, bool COMP>
__device__ __forceinline__ T balance(T a, T b, T c, T d) {
    if constexpr (COMP && sizeof(T) == 4) {
        const float p = __fmul_rn(a, b), pe = __fmaf_rn(a, b, -p);
        const float q = __fmul_rn(c, d), qe = __fmaf_rn(c, d, -q);
        float err;
        const float s = two_sum(-p, -q, err);
        return __fadd_rn(s, __fsub_rn(__fsub_rn(err, pe), qe));
    } else {
        return -a * b - c * d;
    }
}

// Primitive recovery with the fast reciprocal / square root.
template <typename T>
__device__ __forceinline__ Prim<T> eos_fast(const Phys<T> &P, T rho, T mx, T my, T mz, T E) {
    Prim<T> r;
    if (!(rho > P.rho_vac)) {
        r.vac = true;
        r.u[0] = r.u[1] = r.u[2] = T(0);
        r.p = r.phi = T(0);
        return r;
    }
    r.vac = false;
    const T ir = f_rcp_n(rho);  // rho > rho_vac >= 2^-126 (FP32): a normal number
    r.u[0] = mx * ir;
    r.u[1] = my * ir;
    r.u[2] = mz * ir;
    T p = P.gm1 * (E - T(0.5) * (mx * r.u[0] + my * r.u[1] + mz * r.u[2]));
    if (p < T(0)) p = T(0);
    r.p = p;
    r.phi = f_sqrt_n(T(2) * p);
    return r;
}

// Kernel weight gt(q) / 0.75 for the squared distance q2 = q^2 in cell units,
// evaluated without branches: 4 - 3 q (q < 1), (2-q)^2 / q (q < 2), 0 beyond
// (the factor 0.75 is applied once to the pair sum by the caller).  The
// caller passes q2 >= 1e-30 (sq_len), so that two coinciding particles give
// a finite weight and a zero pair vector instead of a NaN.
template <typename T>
__device__ __forceinline__ T gtilde_q2_4_3(T q2) {
    const T rs = f_rsqrt_n(q2);
    const T q = q2 * rs;
    T a = T(2) - q;
    a = a > T(0) ? a : T(0);
    const T outer = a * a * rs;
    const T inner = T(4) - T(3) * q;
    return q < T(1) ? inner : outer;
}

// |r|^2 + 1e-30: the floor costs no instruction (it seeds the sum) and is
// below the rounding of any separation the step produces.
template <typename T>
__device__ __forceinline__ T sq_len(T rx, T ry, T rz) {
    return r_fma(rx, rx, r_fma(ry, ry, r_fma(rz, rz, T(1e-30))));
}

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

// Coordinate of a tile position in the padded arrays: wrapped on periodic
// axes, clamped into the one-cell ghost layer otherwise (positions further
// out only feed values that the boundary fill overwrites or that no output
// cell reads).
__device__ __forceinline__ int map_coord(int a, int n, bool per) {
    if (a >= 0 && a < n) return a;  // the common case, without a division
    if (per) return wrap_idx(a, n);
    return a < -1 ? -1 : (a > n ? n : a);
}

// a mod 3 for a >= -3 (plane indices of the rings start at -2)
__device__ __forceinline__ int mod3(int a) { return (int)((unsigned)(a + 3) % 3u); }

// Elements of a TMA destination slot holding n elements of T: rounded up so
// that every slot starts on a 128-byte boundary (required of tensor-copy
// destinations in shared memory).
template <typename T>
__host__ __device__ constexpr int tma_slot(int n) {
    return (int)(((size_t)n * sizeof(T) + 127) / 128 * 128 / sizeof(T));
}

// ============================================================ Lagrangian stage

// Tensor-map descriptors of the arguments: held inside them (the one-grid
// kernels, which receive the arguments as their kernel parameter), or
// pointers to copies in device memory (the multi-grid kernels, whose kernel
// parameter holds the arguments of a whole group of grids).  at(f) is the
// descriptor's address either way.
template <int N>
struct MapsIn {
    CUtensorMap m[N];
    __device__ __forceinline__ const CUtensorMap *at(int f) const { return &m[f]; }
};
template <int N>
struct MapsAt {
    const CUtensorMap *m[N];
    __device__ __forceinline__ const CUtensorMap *at(int f) const { return m[f]; }
};

template <typename T, template <int> class Maps = MapsIn>
struct LagArgs {
    Maps<5> tmU;  // TMA descriptors of the five U^n fields (box TX+8 x TY+4 x 1)
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

template <int TX, int TY>
struct LagShape {
    static constexpr int BW = TX + 8, BH = TY + 4, NB = BW * BH;  // TMA box: x0-4.., y0-2..
    static constexpr int IX = TX + 4, IY = TY + 4, NI = IX * IY;  // U^n primitives (halo 2)
    static constexpr int PX = TX + 2, PY = TY + 2, NP = PX * PY;  // predictor particles
    static constexpr int NT = TX * TY;
    static constexpr int SLOTS = 2;                               // TMA ring depth
    // FP32 runs the paired tile (two columns per thread, lagrange_pair.cuh)
    template <typename T>
    __host__ __device__ static constexpr int threads() { return sizeof(T) == 4 ? TX * TY / 2 : TX * TY; }
    template <typename T>
    __host__ __device__ static constexpr size_t bytes();
    template <typename T>
    __host__ __device__ static constexpr size_t smem_bytes() {
        // raw U^n boxes, primitives ring V4(u,v,w,phi), predictor ring 2 x V4, barriers
        return (size_t)SLOTS * 5 * tma_slot<T>(NB) * sizeof(T) + 3 * (size_t)NI * sizeof(V4<T>) +
               3 * (size_t)NP * 2 * sizeof(V4<T>) + 64;
    }
};

// Start of a CTA of the Lagrangian kernels: initialises the copy barriers and
// checks that every copy destination starts on a 128-byte boundary (false, and
// the time-out status bit, if one does not).
template <typename T, int TX, int TY>
__device__ __forceinline__ bool lagrange_begin(Ctrl *ctrl) {
    using S = LagShape<TX, TY>;
    constexpr int NB = tma_slot<T>(S::NB), NI = S::NI, NP = S::NP, NT = S::NT;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sraw = reinterpret_cast<T *>(smem_raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(reinterpret_cast<V4<T> *>(sraw + S::SLOTS * 5 * NB) + 3 * NI + 6 * NP);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int q = 0; q < S::SLOTS; ++q) mbar_init(&bar[q], 1);
        mbar_init_fence();
    }
    bool misaligned = false;
    for (int q = tid; q < S::SLOTS * 5; q += NT) misaligned |= (smem_u32(sraw + q * NB) & 127u) != 0;
    if (__syncthreads_or(misaligned)) {
        if (tid == 0) atomicOr(&ctrl->status, ST_TIMEOUT);
        return false;
    }
    return true;
}

// One tile of the Lagrangian stage, one column per thread (the FP64 kernels;
// FP32 runs the paired tile of lagrange_pair.cuh): the TX x TY columns of
// tile (bx, by) over z chunk bz.  INIT: the tile is the CTA's only one and initialises the copy
// barriers itself (the one-grid kernel); otherwise lagrange_begin did, once
// per CTA.  phase_bits carries the barriers' parities from one tile of the
// CTA to the next (every copy a tile issues is waited for before it
// returns).  Returns false after a copy time-out or a misaligned copy
// destination: the CTA must not start another tile.
template <typename T, int TX, int TY, bool COMP, bool INIT, class Args>
__device__ __forceinline__ bool lagrange_tile(const Args &A, const int bx, const int by, const int bz,
                                              uint32_t &phase_bits) {
    using S = LagShape<TX, TY>;
    constexpr int BW = S::BW, NB = tma_slot<T>(S::NB), IX = S::IX, NI = S::NI, PX = S::PX,
                  PY = S::PY, NP = S::NP, NT = S::NT;  // NB: box slot stride (128-byte multiple)
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sraw = reinterpret_cast<T *>(smem_raw);                       // [SLOTS][5][NB]
    V4<T> *sinU = reinterpret_cast<V4<T> *>(sraw + S::SLOTS * 5 * NB); // [3][NI] (u,v,w,phi) of U^n
    V4<T> *spU = sinU + 3 * NI;                                      // [3][NP] (u*,v*,w*,phi*)
    V4<T> *spX = spU + 3 * NP;                                       // [3][NP] (xi*^, rho)
    uint64_t *bar = reinterpret_cast<uint64_t *>(spX + 3 * NP);      // [SLOTS]

    const Grid &G = A.G;
    const Phys<T> &P = A.P;
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const bool perx = P.bc[0] == BC_PERIODIC, pery = P.bc[2] == BC_PERIODIC,
               perz = P.bc[4] == BC_PERIODIC;
    const int tid = threadIdx.x;
    const int x0 = bx * TX, y0 = by * TY;
    const int z0 = bz * A.zchunk;
    const int z1 = min(z0 + A.zchunk, nz);
    const T dt = (T)A.ctrl->dt;
    if (!(dt > T(0))) return true;  // a zero step: the Euler kernel copies U^n
    const int spin = A.ctrl->spin_limit > 0 ? A.ctrl->spin_limit : MBAR_SPIN_LIMIT;
    const bool no_copies = (A.ctrl->inject & INJECT_NO_COPIES) != 0;
    const T h = P.h, inv_h = P.inv_h, half_dt = T(0.5) * dt;
    const T dth = dt * inv_h;                          // dt/h: velocity -> offset in cell units
    const T kf = P.inv_Ch2 * h;                        // 1/(C h): G(r) r = gt(q) r^ / (C h)
    const T kf34 = T(0.75) * kf;                       // the corrector sums gt(q) / 0.75
    const T w1 = P.gt[1], w2 = P.gt[2], w3 = P.gt[3];  // gt(|d|) of the static lattice

    // Padded-array offsets of the tile's columns and rows (for the gravity
    // loads and the corrector's stores; 32-bit offsets are guaranteed by the handle).
    __shared__ int s_colx[IX], s_rowy[S::IY];
    for (int t = tid; t < IX; t += NT) s_colx[t] = map_coord(x0 - 2 + t, nx, perx) + G.ox;
    for (int t = tid; t < S::IY; t += NT) s_rowy[t] = (map_coord(y0 - 2 + t, ny, pery) + GH) * G.px;
    if constexpr (INIT) {
        if (tid == 0) {
            for (int q = 0; q < S::SLOTS; ++q) mbar_init(&bar[q], 1);
            mbar_init_fence();
        }
        // every TMA destination must start on a 128-byte boundary: refuse to run otherwise
        bool misaligned = false;
        for (int q = tid; q < S::SLOTS * 5; q += NT) misaligned |= (smem_u32(sraw + q * NB) & 127u) != 0;
        if (__syncthreads_or(misaligned)) {
            if (tid == 0) atomicOr(&A.ctrl->status, ST_TIMEOUT);
            return false;
        }
    }
    // (otherwise the first reads of s_colx / s_rowy follow the barrier after
    // the first two fetches)
    auto zoff = [&](int gz) { return (map_coord(gz, nz, perz) + GH) * (int)G.plane; };

    // ---- TMA ring: plane q lives in slot q mod 2; box origin (x0-4, y0-2) in
    // cell coordinates, i.e. padded element (x0-4+ox, y0-2+GH, z+GH).  Plane q
    // may be issued once plane q-2 is consumed: converted, and predicted if it
    // is a predictor plane (its raw box supplies the predictor's own U^n).
    // phase_bits: parity of the next completion, per slot (block-uniform)
    uint32_t pending = 0;     // slots with a box in flight (block-uniform)
    int issued = (!perz && z0 == 0) ? -2 : z0 - 3;  // last plane issued (block-uniform)
    static_assert(S::SLOTS == 2, "the TMA ring has two slots");
    auto slot_of = [](int q) { return q & 1; };  // q mod 2, also for negative q
    auto issue = [&](int q) {
        pending |= 1u << slot_of(q);
        if (tid == 0) {
            const int sl = slot_of(q);
            fence_proxy_async();
            mbar_arrive_expect_tx(&bar[sl], (uint32_t)(5 * S::NB * sizeof(T)));
            const int zc = map_coord(q, nz, perz) + GH;
            if (!no_copies)
                for (int f = 0; f < 5; ++f)
                    tma_load_3d(sraw + (sl * 5 + f) * NB, A.tmU.at(f), x0 - 4 + G.ox, y0 - 2 + GH, zc, &bar[sl]);
        }
        issued = q;
    };
    auto issue_upto = [&](int q) {
        while (issued < q) issue(issued + 1);
    };
    // Waits in this thread for plane q's box (bounded); false on a time-out.
    // No barrier: the caller's next barrier publishes what is made from the
    // box and lets every thread agree on a time-out (__syncthreads_or).
    auto wait_box = [&](int q) -> bool {
        const int sl = slot_of(q);
        const bool ok = mbar_wait(&bar[sl], (phase_bits >> sl) & 1u, spin);
        if (ok) {
            phase_bits ^= 1u << sl;
            pending &= ~(1u << sl);
        }
        return ok;
    };
    // After a time-out: waits (bounded) for the boxes still in flight.
    auto drain = [&]() {
        for (int s2 = 0; s2 < S::SLOTS; ++s2)
            if ((pending >> s2) & 1u) mbar_wait(&bar[s2], (phase_bits >> s2) & 1u, spin);
    };
    auto RAW = [&](int q, int f, int bx, int by) -> T { return sraw[(slot_of(q) * 5 + f) * NB + by * BW + bx]; };

    // ---- U^n plane q: raw box -> primitives ring (halo 2)
    auto convert = [&](int q) {
        const int slot = mod3(q);
        for (int t = tid; t < NI; t += NT) {
            const int ix = t % IX, iy = t / IX;
            const int b = (slot_of(q) * 5) * NB + iy * BW + ix + 2;
            const T r = sraw[b];
            const Prim<T> qq = eos_fast(P, r, sraw[b + NB], sraw[b + 2 * NB], sraw[b + 3 * NB], sraw[b + 4 * NB]);
            sinU[slot * NI + t] = V4<T>{qq.u[0], qq.u[1], qq.u[2], qq.phi};
        }
    };
    // Converts this thread's share of plane q (issuing further planes ahead);
    // a barrier must follow before the primitives are read.
    auto fetch = [&](int q) -> bool {
        issue_upto(q);
        if (!wait_box(q)) return false;
        convert(q);
        return true;
    };

    // predictor position of (pass, t): pass 0 = the TX x TY inner block
    // (thread tid owns inner position tid), pass 1 = the one-cell halo ring.
    auto pos_of = [&](int pass, int t, int &px, int &py) {
        if (pass == 0) {
            px = t % TX + 1;
            py = t / TX + 1;
        } else if (t < 2 * PX) {
            px = t % PX;
            py = t < PX ? 0 : PY - 1;
        } else {
            const int r = t - 2 * PX;
            px = (r & 1) ? PX - 1 : 0;
            py = 1 + (r >> 1);
        }
    };

    // ---- predictor force sums as in-plane partial sums (Eq. 7 on the static
    // lattice).  The weight gt(|d|) depends on |d|^2 only, so a particle's
    // 26-neighbour sums split into 3 x 3 sums over each U^n plane it touches:
    // its own plane (role 0, centre excluded) and the planes below and above
    // (role 1, every position, |d|^2 one larger).  Per plane and column, with
    // weight a_j = gt(|d|) phi_j: X, Y = sum of dx a_j, dy a_j; V = sum of
    // a_j (dx u_j + dy v_j); role 1 also Z = sum of a_j and T = sum of a_j w_j
    // (the plane's side gives dz).  Then P^ = (X0 + X1- + X1+, Y0 + Y1- + Y1+,
    // Z+ - Z-) and sum_j a_j d.u_j = V0 + V1- + V1+ + T+ - T-.
    // A thread's inner particle keeps its column's sums of planes p-1 and p
    // from the iterations before, so it reads one plane (9 positions), not 27.
    // The sums use the pinned operations: every call site, and so every chunk
    // and tile, gives the same bits for the same particle.
    struct Sum0 {
        T X, Y, V;
    };
    struct Sum1 {
        T X, Y, V, Z, W;
    };
    auto plane_sums = [&](int slot, int ip, bool want0, bool want1, Sum0 &s0, Sum1 &s1) {
        s0 = Sum0{T(0), T(0), T(0)};
        s1 = Sum1{T(0), T(0), T(0), T(0), T(0)};
        const V4<T> *pl = sinU + slot * NI + ip;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int d2 = dx * dx + dy * dy;
                const V4<T> qj = pl[dy * IX + dx];
                T ru = T(0);  // dx u_j + dy v_j
                if (dx && dy) ru = r_add(dx > 0 ? qj.x : -qj.x, dy > 0 ? qj.y : -qj.y);
                else if (dx) ru = dx > 0 ? qj.x : -qj.x;
                else if (dy) ru = dy > 0 ? qj.y : -qj.y;
                if (want0 && d2 > 0) {
                    const T a = r_mul(d2 == 1 ? w1 : w2, qj.w);
                    if (dx) s0.X = dx > 0 ? r_add(s0.X, a) : r_sub(s0.X, a);
                    if (dy) s0.Y = dy > 0 ? r_add(s0.Y, a) : r_sub(s0.Y, a);
                    s0.V = r_fma(a, ru, s0.V);
                }
                if (want1) {
                    const T b = r_mul(d2 == 0 ? w1 : (d2 == 1 ? w2 : w3), qj.w);
                    if (dx) s1.X = dx > 0 ? r_add(s1.X, b) : r_sub(s1.X, b);
                    if (dy) s1.Y = dy > 0 ? r_add(s1.Y, b) : r_sub(s1.Y, b);
                    if (d2 > 0) s1.V = r_fma(b, ru, s1.V);
                    s1.Z = r_add(s1.Z, b);
                    s1.W = r_fma(b, qj.z, s1.W);
                }
            }
    };
    Sum1 c1m, c1;  // the inner particle's role-1 sums of planes p-1 and p
    Sum0 c0;       // and its role-0 sums of plane p

    // ---- predictor (Eq. 5) for plane p.  own[] receives, for the inner
    // position owned by this thread, (U^n + U*)/2 of m and E, u^n and the
    // lattice gravity D0 (the corrector of the same cell reuses it).
    // Static lattice: r_ij = h d, G(h|d|) h d = gt(|d|) d / (C h); the pressure
    // work sum_j G r.(u_i+u_j)/2 phi_j = (u_i.P^ + sum_j G phi_j r.u_j)/2.
    auto predict = [&](int p, T own[10]) {
        const int sl = mod3(p), sm = mod3(p - 1), sp = mod3(p + 1);
        const int zo = zoff(p);
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            const int t = tid;
            if (pass == 1 && t >= NP - NT) break;
            int px, py;
            pos_of(pass, t, px, py);
            const int ip = (py + 1) * IX + (px + 1);
            // the lattice gravity of the particle, loaded before the plane sums so
            // that their arithmetic covers the global-load latency
            const int c = zo + s_rowy[py + 1] + s_colx[px + 1];
            const T D0[3] = {A.grav[0][c], A.grav[1][c], A.grav[2][c]};
            Sum0 s0, n0;
            Sum1 s1m, s1p, unused1;
            if (pass == 0) {  // plane p+1 is new; p-1 and p come from the column's cache
                plane_sums(sp, ip, true, true, n0, s1p);
                s0 = c0;
                s1m = c1m;
                c1m = c1;
                c1 = s1p;
                c0 = n0;
            } else {
                plane_sums(sm, ip, false, true, n0, s1m);
                plane_sums(sl, ip, true, false, s0, unused1);
                plane_sums(sp, ip, false, true, n0, s1p);
            }
            const T Px = r_add(r_add(s0.X, s1m.X), s1p.X);
            const T Py = r_add(r_add(s0.Y, s1m.Y), s1p.Y);
            const T Pz = r_sub(s1p.Z, s1m.Z);
            const T Wj = r_add(r_add(r_add(s0.V, s1m.V), s1p.V), r_sub(s1p.W, s1m.W));
            const V4<T> qi = sinU[sl * NI + ip];
            const T Wk = T(0.5) * (qi.x * Px + qi.y * Py + qi.z * Pz + Wj);
            const T rhoi = RAW(p, 0, px + 3, py + 1);
            T Q[4] = {T(0), T(0), T(0), T(0)};
            if (rhoi > P.rho_vac) {
                const T pf = qi.w * kf;  // phi_i / (C h)
                Q[0] = balance<T, COMP>(pf, Px, rhoi, D0[0]);
                Q[1] = balance<T, COMP>(pf, Py, rhoi, D0[1]);
                Q[2] = balance<T, COMP>(pf, Pz, rhoi, D0[2]);
                Q[3] = balance<T, COMP>(pf, Wk, rhoi, qi.x * D0[0] + qi.y * D0[1] + qi.z * D0[2]);
            }
            const T m0[3] = {RAW(p, 1, px + 3, py + 1), RAW(p, 2, px + 3, py + 1), RAW(p, 3, px + 3, py + 1)};
            const T E0 = RAW(p, 4, px + 3, py + 1);
            T ms[3];
            for (int e = 0; e < 3; ++e) ms[e] = m0[e] + dt * Q[e];
            const T Es = E0 + dt * Q[3];
            const Prim<T> q = eos_fast(P, rhoi, ms[0], ms[1], ms[2], Es);
            const int pt = sl * NP + py * PX + px;
            spU[pt] = V4<T>{q.u[0], q.u[1], q.u[2], q.phi};
            spX[pt] = V4<T>{dth * T(0.5) * (qi.x + q.u[0]), dth * T(0.5) * (qi.y + q.u[1]),
                            dth * T(0.5) * (qi.z + q.u[2]), rhoi};
            if (pass == 0) {
                for (int e = 0; e < 3; ++e) own[e] = T(0.5) * (m0[e] + ms[e]);
                own[3] = T(0.5) * (E0 + Es);
                own[4] = qi.x;
                own[5] = qi.y;
                own[6] = qi.z;
                own[7] = D0[0];
                own[8] = D0[1];
                own[9] = D0[2];
            }
        }
    };

    // ---- predictor-stage ghost record g from b (boundary) and m (next inward)
    // along axis a of face `face` (indices into the predictor ring).
    auto bc_record = [&](int face, int a, int ig, int ib, int im, long long cg, long long cm) {
        const int kind = P.bc[face];
        if (kind == BC_PERIODIC) return;
        if (kind == BC_OUTFLOW) {
            spU[ig] = spU[ib];
            spX[ig] = spX[ib];
            return;
        }
        if (kind == BC_INFLOW) {
            const bool vac = P.in_vac[face];
            const T u = vac ? T(0) : P.inW[face][1], v = vac ? T(0) : P.inW[face][2],
                    w = vac ? T(0) : P.inW[face][3];
            spU[ig] = V4<T>{u, v, w, P.inPhi[face]};
            spX[ig] = V4<T>{dth * u, dth * v, dth * w, P.inW[face][0]};
            return;
        }
        V4<T> ub = spU[ib], xb = spX[ib];
        const T rb = xb.w, phib = ub.w;
        if (a == 0) { ub.x = -ub.x; xb.x = -xb.x; }
        if (a == 1) { ub.y = -ub.y; xb.y = -xb.y; }
        if (a == 2) { ub.z = -ub.z; xb.z = -xb.z; }
        T phig = T(0), rho_g = rb;
        if (rb > P.rho_vac && phib > T(0)) {
            phig = spU[im].w + rb * (A.psi[cm] - A.psi[cg]) / phib;
            if (phig < T(0)) phig = T(0);
            const T ratio = phig / phib;
            rho_g = rb * ratio * ratio;
        }
        ub.w = phig;
        xb.w = rho_g;
        spU[ig] = ub;
        spX[ig] = xb;
    };

    // ---- x then y ghosts of predictor plane p (block-uniform branches)
    // tiles whose predictor region reaches a non-periodic x or y face (block-uniform)
    const bool edge_tile = (!perx && (x0 == 0 || x0 + TX >= nx)) || (!pery && (y0 == 0 || y0 + TY >= ny));
    auto fill_xy = [&](int p) {
        if (!edge_tile) return;  // nothing to fill; the caller's barrier orders predict and correct
        const int sl = mod3(p) * NP;
        const int zz = map_coord(p, nz, perz);
        __syncthreads();
        if (!perx) {
            for (int side = 0; side < 2; ++side) {
                const int gxg = side ? nx : -1;
                const int pxg = gxg - (x0 - 1);
                if (pxg < 0 || pxg >= PX) continue;
                const int pxb = side ? pxg - 1 : pxg + 1;
                const int pxm = side ? pxg - 2 : pxg + 2;
                // every row whose y resolves inside the domain: the in-range rows,
                // and with periodic y also the wrapped halo rows (x is resolved
                // innermost, so their x ghosts follow the x rule too)
                for (int py = tid; py < PY; py += NT) {
                    const int gy = y0 - 1 + py;
                    if (!pery && (gy < 0 || gy >= ny)) continue;
                    const int gyi = map_coord(gy, ny, pery);
                    bc_record(side, 0, sl + py * PX + pxg, sl + py * PX + pxb, sl + py * PX + pxm,
                              G.at(gxg, gyi, zz), G.at(side ? nx - 2 : 1, gyi, zz));
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
                const int pym = side ? pyg - 2 : pyg + 2;
                for (int px = tid; px < PX; px += NT) {
                    const int gx = map_coord(x0 - 1 + px, nx, perx);
                    bc_record(2 + side, 1, sl + pyg * PX + px, sl + pyb * PX + px, sl + pym * PX + px,
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
        const int pm = side ? nz - 2 : 1;
        __syncthreads();
        for (int t = tid; t < NP; t += NT) {
            const int px = t % PX, py = t / PX;
            const int gx = map_coord(x0 - 1 + px, nx, perx), gy = map_coord(y0 - 1 + py, ny, pery);
            bc_record(4 + side, 2, mod3(pg) * NP + t, mod3(pb) * NP + t, mod3(pm) * NP + t,
                      G.at(gx, gy, pg), G.at(gx, gy, pm));
        }
        __syncthreads();
    };

    // ---- corrector (Eqs. 6-7, particles displaced by xi*) for plane k.
    // r^ = d + xi*^_j - xi*^_i, q = |r^|, G(r) r = gt(q) r^ / (C h).
    const int tx = tid % TX, ty = tid / TX;
    auto correct = [&](int k, const T own[10]) {
        const int gx = x0 + tx, gy = y0 + ty;
        const int sl = mod3(k), sm = mod3(k - 1), sp = mod3(k + 1);
        const int pi = (ty + 1) * PX + (tx + 1);
        const V4<T> qi = spU[sl * NP + pi];
        const V4<T> xi = spX[sl * NP + pi];
        // d - xi*^_i for d = -1, 0, 1 along each axis: r^ = xi*^_j + (d - xi*^_i)
        const T ox[3] = {T(-1) - xi.x, -xi.x, T(1) - xi.x}, oy[3] = {T(-1) - xi.y, -xi.y, T(1) - xi.y},
                oz[3] = {T(-1) - xi.z, -xi.z, T(1) - xi.z};
        T Px = T(0), Py = T(0), Pz = T(0), Wj = T(0);
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const int so = (dz < 0 ? sm : (dz > 0 ? sp : sl)) * NP + pi;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz) continue;
                    const int j = so + dy * PX + dx;
                    const V4<T> qj = spU[j];
                    const V4<T> xj = spX[j];
                    const T rx = xj.x + ox[dx + 1], ry = xj.y + oy[dy + 1], rz = xj.z + oz[dz + 1];
                    const T gp = gtilde_q2_4_3(sq_len(rx, ry, rz)) * qj.w;
                    Px += gp * rx;
                    Py += gp * ry;
                    Pz += gp * rz;
                    Wj += gp * (rx * qj.x + ry * qj.y + rz * qj.z);
                }
        }
        if (gx >= nx || gy >= ny) return;
        const T rhoi = xi.w;
        const T Wk = T(0.5) * (qi.x * Px + qi.y * Py + qi.z * Pz + Wj);
        const int c = (k + GH) * (int)G.plane + s_rowy[ty + 2] + s_colx[tx + 2];
        const T D0[3] = {own[7], own[8], own[9]};
        T Q[4] = {T(0), T(0), T(0), T(0)};
        if (rhoi > P.rho_vac) {
            const T pf = qi.w * kf34;
            Q[0] = balance<T, COMP>(pf, Px, rhoi, D0[0]);
            Q[1] = balance<T, COMP>(pf, Py, rhoi, D0[1]);
            Q[2] = balance<T, COMP>(pf, Pz, rhoi, D0[2]);
            Q[3] = balance<T, COMP>(pf, Wk, rhoi, qi.x * D0[0] + qi.y * D0[1] + qi.z * D0[2]);
        }
        T m[3];
        for (int e = 0; e < 3; ++e) m[e] = own[e] + half_dt * Q[e];
        const T E = own[3] + half_dt * Q[3];
        const Prim<T> q = eos_fast(P, rhoi, m[0], m[1], m[2], E);
        const T xs[3] = {xi.x, xi.y, xi.z};
        bool far = false;
        for (int e = 0; e < 3; ++e) {
            // xi^{n+1} = xi*/2 + dt/2 (u^n + u~)/2, stored in length units
            const T x = h * (T(0.5) * xs[e]) + half_dt * (T(0.5) * (own[4 + e] + q.u[e]));
            A.m[e][c] = m[e];
            A.xi[e][c] = x;
            far |= !(fabs(x) <= h);
        }
        A.E[c] = E;
        if (far) atomicOr(&A.ctrl->status, ST_CFL);
    };

    // issue_upto(p + 2) follows predict(p) and a barrier.
    // last input plane a predictor of this chunk reads (the z ghost nz is
    // filled by the boundary rule, not predicted, on a non-periodic top)
    const int zlast = (!perz && z1 == nz) ? nz : z1 + 1;
    auto timed_out = [&]() {
        if (tid == 0) atomicOr(&A.ctrl->status, ST_TIMEOUT);
    };

    // ---- one march: iteration p predicts plane p (or fills the z ghost plane
    // of a non-periodic top), then corrects plane p - 1.  Every plane is
    // predicted at this one call site, including the planes a chunk shares
    // with its neighbours, so the shared planes carry identical bits whatever
    // the chunk length.  A chunk starts at z0 - 1 (its lower neighbour plane);
    // the first chunk of a non-periodic z starts at 0 and fills the ghost plane
    // -1 once planes 0 and 1 are predicted.
    const bool zero = !perz && z0 == 0;
    const int pfirst = zero ? 0 : z0 - 1;
    bool ok = fetch(pfirst - 1);
    ok = ok && fetch(pfirst);
    // the first in-loop fetch issues a box into the slot that plane pfirst - 1
    // was converted from
    if (__syncthreads_or(!ok)) { drain(); timed_out(); return false; }
    {  // the inner particle's sums of the planes before the first predicted one
        int px, py;
        pos_of(0, tid, px, py);
        const int ip = (py + 1) * IX + (px + 1);
        Sum0 unused0;
        plane_sums(mod3(pfirst - 1), ip, false, true, unused0, c1m);
        plane_sums(mod3(pfirst), ip, true, true, c0, c1);
    }
    T cur[10], nxt[10];
    for (int p = pfirst; p <= z1; ++p) {
        if (!perz && p == nz) {
            fill_z(nz);
        } else {
            // one barrier publishes plane p + 1's primitives and carries the
            // time-out agreement
            if (__syncthreads_or(!fetch(p + 1))) { drain(); timed_out(); return false; }
            predict(p, nxt);
            __syncthreads();
            issue_upto(min(p + 2, zlast));
            fill_xy(p);
        }
        if (zero && p == 1) fill_z(-1);
        if (p - 1 >= z0) correct(p - 1, cur);
#pragma unroll
        for (int e = 0; e < 10; ++e) cur[e] = nxt[e];
        // no barrier here: the next shared-memory write that correct's reads
        // depend on (convert and predict of the next plane, or fill_z) follows
        // the next fetch's barrier or fill_z's leading one
    }
    return true;
}

}  // namespace cspht

#include "lagrange_pair.cuh"

namespace cspht {

// Dynamic shared memory of the Lagrangian kernels of precision T.
template <int TX, int TY>
template <typename T>
__host__ __device__ constexpr size_t LagShape<TX, TY>::bytes() {
    if constexpr (sizeof(T) == 4) return LagPair<TX, TY>::BYTES;
    else return smem_bytes<T>();
}

// The Lagrangian stage of one grid: one CTA per tile and z chunk (FP32: the
// paired tile).
template <typename T, int TX, int TY, bool COMP = false>
__global__ void __launch_bounds__(LagShape<TX, TY>::template threads<T>(), sizeof(T) == 4 ? 3 : 1)
    k_lagrange(const __grid_constant__ LagArgs<T> A) {
    uint32_t phase_bits = 0;
    if constexpr (sizeof(T) == 4)
        lagrange_tile_pair<TX, TY, COMP, true>(A, blockIdx.x, blockIdx.y, blockIdx.z, phase_bits);
    else
        lagrange_tile<T, TX, TY, COMP, true>(A, blockIdx.x, blockIdx.y, blockIdx.z, phase_bits);
}

// Work item of the multi-grid kernels: grid (member) index and tile (bx, by, bz).
struct TileItem {
    int member, bx, by, bz;
};

// The arguments of a group of grids, passed as one kernel parameter (kernel
// parameters may take about 32 KB): the tile bodies then read every field
// from the constant bank, as the one-grid kernels do, instead of holding
// what they read from global memory in registers.
template <typename T, template <int> class Maps>
struct EulArgs;
constexpr int GROUP_PARAM_BYTES = 30000;
template <typename T>
constexpr int group_size() {
    const int a = GROUP_PARAM_BYTES / (int)sizeof(LagArgs<T, MapsAt>),
              b = GROUP_PARAM_BYTES / (int)sizeof(EulArgs<T, MapsAt>);
    return a < b ? a : b;
}
template <typename T>
struct LagGroup {
    LagArgs<T, MapsAt> a[group_size<T>()];
};

// The Lagrangian stage of a group of grids in one launch: a persistent CTA
// takes tile items from a device counter until the group's list is done (the
// list is ordered by decreasing work); every grid has its own dt.
template <typename T, int TX, int TY, bool COMP = false>
__global__ void __launch_bounds__(LagShape<TX, TY>::template threads<T>(), sizeof(T) == 4 ? 3 : 1)
    k_lagrange_multi(const __grid_constant__ LagGroup<T> g, const TileItem *__restrict__ items, int nitems,
                     int *__restrict__ next) {
    const LagArgs<T, MapsAt> *args = g.a;
    if constexpr (sizeof(T) == 4) {
        if (!lagrange_pair_begin<TX, TY>(args[items[0].member].ctrl)) return;
    } else {
        if (!lagrange_begin<T, TX, TY>(args[items[0].member].ctrl)) return;
    }
    __shared__ int s_item;
    uint32_t phase_bits = 0;
    for (;;) {
        __syncthreads();  // the previous tile's readers of shared memory are done
        if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const TileItem w = items[it];
        bool ok;
        if constexpr (sizeof(T) == 4)
            ok = lagrange_tile_pair<TX, TY, COMP, false>(args[w.member], w.bx, w.by, w.bz, phase_bits);
        else
            ok = lagrange_tile<T, TX, TY, COMP, false>(args[w.member], w.bx, w.by, w.bz, phase_bits);
        if (!ok) break;
    }
}

// ============================================================== Eulerian stage

template <typename T, template <int> class Maps = MapsIn>
struct EulArgs {
    Maps<5> tmU;   // U^n fields, box TX+8 x TY+4 x 1 at (x0-4, y0-2)
    Maps<6> tmS;   // m~x, m~y, m~z, E~, xi_x, xi_y, box TX+8 x TY+2 x 1 at (x0-4, y0-1)
    Grid G;
    Phys<T> P;
    const T *U[5];
    const T *m[3];
    const T *E;
    const T *xi[3];
    T *Un[5];
    T *rho_lo;  // FP32 only: density compensation word (rho = rho_hi + rho_lo), or null
    Ctrl *ctrl;
    int zchunk;
};

template <int TX, int TY>
struct EulShape {
    static constexpr int BW = TX + 8, BH = TY + 4, NB = BW * BH;   // U box
    static constexpr int SH = TY + 2, NS = BW * SH;                // corrector-state box
    static constexpr int PX = TX + 2, PY = TY + 2, NP = PX * PY;   // half-step state, halo 1
    static constexpr int NT = TX * TY;
    static constexpr int NFX = (TX + 1) * TY, NFY = TX * (TY + 1); // in-plane faces of the tile
    static constexpr int SLOTS = 2;
    template <typename T>
    __host__ __device__ static constexpr int slot_width() {  // one plane's boxes, each on a 128-byte boundary
        return 5 * tma_slot<T>(NB) + 6 * tma_slot<T>(NS);
    }
    template <typename T>
    __host__ __device__ static constexpr size_t smem_bytes() {
        // TMA ring (U 5 + state 6 per slot); per NP position U^{n+1/2}, theta_x, theta_y (5 each);
        // Courant fluxes of the x and y faces (5 each); barriers
        return sizeof(T) * ((size_t)SLOTS * slot_width<T>() + 15 * (size_t)NP +
                            5 * (size_t)(NFX + NFY)) + 64;
    }
};

// Limited slope in difference units (the oracle's slope times h).
// Branch-free: the limited value is formed unconditionally and selected (a
// zero denominator when ab <= 0 gives inf or NaN, which the select drops).
template <typename T, int LIM>
__device__ __forceinline__ T slope_d(T dp, T dm) {
    const T ab = dp * dm;
    T v;
    if (LIM == LIM_MINMOD) {
        v = fabs(dp) < fabs(dm) ? dp : dm;
    } else if (LIM == LIM_MC) {
        T m = fabs(T(2) * dp);
        if (fabs(T(2) * dm) < m) m = fabs(T(2) * dm);
        if (fabs(T(0.5) * (dp + dm)) < m) m = fabs(T(0.5) * (dp + dm));
        v = dp > T(0) ? m : -m;
    } else {
        // dp + dm is subnormal only if both are, and then ab = 0 drops v
        v = T(2) * ab * f_rcp_n(dp + dm);
    }
    return ab > T(0) ? v : T(0);
}

// Signal speed max_d |u_d| + c of an updated cell (0 for vacuum) in the
// kernel's precision: FP32 with the SFU reciprocal and square root, FP64 as
// the unfused path computes it.
template <typename T>
__device__ __forceinline__ T signal_speed_t(const Phys<T> &P, T rho, T mx, T my, T mz, T E) {
    if constexpr (sizeof(T) == 8) {
        return signal_speed(P, rho, mx, my, mz, E);
    } else {
        if (!(rho > P.rho_vac)) return T(0);
        const T ir = f_rcp_n(rho);
        const T u = mx * ir, v = my * ir, w = mz * ir;
        T p = P.gm1 * (E - T(0.5) * (mx * u + my * v + mz * w));
        if (p < T(0)) p = T(0);
        const T um = fmaxf(fabsf(u), fmaxf(fabsf(v), fabsf(w)));
        return um + f_sqrt_n(P.gamma * p * ir);
    }
}


// Eq. 8 face states: U_L = H_L + (1 - c_L)/2 Theta_L, U_R = H_R - (1 + c_R)/2 Theta_R.
template <typename T>
__device__ __forceinline__ T rec_L(T H, T th, T c) { return r_fma(r_mul(T(0.5), r_sub(T(1), c)), th, H); }
template <typename T>
__device__ __forceinline__ T rec_R(T H, T th, T c) { return r_fma(-r_mul(T(0.5), r_add(T(1), c)), th, H); }

// Courant-scaled Riemann flux G = (dt/h) F of one face with face "speeds"
// cL, cR = xi^ (F_L = cL U_L, F_R = cR U_R), written as G = a U_L + b U_R:
// the weights (a, b) depend on the face only and serve its five fields.
//   LF:    G = (F_L + F_R)/2 - s (U_R - U_L)/2, s = max(|cL|, |cR|):
//          a = (cL + s)/2, b = (cR - s)/2.
//   HLL:   wave speeds SL = min(cL, cR), SR = max(cL, cR); G = F_L if SL >= 0,
//          F_R if SR <= 0, else (SR F_L - SL F_R + SL SR (U_R - U_L)) / (SR - SL),
//          which between the speeds is F_L + F_R if cL > cR (SL = cR, SR = cL)
//          and 0 if cL < cR (SL = cL, SR = cR).
//   swept: c = (cL + cR)/2 carries the upwind state.
template <typename T>
struct FluxW {
    T a, b;
};
template <typename T, int RK>
__device__ __forceinline__ FluxW<T> flux_w(T cL, T cR) {
    if (RK == RIEMANN_HLL) {
        if (cL >= T(0) && cR >= T(0)) return {cL, T(0)};
        if (cL <= T(0) && cR <= T(0)) return {T(0), cR};
        return cL > cR ? FluxW<T>{cL, cR} : FluxW<T>{T(0), T(0)};
    }
    if (RK == RIEMANN_SWEPT) {
        const T c = r_mul(T(0.5), r_add(cL, cR));
        return c >= T(0) ? FluxW<T>{c, T(0)} : FluxW<T>{T(0), c};
    }
    const T s = fabs(cL) > fabs(cR) ? fabs(cL) : fabs(cR);
    return {r_mul(T(0.5), r_add(cL, s)), r_mul(T(0.5), r_sub(cR, s))};
}
template <typename T>
__device__ __forceinline__ T flux_c(const FluxW<T> &w, T UL, T UR) { return r_fma(w.a, UL, r_mul(w.b, UR)); }


__device__ __forceinline__ bool finite_t(float v) { return isfinite(v); }
__device__ __forceinline__ bool finite_t(double v) { return isfinite(v); }

// Start of a CTA of the Eulerian kernels: initialises the copy barriers and
// checks that every copy destination starts on a 128-byte boundary (false, and
// the time-out status bit, if one does not).
template <typename T, int TX, int TY>
__device__ __forceinline__ bool euler_begin(Ctrl *ctrl) {
    using S = EulShape<TX, TY>;
    constexpr int NB = tma_slot<T>(S::NB), NS = tma_slot<T>(S::NS), NP = S::NP, NT = S::NT;
    constexpr int SLOTW = S::template slot_width<T>();
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sbox = reinterpret_cast<T *>(smem_raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sbox + S::SLOTS * SLOTW + 15 * NP + 5 * (S::NFX + S::NFY));
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int q = 0; q < S::SLOTS; ++q) mbar_init(&bar[q], 1);
        mbar_init_fence();
    }
    bool misaligned = false;
    for (int q = tid; q < S::SLOTS * 11; q += NT) {
        const int sl = q / 11, f = q % 11;
        const T *d = sbox + sl * SLOTW + (f < 5 ? f * NB : 5 * NB + (f - 5) * NS);
        misaligned |= (smem_u32(d) & 127u) != 0;
    }
    if (__syncthreads_or(misaligned)) {
        if (tid == 0) atomicOr(&ctrl->status, ST_TIMEOUT);
        return false;
    }
    return true;
}

// One tile of the Eulerian stage: tile (bx, by) over z chunk bz.  INIT: the
// tile is the CTA's only one and initialises the copy barriers itself;
// otherwise euler_begin did.  phase_bits carries the barriers' parities from
// one tile of the CTA to the next.  Returns false after a copy time-out or a
// misaligned copy destination: the CTA must not start another tile.
template <typename T, int TX, int TY, int LIM, int RK, bool INIT, class Args>
__device__ __forceinline__ bool euler_tile(const Args &A, const int bx, const int by, const int bz,
                                           uint32_t &phase_bits) {
    using S = EulShape<TX, TY>;
    // NB, NS: box slot strides (128-byte multiples); S::NB, S::NS: box sizes
    constexpr int BW = S::BW, NB = tma_slot<T>(S::NB), NS = tma_slot<T>(S::NS), PX = S::PX,
                  NP = S::NP, NT = S::NT;
    constexpr int NFX = S::NFX, NFY = S::NFY;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    T *sbox = reinterpret_cast<T *>(smem_raw);        // [SLOTS][5*NB + 6*NS]
    constexpr int SLOTW = S::template slot_width<T>();
    T *sH = sbox + S::SLOTS * SLOTW;                  // [5][NP] U^{n+1/2}
    T *sTx = sH + 5 * NP;                             // [5][NP] theta_x
    T *sTy = sTx + 5 * NP;                            // [5][NP] theta_y
    T *sGx = sTy + 5 * NP;                            // [5][NFX] G on x faces (x = tile column - 1/2)
    T *sGy = sGx + 5 * NFX;                           // [5][NFY] G on y faces
    uint64_t *bar = reinterpret_cast<uint64_t *>(sGy + 5 * NFY);

    const Grid &G = A.G;
    const Phys<T> &P = A.P;
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const bool perx = P.bc[0] == BC_PERIODIC, pery = P.bc[2] == BC_PERIODIC,
               perz = P.bc[4] == BC_PERIODIC;
    const int tid = threadIdx.x, tx = tid % TX, ty = tid / TX;
    const int x0 = bx * TX, y0 = by * TY;
    const int z0 = bz * A.zchunk, z1 = min(z0 + A.zchunk, nz);
    const int gx = x0 + tx, gy = y0 + ty;
    const bool own = gx < nx && gy < ny;
    const T dt = (T)A.ctrl->dt;
    const T inv_h = P.inv_h;
    T smax = T(0);  // largest signal speed of the CTA's updated cells (a NaN sticks)
    int st = 0;
    __shared__ int s_colx[S::PX + 2], s_rowy[S::PY + 2];  // columns x0-2.., rows y0-2..
    for (int t = tid; t < PX + 2; t += NT) s_colx[t] = map_coord(x0 - 2 + t, nx, perx) + G.ox;
    for (int t = tid; t < S::PY + 2; t += NT) s_rowy[t] = (map_coord(y0 - 2 + t, ny, pery) + GH) * G.px;
    if constexpr (INIT) {
        if (tid == 0) {
            for (int q = 0; q < S::SLOTS; ++q) mbar_init(&bar[q], 1);
            mbar_init_fence();
        }
        // every TMA destination must start on a 128-byte boundary: refuse to run otherwise
        bool misaligned = false;
        for (int q = tid; q < S::SLOTS * 11; q += NT) {
            const int sl = q / 11, f = q % 11;
            const T *d = sbox + sl * SLOTW + (f < 5 ? f * NB : 5 * NB + (f - 5) * NS);
            misaligned |= (smem_u32(d) & 127u) != 0;
        }
        if (__syncthreads_or(misaligned)) {  // also publishes the offsets read below
            if (tid == 0) atomicOr(&A.ctrl->status, ST_TIMEOUT);
            return false;
        }
    } else {
        __syncthreads();  // the column and row offsets are read below
    }
    auto zoff = [&](int gz) { return (map_coord(gz, nz, perz) + GH) * (int)G.plane; };
    const int own_xy = s_rowy[ty + 2] + s_colx[tx + 2];  // own column (clamped when ragged)

    if (!(dt > T(0))) {  // zero step: copy U^n
        if (own)
            for (int k = z0; k < z1; ++k) {
                const int c = (k + GH) * (int)G.plane + own_xy;
                T v[5];
                for (int f = 0; f < 5; ++f) A.Un[f][c] = v[f] = A.U[f][c];
                const T sp = signal_speed_t(P, v[0], v[1], v[2], v[3], v[4]);
                if (!(sp <= smax)) smax = sp;
            }
        block_max_to(&A.ctrl->smax_next, (double)smax);
        return true;
    }

    const int spin = A.ctrl->spin_limit > 0 ? A.ctrl->spin_limit : MBAR_SPIN_LIMIT;
    const bool no_copies = (A.ctrl->inject & INJECT_NO_COPIES) != 0;
    const bool wall_x0 = P.bc[0] == BC_WALL, wall_x1 = P.bc[1] == BC_WALL;
    const bool wall_y0 = P.bc[2] == BC_WALL, wall_y1 = P.bc[3] == BC_WALL;
    const bool wz_lo = P.bc[4] == BC_WALL, wz_hi = P.bc[5] == BC_WALL;

    // ---- TMA ring of planes: slot k mod 2 holds U^n(k) and the corrector state (k);
    // phase_bits: parity of the next completion, per slot
    auto issue = [&](int k) {
        if (tid == 0) {
            const int sl = k & 1;
            fence_proxy_async();
            mbar_arrive_expect_tx(&bar[sl], (uint32_t)((5 * S::NB + 6 * S::NS) * sizeof(T)));
            const int zc = map_coord(k, nz, perz) + GH;
            T *b = sbox + sl * SLOTW;
            if (!no_copies) {
                for (int f = 0; f < 5; ++f)
                    tma_load_3d(b + f * NB, A.tmU.at(f), x0 - 4 + G.ox, y0 - 2 + GH, zc, &bar[sl]);
                for (int f = 0; f < 6; ++f)
                    tma_load_3d(b + 5 * NB + f * NS, A.tmS.at(f), x0 - 4 + G.ox, y0 - 1 + GH, zc, &bar[sl]);
            }
        }
    };
    // Waits in this thread (bounded) for plane k's boxes; false on a time-out.
    // No barrier: the barrier before the face phase lets every thread agree on
    // a time-out before anything is written.
    auto arrive = [&](int k) -> bool {
        const int sl = k & 1;
        const bool ok = mbar_wait(&bar[sl], (phase_bits >> sl) & 1u, spin);
        if (ok) phase_bits ^= 1u << sl;
        return ok;
    };

    // own-column values along z: U^n, U^{n+1/2}, xi^_z (plain loads)
    auto colU = [&](int k, T u[5]) {
        const int c = zoff(k) + own_xy;
        for (int f = 0; f < 5; ++f) u[f] = A.U[f][c];
    };
    auto colS = [&](int k, T sv[5]) {  // m~x, m~y, m~z, E~, xi_z
        const int c = zoff(k) + own_xy;
        for (int e = 0; e < 3; ++e) sv[e] = A.m[e][c];
        sv[3] = A.E[c];
        sv[4] = A.xi[2][c];
    };
    auto half = [&](const T u[5], const T sv[5], T hh[5], T &xz) {
        hh[0] = u[0];
        for (int e = 0; e < 3; ++e) hh[1 + e] = T(0.5) * (u[1 + e] + sv[e]);
        hh[4] = T(0.5) * (u[4] + sv[3]);
        xz = sv[4] * inv_h;
    };
    // z slope at cell k of the column (0 at non-periodic z ghosts)
    auto zslope = [&](int k, const T um[5], const T u0[5], const T up[5], T th[5]) {
        const bool ghost = (k < 0 || k >= nz) && !perz;
        for (int f = 0; f < 5; ++f) th[f] = ghost ? T(0) : slope_d<T, LIM>(up[f] - u0[f], u0[f] - um[f]);
    };

    issue(z0);
    if (z0 + 1 < z1) issue(z0 + 1);

    // z window: U at k, k+1; state at k; theta_z at k; flux through k - 1/2
    T U0[5], U1[5], H0[5], T0[5], xz0, Gzm[5];
    {
        T Um[5], Up[5], sv[5], Hm[5], Tm[5], xzm;
        colU(z0 - 2, Um);
        colU(z0 - 1, U0);
        colU(z0, U1);
        colU(z0 + 1, Up);
        zslope(z0 - 1, Um, U0, U1, Tm);
        colS(z0 - 1, sv);
        half(U0, sv, Hm, xzm);
        zslope(z0, U0, U1, Up, T0);
        colS(z0, sv);
        half(U1, sv, H0, xz0);
        const bool wall = wz_lo && z0 == 0;
        const FluxW<T> fw = flux_w<T, RK>(xzm, xz0);
        for (int f = 0; f < 5; ++f) {
            const T UL = rec_L(Hm[f], Tm[f], xzm);
            const T UR = rec_R(H0[f], T0[f], xz0);
            Gzm[f] = wall ? T(0) : flux_c(fw, UL, UR);
            U0[f] = U1[f];  // now U0 = U(z0), U1 = U(z0+1)
            U1[f] = Up[f];
        }
    }
    // prefetched own-column values for the next face: U(k+2) and the state at k+1
    T pU[5], pS[5];
    colU(z0 + 2, pU);
    colS(z0 + 1, pS);

    for (int k = z0; k < z1; ++k) {
        // the own cell's density compensation word, loaded ahead of its use
        float lo_k = 0.0f;
        if constexpr (sizeof(T) == 4)
            if (A.rho_lo && own) lo_k = A.rho_lo[(k + GH) * (int)G.plane + own_xy];
        const bool arrived = arrive(k);  // a time-out is acted on at the barrier before the faces
        const T *bU = sbox + (k & 1) * SLOTW;  // U^n box of plane k
        const T *bS = bU + 5 * NB;             // corrector-state box of plane k
        // ---- half-step state and in-plane slopes on the tile + 1 halo: the
        // first NT positions one per thread with every field, the other NP - NT
        // field by field over all threads (the field index slowest, so that a
        // warp reads neighbouring positions), which evens out the phase
        auto slope_at_field = [&](const int t, const int f) {
            const int px = t % PX, py = t / PX;
            const int cx = x0 - 1 + px, cy = y0 - 1 + py;
            const int bu = (py + 1) * BW + px + 3, bs = py * BW + px + 3;
            const T *uf = bU + f * NB + bu;
            const T u = uf[0];
            const T sv = bS[(f > 0 ? f - 1 : 0) * NS + bs];  // m~ (f = 1..3) or E~ (f = 4)
            sH[f * NP + t] = f == 0 ? u : T(0.5) * (u + sv);
            const bool gxs = (cx < 0 || cx >= nx) && !perx, gys = (cy < 0 || cy >= ny) && !pery;
            sTx[f * NP + t] = gxs ? T(0) : slope_d<T, LIM>(uf[1] - u, u - uf[-1]);
            sTy[f * NP + t] = gys ? T(0) : slope_d<T, LIM>(uf[BW] - u, u - uf[-BW]);
        };
        static_assert(NP >= NT && 5 * (NP - NT) <= 2 * NT, "slope phase: one position per thread, then <= 2 units");
#pragma unroll
        for (int f = 0; f < 5; ++f) slope_at_field(tid, f);
        for (int u = tid; u < 5 * (NP - NT); u += NT) slope_at_field(NT + u % (NP - NT), u / (NP - NT));
        // ---- own column, z: cell k+1 state, face k + 1/2 (from the prefetch)
        T Gzp[5], T1[5], H1[5], xz1;
        zslope(k + 1, U0, U1, pU, T1);
        half(U1, pS, H1, xz1);
        {
            const bool wall = wz_hi && k == nz - 1;
            const FluxW<T> fw = flux_w<T, RK>(xz0, xz1);
            for (int f = 0; f < 5; ++f) {
                const T UL = rec_L(H0[f], T0[f], xz0);
                const T UR = rec_R(H1[f], T1[f], xz1);
                Gzp[f] = wall ? T(0) : flux_c(fw, UL, UR);
            }
        }
        const T Unext[5] = {pU[0], pU[1], pU[2], pU[3], pU[4]};
        if (k + 1 < z1) {  // prefetch for the next iteration
            colU(k + 3, pU);
            colS(k + 2, pS);
        }
        // the own cell's corrector state, read now so that slot k is free after the face barrier
        T base[5];
        {
            const int bs = (ty + 1) * BW + tx + 4;
            base[0] = U0[0];
            for (int e = 0; e < 4; ++e) base[1 + e] = bS[e * NS + bs];
        }
        if (__syncthreads_or(!arrived)) {  // time-out: wait (bounded) for the other box in flight, then leave
            if (tid == 0) atomicOr(&A.ctrl->status, ST_TIMEOUT);
            if (k + 1 < z1) mbar_wait(&bar[(k + 1) & 1], (phase_bits >> ((k + 1) & 1)) & 1u, spin);
            return false;
        }
        // ---- in-plane faces, each once: every thread takes the x face left of
        // its cell and the y face below it; threads 0..TY-1 also take the x face
        // right of the tile's last column (row tid), threads TY..TY+TX-1 the
        // y face above the tile's last row (column tid - TY).
        auto face = [&](const bool isx, const int fx, const int fy) {
            int pL, pR, ixL, ixR, cc, stride;
            bool wall;
            const T *Th;
            T *Gout;
            if (isx) {  // between tile columns fx-1 and fx of row fy
                cc = x0 + fx;
                pL = (fy + 1) * PX + fx;
                pR = pL + 1;
                ixL = 4 * NS + (fy + 1) * BW + fx + 3;
                ixR = ixL + 1;
                wall = (cc == 0 && wall_x0) || (cc == nx && wall_x1);
                Th = sTx;
                Gout = sGx + fy * (TX + 1) + fx;
                stride = NFX;
            } else {  // between tile rows fy-1 and fy of column fx
                cc = y0 + fy;
                pL = fy * PX + fx + 1;
                pR = pL + PX;
                ixL = 5 * NS + fy * BW + fx + 4;
                ixR = ixL + BW;
                wall = (cc == 0 && wall_y0) || (cc == ny && wall_y1);
                Th = sTy;
                Gout = sGy + fy * TX + fx;
                stride = NFY;
            }
            const T cL = bS[ixL] * inv_h, cR = bS[ixR] * inv_h;
            const FluxW<T> fw = flux_w<T, RK>(cL, cR);
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                const T UL = rec_L(sH[f * NP + pL], Th[f * NP + pL], cL);
                const T UR = rec_R(sH[f * NP + pR], Th[f * NP + pR], cR);
                Gout[f * stride] = wall ? T(0) : flux_c(fw, UL, UR);
            }
        };
        face(true, tx, ty);
        face(false, tx, ty);
        static_assert(NT >= TX + TY, "one thread per edge face");
        if (tid < TY) face(true, TX, tid);
        else if (tid < TY + TX) face(false, tid - TY, TY);
        __syncthreads();
        // slot k (read by the slope and face phases above) is free: fetch plane k+2 into it
        if (k + 2 < z1) issue(k + 2);
        // ---- update of the own cell (Eq. 4 in Courant units)
        if (own) {
            const int c = (k + GH) * (int)G.plane + own_xy;
            const int ix0 = ty * (TX + 1) + tx, iy0 = ty * TX + tx;
            T v[5];
#pragma unroll
            for (int f = 0; f < 5; ++f) {
                const T div = (Gzp[f] - Gzm[f]) + (sGx[f * NFX + ix0 + 1] - sGx[f * NFX + ix0]) +
                              (sGy[f * NFY + iy0 + TX] - sGy[f * NFY + iy0]);
                v[f] = base[f] - div;
            }
            if constexpr (sizeof(T) == 4) {
                if (A.rho_lo) {
                    // Compensated mass update: every face flux enters two cells with the
                    // same bits, and the six terms are summed without rounding loss, so
                    // the total mass changes only by the boundary fluxes.
                    float e = lo_k, err;
                    float sm = base[0];
                    const float terms[6] = {-Gzp[0], Gzm[0], -sGx[ix0 + 1], sGx[ix0], -sGy[iy0 + TX], sGy[iy0]};
#pragma unroll
                    for (int q = 0; q < 6; ++q) {
                        sm = two_sum(sm, terms[q], err);
                        e = __fadd_rn(e, err);
                    }
                    const float hi = __fadd_rn(sm, e);
                    A.rho_lo[c] = __fsub_rn(e, __fsub_rn(hi, sm));
                    v[0] = hi;
                }
            }
            for (int f = 0; f < 5; ++f) {
                A.Un[f][c] = v[f];
                if (!finite_t(v[f])) st |= ST_NONFINITE;
            }
            if (v[0] < T(0)) st |= ST_NEGATIVE;
            const T sp = signal_speed_t(P, v[0], v[1], v[2], v[3], v[4]);
            if (!(sp <= smax)) smax = sp;  // keeps a NaN
        }
        // ---- advance the z window
        for (int f = 0; f < 5; ++f) {
            Gzm[f] = Gzp[f];
            U0[f] = U1[f];
            U1[f] = Unext[f];
            H0[f] = H1[f];
            T0[f] = T1[f];
        }
        xz0 = xz1;
        // no barrier here: every thread passed this iteration's second barrier,
        // so the face phase's reads of sH/sTx/sTy are done before the next slope
        // phase rewrites them, and sGx/sGy are rewritten only after the next
        // iteration's first barrier
    }
    if (st) atomicOr(&A.ctrl->status, st);
    block_max_to(&A.ctrl->smax_next, (double)smax);
    return true;
}

// The Eulerian stage of one grid: one CTA per tile and z chunk.
template <typename T, int TX, int TY, int LIM, int RK>
__global__ void __launch_bounds__(TX *TY, sizeof(T) == 4 ? 3 : 1)
    k_euler(const __grid_constant__ EulArgs<T> A) {
    uint32_t phase_bits = 0;
    euler_tile<T, TX, TY, LIM, RK, true>(A, blockIdx.x, blockIdx.y, blockIdx.z, phase_bits);
}

template <typename T>
struct EulGroup {
    EulArgs<T, MapsAt> a[group_size<T>()];
};

// The Eulerian stage of a group of grids in one launch (persistent CTAs
// taking tile items from a device counter; see k_lagrange_multi).
template <typename T, int TX, int TY, int LIM, int RK>
__global__ void __launch_bounds__(TX *TY, sizeof(T) == 4 ? 3 : 1)
    k_euler_multi(const __grid_constant__ EulGroup<T> g, const TileItem *__restrict__ items, int nitems,
                  int *__restrict__ next) {
    const EulArgs<T, MapsAt> *args = g.a;
    if (!euler_begin<T, TX, TY>(args[items[0].member].ctrl)) return;
    __shared__ int s_item;
    uint32_t phase_bits = 0;
    for (;;) {
        __syncthreads();  // the previous tile's readers of shared memory are done
        if (threadIdx.x == 0) s_item = atomicAdd(next, 1);
        __syncthreads();
        const int it = s_item;
        if (it >= nitems) break;
        const TileItem w = items[it];
        if (!euler_tile<T, TX, TY, LIM, RK, false>(args[w.member], w.bx, w.by, w.bz, phase_bits)) break;
    }
}

}  // namespace cspht
