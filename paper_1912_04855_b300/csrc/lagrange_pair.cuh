// The Lagrangian stage in FP32 with two columns per thread (included by fast.cuh).
//
// Same method and stage order as lagrange_tile (Eqs. 5-7: predictor from the
// static-lattice plane sums, corrector over the displaced pairs), laid out for
// the packed FP32 instructions of sm_100+: a thread of a 32 x 8 tile owns the
// columns x and x + 16 of one row, and every per-particle quantity of the two
// is stored side by side, so that one packed add, multiply or fma serves both.
// The arithmetic of a particle is the same in either lane, so a particle
// stored twice (columns 16..19 of the primitives region, 16..17 of the
// predictor region) or computed by two tiles or chunks carries the same bits
// everywhere.
//
// Shared memory (32 x 8 tile, 76.4 KB):
//   raw U^n boxes    2 slots x 5 fields x 40 x 12 floats   (TMA destinations)
//   U^n primitives   3 planes x 12 rows x 20 pair positions (row stride 21)
//                    x 2 float4: (u, v), (w, phi)
//   predictor state  3 planes x 10 rows x 18 pair positions x (3 float4 + float2):
//                    (u*, v*), (w*, phi*), (xi*_x, xi*_y), xi*_z  (xi* in cell units)
//   densities        2 planes x 34 x 10 particles (the corrector's and the
//                    boundary rules' rho)
// Pair position (c, row) holds the columns c and c + 16 of the region.

namespace cspht {

// ---- packed FP32: round-to-nearest, never contracted or reordered
__device__ __forceinline__ float2 p2(float a) { return make_float2(a, a); }
__device__ __forceinline__ float2 add2(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 sub2(float2 a, float2 b) { return __fadd2_rn(a, make_float2(-b.x, -b.y)); }
__device__ __forceinline__ float2 mul2(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 fma2(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 neg2(float2 a) { return make_float2(-a.x, -a.y); }
__device__ __forceinline__ float2 lo2(float4 a) { return make_float2(a.x, a.y); }
__device__ __forceinline__ float2 hi2(float4 a) { return make_float2(a.z, a.w); }
__device__ __forceinline__ float4 cat2(float2 a, float2 b) { return make_float4(a.x, a.y, b.x, b.y); }
__device__ __forceinline__ float2 sel2(bool kx, bool ky, float2 a, float2 b) {
    return make_float2(kx ? a.x : b.x, ky ? a.y : b.y);
}

// Shared-memory layout of the paired FP32 tile (byte offsets).
template <int TX, int TY>
struct LagPair {
    static_assert(TX % 2 == 0 && TX / 2 >= 4, "column pairs x, x + TX/2");
    static constexpr int HX = TX / 2;                         // column pair offset
    static constexpr int BW = TX + 8, BH = TY + 4, NB = BW * BH;  // TMA box: x0-4.., y0-2..
    static constexpr int RAWF = tma_slot<float>(NB);          // box slot stride (floats)
    static constexpr int IX = TX + 4, IY = TY + 4;            // U^n primitives (halo 2)
    static constexpr int ICP = IX - HX, NIQ = ICP * IY;       // their pair columns / positions
    static constexpr int ICS = ICP | 1;                       // row stride: odd, so that rows
                                                              // fall on different bank groups
    static constexpr int PX = TX + 2, PY = TY + 2;            // predictor particles (halo 1)
    static constexpr int PCP = PX - HX, NPQ = PCP * PY;       // their pair columns / positions
    static constexpr int NT = TX * TY / 2;                    // threads: two cells each
    static constexpr int NHT = NPQ - NT;                      // halo pair positions
    static_assert(NHT == 2 * PCP + 2 * TY, "the halo ring: two rows, two pair columns");
    // halo tasks: each row and each pair column starts on a multiple of 8
    // threads (a quarter warp: one shared-memory phase of 16-byte loads)
    static constexpr int R8 = (PCP + 7) / 8 * 8, C8 = (TY + 7) / 8 * 8;
    static constexpr int NHL = 2 * R8 + 2 * C8;               // threads of the halo pass
    static_assert(NHL <= NT, "one halo task per thread");
    static constexpr int SLOTS = 2;
    static constexpr size_t OFF_UA = (size_t)SLOTS * 5 * RAWF * 4;
    static constexpr size_t OFF_UB = OFF_UA + 3 * (size_t)ICS * IY * 16;
    static constexpr size_t OFF_PA = OFF_UB + 3 * (size_t)ICS * IY * 16;
    static constexpr size_t OFF_PB = OFF_PA + 3 * (size_t)NPQ * 16;
    static constexpr size_t OFF_PC = OFF_PB + 3 * (size_t)NPQ * 16;
    static constexpr size_t OFF_PD = OFF_PC + 3 * (size_t)NPQ * 16;
    static constexpr size_t OFF_RHO = OFF_PD + 3 * (size_t)NPQ * 8;  // [2][PX * PY] U^n density
    static constexpr size_t OFF_BAR = OFF_RHO + 2 * (size_t)PX * PY * 4;
    static constexpr size_t BYTES = OFF_BAR + 64;
    static_assert(OFF_UA % 128 == 0 && OFF_BAR % 8 == 0, "alignment");
};

// Packed primitive recovery (eos_fast per lane): vacuum lanes give zeros.
struct Prim2 {
    float2 u, v, w, phi;
};
__device__ __forceinline__ Prim2 eos2(const Phys<float> &P, float2 rho, float2 mx, float2 my, float2 mz, float2 E) {
    const bool gx = rho.x > P.rho_vac, gy = rho.y > P.rho_vac;
    // rho > rho_vac >= 2^-126 in a gas lane: a normal number
    const float2 ir = make_float2(gx ? f_rcp_n(rho.x) : 0.0f, gy ? f_rcp_n(rho.y) : 0.0f);
    Prim2 r;
    r.u = mul2(mx, ir);
    r.v = mul2(my, ir);
    r.w = mul2(mz, ir);
    const float2 ke = fma2(mx, r.u, fma2(my, r.v, mul2(mz, r.w)));  // |m|^2 / rho
    float2 p = mul2(p2(P.gm1), fma2(p2(-0.5f), ke, E));
    p.x = p.x > 0.0f ? p.x : 0.0f;
    p.y = p.y > 0.0f ? p.y : 0.0f;
    r.phi = make_float2(gx ? f_sqrt_n(2.0f * p.x) : 0.0f, gy ? f_sqrt_n(2.0f * p.y) : 0.0f);
    return r;
}

// Packed balance -(a b) - c d (see balance): plain, or with both products
// exact and one rounding of their sum (COMP).
template <bool COMP>
__device__ __forceinline__ float2 balance2(float2 a, float2 b, float2 c, float2 d) {
    if constexpr (COMP) {
        const float2 p = mul2(a, b), pe = fma2(a, b, neg2(p));
        const float2 q = mul2(c, d), qe = fma2(c, d, neg2(q));
        const float2 s = sub2(neg2(p), q);           // -p - q
        const float2 bb = add2(s, p);                // s - (-p)
        const float2 err = add2(sub2(neg2(p), sub2(s, bb)), sub2(neg2(q), bb));
        return add2(s, sub2(sub2(err, pe), qe));
    } else {
        return fma2(neg2(a), b, neg2(mul2(c, d)));
    }
}


// Start of a CTA of the paired kernels: barriers and the alignment check of
// every copy destination (as lagrange_begin).
template <int TX, int TY>
__device__ __forceinline__ bool lagrange_pair_begin(Ctrl *ctrl) {
    using S = LagPair<TX, TY>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *sraw = reinterpret_cast<float *>(smem_raw);
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + S::OFF_BAR);
    const int tid = threadIdx.x;
    if (tid == 0) {
        for (int q = 0; q < S::SLOTS; ++q) mbar_init(&bar[q], 1);
        mbar_init_fence();
    }
    bool misaligned = false;
    for (int q = tid; q < S::SLOTS * 5; q += S::NT) misaligned |= (smem_u32(sraw + q * S::RAWF) & 127u) != 0;
    if (__syncthreads_or(misaligned)) {
        if (tid == 0) atomicOr(&ctrl->status, ST_TIMEOUT);
        return false;
    }
    return true;
}

// One tile of the Lagrangian stage in FP32, two columns per thread: the
// TX x TY columns of tile (bx, by) over z chunk bz.  Arguments, INIT and
// phase_bits as lagrange_tile.
template <int TX, int TY, bool COMP, bool INIT, class Args>
__device__ __forceinline__ bool lagrange_tile_pair(const Args &A, const int bx, const int by, const int bz,
                                                   uint32_t &phase_bits) {
    using S = LagPair<TX, TY>;
    constexpr int BW = S::BW, RAWF = S::RAWF, HX = S::HX, IX = S::IX, ICP = S::ICP, NIQ = S::NIQ,
                  ICS = S::ICS, NIS = ICS * S::IY, PX = S::PX, PY = S::PY, PCP = S::PCP, NPQ = S::NPQ,
                  NT = S::NT, R8 = S::R8, C8 = S::C8;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    float *sraw = reinterpret_cast<float *>(smem_raw);                          // [SLOTS][5][RAWF]
    float4 *sUA = reinterpret_cast<float4 *>(smem_raw + S::OFF_UA);             // [3][IY][ICS] (u, v)
    float4 *sUB = reinterpret_cast<float4 *>(smem_raw + S::OFF_UB);             // [3][IY][ICS] (w, phi)
    float4 *sPA = reinterpret_cast<float4 *>(smem_raw + S::OFF_PA);             // [3][NPQ] (u*, v*)
    float4 *sPB = reinterpret_cast<float4 *>(smem_raw + S::OFF_PB);             // [3][NPQ] (w*, phi*)
    float4 *sPC = reinterpret_cast<float4 *>(smem_raw + S::OFF_PC);             // [3][NPQ] (xi_x, xi_y)
    float2 *sPD = reinterpret_cast<float2 *>(smem_raw + S::OFF_PD);             // [3][NPQ] xi_z
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + S::OFF_BAR);        // [SLOTS]

    const Grid &G = A.G;
    const Phys<float> &P = A.P;
    const int nx = G.n[0], ny = G.n[1], nz = G.n[2];
    const bool perx = P.bc[0] == BC_PERIODIC, pery = P.bc[2] == BC_PERIODIC,
               perz = P.bc[4] == BC_PERIODIC;
    const int tid = threadIdx.x;
    const int x0 = bx * TX, y0 = by * TY;
    const int z0 = bz * A.zchunk;
    const int z1 = min(z0 + A.zchunk, nz);
    const float dt = (float)A.ctrl->dt;
    if (!(dt > 0.0f)) return true;  // a zero step: the Euler kernel copies U^n
    const int spin = A.ctrl->spin_limit > 0 ? A.ctrl->spin_limit : MBAR_SPIN_LIMIT;
    const bool no_copies = (A.ctrl->inject & INJECT_NO_COPIES) != 0;
    const float h = P.h, inv_h = P.inv_h, half_dt = 0.5f * dt;
    const float dth = dt * inv_h;                        // dt/h: velocity -> offset in cell units
    const float kf = P.inv_Ch2 * h;                      // 1/(C h): G(r) r = gt(q) r^ / (C h)
    const float kf34 = 0.75f * kf;                       // the corrector sums gt(q) / 0.75
    const float2 w1 = p2(P.gt[1]), w2 = p2(P.gt[2]), w3 = p2(P.gt[3]);

    __shared__ int s_colx[IX], s_rowy[S::IY];
    for (int t = tid; t < IX; t += NT) s_colx[t] = map_coord(x0 - 2 + t, nx, perx) + G.ox;
    for (int t = tid; t < S::IY; t += NT) s_rowy[t] = (map_coord(y0 - 2 + t, ny, pery) + GH) * G.px;
    if constexpr (INIT) {
        if (tid == 0) {
            for (int q = 0; q < S::SLOTS; ++q) mbar_init(&bar[q], 1);
            mbar_init_fence();
        }
        bool misaligned = false;
        for (int q = tid; q < S::SLOTS * 5; q += NT) misaligned |= (smem_u32(sraw + q * RAWF) & 127u) != 0;
        if (__syncthreads_or(misaligned)) {
            if (tid == 0) atomicOr(&A.ctrl->status, ST_TIMEOUT);
            return false;
        }
    }
    auto zoff = [&](int gz) { return (map_coord(gz, nz, perz) + GH) * (int)G.plane; };

    // ---- TMA ring (as lagrange_tile): plane q in slot q mod 2, box origin
    // (x0-4, y0-2); plane q may be issued once plane q-2 is consumed.
    uint32_t pending = 0;
    int issued = (!perz && z0 == 0) ? -2 : z0 - 3;
    static_assert(S::SLOTS == 2, "the TMA ring has two slots");
    auto slot_of = [](int q) { return q & 1; };
    auto issue = [&](int q) {
        pending |= 1u << slot_of(q);
        if (tid == 0) {
            const int sl = slot_of(q);
            fence_proxy_async();
            mbar_arrive_expect_tx(&bar[sl], (uint32_t)(5 * S::NB * sizeof(float)));
            const int zc = map_coord(q, nz, perz) + GH;
            if (!no_copies)
                for (int f = 0; f < 5; ++f)
                    tma_load_3d(sraw + (sl * 5 + f) * RAWF, A.tmU.at(f), x0 - 4 + G.ox, y0 - 2 + GH, zc, &bar[sl]);
        }
        issued = q;
    };
    auto issue_upto = [&](int q) {
        while (issued < q) issue(issued + 1);
    };
    auto wait_box = [&](int q) -> bool {
        const int sl = slot_of(q);
        const bool ok = mbar_wait(&bar[sl], (phase_bits >> sl) & 1u, spin);
        if (ok) {
            phase_bits ^= 1u << sl;
            pending &= ~(1u << sl);
        }
        return ok;
    };
    auto drain = [&]() {
        for (int s2 = 0; s2 < S::SLOTS; ++s2)
            if ((pending >> s2) & 1u) mbar_wait(&bar[s2], (phase_bits >> s2) & 1u, spin);
    };
    // raw value of field f at box column bx, row by of plane q, for both lanes
    // (columns bx and bx + HX)
    auto RAW2 = [&](int q, int f, int bxx, int byy) -> float2 {
        const float *b = sraw + (slot_of(q) * 5 + f) * RAWF + byy * BW + bxx;
        return make_float2(b[0], b[HX]);
    };

    // ---- U^n plane q: raw box -> primitives ring, pair position (ic, iy) =
    // columns ic and ic + HX of the halo-2 region
    auto convert = [&](int q) {
        const int slot = mod3(q);
        for (int t = tid; t < NIQ; t += NT) {
            const int ic = t % ICP, iy = t / ICP, o = slot * NIS + iy * ICS + ic;
            const Prim2 r = eos2(P, RAW2(q, 0, ic + 2, iy), RAW2(q, 1, ic + 2, iy), RAW2(q, 2, ic + 2, iy),
                                 RAW2(q, 3, ic + 2, iy), RAW2(q, 4, ic + 2, iy));
            sUA[o] = cat2(r.u, r.v);
            sUB[o] = cat2(r.w, r.phi);
        }
    };
    auto fetch = [&](int q) -> bool {
        issue_upto(q);
        if (!wait_box(q)) return false;
        convert(q);
        return true;
    };

    // pair position of the predictor task (pass, t); false: no task.  pass 0 =
    // the thread's inner pair (columns c, c + HX with c in [1, HX]); pass 1 =
    // the halo ring: the first row, the last row, the first pair column and
    // the last pair column of the rows between (whose other lane is an inner
    // particle, stored there too), each from a multiple of 8 threads
    auto pos_of = [&](int pass, int t, int &c, int &py) -> bool {
        c = py = 0;
        if (pass == 0) {
            c = t % HX + 1;
            py = t / HX + 1;
            return true;
        }
        if (t < 2 * R8) {
            c = t % R8;
            py = t < R8 ? 0 : PY - 1;
            return c < PCP;
        }
        if (t < 2 * R8 + 2 * C8) {
            const int r = t - 2 * R8;
            c = r < C8 ? 0 : PCP - 1;
            py = 1 + r % C8;
            return py < PY - 1;
        }
        return false;
    };

    // ---- packed static-lattice plane sums (as lagrange_tile, both lanes at
    // once): role 0 = the particle's own plane without the centre, role 1 =
    // the plane below or above.  iq: pair position of the particles' centre in
    // the primitives ring.
    struct Sum0P {
        float2 X, Y, V;
    };
    struct Sum1P {
        float2 X, Y, V, Z, W;
    };
    auto plane_sums = [&](int slot, int iq, bool want0, bool want1, Sum0P &s0, Sum1P &s1) {
        const float2 z2 = p2(0.0f);
        s0 = Sum0P{z2, z2, z2};
        s1 = Sum1P{z2, z2, z2, z2, z2};
        const float4 *pa = sUA + slot * NIS + iq, *pb = sUB + slot * NIS + iq;
#pragma unroll
        for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
            for (int dx = -1; dx <= 1; ++dx) {
                const int d2 = dx * dx + dy * dy;
                const float4 qa = pa[dy * ICS + dx], qb = pb[dy * ICS + dx];
                const float2 u = lo2(qa), v = hi2(qa), w = lo2(qb), phi = hi2(qb);
                float2 ru = z2;  // dx u_j + dy v_j
                if (dx && dy) ru = add2(dx > 0 ? u : neg2(u), dy > 0 ? v : neg2(v));
                else if (dx) ru = dx > 0 ? u : neg2(u);
                else if (dy) ru = dy > 0 ? v : neg2(v);
                if (want0 && d2 > 0) {
                    const float2 a = mul2(d2 == 1 ? w1 : w2, phi);
                    if (dx) s0.X = dx > 0 ? add2(s0.X, a) : sub2(s0.X, a);
                    if (dy) s0.Y = dy > 0 ? add2(s0.Y, a) : sub2(s0.Y, a);
                    s0.V = fma2(a, ru, s0.V);
                }
                if (want1) {
                    const float2 b = mul2(d2 == 0 ? w1 : (d2 == 1 ? w2 : w3), phi);
                    if (dx) s1.X = dx > 0 ? add2(s1.X, b) : sub2(s1.X, b);
                    if (dy) s1.Y = dy > 0 ? add2(s1.Y, b) : sub2(s1.Y, b);
                    if (d2 > 0) s1.V = fma2(b, ru, s1.V);
                    s1.Z = add2(s1.Z, b);
                    s1.W = fma2(b, w, s1.W);
                }
            }
    };
    Sum1P c1m, c1;  // the thread's inner pair: role-1 sums of planes p-1 and p
    Sum0P c0;       // and role-0 sums of plane p
    float *sRho = reinterpret_cast<float *>(smem_raw + S::OFF_RHO);  // [2][PX * PY], plane parity

    // ---- predictor (Eq. 5) for plane p, one pair position per task.  own[]
    // receives, for the thread's inner pair, (U^n + U*)/2 of m and E, u^n and
    // the lattice gravity D0 (the corrector of the same cells reuses them).
    auto predict = [&](int p, float2 own[10]) {
        const int sl = mod3(p), sm = mod3(p - 1), sp = mod3(p + 1);
        const int zo = zoff(p);
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            const int t = tid;
            int c, py;
            if (!pos_of(pass, t, c, py)) break;
            const int iq = (py + 1) * ICS + (c + 1);
            // the lattice gravity of both particles, loaded before the plane sums
            // so that their arithmetic covers the global-load latency
            const int rowo = zo + s_rowy[py + 1];
            const int ca = rowo + s_colx[c + 1], cb = rowo + s_colx[c + 1 + HX];
            const float2 D0x = make_float2(A.grav[0][ca], A.grav[0][cb]);
            const float2 D0y = make_float2(A.grav[1][ca], A.grav[1][cb]);
            const float2 D0z = make_float2(A.grav[2][ca], A.grav[2][cb]);
            Sum0P s0, n0;
            Sum1P s1m, s1p, unused1;
            if (pass == 0) {  // plane p+1 is new; p-1 and p come from the column cache
                plane_sums(sp, iq, true, true, n0, s1p);
                s0 = c0;
                s1m = c1m;
                c1m = c1;
                c1 = s1p;
                c0 = n0;
            } else {
                plane_sums(sm, iq, false, true, n0, s1m);
                plane_sums(sl, iq, true, false, s0, unused1);
                plane_sums(sp, iq, false, true, n0, s1p);
            }
            const float2 Px = add2(add2(s0.X, s1m.X), s1p.X);
            const float2 Py = add2(add2(s0.Y, s1m.Y), s1p.Y);
            const float2 Pz = sub2(s1p.Z, s1m.Z);
            const float2 Wj = add2(add2(add2(s0.V, s1m.V), s1p.V), sub2(s1p.W, s1m.W));
            const float4 qa = sUA[sl * NIS + iq], qb = sUB[sl * NIS + iq];
            const float2 qu = lo2(qa), qv = hi2(qa), qw = lo2(qb), qphi = hi2(qb);
            // Static lattice: the pressure work sum_j G r.(u_i+u_j)/2 phi_j = (u_i.P^ + sum_j G phi_j r.u_j)/2
            const float2 Wk = mul2(p2(0.5f), fma2(qu, Px, fma2(qv, Py, fma2(qw, Pz, Wj))));
            const float2 rhoi = RAW2(p, 0, c + 3, py + 1);
            const bool gx = rhoi.x > P.rho_vac, gy = rhoi.y > P.rho_vac;
            const float2 pf = mul2(qphi, p2(kf));  // phi_i / (C h)
            const float2 z2 = p2(0.0f);
            const float2 Q0 = sel2(gx, gy, balance2<COMP>(pf, Px, rhoi, D0x), z2);
            const float2 Q1 = sel2(gx, gy, balance2<COMP>(pf, Py, rhoi, D0y), z2);
            const float2 Q2 = sel2(gx, gy, balance2<COMP>(pf, Pz, rhoi, D0z), z2);
            const float2 Q3 = sel2(gx, gy, balance2<COMP>(pf, Wk, rhoi, fma2(qu, D0x, fma2(qv, D0y, mul2(qw, D0z)))), z2);
            const float2 m0x = RAW2(p, 1, c + 3, py + 1), m0y = RAW2(p, 2, c + 3, py + 1),
                         m0z = RAW2(p, 3, c + 3, py + 1), E0 = RAW2(p, 4, c + 3, py + 1);
            const float2 dt2 = p2(dt);
            const float2 msx = fma2(dt2, Q0, m0x), msy = fma2(dt2, Q1, m0y), msz = fma2(dt2, Q2, m0z);
            const float2 Es = fma2(dt2, Q3, E0);
            const Prim2 q = eos2(P, rhoi, msx, msy, msz, Es);
            const int pt = sl * NPQ + py * PCP + c;
            sPA[pt] = cat2(q.u, q.v);
            sPB[pt] = cat2(q.w, q.phi);
            const float2 hd = p2(dth * 0.5f);
            sPC[pt] = cat2(mul2(hd, add2(qu, q.u)), mul2(hd, add2(qv, q.v)));
            sPD[pt] = mul2(hd, add2(qw, q.w));
            float *rr = sRho + (p & 1) * (PX * PY) + py * PX + c;
            rr[0] = rhoi.x;
            rr[HX] = rhoi.y;
            if (pass == 0) {
                const float2 half = p2(0.5f);
                own[0] = mul2(half, add2(m0x, msx));
                own[1] = mul2(half, add2(m0y, msy));
                own[2] = mul2(half, add2(m0z, msz));
                own[3] = mul2(half, add2(E0, Es));
                own[4] = qu;
                own[5] = qv;
                own[6] = qw;
                own[7] = D0x;
                own[8] = D0y;
                own[9] = D0z;
            }
        }
    };

    // ---- one particle's predictor record in the pair layout (boundary rules
    // only): read from its first copy, written to every copy
    struct PRec {
        float u, v, w, phi, xx, xy, xz;
    };
    auto prec_get = [&](int sl, int px, int py) -> PRec {
        const int h = px < PCP ? 0 : 1;
        const int q = sl * NPQ + py * PCP + px - h * HX;
        const float *a = reinterpret_cast<const float *>(sPA + q), *b = reinterpret_cast<const float *>(sPB + q),
                    *cc = reinterpret_cast<const float *>(sPC + q), *d = reinterpret_cast<const float *>(sPD + q);
        return PRec{a[h], a[2 + h], b[h], b[2 + h], cc[h], cc[2 + h], d[h]};
    };
    auto prec_put = [&](int sl, int px, int py, const PRec &r) {
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int c = px - h * HX;
            if (c < 0 || c >= PCP) continue;
            const int q = sl * NPQ + py * PCP + c;
            float *a = reinterpret_cast<float *>(sPA + q), *b = reinterpret_cast<float *>(sPB + q),
                  *cc = reinterpret_cast<float *>(sPC + q), *d = reinterpret_cast<float *>(sPD + q);
            a[h] = r.u;
            a[2 + h] = r.v;
            b[h] = r.w;
            b[2 + h] = r.phi;
            cc[h] = r.xx;
            cc[2 + h] = r.xy;
            d[h] = r.xz;
        }
    };

    // ---- predictor-stage ghost particle (gx_, gy_) of plane slot sl from the
    // boundary particle (bx_, by_) and the next inward (mx_, my_) along axis a of
    // face `face`; rp: density plane of the ghost and boundary (-1: the z ghost
    // planes, whose density no later rule reads); cg, cm: cells of the ghost and
    // the next inward particle (psi).  Rules as lagrange_tile's bc_record.
    auto bc_record = [&](int face, int a, int sl, int gx_, int gy_, int bx_, int by_, int mx_, int my_, int slb,
                         int slm, int rp, int rpb, long long cg, long long cm) {
        const int kind = P.bc[face];
        if (kind == BC_PERIODIC) return;
        float *rho_g = rp >= 0 ? sRho + rp * (PX * PY) + gy_ * PX + gx_ : nullptr;
        const float rb = sRho[rpb * (PX * PY) + by_ * PX + bx_];
        if (kind == BC_OUTFLOW) {
            prec_put(sl, gx_, gy_, prec_get(slb, bx_, by_));
            if (rho_g) *rho_g = rb;
            return;
        }
        if (kind == BC_INFLOW) {
            const bool vac = P.in_vac[face];
            const float u = vac ? 0.0f : P.inW[face][1], v = vac ? 0.0f : P.inW[face][2],
                        w = vac ? 0.0f : P.inW[face][3];
            prec_put(sl, gx_, gy_, PRec{u, v, w, P.inPhi[face], dth * u, dth * v, dth * w});
            if (rho_g) *rho_g = P.inW[face][0];
            return;
        }
        PRec b = prec_get(slb, bx_, by_);
        const float phib = b.phi;
        if (a == 0) { b.u = -b.u; b.xx = -b.xx; }
        if (a == 1) { b.v = -b.v; b.xy = -b.xy; }
        if (a == 2) { b.w = -b.w; b.xz = -b.xz; }
        float phig = 0.0f, rg = rb;
        if (rb > P.rho_vac && phib > 0.0f) {
            phig = prec_get(slm, mx_, my_).phi + rb * (A.psi[cm] - A.psi[cg]) / phib;
            if (phig < 0.0f) phig = 0.0f;
            const float ratio = phig / phib;
            rg = rb * ratio * ratio;
        }
        b.phi = phig;
        prec_put(sl, gx_, gy_, b);
        if (rho_g) *rho_g = rg;
    };

    // ---- x then y ghosts of predictor plane p (block-uniform branches)
    const bool edge_tile = (!perx && (x0 == 0 || x0 + TX >= nx)) || (!pery && (y0 == 0 || y0 + TY >= ny));
    auto fill_xy = [&](int p) {
        if (!edge_tile) return;  // nothing to fill; the caller's barrier orders predict and correct
        const int sl = mod3(p), rp = p & 1;
        const int zz = map_coord(p, nz, perz);
        __syncthreads();
        if (!perx) {
            for (int side = 0; side < 2; ++side) {
                const int gxg = side ? nx : -1;
                const int pxg = gxg - (x0 - 1);
                if (pxg < 0 || pxg >= PX) continue;
                const int pxb = side ? pxg - 1 : pxg + 1;
                const int pxm = side ? pxg - 2 : pxg + 2;
                // every row whose y resolves inside the domain (with periodic y
                // also the wrapped halo rows)
                for (int py = tid; py < PY; py += NT) {
                    const int gy = y0 - 1 + py;
                    if (!pery && (gy < 0 || gy >= ny)) continue;
                    const int gyi = map_coord(gy, ny, pery);
                    bc_record(side, 0, sl, pxg, py, pxb, py, pxm, py, sl, sl, rp, rp, G.at(gxg, gyi, zz),
                              G.at(side ? nx - 2 : 1, gyi, zz));
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
                    bc_record(2 + side, 1, sl, px, pyg, px, pyb, px, pym, sl, sl, rp, rp, G.at(gx, gyg, zz),
                              G.at(gx, side ? ny - 2 : 1, zz));
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
        for (int t = tid; t < PX * PY; t += NT) {
            const int px = t % PX, py = t / PX;
            const int gx = map_coord(x0 - 1 + px, nx, perx), gy = map_coord(y0 - 1 + py, ny, pery);
            bc_record(4 + side, 2, mod3(pg), px, py, px, py, px, py, mod3(pb), mod3(pm), -1, pb & 1,
                      G.at(gx, gy, pg), G.at(gx, gy, pm));
        }
        __syncthreads();
    };

    // ---- corrector (Eqs. 6-7, particles displaced by xi*) for plane k, both
    // cells of the thread (columns pcx and pcx + HX of row ty):
    // r^ = d + xi*^_j - xi*^_i, q = |r^|, G(r) r = gt(q) r^ / (C h).
    const int pcx = tid % HX, ty = tid / HX;
    auto correct = [&](int k, const float2 own[10]) {
        const int sl = mod3(k), sm = mod3(k - 1), sp = mod3(k + 1);
        const int pi = (ty + 1) * PCP + (pcx + 1);
        const float4 qa = sPA[sl * NPQ + pi], qb = sPB[sl * NPQ + pi], xa = sPC[sl * NPQ + pi];
        const float2 xiz = sPD[sl * NPQ + pi];
        const float2 xix = lo2(xa), xiy = hi2(xa);
        // d - xi*^_i for d = -1, 0, 1 along each axis: r^ = xi*^_j + (d - xi*^_i)
        const float2 ox[3] = {sub2(p2(-1.0f), xix), neg2(xix), sub2(p2(1.0f), xix)};
        const float2 oy[3] = {sub2(p2(-1.0f), xiy), neg2(xiy), sub2(p2(1.0f), xiy)};
        const float2 oz[3] = {sub2(p2(-1.0f), xiz), neg2(xiz), sub2(p2(1.0f), xiz)};
        const float2 z2 = p2(0.0f);
        float2 Px = z2, Py = z2, Pz = z2, Wj = z2;
#pragma unroll
        for (int dz = -1; dz <= 1; ++dz) {
            const int so = (dz < 0 ? sm : (dz > 0 ? sp : sl)) * NPQ + pi;
#pragma unroll
            for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
                for (int dx = -1; dx <= 1; ++dx) {
                    if (!dx && !dy && !dz) continue;
                    const int j = so + dy * PCP + dx;
                    const float4 ja = sPA[j], jb = sPB[j], jc = sPC[j];
                    const float2 jd = sPD[j];
                    const float2 rx = add2(lo2(jc), ox[dx + 1]), ry = add2(hi2(jc), oy[dy + 1]),
                                 rz = add2(jd, oz[dz + 1]);
                    // kernel weight gt(q) / 0.75 per lane (gtilde_q2_4_3); q^2 >= 1e-30
                    const float2 q2 = fma2(rx, rx, fma2(ry, ry, fma2(rz, rz, p2(1e-30f))));
                    const float2 rs = make_float2(f_rsqrt_n(q2.x), f_rsqrt_n(q2.y));
                    const float2 q = mul2(q2, rs);
                    float2 a = sub2(p2(2.0f), q);
                    a.x = a.x > 0.0f ? a.x : 0.0f;
                    a.y = a.y > 0.0f ? a.y : 0.0f;
                    const float2 g = sel2(q.x < 1.0f, q.y < 1.0f, fma2(p2(-3.0f), q, p2(4.0f)), mul2(mul2(a, a), rs));
                    const float2 gp = mul2(g, hi2(jb));
                    Px = fma2(gp, rx, Px);
                    Py = fma2(gp, ry, Py);
                    Pz = fma2(gp, rz, Pz);
                    Wj = fma2(gp, fma2(rz, lo2(jb), fma2(ry, hi2(ja), mul2(rx, lo2(ja)))), Wj);
                }
        }
        const float *rr = sRho + (k & 1) * (PX * PY) + (ty + 1) * PX + pcx + 1;
        const float2 rhoi = make_float2(rr[0], rr[HX]);
        const float2 qu = lo2(qa), qv = hi2(qa), qw = lo2(qb), qphi = hi2(qb);
        const float2 Wk = mul2(p2(0.5f), fma2(qu, Px, fma2(qv, Py, fma2(qw, Pz, Wj))));
        const bool gx = rhoi.x > P.rho_vac, gy = rhoi.y > P.rho_vac;
        const float2 pf = mul2(qphi, p2(kf34));
        const float2 Q0 = sel2(gx, gy, balance2<COMP>(pf, Px, rhoi, own[7]), z2);
        const float2 Q1 = sel2(gx, gy, balance2<COMP>(pf, Py, rhoi, own[8]), z2);
        const float2 Q2 = sel2(gx, gy, balance2<COMP>(pf, Pz, rhoi, own[9]), z2);
        const float2 Q3 = sel2(gx, gy, balance2<COMP>(pf, Wk, rhoi, fma2(qu, own[7], fma2(qv, own[8], mul2(qw, own[9])))), z2);
        const float2 hdt = p2(half_dt), half = p2(0.5f), h2 = p2(h);
        const float2 m[3] = {fma2(hdt, Q0, own[0]), fma2(hdt, Q1, own[1]), fma2(hdt, Q2, own[2])};
        const float2 E = fma2(hdt, Q3, own[3]);
        const Prim2 q = eos2(P, rhoi, m[0], m[1], m[2], E);
        const float2 xs[3] = {xix, xiy, xiz}, qq[3] = {q.u, q.v, q.w};
        // xi^{n+1} = xi*/2 + dt/2 (u^n + u~)/2, stored in length units
        float2 xn[3];
        bool far_a = false, far_b = false;
#pragma unroll
        for (int e = 0; e < 3; ++e) {
            xn[e] = fma2(hdt, mul2(half, add2(own[4 + e], qq[e])), mul2(h2, mul2(half, xs[e])));
            far_a |= !(fabsf(xn[e].x) <= h);
            far_b |= !(fabsf(xn[e].y) <= h);
        }
        const int gy_ = y0 + ty, gxa = x0 + pcx, gxb = gxa + HX;
        const bool in_a = gy_ < ny && gxa < nx, in_b = gy_ < ny && gxb < nx;
        const int crow = (k + GH) * (int)G.plane + s_rowy[ty + 2];
        if (in_a) {
            const int c = crow + s_colx[pcx + 2];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                A.m[e][c] = m[e].x;
                A.xi[e][c] = xn[e].x;
            }
            A.E[c] = E.x;
        }
        if (in_b) {
            const int c = crow + s_colx[pcx + 2 + HX];
#pragma unroll
            for (int e = 0; e < 3; ++e) {
                A.m[e][c] = m[e].y;
                A.xi[e][c] = xn[e].y;
            }
            A.E[c] = E.y;
        }
        if ((in_a && far_a) || (in_b && far_b)) atomicOr(&A.ctrl->status, ST_CFL);
    };

    // ---- one march (as lagrange_tile): iteration p predicts plane p (or fills
    // the z ghost plane of a non-periodic top), then corrects plane p - 1.
    const int zlast = (!perz && z1 == nz) ? nz : z1 + 1;
    auto timed_out = [&]() {
        if (tid == 0) atomicOr(&A.ctrl->status, ST_TIMEOUT);
    };
    const bool zero = !perz && z0 == 0;
    const int pfirst = zero ? 0 : z0 - 1;
    bool ok = fetch(pfirst - 1);
    ok = ok && fetch(pfirst);
    if (__syncthreads_or(!ok)) { drain(); timed_out(); return false; }
    {  // the inner pair's sums of the planes before the first predicted one
        int c, py;
        pos_of(0, tid, c, py);
        const int iq = (py + 1) * ICS + (c + 1);
        Sum0P unused0;
        plane_sums(mod3(pfirst - 1), iq, false, true, unused0, c1m);
        plane_sums(mod3(pfirst), iq, true, true, c0, c1);
    }
    float2 cur[10], nxt[10];
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
    }
    return true;
}
}  // namespace cspht
