// noalloc.cu -- one FP32 CSPH-TVD step that allocates no device memory.
//
// Some callers cannot call cudaMalloc: an application whose memory pool
// already owns all of the GPU's memory, or a time-critical loop in which the
// implicit device synchronisation of an allocation is not acceptable.  For
// them cspht_step_noalloc_f32 runs the fused fast-path step on buffers the
// caller owns and keeps every intermediate array in one file-scope device
// array of fixed size (NOALLOC_FLOATS floats, 64 MiB), which every GPU that
// loads the library holds until the process exits.
//
// Host code cannot use the array's name as a device address, so the first
// call on each device looks the address up with cudaGetSymbolAddress (with
// that device current) and remembers it; that first call should come before
// any stream capture.  All calls share the one array and it keeps the last
// call's contents, which may be another grid's and may hold NaN after a
// failed call: every call first clears the part of the array it uses
// (cudaMemsetAsync on its stream, which allocates nothing), so padding that a
// tile copy loads but no stage writes reads as zero.  Calls that overlap on
// the GPU (two streams, or two host threads) race on the array.
#include <cmath>
#include <cstring>

#include "../../include/cspht.h"
#include "common.cuh"
#include "fast.cuh"
#include "ghost.cuh"
#include "plain.cuh"
#include "tma_host.cuh"

using namespace cspht;

namespace {

constexpr long long NOALLOC_FLOATS = 16ll << 20;  // 64 MiB of scratch
constexpr int NA_TX = 32, NA_TY = 8, NA_BX = 64, NA_BY = 4;
constexpr int NA_FIELDS = 21;   // U^n (5), U^{n+1} (5), psi, gravity (3), corrector state (7)
constexpr int NA_CTRL_FLOATS = 64;  // control word at the start (256-byte slot)

static __device__ __align__(256) float g_noalloc_scratch[NOALLOC_FLOATS];

constexpr int NA_MAX_DEVICES = 64;
float *g_base[NA_MAX_DEVICES];  // device address of the scratch, per device (host side)

__global__ void k_na_reset(Ctrl *c, double cfl) {
    c->t = 0.0;
    c->t_end = INFINITY;
    c->cfl = cfl;
    c->dt = 0.0;
    c->smax_cur = 0ull;
    c->smax_next = 0ull;
    c->steps = 0;
    c->status = 0;
    c->inject = 0;
    c->spin_limit = 0;
}

__global__ void k_na_pack(Grid G, const float *__restrict__ src, int nf, UPtr<float> dst) {
    Cell cc;
    if (!interior_cell(G, cc)) return;
    const long long N = G.cells();
    const long long g = ((long long)cc.k * G.n[1] + cc.j) * G.n[0] + cc.i;
    const long long c = G.at(cc.i, cc.j, cc.k);
    for (int f = 0; f < nf; ++f) dst.f[f][c] = src[f * N + g];
}

__global__ void k_na_unpack(Grid G, UPtr<float> src, float *__restrict__ dst) {
    Cell cc;
    if (!interior_cell(G, cc)) return;
    const long long N = G.cells();
    const long long g = ((long long)cc.k * G.n[1] + cc.j) * G.n[0] + cc.i;
    const long long c = G.at(cc.i, cc.j, cc.k);
    for (int f = 0; f < 5; ++f) dst[f * N + g] = src.f[f][c];
}

__global__ void k_na_speed(Grid G, Phys<float> P, UPtr<float> U, Ctrl *ctrl) {
    Cell cc;
    const bool in = interior_cell(G, cc);
    double sp = 0.0;
    if (in) {
        const long long c = G.at(cc.i, cc.j, cc.k);
        sp = signal_speed_t(P, U.f[0][c], U.f[1][c], U.f[2][c], U.f[3][c], U.f[4][c]);
    }
    block_max_to(&ctrl->smax_next, sp);
}

// dt = cfl h / max signal speed (0 when nothing moves; a NaN speed raises the status)
__global__ void k_na_dt(Ctrl *c, double h) {
    const double s = __longlong_as_double((long long)c->smax_next);
    double dt = 0.0;
    if (s != s)
        c->status |= ST_NONFINITE;
    else if (s > 0.0)
        dt = c->cfl * h / s;
    c->dt = dt;
    c->t = dt;
    c->smax_cur = c->smax_next;
    c->smax_next = 0ull;
}

void na_phys(Phys<float> &P, double h, double gamma, const cspht_bcs *bcs) {
    memset(&P, 0, sizeof P);
    P.h = (float)h;
    P.inv_h = (float)(1.0 / h);
    P.gamma = (float)gamma;
    P.gm1 = (float)(gamma - 1.0);
    P.inv_gm1 = (float)(1.0 / (gamma - 1.0));
    P.rho_vac = 1e-10f;
    const double r2 = std::sqrt(2.0), r3 = std::sqrt(3.0);
    const double gt1 = 0.75, gt2 = 0.75 * (2.0 - r2) * (2.0 - r2) / r2,
                 gt3 = 0.75 * (2.0 - r3) * (2.0 - r3) / r3;
    const double C = 2.0 * gt1 + 8.0 * gt2 + 8.0 * gt3;
    P.inv_Ch2 = (float)(1.0 / (C * h * h));
    P.w[1] = (float)(gt1 / (C * h * h));
    P.w[2] = (float)(gt2 / (C * h * h));
    P.w[3] = (float)(gt3 / (C * h * h));
    P.gt[1] = (float)gt1;
    P.gt[2] = (float)gt2;
    P.gt[3] = (float)gt3;
    for (int f = 0; f < 6; ++f) {
        P.bc[f] = bcs ? bcs->type[f] : CSPHT_BC_PERIODIC;
        double w[5] = {0, 0, 0, 0, 0};
        if (bcs)
            for (int c = 0; c < 5; ++c) w[c] = bcs->inflow[f][c];
        for (int c = 0; c < 5; ++c) P.inW[f][c] = (float)w[c];
        P.inU[f][0] = (float)w[0];
        for (int e = 0; e < 3; ++e) P.inU[f][1 + e] = (float)(w[0] * w[1 + e]);
        P.inU[f][4] = (float)(w[4] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]));
        P.in_vac[f] = !(w[0] > 1e-10);
        P.inPhi[f] = P.in_vac[f] ? 0.0f : (float)std::sqrt(2.0 * (w[4] > 0 ? w[4] : 0.0));
    }
    P.limiter = CSPHT_LIMITER_VANLEER;
    P.balance = CSPHT_BALANCE_PLAIN;
    P.riemann = CSPHT_RIEMANN_LF;
}

}  // namespace

extern "C" int cspht_step_noalloc_f32(int nx, int ny, int nz, double h, double gamma,
                                      const cspht_bcs *bcs, const float *U, const float *psi,
                                      float *U_out, double cfl, double *dt_taken, void *stream) {
    if (!U || !psi || !U_out || !(h > 0.0) || !(gamma > 1.0) || !(cfl > 0.0)) return CSPHT_EINVAL;
    // an error left by the caller's earlier work stays the caller's: report it
    // without clearing it and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return CSPHT_ECUDA;
    const int n[3] = {nx, ny, nz};
    for (int d = 0; d < 3; ++d) {
        const int lo = bcs ? bcs->type[2 * d] : 0, hi = bcs ? bcs->type[2 * d + 1] : 0;
        if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return CSPHT_EINVAL;
        if ((lo == CSPHT_BC_PERIODIC) != (hi == CSPHT_BC_PERIODIC)) return CSPHT_EINVAL;
        if (n[d] < 1 || (lo != CSPHT_BC_PERIODIC && n[d] < 2) || n[d] > 65000) return CSPHT_EINVAL;
    }
    const Grid G = make_grid<float>(nx, ny, nz);
    if (NA_CTRL_FLOATS + (long long)NA_FIELDS * G.total > NOALLOC_FLOATS) return CSPHT_ETOOBIG;

    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= NA_MAX_DEVICES) {
        cudaGetLastError();
        return CSPHT_ECUDA;
    }
    if (!g_base[dev]) {  // first call on this device: find the array's device address
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return CSPHT_ECUDA;
        }
        if (cudaFuncSetAttribute(k_lagrange<float, NA_TX, NA_TY>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)LagShape<NA_TX, NA_TY>::bytes<float>()) != cudaSuccess ||
            cudaFuncSetAttribute(k_euler<float, NA_TX, NA_TY, LIM_VANLEER, RIEMANN_LF>,
                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)EulShape<NA_TX, NA_TY>::smem_bytes<float>()) != cudaSuccess) {
            cudaGetLastError();
            return CSPHT_ECUDA;
        }
        g_base[dev] = (float *)p;
    }
    cudaStream_t st = (cudaStream_t)stream;

    // carve the scratch: control word, then NA_FIELDS padded arrays
    float *base = g_base[dev];
    Ctrl *ctrl = reinterpret_cast<Ctrl *>(base);
    float *p = base + NA_CTRL_FLOATS;
    auto take = [&]() {
        float *r = p;
        p += G.total;
        return r;
    };
    UPtr<float> Un, Uo;
    for (int f = 0; f < 5; ++f) Un.f[f] = take();
    for (int f = 0; f < 5; ++f) Uo.f[f] = take();
    float *psip = take();
    float *grav[3] = {take(), take(), take()};
    S2Ptr<float> s2;
    for (int e = 0; e < 3; ++e) s2.m[e] = take();
    s2.E = take();
    for (int e = 0; e < 3; ++e) s2.xi[e] = take();

    Phys<float> P;
    na_phys(P, h, gamma, bcs);
    const dim3 blk(NA_BX, NA_BY), cg((nx + NA_BX - 1) / NA_BX, (ny + NA_BY - 1) / NA_BY, nz);

    // clear the control word and every field this grid uses: the array keeps
    // whatever the previous call left there
    const size_t used = sizeof(float) * (size_t)(NA_CTRL_FLOATS + (long long)NA_FIELDS * G.total);
    if (cudaMemsetAsync(base, 0, used, st) != cudaSuccess) {
        cudaGetLastError();
        return CSPHT_ECUDA;
    }
    k_na_reset<<<1, 1, 0, st>>>(ctrl, cfl);
    UPtr<float> pp;
    pp.f[0] = psip;
    k_na_pack<<<cg, blk, 0, st>>>(G, psi, 1, pp);
    for (int a = 0; a < 3; ++a) {
        const long long nt = ghost_pass_threads(G, a, 2);
        k_ghost_psi<float><<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(G, P, a, psip);
    }
    k_gravity<float><<<cg, blk, 0, st>>>(G, P, psip, grav[0], grav[1], grav[2]);
    k_na_pack<<<cg, blk, 0, st>>>(G, U, 5, Un);
    k_na_speed<<<cg, blk, 0, st>>>(G, P, Un, ctrl);
    k_na_dt<<<1, 1, 0, st>>>(ctrl, h);
    for (int a = 0; a < 3; ++a) {
        const long long nt = ghost_pass_threads(G, a, 2);
        k_ghost_U<float><<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(G, P, a, Un, psip);
    }
    // z chunks as in the allocating fast path
    const int tiles = ((nx + NA_TX - 1) / NA_TX) * ((ny + NA_TY - 1) / NA_TY);
    int nch = (148 * 8 + tiles - 1) / tiles;
    const int maxch = (nz + 7) / 8;
    if (nch > maxch) nch = maxch;
    if (nch < 1) nch = 1;
    const int zchunk = (nz + nch - 1) / nch;
    const dim3 lg((nx + NA_TX - 1) / NA_TX, (ny + NA_TY - 1) / NA_TY, (nz + zchunk - 1) / zchunk);
    LagArgs<float> A;
    EulArgs<float> B;
    for (int f = 0; f < 5; ++f)
        if (!make_tmap<float>(&A.tmU.m[f], Un.f[f], G, NA_TX + 8, NA_TY + 4)) return CSPHT_ECUDA;
    for (int f = 0; f < 5; ++f) B.tmU.m[f] = A.tmU.m[f];
    {
        const float *sf[6] = {s2.m[0], s2.m[1], s2.m[2], s2.E, s2.xi[0], s2.xi[1]};
        for (int f = 0; f < 6; ++f)
            if (!make_tmap<float>(&B.tmS.m[f], sf[f], G, NA_TX + 8, NA_TY + 2)) return CSPHT_ECUDA;
    }
    A.G = G;
    A.P = P;
    for (int f = 0; f < 5; ++f) A.U[f] = Un.f[f];
    A.psi = psip;
    for (int e = 0; e < 3; ++e) {
        A.grav[e] = grav[e];
        A.m[e] = s2.m[e];
        A.xi[e] = s2.xi[e];
    }
    A.E = s2.E;
    A.ctrl = ctrl;
    A.zchunk = zchunk;
    k_lagrange<float, NA_TX, NA_TY>
        <<<lg, LagShape<NA_TX, NA_TY>::threads<float>(), LagShape<NA_TX, NA_TY>::bytes<float>(), st>>>(A);
    for (int a = 0; a < 3; ++a) {
        const long long nt = ghost_pass_threads(G, a);
        k_ghost_S2<float><<<(unsigned)((nt + 255) / 256), 256, 0, st>>>(G, P, a, s2, ctrl);
    }
    B.G = G;
    B.P = P;
    for (int f = 0; f < 5; ++f) {
        B.U[f] = Un.f[f];
        B.Un[f] = Uo.f[f];
    }
    for (int e = 0; e < 3; ++e) {
        B.m[e] = s2.m[e];
        B.xi[e] = s2.xi[e];
    }
    B.E = s2.E;
    B.rho_lo = nullptr;  // no compensation word in this variant
    B.ctrl = ctrl;
    B.zchunk = zchunk;
    k_euler<float, NA_TX, NA_TY, LIM_VANLEER, RIEMANN_LF>
        <<<lg, NA_TX * NA_TY, EulShape<NA_TX, NA_TY>::smem_bytes<float>(), st>>>(B);
    k_na_unpack<<<cg, blk, 0, st>>>(G, Uo, U_out);
    if (cudaGetLastError() != cudaSuccess) return CSPHT_ECUDA;

    // read back dt and the status word (no allocation: a host stack copy)
    Ctrl hc;
    if (cudaMemcpyAsync(&hc, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess) {
        cudaGetLastError();
        return CSPHT_ECUDA;
    }
    if (dt_taken) *dt_taken = hc.dt;
    if (hc.status & ST_TIMEOUT) return CSPHT_ECUDA;
    if (hc.status & ST_NONFINITE) return CSPHT_ENONFINITE;
    if (hc.status & ST_CFL) return CSPHT_ECFL;
    if (hc.status & ST_NEGATIVE) return CSPHT_ENEGATIVE;
    return CSPHT_OK;
}
