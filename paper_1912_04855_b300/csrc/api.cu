// api.cu -- host runtime and C ABI of the B300 CSPH-TVD solver (include/cspht.h).
//
// One handle = one grid on the current CUDA device: padded device arrays,
// a control word (time, dt, status), one stream, and two CUDA graphs that
// replay a whole time step (one per ping-pong parity of the state buffers).
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>
#include <array>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <vector>

#include "../../include/cspht.h"
#include "common.cuh"
#include "ghost.cuh"
#include "plain.cuh"
#include "fast.cuh"
#include "tma_host.cuh"

using namespace cspht;

namespace {

constexpr int BX = 64, BY = 4;  // block shape of the per-cell kernels

// ------------------------------------------------------------ device memory
// A handle's device arrays come from the library's own stream-ordered pool
// (one per device, which keeps freed memory for the next handle) and are
// freed in order on the handle's stream.  Destroying a handle then waits for
// nothing but that stream: a plain cudaFree synchronises the whole device,
// which stalls the work every other handle has in flight (the serving loop
// retires requests while others run).

constexpr int MAX_DEVICES = 64;

cudaMemPool_t lib_pool() {
    static std::mutex mu;
    static cudaMemPool_t pools[MAX_DEVICES] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAX_DEVICES) return nullptr;
    std::lock_guard<std::mutex> lk(mu);
    if (!pools[dev]) {
        cudaMemPoolProps props;
        memset(&props, 0, sizeof props);
        props.allocType = cudaMemAllocationTypePinned;
        props.handleTypes = cudaMemHandleTypeNone;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t mp = nullptr;
        if (cudaMemPoolCreate(&mp, &props) != cudaSuccess) return nullptr;
        uint64_t keep = ~0ull;  // keep freed memory in the pool
        cudaMemPoolSetAttribute(mp, cudaMemPoolAttrReleaseThreshold, &keep);
        pools[dev] = mp;
    }
    return pools[dev];
}

// Device memory for stream s (usable in s's order, or anywhere once s has
// reached this point); false on failure (the error is cleared).
bool dev_alloc(void **p, size_t bytes, cudaStream_t s) {
    *p = nullptr;
    cudaMemPool_t mp = lib_pool();
    if (!mp || cudaMallocFromPoolAsync(p, bytes, mp, s) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}
template <class P>
bool dev_alloc(P **p, size_t bytes, cudaStream_t s) {
    void *q = nullptr;
    const bool ok = dev_alloc(&q, bytes, s);
    *p = static_cast<P *>(q);
    return ok;
}

// Returns p to the pool once the work enqueued on s so far is done.
void dev_free(void *p, cudaStream_t s) {
    if (p && cudaFreeAsync(p, s) != cudaSuccess) cudaGetLastError();
}

// Page-locked host mirrors of the control word, handed out from slabs that
// are never freed (freeing page-locked memory synchronises the device).
std::mutex g_ctrl_mu;
std::vector<Ctrl *> g_ctrl_free;

Ctrl *host_ctrl_alloc() {
    std::lock_guard<std::mutex> lk(g_ctrl_mu);
    if (g_ctrl_free.empty()) {
        constexpr int SLAB = 64;
        void *slab = nullptr;
        if (cudaMallocHost(&slab, SLAB * sizeof(Ctrl)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        for (int i = SLAB - 1; i >= 0; --i) g_ctrl_free.push_back(static_cast<Ctrl *>(slab) + i);
    }
    Ctrl *c = g_ctrl_free.back();
    g_ctrl_free.pop_back();
    return c;
}

void host_ctrl_free(Ctrl *c) {
    if (!c) return;
    std::lock_guard<std::mutex> lk(g_ctrl_mu);
    g_ctrl_free.push_back(c);
}

// ------------------------------------------------------------ small kernels

__global__ void k_set_params(Ctrl *c, double cfl, double t_end) {
    c->cfl = cfl;
    c->t_end = t_end;
}

__global__ void k_set_inject(Ctrl *c, int inject, int spin_limit) {
    c->inject = inject;
    c->spin_limit = spin_limit;
}

__global__ void k_reset_state(Ctrl *c) {
    c->status = 0;
    c->smax_next = 0ull;
}

// Start of a step: dt = cfl h / max signal speed of the current state,
// clipped so the step lands on t_end; dt = 0 makes the step a copy.
__device__ __forceinline__ void dt_update(Ctrl *c, double h) {
    double s = __longlong_as_double((long long)c->smax_next);
    double dt = 0.0;
    if (s != s) {
        c->status |= ST_NONFINITE;
    } else if (s > 0.0) {
        dt = c->cfl * h / s;
    }
    double rem = c->t_end - c->t;
    bool last = false;
    if (dt >= rem) {
        dt = rem > 0.0 ? rem : 0.0;
        last = true;
    }
    if (!(dt > 0.0)) dt = 0.0;
    c->dt = dt;
    c->smax_cur = c->smax_next;
    c->smax_next = 0ull;
    if (dt > 0.0) {
        c->t = last ? c->t_end : c->t + dt;
        c->steps += 1;
    }
}

__global__ void k_dt(Ctrl *c, double h) { dt_update(c, h); }

template <typename T>
__global__ void k_speed(Grid G, Phys<T> P, UPtr<T> U, Ctrl *ctrl, int fused) {
    Cell cc;
    bool in = interior_cell(G, cc);
    double sp = 0.0;
    if (in) {
        long long c = G.at(cc.i, cc.j, cc.k);
        // the speed the path's own Euler epilogue computes, so that a state
        // set from a checkpoint takes the same next dt as the running one
        sp = fused ? (double)signal_speed_t(P, U.f[0][c], U.f[1][c], U.f[2][c], U.f[3][c], U.f[4][c])
                   : signal_speed(P, U.f[0][c], U.f[1][c], U.f[2][c], U.f[3][c], U.f[4][c]);
    }
    block_max_to(&ctrl->smax_next, sp);
}

// compact FP64 SoA (5*N or N) <-> padded arrays
template <typename T, typename S>
__global__ void k_load(Grid G, const S *__restrict__ src, int nf, UPtr<T> dst) {
    Cell cc;
    if (!interior_cell(G, cc)) return;
    long long N = G.cells();
    long long g = ((long long)cc.k * G.n[1] + cc.j) * G.n[0] + cc.i;
    long long c = G.at(cc.i, cc.j, cc.k);
    for (int f = 0; f < nf; ++f) dst.f[f][c] = (T)src[f * N + g];
}

template <typename T>
__global__ void k_load_prim(Grid G, double gamma, const double *__restrict__ W, UPtr<T> dst) {
    Cell cc;
    if (!interior_cell(G, cc)) return;
    long long N = G.cells();
    long long g = ((long long)cc.k * G.n[1] + cc.j) * G.n[0] + cc.i;
    long long c = G.at(cc.i, cc.j, cc.k);
    double r = W[g], u = W[N + g], v = W[2 * N + g], w = W[3 * N + g], p = W[4 * N + g];
    dst.f[0][c] = (T)r;
    dst.f[1][c] = (T)(r * u);
    dst.f[2][c] = (T)(r * v);
    dst.f[3][c] = (T)(r * w);
    dst.f[4][c] = (T)(p / (gamma - 1.0) + 0.5 * r * (u * u + v * v + w * w));
}

template <typename T, typename D>
__global__ void k_store(Grid G, UPtr<T> src, const T *__restrict__ lo, D *__restrict__ dst) {
    Cell cc;
    if (!interior_cell(G, cc)) return;
    long long N = G.cells();
    long long g = ((long long)cc.k * G.n[1] + cc.j) * G.n[0] + cc.i;
    long long c = G.at(cc.i, cc.j, cc.k);
    for (int f = 1; f < 5; ++f) dst[f * N + g] = (D)src.f[f][c];
    // density with its compensation word, summed in FP64 and rounded once
    dst[g] = (D)((double)src.f[0][c] + (lo ? (double)lo[c] : 0.0));
}

// Density compensation word after an upload: the part of the FP64 density
// that the rounded FP32 value lost.
template <typename T>
__global__ void k_rho_lo(Grid G, const double *__restrict__ rho, const T *__restrict__ hi, T *__restrict__ lo) {
    Cell cc;
    if (!interior_cell(G, cc)) return;
    long long g = ((long long)cc.k * G.n[1] + cc.j) * G.n[0] + cc.i;
    long long c = G.at(cc.i, cc.j, cc.k);
    lo[c] = (T)(rho[g] - (double)hi[c]);
}

// FP64 totals: per-block partial sums in a fixed tree order, then one block.
constexpr int TOT_THREADS = 256;

template <typename T>
__global__ void k_totals(Grid G, UPtr<T> U, const T *__restrict__ lo, const T *__restrict__ psi,
                         double *__restrict__ part) {
    __shared__ double s[6][TOT_THREADS];
    long long N = G.cells();
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (long long g = blockIdx.x * (long long)TOT_THREADS + threadIdx.x; g < N;
         g += (long long)gridDim.x * TOT_THREADS) {
        int i = (int)(g % G.n[0]);
        long long r = g / G.n[0];
        int j = (int)(r % G.n[1]), k = (int)(r / G.n[1]);
        long long c = G.at(i, j, k);
        double rho = (double)U.f[0][c] + (lo ? (double)lo[c] : 0.0);
        acc[0] += rho;
        for (int f = 1; f < 5; ++f) acc[f] += (double)U.f[f][c];
        acc[5] += (double)U.f[4][c] + rho * (double)psi[c];
    }
    for (int f = 0; f < 6; ++f) s[f][threadIdx.x] = acc[f];
    __syncthreads();
    for (int w = TOT_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int f = 0; f < 6; ++f) s[f][threadIdx.x] += s[f][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int f = 0; f < 6; ++f) part[blockIdx.x * 6 + f] = s[f][0];
}

__global__ void k_totals_final(const double *__restrict__ part, int nb, double vol, double *out) {
    __shared__ double s[6][TOT_THREADS];
    double acc[6] = {0, 0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nb; b += TOT_THREADS)
        for (int f = 0; f < 6; ++f) acc[f] += part[b * 6 + f];
    for (int f = 0; f < 6; ++f) s[f][threadIdx.x] = acc[f];
    __syncthreads();
    for (int w = TOT_THREADS / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int f = 0; f < 6; ++f) s[f][threadIdx.x] += s[f][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int f = 0; f < 6; ++f) out[f] = s[f][0] * vol;
}

constexpr int TOT_BLOCKS = 1184;  // 8 per SM on 148 SMs

// ------------------------------------------------------------------ solver

// Kernel kinds reported by cspht_profile_read.
enum {
    KK_DT, KK_GHOST_U, KK_PRIM, KK_HFC_PRED, KK_SUL_PRED, KK_GHOST_S1, KK_HFC_CORR, KK_SUL_CORR,
    KK_GHOST_S2, KK_FGC, KK_SUE, KK_LAGRANGE, KK_EULER, KK_COUNT
};
const char *const KK_NAME[KK_COUNT] = {"dt",       "ghost_U",  "prim",     "hfc_pred", "sul_pred",
                                       "ghost_S1", "hfc_corr", "sul_corr", "ghost_S2", "fgc",
                                       "sue",      "lagrange", "euler"};

struct SolverBase {
    virtual ~SolverBase() {
        for (cudaEvent_t e : evpool) cudaEventDestroy(e);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        for (cudaEvent_t e : {ev_up, ev_loaded, ev_stored, ev_down})
            if (e) cudaEventDestroy(e);
        if (s_up) cudaStreamDestroy(s_up);
        if (s_down) cudaStreamDestroy(s_down);
    }
    // Asynchronous FP32 host I/O (cspht_upload_f32_async, cspht_download_f32_async):
    // the copies run on their own streams, so that one step's download overlaps
    // the next step's upload, and events order them with the compute stream:
    // ev_up = the upload copy landed in the staging buffer, ev_loaded = the state
    // was converted from it (the buffer is free again), ev_stored = the state was
    // converted into the output staging buffer, ev_down = that buffer was read out.
    cudaStream_t s_up = nullptr, s_down = nullptr;
    cudaEvent_t ev_up = nullptr, ev_loaded = nullptr, ev_stored = nullptr, ev_down = nullptr;
    bool io_ready = false;  // streams and events all created
    int io_init() {
        if (io_ready) return CSPHT_OK;
        bool ok = cudaStreamCreateWithFlags(&s_up, cudaStreamNonBlocking) == cudaSuccess &&
                  cudaStreamCreateWithFlags(&s_down, cudaStreamNonBlocking) == cudaSuccess;
        for (cudaEvent_t *e : {&ev_up, &ev_loaded, &ev_stored, &ev_down})
            ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
        // nothing in flight yet: the first waits pass at once
        ok = ok && cudaEventRecord(ev_up, s_up) == cudaSuccess &&
             cudaEventRecord(ev_loaded, stream) == cudaSuccess &&
             cudaEventRecord(ev_down, s_down) == cudaSuccess;
        if (!ok) {  // release what was made; a later call tries again
            cudaGetLastError();
            for (cudaEvent_t *e : {&ev_up, &ev_loaded, &ev_stored, &ev_down})
                if (*e) cudaEventDestroy(*e), *e = nullptr;
            for (cudaStream_t *st : {&s_up, &s_down})
                if (*st) cudaStreamDestroy(*st), *st = nullptr;
            err = "could not create the copy streams";
            return CSPHT_ECUDA;
        }
        io_ready = true;
        return CSPHT_OK;
    }
    // Orders the compute stream after an upload copy still in flight (before a
    // synchronous call reuses the staging buffer).
    bool io_fence() { return !io_ready || cudaStreamWaitEvent(stream, ev_up, 0) == cudaSuccess; }
    // Host wait for the copy streams.
    bool io_sync() {
        return !io_ready ||
               (cudaStreamSynchronize(s_up) == cudaSuccess && cudaStreamSynchronize(s_down) == cudaSuccess);
    }
    virtual int upload_f32_async(const float *U) = 0;
    virtual int download_f32_async(float *U) = 0;
    // events of cspht_batch_step: the step forks from the batch stream and
    // joins back into it
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr;
    virtual int create(const double *psi) = 0;
    virtual int set_state(const double *U, bool prim) = 0;
    virtual int get_state(double *U) = 0;
    virtual int set_state_f32(const float *U) = 0;
    virtual int get_state_f32(float *U) = 0;
    virtual int enqueue_step() = 0;  // one step, no sync
    virtual int totals(double out[6]) = 0;
    virtual void reset_graphs() = 0;
    virtual int autotune(int steps, double cfl, int *zchunk_out) = 0;
    virtual int set_tile_depth(int z) = 0;
    cudaStream_t own = nullptr, stream = nullptr;
    Ctrl *ctrl = nullptr;
    Ctrl *hctrl = nullptr;  // pinned mirror
    long long launches = 0;
    bool state_set = false;
    double cfl_dev = -1.0, tend_dev = -2.0;
    std::string err;

    // per-kernel event timing (cspht_profile)
    struct ProfRec {
        int kind;
        cudaEvent_t a, b;
    };
    bool prof_on = false;
    std::vector<ProfRec> prof;
    std::vector<cudaEvent_t> evpool;
    size_t evused = 0;
    cudaEvent_t next_event() {
        if (evused == evpool.size()) {
            cudaEvent_t e;
            if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
            evpool.push_back(e);
        }
        return evpool[evused++];
    }
    // Launches one kernel (the callable f) and counts it; brackets it with
    // events while profiling.
    template <class F>
    int launch(int kind, F &&f) {
        if (prof_on) {
            cudaEvent_t a = next_event(), b = next_event();
            if (a && b) {
                cudaEventRecord(a, stream);
                f();
                cudaEventRecord(b, stream);
                prof.push_back({kind, a, b});
                return 1;
            }
        }
        f();
        return 1;
    }
};

// z-chunk lengths chosen by cspht_autotune, per (grid, precision), for the
// handles this process creates later.
std::mutex zchunk_mu;
std::map<std::array<int, 4>, int> zchunk_tuned;
int zchunk_cache_get(int nx, int ny, int nz, int bytes) {
    std::lock_guard<std::mutex> g(zchunk_mu);
    auto it = zchunk_tuned.find({nx, ny, nz, bytes});
    return it == zchunk_tuned.end() ? 0 : it->second;
}
void zchunk_cache_put(int nx, int ny, int nz, int bytes, int z) {
    std::lock_guard<std::mutex> g(zchunk_mu);
    zchunk_tuned[{nx, ny, nz, bytes}] = z;
}

template <typename T>
struct Solver final : SolverBase {
    Grid G;
    Phys<T> P;
    int path;
    double h, gamma;
    char *pool = nullptr;  // all padded arrays
    size_t pool_bytes = 0;
    T *U[2][5];
    T *psi = nullptr;
    // plain-path scratch
    T *prim0[4], *Q[4], *Us[5], *S1rho, *S1u[3], *S1phi, *S1xi[3], *S2m[3], *S2E, *S2xi[3];
    T *F[3][5];
    T *grav[3];  // fast path: static lattice gravity D0[psi]
    T *rho_lo = nullptr;  // fast FP32 path: density compensation word
    CUtensorMap tmU[2][5], tmS[6];  // fast path: TMA descriptors

    // k_euler specialised on the limiter and the Riemann flux
    static void *euler_fn(int lim, int rk) {
        switch (lim * 3 + rk) {
            case 0: return (void *)k_euler<T, LTX, LTY, LIM_VANLEER, RIEMANN_LF>;
            case 1: return (void *)k_euler<T, LTX, LTY, LIM_VANLEER, RIEMANN_HLL>;
            case 2: return (void *)k_euler<T, LTX, LTY, LIM_VANLEER, RIEMANN_SWEPT>;
            case 3: return (void *)k_euler<T, LTX, LTY, LIM_MINMOD, RIEMANN_LF>;
            case 4: return (void *)k_euler<T, LTX, LTY, LIM_MINMOD, RIEMANN_HLL>;
            case 5: return (void *)k_euler<T, LTX, LTY, LIM_MINMOD, RIEMANN_SWEPT>;
            case 6: return (void *)k_euler<T, LTX, LTY, LIM_MC, RIEMANN_LF>;
            case 7: return (void *)k_euler<T, LTX, LTY, LIM_MC, RIEMANN_HLL>;
            default: return (void *)k_euler<T, LTX, LTY, LIM_MC, RIEMANN_SWEPT>;
        }
    }
    // k_lagrange with plain or compensated FP32 balance terms (the FP64 kernel has one form)
    static void *lagrange_fn(bool comp) {
        if (sizeof(T) == 4 && comp) return (void *)k_lagrange<T, LTX, LTY, true>;
        return (void *)k_lagrange<T, LTX, LTY, false>;
    }
    int zchunk = 1;
    static constexpr int LTX = 32, LTY = 8;
    double *staging = nullptr, *part = nullptr, *tot = nullptr;
    int cur = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    bool graph_tried[2] = {false, false};
    int kernels_per_step = 0;

    ~Solver() override {
        for (int p = 0; p < 2; ++p)
            if (gexec[p]) cudaGraphExecDestroy(gexec[p]);
        io_sync();  // copies into or out of the staging buffers
        // stream-ordered frees: after this handle's work, without a device-wide wait
        cudaStream_t fs = stream ? stream : own;
        dev_free(pool, fs);
        dev_free(split_pool, fs);
        dev_free(staging, fs);
        dev_free(staging_out, fs);
        dev_free(part, fs);
        dev_free(tot, fs);
        dev_free(ctrl, fs);
        if (fs && cudaStreamSynchronize(fs) != cudaSuccess) cudaGetLastError();  // nothing copies into hctrl now
        host_ctrl_free(hctrl);
        if (own) cudaStreamDestroy(own);
    }

    static constexpr int SPLIT_ARRAYS = 4 + 4 + 5 + 1 + 3 + 1 + 3 + 15;  // scratch of the unfused kernels
    char *split_pool = nullptr;  // that scratch, when a fused handle's autotune tries the unfused kernels

    // Points the unfused kernels' scratch arrays at SPLIT_ARRAYS consecutive
    // padded arrays from p.
    void assign_split(T *p) {
        auto take = [&]() {
            T *r = p;
            p += G.total;
            return r;
        };
        for (int e = 0; e < 4; ++e) prim0[e] = take();
        for (int e = 0; e < 4; ++e) Q[e] = take();
        for (int e = 0; e < 5; ++e) Us[e] = take();
        S1rho = take();
        for (int e = 0; e < 3; ++e) S1u[e] = take();
        S1phi = take();
        for (int e = 0; e < 3; ++e) S1xi[e] = take();
        for (int d = 0; d < 3; ++d)
            for (int f = 0; f < 5; ++f) F[d][f] = take();
    }

    int alloc_split() {
        if (split_pool) return CSPHT_OK;
        const size_t bytes = (size_t)SPLIT_ARRAYS * (size_t)G.total * sizeof(T);
        if (!dev_alloc(&split_pool, bytes, stream)) return CSPHT_ENOMEM;
        if (cudaMemsetAsync(split_pool, 0, bytes, stream) != cudaSuccess) {
            cudaGetLastError();
            dev_free(split_pool, stream);
            split_pool = nullptr;
            return CSPHT_ECUDA;
        }
        assign_split(reinterpret_cast<T *>(split_pool));
        return CSPHT_OK;
    }

    UPtr<T> Uc(int p) const {
        UPtr<T> u;
        for (int f = 0; f < 5; ++f) u.f[f] = U[p][f];
        return u;
    }

    dim3 cells_grid(int ex = 0, int ey = 0, int ez = 0) const {
        return dim3((G.n[0] + ex + BX - 1) / BX, (G.n[1] + ey + BY - 1) / BY, G.n[2] + ez);
    }

    int create(const double *hpsi) override {
        G = make_grid<T>(G.n[0], G.n[1], G.n[2]);
        int narr = 10 + 1 + 7;  // U ping-pong, psi, corrector content and offsets
        if (path == CSPHT_PATH_PLAIN) narr += 4 + 4 + 5 + 1 + 3 + 1 + 3 + 15;
        else narr += 3 + (sizeof(T) == 4 ? 1 : 0);  // lattice gravity (+ density compensation)
        pool_bytes = (size_t)narr * (size_t)G.total * sizeof(T);
        // every setup copy and kernel runs in order on the handle's own stream: the
        // stream does not synchronise with the legacy default stream, and a plain
        // cudaMemcpy from pageable memory may return before its data has landed
        // at the greatest priority: a handle created while others run (a server
        // admitting a request) gets its setup through ahead of their kernels
        int least_prio = 0, greatest_prio = 0;
        if (cudaDeviceGetStreamPriorityRange(&least_prio, &greatest_prio) != cudaSuccess) {
            cudaGetLastError();
            greatest_prio = 0;
        }
        if (cudaStreamCreateWithPriority(&own, cudaStreamNonBlocking, greatest_prio) != cudaSuccess)
            return fail_cuda("stream create");
        stream = own;
        if (!dev_alloc(&pool, pool_bytes, stream)) {
            err = "device allocation of " + std::to_string(pool_bytes) + " bytes failed";
            return CSPHT_ENOMEM;
        }
        if (cudaMemsetAsync(pool, 0, pool_bytes, stream) != cudaSuccess) return fail_cuda("memset");
        T *p = (T *)pool;
        auto take = [&]() {
            T *r = p;
            p += G.total;
            return r;
        };
        for (int b = 0; b < 2; ++b)
            for (int f = 0; f < 5; ++f) U[b][f] = take();
        psi = take();
        for (int e = 0; e < 3; ++e) S2m[e] = take();
        S2E = take();
        for (int e = 0; e < 3; ++e) S2xi[e] = take();
        if (path == CSPHT_PATH_PLAIN) {
            assign_split(p);
        } else {
            for (int e = 0; e < 3; ++e) grav[e] = take();
            if (sizeof(T) == 4) rho_lo = take();
        }
        long long N = G.cells();
        if (!dev_alloc(&staging, sizeof(double) * 5 * N, stream) ||
            !dev_alloc(&part, sizeof(double) * 6 * TOT_BLOCKS, stream) ||
            !dev_alloc(&tot, sizeof(double) * 6, stream) || !dev_alloc(&ctrl, sizeof(Ctrl), stream) ||
            !(hctrl = host_ctrl_alloc())) {
            err = "allocation of staging / control buffers failed";
            return CSPHT_ENOMEM;
        }
        Ctrl c0;
        memset(&c0, 0, sizeof c0);
        c0.t_end = INFINITY;
        c0.cfl = 0.4;
        *hctrl = c0;
        if (cudaMemcpyAsync(ctrl, hctrl, sizeof(Ctrl), cudaMemcpyHostToDevice, stream) != cudaSuccess)
            return fail_cuda("ctrl upload");
        // potential with its static ghost layer
        if (cudaMemcpyAsync(staging, hpsi, sizeof(double) * N, cudaMemcpyHostToDevice, stream) != cudaSuccess)
            return fail_cuda("psi upload");
        UPtr<T> pp;
        pp.f[0] = psi;
        k_load<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, staging, 1, pp);
        for (int a = 0; a < 3; ++a) {
            long long nt = ghost_pass_threads(G, a, 2);
            k_ghost_psi<T><<<(unsigned)((nt + 255) / 256), 256, 0, stream>>>(G, P, a, psi);
        }
        launches += 4;
        if (path == CSPHT_PATH_FAST) {
            k_gravity<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, P, psi, grav[0], grav[1], grav[2]);
            launches += 1;
            size_t sm = LagShape<LTX, LTY>::bytes<T>();
            if (cudaFuncSetAttribute(lagrange_fn(P.balance == CSPHT_BALANCE_COMPENSATED),
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm) != cudaSuccess)
                return fail_cuda("lagrange smem attribute");
            size_t se = EulShape<LTX, LTY>::smem_bytes<T>();
            bool ok = true;
            for (int l = 0; l < 3; ++l)      // every limiter
                for (int r = 0; r < 3; ++r)  // every Riemann flux
                    ok &= cudaFuncSetAttribute(euler_fn(l, r), cudaFuncAttributeMaxDynamicSharedMemorySize,
                                               (int)se) == cudaSuccess;
            if (!ok) return fail_cuda("euler smem attribute");
            // TMA descriptors: U^n boxes (both ping-pong buffers) and corrector-state boxes
            for (int b = 0; b < 2; ++b)
                for (int f = 0; f < 5; ++f)
                    if (!make_tmap<T>(&tmU[b][f], U[b][f], G, LTX + 8, LTY + 4)) {
                        err = "TMA descriptor encoding failed";
                        return CSPHT_ECUDA;
                    }
            const T *sf[6] = {S2m[0], S2m[1], S2m[2], S2E, S2xi[0], S2xi[1]};
            for (int f = 0; f < 6; ++f)
                if (!make_tmap<T>(&tmS[f], sf[f], G, LTX + 8, LTY + 2)) {
                    err = "TMA descriptor encoding failed";
                    return CSPHT_ECUDA;
                }
            int tiles = ((G.n[0] + LTX - 1) / LTX) * ((G.n[1] + LTY - 1) / LTY);
            int target = 148 * 8;
            int nch = (target + tiles - 1) / tiles;
            int maxch = (G.n[2] + 7) / 8;
            if (nch > maxch) nch = maxch;
            if (nch < 1) nch = 1;
            zchunk = (G.n[2] + nch - 1) / nch;
            const int tuned = zchunk_cache_get(G.n[0], G.n[1], G.n[2], (int)sizeof(T));
            if (tuned > 0) zchunk = tuned;  // chosen by cspht_autotune for this grid earlier
        }
        if (cudaStreamSynchronize(stream) != cudaSuccess) return fail_cuda("psi setup");
        return CSPHT_OK;
    }

    int fail_cuda(const char *what) {
        cudaError_t e = cudaGetLastError();
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return CSPHT_ECUDA;
    }

    int set_state(const double *hU, bool prim) override {
        long long N = G.cells();
        if (!io_fence() ||
            cudaMemcpyAsync(staging, hU, sizeof(double) * 5 * N, cudaMemcpyHostToDevice, stream) !=
            cudaSuccess)
            return fail_cuda("state upload");
        if (prim)
            k_load_prim<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, gamma, staging, Uc(cur));
        else
            k_load<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, staging, 5, Uc(cur));
        if (rho_lo) {
            k_rho_lo<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, staging, U[cur][0], rho_lo);
            launches += 1;
        }
        k_reset_state<<<1, 1, 0, stream>>>(ctrl);
        k_speed<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, P, Uc(cur), ctrl, path == CSPHT_PATH_FAST);
        launches += 3;
        if (cudaStreamSynchronize(stream) != cudaSuccess) return fail_cuda("set_state");
        state_set = true;
        return CSPHT_OK;
    }

    int get_state(double *hU) override {
        long long N = G.cells();
        if (!io_fence()) return fail_cuda("state download");
        k_store<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, Uc(cur), rho_lo, staging);
        launches += 1;
        if (cudaMemcpyAsync(hU, staging, sizeof(double) * 5 * N, cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess)
            return fail_cuda("state download");
        if (cudaStreamSynchronize(stream) != cudaSuccess) return fail_cuda("get_state");
        return CSPHT_OK;
    }

    // Single-precision host arrays: half the bytes of the FP64 calls.  The
    // upload is exact for an FP32 handle (its compensation word starts at 0).
    int set_state_f32(const float *hU) override {
        long long N = G.cells();
        const float *st = reinterpret_cast<const float *>(staging);
        if (!io_fence() ||
            cudaMemcpyAsync(staging, hU, sizeof(float) * 5 * N, cudaMemcpyHostToDevice, stream) != cudaSuccess)
            return fail_cuda("state upload");
        k_load<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, st, 5, Uc(cur));
        if (rho_lo) {
            if (cudaMemsetAsync(rho_lo, 0, (size_t)G.total * sizeof(T), stream) != cudaSuccess)
                return fail_cuda("state upload");
        }
        k_reset_state<<<1, 1, 0, stream>>>(ctrl);
        k_speed<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, P, Uc(cur), ctrl, path == CSPHT_PATH_FAST);
        launches += 3;
        if (cudaStreamSynchronize(stream) != cudaSuccess) return fail_cuda("set_state");
        state_set = true;
        return CSPHT_OK;
    }

    int get_state_f32(float *hU) override {
        long long N = G.cells();
        float *st = reinterpret_cast<float *>(staging);
        if (!io_fence()) return fail_cuda("state download");
        k_store<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, Uc(cur), rho_lo, st);
        launches += 1;
        if (cudaMemcpyAsync(hU, staging, sizeof(float) * 5 * N, cudaMemcpyDeviceToHost, stream) != cudaSuccess)
            return fail_cuda("state download");
        if (cudaStreamSynchronize(stream) != cudaSuccess) return fail_cuda("get_state");
        return CSPHT_OK;
    }

    // The upload copies into the staging buffer on the upload stream once the
    // previous upload was converted, then converts on the compute stream after
    // the copy: the same work as set_state_f32, without waiting on the host.
    int upload_f32_async(const float *hU) override {
        if (int rc = io_init()) return rc;
        const long long N = G.cells();
        const float *st = reinterpret_cast<const float *>(staging);
        if (cudaStreamWaitEvent(s_up, ev_loaded, 0) != cudaSuccess ||
            cudaMemcpyAsync(staging, hU, sizeof(float) * 5 * N, cudaMemcpyHostToDevice, s_up) != cudaSuccess ||
            cudaEventRecord(ev_up, s_up) != cudaSuccess || cudaStreamWaitEvent(stream, ev_up, 0) != cudaSuccess)
            return fail_cuda("asynchronous upload");
        k_load<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, st, 5, Uc(cur));
        if (rho_lo && cudaMemsetAsync(rho_lo, 0, (size_t)G.total * sizeof(T), stream) != cudaSuccess)
            return fail_cuda("asynchronous upload");
        k_reset_state<<<1, 1, 0, stream>>>(ctrl);
        k_speed<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, P, Uc(cur), ctrl, path == CSPHT_PATH_FAST);
        launches += 3;
        if (cudaEventRecord(ev_loaded, stream) != cudaSuccess) return fail_cuda("asynchronous upload");
        state_set = true;
        return CSPHT_OK;
    }

    // The download converts the state into its own staging buffer on the
    // compute stream once the previous download was read out of it, then copies
    // it to the host on the download stream.
    int download_f32_async(float *hU) override {
        if (int rc = io_init()) return rc;
        const long long N = G.cells();
        if (!staging_out && !dev_alloc(&staging_out, sizeof(float) * 5 * N, stream)) {
            err = "allocation of the download staging buffer failed";
            return CSPHT_ENOMEM;
        }
        if (cudaStreamWaitEvent(stream, ev_down, 0) != cudaSuccess) return fail_cuda("asynchronous download");
        k_store<T><<<cells_grid(), dim3(BX, BY), 0, stream>>>(G, Uc(cur), rho_lo, staging_out);
        launches += 1;
        if (cudaEventRecord(ev_stored, stream) != cudaSuccess || cudaStreamWaitEvent(s_down, ev_stored, 0) != cudaSuccess ||
            cudaMemcpyAsync(hU, staging_out, sizeof(float) * 5 * N, cudaMemcpyDeviceToHost, s_down) != cudaSuccess ||
            cudaEventRecord(ev_down, s_down) != cudaSuccess)
            return fail_cuda("asynchronous download");
        return CSPHT_OK;
    }
    float *staging_out = nullptr;  // output staging buffer of download_f32_async

    int totals(double out[6]) override {
        k_totals<T><<<TOT_BLOCKS, TOT_THREADS, 0, stream>>>(G, Uc(cur), rho_lo, psi, part);
        k_totals_final<<<1, TOT_THREADS, 0, stream>>>(part, TOT_BLOCKS, h * h * h, tot);
        launches += 2;
        if (cudaMemcpyAsync(out, tot, sizeof(double) * 6, cudaMemcpyDeviceToHost, stream) !=
            cudaSuccess)
            return fail_cuda("totals download");
        if (cudaStreamSynchronize(stream) != cudaSuccess) return fail_cuda("totals");
        return CSPHT_OK;
    }

    // ---- one step, plain path: k_dt, ghosts(U), prim, HFC-P, SUL-P,
    // ghosts(S1), HFC-C, SUL-C, ghosts(S2), FGC x3, SUE.
    int launch_plain(int p) {
        int q = 1 - p, nk = 0;
        UPtr<T> Un = Uc(p), Uo = Uc(q);
        dim3 blk(BX, BY);
        nk += launch(KK_DT, [&] { k_dt<<<1, 1, 0, stream>>>(ctrl, h); });
        nk += ghost_U(Un);
        dim3 gpad((G.n[0] + 2 + BX - 1) / BX, (G.n[1] + 2 + BY - 1) / BY, G.n[2] + 2);
        nk += launch(KK_PRIM, [&] {
            k_prim<T><<<gpad, blk, 0, stream>>>(G, P, Un, prim0[0], prim0[1], prim0[2], prim0[3]);
        });
        nk += launch(KK_HFC_PRED, [&] {
            k_hfc<T, false><<<cells_grid(), blk, 0, stream>>>(G, P, Un.f[0], prim0[0], prim0[1],
                                                               prim0[2], prim0[3], nullptr, nullptr,
                                                               nullptr, psi, Q[0], Q[1], Q[2], Q[3]);
        });
        UPtr<T> us;
        for (int f = 0; f < 5; ++f) us.f[f] = Us[f];
        S1Ptr<T> s1;
        s1.rho = S1rho;
        s1.phi = S1phi;
        for (int e = 0; e < 3; ++e) {
            s1.u[e] = S1u[e];
            s1.xi[e] = S1xi[e];
        }
        nk += launch(KK_SUL_PRED, [&] {
            k_sul_pred<T><<<cells_grid(), blk, 0, stream>>>(G, P, ctrl, Un, Q[0], Q[1], Q[2], Q[3],
                                                            prim0[0], prim0[1], prim0[2], us, s1);
        });
        for (int a = 0; a < 3; ++a) {
            long long nt = ghost_pass_threads(G, a);
            nk += launch(KK_GHOST_S1, [&] {
                k_ghost_S1<T><<<(unsigned)((nt + 255) / 256), 256, 0, stream>>>(G, P, a, s1, psi, ctrl);
            });
        }
        nk += launch(KK_HFC_CORR, [&] {
            k_hfc<T, true><<<cells_grid(), blk, 0, stream>>>(G, P, Un.f[0], S1u[0], S1u[1], S1u[2],
                                                              S1phi, S1xi[0], S1xi[1], S1xi[2], psi,
                                                              Q[0], Q[1], Q[2], Q[3]);
        });
        S2Ptr<T> s2;
        s2.E = S2E;
        for (int e = 0; e < 3; ++e) {
            s2.m[e] = S2m[e];
            s2.xi[e] = S2xi[e];
        }
        nk += launch(KK_SUL_CORR, [&] {
            k_sul_corr<T><<<cells_grid(), blk, 0, stream>>>(G, P, ctrl, Un, us, Q[0], Q[1], Q[2], Q[3],
                                                            prim0[0], prim0[1], prim0[2], s1, s2);
        });
        nk += ghost_S2(s2);
        UPtr<T> Fd[3];
        for (int d = 0; d < 3; ++d)
            for (int f = 0; f < 5; ++f) Fd[d].f[f] = F[d][f];
        nk += launch(KK_FGC, [&] {
            k_fgc<T><<<cells_grid(1, 0, 0), blk, 0, stream>>>(G, P, ctrl, 0, Un, s2, Fd[0]);
        });
        nk += launch(KK_FGC, [&] {
            k_fgc<T><<<cells_grid(0, 1, 0), blk, 0, stream>>>(G, P, ctrl, 1, Un, s2, Fd[1]);
        });
        nk += launch(KK_FGC, [&] {
            k_fgc<T><<<cells_grid(0, 0, 1), blk, 0, stream>>>(G, P, ctrl, 2, Un, s2, Fd[2]);
        });
        nk += launch(KK_SUE, [&] {
            k_sue<T><<<cells_grid(), blk, 0, stream>>>(G, P, ctrl, Un, s2, Fd[0], Fd[1], Fd[2], Uo);
        });
        return nk;
    }

    // Two ghost layers of U^n: one launch over the whole shell when the y and
    // z faces are periodic or outflow, else one pass per axis.  zfaces =
    // false: the caller's kernels wrap a periodic z themselves (the fused
    // kernels), so the shell leaves out the z faces.
    int ghost_U(UPtr<T> Un, bool zfaces = true) {
        if (copy_faces_yz(P.bc)) {
            const long long nt = shell_threads(G, 2, zfaces);
            return launch(KK_GHOST_U, [&] {
                k_ghost_U_shell<T><<<(unsigned)((nt + 255) / 256), 256, 0, stream>>>(G, P, Un, psi);
            });
        }
        int nk = 0;
        for (int a = 0; a < 3; ++a) {
            long long nt = ghost_pass_threads(G, a, 2);
            nk += launch(KK_GHOST_U, [&] {
                k_ghost_U<T><<<(unsigned)((nt + 255) / 256), 256, 0, stream>>>(G, P, a, Un, psi);
            });
        }
        return nk;
    }

    // axis_xi: for the fused Eulerian kernel, which reads of a ghost's offset
    // only the component along its face's axis (ghost_S2_shell_at).
    int ghost_S2(S2Ptr<T> s2, bool zfaces = true, bool axis_xi = false) {
        if (copy_faces_yz(P.bc)) {
            const long long nt = shell_threads(G, 1, zfaces);
            return launch(KK_GHOST_S2, [&] {
                k_ghost_S2_shell<T><<<(unsigned)((nt + 255) / 256), 256, 0, stream>>>(G, P, s2, ctrl, axis_xi);
            });
        }
        int nk = 0;
        for (int a = 0; a < 3; ++a) {
            long long nt = ghost_pass_threads(G, a);
            nk += launch(KK_GHOST_S2, [&] {
                k_ghost_S2<T><<<(unsigned)((nt + 255) / 256), 256, 0, stream>>>(G, P, a, s2, ctrl);
            });
        }
        return nk;
    }

    S2Ptr<T> s2() const {
        S2Ptr<T> v;
        v.E = S2E;
        for (int e = 0; e < 3; ++e) {
            v.m[e] = S2m[e];
            v.xi[e] = S2xi[e];
        }
        return v;
    }

    // Arguments of the fused kernels for a step from U[p] to U[1-p].
    LagArgs<T> lag_args(int p) const {
        LagArgs<T> A;
        for (int f = 0; f < 5; ++f) A.tmU.m[f] = tmU[p][f];
        A.G = G;
        A.P = P;
        for (int f = 0; f < 5; ++f) A.U[f] = U[p][f];
        A.psi = psi;
        for (int e = 0; e < 3; ++e) {
            A.grav[e] = grav[e];
            A.m[e] = S2m[e];
            A.xi[e] = S2xi[e];
        }
        A.E = S2E;
        A.ctrl = ctrl;
        A.zchunk = zchunk;
        return A;
    }
    EulArgs<T> eul_args(int p) const {
        EulArgs<T> B;
        for (int f = 0; f < 5; ++f) B.tmU.m[f] = tmU[p][f];
        for (int f = 0; f < 6; ++f) B.tmS.m[f] = tmS[f];
        B.G = G;
        B.P = P;
        for (int f = 0; f < 5; ++f) {
            B.U[f] = U[p][f];
            B.Un[f] = U[1 - p][f];
        }
        for (int e = 0; e < 3; ++e) {
            B.m[e] = S2m[e];
            B.xi[e] = S2xi[e];
        }
        B.E = S2E;
        B.rho_lo = rho_lo;
        B.ctrl = ctrl;
        B.zchunk = zchunk;
        return B;
    }

    // ---- one step, fast path: k_dt, ghosts(U), Lagrangian stage, ghosts(S2), Euler stage.
    int launch_fast(int p) {
        int nk = 0;
        UPtr<T> Un = Uc(p);
        nk += launch(KK_DT, [&] { k_dt<<<1, 1, 0, stream>>>(ctrl, h); });
        // the fused kernels wrap a periodic z (map_coord): no z ghost faces then
        const bool zfaces = P.bc[4] != BC_PERIODIC;
        nk += ghost_U(Un, zfaces);
        LagArgs<T> A = lag_args(p);
        dim3 lg((G.n[0] + LTX - 1) / LTX, (G.n[1] + LTY - 1) / LTY, (G.n[2] + zchunk - 1) / zchunk);
        size_t sm = LagShape<LTX, LTY>::bytes<T>();
        void *lfn = lagrange_fn(P.balance == CSPHT_BALANCE_COMPENSATED);
        void *largs[] = {&A};
        nk += launch(KK_LAGRANGE,
                     [&] { cudaLaunchKernel(lfn, lg, dim3(LagShape<LTX, LTY>::threads<T>()), largs, sm, stream); });
        nk += ghost_S2(s2(), zfaces, true);
        EulArgs<T> B = eul_args(p);
        size_t se = EulShape<LTX, LTY>::smem_bytes<T>();
        void *fn = euler_fn(P.limiter, P.riemann);
        void *args[] = {&B};
        nk += launch(KK_EULER, [&] { cudaLaunchKernel(fn, lg, dim3(LTX * LTY), args, se, stream); });
        return nk;
    }

    int launch_step(int p) { return path == CSPHT_PATH_PLAIN ? launch_plain(p) : launch_fast(p); }

    // Chooses the z extent of the fused kernels' tiles (zchunk planes per CTA
    // column) by timing `steps` steps per candidate on the current state, which
    // is saved first and restored after every trial.  A chunk recomputes two
    // predictor planes at its start; fewer, longer chunks save that work,
    // more chunks fill the SMs in fuller waves.
    int autotune(int steps, double cfl, int *zout) override {
        if (path != CSPHT_PATH_FAST) {  // the unfused kernels have no tile depth to tune
            if (zout) *zout = 0;
            return CSPHT_OK;
        }
        int rc = CSPHT_OK;
        const size_t fb = (size_t)G.total * sizeof(T);
        const size_t lb = rho_lo ? (size_t)G.total * sizeof(T) : 0;
        char *save = nullptr;
        if (cudaMalloc(&save, 5 * fb + lb + sizeof(Ctrl)) != cudaSuccess) {
            cudaGetLastError();
            err = "autotune: no room for the state snapshot";
            return CSPHT_ENOMEM;
        }
        const int cur0 = cur;
        auto copy = [&](bool restore) {
            for (int f = 0; f < 5; ++f) {
                void *d = restore ? (void *)U[cur0][f] : (void *)(save + f * fb);
                const void *sr = restore ? (const void *)(save + f * fb) : (const void *)U[cur0][f];
                cudaMemcpyAsync(d, sr, fb, cudaMemcpyDeviceToDevice, stream);
            }
            if (rho_lo) {
                if (restore) cudaMemcpyAsync(rho_lo, save + 5 * fb, lb, cudaMemcpyDeviceToDevice, stream);
                else cudaMemcpyAsync(save + 5 * fb, rho_lo, lb, cudaMemcpyDeviceToDevice, stream);
            }
            if (restore) cudaMemcpyAsync(ctrl, save + 5 * fb + lb, sizeof(Ctrl), cudaMemcpyDeviceToDevice, stream);
            else cudaMemcpyAsync(save + 5 * fb + lb, ctrl, sizeof(Ctrl), cudaMemcpyDeviceToDevice, stream);
            cur = cur0;
        };
        copy(false);
        // candidate chunk counts (deduplicated by the chunk length they give),
        // down to chunks of 4 planes: small grids need the CTAs more than they
        // lose to the two recomputed predictor planes of each chunk
        const int nz = G.n[2], maxch = (nz + 3) / 4;
        static const int NCH[] = {1, 2, 3, 4, 5, 6, 8, 10, 12, 16, 24, 32, 48, 64};
        std::vector<int> cand;
        for (int c : NCH) {
            if (c > maxch) break;
            const int z = (nz + c - 1) / c;
            if (cand.empty() || cand.back() != z) cand.push_back(z);
        }
        if (std::find(cand.begin(), cand.end(), zchunk) == cand.end()) cand.push_back(zchunk);
        cudaEvent_t a = nullptr, b = nullptr;
        cudaEventCreate(&a);
        cudaEventCreate(&b);
        int best = zchunk;
        float best_ms = 0.0f;
        // times `steps` steps of the current configuration from the snapshot
        auto trial = [&](float &ms) -> int {
            reset_graphs();
            copy(true);
            k_set_params<<<1, 1, 0, stream>>>(ctrl, cfl, INFINITY);  // the snapshot's ctrl has the caller's
            launches += 1;
            int r = enqueue_step();  // captures the graph
            if (r != CSPHT_OK) return r;
            cudaEventRecord(a, stream);
            for (int i = 0; i < steps && r == CSPHT_OK; ++i) r = enqueue_step();
            cudaEventRecord(b, stream);
            if (r != CSPHT_OK) return r;
            if (cudaEventSynchronize(b) != cudaSuccess) return fail_cuda("autotune");
            cudaEventElapsedTime(&ms, a, b);
            return CSPHT_OK;
        };
        for (int z : cand) {
            zchunk = z;
            float ms = 0.0f;
            if ((rc = trial(ms)) != CSPHT_OK) break;
            if (best_ms == 0.0f || ms < best_ms) {
                best_ms = ms;
                best = z;
            }
        }
        // Fused or split stages: in FP64 the unfused kernels (one per paper
        // kernel, global scratch between them) beat the fused ones on the
        // smallest grids, where the fused tiles' recomputed halos and one CTA
        // per SM leave the GPU idle.  (FP32 fused kernels were faster at every
        // size measured, 32^3 to 256^3, so FP32 handles do not try them.)
        bool split = false;
        if (sizeof(T) == 8 && rc == CSPHT_OK && alloc_split() == CSPHT_OK) {
            path = CSPHT_PATH_PLAIN;
            float ms = 0.0f;
            rc = trial(ms);
            split = rc == CSPHT_OK && ms < best_ms;
            path = CSPHT_PATH_FAST;
        }
        cudaEventDestroy(a);
        cudaEventDestroy(b);
        zchunk = best;
        if (split) {
            path = CSPHT_PATH_PLAIN;
        } else if (split_pool) {
            dev_free(split_pool, stream);
            split_pool = nullptr;
        }
        reset_graphs();
        copy(true);
        cfl_dev = -1.0;  // the restored control word holds the caller's step parameters:
        tend_dev = -2.0; // the next advance or run sets its own
        if (cudaStreamSynchronize(stream) != cudaSuccess && rc == CSPHT_OK) rc = fail_cuda("autotune restore");
        cudaFree(save);
        if (rc == CSPHT_OK) zchunk_cache_put(G.n[0], G.n[1], G.n[2], (int)sizeof(T), best);
        if (zout) *zout = split ? 0 : best;
        return rc;
    }

    int set_tile_depth(int z) override {
        if (path != CSPHT_PATH_FAST) return CSPHT_OK;  // no tiles on the unfused path
        zchunk = z < G.n[2] ? z : G.n[2];
        reset_graphs();
        return CSPHT_OK;
    }

    void reset_graphs() override {
        for (int p = 0; p < 2; ++p) {
            if (gexec[p]) cudaGraphExecDestroy(gexec[p]);
            gexec[p] = nullptr;
            graph_tried[p] = false;
        }
    }

    int enqueue_step() override {
        int p = cur;
        // inside a caller's capture (cspht_batch_step) the kernels are captured
        // directly: a graph cannot be launched into a capturing stream
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        if (stream != nullptr && cudaStreamIsCapturing(stream, &cap) == cudaSuccess &&
            cap != cudaStreamCaptureStatusNone) {
            launches += launch_step(p);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) {
                err = std::string("step capture: ") + cudaGetErrorString(e);
                return CSPHT_ECUDA;
            }
            cur = 1 - cur;
            return CSPHT_OK;
        }
        bool capturable = !prof_on && stream != nullptr && stream != cudaStreamLegacy &&
                          stream != cudaStreamPerThread;
        if (capturable && !graph_tried[p]) {
            graph_tried[p] = true;
            cudaGraph_t g = nullptr;
            if (cudaStreamBeginCapture(stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                int nk = launch_step(p);
                if (cudaStreamEndCapture(stream, &g) == cudaSuccess && g) {
                    if (cudaGraphInstantiate(&gexec[p], g, 0) != cudaSuccess) gexec[p] = nullptr;
                    kernels_per_step = nk;
                    cudaGraphDestroy(g);
                }
            }
            cudaGetLastError();
        }
        if (gexec[p] && !prof_on) {
            if (cudaGraphLaunch(gexec[p], stream) != cudaSuccess) return fail_cuda("graph launch");
            launches += kernels_per_step;
        } else {
            launches += launch_step(p);
            cudaError_t e = cudaGetLastError();
            if (e != cudaSuccess) {
                err = std::string("step launch: ") + cudaGetErrorString(e);
                return CSPHT_ECUDA;
            }
        }
        cur = 1 - cur;
        return CSPHT_OK;
    }
};


// ------------------------------------------- many grids, one launch per kernel
//
// A batch advances several handles (its members) in lockstep with one launch
// of each step kernel for all of them: their dt (each member its own), their
// ghost shells, and the two fused stages as persistent kernels that take
// (member, tile, z chunk) items from a device counter.  Items are ordered by
// decreasing z extent, so the long tiles start first and the short ones fill
// the tail.  The fused stages take their members' arguments (tensor-map
// descriptors included) as one kernel parameter, so a launch holds a group of
// up to group_size() members and a larger batch launches once per group; the
// ghost and dt kernels read theirs from device memory.  Argument sets exist
// for both ping-pong parities of the state buffers.

template <typename T>
struct ShellU {  // the U^n ghost shell of one member
    Grid G;
    Phys<T> P;
    UPtr<T> U;
    const T *psi;
    long long threads;
};

template <typename T>
struct ShellS2 {  // the corrector-state ghost shell of one member
    Grid G;
    Phys<T> P;
    S2Ptr<T> S;
    const Ctrl *ctrl;
    long long threads;
    bool axis_xi;  // as Solver::ghost_S2 (the batch runs the fused kernels)
};

struct MemberCtl {
    Ctrl *ctrl;
    double h;
};

template <typename T>
__global__ void k_ghost_U_shell_multi(const ShellU<T> *__restrict__ a) {
    const ShellU<T> &g = a[blockIdx.y];
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < g.threads) ghost_U_shell_at(g.G, g.P, g.U, g.psi, t);
}

template <typename T>
__global__ void k_ghost_S2_shell_multi(const ShellS2<T> *__restrict__ a) {
    const ShellS2<T> &g = a[blockIdx.y];
    const long long t = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (t < g.threads) ghost_S2_shell_at(g.G, g.P, g.S, g.ctrl, t, g.axis_xi);
}

// The start of a step of every member, and the reset of the tile counters.
__global__ void k_dt_multi(const MemberCtl *__restrict__ m, int n, int *__restrict__ counters, int ncounters) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) dt_update(m[i].ctrl, m[i].h);
    for (int i = threadIdx.x; i < ncounters; i += blockDim.x) counters[i] = 0;
}

__global__ void k_set_params_multi(const MemberCtl *__restrict__ m, int n, double cfl, double t_end) {
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        m[i].ctrl->cfl = cfl;
        m[i].ctrl->t_end = t_end;
    }
}

struct BatchBase {
    virtual ~BatchBase() {}
    virtual int advance(long nsteps, double cfl, cudaStream_t st) = 0;
    long long launches = 0;
    std::string err;
};

template <typename T>
struct Batch final : BatchBase {
    static constexpr int LTX = Solver<T>::LTX, LTY = Solver<T>::LTY;
    static constexpr int GS = group_size<T>();  // members per fused-stage launch
    std::vector<Solver<T> *> m;
    int depth = 32;           // z extent of a tile item (make_batch sets it)
    std::vector<int> cur0;    // each member's buffer parity when the arguments were built
    int q = 0;                // parity of the next step relative to cur0
    char *dev = nullptr;      // device copy of `host`
    std::vector<char> host;   // ghost and dt arguments, items, counters (kept until the next build)
    size_t off_su[2], off_ss, off_mc, off_maps, off_items, off_cnt;
    static constexpr int MAPS = 16;  // descriptors per member: U^n of both parities (2 x 5), corrector state (6)
    // fused-stage launches: one per group of up to GS members
    struct Group {
        int first, count;        // members [first, first + count)
        size_t items_off;        // into the item list (host index)
        int nitems;
    };
    std::vector<Group> groups;
    std::vector<LagGroup<T>> lagg[2];
    std::vector<EulGroup<T>> eulg[2];
    int grid = 0;
    unsigned ublocks = 0, sblocks = 0;
    void *lfn = nullptr, *efn = nullptr;
    size_t lsm = 0, esm = 0;
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    cudaStream_t gstream[2] = {nullptr, nullptr};
    cudaEvent_t ev = nullptr;
    double cfl_dev = -1.0;
    cudaStream_t last = nullptr;  // stream of the last advance

    ~Batch() override {
        // kernels in flight read the arguments (and the members' memory, which
        // the members free after this, stream-ordered on their own streams)
        if (dev) cudaStreamSynchronize(last);
        for (int p = 0; p < 2; ++p)
            if (gexec[p]) cudaGraphExecDestroy(gexec[p]);
        if (ev) cudaEventDestroy(ev);
        dev_free(dev, last);
    }

    template <typename X>
    X *at(size_t off) { return reinterpret_cast<X *>(dev + off); }

    void reset_graphs() {
        for (int p = 0; p < 2; ++p) {
            if (gexec[p]) cudaGraphExecDestroy(gexec[p]);
            gexec[p] = nullptr;
            gstream[p] = nullptr;
        }
    }

    // Lays out and uploads every member's arguments and the work lists.
    int build(cudaStream_t st) {
        const int n = (int)m.size();
        if (dev && cudaStreamSynchronize(st) != cudaSuccess) return fail("batch rebuild");
        reset_graphs();
        auto align = [](size_t x) { return (x + 255) / 256 * 256; };
        size_t o = 0;
        for (int p = 0; p < 2; ++p) { off_su[p] = o; o = align(o + sizeof(ShellU<T>) * n); }
        off_ss = o; o = align(o + sizeof(ShellS2<T>) * n);
        off_mc = o; o = align(o + sizeof(MemberCtl) * n);
        off_maps = o; o = align(o + sizeof(CUtensorMap) * MAPS * n);
        // members in groups of up to GS, each group's items ordered by
        // decreasing z extent (member indices local to the group)
        groups.clear();
        std::vector<TileItem> items;
        for (int g0 = 0; g0 < n; g0 += GS) {
            Group gr{g0, std::min(GS, n - g0), items.size(), 0};
            std::vector<TileItem> gi;
            for (int i = 0; i < gr.count; ++i) {
                const Grid &G = m[g0 + i]->G;
                const int d = std::min(depth, G.n[2]);
                for (int bz = 0; bz * d < G.n[2]; ++bz)
                    for (int by = 0; by * LTY < G.n[1]; ++by)
                        for (int bx = 0; bx * LTX < G.n[0]; ++bx) gi.push_back({i, bx, by, bz});
            }
            auto extent = [&](const TileItem &w) {
                const int nz = m[g0 + w.member]->G.n[2], d = std::min(depth, nz);
                return std::min(d, nz - w.bz * d);
            };
            std::stable_sort(gi.begin(), gi.end(),
                             [&](const TileItem &a, const TileItem &b) { return extent(a) > extent(b); });
            gr.nitems = (int)gi.size();
            items.insert(items.end(), gi.begin(), gi.end());
            groups.push_back(gr);
        }
        off_items = o; o = align(o + sizeof(TileItem) * items.size());
        off_cnt = o; o = align(o + 2 * sizeof(int) * groups.size());
        dev_free(dev, st);  // stream-ordered: no wait for the whole device
        dev = nullptr;
        if (!dev_alloc(&dev, o, st)) {
            err = "batch: device allocation failed";
            return CSPHT_ENOMEM;
        }
        host.assign(o, 0);
        ublocks = sblocks = 0;
        cur0.resize(n);
        for (int p = 0; p < 2; ++p) {
            lagg[p].assign(groups.size(), LagGroup<T>{});
            eulg[p].assign(groups.size(), EulGroup<T>{});
        }
        for (int i = 0; i < n; ++i) {
            Solver<T> &s = *m[i];
            cur0[i] = s.cur;
            const int g = i / GS, k = i % GS;
            // the member's descriptors, copied into device memory
            const size_t mo = off_maps + sizeof(CUtensorMap) * MAPS * i;
            const CUtensorMap *dmaps = at<CUtensorMap>(mo);
            for (int p = 0; p < 2; ++p)
                for (int f = 0; f < 5; ++f)
                    memcpy(&host[mo + sizeof(CUtensorMap) * (5 * p + f)], &s.tmU[s.cur ^ p][f], sizeof(CUtensorMap));
            for (int f = 0; f < 6; ++f)
                memcpy(&host[mo + sizeof(CUtensorMap) * (10 + f)], &s.tmS[f], sizeof(CUtensorMap));
            for (int p = 0; p < 2; ++p) {
                const int b = s.cur ^ p;
                LagArgs<T> A = s.lag_args(b);
                EulArgs<T> B = s.eul_args(b);
                A.zchunk = B.zchunk = std::min(depth, s.G.n[2]);
                lagg[p][g].a[k] = lag_ref(A, dmaps + 5 * p);
                eulg[p][g].a[k] = eul_ref(B, dmaps + 5 * p, dmaps + 10);
                ShellU<T> su{s.G, s.P, s.Uc(b), s.psi, shell_threads(s.G, 2, s.P.bc[4] != BC_PERIODIC)};
                memcpy(&host[off_su[p] + sizeof(ShellU<T>) * i], &su, sizeof su);
            }
            ShellS2<T> ss{s.G, s.P, s.s2(), s.ctrl, shell_threads(s.G, 1, s.P.bc[4] != BC_PERIODIC), true};
            memcpy(&host[off_ss + sizeof(ShellS2<T>) * i], &ss, sizeof ss);
            MemberCtl mc{s.ctrl, s.h};
            memcpy(&host[off_mc + sizeof(MemberCtl) * i], &mc, sizeof mc);
            ublocks = std::max(ublocks, (unsigned)((shell_threads(s.G, 2, s.P.bc[4] != BC_PERIODIC) + 255) / 256));
            sblocks = std::max(sblocks, (unsigned)((shell_threads(s.G, 1, s.P.bc[4] != BC_PERIODIC) + 255) / 256));
        }
        memcpy(&host[off_items], items.data(), sizeof(TileItem) * items.size());
        // every copy and kernel in order on the batch's stream (see Solver::create)
        if (cudaMemcpyAsync(dev, host.data(), o, cudaMemcpyHostToDevice, st) != cudaSuccess)
            return fail("batch upload");
        const Solver<T> &s0 = *m[0];
        lfn = lagrange_multi_fn(s0.P.balance == CSPHT_BALANCE_COMPENSATED);
        efn = euler_multi_fn(s0.P.limiter, s0.P.riemann);
        lsm = LagShape<LTX, LTY>::template bytes<T>();
        esm = EulShape<LTX, LTY>::template smem_bytes<T>();
        if (cudaFuncSetAttribute(lfn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm) != cudaSuccess ||
            cudaFuncSetAttribute(efn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)esm) != cudaSuccess)
            return fail("batch smem attribute");
        int dev_id = 0, sms = 0, bl = 0, be = 0;
        if (cudaGetDevice(&dev_id) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev_id) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, lfn, LagShape<LTX, LTY>::template threads<T>(), lsm) !=
                cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&be, efn, LTX * LTY, esm) != cudaSuccess)
            return fail("batch occupancy");
        grid = std::max(1, sms * std::max(1, std::min(bl, be)));
        q = 0;
        // the arguments are in place before any stream reads them
        if (cudaStreamSynchronize(st) != cudaSuccess) return fail("batch upload");
        return CSPHT_OK;
    }

    // The arguments with descriptor pointers (maps: device copies) in place
    // of the descriptors.
    static LagArgs<T, MapsAt> lag_ref(const LagArgs<T> &a, const CUtensorMap *maps) {
        LagArgs<T, MapsAt> r;
        for (int f = 0; f < 5; ++f) {
            r.tmU.m[f] = maps + f;
            r.U[f] = a.U[f];
        }
        r.G = a.G;
        r.P = a.P;
        r.psi = a.psi;
        for (int e = 0; e < 3; ++e) {
            r.grav[e] = a.grav[e];
            r.m[e] = a.m[e];
            r.xi[e] = a.xi[e];
        }
        r.E = a.E;
        r.ctrl = a.ctrl;
        r.zchunk = a.zchunk;
        return r;
    }
    static EulArgs<T, MapsAt> eul_ref(const EulArgs<T> &a, const CUtensorMap *umaps, const CUtensorMap *smaps) {
        EulArgs<T, MapsAt> r;
        for (int f = 0; f < 5; ++f) {
            r.tmU.m[f] = umaps + f;
            r.U[f] = a.U[f];
            r.Un[f] = a.Un[f];
        }
        for (int f = 0; f < 6; ++f) r.tmS.m[f] = smaps + f;
        r.G = a.G;
        r.P = a.P;
        for (int e = 0; e < 3; ++e) {
            r.m[e] = a.m[e];
            r.xi[e] = a.xi[e];
        }
        r.E = a.E;
        r.rho_lo = a.rho_lo;
        r.ctrl = a.ctrl;
        r.zchunk = a.zchunk;
        return r;
    }

    static void *lagrange_multi_fn(bool comp) {
        if (sizeof(T) == 4 && comp) return (void *)k_lagrange_multi<T, LTX, LTY, true>;
        return (void *)k_lagrange_multi<T, LTX, LTY, false>;
    }
    static void *euler_multi_fn(int lim, int rk) {
        switch (lim * 3 + rk) {
            case 0: return (void *)k_euler_multi<T, LTX, LTY, LIM_VANLEER, RIEMANN_LF>;
            case 1: return (void *)k_euler_multi<T, LTX, LTY, LIM_VANLEER, RIEMANN_HLL>;
            case 2: return (void *)k_euler_multi<T, LTX, LTY, LIM_VANLEER, RIEMANN_SWEPT>;
            case 3: return (void *)k_euler_multi<T, LTX, LTY, LIM_MINMOD, RIEMANN_LF>;
            case 4: return (void *)k_euler_multi<T, LTX, LTY, LIM_MINMOD, RIEMANN_HLL>;
            case 5: return (void *)k_euler_multi<T, LTX, LTY, LIM_MINMOD, RIEMANN_SWEPT>;
            case 6: return (void *)k_euler_multi<T, LTX, LTY, LIM_MC, RIEMANN_LF>;
            case 7: return (void *)k_euler_multi<T, LTX, LTY, LIM_MC, RIEMANN_HLL>;
            default: return (void *)k_euler_multi<T, LTX, LTY, LIM_MC, RIEMANN_SWEPT>;
        }
    }

    int fail(const char *what) {
        cudaError_t e = cudaGetLastError();
        err = std::string(what) + ": " + cudaGetErrorString(e);
        return CSPHT_ECUDA;
    }

    // The launches of one step of every member, with argument set p: dt, the
    // U^n shells, the Lagrangian stage per group, the corrector-state shells,
    // the Eulerian stage per group.
    void launch_step(int p, cudaStream_t st) {
        const int n = (int)m.size(), ng = (int)groups.size();
        k_dt_multi<<<1, 256, 0, st>>>(at<MemberCtl>(off_mc), n, at<int>(off_cnt), 2 * ng);
        k_ghost_U_shell_multi<T><<<dim3(ublocks, n), 256, 0, st>>>(at<ShellU<T>>(off_su[p]));
        for (int g = 0; g < ng; ++g) {
            const TileItem *it = at<TileItem>(off_items) + groups[g].items_off;
            int ni = groups[g].nitems, *cnt = at<int>(off_cnt) + 2 * g;
            void *args[] = {&lagg[p][g], &it, &ni, &cnt};
            cudaLaunchKernel(lfn, dim3(std::min(grid, ni)), dim3(LagShape<LTX, LTY>::template threads<T>()), args, lsm,
                             st);
        }
        k_ghost_S2_shell_multi<T><<<dim3(sblocks, n), 256, 0, st>>>(at<ShellS2<T>>(off_ss));
        for (int g = 0; g < ng; ++g) {
            const TileItem *it = at<TileItem>(off_items) + groups[g].items_off;
            int ni = groups[g].nitems, *cnt = at<int>(off_cnt) + 2 * g + 1;
            void *args[] = {&eulg[p][g], &it, &ni, &cnt};
            cudaLaunchKernel(efn, dim3(std::min(grid, ni)), dim3(LTX * LTY), args, esm, st);
        }
        launches += 3 + 2 * ng;
    }

    int advance(long nsteps, double cfl, cudaStream_t st) override {
        const int n = (int)m.size();
        // a member stepped on its own since the build: its buffers no longer
        // match the argument sets
        bool stale = !dev;
        for (int i = 0; i < n && !stale; ++i) stale = m[i]->cur != (cur0[i] ^ q);
        if (stale) {
            if (int rc = build(st)) return rc;
        }
        if (!ev && cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return fail("batch event");
        // order the batch after each member's own work, and each member's later
        // work after the batch
        for (Solver<T> *s : m) {
            if (!s->ev_fork && (cudaEventCreateWithFlags(&s->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                                cudaEventCreateWithFlags(&s->ev_join, cudaEventDisableTiming) != cudaSuccess))
                return s->ev_fork = nullptr, fail("batch event");
            if (s->stream != st && (cudaEventRecord(s->ev_fork, s->stream) != cudaSuccess ||
                                    cudaStreamWaitEvent(st, s->ev_fork, 0) != cudaSuccess))
                return fail("batch fork");
        }
        if (cfl != cfl_dev) {
            k_set_params_multi<<<1, 256, 0, st>>>(at<MemberCtl>(off_mc), n, cfl, INFINITY);
            launches += 1;
            cfl_dev = cfl;
            for (Solver<T> *s : m) {
                s->cfl_dev = cfl;
                s->tend_dev = INFINITY;
            }
        }
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        const bool capturing = cudaStreamIsCapturing(st, &cap) == cudaSuccess && cap != cudaStreamCaptureStatusNone;
        const bool graphable = !capturing && st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
        const long per_step = 3 + 2 * (long)groups.size();
        long done = 0;
        while (done < nsteps) {
            if (graphable && nsteps - done >= 2) {
                // two steps (both parities) replayed from a graph captured on first use
                if (!gexec[q] || gstream[q] != st) {
                    if (gexec[q]) cudaGraphExecDestroy(gexec[q]);
                    gexec[q] = nullptr;
                    cudaGraph_t g = nullptr;
                    if (cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                        launch_step(q, st);
                        launch_step(q ^ 1, st);
                        launches -= 2 * per_step;
                        if (cudaStreamEndCapture(st, &g) == cudaSuccess && g) {
                            if (cudaGraphInstantiate(&gexec[q], g, 0) != cudaSuccess) gexec[q] = nullptr;
                            cudaGraphDestroy(g);
                        }
                    }
                    cudaGetLastError();
                    gstream[q] = st;
                }
                if (gexec[q]) {
                    if (cudaGraphLaunch(gexec[q], st) != cudaSuccess) return fail("batch graph launch");
                    launches += 2 * per_step;
                    done += 2;  // two flips of every member's buffers and of q: no change
                    continue;
                }
            }
            launch_step(q, st);
            if (cudaGetLastError() != cudaSuccess) return fail("batch step launch");
            for (Solver<T> *s : m) s->cur = 1 - s->cur;
            q ^= 1;
            done += 1;
        }
        last = st;
        if (cudaEventRecord(ev, st) != cudaSuccess) return fail("batch join");
        for (Solver<T> *s : m)
            if (s->stream != st && cudaStreamWaitEvent(s->stream, ev, 0) != cudaSuccess) return fail("batch join");
        return CSPHT_OK;
    }
};

}  // namespace

// Grid sizes the handles support: at most 2^20 cells per axis, nz within the
// launch grid's z limit, and padded arrays addressable with 32-bit offsets
// (the fused kernels' address arithmetic).
static bool grid_size_ok(int nx, int ny, int nz) {
    if (nx > (1 << 20) || ny > (1 << 20) || nz > (1 << 20)) return false;
    if ((long long)nz > 65535 - 2) return false;
    const long long px = nx + 2 * GH + 32, total = px * (ny + 2 * GH) * (long long)(nz + 2 * GH);
    return total < (1ll << 31);
}

struct cspht_sim {
    SolverBase *s = nullptr;
    int precision = 64;
};

struct cspht_batch {
    BatchBase *b = nullptr;
};

template <typename T>
static int make_batch(cspht_t *handles, int n, int depth, BatchBase **out) {
    auto *b = new (std::nothrow) Batch<T>;
    if (!b) return CSPHT_ENOMEM;
    b->depth = depth > 0 ? depth : 32;
    int rc = CSPHT_OK;
    for (int i = 0; i < n && rc == CSPHT_OK; ++i) {
        Solver<T> *s = static_cast<Solver<T> *>(handles[i]->s);
        const Solver<T> *f = b->m.empty() ? s : b->m[0];
        if (s->path != CSPHT_PATH_FAST || !copy_faces_yz(s->P.bc) || s->P.limiter != f->P.limiter ||
            s->P.riemann != f->P.riemann || s->P.balance != f->P.balance ||
            std::find(b->m.begin(), b->m.end(), s) != b->m.end())
            rc = CSPHT_EINVAL;
        else if (!s->state_set)
            rc = CSPHT_ESTATE;
        else
            b->m.push_back(s);
    }
    if (rc != CSPHT_OK) {
        delete b;
        return rc;
    }
    if (depth <= 0) {
        // the deepest items (fewer predictor planes recomputed at item starts)
        // that still give every resident CTA slot two items: 3 per SM
        int dev = 0, sms = 148;
        if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            sms = 148;
        }
        const long long want = 2LL * 3 * sms;
        b->depth = 8;
        for (int d : {64, 32, 16}) {
            long long items = 0;
            for (const Solver<T> *s : b->m) {
                const long long tiles = (long long)((s->G.n[0] + Solver<T>::LTX - 1) / Solver<T>::LTX) *
                                        ((s->G.n[1] + Solver<T>::LTY - 1) / Solver<T>::LTY);
                items += tiles * ((s->G.n[2] + d - 1) / d);
            }
            if (items >= want) {
                b->depth = d;
                break;
            }
        }
    }
    *out = b;
    return CSPHT_OK;
}

static int set_params(SolverBase *s, double cfl, double t_end) {
    if (cfl != s->cfl_dev || !(t_end == s->tend_dev)) {
        k_set_params<<<1, 1, 0, s->stream>>>(s->ctrl, cfl, t_end);
        s->launches += 1;
        s->cfl_dev = cfl;
        s->tend_dev = t_end;
    }
    return CSPHT_OK;
}

static int read_status(SolverBase *s) {
    if (cudaMemcpyAsync(s->hctrl, s->ctrl, sizeof(Ctrl), cudaMemcpyDeviceToHost, s->stream) !=
            cudaSuccess ||
        cudaStreamSynchronize(s->stream) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        s->err = std::string("device: ") + cudaGetErrorString(e);
        return CSPHT_ECUDA;
    }
    int st = s->hctrl->status;
    if (st & ST_NONFINITE) {
        s->err = "non-finite value in the state";
        return CSPHT_ENONFINITE;
    }
    if (st & ST_TIMEOUT) {
        s->err = "a device-side wait timed out";
        return CSPHT_ECUDA;
    }
    if (st & ST_CFL) {  // reported first: an oversized step is the usual cause of the rest
        s->err = "a particle moved more than one cell (CFL)";
        return CSPHT_ECFL;
    }
    if (st & ST_NEGATIVE) {
        s->err = "negative density";
        return CSPHT_ENEGATIVE;
    }
    return CSPHT_OK;
}

template <typename T>
static void fill_phys(Phys<T> &P, double h, double gamma, const cspht_bcs *bcs, const cspht_opts &o) {
    P.h = (T)h;
    P.inv_h = (T)(1.0 / h);
    P.gamma = (T)gamma;
    P.gm1 = (T)(gamma - 1.0);
    P.inv_gm1 = (T)(1.0 / (gamma - 1.0));
    P.rho_vac = (T)o.rho_vac;
    // FP32: a density below the smallest normal number is vacuum too (the
    // kernels' reciprocal of a gas density assumes a normal number)
    if (sizeof(T) == 4 && P.rho_vac < (T)1.17549435e-38) P.rho_vac = (T)1.17549435e-38;
    // lattice normalisation: sum over the 26 neighbours of gt(|d|) d_x^2
    const double r2 = std::sqrt(2.0), r3 = std::sqrt(3.0);
    double gt1 = 0.75, gt2 = 0.75 * (2.0 - r2) * (2.0 - r2) / r2, gt3 = 0.75 * (2.0 - r3) * (2.0 - r3) / r3;
    double C = 2.0 * gt1 + 8.0 * gt2 + 8.0 * gt3;
    P.inv_Ch2 = (T)(1.0 / (C * h * h));
    P.w[0] = T(0);
    P.w[1] = (T)(gt1 / (C * h * h));
    P.w[2] = (T)(gt2 / (C * h * h));
    P.w[3] = (T)(gt3 / (C * h * h));
    P.gt[0] = T(0);
    P.gt[1] = (T)gt1;
    P.gt[2] = (T)gt2;
    P.gt[3] = (T)gt3;
    for (int f = 0; f < 6; ++f) {
        P.bc[f] = bcs ? bcs->type[f] : CSPHT_BC_PERIODIC;
        const double *W = bcs ? bcs->inflow[f] : nullptr;
        double w[5] = {0, 0, 0, 0, 0};
        if (W)
            for (int c = 0; c < 5; ++c) w[c] = W[c];
        for (int c = 0; c < 5; ++c) P.inW[f][c] = (T)w[c];
        P.inU[f][0] = (T)w[0];
        for (int e = 0; e < 3; ++e) P.inU[f][1 + e] = (T)(w[0] * w[1 + e]);
        P.inU[f][4] = (T)(w[4] / (gamma - 1.0) + 0.5 * w[0] * (w[1] * w[1] + w[2] * w[2] + w[3] * w[3]));
        P.in_vac[f] = !(w[0] > o.rho_vac);
        P.inPhi[f] = P.in_vac[f] ? T(0) : (T)std::sqrt(2.0 * (w[4] > 0 ? w[4] : 0.0));
    }
    P.limiter = o.limiter;
    P.balance = o.balance;
    // HLLC on the advective system has no contact wave beyond the HLL bounds: HLL
    P.riemann = o.riemann == CSPHT_RIEMANN_HLLC ? CSPHT_RIEMANN_HLL : o.riemann;
}

extern "C" {

void cspht_default_opts(cspht_opts *o) {
    if (!o) return;
    o->precision = 64;
    o->riemann = CSPHT_RIEMANN_LF;
    o->limiter = CSPHT_LIMITER_VANLEER;
    o->path = CSPHT_PATH_FAST;
    o->rho_vac = 1e-10;
    o->balance = CSPHT_BALANCE_PLAIN;
}

int cspht_create(int nx, int ny, int nz, double h, double gamma, const double *psi,
                 const cspht_bcs *bcs, const cspht_opts *opts, cspht_t *out) {
    if (!out || !psi) return CSPHT_EINVAL;
    *out = nullptr;
    cspht_opts o;
    cspht_default_opts(&o);
    if (opts) o = *opts;
    int n[3] = {nx, ny, nz};
    if (!(h > 0.0) || !(gamma > 1.0) || !(o.rho_vac >= 0.0)) return CSPHT_EINVAL;
    if (o.precision != 32 && o.precision != 64) return CSPHT_EINVAL;
    if (o.riemann < 0 || o.riemann > 3 || o.limiter < 0 || o.limiter > 2) return CSPHT_EINVAL;
    if (o.path != CSPHT_PATH_FAST && o.path != CSPHT_PATH_PLAIN) return CSPHT_EINVAL;
    if (o.balance != CSPHT_BALANCE_PLAIN && o.balance != CSPHT_BALANCE_COMPENSATED) return CSPHT_EINVAL;
    for (int d = 0; d < 3; ++d) {
        int lo = bcs ? bcs->type[2 * d] : 0, hi = bcs ? bcs->type[2 * d + 1] : 0;
        if (lo < 0 || lo > 3 || hi < 0 || hi > 3) return CSPHT_EINVAL;
        if ((lo == CSPHT_BC_PERIODIC) != (hi == CSPHT_BC_PERIODIC)) return CSPHT_EINVAL;
        if (n[d] < 1 || (lo != CSPHT_BC_PERIODIC && n[d] < 2)) return CSPHT_EINVAL;
        if (n[d] > (1 << 20)) return CSPHT_EINVAL;
    }
    if (!grid_size_ok(nx, ny, nz)) return CSPHT_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return CSPHT_ECUDA;
    }
    cspht_sim *sim = new (std::nothrow) cspht_sim;
    if (!sim) return CSPHT_ENOMEM;
    sim->precision = o.precision;
    int rc;
    if (o.precision == 32) {
        auto *s = new (std::nothrow) Solver<float>;
        if (!s) { delete sim; return CSPHT_ENOMEM; }
        s->G.n[0] = nx; s->G.n[1] = ny; s->G.n[2] = nz;
        s->path = o.path;
        s->h = h;
        s->gamma = gamma;
        fill_phys(s->P, h, gamma, bcs, o);
        sim->s = s;
        rc = s->create(psi);
    } else {
        auto *s = new (std::nothrow) Solver<double>;
        if (!s) { delete sim; return CSPHT_ENOMEM; }
        s->G.n[0] = nx; s->G.n[1] = ny; s->G.n[2] = nz;
        s->path = o.path;
        s->h = h;
        s->gamma = gamma;
        fill_phys(s->P, h, gamma, bcs, o);
        sim->s = s;
        rc = s->create(psi);
    }
    if (rc != CSPHT_OK) {
        delete sim->s;
        delete sim;
        return rc;
    }
    *out = sim;
    return CSPHT_OK;
}

int cspht_set_state(cspht_t s, const double *U) {
    if (!s || !U) return CSPHT_EINVAL;
    return s->s->set_state(U, false);
}

int cspht_set_primitive(cspht_t s, const double *W) {
    if (!s || !W) return CSPHT_EINVAL;
    return s->s->set_state(W, true);
}

int cspht_set_state_f32(cspht_t s, const float *U) {
    if (!s || !U) return CSPHT_EINVAL;
    return s->s->set_state_f32(U);
}

int cspht_get_state_f32(cspht_t s, float *U) {
    if (!s || !U) return CSPHT_EINVAL;
    if (!s->s->state_set) {
        s->s->err = "no state set";
        return CSPHT_ESTATE;
    }
    return s->s->get_state_f32(U);
}

int cspht_get_state(cspht_t s, double *U) {
    if (!s || !U) return CSPHT_EINVAL;
    if (!s->s->state_set) {
        s->s->err = "no state set";
        return CSPHT_ESTATE;
    }
    return s->s->get_state(U);
}

int cspht_advance(cspht_t s, long nsteps, double cfl) {
    if (!s || nsteps < 0 || !(cfl > 0.0)) return CSPHT_EINVAL;
    SolverBase *b = s->s;
    if (!b->state_set) {
        b->err = "no state set";
        return CSPHT_ESTATE;
    }
    set_params(b, cfl, INFINITY);
    for (long i = 0; i < nsteps; ++i) {
        int rc = b->enqueue_step();
        if (rc) return rc;
    }
    return CSPHT_OK;
}

int cspht_batch_step(cspht_t *handles, int n, double cfl, void *cuda_stream) {
    if (!handles || n < 0 || !(cfl > 0.0) || !cuda_stream) return CSPHT_EINVAL;
    cudaStream_t bs = (cudaStream_t)cuda_stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(bs, &cap) != cudaSuccess) return CSPHT_ECUDA;
    for (int i = 0; i < n; ++i) {
        SolverBase *b = handles[i] ? handles[i]->s : nullptr;
        if (!b) return CSPHT_EINVAL;
        if (!b->state_set) {
            b->err = "no state set";
            return CSPHT_ESTATE;
        }
        // profiling brackets launches with host-read events: not inside a capture
        if (cap != cudaStreamCaptureStatusNone && b->prof_on) {
            b->err = "batch capture of a profiling handle";
            return CSPHT_ESTATE;
        }
    }
    for (int i = 0; i < n; ++i) {
        SolverBase *b = handles[i]->s;
        if (!b->ev_fork && (cudaEventCreateWithFlags(&b->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
                            cudaEventCreateWithFlags(&b->ev_join, cudaEventDisableTiming) != cudaSuccess))
            return b->ev_fork = nullptr, CSPHT_ECUDA;
        if (cudaEventRecord(b->ev_fork, bs) != cudaSuccess || cudaStreamWaitEvent(b->stream, b->ev_fork, 0) != cudaSuccess)
            return CSPHT_ECUDA;
        set_params(b, cfl, INFINITY);
        int rc = b->enqueue_step();
        if (rc) return rc;
        if (cudaEventRecord(b->ev_join, b->stream) != cudaSuccess || cudaStreamWaitEvent(bs, b->ev_join, 0) != cudaSuccess)
            return CSPHT_ECUDA;
    }
    return CSPHT_OK;
}

int cspht_batch_create(cspht_t *handles, int n, int depth, cspht_batch_t *out) {
    if (!out) return CSPHT_EINVAL;
    *out = nullptr;
    if (!handles || n < 1 || depth < 0) return CSPHT_EINVAL;
    for (int i = 0; i < n; ++i)
        if (!handles[i] || handles[i]->precision != handles[0]->precision) return CSPHT_EINVAL;
    cspht_batch *b = new (std::nothrow) cspht_batch;
    if (!b) return CSPHT_ENOMEM;
    const int rc = handles[0]->precision == 32 ? make_batch<float>(handles, n, depth, &b->b)
                                               : make_batch<double>(handles, n, depth, &b->b);
    if (rc != CSPHT_OK) {
        delete b;
        return rc;
    }
    *out = b;
    return CSPHT_OK;
}

int cspht_batch_advance(cspht_batch_t b, long nsteps, double cfl, void *cuda_stream) {
    if (!b || nsteps < 0 || !(cfl > 0.0)) return CSPHT_EINVAL;
    return b->b->advance(nsteps, cfl, (cudaStream_t)cuda_stream);
}

long long cspht_batch_launch_count(cspht_batch_t b) { return b ? b->b->launches : -1; }

const char *cspht_batch_last_error(cspht_batch_t b) { return b ? b->b->err.c_str() : "null batch"; }

void cspht_batch_destroy(cspht_batch_t b) {
    if (!b) return;
    delete b->b;
    delete b;
}

int cspht_step(cspht_t s, double cfl, double *dt_taken) {
    int rc = cspht_advance(s, 1, cfl);
    if (rc) return rc;
    rc = read_status(s->s);
    if (dt_taken) *dt_taken = s->s->hctrl->dt;
    return rc;
}

int cspht_sync(cspht_t s) {
    if (!s) return CSPHT_EINVAL;
    const int rc = read_status(s->s);
    if (!s->s->io_sync()) {
        cudaGetLastError();
        s->s->err = "device: an asynchronous copy failed";
        return CSPHT_ECUDA;
    }
    return rc;
}

int cspht_upload_f32_async(cspht_t s, const float *U) {
    if (!s || !U) return CSPHT_EINVAL;
    return s->s->upload_f32_async(U);
}

int cspht_download_f32_async(cspht_t s, float *U) {
    if (!s || !U) return CSPHT_EINVAL;
    if (!s->s->state_set) {
        s->s->err = "no state set";
        return CSPHT_ESTATE;
    }
    return s->s->download_f32_async(U);
}

int cspht_test_copy_timeout(cspht_t s, int polls) {
    if (!s || polls < 0) return CSPHT_EINVAL;
    SolverBase *b = s->s;
    k_set_inject<<<1, 1, 0, b->stream>>>(b->ctrl, polls > 0 ? INJECT_NO_COPIES : 0, polls);
    b->launches += 1;
    return cudaStreamSynchronize(b->stream) == cudaSuccess ? CSPHT_OK : CSPHT_ECUDA;
}

int cspht_set_tile_depth(cspht_t s, int zchunk) {
    if (!s || zchunk < 1) return CSPHT_EINVAL;
    return s->s->set_tile_depth(zchunk);
}

int cspht_autotune(cspht_t s, int steps, double cfl, int *zchunk) {
    if (!s || steps < 1 || !(cfl > 0.0)) return CSPHT_EINVAL;
    SolverBase *b = s->s;
    if (!b->state_set) {
        b->err = "no state set";
        return CSPHT_ESTATE;
    }
    int rc = read_status(b);
    if (rc) return rc;
    rc = b->autotune(steps, cfl, zchunk);
    if (rc) return rc;
    return read_status(b);
}

int cspht_run(cspht_t s, double t_end, double cfl, long *steps_taken) {
    if (!s || !(cfl > 0.0) || !std::isfinite(t_end)) return CSPHT_EINVAL;
    SolverBase *b = s->s;
    if (!b->state_set) {
        b->err = "no state set";
        return CSPHT_ESTATE;
    }
    int rc = read_status(b);
    if (rc) return rc;
    long long s0 = b->hctrl->steps;
    set_params(b, cfl, t_end);
    long chunk = 4;
    for (;;) {
        if (b->hctrl->t >= t_end) break;
        for (long i = 0; i < chunk; ++i) {
            rc = b->enqueue_step();
            if (rc) return rc;
        }
        rc = read_status(b);
        if (rc) break;
        double dt = b->hctrl->dt;
        if (!(dt > 0.0) && b->hctrl->t < t_end) {
            b->err = "time step collapsed to zero";
            rc = CSPHT_ECFL;
            break;
        }
        double left = (t_end - b->hctrl->t) / dt;
        chunk = left < 1.0 ? 1 : (left > 256.0 ? 256 : (long)left);
    }
    set_params(b, cfl, INFINITY);
    if (steps_taken) *steps_taken = (long)(b->hctrl->steps - s0);
    return rc;
}

int cspht_totals(cspht_t s, double out[6]) {
    if (!s || !out) return CSPHT_EINVAL;
    return s->s->totals(out);
}

int cspht_set_stream(cspht_t s, void *cuda_stream) {
    if (!s) return CSPHT_EINVAL;
    SolverBase *b = s->s;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return CSPHT_ECUDA;
    }
    cudaStream_t ns = cuda_stream ? (cudaStream_t)cuda_stream : b->own;
    if (ns != b->stream) {
        b->stream = ns;
        b->reset_graphs();  // graphs are re-captured on the new stream when first needed
    }
    return CSPHT_OK;
}

double cspht_time(cspht_t s) {
    if (!s) return NAN;
    if (read_status(s->s) == CSPHT_ECUDA) return NAN;
    return s->s->hctrl->t;
}

long long cspht_launch_count(cspht_t s) { return s ? s->s->launches : -1; }

long long cspht_device_bytes(int nx, int ny, int nz, const cspht_opts *opts) {
    cspht_opts o;
    cspht_default_opts(&o);
    if (opts) o = *opts;
    if (nx < 1 || ny < 1 || nz < 1 || (o.precision != 32 && o.precision != 64)) return -1;
    if (!grid_size_ok(nx, ny, nz)) return -1;  // cspht_create would refuse it
    const bool f32 = o.precision == 32;
    const Grid G = f32 ? make_grid<float>(nx, ny, nz) : make_grid<double>(nx, ny, nz);
    long long narr = 10 + 1 + 7;
    if (o.path == CSPHT_PATH_PLAIN) narr += 4 + 4 + 5 + 1 + 3 + 1 + 3 + 15;
    else narr += 3 + (f32 ? 1 : 0);
    const long long N = (long long)nx * ny * nz;
    return narr * G.total * (f32 ? 4 : 8) + 8 * 5 * N + 8 * 6 * TOT_BLOCKS + 8 * 6 + (long long)sizeof(Ctrl);
}

int cspht_profile(cspht_t s, int enable) {
    if (!s) return CSPHT_EINVAL;
    SolverBase *b = s->s;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return CSPHT_ECUDA;
    }
    b->prof.clear();
    b->evused = 0;
    b->prof_on = enable != 0;
    return CSPHT_OK;
}

int cspht_profile_read(cspht_t s, int n, double *ms, long long *launches, char *names,
                       int names_cap) {
    if (!s || n < 0) return CSPHT_EINVAL;
    SolverBase *b = s->s;
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaError_t e = cudaGetLastError();
        b->err = std::string("profile: ") + cudaGetErrorString(e);
        return CSPHT_ECUDA;
    }
    double tot[KK_COUNT] = {0};
    long long cnt[KK_COUNT] = {0};
    for (const auto &r : b->prof) {
        float m = 0.f;
        if (cudaEventElapsedTime(&m, r.a, r.b) == cudaSuccess) {
            tot[r.kind] += m;
            cnt[r.kind] += 1;
        }
    }
    cudaGetLastError();
    for (int i = 0; i < n && i < KK_COUNT; ++i) {
        if (ms) ms[i] = tot[i];
        if (launches) launches[i] = cnt[i];
    }
    if (names && names_cap > 0) {
        std::string all;
        for (int i = 0; i < KK_COUNT; ++i) {
            if (i) all += ";";
            all += KK_NAME[i];
        }
        snprintf(names, (size_t)names_cap, "%s", all.c_str());
    }
    return KK_COUNT;
}

const char *cspht_last_error(cspht_t s) { return s ? s->s->err.c_str() : "null handle"; }

void cspht_destroy(cspht_t s) {
    if (!s) return;
    if (s->s) cudaStreamSynchronize(s->s->stream);
    delete s->s;
    delete s;
}

}  // extern "C"
