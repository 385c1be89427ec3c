/*
 * cspht.h -- C ABI of the B300 CSPH-TVD solver.
 *
 * The library advances the 3D Euler equations of an ideal gamma-law gas in a
 * fixed potential psi (Eqs. 1-3 of Khrapov, Khoperskov & Khoperskov,
 * arXiv 1912.04855, Sec. 2.1) on a uniform Cartesian grid of cell size h with
 * the two-stage CSPH-TVD step of Sec. 2.2:
 *   - a Lagrangian stage: particles that start at the cell centres are moved
 *     by the pressure force and -grad psi with the predictor-corrector of
 *     Eqs. 5-6, the force Q being the modified-SPH sum of Eq. 7;
 *   - an Eulerian stage (Eq. 4): mass, momentum and energy fluxes through the
 *     cell faces from the particle-offset, TVD-limited reconstruction of
 *     Eq. 8 and a Riemann flux (Lax-Friedrichs or HLL, Sec. 2.2).
 * Around them sit the CFL time-step reduction and the boundary and
 * gas-vacuum handling.  All of a step runs in CUDA kernels on one GPU.
 *
 * Conventions
 *  - Every call returns a status code (CSPHT_OK = 0 or a negative CSPHT_E*);
 *    nothing aborts or throws across the ABI.  cspht_last_error() gives a
 *    one-line message for the last failing call on a handle.
 *  - Cell arrays are structure-of-arrays over N = nx*ny*nz cells, x fastest:
 *    field f of cell (i,j,k) is element f*N + (k*ny + j)*nx + i.
 *  - Arrays passed in are HOST pointers and are copied; the caller keeps
 *    ownership.  Arrays passed out are caller-owned host buffers.
 *  - A handle owns its device memory (allocated by cspht_create, released by
 *    cspht_destroy) and one CUDA stream (created at the device's greatest
 *    stream priority; cspht_set_stream replaces it).  A handle is not thread-safe: use
 *    one handle per host thread.
 *  - Single-precision handles take and return FP64 host arrays; values are
 *    rounded on upload.  Totals are always summed in FP64 on the device.
 *  - Device-side faults of the numerics (non-finite values, negative
 *    density, a particle moved further than one cell) set a status word on
 *    the device; it is read back by cspht_step, cspht_run and cspht_sync and
 *    returned as CSPHT_ENONFINITE, CSPHT_ENEGATIVE or CSPHT_ECFL.  Kernels
 *    never trap.
 */
#ifndef CSPHT_H
#define CSPHT_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct cspht_sim *cspht_t; /* opaque handle, owned by the library */

enum {
    CSPHT_OK = 0,
    CSPHT_EINVAL = -1,     /* invalid argument (sizes, BC pairing, options) */
    CSPHT_ENOMEM = -2,     /* device or host allocation failed */
    CSPHT_ECUDA = -3,      /* a CUDA runtime call failed (no device, launch error) */
    CSPHT_ENONFINITE = -4, /* a NaN or Inf appeared in the state */
    CSPHT_ECFL = -5,       /* a particle moved more than one cell in a step */
    CSPHT_ENEGATIVE = -6,  /* a cell density became negative */
    CSPHT_ESTATE = -7,     /* call out of order (e.g. step before set_state) */
    CSPHT_ETOOBIG = -8     /* grid larger than cspht_step_noalloc_f32's fixed scratch */
};

/* Boundary kinds per face (not in the paper; needed by its test problems).
 *  PERIODIC  wrap around; both faces of an axis must be periodic together.
 *  OUTFLOW   zero-gradient: the ghost cell copies the boundary cell, including
 *            its particle offset; ghost slope 0.
 *  INFLOW    fixed primitive state (rho,u,v,w,p) from cspht_bcs.inflow; ghost
 *            particle offset dt*u after the predictor; ghost slope 0.
 *  WALL      reflecting wall: zero flux through the face; ghost velocity and
 *            offset mirrored in the normal direction; ghost phi = sqrt(2p)
 *            extrapolated so that a hydrostatic state is a discrete
 *            equilibrium: phi_g = phi_m + rho_b (psi_m - psi_g) / phi_b, with
 *            b the boundary cell and m the next cell inward. */
enum { CSPHT_BC_PERIODIC = 0, CSPHT_BC_OUTFLOW = 1, CSPHT_BC_INFLOW = 2, CSPHT_BC_WALL = 3 };

typedef struct {
    int type[6];         /* faces -x,+x,-y,+y,-z,+z */
    double inflow[6][5]; /* primitive (rho,u,v,w,p) for INFLOW faces */
} cspht_bcs;

/* Riemann fluxes of the advective system F = a U at a face with the particle
 * speeds a_L, a_R (xi^{n+1}/dt of the two cells) and reconstructed states
 * U_L, U_R (Sec. 2.2 names several solvers without formulas):
 *   LF:    (a_L U_L + a_R U_R)/2 - max(|a_L|, |a_R|) (U_R - U_L)/2
 *   HLL:   the three-branch HLL flux with S_L = min(a_L, a_R), S_R = max(a_L, a_R)
 *   SWEPT: a U_upwind with a = (a_L + a_R)/2 (the volume the face sweeps)
 * All three give a U_upwind for a uniform speed and 0 at rest.
 *   HLLC:  Sec. 2.2 also names HLLC.  HLLC adds a contact wave inside the HLL
 *          fan; on the advective system every component moves with the one
 *          speed a, and the HLL bounds S_L, S_R already are the two particle
 *          speeds, so there is no third wave to resolve and HLLC is read as
 *          HLL here: CSPHT_RIEMANN_HLLC selects the HLL flux (same bits). */
enum { CSPHT_RIEMANN_LF = 0, CSPHT_RIEMANN_HLL = 1, CSPHT_RIEMANN_SWEPT = 2, CSPHT_RIEMANN_HLLC = 3 };
enum { CSPHT_LIMITER_VANLEER = 0, CSPHT_LIMITER_MINMOD = 1, CSPHT_LIMITER_MC = 2 };
enum { CSPHT_PATH_FAST = 0, CSPHT_PATH_PLAIN = 1 };
/* The Lagrangian force of Eq. 7 balances the pressure term phi_i D_i[phi]
 * against gravity rho_i D0_i[psi] (Sec. 2.1, Eqs. 2-3); in a hydrostatic
 * state the two nearly cancel.  BALANCE_COMPENSATED (single precision,
 * fused path) forms both products exactly and their difference with one
 * rounding (TwoProd and TwoSum); BALANCE_PLAIN rounds each product and the
 * difference.  FP64 handles and the unfused path ignore it. */
enum { CSPHT_BALANCE_PLAIN = 0, CSPHT_BALANCE_COMPENSATED = 1 };

typedef struct {
    int precision; /* 32 or 64: storage and arithmetic of the step (default 64) */
    int riemann;   /* CSPHT_RIEMANN_*: Riemann flux at the faces (Sec. 2.2; default LF) */
    int limiter;   /* CSPHT_LIMITER_*: TVD slope limiter Theta of Eq. 8 (default van Leer) */
    int path;      /* CSPHT_PATH_FAST: fused, tiled kernels; CSPHT_PATH_PLAIN: one
                      kernel per paper kernel (HFC, SUL, FGC, SUE) with global scratch */
    double rho_vac; /* vacuum threshold: rho <= rho_vac is vacuum (default 1e-10);
                       FP32 handles raise a smaller value to 2^-126 */
    int balance;    /* CSPHT_BALANCE_*: FP32 balance terms (default plain) */
} cspht_opts;

/* Fills *o with the defaults (FP64, LF, van Leer, fast path, rho_vac 1e-10,
 * plain balance terms). */
void cspht_default_opts(cspht_opts *o);

/* Create a solver for an nx*ny*nz grid of cell size h and adiabatic index gamma
 * (Sec. 2.1).  psi: host array of N potentials (Eqs. 2-3, f = -grad psi),
 * copied.  bcs: boundary kinds (NULL = periodic everywhere).  opts: NULL for the
 * defaults.  Each extent must be >= 1 and >= 2 along non-periodic axes, at
 * most 2^20, with nz <= 65533 and (nx + 36)(ny + 4)(nz + 4) < 2^31 (padded
 * arrays are addressed with 32-bit offsets); larger grids give CSPHT_EINVAL.
 * Allocates all device memory of the handle.  Errors: EINVAL, ENOMEM, ECUDA. */
int cspht_create(int nx, int ny, int nz, double h, double gamma, const double *psi,
                 const cspht_bcs *bcs, const cspht_opts *opts, cspht_t *out);

/* Upload the conserved state U = (rho, mx, my, mz, E) (Eq. 4's U), 5*N host
 * doubles, SoA.  Resets nothing else (time and step count stay). */
int cspht_set_state(cspht_t s, const double *U);

/* Upload a primitive state W = (rho, u, v, w, p), 5*N host doubles, SoA; the
 * library converts it to U on the device (E = p/(gamma-1) + rho|u|^2/2). */
int cspht_set_primitive(cspht_t s, const double *W);

/* Download the conserved state into the caller's 5*N host doubles. */
int cspht_get_state(cspht_t s, double *U);

/* The same upload and download with 5*N host floats (same layout): half the
 * bytes over the bus.  For an FP32 handle the upload is exact and the
 * download rounds the density (kept as a value plus compensation word) once;
 * an FP64 handle converts.  CSPHT_ESTATE if no state was set (download). */
int cspht_set_state_f32(cspht_t s, const float *U);
int cspht_get_state_f32(cspht_t s, float *U);

/* Asynchronous forms of the two calls above, for loops that move the state
 * between host and device every step.  Both return at once.  The copies run
 * on two streams of the handle's own, beside the compute stream, so one
 * step's download overlaps the next step's upload and the upload overlaps the
 * previous step's kernels.  Page-locked host memory is needed for the copies
 * to overlap anything.
 * Ordering: uploads, steps and downloads act on the state in call order, as
 * the synchronous calls do.  An upload waits on the device until the previous
 * upload has been converted; a download converts the state into a second
 * device staging buffer (5*N floats, allocated on the first call) once the
 * previous download has been read out of it.
 * Ownership: U must stay valid and unchanged (upload) or unread (download)
 * until cspht_sync returns, which also waits for both copy streams.
 * Errors: CSPHT_EINVAL for a null handle or pointer, CSPHT_ESTATE for a
 * download before any state was set, CSPHT_ENOMEM if the staging buffer
 * cannot be allocated, CSPHT_ECUDA if a copy or launch cannot be enqueued;
 * copy failures surface at cspht_sync. */
int cspht_upload_f32_async(cspht_t s, const float *U);
int cspht_download_f32_async(cspht_t s, float *U);

/* One time step with dt = cfl * h / max over gas cells of (max_d |u_d| + c),
 * c the sound speed, from the current state.  Waits for the step and
 * returns its device status; *dt_taken (may be NULL) receives dt. */
int cspht_step(cspht_t s, double cfl, double *dt_taken);

/* Enqueue nsteps steps on the handle's stream without waiting (the step is
 * replayed from a CUDA graph when the stream allows capture).  Device status
 * is checked by the next cspht_sync / cspht_step / cspht_run. */
int cspht_advance(cspht_t s, long nsteps, double cfl);

/* Wait for the handle's stream and its two copy streams (if the asynchronous
 * host I/O calls were used) and return the device status. */
int cspht_sync(cspht_t s);

/* Advance until the simulated time reaches t_end (the last step is clipped to
 * land on t_end).  *steps_taken (may be NULL) receives the number of steps. */
int cspht_run(cspht_t s, double t_end, double cfl, long *steps_taken);

/* Totals over the grid, summed in FP64 on the device in a fixed order and
 * multiplied by h^3: mass, x/y/z momentum, total energy E, and E + rho*psi. */
int cspht_totals(cspht_t s, double out[6]);

/* Make the handle launch on the given cudaStream_t (e.g. torch's
 * stream.cuda_stream).  NULL restores the handle's own stream.  The legacy
 * default stream disables graph replay. */
int cspht_set_stream(cspht_t s, void *cuda_stream);

/* One step of each of n handles, run concurrently and ordered against a
 * caller's stream: every handle's step forks from `cuda_stream` (its own stream
 * waits for the work already enqueued there), runs on the handle's stream with
 * the handle's own dt (its CFL condition) and time, and joins back (the caller's
 * stream waits for all n).  Only enqueues.  The call can be captured into a
 * CUDA graph on `cuda_stream` to launch many instances as one graph (the
 * handles' step kernels become nodes of it); a profiling handle cannot be
 * captured (CSPHT_ESTATE).  A captured graph refers to the handles' memory:
 * replay it only while all of them are alive, and an even number of steps
 * per replay keeps each handle's ping-pong buffers where the capture found
 * them.  A device-side error of a handle shows at that handle's next
 * cspht_sync.  cfl > 0; handles and cuda_stream non-NULL. */
int cspht_batch_step(cspht_t *handles, int n, double cfl, void *cuda_stream);

/* Chooses how a fused-path handle runs its steps.  A CTA of the fused
 * kernels owns a 32 x 8 column of cells and marches through `zchunk` planes
 * of it; every chunk recomputes two predictor planes at its start, so long
 * chunks save work while short ones fill the SMs in fuller waves.  This call
 * times `steps` steps with the Courant number `cfl` for each candidate length
 * on the current state (which it saves first and restores after every trial,
 * so the state, time and step count are unchanged on return) and keeps the
 * fastest.  An FP64 handle also tries split stages -- the unfused kernels,
 * one per paper kernel (Sec. 3: HFC, SUL, FGC, SUE) -- which win on the
 * smallest grids; if they are faster the handle switches to them for good
 * (and allocates their scratch, about twice the fused path's memory).  The
 * choice is written to *zchunk (may be NULL): the tile depth, or 0 for the
 * unfused kernels (also on a handle created on the unfused path, which has
 * nothing to tune).  The tile depth is remembered for fused handles of the
 * same grid and precision that this process creates later.  FP32 results do
 * not depend on the choice; in FP64 the two paths agree to rounding (both
 * match the oracle within 1e-10).  Needs a state (CSPHT_ESTATE otherwise)
 * and device memory for one copy of the state (CSPHT_ENOMEM otherwise). */
int cspht_autotune(cspht_t s, int steps, double cfl, int *zchunk);

/* Sets the tile depth of the fused path by hand (planes per CTA column,
 * clamped to nz; a no-op on the unfused path).  CSPHT_EINVAL if zchunk < 1.
 * Results do not depend on it: planes that neighbouring chunks share are
 * computed by the same code with the same bits. */
int cspht_set_tile_depth(cspht_t s, int zchunk);

/* Simulated time of the current state (waits for the stream). */
double cspht_time(cspht_t s);

/* Number of CUDA kernels the handle has launched so far (graph replays
 * count every kernel in the graph). */
long long cspht_launch_count(cspht_t s);

/* Per-kernel timing.  While enabled, steps are launched without graph replay
 * and every kernel launch is bracketed by two CUDA events on the handle's
 * stream.  Enabling clears earlier records. */
int cspht_profile(cspht_t s, int enable);

/* Waits for the stream and sums the recorded event intervals per kernel kind.
 * Writes up to n entries: ms[i] total milliseconds and launches[i] launch
 * count of kind i, and the kind names as one ';'-separated string into names
 * (capacity names_cap bytes, NUL-terminated).  Returns the number of kinds
 * (>= 0) or a negative error code. */
int cspht_profile_read(cspht_t s, int n, double *ms, long long *launches, char *names,
                       int names_cap);

/* One FP32 time step that allocates no device memory.  The paper has no
 * counterpart: this is for callers that cannot call cudaMalloc -- a host
 * application whose memory pool already owns the GPU's memory, or a
 * time-critical loop that cannot accept the device-wide synchronisation an
 * allocation implies.
 *   U      device pointer, 5*N floats, conserved state (rho,mx,my,mz,E) SoA,
 *          x fastest (the layout of cspht_set_state, in single precision);
 *   psi    device pointer, N floats, the potential;
 *   U_out  device pointer, 5*N floats, receives the state after the step
 *          (must not overlap U);
 *   bcs    host struct of boundary kinds (NULL = periodic);
 *   cfl    Courant number; dt = cfl h / max(|u_d| + c) of U, as cspht_step;
 *   dt_taken  host pointer (may be NULL) that receives dt;
 *   stream cudaStream_t to run on (NULL = the legacy default stream).
 * The step is the fused fast path with the default options (LF flux, van
 * Leer limiter, rho_vac 1e-10), without the density compensation word of an
 * FP32 handle: the density is rounded to FP32 at every update, so the total
 * mass drifts by rounding (about 1e-9 relative over hundreds of steps)
 * instead of changing only by boundary fluxes.  Each call ends with a host
 * wait on its stream (to read dt and the status word) and returns the
 * step's status.  All intermediate arrays live in one file-scope device
 * array of 64 MiB that every GPU loading the library holds until exit: the
 * grid must fit 21 padded single-precision fields in it (for example 86^3;
 * 87^3 does not), otherwise the call returns CSPHT_ETOOBIG before touching
 * the device.  The first call on a device looks up that array's address and
 * sets kernel attributes; make it before any stream capture.  Every call
 * reuses the same array and first clears the part it uses (an asynchronous
 * memset on its stream, no allocation), so calls that overlap on the GPU --
 * on two streams or from two host threads -- race and must not be issued.
 * A CUDA error already pending when the call starts is reported as
 * CSPHT_ECUDA and left pending; nothing is launched then. */
int cspht_step_noalloc_f32(int nx, int ny, int nz, double h, double gamma, const cspht_bcs *bcs,
                           const float *U, const float *psi, float *U_out, double cfl,
                           double *dt_taken, void *stream);

/* Many grids advanced together with one launch of each step kernel (the
 * serving loop's batched mode).  The paper's kernels (Sec. 3) run one grid;
 * here the members of a batch take one dt launch, one launch per ghost pass
 * and one persistent launch per fused stage for all of them, whose CTAs take
 * (member, tile, z chunk) work items from a device counter, longest first.
 * Every member keeps its own dt, time and state; results are bit-identical
 * to stepping each member alone.
 *
 * cspht_batch_create: handles[0..n-1] become the members (the array is
 * copied; the handles must outlive the batch and be distinct).  All must
 * have the same precision, the fused path, the same limiter, Riemann flux
 * and balance option, a state set (else CSPHT_ESTATE), and periodic or
 * outflow faces in y and z (ghost layers filled in one pass; else
 * CSPHT_EINVAL).  depth: planes of a work item (0 = the deepest of 64, 32
 * and 16 that gives the members at least two items per resident CTA slot,
 * else 8); results do not depend on it.
 * cspht_batch_advance: nsteps steps of every member at Courant number cfl
 * on cuda_stream (NULL = the legacy stream), after the members' earlier work
 * on their own streams and before their later work there.  Asynchronous:
 * read each member's status with cspht_sync.  Two steps at a time replay a
 * CUDA graph captured on first use (on a stream other than the legacy
 * ones); inside a caller's stream capture the kernels are captured
 * directly.  A member stepped on its own in between is picked up (its
 * arguments are rebuilt, which waits for the stream).
 * Errors: EINVAL, ESTATE, ENOMEM, ECUDA (message in cspht_batch_last_error). */
typedef struct cspht_batch *cspht_batch_t;
int cspht_batch_create(cspht_t *handles, int n, int depth, cspht_batch_t *out);
int cspht_batch_advance(cspht_batch_t b, long nsteps, double cfl, void *cuda_stream);
/* Kernels the batch has launched so far (graph replays count every kernel). */
long long cspht_batch_launch_count(cspht_batch_t b);
const char *cspht_batch_last_error(cspht_batch_t b);
/* Waits for the batch's last stream and frees its device memory (not the members). */
void cspht_batch_destroy(cspht_batch_t b);

/* Device bytes that cspht_create would allocate for this grid and these
 * options (NULL = defaults), without creating anything: used to admit
 * requests against a memory budget.  Returns -1 for invalid arguments and for
 * grids outside cspht_create's limits. */
long long cspht_device_bytes(int nx, int ny, int nz, const cspht_opts *opts);

/* Test hook for the fused path's failure detection.  polls > 0: the next
 * steps post their tile copies' byte counts but issue no copy, and every copy
 * wait gives up after `polls` polls; the kernels then set the time-out status
 * bit, wait (bounded) for the copies they believe in flight and return, and
 * the step reports CSPHT_ECUDA ("a device-side wait timed out") with the
 * context intact.  polls = 0 restores normal operation.  The state of a step
 * that timed out is not meaningful: set it again afterwards. */
int cspht_test_copy_timeout(cspht_t s, int polls);

/* Last error message of the handle ("" if none); owned by the handle. */
const char *cspht_last_error(cspht_t s);

/* Release the handle and all of its device memory.  NULL is a no-op.  The
 * memory is freed in order on the handle's stream (the call waits for that
 * stream, not for the whole device) and returns to the library's per-device
 * pool, which keeps it for the next handle instead of giving it back to the
 * driver. */
void cspht_destroy(cspht_t s);

#ifdef __cplusplus
}
#endif
#endif
