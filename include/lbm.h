/*
 * lbm.h -- C ABI of liblbm.so: the fused per-time-step update of the
 * non-orthogonal multiple-relaxation-time (MRT) lattice Boltzmann method with
 * the square-root pseudopotential multiphase model, on D3Q19 and D3Q27, for
 * one NVIDIA GB300 (sm_103a).
 *
 * Method: Fei, Du, Luo, Succi, Lauricella, Montessori, Wang, "Modeling
 * realistic multiphase flows using a non-orthogonal multiple-relaxation-time
 * lattice Boltzmann method" (arXiv:2306.16274).  One call of lbm_step(ctx, 1)
 * performs, for every fluid cell x:
 *   - pull of the shifted populations f_bar_i (streaming, Eq. e9, kept in place
 *     with the AA access pattern), density rho = sum_i f_bar_i (Sec. II A);
 *   - the interaction force F_int (Eq. e15) from the square-root pseudopotential
 *     psi = sqrt(2 (p_EOS - rho c_s^2) / G) (Sec. II C), the wetting force F_ads
 *     (Sec. III E), the surface-tension tensor Q (Eq. e18) and a body force;
 *   - velocity u = (sum_i f_bar_i e_i + F/2) / rho (Sec. II A);
 *   - m_bar = M f_bar with the non-orthogonal M of Eq. e11 / Eq. "matrix",
 *     relaxation m_bar* = m_bar - S (m_bar - m^eq) + (I - S/2) F~' (Eq. e8) with
 *     m^eq of Eq. e13 and F~ of Eq. e14 modified by Eq. e17;
 *   - f_bar* = M^-1 m_bar* and the store (Eq. e9), with half-way bounce-back at
 *     solid links;
 * then recomputes rho and psi for the next step.
 *
 * Conventions for every entry point
 *   - Fields are structure-of-arrays, x fastest: index (z * ny + y) * nx + x.
 *     A velocity field is three such planes (u_x, u_y, u_z) back to back.
 *     Populations are Q such planes in the velocity order of Eq. e1.
 *   - `ptrs_on_device` != 0 means every array argument of that call is CUDA
 *     device memory of the current device; 0 means host memory.  Host copies
 *     go through the context's stream and the call synchronises that stream.
 *   - The library owns all device state of a context; callers own every buffer
 *     they pass in.  No allocation crosses the ABI.
 *   - Work is enqueued on the CUDA stream given to lbm_create (a cudaStream_t
 *     passed as void*; NULL = the legacy default stream).
 *   - Errors are returned as lbm_status; lbm_last_error(ctx) gives a message.
 *     Nothing throws, exits or traps.  LBM_ERR_UNSTABLE and LBM_ERR_EOS_RANGE
 *     are sticky: further lbm_step calls return them until lbm_init_fields or
 *     lbm_set_populations resets the state.
 *   - One context must not be used from two host threads at once.
 */
#ifndef LBM_H
#define LBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 3

/* Largest nx, ny or nz: the density/psi pass launches one block row per z plane. */
#define LBM_MAX_EXTENT 65535

typedef struct lbm_ctx lbm_ctx;

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = 1,        /* invalid argument or parameter set                        */
    LBM_ERR_OOM = 2,        /* a device allocation failed                               */
    LBM_ERR_CUDA = 3,       /* a CUDA runtime call or kernel launch failed              */
    LBM_ERR_UNSTABLE = 4,   /* NaN / Inf / non-positive density seen on a fluid cell    */
    LBM_ERR_EOS_RANGE = 5,  /* psi^2 < 0 on some cell: density outside the EOS range;   */
                            /* psi was clamped to 0 there                               */
    LBM_ERR_TIMEOUT = 6,    /* a bounded device-side wait gave up                       */
    LBM_ERR_STATE = 7       /* call out of order (e.g. lbm_step before lbm_init_fields) */
} lbm_status;

/* equation of state for psi (Sec. II C, Sec. III A) */
enum {
    LBM_EOS_NONE = 0,       /* single phase: no pseudopotential, F = rho g                */
    LBM_EOS_CS = 1,         /* Carnahan-Starling: eos_p = {a, b, R, T}                     */
    LBM_EOS_PIECEWISE = 2   /* piecewise linear, Eq. e19: eos_p = {rho1, rho2, theta_v,   */
                            /*   theta_m, theta_l}                                        */
};

/* population storage */
enum {
    LBM_STORE_FP32 = 0,     /* FP32 populations                                           */
    LBM_STORE_FP16 = 1      /* shifted FP16: a slot holds f_i / rho_w - omega_i in half   */
                            /* precision, rho_w the density of the cell that wrote it     */
                            /* (kept in FP32, two fields of 4 bytes per cell); FP32 maths */
};

/* per-axis boundary */
enum {
    LBM_BC_PERIODIC = 0,
    LBM_BC_WALL = 1         /* no-slip walls half-way outside the first and last planes   */
                            /* (half-way bounce-back, Sec. IV A / IV B "non-slip")         */
};

typedef struct {
    int32_t lattice;        /* 19 (App. C) or 27 (Sec. II)                                   */
    int32_t nx, ny, nz;     /* cells per axis, 1 .. LBM_MAX_EXTENT, nx ny nz < 2^31          */
    int32_t bc[3];          /* LBM_BC_* for x, y, z                                          */
    int32_t eos;            /* LBM_EOS_*                                                     */
    double eos_p[5];        /* EOS parameters, see above                                     */
    double G;               /* interaction strength of Eq. e15 (Sec. III A uses -1)          */
    double G_ads;           /* fluid-solid strength of F_ads (Sec. III E); 0 = neutral wall  */
    double kappa;           /* surface-tension tuning of Eq. e18                             */
    double sigma;           /* mechanical-stability parameter of Eq. e17                     */
    double s[10];           /* relaxation rates s0, s1, s2, s2b, s3, s3b, s4, s4b, s5, s6    */
                            /* of Eq. e12, each in (0, 2)                                    */
    int32_t variable_nu;    /* 1: nu(rho) = nu_v + (nu_l - nu_v)(rho - rho_v)/(rho_l - rho_v) */
    double nu_l, nu_v;      /* (Sec. IV A) replaces s2 per cell; 0: s2 is used everywhere    */
    double rho_l, rho_v;
    double g[3];            /* body force per unit mass (F includes rho g)                   */
    double psi_ext_rho;     /* C-S only: cells with rho >= this evaluate p_EOS - rho c_s^2   */
                            /* in float-float arithmetic (~44 bits; the liquid branch, where */
                            /* the two terms of p_EOS nearly cancel); a negative value       */
                            /* selects the default b * rho_c = 0.52177 (critical density);   */
                            /* +inf: never                                                   */
    int32_t zchunk;         /* tuning: z planes one collide block marches through; 0 = chosen */
                            /* from the domain size (results do not depend on it)            */
    int32_t store;          /* LBM_STORE_FP32 (default) or LBM_STORE_FP16.  The paper stores */
                            /* populations in full precision; FP16 halves their bytes and    */
                            /* its error against the FP64 oracle is reported per result.     */
                            /* FP16 contexts step with the whole-grid kernels and cannot     */
                            /* join a batch.                                                 */
    int32_t onepass;        /* 1: one pass per step over two population copies (read one,    */
                            /* write the other, pull streaming): the collide pass computes   */
                            /* rho and psi of each tile and a one-cell border itself, so a   */
                            /* step has no separate density/psi pass (psi is formed on       */
                            /* demand for lbm_get_psi / lbm_get_moments); same results bit   */
                            /* for bit, twice the population memory.  Periodic boundaries,   */
                            /* no solid mask, FP32 store; cannot join a batch.  0: the       */
                            /* in-place two-pass step (default).  2 (LBM_ONEPASS_STAGED):    */
                            /* the one-pass step with each plane's populations staged in     */
                            /* shared memory by tensor copies (nx a multiple of 32, ny of 4; */
                            /* see lbm_staged_copies).                                       */
    int32_t store_layout;   /* FP16 store only.  LBM_LAYOUT_AUTO (0, default): when nx is    */
                            /* even, x is periodic and no solid mask is given, one 4-byte    */
                            /* word holds the slots of cells x and x + nx/2 and each thread  */
                            /* updates both (x-paired layout); otherwise one slot per cell.  */
                            /* LBM_LAYOUT_SINGLE (1): always one slot per cell.  Results are */
                            /* the same bit for bit; the layout changes speed only.          */
} lbm_params;

#define LBM_ONEPASS_STAGED 2
#define LBM_LAYOUT_AUTO 0
#define LBM_LAYOUT_SINGLE 1

/* Fills *p with the paper's defaults: D3Q19, 32^3 periodic, no EOS, G = -1,
 * s0 = s1 = 1, s2b = s3b = 0.6, others 1.2 (text after Eq. e12), sigma = 0.1
 * (Sec. III A), everything else 0, psi_ext_rho = -1 (default threshold),
 * zchunk = 0 (automatic). */
void lbm_default_params(lbm_params* p);

/* Validates *params, allocates the device state on the current device and
 * binds the context to `cuda_stream`.  *out receives the context, or NULL on
 * error.  Errors: LBM_ERR_ARG (bad lattice, sizes, rates outside (0,2),
 * G == 0 with an EOS, ...), LBM_ERR_OOM, LBM_ERR_CUDA.  The message of a
 * failed create is returned by lbm_last_error(NULL). */
lbm_status lbm_create(const lbm_params* params, void* cuda_stream, lbm_ctx** out);

/* Sets f_bar(t = 0) = M^-1 m^eq(rho, u) (Eq. e13) on every fluid cell and
 * computes psi.  rho: N floats; u: 3 N floats (u_x, u_y, u_z planes); solid:
 * N bytes (nonzero = solid cell) or NULL for none.  Solid cells carry no
 * populations and report rho = u = 0.  Resets the step counter and any sticky
 * error.  The solid mask may only be passed on the first call or unchanged in
 * "has solid" status (a context created without solids that later gets a mask
 * is accepted; the mask is copied). */
lbm_status lbm_init_fields(lbm_ctx* ctx, const float* rho, const float* u, const uint8_t* solid,
                           int ptrs_on_device);

/* Enqueues n >= 0 time steps on the context's stream and returns without
 * waiting.  Returns a sticky error recorded by an earlier lbm_sync.  A domain
 * with walls or solids is stepped through the tile path of the batches below
 * (same results, solid-free tiles skip the solid tests). */
lbm_status lbm_step(lbm_ctx* ctx, int32_t n);

/* Waits for the context's stream and reads the device status word:
 * LBM_ERR_UNSTABLE (NaN/Inf or rho <= 0 seen) or LBM_ERR_EOS_RANGE (psi^2 < 0
 * seen) become sticky. */
lbm_status lbm_sync(lbm_ctx* ctx);

/* rho (N floats) and u = (sum f e + F/2)/rho (3 N floats) of the current state
 * (Sec. II A).  Either pointer may be NULL.  sums (4 doubles, host, may be
 * NULL) receives the FP64 totals over fluid cells: sum rho, sum rho u_x,
 * sum rho u_y, sum rho u_z, reduced in a fixed order (deterministic).
 * Synchronises the stream and returns the status as lbm_sync does. */
lbm_status lbm_get_moments(lbm_ctx* ctx, float* rho, float* u, double* sums, int ptrs_on_device);

/* psi (Sec. II C) of the current state, N floats (0 on solid cells). */
lbm_status lbm_get_psi(lbm_ctx* ctx, float* psi, int ptrs_on_device);

/* Checkpoint: the populations of the current state in natural order
 * (f_bar_i(x, t) in plane i), Q N floats, whatever the internal AA phase. */
lbm_status lbm_get_populations(lbm_ctx* ctx, float* f, int ptrs_on_device);

/* Restore: sets the populations (Q N floats, natural order), recomputes psi,
 * clears sticky errors.  The step counter is kept. */
lbm_status lbm_set_populations(lbm_ctx* ctx, const float* f, int ptrs_on_device);

/* Rebinds the context to another stream (after the caller ordered the two). */
lbm_status lbm_set_stream(lbm_ctx* ctx, void* cuda_stream);

/* Kernel timing: when enabled, lbm_step records CUDA events on the context's
 * stream between its kernel launches.  lbm_get_kernel_timing synchronises and
 * returns the accumulated milliseconds and launch counts of the two step
 * kernels since the last reset: [0] = density/psi pass, [1] = fused
 * collide-stream pass.  Enabling resets the counters. */
lbm_status lbm_set_kernel_timing(lbm_ctx* ctx, int enable);
lbm_status lbm_get_kernel_timing(lbm_ctx* ctx, double ms[2], int64_t launches[2]);

/* Number of steps taken since lbm_init_fields (or -1 for a NULL context). */
int64_t lbm_step_count(const lbm_ctx* ctx);

/* Total device bytes the context holds.  Calls with host pointers
 * (ptrs_on_device = 0) add a staging buffer on first use -- 4 floats per cell
 * for fields, Q per cell for populations -- that is kept until lbm_destroy. */
size_t lbm_device_bytes(const lbm_ctx* ctx);

/* Device bytes a context created from *params holds after lbm_init_fields
 * with device pointers (with_solid != 0: with a solid mask), without creating
 * it: the populations (Q planes padded to 64 cells; two copies with onepass,
 * half-size slots with the FP16 store plus two FP32 density fields), psi, the
 * status word and the reduction scratch, plus 5 bytes per cell for a mask.  For admission
 * control under a memory budget; the paper has no counterpart.  Errors: as
 * lbm_create's validation (LBM_ERR_ARG), bytes == NULL. */
lbm_status lbm_estimate_bytes(const lbm_params* params, int32_t with_solid, size_t* bytes);

/* Contact detector for droplet impact (Sec. III E: contact time; Sec. IV B:
 * contact time on a wall with a cylinder).  A fluid cell is liquid when its
 * rho (formed as lbm_get_moments forms it) exceeds rho_threshold (the text
 * defines liquid and contact in words; the usual reading is the mid-density
 * (rho_l + rho_v) / 2).  Writes six int32:
 *   out[0] liquid fluid cells with at least one solid lattice neighbour
 *          (an interior solid cell or a wall plane);
 *   out[1] liquid cells in the first layer above a bottom wall (z = 0, only
 *          when z has walls), the spreading footprint;
 *   out[2], out[3] min and max x of those floor cells (INT32_MAX, INT32_MIN
 *          when there are none); out[4], out[5] the same for y.
 * ptrs_on_device != 0: `out` is device memory; the call only enqueues on the
 * context's stream (so many contexts can write into one buffer and be read
 * with one copy).  0: host memory; the call synchronises and returns the
 * status as lbm_sync does.  Domains without walls or solids report 0 contacts.
 * The paper has no such entry point; it reads contact from its snapshots. */
lbm_status lbm_contact(lbm_ctx* ctx, float rho_threshold, int32_t* out, int ptrs_on_device);

/* Frees the device state.  Waits for the stream first.  NULL is ignored. */
void lbm_destroy(lbm_ctx* ctx);

/* ---------------------------------------------------------------- batches
 * Many independent domains advanced together (the paper's method applied to a set
 * of jobs; the paper itself runs one domain at a time).  Every member is cut into
 * tiles (32 x 4 columns by default, see LBM_BATCH_SHAPES) and runs of z planes; a
 * tile whose cells have no solid
 * neighbour (mask or wall) goes to a group without solid handling.  Groups are
 * keyed by (lattice, solid handling, physical parameters); each time step costs,
 * per group and per 64 members, one collide-stream launch and one density/psi
 * launch whose blocks are tiles of all those members, and the groups of one pass
 * run concurrently.  Per cell the arithmetic is the single-domain kernels', so
 * every member evolves bitwise as if stepped alone.  Runs of steps are replayed
 * from one CUDA graph (a device-side loop), so n steps cost one graph launch.
 * lbm_step itself takes this path (a batch of one) for a domain with walls or
 * solids, unless kernel timing is on.
 *
 * lbm_batch_create: ctxs are n >= 1 distinct, initialised contexts on the current
 *   device that have taken the same number of steps modulo 2, each holding fewer
 *   than 2^32 population values (Q x cells rounded up to 64); the batch keeps the
 *   pointers (the caller keeps ownership and must not destroy a member while the
 *   batch exists).  A member re-initialised with another solid mask is re-tiled
 *   at the next lbm_batch_step.  Work is enqueued on cuda_stream; the caller
 *   orders it with the members' streams.  A member's own zchunk, if set, is used
 *   until lbm_batch_tune chooses one.
 *   Errors: LBM_ERR_ARG, LBM_ERR_STATE, LBM_ERR_OOM, LBM_ERR_CUDA (message in
 *   lbm_last_error(NULL)).
 * lbm_batch_step: enqueues n >= 0 steps of every member (does not wait) and
 *   advances their step counters.  LBM_ERR_STATE if members were stepped apart.
 * lbm_batch_sync: waits and returns the first sticky member error (lbm_sync).
 * lbm_batch_tune: autotunes each group's launch shape on the live state, in two
 *   stages, by timing the collide launches of every group for trial_steps steps:
 *   first every tile shape (LBM_BATCH_SHAPES) with automatic z-chunks, then, for
 *   the fastest shape, each candidate z-chunk (automatic, 1, 4, 8, 16, 32 planes
 *   per block, or a whole column per block).  A group and the group of the same lattice and physics
 *   with the other solid handling share members, so they take one shape (the
 *   one with the least summed time); the z-chunk is per group.  Keeps the
 *   fastest per group and writes its z-chunk to
 *   zchunk_out[g] for g < max_groups (0 = automatic, 2^30 = whole columns;
 *   lbm_batch_group reads the shape).  The members advance by 12 x (trial_steps + 1) steps.
 * lbm_batch_info: number of groups, tiles of all launches of one pass, graph mode
 *   (0 not recorded yet, 1 device-side WHILE loop, 2 replayed two-step graph).
 * lbm_batch_group: lattice (19 | 27), solid handling (0 | 1), tile shape and
 *   z-chunk of group `group` in [0, ngroups); NULL outputs are skipped.
 * lbm_batch_set_group: sets a group's tile shape (0 .. LBM_BATCH_SHAPES - 1) and
 *   z-chunk (0 = automatic) and re-tiles it; the group of the same lattice and
 *   physics with the other solid handling takes the same shape.  Results do not
 *   depend on either.
 *   LBM_ERR_ARG for an unknown group, shape or a negative z-chunk.
 * Tile shapes (width x height in cells; resident blocks per SM on D3Q19 / D3Q27):
 *   0: 32 x 4 (7 / 5), the single-domain kernels' shape; 1: 32 x 2 (14 / 10);
 *   2: 16 x 8 (7 / 5); 3: 16 x 4 (14 / 10); 4: 32 x 4 (6 / 4).  16-wide tiles
 *   waste fewer threads on domains whose x extent is not a multiple of 32. */
#define LBM_BATCH_SHAPES 5
typedef struct lbm_batch lbm_batch;
lbm_status lbm_batch_create(lbm_ctx* const* ctxs, int32_t n, void* cuda_stream, lbm_batch** out);
lbm_status lbm_batch_step(lbm_batch* batch, int32_t n);
lbm_status lbm_batch_sync(lbm_batch* batch);
lbm_status lbm_batch_tune(lbm_batch* batch, int32_t trial_steps, int32_t* zchunk_out, int32_t max_groups);
lbm_status lbm_batch_info(const lbm_batch* batch, int32_t* ngroups, int32_t* ntiles, int32_t* graph_mode);
lbm_status lbm_batch_group(const lbm_batch* batch, int32_t group, int32_t* lattice, int32_t* solids, int32_t* shape,
                           int32_t* zchunk);
lbm_status lbm_batch_set_group(lbm_batch* batch, int32_t group, int32_t shape, int32_t zchunk);
void lbm_batch_destroy(lbm_batch* batch);
const char* lbm_batch_last_error(const lbm_batch* batch);

/* Totals without allocation.  The paper has no counterpart: this is a service
 * for callers that cannot allocate device memory while they run -- hosts whose
 * device memory is handed out up front by their own pool allocator (a
 * cudaMalloc from inside them would go around that budget) and real-time loops
 * that may not block on cudaMalloc / cudaFree, which can synchronise the device.
 * Computes, in FP64 and in a fixed order (deterministic), totals[0] = sum rho,
 * totals[1..3] = sum rho u_x, sum rho u_y, sum rho u_z over ncell cells of
 * caller-held arrays rho (ncell floats) and u (3 ncell floats, the layout
 * lbm_get_moments writes) in memory of the current device; totals is a pointer
 * to 4 doubles in memory of the current device.  Pointers that are NULL, not
 * naturally aligned, or not device / managed memory of the current device are
 * refused with LBM_ERR_ARG before any launch.  Enqueued on cuda_stream
 * (NULL = legacy default stream); does not wait.
 * It calls no cudaMalloc / cudaFree: its scratch (one partial sum per block)
 * is a fixed 512 KB device array in the library that every GPU loading the
 * library holds until the process exits, so ncell is limited to
 * LBM_NOALLOC_MAX_CELLS; larger ncell (or ncell < 1) returns LBM_ERR_ARG with a
 * message in lbm_last_error(NULL).  The first call on a device looks up the
 * array's device address (once per device, with that device current) and keeps
 * it for the life of the process; make that first call before any stream
 * capture.  A device reset (cudaDeviceReset) after that first call is not
 * supported: the kept address would be stale.  All calls on one device share
 * the array: calls that may overlap on that GPU (e.g. on two streams) race;
 * serialise them.  The partials are rewritten by every call, so no state
 * carries over between calls. */
#define LBM_NOALLOC_MAX_CELLS 33554432
lbm_status lbm_field_totals_noalloc(const float* rho, const float* u, int64_t ncell, double* totals,
                                    void* cuda_stream);

/* Message of the last error on ctx (ctx == NULL: the last failed lbm_create or
 * lbm_field_totals_noalloc on this thread).  Never NULL. */
const char* lbm_last_error(const lbm_ctx* ctx);

/* Name of a status code. */
const char* lbm_status_string(lbm_status s);

/* Debugging aid (the paper has no counterpart): a library compiled with LBM_BOUNDS_CHECK=1 checks
 * every population, psi and psi-ring access of the step kernels against its array before making
 * it; an access outside is counted and redirected to the array's first element instead of being
 * made.  Returns the count since the library was loaded, on the current device; 0 in the normal
 * build, where the checks are compiled away. */
uint64_t lbm_debug_bounds_violations(void);

/* Staged one-pass step (the paper has no counterpart; a data-movement choice).  A context created
 * with onepass = LBM_ONEPASS_STAGED (nx a multiple of 32, ny of 4) stages, for every z plane a
 * block needs, the pulled populations of its 32 x 4 tile and one-cell border in shared memory with
 * one tensor copy (TMA) per population; the results are those of the other steps bit for bit.  It
 * measured slower than the unstaged one-pass step on one GB300 (256^3: D3Q19 1.00 against 0.68 ms).
 * lbm_staged_copies returns 1 for such a context, 0 otherwise (or for NULL).
 * Every wait of the kernel on its copies is bounded in time (about 2 s); past the limit the block
 * abandons the step, the status word records it and the next lbm_sync / lbm_get_moments returns
 * LBM_ERR_TIMEOUT (sticky until the next lbm_init_fields or lbm_set_populations).
 * lbm_debug_stage_timeout(ctx, 1) makes every later staged step expect more bytes than its copies
 * deliver, with a wait limit of about 10 ms, so that the timeout path can be tested; (ctx, 0)
 * restores normal steps.  LBM_ERR_STATE if ctx does not stage. */
int32_t lbm_staged_copies(const lbm_ctx* ctx);
lbm_status lbm_debug_stage_timeout(lbm_ctx* ctx, int32_t enable);

#ifdef __cplusplus
}
#endif

#endif /* LBM_H */
