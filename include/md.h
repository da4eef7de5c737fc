/*
 * md.h -- C ABI of the GB300 soft-sphere molecular-dynamics library (libmd).
 *
 * The library runs the per-step short-range hot path of Rapaport, "Enhanced
 * molecular dynamics performance with a programmable graphics processor"
 * (arXiv 0911.5631) on one NVIDIA GB300 (sm_103a):
 *
 *   cell binning (Sec. 3.2, Sec. 4.2) -> neighbour list with a shell of
 *   thickness delta (Sec. 3.1, Sec. 3.4) -> pair forces, potential energy
 *   and virial from Eq. (1) (Sec. 3.4) -> velocity-Verlet ("leapfrog")
 *   integration with the delta/2 rebuild rule (Sec. 3.1, steps (a)-(e)),
 *   with periodic cell-order reordering of the atoms (Sec. 3.5).
 *
 * Units are reduced MD units: sigma = epsilon = m = 1.  The region is a
 * rectangular periodic box centred at the origin.
 *
 * Conventions for every call:
 *   - Return value: MD_OK (0) or a negative MD_E* code.  md_last_error()
 *     gives a human-readable message for the handle's most recent failure.
 *   - Host arrays are caller owned; the library copies from/to them and
 *     never keeps a pointer.  "_device" variants take device pointers in the
 *     same layout (for example PyTorch CUDA tensors); the caller must keep
 *     them valid until the call returns.
 *   - Atom arrays are N x 3 row-major doubles (x, y, z per atom) in the
 *     caller's atom order ("user order"); the library's internal reordering
 *     is invisible through this interface.
 *   - A handle is not thread safe; distinct handles may be used from
 *     distinct host threads.
 *   - All work is ordered on the handle's CUDA stream.  Calls that return
 *     data to the host synchronise that stream.
 */
#ifndef MD_H
#define MD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- error codes ------------------------------------------------------ */
#define MD_OK          0
#define MD_EINVAL     -1  /* bad argument (sizes, geometry, NULL pointer)       */
#define MD_ENOMEM     -2  /* device or host allocation failed                    */
#define MD_ECUDA      -3  /* a CUDA runtime call failed; see md_last_error      */
#define MD_ESTATE     -4  /* call order violated (e.g. md_step before state)    */
#define MD_EOVERFLOW  -5  /* neighbour capacity exceeded and regrowth failed    */
#define MD_EUNSTABLE  -6  /* non-finite coordinates or velocities, or two atoms
                             overlapped so closely that a pair force left the
                             representable range                              */
#define MD_ENODEV     -7  /* no usable CUDA device                              */

/* ---- precision forms -------------------------------------------------- */
/* MD_PREC_MIXED: pair arithmetic in FP32 on cell-relative coordinates,
 *   positions held as FP64 cell-relative offsets, per-atom force sums in
 *   int64 fixed point (scale 2^32, independent of summation order),
 *   velocities in FP32, FP64 in the position update and the reductions.
 * MD_PREC_FP64: every arithmetic step in FP64. */
#define MD_PREC_MIXED 0
#define MD_PREC_FP64  1

/* Optional parameters for md_create.  Fill with md_default_params() and
 * change fields as needed. */
typedef struct md_params {
    int32_t precision;        /* MD_PREC_MIXED (default) or MD_PREC_FP64          */
    int32_t reorder_interval; /* N_R of Sec. 5.5: atoms are put back into cell
                                 order at the first rebuild at least this many
                                 steps after the previous reorder; 0 = never.
                                 Default 100.                                  */
    int32_t cell_list_only;   /* 1: no neighbour list; every step re-bins the
                                 atoms and takes forces straight from the 27
                                 cells around each atom (Sec. 3.1, cells only).
                                 Requires skin == 0.  Default 0.               */
    int32_t even_cells;       /* 1: round each G_d down to an even number (the
                                 rule behind the cell counts of Tables 1 and 5).
                                 Default 0: G_d = floor(L_d / r_n) (Sec. 3.1). */
    int32_t nbr_capacity;     /* initial neighbour slots per atom; 0 = estimate
                                 from density and r_n.  Grown automatically.   */
    int32_t use_graphs;       /* 1 (default): md_step replays CUDA graphs whose
                                 rebuild branch is a device-side conditional
                                 node (checked every third step; a step whose
                                 rebuild is due in between waits and runs
                                 before md_step returns); 0: plain stream
                                 launches (same results, bit for bit).         */
    int32_t device;           /* CUDA device ordinal; -1 (default) = current   */
    int32_t shell_bins;       /* 1 (default): the build sorts each atom's list
                                 by distance, and a step reads only the entries
                                 that the largest displacement since the build
                                 can have brought inside r_c.  0: every step
                                 reads every entry (the same forces; in the
                                 mixed form the same bits).                    */
    double ushift;            /* constant added to Eq. (1) for r < r_c.  NaN
                                 (default) = automatic: +1 (epsilon) when r_c is
                                 2^(1/6) to 1e-12 relative (the soft-sphere
                                 potential of Sec. 3.1), else 0.               */
    void* stream;             /* cudaStream_t to run on; NULL (default) = a
                                 stream created and owned by the handle.       */
    int32_t build_kernel;     /* neighbour-list build (Sec. 3.4): MD_BUILD_AUTO
                                 (default, = MD_BUILD_THREAD), MD_BUILD_THREAD
                                 (one thread per atom scans its 27 cells) or
                                 MD_BUILD_WARP (warp-cooperative: one warp per
                                 home cell gathers the 27 cells' candidates
                                 once, its lanes test them against one home
                                 atom at a time).  The lists hold the same
                                 pairs; in the mixed form the trajectories
                                 are the same bits.                           */
    int32_t variant;          /* 0 (default), or one MD_VARIANT_* flag: a step
                                 kernel variant of the paper's ablations (mixed
                                 form with a neighbour list only).  Every
                                 variant gives the default's trajectories, bit
                                 for bit; only the speed differs.             */
    int64_t reserved[5];
} md_params;

/* Kernel variants of the paper's ablations (Sec. 5): */
#define MD_VARIANT_PLAIN_LOADS 1  /* gathers of neighbour coordinates through
                                     plain coherent loads instead of the
                                     read-only path (the texture cache of
                                     Sec. 4.4)                                */
#define MD_VARIANT_LIST_ROWS   2  /* W transposed: each atom's entries
                                     contiguous (entry m of atom i at
                                     i * capacity + m) instead of a warp's 32
                                     columns interleaved                      */
#define MD_VARIANT_BLOCK64     4  /* force + integrate kernel with 64 threads
                                     per block (Table 6; default 128)         */
#define MD_VARIANT_BLOCK256    8  /* ... with 256 threads per block           */

#define MD_BUILD_AUTO   0  /* the faster build on the workloads measured:
                              MD_BUILD_THREAD                                 */
#define MD_BUILD_THREAD 1
#define MD_BUILD_WARP   2

/* Geometry and resource plan, computed on the host without a GPU. */
typedef struct md_plan_t {
    int32_t G[3];             /* cells per dimension                            */
    int32_t nbr_capacity;     /* initial neighbour slots per atom               */
    int64_t n_cells;          /* G[0] * G[1] * G[2]                             */
    double w[3];              /* cell widths L_d / G_d                          */
    double rn;                /* r_c + skin                                     */
    double ushift;            /* resolved potential shift                       */
    int64_t device_bytes;     /* device memory the handle will allocate         */
} md_plan_t;

/* Thermodynamic measurement of the current state (integer time step). */
typedef struct md_measure_t {
    double ke;                /* sum 1/2 v^2                                    */
    double pe;                /* sum over pairs of u(r) (with the shift)        */
    double virial;            /* W = sum over pairs of r_ij . f_ij              */
    double pressure;          /* (2 KE + W) / (3 V)                             */
    double temperature;       /* 2 KE / (3 N)                                   */
    double e_tot_per_atom;    /* (KE + PE) / N                                  */
    double volume;            /* L_x L_y L_z                                    */
    int64_t step;             /* steps taken since md_set_state                 */
    int64_t rebuilds;         /* neighbour-list rebuilds since md_set_state     */
    int64_t reorders;         /* cell-order reorders since md_set_state         */
    int64_t list_entries;     /* current neighbour-list length (both directions,
                                 the paper's N_p for the full list)            */
    int32_t max_neighbors;    /* largest per-atom neighbour count at last build */
    int32_t max_occupancy;    /* largest cell occupancy at last binning (N_l)   */
    int32_t nbr_capacity;     /* current neighbour slots per atom               */
    int32_t reserved;
} md_measure_t;

/* Launch/timing counters for profiling (see md_set_profiling). */
typedef struct md_kernel_stats_t {
    int64_t launches;         /* kernels launched by md_step so far             */
    int64_t step_kernel_launches; /* force+integrate launches timed below       */
    double step_kernel_ms;    /* summed CUDA-event time of those launches       */
    int64_t step_kernel_atoms;/* atoms processed by them                        */
    int64_t step_kernel_bytes;/* algorithmic bytes moved by them: per atom 116 B
                                 of state (184 B in FP64), the list count (1 B
                                 with shell_bins, else 4 B) and 4 B per list
                                 entry the step reads                        */
    int64_t rebuilds_timed;   /* rebuild branches (Sec. 3.1 (b)) timed below    */
    double rebuild_ms;        /* their summed CUDA-event time                   */
} md_kernel_stats_t;

typedef struct md_handle md_handle;

/* Fills *p with the defaults documented in md_params. */
void md_default_params(md_params* p);

/* Plans geometry for a box of edges box[0..2], n atoms, cutoff rc, shell
 * thickness skin (r_n = rc + skin, Sec. 3.1) and time step dt.  Returns
 * MD_EINVAL when n <= 0, n >= 2^26, rc <= 0, skin < 0, dt <= 0, a box edge
 * is not positive, some G_d < 3 (the 27-cell neighbourhood would alias), or
 * cell_list_only is set with skin != 0.  p may be NULL.  Needs no GPU. */
int md_plan(const double box[3], int64_t n, double rc, double skin, double dt,
            const md_params* p, md_plan_t* out);

/* Creates a simulation handle and allocates its device state (Sec. 3.1:
 * region, cutoff, shell, time step).  Same argument checks as md_plan;
 * MD_ENODEV / MD_ENOMEM / MD_ECUDA on device failure.  *out is NULL on
 * error. */
int md_create(const double box[3], int64_t n, double rc, double skin, double dt,
              const md_params* p, md_handle** out);

/* Loads positions and velocities (N x 3 each, user order, host memory).
 * Positions are wrapped into the region; atoms are binned, the neighbour
 * list is built and the forces of this state are computed, so the next
 * md_step starts from true forces.  MD_EINVAL on NULL, MD_EUNSTABLE on
 * non-finite input. */
int md_set_state(md_handle* h, const double* pos, const double* vel);
int md_set_state_device(md_handle* h, const double* pos, const double* vel);

/* Velocity adjustment, Sec. 3.1 step (f) (during equilibration): scales
 * every velocity by s = sqrt(3 N T / (2 KE)), KE the kinetic energy of the
 * current state (after the last md_step or md_set_state), so that the
 * temperature 2 KE / (3 N) becomes T.  Sec. 5's protocol calls it every 20
 * steps during the first 500.  Each velocity is multiplied in FP64 and
 * stored in the form's velocity precision; md_measure then reports the new
 * KE.  MD_EINVAL if T <= 0 or KE is 0; MD_ESTATE before md_set_state. */
int md_rescale(md_handle* h, double T);

/* Advances nsteps velocity-Verlet steps (Sec. 3.1 (a)-(e)).  The neighbour
 * list is rebuilt on the device whenever the largest displacement since the
 * last build reaches skin/2 (every step in cell-list-only mode); atoms are
 * reordered into cell order every reorder_interval steps at a rebuild.  If
 * the list outgrows its capacity the library enlarges it and resumes from
 * the step that overflowed.  Returns after the steps completed on the GPU.
 * nsteps <= 0 is a no-op.  MD_ESTATE before md_set_state. */
int md_step(md_handle* h, int64_t nsteps);

/* Kinetic and potential energy, virial, pressure and counters of the
 * current state (Sec. 3.5 global reductions, Sec. 4.3), reduced on the
 * device in FP64 in a fixed order (run-to-run deterministic). */
int md_measure(md_handle* h, md_measure_t* out);

/* Current positions (wrapped into the region) and velocities, user order. */
int md_get_state(md_handle* h, double* pos, double* vel);
int md_get_state_device(md_handle* h, double* pos, double* vel);

/* Forces on the atoms in the current state (N x 3, user order), as computed
 * by the step kernel for the last completed step. */
int md_get_forces(md_handle* h, double* f);

/* Debug views for parity checks against a reference.
 * md_debug_cells: cell index c = (c_z G_y + c_y) G_x + c_x of every atom as
 *   last binned (N int32, user order).
 * md_debug_neighbors: the unordered pairs of the current neighbour list in
 *   user ids with i < j (2 x int32 per pair, up to capacity pairs written);
 *   *count receives the number of pairs, *entries (may be NULL) the list
 *   length counting both directions. */
int md_debug_cells(md_handle* h, int32_t* cell);
int md_debug_neighbors(md_handle* h, int64_t* count, int64_t* entries, int32_t* pairs,
                       int64_t capacity);

/* Plan of an existing handle (current capacity included). */
int md_get_plan(md_handle* h, md_plan_t* out);

/* Profiling: with on != 0, md_step runs without graphs and brackets every
 * force+integrate kernel with CUDA events on the handle's stream; the
 * totals accumulate in md_kernel_stats. */
int md_set_profiling(md_handle* h, int on);
int md_kernel_stats(md_handle* h, md_kernel_stats_t* out);

/* Blocks until all work queued on the handle's stream is complete; returns
 * any error the device recorded. */
int md_sync(md_handle* h);

/* Frees the handle and all its device memory.  NULL is a no-op. */
void md_destroy(md_handle* h);

/* Message for the handle's last failure ("" if none); h may be NULL for
 * failures of md_create. */
const char* md_last_error(const md_handle* h);

/* Device self-check of the library's integer-pipe number conversions
 * (binary32<->binary64, binary32<->int64 fixed point) against the hardware
 * conversions on n hashed inputs (uses the current device).  failures[0..3]
 * receive the mismatch counts for float->double, double->float,
 * float->int64 and int64->float.  MD_ENODEV without a GPU. */
int md_selftest(int64_t n, int64_t failures[4]);

/* ---- forces without device allocation --------------------------------
 * The paper has no counterpart to this call; it serves callers that may
 * not allocate device memory -- code that runs inside a memory pool or
 * budget it does not own, or on a path where cudaMalloc/cudaFree must not
 * run because they synchronise the whole device.
 *
 * md_forces_noalloc computes, in FP64, the forces of one configuration and
 * its potential energy and virial: positions are wrapped, binned into cells
 * of width >= rc and the pair term of Eq. (1) plus ushift (NaN: the
 * automatic shift of md_params.ushift) is summed over the 27 neighbouring
 * cells -- the same numbers md_set_state + md_get_forces + md_measure give
 * for the FP64 form, up to summation order.
 *   box  region edges; each must hold at least 3 cells of width rc
 *   pos  device, n x 3 doubles;  f  device, n x 3 doubles (out)
 *   pe_vir  device, 2 doubles (out): U and W = sum over pairs of r.f
 *   stream  cudaStream_t the work is queued on (NULL: legacy default
 *           stream).  The call waits for its own work on that stream to
 *           finish before it returns (it reads back a one-word flag), so f
 *           and pe_vir are ready when it returns MD_OK.
 * MD_EUNSTABLE when a position is not finite (f and pe_vir then hold
 * meaningless numbers).
 * It allocates nothing: its working memory is one fixed scratch area of
 * MD_NOALLOC_SCRATCH_BYTES inside the library (a static device array that
 * every GPU which loads the library keeps until the process exits), so
 * n <= MD_NOALLOC_MAX_ATOMS and the cell count <= MD_NOALLOC_MAX_CELLS;
 * larger inputs return MD_EINVAL (message in md_last_error(NULL)).
 * Every call looks up the scratch address on the current device (so a
 * device reset between calls is harmless).  All calls share the scratch area, which keeps the previous call's
 * contents (the call clears what must start at zero): calls whose work
 * overlaps on the GPU -- on different streams or from different host
 * threads -- race and return wrong results. */
#define MD_NOALLOC_MAX_ATOMS 65536
#define MD_NOALLOC_MAX_CELLS 65536
#define MD_NOALLOC_SCRATCH_BYTES (4u << 20)
int md_forces_noalloc(const double box[3], int64_t n, double rc, double ushift, const double* pos,
                      double* f, double* pe_vir, void* stream);

/* ---- ensembles: many independent simulations in one launch -------------
 * The paper runs one simulation at a time.  An ensemble holds many
 * independent replicas of the mixed form (each its own box, N, r_c, skin,
 * dt and state) in one device arena, and md_ensemble_run advances any
 * subset of them in a single kernel launch: each replica is taken by one
 * thread block, or by a thread-block cluster when it is large (see
 * md_ensemble_set_shape), which runs Sec. 3.1's steps (a)-(e) for it as
 * md_set_state/md_step do -- binning, neighbour-list rebuilds at skin/2,
 * reorders every reorder_interval steps, forces, the velocity-Verlet
 * update.  Replicas share nothing, so a replica's trajectory does not
 * depend on what else runs: positions and velocities are bitwise those of
 * md_step from the same state, and KE, PE and W are summed in a fixed
 * order over 32-atom chunks, the same numbers whatever the launch shape.
 *
 * Memory: md_ensemble_create reserves arena_bytes of device memory once;
 * md_ensemble_add carves a replica's arrays out of it (MD_ENOMEM when they
 * do not fit: the caller's admission signal) and md_ensemble_remove gives
 * them back.  Replica ids are small non-negative integers, reused after
 * removal.  One ensemble is not thread-safe; calls are ordered on its
 * stream.  Errors of a replica (overflow of its neighbour capacity, an
 * unstable state) stop that replica only; md_ensemble_status reports them.
 */
typedef struct md_replica_desc {
    double box[3];             /* region edges, each at least 3 (rc + skin)   */
    int64_t n;                 /* atoms, 1 .. 2^26 - 1                         */
    double rc, skin, dt;       /* cutoff, shell, time step (Sec. 3.1)          */
    double ushift;             /* added to u below rc; NaN: +1 for the WCA rc  */
    int32_t reorder_interval;  /* reorder into cell order every this many
                                  steps at the next rebuild (Sec. 5.5); 0 never */
    int32_t nbr_capacity;      /* neighbour slots per atom; 0: from density    */
    int64_t reserved[4];       /* must be zero                                 */
} md_replica_desc;

typedef struct md_ensemble md_ensemble;

/* Creates an ensemble with an arena of arena_bytes on device (-1: current)
 * and up to max_replicas replica ids.  stream: cudaStream_t for all work
 * (NULL: the ensemble creates its own). */
int md_ensemble_create(int64_t arena_bytes, int32_t max_replicas, int32_t device, void* stream,
                       md_ensemble** out);

/* Adds a replica with positions and velocities (host, n x 3 doubles each,
 * copied before return; the copies do not wait for runs in flight).  Its
 * state is loaded (wrapped, binned, listed, forces computed) at the start of
 * the next md_ensemble_run that includes it.  *id receives its id.
 * MD_EINVAL on a bad description, MD_ENOMEM when the arena or the id table
 * is full. */
int md_ensemble_add(md_ensemble* e, const md_replica_desc* d, const double* pos, const double* vel,
                    int32_t* id);

/* Frees a replica's arena space and id (waits for the last run that
 * included it, not for later ones). */
int md_ensemble_remove(md_ensemble* e, int32_t id);

/* Advances replicas ids[0..count) by nsteps[k] >= 0 steps each in one
 * launch (asynchronous; replicas added since their last run are loaded
 * first, so nsteps 0 only loads them).  An id may appear once per call.
 * The launch is replayed from a CUDA graph captured on the ensemble's stream
 * the first time a launch shape is used; a stream that cannot be captured
 * (the legacy default stream) gives MD_ECUDA. */
int md_ensemble_run(md_ensemble* e, int32_t count, const int32_t* ids, const int64_t* nsteps);

/* Waits for the ensemble's stream. */
int md_ensemble_sync(md_ensemble* e);

/* Waits until at most in_flight (0 .. 7) of the runs queued so far are
 * unfinished (0: md_ensemble_sync).  A request loop that queues the next
 * slice before it retires the last one keeps the GPU busy with
 * md_ensemble_wait(e, 1). */
int md_ensemble_wait(md_ensemble* e, int32_t in_flight);

/* MD_OK, or the error that stopped the replica (MD_EOVERFLOW, MD_EUNSTABLE).
 * This, md_ensemble_measure and md_ensemble_get_state wait for the last run
 * that included the replica, not for later runs, and copy on a stream of
 * the ensemble's own, so they overlap runs queued after it. */
int md_ensemble_status(md_ensemble* e, int32_t id);

/* Thermodynamic state of a replica after its last run (as md_measure). */
int md_ensemble_measure(md_ensemble* e, int32_t id, md_measure_t* out);

/* Positions (wrapped) and velocities of a replica in its user order
 * (host, n x 3 doubles each) after its last run. */
int md_ensemble_get_state(md_ensemble* e, int32_t id, double* pos, double* vel);

/* Start and end of each listed replica's work in the last run that
 * included it, in ms after that run's launch began on the device (device
 * clock); -1 for a replica not yet run. */
int md_ensemble_times(md_ensemble* e, int32_t count, const int32_t* ids, double* start_ms, double* end_ms);

/* Launch shape for md_ensemble_run: threads per block (a multiple of 32,
 * 64 .. 1024; 0: 256), blocks (0: as many as fit on the device at once),
 * and teams: a replica of at least team_atoms atoms (0: 8192) is run by a
 * thread-block cluster of `cluster` blocks (1 .. 8; 0: 8) that split its
 * atoms and meet at hardware cluster barriers, so one big replica is not
 * limited to one SM; cluster 1 gives every replica one block. */
int md_ensemble_set_shape(md_ensemble* e, int32_t block, int32_t grid, int32_t cluster, int64_t team_atoms);

/* Autotuner: runs ids for probe_steps steps under each of 6 candidate
 * shapes -- (threads per block, cluster size, team_atoms) -- (these are
 * real steps: the replicas advance by 6 x probe_steps), keeps the fastest
 * and returns its block and cluster size in *block, *cluster (either may
 * be NULL). */
int md_ensemble_autotune(md_ensemble* e, int32_t count, const int32_t* ids, int64_t probe_steps,
                         int32_t* block, int32_t* cluster);

/* Arena bytes a replica of this description needs (0 on a bad one), and
 * the largest free arena block right now. */
int64_t md_ensemble_replica_bytes(const md_replica_desc* d);
int64_t md_ensemble_free_bytes(const md_ensemble* e);

/* Frees everything.  NULL is a no-op. */
void md_ensemble_destroy(md_ensemble* e);

/* Message for the ensemble's last failure ("" if none); e may be NULL for
 * failures of md_ensemble_create. */
const char* md_ensemble_last_error(const md_ensemble* e);

/* Static description of an error code. */
const char* md_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* MD_H */
