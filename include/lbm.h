/*
 * lbm.h — C ABI of the GB300 (sm_103a) library for the growing-tissue lattice
 * Boltzmann method of Killeen, Partridge, Bertrand & Lee (arXiv 2303.02210).
 *
 * One simulation is one D2Q9 lattice, W columns (x, periodic) by H rows
 * (y, the growth direction), whose populations stay resident in device memory.
 * Every call that does arithmetic launches hand-written CUDA kernels on the
 * stream given at creation; nothing is computed on the host except the
 * initial front profile (App. A, first paragraph) and argument marshalling.
 *
 * Conventions for every function:
 *  - Return value: 0 (LBM_OK) on success, a negative LBM_ERR_* code on
 *    error, never an exception or an abort. lbm_strerror() names a code.
 *  - Host pointers are caller-owned and only read or written during the call.
 *  - Device pointers are caller-owned; the library never frees them.
 *  - A handle is not thread-safe: calls on one handle must be serialised.
 *  - Calls marked "syncs" wait for the handle's stream; all others only
 *    enqueue work and return.
 */
#ifndef LBM_GB300_LBM_H
#define LBM_GB300_LBM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- return codes ---- */
#define LBM_OK 0
#define LBM_ERR_INVALID_ARG (-1) /* a parameter is out of range or a pointer is NULL */
#define LBM_ERR_OOM (-2)         /* device allocation failed or the arena is too small */
#define LBM_ERR_CUDA (-3)        /* a CUDA call failed (see lbm_last_cuda_error) */
#define LBM_ERR_CAPACITY (-4)    /* one step asked for more divisions than the planner holds */
#define LBM_ERR_NO_DEVICE (-5)   /* no CUDA device of compute capability 10.3 */
#define LBM_ERR_BATCH_FULL (-6)  /* lbm_batch_attach: every slot of the batch is taken */

/* ---- device status bits (lbm_stats_t.status; sticky until lbm_clear_status) ---- */
#define LBM_STATUS_FRONT_AT_TOP 1   /* mass reached row H-1 (the top wall) */
#define LBM_STATUS_GROWTH_STARVED 2 /* a step accepted fewer than n_s divisions */
#define LBM_STATUS_CAPACITY 4       /* n_s exceeded the planner capacity, or the exact mass sum
                                       overflowed int64 (a runaway lattice); growth skipped */
#define LBM_STATUS_TIMEOUT 8        /* a bulk copy did not complete in time; the step was abandoned */

/* ---- enumerations used in lbm_params_t ---- */
enum {
    LBM_GROW_NONE = 0,
    LBM_GROW_BULK = 1,    /* uniform over occupied active nodes (Sec. III) */
    LBM_GROW_DENSITY = 2, /* accept with p = 1 - rho/rho0 if rho > rho_c (Eq. 5) */
    LBM_GROW_EDGE = 3,    /* occupied and at most edge_depth rows below the front */
    LBM_GROW_BAND = 4     /* occupied and within band_rows of the rear wall (App. B) */
};
enum { LBM_FRONT_FLAT = 0, LBM_FRONT_SINUSOIDAL = 1, LBM_FRONT_FULL = 2 };
enum { LBM_WALL_FIXED = 0, LBM_WALL_ADVANCE = 1 };
enum { LBM_NEGFIX_LITERAL = 0, LBM_NEGFIX_RESCALE = 1 };
enum { LBM_FP32 = 0, LBM_FP64 = 1, LBM_FP16 = 2, LBM_BF16 = 3 };
enum { LBM_D2Q9 = 0, LBM_D2Q7 = 1 };

/*
 * Model parameters (App. A parameter list; Sec. II for the model).
 *  tau          BGK relaxation time, > 1/2 (Eq. 2)
 *  mu           substrate friction, u* = (1 - mu) u (Sec. II, below Eq. 3)
 *  rho_c        occupancy threshold of the two-step bounce-back (Sec. II)
 *  rho_cell     mass of one division (Sec. II)
 *  sigma        noise amplitude, eta~ uniform in [-sigma, sigma] (Eq. 4)
 *  rho0         density where density-dependent growth stops (Eq. 5)
 *  growth_rate  g: n_s = g M / rho_cell sites per step (Sec. II)
 *  rho_init, rho_jitter   initial density rho_init (1 + jitter (2U - 1))
 *  front_row, front_amp   initial front height and perturbation amplitude
 *  front_kmin, front_kmax wavenumbers of the sinusoidal initial front
 *  wall_min_gap, wall_w_factor   rear wall kept max(gap, factor w) behind hbar
 *  edge_depth, band_rows  growth-mode extents
 *  y_periodic   1: periodic in y too, no walls (test lattices)
 *  seed, sim_id Philox key and counter word 3
 *  precision    LBM_FP32 (fast path), LBM_FP64 (debug path, bit-exact
 *               with the CPU oracle), or LBM_FP16 / LBM_BF16: 16-bit storage
 *               of the deviation f_i - c_i from the rest state, c_i =
 *               w_i rho_init rounded to the 16-bit type (exact for the void
 *               and for f_i = c_i), FP32 arithmetic, 36 bytes per node
 *               update
 *  update_kernel 0: choose (the TMA-staged kernel for FP32 and 16-bit
 *               storage with walls in y, else the plain-load kernel; its
 *               form from the library's tuned table, a sweep of the forms
 *               and planner grids measured per storage type and lattice
 *               width (the entry of the largest tuned width not above W);
 *               the bulk-store form (6) only when W is a multiple of 4);
 *               1: plain-load kernel; 2: TMA-staged kernel, two-row form;
 *               3: TMA-staged kernel, four-row form (2-4: not FP64, and
 *               y_periodic = 0 only); 4: the two-row form with the
 *               divisions injected into global memory first; 5: choose for
 *               a simulation that shares the GPU with others (the four-row
 *               form where the TMA-staged kernel applies); 6: the two-row form
 *               whose results leave through a shared output tile and one
 *               bulk tensor store per tile (FP32 only; widths that are not
 *               a multiple of 4 take form 2)
 *  lattice      LBM_D2Q9, or LBM_D2Q7: the paper's triangular lattice (Sec.
 *               II; Eq. 3 with 4, 8, 2, weights 1/2 and 1/12), rows of nodes
 *               along x with the odd rows shifted by half a spacing, rows
 *               sqrt(3)/2 apart, directions 1:(1,0) 2:(1/2,s) 3:(-1/2,s)
 *               4:(-1,0) 5:(-1/2,-s) 6:(1/2,-s), s = sqrt(3)/2; FP32 or FP64,
 *               update_kernel 0, 1, 2 or 5 (0, 2 and 5: the one TMA-staged
 *               D2Q7 kernel, two-row tiles, for FP32 with walls in y, else
 *               the plain-load kernel; 3 and 4 are refused), an even H if
 *               y_periodic. Populations have 7 planes instead of 9
 *  plan_blocks  blocks of the planner's cooperative grid: 0 = the tuned
 *               table's value for the storage type and width (else one block
 *               per 16 mask words or 512 divisions of the capacity, at least
 *               2, at most a quarter of the SMs); 1..1024 = that many, at
 *               most the resident count (more: LBM_ERR_INVALID_ARG). The
 *               results do not depend on it.
 */
typedef struct {
    double tau, mu, rho_c, rho_cell, sigma, rho0, growth_rate;
    double rho_init, rho_jitter, front_row, front_amp, wall_min_gap, wall_w_factor;
    uint64_t seed;
    int32_t width, height, growth_mode, edge_depth, band_rows, front_kind;
    int32_t front_kmin, front_kmax, wall_mode, negfix_mode, y_periodic;
    uint32_t sim_id;
    int32_t precision;
    int32_t update_kernel;
    int32_t lattice;
    int32_t plan_blocks;
} lbm_params_t;

/* Counters and observables after the latest completed step. */
typedef struct {
    int64_t step;          /* completed steps */
    int64_t ns_last;       /* n_s requested by the latest step */
    int64_t ns_total;      /* sum of n_s over all steps */
    int64_t div_total;     /* divisions actually applied */
    int64_t starved_steps; /* steps that accepted fewer than n_s candidates */
    int64_t cand_last;     /* candidates drawn by the latest step */
    int64_t events_last;   /* divisions applied by the latest step */
    int64_t mass_fix;      /* active mass M in units of 2^-24 (exact sum of per-node rounds) */
    int64_t quiescent_fix; /* mass frozen behind the rear wall, same unit */
    int64_t S1, S2;        /* sum h(x), sum h(x)^2 over the columns */
    int64_t node_updates;  /* sum over steps of the nodes updated (active window) */
    int64_t launches;      /* kernels launched by lbm_step so far */
    double mass, quiescent_mass, carry, hbar, w, clip_mass;
    int32_t y_r;           /* rear wall: rows below y_r are quiescent */
    int32_t H_top;         /* max_x h(x) */
    int32_t hmin;          /* min_x h(x) */
    int32_t y_hi;          /* rows >= y_hi hold no mass (window top) */
    int32_t status;        /* LBM_STATUS_* bits */
    int32_t update_kernel; /* kernel used for the fused update: 1 plain loads, 2 TMA-staged */
} lbm_stats_t;

typedef struct lbm_sim lbm_sim;

/* Checks a parameter set without touching any GPU. LBM_OK or
 * LBM_ERR_INVALID_ARG. Limits: 1 <= W, 3 <= H, W, H <= 32768, W*H < 2^30,
 * tau > 1/2, rho_cell > 0, rho_c >= 0, growth_rate >= 0. */
int lbm_validate(const lbm_params_t *params);

/* Device bytes one simulation needs (for a caller-provided arena); host only. */
int lbm_footprint(const lbm_params_t *params, uint64_t *bytes);

/* Divisions per step the planner of such a simulation can hold: four times
 * the initial density's n_s over the whole lattice plus 1024, at most 2^24
 * (more sets LBM_STATUS_CAPACITY). The planner's grid grows with this value
 * and the lattice width (up to a quarter of the SMs); in a batch, members
 * get planner blocks by the work they did last step instead. Host only. */
int lbm_plan_capacity(const lbm_params_t *params, int64_t *ns_max);

/* Creates a simulation and initialises it on `stream` (a cudaStream_t, NULL =
 * legacy default stream): tissue below the initial front with u = 0 and
 * f = f^SS(rho, 0) (App. A, first paragraph), then the occupancy mask, front
 * heights and active mass. `arena` is an optional device buffer of at least
 * lbm_footprint() bytes, 256-byte aligned, owned by the caller and kept alive
 * until lbm_destroy; NULL makes the library allocate (and later free) its own.
 * On success *out holds the handle. Syncs. */
int lbm_create(const lbm_params_t *params, void *stream, void *arena, uint64_t arena_bytes,
               lbm_sim **out);

/* Advances `nsteps` time steps (App. A steps 1-7 each, plus the front
 * heights, Eq. 6 width, rear wall and active mass), all on the device with no
 * host synchronisation. Returns LBM_OK or a launch error; device-side status
 * (LBM_STATUS_*) is reported by lbm_stats. */
int lbm_step(lbm_sim *sim, int64_t nsteps);

/* Front heights h(x) = 1 + highest occupied row of column x (0 if none) into
 * the caller's host array of W int32, and the mean height and interface width
 * w of Eq. 6 (either pointer may be NULL). Syncs. */
int lbm_front_heights(lbm_sim *sim, int32_t *h_host, double *hbar, double *w);

/* The same without waiting: enqueues on the simulation's stream the copies of
 * h(x) into h_host (W int32; NULL skips it) and of the exact Eq. 6 sums
 * S1 = sum h, S2 = sum h^2 into sums_host[0..1]. Host buffers should be
 * pinned (cudaHostAlloc, cudaHostRegister) for the copies to be
 * asynchronous; pinned buffers that the device can address are written by
 * one small kernel, others by cudaMemcpyAsync. They hold the values once
 * the stream has reached this point (lbm_sync). Eq. 6 from the sums:
 * lbm_eq6 or lbm_eq6_n. Enqueues only. */
int lbm_front_heights_async(lbm_sim *sim, int32_t *h_host, int64_t *sums_host);

/* Eq. 6 from the exact sums: hbar = S1 / W, w = sqrt(W S2 - S1^2) / W (IEEE
 * double, as the kernels' FP64 wall rule). Host only. */
int lbm_eq6(int64_t s1, int64_t s2, int32_t width, double *hbar, double *w);

/* lbm_eq6 for n pairs (Sec. III, Eq. 6): sums holds n (S1, S2) pairs, the
 * layout lbm_front_heights_async writes (int64 [n][2]); hbar[i] and w[i]
 * receive pair i's values, bit for bit those of lbm_eq6. All arrays are the
 * caller's host memory. LBM_ERR_INVALID_ARG if width < 1, n < 0, or a
 * pointer is NULL while n > 0. Host only. */
int lbm_eq6_n(const int64_t *sums, int64_t n, int32_t width, double *hbar, double *w);

/* Density rho = sum_i f_i and velocity u = sum_i f_i e_i / rho (Eq. 1; u = 0
 * where rho = 0) of the current populations into caller host arrays of W*H
 * doubles, row-major [y][x]. Syncs. */
int lbm_fields(lbm_sim *sim, double *rho, double *ux, double *uy);

/* Same as lbm_fields into caller device arrays of W*H doubles. Enqueues only. */
int lbm_fields_device(lbm_sim *sim, double *rho, double *ux, double *uy);

/* Current populations into a caller host array of Q*H*W doubles, [q][y][x]
 * with the D2Q9 order 0:(0,0) 1:(1,0) 2:(0,1) 3:(-1,0) 4:(0,-1) 5:(1,1)
 * 6:(-1,1) 7:(-1,-1) 8:(1,-1) (Q = 9), or the D2Q7 order of lbm_params_t
 * (Q = 7). Syncs. */
int lbm_populations(lbm_sim *sim, double *f_host);

/* Replaces the populations with the caller's host array (layout as above,
 * rounded to the storage precision); recomputes the occupancy mask of the
 * active rows, the heights and the active mass; keeps the step count, the
 * rear wall and the carried site fraction. Every value must be finite and
 * non-negative (as after any step), else LBM_ERR_INVALID_ARG. Syncs. */
int lbm_set_populations(lbm_sim *sim, const double *f_host);

/* Occupancy mask (1 where rho >= rho_c after the latest step) into a caller
 * host array of H*W bytes, [y][x]. Syncs. */
int lbm_mask(lbm_sim *sim, uint8_t *mask_host);

/* Divisions applied by the latest step, sorted by (node, pair): node id
 * y*W + x, pair p in 0..3 loading directions (1,3), (2,4), (5,7), (6,8), and
 * the number of times the site was drawn. Writes at most `cap` entries and the
 * total count to *n. Syncs. */
int lbm_last_events(lbm_sim *sim, int64_t *node, int32_t *pair, int32_t *count, int64_t cap,
                    int64_t *n);

/* Counters and observables after the latest step. Syncs. */
int lbm_stats(lbm_sim *sim, lbm_stats_t *out);

/* Clears the sticky device status bits, and restarts the planner's grid-
 * barrier counter and division merge table (which hold nothing between steps;
 * after a step abandoned on LBM_STATUS_TIMEOUT they may be inconsistent).
 * Enqueues only. */
int lbm_clear_status(lbm_sim *sim);

/* Failure-detection test hook (no counterpart in the paper). Every wait in
 * the kernels is bounded: the TMA-staged update's waits for its bulk copies
 * and for its warps, and the cooperative planner's grid barriers give up after
 * a budget of clock cycles (default about two seconds at 2 GHz), raise
 * LBM_STATUS_TIMEOUT, stop waiting, let the copies already issued land and
 * return, so that the context stays usable. This call sets, for the steps
 * that follow on this handle, the budget (budget_cycles > 0; 0 restores the
 * default) and what is withheld so that a wait must run out:
 *  withhold bit 0  the TMA-staged update issues no bulk copies (each thread's
 *                  first wait for a staged tile runs out);
 *  withhold bit 1  the planner's grid barriers wait for one arrival more than
 *                  the grid makes (each block's first barrier runs out).
 * A step run with a bit set is abandoned: its populations, observables and
 * selection are meaningless. Recover with lbm_debug_waits(sim, 0, 0),
 * lbm_clear_status and lbm_set_populations. For tests only; not for a
 * simulation in a batch. Syncs. LBM_ERR_INVALID_ARG for a negative budget or
 * withhold outside 0..3. */
int lbm_debug_waits(lbm_sim *sim, int64_t budget_cycles, int32_t withhold);

/* Kernel timing for throughput measurement: while enabled, every launch of
 * the fused update kernel is bracketed by CUDA events on the simulation's
 * stream (at most `max_launches` of them). lbm_timing_read syncs and returns
 * the number of timed launches, their summed device time in milliseconds and
 * the nodes they updated. Enabling again resets the record. */
int lbm_timing_enable(lbm_sim *sim, int64_t max_launches);
int lbm_timing_read(lbm_sim *sim, int64_t *launches, double *total_ms, int64_t *nodes);
/* Times only one update launch in every `stride` (>= 1, else
 * LBM_ERR_INVALID_ARG) while timing is enabled: an event pair around a launch
 * keeps it from overlapping the preceding planner kernel, so sparse sampling
 * leaves the measured run close to an untimed one. `nodes` from
 * lbm_timing_read still counts every step since lbm_timing_enable. Default 1. */
int lbm_timing_stride(lbm_sim *sim, int64_t stride);

/* Bytes of population traffic one node update moves in the fused update
 * kernel (9 loads + 9 stores of the storage type). */
int lbm_bytes_per_node(lbm_sim *sim, int64_t *bytes);

/* Waits for the stream; returns LBM_OK or LBM_ERR_CUDA. */
int lbm_sync(lbm_sim *sim);

/* Frees the handle and (if the library allocated it) its device memory. */
void lbm_destroy(lbm_sim *sim);

/* Name of a return code; never NULL. */
const char *lbm_strerror(int code);

/* Text of the last CUDA error seen by any handle of this thread; never NULL. */
const char *lbm_last_cuda_error(void);

/* Library version string, e.g. "0.1.0 sm_103a". */
const char *lbm_version(void);

/* ---- batched stepping of independent simulations ----
 * The ensembles the roughness statistics of Sec. III need (many realisations
 * of Eq. 6's w(t)) are many small, independent lattices; stepped one after
 * another they leave most of the GPU idle. A batch advances its simulations
 * together by replaying a CUDA graph. When all members store their
 * populations in the same type on the same lattice, a step of the whole
 * batch is three launches: the injection of every member's divisions, the
 * update over every member's tiles, and the planners, one cooperative
 * launch whose blocks are dealt on the device every step by the members'
 * planner work (the candidates they drew last step, their widths): a heavy
 * member gets blocks in proportion, light ones share blocks, planned one
 * after another; otherwise the graph holds, for each simulation, a chain of steps
 * (update + planner) as an independent branch. Each simulation computes
 * exactly what lbm_step would (the same arithmetic and counters, bit for
 * bit).
 *  sims    n distinct handles on one device, created by lbm_create and not
 *          in kernel timing; the batch keeps the pointers, the caller keeps
 *          ownership and must destroy the batch (or detach the member)
 *          before destroying a member.
 *  stream  cudaStream_t the graphs are launched on (NULL = legacy default).
 * lbm_batch_step enqueues nsteps steps of every member, ordered after the work
 * already on each member's own stream and before the work enqueued there
 * afterwards; queries on a member (lbm_stats, lbm_front_heights, ...) then see
 * the result. Between lbm_batch_step calls the members may also be stepped on
 * their own. The graphs are captured in lbm_batch_create (LBM_ERR_CUDA if
 * capture fails); lbm_batch_create allocates streams, events, graphs and
 * the batched launches' tables in device memory. A batch of n members has n
 * slots. */
typedef struct lbm_batch lbm_batch;
int lbm_batch_create(lbm_sim *const *sims, int32_t n, void *stream, lbm_batch **out);
int lbm_batch_step(lbm_batch *batch, int64_t nsteps);
int lbm_batch_destroy(lbm_batch *batch);
/* 3 if the batch steps with the batched launches and its update is the
 * TMA-staged one with bulk tensor stores (FP32 members all multiples of 4
 * wide and at least as wide as the tuned table's threshold, 4096 columns
 * on GB300), 2 if the TMA-staged one with per-lane
 * stores (all members D2Q9 with FP32 or the same 16-bit storage and walls
 * in y, at most 256 slots: one launch deals all members' 128 x 2 tiles; the
 * divisions are added by the batched injection launch before it),
 * 1 if with the batched launches and the plain-load update (the members
 * share the storage type and the lattice), 0 if with one graph branch per
 * member; LBM_ERR_INVALID_ARG for NULL. */
int lbm_batch_fused(const lbm_batch *batch);

/* Members joining and leaving a batch that steps with the batched launches
 * (lbm_batch_fused >= 1), as a serving loop needs: the tables in device
 * memory have room for more entries than the members use (an unused entry
 * does nothing), so a change of members rewrites table entries and leaves
 * the captured graphs as they are. The graphs are captured again (inside the
 * call) only when a table outgrows its room (its room then doubles) or when
 * a joining member cannot take the batch's form of the update: a member
 * periodic in y ends the staged form, one narrower than the tuned
 * bulk-store width or not a multiple of 4 wide ends the bulk stores
 * (lbm_batch_fused reports the form in use). The staged form is captured
 * with and without Eq. 4's noise, and a step replays the one the current
 * members need.
 * lbm_batch_create_empty: a batch with `slots` empty slots (1..1024; the
 *     staged update for up to 256) for simulations of one lattice
 *     (LBM_D2Q9, LBM_D2Q7) and storage type (LBM_FP32 .. LBM_BF16; D2Q7:
 *     FP32 or FP64) on the current device; LBM_ERR_INVALID_ARG otherwise.
 * lbm_batch_attach: puts `sim` (same lattice, storage type and device, not
 *     in kernel timing, not yet a member) into the first free slot and
 *     writes that slot's index to *slot (may be NULL). LBM_ERR_INVALID_ARG
 *     for a mismatch or a branch-form batch, LBM_ERR_BATCH_FULL if no slot
 *     is free. The batch's next steps come after the work already on the
 *     member's stream. Waits for the batch's stream (the table copies).
 * lbm_batch_detach: empties `sim`'s slot; the member's stream then waits for
 *     the batch's steps already enqueued, so it may be queried, stepped
 *     alone or destroyed. LBM_ERR_INVALID_ARG if `sim` is not a member.
 *     Waits for the batch's stream.
 * lbm_batch_members: the number of members (>= 0), or LBM_ERR_INVALID_ARG.
 * lbm_batch_captures: how many times the batch's graphs have been captured
 *     (1 after creation), or LBM_ERR_INVALID_ARG.
 * Stepping a batch with no members enqueues nothing. */
int lbm_batch_create_empty(int32_t slots, int32_t lattice, int32_t precision, void *stream, lbm_batch **out);
int lbm_batch_attach(lbm_batch *batch, lbm_sim *sim, int32_t *slot);
int lbm_batch_detach(lbm_batch *batch, lbm_sim *sim);
int lbm_batch_members(const lbm_batch *batch);
int lbm_batch_captures(const lbm_batch *batch);

/* ---- allocation-free variant (the paper has no counterpart) ----
 * Front heights h(x) = 1 + highest set row of column x (0 if none) of a
 * caller's occupancy bitmask, plus the mean height and the interface width,
 * the same reduction lbm_step runs after every update, but without allocating
 * anything. For callers that cannot allocate device memory: an application
 * whose device memory is all held by another allocator (a framework's caching
 * pool), or a loop that must never stall on the allocator.
 *  mask_dev    device, read: H rows of (W + 31) / 32 uint32 words; bit (x & 31)
 *              of word (x >> 5) of row y is node (x, y).
 *  heights_dev device, written: W int32.
 *  stats_dev   device, written: two doubles, hbar = sum h / W and
 *              w = sqrt(W sum h^2 - (sum h)^2) / W.
 *  stream      cudaStream_t the work is enqueued on (NULL = legacy default).
 * Its scratch is a fixed device array inside this library, sized for widths up
 * to LBM_NOALLOC_MAX_WIDTH; larger widths (or heights above 32768) return
 * LBM_ERR_INVALID_ARG. Every GPU that loads the library keeps that array until
 * the process exits. The first call on each device looks up the array's device
 * address with that device current, so make it before capturing any stream on
 * that device. Host threads may make first calls concurrently (the lookup is
 * guarded). The address is kept for the life of the process: after a
 * cudaDeviceReset of that device it is stale, so do not use this function on
 * a device that was reset. All calls share the array: calls whose kernels
 * overlap on a GPU race and must be serialised (one stream, or events); each
 * call zeroes the array's completion counter on its stream before its kernel.
 * Enqueues only. */
#define LBM_NOALLOC_MAX_WIDTH 32768
int lbm_front_heights_noalloc(const uint32_t *mask_dev, int32_t width, int32_t height, int32_t *heights_dev,
                              double *stats_dev, void *stream);

#ifdef __cplusplus
}
#endif
#endif /* LBM_GB300_LBM_H */
