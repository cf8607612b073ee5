/*
 * c2f.h -- C ABI of the GB300 Cell2Fire fire-growth library (libc2f.so).
 *
 * The library runs Monte-Carlo replicas of the cell-based fire-growth model
 * of Pais et al., "Cell2Fire: A Cell Based Forest Fire Growth Model"
 * (arXiv:1905.09317) on one NVIDIA GB300 (sm_103a):
 *
 *   Sim(ForestData, FTypes, Ignitions, Weather, TMax, Options)   (Alg. 1)
 *     ForestData/FTypes  -> c2f_load_landscape   (Sec. 3.5 (i), (ii); Table 1)
 *     Weather            -> c2f_set_weather      (Sec. 3.5 (iv); Table 2)
 *     Ignitions, TMax, Options -> c2f_sim_params (Sec. 3.1 uncertainty (1),(2))
 *     Step 0..2          -> c2f_simulate / c2f_simulate_batch / c2f_submit
 *     Step 3 outputs     -> c2f_burn_prob, c2f_get_scars, c2f_get_counters
 *                           (Sec. 3.6: burn grids, burn-probability maps)
 *
 * Conventions (all entry points):
 *  - Every function returns int: C2F_OK (0) or a negative C2F_E* code; no
 *    function aborts the process.  c2f_last_error() describes the last error
 *    raised on a context (per context, per calling thread).
 *  - Host arrays passed in are copied; the caller keeps ownership.  Output
 *    arrays are caller-owned and written only on success (never partially).
 *  - Device memory is owned by the context and freed by c2f_release /
 *    c2f_destroy.  A context is used from one host thread at a time.
 *  - Grids are row-major, row 0 = north, cell id = row * cols + col.
 *  - Fuel codes (uint8, Table 1 style, 1 = C-1): 0 non-fuel, 1 C1, 2 C2,
 *    3 C3, 4 C4, 5 C5, 6 C6, 7 C7, 8 D1, 9 M1, 10 M2, 11 O1a, 12 O1b, 13 S1,
 *    14 S2, 15 S3.  Any other code is C2F_EINVAL.
 */
#ifndef C2F_H
#define C2F_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define C2F_API __attribute__((visibility("default")))

enum {
  C2F_OK = 0,
  C2F_EINVAL = -1,    /* bad argument: sizes, codes, parameters, ids          */
  C2F_ENOMEM = -2,    /* device allocation failed or admission refused       */
  C2F_ECUDA = -3,     /* a CUDA call failed (message in c2f_last_error)      */
  C2F_ETIMEOUT = -4,  /* a bounded wait ran out                               */
  C2F_ENOTFOUND = -5, /* unknown landscape or simulation id                   */
  C2F_EBUSY = -6,     /* the simulation has not finished yet                  */
  C2F_ECANCELED = -7  /* the simulation was cancelled                         */
};

/* output selection bits of c2f_sim_params.outputs */
enum {
  C2F_OUT_SCARS = 1u,     /* keep per-replica burn grids (always kept)          */
  C2F_OUT_IGN_STEPS = 2u, /* keep per-replica ignition steps (int32 per cell)   */
  C2F_OUT_COUNTERS = 8u   /* keep per-replica counters (always kept)            */
};

typedef struct c2f_ctx c2f_ctx;

/* One hour of the weather stream (Sec. 3.5 (iv), Table 2): wind speed
 * (km/h), wind direction the wind blows FROM (degrees clockwise from north),
 * Fine Fuel Moisture Code and Buildup Index of the FWI System. */
typedef struct {
  double ws_kmh;
  double wd_from_deg;
  double ffmc;
  double bui;
} c2f_weather_hour;

/* Simulation options (Alg. 1 "Options"; Sec. 3.1 sources of uncertainty). */
typedef struct {
  uint64_t seed;            /* key of the counter-based Philox4x32-10 draws            */
  int32_t n_replicas;       /* Monte-Carlo replicas, >= 1                               */
  int32_t hours;            /* TMax in weather hours, 1 .. n_hours of the weather       */
  int32_t minutes_per_step; /* fire-period length; must divide 60 (Sec. 3.1: 1 min)     */
  int32_t ignition_mode;    /* 0: fixed ignition_cell; 1: uniform over burnable cells   */
  int32_t ignition_cell;    /* cell id for mode 0; must be burnable                     */
  double ros_sigma;         /* lognormal sigma of the ROS perturbation, 0 .. 1          */
  double ros_threshold;     /* receiver ignites iff ROS * f > threshold (Sec. 3.1)      */
  double burnout_delta;     /* > 0: Burned when ROS * f < delta (A5 (i)); 0 = off       */
  int32_t ellipse_mode;     /* 0: Eq. (1); 1: centre-offset ellipse ray (Sec. 3.7 fig.) */
  double o1_curing_pct;     /* grass curing percent for O1a/O1b (default 60)            */
  double m1_pc;             /* percent conifer for M1/M2 (default 50)                   */
  double const_ros;         /* > 0: every burnable cell spreads at this rate (m/min) on
                               all 8 axes instead of FBP (deterministic test hook)      */
  uint32_t outputs;         /* C2F_OUT_* bits                                           */
  int32_t burn_hours_min;   /* burning hours per day (A5, general fire dynamics (1)):   */
  int32_t burn_hours_max;   /* each replica burns only in weather hours h with h mod 24
                               < B, B drawn uniformly from {min..max} by one Philox4x32-10
                               block at counter (replica, 0, 0, 3), B = min + (x0 (max -
                               min + 1)) >> 32 (min = max: a constant); in the other
                               hours the fire is dormant (no spread, ignition, burn-out
                               or work; progress kept).  0, 0 = no limit; otherwise
                               1 <= min <= max <= 24                                    */
  double const_bros;        /* with const_ros > 0 (test hook): BROS in m/min (0 = const_ros)
                               and the length-to-breadth ratio LB (<= 1: 1); when
                               const_bros > 0 or const_lb > 1 every burnable cell gets the
                               ellipse of Sec. 3.7 (Eqs. 2-4) of HROS = const_ros, BROS and
                               LB, its head along the hour's wind (toward WD + 180), and the
                               8 axis rates of Eq. (1) (or of the ellipse_mode 1 ray);
                               ignored when const_ros is 0.  0 <= const_bros < 1e9,
                               0 <= const_lb <= 1000                                      */
  double const_lb;
} c2f_sim_params;

/* Fills *p with the defaults: seed 0, 1 replica, 1 hour, 1-minute steps,
 * fixed ignition at cell 0, sigma 0, threshold 0, delta 0, Eq. (1),
 * curing 60, PC 50, no constant ROS, scars + counters, no burning-hours limit. */
C2F_API void c2f_default_params(c2f_sim_params *p);

/* Creates a context on CUDA device `device`.  The context owns a stream,
 * all device buffers and the per-device constant tables.
 * Errors: C2F_EINVAL (no such device), C2F_ECUDA. */
C2F_API int c2f_create(c2f_ctx **out, int device);

/* Device-memory hooks.  With hooks, every device buffer of the context comes
 * from alloc(bytes, stream, user) and goes back through free(ptr, bytes,
 * stream, user) instead of cudaMallocAsync / cudaFreeAsync, with the same
 * stream-ordered meaning: the block is used by work on `stream` (and by other
 * streams only between host synchronisations), and a block freed on a stream
 * may be handed out again for work queued later on that stream.  alloc
 * returns NULL when it cannot allocate (the call then fails with
 * C2F_ENOMEM).  A host framework's caching allocator (e.g. PyTorch's) can
 * own the library's memory this way.  The hooks must stay valid until
 * c2f_destroy returns. */
typedef struct {
  void *(*alloc)(size_t bytes, void *stream, void *user);
  void (*free)(void *ptr, size_t bytes, void *stream, void *user);
  void *user;
} c2f_alloc_hooks;

/* c2f_create with allocation hooks (NULL hooks = cudaMallocAsync). */
C2F_API int c2f_create_with_hooks(c2f_ctx **out, int device, const c2f_alloc_hooks *hooks);

/* Makes the context issue its work on `stream` (a cudaStream_t of the same
 * device, e.g. a PyTorch stream); NULL restores the context's own stream. */
C2F_API int c2f_set_stream(c2f_ctx *ctx, void *stream);

/* Frees everything the context owns.  NULL is accepted. */
C2F_API void c2f_destroy(c2f_ctx *ctx);

/* Text of the last error the calling thread got from the library (empty
 * string if none); valid until that thread's next library call. */
C2F_API const char *c2f_last_error(const c2f_ctx *ctx);

/* Loads a landscape (Sec. 3.3 cell fields; Sec. 3.5 (i)): `fuel` codes
 * (rows*cols), `slope_pct` (percent rise over run, NULL = flat),
 * `aspect_deg` (downslope-facing azimuth clockwise from north, NULL = 0)
 * and `unburnable` (NULL or 1 = Harvested / not available, Sec. 3.1).
 * 1 <= rows, cols <= 65535; cell_size_m > 0; slopes finite >= 0.
 * Copies the arrays to the device.  Returns the id in *landscape_id. */
C2F_API int c2f_load_landscape(c2f_ctx *ctx, int32_t rows, int32_t cols, double cell_size_m,
                               const uint8_t *fuel, const float *slope_pct,
                               const float *aspect_deg, const uint8_t *unburnable,
                               int32_t *landscape_id);

/* Sets the hourly weather stream of a landscape (n_hours rows, copied).
 * FFMC must lie in [0, 101), BUI > 0, wind speed >= 0, all finite.
 * Invalidates the cached rate-of-spread tables of the landscape. */
C2F_API int c2f_set_weather(c2f_ctx *ctx, int32_t landscape_id, int32_t n_hours,
                            const c2f_weather_hour *w);

/* Weather scenarios (Sec. 3.1, uncertainty source (3)): n_scenarios hourly
 * streams of n_hours rows each, w[s*n_hours + h] (row-major, copied), scenario
 * s occurring with probability prob[s] / (prob[0] + ... + prob[S-1]).  Every
 * replica of a later simulation on the landscape runs under one scenario,
 * drawn from its own Philox4x32-10 block at counter (replica, 0, 0, 2): with
 * x0 the block's first word it takes the first s with x0 < T_s, where
 * T_s = floor(2^32 (prob[0] + ... + prob[s]) / total) (binary64 sums from the
 * left) and T_{S-1} = 2^32; a scenario of probability 0 is never drawn.  The
 * ignition draw and the perturbations stay keyed by the replica alone, so a
 * replica's fire under scenario s is the one a single-stream run with that
 * stream gives.  The table holds one stacked table per scenario (device
 * memory x n_scenarios).  1 <= n_scenarios <= 4096, n_scenarios * n_hours
 * <= 65535; prob: finite, >= 0, not all 0 (NULL allowed when n_scenarios is
 * 1); weather rows as c2f_set_weather.  c2f_set_weather is the same call
 * with one scenario.  Invalidates the cached tables of the landscape. */
C2F_API int c2f_set_weather_scenarios(c2f_ctx *ctx, int32_t landscape_id, int32_t n_scenarios,
                                      int32_t n_hours, const c2f_weather_hour *w,
                                      const double *prob);

/* The rate-of-spread table of a landscape for the FBP/ellipse options in *p
 * (Sec. 3.7, Eqs. 1-4): per (hour, cell) the 8 directional ROS in 2^32 fixed
 * point per fire period, and HROS.  A table is either eager (every row
 * written up front by the table kernel) or lazy (rows written by the
 * simulations that read them, 32 cells at a time, the first time a burning
 * cell needs them); both hold the same bits wherever a simulation reads.
 *   force 0: make sure an eager table exists (a lazy one is completed);
 *   force 1: discard the table and build a new eager one;
 *   force 2: discard the table; the next simulation fills a new lazy one.
 * c2f_simulate creates a table when none fits (eager by default, see
 * c2f_set_table_mode).  Asynchronous on the context stream; force outside
 * [0, 2] gives C2F_EINVAL. */
C2F_API int c2f_build_ros(c2f_ctx *ctx, int32_t landscape_id, const c2f_sim_params *p,
                          int force);

/* Whether tables that simulations create are eager (nonzero, the default)
 * or lazy (0).  Results are identical either way.  Lazy tables pay for the
 * rows inside the frontier kernel, at a lower FP64 rate than the table
 * kernel; they win only when the replicas touch a small part of the
 * landscape-hours (few replicas on a large landscape). */
C2F_API int c2f_set_table_mode(c2f_ctx *ctx, int eager);

/* Exports one hour of the rate-of-spread table for checking: ros8
 * (rows*cols*8 doubles, m/min, axis k = 45k degrees counter-clockwise from
 * east), hros (rows*cols), base (rows*cols*8 int64: the per-period fixed-point
 * increment before the perturbation).  Any output may be NULL. Synchronous. */
C2F_API int c2f_get_ros(c2f_ctx *ctx, int32_t landscape_id, const c2f_sim_params *p,
                        int32_t hour, double *ros8, double *hros, int64_t *base);

/* c2f_get_ros for weather scenario `scenario` of c2f_set_weather_scenarios
 * (c2f_get_ros is scenario 0); scenario outside [0, n_scenarios) is
 * C2F_EINVAL. */
C2F_API int c2f_get_ros_scenario(c2f_ctx *ctx, int32_t landscape_id, const c2f_sim_params *p,
                                 int32_t scenario, int32_t hour, double *ros8, double *hros,
                                 int64_t *base);

/* Runs all replicas of one simulation (Alg. 1 Steps 0-2 per replica) and
 * returns when they are finished.  The result stays on the device under
 * *sim_id until c2f_release.  Errors: C2F_EINVAL, C2F_ENOMEM, C2F_ECUDA. */
C2F_API int c2f_simulate(c2f_ctx *ctx, int32_t landscape_id, const c2f_sim_params *p,
                         int32_t *sim_id);

/* Runs n simulations (possibly of different landscapes and replica counts)
 * as one batch: one work list, one persistent kernel launch.  Results are
 * identical to n separate c2f_simulate calls.  sim_ids has n entries. */
C2F_API int c2f_simulate_batch(c2f_ctx *ctx, int32_t n, const int32_t *landscape_ids,
                               const c2f_sim_params *params, int32_t *sim_ids);

/* ---------------------------------------------------------------------------
 * Serving: asynchronous simulations with continuous batching.  c2f_submit
 * validates and queues a simulation (building its landscape's rate-of-spread
 * table first if needed) and returns at once.  Queued simulations are
 * launched together as one "epoch" of the frontier kernel when fewer than
 * max_inflight epochs are running and free device memory covers the epoch
 * plus a reserve; epochs run concurrently on their own streams, so requests
 * that arrive while others are on the GPU join the next epoch and overlap on
 * the device.  Results are the same as c2f_simulate's, alone or in any mix.
 * Every serving call (and c2f_pump) finishes epochs that are done and
 * launches queued work.  Free memory for admission is the device's free
 * memory plus what the context's pool keeps unused.  c2f_poll sets *done;
 * c2f_wait blocks until the simulation is finished, holding the context (other
 * threads' calls on it wait too); c2f_cancel drops a queued simulation (a running
 * one finishes, and its result is discarded: later reads give
 * C2F_ECANCELED).  Reading a simulation that is not finished gives C2F_EBUSY.
 * ------------------------------------------------------------------------- */
C2F_API int c2f_submit(c2f_ctx *ctx, int32_t landscape_id, const c2f_sim_params *p, int32_t *sim_id);
C2F_API int c2f_pump(c2f_ctx *ctx);
C2F_API int c2f_poll(c2f_ctx *ctx, int32_t sim_id, int32_t *done);
C2F_API int c2f_wait(c2f_ctx *ctx, int32_t sim_id);
C2F_API int c2f_cancel(c2f_ctx *ctx, int32_t sim_id);

/* Serving limits: concurrent epochs (1..16, default 3), replicas per epoch
 * (default 65536) and device bytes kept free when admitting an epoch
 * (default 2 GiB; an epoch is still admitted when nothing else runs). */
C2F_API int c2f_set_serving(c2f_ctx *ctx, int32_t max_inflight, int64_t max_epoch_replicas,
                            int64_t hbm_reserve_bytes);

/* Serving statistics since the context was created: epochs launched,
 * admission waits (times queued work was held back because free device
 * memory did not cover the epoch plus the reserve while other epochs ran),
 * and the simulations queued and epochs running now.  Any pointer may be
 * NULL.  Does not pump. */
C2F_API int c2f_serving_stats(c2f_ctx *ctx, int64_t *epochs, int64_t *admission_waits, int32_t *queued,
                              int32_t *running);

/* Burn-probability counts (Sec. 3.6 (i), Sec. 3.1 outputs): counts[c] = number
 * of replicas in which cell c ignited, uint32, rows*cols entries, host memory. */
C2F_API int c2f_burn_prob(c2f_ctx *ctx, int32_t sim_id, uint32_t *counts);

/* Burn-probability counts of one weather scenario (Sec. 3.1 (3)): counts[c] =
 * number of the replicas that drew `scenario` in which cell c ignited
 * (rows*cols uint32, host memory).  A landscape with one weather stream has
 * scenario 0 only; scenario outside [0, n_scenarios) is C2F_EINVAL. */
C2F_API int c2f_burn_prob_scenario(c2f_ctx *ctx, int32_t sim_id, int32_t scenario, uint32_t *counts);

/* Same into device memory (`counts_dev`, rows*cols uint32 on the context's
 * device); asynchronous on the context stream. */
C2F_API int c2f_burn_prob_device(c2f_ctx *ctx, int32_t sim_id, uint32_t *counts_dev);

/* Per-replica burn grids (Sec. 3.6 (i)): scars[r*N + c] = 1 if cell c ignited
 * in replica r (n_replicas*N bytes), and, if the simulation kept them,
 * ignition steps ign_step[r*N + c] (-1 = never).  Either pointer may be NULL. */
C2F_API int c2f_get_scars(c2f_ctx *ctx, int32_t sim_id, uint8_t *scars, int32_t *ign_step);

/* One replica's burn grid (N bytes, 1 = ignited) and, if kept, its ignition
 * steps (N int32, -1 = never; NULL to skip).  replica outside [0, n_replicas)
 * is C2F_EINVAL. */
C2F_API int c2f_get_replica_scar(c2f_ctx *ctx, int32_t sim_id, int32_t replica, uint8_t *scar,
                                 int32_t *ign_step);

/* The same burn grids bit-packed, as kept on the device: for replica r, row y
 * and word x (x < wpr = ceil(cols/32)), words[(r*rows + y)*wpr + x] holds
 * cells (y, 32x .. 32x+31), bit b = column 32x+b; padding bits are 0
 * (n_replicas*rows*wpr uint32 words, host memory). */
C2F_API int c2f_get_scar_bits(c2f_ctx *ctx, int32_t sim_id, uint32_t *words);

/* Fire-scar evolution (Sec. 3.6 (ii)): scars[r*N + c] = 1 if cell c ignited in
 * replica r by the end of weather hour `hour` (0-based; fire periods up to
 * (hour+1)*60/minutes_per_step).  Needs the ignition steps
 * (C2F_OUT_IGN_STEPS), else C2F_EINVAL; hour outside [0, hours) is
 * C2F_EINVAL. */
C2F_API int c2f_get_scars_at_hour(c2f_ctx *ctx, int32_t sim_id, int32_t hour, uint8_t *scars);

/* Per-replica counters: work[r] = sum over fire periods of the number of
 * burning cells (cell-updates), ignited[r] = cells ever ignited, ign_cell[r]
 * = ignition cell.  Any pointer may be NULL. */
C2F_API int c2f_get_counters(c2f_ctx *ctx, int32_t sim_id, int64_t *work, int32_t *ignited,
                             int32_t *ign_cell);

/* The weather scenario each replica ran under (n_replicas int32, host
 * memory; all 0 when the landscape had one weather stream). */
C2F_API int c2f_get_scenarios(c2f_ctx *ctx, int32_t sim_id, int32_t *scenario);

/* Fire-scar comparison of Sec. 4.1 between two finished simulations X and Y
 * of the same grid shape and replica count, replica r of X against replica r
 * of Y.  With X^t, Y^t the 0-1 scars at the end of weather hour t (cells
 * ignited at a step <= (t+1)*60/minutes_per_step) and N = rows*cols:
 *   mse[r*H + t]  = (1/N) sum |X^t - Y^t|^2;
 *   ssim[r*H + t] = (2 mu_X mu_Y + C1)(2 sigma_XY + C2) /
 *                   ((mu_X^2 + mu_Y^2 + C1)(sigma_X^2 + sigma_Y^2 + C2)),
 *                   Wang et al.'s structural similarity over the whole grid:
 *                   means, 1/(N-1) variances and covariance, C1 = 0.01^2,
 *                   C2 = 0.03^2 (the paper prints the second denominator
 *                   factor as mu_X^2 + mu_Y^2 + C2; read as Wang et al.'s);
 *   dnorm[r]      = ||X - Y|| (Frobenius) of the final scars.
 * H = hours of the simulations.  mse / ssim (n_replicas*H doubles) need both
 * simulations to have kept ignition steps (C2F_OUT_IGN_STEPS) with equal
 * hours (<= 8192) and minutes_per_step, and N >= 2; dnorm (n_replicas
 * doubles) works from the scars alone.  Any output may be NULL.  Host memory,
 * synchronous.  Errors: C2F_ENOTFOUND, C2F_EBUSY, C2F_EINVAL (shapes or
 * counts differ, steps missing). */
C2F_API int c2f_compare_scars(c2f_ctx *ctx, int32_t sim_x, int32_t sim_y, double *mse, double *ssim,
                              double *dnorm);

/* The same into device memory of the context's device; asynchronous on the
 * context stream. */
C2F_API int c2f_compare_scars_device(c2f_ctx *ctx, int32_t sim_x, int32_t sim_y, double *mse_dev,
                                     double *ssim_dev, double *dnorm_dev);

/* Initial burning-list capacity (entries per CTA) of the frontier kernel;
 * 0 = automatic.  A replica that outgrows it is re-run with a larger one, so
 * results never depend on this value (a tuning and test knob). */
C2F_API int c2f_set_list_capacity(c2f_ctx *ctx, int64_t cap);

/* Bounded waits inside the frontier kernel: a warp that needs a lazy-table
 * chunk which another warp of the launch is computing polls for it (about
 * 130 ns a poll) and gives up after `polls` polls (0 = the default, 2^23,
 * about a second); the simulation then fails with C2F_ETIMEOUT and the
 * context stays usable.  polls outside [0, 2^32) is C2F_EINVAL. */
C2F_API int c2f_set_wait_limit(c2f_ctx *ctx, int64_t polls);

/* Test hook for the bounded wait above; the paper has no counterpart.  Marks
 * the chunk (32 cells of one row of the bit-plane layout) holding `cell` at
 * weather hour `hour` of `scenario` in the landscape's lazy table as being
 * computed by a warp that will never finish, so that a simulation that needs
 * it waits until the wait limit and fails with C2F_ETIMEOUT.  The table is
 * unusable afterwards: rebuild it (c2f_build_ros with force 1 or 2).
 * C2F_EINVAL when the landscape has no lazy table or an index is out of
 * range.  Synchronous. */
C2F_API int c2f_test_hold_chunk(c2f_ctx *ctx, int32_t landscape_id, int32_t scenario, int32_t hour,
                                int32_t cell);

/* Frontier-kernel launch shape: CTA size `threads` (32, 64 or 128; each warp
 * simulates one replica) and whether a window of each replica's bit planes
 * and its burning list are staged in shared memory (`smem` != 0, the default)
 * or kept in global memory (0).  With shared memory, smem = 1 sizes each
 * warp's share so that the launch's own replicas are resident at once (up to
 * 8 warps per SM); smem = N in [2, 16] sizes it for N warps per SM, leaving
 * room for frontier launches that run at the same time (serving epochs,
 * pipelined steps).  Results do not depend on any of this; they are tuning
 * knobs.  smem outside [0, 16] is C2F_EINVAL. */
C2F_API int c2f_set_frontier_config(c2f_ctx *ctx, int threads, int64_t smem);

/* Compaction trigger of the frontier's burning lists: within a weather hour
 * a list is compacted (Burned cells and cells with no open axis dropped) once
 * it holds more than eighths/8 of its capacity (2..7, default 6).  Results do
 * not depend on it (a tuning knob); outside [2, 7] is C2F_EINVAL. */
C2F_API int c2f_set_compaction(c2f_ctx *ctx, int32_t eighths);

/* Autotuner result: the frontier settings it kept on the context. */
typedef struct {
  int32_t threads;          /* CTA size: 32, 64 or 128 (one replica per warp)                */
  int32_t smem_lists;       /* 1: plane windows and lists in shared memory; 0: global memory */
  int32_t warps_per_sm;     /* shared-memory sizing target (0: the launch's own replicas)    */
  int32_t compact_eighths;  /* compaction trigger, eighths of the list capacity              */
  int64_t list_capacity;    /* initial burning-list capacity (0: automatic)                  */
  double frontier_ms;       /* the winner's frontier time on the sample                      */
  int32_t candidates;       /* settings timed                                                */
} c2f_tuning;

/* Launch-shape autotuner for a batch: runs the same mix of simulations,
 * scaled down to about `sample_replicas` replicas, under candidate frontier
 * settings and keeps the fastest on the context.  Coordinate descent, each
 * stage keeping its best for the next: (1) warps per CTA x shared / global
 * lists; (2) the shared-memory sizing (warps per SM: the launch's own, 4, 6,
 * 8, 11) when lists are in shared memory; (3) the compaction trigger (4, 6,
 * 7 eighths of capacity); (4) the initial list capacity (automatic, 2x, 4x)
 * when lists are in global memory.  Candidates are timed by the frontier's
 * kernel events; in stages 2-4 a candidate replaces the incumbent only when
 * it is at least 3 % faster (smaller differences are timing noise, and
 * repeated tunings of one mix then agree).  Results of later runs are the same under any setting; only
 * their speed changes.  `out` may be NULL. */
C2F_API int c2f_autotune_full(c2f_ctx *ctx, int32_t n, const int32_t *landscape_ids,
                              const c2f_sim_params *params, int32_t sample_replicas, c2f_tuning *out);

/* c2f_autotune_full reporting the CTA size, the shared-memory setting (0:
 * global lists; 1: shared, sized for the launch; N >= 2: shared, sized for N
 * warps per SM, as c2f_set_frontier_config takes it) and the frontier time.
 * Outputs may be NULL. */
C2F_API int c2f_autotune(c2f_ctx *ctx, int32_t n, const int32_t *landscape_ids,
                         const c2f_sim_params *params, int32_t sample_replicas, int32_t *best_threads,
                         int32_t *best_smem, double *best_ms);

/* Profiling switches, flags of c2f_profile's `enable` (0 turns both off; other
 * bits give C2F_EINVAL).  C2F_PROFILE_KERNELS: kernel timing as below.
 * C2F_PROFILE_REPLICAS: per-replica frontier counters (c2f_get_replica_profile),
 * recorded by a profiling build of the frontier kernel (one-warp CTAs, the
 * counter code compiled in: a few clock reads and shared-memory adds per
 * visited period), so a timing run should leave them off.  Either switch makes
 * c2f_simulate_batch launch its groups directly instead of through a graph. */
#define C2F_PROFILE_KERNELS 1
#define C2F_PROFILE_REPLICAS 2

/* Kernel timing: with C2F_PROFILE_KERNELS on, the context brackets each launch of its
 * kernel families with CUDA events on its stream.  c2f_kernel_times waits for
 * the stream, writes per family the summed milliseconds and the launch count
 * since the last call, and resets them.  Families (index): 0 ROS table (K1,
 * with its hour prep), 1 ignition (K2), 2 frontier (K3), 3 burn probability
 * (K4).  ms and launches hold C2F_KT_FAMILIES entries. */
#define C2F_KT_FAMILIES 4
C2F_API int c2f_profile(c2f_ctx *ctx, int enable);
C2F_API int c2f_kernel_times(c2f_ctx *ctx, double *ms, int64_t *launches);

/* Launch trace: how the table builds (K1) and the frontier's replicas (K3)
 * share the device over time, e.g. when steps are pipelined.  With tracing on,
 * every K1 CTA and every frontier replica that runs appends one record of
 * four uint64 to records_dev (device memory of the context's device, owned by
 * the caller, at least 32*capacity bytes):
 *   [0] kind | SM id << 8 | aux << 32, kind C2F_TRACE_TABLE (aux = weather
 *       hour of the CTA, which is timed by its first thread) or
 *       C2F_TRACE_REPLICA (aux = replica index; a replica re-run after a list
 *       overflow appends again);
 *   [1] tag: the table's build number / the simulation's creation number,
 *       both counted from 1 per context;
 *   [2], [3] start and end, nanoseconds of the GPU's global timer.
 * Records go in no particular order; once `capacity` are written the rest are
 * counted but dropped.  c2f_trace waits for the context stream and resets the
 * count; NULL with capacity 0 turns tracing off (launches already issued keep
 * their setting).  c2f_trace_count gives the records claimed since, written or
 * not; call it after the traced work has finished.  Other arguments:
 * C2F_EINVAL.  The allocation-free entry point does not trace. */
#define C2F_TRACE_TABLE 1
#define C2F_TRACE_REPLICA 2
C2F_API int c2f_trace(c2f_ctx *ctx, uint64_t *records_dev, int64_t capacity);
C2F_API int c2f_trace_count(c2f_ctx *ctx, int64_t *count);

/* Per-replica frontier profile of a simulation run while C2F_PROFILE_REPLICAS
 * was on (c2f_profile): counters[r*16 + i] for replica r (SM clock cycles, counts),
 * i = 0 cycles of the replica's whole frontier run (its last attempt),
 * 1 cycles at hour boundaries, 2 cycles finding and sending crossings and
 * receiving (A), 3 cycles setting up newly ignited cells (C), 4 fire periods
 * visited, 5 burning cells with a crossing processed, 6 cells ignited,
 * 7 longest burning list, 8 cycles of (A) spent walking the visited period's
 * calendar list, 9 list compactions within an hour, 10 rounds of crossing
 * cells (up to 32 each), 11 new-cell set-up iterations (up to 4 cells each),
 * 12-15 zero.  Host memory, n_replicas*16 int64.  C2F_EINVAL if the
 * simulation ran without per-replica counters. */
C2F_API int c2f_get_replica_profile(c2f_ctx *ctx, int32_t sim_id, int64_t *counters);

/* ---------------------------------------------------------------------------
 * Allocation-free frontier step.  The paper has no counterpart: this entry
 * point exists for callers that cannot allocate device memory (a host
 * application that has handed all device memory to its own allocator and
 * forbids others to take more, a plugin forbidden to allocate after
 * start-up).  It runs Step 2 of Alg. 1 for every replica -- the same kernel
 * and the same results as c2f_simulate -- taking all scratch from one fixed
 * 16 MiB device array inside the library (every GPU that loads the library
 * holds it until exit).  It calls no cudaMalloc, cudaFree or allocating
 * library routine.
 *
 * Inputs (device memory, caller-owned, not modified): the burnable bit plane
 * (rows * ceil(cols/32) 32-bit words, rows padded to whole words, bit = fuel
 * and not harvested), the rate-of-spread table `base` ([hours][rows*cols][8]
 * int64, the per-period fixed-point increments that c2f_get_ros exports for
 * the same minutes_per_step) and `hros` ([hours][rows*cols]), and the
 * ignition cell of every replica: each must be a cell id in [0, rows*cols)
 * whose burnable bit is set, else the call gives C2F_EINVAL (the kernel
 * checks it and touches nothing for that replica).  Outputs (device memory,
 * caller-owned): scars ([n_replicas][rows * ceil(cols/32)] words, same layout
 * as the plane), work and n_ignited per replica.  From *p it uses seed,
 * n_replicas (at most 65536), hours, minutes_per_step, ros_sigma,
 * ros_threshold, burnout_delta, burn_hours_min and burn_hours_max, with the
 * meaning and the checks of c2f_simulate.
 *
 * Limits: the two bit planes of one replica (rows * ceil(cols/32) * 8 bytes)
 * plus 256 burning-list entries of 80 bytes and a header of about 12 bytes
 * per replica must fit the 16 MiB array: about 67 million cells (a square
 * grid of up to 8,180 x 8,180 cells with one replica); larger landscapes give
 * C2F_EINVAL before any device work.  A replica whose burning list outgrows
 * the whole array gives C2F_ENOMEM.  Each call clears what must start at
 * zero; all calls share the array and it keeps the last call's contents, so
 * calls that overlap on the GPU (other streams, other host threads) race.
 * The first call on a device looks up the array's device address and loads
 * the library's constant tables (once per device, with that device current).
 * Synchronous: the call waits for `stream`, reads the replicas' statuses on
 * the host and re-runs replicas whose burning lists overflowed, so it must
 * not be made on a stream that is being captured into a CUDA graph.
 * ------------------------------------------------------------------------- */
typedef struct {
  int32_t rows, cols;
  double cell_size_m;
  const uint32_t *burnable;
  const int64_t *base;
  const double *hros;
  const int32_t *ign_cell;
  uint32_t *scars;
  int64_t *work;
  int32_t *n_ignited;
} c2f_frontier_io;

C2F_API int c2f_frontier_static(const c2f_frontier_io *io, const c2f_sim_params *p, void *stream);

/* Calibration: the device's FP64 fused multiply-add rate (GFLOP/s, 2 flops per
 * FMA), measured with CUDA events on the context stream by a kernel of eight
 * independent FMA chains per thread over 8 CTAs of 256 threads per SM (best of
 * three timed launches, about 0.1 s in all).  The roofline peak of the table
 * kernel, which is FP64-bound.  Synchronous. */
C2F_API int c2f_fp64_peak(c2f_ctx *ctx, double *gflops);

/* Frees a landscape (and its tables) or a simulation result.  A simulation
 * may be released right after an asynchronous read of it (c2f_burn_prob_device,
 * c2f_compare_scars_device): its device memory is returned only after those
 * reads, in the order of the streams they were issued on.  A running
 * simulation is cancelled (its epoch keeps it until the epoch ends). */
C2F_API int c2f_release(c2f_ctx *ctx, int32_t id);

#ifdef __cplusplus
}
#endif

#endif /* C2F_H */
