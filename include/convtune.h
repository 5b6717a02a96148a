/*
 * convtune — auto-tuned direct single-channel 2D correlation for GB300 (sm_103a).
 *
 * The library implements the tunable 2D convolution kernel and the empirical
 * tuning loop studied in "Bringing Auto-tuning to HIP: Analysis of Tuning
 * Impact and Difficulty on AMD and Nvidia GPUs" (Lurati et al., 2024):
 *   - the kernel and its tunable parameters: Sec. 5 "Benchmark kernels",
 *     Table 1 (block_size_x/y, tile_size_x/y, use_shmem) and the loop-unrolling
 *     parameter of Sec. 3;
 *   - compile-and-benchmark of every configuration, timed by events recorded
 *     before and after the kernel: Sec. 3;
 *   - search strategies over the space: Sec. 3 ("optimization algorithms");
 *   - analysis of a full timing table (tuning impact = optimum / median,
 *     Sec. 4; proportion of centrality, Eq. 1; portability, Eqs. 2-3).
 *
 * Operation (the paper gives no formula; the library computes a "valid"
 * cross-correlation, no filter flip, no padding):
 *     out[y][x] = sum_{i<filter_h} sum_{j<filter_w} in[y+i][x+j] * f[i][j]
 *     0 <= y < out_h, 0 <= x < out_w;  in is (out_h+filter_h-1) rows by
 *     (out_w+filter_w-1) columns.
 * Arithmetic: FP32 fused multiply-add per tap, taps added in (i, j) order,
 * identical for every configuration.  BF16 problems store image and filter in
 * BF16 and widen them exactly to FP32; the output is FP32.
 *
 * Conventions for every call:
 *   - No call aborts or exits.  Each returns a ct_status; ct_last_error()
 *     returns a thread-local message for the last failing call of the thread.
 *   - Device pointers ("d_") are CUDA device (or managed) memory owned by the
 *     caller; host pointers ("h_") are ordinary host memory owned by the caller
 *     and are not retained after the call returns.
 *   - Layout: images are row-major with a row pitch in ELEMENTS; every row
 *     must start on a 16-byte boundary (pitch * element size a multiple of 16,
 *     base pointer 16-byte aligned).  The image buffer must hold in_h full
 *     rows of in_pitch elements; the output buffer out_h rows of out_pitch.
 *     Elements between the valid width and the pitch are never used for a
 *     stored output (they may hold anything, including NaN).
 *   - Streams are CUDA runtime streams (cudaStream_t) passed as void*; NULL is
 *     the legacy default stream.
 */
#ifndef CONVTUNE_H
#define CONVTUNE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CT_API __attribute__((visibility("default")))
#else
#define CT_API
#endif

typedef enum {
    CT_OK = 0,
    CT_ERR_INVALID_ARG = -1,    /* null pointer, bad size, pitch or alignment */
    CT_ERR_INVALID_CONFIG = -2, /* config outside the launchable set (threads, smem, tiles) */
    CT_ERR_COMPILE = -3,        /* NVRTC failed for this variant */
    CT_ERR_LAUNCH = -4,         /* the launch was rejected (resources) */
    CT_ERR_CUDA = -5,           /* any other CUDA runtime error */
    CT_ERR_OOM = -6,            /* a host or device allocation failed */
    CT_ERR_TIMEOUT = -7,        /* a bounded wait gave up */
    CT_ERR_UNSUPPORTED = -8     /* no device, or not an sm_103 device */
} ct_status;

typedef enum { CT_F32 = 0, CT_BF16 = 1 } ct_dtype;

/* One correlation problem.  in_w = out_w + filter_w - 1, in_h = out_h + filter_h - 1.
 * 1 <= filter_w, filter_h <= CT_MAX_FILTER; 0 <= out_w, out_h (a zero size is a
 * no-op); in_pitch >= in_w, out_pitch >= out_w, both in elements. */
typedef struct {
    int32_t out_w, out_h;
    int32_t filter_w, filter_h;
    int64_t in_pitch, out_pitch;
    int32_t dtype; /* ct_dtype */
    int32_t reserved;
} ct_problem;

#define CT_MAX_FILTER 32

/* One point of the search space (Table 1 names: block_size_x, block_size_y,
 * tile_size_x, tile_size_y, use_shmem; unroll is Sec. 3's loop unrolling).
 * block_x * block_y <= 1024; 1 <= tile_x, tile_y <= 16; use_smem in {0, 1};
 * unroll in {0, 1, 2, 4}: 0 keeps the loop over filter rows rolled, 1 unrolls
 * the whole body (input rows slide through a register window), 2 and 4 unroll
 * the filter-row loop by that factor (Sec. 3's partial unrolling; JSON spaces
 * may list them, the built-in spaces use {0, 1}).  With use_smem = 1,
 * block_x * tile_x must be a multiple of 4 (the staged tile starts on a
 * 16-byte boundary).
 *
 * persist and taps are not points of the search space but forms of a
 * variant.  persist is chosen at launch (the same compiled variant serves both
 * values): 0 launches one block per output tile; 1 launches as many blocks as
 * the GPU holds at once, each computing every G-th tile in row-major tile
 * order (G = that block count).  ct_tune times both when
 * ct_tune_opts.grid_modes asks for it and reports the faster in each row.
 * taps chooses where the filter lives: 0 in the launch's parameter block (one
 * compiled variant serves every filter of the size); 1 compiled into the
 * variant as immediate operands of the multiply-adds (one variant per filter:
 * the first call with a new filter compiles it; the arithmetic and therefore
 * the result bits are the same).  taps = 1 applies to unroll = 1 variants
 * with finite taps; elsewhere it acts as 0.  ct_tune measures unrolled
 * configurations with taps = 1 when ct_tune_opts.taps_imm is set.
 * fma2 = 1 compiles a variant in which output rows 2k and 2k+1 of a thread
 * pair up and each input row feeds both through one paired FP32 multiply-add
 * (two fma.rn in one instruction, half the issue slots) per column and tap;
 * every output still adds its taps in (i, j) order, so the bits are the same.
 * It applies to unroll = 1, tile_y >= 2, taps = 0 variants; elsewhere it acts
 * as 0.  ct_tune tries it in the re-measurement (remeasure_forms).
 * shfl = 1 compiles a variant in which a thread reads only its own tile_x
 * values of each staged input row and takes the rest of its window from the
 * lanes to its right by warp shuffles (the filter-row reuse across a warp);
 * lanes whose window runs past the warp read theirs whole.  It applies to
 * use_smem = 1 variants with block_x a multiple of 32 and tile_x a multiple
 * of 4; elsewhere it acts as 0.  Same bits; tried by remeasure_forms bit 2. */
typedef struct {
    int32_t block_x, block_y;
    int32_t tile_x, tile_y;
    int32_t use_smem, unroll;
    int32_t persist;       /* 0: one block per tile; 1: persistent grid */
    int32_t taps;          /* 0: taps in the parameter block; 1: compiled into the variant */
    int32_t fma2;          /* 1: paired FP32 multiply-adds over pairs of output rows */
    int32_t shfl;          /* 1: window values from neighbouring lanes by warp shuffles */
} ct_config;

/* Per-variant build facts (from the NVRTC/ptxas log and the launch shape). */
typedef struct {
    int32_t regs;          /* registers per thread */
    int32_t spill_bytes;   /* spill stores + loads reported by ptxas */
    int32_t smem_bytes;    /* dynamic shared memory per block */
    int32_t cubin_bytes;
    double compile_ms;     /* 0 when served from a cache */
    int32_t from_cache;    /* 1: memory or disk cache hit */
    int32_t reserved;
} ct_variant_info;

/* ---- library and device ---------------------------------------------- */

/* Version string naming the target architecture (sm_103a).  Paper: no
 * counterpart (library plumbing). */
CT_API const char* ct_version(void);
/* Thread-local message of the last failing call on this thread ("" if none).
 * Paper: no counterpart (error reporting of the C-ABI). */
CT_API const char* ct_last_error(void);

typedef struct {
    char name[128];
    int32_t sm_count, cc_major, cc_minor;
    int32_t smem_optin_bytes;   /* max dynamic shared memory per block */
    int32_t l2_bytes;
    int32_t clock_max_khz;      /* 0 if unknown */
    int32_t reserved;
} ct_device_info;

/* Current device facts; CT_ERR_UNSUPPORTED when no CUDA device is usable.
 * Paper: Table 2 describes each GPU by these facts (compute units, clock,
 * from which the single-precision peak follows). */
CT_API ct_status ct_device_query(ct_device_info* out);

/* Directory for the on-disk cubin cache (NULL or "" disables it).  The
 * default is taken from the CONVTUNE_CACHE_DIR environment variable.  Paper:
 * Sec. 3 (the runner compiles the kernel once per configuration; the cache
 * keeps those compiles across runs). */
CT_API ct_status ct_set_cache_dir(const char* dir);

/* Drops every loaded variant (modules are unloaded on the current device).
 * Paper: Sec. 3 (compiled configurations held by the runner). */
CT_API ct_status ct_clear_cache(void);

/* ---- configurations and variants -------------------------------------- */

/* The baseline configuration: one output per thread, 32 x 8 threads,
 * global-memory reads, rolled filter-row loop.  Paper: a point of Table 1's
 * space for the 2D convolution kernel of Sec. 5; the paper names no default,
 * so this is the reading used for the tuned-vs-default speedup. */
CT_API ct_status ct_default_config(const ct_problem* p, ct_config* out);

/* Checks that (p, c) is launchable: argument ranges, threads per block and
 * the shared-memory tile against smem_limit_bytes (<= 0: the current
 * device's opt-in limit, or 232448 when there is no device).  Returns
 * CT_ERR_INVALID_CONFIG or CT_ERR_INVALID_ARG with a message otherwise.
 * Paper: Sec. 3 (restrictions the user's tuning script places on the
 * Table 1 values). */
CT_API ct_status ct_check_config(const ct_problem* p, const ct_config* c, int32_t smem_limit_bytes);

/* Compiles (or finds in a cache) the variant for (p, c) without loading it,
 * in the form that keeps the taps in the parameter block (c->taps is not
 * looked at: there is no filter here).
 * Runs on a machine without a GPU: NVRTC targets sm_103a directly.  Paper:
 * Sec. 3 (the runner compiles the kernel source with the configuration's
 * parameter values, including unroll factors, as compile-time constants). */
CT_API ct_status ct_compile(const ct_problem* p, const ct_config* c, ct_variant_info* info);
/* Compiles (or finds in a cache) the variant that ct_conv2d runs for
 * (p, c, h_filter) without loading it: with c->taps = 1 the one specific to
 * this filter, so that a first ct_conv2d call with it does not wait for the
 * compile.  Paper: Sec. 3 (compile per configuration). */
CT_API ct_status ct_compile_filter(const ct_problem* p, const ct_config* c, const void* h_filter,
                                   ct_variant_info* info);

/* ---- the correlation ---------------------------------------------------- */

/* Reads the current device's error word, which a ct_conv2d launch sets when
 * its wait for its tensor copy gave up after about two seconds (that launch
 * then stored nothing).  Synchronous: call it once the launches to check have
 * completed.  CT_OK, or CT_ERR_TIMEOUT (and the word is cleared when clear is
 * nonzero).  ct_tune checks the word after every configuration it times and
 * records such a configuration as failed with CT_ERR_TIMEOUT.  Paper: no
 * counterpart (failure capture of the bounded device waits). */
CT_API ct_status ct_device_check(int32_t clear);

/* out = correlate(image, filter) with configuration c, enqueued on stream.
 * Paper: Sec. 5 "Benchmark kernels" (the 2D convolution kernel), run at one
 * point of Table 1's tunable parameters (block_size_x/y, tile_size_x/y,
 * use_shmem) plus Sec. 3's loop unrolling.
 * d_image: in_h x in_pitch elements of p->dtype.  h_filter: filter_h x
 * filter_w row-major host array (float for CT_F32, raw bf16 bits uint16_t for
 * CT_BF16); it is copied into the launch before return.  d_out: out_h x
 * out_pitch floats.  Asynchronous with respect to the host; the first call
 * for a variant compiles and loads it (synchronously).  Variants that stage
 * their halo in shared memory with a halo of at most 256 x 256 elements load
 * it with one tensor copy (the image's tensor map travels in the launch);
 * their wait for it is bounded (see ct_device_check).  Errors:
 * CT_ERR_INVALID_ARG / CT_ERR_INVALID_CONFIG (nothing enqueued),
 * CT_ERR_COMPILE, CT_ERR_LAUNCH, CT_ERR_CUDA, CT_ERR_UNSUPPORTED. */
CT_API ct_status ct_conv2d(const ct_problem* p, const ct_config* c, const void* d_image,
                           const void* h_filter, float* d_out, void* stream);

/* End-to-end form of ct_conv2d for host-resident data (Paper: the Sec. 5
 * kernel; the host copies have no counterpart): copies h_image to
 * d_image_ws, runs the correlation into d_out_ws and copies the result to
 * h_out, then synchronises `stream`.  The work is split into bands of output
 * rows (up to 8, at least 256 rows each) on library-owned streams so that the
 * copy-in of one band, the correlation of the previous one and the copy-out
 * of the one before overlap; it starts after the work already queued on
 * `stream`.  The workspaces are caller-owned device buffers of the sizes
 * ct_conv2d needs; h_image and h_out should be pinned host memory.  Calls on
 * one device are serialised by the library. */
CT_API ct_status ct_conv2d_host(const ct_problem* p, const ct_config* c, const void* h_image,
                                const void* h_filter, float* h_out, void* d_image_ws,
                                float* d_out_ws, void* stream);
/* (Paper: as ct_conv2d_host.)  ct_conv2d_host with host rows of their own pitch (elements, >= the row
 * width; no alignment needed): only the valid columns are copied, with 2D
 * copies, into the workspaces laid out by p's pitches. */
CT_API ct_status ct_conv2d_host_pitched(const ct_problem* p, const ct_config* c, const void* h_image,
                                        int64_t h_in_pitch, const void* h_filter, float* h_out,
                                        int64_t h_out_pitch, void* d_image_ws, float* d_out_ws, void* stream);
/* (Paper: as ct_conv2d_host.)  Asynchronous form of ct_conv2d_host_pitched: the work starts after what is
 * queued on `stream`, the call returns once it is enqueued, and completion
 * (output in h_out) is recorded on the caller's CUDA event done_event
 * (cudaEvent_t); `stream` is not made to wait.  Consecutive calls therefore
 * overlap (the copy-in of one under the copy-out of the previous): the
 * caller must give overlapping calls different workspaces and host buffers
 * and must not touch them before done_event completes. */
CT_API ct_status ct_conv2d_host_async(const ct_problem* p, const ct_config* c, const void* h_image,
                                      int64_t h_in_pitch, const void* h_filter, float* h_out,
                                      int64_t h_out_pitch, void* d_image_ws, float* d_out_ws, void* stream,
                                      void* done_event);

/* ---- search spaces ------------------------------------------------------- */

typedef struct ct_space ct_space;

/* Built-in spaces (parameter order block_x, block_y, tile_x, tile_y,
 * use_smem, unroll; canonical index = position in the Cartesian product,
 * first parameter outermost):
 *   "small": block_x {16,32,64,128} x block_y {1,2,4,8} x tile {1,2}^2 x
 *            smem {0,1} x unroll {0,1}                      = 256 configs
 *   "full":  block_x {16..256 pow2} x block_y {1..16 pow2} x tile {1..8}^2 x
 *            smem {0,1} x unroll {0,1}                      = 6400 raw
 *   "paper": Table 1's convolution values: block_x 16k (k = 1..16) x
 *            block_y {1,2,4,8,16} x tile {1..4}^2 x smem {0,1} x unroll {0,1}
 * Restrictions (applied per problem): threads per block <= 1024 and the
 * shared-memory tile within the device limit.  Paper: Sec. 3 (the tunable
 * parameters and their values, given by the user's tuning script), Table 1
 * (the 2D convolution kernel's parameters and values). */
CT_API ct_status ct_space_builtin(const char* name, ct_space** out);
/* A space from JSON: {"block_x":[...], "block_y":[...], "tile_x":[...],
 * "tile_y":[...], "use_smem":[...], "unroll":[...]} (missing keys take the
 * single value of the default configuration).  Paper: Sec. 3 (the user's
 * dictionary of tunable parameters and values), Table 1. */
CT_API ct_status ct_space_from_json(const char* json, ct_space** out);
/* Releases a space.  Paper: as ct_space_builtin. */
CT_API void ct_space_free(ct_space* s);
/* Number of raw points and of points valid for p (smem_limit as in
 * ct_check_config).  Paper: Sec. 3 and Sec. 6 (size of each kernel's search
 * space after its restrictions; 4,362 points for the convolution). */
CT_API ct_status ct_space_count(const ct_space* s, const ct_problem* p, int32_t smem_limit_bytes,
                                int64_t* n_raw, int64_t* n_valid);
/* Writes up to cap valid configurations for p, in canonical order, with their
 * canonical indices (either output may be NULL); *n gets the total.  Paper:
 * Sec. 3 (the configurations the strategies draw from), Table 1 order. */
CT_API ct_status ct_space_enumerate(const ct_space* s, const ct_problem* p, int32_t smem_limit_bytes,
                                    ct_config* cfgs, int64_t* indices, int64_t cap, int64_t* n);

/* ---- tuning --------------------------------------------------------------- */

typedef enum { CT_BRUTE = 0, CT_RANDOM = 1, CT_ANNEAL = 2 } ct_strategy;

typedef struct {
    uint64_t seed;            /* strategy randomness and scratch inputs */
    double sample_fraction;   /* budget of RANDOM/ANNEAL as a fraction of the valid configs (0: 0.10) */
    int32_t max_evals;        /* > 0: overrides the budget */
    int32_t repeats;          /* timed launches per config (0: 7) */
    int32_t warmup;           /* untimed launches before timing (0: 1) */
    int32_t flush_l2;         /* 1: overwrite L2 before every timed launch */
    int32_t compile_threads;  /* 0: one per host core */
    int32_t graph_below_us;   /* kernels shorter than this are timed as a graph of
                                 back-to-back launches (0: 50 us; < 0: never) */
    int32_t anneal_chains;    /* ANNEAL: independent walkers (0: 1); each keeps one
                                 candidate in flight, and the next measured is that
                                 of the first walker, in round-robin order, whose
                                 compile has finished.  On the GPU that order depends
                                 on compile times, so a seeded annealing run is
                                 reproducible only under ct_tune_replay (where every
                                 candidate is ready at once) */
    int32_t reserved;
    const char* cache_dir;    /* cubin cache for this run (NULL: library setting) */
    const char* resume_path;  /* JSONL table: rows found there are not re-measured,
                                 new rows are appended (NULL: none) */
    const char* trace_path;   /* ANNEAL: JSONL trace of every walker step, restart
                                 and start point, appended (NULL: none) */
    int32_t grid_modes;       /* 0: time one block per tile only; 1: also time the
                                 persistent grid (cfg.persist = 1) whenever the
                                 problem has more tiles than the GPU holds at once,
                                 and keep the faster (same compile, one more timing) */
    int32_t remeasure_top;    /* > 0: after the strategy, measure the k fastest
                                 configurations again, interleaved, with
                                 remeasure_repeats launches each, and rank them by
                                 those times (ct_table_info.remeasured) */
    int32_t remeasure_repeats;/* launches per re-measured configuration (0: 31) */
    int32_t taps_imm;         /* 1: measure every unroll = 1 configuration with the
                                 problem's taps compiled in (cfg.taps = 1 in its row);
                                 the compiles are then specific to this filter */
    int32_t remeasure_forms;  /* bit 0: the re-measurement also times each unrolled
                                 candidate in the other tap form; bit 1: also in the
                                 paired multiply-add form (fma2); bit 2: also with
                                 shuffled windows (shfl); each row keeps its fastest
                                 form (cfg.taps, cfg.fma2, cfg.shfl) */
    int32_t sweep_fma2;       /* 1: the strategy measures every configuration that
                                 admits it in the paired multiply-add form (cfg.fma2 = 1
                                 in its row) instead of the scalar one */
} ct_tune_opts;

/* One row of a timing table. */
typedef struct {
    ct_config cfg;
    int64_t index;            /* canonical index in the space */
    int32_t status;           /* ct_status of compile/launch for this config */
    int32_t n;                /* timed samples */
    double t_med_ms, t_min_ms, t_std_ms;
    double gflops;            /* 2 * out_w * out_h * filter_w * filter_h / t_med */
    int32_t regs, spill_bytes, smem_bytes;
    int32_t eval_order;       /* 0-based order in which the strategy measured it */
    double compile_ms;
    double t_tiles_ms;        /* median with one block per tile (cfg.persist = 0) */
    double t_persist_ms;      /* median with the persistent grid (NaN: not timed);
                                 t_med_ms is the smaller, cfg.persist says which */
    double t_remeasured_ms;   /* median of the re-measurement (NaN: not re-measured) */
    int32_t sm_mhz;           /* SM clock sampled right after the timing (0: unknown) */
    int32_t reserved;
} ct_row;

typedef struct {
    int32_t strategy;         /* ct_strategy */
    int32_t n_rows;           /* configurations measured (or failed) */
    int64_t n_valid_space;    /* valid configurations of the space for the problem */
    int64_t best_row;         /* row index of the optimum (-1 if none) */
    double wall_ms;           /* whole ct_tune call */
    double compile_wall_ms;   /* wall time the benchmark loop waited on compiles */
    double compile_cpu_ms;    /* sum of NVRTC compile times */
    double bench_ms;          /* wall time spent launching and timing */
    double remeasure_ms;      /* wall time of the re-measurement (0: none) */
    int32_t remeasured;       /* configurations re-measured; when > 0, best_row is
                                 the fastest of them by t_remeasured_ms */
    int32_t sm_mhz_median;    /* median of the rows' sm_mhz samples (0: unknown) */
} ct_table_info;

typedef struct ct_table ct_table;

/* Tunes p over space s with strategy st: every visited configuration is
 * compiled (in parallel on host threads), launched, timed with CUDA events on
 * a private stream (median of opts->repeats), and recorded.  Failing
 * configurations become rows with a non-zero status and tuning continues.
 * d_image / d_out may be NULL, in which case the library allocates scratch
 * buffers filled from opts->seed and frees them before return; h_filter may
 * be NULL (seeded filter).  Synchronous.  *best_out gets the fastest config
 * (ties: lower canonical index); *table_out a library-owned table (free with
 * ct_table_free).  Paper: Sec. 3 (the strategies layer chooses the
 * configurations to try; the runners compile, launch and time each one with
 * events recorded before and after the kernel, and every configuration's
 * result is returned). */
CT_API ct_status ct_tune(const ct_problem* p, const ct_space* s, ct_strategy st,
                         const ct_tune_opts* opts, const void* d_image, const void* h_filter,
                         float* d_out, ct_config* best_out, ct_table** table_out);

/* The same strategies driven by a given timing landscape instead of the GPU:
 * the "measurement" of the configuration with canonical index k is
 * times_ms[k] (k < n_times; NaN or <= 0 marks a failing configuration).
 * Needs no device.  Used to study and test strategies offline.  Paper: Sec. 3
 * (the strategies layer, here driven by a recorded landscape). */
CT_API ct_status ct_tune_replay(const ct_problem* p, const ct_space* s, ct_strategy st,
                                const ct_tune_opts* opts, const double* times_ms, int64_t n_times,
                                ct_config* best_out, ct_table** table_out);

/* Access to a timing table: its row count, row i (0-based, in evaluation
 * order), the run's summary, a JSON-lines copy (one object per row; the
 * format ct_tune_opts.resume_path reads back), and its release.  Paper: Sec. 3
 * (the result of every configuration tried is returned to the user), Table 5
 * (the best configurations listed with their parameter values). */
CT_API int64_t ct_table_size(const ct_table* t);
CT_API ct_status ct_table_row(const ct_table* t, int64_t i, ct_row* out);
CT_API ct_status ct_table_info_get(const ct_table* t, ct_table_info* out);
CT_API ct_status ct_table_write(const ct_table* t, const char* path);
CT_API void ct_table_free(ct_table* t);

/* Analysis of a timing table (the configurations it measured):
 *   tuning impact = optimum performance / median performance (Sec. 4,
 *   Table 4; median of an even count = mean of the two middle values),
 *   tuned/median time, the fraction within 10 % of the optimum, performance
 *   quantiles p0/p10/p25/p50/p75/p90/p100 (linear interpolation), and the
 *   proportion of centrality C_p of Eq. 1 for each p: PageRank (damping 0.85,
 *   sinks spread uniformly) on the fitness flow graph whose edges join
 *   neighbouring configurations (one parameter one step apart in the space's
 *   value lists) towards the faster one; C_p = centrality of the local minima
 *   with time <= (1+p) * optimum over that of all local minima.  flops > 0
 *   expresses performance in GFLOP/s (else 1/time). */
typedef struct {
    int64_t n_valid, n_minima, best_index;
    double p_max, p_median, impact, tuned_vs_median, frac_within_10pct;
    double quantiles[7];
    int32_t n_p, reserved;
    double p[16], cp[16];
} ct_analysis;
CT_API ct_status ct_table_analyze(const ct_table* t, const ct_space* s, double flops, const double* p_values,
                                  int32_t n_p, ct_analysis* out);


/* ---- batched uneven problems (one graph launch) --------------------------
 *
 * Many correlations of different image and filter sizes run in ONE launch of
 * a CUDA graph, whose core is a persistent kernel.  Problems are grouped into
 * buckets (same filter size; image side below / at-or-above a split), each
 * bucket gets its own compile-time tile routine, and every block of the launch
 * takes (problem, tile) work items from a global counter until the list is
 * empty.  Bucket tile shapes are chosen by measurement on the bucket's own
 * problems; the default objective is the performance portability PP of Eq. 2
 * over the bucket's shapes (harmonic mean of the per-shape efficiencies of
 * Eq. 3), the alternative the bucket's summed time.  Results are bit-identical
 * to ct_conv2d on each problem.
 *
 * Problems big enough to fill a good part of the GPU (opts->solo_wave_pct)
 * run instead as their own launch of the single-problem kernel, whose taps
 * come from its parameter block; its configuration is tuned per filter size at
 * create (annealing, opts->solo_evals evaluations, the five fastest timed
 * again in the scalar and the paired multiply-add forms, on the largest such
 * problem, whose buffers the tuner uses).  The plan's graph holds these
 * launches, largest first, spread over opts->solo_branches parallel branches
 * (so small ones run beside each other), and the persistent launch of the
 * other problems, either after the solo launches or on a branch of its own
 * beside them; its work list either takes the buckets one after another
 * (most expensive tiles first) or interleaves them, so that tiles bound by
 * memory bandwidth run beside tiles bound by the FMA pipe.  The graph is
 * captured in each of these layouts and orders and, when some solo
 * configurations won in the paired multiply-add form, also with their scalar
 * twins; all are timed (replays, which write every output) and the fastest
 * graph is kept.
 *
 * Each item's input halo and filter taps reach shared memory by tensor-memory
 * copies (one 2D tensor map per problem, encoded at create for the bucket's
 * tile); a tile's halo box is at most 256 x 256 elements, and a problem spans
 * at most 65535 tiles along each side (otherwise CT_ERR_UNSUPPORTED).  A block
 * that waits more than about two seconds for its copies gives up, records the
 * failure in the plan's error word and exits; ct_batch_check reports it.
 *
 * Paper: batching has no counterpart in the paper (it tunes one problem at a
 * time, Sec. 3); the per-bucket choice of tile uses its performance
 * portability, Eq. 2, over the application efficiencies of Eq. 3, with the
 * bucket's problem shapes in the role of the platforms. */

typedef struct {
    const void* d_image;   /* in_h x in_pitch elements of the batch dtype (caller-owned, kept alive) */
    float* d_out;          /* out_h x out_pitch floats (caller-owned, kept alive) */
    const void* h_filter;  /* filter_h x filter_w host array (float or bf16 bits); copied at create */
    int32_t out_w, out_h, filter_w, filter_h;
    int64_t in_pitch, out_pitch;   /* elements; same alignment rules as ct_problem */
} ct_batch_item;

typedef struct {
    int32_t block_x, block_y, tile_x, tile_y;
    int32_t unroll;          /* 1: the input-row loop is unrolled */
    int32_t fma2;            /* 1: paired multiply-adds over output-row pairs (as ct_config.fma2) */
} ct_bucket_config;

typedef struct {
    int32_t dtype;          /* ct_dtype of every image in the batch */
    int32_t threads;        /* threads per block of the persistent kernel (0: 256) */
    int32_t tune;           /* 1: choose each bucket's tile by measurement; 0: fixed default tiles */
    int32_t objective;      /* 0: maximise PP over the bucket's shapes (Eq. 2); 1: minimise bucket time */
    int32_t side_split;     /* image side splitting a filter size into two buckets (0: 512; < 0: no split) */
    int32_t blocks_per_sm;  /* resident blocks per SM of the persistent grid (0: occupancy query) */
    int32_t max_tune_items; /* problems per bucket measured while tuning (0: 12) */
    int32_t solo_wave_pct;  /* a problem whose tiles under its solo configuration fill at least this
                               percentage of one wave of the GPU runs as its own ct_corr2d launch in the
                               plan's graph (0: 10; < 0: every problem goes to the persistent launch) */
    int32_t solo_evals;     /* annealing budget per filter size for the solo configuration (0: 60) */
    int32_t solo_branches;  /* parallel graph branches the solo launches are spread over (0: 12) */
    int32_t bucket_forms;   /* bucket tiles tried when tuning: 0 scalar and paired multiply-adds, 1 scalar
                               only, 2 paired only where a tile allows it (with tune = 0: the default
                               tile in the paired form) */
    int32_t persistent_layout; /* the persistent launch in the graph: 0 timed both ways, the faster kept;
                                  1 after the solo launches; 2 on a branch beside them */
    int32_t work_order;     /* the persistent launch's work list: 0 timed both ways, the faster kept;
                               1 bucket by bucket, most expensive tiles first; 2 buckets interleaved,
                               each advancing through its tiles at the same relative rate */
    int32_t min_blocks_per_sm; /* resident blocks per SM the persistent kernel's registers must allow
                                  (1..8; 0: 4); bucket tiles whose two item buffers do not fit that
                                  many blocks' share of shared memory are not tried */
} ct_batch_opts;

typedef struct {
    int32_t n_items, n_buckets;
    int64_t n_work;         /* work items (tiles) of the persistent launch per run */
    int32_t grid, threads;
    int32_t smem_bytes, regs;
    double plan_ms, tune_ms, compile_cpu_ms;
    int32_t n_solo;         /* problems run as their own launch */
    int32_t n_solo_fma2;    /* of them, launches in the paired multiply-add form */
    int32_t persistent_beside; /* 1: the persistent launch runs on a graph branch beside the solo
                                  launches; 0: after them */
    int32_t work_interleaved;  /* 1: the persistent launch takes its buckets' tiles interleaved; 0: bucket
                                  by bucket */
} ct_batch_info;

typedef struct ct_batch ct_batch;

/* Plans a batch: validates every item (as ct_conv2d would), picks the solo
 * problems (tuning their configuration per filter size, which runs kernels on
 * the largest one's buffers), buckets the rest, tunes (opts->tune) and
 * compiles the persistent kernel, uploads the problem table, tensor maps,
 * filters and work list, and captures the solo launches plus the persistent
 * launch (work counter reset + kernel) in a CUDA graph.  Synchronous; device
 * memory for the tables is owned by the plan.  Up to 16 buckets per batch.
 * Paper: Eqs. 2-3 (bucket tiles), Sec. 3 (per-size tuning of the solo
 * launches); the batch itself has no counterpart. */
CT_API ct_status ct_batch_create(const ct_batch_item* items, int32_t n, const ct_batch_opts* opts,
                                 ct_batch** out);
/* Runs the planned batch once on `stream` (one graph launch; asynchronous).
 * Runs of one plan must not overlap: they share its work counter.  Paper: no
 * counterpart (each problem's arithmetic is the Sec. 5 kernel's). */
CT_API ct_status ct_batch_run(ct_batch* b, void* stream);
/* Reads the plan's error word (synchronously; call it after the runs have
 * completed): CT_OK, or CT_ERR_TIMEOUT when a block of an earlier run gave up
 * waiting for its input copies (its outputs are then incomplete).  The word is
 * sticky for the life of the plan.  A plan with solo launches also reports
 * the device's error word (see ct_device_check; not cleared here).  Paper:
 * no counterpart (failure capture). */
CT_API ct_status ct_batch_check(const ct_batch* b);
/* The plan's shape, timings and persistent-launch resources.  Paper: no
 * counterpart. */
CT_API ct_status ct_batch_info_get(const ct_batch* b, ct_batch_info* out);
/* Bucket k: its filter size, number of problems, tile configuration and the
 * PP score (Eq. 2) of that configuration over the bucket's measured shapes
 * (NaN when the bucket was not tuned).  Paper: Eq. 2 (PP), Eq. 3. */
CT_API ct_status ct_batch_bucket(const ct_batch* b, int32_t k, int32_t* filter_w, int32_t* filter_h,
                                 int32_t* n_items, ct_bucket_config* cfg, double* pp);
/* Bucket index of item i (in the order given to ct_batch_create); -1 for a
 * problem that runs as its own launch.  Paper: no counterpart. */
CT_API int32_t ct_batch_item_bucket(const ct_batch* b, int32_t i);
/* Releases the plan, its graph and its device tables.  Paper: no counterpart. */
CT_API void ct_batch_free(ct_batch* b);

/* ---- serving: continuous batching under a device-memory budget ------------
 *
 * A server owns a device-memory budget (one arena) and a dispatcher thread.
 * Each submitted request is admitted, in arrival order, as soon as its image
 * and output fit the budget; its image is copied in; once the copy has landed
 * it joins the next launch of the persistent batch kernel (see ct_batch_*).
 * Up to max_launches launches run at once on separate streams, so requests
 * arriving while others are on the GPU are admitted and launched as memory
 * and launch slots free up, and their work overlaps with the running work.
 * A launch starts at once when none of the server's launches is running,
 * otherwise when max_batch requests are ready or the oldest ready request has
 * waited max_wait_us.  Each square filter size of [filter_min, filter_max]
 * (same parity as filter_min) has one resident tile configuration, tuned at
 * creation when opts->tune is set, so a result does not depend on which
 * requests shared its launch.  All waits are host-side and bounded by the
 * caller's timeout; no device code waits.
 *
 * Paper: serving has no counterpart in the paper; the resident per-size tile
 * configurations are tuned as in Sec. 3, and each request's arithmetic is the
 * Sec. 5 kernel's.  Every ct_server_* call below falls under this note. */

typedef struct {
    int64_t mem_budget_bytes; /* device memory for images, outputs and launch tables */
    int32_t dtype;            /* ct_dtype of all images */
    int32_t max_batch;        /* requests per launch (0: 64) */
    int32_t max_launches;     /* launches in flight at once (0: 3) */
    int32_t max_wait_us;      /* batching delay while other launches run (0: 200) */
    int32_t tune;             /* 1: tune each filter size's tile at creation */
    int32_t filter_min, filter_max;  /* served square filter sizes (0: 3 and 17) */
    int32_t reserved;
    int64_t staging_bytes;    /* pinned host staging per launch slot for the tables (0: 16 MiB) */
} ct_server_opts;

typedef struct {
    const void* h_image;   /* in_h x in_pitch host elements (pinned for asynchronous copies), read after
                              admission and until the request completes; or NULL with image_id */
    uint64_t image_id;     /* a resident image (ct_server_image_register), 0 for none */
    float* h_out;          /* out_h x out_pitch host floats (pinned), written when the request completes */
    const void* h_filter;  /* filter_h x filter_w (float or bf16 bits), copied at submit */
    int32_t out_w, out_h, filter_w, filter_h;
    int64_t in_pitch, out_pitch;   /* host row pitches in elements (any value >= the row width); on the
                                      device the server keeps compact rows and copies with 2D copies */
} ct_request;

typedef struct {
    int64_t submitted, completed, failed, launches;
    double mean_batch;     /* requests per launch */
    double p50_ms, p99_ms, mean_ms, max_ms;   /* submit -> output on the host */
    double wall_s;         /* first submit to last completion since the last reset */
    double req_per_s, gflops;
    int64_t peak_mem_bytes;
    double kernel_busy_s;      /* time some launch's kernel was running (union of the intervals
                                  between events recorded around each kernel) */
    double kernel_busy_frac;   /* kernel_busy_s / wall_s */
} ct_server_stats;

typedef struct ct_server ct_server;

/* Creates a server on the current device: tunes (opts->tune) and compiles the
 * persistent kernel for the served filter sizes, allocates the budget and
 * starts the dispatcher thread. */
CT_API ct_status ct_server_create(const ct_server_opts* opts, ct_server** out);
/* Uploads an image that stays resident (counted in the budget) until
 * released; requests can name it instead of carrying a host image.
 * Synchronous.  CT_ERR_OOM when it does not fit the budget now. */
CT_API ct_status ct_server_image_register(ct_server* s, const void* h_image, int32_t in_w, int32_t in_h,
                                          int64_t in_pitch, uint64_t* image_id);
CT_API ct_status ct_server_image_release(ct_server* s, uint64_t image_id);
/* Queues one request; returns at once with its id.  CT_ERR_UNSUPPORTED for a
 * filter size the server does not serve, CT_ERR_OOM for a request larger
 * than the whole budget.  Every request must be collected with
 * ct_server_wait. */
CT_API ct_status ct_server_submit(ct_server* s, const ct_request* rq, uint64_t* request_id);
/* Waits up to timeout_us (< 0: no limit) for the request; on success h_out
 * holds the result and *latency_ms the time from submit to completion.
 * CT_ERR_TIMEOUT when it is not done in time (the request stays queued and
 * can be waited again). */
CT_API ct_status ct_server_wait(ct_server* s, uint64_t request_id, int64_t timeout_us, double* latency_ms);
/* Waits until nothing is queued or running (timeout as above). */
CT_API ct_status ct_server_drain(ct_server* s, int64_t timeout_us);
CT_API ct_status ct_server_stats_get(ct_server* s, ct_server_stats* out);
CT_API ct_status ct_server_stats_reset(ct_server* s);
/* A request stream driven from native threads, so that the caller's
 * language does not set the rate: requests[k] is submitted at arrival_s[k]
 * seconds after the start (open loop; NULL: as soon as allowed, closed loop),
 * never with more than max_in_flight requests submitted and not yet
 * collected; a second thread collects them in submission order (each wait
 * bounded by timeout_us; < 0: none).  Requests that share an output buffer
 * must be at least max_in_flight apart.  latency_ms (n values, may be NULL)
 * receives each request's submit-to-done time (NaN when it failed). */
typedef struct {
    int64_t n;
    const ct_request* requests;
    const double* arrival_s;
    int32_t max_in_flight;
    int32_t reserved;
    int64_t timeout_us;
    double* latency_ms;
} ct_server_run_opts;

/* Waits until the server is idle, resets its statistics, runs the stream and
 * returns the statistics of this run in *out (may be NULL).  Synchronous.
 * Errors: the first failing submission's status, or CT_ERR_TIMEOUT when a
 * wait ran out (the run stops submitting; submitted requests are collected). */
CT_API ct_status ct_server_run(ct_server* s, const ct_server_run_opts* opts, ct_server_stats* out);
/* Stops the dispatcher after the queued work finishes and frees everything. */
CT_API void ct_server_destroy(ct_server* s);

/* ---- batched correlation without allocation ------------------------------
 *
 * The paper has no counterpart to this entry point.  It serves callers that
 * cannot allocate device memory when they need the work done (a process whose
 * device memory is fully budgeted, a latency-critical path that must not
 * allocate or synchronise on an allocation, a plugin whose host application
 * owns every allocation).  It runs the same correlations as a batch, with the
 * same per-output arithmetic as ct_conv2d (taps in (i, j) order, one FMA each),
 * but with a kernel compiled ahead of time and all per-call scratch (work
 * counter, problem table, tile prefix sums, FP32 filters) in one statically
 * allocated 1 MiB device array: it calls no cudaMalloc, cudaFree or other
 * allocating routine.  Its outputs are bit-identical to ct_conv2d's.  Every GPU that loads the library holds that array until
 * the process exits.
 *
 * items / n / dtype as for ct_batch_create (n <= 1024; the problem table, the
 * prefix sums and every filter must fit the 1 MiB scratch, otherwise
 * CT_ERR_INVALID_ARG with the needed size).  Enqueued on `stream`: one
 * host-to-device copy of the tables (from a library-owned host staging area,
 * filled under a lock) followed by one kernel launch.  The first call on a
 * device looks up the scratch array's device address (make that first call
 * before any stream capture).  All calls share
 * the one array and each overwrites it (the work counter is reset by every
 * call): calls whose work overlaps on the GPU race, so serialise them (one
 * stream, or wait for the previous call). */
CT_API ct_status ct_batch_run_noalloc(const ct_batch_item* items, int32_t n, int32_t dtype, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CONVTUNE_H */
