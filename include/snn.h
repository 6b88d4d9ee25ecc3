/*
 * snn.h -- C ABI of libsnn.so: the per-timestep hot path of the DPSNN cortical
 * simulator (Pastorelli et al., "Gaussian and exponential lateral connectivity
 * on distributed spiking neural network simulation", PDP 2018) on one GB300.
 *
 * Model.  LIF neurons with spike-frequency adaptation (Eq. 1-2, Sec. III-A),
 * grouped in cortical modules of M neurons (80 % excitatory) on a 2-D grid
 * with spacing alpha (Sec. III-B).  Every neuron i projects K synapses with
 * target K^{ij}, delay D^{ij} and weight W^{ij} (Sec. II-B); the target module
 * is drawn from a Gaussian B exp(-r^2/2 sigma^2) or exponential A exp(-r/lambda)
 * lateral kernel (Sec. I, Sec. III-B) normalised over the in-grid modules
 * within a cut-off radius.  External synapses are a Poisson process (Sec. III-A).
 * Simulation is the mixed time/event-driven loop of Sec. II-A with a 1 ms
 * exchange step: integrate, identify spikers, queue each spike at its targets
 * for the step given by the synaptic delay.
 *
 * Conventions (every function):
 *   - Returns an snn_status; nothing throws across the ABI.  On failure a
 *     message is available from snn_last_error() (per calling thread).
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream.  Functions marked "async" only enqueue work on that stream.
 *   - Device memory comes from the caller's allocator hook (alloc_fn/free_fn),
 *     or from cudaMalloc/cudaFree when the hook is NULL.  Host buffers are
 *     caller-owned and must hold the sizes stated.
 *   - The network object is library-owned; destroy it with snn_destroy.
 *   - One network must not be used from two host threads at once.
 *
 * Units: um, ms, mV, Hz.  Input to a neuron is accumulated in int32 fixed
 * point with a quantum of 2^-fx_shift mV, so delivery order never changes a
 * result (this replaces the sorting of inputs of flow step 5, Sec. II-A).
 */
#ifndef SNN_H
#define SNN_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SNN_API __attribute__((visibility("default")))
#else
#define SNN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum snn_status {
    SNN_OK = 0,
    SNN_EINVAL = -1,    /* invalid argument or network description */
    SNN_ENOMEM = -2,    /* the allocator hook returned NULL */
    SNN_ECUDA = -3,     /* a CUDA runtime call failed (message in snn_last_error) */
    SNN_EOVERFLOW = -4, /* the device raster filled up; spikes past capacity were dropped */
    SNN_ETIMEOUT = -5,  /* a bounded device-side wait gave up */
    SNN_EBUDGET = -6    /* a request does not fit the memory budget */
} snn_status;

enum { SNN_KERNEL_GAUSS = 0, SNN_KERNEL_EXP = 1 };
enum { SNN_WEIGHT_F32 = 0, SNN_WEIGHT_BF16 = 1 };
enum { SNN_LAYOUT_DRAW = 0, SNN_LAYOUT_GROUPED = 1 };
enum { SNN_RULE_FIXED_K = 0, SNN_RULE_PAIRWISE = 1 };
enum { SNN_WDIST_UNIFORM = 0, SNN_WDIST_GAUSS = 1 };
enum { SNN_DDIST_UNIFORM = 0, SNN_DDIST_EXP = 1 };

/* Network description; plain data, copied by snn_build_network. */
typedef struct snn_config {
    uint32_t grid_w, grid_h;     /* modules along x and y (Sec. III-B, Table I) */
    uint32_t neurons_per_module; /* M; neuron i lives in module i / M */
    float exc_fraction;          /* excitatory share; neuron i is excitatory if
                                    i % M < floor(exc_fraction * M + 0.5) */
    float spacing_um;            /* grid step alpha (Sec. III-B) */
    uint32_t K;                  /* out-degree: synapses projected per neuron (Sec. II-B) */
    int32_t kernel;              /* SNN_KERNEL_GAUSS or SNN_KERNEL_EXP */
    double sigma_um;             /* Gaussian width */
    double lambda_um;            /* exponential decay length */
    double cutoff_um;            /* keep modules with dx^2 + dy^2 <= floor((cutoff/spacing)^2) */
    float w_exc_lo, w_exc_hi;    /* excitatory weight: w_lo + (w_hi - w_lo) * U[0,1) (mV) */
    float w_inh;                 /* inhibitory weight (mV) */
    uint32_t d_exc_lo, d_exc_hi; /* excitatory delay: uniform integer in [lo, hi] steps */
    uint32_t d_inh;              /* inhibitory delay (steps); all delays in [1, 255] */
    float tau_m_ms, E_mV, V_th_mV, V_reset_mV, t_ref_ms; /* Eq. 1 and reset rules */
    float tau_c_ms, alpha_c, g_c_mV;                     /* Eq. 2, SFA increment, coupling */
    float dt_ms;                 /* time step (the paper's 1 ms exchange step) */
    float ext_rate_hz, J_ext_mV; /* external Poisson synapses (Sec. III-A) */
    float imposed_rate_hz;       /* extra Bernoulli spikes per neuron and step
                                    (0 = off); a workload knob, not part of the model */
    int32_t weight_dtype;        /* SNN_WEIGHT_F32 or SNN_WEIGHT_BF16 (stored weights) */
    uint32_t fx_shift;           /* fixed-point quantum 2^-fx_shift mV, in [8, 24] */
    uint64_t seed;               /* Philox4x32-10 key */
    uint64_t raster_capacity;    /* device raster entries (spikes) kept before overflow */
    int32_t table_layout;        /* SNN_LAYOUT_DRAW: row i holds synapses k = 0..K-1 in draw order;
                                    SNN_LAYOUT_GROUPED: the same synapses stably grouped by target
                                    module (stencil order), plus a per-row segment index; needed
                                    by schedule 3 */
    /* Connection law (Sec. III-B).  SNN_RULE_FIXED_K: every neuron projects K
     * synapses whose target module is drawn from the normalised kernel
     * (fields above).  SNN_RULE_PAIRWISE: every ordered pair of distinct
     * neurons in one module is connected with probability p_local, a pair at
     * module distance r > 0 with probability A_remote f(r) (f the Gaussian or
     * exponential shape of `kernel`, unnormalised), modules where that falls
     * to p_min or below get none; one draw per pair (no autapses, no
     * multapses); K is ignored and the out-degree varies per neuron; rows are
     * ordered by target module (stencil order) and by neuron.  Needs
     * table_layout = SNN_LAYOUT_DRAW and neurons_per_module <= 65535. */
    int32_t conn_rule;
    float p_local;               /* pairwise: local connection probability (the paper: 0.8) */
    double A_remote;             /* pairwise: remote amplitude A (the paper: 0.05 Gaussian, 0.03 exponential) */
    double p_min;                /* pairwise: stencil cut (the paper: 1/1000) */
    int32_t inh_local_only;      /* pairwise: inhibitory neurons project inside their module only */
    /* Efficacies (Sec. II-B), either rule.  SNN_WDIST_UNIFORM: excitatory
     * w_exc_lo + (w_exc_hi - w_exc_lo) U[0,1), inhibitory w_inh.
     * SNN_WDIST_GAUSS: excitatory N((w_exc_lo + w_exc_hi) / 2, w_exc_sd^2),
     * inhibitory N(w_inh, w_inh_sd^2), each the (k + 1/2)/4096 quantile for a
     * uniform k in [0, 4096), clipped to the sign of the population. */
    int32_t weight_dist;
    float w_exc_sd, w_inh_sd;
    /* Excitatory delays, either rule.  SNN_DDIST_UNIFORM: uniform integer in
     * [d_exc_lo, d_exc_hi].  SNN_DDIST_EXP: an exponential of mean
     * delay_tau_ms floored onto whole steps from d_exc_lo and truncated at
     * d_exc_hi (renormalised).  Inhibitory delays stay d_inh. */
    int32_t delay_dist;
    float delay_tau_ms;
    /* Spike-timing dependent plasticity (Sec. II-A: contributions at each
     * post-synaptic spike and each pre-synaptic arrival, integrated into a
     * long-term change of every synapse every period; disabled in all of the
     * paper's measurements, Sec. III-A, which give no rule or parameters).
     * stdp = 1: pair-based with exponential traces, excitatory synapses only.
     * At a post-synaptic spike at step t a synapse gains stdp_A_plus times
     * the sum over its arrivals a < t of exp(-(t - a)/tau_plus); at an arrival
     * at step t it loses stdp_A_minus times the sum over the post-synaptic
     * spikes b <= t of exp(-(t - b)/tau_minus).  Each contribution is rounded
     * to 2^-16 mV and summed exactly (int32); at the end of every
     * stdp_period_steps steps the sum is added to the weight, clipped to
     * [0, stdp_w_max], and restarts.  Needs f32 weights and schedule 0 or 1;
     * no snapshots, batches or serving. */
    int32_t stdp;
    float stdp_A_plus, stdp_A_minus;          /* mV */
    float stdp_tau_plus_ms, stdp_tau_minus_ms;
    float stdp_w_max;                         /* mV */
    uint32_t stdp_period_steps;               /* 1000 = the paper's one second */
} snn_config;

typedef struct snn_stats {
    uint64_t steps;          /* time steps simulated so far */
    uint64_t n_spikes;       /* spikes emitted (including any beyond raster capacity) */
    uint64_t rec_events;     /* recurrent synaptic events delivered: sum over spikes of the out-degree */
    uint64_t ext_events;     /* external Poisson events received */
    uint64_t raster_count;   /* spikes recorded since the last snn_clear_raster */
    uint64_t raster_capacity;
    uint64_t neuron_phase_ns;  /* schedule 2: GPU-timer time of the neuron phases (with their barrier) */
    uint64_t deliver_phase_ns; /* schedule 2: same for the delivery phases */
} snn_stats;

typedef struct snn_net snn_net; /* opaque, library-owned */

typedef void* (*snn_alloc_fn)(size_t bytes, void* ctx);
typedef void (*snn_free_fn)(void* ptr, void* ctx);

/* Construction phase (Sec. II-A phase 1; Sec. II-B; Sec. III-B).  Validates
 * `cfg`, builds per source module the FP64 cumulative target-module table of
 * the normalised lateral kernel, draws the synapses with counter-based Philox
 * (N*K under the fixed out-degree law; one draw per candidate pair under the
 * pairwise law, which first counts every row to size the table) into a
 * row-per-neuron table (one 32-bit word target | delay << 24, f32 or bf16
 * weight), and sets the initial state: V = V_th * U[0,1), c = 0, empty delay
 * ring.  Async on `stream` except for argument checks, allocation and the
 * pairwise law's row count.  Errors: SNN_EINVAL (bad description), SNN_ENOMEM,
 * SNN_ECUDA.  *out is set only on success. */
SNN_API snn_status snn_build_network(const snn_config* cfg, snn_alloc_fn alloc_fn, snn_free_fn free_fn,
                             void* alloc_ctx, void* stream, snn_net** out);

/* Simulation phase (Sec. II-A, flow steps 1-6) for n_steps time steps.  Each
 * step: every neuron reads and clears its ring slot for this step, adds its
 * Poisson external input, integrates Eq. 1-2 exactly over dt, applies
 * threshold / reset / refractory / adaptation, and the spikes of the step
 * (ids in increasing order) are appended to the device raster; then every
 * spike adds its K weights into ring[(t + delay) mod D][target].  Async.
 * Errors: SNN_EINVAL (NULL net), SNN_ECUDA. */
SNN_API snn_status snn_step(snn_net* net, uint32_t n_steps, void* stream);

/* Copies the recorded spikes (AER events: step, neuron id; Sec. II-C),
 * ordered by (step, id), into caller-owned host arrays of `cap` entries.
 * *n_out = entries copied = min(recorded, raster capacity, cap).  Synchronises
 * `stream`.  Returns SNN_EOVERFLOW (after copying) if the device raster had
 * to drop spikes. */
SNN_API snn_status snn_read_spikes(snn_net* net, uint32_t* steps, uint32_t* ids, size_t cap,
                           size_t* n_out, void* stream);

/* Empties the device raster (async). */
SNN_API snn_status snn_clear_raster(snn_net* net, void* stream);

/* Counters of Sec. III-D's normalised cost: spikes, recurrent and external
 * ("total equivalent") synaptic events.  Synchronises `stream`.  Returns
 * SNN_ETIMEOUT (after filling *out) if a device-side wait ran out. */
SNN_API snn_status snn_get_stats(snn_net* net, snn_stats* out, void* stream);

/* Dynamic state (V, c, refractory counters, delay ring, time, counters) as an
 * opaque host blob; the synapse table is not included (it is a pure function
 * of the description).  With host_buf == NULL, *n = bytes needed.  snn_restore
 * takes a blob of the same network description.  Both synchronise `stream`. */
SNN_API snn_status snn_snapshot(snn_net* net, void* host_buf, size_t cap, size_t* n, void* stream);
SNN_API snn_status snn_restore(snn_net* net, const void* host_buf, size_t n, void* stream);

/* Copies of device data for inspection (all synchronise `stream`; any
 * pointer may be NULL to skip that array):
 *   snn_get_table:  synapse table, rows of neurons 0..N-1 back to back
 *                   (padding removed; row i has K entries under the fixed
 *                   out-degree rule, snn_get_row_lengths entries under the
 *                   pairwise rule); weights as float.
 *   snn_get_cdf:    per source module m, entries [m*max_offsets, ...):
 *                   thresholds (uint32; target j = #{thresholds <= u}) and
 *                   target modules, plus counts[m]; *max_offsets set.
 *   snn_get_state:  V, c (float), ref (uint8) of N neurons; ring as D rows of
 *                   N int32 (row r = inputs of steps t with t % D == r); *t.
 *   snn_set_state:  overwrites V, c, ref (NULL keeps the current values). */
SNN_API snn_status snn_get_table(snn_net* net, uint32_t* tgt, float* w, uint8_t* d, void* stream);
/* Segment index (grouped layout; under the pairwise law every row is grouped,
 * with one entry per stencil offset including those outside the grid and the
 * row length last): segment starts of rows [first, first + count), each
 * row `*stride` uint16 entries (stride = stencil size + 1): entry j is the
 * position in the row of the first synapse to the source module's j-th
 * in-grid stencil module (stencil order as in snn_get_cdf); entries from the
 * module's stencil count on equal K.  With seg == NULL only *stride is set. */
SNN_API snn_status snn_get_segments(snn_net* net, uint32_t first, uint32_t count, uint16_t* seg, uint32_t* stride,
                                    void* stream);
/* Rows [first, first + count) of the synapse table, back to back as in
 * snn_get_table.  Errors: SNN_EINVAL if the rows are out of range. */
SNN_API snn_status snn_get_rows(snn_net* net, uint32_t first, uint32_t count, uint32_t* tgt, float* w,
                                uint8_t* d, void* stream);
SNN_API snn_status snn_get_cdf(snn_net* net, uint32_t* thresh, uint32_t* tgt_module, uint32_t* counts,
                       uint32_t* max_offsets, void* stream);
SNN_API snn_status snn_get_state(snn_net* net, float* V, float* c, uint8_t* ref, int32_t* ring,
                         uint32_t* t, void* stream);
SNN_API snn_status snn_set_state(snn_net* net, const float* V, const float* c, const uint8_t* ref,
                         void* stream);

/* STDP state (stdp = 1): the change accumulated by every synapse since the
 * last period's application (int32, units of 2^-16 mV; rows back to back as
 * snn_get_table), and the post- and pre-synaptic traces y, x of every neuron
 * (any pointer may be NULL).  Synchronises `stream`.  Errors: SNN_EINVAL if
 * the network has no plasticity. */
SNN_API snn_status snn_get_stdp(snn_net* net, int32_t* delta, float* y, float* x, void* stream);

/* Out-degree of rows [first, first + count) (K each under the fixed rule).
 * Errors: SNN_EINVAL if the rows are out of range. */
SNN_API snn_status snn_get_row_lengths(snn_net* net, uint32_t first, uint32_t count, uint32_t* len, void* stream);

/* The construction tables the library derives on the host in FP64 from a
 * description, without building anything (any pointer may be NULL):
 * Gaussian efficacy quantiles (2 x 4096 floats, excitatory then inhibitory;
 * weight_dist = SNN_WDIST_GAUSS), exponential delay thresholds (*n_dthr
 * entries, an excitatory delay is d_exc_lo + #{k : dthr[k] <= u}), and the
 * pairwise stencil (*n_pair entries of dx, dy and floor(p 2^32), at most cap
 * written).  No GPU work.  Errors: SNN_EINVAL (invalid description or cap). */
SNN_API snn_status snn_construction_tables(const snn_config* cfg, float* wtab, uint64_t* dthr, uint32_t* n_dthr,
                                           int32_t* pair_dx, int32_t* pair_dy, uint64_t* pair_thr, uint32_t cap,
                                           uint32_t* n_pair);

/* Sizes of the network: N neurons, K (the largest out-degree), D ring rows,
 * bytes of device memory. */
SNN_API snn_status snn_get_dims(snn_net* net, uint32_t* N, uint32_t* K, uint32_t* D, uint64_t* device_bytes);

/* Execution schedule of snn_step.
 *   0: two launches per time step (neuron kernel, then delivery kernel); the
 *      delivery walks each spike's synapses one warp per 128-synapse chunk
 *      with 16-byte vector loads.
 *   1: as 0, but one thread per synapse over the flattened (spike, synapse)
 *      range.
 *   2: one cooperative (persistent) launch per snn_step call that runs all
 *      n_steps time steps, with two grid barriers per step; the delivery is
 *      that of schedule 0.  Every barrier wait is bounded (snn_set_wait_limit);
 *      if one runs out the launch stops and later calls report SNN_ETIMEOUT.
 *   3: as 2, but target-owned delivery: each CTA gathers, for a target module,
 *      the row segments of the step's spikes that target it, accumulates them
 *      in a shared-memory tile of (D - 1) x M int32 and adds the tile into the
 *      ring with plain coalesced writes.  Needs table_layout =
 *      SNN_LAYOUT_GROUPED and a tile that fits in shared memory.
 *   4: one cooperative launch per call, one CTA per SM, each CTA owning a
 *      band of ceil(N / SMs) neurons: it integrates them and keeps the delay
 *      ring rows of the next W steps of its band in shared memory (the
 *      window, snn_set_window).  Rows are pushed as in schedule 2; an event
 *      with delay <= W becomes a record in the owner band's queue, applied by
 *      the owner with shared-memory atomics, one with a longer delay goes into
 *      the ring with an L2 reduction.  Between calls the ring holds the same
 *      values as under the other schedules.  Two grid barriers per step,
 *      bounded like those of schedule 2.  Errors: SNN_EINVAL if no window
 *      row fits in shared memory, SNN_ENOMEM for the queues (G x G x cap x
 *      8 bytes, G = SMs).
 *   5: as 4 (one band of neurons per SM, a delay window of W steps per band
 *      in shared memory, snn_set_pull_window), but pulled: after the
 *      neuron phase every CTA reads, from the row of each spike whose source
 *      module's stencil reaches its band, the one contiguous range of
 *      synapses that targets the band's modules (the rows are grouped by
 *      target module), adds the events of delay <= W into its window with
 *      shared-memory atomics and those of longer delay into the ring with L2
 *      reductions.  One grid barrier per step.  Needs rows grouped by target
 *      module -- table_layout = SNN_LAYOUT_GROUPED under the fixed out-degree
 *      law, any layout under the per-pair law (its rows are grouped by
 *      stencil offset) -- of at most 8188 synapses.  The band's neuron state
 *      stays in the SM's tensor memory for the launch (bands of at most
 *      28,672 neurons).  Errors: SNN_EINVAL (no grouped rows, a row too
 *      long, no window row fits in shared memory, or the band's state does
 *      not fit in tensor memory), SNN_ENOMEM.
 * All schedules give bit-identical results.  block: threads per block of the
 * delivery kernel for schedules 0 and 1 (multiple of 32 in [32, 256], 0 =
 * default); ignored by schedule 2.  Errors: SNN_EINVAL. */
SNN_API snn_status snn_set_schedule(snn_net* net, int32_t schedule, int32_t block);

/* Delay window of schedule 4 (no counterpart in the paper; the delay queues
 * are those of flow step 3, Sec. II-A): window = steps of the ring each band
 * keeps in shared memory (0 = the most that fit, at most D - 1), queue_cap =
 * records per (owner, producer) queue and step (0 = a default from the
 * expected events of a step).  A queue that fills up sends its further
 * events to the ring and the owner folds them in, so any capacity gives the
 * same results.  Outputs (may be NULL): the window and capacity in use.
 * Synchronises `stream`.  Errors: SNN_EINVAL (window too large, capacity >
 * 2^20), SNN_ENOMEM. */
SNN_API snn_status snn_set_window(snn_net* net, uint32_t window, uint32_t queue_cap, uint32_t* window_out,
                                  uint32_t* cap_out, void* stream);

/* Bands and delay window of schedule 5 (no counterpart in the paper; the
 * window holds the band's part of the delay queues of flow step 3, Sec. II-A).
 * band_mode 1: every CTA owns ceil(N / SMs) neurons (rounded to 4), so a band
 * also reads the synapses of the modules it shares with its neighbours and
 * skips those targets; 2: band boundaries only at module boundaries that fall
 * on a multiple of 4 neurons (every 4 / gcd(M, 4)-th module), so a band reads
 * only its own synapses but bands differ in size; 0: 2 where its largest band
 * is no larger than a band of mode 1 plus one module, else 1.  window = steps
 * each band keeps in shared memory (0 = the most that fit, at most D - 1);
 * events of a longer delay go through the ring in global memory.  Every
 * choice gives the same results.  Outputs (may be NULL): the window and the
 * band mode in use.  Synchronises `stream`.  Errors: SNN_EINVAL (rows not
 * grouped, band_mode not 0-2, window too large), SNN_ENOMEM. */
SNN_API snn_status snn_set_pull_window(snn_net* net, uint32_t window, int32_t band_mode, uint32_t* window_out,
                                       int32_t* mode_out, void* stream);

/* Banded delivery of schedule 2 (no counterpart in the paper, whose processes
 * each own a tile of the grid): the target module rows are split into `bands`
 * equal bands delivered one after another in every step, behind a grid
 * barrier each, so that one band's columns of the delay ring stay in L2 when
 * the whole ring does not (Table I's 48x48 and 96x96 grids).  A spike takes
 * part in the bands its stencil reaches, with the synapses of its row that
 * target the band (rows must be grouped by target module: table_layout =
 * SNN_LAYOUT_GROUPED, or the pairwise law).  bands = 0 picks ceil(ring bytes /
 * (L2 / 2)), at most grid_h / (2 R + 1) for a stencil reaching R module rows
 * up and down; every network starts with that choice.
 * *chosen (may be NULL) receives the count in use.  Results are identical for
 * every band count.  Synchronises `stream`.  Errors: SNN_EINVAL (bands >
 * grid_h, or > 1 without a segment index). */
SNN_API snn_status snn_set_bands(snn_net* net, uint32_t bands, uint32_t* chosen, void* stream);

/* Resident neuron state of schedule 2 (no counterpart in the paper; the state
 * is that of Eq. 1-2 and the refractory counter, Sec. III-A): every CTA of
 * the persistent launch keeps V, c and ref of its neurons in shared memory
 * for the whole launch
 * (read at the start, written back at the end), when they fit next to the
 * kernel's other shared memory (36 B per 4 neurons: up to ~5,000 quads per
 * CTA on a GB300; the 96x96 grid does not fit and keeps them in global
 * memory).  enable = 0 keeps them in global memory, 1 (the default) restores
 * the choice.  *resident (may be NULL) receives 1 if the launches keep the
 * state resident.  Results are identical either way.  Synchronises `stream`.
 * Errors: SNN_EINVAL. */
SNN_API snn_status snn_set_resident_state(snn_net* net, int32_t enable, int32_t* resident, void* stream);

/* Autotuner: runs every applicable schedule (0 and 1 at 128 and 256 threads
 * per delivery block, 2, 3 if the network has the grouped layout and its
 * tile fits, 4 if a delay window fits, 5 if the rows are grouped by target
 * module: the grouped layout, or the per-pair law) for trial_steps steps
 * from the same snapshot of the dynamic state, times each with CUDA events, restores the state (the raster and the
 * counters are as before the call) and selects the fastest.  If cache_path
 * is not NULL the choice is looked up there first and appended after
 * tuning; the key holds the network's shape, weight type, layout, rates and
 * the GPU name.  Outputs (may be NULL): the chosen schedule and block, and
 * the measured ms per step (-1 on a cache hit).  Synchronises `stream`. */
SNN_API snn_status snn_autotune(snn_net* net, uint32_t trial_steps, const char* cache_path, int32_t* schedule,
                                int32_t* block, double* best_ms_per_step, void* stream);

/* Kernel timing: with every = n >= 1, the launches of every n-th snn_step
 * time step (schedules 0, 1) or every persistent launch (schedule 2) are
 * bracketed by CUDA events on the launching stream (0 = off).
 * snn_kernel_time returns, for `which` (SNN_TIMER_NEURON, SNN_TIMER_DELIVER,
 * SNN_TIMER_PERSISTENT), the summed device time in ms and the number of timed
 * launches.  Synchronises the stream of the timed launches. */
enum { SNN_TIMER_NEURON = 0, SNN_TIMER_DELIVER = 1, SNN_TIMER_PERSISTENT = 2 };
SNN_API snn_status snn_set_timing(snn_net* net, int32_t every);
SNN_API snn_status snn_kernel_time(snn_net* net, int32_t which, double* ms, uint64_t* launches);

/* Bound of every device-side wait (the persistent kernel's grid barriers),
 * in ns of the GPU's global timer; default 2e9 (2 s).  Errors: SNN_EINVAL
 * for 0. */
SNN_API snn_status snn_set_wait_limit(snn_net* net, uint64_t ns);

/* Testing aid for the failure path: the persistent kernel's barriers expect
 * `extra` arrivals beyond the grid, which never come, so every wait runs out
 * after the wait limit and the launch reports SNN_ETIMEOUT.  0 = normal.
 * Nothing faults or hangs: the waits are bounded. */
SNN_API snn_status snn_set_barrier_extra(snn_net* net, uint32_t extra);

/* Clears the sticky device error state (after SNN_ETIMEOUT).  The network's
 * dynamic state is then undefined until snn_restore.  Synchronises. */
SNN_API snn_status snn_clear_error(snn_net* net, void* stream);

/* Number of this library's kernel launches issued so far (all networks). */
SNN_API uint64_t snn_launch_count(void);

/* Target-module tables without any device allocation.  The paper has no
 * counterpart: this exists for callers that cannot let the library allocate
 * device memory -- a process whose device memory belongs to a pool or arena
 * that must not be fragmented behind its back, or a latency-critical loop
 * that cannot afford the device-wide synchronisation of cudaMalloc/cudaFree.
 * It writes the same tables snn_build_network builds (see snn_get_cdf) into
 * caller-owned DEVICE buffers: thresh and tgt_module of n_modules *
 * max_offsets uint32 each (row m = source module m, entries j < counts[m]
 * valid) and counts of n_modules uint32.  With all three NULL it only sets
 * *max_offsets (host) and returns.  Async on `stream`.
 * Scratch: a fixed array inside the library image (4 MiB of FP64 plus a
 * 16 KiB offset list) that every GPU loading the library holds until the
 * process exits; n_modules * max_offsets must be <= 524,288 and
 * max_offsets <= 4,096, else SNN_EINVAL.  No cudaMalloc, cudaFree or other
 * allocating call is made.
 * The first call on a device looks up the scratch's device address
 * (cudaGetSymbolAddress, with that device current); make it before any stream
 * capture.  Every later call only enqueues two kernels on `stream` (the
 * stencil offsets are generated on the device, no host-to-device copy), so it
 * may be captured into a CUDA graph.  The looked-up addresses are kept per
 * device index for the life of the process: do not call this entry point
 * after cudaDeviceReset (or any teardown of the device's primary context).
 * Calls share the scratch, so calls that overlap on the GPU (on
 * different streams, or from different threads) race and must be serialised
 * by the caller.  The scratch needs no clearing: every entry read is first
 * written by the same call.
 * Errors: SNN_EINVAL (bad description, sizes over the limit, partial
 * outputs), SNN_ECUDA. */
SNN_API snn_status snn_build_cdf_static(const snn_config* cfg, uint32_t* thresh, uint32_t* tgt_module,
                                        uint32_t* counts, uint32_t* max_offsets, void* stream);

/* ---- Batched execution: many independent networks in one persistent launch
 * (no counterpart in the paper, which simulates one network per run; each
 * network's time steps are those of snn_step, Sec. II-A flow steps 1-6).
 * Network i is advanced steps[i] time steps per call.  Results are
 * bit-identical to running each network alone.  The networks are grouped into
 * waves (below); a wave of one network runs the persistent kernel of
 * schedule 2, a wave of several runs one cooperative launch laid out in one
 * of two ways (snn_batch_set_mode):
 *  - groups: every network on a group of CTAs of its own (one CTA per SM),
 *    sized so that the groups finish together by a cost model of a step,
 *    (a fixed latency plus work over the group's CTAs) refined by the groups'
 *    measured times of the previous call; each group passes its own
 *    network's grid barriers with that network's wait limit and test knob;
 *  - global: all networks share one global space of neurons and, every step,
 *    one global space of delivery tasks, each split evenly over every warp of
 *    the grid, with one pair of grid barriers per step for the whole wave,
 *    using the smallest wait limit and the largest test knob of the wave.
 * The nets stay owned by the caller and must outlive the batch.  Errors:
 * SNN_EINVAL (NULL or repeated nets, a batch too large), SNN_ENOMEM,
 * SNN_ECUDA.  A barrier wait that runs out marks its network (groups) or
 * every network of the wave (global): their snn_get_stats returns
 * SNN_ETIMEOUT. */
typedef struct snn_batch snn_batch;
SNN_API snn_status snn_batch_create(snn_net* const* nets, uint32_t n, snn_alloc_fn alloc_fn, snn_free_fn free_fn,
                                    void* alloc_ctx, snn_batch** out);
/* Networks are grouped, in order, into waves whose delay rings fit together
 * in half the L2 cache (the ring takes one random reduction per synaptic
 * event, which is several times slower once the rings spill to DRAM); each
 * wave is one launch.  snn_batch_waves reports the wave count and the ring
 * budget in bytes. */
SNN_API snn_status snn_batch_waves(snn_batch* b, uint32_t* waves, uint64_t* ring_budget);
/* Regroups the networks into waves for another ring budget (bytes > 0). */
SNN_API snn_status snn_batch_set_ring_budget(snn_batch* b, uint64_t bytes);
/* Runs network i for steps[i] (host array of n; 0 = idle) time steps.  Async;
 * a call first synchronises `stream`, whose previous call on this batch may
 * still read the batch's pinned staging: keep one stream per batch. */
SNN_API snn_status snn_batch_step(snn_batch* b, const uint32_t* steps, void* stream);
/* enable != 0: snn_batch_step replays a CUDA graph holding the launches of
 * all waves (captured on first use, and again when a wave's longest step
 * count changes). */
SNN_API snn_status snn_batch_set_graph(snn_batch* b, int32_t enable);
/* Layout of the waves of two or more networks.  SNN_BATCH_GROUPS (the
 * default): groups, except for a wave with more networks than SMs or with a
 * banded network (snn_set_bands), which runs global.  SNN_BATCH_GLOBAL:
 * global always.  Regroups the waves (synchronises the device).  Errors:
 * SNN_EINVAL (NULL batch, unknown mode). */
enum { SNN_BATCH_GROUPS = 0, SNN_BATCH_GLOBAL = 1 };
SNN_API snn_status snn_batch_set_mode(snn_batch* b, int32_t mode);
/* Launch shape of the waves laid out globally: 0 (default) two CTAs per SM
 * with four delivery tasks in flight per warp, 1 one CTA per SM with six.
 * Regroups the waves (synchronises the device).  Errors: SNN_EINVAL. */
SNN_API snn_status snn_batch_set_shape(snn_batch* b, int32_t shape);
/* Layout, launch shape and ring budget in one regrouping (as snn_batch_set_mode,
 * snn_batch_set_shape and snn_batch_set_ring_budget together).  Errors:
 * SNN_EINVAL. */
SNN_API snn_status snn_batch_set_layout(snn_batch* b, int32_t mode, int32_t shape, uint64_t ring_budget);
/* Autotuner of the batch (no counterpart in the paper): times every
 * combination of layout (SNN_BATCH_GROUPS, SNN_BATCH_GLOBAL), launch shape (0,
 * 1) and ring budget (0.35, 0.5, 0.65 of the L2) that gives a distinct wave
 * plan, on trial_steps steps of every network from one snapshot of all their
 * states (restored after each trial, so tuning changes no result), and keeps
 * the fastest.  With cache_path != NULL the choice is looked up first and
 * appended after tuning, keyed by the GPU, the networks' shapes and
 * trial_steps.  Outputs (may be NULL): the chosen layout, shape and budget,
 * the measured ms per step (-1 on a cache hit), and trial_ms[12], the ms per
 * step of every candidate in the order layout x shape x budget (-1 where a
 * candidate repeated an earlier wave plan, or on a cache hit).  Synchronises
 * `stream`.  Errors: SNN_EINVAL (NULL batch, trial_steps = 0, a network with
 * stdp). */
enum { SNN_BATCH_TUNE_CANDIDATES = 12 };
SNN_API snn_status snn_batch_autotune(snn_batch* b, uint32_t trial_steps, const char* cache_path, int32_t* mode,
                                      int32_t* shape, uint64_t* ring_budget, double* best_ms_per_step,
                                      double* trial_ms, void* stream);
/* cta (host array of n): the CTAs each network's group had in the last
 * snn_batch_step (0: idle, alone in its wave, or in a global wave). */
SNN_API snn_status snn_batch_groups(snn_batch* b, uint32_t* cta);
/* The CTA split of a grouped wave, host only: network i runs steps[i] steps
 * of an estimated work[i] CTA-microseconds each (finite, >= 0), a step on G
 * CTAs taking 8 us + work[i] / G.  Writes cta[i] (0 iff steps[i] == 0; they
 * sum to ctas when any network runs) minimising the largest
 * steps[i] (8 + work[i] / cta[i]).  Errors: SNN_EINVAL (NULL arrays, n = 0,
 * n > ctas, a work that is negative or not finite). */
/* The bands and run tables of schedule 5, host only (no counterpart in the
 * paper): for a description and `sms` CTAs (one per SM), band_mode 1 (uniform
 * bands of ceil(N / 4 / sms) quads) or 2 (module-aligned bands).  Writes bq
 * (sms + 1 entries: band b owns the quads [bq[b], bq[b + 1]), bq[sms] =
 * ceil(N / 4)), run_ptr (sms + 1: the runs of band b are [run_ptr[b],
 * run_ptr[b + 1])) and runs (pairs {source module, j0 | j1 << 16}: the band
 * reads, from each spike of that source module, the stencil entries [j0, j1)
 * of the source's in-grid stencil, the ones whose target modules overlap the
 * band) and *n_runs.  Errors: SNN_EINVAL (NULL arrays, sms = 0, band_mode not
 * 1 or 2, an empty grid, N >= 2^24), SNN_EOVERFLOW (more than cap runs; *n_runs,
 * bq and run_ptr are set, so a second call can size runs). */
SNN_API snn_status snn_plan_pull_bands(const snn_config* cfg, uint32_t sms, int32_t band_mode, uint32_t* bq,
                                       uint32_t* run_ptr, uint32_t* runs, uint32_t cap, uint32_t* n_runs);

SNN_API snn_status snn_plan_groups(const uint32_t* steps, const double* work, uint32_t n, uint32_t ctas,
                                   uint32_t* cta);
/* CUDA-event time (ms) and count of the batch launches since creation. */
SNN_API snn_status snn_batch_time(snn_batch* b, double* ms, uint64_t* launches);
SNN_API void snn_batch_destroy(snn_batch* b);

/* ---- Serving: a continuous-batching loop over simulation requests.
 * snn_server_submit queues a request (description, number of time steps,
 * arrival time in ns of the host's monotonic clock, 0 = now); it is rejected
 * with SNN_EBUDGET if it could never fit the device-memory budget.  Each
 * snn_server_tick admits queued requests in arrival order while their
 * estimated footprint (snn_estimate_bytes) fits the budget and a slot is
 * free, advances every resident network by up to `chunk_steps` steps in one
 * batched persistent launch (snn_batch_*), synchronises, and retires the
 * finished networks: their results (counters, hashes of raster and final V,
 * queueing and total latency) become available to snn_server_poll and their
 * memory returns to the budget.  Results do not depend on which other
 * requests shared a launch. */
typedef struct snn_server snn_server;
typedef struct snn_request_result {
    uint64_t request_id;
    uint64_t steps, n_spikes, rec_events, ext_events;
    uint64_t raster_hash; /* FNV-1a over the (step, id) raster arrays */
    uint64_t state_hash;  /* FNV-1a over the final membrane potentials */
    double queue_ms;      /* arrival -> admission */
    double latency_ms;    /* arrival -> completion */
    int32_t status;          /* snn_status of the request */
    int32_t raster_overflow; /* 1 if the request's raster capacity was exceeded (hash over the kept part) */
} snn_request_result;
typedef struct snn_server_stats_t {
    uint64_t ticks, launches, rec_events, ext_events, steps, busy_ns, used_bytes;
    uint32_t active, queued;
} snn_server_stats_t;
SNN_API uint64_t snn_estimate_bytes(const snn_config* cfg);
SNN_API snn_status snn_server_create(uint64_t budget_bytes, uint32_t chunk_steps, uint32_t max_slots,
                                     snn_alloc_fn alloc_fn, snn_free_fn free_fn, void* alloc_ctx, void* stream,
                                     snn_server** out);
SNN_API snn_status snn_server_submit(snn_server* s, const snn_config* cfg, uint32_t n_steps, uint64_t arrival_ns,
                                     uint64_t* request_id);
/* Layout of every tick's batch (snn_batch_set_layout; e.g. the choice of
 * snn_batch_autotune on a sample of the request mix); ring_budget 0 keeps the
 * batch's default.  Errors: SNN_EINVAL. */
SNN_API snn_status snn_server_set_batch(snn_server* s, int32_t mode, int32_t shape, uint64_t ring_budget);
SNN_API snn_status snn_server_tick(snn_server* s, uint32_t* n_active, uint32_t* n_queued);
SNN_API snn_status snn_server_poll(snn_server* s, snn_request_result* out, uint32_t cap, uint32_t* n_out);
SNN_API snn_status snn_server_stats(snn_server* s, snn_server_stats_t* out);
/* Host monotonic clock in ns (the time base of arrival_ns). */
SNN_API uint64_t snn_now_ns(void);
SNN_API void snn_server_destroy(snn_server* s);

/* ---- Spatial decomposition (Sec. II-D) with the two-step spike exchange
 * (Sec. II-E) and deferred arborization (Sec. II-C).  The paper runs one
 * network on many processes, each owning a tile of modules; a shard here owns
 * the module rows [H k / n, H (k + 1) / n) of an n-way split of the grid (its
 * neurons are one contiguous id range), their state and delay ring, and a
 * target-side copy of the synapses that the halo sources -- every neuron
 * within the stencil's row radius of the stripe -- project into it (rows of
 * the fixed out-degree law drawn exactly as snn_build_network draws them,
 * restricted to targets in the stripe, draw order kept).  A time step is:
 *   snn_shard_integrate  the stripe's neurons; the step's spikes (global ids,
 *                        increasing) and their count are left in the shard's
 *                        outbox (device memory, snn_shard_outbox) and in its
 *                        raster;
 *   exchange             every shard sends its spike count, then its ids, to
 *                        the shards whose halo covers it (its peers: indexes
 *                        peer_lo .. peer_hi of snn_shard_info, itself included);
 *   snn_shard_deliver    the inbound lists (device pointers to ids and to
 *                        their count, one list per peer, the shard's own
 *                        outbox included) through the target-side table into
 *                        the shard's ring; the step ends.
 * The union of the shards' rasters and states is bit-identical to
 * snn_build_network's network of the same description.  snn_shards_run runs
 * all n shards of one decomposition on the current device, exchanging through
 * the outboxes in place.  Only the fixed out-degree law is supported.
 * Errors: SNN_EINVAL (pairwise law, index >= n_shards, n_shards > grid_h, a
 * shard reaching more than 16 shards), SNN_ENOMEM, SNN_ECUDA. */
typedef struct snn_shard snn_shard;
typedef struct snn_shard_info_t {
    uint32_t n_shards, index;
    uint32_t row0, row1;        /* module rows owned */
    uint32_t n0, n1;            /* neurons owned [n0, n1) */
    uint32_t h0, h1;            /* halo sources [h0, h1) whose rows are copied */
    uint32_t peer_lo, peer_hi;  /* shards whose spikes can reach this one */
    uint32_t D, t;              /* ring rows; next time step */
    uint64_t table_synapses;    /* synapses in the target-side copy */
    uint64_t device_bytes;
} snn_shard_info_t;
SNN_API snn_status snn_shard_build(const snn_config* cfg, uint32_t n_shards, uint32_t index, snn_alloc_fn alloc_fn,
                                   snn_free_fn free_fn, void* alloc_ctx, void* stream, snn_shard** out);
SNN_API snn_status snn_shard_info(snn_shard* shard, snn_shard_info_t* out);
/* Async. */
SNN_API snn_status snn_shard_integrate(snn_shard* shard, void* stream);
/* Device pointers of the outbox: ids (capacity n1 - n0) and the count. */
SNN_API snn_status snn_shard_outbox(snn_shard* shard, uint32_t** ids, uint32_t** count);
/* Async; ids and counts are host arrays of n_lists (<= 16) device pointers. */
SNN_API snn_status snn_shard_deliver(snn_shard* shard, const uint32_t* const* ids, const uint32_t* const* counts,
                                     uint32_t n_lists, void* stream);
/* n_steps steps of shards[0..n) (indexes 0..n-1 of one decomposition, at one
 * time step, on one device).  Async. */
SNN_API snn_status snn_shards_run(snn_shard* const* shards, uint32_t n, uint32_t n_steps, void* stream);
/* The shard's raster ((step, id), ordered) as snn_read_spikes; its state: V,
 * c, ref of its n1 - n0 neurons and the ring as D rows of n1 - n0 int32;
 * counters (n_spikes and rec_events count its own spikes, ext_events its own
 * neurons' drive).  All synchronise `stream`. */
SNN_API snn_status snn_shard_read_spikes(snn_shard* shard, uint32_t* steps, uint32_t* ids, size_t cap, size_t* n_out,
                                         void* stream);
SNN_API snn_status snn_shard_get_state(snn_shard* shard, float* V, float* c, uint8_t* ref, int32_t* ring,
                                       void* stream);
SNN_API snn_status snn_shard_stats(snn_shard* shard, snn_stats* out, void* stream);
SNN_API void snn_shard_destroy(snn_shard* shard);

SNN_API void snn_destroy(snn_net* net);
SNN_API const char* snn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
