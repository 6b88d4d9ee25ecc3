/*
 * snn_oracle.h -- correctness oracle for the DPSNN per-timestep method
 * (Pastorelli et al., "Gaussian and exponential lateral connectivity on
 * distributed spiking neural network simulation", PDP 2018).
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, single-threaded CPU
 * restatement of what the simulator computes, written from the paper.  Only
 * the test suite, the smoke check and the CPU-baseline leg of the benchmark
 * may load it.  It shares no code, header, table or constant generator with
 * the CUDA library under paper_1803_08833_gb300/: every constant it uses is
 * derived here, independently.
 *
 * Parity status per function (what pins it is listed in tests/):
 *   or_philox            pinned: published Philox4x32-10 known-answer vectors
 *   or_cdf_table         pinned: closed-form kernel probabilities (2x2 grid),
 *                        stencil sizes, chi-square of drawn distances
 *   synapse generation   pinned: N*K total, weight/delay ranges and chi-square,
 *                        uniform in-degree, 2x2 all-pairs frequencies
 *   per-pair law         pinned: pair frequencies per offset against p_local and
 *   (rule 1)             A f(r) (binomial bounds), stencil against the p_min
 *                        cut, no autapses or multapses, inhibitory rows local,
 *                        Table I synapse totals of the expected out-degree
 *   Gaussian efficacies  pinned: table against normal quantiles (scipy)
 *   exponential delays   pinned: thresholds against the truncated geometric law
 *   or_lif_update        pinned: discrete closed-form f-I curve, continuous f-I
 *                        within O(dt), propagator vs numerical ODE solution,
 *                        adaptation steady state
 *   or_lif_update64      pinned: the same closed forms in double (exact ISI away
 *   (FP64 mode)          from ties, propagator within 1e-9), and the FP64 step
 *                        loop against trajectories rebuilt from it and the
 *                        drive draws, its ring against sums of the FP64 weights
 *   Poisson drive        pinned: table vs Poisson CDF, mean/variance, chi-square
 *   delivery             pinned: order independence, delay/weight arrival trace
 *   STDP (stdp = 1)      pinned: the accumulated change of every synapse against
 *                        the closed-form pair sum over the raster, weights after
 *                        a period against the clipped sums, inhibitory synapses
 *                        and zero amplitudes unchanged
 *   whole-network rates  parity unpinned against the paper (its drive is not
 *                        given and its connection rule differs from this one)
 */
#ifndef SNN_ORACLE_H
#define SNN_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Network description (Sec. III-A neuron, Sec. III-B modules and lateral
 * kernels, Sec. II-B synapse generation).  Units: um, ms, mV, Hz. */
typedef struct or_params {
    uint32_t grid_w, grid_h;        /* modules in x and y (Sec. III-B) */
    uint32_t neurons_per_module;    /* M */
    float exc_fraction;             /* 0.8 (Sec. III-B) */
    float spacing_um;               /* inter-columnar step alpha (Sec. III-B) */
    uint32_t K;                     /* synapses projected per neuron (Sec. II-B) */
    int32_t kernel;                 /* 0: B exp(-r^2/2 sigma^2), 1: A exp(-r/lambda) */
    double sigma_um, lambda_um, cutoff_um;
    float w_exc_lo, w_exc_hi, w_inh;
    uint32_t d_exc_lo, d_exc_hi, d_inh;
    float tau_m, E, V_th, V_reset, t_ref, tau_c, alpha_c, g_c, dt; /* Eq. 1-2 */
    float ext_rate_hz, J_ext;       /* external Poisson synapses (Sec. III-A) */
    float imposed_rate_hz;          /* benchmark knob: forced Bernoulli spikes */
    int32_t weight_bf16;            /* 1: weights rounded to bfloat16 */
    uint32_t fx_shift;              /* fixed-point input scale 2^-fx_shift mV */
    uint64_t seed;
    /* connection law and the distributions of efficacies and delays (Sec. II-B,
     * Sec. III-B); all zero = the fixed out-degree rule with uniform draws */
    int32_t conn_rule;              /* 0: K synapses per neuron, target module drawn from the
                                       normalised kernel; 1: the per-pair law of Sec. III-B */
    float p_local;                  /* rule 1: synapse probability to each other neuron of the
                                       source's own module (Sec. III-B: 80 %) */
    double A_remote;                /* rule 1: probability A f(r) to each neuron of a module at
                                       distance r > 0, f the Gaussian or exponential shape */
    double p_min;                   /* rule 1: modules with A f(r) <= p_min get no synapse */
    int32_t inh_local_only;         /* rule 1: inhibitory neurons project inside their module only */
    int32_t weight_dist;            /* 0: exc uniform [w_exc_lo, w_exc_hi), inh w_inh;
                                       1: Gaussian, exc mean (lo + hi) / 2, inh mean w_inh */
    float w_exc_sd, w_inh_sd;       /* standard deviations of the Gaussian efficacies */
    int32_t delay_dist;             /* 0: exc uniform integer in [d_exc_lo, d_exc_hi];
                                       1: exponential of mean delay_tau_ms, truncated to it */
    float delay_tau_ms;
    /* Spike-timing dependent plasticity (Sec. II-A: contributions at each
     * post-synaptic spike, flow step 1, and at each pre-synaptic arrival,
     * flow step 4, integrated into a long-term change of every synapse every
     * stdp_period_steps; the paper gives no rule and no parameters).  Pair-based
     * with exponential traces, excitatory synapses only: at a post-synaptic
     * spike at step t a synapse gains A_plus * sum over its arrivals a < t of
     * exp(-(t - a)/tau_plus); at an arrival at step t it loses A_minus * sum
     * over post-synaptic spikes b <= t of exp(-(t - b)/tau_minus).  Each
     * contribution is rounded to the 2^-16 mV grid and summed exactly; every
     * period the sum is added to the weight, clipped to [0, w_max]. */
    int32_t stdp;
    float stdp_A_plus, stdp_A_minus;          /* mV */
    float stdp_tau_plus_ms, stdp_tau_minus_ms;
    float stdp_w_max;                         /* mV */
    uint32_t stdp_period_steps;               /* 1000 = the paper's one second */
} or_params;

typedef struct or_consts {
    uint32_t N, n_modules, n_exc, D, ref_steps, R2, max_offsets;
    float a_m, a_c, kc;
    int32_t J_ext_fx;
    uint64_t imposed_thresh;        /* forced spike when u1 < this (2^32 = always) */
    uint32_t pois_len;
    uint64_t pois[64];              /* n_ext = #{k : pois[k] <= u0} */
    uint32_t n_pair_offsets;        /* rule 1: stencil size, local offset included; else 0 */
} or_consts;

typedef struct or_net or_net;

void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
uint16_t or_bf16_bits(float w);
float or_bf16_to_float(uint16_t b);

/* 0 on success, negative on an invalid description. */
int or_constants(const or_params* p, or_consts* c);

/* Target-module table of one source module.  thresh[j], tgt_module[j] for
 * j < *n_out; prob[j] (optional) is the FP64 normalised kernel value. */
int or_cdf_table(const or_params* p, uint32_t module, uint32_t* thresh,
                 uint32_t* tgt_module, double* prob, uint32_t cap, uint32_t* n_out);

/* One LIF+SFA update (Eq. 1-2 with the threshold/reset rules).  I_fx is the
 * total input of the step in fixed point.  Returns 1 on a spike. */
/* FP64 reference mode: the propagator constants of Eq. 1-2 kept in double,
 * a_m = exp(-dt/tau_m), a_c = exp(-dt/tau_c),
 * kc = g_c tau_m tau_c / (tau_c - tau_m) (a_c - a_m)  (g_c dt a_m if tau_c = tau_m),
 * and one neuron update in double with the input I in mV (no fixed point):
 * the same rules as or_lif_update. */
typedef struct or_consts64 {
    double a_m, a_c, kc;
} or_consts64;
int or_constants64(const or_params* p, or_consts64* k);
int or_lif_update64(const or_consts64* k, const or_params* p, uint32_t ref_steps, double* V, double* c,
                    uint8_t* ref, int exc, double I, int forced);
int or_lif_update(const or_consts* c, const or_params* p, float* V, float* cf,
                  uint8_t* ref, int exc, int32_t I_fx, int forced);
uint32_t or_poisson_count(const or_consts* c, uint32_t u0);

/* Synapse rows [first, first + count) of the network described by p, without
 * building the rest of it (row i holds entries [i*K, (i+1)*K) of the output,
 * counted from `first`).  For sampled checks of networks too large to build. */
/* Rows of the neurons ids[0 .. count) back to back (either rule), at most cap
 * synapses in all; len[r] = length of row r. */
int or_gen_rows_list(const or_params* p, const uint32_t* ids, uint32_t count, uint64_t cap, uint32_t* tgt,
                     float* w, uint8_t* d, uint32_t* len);
int or_gen_rows(const or_params* p, uint32_t first, uint32_t count, uint32_t* tgt, float* w,
                uint8_t* d);
/* Initial membrane potential of neuron i, and its external count / forced
 * flag at step t. */
float or_initial_V(const or_params* p, uint32_t i);
void or_drive(const or_params* p, const or_consts* c, uint32_t i, uint32_t t, uint32_t* n_ext,
              int* forced);

/* Rule 1 stencil (Sec. III-B): the offsets (dx, dy), in the fixed order dy
 * outer, dx inner, whose pair probability exceeds p_min; prob[j] is the
 * probability of a synapse to each neuron of the module at that offset
 * (p_local at (0, 0)), thresh[j] = floor(prob[j] * 2^32) (2^32 if prob >= 1). */
int or_pair_stencil(const or_params* p, int32_t* dx, int32_t* dy, double* prob, uint64_t* thresh,
                    uint32_t cap, uint32_t* n_out);
/* Gaussian efficacies: entry k of the 4096-entry table is the (k + 1/2)/4096
 * quantile of N(mean, sd) (clipped to the sign of the population), as float
 * and (tab64) as double; a synapse takes entry u2 >> 20. */
int or_weight_table(const or_params* p, int exc, float* tab, double* tab64);
/* Exponential delays: thresholds thr[k], k < *n_out = d_exc_hi - d_exc_lo,
 * and an excitatory delay is d_exc_lo + #{k : thr[k] <= u3}. */
int or_delay_table(const or_params* p, uint64_t* thr, uint32_t* n_out);
/* Rows [first, first + count) of either rule stored back to back: row
 * first + r has len[r] synapses; at most `cap` synapses in all. */
int or_gen_rows_v(const or_params* p, uint32_t first, uint32_t count, uint64_t cap, uint32_t* tgt,
                  float* w, uint8_t* d, uint32_t* len);

/* fp64 != 0 builds the double-precision variant (double state, double
 * weights, no fixed point) used as the precision reference. */
or_net* or_create(const or_params* p, int fp64);
void or_destroy(or_net* net);
const char* or_error(void);

uint64_t or_n_synapses(const or_net* net);
/* Row offsets of the synapse table (N + 1 entries): row i is [row_ptr[i], row_ptr[i + 1]). */
void or_get_row_ptr(const or_net* net, uint64_t* row_ptr);
void or_get_csr(const or_net* net, uint32_t* tgt, float* w, uint8_t* d);
void or_get_csr_f64(const or_net* net, double* w);

/* Delivery in a shuffled order (order-independence check); 0 = id order. */
void or_set_delivery_shuffle(or_net* net, uint64_t shuffle_seed);

/* Advance n_steps time steps.  0 on success, -1 if an int32 input overflowed. */
int or_step(or_net* net, uint32_t n_steps);

uint64_t or_raster_size(const or_net* net);
void or_get_raster(const or_net* net, uint32_t* steps, uint32_t* ids);
void or_clear_raster(or_net* net);

uint32_t or_time(const or_net* net);
void or_get_state(const or_net* net, float* V, float* c, uint8_t* ref, int32_t* ring);
/* STDP state: the accumulated change of every synapse (2^-16 mV units; CSR
 * order), the post-synaptic trace y and the pre-synaptic trace x of every
 * neuron (any pointer may be NULL). */
void or_get_stdp(const or_net* net, int64_t* delta, float* y, float* x);
void or_get_state_f64(const or_net* net, double* V, double* c);
void or_set_state_f64(or_net* net, const double* V, const double* c);
/* FP64 mode: the delay ring, D rows of N doubles (row r = inputs of steps with t % D == r) */
void or_get_ring_f64(const or_net* net, double* ring);
void or_set_state(or_net* net, const float* V, const float* c, const uint8_t* ref);
void or_get_stats(const or_net* net, uint64_t* spikes, uint64_t* rec_events, uint64_t* ext_events);

#ifdef __cplusplus
}
#endif
#endif
