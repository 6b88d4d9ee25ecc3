/*
 * snn_oracle.c -- correctness oracle for the DPSNN per-timestep method
 * (Pastorelli et al., PDP 2018).  TEST INFRASTRUCTURE ONLY: see snn_oracle.h.
 *
 * Plain single-threaded C, compiled with -ffp-contract=off so that every
 * floating-point expression is evaluated exactly as written (no fused
 * multiply-add on any host).  The method, in the paper's order:
 *
 *   construction (Sec. II-B, Sec. III-B): every neuron i projects K synapses;
 *     synapse j gets a target K^{ij} drawn from the normalised lateral kernel,
 *     a delay D^{ij} and a weight W^{ij};
 *   simulation (Sec. II-A, steps 1-6 of the execution flow): each 1 ms step,
 *     neurons integrate the inputs queued for this step (recurrent + external
 *     Poisson synapses, Sec. III-A), spiking neurons are identified, and their
 *     spikes are queued at the targets for the step given by each delay.
 *
 * Readings of the paper used here (where it is silent or ambiguous):
 *   - Eq. 1 prints +(V-E)/tau_m; the leak is read as -(V-E)/tau_m (the
 *     standard LIF of the cited Gigante et al. model).  E = 0 by default and
 *     C_m is absorbed into g_c.
 *   - The event-driven solver of flow step 6 is the exact propagator of
 *     Eq. 1-2 over one step: with integer delays every input arrives on a step
 *     boundary, so integrating each arrival exactly equals decaying V and c
 *     over dt and then adding the step's summed jumps.
 *   - "exceeds" the threshold is a strict >; after a spike V is held at V_r
 *     for round(tau_arp/dt) steps, inputs arriving then are discarded, c keeps
 *     decaying; c += alpha_c on a spike of an excitatory neuron (Sec. III-A:
 *     the SFA term is zero for inhibitory neurons).
 *   - The target module is drawn from one kernel normalised over all in-grid
 *     modules within the cut-off radius, including the source (r = 0); open
 *     grid boundaries; draws with replacement (autapses/multapses allowed).
 *   - Flow step 5 (sorting the inputs) is replaced by an exact int32 fixed
 *     point sum: integer addition does not depend on the order.
 *   - The per-pair law of Sec. III-B (conn_rule 1): every ordered pair of
 *     distinct neurons in one module is connected with probability p_local,
 *     a pair at module distance r > 0 with probability A f(r) (f the
 *     Gaussian or exponential shape), modules with A f(r) <= p_min get none;
 *     one independent draw per pair, so no autapses and no multapses, and the
 *     out-degree varies from neuron to neuron; inhibitory neurons connect
 *     inside their module only (the caption of Fig. 3); open boundaries.
 *   - Gaussian efficacies (Sec. II-B) are drawn by inverse CDF from a
 *     4096-quantile table; exponential delays are the continuous law of mean
 *     delay_tau_ms floored onto whole steps from d_exc_lo and truncated at
 *     d_exc_hi (renormalised).  The paper gives neither's parameters.
 */
#include "snn_oracle.h"

#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#define OR_TAG_GEN 0u
#define OR_TAG_DRIVE 1u
#define OR_TAG_INIT 2u
#define OR_TAG_CONN 3u
#define OR_WTAB 4096u

static char g_err[256];

static void set_err(const char* msg) {
    snprintf(g_err, sizeof g_err, "%s", msg);
}

const char* or_error(void) { return g_err; }

/* ------------------------------------------------------------------------ */
/* Philox4x32-10, from Salmon, Moraes, Dror, Shaw, "Parallel Random Numbers:
 * As Easy as 1, 2, 3" (SC'11): ten rounds of two 32x32->64 multiplications
 * with the round key bumped by the Weyl constants between rounds. */
void or_philox(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
    uint32_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int round = 0; round < 10; ++round) {
        if (round > 0) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
        uint64_t p0 = (uint64_t)0xD2511F53u * (uint64_t)x0;
        uint64_t p1 = (uint64_t)0xCD9E8D57u * (uint64_t)x2;
        uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
        uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
        uint32_t y0 = hi1 ^ x1 ^ k0;
        uint32_t y1 = lo1;
        uint32_t y2 = hi0 ^ x3 ^ k1;
        uint32_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

static void draw(const or_params* p, uint32_t a, uint32_t b, uint32_t tag, uint32_t out[4]) {
    uint32_t ctr[4] = {a, b, tag, 0u};
    uint32_t key[2] = {(uint32_t)p->seed, (uint32_t)(p->seed >> 32)};
    or_philox(ctr, key, out);
}

/* 24-bit uniform in [0, 1): top 24 bits of a word times 2^-24 (exact). */
static float unit24(uint32_t u) { return (float)(u >> 8) * (1.0f / 16777216.0f); }
static double unit24d(uint32_t u) { return (double)(u >> 8) * (1.0 / 16777216.0); }

/* Round-to-nearest-even to bfloat16 (the top 16 bits of an IEEE binary32). */
uint16_t or_bf16_bits(float w) {
    uint32_t bits;
    memcpy(&bits, &w, 4);
    if ((bits & 0x7F800000u) == 0x7F800000u && (bits & 0x007FFFFFu))
        return (uint16_t)((bits >> 16) | 0x40u); /* quiet NaN */
    uint32_t lsb = (bits >> 16) & 1u;
    bits += 0x7FFFu + lsb;
    return (uint16_t)(bits >> 16);
}

float or_bf16_to_float(uint16_t b) {
    uint32_t bits = (uint32_t)b << 16;
    float w;
    memcpy(&w, &bits, 4);
    return w;
}

/* ------------------------------------------------------------------------ */
/* Constants of the method, all derived here in FP64 and rounded once. */
int or_constants(const or_params* p, or_consts* c) {
    memset(c, 0, sizeof *c);
    if (p->grid_w == 0 || p->grid_h == 0 || p->neurons_per_module == 0) {
        set_err("empty grid");
        return -1;
    }
    if (!(p->spacing_um > 0.0f) || !(p->dt > 0.0f) || !(p->tau_m > 0.0f) || !(p->tau_c > 0.0f)) {
        set_err("spacing, dt, tau_m and tau_c must be positive");
        return -1;
    }
    if (p->kernel != 0 && p->kernel != 1) {
        set_err("kernel must be 0 (Gaussian) or 1 (exponential)");
        return -1;
    }
    if ((p->kernel == 0 && !(p->sigma_um > 0.0)) || (p->kernel == 1 && !(p->lambda_um > 0.0))) {
        set_err("kernel length scale must be positive");
        return -1;
    }
    if (!(p->cutoff_um >= 0.0)) {
        set_err("cutoff must be non-negative");
        return -1;
    }
    if (p->d_exc_lo < 1 || p->d_exc_hi < p->d_exc_lo || p->d_inh < 1 || p->d_exc_hi > 255 ||
        p->d_inh > 255) {
        set_err("delays must satisfy 1 <= lo <= hi <= 255");
        return -1;
    }
    if (p->conn_rule != 0 && p->conn_rule != 1) {
        set_err("conn_rule must be 0 or 1");
        return -1;
    }
    if (p->conn_rule == 1 &&
        (!(p->p_local >= 0.0f && p->p_local <= 1.0f) || !(p->A_remote >= 0.0 && p->A_remote <= 1.0) ||
         !(p->p_min > 0.0 && p->p_min < 1.0))) {
        set_err("rule 1 needs 0 <= p_local <= 1, 0 <= A_remote <= 1, 0 < p_min < 1");
        return -1;
    }
    if ((p->weight_dist != 0 && p->weight_dist != 1) || !(p->w_exc_sd >= 0.0f) || !(p->w_inh_sd >= 0.0f)) {
        set_err("weight_dist must be 0 or 1 with non-negative deviations");
        return -1;
    }
    if ((p->delay_dist != 0 && p->delay_dist != 1) || (p->delay_dist == 1 && !(p->delay_tau_ms > 0.0f))) {
        set_err("delay_dist must be 0 or 1, with delay_tau_ms > 0 for 1");
        return -1;
    }
    if (p->fx_shift < 8 || p->fx_shift > 24) {
        set_err("fx_shift must be in [8, 24]");
        return -1;
    }
    if (p->stdp && (!(p->stdp_tau_plus_ms > 0.0f) || !(p->stdp_tau_minus_ms > 0.0f) ||
                    !(p->stdp_w_max >= 0.0f) || p->stdp_period_steps == 0 || p->weight_bf16)) {
        set_err("stdp needs positive time constants, w_max >= 0, a period >= 1 and f32 weights");
        return -1;
    }
    uint64_t N = (uint64_t)p->grid_w * p->grid_h * p->neurons_per_module;
    if (N > 0xFFFFFFF0ull) {
        set_err("too many neurons");
        return -1;
    }
    c->N = (uint32_t)N;
    c->n_modules = p->grid_w * p->grid_h;
    double ne = floor((double)p->exc_fraction * (double)p->neurons_per_module + 0.5);
    if (ne < 0.0) ne = 0.0;
    if (ne > (double)p->neurons_per_module) ne = (double)p->neurons_per_module;
    c->n_exc = (uint32_t)ne;
    uint32_t dmax = p->d_exc_hi > p->d_inh ? p->d_exc_hi : p->d_inh;
    c->D = dmax + 1u;
    c->ref_steps = (uint32_t)lround((double)p->t_ref / (double)p->dt);

    double q = p->cutoff_um / (double)p->spacing_um;
    c->R2 = (uint32_t)floor(q * q + 1e-9);
    uint32_t R = 0;
    while ((R + 1) * (R + 1) <= c->R2) ++R;
    uint32_t cnt = 0;
    for (int32_t dy = -(int32_t)R; dy <= (int32_t)R; ++dy)
        for (int32_t dx = -(int32_t)R; dx <= (int32_t)R; ++dx)
            if ((uint32_t)(dx * dx + dy * dy) <= c->R2) ++cnt;
    c->max_offsets = cnt;

    double dt = (double)p->dt, tm = (double)p->tau_m, tc = (double)p->tau_c;
    double em = exp(-dt / tm);
    double ec = exp(-dt / tc);
    c->a_m = (float)em;
    c->a_c = (float)ec;
    double kc;
    if (tc == tm)
        kc = (double)p->g_c * dt * em;
    else
        kc = (double)p->g_c * (tm * tc / (tc - tm)) * (ec - em);
    c->kc = (float)kc;

    float scale = ldexpf(1.0f, (int)p->fx_shift);
    c->J_ext_fx = (int32_t)lrintf(p->J_ext * scale);

    double lam = (double)p->ext_rate_hz * dt / 1000.0;
    c->pois_len = 0;
    if (lam < 0.0) {
        set_err("negative external rate");
        return -1;
    }
    if (lam > 0.0) {
        double pk = exp(-lam), cdf = 0.0;
        for (uint32_t k = 0; k < 64; ++k) {
            cdf = cdf + pk;
            double x = floor(cdf * 4294967296.0);
            if (x >= 4294967295.0) break;
            c->pois[c->pois_len++] = (uint64_t)x;
            pk = pk * lam / (double)(k + 1);
        }
        if (c->pois_len == 64) {
            set_err("external rate too high for the Poisson table");
            return -1;
        }
    }
    double pf = (double)p->imposed_rate_hz * dt / 1000.0;
    if (pf < 0.0) pf = 0.0;
    if (pf > 1.0) pf = 1.0;
    c->imposed_thresh = (uint64_t)floor(pf * 4294967296.0);
    c->n_pair_offsets = 0;
    if (p->conn_rule == 1) {
        uint32_t n = 0;
        if (or_pair_stencil(p, NULL, NULL, NULL, NULL, 0, &n)) return -1;
        c->n_pair_offsets = n;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Lateral kernels (Sec. I and Sec. III-B): Gaussian B exp(-r^2 / 2 sigma^2),
 * exponential A exp(-r / lambda); r = spacing * grid distance.  The
 * normalisation constants A and B are 1 / (sum over the stencil). */
static double kernel_value(const or_params* p, uint32_t d2) {
    double s = (double)p->spacing_um;
    if (p->kernel == 0) {
        double num = (double)d2 * s * s;
        double den = 2.0 * p->sigma_um * p->sigma_um;
        return exp(-(num / den));
    }
    double r = s * sqrt((double)d2);
    return exp(-(r / p->lambda_um));
}

int or_cdf_table(const or_params* p, uint32_t module, uint32_t* thresh, uint32_t* tgt_module,
                 double* prob, uint32_t cap, uint32_t* n_out) {
    or_consts c;
    if (or_constants(p, &c)) return -1;
    if (module >= c.n_modules) {
        set_err("module out of range");
        return -1;
    }
    double* pre = (double*)malloc(sizeof(double) * (c.max_offsets + 1));
    double* f = (double*)malloc(sizeof(double) * (c.max_offsets + 1));
    uint32_t* tg = (uint32_t*)malloc(sizeof(uint32_t) * (c.max_offsets + 1));
    if (!pre || !f || !tg) {
        free(pre); free(f); free(tg);
        set_err("out of memory");
        return -1;
    }
    int32_t sx = (int32_t)(module % p->grid_w), sy = (int32_t)(module / p->grid_w);
    uint32_t R = 0;
    while ((R + 1) * (R + 1) <= c.R2) ++R;
    uint32_t n = 0;
    double P = 0.0;
    for (int32_t dy = -(int32_t)R; dy <= (int32_t)R; ++dy) {
        for (int32_t dx = -(int32_t)R; dx <= (int32_t)R; ++dx) {
            uint32_t d2 = (uint32_t)(dx * dx + dy * dy);
            if (d2 > c.R2) continue;
            int32_t tx = sx + dx, ty = sy + dy;
            if (tx < 0 || ty < 0 || tx >= (int32_t)p->grid_w || ty >= (int32_t)p->grid_h) continue;
            f[n] = kernel_value(p, d2);
            P = P + f[n];
            pre[n] = P;
            tg[n] = (uint32_t)ty * p->grid_w + (uint32_t)tx;
            ++n;
        }
    }
    if (n > cap) {
        free(pre); free(f); free(tg);
        set_err("table capacity too small");
        return -1;
    }
    double S = pre[n - 1];
    for (uint32_t j = 0; j < n; ++j) {
        uint32_t T = 0xFFFFFFFFu;
        if (j + 1 < n) {
            double x = floor(pre[j] / S * 4294967296.0);
            T = x >= 4294967295.0 ? 0xFFFFFFFFu : (uint32_t)x;
        }
        thresh[j] = T;
        tgt_module[j] = tg[j];
        if (prob) prob[j] = f[j] / S;
    }
    *n_out = n;
    free(pre); free(f); free(tg);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* The per-pair law (Sec. III-B).  The stencil radius grows while the pair
 * probability on an axis still exceeds p_min (f decreases with r). */
int or_pair_stencil(const or_params* p, int32_t* dx, int32_t* dy, double* prob, uint64_t* thresh,
                    uint32_t cap, uint32_t* n_out) {
    if (p->conn_rule != 1) {
        set_err("the pair stencil belongs to conn_rule 1");
        return -1;
    }
    uint32_t R = 0;
    while (R < 4096 && p->A_remote * kernel_value(p, (R + 1) * (R + 1)) > p->p_min) ++R;
    uint32_t n = 0;
    for (int32_t y = -(int32_t)R; y <= (int32_t)R; ++y) {
        for (int32_t x = -(int32_t)R; x <= (int32_t)R; ++x) {
            double pr;
            if (x == 0 && y == 0)
                pr = (double)p->p_local;
            else {
                pr = p->A_remote * kernel_value(p, (uint32_t)(x * x + y * y));
                if (!(pr > p->p_min)) continue;
            }
            if (dx) {
                if (n >= cap) {
                    set_err("stencil capacity too small");
                    return -1;
                }
                dx[n] = x;
                dy[n] = y;
                if (prob) prob[n] = pr;
                if (thresh) thresh[n] = pr >= 1.0 ? 4294967296ull : (uint64_t)floor(pr * 4294967296.0);
            }
            ++n;
        }
    }
    *n_out = n;
    return 0;
}

/* Standard normal CDF and its inverse by bisection to the resolution of a
 * double (slow, but only 4096 values per table). */
static double std_normal_cdf(double x) { return 0.5 * erfc(-x / sqrt(2.0)); }

static double std_normal_quantile(double q) {
    double lo = -40.0, hi = 40.0;
    for (int it = 0; it < 4000; ++it) {
        double mid = 0.5 * (lo + hi);
        if (!(mid > lo && mid < hi)) break;
        if (std_normal_cdf(mid) < q)
            lo = mid;
        else
            hi = mid;
    }
    return fabs(std_normal_cdf(lo) - q) <= fabs(std_normal_cdf(hi) - q) ? lo : hi;
}

int or_weight_table(const or_params* p, int exc, float* tab, double* tab64) {
    double mean = exc ? 0.5 * ((double)p->w_exc_lo + (double)p->w_exc_hi) : (double)p->w_inh;
    double sd = exc ? (double)p->w_exc_sd : (double)p->w_inh_sd;
    for (uint32_t k = 0; k < OR_WTAB; ++k) {
        double z = std_normal_quantile(((double)k + 0.5) / (double)OR_WTAB);
        double w = mean + sd * z;
        if (exc && w < 0.0) w = 0.0; /* an efficacy keeps the sign of its population */
        if (!exc && w > 0.0) w = 0.0;
        if (tab) tab[k] = (float)w;
        if (tab64) tab64[k] = w;
    }
    return 0;
}

/* P(delay <= d_lo + k) = (1 - e^{-(k+1)/tau}) / (1 - e^{-span/tau}), tau in steps. */
int or_delay_table(const or_params* p, uint64_t* thr, uint32_t* n_out) {
    uint32_t span = p->d_exc_hi - p->d_exc_lo + 1u;
    double tau = (double)p->delay_tau_ms / (double)p->dt;
    if (!(tau > 0.0)) {
        set_err("delay_tau_ms must be positive");
        return -1;
    }
    double Z = 1.0 - exp(-(double)span / tau);
    for (uint32_t k = 0; k + 1 < span; ++k) {
        double F = (1.0 - exp(-(double)(k + 1) / tau)) / Z;
        double x = floor(F * 4294967296.0);
        thr[k] = x >= 4294967296.0 ? 4294967296ull : (uint64_t)x;
    }
    *n_out = span - 1u;
    return 0;
}

/* ------------------------------------------------------------------------ */
int or_lif_update(const or_consts* c, const or_params* p, float* V, float* cf, uint8_t* ref,
                  int exc, int32_t I_fx, int forced) {
    int was_ref = *ref > 0;
    if (was_ref) {
        *ref = (uint8_t)(*ref - 1);
        *V = p->V_reset;
    } else {
        /* exact propagator of Eq. 1-2 over dt, then this step's jumps */
        float v = *V - p->E;
        v = v * c->a_m;
        v = v + p->E;
        float adapt = c->kc * *cf;
        v = v - adapt;
        float inp = (float)I_fx * ldexpf(1.0f, -(int)p->fx_shift);
        v = v + inp;
        *V = v;
    }
    *cf = *cf * c->a_c;
    int spike = !was_ref && (*V > p->V_th || forced);
    if (spike) {
        *V = p->V_reset;
        *ref = (uint8_t)c->ref_steps;
        if (exc) *cf = *cf + p->alpha_c;
    }
    return spike;
}

int or_constants64(const or_params* p, or_consts64* k) {
    if (!(p->dt > 0.0f) || !(p->tau_m > 0.0f) || !(p->tau_c > 0.0f)) {
        set_err("dt, tau_m and tau_c must be positive");
        return -1;
    }
    double dt = (double)p->dt, tm = (double)p->tau_m, tc = (double)p->tau_c;
    k->a_m = exp(-dt / tm);
    k->a_c = exp(-dt / tc);
    k->kc = tc == tm ? (double)p->g_c * dt * k->a_m : (double)p->g_c * (tm * tc / (tc - tm)) * (k->a_c - k->a_m);
    return 0;
}

int or_lif_update64(const or_consts64* k, const or_params* p, uint32_t ref_steps, double* V, double* c,
                    uint8_t* ref, int exc, double I, int forced) {
    int was_ref = *ref > 0;
    if (was_ref) {
        *ref = (uint8_t)(*ref - 1);
        *V = (double)p->V_reset;
    } else {
        /* exact propagator of Eq. 1-2 over dt, then this step's jumps */
        double E = (double)p->E;
        *V = ((*V - E) * k->a_m + E) - k->kc * *c + I;
    }
    *c = *c * k->a_c;
    int spike = !was_ref && (*V > (double)p->V_th || forced);
    if (spike) {
        *V = (double)p->V_reset;
        *ref = (uint8_t)ref_steps;
        if (exc) *c = *c + (double)p->alpha_c;
    }
    return spike;
}

uint32_t or_poisson_count(const or_consts* c, uint32_t u0) {
    uint32_t n = 0;
    for (uint32_t k = 0; k < c->pois_len; ++k)
        if (c->pois[k] <= (uint64_t)u0) ++n;
    return n;
}

/* ------------------------------------------------------------------------ */
struct or_net {
    or_params p;
    or_consts c;
    int fp64;
    uint32_t N, M;
    uint64_t nsyn;
    uint64_t* row_ptr;  /* N + 1 row offsets */
    uint32_t* tgt;
    float* w;
    double* w64;
    uint8_t* d;
    float* V;
    float* cf;
    double* V64;
    double* c64;
    uint8_t* ref;
    int64_t* ring;
    double* ring64;
    uint32_t t;
    uint32_t* spk;
    uint32_t* rst_t;
    uint32_t* rst_id;
    uint64_t rst_n, rst_cap;
    uint64_t n_spikes, rec, ext;
    uint64_t shuffle_seed;
    or_consts64 k64;  /* FP64 mode: propagator constants in double */
    /* STDP */
    float sa_p, sa_m;     /* trace decays exp(-dt/tau_plus), exp(-dt/tau_minus) */
    float* sy;            /* post-synaptic trace of every neuron */
    float* sx;            /* pre-synaptic trace of every neuron */
    float* sxh;           /* sx of the last D + 1 steps, row t % (D + 1) */
    int64_t* sdelta;      /* accumulated change of every synapse, 2^-16 mV */
    uint64_t* in_ptr;     /* synapses targeting neuron j: in_syn[in_ptr[j] .. in_ptr[j + 1]) */
    uint64_t* in_syn;
    uint64_t** arr;       /* arrival lists, one per ring slot (flow step 3) */
    uint64_t* arr_n;
    uint64_t* arr_cap;
};

static int is_exc(const or_net* n, uint32_t i) { return (i % n->M) < n->c.n_exc; }

void or_destroy(or_net* n) {
    if (!n) return;
    free(n->row_ptr); free(n->tgt); free(n->w); free(n->w64); free(n->d);
    free(n->V); free(n->cf); free(n->V64); free(n->c64); free(n->ref);
    free(n->ring); free(n->ring64); free(n->spk); free(n->rst_t); free(n->rst_id);
    free(n->sy); free(n->sx); free(n->sxh); free(n->sdelta); free(n->in_ptr); free(n->in_syn);
    if (n->arr)
        for (uint32_t k = 0; k < n->c.D; ++k) free(n->arr[k]);
    free(n->arr); free(n->arr_n); free(n->arr_cap);
    free(n);
}

/* What synapse generation needs besides the description: the target-module
 * tables (rule 0) or the pair stencil (rule 1), and the efficacy and delay
 * tables of the chosen distributions. */
typedef struct gen_ctx {
    const or_params* p;
    const or_consts* c;
    uint32_t cap;                 /* rule 0: table entries per module */
    uint32_t *T, *TM, *cnt;       /* rule 0: per-module thresholds, targets, sizes */
    uint32_t ns;                  /* rule 1: stencil size */
    int32_t *sdx, *sdy;           /* rule 1: stencil offsets */
    uint64_t* sthr;               /* rule 1: pair thresholds */
    float *wt_e, *wt_i;           /* Gaussian efficacy tables */
    double *wt64_e, *wt64_i;
    uint64_t dthr[256];           /* exponential delay thresholds */
    uint32_t n_dthr;
} gen_ctx;

static void gen_free(gen_ctx* g) {
    free(g->T); free(g->TM); free(g->cnt); free(g->sdx); free(g->sdy); free(g->sthr);
    free(g->wt_e); free(g->wt_i); free(g->wt64_e); free(g->wt64_i);
    memset(g, 0, sizeof *g);
}

/* Prepares generation of rows [first, first + count). */
static int gen_init(gen_ctx* g, const or_params* p, const or_consts* c, uint32_t first, uint32_t count) {
    memset(g, 0, sizeof *g);
    g->p = p;
    g->c = c;
    uint32_t M = p->neurons_per_module, nm = c->n_modules;
    if (p->conn_rule == 0) {
        g->cap = c->max_offsets;
        g->T = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)g->cap * nm);
        g->TM = (uint32_t*)malloc(sizeof(uint32_t) * (size_t)g->cap * nm);
        g->cnt = (uint32_t*)calloc(nm, sizeof(uint32_t));
        if (!g->T || !g->TM || !g->cnt) goto oom;
        uint32_t m0 = first / M, m1 = count ? (first + count - 1) / M : m0;
        for (uint32_t m = m0; m <= m1 && m < nm; ++m)
            if (or_cdf_table(p, m, g->T + (size_t)m * g->cap, g->TM + (size_t)m * g->cap, NULL, g->cap,
                             &g->cnt[m])) {
                gen_free(g);
                return -1;
            }
    } else {
        g->ns = c->n_pair_offsets;
        g->sdx = (int32_t*)malloc(sizeof(int32_t) * g->ns);
        g->sdy = (int32_t*)malloc(sizeof(int32_t) * g->ns);
        g->sthr = (uint64_t*)malloc(sizeof(uint64_t) * g->ns);
        if (!g->sdx || !g->sdy || !g->sthr) goto oom;
        uint32_t n = 0;
        if (or_pair_stencil(p, g->sdx, g->sdy, NULL, g->sthr, g->ns, &n)) {
            gen_free(g);
            return -1;
        }
    }
    if (p->weight_dist == 1) {
        g->wt_e = (float*)malloc(sizeof(float) * OR_WTAB);
        g->wt_i = (float*)malloc(sizeof(float) * OR_WTAB);
        g->wt64_e = (double*)malloc(sizeof(double) * OR_WTAB);
        g->wt64_i = (double*)malloc(sizeof(double) * OR_WTAB);
        if (!g->wt_e || !g->wt_i || !g->wt64_e || !g->wt64_i) goto oom;
        or_weight_table(p, 1, g->wt_e, g->wt64_e);
        or_weight_table(p, 0, g->wt_i, g->wt64_i);
    }
    if (p->delay_dist == 1 && or_delay_table(p, g->dthr, &g->n_dthr)) {
        gen_free(g);
        return -1;
    }
    return 0;
oom:
    gen_free(g);
    set_err("out of memory");
    return -1;
}

/* Efficacy and delay of one synapse from words u2 (efficacy) and u3 (delay)
 * of its Philox block. */
static void syn_attr(const gen_ctx* g, int exc, const uint32_t u[4], float* w, double* w64, uint8_t* d) {
    const or_params* p = g->p;
    if (exc) {
        if (p->delay_dist == 0) {
            uint32_t dspan = p->d_exc_hi - p->d_exc_lo + 1u;
            *d = (uint8_t)(p->d_exc_lo + (uint32_t)(((uint64_t)u[3] * dspan) >> 32));
        } else {
            uint32_t k = 0;
            for (uint32_t j = 0; j < g->n_dthr; ++j)
                if (g->dthr[j] <= (uint64_t)u[3]) ++k;
            *d = (uint8_t)(p->d_exc_lo + k);
        }
        if (p->weight_dist == 0) {
            if (w64) {
                double lo = (double)p->w_exc_lo, hi = (double)p->w_exc_hi;
                *w64 = lo + (hi - lo) * unit24d(u[2]);
            } else {
                float x = (p->w_exc_hi - p->w_exc_lo) * unit24(u[2]);
                *w = p->w_exc_lo + x;
            }
        } else {
            if (w64)
                *w64 = g->wt64_e[u[2] >> 20];
            else
                *w = g->wt_e[u[2] >> 20];
        }
    } else {
        *d = (uint8_t)p->d_inh;
        if (p->weight_dist == 0) {
            if (w64)
                *w64 = (double)p->w_inh;
            else
                *w = p->w_inh;
        } else {
            if (w64)
                *w64 = g->wt64_i[u[2] >> 20];
            else
                *w = g->wt_i[u[2] >> 20];
        }
    }
    if (!w64 && p->weight_bf16) *w = or_bf16_to_float(or_bf16_bits(*w));
}

/* Row of neuron i (Sec. II-B), written at out[0 ..).  Rule 0: synapse k draws
 * one Philox block (i, k, GEN); u0 picks the target module by inverse CDF, u1
 * the neuron inside it.  Rule 1: for every stencil offset (index o) inside
 * the grid and every neuron j of that module, word j % 4 of the block
 * (i, o * ceil(M/4) + j / 4, CONN) below the pair threshold makes a synapse;
 * the k-th synapse of the row takes its efficacy and delay from words u2, u3
 * of block (i, k, GEN) in both rules.  Returns the row length, or -1 if it
 * would pass `cap` (a NULL tgt only counts). */
static int64_t gen_row(const gen_ctx* g, uint32_t i, uint64_t cap, uint32_t* tgt, float* w, double* w64,
                       uint8_t* d) {
    const or_params* p = g->p;
    uint32_t M = p->neurons_per_module;
    uint32_t s = i / M;
    int exc = (i % M) < g->c->n_exc;
    if (p->conn_rule == 0) {
        if ((uint64_t)p->K > cap) return -1;
        const uint32_t* Ts = g->T + (size_t)s * g->cap;
        const uint32_t* TMs = g->TM + (size_t)s * g->cap;
        uint32_t ns = g->cnt[s];
        for (uint32_t k = 0; k < p->K; ++k) {
            uint32_t u[4];
            draw(p, i, k, OR_TAG_GEN, u);
            if (!tgt) continue;
            uint32_t j = 0;
            while (j + 1 < ns && Ts[j] <= u[0]) ++j; /* first entry with u0 < T */
            tgt[k] = TMs[j] * M + (uint32_t)(((uint64_t)u[1] * M) >> 32);
            syn_attr(g, exc, u, w ? w + k : NULL, w64 ? w64 + k : NULL, d + k);
        }
        return p->K;
    }
    int32_t sx = (int32_t)(s % p->grid_w), sy = (int32_t)(s / p->grid_w);
    uint32_t a = i % M, c4 = (M + 3u) / 4u;
    uint64_t k = 0;
    for (uint32_t o = 0; o < g->ns; ++o) {
        int local = g->sdx[o] == 0 && g->sdy[o] == 0;
        if (!exc && p->inh_local_only && !local) continue;
        int32_t tx = sx + g->sdx[o], ty = sy + g->sdy[o];
        if (tx < 0 || ty < 0 || tx >= (int32_t)p->grid_w || ty >= (int32_t)p->grid_h) continue;
        uint32_t base = ((uint32_t)ty * p->grid_w + (uint32_t)tx) * M;
        for (uint32_t j = 0; j < M; ++j) {
            if (local && j == a) continue; /* no autapse */
            uint32_t u[4];
            draw(p, i, o * c4 + j / 4u, OR_TAG_CONN, u);
            if ((uint64_t)u[j % 4u] >= g->sthr[o]) continue;
            if (k >= cap) return -1;
            if (tgt) {
                uint32_t v[4];
                draw(p, i, (uint32_t)k, OR_TAG_GEN, v);
                tgt[k] = base + j;
                syn_attr(g, exc, v, w ? w + k : NULL, w64 ? w64 + k : NULL, d + k);
            }
            ++k;
        }
    }
    return (int64_t)k;
}

static int grow(or_net* n, uint64_t need) {
    uint64_t cap = n->nsyn ? n->nsyn : 1;
    if (need <= cap) return 0;
    while (cap < need) cap *= 2;
    uint32_t* t = (uint32_t*)realloc(n->tgt, sizeof(uint32_t) * cap);
    if (!t) return -1;
    n->tgt = t;
    uint8_t* d = (uint8_t*)realloc(n->d, cap);
    if (!d) return -1;
    n->d = d;
    if (n->fp64) {
        double* w = (double*)realloc(n->w64, sizeof(double) * cap);
        if (!w) return -1;
        n->w64 = w;
    } else {
        float* w = (float*)realloc(n->w, sizeof(float) * cap);
        if (!w) return -1;
        n->w = w;
    }
    n->nsyn = cap; /* capacity while generating; set to the total afterwards */
    return 0;
}

/* The whole table, rows back to back. */
static int generate(or_net* n) {
    gen_ctx g;
    if (gen_init(&g, &n->p, &n->c, 0, n->N)) return -1;
    uint64_t used = 0;
    int rc = 0;
    n->row_ptr[0] = 0;
    for (uint32_t i = 0; i < n->N && rc == 0; ++i) {
        for (;;) {
            uint64_t room = n->nsyn - used;
            int64_t len = gen_row(&g, i, room, n->tgt + used, n->w ? n->w + used : NULL,
                                  n->w64 ? n->w64 + used : NULL, n->d + used);
            if (len >= 0) {
                used += (uint64_t)len;
                break;
            }
            if (grow(n, n->nsyn + (uint64_t)n->M * g.ns + n->p.K + 1)) {
                set_err("out of memory");
                rc = -1;
                break;
            }
        }
        n->row_ptr[i + 1] = used;
    }
    gen_free(&g);
    n->nsyn = used;
    return rc;
}

int or_gen_rows_v(const or_params* p, uint32_t first, uint32_t count, uint64_t cap, uint32_t* tgt,
                  float* w, uint8_t* d, uint32_t* len) {
    or_consts c;
    if (or_constants(p, &c)) return -1;
    if ((uint64_t)first + count > c.N) {
        set_err("rows out of range");
        return -1;
    }
    gen_ctx g;
    if (gen_init(&g, p, &c, first, count)) return -1;
    uint64_t used = 0;
    for (uint32_t r = 0; r < count; ++r) {
        int64_t n = gen_row(&g, first + r, cap - used, tgt + used, w + used, NULL, d + used);
        if (n < 0) {
            gen_free(&g);
            set_err("row capacity too small");
            return -1;
        }
        len[r] = (uint32_t)n;
        used += (uint64_t)n;
    }
    gen_free(&g);
    return 0;
}

int or_gen_rows_list(const or_params* p, const uint32_t* ids, uint32_t count, uint64_t cap, uint32_t* tgt,
                     float* w, uint8_t* d, uint32_t* len) {
    or_consts c;
    if (or_constants(p, &c)) return -1;
    for (uint32_t r = 0; r < count; ++r)
        if (ids[r] >= c.N) {
            set_err("row out of range");
            return -1;
        }
    gen_ctx g;
    if (gen_init(&g, p, &c, 0, c.N)) return -1;
    uint64_t used = 0;
    for (uint32_t r = 0; r < count; ++r) {
        int64_t n = gen_row(&g, ids[r], cap - used, tgt + used, w + used, NULL, d + used);
        if (n < 0) {
            gen_free(&g);
            set_err("row capacity too small");
            return -1;
        }
        len[r] = (uint32_t)n;
        used += (uint64_t)n;
    }
    gen_free(&g);
    return 0;
}

int or_gen_rows(const or_params* p, uint32_t first, uint32_t count, uint32_t* tgt, float* w,
                uint8_t* d) {
    if (p->conn_rule != 0) {
        set_err("rows of variable length: use or_gen_rows_v");
        return -1;
    }
    uint32_t* len = (uint32_t*)malloc(sizeof(uint32_t) * (count ? count : 1));
    if (!len) {
        set_err("out of memory");
        return -1;
    }
    int r = or_gen_rows_v(p, first, count, (uint64_t)count * p->K, tgt, w, d, len);
    free(len);
    return r;
}

float or_initial_V(const or_params* p, uint32_t i) {
    uint32_t u[4];
    draw(p, i, 0u, OR_TAG_INIT, u);
    return p->V_th * unit24(u[0]);
}

void or_drive(const or_params* p, const or_consts* c, uint32_t i, uint32_t t, uint32_t* n_ext,
              int* forced) {
    uint32_t u[4];
    draw(p, i, t, OR_TAG_DRIVE, u);
    *n_ext = or_poisson_count(c, u[0]);
    *forced = (uint64_t)u[1] < c->imposed_thresh;
}

/* STDP state: traces, their history, the change accumulators, the arrival
 * lists and, for the potentiation at a post-synaptic spike, every neuron's
 * incoming synapses (a target-major index of the CSR). */
static int stdp_setup(or_net* n) {
    const or_params* p = &n->p;
    if (n->fp64) {
        set_err("stdp is not modelled in the FP64 mode");
        return -1;
    }
    double dt = (double)p->dt;
    n->sa_p = (float)exp(-dt / (double)p->stdp_tau_plus_ms);
    n->sa_m = (float)exp(-dt / (double)p->stdp_tau_minus_ms);
    uint32_t D = n->c.D;
    n->sy = (float*)calloc(n->N, sizeof(float));
    n->sx = (float*)calloc(n->N, sizeof(float));
    n->sxh = (float*)calloc((size_t)(D + 1) * n->N, sizeof(float));
    n->sdelta = (int64_t*)calloc(n->nsyn, sizeof(int64_t));
    n->in_ptr = (uint64_t*)calloc((size_t)n->N + 1, sizeof(uint64_t));
    n->in_syn = (uint64_t*)malloc(sizeof(uint64_t) * (n->nsyn ? n->nsyn : 1));
    n->arr = (uint64_t**)calloc(D, sizeof(uint64_t*));
    n->arr_n = (uint64_t*)calloc(D, sizeof(uint64_t));
    n->arr_cap = (uint64_t*)calloc(D, sizeof(uint64_t));
    if (!n->sy || !n->sx || !n->sxh || !n->sdelta || !n->in_ptr || !n->in_syn || !n->arr || !n->arr_n || !n->arr_cap) {
        set_err("out of memory");
        return -1;
    }
    uint64_t total = n->row_ptr[n->N];
    for (uint64_t e = 0; e < total; ++e) n->in_ptr[n->tgt[e] + 1] += 1;
    for (uint32_t j = 0; j < n->N; ++j) n->in_ptr[j + 1] += n->in_ptr[j];
    uint64_t* fill = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n->N + 1));
    if (!fill) {
        set_err("out of memory");
        return -1;
    }
    memcpy(fill, n->in_ptr, sizeof(uint64_t) * ((size_t)n->N + 1));
    for (uint64_t e = 0; e < total; ++e) n->in_syn[fill[n->tgt[e]]++] = e;
    free(fill);
    return 0;
}

static int arrival_push(or_net* n, uint32_t slot, uint64_t e) {
    if (n->arr_n[slot] == n->arr_cap[slot]) {
        uint64_t nc = n->arr_cap[slot] ? 2 * n->arr_cap[slot] : 1024;
        uint64_t* a = (uint64_t*)realloc(n->arr[slot], sizeof(uint64_t) * nc);
        if (!a) return -1;
        n->arr[slot] = a;
        n->arr_cap[slot] = nc;
    }
    n->arr[slot][n->arr_n[slot]++] = e;
    return 0;
}

static uint32_t source_of(const or_net* n, uint64_t e) {
    uint32_t lo = 0, hi = n->N;  /* the row holding synapse e: row_ptr[lo] <= e < row_ptr[lo + 1] */
    while (hi - lo > 1) {
        uint32_t mid = (lo + hi) / 2;
        if (n->row_ptr[mid] <= e)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

/* The plasticity of step t, after every neuron has been updated (its spikes
 * are spk[0 .. nspk)): traces, depression at this step's arrivals, then
 * potentiation at this step's post-synaptic spikes. */
static void stdp_step(or_net* n, uint32_t t, uint32_t nspk) {
    const or_params* p = &n->p;
    uint32_t D = n->c.D;
    float scale = ldexpf(1.0f, 16);
    for (uint32_t i = 0; i < n->N; ++i) {
        n->sy[i] = n->sy[i] * n->sa_m;
        n->sx[i] = n->sx[i] * n->sa_p;
    }
    for (uint32_t s = 0; s < nspk; ++s) {
        n->sy[n->spk[s]] = n->sy[n->spk[s]] + 1.0f;
        n->sx[n->spk[s]] = n->sx[n->spk[s]] + 1.0f;
    }
    memcpy(n->sxh + (size_t)(t % (D + 1)) * n->N, n->sx, sizeof(float) * n->N);
    /* flow step 4: each arrival of this step against the post-synaptic trace,
     * which includes a spike of this step */
    uint32_t slot = t % D;
    for (uint64_t k = 0; k < n->arr_n[slot]; ++k) {
        uint64_t e = n->arr[slot][k];
        float c = p->stdp_A_minus * n->sy[n->tgt[e]];
        n->sdelta[e] -= (int64_t)lrintf(c * scale);
    }
    n->arr_n[slot] = 0;
    /* flow step 1: each post-synaptic spike against the trace of the arrivals
     * strictly before it: x of the source d + 1 steps ago, decayed one step */
    for (uint32_t s = 0; s < nspk; ++s) {
        uint32_t j = n->spk[s];
        for (uint64_t q = n->in_ptr[j]; q < n->in_ptr[j + 1]; ++q) {
            uint64_t e = n->in_syn[q];
            uint32_t i = source_of(n, e);
            if (!is_exc(n, i)) continue;
            uint32_t d = n->d[e];
            if (t < d + 1) continue;  /* no arrival can precede the start */
            float xa = n->sxh[(size_t)((t - d - 1) % (D + 1)) * n->N + i] * n->sa_p;
            float c = p->stdp_A_plus * xa;
            n->sdelta[e] += (int64_t)lrintf(c * scale);
        }
    }
}

/* Every stdp_period_steps: the accumulated changes into the excitatory
 * weights (each change must fit an int32, the accumulator of the CUDA path). */
static int stdp_apply(or_net* n) {
    float inv = ldexpf(1.0f, -16);
    for (uint32_t i = 0; i < n->N; ++i) {
        if (!is_exc(n, i)) continue;
        for (uint64_t e = n->row_ptr[i]; e < n->row_ptr[i + 1]; ++e) {
            if (n->sdelta[e] > INT32_MAX || n->sdelta[e] < INT32_MIN) {
                set_err("stdp change overflows int32");
                return -1;
            }
            float w = n->w[e] + (float)n->sdelta[e] * inv;
            if (w < 0.0f) w = 0.0f;
            if (w > n->p.stdp_w_max) w = n->p.stdp_w_max;
            n->w[e] = w;
            n->sdelta[e] = 0;
        }
    }
    return 0;
}

void or_get_stdp(const or_net* n, int64_t* delta, float* y, float* x) {
    if (delta && n->sdelta) memcpy(delta, n->sdelta, sizeof(int64_t) * n->row_ptr[n->N]);
    if (y && n->sy) memcpy(y, n->sy, sizeof(float) * n->N);
    if (x && n->sx) memcpy(x, n->sx, sizeof(float) * n->N);
}

or_net* or_create(const or_params* p, int fp64) {
    or_consts c;
    if (or_constants(p, &c)) return NULL;
    or_net* n = (or_net*)calloc(1, sizeof *n);
    if (!n) {
        set_err("out of memory");
        return NULL;
    }
    n->p = *p;
    n->c = c;
    n->fp64 = fp64 ? 1 : 0;
    n->N = c.N;
    n->M = p->neurons_per_module;
    n->nsyn = p->conn_rule == 0 ? (uint64_t)n->N * p->K : (uint64_t)n->N * 64u;
    size_t ns = (size_t)n->nsyn ? (size_t)n->nsyn : 1;
    n->nsyn = ns;
    n->row_ptr = (uint64_t*)malloc(sizeof(uint64_t) * ((size_t)n->N + 1));
    n->tgt = (uint32_t*)malloc(sizeof(uint32_t) * ns);
    n->d = (uint8_t*)malloc(ns);
    if (n->fp64)
        n->w64 = (double*)malloc(sizeof(double) * ns);
    else
        n->w = (float*)malloc(sizeof(float) * ns);
    n->ref = (uint8_t*)calloc(n->N, 1);
    n->spk = (uint32_t*)malloc(sizeof(uint32_t) * n->N);
    if (n->fp64) {
        n->V64 = (double*)malloc(sizeof(double) * n->N);
        n->c64 = (double*)calloc(n->N, sizeof(double));
        n->ring64 = (double*)calloc((size_t)c.D * n->N, sizeof(double));
    } else {
        n->V = (float*)malloc(sizeof(float) * n->N);
        n->cf = (float*)calloc(n->N, sizeof(float));
        n->ring = (int64_t*)calloc((size_t)c.D * n->N, sizeof(int64_t));
    }
    if (!n->row_ptr || !n->tgt || !n->d || (!n->w && !n->w64) || !n->ref || !n->spk ||
        (n->fp64 ? (!n->V64 || !n->c64 || !n->ring64) : (!n->V || !n->cf || !n->ring))) {
        or_destroy(n);
        set_err("out of memory");
        return NULL;
    }
    if (generate(n)) {
        or_destroy(n);
        return NULL;
    }
    /* initial state (the paper is silent): V0 = V_th * U[0,1), c = 0, ring = 0 */
    for (uint32_t i = 0; i < n->N; ++i) {
        if (n->fp64) {
            uint32_t u[4];
            draw(p, i, 0u, OR_TAG_INIT, u);
            n->V64[i] = (double)p->V_th * unit24d(u[0]);
        } else {
            n->V[i] = or_initial_V(p, i);
        }
    }
    or_constants64(p, &n->k64);
    if (p->stdp && stdp_setup(n)) {
        or_destroy(n);
        return NULL;
    }
    return n;
}

uint64_t or_n_synapses(const or_net* n) { return n->nsyn; }

void or_get_row_ptr(const or_net* n, uint64_t* row_ptr) {
    memcpy(row_ptr, n->row_ptr, sizeof(uint64_t) * ((size_t)n->N + 1));
}

void or_get_csr(const or_net* n, uint32_t* tgt, float* w, uint8_t* d) {
    if (tgt) memcpy(tgt, n->tgt, sizeof(uint32_t) * n->nsyn);
    if (w && n->w) memcpy(w, n->w, sizeof(float) * n->nsyn);
    if (d) memcpy(d, n->d, n->nsyn);
}

void or_get_csr_f64(const or_net* n, double* w) {
    if (w && n->w64) memcpy(w, n->w64, sizeof(double) * n->nsyn);
}

void or_set_delivery_shuffle(or_net* n, uint64_t s) { n->shuffle_seed = s; }

/* splitmix64: only used to permute the delivery order in the order-independence check */
static uint64_t mix64(uint64_t* s) {
    uint64_t z = (*s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

static int raster_push(or_net* n, uint32_t t, uint32_t id) {
    if (n->rst_n == n->rst_cap) {
        uint64_t nc = n->rst_cap ? n->rst_cap * 2 : 4096;
        uint32_t* a = (uint32_t*)realloc(n->rst_t, sizeof(uint32_t) * nc);
        if (!a) return -1;
        n->rst_t = a;
        uint32_t* b = (uint32_t*)realloc(n->rst_id, sizeof(uint32_t) * nc);
        if (!b) return -1;
        n->rst_id = b;
        n->rst_cap = nc;
    }
    n->rst_t[n->rst_n] = t;
    n->rst_id[n->rst_n] = id;
    ++n->rst_n;
    return 0;
}

static int deliver_one(or_net* n, uint32_t t, uint32_t src, uint32_t k) {
    size_t e = (size_t)n->row_ptr[src] + k;
    uint32_t slot = (t + n->d[e]) % n->c.D;
    size_t r = (size_t)slot * n->N + n->tgt[e];
    /* flow step 3: plastic synapses are also queued for their arrival step */
    if (n->p.stdp && is_exc(n, src) && arrival_push(n, slot, e)) return -1;
    if (n->fp64) {
        n->ring64[r] += n->w64[e];
    } else {
        float scale = ldexpf(1.0f, (int)n->p.fx_shift);
        n->ring[r] += (int64_t)lrintf(n->w[e] * scale);
    }
    return 0;
}

static int step_once(or_net* n) {
    const or_params* p = &n->p;
    const or_consts* c = &n->c;
    uint32_t t = n->t;
    uint32_t slot = t % c->D;
    uint32_t nspk = 0;
    /* flow steps 4-6: inject the inputs queued for this step and integrate */
    for (uint32_t i = 0; i < n->N; ++i) {
        uint32_t next;
        int forced;
        or_drive(p, c, i, t, &next, &forced);
        int exc = is_exc(n, i);
        int spike;
        n->ext += next;
        size_t r = (size_t)slot * n->N + i;
        if (n->fp64) {
            double I = n->ring64[r] + (double)next * (double)p->J_ext;
            n->ring64[r] = 0.0;
            spike = or_lif_update64(&n->k64, p, c->ref_steps, &n->V64[i], &n->c64[i], &n->ref[i], exc, I, forced);
        } else {
            int64_t I = n->ring[r] + (int64_t)next * c->J_ext_fx;
            n->ring[r] = 0;
            if (I > INT32_MAX || I < INT32_MIN) {
                set_err("int32 fixed-point input overflow");
                return -1;
            }
            spike = or_lif_update(c, p, &n->V[i], &n->cf[i], &n->ref[i], exc, (int32_t)I, forced);
        }
        /* flow step 1: neurons that spiked in this step, in id order */
        if (spike) {
            n->spk[nspk++] = i;
            if (raster_push(n, t, i)) {
                set_err("out of memory");
                return -1;
            }
        }
    }
    n->n_spikes += nspk;
    if (n->p.stdp) stdp_step(n, t, nspk);
    uint64_t total = 0;
    for (uint32_t s = 0; s < nspk; ++s) total += n->row_ptr[n->spk[s] + 1] - n->row_ptr[n->spk[s]];
    n->rec += total;
    /* flow steps 2-3: queue every spike at its targets, in the slot of the
     * step at which it arrives (t + delay) */
    if (n->shuffle_seed == 0) {
        for (uint32_t s = 0; s < nspk; ++s) {
            uint32_t len = (uint32_t)(n->row_ptr[n->spk[s] + 1] - n->row_ptr[n->spk[s]]);
            for (uint32_t k = 0; k < len; ++k)
                if (deliver_one(n, t, n->spk[s], k)) {
                    set_err("out of memory");
                    return -1;
                }
        }
    } else {
        /* every (spike, synapse) event in a random order */
        uint64_t st = n->shuffle_seed ^ ((uint64_t)t << 32);
        uint32_t* src = (uint32_t*)malloc(sizeof(uint32_t) * (total ? total : 1));
        uint32_t* syn = (uint32_t*)malloc(sizeof(uint32_t) * (total ? total : 1));
        if (!src || !syn) {
            free(src);
            free(syn);
            set_err("out of memory");
            return -1;
        }
        uint64_t e = 0;
        for (uint32_t s = 0; s < nspk; ++s) {
            uint32_t len = (uint32_t)(n->row_ptr[n->spk[s] + 1] - n->row_ptr[n->spk[s]]);
            for (uint32_t k = 0; k < len; ++k, ++e) {
                src[e] = n->spk[s];
                syn[e] = k;
            }
        }
        for (e = total; e > 1; --e) {
            uint64_t j = mix64(&st) % e;
            uint32_t a = src[e - 1], b = syn[e - 1];
            src[e - 1] = src[j];
            syn[e - 1] = syn[j];
            src[j] = a;
            syn[j] = b;
        }
        int bad = 0;
        for (e = 0; e < total; ++e) bad |= deliver_one(n, t, src[e], syn[e]);
        free(src);
        free(syn);
        if (bad) {
            set_err("out of memory");
            return -1;
        }
    }
    /* the long-term plasticity of the period that ends with this step */
    if (n->p.stdp && (t + 1) % n->p.stdp_period_steps == 0 && stdp_apply(n)) return -1;
    n->t = t + 1;
    return 0;
}

int or_step(or_net* n, uint32_t n_steps) {
    for (uint32_t s = 0; s < n_steps; ++s)
        if (step_once(n)) return -1;
    return 0;
}

uint64_t or_raster_size(const or_net* n) { return n->rst_n; }

void or_get_raster(const or_net* n, uint32_t* steps, uint32_t* ids) {
    if (steps) memcpy(steps, n->rst_t, sizeof(uint32_t) * n->rst_n);
    if (ids) memcpy(ids, n->rst_id, sizeof(uint32_t) * n->rst_n);
}

void or_clear_raster(or_net* n) { n->rst_n = 0; }

uint32_t or_time(const or_net* n) { return n->t; }

void or_get_state(const or_net* n, float* V, float* c, uint8_t* ref, int32_t* ring) {
    if (V && n->V) memcpy(V, n->V, sizeof(float) * n->N);
    if (c && n->cf) memcpy(c, n->cf, sizeof(float) * n->N);
    if (ref) memcpy(ref, n->ref, n->N);
    if (ring && n->ring) {
        /* ring rows in absolute-slot order: row r holds inputs for steps with t % D == r */
        size_t tot = (size_t)n->c.D * n->N;
        for (size_t e = 0; e < tot; ++e) ring[e] = (int32_t)(uint32_t)(uint64_t)n->ring[e];
    }
}

void or_get_state_f64(const or_net* n, double* V, double* c) {
    if (V && n->V64) memcpy(V, n->V64, sizeof(double) * n->N);
    if (c && n->c64) memcpy(c, n->c64, sizeof(double) * n->N);
}

void or_set_state_f64(or_net* n, const double* V, const double* c) {
    if (V && n->V64) memcpy(n->V64, V, sizeof(double) * n->N);
    if (c && n->c64) memcpy(n->c64, c, sizeof(double) * n->N);
}

void or_get_ring_f64(const or_net* n, double* ring) {
    if (ring && n->ring64) memcpy(ring, n->ring64, sizeof(double) * (size_t)n->c.D * n->N);
}

void or_set_state(or_net* n, const float* V, const float* c, const uint8_t* ref) {
    if (V && n->V) memcpy(n->V, V, sizeof(float) * n->N);
    if (c && n->cf) memcpy(n->cf, c, sizeof(float) * n->N);
    if (ref) memcpy(n->ref, ref, n->N);
}

void or_get_stats(const or_net* n, uint64_t* spikes, uint64_t* rec, uint64_t* ext) {
    if (spikes) *spikes = n->n_spikes;
    if (rec) *rec = n->rec;
    if (ext) *ext = n->ext;
}
