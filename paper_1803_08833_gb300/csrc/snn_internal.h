// snn_internal.h -- shared declarations of libsnn.so's host runtime and kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include <nvtx3/nvToolsExt.h>

struct snn_config;

namespace snn {

// An NVTX range for the lifetime of the object: profilers show the library's
// phases (construction, steps, launches); free when no tool is attached.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// Philox counter layout (c0, c1, c2, c3) = (a, b, tag, 0).
constexpr uint32_t TAG_GEN = 0u;    // (neuron i, synapse k): target, weight, delay
constexpr uint32_t TAG_DRIVE = 1u;  // (neuron i, step t): external Poisson count, forced spike
constexpr uint32_t TAG_INIT = 2u;   // (neuron i, 0): initial membrane potential
constexpr uint32_t TAG_CONN = 3u;   // (neuron i, 4-candidate group): pairwise connection draws
constexpr uint32_t WTAB = 4096;     // Gaussian efficacy quantiles per population
constexpr uint32_t MAX_ROW = 65535; // longest row of the pairwise rule

constexpr int NEURON_THREADS = 256;
#ifndef SNN_PERSIST_THREADS
#define SNN_PERSIST_THREADS 256
#endif
constexpr int PERSIST_THREADS = SNN_PERSIST_THREADS;  // threads per CTA of the persistent kernel
constexpr int PERSIST_WARPS = PERSIST_THREADS / 32;
constexpr uint32_t ERR_BARRIER_TIMEOUT = 1u;         // DevState::err bits
constexpr uint32_t ERR_ALIGNMENT = 2u;               // a bulk copy address was not 16-byte aligned (skipped)
constexpr uint32_t ERR_BOUNDS = 4u;                  // a device bounds check failed (checked builds, -DSNN_CHECK)
constexpr int NEURONS_PER_THREAD = 4;
constexpr int NEURONS_PER_BLOCK = NEURON_THREADS * NEURONS_PER_THREAD;  // 1024
constexpr int MAX_POIS = 64;  // Poisson table entries (padded to a power of two)
constexpr uint32_t K_ALIGN = 8;  // rows padded to 8 synapses: 32 B f32 / 16 B bf16 / 8 B delay
constexpr uint32_t MAX_NEURON_BLOCKS = 16384;

// Device-resident simulation state shared by consecutive kernels of one network.
struct DevState {
    uint32_t t;          // next step the neuron kernel integrates
    uint32_t t_deliver;  // step whose spikes are staged for the delivery kernel
    uint32_t n_spk;      // spikes staged
    uint32_t done;       // arrival ticket of the neuron kernel's blocks
    uint64_t raster_count;  // spikes recorded since the raster was cleared
    uint64_t raster_base;   // raster index of the first staged spike
    uint64_t n_spikes, rec_events, ext_events;
    uint32_t err;        // sticky error bits (ERR_*)
    uint32_t bar_count;  // grid-barrier arrivals of the current persistent launch
    uint32_t pad0;
    uint32_t pad;
    uint64_t phase_ns[2];  // persistent kernel, CTA 0: neuron phase + barrier, delivery phase + barrier
};

// Everything a kernel needs, passed by value (kernel parameter space).
struct NetView {
    uint32_t N, Npad, M, K, Kpad, n_exc, D, ref_steps, nb;
    uint32_t key0, key1;
    float a_m, a_c, kc, E, V_th, V_reset, alpha_c, in_scale, w_scale;
    int32_t J_ext_fx;
    uint32_t pois_len;  // stored thresholds
    uint32_t pois_pad;  // pois_len rounded up to a power of two (0 if no drive)
    uint64_t imposed_thresh;
    uint32_t pois32[MAX_POIS];  // thresholds, then 0xFFFFFFFF padding
    int32_t w_bf16;
    // synapse table, rows of Kpad entries per neuron: target | delay << 24 in one
    // word (N <= 2^24, delays <= 255) and the weight
    uint32_t* td;
    void* w;
    const uint32_t* row_len;  // pairwise rule: synapses of each row (K = the longest); NULL: K each
    // neuron state (Npad entries) and delay ring (D rows of Npad)
    float* V;
    float* c;
    uint8_t* ref;
    int32_t* ring;
    // per-step spike staging
    uint32_t* seg;      // nb segments of NEURONS_PER_BLOCK ids
    uint32_t* blk_cnt;  // spikes per neuron block
    uint32_t* blk_off;  // exclusive prefix of blk_cnt, nb + 1 entries
    uint64_t* blk_ext;  // external events per neuron block
    uint64_t* blk_rec;  // pairwise rule: recurrent events (row lengths of the spikes) per neuron block
    uint32_t* raster_t;
    uint32_t* raster_id;
    uint64_t raster_cap;
    DevState* st;
    // persistent kernel: per-warp spike offsets within the CTA, per-CTA counts
    uint32_t* woff;
    uint32_t* cta_cnt;
    uint32_t* cta_speed;      // persistent kernel: delivery speed of each CTA (tasks per ns x 2^20, 0 = unmeasured)
    uint32_t res_quads;       // persistent kernel: quads of V, c, ref each CTA keeps in shared memory for the
                              // launch (0: the state stays in global memory); set per launch
    uint64_t wait_limit_ns;   // bound of every grid-barrier wait
    uint32_t barrier_extra;   // test knob: arrivals expected beyond the grid (never satisfied)
    // tiled delivery (grouped layout): per-row segment starts, incoming stencil lists
    uint32_t n_modules, max_off, seg_stride;
    const uint16_t* segidx;   // N x seg_stride: start of the synapses to stencil entry j
    const uint32_t* in_src;   // n_modules x max_off: source modules of target module m
    const uint32_t* in_j;     // ... and the stencil index of m in each source's list
    const uint32_t* in_cnt;   // n_modules
    uint32_t* mod_cnt;        // 2 x n_modules spike counts (double-buffered by step parity)
    uint32_t* seg_mod;        // Npad: spikes of module m at [m M, m M + mod_cnt)
    // banded delivery (schedule 2): the target module rows split into n_bands
    // bands delivered one after another, each band's ring columns L2-resident
    uint32_t n_bands;         // 1: no banding
    uint32_t grid_w;
    uint32_t band_key_row;    // band_rng is indexed by source module row (1) or source module (0)
    const uint2* band_ids;    // n_bands: neuron ids [x, y) of the sources whose stencil reaches the band
    const uint32_t* band_rng; // keys x n_bands: segment-index entries [j0, j1) of the band, j0 | j1 << 16
    // owner-windowed delivery (schedule 4): CTA b owns the quads [b BQ, (b + 1) BQ)
    // and keeps the ring rows of the next own_W steps of its band in shared memory
    uint32_t own_W;           // window steps (1 <= own_W <= D - 1)
    uint32_t own_BQ;          // quads per band
    uint32_t own_cap;         // records per (owner, producer) queue
    uint64_t own_magic;       // ceil(2^32 / own_BQ): band of quad q = (q * own_magic) >> 32, corrected down
    int2* own_rec;            // G x G x own_cap records {window index, fixed-point weight}, owner-major
    uint32_t* own_cnt;        // G x G records queued by producer p for owner b at [b G + p]
    uint32_t* own_ovf;        // G flags: a producer's queue for this owner overflowed (events went to the ring)
    // pulled windowed delivery (schedule 5, grouped layout): CTA b owns the quads
    // [b BQ, (b + 1) BQ), keeps the input of its band for the next pull_W steps in
    // shared memory and pulls, from every spiking row, the range of synapses
    // whose target modules overlap the band
    uint32_t pull_W;          // window steps (1 <= pull_W <= D - 1)
    uint32_t pull_BQ;         // quads of the largest band (the window row)
    const uint32_t* pull_bq;  // G + 1: band b = the quads [pull_bq[b], pull_bq[b + 1])
    uint32_t pull_aligned;    // bands on module boundaries, at most pull_mods_max() modules each
    uint32_t pull_R_max;      // most runs of one band
    uint32_t pull_tmem_chunks;  // chunks of 32 quads per warp whose state is in tensor memory
    uint32_t pull_tmem_cols;    // tensor-memory columns allocated per CTA (a power of 2, 32 .. 512)
    const uint2* pull_runs;   // runs of all bands: {source module, stencil entries j0 | j1 << 16}
    const uint32_t* pull_run_ptr;  // G + 1: runs of band b at [ptr[b], ptr[b + 1])
    uint32_t* pull_seg;       // 2 x Npad: spikes per warp in id order (by step parity)
    uint32_t* pull_segmod;    // 2 x Npad: spikes of module m at [m M, m M + count) (by step parity)
    uint32_t* pull_mcnt;      // 3 x n_modules spike counts (by step mod 3)
    uint32_t* pull_woff;      // 2 x G x warps per CTA: spikes per warp (by step parity)
};

// One shard of a spatially decomposed network (Sec. II-D): the neurons
// [n0, n0 + Nl) of a stripe of module rows, their state and delay ring, and the
// target-side copy of the rows of the halo sources [h0, h0 + rows) restricted
// to the stripe (deferred arborization, Sec. II-C).
struct ShardCounters {
    uint64_t raster_count, n_spikes, rec_events, ext_events;
};
struct ShardView {
    uint32_t n0, Nl, Nlpad;   // first neuron, neurons, ring row stride
    uint32_t h0, rows;        // halo sources
    const uint64_t* row_ptr;  // rows + 1
    const uint32_t* td;       // target - n0 | delay << 24
    const void* w;            // f32 or bf16
    float* V;
    float* c;
    uint8_t* ref;
    int32_t* ring;            // D rows of Nlpad
    uint32_t* spk_bits;       // one bit per neuron of the step
    uint32_t* out_ids;        // outbox: the step's spikes (global ids, increasing)
    uint32_t* out_cnt;        // outbox: their count
    uint32_t* raster_t;
    uint32_t* raster_id;
    uint64_t raster_cap;
    ShardCounters* cnt;
};
constexpr uint32_t SHARD_MAX_LISTS = 16;
struct ShardInbound {  // spike lists delivered into one shard in one step
    const uint32_t* ids[SHARD_MAX_LISTS];
    const uint32_t* cnt[SHARD_MAX_LISTS];
    uint32_t n;
};
cudaError_t launch_shard_step(const NetView& v, const ShardView& sv, uint32_t t, cudaStream_t s);
cudaError_t launch_shard_deliver(const NetView& v, const ShardView& sv, const ShardInbound& in, uint32_t t,
                                 cudaStream_t s);

// Spike-timing dependent plasticity of a network (stdp_kernels.cu).
struct StdpView {
    float* y;              // post-synaptic trace, Npad
    float* x;              // pre-synaptic trace, Npad
    float* xh;             // x of the last D + 1 steps, row t % (D + 1), stride Npad
    uint32_t* hist;        // spike ids of the last D steps, row t % D, stride Npad
    uint32_t* hist_cnt;    // D counts
    int32_t* delta;        // N x Kpad accumulated changes (2^-16 mV)
    const uint64_t* in_ptr;  // N + 1: incoming synapses of neuron j at in_syn[in_ptr[j] .. in_ptr[j + 1])
    const uint64_t* in_syn;  // synapse indices source * Kpad + k
    float a_plus, a_minus;   // trace decays per step
    float A_plus, A_minus, w_max;
    uint32_t period;
};
cudaError_t launch_stdp_index(const NetView& v, uint64_t* cnt_or_cursor, uint64_t* in_syn, cudaStream_t s);
cudaError_t launch_stdp_pre_delivery(const NetView& v, const StdpView& p, cudaStream_t s);
cudaError_t launch_stdp_apply(const NetView& v, const StdpView& p, cudaStream_t s);

// Parameters of the construction kernels.
struct BuildView {
    uint32_t grid_w, grid_h, n_modules, max_off, M, N, Npad, K, Kpad, n_exc;
    uint32_t d_lo, d_span, d_inh;
    uint32_t key0, key1;
    int32_t kernel;
    double spacing, sigma, lambda;
    float w_lo, w_span, w_inh, V_th;
    int32_t w_bf16;
    const int16_t* offsets;  // max_off (dx, dy) pairs in (dy, dx) raster order
    double* scratch;         // n_modules * max_off doubles
    uint32_t* cdf_T;
    uint32_t* cdf_mod;
    uint32_t* cdf_n;
    uint16_t* segidx;  // grouped layout: per neuron max_off + 1 segment starts
    // efficacy and delay laws
    int32_t weight_dist, delay_dist;
    const float* wtab;        // 2 x WTAB Gaussian quantiles (excitatory, then inhibitory)
    const uint64_t* dthr;     // exponential delays: excitatory delay = d_lo + #{k : dthr[k] <= u}
    uint32_t n_dthr;
    // pairwise rule
    uint32_t pair_n;          // stencil entries
    int32_t inh_local_only;
    const int32_t* pair_dx;   // pair_n offsets in (dy, dx) order
    const int32_t* pair_dy;
    const uint64_t* pair_thr; // floor(p 2^32) (2^32: always)
    uint16_t* pair_cnt;       // N x (pair_n + 1): synapses per stencil entry, then their row offsets
    uint32_t* row_len;        // N
    uint32_t* max_len;        // 1: the longest row
};

// Launch wrappers (return the launch error).
cudaError_t launch_build_cdf(const BuildView& b, cudaStream_t s);
cudaError_t launch_gen_synapses(const BuildView& b, uint32_t* td, void* w, cudaStream_t s);
cudaError_t launch_gen_grouped(const BuildView& b, uint32_t* td, void* w, cudaStream_t s);
cudaError_t launch_pair_count(const BuildView& b, cudaStream_t s);
cudaError_t launch_pair_rows(const BuildView& b, cudaStream_t s);
cudaError_t launch_pair_fill(const BuildView& b, uint32_t* td, void* w, cudaStream_t s);
cudaError_t launch_shard_count(const BuildView& b, uint32_t h0, uint32_t rows, uint32_t n0, uint32_t n1, uint32_t* cnt,
                               cudaStream_t s);
cudaError_t launch_shard_fill(const BuildView& b, uint32_t h0, uint32_t rows, uint32_t n0, uint32_t n1,
                              const uint64_t* row_ptr, uint32_t* td, void* w, cudaStream_t s);
cudaError_t launch_shard_init(const BuildView& b, uint32_t n0, uint32_t count, float* V, float* c, uint8_t* ref,
                              cudaStream_t s);
cudaError_t launch_init_state(const BuildView& b, float* V, float* c, uint8_t* ref,
                              cudaStream_t s);
cudaError_t launch_neuron_step(const NetView& v, cudaStream_t s);
cudaError_t launch_deliver(const NetView& v, int schedule, int block, int grid, cudaStream_t s);
int deliver_default_grid(int schedule, int block, uint32_t nb, bool bf16);
int persistent_grid(bool bf16);
// Batched execution: n networks in one global quad / task space.
struct BatchMeta {
    const NetView* views;   // n
    const uint32_t* qoff;   // n + 1: global quad offsets of the networks
    const uint32_t* cbase;  // n + 1: first (network, warp) segment of each network
    const uint32_t* wlo;    // n: first warp whose quads overlap the network
    uint32_t* wcnt;         // n_seg spike counts of the (network, warp) segments
    const uint32_t* steps;  // n: steps of this launch per network
    DevState* bst;          // barrier state of the batch
    uint64_t wait_limit_ns;
    uint32_t barrier_extra;
    uint32_t n, n_seg, Qtot;
};
int batch_grid(uint32_t n, uint32_t n_seg_bound, int shape);
cudaError_t launch_batch(const BatchMeta& bm, uint32_t n_steps, int grid, int shape, cudaStream_t s);
// Grouped batched execution: network k on its own CTAs [gcta[k], gcta[k+1]).
struct GroupMeta {
    const NetView* views;   // n
    const uint32_t* gcta;   // n + 1: CTA prefix of the groups (an empty group: the network is idle)
    const uint32_t* steps;  // n: steps of this launch per network
    uint64_t* gns;          // n: %globaltimer ns each group took (written by its first CTA)
    uint32_t n;
    uint32_t res_quads;     // resident-state capacity of every CTA (set by launch_groups)
};
int groups_grid();  // co-resident grid of the grouped kernel (one CTA per SM)
cudaError_t launch_groups(const GroupMeta& gm, int grid, cudaStream_t s);
int tiled_grid(const NetView& v);  // 0 if the tile does not fit in shared memory
cudaError_t launch_tiled(const NetView& v, uint32_t n_steps, int grid, cudaStream_t s);
cudaError_t launch_persistent(const NetView& v, uint32_t n_steps, int grid, cudaStream_t s);
// Owner-windowed persistent kernel (schedule 4): the largest window (steps) that
// fits next to the kernel's other shared memory on `grid` CTAs for bands of BQ
// quads (0 if none), and the launch.
uint32_t owned_max_window(const NetView& v, int grid, uint32_t BQ);
int owned_grid();
size_t owned_smem_bytes(uint32_t W, uint32_t BQ, int grid);
cudaError_t launch_owned(const NetView& v, uint32_t n_steps, int grid, cudaStream_t s);
uint32_t pull_build_runs(uint32_t N, uint32_t M, uint32_t gw, uint32_t gh, const std::vector<int16_t>& off,
                         const std::vector<uint32_t>& bq, std::vector<uint2>& runs, std::vector<uint32_t>& ptr,
                         bool all_entries);
std::vector<uint32_t> pull_bands(uint32_t N, uint32_t M, uint32_t Q, uint32_t G, bool aligned);
uint32_t pull_max_window(const NetView& v, int grid, uint32_t BQ, uint32_t R_max);
size_t pull_smem_bytes(uint32_t W, uint32_t BQ, int grid, uint32_t R_max);
uint32_t pull_warps();
uint32_t pull_mods_max();
uint32_t pull_k_max();
uint32_t pull_tmem_cols(uint32_t BQ, uint32_t* chunks);
cudaError_t launch_pull(const NetView& v, uint32_t n_steps, int grid, cudaStream_t s);
uint32_t persistent_resident_quads(const NetView& v, int grid);  // 0: the state cannot stay in shared memory
// In-disc grid offsets (dx, dy pairs) of the cut-off radius, dx^2 + dy^2 <=
// R2 = floor((cutoff / spacing)^2), in (dy, dx) raster order (the stencil order
// of the target-module tables); *R2_out receives R2.
std::vector<int16_t> disc_offsets(const snn_config& c, uint32_t* R2_out);
cudaError_t prepare_deliver(uint32_t nb);

void count_launch(uint64_t n);
void pairwise_bounds(const snn_config& c, uint32_t* max_row, uint32_t* stencil);
void set_last_error(const char* msg);  // message returned by snn_last_error()

}  // namespace snn

// Host-side accessors of a network for the library's own runtime parts.
struct snn_net;
struct snn_config;
const snn_config* snn_config_of(const snn_net* net);
cudaError_t snn_set_raster_count(snn_net* net, uint64_t count, cudaStream_t s);
