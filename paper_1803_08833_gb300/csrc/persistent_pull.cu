// persistent_pull.cu -- persistent multi-step kernel: band-owned delay windows
// filled by pulling each band's piece of every spiking row.
//
// The push delivery (k_run_steps) costs one random L2 reduction per synaptic
// event, and L2 takes scattered 8-byte stores at about the same sector rate
// (k_run_steps_owned, which queued near events as records, measured that).
// Here no event is written to L2 unless its delay is longer than the window.
// Every CTA owns a band of quads for the whole launch (uniform bands, or bands
// cut only at module boundaries) and keeps in shared memory a window of W rows
// of the band: row (t + d) mod W collects the input its band receives at step
// t + d from events of delay d <= W.  Events of longer delay go to the delay
// ring in global memory as before.  One step t:
//
//   N  the band's neurons (flow steps 4-6, Sec. II-A): the input of step t is
//      window row t mod W; the neuron state (V, c, refractory counters) stays
//      in the SM's tensor memory for the whole launch, so the phase reads
//      nothing from global memory; spikes are staged in id order per warp (for
//      the raster) and appended to their module's list (counted by the
//      module's owner in shared memory when the bands are module-aligned);
//   -- grid barrier, split: between arriving and waiting each CTA fills the
//      step's per-delay destinations, draws the next step's external drive and
//      starts copying its band's slice of ring row (t + W) mod D into window
//      row t mod W (the row N(t) has consumed): every far event of step t + W
//      has a delay > W, so it came from a step < t and the slice is final.
//      The copy lands before D(t) adds the events of delay W into that row,
//      and the slice is then cleared in the ring --
//   D  (flow steps 2-3) every CTA writes the raster entries of every G-th
//      spike; then it walks its band's runs: for every source module whose
//      stencil reaches the band, the spikes of that module and, in each
//      spike's row, the one contiguous range of synapses whose target modules
//      overlap the band -- the grouped row is ordered by target module and the
//      stencil order is increasing in module index, so the range is
//      [seg[j0], seg[j1]) of the row's segment index.  The ranges (pieces) of
//      a batch are flattened into one index of 16-byte quads, 32 quads per
//      warp instruction, so short pieces waste no lanes.  Every synapse of a
//      piece whose target lies in the band adds its weight into the window
//      with a shared-memory atomic (d <= W) or into the ring with an L2
//      reduction (d > W).
//
// There is one grid barrier per step.  A CTA may start N(t + 1) while others
// are still in D(t): every event a CTA delivers targets its own band, so its
// window and its band's columns of the ring are written by it alone, and the
// spike lists are kept by step parity (the module counters by step mod 3, so
// that each can be cleared two steps after its use while nobody reads or
// writes it).
//
// At the start of a launch the window takes ring rows t0 .. t0 + W - 1 of the
// band (cleared there) and the state moves into tensor memory; at the end the
// window is added back into the ring and the state written back, so between
// calls the ring and the state hold exactly what the push delivery would hold.
// Integer sums: results are bit-identical to every other schedule.
// Every barrier wait is bounded (grid_common.cuh).
#include "grid_common.cuh"

#include <algorithm>
#include <numeric>
#include <vector>

namespace snn {

#ifndef SNN_PULL_THREADS
#define SNN_PULL_THREADS 512
#endif
#ifndef SNN_PULL_UNROLL
#define SNN_PULL_UNROLL 4
#endif
constexpr int PULL_THREADS = SNN_PULL_THREADS;
constexpr int PULL_WARPS = PULL_THREADS / 32;
constexpr int PULL_DRV = 4;                     // chunks per thread whose next-step drive is drawn during delivery
constexpr uint32_t PULL_PIECES = PULL_THREADS;  // (spike, run) pieces staged per batch: one per thread
constexpr int PULL_UNROLL = SNN_PULL_UNROLL;    // chunks of 32 quads in flight per warp
constexpr uint32_t PULL_K_MAX = 8188;           // longest row: a piece spans at most 2^11 quads
constexpr uint32_t PULL_MODS_MAX = 64;          // modules of a band counted in shared memory
static_assert(PULL_PIECES < 1024u && (uint64_t)PULL_PIECES * ((PULL_K_MAX + 3) / 4 + 1) < (1u << 22),
              "the compaction key of a batch holds 10 bits of rank and 22 bits of quads");

// Shared memory other than the window, in 32-bit words: per-warp spike
// offsets (TW + 1), drawn-ahead drives, the staged pieces (row, start | length
// << 16, quad prefix), the band's runs (source module, j0 | j1 << 16, spike
// prefix), the compaction of a batch, the per-delay destinations of a step,
// the first quad of every band (G + 1); padded to 16 B.
__host__ __device__ constexpr uint32_t pull_aux_words(uint32_t G, uint32_t R_max) {
    return ((G * PULL_WARPS + 1) + PULL_DRV * PULL_THREADS + 3 * PULL_PIECES + 1 + 2 * R_max + (R_max + 1) +
            (PULL_PIECES + 1) + 256 + (G + 1) + 3) &
           ~3u;
}

// Neuron id of spike j of the step: its warp by binary search over the
// per-warp prefix, then that warp's staging segment of `seg`.
__device__ __forceinline__ uint32_t pull_spike_id(const uint32_t* seg, const uint32_t* s_wpre, uint32_t TW,
                                                  const uint32_t* s_bq, uint32_t j) {
    uint32_t lo = 0, hi = TW;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_wpre[mid] <= j)
            lo = mid;
        else
            hi = mid;
    }
    const uint32_t b = lo / PULL_WARPS, w = lo - b * PULL_WARPS;
    const uint32_t q0 = s_bq[b], q1 = s_bq[b + 1];
    const uint32_t qa = q0 + (q1 - q0) * w / PULL_WARPS;
    return __ldcg(seg + ((size_t)qa << 2) + (j - s_wpre[lo]));
}

// The L2 line holding p.
__device__ __forceinline__ void prefetch_line(const void* p) { asm volatile("prefetch.global.L2 [%0];" ::"l"(p)); }

// Largest k < n with pre[k] <= x (pre nondecreasing, pre[0] = 0 <= x).
__device__ __forceinline__ uint32_t pull_slot(const uint32_t* pre, uint32_t n, uint32_t x) {
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= x)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

// L2 reduction without a compiler memory barrier: nothing in the delivery
// phase reads the ring (the next step's barrier orders the reductions).
__device__ __forceinline__ void red_far(int32_t* p, int32_t x) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(x));
}

// L2 policy of the row reads: the bands of a row read it within one phase.
__device__ __forceinline__ uint64_t evict_normal_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// The synapses [a, a + len) of a piece are read as the quads (aligned groups
// of four) that hold them: quads (a >> 2) .. ((a + len - 1) >> 2) of the row,
// so every quad is one 16-byte vector (rows start 32-byte aligned and hold
// Kpad >= a + len entries: a vector never leaves its row).
// Tensor memory (128 lanes x 512 columns of 32 bits per SM, Blackwell) holds
// the band's neuron state for a launch.  Warp w reaches the lanes 32 (w mod 4)
// .. 32 (w mod 4) + 31; lane i of chunk k of the warp is the quad of its lane i,
// with V and c in 8 columns (8-aligned) and the refractory bytes in one:
// columns 8 (MC (w / 4) + k) .. + 7 and 32 MC + MC (w / 4) + k, MC = chunks per
// warp (36 MC columns in all).  Loads and stores wait for completion inside
// the same asm statement, so no register is read before its data arrived.
__device__ __forceinline__ void tmem_alloc(uint32_t* s_dst, uint32_t ncols) {
    asm volatile(
        "tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n\t"
        "tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::"r"((uint32_t)__cvta_generic_to_shared(s_dst)),
        "r"(ncols)
        : "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_fence_before_sync() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tmem_ld9(uint32_t a8, uint32_t a1, uint32_t (&r)[9]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%9];\n\t"
        "tcgen05.ld.sync.aligned.32x32b.x1.b32 {%8}, [%10];\n\t"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8])
        : "r"(a8), "r"(a1)
        : "memory");
}
__device__ __forceinline__ void tmem_st9(uint32_t a8, uint32_t a1, const uint32_t (&r)[9]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%2, %3, %4, %5, %6, %7, %8, %9};\n\t"
        "tcgen05.st.sync.aligned.32x32b.x1.b32 [%1], {%10};\n\t"
        "tcgen05.wait::st.sync.aligned;" ::"r"(a8),
        "r"(a1), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]), "r"(r[8])
        : "memory");
}
// The quad's state as 9 words: V (4), c (4), refractory bytes.
__device__ __forceinline__ void state_words(const float4& V, const float4& C, uint32_t R, uint32_t (&r)[9]) {
    r[0] = __float_as_uint(V.x);
    r[1] = __float_as_uint(V.y);
    r[2] = __float_as_uint(V.z);
    r[3] = __float_as_uint(V.w);
    r[4] = __float_as_uint(C.x);
    r[5] = __float_as_uint(C.y);
    r[6] = __float_as_uint(C.z);
    r[7] = __float_as_uint(C.w);
    r[8] = R;
}

// 16 bytes global -> shared without registers (L2 only), and the wait for
// every such copy this thread issued.
__device__ __forceinline__ void cp_async16(void* s_dst, const void* g_src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(s_dst)),
                 "l"(g_src)
                 : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

__device__ __forceinline__ uint32_t pull_piece_quads(uint32_t a, uint32_t len) {
    return len ? ((a + len + 3) >> 2) - (a >> 2) : 0u;
}

// One warp delivers the quads of up to PULL_UNROLL chunks from chunk c (chunk
// x = the quads [32 x, 32 x + 32) of the staged batch, below cend), lane l
// taking quad 32 x + l.  pp is the piece holding quad 32 c.  The 32 pieces from
// pp are held one per lane (start quad of the next piece, row, range, start
// quad); a lane's piece is pp + the count of those next-piece starts at or
// before its quad.  The pieces of the batch are non-empty, so a chunk whose
// last quad lies before the start of piece pp + 32 is covered by the window;
// the first chunk that is not ends the call.  Synapses of the piece whose
// target lies in the band [n0, n0 + nband) add their weight where s_dtab[d]
// says: window row (t + d) mod W if d <= W, else ring row (t + d) mod D.
// Advances c and pp past the chunks delivered.
template <bool BF16>
__device__ __forceinline__ void pull_chunks(const NetView& v, uint32_t& c, uint32_t cend, uint32_t& pp,
                                            uint32_t np, uint32_t Qt, const uint32_t* s_pid, const uint32_t* s_pa,
                                            const uint32_t* s_pre, const uint32_t* s_dtab, int32_t* win, uint32_t n0,
                                            uint32_t nband, uint32_t W, uint32_t BN, uint32_t lane, uint64_t pol) {
    uint4 tg[PULL_UNROLL], wr[PULL_UNROLL];
    uint32_t vm[PULL_UNROLL];                    // the lane's synapses of its piece: bit q for synapse q of the quad
    const uint32_t le_mask = (2u << lane) - 1u;  // lanes <= this one (all 32 for lane 31)
    const uint32_t j = pp + lane;                // the window: pieces pp .. pp + 31
    const uint32_t nxt = j + 1 <= np ? s_pre[j + 1] : 0xFFFFFFFFu;
    const uint32_t wid = j < np ? s_pid[j] : 0u, wpa = j < np ? s_pa[j] : 0u, wqs = j < np ? s_pre[j] : 0u;
    uint32_t done = 0;  // chunks covered by the window (warp-uniform)
#pragma unroll
    for (int u = 0; u < PULL_UNROLL; ++u) {
        const uint32_t cu = c + (uint32_t)u;
        vm[u] = 0;
        const uint32_t cbase = cu << 5;
        // next-piece starts at or before the chunk's first quad, and those inside it
        const uint32_t before = __popc(__ballot_sync(0xFFFFFFFFu, nxt <= cbase));
        const uint32_t pos = nxt - cbase;  // inside the chunk: 1 .. 31
        const uint32_t bits = __reduce_or_sync(0xFFFFFFFFu, pos - 1u < 31u ? 1u << pos : 0u);
        const bool fits = before + __popc(bits) < 32u;  // the chunk's last quad lies in the window
        if (cu < cend && fits && done == (uint32_t)u) {  // warp-uniform
            done = u + 1;
            const uint32_t k = before + __popc(bits & le_mask);  // the lane's piece: pp + k
            const uint32_t id = __shfl_sync(0xFFFFFFFFu, wid, k);
            const uint32_t pa = __shfl_sync(0xFFFFFFFFu, wpa, k);
            const uint32_t qs = __shfl_sync(0xFFFFFFFFu, wqs, k);
            const uint32_t qi = cbase + lane;
            if (qi < Qt) {
                const uint32_t a = pa & 0xFFFFu, end = a + (pa >> 16);
                const uint32_t k0 = (a & ~3u) + ((qi - qs) << 2);
                const uint32_t lo = a > k0 ? a - k0 : 0u, hi = min(4u, end - k0);
                vm[u] = (0xFu >> (4u - hi)) & (0xFu << lo);
                const size_t e = (size_t)id * v.Kpad + k0;
                if (SNN_BOUND(v.st, k0 < end && id < v.N)) {
                    tg[u] = ld_u4(v.td + e, pol);
                    if (BF16) {
                        const uint2 wb = ld_u2(reinterpret_cast<const uint16_t*>(v.w) + e, pol);
                        wr[u] = make_uint4(wb.x, wb.y, 0u, 0u);
                    } else {
                        wr[u] = ld_u4(reinterpret_cast<const float*>(v.w) + e, pol);
                    }
                } else {
                    vm[u] = 0;
                }
            }
        }
    }
    // the events: every quantity computed for all 4 synapses, the adds predicated
#pragma unroll
    for (int u = 0; u < PULL_UNROLL; ++u) {
        if ((uint32_t)u < done) {
            const uint32_t tq[4] = {tg[u].x, tg[u].y, tg[u].z, tg[u].w};
            const uint32_t wq[4] = {wr[u].x, wr[u].y, wr[u].z, wr[u].w};
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const uint32_t tgt = tq[q] & 0xFFFFFFu;
                const uint32_t loc = tgt - n0;
                const bool ok = ((vm[u] >> q) & 1u) & (loc < nband);
                const uint32_t dt = s_dtab[tq[q] >> 24];
                const float wv = BF16 ? ((q & 1) ? bf16_hi(wq[q >> 1]) : bf16_lo(wq[q >> 1])) : __uint_as_float(wq[q]);
                const int32_t fx = fx_weight(v, wv);
                if (ok & ((int32_t)dt >= 0)) {
                    if (SNN_BOUND(v.st, dt < W * BN)) atomicAdd(win + dt + loc, fx);
                }
                if (ok & ((int32_t)dt < 0)) {
                    const uint32_t sf = dt & 0x7FFFFFFFu;
                    if (SNN_BOUND(v.st, sf < v.D && tgt < v.N)) red_far(v.ring + (size_t)sf * v.Npad + tgt, fx);
                }
            }
        }
    }
    // the piece holding the first quad after the delivered chunks
    const uint32_t cn = (c + done) << 5;
    pp += __popc(__ballot_sync(0xFFFFFFFFu, nxt <= cn));
    c += done;
}

template <bool BF16>
__global__ void __launch_bounds__(PULL_THREADS, 1) k_run_steps_pull(NetView v, uint32_t n_steps) {
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t G = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
    const uint32_t TW = G * PULL_WARPS;
    const uint32_t Q = v.Npad >> 2, M = v.M, nm = v.n_modules, D = v.D;
    const uint32_t W = v.pull_W, BQ = v.pull_BQ, BN = BQ << 2;  // BQ: quads of the largest band
    const uint32_t q0 = v.pull_bq[bid], q1 = v.pull_bq[bid + 1], nq = q1 - q0;  // this CTA's band of quads
    const uint32_t n0 = q0 << 2, nband = nq << 2;                              // its neurons [n0, n0 + nband)
    const uint32_t rbase = v.pull_run_ptr[bid], nr = v.pull_run_ptr[bid + 1] - rbase;
    int4* win4 = reinterpret_cast<int4*>(smem);  // W rows of BQ quads
    int32_t* win = reinterpret_cast<int32_t*>(smem);
    uint32_t* s_wpre = smem + (size_t)W * BQ * 4;       // TW + 1
    uint32_t* s_drv = s_wpre + TW + 1;                  // PULL_DRV x PULL_THREADS
    uint32_t* s_pid = s_drv + PULL_DRV * PULL_THREADS;  // staged pieces: row
    uint32_t* s_pa = s_pid + PULL_PIECES;               //   its range: first synapse | length << 16
    uint32_t* s_pre = s_pa + PULL_PIECES;               //   quad prefix (PULL_PIECES + 1)
    uint32_t* s_rsrc = s_pre + PULL_PIECES + 1;         // the band's runs: source module
    uint32_t* s_rj = s_rsrc + v.pull_R_max;             //   stencil entries j0 | j1 << 16
    uint32_t* s_rpre = s_rj + v.pull_R_max;             //   spike prefix (R_max + 1)
    uint32_t* s_tmp = s_rpre + v.pull_R_max + 1;        // compaction of a batch (PULL_PIECES + 1)
    uint32_t* s_dtab = s_tmp + PULL_PIECES + 1;         // per delay d: where the events of this step go (256)
    uint32_t* s_bq = s_dtab + 256;                      // first quad of every band (G + 1)
    __shared__ uint32_t s_t0;
    __shared__ unsigned long long s_rc0;
    __shared__ uint32_t s_ext[PULL_WARPS];
    __shared__ unsigned long long s_rec[PULL_WARPS];
    __shared__ uint32_t s_pois[MAX_POIS];
    __shared__ uint32_t s_mc[PULL_MODS_MAX];  // module-aligned bands: spikes per module of the band this step
    __shared__ uint32_t s_tmem;               // tensor memory of the band's state
    load_poisson_table(v, s_pois);
    uint32_t gen = 0;
    if (tid == 0) {
        s_t0 = v.st->t;
        s_rc0 = v.st->raster_count;
    }
    // With module-aligned bands every module has one owner, which counts its
    // spikes in shared memory and publishes the count before the barrier.
    const bool own_mods = v.pull_aligned != 0;
    const uint32_t m_lo = n0 / M, nmb = nband ? (n0 + nband - 1) / M - m_lo + 1 : 0u;
    for (uint32_t m = tid; m < PULL_MODS_MAX; m += PULL_THREADS) s_mc[m] = 0;
    for (uint32_t r = tid; r < nr; r += PULL_THREADS) {
        const uint2 x = v.pull_runs[rbase + r];
        s_rsrc[r] = x.x;
        s_rj[r] = x.y;
    }
    for (uint32_t x = tid; x < W * BQ; x += PULL_THREADS) win4[x] = make_int4(0, 0, 0, 0);
    for (uint32_t b = tid; b <= G; b += PULL_THREADS) s_bq[b] = v.pull_bq[b];
    for (uint32_t m = bid * PULL_THREADS + tid; m < 3 * nm; m += G * PULL_THREADS) v.pull_mcnt[m] = 0;
    const uint32_t lane = tid & 31, warp = tid >> 5;
    const uint32_t lt_mask = (1u << lane) - 1u;
    const uint32_t wg = bid * PULL_WARPS + warp;
    const uint32_t qa = q0 + nq * warp / PULL_WARPS, qb = q0 + nq * (warp + 1) / PULL_WARPS;
    // the band's state into tensor memory: this warp's chunks of 32 quads
    const uint32_t MC = v.pull_tmem_chunks, tcols = v.pull_tmem_cols;
    if (warp == 0) tmem_alloc(&s_tmem, tcols);
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    const uint32_t tm_lane = s_tmem + (((warp & 3u) * 32u) << 16);
    const uint32_t tm_vc = tm_lane + 8u * MC * (warp >> 2), tm_r = tm_lane + 32u * MC + MC * (warp >> 2);
    {
        uint32_t k = 0;
        for (uint32_t qc = qa; qc < qb; qc += 32, ++k) {
            const uint32_t q = qc + lane;
            uint32_t w9[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
            if (q < qb) {
                QuadIn in;
                load_state(v, q << 2, in);
                state_words(in.V, in.C, in.R, w9);
            }
            __syncwarp();
            if (SNN_BOUND(v.st, k < MC)) tmem_st9(tm_vc + 8u * k, tm_r + k, w9);
        }
    }
    bool ok = grid_barrier(v, G, gen);  // (starts with a CTA barrier) the module counters are clear everywhere
    const uint32_t t0 = s_t0;
    int4* ring4 = reinterpret_cast<int4*>(v.ring);
    const uint32_t Q4 = v.Npad >> 2;  // int4 per ring row
    // the window takes the band's ring rows of steps t0 .. t0 + W - 1 (final:
    // their far events came from earlier launches), cleared in the ring
    // (all copies in flight at once; each cleared once it has landed)
    for (uint32_t x = tid; x < W * nq; x += PULL_THREADS) {
        const uint32_t k = x / nq, lq = x - k * nq;
        cp_async16(win4 + (size_t)((t0 + k) % W) * BQ + lq, ring4 + (size_t)((t0 + k) % D) * Q4 + q0 + lq);
    }
    cp_async_wait_all();
    for (uint32_t x = tid; x < W * nq; x += PULL_THREADS) {
        const uint32_t k = x / nq, lq = x - k * nq;
        ring4[(size_t)((t0 + k) % D) * Q4 + q0 + lq] = make_int4(0, 0, 0, 0);
    }
    __syncthreads();
    const uint32_t Kpad = v.Kpad, stride = v.seg_stride;
    const uint64_t pol = evict_normal_policy();

    uint64_t rc = s_rc0;
    uint64_t spikes = 0;
    uint32_t ext = 0;
    uint64_t rec = 0;
    uint32_t done = 0;
    uint64_t ph_n = 0, ph_d = 0, stamp = 0;
    if (bid == 0 && tid == 0) stamp = global_ns();
    const uint32_t nchunk = qa + lane < qb ? (qb - qa - lane + 31) / 32 : 0u;
    const uint32_t nd_max = nchunk < (uint32_t)PULL_DRV ? nchunk : (uint32_t)PULL_DRV;
    uint32_t ndrv = 0;  // chunks whose drive for the coming step is in s_drv
    auto drive_of = [&](uint32_t k, uint32_t tt) -> uint32_t {
        return k < ndrv ? s_drv[k * PULL_THREADS + tid] : quad_drive(v, s_pois, (qa + lane + 32 * k) << 2, tt);
    };

    for (uint32_t step = 0; ok && step < n_steps; ++step) {
        const uint32_t t = t0 + step;
        const uint32_t par = t & 1u;
        const uint32_t wslot = t % W, slot0 = t % D;
        uint32_t* seg = v.pull_seg + (size_t)par * v.Npad;     // spikes per warp, id order
        uint32_t* segm = v.pull_segmod + (size_t)par * v.Npad;  // spikes of module m at [m M, m M + mcnt[m])
        uint32_t* mcnt = v.pull_mcnt + (size_t)(t % 3u) * nm;
        uint32_t* woff = v.pull_woff + (size_t)par * TW;
        // ---- phase N: input = window row t mod W (the ring's far events of the
        // step were folded into it W steps ago); state in tensor memory; spikes staged
        uint32_t run = 0;
        {
            uint32_t k = 0;
            for (uint32_t qc = qa; qc < qb; qc += 32, ++k) {
                const uint32_t q = qc + lane;
                uint32_t w9[9];
                __syncwarp();
                tmem_ld9(tm_vc + 8u * k, tm_r + k, w9);
                uint32_t spk = 0;
                if (q < qb) {
                    QuadIn cur;
                    cur.V = make_float4(__uint_as_float(w9[0]), __uint_as_float(w9[1]), __uint_as_float(w9[2]),
                                        __uint_as_float(w9[3]));
                    cur.C = make_float4(__uint_as_float(w9[4]), __uint_as_float(w9[5]), __uint_as_float(w9[6]),
                                        __uint_as_float(w9[7]));
                    cur.R = w9[8];
                    cur.drive = drive_of(k, t);
                    cur.I = win4[(size_t)wslot * BQ + (q - q0)];
                    QuadOut o;
                    spk = integrate_quad<false>(v, q << 2, 0u, cur, ext, rec, o);
                    state_words(o.V, o.C, o.R, w9);
                }
                __syncwarp();
                tmem_st9(tm_vc + 8u * k, tm_r + k, w9);
                const uint32_t cnt = __popc(spk);
                uint32_t incl = cnt;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                    if (lane >= (uint32_t)o) incl += y;
                }
                uint32_t pos = (qa << 2) + run + incl - cnt;
#pragma unroll
                for (int b = 0; b < 4; ++b)
                    if (spk & (1u << b)) {
                        const uint32_t id = (q << 2) + b;
                        if (SNN_BOUND(v.st, pos < (qb << 2))) seg[pos] = id;
                        ++pos;
                        prefetch_line(v.segidx + (size_t)id * stride);  // read by the bands in the next phase
                    }
                run += __shfl_sync(0xFFFFFFFFu, incl, 31);
                if (__any_sync(0xFFFFFFFFu, spk != 0)) {  // module lists: one atomic per module and bit
                    const uint32_t m0 = (q << 2) / M, r0 = (q << 2) - m0 * M;
#pragma unroll
                    for (int b = 0; b < 4; ++b) {
                        const bool has = (spk >> b) & 1u;
                        const uint32_t mb = m0 + (r0 + b) / M;
                        const uint32_t key = has ? mb : 0xFFFFFFFFu;
                        const uint32_t peers = __match_any_sync(0xFFFFFFFFu, key);
                        const uint32_t leader = __ffs(peers) - 1;
                        uint32_t base = 0;
                        if (has && lane == leader) {
                            if (own_mods)
                                base = SNN_BOUND(v.st, mb - m_lo < nmb && nmb <= PULL_MODS_MAX)
                                           ? atomicAdd(s_mc + (mb - m_lo), (uint32_t)__popc(peers))
                                           : M;
                            else
                                base = atomicAdd(mcnt + mb, (uint32_t)__popc(peers));
                        }
                        base = __shfl_sync(0xFFFFFFFFu, base, leader);
                        const uint32_t at = base + __popc(peers & lt_mask);
                        if (has && SNN_BOUND(v.st, mb < nm && at < M)) segm[(size_t)mb * M + at] = (q << 2) + b;
                    }
                }
            }
        }
        if (lane == 0) woff[wg] = run;
        if (own_mods) {  // the band's module counts, published (and cleared for the next step)
            __syncthreads();
            for (uint32_t m = tid; m < nmb; m += PULL_THREADS) {
                mcnt[m_lo + m] = s_mc[m];
                s_mc[m] = 0;
            }
        }
        // split barrier: arrive, then do what needs nobody else's data -- this
        // step's per-delay destinations and the next step's external drive --
        // while the other CTAs finish, then wait
        grid_arrive(v.st, gen);
        // d <= W: word offset of window row (t + d) mod W; else 2^31 | ring row (t + d) mod D
        for (uint32_t d = tid; d < 256; d += PULL_THREADS) {
            const uint32_t ws = (wslot + d) % W, rs = (slot0 + d) % D;
            s_dtab[d] = d <= W ? ws * BN : 0x80000000u | rs;
        }
        // ring row (t + W) mod D of the band into window row t mod W (waited for
        // before the first event of delay W lands there, cleared in the ring then)
        int4* fold = ring4 + (size_t)((t + W) % D) * Q4 + q0;
        for (uint32_t x = tid; x < nq; x += PULL_THREADS) cp_async16(win4 + (size_t)wslot * BQ + x, fold + x);
        ndrv = 0;
        if (step + 1 < n_steps)
            for (; ndrv < nd_max; ++ndrv)
                s_drv[ndrv * PULL_THREADS + tid] = quad_drive(v, s_pois, (qa + lane + 32 * ndrv) << 2, t + 1);
        if (!grid_wait(v.st, G + v.barrier_extra, v.wait_limit_ns, gen)) break;
        if (bid == 0 && tid == 0) {
            const uint64_t now = global_ns();
            ph_n += now - stamp;
            stamp = now;
        }

        // ---- phase D: raster of every G-th spike, then the band's pieces
        {
            uint32_t* mclr = v.pull_mcnt + (size_t)((t + 2u) % 3u) * nm;  // the counters of step t - 1
            for (uint32_t m = bid * PULL_THREADS + tid; m < nm; m += G * PULL_THREADS) mclr[m] = 0;
        }
        // the runs' spike counts and the per-warp spike counts: loads in flight together
        for (uint32_t r = tid; r < nr; r += PULL_THREADS) s_rpre[r] = __ldcg(mcnt + s_rsrc[r]);
        block_exclusive_scan(woff, TW, s_wpre);  // ends with a CTA barrier
        const uint32_t total = s_wpre[TW];
        block_scan_inplace(s_rpre, nr);  // s_rpre[nr] = pieces of the step
        const uint32_t P = s_rpre[nr];
        // piece p: spike (p - s_rpre[r]) of run r's source module; its range [a, a + len) of the row
        auto piece_id = [&](uint32_t p, uint32_t& r) -> uint32_t {
            r = pull_slot(s_rpre, nr, p);
            const uint32_t k = p - s_rpre[r];
            return SNN_BOUND(v.st, s_rsrc[r] < nm && k < M) ? __ldcg(segm + (size_t)s_rsrc[r] * M + k) : 0u;
        };
        auto piece_range = [&](uint32_t id, uint32_t r, uint32_t& a, uint32_t& len) {
            const uint16_t* sg = v.segidx + (size_t)id * stride;
            const uint32_t jj = s_rj[r];
            a = __ldg(sg + (jj & 0xFFFFu));
            len = __ldg(sg + (jj >> 16)) - a;
        };
        // pieces are loaded two batches ahead (the row id) and one ahead (its
        // range); the raster entries are written while the first loads are in flight
        uint32_t idA = 0, aA = 0, lA = 0, idB = 0, rB = 0;
        {
            uint32_t rA = 0;
            if (tid < P) idA = piece_id(tid, rA);
            if (PULL_PIECES + tid < P) idB = piece_id(PULL_PIECES + tid, rB);
            for (uint32_t j = bid + G * tid; j < total; j += G * PULL_THREADS) {
                const uint32_t id = pull_spike_id(seg, s_wpre, TW, s_bq, j);
                const uint64_t r = rc + j;
                if (r < v.raster_cap) {
                    v.raster_t[r] = t;
                    v.raster_id[r] = id;
                }
            }
            if (tid < P) piece_range(idA, rA, aA, lA);
        }
        // the fold has landed (visible to the CTA after the batch's first barrier)
        cp_async_wait_all();
        for (uint32_t x = tid; x < nq; x += PULL_THREADS) fold[x] = make_int4(0, 0, 0, 0);
        for (uint32_t pb = 0; pb < P; pb += PULL_PIECES) {
            const uint32_t nb = min(PULL_PIECES, P - pb);
            // the batch's non-empty pieces, compacted: (rank << 22) | quads, scanned
            // (at most 2^10 - 1 pieces of at most 2^11 quads: K <= PULL_K_MAX)
            const uint32_t nqp = tid < nb ? pull_piece_quads(aA, lA) : 0u;
            s_tmp[tid] = nqp ? (1u << 22) | nqp : 0u;
            __syncthreads();
            block_scan_inplace(s_tmp, PULL_PIECES);
            if (nqp) {
                const uint32_t x = s_tmp[tid], ci = x >> 22;
                s_pid[ci] = idA;
                s_pa[ci] = aA | (lA << 16);
                s_pre[ci] = x & 0x3FFFFFu;
            }
            const uint32_t np = s_tmp[PULL_PIECES] >> 22, Qt = s_tmp[PULL_PIECES] & 0x3FFFFFu;
            if (tid == 0) s_pre[np] = Qt;
            __syncthreads();
            uint32_t idC = 0, rC = 0, aB = 0, lB = 0;
            if (pb + 2 * PULL_PIECES + tid < P) idC = piece_id(pb + 2 * PULL_PIECES + tid, rC);
            if (pb + PULL_PIECES + tid < P) piece_range(idB, rB, aB, lB);
            const uint32_t C = (Qt + 31) >> 5;  // chunks of 32 quads; warp w takes a contiguous share
            const uint32_t c0 = (uint32_t)((uint64_t)C * warp / PULL_WARPS);
            const uint32_t c1 = (uint32_t)((uint64_t)C * (warp + 1) / PULL_WARPS);
            if (c0 < c1) {
                uint32_t pp = pull_slot(s_pre, np, c0 << 5);
                for (uint32_t c = c0; c < c1;)
                    pull_chunks<BF16>(v, c, c1, pp, np, Qt, s_pid, s_pa, s_pre, s_dtab, win, n0, nband, W, BN, lane,
                                      pol);
            }
            __syncthreads();  // the staged batch is read by every warp before the next is written
            idA = idB;
            aA = aB;
            lA = lB;
            idB = idC;
            rB = rC;
        }
        rc += total;
        spikes += total;
        __syncthreads();  // every event of the step is in the window before N(t + 1) reads it
        if (bid == 0 && tid == 0) {
            const uint64_t now = global_ns();
            ph_d += now - stamp;
            stamp = now;
        }
        done = step + 1;
    }

    // ---- epilogue: the window back into the ring (rows te .. te + W - 1: no
    // other CTA's far reduction of the last step lands there), the state back
    // from tensor memory, counters
    cp_async_wait_all();  // a step left by a barrier timeout may have a fold in flight
    __syncthreads();
    {
        const uint32_t te = t0 + done, nx = W * nq;
        for (uint32_t x0 = 0; x0 < nx; x0 += 8 * PULL_THREADS) {  // eight ring loads in flight per thread
            int4 a[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t x = x0 + u * PULL_THREADS + tid;
                if (x < nx) {
                    const uint32_t k = x / nq, lq = x - k * nq;
                    a[u] = __ldcg(ring4 + (size_t)((te + k) % D) * Q4 + q0 + lq);
                }
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const uint32_t x = x0 + u * PULL_THREADS + tid;
                if (x < nx) {
                    const uint32_t k = x / nq, lq = x - k * nq;
                    const int4 c = win4[(size_t)((te + k) % W) * BQ + lq];
                    ring4[(size_t)((te + k) % D) * Q4 + q0 + lq] =
                        make_int4(a[u].x + c.x, a[u].y + c.y, a[u].z + c.z, a[u].w + c.w);
                }
            }
        }
    }
    {
        uint32_t k = 0;
        for (uint32_t qc = qa; qc < qb; qc += 32, ++k) {
            const uint32_t q = qc + lane;
            uint32_t w9[9];
            tmem_ld9(tm_vc + 8u * k, tm_r + k, w9);
            if (q < qb) {
                QuadOut o;
                o.V = make_float4(__uint_as_float(w9[0]), __uint_as_float(w9[1]), __uint_as_float(w9[2]),
                                  __uint_as_float(w9[3]));
                o.C = make_float4(__uint_as_float(w9[4]), __uint_as_float(w9[5]), __uint_as_float(w9[6]),
                                  __uint_as_float(w9[7]));
                o.R = w9[8];
                store_state(v, q << 2, o);
            }
            __syncwarp();
        }
    }
    tmem_fence_before_sync();
    __syncthreads();
    tmem_fence_after_sync();
    if (warp == 0) tmem_dealloc(s_tmem, tcols);
    uint32_t e = ext;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
        rec += __shfl_xor_sync(0xFFFFFFFFu, rec, o);
    }
    if (lane == 0) {
        s_ext[warp] = e;
        s_rec[warp] = rec;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long be = 0, br = 0;
        for (int w = 0; w < PULL_WARPS; ++w) {
            be += s_ext[w];
            br += s_rec[w];
        }
        atomicAdd(reinterpret_cast<unsigned long long*>(&v.st->ext_events), be);
        if (v.row_len && br) atomicAdd(reinterpret_cast<unsigned long long*>(&v.st->rec_events), br);
        if (bid == 0 && done == n_steps) {
            DevState* st = v.st;
            st->t = t0 + n_steps;
            st->raster_count = rc;
            st->n_spikes += spikes;
            if (!v.row_len) st->rec_events += spikes * v.K;
            st->n_spk = 0;
            st->phase_ns[0] += ph_n;
            st->phase_ns[1] += ph_d;
        }
    }
}

static const void* pull_fn(bool bf16) {
    return bf16 ? (const void*)k_run_steps_pull<true> : (const void*)k_run_steps_pull<false>;
}

size_t pull_smem_bytes(uint32_t W, uint32_t BQ, int grid, uint32_t R_max) {
    return ((size_t)W * BQ * 4 + pull_aux_words((uint32_t)grid, R_max)) * sizeof(uint32_t);
}

uint32_t pull_warps() { return PULL_WARPS; }
uint32_t pull_mods_max() { return PULL_MODS_MAX; }
uint32_t pull_k_max() { return PULL_K_MAX; }

// Tensor-memory columns for bands of at most BQ quads (0: more than the 512 of
// an SM), and the chunks of 32 quads per warp they hold: a warp's share of a
// band is at most ceil(BQ / warps) quads, 9 columns per chunk, four warps per
// lane quarter.
uint32_t pull_tmem_cols(uint32_t BQ, uint32_t* chunks) {
    const uint32_t per_warp = (BQ + PULL_WARPS - 1) / PULL_WARPS;
    const uint32_t mc = std::max(1u, (per_warp + 31) / 32);
    *chunks = mc;
    const uint32_t need = 4u * 9u * mc;
    if (need > 512u) return 0;
    uint32_t cols = 32;
    while (cols < need) cols <<= 1;
    return cols;
}

// The runs of every band (band b = the quads [bq[b], bq[b + 1]) of Q): for
// each source module whose in-grid stencil reaches a module the band's
// neurons touch, the stencil entries [j0, j1) of those target modules.  The
// stencil offsets are in (dy, dx) raster order, so the in-grid entries of a
// source are in increasing target module order and [j0, j1) is contiguous.
// Entries are numbered over the in-grid offsets only (the fixed law's segment
// index), or, with all_entries, over every offset (the per-pair law's rows,
// whose out-of-grid entries are empty segments).  Returns R_max, the most
// runs of one band.
uint32_t pull_build_runs(uint32_t N, uint32_t M, uint32_t gw, uint32_t gh, const std::vector<int16_t>& off,
                         const std::vector<uint32_t>& bq, std::vector<uint2>& runs, std::vector<uint32_t>& ptr,
                         bool all_entries) {
    const uint32_t G = (uint32_t)bq.size() - 1;
    runs.clear();
    ptr.assign(G + 1, 0);
    int R = 0;  // row radius of the stencil
    for (size_t o = 0; o < off.size(); o += 2) R = std::max(R, std::abs((int)off[o + 1]));
    uint32_t R_max = 0;
    for (uint32_t b = 0; b < G; ++b) {
        ptr[b] = (uint32_t)runs.size();
        const uint32_t n0 = bq[b] * 4, n1 = std::min(bq[b + 1] * 4, N);
        if (n1 <= n0) continue;
        const uint32_t m_lo = n0 / M, m_hi = (n1 - 1) / M;
        const int y_lo = std::max(0, (int)(m_lo / gw) - R), y_hi = std::min((int)gh - 1, (int)(m_hi / gw) + R);
        for (int sy = y_lo; sy <= y_hi; ++sy)
            for (uint32_t sx = 0; sx < gw; ++sx) {
                uint32_t j = 0, j0 = 0, j1 = 0;
                for (size_t o = 0; o < off.size(); o += 2) {
                    const int tx = (int)sx + off[o], ty = sy + off[o + 1];
                    if (tx < 0 || ty < 0 || tx >= (int)gw || ty >= (int)gh) {
                        if (all_entries) {  // an empty segment: inside the range if a later entry is
                            if (j0 == j) j0 = j + 1;
                            ++j;
                        }
                        continue;
                    }
                    const uint32_t tm = (uint32_t)ty * gw + (uint32_t)tx;
                    if (tm < m_lo) j0 = j + 1;
                    if (tm <= m_hi) j1 = j + 1;
                    ++j;
                }
                if (j1 > j0) runs.push_back(make_uint2((uint32_t)sy * gw + sx, j0 | (j1 << 16)));
            }
        R_max = std::max<uint32_t>(R_max, (uint32_t)runs.size() - ptr[b]);
    }
    ptr[G] = (uint32_t)runs.size();
    return R_max;
}

// The bands: G contiguous ranges of quads, bq[0] = 0 and bq[G] = ceil(N / 4)
// (the padding quads up to Q hold no neuron, receive nothing and are left
// alone).  Uniform: ceil(N / 4 / G) quads each.  Module-aligned: every boundary
// falls on a module boundary that is also a quad boundary (every u-th module,
// u = 4 / gcd(M, 4)), the units of u modules split as evenly as possible; a
// band then reads no synapse of a module it does not own.
std::vector<uint32_t> pull_bands(uint32_t N, uint32_t M, uint32_t Q, uint32_t G, bool aligned) {
    Q = std::min(Q, (N + 3) / 4);
    std::vector<uint32_t> bq(G + 1, Q);
    bq[0] = 0;
    if (!aligned) {
        const uint32_t BQ = (Q + G - 1) / G;
        for (uint32_t b = 1; b < G; ++b) bq[b] = std::min(b * BQ, Q);
        return bq;
    }
    const uint32_t u = 4 / std::gcd(M, 4u);
    const uint32_t nm = (N + M - 1) / M, U = (nm + u - 1) / u;
    for (uint32_t b = 1; b < G; ++b) {
        const uint64_t unit = (uint64_t)U * b / G;
        bq[b] = (uint32_t)std::min<uint64_t>(unit * u * M / 4, Q);
    }
    return bq;
}

uint32_t pull_max_window(const NetView& v, int grid, uint32_t BQ, uint32_t R_max) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (grid <= 0 || BQ == 0 || v.D < 2) return 0;
    uint32_t best = 0;
    for (int bf = 0; bf < 2; ++bf) {
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, pull_fn(bf != 0)) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        const size_t aux = pull_smem_bytes(0, BQ, grid, R_max) + fa.sharedSizeBytes + 1024;  // + the runtime's own
        if (aux >= (size_t)optin) return 0;
        uint32_t W = (uint32_t)(((size_t)optin - aux) / ((size_t)BQ * 16));
        W = std::min<uint32_t>(W, v.D - 1);
        best = bf == 0 ? W : std::min(best, W);
    }
    for (; best > 0; --best) {  // one CTA per SM must fit at that shared memory
        const size_t smem = pull_smem_bytes(best, BQ, grid, R_max);
        bool ok = true;
        for (int bf = 0; bf < 2 && ok; ++bf) {
            int fit = 0;
            if (cudaFuncSetAttribute(pull_fn(bf != 0), cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
                    cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, pull_fn(bf != 0), PULL_THREADS, smem) !=
                    cudaSuccess ||
                fit < 1) {
                cudaGetLastError();
                ok = false;
            }
        }
        if (ok) return best;
    }
    return 0;
}

cudaError_t launch_pull(const NetView& v, uint32_t n_steps, int grid, cudaStream_t s) {
    const void* fn = pull_fn(v.w_bf16 != 0);
    const size_t smem = pull_smem_bytes(v.pull_W, v.pull_BQ, grid, v.pull_R_max);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // CTAs sharing an SM share its 512 tensor-memory columns: an allocation
    // waiting for another CTA's columns would wait at the grid barrier forever
    int fit = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, PULL_THREADS, smem);
    if (e != cudaSuccess) return e;
    if (fit < 1 || (uint64_t)fit * v.pull_tmem_cols > 512u || v.pull_tmem_cols < 32u) return cudaErrorInvalidConfiguration;
    NetView vv = v;
    uint32_t ns = n_steps;
    void* args[] = {&vv, &ns};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(PULL_THREADS), args, smem, s);
    count_launch(1);
    return e;
}

}  // namespace snn
