// persistent_owned.cu -- persistent multi-step kernel with band-owned delay windows.
//
// The push delivery of k_run_steps adds every synaptic event into the delay
// ring with one random L2 reduction, and on GB300 those top out near 2.2e11/s
// while the table stream alone could go several times faster.  Shared-memory
// atomics run at ~1.4e12/s, but the whole ring (D rows x N) is larger than
// all shared memory of the GPU together, so it cannot simply move there.
//
// Here every CTA owns a band of neurons -- the quads [b BQ, (b + 1) BQ) -- for
// the whole launch: it integrates them (flow steps 4-6, Sec. II-A) and keeps,
// in shared memory, the ring rows of the next W steps of its band (the delay
// window; W is as large as the shared memory allows, ~10 of the 20 delays of
// the benchmark network).  One time step is
//
//   N  each CTA integrates its band; the input of step t is window row t mod W,
//      which is then refilled with ring row (t + W) mod D of the band, the
//      step that enters the window (its events all arrived in earlier steps);
//   -- grid barrier --
//   A  push delivery, every CTA taking every G-th spike (flow steps 2-3): the
//      rows are streamed as in k_run_steps; an event with delay d > W is added
//      into the ring with an L2 reduction; one with d <= W becomes an 8-byte
//      record {window index, fixed-point weight} in the queue of (owner band,
//      this CTA), its position taken from a shared-memory counter per band
//      (one warp-aggregated atomic per band and instruction);
//   -- grid barrier --
//   B  each CTA applies the records queued for its band by every producer with
//      shared-memory atomics into its window, and goes on with step t + 1
//      without a barrier: nothing another CTA writes is read before the next
//      one.
//
// A queue that fills up (more than own_cap records from one producer for one
// band in one step) sends the rest of its events to the ring by reduction and
// flags the band; the owner then folds the ring rows of its window steps into
// the window in B.  At the start of a launch the window is loaded from the
// ring (and those ring cells cleared); at the end it is added back, so between
// launches the ring holds exactly what the push delivery would hold and every
// other call (state reads, snapshots, the other schedules) sees the same
// state.  Integer sums do not depend on the order, so results are bit-identical
// to every other schedule.
//
// Every barrier wait is bounded (grid_common.cuh); a CTA that gives up sets
// ERR_BARRIER_TIMEOUT and every CTA stops at its next barrier.
#include "grid_common.cuh"

#include <algorithm>

namespace snn {

#ifndef SNN_OWN_THREADS
#define SNN_OWN_THREADS 512
#endif
#ifndef SNN_OWN_UNROLL
#define SNN_OWN_UNROLL 2
#endif
constexpr int OWN_THREADS = SNN_OWN_THREADS;
constexpr int OWN_WARPS = OWN_THREADS / 32;
constexpr int OWN_UNROLL = SNN_OWN_UNROLL;  // delivery tasks in flight per warp
constexpr int OWN_DRV = 4;                  // chunks per thread whose next-step drive is drawn during delivery
constexpr int REC_UNROLL = 16;              // queued records in flight per lane in phase B

// Shared memory other than the window, in 32-bit words: per-warp spike
// offsets (TW + 1), staged spike ids, per-band record counters (G), the
// owner's prefix over producers (G + 1), drawn-ahead drives; padded to 16 B.
__host__ __device__ constexpr uint32_t owned_aux_words(uint32_t G) {
    return ((G * OWN_WARPS + 1) + OWN_THREADS + G + (G + 1) + OWN_DRV * OWN_THREADS + 3) & ~3u;
}

// First quad of global warp wg: warp w of CTA b covers its share of the band.
__device__ __forceinline__ uint32_t owned_warp_q(uint32_t wg, uint32_t BQ, uint32_t Q) {
    const uint32_t b = wg / OWN_WARPS, w = wg - b * OWN_WARPS;
    const uint32_t q0 = min(b * BQ, Q), q1 = min(q0 + BQ, Q);
    return q0 + (q1 - q0) * w / OWN_WARPS;
}

// Neuron id of spike j of the step: its warp by binary search over the
// per-warp prefix, then that warp's staging segment.
__device__ __forceinline__ uint32_t owned_spike_id(const NetView& v, const uint32_t* s_wpre, uint32_t TW, uint32_t Q,
                                                   uint32_t j) {
    uint32_t lo = 0, hi = TW;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_wpre[mid] <= j)
            lo = mid;
        else
            hi = mid;
    }
    return __ldcg(v.seg + ((size_t)owned_warp_q(lo, v.own_BQ, Q) << 2) + (j - s_wpre[lo]));
}

// L2 reduction without a compiler memory barrier: nothing in the delivery
// phase reads the ring, so the reductions may be scheduled freely around the
// queue bookkeeping (the grid barrier after the phase orders them).
__device__ __forceinline__ void red_add_free(int32_t* p, int32_t v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v));
}

// One warp delivers up to OWN_UNROLL tasks (spike, 128-synapse chunk), task
// tk + u * tstride below `hi` (local spike jj = task / chunks, with
// inv_chunks = 1 / chunks rounded up); ids[jj - j0] is the neuron of local
// spike jj.  Far events (delay > W) go to the ring, near ones to the owners'
// queues: the reductions are issued first, then the band of every near event
// is matched across the warp, one shared-memory atomic per band reserves the
// queue positions, and the records are stored.
template <bool BF16, class Hook>
__device__ __forceinline__ void deliver_owned(const NetView& v, uint32_t tk, uint32_t tstride, uint32_t hi,
                                              uint32_t chunks, float inv_chunks, const uint32_t* ids, uint32_t j0,
                                              uint32_t slot0, uint32_t wbase, uint32_t lane, uint64_t pol,
                                              uint32_t* s_bcnt, uint32_t bid, uint32_t G, Hook hook) {
    constexpr int NE = OWN_UNROLL * 4;
    uint4 tg[OWN_UNROLL];
    uint4 wr[OWN_UNROLL];
    uint32_t nv[OWN_UNROLL];
#pragma unroll
    for (int u = 0; u < OWN_UNROLL; ++u) {
        const uint32_t task = tk + (uint32_t)u * tstride;
        nv[u] = 0;
        if (task < hi) {
            uint32_t jj = __float2uint_rz(__fmul_rz(__uint2float_rz(task), inv_chunks));
            if (jj * chunks > task) --jj;
            if ((jj + 1) * chunks <= task) ++jj;
            const uint32_t ch = task - jj * chunks;
            const uint32_t k0 = (ch << 7) + (lane << 2);
            const uint32_t id = ids[jj - j0];
            const uint32_t L = v.row_len ? __ldg(v.row_len + id) : v.K;
            if (k0 < L) {
                nv[u] = min(4u, L - k0);
                const size_t e = (size_t)id * v.Kpad + k0;
                tg[u] = ld_u4(v.td + e, pol);
                if (BF16) {
                    const uint2 wb = ld_u2(reinterpret_cast<const uint16_t*>(v.w) + e, pol);
                    wr[u] = make_uint4(wb.x, wb.y, 0u, 0u);
                } else {
                    wr[u] = ld_u4(reinterpret_cast<const float*>(v.w) + e, pol);
                }
            }
        }
    }
    hook();
    const uint32_t W = v.own_W, BQ = v.own_BQ, BN = BQ << 2, cap = v.own_cap;
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t key[NE], widx[NE];
    int32_t fx[NE];
    // far events to the ring; near events: owner band and window index
#pragma unroll
    for (int u = 0; u < OWN_UNROLL; ++u) {
        const uint32_t tq[4] = {tg[u].x, tg[u].y, tg[u].z, tg[u].w};
        const uint32_t wq[4] = {wr[u].x, wr[u].y, wr[u].z, wr[u].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int i = u * 4 + q;
            const bool valid = (uint32_t)q < nv[u];
            const uint32_t tgt = tq[q] & 0xFFFFFFu, d = tq[q] >> 24;
            const float wv = BF16 ? ((q & 1) ? bf16_hi(wq[q >> 1]) : bf16_lo(wq[q >> 1])) : __uint_as_float(wq[q]);
            fx[i] = fx_weight(v, wv);
            key[i] = 0xFFFFFFFFu;
            widx[i] = 0;
            if (valid) {
                if (d > W) {
                    uint32_t s = slot0 + d;
                    if (s >= v.D) s -= v.D;
                    if (SNN_BOUND(v.st, s < v.D && tgt < v.N)) red_add_free(v.ring + (size_t)s * v.Npad + tgt, fx[i]);
                } else {
                    const uint32_t qt = tgt >> 2;
                    uint32_t b = (uint32_t)(((uint64_t)qt * v.own_magic) >> 32);
                    if (b * BQ > qt) --b;
                    uint32_t ws = wbase + d;
                    if (ws >= W) ws -= W;
                    key[i] = SNN_BOUND(v.st, b < G && tgt < v.N) ? b : 0xFFFFFFFFu;
                    widx[i] = ws * BN + (tgt - b * BN);
                }
            }
        }
    }
    // one shared-memory atomic per owner band and event slot across the warp
    uint32_t peers[NE], pos[NE];
#pragma unroll
    for (int i = 0; i < NE; ++i) peers[i] = __match_any_sync(0xFFFFFFFFu, key[i]);
#pragma unroll
    for (int i = 0; i < NE; ++i) {
        const uint32_t leader = __ffs(peers[i]) - 1;
        pos[i] = 0;
        if (key[i] != 0xFFFFFFFFu && lane == leader) pos[i] = atomicAdd(s_bcnt + key[i], (uint32_t)__popc(peers[i]));
    }
#pragma unroll
    for (int i = 0; i < NE; ++i) {
        const uint32_t leader = __ffs(peers[i]) - 1;
        const uint32_t base = __shfl_sync(0xFFFFFFFFu, pos[i], leader);
        if (key[i] != 0xFFFFFFFFu) {
            const uint32_t p = base + __popc(peers[i] & lt);
            const uint32_t b = key[i];
            if (p < cap) {
                *reinterpret_cast<int2*>(v.own_rec + ((size_t)b * G + bid) * cap + p) = make_int2((int32_t)widx[i], fx[i]);
            } else {  // queue full: the event goes to the ring; the owner folds it in
                const uint32_t tgt = b * BN + (widx[i] % BN);
                uint32_t ws = widx[i] / BN;  // window slot (t + d) mod W -> ring row (t + d) mod D
                uint32_t d = ws >= wbase ? ws - wbase : ws + W - wbase;
                if (d == 0) d = W;
                uint32_t s = slot0 + d;
                if (s >= v.D) s -= v.D;
                red_add_free(v.ring + (size_t)s * v.Npad + tgt, fx[i]);
                v.own_ovf[b] = 1u;
            }
        }
    }
}

template <bool BF16>
__global__ void __launch_bounds__(OWN_THREADS, 1) k_run_steps_owned(NetView v, uint32_t n_steps) {
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t G = gridDim.x, bid = blockIdx.x, tid = threadIdx.x;
    const uint32_t TW = G * OWN_WARPS;
    const uint32_t Q = v.Npad >> 2;
    const uint32_t W = v.own_W, BQ = v.own_BQ;
    const uint32_t q0 = min(bid * BQ, Q), q1 = min(q0 + BQ, Q), nq = q1 - q0;  // this CTA's band
    int4* win4 = reinterpret_cast<int4*>(smem);  // W rows of BQ quads
    int32_t* win = reinterpret_cast<int32_t*>(smem);
    uint32_t* s_wpre = smem + (size_t)W * BQ * 4;  // TW + 1
    uint32_t* s_id = s_wpre + TW + 1;              // OWN_THREADS
    uint32_t* s_bcnt = s_id + OWN_THREADS;         // G
    uint32_t* s_rpre = s_bcnt + G;                 // G + 1
    uint32_t* s_drv = s_rpre + G + 1;              // OWN_DRV x OWN_THREADS
    __shared__ uint32_t s_t0, s_ovf;
    __shared__ unsigned long long s_rc0;
    __shared__ uint32_t s_ext[OWN_WARPS];
    __shared__ unsigned long long s_rec[OWN_WARPS];
    __shared__ uint32_t s_pois[MAX_POIS];
    load_poisson_table(v, s_pois);
    uint32_t gen = 0;
    if (tid == 0) {
        s_t0 = v.st->t;
        s_rc0 = v.st->raster_count;
    }
    __syncthreads();
    const uint32_t t0 = s_t0;
    const uint32_t lane = tid & 31, warp = tid >> 5;
    const uint32_t wg = bid * OWN_WARPS + warp;
    const uint32_t qa = q0 + nq * warp / OWN_WARPS, qb = q0 + nq * (warp + 1) / OWN_WARPS;
    const uint64_t pol = evict_first_policy();
    int4* ring4 = reinterpret_cast<int4*>(v.ring);
    const uint32_t Q4 = v.Npad >> 2;  // int4 per ring row

    // the window starts as ring rows t0 .. t0 + W - 1 of the band
    for (uint32_t x = tid; x < W * nq; x += OWN_THREADS) {
        const uint32_t k = x / nq, lq = x - k * nq;
        const size_t g = (size_t)((t0 + k) % v.D) * Q4 + q0 + lq;
        win4[(size_t)((t0 + k) % W) * BQ + lq] = __ldcg(ring4 + g);
        ring4[g] = make_int4(0, 0, 0, 0);
    }
    __syncthreads();

    const uint32_t chunks = (v.K + 127) >> 7;
    const float inv_chunks = chunks ? __frcp_ru((float)chunks) : 0.0f;
    uint64_t rc = s_rc0;
    uint64_t spikes = 0;
    uint32_t ext = 0;
    uint64_t rec = 0;
    uint32_t done = 0;
    uint64_t ph_n = 0, ph_d = 0, stamp = 0;
    if (bid == 0 && tid == 0) stamp = global_ns();
    const uint32_t nchunk = qa + lane < qb ? (qb - qa - lane + 31) / 32 : 0u;
    const uint32_t nd_max = nchunk < (uint32_t)OWN_DRV ? nchunk : (uint32_t)OWN_DRV;
    uint32_t ndrv = 0;  // chunks whose drive for the coming step is in s_drv
    auto drive_of = [&](uint32_t k, uint32_t tt) -> uint32_t {
        return k < ndrv ? s_drv[k * OWN_THREADS + tid] : quad_drive(v, s_pois, (qa + lane + 32 * k) << 2, tt);
    };

    for (uint32_t step = 0; step < n_steps; ++step) {
        const uint32_t t = t0 + step;
        const uint32_t wslot = t % W;
        const uint32_t rfar = (t + W) % v.D;  // ring row of the step entering the window
        // ---- phase N: the band's neurons, spikes compacted in id order per warp
        uint32_t run = 0;
        {
            QuadIn nx;
            int4 nF = make_int4(0, 0, 0, 0);
            auto load_in = [&](uint32_t q, uint32_t k, QuadIn& in, int4& F) {
                load_state(v, q << 2, in);
                F = __ldcg(ring4 + (size_t)rfar * Q4 + q);
                in.drive = drive_of(k, t);
            };
            if (qa + lane < qb) load_in(qa + lane, 0, nx, nF);
            uint32_t k = 0;
            for (uint32_t qc = qa; qc < qb; qc += 32, ++k) {
                const uint32_t q = qc + lane;
                QuadIn cur = nx;
                const int4 cF = nF;
                if (q + 32 < qb) load_in(q + 32, k + 1, nx, nF);
                uint32_t spk = 0;
                if (q < qb) {
                    int4* wp = win4 + (size_t)wslot * BQ + (q - q0);
                    cur.I = *wp;
                    *wp = cF;  // step t + W enters the window
                    ring4[(size_t)rfar * Q4 + q] = make_int4(0, 0, 0, 0);
                    QuadOut o;
                    spk = integrate_quad<false>(v, q << 2, 0u, cur, ext, rec, o);
                    store_state(v, q << 2, o);
                }
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
                    if (spk & (1u << b)) v.seg[pos++] = (q << 2) + b;
                run += __shfl_sync(0xFFFFFFFFu, incl, 31);
            }
        }
        if (lane == 0) v.woff[wg] = run;
        if (!grid_barrier(v, G, gen)) break;
        if (bid == 0 && tid == 0) {
            const uint64_t now = global_ns();
            ph_n += now - stamp;
            stamp = now;
        }

        // ---- phase A: every G-th spike of the step, pushed; near events queued
        ndrv = 0;
        const bool next = step + 1 < n_steps;
        auto draw_next = [&]() {
            if (next && ndrv < nd_max) {
                s_drv[ndrv * OWN_THREADS + tid] = quad_drive(v, s_pois, (qa + lane + 32 * ndrv) << 2, t + 1);
                ++ndrv;
            }
        };
        for (uint32_t b = tid; b < G; b += OWN_THREADS) s_bcnt[b] = 0;
        block_exclusive_scan(v.woff, TW, s_wpre);  // ends with a CTA barrier
        const uint32_t total = s_wpre[TW];
        const uint32_t slot0 = t % v.D;
        const uint32_t nl = total > bid ? (total - bid - 1) / G + 1 : 0u;  // spikes j = bid + G li
        for (uint32_t lb = 0; lb < nl; lb += OWN_THREADS) {
            const uint32_t li = lb + tid;
            if (li < nl) {
                const uint32_t j = bid + G * li;
                const uint32_t id = owned_spike_id(v, s_wpre, TW, Q, j);
                s_id[tid] = id;
                const uint64_t r = rc + j;
                if (r < v.raster_cap) {
                    v.raster_t[r] = t;
                    v.raster_id[r] = id;
                }
            }
            __syncthreads();
            if (chunks > 0) {
                const uint32_t lo = lb * chunks;
                const uint32_t hi = min(nl, lb + OWN_THREADS) * chunks;
                for (uint32_t tk = lo + warp; tk < hi; tk += OWN_WARPS * OWN_UNROLL)
                    deliver_owned<BF16>(v, tk, OWN_WARPS, hi, chunks, inv_chunks, s_id, lb, slot0, wslot, lane, pol,
                                        s_bcnt, bid, G, draw_next);
            }
            __syncthreads();
        }
        for (uint32_t b = tid; b < G; b += OWN_THREADS) v.own_cnt[(size_t)b * G + bid] = s_bcnt[b];
        rc += total;
        spikes += total;
        if (!grid_barrier(v, G, gen)) break;

        // ---- phase B: this band's queues into the window
        for (uint32_t p = tid; p < G; p += OWN_THREADS) s_rpre[p] = min(__ldcg(v.own_cnt + (size_t)bid * G + p), v.own_cap);
        if (tid == 0) s_ovf = __ldcg(v.own_ovf + bid);
        __syncthreads();
        block_scan_inplace(s_rpre, G);  // exclusive, s_rpre[G] = records
        {
            const uint32_t R = s_rpre[G];
            const uint32_t e0 = (uint32_t)((uint64_t)R * warp / OWN_WARPS);
            const uint32_t e1 = (uint32_t)((uint64_t)R * (warp + 1) / OWN_WARPS);
            uint32_t pp = 0;  // producer of the lane's next record: largest p with s_rpre[p] <= e
            {
                const uint32_t e = e0 + lane;
                uint32_t lo = 0, hi = G;
                while (hi - lo > 1) {
                    const uint32_t mid = (lo + hi) >> 1;
                    if (s_rpre[mid] <= e)
                        lo = mid;
                    else
                        hi = mid;
                }
                pp = lo;
            }
            const int2* qbase = v.own_rec + (size_t)bid * G * v.own_cap;
            for (uint32_t base = e0; base < e1; base += 32 * REC_UNROLL) {
                int2 r[REC_UNROLL];
#pragma unroll
                for (int u = 0; u < REC_UNROLL; ++u) {
                    const uint32_t e = base + u * 32 + lane;
                    r[u] = make_int2(-1, 0);
                    if (e < e1) {
                        while (pp + 1 < G && s_rpre[pp + 1] <= e) ++pp;
                        r[u] = __ldcg(qbase + (size_t)pp * v.own_cap + (e - s_rpre[pp]));
                    }
                }
#pragma unroll
                for (int u = 0; u < REC_UNROLL; ++u)
                    if (r[u].x >= 0 && SNN_BOUND(v.st, (uint32_t)r[u].x < W * BQ * 4)) atomicAdd(win + r[u].x, r[u].y);
            }
        }
        if (s_ovf) {  // some events for this band went to the ring: fold the window's rows in
            __syncthreads();
            for (uint32_t x = tid; x < W * nq; x += OWN_THREADS) {
                const uint32_t k = x / nq, lq = x - k * nq;
                const uint32_t ts = t + 1 + k;
                const size_t g = (size_t)(ts % v.D) * Q4 + q0 + lq;
                const int4 a = __ldcg(ring4 + g);
                int4* wp = win4 + (size_t)(ts % W) * BQ + lq;
                int4 c = *wp;
                c.x += a.x;
                c.y += a.y;
                c.z += a.z;
                c.w += a.w;
                *wp = c;
                ring4[g] = make_int4(0, 0, 0, 0);
            }
            if (tid == 0) v.own_ovf[bid] = 0u;
        }
        __syncthreads();  // the window holds every input of step t + 1
        if (bid == 0 && tid == 0) {
            const uint64_t now = global_ns();
            ph_d += now - stamp;
            stamp = now;
        }
        done = step + 1;
    }

    // ---- epilogue: the window back into the ring, counters of the launch
    __syncthreads();
    {
        const uint32_t te = t0 + done;
        for (uint32_t x = tid; x < W * nq; x += OWN_THREADS) {
            const uint32_t k = x / nq, lq = x - k * nq;
            const size_t g = (size_t)((te + k) % v.D) * Q4 + q0 + lq;
            const int4 a = __ldcg(ring4 + g);
            const int4 c = win4[(size_t)((te + k) % W) * BQ + lq];
            ring4[g] = make_int4(a.x + c.x, a.y + c.y, a.z + c.z, a.w + c.w);
        }
    }
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
        for (int w = 0; w < OWN_WARPS; ++w) {
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

static const void* owned_fn(bool bf16) {
    return bf16 ? (const void*)k_run_steps_owned<true> : (const void*)k_run_steps_owned<false>;
}

size_t owned_smem_bytes(uint32_t W, uint32_t BQ, int grid) {
    return ((size_t)W * BQ * 4 + owned_aux_words((uint32_t)grid)) * sizeof(uint32_t);
}

int owned_grid() {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    return sms;
}

uint32_t owned_max_window(const NetView& v, int grid, uint32_t BQ) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (grid <= 0 || BQ == 0 || v.D < 2) return 0;
    uint32_t best = 0;
    for (int bf = 0; bf < 2; ++bf) {
        const void* fn = owned_fn(bf != 0);
        cudaFuncAttributes fa{};
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess) {
            cudaGetLastError();
            return 0;
        }
        const size_t aux = owned_smem_bytes(0, BQ, grid) + fa.sharedSizeBytes + 1024;  // + the runtime's own
        if (aux >= (size_t)optin) return 0;
        uint32_t W = (uint32_t)(((size_t)optin - aux) / ((size_t)BQ * 16));
        W = std::min<uint32_t>(W, v.D - 1);
        best = bf == 0 ? W : std::min(best, W);
    }
    // the co-residency of one CTA per SM at that shared memory
    for (; best > 0; --best) {
        const size_t smem = owned_smem_bytes(best, BQ, grid);
        bool ok = true;
        for (int bf = 0; bf < 2 && ok; ++bf) {
            const void* fn = owned_fn(bf != 0);
            int fit = 0;
            if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess ||
                cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, OWN_THREADS, smem) != cudaSuccess || fit < 1) {
                cudaGetLastError();
                ok = false;
            }
        }
        if (ok) return best;
    }
    return 0;
}

cudaError_t launch_owned(const NetView& v, uint32_t n_steps, int grid, cudaStream_t s) {
    const void* fn = owned_fn(v.w_bf16 != 0);
    const size_t smem = owned_smem_bytes(v.own_W, v.own_BQ, grid);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    NetView vv = v;
    uint32_t ns = n_steps;
    void* args[] = {&vv, &ns};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(OWN_THREADS), args, smem, s);
    count_launch(1);
    return e;
}

}  // namespace snn
