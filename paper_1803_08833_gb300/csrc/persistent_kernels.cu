// persistent_kernels.cu -- many simulation time steps in one cooperative launch.
//
// The per-step kernels pay, every 1 ms step, two launches and the latency
// chains of their prologue/epilogue.  k_run_steps keeps one resident grid for
// n steps: phase N (flow steps 1, 4-6: every neuron integrates, spikes are
// compacted in id order per warp-owned neuron range), a grid barrier, phase D
// (flow steps 2-4: the spikes' synapses are added into the delay ring, raster
// entries written), a grid barrier.  Results are identical to the per-step
// kernels: the same update, the same (step, id) spike order, the same integer
// sums.  Work that depends on no other CTA is moved off the critical path:
// the next step's external drive is drawn between delivery loads and their
// reductions, and the state of each warp's first neuron chunks is loaded
// between arriving at the step's last barrier and waiting on it.
//
// Every barrier wait is bounded by v.wait_limit_ns of %globaltimer: a CTA that
// waits longer sets ERR_BARRIER_TIMEOUT in the device state and returns, and
// every CTA stops at its next barrier once the flag is set; the host reports
// SNN_ETIMEOUT.
#include "grid_common.cuh"

#include <algorithm>

namespace snn {

constexpr int MAX_DRV = 8;  // chunks per thread whose external drive is drawn ahead
constexpr uint32_t REBALANCE_STEPS = 32;  // steps between re-weightings of the delivery split
constexpr uint32_t MIN_SPEED_TASKS = 64;   // tasks a CTA must have delivered for its speed to count
constexpr int PF_CHUNKS = 5;  // resident state: a warp with at most this many chunks loads all its ring slots at once

#ifndef SNN_PERSIST_MIN_BLOCKS
#define SNN_PERSIST_MIN_BLOCKS 1  // one CTA per SM: registers for deep delivery unrolling
#endif

// Neuron id of staged spike j: the warp by binary search over the per-warp
// spike prefix, then that warp's staging segment.
__device__ __forceinline__ uint32_t warp_spike_id(const NetView& v, const uint32_t* s_wpre, uint32_t TW, uint32_t Q,
                                                  uint32_t j) {
    uint32_t lo = 0, hi = TW;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_wpre[mid] <= j)
            lo = mid;
        else
            hi = mid;
    }
    const uint32_t qa = (uint32_t)((uint64_t)Q * lo / TW);
    return __ldcg(v.seg + ((size_t)qa << 2) + (j - s_wpre[lo]));
}

// The warp (of TW) whose quad range [Q w / TW, Q (w + 1) / TW) holds neuron id
// (TW if the neuron is past the last quad).
__device__ __forceinline__ uint32_t warp_of_neuron(uint32_t id, uint32_t Q, uint32_t TW) {
    const uint32_t qd = id >> 2;
    if (qd >= Q) return TW;
    uint32_t w = (uint32_t)((uint64_t)qd * TW / Q);
    while (w > 0 && (uint32_t)((uint64_t)Q * w / TW) > qd) --w;
    while (w + 1 < TW && (uint32_t)((uint64_t)Q * (w + 1) / TW) <= qd) ++w;
    return w;
}

// Dynamic shared memory of run_steps on G CTAs: per-warp offsets (TW + 1),
// staged ids and band ranges (3 x threads), split weights (G + 1), padded to
// 16 B; then the resident state (36 B per quad) when there is one.
__host__ __device__ constexpr uint32_t state_offset_words(uint32_t G) {
    return (G * (PERSIST_WARPS + 1) + 2 + 3 * PERSIST_THREADS + 3) & ~3u;
}

// Delivery split weights: the CTAs' measured speeds (v.cta_speed, G words; 0
// = not measured, replaced by the mean of the measured ones) as an inclusive
// prefix s_wp[0..G], s_wp[0] = 0.  Every CTA computes the same prefix from the
// same words, so the task ranges still partition the task space.
__device__ inline void load_split_weights(const NetView& v, uint32_t G, uint32_t* s_wp) {
    __shared__ unsigned long long s_sum;
    __shared__ uint32_t s_cnt;
    if (threadIdx.x == 0) {
        s_sum = 0;
        s_cnt = 0;
    }
    __syncthreads();
    unsigned long long sum = 0;
    uint32_t cnt = 0;
    for (uint32_t i = threadIdx.x; i < G; i += blockDim.x) {
        const uint32_t w = __ldcg(v.cta_speed + i);
        s_wp[i] = w;
        sum += w;
        cnt += w != 0;
    }
    if (sum) atomicAdd(&s_sum, sum);
    if (cnt) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    const uint32_t mean = s_cnt ? (uint32_t)(s_sum / s_cnt) : 1u;
    for (uint32_t i = threadIdx.x; i < G; i += blockDim.x)
        if (s_wp[i] == 0) s_wp[i] = mean > 0 ? mean : 1u;
    __syncthreads();
    block_scan_inplace(s_wp, G);
}

// n_steps time steps of network v on a group of G CTAs; `bid` is this CTA's
// index in the group.  smem: persistent_smem(G) bytes, then 36 B per quad of
// resident neuron state for up to v.res_quads quads.
//
// Resident state: a CTA's neurons never change owner during a launch, so a
// CTA whose quads fit (at most v.res_quads) copies their V, c and ref into
// shared memory at the start, integrates them there, and writes them back at
// the end; its neuron phase then reads only the ring slot and the drive from
// memory.  A CTA whose quads do not fit keeps them in global memory.
//
// The delivery tasks of a step are split over the CTAs in proportion to each
// CTA's measured delivery speed (tasks per ns over the last REBALANCE_STEPS
// steps; equal shares until the first measurement): the SMs of one GB300 do
// not deliver equally fast (a stable 15 % spread between SMs at the same
// task count), and with an even split every step waits for the slowest.
template <bool BF16, bool BANDED>
__device__ __forceinline__ void run_steps(const NetView& v, uint32_t n_steps, uint32_t G, uint32_t bid,
                                          uint32_t* smem) {
    const uint32_t TW = G * PERSIST_WARPS;
    uint32_t* s_wpre = smem;          // TW + 1 per-warp spike offsets
    uint32_t* s_id = s_wpre + TW + 1;  // staged spike ids
    uint32_t* s_lo = s_id + PERSIST_THREADS;  // banded delivery: synapse range of each staged spike
    uint32_t* s_hi = s_lo + PERSIST_THREADS;
    uint32_t* s_wp = s_hi + PERSIST_THREADS;  // G + 1: prefix of the delivery split weights
    for (uint32_t i = threadIdx.x; i <= G; i += blockDim.x) s_wp[i] = i;
    float4* s_V = reinterpret_cast<float4*>(smem + state_offset_words(G));  // resident state
    float4* s_C = s_V + v.res_quads;
    uint32_t* s_R = reinterpret_cast<uint32_t*>(s_C + v.res_quads);
    __shared__ uint32_t s_t0;
    __shared__ unsigned long long s_rc0;
    __shared__ uint32_t s_ext[PERSIST_WARPS];
    __shared__ uint32_t s_pois[MAX_POIS];
    load_poisson_table(v, s_pois);
    uint32_t gen = 0;
    if (threadIdx.x == 0) {
        s_t0 = v.st->t;
        s_rc0 = v.st->raster_count;
    }
    __syncthreads();
    const uint32_t t0 = s_t0;
    const uint32_t lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t wg = bid * PERSIST_WARPS + warp;
    const uint32_t Q = v.Npad >> 2;
    const uint32_t qa = (uint32_t)((uint64_t)Q * wg / TW);
    const uint32_t qb = (uint32_t)((uint64_t)Q * (wg + 1) / TW);
    const uint64_t pol = evict_first_policy();
    // this CTA's quads (the union of its warps' ranges)
    const uint32_t cq0 = (uint32_t)((uint64_t)Q * (bid * PERSIST_WARPS) / TW);
    const uint32_t cq1 = (uint32_t)((uint64_t)Q * (bid * PERSIST_WARPS + PERSIST_WARPS) / TW);
    const bool res = cq1 - cq0 <= v.res_quads;  // this CTA's state fits the launch's shared memory
    if (res) {
        for (uint32_t q = cq0 + threadIdx.x; q < cq1; q += blockDim.x) {
            s_V[q - cq0] = *reinterpret_cast<const float4*>(v.V + ((size_t)q << 2));
            s_C[q - cq0] = *reinterpret_cast<const float4*>(v.c + ((size_t)q << 2));
            s_R[q - cq0] = *reinterpret_cast<const uint32_t*>(v.ref + ((size_t)q << 2));
        }
        __syncthreads();
    }
    auto load_st = [&](uint32_t q, QuadIn& in) {
        if (res) {
            in.V = s_V[q - cq0];
            in.C = s_C[q - cq0];
            in.R = s_R[q - cq0];
        } else {
            load_state(v, q << 2, in);
        }
    };
    const uint32_t chunks = (v.K + 127) >> 7;
    uint64_t rc = s_rc0;
    uint64_t spikes = 0;
    uint32_t ext = 0;
    uint64_t rec = 0;  // pairwise rule: row lengths of this thread's spikes
    uint32_t done = 0;
    uint64_t ph_n = 0, ph_d = 0, stamp = 0;
    uint64_t d_ns = 0, d_tasks = 0, d_t0 = 0;  // thread 0: this CTA's delivery time and tasks since the last weighting
    if (bid == 0 && threadIdx.x == 0) stamp = global_ns();
    // External drives of step t + 1 are drawn during the delivery of step t,
    // between each delivery round's table loads and its reductions (the ALU
    // is idle there), for up to MAX_DRV chunks of each thread; the rest are
    // drawn in the neuron phase.
    __shared__ uint32_t s_drv[MAX_DRV * PERSIST_THREADS];
    const uint32_t nchunk = qa + lane < qb ? (qb - qa - lane + 31) / 32 : 0u;
    const uint32_t nd_max = nchunk < (uint32_t)MAX_DRV ? nchunk : (uint32_t)MAX_DRV;
    uint32_t ndrv = 0;  // chunks whose drive for the coming step is in s_drv
    auto drive_of = [&](uint32_t k, uint32_t tt) -> uint32_t {
        return k < ndrv ? s_drv[k * PERSIST_THREADS + threadIdx.x]
                        : quad_drive(v, s_pois, (qa + lane + 32 * k) << 2, tt);
    };
    // The first two chunks of every warp are prepared ahead: their state and
    // external drive do not depend on other CTAs, so for step t + 1 they are
    // loaded while this CTA waits at the barrier that ends step t.
    QuadIn n1, n2;
    const uint32_t qa0 = qa + lane, qa1 = qa + 32 + lane;
    auto prepare = [&](uint32_t tt) {
        if (qa0 < qb) {
            load_st(qa0, n1);
            n1.drive = drive_of(0, tt);
        }
        if (qa1 < qb) {
            load_st(qa1, n2);
            n2.drive = drive_of(1, tt);
        }
    };
    prepare(t0);
    for (uint32_t step = 0; step < n_steps; ++step) {
        const uint32_t t = t0 + step;
        const uint32_t slot = t % v.D;
        // ---- phase N: this warp's neurons, 4 per lane, spikes compacted in id order
        uint32_t run = 0;
        // Compacts this lane's spikes of chunk quad q into the warp's staging, in id order.
        auto stage = [&](uint32_t q, uint32_t spk) {
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
                    if (SNN_BOUND(v.st, pos < (qb << 2))) v.seg[pos] = (q << 2) + b;
                    ++pos;
                }
            run += __shfl_sync(0xFFFFFFFFu, incl, 31);
        };
        if (res && qb - qa <= 32u * PF_CHUNKS) {
            // resident state and few chunks: every ring-slot load of the warp is in
            // flight at once (one L2 round trip), then the chunks are integrated
            int4 Ipf[PF_CHUNKS];
#pragma unroll
            for (int c = 0; c < PF_CHUNKS; ++c)
                if (qa + 32u * c + lane < qb) Ipf[c] = load_slot(v, (qa + 32u * c + lane) << 2, slot);
            // external drives not drawn ahead are drawn while the loads are in flight
            uint32_t drv[PF_CHUNKS];
#pragma unroll
            for (int c = 0; c < PF_CHUNKS; ++c) {
                drv[c] = 0;
                if (qa + 32u * c + lane < qb) drv[c] = c == 0 ? n1.drive : c == 1 ? n2.drive : drive_of(c, t);
            }
#pragma unroll
            for (int c = 0; c < PF_CHUNKS; ++c) {
                const uint32_t q = qa + 32u * c + lane;
                if (qa + 32u * c >= qb) break;  // warp-uniform
                uint32_t spk = 0;
                if (q < qb) {
                    QuadIn in;
                    if (c == 0) {
                        in = n1;  // state prepared while waiting at the last barrier
                    } else if (c == 1) {
                        in = n2;
                    } else {
                        load_st(q, in);
                    }
                    in.I = Ipf[c];
                    in.drive = drv[c];
                    QuadOut o;
                    spk = integrate_quad(v, q << 2, slot, in, ext, rec, o);
                    s_V[q - cq0] = o.V;
                    s_C[q - cq0] = o.C;
                    s_R[q - cq0] = o.R;
                }
                stage(q, spk);
            }
        } else {
            // the loads of the next two chunks are in flight while a chunk is integrated
            if (qa0 < qb) n1.I = load_slot(v, qa0 << 2, slot);
            if (qa1 < qb) n2.I = load_slot(v, qa1 << 2, slot);
            uint32_t k = 0;
            for (uint32_t qc = qa; qc < qb; qc += 32, ++k) {
                const uint32_t q = qc + lane;
                const QuadIn cur = n1;
                n1 = n2;
                if (q + 64 < qb) {
                    n2.I = load_slot(v, (q + 64) << 2, slot);
                    load_st(q + 64, n2);
                    n2.drive = drive_of(k + 2, t);
                }
                uint32_t spk = 0;
                if (q < qb) {
                    QuadOut o;
                    spk = integrate_quad(v, q << 2, slot, cur, ext, rec, o);
                    if (res) {
                        s_V[q - cq0] = o.V;
                        s_C[q - cq0] = o.C;
                        s_R[q - cq0] = o.R;
                    } else {
                        store_state(v, q << 2, o);
                    }
                }
                stage(q, spk);
            }
        }
        if (lane == 0) v.woff[wg] = run;  // spike count of this warp
        const bool reweigh = step > 0 && step % REBALANCE_STEPS == 0;
        if (reweigh && threadIdx.x == 0) {
            v.cta_speed[bid] = d_tasks >= MIN_SPEED_TASKS
                                   ? (uint32_t)min((d_tasks << 20) / max(d_ns, (uint64_t)1), (uint64_t)1 << 20) | 1u
                                   : 0u;
            d_ns = 0;
            d_tasks = 0;
        }
        if (!grid_barrier(v, G, gen)) break;
        if (bid == 0 && threadIdx.x == 0) {
            const uint64_t now = global_ns();
            ph_n += now - stamp;
            stamp = now;
        }

        // ---- phase D: per-warp offsets (one coalesced pass), delivery, raster
        ndrv = 0;
        const bool next = step + 1 < n_steps;
        auto draw_next = [&]() {
            if (next && ndrv < nd_max) {
                s_drv[ndrv * PERSIST_THREADS + threadIdx.x] =
                    quad_drive(v, s_pois, (qa + lane + 32 * ndrv) << 2, t + 1);
                ++ndrv;
            }
        };
        block_exclusive_scan(v.woff, TW, s_wpre);
        if (reweigh) load_split_weights(v, G, s_wp);
        const uint32_t total = s_wpre[TW];
        if (threadIdx.x == 0) (void)SNN_BOUND(v.st, total <= v.N);  // at most one spike per neuron and step
        const uint32_t slot0 = t % v.D;
        const uint64_t wa = s_wp[bid], wb = s_wp[bid + 1], wt = s_wp[G];
        uint64_t my_tasks = 0;
        if (threadIdx.x == 0) d_t0 = global_ns();
        bool ok = true;
        if (chunks > 0 && total > 0) {
            if constexpr (!BANDED) {
                const uint64_t n_tasks = (uint64_t)total * chunks;
                const uint64_t ta = n_tasks * wa / wt;
                const uint64_t tb = n_tasks * wb / wt;
                my_tasks = tb - ta;
                if (ta < tb) {
                    const uint32_t j_last = (uint32_t)((tb - 1) / chunks);
                    for (uint32_t jb = (uint32_t)(ta / chunks); jb <= j_last; jb += blockDim.x) {
                        const uint32_t j = jb + threadIdx.x;
                        if (j <= j_last) {
                            const uint32_t id = warp_spike_id(v, s_wpre, TW, Q, j);
                            s_id[threadIdx.x] = id;
                            // raster entry of every staged spike (a spike staged by two
                            // CTAs is written twice with the same value)
                            const uint64_t r = rc + j;
                            if (r < v.raster_cap) {
                                v.raster_t[r] = t;
                                v.raster_id[r] = id;
                            }
                        }
                        __syncthreads();
                        const uint64_t lo = max(ta, (uint64_t)jb * chunks);
                        const uint64_t hi = min(tb, (uint64_t)(jb + blockDim.x) * chunks);
                        for (uint64_t tk = lo + warp; tk < hi; tk += (uint64_t)PERSIST_WARPS * DELIVER_UNROLL)
                            deliver_tasks<BF16>(v, tk, PERSIST_WARPS, hi, chunks, s_id, jb, slot0, lane, pol,
                                                draw_next);
                        __syncthreads();
                    }
                }
            } else {
                // raster entries of every spike, independent of the bands
                for (uint32_t j = bid * blockDim.x + threadIdx.x; j < total; j += G * blockDim.x) {
                    const uint64_t r = rc + j;
                    if (r >= v.raster_cap) break;
                    v.raster_t[r] = t;
                    v.raster_id[r] = warp_spike_id(v, s_wpre, TW, Q, j);
                }
                // Banded delivery: the targets are split into B bands of module rows
                // delivered one after another behind grid barriers, so that one
                // band's ring columns stay in L2; a spike takes part in the bands its
                // stencil reaches, with the synapses [lo, hi) of its grouped row that
                // target the band.
                const uint32_t B = v.n_bands > 1 ? v.n_bands : 1u;
                for (uint32_t band = 0; band < B; ++band) {
                    if (band > 0 && !grid_barrier(v, G, gen)) {
                        ok = false;
                        break;
                    }
                    // spikes that can reach this band (warp-granular superset)
                    const uint2 ir = v.band_ids[band];
                    const uint32_t jl = s_wpre[warp_of_neuron(ir.x, Q, TW)];
                    const uint32_t jh = ir.y == 0 ? 0u : s_wpre[min(warp_of_neuron(ir.y - 1, Q, TW) + 1, TW)];
                    if (jh <= jl) continue;
                    const uint64_t n_tasks = (uint64_t)(jh - jl) * chunks;
                    const uint64_t ta = n_tasks * wa / wt;
                    const uint64_t tb = n_tasks * wb / wt;
                    if (ta >= tb) continue;
                    my_tasks += tb - ta;
                    const uint32_t j_last = jl + (uint32_t)((tb - 1) / chunks);
                    for (uint32_t jb = jl + (uint32_t)(ta / chunks); jb <= j_last; jb += blockDim.x) {
                        const uint32_t j = jb + threadIdx.x;
                        if (j <= j_last) {
                            const uint32_t id = warp_spike_id(v, s_wpre, TW, Q, j);
                            s_id[threadIdx.x] = id;
                            const uint32_t src = id / v.M;
                            const uint32_t key = v.band_key_row ? src / v.grid_w : src;
                            const uint32_t rng = __ldg(v.band_rng + (size_t)key * B + band);
                            const uint16_t* sg = v.segidx + (size_t)id * v.seg_stride;
                            s_lo[threadIdx.x] = __ldg(sg + (rng & 0xFFFFu));
                            s_hi[threadIdx.x] = __ldg(sg + (rng >> 16));
                        }
                        __syncthreads();
                        const uint64_t lo = max(ta, (uint64_t)(jb - jl) * chunks);
                        const uint64_t hi = min(tb, (uint64_t)(jb - jl + blockDim.x) * chunks);
                        for (uint64_t tk = lo + warp; tk < hi; tk += (uint64_t)PERSIST_WARPS * DELIVER_UNROLL)
                            deliver_tasks_range<BF16>(v, tk, PERSIST_WARPS, hi, chunks, s_id, s_lo, s_hi, jb - jl,
                                                      slot0, lane, pol, draw_next);
                        __syncthreads();
                    }
                }
            }
        } else {  // no synapses: the raster alone
            for (uint32_t j = bid * blockDim.x + threadIdx.x; j < total; j += G * blockDim.x) {
                const uint64_t r = rc + j;
                if (r >= v.raster_cap) break;
                v.raster_t[r] = t;
                v.raster_id[r] = warp_spike_id(v, s_wpre, TW, Q, j);
            }
        }
        if (!ok) break;
        rc += total;
        spikes += total;
        __syncthreads();  // this CTA's delivery is done
        if (threadIdx.x == 0) {
            d_ns += global_ns() - d_t0;
            d_tasks += my_tasks;
        }
        grid_arrive(v.st, gen);
        if (step + 1 < n_steps) prepare(t + 1);
        if (!grid_wait(v.st, G + v.barrier_extra, v.wait_limit_ns, gen)) break;
        if (bid == 0 && threadIdx.x == 0) {
            const uint64_t now = global_ns();
            ph_d += now - stamp;
            stamp = now;
        }
        done = step + 1;
    }

    // ---- epilogue: resident state back to memory, counters of the launch
    if (res) {
        __syncthreads();
        for (uint32_t q = cq0 + threadIdx.x; q < cq1; q += blockDim.x) {
            *reinterpret_cast<float4*>(v.V + ((size_t)q << 2)) = s_V[q - cq0];
            *reinterpret_cast<float4*>(v.c + ((size_t)q << 2)) = s_C[q - cq0];
            *reinterpret_cast<uint32_t*>(v.ref + ((size_t)q << 2)) = s_R[q - cq0];
        }
    }
    uint32_t e = ext;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
        rec += __shfl_xor_sync(0xFFFFFFFFu, rec, o);
    }
    __shared__ unsigned long long s_rec[PERSIST_WARPS];
    if (lane == 0) {
        s_ext[warp] = e;
        s_rec[warp] = rec;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long be = 0, br = 0;
        for (int w = 0; w < PERSIST_WARPS; ++w) {
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

// BANDED: the banded delivery of networks whose delay ring outgrows the L2
// budget (n_bands > 1); the unbanded instance keeps the plain row walk.
template <bool BF16, bool BANDED>
__global__ void __launch_bounds__(PERSIST_THREADS, SNN_PERSIST_MIN_BLOCKS) k_run_steps(NetView v, uint32_t n_steps) {
    extern __shared__ __align__(16) uint32_t smem[];
    run_steps<BF16, BANDED>(v, n_steps, gridDim.x, blockIdx.x, smem);
}

// Several independent networks in one cooperative launch, each on a group of
// its own: CTAs [gcta[k], gcta[k+1]) run network k's steps with the loop
// above, passing the barriers of the network's own device state, and no group
// ever waits on another.  A small network's step is bound by its latency
// chain (two barriers, a scan, dependent loads) rather than by traffic; side
// by side, the groups overlap those chains instead of paying them one network
// after another.  Banded networks are not grouped (the host keeps them out).
__global__ void __launch_bounds__(PERSIST_THREADS, SNN_PERSIST_MIN_BLOCKS) k_run_groups(GroupMeta gm) {
    extern __shared__ __align__(16) uint32_t smem[];
    __shared__ NetView s_v;
    __shared__ uint32_t s_k;
    if (threadIdx.x == 0) s_k = gm.n;  // no group: a CTA past the last one
    __syncthreads();
    for (uint32_t k = threadIdx.x; k < gm.n; k += blockDim.x)  // the groups are disjoint: one k matches
        if (gm.gcta[k] <= blockIdx.x && blockIdx.x < gm.gcta[k + 1]) s_k = k;
    __syncthreads();
    const uint32_t k = s_k;
    if (k >= gm.n) return;  // a CTA past the last group
    const uint32_t g0 = gm.gcta[k], G = gm.gcta[k + 1] - g0;
    const uint32_t* src = reinterpret_cast<const uint32_t*>(gm.views + k);
    uint32_t* dst = reinterpret_cast<uint32_t*>(&s_v);
    for (uint32_t i = threadIdx.x; i < (uint32_t)(sizeof(NetView) / 4); i += blockDim.x) dst[i] = src[i];
    __syncthreads();
    if (threadIdx.x == 0) s_v.res_quads = gm.res_quads;  // the launch's shared memory, whatever the group
    __syncthreads();
    const uint64_t start = global_ns();
    if (s_v.w_bf16)
        run_steps<true, false>(s_v, gm.steps[k], G, blockIdx.x - g0, smem);
    else
        run_steps<false, false>(s_v, gm.steps[k], G, blockIdx.x - g0, smem);
    if (blockIdx.x == g0 && threadIdx.x == 0) gm.gns[k] = global_ns() - start;
}

static const void* persistent_fn(bool bf16, bool banded) {
    if (banded) return bf16 ? (const void*)k_run_steps<true, true> : (const void*)k_run_steps<false, true>;
    return bf16 ? (const void*)k_run_steps<true, false> : (const void*)k_run_steps<false, false>;
}

static size_t persistent_smem(int grid) { return (size_t)state_offset_words((uint32_t)grid) * sizeof(uint32_t); }

// Raises fn's dynamic shared-memory limit to `bytes` (never lowers it: other
// networks' launches, also from captured graphs, may need more).
static cudaError_t raise_smem_limit(const void* fn, size_t bytes) {
    if (bytes <= 48 * 1024) return cudaSuccess;
    cudaFuncAttributes fa{};
    cudaError_t e = cudaFuncGetAttributes(&fa, fn);
    if (e != cudaSuccess || (size_t)fa.maxDynamicSharedSizeBytes >= bytes) return e;
    return cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
}

// Quads of resident state per CTA for network v on `grid` CTAs (the largest
// CTA range), or 0 if they do not fit in shared memory next to everything else
// at the occupancy the grid needs, for both the banded and the unbanded
// instance (bands can be set later).  Raises the kernels' shared-memory limit.
uint32_t persistent_resident_quads(const NetView& v, int grid) {
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    if (grid <= 0 || sms <= 0) return 0;
    const uint64_t Q = v.Npad >> 2, TW = (uint64_t)grid * PERSIST_WARPS;
    uint64_t most = 0;
    for (uint64_t b = 0; b < (uint64_t)grid; ++b)
        most = std::max(most, Q * (b * PERSIST_WARPS + PERSIST_WARPS) / TW - Q * (b * PERSIST_WARPS) / TW);
    const size_t need = persistent_smem(grid) + most * 36;
    if (most == 0) return 0;
    for (int banded = 0; banded < 2; ++banded) {
        const void* fn = persistent_fn(v.w_bf16 != 0, banded != 0);
        cudaFuncAttributes fa{};
        int fit = 0;
        if (cudaFuncGetAttributes(&fa, fn) != cudaSuccess || need + fa.sharedSizeBytes > (size_t)optin ||
            raise_smem_limit(fn, need) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, PERSIST_THREADS, need) != cudaSuccess ||
            (int64_t)fit * sms < grid) {
            cudaGetLastError();
            return 0;
        }
    }
    return (uint32_t)most;
}

// Co-resident grid: occupancy per SM x SMs, with the grid-dependent shared
// memory accounted for (largest grid that still fits).
int persistent_grid(bool bf16) {
    int dev = 0, sms = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    for (int per_sm = 8; per_sm >= 1; --per_sm) {
        const int grid = per_sm * sms;
        int fit = 0, fit_b = 0;  // the grid must fit both instances (bands can change later)
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, persistent_fn(bf16, false), PERSIST_THREADS,
                                                          persistent_smem(grid)) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit_b, persistent_fn(bf16, true), PERSIST_THREADS,
                                                          persistent_smem(grid)) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (fit >= per_sm && fit_b >= per_sm) return grid;
    }
    return sms;
}

cudaError_t launch_persistent(const NetView& v, uint32_t n_steps, int grid, cudaStream_t s) {
    const void* fn = persistent_fn(v.w_bf16 != 0, v.n_bands > 1);
    NetView vv = v;  // v.res_quads: from persistent_resident_quads for this grid, or 0
    const size_t smem = persistent_smem(grid) + (size_t)vv.res_quads * 36;
    cudaError_t e0 = raise_smem_limit(fn, smem);
    if (e0 != cudaSuccess) return e0;
    uint32_t ns = n_steps;
    void* args[] = {&vv, &ns};
    cudaError_t e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(PERSIST_THREADS), args, smem, s);
    count_launch(1);
    return e;
}

// Quads of resident state per CTA the grouped kernel's launches offer: what
// the opt-in shared memory leaves next to the kernel's own, at one CTA per SM.
static uint32_t groups_resident_quads(int grid) {
    int dev = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    cudaFuncAttributes fa{};
    if (cudaFuncGetAttributes(&fa, (const void*)k_run_groups) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    const size_t base = persistent_smem(grid) + fa.sharedSizeBytes + 1024;  // + margin for the runtime's own
    return (size_t)optin > base ? (uint32_t)(((size_t)optin - base) / 36) : 0u;
}

int groups_grid() {
    int dev = 0, sms = 0, fit = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const size_t smem = persistent_smem(sms) + (size_t)groups_resident_quads(sms) * 36;
    if (raise_smem_limit((const void*)k_run_groups, smem) != cudaSuccess ||
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, (const void*)k_run_groups, PERSIST_THREADS, smem) !=
            cudaSuccess ||
        fit < 1) {
        cudaGetLastError();
        return 0;
    }
    return sms;
}

cudaError_t launch_groups(const GroupMeta& gm, int grid, cudaStream_t s) {
    GroupMeta m = gm;
    m.res_quads = groups_resident_quads(grid);
    const size_t smem = persistent_smem(grid) + (size_t)m.res_quads * 36;
    cudaError_t e0 = raise_smem_limit((const void*)k_run_groups, smem);
    if (e0 != cudaSuccess) return e0;
    void* args[] = {&m};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_run_groups, dim3(grid), dim3(PERSIST_THREADS), args,
                                                smem, s);
    count_launch(1);
    return e;
}

}  // namespace snn
