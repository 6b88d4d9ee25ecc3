// persistent_tiled.cu -- persistent multi-step kernel with target-owned delivery.
//
// The push delivery adds every synaptic event into the delay ring with one
// random L2 reduction; on GB300 random 4-byte reductions into a 60 MB buffer
// top out near 2.2e11/s, below what the table stream alone could sustain.
// Here each CTA owns target modules instead.  For target module m it gathers,
// from every source module s whose stencil contains m, the spikes of the step
// and the segment of each spiking neuron's row that targets m (rows are
// grouped by target module, with a per-row segment index), and accumulates
// the events with shared-memory atomics in a tile of (D - 1) future slots x M
// neurons.  The tile then goes to ring columns [m M, (m + 1) M) of the D - 1
// future slots by bulk reductions (cp.reduce.async.bulk .add.s32, one per
// slot row, issued by one thread and performed by the TMA unit at L2): the
// 16-byte aligned interior of each row; the at most 3 + 3 cells at its ends
// go by ordinary reductions.  No other CTA touches those columns in this
// phase.  The integer sums, and so the results, are the same as with the
// push delivery.
//
// Two CTAs share an SM (a tile of 20 x 1,256 cells is 100 KB), so the latency
// chain of one CTA's tile (spike counts, segment starts, table loads, flush)
// overlaps the other's.
#include "grid_common.cuh"

namespace snn {

constexpr int TILE_THREADS = 256;
constexpr int TILE_WARPS = TILE_THREADS / 32;
constexpr int TILE_MIN_BLOCKS = 2;
constexpr uint32_t PAIR_CAP = 512;  // (spike, segment) pairs staged per batch
constexpr int EV_UNROLL = 16;       // events in flight per lane

__device__ __forceinline__ uint32_t ld_nc_u32(const uint32_t* p, uint64_t pol) {
    uint32_t r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint32_t ld_nc_u16(const uint16_t* p, uint64_t pol) {
    uint16_t r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u16 %0, [%1], %2;" : "=h"(r) : "l"(p), "l"(pol));
    return r;
}

// Bulk reduction global[0 .. bytes) += shared[0 .. bytes) (s32), TMA engine;
// both addresses 16-byte aligned, bytes a multiple of 16.
__device__ __forceinline__ void bulk_add_s32(int32_t* g, const int32_t* s, uint32_t bytes) {
    const uint32_t sa = (uint32_t)__cvta_generic_to_shared(s);
    asm volatile("cp.reduce.async.bulk.global.shared::cta.bulk_group.add.s32 [%0], [%1], %2;" ::"l"(g), "r"(sa),
                 "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ void bulk_commit() { asm volatile("cp.async.bulk.commit_group;" ::: "memory"); }
// Source shared memory of every committed bulk operation has been read.
__device__ __forceinline__ void bulk_wait_read() { asm volatile("cp.async.bulk.wait_group.read 0;" ::: "memory"); }
// Every committed bulk operation has completed (its global writes performed).
__device__ __forceinline__ void bulk_wait_all() { asm volatile("cp.async.bulk.wait_group 0;" ::: "memory"); }
// Orders this thread's generic-proxy shared-memory accesses before later
// async-proxy (bulk) accesses.
__device__ __forceinline__ void fence_async_shared() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }
// The same for global memory.
__device__ __forceinline__ void fence_async_global() { asm volatile("fence.proxy.async.global;" ::: "memory"); }

// Tile row stride (cells): covers [floor4(g), floor4(g) + RS) for any module
// base g, so that a 16-byte aligned global cell sits on a 16-byte aligned
// shared cell.
__host__ __device__ __forceinline__ uint32_t tile_row_stride(uint32_t M) { return (M + 3u + 3u) & ~3u; }

static size_t tiled_smem(const NetView& v, int grid) {
    const size_t tile = (size_t)(v.D - 1) * tile_row_stride(v.M) * sizeof(int32_t);
    const size_t ids = (size_t)(grid + 1 + grid * TILE_WARPS) * sizeof(uint32_t);  // aliased with the tile
    return (tile > ids ? tile : ids)                                                //
           + (size_t)(3 * PAIR_CAP + 1) * sizeof(uint32_t)                          // pair id, start, prefix
           + (size_t)(v.max_off + 1) * sizeof(uint32_t);                           // source prefix
}

template <bool BF16>
__global__ void __launch_bounds__(TILE_THREADS, TILE_MIN_BLOCKS) k_run_steps_tiled(NetView v, uint32_t n_steps) {
    extern __shared__ __align__(16) uint32_t smem[];
    const uint32_t G = gridDim.x, TW = G * TILE_WARPS;
    const uint32_t M = v.M, Dm1 = v.D - 1, nm = v.n_modules;
    const uint32_t RS = tile_row_stride(M);
    int32_t* tile = reinterpret_cast<int32_t*>(smem);
    const size_t tile_words = (size_t)Dm1 * RS;
    const size_t ids_words = (size_t)G + 1 + (size_t)G * TILE_WARPS;
    uint32_t* s_pid = smem + (tile_words > ids_words ? tile_words : ids_words);
    uint32_t* s_pa = s_pid + PAIR_CAP;
    uint32_t* s_pref = s_pa + PAIR_CAP;
    uint32_t* s_src = s_pref + PAIR_CAP + 1;
    uint32_t* s_cta = smem;  // raster phase only: shares the tile's space
    uint32_t* s_woff = s_cta + G + 1;
    __shared__ uint32_t s_t0, s_wcnt[TILE_WARPS], s_ext[TILE_WARPS];
    __shared__ unsigned long long s_rc0;
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
    const uint32_t wg = blockIdx.x * TILE_WARPS + warp;
    const uint32_t Q = v.Npad >> 2;
    const uint32_t qa = (uint32_t)((uint64_t)Q * wg / TW);
    const uint32_t qb = (uint32_t)((uint64_t)Q * (wg + 1) / TW);
    const uint64_t pol = evict_first_policy();
    const uint32_t lt_mask = (1u << lane) - 1u;
    uint64_t rc = s_rc0;
    uint64_t spikes = 0;
    uint32_t ext = 0, done = 0;
    uint64_t rec_unused = 0;  // the grouped layout exists for the fixed out-degree rule only
    uint64_t ph_n = 0, ph_d = 0, stamp = 0;
    if (blockIdx.x == 0 && threadIdx.x == 0) stamp = global_ns();

    for (uint32_t step = 0; step < n_steps; ++step) {
        const uint32_t t = t0 + step;
        const uint32_t slot = t % v.D;
        const uint32_t par = t & 1u;
        uint32_t* mcnt = v.mod_cnt + (size_t)par * nm;
        // ---- phase N: update, id-ordered warp segments (raster), per-module lists (delivery)
        uint32_t run = 0;
        QuadIn nxt;  // the next chunk's loads are issued before this chunk is integrated
        if (qa + lane < qb) nxt = load_quad(v, s_pois, (qa + lane) << 2, t, slot);
        for (uint32_t qc = qa; qc < qb; qc += 32) {
            const uint32_t q = qc + lane;
            const QuadIn cur = nxt;
            if (q + 32 < qb) nxt = load_quad(v, s_pois, (q + 32) << 2, t, slot);
            uint32_t spk = 0;
            if (q < qb) spk = compute_quad(v, q << 2, slot, cur, ext, rec_unused);
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
            if (__any_sync(0xFFFFFFFFu, spk != 0)) {
                const uint32_t m0 = (q << 2) / M, r0 = (q << 2) - m0 * M;
#pragma unroll
                for (int b = 0; b < 4; ++b) {
                    const bool has = (spk >> b) & 1u;
                    const uint32_t mb = m0 + (r0 + b >= M ? (r0 + b) / M : 0u);
                    const uint32_t key = has ? mb : 0xFFFFFFFFu;
                    const uint32_t peers = __match_any_sync(0xFFFFFFFFu, key);
                    const uint32_t leader = __ffs(peers) - 1;
                    uint32_t base = 0;
                    if (has && lane == leader) base = atomicAdd(mcnt + mb, (uint32_t)__popc(peers));
                    base = __shfl_sync(0xFFFFFFFFu, base, leader);
                    if (has) v.seg_mod[(size_t)mb * M + base + __popc(peers & lt_mask)] = (q << 2) + b;
                }
            }
        }
        if (lane == 0) s_wcnt[warp] = run;
        __syncthreads();
        if (threadIdx.x == 0) {
            uint32_t acc = 0;
            for (int w = 0; w < TILE_WARPS; ++w) {
                v.woff[blockIdx.x * TILE_WARPS + w] = acc;
                acc += s_wcnt[w];
            }
            v.cta_cnt[blockIdx.x] = acc;
        }
        if (!grid_barrier(v, G, gen)) break;
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const uint64_t now = global_ns();
            ph_n += now - stamp;
            stamp = now;
        }

        // ---- phase D: raster entries
        block_exclusive_scan(v.cta_cnt, G, s_cta);
        for (uint32_t i = threadIdx.x; i < TW; i += blockDim.x) s_woff[i] = __ldcg(v.woff + i);
        __syncthreads();
        const uint32_t total = s_cta[G];
        for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j < total; j += G * blockDim.x) {
            const uint64_t r = rc + j;
            if (r >= v.raster_cap) break;
            v.raster_t[r] = t;
            v.raster_id[r] = spike_id<TILE_WARPS>(v, s_cta, s_woff, j, Q, TW, G);
        }
        // the other parity's counters were last used by the previous step
        for (uint32_t m = blockIdx.x * blockDim.x + threadIdx.x; m < nm; m += G * blockDim.x)
            v.mod_cnt[(size_t)(par ^ 1u) * nm + m] = 0;
        __syncthreads();  // s_cta / s_woff are dead: the tile may now be written

        // ---- phase D: target tiles
        for (uint32_t m = blockIdx.x; m < nm && v.K > 0; m += G) {
            const uint32_t g = m * M;           // first ring column of the module
            const uint32_t g4 = g & ~3u;        // tile cell 0 of every row
            const uint32_t nin = v.in_cnt[m];
            const uint32_t* isrc = v.in_src + (size_t)m * v.max_off;
            const uint32_t* ij = v.in_j + (size_t)m * v.max_off;
            for (uint32_t k = threadIdx.x; k < nin; k += blockDim.x) s_src[k] = __ldcg(mcnt + isrc[k]);
            __syncthreads();
            if (warp == 0) {  // exclusive prefix over the incoming sources, in place
                uint32_t run2 = 0;
                for (uint32_t k0 = 0; k0 < nin; k0 += 32) {
                    const uint32_t k = k0 + lane;
                    const uint32_t x = k < nin ? s_src[k] : 0u;
                    uint32_t incl = x;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
                        if (lane >= (uint32_t)o) incl += y;
                    }
                    __syncwarp();
                    if (k < nin) s_src[k] = run2 + incl - x;
                    run2 += __shfl_sync(0xFFFFFFFFu, incl, 31);
                }
                if (lane == 0) s_src[nin] = run2;
            }
            __syncthreads();
            const uint32_t P = s_src[nin];
            if (P == 0) {  // no spike reaches this module: nothing to add
                __syncthreads();  // s_src is rewritten by the next module
                continue;
            }
            for (uint32_t pb = 0; pb < P; pb += PAIR_CAP) {
                const uint32_t np = min(PAIR_CAP, P - pb);
                for (uint32_t p = threadIdx.x; p < np; p += blockDim.x) {
                    const uint32_t gp = pb + p;
                    uint32_t lo = 0, hi = nin;  // largest k with s_src[k] <= gp
                    while (hi - lo > 1) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (s_src[mid] <= gp)
                            lo = mid;
                        else
                            hi = mid;
                    }
                    const uint32_t id = __ldcg(v.seg_mod + (size_t)isrc[lo] * M + (gp - s_src[lo]));
                    const uint16_t* sg = v.segidx + (size_t)id * v.seg_stride + ij[lo];
                    const uint32_t a = __ldg(sg), b = __ldg(sg + 1);
                    s_pid[p] = id;
                    s_pa[p] = a;
                    s_pref[p] = b - a;
                }
                if (pb == 0) {
                    // the previous module's flush has finished reading the tile
                    if (threadIdx.x == 0) bulk_wait_read();
                    __syncthreads();
                    int4* t4 = reinterpret_cast<int4*>(tile);
                    for (uint32_t x = threadIdx.x; x < (Dm1 * RS) >> 2; x += blockDim.x) t4[x] = make_int4(0, 0, 0, 0);
                }
                __syncthreads();
                block_scan_inplace(s_pref, np);  // exclusive, s_pref[np] = events of the batch
                const uint32_t E = s_pref[np];
                const uint32_t e0 = (uint32_t)((uint64_t)E * warp / TILE_WARPS);
                const uint32_t e1 = (uint32_t)((uint64_t)E * (warp + 1) / TILE_WARPS);
                // pair of the lane's first event: largest p with s_pref[p] <= e
                uint32_t pp = 0;
                {
                    const uint32_t e = e0 + lane;
                    uint32_t lo = 0, hi = np;
                    while (hi - lo > 1) {
                        const uint32_t mid = (lo + hi) >> 1;
                        if (s_pref[mid] <= e)
                            lo = mid;
                        else
                            hi = mid;
                    }
                    pp = lo;
                }
                const uint32_t ph = g - g4;  // tile column of ring column g
                for (uint32_t base = e0; base < e1; base += 32 * EV_UNROLL) {
                    uint32_t tg[EV_UNROLL], wb[EV_UNROLL], dd[EV_UNROLL];
#pragma unroll
                    for (int u = 0; u < EV_UNROLL; ++u) {
                        const uint32_t e = base + u * 32 + lane;
                        tg[u] = 0xFFFFFFFFu;
                        wb[u] = 0;
                        dd[u] = 0;
                        if (e < e1) {
                            while (pp + 1 < np && s_pref[pp + 1] <= e) ++pp;
                            const size_t idx = (size_t)s_pid[pp] * v.Kpad + s_pa[pp] + (e - s_pref[pp]);
                            const uint32_t x = ld_nc_u32(v.td + idx, pol);
                            tg[u] = x & 0xFFFFFFu;
                            dd[u] = x >> 24;
                            wb[u] = BF16 ? ld_nc_u16(reinterpret_cast<const uint16_t*>(v.w) + idx, pol)
                                         : ld_nc_u32(reinterpret_cast<const uint32_t*>(v.w) + idx, pol);
                        }
                    }
#pragma unroll
                    for (int u = 0; u < EV_UNROLL; ++u) {
                        const uint32_t col = tg[u] - g, row = dd[u] - 1u;
                        if (col < M && row < Dm1) {
                            const float w = BF16 ? __uint_as_float(wb[u] << 16) : __uint_as_float(wb[u]);
                            atomicAdd(tile + (size_t)row * RS + ph + col, fx_weight(v, w));
                        }
                    }
                }
                __syncthreads();
            }
            // flush: ring[(t + 1 + r) mod D][g .. g + M) += tile row r
            fence_async_shared();
            __syncthreads();
            const uint32_t a4 = (g + 3u) & ~3u, b4 = (g + M) & ~3u;  // aligned interior [a4, b4)
            const bool bulk = b4 > a4;
            if (threadIdx.x == 0 && bulk) {
                for (uint32_t r = 0; r < Dm1; ++r) {
                    uint32_t sl = slot + r + 1;
                    if (sl >= v.D) sl -= v.D;
                    int32_t* gp = v.ring + (size_t)sl * v.Npad + a4;
                    const int32_t* sp = tile + (size_t)r * RS + (a4 - g4);
                    const uint32_t bytes = (b4 - a4) * 4u;
                    if ((((uintptr_t)gp | (uintptr_t)sp | bytes) & 15u) == 0)
                        bulk_add_s32(gp, sp, bytes);
                    else
                        atomicOr(&v.st->err, ERR_ALIGNMENT);  // never expected: skip rather than fault
                }
                bulk_commit();
            }
            // the cells outside the aligned interior
            const uint32_t ne = bulk ? (a4 - g) + (g + M - b4) : M;
            for (uint32_t x = threadIdx.x; x < Dm1 * ne; x += blockDim.x) {
                const uint32_t r = x / ne, k = x - r * ne;
                const uint32_t c = !bulk ? g + k : (k < a4 - g ? g + k : b4 + (k - (a4 - g)));
                const int32_t val = tile[(size_t)r * RS + (c - g4)];
                if (val != 0) {
                    uint32_t sl = slot + r + 1;
                    if (sl >= v.D) sl -= v.D;
                    red_add(v.ring + (size_t)sl * v.Npad + c, val);
                }
            }
        }
        // every bulk reduction of this step has landed before the barrier
        if (threadIdx.x == 0) {
            bulk_wait_all();
            fence_async_global();
        }
        rc += total;
        spikes += total;
        if (!grid_barrier(v, G, gen)) break;
        if (threadIdx.x == 0) fence_async_global();  // generic writes of other CTAs before our next bulk reads
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            const uint64_t now = global_ns();
            ph_d += now - stamp;
            stamp = now;
        }
        done = step + 1;
    }
    if (threadIdx.x == 0) bulk_wait_all();  // also on an early exit

    uint32_t e = ext;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) e += __shfl_xor_sync(0xFFFFFFFFu, e, o);
    if (lane == 0) s_ext[warp] = e;
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned long long be = 0;
        for (int w = 0; w < TILE_WARPS; ++w) be += s_ext[w];
        atomicAdd(reinterpret_cast<unsigned long long*>(&v.st->ext_events), be);
        if (blockIdx.x == 0 && done == n_steps) {
            DevState* st = v.st;
            st->t = t0 + n_steps;
            st->raster_count = rc;
            st->n_spikes += spikes;
            st->rec_events += spikes * v.K;
            st->n_spk = 0;
            st->phase_ns[0] += ph_n;
            st->phase_ns[1] += ph_d;
        }
    }
}

static const void* tiled_fn(bool bf16) {
    return bf16 ? (const void*)k_run_steps_tiled<true> : (const void*)k_run_steps_tiled<false>;
}

// Co-resident grid: up to TILE_MIN_BLOCKS CTAs per SM, 0 if the tile does not fit.
int tiled_grid(const NetView& v) {
    int dev = 0, sms = 0, optin = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const void* fn = tiled_fn(v.w_bf16 != 0);
    for (int per_sm = TILE_MIN_BLOCKS; per_sm >= 1; --per_sm) {
        const int grid = per_sm * sms;
        const size_t smem = tiled_smem(v, grid);
        if (smem > (size_t)optin) continue;
        if (cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        int fit = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&fit, fn, TILE_THREADS, smem) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (fit >= per_sm) return grid;
    }
    return 0;
}

cudaError_t launch_tiled(const NetView& v, uint32_t n_steps, int grid, cudaStream_t s) {
    const size_t smem = tiled_smem(v, grid);
    const void* fn = tiled_fn(v.w_bf16 != 0);
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    NetView vv = v;
    uint32_t ns = n_steps;
    void* args[] = {&vv, &ns};
    e = cudaLaunchCooperativeKernel(fn, dim3(grid), dim3(TILE_THREADS), args, smem, s);
    count_launch(1);
    return e;
}

}  // namespace snn
