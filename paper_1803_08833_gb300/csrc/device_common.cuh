// device_common.cuh -- device functions shared by the per-step kernels and
// the persistent multi-step kernel.
#pragma once

#include "philox.cuh"
#include "snn_internal.h"

namespace snn {

// Checked builds (-DSNN_CHECK): bounds checks on the hot path's indexed
// writes.  A failed check sets ERR_BOUNDS in the network's device state and
// the access is skipped -- no trap, no fault; the host reports the bit.
// Release builds compile every check to `true`.
#ifdef SNN_CHECK
#define SNN_BOUND(st, cond) ((cond) ? true : (atomicOr(&(st)->err, ERR_BOUNDS), false))
#else
#define SNN_BOUND(st, cond) true
#endif

__device__ __forceinline__ void red_add(int32_t* p, int32_t v) {
    asm volatile("red.relaxed.gpu.global.add.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// ---------------------------------------------------------------------------
// Neuron update (Eq. 1-2).  Exact propagator over dt with the input of the step
// added after the decay:
//   V <- ((V - E) a_m + E) - k_c c + I 2^-fx,   c <- c a_c,
// a_m = exp(-dt/tau_m), a_c = exp(-dt/tau_c),
// k_c = g_c tau_m tau_c / (tau_c - tau_m) (exp(-dt/tau_c) - exp(-dt/tau_m)).
// While refractory V is held at V_r and the input is discarded.  A spike
// (V > V_th, or a forced spike) resets V, starts the refractory count and,
// for excitatory neurons, adds alpha_c to c.
__device__ __forceinline__ bool lif_update(const NetView& v, float& V, float& c, uint32_t& ref, bool exc,
                                           int32_t I, bool forced) {
    const bool was_ref = ref > 0;
    if (was_ref) {
        ref -= 1;
        V = v.V_reset;
    } else {
        float x = __fsub_rn(V, v.E);
        x = __fmul_rn(x, v.a_m);
        x = __fadd_rn(x, v.E);
        x = __fsub_rn(x, __fmul_rn(v.kc, c));
        x = __fadd_rn(x, __fmul_rn(__int2float_rn(I), v.in_scale));
        V = x;
    }
    c = __fmul_rn(c, v.a_c);
    const bool spike = !was_ref && (V > v.V_th || forced);
    if (spike) {
        V = v.V_reset;
        ref = v.ref_steps;
        if (exc) c = __fadd_rn(c, v.alpha_c);
    }
    return spike;
}

// External Poisson count: #{k : P[k] <= u}.  `tab` (shared memory) holds the
// stored thresholds (all <= 2^32 - 2) padded to `pad` (a power of two, 0 if
// there is no drive) with 0xFFFFFFFF; with u clamped to 2^32 - 2 the padding
// never counts.  Branch-free binary search; the table sits in shared memory
// because lanes index it divergently.
__device__ __forceinline__ uint32_t poisson_count(const uint32_t* tab, uint32_t pad, uint32_t u) {
    const uint32_t x = min(u, 0xFFFFFFFEu);
    uint32_t pos = 0;
    for (uint32_t step = pad >> 1; step >= 1; step >>= 1)
        if (tab[pos + step - 1] <= x) pos += step;
    if (pad && tab[pos] <= x) pos += 1;
    return pos;
}

// Copies the Poisson table into shared memory (call from every thread, then sync).
__device__ __forceinline__ void load_poisson_table(const NetView& v, uint32_t* s_pois) {
    for (uint32_t k = threadIdx.x; k < (uint32_t)MAX_POIS; k += blockDim.x) s_pois[k] = v.pois32[k];
}

// State of four consecutive neurons as loaded from memory, with their ring
// slot and their external drive of the step.
struct QuadIn {
    int4 I;
    float4 V, C;
    uint32_t R;
    uint32_t drive;  // byte q: n_ext of neuron q | forced << 7
};

// External drive of neurons base .. base+3 at step t (Philox (i, t, DRIVE)):
// the Poisson count of word u0 and the imposed spike of word u1, one byte per
// neuron.  The four draws are computed first, unconditionally (neurons past N
// are padding and are not updated later), so their dependency chains interleave.
__device__ __forceinline__ uint32_t quad_drive(const NetView& v, const uint32_t* s_pois, uint32_t base, uint32_t t) {
    U4 u[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) u[q] = philox4x32_10(base + q, t, TAG_DRIVE, 0u, v.key0, v.key1);
    uint32_t pk = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t n_ext = poisson_count(s_pois, v.pois_pad, u[q].x);  // < MAX_POIS
        const uint32_t forced = (uint64_t)u[q].y < v.imposed_thresh ? 0x80u : 0u;
        pk |= (n_ext | forced) << (8 * q);
    }
    return pk;
}

// V, c, ref of neurons base .. base+3 (base a multiple of 4, < Npad): the
// part of a quad that does not depend on the step's deliveries.
__device__ __forceinline__ void load_state(const NetView& v, uint32_t base, QuadIn& in) {
    in.V = *reinterpret_cast<const float4*>(v.V + base);
    in.C = *reinterpret_cast<const float4*>(v.c + base);
    in.R = *reinterpret_cast<const uint32_t*>(v.ref + base);
}

// The ring slot was last written by other SMs' L2 reductions: read at L2 (.cg).
__device__ __forceinline__ int4 load_slot(const NetView& v, uint32_t base, uint32_t slot) {
    return __ldcg(reinterpret_cast<const int4*>(v.ring + (size_t)slot * v.Npad + base));
}

// Everything a quad needs for step t.
__device__ __forceinline__ QuadIn load_quad(const NetView& v, const uint32_t* s_pois, uint32_t base, uint32_t t,
                                            uint32_t slot) {
    QuadIn in;
    in.I = load_slot(v, base, slot);
    load_state(v, base, in);
    in.drive = quad_drive(v, s_pois, base, t);
    return in;
}

// New state of a quad, before it is stored.
struct QuadOut {
    float4 V, C;
    uint32_t R;
};

// Integrates the loaded quad into `out` and (CLEAR) clears the ring slot.
// Returns a 4-bit spike mask; adds the external events to `ext` and, under the
// pairwise rule, the spiking rows' lengths to `rec`.
template <bool CLEAR = true>
__device__ __forceinline__ uint32_t integrate_quad(const NetView& v, uint32_t base, uint32_t slot, const QuadIn& in,
                                                   uint32_t& ext, uint64_t& rec, QuadOut& out) {
    if (CLEAR) *reinterpret_cast<int4*>(v.ring + (size_t)slot * v.Npad + base) = make_int4(0, 0, 0, 0);
    float Vq[4] = {in.V.x, in.V.y, in.V.z, in.V.w};
    float Cq[4] = {in.C.x, in.C.y, in.C.z, in.C.w};
    const int32_t Iq[4] = {in.I.x, in.I.y, in.I.z, in.I.w};
    uint32_t spk = 0, Rout = 0;
    uint32_t mi = base % v.M;  // position of neuron `base` inside its module
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const uint32_t i = base + q;
        uint32_t r = (in.R >> (8 * q)) & 0xFFu;
        const uint32_t dq = in.drive >> (8 * q);
        const uint32_t n_ext = dq & 0x7Fu;
        const bool forced = (dq & 0x80u) != 0;
        const int32_t I = (int32_t)((uint32_t)Iq[q] + n_ext * (uint32_t)v.J_ext_fx);
        float Vn = Vq[q], Cn = Cq[q];
        uint32_t rn = r;
        const bool s = lif_update(v, Vn, Cn, rn, mi < v.n_exc, I, forced);
        if (i < v.N) {
            ext += n_ext;
            Vq[q] = Vn;
            Cq[q] = Cn;
            r = rn;
            if (s) spk |= 1u << q;
        }
        Rout |= r << (8 * q);
        mi += 1;
        if (mi >= v.M) mi = 0;
    }
    out.V = make_float4(Vq[0], Vq[1], Vq[2], Vq[3]);
    out.C = make_float4(Cq[0], Cq[1], Cq[2], Cq[3]);
    out.R = Rout;
    if (v.row_len != nullptr && spk != 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
            if (spk & (1u << q)) rec += __ldg(v.row_len + base + q);
    }
    return spk;
}

__device__ __forceinline__ void store_state(const NetView& v, uint32_t base, const QuadOut& o) {
    *reinterpret_cast<float4*>(v.V + base) = o.V;
    *reinterpret_cast<float4*>(v.c + base) = o.C;
    *reinterpret_cast<uint32_t*>(v.ref + base) = o.R;
}

// Integrates the loaded quad, stores the new state, clears the ring slot.
__device__ __forceinline__ uint32_t compute_quad(const NetView& v, uint32_t base, uint32_t slot, const QuadIn& in,
                                                 uint32_t& ext, uint64_t& rec) {
    QuadOut o;
    const uint32_t spk = integrate_quad(v, base, slot, in, ext, rec, o);
    store_state(v, base, o);
    return spk;
}

__device__ __forceinline__ uint32_t update_quad(const NetView& v, const uint32_t* s_pois, uint32_t base, uint32_t t,
                                                uint32_t slot, uint32_t& ext, uint64_t& rec) {
    return compute_quad(v, base, slot, load_quad(v, s_pois, base, t, slot), ext, rec);
}

// ---------------------------------------------------------------------------
// Delivery helpers.

__device__ __forceinline__ int32_t fx_weight(const NetView& v, float w) {
    return __float2int_rn(__fmul_rn(w, v.w_scale));
}
__device__ __forceinline__ float bf16_lo(uint32_t x) { return __uint_as_float(x << 16); }
__device__ __forceinline__ float bf16_hi(uint32_t x) { return __uint_as_float(x & 0xFFFF0000u); }

// The synapse table is read once per spike: no L1 allocation, and an L2
// evict-first policy so the streamed table does not push the ring out of L2.
__device__ __forceinline__ uint64_t evict_first_policy() {
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}
__device__ __forceinline__ uint4 ld_u4(const void* p, uint64_t pol) {
    uint4 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                 : "=r"(r.x), "=r"(r.y), "=r"(r.z), "=r"(r.w)
                 : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint2 ld_u2(const void* p, uint64_t pol) {
    uint2 r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.v2.u32 {%0,%1}, [%2], %3;"
                 : "=r"(r.x), "=r"(r.y)
                 : "l"(p), "l"(pol));
    return r;
}
__device__ __forceinline__ uint32_t ld_u1(const void* p, uint64_t pol) {
    uint32_t r;
    asm volatile("ld.global.nc.L1::no_allocate.L2::cache_hint.u32 %0, [%1], %2;" : "=r"(r) : "l"(p), "l"(pol));
    return r;
}

#ifndef SNN_DELIVER_UNROLL
#define SNN_DELIVER_UNROLL 6
#endif
constexpr int DELIVER_UNROLL = SNN_DELIVER_UNROLL;

// One warp delivers up to DELIVER_UNROLL tasks (spike, 128-synapse chunk):
// task tk + u * tstride for u < DELIVER_UNROLL, each below `hi`.  ids[j - j0]
// gives the neuron of staged spike j.  Each lane loads 4 consecutive synapses
// of every task first (16 B of target | delay << 24 words, 16 B f32 or 8 B
// bf16 weights), then issues the reductions.
struct NoHook {
    __device__ __forceinline__ void operator()() const {}
};

// `hook` runs between the loads and the reductions: independent arithmetic
// placed there overlaps the table loads' latency.
template <bool BF16, int DELIVER_UNROLL = snn::DELIVER_UNROLL, class Hook = NoHook>
__device__ __forceinline__ void deliver_tasks(const NetView& v, uint64_t tk, uint64_t tstride, uint64_t hi,
                                              uint32_t chunks, const uint32_t* ids, uint32_t j0, uint32_t slot0,
                                              uint32_t lane, uint64_t pol, Hook hook = Hook()) {
    uint4 tg[DELIVER_UNROLL];
    uint4 wr[DELIVER_UNROLL];  // raw weight bits: converted after every load of the round is issued
    uint32_t nv[DELIVER_UNROLL];
#pragma unroll
    for (int u = 0; u < DELIVER_UNROLL; ++u) {
        const uint64_t task = tk + (uint64_t)u * tstride;
        nv[u] = 0;
        if (task < hi) {
            const uint32_t jj = (uint32_t)(task / chunks);
            const uint32_t ch = (uint32_t)(task - (uint64_t)jj * chunks);
            const uint32_t k0 = (ch << 7) + (lane << 2);
            const uint32_t id = ids[jj - j0];
            const uint32_t L = v.row_len ? __ldg(v.row_len + id) : v.K;  // row length
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
#pragma unroll
    for (int u = 0; u < DELIVER_UNROLL; ++u) {
        const uint32_t tq[4] = {tg[u].x, tg[u].y, tg[u].z, tg[u].w};
        const uint32_t wq[4] = {wr[u].x, wr[u].y, wr[u].z, wr[u].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if ((uint32_t)q < nv[u]) {
                uint32_t s = slot0 + (tq[q] >> 24);
                if (s >= v.D) s -= v.D;
                const float wv = BF16 ? ((q & 1) ? bf16_hi(wq[q >> 1]) : bf16_lo(wq[q >> 1])) : __uint_as_float(wq[q]);
                if (SNN_BOUND(v.st, s < v.D && (tq[q] & 0xFFFFFFu) < v.N))
                    red_add(v.ring + (size_t)s * v.Npad + (tq[q] & 0xFFFFFFu), fx_weight(v, wv));
            }
        }
    }
}

// As deliver_tasks, but only synapses [rlo, rhi) of each staged spike's row
// (the synapses that target one band of module rows).
template <bool BF16, int DELIVER_UNROLL = snn::DELIVER_UNROLL, class Hook = NoHook>
__device__ __forceinline__ void deliver_tasks_range(const NetView& v, uint64_t tk, uint64_t tstride, uint64_t hi,
                                                    uint32_t chunks, const uint32_t* ids, const uint32_t* rlo,
                                                    const uint32_t* rhi, uint32_t j0, uint32_t slot0, uint32_t lane,
                                                    uint64_t pol, Hook hook = Hook()) {
    uint4 tg[DELIVER_UNROLL];
    uint4 wr[DELIVER_UNROLL];  // raw weight bits: converted after every load of the round is issued
    uint32_t msk[DELIVER_UNROLL];  // bit q: synapse k0 + q is delivered
#pragma unroll
    for (int u = 0; u < DELIVER_UNROLL; ++u) {
        const uint64_t task = tk + (uint64_t)u * tstride;
        msk[u] = 0;
        if (task < hi) {
            const uint32_t jj = (uint32_t)(task / chunks);
            const uint32_t ch = (uint32_t)(task - (uint64_t)jj * chunks);
            const uint32_t k0 = (ch << 7) + (lane << 2);
            const uint32_t a = rlo[jj - j0], L = rhi[jj - j0];
            if (k0 < L && k0 + 4 > a) {
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (k0 + q >= a && k0 + q < L) msk[u] |= 1u << q;
                const size_t e = (size_t)ids[jj - j0] * v.Kpad + k0;
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
#pragma unroll
    for (int u = 0; u < DELIVER_UNROLL; ++u) {
        const uint32_t tq[4] = {tg[u].x, tg[u].y, tg[u].z, tg[u].w};
        const uint32_t wq[4] = {wr[u].x, wr[u].y, wr[u].z, wr[u].w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            if (msk[u] & (1u << q)) {
                uint32_t s = slot0 + (tq[q] >> 24);
                if (s >= v.D) s -= v.D;
                const float wv = BF16 ? ((q & 1) ? bf16_hi(wq[q >> 1]) : bf16_lo(wq[q >> 1])) : __uint_as_float(wq[q]);
                if (SNN_BOUND(v.st, s < v.D && (tq[q] & 0xFFFFFFu) < v.N))
                    red_add(v.ring + (size_t)s * v.Npad + (tq[q] & 0xFFFFFFu), fx_weight(v, wv));
            }
        }
    }
}

}  // namespace snn
