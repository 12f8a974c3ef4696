// PTX helpers and the row epilogue shared by the tensor-core kernels (tcgen05,
// TMA, mbarrier) of k_tc.cu and k_chain.cu.
#pragma once
#include <cuda.h>
#include "dae_internal.h"
#include "epilogue.cuh"

namespace dae {
namespace tc {

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count));
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                 "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

constexpr uint64_t kWaitNs = 2000000000ull;   // 2 s

// Bounded wait for the phase of `bar` with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = globaltimer();
    while (true) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > kWaitNs) return false;
    }
}

__device__ __forceinline__ void fence_barrier_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void tma_load_2d(void* dst, const CUtensorMap* map, uint64_t* bar, int c0,
                                            int c1) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4}], [%2];" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(smem_u32(bar)), "r"(c0), "r"(c1)
        : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* dst, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
                 "r"(ncols));
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols));
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// Shared-memory matrix descriptor: K-major operand, rows of 128 bytes with the
// 128-byte swizzle, 8-row groups 1024 bytes apart (SBO), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t saddr) {
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;              // leading byte offset (unused with 128B swizzle, K-major)
    d |= (uint64_t)(1024 >> 4) << 32;    // stride byte offset
    d |= (uint64_t)1 << 46;              // descriptor version
    d |= (uint64_t)2 << 61;              // 128-byte swizzle
    return d;
}

// Instruction descriptor: FP32 accumulator, A/B format (1 = BF16, 2 = TF32),
// both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
__host__ __device__ constexpr uint32_t idesc(uint32_t fmt, int M, int N) {
    return (1u << 4) | (fmt << 7) | (fmt << 10) | ((uint32_t)(N >> 3) << 17) |
           ((uint32_t)(M >> 4) << 24);
}

template <int PREC>
__device__ __forceinline__ void mma(uint32_t d, uint64_t a, uint64_t b, uint32_t id, uint32_t acc) {
    if constexpr (PREC == DAE_TF32) {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(id), "r"(acc));
    } else {
        asm volatile(
            "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
            "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d),
            "l"(a), "l"(b), "r"(id), "r"(acc));
    }
}

__device__ __forceinline__ void mbar_arrive(uint64_t* bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t* bar) {
    asm volatile(
        "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
            smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
          "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
          "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
__device__ __forceinline__ void tmem_wait_ld() {
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Epilogue of one output row whose Cp accumulator columns sit in shared memory
// (v[c], stride 1).  Runtime loops keep the executed code small: the kernel runs
// each epilogue once per CTA, so straight-line unrolled code would be fetched
// cold from memory.
__device__ __forceinline__ void put_act(const FwdArgs& A, size_t idx, float x) {
    if (A.out_f32) A.Y[idx] = x;
    if (A.out_bf16) {
        const __nv_bfloat16 hi = __float2bfloat16_rn(x);
        A.Yh[idx] = hi;
        if (A.out_bf16 == 2) A.Yl[idx] = __float2bfloat16_rn(x - __bfloat162float(hi));
    }
}

static __device__ __noinline__ void row_epilogue(const FwdArgs& A, int n, const float* v) {
    const int r = A.r, CP = A.Cp, C = n_cols(r);
    if (A.mode == 2) {
        // reverse pass: delta of this layer's input -> g of the layer below,
        // Re g = Re d s1, Im_j g = Im_j d s1 + Re d (s2 b_j)   (Sec. 4.4 complex BP)
        if (n >= A.ldy) return;
        const size_t ldy = A.ldy;
        if (n >= A.n_out) {
            for (int c = 0; c < CP; ++c) put_act(A, (size_t)c * ldy + n, 0.f);
            return;
        }
        const float s1 = A.S1[n];
        const float re = v[0];
        put_act(A, n, re * s1);
        for (int c0 = 1; c0 < CP; c0 += 8) {
            float tv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                tv[i] = (c0 + i <= r) ? A.T[(size_t)(c0 + i - 1) * A.n_out + n] : 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = c0 + i;
                if (c < CP) put_act(A, (size_t)c * ldy + n, c <= r ? fmaf(v[c], s1, re * tv[i]) : 0.f);
            }
        }
        return;
    }
    if (A.mode == 3) {
        // reverse pass at the network input: Re = J^T a, Im_j = h (a^T H)[:, j]
        if (n >= A.n_out) return;
        for (int c = 0; c <= r; ++c) A.dout[(size_t)c * A.n_out + n] = v[c];
        return;
    }
    if (A.mode == 0) {
        if (n >= A.ldy) return;
        const size_t ldy = A.ldy;
        if (n >= A.n_out) {
            for (int c = 0; c < CP; ++c) put_act(A, (size_t)c * ldy + n, 0.f);
            return;
        }
        const ActD D = act_d(A.act, v[0] + A.bias[n]);
        const float c = v[1], gw = v[2];
        float oc, ogw, og0;
        mc_shared(D, c, gw, v[3], oc, ogw, og0);
        put_act(A, n, D.s0);
        put_act(A, ldy + n, oc);
        put_act(A, 2 * ldy + n, ogw);
        put_act(A, 3 * ldy + n, og0);
        if (A.S1) A.S1[n] = D.s1;
        for (int j = 0; j < r; ++j) {
            const int cb = kShared + 3 * j;
            float ob, od, oh;
            mc_group(D, c, gw, v[cb], v[cb + 1], v[cb + 2], ob, od, oh);
            put_act(A, (size_t)cb * ldy + n, ob);
            put_act(A, (size_t)(cb + 1) * ldy + n, od);
            put_act(A, (size_t)(cb + 2) * ldy + n, oh);
            if (A.T) A.T[(size_t)j * A.n_out + n] = D.s2 * v[cb];
        }
        for (int cc = C; cc < CP; ++cc) put_act(A, (size_t)cc * ldy + n, 0.f);
        return;
    }
    // mode 1: output layer
    if (n >= A.n_out) return;
    const size_t N = A.n_out;
    if (A.u) A.u[n] = v[0] + A.bias[n];
    if (A.HDD) A.HDD[n] = (float)(v[3] * A.inv_h2);
    if (A.Hqq) A.Hqq[n] = (float)(v[3] * A.inv_h2 * A.inv_dt2);
    for (int j = 0; j < r; ++j) {
        const int cb = kShared + 3 * j;
        if (A.J) A.J[(size_t)j * N + n] = (float)(v[cb] * A.inv_h);
        if (A.dJ) A.dJ[(size_t)j * N + n] = (float)(v[cb + 2] * A.inv_h3);
    }
}


}  // namespace tc
}  // namespace dae
