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

// AND of `ok` over the 128 epilogue threads (named barrier 1): every epilogue warp
// takes the same branch afterwards, so later named barriers cannot lose a member.
__device__ __forceinline__ bool epi_all(bool ok) {
    uint32_t all;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 1, 128, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(all)
        : "r"(ok ? 1u : 0u)
        : "memory");
    return all != 0;
}

__device__ __forceinline__ void prefetch_tmap(const CUtensorMap* map) {
    asm volatile("prefetch.tensormap [%0];" ::"l"(reinterpret_cast<uint64_t>(map)) : "memory");
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
// (v[c], stride 1).  Runtime loops keep the executed code small; every argument
// is read once into a register-resident local (the stores below cannot alias
// them), so the loops issue stores back to back.
struct ActOut {
    float* __restrict__ Y;
    __nv_bfloat16* __restrict__ Yh;
    __nv_bfloat16* __restrict__ Yl;
    int f32, bf16;   // f32: 1 FP32, 2 FP32 rounded to TF32; bf16: 1 hi, 2 hi + lo
    __device__ __forceinline__ void put(size_t idx, float x) const {
        if (f32) Y[idx] = (f32 == 2) ? tf32_rna(x) : x;
        if (bf16) {
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            Yh[idx] = hi;
            if (bf16 == 2) Yl[idx] = __float2bfloat16_rn(x - __bfloat162float(hi));
        }
    }
};

// Output row n (a cubature DOF) of stacked row i in the compact form the cubature reads:
// Jc[0][i] = u_n, Jc[1 + j][i] = J_nj (consecutive rows i of a warp: coalesced stores).
static __device__ __noinline__ void compact_epilogue(const FwdArgs& A, int i, int n,
                                                     const float* __restrict__ v) {
    const size_t ld = A.ldc;
    float* __restrict__ Jc = A.Jc;
    const float fh = (float)A.inv_h;   // exact for the power-of-two steps the library uses
    Jc[i] = v[0] + A.bias[n];
    for (int j = 0; j < A.r; ++j) Jc[(size_t)(1 + j) * ld + i] = v[kShared + 3 * j] * fh;
}

static __device__ __noinline__ void row_epilogue(const FwdArgs& A, int n, const float* __restrict__ v) {
    const int mode = A.mode, r = A.r, CP = A.Cp, C = n_cols(r);
    const int n_out = A.n_out;
    if (mode == 3) {
        // reverse pass at the network input: Re = J^T a, Im_j = h (a^T H)[:, j]
        if (n >= n_out) return;
        float* __restrict__ dout = A.dout;
        for (int c = 0; c <= r; ++c) dout[(size_t)c * n_out + n] = v[c];
        return;
    }
    if (mode == 1) {
        if (n >= n_out) return;
        const size_t N = n_out;
        float* __restrict__ u = A.u;
        float* __restrict__ J = A.J;
        float* __restrict__ dJ = A.dJ;
        float* __restrict__ HDD = A.HDD;
        float* __restrict__ Hqq = A.Hqq;
        const double ih2 = A.inv_h2, idt2 = A.inv_dt2;
        // 1/h and 1/h^3 in FP32 (exact for the power-of-two steps the library uses)
        const float fh = (float)A.inv_h, fh3 = (float)A.inv_h3;
        if (u) u[n] = v[0] + A.bias[n];
        if (HDD) HDD[n] = (float)(v[3] * ih2);
        if (Hqq) Hqq[n] = (float)(v[3] * ih2 * idt2);
        if (J && dJ) {
#pragma unroll 5
            for (int j = 0; j < r; ++j) {
                const int cb = kShared + 3 * j;
                const float a = v[cb], b = v[cb + 2];
                J[(size_t)j * N + n] = a * fh;
                dJ[(size_t)j * N + n] = b * fh3;
            }
        } else {
            for (int j = 0; j < r; ++j) {
                const int cb = kShared + 3 * j;
                if (J) J[(size_t)j * N + n] = v[cb] * fh;
                if (dJ) dJ[(size_t)j * N + n] = v[cb + 2] * fh3;
            }
        }
        return;
    }
    const ActOut o{A.Y, A.Yh, A.Yl, A.out_f32, A.out_bf16};
    const int ldy_i = A.ldy;
    if (n >= ldy_i) return;
    const size_t ldy = ldy_i;
    if (n >= n_out) {
        for (int c = 0; c < CP; ++c) o.put((size_t)c * ldy + n, 0.f);
        return;
    }
    const float* __restrict__ T = A.T;
    if (mode == 2) {
        // reverse pass: delta of this layer's input -> g of the layer below,
        // Re g = Re d s1, Im_j g = Im_j d s1 + Re d (s2 b_j)   (Sec. 4.4 complex BP)
        const float s1 = A.S1[n];
        const float re = v[0];
        o.put(n, re * s1);
        for (int c0 = 1; c0 < CP; c0 += 8) {
            float tv[8];
#pragma unroll
            for (int i = 0; i < 8; ++i)
                tv[i] = (c0 + i <= r) ? T[(size_t)(c0 + i - 1) * n_out + n] : 0.f;
#pragma unroll
            for (int i = 0; i < 8; ++i) {
                const int c = c0 + i;
                if (c < CP) o.put((size_t)c * ldy + n, c <= r ? fmaf(v[c], s1, re * tv[i]) : 0.f);
            }
        }
        return;
    }
    // mode 0: hidden layer, multicomplex activation (epilogue.cuh)
    float* __restrict__ S1 = A.S1;
    float* __restrict__ Tw = A.T;
    const ActD D = act_d(A.act, v[0] + A.bias[n]);
    const float c = v[1], gw = v[2];
    float oc, ogw, og0;
    mc_shared(D, c, gw, v[3], oc, ogw, og0);
    o.put(n, D.s0);
    o.put(ldy + n, oc);
    o.put(2 * ldy + n, ogw);
    o.put(3 * ldy + n, og0);
    if (S1) S1[n] = D.s1;
    for (int j = 0; j < r; ++j) {
        const int cb = kShared + 3 * j;
        float ob, od, oh;
        mc_group(D, c, gw, v[cb], v[cb + 1], v[cb + 2], ob, od, oh);
        o.put((size_t)cb * ldy + n, ob);
        o.put((size_t)(cb + 1) * ldy + n, od);
        o.put((size_t)(cb + 2) * ldy + n, oh);
        if (Tw) Tw[(size_t)j * n_out + n] = D.s2 * v[cb];
    }
    for (int cc = C; cc < CP; ++cc) o.put((size_t)cc * ldy + n, 0.f);
}


// Output store of the layer-chain epilogue: BF16 hi (and lo for the split form) by
// precision, FP32 (rounded to TF32 for the tf32 form) when f32 is set.
template <int PREC>
struct SliceOut {
    float* __restrict__ Y;
    __nv_bfloat16* __restrict__ Yh;
    __nv_bfloat16* __restrict__ Yl;
    int f32;
    __device__ __forceinline__ void put(size_t idx, float x) const {
        if constexpr (PREC == DAE_TF32) {
            Y[idx] = tf32_rna(x);
        } else {
            if (f32) Y[idx] = x;
            const __nv_bfloat16 hi = __float2bfloat16_rn(x);
            Yh[idx] = hi;
            if constexpr (PREC == DAE_BF16X3) Yl[idx] = __float2bfloat16_rn(x - __bfloat162float(hi));
        }
    }
};

// Epilogue of rows [r0, r0 + R) of tile `tl` (R divides 128) whose accumulator
// columns sit in shared memory (row stride TS), by the 128 epilogue threads: thread
// t takes row r0 + t % R (consecutive threads, consecutive rows: coalesced stores)
// and every (128/R)-th column group from t / R.  Modes 0 (hidden layer,
// multicomplex activation), 2 (reverse pass, next g) and 3 (reverse pass at the
// network input); see row_epilogue for the arithmetic of each.
template <int PREC>
static __device__ __noinline__ void slice_epilogue(const FwdArgs& A, const float* __restrict__ tile,
                                                   int TS, int tl, int r0, int R, int t) {
    const int tpr = 128 / R, rl = t % R, sub = t / R;
    const int n = tl * 128 + r0 + rl;
    const float* __restrict__ v = tile + (size_t)(r0 + rl) * TS;
    const int mode = A.mode, r = A.r, CP = A.Cp, n_out = A.n_out;
    if (mode == 3) {
        if (n >= n_out) return;
        float* __restrict__ dout = A.dout;
        for (int c = sub; c <= r; c += tpr) dout[(size_t)c * n_out + n] = v[c];
        return;
    }
    const SliceOut<PREC> o{A.Y, A.Yh, A.Yl, A.out_f32};
    const int ldy_i = A.ldy;
    if (n >= ldy_i) return;
    const size_t ldy = ldy_i;
    if (n >= n_out) {
        for (int c = sub; c < CP; c += tpr) o.put((size_t)c * ldy + n, 0.f);
        return;
    }
    const float* __restrict__ T = A.T;
    if (mode == 2) {
        const float s1 = A.S1[n];
        const float re = v[0];
#pragma unroll 4
        for (int c = sub; c < CP; c += tpr) {
            float x = 0.f;
            if (c == 0) x = re * s1;
            else if (c <= r) x = fmaf(v[c], s1, re * T[(size_t)(c - 1) * n_out + n]);
            o.put((size_t)c * ldy + n, x);
        }
        return;
    }
    // mode 0
    const ActD D = act_d(A.act, v[0] + A.bias[n]);
    const float c = v[1], gw = v[2];
    if (sub == 0) {
        float oc, ogw, og0;
        mc_shared(D, c, gw, v[3], oc, ogw, og0);
        o.put(n, D.s0);
        o.put(ldy + n, oc);
        o.put(2 * ldy + n, ogw);
        o.put(3 * ldy + n, og0);
        if (A.S1) A.S1[n] = D.s1;
    }
    float* __restrict__ Tw = A.T;
#pragma unroll 2
    for (int j = sub; j < r; j += tpr) {
        const int cb = kShared + 3 * j;
        float ob, od, oh;
        mc_group(D, c, gw, v[cb], v[cb + 1], v[cb + 2], ob, od, oh);
        o.put((size_t)cb * ldy + n, ob);
        o.put((size_t)(cb + 1) * ldy + n, od);
        o.put((size_t)(cb + 2) * ldy + n, oh);
        if (Tw) Tw[(size_t)j * n_out + n] = D.s2 * v[cb];
    }
    for (int cc = n_cols(r) + sub; cc < CP; cc += tpr) o.put((size_t)cc * ldy + n, 0.f);
}

// Partials of one block of NR rows held in shared memory (row stride TS): per row k a
// left factor L_k,i (column kShared + 3i + xoff), right factors R_k,j (column kShared +
// 3j: J side; + 2: dJ side), a weight ms[k] and a scalar as[k] (ms, as after the NR
// rows);
//   out = [sum_k L_k,i as_k | sum_k ms_k L_k,i R_k,j (upper) | sum_k ms_k L_k,i R'_k,j]
// in the layout of k_row_reduce (partial row tl), by 128 threads (named barrier 1;
// thread `row` owns a 4 x 4 block of one of the two r x r sums).
template <int NR = 128>
static __device__ __forceinline__ void reduce_row_block(const FwdArgs& A, float* tile, int TS,
                                                     int row, int tl, int xoff) {
    const int r = A.r;
    float* __restrict__ out = A.row_part + (size_t)tl * A.row_stride;
    float* ms = tile + (size_t)NR * TS;
    float* as = ms + NR;
    asm volatile("bar.sync 1, 128;" ::: "memory");
    const int nsym = r * (r + 1) / 2;
    // 4x4 register blocks: threads 0-63 own blocks of J^T M J, 64-127 of J^T M dJ;
    // threads with bj == 0 of the first half also form J^T a
    const int mat = row >> 6, blk = row & 63, bi = blk >> 3, bj = blk & 7;
    int ci[4], cj[4];
    bool vi[4], vj[4];
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int i = 4 * bi + q, j = 4 * bj + q;
        vi[q] = i < r;
        vj[q] = j < r;
        ci[q] = kShared + 3 * (vi[q] ? i : 0) + xoff;
        cj[q] = kShared + 3 * (vj[q] ? j : 0) + (mat ? 2 : 0);
    }
    float acc[4][4], accp[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        accp[p] = 0.f;
#pragma unroll
        for (int q = 0; q < 4; ++q) acc[p][q] = 0.f;
    }
    const bool do_phi = (mat == 0 && bj == 0);
#pragma unroll 8
    for (int k = 0; k < NR; ++k) {
        const float* tk = tile + k * TS;
        const float mk = ms[k], ak = as[k];
        float Ji[4], Xj[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) { Ji[q] = tk[ci[q]]; Xj[q] = tk[cj[q]]; }
        if (do_phi) {
#pragma unroll
            for (int p = 0; p < 4; ++p) accp[p] = fmaf(Ji[p], ak, accp[p]);
        }
#pragma unroll
        for (int p = 0; p < 4; ++p) {
            const float mJ = mk * Ji[p];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[p][q] = fmaf(mJ, Xj[q], acc[p][q]);
        }
    }
#pragma unroll
    for (int p = 0; p < 4; ++p) {
        const int i = 4 * bi + p;
        if (!vi[p]) continue;
        if (do_phi) out[i] = accp[p];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int j = 4 * bj + q;
            if (!vj[q]) continue;
            if (mat == 0) {
                if (i <= j) out[r + i * r - i * (i - 1) / 2 + (j - i)] = acc[p][q];
            } else {
                out[r + nsym + i * r + j] = acc[p][q];
            }
        }
    }
    asm volatile("bar.sync 1, 128;" ::: "memory");   // the tile is reused afterwards
}

// 128 rows held in shared memory (row stride TS):  y_n = sum_j J_nj z_j + H[D,D]_n,
// a_n = m_n y_n - dt^2 f_ext,n;  partials [J^T a | J^T M J (upper) | J^T M dJ] of
// tile `tl` go to A.row_part (the layout of k_row_reduce).  All 128 epilogue
// threads call this together (named barrier 1); `tile` needs 128*TS + 256 floats.
// zs: z = (q - qbar) - dt qbar_dot (r floats) staged in shared memory by the caller.
static __device__ __forceinline__ void fused_row_reduce(const FwdArgs& A, float* tile, int TS,
                                                     int row, int n, bool wok, int tl,
                                                     const float* zs) {
    const int r = A.r, N = A.n_out, CP = A.Cp;
    const float ih = (float)A.inv_h, ih2 = (float)A.inv_h2, ih3 = (float)A.inv_h3;
    const float* __restrict__ mdof = A.mdof;
    const float* __restrict__ f_ext = A.f_ext;
    float* __restrict__ a_out = A.a_out;
    const double dt2 = A.dt * A.dt;
    float* vrow = tile + (size_t)row * TS;
    float* ms = tile + (size_t)128 * TS;
    float* as = ms + 128;
    float m = 0.f, av = 0.f;
    if (wok && n < N) {
        m = mdof[n];
        const float fe = f_ext ? f_ext[n] : 0.f;
        // this row's J and dJ in physical units (in place: the outputs are written);
        // eight columns' loads issue before their stores
        float y = vrow[3] * ih2;
        for (int j0 = 0; j0 < r; j0 += 8) {
            float Jv[8], dv[8], z[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                const int j = j0 + u < r ? j0 + u : r - 1;
                Jv[u] = vrow[kShared + 3 * j] * ih;
                dv[u] = vrow[kShared + 3 * j + 2] * ih3;
                z[u] = zs[j];
            }
#pragma unroll
            for (int u = 0; u < 8; ++u) {
                if (j0 + u < r) {
                    vrow[kShared + 3 * (j0 + u)] = Jv[u];
                    vrow[kShared + 3 * (j0 + u) + 2] = dv[u];
                    y = fmaf(Jv[u], z[u], y);
                }
            }
        }
        av = (float)((double)m * y - dt2 * (double)fe);
        if (a_out) a_out[n] = av;
    } else {
        // failed tile, or rows past N (zero rows of the padded weights): no contribution
        for (int c = 0; c < CP; ++c) vrow[c] = 0.f;
    }
    ms[row] = m;
    as[row] = av;
    reduce_row_block(A, tile, TS, row, tl, 0);
}

// Gram form of the reductions: row k < K of the block holds p = (G X)[k] (G = W_L^T M W_L,
// X the output layer's input columns).  With the column maps of the output epilogue
// (J_j = col(kShared+3j)/h, dJ_j = col(kShared+3j+2)/h^3, y = col(3)/h^2 + J z) applied
// to p and to x = X[:, k], and W_L linear,
//   J^T M J = sum_k xJ_k pJ_k^T,  J^T M dJ = sum_k xJ_k pdJ_k^T,
//   J^T (M y - dt^2 f_ext) = sum_k xJ_k (py_k - dt^2 (W_L^T f_ext)_k),
// the same partials as fused_row_reduce over the N output rows.  py = (G x_y)_k goes to
// A.gy (the reverse pass's seed W_L^T M y).
// NR rows per block: threads row < NR form their row's terms, all 128 the sums.
template <int NR = 128>
static __device__ __forceinline__ void gram_row_reduce(const FwdArgs& A, float* tile, int TS,
                                                    int row, int k, bool wok, int tl,
                                                    const float* zs) {
    const int r = A.r, K = A.K, CP = A.Cp;
    const float ih = (float)A.inv_h, ih2 = (float)A.inv_h2, ih3 = (float)A.inv_h3;
    const double dt2 = A.dt * A.dt;
    float* vrow = tile + (size_t)row * TS;
    float* ms = tile + (size_t)NR * TS;
    float* as = ms + NR;
    float av = 0.f;
    if (row >= NR) {
        // no row of this block
    } else if (wok && k < K) {
        const float* __restrict__ X = A.Xg;
        const size_t ldx = A.ldxg;
        float py = vrow[3] * ih2;
        // the row's input activations of every group first: all r global loads in flight
        float xj[kMaxR];
#pragma unroll
        for (int j = 0; j < kMaxR; ++j)
            xj[j] = j < r ? X[(size_t)(kShared + 3 * j) * ldx + k] : 0.f;
#pragma unroll
        for (int j = 0; j < kMaxR; ++j) {
            if (j < r) {
                const int cb = kShared + 3 * j;
                const float pj = vrow[cb] * ih;
                vrow[cb] = pj;
                vrow[cb + 1] = xj[j] * ih;
                vrow[cb + 2] = vrow[cb + 2] * ih3;
                py = fmaf(pj, zs[j], py);
            }
        }
        if (A.gy) A.gy[k] = py;
        av = (float)((double)py - (A.pext ? dt2 * (double)A.pext[k] : 0.0));
    } else {
        for (int c = 0; c < CP; ++c) vrow[c] = 0.f;
    }
    if (row < NR) {
        ms[row] = 1.f;
        as[row] = av;
    }
    reduce_row_block<NR>(A, tile, TS, row, tl, 1);
}

}  // namespace tc
}  // namespace dae
