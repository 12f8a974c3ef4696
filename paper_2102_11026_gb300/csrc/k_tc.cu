// Tensor-core forward GEMMs of the stacked complex-step batch (Sec. 4.3, Sec. 6
// "CR formulation": real weights act on every stacked component column, so each
// layer is one dense real GEMM).  sm_103a: TMA tile loads into 128B-swizzled
// shared memory, tcgen05.mma (one issuing thread) accumulating in TMEM,
// epilogue warps reading TMEM with tcgen05.ld and applying the multicomplex
// activation / output epilogue of epilogue.cuh.
//
// Tile: 128 output rows (TMEM lanes) x Cp component columns (TMEM columns), the
// whole K loop in one CTA.  Warp 0: TMA producer; warp 1: TMEM owner + MMA
// issuer; warps 2-5: epilogue.  Every mbarrier wait is bounded (2 s of
// %globaltimer); a wait that gives up records DAE_ERR_TIMEOUT and the CTA
// drains its copies, frees TMEM and exits.
#include <cuda.h>
#include <algorithm>
#include "dae_internal.h"
#include "epilogue.cuh"
#include "tc_common.cuh"

namespace dae {

namespace {

using namespace tc;

constexpr int kMaxStages = 8;
constexpr int kThreads = 192;

template <int NC, int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    k_fwd_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmAlo,
             const __grid_constant__ CUtensorMap tmB, const __grid_constant__ CUtensorMap tmBlo,
             FwdArgs A, int nk, int stages, int split) {
    constexpr int CP = 16 * NC;
    constexpr bool X3 = (PREC == DAE_BF16X3);
    constexpr int KB = (PREC == DAE_TF32) ? 32 : 64;         // K elements per 128-byte row
    constexpr uint32_t A_BYTES = 128 * 128;
    constexpr uint32_t B_BYTES = CP * 128;
    constexpr uint32_t STAGE = (A_BYTES + B_BYTES) * (X3 ? 2 : 1);
    constexpr uint32_t TMEM_COLS = (CP <= 32) ? 32 : (CP <= 64 ? 64 : 128);
    constexpr uint32_t ID = idesc(PREC == DAE_TF32 ? 2u : 1u, 128, CP);

    // the reverse-pass modes (2, 3) also stop when the evaluation needs no Newton matrix
    if (A.ns && (A.ns->done || (A.mode >= 2 && A.ns->skip_rev))) return;

    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], tfull;
    __shared__ uint32_t tmem_base;
    __shared__ int fail;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * 128;
    // split-K: this CTA takes k-blocks [kb0, kb1)
    const int kb0 = (int)((long long)nk * blockIdx.y / split);
    const int kb1 = (int)((long long)nk * (blockIdx.y + 1) / split);
    const int nkl = kb1 - kb0;
    __shared__ int is_last;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&tfull, 1);
        fail = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(&tmem_base, TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;

    if (warp == 0) {
        if (lane == 0) {
            int issued = 0;
            for (int kb = 0; kb < nkl; ++kb) {
                const int s = kb % stages;
                const uint32_t ph = (kb / stages) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1)) { fail = 1; break; }
                mbar_expect_tx(&full[s], STAGE);
                uint8_t* base = smem + (size_t)s * STAGE;
                const int kx = (kb0 + kb) * KB;
                tma_load_2d(base, &tmA, &full[s], kx, m0);
                tma_load_2d(base + A_BYTES, &tmB, &full[s], kx, 0);
                if constexpr (X3) {
                    tma_load_2d(base + A_BYTES + B_BYTES, &tmAlo, &full[s], kx, m0);
                    tma_load_2d(base + 2 * A_BYTES + B_BYTES, &tmBlo, &full[s], kx, 0);
                }
                ++issued;
            }
            // drain: the last load of every stage has landed before the CTA may exit
            for (int kb = (issued > stages ? issued - stages : 0); kb < issued; ++kb) {
                if (!mbar_wait(&full[kb % stages], (kb / stages) & 1)) fail = 1;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            bool ok = true;
            for (int kb = 0; kb < nkl; ++kb) {
                const int s = kb % stages;
                const uint32_t ph = (kb / stages) & 1;
                if (!mbar_wait(&full[s], ph)) { ok = false; fail = 1; break; }
                tc_fence_after();
                const uint32_t base = smem_u32(smem + (size_t)s * STAGE);
                const uint64_t da = sdesc(base), db = sdesc(base + A_BYTES);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const uint32_t acc = (kb | k) != 0;
                    mma<PREC>(tmem, da + 2 * k, db + 2 * k, ID, acc);
                    if constexpr (X3) {
                        const uint64_t dal = sdesc(base + A_BYTES + B_BYTES);
                        const uint64_t dbl = sdesc(base + 2 * A_BYTES + B_BYTES);
                        mma<PREC>(tmem, da + 2 * k, dbl + 2 * k, ID, 1u);
                        mma<PREC>(tmem, dal + 2 * k, db + 2 * k, ID, 1u);
                    }
                }
                mma_commit(&empty[s]);
            }
            mma_commit(&tfull);
            (void)ok;
        }
    } else {
        const bool ok = mbar_wait(&tfull, 0);
        tc_fence_after();
        const int lane_base = 32 * (warp & 3);
        const int row = lane_base + lane;
        const int n = m0 + row;
        // the pipeline buffers are idle once the accumulator is complete: stage the
        // tile there, one row per thread (odd stride: conflict-free)
        constexpr int TS = CP + 1;
        float* tile = reinterpret_cast<float*>(smem);
        float* vrow = tile + (size_t)row * TS;
        const bool wok = epi_all(ok);
        if (wok) {
#pragma unroll
            for (int c = 0; c < NC; ++c) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)lane_base << 16) + 16 * c, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) vrow[16 * c + i] = v[i];
            }
        } else {
            fail = 1;
            for (int c = 0; c < CP; ++c) vrow[c] = 0.f;
        }
        if (split == 1) {
            if (wok) row_epilogue(A, n, vrow);
            if (A.mode == 1 && A.row_part) {
                __shared__ float s_z[kMaxR];
                if (row < A.r) s_z[row] = A.zvec[row];
                asm volatile("bar.sync 1, 128;" ::: "memory");
                fused_row_reduce(A, tile, TS, row, n, wok, blockIdx.x, s_z);
            }
        } else {
            // write this split's partial tile [tile][split][c][128 rows]; the last CTA of the
            // tile (atomic count, no waiting) sums the partials in split order and finishes
            float* part = A.split_part + ((size_t)blockIdx.x * split + blockIdx.y) * CP * 128;
            for (int c = 0; c < CP; ++c) part[(size_t)c * 128 + row] = vrow[c];
            __threadfence();
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (warp == 2 && lane == 0) {
                const int old = atomicAdd(A.split_cnt + blockIdx.x, 1);
                is_last = (old == split - 1);
                if (is_last) A.split_cnt[blockIdx.x] = 0;
            }
            asm volatile("bar.sync 1, 128;" ::: "memory");
            if (is_last) {
                __threadfence();
                const float* tp = A.split_part + (size_t)blockIdx.x * split * CP * 128;
                for (int c = 0; c < CP; ++c) {
                    float acc = 0.f;
                    for (int s = 0; s < split; ++s) acc += __ldcg(tp + ((size_t)s * CP + c) * 128 + row);
                    vrow[c] = acc;
                }
                row_epilogue(A, n, vrow);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
    if (threadIdx.x == 0 && fail && A.status) atomicCAS(A.status, 0, (int)DAE_ERR_TIMEOUT);
}

template <int NC, int PREC>
bool launch_inst(cudaStream_t s, const FwdArgs& a, int split) {
    constexpr int CP = 16 * NC;
    constexpr bool X3 = (PREC == DAE_BF16X3);
    constexpr uint32_t STAGE = (128 * 128 + CP * 128) * (X3 ? 2 : 1);
    // the output layer streams many tiles: two CTAs per SM (about 110 KB each) so one
    // CTA's epilogue overlaps the other's loads; single-tile layers take deep pipelines
    const size_t budget = 200 * 1024;
    int stages = (int)(budget / STAGE);
    stages = stages < 2 ? 2 : (stages > kMaxStages ? kMaxStages : stages);
    const size_t tile_need = (size_t)128 * (CP + 1) * 4 + 256 * 4;
    while ((size_t)stages * STAGE < tile_need) ++stages;
    const size_t smem = (size_t)stages * STAGE + 1024;
    static size_t configured = 0;
    if (smem > configured) {
        if (cudaFuncSetAttribute(k_fwd_tc<NC, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)std::max(smem, (size_t)200 * 1024 + 1024)) != cudaSuccess)
            return false;
        configured = std::max(smem, (size_t)200 * 1024 + 1024);
    }
    const int KB = (PREC == DAE_TF32) ? 32 : 64;
    const int nk = a.ld / KB;
    const CUtensorMap* tm = reinterpret_cast<const CUtensorMap*>(a.tmaps);
    dim3 grid(a.m_pad / 128, split);
    k_fwd_tc<NC, PREC><<<grid, kThreads, smem, s>>>(tm[0], tm[1], tm[2], tm[3], a, nk, stages,
                                                   split);
    return cudaPeekAtLastError() == cudaSuccess;
}

template <int PREC>
bool launch_prec(cudaStream_t s, const FwdArgs& a, int split) {
    switch (a.Cp / 16) {
        case 1: return launch_inst<1, PREC>(s, a, split);
        case 2: return launch_inst<2, PREC>(s, a, split);
        case 3: return launch_inst<3, PREC>(s, a, split);
        case 4: return launch_inst<4, PREC>(s, a, split);
        case 5: return launch_inst<5, PREC>(s, a, split);
        case 6: return launch_inst<6, PREC>(s, a, split);
        case 7: return launch_inst<7, PREC>(s, a, split);
    }
    return false;
}

}  // namespace

// Split-K factor: fill about one CTA per SM with at least 4 k-blocks per split;
// the output layer (and any layer with enough row tiles) runs unsplit.
int tc_split(int m_pad, int ld, dae_prec prec, int sm_count) {
    const int tiles = m_pad / 128;
    const int nk = ld / (prec == DAE_TF32 ? 32 : 64);
    int split = sm_count / tiles;
    split = std::min(split, nk / 4);
    split = std::min(split, kMaxSplit);
    return split < 2 ? 1 : split;
}

bool launch_fwd_tc(cudaStream_t s, const FwdArgs& a, dae_prec prec, int sm_count) {
    if (!a.tmaps || a.m_pad % 128 != 0) return false;
    int split = (a.mode == 1) ? 1 : tc_split(a.m_pad, a.ld, prec, sm_count);
    if (!a.split_part || !a.split_cnt) split = 1;
    switch (prec) {
        case DAE_TF32: return launch_prec<DAE_TF32>(s, a, split);
        case DAE_BF16: return launch_prec<DAE_BF16>(s, a, split);
        case DAE_BF16X3: return launch_prec<DAE_BF16X3>(s, a, split);
        default: return false;
    }
}

// ------------------------------------------------------------ tensor maps --
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiledFn>(p);
        cudaGetLastError();
    }
    return fn;
}

// 2-D row-major matrix [rows][ld] of `elem` bytes, box {box_k elements, box_rows}, 128B swizzle.
bool make_tmap(void* out, const void* base, bool fp32, int ld, int rows, int box_rows) {
    EncodeTiledFn fn = encode_fn();
    if (!fn || !base) return false;
    const int esz = fp32 ? 4 : 2;
    cuuint64_t dims[2] = {(cuuint64_t)ld, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)ld * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1, 1};
    CUresult r = fn(reinterpret_cast<CUtensorMap*>(out),
                    fp32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                    const_cast<void*>(base), dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                    CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                    CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

}  // namespace dae
