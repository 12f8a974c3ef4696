// Persistent tensor-core kernel for a chain of small GEMM layers: the hidden
// layers of the stacked complex-step forward pass (Sec. 4.3) and the hidden
// layers of the complex-step reverse pass (Sec. 4.4).
//
// One CTA per SM for the whole chain (cooperative launch): barriers, TMEM and
// the instruction stream are set up once instead of once per layer.  Each layer
// ("job") is split into work items (128-row tile x K chunk) dealt round-robin to
// the CTAs; a grid-wide barrier separates the layers (the next layer's TMA reads
// the activations the previous layer's epilogue wrote).  K-split partial tiles go
// to global scratch and are reduced, in split order, after a second barrier.
//
// Roles as in k_tc.cu: warp 0 TMA producer, warp 1 TMEM owner + MMA issuer,
// warps 2-5 epilogue.  The accumulator is staged through a shared-memory tile so
// the MMA of the next item can start while the epilogue runs.  Every wait
// (mbarrier or grid barrier) is bounded; a wait that gives up records
// DAE_ERR_TIMEOUT, and the CTA stops issuing work, drains and exits.
#include <algorithm>
#include "tc_common.cuh"

namespace dae {

using namespace tc;

namespace {

constexpr int kThreads = 192;
constexpr int kMaxStages = 8;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Sense-reversing grid barrier, thread 0 of each CTA; false on timeout.
__device__ bool grid_barrier(GridBar* gb, unsigned nblocks, unsigned& gen) {
    __threadfence();
    const unsigned g = gen;
    const unsigned arrived = atomicAdd(&gb->count, 1u) + 1u;
    if (arrived == nblocks) {
        gb->count = 0u;
        __threadfence();
        atomicExch(&gb->gen, g + 1u);
    } else {
        const uint64_t t0 = globaltimer();
        while (ld_acquire(&gb->gen) == g) {
            if (globaltimer() - t0 > kWaitNs) return false;
        }
    }
    gen = g + 1u;
    __threadfence();
    return true;
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}

template <int NC, int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    k_chain(const ChainJob* __restrict__ jobs, int n_jobs, GridBar* gb, const NewtonState* ns,
            int* status, float* split_part, int* split_cnt, int stages) {
    constexpr int CP = 16 * NC;
    constexpr bool X3 = (PREC == DAE_BF16X3);
    constexpr int KB = (PREC == DAE_TF32) ? 32 : 64;
    constexpr uint32_t A_BYTES = 128 * 128;
    constexpr uint32_t B_BYTES = CP * 128;
    constexpr uint32_t STAGE = (A_BYTES + B_BYTES) * (X3 ? 2 : 1);
    constexpr uint32_t TMEM_COLS = (CP <= 32) ? 32 : (CP <= 64 ? 64 : 128);
    constexpr uint32_t ID = idesc(PREC == DAE_TF32 ? 2u : 1u, 128, CP);
    constexpr int TS = CP + 1;

    if (ns && ns->done) return;   // uniform: every CTA reads the same flag

    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], tfull, tempty;
    __shared__ uint32_t tmem_base;
    __shared__ int fail;
    __shared__ int is_last;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~(uintptr_t)1023);
    float* tile = reinterpret_cast<float*>(smem + (size_t)stages * STAGE);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const unsigned G = gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < stages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&tfull, 1);
        mbar_init(&tempty, 128);
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
    unsigned gen = 0;
    if (threadIdx.x == 0) gen = *(volatile unsigned*)&gb->gen;

    uint32_t pk = 0;   // stage-ring position (producer and MMA walk it identically)
    uint32_t it = 0;   // items taken by this CTA (tfull / tempty phases)
    for (int j = 0; j < n_jobs; ++j) {
        const ChainJob& Jb = jobs[j];
        const int tiles = Jb.tiles, split = Jb.split, nk = Jb.nk;
        const int items = tiles * split;
        const CUtensorMap* tmA = &Jb.tm[0];
        const CUtensorMap* tmAlo = &Jb.tm[1];
        const CUtensorMap* tmB = &Jb.tm[2];
        const CUtensorMap* tmBlo = &Jb.tm[3];
        if (warp == 0) {
            if (lane == 0 && !fail) {
                if ((int)blockIdx.x < items) {
                    prefetch_tmap(tmA);
                    prefetch_tmap(tmB);
                    if constexpr (X3) { prefetch_tmap(tmAlo); prefetch_tmap(tmBlo); }
                }
                for (int item = blockIdx.x; item < items && !fail; item += G) {
                    const int tl = item / split, ks = item % split;
                    const int kb0 = (int)((long long)nk * ks / split);
                    const int kb1 = (int)((long long)nk * (ks + 1) / split);
                    for (int kb = kb0; kb < kb1; ++kb, ++pk) {
                        const int s = pk % stages;
                        const uint32_t ph = (pk / stages) & 1;
                        if (!mbar_wait(&empty[s], ph ^ 1)) { fail = 1; break; }
                        mbar_expect_tx(&full[s], STAGE);
                        uint8_t* base = smem + (size_t)s * STAGE;
                        tma_load_2d(base, tmA, &full[s], kb * KB, tl * 128);
                        tma_load_2d(base + A_BYTES, tmB, &full[s], kb * KB, 0);
                        if constexpr (X3) {
                            tma_load_2d(base + A_BYTES + B_BYTES, tmAlo, &full[s], kb * KB, tl * 128);
                            tma_load_2d(base + 2 * A_BYTES + B_BYTES, tmBlo, &full[s], kb * KB, 0);
                        }
                    }
                }
            }
        } else if (warp == 1) {
            if (lane == 0 && !fail) {
                for (int item = blockIdx.x; item < items && !fail; item += G, ++it) {
                    const int ks = item % split;
                    const int kb0 = (int)((long long)nk * ks / split);
                    const int kb1 = (int)((long long)nk * (ks + 1) / split);
                    if (!mbar_wait(&tempty, (it & 1) ^ 1)) { fail = 1; break; }
                    tc_fence_after();
                    for (int kb = kb0; kb < kb1; ++kb, ++pk) {
                        const int s = pk % stages;
                        const uint32_t ph = (pk / stages) & 1;
                        if (!mbar_wait(&full[s], ph)) { fail = 1; break; }
                        tc_fence_after();
                        const uint32_t base = smem_u32(smem + (size_t)s * STAGE);
                        const uint64_t da = sdesc(base), db = sdesc(base + A_BYTES);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t acc = (kb > kb0 || k > 0) ? 1u : 0u;
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
                }
            }
        } else {
            const int lane_base = 32 * (warp & 3);
            const int row = lane_base + lane;
            float* vrow = tile + (size_t)row * TS;
            for (int item = blockIdx.x; item < items; item += G, ++it) {
                const int tl = item / split, ks = item % split;
                const bool ok = mbar_wait(&tfull, it & 1);
                tc_fence_after();
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
                }
                tc_fence_before();
                mbar_arrive(&tempty);          // TMEM may be overwritten by the next item
                if (!wok) break;
                if (split == 1) {
                    row_epilogue(Jb.a, tl * 128 + row, vrow);
                    if (Jb.a.mode == 1 && Jb.a.row_part)
                        fused_row_reduce(Jb.a, tile, TS, row, tl * 128 + row, true, tl);
                } else {
                    // K-split partial tile; the last CTA to finish this tile (atomic count,
                    // no waiting) sums the partials in split order and runs the epilogue
                    float* part = split_part + ((size_t)tl * split + ks) * CP * 128;
#pragma unroll 8
                    for (int c = 0; c < CP; ++c) part[(size_t)c * 128 + row] = vrow[c];
                    __threadfence();
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    if (warp == 2 && lane == 0) {
                        const int old = atomicAdd(split_cnt + tl, 1);
                        is_last = (old == split - 1);
                        if (is_last) split_cnt[tl] = 0;
                    }
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    if (is_last) {
                        __threadfence();
                        const float* tp = split_part + (size_t)tl * split * CP * 128 + row;
                        for (int c0 = 0; c0 < CP; c0 += 8) {
                            float acc[8];
#pragma unroll
                            for (int i = 0; i < 8; ++i) acc[i] = 0.f;
                            for (int s = 0; s < split; ++s) {
#pragma unroll
                                for (int i = 0; i < 8; ++i)
                                    acc[i] += __ldcg(tp + ((size_t)s * CP + c0 + i) * 128);
                            }
#pragma unroll
                            for (int i = 0; i < 8; ++i) vrow[c0 + i] = acc[i];
                        }
                        row_epilogue(Jb.a, tl * 128 + row, vrow);
                    }
                    asm volatile("bar.sync 1, 128;" ::: "memory");   // is_last reused next item
                }
            }
            fence_proxy_async_global();       // epilogue stores feed the next layer's TMA
        }
        __syncthreads();
        if (threadIdx.x == 0 && !grid_barrier(gb, G, gen)) fail = 1;
        __syncthreads();
        if (fail) break;
    }
    // drain: nothing in flight may outlive the CTA
    if (warp == 0 && lane == 0) {
        for (uint32_t k = (pk > (uint32_t)stages ? pk - stages : 0); k < pk; ++k)
            if (!mbar_wait(&full[k % stages], (k / stages) & 1)) fail = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, TMEM_COLS);
    }
    if (threadIdx.x == 0 && fail && status) atomicCAS(status, 0, (int)DAE_ERR_TIMEOUT);
}

template <int NC, int PREC>
bool launch_chain_inst(cudaStream_t s, const ChainLaunch& c) {
    constexpr int CP = 16 * NC;
    constexpr bool X3 = (PREC == DAE_BF16X3);
    constexpr uint32_t STAGE = (128 * 128 + CP * 128) * (X3 ? 2 : 1);
    const size_t tile_bytes = (size_t)128 * (CP + 1) * 4 + 256 * 4;
    const size_t budget = 220 * 1024 - tile_bytes - 1024;
    int stages = (int)(budget / STAGE);
    stages = stages < 2 ? 2 : (stages > kMaxStages ? kMaxStages : stages);
    const size_t smem = (size_t)stages * STAGE + tile_bytes + 1024;
    static bool configured = false;
    if (!configured) {
        if (cudaFuncSetAttribute(k_chain<NC, PREC>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem) != cudaSuccess)
            return false;
        configured = true;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c.grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_chain<NC, PREC>, c.jobs, c.n_jobs, c.gb, c.ns, c.status,
                              c.split_part, c.split_cnt, stages) == cudaSuccess;
}

template <int PREC>
bool launch_chain_prec(cudaStream_t s, const ChainLaunch& c) {
    switch (c.Cp / 16) {
        case 1: return launch_chain_inst<1, PREC>(s, c);
        case 2: return launch_chain_inst<2, PREC>(s, c);
        case 3: return launch_chain_inst<3, PREC>(s, c);
        case 4: return launch_chain_inst<4, PREC>(s, c);
        case 5: return launch_chain_inst<5, PREC>(s, c);
        case 6: return launch_chain_inst<6, PREC>(s, c);
        case 7: return launch_chain_inst<7, PREC>(s, c);
    }
    return false;
}

}  // namespace

// Self-test of the bounded waits: an mbarrier that nothing arrives on and a grid
// barrier that expects one CTA more than the grid has.  Both must give up within
// their limit; out[b] = 1 when CTA b saw both time out.
__global__ void k_wait_selftest(GridBar* gb, int* out) {
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool mb = mbar_wait(&bar, 0);               // no arrival: must time out
        unsigned gen = *(volatile unsigned*)&gb->gen;
        const bool gbok = grid_barrier(gb, gridDim.x + 1, gen);   // one CTA short: times out
        out[blockIdx.x] = (!mb && !gbok) ? 1 : 0;
    }
}

int run_wait_selftest(cudaStream_t s, GridBar* gb, int* out, int nblocks) {
    k_wait_selftest<<<nblocks, 32, 0, s>>>(gb, out);
    return cudaGetLastError() == cudaSuccess ? 0 : 1;
}

// Writes one job into device memory (stream-ordered; the job travels as a kernel
// parameter, so the caller's copy may change right after the launch).
__global__ void k_store_job(ChainJob* dst, ChainJob job) {
    const int n = sizeof(ChainJob) / sizeof(int);
    const int* src = reinterpret_cast<const int*>(&job);
    for (int i = threadIdx.x; i < n; i += blockDim.x) reinterpret_cast<int*>(dst)[i] = src[i];
}

void launch_store_job(cudaStream_t s, ChainJob* dst, const ChainJob& job) {
    k_store_job<<<1, 128, 0, s>>>(dst, job);
}

bool launch_chain(cudaStream_t s, const ChainLaunch& c, dae_prec prec) {
    switch (prec) {
        case DAE_TF32: return launch_chain_prec<DAE_TF32>(s, c);
        case DAE_BF16: return launch_chain_prec<DAE_BF16>(s, c);
        case DAE_BF16X3: return launch_chain_prec<DAE_BF16X3>(s, c);
        default: return false;
    }
}

// Items per job: enough K chunks that tiles x split covers the grid, at least
// 4 k-blocks per chunk.
int chain_split(int tiles, int nk, int grid) {
    int split = grid / std::max(tiles, 1);
    split = std::min(split, nk / 4);
    split = std::min(split, kMaxSplit);
    return split < 2 ? 1 : split;
}

}  // namespace dae
