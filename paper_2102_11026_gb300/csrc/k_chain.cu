// Persistent tensor-core kernel for a chain of GEMM layers: the hidden layers of
// the stacked complex-step forward pass (Sec. 4.3), the hidden layers of the
// complex-step reverse pass (Sec. 4.4), and (as a one-job chain) the output layer.
//
// One CTA per SM for the whole chain (cooperative launch): barriers, TMEM and the
// instruction stream are set up once instead of once per layer.  Each layer
// ("job") is cut into items (128-row tile x K range) dealt round-robin to the CTAs.
// In a single decoder's chain a layer's k-block is loaded once the tile of the layer
// before that wrote its rows is complete (per-tile ready counters, no barrier between
// layers); grouped launches put a grid-wide barrier between their stages.
//
// Short-K layers replicate the whole K loop on `rep` CTAs per tile; long-K layers
// split K over `split` CTAs per tile, which publish the partners' slices of their
// partial tiles (bulk copies), wait for one another and bulk-load the partners' slices
// of their own rows into the spare rows of the staging tile before summing.  Either way each of
// the P CTAs of a tile finishes 128/P rows, so the activation epilogue of a layer is
// spread over tiles x P CTAs instead of one CTA per tile.  The producer issues each
// k-block's weight half at once (weights do not depend on the layer in flight) and its
// activation half once the tile that wrote those rows is complete, so a CTA's next
// layer streams while its own epilogue of the layer before still runs.
//
// Roles: warp 0 TMA producer, warp 1 TMEM owner + MMA issuer, warps 2-5 epilogue.
// The accumulator is staged through a shared-memory tile so the MMA of the next
// item can start while the epilogue runs.  Every wait (mbarrier, partner tiles,
// grid barrier) is bounded; a wait that gives up records DAE_ERR_TIMEOUT, and the
// CTA stops issuing work, drains and exits.
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


// Grid barrier, thread 0 of each CTA (after a __syncthreads of its CTA); false on
// timeout.  The arrival counter only grows: the barrier of generation g completes at
// (g + 1) * nblocks arrivals, so nothing is reset (count == gen * nblocks between
// barriers; the host zeroes both after a timed-out launch).  The arrival is a release
// (it publishes the CTA's writes, ordered before it by the CTA barrier), the wait an
// acquire.
__device__ bool grid_barrier(GridBar* gb, unsigned nblocks, unsigned& gen) {
    const unsigned g = gen;
    const unsigned target = (g + 1u) * nblocks;
    unsigned old;
    asm volatile("atom.add.release.gpu.u32 %0, [%1], 1;" : "=r"(old) : "l"(&gb->count) : "memory");
    if (old + 1u == target) {
        asm volatile("st.release.gpu.u32 [%0], %1;" ::"l"(&gb->gen), "r"(g + 1u) : "memory");
    } else {
        const uint64_t t0 = globaltimer();
        while (ld_acquire(&gb->gen) == g) {
            if (globaltimer() - t0 > kWaitNs) return false;
        }
    }
    gen = g + 1u;
    return true;
}

// Bounded wait (one thread) until a producer tile's ready counter reaches `target`
// arrivals; then the async proxy (the TMA loads that follow) may read what they wrote.
__device__ bool wait_ready(const unsigned* cnt, unsigned target) {
    if (ld_acquire(cnt) < target) {
        const uint64_t t0 = globaltimer();
        while (ld_acquire(cnt) < target) {
            if (globaltimer() - t0 > kWaitNs) return false;
            __nanosleep(32);   // fewer polls of a line the finishers update
        }
    }
    asm volatile("fence.proxy.async.global;" ::: "memory");
    return true;
}

__device__ __forceinline__ void fence_proxy_async_global() {
    asm volatile("fence.proxy.async.global;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// Bulk copy of `bytes` (multiple of 16) from shared to global memory, waited for.
__device__ __forceinline__ void bulk_store_wait(void* gdst, const void* ssrc, uint32_t bytes) {
    asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(gdst),
                 "r"(smem_u32(ssrc)), "r"(bytes)
                 : "memory");
    asm volatile("cp.async.bulk.commit_group;" ::: "memory");
    asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
}

// Bulk copy of `bytes` (multiple of 16) from global to shared memory, completing on
// the transaction count of `bar`.
// Counts `bytes` of an mbarrier's expected transactions as done (for loads never issued).
__device__ __forceinline__ void mbar_complete_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.complete_tx.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ void bulk_load(void* sdst, const void* gsrc, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(sdst)),
        "l"(gsrc), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

__device__ __forceinline__ void prefetch_line_l2(const void* p) {
    asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}

struct Item {
    int tl, ks, kb0, kb1;
};

__device__ __forceinline__ Item item_of(int item, int P, int split, int nk) {
    Item it;
    it.tl = item / P;
    it.ks = item % P;
    if (split > 1) {
        it.kb0 = nk * it.ks / split;          // nk * split < 2^31: 32-bit integer division
        it.kb1 = nk * (it.ks + 1) / split;
    } else {
        it.kb0 = 0;
        it.kb1 = nk;
    }
    return it;
}

// The items of one job for CTA c.  Split / replicated jobs: items (tile, ks) dealt
// round-robin.  Stream jobs (T >= G): the CTA takes the contiguous range
// [c T / G, (c+1) T / G) of the job's T = tiles x nk k-blocks, so every CTA streams the
// same number (at least one) of k-blocks.  The range is cut at tile edges into a head piece (end of a tile begun by
// the previous CTA), a tail piece (start of a tile the next CTA ends) and whole
// tiles, taken as tail, one whole tile, head, the other whole tiles: every CTA
// publishes its tail piece first and finishes (last to arrive) the tile of its head
// piece after one whole tile, so no CTA's finishing work delays a piece another CTA
// waits for (a finishing epilogue, e.g. the Gram rows' reductions, takes several
// microseconds), and every CTA ends on whole tiles.
struct Walk {
    int P, split, nk, items, stream, G;
    long long T, g0, g1, hb, tb, cur;
    int item, stage;
    __device__ Walk(const ChainJob& J, int c, int G_) {
        split = J.split;
        P = split > J.rep ? split : J.rep;
        nk = J.nk;
        items = J.tiles * P;
        stream = J.stream;
        G = G_;
        stage = 0;
        item = c;
        if (J.solo) {            // a solo layer: every tile on CTA 0, in order
            G = 1;
            item = c == 0 ? 0 : items;
        }
        T = g0 = g1 = hb = tb = cur = 0;
        if (stream) {                   // 64-bit divisions only where the ranges are used
            T = (long long)J.tiles * nk;
            g0 = T * c / G;
            g1 = T * (c + 1) / G;
            hb = (g0 + nk - 1) / nk * nk;   // first tile edge at or after g0
            tb = g1 / nk * nk;              // last tile edge at or before g1
            cur = hb;
        }
    }
    __device__ void seg(Item& I, long long a, long long b) const {
        I.tl = (int)(a / nk);
        I.ks = 0;
        I.kb0 = (int)(a - (long long)I.tl * nk);
        I.kb1 = I.kb0 + (int)(b - a);
    }
    __device__ bool next(Item& I) {
        if (stream) {
            if (g0 >= g1) return false;
            if (hb > g1) {                       // the range lies inside one tile
                if (stage++ > 0) return false;
                seg(I, g0, g1);
                return true;
            }
            if (stage == 0) {                    // tail piece
                stage = 1;
                if (tb < g1 && tb >= hb) { seg(I, tb, g1); return true; }
            }
            if (stage == 1) {                    // first whole tile
                stage = 2;
                if (cur < tb) { seg(I, cur, cur + nk); cur += nk; return true; }
            }
            if (stage == 2) {                    // head piece
                stage = 3;
                if (g0 < hb) { seg(I, g0, hb); return true; }
            }
            if (cur < tb) {                      // other whole tiles
                seg(I, cur, cur + nk);
                cur += nk;
                return true;
            }
            return false;
        }
        if (item >= items) return false;
        I = item_of(item, P, split, nk);
        item += G;
        return true;
    }
};

// CTA of a stream job whose k-block range holds global k-block g.
__device__ __forceinline__ int stream_cta(long long g, long long T, int G) {
    return (int)(((g + 1) * G + T - 1) / T) - 1;
}

// The items of one stage for CTA c.  A single-decoder stage is one job walked by
// Walk.  A grouped stage is the list of its jobs' tiles (job t's tiles start at
// base[t], a table in shared memory), dealt round-robin over the grid; the tiles of
// jobs marked in skip are passed over.  Every role of a CTA walks the same sequence.
struct StageWalk {
    Walk w;
    const ChainJob* jobs;
    const int* base;
    const unsigned char* skip;
    int nj, total, item, G;
    bool grouped;
    __device__ StageWalk(const ChainJob* jobs_, int j0, int nj_, bool grouped_, const int* base_,
                         const unsigned char* skip_, int c, int G_)
        : w(jobs_[j0], c, G_), jobs(jobs_ + j0), base(base_), skip(skip_), nj(nj_),
          total(grouped_ ? base_[nj_] : 0), item(c), G(G_), grouped(grouped_) {}
    __device__ bool next(const ChainJob*& J, Item& I) {
        if (!grouped) {
            J = jobs;
            return w.next(I);
        }
        while (item < total) {
            const int i = item;
            item += G;
            int lo = 0, hi = nj - 1;   // last job whose first tile is at or before i
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (base[mid] <= i) lo = mid; else hi = mid - 1;
            }
            if (skip[lo]) continue;
            J = jobs + lo;
            I.tl = i - base[lo];
            I.ks = 0;
            I.kb0 = 0;
            I.kb1 = J->nk;
            return true;
        }
        return false;
    }
};

template <int NC, int PREC>
__global__ void __launch_bounds__(kThreads, 1)
    k_chain(const ChainJob* __restrict__ jobs, int n_jobs, GridBar* gb, const NewtonState* ns,
            int* status, float* split_part, unsigned* split_cnt, int stages,
            const int* __restrict__ stage_off, int n_stages) {
    constexpr int CP = 16 * NC;
    constexpr bool X3 = (PREC == DAE_BF16X3);
    constexpr int KB = (PREC == DAE_TF32) ? 32 : 64;
    constexpr uint32_t A_BYTES = 128 * 128;
    constexpr uint32_t B_BYTES = CP * 128;
    constexpr uint32_t STAGE = (A_BYTES + B_BYTES) * (X3 ? 2 : 1);
    constexpr uint32_t ACC_COLS = (CP <= 32) ? 32 : (CP <= 64 ? 64 : 128);
    constexpr uint32_t TMEM_COLS = 2 * ACC_COLS;   // two accumulators: MMA runs one item ahead
    constexpr uint32_t ID = idesc(PREC == DAE_TF32 ? 2u : 1u, 128, CP);
    constexpr int TS = CP + 1;
    constexpr uint32_t TILE_BYTES = 128u * TS * 4u;   // a partial tile as staged (multiple of 16)

    // uniform: every CTA reads the same flags; a reverse chain (modes 2, 3) also stops
    // when this evaluation needs no Newton matrix
    if (ns && (ns->done || (jobs[0].a.mode >= 2 && ns->skip_rev))) return;

    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kMaxStages], empty[kMaxStages], tfull[2], tempty[2], rbar;
    __shared__ uint32_t tmem_base;
    __shared__ int fail;
    __shared__ int s_last;
    __shared__ float s_z[kMaxR];   // z of the fused row reductions (output layer)
    __shared__ int s_base[kMaxGroupJobs + 1];           // grouped stage: first tile per job
    __shared__ unsigned char s_skip[kMaxGroupJobs];     // grouped stage: job skipped
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
        mbar_init(&tfull[0], 1);
        mbar_init(&tfull[1], 1);
        mbar_init(&tempty[0], 128);
        mbar_init(&tempty[1], 128);
        mbar_init(&rbar, 1);
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
    unsigned gen = 0;   // grid-barrier generation (thread 0)
    if (threadIdx.x == 0) gen = *(volatile unsigned*)&gb->gen;

    uint32_t pk = 0;   // stage-ring position (producer and MMA walk it identically)
    uint32_t it = 0;   // items taken by this CTA: accumulator it & 1, its use it >> 1
    uint32_t nred = 0; // split reductions of this CTA (rbar phases)
    const bool grouped = stage_off != nullptr;
    const int n_st = grouped ? n_stages : n_jobs;
    // a single decoder's chain runs without grid barriers between its layers: each CTA
    // finishing rows of a tile counts itself on the tile's ready counter, and a k-block's
    // activations are loaded once the tile that wrote them is complete (one grid barrier
    // at the end, after which the counters are zeroed for the next launch).  Two
    // activation buffers suffice: a layer's rows are written only after its CTAs (or their
    // split partners) consumed every tile of the layer before, hence after every read of
    // the buffer they overwrite.
    const bool flow = !grouped && n_jobs > 1;
    for (int st = 0; st < n_st; ++st) {
        const int j0 = grouped ? stage_off[st] : st;
        const int nj = grouped ? stage_off[st + 1] - j0 : 1;
        if (grouped) {
            // the stage's job table (the done flags are not written during the launch)
            for (int t = threadIdx.x; t < nj; t += blockDim.x) {
                const ChainJob& Jt = jobs[j0 + t];
                s_base[t] = Jt.item_base;
                s_skip[t] = (Jt.a.ns && (*(volatile const int*)&Jt.a.ns->done ||
                                         (Jt.a.mode >= 2 && *(volatile const int*)&Jt.a.ns->skip_rev)))
                                ? 1 : 0;
            }
            if (threadIdx.x == 0) s_base[nj] = jobs[j0 + nj - 1].item_base + jobs[j0 + nj - 1].tiles;
            __syncthreads();
        }
        if (warp == 0) {
            if (lane == 0 && !*(volatile int*)&fail) {
                StageWalk W(jobs, j0, nj, grouped, s_base, s_skip, blockIdx.x, G);
                const ChainJob* Jp;
                const ChainJob* Jlast = nullptr;
                Item I;
                if (grouped) {
                    // a grouped stage's items mostly belong to different jobs: fetch all of
                    // this CTA's descriptors up front so their latencies overlap
                    StageWalk Wd(jobs, j0, nj, grouped, s_base, s_skip, blockIdx.x, G);
                    while (Wd.next(Jp, I)) {
                        prefetch_tmap(&Jp->tm[0]);
                        prefetch_tmap(&Jp->tm[2]);
                        if constexpr (X3) { prefetch_tmap(&Jp->tm[1]); prefetch_tmap(&Jp->tm[3]); }
                    }
                }
                int rdy_tile = -1;   // previous layer's tile known complete (flow)
                while (!fail && W.next(Jp, I)) {
                    const CUtensorMap* tmA = &Jp->tm[0];
                    const CUtensorMap* tmAlo = &Jp->tm[1];
                    const CUtensorMap* tmB = &Jp->tm[2];
                    const CUtensorMap* tmBlo = &Jp->tm[3];
                    if (Jp != Jlast) {
                        prefetch_tmap(tmA);
                        prefetch_tmap(tmB);
                        if constexpr (X3) { prefetch_tmap(tmAlo); prefetch_tmap(tmBlo); }
                        Jlast = Jp;
                    }
                    for (int kb = I.kb0; kb < I.kb1; ++kb, ++pk) {
                        const int s = pk % stages;
                        const uint32_t ph = (pk / stages) & 1;
                        if (!mbar_wait(&empty[s], ph ^ 1)) { fail = 1; break; }
                        mbar_expect_tx(&full[s], STAGE);
                        uint8_t* base = smem + (size_t)s * STAGE;
                        tma_load_2d(base, tmA, &full[s], kb * KB, I.tl * 128);
                        if constexpr (X3) tma_load_2d(base + A_BYTES + B_BYTES, tmAlo, &full[s], kb * KB, I.tl * 128);
                        if (flow && st > 0) {
                            // the previous layer's tile holding this k-block's rows
                            const int pt = kb * KB / 128;
                            if (pt != rdy_tile) {
                                const ChainJob& Pb = jobs[st - 1];
                                const unsigned P = (unsigned)(Pb.split > Pb.rep ? Pb.split : Pb.rep);
                                if (!wait_ready(split_cnt + Pb.rdy_off + pt * kRdyStride, P)) {
                                    // settle the slot so that the MMA warp is not left waiting
                                    mbar_complete_tx(&full[s], B_BYTES * (X3 ? 2u : 1u));
                                    fail = 1;
                                    break;
                                }
                                rdy_tile = pt;
                            }
                        }
                        tma_load_2d(base + A_BYTES, tmB, &full[s], kb * KB, 0);
                        if constexpr (X3) tma_load_2d(base + 2 * A_BYTES + B_BYTES, tmBlo, &full[s], kb * KB, 0);
                    }
                }
            }
        } else if (warp == 1) {
            if (lane == 0 && !*(volatile int*)&fail) {
                StageWalk W(jobs, j0, nj, grouped, s_base, s_skip, blockIdx.x, G);
                const ChainJob* Jp;
                Item I;
                for (; !fail && W.next(Jp, I); ++it) {
                    const uint32_t ab = it & 1, au = (it >> 1) & 1;
                    const uint32_t dacc = tmem + ab * ACC_COLS;
                    if (!mbar_wait(&tempty[ab], au ^ 1)) { fail = 1; break; }
                    tc_fence_after();
                    for (int kb = I.kb0; kb < I.kb1; ++kb, ++pk) {
                        const int s = pk % stages;
                        const uint32_t ph = (pk / stages) & 1;
                        if (!mbar_wait(&full[s], ph)) { fail = 1; break; }
                        tc_fence_after();
                        const uint32_t base = smem_u32(smem + (size_t)s * STAGE);
                        const uint64_t da = sdesc(base), db = sdesc(base + A_BYTES);
#pragma unroll
                        for (int k = 0; k < 4; ++k) {
                            const uint32_t acc = (kb > I.kb0 || k > 0) ? 1u : 0u;
                            mma<PREC>(dacc, da + 2 * k, db + 2 * k, ID, acc);
                            if constexpr (X3) {
                                const uint64_t dal = sdesc(base + A_BYTES + B_BYTES);
                                const uint64_t dbl = sdesc(base + 2 * A_BYTES + B_BYTES);
                                mma<PREC>(dacc, da + 2 * k, dbl + 2 * k, ID, 1u);
                                mma<PREC>(dacc, dal + 2 * k, db + 2 * k, ID, 1u);
                            }
                        }
                        mma_commit(&empty[s]);
                    }
                    mma_commit(&tfull[ab]);
                }
            }
        } else {
            const int et = threadIdx.x - 64;          // epilogue thread 0..127
            const int lane_base = 32 * (warp & 3);    // TMEM lane quarter of this warp
            const int row = lane_base + lane;
            float* vrow = tile + (size_t)row * TS;
            StageWalk W(jobs, j0, nj, grouped, s_base, s_skip, blockIdx.x, G);
            const ChainJob* Jp;
            const ChainJob* Jlast = nullptr;
            Item I;
            // without barriers between layers, a failure elsewhere in the CTA ends the
            // epilogue's layers too (decided by all its threads together)
            const bool go = !flow || epi_all(!*(volatile int*)&fail);
            for (; go && W.next(Jp, I); ++it) {
                const ChainJob& Jb = *Jp;
                const int tiles = Jb.tiles, split = Jb.split, nk = Jb.nk;
                const int P = split > Jb.rep ? split : Jb.rep;
                const int R = 128 / P;
                if (Jp != Jlast) {
                    if (Jb.a.mode == 1 && Jb.a.row_part) {
                        // z of this job's fused row reductions (the previous job's
                        // reductions are done once every epilogue thread is here)
                        asm volatile("bar.sync 1, 128;" ::: "memory");
                        if (et < Jb.a.r) s_z[et] = Jb.a.zvec[et];
                        asm volatile("bar.sync 1, 128;" ::: "memory");
                    }
                    Jlast = Jp;
                }
                if (Jb.a.mode != 1) {
                    // this slice's epilogue inputs into L2 while the MMAs run (one row of T
                    // per thread: a single thread issuing them all held the whole epilogue
                    // back when the MMAs were already done)
                    const int n0 = I.tl * 128 + I.ks * R;
                    const int n1 = min(n0 + R, Jb.a.n_out);
                    const int n_out = Jb.a.n_out;
                    if (Jb.a.mode == 2 && n0 < n1) {
                        if (et < Jb.a.r)
                            for (int nn = n0; nn < n1; nn += 32)
                                prefetch_line_l2(Jb.a.T + (size_t)et * n_out + nn);
                        else if (et == Jb.a.r)
                            prefetch_line_l2(Jb.a.S1 + n0);
                    } else if (Jb.a.mode == 0 && n0 < n1 && et == 0) {
                        prefetch_line_l2(Jb.a.bias + n0);
                    }
                }
                const uint32_t ab = it & 1;
                const bool ok = mbar_wait(&tfull[ab], (it >> 1) & 1);
                tc_fence_after();
                bool wok = epi_all(ok);
                if (wok) {
                    // up to three 16-column loads in flight before each wait
                    constexpr int LB = NC < 3 ? NC : 3;
#pragma unroll
                    for (int c0 = 0; c0 < NC; c0 += LB) {
                        float v[LB][16];
#pragma unroll
                        for (int u = 0; u < LB; ++u)
                            if (c0 + u < NC)
                                tmem_ld16(tmem + ab * ACC_COLS + ((uint32_t)lane_base << 16) + 16 * (c0 + u), v[u]);
                        tmem_wait_ld();
#pragma unroll
                        for (int u = 0; u < LB; ++u)
                            if (c0 + u < NC)
#pragma unroll
                                for (int i = 0; i < 16; ++i) vrow[16 * (c0 + u) + i] = v[u][i];
                    }
                } else {
                    fail = 1;
                }
                tc_fence_before();
                mbar_arrive(&tempty[ab]);      // this accumulator may be overwritten
                if (!wok) break;
                if (Jb.raw) {
                    // store the item unfinished: k_out_finish sums each tile's items in
                    // CTA order and finishes the tile (slot: this CTA's tiles in order)
                    fence_proxy_async_smem();
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    if (et == 0) {
                        const long long Tt = (long long)tiles * nk;
                        const int ft = (int)((Tt * blockIdx.x / G) / nk);
                        float* dst = Jb.raw_part +
                                     ((size_t)blockIdx.x * Jb.raw_m + (size_t)(I.tl - ft)) * (TILE_BYTES / 4);
                        bulk_store_wait(dst, tile, TILE_BYTES);
                    }
                    asm volatile("bar.sync 1, 128;" ::: "memory");   // the tile is reused next item
                    continue;
                }
                if (Jb.a.mode == 1) {
                    // output layer (one row per thread, fused row reductions)
                    if (I.tl < Jb.a.gram_tiles && et < 4 * Jb.a.r) {
                        // the Gram rows' reductions read this tile's rows of the input
                        // activations X (i1 columns): into L2 now, while the pieces settle
                        // (the operand stream has evicted them)
                        const int j = et >> 2, ln = et & 3;
                        prefetch_line_l2(Jb.a.Xg + (size_t)(kShared + 3 * j) * Jb.a.ldxg +
                                         (size_t)I.tl * 128 + 32 * ln);
                    }
                    if (Jb.stream && (I.kb0 > 0 || I.kb1 < nk)) {
                        // a tile cut between CTAs: publish this piece; the last of the
                        // tile's CTAs sums the pieces in CTA order and finishes the tile
                        const long long Tt = (long long)tiles * nk;
                        const int cf = stream_cta((long long)I.tl * nk, Tt, G);
                        const int cl = stream_cta((long long)(I.tl + 1) * nk - 1, Tt, G);
                        auto slot_of = [&](int cc) {
                            return (int)((Tt * cc / G) / nk) == I.tl ? 0 : 1;
                        };
                        fence_proxy_async_smem();
                        asm volatile("bar.sync 1, 128;" ::: "memory");
                        if (et == 0) {
                            float* dst = split_part + ((size_t)blockIdx.x * 2 + slot_of(blockIdx.x)) * (TILE_BYTES / 4);
                            bulk_store_wait(dst, tile, TILE_BYTES);
                            fence_proxy_async_global();
                            __threadfence();
                            unsigned* cnt = split_cnt + Jb.cnt_off + I.tl;
                            const unsigned old = atomicAdd(cnt, 1u);
                            s_last = (old + 1 == (unsigned)(cl - cf + 1));
                            if (s_last) *cnt = 0u;
                            __threadfence();
                        }
                        asm volatile("bar.sync 1, 128;" ::: "memory");
                        if (!s_last) continue;
                        float4* own4 = reinterpret_cast<float4*>(tile);
                        constexpr int NE = (int)(TILE_BYTES / 16);
                        // the partners' pieces into L2 first: every line's miss in flight at
                        // once instead of eight loads per thread at a time
                        for (int cc = cf; cc <= cl; ++cc) {
                            if (cc == (int)blockIdx.x) continue;
                            const char* src = reinterpret_cast<const char*>(
                                split_part + ((size_t)cc * 2 + slot_of(cc)) * (TILE_BYTES / 4));
                            for (uint32_t b = (uint32_t)et * 128u; b < TILE_BYTES; b += 128u * 128u)
                                prefetch_line_l2(src + b);
                        }
                        for (int e0 = et; e0 < NE; e0 += 128 * 8) {
                            // eight float4 of up to three pieces in flight at once (the
                            // loads of the pieces do not wait for one another), summed in
                            // CTA order
                            float4 acc[8];
                            for (int c0 = cf; c0 <= cl; c0 += 3) {
                                float4 v[3][8];
#pragma unroll
                                for (int pc = 0; pc < 3; ++pc) {
                                    const int cc = c0 + pc;
                                    const float4* src = reinterpret_cast<const float4*>(
                                        split_part + ((size_t)cc * 2 + slot_of(cc)) * (TILE_BYTES / 4));
#pragma unroll
                                    for (int u = 0; u < 8; ++u) {
                                        const int e = e0 + u * 128;
                                        v[pc][u] = make_float4(0.f, 0.f, 0.f, 0.f);
                                        if (cc <= cl && e < NE)
                                            v[pc][u] = (cc == (int)blockIdx.x) ? own4[e] : __ldcg(src + e);
                                    }
                                }
#pragma unroll
                                for (int pc = 0; pc < 3; ++pc) {
                                    if (c0 + pc > cl) break;
#pragma unroll
                                    for (int u = 0; u < 8; ++u) {
                                        if (c0 + pc == cf) {
                                            acc[u] = v[pc][u];
                                        } else {
                                            acc[u].x += v[pc][u].x; acc[u].y += v[pc][u].y;
                                            acc[u].z += v[pc][u].z; acc[u].w += v[pc][u].w;
                                        }
                                    }
                                }
                            }
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (e0 + u * 128 < NE) own4[e0 + u * 128] = acc[u];
                        }
                        asm volatile("bar.sync 1, 128;" ::: "memory");
                    }
                    if (I.tl < Jb.a.gram_tiles) {
                        // Gram rows: reductions over K (and G x_y)
                        gram_row_reduce(Jb.a, tile, TS, row, I.tl * 128 + row, true, I.tl, s_z);
                    } else if (Jb.a.row_map) {
                        // output rows of the cubature DOFs
                        const int i = (I.tl - Jb.a.gram_tiles) * 128 + row;
                        const int n = i < Jb.a.n_map ? Jb.a.row_map[i] : -1;
                        if (Jb.a.Jc) {
                            if (n >= 0) compact_epilogue(Jb.a, i, n, vrow);
                        } else {
                            row_epilogue(Jb.a, n < 0 ? Jb.a.n_out : n, vrow);
                        }
                    } else {
                        row_epilogue(Jb.a, I.tl * 128 + row, vrow);
                        if (Jb.a.row_part)
                            fused_row_reduce(Jb.a, tile, TS, row, I.tl * 128 + row, true, I.tl, s_z);
                    }
                    continue;
                }
                if (split > 1) {
                    // publish this K chunk's partial tile, wait for the tile's other
                    // chunks, then sum rows [ks R, ks R + R) of all chunks in order
                    fence_proxy_async_smem();
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    unsigned* cnt = split_cnt + Jb.cnt_off + I.tl;
                    bool got = true;
                    if (et == 0) {
                        // the partners' slices of this chunk's partial tile (this chunk's own
                        // slice stays here), then a release on the tile's counter
                        float* dst = split_part + ((size_t)I.tl * split + I.ks) * (TILE_BYTES / 4);
                        const uint32_t sf = (uint32_t)R * TS;
                        for (int c = 0; c < split; ++c)
                            if (c != I.ks)
                                asm volatile("cp.async.bulk.global.shared::cta.bulk_group [%0], [%1], %2;" ::"l"(
                                                 dst + (size_t)c * sf),
                                             "r"(smem_u32(tile + (size_t)c * sf)), "r"(sf * 4u)
                                             : "memory");
                        asm volatile("cp.async.bulk.commit_group;" ::: "memory");
                        asm volatile("cp.async.bulk.wait_group 0;" ::: "memory");
                        fence_proxy_async_global();
                        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(cnt) : "memory");
                        const uint64_t t0 = globaltimer();
                        while (ld_acquire(cnt) != (unsigned)split) {
                            if (globaltimer() - t0 > kWaitNs) { got = false; break; }
                        }
                        // the partners' slices are read by the bulk loads below (async proxy)
                        fence_proxy_async_global();
                    }
                    // chunk s's rows [r0, r0 + R) into this tile's rows [s R, s R + R): the
                    // tile is published, its own rows stay in place, and the split * R = 128
                    // rows hold all chunks (the stage ring stays free for the next layer)
                    const int r0 = I.ks * R;
                    const uint32_t slice_f = (uint32_t)R * TS;   // floats of one chunk's slice
                    const float* src = split_part + (size_t)I.tl * split * (TILE_BYTES / 4) + (size_t)r0 * TS;
                    if (et == 0 && got) {
                        mbar_expect_tx(&rbar, (uint32_t)(split - 1) * slice_f * 4u);
                        for (int s = 0; s < split; ++s) {
                            if (s == I.ks) continue;
                            bulk_load(tile + (size_t)s * slice_f, src + (size_t)s * (TILE_BYTES / 4),
                                      slice_f * 4u, &rbar);
                        }
                    }
                    wok = epi_all(got || et != 0);
                    if (!wok) { fail = 1; break; }
                    wok = epi_all(mbar_wait(&rbar, nred & 1));
                    ++nred;
                    if (!wok) { fail = 1; break; }
                    // sum in chunk order (bitwise reproducible), four floats at a time (a
                    // slice is R x TS floats, R a multiple of 4: 16-byte aligned)
                    float4* own4 = reinterpret_cast<float4*>(tile + (size_t)r0 * TS);
                    const float4* t4 = reinterpret_cast<const float4*>(tile);
                    const int n4 = (int)slice_f / 4;
                    for (int e = et; e < n4; e += 128) {
                        float4 v[8];
#pragma unroll
                        for (int c = 0; c < 8; ++c)
                            if (c < split) v[c] = t4[(size_t)c * n4 + e];
                        float4 a = v[0];
#pragma unroll
                        for (int c = 1; c < 8; ++c)
                            if (c < split) { a.x += v[c].x; a.y += v[c].y; a.z += v[c].z; a.w += v[c].w; }
                        own4[e] = a;
                    }
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");
                slice_epilogue<PREC>(Jb.a, tile, TS, I.tl, I.ks * R, R, et);
                if (flow) {
                    // this CTA's rows of the tile are written: count it on the tile's ready
                    // counter (the stores fenced for the consumers' TMA, then a release)
                    fence_proxy_async_global();
                    asm volatile("bar.sync 1, 128;" ::: "memory");
                    if (et == 0)
                        asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(split_cnt + Jb.rdy_off + I.tl * kRdyStride)
                                     : "memory");
                }
                asm volatile("bar.sync 1, 128;" ::: "memory");   // the tile is reused next item
            }
            fence_proxy_async_global();       // epilogue stores feed the next layer's TMA
        }
        if (flow && st + 1 < n_st) continue;   // each role goes on with the next layer
        __syncthreads();
        if (threadIdx.x == 0 && !grid_barrier(gb, G, gen)) fail = 1;
        __syncthreads();
        if (fail) break;
    }
    if (flow) {
        // every CTA is past every wait (the grid barrier after the last layer): zero the
        // split and ready counters of all layers for the next launch
        __syncthreads();
        if (!fail && blockIdx.x == 0)
            for (int j = 0; j < n_jobs; ++j) {
                const ChainJob& Pb = jobs[j];
                if (Pb.stream) continue;   // the output stage: no split or ready counters
                for (int t = threadIdx.x; t < Pb.tiles; t += blockDim.x) {
                    if (Pb.split > 1) split_cnt[Pb.cnt_off + t] = 0u;
                    split_cnt[Pb.rdy_off + t * kRdyStride] = 0u;
                }
            }
    } else if (!fail && n_jobs > 0 && blockIdx.x == 0 && threadIdx.x == 0) {
        const ChainJob& Pb = jobs[n_jobs - 1];
        if (Pb.split > 1)
            for (int t = 0; t < Pb.tiles; ++t) split_cnt[Pb.cnt_off + t] = 0u;
    }
    // drain: nothing in flight may outlive the CTA
    if (warp == 0 && lane == 0) {
        const uint32_t end = pk;
        for (uint32_t k = (end > (uint32_t)stages ? end - stages : 0); k < end; ++k)
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
    // dynamic shared memory <= 220 KB: with the static part (barriers, z, the grouped
    // stage's job table, < 3 KB) within the 227 KB a CTA may hold
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
                              c.split_part, c.split_cnt, stages, c.stage_off, c.n_stages) == cudaSuccess;
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

// The output stage's raw items finished.  Block (t, b) takes rows [32 b, 32 b + 32) of
// tile t: it sums the items of the tile's CTAs cf..cl in CTA order (bitwise
// reproducible), then a G tile's rows give the reductions over their 32 rows (one
// partial row per block) and G x_y, a cubature tile's rows their u and J.
__global__ void __launch_bounds__(128) k_out_finish(const ChainJob* __restrict__ pj,
                                                    const float* __restrict__ part, int G,
                                                    const NewtonState* ns) {
    if (ns && ns->done) return;
    extern __shared__ __align__(16) float fsm[];
    __shared__ float s_z[kMaxR];
    const ChainJob& J = *pj;
    const FwdArgs& A = J.a;
    const int t = blockIdx.x, b = blockIdx.y, et = threadIdx.x;
    const int TS = A.Cp + 1, nk = J.nk;
    const long long T = (long long)J.tiles * nk;
    const int cf = stream_cta((long long)t * nk, T, G);
    const int cl = stream_cta((long long)(t + 1) * nk - 1, T, G);
    const size_t tile_f = (size_t)128 * TS;
    const int NE4 = kFinishRows * TS / 4;   // float4 of this block's rows (TS * 32 / 4)
    float4* tile4 = reinterpret_cast<float4*>(fsm);
    constexpr int EB = 8;                   // float4 loads in flight per thread and item
    for (int e0 = et; e0 < NE4; e0 += 128 * EB) {
        float4 acc[EB];
        for (int c = cf; c <= cl; ++c) {
            const int ft = (int)((T * c / G) / nk);
            const float4* src = reinterpret_cast<const float4*>(
                                    part + ((size_t)c * J.raw_m + (size_t)(t - ft)) * tile_f) +
                                (size_t)b * NE4;
            float4 v[EB];
#pragma unroll
            for (int u = 0; u < EB; ++u) {
                const int e = e0 + u * 128;
                v[u] = e < NE4 ? __ldcg(src + e) : make_float4(0.f, 0.f, 0.f, 0.f);
            }
#pragma unroll
            for (int u = 0; u < EB; ++u) {
                if (c == cf) {
                    acc[u] = v[u];
                } else {
                    acc[u].x += v[u].x; acc[u].y += v[u].y; acc[u].z += v[u].z; acc[u].w += v[u].w;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < EB; ++u)
            if (e0 + u * 128 < NE4) tile4[e0 + u * 128] = acc[u];
    }
    if (t < A.gram_tiles && et < A.r) s_z[et] = A.zvec[et];
    __syncthreads();
    const int row = et;
    if (t < A.gram_tiles) {
        gram_row_reduce<kFinishRows>(A, fsm, TS, row, t * 128 + b * kFinishRows + row, true,
                                     t * kFinishBlocks + b, s_z);
    } else if (row < kFinishRows) {
        const int i = (t - A.gram_tiles) * 128 + b * kFinishRows + row;
        const int n = i < A.n_map ? A.row_map[i] : -1;
        const float* vrow = fsm + (size_t)row * TS;
        if (A.Jc) {
            if (n >= 0) compact_epilogue(A, i, n, vrow);
        } else {
            row_epilogue(A, n < 0 ? A.n_out : n, vrow);
        }
    }
}

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

void launch_out_finish(cudaStream_t s, const ChainJob* d_job, int tiles, int Cp, const float* part,
                       int grid, const NewtonState* ns) {
    // the block's rows (Cp + 1 floats each) and their weights and scalars
    const size_t smem = ((size_t)kFinishRows * (Cp + 1) + 2 * kFinishRows) * sizeof(float);
    k_out_finish<<<dim3(tiles, kFinishBlocks), 128, smem, s>>>(d_job, part, grid, ns);
}

bool launch_chain(cudaStream_t s, const ChainLaunch& c, dae_prec prec) {
    switch (prec) {
        case DAE_TF32: return launch_chain_prec<DAE_TF32>(s, c);
        case DAE_BF16: return launch_chain_prec<DAE_BF16>(s, c);
        case DAE_BF16X3: return launch_chain_prec<DAE_BF16X3>(s, c);
        default: return false;
    }
}

// Items of a layer: P = max(split, rep) CTAs per 128-row tile with tiles x P <= grid
// and P a power of two <= 8 (each finishes 128/P rows).  K loops of at most 8
// k-blocks are replicated (the weights are a few hundred KB, read from L2 by each
// copy); longer ones are split, at least 4 k-blocks per chunk.
#ifndef DAE_REP_MAX_NK
#define DAE_REP_MAX_NK 8
#endif
void chain_plan(ChainJob& job, int grid) {
    job.split = 1;
    job.rep = 1;
    int pmax = 1;
    while (pmax * 2 <= 8 && job.tiles * pmax * 2 <= grid) pmax *= 2;
    if (job.nk <= DAE_REP_MAX_NK) {
        job.rep = pmax;
    } else {
        int s = 1;
        while (s * 2 <= pmax && job.nk / (s * 2) >= 4) s *= 2;
        job.split = s;
    }
}

}  // namespace dae
