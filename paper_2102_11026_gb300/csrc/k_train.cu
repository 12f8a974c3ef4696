// Kernels of the decoder training pass: a batched first-order forward of
// u = D(q) and J = dD/dq and its reverse sweep (gradients w.r.t. the latents,
// weights and biases), the backpropagation the paper trains its autoencoder with
// (Sec. 4.4, Sec. 5).
//
// A batch of B latents carries C = B (1 + r) columns, ordered component-major:
// column c = comp * B + s is the value (comp 0) or the tangent along e_j
// (comp 1 + j) of sample s.  Every layer then is a dense real GEMM over all columns:
//   forward      Z_l   = W_l X_{l-1}   (+ b_l on the value columns)
//   reverse      X̄_l-1 = W_l^T Z̄_l
//   weights      W̄_l   = Z̄_l X_{l-1}^T  (contraction over the C columns)
// k_gemm_x3 runs them on the tensor cores in split BF16x3 (hi*hi + hi*lo + lo*hi
// into one FP32 TMEM accumulator).  The elementwise kernels apply the activation
// and its reverse and write each operand in the two layouts the GEMMs read:
// column-major planes [c][k] (K = neurons contiguous) and neuron-major rows
// [k][c] (K = columns contiguous).
#include <algorithm>
#include "tc_common.cuh"
#include "train_internal.h"

namespace dae {

using namespace tc;

namespace {

constexpr int kGThreads = 192;
constexpr int kGStages = 3;
constexpr uint32_t kOpBytes = 128 * 128;        // one 128-row x 64-element BF16 tile
constexpr uint32_t kGStage = 4 * kOpBytes;      // A hi, A lo, B hi, B lo
constexpr uint32_t kGTmemCols = 128;
constexpr int kTS = 129;                        // staged tile row stride (floats)

// D[M][N] = A[M][K] B[N][K]^T, one 128 x 128 tile per CTA.  Warp 0: TMA producer;
// warp 1: TMEM owner + MMA issuer; warps 2-5: epilogue (TMEM -> shared tile ->
// coalesced global stores).  Every wait is bounded (2 s); a wait that gives up
// records DAE_ERR_TIMEOUT, drains the copies in flight, frees TMEM and returns.
__global__ void __launch_bounds__(kGThreads, 1) k_gemm_x3(const __grid_constant__ GemmArgs G) {
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[kGStages], empty[kGStages], tfull;
    __shared__ uint32_t tmem_base;
    __shared__ int fail;
    uint8_t* smem = reinterpret_cast<uint8_t*>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) &
                                               ~(uintptr_t)1023);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int m0 = blockIdx.x * 128, n0 = blockIdx.y * 128;
    constexpr uint32_t ID = idesc(1u, 128, 128);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kGStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        mbar_init(&tfull, 1);
        fail = 0;
        fence_barrier_init();
    }
    if (warp == 1) {
        tmem_alloc(&tmem_base, kGTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_base;
    const int nk = G.nk;
    int issued = 0;
    if (warp == 0) {
        if (lane == 0) {
            for (int kb = 0; kb < nk; ++kb) {
                const int s = kb % kGStages;
                const uint32_t ph = (kb / kGStages) & 1;
                if (!mbar_wait(&empty[s], ph ^ 1)) { fail = 1; break; }
                mbar_expect_tx(&full[s], kGStage);
                uint8_t* base = smem + (size_t)s * kGStage;
                tma_load_2d(base, &G.tm[0], &full[s], kb * 64, m0);
                tma_load_2d(base + kOpBytes, &G.tm[1], &full[s], kb * 64, m0);
                tma_load_2d(base + 2 * kOpBytes, &G.tm[2], &full[s], kb * 64, n0);
                tma_load_2d(base + 3 * kOpBytes, &G.tm[3], &full[s], kb * 64, n0);
                ++issued;
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            for (int kb = 0; kb < nk && !fail; ++kb) {
                const int s = kb % kGStages;
                const uint32_t ph = (kb / kGStages) & 1;
                if (!mbar_wait(&full[s], ph)) { fail = 1; break; }
                tc_fence_after();
                const uint32_t base = smem_u32(smem + (size_t)s * kGStage);
                const uint64_t dah = sdesc(base), dal = sdesc(base + kOpBytes);
                const uint64_t dbh = sdesc(base + 2 * kOpBytes), dbl = sdesc(base + 3 * kOpBytes);
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    mma<DAE_BF16X3>(tmem, dah + 2 * k, dbh + 2 * k, ID, (kb > 0 || k > 0) ? 1u : 0u);
                    mma<DAE_BF16X3>(tmem, dah + 2 * k, dbl + 2 * k, ID, 1u);
                    mma<DAE_BF16X3>(tmem, dal + 2 * k, dbh + 2 * k, ID, 1u);
                }
                mma_commit(&empty[s]);
            }
            mma_commit(&tfull);
        }
    } else {
        const int et = threadIdx.x - 64;
        const int lane_base = 32 * (warp & 3);
        const int row = lane_base + lane;
        const bool ok = mbar_wait(&tfull, 0);
        tc_fence_after();
        const bool wok = epi_all(ok);
        // every MMA has completed: the stage buffers are idle and hold the staged tile
        float* tile = reinterpret_cast<float*>(smem);
        if (wok) {
#pragma unroll
            for (int c = 0; c < 8; ++c) {
                float v[16];
                tmem_ld16(tmem + ((uint32_t)lane_base << 16) + 16 * c, v);
                tmem_wait_ld();
#pragma unroll
                for (int i = 0; i < 16; ++i) tile[row * kTS + 16 * c + i] = v[i];
            }
        } else {
            fail = 1;
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (wok) {
            float* __restrict__ out = G.out;
            const size_t ldo = G.ldo;
            if (G.out_mode == 1) {
                // out[n][m]: a warp stores 32 consecutive m of one column n
                const int m = m0 + et;
                const float bv = (G.bias && m < G.M) ? G.bias[m] : 0.f;
                if (m < G.M) {
                    for (int j = 0; j < 128; ++j) {
                        const int n = n0 + j;
                        if (n >= G.N) break;
                        out[(size_t)n * ldo + m] = tile[et * kTS + j] + (n < G.bias_cols ? bv : 0.f);
                    }
                }
            } else {
                // out[m][n]: a warp stores 32 consecutive n of one row m
                const int n = n0 + et;
                if (n < G.N) {
                    for (int i = 0; i < 128; ++i) {
                        const int m = m0 + i;
                        if (m >= G.M) break;
                        out[(size_t)m * ldo + n] = tile[i * kTS + et];
                    }
                }
            }
        }
    }
    // drain: no copy may outlive the CTA
    if (warp == 0 && lane == 0) {
        for (int kb = (issued > kGStages ? issued - kGStages : 0); kb < issued; ++kb)
            if (!mbar_wait(&full[kb % kGStages], (kb / kGStages) & 1)) fail = 1;
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, kGTmemCols);
    }
    if (threadIdx.x == 0 && fail && G.status) atomicCAS(G.status, 0, (int)DAE_ERR_TIMEOUT);
}

__device__ __forceinline__ void split_store(float v, __nv_bfloat16* hi, __nv_bfloat16* lo, size_t i) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    hi[i] = h;
    lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
}

// One element of an operand: FP32 (FP32 form) or split BF16 hi / lo.
__device__ __forceinline__ void op_store_c(const Operand& P, size_t i, float v) {
    if (P.cf) P.cf[i] = v; else split_store(v, P.ch, P.cl, i);
}
__device__ __forceinline__ void op_store_n(const Operand& P, size_t i, float v) {
    if (P.nf) P.nf[i] = v; else split_store(v, P.nh, P.nl, i);
}

// Writes a 32 (k) x 32 (s) tile of comp's columns in both layouts: planes [c][k]
// (ldc) and rows [k][c] (ldn), through a shared transpose so both stores coalesce.
// v[ty][tx] holds neuron k0 + tx, sample s0 + ty.
__device__ __forceinline__ void store_both(const float (*v)[33], int k0, int s0, int comp, int B,
                                           int n, int nb, const Operand& P) {
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8 threads
    for (int yy = ty; yy < 32; yy += 8) {
        const int s = s0 + yy, k = k0 + tx;
        if (s < nb && k < n) op_store_c(P, (size_t)(comp * B + s) * P.ldc + k, v[yy][tx]);
    }
    for (int yy = ty; yy < 32; yy += 8) {
        const int k = k0 + yy, s = s0 + tx;
        if (s < nb && k < n) op_store_n(P, (size_t)k * P.ldn + comp * B + s, v[tx][yy]);
    }
}

}  // namespace

// ------------------------------------------------------------------ seed --
// X_0 for a batch: value columns q_s (FP64 rounded once), tangent columns e_j.
__global__ void k_train_seed(const double* q, int B, int r, Operand X) {
    const int c = blockIdx.x, k = threadIdx.x;
    if (k >= r || c >= B * (1 + r)) return;
    const int comp = c / B, s = c % B;
    const float v = comp == 0 ? (float)q[(size_t)s * r + k] : (comp - 1 == k ? 1.f : 0.f);
    op_store_c(X, (size_t)c * X.ldc + k, v);
    op_store_n(X, (size_t)k * X.ldn + c, v);
}

// ------------------------------------------------------------ activation --
// X = act(Z) in first-order dual arithmetic: value act(z), tangents act'(z) z_j.
// Grid (ceil(n/32), ceil(B/32)), 256 threads; Z planes [c][k] (ldz).
__global__ void __launch_bounds__(256) k_train_act(const float* Z, int ldz, int n, int B, int r,
                                                   int act, Operand X) {
    __shared__ float v[32][33], s1v[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int k0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    for (int yy = ty; yy < 32; yy += 8) {
        const int s = s0 + yy, k = k0 + tx;
        float val = 0.f, d1 = 0.f;
        if (s < B && k < n) {
            const ActD D = act_d(act, Z[(size_t)s * ldz + k]);
            val = D.s0;
            d1 = D.s1;
        }
        v[yy][tx] = val;
        s1v[yy][tx] = d1;
    }
    __syncthreads();
    store_both(v, k0, s0, 0, B, n, B, X);
    for (int j = 0; j < r; ++j) {
        __syncthreads();
        for (int yy = ty; yy < 32; yy += 8) {
            const int s = s0 + yy, k = k0 + tx;
            v[yy][tx] = (s < B && k < n) ? s1v[yy][tx] * Z[(size_t)((1 + j) * B + s) * ldz + k] : 0.f;
        }
        __syncthreads();
        store_both(v, k0, s0, 1 + j, B, n, B, X);
    }
}

// Reverse of the activation: from X̄ (planes, ldx) and Z (planes, ldz)
//   Z̄ value = act'(z) x̄ + act''(z) sum_j z_j x̄_j,   Z̄_j = act'(z) x̄_j;
// writes Z̄ in both layouts and its value rows in FP32 (bias gradient, latent gradient).
__global__ void __launch_bounds__(256) k_train_act_bwd(const float* Xb, int ldx, const float* Z, int ldz,
                                                       int n, int B, int r, int act, Operand Zb,
                                                       float* zb_val) {
    __shared__ float v[32][33], s1v[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int k0 = blockIdx.x * 32, s0 = blockIdx.y * 32;
    float acc[4];
    for (int i = 0; i < 4; ++i) acc[i] = 0.f;
    for (int yy = ty, i = 0; yy < 32; yy += 8, ++i) {
        const int s = s0 + yy, k = k0 + tx;
        float d1 = 0.f, d2 = 0.f, xv = 0.f;
        if (s < B && k < n) {
            const ActD D = act_d(act, Z[(size_t)s * ldz + k]);
            d1 = D.s1;
            d2 = D.s2;
            xv = Xb[(size_t)s * ldx + k];
            float t = 0.f;
            for (int j = 0; j < r; ++j) {
                const size_t cj = (size_t)((1 + j) * B + s);
                t = fmaf(Z[cj * ldz + k], Xb[cj * ldx + k], t);
            }
            acc[i] = fmaf(d1, xv, d2 * t);
            zb_val[(size_t)s * n + k] = acc[i];
        }
        s1v[yy][tx] = d1;
        v[yy][tx] = acc[i];
    }
    __syncthreads();
    store_both(v, k0, s0, 0, B, n, B, Zb);
    for (int j = 0; j < r; ++j) {
        __syncthreads();
        for (int yy = ty; yy < 32; yy += 8) {
            const int s = s0 + yy, k = k0 + tx;
            v[yy][tx] = (s < B && k < n) ? s1v[yy][tx] * Xb[(size_t)((1 + j) * B + s) * ldx + k] : 0.f;
        }
        __syncthreads();
        store_both(v, k0, s0, 1 + j, B, n, B, Zb);
    }
}

// The output layer's cotangents [c][n] (FP32, the caller's layout) in both operand
// layouts.  Grid (ceil(n/32), ceil(B/32), 1 + r).
__global__ void __launch_bounds__(256) k_train_split(const float* g, int n, int B, Operand Zb) {
    __shared__ float v[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int k0 = blockIdx.x * 32, s0 = blockIdx.y * 32, comp = blockIdx.z;
    for (int yy = ty; yy < 32; yy += 8) {
        const int s = s0 + yy, k = k0 + tx;
        v[yy][tx] = (s < B && k < n) ? g[(size_t)(comp * B + s) * n + k] : 0.f;
    }
    __syncthreads();
    store_both(v, k0, s0, comp, B, n, B, Zb);
}

// Bias gradient: g_b[k] = sum_s Z̄_value[s][k] (fixed order).
__global__ void k_train_bias_grad(const float* zb_val, int ld, int n, int B, float* gb) {
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= n) return;
    float acc = 0.f;
    for (int s = 0; s < B; ++s) acc += zb_val[(size_t)s * ld + k];
    gb[k] = acc;
}

// Latent gradient: g_q[s][j] = sum_k Z̄_1 value[s][k] W_1[k][j] (FP32 sums, FP64 out).
__global__ void k_train_grad_q(const float* zb_val, int n1, const float* W1, int ldw, int B, int r,
                               double* gq) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= B * r) return;
    const int s = i / r, j = i % r;
    float acc = 0.f;
    for (int k = 0; k < n1; ++k) acc = fmaf(zb_val[(size_t)s * n1 + k], W1[(size_t)k * ldw + j], acc);
    gq[i] = acc;
}

// Padded BF16 hi/lo copies of W ([m_pad][ld], zero padding) and of W^T ([n_pad][ldT]).
__global__ void k_train_weights(const float* W, int n_out, int n_in, __nv_bfloat16* h,
                                __nv_bfloat16* l, int ld, __nv_bfloat16* th, __nv_bfloat16* tl,
                                int ldT) {
    __shared__ float t[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;   // rows i (out), columns k (in)
    for (int yy = ty; yy < 32; yy += 8) {
        const int i = i0 + yy, k = k0 + tx;
        const float v = (i < n_out && k < n_in) ? W[(size_t)i * n_in + k] : 0.f;
        t[yy][tx] = v;
        if (i < n_out && k < n_in) split_store(v, h, l, (size_t)i * ld + k);
    }
    if (th == nullptr) return;   // uniform: no transposed copy wanted
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int k = k0 + yy, i = i0 + tx;
        if (i < n_out && k < n_in) split_store(t[tx][yy], th, tl, (size_t)k * ldT + i);
    }
}

// ------------------------------------------------------------ FP32 form --
// D[M][N] = A[M][K] B[N][K]^T in FP32 on the CUDA cores: a 64 x 64 output tile per CTA,
// 256 threads with 4 x 4 outputs each, K in blocks of 32 staged through shared memory
// as [k][row] (row stride 65: the stores of a warp hit distinct banks).  Rows up to the
// tile edge and K up to nk x 64 lie inside the padded operands (zero padding).
__global__ void __launch_bounds__(256) k_gemm_f32(const GemmArgs G) {
    __shared__ float As[32][65], Bs[32][65];
    const int t = threadIdx.x;
    const int m0 = blockIdx.x * 64, n0 = blockIdx.y * 64;
    const int tm = t >> 4, tn = t & 15;
    float acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = 0.f;
    const int K = G.nk * 64;
    for (int k0 = 0; k0 < K; k0 += 32) {
        for (int e = t; e < 64 * 32; e += 256) {
            const int row = e >> 5, kk = e & 31;
            As[kk][row] = G.a32[(size_t)(m0 + row) * G.lda + k0 + kk];
            Bs[kk][row] = G.b32[(size_t)(n0 + row) * G.ldb + k0 + kk];
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < 32; ++kk) {
            float a[4], b[4];
#pragma unroll
            for (int i = 0; i < 4; ++i) { a[i] = As[kk][tm + 16 * i]; b[i] = Bs[kk][tn + 16 * i]; }
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], b[j], acc[i][j]);
        }
        __syncthreads();
    }
    float* __restrict__ out = G.out;
    const size_t ldo = G.ldo;
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        const int m = m0 + tm + 16 * i;
        if (m >= G.M) continue;
        const float bv = (G.bias && G.out_mode == 1) ? G.bias[m] : 0.f;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const int n = n0 + tn + 16 * j;
            if (n >= G.N) continue;
            if (G.out_mode == 1) out[(size_t)n * ldo + m] = acc[i][j] + (n < G.bias_cols ? bv : 0.f);
            else out[(size_t)m * ldo + n] = acc[i][j];
        }
    }
}

// Padded FP32 copies of W ([m_pad][ld]) and of W^T ([n_pad][ldT]); the padding stays
// zero from the allocation.
__global__ void k_train_weights_f32(const float* W, int n_out, int n_in, float* w, int ld, float* wt,
                                    int ldT) {
    __shared__ float tt[32][33];
    const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;
    const int i0 = blockIdx.y * 32, k0 = blockIdx.x * 32;
    for (int yy = ty; yy < 32; yy += 8) {
        const int i = i0 + yy, k = k0 + tx;
        const float v = (i < n_out && k < n_in) ? W[(size_t)i * n_in + k] : 0.f;
        tt[yy][tx] = v;
        if (i < n_out && k < n_in) w[(size_t)i * ld + k] = v;
    }
    if (wt == nullptr) return;   // uniform
    __syncthreads();
    for (int yy = ty; yy < 32; yy += 8) {
        const int k = k0 + yy, i = i0 + tx;
        if (i < n_out && k < n_in) wt[(size_t)k * ldT + i] = tt[tx][yy];
    }
}

bool launch_gemm_f32(cudaStream_t s, const GemmArgs& g) {
    k_gemm_f32<<<dim3((g.M + 63) / 64, (g.N + 63) / 64), 256, 0, s>>>(g);
    return cudaGetLastError() == cudaSuccess;
}

void launch_train_weights_f32(cudaStream_t s, const float* W, int n_out, int n_in, float* w, int ld,
                              float* wt, int ldT) {
    k_train_weights_f32<<<dim3((n_in + 31) / 32, (n_out + 31) / 32), 256, 0, s>>>(W, n_out, n_in, w, ld,
                                                                                  wt, ldT);
}

// ----------------------------------------------------------------- launches --
bool launch_gemm_x3(cudaStream_t s, const GemmArgs& g, int m_tiles, int n_tiles) {
    const size_t smem = (size_t)kGStages * kGStage + 1024;
    static bool configured = false;
    if (!configured) {
        if (cudaFuncSetAttribute(k_gemm_x3, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) !=
            cudaSuccess)
            return false;
        configured = true;
    }
    k_gemm_x3<<<dim3(m_tiles, n_tiles), kGThreads, smem, s>>>(g);
    return cudaGetLastError() == cudaSuccess;
}

void launch_train_seed(cudaStream_t s, const double* q, int B, int r, const Operand& X) {
    k_train_seed<<<B * (1 + r), 32, 0, s>>>(q, B, r, X);
}

void launch_train_act(cudaStream_t s, const float* Z, int ldz, int n, int B, int r, int act,
                      const Operand& X) {
    k_train_act<<<dim3((n + 31) / 32, (B + 31) / 32), 256, 0, s>>>(Z, ldz, n, B, r, act, X);
}

void launch_train_act_bwd(cudaStream_t s, const float* Xb, int ldx, const float* Z, int ldz, int n,
                          int B, int r, int act, const Operand& Zb, float* zb_val) {
    k_train_act_bwd<<<dim3((n + 31) / 32, (B + 31) / 32), 256, 0, s>>>(Xb, ldx, Z, ldz, n, B, r, act,
                                                                       Zb, zb_val);
}

void launch_train_split(cudaStream_t s, const float* g, int n, int B, int r, const Operand& Zb) {
    k_train_split<<<dim3((n + 31) / 32, (B + 31) / 32, 1 + r), 256, 0, s>>>(g, n, B, Zb);
}

void launch_train_bias_grad(cudaStream_t s, const float* zb_val, int ld, int n, int B, float* gb) {
    k_train_bias_grad<<<(n + 127) / 128, 128, 0, s>>>(zb_val, ld, n, B, gb);
}

void launch_train_grad_q(cudaStream_t s, const float* zb_val, int n1, const float* W1, int ldw, int B,
                         int r, double* gq) {
    k_train_grad_q<<<(B * r + 127) / 128, 128, 0, s>>>(zb_val, n1, W1, ldw, B, r, gq);
}

void launch_train_weights(cudaStream_t s, const float* W, int n_out, int n_in, __nv_bfloat16* h,
                          __nv_bfloat16* l, int ld, __nv_bfloat16* th, __nv_bfloat16* tl, int ldT) {
    k_train_weights<<<dim3((n_in + 31) / 32, (n_out + 31) / 32), 256, 0, s>>>(W, n_out, n_in, h, l, ld,
                                                                              th, tl, ldT);
}

}  // namespace dae
