// Forward pass of the stacked complex-step batch: seed columns, CUDA-core FP32
// layer GEMM with the fused multicomplex activation / output epilogue.
#include "dae_internal.h"
#include "epilogue.cuh"
#include "multicomplex.cuh"

namespace dae {

// ------------------------------------------------------------------- seed --
// Input components of q* = q + h e_j i1 + h c i2 + h c i3 + h^2 g i2i3 (Sec. 4.3),
// c = Delta (0 in SEED_HW), g = w (0 in SEED_SDD); column layout in dae_internal.h.
__device__ __forceinline__ void seed_impl(const NewtonState* ns, const double* q_override,
                                          const double* qbar, const double* qbar_dot, double dt,
                                          double h, int mode, int r, int Cp, int ld0, float* X,
                                          __nv_bfloat16* Xh, __nv_bfloat16* Xl, int out_bf16,
                                          float* zvec, int off) {
    if (ns && ns->done) return;
    const double* q = (q_override ? q_override : ns->q_trial) + off;
    const int C = n_cols(r);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < Cp * ld0;
         idx += gridDim.x * blockDim.x) {
        int c = idx / ld0, k = idx % ld0;
        double v = 0.0;
        if (k < r && c < C) {
            double D = q[k] - qbar[k];
            double w = 3.0 * D - dt * qbar_dot[k];
            if (c == 0) v = q[k];
            else if (c == 1) v = (mode == SEED_HW) ? 0.0 : h * D;
            else if (c == 2) v = (mode == SEED_SDD) ? 0.0 : h * h * w;
            else if (c >= kShared && (c - kShared) % 3 == 0) v = ((c - kShared) / 3 == k) ? h : 0.0;
        }
        store_act((float)v, X, Xh, Xl, (size_t)c * ld0 + k, out_bf16);
    }
    if (blockIdx.x == 0 && threadIdx.x < r && zvec) {
        int k = threadIdx.x;
        zvec[k] = (float)((q[k] - qbar[k]) - dt * qbar_dot[k]);
    }
}

__global__ void k_seed(const NewtonState* ns, const double* q_override, const double* qbar,
                       const double* qbar_dot, double dt, double h, int mode, int r, int Cp,
                       int ld0, float* X, __nv_bfloat16* Xh, __nv_bfloat16* Xl, int out_bf16,
                       float* zvec, int off) {
    seed_impl(ns, q_override, qbar, qbar_dot, dt, h, mode, r, Cp, ld0, X, Xh, Xl, out_bf16, zvec, off);
}

// Grouped form (z = system): the full seed at each system's trial iterate.
__global__ void k_seed_b(const SeedArgs* __restrict__ args) {
    const SeedArgs& a = args[blockIdx.z];
    seed_impl(a.ns, nullptr, a.qbar, a.qbar_dot, a.dt, a.h, SEED_FULL, a.r, a.Cp, a.ld0, a.X,
              a.Xh, a.Xl, a.out_bf16, a.zvec, a.off);
}

void launch_seed_batched(cudaStream_t s, const SeedArgs* d_args, int n_sys, int max_elems) {
    if (n_sys <= 0) return;
    const int bx = (max_elems + 255) / 256;
    k_seed_b<<<dim3(bx < 1 ? 1 : bx, 1, n_sys), 256, 0, s>>>(d_args);
}

void launch_seed(cudaStream_t s, const NewtonState* ns, const double* q_override,
                 const double* qbar, const double* qbar_dot, double dt, double h, int mode,
                 int r, int Cp, int ld0, float* X, __nv_bfloat16* Xh, __nv_bfloat16* Xl,
                 int out_bf16, float* zvec, int off) {
    int n = Cp * ld0;
    k_seed<<<(n + 255) / 256, 256, 0, s>>>(ns, q_override, qbar, qbar_dot, dt, h, mode, r, Cp,
                                          ld0, X, Xh, Xl, out_bf16, zvec, off);
}

// Exact multicomplex columns (layout at n_cols_exact): column 0 = q; the number
// q + h c (i2 + i3) in columns 1-3; per direction j the number
// q + h e_j i1 + h c (i2 + i3) + h^2 g i2i3, c = Delta (0 in SEED_HW), g = w (0 in SEED_SDD).
__global__ void k_seed_exact(const double* q, const double* qbar, const double* qbar_dot, double dt,
                             double h, int mode, int r, int Cp, int ld0, float* X) {
    const int C = n_cols_exact(r);
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < Cp * ld0; idx += gridDim.x * blockDim.x) {
        const int c = idx / ld0, k = idx % ld0;
        double v = 0.0;
        if (k < r && c < C) {
            const double D = q[k] - qbar[k];
            const double w = 3.0 * D - dt * qbar_dot[k];
            const double hc = (mode == SEED_HW) ? 0.0 : h * D;
            const double hg = (mode == SEED_SDD) ? 0.0 : h * h * w;
            if (c == 0 || c == 1) {
                v = q[k];
            } else if (c == 2) {
                v = hc;
            } else if (c >= kSharedX) {
                const int j = (c - kSharedX) / 6, comp = (c - kSharedX) % 6;
                if (comp == 0) v = q[k];
                else if (comp == 1) v = (j == k) ? h : 0.0;
                else if (comp == 2) v = hc;
                else if (comp == 4) v = hg;
            }
        }
        X[(size_t)c * ld0 + k] = (float)v;
    }
}

void launch_seed_exact(cudaStream_t s, const double* q, const double* qbar, const double* qbar_dot,
                       double dt, double h, int mode, int r, int Cp, int ld0, float* X) {
    const int n = Cp * ld0;
    k_seed_exact<<<(n + 255) / 256, 256, 0, s>>>(q, qbar, qbar_dot, dt, h, mode, r, Cp, ld0, X);
}

// Exact multicomplex epilogue of one row (hidden layer: the activation of every number
// in the row, outputs in the same layout; output layer: u, J, H[D,D] and dJ from the
// linear layer's components).
__device__ void exact_row(const FwdArgs& A, const float* v, int n, int grp) {
    using namespace mc;
    const int r = A.r;
    if (!A.last) {
        const size_t ldy = A.ldy;
        float* Y = A.Y;
        if (n >= A.n_out) {
            for (int c = grp; c < A.Cp; c += 4) Y[(size_t)c * ldy + n] = 0.f;
            return;
        }
        const float b = A.bias[n];
        if (grp == 0) {
            Y[n] = act(A.act, v[0] + b);
            // q + h c (i2 + i3): (re + i2 c) + i3 (c + i2 g)
            const C2 z{C1{v[1] + b, v[2]}, C1{v[2], v[3]}};
            const C2 o = act(A.act, z);
            Y[ldy + n] = o.x.x;
            Y[2 * ldy + n] = o.x.y;
            Y[3 * ldy + n] = o.y.y;
            for (int cc = n_cols_exact(r); cc < A.Cp; ++cc) Y[(size_t)cc * ldy + n] = 0.f;
        }
        for (int j = grp; j < r; j += 4) {
            const int cb = kSharedX + 6 * j;
            // [real, i1, i2, i1i2, i2i3, i1i2i3] with i3 = i2 and i1i3 = i1i2
            const C3 z{C2{C1{v[cb] + b, v[cb + 2]}, C1{v[cb + 2], v[cb + 4]}},
                       C2{C1{v[cb + 1], v[cb + 3]}, C1{v[cb + 3], v[cb + 5]}}};
            const C3 o = act(A.act, z);
            Y[(size_t)cb * ldy + n] = o.x.x.x;
            Y[(size_t)(cb + 1) * ldy + n] = o.y.x.x;
            Y[(size_t)(cb + 2) * ldy + n] = o.x.x.y;
            Y[(size_t)(cb + 3) * ldy + n] = o.y.x.y;
            Y[(size_t)(cb + 4) * ldy + n] = o.x.y.y;
            Y[(size_t)(cb + 5) * ldy + n] = o.y.y.y;
        }
    } else {
        if (n >= A.n_out) return;
        const size_t N = A.n_out;
        if (grp == 0) {
            if (A.u) A.u[n] = v[0] + A.bias[n];
            if (A.HDD) A.HDD[n] = (float)(v[3] * A.inv_h2);
            if (A.Hqq) A.Hqq[n] = (float)(v[3] * A.inv_h2 * A.inv_dt2);
        }
        for (int j = grp; j < r; j += 4) {
            const int cb = kSharedX + 6 * j;
            if (A.J) A.J[(size_t)j * N + n] = (float)(v[cb + 1] * A.inv_h);
            if (A.dJ) A.dJ[(size_t)j * N + n] = (float)(v[cb + 5] * A.inv_h3);
        }
    }
}

// ------------------------------------------------------- CUDA-core GEMM --
// Tile: 64 output rows x Cp component columns, K step 32, 256 threads; thread
// (ty, tx) accumulates rows 4ty..4ty+3 and columns tx + 16 i.
constexpr int SB_M = 64, SB_K = 32;

template <int NC>
struct SimtSmem {
    static constexpr int CP = 16 * NC;
    union {
        struct {
            float Ws[SB_K][SB_M + 4];
            float Xs[SB_K][CP + 4];
        } mm;
        float tile[SB_M][CP + 1];
    };
};

// Row epilogue on a tile in shared memory: thread t handles row t%64 and the
// component groups j = t/64, t/64 + 4, ...
template <int NC>
__device__ void simt_epilogue(const FwdArgs& A, float (*tile)[16 * NC + 1], int m0) {
    const int t = threadIdx.x;
    const int row = t & (SB_M - 1), grp = t >> 6;
    const int n = m0 + row;
    const int r = A.r, C = n_cols(r);
    const float* v = tile[row];
    if (A.exact) {
        exact_row(A, v, n, grp);
        return;
    }
    if (!A.last) {
        if (n >= A.ldy) return;
        const size_t ldy = A.ldy;
        if (n >= A.n_out) {   // zero padding rows of the next layer's input
            for (int c = grp; c < A.Cp; c += 4) store_act(0.f, A.Y, A.Yh, A.Yl, c * ldy + n, A.out_bf16);
            return;
        }
        ActD D = act_d(A.act, v[0] + A.bias[n]);
        const float c = v[1], gw = v[2];
        if (grp == 0) {
            float oc, ogw, og0;
            mc_shared(D, c, gw, v[3], oc, ogw, og0);
            store_act(D.s0, A.Y, A.Yh, A.Yl, 0 * ldy + n, A.out_bf16);
            store_act(oc, A.Y, A.Yh, A.Yl, 1 * ldy + n, A.out_bf16);
            store_act(ogw, A.Y, A.Yh, A.Yl, 2 * ldy + n, A.out_bf16);
            store_act(og0, A.Y, A.Yh, A.Yl, 3 * ldy + n, A.out_bf16);
            for (int cc = C; cc < A.Cp; ++cc) store_act(0.f, A.Y, A.Yh, A.Yl, cc * ldy + n, A.out_bf16);
            if (A.S1) A.S1[n] = D.s1;
        }
        for (int j = grp; j < r; j += 4) {
            const int cb = kShared + 3 * j;
            float ob, od, oh;
            mc_group(D, c, gw, v[cb], v[cb + 1], v[cb + 2], ob, od, oh);
            store_act(ob, A.Y, A.Yh, A.Yl, (size_t)cb * ldy + n, A.out_bf16);
            store_act(od, A.Y, A.Yh, A.Yl, (size_t)(cb + 1) * ldy + n, A.out_bf16);
            store_act(oh, A.Y, A.Yh, A.Yl, (size_t)(cb + 2) * ldy + n, A.out_bf16);
            if (A.T) A.T[(size_t)j * A.n_out + n] = D.s2 * v[cb];
        }
    } else {
        if (n >= A.n_out) return;
        const size_t N = A.n_out;
        if (grp == 0) {
            if (A.u) A.u[n] = v[0] + A.bias[n];
            float hdd = (float)(v[3] * A.inv_h2);
            if (A.HDD) A.HDD[n] = hdd;
            if (A.Hqq) A.Hqq[n] = (float)(v[3] * A.inv_h2 * A.inv_dt2);
        }
        for (int j = grp; j < r; j += 4) {
            const int cb = kShared + 3 * j;
            if (A.J) A.J[(size_t)j * N + n] = (float)(v[cb] * A.inv_h);
            if (A.dJ) A.dJ[(size_t)j * N + n] = (float)(v[cb + 2] * A.inv_h3);
        }
    }
}

template <int NC>
__global__ void __launch_bounds__(256) k_fwd_simt(FwdArgs A) {
    if (A.ns && A.ns->done) return;
    __shared__ SimtSmem<NC> sm;
    constexpr int CP = 16 * NC;
    const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
    const int m0 = blockIdx.x * SB_M;
    float acc[4][NC];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < NC; ++j) acc[i][j] = 0.f;
    const int K = A.ld;
    for (int k0 = 0; k0 < K; k0 += SB_K) {
        for (int i = tid; i < SB_M * (SB_K / 4); i += 256) {
            int row = i >> 3, kq = i & 7;
            float4 w = *reinterpret_cast<const float4*>(A.W + (size_t)(m0 + row) * A.ld + k0 + kq * 4);
            sm.mm.Ws[kq * 4 + 0][row] = w.x;
            sm.mm.Ws[kq * 4 + 1][row] = w.y;
            sm.mm.Ws[kq * 4 + 2][row] = w.z;
            sm.mm.Ws[kq * 4 + 3][row] = w.w;
        }
        for (int i = tid; i < CP * (SB_K / 4); i += 256) {
            int c = i >> 3, kq = i & 7;
            float4 x = *reinterpret_cast<const float4*>(A.X + (size_t)c * A.ld + k0 + kq * 4);
            sm.mm.Xs[kq * 4 + 0][c] = x.x;
            sm.mm.Xs[kq * 4 + 1][c] = x.y;
            sm.mm.Xs[kq * 4 + 2][c] = x.z;
            sm.mm.Xs[kq * 4 + 3][c] = x.w;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < SB_K; ++kk) {
            float4 w4 = *reinterpret_cast<const float4*>(&sm.mm.Ws[kk][ty * 4]);
            float wv[4] = {w4.x, w4.y, w4.z, w4.w};
            float xv[NC];
#pragma unroll
            for (int j = 0; j < NC; ++j) xv[j] = sm.mm.Xs[kk][tx + 16 * j];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < NC; ++j) acc[i][j] = fmaf(wv[i], xv[j], acc[i][j]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < NC; ++j) sm.tile[ty * 4 + i][tx + 16 * j] = acc[i][j];
    __syncthreads();
    simt_epilogue<NC>(A, sm.tile, m0);
}

void launch_fwd_simt(cudaStream_t s, const FwdArgs& a) {
    dim3 grid(a.m_pad / SB_M);
    switch (a.Cp / 16) {
        case 1: k_fwd_simt<1><<<grid, 256, 0, s>>>(a); break;
        case 2: k_fwd_simt<2><<<grid, 256, 0, s>>>(a); break;
        case 3: k_fwd_simt<3><<<grid, 256, 0, s>>>(a); break;
        case 4: k_fwd_simt<4><<<grid, 256, 0, s>>>(a); break;
        case 5: k_fwd_simt<5><<<grid, 256, 0, s>>>(a); break;
        case 6: k_fwd_simt<6><<<grid, 256, 0, s>>>(a); break;
        case 7: k_fwd_simt<7><<<grid, 256, 0, s>>>(a); break;
        default: break;
    }
}

// ------------------------------------------------------------ BF16 split --
__global__ void k_split_bf16(const float* W, __nv_bfloat16* hi, __nv_bfloat16* lo, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x) {
        float v = W[i];
        __nv_bfloat16 h = __float2bfloat16_rn(v);
        hi[i] = h;
        if (lo) lo[i] = __float2bfloat16_rn(v - __bfloat162float(h));
    }
}

void launch_split_bf16(cudaStream_t s, const float* W, __nv_bfloat16* hi, __nv_bfloat16* lo,
                       size_t n) {
    k_split_bf16<<<1024, 256, 0, s>>>(W, hi, lo, n);
}

// ------------------------------------------------------------ TF32 copy --
__global__ void k_round_tf32(const float* W, float* out, size_t n) {
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        out[i] = tf32_rna(W[i]);
}

void launch_round_tf32(cudaStream_t s, const float* W, float* out, size_t n) {
    k_round_tf32<<<1024, 256, 0, s>>>(W, out, n);
}

// ---------------------------------------------------- cubature-row gather --
__device__ __forceinline__ void gather_row_impl(const GatherArgs& A, int i) {
    if (i >= A.n_rows) return;
    int dof = -1;
    if (i < 12 * A.n_cub) {
        const int e = A.cub_tets[i / 12], a = (i % 12) / 3, d = i % 3;
        dof = 3 * A.tets[4 * e + a] + d;
    }
    // a row that already holds this DOF is current: the operand rows change only here
    // (the map reads -1 after allocation, and no DOF is negative)
    const bool current = dof >= 0 && A.map[i] == dof;
    __syncthreads();
    if (current) return;
    if (threadIdx.x == 0) A.map[i] = dof;
    const size_t dst = (size_t)(A.row0 + i) * A.ld;
    if (A.dst32) {
        const uint4* src = reinterpret_cast<const uint4*>(A.src32 + (size_t)(dof < 0 ? 0 : dof) * A.ld);
        uint4* out = reinterpret_cast<uint4*>(A.dst32 + dst);
        for (int c = threadIdx.x; c < A.ld / 4; c += blockDim.x)
            out[c] = dof < 0 ? make_uint4(0, 0, 0, 0) : src[c];
    }
    if (A.dsth) {
        const size_t so = (size_t)(dof < 0 ? 0 : dof) * A.ld;
        const uint4* sh = reinterpret_cast<const uint4*>(A.srch + so);
        uint4* oh = reinterpret_cast<uint4*>(A.dsth + dst);
        for (int c = threadIdx.x; c < A.ld / 8; c += blockDim.x)
            oh[c] = dof < 0 ? make_uint4(0, 0, 0, 0) : sh[c];
        if (A.dstl) {
            const uint4* sl = reinterpret_cast<const uint4*>(A.srcl + so);
            uint4* ol = reinterpret_cast<uint4*>(A.dstl + dst);
            for (int c = threadIdx.x; c < A.ld / 8; c += blockDim.x)
                ol[c] = dof < 0 ? make_uint4(0, 0, 0, 0) : sl[c];
        }
    }
}

__global__ void k_gather_cub_rows(GatherArgs A) { gather_row_impl(A, blockIdx.x); }

__global__ void k_gather_cub_rows_b(const GatherArgs* __restrict__ args) {
    gather_row_impl(args[blockIdx.z], blockIdx.x);
}

void launch_gather_cub_rows(cudaStream_t s, const GatherArgs* d_args, const GatherArgs& host_args,
                            int n_sys) {
    if (host_args.n_rows <= 0) return;
    if (d_args)
        k_gather_cub_rows_b<<<dim3(host_args.n_rows, 1, n_sys), 128, 0, s>>>(d_args);
    else
        k_gather_cub_rows<<<host_args.n_rows, 128, 0, s>>>(host_args);
}

}  // namespace dae
